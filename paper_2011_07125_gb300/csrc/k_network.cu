// Streaming kernels of the permutation-equivariant network: input features,
// spin-averaged means, the forward-Laplacian tanh step of the one-electron
// stream and the fused two-electron layer.
//
// Forward-Laplacian propagation (Sec. 3 computes the kinetic energy with
// forward-mode derivatives): every activation carries, besides its value, its
// derivative along each of the 3n electron coordinates and its Laplacian.  A
// linear map acts on all columns alike (the bias only on the value); for
// y = tanh(z):  dy = (1 - y^2) dz,  lap y = (1 - y^2) lap z - 2 y (1 - y^2) |dz|^2.
#include "fn_internal.cuh"

namespace fn {
namespace {

__device__ __forceinline__ int geo_of(const Geo& g, long wg) { return g.geo ? g.geo[wg] : 0; }

// h^0_i = [r_i - R_I, |r_i - R_I|]_I, one thread per (walker, electron, column).
__global__ void k_feat1(const float* __restrict__ x, long Bc, long w0, int n, int N, int C, Geo g,
                        float* __restrict__ H0) {
  long idx = (long)blockIdx.x * blockDim.x + threadIdx.x;
  long tot = Bc * n * C;
  if (idx >= tot) return;
  int c = (int)(idx % C);
  long wi = idx / C;
  int i = (int)(wi % n);
  long w = wi / n;
  const float* R = g.R + (long)geo_of(g, w0 + w) * N * 3;
  const float* xi = x + (w * n + i) * 3;
  float* out = H0 + idx * 4 * N;
  const int n3 = 3 * n;
  for (int I = 0; I < N; ++I) {
    float d0 = xi[0] - R[3 * I], d1 = xi[1] - R[3 * I + 1], d2 = xi[2] - R[3 * I + 2];
    float r = sqrtf(d0 * d0 + d1 * d1 + d2 * d2);
    float v[4] = {0.f, 0.f, 0.f, 0.f};
    if (c == 0) {
      v[0] = d0; v[1] = d1; v[2] = d2; v[3] = r;
    } else if (c <= n3) {
      int e = (c - 1) / 3, dd = (c - 1) % 3;
      if (e == i) {
        v[dd] = 1.f;
        float dv = dd == 0 ? d0 : (dd == 1 ? d1 : d2);
        v[3] = r > 0.f ? dv / r : 0.f;
      }
    } else if (c == n3 + 1) {
      v[3] = r > 0.f ? 2.f / r : 0.f;
    }
    *reinterpret_cast<float4*>(out + 4 * I) = make_float4(v[0], v[1], v[2], v[3]);
  }
}

// The same rows staged per warp in shared memory (32 rows of 4N floats,
// stride 4N + 4) and written out as contiguous 16-byte stores: a warp's rows
// are adjacent in H0, so its stores cover one contiguous range.
__global__ void __launch_bounds__(128) k_feat1_staged(const float* __restrict__ x, long Bc, long w0, int n, int N,
                                                      int C, Geo g, float* __restrict__ H0) {
  extern __shared__ __align__(16) float fsh[];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int RS = 4 * N + 4;
  float* wsh = fsh + warp * 32 * RS;
  const long tot = Bc * n * C;
  const long r0 = ((long)blockIdx.x * 4 + warp) * 32;
  if (r0 >= tot) return;  // warp-uniform
  const int nr = (int)min(32L, tot - r0);
  const long idx = r0 + lane;
  if (lane < nr) {
    const int c = (int)(idx % C);
    const long wi = idx / C;
    const int i = (int)(wi % n);
    const long w = wi / n;
    const float* R = g.R + (long)geo_of(g, w0 + w) * N * 3;
    const float* xi = x + (w * n + i) * 3;
    float* out = wsh + lane * RS;
    const int n3 = 3 * n;
    for (int I = 0; I < N; ++I) {
      float d0 = xi[0] - R[3 * I], d1 = xi[1] - R[3 * I + 1], d2 = xi[2] - R[3 * I + 2];
      float r = sqrtf(d0 * d0 + d1 * d1 + d2 * d2);
      float v[4] = {0.f, 0.f, 0.f, 0.f};
      if (c == 0) {
        v[0] = d0; v[1] = d1; v[2] = d2; v[3] = r;
      } else if (c <= n3) {
        int e = (c - 1) / 3, dd = (c - 1) % 3;
        if (e == i) {
          v[dd] = 1.f;
          float dv = dd == 0 ? d0 : (dd == 1 ? d1 : d2);
          v[3] = r > 0.f ? dv / r : 0.f;
        }
      } else if (c == n3 + 1) {
        v[3] = r > 0.f ? 2.f / r : 0.f;
      }
      *reinterpret_cast<float4*>(out + 4 * I) = make_float4(v[0], v[1], v[2], v[3]);
    }
  }
  __syncwarp();
  float4* dst = reinterpret_cast<float4*>(H0 + r0 * 4 * N);
  for (int k = lane; k < nr * N; k += 32) {
    const int row = k / N, I = k - row * N;
    dst[k] = *reinterpret_cast<const float4*>(wsh + row * RS + 4 * I);
  }
}

// h^0_ij = [r_i - r_j, |r_i - r_j|]; Q = 5 rows (value, d/dr_i xyz, full
// Laplacian = 2 * (2 / r) for the distance) or Q = 1.  Zero for i = j.
__global__ void k_feat2(const float* __restrict__ x, long Bc, int n, int Q, float* __restrict__ E0) {
  long idx = (long)blockIdx.x * blockDim.x + threadIdx.x;
  long tot = Bc * n * n;
  if (idx >= tot) return;
  int j = (int)(idx % n);
  long wi = idx / n;
  int i = (int)(wi % n);
  long w = wi / n;
  float* out = E0 + idx * Q * 4;
  if (i == j) {
    for (int q = 0; q < Q * 4; ++q) out[q] = 0.f;
    return;
  }
  const float* xi = x + (w * n + i) * 3;
  const float* xj = x + (w * n + j) * 3;
  float d[3] = {xi[0] - xj[0], xi[1] - xj[1], xi[2] - xj[2]};
  float r = sqrtf(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
  *reinterpret_cast<float4*>(out) = make_float4(d[0], d[1], d[2], r);
  if (Q == 1) return;
  float ir = r > 0.f ? 1.f / r : 0.f;
  for (int dd = 0; dd < 3; ++dd) {
    float v[4] = {0.f, 0.f, 0.f, d[dd] * ir};
    v[dd] = 1.f;
    *reinterpret_cast<float4*>(out + 4 * (1 + dd)) = make_float4(v[0], v[1], v[2], v[3]);
  }
  *reinterpret_cast<float4*>(out + 16) = make_float4(0.f, 0.f, 0.f, 4.f * ir);
}

// Dense-column spin means of the two-electron stream, one block per
// (walker, electron i): the pair rows h_ij (all j, all Q quantities) are staged
// in shared memory with the per-spin sums, then the C x ldb output block is
// written with 32-bit indexing.  Output as FP32 (out32) or BF16 hi / lo (lo may
// be null); columns 2 din2 .. ldb-1 are zero.  Column layout as in k_mean2.
template <int MAXN>
__global__ void __launch_bounds__(256) k_mean2_rows(const float* __restrict__ E, int n, int n_up, int Q, int din2,
                                                    int C, float* __restrict__ out32, __nv_bfloat16* __restrict__ hi,
                                                    __nv_bfloat16* __restrict__ lo, int ldb) {
  extern __shared__ float sh[];
  float* Es = sh;                              // [n][Q][din2]
  float* Ss = sh + n * Q * din2;               // [2][Q][din2] per-spin sums
  const long wi = blockIdx.x;
  const int i = (int)(wi % n);
  const int QD = Q * din2;
  const float* src = E + wi * (long)n * QD;
  for (int t = threadIdx.x; t < n * QD; t += blockDim.x) Es[t] = src[t];
  __syncthreads();
  for (int t = threadIdx.x; t < 2 * QD; t += blockDim.x) {
    const int s = t / QD, qf = t % QD;
    const int j0 = s == 0 ? 0 : n_up, j1 = s == 0 ? n_up : n;
    float a = 0.f;
    for (int j = j0; j < j1; ++j) a += Es[j * QD + qf];
    Ss[t] = a;
  }
  __syncthreads();
  const int n3 = 3 * n;
  const int tot = C * ldb;
  const long obase = wi * (long)tot;
  for (int t = threadIdx.x; t < tot; t += blockDim.x) {
    const int c = t / ldb, col = t % ldb;
    float v = 0.f;
    if (col < 2 * din2) {
      const int s = col / din2, f = col % din2;
      const int j0 = s == 0 ? 0 : n_up, j1 = s == 0 ? n_up : n;
      const int ns = j1 - j0;
      if (ns > 0) {
        const float inv = 1.f / (float)ns;
        if (c == 0) {
          v = Ss[s * QD + f] * inv;
        } else if (Q > 1 && c <= n3) {
          const int e = (c - 1) / 3, dd = (c - 1) % 3;
          if (e == i) v = Ss[s * QD + (1 + dd) * din2 + f] * inv;
          else if (e >= j0 && e < j1) v = -Es[e * QD + (1 + dd) * din2 + f] * inv;
        } else if (Q > 1 && c == n3 + 1) {
          v = Ss[s * QD + 4 * din2 + f] * inv;
        }
      }
    }
    if (out32) {
      out32[obase + t] = v;
    } else {
      const __nv_bfloat16 h = __float2bfloat16_rn(v);
      hi[obase + t] = h;
      if (lo) lo[obase + t] = __float2bfloat16_rn(v - __bfloat162float(h));
    }
  }
}

// Spin means of a one-electron activation, one block per (walker, column c):
// out[w][c][s*din + f] = mean over electrons i of spin s of H[w][i][c][f], H
// either FP32 (h32, row stride ldin) or BF16 hi + lo; output FP32 (out32,
// stride ldout) or BF16 hi / lo (stride ldout, padding zeroed).
__global__ void __launch_bounds__(256) k_mean1_rows(const float* __restrict__ h32,
                                                    const __nv_bfloat16* __restrict__ hhi,
                                                    const __nv_bfloat16* __restrict__ hlo, int ldin, int n, int n_up,
                                                    int C, int din, float* __restrict__ out32,
                                                    __nv_bfloat16* __restrict__ ohi, __nv_bfloat16* __restrict__ olo,
                                                    int ldout) {
  const long wc = blockIdx.x;
  const long w = wc / C;
  const int c = (int)(wc % C);
  const long rowc = (w * n) * (long)C + c;  // row of electron 0, column c
  const long ob = wc * (long)ldout;
  for (int col = threadIdx.x; col < ldout; col += blockDim.x) {
    float v = 0.f;
    if (col < 2 * din) {
      const int s = col / din, f = col % din;
      const int i0 = s == 0 ? 0 : n_up, i1 = s == 0 ? n_up : n;
      float a = 0.f;
      for (int i = i0; i < i1; ++i) {
        const long r = (rowc + (long)i * C) * ldin + f;
        a += h32 ? h32[r] : __bfloat162float(hhi[r]) + (hlo ? __bfloat162float(hlo[r]) : 0.f);
      }
      v = i1 > i0 ? a / (float)(i1 - i0) : 0.f;
    }
    if (out32) {
      out32[ob + col] = v;
    } else {
      const __nv_bfloat16 h = __float2bfloat16_rn(v);
      ohi[ob + col] = h;
      if (olo) olo[ob + col] = __float2bfloat16_rn(v - __bfloat162float(h));
    }
  }
}

// Same spin means with 16-byte accesses: one thread per 8 output columns of a
// (walker, column c) row, loading 8 features of every electron of its spin
// (all loads independent).  din and the row strides are multiples of 8; the
// sum runs over i in order and is divided by the count, as k_mean1_rows.
template <bool BF>
__global__ void __launch_bounds__(256) k_mean1_vec(const float* __restrict__ h32,
                                                   const __nv_bfloat16* __restrict__ hhi,
                                                   const __nv_bfloat16* __restrict__ hlo, int ldin, long rows,
                                                   int n, int n_up, int C, int din, float* __restrict__ out32,
                                                   __nv_bfloat16* __restrict__ ohi, __nv_bfloat16* __restrict__ olo,
                                                   int ldout) {
  const int cpr = ldout / 8;
  const long t = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= rows * cpr) return;
  const long wc = t / cpr;
  const int col0 = (int)(t - wc * cpr) * 8;
  const long w = wc / C;
  const int c = (int)(wc - w * C);
  float v[8] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
  if (col0 < 2 * din) {
    const int s = col0 / din, f0 = col0 - s * din;
    const int i0 = s == 0 ? 0 : n_up, i1 = s == 0 ? n_up : n;
    float a[8] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
#pragma unroll 5
    for (int i = i0; i < i1; ++i) {
      const long r = ((w * n + i) * (long)C + c) * ldin + f0;
      if (BF) {
        const uint4 hv = *reinterpret_cast<const uint4*>(hhi + r);
        const uint4 lv = hlo ? *reinterpret_cast<const uint4*>(hlo + r) : make_uint4(0u, 0u, 0u, 0u);
        const __nv_bfloat16* hb = reinterpret_cast<const __nv_bfloat16*>(&hv);
        const __nv_bfloat16* lb = reinterpret_cast<const __nv_bfloat16*>(&lv);
#pragma unroll
        for (int j = 0; j < 8; ++j) a[j] += __bfloat162float(hb[j]) + __bfloat162float(lb[j]);
      } else {
        const float4 x0 = *reinterpret_cast<const float4*>(h32 + r);
        const float4 x1 = *reinterpret_cast<const float4*>(h32 + r + 4);
        a[0] += x0.x; a[1] += x0.y; a[2] += x0.z; a[3] += x0.w;
        a[4] += x1.x; a[5] += x1.y; a[6] += x1.z; a[7] += x1.w;
      }
    }
    if (i1 > i0) {
#pragma unroll
      for (int j = 0; j < 8; ++j) v[j] = a[j] / (float)(i1 - i0);
    }
  }
  const long ob = wc * ldout + col0;
  if (out32) {
    *reinterpret_cast<float4*>(out32 + ob) = make_float4(v[0], v[1], v[2], v[3]);
    *reinterpret_cast<float4*>(out32 + ob + 4) = make_float4(v[4], v[5], v[6], v[7]);
  } else {
    __align__(16) __nv_bfloat16 hi[8], lo[8];
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      hi[j] = __float2bfloat16_rn(v[j]);
      lo[j] = __float2bfloat16_rn(v[j] - __bfloat162float(hi[j]));
    }
    *reinterpret_cast<uint4*>(ohi + ob) = *reinterpret_cast<const uint4*>(hi);
    if (olo) *reinterpret_cast<uint4*>(olo + ob) = *reinterpret_cast<const uint4*>(lo);
  }
}

__global__ void k_split_bf16(const float* __restrict__ src, long src_ld, long rows, long cols,
                             __nv_bfloat16* __restrict__ hi, __nv_bfloat16* __restrict__ lo, long dst_ld) {
  long idx = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= rows * dst_ld) return;
  const long r = idx / dst_ld, c = idx % dst_ld;
  const float v = c < cols ? src[r * src_ld + c] : 0.f;
  const __nv_bfloat16 h = __float2bfloat16_rn(v);
  hi[idx] = h;
  if (lo) lo[idx] = __float2bfloat16_rn(v - __bfloat162float(h));
}

// The same split, 8 destination columns per thread (16-byte stores of hi and
// lo; dst_ld a multiple of 8 and both outputs 16-byte aligned).
__global__ void k_split_bf16_v8(const float* __restrict__ src, long src_ld, long rows, long cols,
                                __nv_bfloat16* __restrict__ hi, __nv_bfloat16* __restrict__ lo, long dst_ld,
                                int src_vec) {
  const long cpr = dst_ld >> 3;
  const long t = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= rows * cpr) return;
  const long r = t / cpr, c0 = (t - r * cpr) * 8;
  const float* sp = src + r * src_ld + c0;
  float v[8];
  if (src_vec && c0 + 8 <= cols) {
    const float4 a = reinterpret_cast<const float4*>(sp)[0];
    const float4 b = reinterpret_cast<const float4*>(sp)[1];
    v[0] = a.x; v[1] = a.y; v[2] = a.z; v[3] = a.w;
    v[4] = b.x; v[5] = b.y; v[6] = b.z; v[7] = b.w;
  } else {
#pragma unroll
    for (int j = 0; j < 8; ++j) v[j] = c0 + j < cols ? sp[j] : 0.f;
  }
  __align__(16) __nv_bfloat16 h[8], l[8];
#pragma unroll
  for (int j = 0; j < 8; ++j) {
    h[j] = __float2bfloat16_rn(v[j]);
    l[j] = __float2bfloat16_rn(v[j] - __bfloat162float(h[j]));
  }
  const long o = r * dst_ld + c0;
  *reinterpret_cast<uint4*>(hi + o) = *reinterpret_cast<const uint4*>(h);
  if (lo) *reinterpret_cast<uint4*>(lo + o) = *reinterpret_cast<const uint4*>(l);
}

// One-electron tanh with forward-Laplacian columns, plus residual.
__global__ void k_tanh_fl(const float* __restrict__ Z, const float* __restrict__ Hres, long Bc, int n, int C,
                          int d1, float* __restrict__ Hout, float* __restrict__ Y) {
  long idx = (long)blockIdx.x * blockDim.x + threadIdx.x;
  long tot = Bc * n * d1;
  if (idx >= tot) return;
  int f = (int)(idx % d1);
  long wi = idx / d1;
  const long base = wi * C * d1 + f;
  float z0 = Z[base];
  float y = tanhf(z0);
  float s = 1.f - y * y;
  if (Y) Y[idx] = y;
  Hout[base] = y + (Hres ? Hres[base] : 0.f);
  if (C == 1) return;
  const int n3 = 3 * n;
  float sq = 0.f;
  for (int c = 1; c <= n3; ++c) {
    float zc = Z[base + (long)c * d1];
    sq = fmaf(zc, zc, sq);
    Hout[base + (long)c * d1] = s * zc + (Hres ? Hres[base + (long)c * d1] : 0.f);
  }
  float zl = Z[base + (long)(n3 + 1) * d1];
  Hout[base + (long)(n3 + 1) * d1] = s * zl - 2.f * y * s * sq + (Hres ? Hres[base + (long)(n3 + 1) * d1] : 0.f);
  for (int c = n3 + 2; c < C; ++c) Hout[base + (long)c * d1] = 0.f;
}

// Two-electron layer h_ij -> tanh(W h_ij + c) (+ h_ij).  One warp per pair at
// a time (grid-stride over pairs), lane f = output feature, its row of W held
// in registers; the pair's Q x DIN input rows are staged in shared memory and
// read as broadcasts.  The Laplacian rule uses |dz|^2 = 2 |dz/dr_i|^2 because
// dz/dr_j = -dz/dr_i.
template <int DIN>
__device__ __forceinline__ void two_layer_pair(const float (&wr)[DIN], float bias, const float* sh, long p, int Q,
                                               int d2, int f, int residual, float* __restrict__ Eout,
                                               float* __restrict__ Y2) {
  float z[kQ] = {0.f, 0.f, 0.f, 0.f, 0.f};
#pragma unroll
  for (int k = 0; k < DIN; ++k) {
    z[0] = fmaf(wr[k], sh[k], z[0]);
    if (Q > 1) {
#pragma unroll
      for (int q = 1; q < kQ; ++q) z[q] = fmaf(wr[k], sh[q * DIN + k], z[q]);
    }
  }
  if (f >= d2) return;
  z[0] += bias;
  const float y = tanhf(z[0]);
  const float s = 1.f - y * y;
  if (Y2) Y2[p * d2 + f] = y;
  float* out = Eout + p * Q * d2;
  out[f] = y + (residual ? sh[f] : 0.f);
  if (Q > 1) {
    const float sq = z[1] * z[1] + z[2] * z[2] + z[3] * z[3];
#pragma unroll
    for (int q = 1; q <= 3; ++q) out[q * d2 + f] = s * z[q] + (residual ? sh[q * DIN + f] : 0.f);
    out[4 * d2 + f] = s * z[4] - 4.f * y * s * sq + (residual ? sh[4 * DIN + f] : 0.f);
  }
}

// Two-electron layer h_ij -> tanh(W h_ij + c) (+ h_ij).  One warp handles two
// pairs per iteration (grid-stride over pairs), lane f = output feature, its row
// of W held in registers; the pairs' Q x DIN input rows are staged in shared
// memory and read as broadcasts.  The Laplacian rule uses |dz|^2 = 2 |dz/dr_i|^2
// because dz/dr_j = -dz/dr_i.
template <int DIN>
__global__ void __launch_bounds__(256) k_two_layer(const float* __restrict__ Ein, long pairs, int Q, int din2,
                                                   int d2, const float* __restrict__ W,
                                                   const float* __restrict__ cb, int residual,
                                                   float* __restrict__ Eout, float* __restrict__ Y2) {
  __shared__ __align__(16) float in_s[8][2][kQ * DIN];
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  const int f = lane;
  float wr[DIN];
#pragma unroll
  for (int k = 0; k < DIN; ++k) wr[k] = (f < d2 && k < din2) ? W[(long)f * din2 + k] : 0.f;
  const float bias = f < d2 ? cb[f] : 0.f;
  const long nwarps = (long)gridDim.x * 8;
  const int QD = Q * DIN;
  for (long p0 = (long)blockIdx.x * 8 + wib; p0 < pairs; p0 += 2 * nwarps) {
    const long p1 = p0 + nwarps;
    const bool has1 = p1 < pairs;
    const float* in0 = Ein + p0 * Q * din2;
    const float* in1 = Ein + p1 * Q * din2;
    for (int t = lane; t < QD; t += 32) {
      const int q = t / DIN, k = t % DIN;
      in_s[wib][0][t] = k < din2 ? in0[q * din2 + k] : 0.f;
      in_s[wib][1][t] = (has1 && k < din2) ? in1[q * din2 + k] : 0.f;
    }
    __syncwarp();
    two_layer_pair<DIN>(wr, bias, in_s[wib][0], p0, Q, d2, f, residual, Eout, Y2);
    if (has1) two_layer_pair<DIN>(wr, bias, in_s[wib][1], p1, Q, d2, f, residual, Eout, Y2);
    __syncwarp();
  }
}

inline unsigned nblk(long tot, int bs) { return (unsigned)((tot + bs - 1) / bs); }

}  // namespace

void launch_features(cudaStream_t s, const float* x, long Bc, long w0, int n, int N, int C, int Q, Geo g, float* H0,
                     float* E0) {
  long t1 = Bc * n * C;
  const size_t fsm = sizeof(float) * 4 * 32 * (4 * N + 4);
  if (t1 > 0 && fsm <= 48 * 1024 && (uintptr_t)H0 % 16 == 0)
    FN_COUNT(1), k_feat1_staged<<<(unsigned)((t1 + 127) / 128), 128, fsm, s>>>(x, Bc, w0, n, N, C, g, H0);
  else if (t1 > 0)
    FN_COUNT(1), k_feat1<<<nblk(t1, 256), 256, 0, s>>>(x, Bc, w0, n, N, C, g, H0);
  long t2 = Bc * n * n;
  if (t2 > 0) FN_COUNT(1), k_feat2<<<nblk(t2, 256), 256, 0, s>>>(x, Bc, n, Q, E0);
}

void launch_mean1(cudaStream_t s, const float* H, long Bc, int n, int n_up, int C, int din, float* M1) {
  if (Bc * C <= 0) return;
  if (din % 8 == 0) {
    const long tot = Bc * C * (2L * din / 8);
    FN_COUNT(1), k_mean1_vec<false><<<nblk(tot, 256), 256, 0, s>>>(H, nullptr, nullptr, din, Bc * C, n, n_up, C, din,
                                                                   M1, nullptr, nullptr, 2 * din);
    return;
  }
  FN_COUNT(1), k_mean1_rows<<<(unsigned)(Bc * C), 256, 0, s>>>(H, nullptr, nullptr, din, n, n_up, C, din, M1, nullptr,
                                                               nullptr, 2 * din);
}

void launch_mean2(cudaStream_t s, const float* E, long Bc, int n, int n_up, int Q, int din2, int C, float* M2) {
  if (Bc * n <= 0) return;
  const size_t smem = sizeof(float) * ((size_t)(n + 2) * Q * din2);
  const int bs = C * 2 * din2 >= 1024 ? 256 : 64;
  FN_COUNT(1), k_mean2_rows<64><<<(unsigned)(Bc * n), bs, smem, s>>>(E, n, n_up, Q, din2, C, M2, nullptr, nullptr,
                                                                     2 * din2);
}

void launch_mean2_bf16(cudaStream_t s, const float* E, long Bc, int n, int n_up, int Q, int din2, int C,
                       __nv_bfloat16* hi, __nv_bfloat16* lo, long ldb) {
  if (Bc * n <= 0) return;
  const size_t smem = sizeof(float) * ((size_t)(n + 2) * Q * din2);
  const int bs = C * ldb >= 1024 ? 256 : 64;
  FN_COUNT(1), k_mean2_rows<64><<<(unsigned)(Bc * n), bs, smem, s>>>(E, n, n_up, Q, din2, C, nullptr, hi, lo, (int)ldb);
}

void launch_mean1_bf16(cudaStream_t s, const __nv_bfloat16* hi, const __nv_bfloat16* lo, long ldin, long Bc, int n,
                       int n_up, int C, int din, __nv_bfloat16* ohi, __nv_bfloat16* olo, long ldout) {
  if (Bc * C <= 0) return;
  if (din % 8 == 0 && ldin % 8 == 0 && ldout % 8 == 0) {
    const long tot = Bc * C * (ldout / 8);
    FN_COUNT(1), k_mean1_vec<true><<<nblk(tot, 256), 256, 0, s>>>(nullptr, hi, lo, (int)ldin, Bc * C, n, n_up, C, din,
                                                                  nullptr, ohi, olo, (int)ldout);
    return;
  }
  FN_COUNT(1), k_mean1_rows<<<(unsigned)(Bc * C), 256, 0, s>>>(nullptr, hi, lo, (int)ldin, n, n_up, C, din, nullptr, ohi,
                                                               olo, (int)ldout);
}

void launch_split_bf16(cudaStream_t s, const float* src, long src_ld, long rows, long cols, __nv_bfloat16* hi,
                       __nv_bfloat16* lo, long dst_ld) {
  long tot = rows * dst_ld;
  if (tot <= 0) return;
  if (dst_ld % 8 == 0 && ((uintptr_t)hi | (uintptr_t)lo) % 16 == 0) {
    const int src_vec = (src_ld % 4 == 0 && (uintptr_t)src % 16 == 0) ? 1 : 0;
    FN_COUNT(1), k_split_bf16_v8<<<nblk(tot / 8, 256), 256, 0, s>>>(src, src_ld, rows, cols, hi, lo, dst_ld, src_vec);
    return;
  }
  FN_COUNT(1), k_split_bf16<<<nblk(tot, 256), 256, 0, s>>>(src, src_ld, rows, cols, hi, lo, dst_ld);
}

void launch_tanh_fl(cudaStream_t s, const float* Z, const float* Hres, long Bc, int n, int C, int d1, float* Hout,
                    float* Y) {
  long tot = Bc * n * d1;
  if (tot > 0) FN_COUNT(1), k_tanh_fl<<<nblk(tot, 256), 256, 0, s>>>(Z, Hres, Bc, n, C, d1, Hout, Y);
}

void launch_two_layer(cudaStream_t s, const float* Ein, long Bc, int n, int Q, int din2, int d2, const float* W,
                      const float* c, bool residual, float* Eout, float* Y2) {
  const long pairs = Bc * n * n;
  if (pairs <= 0) return;
  long blocks = (pairs + 7) / 8;
  if (blocks > 152 * 8) blocks = 152 * 8;
  const int r = residual ? 1 : 0;
  if (din2 <= 4)
    FN_COUNT(1), k_two_layer<4><<<(unsigned)blocks, 256, 0, s>>>(Ein, pairs, Q, din2, d2, W, c, r, Eout, Y2);
  else if (din2 <= 8)
    FN_COUNT(1), k_two_layer<8><<<(unsigned)blocks, 256, 0, s>>>(Ein, pairs, Q, din2, d2, W, c, r, Eout, Y2);
  else if (din2 <= 16)
    FN_COUNT(1), k_two_layer<16><<<(unsigned)blocks, 256, 0, s>>>(Ein, pairs, Q, din2, d2, W, c, r, Eout, Y2);
  else
    FN_COUNT(1), k_two_layer<32><<<(unsigned)blocks, 256, 0, s>>>(Ein, pairs, Q, din2, d2, W, c, r, Eout, Y2);
}

}  // namespace fn
