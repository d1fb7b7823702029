// Adjoint of log|psi| with respect to the parameters (reverse mode over the
// value pass), used for the VMC energy gradient of Eq. 2.
//
// Seeds c_w scale each walker's cotangent.  Through the determinant sum
// (Eq. 3) d log|psi| / d l_k = psi_k / psi; through each slogdet
// d log|det A| / d A_ij = (A^-1)_ji (the stored inverse); through A = o * e
// the cotangent splits onto the orbital GEMM output o and the envelope e
// (Eq. 4).  The dense-layer cotangents then flow through plain GEMMs
// (k_gemm.cu) and the small elementwise kernels below.
#include <math.h>

#include "fn_internal.cuh"

namespace fn {
namespace {

__device__ __forceinline__ int geo_of(const Geo& g, long wg) { return g.geo ? g.geo[wg] : 0; }

// One block per (walker, determinant, spin) matrix.
__global__ void __launch_bounds__(128) k_adj_det(AdjDetArgs a) {
  __shared__ float Eb[32 * 32];
  const long mat = blockIdx.x;
  const long w = mat / (2 * a.K);
  const int r = (int)(mat % (2 * a.K));
  const int k = r / 2, s = r % 2;
  const int ns = s == 0 ? a.n_up : a.n - a.n_up;
  if (ns == 0) return;
  const int j0 = s == 0 ? 0 : a.n_up;
  const long Ktot = (long)a.K * a.n;
  const long q0 = (s == 0 ? 0L : (long)a.K * a.n_up) + (long)k * ns;
  const float lbar = a.seeds[w] * a.wdet[w * a.K + k];
  const long NSS = (long)a.NS * a.NS;
  const float* M = a.minv + mat * NSS;
  const float* E = a.env + mat * NSS;
  for (int t = threadIdx.x; t < ns * ns; t += blockDim.x) {
    const int i = t / ns, j = t % ns;
    const long slot = (w * a.n + j0 + j) * Ktot + q0 + i;
    const float Abar = lbar * M[j * ns + i];
    a.Obar[slot] = Abar * E[i * ns + j];
    Eb[i * ns + j] = Abar * a.O[slot];
  }
  __syncthreads();
  const float* R = a.g.R + (long)geo_of(a.g, a.w0 + w) * a.N * 3;
  const long KnN = (long)a.K * a.n * a.N;
  const long pioff = s == 0 ? 0L : (long)a.K * a.n_up * a.N;
  const int sz = a.full_env ? 9 : 1;
  float* eg_w = a.envgrad + w * (1 + sz) * KnN;
  for (int t = threadIdx.x; t < ns * a.N; t += blockDim.x) {
    const int i = t / a.N, m = t % a.N;
    const long pm = ((long)k * ns + i) * a.N + m;
    const float pv = a.pi[s][pm];
    if (a.full_env) {
      // d exp(-rho) / d Sigma_ab = -exp(-rho) v_a d_b / rho, v = Sigma d
      const float* S = a.sigma[s] + pm * 9;
      float gp = 0.f, gS[9];
#pragma unroll
      for (int q = 0; q < 9; ++q) gS[q] = 0.f;
      for (int j = 0; j < ns; ++j) {
        const float* xj = a.x + (w * a.n + j0 + j) * 3;
        const float d[3] = {xj[0] - R[3 * m], xj[1] - R[3 * m + 1], xj[2] - R[3 * m + 2]};
        float v[3];
#pragma unroll
        for (int q = 0; q < 3; ++q) v[q] = S[3 * q] * d[0] + S[3 * q + 1] * d[1] + S[3 * q + 2] * d[2];
        const float rho = sqrtf(v[0] * v[0] + v[1] * v[1] + v[2] * v[2]);
        const float ex = expf(-rho);
        const float eb = Eb[i * ns + j];
        gp = fmaf(eb, ex, gp);
        const float c = rho > 0.f ? -eb * pv * ex / rho : 0.f;
#pragma unroll
        for (int q = 0; q < 3; ++q)
#pragma unroll
          for (int b = 0; b < 3; ++b) gS[3 * q + b] = fmaf(c * v[q], d[b], gS[3 * q + b]);
      }
      eg_w[pioff + pm] = gp;
#pragma unroll
      for (int q = 0; q < 9; ++q) eg_w[KnN + (pioff + pm) * 9 + q] = gS[q];
    } else {
      const float sg = a.sigma[s][pm];
      const float as = fabsf(sg), sgn = sg > 0.f ? 1.f : (sg < 0.f ? -1.f : 0.f);
      float gp = 0.f, gs = 0.f;
      for (int j = 0; j < ns; ++j) {
        const float* xj = a.x + (w * a.n + j0 + j) * 3;
        float d0 = xj[0] - R[3 * m], d1 = xj[1] - R[3 * m + 1], d2 = xj[2] - R[3 * m + 2];
        float rr = sqrtf(d0 * d0 + d1 * d1 + d2 * d2);
        float ex = expf(-as * rr);
        float eb = Eb[i * ns + j];
        gp = fmaf(eb, ex, gp);
        gs = fmaf(eb * pv * ex, -rr * sgn, gs);
      }
      eg_w[pioff + pm] = gp;
      eg_w[KnN + pioff + pm] = gs;
    }
  }
}

__global__ void k_colsum_part(const float* __restrict__ X, long rows, long cols, long ldx, long rpc,
                              double* __restrict__ part) {
  __shared__ double sh[8][33];
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
  const long c = (long)blockIdx.x * 32 + tx;
  const long r0 = (long)blockIdx.y * rpc;
  const long r1 = min(rows, r0 + rpc);
  // FP32 over this thread's rows (a few hundred) in eight interleaved partial
  // sums (eight loads in flight), FP64 from here on
  float s = 0.f;
  if (c < cols) {
    float p[8] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
    long r = r0 + ty;
    for (; r + 56 < r1; r += 64) {
#pragma unroll
      for (int u = 0; u < 8; ++u) p[u] += X[(r + 8 * u) * ldx + c];
    }
    for (; r < r1; r += 8) p[0] += X[r * ldx + c];
    s = ((p[0] + p[1]) + (p[2] + p[3])) + ((p[4] + p[5]) + (p[6] + p[7]));
  }
  sh[ty][tx] = (double)s;
  __syncthreads();
  if (ty == 0 && c < cols) {
    double t = 0.0;
#pragma unroll
    for (int q = 0; q < 8; ++q) t += sh[q][tx];
    part[(long)blockIdx.y * cols + c] = t;
  }
}

__global__ void k_colsum_final(const double* __restrict__ part, long nch, long cols, double* grad) {
  long c = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= cols) return;
  double s = 0.0;
#pragma unroll 8  // loads ahead of the (unchanged) summation order
  for (long q = 0; q < nch; ++q) s += part[q * cols + c];
  grad[c] += s;
}

__global__ void k_tanh_bwd(const float* __restrict__ hbar, const float* __restrict__ Y, long tot,
                           float* __restrict__ zbar) {
  long i = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= tot) return;
  float y = Y[i];
  zbar[i] = hbar[i] * (1.f - y * y);
}

__global__ void k_walker_sum(const float* __restrict__ X, long Bc, int n, int d, float* __restrict__ S) {
  long idx = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= Bc * d) return;
  long w = idx / d;
  int f = (int)(idx % d);
  float s = 0.f;
  for (int i = 0; i < n; ++i) s += X[(w * n + i) * d + f];
  S[idx] = s;
}

__global__ void k_spread_mean1(const float* __restrict__ m1bar, long Bc, int n, int n_up, int din,
                               float* __restrict__ hbar) {
  long idx = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= Bc * n * din) return;
  int f = (int)(idx % din);
  long wi = idx / din;
  int i = (int)(wi % n);
  long w = wi / n;
  int s = i < n_up ? 0 : 1;
  int ns = s == 0 ? n_up : n - n_up;
  hbar[idx] += m1bar[w * 2 * din + s * din + f] / (float)ns;
}

__global__ void k_spread_mean2(const float* __restrict__ m2bar, long Bc, int n, int n_up, int din2,
                               float* __restrict__ ebar) {
  long idx = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= Bc * n * n * din2) return;
  int f = (int)(idx % din2);
  long p = idx / din2;
  int j = (int)(p % n);
  long wi = p / n;
  int s = j < n_up ? 0 : 1;
  int ns = s == 0 ? n_up : n - n_up;
  ebar[idx] += m2bar[wi * 2 * din2 + s * din2 + f] / (float)ns;
}

// Four elements per thread (16-byte loads and stores) for the elementwise
// kernels below when the sizes and pointers allow it.
__global__ void k_tanh_bwd4(const float4* __restrict__ hbar, const float4* __restrict__ Y, long tot4,
                            float4* __restrict__ zbar) {
  const long i = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= tot4) return;
  const float4 y = Y[i], h = hbar[i];
  zbar[i] = make_float4(h.x * (1.f - y.x * y.x), h.y * (1.f - y.y * y.y), h.z * (1.f - y.z * y.z),
                        h.w * (1.f - y.w * y.w));
}

__global__ void k_spread_mean1_4(const float* __restrict__ m1bar, long Bc, int n, int n_up, int din,
                                 float* __restrict__ hbar) {
  const long idx = (long)blockIdx.x * blockDim.x + threadIdx.x;
  const int d4 = din >> 2;
  if (idx >= Bc * n * d4) return;
  const int f = (int)(idx % d4) * 4;
  const long wi = idx / d4;
  const int i = (int)(wi % n);
  const long w = wi / n;
  const int s = i < n_up ? 0 : 1;
  const float ns = (float)(s == 0 ? n_up : n - n_up);
  const float4 m = *reinterpret_cast<const float4*>(m1bar + w * 2 * din + s * din + f);
  float4* h = reinterpret_cast<float4*>(hbar + wi * din + f);
  float4 v = *h;
  v.x += m.x / ns;
  v.y += m.y / ns;
  v.z += m.z / ns;
  v.w += m.w / ns;
  *h = v;
}

__global__ void k_add4(float4* __restrict__ dst, const float4* __restrict__ src, long n4) {
  const long i = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n4) return;
  const float4 a = dst[i], b = src[i];
  dst[i] = make_float4(a.x + b.x, a.y + b.y, a.z + b.z, a.w + b.w);
}

__global__ void k_add(float* __restrict__ dst, const float* __restrict__ src, long n) {
  long i = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) dst[i] += src[i];
}

inline unsigned nblk(long tot, int bs) { return (unsigned)((tot + bs - 1) / bs); }

}  // namespace

void launch_adj_det(cudaStream_t s, const AdjDetArgs& a) {
  long nmat = a.Bc * a.K * 2;
  if (nmat > 0) FN_COUNT(1), k_adj_det<<<(unsigned)nmat, 128, 0, s>>>(a);
}

long colsum_scratch_elems(long rows, long cols) {
  long cb = (cols + 31) / 32;
  long nch = (rows + 255) / 256;
  long cap = (4 * 152 + cb - 1) / cb;
  if (nch > cap) nch = cap;
  if (nch < 1) nch = 1;
  return nch * cols;
}

void launch_colsum_accum(cudaStream_t s, const float* X, long rows, long cols, long ldx, double* grad,
                         double* scratch) {
  if (rows <= 0 || cols <= 0) return;
  long cb = (cols + 31) / 32;
  long nch = colsum_scratch_elems(rows, cols) / cols;
  long rpc = (rows + nch - 1) / nch;
  dim3 grid((unsigned)cb, (unsigned)nch);
  FN_COUNT(1), k_colsum_part<<<grid, 256, 0, s>>>(X, rows, cols, ldx, rpc, scratch);
  FN_COUNT(1), k_colsum_final<<<nblk(cols, 256), 256, 0, s>>>(scratch, nch, cols, grad);
}

void launch_tanh_bwd(cudaStream_t s, const float* hbar, const float* Y, long rows, int d, float* zbar) {
  long tot = rows * d;
  if (tot <= 0) return;
  if (tot % 4 == 0 && ((uintptr_t)hbar | (uintptr_t)Y | (uintptr_t)zbar) % 16 == 0) {
    FN_COUNT(1), k_tanh_bwd4<<<nblk(tot / 4, 256), 256, 0, s>>>(reinterpret_cast<const float4*>(hbar),
                                                               reinterpret_cast<const float4*>(Y), tot / 4,
                                                               reinterpret_cast<float4*>(zbar));
    return;
  }
  FN_COUNT(1), k_tanh_bwd<<<nblk(tot, 256), 256, 0, s>>>(hbar, Y, tot, zbar);
}

void launch_walker_sum(cudaStream_t s, const float* X, long Bc, int n, int d, float* S) {
  long tot = Bc * d;
  if (tot > 0) FN_COUNT(1), k_walker_sum<<<nblk(tot, 256), 256, 0, s>>>(X, Bc, n, d, S);
}

void launch_spread_mean1(cudaStream_t s, const float* m1bar, long Bc, int n, int n_up, int din, float* hbar) {
  long tot = Bc * n * din;
  if (tot <= 0) return;
  if (din % 4 == 0 && ((uintptr_t)m1bar | (uintptr_t)hbar) % 16 == 0) {
    FN_COUNT(1), k_spread_mean1_4<<<nblk(tot / 4, 256), 256, 0, s>>>(m1bar, Bc, n, n_up, din, hbar);
    return;
  }
  FN_COUNT(1), k_spread_mean1<<<nblk(tot, 256), 256, 0, s>>>(m1bar, Bc, n, n_up, din, hbar);
}

void launch_spread_mean2(cudaStream_t s, const float* m2bar, long Bc, int n, int n_up, int din2, float* ebar) {
  long tot = Bc * n * n * din2;
  if (tot > 0) FN_COUNT(1), k_spread_mean2<<<nblk(tot, 256), 256, 0, s>>>(m2bar, Bc, n, n_up, din2, ebar);
}

void launch_add(cudaStream_t s, float* dst, const float* src, long n) {
  if (n <= 0) return;
  if (n % 4 == 0 && ((uintptr_t)dst | (uintptr_t)src) % 16 == 0) {
    FN_COUNT(1), k_add4<<<nblk(n / 4, 256), 256, 0, s>>>(reinterpret_cast<float4*>(dst),
                                                        reinterpret_cast<const float4*>(src), n / 4);
    return;
  }
  FN_COUNT(1), k_add<<<nblk(n, 256), 256, 0, s>>>(dst, src, n);
}

}  // namespace fn
