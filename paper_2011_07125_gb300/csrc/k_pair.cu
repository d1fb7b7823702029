// Fused two-electron layer and spin means of the two-electron stream.
//
// Layer l of the two-electron stream maps every pair row h_ij to
// tanh(W h_ij + c) (+ h_ij for l >= 1), carrying Q quantities per pair: the
// value, d/dr_i (x, y, z) and the Laplacian over all coordinates (d/dr_j is
// -d/dr_i because h_ij depends on r_i - r_j only, so |dz|^2 = 2 |dz/dr_i|^2).
// The one-electron update of the next layer needs, for every electron i, the
// mean of h_ij over the electrons j of each spin (the g_i of Eq. 3's network),
// laid out as dense tangent columns: column 0 the value, column 1 + 3e + d the
// derivative along coordinate d of electron e, column 3n + 1 the Laplacian.
//
// One pass does both.  A block stages the pair rows of whole (walker,
// electron i) groups in shared memory (cp.async), applies the layer with 8
// output features (4 when Q = 5) x Q quantities per thread (weights
// transposed in shared memory), writes the new rows where a later kernel reads them, then expands
// the per-spin sums of the new rows into the dense mean rows (FP32, or BF16
// hi + lo for the tensor-core GEMM).  Without weights the block only forms the
// means of its input (the input features h^0_ij).
#include <mutex>

#include "f32x2.cuh"
#include "fn_internal.cuh"

namespace fn {
namespace {

constexpr int kPairThreads = 256;
constexpr int kSmemPerSM = 227 * 1024;

__device__ __forceinline__ void cp_async16(void* smem, const void* gmem) {
  const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(sa), "l"(gmem));
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_group 0;\n" ::); }

__device__ __forceinline__ float comp(const float4& v, int k) {
  return k == 0 ? v.x : (k == 1 ? v.y : (k == 2 ? v.z : v.w));
}
__device__ __forceinline__ float4 scale4(const float4& v, float a) {
  return make_float4(v.x * a, v.y * a, v.z * a, v.w * a);
}

// Shared-memory pair strides (floats): Q rows of DIN (input) or DO (output)
// features, plus 4 so that neighbouring pairs fall on different banks.
template <int DIN, int Q>
constexpr int in_stride() { return Q * DIN + 4; }
template <int DO, int Q>
constexpr int out_stride() { return Q * DO + 4; }
// Rows per thread task: the Q quantities of one pair, or (value pass) four pairs.
template <int Q>
constexpr int task_rows() { return Q == 1 ? 4 : Q; }
// Resident blocks per SM the kernel is built for (registers and shared memory):
// three for every layer instance, the warp-MMA one included; LARGE: a layer of
// the local-energy pass whose one-group tile needs the shared-memory share of
// two blocks (many electrons).
template <int Q, bool LAYER, bool MMA = false, bool LARGE = false>
constexpr int min_blocks() { return LARGE ? 2 : (LAYER ? 3 : 4); }
// Features per layer task (see k_pair_layer).
template <int Q, bool LAYER, bool MMA = false>
constexpr int task_features() { return (LAYER && Q > 1 && !MMA) ? 4 : 8; }

// D += A B for one m16n8k16 BF16 tile (A row-major 16 x 16, B column-major
// 16 x 8), FP32 accumulation.
__device__ __forceinline__ void mma_bf16_16816(float (&d)[4], const uint32_t (&a)[4], uint32_t b0, uint32_t b1) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0, %1, %2, %3}, {%4, %5, %6, %7}, {%8, %9}, "
      "{%0, %1, %2, %3};"
      : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

// Two FP32 values as packed BF16 hi (x0 in the low half) and the packed
// BF16 remainders.
__device__ __forceinline__ void split_bf16x2(float x0, float x1, uint32_t& hi, uint32_t& lo) {
  const __nv_bfloat162 h = __floats2bfloat162_rn(x0, x1);
  const __nv_bfloat162 l = __floats2bfloat162_rn(x0 - __low2float(h), x1 - __high2float(h));
  hi = *reinterpret_cast<const uint32_t*>(&h);
  lo = *reinterpret_cast<const uint32_t*>(&l);
}

template <int DIN, int DO, int Q, bool LAYER>
size_t pair_smem_bytes(int n, int tg) {
  // layer: one input tile (refilled while the means of the previous tile are
  // written) + output tile + weights; means only: two input tiles
  const size_t in = (size_t)(LAYER ? 1 : 2) * tg * n * in_stride<DIN, Q>();
  const size_t out = LAYER ? (size_t)tg * n * out_stride<DO, Q>() : 0;
  const size_t w = LAYER ? (size_t)DIN * DO + DO : 0;
  const size_t sums = (size_t)tg * 2 * Q * DO;
  return sizeof(float) * (in + out + w + sums);
}

// Stages the pair rows of groups [g0, g0 + tge) (contiguous in global memory)
// into a padded shared tile with 16-byte cp.async copies.
template <int DIN, int Q>
__device__ __forceinline__ void load_tile(const float* Ein, long g0, int tge, int n, float* dst) {
  constexpr int IPS = in_stride<DIN, Q>();
  constexpr int V = Q * DIN / 4;  // float4 per pair
  const float4* src = reinterpret_cast<const float4*>(Ein + g0 * n * (long)(Q * DIN));
  const int np = tge * n;
  for (int t = threadIdx.x; t < np * V; t += kPairThreads) {
    const int p = t / V, r = t - p * V;
    cp_async16(dst + p * IPS + 4 * r, src + t);
  }
  cp_async_commit();
}

// Writes the dense mean rows of the tile's groups: 8 columns per thread and
// step, decided per column quad (a quad never straddles the two spins).
template <int Q, int ORS, int OPS>
__device__ __forceinline__ void dense_means(const PairArgs& a, long g0, int tge, const float* sout, const float* sS,
                                            float inv0, float inv1) {
  const int n = a.n, n3 = 3 * n;
  const int cpr = (int)(a.ldm / 8);
  const int per_group = a.C * cpr;
  for (int t = threadIdx.x; t < tge * per_group; t += kPairThreads) {
    const int gq = t / per_group, r = t - gq * per_group;
    const int c = r / cpr, col0 = (r - c * cpr) * 8;
    const long G = g0 + gq;
    const int i = (int)(G % n);
    // row kind: 0 value, 1 own coordinate (sum), 2 another electron's coordinate, 3 Laplacian, -1 zero
    int kind = -1, e = 0, q = 0;
    if (c == 0) {
      kind = 0;
    } else if (Q > 1 && c <= n3) {
      e = (c - 1) / 3;
      q = 1 + (c - 1) - 3 * e;
      kind = e == i ? 1 : 2;
    } else if (Q > 1 && c == n3 + 1) {
      kind = 3;
      q = 4;
    }
    const float* S = sS + gq * 2 * Q * ORS;
    float4 v[2];
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      v[h] = make_float4(0.f, 0.f, 0.f, 0.f);
      const int col = col0 + 4 * h;
      if (kind >= 0 && col < 2 * ORS) {
        const int s = col / ORS, f = col - s * ORS;
        const float inv = s == 0 ? inv0 : inv1;
        if (kind == 2) {
          if ((e < a.n_up ? 0 : 1) == s)
            v[h] = scale4(*reinterpret_cast<const float4*>(sout + (gq * n + e) * OPS + q * ORS + f), -inv);
        } else {
          v[h] = scale4(*reinterpret_cast<const float4*>(S + (s * Q + q) * ORS + f), inv);
        }
      }
    }
    const long ob = (G * a.C + c) * a.ldm + col0;
    if (a.m32) {
      *reinterpret_cast<float4*>(a.m32 + ob) = v[0];
      *reinterpret_cast<float4*>(a.m32 + ob + 4) = v[1];
    } else {
      const float x[8] = {v[0].x, v[0].y, v[0].z, v[0].w, v[1].x, v[1].y, v[1].z, v[1].w};
      __align__(16) __nv_bfloat16 hi[8], lo[8];
#pragma unroll
      for (int jj = 0; jj < 8; ++jj) {
        hi[jj] = __float2bfloat16_rn(x[jj]);
        lo[jj] = __float2bfloat16_rn(x[jj] - __bfloat162float(hi[jj]));
      }
      *reinterpret_cast<uint4*>(a.mhi + ob) = *reinterpret_cast<const uint4*>(hi);
      if (a.mlo) *reinterpret_cast<uint4*>(a.mlo + ob) = *reinterpret_cast<const uint4*>(lo);
    }
  }
}

// Per-spin sums of every quantity of the tile's groups (sequential over j).
template <int Q, int ORS, int OPS>
__device__ __forceinline__ void spin_sums(const PairArgs& a, int tge, const float* sout, float* sS) {
  const int n = a.n;
  for (int t = threadIdx.x; t < tge * 2 * Q * ORS; t += kPairThreads) {
    const int gq = t / (2 * Q * ORS), r = t - gq * (2 * Q * ORS);
    const int s = r / (Q * ORS), qf = r - s * (Q * ORS);
    const int j0 = s == 0 ? 0 : a.n_up, j1 = s == 0 ? a.n_up : n;
    float acc = 0.f;
    for (int j = j0; j < j1; ++j) acc += sout[(gq * n + j) * OPS + qf];
    sS[t] = acc;
  }
}

template <int DIN, int DO, int Q, bool LAYER, bool MMA, bool LARGE>
__global__ void __launch_bounds__(kPairThreads, min_blocks<Q, LAYER, MMA, LARGE>()) k_pair_layer(PairArgs a) {
  static_assert(DIN % 4 == 0 && (DO % 8 == 0 || !LAYER), "feature counts");
  static_assert(!MMA || (LAYER && DIN == 32 && DO == 32), "warp-MMA contraction: 32 -> 32 layers");
  constexpr int IPS = in_stride<DIN, Q>();
  constexpr int OPS = LAYER ? out_stride<DO, Q>() : IPS;
  constexpr int ORS = LAYER ? DO : DIN;  // row stride of one quantity in the output tile
  // features per layer task: 8, or 4 in the local-energy pass (Q = 5), whose
  // five accumulated quantities per feature would otherwise hold the kernel
  // to two blocks per SM
  constexpr int FW = task_features<Q, LAYER, MMA>();
  constexpr int FG = LAYER ? DO / FW : 1;
  static_assert(!MMA || FW == 8, "warp-MMA tasks cover 8 features");
  constexpr int R = task_rows<Q>();
  extern __shared__ __align__(16) float smem[];
  const int n = a.n, tg = a.tg, tid = threadIdx.x;
  // layer:      [tg n][IPS] input | [tg n][OPS] output | [DIN][DO] weights^T | [DO] bias | [tg][2][Q][DO] sums
  // means only: 2 x [tg n][IPS] input | [tg][2][Q][DIN] sums
  float* sin = smem;
  float* after_in = sin + (size_t)(LAYER ? 1 : 2) * tg * n * IPS;
  float* sout_l = after_in;
  float* sW = LAYER ? after_in + (size_t)tg * n * OPS : after_in;
  float* sb = sW + (LAYER ? DIN * DO : 0);
  float* sS = sb + (LAYER ? DO : 0);
  if (LAYER) {
    for (int t = tid; t < DIN * DO; t += kPairThreads) {
      const int k = t / DO, f = t % DO;
      sW[t] = a.W[f * DIN + k];
    }
    for (int t = tid; t < DO; t += kPairThreads) sb[t] = a.cb[t];
  }
  // warp-MMA contraction: W^T as the B operand (k = input feature, n = output
  // feature), fragments for two k-steps and four column tiles, split hi + lo
  const int lane = tid & 31, warp = tid >> 5, fgr = lane >> 2, fq = lane & 3;
  uint32_t wbh[MMA ? 2 : 1][MMA ? 4 : 1][2], wbl[MMA ? 2 : 1][MMA ? 4 : 1][2];
  if constexpr (MMA) {
    __syncthreads();  // sW is complete
#pragma unroll
    for (int ks = 0; ks < 2; ++ks)
#pragma unroll
      for (int nt = 0; nt < 4; ++nt)
#pragma unroll
        for (int h = 0; h < 2; ++h) {
          const int k = ks * 16 + 2 * fq + 8 * h, f = nt * 8 + fgr;
          split_bf16x2(sW[k * DO + f], sW[(k + 1) * DO + f], wbh[ks][nt][h], wbl[ks][nt][h]);
        }
  }
  const float inv0 = a.n_up > 0 ? 1.f / (float)a.n_up : 0.f;
  const float inv1 = n - a.n_up > 0 ? 1.f / (float)(n - a.n_up) : 0.f;
  const long n_tiles = (a.groups + tg - 1) / tg;
  long tile = blockIdx.x;
  if (tile < n_tiles) load_tile<DIN, Q>(a.Ein, tile * tg, (int)min((long)tg, a.groups - tile * tg), n, sin);
  for (int it = 0; tile < n_tiles; tile += gridDim.x, ++it) {
    const long g0 = tile * tg;
    const int tge = (int)min((long)tg, a.groups - g0);
    const int np = tge * n;  // pairs in this tile
    const long next = tile + gridDim.x;
    cp_async_wait_all();
    __syncthreads();  // this tile's rows are in; every thread is done with the previous tile
    if (!LAYER) {
      float* cur = sin + (size_t)(it & 1) * tg * n * IPS;
      if (next < n_tiles)
        load_tile<DIN, Q>(a.Ein, next * tg, (int)min((long)tg, a.groups - next * tg), n,
                          sin + (size_t)((it + 1) & 1) * tg * n * IPS);
      spin_sums<Q, ORS, OPS>(a, tge, cur, sS);
      __syncthreads();
      dense_means<Q, ORS, OPS>(a, g0, tge, cur, sS, inv0, inv1);
      continue;
    }
    if constexpr (MMA) {
      // ---- the layer on warp MMAs: pre-activations of 16-row strips (row
      // p Q + q is quantity q of pair p) into the output tile, then the
      // forward-Laplacian tanh rule per (pair, 8 features) in place ----
      const int rows = np * Q;
      for (int st = warp; st * 16 < rows; st += kPairThreads / 32) {
        const int r0 = st * 16 + fgr, r1 = r0 + 8;
        const float* x0 = r0 < rows ? sin + (r0 / Q) * IPS + (r0 % Q) * DIN : nullptr;
        const float* x1 = r1 < rows ? sin + (r1 / Q) * IPS + (r1 % Q) * DIN : nullptr;
        float acc[4][4];
#pragma unroll
        for (int nt = 0; nt < 4; ++nt)
#pragma unroll
          for (int r = 0; r < 4; ++r) acc[nt][r] = 0.f;
#pragma unroll
        for (int ks = 0; ks < 2; ++ks) {
          uint32_t ah[4], al[4];
          const int k = ks * 16 + 2 * fq;
          const float2 v00 = x0 ? *reinterpret_cast<const float2*>(x0 + k) : make_float2(0.f, 0.f);
          const float2 v10 = x1 ? *reinterpret_cast<const float2*>(x1 + k) : make_float2(0.f, 0.f);
          const float2 v01 = x0 ? *reinterpret_cast<const float2*>(x0 + k + 8) : make_float2(0.f, 0.f);
          const float2 v11 = x1 ? *reinterpret_cast<const float2*>(x1 + k + 8) : make_float2(0.f, 0.f);
          split_bf16x2(v00.x, v00.y, ah[0], al[0]);
          split_bf16x2(v10.x, v10.y, ah[1], al[1]);
          split_bf16x2(v01.x, v01.y, ah[2], al[2]);
          split_bf16x2(v11.x, v11.y, ah[3], al[3]);
#pragma unroll
          for (int nt = 0; nt < 4; ++nt) {
            mma_bf16_16816(acc[nt], al, wbh[ks][nt][0], wbh[ks][nt][1]);
            mma_bf16_16816(acc[nt], ah, wbl[ks][nt][0], wbl[ks][nt][1]);
            mma_bf16_16816(acc[nt], ah, wbh[ks][nt][0], wbh[ks][nt][1]);
          }
        }
#pragma unroll
        for (int nt = 0; nt < 4; ++nt) {
          const int f = nt * 8 + 2 * fq;
          if (r0 < rows)
            *reinterpret_cast<float2*>(sout_l + (r0 / Q) * OPS + (r0 % Q) * DO + f) = make_float2(acc[nt][0], acc[nt][1]);
          if (r1 < rows)
            *reinterpret_cast<float2*>(sout_l + (r1 / Q) * OPS + (r1 % Q) * DO + f) = make_float2(acc[nt][2], acc[nt][3]);
        }
      }
      __syncthreads();  // every pre-activation of the tile is in the output tile
      for (int task = tid; task < np * FG; task += kPairThreads) {
        const int p = task / FG, fg = task - p * FG;
        const float* ip = sin + p * IPS;
        float* op = sout_l + p * OPS;
        float zq[Q][8], ov[Q][8], yv[8];
#pragma unroll
        for (int q = 0; q < Q; ++q) {
          const float4 z0 = *reinterpret_cast<const float4*>(op + q * DO + fg * 8);
          const float4 z1 = *reinterpret_cast<const float4*>(op + q * DO + fg * 8 + 4);
          zq[q][0] = z0.x; zq[q][1] = z0.y; zq[q][2] = z0.z; zq[q][3] = z0.w;
          zq[q][4] = z1.x; zq[q][5] = z1.y; zq[q][6] = z1.z; zq[q][7] = z1.w;
        }
#pragma unroll
        for (int j = 0; j < 8; ++j) {
          const int f = fg * 8 + j;
          const float y = tanhf(zq[0][j] + sb[f]);
          const float s = 1.f - y * y;
          yv[j] = y;
          ov[0][j] = y + (a.residual ? ip[f] : 0.f);
          if (Q > 1) {
            const float sq = zq[1][j] * zq[1][j] + zq[2][j] * zq[2][j] + zq[3][j] * zq[3][j];
#pragma unroll
            for (int q = 1; q <= 3 && q < Q; ++q) ov[q][j] = s * zq[q][j] + (a.residual ? ip[q * DIN + f] : 0.f);
            if (Q > 4) ov[4][j] = s * zq[4][j] - 4.f * y * s * sq + (a.residual ? ip[4 * DIN + f] : 0.f);
          }
        }
        const long gp = g0 * n + p;  // global pair index
#pragma unroll
        for (int q = 0; q < Q; ++q) {
          const float4 o0 = make_float4(ov[q][0], ov[q][1], ov[q][2], ov[q][3]);
          const float4 o1 = make_float4(ov[q][4], ov[q][5], ov[q][6], ov[q][7]);
          float* so = op + q * DO + fg * 8;
          *reinterpret_cast<float4*>(so) = o0;
          *reinterpret_cast<float4*>(so + 4) = o1;
          if (a.Eout) {
            float* go = a.Eout + (gp * Q + q) * DO + fg * 8;
            *reinterpret_cast<float4*>(go) = o0;
            *reinterpret_cast<float4*>(go + 4) = o1;
          }
        }
        if (a.Y2) {
          float* gy = a.Y2 + gp * DO + fg * 8;
          *reinterpret_cast<float4*>(gy) = make_float4(yv[0], yv[1], yv[2], yv[3]);
          *reinterpret_cast<float4*>(gy + 4) = make_float4(yv[4], yv[5], yv[6], yv[7]);
        }
      }
    } else {
    // ---- the layer: R rows x FW features per task ----
    const int nq = Q == 1 ? (np + 3) / 4 : np;  // tasks per feature group
    for (int task = tid; task < nq * FG; task += kPairThreads) {
      const int pq = task / FG, fg = task - pq * FG;
      int prow[R];  // shared offset of each row
#pragma unroll
      for (int r = 0; r < R; ++r)
        prow[r] = Q == 1 ? min(pq + r * nq, np - 1) * IPS : pq * IPS + r * DIN;
      // accumulators as feature pairs (2j, 2j + 1): packed FMAs
      f2_t acc2[R][FW / 2];
#pragma unroll
      for (int r = 0; r < R; ++r)
#pragma unroll
        for (int j = 0; j < FW / 2; ++j) acc2[r][j] = 0ull;
#pragma unroll
      for (int k = 0; k < DIN; k += 4) {
        float4 xv[R];
#pragma unroll
        for (int r = 0; r < R; ++r) xv[r] = *reinterpret_cast<const float4*>(sin + prow[r] + k);
#pragma unroll
        for (int kk = 0; kk < 4; ++kk) {
          ulonglong2 w[FW / 4];
#pragma unroll
          for (int h = 0; h < FW / 4; ++h)
            w[h] = *reinterpret_cast<const ulonglong2*>(sW + (k + kk) * DO + fg * FW + 4 * h);
#pragma unroll
          for (int r = 0; r < R; ++r) {
            const f2_t xr = f2_splat(comp(xv[r], kk));
#pragma unroll
            for (int h = 0; h < FW / 4; ++h) {
              f2_fma(acc2[r][2 * h], w[h].x, xr);
              f2_fma(acc2[r][2 * h + 1], w[h].y, xr);
            }
          }
        }
      }
      float acc[R][FW];
#pragma unroll
      for (int r = 0; r < R; ++r)
#pragma unroll
        for (int j = 0; j < FW / 2; ++j) {
          acc[r][2 * j] = f2_lo(acc2[r][j]);
          acc[r][2 * j + 1] = f2_hi(acc2[r][j]);
        }
      // forward-Laplacian tanh, residual, stores (shared output tile, new rows, tanh values)
      const int npair = Q == 1 ? R : 1;
#pragma unroll
      for (int u = 0; u < npair; ++u) {
        const int p = Q == 1 ? pq + u * nq : pq;
        if (p >= np) break;
        const float* ip = sin + p * IPS;
        float ov[Q][FW], yv[FW];
#pragma unroll
        for (int j = 0; j < FW; ++j) {
          const int f = fg * FW + j;
          const float z0 = Q == 1 ? acc[u][j] : acc[0][j];
          const float y = tanhf(z0 + sb[f]);
          const float s = 1.f - y * y;
          yv[j] = y;
          ov[0][j] = y + (a.residual ? ip[f] : 0.f);
          if (Q > 1) {
            const float sq = acc[1][j] * acc[1][j] + acc[2][j] * acc[2][j] + acc[3][j] * acc[3][j];
#pragma unroll
            for (int q = 1; q <= 3 && q < Q; ++q) ov[q][j] = s * acc[q][j] + (a.residual ? ip[q * DIN + f] : 0.f);
            if (Q > 4) ov[4][j] = s * acc[4][j] - 4.f * y * s * sq + (a.residual ? ip[4 * DIN + f] : 0.f);
          }
        }
        const long gp = g0 * n + p;  // global pair index
#pragma unroll
        for (int q = 0; q < Q; ++q) {
#pragma unroll
          for (int h = 0; h < FW / 4; ++h) {
            const float4 o = make_float4(ov[q][4 * h], ov[q][4 * h + 1], ov[q][4 * h + 2], ov[q][4 * h + 3]);
            *reinterpret_cast<float4*>(sout_l + p * OPS + q * DO + fg * FW + 4 * h) = o;
            if (a.Eout) *reinterpret_cast<float4*>(a.Eout + (gp * Q + q) * DO + fg * FW + 4 * h) = o;
          }
        }
        if (a.Y2) {
#pragma unroll
          for (int h = 0; h < FW / 4; ++h)
            *reinterpret_cast<float4*>(a.Y2 + gp * DO + fg * FW + 4 * h) =
                make_float4(yv[4 * h], yv[4 * h + 1], yv[4 * h + 2], yv[4 * h + 3]);
        }
      }
    }
    }  // SIMT contraction
    __syncthreads();  // output tile complete; the input tile is free
    if (next < n_tiles) load_tile<DIN, Q>(a.Ein, next * tg, (int)min((long)tg, a.groups - next * tg), n, sin);
    spin_sums<Q, ORS, OPS>(a, tge, sout_l, sS);
    __syncthreads();
    dense_means<Q, ORS, OPS>(a, g0, tge, sout_l, sS, inv0, inv1);
  }
  cp_async_wait_all();  // no copy outlives the block
}

template <int DIN, int DO, int Q, bool LAYER, bool MMA = false, bool LARGE = false>
void launch_inst(cudaStream_t s, PairArgs a) {
  auto kern = k_pair_layer<DIN, DO, Q, LAYER, MMA, LARGE>;
  constexpr int MB = min_blocks<Q, LAYER, MMA, LARGE>();
  const size_t budget = kSmemPerSM / MB - 1024;
  static PerDeviceOnce attr;  // the attribute is per function and device
  attr([&] { cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)budget); });
  // groups per tile: about one task (layer) or two output steps (means) per
  // thread, within the shared-memory share of the resident blocks
  constexpr int FW = task_features<Q, LAYER, MMA>();
  const int per_group = LAYER ? (a.n * (DO / FW) + (Q == 1 ? 3 : 0)) / (Q == 1 ? 4 : 1) : a.C * (int)(a.ldm / 8);
  const int target = LAYER ? kPairThreads : 2 * kPairThreads;
  int tg = (target + per_group - 1) / per_group;
  if (tg < 1) tg = 1;
  while (tg > 1 && pair_smem_bytes<DIN, DO, Q, LAYER>(a.n, tg) > budget) --tg;
  a.tg = tg;
  const size_t smem = pair_smem_bytes<DIN, DO, Q, LAYER>(a.n, tg);
  int occ = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, kPairThreads, smem) != cudaSuccess || occ < 1) occ = 1;
  int dev = 0, sms = 152;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const long tiles = (a.groups + tg - 1) / tg;
  const long blocks = std::min<long>(tiles, (long)sms * occ);  // persistent
  FN_COUNT(1), kern<<<(unsigned)blocks, kPairThreads, smem, s>>>(a);
}

// A layer launch: in the local-energy pass, the two-block instance when one
// group of pair rows does not fit the shared-memory share of three blocks.
template <int DIN, int DO, int Q>
void launch_layer(cudaStream_t s, const PairArgs& a) {
  if constexpr (Q > 1) {
    if (pair_smem_bytes<DIN, DO, Q, true>(a.n, 1) > kSmemPerSM / min_blocks<Q, true>() - 1024) {
      launch_inst<DIN, DO, Q, true, false, true>(s, a);
      return;
    }
  }
  launch_inst<DIN, DO, Q, true>(s, a);
}

template <int Q>
bool dispatch(cudaStream_t s, const PairArgs& a, int din, int dout) {
  if (!a.W) {
    switch (din) {
      case 4: launch_inst<4, 4, Q, false>(s, a); return true;
      case 8: launch_inst<8, 8, Q, false>(s, a); return true;
      case 16: launch_inst<16, 16, Q, false>(s, a); return true;
      case 32: launch_inst<32, 32, Q, false>(s, a); return true;
      default: return false;
    }
  }
  if (din == 4 && dout == 8) return launch_layer<4, 8, Q>(s, a), true;
  if (din == 8 && dout == 8) return launch_layer<8, 8, Q>(s, a), true;
  if (din == 4 && dout == 16) return launch_layer<4, 16, Q>(s, a), true;
  if (din == 16 && dout == 16) return launch_layer<16, 16, Q>(s, a), true;
  if (din == 4 && dout == 32) return launch_layer<4, 32, Q>(s, a), true;
  if (din == 32 && dout == 32) {
    // value rows only: in the local-energy pass (Q = 5) the contraction is a
    // small share of the layer, which keeps its FP32 FMAs
    if (Q == 1 && a.mma) return launch_inst<32, 32, 1, true, true>(s, a), true;
    return launch_layer<32, 32, Q>(s, a), true;
  }
  return false;
}

// ---------------------------------------------------------------------------
// Backward of the two-electron layer (value pass, for the parameter adjoint)

constexpr int kBwdPairs = 96;  // pairs per tile (static shared memory under 48 KB)
constexpr int kBwdMaxBlocks = 152 * 4;

// One tile of kBwdPairs pairs per step of a persistent grid.  Shared tiles:
// Zbar and Eout_bar [P][DO + 1], Ein [P][DIN + 1], W [DO][DIN].  Thread t owns
// dW[f][k0 .. k0 + 3] (f = t / (DIN / 4)) and, for k0 == 0, dc[f]; the
// input-gradient rows are 4 features per task.
template <int DIN, int DO>
__global__ void __launch_bounds__(256) k_pair_bwd(PairBwdArgs a) {
  // Ein rows padded to a multiple of 4 floats: the dW loop reads 4 features of
  // one row per thread (all threads on the same row: no bank conflict)
  constexpr int P = kBwdPairs, ZS = DO + 1, ES = DIN + 4;
  __shared__ float Zt[P * ZS];
  __shared__ float Ot[P * ZS];
  __shared__ __align__(16) float Et[P * ES];
  __shared__ __align__(16) float Ws[DO * DIN];
  const int tid = threadIdx.x;
  for (int t = tid; t < DO * DIN; t += 256) Ws[t] = a.W[t];
  constexpr int NW = DO * DIN / 4;  // dW owners
  const bool own = tid < NW;
  const int f = own ? tid / (DIN / 4) : 0, k0 = own ? (tid % (DIN / 4)) * 4 : 0;
  float acc[4] = {0.f, 0.f, 0.f, 0.f}, cacc = 0.f;
  const long n_tiles = (a.pairs + P - 1) / P;
  for (long tile = blockIdx.x; tile < n_tiles; tile += gridDim.x) {
    const long p0 = tile * P;
    const int np = (int)min((long)P, a.pairs - p0);
    __syncthreads();  // previous tile fully used
    for (int t = tid; t < np * (DO / 4); t += 256) {
      const int p = t / (DO / 4), q = (t % (DO / 4)) * 4;
      float4 ob = a.Eout_bar ? *reinterpret_cast<const float4*>(a.Eout_bar + (p0 + p) * DO + q)
                             : make_float4(0.f, 0.f, 0.f, 0.f);
      if (a.M2bar) {  // the next layer's pair-mean gradient, spread over the pairs it averaged
        const long gp = p0 + p, wi = gp / a.n;
        const int j = (int)(gp - wi * a.n), sj = j < a.n_up ? 0 : 1;
        const float ns = (float)(sj == 0 ? a.n_up : a.n - a.n_up);
        const float4 m = *reinterpret_cast<const float4*>(a.M2bar + wi * 2 * DO + sj * DO + q);
        ob.x += m.x / ns;
        ob.y += m.y / ns;
        ob.z += m.z / ns;
        ob.w += m.w / ns;
      }
      const float4 y = *reinterpret_cast<const float4*>(a.Y + (p0 + p) * DO + q);
      float* zr = Zt + p * ZS + q;
      float* orr = Ot + p * ZS + q;
      zr[0] = ob.x * (1.f - y.x * y.x);
      zr[1] = ob.y * (1.f - y.y * y.y);
      zr[2] = ob.z * (1.f - y.z * y.z);
      zr[3] = ob.w * (1.f - y.w * y.w);
      orr[0] = ob.x;
      orr[1] = ob.y;
      orr[2] = ob.z;
      orr[3] = ob.w;
    }
    for (int t = tid; t < np * (DIN / 4); t += 256) {
      const int p = t / (DIN / 4), q = (t % (DIN / 4)) * 4;
      *reinterpret_cast<float4*>(Et + p * ES + q) = *reinterpret_cast<const float4*>(a.Ein + (p0 + p) * DIN + q);
    }
    __syncthreads();
    if (own) {
      for (int p = 0; p < np; ++p) {
        const float z = Zt[p * ZS + f];
        const float4 e = *reinterpret_cast<const float4*>(Et + p * ES + k0);
        acc[0] = fmaf(z, e.x, acc[0]);
        acc[1] = fmaf(z, e.y, acc[1]);
        acc[2] = fmaf(z, e.z, acc[2]);
        acc[3] = fmaf(z, e.w, acc[3]);
        cacc += z;
      }
    }
    if (a.Ein_bar) {
      for (int t = tid; t < np * (DIN / 4); t += 256) {
        const int p = t / (DIN / 4), q = (t % (DIN / 4)) * 4;
        const float* z = Zt + p * ZS;
        float o[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll 8
        for (int ff = 0; ff < DO; ++ff) {
          const float zf = z[ff];
          const float4 w = *reinterpret_cast<const float4*>(Ws + ff * DIN + q);
          o[0] = fmaf(zf, w.x, o[0]);
          o[1] = fmaf(zf, w.y, o[1]);
          o[2] = fmaf(zf, w.z, o[2]);
          o[3] = fmaf(zf, w.w, o[3]);
        }
        if (a.residual) {
          const float* r = Ot + p * ZS + q;
          o[0] += r[0];
          o[1] += r[1];
          o[2] += r[2];
          o[3] += r[3];
        }
        *reinterpret_cast<float4*>(a.Ein_bar + (p0 + p) * DIN + q) = make_float4(o[0], o[1], o[2], o[3]);
      }
    }
  }
  // this block's partial sums
  constexpr int PS = DO * DIN + DO;
  float* part = a.partial + (long)blockIdx.x * PS;
  if (own) {
    part[f * DIN + k0] = acc[0];
    part[f * DIN + k0 + 1] = acc[1];
    part[f * DIN + k0 + 2] = acc[2];
    part[f * DIN + k0 + 3] = acc[3];
    if (k0 == 0) part[DO * DIN + f] = cacc;
  }
}

// Mixed-path variant for 32 -> 32 layers: the staging, Zbar and dc as in
// k_pair_bwd; dW = Zbar^T Ein (M = output feature, N = input feature, K =
// the tile's pairs) and Ein_bar = Zbar W (M = pair, N = input feature, K =
// output feature) on m16n8k16 warp MMAs with BF16 hi + lo operands (three
// products, FP32 accumulation).  Warp w owns the dW block of rows 16 (w / 4)
// and columns 8 (w % 4); the Ein_bar blocks of a tile go round the warps.
// Fragments (g = lane / 4, q = lane % 4): A rows g, g + 8 and columns 2q,
// 2q + 1 (+ 8); B rows 2q, 2q + 1 (+ 8) and column g; the result rows g, g + 8
// and columns 2q, 2q + 1.
template <int DIN, int DO>
__global__ void __launch_bounds__(256) k_pair_bwd_mma(PairBwdArgs a) {
  static_assert(DIN == 32 && DO == 32, "warp-MMA pair backward: 32 -> 32 layers");
  // Zbar rows padded to 36 floats: the dW fragments read Zbar down the pairs,
  // lane (g, q) at row 2q, column g, which lands on bank 8q + g
  constexpr int P = kBwdPairs, ZS = DO + 4, ES = DIN + 4;
  static_assert(P % 16 == 0, "whole 16-pair steps");
  __shared__ float Zt[P * ZS];
  __shared__ float Ot[P * ZS];
  __shared__ __align__(16) float Et[P * ES];
  __shared__ __align__(16) float Ws[DO * DIN];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, g = lane >> 2, q = lane & 3;
  for (int t = tid; t < DO * DIN; t += 256) Ws[t] = a.W[t];
  __syncthreads();
  // W as the B operand of Ein_bar (k = output feature f, n = input feature)
  uint32_t wbh[2][4][2], wbl[2][4][2];
#pragma unroll
  for (int ks = 0; ks < 2; ++ks)
#pragma unroll
    for (int nt = 0; nt < 4; ++nt)
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const int f = ks * 16 + 2 * q + 8 * h, k = nt * 8 + g;
        split_bf16x2(Ws[f * DIN + k], Ws[(f + 1) * DIN + k], wbh[ks][nt][h], wbl[ks][nt][h]);
      }
  const int mt = warp >> 2, nt0 = warp & 3;
  float dacc[4] = {0.f, 0.f, 0.f, 0.f}, cacc = 0.f;
  const long n_tiles = (a.pairs + P - 1) / P;
  for (long tile = blockIdx.x; tile < n_tiles; tile += gridDim.x) {
    const long p0 = tile * P;
    const int np = (int)min((long)P, a.pairs - p0);
    __syncthreads();  // previous tile fully used
    for (int t = tid; t < P * (DO / 4); t += 256) {
      const int p = t / (DO / 4), qq = (t % (DO / 4)) * 4;
      float* zr = Zt + p * ZS + qq;
      float* orr = Ot + p * ZS + qq;
      if (p >= np) {  // rows past the tile's pairs add nothing to the MMAs
        zr[0] = zr[1] = zr[2] = zr[3] = 0.f;
        orr[0] = orr[1] = orr[2] = orr[3] = 0.f;
        continue;
      }
      float4 ob = a.Eout_bar ? *reinterpret_cast<const float4*>(a.Eout_bar + (p0 + p) * DO + qq)
                             : make_float4(0.f, 0.f, 0.f, 0.f);
      if (a.M2bar) {
        const long gp = p0 + p, wi = gp / a.n;
        const int j = (int)(gp - wi * a.n), sj = j < a.n_up ? 0 : 1;
        const float ns = (float)(sj == 0 ? a.n_up : a.n - a.n_up);
        const float4 m = *reinterpret_cast<const float4*>(a.M2bar + wi * 2 * DO + sj * DO + qq);
        ob.x += m.x / ns;
        ob.y += m.y / ns;
        ob.z += m.z / ns;
        ob.w += m.w / ns;
      }
      const float4 y = *reinterpret_cast<const float4*>(a.Y + (p0 + p) * DO + qq);
      zr[0] = ob.x * (1.f - y.x * y.x);
      zr[1] = ob.y * (1.f - y.y * y.y);
      zr[2] = ob.z * (1.f - y.z * y.z);
      zr[3] = ob.w * (1.f - y.w * y.w);
      orr[0] = ob.x;
      orr[1] = ob.y;
      orr[2] = ob.z;
      orr[3] = ob.w;
    }
    for (int t = tid; t < P * (DIN / 4); t += 256) {
      const int p = t / (DIN / 4), qq = (t % (DIN / 4)) * 4;
      *reinterpret_cast<float4*>(Et + p * ES + qq) =
          p < np ? *reinterpret_cast<const float4*>(a.Ein + (p0 + p) * DIN + qq) : make_float4(0.f, 0.f, 0.f, 0.f);
    }
    __syncthreads();
    if (tid < DO)
      for (int p = 0; p < np; ++p) cacc += Zt[p * ZS + tid];
    // dW block (rows 16 mt, columns 8 nt0) over the tile's pairs
#pragma unroll 2
    for (int ks = 0; ks < P / 16; ++ks) {
      const int pa = ks * 16 + 2 * q, f0 = mt * 16 + g, k0 = nt0 * 8 + g;
      uint32_t ah[4], al[4], bh[2], bl[2];
      split_bf16x2(Zt[pa * ZS + f0], Zt[(pa + 1) * ZS + f0], ah[0], al[0]);
      split_bf16x2(Zt[pa * ZS + f0 + 8], Zt[(pa + 1) * ZS + f0 + 8], ah[1], al[1]);
      split_bf16x2(Zt[(pa + 8) * ZS + f0], Zt[(pa + 9) * ZS + f0], ah[2], al[2]);
      split_bf16x2(Zt[(pa + 8) * ZS + f0 + 8], Zt[(pa + 9) * ZS + f0 + 8], ah[3], al[3]);
      split_bf16x2(Et[pa * ES + k0], Et[(pa + 1) * ES + k0], bh[0], bl[0]);
      split_bf16x2(Et[(pa + 8) * ES + k0], Et[(pa + 9) * ES + k0], bh[1], bl[1]);
      mma_bf16_16816(dacc, al, bh[0], bh[1]);
      mma_bf16_16816(dacc, ah, bl[0], bl[1]);
      mma_bf16_16816(dacc, ah, bh[0], bh[1]);
    }
    if (a.Ein_bar) {
      for (int blk = warp; blk < (P / 16) * 4; blk += 8) {
        const int pm = blk >> 2, nt = blk & 3, pr = pm * 16 + g;
        float acc[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
        for (int ks = 0; ks < 2; ++ks) {
          const int fa = ks * 16 + 2 * q;
          uint32_t ah[4], al[4];
          split_bf16x2(Zt[pr * ZS + fa], Zt[pr * ZS + fa + 1], ah[0], al[0]);
          split_bf16x2(Zt[(pr + 8) * ZS + fa], Zt[(pr + 8) * ZS + fa + 1], ah[1], al[1]);
          split_bf16x2(Zt[pr * ZS + fa + 8], Zt[pr * ZS + fa + 9], ah[2], al[2]);
          split_bf16x2(Zt[(pr + 8) * ZS + fa + 8], Zt[(pr + 8) * ZS + fa + 9], ah[3], al[3]);
          mma_bf16_16816(acc, al, wbh[ks][nt][0], wbh[ks][nt][1]);
          mma_bf16_16816(acc, ah, wbl[ks][nt][0], wbl[ks][nt][1]);
          mma_bf16_16816(acc, ah, wbh[ks][nt][0], wbh[ks][nt][1]);
        }
        const int k = nt * 8 + 2 * q;
#pragma unroll
        for (int h = 0; h < 2; ++h) {
          const int p = pr + 8 * h;
          if (p >= np) continue;
          float o0 = acc[2 * h], o1 = acc[2 * h + 1];
          if (a.residual) {
            o0 += Ot[p * ZS + k];
            o1 += Ot[p * ZS + k + 1];
          }
          *reinterpret_cast<float2*>(a.Ein_bar + (p0 + p) * DIN + k) = make_float2(o0, o1);
        }
      }
    }
  }
  // this block's partial sums, laid out as in k_pair_bwd
  constexpr int PS = DO * DIN + DO;
  float* part = a.partial + (long)blockIdx.x * PS;
  {
    const int f = mt * 16 + g, k = nt0 * 8 + 2 * q;
    part[f * DIN + k] = dacc[0];
    part[f * DIN + k + 1] = dacc[1];
    part[(f + 8) * DIN + k] = dacc[2];
    part[(f + 8) * DIN + k + 1] = dacc[3];
  }
  if (tid < DO) part[DO * DIN + tid] = cacc;
}

// grad[j] += sum over blocks of the partials, in FP64 and block order.
__global__ void k_pair_bwd_reduce(const float* __restrict__ part, int nblocks, int ps, int nw, double* grad_W,
                                  double* grad_c) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= ps) return;
  double s = 0.0;
#pragma unroll 8  // loads ahead of the (unchanged) summation order
  for (int b = 0; b < nblocks; ++b) s += (double)part[(long)b * ps + j];
  if (j < nw) grad_W[j] += s;
  else grad_c[j - nw] += s;
}

template <int DIN, int DO, bool MMA = false>
void launch_bwd_inst(cudaStream_t s, const PairBwdArgs& a) {
  int occ = 0, dev = 0, sms = 152;
  auto kern = MMA ? k_pair_bwd_mma<32, 32> : k_pair_bwd<DIN, DO>;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, 256, 0) != cudaSuccess || occ < 1)
    occ = 1;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const long tiles = (a.pairs + kBwdPairs - 1) / kBwdPairs;
  long blocks = std::min<long>(tiles, (long)sms * occ);
  if (blocks > kBwdMaxBlocks) blocks = kBwdMaxBlocks;
  FN_COUNT(1), kern<<<(unsigned)blocks, 256, 0, s>>>(a);
  const int ps = DO * DIN + DO;
  FN_COUNT(1), k_pair_bwd_reduce<<<(ps + 255) / 256, 256, 0, s>>>(a.partial, (int)blocks, ps, DO * DIN, a.grad_W,
                                                                   a.grad_c);
}

}  // namespace

bool pair_bwd_supported(int din, int dout) {
  return (dout == 8 || dout == 16 || dout == 32) && (din == 4 || din == dout);
}

long pair_bwd_scratch_floats(int din, int dout) { return (long)kBwdMaxBlocks * (dout * din + dout); }

bool launch_pair_bwd(cudaStream_t s, const PairBwdArgs& a, int din, int dout) {
  if (a.pairs <= 0) return true;
  if (din == 4 && dout == 8) return launch_bwd_inst<4, 8>(s, a), true;
  if (din == 8 && dout == 8) return launch_bwd_inst<8, 8>(s, a), true;
  if (din == 4 && dout == 16) return launch_bwd_inst<4, 16>(s, a), true;
  if (din == 16 && dout == 16) return launch_bwd_inst<16, 16>(s, a), true;
  if (din == 4 && dout == 32) return launch_bwd_inst<4, 32>(s, a), true;
  if (din == 32 && dout == 32) {
    if (a.mma) return launch_bwd_inst<32, 32, true>(s, a), true;
    return launch_bwd_inst<32, 32>(s, a), true;
  }
  return false;
}

bool pair_layer_supported(int n, int din, int dout, bool layer, int Q, int C, long ldm) {
  const bool din_ok = din == 4 || din == 8 || din == 16 || din == 32;
  const bool dout_ok = !layer || ((dout == 8 || dout == 16 || dout == 32) && (din == 4 || din == dout));
  const int d = layer ? dout : din;
  if (!(din_ok && dout_ok && (Q == 1 || Q == kQ) && ldm % 8 == 0 && ldm >= 2 * d && C >= 1)) return false;
  if (Q == kQ && C < 3 * n + 2) return false;
  // one group per tile must fit in the shared-memory share of a block
  const int mb = layer ? (Q == 1 ? min_blocks<1, true>() : min_blocks<kQ, true, false, true>()) : min_blocks<1, false>();
  const size_t in = (size_t)(layer ? 1 : 2) * n * (Q * din + 4), out = layer ? (size_t)n * (Q * dout + 4) : 0;
  const size_t w = layer ? (size_t)din * dout + dout : 0;
  return sizeof(float) * (in + out + w + 2 * Q * d) <= (size_t)(kSmemPerSM / mb - 1024);
}

bool launch_pair_layer(cudaStream_t s, const PairArgs& a, int din, int dout, int Q) {
  if (a.groups <= 0) return true;
  return Q == 1 ? dispatch<1>(s, a, din, dout) : dispatch<kQ>(s, a, din, dout);
}

}  // namespace fn
