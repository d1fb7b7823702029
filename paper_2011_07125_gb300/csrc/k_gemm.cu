// FP32 SIMT GEMM for the plain-FP32 path and the adjoint: 128x128 CTA tile,
// 16-deep K slices double-buffered through shared memory, 8x8 outputs per
// thread.  Three operand orientations (NT forward, NN backward-data, TN
// backward-weights with split-K and an FP64 reduction of the partials).
#include "fn_internal.cuh"

namespace fn {
namespace {

constexpr int BM = 128, BN = 128, BK = 16, NT = 256;

// One 8-element run of a 128 x 16 operand tile per thread: along k when the
// operand is K-contiguous (row = t / 2, k offset 8 (t % 2)), along m/n
// otherwise (k = t / 16, offset 8 (t % 16)).  float4 loads when the run is in
// bounds and the row stride allows it.
template <bool KM>
__device__ __forceinline__ void load_run(const float* __restrict__ P, long ld, long r0, long R, long k0, long k1,
                                         int tid, bool vec, float (&v)[8]) {
  if (KM) {
    const long r = r0 + (tid >> 1);
    const long k = k0 + (tid & 1) * 8;
    if (r < R) {
      const float* p = P + r * ld + k;
      if (vec && k + 8 <= k1) {
        const float4 a = reinterpret_cast<const float4*>(p)[0];
        const float4 b = reinterpret_cast<const float4*>(p)[1];
        v[0] = a.x; v[1] = a.y; v[2] = a.z; v[3] = a.w; v[4] = b.x; v[5] = b.y; v[6] = b.z; v[7] = b.w;
        return;
      }
#pragma unroll
      for (int q = 0; q < 8; ++q) v[q] = (k + q < k1) ? p[q] : 0.f;
    } else {
#pragma unroll
      for (int q = 0; q < 8; ++q) v[q] = 0.f;
    }
  } else {
    const long k = k0 + (tid >> 4);
    const long r = r0 + (tid & 15) * 8;
    if (k < k1) {
      const float* p = P + k * ld + r;
      if (vec && r + 8 <= R) {
        const float4 a = reinterpret_cast<const float4*>(p)[0];
        const float4 b = reinterpret_cast<const float4*>(p)[1];
        v[0] = a.x; v[1] = a.y; v[2] = a.z; v[3] = a.w; v[4] = b.x; v[5] = b.y; v[6] = b.z; v[7] = b.w;
        return;
      }
#pragma unroll
      for (int q = 0; q < 8; ++q) v[q] = (r + q < R) ? p[q] : 0.f;
    } else {
#pragma unroll
      for (int q = 0; q < 8; ++q) v[q] = 0.f;
    }
  }
}

template <bool KM>
__device__ __forceinline__ void store_run(float (*S)[BM], int tid, const float (&v)[8]) {
  if (KM) {
    const int r = tid >> 1, k = (tid & 1) * 8;
#pragma unroll
    for (int q = 0; q < 8; ++q) S[k + q][r] = v[q];
  } else {
    const int k = tid >> 4, r = (tid & 15) * 8;
    reinterpret_cast<float4*>(&S[k][r])[0] = make_float4(v[0], v[1], v[2], v[3]);
    reinterpret_cast<float4*>(&S[k][r])[1] = make_float4(v[4], v[5], v[6], v[7]);
  }
}

// A_KM: A stored [M][K] (k contiguous) else [K][M].
// B_KM: B stored [N][K] (k contiguous) else [K][N].
template <bool A_KM, bool B_KM>
__global__ void __launch_bounds__(NT, 2) k_sgemm(long M, long N, long K, const float* __restrict__ A, long lda,
                                              const float* __restrict__ B, long ldb, float* __restrict__ Cm,
                                              long ldc, Epi e, long k_per_split, int partial, int vec_a,
                                              int vec_b) {
  __shared__ __align__(16) float As[2][BK][BM];
  __shared__ __align__(16) float Bs[2][BK][BN];
  const int tid = threadIdx.x;
  const long m0 = (long)blockIdx.x * BM, n0 = (long)blockIdx.y * BN;
  const long kz0 = (long)blockIdx.z * k_per_split;
  const long kz1 = min(K, kz0 + k_per_split);
  if (partial) Cm += (long)blockIdx.z * M * ldc;

  float ra[8], rb[8];
  float acc[8][8];
#pragma unroll
  for (int i = 0; i < 8; ++i)
#pragma unroll
    for (int j = 0; j < 8; ++j) acc[i][j] = 0.f;

  const int ty = tid >> 4, tx = tid & 15;
  long kt = kz0;
  if (kt < kz1) {
    load_run<A_KM>(A, lda, m0, M, kt, kz1, tid, vec_a, ra);
    load_run<B_KM>(B, ldb, n0, N, kt, kz1, tid, vec_b, rb);
    store_run<A_KM>(As[0], tid, ra);
    store_run<B_KM>(Bs[0], tid, rb);
  }
  __syncthreads();
  int buf = 0;
  for (; kt < kz1; kt += BK) {
    const bool more = kt + BK < kz1;
    if (more) {
      load_run<A_KM>(A, lda, m0, M, kt + BK, kz1, tid, vec_a, ra);
      load_run<B_KM>(B, ldb, n0, N, kt + BK, kz1, tid, vec_b, rb);
    }
#pragma unroll
    for (int k = 0; k < BK; ++k) {
      float4 a0 = *reinterpret_cast<const float4*>(&As[buf][k][ty * 4]);
      float4 a1 = *reinterpret_cast<const float4*>(&As[buf][k][64 + ty * 4]);
      float4 b0 = *reinterpret_cast<const float4*>(&Bs[buf][k][tx * 4]);
      float4 b1 = *reinterpret_cast<const float4*>(&Bs[buf][k][64 + tx * 4]);
      float av[8] = {a0.x, a0.y, a0.z, a0.w, a1.x, a1.y, a1.z, a1.w};
      float bv[8] = {b0.x, b0.y, b0.z, b0.w, b1.x, b1.y, b1.z, b1.w};
#pragma unroll
      for (int i = 0; i < 8; ++i)
#pragma unroll
        for (int j = 0; j < 8; ++j) acc[i][j] = fmaf(av[i], bv[j], acc[i][j]);
    }
    if (more) {
      store_run<A_KM>(As[buf ^ 1], tid, ra);
      store_run<B_KM>(Bs[buf ^ 1], tid, rb);
    }
    __syncthreads();
    buf ^= 1;
  }

#pragma unroll
  for (int i = 0; i < 8; ++i) {
    const long r = m0 + (i < 4 ? ty * 4 + i : 64 + ty * 4 + (i - 4));
    if (r >= M) continue;
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      const long c = n0 + (j < 4 ? tx * 4 + j : 64 + tx * 4 + (j - 4));
      if (c >= N) continue;
      float v = acc[i][j];
      if (!partial) {
        if (e.beta != 0.f) v += e.beta * Cm[r * ldc + c];
        if (e.bias && (r % e.bias_period) == 0) v += e.bias[c];
        if (e.U) v += e.U[((r / e.u_div) * e.u_mul + r % e.u_mod) * e.ldu + c];
        if (e.act == 1) v = tanhf(v);
        if (e.res) v += e.res[r * e.ldr + c];
      }
      Cm[r * ldc + c] = v;
    }
  }
}

__global__ void k_reduce_partials(const float* __restrict__ part, int splits, long M, long N, double* grad,
                                  long ldg) {
  long idx = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= M * N) return;
  long m = idx / N, c = idx % N;
  double s = 0.0;
#pragma unroll 8  // loads ahead of the (unchanged) summation order
  for (int z = 0; z < splits; ++z) s += (double)part[(long)z * M * N + idx];
  grad[m * ldg + c] += s;
}

template <bool A_KM, bool B_KM>
void run(cudaStream_t s, long M, long N, long K, const float* A, long lda, const float* B, long ldb, float* C,
         long ldc, const Epi& e, long kps, int splits, int partial) {
  if (M <= 0 || N <= 0) return;
  const int va = (lda % 4 == 0) && ((uintptr_t)A % 16 == 0);
  const int vb = (ldb % 4 == 0) && ((uintptr_t)B % 16 == 0);
  dim3 grid((unsigned)((M + BM - 1) / BM), (unsigned)((N + BN - 1) / BN), (unsigned)splits);
  FN_COUNT(1), k_sgemm<A_KM, B_KM><<<grid, NT, 0, s>>>(M, N, K, A, lda, B, ldb, C, ldc, e, kps, partial, va, vb);
}
}  // namespace

void gemm_nt(cudaStream_t s, long M, long N, long K, const float* A, long lda, const float* B, long ldb, float* C,
             long ldc, const Epi& e) {
  run<true, true>(s, M, N, K, A, lda, B, ldb, C, ldc, e, K > 0 ? K : 1, 1, 0);
}

void gemm_nn(cudaStream_t s, long M, long N, long K, const float* A, long lda, const float* B, long ldb, float* C,
             long ldc, const Epi& e) {
  run<true, false>(s, M, N, K, A, lda, B, ldb, C, ldc, e, K > 0 ? K : 1, 1, 0);
}

int gemm_tn_splits(long M, long N, long K) {
  long tiles = ((M + BM - 1) / BM) * ((N + BN - 1) / BN);
  long want = (4 * 152 + tiles - 1) / tiles;  // about two waves of two CTAs per SM
  long maxs = (K + 511) / 512;                 // at least 512 rows per split
  long sp = want < maxs ? want : maxs;
  if (sp < 1) sp = 1;
  if (sp > 1024) sp = 1024;
  return (int)sp;
}

void gemm_tn_accum(cudaStream_t s, long M, long N, long K, const float* A, long lda, const float* B, long ldb,
                   double* grad, long ldg, float* scratch, int splits) {
  if (M <= 0 || N <= 0 || K <= 0) return;
  long kps = (K + splits - 1) / splits;
  kps = ((kps + BK - 1) / BK) * BK;
  Epi e;
  run<false, false>(s, M, N, K, A, lda, B, ldb, scratch, N, e, kps, splits, 1);
  long tot = M * N;
  FN_COUNT(1), k_reduce_partials<<<(unsigned)((tot + 255) / 256), 256, 0, s>>>(scratch, splits, M, N, grad, ldg);
}

void launch_reduce_partials(cudaStream_t s, const float* part, int splits, long M, long N, double* grad, long ldg) {
  const long tot = M * N;
  if (tot > 0)
    FN_COUNT(1), k_reduce_partials<<<(unsigned)((tot + 255) / 256), 256, 0, s>>>(part, splits, M, N, grad, ldg);
}

}  // namespace fn
