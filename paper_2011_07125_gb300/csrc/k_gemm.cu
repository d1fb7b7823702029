// FP32 SIMT GEMM for the plain-FP32 path and the adjoint: 128x128 CTA tile,
// 8-deep K slices double-buffered through shared memory, 8x8 outputs per
// thread.  Three operand orientations (NT forward, NN backward-data, TN
// backward-weights with split-K and an FP64 reduction of the partials).
#include "fn_internal.cuh"

namespace fn {
namespace {

constexpr int BM = 128, BN = 128, BK = 8, NT = 256;

// A_KM: A stored [M][K] (k contiguous) else [K][M].
// B_KM: B stored [N][K] (k contiguous) else [K][N].
template <bool A_KM, bool B_KM>
__global__ void __launch_bounds__(NT) k_sgemm(long M, long N, long K, const float* __restrict__ A, long lda,
                                              const float* __restrict__ B, long ldb, float* __restrict__ Cm,
                                              long ldc, Epi e, long k_per_split, int partial) {
  __shared__ __align__(16) float As[2][BK][BM];
  __shared__ __align__(16) float Bs[2][BK][BN];
  const int tid = threadIdx.x;
  const long m0 = (long)blockIdx.x * BM, n0 = (long)blockIdx.y * BN;
  const long kz0 = (long)blockIdx.z * k_per_split;
  const long kz1 = min(K, kz0 + k_per_split);
  if (partial) Cm += (long)blockIdx.z * M * ldc;

  float ra[4], rb[4];
  auto load = [&](long k0) {
    if (A_KM) {
      long m = m0 + (tid >> 1);
      long k = k0 + (tid & 1) * 4;
#pragma unroll
      for (int q = 0; q < 4; ++q) ra[q] = (m < M && k + q < kz1) ? A[m * lda + k + q] : 0.f;
    } else {
      long k = k0 + (tid >> 5);
      long m = m0 + (tid & 31) * 4;
#pragma unroll
      for (int q = 0; q < 4; ++q) ra[q] = (k < kz1 && m + q < M) ? A[k * lda + m + q] : 0.f;
    }
    if (B_KM) {
      long nn = n0 + (tid >> 1);
      long k = k0 + (tid & 1) * 4;
#pragma unroll
      for (int q = 0; q < 4; ++q) rb[q] = (nn < N && k + q < kz1) ? B[nn * ldb + k + q] : 0.f;
    } else {
      long k = k0 + (tid >> 5);
      long nn = n0 + (tid & 31) * 4;
#pragma unroll
      for (int q = 0; q < 4; ++q) rb[q] = (k < kz1 && nn + q < N) ? B[k * ldb + nn + q] : 0.f;
    }
  };
  auto store = [&](int buf) {
    if (A_KM) {
      int m = tid >> 1, k = (tid & 1) * 4;
#pragma unroll
      for (int q = 0; q < 4; ++q) As[buf][k + q][m] = ra[q];
    } else {
      int k = tid >> 5, m = (tid & 31) * 4;
      *reinterpret_cast<float4*>(&As[buf][k][m]) = make_float4(ra[0], ra[1], ra[2], ra[3]);
    }
    if (B_KM) {
      int nn = tid >> 1, k = (tid & 1) * 4;
#pragma unroll
      for (int q = 0; q < 4; ++q) Bs[buf][k + q][nn] = rb[q];
    } else {
      int k = tid >> 5, nn = (tid & 31) * 4;
      *reinterpret_cast<float4*>(&Bs[buf][k][nn]) = make_float4(rb[0], rb[1], rb[2], rb[3]);
    }
  };

  float acc[8][8];
#pragma unroll
  for (int i = 0; i < 8; ++i)
#pragma unroll
    for (int j = 0; j < 8; ++j) acc[i][j] = 0.f;

  const int ty = tid >> 4, tx = tid & 15;
  long kt = kz0;
  if (kt < kz1) {
    load(kt);
    store(0);
  }
  __syncthreads();
  int buf = 0;
  for (; kt < kz1; kt += BK) {
    const bool more = kt + BK < kz1;
    if (more) load(kt + BK);
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
    if (more) store(buf ^ 1);
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
  for (int z = 0; z < splits; ++z) s += (double)part[(long)z * M * N + idx];
  grad[m * ldg + c] += s;
}

template <bool A_KM, bool B_KM>
void run(cudaStream_t s, long M, long N, long K, const float* A, long lda, const float* B, long ldb, float* C,
         long ldc, const Epi& e, long kps, int splits, int partial) {
  if (M <= 0 || N <= 0) return;
  dim3 grid((unsigned)((M + BM - 1) / BM), (unsigned)((N + BN - 1) / BN), (unsigned)splits);
  FN_COUNT(1), k_sgemm<A_KM, B_KM><<<grid, NT, 0, s>>>(M, N, K, A, lda, B, ldb, C, ldc, e, kps, partial);
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
  long want = (2 * 152 + tiles - 1) / tiles;  // about two waves of CTAs
  long maxs = (K + 255) / 256;                 // at least 256 rows per split
  long sp = want < maxs ? want : maxs;
  if (sp < 1) sp = 1;
  if (sp > 64) sp = 64;
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

}  // namespace fn
