// Transposing BF16 hi + lo splits for the tensor-core adjoint: the weight
// gradients contract over activation rows, so both operands are needed with
// the rows contiguous (K-major); the backward-data products need the weights
// with the output features contiguous.
#include <cuda_bf16.h>

#include "fn_internal.cuh"

namespace fn {
namespace {

constexpr int TT = 32;

// dst[c][r] (c < cols, r < ld_dst) = split of src[r][c] for r < rows, zero for
// rows <= r < ld_dst.  FP32 source.
__global__ void k_t_split(const float* __restrict__ src, long ld_src, long rows, long cols,
                          __nv_bfloat16* __restrict__ hi, __nv_bfloat16* __restrict__ lo, long ld_dst) {
  __shared__ float t[TT][TT + 1];
  const long r0 = (long)blockIdx.x * TT, c0 = (long)blockIdx.y * TT;
  for (int i = threadIdx.y; i < TT; i += blockDim.y) {
    const long r = r0 + i, c = c0 + threadIdx.x;
    t[i][threadIdx.x] = (r < rows && c < cols) ? src[r * ld_src + c] : 0.f;
  }
  __syncthreads();
  for (int i = threadIdx.y; i < TT; i += blockDim.y) {
    const long c = c0 + i, r = r0 + threadIdx.x;
    if (c < cols && r < ld_dst) {
      const float v = t[threadIdx.x][i];
      const __nv_bfloat16 h = __float2bfloat16_rn(v);
      hi[c * ld_dst + r] = h;
      if (lo) lo[c * ld_dst + r] = __float2bfloat16_rn(v - __bfloat162float(h));
    }
  }
}

// The same for a source already split into BF16 hi + lo (each part moved as
// it is).
__global__ void k_t_bf16(const __nv_bfloat16* __restrict__ shi, const __nv_bfloat16* __restrict__ slo, long ld_src,
                         long rows, long cols, __nv_bfloat16* __restrict__ hi, __nv_bfloat16* __restrict__ lo,
                         long ld_dst) {
  __shared__ __nv_bfloat16 th[TT][TT + 2], tl[TT][TT + 2];
  const long r0 = (long)blockIdx.x * TT, c0 = (long)blockIdx.y * TT;
  const __nv_bfloat16 z = __float2bfloat16_rn(0.f);
  for (int i = threadIdx.y; i < TT; i += blockDim.y) {
    const long r = r0 + i, c = c0 + threadIdx.x;
    const bool in = r < rows && c < cols;
    th[i][threadIdx.x] = in ? shi[r * ld_src + c] : z;
    tl[i][threadIdx.x] = (in && slo) ? slo[r * ld_src + c] : z;
  }
  __syncthreads();
  for (int i = threadIdx.y; i < TT; i += blockDim.y) {
    const long c = c0 + i, r = r0 + threadIdx.x;
    if (c < cols && r < ld_dst) {
      hi[c * ld_dst + r] = th[threadIdx.x][i];
      if (lo) lo[c * ld_dst + r] = tl[threadIdx.x][i];
    }
  }
}

}  // namespace

void launch_t_split(cudaStream_t s, const float* src, long ld_src, long rows, long cols, __nv_bfloat16* hi,
                    __nv_bfloat16* lo, long ld_dst) {
  if (cols <= 0 || ld_dst <= 0) return;
  dim3 grid((unsigned)((ld_dst + TT - 1) / TT), (unsigned)((cols + TT - 1) / TT));
  FN_COUNT(1), k_t_split<<<grid, dim3(TT, 8), 0, s>>>(src, ld_src, rows, cols, hi, lo, ld_dst);
}

void launch_t_bf16(cudaStream_t s, const __nv_bfloat16* shi, const __nv_bfloat16* slo, long ld_src, long rows,
                   long cols, __nv_bfloat16* hi, __nv_bfloat16* lo, long ld_dst) {
  if (cols <= 0 || ld_dst <= 0) return;
  dim3 grid((unsigned)((ld_dst + TT - 1) / TT), (unsigned)((cols + TT - 1) / TT));
  FN_COUNT(1), k_t_bf16<<<grid, dim3(TT, 8), 0, s>>>(shi, slo, ld_src, rows, cols, hi, lo, ld_dst);
}

}  // namespace fn
