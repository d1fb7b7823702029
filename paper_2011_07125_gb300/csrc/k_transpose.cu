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

// 64 x 64 tiles moving pairs of elements per access (8-byte FP32 pairs in,
// 4-byte BF16 pairs out): the same values as k_t_split / k_t_bf16 with half
// the load and store instructions and 128-byte warp stores.  Needs even ld_src
// and ld_dst and sources aligned to a pair.
constexpr int T2 = 64;

__global__ void k_t_split2(const float* __restrict__ src, long ld_src, long rows, long cols,
                           __nv_bfloat16* __restrict__ hi, __nv_bfloat16* __restrict__ lo, long ld_dst) {
  __shared__ float t[T2][T2 + 1];
  const long r0 = (long)blockIdx.x * T2, c0 = (long)blockIdx.y * T2;
  const int tx = threadIdx.x, ty = threadIdx.y;
  for (int i = ty; i < T2; i += 8) {
    const long r = r0 + i, c = c0 + 2 * tx;
    float2 v = make_float2(0.f, 0.f);
    if (r < rows) {
      if (c + 1 < cols) v = *reinterpret_cast<const float2*>(src + r * ld_src + c);
      else if (c < cols) v.x = src[r * ld_src + c];
    }
    t[i][2 * tx] = v.x;
    t[i][2 * tx + 1] = v.y;
  }
  __syncthreads();
  for (int j = ty; j < T2; j += 8) {
    const long c = c0 + j, r = r0 + 2 * tx;
    if (c < cols && r < ld_dst) {  // ld_dst even: r + 1 < ld_dst too
      const float v0 = t[2 * tx][j], v1 = t[2 * tx + 1][j];
      const __nv_bfloat162 h = __floats2bfloat162_rn(v0, v1);
      *reinterpret_cast<__nv_bfloat162*>(hi + c * ld_dst + r) = h;
      if (lo)
        *reinterpret_cast<__nv_bfloat162*>(lo + c * ld_dst + r) =
            __floats2bfloat162_rn(v0 - __low2float(h), v1 - __high2float(h));
    }
  }
}

__global__ void k_t_bf16_2(const __nv_bfloat16* __restrict__ shi, const __nv_bfloat16* __restrict__ slo, long ld_src,
                           long rows, long cols, __nv_bfloat16* __restrict__ hi, __nv_bfloat16* __restrict__ lo,
                           long ld_dst) {
  __shared__ __nv_bfloat16 th[T2][T2 + 2], tl[T2][T2 + 2];
  const long r0 = (long)blockIdx.x * T2, c0 = (long)blockIdx.y * T2;
  const int tx = threadIdx.x, ty = threadIdx.y;
  const __nv_bfloat16 z = __float2bfloat16_rn(0.f);
  for (int i = ty; i < T2; i += 8) {
    const long r = r0 + i, c = c0 + 2 * tx;
    __nv_bfloat162 h = __halves2bfloat162(z, z), l = h;
    if (r < rows) {
      if (c + 1 < cols) {
        h = *reinterpret_cast<const __nv_bfloat162*>(shi + r * ld_src + c);
        if (slo) l = *reinterpret_cast<const __nv_bfloat162*>(slo + r * ld_src + c);
      } else if (c < cols) {
        h.x = shi[r * ld_src + c];
        if (slo) l.x = slo[r * ld_src + c];
      }
    }
    th[i][2 * tx] = h.x;
    th[i][2 * tx + 1] = h.y;
    tl[i][2 * tx] = l.x;
    tl[i][2 * tx + 1] = l.y;
  }
  __syncthreads();
  for (int j = ty; j < T2; j += 8) {
    const long c = c0 + j, r = r0 + 2 * tx;
    if (c < cols && r < ld_dst) {
      *reinterpret_cast<__nv_bfloat162*>(hi + c * ld_dst + r) = __halves2bfloat162(th[2 * tx][j], th[2 * tx + 1][j]);
      if (lo)
        *reinterpret_cast<__nv_bfloat162*>(lo + c * ld_dst + r) = __halves2bfloat162(tl[2 * tx][j], tl[2 * tx + 1][j]);
    }
  }
}

}  // namespace

void launch_t_split(cudaStream_t s, const float* src, long ld_src, long rows, long cols, __nv_bfloat16* hi,
                    __nv_bfloat16* lo, long ld_dst) {
  if (cols <= 0 || ld_dst <= 0) return;
  if (ld_src % 2 == 0 && ld_dst % 2 == 0 && (uintptr_t)src % 8 == 0 && ((uintptr_t)hi | (uintptr_t)lo) % 4 == 0) {
    dim3 grid((unsigned)((ld_dst + T2 - 1) / T2), (unsigned)((cols + T2 - 1) / T2));
    FN_COUNT(1), k_t_split2<<<grid, dim3(32, 8), 0, s>>>(src, ld_src, rows, cols, hi, lo, ld_dst);
    return;
  }
  dim3 grid((unsigned)((ld_dst + TT - 1) / TT), (unsigned)((cols + TT - 1) / TT));
  FN_COUNT(1), k_t_split<<<grid, dim3(TT, 8), 0, s>>>(src, ld_src, rows, cols, hi, lo, ld_dst);
}

void launch_t_bf16(cudaStream_t s, const __nv_bfloat16* shi, const __nv_bfloat16* slo, long ld_src, long rows,
                   long cols, __nv_bfloat16* hi, __nv_bfloat16* lo, long ld_dst) {
  if (cols <= 0 || ld_dst <= 0) return;
  if (ld_src % 2 == 0 && ld_dst % 2 == 0 && ((uintptr_t)shi | (uintptr_t)slo | (uintptr_t)hi | (uintptr_t)lo) % 4 == 0) {
    dim3 grid((unsigned)((ld_dst + T2 - 1) / T2), (unsigned)((cols + T2 - 1) / T2));
    FN_COUNT(1), k_t_bf16_2<<<grid, dim3(32, 8), 0, s>>>(shi, slo, ld_src, rows, cols, hi, lo, ld_dst);
    return;
  }
  dim3 grid((unsigned)((ld_dst + TT - 1) / TT), (unsigned)((cols + TT - 1) / TT));
  FN_COUNT(1), k_t_bf16<<<grid, dim3(TT, 8), 0, s>>>(shi, slo, ld_src, rows, cols, hi, lo, ld_dst);
}

}  // namespace fn
