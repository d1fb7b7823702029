// KFAC pieces (the optimiser the paper credits for FermiNet's accuracy, Sec. 1;
// Martens and Grosse 2015): the transposed row matrices whose Gram products
// (tensor cores) give the Kronecker factors, squared column sums for the
// diagonal envelope block, the normalisation of the factor sums, a batched
// FP64 Gauss-Jordan inversion of the damped factors and the gather / scatter
// of layer gradients as [W b] matrices.
#include <cuda_bf16.h>

#include "fn_internal.cuh"

namespace fn {
namespace {

constexpr int TT = 32;

// out[c][r] (c < cols, r < ld_out): the KFAC input row r (see KfacRows).
__global__ void k_kfac_rows(KfacRows a, __nv_bfloat16* __restrict__ hi, __nv_bfloat16* __restrict__ lo,
                            long ld_out) {
  __shared__ __nv_bfloat16 th[TT][TT + 2], tl[TT][TT + 2];
  const long r0 = (long)blockIdx.x * TT, c0 = (long)blockIdx.y * TT;
  const __nv_bfloat16 z = __float2bfloat16_rn(0.f), one = __float2bfloat16_rn(1.f);
  for (int i = threadIdx.y; i < TT; i += blockDim.y) {
    const long r = r0 + i, c = c0 + threadIdx.x;
    __nv_bfloat16 vh = z, vl = z;
    const bool live = r < a.rows && c < a.cols && (a.spin < 0 || ((int)(r % a.n) < a.n_up) == (a.spin == 0));
    if (live) {
      if (c == a.cols - 1) {
        vh = one;
      } else {
        for (int sgi = 0; sgi < a.nseg; ++sgi) {
          const KfacRows::Seg& sg = a.seg[sgi];
          if (c >= sg.col0 && c < sg.col0 + sg.ncols) {
            const long rr = r / sg.row_div;
            const long ix = rr * sg.ld + (c - sg.col0);
            vh = sg.hi[ix];
            if (sg.lo) vl = sg.lo[ix];
          }
        }
      }
    }
    th[i][threadIdx.x] = vh;
    tl[i][threadIdx.x] = vl;
  }
  __syncthreads();
  for (int i = threadIdx.y; i < TT; i += blockDim.y) {
    const long c = c0 + i, r = r0 + threadIdx.x;
    if (c < a.cols && r < ld_out) {
      hi[c * ld_out + r] = th[threadIdx.x][i];
      if (lo) lo[c * ld_out + r] = tl[threadIdx.x][i];
    }
  }
}

// out[c] += sum_r X[r][c]^2 in FP64 (a thread per column).
__global__ void k_colsq_accum(const float* __restrict__ X, long rows, long cols, long ldx, double* __restrict__ out) {
  const long c = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= cols) return;
  double s = 0.0;
  for (long r = 0; r < rows; ++r) {
    const double v = X[r * ldx + c];
    s += v * v;
  }
  out[c] += s;
}

// Two-electron input factors: the bias row was summed on its own; mirror it
// into the bias column and put the row count in the corner (raw sums).
__global__ void k_kfac_mirror(double* __restrict__ F, const KfacBlock* __restrict__ blk, int nblk) {
  const int b = blockIdx.y;
  if (b >= nblk) return;
  const KfacBlock kb = blk[b];
  if (!kb.mirror_bias || kb.diag) return;
  const long d = kb.dim;
  double* M = F + kb.off;
  for (long r = (long)blockIdx.x * blockDim.x + threadIdx.x; r < d; r += (long)gridDim.x * blockDim.x)
    M[r * d + d - 1] = r == d - 1 ? kb.count : M[(d - 1) * d + r];
}

// Factor sums -> averages.
__global__ void k_kfac_scale(double* __restrict__ F, const KfacBlock* __restrict__ blk, int nblk) {
  const int b = blockIdx.y;
  if (b >= nblk) return;
  const KfacBlock kb = blk[b];
  const long tot = kb.diag ? kb.dim : kb.dim * kb.dim;
  double* M = F + kb.off;
  for (long i = (long)blockIdx.x * blockDim.x + threadIdx.x; i < tot; i += (long)gridDim.x * blockDim.x)
    M[i] *= kb.scale;
}

// One Gauss-Jordan pivot step k of every listed matrix, from src to dst (the
// two copies alternate, so no element is read after it is written):
//   p = a_kk; row k / p; every other row i minus a_ik times the new row k;
// column k becomes that of the inverse (1 / p on the pivot, -a_ik / p else).
// The matrices are damped symmetric positive definite factors, so no pivoting.
__global__ void k_gj_step(const double* __restrict__ src, double* __restrict__ dst, const KfacBlock* __restrict__ blk,
                          int nblk, int k) {
  const int b = blockIdx.y;
  if (b >= nblk) return;
  const KfacBlock kb = blk[b];
  const long d = kb.dim;
  if (kb.diag || k >= d) return;
  const double* a = src + kb.woff;
  double* o = dst + kb.woff;
  const double p = a[(long)k * d + k];
  for (long t = (long)blockIdx.x * blockDim.x + threadIdx.x; t < d * d; t += (long)gridDim.x * blockDim.x) {
    const long i = t / d, j = t % d;
    double v;
    if (i == k) v = (j == k) ? 1.0 / p : a[k * d + j] / p;
    else if (j == k) v = -a[i * d + k] / p;
    else v = a[i * d + j] - a[i * d + k] * a[k * d + j] / p;
    o[t] = v;
  }
}

// Damped copies: W[i][j] = F[i][j] + (i == j ? gamma : 0).
__global__ void k_damp_copy(const double* __restrict__ F, double* __restrict__ W, const KfacBlock* __restrict__ blk,
                            int nblk, double gamma) {
  const int b = blockIdx.y;
  if (b >= nblk) return;
  const KfacBlock kb = blk[b];
  if (kb.diag) return;
  const long d = kb.dim;
  for (long t = (long)blockIdx.x * blockDim.x + threadIdx.x; t < d * d; t += (long)gridDim.x * blockDim.x)
    W[kb.woff + t] = F[kb.off + t] + ((t / d == t % d) ? gamma : 0.0);
}

__global__ void k_to_float(const double* __restrict__ a, float* __restrict__ b, long n) {
  const long i = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) b[i] = (float)a[i];
}

// M[r][c] = c < cols - 1 ? g[w_off + r * (cols - 1) + c] : g[b_off + r]
__global__ void k_gather_wb(const float* __restrict__ g, long w_off, long b_off, long rows, long cols,
                            float* __restrict__ M) {
  const long t = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= rows * cols) return;
  const long r = t / cols, c = t % cols;
  M[t] = c < cols - 1 ? g[w_off + r * (cols - 1) + c] : g[b_off + r];
}

__global__ void k_scatter_wb(const float* __restrict__ M, long w_off, long b_off, long rows, long cols,
                             float* __restrict__ g) {
  const long t = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= rows * cols) return;
  const long r = t / cols, c = t % cols;
  if (c < cols - 1) g[w_off + r * (cols - 1) + c] = M[t];
  else g[b_off + r] = M[t];
}

__global__ void k_diag_precond(const float* __restrict__ g, const double* __restrict__ D, long n, double lambda,
                               float* __restrict__ out) {
  const long i = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) out[i] = (float)((double)g[i] / (D[i] + lambda));
}

inline unsigned nb(long n, int bs) { return (unsigned)((n + bs - 1) / bs); }

}  // namespace

void launch_kfac_rows(cudaStream_t s, const KfacRows& a, __nv_bfloat16* hi, __nv_bfloat16* lo, long ld_out) {
  if (a.cols <= 0 || ld_out <= 0) return;
  dim3 grid(nb(ld_out, TT), nb(a.cols, TT));
  FN_COUNT(1), k_kfac_rows<<<grid, dim3(TT, 8), 0, s>>>(a, hi, lo, ld_out);
}

void launch_colsq_accum(cudaStream_t s, const float* X, long rows, long cols, long ldx, double* out) {
  if (cols > 0) FN_COUNT(1), k_colsq_accum<<<nb(cols, 256), 256, 0, s>>>(X, rows, cols, ldx, out);
}

void launch_kfac_finalize(cudaStream_t s, double* F, const KfacBlock* d_blk, int nblk) {
  if (nblk <= 0) return;
  FN_COUNT(1), k_kfac_mirror<<<dim3(1, nblk), 256, 0, s>>>(F, d_blk, nblk);
  FN_COUNT(1), k_kfac_scale<<<dim3(64, nblk), 256, 0, s>>>(F, d_blk, nblk);
}

void launch_kfac_invert(cudaStream_t s, const double* F, const KfacBlock* d_blk, int nblk, int max_dim, double gamma,
                        double* w0, double* w1) {
  if (nblk <= 0) return;
  FN_COUNT(1), k_damp_copy<<<dim3(64, nblk), 256, 0, s>>>(F, w0, d_blk, nblk, gamma);
  for (int k = 0; k < max_dim; ++k)
    FN_COUNT(1), k_gj_step<<<dim3(64, nblk), 256, 0, s>>>(k % 2 ? w1 : w0, k % 2 ? w0 : w1, d_blk, nblk, k);
}

void launch_to_float(cudaStream_t s, const double* a, float* b, long n) {
  if (n > 0) FN_COUNT(1), k_to_float<<<nb(n, 256), 256, 0, s>>>(a, b, n);
}

void launch_gather_wb(cudaStream_t s, const float* g, long w_off, long b_off, long rows, long cols, float* M) {
  if (rows * cols > 0) FN_COUNT(1), k_gather_wb<<<nb(rows * cols, 256), 256, 0, s>>>(g, w_off, b_off, rows, cols, M);
}

void launch_scatter_wb(cudaStream_t s, const float* M, long w_off, long b_off, long rows, long cols, float* g) {
  if (rows * cols > 0)
    FN_COUNT(1), k_scatter_wb<<<nb(rows * cols, 256), 256, 0, s>>>(M, w_off, b_off, rows, cols, g);
}

void launch_diag_precond(cudaStream_t s, const float* g, const double* D, long n, double lambda, float* out) {
  if (n > 0) FN_COUNT(1), k_diag_precond<<<nb(n, 256), 256, 0, s>>>(g, D, n, lambda, out);
}

}  // namespace fn
