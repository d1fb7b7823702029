// Per-walker combination of the determinants into log|psi| and the local
// energy, the Coulomb terms, Gaussian Metropolis moves and the FP64 batch
// reductions of the VMC gradient.
#include <math.h>

#include <algorithm>

#include "fn_internal.cuh"

namespace fn {
namespace {

constexpr unsigned FULL = 0xffffffffu;

__device__ __forceinline__ int geo_of(const Geo& g, long wg) { return g.geo ? g.geo[wg] : 0; }

__device__ __forceinline__ double warp_sum_d(double v) {
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(FULL, v, off);
  return v;
}

// One warp per walker.
//   psi = sum_k s_k exp(l_k),  l_k = log|det A^{k up}| + log|det A^{k down}|   (Eq. 3)
//   w_k = psi_k / psi
//   T   = -1/2 sum_k w_k (lap l_k + |grad l_k|^2)  = -1/2 (lap psi) / psi
//   V   = sum_{i<j} 1/r_ij - sum_{i,I} Z_I / r_iI + E_nn                      (Eq. 1)
__global__ void k_combine(const float* __restrict__ logdet, const float* __restrict__ sign,
                          const float* __restrict__ dgrad, const float* __restrict__ dlap,
                          const float* __restrict__ x, long Bc, long w0, int n, int K, int N, Geo g, int tangent,
                          float* logpsi, float* psign, float* eloc, float* kinetic, float* wdet,
                          unsigned* status) {
  const int lane = threadIdx.x & 31;
  const long w = (long)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  if (w >= Bc) return;
  // log-sum-exp over determinants
  float lmax = -INFINITY;
  for (int k = lane; k < K; k += 32) {
    long b = (w * K + k) * 2;
    float sk = sign[b] * sign[b + 1];
    float lk = logdet[b] + logdet[b + 1];
    if (sk != 0.f) lmax = fmaxf(lmax, lk);
  }
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) lmax = fmaxf(lmax, __shfl_xor_sync(FULL, lmax, off));
  double acc = 0.0;
  for (int k = lane; k < K; k += 32) {
    long b = (w * K + k) * 2;
    float sk = sign[b] * sign[b + 1];
    if (sk != 0.f) acc += (double)sk * exp((double)(logdet[b] + logdet[b + 1]) - (double)lmax);
  }
  acc = warp_sum_d(acc);
  const float sp = acc > 0.0 ? 1.f : (acc < 0.0 ? -1.f : 0.f);
  const double lp = acc == 0.0 ? -INFINITY : (double)lmax + log(fabs(acc));
  if (lane == 0) {
    if (logpsi) logpsi[w] = (float)lp;
    if (psign) psign[w] = sp;
  }
  if (wdet) {
    for (int k = lane; k < K; k += 32) {
      long b = (w * K + k) * 2;
      float sk = sign[b] * sign[b + 1];
      wdet[w * K + k] = (sk != 0.f && sp != 0.f)
                            ? (float)((double)(sk * sp) * exp((double)(logdet[b] + logdet[b + 1]) - lp))
                            : 0.f;
    }
  }
  if (!tangent) {
    if (lane == 0 && !(isfinite(lp))) atomicOr(status, (unsigned)ST_NONFINITE);
    return;
  }
  const int n3 = 3 * n;
  double T = 0.0;
  for (int k = 0; k < K; ++k) {
    long b = (w * K + k) * 2;
    float sk = sign[b] * sign[b + 1];
    if (sk == 0.f || sp == 0.f) continue;
    double wk = (double)(sk * sp) * exp((double)(logdet[b] + logdet[b + 1]) - lp);
    const float* g0 = dgrad + b * n3;
    const float* g1 = g0 + n3;
    double sq = 0.0;
    for (int c = lane; c < n3; c += 32) {
      double gc = (double)g0[c] + (double)g1[c];
      sq += gc * gc;
    }
    sq = warp_sum_d(sq);
    T += wk * ((double)dlap[b] + (double)dlap[b + 1] + sq);
  }
  T *= -0.5;
  // Coulomb
  const int gi = geo_of(g, w0 + w);
  const float* R = g.R + (long)gi * N * 3;
  const float* Z = g.Z + (long)gi * N;
  const float* xw = x + w * n3;
  double V = 0.0;
  const int npair = n * (n - 1) / 2;
  for (int p = lane; p < npair; p += 32) {
    // p -> (i, j), i > j
    int i = (int)((1.0 + sqrt(1.0 + 8.0 * p)) * 0.5);
    while (i * (i - 1) / 2 > p) --i;
    while ((i + 1) * i / 2 <= p) ++i;
    int j = p - i * (i - 1) / 2;
    double d0 = (double)xw[3 * i] - xw[3 * j], d1 = (double)xw[3 * i + 1] - xw[3 * j + 1],
           d2 = (double)xw[3 * i + 2] - xw[3 * j + 2];
    V += 1.0 / sqrt(d0 * d0 + d1 * d1 + d2 * d2);
  }
  for (int p = lane; p < n * N; p += 32) {
    int i = p / N, I = p % N;
    double d0 = (double)xw[3 * i] - R[3 * I], d1 = (double)xw[3 * i + 1] - R[3 * I + 1],
           d2 = (double)xw[3 * i + 2] - R[3 * I + 2];
    V -= (double)Z[I] / sqrt(d0 * d0 + d1 * d1 + d2 * d2);
  }
  V = warp_sum_d(V) + g.Enn[gi];
  if (lane == 0) {
    double E = T + V;
    eloc[w] = (float)E;
    if (kinetic) kinetic[w] = (float)T;
    if (!isfinite(E) || !isfinite(lp)) atomicOr(status, (unsigned)ST_NONFINITE);
  }
}

// Philox4x32-10 (Salmon et al., SC'11).
__device__ __forceinline__ uint4 philox10(uint4 c, uint2 k) {
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    if (r > 0) {
      k.x += 0x9E3779B9u;
      k.y += 0xBB67AE85u;
    }
    const unsigned lo0 = 0xD2511F53u * c.x, hi0 = __umulhi(0xD2511F53u, c.x);
    const unsigned lo1 = 0xCD9E8D57u * c.z, hi1 = __umulhi(0xCD9E8D57u, c.z);
    c = make_uint4(hi1 ^ c.y ^ k.x, lo1, hi0 ^ c.w ^ k.y, lo0);
  }
  return c;
}

__device__ __forceinline__ float u01(unsigned v) { return ((float)(v >> 9) + 0.5f) * (1.f / 8388608.f); }

__device__ __forceinline__ void box_muller(unsigned a, unsigned b, float& z0, float& z1) {
  float r = sqrtf(-2.f * logf(u01(a)));
  float sn, cs;
  sincospif(2.f * u01(b), &sn, &cs);
  z0 = r * cs;
  z1 = r * sn;
}

__global__ void k_propose(const float* __restrict__ x, float* __restrict__ xp, long B, int n3, float width,
                          uint64_t seed, uint64_t t, const uint64_t* __restrict__ dctr,
                          const float* __restrict__ dwidth) {
  if (dctr) t += *dctr;  // graph replays read the step's base counter from device memory
  if (dwidth) width = *dwidth;  // adaptive width, kept in device memory
  const int nb = (n3 + 3) / 4;
  long idx = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= B * nb) return;
  long w = idx / nb;
  int b = (int)(idx % nb);
  uint4 o = philox10(make_uint4((unsigned)w, (unsigned)b, (unsigned)t, (unsigned)(t >> 32)),
                     make_uint2((unsigned)seed, (unsigned)(seed >> 32)));
  float z[4];
  box_muller(o.x, o.y, z[0], z[1]);
  box_muller(o.z, o.w, z[2], z[3]);
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    int c = 4 * b + q;
    if (c < n3) xp[w * n3 + c] = fmaf(width, z[q], x[w * n3 + c]);
  }
}

__global__ void k_accept(float* __restrict__ x, const float* __restrict__ xp, float* __restrict__ logpsi,
                         const float* __restrict__ lpp, long B, int n3, uint64_t seed, uint64_t t, int* accepted,
                         const uint64_t* __restrict__ dctr) {
  if (dctr) t += *dctr;
  long w = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (w >= B) return;
  uint4 o = philox10(make_uint4((unsigned)w, 0xFFFFFFFFu, (unsigned)t, (unsigned)(t >> 32)),
                     make_uint2((unsigned)seed, (unsigned)(seed >> 32)));
  float lu = logf(u01(o.x));
  float crit = 2.f * (lpp[w] - logpsi[w]);
  if (lu < crit) {
    for (int c = 0; c < n3; ++c) x[w * n3 + c] = xp[w * n3 + c];
    logpsi[w] = lpp[w];
    if (accepted) accepted[w] += 1;
  }
}

// One block per geometry: deterministic tree sum in FP64; the mean when
// `mean` is set, else the sum.
__global__ void k_emean(const float* __restrict__ eloc, const long* __restrict__ off, const long* __restrict__ cnt,
                        long B1, int mean, double* emean) {
  __shared__ double sh[256];
  const int g = blockIdx.x;
  const long o = B1 >= 0 ? 0 : off[g], c = B1 >= 0 ? B1 : cnt[g];
  double s = 0.0;
  for (long i = threadIdx.x; i < c; i += 256) s += (double)eloc[o + i];
  sh[threadIdx.x] = s;
  __syncthreads();
  for (int st = 128; st > 0; st >>= 1) {
    if (threadIdx.x < st) sh[threadIdx.x] += sh[threadIdx.x + st];
    __syncthreads();
  }
  if (threadIdx.x == 0) emean[g] = !mean ? sh[0] : (c > 0 ? sh[0] / (double)c : 0.0);
}

__global__ void k_seeds(const float* __restrict__ eloc, long B, const int* __restrict__ geo,
                        const double* __restrict__ emean, const long* __restrict__ cnt, long B1, float* seeds) {
  long w = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (w >= B) return;
  int g = geo ? geo[w] : 0;
  double c = B1 >= 0 ? (double)B1 : (double)cnt[g];
  seeds[w] = (float)(2.0 * ((double)eloc[w] - emean[g]) / c);
}

// Seeds of the replica form: the energy sum and the walker count of every
// geometry over the whole batch (all replicas) give its mean in FP64; threads
// w < G also store that mean.
__global__ void k_seeds_given(const float* __restrict__ eloc, long B, const int* __restrict__ geo,
                              const double* __restrict__ sums, const double* __restrict__ count, int G,
                              double* __restrict__ emean, float* seeds) {
  long w = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (emean && w < G) emean[w] = count[w] > 0.0 ? sums[w] / count[w] : 0.0;
  if (w >= B) return;
  int g = geo ? geo[w] : 0;
  const double m = sums[g] / count[g];
  seeds[w] = (float)(2.0 * ((double)eloc[w] - m) / count[g]);
}

// Orderable unsigned key of a float (a < b  <=>  key(a) < key(b) for non-NaN).
__device__ __forceinline__ unsigned fkey(float f) {
  const unsigned u = __float_as_uint(f);
  return (u & 0x80000000u) ? ~u : (u | 0x80000000u);
}
__device__ __forceinline__ float fkey_inv(unsigned k) {
  return __uint_as_float((k & 0x80000000u) ? (k & 0x7FFFFFFFu) : ~k);
}

constexpr int kClipThreads = 512;

// Block sum of one double per thread (thread 0 gets the total).
__device__ double block_sum(double v, double* sh) {
  sh[threadIdx.x] = v;
  __syncthreads();
  for (int st = kClipThreads / 2; st > 0; st >>= 1) {
    if (threadIdx.x < st) sh[threadIdx.x] += sh[threadIdx.x + st];
    __syncthreads();
  }
  const double r = sh[0];
  __syncthreads();
  return r;
}

// Clipping statistics of one geometry per block: the two middle order
// statistics by a radix select over the orderable keys (four 8-bit passes,
// both ranks at once), the median m, tv = mean |E_L - m| and the mean of the
// clipped energies, all in FP64: stats[3 g + {0, 1, 2}].
__global__ void __launch_bounds__(kClipThreads) k_clip_stats(const float* __restrict__ eloc,
                                                             const long* __restrict__ off,
                                                             const long* __restrict__ cnt, long B1, double scale,
                                                             double* __restrict__ stats) {
  __shared__ unsigned hist[2][256];
  __shared__ unsigned pre[2], rank[2];
  __shared__ double sh[kClipThreads];
  const int g = blockIdx.x;
  const long o = B1 >= 0 ? 0 : off[g], c = B1 >= 0 ? B1 : cnt[g];
  if (c <= 0) {
    if (threadIdx.x == 0) stats[3 * g] = stats[3 * g + 1] = stats[3 * g + 2] = 0.0;
    return;
  }
  if (threadIdx.x == 0) {
    pre[0] = pre[1] = 0u;
    rank[0] = (unsigned)((c - 1) / 2);
    rank[1] = (unsigned)(c / 2);
  }
  unsigned mask = 0u;
  for (int shift = 24; shift >= 0; shift -= 8) {
    for (int i = threadIdx.x; i < 512; i += kClipThreads) (&hist[0][0])[i] = 0u;
    __syncthreads();
    const unsigned p0 = pre[0], p1 = pre[1];
    for (long i = threadIdx.x; i < c; i += kClipThreads) {
      const unsigned k = fkey(eloc[o + i]);
      const unsigned b = (k >> shift) & 255u;
      if ((k & mask) == p0) atomicAdd(&hist[0][b], 1u);
      if ((k & mask) == p1) atomicAdd(&hist[1][b], 1u);
    }
    __syncthreads();
    if (threadIdx.x < 2) {
      const int s = threadIdx.x;
      unsigned r = rank[s], b = 0;
      while (b < 255u && hist[s][b] <= r) {  // the rank lies in a later bucket
        r -= hist[s][b];
        ++b;
      }
      rank[s] = r;
      pre[s] |= b << shift;
    }
    mask |= 255u << shift;
    __syncthreads();
  }
  const double m = 0.5 * ((double)fkey_inv(pre[0]) + (double)fkey_inv(pre[1]));
  double a = 0.0;
  for (long i = threadIdx.x; i < c; i += kClipThreads) a += fabs((double)eloc[o + i] - m);
  const double tv = block_sum(a, sh) / (double)c;
  const double lo = m - scale * tv, hi = m + scale * tv;
  double cs = 0.0;
  for (long i = threadIdx.x; i < c; i += kClipThreads) cs += fmin(fmax((double)eloc[o + i], lo), hi);
  const double cbar = block_sum(cs, sh) / (double)c;
  if (threadIdx.x == 0) {
    stats[3 * g] = m;
    stats[3 * g + 1] = tv;
    stats[3 * g + 2] = cbar;
  }
}

__global__ void k_seeds_clip(const float* __restrict__ eloc, long B, const int* __restrict__ geo,
                             const double* __restrict__ stats, const long* __restrict__ cnt, long B1, double scale,
                             float* seeds) {
  long w = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (w >= B) return;
  const int g = geo ? geo[w] : 0;
  const double c = B1 >= 0 ? (double)B1 : (double)cnt[g];
  const double m = stats[3 * g], tv = stats[3 * g + 1], cbar = stats[3 * g + 2];
  const double e = fmin(fmax((double)eloc[w], m - scale * tv), m + scale * tv);
  seeds[w] = (float)(2.0 * (e - cbar) / c);
}

// Proposal-width adaptation from the acceptance counts of the last moves.
__global__ void __launch_bounds__(kClipThreads) k_adapt_width(const int* __restrict__ accepted, long B,
                                                              int n_steps, float* width, double lo, double hi,
                                                              double factor) {
  __shared__ double sh[kClipThreads];
  double a = 0.0;
  for (long i = threadIdx.x; i < B; i += kClipThreads) a += (double)accepted[i];
  const double tot = block_sum(a, sh);
  if (threadIdx.x == 0 && B > 0 && n_steps > 0) {
    const double p = tot / ((double)B * (double)n_steps);
    const double w = (double)*width;
    if (p > hi) *width = (float)(w * factor);
    else if (p < lo) *width = (float)(w / factor);
  }
}

__global__ void k_d2f(const double* a, float* b, long n) {
  long i = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) b[i] = (float)a[i];
}
__global__ void k_fill(float* p, float v, long n) {
  long i = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) p[i] = v;
}
__global__ void k_zero_d(double* p, long n) {
  long i = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) p[i] = 0.0;
}

inline unsigned nblk(long tot, int bs) { return (unsigned)((tot + bs - 1) / bs); }

}  // namespace

void launch_combine(cudaStream_t s, const float* logdet, const float* sign, const float* dgrad, const float* dlap,
                    const float* x, long Bc, long w0, int n, int K, int N, Geo g, bool tangent, float* logpsi,
                    float* psign, float* eloc, float* kinetic, float* wdet, unsigned* status) {
  if (Bc <= 0) return;
  FN_COUNT(1), k_combine<<<nblk(Bc, 4), 128, 0, s>>>(logdet, sign, dgrad, dlap, x, Bc, w0, n, K, N, g, tangent ? 1 : 0, logpsi,
                                        psign, eloc, kinetic, wdet, status);
}

void launch_propose(cudaStream_t s, const float* x, float* xp, long B, int n3, float width, uint64_t seed,
                    uint64_t t, const uint64_t* dctr, const float* dwidth) {
  long tot = B * ((n3 + 3) / 4);
  if (tot > 0) FN_COUNT(1), k_propose<<<nblk(tot, 256), 256, 0, s>>>(x, xp, B, n3, width, seed, t, dctr, dwidth);
}

void launch_accept(cudaStream_t s, float* x, const float* xp, float* logpsi, const float* lp_prop, long B, int n3,
                   uint64_t seed, uint64_t t, int* accepted, const uint64_t* dctr) {
  if (B > 0)
    FN_COUNT(1), k_accept<<<nblk(B, 256), 256, 0, s>>>(x, xp, logpsi, lp_prop, B, n3, seed, t, accepted, dctr);
}

__global__ void k_set_u64(uint64_t* p, uint64_t v) { *p = v; }

void launch_set_u64(cudaStream_t s, uint64_t* p, uint64_t v) { FN_COUNT(1), k_set_u64<<<1, 1, 0, s>>>(p, v); }

void launch_emean(cudaStream_t s, const float* eloc, int G, const long* d_off, const long* d_cnt, long B1,
                  double* emean) {
  if (G > 0) FN_COUNT(1), k_emean<<<G, 256, 0, s>>>(eloc, d_off, d_cnt, B1, 1, emean);
}

void launch_esum(cudaStream_t s, const float* eloc, int G, const long* d_off, const long* d_cnt, long B1,
                 double* sums) {
  if (G > 0) FN_COUNT(1), k_emean<<<G, 256, 0, s>>>(eloc, d_off, d_cnt, B1, 0, sums);
}

void launch_seeds_given(cudaStream_t s, const float* eloc, long B, const int* geo, const double* sums,
                        const double* count, int G, double* emean, float* seeds) {
  const long n = std::max<long>(B, emean ? G : 0);
  if (n > 0) FN_COUNT(1), k_seeds_given<<<nblk(n, 256), 256, 0, s>>>(eloc, B, geo, sums, count, G, emean, seeds);
}

void launch_seeds(cudaStream_t s, const float* eloc, long B, const int* geo, const double* emean, const long* d_cnt,
                  long B1, float* seeds) {
  if (B > 0) FN_COUNT(1), k_seeds<<<nblk(B, 256), 256, 0, s>>>(eloc, B, geo, emean, d_cnt, B1, seeds);
}

void launch_clip_seeds(cudaStream_t s, const float* eloc, long B, const int* geo, int G, const long* d_off,
                       const long* d_cnt, long B1, double scale, double* stats, float* seeds) {
  if (G > 0) FN_COUNT(1), k_clip_stats<<<G, kClipThreads, 0, s>>>(eloc, d_off, d_cnt, B1, scale, stats);
  if (B > 0) FN_COUNT(1), k_seeds_clip<<<nblk(B, 256), 256, 0, s>>>(eloc, B, geo, stats, d_cnt, B1, scale, seeds);
}

void launch_adapt_width(cudaStream_t s, const int* accepted, long B, int n_steps, float* width, double lo,
                        double hi, double factor) {
  FN_COUNT(1), k_adapt_width<<<1, kClipThreads, 0, s>>>(accepted, B, n_steps, width, lo, hi, factor);
}

void launch_d2f(cudaStream_t s, const double* a, float* b, long n) {
  if (n > 0) FN_COUNT(1), k_d2f<<<nblk(n, 256), 256, 0, s>>>(a, b, n);
}
void launch_fill(cudaStream_t s, float* p, float v, long n) {
  if (n > 0) FN_COUNT(1), k_fill<<<nblk(n, 256), 256, 0, s>>>(p, v, n);
}
void launch_zero_d(cudaStream_t s, double* p, long n) {
  if (n > 0) FN_COUNT(1), k_zero_d<<<nblk(n, 256), 256, 0, s>>>(p, n);
}

}  // namespace fn
