// Orbital matrices, envelopes and determinants (Eq. 3-4).
//
// For determinant k and spin s the n_s x n_s matrix is
//   A_ij = o_ij * e_ij,   o_ij = w^{ks}_i . h^L_j + g^{ks}_i   (orbital GEMM output)
//   e_ij = sum_m pi^{ks}_im exp(-|sigma^{ks}_im| |r_j - R_m|)  (isotropic envelope)
// Each matrix is inverted by one warp (Gauss-Jordan with partial pivoting, one
// row per lane, rows exchanged with shuffles), giving sign, log|det| and A^-1.
// In the tangent pass the block then forms, for every coordinate c,
//   d_c log|det A| = tr(A^-1 d_c A)
//   lap log|det A| = tr(A^-1 lap A) - sum_c tr((A^-1 d_c A)^2),
// with d_c A and lap A assembled from the orbital columns and the envelope
// derivatives (product rule; the envelope depends on r_j only).
#include <math.h>

#include <type_traits>

#include "fn_internal.cuh"

namespace fn {
namespace {

constexpr unsigned FULL = 0xffffffffu;

__device__ __forceinline__ int geo_of(const Geo& g, long wg) { return g.geo ? g.geo[wg] : 0; }

// Gauss-Jordan inversion of an n x n matrix (n <= NM <= 32) held one row per
// lane in a[]; b[] starts as the identity row of the lane and ends as the row
// of A^-1.  Lanes n..NM-1 hold identity padding rows.  All lanes end with the
// same logabs, sign and pivot extremes.  With INV false b[] is left alone
// (the determinant alone: no inverse rows are swapped or eliminated).
template <int NM, class T, int WIDTH = 32, bool INV = true>
__device__ __forceinline__ void warp_gj(T (&a)[NM], T (&b)[NM], int n, int lane, T& logabs, T& sgn, T& pmin,
                                        T& pmax, bool& sing, int nreal = 1 << 30) {
  logabs = T(0);
  sgn = T(1);
  pmin = T(INFINITY);
  pmax = T(0);
  sing = false;
#pragma unroll
  for (int k = 0; k < NM; ++k) {
    if (k >= n) break;
    T v = (lane >= k && lane < n) ? fabs(a[k]) : T(-1);
    int idx = lane;
#pragma unroll
    for (int off = WIDTH / 2; off > 0; off >>= 1) {
      T ov = __shfl_xor_sync(FULL, v, off, WIDTH);
      int oi = __shfl_xor_sync(FULL, idx, off, WIDTH);
      if (ov > v || (ov == v && oi < idx)) {
        v = ov;
        idx = oi;
      }
    }
    const int p = idx;
    // segments of one warp may differ in p: every lane takes part in the shuffles
    if (__any_sync(FULL, p != k)) {
      const int src = lane == k ? p : (lane == p ? k : lane);
#pragma unroll
      for (int c = 0; c < NM; ++c) {
        if (c >= k) a[c] = __shfl_sync(FULL, a[c], src, WIDTH);  // columns < k are eliminated
        if (INV) b[c] = __shfl_sync(FULL, b[c], src, WIDTH);
      }
      if (p != k) sgn = -sgn;
    }
    const T u = __shfl_sync(FULL, a[k], k, WIDTH);
    const T au = fabs(u);
    if (k < nreal) {  // padding pivots (identity rows) do not enter the ratio
      pmin = fmin(pmin, au);
      pmax = fmax(pmax, au);
    }
    if (!(au > T(0))) sing = true;
    // a singular segment keeps taking part in the shuffles (its results are
    // discarded); the warp stops once every segment is singular
    if (__all_sync(FULL, sing)) break;
    if (!sing) {
      logabs += log(au);
      if (u < T(0)) sgn = -sgn;
    }
    const T iu = sing ? T(0) : T(1) / u;
    const T fct = a[k];
#pragma unroll
    for (int c = 0; c < NM; ++c) {
      if (c >= k) {
        T rk = __shfl_sync(FULL, a[c], k, WIDTH) * iu;
        a[c] = (lane == k) ? rk : fma(-fct, rk, a[c]);
      }
      if (INV) {
        T rb = __shfl_sync(FULL, b[c], k, WIDTH) * iu;
        b[c] = (lane == k) ? rb : fma(-fct, rb, b[c]);
      }
    }
  }
}

// log|det| and sign of the n x n matrices held by the two 16-lane halves of a
// warp (row sl in lane sl of each half; rows n..15 unused), by LU with partial
// pivoting in FP32, without inverse rows.  Rows are never moved: the pivot of
// step k is the unused row with the largest |a_k| (one warp-wide max over
// 32-bit keys whose low 4 bits hold 15 - row, so ties go to the lower row), and
// the sign of the row permutation is counted from the rows already pivoted.
// The product of pivots is kept as mantissa and exponent (one log at the end).
// All lanes of a half end with the same results; padding rows (index >= nreal)
// do not enter the pivot extremes.  A pivot below the smallest normal float
// leaves the matrix to the FP64 redo (the pivot ratio flags it).
template <int NM>
__device__ __forceinline__ void warp_lu16(float (&a)[NM], int n, int sl, float& logabs, float& sgn, float& pmin,
                                          float& pmax, bool& sing, int nreal) {
  const int half = (threadIdx.x >> 4) & 1;
  const unsigned hbits = half ? 0xFFFF0000u : 0x0000FFFFu;
  bool pivoted = false;
  float mant = 1.f, s = 1.f;
  int expo = 0;
  pmin = INFINITY;
  pmax = 0.f;
  sing = false;
#pragma unroll
  for (int k = 0; k < NM; ++k) {
    if (k >= n) break;
    const unsigned cand = (!pivoted && sl < n)
                              ? ((__float_as_uint(fabsf(a[k])) & ~0xFu) | (unsigned)(15 - sl))
                              : 0u;
    const unsigned m0 = __reduce_max_sync(FULL, half ? 0u : cand);
    const unsigned m1 = __reduce_max_sync(FULL, half ? cand : 0u);
    const int p = 15 - (int)((half ? m1 : m0) & 0xFu);
    // rows pivoted before p with a larger index: inversions of the permutation
    const unsigned done = __ballot_sync(FULL, pivoted) & hbits;
    const unsigned above = (half ? (0xFFFF0000u << (p + 1)) : ((0xFFFFu << (p + 1)) & 0xFFFFu)) & done;
    if (__popc(above) & 1) s = -s;
    const float u = __shfl_sync(FULL, a[k], p, 16);
    const float au = fabsf(u);
    if (k < nreal) {
      pmin = fminf(pmin, au);
      pmax = fmaxf(pmax, au);
    }
    if (!(au > 0.f)) sing = true;
    if (u < 0.f) s = -s;
    // running product of |pivots| as mant * 2^expo
    mant *= sing ? 1.f : au;
    const unsigned mb = __float_as_uint(mant);
    expo += (int)((mb >> 23) & 0xFFu) - 127;
    mant = __uint_as_float((mb & 0x807FFFFFu) | 0x3F800000u);
    if (sl == p) pivoted = true;
    // the update of Gauss-Jordan: the pivot row is scaled first, so a column
    // equal to an earlier one eliminates to an exact zero
    const float iu = sing ? 0.f : 1.f / u;
    const float fct = pivoted ? 0.f : a[k];
#pragma unroll
    for (int c = 0; c < NM; ++c) {
      if (c > k) {
        const float rk = __shfl_sync(FULL, a[c], p, 16) * iu;
        a[c] = fmaf(-fct, rk, a[c]);
      }
    }
  }
  logabs = logf(mant) + (float)expo * 0.69314718055994531f;
  sgn = s;
}

struct MatId {
  long w;
  int k, s, ns, j0;
  long q0;
};

__device__ __forceinline__ MatId mat_id(long mat, const DetArgs& a) {
  MatId m;
  m.w = mat / (2 * a.K);
  int r = (int)(mat % (2 * a.K));
  m.k = r / 2;
  m.s = r % 2;
  m.ns = m.s == 0 ? a.n_up : a.n - a.n_up;
  m.j0 = m.s == 0 ? 0 : a.n_up;
  m.q0 = (m.s == 0 ? 0L : (long)a.K * a.n_up) + (long)m.k * m.ns;
  return m;
}

// Envelope of orbital i at electron jg, with its gradient along r_jg and its
// Laplacian, in precision T.
template <class T>
__device__ __forceinline__ void envelope(const DetArgs& a, const MatId& m, int i, int jg, const float* R, T& ev,
                                         T* eg, T& el, bool deriv) {
  const float* xj = a.x + (m.w * a.n + jg) * 3;
  const float* pi = a.pi[m.s] + ((long)m.k * m.ns + i) * a.N;
  const float* sg = a.sigma[m.s] + ((long)m.k * m.ns + i) * a.N;
  ev = T(0);
  el = T(0);
  eg[0] = eg[1] = eg[2] = T(0);
  for (int mm = 0; mm < a.N; ++mm) {
    T d0 = (T)xj[0] - (T)R[3 * mm], d1 = (T)xj[1] - (T)R[3 * mm + 1], d2 = (T)xj[2] - (T)R[3 * mm + 2];
    T r = sqrt(d0 * d0 + d1 * d1 + d2 * d2);
    T s = fabs((T)sg[mm]);
    T ex = (T)pi[mm] * exp(-s * r);
    ev += ex;
    if (deriv) {
      T ir = r > T(0) ? T(1) / r : T(0);
      T gs = -s * ex * ir;
      eg[0] = fma(gs, d0, eg[0]);
      eg[1] = fma(gs, d1, eg[1]);
      eg[2] = fma(gs, d2, eg[2]);
      el = fma(ex, s * s - T(2) * s * ir, el);
    }
  }
}

// One warp, one matrix, value pass, in precision T.  Writes sign, log|det| and
// (optionally) the inverse and envelopes; returns whether the pivot ratio
// flags the matrix as ill-conditioned (warp-uniform).
template <int NM, class T>
__device__ bool det_value_body(const DetArgs& a, long mat, const MatId& m, int lane, const float* R,
                               bool count) {
  T ra[NM], rb[NM];
  const long NSS = a.nss;
#pragma unroll
  for (int c = 0; c < NM; ++c) {
    ra[c] = (c == lane) ? T(1) : T(0);
    rb[c] = (c == lane) ? T(1) : T(0);
  }
  if (lane < m.ns) {
#pragma unroll
    for (int c = 0; c < NM; ++c) {
      if (c < m.ns) {
        const int jg = m.j0 + c;
        T o = (T)a.O[((m.w * a.n + jg) * (long)a.C) * a.ldo + m.q0 + lane];
        T ev, eg[3], el;
        envelope<T>(a, m, lane, jg, R, ev, eg, el, false);
        ra[c] = o * ev;
        if (a.env) a.env[mat * NSS + lane * m.ns + c] = (float)ev;
      }
    }
  }
  T logabs, sgn, pmin, pmax;
  bool sing;
  warp_gj<NM, T>(ra, rb, m.ns, lane, logabs, sgn, pmin, pmax, sing);
  const bool flag = !sing && pmin < (T)a.pivot_tau * pmax;
  if (lane == 0) {
    a.logdet[mat] = sing ? -INFINITY : (float)logabs;
    a.sign[mat] = sing ? 0.f : (float)sgn;
    // a singular result is reported by whichever pass settles the matrix
    // (the FP64 redo included); the flagged count belongs to the FP32 pass
    if (sing) atomicOr(a.status, (unsigned)ST_SINGULAR);
    else if (flag && count) atomicAdd(a.flagged, 1ull);
  }
  if (a.minv && lane < m.ns) {
#pragma unroll
    for (int c = 0; c < NM; ++c)
      if (c < m.ns) a.minv[mat * NSS + lane * m.ns + c] = sing ? 0.f : (float)rb[c];
  }
  return flag;
}

// Value pass: one warp per matrix, four matrices per block; FP64 redo of
// matrices whose FP32 pivot ratio falls below pivot_tau.
template <int NM>
__global__ void __launch_bounds__(128) k_det_value(DetArgs a) {
  const int lane = threadIdx.x & 31;
  const long mat = (long)blockIdx.x * 4 + (threadIdx.x >> 5);
  const long nmat = a.Bc * a.K * 2;
  if (mat >= nmat) return;
  const MatId m = mat_id(mat, a);
  if (m.ns == 0) {
    if (lane == 0) {
      a.logdet[mat] = 0.f;
      a.sign[mat] = 1.f;
    }
    return;
  }
  const float* R = a.g.R + (long)geo_of(a.g, a.w0 + m.w) * a.N * 3;
  const bool flag = det_value_body<NM, float>(a, mat, m, lane, R, true);
  if (flag || a.force64) det_value_body<NM, double>(a, mat, m, lane, R, false);
}

// Value pass for NM <= 16: one warp holds the up- and down-spin matrices of one
// (walker, determinant) in its two 16-lane halves, padded with identity rows to
// the larger of the two sizes; the electron-nucleus distances of the walker are
// computed once per warp into shared memory.  Matrices flagged by the FP32
// pivot ratio are redone in FP64 by the whole warp.
template <int NM, class T>
__device__ bool det_pair_body(const DetArgs& a, long mat, const MatId& m, int sl, int nmax, const float* dist,
                              bool count) {
  T ra[NM], rb[NM];
  const long NSS = a.nss;
  // determinant only, in FP32: half-warp LU and fast exponentials (the stored
  // forward of the adjoint keeps the accurate path)
  bool fast = false;
  if constexpr (std::is_same<T, float>::value) fast = !a.minv && !a.env;
#pragma unroll
  for (int c = 0; c < NM; ++c) {
    ra[c] = (c == sl) ? T(1) : T(0);
    rb[c] = (c == sl) ? T(1) : T(0);
  }
  if (fast && sl < m.ns) {
    // nuclei outer, this lane's columns inner: pi and sigma loaded once per
    // nucleus, exp(-|sigma| d) as 2^(-|sigma| log2(e) d)
    const float* pi = a.pi[m.s] + ((long)m.k * m.ns + sl) * a.N;
    const float* sg = a.sigma[m.s] + ((long)m.k * m.ns + sl) * a.N;
    float ev[NM];
#pragma unroll
    for (int c = 0; c < NM; ++c) ev[c] = 0.f;
    for (int mm = 0; mm < a.N; ++mm) {
      const float pm = pi[mm], sm2 = -fabsf(sg[mm]) * 1.4426950408889634f;
      const float* dm = dist + m.j0 * a.N + mm;
#pragma unroll
      for (int c = 0; c < NM; ++c)
        if (c < m.ns) ev[c] = fmaf(pm, exp2f(sm2 * dm[c * a.N]), ev[c]);
    }
    const float* ob = a.O + (m.w * a.n + m.j0) * (long)a.C * a.ldo + m.q0 + sl;
    const int ostride = (int)(a.C * a.ldo);
#pragma unroll
    for (int c = 0; c < NM; ++c)
      if (c < m.ns) ra[c] = (T)(ob[c * ostride] * ev[c]);
  } else if (sl < m.ns) {
    const float* pi = a.pi[m.s] + ((long)m.k * m.ns + sl) * a.N;
    const float* sg = a.sigma[m.s] + ((long)m.k * m.ns + sl) * a.N;
#pragma unroll
    for (int c = 0; c < NM; ++c) {
      if (c < m.ns) {
        const int jg = m.j0 + c;
        const T o = (T)a.O[((m.w * a.n + jg) * (long)a.C) * a.ldo + m.q0 + sl];
        const float* dj = dist + jg * a.N;
        T ev = T(0);
        for (int mm = 0; mm < a.N; ++mm) ev += (T)pi[mm] * exp(-fabs((T)sg[mm]) * (T)dj[mm]);
        ra[c] = o * ev;
        if (a.env) a.env[mat * NSS + sl * m.ns + c] = (float)ev;
      }
    }
  }
  T logabs, sgn, pmin, pmax;
  bool sing;
  bool done = false;
  if (a.minv) {
    warp_gj<NM, T, 16, true>(ra, rb, nmax, sl, logabs, sgn, pmin, pmax, sing, m.ns);
    done = true;
  }
  if constexpr (std::is_same<T, float>::value) {
    if (!done && fast) {
      warp_lu16<NM>(ra, nmax, sl, logabs, sgn, pmin, pmax, sing, m.ns);
      done = true;
    }
  }
  if (!done) warp_gj<NM, T, 16, false>(ra, rb, nmax, sl, logabs, sgn, pmin, pmax, sing, m.ns);
  const bool flag = !sing && pmin < (T)a.pivot_tau * pmax;
  if (sl == 0) {
    a.logdet[mat] = sing ? -INFINITY : (float)logabs;
    a.sign[mat] = sing ? 0.f : (float)sgn;
    // a singular result is reported by whichever pass settles the matrix
    // (the FP64 redo included); the flagged count belongs to the FP32 pass
    if (sing) atomicOr(a.status, (unsigned)ST_SINGULAR);
    else if (flag && count) atomicAdd(a.flagged, 1ull);
  }
  if (a.minv && sl < m.ns) {
#pragma unroll
    for (int c = 0; c < NM; ++c)
      if (c < m.ns) a.minv[mat * NSS + sl * m.ns + c] = sing ? 0.f : (float)rb[c];
  }
  return flag;
}

// Distances |r_j - R_m| of walker w for all electrons and nuclei, in the warp's
// shared slice.
__device__ __forceinline__ void pair_distances(const DetArgs& a, const MatId& m, int lane, float* dist) {
  const float* R = a.g.R + (long)geo_of(a.g, a.w0 + m.w) * a.N * 3;
  for (int t = lane; t < a.n * a.N; t += 32) {
    const int j = t / a.N, mm = t % a.N;
    const float* xj = a.x + (m.w * a.n + j) * 3;
    const float d0 = xj[0] - R[3 * mm], d1 = xj[1] - R[3 * mm + 1], d2 = xj[2] - R[3 * mm + 2];
    dist[t] = sqrtf(d0 * d0 + d1 * d1 + d2 * d2);
  }
  __syncwarp();
}

// Value pass: a warp per determinant k of a walker, its two spin matrices in
// the 16-lane halves.  A pair with a matrix whose FP32 pivot ratio falls below
// pivot_tau is appended to the list a.redo and done again in FP64 by
// k_det_value_pair_redo (kept out of this kernel, whose registers it would
// otherwise set).
template <int NM>
__global__ void __launch_bounds__(128) k_det_value_pair(DetArgs a) {
  extern __shared__ float dsh[];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int half = lane >> 4, sl = lane & 15;
  const long pair = (long)blockIdx.x * 4 + warp;
  const long npair = a.Bc * a.K;
  if (pair >= npair) return;  // warp-uniform
  const long mat = 2 * pair + half;
  const MatId m = mat_id(mat, a);
  float* dist = dsh + warp * a.n * a.N;
  pair_distances(a, m, lane, dist);
  const int nmax = a.n_up > a.n - a.n_up ? a.n_up : a.n - a.n_up;
  // an empty spin channel (ns = 0) still takes part in the warp-wide shuffles
  const bool flag = det_pair_body<NM, float>(a, mat, m, sl, nmax, dist, true) && m.ns > 0;
  if (m.ns == 0 && sl == 0) {
    a.logdet[mat] = 0.f;
    a.sign[mat] = 1.f;
  }
  if (__any_sync(FULL, flag || a.force64) && lane == 0) a.redo[1 + atomicAdd(a.redo, 1)] = (int)pair;
}

// FP64 redo of the listed pairs (a.redo[0] of them), a warp per pair.
template <int NM>
__global__ void __launch_bounds__(128) k_det_value_pair_redo(DetArgs a) {
  extern __shared__ float dsh[];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int half = lane >> 4, sl = lane & 15;
  const int count = a.redo[0];
  float* dist = dsh + warp * a.n * a.N;
  const int nmax = a.n_up > a.n - a.n_up ? a.n_up : a.n - a.n_up;
  for (int q = blockIdx.x * 4 + warp; q < count; q += gridDim.x * 4) {  // warp-uniform
    const long pair = a.redo[1 + q];
    const long mat = 2 * pair + half;
    const MatId m = mat_id(mat, a);
    pair_distances(a, m, lane, dist);
    det_pair_body<NM, double>(a, mat, m, sl, nmax, dist, false);
    if (m.ns == 0 && sl == 0) {
      a.logdet[mat] = 0.f;
      a.sign[mat] = 1.f;
    }
    __syncwarp();  // the distance slice is refilled for the next pair
  }
}

// Coordinates handled together in the tangent pass: NM threads per coordinate.
template <int NM>
constexpr int coord_batch() { return 128 / NM; }

template <int NM, class T>
struct TangentSmem {
  T Ms[NM][NM];        // A^-1, zero padded
  T Os[NM][NM + 1];    // orbital values o_i(r_j)
  T Es[NM][NM + 1];    // envelopes e_i(r_j)
  T Eg[3][NM][NM + 1];
  T El[NM][NM + 1];
  // rows padded to NM + 1: the threads of a coordinate read one row each
  T ET[NM][NM + 1];        // Es transposed [j][i], zero padded
  T OT[NM][NM + 1];        // Os transposed
  T EgT[3][NM][NM + 1];    // Eg transposed
  float Draw[2][coord_batch<NM>()][NM][NM + 1];  // d o_i(r_j) / d x_c as [c][j][i], two buffers
  T Xs[coord_batch<NM>()][NM * (NM + 1)];        // X_c = A^-1 d_c A, column j at j (NM + 1)
};

__device__ __forceinline__ void cp_async4(void* smem, const void* gmem) {
  const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(sa), "l"(gmem));
}

// Tangent-pass body for one matrix in precision T (128 threads).  Returns
// whether the pivot ratio flags the matrix (block-uniform).
//
// d log|det A| / d x_c = tr(X_c) and lap log|det A| = tr(A^-1 lap A) -
// sum_c tr(X_c^2) with X_c = A^-1 d_c A, where A_ij = o_i(r_j) e_i(r_j) and
// d_c A_ij = (d_c o_i(r_j)) e_i(r_j) + [c is a coordinate of electron j]
// o_i(r_j) d_c e_i(r_j).  The orbital tangents of a batch of coordinates are
// copied into shared memory while the previous batch is reduced.
template <int NM, class T>
__device__ bool det_tangent_body(const DetArgs& a, long mat, const MatId& m, const float* R, char* raw,
                                 bool count) {
  constexpr int CB = coord_batch<NM>();
  TangentSmem<NM, T>& sm = *reinterpret_cast<TangentSmem<NM, T>*>(raw);
  __shared__ double red[4];
  __shared__ int sing_s, flag_s;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int n3 = 3 * a.n;
  const int ns = m.ns;
  auto orow = [&](int jg, int c) -> const float* {
    return a.O + ((m.w * a.n + jg) * (long)a.C + c) * a.ldo + m.q0;
  };
  // zero padding of the transposed tiles and of both raw buffers (the copies
  // below only ever write entries i, j < ns)
  for (int t = tid; t < NM * (NM + 1); t += 128) {
    (&sm.ET[0][0])[t] = T(0);
    (&sm.OT[0][0])[t] = T(0);
    (&sm.EgT[0][0][0])[t] = T(0);
    (&sm.EgT[1][0][0])[t] = T(0);
    (&sm.EgT[2][0][0])[t] = T(0);
  }
  for (int t = tid; t < 2 * CB * NM * (NM + 1); t += 128) (&sm.Draw[0][0][0][0])[t] = 0.f;
  __syncthreads();
  const int nb = (n3 + CB - 1) / CB;
  // raw tangents of batch b: the NM lanes of a run slot copy consecutive
  // orbitals i of one (coordinate, electron) run
  const int li = tid % NM, slot = tid / NM;
  const float* obase = a.O + (m.w * a.n + m.j0) * (long)a.C * a.ldo + m.q0 + li;
  const int ldo_i = (int)a.ldo;
  auto stage = [&](int b) {
#pragma unroll 1
    for (int r = slot; r < CB * NM; r += 128 / NM) {
      const int cl = r / NM, j = r % NM, c = b * CB + cl;
      if (j < ns && li < ns && c < n3)
        cp_async4(&sm.Draw[b & 1][cl][j][li], obase + (long)((j * a.C + 1 + c) * ldo_i));
    }
    asm volatile("cp.async.commit_group;\n" ::);
  };
  stage(0);
  for (int t = tid; t < ns * ns; t += 128) {
    int i = t / ns, j = t % ns;
    T ev, eg[3], el;
    envelope<T>(a, m, i, m.j0 + j, R, ev, eg, el, true);
    const T o = (T)orow(m.j0 + j, 0)[i];
    sm.Es[i][j] = ev;
    sm.Eg[0][i][j] = eg[0];
    sm.Eg[1][i][j] = eg[1];
    sm.Eg[2][i][j] = eg[2];
    sm.El[i][j] = el;
    sm.Os[i][j] = o;
    sm.ET[j][i] = ev;
    sm.OT[j][i] = o;
    sm.EgT[0][j][i] = eg[0];
    sm.EgT[1][j][i] = eg[1];
    sm.EgT[2][j][i] = eg[2];
  }
  __syncthreads();
  if (warp == 0) {
    T ra[NM], rb[NM];
#pragma unroll
    for (int c = 0; c < NM; ++c) {
      ra[c] = (c == lane) ? T(1) : T(0);
      rb[c] = (c == lane) ? T(1) : T(0);
    }
    if (lane < ns) {
#pragma unroll
      for (int c = 0; c < NM; ++c)
        if (c < ns) ra[c] = sm.Os[lane][c] * sm.Es[lane][c];
    }
    T logabs, sgn, pmin, pmax;
    bool sing;
    warp_gj<NM, T>(ra, rb, ns, lane, logabs, sgn, pmin, pmax, sing);
    if (lane < NM) {
#pragma unroll
      for (int c = 0; c < NM; ++c) sm.Ms[lane][c] = (lane < ns && c < ns) ? rb[c] : T(0);
    }
    if (lane == 0) {
      const bool flag = !sing && pmin < (T)a.pivot_tau * pmax;
      a.logdet[mat] = sing ? -INFINITY : (float)logabs;
      a.sign[mat] = sing ? 0.f : (float)sgn;
      sing_s = sing ? 1 : 0;
      flag_s = flag ? 1 : 0;
      // a singular result is reported by whichever pass settles the matrix
      // (the FP64 redo included); the flagged count belongs to the FP32 pass
      if (sing) atomicOr(a.status, (unsigned)ST_SINGULAR);
      else if (flag && count) atomicAdd(a.flagged, 1ull);
    }
  }
  __syncthreads();
  const bool flag = flag_s != 0;
  if (sing_s) {
    asm volatile("cp.async.wait_group 0;\n" ::);
    if (tid == 0) a.dlap[mat] = 0.f;
    for (int c = tid; c < n3; c += 128) a.dgrad[mat * n3 + c] = 0.f;
    __syncthreads();
    return false;
  }
  // tr(A^-1 lap A), lap A_ij = lap o e + o lap e + 2 grad_j o . grad_j e
  double part = 0.0;
  for (int t = tid; t < ns * ns; t += 128) {
    int i = t / ns, j = t % ns, jg = m.j0 + j;
    T lo = (T)orow(jg, n3 + 1)[i];
    T cross = (T)orow(jg, 1 + 3 * jg)[i] * sm.Eg[0][i][j] + (T)orow(jg, 2 + 3 * jg)[i] * sm.Eg[1][i][j] +
              (T)orow(jg, 3 + 3 * jg)[i] * sm.Eg[2][i][j];
    T la = lo * sm.Es[i][j] + sm.Os[i][j] * sm.El[i][j] + T(2) * cross;
    part += (double)(sm.Ms[j][i] * la);
  }
  // coordinates in batches of CB: thread (cl, j) forms column j of X_c
  const int cl = tid / NM, j = tid % NM;
  for (int b = 0; b < nb; ++b) {
    if (b + 1 < nb) {
      stage(b + 1);
      asm volatile("cp.async.wait_group 1;\n" ::);
    } else {
      asm volatile("cp.async.wait_group 0;\n" ::);
    }
    __syncthreads();  // batch b's tangents are visible to every thread
    const int c = b * CB + cl;
    const bool act = c < n3;
    T x[NM];
    if (act) {
      const int e = c / 3, dd = c - 3 * e;
      const bool own = e == m.j0 + j && j < ns;
      const float* rw = &sm.Draw[b & 1][cl][j][0];
      T d[NM];
#pragma unroll
      for (int l = 0; l < NM; ++l) {
        const T v = (T)rw[l] * sm.ET[j][l];
        d[l] = own ? fma(sm.OT[j][l], sm.EgT[dd][j][l], v) : v;
      }
#pragma unroll
      for (int i = 0; i < NM; ++i) {
        T acc = T(0);
#pragma unroll
        for (int l = 0; l < NM; ++l) acc = fma(sm.Ms[i][l], d[l], acc);  // row i: a broadcast read
        x[i] = acc;
      }
#pragma unroll
      for (int i = 0; i < NM; ++i) sm.Xs[cl][j * (NM + 1) + i] = x[i];
    }
    __syncwarp();
    T tr = T(0), tr2 = T(0);
    if (act) {
      tr = sm.Xs[cl][j * (NM + 1) + j];
#pragma unroll
      for (int i = 0; i < NM; ++i) tr2 = fma(x[i], sm.Xs[cl][i * (NM + 1) + j], tr2);  // X_ij X_ji
    }
#pragma unroll
    for (int off = NM / 2; off > 0; off >>= 1) {
      tr += __shfl_xor_sync(FULL, tr, off, NM < 32 ? NM : 32);
      tr2 += __shfl_xor_sync(FULL, tr2, off, NM < 32 ? NM : 32);
    }
    if (act && j == 0) {
      a.dgrad[mat * n3 + c] = (float)tr;
      part -= (double)tr2;
    }
    __syncthreads();  // Draw[b & 1] and Xs are refilled next
  }
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) part += __shfl_xor_sync(FULL, part, off);
  if (lane == 0) red[warp] = part;
  __syncthreads();
  if (tid == 0) a.dlap[mat] = (float)(red[0] + red[1] + red[2] + red[3]);
  __syncthreads();
  return flag;
}

// Tangent pass: one 128-thread block per matrix in FP32.  A matrix whose FP32
// pivot ratio falls below pivot_tau is appended to the list a.redo and done
// again in FP64 by k_det_tangent_redo.
template <int NM>
constexpr int det_tangent_min_blocks() { return NM <= 16 ? 4 : 1; }  // 4 x 39 KB of shared memory at NM = 16

template <int NM>
__global__ void __launch_bounds__(128, det_tangent_min_blocks<NM>()) k_det_tangent(DetArgs a) {
  extern __shared__ __align__(16) char raw[];
  const long mat = blockIdx.x;
  const MatId m = mat_id(mat, a);
  const int n3 = 3 * a.n, tid = threadIdx.x;
  if (m.ns == 0) {
    if (tid == 0) {
      a.logdet[mat] = 0.f;
      a.sign[mat] = 1.f;
      a.dlap[mat] = 0.f;
    }
    for (int c = tid; c < n3; c += 128) a.dgrad[mat * n3 + c] = 0.f;
    return;
  }
  const float* R = a.g.R + (long)geo_of(a.g, a.w0 + m.w) * a.N * 3;
  const bool flag = det_tangent_body<NM, float>(a, mat, m, R, raw, true);
  if (tid == 0 && (flag || a.force64)) a.redo[1 + atomicAdd(a.redo, 1)] = (int)mat;
}

// FP64 redo of the listed matrices (a.redo[0] of them): a small persistent grid.
template <int NM>
__global__ void __launch_bounds__(128) k_det_tangent_redo(DetArgs a) {
  extern __shared__ __align__(16) char raw[];
  const int count = a.redo[0];
  for (int q = blockIdx.x; q < count; q += gridDim.x) {  // block-uniform
    const long mat = a.redo[1 + q];
    const MatId m = mat_id(mat, a);
    const float* R = a.g.R + (long)geo_of(a.g, a.w0 + m.w) * a.N * 3;
    det_tangent_body<NM, double>(a, mat, m, R, raw, false);
  }
}

template <int NM>
void launch_nm(cudaStream_t s, const DetArgs& a) {
  long nmat = a.Bc * a.K * 2;
  if (nmat <= 0) return;
  if (a.tangent) {
    const int smem = (int)sizeof(TangentSmem<NM, float>);
    const int smem64 = (int)sizeof(TangentSmem<NM, double>);
    static bool attr = false;  // set once per process (the attribute is per function)
    if (!attr) {
      cudaFuncSetAttribute(k_det_tangent<NM>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
      cudaFuncSetAttribute(k_det_tangent_redo<NM>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem64);
      attr = true;
    }
    cudaMemsetAsync(a.redo, 0, sizeof(int), s);  // empty redo list
    FN_COUNT(1), k_det_tangent<NM><<<(unsigned)nmat, 128, smem, s>>>(a);
    const long redo_blocks = std::min<long>(nmat, 152L * 2);
    FN_COUNT(1), k_det_tangent_redo<NM><<<(unsigned)redo_blocks, 128, smem64, s>>>(a);
  } else if (NM <= 16 && a.redo && (long)a.n * a.N * 4 * sizeof(float) <= 32768) {
    const long npair = a.Bc * a.K;
    const size_t sm = sizeof(float) * 4 * a.n * a.N;
    cudaMemsetAsync(a.redo, 0, sizeof(int), s);  // empty redo list
    FN_COUNT(1), k_det_value_pair<NM <= 16 ? NM : 16><<<(unsigned)((npair + 3) / 4), 128, sm, s>>>(a);
    const long redo_blocks = std::min<long>((npair + 3) / 4, 152L * 2);
    FN_COUNT(1), k_det_value_pair_redo<NM <= 16 ? NM : 16><<<(unsigned)redo_blocks, 128, sm, s>>>(a);
  } else {
    FN_COUNT(1), k_det_value<NM><<<(unsigned)((nmat + 3) / 4), 128, 0, s>>>(a);
  }
}

}  // namespace

void launch_det(cudaStream_t s, const DetArgs& a) {
  int ns = a.n_up > a.n - a.n_up ? a.n_up : a.n - a.n_up;
  if (ns <= 4)
    launch_nm<4>(s, a);
  else if (ns <= 8)
    launch_nm<8>(s, a);
  else if (ns <= 16)
    launch_nm<16>(s, a);
  else
    launch_nm<32>(s, a);
}

}  // namespace fn
