// Shared device code of the determinant kernels (k_det.cu: value passes,
// k_det_tangent.cu: local-energy pass): warp elimination, matrix indexing and
// the isotropic envelope (Eq. 4).
#pragma once

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
// Laplacian, in precision T.  Isotropic (Sec. 3): sum_m pi_m exp(-|sigma_m| r)
// with r = |r_jg - R_m|.  Full covariance (Eq. 4): sum_m pi_m exp(-rho) with
// v = Sigma_m d, rho = |v|, d = r_jg - R_m; with u = Sigma^T v (= M d for
// M = Sigma^T Sigma) the gradient of exp(-rho) is -exp(-rho) u / rho and its
// Laplacian exp(-rho) (|u|^2 / rho^2 - tr M / rho + |u|^2 / rho^3).
template <class T>
__device__ __forceinline__ void envelope(const DetArgs& a, const MatId& m, int i, int jg, const float* R, T& ev,
                                         T* eg, T& el, bool deriv) {
  const float* xj = a.x + (m.w * a.n + jg) * 3;
  const float* pi = a.pi[m.s] + ((long)m.k * m.ns + i) * a.N;
  ev = T(0);
  el = T(0);
  eg[0] = eg[1] = eg[2] = T(0);
  if (a.full_env) {
    const float* S = a.sigma[m.s] + ((long)m.k * m.ns + i) * a.N * 9;
    for (int mm = 0; mm < a.N; ++mm) {
      const float* Sm = S + 9 * mm;
      T d0 = (T)xj[0] - (T)R[3 * mm], d1 = (T)xj[1] - (T)R[3 * mm + 1], d2 = (T)xj[2] - (T)R[3 * mm + 2];
      T v0 = (T)Sm[0] * d0 + (T)Sm[1] * d1 + (T)Sm[2] * d2;
      T v1 = (T)Sm[3] * d0 + (T)Sm[4] * d1 + (T)Sm[5] * d2;
      T v2 = (T)Sm[6] * d0 + (T)Sm[7] * d1 + (T)Sm[8] * d2;
      T rho = sqrt(v0 * v0 + v1 * v1 + v2 * v2);
      T ex = (T)pi[mm] * exp(-rho);
      ev += ex;
      if (deriv) {
        T u0 = (T)Sm[0] * v0 + (T)Sm[3] * v1 + (T)Sm[6] * v2;
        T u1 = (T)Sm[1] * v0 + (T)Sm[4] * v1 + (T)Sm[7] * v2;
        T u2 = (T)Sm[2] * v0 + (T)Sm[5] * v1 + (T)Sm[8] * v2;
        T tr = T(0);
#pragma unroll
        for (int q = 0; q < 9; ++q) tr += (T)Sm[q] * (T)Sm[q];
        T ir = rho > T(0) ? T(1) / rho : T(0);
        T uu = u0 * u0 + u1 * u1 + u2 * u2;
        T gs = -ex * ir;
        eg[0] = fma(gs, u0, eg[0]);
        eg[1] = fma(gs, u1, eg[1]);
        eg[2] = fma(gs, u2, eg[2]);
        el = fma(ex, uu * ir * ir - tr * ir + uu * ir * ir * ir, el);
      }
    }
    return;
  }
  const float* sg = a.sigma[m.s] + ((long)m.k * m.ns + i) * a.N;
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

}  // namespace
}  // namespace fn
