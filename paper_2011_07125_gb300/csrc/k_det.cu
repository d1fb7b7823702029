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
//
// This file holds the paired value-pass kernels and the dispatcher; the
// warp-per-matrix value kernel is in k_det_value.cu, the local-energy pass in
// k_det_tangent.cu, the shared device code in det_common.cuh.
#include "det_common.cuh"

namespace fn {
namespace {

// Value pass for NM <= 16: one warp holds the up- and down-spin matrices of one
// (walker, determinant) in its two 16-lane halves, padded with identity rows to
// the larger of the two sizes; the electron-nucleus distances of the walker are
// computed once per warp into shared memory.
template <int NM, class T>
__device__ bool det_pair_body(const DetArgs& a, long mat, const MatId& m, int sl, int nmax, const float* dist,
                              bool count) {
  T ra[NM], rb[NM];
  const long NSS = a.nss;
  // isotropic envelope: from FP32 exponentials in both precisions (the FP64
  // redo of an ill-conditioned pair repeats the elimination, not the FP32
  // inputs), stored for the adjoint when asked; determinant only (no stored
  // inverse or envelope) in FP32: the half-warp LU
  const bool fast_env = !a.full_env;
  bool fast = false;
  if constexpr (std::is_same<T, float>::value) fast = fast_env && !a.minv && !a.env;
#pragma unroll
  for (int c = 0; c < NM; ++c) {
    ra[c] = (c == sl) ? T(1) : T(0);
    rb[c] = (c == sl) ? T(1) : T(0);
  }
  if (fast_env && sl < m.ns) {
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
      if (c < m.ns) ra[c] = (T)ob[c * ostride] * (T)ev[c];
    if (a.env) {
#pragma unroll
      for (int c = 0; c < NM; ++c)
        if (c < m.ns) a.env[mat * NSS + sl * m.ns + c] = ev[c];
    }
  } else if (sl < m.ns) {
    const float* pi = a.pi[m.s] + ((long)m.k * m.ns + sl) * a.N;
    const float* sg = a.sigma[m.s] + ((long)m.k * m.ns + sl) * a.N;
    const float* R = a.g.R + (long)geo_of(a.g, a.w0 + m.w) * a.N * 3;
#pragma unroll
    for (int c = 0; c < NM; ++c) {
      if (c < m.ns) {
        const int jg = m.j0 + c;
        const T o = (T)a.O[((m.w * a.n + jg) * (long)a.C) * a.ldo + m.q0 + sl];
        const float* dj = dist + jg * a.N;
        T ev = T(0);
        if (a.full_env) {
          T eg[3], el;
          envelope<T>(a, m, sl, jg, R, ev, eg, el, false);
        } else {
          for (int mm = 0; mm < a.N; ++mm) ev += (T)pi[mm] * exp(-fabs((T)sg[mm]) * (T)dj[mm]);
        }
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
__global__ void __launch_bounds__(128, 6) k_det_value_pair(DetArgs a) {
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
void launch_value_nm(cudaStream_t s, const DetArgs& a) {
  const long nmat = a.Bc * a.K * 2;
  if (nmat <= 0) return;
  if (NM <= 16 && a.redo && (long)a.n * a.N * 4 * sizeof(float) <= 32768) {
    const long npair = a.Bc * a.K;
    const size_t sm = sizeof(float) * 4 * a.n * a.N;
    cudaMemsetAsync(a.redo, 0, sizeof(int), s);  // empty redo list
    FN_COUNT(1), k_det_value_pair<NM <= 16 ? NM : 16><<<(unsigned)((npair + 3) / 4), 128, sm, s>>>(a);
    const long redo_blocks = std::min<long>((npair + 3) / 4, 2L * device_sm_count());
    FN_COUNT(1), k_det_value_pair_redo<NM <= 16 ? NM : 16><<<(unsigned)redo_blocks, 128, sm, s>>>(a);
  } else {
    launch_det_value_warp(s, a);
  }
}

}  // namespace

void launch_det(cudaStream_t s, const DetArgs& a) {
  if (a.tangent) {
    launch_det_tangent(s, a);
    return;
  }
  int ns = a.n_up > a.n - a.n_up ? a.n_up : a.n - a.n_up;
  if (ns <= 4)
    launch_value_nm<4>(s, a);
  else if (ns <= 8)
    launch_value_nm<8>(s, a);
  else if (ns <= 16)
    launch_value_nm<16>(s, a);
  else
    launch_value_nm<32>(s, a);
}

}  // namespace fn
