// Value-pass determinants, one warp per matrix (Eq. 3-4): the general form,
// used where the paired kernel of k_det.cu does not apply (spin blocks above
// 16 electrons, or distance tables too large for its shared memory).  Shared
// device code is in det_common.cuh.
#include "det_common.cuh"

namespace fn {
namespace {

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

template <int NM>
void launch_nm(cudaStream_t s, const DetArgs& a) {
  const long nmat = a.Bc * a.K * 2;
  if (nmat > 0) FN_COUNT(1), k_det_value<NM><<<(unsigned)((nmat + 3) / 4), 128, 0, s>>>(a);
}

}  // namespace

void launch_det_value_warp(cudaStream_t s, const DetArgs& a) {
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
