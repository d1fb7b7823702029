// Determinants in the local-energy pass (Eq. 3-4 with the kinetic energy of
// Eq. 1 in forward mode): for every orbital matrix A, one block forms A^-1,
// log|det A|, d_c log|det A| = tr(A^-1 d_c A) for the 3n coordinates and
//   lap log|det A| = tr(A^-1 lap A) - sum_c tr((A^-1 d_c A)^2).
// The shared device code is in det_common.cuh; the value-pass kernels and the
// dispatcher in k_det.cu.
#include <algorithm>
#include <mutex>

#include "det_common.cuh"

namespace fn {
namespace {

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
    asm volatile("cp.async.wait_group 0;\n" ::);  // batch b, the only copy group in flight
    // batch b's tangents are visible to every thread, and every thread is done
    // with batch b - 1: its raw buffer and the X_c tiles may be refilled
    __syncthreads();
    if (b + 1 < nb) stage(b + 1);  // lands while batch b is reduced
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
void launch_tangent_nm(cudaStream_t s, const DetArgs& a) {
  const long nmat = a.Bc * a.K * 2;
  if (nmat <= 0) return;
  const int smem = (int)sizeof(TangentSmem<NM, float>);
  const int smem64 = (int)sizeof(TangentSmem<NM, double>);
  static PerDeviceOnce attr;  // the attribute is per function and device
  attr([&] {
    cudaFuncSetAttribute(k_det_tangent<NM>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    cudaFuncSetAttribute(k_det_tangent_redo<NM>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem64);
  });
  cudaMemsetAsync(a.redo, 0, sizeof(int), s);  // empty redo list
  FN_COUNT(1), k_det_tangent<NM><<<(unsigned)nmat, 128, smem, s>>>(a);
  const long redo_blocks = std::min<long>(nmat, 2L * device_sm_count());
  FN_COUNT(1), k_det_tangent_redo<NM><<<(unsigned)redo_blocks, 128, smem64, s>>>(a);
}

}  // namespace

void launch_det_tangent(cudaStream_t s, const DetArgs& a) {
  int ns = a.n_up > a.n - a.n_up ? a.n_up : a.n - a.n_up;
  if (ns <= 4)
    launch_tangent_nm<4>(s, a);
  else if (ns <= 8)
    launch_tangent_nm<8>(s, a);
  else if (ns <= 16)
    launch_tangent_nm<16>(s, a);
  else
    launch_tangent_nm<32>(s, a);
}

}  // namespace fn
