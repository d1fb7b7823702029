// C ABI of the FermiNet VMC hot path: context, parameter layout, workspace
// planning and the per-call kernel schedules.
//
// Schedule of one network pass over a chunk of Bc walkers (value pass: one
// column per activation row; tangent pass: C = tangent_cols(n) columns):
//   features -> for each layer l:
//       spin means of h^l (M1) and of h^l_ij (M2, expanded to dense columns)
//       U  = M1 . [V_b V_c]^T            (per-walker part of the factored layer)
//       Z  = h^l . V_a^T + M2 . [V_d V_e]^T + b + U
//       h^{l+1} = tanh(Z) (+ h^l), forward-Laplacian rule on the columns
//       h^{l+1}_ij = tanh(W h^l_ij + c) (+ h^l_ij)
//   orbitals O = h^L . W_orb^T + g  -> determinants -> log|psi|, E_L.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>

#include "fn_internal.cuh"
#include "tc_gemm.cuh"

namespace fn {

std::atomic<long long> g_launches{0};

void build_layout(const fn_net& t, Layout* L, bool with_entries) {
  L->entries.clear();
  long off = 0;
  auto add = [&](long* field, const char* nm, long cnt, long fan, int kind) {
    if (field) *field = off;
    if (with_entries) {
      fn_param_entry e{};
      snprintf(e.name, sizeof e.name, "%s", nm);
      e.offset = off;
      e.count = cnt;
      e.fan_in = fan;
      e.kind = kind;
      L->entries.push_back(e);
    }
    off += cnt;
  };
  char nm[32];
  for (int l = 0; l < t.n_layers; ++l) {
    long a = din1_of(t, l), e = din2_of(t, l), fan = 3 * a + 2 * e;
    snprintf(nm, sizeof nm, "V%d", l);
    add(&L->V[l], nm, (long)t.d1 * fan, fan, 0);
    snprintf(nm, sizeof nm, "b%d", l);
    add(&L->b[l], nm, t.d1, 1, 1);
    if (l < t.n_layers - 1) {
      snprintf(nm, sizeof nm, "W%d", l);
      add(&L->W[l], nm, (long)t.d2 * e, e, 0);
      snprintf(nm, sizeof nm, "c%d", l);
      add(&L->c[l], nm, t.d2, 1, 1);
    }
  }
  const long K = t.n_det;
  add(&L->w_orb, "w_orb_up", K * t.n_up * t.d1, t.d1, 0);
  add(nullptr, "w_orb_down", K * t.n_down * t.d1, t.d1, 0);
  add(&L->g_orb, "g_orb_up", K * t.n_up, 1, 1);
  add(nullptr, "g_orb_down", K * t.n_down, 1, 1);
  add(&L->pi[0], "pi_up", K * t.n_up * t.n_nuc, 1, 2);
  add(&L->pi[1], "pi_down", K * t.n_down * t.n_nuc, 1, 2);
  // isotropic: one scalar sigma per (k, spin, i, m), init 1; full covariance
  // (Eq. 4): one row-major 3x3 Sigma each, init the identity (kind 3)
  const long sz = t.envelope ? 9 : 1;
  const int skind = t.envelope ? 3 : 2;
  add(&L->sigma[0], "sigma_up", K * t.n_up * t.n_nuc * sz, 1, skind);
  add(&L->sigma[1], "sigma_down", K * t.n_down * t.n_nuc * sz, 1, skind);
  L->total = off;
}

}  // namespace fn

using namespace fn;

namespace {

// Bump allocator over the context workspace.  In measuring mode it hands out
// fake addresses and only records the total size.
struct Arena {
  char* base = nullptr;
  size_t off = 0;
  bool measure = true;
  template <class T>
  T* get(size_t n) {
    size_t bytes = ((n * sizeof(T) + 255) / 256) * 256;
    T* p = measure ? reinterpret_cast<T*>((uintptr_t)(4096 + off)) : reinterpret_cast<T*>(base + off);
    off += bytes;
    return p;
  }
};

struct FwdOut {
  float* logpsi = nullptr;
  float* sign = nullptr;
  float* eloc = nullptr;
  float* kinetic = nullptr;
};

// Value-pass activations kept for the adjoint.
struct Stored {
  // tensor-core store (mixed precision): activations and spin means as BF16
  // hi + lo, tanh values as FP32; otherwise everything FP32
  bool tc = false;
  __nv_bfloat16* Hb[17][2] = {};
  __nv_bfloat16* M1b[16][2] = {};
  __nv_bfloat16* M2b[16][2] = {};
  float* H[17] = {};
  float* Y[16] = {};
  float* E[17] = {};
  float* Y2[16] = {};
  float* M1[16] = {};
  float* M2[16] = {};
  float* O = nullptr;
  float* minv = nullptr;
  float* env = nullptr;
  float* wdet = nullptr;
};

fn_status fail(fn_ctx* c, fn_status st, const char* msg) {
  if (c) c->err = msg;
  return st;
}

fn_status cuda_check(fn_ctx* c, cudaError_t e, const char* where) {
  if (e == cudaSuccess) return FN_OK;
  if (c) c->err = std::string(where) + ": " + cudaGetErrorString(e);
  return FN_ECUDA;
}

#define CK(call)                                                 \
  do {                                                           \
    fn_status _st = cuda_check(c, (call), #call);                \
    if (_st != FN_OK) return _st;                                \
  } while (0)

cudaEvent_t take_event(fn_ctx* c) {
  if (!c->ev_pool.empty()) {
    cudaEvent_t e = c->ev_pool.back();
    c->ev_pool.pop_back();
    return e;
  }
  cudaEvent_t e = nullptr;
  cudaEventCreate(&e);
  return e;
}

// Brackets the launches issued during its lifetime with events on the context
// stream when profiling is on.
struct Prof {
  fn_ctx* c;
  int cls;
  double flops;
  cudaEvent_t e0 = nullptr;
  Prof(fn_ctx* c_, int cls_, double fl) : c(c_), cls(cls_), flops(fl) {
    if (c->prof_on && cls < FN_KC_COUNT) {
      e0 = take_event(c);
      cudaEventRecord(e0, c->stream);
    }
  }
  ~Prof() {
    if (e0) {
      cudaEvent_t e1 = take_event(c);
      cudaEventRecord(e1, c->stream);
      c->pending.push_back({cls, e0, e1, flops});
    }
  }
};

void drain_profile(fn_ctx* c) {
  if (c->pending.empty()) return;
  cudaStreamSynchronize(c->stream);
  for (auto& p : c->pending) {
    float ms = 0.f;
    cudaEventElapsedTime(&ms, p.e0, p.e1);
    c->prof_ms[p.cls] += ms;
    c->prof_n[p.cls] += 1;
    c->prof_flops[p.cls] += p.flops;
    c->ev_pool.push_back(p.e0);
    c->ev_pool.push_back(p.e1);
  }
  c->pending.clear();
}

Geo geo_of(fn_ctx* c) { return Geo{c->d_R, c->d_Z, c->d_Enn64, c->G > 1 ? c->d_geo : nullptr}; }

inline long pad64(long v) { return ((v + 63) / 64) * 64; }

// Rows-on-lanes orientation: activations as the A operand (128 rows per tile)
// and weights as B (features per tile = tile_n).
bool tc_segment_rm(TcGemmArgs& g, int seg, const __nv_bfloat16* x_hi, const __nv_bfloat16* x_lo, long rows, long lda,
                   const __nv_bfloat16* w_hi, const __nv_bfloat16* w_lo, long mfeat, long ldw, int tile_n) {
  if (ldw != lda) return false;
  bool ok = tc_make_map(&g.A[seg][0], x_hi, rows, lda, 128) && tc_make_map(&g.B[seg][0], w_hi, mfeat, ldw, tile_n);
  if (w_lo && x_lo)
    ok = ok && tc_make_map(&g.A[seg][1], x_lo, rows, lda, 128) && tc_make_map(&g.B[seg][1], w_lo, mfeat, ldw, tile_n);
  else {
    g.A[seg][1] = g.A[seg][0];
    g.B[seg][1] = g.B[seg][0];
  }
  g.kblocks[seg] = (int)(lda / 64);
  return ok;
}

// Features per tile in the rows-on-lanes orientation (<= cap, multiple of 16).
int feature_tile(long mfeat, int* n_tiles, int cap = 256) {
  if (cap < 16 || cap > 256 || cap % 16) cap = 256;
  const long nt = (mfeat + cap - 1) / cap;
  const long per = (mfeat + nt - 1) / nt;
  *n_tiles = (int)nt;
  return (int)(((per + 15) / 16) * 16);
}

// Rows per tile of the fused layer epilogue: whole (walker, electron) groups of
// C columns, at most 256 rows, a multiple of 16.
int layer_tile(int C, int groups = 0) {
  if (groups > 0 && groups * C <= 256 && (groups * C) % 16 == 0) return groups * C;
  for (int g = 256 / C; g >= 1; --g)
    if ((g * C) % 16 == 0) return g * C;
  return 0;
}

int plain_tile(long rows) { return rows >= 256 ? 256 : (int)(((rows + 15) / 16) * 16); }

// Tensor maps of one GEMM segment: weights (hi, lo) [mfeat][ldw] and
// activations (hi, lo) [rows][lda].
bool tc_segment(TcGemmArgs& g, int seg, const __nv_bfloat16* w_hi, const __nv_bfloat16* w_lo, long mfeat, long ldw,
                const __nv_bfloat16* x_hi, const __nv_bfloat16* x_lo, long rows, long lda, int tile_n) {
  if (ldw != lda) return false;
  bool ok = tc_make_map(&g.A[seg][0], w_hi, mfeat, ldw, 128) && tc_make_map(&g.B[seg][0], x_hi, rows, lda, tile_n);
  if (w_lo && x_lo)
    ok = ok && tc_make_map(&g.A[seg][1], w_lo, mfeat, ldw, 128) && tc_make_map(&g.B[seg][1], x_lo, rows, lda, tile_n);
  else {
    g.A[seg][1] = g.A[seg][0];
    g.B[seg][1] = g.B[seg][0];
  }
  g.kblocks[seg] = (int)(lda / 64);
  return ok;
}

// Whether the value pass that the adjoint stores runs on the tensor cores
// (mixed precision; the stored tanh values come from the rows-on-lanes layer
// epilogue, which needs d1 % 8 == 0).
bool tc_store_ok(const fn_ctx* c) {
  return c->prec == FN_PREC_MIXED && c->tc_ok && c->net.d1 % 8 == 0 && c->tune.adjoint_simt == 0;
}

// One network pass (see the file comment) over walkers [w0, w0 + Bc).
void forward(fn_ctx* c, Arena& ar, const float* x, long Bc, long w0, bool tangent, bool store, const FwdOut& out,
             Stored* st) {
  const fn_net& t = c->net;
  const int n = c->n, N = c->N, L = t.n_layers, K = t.n_det, d1 = t.d1, d2 = t.d2;
  const int C = tangent ? c->Ct : 1, Q = tangent ? kQ : 1;
  const int Creal = tangent ? 3 * n + 2 : 1;
  const long Ktot = (long)K * n;
  const long rows = Bc * n * C;
  const long pairs = Bc * n * n;
  int max_din1 = std::max(4 * N, d1), max_din2 = std::max(4, d2);
  float* H0 = ar.get<float>(rows * 4 * N);
  float* E0 = ar.get<float>(pairs * Q * 4);
  float *Ha = nullptr, *Hb = nullptr, *Ea = nullptr, *Eb = nullptr, *M1 = nullptr, *M2 = nullptr;
  const bool tc = c->prec == FN_PREC_MIXED && c->tc_ok && layer_tile(C) > 0 && (!store || tc_store_ok(c));
  const bool two = c->terms > 1;
  if (store && tc) {
    st->tc = true;
    st->E[0] = E0;
    for (int l = 0; l < L; ++l) {
      st->Y[l] = ar.get<float>(Bc * n * d1);
      if (l < L - 1) {
        st->E[l + 1] = ar.get<float>(pairs * Q * d2);
        st->Y2[l] = ar.get<float>(pairs * d2);
      }
      for (int h = 0; h < (two ? 2 : 1); ++h) {
        st->Hb[l + 1][h] = ar.get<__nv_bfloat16>(rows * pad64(d1));
        st->M1b[l][h] = ar.get<__nv_bfloat16>(Bc * C * pad64(2 * din1_of(t, l)));
        st->M2b[l][h] = ar.get<__nv_bfloat16>(rows * pad64(2 * din2_of(t, l)));
      }
    }
    M1 = ar.get<float>(Bc * C * 2 * max_din1);  // layer 0's means before their split
  } else if (store) {
    st->H[0] = H0;
    st->E[0] = E0;
    for (int l = 0; l < L; ++l) {
      st->H[l + 1] = ar.get<float>(rows * d1);
      st->Y[l] = ar.get<float>(Bc * n * d1);
      st->M1[l] = ar.get<float>(Bc * C * 2 * din1_of(t, l));
      st->M2[l] = ar.get<float>(rows * 2 * din2_of(t, l));
      if (l < L - 1) {
        st->E[l + 1] = ar.get<float>(pairs * Q * d2);
        st->Y2[l] = ar.get<float>(pairs * d2);
      }
    }
  } else {
    if (!(c->prec == FN_PREC_MIXED && c->tc_ok && layer_tile(C) > 0)) {
      Ha = ar.get<float>(rows * d1);
      Hb = ar.get<float>(rows * d1);
    }
    if (L > 1) {
      Ea = ar.get<float>(pairs * Q * d2);
      Eb = ar.get<float>(pairs * Q * d2);
    }
    M1 = ar.get<float>(Bc * C * 2 * max_din1);
    M2 = ar.get<float>(rows * 2 * max_din2);
  }
  float* U = ar.get<float>(Bc * C * d1);
  float* Z = tc ? nullptr : ar.get<float>(rows * d1);
  __nv_bfloat16 *H0b[2] = {}, *Hab[2] = {}, *Hbb[2] = {}, *M1b[2] = {}, *M2b[2] = {};
  const long ldh0 = pad64(4 * N), ldh = pad64(d1), ldm1 = pad64(2 * max_din1), ldm2 = pad64(2 * max_din2);
  __nv_bfloat16* Ub[2] = {};
  if (tc && tangent)
    for (int h = 0; h < (two ? 2 : 1); ++h) Ub[h] = ar.get<__nv_bfloat16>(Bc * C * ldh);
  if (tc) {
    for (int h = 0; h < (two ? 2 : 1); ++h) {
      H0b[h] = ar.get<__nv_bfloat16>(rows * ldh0);
      if (!store) {
        Hab[h] = ar.get<__nv_bfloat16>(rows * ldh);
        Hbb[h] = ar.get<__nv_bfloat16>(rows * ldh);
        M1b[h] = ar.get<__nv_bfloat16>(Bc * C * ldm1);
        M2b[h] = ar.get<__nv_bfloat16>(rows * ldm2);
      }
    }
    if (store) {
      st->Hb[0][0] = H0b[0];
      st->Hb[0][1] = H0b[1];
    }
  }
  float* O = ar.get<float>(rows * Ktot);
  float* logdet = ar.get<float>(Bc * K * 2);
  float* sgn = ar.get<float>(Bc * K * 2);
  float* dgrad = tangent ? ar.get<float>(Bc * K * 2 * 3 * n) : nullptr;
  float* dlap = tangent ? ar.get<float>(Bc * K * 2) : nullptr;
  int* redo = ar.get<int>(1 + Bc * K * 2);  // FP64 redo list of the determinant kernels
  const long nss = (long)c->ns_max * c->ns_max;
  if (store) {
    st->O = O;
    st->minv = ar.get<float>(Bc * K * 2 * nss);
    st->env = ar.get<float>(Bc * K * 2 * nss);
    st->wdet = ar.get<float>(Bc * K);
  }
  if (ar.measure) return;

  cudaStream_t s = c->stream;
  const float* P = c->d_params;
  const Geo g = geo_of(c);
  // Two-electron layers and their spin means in one fused pass (k_pair.cu)
  // when its kernels cover every layer's shapes; the means of layer l + 1 are
  // then produced by layer l's two-electron kernel.
  auto m2_ld = [&](int l) -> long { return tc ? pad64(2 * din2_of(t, l)) : 2L * din2_of(t, l); };
  bool fused = c->tune.pair_unfused == 0 && pair_layer_supported(n, 4, 4, false, Q, C, m2_ld(0));
  for (int l = 0; l < L - 1 && fused; ++l)
    fused = pair_layer_supported(n, din2_of(t, l), d2, true, Q, C, m2_ld(l + 1)) && (l == 0 || din2_of(t, l) == d2);
  auto pair_means = [&](const float* E, int din, float* m32, __nv_bfloat16* mhi, __nv_bfloat16* mlo, long ldm) {
    PairArgs pa{};
    pa.Ein = E;
    pa.groups = Bc * n;
    pa.n = n;
    pa.n_up = t.n_up;
    pa.C = C;
    pa.m32 = m32;
    pa.mhi = mhi;
    pa.mlo = mlo;
    pa.ldm = ldm;
    if (!launch_pair_layer(s, pa, din, din, Q)) c->host_fail = true;
  };
  auto pair_layer = [&](int l, const float* E, float* Eout, float* Y2, float* m32, __nv_bfloat16* mhi,
                        __nv_bfloat16* mlo) {
    PairArgs pa{};
    pa.Ein = E;
    pa.groups = Bc * n;
    pa.n = n;
    pa.n_up = t.n_up;
    pa.C = C;
    pa.W = P + c->lay.W[l];
    pa.cb = P + c->lay.c[l];
    pa.residual = l >= 1 ? 1 : 0;
    pa.Eout = Eout;
    pa.Y2 = Y2;
    pa.m32 = m32;
    pa.mhi = mhi;
    pa.mlo = mlo;
    pa.ldm = m2_ld(l + 1);
    pa.mma = c->prec == FN_PREC_MIXED ? 1 : 0;
    if (!launch_pair_layer(s, pa, din2_of(t, l), d2, Q)) c->host_fail = true;
  };
  launch_features(s, x, Bc, w0, n, N, C, Q, g, H0, E0);
  const float* Hc = H0;
  const float* Ec = E0;
  if (tc) {
    // Local-energy pass on the tensor cores: BF16 operands (hi, or hi + lo),
    // FP32 accumulation, fused forward-Laplacian tanh epilogue.
    const double fl_rows = 2.0 * (double)Bc * Creal;
    launch_split_bf16(s, H0, 4 * N, rows, 4 * N, H0b[0], H0b[1], ldh0);
    const __nv_bfloat16* Hcb[2] = {H0b[0], H0b[1]};
    long ldc_b = ldh0;
    const int tl = tangent ? layer_tile(C, c->tune.layer_groups) : plain_tile(rows);
    if (ldh != d1) {  // padding columns must read as zeros in the MMAs
      for (int h = 0; h < (two ? 2 : 1); ++h) {
        if (Hab[h]) cudaMemsetAsync(Hab[h], 0, sizeof(__nv_bfloat16) * rows * ldh, s);
        if (Hbb[h]) cudaMemsetAsync(Hbb[h], 0, sizeof(__nv_bfloat16) * rows * ldh, s);
        if (Ub[h]) cudaMemsetAsync(Ub[h], 0, sizeof(__nv_bfloat16) * Bc * C * ldh, s);
        for (int l = 1; store && l <= L; ++l)
          cudaMemsetAsync(st->Hb[l][h], 0, sizeof(__nv_bfloat16) * rows * ldh, s);
      }
    }
    for (int l = 0; l < L; ++l) {
      const int a1 = din1_of(t, l), a2 = din2_of(t, l);
      const long l1 = pad64(2 * a1), l2 = pad64(2 * a2);
      if (store)  // this layer's stored spin means (the fused pair kernel of layer l - 1 wrote M2b)
        for (int h = 0; h < 2; ++h) {
          M1b[h] = st->M1b[l][h];
          M2b[h] = st->M2b[l][h];
        }
      {
        Prof pm(c, tangent ? FN_KC_MEANS : FN_KC_COUNT, 0.0);
        if (l == 0) {
          launch_mean1(s, H0, Bc, n, t.n_up, C, a1, M1);
          launch_split_bf16(s, M1, 2 * a1, Bc * C, 2 * a1, M1b[0], M1b[1], l1);
        } else {
          launch_mean1_bf16(s, Hcb[0], Hcb[1], ldc_b, Bc, n, t.n_up, C, a1, M1b[0], M1b[1], l1);
        }
        if (!fused) launch_mean2_bf16(s, Ec, Bc, n, t.n_up, Q, a2, C, M2b[0], M2b[1], l2);
        else if (l == 0) pair_means(Ec, a2, nullptr, M2b[0], M2b[1], l2);
      }
      {
        Prof pg(c, tangent ? FN_KC_TANGENT_GEMM : FN_KC_COUNT, fl_rows * d1 * 2.0 * a1);
        TcGemmArgs u{};
        int ntf = 1;
        const int tu = feature_tile(d1, &ntf, c->tune.feature_tile);
        bool ok = tc_segment_rm(u, 0, M1b[0], M1b[1], Bc * C, l1, c->wb_hi + c->wb_bc[l],
                                two ? c->wb_lo + c->wb_bc[l] : nullptr, d1, c->ld_bc[l], tu);
        u.rm = 1;
        u.nseg = 1;
        u.terms = c->terms;
        u.seg_terms[0] = c->terms;
        u.rows = Bc * C;
        u.mfeat = d1;
        u.tile_n = tu;
        u.n_tiles_n = ntf;
        u.n_tiles_m = (int)((Bc * C + 127) / 128);
        u.mode = 0;
        u.out = U;
        u.ldo = d1;
        if (tangent) {  // stored as BF16 hi + lo: the operand of the folded segment below
          u.hb_hi = Ub[0];
          u.hb_lo = two ? Ub[1] : nullptr;
          u.ldhb = ldh;
        }
        u.bias_period = 1;
        u.status = c->d_status;
        if (!ok || tc_gemm_launch(s, u) != FN_OK) c->host_fail = true;
      }
      __nv_bfloat16** Hnb = store ? st->Hb[l + 1] : ((l % 2 == 0) ? Hab : Hbb);
      {
        Prof pg(c, tangent ? FN_KC_TANGENT_GEMM : FN_KC_COUNT, fl_rows * n * d1 * (double)(a1 + 2 * a2));
        TcGemmArgs m{};
        const bool rm = !tangent && d1 % 8 == 0;
        int ntf = 1;
        const int tf = rm ? feature_tile(d1, &ntf, c->tune.feature_tile) : 0;
        bool ok;
        if (rm) {
          ok = tc_segment_rm(m, 0, Hcb[0], Hcb[1], rows, ldc_b, c->wb_hi + c->wb_a[l],
                             two ? c->wb_lo + c->wb_a[l] : nullptr, d1, c->ld_a[l], tf);
          ok = ok && tc_segment_rm(m, 1, M2b[0], M2b[1], rows, l2, c->wb_hi + c->wb_de[l],
                                   two ? c->wb_lo + c->wb_de[l] : nullptr, d1, c->ld_de[l], tf);
        } else {
          ok = tc_segment(m, 0, c->wb_hi + c->wb_a[l], two ? c->wb_lo + c->wb_a[l] : nullptr, d1, c->ld_a[l],
                          Hcb[0], Hcb[1], rows, ldc_b, tl);
          ok = ok && tc_segment(m, 1, c->wb_hi + c->wb_de[l], two ? c->wb_lo + c->wb_de[l] : nullptr, d1,
                                c->ld_de[l], M2b[0], M2b[1], rows, l2, tl);
        }
        m.nseg = 2;
        m.terms = c->terms;
        m.seg_terms[0] = m.seg_terms[1] = c->terms;
        if (tangent) {
          // U[walker, column] enters the accumulator as a third segment: a 128 x 128
          // identity (exact in BF16) times the walker's U rows, gathered per group
          ok = ok && tc_make_map(&m.A[2][0], c->ident, 128, 128, 128) &&
               tc_make_map(&m.B[2][0], Ub[0], Bc * C, ldh, C);
          m.A[2][1] = m.A[2][0];
          if (two) ok = ok && tc_make_map(&m.B[2][1], Ub[1], Bc * C, ldh, C);
          else m.B[2][1] = m.B[2][0];
          m.kblocks[2] = 2;
          m.seg_terms[2] = two ? 2 : 1;
          m.seg_group[2] = C;
          m.nseg = 3;
        }
        m.rows = rows;
        m.mfeat = d1;
        if (rm) {
          m.rm = 1;
          m.tile_n = tf;
          m.n_tiles_n = ntf;
          m.n_tiles_m = (int)((rows + 127) / 128);
        } else {
          m.tile_n = tl;
          m.n_tiles_n = (int)((rows + tl - 1) / tl);
          m.n_tiles_m = (d1 + 127) / 128;
        }
        m.mode = tangent ? 1 : 2;
        m.bias = P + c->lay.b[l];
        m.bias_period = C;
        m.C = C;
        m.n3 = 3 * n;
        m.U = tangent ? nullptr : U;
        m.u_div = (long)n * C;
        m.ldu = d1;
        m.res_hi = l >= 1 ? Hcb[0] : nullptr;
        m.res_lo = (l >= 1 && two) ? Hcb[1] : nullptr;
        // the residual h^l is segment 0's B operand: read it from shared memory
        m.res_smem = (tangent && l >= 1 && !rm && c->tune.residual_smem == 1) ? 1 : 0;
        m.hb_hi = Hnb[0];
        m.hb_lo = two ? Hnb[1] : nullptr;
        m.ldhb = ldh;
        if (store) {  // tanh values for the adjoint
          m.y_out = st->Y[l];
          m.ldy = d1;
        }
        m.status = c->d_status;
        if (!ok || tc_gemm_launch(s, m) != FN_OK) c->host_fail = true;
      }
      if (l < L - 1) {
        float* En = store ? st->E[l + 1] : ((l % 2 == 0) ? Ea : Eb);
        float* Y2 = store ? st->Y2[l] : nullptr;
        __nv_bfloat16** M2n = store ? st->M2b[l + 1] : M2b;
        Prof p2(c, FN_KC_TWO_LAYER, 2.0 * (double)pairs * Q * d2 * a2);
        if (fused)  // after this layer's GEMMs have read M2b: it now receives layer l + 1's means
          pair_layer(l, Ec, (store || l + 1 < L - 1) ? En : nullptr, Y2, nullptr, M2n[0], two ? M2n[1] : nullptr);
        else
          launch_two_layer(s, Ec, Bc, n, Q, a2, d2, P + c->lay.W[l], P + c->lay.c[l], l >= 1, En, Y2);
        Ec = En;
      }
      Hcb[0] = Hnb[0];
      Hcb[1] = Hnb[1];
      ldc_b = ldh;
    }
    {
      const double same_spin = (double)t.n_up * t.n_up + (double)t.n_down * t.n_down;
      Prof pg(c, tangent ? FN_KC_TANGENT_GEMM : FN_KC_COUNT, 2.0 * (double)Bc * Creal * d1 * K * same_spin);
      // Per spin when the shapes allow: electron j of spin s only meets the
      // orbitals of spin s (Eq. 3), so each spin's rows (a block of n_s C rows
      // per walker, through a 3-D tensor map) meet that spin's K n_s orbitals;
      // the other-spin blocks of O are never computed nor read.
      const long q_up = (long)K * t.n_up;
      const bool per_spin = c->tune.orbital_joint == 0 && Ktot % 4 == 0 && q_up % 4 == 0 && t.n_up > 0 &&
                            t.n_down > 0;
      for (int sp = 0; sp < (per_spin ? 2 : 1); ++sp) {
        TcGemmArgs o{};
        const bool rm = Ktot % 4 == 0;
        const long q0 = per_spin && sp == 1 ? q_up : 0;
        const long nq = per_spin ? (long)K * (sp == 0 ? t.n_up : t.n_down) : Ktot;
        bool ok;
        if (per_spin) {
          const long ns = sp == 0 ? t.n_up : t.n_down, s_off = sp == 0 ? 0 : t.n_up;
          int ntf = 1;
          const int tf = feature_tile(nq, &ntf, c->tune.feature_tile);
          o.blk = 1;
          o.blk_rows = ns * C;
          o.blk_stride = (long)n * C;
          o.blk_off = s_off * C;
          o.n_blk = Bc;
          o.box_y = (int)std::min<long>(o.blk_rows, 128);
          o.box_z = o.blk_rows >= 128 ? 1 : (int)(128 / o.blk_rows);
          o.tiles_per_blk = (int)((o.blk_rows + o.box_y - 1) / o.box_y);
          const __nv_bfloat16* a_hi = Hcb[0] + o.blk_off * ldh;
          const __nv_bfloat16* a_lo = two ? Hcb[1] + o.blk_off * ldh : nullptr;
          const __nv_bfloat16* w_hi = c->wb_hi + c->wb_orb + q0 * c->ld_orb;
          const __nv_bfloat16* w_lo = two ? c->wb_lo + c->wb_orb + q0 * c->ld_orb : nullptr;
          ok = ldh == c->ld_orb && tc_make_map3(&o.A[0][0], a_hi, o.blk_rows, Bc, o.blk_stride, ldh, o.box_y, o.box_z) &&
               tc_make_map(&o.B[0][0], w_hi, nq, ldh, tf);
          if (two)
            ok = ok && tc_make_map3(&o.A[0][1], a_lo, o.blk_rows, Bc, o.blk_stride, ldh, o.box_y, o.box_z) &&
                 tc_make_map(&o.B[0][1], w_lo, nq, ldh, tf);
          else {
            o.A[0][1] = o.A[0][0];
            o.B[0][1] = o.B[0][0];
          }
          o.kblocks[0] = (int)(ldh / 64);
          o.rm = 1;
          o.tile_n = tf;
          o.n_tiles_n = ntf;
          o.n_tiles_m = (int)(o.box_z == 1 ? Bc * o.tiles_per_blk : (Bc + o.box_z - 1) / o.box_z);
        } else if (rm) {
          int ntf = 1;
          const int tf = feature_tile(Ktot, &ntf, c->tune.feature_tile);
          ok = tc_segment_rm(o, 0, Hcb[0], Hcb[1], rows, ldh, c->wb_hi + c->wb_orb,
                             two ? c->wb_lo + c->wb_orb : nullptr, Ktot, c->ld_orb, tf);
          o.rm = 1;
          o.tile_n = tf;
          o.n_tiles_n = ntf;
          o.n_tiles_m = (int)((rows + 127) / 128);
        } else {
          const int to = plain_tile(rows);
          ok = tc_segment(o, 0, c->wb_hi + c->wb_orb, two ? c->wb_lo + c->wb_orb : nullptr, Ktot, c->ld_orb,
                          Hcb[0], Hcb[1], rows, ldh, to);
          o.tile_n = to;
          o.n_tiles_n = (int)((rows + to - 1) / to);
          o.n_tiles_m = (int)((Ktot + 127) / 128);
        }
        o.nseg = 1;
        o.terms = c->terms;
        o.seg_terms[0] = c->terms;
        o.rows = rows;
        o.mfeat = (int)nq;
        o.mode = 0;
        o.out = O + q0;
        o.ldo = Ktot;
        o.bias = P + c->lay.g_orb + q0;
        o.bias_period = C;
        o.status = c->d_status;
        if (!ok || tc_gemm_launch(s, o) != FN_OK) c->host_fail = true;
      }
    }
  }
  for (int l = 0; l < L && !tc; ++l) {
    const int a1 = din1_of(t, l), a2 = din2_of(t, l), wV = 3 * a1 + 2 * a2;
    const float* V = P + c->lay.V[l];
    float* M1l = store ? st->M1[l] : M1;
    float* M2l = store ? st->M2[l] : M2;
    {
      Prof pm(c, tangent ? FN_KC_MEANS : FN_KC_COUNT, 0.0);
      launch_mean1(s, Hc, Bc, n, t.n_up, C, a1, M1l);
      if (!fused) launch_mean2(s, Ec, Bc, n, t.n_up, Q, a2, C, M2l);
      else if (l == 0) pair_means(Ec, a2, M2l, nullptr, nullptr, 2L * a2);
    }
    const double fl_rows = 2.0 * (double)Bc * Creal;  // algorithmic rows per walker-column, x2 for FMA
    {
      Prof pg(c, tangent ? FN_KC_TANGENT_GEMM : FN_KC_COUNT, fl_rows * d1 * 2.0 * a1);
      gemm_nt(s, Bc * C, d1, 2 * a1, M1l, 2 * a1, V + a1, wV, U, d1, Epi{});
    }
    {
      Prof pg(c, tangent ? FN_KC_TANGENT_GEMM : FN_KC_COUNT, fl_rows * n * d1 * (double)a1);
      gemm_nt(s, rows, d1, a1, Hc, a1, V, wV, Z, d1, Epi{});
    }
    Epi e;
    e.beta = 1.f;
    e.bias = P + c->lay.b[l];
    e.bias_period = C;
    e.U = U;
    e.u_div = (long)n * C;
    e.u_mul = C;
    e.u_mod = C;
    e.ldu = d1;
    {
      Prof pg(c, tangent ? FN_KC_TANGENT_GEMM : FN_KC_COUNT, fl_rows * n * d1 * 2.0 * a2);
      gemm_nt(s, rows, d1, 2 * a2, M2l, 2 * a2, V + 3 * a1, wV, Z, d1, e);
    }
    float* Hn = store ? st->H[l + 1] : ((l % 2 == 0) ? Ha : Hb);
    {
      Prof pt(c, tangent ? FN_KC_TANH : FN_KC_COUNT, 0.0);
      launch_tanh_fl(s, Z, l >= 1 ? Hc : nullptr, Bc, n, C, d1, Hn, store ? st->Y[l] : nullptr);
    }
    if (l < L - 1) {
      float* En = store ? st->E[l + 1] : ((l % 2 == 0) ? Ea : Eb);
      Prof p2(c, FN_KC_TWO_LAYER, 2.0 * (double)pairs * (tangent ? kQ : 1) * d2 * a2);
      if (fused)  // after this layer's GEMMs have read M2: it now receives layer l + 1's means
        pair_layer(l, Ec, (store || l + 1 < L - 1) ? En : nullptr, store ? st->Y2[l] : nullptr,
                   store ? st->M2[l + 1] : M2, nullptr, nullptr);
      else
        launch_two_layer(s, Ec, Bc, n, Q, a2, d2, P + c->lay.W[l], P + c->lay.c[l], l >= 1, En,
                         store ? st->Y2[l] : nullptr);
      Ec = En;
    }
    Hc = Hn;
  }
  Epi eo;
  eo.bias = P + c->lay.g_orb;
  eo.bias_period = C;
  if (!tc) {
    const double same_spin = (double)t.n_up * t.n_up + (double)t.n_down * t.n_down;
    Prof pg(c, tangent ? FN_KC_TANGENT_GEMM : FN_KC_COUNT, 2.0 * (double)Bc * Creal * d1 * K * same_spin);
    gemm_nt(s, rows, Ktot, d1, Hc, d1, P + c->lay.w_orb, d1, O, Ktot, eo);
  }
  DetArgs da{};
  da.O = O;
  da.ldo = Ktot;
  da.C = C;
  da.n = n;
  da.n_up = t.n_up;
  da.K = K;
  da.N = N;
  da.x = x;
  da.g = g;
  da.w0 = w0;
  da.Bc = Bc;
  da.pi[0] = P + c->lay.pi[0];
  da.pi[1] = P + c->lay.pi[1];
  da.sigma[0] = P + c->lay.sigma[0];
  da.sigma[1] = P + c->lay.sigma[1];
  da.full_env = t.envelope;
  da.tangent = tangent;
  da.logdet = logdet;
  da.sign = sgn;
  da.dgrad = dgrad;
  da.dlap = dlap;
  da.minv = store ? st->minv : nullptr;
  da.env = store ? st->env : nullptr;
  da.status = c->d_status;
  da.flagged = c->d_flagged;
  da.pivot_tau = c->pivot_tau;
  da.force64 = c->force64;
  da.nss = nss;
  da.redo = redo;
  {
    double fl = 0.0;
    for (int sp = 0; sp < 2; ++sp) {
      const double ns = sp == 0 ? t.n_up : t.n_down;
      fl += 2.0 * ns * ns * ns * 3.0 * n;
    }
    Prof pd(c, tangent ? FN_KC_DET_TANGENT : FN_KC_COUNT, fl * Bc * K);
    launch_det(s, da);
  }
  launch_combine(s, logdet, sgn, dgrad, dlap, x, Bc, w0, n, K, N, g, tangent, out.logpsi, out.sign, out.eloc,
                 out.kinetic, store ? st->wdet : nullptr, c->d_status);
}

// ---------------------------------------------------------------------------
// KFAC factor buffer (the same layout as the oracle's): per one-electron layer
// A1 [wV+1]^2, G1 [d1]^2; per two-electron layer A2 [din2+1]^2, G2 [d2]^2; per
// spin Ao [d1+1]^2, Go [K n_s]^2; then the envelope diagonal D.
struct KfacLayout {
  long A1[16] = {}, G1[16] = {}, A2[16] = {}, G2[16] = {}, Ao[2] = {}, Go[2] = {}, D = 0, total = 0;
  long dA1[16] = {}, dA2[16] = {}, dGo[2] = {};
};

void kfac_layout(const fn_net& t, const Layout& lay, KfacLayout* K) {
  long off = 0;
  for (int l = 0; l < t.n_layers; ++l) {
    K->dA1[l] = 3L * din1_of(t, l) + 2L * din2_of(t, l) + 1;
    K->A1[l] = off;
    off += K->dA1[l] * K->dA1[l];
    K->G1[l] = off;
    off += (long)t.d1 * t.d1;
  }
  for (int l = 0; l < t.n_layers - 1; ++l) {
    K->dA2[l] = din2_of(t, l) + 1;
    K->A2[l] = off;
    off += K->dA2[l] * K->dA2[l];
    K->G2[l] = off;
    off += (long)t.d2 * t.d2;
  }
  for (int s = 0; s < 2; ++s) {
    K->dGo[s] = (long)t.n_det * (s == 0 ? t.n_up : t.n_down);
    K->Ao[s] = off;
    off += (long)(t.d1 + 1) * (t.d1 + 1);
    K->Go[s] = off;
    off += K->dGo[s] * K->dGo[s];
  }
  K->D = off;
  off += lay.total - lay.pi[0];
  K->total = off;
}

// Factor accumulation during an adjoint with unit seeds.
struct KfacAcc {
  double* F;
  KfacLayout L;
};

// ---------------------------------------------------------------------------
// Tensor-core contractions of the adjoint (BF16 hi + lo operands, FP32
// accumulation in TMEM).

inline void fail_if_gram(fn_ctx* c, bool ok) {
  if (!ok) c->host_fail = true;
}

// Split count of a weight-gradient contraction: about two waves of tiles.
int tn_ksplit(long Pn, long Qn, long K) {
  int ntn = 1;
  feature_tile(Pn, &ntn);
  const long tiles = (long)ntn * ((Qn + 127) / 128);
  const long kb = K / 64;
  long want = (2L * device_sm_count() + tiles - 1) / tiles;
  if (want > kb) want = kb;
  if (want < 1) want = 1;
  const long kps = (kb + want - 1) / want;
  return (int)((kb + kps - 1) / kps);
}

// grad[p * ldg + q] += sum_k Bt[p][k] At[q][k] (k < K, a multiple of 64):
// features-on-M GEMM split over k, FP32 partials reduced in FP64.
bool tc_tn(fn_ctx* c, cudaStream_t s, long Pn, long Qn, long K, __nv_bfloat16* const at[2],
           __nv_bfloat16* const bt[2], double* grad, long ldg, float* part) {
  const bool two = c->terms > 1;
  TcGemmArgs g{};
  int ntn = 1;
  const int tn = feature_tile(Pn, &ntn);
  bool ok = tc_make_map(&g.A[0][0], at[0], Qn, K, 128) && tc_make_map(&g.B[0][0], bt[0], Pn, K, tn);
  if (two)
    ok = ok && tc_make_map(&g.A[0][1], at[1], Qn, K, 128) && tc_make_map(&g.B[0][1], bt[1], Pn, K, tn);
  else {
    g.A[0][1] = g.A[0][0];
    g.B[0][1] = g.B[0][0];
  }
  if (!ok) return false;
  g.kblocks[0] = (int)(K / 64);
  g.nseg = 1;
  g.terms = c->terms;
  g.seg_terms[0] = c->terms;
  g.rows = Pn;
  g.mfeat = (int)Qn;
  g.tile_n = tn;
  g.n_tiles_n = ntn;
  g.n_tiles_m = (int)((Qn + 127) / 128);
  g.mode = 0;
  g.out = part;
  g.ldo = Qn;
  g.bias_period = 1;
  const int ks = tn_ksplit(Pn, Qn, K);
  g.ksplit = ks;
  g.kb_per_split = (int)((K / 64 + ks - 1) / ks);
  g.split_stride = Pn * Qn;
  g.status = c->d_status;
  if (tc_gemm_launch(s, g) != FN_OK) return false;
  launch_reduce_partials(s, part, ks, Pn, Qn, grad, ldg);
  return true;
}

// out[r][j] = sum_k X[r][k] Wt[j][k] (j < Nn; k < K, a multiple of 64) in FP32:
// rows-on-lanes GEMM.
bool tc_nn(fn_ctx* c, cudaStream_t s, long rows, long Nn, long K, __nv_bfloat16* const xs[2],
           const __nv_bfloat16* wt_hi, const __nv_bfloat16* wt_lo, float* out, long ldo) {
  const bool two = c->terms > 1;
  TcGemmArgs g{};
  int ntf = 1;
  const int tf = feature_tile(Nn, &ntf, c->tune.feature_tile);
  if (!tc_segment_rm(g, 0, xs[0], two ? xs[1] : nullptr, rows, K, wt_hi, two ? wt_lo : nullptr, Nn, K, tf))
    return false;
  g.rm = 1;
  g.nseg = 1;
  g.terms = c->terms;
  g.seg_terms[0] = c->terms;
  g.rows = rows;
  g.mfeat = (int)Nn;
  g.tile_n = tf;
  g.n_tiles_n = ntf;
  g.n_tiles_m = (int)((rows + 127) / 128);
  g.mode = 0;
  g.out = out;
  g.ldo = ldo;
  g.bias_period = 1;
  g.status = c->d_status;
  return tc_gemm_launch(s, g) == FN_OK;
}

// Adjoint over one chunk on the tensor cores: the value pass is stored by the
// tensor-core forward (activations and spin means as BF16 hi + lo, tanh values
// FP32), and every contraction of the reverse pass -- weight gradients over
// the rows (operands transposed so that the rows are contiguous, split over k
// with an FP64 reduction) and backward-data products (transposed weights) --
// runs on tcgen05.  Elementwise steps, the determinant adjoint and the
// two-electron backward are those of the FP32 schedule.
void vjp_chunk_tc(fn_ctx* c, Arena& ar, const float* x, long Bc, long w0, const float* seeds, double* grad,
                  const KfacAcc* kf = nullptr) {
  const fn_net& t = c->net;
  const int n = c->n, N = c->N, L = t.n_layers, K = t.n_det, d1 = t.d1, d2 = t.d2;
  const long Ktot = (long)K * n, rows = Bc * n, pairs = Bc * n * n;
  const bool two = c->terms > 1;
  Stored st;
  float* lp = ar.get<float>(Bc);
  forward(c, ar, x, Bc, w0, false, true, FwdOut{lp, nullptr, nullptr, nullptr}, &st);
  const int max_din1 = std::max(4 * N, d1), max_din2 = std::max(4, d2);
  const long ldk = pad64(rows), ldkw = pad64(Bc), lko = pad64(Ktot), ldh = pad64(d1), ldh0 = pad64(4 * N);
  float* Obar = ar.get<float>(rows * Ktot);
  const long env_cols = (t.envelope ? 10 : 2) * Ktot * N;  // pi part, then sigma part
  float* envg = ar.get<float>(Bc * env_cols);
  float* Hbar[2] = {ar.get<float>(rows * max_din1), ar.get<float>(rows * max_din1)};
  float* Zbar = ar.get<float>(rows * d1);
  float* Ebar[2] = {ar.get<float>(pairs * max_din2), ar.get<float>(pairs * max_din2)};
  float* Z2bar = ar.get<float>(pairs * d2);
  float* S = ar.get<float>(Bc * d1);
  float* M1bar = ar.get<float>(Bc * 2 * max_din1);
  float* M2bar = ar.get<float>(rows * 2 * max_din2);
  long ta_rows = d1;
  for (int l = 0; l < L; ++l)
    ta_rows = std::max<long>({ta_rows, (long)din1_of(t, l), 2L * din2_of(t, l), 2L * din1_of(t, l)});
  __nv_bfloat16 *Xs[2] = {}, *Ss[2] = {}, *TA[2] = {}, *TB[2] = {};
  for (int h = 0; h < (two ? 2 : 1); ++h) {
    Xs[h] = ar.get<__nv_bfloat16>(rows * std::max(lko, ldh));
    Ss[h] = ar.get<__nv_bfloat16>(Bc * ldh);
    TA[h] = ar.get<__nv_bfloat16>(ta_rows * ldk);
    TB[h] = ar.get<__nv_bfloat16>(std::max<long>(Ktot, d1) * ldk);
  }
  long part_max = 0, cs_max = 0, tn_max = 0;
  auto part_need = [&](long Pn, long Qn, long Kk) { part_max = std::max(part_max, tn_ksplit(Pn, Qn, Kk) * Pn * Qn); };
  auto cs_need = [&](long r, long cl) { cs_max = std::max(cs_max, colsum_scratch_elems(r, cl)); };
  part_need(Ktot, d1, ldk);
  cs_need(Bc, env_cols);
  cs_need(rows, Ktot);
  for (int l = 0; l < L; ++l) {
    const int a1 = din1_of(t, l), a2 = din2_of(t, l);
    part_need(d1, a1, ldk);
    part_need(d1, 2 * a2, ldk);
    part_need(d1, 2 * a1, ldkw);
    cs_need(rows, d1);
    cs_need(pairs, d2);
    tn_max = std::max(tn_max, (long)gemm_tn_splits(d2, a2, pairs) * d2 * a2);
  }
  // KFAC: transposed input rows of the factor Grams, more split-K partials,
  // and the two-electron gradients materialised (separate backward kernels)
  __nv_bfloat16* TK[2] = {};
  if (kf) {
    long tk_rows = t.d1 + 1;
    for (int l = 0; l < L; ++l) {
      tk_rows = std::max(tk_rows, kf->L.dA1[l]);
      part_need(kf->L.dA1[l], kf->L.dA1[l], ldk);
      tn_max = std::max(tn_max, (long)gemm_tn_splits(din2_of(t, l), din2_of(t, l), pairs) * din2_of(t, l) *
                                    din2_of(t, l));
      tn_max = std::max(tn_max, (long)gemm_tn_splits(d2, d2, pairs) * d2 * d2);
      cs_need(pairs, din2_of(t, l));
    }
    part_need(d1, d1, ldk);
    part_need(t.d1 + 1, t.d1 + 1, ldk);
    for (int sp = 0; sp < 2; ++sp) part_need(kf->L.dGo[sp], kf->L.dGo[sp], ldk);
    for (int h = 0; h < (two ? 2 : 1); ++h) TK[h] = ar.get<__nv_bfloat16>(tk_rows * ldk);
  }
  float* part = ar.get<float>(part_max);
  double* cs_scr = ar.get<double>(cs_max);
  bool pair_bwd = c->tune.pair_unfused == 0 && !kf;
  for (int l = 0; l < L - 1 && pair_bwd; ++l) pair_bwd = pair_bwd_supported(din2_of(t, l), d2);
  float* pb_scr = pair_bwd ? ar.get<float>(pair_bwd_scratch_floats(d2, d2)) : nullptr;
  float* tn_scr = pair_bwd ? nullptr : ar.get<float>(tn_max);
  if (ar.measure) return;
  auto gram = [&](long dim, __nv_bfloat16* const rows_t[2], long ldr, double* dst) {
    if (dim > 0) fail_if_gram(c, tc_tn(c, c->stream, dim, dim, ldr, rows_t, rows_t, dst, dim, part));
  };

  cudaStream_t s = c->stream;
  const float* P = c->d_params;
  const Layout& Lo = c->lay;
  auto fail_if = [&](bool ok) {
    if (!ok) c->host_fail = true;
  };
  cudaMemsetAsync(Obar, 0, sizeof(float) * rows * Ktot, s);
  AdjDetArgs ad{};
  ad.O = st.O;
  ad.minv = st.minv;
  ad.env = st.env;
  ad.wdet = st.wdet;
  ad.seeds = seeds;
  ad.x = x;
  ad.g = geo_of(c);
  ad.w0 = w0;
  ad.Bc = Bc;
  ad.n = n;
  ad.n_up = t.n_up;
  ad.K = K;
  ad.N = N;
  ad.NS = c->ns_max;
  ad.pi[0] = P + Lo.pi[0];
  ad.pi[1] = P + Lo.pi[1];
  ad.sigma[0] = P + Lo.sigma[0];
  ad.sigma[1] = P + Lo.sigma[1];
  ad.full_env = t.envelope;
  ad.Obar = Obar;
  ad.envgrad = envg;
  launch_adj_det(s, ad);
  launch_colsum_accum(s, envg, Bc, env_cols, env_cols, grad + Lo.pi[0], cs_scr);
  if (kf) launch_colsq_accum(s, envg, Bc, env_cols, env_cols, kf->F + kf->L.D);
  // orbital weights: grad[q][f] += sum_r Obar[r][q] h^L[r][f]
  launch_t_bf16(s, st.Hb[L][0], st.Hb[L][1], ldh, rows, d1, TA[0], TA[1], ldk);
  launch_t_split(s, Obar, Ktot, rows, Ktot, TB[0], TB[1], ldk);
  fail_if(tc_tn(c, s, Ktot, d1, ldk, TA, TB, grad + Lo.w_orb, d1, part));
  if (kf) {  // orbital factors per spin: gradient rows over the spin's orbitals, inputs [h^L, 1]
    for (int sp = 0; sp < 2; ++sp) {
      const int nsp = sp == 0 ? t.n_up : t.n_down;
      if (nsp == 0) continue;
      const long q0 = sp == 0 ? 0 : (long)K * t.n_up;
      __nv_bfloat16* const gq[2] = {TB[0] + q0 * ldk, two ? TB[1] + q0 * ldk : nullptr};
      gram(kf->L.dGo[sp], gq, ldk, kf->F + kf->L.Go[sp]);
      KfacRows kr{};
      kr.seg[0] = {st.Hb[L][0], st.Hb[L][1], ldh, 0, d1, 1};
      kr.nseg = 1;
      kr.rows = rows;
      kr.cols = d1 + 1;
      kr.spin = sp;
      kr.n = n;
      kr.n_up = t.n_up;
      launch_kfac_rows(s, kr, TK[0], TK[1], ldk);
      gram(d1 + 1, TK, ldk, kf->F + kf->L.Ao[sp]);
    }
  }
  launch_colsum_accum(s, Obar, rows, Ktot, Ktot, grad + Lo.g_orb, cs_scr);
  // h^L gradient: Obar W_orb
  launch_split_bf16(s, Obar, Ktot, rows, Ktot, Xs[0], Xs[1], lko);
  fail_if(tc_nn(c, s, rows, d1, lko, Xs, c->wt_hi + c->wt_orb, c->wt_lo + c->wt_orb, Hbar[0], d1));
  int hb = 0, eb = 0;
  float* Enext = nullptr;
  bool spread_pending = false;
  for (int l = L - 1; l >= 0; --l) {
    const int a1 = din1_of(t, l), a2 = din2_of(t, l), wV = 3 * a1 + 2 * a2;
    float* Ecur = Ebar[eb];
    if (l < L - 1 && pair_bwd) {
      PairBwdArgs pb{};
      pb.Eout_bar = Enext;
      pb.M2bar = spread_pending ? M2bar : nullptr;
      pb.n = n;
      pb.n_up = t.n_up;
      pb.Y = st.Y2[l];
      pb.Ein = st.E[l];
      pb.W = P + Lo.W[l];
      pb.Ein_bar = l >= 1 ? Ecur : nullptr;
      pb.residual = l >= 1 ? 1 : 0;
      pb.pairs = pairs;
      pb.grad_W = grad + Lo.W[l];
      pb.grad_c = grad + Lo.c[l];
      pb.partial = pb_scr;
      pb.mma = 1;  // the tensor-core adjoint (mixed path)
      fail_if(launch_pair_bwd(s, pb, a2, d2));
    } else if (l < L - 1) {
      launch_tanh_bwd(s, Enext, st.Y2[l], pairs, d2, Z2bar);
      gemm_tn_accum(s, d2, a2, pairs, Z2bar, d2, st.E[l], a2, grad + Lo.W[l], a2, tn_scr,
                    gemm_tn_splits(d2, a2, pairs));
      if (kf) {  // two-electron factors (FP32 SIMT Grams over the pair rows, FP64 sums)
        gemm_tn_accum(s, d2, d2, pairs, Z2bar, d2, Z2bar, d2, kf->F + kf->L.G2[l], d2, tn_scr,
                      gemm_tn_splits(d2, d2, pairs));
        gemm_tn_accum(s, a2, a2, pairs, st.E[l], a2, st.E[l], a2, kf->F + kf->L.A2[l], a2 + 1, tn_scr,
                      gemm_tn_splits(a2, a2, pairs));
        launch_colsum_accum(s, st.E[l], pairs, a2, a2, kf->F + kf->L.A2[l] + (long)a2 * (a2 + 1), cs_scr);
      }
      launch_colsum_accum(s, Z2bar, pairs, d2, d2, grad + Lo.c[l], cs_scr);
      gemm_nn(s, pairs, a2, d2, Z2bar, d2, P + Lo.W[l], a2, Ecur, a2, Epi{});
      if (l >= 1) launch_add(s, Ecur, Enext, pairs * a2);
    } else if (!pair_bwd) {
      cudaMemsetAsync(Ecur, 0, sizeof(float) * pairs * a2, s);
    }
    float* Hcur = Hbar[hb];
    launch_tanh_bwd(s, Hcur, st.Y[l], rows, d1, Zbar);
    // V_a: grad[f][i] += sum_r Zbar[r][f] h^l[r][i]
    launch_t_bf16(s, st.Hb[l][0], st.Hb[l][1], l == 0 ? ldh0 : ldh, rows, a1, TA[0], TA[1], ldk);
    launch_t_split(s, Zbar, d1, rows, d1, TB[0], TB[1], ldk);
    fail_if(tc_tn(c, s, d1, a1, ldk, TA, TB, grad + Lo.V[l], wV, part));
    if (kf) {  // one-electron factors: pre-activation gradients and inputs [h, m_up, m_down, m2_up, m2_down, 1]
      gram(d1, TB, ldk, kf->F + kf->L.G1[l]);
      KfacRows kr{};
      kr.seg[0] = {st.Hb[l][0], st.Hb[l][1], l == 0 ? ldh0 : ldh, 0, a1, 1};
      kr.seg[1] = {st.M1b[l][0], st.M1b[l][1], pad64(2 * a1), a1, 2 * a1, n};
      kr.seg[2] = {st.M2b[l][0], st.M2b[l][1], pad64(2 * a2), 3 * a1, 2 * a2, 1};
      kr.nseg = 3;
      kr.rows = rows;
      kr.cols = wV + 1;
      kr.spin = -1;
      kr.n = n;
      kr.n_up = t.n_up;
      launch_kfac_rows(s, kr, TK[0], TK[1], ldk);
      gram(wV + 1, TK, ldk, kf->F + kf->L.A1[l]);
    }
    // V_de: the pair means
    launch_t_bf16(s, st.M2b[l][0], st.M2b[l][1], pad64(2 * a2), rows, 2 * a2, TA[0], TA[1], ldk);
    fail_if(tc_tn(c, s, d1, 2 * a2, ldk, TA, TB, grad + Lo.V[l] + 3 * a1, wV, part));
    // V_bc: per-walker sums of Zbar against the one-electron means
    launch_walker_sum(s, Zbar, Bc, n, d1, S);
    launch_t_bf16(s, st.M1b[l][0], st.M1b[l][1], pad64(2 * a1), Bc, 2 * a1, TA[0], TA[1], ldkw);
    launch_t_split(s, S, d1, Bc, d1, TB[0], TB[1], ldkw);
    fail_if(tc_tn(c, s, d1, 2 * a1, ldkw, TA, TB, grad + Lo.V[l] + a1, wV, part));
    launch_colsum_accum(s, Zbar, rows, d1, d1, grad + Lo.b[l], cs_scr);
    if (l >= 1) {
      float* Hprev = Hbar[hb ^ 1];
      launch_split_bf16(s, Zbar, d1, rows, d1, Xs[0], Xs[1], ldh);
      fail_if(tc_nn(c, s, rows, a1, ldh, Xs, c->wt_hi + c->wt_a[l], c->wt_lo + c->wt_a[l], Hprev, a1));
      launch_add(s, Hprev, Hcur, rows * a1);
      launch_split_bf16(s, S, d1, Bc, d1, Ss[0], Ss[1], ldh);
      fail_if(tc_nn(c, s, Bc, 2 * a1, ldh, Ss, c->wt_hi + c->wt_bc[l], c->wt_lo + c->wt_bc[l], M1bar, 2 * a1));
      launch_spread_mean1(s, M1bar, Bc, n, t.n_up, a1, Hprev);
      fail_if(tc_nn(c, s, rows, 2 * a2, ldh, Xs, c->wt_hi + c->wt_de[l], c->wt_lo + c->wt_de[l], M2bar, 2 * a2));
      if (pair_bwd) spread_pending = true;
      else launch_spread_mean2(s, M2bar, Bc, n, t.n_up, a2, Ecur);
      hb ^= 1;
    }
    Enext = (pair_bwd && l == L - 1) ? nullptr : Ecur;
    eb ^= 1;
  }
}

// Adjoint over one chunk: grad64 += sum_w seeds[w] d log|psi_w| / d theta.
void vjp_chunk(fn_ctx* c, Arena& ar, const float* x, long Bc, long w0, const float* seeds, double* grad) {
  if (tc_store_ok(c)) {
    vjp_chunk_tc(c, ar, x, Bc, w0, seeds, grad);
    return;
  }
  const fn_net& t = c->net;
  const int n = c->n, N = c->N, L = t.n_layers, K = t.n_det, d1 = t.d1, d2 = t.d2;
  const long Ktot = (long)K * n, rows = Bc * n, pairs = Bc * n * n;
  Stored st;
  float* lp = ar.get<float>(Bc);
  forward(c, ar, x, Bc, w0, false, true, FwdOut{lp, nullptr, nullptr, nullptr}, &st);
  const int max_din1 = std::max(4 * N, d1), max_din2 = std::max(4, d2);
  float* Obar = ar.get<float>(rows * Ktot);
  const long env_cols = (t.envelope ? 10 : 2) * Ktot * N;  // pi part, then sigma part
  float* envg = ar.get<float>(Bc * env_cols);
  float* Hbar[2] = {ar.get<float>(rows * max_din1), ar.get<float>(rows * max_din1)};
  float* Zbar = ar.get<float>(rows * d1);
  float* Ebar[2] = {ar.get<float>(pairs * max_din2), ar.get<float>(pairs * max_din2)};
  float* Z2bar = ar.get<float>(pairs * d2);
  float* S = ar.get<float>(Bc * d1);
  float* M1bar = ar.get<float>(Bc * 2 * max_din1);
  float* M2bar = ar.get<float>(rows * 2 * max_din2);
  // scratch for split-K partials and column sums
  long tn_max = 0, cs_max = 0;
  auto tn_need = [&](long M, long Nn, long Kk) {
    tn_max = std::max(tn_max, (long)gemm_tn_splits(M, Nn, Kk) * M * Nn);
  };
  auto cs_need = [&](long r, long cl) { cs_max = std::max(cs_max, colsum_scratch_elems(r, cl)); };
  tn_need(Ktot, d1, rows);
  cs_need(Bc, env_cols);
  cs_need(rows, Ktot);
  for (int l = 0; l < L; ++l) {
    const int a1 = din1_of(t, l), a2 = din2_of(t, l);
    tn_need(d2, a2, pairs);
    cs_need(pairs, d2);
    tn_need(d1, a1, rows);
    tn_need(d1, 2 * a2, rows);
    tn_need(d1, 2 * a1, Bc);
    cs_need(rows, d1);
  }
  float* tn_scr = ar.get<float>(tn_max);
  double* cs_scr = ar.get<double>(cs_max);
  // fused two-electron backward (k_pair.cu) where its kernels cover the widths
  bool pair_bwd = c->tune.pair_unfused == 0;
  for (int l = 0; l < L - 1 && pair_bwd; ++l) pair_bwd = pair_bwd_supported(din2_of(t, l), d2);
  float* pb_scr = pair_bwd ? ar.get<float>(pair_bwd_scratch_floats(d2, d2)) : nullptr;
  if (ar.measure) return;

  cudaStream_t s = c->stream;
  const float* P = c->d_params;
  const Layout& Lo = c->lay;
  auto TN = [&](long M, long Nn, long Kk, const float* A, long lda, const float* Bm, long ldb, double* gdst,
                long ldg) {
    gemm_tn_accum(s, M, Nn, Kk, A, lda, Bm, ldb, gdst, ldg, tn_scr, gemm_tn_splits(M, Nn, Kk));
  };
  cudaMemsetAsync(Obar, 0, sizeof(float) * rows * Ktot, s);
  AdjDetArgs ad{};
  ad.O = st.O;
  ad.minv = st.minv;
  ad.env = st.env;
  ad.wdet = st.wdet;
  ad.seeds = seeds;
  ad.x = x;
  ad.g = geo_of(c);
  ad.w0 = w0;
  ad.Bc = Bc;
  ad.n = n;
  ad.n_up = t.n_up;
  ad.K = K;
  ad.N = N;
  ad.NS = c->ns_max;
  ad.pi[0] = P + Lo.pi[0];
  ad.pi[1] = P + Lo.pi[1];
  ad.sigma[0] = P + Lo.sigma[0];
  ad.sigma[1] = P + Lo.sigma[1];
  ad.full_env = t.envelope;
  ad.Obar = Obar;
  ad.envgrad = envg;
  launch_adj_det(s, ad);
  launch_colsum_accum(s, envg, Bc, env_cols, env_cols, grad + Lo.pi[0], cs_scr);
  TN(Ktot, d1, rows, Obar, Ktot, st.H[L], d1, grad + Lo.w_orb, d1);
  launch_colsum_accum(s, Obar, rows, Ktot, Ktot, grad + Lo.g_orb, cs_scr);
  gemm_nn(s, rows, d1, Ktot, Obar, Ktot, P + Lo.w_orb, d1, Hbar[0], d1, Epi{});
  int hb = 0, eb = 0;
  float* Enext = nullptr;
  bool spread_pending = false;  // fused path: M2bar holds layer l + 1's pair-mean gradient
  for (int l = L - 1; l >= 0; --l) {
    const int a1 = din1_of(t, l), a2 = din2_of(t, l), wV = 3 * a1 + 2 * a2;
    const float* V = P + Lo.V[l];
    float* Ecur = Ebar[eb];
    if (l < L - 1 && pair_bwd) {
      // one pass: tanh backward, dW, dc and (l >= 1) the input gradient with
      // the residual; layer 0's input gradient is not needed
      PairBwdArgs pb{};
      pb.Eout_bar = Enext;
      pb.M2bar = spread_pending ? M2bar : nullptr;
      pb.n = n;
      pb.n_up = t.n_up;
      pb.Y = st.Y2[l];
      pb.Ein = st.E[l];
      pb.W = P + Lo.W[l];
      pb.Ein_bar = l >= 1 ? Ecur : nullptr;
      pb.residual = l >= 1 ? 1 : 0;
      pb.pairs = pairs;
      pb.grad_W = grad + Lo.W[l];
      pb.grad_c = grad + Lo.c[l];
      pb.partial = pb_scr;
      if (!launch_pair_bwd(s, pb, a2, d2)) c->host_fail = true;
    } else if (l < L - 1) {
      launch_tanh_bwd(s, Enext, st.Y2[l], pairs, d2, Z2bar);
      TN(d2, a2, pairs, Z2bar, d2, st.E[l], a2, grad + Lo.W[l], a2);
      launch_colsum_accum(s, Z2bar, pairs, d2, d2, grad + Lo.c[l], cs_scr);
      gemm_nn(s, pairs, a2, d2, Z2bar, d2, P + Lo.W[l], a2, Ecur, a2, Epi{});
      if (l >= 1) launch_add(s, Ecur, Enext, pairs * a2);
    } else if (!pair_bwd) {
      cudaMemsetAsync(Ecur, 0, sizeof(float) * pairs * a2, s);
    }
    float* Hcur = Hbar[hb];
    launch_tanh_bwd(s, Hcur, st.Y[l], rows, d1, Zbar);
    TN(d1, a1, rows, Zbar, d1, st.H[l], a1, grad + Lo.V[l], wV);
    TN(d1, 2 * a2, rows, Zbar, d1, st.M2[l], 2 * a2, grad + Lo.V[l] + 3 * a1, wV);
    launch_walker_sum(s, Zbar, Bc, n, d1, S);
    TN(d1, 2 * a1, Bc, S, d1, st.M1[l], 2 * a1, grad + Lo.V[l] + a1, wV);
    launch_colsum_accum(s, Zbar, rows, d1, d1, grad + Lo.b[l], cs_scr);
    if (l >= 1) {
      float* Hprev = Hbar[hb ^ 1];
      gemm_nn(s, rows, a1, d1, Zbar, d1, V, wV, Hprev, a1, Epi{});
      launch_add(s, Hprev, Hcur, rows * a1);
      gemm_nn(s, Bc, 2 * a1, d1, S, d1, V + a1, wV, M1bar, 2 * a1, Epi{});
      launch_spread_mean1(s, M1bar, Bc, n, t.n_up, a1, Hprev);
      gemm_nn(s, rows, 2 * a2, d1, Zbar, d1, V + 3 * a1, wV, M2bar, 2 * a2, Epi{});
      if (pair_bwd) spread_pending = true;  // added by the next pair backward as it loads
      else launch_spread_mean2(s, M2bar, Bc, n, t.n_up, a2, Ecur);
      hb ^= 1;
    }
    Enext = (pair_bwd && l == L - 1) ? nullptr : Ecur;
    eb ^= 1;
  }
}

size_t ws_bytes(fn_ctx* c, long Bc, int mode) {
  Arena ar;
  ar.measure = true;
  if (mode == 0) forward(c, ar, nullptr, Bc, 0, false, false, FwdOut{}, nullptr);
  if (mode == 1) forward(c, ar, nullptr, Bc, 0, true, false, FwdOut{}, nullptr);
  if (mode == 2) vjp_chunk(c, ar, nullptr, Bc, 0, nullptr, nullptr);
  if (mode == 3) {  // KFAC factors: the tensor-core adjoint with the factor Grams
    KfacAcc kf{};
    kfac_layout(c->net, c->lay, &kf.L);
    vjp_chunk_tc(c, ar, nullptr, Bc, 0, nullptr, nullptr, &kf);
  }
  return ar.off;
}

// Workspace budget: 30% of the device's memory, at most 80 GB (GB300: the
// whole 4096-walker local-energy pass in one chunk); FERMINET_WS_GB overrides.
double default_ws_gb() {
  static double gb[kMaxDevices];
  static PerDeviceOnce once;
  int d = 0;
  if (cudaGetDevice(&d) != cudaSuccess || d < 0 || d >= kMaxDevices) {
    cudaGetLastError();
    return 24.0;
  }
  once([&] {
    size_t freeb = 0, total = 0;
    gb[d] = 24.0;
    if (cudaMemGetInfo(&freeb, &total) == cudaSuccess && total > 0)
      gb[d] = std::min(80.0, 0.3 * (double)total / (double)(1ull << 30));
    else
      cudaGetLastError();
  });
  return gb[d];
}

// Largest chunk whose workspace fits the budget.
long chunk_for(fn_ctx* c, long B, int mode) {
  double gb = default_ws_gb();
  if (const char* v = getenv("FERMINET_WS_GB")) gb = atof(v);
  const double budget = gb * (1ull << 30);
  const double b1 = (double)ws_bytes(c, 1, mode), b2 = (double)ws_bytes(c, 2, mode);
  const double per = std::max(1.0, b2 - b1), base = std::max(0.0, b1 - per);
  long ch = (long)((budget - base) / per);
  if (ch < 1) ch = 1;
  if (ch > B) ch = B;
  if (mode == 1 && c->tune.tangent_chunk > 0 && c->tune.tangent_chunk < ch) ch = c->tune.tangent_chunk;
  if (const char* v = getenv("FERMINET_CHUNK")) {
    long f = atol(v);
    if (f > 0 && f < ch) ch = f;
  }
  return ch;
}

fn_status ensure_ws(fn_ctx* c, size_t bytes) {
  if (bytes <= c->ws_size) return FN_OK;
  CK(cudaStreamSynchronize(c->stream));
  if (c->ws) cudaFree(c->ws);
  c->ws = nullptr;
  c->ws_size = 0;
  if (cudaMalloc(&c->ws, bytes) != cudaSuccess) {
    cudaGetLastError();
    return fail(c, FN_ENOMEM, "workspace allocation failed");
  }
  c->ws_size = bytes;
  return FN_OK;
}

fn_status ensure_aux(fn_ctx* c, long B) {
  if (B <= c->aux_cap) return FN_OK;
  CK(cudaStreamSynchronize(c->stream));
  if (c->aux) cudaFree(c->aux);
  c->aux = nullptr;
  c->aux_cap = 0;
  size_t bytes = (size_t)B * (3 * c->n + 4) * sizeof(float);
  if (cudaMalloc(&c->aux, bytes) != cudaSuccess) {
    cudaGetLastError();
    return fail(c, FN_ENOMEM, "auxiliary allocation failed");
  }
  c->aux_cap = B;
  return FN_OK;
}

fn_status check_batch(fn_ctx* c, const void* x, long B) {
  if (!x && B > 0) return fail(c, FN_EINVAL, "null walker pointer");
  if (B < 0) return fail(c, FN_EINVAL, "negative batch size");
  if (c->G > 1 && B != c->geo_total)
    return fail(c, FN_EINVAL, "batch size must equal the walker total of the geometry table");
  return FN_OK;
}

fn_status after_launch(fn_ctx* c) {
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_check(c, e, "kernel launch");
  c->err.clear();
  return FN_OK;
}

// Runs `mode` passes (0 value, 1 tangent) over the batch in chunks.
fn_status run_passes(fn_ctx* c, const float* x, long B, bool tangent, const FwdOut& out) {
  if (B == 0) return FN_OK;
  const int mode = tangent ? 1 : 0;
  const long ch = chunk_for(c, B, mode);
  fn_status st = ensure_ws(c, ws_bytes(c, ch, mode));
  if (st != FN_OK) return st;
  const long n3 = 3L * c->n;
  for (long w0 = 0; w0 < B; w0 += ch) {
    const long Bc = std::min(ch, B - w0);
    Arena ar;
    ar.measure = false;
    ar.base = c->ws;
    FwdOut o;
    o.logpsi = out.logpsi ? out.logpsi + w0 : nullptr;
    o.sign = out.sign ? out.sign + w0 : nullptr;
    o.eloc = out.eloc ? out.eloc + w0 : nullptr;
    o.kinetic = out.kinetic ? out.kinetic + w0 : nullptr;
    Prof pv(c, tangent ? FN_KC_COUNT : FN_KC_VALUE_PASS, 0.0);
    forward(c, ar, x + w0 * n3, Bc, w0, tangent, false, o, nullptr);
    if (c->host_fail) {
      c->host_fail = false;
      return fail(c, FN_ECUDA, "tensor-core GEMM set-up failed (tensor map or launch)");
    }
  }
  return after_launch(c);
}

// Accumulates sum_w seeds[w] d log|psi_w| / d theta in FP64 into grad64 (the
// context's buffer unless the caller supplies one); stores it as float into
// grad when grad is given.
fn_status run_vjp(fn_ctx* c, const float* x, long B, const float* seeds, float* grad, double* grad64 = nullptr) {
  cudaStream_t s = c->stream;
  if (!grad64) grad64 = c->d_grad64;
  launch_zero_d(s, grad64, c->lay.total);
  if (B > 0) {
    const long ch = chunk_for(c, B, 2);
    fn_status st = ensure_ws(c, ws_bytes(c, ch, 2));
    if (st != FN_OK) return st;
    const long n3 = 3L * c->n;
    for (long w0 = 0; w0 < B; w0 += ch) {
      const long Bc = std::min(ch, B - w0);
      Arena ar;
      ar.measure = false;
      ar.base = c->ws;
      Prof pa(c, FN_KC_ADJOINT, 0.0);
      vjp_chunk(c, ar, x + w0 * n3, Bc, w0, seeds + w0, grad64);
    }
  }
  if (grad) launch_d2f(s, grad64, grad, c->lay.total);
  return after_launch(c);
}

// KFAC factor sums over the batch (unit seeds), then their averages.
fn_status run_kfac(fn_ctx* c, const float* x, long B, double* F) {
  cudaStream_t s = c->stream;
  KfacAcc kf{};
  kf.F = F;
  kfac_layout(c->net, c->lay, &kf.L);
  launch_zero_d(s, F, kf.L.total);
  const long ch = chunk_for(c, B, 3);
  fn_status st = ensure_ws(c, ws_bytes(c, ch, 3));
  if (st != FN_OK) return st;
  st = ensure_aux(c, std::max<long>(B, 1));
  if (st != FN_OK) return st;
  float* ones = c->aux;
  launch_fill(s, ones, 1.f, B);
  launch_zero_d(s, c->d_grad64, c->lay.total);
  const long n3 = 3L * c->n;
  for (long w0 = 0; w0 < B; w0 += ch) {
    const long Bc = std::min(ch, B - w0);
    Arena ar;
    ar.measure = false;
    ar.base = c->ws;
    vjp_chunk_tc(c, ar, x + w0 * n3, Bc, w0, ones + w0, c->d_grad64, &kf);
  }
  if (c->host_fail) {
    c->host_fail = false;
    return fail(c, FN_ECUDA, "tensor-core GEMM set-up failed (tensor map or launch)");
  }
  // averages: inputs over rows, gradients and the envelope diagonal over walkers
  const fn_net& t = c->net;
  const double Bd = (double)B, n = (double)c->n;
  std::vector<KfacBlock> blk;
  auto add = [&](long off, long dim, int diag, double scale, int mirror, double count) {
    KfacBlock b{};
    b.off = off;
    b.dim = dim;
    b.diag = diag;
    b.scale = scale;
    b.mirror_bias = mirror;
    b.count = count;
    blk.push_back(b);
  };
  for (int l = 0; l < t.n_layers; ++l) {
    add(kf.L.A1[l], kf.L.dA1[l], 0, 1.0 / (Bd * n), 0, 0.0);
    add(kf.L.G1[l], t.d1, 0, 1.0 / Bd, 0, 0.0);
  }
  for (int l = 0; l < t.n_layers - 1; ++l) {
    add(kf.L.A2[l], kf.L.dA2[l], 0, 1.0 / (Bd * n * n), 1, Bd * n * n);
    add(kf.L.G2[l], t.d2, 0, 1.0 / Bd, 0, 0.0);
  }
  for (int sp = 0; sp < 2; ++sp) {
    const double ns = sp == 0 ? t.n_up : t.n_down;
    add(kf.L.Ao[sp], t.d1 + 1, 0, ns > 0 ? 1.0 / (Bd * ns) : 0.0, 0, 0.0);
    add(kf.L.Go[sp], kf.L.dGo[sp], 0, 1.0 / Bd, 0, 0.0);
  }
  add(kf.L.D, kf.L.total - kf.L.D, 1, 1.0 / Bd, 0, 0.0);
  KfacBlock* d_blk = reinterpret_cast<KfacBlock*>(c->ws);  // the workspace is free again
  CK(cudaMemcpyAsync(d_blk, blk.data(), sizeof(KfacBlock) * blk.size(), cudaMemcpyHostToDevice, s));
  launch_kfac_finalize(s, F, d_blk, (int)blk.size());
  CK(cudaStreamSynchronize(s));  // the block table lives in pageable host memory
  return after_launch(c);
}

}  // namespace

namespace fn {

int device_sm_count() {
  static int n[kMaxDevices];
  static PerDeviceOnce once;
  int d = 0;
  if (cudaGetDevice(&d) != cudaSuccess || d < 0 || d >= kMaxDevices) {
    cudaGetLastError();
    return 148;
  }
  once([&] {
    int v = 0;
    if (cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, d) != cudaSuccess || v <= 0) {
      cudaGetLastError();
      v = 148;
    }
    n[d] = v;
  });
  return n[d];
}

// Value pass over B walkers of one geometry with a caller-supplied workspace
// and no allocation of any kind (host or device).  The first 256 bytes of ws
// hold the status and flag words; the rest is cut into walker chunks.
fn_status value_pass_fixed_workspace(const fn_net& net, const float* d_params, const float* d_R, const float* d_x,
                                     long B, float* d_logpsi, float* d_sign, cudaStream_t s, char* ws,
                                     size_t ws_size) {
  fn_ctx c;
  c.net = net;
  c.n = net.n_up + net.n_down;
  c.N = net.n_nuc;
  c.G = 1;
  c.Ct = tangent_cols(c.n);
  c.stream = s;
  c.ns_max = std::max(net.n_up, net.n_down);
  // parameter offsets only: the entry table (host memory) is not built
  build_layout(net, &c.lay, false);
  // the FP64 redo settings of ferminet_init
  if (const char* v = getenv("FERMINET_PIVOT_TAU")) c.pivot_tau = (float)atof(v);
  if (const char* v = getenv("FERMINET_DET64")) c.force64 = atoi(v) != 0;
  c.d_params = const_cast<float*>(d_params);
  c.d_R = const_cast<float*>(d_R);
  c.d_status = reinterpret_cast<unsigned*>(ws);
  c.d_flagged = reinterpret_cast<unsigned long long*>(ws + 64);
  const size_t head = 256;
  if (ws_size <= head) return FN_ENOMEM;
  const size_t avail = ws_size - head;
  const size_t b1 = ws_bytes(&c, 1, 0), b2 = ws_bytes(&c, 2, 0);
  if (b1 > avail) return FN_ENOMEM;
  const size_t per = b2 > b1 ? b2 - b1 : 1, base = b1 > per ? b1 - per : 0;
  long ch = (long)((avail - base) / per);
  if (ch < 1) ch = 1;
  while (ch > 1 && ws_bytes(&c, ch, 0) > avail) --ch;
  if (ch > B) ch = B;
  // launch errors of this call: an error already pending on this thread
  // belongs to earlier work and is left in place
  const cudaError_t prior = cudaPeekAtLastError();
  if (cudaMemsetAsync(ws, 0, head, s) != cudaSuccess) return FN_ECUDA;
  const long n3 = 3L * c.n;
  for (long w0 = 0; w0 < B; w0 += ch) {
    const long Bc = std::min(ch, B - w0);
    Arena ar;
    ar.measure = false;
    ar.base = ws + head;
    FwdOut o;
    o.logpsi = d_logpsi + w0;
    o.sign = d_sign ? d_sign + w0 : nullptr;
    forward(&c, ar, d_x + w0 * n3, Bc, w0, false, false, o, nullptr);
  }
  const cudaError_t e = cudaPeekAtLastError();
  if (e == cudaSuccess || e == prior) return FN_OK;
  cudaGetLastError();  // this call's own launch error
  return FN_ECUDA;
}

}  // namespace fn

namespace {

// Metropolis moves over the batch (counter = base + s, the base either
// `counter` or, when dctr is set, read from device memory); with the training
// option d_width the width comes from device memory and is adapted from the
// acceptance of these moves afterwards.
fn_status run_moves(fn_ctx* c, float* x, float* lp, long B, int n_steps, float width, uint64_t seed,
                    uint64_t counter, const uint64_t* dctr, int* acc) {
  const int n3 = 3 * c->n;
  float* xp = c->aux;
  float* lpp = c->aux + (size_t)B * n3;
  float* dw = c->train.d_width;
  if (dw && !acc) acc = reinterpret_cast<int*>(c->aux + (size_t)B * (n3 + 1));  // counts for the adaptation
  if (acc) cudaMemsetAsync(acc, 0, sizeof(int) * B, c->stream);
  for (int s = 0; s < n_steps; ++s) {
    const uint64_t t = (dctr ? 0 : counter) + (uint64_t)s;
    launch_propose(c->stream, x, xp, B, n3, width, seed, t, dctr, dw);
    fn_status st = run_passes(c, xp, B, false, FwdOut{lpp, nullptr, nullptr, nullptr});
    if (st != FN_OK) return st;
    launch_accept(c->stream, x, xp, lp, lpp, B, n3, seed, t, acc, dctr);
  }
  if (dw && n_steps > 0)
    launch_adapt_width(c->stream, acc, B, n_steps, dw, c->train.accept_lo, c->train.accept_hi,
                       c->train.width_factor);
  return FN_OK;
}

// Per-geometry mean energies into emean and the gradient seeds (clipped when
// the training option asks for it).
void energy_seeds(fn_ctx* c, const float* eloc, long B, double* emean, float* seeds) {
  const long B1 = c->G > 1 ? -1 : B;
  const int* geo = c->G > 1 ? c->d_geo : nullptr;
  launch_emean(c->stream, eloc, c->G, c->d_geo_off, c->d_geo_cnt, B1, emean);
  if (c->train.clip_scale > 0.f)
    launch_clip_seeds(c->stream, eloc, B, geo, c->G, c->d_geo_off, c->d_geo_cnt, B1, (double)c->train.clip_scale,
                      c->d_clip_stats, seeds);
  else
    launch_seeds(c->stream, eloc, B, geo, emean, c->d_geo_cnt, B1, seeds);
}

// The whole VMC step: n_steps Metropolis moves, then the local energy at the
// new positions, then the VMC energy gradient.
fn_status run_step(fn_ctx* c, float* x, float* lp, long B, int n_steps, float width, uint64_t seed,
                   uint64_t counter, const uint64_t* dctr, float* eloc, double* emean, float* grad, int* acc) {
  float* seeds = c->aux;  // reused after the moves
  fn_status st = run_moves(c, x, lp, B, n_steps, width, seed, counter, dctr, acc);
  if (st != FN_OK) return st;
  st = run_passes(c, x, B, true, FwdOut{nullptr, nullptr, eloc, nullptr});
  if (st != FN_OK) return st;
  energy_seeds(c, eloc, B, emean, seeds);
  return run_vjp(c, x, B, seeds, grad);
}

// Workspace large enough for every pass of a step (so a captured step never
// allocates).
fn_status ensure_step_ws(fn_ctx* c, long B) {
  size_t need = 0;
  for (int mode = 0; mode < 3; ++mode) {
    const long ch = chunk_for(c, B, mode);
    need = std::max(need, ws_bytes(c, ch, mode));
  }
  return ensure_ws(c, need);
}

}  // namespace

// ---------------------------------------------------------------------------
// C ABI
// ---------------------------------------------------------------------------

extern "C" {

fn_status ferminet_init(const fn_net* net, const fn_geometry* geoms, int n_geoms, fn_precision prec, void* stream,
                        fn_ctx** out) {
  if (!out) return FN_EINVAL;
  *out = nullptr;
  if (!net || !geoms || n_geoms < 1) return FN_EINVAL;
  const fn_net& t = *net;
  if (t.n_layers < 1 || t.n_layers > 16 || t.d1 < 1 || t.d2 < 1 || t.d2 > 32 || t.n_det < 1 || t.n_up < 0 ||
      t.n_down < 0 || t.n_up + t.n_down < 1 || t.n_up > 32 || t.n_down > 32 || t.n_nuc < 1 ||
      t.envelope < 0 || t.envelope > 1)
    return FN_EINVAL;
  if (prec != FN_PREC_FP32 && prec != FN_PREC_MIXED) return FN_EINVAL;
  for (int g = 0; g < n_geoms; ++g)
    if (!geoms[g].R || !geoms[g].Z) return FN_EINVAL;
  fn_ctx* c = new fn_ctx();
  c->net = t;
  c->n = t.n_up + t.n_down;
  c->N = t.n_nuc;
  c->G = n_geoms;
  c->Ct = tangent_cols(c->n);
  c->prec = prec;
  c->stream = (cudaStream_t)stream;
  c->ns_max = std::max(t.n_up, t.n_down);
  if (const char* v = getenv("FERMINET_PIVOT_TAU")) c->pivot_tau = (float)atof(v);
  if (const char* v = getenv("FERMINET_DET64")) c->force64 = atoi(v) != 0;
  build_layout(t, &c->lay);
  // geometry table
  if (n_geoms > 1) {
    std::vector<std::pair<long, long>> r;
    for (int g = 0; g < n_geoms; ++g) r.push_back({geoms[g].walker_offset, geoms[g].walker_count});
    long expect = 0;
    for (int g = 0; g < n_geoms; ++g) {
      if (r[g].first != expect || r[g].second < 0) {
        delete c;
        return FN_EINVAL;
      }
      expect += r[g].second;
    }
    c->geo_total = expect;
  }
  std::vector<float> R((size_t)n_geoms * c->N * 3), Z((size_t)n_geoms * c->N);
  std::vector<double> Enn(n_geoms);
  std::vector<long> off(n_geoms), cnt(n_geoms);
  std::vector<int> geo(std::max<long>(c->geo_total, 1));
  for (int g = 0; g < n_geoms; ++g) {
    double e = 0.0;
    for (int I = 0; I < c->N; ++I) {
      for (int a = 0; a < 3; ++a) R[((size_t)g * c->N + I) * 3 + a] = (float)geoms[g].R[3 * I + a];
      Z[(size_t)g * c->N + I] = (float)geoms[g].Z[I];
      for (int J = 0; J < I; ++J) {
        double d2 = 0;
        for (int a = 0; a < 3; ++a) {
          double d = geoms[g].R[3 * I + a] - geoms[g].R[3 * J + a];
          d2 += d * d;
        }
        e += geoms[g].Z[I] * geoms[g].Z[J] / std::sqrt(d2);
      }
    }
    Enn[g] = e;
    off[g] = geoms[g].walker_offset;
    cnt[g] = geoms[g].walker_count;
    if (n_geoms > 1)
      for (long w = 0; w < cnt[g]; ++w) geo[off[g] + w] = g;
  }
  auto bad = [&](cudaError_t e) {
    if (e != cudaSuccess) {
      cudaGetLastError();
      ferminet_destroy(c);
      return true;
    }
    return false;
  };
  if (bad(cudaGetDevice(&c->device))) return FN_ECUDA;
  if (bad(cudaMalloc(&c->d_params, sizeof(float) * std::max<long>(c->lay.total, 1)))) return FN_ENOMEM;
  if (bad(cudaMalloc(&c->d_grad64, sizeof(double) * std::max<long>(c->lay.total, 1)))) return FN_ENOMEM;
  if (bad(cudaMalloc(&c->d_R, sizeof(float) * R.size()))) return FN_ENOMEM;
  if (bad(cudaMalloc(&c->d_Z, sizeof(float) * Z.size()))) return FN_ENOMEM;
  if (bad(cudaMalloc(&c->d_Enn64, sizeof(double) * n_geoms))) return FN_ENOMEM;
  if (bad(cudaMalloc(&c->d_geo, sizeof(int) * geo.size()))) return FN_ENOMEM;
  if (bad(cudaMalloc(&c->d_geo_off, sizeof(long) * n_geoms))) return FN_ENOMEM;
  if (bad(cudaMalloc(&c->d_geo_cnt, sizeof(long) * n_geoms))) return FN_ENOMEM;
  if (bad(cudaMalloc(&c->d_clip_stats, sizeof(double) * 3 * n_geoms))) return FN_ENOMEM;
  if (bad(cudaMalloc(&c->d_status, sizeof(unsigned)))) return FN_ENOMEM;
  if (bad(cudaMalloc(&c->d_flagged, sizeof(unsigned long long)))) return FN_ENOMEM;
  if (bad(cudaMemset(c->d_params, 0, sizeof(float) * std::max<long>(c->lay.total, 1)))) return FN_ECUDA;
  if (bad(cudaMemcpy(c->d_R, R.data(), sizeof(float) * R.size(), cudaMemcpyHostToDevice))) return FN_ECUDA;
  if (bad(cudaMemcpy(c->d_Z, Z.data(), sizeof(float) * Z.size(), cudaMemcpyHostToDevice))) return FN_ECUDA;
  if (bad(cudaMemcpy(c->d_Enn64, Enn.data(), sizeof(double) * n_geoms, cudaMemcpyHostToDevice))) return FN_ECUDA;
  if (bad(cudaMemcpy(c->d_geo, geo.data(), sizeof(int) * geo.size(), cudaMemcpyHostToDevice))) return FN_ECUDA;
  if (bad(cudaMemcpy(c->d_geo_off, off.data(), sizeof(long) * n_geoms, cudaMemcpyHostToDevice))) return FN_ECUDA;
  if (bad(cudaMemcpy(c->d_geo_cnt, cnt.data(), sizeof(long) * n_geoms, cudaMemcpyHostToDevice))) return FN_ECUDA;
  if (bad(cudaMemset(c->d_status, 0, sizeof(unsigned)))) return FN_ECUDA;
  if (bad(cudaMemset(c->d_flagged, 0, sizeof(unsigned long long)))) return FN_ECUDA;
  if (prec == FN_PREC_MIXED) {
    c->terms = 3;
    if (const char* v = getenv("FERMINET_MIXED_TERMS")) c->terms = atoi(v) == 1 ? 1 : 3;
    long off = 0;
    for (int l = 0; l < t.n_layers; ++l) {
      const int a1 = din1_of(t, l), a2 = din2_of(t, l);
      c->ld_a[l] = pad64(a1);
      c->ld_bc[l] = pad64(2 * a1);
      c->ld_de[l] = pad64(2 * a2);
      c->wb_a[l] = off;
      off += (long)t.d1 * c->ld_a[l];
      c->wb_bc[l] = off;
      off += (long)t.d1 * c->ld_bc[l];
      c->wb_de[l] = off;
      off += (long)t.d1 * c->ld_de[l];
    }
    c->ld_orb = pad64(t.d1);
    c->wb_orb = off;
    off += (long)t.n_det * c->n * c->ld_orb;
    c->wb_total = off;
    long toff = 0;
    const long ldt = pad64(t.d1);
    for (int l = 0; l < t.n_layers; ++l) {
      const int a1 = din1_of(t, l), a2 = din2_of(t, l);
      c->wt_a[l] = toff;
      toff += (long)a1 * ldt;
      c->wt_bc[l] = toff;
      toff += 2L * a1 * ldt;
      c->wt_de[l] = toff;
      toff += 2L * a2 * ldt;
    }
    c->wt_orb = toff;
    toff += (long)t.d1 * pad64((long)t.n_det * c->n);
    if (bad(cudaMalloc(&c->wt_hi, sizeof(__nv_bfloat16) * toff))) return FN_ENOMEM;
    if (bad(cudaMalloc(&c->wt_lo, sizeof(__nv_bfloat16) * toff))) return FN_ENOMEM;
    if (bad(cudaMalloc(&c->wb_hi, sizeof(__nv_bfloat16) * off))) return FN_ENOMEM;
    if (bad(cudaMalloc(&c->wb_lo, sizeof(__nv_bfloat16) * off))) return FN_ENOMEM;
    if (bad(cudaMemset(c->wb_hi, 0, sizeof(__nv_bfloat16) * off))) return FN_ECUDA;
    if (bad(cudaMemset(c->wb_lo, 0, sizeof(__nv_bfloat16) * off))) return FN_ECUDA;
    c->tc_ok = tc_encode_ready();
    std::vector<__nv_bfloat16> eye(128 * 128, __float2bfloat16(0.f));
    for (int i = 0; i < 128; ++i) eye[i * 128 + i] = __float2bfloat16(1.f);
    if (bad(cudaMalloc(&c->ident, sizeof(__nv_bfloat16) * eye.size()))) return FN_ENOMEM;
    if (bad(cudaMemcpy(c->ident, eye.data(), sizeof(__nv_bfloat16) * eye.size(), cudaMemcpyHostToDevice)))
      return FN_ECUDA;
  }
  *out = c;
  return FN_OK;
}

fn_status ferminet_param_layout(const fn_ctx* c, fn_param_entry* out, int max_entries, int* n_entries,
                                long* n_params) {
  if (!c) return FN_EINVAL;
  const int ne = (int)c->lay.entries.size();
  if (out)
    for (int i = 0; i < ne && i < max_entries; ++i) out[i] = c->lay.entries[i];
  if (n_entries) *n_entries = ne;
  if (n_params) *n_params = c->lay.total;
  return FN_OK;
}

fn_status ferminet_net_layout(const fn_net* net, fn_param_entry* out, int max_entries, int* n_entries,
                              long* n_params) {
  if (!net || net->n_layers < 1 || net->n_layers > 16 || net->d1 < 1 || net->d2 < 1 || net->n_det < 1 ||
      net->n_up < 0 || net->n_down < 0 || net->n_up + net->n_down < 1 || net->n_nuc < 1 ||
      net->envelope < 0 || net->envelope > 1)
    return FN_EINVAL;
  Layout L;
  build_layout(*net, &L);
  const int ne = (int)L.entries.size();
  if (out)
    for (int i = 0; i < ne && i < max_entries; ++i) out[i] = L.entries[i];
  if (n_entries) *n_entries = ne;
  if (n_params) *n_params = L.total;
  return FN_OK;
}

fn_status ferminet_set_params(fn_ctx* c, const float* d_params) {
  if (!c) return FN_EINVAL;
  if (!d_params) return fail(c, FN_EINVAL, "null parameter pointer");
  CK(cudaMemcpyAsync(c->d_params, d_params, sizeof(float) * c->lay.total, cudaMemcpyDeviceToDevice, c->stream));
  if (c->prec == FN_PREC_MIXED && c->wb_hi) {
    const fn_net& t = c->net;
    const float* P = c->d_params;
    for (int l = 0; l < t.n_layers; ++l) {
      const int a1 = din1_of(t, l), a2 = din2_of(t, l), wV = 3 * a1 + 2 * a2;
      const float* V = P + c->lay.V[l];
      launch_split_bf16(c->stream, V, wV, t.d1, a1, c->wb_hi + c->wb_a[l], c->wb_lo + c->wb_a[l], c->ld_a[l]);
      launch_split_bf16(c->stream, V + a1, wV, t.d1, 2 * a1, c->wb_hi + c->wb_bc[l], c->wb_lo + c->wb_bc[l],
                        c->ld_bc[l]);
      launch_split_bf16(c->stream, V + 3 * a1, wV, t.d1, 2 * a2, c->wb_hi + c->wb_de[l], c->wb_lo + c->wb_de[l],
                        c->ld_de[l]);
    }
    launch_split_bf16(c->stream, P + c->lay.w_orb, t.d1, (long)t.n_det * c->n, t.d1, c->wb_hi + c->wb_orb,
                      c->wb_lo + c->wb_orb, c->ld_orb);
    // transposed copies for the backward-data products of the adjoint
    const long ldt = pad64(t.d1), Ktot = (long)t.n_det * c->n;
    for (int l = 0; l < t.n_layers; ++l) {
      const int a1 = din1_of(t, l), a2 = din2_of(t, l), wV = 3 * a1 + 2 * a2;
      const float* V = P + c->lay.V[l];
      launch_t_split(c->stream, V, wV, t.d1, a1, c->wt_hi + c->wt_a[l], c->wt_lo + c->wt_a[l], ldt);
      launch_t_split(c->stream, V + a1, wV, t.d1, 2 * a1, c->wt_hi + c->wt_bc[l], c->wt_lo + c->wt_bc[l], ldt);
      launch_t_split(c->stream, V + 3 * a1, wV, t.d1, 2 * a2, c->wt_hi + c->wt_de[l], c->wt_lo + c->wt_de[l], ldt);
    }
    launch_t_split(c->stream, P + c->lay.w_orb, t.d1, Ktot, t.d1, c->wt_hi + c->wt_orb, c->wt_lo + c->wt_orb,
                   pad64(Ktot));
    CK(cudaGetLastError());
  }
  c->err.clear();
  return FN_OK;
}

fn_status ferminet_logpsi(fn_ctx* c, const float* d_x, long B, float* d_logpsi, float* d_sign) {
  if (!c) return FN_EINVAL;
  fn_status st = check_batch(c, d_x, B);
  if (st != FN_OK) return st;
  if (!d_logpsi && B > 0) return fail(c, FN_EINVAL, "null logpsi pointer");
  return run_passes(c, d_x, B, false, FwdOut{d_logpsi, d_sign, nullptr, nullptr});
}

fn_status ferminet_local_energy(fn_ctx* c, const float* d_x, long B, float* d_eloc, float* d_logpsi, float* d_sign,
                                float* d_kinetic) {
  if (!c) return FN_EINVAL;
  fn_status st = check_batch(c, d_x, B);
  if (st != FN_OK) return st;
  if (!d_eloc && B > 0) return fail(c, FN_EINVAL, "null eloc pointer");
  return run_passes(c, d_x, B, true, FwdOut{d_logpsi, d_sign, d_eloc, d_kinetic});
}

fn_status ferminet_logpsi_vjp(fn_ctx* c, const float* d_x, long B, const float* d_seeds, float* d_grad) {
  if (!c) return FN_EINVAL;
  fn_status st = check_batch(c, d_x, B);
  if (st != FN_OK) return st;
  if (!d_grad || (!d_seeds && B > 0)) return fail(c, FN_EINVAL, "null seeds or grad pointer");
  return run_vjp(c, d_x, B, d_seeds, d_grad);
}

fn_status ferminet_energy_grad(fn_ctx* c, const float* d_x, long B, const float* d_eloc, double* d_emean,
                               float* d_grad) {
  if (!c) return FN_EINVAL;
  fn_status st = check_batch(c, d_x, B);
  if (st != FN_OK) return st;
  if (!d_grad || !d_emean || (!d_eloc && B > 0)) return fail(c, FN_EINVAL, "null eloc, emean or grad pointer");
  st = ensure_aux(c, std::max<long>(B, 1));
  if (st != FN_OK) return st;
  float* seeds = c->aux;
  energy_seeds(c, d_eloc, B, d_emean, seeds);
  return run_vjp(c, d_x, B, seeds, d_grad);
}

fn_status ferminet_energy_sums(fn_ctx* c, const float* d_eloc, long B, double* d_sums) {
  if (!c) return FN_EINVAL;
  if (B < 0) return fail(c, FN_EINVAL, "negative batch size");
  if (c->G > 1 && B != c->geo_total)
    return fail(c, FN_EINVAL, "batch size must equal the walker total of the geometry table");
  if (!d_sums || (!d_eloc && B > 0)) return fail(c, FN_EINVAL, "null eloc or sums pointer");
  launch_esum(c->stream, d_eloc, c->G, c->d_geo_off, c->d_geo_cnt, c->G > 1 ? -1 : B, d_sums);
  return after_launch(c);
}

fn_status ferminet_energy_grad_partial(fn_ctx* c, const float* d_x, long B, const float* d_eloc,
                                       const double* d_esum, const double* d_count, double* d_emean,
                                       double* d_grad64) {
  if (!c) return FN_EINVAL;
  fn_status st = check_batch(c, d_x, B);
  if (st != FN_OK) return st;
  if (!d_grad64 || !d_esum || !d_count || (!d_eloc && B > 0))
    return fail(c, FN_EINVAL, "null eloc, energy sum, count or grad pointer");
  if (c->train.clip_scale > 0.f)
    return fail(c, FN_EINVAL, "the replica form does not clip: a median is not a sum over processes");
  st = ensure_aux(c, std::max<long>(B, 1));
  if (st != FN_OK) return st;
  float* seeds = c->aux;
  launch_seeds_given(c->stream, d_eloc, B, c->G > 1 ? c->d_geo : nullptr, d_esum, d_count, c->G, d_emean, seeds);
  return run_vjp(c, d_x, B, seeds, nullptr, d_grad64);
}

fn_status ferminet_mcmc_step(fn_ctx* c, float* d_x, float* d_logpsi, long B, int n_steps, float width, uint64_t seed,
                             uint64_t counter, int* d_accepted) {
  if (!c) return FN_EINVAL;
  fn_status st = check_batch(c, d_x, B);
  if (st != FN_OK) return st;
  if (!d_logpsi && B > 0) return fail(c, FN_EINVAL, "null logpsi pointer");
  if (n_steps < 0 || !(width >= 0.f)) return fail(c, FN_EINVAL, "bad step count or width");
  if (B == 0) return FN_OK;
  st = ensure_aux(c, B);
  if (st != FN_OK) return st;
  st = run_moves(c, d_x, d_logpsi, B, n_steps, width, seed, counter, nullptr, d_accepted);
  if (st != FN_OK) return st;
  return after_launch(c);
}

fn_status ferminet_set_train_opts(fn_ctx* c, const fn_train_opts* o) {
  if (!c || !o) return FN_EINVAL;
  if (!(o->clip_scale >= 0.f)) return fail(c, FN_EINVAL, "clip_scale must be >= 0");
  if (o->d_width && !(o->width_factor >= 1.f && o->accept_lo >= 0.f && o->accept_lo <= o->accept_hi &&
                      o->accept_hi <= 1.f))
    return fail(c, FN_EINVAL, "width adaptation needs 0 <= accept_lo <= accept_hi <= 1 and width_factor >= 1");
  c->train = *o;
  if (c->step_exec) {  // a captured step holds the old options
    cudaGraphExecDestroy(c->step_exec);
    c->step_exec = nullptr;
  }
  return FN_OK;
}

fn_status ferminet_kfac_size(const fn_net* net, long* n_doubles) {
  if (!net || !n_doubles) return FN_EINVAL;
  long np = 0;
  int ne = 0;
  fn_status st = ferminet_net_layout(net, nullptr, 0, &ne, &np);
  if (st != FN_OK) return st;
  Layout lay;
  build_layout(*net, &lay, false);
  KfacLayout K;
  kfac_layout(*net, lay, &K);
  *n_doubles = K.total;
  return FN_OK;
}

fn_status ferminet_kfac_factors(fn_ctx* c, const float* d_x, long B, double* d_factors) {
  if (!c) return FN_EINVAL;
  fn_status st = check_batch(c, d_x, B);
  if (st != FN_OK) return st;
  if (B < 1 || !d_factors) return fail(c, FN_EINVAL, "empty batch or null factor buffer");
  if (!tc_store_ok(c)) return fail(c, FN_EINVAL, "KFAC factors need a mixed-precision context (tensor-core adjoint)");
  return run_kfac(c, d_x, B, d_factors);
}

fn_status ferminet_kfac_precondition(fn_ctx* c, const double* d_factors, const float* d_grad, float lambda,
                                     float* d_out) {
  if (!c) return FN_EINVAL;
  if (!d_factors || !d_grad || !d_out) return fail(c, FN_EINVAL, "null factor, gradient or output pointer");
  if (!(lambda > 0.f)) return fail(c, FN_EINVAL, "lambda must be positive");
  const fn_net& t = c->net;
  const Layout& Lo = c->lay;
  cudaStream_t s = c->stream;
  KfacLayout K;
  kfac_layout(t, Lo, &K);
  // blocks to invert, each with its slot in the two inversion workspaces
  struct Blk {
    long W_off, b_off, rows, cols;  // gradient block [rows][cols - 1] + bias [rows]
    int gi, ai;                     // indices of its G and A factors in the table
  };
  std::vector<KfacBlock> tab;
  std::vector<Blk> work;
  long wsz = 0, maxd = 0, maxm = 0;
  auto fac = [&](long off, long dim) {
    KfacBlock b{};
    b.off = off;
    b.dim = dim;
    b.woff = wsz;
    wsz += dim * dim;
    maxd = std::max(maxd, dim);
    tab.push_back(b);
    return (int)tab.size() - 1;
  };
  for (int l = 0; l < t.n_layers; ++l) {
    const long a = K.dA1[l];
    work.push_back({Lo.V[l], Lo.b[l], (long)t.d1, a, fac(K.G1[l], t.d1), fac(K.A1[l], a)});
  }
  for (int l = 0; l < t.n_layers - 1; ++l) {
    const long a = K.dA2[l];
    work.push_back({Lo.W[l], Lo.c[l], (long)t.d2, a, fac(K.G2[l], t.d2), fac(K.A2[l], a)});
  }
  for (int sp = 0; sp < 2; ++sp) {
    if (K.dGo[sp] == 0) continue;
    const long wo = sp == 0 ? Lo.w_orb : Lo.w_orb + (long)t.n_det * t.n_up * t.d1;
    const long go = sp == 0 ? Lo.g_orb : Lo.g_orb + (long)t.n_det * t.n_up;
    work.push_back({wo, go, K.dGo[sp], (long)t.d1 + 1, fac(K.Go[sp], K.dGo[sp]), fac(K.Ao[sp], t.d1 + 1)});
  }
  for (const Blk& b : work) maxm = std::max(maxm, b.rows * b.cols);
  // workspace: block table, two FP64 inversion copies, FP32 inverses and products
  const size_t bytes = 256 * ((sizeof(KfacBlock) * tab.size() + 255) / 256) + sizeof(double) * 2 * wsz +
                       sizeof(float) * (wsz + 3 * maxm) + 1024;
  fn_status st = ensure_ws(c, bytes);
  if (st != FN_OK) return st;
  Arena ar;
  ar.measure = false;
  ar.base = c->ws;
  KfacBlock* d_tab = ar.get<KfacBlock>(tab.size());
  double* w0 = ar.get<double>(wsz);
  double* w1 = ar.get<double>(wsz);
  float* inv32 = ar.get<float>(wsz);
  float* M = ar.get<float>(maxm);
  float* X = ar.get<float>(maxm);
  float* Dl = ar.get<float>(maxm);
  CK(cudaMemcpyAsync(d_tab, tab.data(), sizeof(KfacBlock) * tab.size(), cudaMemcpyHostToDevice, s));
  launch_kfac_invert(s, d_factors, d_tab, (int)tab.size(), (int)maxd, std::sqrt((double)lambda), w0, w1);
  for (const KfacBlock& b : tab)  // the inverse of a block of dimension d ends in w0 (d even) or w1 (d odd)
    launch_to_float(s, (b.dim % 2 == 0 ? w0 : w1) + b.woff, inv32 + b.woff, b.dim * b.dim);
  // grad entries not covered by a block (none with this layout) pass through
  CK(cudaMemcpyAsync(d_out, d_grad, sizeof(float) * Lo.total, cudaMemcpyDeviceToDevice, s));
  for (const Blk& b : work) {
    const float* Gi = inv32 + tab[b.gi].woff;
    const float* Ai = inv32 + tab[b.ai].woff;
    launch_gather_wb(s, d_grad, b.W_off, b.b_off, b.rows, b.cols, M);
    gemm_nn(s, b.rows, b.cols, b.rows, Gi, b.rows, M, b.cols, X, b.cols, Epi{});
    gemm_nn(s, b.rows, b.cols, b.cols, X, b.cols, Ai, b.cols, Dl, b.cols, Epi{});
    launch_scatter_wb(s, Dl, b.W_off, b.b_off, b.rows, b.cols, d_out);
  }
  launch_diag_precond(s, d_grad + Lo.pi[0], d_factors + K.D, Lo.total - Lo.pi[0], (double)lambda,
                      d_out + Lo.pi[0]);
  CK(cudaStreamSynchronize(s));  // the block table lives in pageable host memory
  return after_launch(c);
}

fn_status ferminet_step(fn_ctx* c, float* d_x, float* d_logpsi, long B, int n_steps, float width, uint64_t seed,
                        uint64_t counter, float* d_eloc, double* d_emean, float* d_grad, int* d_accepted,
                        int use_graph) {
  if (!c) return FN_EINVAL;
  fn_status st = check_batch(c, d_x, B);
  if (st != FN_OK) return st;
  if (B < 1 || !d_logpsi || !d_eloc || !d_emean || !d_grad) return fail(c, FN_EINVAL, "null step buffer");
  if (n_steps < 0 || !(width >= 0.f)) return fail(c, FN_EINVAL, "bad step count or width");
  st = ensure_aux(c, B);
  if (st != FN_OK) return st;
  st = ensure_step_ws(c, B);
  if (st != FN_OK) return st;
  if (!use_graph)
    return run_step(c, d_x, d_logpsi, B, n_steps, width, seed, counter, nullptr, d_eloc, d_emean, d_grad,
                    d_accepted) == FN_OK
               ? after_launch(c)
               : FN_ECUDA;
  if (!c->d_counter) CK(cudaMalloc(&c->d_counter, sizeof(uint64_t)));
  if (!c->graph_stream) {
    CK(cudaStreamCreateWithFlags(&c->graph_stream, cudaStreamNonBlocking));
    CK(cudaEventCreateWithFlags(&c->ev_in, cudaEventDisableTiming));
    CK(cudaEventCreateWithFlags(&c->ev_out, cudaEventDisableTiming));
  }
  cudaStream_t user = c->stream, gs = c->graph_stream;
  CK(cudaEventRecord(c->ev_in, user));
  CK(cudaStreamWaitEvent(gs, c->ev_in, 0));
  fn_ctx::StepKey key;
  memset(&key, 0, sizeof key);  // padding bytes take part in the comparison
  key.B = B;
  key.n_steps = n_steps;
  key.width = width;
  key.seed = seed;
  key.x = d_x;
  key.lp = d_logpsi;
  key.eloc = d_eloc;
  key.emean = d_emean;
  key.grad = d_grad;
  key.acc = d_accepted;
  key.ws = c->ws;
  key.aux = c->aux;
  key.ws_size = c->ws_size;
  key.dwidth = c->train.d_width;
  key.clip = c->train.clip_scale;
  const bool same = c->step_exec && memcmp(&key, &c->step_key, sizeof key) == 0;
  launch_set_u64(gs, c->d_counter, counter);
  if (!same) {
    if (c->step_exec) {
      cudaGraphExecDestroy(c->step_exec);
      c->step_exec = nullptr;
    }
    const bool prof = c->prof_on;
    c->prof_on = false;  // no event records inside the captured graph
    cudaGraph_t graph = nullptr;
    CK(cudaStreamBeginCapture(gs, cudaStreamCaptureModeThreadLocal));
    c->stream = gs;
    fn_status rs = run_step(c, d_x, d_logpsi, B, n_steps, width, seed, 0, c->d_counter, d_eloc, d_emean, d_grad,
                            d_accepted);
    c->stream = user;
    cudaError_t ce = cudaStreamEndCapture(gs, &graph);
    c->prof_on = prof;
    if (rs != FN_OK || ce != cudaSuccess) {
      if (graph) cudaGraphDestroy(graph);
      cudaGetLastError();
      return fail(c, FN_ECUDA, "step capture failed");
    }
    cudaError_t ie = cudaGraphInstantiate(&c->step_exec, graph, 0);
    cudaGraphDestroy(graph);
    if (ie != cudaSuccess) {
      c->step_exec = nullptr;
      cudaGetLastError();
      return fail(c, FN_ECUDA, "step graph instantiation failed");
    }
    c->step_key = key;
  }
  CK(cudaGraphLaunch(c->step_exec, gs));
  CK(cudaEventRecord(c->ev_out, gs));
  CK(cudaStreamWaitEvent(user, c->ev_out, 0));
  return after_launch(c);
}

fn_status ferminet_get_tuning(const fn_ctx* c, fn_tuning* out) {
  if (!c || !out) return FN_EINVAL;
  *out = c->tune;
  return FN_OK;
}

fn_status ferminet_set_tuning(fn_ctx* c, const fn_tuning* t) {
  if (!c || !t) return FN_EINVAL;
  if (t->layer_groups < 0 || t->feature_tile < 0 || t->tangent_chunk < 0 || t->residual_smem < 0 ||
      t->residual_smem > 1 || t->pair_unfused < 0 || t->pair_unfused > 1 || t->adjoint_simt < 0 ||
      t->adjoint_simt > 1 || t->orbital_joint < 0 || t->orbital_joint > 1)
    return fail(c, FN_EINVAL, "bad tuning value");
  if (t->layer_groups > 0 && (t->layer_groups * c->Ct > 256 || (t->layer_groups * c->Ct) % 16))
    return fail(c, FN_EINVAL, "layer_groups gives an invalid tile");
  if (t->feature_tile > 0 && (t->feature_tile > 256 || t->feature_tile % 16))
    return fail(c, FN_EINVAL, "feature_tile must be a multiple of 16 up to 256");
  c->tune = *t;
  if (c->step_exec) {  // a captured step holds the old tile shapes
    cudaGraphExecDestroy(c->step_exec);
    c->step_exec = nullptr;
  }
  return FN_OK;
}

fn_status ferminet_autotune(fn_ctx* c, const float* d_x, long B, int repeats, fn_tuning* best) {
  if (!c) return FN_EINVAL;
  fn_status st = check_batch(c, d_x, B);
  if (st != FN_OK) return st;
  if (B < 1) return fail(c, FN_EINVAL, "empty batch");
  if (repeats < 1) repeats = 1;
  float* eloc = nullptr;
  CK(cudaMalloc(&eloc, sizeof(float) * B));
  std::vector<int> groups = {0};
  for (int g = 1; g * c->Ct <= 256; ++g)
    if ((g * c->Ct) % 16 == 0) groups.push_back(g);
  const std::vector<int> ftiles = {0, 128, 192};
  const long full = chunk_for(c, B, 1);
  std::vector<long> chunks = {0};
  if (full > 1) chunks.push_back((full + 1) / 2);
  cudaEvent_t e0, e1;
  CK(cudaEventCreate(&e0));
  CK(cudaEventCreate(&e1));
  const fn_tuning saved = c->tune;
  fn_tuning bestt = saved;
  float best_ms = 1e30f;
  for (int g : groups)
    for (int ft : ftiles)
      for (long ch : chunks)
        for (int rs = 0; rs < 2; ++rs) {
        c->tune.layer_groups = g;
        c->tune.feature_tile = ft;
        c->tune.tangent_chunk = ch;
        c->tune.residual_smem = rs;
        float tmin = 1e30f;
        for (int r = 0; r <= repeats; ++r) {  // first run warms up (and sizes the workspace)
          cudaEventRecord(e0, c->stream);
          st = run_passes(c, d_x, B, true, FwdOut{nullptr, nullptr, eloc, nullptr});
          cudaEventRecord(e1, c->stream);
          if (st != FN_OK) break;
          cudaEventSynchronize(e1);
          float ms = 0.f;
          cudaEventElapsedTime(&ms, e0, e1);
          if (r > 0 && ms < tmin) tmin = ms;
        }
        if (st != FN_OK) break;
        if (tmin < best_ms) {
          best_ms = tmin;
          bestt = c->tune;
        }
        }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaFree(eloc);
  if (st != FN_OK) {
    c->tune = saved;
    return st;
  }
  c->tune = bestt;
  if (c->step_exec) {
    cudaGraphExecDestroy(c->step_exec);
    c->step_exec = nullptr;
  }
  if (best) *best = bestt;
  return after_launch(c);
}

fn_status ferminet_sync(fn_ctx* c) {
  if (!c) return FN_EINVAL;
  CK(cudaStreamSynchronize(c->stream));
  unsigned st = 0;
  CK(cudaMemcpy(&st, c->d_status, sizeof st, cudaMemcpyDeviceToHost));
  CK(cudaMemset(c->d_status, 0, sizeof(unsigned)));
  if (st & ST_SINGULAR) return fail(c, FN_ESINGULAR, "singular orbital matrix");
  if (st & ST_NONFINITE) return fail(c, FN_ENONFINITE, "non-finite walker output");
  if (st & ST_TIMEOUT) return fail(c, FN_ETIMEOUT, "device wait timed out");
  return FN_OK;
}

long ferminet_flagged_matrices(fn_ctx* c) {
  if (!c) return -1;
  if (cudaStreamSynchronize(c->stream) != cudaSuccess) return -1;
  unsigned long long v = 0;
  if (cudaMemcpy(&v, c->d_flagged, sizeof v, cudaMemcpyDeviceToHost) != cudaSuccess) return -1;
  cudaMemset(c->d_flagged, 0, sizeof v);
  return (long)v;
}

fn_status ferminet_profile(fn_ctx* c, int enable) {
  if (!c) return FN_EINVAL;
  drain_profile(c);
  for (int k = 0; k < FN_KC_COUNT; ++k) {
    c->prof_ms[k] = 0.0;
    c->prof_n[k] = 0;
    c->prof_flops[k] = 0.0;
  }
  c->prof_on = enable != 0;
  return FN_OK;
}

fn_status ferminet_profile_read(fn_ctx* c, int kc, double* total_ms, long* launches, double* alg_flops) {
  if (!c || kc < 0 || kc >= FN_KC_COUNT) return FN_EINVAL;
  drain_profile(c);
  if (total_ms) *total_ms = c->prof_ms[kc];
  if (launches) *launches = c->prof_n[kc];
  if (alg_flops) *alg_flops = c->prof_flops[kc];
  return FN_OK;
}

long long ferminet_launch_count(void) { return fn::g_launches.load(); }

const char* ferminet_last_error(const fn_ctx* c) { return c ? c->err.c_str() : "null context"; }

void ferminet_destroy(fn_ctx* c) {
  if (!c) return;
  if (c->stream) cudaStreamSynchronize(c->stream);
  cudaFree(c->d_params);
  cudaFree(c->d_grad64);
  cudaFree(c->d_R);
  cudaFree(c->d_Z);
  cudaFree(c->d_Enn64);
  cudaFree(c->d_geo);
  cudaFree(c->d_geo_off);
  cudaFree(c->d_geo_cnt);
  cudaFree(c->d_clip_stats);
  cudaFree(c->d_status);
  cudaFree(c->d_flagged);
  cudaFree(c->ws);
  cudaFree(c->aux);
  cudaFree(c->wt_hi);
  cudaFree(c->wt_lo);
  cudaFree(c->wb_hi);
  cudaFree(c->wb_lo);
  cudaFree(c->ident);
  cudaFree(c->d_counter);
  if (c->step_exec) cudaGraphExecDestroy(c->step_exec);
  if (c->graph_stream) {
    cudaStreamSynchronize(c->graph_stream);
    cudaStreamDestroy(c->graph_stream);
  }
  if (c->ev_in) cudaEventDestroy(c->ev_in);
  if (c->ev_out) cudaEventDestroy(c->ev_out);
  drain_profile(c);
  for (auto e : c->ev_pool) cudaEventDestroy(e);
  delete c;
}

}  // extern "C"
