// Library-internal declarations shared by the translation units of libferminet.
#pragma once

#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <atomic>
#include <mutex>
#include <string>
#include <vector>

#include "../../include/ferminet.h"

namespace fn {

// Columns of a one-electron activation row in the tangent (local-energy) pass:
//   c = 0            value
//   c = 1 + 3 e + d  d/d x_{e,d} (electron e, component d)
//   c = 3 n + 1      Laplacian over all 3n coordinates
//   c > 3 n + 1      zero padding up to a multiple of 8
// The value pass uses a single column.
inline int tangent_cols(int n) { return ((3 * n + 2 + 7) / 8) * 8; }
// Two-electron rows carry Q = 5 quantities in the tangent pass: value,
// d/d r_i (3 components; d/d r_j is its negative) and the Laplacian over all
// coordinates; Q = 1 in the value pass.
constexpr int kQ = 5;

// Per-device state.  Kernel attributes (the dynamic shared-memory limit) and
// device properties belong to one device, and one process may drive several,
// so everything the library sets up once is set up once per device: the
// device current at the call.
constexpr int kMaxDevices = 64;
class PerDeviceOnce {
 public:
  template <class F>
  void operator()(F&& f) {
    int d = 0;
    if (cudaGetDevice(&d) != cudaSuccess || d < 0 || d >= kMaxDevices) {
      cudaGetLastError();
      f();
      return;
    }
    if (done_[d].load(std::memory_order_acquire)) return;
    std::lock_guard<std::mutex> lk(mu_);
    if (!done_[d].load(std::memory_order_relaxed)) {
      f();
      done_[d].store(true, std::memory_order_release);
    }
  }

 private:
  std::atomic<bool> done_[kMaxDevices] = {};
  std::mutex mu_;
};
// Multiprocessor count of the current device (cached per device).
int device_sm_count();

// Kernels launched by the library (every launch site adds one).
extern std::atomic<long long> g_launches;
#define FN_COUNT(n) (::fn::g_launches.fetch_add((n), std::memory_order_relaxed))

// Device status bits.
enum : unsigned { ST_SINGULAR = 1u, ST_NONFINITE = 2u, ST_TIMEOUT = 4u };

// ---------------------------------------------------------------------------
// Parameter offsets (same layout as ferminet_param_layout documents).
struct Layout {
  long V[16], b[16], W[16], c[16];
  long w_orb, g_orb, pi[2], sigma[2];
  long total;
  std::vector<fn_param_entry> entries;
};
// with_entries = false fills the offsets only and allocates nothing.
void build_layout(const fn_net& t, Layout* L, bool with_entries = true);

inline int din1_of(const fn_net& t, int l) { return l == 0 ? 4 * t.n_nuc : t.d1; }
inline int din2_of(const fn_net& t, int l) { return l == 0 ? 4 : t.d2; }

// ---------------------------------------------------------------------------
// GEMM (FP32 SIMT): C[M][N] = A * B (+ epilogue).
struct Epi {
  float beta = 0.f;                 // C = acc + beta * C
  const float* bias = nullptr;      // + bias[n] on rows with r % bias_period == 0
  int bias_period = 1;
  const float* U = nullptr;         // + U[((r / u_div) * u_mul + r % u_mod) * ldu + n]
  long u_div = 1, u_mul = 1, u_mod = 1, ldu = 0;
  int act = 0;                      // 1: tanh after the above (value pass only)
  const float* res = nullptr;       // + res[r * ldr + n] after the activation
  long ldr = 0;
};
// A [M][K] (lda), B [N][K] (ldb):  C = A B^T
void gemm_nt(cudaStream_t s, long M, long N, long K, const float* A, long lda, const float* B, long ldb, float* C,
             long ldc, const Epi& e);
// A [M][K] (lda), B [K][N] (ldb):  C = A B
void gemm_nn(cudaStream_t s, long M, long N, long K, const float* A, long lda, const float* B, long ldb, float* C,
             long ldc, const Epi& e);
// A [K][M] (lda), B [K][N] (ldb):  partial[z] = A^T B over the z-th K slice,
// then grad[m * ldg + n] += sum_z partial[z] in FP64.  scratch holds
// splits * M * N floats.
void gemm_tn_accum(cudaStream_t s, long M, long N, long K, const float* A, long lda, const float* B, long ldb,
                   double* grad, long ldg, float* scratch, int splits);
int gemm_tn_splits(long M, long N, long K);
// grad[m * ldg + n] += sum_z part[z][m][n] in FP64 (z < splits, [M][N] each).
void launch_reduce_partials(cudaStream_t s, const float* part, int splits, long M, long N, double* grad, long ldg);

// ---------------------------------------------------------------------------
// Network kernels (k_network.cu)
struct Geo {
  const float* R;      // [G][N][3]
  const float* Z;      // [G][N]
  const double* Enn;   // [G] nuclear repulsion
  const int* geo;      // [B_total] or nullptr (all geometry 0)
};
void launch_features(cudaStream_t s, const float* x, long Bc, long w0, int n, int N, int C, int Q, Geo g,
                     float* H0, float* E0);
void launch_mean1(cudaStream_t s, const float* H, long Bc, int n, int n_up, int C, int din, float* M1);
void launch_mean2(cudaStream_t s, const float* E, long Bc, int n, int n_up, int Q, int din2, int C, float* M2);
// Same means written as BF16 hi / lo parts (lo may be null) with row stride ldb
// (>= 2 din2, padding columns zeroed).
void launch_mean2_bf16(cudaStream_t s, const float* E, long Bc, int n, int n_up, int Q, int din2, int C,
                       __nv_bfloat16* hi, __nv_bfloat16* lo, long ldb);
// Spin means of a BF16 hi + lo activation, written as BF16 hi + lo (padded).
void launch_mean1_bf16(cudaStream_t s, const __nv_bfloat16* hi, const __nv_bfloat16* lo, long ldin, long Bc, int n,
                       int n_up, int C, int din, __nv_bfloat16* ohi, __nv_bfloat16* olo, long ldout);
// dst_hi/lo[r][c] = split of src[r * src_ld + c] for c < cols, 0 for cols <= c < dst_ld.
void launch_split_bf16(cudaStream_t s, const float* src, long src_ld, long rows, long cols, __nv_bfloat16* hi,
                       __nv_bfloat16* lo, long dst_ld);
// Transposed splits (k_transpose.cu): dst_hi/lo[c][r] for c < cols and
// r < ld_dst from src[r][c] (r < rows; zero for rows <= r < ld_dst), from FP32
// or from BF16 hi + lo (lo parts may be null).
void launch_t_split(cudaStream_t s, const float* src, long ld_src, long rows, long cols, __nv_bfloat16* hi,
                    __nv_bfloat16* lo, long ld_dst);
void launch_t_bf16(cudaStream_t s, const __nv_bfloat16* shi, const __nv_bfloat16* slo, long ld_src, long rows,
                   long cols, __nv_bfloat16* hi, __nv_bfloat16* lo, long ld_dst);
void launch_tanh_fl(cudaStream_t s, const float* Z, const float* Hres, long Bc, int n, int C, int d1, float* Hout,
                    float* Y);
void launch_two_layer(cudaStream_t s, const float* Ein, long Bc, int n, int Q, int din2, int d2, const float* W,
                      const float* c, bool residual, float* Eout, float* Y2);

// Fused two-electron layer and dense spin means of its output (k_pair.cu).
// With W null the kernel forms the means of Ein itself.
struct PairArgs {
  const float* Ein;     // [groups][n][Q][din] pair rows, 16-byte aligned
  long groups;          // walkers x electrons
  int n, n_up, C;       // electrons, spin-up electrons, dense mean columns (1 in a value pass)
  const float* W;       // [dout][din], or null
  const float* cb;      // [dout]
  int residual;         // add the input rows (din == dout)
  float* Eout;          // [groups][n][Q][dout] new rows, or null when no later kernel reads them
  float* Y2;            // [groups][n][dout] tanh values (adjoint), or null
  float* m32;           // dense means [groups][C][ldm] as FP32, or
  __nv_bfloat16* mhi;   //   as BF16 hi / lo (lo may be null); columns 2 dout .. ldm-1 zero
  __nv_bfloat16* mlo;
  long ldm;
  int mma;              // 32 -> 32 layers of a value pass (Q = 1): the contraction on warp
                        // MMAs with BF16 hi + lo operands (three products, FP32 accumulation)
  int tg;               // set by the launcher
};
bool pair_layer_supported(int n, int din, int dout, bool layer, int Q, int C, long ldm);
bool launch_pair_layer(cudaStream_t s, const PairArgs& a, int din, int dout, int Q);

// Backward of a two-electron layer of the value pass (k_pair.cu): with
// Zbar = Eout_bar * (1 - y^2), accumulates dW = Zbar^T Ein and dc = sum Zbar
// into grad (FP64, by way of per-block FP32 partials summed in block order) and
// writes Ein_bar = Zbar W (+ Eout_bar when residual) unless Ein_bar is null.
struct PairBwdArgs {
  const float* Eout_bar;  // [pairs][dout], or null (zero)
  const float* M2bar;     // gradient of the next layer's pair means [groups][2 dout], or null: its
  int n, n_up;            // share M2bar[w i][spin(j)] / n_spin(j) is added to Eout_bar of pair (i, j)
  const float* Y;         // [pairs][dout] tanh values
  const float* Ein;       // [pairs][din]
  const float* W;         // [dout][din]
  float* Ein_bar;         // [pairs][din] or null
  int residual;
  long pairs;
  double* grad_W;         // [dout][din]
  double* grad_c;         // [dout]
  float* partial;         // scratch: pair_bwd_scratch_floats(din, dout) floats
  int mma;                // 32 -> 32 layers: dW and Ein_bar on warp MMAs with BF16 hi + lo
                          // operands (three products, FP32 accumulation)
};
bool pair_bwd_supported(int din, int dout);
long pair_bwd_scratch_floats(int din, int dout);
bool launch_pair_bwd(cudaStream_t s, const PairBwdArgs& a, int din, int dout);

// ---------------------------------------------------------------------------
// Determinants (k_det.cu)
struct DetArgs {
  const float* O;      // orbitals [Bc][n][C][Ktot]
  long ldo;            // Ktot = K * n
  int C, n, n_up, K, N;
  const float* x;      // chunk walkers [Bc][n][3]
  Geo g;
  long w0, Bc;
  const float* pi[2];
  const float* sigma[2];  // [K][n_s][N] scalars, or [K][n_s][N][3][3] with full_env
  int full_env;           // 1: full-covariance envelope exp(-|Sigma (r - R_m)|)
  bool tangent;
  float* logdet;       // [Bc][K][2]
  float* sign;         // [Bc][K][2]
  float* dgrad;        // [Bc][K][2][3n]   (tangent)
  float* dlap;         // [Bc][K][2]       (tangent)
  float* minv;         // [Bc][K][2][ns*ns] inverses (value pass, optional)
  float* env;          // [Bc][K][2][ns*ns] envelopes (value pass, optional)
  unsigned* status;
  unsigned long long* flagged;
  float pivot_tau;
  long nss;            // stride between stored matrices (ns_max^2)
  int force64;         // redo every matrix in FP64 (diagnostics)
  int* redo;           // [1 + Bc K 2]: count, then the matrices (tangent pass) or determinant
                       // pairs (value pass) to redo in FP64
};
void launch_det(cudaStream_t s, const DetArgs& a);
void launch_det_tangent(cudaStream_t s, const DetArgs& a);     // k_det_tangent.cu (called by launch_det)
void launch_det_value_warp(cudaStream_t s, const DetArgs& a);  // k_det_value.cu (called by launch_det)

// ---------------------------------------------------------------------------
// Energies, Metropolis, reductions (k_energy.cu)
void launch_combine(cudaStream_t s, const float* logdet, const float* sign, const float* dgrad, const float* dlap,
                    const float* x, long Bc, long w0, int n, int K, int N, Geo g, bool tangent, float* logpsi,
                    float* psign, float* eloc, float* kinetic, float* wdet, unsigned* status);
// Metropolis kernels; with dctr non-null the counter is t + *dctr (device
// memory); with dwidth non-null the proposal width is *dwidth.
void launch_propose(cudaStream_t s, const float* x, float* xp, long B, int n3, float width, uint64_t seed,
                    uint64_t t, const uint64_t* dctr, const float* dwidth);
void launch_accept(cudaStream_t s, float* x, const float* xp, float* logpsi, const float* lp_prop, long B, int n3,
                   uint64_t seed, uint64_t t, int* accepted, const uint64_t* dctr);
void launch_set_u64(cudaStream_t s, uint64_t* p, uint64_t v);
// With G == 1 the single geometry holds all B walkers (B1 = B >= 0); with
// B1 < 0 the device tables d_off / d_cnt give each geometry's walker range.
// launch_esum writes sums instead of means; launch_seeds_given takes the
// energy sum and the walker count of every geometry over the whole
// (replicated) batch, divides them in FP64 and stores the means in emean
// (when not null).
void launch_emean(cudaStream_t s, const float* eloc, int G, const long* d_off, const long* d_cnt, long B1,
                  double* emean);
void launch_seeds(cudaStream_t s, const float* eloc, long B, const int* geo, const double* emean,
                  const long* d_cnt, long B1, float* seeds);
void launch_esum(cudaStream_t s, const float* eloc, int G, const long* d_off, const long* d_cnt, long B1,
                 double* sums);
void launch_seeds_given(cudaStream_t s, const float* eloc, long B, const int* geo, const double* sums,
                        const double* count, int G, double* emean, float* seeds);
// Clipped gradient seeds (per geometry: median, mean absolute deviation and
// clipped mean in FP64 into stats [3 G], then the seeds).
void launch_clip_seeds(cudaStream_t s, const float* eloc, long B, const int* geo, int G, const long* d_off,
                       const long* d_cnt, long B1, double scale, double* stats, float* seeds);
// *width adapted from the acceptance fraction sum(accepted) / (B n_steps).
void launch_adapt_width(cudaStream_t s, const int* accepted, long B, int n_steps, float* width, double lo,
                        double hi, double factor);
void launch_d2f(cudaStream_t s, const double* a, float* b, long n);
void launch_fill(cudaStream_t s, float* p, float v, long n);
void launch_zero_d(cudaStream_t s, double* p, long n);

// ---------------------------------------------------------------------------
// Adjoint kernels (k_adjoint.cu)
struct AdjDetArgs {
  const float* O;        // value-pass orbitals [Bc][n][Ktot]
  const float* minv;     // [Bc][K][2][NS*NS]
  const float* env;      // [Bc][K][2][NS*NS]
  const float* wdet;     // [Bc][K]  psi_k / psi
  const float* seeds;    // [Bc]
  const float* x;        // chunk walkers [Bc][n][3]
  Geo g;
  long w0, Bc;
  int n, n_up, K, N, NS;
  const float* pi[2];
  const float* sigma[2];
  int full_env;          // 1: sigma holds 3x3 matrices (9 gradient entries each)
  float* Obar;           // [Bc][n][Ktot]
  float* envgrad;        // per walker [K*n*N] pi part, then [K*n*N*(9 or 1)] sigma part
};
void launch_adj_det(cudaStream_t s, const AdjDetArgs& a);
// grad[c] += sum_r X[r * ldx + c] in FP64 (two-pass, deterministic);
// scratch holds colsum_scratch_elems(rows, cols) doubles.
long colsum_scratch_elems(long rows, long cols);
void launch_colsum_accum(cudaStream_t s, const float* X, long rows, long cols, long ldx, double* grad,
                         double* scratch);
void launch_tanh_bwd(cudaStream_t s, const float* hbar, const float* Y, long rows, int d, float* zbar);
void launch_walker_sum(cudaStream_t s, const float* X, long Bc, int n, int d, float* S);
void launch_spread_mean1(cudaStream_t s, const float* m1bar, long Bc, int n, int n_up, int din, float* hbar);
void launch_spread_mean2(cudaStream_t s, const float* m2bar, long Bc, int n, int n_up, int din2, float* ebar);
void launch_add(cudaStream_t s, float* dst, const float* src, long n);

// ---------------------------------------------------------------------------
// KFAC (k_kfac.cu)
// Transposed KFAC input rows: column c of row r is taken from the segment
// whose column range holds c (source row r / row_div, BF16 hi + lo), the last
// column is 1; rows r >= rows, and with spin >= 0 rows whose electron
// (r % n) is not of that spin, are zero.
struct KfacRows {
  struct Seg {
    const __nv_bfloat16* hi;
    const __nv_bfloat16* lo;
    long ld;
    int col0, ncols;
    long row_div;
  } seg[3];
  int nseg;
  long rows;
  int cols;
  int spin, n, n_up;
};
// One factor block of the buffer: off (offset in the factor buffer), dim,
// woff (offset in the inversion workspaces), diag (a diagonal block of dim
// entries), scale (sum -> average), and for the two-electron input factors
// mirror_bias with the row count.
struct KfacBlock {
  long off, dim, woff;
  int diag, mirror_bias;
  double scale, count;
};
void launch_kfac_rows(cudaStream_t s, const KfacRows& a, __nv_bfloat16* hi, __nv_bfloat16* lo, long ld_out);
void launch_colsq_accum(cudaStream_t s, const float* X, long rows, long cols, long ldx, double* out);
void launch_kfac_finalize(cudaStream_t s, double* F, const KfacBlock* d_blk, int nblk);
// Damped copies of every non-diagonal block (gamma on the diagonal) inverted
// in FP64 by Gauss-Jordan, one launch per pivot step alternating between the
// workspaces w0 and w1 (each holding every block at its woff); a block of
// dimension d is done after step d - 1, so its inverse ends in w0 when d is
// even and in w1 when d is odd.
void launch_kfac_invert(cudaStream_t s, const double* F, const KfacBlock* d_blk, int nblk, int max_dim, double gamma,
                        double* w0, double* w1);
void launch_to_float(cudaStream_t s, const double* a, float* b, long n);
void launch_gather_wb(cudaStream_t s, const float* g, long w_off, long b_off, long rows, long cols, float* M);
void launch_scatter_wb(cudaStream_t s, const float* M, long w_off, long b_off, long rows, long cols, float* g);
void launch_diag_precond(cudaStream_t s, const float* g, const double* D, long n, double lambda, float* out);

}  // namespace fn

// ---------------------------------------------------------------------------
// The context.
struct fn_ctx {
  fn_net net{};
  int n = 0, N = 0, G = 0, Ct = 0;
  fn_precision prec = FN_PREC_FP32;
  cudaStream_t stream = nullptr;
  fn::Layout lay;
  std::vector<long> geo_off, geo_cnt;
  long geo_total = 0;
  // device
  float* d_params = nullptr;
  float* d_R = nullptr;
  float* d_Z = nullptr;
  int* d_geo = nullptr;
  long* d_geo_cnt = nullptr;
  long* d_geo_off = nullptr;
  double* d_Enn64 = nullptr;
  unsigned* d_status = nullptr;
  unsigned long long* d_flagged = nullptr;
  double* d_grad64 = nullptr;
  char* ws = nullptr;
  size_t ws_size = 0;
  float* aux = nullptr;   // Metropolis proposals / seeds
  long aux_cap = 0;
  std::string err;
  int device = 0;
  int ns_max = 0;
  float pivot_tau = 1e-4f;  // FP32 pivot-ratio threshold of the FP64 redo
  // mixed precision: BF16 hi/lo copies of the layer weights, padded to 64 columns
  bool tc_ok = false;
  bool host_fail = false;  // set when a tensor-core launch could not be prepared
  int terms = 3;
  __nv_bfloat16* wb_hi = nullptr;
  __nv_bfloat16* wb_lo = nullptr;
  long wb_a[16] = {}, wb_bc[16] = {}, wb_de[16] = {}, wb_orb = 0;
  long ld_a[16] = {}, ld_bc[16] = {}, ld_de[16] = {}, ld_orb = 0;
  long wb_total = 0;
  // transposed BF16 hi/lo weight blocks for the backward-data products of the
  // tensor-core adjoint: V_a^T [a1][pad64(d1)], V_bc^T [2 a1][..], V_de^T
  // [2 a2][..], W_orb^T [d1][pad64(K n)]
  __nv_bfloat16* wt_hi = nullptr;
  __nv_bfloat16* wt_lo = nullptr;
  long wt_a[16] = {}, wt_bc[16] = {}, wt_de[16] = {}, wt_orb = 0;
  __nv_bfloat16* ident = nullptr;  // 128 x 128 BF16 identity (operand of the folded per-walker term)
  int force64 = 0;
  fn_tuning tune{};  // 0 fields: defaults
  fn_train_opts train{};       // clipping and width adaptation (off)
  double* d_clip_stats = nullptr;  // [3 G]: median, spread, clipped mean per geometry
  // captured full step (ferminet_step with use_graph)
  uint64_t* d_counter = nullptr;
  cudaGraphExec_t step_exec = nullptr;
  cudaStream_t graph_stream = nullptr;  // captures and replays (the legacy default stream cannot capture)
  cudaEvent_t ev_in = nullptr, ev_out = nullptr;
  struct StepKey {
    long B;
    int n_steps;
    float width;
    uint64_t seed;
    const void *x, *lp, *eloc, *emean, *grad, *acc, *ws, *aux, *dwidth;
    float clip;
    size_t ws_size;
  } step_key{};
  // per-class event timing
  bool prof_on = false;
  struct Pending {
    int cls;
    cudaEvent_t e0, e1;
    double flops;
  };
  std::vector<Pending> pending;
  std::vector<cudaEvent_t> ev_pool;
  double prof_ms[FN_KC_COUNT] = {};
  long prof_n[FN_KC_COUNT] = {};
  double prof_flops[FN_KC_COUNT] = {};
};

namespace fn {
// Value pass with a caller-supplied workspace; allocates nothing (ferminet.cu).
fn_status value_pass_fixed_workspace(const fn_net& net, const float* d_params, const float* d_R, const float* d_x,
                                     long B, float* d_logpsi, float* d_sign, cudaStream_t s, char* ws,
                                     size_t ws_size);
}  // namespace fn
