/*
 * ferminet.h — C ABI of the GB300 (sm_103a) FermiNet VMC hot path.
 *
 * Method: "Better, Faster Fermionic Neural Networks" (Spencer, Pfau, Botev,
 * Foulkes, arXiv:2011.07125).  Over a batch of MCMC walkers the library
 * evaluates
 *   - log|psi| and sign of the multi-determinant Ansatz of Eq. 3 (determinant
 *     weights omega_k removed, Sec. 3) built from the isotropic-envelope
 *     orbitals of Eq. 4 (scalar sigma per orbital and nucleus, Sec. 3);
 *   - the local energy psi^-1 H psi of the Born-Oppenheimer Hamiltonian of
 *     Eq. 1: kinetic -1/2 (lap log|psi| + |grad log|psi||^2) over all 3n
 *     electron coordinates (forward-mode derivatives, Sec. 3) plus the
 *     electron-electron, electron-nucleus and nucleus-nucleus Coulomb sums;
 *   - the gradient of the VMC energy of Eq. 2 with respect to the parameters,
 *     2/B sum_w (E_L,w - E_mean) d log|psi_w| / d theta, through a hand-written
 *     adjoint;
 *   - Gaussian all-electron Metropolis moves sampling |psi|^2 (Eq. 2).
 *
 * Conventions (all entry points):
 *   - Every pointer argument named d_* is a DEVICE pointer owned by the caller;
 *     the library never frees it and keeps no reference after the call returns.
 *     Host pointers (geometry arrays, the layout table) are read during the call.
 *   - Electron coordinates are float32, row-major [walker][electron][xyz],
 *     up-spin electrons first.  Units are bohr and hartree.
 *   - All device work is enqueued asynchronously on the stream given to
 *     ferminet_init; results are valid once that stream has been synchronised.
 *   - Argument errors are reported synchronously through the return status
 *     (FN_EINVAL) and ferminet_last_error(); no exception crosses the ABI.
 *   - Device-side conditions (a singular orbital matrix, non-finite output) are
 *     counted in a device status word read by ferminet_sync().
 *   - A context is not thread-safe; use one context per host thread.
 */
#ifndef FERMINET_H
#define FERMINET_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  FN_OK = 0,
  FN_EINVAL = 1,     /* bad argument (shape, null pointer, batch size)          */
  FN_ECUDA = 2,      /* a CUDA runtime call failed                             */
  FN_ENOMEM = 3,     /* device workspace could not be allocated                */
  FN_ENONFINITE = 4, /* ferminet_sync: some walker produced a non-finite value */
  FN_ETIMEOUT = 5,   /* a bounded device wait expired                          */
  FN_ESINGULAR = 6   /* ferminet_sync: some orbital matrix was singular        */
} fn_status;

typedef enum {
  FN_PREC_FP32 = 0,  /* every contraction in FP32 on the CUDA cores            */
  FN_PREC_MIXED = 1  /* tangent-pass layer GEMMs in BF16 on tcgen05 tensor
                        cores with FP32 accumulation; orbitals, determinants
                        and energies in FP32; reductions in FP64              */
} fn_precision;

/* Network shape.  L = n_layers one-electron layers (widths d1) and L-1
 * two-electron layers (widths d2); K = n_det determinants; n_nuc nuclei per
 * geometry (all geometries of a context share it). */
typedef struct {
  int n_layers, d1, d2, n_det, n_up, n_down, n_nuc;
  int envelope;  /* 0: isotropic, exp(-|sigma| |r - R_m|) with a scalar sigma per
                    (k, spin, i, m) (Sec. 3); 1: full covariance,
                    exp(-|Sigma (r - R_m)|) with a 3x3 Sigma each (Eq. 4) */
} fn_net;

/* One nuclear geometry (host pointers): R [n_nuc][3] bohr, Z [n_nuc].
 * Walkers [walker_offset, walker_offset + walker_count) of every batch belong
 * to it.  With a single geometry the range is ignored (all walkers use it). */
typedef struct {
  const double* R;
  const double* Z;
  long walker_offset, walker_count;
} fn_geometry;

/* One block of the flat FP32 parameter vector.  kind: 0 = dense weight
 * (conventionally initialised N(0, 1/fan_in)), 1 = bias (0), 2 = envelope
 * weight pi or isotropic exponent sigma (1), 3 = full-covariance envelope
 * matrices (3x3 identities, row-major). */
typedef struct {
  char name[32];
  long offset, count, fan_in;
  int kind, pad;
} fn_param_entry;

typedef struct fn_ctx fn_ctx;

/* Creates a context.  geoms: n_geoms >= 1 geometries; with n_geoms > 1 their
 * walker ranges must tile [0, total) without overlap and every batch passed
 * later must have B == total.  stream: a cudaStream_t (NULL = legacy default
 * stream).  On success *out owns device memory until ferminet_destroy.
 * Parameters start as all zeros; call ferminet_set_params. */
fn_status ferminet_init(const fn_net* net, const fn_geometry* geoms, int n_geoms, fn_precision prec,
                        void* stream, fn_ctx** out);

/* Parameter layout (Eq. 3-4 plus the equivariant layers): fills up to
 * max_entries entries of out (may be NULL), the entry count and the total
 * parameter count.  Blocks, in order: for each layer l: V_l [d1][3 a + 2 e]
 * (acting on [h_i, mean_up h, mean_down h, mean_up h_i., mean_down h_i.],
 * a = 4 n_nuc or d1, e = 4 or d2), b_l [d1], and for l < L-1: W_l [d2][e],
 * c_l [d2]; then w_orb_up [K][n_up][d1], w_orb_down [K][n_down][d1],
 * g_orb_up [K][n_up], g_orb_down [K][n_down], pi_up / pi_down [K][n_s][n_nuc],
 * sigma_up / sigma_down [K][n_s][n_nuc] (isotropic envelope) or
 * [K][n_s][n_nuc][3][3] (full covariance). */
fn_status ferminet_param_layout(const fn_ctx* ctx, fn_param_entry* out, int max_entries, int* n_entries,
                                long* n_params);

/* Same layout as ferminet_param_layout, computed from the shape alone (no
 * context and no device needed).  Returns FN_EINVAL for an invalid shape. */
fn_status ferminet_net_layout(const fn_net* net, fn_param_entry* out, int max_entries, int* n_entries,
                              long* n_params);

/* Copies n_params floats from d_params (device) into the library's parameter
 * buffers (and refreshes the BF16 copies of the mixed path).  Stream-ordered. */
fn_status ferminet_set_params(fn_ctx* ctx, const float* d_params);

/* log|psi| and sign, like ferminet_logpsi, for callers that cannot allocate
 * device memory: code embedded in a host framework that owns every device
 * buffer and forbids allocation inside its callbacks, or a process whose device
 * memory is already fully reserved by another allocator.  The paper has no
 * counterpart; this is an interface convenience.
 *
 * Needs no context: net, d_params (n_params floats, device, in the layout of
 * ferminet_net_layout), d_R ([n_nuc][3] float32, device, one geometry for all
 * walkers), d_x ([B][n][3]), d_logpsi ([B]) and d_sign ([B], may be NULL) are
 * all caller-owned.  The workspace is a fixed 32 MiB device array inside the
 * library (held by every GPU that loads the library until the process exits);
 * the call allocates nothing, host or device.  Large batches are processed in
 * walker chunks that fit the array.  Returns FN_ENOMEM, without launching
 * anything, when a single walker needs more than the 32 MiB (a very wide or
 * very large network); FN_EINVAL for bad arguments.
 *
 * The first call on a device looks up the array's device address (once per
 * device, with that device current); make that first call before any stream
 * capture.  Work is enqueued on `stream` (a cudaStream_t, NULL = default).
 * All calls share the one array and each call rewrites what it reads, but two
 * calls whose work overlaps on the GPU (different streams, or different host
 * threads on the same device) race on it: serialise them.  Ill-conditioning
 * and singularity counters are cleared at every call and are not reported.
 * The FP64 redo follows the same environment settings as ferminet_init
 * (FERMINET_PIVOT_TAU, FERMINET_DET64).  FN_ECUDA reports a failed launch of
 * this call; a CUDA error already pending on the calling thread is left in
 * place and not reported. */
fn_status ferminet_logpsi_noalloc(const fn_net* net, const float* d_params, const float* d_R, const float* d_x,
                                  long B, float* d_logpsi, float* d_sign, void* stream);

/* log|psi| and sign (Eq. 3) for B walkers.  d_x [B][n][3]; d_logpsi, d_sign [B]
 * (d_sign may be NULL).  A walker whose psi is exactly zero gets -inf and 0. */
fn_status ferminet_logpsi(fn_ctx* ctx, const float* d_x, long B, float* d_logpsi, float* d_sign);

/* Local energy E_L = -1/2 (lap log|psi| + |grad log|psi||^2) + V (Eq. 1) for B
 * walkers.  d_eloc [B] required; d_logpsi, d_sign, d_kinetic [B] optional
 * (NULL to skip).  In FN_PREC_MIXED the tangent-pass layer GEMMs run in BF16. */
fn_status ferminet_local_energy(fn_ctx* ctx, const float* d_x, long B, float* d_eloc, float* d_logpsi,
                                float* d_sign, float* d_kinetic);

/* Vector-Jacobian product of log|psi|: d_grad [n_params] (float) receives
 * sum_w d_seeds[w] * d log|psi_w| / d theta.  d_seeds [B] float.  Used by the
 * autograd binding (forward = log|psi|, backward = this call). */
fn_status ferminet_logpsi_vjp(fn_ctx* ctx, const float* d_x, long B, const float* d_seeds, float* d_grad);

/* VMC energy gradient (Eq. 2 differentiated with E_L held fixed).  For every
 * geometry g, d_emean[g] (double, [n_geoms]) = mean of d_eloc over its walkers,
 * and d_grad [n_params] = sum_g 2/B_g sum_{w in g} (E_L,w - E_mean,g)
 * d log|psi_w| / d theta, stored as float.  The sum over walkers runs in FP32
 * over blocks of at most a few thousand rows and in FP64 across blocks. */
fn_status ferminet_energy_grad(fn_ctx* ctx, const float* d_x, long B, const float* d_eloc, double* d_emean,
                               float* d_grad);

/* Replica form of ferminet_energy_grad, for a batch whose walkers are split over
 * several processes (data parallelism over walkers; Eq. 2's expectation is a
 * mean over every walker of the batch).  The gradient weights each walker by
 * E_L,w minus the mean over the whole batch, so it takes two exchanges:
 *   1. ferminet_energy_sums: d_sums [n_geoms] (double) = FP64 sum of d_eloc
 *      over this process's walkers of each geometry.  The caller adds d_sums
 *      and the walker counts over the processes (an all-reduce).
 *   2. ferminet_energy_grad_partial: with d_esum and d_count [n_geoms]
 *      (double) the energy sums and walker counts over the whole batch, the
 *      library forms E_mean,g = d_esum[g] / d_count[g] in FP64 on the device
 *      (stored into d_emean [n_geoms] when it is not NULL) and accumulates
 *      d_grad64 [n_params] (double) =
 *      sum_g 2/count_g sum_{w of g here} (E_L,w - E_mean,g) d log|psi_w|/d theta
 *      in FP64.  The sum of d_grad64 over the processes is the gradient
 *      ferminet_energy_grad computes on the whole batch.
 * With one process (count_g = this batch's) the two calls reproduce
 * ferminet_energy_grad.  A geometry with walkers here must have count_g > 0
 * (E_mean,g of a geometry with count_g = 0 is stored as 0).
 * B follows the rules of ferminet_energy_grad (with several geometries, B
 * equals the walker total of the geometry table). */
fn_status ferminet_energy_sums(fn_ctx* ctx, const float* d_eloc, long B, double* d_sums);
fn_status ferminet_energy_grad_partial(fn_ctx* ctx, const float* d_x, long B, const float* d_eloc,
                                       const double* d_esum, const double* d_count, double* d_emean,
                                       double* d_grad64);

/* Options of the training loop around the hot path.  The paper states
 * neither; both follow the practice of the FermiNet training it builds on
 * (Sec. 2 raises the Metropolis moves between updates from 10 to 20, Table 2
 * runs 50).
 *   clip_scale > 0: the VMC gradient (ferminet_energy_grad, ferminet_step)
 *     uses clipped local energies.  Per geometry g: m_g = median of E_L (the
 *     mean of the two middle values for an even count), tv_g = mean of
 *     |E_L - m_g|, c_w = E_L,w clamped to [m_g - clip_scale tv_g,
 *     m_g + clip_scale tv_g], and walker w gets the weight
 *     2 (c_w - mean_g c) / B_g.  d_emean still receives the plain mean of E_L.
 *     Medians, spreads and means are formed in FP64 on the device.  0 = off
 *     (the default).  The replica form (ferminet_energy_grad_partial) refuses
 *     clipping (FN_EINVAL): a median is not a sum over processes.
 *   d_width (device float, or NULL = off): the Metropolis moves of
 *     ferminet_mcmc_step and ferminet_step read the proposal width from
 *     *d_width (their width argument is ignored), and after the moves of each
 *     call the library updates it from that call's acceptance fraction
 *     p = accepted / (B n_steps): *d_width *= width_factor if p > accept_hi,
 *     /= width_factor if p < accept_lo (in FP64, stored as float).  The
 *     buffer is caller-owned and must outlive its use; a captured step keeps
 *     reading it on every replay.
 * Changing the options re-captures the graph of ferminet_step. */
typedef struct {
  float clip_scale;
  float* d_width;
  float accept_lo, accept_hi, width_factor;
} fn_train_opts;
fn_status ferminet_set_train_opts(fn_ctx* ctx, const fn_train_opts* opts);

/* KFAC, the second-order optimiser the paper credits for FermiNet's accuracy
 * (Sec. 1; Martens and Grosse 2015).  The paper gives no detail; the reading:
 * Kronecker factors of the Fisher of log|psi| for every dense layer.
 *   ferminet_kfac_size: length of the factor buffer in doubles.  Layout: for
 *     each layer l, A1_l [wV+1]^2 (one-electron inputs [h_i, mean_up h,
 *     mean_down h, mean_up h_i., mean_down h_i., 1], wV = 3 a + 2 e) and
 *     G1_l [d1]^2 (gradients of log|psi| with respect to the pre-activations);
 *     for each l < L-1, A2_l [e+1]^2 (pair inputs [h_ij, 1]) and G2_l [d2]^2;
 *     for each spin, Ao [d1+1]^2 (inputs [h^L_j, 1] of that spin's electrons)
 *     and Go [K n_s]^2 (gradients over that spin's orbitals); then D, one
 *     entry per envelope parameter (pi and sigma blocks in layout order).
 *     Every A is averaged over its rows (B n, B n^2, B n_s), every G and D
 *     over the B walkers; D is the mean squared per-walker gradient.
 *   ferminet_kfac_factors: fills d_factors (device, FP64) for the batch d_x.
 *     Mixed-precision contexts only (FN_EINVAL otherwise): it runs the
 *     tensor-core adjoint with unit seeds and forms the factors as tensor-core
 *     Gram products of the stored rows (two-electron factors: FP32 SIMT).
 *     Synchronises the stream.
 *   ferminet_kfac_precondition: d_out [n_params] (float) = the update for the
 *     gradient d_grad [n_params]: for each layer, with M = [W b] its gradient,
 *     (G + sqrt(lambda) I)^-1 M (A + sqrt(lambda) I)^-1 (orbital layers per
 *     spin, weights and biases of the K n_s orbitals); envelope entries
 *     grad / (D + lambda).  The damped factors are inverted in FP64 on the
 *     device (Gauss-Jordan, one launch per pivot step, every factor at once);
 *     the products run in FP32.  lambda > 0.  Synchronises the stream. */
fn_status ferminet_kfac_size(const fn_net* net, long* n_doubles);
fn_status ferminet_kfac_factors(fn_ctx* ctx, const float* d_x, long B, double* d_factors);
fn_status ferminet_kfac_precondition(fn_ctx* ctx, const double* d_factors, const float* d_grad, float lambda,
                                     float* d_out);

/* n_steps Gaussian all-electron Metropolis moves sampling |psi|^2 (Eq. 2).
 * Step s uses counter t = counter + s.  For walker w the proposal is
 * x' = x + width * z with z drawn by Philox4x32-10 (key {seed lo, seed hi},
 * counter {w, b, t lo, t hi} for normals 4b..4b+3 via Box-Muller, cos then
 * sin, uniforms ((u32 >> 9) + 0.5) * 2^-23), and the move is accepted iff
 * log u < 2 (log|psi(x')| - log|psi(x)|) with u from counter
 * {w, 0xFFFFFFFF, t lo, t hi}, word 0.  d_x [B][n][3] and d_logpsi [B] are
 * updated in place (d_logpsi must hold log|psi(d_x)| on entry);
 * d_accepted [B] (int, may be NULL) receives the accepted-move count. */
fn_status ferminet_mcmc_step(fn_ctx* ctx, float* d_x, float* d_logpsi, long B, int n_steps, float width,
                             uint64_t seed, uint64_t counter, int* d_accepted);

/* One whole VMC step over the batch (the path of Eq. 2 per optimisation
 * iteration): n_steps Metropolis moves exactly as ferminet_mcmc_step (counter
 * t = counter + s), then the local energy at the new positions (d_eloc [B]),
 * then the VMC energy gradient (d_emean [n_geoms] double, d_grad [n_params]) as
 * ferminet_energy_grad.  d_x and d_logpsi are updated in place; d_accepted may
 * be NULL.  With use_graph != 0 the step's kernels are captured once into a
 * CUDA graph (keyed by B, n_steps, width, seed and the buffer addresses) and
 * replayed on later calls; the counter is passed through device memory, so a
 * new counter does not re-capture.  Results are identical with and without the
 * graph.  Per-class profiling does not see graph replays. */
fn_status ferminet_step(fn_ctx* ctx, float* d_x, float* d_logpsi, long B, int n_steps, float width, uint64_t seed,
                        uint64_t counter, float* d_eloc, double* d_emean, float* d_grad, int* d_accepted,
                        int use_graph);

/* Tile shapes of the tensor-core local-energy pass and the walker chunk.
 * 0 in a field means the built-in default.
 *   layer_groups:  (walker, electron) groups per tile of the fused layer GEMM
 *                  (tile width = layer_groups * columns per group, <= 256 and a
 *                  multiple of 16);
 *   feature_tile:  features per tile of the rows-on-lanes GEMMs (orbitals and
 *                  per-walker terms; a multiple of 16, <= 256);
 *   tangent_chunk: walkers per local-energy chunk (bounded by the workspace
 *                  budget);
 *   residual_smem: 1 = the layer GEMM loads the k-blocks of its residual once
 *                  into a dedicated shared-memory region used by both the MMAs
 *                  and the epilogue (less DRAM traffic, shallower pipeline);
 *                  0 = the epilogue reads the residual from global memory;
 *   pair_unfused:  1 = the two-electron layer and the spin means of the
 *                  two-electron stream run as separate kernels (the plain
 *                  schedule, kept for comparison and for shapes the fused
 *                  kernel does not cover); 0 = one fused pass (default).
 *                  Not varied by the autotuner;
 *   adjoint_simt:  FN_PREC_MIXED only: 1 = the adjoint (its stored value
 *                  pass and its contractions) runs on the FP32 SIMT GEMMs;
 *                  0 = on the tensor cores with BF16 hi + lo operands and FP32
 *                  accumulation (default).  Not varied by the autotuner;
 *   orbital_joint: FN_PREC_MIXED only: 1 = one orbital GEMM over every row and
 *                  all K n orbitals; 0 = one per spin, each spin's electrons
 *                  against that spin's orbitals only (half the work; default).
 *                  Not varied by the autotuner. */
typedef struct {
  int layer_groups;
  int feature_tile;
  long tangent_chunk;
  int residual_smem;
  int pair_unfused;
  int adjoint_simt;
  int orbital_joint;
} fn_tuning;

fn_status ferminet_get_tuning(const fn_ctx* ctx, fn_tuning* out);
/* Invalid fields (shapes the kernels cannot run) are rejected with FN_EINVAL. */
fn_status ferminet_set_tuning(fn_ctx* ctx, const fn_tuning* t);

/* Autotuner: times the local-energy pass on d_x [B][n][3] (repeats times per
 * candidate, minimum kept) for every candidate combination of layer_groups,
 * feature_tile, tangent_chunk and residual_smem, installs the fastest in the
 * context and returns it in *best (may be NULL).  Synchronises the stream.
 * Only meaningful in FN_PREC_MIXED.  The built-in defaults (all fields 0) read
 * the layer residual from global memory; on GB300 the autotuner picks
 * residual_smem = 1 for the C4H6 and eight-geometry C4H4 workloads, whose
 * tensor-core GEMMs then take about a third less time. */
fn_status ferminet_autotune(fn_ctx* ctx, const float* d_x, long B, int repeats, fn_tuning* best);

/* Synchronises the context stream and reads the device status word:
 * FN_ESINGULAR / FN_ENONFINITE if any walker since the last sync had a
 * singular orbital matrix or a non-finite output, else FN_OK or a CUDA error.
 * Clears the status word. */
fn_status ferminet_sync(fn_ctx* ctx);

/* Number of orbital matrices whose FP32 pivot ratio min|u_kk| / max|u_kk| fell
 * below the ill-conditioning threshold since the last call (reads a device
 * counter; synchronises the stream). */
long ferminet_flagged_matrices(fn_ctx* ctx);

/* Kernel classes timed by ferminet_profile_read. */
typedef enum {
  FN_KC_TANGENT_GEMM = 0, /* layer and orbital GEMMs of the local-energy pass  */
  FN_KC_DET_TANGENT = 1,  /* determinant + derivative-trace kernel (E_L pass)  */
  FN_KC_TWO_LAYER = 2,    /* two-electron layer kernel (all passes)            */
  FN_KC_MEANS = 3,        /* spin-mean kernels of the local-energy pass        */
  FN_KC_TANH = 4,         /* forward-Laplacian tanh kernel                     */
  FN_KC_VALUE_PASS = 5,   /* one whole value pass (log|psi| only)              */
  FN_KC_ADJOINT = 6,      /* one whole adjoint (d log|psi| / d theta)          */
  FN_KC_COUNT = 7
} fn_kernel_class;

/* Turns per-class timing on (enable != 0) or off and clears the totals.  While
 * on, each launch of a timed class is bracketed by CUDA events recorded on the
 * context stream. */
fn_status ferminet_profile(fn_ctx* ctx, int enable);

/* Synchronises the stream and returns, for one class since ferminet_profile:
 * total event time (ms), number of timed launches, and the algorithmic
 * floating-point operations of those launches (multiply-adds count 2; tangent
 * columns counted without padding; orbital GEMMs counted for the same-spin
 * block only).  Any output pointer may be NULL. */
fn_status ferminet_profile_read(fn_ctx* ctx, int kernel_class, double* total_ms, long* launches,
                                double* alg_flops);

/* Kernels launched by this library in this process so far (all contexts). */
long long ferminet_launch_count(void);

/* Message of the last failing call on this context ("" if none). */
const char* ferminet_last_error(const fn_ctx* ctx);

/* Releases all device memory of the context.  NULL is ignored. */
void ferminet_destroy(fn_ctx* ctx);

#ifdef __cplusplus
}
#endif

#endif /* FERMINET_H */
