/*
 * FP64 CPU oracle for the FermiNet VMC hot path (arXiv:2011.07125).
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test suite, the smoke check and the
 * benchmark's CPU-baseline / reference legs load this file.  It shares no code,
 * header, table or helper with the CUDA path, and never calls it.
 *
 * What it computes, all in double precision and written for reading, not speed:
 *   - log|psi| and sign of the multi-determinant Ansatz, Eq. 3 (determinant
 *     weights omega_k dropped, Sec. 3), with the isotropic-envelope orbitals of
 *     Eq. 4 (scalar sigma, Sec. 3) on top of a permutation-equivariant network
 *     h^L whose layers the paper does not spell out (Sec. 3 defers to the
 *     original FermiNet); the reading used is the one documented at
 *     oracle_fwd below.
 *   - derivatives of log|psi| with respect to each of the 3n electron
 *     coordinates by univariate second-order Taylor ("jet") arithmetic: one full
 *     forward pass per coordinate, seeded with (x, 1, 0).  Exact to rounding.
 *   - the local energy psi^-1 H psi with H the Born-Oppenheimer Hamiltonian of
 *     Eq. 1: kinetic -1/2 sum_c (d_c^2 log|psi| + (d_c log|psi|)^2) plus the
 *     electron-electron, electron-nucleus and nucleus-nucleus Coulomb sums.
 *   - d log|psi| / d theta by a hand-written reverse pass over the plain
 *     forward, and the VMC energy gradient of Eq. 2,
 *     2/B sum_w (E_L,w - E_mean) d log|psi_w| / d theta (E_L held fixed).
 *   - Gaussian all-electron Metropolis moves sampling |psi|^2 (Sec. 1, Eq. 2),
 *     driven by Philox4x32-10 (Salmon et al., SC'11) and the Box-Muller
 *     transform, both written from their published definitions.
 *
 * Parity status: every function here is pinned by tests against closed forms,
 * invariants, finite differences or brute force (hydrogenic exact states,
 * antisymmetry, Leibniz determinants, translation invariance, Coulomb pair
 * sums, Philox known-answer vectors).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <stdio.h>

/* ------------------------------------------------------------------------ */
/* Network shape and parameter layout                                        */
/* ------------------------------------------------------------------------ */

/* envelope 0: isotropic, exp(-|sigma| |r - R_m|) with one scalar sigma per
 * (k, spin, i, m) (Sec. 3); envelope 1: full covariance, exp(-|Sigma (r - R_m)|)
 * with one 3x3 matrix Sigma per (k, spin, i, m) (Eq. 4), stored row-major. */
typedef struct {
  int n_layers, d1, d2, n_det, n_up, n_down, n_nuc, envelope;
} onet;

enum { O_INIT_NORMAL = 0, O_INIT_ZERO = 1, O_INIT_ONE = 2, O_INIT_EYE3 = 3 };

typedef struct {
  char name[32];
  long offset, count, fan_in;
  int kind, pad;
} oentry;

/* Offsets of every parameter block, computed from the shape. */
typedef struct {
  long V[16], b[16], W[16], c[16];
  long w_orb[2], g_orb[2], pi[2], sigma[2];
  long total;
} olayout;

static int din1_of(const onet* t, int l) { return l == 0 ? 4 * t->n_nuc : t->d1; }
static int din2_of(const onet* t, int l) { return l == 0 ? 4 : t->d2; }
static int nspin(const onet* t, int s) { return s == 0 ? t->n_up : t->n_down; }

/* One envelope term of Eq. 4 for displacement d = r_j - R_m: exp(-|sigma| |d|)
 * (isotropic, sg[0] = sigma) or exp(-|Sigma d|) (full, sg = Sigma row-major). */
static double env_term(const onet* t, const double* sg, const double d[3]) {
  if (!t->envelope) return exp(-fabs(sg[0]) * sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]));
  double v2 = 0.0;
  for (int a = 0; a < 3; ++a) {
    const double va = sg[3 * a] * d[0] + sg[3 * a + 1] * d[1] + sg[3 * a + 2] * d[2];
    v2 += va * va;
  }
  return exp(-sqrt(v2));
}

/* Layout, in this order:
 *   for each layer l: V_l [d1][3*din1 + 2*din2], b_l [d1],
 *                     and for l < L-1: W_l [d2][din2], c_l [d2]
 *   w_orb_up [K][n_up][d1], w_orb_down [K][n_down][d1],
 *   g_orb_up [K][n_up], g_orb_down [K][n_down],
 *   pi_up [K][n_up][N], pi_down [K][n_down][N],
 *   sigma_up [K][n_up][N], sigma_down [K][n_down][N] (isotropic), or
 *   [K][n_up][N][3][3], [K][n_down][N][3][3] (full covariance, identity init).
 * V_l acts on g_i = [h_i, mean_up h, mean_down h, mean_up h_i., mean_down h_i.]. */
static int build_layout(const onet* t, olayout* L, oentry* ent, int max_ent) {
  long off = 0;
  int ne = 0;
#define ADD(field, nm, cnt, fan, knd)                                   \
  do {                                                                  \
    field = off;                                                        \
    if (ent && ne < max_ent) {                                          \
      snprintf(ent[ne].name, sizeof ent[ne].name, "%s", nm);            \
      ent[ne].offset = off; ent[ne].count = (cnt); ent[ne].fan_in = (fan); \
      ent[ne].kind = (knd); ent[ne].pad = 0;                            \
    }                                                                   \
    ne++; off += (cnt);                                                 \
  } while (0)
  char nm[32];
  for (int l = 0; l < t->n_layers; ++l) {
    int a = din1_of(t, l), e = din2_of(t, l);
    long fan = 3L * a + 2L * e;
    snprintf(nm, sizeof nm, "V%d", l); ADD(L->V[l], nm, (long)t->d1 * fan, fan, O_INIT_NORMAL);
    snprintf(nm, sizeof nm, "b%d", l); ADD(L->b[l], nm, (long)t->d1, 1, O_INIT_ZERO);
    if (l < t->n_layers - 1) {
      snprintf(nm, sizeof nm, "W%d", l); ADD(L->W[l], nm, (long)t->d2 * e, e, O_INIT_NORMAL);
      snprintf(nm, sizeof nm, "c%d", l); ADD(L->c[l], nm, (long)t->d2, 1, O_INIT_ZERO);
    }
  }
  long K = t->n_det;
  ADD(L->w_orb[0], "w_orb_up", K * t->n_up * t->d1, t->d1, O_INIT_NORMAL);
  ADD(L->w_orb[1], "w_orb_down", K * t->n_down * t->d1, t->d1, O_INIT_NORMAL);
  ADD(L->g_orb[0], "g_orb_up", K * t->n_up, 1, O_INIT_ZERO);
  ADD(L->g_orb[1], "g_orb_down", K * t->n_down, 1, O_INIT_ZERO);
  ADD(L->pi[0], "pi_up", K * t->n_up * t->n_nuc, 1, O_INIT_ONE);
  ADD(L->pi[1], "pi_down", K * t->n_down * t->n_nuc, 1, O_INIT_ONE);
  const long sz = t->envelope ? 9 : 1;
  const int skind = t->envelope ? O_INIT_EYE3 : O_INIT_ONE;
  ADD(L->sigma[0], "sigma_up", K * t->n_up * t->n_nuc * sz, 1, skind);
  ADD(L->sigma[1], "sigma_down", K * t->n_down * t->n_nuc * sz, 1, skind);
#undef ADD
  L->total = off;
  return ne;
}

static int check_net(const onet* t) {
  if (t->n_layers < 1 || t->n_layers > 16 || t->d1 < 1 || t->d2 < 1 || t->n_det < 1 ||
      t->n_up < 0 || t->n_down < 0 || t->n_up + t->n_down < 1 || t->n_nuc < 1 || t->envelope < 0 ||
      t->envelope > 1)
    return -1;
  return 0;
}

/* Returns the number of entries; fills up to max_ent of them and *n_params. */
int oracle_param_layout(const onet* t, oentry* out, int max_ent, long* n_params) {
  if (check_net(t)) return -1;
  olayout L;
  int ne = build_layout(t, &L, out, max_ent);
  if (n_params) *n_params = L.total;
  return ne;
}

/* ------------------------------------------------------------------------ */
/* Determinants: LU with partial pivoting (Doolittle) and Leibniz expansion  */
/* ------------------------------------------------------------------------ */

/* In-place LU of an n x n row-major matrix with row pivoting.  Returns the
 * sign of the row permutation in *perm_sign and the permutation in piv
 * (piv[k] = original row now at position k). */
static void lu_inplace(int n, double* a, int* piv, int* perm_sign) {
  int s = 1;
  for (int i = 0; i < n; ++i) piv[i] = i;
  for (int k = 0; k < n; ++k) {
    int p = k;
    double best = fabs(a[k * n + k]);
    for (int i = k + 1; i < n; ++i)
      if (fabs(a[i * n + k]) > best) { best = fabs(a[i * n + k]); p = i; }
    if (p != k) {
      for (int j = 0; j < n; ++j) { double t = a[k * n + j]; a[k * n + j] = a[p * n + j]; a[p * n + j] = t; }
      int t = piv[k]; piv[k] = piv[p]; piv[p] = t;
      s = -s;
    }
    double u = a[k * n + k];
    if (u == 0.0) continue;
    for (int i = k + 1; i < n; ++i) {
      double l = a[i * n + k] / u;
      a[i * n + k] = l;
      for (int j = k + 1; j < n; ++j) a[i * n + j] -= l * a[k * n + j];
    }
  }
  *perm_sign = s;
}

/* sign and log|det| by LU; sign 0 and -inf for a singular matrix. */
void oracle_slogdet(int n, const double* A, double* sign, double* logabs) {
  if (n == 0) { *sign = 1.0; *logabs = 0.0; return; }
  double* a = malloc(sizeof(double) * n * n);
  int* piv = malloc(sizeof(int) * n);
  memcpy(a, A, sizeof(double) * n * n);
  int ps;
  lu_inplace(n, a, piv, &ps);
  double s = ps, la = 0.0;
  for (int k = 0; k < n; ++k) {
    double u = a[k * n + k];
    if (u == 0.0) { s = 0.0; la = -INFINITY; break; }
    if (u < 0) s = -s;
    la += log(fabs(u));
  }
  *sign = s; *logabs = la;
  free(a); free(piv);
}

/* Inverse by LU (solves A X = I column by column).  Returns -1 if singular. */
static int lu_inverse(int n, const double* A, double* inv) {
  double* a = malloc(sizeof(double) * n * n);
  int* piv = malloc(sizeof(int) * n);
  memcpy(a, A, sizeof(double) * n * n);
  int ps;
  lu_inplace(n, a, piv, &ps);
  int bad = 0;
  for (int k = 0; k < n; ++k) if (a[k * n + k] == 0.0) bad = 1;
  if (!bad) {
    double* y = malloc(sizeof(double) * n);
    for (int col = 0; col < n; ++col) {
      /* P A = L U ; solve L y = P e_col, then U x = y */
      for (int i = 0; i < n; ++i) y[i] = (piv[i] == col) ? 1.0 : 0.0;
      for (int i = 0; i < n; ++i)
        for (int j = 0; j < i; ++j) y[i] -= a[i * n + j] * y[j];
      for (int i = n - 1; i >= 0; --i) {
        for (int j = i + 1; j < n; ++j) y[i] -= a[i * n + j] * y[j];
        y[i] /= a[i * n + i];
      }
      for (int i = 0; i < n; ++i) inv[i * n + col] = y[i];
    }
    free(y);
  }
  free(a); free(piv);
  return bad ? -1 : 0;
}

/* det by the Leibniz permutation expansion (Heap's algorithm), n <= 8. */
double oracle_det_leibniz(int n, const double* A) {
  if (n == 0) return 1.0;
  if (n > 8) return NAN;
  int p[8], c[8];
  for (int i = 0; i < n; ++i) { p[i] = i; c[i] = 0; }
  int sgn = 1;
  double total = 0.0;
  for (;;) {
    double prod = sgn;
    for (int i = 0; i < n; ++i) prod *= A[i * n + p[i]];
    total += prod;
    int i = 1;
    while (i < n && c[i] >= i) { c[i] = 0; ++i; }
    if (i >= n) break;
    int j = (i % 2 == 0) ? 0 : c[i];
    int t = p[i]; p[i] = p[j]; p[j] = t;
    sgn = -sgn;
    c[i]++;
  }
  return total;
}

/* ------------------------------------------------------------------------ */
/* Plain forward pass with stored activations (value only)                   */
/* ------------------------------------------------------------------------ */

/* Everything the reverse pass needs from one walker's forward. */
typedef struct {
  const onet* t;
  int n, N, L;
  double* h[17];     /* h[l]: [n][din1(l)], l = 0..L (h[L] width d1)          */
  double* e[17];     /* e[l]: [n][n][din2(l)], l = 0..L-1                    */
  double* m1[16];    /* [2][din1(l)] spin means of h[l]                      */
  double* m2[16];    /* [n][2][din2(l)] spin means over j of e[l][i][j]      */
  double* y1[16];    /* tanh outputs of one-electron layer l: [n][d1]        */
  double* y2[16];    /* tanh outputs of two-electron layer l: [n][n][d2]     */
  double* orb[2];    /* o [K][n_s][n_s] (orbital i, electron j)              */
  double* env[2];    /* envelope [K][n_s][n_s]                               */
  double* A[2];      /* A = o * env [K][n_s][n_s]                            */
  double* Ainv[2];   /* inverses [K][n_s][n_s]                               */
  double* dist;      /* [n][N] electron-nucleus distances                    */
  double* ldet;      /* [K][2] log|det|                                      */
  double* sdet;      /* [K][2] signs                                         */
  double logpsi, sign;
  int singular;
} ofwd;

static void fwd_free(ofwd* f) {
  for (int l = 0; l <= f->L; ++l) { free(f->h[l]); }
  for (int l = 0; l < f->L; ++l) { free(f->e[l]); free(f->m1[l]); free(f->m2[l]); free(f->y1[l]); free(f->y2[l]); }
  for (int s = 0; s < 2; ++s) { free(f->orb[s]); free(f->env[s]); free(f->A[s]); free(f->Ainv[s]); }
  free(f->dist); free(f->ldet); free(f->sdet);
}

/*
 * The network (reading of Sec. 3, which names h^L as "the last layer of a
 * permutation-equivariant neural network" and defers its definition to the
 * original FermiNet):
 *   h^0_i  = [r_i - R_I, |r_i - R_I|] over nuclei I      (width 4N)
 *   h^0_ij = [r_i - r_j, |r_i - r_j|]                    (width 4; 0 for i=j)
 *   g^l_i  = [h^l_i, mean_{j up} h^l_j, mean_{j down} h^l_j,
 *             mean_{j up} h^l_ij, mean_{j down} h^l_ij]   (means include j=i;
 *             an empty spin channel gives the zero vector)
 *   h^{l+1}_i  = tanh(V_l g^l_i + b_l)  (+ h^l_i for l >= 1)
 *   h^{l+1}_ij = tanh(W_l h^l_ij + c_l) (+ h^l_ij for l >= 1), l < L-1
 * Orbitals (Eq. 4, isotropic envelope):
 *   phi^{ka}_i(r_j) = (w^{ka}_i . h^L_j + g^{ka}_i)
 *                     * sum_m pi^{ka}_im exp(-|sigma^{ka}_im| |r_j - R_m|)
 * psi = sum_k det[phi^{k up}] det[phi^{k down}]  (Eq. 3 with omega_k dropped).
 */
static void oracle_fwd(const onet* t, const olayout* Lo, const double* P, const double* R,
                       const double* x, ofwd* f) {
  const int n = t->n_up + t->n_down, N = t->n_nuc, L = t->n_layers, K = t->n_det;
  memset(f, 0, sizeof *f);
  f->t = t; f->n = n; f->N = N; f->L = L;
  f->dist = calloc((size_t)n * N, sizeof(double));
  /* layer-0 inputs */
  f->h[0] = calloc((size_t)n * 4 * N, sizeof(double));
  for (int i = 0; i < n; ++i)
    for (int I = 0; I < N; ++I) {
      double d[3], r2 = 0;
      for (int a = 0; a < 3; ++a) { d[a] = x[3 * i + a] - R[3 * I + a]; r2 += d[a] * d[a]; }
      double r = sqrt(r2);
      f->dist[i * N + I] = r;
      for (int a = 0; a < 3; ++a) f->h[0][(size_t)i * 4 * N + 4 * I + a] = d[a];
      f->h[0][(size_t)i * 4 * N + 4 * I + 3] = r;
    }
  f->e[0] = calloc((size_t)n * n * 4, sizeof(double));
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < n; ++j) {
      if (i == j) continue;
      double d[3], r2 = 0;
      for (int a = 0; a < 3; ++a) { d[a] = x[3 * i + a] - x[3 * j + a]; r2 += d[a] * d[a]; }
      for (int a = 0; a < 3; ++a) f->e[0][((size_t)i * n + j) * 4 + a] = d[a];
      f->e[0][((size_t)i * n + j) * 4 + 3] = sqrt(r2);
    }
  /* layers */
  for (int l = 0; l < L; ++l) {
    const int a1 = din1_of(t, l), a2 = din2_of(t, l), d1 = t->d1, d2 = t->d2;
    const int wV = 3 * a1 + 2 * a2;
    const double* V = P + Lo->V[l];
    const double* b = P + Lo->b[l];
    f->m1[l] = calloc((size_t)2 * a1, sizeof(double));
    f->m2[l] = calloc((size_t)n * 2 * a2, sizeof(double));
    for (int i = 0; i < n; ++i) {
      int s = i < t->n_up ? 0 : 1;
      for (int k = 0; k < a1; ++k) f->m1[l][s * a1 + k] += f->h[l][(size_t)i * a1 + k] / nspin(t, s);
    }
    for (int i = 0; i < n; ++i)
      for (int j = 0; j < n; ++j) {
        int s = j < t->n_up ? 0 : 1;
        for (int k = 0; k < a2; ++k)
          f->m2[l][((size_t)i * 2 + s) * a2 + k] += f->e[l][((size_t)i * n + j) * a2 + k] / nspin(t, s);
      }
    f->h[l + 1] = calloc((size_t)n * d1, sizeof(double));
    f->y1[l] = calloc((size_t)n * d1, sizeof(double));
    double* g = malloc(sizeof(double) * wV);
    for (int i = 0; i < n; ++i) {
      memcpy(g, f->h[l] + (size_t)i * a1, sizeof(double) * a1);
      memcpy(g + a1, f->m1[l], sizeof(double) * 2 * a1);
      memcpy(g + 3 * a1, f->m2[l] + (size_t)i * 2 * a2, sizeof(double) * 2 * a2);
      for (int o = 0; o < d1; ++o) {
        double z = b[o];
        for (int k = 0; k < wV; ++k) z += V[(size_t)o * wV + k] * g[k];
        double y = tanh(z);
        f->y1[l][(size_t)i * d1 + o] = y;
        f->h[l + 1][(size_t)i * d1 + o] = y + (l >= 1 ? f->h[l][(size_t)i * a1 + o] : 0.0);
      }
    }
    free(g);
    if (l < L - 1) {
      const double* W = P + Lo->W[l];
      const double* c = P + Lo->c[l];
      f->e[l + 1] = calloc((size_t)n * n * d2, sizeof(double));
      f->y2[l] = calloc((size_t)n * n * d2, sizeof(double));
      for (int p = 0; p < n * n; ++p)
        for (int o = 0; o < d2; ++o) {
          double z = c[o];
          for (int k = 0; k < a2; ++k) z += W[(size_t)o * a2 + k] * f->e[l][(size_t)p * a2 + k];
          double y = tanh(z);
          f->y2[l][(size_t)p * d2 + o] = y;
          f->e[l + 1][(size_t)p * d2 + o] = y + (l >= 1 ? f->e[l][(size_t)p * a2 + o] : 0.0);
        }
    }
  }
  /* orbitals, envelopes, determinants */
  f->ldet = calloc((size_t)K * 2, sizeof(double));
  f->sdet = calloc((size_t)K * 2, sizeof(double));
  const double* hL = f->h[L];
  for (int s = 0; s < 2; ++s) {
    const int ns = nspin(t, s), j0 = s == 0 ? 0 : t->n_up;
    size_t mat = (size_t)ns * ns;
    f->orb[s] = calloc(K * mat + 1, sizeof(double));
    f->env[s] = calloc(K * mat + 1, sizeof(double));
    f->A[s] = calloc(K * mat + 1, sizeof(double));
    f->Ainv[s] = calloc(K * mat + 1, sizeof(double));
    const double* w = P + Lo->w_orb[s];
    const double* go = P + Lo->g_orb[s];
    const double* pi = P + Lo->pi[s];
    const double* sg = P + Lo->sigma[s];
    for (int k = 0; k < K; ++k) {
      for (int i = 0; i < ns; ++i)
        for (int j = 0; j < ns; ++j) {
          double o = go[k * ns + i];
          for (int q = 0; q < t->d1; ++q) o += w[((size_t)k * ns + i) * t->d1 + q] * hL[(size_t)(j0 + j) * t->d1 + q];
          double en = 0.0;
          for (int m = 0; m < N; ++m) {
            size_t pm = ((size_t)k * ns + i) * N + m;
            const double* dv = f->h[0] + (size_t)(j0 + j) * 4 * N + 4 * m;  /* r_j - R_m */
            en += pi[pm] * env_term(t, sg + pm * (t->envelope ? 9 : 1), dv);
          }
          f->orb[s][k * mat + i * ns + j] = o;
          f->env[s][k * mat + i * ns + j] = en;
          f->A[s][k * mat + i * ns + j] = o * en;
        }
      double sgn, la;
      oracle_slogdet(ns, f->A[s] + k * mat, &sgn, &la);
      f->sdet[k * 2 + s] = sgn;
      f->ldet[k * 2 + s] = la;
      if (ns > 0 && lu_inverse(ns, f->A[s] + k * mat, f->Ainv[s] + k * mat)) f->singular = 1;
    }
  }
  /* signed log-sum-exp over determinants */
  double lmax = -INFINITY;
  for (int k = 0; k < K; ++k) {
    double lk = f->ldet[2 * k] + f->ldet[2 * k + 1];
    if (lk > lmax) lmax = lk;
  }
  double acc = 0.0;
  for (int k = 0; k < K; ++k) {
    double lk = f->ldet[2 * k] + f->ldet[2 * k + 1];
    double sk = f->sdet[2 * k] * f->sdet[2 * k + 1];
    if (sk != 0.0) acc += sk * exp(lk - lmax);
  }
  f->sign = acc > 0 ? 1.0 : (acc < 0 ? -1.0 : 0.0);
  f->logpsi = (acc == 0.0) ? -INFINITY : lmax + log(fabs(acc));
}

/* ------------------------------------------------------------------------ */
/* Reverse pass: seed * d log|psi| / d theta, accumulated into grad          */
/* ------------------------------------------------------------------------ */

/* Optional per-row accumulation of Kronecker factors during the reverse pass
 * (KFAC; see oracle_kfac_factors).  Each matrix is summed, not averaged. */
typedef struct {
  double* A1[16]; double* G1[16];   /* one-electron layers: [wV+1]^2, [d1]^2   */
  double* A2[16]; double* G2[16];   /* two-electron layers: [din2+1]^2, [d2]^2 */
  double* Ao[2]; double* Go[2];     /* orbital blocks per spin: [d1+1]^2, [K n_s]^2 */
} okfac;

static void outer_acc(double* M, const double* u, int n) {
  for (int a = 0; a < n; ++a)
    if (u[a] != 0.0)
      for (int b = 0; b < n; ++b) M[(size_t)a * n + b] += u[a] * u[b];
}

static void oracle_bwd(const onet* t, const olayout* Lo, const double* P, const double* R,
                       const ofwd* f, double seed, double* G, okfac* kf) {
  const int n = f->n, N = f->N, L = f->L, K = t->n_det, d1 = t->d1, d2 = t->d2;
  (void)R;
  if (f->sign == 0.0) return;
  /* d logpsi / d l_k = psi_k / psi */
  double* hbar = calloc((size_t)n * d1, sizeof(double));        /* d/d h^L */
  for (int s = 0; s < 2; ++s) {
    const int ns = nspin(t, s), j0 = s == 0 ? 0 : t->n_up;
    if (ns == 0) continue;
    size_t mat = (size_t)ns * ns;
    const double* w = P + Lo->w_orb[s];
    const double* pi = P + Lo->pi[s];
    const double* sg = P + Lo->sigma[s];
    /* KFAC rows of the orbital layer: electron j's gradient over this spin's
     * K n_s orbitals, and its input [h^L_j, 1] */
    double* orow = kf ? calloc((size_t)ns * K * ns, sizeof(double)) : NULL;
    for (int k = 0; k < K; ++k) {
      double lk = f->ldet[2 * k] + f->ldet[2 * k + 1];
      double sk = f->sdet[2 * k] * f->sdet[2 * k + 1];
      double wk = sk * f->sign * exp(lk - f->logpsi);
      double lbar = seed * wk;
      for (int i = 0; i < ns; ++i)
        for (int j = 0; j < ns; ++j) {
          /* d log|det A| / d A_ij = (A^-1)_ji */
          double Abar = lbar * f->Ainv[s][k * mat + j * ns + i];
          double obar = Abar * f->env[s][k * mat + i * ns + j];
          double ebar = Abar * f->orb[s][k * mat + i * ns + j];
          /* o = w_i . h_j + g_i */
          G[Lo->g_orb[s] + k * ns + i] += obar;
          if (orow) orow[(size_t)j * K * ns + k * ns + i] = obar;
          for (int q = 0; q < d1; ++q) {
            G[Lo->w_orb[s] + ((size_t)k * ns + i) * d1 + q] += obar * f->h[L][(size_t)(j0 + j) * d1 + q];
            hbar[(size_t)(j0 + j) * d1 + q] += obar * w[((size_t)k * ns + i) * d1 + q];
          }
          /* env = sum_m pi exp(-|sigma| r), or sum_m pi exp(-|Sigma d|) */
          for (int m = 0; m < N; ++m) {
            size_t pm = ((size_t)k * ns + i) * N + m;
            if (!t->envelope) {
              double r = f->dist[(j0 + j) * N + m];
              double ex = exp(-fabs(sg[pm]) * r);
              double sgn = sg[pm] > 0 ? 1.0 : (sg[pm] < 0 ? -1.0 : 0.0);
              G[Lo->pi[s] + pm] += ebar * ex;
              G[Lo->sigma[s] + pm] += ebar * pi[pm] * ex * (-r) * sgn;
            } else {
              /* v = Sigma d, rho = |v|: d exp(-rho) / d Sigma_ab = -exp(-rho) v_a d_b / rho */
              const double* dv = f->h[0] + (size_t)(j0 + j) * 4 * N + 4 * m;
              const double* S = sg + pm * 9;
              double v[3], rho2 = 0.0;
              for (int a = 0; a < 3; ++a) {
                v[a] = S[3 * a] * dv[0] + S[3 * a + 1] * dv[1] + S[3 * a + 2] * dv[2];
                rho2 += v[a] * v[a];
              }
              const double rho = sqrt(rho2), ex = exp(-rho);
              G[Lo->pi[s] + pm] += ebar * ex;
              if (rho > 0.0)
                for (int a = 0; a < 3; ++a)
                  for (int b = 0; b < 3; ++b)
                    G[Lo->sigma[s] + pm * 9 + 3 * a + b] += ebar * pi[pm] * ex * (-v[a] * dv[b] / rho);
            }
          }
        }
    }
    if (orow) {
      double* ab = malloc(sizeof(double) * (d1 + 1));
      for (int j = 0; j < ns; ++j) {
        outer_acc(kf->Go[s], orow + (size_t)j * K * ns, K * ns);
        memcpy(ab, f->h[L] + (size_t)(j0 + j) * d1, sizeof(double) * d1);
        ab[d1] = 1.0;
        outer_acc(kf->Ao[s], ab, d1 + 1);
      }
      free(ab);
      free(orow);
    }
  }
  /* layers, last to first */
  double* ebar_next = NULL;  /* d/d e[l+1] */
  for (int l = L - 1; l >= 0; --l) {
    const int a1 = din1_of(t, l), a2 = din2_of(t, l), wV = 3 * a1 + 2 * a2;
    double* ebar = calloc((size_t)n * n * a2, sizeof(double));    /* d/d e[l] */
    /* two-electron layer l maps e[l] -> e[l+1] */
    if (l < L - 1) {
      const double* W = P + Lo->W[l];
      double* zrow = kf ? malloc(sizeof(double) * d2) : NULL;
      double* arow = kf ? malloc(sizeof(double) * (a2 + 1)) : NULL;
      for (int p = 0; p < n * n; ++p) {
        for (int o = 0; o < d2; ++o) {
          double eb = ebar_next[(size_t)p * d2 + o];
          double y = f->y2[l][(size_t)p * d2 + o];
          double zb = eb * (1.0 - y * y);
          if (zrow) zrow[o] = zb;
          G[Lo->c[l] + o] += zb;
          for (int k = 0; k < a2; ++k) {
            G[Lo->W[l] + (size_t)o * a2 + k] += zb * f->e[l][(size_t)p * a2 + k];
            ebar[(size_t)p * a2 + k] += zb * W[(size_t)o * a2 + k];
          }
          if (l >= 1) ebar[(size_t)p * a2 + o] += eb;
        }
        if (kf) {
          outer_acc(kf->G2[l], zrow, d2);
          memcpy(arow, f->e[l] + (size_t)p * a2, sizeof(double) * a2);
          arow[a2] = 1.0;
          outer_acc(kf->A2[l], arow, a2 + 1);
        }
      }
      free(zrow);
      free(arow);
    }
    /* one-electron layer l maps h[l] -> h[l+1] */
    const double* V = P + Lo->V[l];
    double* hbar_prev = calloc((size_t)n * a1, sizeof(double));
    double* m1bar = calloc((size_t)2 * a1, sizeof(double));
    double* gbar = malloc(sizeof(double) * wV);
    double* g = malloc(sizeof(double) * (wV + 1));
    double* zrow = kf ? malloc(sizeof(double) * d1) : NULL;
    for (int i = 0; i < n; ++i) {
      memcpy(g, f->h[l] + (size_t)i * a1, sizeof(double) * a1);
      memcpy(g + a1, f->m1[l], sizeof(double) * 2 * a1);
      memcpy(g + 3 * a1, f->m2[l] + (size_t)i * 2 * a2, sizeof(double) * 2 * a2);
      memset(gbar, 0, sizeof(double) * wV);
      for (int o = 0; o < d1; ++o) {
        double hb = hbar[(size_t)i * d1 + o];
        double y = f->y1[l][(size_t)i * d1 + o];
        double zb = hb * (1.0 - y * y);
        if (zrow) zrow[o] = zb;
        G[Lo->b[l] + o] += zb;
        for (int k = 0; k < wV; ++k) {
          G[Lo->V[l] + (size_t)o * wV + k] += zb * g[k];
          gbar[k] += zb * V[(size_t)o * wV + k];
        }
        if (l >= 1) hbar_prev[(size_t)i * a1 + o] += hb;
      }
      if (kf) {  /* KFAC row: input [g_i, 1] and pre-activation gradient */
        g[wV] = 1.0;
        outer_acc(kf->A1[l], g, wV + 1);
        outer_acc(kf->G1[l], zrow, d1);
      }
      for (int k = 0; k < a1; ++k) hbar_prev[(size_t)i * a1 + k] += gbar[k];
      for (int k = 0; k < 2 * a1; ++k) m1bar[k] += gbar[a1 + k];
      /* m2[i][s] = mean_{j in s} e[l][i][j] */
      for (int j = 0; j < n; ++j) {
        int s = j < t->n_up ? 0 : 1;
        for (int k = 0; k < a2; ++k)
          ebar[((size_t)i * n + j) * a2 + k] += gbar[3 * a1 + s * a2 + k] / nspin(t, s);
      }
    }
    for (int i = 0; i < n; ++i) {
      int s = i < t->n_up ? 0 : 1;
      for (int k = 0; k < a1; ++k) hbar_prev[(size_t)i * a1 + k] += m1bar[s * a1 + k] / nspin(t, s);
    }
    free(gbar); free(g); free(m1bar); free(zrow);
    free(hbar); hbar = hbar_prev;
    free(ebar_next); ebar_next = ebar;
  }
  free(hbar); free(ebar_next);
}

/* ------------------------------------------------------------------------ */
/* Jet (univariate second-order Taylor) arithmetic                           */
/* ------------------------------------------------------------------------ */

typedef struct { double v, d, dd; } jet;

static jet jc(double v) { jet r = {v, 0, 0}; return r; }
static jet jadd(jet a, jet b) { jet r = {a.v + b.v, a.d + b.d, a.dd + b.dd}; return r; }
static jet jsub(jet a, jet b) { jet r = {a.v - b.v, a.d - b.d, a.dd - b.dd}; return r; }
static jet jscale(jet a, double s) { jet r = {a.v * s, a.d * s, a.dd * s}; return r; }
static jet jmul(jet a, jet b) {
  jet r = {a.v * b.v, a.d * b.v + a.v * b.d, a.dd * b.v + 2 * a.d * b.d + a.v * b.dd};
  return r;
}
static jet jdiv(jet a, jet b) {
  jet q; q.v = a.v / b.v;
  q.d = (a.d - q.v * b.d) / b.v;
  q.dd = (a.dd - 2 * q.d * b.d - q.v * b.dd) / b.v;
  return q;
}
static jet jtanh(jet a) {
  double y = tanh(a.v), s = 1 - y * y;
  jet r = {y, s * a.d, s * a.dd - 2 * y * s * a.d * a.d};
  return r;
}
static jet jexp(jet a) {
  double e = exp(a.v);
  jet r = {e, e * a.d, e * (a.dd + a.d * a.d)};
  return r;
}
static jet jlogabs(jet a) {
  jet r = {log(fabs(a.v)), a.d / a.v, a.dd / a.v - (a.d * a.d) / (a.v * a.v)};
  return r;
}
/* sqrt of a jet; a jet that is identically zero maps to zero (the |r| of a
 * coincident pair, e.g. h^0_ii, whose derivative is taken as 0). */
static jet jsqrt(jet a) {
  if (a.v == 0.0) return jc(0.0);
  double s = sqrt(a.v);
  jet r = {s, a.d / (2 * s), a.dd / (2 * s) - a.d * a.d / (4 * s * s * s)};
  return r;
}

/* log|det| and sign of a jet-valued matrix by LU with partial pivoting on the
 * value part.  Returns sign 0 for a singular value matrix. */
static void jslogdet(int n, jet* a, double* sign, jet* logabs) {
  double s = 1.0;
  jet la = jc(0.0);
  for (int k = 0; k < n; ++k) {
    int p = k;
    double best = fabs(a[k * n + k].v);
    for (int i = k + 1; i < n; ++i)
      if (fabs(a[i * n + k].v) > best) { best = fabs(a[i * n + k].v); p = i; }
    if (p != k) {
      for (int j = 0; j < n; ++j) { jet t = a[k * n + j]; a[k * n + j] = a[p * n + j]; a[p * n + j] = t; }
      s = -s;
    }
    jet u = a[k * n + k];
    if (u.v == 0.0) { *sign = 0.0; logabs->v = -INFINITY; logabs->d = logabs->dd = 0; return; }
    if (u.v < 0) s = -s;
    la = jadd(la, jlogabs(u));
    for (int i = k + 1; i < n; ++i) {
      jet l = jdiv(a[i * n + k], u);
      for (int j = k + 1; j < n; ++j) a[i * n + j] = jsub(a[i * n + j], jmul(l, a[k * n + j]));
    }
  }
  *sign = s; *logabs = la;
}

/* log|psi| as a jet in the single coordinate `seed_coord` (electron
 * seed_coord/3, component seed_coord%3); seed_coord < 0 seeds nothing.
 * Same network as oracle_fwd, evaluated in jet arithmetic. */
static jet oracle_fwd_jet(const onet* t, const olayout* Lo, const double* P, const double* R,
                          const double* x, int seed_coord, double* sign_out) {
  const int n = t->n_up + t->n_down, N = t->n_nuc, L = t->n_layers, K = t->n_det;
  jet* xr = malloc(sizeof(jet) * 3 * n);
  for (int q = 0; q < 3 * n; ++q) { xr[q] = jc(x[q]); if (q == seed_coord) xr[q].d = 1.0; }
  jet* dist = malloc(sizeof(jet) * n * N);
  jet* disp = malloc(sizeof(jet) * n * N * 3);  /* r_i - R_I, for the full-covariance envelope */
  int maxw = 4 * N > t->d1 ? 4 * N : t->d1;
  int maxw2 = t->d2 > 4 ? t->d2 : 4;
  jet* h = calloc((size_t)n * maxw, sizeof(jet));
  jet* hn = calloc((size_t)n * maxw, sizeof(jet));
  jet* e = calloc((size_t)n * n * maxw2, sizeof(jet));
  jet* en = calloc((size_t)n * n * maxw2, sizeof(jet));
  for (int i = 0; i < n; ++i)
    for (int I = 0; I < N; ++I) {
      jet r2 = jc(0.0), d[3];
      for (int a = 0; a < 3; ++a) { d[a] = jsub(xr[3 * i + a], jc(R[3 * I + a])); r2 = jadd(r2, jmul(d[a], d[a])); }
      jet r = jsqrt(r2);
      dist[i * N + I] = r;
      for (int a = 0; a < 3; ++a) disp[((size_t)i * N + I) * 3 + a] = d[a];
      for (int a = 0; a < 3; ++a) h[(size_t)i * 4 * N + 4 * I + a] = d[a];
      h[(size_t)i * 4 * N + 4 * I + 3] = r;
    }
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < n; ++j) {
      jet* dst = e + ((size_t)i * n + j) * 4;
      if (i == j) { for (int a = 0; a < 4; ++a) dst[a] = jc(0.0); continue; }
      jet r2 = jc(0.0);
      for (int a = 0; a < 3; ++a) { dst[a] = jsub(xr[3 * i + a], xr[3 * j + a]); r2 = jadd(r2, jmul(dst[a], dst[a])); }
      dst[3] = jsqrt(r2);
    }
  for (int l = 0; l < L; ++l) {
    const int a1 = din1_of(t, l), a2 = din2_of(t, l), d1 = t->d1, d2 = t->d2, wV = 3 * a1 + 2 * a2;
    const double* V = P + Lo->V[l];
    const double* b = P + Lo->b[l];
    jet* m1 = calloc((size_t)2 * a1, sizeof(jet));
    jet* m2 = calloc((size_t)n * 2 * a2, sizeof(jet));
    for (int i = 0; i < n; ++i) {
      int s = i < t->n_up ? 0 : 1;
      for (int k = 0; k < a1; ++k) m1[s * a1 + k] = jadd(m1[s * a1 + k], jscale(h[(size_t)i * a1 + k], 1.0 / nspin(t, s)));
    }
    for (int i = 0; i < n; ++i)
      for (int j = 0; j < n; ++j) {
        int s = j < t->n_up ? 0 : 1;
        for (int k = 0; k < a2; ++k)
          m2[((size_t)i * 2 + s) * a2 + k] = jadd(m2[((size_t)i * 2 + s) * a2 + k],
                                                  jscale(e[((size_t)i * n + j) * a2 + k], 1.0 / nspin(t, s)));
      }
    jet* g = malloc(sizeof(jet) * wV);
    for (int i = 0; i < n; ++i) {
      memcpy(g, h + (size_t)i * a1, sizeof(jet) * a1);
      memcpy(g + a1, m1, sizeof(jet) * 2 * a1);
      memcpy(g + 3 * a1, m2 + (size_t)i * 2 * a2, sizeof(jet) * 2 * a2);
      for (int o = 0; o < d1; ++o) {
        jet z = jc(b[o]);
        for (int k = 0; k < wV; ++k) z = jadd(z, jscale(g[k], V[(size_t)o * wV + k]));
        jet y = jtanh(z);
        hn[(size_t)i * d1 + o] = l >= 1 ? jadd(y, h[(size_t)i * a1 + o]) : y;
      }
    }
    free(g); free(m1); free(m2);
    if (l < L - 1) {
      const double* W = P + Lo->W[l];
      const double* c = P + Lo->c[l];
      for (int p = 0; p < n * n; ++p)
        for (int o = 0; o < d2; ++o) {
          jet z = jc(c[o]);
          for (int k = 0; k < a2; ++k) z = jadd(z, jscale(e[(size_t)p * a2 + k], W[(size_t)o * a2 + k]));
          jet y = jtanh(z);
          en[(size_t)p * d2 + o] = l >= 1 ? jadd(y, e[(size_t)p * a2 + o]) : y;
        }
      jet* tmp = e; e = en; en = tmp;
    }
    jet* tmp = h; h = hn; hn = tmp;
  }
  /* determinants */
  jet* lk = malloc(sizeof(jet) * K);
  double* sk = malloc(sizeof(double) * K);
  for (int k = 0; k < K; ++k) { lk[k] = jc(0.0); sk[k] = 1.0; }
  for (int s = 0; s < 2; ++s) {
    const int ns = nspin(t, s), j0 = s == 0 ? 0 : t->n_up;
    if (ns == 0) continue;
    const double* w = P + Lo->w_orb[s];
    const double* go = P + Lo->g_orb[s];
    const double* pi = P + Lo->pi[s];
    const double* sg = P + Lo->sigma[s];
    jet* A = malloc(sizeof(jet) * ns * ns);
    for (int k = 0; k < K; ++k) {
      for (int i = 0; i < ns; ++i)
        for (int j = 0; j < ns; ++j) {
          jet o = jc(go[k * ns + i]);
          for (int q = 0; q < t->d1; ++q)
            o = jadd(o, jscale(h[(size_t)(j0 + j) * t->d1 + q], w[((size_t)k * ns + i) * t->d1 + q]));
          jet env = jc(0.0);
          for (int m = 0; m < N; ++m) {
            size_t pm = ((size_t)k * ns + i) * N + m;
            if (!t->envelope) {
              env = jadd(env, jscale(jexp(jscale(dist[(j0 + j) * N + m], -fabs(sg[pm]))), pi[pm]));
            } else {
              const double* S = sg + pm * 9;
              const jet* dv = disp + ((size_t)(j0 + j) * N + m) * 3;
              jet rho2 = jc(0.0);
              for (int a = 0; a < 3; ++a) {
                jet va = jadd(jadd(jscale(dv[0], S[3 * a]), jscale(dv[1], S[3 * a + 1])), jscale(dv[2], S[3 * a + 2]));
                rho2 = jadd(rho2, jmul(va, va));
              }
              env = jadd(env, jscale(jexp(jscale(jsqrt(rho2), -1.0)), pi[pm]));
            }
          }
          A[i * ns + j] = jmul(o, env);
        }
      double sgn; jet la;
      jslogdet(ns, A, &sgn, &la);
      sk[k] *= sgn;
      lk[k] = jadd(lk[k], la);
    }
    free(A);
  }
  /* signed log-sum-exp in jets: lmax + log|sum_k s_k exp(l_k - lmax)| */
  int kmax = -1;
  for (int k = 0; k < K; ++k) if (sk[k] != 0.0 && (kmax < 0 || lk[k].v > lk[kmax].v)) kmax = k;
  jet out;
  if (kmax < 0) { out.v = -INFINITY; out.d = out.dd = 0; *sign_out = 0.0; }
  else {
    jet acc = jc(0.0);
    for (int k = 0; k < K; ++k)
      if (sk[k] != 0.0) acc = jadd(acc, jscale(jexp(jsub(lk[k], lk[kmax])), sk[k]));
    *sign_out = acc.v > 0 ? 1.0 : (acc.v < 0 ? -1.0 : 0.0);
    out = acc.v == 0.0 ? jc(-INFINITY) : jadd(lk[kmax], jlogabs(acc));
  }
  free(lk); free(sk); free(xr); free(dist); free(disp); free(h); free(hn); free(e); free(en);
  return out;
}

/* ------------------------------------------------------------------------ */
/* Coulomb potential (Eq. 1)                                                 */
/* ------------------------------------------------------------------------ */

double oracle_nuclear_repulsion(int N, const double* R, const double* Z) {
  double v = 0.0;
  for (int I = 0; I < N; ++I)
    for (int J = 0; J < I; ++J) {
      double r2 = 0;
      for (int a = 0; a < 3; ++a) { double d = R[3 * I + a] - R[3 * J + a]; r2 += d * d; }
      v += Z[I] * Z[J] / sqrt(r2);
    }
  return v;
}

/* V = sum_{i>j} 1/r_ij - sum_{i,I} Z_I / r_iI + sum_{I>J} Z_I Z_J / R_IJ */
double oracle_potential(int n, int N, const double* R, const double* Z, const double* x) {
  double v = 0.0;
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < i; ++j) {
      double r2 = 0;
      for (int a = 0; a < 3; ++a) { double d = x[3 * i + a] - x[3 * j + a]; r2 += d * d; }
      v += 1.0 / sqrt(r2);
    }
  for (int i = 0; i < n; ++i)
    for (int I = 0; I < N; ++I) {
      double r2 = 0;
      for (int a = 0; a < 3; ++a) { double d = x[3 * i + a] - R[3 * I + a]; r2 += d * d; }
      v -= Z[I] / sqrt(r2);
    }
  return v + oracle_nuclear_repulsion(N, R, Z);
}

/* ------------------------------------------------------------------------ */
/* Batch entry points (one geometry index per walker)                        */
/* ------------------------------------------------------------------------ */

/* Walker w uses nuclei R[geo[w]] [N][3] and charges Z[geo[w]] [N]; geo may be
 * NULL (all walkers on geometry 0). */
#define GEO(w) (geo ? geo[w] : 0)

int oracle_logpsi(const onet* t, const double* P, const double* R, const double* Z, const int* geo,
                  long B, const double* x, double* logpsi, double* sign) {
  (void)Z;
  if (check_net(t)) return -1;
  olayout Lo; build_layout(t, &Lo, NULL, 0);
  const int n = t->n_up + t->n_down, N = t->n_nuc;
#pragma omp parallel for schedule(dynamic, 1)
  for (long w = 0; w < B; ++w) {
    ofwd f;
    oracle_fwd(t, &Lo, P, R + (size_t)GEO(w) * 3 * N, x + (size_t)w * 3 * n, &f);
    logpsi[w] = f.logpsi;
    sign[w] = f.sign;
    fwd_free(&f);
  }
  return 0;
}

/* Jet evaluation: logpsi, sign, grad [B][3n] (may be NULL), per-coordinate
 * second derivatives d2 [B][3n] (may be NULL), kinetic, potential, E_L. */
int oracle_local_energy(const onet* t, const double* P, const double* R, const double* Z, const int* geo,
                        long B, const double* x, double* logpsi, double* sign, double* grad, double* d2,
                        double* kinetic, double* potential, double* eloc) {
  if (check_net(t)) return -1;
  olayout Lo; build_layout(t, &Lo, NULL, 0);
  const int n = t->n_up + t->n_down, N = t->n_nuc;
#pragma omp parallel for schedule(dynamic, 1)
  for (long w = 0; w < B; ++w) {
    const double* Rw = R + (size_t)GEO(w) * 3 * N;
    const double* Zw = Z + (size_t)GEO(w) * N;
    const double* xw = x + (size_t)w * 3 * n;
    double T = 0.0, sg = 0.0;
    jet lp = jc(0.0);
    for (int c = 0; c < 3 * n; ++c) {
      lp = oracle_fwd_jet(t, &Lo, P, Rw, xw, c, &sg);
      if (grad) grad[(size_t)w * 3 * n + c] = lp.d;
      if (d2) d2[(size_t)w * 3 * n + c] = lp.dd;
      T += -0.5 * (lp.dd + lp.d * lp.d);
    }
    double V = oracle_potential(n, N, Rw, Zw, xw);
    if (logpsi) logpsi[w] = lp.v;
    if (sign) sign[w] = sg;
    if (kinetic) kinetic[w] = T;
    if (potential) potential[w] = V;
    if (eloc) eloc[w] = T + V;
  }
  return 0;
}

/* grad_theta[P] = sum_w seeds[w] * d log|psi_w| / d theta. */
int oracle_logpsi_vjp(const onet* t, const double* P, const double* R, const double* Z, const int* geo,
                      long B, const double* x, const double* seeds, double* grad) {
  (void)Z;
  if (check_net(t)) return -1;
  olayout Lo; build_layout(t, &Lo, NULL, 0);
  const int n = t->n_up + t->n_down, N = t->n_nuc;
  memset(grad, 0, sizeof(double) * Lo.total);
  for (long w = 0; w < B; ++w) {
    ofwd f;
    oracle_fwd(t, &Lo, P, R + (size_t)GEO(w) * 3 * N, x + (size_t)w * 3 * n, &f);
    oracle_bwd(t, &Lo, P, R + (size_t)GEO(w) * 3 * N, &f, seeds[w], grad, NULL);
    fwd_free(&f);
  }
  return 0;
}

/* ------------------------------------------------------------------------ */
/* KFAC (the optimiser the paper credits for FermiNet's accuracy, Sec. 1;    */
/* Martens and Grosse 2015): Kronecker factors of the Fisher of log|psi|     */
/* per layer, and the damped preconditioned update                           */
/* ------------------------------------------------------------------------ */

/* Factor buffer layout (doubles), in this order:
 *   for each layer l: A1_l [wV+1]^2 (inputs [g_i, 1]), G1_l [d1]^2
 *                     (pre-activation gradients of log|psi|);
 *   for each l < L-1: A2_l [din2+1]^2 (inputs [e_ij, 1]), G2_l [d2]^2;
 *   for each spin s:  Ao_s [d1+1]^2 (inputs [h^L_j, 1]), Go_s [K n_s]^2
 *                     (gradients over the spin's K n_s orbitals);
 *   D: the envelope parameters (pi and sigma blocks, in layout order), the
 *      mean over walkers of the squared per-walker gradient (diagonal).
 * Averages: A1 over B n rows, A2 over B n^2 rows, Ao_s over B n_s rows; every
 * G and D over the B walkers (summed over a walker's rows). */
typedef struct { long A1[16], G1[16], A2[16], G2[16], Ao[2], Go[2], D, total; } okfac_layout;

static void kfac_layout(const onet* t, const olayout* Lo, okfac_layout* K) {
  long off = 0;
  const int L = t->n_layers;
  for (int l = 0; l < L; ++l) {
    const long a = 3L * din1_of(t, l) + 2L * din2_of(t, l) + 1;
    K->A1[l] = off; off += a * a;
    K->G1[l] = off; off += (long)t->d1 * t->d1;
  }
  for (int l = 0; l < L - 1; ++l) {
    const long a = din2_of(t, l) + 1;
    K->A2[l] = off; off += a * a;
    K->G2[l] = off; off += (long)t->d2 * t->d2;
  }
  for (int s = 0; s < 2; ++s) {
    const long g = (long)t->n_det * nspin(t, s);
    K->Ao[s] = off; off += (long)(t->d1 + 1) * (t->d1 + 1);
    K->Go[s] = off; off += g * g;
  }
  K->D = off; off += Lo->total - Lo->pi[0];
  K->total = off;
}

long oracle_kfac_size(const onet* t) {
  if (check_net(t)) return -1;
  olayout Lo; build_layout(t, &Lo, NULL, 0);
  okfac_layout K; kfac_layout(t, &Lo, &K);
  return K.total;
}

/* Kronecker factors over the batch (every walker on geometry geo[w]). */
int oracle_kfac_factors(const onet* t, const double* P, const double* R, const double* Z, const int* geo, long B,
                        const double* x, double* F) {
  (void)Z;
  if (check_net(t) || B < 1) return -1;
  olayout Lo; build_layout(t, &Lo, NULL, 0);
  okfac_layout KL; kfac_layout(t, &Lo, &KL);
  const int n = t->n_up + t->n_down, N = t->n_nuc, L = t->n_layers;
  memset(F, 0, sizeof(double) * KL.total);
  okfac kf;
  memset(&kf, 0, sizeof kf);
  for (int l = 0; l < L; ++l) { kf.A1[l] = F + KL.A1[l]; kf.G1[l] = F + KL.G1[l]; }
  for (int l = 0; l < L - 1; ++l) { kf.A2[l] = F + KL.A2[l]; kf.G2[l] = F + KL.G2[l]; }
  for (int s = 0; s < 2; ++s) { kf.Ao[s] = F + KL.Ao[s]; kf.Go[s] = F + KL.Go[s]; }
  const long ne = Lo.total - Lo.pi[0];
  double* gw = malloc(sizeof(double) * Lo.total);
  for (long w = 0; w < B; ++w) {
    ofwd f;
    oracle_fwd(t, &Lo, P, R + (size_t)GEO(w) * 3 * N, x + (size_t)w * 3 * n, &f);
    memset(gw, 0, sizeof(double) * Lo.total);
    oracle_bwd(t, &Lo, P, R + (size_t)GEO(w) * 3 * N, &f, 1.0, gw, &kf);
    for (long k = 0; k < ne; ++k) F[KL.D + k] += gw[Lo.pi[0] + k] * gw[Lo.pi[0] + k];
    fwd_free(&f);
  }
  free(gw);
  /* averages */
  for (int l = 0; l < L; ++l) {
    const long a = 3L * din1_of(t, l) + 2L * din2_of(t, l) + 1;
    for (long k = 0; k < a * a; ++k) F[KL.A1[l] + k] /= (double)B * n;
    for (long k = 0; k < (long)t->d1 * t->d1; ++k) F[KL.G1[l] + k] /= (double)B;
  }
  for (int l = 0; l < L - 1; ++l) {
    const long a = din2_of(t, l) + 1;
    for (long k = 0; k < a * a; ++k) F[KL.A2[l] + k] /= (double)B * n * n;
    for (long k = 0; k < (long)t->d2 * t->d2; ++k) F[KL.G2[l] + k] /= (double)B;
  }
  for (int s = 0; s < 2; ++s) {
    const long g = (long)t->n_det * nspin(t, s);
    for (long k = 0; k < (long)(t->d1 + 1) * (t->d1 + 1); ++k)
      F[KL.Ao[s] + k] = nspin(t, s) ? F[KL.Ao[s] + k] / ((double)B * nspin(t, s)) : 0.0;
    for (long k = 0; k < g * g; ++k) F[KL.Go[s] + k] /= (double)B;
  }
  for (long k = 0; k < ne; ++k) F[KL.D + k] /= (double)B;
  return 0;
}

/* Inverse of a symmetric positive definite n x n matrix by Gauss-Jordan
 * elimination (row pivoting kept for safety). */
static int gj_inverse(int n, const double* M, double* inv) {
  double* a = malloc(sizeof(double) * (size_t)n * n);
  memcpy(a, M, sizeof(double) * (size_t)n * n);
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < n; ++j) inv[(size_t)i * n + j] = i == j ? 1.0 : 0.0;
  for (int k = 0; k < n; ++k) {
    int p = k;
    for (int i = k + 1; i < n; ++i) if (fabs(a[(size_t)i * n + k]) > fabs(a[(size_t)p * n + k])) p = i;
    if (a[(size_t)p * n + k] == 0.0) { free(a); return -1; }
    if (p != k)
      for (int j = 0; j < n; ++j) {
        double u = a[(size_t)k * n + j]; a[(size_t)k * n + j] = a[(size_t)p * n + j]; a[(size_t)p * n + j] = u;
        u = inv[(size_t)k * n + j]; inv[(size_t)k * n + j] = inv[(size_t)p * n + j]; inv[(size_t)p * n + j] = u;
      }
    const double piv = a[(size_t)k * n + k];
    for (int j = 0; j < n; ++j) { a[(size_t)k * n + j] /= piv; inv[(size_t)k * n + j] /= piv; }
    for (int i = 0; i < n; ++i) {
      if (i == k) continue;
      const double fct = a[(size_t)i * n + k];
      if (fct == 0.0) continue;
      for (int j = 0; j < n; ++j) {
        a[(size_t)i * n + j] -= fct * a[(size_t)k * n + j];
        inv[(size_t)i * n + j] -= fct * inv[(size_t)k * n + j];
      }
    }
  }
  free(a);
  return 0;
}

/* Delta = (G + gamma I)^-1 M (A + gamma I)^-1 for M [g][a]. */
static int kfac_block(int g, int a, const double* G, const double* A, double gamma, const double* M, double* out) {
  double* Gi = malloc(sizeof(double) * (size_t)g * g);
  double* Ai = malloc(sizeof(double) * (size_t)a * a);
  double* Gd = malloc(sizeof(double) * (size_t)g * g);
  double* Ad = malloc(sizeof(double) * (size_t)a * a);
  double* X = calloc((size_t)g * a, sizeof(double));
  memcpy(Gd, G, sizeof(double) * (size_t)g * g);
  memcpy(Ad, A, sizeof(double) * (size_t)a * a);
  for (int i = 0; i < g; ++i) Gd[(size_t)i * g + i] += gamma;
  for (int i = 0; i < a; ++i) Ad[(size_t)i * a + i] += gamma;
  int rc = gj_inverse(g, Gd, Gi) | gj_inverse(a, Ad, Ai);
  if (!rc) {
    for (int i = 0; i < g; ++i)
      for (int k = 0; k < g; ++k) {
        const double c = Gi[(size_t)i * g + k];
        for (int j = 0; j < a; ++j) X[(size_t)i * a + j] += c * M[(size_t)k * a + j];
      }
    for (int i = 0; i < g; ++i)
      for (int j = 0; j < a; ++j) {
        double v = 0.0;
        for (int k = 0; k < a; ++k) v += X[(size_t)i * a + k] * Ai[(size_t)k * a + j];
        out[(size_t)i * a + j] = v;
      }
  }
  free(Gi); free(Ai); free(Gd); free(Ad); free(X);
  return rc;
}

/* KFAC-preconditioned update of a gradient over the whole parameter vector:
 * for each layer block (weights and bias together as M = [W b]),
 * Delta = (G + sqrt(lambda) I)^-1 M (A + sqrt(lambda) I)^-1; envelope entries
 * grad / (D + lambda). */
int oracle_kfac_precondition(const onet* t, const double* F, const double* grad, double lambda, double* out) {
  if (check_net(t) || !(lambda > 0)) return -1;
  olayout Lo; build_layout(t, &Lo, NULL, 0);
  okfac_layout KL; kfac_layout(t, &Lo, &KL);
  const int L = t->n_layers, d1 = t->d1, d2 = t->d2;
  const double gamma = sqrt(lambda);
  int rc = 0;
  for (int l = 0; l < L; ++l) {
    const int wV = 3 * din1_of(t, l) + 2 * din2_of(t, l), a = wV + 1;
    double* M = malloc(sizeof(double) * (size_t)d1 * a);
    double* D = malloc(sizeof(double) * (size_t)d1 * a);
    for (int o = 0; o < d1; ++o) {
      for (int k = 0; k < wV; ++k) M[(size_t)o * a + k] = grad[Lo.V[l] + (size_t)o * wV + k];
      M[(size_t)o * a + wV] = grad[Lo.b[l] + o];
    }
    rc |= kfac_block(d1, a, F + KL.G1[l], F + KL.A1[l], gamma, M, D);
    for (int o = 0; o < d1; ++o) {
      for (int k = 0; k < wV; ++k) out[Lo.V[l] + (size_t)o * wV + k] = D[(size_t)o * a + k];
      out[Lo.b[l] + o] = D[(size_t)o * a + wV];
    }
    free(M); free(D);
  }
  for (int l = 0; l < L - 1; ++l) {
    const int a2 = din2_of(t, l), a = a2 + 1;
    double* M = malloc(sizeof(double) * (size_t)d2 * a);
    double* D = malloc(sizeof(double) * (size_t)d2 * a);
    for (int o = 0; o < d2; ++o) {
      for (int k = 0; k < a2; ++k) M[(size_t)o * a + k] = grad[Lo.W[l] + (size_t)o * a2 + k];
      M[(size_t)o * a + a2] = grad[Lo.c[l] + o];
    }
    rc |= kfac_block(d2, a, F + KL.G2[l], F + KL.A2[l], gamma, M, D);
    for (int o = 0; o < d2; ++o) {
      for (int k = 0; k < a2; ++k) out[Lo.W[l] + (size_t)o * a2 + k] = D[(size_t)o * a + k];
      out[Lo.c[l] + o] = D[(size_t)o * a + a2];
    }
    free(M); free(D);
  }
  for (int s = 0; s < 2; ++s) {
    const int g = t->n_det * nspin(t, s), a = d1 + 1;
    if (g == 0) continue;
    double* M = malloc(sizeof(double) * (size_t)g * a);
    double* D = malloc(sizeof(double) * (size_t)g * a);
    for (int q = 0; q < g; ++q) {
      for (int f = 0; f < d1; ++f) M[(size_t)q * a + f] = grad[Lo.w_orb[s] + (size_t)q * d1 + f];
      M[(size_t)q * a + d1] = grad[Lo.g_orb[s] + q];
    }
    rc |= kfac_block(g, a, F + KL.Go[s], F + KL.Ao[s], gamma, M, D);
    for (int q = 0; q < g; ++q) {
      for (int f = 0; f < d1; ++f) out[Lo.w_orb[s] + (size_t)q * d1 + f] = D[(size_t)q * a + f];
      out[Lo.g_orb[s] + q] = D[(size_t)q * a + d1];
    }
    free(M); free(D);
  }
  for (long k = 0; k < Lo.total - Lo.pi[0]; ++k) out[Lo.pi[0] + k] = grad[Lo.pi[0] + k] / (F[KL.D + k] + lambda);
  return rc ? -1 : 0;
}

/* VMC energy gradient (Eq. 2 differentiated with E_L held fixed): per
 * geometry g, E_mean[g] = mean of eloc over its walkers, and
 * grad = sum_g 2/B_g sum_{w in g} (eloc_w - E_mean[g]) d log|psi_w| / d theta. */
int oracle_energy_grad(const onet* t, const double* P, const double* R, const double* Z, const int* geo,
                       int n_geo, long B, const double* x, const double* eloc, double* emean, double* grad) {
  if (check_net(t) || n_geo < 1) return -1;
  double* sum = calloc(n_geo, sizeof(double));
  long* cnt = calloc(n_geo, sizeof(long));
  for (long w = 0; w < B; ++w) { sum[GEO(w)] += eloc[w]; cnt[GEO(w)]++; }
  for (int g = 0; g < n_geo; ++g) emean[g] = cnt[g] ? sum[g] / cnt[g] : 0.0;
  double* seeds = malloc(sizeof(double) * (B > 0 ? B : 1));
  for (long w = 0; w < B; ++w) seeds[w] = 2.0 * (eloc[w] - emean[GEO(w)]) / cnt[GEO(w)];
  int rc = oracle_logpsi_vjp(t, P, R, Z, geo, B, x, seeds, grad);
  free(seeds); free(sum); free(cnt);
  return rc;
}

/* ------------------------------------------------------------------------ */
/* Training-loop pieces around the gradient (FermiNet practice; the paper    */
/* is silent on both): local-energy clipping and proposal-width adaptation   */
/* ------------------------------------------------------------------------ */

static int cmp_double(const void* a, const void* b) {
  double x = *(const double*)a, y = *(const double*)b;
  return (x > y) - (x < y);
}

/* Clipped gradient seeds.  For every geometry g (walkers W_g): the median m_g
 * of E_L over W_g (the mean of the two middle values when |W_g| is even),
 * the spread tv_g = mean over W_g of |E_L - m_g|, the clipped energies
 * c_w = min(max(E_L,w, m_g - scale tv_g), m_g + scale tv_g), their mean
 * cbar_g, and seeds[w] = 2 (c_w - cbar_g) / |W_g|.  stats (may be NULL)
 * receives {m_g, tv_g, cbar_g} per geometry. */
int oracle_clip_seeds(int n_geo, long B, const int* geo, const double* eloc, double scale, double* seeds,
                      double* stats) {
  if (n_geo < 1 || scale < 0) return -1;
  double* buf = malloc(sizeof(double) * (B > 0 ? B : 1));
  for (int g = 0; g < n_geo; ++g) {
    long c = 0;
    for (long w = 0; w < B; ++w)
      if ((geo ? geo[w] : 0) == g) buf[c++] = eloc[w];
    double m = 0.0, tv = 0.0, cbar = 0.0;
    if (c > 0) {
      qsort(buf, (size_t)c, sizeof(double), cmp_double);
      m = (c % 2) ? buf[c / 2] : 0.5 * (buf[c / 2 - 1] + buf[c / 2]);
      for (long i = 0; i < c; ++i) tv += fabs(buf[i] - m);
      tv /= (double)c;
      const double lo = m - scale * tv, hi = m + scale * tv;
      for (long w = 0; w < B; ++w)
        if ((geo ? geo[w] : 0) == g) cbar += fmin(fmax(eloc[w], lo), hi);
      cbar /= (double)c;
      for (long w = 0; w < B; ++w)
        if ((geo ? geo[w] : 0) == g) seeds[w] = 2.0 * (fmin(fmax(eloc[w], lo), hi) - cbar) / (double)c;
    }
    if (stats) { stats[3 * g] = m; stats[3 * g + 1] = tv; stats[3 * g + 2] = cbar; }
  }
  free(buf);
  return 0;
}

/* VMC energy gradient with clipped local energies: emean[g] is the plain
 * mean of E_L over geometry g (the energy estimate), and grad =
 * sum_w seeds[w] d log|psi_w| / d theta with the seeds of oracle_clip_seeds. */
int oracle_energy_grad_clipped(const onet* t, const double* P, const double* R, const double* Z, const int* geo,
                               int n_geo, long B, const double* x, const double* eloc, double scale, double* emean,
                               double* grad) {
  if (check_net(t) || n_geo < 1) return -1;
  double* sum = calloc(n_geo, sizeof(double));
  long* cnt = calloc(n_geo, sizeof(long));
  for (long w = 0; w < B; ++w) { sum[GEO(w)] += eloc[w]; cnt[GEO(w)]++; }
  for (int g = 0; g < n_geo; ++g) emean[g] = cnt[g] ? sum[g] / cnt[g] : 0.0;
  double* seeds = malloc(sizeof(double) * (B > 0 ? B : 1));
  int rc = oracle_clip_seeds(n_geo, B, geo, eloc, scale, seeds, NULL);
  if (!rc) rc = oracle_logpsi_vjp(t, P, R, Z, geo, B, x, seeds, grad);
  free(seeds); free(sum); free(cnt);
  return rc;
}

/* Proposal-width adaptation from the acceptance fraction of the last moves:
 * p = accepted / moves; the width grows by `factor` when p > hi, shrinks by
 * it when p < lo, and stays otherwise. */
double oracle_adapt_width(double width, double accepted, double moves, double lo, double hi, double factor) {
  if (moves <= 0) return width;
  const double p = accepted / moves;
  if (p > hi) return width * factor;
  if (p < lo) return width / factor;
  return width;
}

/* ------------------------------------------------------------------------ */
/* Philox4x32-10 and Metropolis                                              */
/* ------------------------------------------------------------------------ */

/* Philox4x32 with 10 rounds (Salmon, Moraes, Dror, Shaw, SC'11): each round
 * multiplies words 0 and 2 by the two round constants, splits the 64-bit
 * products into high and low halves and mixes in words 1 and 3 and the key;
 * the key is advanced by the two Weyl constants between rounds. */
void oracle_philox4x32_10(const uint32_t ctr_in[4], const uint32_t key_in[2], uint32_t out[4]) {
  uint32_t c0 = ctr_in[0], c1 = ctr_in[1], c2 = ctr_in[2], c3 = ctr_in[3];
  uint32_t k0 = key_in[0], k1 = key_in[1];
  for (int r = 0; r < 10; ++r) {
    if (r > 0) { k0 += 0x9E3779B9u; k1 += 0xBB67AE85u; }
    uint64_t p0 = (uint64_t)0xD2511F53u * c0;
    uint64_t p1 = (uint64_t)0xCD9E8D57u * c2;
    uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
    uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
    uint32_t n0 = hi1 ^ c1 ^ k0, n1 = lo1, n2 = hi0 ^ c3 ^ k1, n3 = lo0;
    c0 = n0; c1 = n1; c2 = n2; c3 = n3;
  }
  out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

/* uint32 -> uniform in (0,1): ((x >> 9) + 0.5) * 2^-23 (exact in float32). */
static double u01(uint32_t x) { return ((double)(x >> 9) + 0.5) * (1.0 / 8388608.0); }

/* Random numbers of one Metropolis move of walker w at step counter t:
 * normals z[0..3n) for the proposal and one uniform u for the acceptance.
 * Normals: block b = q/4 uses counter {w, b, t_lo, t_hi} and key
 * {seed_lo, seed_hi}; its words (0,1) and (2,3) each give two normals by
 * Box-Muller (r = sqrt(-2 ln u_a), angle 2 pi u_b; cos then sin).
 * Uniform: counter {w, 0xFFFFFFFF, t_lo, t_hi}, word 0. */
void oracle_mcmc_randoms(int n3, unsigned long long w, unsigned long long seed, unsigned long long tctr,
                         double* z, double* u) {
  uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
  for (int b = 0; b * 4 < n3; ++b) {
    uint32_t ctr[4] = {(uint32_t)w, (uint32_t)b, (uint32_t)tctr, (uint32_t)(tctr >> 32)}, o[4];
    oracle_philox4x32_10(ctr, key, o);
    for (int pr = 0; pr < 2; ++pr) {
      double ua = u01(o[2 * pr]), ub = u01(o[2 * pr + 1]);
      double r = sqrt(-2.0 * log(ua)), th = 2.0 * M_PI * ub;
      int q = 4 * b + 2 * pr;
      if (q < n3) z[q] = r * cos(th);
      if (q + 1 < n3) z[q + 1] = r * sin(th);
    }
  }
  uint32_t ctr[4] = {(uint32_t)w, 0xFFFFFFFFu, (uint32_t)tctr, (uint32_t)(tctr >> 32)}, o[4];
  oracle_philox4x32_10(ctr, key, o);
  *u = u01(o[0]);
}

/* n_steps Gaussian all-electron Metropolis moves targeting |psi|^2.  Step s
 * uses counter t = counter + s; walker index w is the batch index.  Proposal
 * x' = x + width * z; accept iff log u < 2 (log|psi(x')| - log|psi(x)|).
 * x and logpsi are updated in place; accepted[w] counts accepted moves;
 * margin[w] (may be NULL) receives min over steps of |2 dlogpsi - log u|. */
int oracle_mcmc(const onet* t, const double* P, const double* R, const double* Z, const int* geo,
                long B, double* x, double* logpsi, int n_steps, double width, unsigned long long seed,
                unsigned long long counter, int* accepted, double* margin) {
  (void)Z;
  if (check_net(t)) return -1;
  olayout Lo; build_layout(t, &Lo, NULL, 0);
  const int n = t->n_up + t->n_down, N = t->n_nuc;
#pragma omp parallel for schedule(dynamic, 1)
  for (long w = 0; w < B; ++w) {
    double* xw = x + (size_t)w * 3 * n;
    double* z = malloc(sizeof(double) * 3 * n);
    double* xp = malloc(sizeof(double) * 3 * n);
    int acc = 0;
    double mg = INFINITY;
    for (int s = 0; s < n_steps; ++s) {
      double u;
      oracle_mcmc_randoms(3 * n, (unsigned long long)w, seed, counter + (unsigned long long)s, z, &u);
      for (int q = 0; q < 3 * n; ++q) xp[q] = xw[q] + width * z[q];
      ofwd f;
      oracle_fwd(t, &Lo, P, R + (size_t)GEO(w) * 3 * N, xp, &f);
      double lp = f.logpsi;
      fwd_free(&f);
      double crit = 2.0 * (lp - logpsi[w]);
      double lu = log(u);
      if (fabs(crit - lu) < mg) mg = fabs(crit - lu);
      if (lu < crit) {
        memcpy(xw, xp, sizeof(double) * 3 * n);
        logpsi[w] = lp;
        acc++;
      }
    }
    if (accepted) accepted[w] = acc;
    if (margin) margin[w] = mg;
    free(z); free(xp);
  }
  return 0;
}

/* Single-walker access to the jet forward, for derivative pins. */
int oracle_logpsi_jet(const onet* t, const double* P, const double* R, const double* x, int seed_coord,
                      double* out3, double* sign) {
  if (check_net(t)) return -1;
  olayout Lo; build_layout(t, &Lo, NULL, 0);
  jet j = oracle_fwd_jet(t, &Lo, P, R, x, seed_coord, sign);
  out3[0] = j.v; out3[1] = j.d; out3[2] = j.dd;
  return 0;
}
