/*
 * lqcd_oracle.c -- plain, slow, FP64 CPU oracle for the twisted-mass Wilson
 * hot path of "Lattice QCD based on OpenCL" (Bach, Lindenstruth, Philipsen,
 * Pinke, arXiv:1209.5942).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product library links, loads or
 * calls this file.  Only the tests, the smoke check and the CPU-baseline leg
 * of the benchmark use it.  It shares no code, headers, tables or helpers with
 * the CUDA path.
 *
 * Everything is written straight from the definitions, in the order the
 * paper states them, with no blocking or fusion:
 *   - fields are lexicographic array-of-structures, complex double:
 *       site i = x + Lx*(y + Ly*(z + Lz*t))
 *       gauge  U[i][mu][a][b]     (mu = 0,1,2,3 = x,y,z,t)
 *       spinor psi[i][spin][colour]
 *       algebra fields (momenta, forces) P[mu][i][8], P = sum_a p^a lambda^a/2
 *   - gamma matrices are built as dense 4x4 complex matrices from the Pauli
 *     matrices (chiral basis) and applied as dense matrix products.
 *
 * Sections of the paper followed:
 *   Sec. 2.1, eq. "D_tm"          : twisted-mass Wilson matrix, hopping term
 *   Sec. 2.1, eq. "S_tlsym"       : Wilson plaquette action (c1 = 0) and the
 *                                   tree-level Symanzik action with 2x1 loops
 *   Sec. 2.1, eq. "solvereq"      : D phi = psi solved by CG
 *   Sec. 2.2, Sec. 5.3            : HMC (Hamiltonian, leapfrog, the 2MN scheme
 *                                   on separate gauge and fermion time scales,
 *                                   Metropolis),
 *                                   fermion force through dD^-1 = -D^-1 dD D^-1,
 *                                   Cabibbo-Marinari heatbath with the exact
 *                                   SU(2) update (Fig. "heatbath algorithm")
 *   Sec. 4.1                      : REC12 third-row reconstruction
 * Readings where the paper is silent or garbled are listed in the design
 * notes; the ones that matter here are repeated next to the code.
 *
 * Parity status: every function here is pinned by a test against a closed
 * form, an invariant, brute force or a library routine (see tests/).
 */
#include <complex.h>
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

typedef double complex cplx;

/* ------------------------------------------------------------------ */
/* Geometry (Sec. 2.1: V = Ns^3 x Nt; directions x,y,z,t)              */
/* ------------------------------------------------------------------ */

static long volume(const int *L) { return (long)L[0] * L[1] * L[2] * L[3]; }

static void coords(long i, const int *L, int c[4]) {
  c[0] = (int)(i % L[0]); i /= L[0];
  c[1] = (int)(i % L[1]); i /= L[1];
  c[2] = (int)(i % L[2]); i /= L[2];
  c[3] = (int)i;
}

static long index_of(const int c[4], const int *L) {
  return c[0] + (long)L[0] * (c[1] + (long)L[1] * (c[2] + (long)L[2] * c[3]));
}

/* neighbour x + s*mu_hat, periodic */
static long neighbour(long i, int mu, int s, const int *L) {
  int c[4];
  coords(i, L, c);
  c[mu] = (c[mu] + s + L[mu]) % L[mu];
  return index_of(c, L);
}

int or_parity(long i, const int *L) {
  int c[4];
  coords(i, L, c);
  return (c[0] + c[1] + c[2] + c[3]) & 1;
}

/* Fermion boundary factor of the hop from x to x + s*mu_hat: -1 when the hop
 * crosses the time boundary and the fermions are antiperiodic in time. */
static double bc_factor(long i, int mu, int s, const int *L, int antiperiodic_t) {
  if (mu != 3 || !antiperiodic_t) return 1.0;
  int c[4];
  coords(i, L, c);
  if (s > 0 && c[3] == L[3] - 1) return -1.0;
  if (s < 0 && c[3] == 0) return -1.0;
  return 1.0;
}

/* ------------------------------------------------------------------ */
/* Dirac algebra: chiral basis built from the Pauli matrices            */
/*   gamma_k = [[0, -i sigma_k], [i sigma_k, 0]]  (k = x, y, z)          */
/*   gamma_t = [[0, 1], [1, 0]]                                          */
/*   gamma_5 = gamma_x gamma_y gamma_z gamma_t                           */
/* ------------------------------------------------------------------ */

static void build_generators(void);
static cplx G[5][4][4]; /* G[0..3] = gamma_mu, G[4] = gamma_5 */
static int gamma_ready = 0;
/* The tables are filled on first use by the exported entry points, always
 * before any OpenMP parallel region starts. */

static void build_gammas(void) {
  if (gamma_ready) return;
  cplx sig[3][2][2] = {
      {{0, 1}, {1, 0}},
      {{0, -I}, {I, 0}},
      {{1, 0}, {0, -1}},
  };
  memset(G, 0, sizeof(G));
  for (int k = 0; k < 3; k++)
    for (int a = 0; a < 2; a++)
      for (int b = 0; b < 2; b++) {
        G[k][a][2 + b] = -I * sig[k][a][b];
        G[k][2 + a][b] = I * sig[k][a][b];
      }
  for (int a = 0; a < 2; a++) {
    G[3][a][2 + a] = 1;
    G[3][2 + a][a] = 1;
  }
  /* gamma_5 = product of the four */
  cplx t1[4][4], t2[4][4];
  for (int a = 0; a < 4; a++)
    for (int b = 0; b < 4; b++) {
      cplx s = 0;
      for (int c = 0; c < 4; c++) s += G[0][a][c] * G[1][c][b];
      t1[a][b] = s;
    }
  for (int a = 0; a < 4; a++)
    for (int b = 0; b < 4; b++) {
      cplx s = 0;
      for (int c = 0; c < 4; c++) s += t1[a][c] * G[2][c][b];
      t2[a][b] = s;
    }
  for (int a = 0; a < 4; a++)
    for (int b = 0; b < 4; b++) {
      cplx s = 0;
      for (int c = 0; c < 4; c++) s += t2[a][c] * G[3][c][b];
      G[4][a][b] = s;
    }
  gamma_ready = 1;
}

/* Export gamma_mu (mu = 0..3) or gamma_5 (mu = 4) as 16 complex numbers. */
void or_gamma(int mu, double *out) {
  build_gammas();
  for (int a = 0; a < 4; a++)
    for (int b = 0; b < 4; b++) {
      out[2 * (4 * a + b)] = creal(G[mu][a][b]);
      out[2 * (4 * a + b) + 1] = cimag(G[mu][a][b]);
    }
}

/* ------------------------------------------------------------------ */
/* Field access helpers                                                 */
/* ------------------------------------------------------------------ */

static const cplx *link_at(const double *U, long i, int mu) {
  return (const cplx *)(U + 2 * 9 * (4 * i + mu));
}
static cplx *link_mut(double *U, long i, int mu) { return (cplx *)(U + 2 * 9 * (4 * i + mu)); }
static const cplx *spinor_at(const double *psi, long i) { return (const cplx *)(psi + 2 * 12 * i); }
static cplx *spinor_mut(double *psi, long i) { return (cplx *)(psi + 2 * 12 * i); }

/* ------------------------------------------------------------------ */
/* Hopping term (Sec. 2.1, eq. "D_tm")                                 */
/*   H psi(x) = sum_mu  (1 - gamma_mu) U_mu(x)       psi(x + mu)         */
/*                    + (1 + gamma_mu) U_mu(x - mu)^+ psi(x - mu)        */
/* with the fermion boundary factor on hops across the time boundary.   */
/* Its adjoint (derived from the matrix elements) is the same sum with  */
/* gamma_mu -> -gamma_mu:                                               */
/*   H^+ psi(x) = sum_mu (1 + gamma_mu) U_mu(x) psi(x + mu)             */
/*                     + (1 - gamma_mu) U_mu(x - mu)^+ psi(x - mu)       */
/* Reading: the prefactor is kappa (not kappa/2), n == x, and the       */
/* forward hop carries (1 - gamma_mu) as printed.                       */
/* ------------------------------------------------------------------ */

static void hop_site(const double *U, const double *psi, cplx out[12], long i, const int *L,
                     int antiperiodic_t, int dagger) {
  for (int k = 0; k < 12; k++) out[k] = 0;
  for (int mu = 0; mu < 4; mu++) {
    for (int s = -1; s <= 1; s += 2) {
      long j = neighbour(i, mu, s, L);
      double bc = bc_factor(i, mu, s, L, antiperiodic_t);
      /* colour matrix: U_mu(x) forward, U_mu(x - mu)^+ backward */
      cplx Uc[3][3];
      if (s > 0) {
        const cplx *u = link_at(U, i, mu);
        for (int a = 0; a < 3; a++)
          for (int b = 0; b < 3; b++) Uc[a][b] = u[3 * a + b];
      } else {
        const cplx *u = link_at(U, j, mu);
        for (int a = 0; a < 3; a++)
          for (int b = 0; b < 3; b++) Uc[a][b] = conj(u[3 * b + a]);
      }
      /* spin matrix: (1 - s_eff gamma_mu) with s_eff = s (or -s for H^+) */
      double sg = dagger ? -(double)s : (double)s;
      cplx P[4][4];
      for (int a = 0; a < 4; a++)
        for (int b = 0; b < 4; b++) P[a][b] = (a == b ? 1.0 : 0.0) - sg * G[mu][a][b];
      const cplx *ps = spinor_at(psi, j);
      for (int a = 0; a < 4; a++)
        for (int c = 0; c < 3; c++) {
          cplx acc = 0;
          for (int b = 0; b < 4; b++)
            for (int d = 0; d < 3; d++) acc += P[a][b] * Uc[c][d] * ps[3 * b + d];
          out[3 * a + c] += bc * acc;
        }
    }
  }
}

void or_hop(const double *U, const double *psi, double *out, const int *L, int antiperiodic_t,
            int dagger) {
  build_gammas(); /* tables are filled here, never inside a parallel region */
  long V = volume(L);
#pragma omp parallel for schedule(static)
  for (long i = 0; i < V; i++) {
    cplx o[12];
    hop_site(U, psi, o, i, L, antiperiodic_t, dagger);
    cplx *dst = spinor_mut(out, i);
    for (int k = 0; k < 12; k++) dst[k] = o[k];
  }
}

/* ------------------------------------------------------------------ */
/* Twisted-mass matrix (Sec. 2.1, eq. "D_tm"), flavour "+":             */
/*   M = (1 + i a gamma_5) - kappa H,  a = 2 kappa mu                    */
/*   M^+ = (1 - i a gamma_5) - kappa H^+                                 */
/* ------------------------------------------------------------------ */

static void diag_site(const cplx in[12], cplx out[12], double a, double sign) {
  /* out = (1 + i sign a gamma_5) in */
  for (int s = 0; s < 4; s++)
    for (int c = 0; c < 3; c++) {
      cplx g5 = 0;
      for (int r = 0; r < 4; r++) g5 += G[4][s][r] * in[3 * r + c];
      out[3 * s + c] = in[3 * s + c] + I * sign * a * g5;
    }
}

void or_apply_M(const double *U, const double *psi, double *out, const int *L, int antiperiodic_t,
                double kappa, double mu, int dagger) {
  build_gammas();
  long V = volume(L);
  double a = 2.0 * kappa * mu;
#pragma omp parallel for schedule(static)
  for (long i = 0; i < V; i++) {
    cplx h[12], d[12];
    hop_site(U, psi, h, i, L, antiperiodic_t, dagger);
    diag_site(spinor_at(psi, i), d, a, dagger ? -1.0 : 1.0);
    cplx *dst = spinor_mut(out, i);
    for (int k = 0; k < 12; k++) dst[k] = d[k] - kappa * h[k];
  }
}

/* Site-diagonal factor A = 1 + i a gamma_5 and its inverse
 * A^-1 = (1 - i a gamma_5)/(1 + a^2) (gamma_5^2 = 1), applied on the sites
 * of one parity of a full-size field; other sites are left untouched.
 * mode 0: A, 1: A^-1, 2: A^+ = 1 - i a g5, 3: A^-+ = (1 + i a g5)/(1 + a^2) */
static void apply_diag_parity(double *f, const int *L, int parity, double a, int mode) {
  long V = volume(L);
  for (long i = 0; i < V; i++) {
    if (or_parity(i, L) != parity) continue;
    cplx in[12], out[12];
    cplx *p = spinor_mut(f, i);
    for (int k = 0; k < 12; k++) in[k] = p[k];
    double sign = (mode == 0 || mode == 3) ? 1.0 : -1.0;
    diag_site(in, out, a, sign);
    double norm = (mode == 1 || mode == 3) ? 1.0 / (1.0 + a * a) : 1.0;
    for (int k = 0; k < 12; k++) p[k] = norm * out[k];
  }
}

static void zero_parity(double *f, const int *L, int parity) {
  long V = volume(L);
  for (long i = 0; i < V; i++)
    if (or_parity(i, L) == parity) memset(spinor_mut(f, i), 0, 12 * sizeof(cplx));
}

/* ------------------------------------------------------------------ */
/* Even-odd preconditioning (Sec. 2.1, "even-odd-preconditioning").      */
/* The paper names the technique only; the Schur complement on the even  */
/* sites is used:                                                        */
/*   Mhat   = A_e - kappa^2 H_eo A_o^-1 H_oe                             */
/*   Mhat^+ = A_e^+ - kappa^2 H_eo^+ A_o^-+ H_oe^+                       */
/* Fields are full-size; only even sites of the input are read and only  */
/* even sites of the output are meaningful (odd sites are set to zero).  */
/* ------------------------------------------------------------------ */

void or_apply_Mhat(const double *U, const double *psi, double *out, const int *L,
                   int antiperiodic_t, double kappa, double mu, int dagger) {
  build_gammas();
  build_generators();
  long V = volume(L);
  size_t n = (size_t)V * 24;
  double a = 2.0 * kappa * mu;
  double *pe = malloc(n * sizeof(double));
  double *t = malloc(n * sizeof(double));
  double *h = malloc(n * sizeof(double));
  memcpy(pe, psi, n * sizeof(double));
  zero_parity(pe, L, 1);
  or_hop(U, pe, t, L, antiperiodic_t, dagger); /* H_oe psi_e on odd sites */
  zero_parity(t, L, 0);
  apply_diag_parity(t, L, 1, a, dagger ? 3 : 1); /* A_o^-1 (or A_o^-+) */
  or_hop(U, t, h, L, antiperiodic_t, dagger);    /* H_eo on even sites */
  memcpy(out, pe, n * sizeof(double));
  apply_diag_parity(out, L, 0, a, dagger ? 2 : 0); /* A_e psi_e */
  for (long i = 0; i < V; i++) {
    cplx *o = spinor_mut(out, i);
    const cplx *hh = spinor_at(h, i);
    if (or_parity(i, L) == 0)
      for (int k = 0; k < 12; k++) o[k] -= kappa * kappa * hh[k];
    else
      for (int k = 0; k < 12; k++) o[k] = 0;
  }
  free(pe);
  free(t);
  free(h);
}

/* Source preparation and reconstruction for M x = b through the even
 * Schur complement:
 *   bhat_e = b_e + kappa H_eo A_o^-1 b_o
 *   x_o    = A_o^-1 (b_o + kappa H_oe x_e)                               */
void or_eo_prepare(const double *U, const double *b, double *bhat, const int *L,
                   int antiperiodic_t, double kappa, double mu) {
  build_gammas();
  build_generators();
  long V = volume(L);
  size_t n = (size_t)V * 24;
  double a = 2.0 * kappa * mu;
  double *bo = malloc(n * sizeof(double));
  double *h = malloc(n * sizeof(double));
  memcpy(bo, b, n * sizeof(double));
  zero_parity(bo, L, 0);
  apply_diag_parity(bo, L, 1, a, 1);
  or_hop(U, bo, h, L, antiperiodic_t, 0);
  for (long i = 0; i < V; i++) {
    cplx *o = spinor_mut(bhat, i);
    const cplx *bb = spinor_at(b, i);
    const cplx *hh = spinor_at(h, i);
    if (or_parity(i, L) == 0)
      for (int k = 0; k < 12; k++) o[k] = bb[k] + kappa * hh[k];
    else
      for (int k = 0; k < 12; k++) o[k] = 0;
  }
  free(bo);
  free(h);
}

void or_eo_reconstruct(const double *U, const double *b, double *x, const int *L,
                       int antiperiodic_t, double kappa, double mu) {
  build_gammas();
  build_generators();
  long V = volume(L);
  size_t n = (size_t)V * 24;
  double a = 2.0 * kappa * mu;
  double *xe = malloc(n * sizeof(double));
  double *h = malloc(n * sizeof(double));
  memcpy(xe, x, n * sizeof(double));
  zero_parity(xe, L, 1);
  or_hop(U, xe, h, L, antiperiodic_t, 0);
  for (long i = 0; i < V; i++) {
    if (or_parity(i, L) != 1) continue;
    cplx *o = spinor_mut(x, i);
    const cplx *bb = spinor_at(b, i);
    const cplx *hh = spinor_at(h, i);
    for (int k = 0; k < 12; k++) o[k] = bb[k] + kappa * hh[k];
  }
  apply_diag_parity(x, L, 1, a, 1);
  free(xe);
  free(h);
}

/* ------------------------------------------------------------------ */
/* Linear algebra on full-size spinor fields                            */
/* ------------------------------------------------------------------ */

static double norm2(const double *f, size_t n) {
  double s = 0;
  for (size_t k = 0; k < n; k++) s += f[k] * f[k];
  return s;
}
static double dot_re(const double *f, const double *g, size_t n) {
  double s = 0;
  for (size_t k = 0; k < n; k++) s += f[k] * g[k];
  return s;
}

/* Plain conjugate gradient (Sec. 2.1, eq. "solvereq": "the most common
 * solvers used are CG ...") on the normal equations.
 *   eo = 0: M^+ M x = M^+ b on the full lattice (unpreconditioned)
 *   eo = 1: Mhat^+ Mhat x = rhs on the even sites (rhs given directly)
 * Stops when ||b - M x|| / ||b|| <= tol (eo = 0) or when the normal-equation
 * residual satisfies ||rhs - Mhat^+ Mhat x|| / ||rhs|| <= tol (eo = 1).
 * Returns the iteration count, or -1 when max_iter is reached.            */
int or_cg(const double *U, const double *b, double *x, const int *L, int antiperiodic_t,
          double kappa, double mu, double tol, int max_iter, int eo, double *resid_out) {
  build_gammas();
  build_generators();
  long V = volume(L);
  size_t n = (size_t)V * 24;
  double *r = malloc(n * sizeof(double));
  double *p = malloc(n * sizeof(double));
  double *q = malloc(n * sizeof(double));
  double *t = malloc(n * sizeof(double));
  double *rhs = malloc(n * sizeof(double));
  if (eo) {
    memcpy(rhs, b, n * sizeof(double));
    zero_parity(rhs, L, 1);
  } else {
    or_apply_M(U, b, rhs, L, antiperiodic_t, kappa, mu, 1);
  }
  /* x = 0 start */
  memset(x, 0, n * sizeof(double));
  memcpy(r, rhs, n * sizeof(double));
  memcpy(p, r, n * sizeof(double));
  double rr = norm2(r, n);
  double bnorm = eo ? sqrt(norm2(rhs, n)) : sqrt(norm2(b, n));
  int it = 0, done = 0;
  double res = 1.0;
  for (it = 0; it < max_iter; it++) {
    if (eo) {
      or_apply_Mhat(U, p, t, L, antiperiodic_t, kappa, mu, 0);
      or_apply_Mhat(U, t, q, L, antiperiodic_t, kappa, mu, 1);
    } else {
      or_apply_M(U, p, t, L, antiperiodic_t, kappa, mu, 0);
      or_apply_M(U, t, q, L, antiperiodic_t, kappa, mu, 1);
    }
    double alpha = rr / dot_re(p, q, n);
    for (size_t k = 0; k < n; k++) {
      x[k] += alpha * p[k];
      r[k] -= alpha * q[k];
    }
    double rr_new = norm2(r, n);
    if (eo) {
      res = sqrt(rr_new) / bnorm;
    } else {
      /* true residual of the unsquared system */
      or_apply_M(U, x, t, L, antiperiodic_t, kappa, mu, 0);
      double s = 0;
      for (size_t k = 0; k < n; k++) s += (b[k] - t[k]) * (b[k] - t[k]);
      res = sqrt(s) / bnorm;
    }
    if (res <= tol) {
      done = 1;
      it++;
      break;
    }
    double beta = rr_new / rr;
    rr = rr_new;
    for (size_t k = 0; k < n; k++) p[k] = r[k] + beta * p[k];
  }
  if (resid_out) *resid_out = res;
  free(r);
  free(p);
  free(q);
  free(t);
  free(rhs);
  return done ? it : -1;
}

/* Fixed number of CG iterations on the normal equations of the even
 * Schur complement, each iteration being two Mhat and two Mhat^+ products
 * (the same work per iteration as the solver of the product path); used
 * only to time the oracle on a bounded sample of a large workload.      */
double or_cg_fixed_iters(const double *U, const double *bhat, double *x, const int *L,
                         int antiperiodic_t, double kappa, double mu, int iters) {
  build_gammas();
  build_generators();
  long V = volume(L);
  size_t n = (size_t)V * 24;
  double *rhs = malloc(n * sizeof(double));
  double *r = malloc(n * sizeof(double));
  double *p = malloc(n * sizeof(double));
  double *q = malloc(n * sizeof(double));
  double *t = malloc(n * sizeof(double));
  or_apply_Mhat(U, bhat, rhs, L, antiperiodic_t, kappa, mu, 1); /* Mhat^+ bhat */
  memset(x, 0, n * sizeof(double));
  memcpy(r, rhs, n * sizeof(double));
  memcpy(p, r, n * sizeof(double));
  double rr = norm2(r, n);
  for (int it = 0; it < iters; it++) {
    or_apply_Mhat(U, p, t, L, antiperiodic_t, kappa, mu, 0);
    or_apply_Mhat(U, t, q, L, antiperiodic_t, kappa, mu, 1);
    double alpha = rr / dot_re(p, q, n);
    for (size_t k = 0; k < n; k++) {
      x[k] += alpha * p[k];
      r[k] -= alpha * q[k];
    }
    double rr_new = norm2(r, n);
    double beta = rr_new / rr;
    rr = rr_new;
    for (size_t k = 0; k < n; k++) p[k] = r[k] + beta * p[k];
  }
  double res = sqrt(rr / norm2(rhs, n));
  free(rhs);
  free(r);
  free(p);
  free(q);
  free(t);
  return res;
}

/* ------------------------------------------------------------------ */
/* SU(3) helpers                                                        */
/* ------------------------------------------------------------------ */

static void mat_mul(const cplx *A, const cplx *B, cplx *C) { /* C = A B */
  cplx T[9];
  for (int a = 0; a < 3; a++)
    for (int b = 0; b < 3; b++) {
      cplx s = 0;
      for (int c = 0; c < 3; c++) s += A[3 * a + c] * B[3 * c + b];
      T[3 * a + b] = s;
    }
  memcpy(C, T, sizeof(T));
}
static void mat_dag(const cplx *A, cplx *B) {
  cplx T[9];
  for (int a = 0; a < 3; a++)
    for (int b = 0; b < 3; b++) T[3 * a + b] = conj(A[3 * b + a]);
  memcpy(B, T, sizeof(T));
}
static cplx mat_trace(const cplx *A) { return A[0] + A[4] + A[8]; }

/* Gell-Mann matrices lambda^a (a = 1..8) as T^a = lambda^a / 2. */
static cplx Tgen[8][9];
static int gen_ready = 0;
static void build_generators(void) {
  if (gen_ready) return;
  memset(Tgen, 0, sizeof(Tgen));
  /* lambda_1 */ Tgen[0][1] = 1; Tgen[0][3] = 1;
  /* lambda_2 */ Tgen[1][1] = -I; Tgen[1][3] = I;
  /* lambda_3 */ Tgen[2][0] = 1; Tgen[2][4] = -1;
  /* lambda_4 */ Tgen[3][2] = 1; Tgen[3][6] = 1;
  /* lambda_5 */ Tgen[4][2] = -I; Tgen[4][6] = I;
  /* lambda_6 */ Tgen[5][5] = 1; Tgen[5][7] = 1;
  /* lambda_7 */ Tgen[6][5] = -I; Tgen[6][7] = I;
  /* lambda_8 */ Tgen[7][0] = 1 / sqrt(3.0); Tgen[7][4] = 1 / sqrt(3.0); Tgen[7][8] = -2 / sqrt(3.0);
  for (int a = 0; a < 8; a++)
    for (int k = 0; k < 9; k++) Tgen[a][k] *= 0.5;
  gen_ready = 1;
}

void or_generator(int a, double *out) {
  build_generators();
  for (int k = 0; k < 9; k++) {
    out[2 * k] = creal(Tgen[a][k]);
    out[2 * k + 1] = cimag(Tgen[a][k]);
  }
}

/* ------------------------------------------------------------------ */
/* Plaquette and Wilson gauge action (Sec. 2.1, eq. "S_tlsym", c1 = 0)   */
/*   U_munu(x) = U_mu(x) U_nu(x+mu) U_mu(x+nu)^+ U_nu(x)^+               */
/*   plaquette  = (1/(6V)) sum_{x, mu<nu} (1/3) Re Tr U_munu(x)           */
/*   S_g        = (beta/3) sum_{x, mu<nu} (3 - Re Tr U_munu(x))           */
/* (S_g differs from the printed normalisation by a constant only.)     */
/* ------------------------------------------------------------------ */

static double re_tr_plaq(const double *U, long i, int mu, int nu, const int *L) {
  cplx A[9], B[9];
  long ipm = neighbour(i, mu, 1, L), ipn = neighbour(i, nu, 1, L);
  mat_mul(link_at(U, i, mu), link_at(U, ipm, nu), A);
  mat_dag(link_at(U, ipn, mu), B);
  mat_mul(A, B, A);
  mat_dag(link_at(U, i, nu), B);
  mat_mul(A, B, A);
  return creal(mat_trace(A));
}

double or_plaquette(const double *U, const int *L) {
  long V = volume(L);
  double s = 0;
#pragma omp parallel for reduction(+ : s) schedule(static)
  for (long i = 0; i < V; i++)
    for (int mu = 0; mu < 4; mu++)
      for (int nu = mu + 1; nu < 4; nu++) s += re_tr_plaq(U, i, mu, nu, L);
  return s / (3.0 * 6.0 * (double)V);
}

double or_gauge_action(const double *U, const int *L, double beta) {
  long V = volume(L);
  double s = 0;
#pragma omp parallel for reduction(+ : s) schedule(static)
  for (long i = 0; i < V; i++)
    for (int mu = 0; mu < 4; mu++)
      for (int nu = mu + 1; nu < 4; nu++) s += 3.0 - re_tr_plaq(U, i, mu, nu, L);
  return beta / 3.0 * s;
}

/* Staple sum A_mu(x) (Sec. 2.2: the plaquette product without U_mu(x)),
 * defined so that the plaquettes containing U_mu(x) sum to Re Tr(U_mu(x) A):
 *   A = sum_{nu != mu} U_nu(x+mu) U_mu(x+nu)^+ U_nu(x)^+
 *                    + U_nu(x+mu-nu)^+ U_mu(x-nu)^+ U_nu(x-nu)           */
void or_staple(const double *U, const int *L, long i, int mu, double *out) {
  cplx S[9] = {0}, A[9], B[9];
  long ipm = neighbour(i, mu, 1, L);
  for (int nu = 0; nu < 4; nu++) {
    if (nu == mu) continue;
    long ipn = neighbour(i, nu, 1, L), imn = neighbour(i, nu, -1, L);
    long ipm_mn = neighbour(ipm, nu, -1, L);
    /* upper */
    mat_dag(link_at(U, ipn, mu), B);
    mat_mul(link_at(U, ipm, nu), B, A);
    mat_dag(link_at(U, i, nu), B);
    mat_mul(A, B, A);
    for (int k = 0; k < 9; k++) S[k] += A[k];
    /* lower */
    mat_dag(link_at(U, ipm_mn, nu), A);
    mat_dag(link_at(U, imn, mu), B);
    mat_mul(A, B, A);
    mat_mul(A, link_at(U, imn, nu), A);
    for (int k = 0; k < 9; k++) S[k] += A[k];
  }
  memcpy(out, S, sizeof(S));
}

/* dS_g/domega^a_mu(x) for U_mu(x) -> exp(i omega^a T^a) U_mu(x):
 *   dS_g/domega^a = -(beta/3) Re Tr[i T^a U_mu(x) A_mu(x)]
 * Output layout [mu][V][8].  The molecular-dynamics force is its negative. */
void or_gauge_dSdw(const double *U, const int *L, double beta, double *out) {
  build_generators();
  build_gammas();
  long V = volume(L);
#pragma omp parallel for schedule(static)
  for (long i = 0; i < V; i++)
    for (int mu = 0; mu < 4; mu++) {
      cplx A[9], W[9], TW[9];
      or_staple(U, L, i, mu, (double *)A);
      mat_mul(link_at(U, i, mu), A, W);
      for (int a = 0; a < 8; a++) {
        mat_mul(Tgen[a], W, TW);
        out[((long)mu * V + i) * 8 + a] = -(beta / 3.0) * creal(I * mat_trace(TW));
      }
    }
}

/* ------------------------------------------------------------------ */
/* Tree-level Symanzik gauge action (Sec. 2.1, eq. "S_tlsym"):            */
/*   S = (beta/3) sum_x [ c0 sum_{mu<nu} (3 - Re Tr P_munu(x))             */
/*                       + c1 sum_{mu != nu} (3 - Re Tr R_munu(x)) ]        */
/* with c0 = 1 - 8 c1 and R_munu(x) the 2x1 loop that runs two links along  */
/* mu, one along nu, two back along mu and one back along nu.  The paper's  */
/* printed c1 = 1/12 is read as the tree-level value c1 = -1/12; c1 is an   */
/* argument here, and c1 = 0 gives the Wilson action above.                 */
/*                                                                          */
/* A loop is a list of steps (direction, sign); a step +d from site s uses  */
/* U_d(s), a step -d uses U_d(s - d)^+.  The derivative is assembled loop by */
/* loop, straight from the definition: U_mu(x) -> exp(i w T^a) U_mu(x)       */
/* changes Re Tr(loop) = Re Tr(U_mu(x) W) at rate -Im Tr(T^a U_mu(x) W),      */
/* where W is the product of the loop's other links in loop order (taken    */
/* daggered when the loop runs through U_mu(x) backwards).                  */
/* ------------------------------------------------------------------ */

typedef struct {
  int dir, sgn;
} step_t;

/* the matrix of step st taken from site s (into M); returns the next site */
static long loop_step(const double *U, long s, step_t st, const int *L, cplx *M) {
  if (st.sgn > 0) {
    memcpy(M, link_at(U, s, st.dir), 9 * sizeof(cplx));
    return neighbour(s, st.dir, 1, L);
  }
  long b = neighbour(s, st.dir, -1, L);
  mat_dag(link_at(U, b, st.dir), M);
  return b;
}

/* site reached from y after the first k steps */
static long loop_walk(long y, const step_t *st, int k, const int *L) {
  for (int j = 0; j < k; j++) y = neighbour(y, st[j].dir, st[j].sgn, L);
  return y;
}

/* product of `count` consecutive steps of the closed loop (y, st[0..n)),
 * starting with step k0 (indices taken cyclically) */
static void loop_product(const double *U, long y, const step_t *st, int n, int k0, int count,
                         const int *L, cplx *out) {
  cplx M[9];
  long s = loop_walk(y, st, k0, L);
  for (int k = 0; k < 9; k++) out[k] = (k % 4 == 0) ? 1.0 : 0.0;
  for (int j = 0; j < count; j++) {
    s = loop_step(U, s, st[(k0 + j) % n], L, M);
    mat_mul(out, M, out);
  }
}

static void plaquette_steps(int mu, int nu, step_t st[4]) {
  st[0] = (step_t){mu, 1}; st[1] = (step_t){nu, 1}; st[2] = (step_t){mu, -1}; st[3] = (step_t){nu, -1};
}
static void rectangle_steps(int mu, int nu, step_t st[6]) {
  st[0] = (step_t){mu, 1}; st[1] = (step_t){mu, 1}; st[2] = (step_t){nu, 1};
  st[3] = (step_t){mu, -1}; st[4] = (step_t){mu, -1}; st[5] = (step_t){nu, -1};
}

static double re_tr_loop(const double *U, long y, const step_t *st, int n, const int *L) {
  cplx P[9];
  loop_product(U, y, st, n, 0, n, L, P);
  return creal(mat_trace(P));
}

/* sum_{x, mu != nu} (3 - Re Tr R_munu(x)) */
double or_rectangle_sum(const double *U, const int *L) {
  long V = volume(L);
  double s = 0;
#pragma omp parallel for reduction(+ : s) schedule(static)
  for (long i = 0; i < V; i++)
    for (int mu = 0; mu < 4; mu++)
      for (int nu = 0; nu < 4; nu++) {
        if (nu == mu) continue;
        step_t st[6];
        rectangle_steps(mu, nu, st);
        s += 3.0 - re_tr_loop(U, i, st, 6, L);
      }
  return s;
}

double or_gauge_action_sym(const double *U, const int *L, double beta, double c1) {
  long V = volume(L);
  double sp = 0;
#pragma omp parallel for reduction(+ : sp) schedule(static)
  for (long i = 0; i < V; i++)
    for (int mu = 0; mu < 4; mu++)
      for (int nu = mu + 1; nu < 4; nu++) {
        step_t st[4];
        plaquette_steps(mu, nu, st);
        sp += 3.0 - re_tr_loop(U, i, st, 4, L);
      }
  double sr = c1 != 0.0 ? or_rectangle_sum(U, L) : 0.0;
  return beta / 3.0 * ((1.0 - 8.0 * c1) * sp + c1 * sr);
}

/* W_mu(x) += coef * (other links of loop (y, st)) for every position of the
 * loop at which it runs through a link; accumulated serially into W[V][4][9] */
static void add_loop_staples(const double *U, long y, const step_t *st, int n, double coef, const int *L,
                             cplx *W) {
  long s = y;
  for (int k = 0; k < n; k++) {
    long x;
    int back = st[k].sgn < 0;
    if (!back) x = s;                                  /* runs through U_d(s) forwards   */
    else x = neighbour(s, st[k].dir, -1, L);           /* runs through U_d(s - d) back   */
    cplx R[9], Rd[9];
    loop_product(U, y, st, n, (k + 1) % n, n - 1, L, R);
    cplx *w = W + ((size_t)x * 4 + st[k].dir) * 9;
    if (back) {
      mat_dag(R, Rd);
      for (int q = 0; q < 9; q++) w[q] += coef * Rd[q];
    } else {
      for (int q = 0; q < 9; q++) w[q] += coef * R[q];
    }
    s = neighbour(s, st[k].dir, st[k].sgn, L);
  }
}

/* dS/domega^a_mu(x) of the tlSym action, [mu][V][8]:
 *   dS/domega^a = -(beta/3) Re Tr[i T^a U_mu(x) W_mu(x)],
 *   W = c0 (plaquette staples) + c1 (rectangle staples).                   */
void or_gauge_dSdw_sym(const double *U, const int *L, double beta, double c1, double *out) {
  build_generators();
  build_gammas();
  long V = volume(L);
  cplx *W = calloc((size_t)V * 4 * 9, sizeof(cplx));
  for (long y = 0; y < V; y++)
    for (int mu = 0; mu < 4; mu++)
      for (int nu = 0; nu < 4; nu++) {
        if (nu == mu) continue;
        if (nu > mu) {
          step_t sp[4];
          plaquette_steps(mu, nu, sp);
          add_loop_staples(U, y, sp, 4, 1.0 - 8.0 * c1, L, W);
        }
        if (c1 != 0.0) {
          step_t sr[6];
          rectangle_steps(mu, nu, sr);
          add_loop_staples(U, y, sr, 6, c1, L, W);
        }
      }
#pragma omp parallel for schedule(static)
  for (long i = 0; i < V; i++)
    for (int mu = 0; mu < 4; mu++) {
      cplx UW[9], TW[9];
      mat_mul(link_at(U, i, mu), W + ((size_t)i * 4 + mu) * 9, UW);
      for (int a = 0; a < 8; a++) {
        mat_mul(Tgen[a], UW, TW);
        out[((long)mu * V + i) * 8 + a] = -(beta / 3.0) * creal(I * mat_trace(TW));
      }
    }
  free(W);
}

/* ------------------------------------------------------------------ */
/* Fermion force (Sec. 2.2: dD^-1 = -D^-1 (dD) D^-1; only the hopping     */
/* term depends on U).  For S_pf = phi^+ (Mhat^+ Mhat)^-1 phi on the even */
/* sites, with X = (Mhat^+ Mhat)^-1 phi and Y = Mhat X,                   */
/*   dS = -2 Re[Y^+ dMhat X],                                             */
/*   dMhat = -kappa^2 (dH_eo A_o^-1 H_oe + H_eo A_o^-1 dH_oe),            */
/* so dS = 2 kappa^2 Re[Lf^+ dH Rf] with the full-lattice fields         */
/*   Lf = (Y_e, W_o),  W_o = A_o^-+ H_eo^+ Y_e                            */
/*   Rf = (X_e, Z_o),  Z_o = A_o^-1 H_oe X_e.                             */
/* For one link U_mu(x) -> exp(i w^a T^a) U_mu(x):                        */
/*   d/dw^a Re[Lf^+ dH Rf] = Re Tr[i T^a (C1 - C2)] * bc                  */
/*   C1 = sum_spin (U_mu(x) Rf(x+mu)) (x) ((1 - g_mu) Lf(x))^+            */
/*   C2 = sum_spin Rf(x) (x) (U_mu(x) (1 + g_mu) Lf(x+mu))^+              */
/* eo = 0 gives the unpreconditioned S = phi^+ (M^+ M)^-1 phi instead:     */
/*   dS = 2 kappa Re[Y^+ dH X],  Lf = Y = M X,  Rf = X.                    */
/* X must be supplied (already solved); output layout [mu][V][8].         */
/* ------------------------------------------------------------------ */

/* -2 Re[Y^+ dMhat X] / domega for given left and right vectors Y, X on the
 * even sites (eo = 1; Y = Mhat X gives the force of phi^+ (Mhat^+ Mhat)^-1
 * phi), or -2 Re[Y^+ dM X] on the full lattice (eo = 0).  Y = NULL: Y =
 * Mhat X (or M X). */
void or_fermion_dSdw_lr(const double *U, const double *Yin, const double *X, const int *L,
                        int antiperiodic_t, double kappa, double mu_tm, int eo, double *out) {
  build_gammas();
  build_generators();
  long V = volume(L);
  size_t n = (size_t)V * 24;
  double a = 2.0 * kappa * mu_tm;
  double *Lf = calloc(n, sizeof(double));
  double *Rf = calloc(n, sizeof(double));
  double pref;
  if (eo) {
    double *Y = malloc(n * sizeof(double));
    double *t = malloc(n * sizeof(double));
    if (Yin) {
      memcpy(Y, Yin, n * sizeof(double));
      zero_parity(Y, L, 1);
    } else {
      or_apply_Mhat(U, X, Y, L, antiperiodic_t, kappa, mu_tm, 0); /* Y_e (odd zero) */
    }
    /* W_o = A_o^-+ H^+ Y_e restricted to odd */
    or_hop(U, Y, t, L, antiperiodic_t, 1);
    zero_parity(t, L, 0);
    apply_diag_parity(t, L, 1, a, 3);
    for (size_t k = 0; k < n; k++) Lf[k] = Y[k] + t[k];
    /* Z_o = A_o^-1 H X_e restricted to odd */
    double *xe = malloc(n * sizeof(double));
    memcpy(xe, X, n * sizeof(double));
    zero_parity(xe, L, 1);
    or_hop(U, xe, t, L, antiperiodic_t, 0);
    zero_parity(t, L, 0);
    apply_diag_parity(t, L, 1, a, 1);
    for (size_t k = 0; k < n; k++) Rf[k] = xe[k] + t[k];
    pref = 2.0 * kappa * kappa;
    free(Y);
    free(t);
    free(xe);
  } else {
    if (Yin) memcpy(Lf, Yin, n * sizeof(double));
    else or_apply_M(U, X, Lf, L, antiperiodic_t, kappa, mu_tm, 0);
    memcpy(Rf, X, n * sizeof(double));
    pref = 2.0 * kappa;
  }
#pragma omp parallel for schedule(static)
  for (long i = 0; i < V; i++)
    for (int mu = 0; mu < 4; mu++) {
      long j = neighbour(i, mu, 1, L);
      double bc = bc_factor(i, mu, 1, L, antiperiodic_t);
      const cplx *u = link_at(U, i, mu);
      const cplx *Rj = spinor_at(Rf, j), *Ri = spinor_at(Rf, i);
      const cplx *Li = spinor_at(Lf, i), *Lj = spinor_at(Lf, j);
      cplx PL[12], QL[12], URj[12], UQ[12];
      /* PL = (1 - g_mu) Lf(x), QL = (1 + g_mu) Lf(x + mu) */
      for (int s = 0; s < 4; s++)
        for (int c = 0; c < 3; c++) {
          cplx s1 = 0, s2 = 0;
          for (int r = 0; r < 4; r++) {
            cplx m1 = (s == r ? 1.0 : 0.0) - G[mu][s][r];
            cplx m2 = (s == r ? 1.0 : 0.0) + G[mu][s][r];
            s1 += m1 * Li[3 * r + c];
            s2 += m2 * Lj[3 * r + c];
          }
          PL[3 * s + c] = s1;
          QL[3 * s + c] = s2;
        }
      for (int s = 0; s < 4; s++)
        for (int c = 0; c < 3; c++) {
          cplx s1 = 0, s2 = 0;
          for (int d = 0; d < 3; d++) {
            s1 += u[3 * c + d] * Rj[3 * s + d];
            s2 += u[3 * c + d] * QL[3 * s + d];
          }
          URj[3 * s + c] = s1;
          UQ[3 * s + c] = s2;
        }
      cplx C[9];
      for (int c = 0; c < 3; c++)
        for (int d = 0; d < 3; d++) {
          cplx s1 = 0;
          for (int s = 0; s < 4; s++)
            s1 += URj[3 * s + c] * conj(PL[3 * s + d]) - Ri[3 * s + c] * conj(UQ[3 * s + d]);
          C[3 * c + d] = s1;
        }
      for (int aa = 0; aa < 8; aa++) {
        cplx TC[9];
        mat_mul(Tgen[aa], C, TC);
        out[((long)mu * V + i) * 8 + aa] = pref * bc * creal(I * mat_trace(TC));
      }
    }
  free(Lf);
  free(Rf);
}

void or_fermion_dSdw(const double *U, const double *X, const int *L, int antiperiodic_t,
                     double kappa, double mu_tm, int eo, double *out) {
  or_fermion_dSdw_lr(U, NULL, X, L, antiperiodic_t, kappa, mu_tm, eo, out);
}

/* Pseudofermion action S_pf = phi^+ (Mhat^+ Mhat)^-1 phi = phi^+ X (eo = 1)
 * or phi^+ (M^+ M)^-1 phi (eo = 0), by plain CG to tolerance tol.  X is
 * returned. (Sec. 2, eq. "pseudo fermions", read for two flavours as
 * det(D+ D-) = det(M^+ M).)                                               */
double or_pseudofermion_action(const double *U, const double *phi, double *X, const int *L,
                               int antiperiodic_t, double kappa, double mu, int eo, double tol,
                               int max_iter) {
  build_gammas();
  build_generators();
  long V = volume(L);
  size_t n = (size_t)V * 24;
  double resid;
  if (eo) {
    or_cg(U, phi, X, L, antiperiodic_t, kappa, mu, tol, max_iter, 1, &resid);
  } else {
    /* X = (M^+ M)^-1 phi: CG on M^+ M with right-hand side phi directly */
    double *r = malloc(n * sizeof(double)), *p = malloc(n * sizeof(double));
    double *q = malloc(n * sizeof(double)), *t = malloc(n * sizeof(double));
    memset(X, 0, n * sizeof(double));
    memcpy(r, phi, n * sizeof(double));
    memcpy(p, r, n * sizeof(double));
    double rr = norm2(r, n), b2 = rr;
    for (int it = 0; it < max_iter && rr > tol * tol * b2; it++) {
      or_apply_M(U, p, t, L, antiperiodic_t, kappa, mu, 0);
      or_apply_M(U, t, q, L, antiperiodic_t, kappa, mu, 1);
      double alpha = rr / dot_re(p, q, n);
      for (size_t k = 0; k < n; k++) {
        X[k] += alpha * p[k];
        r[k] -= alpha * q[k];
      }
      double rn = norm2(r, n);
      double beta = rn / rr;
      rr = rn;
      for (size_t k = 0; k < n; k++) p[k] = r[k] + beta * p[k];
    }
    free(r);
    free(p);
    free(q);
    free(t);
  }
  double s = 0;
  for (size_t k = 0; k < n; k++) s += phi[k] * X[k];
  return s;
}

/* ------------------------------------------------------------------ */
/* Link compression REC12 (Sec. 4.1): keep rows 0 and 1; the third row    */
/* follows from unitarity and det = 1 as the complex conjugate of the     */
/* cross product of the first two (the printed "c = a x b" reads with     */
/* the conjugate).                                                        */
/* ------------------------------------------------------------------ */

void or_rec12_third_row(const double *link, double *row3) {
  const cplx *u = (const cplx *)link;
  cplx *r = (cplx *)row3;
  r[0] = conj(u[1] * u[5] - u[2] * u[4]);
  r[1] = conj(u[2] * u[3] - u[0] * u[5]);
  r[2] = conj(u[0] * u[4] - u[1] * u[3]);
}

/* Reunitarisation: Gram-Schmidt on rows 0 and 1, row 2 from REC12. */
void or_reunitarize(double *U, long nlinks) {
#pragma omp parallel for schedule(static)
  for (long l = 0; l < nlinks; l++) {
    cplx *u = (cplx *)(U + 18 * l);
    double n0 = 0;
    for (int k = 0; k < 3; k++) n0 += creal(u[k] * conj(u[k]));
    n0 = 1.0 / sqrt(n0);
    for (int k = 0; k < 3; k++) u[k] *= n0;
    cplx d = 0;
    for (int k = 0; k < 3; k++) d += conj(u[k]) * u[3 + k];
    for (int k = 0; k < 3; k++) u[3 + k] -= d * u[k];
    double n1 = 0;
    for (int k = 0; k < 3; k++) n1 += creal(u[3 + k] * conj(u[3 + k]));
    n1 = 1.0 / sqrt(n1);
    for (int k = 0; k < 3; k++) u[3 + k] *= n1;
    or_rec12_third_row((double *)u, (double *)(u + 6));
  }
}

/* ------------------------------------------------------------------ */
/* Matrix exponential exp(i eps P) for P = sum_a p^a T^a (Hermitian,       */
/* traceless), by scaling and squaring of the Taylor series.  Plain and    */
/* slow; the truncation order is chosen so the remainder is below 1e-17.  */
/* ------------------------------------------------------------------ */

void or_expi(const double *p8, double eps, double *out) {
  build_generators();
  cplx X[9] = {0};
  for (int a = 0; a < 8; a++)
    for (int k = 0; k < 9; k++) X[k] += I * eps * p8[a] * Tgen[a][k];
  double nrm = 0;
  for (int k = 0; k < 9; k++) nrm += creal(X[k] * conj(X[k]));
  nrm = sqrt(nrm);
  int s = 0;
  while (nrm > 0.125) {
    nrm *= 0.5;
    s++;
  }
  double scale = ldexp(1.0, -s);
  for (int k = 0; k < 9; k++) X[k] *= scale;
  cplx E[9] = {1, 0, 0, 0, 1, 0, 0, 0, 1}, term[9] = {1, 0, 0, 0, 1, 0, 0, 0, 1};
  for (int n = 1; n <= 20; n++) {
    mat_mul(term, X, term);
    for (int k = 0; k < 9; k++) term[k] /= n;
    for (int k = 0; k < 9; k++) E[k] += term[k];
  }
  for (int q = 0; q < s; q++) mat_mul(E, E, E);
  memcpy(out, E, sizeof(E));
}

/* U_mu(x) <- exp(i eps P_mu(x)) U_mu(x) for every link; P layout [mu][V][8]. */
void or_update_links(double *U, const double *P, const int *L, double eps) {
  build_generators();
  long V = volume(L);
#pragma omp parallel for schedule(static)
  for (long i = 0; i < V; i++)
    for (int mu = 0; mu < 4; mu++) {
      cplx E[9];
      or_expi(P + ((long)mu * V + i) * 8, eps, (double *)E);
      cplx *u = link_mut(U, i, mu);
      mat_mul(E, u, u);
    }
}

/* ------------------------------------------------------------------ */
/* Philox4x32-10 (Salmon, Moraes, Dror, Shaw, "Parallel random numbers:   */
/* as easy as 1, 2, 3", SC'11).  Replaces the paper's RANLUX generator;    */
/* the paper prints no number that depends on the generator.              */
/* Round: (hi0, lo0) = mulhilo(M0, c0), (hi1, lo1) = mulhilo(M1, c2),      */
/*        c = (hi1 ^ c1 ^ k0, lo1, hi0 ^ c3 ^ k1, lo0);                    */
/* key bump between rounds: k0 += W0, k1 += W1.                            */
/* ------------------------------------------------------------------ */

void or_philox4x32_10(const uint32_t ctr_in[4], const uint32_t key_in[2], uint32_t out[4]) {
  const uint32_t M0 = 0xD2511F53u, M1 = 0xCD9E8D57u, W0 = 0x9E3779B9u, W1 = 0xBB67AE85u;
  uint32_t c0 = ctr_in[0], c1 = ctr_in[1], c2 = ctr_in[2], c3 = ctr_in[3];
  uint32_t k0 = key_in[0], k1 = key_in[1];
  for (int r = 0; r < 10; r++) {
    uint64_t p0 = (uint64_t)M0 * c0, p1 = (uint64_t)M1 * c2;
    uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
    uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
    uint32_t n0 = hi1 ^ c1 ^ k0, n1 = lo1, n2 = hi0 ^ c3 ^ k1, n3 = lo0;
    c0 = n0; c1 = n1; c2 = n2; c3 = n3;
    if (r < 9) {
      k0 += W0;
      k1 += W1;
    }
  }
  out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

/* Two uniforms in (0,1) from one Philox block: 52 bits each,
 *   u = (k + 1/2) 2^-52,  k = (w_hi << 20) | (w_lo >> 12).                 */
static void philox_uniform2(uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3, uint64_t seed,
                            double u[2]) {
  uint32_t ctr[4] = {c0, c1, c2, c3}, key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)}, w[4];
  or_philox4x32_10(ctr, key, w);
  uint64_t ka = ((uint64_t)w[0] << 20) | (w[1] >> 12);
  uint64_t kb = ((uint64_t)w[2] << 20) | (w[3] >> 12);
  u[0] = ((double)ka + 0.5) * 0x1p-52;
  u[1] = ((double)kb + 0.5) * 0x1p-52;
}

void or_philox_uniform2(uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3, uint64_t seed,
                        double *u) {
  philox_uniform2(c0, c1, c2, c3, seed, u);
}

/* Stream tags in counter word 2 (bits 8..15). */
enum { TAG_HEATBATH = 0, TAG_MOMENTUM = 1, TAG_ETA = 2, TAG_DIRECTION = 3 };

/* Gaussian momenta p^a ~ N(0,1) (Sec. 2.2, "Gaussian momenta P") for
 * trajectory traj: link (x, mu) uses counters (x, traj, mu | TAG<<8, k),
 * k = 0..3, each block giving one Box-Muller pair.  Layout [mu][V][8].   */
void or_momenta(double *P, const int *L, uint64_t seed, uint32_t traj) {
  long V = volume(L);
  for (long i = 0; i < V; i++)
    for (int mu = 0; mu < 4; mu++)
      for (int k = 0; k < 4; k++) {
        double u[2];
        philox_uniform2((uint32_t)i, traj, (uint32_t)mu | (TAG_MOMENTUM << 8), (uint32_t)k, seed, u);
        double r = sqrt(-2.0 * log(u[0]));
        P[((long)mu * V + i) * 8 + 2 * k] = r * cos(2.0 * M_PI * u[1]);
        P[((long)mu * V + i) * 8 + 2 * k + 1] = r * sin(2.0 * M_PI * u[1]);
      }
}

/* Gaussian spinor field eta with density ~ exp(-eta^+ eta): every real
 * component ~ N(0, 1/2).  Site x uses counters (x, traj, TAG<<8, k),
 * k = 0..11; block k gives the real and imaginary part of component k.   */
void or_gaussian_spinor(double *eta, const int *L, uint64_t seed, uint32_t traj) {
  long V = volume(L);
  for (long i = 0; i < V; i++)
    for (int k = 0; k < 12; k++) {
      double u[2];
      philox_uniform2((uint32_t)i, traj, (uint32_t)(TAG_ETA << 8), (uint32_t)k, seed, u);
      double r = sqrt(-2.0 * log(u[0])) * sqrt(0.5);
      eta[24 * i + 2 * k] = r * cos(2.0 * M_PI * u[1]);
      eta[24 * i + 2 * k + 1] = r * sin(2.0 * M_PI * u[1]);
    }
}

/* ------------------------------------------------------------------ */
/* Heatbath (Sec. 2.2, Fig. "heatbath algorithm"; Creutz, Cabibbo-Marinari, */
/* Kennedy-Pendleton).  For one link U with staple sum A and each SU(2)     */
/* subgroup (i, j) in the order (0,1), (1,2), (0,2):                        */
/*   W = U A at the current U; w = 2x2 block (i, j) of W;                   */
/*   w_q = quaternion (SU(2)-proportional) part of w, k = sqrt(det w_q),    */
/*   w_hat = w_q / k;                                                       */
/*   draw y in SU(2) with density ~ sqrt(1 - y0^2) exp(b y0) dy0 dOmega,     */
/*   b = 2 beta k / 3 (Creutz for small b, Kennedy-Pendleton for large b);  */
/*   v = y w_hat^+, V = v embedded at (i, j), U <- V U.                      */
/* Reading: the printed sketch uses L(i) before defining it and multiplies  */
/* on the right; the update is applied on the left at the current U.       */
/* Random numbers: link (x, mu), subgroup g, attempt n uses the blocks     */
/*   (x, sweep, mu | g << 2 | TAG_HEATBATH << 8, 2n) and (..., 2n + 1)      */
/* (see su2_sample_y0) and the direction block                              */
/*   (x, sweep, mu | g << 2 | TAG_DIRECTION << 8, 0) -> (u5, u6):           */
/*   cos(theta) = 2 u5 - 1, phi = 2 pi u6.                                  */
/* After HB_MAX_ATTEMPTS rejections the subgroup is left unchanged.          */
/* ------------------------------------------------------------------ */

#define HB_MAX_ATTEMPTS 1024
#define HB_B_SWITCH 1.5

/* Draw y0 with density ~ sqrt(1 - y0^2) exp(b y0) on [-1, 1] using counter
 * words (c0, c1, c2); attempt n uses the blocks c3 = 2n and 2n + 1.
 * Two exact rejection methods, both cited by the paper (Sec. 2.2):
 *   b <  HB_B_SWITCH: Creutz -- y0 from exp(b y0) by inversion,
 *       y0 = 1 + log1p(expm1(-2b) (1 - u1)) / b, accepted when
 *       u2^2 <= 1 - y0^2 (uses only block 2n);
 *   b >= HB_B_SWITCH: Kennedy-Pendleton -- lambda^2 = -(ln r1 +
 *       cos^2(2 pi r2) ln r3) / (2b), accepted when r4^2 <= 1 - lambda^2,
 *       y0 = 1 - 2 lambda^2.
 * Returns the number of attempts used, or 0 when HB_MAX_ATTEMPTS ran out. */
static int su2_sample_y0(double b, uint32_t c0, uint32_t c1, uint32_t c2, uint64_t seed,
                         double *y0) {
  for (int n = 0; n < HB_MAX_ATTEMPTS; n++) {
    double u12[2], u34[2];
    philox_uniform2(c0, c1, c2, (uint32_t)(2 * n), seed, u12);
    if (b < HB_B_SWITCH) {
      /* b -> 0 limit of the inversion (beta = 0): y0 uniform on [-1, 1] */
      double y = b > 1e-300 ? 1.0 + log1p(expm1(-2.0 * b) * (1.0 - u12[0])) / b : 2.0 * u12[0] - 1.0;
      if (u12[1] * u12[1] <= 1.0 - y * y) {
        *y0 = y;
        return n + 1;
      }
      continue;
    }
    philox_uniform2(c0, c1, c2, (uint32_t)(2 * n + 1), seed, u34);
    double c = cos(2.0 * M_PI * u12[1]);
    double lam2 = -(log(u12[0]) + c * c * log(u34[0])) / (2.0 * b);
    if (u34[1] * u34[1] <= 1.0 - lam2) {
      *y0 = 1.0 - 2.0 * lam2;
      return n + 1;
    }
  }
  return 0;
}

/* Exposed for the sampler distribution test: n samples at parameter b. */
void or_su2_y0_samples(double b, uint64_t seed, int n, double *out) {
  for (int k = 0; k < n; k++) {
    double y0 = 2.0;
    su2_sample_y0(b, (uint32_t)k, 0u, (uint32_t)(TAG_HEATBATH << 8), seed, &y0);
    out[k] = y0;
  }
}

static const int SUBGROUP[3][2] = {{0, 1}, {1, 2}, {0, 2}};

/* One heatbath update of link (i, mu); returns the number of subgroups
 * left unchanged because the rejection loop gave up.                   */
static int heatbath_link(double *U, const int *L, long i, int mu, double beta, uint64_t seed,
                         uint32_t sweep) {
  cplx A[9];
  or_staple(U, L, i, mu, (double *)A);
  cplx *u = link_mut(U, i, mu);
  int failures = 0;
  for (int g = 0; g < 3; g++) {
    int p = SUBGROUP[g][0], q = SUBGROUP[g][1];
    cplx W[9];
    mat_mul(u, A, W);
    cplx wa = W[3 * p + p], wb = W[3 * p + q], wc = W[3 * q + p], wd = W[3 * q + q];
    double q0 = 0.5 * creal(wa + wd), q3 = 0.5 * cimag(wa - wd);
    double q1 = 0.5 * cimag(wb + wc), q2 = 0.5 * creal(wb - wc);
    double k = sqrt(q0 * q0 + q1 * q1 + q2 * q2 + q3 * q3);
    if (!(k > 1e-300)) {
      failures++;
      continue;
    }
    double b = 2.0 * beta * k / 3.0;
    uint32_t c2 = (uint32_t)mu | ((uint32_t)g << 2) | (TAG_HEATBATH << 8);
    double y0;
    if (!su2_sample_y0(b, (uint32_t)i, sweep, c2, seed, &y0)) {
      failures++;
      continue;
    }
    double ud[2];
    philox_uniform2((uint32_t)i, sweep, (uint32_t)mu | ((uint32_t)g << 2) | (TAG_DIRECTION << 8), 0u,
                    seed, ud);
    double ct = 2.0 * ud[0] - 1.0, st = sqrt(1.0 - ct * ct), ph = 2.0 * M_PI * ud[1];
    double rr = sqrt(1.0 - y0 * y0 > 0 ? 1.0 - y0 * y0 : 0.0);
    double y1 = rr * st * cos(ph), y2 = rr * st * sin(ph), y3 = rr * ct;
    /* y and w_hat as 2x2 matrices: [[a0 + i a3, a2 + i a1], [-a2 + i a1, a0 - i a3]] */
    cplx Y[2][2] = {{y0 + I * y3, y2 + I * y1}, {-y2 + I * y1, y0 - I * y3}};
    double h0 = q0 / k, h1 = q1 / k, h2 = q2 / k, h3 = q3 / k;
    cplx Wh[2][2] = {{h0 + I * h3, h2 + I * h1}, {-h2 + I * h1, h0 - I * h3}};
    cplx v[2][2];
    for (int r = 0; r < 2; r++)
      for (int c = 0; c < 2; c++) v[r][c] = Y[r][0] * conj(Wh[c][0]) + Y[r][1] * conj(Wh[c][1]);
    cplx Vm[9] = {1, 0, 0, 0, 1, 0, 0, 0, 1};
    Vm[3 * p + p] = v[0][0];
    Vm[3 * p + q] = v[0][1];
    Vm[3 * q + p] = v[1][0];
    Vm[3 * q + q] = v[1][1];
    mat_mul(Vm, u, u);
  }
  return failures;
}

/* One sweep: for mu = 0..3, for parity = even, odd: every link (x, mu) with
 * x of that parity (these links do not appear in each other's staples).  */
int or_heatbath_sweep(double *U, const int *L, double beta, uint64_t seed, uint32_t sweep) {
  build_gammas();
  build_generators();
  long V = volume(L);
  int failures = 0;
  for (int mu = 0; mu < 4; mu++)
    for (int par = 0; par < 2; par++) {
#pragma omp parallel for reduction(+ : failures) schedule(static)
      for (long i = 0; i < V; i++)
        if (or_parity(i, L) == par) failures += heatbath_link(U, L, i, mu, beta, seed, sweep);
    }
  return failures;
}

/* ------------------------------------------------------------------ */
/* Overrelaxation (Sec. 2.2: the update routine of the heatbath figure is */
/* either the exact SU(2) update or an overrelaxation step, which moves   */
/* through configuration space faster; Sec. 5.1 measures both kernels).   */
/* For one link U with staple sum A and each SU(2) subgroup (i, j) in the */
/* heatbath's order, w_hat is the unit quaternion of block (i, j) of      */
/* W = U A at the current U, exactly as in the heatbath, and the subgroup  */
/* element is replaced by its reflection:  v = (w_hat^+)^2, U <- V U with  */
/* v embedded at (i, j).  Then block (i, j) of V U A is v k w_hat =        */
/* k w_hat^+, whose real trace equals that of k w_hat: Re Tr(U A), and so  */
/* the action, is unchanged (microcanonical), and reflecting one subgroup */
/* twice with the same staple gives back U.  No random numbers.           */
/* ------------------------------------------------------------------ */

/* Reflects the subgroups g in gmask (bit g, order g = 0, 1, 2) of one link
 * (complex 3x3, row-major) for staple sum A; returns the number of
 * subgroups skipped because their block has no quaternion part (k = 0). */
int or_overrelax_link(double *link, const double *staple, int gmask) {
  cplx *u = (cplx *)link;
  const cplx *A = (const cplx *)staple;
  int skipped = 0;
  for (int g = 0; g < 3; g++) {
    if (!(gmask & (1 << g))) continue;
    int p = SUBGROUP[g][0], q = SUBGROUP[g][1];
    cplx W[9];
    mat_mul(u, A, W);
    cplx wa = W[3 * p + p], wb = W[3 * p + q], wc = W[3 * q + p], wd = W[3 * q + q];
    double q0 = 0.5 * creal(wa + wd), q3 = 0.5 * cimag(wa - wd);
    double q1 = 0.5 * cimag(wb + wc), q2 = 0.5 * creal(wb - wc);
    double k = sqrt(q0 * q0 + q1 * q1 + q2 * q2 + q3 * q3);
    if (!(k > 1e-300)) {
      skipped++;
      continue;
    }
    double h0 = q0 / k, h1 = q1 / k, h2 = q2 / k, h3 = q3 / k;
    cplx Wh[2][2] = {{h0 + I * h3, h2 + I * h1}, {-h2 + I * h1, h0 - I * h3}};
    cplx Whd[2][2];
    for (int r = 0; r < 2; r++)
      for (int c = 0; c < 2; c++) Whd[r][c] = conj(Wh[c][r]);
    cplx Vm[9] = {1, 0, 0, 0, 1, 0, 0, 0, 1};
    for (int r = 0; r < 2; r++)
      for (int c = 0; c < 2; c++) {
        cplx v = Whd[r][0] * Whd[0][c] + Whd[r][1] * Whd[1][c];
        Vm[3 * (r ? q : p) + (c ? q : p)] = v;
      }
    mat_mul(Vm, u, u);
  }
  return skipped;
}

/* One overrelaxation sweep in the heatbath's checkerboard order: for mu =
 * 0..3, parity even, odd, every link of that class with all three
 * subgroups.  Returns the number of skipped subgroups.                   */
int or_overrelax_sweep(double *U, const int *L) {
  long V = volume(L);
  int skipped = 0;
  for (int mu = 0; mu < 4; mu++)
    for (int par = 0; par < 2; par++) {
#pragma omp parallel for reduction(+ : skipped) schedule(static)
      for (long i = 0; i < V; i++)
        if (or_parity(i, L) == par) {
          double A[18];
          or_staple(U, L, i, mu, A);
          skipped += or_overrelax_link((double *)link_mut(U, i, mu), A, 7);
        }
    }
  return skipped;
}

/* ------------------------------------------------------------------ */
/* HMC (Sec. 2.2): H = 1/2 sum p^2 + S_g + S_pf; leapfrog with n steps of   */
/* size eps:                                                                */
/*   p <- p + eps/2 F;  (U <- exp(i eps P) U; p <- p + eps F) x (n-1);       */
/*   U <- exp(i eps P) U;  p <- p + eps/2 F,   F = -dS/domega.               */
/* Metropolis: accept with min(1, exp(-(H' - H))) (the printed exponent's     */
/* sign is read as exp(-dH)).  The pseudofermion field phi = Mhat^+ eta on   */
/* the even sites is fixed for the trajectory.  With nf = 0 only S_g.         */
/* ------------------------------------------------------------------ */

static double kinetic(const double *P, long n) {
  double s = 0;
  for (long k = 0; k < n; k++) s += P[k] * P[k];
  return 0.5 * s;
}

static void total_dSdw(const double *U, const double *phi, double *X, const int *L, double beta,
                       double kappa, double mu, int nf, double tol, int max_iter, double *F) {
  long V = volume(L);
  long nP = 32 * V;
  or_gauge_dSdw(U, L, beta, F);
  if (nf) {
    double *Ff = malloc(nP * sizeof(double));
    double resid;
    or_cg(U, phi, X, L, 1, kappa, mu, tol, max_iter, 1, &resid);
    or_fermion_dSdw(U, X, L, 1, kappa, mu, 1, Ff);
    for (long k = 0; k < nP; k++) F[k] += Ff[k];
    free(Ff);
  }
}

/* Runs the molecular-dynamics part on (U, P) in place and returns dH.
 * h_out[0..2] = (H0, H1, S_pf0) for inspection.                          */
double or_hmc_md(double *U, double *P, const double *phi, const int *L, double beta, double kappa,
                 double mu, int nf, int nsteps, double tau, double tol, int max_iter,
                 double *h_out) {
  build_gammas();
  build_generators();
  long V = volume(L);
  long nP = 32 * V;
  size_t n = (size_t)V * 24;
  double eps = tau / nsteps;
  double *F = malloc(nP * sizeof(double));
  double *X = calloc(n, sizeof(double));
  double S0 = or_gauge_action(U, L, beta), Sf0 = 0;
  if (nf) Sf0 = or_pseudofermion_action(U, phi, X, L, 1, kappa, mu, 1, tol, max_iter);
  double H0 = kinetic(P, nP) + S0 + Sf0;
  total_dSdw(U, phi, X, L, beta, kappa, mu, nf, tol, max_iter, F);
  for (long k = 0; k < nP; k++) P[k] -= 0.5 * eps * F[k];
  for (int s = 0; s < nsteps; s++) {
    or_update_links(U, P, L, eps);
    total_dSdw(U, phi, X, L, beta, kappa, mu, nf, tol, max_iter, F);
    double w = (s == nsteps - 1) ? 0.5 * eps : eps;
    for (long k = 0; k < nP; k++) P[k] -= w * F[k];
  }
  double S1 = or_gauge_action(U, L, beta), Sf1 = 0;
  if (nf) Sf1 = or_pseudofermion_action(U, phi, X, L, 1, kappa, mu, 1, tol, max_iter);
  double H1 = kinetic(P, nP) + S1 + Sf1;
  if (h_out) {
    h_out[0] = H0;
    h_out[1] = H1;
    h_out[2] = Sf0;
  }
  free(F);
  free(X);
  return H1 - H0;
}

/* ------------------------------------------------------------------ */
/* HMC with the second-order minimum-norm (2MN, Omelyan) integrator on   */
/* two time scales (Sec. 2.2: "2MN scheme", "multiple timescales"; Sec.  */
/* 5.3: separate scales for the gauge and fermion parts, 2MN on each).   */
/* One 2MN step of size e for a force F and position update Q(h):        */
/*   P -= lambda e dS;  Q(e/2);  P -= (1 - 2 lambda) e dS;  Q(e/2);       */
/*   P -= lambda e dS.                                                    */
/* Outer scale: the fermion force, n_f steps over tau.  Every outer      */
/* position update Q(h) is the inner integration of the gauge force over  */
/* time h with n_g 2MN steps, whose own position update is               */
/* U <- exp(i h' P) U.  Each force is evaluated where the scheme needs it */
/* (no merging of consecutive momentum updates).  With nf = 0 only the    */
/* gauge force acts.  Returns dH; h_out = (H0, H1, S_pf0).                */
/* ------------------------------------------------------------------ */

typedef struct {
  const int *L;
  double beta, c1, kappa, mu, lambda, tol;
  int nf, ng, max_iter;
  const double *phi;
  double *X, *F;
  long nP;
} md_ctx;

static void p_update(double *P, const double *F, double w, long n) {
  for (long k = 0; k < n; k++) P[k] -= w * F[k];
}

static void inner_gauge_2mn(md_ctx *c, double *U, double *P, double h) {
  double d = h / c->ng;
  for (int s = 0; s < c->ng; s++) {
    or_gauge_dSdw_sym(U, c->L, c->beta, c->c1, c->F);
    p_update(P, c->F, c->lambda * d, c->nP);
    or_update_links(U, P, c->L, 0.5 * d);
    or_gauge_dSdw_sym(U, c->L, c->beta, c->c1, c->F);
    p_update(P, c->F, (1.0 - 2.0 * c->lambda) * d, c->nP);
    or_update_links(U, P, c->L, 0.5 * d);
    or_gauge_dSdw_sym(U, c->L, c->beta, c->c1, c->F);
    p_update(P, c->F, c->lambda * d, c->nP);
  }
}

static void fermion_step(md_ctx *c, const double *U, double *P, double w) {
  if (!c->nf) return;
  double resid;
  or_cg(U, c->phi, c->X, c->L, 1, c->kappa, c->mu, c->tol, c->max_iter, 1, &resid);
  or_fermion_dSdw(U, c->X, c->L, 1, c->kappa, c->mu, 1, c->F);
  p_update(P, c->F, w, c->nP);
}

double or_hmc_md_2mn(double *U, double *P, const double *phi, const int *L, double beta, double c1,
                     double kappa, double mu, int nf, int nsteps_f, int nsteps_g, double lambda,
                     double tau, double tol, int max_iter, double *h_out) {
  build_gammas();
  build_generators();
  long V = volume(L);
  md_ctx c = {L, beta, c1, kappa, mu, lambda, tol, nf, nsteps_g, max_iter, phi, NULL, NULL, 32 * V};
  c.F = malloc(c.nP * sizeof(double));
  c.X = calloc((size_t)V * 24, sizeof(double));
  double S0 = or_gauge_action_sym(U, L, beta, c1), Sf0 = 0;
  if (nf) Sf0 = or_pseudofermion_action(U, phi, c.X, L, 1, kappa, mu, 1, tol, max_iter);
  double H0 = kinetic(P, c.nP) + S0 + Sf0;
  double e = tau / nsteps_f;
  for (int s = 0; s < nsteps_f; s++) {
    fermion_step(&c, U, P, lambda * e);
    inner_gauge_2mn(&c, U, P, 0.5 * e);
    fermion_step(&c, U, P, (1.0 - 2.0 * lambda) * e);
    inner_gauge_2mn(&c, U, P, 0.5 * e);
    fermion_step(&c, U, P, lambda * e);
  }
  double S1 = or_gauge_action_sym(U, L, beta, c1), Sf1 = 0;
  if (nf) Sf1 = or_pseudofermion_action(U, phi, c.X, L, 1, kappa, mu, 1, tol, max_iter);
  double H1 = kinetic(P, c.nP) + S1 + Sf1;
  if (h_out) {
    h_out[0] = H0;
    h_out[1] = H1;
    h_out[2] = Sf0;
  }
  free(c.F);
  free(c.X);
  return H1 - H0;
}
