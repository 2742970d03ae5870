/*
 * nrmg_oracle.c -- plain, serial, FP64 CPU oracle of the regularized-moment
 * nonlinear multigrid solver of Hu & Li, "An efficient nonlinear multigrid
 * solver for the simulation of rarefied gas cavity flow" (arXiv 2206.13164).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path may link, load or
 * call this file: only the test suite, the smoke check and the CPU-baseline
 * leg of the benchmark use it.  It shares no code, header, table or
 * generator with the CUDA library; both are written independently from the
 * paper.
 *
 * Every function follows the paper's definitions step by step, in the
 * paper's order and notation, with no blocking, fusion or reordering:
 *   - Hermite basis, Grad relations .............. Sec. 2.2, eq. (dis-expansion),
 *                                                  eq. (moments-relation), eq. (truncated-dis)
 *   - basis transformation F_M^[w,t] -> F_M^[w~,t~] Sec. 2.3 (projection of fluxes)
 *   - finite-volume residual R_ij ................. Sec. 2.3, eq. (ode-system),
 *                                                  eq. (flux-force-expansion), eq. (moments-recon)
 *   - BGK / Shakhov / ES-BGK collision ............ Sec. 2.1, eq. (col-relaxation),
 *                                                  eq. (BGK-f^E), eq. (Shakhov-f^E), eq. (ES-f^E);
 *                                                  Sec. 4, eq. (nu-shakhov)
 *   - local time step, two-step update ............ Sec. 2.4, eq. (local-CFL)
 *   - forward Euler step .......................... Sec. 2.4, eq. (euler-scheme), eq. (global-CFL)
 *   - fast sweeping step FS(f, r) ................. Sec. 3.1, Algorithm 1
 *   - restriction / prolongation .................. Sec. 3.2.2, eq. (uH-thetaH-computation),
 *                                                  eq. (fH), eq. (rewritten-update)
 *   - (k+1)-level NMG step ........................ Sec. 3.2.3, Algorithm 2
 *   - relative residual and its norm .............. Sec. 3.2.3, eq. (relative-residual)
 *
 * Where the paper does not print a formula, the oracle takes one reading and
 * says so at the function:
 *   - interior numerical flux: HLL form of the regularized operator
 *     P_M xi P_M (the paper defers to an external reference)  -- parity with
 *     the paper's own flux is UNPINNED; the flux is pinned to its own
 *     definition (consistency, upwind limits, conservation, Maxwellian fixed
 *     point, and in its middle branch the intermediate-state form of the HLL
 *     flux and its Rusanov special case);
 *   - Maxwell wall: kinetic half-range flux with zero wall mass flux  --
 *     parity with the paper's own boundary condition is UNPINNED; pinned to
 *     velocity-space quadrature of that reading;
 *   - limited slope: van Albada average (the paper prints central slopes);
 *     pinned to its defining properties (central slope for equal one-sided
 *     differences, zero for opposite ones and at a flat side, symmetry,
 *     convexity, Sweby's limiter function, second-order accuracy);
 *   - the "correction" applied after each NMG step: total-mass rescaling --
 *     parity UNPINNED (the paper names it only by reference);
 *   - local norm of R_ij: weighted L2 norm of F_M, weight alpha! theta^-|alpha|
 *     -- pinned up to a constant factor by quadrature.
 *
 * OpenMP mode (or_set_threads, n > 1; used only to time the oracle on many
 * cores): a sweep takes its cells by anti-diagonals of its own visiting order,
 * the cells of one diagonal in parallel, and the residual, restriction and
 * coarse-grid update run their independent cells in parallel with sums kept
 * in the serial order.  Every cell reads the same values as in the serial
 * order, so both modes give the same results bit for bit (tested).
 *
 * Units are nondimensional (m_* = 1).  Multi-indices alpha, |alpha| <= M, are
 * enumerated in graded order: |alpha| ascending, then alpha_1 descending, then
 * alpha_2 descending.  A cell state is (u_1, u_2, u_3, theta) plus N_M
 * coefficients.  Cells are stored row-major, index j*nx + i, with i along x.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>

#define OR_MAXM 20
#define OR_MAXN 1771 /* C(23,3) */
#define OR_MAXLEV 16

enum { OR_OK = 0, OR_ERR_ARG = 1, OR_ERR_NONPHYSICAL = 4, OR_ERR_NOT_CONVERGED = 5 };
enum { OR_BGK = 0, OR_SHAKHOV = 1, OR_ESBGK = 2 };

/* van Albada smoothing constant (squared), nondimensional */
#define OR_VA_EPS2 1e-12

/* ------------------------------------------------------------------ */
/* Multi-index enumeration (Sec. 2.2, eq. truncated-dis)               */
/* ------------------------------------------------------------------ */
typedef struct {
  int M, n;
  int a[OR_MAXN][3];
  int *cube; /* (M+1)^3, -1 where |alpha| > M */
} basis_t;

static basis_t *g_basis[OR_MAXM + 1];

static const basis_t *basis(int M) {
  if (g_basis[M]) return g_basis[M];
  basis_t *b = (basis_t *)calloc(1, sizeof(basis_t));
  int m1 = M + 1;
  b->M = M;
  b->cube = (int *)malloc(sizeof(int) * m1 * m1 * m1);
  for (int q = 0; q < m1 * m1 * m1; ++q) b->cube[q] = -1;
  int k = 0;
  for (int deg = 0; deg <= M; ++deg)
    for (int a1 = deg; a1 >= 0; --a1)
      for (int a2 = deg - a1; a2 >= 0; --a2) {
        int a3 = deg - a1 - a2;
        b->a[k][0] = a1;
        b->a[k][1] = a2;
        b->a[k][2] = a3;
        b->cube[(a1 * m1 + a2) * m1 + a3] = k;
        ++k;
      }
  b->n = k;
  g_basis[M] = b;
  return b;
}

/* index of (a1,a2,a3), or -1 when outside {|alpha| <= M} */
static int idx3(const basis_t *b, int a1, int a2, int a3) {
  if (a1 < 0 || a2 < 0 || a3 < 0 || a1 + a2 + a3 > b->M) return -1;
  int m1 = b->M + 1;
  return b->cube[(a1 * m1 + a2) * m1 + a3];
}

static int idx_shift(const basis_t *b, int o, int d, int k) {
  int t[3] = {b->a[o][0], b->a[o][1], b->a[o][2]};
  t[d] += k;
  return idx3(b, t[0], t[1], t[2]);
}

static double factorial(int k) {
  double r = 1.0;
  for (int q = 2; q <= k; ++q) r *= q;
  return r;
}

int or_nmom(int M) { return (M + 1) * (M + 2) * (M + 3) / 6; }

void or_alphas(int M, int *out) {
  const basis_t *b = basis(M);
  for (int o = 0; o < b->n; ++o)
    for (int d = 0; d < 3; ++d) out[3 * o + d] = b->a[o][d];
}

/* ------------------------------------------------------------------ */
/* Largest root C_n of He_n (Sec. 2.4, eq. local-CFL)                  */
/* Newton's method from an upper bound of the spectrum; the iteration  */
/* decreases monotonically to the largest root.                        */
/* ------------------------------------------------------------------ */
static void hermite_eval(int n, double x, double *p, double *dp) {
  /* He_{k+1}(x) = x He_k(x) - k He_{k-1}(x);  He_n' = n He_{n-1} */
  double hm = 1.0, h = x;
  if (n == 0) { *p = 1.0; *dp = 0.0; return; }
  for (int k = 1; k < n; ++k) {
    double hp = x * h - k * hm;
    hm = h;
    h = hp;
  }
  *p = h;
  *dp = n * hm;
}

double or_hermite_max_root(int n) {
  if (n <= 1) return 0.0;
  double x = sqrt(4.0 * n + 2.0);
  for (int it = 0; it < 200; ++it) {
    double p, dp;
    hermite_eval(n, x, &p, &dp);
    double xn = x - p / dp;
    if (!(xn < x)) break;
    x = xn;
  }
  return x;
}

/* ------------------------------------------------------------------ */
/* Basis transformation (Sec. 2.3): re-expand f in F_M^[src] into      */
/* F_M^[dst].  Along the straight path between the two parameter sets  */
/* dH_alpha/dw_d = H_{alpha+e_d} and dH_alpha/dt = 1/2 sum_d           */
/* H_{alpha+2e_d}, so the coefficients obey g' = -(sum_d a_d S_d +     */
/* b S_d^2) g with S_d the index shift alpha-e_d -> alpha, a_d = w~_d - */
/* w_d, b = (t~ - t)/2.  Hence g = prod_d exp(-a_d S_d - b S_d^2) f,   */
/* and the series exp(-a z - b z^2) = sum c_k z^k has c_0 = 1,         */
/* c_1 = -a, (k+1) c_{k+1} = -a c_k - 2 b c_{k-1}.  Every output       */
/* coefficient depends only on inputs of lower or equal degree, so the */
/* truncation to |alpha| <= M is exact.  g may alias f.                */
/* ------------------------------------------------------------------ */
void or_transform(int M, const double *src, const double *dst, const double *f, double *g) {
  const basis_t *b = basis(M);
  double cur[OR_MAXN], nxt[OR_MAXN];
  memcpy(cur, f, sizeof(double) * b->n);
  double bb = 0.5 * (dst[3] - src[3]);
  for (int d = 0; d < 3; ++d) {
    double a = dst[d] - src[d];
    double c[OR_MAXM + 2];
    c[0] = 1.0;
    c[1] = -a;
    for (int k = 1; k < M; ++k) c[k + 1] = (-a * c[k] - 2.0 * bb * c[k - 1]) / (k + 1);
    for (int o = 0; o < b->n; ++o) {
      double s = 0.0;
      for (int k = 0; k <= b->a[o][d]; ++k) s += c[k] * cur[idx_shift(b, o, d, -k)];
      nxt[o] = s;
    }
    memcpy(cur, nxt, sizeof(double) * b->n);
  }
  memcpy(g, cur, sizeof(double) * b->n);
}

/* ------------------------------------------------------------------ */
/* Multiplication by xi_d, projected on F_M (Sec. 2.2).  From          */
/* v He_n = He_{n+1} + n He_{n-1} and the basis definition,            */
/* xi_d H_alpha = t H_{alpha+e_d} + w_d H_alpha + alpha_d H_{alpha-e_d}, */
/* so (xi_d f)_alpha = w_d f_alpha + t f_{alpha-e_d}                   */
/* + (alpha_d+1) f_{alpha+e_d}; the last term is absent for |alpha|=M  */
/* (the regularized operator P_M xi_d P_M).                            */
/* ------------------------------------------------------------------ */
void or_xi_mul(int M, int d, const double *p, const double *f, double *g) {
  const basis_t *b = basis(M);
  for (int o = 0; o < b->n; ++o) {
    int om = idx_shift(b, o, d, -1), op = idx_shift(b, o, d, +1);
    double s = p[d] * f[o];
    if (om >= 0) s += p[3] * f[om];
    if (op >= 0) s += (b->a[o][d] + 1) * f[op];
    g[o] = s;
  }
}

/* ------------------------------------------------------------------ */
/* Macroscopic rho, u, theta of f in a general basis [w, t]            */
/* (eq. rho-u-theta with the moments of H_alpha):                      */
/*   rho = f_0,  rho u_d = rho w_d + f_{e_d},                          */
/*   rho|u|^2 + 3 rho theta = rho(|w|^2 + 3t) + 2 w.f_e + 2 sum f_{2e_d} */
/* out = {rho, u1, u2, u3, theta}.                                     */
/* ------------------------------------------------------------------ */
void or_macros(int M, const double *p, const double *f, double *out) {
  const basis_t *b = basis(M);
  double rho = f[0];
  double fe[3], f2 = 0.0, fe2 = 0.0;
  for (int d = 0; d < 3; ++d) {
    int e[3] = {0, 0, 0};
    e[d] = 1;
    fe[d] = f[idx3(b, e[0], e[1], e[2])];
    e[d] = 2;
    f2 += f[idx3(b, e[0], e[1], e[2])];
    fe2 += fe[d] * fe[d];
  }
  out[0] = rho;
  for (int d = 0; d < 3; ++d) out[1 + d] = p[d] + fe[d] / rho;
  out[4] = p[3] + (2.0 * f2 - fe2 / rho) / (3.0 * rho);
}

/* Grad-basis fields (eq. moments-relation):                           */
/* out = rho, u1,u2,u3, theta, s11,s12,s13,s22,s23,s33, q1,q2,q3.      */
void or_cell_fields(int M, const double *p, const double *f, double *out) {
  const basis_t *b = basis(M);
  out[0] = f[0];
  for (int d = 0; d < 3; ++d) out[1 + d] = p[d];
  out[4] = p[3];
  int k = 5;
  for (int i = 0; i < 3; ++i)
    for (int j = i; j < 3; ++j) {
      int e[3] = {0, 0, 0};
      e[i] += 1;
      e[j] += 1;
      out[k++] = (1.0 + (i == j)) * f[idx3(b, e[0], e[1], e[2])];
    }
  for (int i = 0; i < 3; ++i) {
    int e[3] = {0, 0, 0};
    e[i] = 3;
    double q = 2.0 * f[idx3(b, e[0], e[1], e[2])];
    for (int d = 0; d < 3; ++d) {
      int t[3] = {0, 0, 0};
      t[d] += 2;
      t[i] += 1;
      q += f[idx3(b, t[0], t[1], t[2])];
    }
    out[k++] = q;
  }
}

/* ------------------------------------------------------------------ */
/* Half-range integrals for the Maxwell wall (reading of Sec. 2.3's    */
/* boundary treatment).  phi(v) = exp(-v^2/2)/sqrt(2 pi).              */
/*   I_{k,m} = int_0^inf He_k He_m e^{-v^2/2} dv                       */
/*           = He_k(0) He_{m-1}(0) + k I_{k-1,m-1}   (m >= 1),         */
/*   I_{k,0} = He_{k-1}(0) (k >= 1),  I_{0,0} = sqrt(pi/2)            */
/* (integration by parts with He_m e^{-v^2/2} = -(He_{m-1} e^{..})').  */
/*   J+_{k,m} = int_{v>0} v He_k He_m phi dv                           */
/*            = (I_{k,m+1} + m I_{k,m-1}) / sqrt(2 pi),                */
/*   J-_{k,m} = (-1)^{k+m+1} J+_{k,m}.                                 */
/* J is (K+1)x(K+1), row k, column m; s = +1 or -1.                    */
/* ------------------------------------------------------------------ */
void or_halfrange(int K, int s, double *J) {
  int L = K + 2;
  double he0[OR_MAXM + 8];
  he0[0] = 1.0;
  he0[1] = 0.0;
  for (int n = 1; n + 1 < L + 1; ++n) he0[n + 1] = -n * he0[n - 1];
  double I[OR_MAXM + 8][OR_MAXM + 8];
  for (int k = 0; k <= L; ++k)
    for (int m = 0; m <= L; ++m) {
      if (m == 0)
        I[k][m] = (k == 0) ? sqrt(M_PI / 2.0) : he0[k - 1];
      else
        I[k][m] = he0[k] * he0[m - 1] + (k >= 1 ? k * I[k - 1][m - 1] : 0.0);
    }
  for (int k = 0; k <= K; ++k)
    for (int m = 0; m <= K; ++m) {
      double jp = (I[k][m + 1] + (m >= 1 ? m * I[k][m - 1] : 0.0)) / sqrt(2.0 * M_PI);
      double sg = ((k + m + 1) % 2 == 0) ? 1.0 : -1.0;
      J[k * (K + 1) + m] = (s > 0) ? jp : sg * jp;
    }
}

/* ------------------------------------------------------------------ */
/* Problem description and solver state                                */
/* ------------------------------------------------------------------ */
typedef struct {
  int nx, ny;
  double lx, ly;
  int levels;
  int M;
  double Kn;
  int model;
  double Pr, omega, beta;
  int order, slope;
  double cfl;
  int s1, s2, s3, gamma;
  double wall_u[4][3]; /* walls: 0 bottom y=0, 1 right x=lx, 2 top y=ly, 3 left x=0 */
  double wall_theta[4];
  double wall_chi[4];
  double dtnu; /* > 0: local time step capped at dtnu / nu (0: the CFL step alone) */
  /* non-uniform grid (Sec. 2.4: the local time step serves non-uniform grids): the widths of
   * the finest level's columns hx[nx] and rows hy[ny], summing to lx and ly; NULL: uniform */
  const double *hx, *hy;
} or_config;

typedef struct {
  int nx, ny;
  double dx, dy;      /* uniform widths (lx / nx, ly / ny) */
  double *hx, *hy;    /* width of each column and row (all dx, dy on a uniform grid) */
  int uniform;
  double *P, *F;     /* state: [cell][4], [cell][n] */
  double *rP, *rF;   /* right-hand side r and the basis it is expanded in */
  int has_r;
  double *bP, *bF;   /* restricted state saved for the coarse-grid update */
  double *D;         /* defect r - R(f) in the cell basis */
} or_level;

typedef struct {
  or_config c;
  int n;        /* N_M */
  double C;     /* C_{M+1} */
  double m0;    /* reference total mass */
  double res0;  /* ||R(f^0)|| of the finest level */
  int have_res0;
  int threads;  /* > 1: the OpenMP mode (same results, bit for bit); otherwise serial */
  or_level lev[OR_MAXLEV];
} or_solver;

static void set_maxwellian(or_solver *S, int l) {
  or_level *L = &S->lev[l];
  int nc = L->nx * L->ny;
  for (int c = 0; c < nc; ++c) {
    L->P[4 * c + 0] = 0.0;
    L->P[4 * c + 1] = 0.0;
    L->P[4 * c + 2] = 0.0;
    L->P[4 * c + 3] = 1.0;
    for (int o = 0; o < S->n; ++o) L->F[(size_t)c * S->n + o] = 0.0;
    L->F[(size_t)c * S->n] = 1.0;
  }
}

static double total_mass(const or_solver *S, int l) {
  const or_level *L = &S->lev[l];
  double m = 0.0;
  for (int c = 0; c < L->nx * L->ny; ++c) m += L->F[(size_t)c * S->n] * L->hx[c % L->nx] * L->hy[c / L->nx];
  return m;
}

or_solver *or_create(const or_config *cfg) {
  if (cfg->M < 3 || cfg->M > OR_MAXM || cfg->levels < 1 || cfg->levels > OR_MAXLEV) return NULL;
  or_solver *S = (or_solver *)calloc(1, sizeof(or_solver));
  S->c = *cfg;
  S->n = or_nmom(cfg->M);
  S->C = or_hermite_max_root(cfg->M + 1);
  basis(cfg->M);
  for (int l = cfg->levels - 1; l >= 0; --l) {
    or_level *L = &S->lev[l];
    int sh = cfg->levels - 1 - l;
    L->nx = cfg->nx >> sh;
    L->ny = cfg->ny >> sh;
    if ((L->nx << sh) != cfg->nx || (L->ny << sh) != cfg->ny || L->nx < 1 || L->ny < 1) {
      free(S);
      return NULL;
    }
    L->dx = cfg->lx / L->nx;
    L->dy = cfg->ly / L->ny;
    L->hx = (double *)malloc(sizeof(double) * L->nx);
    L->hy = (double *)malloc(sizeof(double) * L->ny);
    L->uniform = !(cfg->hx && cfg->hy);
    /* the finest level takes the given widths; a coarse cell merges two columns (rows) of the
     * next finer level, whose widths add */
    for (int i = 0; i < L->nx; ++i)
      L->hx[i] = L->uniform ? L->dx : (sh == 0 ? cfg->hx[i] : S->lev[l + 1].hx[2 * i] + S->lev[l + 1].hx[2 * i + 1]);
    for (int j = 0; j < L->ny; ++j)
      L->hy[j] = L->uniform ? L->dy : (sh == 0 ? cfg->hy[j] : S->lev[l + 1].hy[2 * j] + S->lev[l + 1].hy[2 * j + 1]);
    size_t nc = (size_t)L->nx * L->ny;
    L->P = (double *)calloc(nc * 4, sizeof(double));
    L->F = (double *)calloc(nc * S->n, sizeof(double));
    L->rP = (double *)calloc(nc * 4, sizeof(double));
    L->rF = (double *)calloc(nc * S->n, sizeof(double));
    L->bP = (double *)calloc(nc * 4, sizeof(double));
    L->bF = (double *)calloc(nc * S->n, sizeof(double));
    L->D = (double *)calloc(nc * S->n, sizeof(double));
    set_maxwellian(S, l);
  }
  S->m0 = total_mass(S, cfg->levels - 1);
  S->c.hx = S->c.hy = NULL; /* copied into the levels; the caller's arrays may go */
  return S;
}

void or_destroy(or_solver *S) {
  if (!S) return;
  for (int l = 0; l < S->c.levels; ++l) {
    or_level *L = &S->lev[l];
    free(L->P); free(L->F); free(L->rP); free(L->rF); free(L->bP); free(L->bF); free(L->D);
    free(L->hx); free(L->hy);
  }
  free(S);
}

/* n > 1 selects the OpenMP mode with n threads (results identical to the serial mode) */
void or_set_threads(or_solver *S, int n) { S->threads = n; }

int or_level_nx(const or_solver *S, int l) { return S->lev[l].nx; }
int or_level_ny(const or_solver *S, int l) { return S->lev[l].ny; }
double or_c_m1(const or_solver *S) { return S->C; }

void or_set_state(or_solver *S, int l, const double *P, const double *F) {
  or_level *L = &S->lev[l];
  size_t nc = (size_t)L->nx * L->ny;
  memcpy(L->P, P, nc * 4 * sizeof(double));
  memcpy(L->F, F, nc * S->n * sizeof(double));
  if (l == S->c.levels - 1) {
    S->m0 = total_mass(S, l);
    S->have_res0 = 0;
  }
}

void or_get_state(const or_solver *S, int l, double *P, double *F) {
  const or_level *L = &S->lev[l];
  size_t nc = (size_t)L->nx * L->ny;
  if (P) memcpy(P, L->P, nc * 4 * sizeof(double));
  if (F) memcpy(F, L->F, nc * S->n * sizeof(double));
}

/* r for level l, expanded in the bases rP; NULL clears it (r = 0) */
void or_set_rhs(or_solver *S, int l, const double *rP, const double *rF) {
  or_level *L = &S->lev[l];
  size_t nc = (size_t)L->nx * L->ny;
  if (!rP || !rF) {
    L->has_r = 0;
    return;
  }
  memcpy(L->rP, rP, nc * 4 * sizeof(double));
  memcpy(L->rF, rF, nc * S->n * sizeof(double));
  L->has_r = 1;
}

void or_get_rhs(const or_solver *S, int l, double *rP, double *rF) {
  const or_level *L = &S->lev[l];
  size_t nc = (size_t)L->nx * L->ny;
  memcpy(rP, L->rP, nc * 4 * sizeof(double));
  memcpy(rF, L->rF, nc * S->n * sizeof(double));
}

double or_mass(const or_solver *S) { return total_mass(S, S->c.levels - 1); }

/* ------------------------------------------------------------------ */
/* Reconstruction of face states (Sec. 2.3, eq. moments-recon).        */
/* Second order: u, theta and every coefficient of the cell's own      */
/* basis get a slope; the face state lives in the basis [u+-, t+-].    */
/* A cell whose neighbour along the axis is a wall gets zero slope     */
/* along that axis (the paper is silent there).                        */
/* ------------------------------------------------------------------ */
/* van Albada et al. (1982) smooth limited average of the one-sided differences a, b of a cell
 * of width h, as a slope */
static double va_slope(double a, double b, double h) {
  return ((b * b + OR_VA_EPS2) * a + (a * a + OR_VA_EPS2) * b) / ((a * a + b * b + 2.0 * OR_VA_EPS2) * h);
}

static double slope_of(int kind, double qm, double q0, double qp, double h) {
  if (kind == 1) return (qp - qm) / (2.0 * h); /* central, as printed */
  double a = q0 - qm, b = qp - q0;
  return va_slope(a, b, h);
}

/* The same slopes on a non-uniform grid: the cell of width h lies at centre distances hm and
 * hp from its lower and upper neighbours.  Central: (qp - qm) / (hm + hp); van Albada: the
 * same average of the one-sided differences scaled to the cell's width, a = (q0 - qm) h / hm,
 * b = (qp - q0) h / hp (on a uniform grid hm = hp = h and both reduce to the slopes above). */
static double slope_nu(int kind, double qm, double q0, double qp, double h, double hm, double hp) {
  if (kind == 1) return (qp - qm) / (hm + hp);
  return va_slope((q0 - qm) * (h / hm), (qp - q0) * (h / hp), h);
}

/* the slope of one coefficient from its three cell values along an axis (kind 1 central, */
/* 2 van Albada), exposed so that tests can check it against its defining properties      */
double or_slope(int kind, double qm, double q0, double qp, double h) { return slope_of(kind, qm, q0, qp, h); }

/* face state of cell (i,j) of level L on side sd (+1: east/north face, -1: west/south) of axis ax */
static void face_state(const or_solver *S, const or_level *L, int i, int j, int ax, int sd, double *p, double *f) {
  int n = S->n;
  int c = j * L->nx + i;
  memcpy(p, L->P + 4 * c, 4 * sizeof(double));
  memcpy(f, L->F + (size_t)c * n, n * sizeof(double));
  if (S->c.order != 2 || S->c.slope == 0) return;
  int len = ax == 0 ? L->nx : L->ny;
  int pos = ax == 0 ? i : j;
  if (pos == 0 || pos == len - 1) return; /* wall-adjacent: zero slope */
  int cm = ax == 0 ? c - 1 : c - L->nx;
  int cp = ax == 0 ? c + 1 : c + L->nx;
  const double *hs = ax == 0 ? L->hx : L->hy;
  double h = hs[pos], hm = 0.5 * (hs[pos - 1] + h), hp = 0.5 * (h + hs[pos + 1]);
  for (int q = 0; q < 4; ++q) {
    double g = L->uniform ? slope_of(S->c.slope, L->P[4 * cm + q], L->P[4 * c + q], L->P[4 * cp + q], h)
                          : slope_nu(S->c.slope, L->P[4 * cm + q], L->P[4 * c + q], L->P[4 * cp + q], h, hm, hp);
    p[q] = p[q] + sd * (0.5 * h) * g;
  }
  for (int o = 0; o < n; ++o) {
    double qm = L->F[(size_t)cm * n + o], q0 = L->F[(size_t)c * n + o], qp = L->F[(size_t)cp * n + o];
    double g = L->uniform ? slope_of(S->c.slope, qm, q0, qp, h) : slope_nu(S->c.slope, qm, q0, qp, h, hm, hp);
    f[o] = f[o] + sd * (0.5 * h) * g;
  }
}

/* face state of cell (i, j) of level l on side sd of axis ax (params p[4], coefficients f) */
void or_face_state(const or_solver *S, int l, int i, int j, int ax, int sd, double *p, double *f) {
  face_state(S, &S->lev[l], i, j, ax, sd, p, f);
}

/* ------------------------------------------------------------------ */
/* Interior numerical flux (reading: HLL form of P_M xi_n P_M).        */
/* Both face states are first projected into the cell basis pc         */
/* (eq. flux-force-expansion); the wave-speed bounds use C_{M+1}, the  */
/* largest |eigenvalue| of the regularized operator (eq. local-CFL).   */
/*   F = Xi a-                             if s_L >= 0                 */
/*   F = Xi a+                             else if s_R <= 0            */
/*   F = [s_R Xi a- - s_L Xi a+ + s_L s_R (a+ - a-)] / (s_R - s_L)      */
/* Parity with the paper's own flux: UNPINNED (formula not printed).   */
/* ------------------------------------------------------------------ */
void or_hll_flux(int M, double C, int ax, const double *pc, const double *pm, const double *fm,
                 const double *pp, const double *fp, double *F) {
  int n = or_nmom(M);
  double am[OR_MAXN], ap[OR_MAXN], xm[OR_MAXN], xp[OR_MAXN];
  or_transform(M, pm, pc, fm, am);
  or_transform(M, pp, pc, fp, ap);
  double sL = fmin(pm[ax] - C * sqrt(pm[3]), pp[ax] - C * sqrt(pp[3]));
  double sR = fmax(pm[ax] + C * sqrt(pm[3]), pp[ax] + C * sqrt(pp[3]));
  or_xi_mul(M, ax, pc, am, xm);
  or_xi_mul(M, ax, pc, ap, xp);
  if (sL >= 0.0) {
    memcpy(F, xm, n * sizeof(double));
  } else if (sR <= 0.0) {
    memcpy(F, xp, n * sizeof(double));
  } else {
    for (int o = 0; o < n; ++o) F[o] = (sR * xm[o] - sL * xp[o] + sL * sR * (ap[o] - am[o])) / (sR - sL);
  }
}

/* ------------------------------------------------------------------ */
/* Maxwell wall flux (reading of the paper's Maxwell boundary          */
/* condition; all walls of the paper are fully diffusive).  Wall w has */
/* axis n and outward sign s; its basis is [u_w, theta_w] (u_{w,n}=0).  */
/*  1. a = T(face -> wall) f_face;                                     */
/*  2. leaving particles (s xi_n > 0) carry f_face, entering ones carry */
/*     chi rho_w M_w + (1-chi) (f_face reflected in xi_n);              */
/*  3. in the wall basis, with v = xi_n / sqrt(theta_w),               */
/*     G_(k,a') = sum_m a_(m,a') theta_w^((k-m+1)/2)/k! *               */
/*                 [J^s_{k,m} + (1-chi)(-1)^m J^{-s}_{k,m}]             */
/*              + [a'=0] chi rho_w theta_w^((k+1)/2)/k! J^{-s}_{k,0};   */
/*  4. rho_w makes the mass flux G_0 vanish:                           */
/*     rho_w = s sqrt(2 pi) sum_m a_(m e_n) theta_w^(-m/2) J^s_{0,m};   */
/*  5. F = T(wall -> cell) G.                                          */
/* Parity with the paper's own boundary condition: UNPINNED.           */
/* ------------------------------------------------------------------ */
static const int wall_axis[4] = {1, 0, 1, 0};
static const int wall_sign[4] = {-1, +1, +1, -1};

void or_wall_flux(int M, const double *uw, double thw, double chi, int w, const double *pc,
                  const double *pf, const double *ff, double *F) {
  const basis_t *b = basis(M);
  int n = b->n, ax = wall_axis[w], s = wall_sign[w];
  double pw[4] = {uw[0], uw[1], uw[2], thw};
  double a[OR_MAXN], G[OR_MAXN];
  double Js[(OR_MAXM + 1) * (OR_MAXM + 1)], Jm[(OR_MAXM + 1) * (OR_MAXM + 1)];
  or_halfrange(M, s, Js);
  or_halfrange(M, -s, Jm);
  int K = M + 1;
  or_transform(M, pf, pw, ff, a);
  double rho_w = 0.0;
  for (int m = 0; m <= M; ++m) {
    int e[3] = {0, 0, 0};
    e[ax] = m;
    rho_w += a[idx3(b, e[0], e[1], e[2])] * pow(thw, -0.5 * m) * Js[0 * K + m];
  }
  rho_w = s * sqrt(2.0 * M_PI) * rho_w;
  for (int o = 0; o < n; ++o) {
    int k = b->a[o][ax];
    int perp[3] = {b->a[o][0], b->a[o][1], b->a[o][2]};
    perp[ax] = 0;
    int lp = perp[0] + perp[1] + perp[2];
    double g = 0.0;
    for (int m = 0; m <= M - lp; ++m) {
      int t[3] = {perp[0], perp[1], perp[2]};
      t[ax] = m;
      double sgn = (m % 2 == 0) ? 1.0 : -1.0;
      g += a[idx3(b, t[0], t[1], t[2])] * pow(thw, 0.5 * (k - m + 1)) / factorial(k) *
           (Js[k * K + m] + (1.0 - chi) * sgn * Jm[k * K + m]);
    }
    if (lp == 0) g += chi * rho_w * pow(thw, 0.5 * (k + 1)) / factorial(k) * Jm[k * K + 0];
    G[o] = g;
  }
  or_transform(M, pw, pc, G, F);
}

/* ------------------------------------------------------------------ */
/* Collision term (Sec. 2.1 and 2.3).  Q = nu (f^E - f) projected on   */
/* the cell's Grad basis; nu = beta sqrt(pi/2) rho theta^(1-w) / Kn    */
/* (eq. nu-shakhov).  BGK: f^E = rho H_0.  Shakhov (eq. Shakhov-f^E):  */
/* with v = (xi-u)/sqrt(theta), v_i(|v|^2-5) = He_3(v_i) +             */
/* sum_{d!=i} He_1(v_i) He_2(v_d), so f^E has coefficient              */
/* (1-Pr) q_i / 5 at 3e_i and at e_i + 2e_d (d != i), besides rho at 0. */
/* ES-BGK (eq. ES-f^E): f^E is the Gaussian of covariance Lambda.  In   */
/* the variable v the generating function sum_alpha He_alpha(v)        */
/* t^alpha / alpha! = exp(t.v - |t|^2/2) has, under that Gaussian, the */
/* mean exp(t^T (Lambda/theta - I) t / 2); with the coefficient        */
/* formula f_alpha = theta^{|alpha|/2}/alpha! int He_alpha(v) f dxi    */
/* this gives f^E_alpha = rho [s^alpha] exp(s^T B s / 2), where        */
/* B = Lambda - theta I = (1 - 1/Pr) sigma / rho and sigma_ij =        */
/* (1 + delta_ij) f_{e_i+e_j} (eq. moments-relation).  The exponential  */
/* is summed as its power series, truncated at degree M.               */
/* ------------------------------------------------------------------ */
static void esbgk_equilibrium(const basis_t *b, double Pr, const double *f, double *fE) {
  int n = b->n, M = b->M;
  double rho = f[0];
  /* q(s) = s^T B s / 2 as coefficients of the monomials s_i s_j, i <= j */
  double qc[3][3];
  for (int i = 0; i < 3; ++i)
    for (int j = i; j < 3; ++j) {
      int t[3] = {0, 0, 0};
      t[i] += 1;
      t[j] += 1;
      double sigma = (i == j ? 2.0 : 1.0) * f[idx3(b, t[0], t[1], t[2])];
      double Bij = (1.0 - 1.0 / Pr) * sigma / rho;
      qc[i][j] = (i == j) ? 0.5 * Bij : Bij;
    }
  double term[OR_MAXN], next[OR_MAXN];
  for (int o = 0; o < n; ++o) term[o] = fE[o] = 0.0;
  term[0] = 1.0;
  fE[0] = 1.0;
  /* term_k = q^k / k!, from term_{k-1} * q / k */
  for (int k = 1; 2 * k <= M; ++k) {
    for (int o = 0; o < n; ++o) {
      double acc = 0.0;
      for (int i = 0; i < 3; ++i)
        for (int j = i; j < 3; ++j) {
          int t[3] = {b->a[o][0], b->a[o][1], b->a[o][2]};
          t[i] -= 1;
          t[j] -= 1;
          int p = idx3(b, t[0], t[1], t[2]);
          if (p >= 0) acc += qc[i][j] * term[p];
        }
      next[o] = acc / k;
    }
    for (int o = 0; o < n; ++o) {
      term[o] = next[o];
      fE[o] += term[o];
    }
  }
  for (int o = 0; o < n; ++o) fE[o] *= rho;
}

void or_collision(int M, int model, double Kn, double Pr, double omega, double beta, const double *pc,
                  const double *f, double *Q) {
  const basis_t *b = basis(M);
  int n = b->n;
  double rho = f[0], th = pc[3];
  double nu = beta * sqrt(M_PI / 2.0) * rho * pow(th, 1.0 - omega) / Kn;
  double fE[OR_MAXN];
  for (int o = 0; o < n; ++o) fE[o] = 0.0;
  fE[0] = rho;
  if (model == OR_SHAKHOV) {
    for (int i = 0; i < 3; ++i) {
      int e[3] = {0, 0, 0};
      e[i] = 3;
      double q = 2.0 * f[idx3(b, e[0], e[1], e[2])];
      for (int d = 0; d < 3; ++d) {
        int t[3] = {0, 0, 0};
        t[d] += 2;
        t[i] += 1;
        q += f[idx3(b, t[0], t[1], t[2])];
      }
      fE[idx3(b, e[0], e[1], e[2])] = (1.0 - Pr) * q / 5.0;
      for (int d = 0; d < 3; ++d) {
        if (d == i) continue;
        int t[3] = {0, 0, 0};
        t[d] += 2;
        t[i] += 1;
        fE[idx3(b, t[0], t[1], t[2])] = (1.0 - Pr) * q / 5.0;
      }
    }
  } else if (model == OR_ESBGK) {
    esbgk_equilibrium(b, Pr, f, fE);
  }
  for (int o = 0; o < n; ++o) Q[o] = nu * (fE[o] - f[o]);
}

/* ------------------------------------------------------------------ */
/* R_ij(f) in the cell basis (eq. ode-system):                         */
/*   R = -(F_E - F_W)/dx - (F_N - F_S)/dy + Q                          */
/* ------------------------------------------------------------------ */
static void cell_R(const or_solver *S, const or_level *L, int i, int j, double *R) {
  const or_config *cf = &S->c;
  int n = S->n, M = cf->M;
  int c = j * L->nx + i;
  const double *pc = L->P + 4 * c, *fc = L->F + (size_t)c * n;
  double FE[OR_MAXN], FW[OR_MAXN], FN[OR_MAXN], FS[OR_MAXN], Q[OR_MAXN];
  double pm[4], pp[4], fm[OR_MAXN], fp[OR_MAXN];
  /* x faces */
  if (i == L->nx - 1) {
    face_state(S, L, i, j, 0, +1, pm, fm);
    or_wall_flux(M, cf->wall_u[1], cf->wall_theta[1], cf->wall_chi[1], 1, pc, pm, fm, FE);
  } else {
    face_state(S, L, i, j, 0, +1, pm, fm);
    face_state(S, L, i + 1, j, 0, -1, pp, fp);
    or_hll_flux(M, S->C, 0, pc, pm, fm, pp, fp, FE);
  }
  if (i == 0) {
    face_state(S, L, i, j, 0, -1, pp, fp);
    or_wall_flux(M, cf->wall_u[3], cf->wall_theta[3], cf->wall_chi[3], 3, pc, pp, fp, FW);
  } else {
    face_state(S, L, i - 1, j, 0, +1, pm, fm);
    face_state(S, L, i, j, 0, -1, pp, fp);
    or_hll_flux(M, S->C, 0, pc, pm, fm, pp, fp, FW);
  }
  /* y faces */
  if (j == L->ny - 1) {
    face_state(S, L, i, j, 1, +1, pm, fm);
    or_wall_flux(M, cf->wall_u[2], cf->wall_theta[2], cf->wall_chi[2], 2, pc, pm, fm, FN);
  } else {
    face_state(S, L, i, j, 1, +1, pm, fm);
    face_state(S, L, i, j + 1, 1, -1, pp, fp);
    or_hll_flux(M, S->C, 1, pc, pm, fm, pp, fp, FN);
  }
  if (j == 0) {
    face_state(S, L, i, j, 1, -1, pp, fp);
    or_wall_flux(M, cf->wall_u[0], cf->wall_theta[0], cf->wall_chi[0], 0, pc, pp, fp, FS);
  } else {
    face_state(S, L, i, j - 1, 1, +1, pm, fm);
    face_state(S, L, i, j, 1, -1, pp, fp);
    or_hll_flux(M, S->C, 1, pc, pm, fm, pp, fp, FS);
  }
  or_collision(M, cf->model, cf->Kn, cf->Pr, cf->omega, cf->beta, pc, fc, Q);
  for (int o = 0; o < n; ++o) R[o] = -(FE[o] - FW[o]) / L->hx[i] - (FN[o] - FS[o]) / L->hy[j] + Q[o];
}

/* r of level L in the basis pc (zero when the level has no r) */
static void rhs_in(const or_solver *S, const or_level *L, int c, const double *pc, double *r) {
  if (!L->has_r) {
    for (int o = 0; o < S->n; ++o) r[o] = 0.0;
    return;
  }
  or_transform(S->c.M, L->rP + 4 * c, pc, L->rF + (size_t)c * S->n, r);
}

/* ------------------------------------------------------------------ */
/* Back to Grad form (Sec. 2.4, two-step update): compute u, theta of  */
/* g (basis p) by the general-basis macroscopics, project g into       */
/* F_M^[u,theta], then set f_{e_d} := 0 and remove the round-off mean  */
/* of f_{2e_d}, both zero in exact arithmetic.                         */
/* ------------------------------------------------------------------ */
static int regrad(const or_solver *S, const double *p, const double *g, double *pn, double *fn) {
  const basis_t *b = basis(S->c.M);
  double mac[5];
  or_macros(S->c.M, p, g, mac);
  pn[0] = mac[1];
  pn[1] = mac[2];
  pn[2] = mac[3];
  pn[3] = mac[4];
  or_transform(S->c.M, p, pn, g, fn);
  fn[idx3(b, 1, 0, 0)] = 0.0;
  fn[idx3(b, 0, 1, 0)] = 0.0;
  fn[idx3(b, 0, 0, 1)] = 0.0;
  int i1 = idx3(b, 2, 0, 0), i2 = idx3(b, 0, 2, 0), i3 = idx3(b, 0, 0, 2);
  double s3 = (fn[i1] + fn[i2] + fn[i3]) / 3.0;
  fn[i1] -= s3;
  fn[i2] -= s3;
  fn[i3] -= s3;
  int ok = isfinite(mac[0]) && isfinite(mac[4]) && mac[0] > 0.0 && mac[4] > 0.0;
  for (int o = 0; o < S->n && ok; ++o) ok = isfinite(fn[o]);
  return ok ? OR_OK : OR_ERR_NONPHYSICAL;
}

/* ------------------------------------------------------------------ */
/* One Gauss-Seidel cell update of Algorithm 1:                        */
/*   dt from eq. (local-CFL) with the current state, CFL number cfl;   */
/*   optionally capped at dtnu / nu (reading for small Kn, where the    */
/*   explicit collision step nu dt would exceed its stability bound;    */
/*   the cap changes the iteration, not its fixed point);               */
/*   f <- f + dt (R_ij(f) - r_ij), then back to Grad form.             */
/* ------------------------------------------------------------------ */
static double local_dt(const or_solver *S, const or_level *L, int c) {
  const double *pc = L->P + 4 * c, *fc = L->F + (size_t)c * S->n;
  double sq = sqrt(pc[3]);
  double dt = S->c.cfl / ((fabs(pc[0]) + S->C * sq) / L->hx[c % L->nx] + (fabs(pc[1]) + S->C * sq) / L->hy[c / L->nx]);
  if (S->c.dtnu > 0.0) {
    double nu = S->c.beta * sqrt(M_PI / 2.0) * fc[0] * pow(pc[3], 1.0 - S->c.omega) / S->c.Kn;
    dt = fmin(dt, S->c.dtnu / nu);
  }
  return dt;
}

static int cell_update(or_solver *S, or_level *L, int i, int j) {
  int n = S->n, c = j * L->nx + i;
  double *pc = L->P + 4 * c, *fc = L->F + (size_t)c * n;
  double R[OR_MAXN], r[OR_MAXN], g[OR_MAXN], pn[4], fn[OR_MAXN];
  double dt = local_dt(S, L, c);
  cell_R(S, L, i, j, R);
  rhs_in(S, L, c, pc, r);
  for (int o = 0; o < n; ++o) g[o] = fc[o] + dt * (R[o] - r[o]);
  int st = regrad(S, pc, g, pn, fn);
  memcpy(pc, pn, 4 * sizeof(double));
  memcpy(fc, fn, n * sizeof(double));
  return st;
}

/* Directional sweep Dk, k = 1..4 (Sec. 3.1): the outer loop runs over  */
/* i, the inner over j, ascending or descending as listed there.       */
/* OpenMP mode of the sweep: the cells of Dk taken by anti-diagonals ii + jj = d of the    */
/* sweep's own index order, the cells of one diagonal in parallel.  The stencil of R_ij is */
/* a cross (no diagonal neighbours), so a neighbour on a smaller diagonal is one the       */
/* serial order visits earlier and one on a larger diagonal one it visits later: every      */
/* cell reads exactly the values the serial sweep gives it, and the result is the same    */
/* bit for bit.                                                                             */
static int sweep_by_diagonals(or_solver *S, int l, int k) {
  or_level *L = &S->lev[l];
  int idesc = (k == 2 || k == 3), jdesc = (k == 3 || k == 4);
  int st = OR_OK;
  for (int d = 0; d <= L->nx + L->ny - 2; ++d) {
    int lo = d - (L->ny - 1) > 0 ? d - (L->ny - 1) : 0;
    int hi = d < L->nx - 1 ? d : L->nx - 1;
#pragma omp parallel for num_threads(S->threads) schedule(dynamic, 1)
    for (int ii = lo; ii <= hi; ++ii) {
      int jj = d - ii;
      int i = idesc ? L->nx - 1 - ii : ii;
      int j = jdesc ? L->ny - 1 - jj : jj;
      int s = cell_update(S, L, i, j);
      if (s != OR_OK) {
#pragma omp atomic write
        st = s;
      }
    }
  }
  return st;
}

int or_sweep(or_solver *S, int l, int k) {
  if (S->threads > 1) return sweep_by_diagonals(S, l, k);
  or_level *L = &S->lev[l];
  int idesc = (k == 2 || k == 3), jdesc = (k == 3 || k == 4);
  int st = OR_OK;
  for (int ii = 0; ii < L->nx; ++ii) {
    int i = idesc ? L->nx - 1 - ii : ii;
    for (int jj = 0; jj < L->ny; ++jj) {
      int j = jdesc ? L->ny - 1 - jj : jj;
      int s = cell_update(S, L, i, j);
      if (s != OR_OK) st = s;
    }
  }
  return st;
}

/* steps applications of FS(f, r) (Algorithm 1) on level l */
int or_smooth(or_solver *S, int l, int steps) {
  int st = OR_OK;
  for (int s = 0; s < steps; ++s)
    for (int k = 1; k <= 4; ++k) {
      int e = or_sweep(S, l, k);
      if (e != OR_OK) st = e;
    }
  return st;
}

/* ------------------------------------------------------------------ */
/* Forward Euler (Sec. 2.4, eq. euler-scheme): every cell advances     */
/* from the same old state f^n, with one step for the whole level: the */
/* smallest local step of eq. (local-CFL) (eq. global-CFL; with the    */
/* dtnu cap when it is set); then each cell returns to Grad form.      */
/* ------------------------------------------------------------------ */
int or_euler(or_solver *S, int l, int steps) {
  or_level *L = &S->lev[l];
  int n = S->n, nc = L->nx * L->ny, st = OR_OK;
  double *G = (double *)malloc(sizeof(double) * (size_t)nc * n);
  double R[OR_MAXN], r[OR_MAXN], pn[4], fn[OR_MAXN];
  for (int s = 0; s < steps; ++s) {
    double dt = INFINITY;
    for (int c = 0; c < nc; ++c) dt = fmin(dt, local_dt(S, L, c));
    for (int j = 0; j < L->ny; ++j)
      for (int i = 0; i < L->nx; ++i) {
        int c = j * L->nx + i;
        cell_R(S, L, i, j, R);
        rhs_in(S, L, c, L->P + 4 * c, r);
        for (int o = 0; o < n; ++o) G[(size_t)c * n + o] = L->F[(size_t)c * n + o] + dt * (R[o] - r[o]);
      }
    for (int c = 0; c < nc; ++c) {
      int e = regrad(S, L->P + 4 * c, G + (size_t)c * n, pn, fn);
      if (e != OR_OK) st = e;
      memcpy(L->P + 4 * c, pn, 4 * sizeof(double));
      memcpy(L->F + (size_t)c * n, fn, n * sizeof(double));
    }
  }
  free(G);
  return st;
}

/* R_ij(f) - r_ij of every cell (cell basis) and the norm of           */
/* eq. (relative-residual): ||R||^2 = 1/(LxLy) sum_ij ||R_ij||^2 ds,   */
/* ||R_ij||^2 = sum_alpha alpha! theta^-|alpha| R_alpha^2.             */
static double local_norm2(const or_solver *S, const double *pc, const double *R) {
  const basis_t *b = basis(S->c.M);
  double s = 0.0;
  for (int o = 0; o < S->n; ++o) {
    int a1 = b->a[o][0], a2 = b->a[o][1], a3 = b->a[o][2];
    double w = factorial(a1) * factorial(a2) * factorial(a3) * pow(pc[3], -(double)(a1 + a2 + a3));
    s += w * R[o] * R[o];
  }
  return s;
}

void or_cell_residual(const or_solver *S, int l, int i, int j, double *out) {
  const or_level *L = &S->lev[l];
  int c = j * L->nx + i;
  double R[OR_MAXN], r[OR_MAXN];
  cell_R(S, L, i, j, R);
  rhs_in(S, L, c, L->P + 4 * c, r);
  for (int o = 0; o < S->n; ++o) out[o] = R[o] - r[o];
}

double or_residual(const or_solver *S, int l, double *Rout) {
  const or_level *L = &S->lev[l];
  double R[OR_MAXN];
  double acc = 0.0;
  if (S->threads > 1) {
    /* OpenMP mode: the cells' terms in parallel, summed in the serial order */
    int nc = L->nx * L->ny;
    double *term = (double *)malloc(sizeof(double) * (size_t)nc);
#pragma omp parallel for num_threads(S->threads) schedule(dynamic, 4)
    for (int c = 0; c < nc; ++c) {
      double Rc[OR_MAXN];
      or_cell_residual(S, l, c % L->nx, c / L->nx, Rc);
      if (Rout) memcpy(Rout + (size_t)c * S->n, Rc, S->n * sizeof(double));
      term[c] = local_norm2(S, L->P + 4 * c, Rc) * L->hx[c % L->nx] * L->hy[c / L->nx];
    }
    for (int c = 0; c < nc; ++c) acc += term[c];
    free(term);
    return sqrt(acc / (S->c.lx * S->c.ly));
  }
  for (int j = 0; j < L->ny; ++j)
    for (int i = 0; i < L->nx; ++i) {
      int c = j * L->nx + i;
      or_cell_residual(S, l, i, j, R);
      if (Rout) memcpy(Rout + (size_t)c * S->n, R, S->n * sizeof(double));
      acc += local_norm2(S, L->P + 4 * c, R) * L->hx[i] * L->hy[j];
    }
  return sqrt(acc / (S->c.lx * S->c.ly));
}

/* ------------------------------------------------------------------ */
/* Restriction (Sec. 3.2.2).  Coarse cell (I,J) merges the fine cells   */
/* (2I,2J), (2I+1,2J), (2I,2J+1), (2I+1,2J+1) (taken in that order).   */
/* (u_H, theta_H) from conservation of mass, momentum and energy       */
/* (eq. uH-thetaH-computation); f_H and R_H are the area means of the  */
/* fine functions projected into F_M^[u_H,theta_H] (eq. fH).  The fine  */
/* areas are a quarter of the coarse area.                            */
/* ------------------------------------------------------------------ */
static void restrict_level(or_solver *S, int lf) {
  or_level *Lf = &S->lev[lf], *Lc = &S->lev[lf - 1];
  const basis_t *b = basis(S->c.M);
  int n = S->n;
#pragma omp parallel for num_threads(S->threads) if (S->threads > 1) schedule(dynamic, 1)
  for (int J = 0; J < Lc->ny; ++J)
    for (int I = 0; I < Lc->nx; ++I) {
      double tf[OR_MAXN], tr[OR_MAXN];
      int C = J * Lc->nx + I;
      int fi[4] = {(2 * J) * Lf->nx + 2 * I, (2 * J) * Lf->nx + 2 * I + 1, (2 * J + 1) * Lf->nx + 2 * I,
                   (2 * J + 1) * Lf->nx + 2 * I + 1};
      /* area weights of the children (equal areas: the plain mean, as 1 each and 1/4 at the end) */
      double wq[4];
      for (int q = 0; q < 4; ++q)
        wq[q] = Lf->uniform ? 1.0
                            : Lf->hx[fi[q] % Lf->nx] * Lf->hy[fi[q] / Lf->nx] / (Lc->hx[I] * Lc->hy[J]);
      const double mean = Lf->uniform ? 0.25 : 1.0;
      double rho = 0.0, mom[3] = {0, 0, 0}, en = 0.0;
      for (int q = 0; q < 4; ++q) {
        const double *p = Lf->P + 4 * fi[q];
        double r = wq[q] * Lf->F[(size_t)fi[q] * n];
        rho += r;
        for (int d = 0; d < 3; ++d) mom[d] += r * p[d];
        en += r * (p[0] * p[0] + p[1] * p[1] + p[2] * p[2]) + 3.0 * r * p[3];
      }
      rho *= mean;
      for (int d = 0; d < 3; ++d) mom[d] *= mean;
      en *= mean;
      double pH[4];
      for (int d = 0; d < 3; ++d) pH[d] = mom[d] / rho;
      pH[3] = (en - rho * (pH[0] * pH[0] + pH[1] * pH[1] + pH[2] * pH[2])) / (3.0 * rho);
      double *fH = Lc->F + (size_t)C * n, *RH = Lc->rF + (size_t)C * n;
      for (int o = 0; o < n; ++o) {
        fH[o] = 0.0;
        RH[o] = 0.0;
      }
      for (int q = 0; q < 4; ++q) {
        or_transform(S->c.M, Lf->P + 4 * fi[q], pH, Lf->F + (size_t)fi[q] * n, tf);
        or_transform(S->c.M, Lf->P + 4 * fi[q], pH, Lf->D + (size_t)fi[q] * n, tr);
        for (int o = 0; o < n; ++o) {
          fH[o] += wq[q] * tf[o];
          RH[o] += wq[q] * tr[o];
        }
      }
      for (int o = 0; o < n; ++o) {
        fH[o] *= mean;
        RH[o] *= mean;
      }
      /* f_H is in Grad form up to round-off; make it exact */
      fH[idx3(b, 1, 0, 0)] = 0.0;
      fH[idx3(b, 0, 1, 0)] = 0.0;
      fH[idx3(b, 0, 0, 1)] = 0.0;
      int i1 = idx3(b, 2, 0, 0), i2 = idx3(b, 0, 2, 0), i3 = idx3(b, 0, 0, 2);
      double s3 = (fH[i1] + fH[i2] + fH[i3]) / 3.0;
      fH[i1] -= s3;
      fH[i2] -= s3;
      fH[i3] -= s3;
      memcpy(Lc->P + 4 * C, pH, 4 * sizeof(double));
      memcpy(Lc->rP + 4 * C, pH, 4 * sizeof(double));
      memcpy(Lc->bP + 4 * C, pH, 4 * sizeof(double));
      memcpy(Lc->bF + (size_t)C * n, fH, n * sizeof(double));
    }
}

/* ------------------------------------------------------------------ */
/* Coarse-grid correction with identity prolongation                  */
/* (eq. rewritten-update): f^_h = f_h - f_H(restricted) + f~_H, every   */
/* term projected into the fine cell's basis, then back to Grad form.  */
/* ------------------------------------------------------------------ */
static int prolong_update(or_solver *S, int lf) {
  or_level *Lf = &S->lev[lf], *Lc = &S->lev[lf - 1];
  int n = S->n, st = OR_OK;
#pragma omp parallel for num_threads(S->threads) if (S->threads > 1) schedule(dynamic, 1)
  for (int j = 0; j < Lf->ny; ++j)
    for (int i = 0; i < Lf->nx; ++i) {
      double tb[OR_MAXN], tt[OR_MAXN], g[OR_MAXN], pn[4], fn[OR_MAXN];
      int c = j * Lf->nx + i, C = (j / 2) * Lc->nx + i / 2;
      double *pc = Lf->P + 4 * c, *fc = Lf->F + (size_t)c * n;
      or_transform(S->c.M, Lc->bP + 4 * C, pc, Lc->bF + (size_t)C * n, tb);
      or_transform(S->c.M, Lc->P + 4 * C, pc, Lc->F + (size_t)C * n, tt);
      for (int o = 0; o < n; ++o) g[o] = (fc[o] - tb[o]) + tt[o];
      int s = regrad(S, pc, g, pn, fn);
      if (s != OR_OK) {
#pragma omp atomic write
        st = s;
      }
      memcpy(pc, pn, 4 * sizeof(double));
      memcpy(fc, fn, n * sizeof(double));
    }
  return st;
}

/* ------------------------------------------------------------------ */
/* The coarse problem of Algorithm 2 built from fine level lf:         */
/*   R_bar_h = r_h - R_h(f_bar_h) in each fine cell's basis (the       */
/*   defect; eq. coarse-grid-problem with r_h projected in);           */
/*   f_bar_H = I f_bar_h and R_bar_H = I R_bar_h (restriction);        */
/*   r_H = R_H(f_bar_H) + R_bar_H, in the basis of f_bar_H.            */
/* ------------------------------------------------------------------ */
static void two_grid_setup(or_solver *S, int lf) {
  or_level *Lf = &S->lev[lf], *Lc = &S->lev[lf - 1];
#pragma omp parallel for num_threads(S->threads) if (S->threads > 1) schedule(dynamic, 1)
  for (int j = 0; j < Lf->ny; ++j)
    for (int i = 0; i < Lf->nx; ++i) {
      double R[OR_MAXN];
      or_cell_residual(S, lf, i, j, R);
      for (int o = 0; o < S->n; ++o) Lf->D[(size_t)(j * Lf->nx + i) * S->n + o] = -R[o];
    }
  /* f_bar_H = I f_bar, R_bar_H = I R_bar (stored in rF for now) */
  restrict_level(S, lf);
  Lc->has_r = 0;
#pragma omp parallel for num_threads(S->threads) if (S->threads > 1) schedule(dynamic, 1)
  for (int j = 0; j < Lc->ny; ++j)
    for (int i = 0; i < Lc->nx; ++i) {
      double R[OR_MAXN];
      int c = j * Lc->nx + i;
      cell_R(S, Lc, i, j, R);
      for (int o = 0; o < S->n; ++o) Lc->D[(size_t)c * S->n + o] = R[o];
    }
  for (size_t q = 0; q < (size_t)Lc->nx * Lc->ny * S->n; ++q) Lc->rF[q] = Lc->D[q] + Lc->rF[q];
  Lc->has_r = 1;
}

/* ------------------------------------------------------------------ */
/* Algorithm 2: one step of the (k+1)-level NMG iteration on level k.  */
/* ------------------------------------------------------------------ */
static int nmg(or_solver *S, int k) {
  const or_config *cf = &S->c;
  if (k == 0) return or_smooth(S, 0, cf->s3); /* coarsest solver: s3 FS steps */
  int st = or_smooth(S, k, cf->s1);           /* pre-smoothing */
  two_grid_setup(S, k);                        /* f_bar_H, R_bar_H and r_H */
  for (int g = 0; g < cf->gamma; ++g) {
    int e = nmg(S, k - 1);
    if (e != OR_OK) st = e;
  }
  int e = prolong_update(S, k);
  if (e != OR_OK) st = e;
  e = or_smooth(S, k, cf->s2); /* post-smoothing */
  if (e != OR_OK) st = e;
  return st;
}

/* The correction applied after each NMG step (reading): rescale every  */
/* coefficient of the finest level so that the total mass returns to   */
/* its reference value; u and theta are unchanged.  Parity UNPINNED.    */
void or_mass_correct(or_solver *S) {
  int l = S->c.levels - 1;
  or_level *L = &S->lev[l];
  double sc = S->m0 / total_mass(S, l);
  for (size_t q = 0; q < (size_t)L->nx * L->ny * S->n; ++q) L->F[q] *= sc;
}

/* one NMG_K(f, 0) step plus the mass correction; returns the relative  */
/* residual of eq. (relative-residual) in *rel                          */
int or_fas_cycle(or_solver *S, double *rel) {
  int K = S->c.levels - 1;
  if (!S->have_res0) {
    S->res0 = or_residual(S, K, NULL);
    S->have_res0 = 1;
  }
  S->lev[K].has_r = 0;
  int st = nmg(S, K);
  or_mass_correct(S);
  double r = or_residual(S, K, NULL);
  if (rel) *rel = S->res0 > 0.0 ? r / S->res0 : 0.0;
  return st;
}

int or_solve(or_solver *S, double tol, int max_cycles, int *cycles, double *rel) {
  int K = S->c.levels - 1;
  S->lev[K].has_r = 0;
  S->res0 = or_residual(S, K, NULL);
  S->have_res0 = 1;
  double rr = S->res0 > 0.0 ? 1.0 : 0.0;
  int it = 0, st = OR_OK;
  while (rr > tol && it < max_cycles) {
    st = or_fas_cycle(S, &rr);
    ++it;
    if (st != OR_OK) break;
  }
  if (cycles) *cycles = it;
  if (rel) *rel = rr;
  if (st == OR_OK && rr > tol) st = OR_ERR_NOT_CONVERGED;
  return st;
}

double or_res0(const or_solver *S) { return S->res0; }

/* fields of the finest level: [cell][14] */
void or_fields(const or_solver *S, double *out) {
  const or_level *L = &S->lev[S->c.levels - 1];
  for (int c = 0; c < L->nx * L->ny; ++c) or_cell_fields(S->c.M, L->P + 4 * c, L->F + (size_t)c * S->n, out + 14 * c);
}

/* expose the restriction / coarse right-hand side / update for tests:  */
/* builds level lf-1 from level lf exactly as Algorithm 2 does          */
int or_two_grid_setup(or_solver *S, int lf) {
  two_grid_setup(S, lf);
  return OR_OK;
}

int or_two_grid_update(or_solver *S, int lf) { return prolong_update(S, lf); }

/* restricted state saved for the update (level l = coarse level) */
void or_get_saved(const or_solver *S, int l, double *P, double *F) {
  const or_level *L = &S->lev[l];
  size_t nc = (size_t)L->nx * L->ny;
  memcpy(P, L->bP, nc * 4 * sizeof(double));
  memcpy(F, L->bF, nc * S->n * sizeof(double));
}
