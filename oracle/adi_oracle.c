/*
 * adi_oracle.c -- plain FP64 CPU oracle for the Peaceman-Rachford ADI step of the two
 * 2-D acoustic schemes of Otero, Rojas, Moya and Castillo (arXiv 2006.07583):
 *   - CFD: fourth-order compact differences on the nodal mesh (Sec. 2.1, App. A),
 *   - MFD: fourth-order mimetic D/G operators on the staggered mesh (Sec. 2.2, App. B).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path may include, link, call or run
 * this file; only tests/, __graft_entry__.smoke() and bench.py's cpu_baseline leg (and its
 * --impl reference arm) use it.  It shares no code, header, table or helper with the CUDA
 * path.
 *
 * What it computes.  One time step is the Peaceman-Rachford split of the Crank-Nicolson
 * system (Eq. 5): stage 1 (Eq. 6) is implicit along x-lines, stage 2 (Eq. 7) along
 * y-lines, with the x/y operators A1h, A2h of Eq. 4 (CFD) or Eq. 12 (MFD).  Material
 * scaling is applied pointwise after differentiation, as the pseudo-code of Algorithms
 * 3/4 does (K.*, R.*).  Each stage's coupled line system (Eq. 8 / Eq. 10) is solved
 * EXACTLY -- the fixed point that the paper's iteration (Eq. 9) approaches -- by banded
 * Gaussian elimination with partial pivoting on the plain definition
 *     u_bar + alpha .* e = a,        e = Dv v      (CFD: Pbar e = Qbar v ; MFD: e = D v)
 *     v     + beta  .* g = v^m,      g = Du u      (CFD: P g = Q u       ; MFD: g = G u)
 * where u is the whole line including its Dirichlet end values.  An optional mode runs
 * the paper's own fixed-point iteration (Eq. 9, Algorithms 3-4) instead.
 *
 * Readings of the paper (each also listed in the design notes):
 *   - reduced CFD operators are (N-1)x(N-1) and (N-1)x(N+1) (App. A prints N-2);
 *   - mimetic D and G carry a 1/h factor and their last rows mirror the first rows with
 *     a sign change (App. B prints only the leading rows, without 1/h);
 *   - explicit y/x derivatives of pressure act on the whole line including its boundary
 *     values (Alg. 1/2 print reduced index sets there);
 *   - rho = 1, kappa = c^2, so alpha = dt/2 * kappa and beta = dt/2;
 *   - Dirichlet data are time independent (u* keeps them), except in the time-harmonic
 *     mode of the manufactured problem (Eq. 11), where u* on the x-line ends takes the
 *     wall value at the half step t_m + dt/2.
 *
 * Array layouts (row-major, i = y index, j = x index):
 *   CFD: U, V, W, kappa are (ny+1) x (nx+1) nodal arrays.
 *   MFD: U, kappa are (ny+2) x (nx+2) (cell centres plus edges), V is (ny+2) x (nx+1),
 *        W is (ny+1) x (nx+2).
 * Parity status: every function here is pinned by a test (operator exactness on
 * polynomials, dense LU, the dense 2-D Kronecker step, time reversal, the exact standing
 * wave and its convergence rate).
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

enum { OR_CFD = 0, OR_MFD = 1 };

/* ------------------------------------------------------------------------------------ */
/* 1-D operators as dense row-major matrices.                                            */
/* ------------------------------------------------------------------------------------ */

/* CFD P4 ((N+1)x(N+1)), App. A: boundary rows (6, 18) / (18, 6), interior (1, 4, 1). */
static void cfd_P(int N, double *P) {
    int n = N + 1;
    memset(P, 0, sizeof(double) * n * n);
    P[0 * n + 0] = 6.0;  P[0 * n + 1] = 18.0;
    for (int i = 1; i < N; ++i) {
        P[i * n + i - 1] = 1.0; P[i * n + i] = 4.0; P[i * n + i + 1] = 1.0;
    }
    P[N * n + N - 1] = 18.0; P[N * n + N] = 6.0;
}

/* CFD Q4 ((N+1)x(N+1)), App. A, with its 1/h: (-17, 9, 9, -1), interior (-3, 0, 3),
 * last row (1, -9, -9, 17). */
static void cfd_Q(int N, double h, double *Q) {
    int n = N + 1;
    memset(Q, 0, sizeof(double) * n * n);
    Q[0] = -17.0 / h; Q[1] = 9.0 / h; Q[2] = 9.0 / h; Q[3] = -1.0 / h;
    for (int i = 1; i < N; ++i) { Q[i * n + i - 1] = -3.0 / h; Q[i * n + i + 1] = 3.0 / h; }
    Q[N * n + N - 3] = 1.0 / h; Q[N * n + N - 2] = -9.0 / h;
    Q[N * n + N - 1] = -9.0 / h; Q[N * n + N] = 17.0 / h;
}

/* Reduced CFD Pbar4 ((N-1)x(N-1)), App. A: rows (6, 6), (1, 4, 1), (6, 6).
 * Row r corresponds to interior node r+1. */
static void cfd_Pbar(int N, double *P) {
    int n = N - 1;
    memset(P, 0, sizeof(double) * n * n);
    P[0] = 6.0; P[1] = 6.0;
    for (int r = 1; r < n - 1; ++r) {
        P[r * n + r - 1] = 1.0; P[r * n + r] = 4.0; P[r * n + r + 1] = 1.0;
    }
    P[(n - 1) * n + n - 2] = 6.0; P[(n - 1) * n + n - 1] = 6.0;
}

/* Reduced CFD Qbar4 ((N-1)x(N+1)), App. A, with 1/h: first row (-1, -9, 9, 1) on nodes
 * 0..3, interior (-3, 0, 3) around the node, last row (-1, -9, 9, 1) on nodes N-3..N. */
static void cfd_Qbar(int N, double h, double *Q) {
    int n = N - 1, m = N + 1;
    memset(Q, 0, sizeof(double) * n * m);
    Q[0] = -1.0 / h; Q[1] = -9.0 / h; Q[2] = 9.0 / h; Q[3] = 1.0 / h;
    for (int r = 1; r < n - 1; ++r) {
        int node = r + 1;
        Q[r * m + node - 1] = -3.0 / h; Q[r * m + node + 1] = 3.0 / h;
    }
    Q[(n - 1) * m + N - 3] = -1.0 / h; Q[(n - 1) * m + N - 2] = -9.0 / h;
    Q[(n - 1) * m + N - 1] = 9.0 / h;  Q[(n - 1) * m + N] = 1.0 / h;
}

/* Mimetic D4 (N x (N+1)), App. B, with 1/h.  Row 0 as printed, interior rows
 * (1/24, -9/8, 9/8, -1/24) on nodes r-1..r+2, last row the sign-flipped mirror. */
static void mfd_D(int N, double h, double *D) {
    int m = N + 1;
    static const double r0[6] = {-4751.0 / 5192.0, 909.0 / 1298.0, 6091.0 / 15576.0,
                                 -1165.0 / 5192.0, 129.0 / 2596.0, -25.0 / 15576.0};
    memset(D, 0, sizeof(double) * N * m);
    for (int c = 0; c < 6; ++c) D[c] = r0[c] / h;
    for (int r = 1; r < N - 1; ++r) {
        D[r * m + r - 1] = (1.0 / 24.0) / h;  D[r * m + r] = (-9.0 / 8.0) / h;
        D[r * m + r + 1] = (9.0 / 8.0) / h;   D[r * m + r + 2] = (-1.0 / 24.0) / h;
    }
    for (int c = 0; c < 6; ++c) D[(N - 1) * m + (N - c)] = -r0[c] / h;
}

/* Mimetic G4 ((N+1) x (N+2)), App. B, with 1/h.  Rows 0 and 1 as printed, interior rows
 * (1/24, -9/8, 9/8, -1/24) on entries j-1..j+2, last two rows the sign-flipped mirror. */
static void mfd_G(int N, double h, double *G) {
    int m = N + 2;
    static const double r0[6] = {-47888.0 / 14245.0, 1790.0 / 407.0, -14545.0 / 9768.0,
                                 8997.0 / 16280.0, -2335.0 / 22792.0, 25.0 / 9768.0};
    static const double r1[5] = {16.0 / 105.0, -31.0 / 24.0, 29.0 / 24.0, -3.0 / 40.0,
                                 1.0 / 168.0};
    memset(G, 0, sizeof(double) * (N + 1) * m);
    for (int c = 0; c < 6; ++c) G[c] = r0[c] / h;
    for (int c = 0; c < 5; ++c) G[m + c] = r1[c] / h;
    for (int j = 2; j < N - 1; ++j) {
        G[j * m + j - 1] = (1.0 / 24.0) / h;  G[j * m + j] = (-9.0 / 8.0) / h;
        G[j * m + j + 1] = (9.0 / 8.0) / h;   G[j * m + j + 2] = (-1.0 / 24.0) / h;
    }
    for (int c = 0; c < 6; ++c) G[N * m + (N + 1 - c)] = -r0[c] / h;
    for (int c = 0; c < 5; ++c) G[(N - 1) * m + (N + 1 - c)] = -r1[c] / h;
}

/* Exported for the operator tests: which = 0 P, 1 Q, 2 Pbar, 3 Qbar, 4 D, 5 G. */
int oracle_operator(int which, int N, double h, double *out) {
    if (N < 8) return -1;
    switch (which) {
    case 0: cfd_P(N, out); return 0;
    case 1: cfd_Q(N, h, out); return 0;
    case 2: cfd_Pbar(N, out); return 0;
    case 3: cfd_Qbar(N, h, out); return 0;
    case 4: mfd_D(N, h, out); return 0;
    case 5: mfd_G(N, h, out); return 0;
    }
    return -1;
}

/* ------------------------------------------------------------------------------------ */
/* Banded Gaussian elimination with partial pivoting (the textbook LAPACK gbsv scheme). */
/* Element (i, j) lives at ab[(kl + ku + i - j) + j * ld], ld = 2*kl + ku + 1.           */
/* ------------------------------------------------------------------------------------ */

typedef struct {
    int n, kl, ku, ld;
    double *ab;
} band_t;

static void band_init(band_t *b, int n, int kl, int ku) {
    b->n = n; b->kl = kl; b->ku = ku; b->ld = 2 * kl + ku + 1;
    b->ab = (double *)calloc((size_t)b->ld * n, sizeof(double));
}
static void band_free(band_t *b) { free(b->ab); b->ab = NULL; }
static double *band_at(band_t *b, int i, int j) {
    return &b->ab[(b->kl + b->ku + i - j) + (size_t)j * b->ld];
}

/* Solves A x = rhs in place (rhs becomes x).  Returns 0, or -1 for an exactly singular
 * pivot. */
static int band_solve(band_t *b, double *rhs) {
    int n = b->n, kl = b->kl, ku = b->ku;
    int kv = ku + kl; /* upper bandwidth after fill-in */
    int *piv = (int *)malloc(sizeof(int) * n);
    for (int j = 0; j < n; ++j) {
        int last = j + kl < n - 1 ? j + kl : n - 1;
        int p = j;
        double best = fabs(*band_at(b, j, j));
        for (int i = j + 1; i <= last; ++i) {
            double v = fabs(*band_at(b, i, j));
            if (v > best) { best = v; p = i; }
        }
        piv[j] = p;
        if (best == 0.0) { free(piv); return -1; }
        int cmax = j + kv < n - 1 ? j + kv : n - 1;
        if (p != j) {
            for (int c = j; c <= cmax; ++c) {
                double t = *band_at(b, j, c);
                *band_at(b, j, c) = *band_at(b, p, c);
                *band_at(b, p, c) = t;
            }
            double t = rhs[j]; rhs[j] = rhs[p]; rhs[p] = t;
        }
        double d = *band_at(b, j, j);
        for (int i = j + 1; i <= last; ++i) {
            double l = *band_at(b, i, j) / d;
            if (l == 0.0) continue;
            *band_at(b, i, j) = l;
            for (int c = j + 1; c <= cmax; ++c) *band_at(b, i, c) -= l * *band_at(b, j, c);
            rhs[i] -= l * rhs[j];
        }
    }
    for (int i = n - 1; i >= 0; --i) {
        int cmax = i + kv < n - 1 ? i + kv : n - 1;
        double s = rhs[i];
        for (int c = i + 1; c <= cmax; ++c) s -= *band_at(b, i, c) * rhs[c];
        rhs[i] = s / *band_at(b, i, i);
    }
    free(piv);
    return 0;
}

/* Tridiagonal-or-wider square solve L x = rhs for a dense operator matrix with a known
 * band, used for the explicit derivatives (P e = Q u along a line). */
static int dense_band_solve(const double *L, int n, double *rhs) {
    int kl = 0, ku = 0;
    for (int i = 0; i < n; ++i)
        for (int j = 0; j < n; ++j)
            if (L[(size_t)i * n + j] != 0.0) {
                if (i - j > kl) kl = i - j;
                if (j - i > ku) ku = j - i;
            }
    band_t b;
    band_init(&b, n, kl, ku);
    for (int i = 0; i < n; ++i)
        for (int j = 0; j < n; ++j)
            if (L[(size_t)i * n + j] != 0.0) *band_at(&b, i, j) = L[(size_t)i * n + j];
    int rc = band_solve(&b, rhs);
    band_free(&b);
    return rc;
}

/* ------------------------------------------------------------------------------------ */
/* Per-method operator set along one line of N cells.                                    */
/* ------------------------------------------------------------------------------------ */

typedef struct {
    int method, N;
    int np;  /* interior pressure unknowns on a line: CFD N-1, MFD N */
    int nv;  /* velocity points on a line: N+1 */
    int nu;  /* full pressure line including both ends: CFD N+1, MFD N+2 */
    double *Le, *Re; /* e-equation: Le e = Re v   (Le: np x np, Re: np x nv) */
    double *Lg, *Rg; /* g-equation: Lg g = Rg u   (Lg: nv x nv, Rg: nv x nu) */
} ops_t;

static void ops_init(ops_t *o, int method, int N, double h) {
    o->method = method; o->N = N; o->nv = N + 1;
    if (method == OR_CFD) {
        o->np = N - 1; o->nu = N + 1;
        o->Le = (double *)malloc(sizeof(double) * o->np * o->np);
        o->Re = (double *)malloc(sizeof(double) * o->np * o->nv);
        o->Lg = (double *)malloc(sizeof(double) * o->nv * o->nv);
        o->Rg = (double *)malloc(sizeof(double) * o->nv * o->nu);
        cfd_Pbar(N, o->Le); cfd_Qbar(N, h, o->Re); cfd_P(N, o->Lg); cfd_Q(N, h, o->Rg);
    } else {
        o->np = N; o->nu = N + 2;
        o->Le = (double *)calloc((size_t)o->np * o->np, sizeof(double));
        o->Re = (double *)malloc(sizeof(double) * o->np * o->nv);
        o->Lg = (double *)calloc((size_t)o->nv * o->nv, sizeof(double));
        o->Rg = (double *)malloc(sizeof(double) * o->nv * o->nu);
        for (int i = 0; i < o->np; ++i) o->Le[i * o->np + i] = 1.0;
        for (int i = 0; i < o->nv; ++i) o->Lg[i * o->nv + i] = 1.0;
        mfd_D(N, h, o->Re); mfd_G(N, h, o->Rg);
    }
}
static void ops_free(ops_t *o) { free(o->Le); free(o->Re); free(o->Lg); free(o->Rg); }

/* Explicit derivative of a velocity line at the interior pressure points:
 * out = Le^{-1} Re v  (CFD Pbar^{-1} Qbar v ; MFD D v). */
static void deriv_v(const ops_t *o, const double *v, double *out) {
    for (int i = 0; i < o->np; ++i) {
        double s = 0.0;
        for (int j = 0; j < o->nv; ++j) s += o->Re[(size_t)i * o->nv + j] * v[j];
        out[i] = s;
    }
    if (o->method == OR_CFD) dense_band_solve(o->Le, o->np, out);
}

/* Explicit derivative of a full pressure line at the velocity points:
 * out = Lg^{-1} Rg u  (CFD P^{-1} Q u ; MFD G u). */
static void deriv_u(const ops_t *o, const double *u, double *out) {
    for (int i = 0; i < o->nv; ++i) {
        double s = 0.0;
        for (int j = 0; j < o->nu; ++j) s += o->Rg[(size_t)i * o->nu + j] * u[j];
        out[i] = s;
    }
    if (o->method == OR_CFD) dense_band_solve(o->Lg, o->nv, out);
}

/* ------------------------------------------------------------------------------------ */
/* The coupled line system of Eq. 8 / Eq. 10, solved exactly.                            */
/*   unknowns: ubar (np), v (nv), e (np), g (nv)                                         */
/*   ubar + alpha .* e = a                                                               */
/*   v    + beta  .* g = vm                                                              */
/*   Le e - Re v       = 0                                                               */
/*   Lg g - Rg_int ubar = Rg_bnd [ub0, ub1]                                              */
/* Unknowns are ordered by their position along the line so that the matrix is banded. */
/* ------------------------------------------------------------------------------------ */

enum { T_U = 0, T_E = 1, T_V = 2, T_G = 3 };

typedef struct { int pos, type, k; } unk_t;

static int unk_cmp(const void *a, const void *b) {
    const unk_t *x = (const unk_t *)a, *y = (const unk_t *)b;
    if (x->pos != y->pos) return x->pos - y->pos;
    return x->type - y->type;
}

/* Position (in half-cell units) of the k-th interior pressure unknown and of velocity
 * point j.  CFD: both on nodes.  MFD: pressure at cell centres, velocity on nodes. */
static int pos_p(int method, int k) { return method == OR_CFD ? 2 * (k + 1) : 2 * k + 1; }
static int pos_v(int j) { return 2 * j; }

typedef struct {
    int n;
    int *idx[4];
} layout_t;

static void layout_build(const ops_t *o, layout_t *L) {
    int n = 2 * o->np + 2 * o->nv;
    unk_t *u = (unk_t *)malloc(sizeof(unk_t) * n);
    int c = 0;
    for (int k = 0; k < o->np; ++k) { u[c++] = (unk_t){pos_p(o->method, k), T_U, k}; }
    for (int k = 0; k < o->np; ++k) { u[c++] = (unk_t){pos_p(o->method, k), T_E, k}; }
    for (int j = 0; j < o->nv; ++j) { u[c++] = (unk_t){pos_v(j), T_V, j}; }
    for (int j = 0; j < o->nv; ++j) { u[c++] = (unk_t){pos_v(j), T_G, j}; }
    qsort(u, n, sizeof(unk_t), unk_cmp);
    L->n = n;
    L->idx[T_U] = (int *)malloc(sizeof(int) * o->np);
    L->idx[T_E] = (int *)malloc(sizeof(int) * o->np);
    L->idx[T_V] = (int *)malloc(sizeof(int) * o->nv);
    L->idx[T_G] = (int *)malloc(sizeof(int) * o->nv);
    for (int i = 0; i < n; ++i) L->idx[u[i].type][u[i].k] = i;
    free(u);
}
static void layout_free(layout_t *L) { for (int t = 0; t < 4; ++t) free(L->idx[t]); }

/* Visits every nonzero of the line matrix: f(row, col, value). */
typedef void (*visit_fn)(void *ctx, int i, int j, double v);

static void line_matrix_visit(const ops_t *o, const layout_t *L, const double *alpha,
                              double beta, visit_fn f, void *ctx) {
    int np = o->np, nv = o->nv, nu = o->nu;
    for (int k = 0; k < np; ++k) {
        int r = L->idx[T_U][k];
        f(ctx, r, r, 1.0);
        f(ctx, r, L->idx[T_E][k], alpha[k]);
    }
    for (int j = 0; j < nv; ++j) {
        int r = L->idx[T_V][j];
        f(ctx, r, r, 1.0);
        f(ctx, r, L->idx[T_G][j], beta);
    }
    for (int k = 0; k < np; ++k) {
        int r = L->idx[T_E][k];
        for (int kk = 0; kk < np; ++kk) {
            double c = o->Le[(size_t)k * np + kk];
            if (c != 0.0) f(ctx, r, L->idx[T_E][kk], c);
        }
        for (int j = 0; j < nv; ++j) {
            double c = o->Re[(size_t)k * nv + j];
            if (c != 0.0) f(ctx, r, L->idx[T_V][j], -c);
        }
    }
    for (int j = 0; j < nv; ++j) {
        int r = L->idx[T_G][j];
        for (int jj = 0; jj < nv; ++jj) {
            double c = o->Lg[(size_t)j * nv + jj];
            if (c != 0.0) f(ctx, r, L->idx[T_G][jj], c);
        }
        /* interior pressure entries of the full line are columns 1..nu-2 */
        for (int m = 1; m < nu - 1; ++m) {
            double c = o->Rg[(size_t)j * nu + m];
            if (c != 0.0) f(ctx, r, L->idx[T_U][m - 1], -c);
        }
    }
}

typedef struct { int kl, ku; } bw_t;
static void visit_bw(void *ctx, int i, int j, double v) {
    (void)v;
    bw_t *b = (bw_t *)ctx;
    if (i - j > b->kl) b->kl = i - j;
    if (j - i > b->ku) b->ku = j - i;
}
static void visit_band(void *ctx, int i, int j, double v) { *band_at((band_t *)ctx, i, j) += v; }

typedef struct { int n; double *A; } dense_t;
static void visit_dense(void *ctx, int i, int j, double v) {
    dense_t *d = (dense_t *)ctx;
    d->A[(size_t)i * d->n + j] += v;
}

static void line_rhs(const ops_t *o, const layout_t *L, const double *a, const double *vm,
                     double ub0, double ub1, double *rhs) {
    int np = o->np, nv = o->nv, nu = o->nu;
    memset(rhs, 0, sizeof(double) * L->n);
    for (int k = 0; k < np; ++k) rhs[L->idx[T_U][k]] = a[k];
    for (int j = 0; j < nv; ++j) rhs[L->idx[T_V][j]] = vm[j];
    for (int j = 0; j < nv; ++j)
        rhs[L->idx[T_G][j]] = o->Rg[(size_t)j * nu + 0] * ub0 + o->Rg[(size_t)j * nu + nu - 1] * ub1;
}

/* Exact solve of one line system.  alpha, a: np values; vm: nv values.
 * Writes ubar (np) and v (nv).  Returns 0 or -1 (singular). */
static int line_solve(const ops_t *o, const layout_t *L, const double *alpha, double beta,
                      const double *a, const double *vm, double ub0, double ub1,
                      double *ubar, double *v) {
    bw_t bw = {0, 0};
    line_matrix_visit(o, L, alpha, beta, visit_bw, &bw);
    band_t b;
    band_init(&b, L->n, bw.kl, bw.ku);
    line_matrix_visit(o, L, alpha, beta, visit_band, &b);
    double *x = (double *)malloc(sizeof(double) * L->n);
    line_rhs(o, L, a, vm, ub0, ub1, x);
    int rc = band_solve(&b, x);
    for (int k = 0; k < o->np; ++k) ubar[k] = x[L->idx[T_U][k]];
    for (int j = 0; j < o->nv; ++j) v[j] = x[L->idx[T_V][j]];
    free(x);
    band_free(&b);
    return rc;
}

/* Exported single-line solve for tests.  dense != 0 uses a dense Gaussian elimination with
 * partial pivoting on the same system instead of the banded one. */
int oracle_line_solve(int method, int N, double h, const double *alpha, double beta,
                      const double *a, const double *vm, double ub0, double ub1,
                      double *ubar, double *v, int dense) {
    if (N < 8) return -1;
    ops_t o;
    ops_init(&o, method, N, h);
    layout_t L;
    layout_build(&o, &L);
    int rc = 0;
    if (!dense) {
        rc = line_solve(&o, &L, alpha, beta, a, vm, ub0, ub1, ubar, v);
    } else {
        int n = L.n;
        dense_t d = {n, (double *)calloc((size_t)n * n, sizeof(double))};
        line_matrix_visit(&o, &L, alpha, beta, visit_dense, &d);
        double *x = (double *)malloc(sizeof(double) * n);
        line_rhs(&o, &L, a, vm, ub0, ub1, x);
        double *A = d.A;
        for (int c = 0; c < n && rc == 0; ++c) {
            int p = c;
            for (int i = c + 1; i < n; ++i)
                if (fabs(A[(size_t)i * n + c]) > fabs(A[(size_t)p * n + c])) p = i;
            if (A[(size_t)p * n + c] == 0.0) { rc = -1; break; }
            if (p != c) {
                for (int j = 0; j < n; ++j) {
                    double t = A[(size_t)c * n + j];
                    A[(size_t)c * n + j] = A[(size_t)p * n + j];
                    A[(size_t)p * n + j] = t;
                }
                double t = x[c]; x[c] = x[p]; x[p] = t;
            }
            for (int i = c + 1; i < n; ++i) {
                double l = A[(size_t)i * n + c] / A[(size_t)c * n + c];
                if (l == 0.0) continue;
                for (int j = c; j < n; ++j) A[(size_t)i * n + j] -= l * A[(size_t)c * n + j];
                x[i] -= l * x[c];
            }
        }
        for (int i = n - 1; i >= 0 && rc == 0; --i) {
            double s = x[i];
            for (int j = i + 1; j < n; ++j) s -= A[(size_t)i * n + j] * x[j];
            x[i] = s / A[(size_t)i * n + i];
        }
        for (int k = 0; k < o.np; ++k) ubar[k] = x[L.idx[T_U][k]];
        for (int j = 0; j < o.nv; ++j) v[j] = x[L.idx[T_V][j]];
        free(x);
        free(A);
    }
    layout_free(&L);
    ops_free(&o);
    return rc;
}

/* ------------------------------------------------------------------------------------ */
/* Source: a Ricker point source s(t) at one interior pressure point, f = s / h^2.       */
/* ------------------------------------------------------------------------------------ */

typedef struct { int on, is, js; double amp, f0, tdelay; } src_t;

static double ricker(const src_t *s, double t) {
    const double pi = 3.14159265358979323846;
    double tau = t - s->tdelay;
    double q = pi * pi * s->f0 * s->f0 * tau * tau;
    return s->amp * (1.0 - 2.0 * q) * exp(-q);
}

/* ------------------------------------------------------------------------------------ */
/* Time-harmonic Dirichlet data and distributed forcing (the manufactured problem of      */
/* Sec. 4, Eq. 11): u = B cos(omega t + phb) on the outer rows/columns of U, and           */
/* f = F cos(omega t + phf) at the interior pressure points.                              */
/* ------------------------------------------------------------------------------------ */

typedef struct { const double *B, *F; double omega, phb, phf; } harm_t;

static double harm_b(const harm_t *hb, size_t p, double t) {
    return hb->B[p] * cos(hb->omega * t + hb->phb);
}

/* Writes B cos(omega t + phb) into the given edges of a U-shaped array: rows 0 and
 * rows_u - 1 (south/north) and/or columns 0 and ldu - 1 (west/east). */
static void harm_edges(const harm_t *hb, double *U, int rows_u, int ldu, double t, int sn, int we) {
    if (sn)
        for (int j = 0; j < ldu; ++j) {
            U[j] = harm_b(hb, (size_t)j, t);
            U[(size_t)(rows_u - 1) * ldu + j] = harm_b(hb, (size_t)(rows_u - 1) * ldu + j, t);
        }
    if (we)
        for (int i = 0; i < rows_u; ++i) {
            U[(size_t)i * ldu] = harm_b(hb, (size_t)i * ldu, t);
            U[(size_t)i * ldu + ldu - 1] = harm_b(hb, (size_t)i * ldu + ldu - 1, t);
        }
}

/* ------------------------------------------------------------------------------------ */
/* One Peaceman-Rachford step on the whole grid (Eqs. 6-7 with Eq. 8 / Eq. 10).           */
/* ------------------------------------------------------------------------------------ */

typedef struct {
    int method, nx, ny;
    double h, dt;
    int ldu, ldv, ldw; /* row strides of U, V, W */
    int rows_u;        /* rows of U */
    int rows_v, rows_w;
    ops_t ox, oy;      /* operators along x lines (N = nx) and y lines (N = ny) */
    layout_t lx, ly;
} grid_t;

static void grid_init(grid_t *g, int method, int nx, int ny, double h, double dt) {
    g->method = method; g->nx = nx; g->ny = ny; g->h = h; g->dt = dt;
    if (method == OR_CFD) {
        g->ldu = g->ldv = g->ldw = nx + 1;
        g->rows_u = g->rows_v = g->rows_w = ny + 1;
    } else {
        g->ldu = nx + 2; g->ldv = nx + 1; g->ldw = nx + 2;
        g->rows_u = ny + 2; g->rows_v = ny + 2; g->rows_w = ny + 1;
    }
    ops_init(&g->ox, method, nx, h);
    ops_init(&g->oy, method, ny, h);
    layout_build(&g->ox, &g->lx);
    layout_build(&g->oy, &g->ly);
}
static void grid_free(grid_t *g) {
    ops_free(&g->ox); ops_free(&g->oy); layout_free(&g->lx); layout_free(&g->ly);
}

/* Number of interior pressure rows/cols: CFD N-1 (indices 1..N-1), MFD N (1..N). */
static int n_int(const grid_t *g, int N) { return g->method == OR_CFD ? N - 1 : N; }

static double frob_diff(const double *a, const double *b, size_t n) {
    double s = 0.0;
    for (size_t i = 0; i < n; ++i) { double d = a[i] - b[i]; s += d * d; }
    return sqrt(s);
}

/* kmax == 0: exact line solves.  kmax > 0: the paper's fixed-point iteration (Eq. 9,
 * Algorithms 3/4) with at most kmax sweeps and stopping threshold eps on the sum of the
 * Frobenius norms of the updates. */
static int pr_step(grid_t *g, const double *kappa, double *U, double *V, double *W,
                   double t, const src_t *src, const harm_t *hb, int kmax, double eps,
                   int nthreads, int *sweeps) {
    const int nx = g->nx, ny = g->ny;
    const int ldu = g->ldu, ldv = g->ldv, ldw = g->ldw;
    const int pix = n_int(g, nx), piy = n_int(g, ny); /* interior pressure counts */
    const double dt = g->dt, beta = 0.5 * dt;
    const size_t nU = (size_t)g->rows_u * ldu, nV = (size_t)g->rows_v * ldv,
                 nW = (size_t)g->rows_w * ldw;
    double *Ws = (double *)malloc(sizeof(double) * nW);
    double *Us = (double *)malloc(sizeof(double) * nU);
    double *Vs = (double *)malloc(sizeof(double) * nV);
    double *A = (double *)calloc(nU, sizeof(double));
    int fail = 0;
    (void)nthreads;
    memcpy(Ws, W, sizeof(double) * nW);
    memcpy(Us, U, sizeof(double) * nU);
    memcpy(Vs, V, sizeof(double) * nV);

    /* ---- stage 1 right-hand sides: w* and A (explicit in y) ---- */
#pragma omp parallel for schedule(static) num_threads(nthreads > 0 ? nthreads : 1)
    for (int j = 1; j <= pix; ++j) {
        double *ucol = (double *)malloc(sizeof(double) * g->oy.nu);
        double *wcol = (double *)malloc(sizeof(double) * g->oy.nv);
        double *dg = (double *)malloc(sizeof(double) * g->oy.nv);
        double *de = (double *)malloc(sizeof(double) * g->oy.np);
        for (int i = 0; i < g->oy.nu; ++i) ucol[i] = U[(size_t)i * ldu + j];
        for (int i = 0; i < g->oy.nv; ++i) wcol[i] = W[(size_t)i * ldw + j];
        deriv_u(&g->oy, ucol, dg);  /* D_y u on the whole column */
        deriv_v(&g->oy, wcol, de);  /* Dbar_y w at interior pressure points */
        for (int i = 0; i < g->oy.nv; ++i) Ws[(size_t)i * ldw + j] = wcol[i] - beta * dg[i];
        for (int i = 1; i <= piy; ++i) {
            size_t p = (size_t)i * ldu + j;
            A[p] = U[p] - 0.5 * dt * kappa[p] * de[i - 1];
        }
        free(ucol); free(wcol); free(dg); free(de);
    }
    if (src->on) A[(size_t)src->is * ldu + src->js] += 0.5 * dt * ricker(src, t) / (g->h * g->h);
    if (hb && hb->F) {
        const double ft = cos(hb->omega * t + hb->phf);
        for (int i = 1; i <= piy; ++i)
            for (int j = 1; j <= pix; ++j) {
                size_t p = (size_t)i * ldu + j;
                A[p] += 0.5 * dt * hb->F[p] * ft;
            }
    }
    /* the intermediate u* at the ends of the x-lines (west/east walls): u0(t + dt/2) */
    if (hb) harm_edges(hb, Us, g->rows_u, ldu, t + 0.5 * dt, 0, 1);

    /* ---- stage 1 implicit x-lines: (ubar*, v*) ---- */
    if (kmax == 0) {
#pragma omp parallel for schedule(static) num_threads(nthreads > 0 ? nthreads : 1)
        for (int i = 1; i <= piy; ++i) {
            double *al = (double *)malloc(sizeof(double) * pix);
            double *ub = (double *)malloc(sizeof(double) * pix);
            for (int k = 0; k < pix; ++k) al[k] = 0.5 * dt * kappa[(size_t)i * ldu + k + 1];
            int rc = line_solve(&g->ox, &g->lx, al, beta, &A[(size_t)i * ldu + 1],
                                &V[(size_t)i * ldv], Us[(size_t)i * ldu],
                                Us[(size_t)i * ldu + g->ox.nu - 1], ub, &Vs[(size_t)i * ldv]);
            if (rc) fail = 1;
            for (int k = 0; k < pix; ++k) Us[(size_t)i * ldu + k + 1] = ub[k];
            free(al); free(ub);
        }
    } else {
        /* Algorithm 3/4 ADI-rows: U_{k+1} = A - dt/2 K.*Dbar_x V_k ; V_{k+1} = B - dt/2 R.*D_x U_{k+1} */
        double *Uk = (double *)malloc(sizeof(double) * nU);
        double *Vk = (double *)malloc(sizeof(double) * nV);
        memcpy(Uk, U, sizeof(double) * nU);
        memcpy(Vk, V, sizeof(double) * nV);
        int k = 0;
        for (;;) {
            for (int i = 1; i <= piy; ++i) {
                double *de = (double *)malloc(sizeof(double) * g->ox.np);
                double *dg = (double *)malloc(sizeof(double) * g->ox.nv);
                deriv_v(&g->ox, &Vk[(size_t)i * ldv], de);
                for (int c = 1; c <= pix; ++c) {
                    size_t p = (size_t)i * ldu + c;
                    Us[p] = A[p] - 0.5 * dt * kappa[p] * de[c - 1];
                }
                deriv_u(&g->ox, &Us[(size_t)i * ldu], dg);
                for (int c = 0; c < g->ox.nv; ++c)
                    Vs[(size_t)i * ldv + c] = V[(size_t)i * ldv + c] - beta * dg[c];
                free(de); free(dg);
            }
            double test = frob_diff(Us, Uk, nU) + frob_diff(Vs, Vk, nV);
            memcpy(Uk, Us, sizeof(double) * nU);
            memcpy(Vk, Vs, sizeof(double) * nV);
            ++k;
            if (test <= eps || k >= kmax) break;
        }
        if (sweeps) sweeps[0] = k;
        free(Uk); free(Vk);
    }

    /* ---- stage 2 right-hand sides: v^{m+1} and C (explicit in x) ---- */
    double *Vn = (double *)malloc(sizeof(double) * nV);
    memcpy(Vn, Vs, sizeof(double) * nV);
#pragma omp parallel for schedule(static) num_threads(nthreads > 0 ? nthreads : 1)
    for (int i = 1; i <= piy; ++i) {
        double *dg = (double *)malloc(sizeof(double) * g->ox.nv);
        double *de = (double *)malloc(sizeof(double) * g->ox.np);
        deriv_u(&g->ox, &Us[(size_t)i * ldu], dg);
        deriv_v(&g->ox, &Vs[(size_t)i * ldv], de);
        for (int c = 0; c < g->ox.nv; ++c)
            Vn[(size_t)i * ldv + c] = Vs[(size_t)i * ldv + c] - beta * dg[c];
        for (int c = 1; c <= pix; ++c) {
            size_t p = (size_t)i * ldu + c;
            A[p] = Us[p] - 0.5 * dt * kappa[p] * de[c - 1]; /* A now holds C */
        }
        free(dg); free(de);
    }
    if (src->on)
        A[(size_t)src->is * ldu + src->js] += 0.5 * dt * ricker(src, t + dt) / (g->h * g->h);
    if (hb && hb->F) {
        const double ft = cos(hb->omega * (t + dt) + hb->phf);
        for (int i = 1; i <= piy; ++i)
            for (int j = 1; j <= pix; ++j) {
                size_t p = (size_t)i * ldu + j;
                A[p] += 0.5 * dt * hb->F[p] * ft;
            }
    }

    /* ---- stage 2 implicit y-lines: (ubar^{m+1}, w^{m+1}) ---- */
    double *Wn = (double *)malloc(sizeof(double) * nW);
    memcpy(Wn, Ws, sizeof(double) * nW);
    double *Un = (double *)malloc(sizeof(double) * nU);
    memcpy(Un, Us, sizeof(double) * nU);
    /* the ends of the y-lines (south/north walls) at the new time level */
    if (hb) harm_edges(hb, Un, g->rows_u, ldu, t + dt, 1, 0);
    if (kmax == 0) {
#pragma omp parallel for schedule(static) num_threads(nthreads > 0 ? nthreads : 1)
        for (int j = 1; j <= pix; ++j) {
            double *al = (double *)malloc(sizeof(double) * piy);
            double *cc = (double *)malloc(sizeof(double) * piy);
            double *wv = (double *)malloc(sizeof(double) * g->oy.nv);
            double *ub = (double *)malloc(sizeof(double) * piy);
            double *wo = (double *)malloc(sizeof(double) * g->oy.nv);
            for (int k = 0; k < piy; ++k) {
                size_t p = (size_t)(k + 1) * ldu + j;
                al[k] = 0.5 * dt * kappa[p];
                cc[k] = A[p];
            }
            for (int r = 0; r < g->oy.nv; ++r) wv[r] = Ws[(size_t)r * ldw + j];
            int rc = line_solve(&g->oy, &g->ly, al, beta, cc, wv, Un[j],
                                Un[(size_t)(g->oy.nu - 1) * ldu + j], ub, wo);
            if (rc) fail = 1;
            for (int k = 0; k < piy; ++k) Un[(size_t)(k + 1) * ldu + j] = ub[k];
            for (int r = 0; r < g->oy.nv; ++r) Wn[(size_t)r * ldw + j] = wo[r];
            free(al); free(cc); free(wv); free(ub); free(wo);
        }
    } else {
        /* Algorithm 3/4 ADI-columns: U_{k+1} = C - dt/2 K.*Dbar_y W_k ; W_{k+1} = D - dt/2 R.*D_y U_{k+1} */
        double *Uk = (double *)malloc(sizeof(double) * nU);
        double *Wk = (double *)malloc(sizeof(double) * nW);
        memcpy(Uk, Us, sizeof(double) * nU);
        memcpy(Wk, W, sizeof(double) * nW);
        int k = 0;
        for (;;) {
            for (int j = 1; j <= pix; ++j) {
                double *wcol = (double *)malloc(sizeof(double) * g->oy.nv);
                double *ucol = (double *)malloc(sizeof(double) * g->oy.nu);
                double *de = (double *)malloc(sizeof(double) * g->oy.np);
                double *dg = (double *)malloc(sizeof(double) * g->oy.nv);
                for (int r = 0; r < g->oy.nv; ++r) wcol[r] = Wk[(size_t)r * ldw + j];
                deriv_v(&g->oy, wcol, de);
                for (int r = 1; r <= piy; ++r) {
                    size_t p = (size_t)r * ldu + j;
                    Un[p] = A[p] - 0.5 * dt * kappa[p] * de[r - 1];
                }
                for (int r = 0; r < g->oy.nu; ++r) ucol[r] = Un[(size_t)r * ldu + j];
                deriv_u(&g->oy, ucol, dg);
                for (int r = 0; r < g->oy.nv; ++r)
                    Wn[(size_t)r * ldw + j] = Ws[(size_t)r * ldw + j] - beta * dg[r];
                free(wcol); free(ucol); free(de); free(dg);
            }
            double test = frob_diff(Un, Uk, nU) + frob_diff(Wn, Wk, nW);
            memcpy(Uk, Un, sizeof(double) * nU);
            memcpy(Wk, Wn, sizeof(double) * nW);
            ++k;
            if (test <= eps || k >= kmax) break;
        }
        if (sweeps) sweeps[1] = k;
        free(Uk); free(Wk);
    }

    /* every wall at the new time level */
    if (hb) harm_edges(hb, Un, g->rows_u, ldu, t + dt, 1, 1);
    memcpy(U, Un, sizeof(double) * nU);
    memcpy(V, Vn, sizeof(double) * nV);
    memcpy(W, Wn, sizeof(double) * nW);
    free(Ws); free(Us); free(Vs); free(A); free(Vn); free(Wn); free(Un);
    return fail ? -1 : 0;
}

/* ------------------------------------------------------------------------------------ */
/* Exported driver.                                                                       */
/* ------------------------------------------------------------------------------------ */

/* Advances (U, V, W) by nsteps Peaceman-Rachford steps starting at time t0.
 * src: NULL, or {is, js, amp, f0, tdelay} for a Ricker point source at U[is][js].
 * kmax: 0 for exact line solves, > 0 for the paper's fixed-point iteration.
 * nthreads: OpenMP threads over grid lines (1 = sequential).
 * sweeps: NULL, or 2 * nsteps ints that receive, per step, the fixed-point sweeps that
 * stage 1 and stage 2 took (kmax > 0 only; left untouched for exact solves).
 * Returns 0, -1 for invalid arguments, -2 for a singular line system. */
/* ------------------------------------------------------------------------------------ */
/* Absorbing layers: Cerjan's damping (named in Sec. 2.1 as the absorbing technique the    */
/* CFD formulation admits).  After every full step each field value at a point whose       */
/* distance to the nearest wall is delta cells, delta < width, is multiplied by            */
/*     g = exp(-(a (width - delta))^2);                                                    */
/* pressure values on the walls themselves (the Dirichlet data) are left alone.            */
/* ------------------------------------------------------------------------------------ */

typedef struct { double width, a; } sponge_t;

/* Coordinates in cells of the points of U (kind 0), V (1), W (2) along x (row index j) and
 * y (row index i): CFD nodes; MFD cell centres plus edges for pressure, nodes across the
 * velocity's own direction. */
static double coord(int method, int kind_axis_staggered, int k, int n) {
    if (method == OR_CFD || !kind_axis_staggered) return (double)k;
    if (k == 0) return 0.0;
    if (k == n + 1) return (double)n;
    return k - 0.5;
}

static double sponge_g(const sponge_t *sp, double x, double y, int nx, int ny) {
    double d = x;
    if (nx - x < d) d = nx - x;
    if (y < d) d = y;
    if (ny - y < d) d = ny - y;
    if (d >= sp->width) return 1.0;
    double q = sp->a * (sp->width - d);
    return exp(-q * q);
}

static void sponge_apply(const grid_t *g, const sponge_t *sp, double *U, double *V, double *W) {
    const int nx = g->nx, ny = g->ny, m = g->method;
    /* U: staggered (MFD centres) along both axes; walls excluded */
    for (int i = 1; i < g->rows_u - 1; ++i)
        for (int j = 1; j < g->ldu - 1; ++j)
            U[(size_t)i * g->ldu + j] *= sponge_g(sp, coord(m, 1, j, nx), coord(m, 1, i, ny), nx, ny);
    /* V: x on nodes, y staggered (MFD) */
    for (int i = 0; i < g->rows_v; ++i)
        for (int j = 0; j < g->ldv; ++j)
            V[(size_t)i * g->ldv + j] *= sponge_g(sp, (double)j, coord(m, 1, i, ny), nx, ny);
    /* W: x staggered (MFD), y on nodes */
    for (int i = 0; i < g->rows_w; ++i)
        for (int j = 0; j < g->ldw; ++j)
            W[(size_t)i * g->ldw + j] *= sponge_g(sp, coord(m, 1, j, nx), (double)i, nx, ny);
}

static int run_all(int method, int nx, int ny, double h, double dt, const double *kappa,
                   double *U, double *V, double *W, int nsteps, double t0, const double *src,
                   const harm_t *hb, int kmax, double eps, int nthreads, int *sweeps,
                   const sponge_t *sponge) {
    if ((method != OR_CFD && method != OR_MFD) || nx < 8 || ny < 8 || !(h > 0.0) ||
        !(dt > 0.0) || nsteps < 0 || kmax < 0)
        return -1;
    grid_t g;
    grid_init(&g, method, nx, ny, h, dt);
    src_t s = {0, 0, 0, 0.0, 0.0, 0.0};
    if (src) {
        s.on = 1; s.is = (int)src[0]; s.js = (int)src[1];
        s.amp = src[2]; s.f0 = src[3]; s.tdelay = src[4];
        int lo = 1, hix = n_int(&g, nx), hiy = n_int(&g, ny);
        if (s.is < lo || s.is > hiy || s.js < lo || s.js > hix) { grid_free(&g); return -1; }
    }
    int rc = 0;
    for (int m = 0; m < nsteps && rc == 0; ++m) {
        if (pr_step(&g, kappa, U, V, W, t0 + m * dt, &s, hb, kmax, eps, nthreads,
                    sweeps ? sweeps + 2 * m : NULL))
            rc = -2;
        if (sponge && rc == 0) sponge_apply(&g, sponge, U, V, W);
    }
    grid_free(&g);
    return rc;
}

int oracle_run(int method, int nx, int ny, double h, double dt, const double *kappa,
               double *U, double *V, double *W, int nsteps, double t0, const double *src,
               int kmax, double eps, int nthreads, int *sweeps) {
    return run_all(method, nx, ny, h, dt, kappa, U, V, W, nsteps, t0, src, NULL, kmax, eps,
                   nthreads, sweeps, NULL);
}

/* oracle_run with Cerjan absorbing layers of `width` cells and strength `a` along every wall
 * (width 0 or a 0: no damping). */
int oracle_run_sponge(int method, int nx, int ny, double h, double dt, const double *kappa,
                      double *U, double *V, double *W, int nsteps, double t0, const double *src,
                      double width, double a, int nthreads) {
    if (!(width >= 0.0) || !(a >= 0.0)) return -1;
    sponge_t sp = {width, a};
    return run_all(method, nx, ny, h, dt, kappa, U, V, W, nsteps, t0, src, NULL, 0, 0.0,
                   nthreads, NULL, &sp);
}

/* oracle_run with time-harmonic Dirichlet data and forcing (Sec. 4, Eq. 11):
 *   B      U-shaped; u = B cos(omega t + phb) on U's outer rows and columns.  The caller's
 *          U must already hold the walls at t0.
 *   F      U-shaped or NULL; f = F cos(omega t + phf) at the interior pressure points, added
 *          as Eqs. 6-7 add the source (dt/2 f(t_m) in stage 1, dt/2 f(t_{m+1}) in stage 2).
 * The intermediate u* at the x-line ends (west and east walls) is u0(t_m + dt/2); the
 * y-line ends (south and north walls) take u0(t_{m+1}).  sponge_width, sponge_a > 0 add the
 * absorbing layers of oracle_run_sponge after every step. */
int oracle_run_harmonic(int method, int nx, int ny, double h, double dt, const double *kappa,
                        double *U, double *V, double *W, int nsteps, double t0,
                        const double *src, const double *B, const double *F, double omega,
                        double phb, double phf, int kmax, double eps, int nthreads,
                        double sponge_width, double sponge_a) {
    if (!B || !(sponge_width >= 0.0) || !(sponge_a >= 0.0)) return -1;
    harm_t hb = {B, F, omega, phb, phf};
    sponge_t sp = {sponge_width, sponge_a};
    return run_all(method, nx, ny, h, dt, kappa, U, V, W, nsteps, t0, src, &hb, kmax, eps,
                   nthreads, NULL, sponge_width > 0.0 && sponge_a > 0.0 ? &sp : NULL);
}

int oracle_num_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}
