/*
 * Iterative FP64 CPU solver of the blob systems (oracle side; TEST
 * INFRASTRUCTURE ONLY: only the tests, the smoke check and the benchmark's
 * CPU-baseline leg load it; the CUDA library never links or calls it, and it
 * shares no code with the CUDA library).
 *
 * It is the paper's own method written out plainly for the host cores, so
 * that a full solve of the benchmark workload can be timed on the CPU:
 *
 *   - flexible GMRES(restart) with modified Gram-Schmidt (Sec. III.E), right
 *     preconditioned, stopping on the true relative residual ||b - K x|| / ||b||;
 *   - the reaction-limited system (alpha I - chi L + S kappa J) c = g
 *     (Eqs. unsteady_system, steady_state), preconditioned by n multigrid
 *     V-cycles of (sigma I - chi L) with sigma = alpha when alpha > 0, else
 *     sum(kappa) / V_Omega, the mean of S kappa J on constants (the paper's
 *     (alpha I - chi L)^-1 is singular in the steady periodic case);
 *   - the saddle point [A zeta S; xi J 0] [c; lambda] = [g; f] (Eq.
 *     saddle_point), preconditioned by the five steps of Appendix A with the
 *     approximate Schur complement (GMRES(m) on J A~_1^-1 S from zero);
 *   - the multigrid V-cycle (Sec. III.E delegates it to a library; the
 *     readings are the same as the NumPy oracle's): levels halve every side
 *     while all sides are even and >= 4, red-black Gauss-Seidel (red = i+j+k
 *     even, red then black), nu1 / nu2 sweeps, restriction by the 8-cell
 *     mean, cell-centred trilinear prolongation (3/4, 1/4 per axis),
 *     re-discretised coarse operators, the coarsest level solved exactly
 *     (dense LU; with a singular operator the mean-zero solution of
 *     (A + 1 1^T / n) x = b), and for alpha = 0 the right-hand side projected
 *     to mean zero before the cycle and the result after it (the restricted
 *     inverse of Appendix A);
 *   - J and S with Peskin's 4- or 3-point kernel (Sec. III.A, Eq.
 *     tensor_product; S = h^-3 J^T).
 *
 * Grid loops run on all host threads with OpenMP; the code is otherwise
 * written for clarity, not tuned. Fields are x-fastest, cell (i, j, k) at
 * index i + nx (j + ny k), centre ((i + 1/2) h, (j + 1/2) h, (k + 1/2) h).
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>
#include <omp.h>

#define MAX_LEVELS 24 /* levels of the hierarchy (3 workspace slots each) */

/* ----------------------------------------------------------- vector ops */
static double vdot(const double* a, const double* b, long n) {
  double s = 0.0;
#pragma omp parallel for reduction(+ : s) schedule(static)
  for (long i = 0; i < n; ++i) s += a[i] * b[i];
  return s;
}
static double vnorm(const double* a, long n) { return sqrt(vdot(a, a, n)); }
static void vaxpy(double a, const double* x, double* y, long n) {
#pragma omp parallel for schedule(static)
  for (long i = 0; i < n; ++i) y[i] += a * x[i];
}
static void vscale_copy(double a, const double* x, double* y, long n) {
#pragma omp parallel for schedule(static)
  for (long i = 0; i < n; ++i) y[i] = a * x[i];
}
static void vzero(double* y, long n) {
#pragma omp parallel for schedule(static)
  for (long i = 0; i < n; ++i) y[i] = 0.0;
}
static double vmean(const double* a, long n) {
  double s = 0.0;
#pragma omp parallel for reduction(+ : s) schedule(static)
  for (long i = 0; i < n; ++i) s += a[i];
  return s / (double)n;
}
static void vshift(double* a, double c, long n) {
#pragma omp parallel for schedule(static)
  for (long i = 0; i < n; ++i) a[i] += c;
}

/* periodic index of any integer i */
static int wrapi(int i, int n) {
  i %= n;
  return i < 0 ? i + n : i;
}
/* periodic index of a neighbour, -1 <= i <= n */
static int wrap1(int i, int n) { return i < 0 ? i + n : (i >= n ? i - n : i); }

/* Grow-only workspaces kept between solves (a solver library keeps its
 * buffers; re-allocating and first-touching the Krylov basis every solve would
 * dominate a timed step). Slot s holds one buffer; contents are not kept. */
#define N_SLOTS 96
static void* g_slot[N_SLOTS];
static size_t g_cap[N_SLOTS];
static void* scratch(int s, size_t bytes) {
  if (bytes == 0) bytes = 8;
  if (g_cap[s] < bytes) {
    free(g_slot[s]);
    g_slot[s] = malloc(bytes);
    g_cap[s] = g_slot[s] ? bytes : 0;
  }
  return g_slot[s];
}
enum { SLOT_V = 0, SLOT_Z, SLOT_R, SLOT_B, SLOT_T1, SLOT_T2, SLOT_T3, SLOT_T4, SLOT_LEVEL0 };

/* ----------------------------------------------------------- multigrid */
typedef struct {
  int nx, ny, nz;
  long n;
  double h;
  double *x, *b, *r;
} level_t;

typedef struct {
  int nl;
  level_t lv[MAX_LEVELS];
  double chi, shift; /* operator shift I - chi L */
  int singular;      /* shift == 0: the periodic operator has the constants as null space */
  int nu1, nu2;
  double* lu; /* LU factors of the coarsest operator (row major), with pivots */
  int* piv;
  int nc;
} mg_t;

static long cells(int nx, int ny, int nz) { return (long)nx * ny * nz; }

/* y = (shift + 6 chi/h^2) x - chi/h^2 (sum of the 6 periodic neighbours) */
static void apply_level(const level_t* L, double chi, double shift, const double* x, double* y) {
  const int nx = L->nx, ny = L->ny, nz = L->nz;
  const double off = chi / (L->h * L->h), diag = shift + 6.0 * off;
#pragma omp parallel for schedule(static)
  for (int k = 0; k < nz; ++k) {
    const int km = wrap1(k - 1, nz), kp = wrap1(k + 1, nz);
    for (int j = 0; j < ny; ++j) {
      const int jm = wrap1(j - 1, ny), jp = wrap1(j + 1, ny);
      for (int i = 0; i < nx; ++i) {
        const int im = wrap1(i - 1, nx), ip = wrap1(i + 1, nx);
        const long c = i + (long)nx * (j + (long)ny * k);
        const double s = x[im + (long)nx * (j + (long)ny * k)] + x[ip + (long)nx * (j + (long)ny * k)] +
                         x[i + (long)nx * (jm + (long)ny * k)] + x[i + (long)nx * (jp + (long)ny * k)] +
                         x[i + (long)nx * (j + (long)ny * km)] + x[i + (long)nx * (j + (long)ny * kp)];
        y[c] = diag * x[c] - off * s;
      }
    }
  }
}

/* Gauss-Seidel update of every cell of one colour (red: i+j+k even) */
static void half_sweep(const level_t* L, double chi, double shift, double* x, const double* b, int colour) {
  const int nx = L->nx, ny = L->ny, nz = L->nz;
  const double off = chi / (L->h * L->h), diag = shift + 6.0 * off;
#pragma omp parallel for schedule(static)
  for (int k = 0; k < nz; ++k) {
    const int km = wrap1(k - 1, nz), kp = wrap1(k + 1, nz);
    for (int j = 0; j < ny; ++j) {
      const int jm = wrap1(j - 1, ny), jp = wrap1(j + 1, ny);
      for (int i = (colour + j + k) & 1; i < nx; i += 2) {
        const int im = wrap1(i - 1, nx), ip = wrap1(i + 1, nx);
        const long c = i + (long)nx * (j + (long)ny * k);
        const double s = x[im + (long)nx * (j + (long)ny * k)] + x[ip + (long)nx * (j + (long)ny * k)] +
                         x[i + (long)nx * (jm + (long)ny * k)] + x[i + (long)nx * (jp + (long)ny * k)] +
                         x[i + (long)nx * (j + (long)ny * km)] + x[i + (long)nx * (j + (long)ny * kp)];
        x[c] = (b[c] + off * s) / diag;
      }
    }
  }
}

static void rb_sweep(const level_t* L, double chi, double shift, double* x, const double* b) {
  half_sweep(L, chi, shift, x, b, 0);
  half_sweep(L, chi, shift, x, b, 1);
}

/* coarse b = mean of the 8 fine children of r */
static void restrict8(const level_t* F, const double* r, const level_t* C, double* bc) {
  const int nx = F->nx, ny = F->ny;
#pragma omp parallel for schedule(static)
  for (int K = 0; K < C->nz; ++K)
    for (int J = 0; J < C->ny; ++J)
      for (int I = 0; I < C->nx; ++I) {
        double s = 0.0;
        for (int dz = 0; dz < 2; ++dz)
          for (int dy = 0; dy < 2; ++dy)
            for (int dx = 0; dx < 2; ++dx)
              s += r[(2 * I + dx) + (long)nx * ((2 * J + dy) + (long)ny * (2 * K + dz))];
        bc[I + (long)C->nx * (J + (long)C->ny * K)] = 0.125 * s;
      }
}

/* x_fine += trilinear cell-centred interpolation of the coarse field e: fine
 * cell 2I takes 3/4 of coarse I and 1/4 of coarse I-1, fine cell 2I+1 3/4 of
 * I and 1/4 of I+1, per axis */
static void prolong_add(const level_t* C, const double* e, const level_t* F, double* x) {
  const int nxc = C->nx, nyc = C->ny, nzc = C->nz;
#pragma omp parallel for schedule(static)
  for (int k = 0; k < F->nz; ++k) {
    const int K = k >> 1, K2 = wrap1((k & 1) ? K + 1 : K - 1, nzc);
    for (int j = 0; j < F->ny; ++j) {
      const int J = j >> 1, J2 = wrap1((j & 1) ? J + 1 : J - 1, nyc);
      for (int i = 0; i < F->nx; ++i) {
        const int I = i >> 1, I2 = wrap1((i & 1) ? I + 1 : I - 1, nxc);
#define E(kk, jj, ii) e[(ii) + (long)nxc * ((jj) + (long)nyc * (kk))]
        const double v = 0.75 * (0.75 * (0.75 * E(K, J, I) + 0.25 * E(K, J, I2)) +
                                 0.25 * (0.75 * E(K, J2, I) + 0.25 * E(K, J2, I2))) +
                         0.25 * (0.75 * (0.75 * E(K2, J, I) + 0.25 * E(K2, J, I2)) +
                                 0.25 * (0.75 * E(K2, J2, I) + 0.25 * E(K2, J2, I2)));
#undef E
        x[i + (long)F->nx * (j + (long)F->ny * k)] += v;
      }
    }
  }
}

/* LU with partial pivoting of a dense n x n matrix (row major, in place) */
static int lu_factor(double* a, int* piv, int n) {
  for (int c = 0; c < n; ++c) {
    int p = c;
    for (int r = c + 1; r < n; ++r)
      if (fabs(a[(long)r * n + c]) > fabs(a[(long)p * n + c])) p = r;
    piv[c] = p;
    if (a[(long)p * n + c] == 0.0) return -1;
    if (p != c)
      for (int q = 0; q < n; ++q) {
        const double t = a[(long)c * n + q];
        a[(long)c * n + q] = a[(long)p * n + q];
        a[(long)p * n + q] = t;
      }
    for (int r = c + 1; r < n; ++r) {
      const double m = a[(long)r * n + c] / a[(long)c * n + c];
      a[(long)r * n + c] = m;
      for (int q = c + 1; q < n; ++q) a[(long)r * n + q] -= m * a[(long)c * n + q];
    }
  }
  return 0;
}

static void lu_solve(const double* a, const int* piv, int n, double* x) {
  for (int c = 0; c < n; ++c) {
    const double t = x[c];
    x[c] = x[piv[c]];
    x[piv[c]] = t;
  }
  for (int r = 0; r < n; ++r)
    for (int q = 0; q < r; ++q) x[r] -= a[(long)r * n + q] * x[q];
  for (int r = n - 1; r >= 0; --r) {
    for (int q = r + 1; q < n; ++q) x[r] -= a[(long)r * n + q] * x[q];
    x[r] /= a[(long)r * n + r];
  }
}

static void mg_free(mg_t* m) {
  free(m->lu);
  free(m->piv);
  memset(m, 0, sizeof(*m));
}

static int mg_init(mg_t* m, int nx, int ny, int nz, double h, double chi, double shift, int nu1, int nu2) {
  memset(m, 0, sizeof(*m));
  m->chi = chi;
  m->shift = shift;
  m->singular = shift == 0.0;
  m->nu1 = nu1;
  m->nu2 = nu2;
  int l = 0;
  for (;;) {
    level_t* L = &m->lv[l];
    L->nx = nx, L->ny = ny, L->nz = nz, L->h = h;
    L->n = cells(nx, ny, nz);
    L->x = (double*)scratch(SLOT_LEVEL0 + 3 * l, sizeof(double) * (size_t)L->n);
    L->b = (double*)scratch(SLOT_LEVEL0 + 3 * l + 1, sizeof(double) * (size_t)L->n);
    L->r = (double*)scratch(SLOT_LEVEL0 + 3 * l + 2, sizeof(double) * (size_t)L->n);
    ++l;
    m->nl = l;
    if (!L->x || !L->b || !L->r) return -1;
    if (nx % 2 || ny % 2 || nz % 2 || nx < 4 || ny < 4 || nz < 4 || l == MAX_LEVELS) break;
    nx /= 2, ny /= 2, nz /= 2, h *= 2.0;
  }
  /* dense coarsest operator from unit vectors, plus 1/n everywhere when singular */
  level_t* C = &m->lv[m->nl - 1];
  const int n = (int)C->n;
  if (n > 4096) return -2;
  m->nc = n;
  m->lu = (double*)malloc(sizeof(double) * (size_t)n * n);
  m->piv = (int*)malloc(sizeof(int) * (size_t)n);
  double* e = (double*)calloc((size_t)n, sizeof(double));
  double* col = (double*)malloc(sizeof(double) * (size_t)n);
  if (!m->lu || !m->piv || !e || !col) return -1;
  for (int q = 0; q < n; ++q) {
    e[q] = 1.0;
    apply_level(C, chi, shift, e, col);
    e[q] = 0.0;
    for (int r = 0; r < n; ++r) m->lu[(long)r * n + q] = col[r] + (m->singular ? 1.0 / n : 0.0);
  }
  free(e);
  free(col);
  return lu_factor(m->lu, m->piv, n);
}

static void vcycle_rec(mg_t* m, int l) {
  level_t* L = &m->lv[l];
  if (l == m->nl - 1) {
    memcpy(L->x, L->b, sizeof(double) * (size_t)L->n);
    lu_solve(m->lu, m->piv, m->nc, L->x);
    return;
  }
  for (int s = 0; s < m->nu1; ++s) rb_sweep(L, m->chi, m->shift, L->x, L->b);
  apply_level(L, m->chi, m->shift, L->x, L->r);
#pragma omp parallel for schedule(static)
  for (long c = 0; c < L->n; ++c) L->r[c] = L->b[c] - L->r[c];
  level_t* C = &m->lv[l + 1];
  restrict8(L, L->r, C, C->b);
  vzero(C->x, C->n);
  vcycle_rec(m, l + 1);
  prolong_add(C, C->x, L, L->x);
  for (int s = 0; s < m->nu2; ++s) rb_sweep(L, m->chi, m->shift, L->x, L->b);
}

/* x = one V-cycle on A x = b from x (zero_guess: from x = 0) */
static void vcycle(mg_t* m, const double* b, double* x, int zero_guess) {
  level_t* L = &m->lv[0];
  memcpy(L->b, b, sizeof(double) * (size_t)L->n);
  if (m->singular) vshift(L->b, -vmean(L->b, L->n), L->n);
  if (zero_guess)
    vzero(L->x, L->n);
  else
    memcpy(L->x, x, sizeof(double) * (size_t)L->n);
  vcycle_rec(m, 0);
  if (m->singular) vshift(L->x, -vmean(L->x, L->n), L->n);
  memcpy(x, L->x, sizeof(double) * (size_t)L->n);
}

/* n cycles of multigrid from a zero (or given) guess */
static void vcycles(mg_t* m, const double* b, double* x, int n, int zero_guess) {
  for (int c = 0; c < n; ++c) vcycle(m, b, x, zero_guess && c == 0);
}

/* ----------------------------------------------------------- blobs */
static double peskin4(double r) {
  r = fabs(r);
  if (r < 1.0) return (3.0 - 2.0 * r + sqrt(1.0 + 4.0 * r - 4.0 * r * r)) / 8.0;
  if (r < 2.0) return (5.0 - 2.0 * r - sqrt(-7.0 + 12.0 * r - 4.0 * r * r)) / 8.0;
  return 0.0;
}
static double peskin3(double r) {
  r = fabs(r);
  if (r <= 0.5) return (1.0 + sqrt(1.0 - 3.0 * r * r)) / 3.0;
  if (r < 1.5) return (5.0 - 3.0 * r - sqrt(1.0 - 3.0 * (1.0 - r) * (1.0 - r))) / 6.0;
  return 0.0;
}

typedef struct {
  int n, w;
  int* idx;  /* n x 3 x w wrapped cell indices per axis */
  double* wt; /* n x 3 x w kernel weights per axis */
} blobs_t;

static int blobs_init(blobs_t* B, const double* q, int n, int w, int nx, int ny, int nz, double h) {
  B->n = n, B->w = w;
  B->idx = (int*)malloc(sizeof(int) * (size_t)(n > 0 ? n : 1) * 3 * w);
  B->wt = (double*)malloc(sizeof(double) * (size_t)(n > 0 ? n : 1) * 3 * w);
  if (!B->idx || !B->wt) return -1;
  const int dims[3] = {nx, ny, nz};
  for (int b = 0; b < n; ++b)
    for (int a = 0; a < 3; ++a) {
      const double len = dims[a] * h;
      double p = q[3 * b + a];
      p -= floor(p / len) * len;
      const double u = p / h;
      /* first cell of the support: centres (i + 1/2) h within w/2 cells of u */
      const int i0 = w == 4 ? (int)floor(u - 0.5) - 1 : (int)floor(u) - 1;
      for (int t = 0; t < w; ++t) {
        const int i = i0 + t;
        const double d = u - (i + 0.5);
        B->idx[(b * 3 + a) * w + t] = wrapi(i, dims[a]);
        B->wt[(b * 3 + a) * w + t] = w == 4 ? peskin4(d) : peskin3(d);
      }
    }
  return 0;
}

static void blobs_free(blobs_t* B) {
  free(B->idx);
  free(B->wt);
}

/* out_b = (J c)_b = sum over the support of phi(x) phi(y) phi(z) c */
static void interp(const blobs_t* B, int nx, int ny, const double* c, double* out) {
  const int w = B->w;
#pragma omp parallel for schedule(static)
  for (int b = 0; b < B->n; ++b) {
    const int *ix = B->idx + (b * 3 + 0) * w, *iy = B->idx + (b * 3 + 1) * w, *iz = B->idx + (b * 3 + 2) * w;
    const double *wx = B->wt + (b * 3 + 0) * w, *wy = B->wt + (b * 3 + 1) * w, *wz = B->wt + (b * 3 + 2) * w;
    double s = 0.0;
    for (int c3 = 0; c3 < w; ++c3)
      for (int c2 = 0; c2 < w; ++c2)
        for (int c1 = 0; c1 < w; ++c1)
          s += wz[c3] * wy[c2] * wx[c1] * c[ix[c1] + (long)nx * (iy[c2] + (long)ny * iz[c3])];
    out[b] = s;
  }
}

/* field += a h^-3 sum_b phi phi phi lam_b (S = h^-3 J^T); blobs in order */
static void spread_add(const blobs_t* B, int nx, int ny, double h, double a, const double* lam, double* field) {
  const int w = B->w;
  const double s0 = a / (h * h * h);
  for (int b = 0; b < B->n; ++b) {
    const int *ix = B->idx + (b * 3 + 0) * w, *iy = B->idx + (b * 3 + 1) * w, *iz = B->idx + (b * 3 + 2) * w;
    const double *wx = B->wt + (b * 3 + 0) * w, *wy = B->wt + (b * 3 + 1) * w, *wz = B->wt + (b * 3 + 2) * w;
    for (int c3 = 0; c3 < w; ++c3)
      for (int c2 = 0; c2 < w; ++c2)
        for (int c1 = 0; c1 < w; ++c1)
          field[ix[c1] + (long)nx * (iy[c2] + (long)ny * iz[c3])] += s0 * lam[b] * wz[c3] * wy[c2] * wx[c1];
  }
}

/* ----------------------------------------------------------- FGMRES */
typedef struct solver_s solver_t;
typedef void (*op_fn)(solver_t*, const double* in, double* out);

struct solver_s {
  /* problem */
  int nx, ny, nz, nb;
  long nc;
  double h, chi, alpha, zeta, xi;
  const double* kappa;
  blobs_t B;
  mg_t mg;
  /* options */
  int restart, max_iter, mg_cycles, schur_m;
  double tol;
  /* work */
  double *t1, *t2, *t3, *t4; /* grid-sized scratch */
  double *nv1, *nv2;         /* blob-sized scratch */
  double *sv, *sh, *sz, *sg, *scs, *ssn; /* inner GMRES workspace */
  op_fn apply, precond;
  /* counters */
  long vcycles;
  int outer_iters, inner_iters;
};

/* one V-cycle count-tracked wrapper */
static void mg_solve(solver_t* S, const double* b, double* x, int n, int zero_guess) {
  vcycles(&S->mg, b, x, n, zero_guess);
  S->vcycles += n;
}

/* reaction-limited operator y = A c + S (kappa * J c) */
static void reaction_apply(solver_t* S, const double* c, double* y) {
  apply_level(&S->mg.lv[0], S->chi, S->alpha, c, y);
  interp(&S->B, S->nx, S->ny, c, S->nv1);
  for (int b = 0; b < S->nb; ++b) S->nv1[b] *= S->kappa[b];
  spread_add(&S->B, S->nx, S->ny, S->h, 1.0, S->nv1, y);
}

/* n V-cycles of (sigma I - chi L) from zero */
static void reaction_precond(solver_t* S, const double* r, double* z) { mg_solve(S, r, z, S->mg_cycles, 1); }

/* saddle operator [A c + zeta S lam; xi J c] on the vector [c; lam] */
static void saddle_apply(solver_t* S, const double* v, double* y) {
  apply_level(&S->mg.lv[0], S->chi, S->alpha, v, y);
  spread_add(&S->B, S->nx, S->ny, S->h, S->zeta, v + S->nc, y);
  interp(&S->B, S->nx, S->ny, v, y + S->nc);
  for (int b = 0; b < S->nb; ++b) y[S->nc + b] *= S->xi;
}

/* Schur operator v -> J A~_1^-1 S v (one V-cycle from zero) */
static void schur_apply(solver_t* S, const double* v, double* y) {
  vzero(S->t3, S->nc);
  spread_add(&S->B, S->nx, S->ny, S->h, 1.0, v, S->t3);
  mg_solve(S, S->t3, S->t4, 1, 1);
  interp(&S->B, S->nx, S->ny, S->t4, y);
}

/* m iterations of GMRES (modified Gram-Schmidt) on the N x N Schur system
 * from a zero guess: x = argmin over the Krylov space of ||rhs - M x|| */
static void schur_gmres(solver_t* S, const double* rhs, double* x) {
  const int N = S->nb, m = S->schur_m;
  double* V = S->sv;  /* (m + 1) x N */
  double* H = S->sh;  /* (m + 1) x m, column major: H[i + (m + 1) j] */
  double* g = S->sg;  /* m + 1 */
  double *cs = S->scs, *sn = S->ssn;
  for (int b = 0; b < N; ++b) x[b] = 0.0;
  double beta = 0.0;
  for (int b = 0; b < N; ++b) beta += rhs[b] * rhs[b];
  beta = sqrt(beta);
  if (beta == 0.0) return;
  for (int b = 0; b < N; ++b) V[b] = rhs[b] / beta;
  for (int i = 0; i <= m; ++i) g[i] = 0.0;
  g[0] = beta;
  int k = 0;
  for (int j = 0; j < m; ++j) {
    double* w = V + (long)(j + 1) * N;
    schur_apply(S, V + (long)j * N, w);
    S->inner_iters++;
    for (int i = 0; i <= j; ++i) {
      double d = 0.0;
      for (int b = 0; b < N; ++b) d += w[b] * V[(long)i * N + b];
      H[i + (m + 1) * j] = d;
      for (int b = 0; b < N; ++b) w[b] -= d * V[(long)i * N + b];
    }
    double nw = 0.0;
    for (int b = 0; b < N; ++b) nw += w[b] * w[b];
    nw = sqrt(nw);
    H[j + 1 + (m + 1) * j] = nw;
    for (int i = 0; i < j; ++i) {
      const double a = H[i + (m + 1) * j], bb = H[i + 1 + (m + 1) * j];
      H[i + (m + 1) * j] = cs[i] * a + sn[i] * bb;
      H[i + 1 + (m + 1) * j] = -sn[i] * a + cs[i] * bb;
    }
    const double a = H[j + (m + 1) * j], bb = H[j + 1 + (m + 1) * j];
    const double rr = sqrt(a * a + bb * bb);
    cs[j] = rr > 0.0 ? a / rr : 1.0;
    sn[j] = rr > 0.0 ? bb / rr : 0.0;
    H[j + (m + 1) * j] = rr;
    H[j + 1 + (m + 1) * j] = 0.0;
    g[j + 1] = -sn[j] * g[j];
    g[j] = cs[j] * g[j];
    k = j + 1;
    if (nw == 0.0) break;
    for (int b = 0; b < N; ++b) w[b] /= nw;
  }
  /* y = H^-1 g (upper triangular k x k), x = V y */
  double y[256];
  for (int i = k - 1; i >= 0; --i) {
    double s = g[i];
    for (int q = i + 1; q < k; ++q) s -= H[i + (m + 1) * q] * y[q];
    y[i] = H[i + (m + 1) * i] != 0.0 ? s / H[i + (m + 1) * i] : 0.0;
  }
  for (int i = 0; i < k; ++i)
    for (int b = 0; b < N; ++b) x[b] += y[i] * V[(long)i * N + b];
}

/* Appendix A, steps 1-5, applied to the residual [r_c; r_lam] */
static void saddle_precond(solver_t* S, const double* r, double* z) {
  const long nc = S->nc;
  const int N = S->nb;
  const int singular = S->alpha == 0.0;
  const double* rg = r;
  const double* rf = r + nc;
  double* zc = z;
  double* zl = z + nc;
  double* gt = S->t1; /* g~ */
  double* cs = S->t2; /* c~* */
  /* step 1: g~ = g - zeta S lam0 with lam0 = V_Omega <g> / (zeta N) when
   * singular; c~* = A~_n^-1 g~ from zero */
  memcpy(gt, rg, sizeof(double) * (size_t)nc);
  double lam0 = 0.0;
  if (singular) {
    const double vol = (double)nc * S->h * S->h * S->h;
    lam0 = vol * vmean(rg, nc) / (S->zeta * N);
    for (int b = 0; b < N; ++b) S->nv1[b] = lam0;
    spread_add(&S->B, S->nx, S->ny, S->h, -S->zeta, S->nv1, gt);
  }
  mg_solve(S, gt, cs, S->mg_cycles, 1);
  /* step 2: h~ = xi J c~* - f; solve (J A~_1^-1 S) lam~ = h~ / (zeta xi)
   * approximately by GMRES(m); mean removed when singular */
  interp(&S->B, S->nx, S->ny, cs, S->nv1);
  for (int b = 0; b < N; ++b) S->nv1[b] = (S->xi * S->nv1[b] - rf[b]) / (S->zeta * S->xi);
  schur_gmres(S, S->nv1, zl);
  if (singular) {
    double mu = 0.0;
    for (int b = 0; b < N; ++b) mu += zl[b];
    mu /= N;
    for (int b = 0; b < N; ++b) zl[b] -= mu;
  }
  /* step 3: c~ = A~_n^-1 (g~ - zeta S lam~) from c~* */
  spread_add(&S->B, S->nx, S->ny, S->h, -S->zeta, zl, gt);
  memcpy(zc, cs, sizeof(double) * (size_t)nc);
  mg_solve(S, gt, zc, S->mg_cycles, 0);
  if (singular) {
    /* step 4: cbar = <f / xi - J c~> over the blobs */
    interp(&S->B, S->nx, S->ny, zc, S->nv2);
    double cbar = 0.0;
    for (int b = 0; b < N; ++b) cbar += rf[b] / S->xi - S->nv2[b];
    cbar /= N;
    /* step 5: lam = lam~ + lam0, c = c~ + cbar */
    for (int b = 0; b < N; ++b) zl[b] += lam0;
    vshift(zc, cbar, nc);
  }
}

/* flexible GMRES(restart), MGS, right preconditioning; returns 0 when the
 * true relative residual reached tol, 1 otherwise */
static int fgmres(solver_t* S, long n, const double* b, double* x, double* rel_out) {
  const int m = S->restart;
  double* V = (double*)scratch(SLOT_V, sizeof(double) * (size_t)n * (m + 1));
  double* Z = (double*)scratch(SLOT_Z, sizeof(double) * (size_t)n * m);
  double* r = (double*)scratch(SLOT_R, sizeof(double) * (size_t)n);
  double* H = (double*)calloc((size_t)(m + 1) * m, sizeof(double));
  double* g = (double*)calloc((size_t)(m + 1), sizeof(double));
  double* cs = (double*)calloc((size_t)m, sizeof(double));
  double* sn = (double*)calloc((size_t)m, sizeof(double));
  double* y = (double*)calloc((size_t)m, sizeof(double));
  if (!V || !Z || !r || !H || !g || !cs || !sn || !y) {
    free(H), free(g), free(cs), free(sn), free(y);
    *rel_out = -1.0;
    return -1;
  }
  const double bn = vnorm(b, n);
  int status = 1;
  double rel = 0.0;
  for (;;) {
    /* true residual */
    S->apply(S, x, r);
#pragma omp parallel for schedule(static)
    for (long i = 0; i < n; ++i) r[i] = b[i] - r[i];
    const double beta = vnorm(r, n);
    rel = bn > 0.0 ? beta / bn : 0.0;
    if (rel <= S->tol) {
      status = 0;
      break;
    }
    if (S->outer_iters >= S->max_iter) break;
    vscale_copy(1.0 / beta, r, V, n);
    for (int i = 0; i <= m; ++i) g[i] = 0.0;
    g[0] = beta;
    int k = 0;
    for (int j = 0; j < m && S->outer_iters < S->max_iter; ++j) {
      double* vj = V + (long)j * n;
      double* zj = Z + (long)j * n;
      double* w = V + (long)(j + 1) * n;
      S->precond(S, vj, zj);
      S->apply(S, zj, w);
      S->outer_iters++;
      for (int i = 0; i <= j; ++i) {
        const double d = vdot(w, V + (long)i * n, n);
        H[i + (m + 1) * j] = d;
        vaxpy(-d, V + (long)i * n, w, n);
      }
      const double nw = vnorm(w, n);
      H[j + 1 + (m + 1) * j] = nw;
      for (int i = 0; i < j; ++i) {
        const double a = H[i + (m + 1) * j], bb = H[i + 1 + (m + 1) * j];
        H[i + (m + 1) * j] = cs[i] * a + sn[i] * bb;
        H[i + 1 + (m + 1) * j] = -sn[i] * a + cs[i] * bb;
      }
      const double a = H[j + (m + 1) * j], bb = H[j + 1 + (m + 1) * j];
      const double rr = sqrt(a * a + bb * bb);
      cs[j] = rr > 0.0 ? a / rr : 1.0;
      sn[j] = rr > 0.0 ? bb / rr : 0.0;
      H[j + (m + 1) * j] = rr;
      H[j + 1 + (m + 1) * j] = 0.0;
      g[j + 1] = -sn[j] * g[j];
      g[j] = cs[j] * g[j];
      k = j + 1;
      if (fabs(g[j + 1]) <= S->tol * bn || nw == 0.0) break;
      vscale_copy(1.0 / nw, w, w, n);
    }
    /* x += Z y with H y = g */
    for (int i = k - 1; i >= 0; --i) {
      double s = g[i];
      for (int q = i + 1; q < k; ++q) s -= H[i + (m + 1) * q] * y[q];
      y[i] = H[i + (m + 1) * i] != 0.0 ? s / H[i + (m + 1) * i] : 0.0;
    }
    for (int i = 0; i < k; ++i) vaxpy(y[i], Z + (long)i * n, x, n);
  }
  *rel_out = rel;
  free(H), free(g), free(cs), free(sn), free(y);
  return status;
}

/* ----------------------------------------------------------- entry points */
typedef struct {
  int status;       /* 0 converged, 1 not converged, < 0 setup failure */
  int outer_iters;  /* FGMRES iterations */
  int inner_iters;  /* Schur GMRES iterations (saddle) */
  long vcycles;     /* V-cycles run */
  int threads;      /* OpenMP threads used */
  double rel_residual;
} cpu_info_t;

static int solver_setup(solver_t* S, int nx, int ny, int nz, double h, double chi, double alpha, const double* q,
                        int nb, int w, double shift, int restart, int max_iter, double tol, int mg_cycles, int nu1,
                        int nu2, int schur_m) {
  memset(S, 0, sizeof(*S));
  S->nx = nx, S->ny = ny, S->nz = nz, S->nb = nb, S->nc = cells(nx, ny, nz);
  S->h = h, S->chi = chi, S->alpha = alpha;
  S->restart = restart, S->max_iter = max_iter, S->tol = tol, S->mg_cycles = mg_cycles;
  S->schur_m = schur_m;
  if (restart < 1 || restart > 256 || schur_m < 1 || schur_m > 255 || mg_cycles < 1) return -3;
  if (blobs_init(&S->B, q, nb, w, nx, ny, nz, h)) return -1;
  int rc = mg_init(&S->mg, nx, ny, nz, h, chi, shift, nu1, nu2);
  if (rc) return rc == -1 ? -1 : -2;
  const size_t nc = (size_t)S->nc, nbs = (size_t)(nb > 0 ? nb : 1);
  S->t1 = (double*)scratch(SLOT_T1, nc * sizeof(double));
  S->t2 = (double*)scratch(SLOT_T2, nc * sizeof(double));
  S->t3 = (double*)scratch(SLOT_T3, nc * sizeof(double));
  S->t4 = (double*)scratch(SLOT_T4, nc * sizeof(double));
  S->nv1 = (double*)calloc(nbs, sizeof(double));
  S->nv2 = (double*)calloc(nbs, sizeof(double));
  S->sv = (double*)calloc(nbs * (schur_m + 1), sizeof(double));
  S->sh = (double*)calloc((size_t)(schur_m + 1) * schur_m, sizeof(double));
  S->sg = (double*)calloc((size_t)schur_m + 1, sizeof(double));
  S->scs = (double*)calloc((size_t)schur_m, sizeof(double));
  S->ssn = (double*)calloc((size_t)schur_m, sizeof(double));
  if (!S->t1 || !S->t2 || !S->t3 || !S->t4 || !S->nv1 || !S->nv2 || !S->sv || !S->sh || !S->sg || !S->scs ||
      !S->ssn)
    return -1;
  return 0;
}

static void solver_free(solver_t* S) {
  blobs_free(&S->B);
  mg_free(&S->mg);
  free(S->nv1), free(S->nv2);
  free(S->sv), free(S->sh), free(S->sg), free(S->scs), free(S->ssn);
}

static void fill_info(cpu_info_t* info, int status, const solver_t* S, double rel) {
  info->status = status;
  info->outer_iters = S->outer_iters;
  info->inner_iters = S->inner_iters;
  info->vcycles = S->vcycles;
  info->threads = omp_get_max_threads();
  info->rel_residual = rel;
}

/* Reaction-limited solve; c holds the initial guess on entry (zeros for the
 * paper's start) and the solution on return. */
int cpu_solve_reaction(int nx, int ny, int nz, double h, double chi, double alpha, int kernel_w, const double* q,
                       int nb, const double* kappa, const double* g, double* c, double tol, int restart,
                       int max_iter, int mg_cycles, int nu1, int nu2, int threads, cpu_info_t* info) {
  if (threads > 0) omp_set_num_threads(threads);
  double ksum = 0.0;
  for (int b = 0; b < nb; ++b) ksum += kappa[b];
  const double vol = (double)nx * ny * nz * h * h * h;
  const double sigma = alpha > 0.0 ? alpha : ksum / vol;
  solver_t S;
  int rc = solver_setup(&S, nx, ny, nz, h, chi, alpha, q, nb, kernel_w, sigma, restart, max_iter, tol, mg_cycles,
                        nu1, nu2, 1);
  if (rc || !(sigma > 0.0)) {
    solver_free(&S);
    info->status = rc ? rc : -3;
    return info->status;
  }
  S.kappa = kappa;
  S.apply = reaction_apply;
  S.precond = reaction_precond;
  double rel = 0.0;
  const int st = fgmres(&S, S.nc, g, c, &rel);
  fill_info(info, st, &S, rel);
  solver_free(&S);
  return st;
}

/* Diffusion-limited (saddle-point) solve; x = [c; lambda] holds the initial
 * guess on entry and the solution on return; f may be NULL (zero). */
int cpu_solve_saddle(int nx, int ny, int nz, double h, double chi, double alpha, int kernel_w, const double* q,
                     int nb, const double* g, const double* f, double zeta, double xi, double* x, double tol,
                     int restart, int max_iter, int mg_cycles, int schur_m, int nu1, int nu2, int threads,
                     cpu_info_t* info) {
  if (threads > 0) omp_set_num_threads(threads);
  solver_t S;
  int rc = solver_setup(&S, nx, ny, nz, h, chi, alpha, q, nb, kernel_w, alpha, restart, max_iter, tol, mg_cycles,
                        nu1, nu2, schur_m);
  if (rc || nb < 1) {
    solver_free(&S);
    info->status = rc ? rc : -3;
    return info->status;
  }
  S.zeta = zeta;
  S.xi = xi;
  S.apply = saddle_apply;
  S.precond = saddle_precond;
  const long n = S.nc + nb;
  double* b = (double*)scratch(SLOT_B, sizeof(double) * (size_t)n);
  if (!b) {
    solver_free(&S);
    info->status = -1;
    return -1;
  }
  memcpy(b, g, sizeof(double) * (size_t)S.nc);
  for (int i = 0; i < nb; ++i) b[S.nc + i] = f ? f[i] : 0.0;
  double rel = 0.0;
  const int st = fgmres(&S, n, b, x, &rel);
  fill_info(info, st, &S, rel);
  solver_free(&S);
  return st;
}

/* One V-cycle of A = shift I - chi L on b from x (zero_guess: from 0); for
 * the pin against the NumPy V-cycle. */
int cpu_vcycle(int nx, int ny, int nz, double h, double chi, double shift, int nu1, int nu2, const double* b,
               double* x, int zero_guess, int threads) {
  if (threads > 0) omp_set_num_threads(threads);
  mg_t m;
  const int rc = mg_init(&m, nx, ny, nz, h, chi, shift, nu1, nu2);
  if (rc == 0) vcycle(&m, b, x, zero_guess);
  mg_free(&m);
  return rc;
}
