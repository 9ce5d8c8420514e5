/*
 * ibrd.h -- C ABI of the GB300 reactive-blob reaction-diffusion library.
 *
 * The library solves the linear systems of the minimally-resolved blob model
 * (Bhalla, Griffith, Patankar, Donev; arXiv:1306.3159) on a periodic,
 * cell-centred 3-D grid, entirely on one NVIDIA GB300 GPU:
 *
 *   reaction-limited (Eq. unsteady_system, Eq. steady_state):
 *       (alpha I - chi L + S kappa J) c = g
 *   diffusion-limited saddle point (Eq. saddle_point):
 *       A c + zeta S lambda = g,   xi J c = f,   A = alpha I - chi L
 *
 * with alpha = 1/dt (alpha = 0: steady state), L the 7-point Laplacian
 * (Sec. III.A), J the tensor-product Peskin-kernel averaging operator
 * (Sec. III.A, Eq. tensor_product) and S = h^-3 J^T the spreading operator.
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 * - Grid: n_x x n_y x n_z cells of spacing h; the domain is [0, n h) per axis
 *   and periodic; cell (i, j, k) has centre ((i+1/2)h, (j+1/2)h, (k+1/2)h).
 * - Fields are contiguous FP64 arrays of n_x*n_y*n_z values, index
 *   i + n_x*(j + n_y*k) (x fastest).
 * - Blob arrays are contiguous FP64 arrays of N values, in the order the blobs
 *   were given to ibrd_set_blobs.
 * - Every pointer argument is a DEVICE pointer on the device that was current
 *   when the handle was created, caller-owned, unless its description says
 *   HOST; the library never frees it.
 *   All work is ordered on the stream given to ibrd_grid_create. Entry points
 *   that return a status synchronize that stream only where stated.
 * - No exception crosses the ABI. On failure a call returns a non-zero status;
 *   ibrd_last_error(handle) then returns a message owned by the handle.
 * - A handle is not thread-safe: calls on one handle must not overlap. Calls
 *   on different handles may run at the same time from different host
 *   threads (the batched entry points do so).
 */
#ifndef IBRD_H
#define IBRD_H

#ifdef __cplusplus
extern "C" {
#endif

typedef struct ibrd_grid_s* ibrd_grid;

typedef enum {
  IBRD_OK = 0,
  IBRD_ERR_ARG = 1,            /* invalid argument or size */
  IBRD_ERR_CUDA = 2,           /* a CUDA runtime call failed */
  IBRD_ERR_OOM = 3,            /* device allocation failed */
  IBRD_ERR_NOT_CONVERGED = 4,  /* max_iter reached; best iterate written */
  IBRD_ERR_BREAKDOWN = 5,      /* Krylov breakdown before convergence */
  IBRD_ERR_NONFINITE = 6,      /* NaN/Inf in an input or a residual */
  IBRD_ERR_TIMEOUT = 7,        /* a bounded device wait gave up (see ibrd_set_wait_limit) */
  IBRD_ERR_STATE = 8           /* call needs state not set (e.g. no blobs) */
} ibrd_status;

enum { IBRD_PESKIN4 = 4, IBRD_PESKIN3 = 3 };          /* kernel width w */
enum { IBRD_FP64 = 0, IBRD_MIXED_FP32 = 1, IBRD_MIXED_REFINE = 2 };  /* precision */
/* saddle preconditioner: approximate Schur complement, diagonal (Eq.
   Schur_diagonal), or chosen by blob count (AUTO: diagonal for at most 512
   blobs in the mixed-precision modes and at most 2048 in FP64, where it was
   measured faster at 128^3 and 256^3; approximate Schur above) */
enum { IBRD_PRECOND_SCHUR = 0, IBRD_PRECOND_DIAG = 1, IBRD_PRECOND_AUTO = 2, IBRD_PRECOND_BLOCK = 3 };
enum { IBRD_GUESS_NONE = 0, IBRD_GUESS_UNIFORM = 1, IBRD_GUESS_GIVEN = 2, IBRD_GUESS_PENALTY = 3 }; /* saddle start */

/* Solver options. ibrd_default_opts fills the defaults noted here. */
typedef struct {
  double tol;        /* relative true residual ||b - K x||_2 / ||b||_2 (1e-8) */
  int max_iter;      /* total FGMRES iterations, over all refinement steps of
                        a mixed-precision solve (1000) */
  int restart;       /* FGMRES restart length (30, Sec. III.E Figs. 3, 5) */
  int mg_cycles;     /* n: V-cycles per approximate Helmholtz solve (1) */
  int schur_inner;   /* m: inner Krylov iterations of the approximate Schur
                        preconditioner (5, Sec. III.E / Appendix A) */
  int precond;       /* IBRD_PRECOND_AUTO (default), _SCHUR, _DIAG or _BLOCK.
                        The diagonal preconditioner's gamma = M_11 is computed
                        once per handle (40 FP64 V-cycles on the first blob
                        the first such solve sees) and kept when the blobs
                        change: it depends on the system size and only at the
                        percent level on a blob's position (Sec. III.E).
                        _BLOCK (not in the paper; alpha = 0 only, else it runs
                        as _SCHUR): the approximate Schur preconditioner whose
                        m inner GMRES iterations are left-preconditioned by a
                        sparse approximate inverse P of M = J A^-1 S. Row i of
                        P is row i of the inverse of M restricted to blob i
                        and its neighbours within block_cutoff (at most 31,
                        the nearest), with M_ij for i != j from the periodic
                        Green's function of chi L at the blobs' distance r:
                        1 / (4 pi chi r) + C_box / chi + r^2 / (6 chi V)
                        (C_box = ibrd_periodic_constant of the box) and
                        M_ii = gamma as above. Built on the first such solve
                        after the blobs change. _AUTO: _DIAG up to 512 blobs
                        (2048 in IBRD_FP64), _BLOCK above (_SCHUR when
                        alpha != 0), from timings at 128^3 and 256^3 with
                        m = 5. */
  double zeta;       /* scaling zeta of Eq. saddle_point (1) */
  double xi;         /* scaling xi; <= 0 selects zeta / h^3 (Eq. saddle_point) */
  int nu1, nu2;      /* red-black Gauss-Seidel sweeps before/after (2, 2) */
  int precision;     /* IBRD_FP64: FGMRES on FP64 vectors with FP64 V-cycles.
                        IBRD_MIXED_FP32: FGMRES on FP64 vectors (FP64
                        operator, residual, Arnoldi, dot products and the
                        inner Schur update) preconditioned by FP32 V-cycles
                        and FP32 spreading/interpolation.
                        IBRD_MIXED_REFINE: iterative refinement, each step an
                        FP32 FGMRES solve (FP32 vectors, operator, V-cycles,
                        spreading, inner Schur GMRES) of K d = r for the FP64
                        residual r = b - K x, then x += d in FP64.
                        Every mode stops on the FP64 true residual.
                        -1 = the handle's */
  int use_guess;     /* 1: c (and lambda) hold an initial guess; 0: start at 0 */
  double reorth_eta; /* classical Gram-Schmidt takes a second pass when the
                        orthogonalised vector's norm falls below reorth_eta
                        times its norm before (DGKS test): 1/sqrt(2) (default),
                        0 never, >= 1 always */
  int graphs;        /* 1 (default): replay each preconditioner application
                        from a captured CUDA graph after its first use; 0: launch
                        every kernel directly; 2 (IBRD_MIXED_REFINE): from the
                        second solve of a configuration on, run the whole solve
                        as one CUDA graph whose refinement steps, restart cycles
                        and iterations are conditional nodes decided on the
                        device (no host read until the solve ends; the same
                        iterates as 1, bit for bit) */
  double inner_tol;  /* IBRD_MIXED_REFINE: relative residual each FP32 FGMRES
                        solve aims for, unless less is needed to reach tol
                        (1e-4; the FP32 rounding floor of the operator is
                        near 1e-6 on the grids of Sec. IV) */
  int lambda_guess;  /* saddle solves with use_guess = 0: start from a guess
                        lambda0 of the multipliers instead of zero.
                        IBRD_GUESS_NONE (default): start at 0.
                        IBRD_GUESS_UNIFORM: lambda0_i = h^3 sum(g) / (zeta N).
                        IBRD_GUESS_GIVEN: lambda0 = the incoming lambda (c is
                        ignored), scaled when alpha = 0 so that
                        zeta sum(lambda0) = h^3 sum(g) (the solvability
                        condition of Appendix A; the uniform share if its sum
                        is 0). The grid part of the start is
                        c0 = A~^-1 (g - zeta S lambda0) by warm_cycles V-cycles
                        in the preconditioner's precision plus, when
                        alpha = 0, the constant <f/xi - J c~> (Appendix A
                        steps 3-5 with lambda0 for the Schur solution). The
                        solve then runs to tol as from any other start.
                        IBRD_GUESS_PENALTY: [c0; lambda0] from the penalty
                        form (Sec. II.B: the reaction-limited system with a
                        large rate): c0 solves
                        (A + zeta kappa_p S J) c0 = g + (zeta kappa_p / xi) S f
                        to relative residual penalty_tol (a reaction-limited
                        solve with uniform rate zeta kappa_p, in this solve's
                        precision mode, its V-cycles counted in vcycles), and
                        lambda0 = kappa_p (J c0 - f / xi). */
  int warm_cycles;   /* V-cycles forming c0 of a warm start (2) */
  double penalty_kappa; /* kappa_p of IBRD_GUESS_PENALTY (1000) */
  double penalty_tol;   /* relative residual of its reaction solve (1e-2) */
  double block_cutoff;  /* IBRD_PRECOND_BLOCK: neighbour cutoff, same unit as
                           the positions; <= 0 (default) chooses about 12
                           neighbours per blob at the mean blob density:
                           (9 V / (pi N))^(1/3); at most half the shortest
                           box side */
} ibrd_solve_opts;

/* Solve report. residual_history, if non-NULL, is a caller-owned HOST array
   of history_cap doubles that receives the relative residual estimate after
   each FGMRES iteration (history_len entries are written); in a
   mixed-precision solve an entry is the FP32 solve's estimate times the FP64
   relative residual its refinement step started from. */
typedef struct {
  int status;          /* same value the solve returned */
  int outer_iters;     /* FGMRES iterations (all refinement steps) */
  int inner_iters;     /* inner Schur Krylov iterations (saddle) */
  int vcycles;         /* V-cycles applied (the paper's cost proxy, Sec. III.E) */
  int reorths;         /* Gram-Schmidt second passes taken */
  double rel_residual; /* final relative true residual */
  double sum_lambda;   /* sum_i lambda_i (saddle) or sum_i kappa_i (J c)_i */
  double cbar;         /* mean of c over all cells (Sec. IV.A) */
  double rate_K;       /* K = sum_i lambda_i / (N cbar) (Sec. I.A) */
  double seconds;      /* wall time of the solve on the host clock */
  double* residual_history;
  int history_len;
  int history_cap;
  int refinements;     /* IBRD_MIXED_REFINE: refinement steps (FP32 solves) */
  double a_L;          /* reaction radius a_L = K / (4 pi chi) (Sec. IV.A) */
  int precond;         /* saddle solves: the preconditioner that ran
                          (IBRD_PRECOND_SCHUR, _DIAG or _BLOCK); -1 for reaction
                          solves */
} ibrd_solve_info;

/* Fill *opts with the defaults listed in ibrd_solve_opts. */
void ibrd_default_opts(ibrd_solve_opts* opts);

/* Create a handle for an n_x x n_y x n_z periodic grid (each side >= 4) with
   spacing h > 0, diffusion coefficient chi > 0 (Sec. I.A) and shift
   alpha >= 0 (alpha = 1/dt of Eq. unsteady_system; 0 = steady state,
   Eq. steady_state). kernel is IBRD_PESKIN4 (Sec. III.A, Delta V = (8/3)^3 h^3)
   or IBRD_PESKIN3 (Delta V = 8 h^3). precision is the default precision of
   solves. stream is a cudaStream_t (NULL = legacy default stream). The
   multigrid hierarchy halves every side while all sides are even and >= 4;
   the coarsest level must hold at most 512 cells (else IBRD_ERR_ARG).
   On success *out owns device workspaces until ibrd_grid_destroy. */
ibrd_status ibrd_grid_create(ibrd_grid* out, int nx, int ny, int nz, double h, double chi,
                             double alpha, int kernel, int precision, void* stream);

/* Release a handle and all its device memory. NULL is ignored. */
void ibrd_grid_destroy(ibrd_grid g);

/* Set the blob configuration Q = {q_1..q_N} (Sec. II.A): q is a device array
   of N x 3 FP64 values (x, y, z per blob, AoS). Positions are wrapped into the
   periodic box. Computes each blob's 1-D kernel weights and bins blobs by
   8 x 8 x 8 cell tile for spreading. N >= 0; N = 0 clears the blobs.
   Synchronizes the stream (it reads back the number of occupied tiles). */
ibrd_status ibrd_set_blobs(ibrd_grid g, const double* q, int n_blobs);

/* y = A c = alpha c - chi L c (Sec. III.A, Eq. Helmholtz). c and y must not
   overlap. */
ibrd_status ibrd_apply_L(ibrd_grid g, const double* c, double* y);

/* r = rhs - A c (Sec. III.A, Eq. Helmholtz), the grid part of every FP64
   residual the solvers form (each refinement step's, each restart's, for
   tolerances of 1e-13 and above). On grids with nx a multiple of 32 and ny a
   multiple of 8, while the largest |c| lies in [2^-900, 2^900]: c scaled by a
   power of two into 64-bit integers, so that L c (the neighbour sums) is
   exact, then r = fma(-alpha, c, fma(chi / h^2 2^-S, L c, rhs)) -- within
   2^-52 of |r| + |alpha c| + chi / h^2 |L c| per cell plus 2^-55 chi / h^2
   max|c|, where the FP64 form rounds terms of size 6 chi / h^2 |c| -- with
   one or two FP64 instructions per cell (GB300's FP64 pipe issues about two
   per SM per clock). Elsewhere the FP64 form. Non-finite c gives non-finite
   r. All fields device, N_c doubles, non-overlapping; asynchronous on the
   handle's stream. */
ibrd_status ibrd_residual(ibrd_grid g, const double* rhs, const double* c, double* r);

/* One multigrid V-cycle (FP64) for A x = rhs (Sec. III.E): red-black
   Gauss-Seidel (nu1 = nu2 = 2), 8-cell-mean restriction, trilinear
   cell-centred prolongation, exact coarsest solve. With alpha = 0 the
   right-hand side is projected to mean zero and the result is returned with
   mean zero (the restricted inverse of Appendix A). zero_initial_guess != 0
   ignores the incoming x. rhs and x must not overlap. */
ibrd_status ibrd_vcycle(ibrd_grid g, const double* rhs, double* x, int zero_initial_guess);

/* ibrd_vcycle for callers that cannot allocate device memory (no counterpart
   in the paper: it is a packaging of the V-cycle above). Some callers may not
   call cudaMalloc at all: code running under a device-memory budget fixed at
   start-up, code inside another library that may only use the memory it is
   handed, or a process whose device memory already belongs to a framework's
   caching allocator. This entry point needs no grid handle and allocates
   nothing: the V-cycle's workspaces come from one 16 MiB scratch array in
   static device memory, which a GPU holds from the first call on it until the
   process exits. Under CUDA's default lazy module loading the array is
   reserved on a device by that first call, not when the library is loaded: a
   caller whose memory budget is fixed at start-up must make one call on each
   device before it locks the budget (or set CUDA_MODULE_LOADING=EAGER so the
   array is reserved when the library's module is loaded). If that
   reservation fails the call returns IBRD_ERR_OOM. The size limits the grid
   to about 1.4 million cells (96^3 and 112^3 fit; 120^3 and 128^3 do not);
   larger grids return IBRD_ERR_ARG without any GPU work. The grid, h, chi and alpha are passed directly; rhs and x are
   caller-owned device arrays as for ibrd_vcycle (rhs != x), and the result is
   the one ibrd_vcycle computes. stream is a cudaStream_t (NULL = legacy
   default stream); the call only enqueues work on it and does not synchronize.
   The first call on a device looks up the scratch array's device address
   (cudaGetSymbolAddress) once, with that device current; make that first call
   before any stream capture. Every call uses the same scratch and leaves its
   contents behind (nothing in it is read before the call writes it), so calls
   whose GPU work overlaps (different streams or host threads, same device)
   race on it: serialize them. The scratch address is cached per device for
   the process, so do not call this entry point on a device after a
   cudaDeviceReset of it. Returns IBRD_ERR_CUDA if a CUDA call fails
   (IBRD_ERR_OOM for an allocation failure). */
ibrd_status ibrd_vcycle_noalloc(int nx, int ny, int nz, double h, double chi, double alpha, const double* rhs,
                                double* x, int zero_initial_guess, void* stream);

/* The V-cycle with FP32 fields and FP32 arithmetic (the multigrid used inside
   the mixed-precision solves). Its hierarchy ends at the first level with at
   most 32768 cells and no side above 64, which is solved exactly by the
   separable Hartley transform (pseudo-inverse when alpha = 0); without such a
   level it coarsens like the FP64 V-cycle. rhs, x: FP32 device fields. */
ibrd_status ibrd_vcycle_f32(ibrd_grid g, const float* rhs, float* x, int zero_initial_guess);

/* ibrd_vcycle_f32 with nu1 pre- and nu2 post-smoothing sweeps (0 to 16 each;
   ibrd_vcycle_f32 uses 2 and 2): the V-cycle the mixed-precision solves run
   with the ibrd_solve_opts sweep counts. Same arguments and errors. */
ibrd_status ibrd_vcycle_f32_sweeps(ibrd_grid g, const float* rhs, float* x, int zero_initial_guess, int nu1,
                                   int nu2);

/* grid_out (+)= S lambda, (S lambda)_k = h^-3 sum_i phi(q_i - r_k) lambda_i
   (Sec. III.A). accumulate = 0 overwrites grid_out (zero away from blobs).
   Deterministic: each cell sums its blobs in increasing blob index. */
ibrd_status ibrd_spread(ibrd_grid g, const double* lambda, double* grid_out, int accumulate);

/* out_n = J c, (J c)_i = sum_k phi(q_i - r_k) c_k (Sec. III.A). */
ibrd_status ibrd_interp(ibrd_grid g, const double* c, double* out_n);

/* Solve (alpha I - chi L + S diag(kappa) J) c = g (Eq. unsteady_system; with
   alpha = 0, Eq. steady_state) by right-preconditioned flexible GMRES whose
   preconditioner is opts->mg_cycles V-cycles of (sigma I - chi L), sigma =
   alpha if alpha > 0 else sum_i kappa_i / V_Omega (Sec. III.E,
   Eq. Pinv_Poisson). kappa: N rates >= 0 (device). g: source field. c: in
   (if opts->use_guess) / out. With alpha = 0 at least one kappa_i must be
   positive. info may be NULL. Synchronizes the stream. */
ibrd_status ibrd_solve_reaction(ibrd_grid g, const double* kappa, const double* rhs, double* c,
                                const ibrd_solve_opts* opts, ibrd_solve_info* info);

/* Solve the saddle point A c + zeta S lambda = g, xi J c = f (Eq. saddle_point)
   by flexible GMRES on [c; lambda] preconditioned with the approximate Schur
   complement (or diagonal) preconditioner of Sec. III.E and Appendix A,
   including its null-space handling when alpha = 0. f may be NULL (f = 0).
   c, lambda: in (if opts->use_guess) / out. Requires N >= 1. info may be NULL.
   Synchronizes the stream. */
ibrd_status ibrd_solve_saddle(ibrd_grid g, const double* rhs, const double* f, double* c,
                              double* lambda, const ibrd_solve_opts* opts, ibrd_solve_info* info);

/* Batched solves: count independent problems, problem i on handle grids[i]
   with its own grid size, blobs and stream (e.g. the disordered suspensions of
   Sec. IV.B, one realisation per handle). Each problem is solved exactly as
   the single-problem call would solve it, with the same result. The library
   runs the solves on `threads` host threads of its own (<= 0: 16; never more
   than count or 64), taking the problems with the most cells and blobs first;
   solves on handles whose streams differ (give each handle its own
   non-blocking stream) overlap on the GPU. Handles must be distinct and
   non-NULL (else IBRD_ERR_ARG before any work). kappa, rhs, f, c and lambda
   are HOST arrays of count device pointers, entry i meaning what the
   single-problem argument means for problem i; f may be NULL (all f = 0), as
   may any f[i]. opts (shared by all problems) may be NULL. infos, if non-NULL,
   is an array of count reports; infos[i].status is set for every problem,
   also when its solve fails. Returns the first non-OK status in index order
   (every problem is still attempted); the message is on that problem's
   handle. Returns after every solve has finished and synchronized its
   stream. */
ibrd_status ibrd_solve_reaction_batch(int count, const ibrd_grid* grids, const double* const* kappa,
                                      const double* const* rhs, double* const* c,
                                      const ibrd_solve_opts* opts, ibrd_solve_info* infos, int threads);

ibrd_status ibrd_solve_saddle_batch(int count, const ibrd_grid* grids, const double* const* rhs,
                                    const double* const* f, double* const* c, double* const* lambda,
                                    const ibrd_solve_opts* opts, ibrd_solve_info* infos, int threads);

/* Independent solves of either kind at once: item i is a reaction-limited
   (kind IBRD_SOLVE_REACTION: kappa, rhs, c) or saddle-point (kind
   IBRD_SOLVE_SADDLE: rhs, f (may be NULL), c, lambda) solve on its own handle
   with its own options (opts may be NULL) and report (info may be NULL; its
   status is set for every item). The pointers mean what they mean in
   ibrd_solve_reaction / ibrd_solve_saddle. If q is non-NULL the item first
   sets the handle's blobs (ibrd_set_blobs(grid, q, n_blobs)). If c_host
   (lambda_host) is non-NULL, a HOST buffer of N_c (N) doubles (pinned for an
   asynchronous copy), the solution is copied there on the handle's stream
   after the solve, before the item ends, so that one item's download
   overlaps the others' solves. Scheduling, handle rules and the return value
   are those of the batched calls above; e.g. the two solves of one
   configuration (Sec. III.C and III.D) on two handles with their own streams
   overlap on the GPU. items is a HOST array. */
enum { IBRD_SOLVE_REACTION = 0, IBRD_SOLVE_SADDLE = 1 };
typedef struct {
  int kind;
  ibrd_grid grid;
  const double* kappa;
  const double* rhs;
  const double* f;
  double* c;
  double* lambda;
  const ibrd_solve_opts* opts;
  ibrd_solve_info* info;
  const double* q;     /* blob positions to set first (device, n_blobs x 3), or NULL */
  int n_blobs;
  double* c_host;      /* host destination of c after the solve, or NULL */
  double* lambda_host; /* host destination of lambda (saddle), or NULL */
} ibrd_solve_item;

ibrd_status ibrd_solve_many(int count, const ibrd_solve_item* items, int threads);

/* Autotuner (not in the paper: launch-shape selection for this library's
   kernels). For every multigrid level whose red-black sweeps (Sec. III.E) run
   as a fused one-pass sweep kernel, times candidate launch shapes of the
   sweep -- the row-resident FP32 kernel (levels whose rows are 128 or 256
   cells; tx = nx) or the tiled kernel with tile width 32 or 64 cells (FP32)
   or 32 (FP64), each with z-march depths (planes per CTA, 2 to 512) -- and
   the z-march depth of the stencil pass that forms the first
   sweep from a zero guess (FP32), on scratch fields of the level's size with
   CUDA events, and keeps a shape only when it is at least 3 % faster than the
   built-in one. Shapes tuned before in this process for the same device and
   grid are reused without timing unless retune != 0. Every later call on the
   handle launches the kept shapes; results can change in the last bits only
   (per-CTA partial sums group differently). Drops the handle's captured CUDA
   graphs. precision: IBRD_FP64 tunes the FP64 kernels, either mixed mode the
   FP32 ones, -1 both. out (may be NULL if cap = 0) receives up to cap
   records; *n_out (may be NULL) the number of records. Allocates six
   scratch fields of the finest grid for the duration of the call (two sets
   of x in, x out and b that consecutive timed sweeps alternate between, so
   that levels larger than half the L2 stream from DRAM as in a V-cycle).
   Synchronizes the stream. */
typedef struct {
  int nx, ny, nz;    /* level grid */
  int elem_bytes;    /* 4 (FP32) or 8 (FP64) */
  int kind;          /* 0: fused sweep; 1: stencil pass of a sweep from zero */
  int tx, zc;        /* kept tile width (0: built-in; nx: row-resident kernel) and z-march depth (0: built-in) */
  double us_default; /* average launch time of the built-in shape, microseconds */
  double us_tuned;   /* average launch time of the kept shape */
  int cached;        /* 1: reused from an earlier tuning in this process */
} ibrd_tune_entry;

ibrd_status ibrd_autotune(ibrd_grid g, int precision, int retune, ibrd_tune_entry* out, int cap, int* n_out);

/* The constant C of the zero-mean periodic Green's function of -Laplace in a
   box lx x ly x lz (all > 0): G(r) = 1 / (4 pi r) + C + r^2 / (6 V) + ... for
   small r. For a cube of side L, C = -2.837297 / (4 pi L): the constant of
   the finite-size correction of the reaction radius (Sec. IV.A, Eq. a_phi).
   By an Ewald sum to double precision (image and reciprocal shells per axis
   from the box's shape). Host only; NaN for a non-positive side. */
double ibrd_periodic_constant(double lx, double ly, double lz);

/* Set one launch shape by hand (as ibrd_autotune would keep it): elem_bytes
   4 or 8, kind 0 or 1 as in ibrd_tune_entry, (nx, ny, nz) a level of the
   handle's hierarchy, tx in {0, 32, 64} or tx = nx (0 for kind 1; 64 only
   for FP32 and when 64 divides nx, else ignored; nx selects the row-resident
   FP32 sweep on levels whose rows are 128 or 256 cells, ny a multiple of 8
   and nz even), zc >= 0 (0 = built-in; clamped to the level's nz).
   kind 2 (FP32 only, zc = 0) is the coarse-grid correction of the level: on
   levels the row-resident sweep serves, the V-cycle adds the prolongation of
   the coarse correction inside the first post-smoothing sweep (one pass over
   x instead of two; the same values bit for bit); tx = 1 keeps it a separate
   kernel, tx = 0 restores the default. Drops the handle's captured CUDA
   graphs. */
ibrd_status ibrd_tune_set(ibrd_grid g, int elem_bytes, int kind, int nx, int ny, int nz, int tx, int zc);

/* Bound on the device waits of this handle's kernels (not in the paper). The
   row-resident FP32 sweep waits in every plane step for its TMA copies on an
   mbarrier; each wait makes at most `tries` polls (mbarrier try_wait, each of
   which may suspend the thread for a short hardware-defined time) before it
   gives up. A wait that gives up makes its CTA wait (with a fixed larger
   bound) for its copies still in flight and stop; the launch's output is then
   incomplete, and the solve that ran it returns IBRD_ERR_TIMEOUT (its
   iterate is not a solution), as does ibrd_vcycle / ibrd_vcycle_f32 when the
   stream is not being captured. Default 2^24 polls, far beyond any copy's
   latency; 0 makes every such wait give up at once (for testing the error
   path; no wait ever spins without bound). */
ibrd_status ibrd_set_wait_limit(ibrd_grid g, unsigned tries);

/* Forget the handle's tuned shapes (back to the built-in ones); drops its
   captured CUDA graphs. */
ibrd_status ibrd_tune_clear(ibrd_grid g);

/* ---------------------------------------------------------------------
   Learned multiplier predictor (not in the paper). The paper leaves a good
   treatment of the Schur complement J A^-1 S of the saddle point for many
   blobs open (Sec. III.E, Sec. V). This is a small graph network over each
   blob's neighbours (minimum-image distance below the cutoff in the periodic
   box) that predicts the relative sink strengths lambda_i / <lambda>, used as
   the initial guess of the multipliers (ibrd_solve_opts.lambda_guess =
   IBRD_GUESS_GIVEN). Definition, with s = r / R, f_c = (1 - s)^2 and K = 16
   radial bases b_k = f_c exp(-((s - k/15) / 0.1)^2), width 64, L = 3
   message-passing layers:
     x_i = sum_j b(r_ij);  h0_i = relu(W0 x_i + c0);
     for l = 1 .. 3:
       m_i = sum_j f_c(r_ij) relu(E_l b(r_ij) + e_l) * h_{l-1,j} (elementwise);
       h_{l,i} = h_{l-1,i} + relu(W_l m_i + V_l h_{l-1,i} + c_l);
     y_i = o . h_{3,i} + o0;  lambda0_i = total exp(y_i) / sum_k exp(y_k).
   Training minimises <((y - <y>) - (t - <t>))^2>, t_i = log lambda_i, over
   (configuration, lambda) pairs from saddle solves, by Adam (beta 0.9,
   0.999, eps 1e-8). Parameters are FP32, in the order W0 (64 x 16, row
   major), c0 (64), then per layer l = 1, 2, 3: E_l (64 x 16), e_l (64), W_l
   (64 x 64), V_l (64 x 64), c_l (64); then o (64), o0 (1). Training,
   ibrd_gnn_loss_grad and ibrd_gnn_forward compute in FP32;
   ibrd_gnn_predict runs the products E_l b, W_l m and V_l h on the tensor
   cores with bfloat16 operands (the FP32 values rounded to nearest, ties to
   even) and FP32 accumulation, everything else in FP32.
   Positions q are DEVICE arrays of n x 3 FP64 values (as for
   ibrd_set_blobs) in a periodic box lx x ly x lz, within 100 box lengths of
   the origin; the cutoff must not exceed half the shortest side. A blob with more than max_neighbours neighbours
   makes the call fail with IBRD_ERR_ARG. Multipliers lam must be > 0. Every
   call orders its work on the handle's stream and synchronizes it. */
typedef struct ibrd_gnn_s* ibrd_gnn;

/* Number of parameters (29185). */
int ibrd_gnn_num_params(void);

/* New model with all parameters 0 (set them with ibrd_gnn_set_params).
   cutoff > 0 (same length unit as positions), 1 <= max_neighbours <= 1024. */
ibrd_status ibrd_gnn_create(ibrd_gnn* out, double cutoff, int max_neighbours, void* stream);
void ibrd_gnn_destroy(ibrd_gnn m);
const char* ibrd_gnn_last_error(ibrd_gnn m);

/* theta: HOST array of ibrd_gnn_num_params() FP32 values. reset_optimizer != 0
   also zeroes Adam's moments and step count. */
ibrd_status ibrd_gnn_set_params(ibrd_gnn m, const float* theta, int reset_optimizer);
ibrd_status ibrd_gnn_get_params(ibrd_gnn m, float* theta);

/* Seeded initial parameters: every weight matrix (and o) uniform in
   +-1/sqrt(fan in) from a splitmix64 stream started at seed, biases 0; zeroes
   Adam's state. */
ibrd_status ibrd_gnn_init_params(ibrd_gnn m, unsigned long long seed);

/* Neighbour lists of a configuration (DEVICE outputs): count[n], index[n x
   max_neighbours] (increasing j, then unused), dist[n x max_neighbours] (FP32
   distances; the neighbour sets follow the FP64 minimum-image distance, a
   stored distance may be the FP32 one, within a few ulps of the box side). */
ibrd_status ibrd_gnn_neighbours(ibrd_gnn m, const double* q, int n, double lx, double ly, double lz, int* count,
                                int* index, float* dist);

/* y (DEVICE, n FP32 values): the network's outputs (FP32 arithmetic). */
ibrd_status ibrd_gnn_forward(ibrd_gnn m, const double* q, int n, double lx, double ly, double lz, float* y);

/* lambda0 (DEVICE, n FP64 values) = total * softmax(y), y from the
   bfloat16 tensor-core inference path. */
ibrd_status ibrd_gnn_predict(ibrd_gnn m, const double* q, int n, double lx, double ly, double lz, double total,
                             double* lambda0);

/* Loss of one configuration with multipliers lam (DEVICE, n FP64 values) into
   *loss (host, may be NULL) and its gradient into grad (DEVICE, num_params FP32
   values, may be NULL). Parameters unchanged. */
ibrd_status ibrd_gnn_loss_grad(ibrd_gnn m, const double* q, int n, double lx, double ly, double lz,
                               const double* lam, double* loss, float* grad);

/* One Adam step with gradient grad (DEVICE) and learning rate lr > 0. */
ibrd_status ibrd_gnn_adam_step(ibrd_gnn m, const float* grad, double lr);

/* epochs passes over count configurations in index order, one Adam step per
   configuration. q[c], lam[c]: DEVICE arrays; n[c]: blob counts (HOST);
   boxes: HOST array of 3 count box sides; epoch_loss (HOST, may be NULL):
   mean loss of each epoch (losses before each step). */
ibrd_status ibrd_gnn_train(ibrd_gnn m, int count, const double* const* q, const int* n, const double* boxes,
                           const double* const* lam, int epochs, double lr, double* epoch_loss);

/* Launch profiler (not in the paper: instrumentation of this library).
   Every kernel the library launches is counted per kernel class; with timing
   enabled each launch is also bracketed by CUDA events on the handle's stream,
   which adds a few microseconds of host time per launch. */
#define IBRD_PROF_NCLASS 19
typedef struct {
  long long launches;                 /* kernels launched since the last reset */
  int nclass;                         /* number of classes filled (<= IBRD_PROF_NCLASS) */
  int overflow;                       /* 1 if the event pool ran out (times partial) */
  long long count[IBRD_PROF_NCLASS];  /* launches per class */
  long long timed[IBRD_PROF_NCLASS];  /* timed launches per class */
  double ms[IBRD_PROF_NCLASS];        /* summed event time per class, milliseconds */
  double bytes[IBRD_PROF_NCLASS];     /* summed algorithmic bytes per class: each
                                         input read once, each output written once */
  double max_launch_bytes[IBRD_PROF_NCLASS]; /* largest single launch of the class */
  double timed_bytes[IBRD_PROF_NCLASS];      /* algorithmic bytes of the timed launches */
} ibrd_profile;

/* Time the launches of every class c with bit c set in class_mask (0 turns
   timing off) whose algorithmic bytes are >= min_bytes (e.g. only the finest
   multigrid level). Counting is always on. */
ibrd_status ibrd_profile_enable(ibrd_grid g, unsigned class_mask, double min_bytes);

/* Synchronize the handle's stream and report counts and times since the last
   reset; reset != 0 clears them. */
ibrd_status ibrd_profile_read(ibrd_grid g, ibrd_profile* out, int reset);

/* Static name of profiler class cls ("" if out of range). */
const char* ibrd_profile_class_name(int cls);

/* Message of the last failed call on this handle ("" if none). */
const char* ibrd_last_error(ibrd_grid g);

/* Static name of a status code. */
const char* ibrd_status_string(int status);

#ifdef __cplusplus
}
#endif
#endif /* IBRD_H */
