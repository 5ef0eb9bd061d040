/*
 * klecgc.h - C ABI of the GB300 (sm_103a) KLE-PCGC solver.
 *
 * The library evaluates, for a batch of random-input samples xi, the online
 * part of Algorithm 3 of "A parallel solver for random input problems via
 * Karhunen-Loeve expansion and diagonalized coarse grid correction"
 * (arXiv 2510.26180): the KL/gPC surrogate initial guess (Algorithm 3,
 * step 6), then parareal iterations with the alpha-circulant diagonalized
 * coarse grid correction (Algorithm 2; Section 3.2, eqs. PGC_step1,
 * PGC_step2, matrix_NT, Newton2, three steps).
 *
 * Problem (eq. psys with f(u) = div(a grad u) - c u + f0, Section 4.1
 * eq. ODE): zero Dirichlet data on (0,1)^dim, a(x; xi) = exp(g(x; xi)),
 * g = sum_m sqrt(lambda_m) phi_m(x) xi_m the KL expansion of a Gaussian
 * field with covariance sigma^2 exp(-|x - y| / corr_len).  Both propagators
 * are backward Euler (Section 5): G with step dT, F with J steps dT/J.
 * Variants selected by klecgc_problem: a 2D upwind convection b . grad u
 * with b = b0 (x2, x1) (advection-diffusion, Section 5), and the nonlinear
 * reactions of reaction_kind 1 (cubic, Allen-Cahn type) and 2 (convection
 * (u^2/2)_x, Burgers type) with Newton propagators and the simplified-Newton
 * CGC (Section 3.2).  The offline part of Algorithm 3 (snapshots, snapshot
 * KL, gPC least squares) runs in klecgc_setup, on the device.
 *
 * Conventions shared by every entry point
 *  - Every array is owned by the caller.  The library owns the context and
 *    the device tables and scratch it allocates inside it.
 *  - Array arguments may be host or device pointers (CUDA unified
 *    addressing decides which); host arrays are staged through the
 *    library's device scratch on the given stream.
 *  - `stream` is a cudaStream_t (NULL = legacy default stream).  Work is
 *    enqueued on it; every entry point returns after that work has
 *    completed, so the returned status is final.
 *  - Layouts are row-major.  A solution batch U has shape [S][N][nx^dim]:
 *    U[s][n][i] approximates u(x_i, T_{n+1}) for n = 0..N-1 (U_1..U_N of the
 *    paper), x_i the interior grid points in lexicographic order (2D:
 *    i = iy*nx + ix for the point ((ix+1)h, (iy+1)h)).
 *  - dim = 2 uses the five-point flux-form operator with the coefficient at
 *    the edge midpoints; its linear systems (the backward-Euler steps of F
 *    and the shifted CGC systems of eq. three steps (b)) are solved by
 *    Jacobi-preconditioned CG / COCG (BiCGStab with convection) to a
 *    relative residual (see klecgc_set_krylov), or, in FP64 on grids with
 *    nx <= 32 (64 on request), by banded LU factorizations made once per
 *    call (see klecgc_set_2d_method).  2D takes
 *    precision KLECGC_FP64 (FP64 Krylov solves) or KLECGC_MIXED (each step of
 *    F by FP64 iterative refinement around an FP32 Jacobi-PCG: the residual
 *    is kept in FP64, so the result meets the same FP64 residual test; the
 *    shifted CGC systems likewise around an FP32 COCG); it has no learned
 *    guess.
 *  - No exception crosses the ABI and no device trap is used: every error
 *    is a status code; klecgc_last_error() returns a one-line detail for
 *    the calling thread.
 */
#ifndef KLECGC_H
#define KLECGC_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct klecgc_ctx klecgc_ctx;

typedef enum {
    KLECGC_OK = 0,
    KLECGC_E_INVALID_ARG = 1,   /* an argument is out of range or inconsistent */
    KLECGC_E_OUT_OF_MEMORY = 2, /* a device allocation failed */
    KLECGC_E_NOT_CONVERGED = 3, /* some sample did not reach tol in kmax iterations */
    KLECGC_E_NONFINITE = 4,     /* NaN/Inf in an input or an iterate */
    KLECGC_E_CUDA = 5,          /* a CUDA runtime call failed */
    KLECGC_E_UNSUPPORTED = 6    /* valid, but not implemented (e.g. N not a power of 2) */
} klecgc_status;

/* Arithmetic of klecgc_solve. */
enum {
    /* Everything in FP64. */
    KLECGC_FP64 = 0,
    /* Fine propagator in FP32 (increment form, see below); jump, CGC,
       update and convergence norm in FP64. */
    KLECGC_MIXED = 1,
    /* Fine propagator in FP32 (increment form); the CGC is applied in FP32 to
       the FP64 defect F(U^k) - U^k (defect-correction form of Algorithm 2,
       algebraically identical); update and convergence norm in FP64. */
    KLECGC_MIXED_DEFECT = 2
};

/* Initial guess U^0 of klecgc_solve. */
enum {
    KLECGC_GUESS_GPC = 0,   /* KL + gPC surrogate (Algorithm 3, step 6) */
    KLECGC_GUESS_ZERO = 1,  /* U^0 = 0 */
    KLECGC_GUESS_USER = 2,  /* U^0 given by the caller in U_guess */
    KLECGC_GUESS_COARSE = 3, /* U^0_n = G(U^0_{n-1}), U^0_0 = u0 (Section 3.1) */
    KLECGC_GUESS_MLP = 4     /* learned network (klecgc_mlp_*); the gPC surrogate is its
                                fallback when an output is not finite */
};

typedef struct {
    int32_t dim;          /* space dimension: 1 or 2 ((0,1)^2, nx <= 2047) */
    int32_t nx;           /* interior points per direction, h = 1/(nx+1) */
    double T;             /* final time */
    double sigma;         /* std-dev of the Gaussian log-coefficient g */
    double corr_len;      /* correlation length of exp(-|x-y|/corr_len) */
    int32_t M;            /* input KL terms (length of xi) */
    int32_t gpc_degree;   /* total degree p of the Hermite gPC basis */
    int32_t n_train;      /* |Xi_t|, training samples of the surrogate */
    double eps_kl;        /* snapshot-KL energy tolerance eps^KL */
    int32_t N;            /* coarse intervals of the surrogate's time grid */
    int32_t J;            /* fine steps per interval used for the snapshots */
    double reaction;      /* c >= 0 in div(a grad u) - c u + f0 */
    double forcing;       /* f0 (constant source) */
    int32_t u0_kind;      /* 0: u0 = sin(pi x) (product of sines in 2D); 1: u0 = 0;
                             2 (2D): u0 = sin(pi x1) sin(2 pi x2) */
    int32_t reaction_kind; /* 0: linear reaction -c u; 1: cubic -c (u^3 - u)
                              (Allen-Cahn type); 2: convection -c (u^2/2)_x,
                              Engquist-Osher upwind (Burgers type); 1 and 2
                              are 1D and FP64 (see klecgc_solve) */
    int32_t cgc_newton;    /* simplified Newton steps per CGC for reaction_kind
                              1 and 2 (eq. Newton2); 0 means 1 */
    double advection;      /* b0 >= 0 of the convection b . grad u, b = b0 (x2, x1)
                              (advection-diffusion, Section 5), first-order
                              upwind; 2D, reaction_kind 0, FP64 only; 0: none */
} klecgc_problem;

typedef struct {
    int32_t nx, N, J, M, P;   /* P = number of gPC basis functions */
    int32_t MQ;               /* retained snapshot-KL modes (Algorithm 3, step 2) */
    double lambda_sum;        /* sum of all snapshot-KL eigenvalues */
    double lambda_kept;       /* sum of the retained ones */
    int32_t n_unknowns;       /* nx^dim */
    int32_t device;           /* CUDA device of the context */
} klecgc_info_t;

/*
 * klecgc_setup - offline part of Algorithm 3 (steps 1-6).
 *   1. input-field KL eigenpairs of the exponential covariance (roots of
 *      the transcendental equations), coefficient field at the cell faces;
 *   2. snapshots: the sequential fine solution (the paper's reference
 *      solution) at the N coarse times for every xi in Xi_t;
 *   3. snapshot mean, covariance C (Section 2.1), its eigenpairs and M_Q:
 *      the smallest M_Q capturing a fraction >= 1 - eps_kl of the energy
 *      (Algorithm 3 step 2 prints "<="; read as ">="), at most n_train-1;
 *   4. modes g_k (eq. KLE basis) and coefficients zeta_k (eq. KLE parameter);
 *   5. least squares h = argmin ||B h - D|| per mode (eq. least square
 *      problem) with the total-degree Hermite basis (eq. complete);
 *   6. stores ubar and W = (H diag(sqrt(lambda))) G so that the surrogate
 *      U^0(xi) = ubar + psi(xi) W (step 6's double sum, regrouped).
 * xi_train: [n_train][M] FP64, host or device.  Runs on the current CUDA
 * device.  On success *out owns the context (free with klecgc_free).
 * Errors: INVALID_ARG (NULL pointers; a problem field out of range: nx,
 * M or J below 1, n_train below 2, gpc_degree < 0, T or corr_len not > 0,
 * sigma, eps_kl or reaction negative or NaN, advection negative or not
 * finite, forcing not finite, u0_kind or reaction_kind outside 0..2,
 * cgc_newton < 0), all
 * checked before any CUDA call; OUT_OF_MEMORY, NONFINITE (xi_train), CUDA,
 * UNSUPPORTED (dim not 1 or 2, 2D with nx > 2047, N not a power of 2 in
 * [2, 64], u0_kind 2 or advection in 1D, advection with reaction_kind 1 or
 * 2, reaction_kind 1 or 2 in 2D), NOT_CONVERGED (2D: a snapshot's Krylov
 * solve reached the iteration cap).  On any error *out is NULL.
 * 2D input KL: the covariance sigma^2 exp(-|x1-y1|/l) exp(-|x2-y2|/l) is
 * separable; its eigenpairs are (sigma^2 mu_i mu_j, phi_i(x1) phi_j(x2)) of the
 * unit-variance 1D pairs, ordered by decreasing eigenvalue, ties (i, j) /
 * (j, i) by smaller i + j, then smaller i; the first M are used.
 */
klecgc_status klecgc_setup(const klecgc_problem* problem, const double* xi_train,
                           klecgc_ctx** out, void* stream);

/*
 * klecgc_solve - online part of Algorithm 3 for S samples.
 *   xi:        [S][M] FP64 KL coefficients (host or device).
 *   dT, J, N:  coarse step, fine steps per interval, intervals; N*dT must
 *              equal T to 1e-12 relative; N a power of two in [2, 64] and,
 *              for the gPC guess, equal to the setup's N.
 *   alpha:     twist of the coarse problem u(0) = alpha u(T), 0 < alpha < 1.
 *   tol:       a sample stops after the first iteration k with
 *              max_n ||U^{k}_n - U^{k-1}_n||_inf <= tol (the paper fixes no
 *              rule; this is the per-sample increment).
 *   kmax:      iteration cap (>= 1).
 *   precision: KLECGC_FP64 / KLECGC_MIXED / KLECGC_MIXED_DEFECT (2D: FP64
 *              or MIXED, else UNSUPPORTED).
 *   guess:     KLECGC_GUESS_*; U_guess ([S][N][nx]) is read only for USER.
 *   U_out:     [S][N][nx] FP64: the last iterate of every sample.
 *   iters_out: [S] int32: CGC updates performed until tol was met, -1 when
 *              kmax was reached first, -2 for a non-finite iterate.  May be NULL.
 *   status_out:[S] int32 klecgc_status per sample.  May be NULL.
 * S == 0 is valid and does nothing.  Returns OK when every sample
 * converged, NONFINITE if any sample produced NaN/Inf (or xi had one),
 * else NOT_CONVERGED if any sample hit kmax; INVALID_ARG / UNSUPPORTED /
 * OUT_OF_MEMORY / CUDA for argument and runtime errors (nothing written).
 * Each sample's iterates are independent of the other samples.
 * Nonlinear problems (1D): problem reaction_kind 1, f(u) = div(a grad u) -
 * c (u^3 - u) + f0 (Allen-Cahn type), and reaction_kind 2, f(u) =
 * div(a grad u) - c (u^2/2)_x + f0 (Burgers type; Section 5 discretizes the
 * convection by upwinding, here the conservative Engquist-Osher flux
 * (max(u_l, 0)^2 + min(u_r, 0)^2) / 2 at each face, zero boundary values):
 * F and G take Newton iterations for every backward-Euler step (tridiagonal
 * Jacobian, to 1e-14 relative); the CGC solves eq. matrix_NT by
 * problem.cgc_newton simplified Newton steps of eq. Newton2 with the
 * time-averaged Jacobian of eq. Jac (non-symmetric tridiagonal for kind 2),
 * each diagonalized like the linear CGC.  FP64 only; guesses GPC, ZERO,
 * USER, COARSE; the stage entry points, the batch and the learned guess
 * take linear problems only.
 */
klecgc_status klecgc_solve(klecgc_ctx* ctx, const double* xi, int64_t S,
                           double dT, int32_t J, int32_t N, double alpha, double tol,
                           int32_t kmax, int32_t precision, int32_t guess,
                           const double* U_guess, double* U_out, int32_t* iters_out,
                           int32_t* status_out, void* stream);

/*
 * klecgc_solve_parareal - classical parareal (Algorithm 1, eq. pred_correc),
 * the paper's comparison method: every iteration runs F on all intervals in
 * parallel and then the sequential coarse correction
 *     U^{k+1}_n = G(U^{k+1}_{n-1}) + F(U^k_{n-1}) - G(U^k_{n-1}),  U_0 = u0,
 * with G one backward-Euler step of dT, per sample in order of n (no alpha
 * twist, no diagonalization).  FP64, 1D contexts (UNSUPPORTED for dim = 2);
 * for the nonlinear problems (reaction_kind 1, 2) F and G are the Newton
 * backward-Euler propagators of klecgc_solve (KLE-CGC of Section 5 with the
 * gPC guess).
 * Arguments, stopping rule, outputs and return as klecgc_solve, except: any
 * N >= 1 (no FFT); guess KLECGC_GUESS_GPC (N must be the setup's N), _ZERO,
 * _USER or _COARSE (the usual parareal start, U^0_n = G(U^0_{n-1})).
 */
klecgc_status klecgc_solve_parareal(klecgc_ctx* ctx, const double* xi, int64_t S, double dT,
                                    int32_t J, int32_t N, double tol, int32_t kmax,
                                    int32_t guess, const double* U_guess, double* U_out,
                                    int32_t* iters_out, int32_t* status_out, void* stream);

/*
 * klecgc_solve_batch - klecgc_solve for an uneven batch of n instances whose
 * grids, time partitions and fine steps differ (a library facility for
 * many small problems at once; the paper solves one configuration at a
 * time).  Instance i uses context ctxs[inst[i].ctx] (its problem, nx, N =
 * the setup's N, dT = T / N, and surrogate) and inst[i].J fine steps per
 * interval.  Instances of equal (context, J) form a class solved as one
 * batch; the classes run concurrently on a pool of streams, iteration by
 * iteration, until each class's samples have met tol or kmax.
 *   xi:        [n][M] FP64 (host or device), every context has the same M.
 *   guess:     KLECGC_GUESS_GPC, _ZERO or _COARSE.
 *   U_out:     packed FP64 output (host or device): instance i's [N_i][n_i]
 *              block starts at sum_{j<i} N_j n_j (n_i = nx^dim of its context).
 *   iters_out, status_out: [n] int32 as for klecgc_solve (may be NULL).
 * Return and per-instance status as klecgc_solve.  Every context must live
 * on the current device; 2D contexts need precision KLECGC_FP64 or
 * KLECGC_MIXED.  The
 * per-class scratch stays in the contexts for reuse until klecgc_free.
 */
typedef struct {
    int32_t ctx;  /* index into ctxs */
    int32_t J;    /* fine steps per coarse interval (>= 1) */
} klecgc_instance;

klecgc_status klecgc_solve_batch(klecgc_ctx* const* ctxs, int32_t n_ctx,
                                 const klecgc_instance* inst, int64_t n, const double* xi,
                                 double alpha, double tol, int32_t kmax, int32_t precision,
                                 int32_t guess, double* U_out, int32_t* iters_out,
                                 int32_t* status_out, void* stream);

/* Stage entry points (one step of the hot path each; used for stage-level
 * checks).  Arguments have the meanings given for klecgc_solve. */

/* Coefficient field a(x_{i+1/2}; xi) = exp(g) at the nx+1 faces of every
 * sample: a_out [S][nx+1] FP64.  2D: a_out [S][2 nx (nx+1)], the x-faces
 * [nx][nx+1] at ((fx+1/2)h, (iy+1)h) first, then the y-faces [nx+1][nx] at
 * ((ix+1)h, (fy+1/2)h). */
klecgc_status klecgc_field(klecgc_ctx* ctx, const double* xi, int64_t S,
                           double* a_out, void* stream);

/* Surrogate guess U^0(xi) = ubar + sum_k sqrt(lambda_k) zeta_k(xi) g_k
 * (Algorithm 3 step 6) on the setup's grid: U0_out [S][N][nx].
 * precision FP64 evaluates it in FP64; the mixed modes in FP32 with FP64
 * output. */
klecgc_status klecgc_guess(klecgc_ctx* ctx, const double* xi, int64_t S,
                           int32_t precision, double* U0_out, void* stream);

/* Step 1 of Algorithm 2 plus the right-hand side of the CGC system
 * (eq. matrix_NT at the Newton point of eq. Newton2): for every sample and
 * n = 1..N, Ftilde_n = F(start_n) with start_1 = u0 and start_n = U_{n-1},
 * and r_n = (I + dT A) Ftilde_n - prev_n with prev_1 = alpha U_N and
 * prev_n = U_{n-1}; this equals (I + dT A) b_n + dT f0 for the jump b of
 * Section 3.2.  U_in, r_out: [S][N][nx] FP64.  precision selects the
 * arithmetic of F (FP64, or FP32 increment form for the mixed modes). */
klecgc_status klecgc_fine_sweep(klecgc_ctx* ctx, const double* xi, int64_t S, int32_t N,
                                const double* U_in, double dT, int32_t J, double alpha,
                                int32_t precision, double* r_out, void* stream);

/* Diagonalized CGC solve (eq. three steps): u = (C_alpha (x) I + dT I (x) A)^{-1} r
 * by (a) p = F_N^* Lambda_alpha r along n, (b) (lambda_n I + dT A) q_n = p_n,
 * (c) u = Lambda_alpha^{-1} F_N q, with Lambda_alpha = diag(alpha^{(n-1)/N})
 * and lambda_n = 1 - alpha^{1/N} exp(-2 pi i (n-1)/N).  (The printed
 * eigenvector matrix Lambda_alpha F_N does not diagonalize C_alpha; its
 * inverse scaling does.)  r_in, u_out: [S][N][nx] FP64; precision FP64 or
 * KLECGC_MIXED_DEFECT (FP32 transform and solves); 2D: FP64 or KLECGC_MIXED
 * (FP64 refinement around FP32 COCG, same FP64 residual test). */
klecgc_status klecgc_cgc_apply(klecgc_ctx* ctx, const double* xi, int64_t S, int32_t N,
                               const double* r_in, double dT, double alpha,
                               int32_t precision, double* u_out, void* stream);

/* The paper's reference solution (Section 2, remark after eq. psys): the
 * sequential fine solution U*_n, n = 1..N, in FP64: U_out [S][N][nx]. */
klecgc_status klecgc_reference(klecgc_ctx* ctx, const double* xi, int64_t S, int32_t N,
                               int32_t J, double* U_out, void* stream);

/*
 * klecgc_reference_noalloc - klecgc_reference for callers that cannot
 * allocate device memory (the paper has no counterpart: this is a library
 * facility).  Such callers include code running under another framework's
 * caching allocator that owns the free device memory, hosts that forbid
 * allocation after start-up, and callbacks that must not let
 * cudaMalloc/cudaFree synchronize the device.  The result equals
 * klecgc_reference's; the working memory is one 32 MiB array compiled into
 * the library, which every GPU that loads the library holds until exit.
 *   xi:    [S][M] FP64 device array; U_out: [S][N][nx] FP64 device array.
 *   Requires S * (6 nx + 5) <= 4194304 (32 MiB of doubles), else
 *   INVALID_ARG with the sizes in klecgc_last_error(); host arrays, arrays
 *   on a device other than the context's, and a current device other than
 *   the context's also give INVALID_ARG (managed arrays are accepted).
 * Allocates nothing (no cudaMalloc/cudaFree, no allocating library call).
 * 1D contexts only (UNSUPPORTED for dim = 2).
 * The first call on a device looks up the array's device address with
 * cudaGetSymbolAddress; make that first call before any stream capture.
 * Every call shares the array: calls whose GPU work overlaps (e.g. on two
 * streams at once) race and must be serialized by the caller.  Nothing in
 * the array needs to start at zero (each call writes what it reads).
 */
klecgc_status klecgc_reference_noalloc(klecgc_ctx* ctx, const double* xi, int64_t S, int32_t N,
                                       int32_t J, double* U_out, void* stream);

/*
 * Learned initial guess.  The paper's guess is the KL/gPC surrogate
 * (Algorithm 3, step 6); these entry points add a learned one with the same
 * role: an MLP M -> 256 -> 256 -> 256 -> 64 N (ReLU hidden layers) maps xi to
 * the state at the N coarse times sampled at x_m = (m+1)/65, m = 0..63,
 * normalized per output column ((y - mean) / std); the guess is its output
 * de-normalized and linearly interpolated (zero boundary values) to the grid.
 * Parameters: one flat FP32 vector [W1, b1, W2, b2, W3, b3, W4, b4], W_l
 * stored [out][in].  GEMMs use BF16 operands with FP32 accumulation; master
 * weights, Adam moments, activations before the BF16 rounding and the loss
 * are FP32.  1D contexts only (UNSUPPORTED for dim = 2).
 */

/* Sets the parameters (n_params floats, host or device) and the output
 * normalization (out_mean/out_std: 64 N floats each; NULL = 0 and 1).
 * INVALID_ARG if n_params does not match the architecture or std <= 0. */
klecgc_status klecgc_mlp_set(klecgc_ctx* ctx, const float* params, int64_t n_params,
                             const float* out_mean, const float* out_std);

/* Copies the parameters and normalization out (each may be NULL); *n_params
 * receives the parameter count (also when no network is set). */
klecgc_status klecgc_mlp_get(const klecgc_ctx* ctx, float* params, float* out_mean,
                             float* out_std, int64_t* n_params);

/* Mean squared error over B samples of the normalized targets
 * (targets: [B][N][64] raw FP32, normalized with the context's mean/std)
 * and its gradient w.r.t. the parameters (grad_out: n_params FP32, host or
 * device; may be NULL). */
klecgc_status klecgc_mlp_loss_grad(klecgc_ctx* ctx, const double* xi, const float* targets,
                                   int64_t B, double* loss_out, float* grad_out, void* stream);

/* Trains from the current parameters with Adam (beta 0.9/0.999, eps 1e-8),
 * mini-batches of `batch` rows of a permutation drawn per epoch from `seed`
 * (xorshift64*), learning rate cosine-annealed from lr to lr_final over all
 * steps.  fit_norm != 0 first sets the output normalization to the
 * per-column mean and std of the targets.  xi: [n][M] FP64, targets:
 * [n][N][64] FP32 (host or device).  epoch_loss (host, may be NULL)
 * receives the mean loss of each epoch.  NONFINITE if the loss diverges. */
klecgc_status klecgc_mlp_train(klecgc_ctx* ctx, const double* xi, const float* targets, int64_t n,
                               int32_t epochs, int32_t batch, double lr, double lr_final,
                               uint64_t seed, int32_t fit_norm, float* epoch_loss, void* stream);

/* Learned guess U0_out [S][N][nx] FP64 for S samples (NONFINITE if an output
 * is not finite; the solve then uses the gPC surrogate instead). */
klecgc_status klecgc_mlp_guess(klecgc_ctx* ctx, const double* xi, int64_t S, double* U0_out,
                               void* stream);

/* Samples a batch U [S][N][nx] (FP64) at the 64 network points:
 * T_out [S][N][64] FP32, linear interpolation with zero boundary values. */
klecgc_status klecgc_downsample(klecgc_ctx* ctx, const double* U, int64_t S, int32_t N,
                                float* T_out, void* stream);

/* Learned-guess mode: residual = 0 (default) the guess is the network's
 * output as above; residual = 1 the network's output (de-normalized,
 * interpolated) is a correction added to the gPC surrogate guess of the
 * same xi, U0 = ubar + psi(xi) W + network(xi), so the network only has to
 * learn what the surrogate misses (kept in context files).  INVALID_ARG for
 * another value; UNSUPPORTED outside the linear 1D problem. */
klecgc_status klecgc_mlp_set_residual(klecgc_ctx* ctx, int32_t residual);

/* Training targets for the current mode: T_out [S][N][64] FP32 = the
 * reference solutions U [S][N][nx] (FP64) at the network points, minus the
 * gPC surrogate guess of xi [S][M] there in residual mode (arrays host or
 * device; the stream is synchronized). */
klecgc_status klecgc_mlp_targets(klecgc_ctx* ctx, const double* xi, const double* U, int64_t S,
                                 float* T_out, void* stream);

/*
 * 2D Krylov solves (dim = 2 only; 1D uses direct factorizations).
 * Each backward-Euler step (I + dt(A + cI)) v' = v + dt f0 of F is solved by
 * Jacobi-preconditioned CG warm-started from v, stopped when
 * ||b - M v'||_2 <= rtol_fine ||b||_2; each shifted CGC system
 * (lambda_k I + dT(A + cI)) q_k = p_k (eq. three steps (b)) by
 * Jacobi-preconditioned COCG from zero, stopped when ||r||_2 <= rtol_cgc
 * ||p_k||_2.  Either stops after maxit iterations at most; a sample with
 * such a solve gets status NOT_CONVERGED.  Defaults 1e-10, 1e-10, 10000.
 * INVALID_ARG unless 0 < rtol < 1 and maxit >= 1.
 */
klecgc_status klecgc_set_krylov(klecgc_ctx* ctx, double rtol_fine, double rtol_cgc,
                                int32_t maxit);

/*
 * Scratch budget: the device scratch the context grows for its calls (the
 * batch-sized buffers; not the set-up tables it owns) may total at most
 * `bytes` (0 = no limit, the default).  A call that would exceed it fails
 * with OUT_OF_MEMORY before allocating, and the context stays usable for
 * smaller calls.  INVALID_ARG for a negative budget.
 */
klecgc_status klecgc_set_scratch_limit(klecgc_ctx* ctx, int64_t bytes);

/*
 * 2D linear-solve method: 0 (default) banded LU in FP64 for nx <= 32 and
 * Krylov otherwise (and on the MIXED path); 1 Krylov always; 2 banded LU
 * (FP64; UNSUPPORTED for dim = 1 or nx > 64); 3 Krylov, with every MIXED
 * fine-propagator system held by a thread-block cluster (the layout methods
 * 0 and 1 pick by themselves when a system does not fit one CTA's shared
 * memory, e.g. nx = 255; UNSUPPORTED for dim = 1).  Banded LU factors each
 * backward-Euler matrix I + dt(A + cI) once per sample and each shifted
 * matrix lambda_k I + dT(A + cI) once per (sample, k) per call (bandwidth
 * nx, no pivoting: the matrices are diagonally dominant), then every step
 * or shifted solve is one forward and one backward substitution; the
 * result is the exact solve up to rounding (no Krylov tolerance).
 * INVALID_ARG for another method.
 */
klecgc_status klecgc_set_2d_method(klecgc_ctx* ctx, int32_t method);

/*
 * How the parareal iterations of Algorithms 1 and 2 (the loop that ends at
 * the stopping rule of Step 3) are driven, for klecgc_solve and
 * klecgc_solve_parareal: 0 (default) on the device, as a CUDA graph whose
 * conditional WHILE node repeats one captured iteration while a sample is
 * active and fewer than kmax iterations have run (no host round trip per
 * iteration); 1 from the host, with a readback of the active count after
 * each iteration.  Both launch the same kernels in the same order and give
 * bitwise-equal results.  With CUDA-event timing enabled
 * (klecgc_profile_enable(ctx, 1)) the host loop is used, since per-launch
 * events cannot sit inside a graph loop.  klecgc_solve_batch always drives
 * its classes from the host.  INVALID_ARG for another mode.
 */
klecgc_status klecgc_set_loop(klecgc_ctx* ctx, int32_t mode);

/*
 * Launch-shape autotuner (a library facility; the paper has no counterpart).
 * mode 1 (default): the first solve of a context for a given (nx, N, J) on a
 * given GPU times every candidate launch shape of the FP32 fine propagator
 * ("W<W>R<R>": W warps per pair of intervals, R rows per lane, 32 W R >=
 * nx + 1, W = 0 the shared-memory kernel; "L<L>R<R>": one interval per warp
 * with the factors in registers, L intervals per warp in turn; "P1R<R>": one
 * interval per warp, each lane's R rows as two halves swept together in
 * packed FP32x2) on up to 512 of its samples and keeps the fastest; later
 * solves reuse the choice.
 * Every shape computes the same backward-Euler steps; the shapes split the
 * rows of a system differently between lanes, so results agree to FP32
 * rounding of the fine propagator, not bit for bit: a solve is reproducible
 * for a fixed choice (pin it with cache_path).  mode 0: fixed rules, no
 * timing.
 * cache_path (may be NULL): a JSON file of the choices, read now and
 * rewritten after every new choice, so that other processes and contexts can
 * skip the timing.  INVALID_ARG for another mode.
 */
klecgc_status klecgc_set_tuning(klecgc_ctx* ctx, int32_t mode, const char* cache_path);

/* The autotuner's choices as a JSON object of "<GPU>|<kernel>|nx=..|N=..|J=..":
 * "<shape>" strings, plus for each shape timed by this context a
 * "<same key>|ms@S=<samples>": "<shape>:<ms per launch> ..." record of the
 * candidates, NUL-terminated into buf (capacity bytes, truncated if short;
 * buf may be NULL); *length receives the full length. */
klecgc_status klecgc_tuning_report(const klecgc_ctx* ctx, char* buf, int64_t capacity,
                                   int64_t* length);

/* Krylov iterations of the last 2D call (klecgc_solve, klecgc_fine_sweep,
 * klecgc_cgc_apply, klecgc_reference), summed over all linear systems, for
 * F and for the CGC solves; for the cubic reaction (reaction_kind 1) the
 * Newton iterations of F and G of the last klecgc_solve (its_cgc = 0).
 * Either pointer may be NULL. */
klecgc_status klecgc_krylov_stats(const klecgc_ctx* ctx, int64_t* its_fine, int64_t* its_cgc);

/*
 * Context persistence (a library facility; the paper's offline stage is
 * re-run otherwise).  klecgc_save writes the problem, the surrogate tables
 * (input-KL basis, u0, gPC multi-indices, ubar, W), the Krylov settings, the
 * 2D solve method, the autotuner's choices and,
 * when set, the learned network to `path` (a binary file of this library's
 * own format, native byte order).  klecgc_load creates a context on the
 * current CUDA device from such a file: its guesses and solves equal those
 * of the saved context (bit for bit on the same GPU model, whose launch
 * shapes the saved choices name).  Errors: INVALID_ARG (cannot open, not a context
 * file, inconsistent or truncated), OUT_OF_MEMORY, CUDA.
 */
klecgc_status klecgc_save(const klecgc_ctx* ctx, const char* path);
klecgc_status klecgc_load(const char* path, klecgc_ctx** out, void* stream);

/* Sizes of the context (M_Q, P, ...). */
klecgc_status klecgc_info(const klecgc_ctx* ctx, klecgc_info_t* out);

/*
 * klecgc_kl_basis - the input-field KL basis b_m(x) = sqrt(lambda_m) phi_m(x),
 * m = 0..M-1, that klecgc_setup uses for a = exp(sum_m b_m(x) xi_m) (the
 * problem statement's log-normal coefficient), evaluated at npts points.
 * dim 1: eigenpairs of sigma^2 exp(-|x - y| / corr_len) on [0,1] (roots of
 * the transcendental equations, decreasing lambda); dim 2: the separable
 * product modes on [0,1]^2, ordered as klecgc_setup orders them.  The values
 * are those klecgc_setup computes at its face points, bit for bit.
 * Host only: runs on the calling thread and makes no CUDA call.
 * x: host FP64, [npts] (dim 1) or [npts][2] (dim 2, (x1, x2) pairs);
 * out: host FP64 [M][npts]; lambda_out: host FP64 [M] or NULL.
 * Errors: UNSUPPORTED (dim not 1 or 2), INVALID_ARG (M outside 1..65536 in
 * 1D or 1..1024 in 2D, npts < 0, NULL x or out with npts > 0, corr_len not
 * finite and > 0, sigma not finite and >= 0).
 */
klecgc_status klecgc_kl_basis(int32_t dim, double corr_len, double sigma, int32_t M,
                              const double* x, int64_t npts, double* out, double* lambda_out);

/*
 * klecgc_gpc_indices - the multi-indices k of the total-degree Hermite gPC
 * basis psi_k(xi) = prod_l He_{k_l}(xi_l) / sqrt(k_l!), |k|_1 <= p (Section
 * 2.2, eq. complete), in the order of the surrogate's coefficient rows: by
 * total degree, and within a degree in decreasing lexicographic order of
 * (k_1, ..., k_M).  *P_out = P = (M + p)! / (M! p!).  With out non-NULL,
 * out (host int32 [P][M], capacity >= P rows) receives the indices.
 * Host only: makes no CUDA call.
 * Errors: INVALID_ARG (M < 1, p < 0, capacity < 0, NULL P_out, out non-NULL
 * and capacity < P), UNSUPPORTED (P > 2^24 or M P > 2^28).
 */
klecgc_status klecgc_gpc_indices(int32_t M, int32_t p, int32_t* out, int64_t capacity,
                                 int64_t* P_out);


/* Kernel classes of the profile (index into klecgc_profile_t arrays). */
enum {
    KLECGC_K_FIELD = 0,     /* coefficient field and face weights          */
    KLECGC_K_FACTORS = 1,   /* fine and CGC factorizations                  */
    KLECGC_K_GUESS = 2,     /* gPC basis and surrogate contraction          */
    KLECGC_K_FINE = 3,      /* fine propagator + CGC right-hand side        */
    KLECGC_K_CGC_FWD = 4,   /* step (a): DFT along the coarse times         */
    KLECGC_K_CGC_SOLVE = 5, /* step (b): shifted tridiagonal solves         */
    KLECGC_K_CGC_INV = 6,   /* step (c): inverse DFT, update, increment norm */
    KLECGC_K_CONV = 7,      /* stopping rule                                */
    KLECGC_K_LAYOUT = 8,    /* layout changes, checks                       */
    KLECGC_K_COUNT = 9
};

typedef struct {
    int64_t launches[16]; /* kernel launches per class since the last enable */
    double ms[16];        /* summed CUDA-event time per class (0 when timing is off) */
    int32_t n_classes;    /* KLECGC_K_COUNT */
} klecgc_profile_t;

/* Resets the per-class launch counters; with `timing` != 0, klecgc_solve also
 * brackets every kernel launch with CUDA events on its stream and sums the
 * elapsed times per class. */
klecgc_status klecgc_profile_enable(klecgc_ctx* ctx, int32_t timing);

/* Reads the counters and summed times accumulated since the last enable. */
klecgc_status klecgc_profile_read(const klecgc_ctx* ctx, klecgc_profile_t* out);

/* Releases the context and everything it allocated.  NULL is allowed. */
void klecgc_free(klecgc_ctx* ctx);

/* Static description of a status code. */
const char* klecgc_status_string(klecgc_status s);

/* Detail of the last error reported on the calling thread ("" if none). */
const char* klecgc_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* KLECGC_H */
