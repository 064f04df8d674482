/*
 * ehs.h - C ABI of the GB300 elastic Helmholtz shifted-Laplacian solver.
 *
 * The library solves the mixed (displacement / pressure) staggered-grid
 * discretisation of the elastic Helmholtz equation,
 *
 *     K [u; p] = [q; 0],   K = [[L_mu - w^2 M,  G           ],
 *                               [G^T,          -D(1/(l+mu))]]
 *
 * (Treister & Yovel, Sec. 2.1 eq. elasticHelmSystem and eq.
 * elasticHelmMass, Sec. 3 eq. pressure and eq.
 * elasticHelmReformulatedSystem), with a flexible GMRES preconditioned by a
 * multigrid cycle of the shifted operator K_s = K + i alpha w^2 diag(A_f(rho), 0)
 * (Sec. 2.2 eq. shift; Sec. 3 zero-padded shift), red-black cell-wise
 * (Vanka) relaxation (Sec. 3), Galerkin coarse operators (Sec. 2.2 eq.
 * coarseGridMatrix) and an exact FP64 coarsest solve; optionally wrapped in
 * the multicolour overlapping domain decomposition of Sec. 2.3 Algorithm DD
 * (DD-MG of Sec. 4).
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 * Grid: n[0] x n[1] x n[2] cells (x fastest; n[2] = 1 in 2D), spacing h.
 * Media: cell-centred lambda, mu, rho, double, [nmedia][n_z][n_y][n_x].
 * Vector ("slot layout"): per item, d+1 component arrays of ncell complex
 *   numbers (interleaved re, im): u_1 .. u_d, p.  u_k[c] lives on the low
 *   face of cell c in direction k; slots with index 0 along k are Dirichlet
 *   boundary faces and must be zero on input (they are zero on output).
 *   A batch of items is stacked on the slowest axis; item b uses medium
 *   b / nrhs.  Double-precision vectors hold complex128, single-precision
 *   vectors complex64.
 * Pointers: vector arguments of ehs_op_apply, ehs_smooth, ehs_vcycle and
 *   ehs_dd_precond are device pointers; ehs_fgmres_solve and
 *   ehs_adjoint_solve accept host or device pointers (host buffers are
 *   copied in and out by the call).  The caller owns every buffer it passes;
 *   the context owns its hierarchy and workspaces.
 * Streams: every call is ordered on the stream given to ehs_create; only the
 *   solves synchronise it (they read residual norms on the host).
 * Errors: no call throws; a failed call returns a non-zero ehs_status,
 *   ehs_last_error() describes it, outputs are unspecified except for
 *   EHS_ERR_NOCONV / EHS_ERR_BREAKDOWN, which return the best iterate.
 *   Arguments are validated before any launch.
 */
#ifndef EHS_H
#define EHS_H

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  EHS_OK = 0,
  EHS_ERR_ARG = 1,        /* invalid argument (sizes, divisibility, media) */
  EHS_ERR_CUDA = 2,       /* a CUDA call failed */
  EHS_ERR_OOM = 3,        /* device allocation failed */
  EHS_ERR_NOCONV = 4,     /* maxit reached before tol */
  EHS_ERR_BREAKDOWN = 5,  /* Arnoldi breakdown before tol */
  EHS_ERR_TIMEOUT = 6,    /* a bounded device wait gave up: the grid barrier of a persistent
                             launch (the MG-DD coarsest solve of the 2D complex64 cycle) waited
                             past about a second because other work held the SMs; returned by
                             the solves and by ehs_sync, the outputs are then unspecified */
  EHS_ERR_NONFINITE = 7,  /* NaN / Inf in a residual norm or a pivot */
  EHS_ERR_UNSUPPORTED = 8 /* reserved for an option combination that is not built; this version
                             rejects unknown option values with EHS_ERR_ARG instead */
} ehs_status;

typedef enum { EHS_C128 = 0, EHS_C64 = 1 } ehs_prec;
typedef enum { EHS_PRECOND_MG = 0, EHS_PRECOND_DD = 1 } ehs_precond;

typedef struct ehs_ctx ehs_ctx; /* opaque, owned by the library */

typedef struct {
  int dim;               /* 2 or 3 */
  int n[3];              /* cells along x, y, z */
  double h;              /* grid spacing */
  double omega;          /* angular frequency (all media) */
  const double* omegas;  /* optional host array [nmedia] of per-medium frequencies; NULL = omega */
  int nmedia;            /* independent media (coefficient sets), >= 1 */
  const double* lambda;  /* [nmedia][ncell], host or device, read during ehs_create only */
  const double* mu;
  const double* rho;
  int abl_cells;         /* absorbing layer width on every side (cells) */
  double abl_max;        /* gamma/omega reached at the outer edge (eq. elasticHelmMass) */
  double gamma_add;      /* constant attenuation added everywhere (0.01 pi in Sec. 6) */
} ehs_problem;

typedef struct {
  int levels;            /* multigrid levels >= 2; every n[k] divisible by 2^(levels-1) */
  double alpha;          /* shift (Sec. 2.2 eq. shift) */
  double w[8];           /* Vanka damping of level l (Sec. 6: 0.75, 0.5, 0.25) */
  double wp_ratio;       /* w_p = w_l * wp_ratio (Sec. 5.4 component damping); 1 = same */
  int nu_pre, nu_post;   /* relaxation sweeps (one sweep = red + black) */
  int cycle;             /* 1 = V-cycle, 2 = W-cycle */
  int restart;           /* FGMRES restart length m (1..11) */
  int maxit;             /* max preconditioner applications per solve */
  double tol;            /* relative residual of the mixed system */
  int precond;           /* ehs_precond */
  int prec;              /* ehs_prec of the preconditioner cycle.  EHS_C128: complex128 cycle
                            and FP64 Krylov solve (the plain FP64 form).  EHS_C64: complex64
                            cycle and a double-float Krylov solve (pairs of FP32 numbers,
                            about 48-bit significands: FP64-class, not IEEE FP64), with the
                            true residual recomputed in double-float */
  int nrhs;              /* right-hand sides per medium; items = nmedia * nrhs */
  int dd[3];             /* subdomains per axis (DD only) */
  int dd_overlap;        /* overlap in cells (DD only) */
  int dd_pad;            /* absorbing padding in cells on interface sides (DD only) */
  double dd_abl_max;     /* gamma/omega at the outer edge of the padding (DD only) */
  int coef_half;         /* storage of the Galerkin stencil coefficients used by the
                            complex64 cycle: 0 complex64, 1 FP16 pairs, 2 BF16 pairs
                            (products accumulate in FP32; the FP64 masters stay) */
  int vanka_full;        /* cell-wise relaxation block (Sec. 4.2): 0 economic (eq.
                            RelaxationMatrix, the default), 1 full (2d+1)^2 block; on
                            Galerkin levels the full block inverses are formed at setup in
                            FP64 and stored per colour in the cycle's precision (FP16 /
                            BF16 pairs with coef_half, as the implementation remark of
                            Sec. 4 stores them in half precision) */
  int coarse_dd[3];      /* MG-DD (Sec. 4): subdomains per axis of the coarsest grid, which is
                            then solved by one multiplicative sweep of Algorithm DD (colours by
                            index parity, exact dense local solves on the unknowns inside each
                            overlapping box; faces on a box surface are Dirichlet) instead of
                            the exact dense solve; all <= 1: exact.  With precond = DD this
                            gives DD-MG-DD: every subdomain hierarchy's coarsest grid is split
                            the same way */
  int coarse_dd_overlap; /* overlap of the coarsest-grid subdomains in cells (>= 1, at most half
                            the smallest core) */
  int coarse_fmt;        /* storage of the coarsest inverses (exact or MG-DD) used by the complex64
                            cycle: 0 complex double-float (FP64-class), 1 complex64, 2 FP16
                            pairs, 3 BF16 pairs; products accumulate in FP32 (double-float
                            for 0); formed in FP64 at setup in every case */
  int coarse_persist;    /* 1: the MG-DD coarsest solve of the 2D complex64 cycle (coarse_fmt 1..3)
                            runs as one persistent launch per solve -- every colour's residual,
                            local products and scatter, separated by bounded grid barriers --
                            instead of graph-replayed per-colour launches; same results.  0 (the
                            default): per-colour launches */
  int ortho;             /* Arnoldi orthogonalisation of the double-float solve (prec = EHS_C64; the
                            FP64 form always uses CGS2).  0: CGS2, three passes over the basis
                            per step (first projection, second projection with the norm,
                            update), compensated double-float sums throughout.  1 (the default):
                            delayed CGS2, two passes per step: the second projection of a
                            direction (compensated double-float sums) is formed together with
                            the first projection of the next one (FP32 products: the next
                            step's second projection removes their rounding, and the Hessenberg
                            matrix records what was subtracted); the preconditioner is applied
                            to the once-orthogonalised direction, which flexible GMRES allows.
                            The same basis and Hessenberg matrix as CGS2 in exact arithmetic */
} ehs_opts;

typedef struct {
  int iters;             /* preconditioner applications */
  double relres;         /* true ||q - K u|| / ||q|| at exit */
  int converged;         /* 1 if relres <= tol */
} ehs_solve_info;

/* Fill *o with the defaults of Sec. 6 (3 levels, alpha 0.2, w 0.75/0.5/0.25,
 * V(1,1), FGMRES(10), tol 1e-6, MG preconditioner in complex64). */
void ehs_default_opts(ehs_opts* o);

/* Build the hierarchy (coefficients, Galerkin operators, coarsest inverse,
 * and the DD subdomain hierarchies when opts->precond is DD) for every
 * medium.  stream: a cudaStream_t (NULL = legacy default stream).
 * Returns EHS_ERR_ARG for invalid sizes or media (rho <= 0, mu < 0,
 * lambda + mu <= 0, non-finite omega, n not divisible), for options out of
 * range, and for a coarsest level whose dense inverse (the whole level, or
 * every MG-DD box) would exceed 16384 unknowns; options and sizes are checked
 * on the host before any device work, the media values after they are read.
 * On failure *out is NULL and ehs_last_error(NULL) holds the reason. */
ehs_status ehs_create(const ehs_problem* prob, const ehs_opts* opts, void* stream, ehs_ctx** out);
ehs_status ehs_destroy(ehs_ctx* ctx);

/* y = K_l x for all items.  level 0: the fine operator, unshifted
 * (shifted = 0, the Krylov operator K) or shifted (K_s); level l >= 1: the
 * Galerkin operator P^T K_{l-1} P (always shifted).  prec selects complex128
 * or complex64 vectors and arithmetic.  Device pointers, slot layout of the
 * level's grid. */
ehs_status ehs_op_apply(ehs_ctx* ctx, int level, int shifted, int prec, const void* x, void* y);

/* nsweeps red-black cell-wise relaxation sweeps of level l on K_l x = b
 * (Sec. 3, economic block of eq. RelaxationMatrix, damping w_l); x is
 * updated in place.  Device pointers. */
ehs_status ehs_smooth(ehs_ctx* ctx, int level, int nsweeps, int prec, const void* b, void* x);

/* x := one multigrid cycle (Algorithm TwoCycle, recursive) for K_s x = b
 * from a zero initial guess.  Device pointers, fine-grid slot layout. */
ehs_status ehs_vcycle(ehs_ctx* ctx, int prec, const void* b, void* x);

/* Fine-to-coarse half of the coarse-grid correction (Algorithm TwoCycle step 2):
 *   rc = P_l^T (b - K_l x)
 * for every item: the residual of the shifted operator of level l restricted to
 * level l+1 with the transpose of the staggered bilinear prolongation (Sec. 3).
 * 0 <= level <= levels-2.  b, x: device vectors of level l, rc: device vector of
 * level l+1 (slot layouts; rc's Dirichlet slots are written as zero).  In the
 * complex64 form on a 2D fine level whose sizes split into the fused kernel's
 * tiles (n_x divisible by 32, n_y by 16) this is one pass that never writes the
 * fine residual; otherwise the residual goes through the level's scratch.  MG
 * contexts only. */
ehs_status ehs_residual_restrict(ehs_ctx* ctx, int level, int prec, const void* b, const void* x, void* rc);
/* Coarse-to-fine half (Algorithm TwoCycle step 4): x += P_l ec for every item;
 * ec: device vector of level l+1, x: device vector of level l, updated in place.
 * 0 <= level <= levels-2.  MG contexts only. */
ehs_status ehs_prolong_add(ehs_ctx* ctx, int level, int prec, const void* ec, void* x);

/* Coarsest-level solve (Algorithm TwoCycle step 3 at the last level): x = K_c^{-1} b through
   the stored dense inverse (exact), or by the MG-DD sweep of Sec. 4 when opts.coarse_dd splits
   the coarsest grid.  b, x: device, [items][(d+1) * ncell_c] complex of prec (ehs_level_len of
   the last level).  MG contexts only (EHS_ERR_ARG otherwise). */
ehs_status ehs_coarse_solve(ehs_ctx* ctx, int prec, const void* b, void* x);
/* Shape of the coarsest local solves: nsub subdomains (1 for the exact solve), padded local size
   nloc (local vectors are [nmedia][nsub][nrhs][nloc]), and, if sizes is not NULL, the live unknowns of
   each subdomain (host array of nsub ints).  MG contexts only. */
ehs_status ehs_coarse_dims(const ehs_ctx* ctx, int* nsub, int* nloc, int* sizes);
/* One launch of the coarsest local products z_loc = A_s^{-1} r_loc for every subdomain s of
   colour `colour` (0 .. 2^d - 1; the exact solve has colour 0 only), i.e. step 2 of Algorithm DD
   on the coarsest grid with the inverses formed at setup.  r_loc, z_loc: device [nmedia][nsub][nrhs][nloc]
   complex of prec; entries of other colours' subdomains and of padding rows are left unspecified.
   The complex64 form reads the inverses in opts.coarse_fmt storage. */
ehs_status ehs_coarse_local_apply(ehs_ctx* ctx, int prec, int colour, const void* r_loc, void* z_loc);
/* The same local products added into a coarsest vector, as the MG-DD sweep applies them (steps 2
   and 3 of Algorithm DD on the coarsest grid): x[item] += R_s^T A_s^{-1} r_loc[item][s] for every
   subdomain s of colour `colour`, R_s^T placing the box unknowns at their coarsest slots (boxes of
   one colour are disjoint).  r_loc as for ehs_coarse_local_apply; x: device [items][(d+1) *
   ncell_c] complex of prec, read and written.  In the complex64 form one launch does both.  MG-DD
   contexts only (EHS_ERR_ARG otherwise, or for a colour without subdomains). */
ehs_status ehs_coarse_local_add(ehs_ctx* ctx, int prec, int colour, const void* r_loc, void* x);

/* z := one sweep of Algorithm DD on K z = r (global residual recomputed
 * before each colour, subdomain corrections by one multigrid cycle of the
 * shifted subdomain operator).  Requires a context created with
 * precond = EHS_PRECOND_DD.  Device pointers. */
ehs_status ehs_dd_precond(ehs_ctx* ctx, int prec, const void* r, void* z);

/* Solve K u = q for every item with right-preconditioned FGMRES(m) from a
 * zero initial guess (Sec. 6).  q, u: complex128, host or device.
 * info: host array of nmedia*nrhs entries (may be NULL). */
ehs_status ehs_fgmres_solve(ehs_ctx* ctx, const void* q, void* u, ehs_solve_info* info);

/* Solve K^H w = g (adjoint state).  K is complex symmetric (K = K^T), so
 * K^H = conj(K) and w = conj(K^{-1} conj(g)); the same preconditioner is
 * used.  Same argument conventions as ehs_fgmres_solve. */
ehs_status ehs_adjoint_solve(ehs_ctx* ctx, const void* g, void* w, ehs_solve_info* info);

/* Adjoint-state gradient with respect to the cell-centred medium:
 *   g_m(c) = -Re( w^H (dK/dm_c) x ),  m in {lambda, mu, rho},
 * summed over the right-hand sides of each medium, where x solves K x = q
 * (ehs_fgmres_solve) and w solves K^H w = e (ehs_adjoint_solve with e the
 * derivative of a real misfit J with respect to conj(x)); then g = dJ/dm.
 * Frequency-domain full-waveform inversion, the application of Sec. 1.
 * x, w: device complex128 vectors (all items); g_*: device double arrays
 * [nmedia][ncell], overwritten. */
ehs_status ehs_gradient(ehs_ctx* ctx, const void* x, const void* w, double* g_lambda, double* g_mu,
                        double* g_rho);

/* Allocation-free fine-level smoothing.  The paper has no counterpart: this
 * entry point exists for callers that may not allocate device memory when
 * they need to relax a vector, and therefore cannot build a context with
 * ehs_create -- for example a host program that gives all of the device
 * memory to its own pool at start-up and forbids the libraries it loads to
 * call cudaMalloc (so that its footprint stays fixed and known), or a
 * latency-bound loop that must not stall on the allocator (cudaFree waits for
 * the whole device).  It performs nsweeps red-black economic cell-wise
 * relaxation sweeps of the shifted fine operator K_s (the same kernels and
 * result as ehs_smooth on level 0 of a context built from the same problem)
 * without any cudaMalloc / cudaFree or allocating library call.
 *   prob: as for ehs_create, but lambda, mu, rho must be DEVICE pointers of
 *     the current device and nmedia <= 32; every n[k] even; 0 <= abl_cells
 *     <= min n[k] / 2.  The media VALUES are not checked here (ehs_create
 *     checks them): rho <= 0, lambda + mu <= 0 or non-finite entries give
 *     non-finite x instead of an error.  nrhs: items per medium; items =
 *     nmedia * nrhs.  alpha: shift; w, wp: damping of the u and p unknowns.
 *   prec: EHS_C64 or EHS_C128; b, x: device vectors of that precision on the
 *     current device, in the slot layout (x is relaxed in place).
 *   stream: a cudaStream_t or NULL.
 * Scratch: the cell coefficients, the frequencies and the ping-pong vector
 *   live in one static 32 MiB device array per GPU, held from library load
 *   until process exit; problems needing more return EHS_ERR_OOM.  Every call
 *   shares that array (each call clears and rewrites what it uses), so calls
 *   whose GPU work can overlap -- other streams or host threads -- race and
 *   must be serialised by the caller.  The first call on each device looks up
 *   the array's device address; make that first call before any stream
 *   capture begins.
 * Returns EHS_ERR_ARG for invalid arguments, host pointers or memory of
 *   another device, EHS_ERR_OOM for a problem larger than the scratch,
 *   EHS_ERR_CUDA if a launch fails. */
ehs_status ehs_fine_smooth_noalloc(const ehs_problem* prob, int nrhs, double alpha, double w,
                                   double wp, int nsweeps, int prec, const void* b, void* x,
                                   void* stream);

/* Sizes: items of a vector batch (0 for a NULL context), complex values per item at level l
   (-1 for a NULL context or a level out of range), and the cells per axis of level l written to
   the host array n[3] (returns 0; -1 and nothing written for a NULL context or n, or a level out
   of range). */
int ehs_items(const ehs_ctx* ctx);
long long ehs_level_len(const ehs_ctx* ctx, int level);
int ehs_level_dims(const ehs_ctx* ctx, int level, int n[3]);

/* Wait for all work issued on the context's stream. */
ehs_status ehs_sync(ehs_ctx* ctx);

/* Number of kernels this library has launched since load (diagnostics). */
long long ehs_kernel_launches(void);

/* Message of the last failed call of ctx (or of ehs_create when ctx is NULL). */
const char* ehs_last_error(const ehs_ctx* ctx);

#ifdef __cplusplus
}
#endif
#endif /* EHS_H */
