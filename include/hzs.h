/*
 * hzs.h - C ABI of a GPU solver for the 2-D Helmholtz equation with two-level
 * Schwarz preconditioned GMRES and quadratic B-spline (B_2) coarse spaces.
 *
 * Method: Sieburgh, Heinlein, Dwarka, Vuik, "Coarse Spaces Based on
 * Higher-Order Interpolation for Schwarz Preconditioners for Helmholtz
 * Problems" (arXiv 2408.03571).  Section numbers and equation numbers below
 * refer to that paper.
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 * - Grid functions live on the uniform n x n grid of the unit square, n odd,
 *   h = 1/(n-1) (Section 2).  A grid function is n*n interleaved complex
 *   doubles (re, im), row-major, node (i, j) (i = x index, j = y index) at
 *   flat index j*n + i.  That is the layout of a C-contiguous
 *   torch.complex128 tensor of shape (n, n).  Several right-hand sides are
 *   stored back to back (shape (nrhs, n, n)).
 * - MP-1 (Dirichlet, Eq. 1): the boundary nodes are not unknowns.  Inputs
 *   are read on interior nodes only; outputs are written as 0 on the boundary.
 *   MP-2 (Sommerfeld, Eq. 2): all n*n nodes are unknowns.
 * - All pointers named *_dev are device pointers on the current CUDA device;
 *   the caller allocates, owns and frees them.  Buffers must be 16-byte
 *   aligned.  Input and output buffers must not overlap unless stated.
 * - The library allocates (cudaMalloc) and owns the factors and work space
 *   of a handle; they are freed by the matching destroy call.  A handle must
 *   not be used from two host threads at once.
 * - All work of a handle is issued on the CUDA stream given at grid
 *   creation.  Calls that return results to host memory (hzs_solve_info)
 *   synchronise that stream before returning; the others only enqueue.
 * - Every call returns an hzs_status.  No call aborts or throws.  A
 *   message for the last failure of a handle is available from
 *   hzs_last_error().  Asynchronous device errors surface as HZS_ERR_CUDA at
 *   the next synchronising call.
 */
#ifndef HZS_H
#define HZS_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    HZS_OK = 0,
    HZS_NOT_CONVERGED = 1,        /* soft result: u holds the last iterate, info is filled */
    HZS_ERR_INVALID_ARG = -1,
    HZS_ERR_CUDA = -2,
    HZS_ERR_OOM = -3,
    HZS_ERR_SINGULAR_LOCAL = -4,  /* a zero pivot in a subdomain factorisation */
    HZS_ERR_SINGULAR_COARSE = -5, /* a zero pivot in the coarse factorisation */
    HZS_ERR_NONFINITE = -6,       /* NaN/Inf in the right-hand side or the iteration */
    HZS_ERR_TIMEOUT = -7,
    HZS_ERR_BREAKDOWN = -8
} hzs_status;

/* Boundary condition (Section 2). */
typedef enum { HZS_DIRICHLET = 0 /* MP-1 */, HZS_SOMMERFELD = 1 /* MP-2 */ } hzs_bc;

/* Schwarz preconditioner (Section 3).  Q = R_0^T (R_0 A R_0^T)^{-1} R_0.
 *   HZS_AS1  : sum_i R_i^T A_i^{-1} R_i                      (one level, Section 3)
 *   HZS_AS2  : Q + sum_i R_i^T A_i^{-1} R_i                  (Eq. 4)
 *   HZS_SAS2 : Q + sum_i R_i^T D_i A_i^{-1} R_i              (Eq. 5)
 *   HZS_SHS2 : Q + (sum_i R_i^T D_i A_i^{-1} R_i)(I - A Q)    (Eq. 6)
 * with A_i = R_i A R_i^T solved exactly and D_i the 0/1 owner indicator. */
typedef enum { HZS_AS1 = 0, HZS_AS2 = 1, HZS_SAS2 = 2, HZS_SHS2 = 3 } hzs_precond_kind;

/* Coarse basis (Section 4): linear hats (P_1) or quadratic B-splines of knot
 * spacing H (B_2; for H = 2h these are the weights of Eq. 7). */
typedef enum { HZS_COARSE_NONE = 0, HZS_COARSE_P1 = 1, HZS_COARSE_B2 = 2 } hzs_coarse_kind;

/* HZS_FP64: every step in complex128.  HZS_MIXED: flexible GMRES (Section 5)
 * around a preconditioner whose stencil, transfers and subdomain solves run in
 * complex64, with the coarse solve in FP64 (its factorisation and its product).  The outer
 * matrix-vector product, the Krylov basis (complex128), the Hessenberg least
 * squares and the solution are FP64; the orthogonalisation is the delayed CGS2
 * whose reorthogonalisation coefficients and first-projection update are FP64
 * (see HZS_SOLVE_ORTH_FP64 and HZS_SOLVE_BASIS_DF for the alternatives). */
typedef enum { HZS_FP64 = 0, HZS_MIXED = 1 } hzs_precision;

/* Problem and decomposition (Sections 2 and 3).
 *   n        : grid nodes per axis, odd, >= 5.
 *   bc       : boundary condition.
 *   k        : constant wavenumber, used when kappa_dev is NULL (kappa = k^2).
 *   kappa_dev: optional device array of n*n doubles, the squared wavenumber
 *              kappa = k(x,y)^2 > 0 at every node; copied at creation.
 *   nsub     : subdomains along x; must divide n-1.  Subdomain a owns grid
 *              nodes [a w, (a+1) w) along x, w = (n-1)/nsub, the last one
 *              also node n-1 (MP-1 drops the boundary nodes).
 *   overlap  : node layers added on each side of an owned block, >= 0, at
 *              most half the narrower subdomain width.
 *   nsub_y   : subdomains along y (same rule); 0 = nsub (a square grid of
 *              subdomains). */
typedef struct {
    int n;
    hzs_bc bc;
    double k;
    const double* kappa_dev;
    int nsub;
    int overlap;
    int nsub_y;
} hzs_grid_desc;

/* How the coarse solve A_0^{-1} (Eq. 4) is carried out.  DENSE and BLOCK are exact
 * up to rounding; they differ in cost.  DENSE: explicit inverse by Gauss-Jordan,
 * one dense matrix-vector product per apply (memory |G_H|^2).  BLOCK: block-
 * tridiagonal LU over groups of coarse rows (2 rows for B_2, 1 for P_1), one
 * launch per block step (memory ~3 |G_H|^{3/2} s); with more than two right-hand
 * sides its dense block products run on the tensor cores as FP64-accurate digit-slice
 * products (blocks up to 520 wide; their slices add about 32 s |G_H|^{3/2} bytes;
 * HZS_COARSE_TC=0 in the environment at set-up keeps them on the FP64 pipe, and
 * hzs_precond_info.coarse_tensor_cores reports which).  AUTO: DENSE up to 4096 coarse
 * unknowns, BLOCK above.  MULTILEVEL (never chosen by AUTO; Section 5 names the
 * exact coarse solve as the cost that grows with |G_H|): A_0^{-1} replaced by one
 * application of SHS2 (Eq. 6) on the coarse grid G_H itself - G_H taken as a grid
 * (MP-1: the interior of a Dirichlet grid of nc1 + 2 nodes per axis, MP-2: all nc1),
 * ml_nsub x ml_nsub coarse subdomains with ml_overlap layers of overlap and exact
 * solves of their blocks of A_0, and a B_2 coarse-of-coarse space of ratio ml_ratio
 * with its own exact Galerkin solve; FP64.  It is not exact, so the solve around a
 * preconditioner using it is flexible GMRES (HZS_MIXED) or its step count grows. */
typedef enum {
    HZS_COARSE_SOLVER_AUTO = 0,
    HZS_COARSE_SOLVER_DENSE = 1,
    HZS_COARSE_SOLVER_BLOCK = 2,
    HZS_COARSE_SOLVER_MULTILEVEL = 3
} hzs_coarse_solver;

/* The diagonal D_i of SAS2 and SHS2 (Eqs. 5-6; Section 3 asks only for
 * sum_i R_i^T D_i R_i = I).  OWNER: 1 on the nodes subdomain i owns, 0 on its
 * overlap (restricted additive Schwarz).  MULTIPLICITY: 1/m(x) on every node x
 * of subdomain i, m(x) the number of subdomains containing x. */
typedef enum { HZS_SCALING_OWNER = 0, HZS_SCALING_MULTIPLICITY = 1 } hzs_scaling_mode;

/* Preconditioner set-up (Sections 3 and 4).
 *   coarse_ratio : p = H/h, >= 2, must divide n-1 (ignored for HZS_AS1).
 *   dedup_tiles  : nonzero lets subdomains with identical local matrices share
 *                  one factorisation (only possible for constant k).
 *   coarse_solver: an hzs_coarse_solver (0 = AUTO).
 *   autotune     : 0 = the subdomain solve (Section 3, the exact local solves)
 *                  launches with its fixed default shape; 1 = set-up times the
 *                  shapes that fit (tiles per thread block, depth of the
 *                  factor-block copy ring, threads per block row) on this handle
 *                  and keeps the fastest (more than 2 % ahead of the default, else
 *                  the default), reusing the choice made earlier in the process
 *                  for a problem of the same size and decomposition; 2 = re-time
 *                  even then.  Every shape solves the same tile systems exactly;
 *                  results differ only in the rounding order of block-row sums.
 *                  The paper has no counterpart (it concerns the launch, not the
 *                  method).  Timing synchronises the stream. */
typedef struct {
    hzs_precond_kind kind;
    hzs_coarse_kind coarse;
    int coarse_ratio;
    hzs_precision precision;
    int dedup_tiles;
    int coarse_solver;
    int autotune;
    int scaling_mode;      /* an hzs_scaling_mode (0 = OWNER); used by SAS2 and SHS2 */
    /* HZS_COARSE_SOLVER_MULTILEVEL only: coarse subdomains per axis (must divide the
     * coarse grid's nodes per axis minus one), their overlap in coarse node layers
     * (at most half their width), and the coarse-of-coarse ratio (>= 2, must divide
     * the same number; at most 8192 coarse-of-coarse unknowns).  Invalid values fail
     * set-up with HZS_ERR_INVALID_ARG. */
    int ml_nsub;
    int ml_overlap;
    int ml_ratio;
} hzs_precond_desc;

/* GMRES controls (Section 5): right preconditioning, zero initial guess, no
 * restart; stop when ||f - A u||_2 <= tol ||f||_2 (the GMRES estimate) or
 * after maxit steps. */
typedef struct {
    double tol;
    int maxit;
    int flags;             /* HZS_SOLVE_PROFILE: time the phases of every step */
} hzs_solve_desc;

#define HZS_SOLVE_PROFILE 1
/* Orthogonalisation of the HZS_MIXED solve.  Default: the delayed CGS2
 * (reorthogonalisation of vector j fused with the first projection of step j+1:
 * two passes over the basis per step) on an FP64 basis, with the
 * reorthogonalisation dot products, the norms and the first-projection update
 * computed to FP64 accuracy and the first-projection dot products in complex64 on
 * the leading 24 bits of each entry (the reorthogonalisation of the next step
 * removes what their rounding leaves).  The basis holds each FP64 value exactly
 * as an FP32 head and a 29-bit tail (16 bytes a complex entry, as complex128), and
 * each pass sums part of the basis with FP64 fused multiply-adds and the rest in
 * FP32 three-word expansions whose error bound is below FP64's (the FP64 pipe of
 * the part is 1/64 of its FP32 rate).  HZS_SOLVE_ORTH_DFMA: the same delayed CGS2
 * with every one of those sums in FP64 fused multiply-adds on a complex128 basis
 * (also taken by default when maxit exceeds about 2300).  The environment
 * variables HZS_F53_MASK, _OCC, _DOT_OCC, _WS, _GROUP, _G64, _RING and _UPD_E, read
 * when a solve first makes its work space on a handle, select other launch
 * variants of the default (which vectors take which pipe, blocks per SM, task
 * sizes); every variant computes the same FP64 Arnoldi process and the defaults
 * are the fastest measured.  HZS_SOLVE_ORTH_FP64:
 * classical CGS2 with every dot product and update in FP64 (four passes per
 * step), as HZS_FP64 uses.  HZS_SOLVE_BASIS_DF: the delayed CGS2 on a narrower
 * double-float basis (complex64 rounding + remainder, see HZS_SOLVE_BASIS_WIDE)
 * with complex64 dot products and double-float updates: fewer bytes and no FP64
 * arithmetic, but neither the basis nor its arithmetic is FP64.  No effect with
 * HZS_FP64. */
#define HZS_SOLVE_ORTH_FP64 2
#define HZS_SOLVE_BASIS_DF 16
#define HZS_SOLVE_ORTH_DFMA 32
/* With HZS_SOLVE_BASIS_DF: the basis stores its remainders as complex64 (about
 * 48 significant bits, 16 bytes an entry in all) when tol < 1e-7, else as bf16
 * pairs (about 32 significant bits, 12 bytes an entry: a quarter less basis
 * traffic).  This flag keeps the complex64 remainders at any tol. */
#define HZS_SOLVE_BASIS_WIDE 4
/* Issue the Arnoldi steps (Section 5: preconditioner apply, matrix-vector
 * product, orthogonalisation and Givens update of every right-hand side) as
 * CUDA graphs: chunks of 8 steps are captured on a private stream of the
 * handle and replayed on the grid's stream, the executable graphs updated in
 * place from one chunk to the next and kept by the handle for later solves.
 * Same kernels, arguments and order as without the flag, so the same results;
 * the convergence count is read back once per chunk instead of once per step
 * (steps issued after convergence return at once on the device).  Not
 * combined with HZS_SOLVE_PROFILE (the flag is ignored there). */
#define HZS_SOLVE_GRAPH 8

/* Per right-hand side results. */
typedef struct {
    int iterations;        /* Arnoldi steps taken */
    int converged;         /* 1 if the estimate met tol */
    double relres_est;     /* GMRES residual estimate / ||f|| */
    double relres_true;    /* ||f - A u|| / ||f|| recomputed in FP64 */
    double t_solve_ms;     /* device time of this solve (CUDA events on the stream) */
    double t_precond_ms;   /* with HZS_SOLVE_PROFILE: device time in the preconditioner, */
    double t_matvec_ms;    /*   in the matrix-vector products, */
    double t_orth_ms;      /*   and in the orthogonalisation and Givens update; else 0 */
    double t_orth_dot_ms;  /* with HZS_SOLVE_PROFILE on the delayed-CGS2 path: device time of the */
    double t_orth_update_ms; /*   basis dot pass and of the basis update pass (parts of t_orth_ms); else 0 */
    long long launches;    /* kernel launches this solve issued */
    int basis_bits;        /* significant bits of the Krylov basis: 53 (complex128), 48 or 32 */
    int orth_kind;         /* 0: CGS2 in FP64; 1: delayed CGS2 on the FP64 basis, FP64 and FP32
                              pipes (the HZS_MIXED default); 2: delayed CGS2 on the double-float
                              basis; 3: delayed CGS2 on the FP64 basis, FP64 FMAs only */
    hzs_status status;
} hzs_solve_info;

typedef struct hzs_grid hzs_grid;
typedef struct hzs_precond hzs_precond;

/* Creates the grid, operator and decomposition of Sections 2-3.  cuda_stream
 * is a cudaStream_t (NULL = legacy default stream).  On success *out is a new
 * handle; on failure *out is NULL. */
hzs_status hzs_grid_create(const hzs_grid_desc* desc, void* cuda_stream, hzs_grid** out);
void hzs_grid_destroy(hzs_grid* g);

/* Factorises the subdomain matrices A_i = R_i A R_i^T (exactly, Section 3) and
 * the coarse matrix A_0 = R_0 A R_0^T (Eq. 4, Section 4).  The grid must
 * outlive the preconditioner.  Synchronises the stream. */
hzs_status hzs_precond_setup(hzs_grid* g, const hzs_precond_desc* desc, hzs_precond** out);
void hzs_precond_destroy(hzs_precond* p);

/* y = A x for nrhs grid functions (Eq. 3, second-order finite differences;
 * MP-2 boundary rows are the symmetric ghost-node form).  x_dev and y_dev
 * must not overlap. */
hzs_status hzs_apply_operator(hzs_precond* p, const void* x_dev, void* y_dev, int nrhs);

/* z = M^{-1} v for nrhs grid functions (Eqs. 4-6 or one-level AS), in the
 * preconditioner's precision (complex128 in and out either way). */
hzs_status hzs_apply_precond(hzs_precond* p, const void* v_dev, void* z_dev, int nrhs);

/* Solves A u = f for nrhs right-hand sides with preconditioned GMRES
 * (Section 5; flexible GMRES when the preconditioner is HZS_MIXED).
 * info points to nrhs host structs.  Returns HZS_NOT_CONVERGED if any
 * right-hand side missed tol within maxit. */
hzs_status hzs_solve(hzs_precond* p, const hzs_solve_desc* sd, const void* f_dev, void* u_dev,
                     int nrhs, hzs_solve_info* info);

/* Batched solve of several problems (wavenumbers, grid sizes, decompositions:
 * one preconditioner handle each, all distinct) with several right-hand sides
 * each; the paper solves one right-hand side at a time, this is its batched
 * form.  Problem k solves nrhs[k] right-hand sides f_dev[k] -> u_dev[k] (grid
 * layout as hzs_solve); its info entries follow those of problems 0..k-1.
 * Within a problem the right-hand sides advance in lockstep: every Arnoldi
 * step is one set of kernel launches over all of them, and those that have
 * converged are skipped on the device.  Problems run concurrently on their
 * own host threads; their GPU work overlaps when their grids were created on
 * different streams.  Right-hand sides are taken in chunks as large as the
 * free device memory allows for maxit Krylov vectors each.  hzs_solve with
 * nrhs > 1 uses the same lockstep batches. */
hzs_status hzs_solve_batched(int nprob, hzs_precond* const* probs, const hzs_solve_desc* sd,
                             const void* const* f_dev, void* const* u_dev, const int* nrhs,
                             hzs_solve_info* info);

/* Solves the adjoint system conj(A) lambda = g with the same preconditioned
 * GMRES (as A mu = conj(g), lambda = conj(mu), since A = A^T, Section 2).
 * The paper has no adjoint; it serves the kappa gradient below. */
hzs_status hzs_adjoint_solve(hzs_precond* p, const hzs_solve_desc* sd, const void* g_dev,
                             void* lam_dev, int nrhs, hzs_solve_info* info);

/* grad[node] = -Re( conj(lam[node]) * dA_PP/dkappa_P * u[node] ) for one
 * right-hand side: the gradient of a real loss L(u) w.r.t. the squared
 * wavenumber field, given u = A^{-1} f and lam from hzs_adjoint_solve with
 * g = dL/d(conj u).  grad_dev is n*n doubles (0 on MP-1 boundary nodes).
 * The paper has no counterpart. */
hzs_status hzs_kappa_gradient(hzs_precond* p, const void* u_dev, const void* lam_dev,
                              double* grad_dev);

/* What set-up built and chose for a preconditioner (host struct). */
typedef struct {
    int nfactors;              /* distinct subdomain factorisations (Section 3) */
    int coarse_unknowns;       /* |G_H| unknowns of A_0 (Section 4); 0 for HZS_AS1 */
    int coarse_solver;         /* HZS_COARSE_SOLVER_DENSE, _BLOCK or _MULTILEVEL as resolved; 0 for HZS_AS1 */
    double coarse_min_pivot;   /* smallest pivot magnitude of the coarse factorisation */
    int tile_group;            /* launch shape of the subdomain solve: tiles per thread block, */
    int tile_stages;           /*   depth of the factor-block copy ring, */
    int tile_threads_per_row;  /*   threads per block row */
    int autotuned;             /* 1 if set-up picked that shape by timing (hzs_precond_desc.autotune) */
    double apply_us_default;   /* with autotuning: one preconditioner apply with the default shape, */
    double apply_us_tuned;     /*   and with the chosen one (microseconds, one right-hand side) */
    int coarse_tensor_cores;   /* 1 if the block coarse solve forms the dense products of its sweeps
                                  with more than two right-hand sides on the tensor cores (FP64-
                                  accurate digit-slice products); 0 if on the FP64 pipe */
} hzs_precond_info;

/* Fills *out for p.  The paper has no counterpart. */
hzs_status hzs_precond_get_info(const hzs_precond* p, hzs_precond_info* out);

/* Allocation-free variant of hzs_apply_precond for SAS2 preconditioners
 * (the paper has no counterpart: it concerns how memory is obtained, not the
 * method).  For callers that may not allocate device memory when they apply
 * the preconditioner - hosts that forbid allocation after start-up, or
 * applications that hand all device memory to their own pool.  Computes the same
 * z = M^{-1} v as hzs_apply_precond (same kernels, same result) but takes its
 * work space (the partial restriction sums and the two coarse vectors) from a
 * fixed 1 MiB device array inside the library instead of the handle, and calls
 * no cudaMalloc, cudaFree or other allocating routine.  The caller passes the
 * input v_dev and output z_dev as for hzs_apply_precond.
 * - Only HZS_SAS2 handles are accepted (the other kinds need grid-sized work
 *   space); others, and problems whose work space exceeds 1 MiB
 *   (n * (coarse nodes per axis) complex values plus two coarse vectors),
 *   return HZS_ERR_INVALID_ARG with a message.
 * - The first call on each device looks up the array's device address
 *   (cudaGetSymbolAddress) with that device current; make it before any
 *   stream capture.
 * - Every call shares the one array: calls that overlap on the GPU (other
 *   streams, threads or handles) race and must be serialised by the caller.
 *   Nothing in it needs clearing between calls (each call writes what it reads). */
hzs_status hzs_apply_precond_noalloc(hzs_precond* p, const void* v_dev, void* z_dev, int nrhs);

/* Measured arithmetic rates of the current GPU (operations per second over the
 * whole device; a fused multiply-add counts as 2 flops).  The paper has no
 * counterpart: these are the peaks against which the ALU-bound kernels of this
 * library (the FP64 Gram-Schmidt passes, the FP32 error-free arithmetic) are
 * reported.  Measured, not taken from a data sheet: each rate is one kernel of
 * independent dependency chains of one instruction kind filling the GPU, timed
 * with CUDA events (about a second in all; synchronises a private stream). */
typedef struct {
    double fp32_tflops;    /* FMA.F32 */
    double fp32x2_tflops;  /* packed fma.rn.f32x2 (4 flops an instruction) */
    double fp64_tflops;    /* FMA.F64 */
    double int_tops;       /* 3-input logic op and funnel shift, 10^12 per second */
    double cvt_tops;       /* FP64 <-> FP32 conversions, 10^12 per second */
    double mix_overlap;    /* FP32 and FP64 chains in one kernel: (t_fp32 + t_fp64) / t_both; 2 = full overlap */
    int sms;
    double clock_mhz;      /* the device's nominal SM clock (attribute, not a sample) */
} hzs_pipe_rates;

/* Fills *out for the current device.  Errors: HZS_ERR_INVALID_ARG (out NULL),
 * HZS_ERR_CUDA. */
hzs_status hzs_pipe_peaks(hzs_pipe_rates* out);

/* Human-readable text of a status; never NULL. */
const char* hzs_status_string(hzs_status s);
/* Message of the last failure on this grid (or of the last global failure
 * if g is NULL); never NULL, empty if none. */
const char* hzs_last_error(const hzs_grid* g);

/* Library version string. */
const char* hzs_version(void);

#ifdef __cplusplus
}
#endif
#endif /* HZS_H */
