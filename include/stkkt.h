/*
 * stkkt.h -- C ABI of the GB300 space-time KKT library.
 *
 * The library solves the all-at-once optimality (KKT) system of the 3D
 * unsteady convection-diffusion inverse source problem of Deng, Cai and Zou,
 * "Two-level space-time domain decomposition methods for unsteady inverse
 * problems" (arXiv 1508.06103):
 *
 *   state   C_t = div(a grad C) - div(v C) + f     (Eq. 1)
 *   misfit  J(f) = 1/2 int sum_i (C(x_i,t) - Ceps_i(t))^2 + N_beta(f)   (Eq. 2-3)
 *
 * discretised with trilinear (Q1) finite elements in space on a uniform box,
 * a theta scheme in time (theta = 1/2 is the paper's Crank-Nicolson, Eq. 8)
 * for the state C and adjoint G, and space-time linear elements for the
 * source f (Eq. 9).  The discrete system F_h U = b (Sec. 3.2, Appendix) is
 * solved by right-preconditioned (flexible) GMRES with the one-level
 * space-time restricted additive Schwarz preconditioner (Sec. 3.2) or the
 * two-level multiplicative hybrid with a coarse space-time GMRES solve.
 *
 * Conventions shared by every call
 * --------------------------------
 * Vectors use the paper's point-block order (Sec. 3.2):
 *     U[((n * N + j) * 3 + c)],  c = 0 (C), 1 (G), 2 (f),
 *     node j = ix + nx * (iy + ny * iz), level n = 0..M,  N = nx*ny*nz.
 * Vector arguments are DEVICE pointers (memory of the current CUDA device,
 * e.g. from torch) unless a parameter says "host".  The caller owns them;
 * the library owns its handles and every internal buffer.  Calls are
 * stream-ordered on `stream` (a cudaStream_t passed as void*, NULL = legacy
 * default stream) and do not synchronise, except where stated.
 * Every call returns a kkt_status; on an error the output buffers are
 * unspecified and kkt_last_error() describes the failure.  A *_destroy(NULL)
 * is a no-op.  Handles are not thread-safe: one host thread per handle.
 */
#ifndef STKKT_H
#define STKKT_H

#ifdef __cplusplus
extern "C" {
#endif

typedef int kkt_status;
#define KKT_OK                 0
#define KKT_NOT_CONVERGED      1   /* iteration limit reached            */
#define KKT_BREAKDOWN          2   /* Krylov breakdown before tolerance  */
#define KKT_ERR_ARG           -1   /* invalid argument                   */
#define KKT_ERR_NOMEM         -2   /* device or host allocation failed   */
#define KKT_ERR_CUDA          -3   /* CUDA runtime error                 */
#define KKT_ERR_NONFINITE     -4   /* NaN/Inf met in the solver          */
#define KKT_ERR_ZERO_PIVOT    -5   /* a subdomain factor hit a zero pivot */

/* Face bits of the Dirichlet part Gamma_1 of the boundary (Eq. 1). */
#define KKT_FACE_X0 1u
#define KKT_FACE_X1 2u
#define KKT_FACE_Y0 4u
#define KKT_FACE_Y1 8u
#define KKT_FACE_Z0 16u
#define KKT_FACE_Z1 32u

/* Spatial elements on the grid's cells (Sec. 3.1; kkt_set_element). */
#define KKT_ELEM_Q1 0   /* trilinear elements on the hexahedral cells (the default) */
#define KKT_ELEM_P1 1   /* linear elements on the Kuhn split of every cell into six tetrahedra */

/* Uniform grid of cx*cy*cz hexahedral cells on [0,lx]x[0,ly]x[0,lz]. */
typedef struct {
  int cx, cy, cz;
  double lx, ly, lz;
  unsigned dirichlet_faces;   /* bit mask of KKT_FACE_*; the rest is Neumann */
} kkt_grid;

typedef struct kkt_problem kkt_problem;     /* opaque */
typedef struct ras_precond ras_precond;     /* opaque */
typedef struct coarse_level coarse_level;   /* opaque */

/* Text of the last error on the calling thread (static storage). */
const char* kkt_last_error(void);

/* Library version string. */
const char* kkt_version(void);

/*
 * kkt_create -- build the discrete KKT operator F_h (Sec. 3.1, Appendix).
 *   g           grid and Dirichlet faces (host).
 *   nt, dt      M = nt time steps of size tau = dt (levels 0..M).
 *   a_cell      host, cx*cy*cz values of the diffusivity a at cell centroids
 *               (cell id ex + cx*(ey + cy*ez)); a is constant per cell.
 *   v_cell      host, 3*cx*cy*cz values (vx, vy, vz per cell) of the velocity.
 *   sensor_node host, nsens node ids of the sensors (already snapped to nodes;
 *               repeats count twice; sensors on Dirichlet nodes are ignored,
 *               their rows being identity rows).  May be NULL if nsens == 0.
 *   beta1, beta2 regularisation weights of N_beta (Eq. 3).
 *   theta       time weight: 0.5 = Crank-Nicolson (Eq. 8), 1 = implicit Euler;
 *               must lie in [0.5, 1].
 *   out         receives the handle.
 * Runs synchronously (uploads the stencil coefficients); errors: ARG, NOMEM, CUDA.
 */
kkt_status kkt_create(const kkt_grid* g, int nt, double dt, const double* a_cell,
                      const double* v_cell, const int* sensor_node, int nsens,
                      double beta1, double beta2, double theta, kkt_problem** out);

/*
 * kkt_set_regularization -- choose the source regularisation of the f rows.
 *   reg 0: H1-H1, N_beta of Eq. 3 (the default after kkt_create): the beta2
 *          term of W^{nm} is beta2 Mt[n,m] K (the (grad f, grad g) form of Eq. 9);
 *   reg 1: H1-L2 of Sec. 4 (Example 2), beta2 |grad f|^2 replaced by beta2 f^2:
 *          the beta2 term is beta2 Mt[n,m] B.
 * kkt_apply, kkt_residual and gmres_solve read the setting at each call;
 * ras_setup / coarse_setup (and their refactorisations) build their matrices
 * from it, so set it before creating the preconditioners of this problem.
 * Host only, no device work.  Errors: ARG (null problem, reg not 0 or 1).
 */
kkt_status kkt_set_regularization(kkt_problem* p, int reg);

/*
 * kkt_set_element -- choose the spatial element of B, A, E_s and K (Sec. 3.1:
 * continuous piecewise-linear elements on a regular triangulation).
 *   elem KKT_ELEM_Q1: trilinear elements on the hexahedral cells (the default
 *        after kkt_create; 27-point stencils);
 *   elem KKT_ELEM_P1: linear elements on the Kuhn split of every cell into six
 *        tetrahedra around its main diagonal (0,0,0)-(1,1,1), the same split in
 *        every cell (a conforming triangulation); each node couples with the 14
 *        neighbours whose offset has all nonzero components of one sign.
 * The block rows of F_h (Appendix) are the same for both.  The subdomain
 * factorisations keep the 27-point structural pattern of the grid: under P1
 * the 12 couplings the split does not make are structural zeros, and ILU(0)
 * admits fill there.  Reassembles the coefficients from the a and v given to
 * kkt_create (synchronous, on the legacy default stream); set it before
 * creating the preconditioners of this problem, as with
 * kkt_set_regularization; coarse_setup copies the fine level's element.
 * Errors: ARG (null problem, unknown elem), NOMEM, CUDA (the problem then
 * keeps its previous element).
 */
kkt_status kkt_set_element(kkt_problem* p, int elem);

/* Sizes of a problem: nodes per axis, N, levels M+1 and unknowns 3*N*(M+1). */
kkt_status kkt_sizes(const kkt_problem* p, int* nx, int* ny, int* nz, int* levels,
                     long long* unknowns);

/*
 * kkt_rhs -- right-hand side b of F_h U = b (Appendix):
 *   C slot at level 0 = c0 (zero if c0 == NULL; zero on Dirichlet nodes),
 *   G slot at level n < M = tau * sum_{sensors k at node j}
 *                            ((1-theta) c_obs[n][k] + theta c_obs[n+1][k]),
 *   every other slot 0 (homogeneous Dirichlet data p and Neumann data q).
 *   c_obs  device, (M+1) x nsens observations Ceps, row = time level.
 *   c0     device, N initial values, or NULL.
 *   b      device, 3*N*(M+1) output.
 */
kkt_status kkt_rhs(kkt_problem* p, const double* c_obs, const double* c0, double* b, void* stream);

/*
 * kkt_apply -- y = F_h x, the KKT matvec (Appendix block rows, Eq. 8-9),
 *   one fused 4D stencil pass over C, G and f.
 *   precision 64: x, y are double*;  32: x, y are float* (FP32 arithmetic).
 *   x and y must not overlap.
 */
kkt_status kkt_apply(kkt_problem* p, const void* x, void* y, int precision, void* stream);

/*
 * kkt_residual -- r = b - F_h x in FP64 (the true residual of Sec. 4's stop test).
 */
kkt_status kkt_residual(kkt_problem* p, const double* b, const double* x, double* r, void* stream);

/*
 * ras_local_pattern -- slots per row type (C, G, f) of an interior point under a
 *   subdomain solver: local 0 ILU(0) (F_h's structural pattern: 108, 56, 162),
 *   2 ILU(1) (the pattern with one level of fill, Sec. 4 Table 1), 3 the 3x3
 *   point-block ILU(0) (243 each: the 81-point neighbourhood, all components).
 *   Host only, no device work.  Errors: ARG.
 */
kkt_status ras_local_pattern(int local, int counts[3]);

/*
 * ras_setup -- one-level space-time restricted additive Schwarz preconditioner
 *   (Sec. 3.2): nsub[0..3] = subdomains along x, y, z and time (part k of n
 *   nodes or levels holds floor(n/p) + (k < n mod p)); each box is extended
 *   by `overlap` nodes/levels per side and trimmed to the domain.  The
 *   subdomain matrix is the principal submatrix of F_h on the extended box
 *   (homogeneous Dirichlet conditions on all cut space and time faces,
 *   Eq. 10-12) and is factored by ILU(0) on its structural pattern.
 *   local        0 = ILU(0); 1 = exact LU with partial pivoting of every box
 *                matrix, stored as a band in the box's natural point-block
 *                order (FP64 only; for small boxes: at most 28,672 unknowns
 *                and half-bandwidth 2,048 per box, else KKT_ERR_ARG, and the
 *                bands must fit in 80 % of free device memory, else
 *                KKT_ERR_NOMEM); 2 = ILU(1), the incomplete factorisation on
 *                the pattern with one level of fill (Sec. 4, Table 1; per
 *                point, so boxes near faces keep only the fill their own
 *                elimination paths make); 3 = 3x3 point-block ILU(0), the
 *                incomplete factorisation on the pattern of whole point
 *                blocks of the 81-point neighbourhood (Sec. 3.2 point-block
 *                ordering; diagonal blocks factored exactly).  2 and 3: FP64
 *                or FP32 (factor_prec 64 or 32), one problem, factor values
 *                stored point-major per box (ras_local_pattern slots per row),
 *                no static apply; their solve runs one CTA per box with a
 *                barrier per wavefront.
 *   factor_prec  64 = factor and solve in FP64, 32 = FP32, 16 = factor in FP32
 *                and store the factors as BF16 (round to nearest); the solve
 *                converts them to FP32 and accumulates in FP32.
 *   All boxes factor in one launch, synchronously; errors: ARG, NOMEM, CUDA,
 *   ZERO_PIVOT.
 */
kkt_status ras_setup(kkt_problem* p, const int nsub[4], int overlap, int local, int factor_prec,
                     ras_precond** out);

/*
 * ras_setup_shape -- ras_setup with a requested shape of the subdomain solve
 *   (a tuning and testing hook; the paper has no counterpart).  The shape
 *   decides how the solve kernel runs, not what it computes: every compiled
 *   shape applies the same ILU(0) factors.
 *   shape[0]  points per chunk of a wavefront (FP64: 34, 26, 18; FP32: 52, 36,
 *             20; BF16: 72, 40, 8)
 *   shape[1]  buffers of the factor-copy ring, 2..4
 *   shape[2]  lanes per point: 4 (the one compiled)
 *   shape[3]  1 = local vectors in shared memory, 2 = in global memory
 *   A 0 in a field leaves that choice to the library (as ras_setup does).
 *   Errors: ARG when no compiled shape matches or the chosen one does not fit
 *   the device's shared memory; otherwise those of ras_setup.
 */
kkt_status ras_setup_shape(kkt_problem* p, const int nsub[4], int overlap, int local, int factor_prec,
                           const int shape[4], ras_precond** out);

/*
 * ras_setup_batch -- one-level RAS of several independent problems solved
 *   together (a batching form of this library; the paper solves one problem):
 *   every problem is split by nsub (overlap, ILU(0) local solves, factor_prec as
 *   in ras_setup) and the boxes of all problems form one list, largest first,
 *   so one factorisation launch and one subdomain-solve launch cover all of
 *   them.  Vectors of such a preconditioner concatenate the problems' unknowns
 *   in the order given (problem k starts after the 3*N*(M+1) unknowns of
 *   problems 0..k-1).  shape: NULL or as in ras_setup_shape (e.g. from
 *   ras_autotune).  The problems must outlive the handle.  Synchronous;
 *   errors: ARG, NOMEM, CUDA, ZERO_PIVOT.
 */
kkt_status ras_setup_batch(kkt_problem* const* probs, int nprob, const int nsub[4], int overlap,
                           int factor_prec, const int shape[4], ras_precond** out);

/*
 * ras_autotune -- choose the subdomain solve's shape by measurement: every
 *   compiled chunk size with 2 and 3 copy buffers is set up on these problems
 *   (split as in ras_setup_batch, ILU(0), factor_prec) and timed over `reps`
 *   applies with CUDA events; shape_out gets the fastest {chunk points, ring
 *   buffers, 4, 0} and *best_ms (may be NULL) its time per apply.  With a
 *   cache_path (may be NULL) an earlier result for the same problem sizes,
 *   split, precision and device is read from that text file instead, and a
 *   new one is appended.  Synchronous; a tuning aid with no counterpart in the
 *   paper.  Errors: ARG, NOMEM, CUDA, ZERO_PIVOT.
 */
kkt_status ras_autotune(kkt_problem* const* probs, int nprob, const int nsub[4], int overlap, int factor_prec,
                        int reps, const char* cache_path, int shape_out[4], double* best_ms);

/*
 * ras_info -- sizes of a preconditioner: boxes, points of all extended boxes
 *   (with overlap), stored factor values and bytes per value.  Any output may
 *   be NULL.
 */
kkt_status ras_info(const ras_precond* m, int* nbox, long long* points, long long* factor_values,
                    int* value_bytes);

/*
 * ras_solve_shape -- how the subdomain solve of a preconditioner runs (chosen
 *   at ras_setup from the boxes' sizes and the device's occupancy): points per
 *   chunk of a wavefront, buffers of its factor-copy ring, lanes per point,
 *   and 1 if the local vectors live in shared memory.  Any output may be
 *   NULL.  Reporting only; the paper has no counterpart.
 */
kkt_status ras_solve_shape(const ras_precond* m, int* chunk_points, int* stages, int* lanes, int* smem_vectors);

/*
 * ras_status -- the preconditioner's device status word, read on `stream`
 *   (synchronises that stream): 0 = fine; 1 = the last factorisation met a
 *   zero or non-finite pivot (returns ZERO_PIVOT); 2 = a subdomain solve gave
 *   up waiting for a factor copy after its 2 s limit and left z unwritten
 *   (returns ERR_CUDA).  ras_apply and ras_apply_static never synchronise, so
 *   a caller that does not go through gmres_solve reads the outcome of its
 *   applies here.  The word is cleared by ras_refactor.
 */
kkt_status ras_status(ras_precond* m, int* code, void* stream);

/*
 * ras_selftest_wait -- test hook for the bounded waits (no counterpart in the
 *   paper): launches one thread that waits, for limit_ms milliseconds
 *   (0 < limit_ms <= 1000), on an mbarrier that nothing completes, with the
 *   same bounded wait the subdomain solve uses; the wait gives up, sets the
 *   status word of m to 2 and the kernel returns.  Nothing is copied; the
 *   device and the handle stay usable (ras_refactor clears the word).
 */
kkt_status ras_selftest_wait(ras_precond* m, double limit_ms, void* stream);

/*
 * ras_apply -- z = sum_ij (R^0_ij)^T M_ij^{-1} R^delta_ij r (restricted prolongation,
 *   Cai-Sarkis form cited in Sec. 3.2); all boxes in one launch.  r, z FP64,
 *   3*N*(M+1) values each; the two spans must not overlap (ERR_ARG).  Does not
 *   synchronise; a solve that gave up on a factor copy is reported by
 *   ras_status (and by gmres_solve).
 */
kkt_status ras_apply(ras_precond* m, const double* r, double* z, void* stream);

/*
 * ras_apply_static -- the same one-level RAS apply as ras_apply, for callers
 *   that cannot call cudaMalloc: code running while another component owns the
 *   device's memory pool, or a loop that must never trigger the device-wide
 *   synchronisation an allocation can cause.  It allocates nothing: besides r,
 *   z and the factors held by the handle, the only memory it touches is one
 *   fixed 32 MiB array compiled into the library, which every GPU that loads
 *   the library holds until the process exits.  (The paper has no counterpart;
 *   this is an interface convenience.)
 *   Limit: when the solve keeps the local vectors in global memory
 *   (ras_solve_shape reports smem_vectors = 0), the padded local vectors of
 *   all subdomains must fit in the array, i.e. 4 * sum over boxes of
 *   (lx+2)(ly+2)(lz+2)(lt+2) values of the factor precision (FP32 for BF16
 *   factors; 4 values per padded point) <= 32 MiB; larger handles get
 *   KKT_ERR_ARG (use ras_apply).  A
 *   solve whose local vectors live in shared memory does not touch the array
 *   and has no limit.
 *   The first call on a device looks the array's device address up
 *   (cudaGetSymbolAddress) and caches it; make that first call before any
 *   stream capture.  Every call that uses the array clears the part it uses on
 *   `stream` before the solve.  All calls share the one array, so calls whose
 *   work overlaps on the GPU (other streams, other threads) race: order them.
 */
kkt_status ras_apply_static(ras_precond* m, const double* r, double* z, void* stream);

/*
 * coarse_setup -- the coarse space-time level of the two-level method (Sec. 3.2):
 *   a nested coarse mesh of ccx x ccy x ccz cells and cnt steps (each must
 *   divide the fine one), rediscretised with cell-mean a and v and with each
 *   fine sensor node snapped to the nearest coarse node; a one-level RAS on
 *   it with nsub_c subdomains and overlap c_overlap; interpolation I^h_c
 *   multilinear in (x, y, z, t) and restriction I^c_h = (I^h_c)^T; the coarse
 *   solve F_c^{-1} is GMRES right-preconditioned by that RAS, stopped at
 *   relative residual c_rtol or after c_maxit iterations.  Synchronous.
 */
kkt_status coarse_setup(kkt_problem* fine, int ccx, int ccy, int ccz, int cnt, const int nsub_c[4],
                        int c_overlap, double c_rtol, int c_maxit, int factor_prec,
                        coarse_level** out);

/*
 * two_level_apply -- z = y + M_one^{-1}(x - F_h y), y = I^h_c F_c^{-1} I^c_h x
 *   (the multiplicative hybrid of Sec. 3.2).  Synchronises the stream once
 *   per coarse GMRES iteration.
 */
kkt_status two_level_apply(coarse_level* c, ras_precond* fine, const double* x, double* z, void* stream);

/*
 * gmres_solve -- right-preconditioned restarted GMRES(restart) (flexible when
 *   `flexible` != 0, required with a coarse level) for F_h x = b (Sec. 3.2, 4).
 *   Orthogonalisation is classical Gram-Schmidt applied twice; Arnoldi vectors,
 *   Givens rotations and the true residual are FP64.  The method stops when
 *   the true residual ||b - F_h x||_2 <= rtol ||b||_2 (checked when the
 *   Arnoldi estimate passes) or after maxit iterations.
 *   m      one-level preconditioner or NULL (unpreconditioned).
 *   c      coarse level or NULL (one-level).
 *   x      device FP64; holds the initial guess on entry (zero in the paper).
 *   iters, true_relres  host outputs (may be NULL).
 *   Synchronises the stream; returns OK, NOT_CONVERGED, BREAKDOWN or an error.
 */
kkt_status gmres_solve(kkt_problem* p, ras_precond* m, coarse_level* c, const double* b, double* x,
                       int restart, double rtol, int maxit, int flexible, int* iters,
                       double* true_relres, void* stream);

/*
 * reduced_solve -- the KKT solution by the reduced-space ("traditional")
 *   method of Sec. 1, the approach the all-at-once solve is compared with: f
 *   is the only unknown, and every application of the reduced operator
 *     H f = W f - D G_lin(C_lin(f)),  W = beta1 Lt (x) B + beta2 Mt (x) K
 *     (H1-L2: Mt (x) B),  D = Mt (x) B   (the f rows of the Appendix)
 *   is a forward march of the M state steps of Eq. 8 and a backward march of
 *   the M adjoint steps.  H f = D G0 (G0: the adjoint of the state from c0
 *   against the data) is solved by GMRES(restart), right-preconditioned by
 *   P = W + sigma Mt (x) B applied by fast diagonalisation (exact for trilinear
 *   elements; an approximation under P1), to relative residual rtol or maxit
 *   iterations; then U = (C, G, f) with the state and adjoint of f.  Each
 *   spatial step (B + theta tau S, or S^T; identity rows on Dirichlet nodes)
 *   is solved by Jacobi-preconditioned GMRES(40) on the device to relative
 *   residual step_rtol, from the neighbouring level.
 *   c_obs  device FP64, (M+1) x nsens sensor values (may be NULL if nsens == 0);
 *   c0     device FP64, N initial state values, or NULL (zero);
 *   U      device FP64, 3 N (M+1): the KKT solution, point-block order;
 *   iters, relres  host: outer GMRES iterations and relative residual of the
 *          reduced system (may be NULL);
 *   stats  host, 4 values (may be NULL): applications of H, step solves, step
 *          GMRES iterations in total, the most in one step solve.
 *   Allocates its workspace for the call (restart + 1 vectors of N (M+1)
 *   values, 6 N (M+1) more, 2 x 41 level vectors) and synchronises the stream
 *   once per step solve.  Returns OK, NOT_CONVERGED (outer iteration limit) or
 *   BREAKDOWN (outer Krylov breakdown) with U written, or an error; a step
 *   solve that misses step_rtol within 2,000 iterations returns NOT_CONVERGED
 *   (BREAKDOWN on a breakdown) before U is written.
 */
kkt_status reduced_solve(kkt_problem* p, const double* c_obs, const double* c0, double* U, int restart,
                         double rtol, int maxit, double step_rtol, int* iters, double* relres,
                         long long stats[4], void* stream);

/*
 * gmres_solve_batch -- flexible GMRES(restart) on several independent problems
 *   at once, right-preconditioned by their ras_setup_batch preconditioner m
 *   (probs in the same order): b, x device FP64 vectors over the concatenated
 *   unknowns (x's initial contents are ignored: zero initial guess).  The
 *   problems step in lockstep; every problem has its own Arnoldi process,
 *   rotations and stop test on the device (stop at its own true residual
 *   ||b_k - F_k x_k|| <= rtol ||b_k||), and a problem that has stopped no
 *   longer does work.  A restart cycle of all problems is one captured CUDA
 *   graph, replayed with one host round trip per cycle.  iters, true_relres,
 *   status: host arrays of nprob entries (may be NULL).  Returns OK when every
 *   problem converged, else the most severe problem status (errors first).
 *   Synchronises the stream.
 */
kkt_status gmres_solve_batch(kkt_problem* const* probs, int nprob, ras_precond* m, const double* b, double* x,
                             int restart, double rtol, int maxit, int* iters, double* true_relres, int* status,
                             void* stream);

/*
 * ras_refactor -- recompute the ILU(0) factors of an existing preconditioner in
 *   place from its problem's current coefficients (the factorisation step of
 *   ras_setup without any allocation).  Enqueued on `stream`, then synchronises
 *   it to report a zero pivot.  Errors: ARG, CUDA, ZERO_PIVOT.
 */
kkt_status ras_refactor(ras_precond* m, void* stream);

/* coarse_refactor -- ras_refactor of the coarse level's one-level RAS. */
kkt_status coarse_refactor(coarse_level* c, void* stream);

/*
 * two_level_refactor -- ras_refactor of `fine` and coarse_refactor of `c`
 *   together: the coarse factorisation runs on a second stream of the library
 *   (created on the first call) forked from and joined back into `stream`, so
 *   it can use the SMs the fine one leaves idle.  Synchronises `stream` once;
 *   errors: ARG (fine is not c's fine level), CUDA, ZERO_PIVOT.  A scheduling
 *   convenience of this library; the paper has no counterpart.
 */
kkt_status two_level_refactor(coarse_level* c, ras_precond* fine, void* stream);

/*
 * Instrumentation (no effect on results).
 * kkt_launch_count  -- number of CUDA kernels the library has launched since it
 *                      was loaded (all handles, all threads).
 * kkt_timing_enable -- 1: bracket every launch of the outer KKT matvec and of the
 *                      RAS subdomain-solve kernel with CUDA events on the launch
 *                      stream; 0: stop.  Returns the previous setting.
 * kkt_timing_read   -- accumulated event time (ms) and launch count of the FP64
 *                      matvecs issued by the solver on problem p (synchronises
 *                      on the recorded events).
 * ras_timing_read   -- the same for launches of RAS m: kernel 0 = subdomain
 *                      solve, 1 = ILU(0) factorisation.
 * kkt_timing_reset  -- clear the accumulators of p and m (either may be NULL).
 */
long long kkt_launch_count(void);
int kkt_timing_enable(int on);
kkt_status kkt_timing_read(kkt_problem* p, double* total_ms, long long* launches);
kkt_status ras_timing_read(ras_precond* m, int kernel, double* total_ms, long long* launches);
kkt_status kkt_timing_reset(kkt_problem* p, ras_precond* m);

/*
 * kkt_fma_peak -- measured multiply-add rate of the current device in FP64
 *   (precision 64) or FP32 (32), in TFLOP/s (2 flops per FMA), from one
 *   launch of independent register-resident FMA chains on every SM, timed
 *   with CUDA events on `stream` (synchronises it); *ms (may be NULL) gets
 *   the launch time.  Instrumentation: the denominator of the FP64 KKT
 *   matvec's pipe fraction; the paper has no counterpart.  Errors: ARG, CUDA.
 */
kkt_status kkt_fma_peak(int precision, double* tflops, double* ms, void* stream);

/*
 * kkt_mma_peak -- measured FP64 tensor-core rate of the current device: every
 *   warp runs 8 independent chains of the m8n8k4 FP64 warp-level
 *   matrix multiply-accumulate (512 flops per instruction) on register
 *   operands; CUDA events on `stream`.  Instrumentation beside kkt_fma_peak (it
 *   decides whether FP64 MMA could beat the FP64 FMA pipe on dense panels).
 *   tflops (host) required, ms (host) optional.  Errors: ARG, CUDA.
 */
kkt_status kkt_mma_peak(double* tflops, double* ms, void* stream);

/*
 * recover_source -- f of the point-block vector U as an (M+1) x N array
 *   (Sec. 3.2 ordering; the recovered source of the inverse problem).
 */
kkt_status recover_source(kkt_problem* p, const double* U, double* f, void* stream);

void kkt_destroy(kkt_problem* p);
void ras_destroy(ras_precond* m);
void coarse_destroy(coarse_level* c);

#ifdef __cplusplus
}
#endif
#endif /* STKKT_H */
