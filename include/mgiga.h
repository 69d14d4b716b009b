/*
 * mgiga.h -- C ABI of libmgiga, a GB300 (sm_103a) multigrid solver for
 * multi-patch isogeometric Poisson problems.
 *
 * Method: Takacs, "Fast multigrid solvers for conforming and non-conforming
 * multi-patch Isogeometric Analysis" (arXiv:1902.01818).
 *   - Poisson problem -Laplace u = f, u = 0 on the boundary (Sec. 2, Eq. model0,
 *     Eq. model after homogenisation).
 *   - multi-patch domain, patches G_k((0,1)^d) (Sec. 2, Eq. omega:1/2), tensor
 *     B-splines of degree p and maximal smoothness on every patch (Eq. local).
 *   - conforming coupling (Sec. 2, Eq. igaspace0) or symmetric interior penalty
 *     (SIPG) coupling of non-matching patches (Sec. 3, Eq. model:discr2).
 *   - V-cycle multigrid (Algorithm 1) with the subspace-corrected mass smoother
 *     (Sec. 5, Eq. Ldef), Gauss-Seidel (Sec. 4) or the hybrid smoother
 *     (Algorithm 2), used directly or as preconditioner of CG (Sec. 4).
 *
 * Conventions (all entry points):
 *   - Every call returns an mgiga_status and never aborts.  After an error the
 *     handle stays valid for mgiga_last_error() and mgiga_destroy().
 *   - Input arrays are borrowed for the duration of the call only (copied).
 *     Output arrays are allocated by the caller.
 *   - Host-pointer entry points take host memory.  Entry points with the
 *     suffix _d take device pointers (CUDA global memory of the current
 *     device, e.g. the data pointer of a torch tensor) and run on the
 *     handle's stream; they return when the result is ready.
 *   - Global DoF order of a level (integer work): patches in id order; within
 *     a patch the local order i_0 + N_0 (i_1 + N_1 i_2) (xi_0 fastest, N_a the
 *     number of B-splines in direction a); DoFs with a nonzero trace on a
 *     patch side that is listed in no interface are Dirichlet DoFs and are
 *     skipped; in the conforming case a DoF already numbered through a
 *     lower-id patch is skipped.
 *   - A handle is used by one host thread at a time.
 *   - The library allocates its own device memory with cudaMalloc when
 *     mgiga_assemble() runs and frees it in mgiga_destroy().
 */
#ifndef MGIGA_H
#define MGIGA_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct mgiga_handle mgiga_handle;

typedef enum {
  MGIGA_OK = 0,
  MGIGA_EINVAL = 1,      /* invalid argument or problem description */
  MGIGA_ENOMEM = 2,      /* host or device allocation failed, or hbm_budget exceeded */
  MGIGA_ECUDA = 3,       /* a CUDA runtime call failed (text in mgiga_last_error) */
  MGIGA_ENOTSPD = 4,     /* a Cholesky factorisation broke down (penalty too small, bad geometry) */
  MGIGA_ENOCONV = 5,     /* max_iter reached; the output holds the last iterate */
  MGIGA_EBREAKDOWN = 6,  /* NaN/Inf or p^T A p <= 0 in CG */
  MGIGA_ETIMEOUT = 7,    /* a bounded device wait expired */
  MGIGA_ESTATE = 8       /* call out of order (e.g. solve before assemble) */
} mgiga_status;

/* coupling */
enum { MGIGA_CONFORMING = 0, MGIGA_SIPG = 1 };
/* smoother: subspace-corrected mass smoother (Sec. 5), Gauss-Seidel (Sec. 4),
 * hybrid (Algorithm 2) */
enum { MGIGA_SMOOTHER_SCMS = 0, MGIGA_SMOOTHER_GS = 1, MGIGA_SMOOTHER_HYBRID = 2 };
/* outer iteration: CG preconditioned by one V-cycle, or the V-cycle as solver */
enum { MGIGA_OUTER_PCG = 0, MGIGA_OUTER_DIRECT = 1 };
/* arithmetic of the preconditioner (the outer CG is always FP64):
 * MGIGA_PREC_FP64: everything FP64 (the path checked against the oracle).
 * MGIGA_PREC_FP32: inside the cycle, on every level but the coarsest, the
 *   fast-diagonalisation contractions, the Gauss-Seidel sweeps (a colour-ordered
 *   FP32 copy of the band), the interface-piece solves (FP32 inverses), the
 *   residuals (FP32 band coefficients and FP32 sums; the SIPG cross-patch
 *   terms stay FP64) and the transfers compute in FP32, while the vectors
 *   between the stages are stored in FP64.  The coarse Cholesky solve, the
 *   CG band product, all CG vectors and inner products stay FP64, and CG
 *   uses the flexible (Polak-Ribiere) beta.
 * MGIGA_PREC_TF32 / MGIGA_PREC_BF16: as FP32, with the fast-diagonalisation
 *   contractions of large patch interiors on the tensor cores (tcgen05, TF32
 *   or BF16 operands, FP32 accumulation). */
enum { MGIGA_PREC_FP64 = 0, MGIGA_PREC_FP32 = 1, MGIGA_PREC_TF32 = 2, MGIGA_PREC_BF16 = 3 };

/* One interface between side_a of patch_a and side_b of patch_b.
 * side: 2a + 0 is xi_a = 0, 2a + 1 is xi_a = 1 (a = 0..d-1).
 * The tangential directions of a side are the other directions in increasing
 * order.  orient maps the tangential parameter s of side_a to side_b: bit 2
 * (d = 3) swaps the two coordinates, then bit m flips coordinate m of side_b
 * (s_m -> 1 - s_m).  The geometry maps must agree on the interface under this
 * map (Sec. 3, Theorem 2 assumption).  A patch side listed in no interface
 * carries the homogeneous Dirichlet condition (Sec. 3, Eq. igaspace). */
typedef struct {
  int patch_a, side_a, patch_b, side_b;
  unsigned orient;
} mgiga_interface;

/* Problem statement (Sec. 2 Eq. omega:1/2 and Eq. local; Sec. 3).
 * Every patch has one spline degree p_k >= 1 in all directions, maximal
 * smoothness (simple interior knots) and open knot vectors (end multiplicity
 * p_k + 1).  degrees: NULL (every patch has degree `degree`) or num_patches
 * degrees, one per patch, whose largest must equal `degree` -- the
 * non-matching spaces of the SIPG experiments of Sec. 5 (Table SCMS2: one
 * third of the patches S_{p,h}, one third S_{p+1,2h}, one third S_{p,2h});
 * conforming coupling needs equal degrees on both sides of every interface.
 * The patch bands of all levels then span offsets -degree .. degree (the
 * coefficients beyond a patch's own degree are zero) and the Gauss-Seidel
 * colours use degree + 1 as modulus.  The knot vector of level l-1 keeps every other
 * breakpoint of level l (uniform refinement, Sec. 2), so every direction of
 * every patch needs an even number of intervals on all but the coarsest level.
 *   num_knots[k*dim + a]      length of the knot vector of patch k, direction a
 *   knots                     all knot vectors concatenated (k major, then a)
 *   geo_degree                degree q of the geometry splines (1 = multilinear)
 *   geo_num_knots[k*dim + a]  lengths of the geometry knot vectors
 *   geo_knots                 geometry knot vectors concatenated
 *   geo_ctrl                  control points, per patch prod_a(n_cp,a) points of
 *                             dim doubles, xi_0 fastest; patches concatenated
 *   coupling                  MGIGA_CONFORMING (matching interfaces, Assumption 2)
 *                             or MGIGA_SIPG
 *   sipg_penalty              C of the penalty eta = C / h_I on an interface,
 *                             h_I = min(h_a, h_b), h of a patch its largest
 *                             finest-level knot span; eta is frozen on coarse
 *                             levels (Sec. 3, Eq. a:galerkin).  The workloads
 *                             use C = 5 (p + 1)^2. */
typedef struct {
  int dim, num_patches, degree;
  const int* num_knots;
  const double* knots;
  int geo_degree;
  const int* geo_num_knots;
  const double* geo_knots;
  const double* geo_ctrl;
  int num_interfaces;
  const mgiga_interface* interfaces;
  int coupling;
  double sipg_penalty;
  const int* degrees;
} mgiga_problem;

/* Solver options.  levels: number of grid levels (0 = coarsen while every
 * patch direction has an even interval count whose half is >= 2 (d=2) or
 * >= 3 (d=3)).  tau: damping of the smoother (Eq. Ldef); delta: scaling, the
 * interior operator's mass term is 1/(delta h_l^2) (Sec. 5).  nu: smoothing
 * steps; mu: 1 = V-cycle.  max_iter bounds the outer iterations.
 * hbm_budget: 0 = no limit, else mgiga_assemble fails with MGIGA_ENOMEM when
 * its device footprint would exceed it (before any host assembly when the
 * FP64 operators of all levels alone exceed it).  stream: a cudaStream_t on which all
 * device work of the handle runs (NULL: the handle creates its own
 * non-blocking stream; set-up copies run on it, and the _d entry points order
 * it after work already queued on the legacy default stream).  Handles used
 * from different host threads may set up and solve concurrently.
 * gs_cluster: 0 = automatic; 2, 4, 8 or 16 = the thread-block cluster size
 * (CTAs per patch) preferred by the patch-parallel Gauss-Seidel sweep of the
 * mixed path on large levels.  Automatic takes 16 (fastest when the handle has
 * the GPU to itself); when several handles solve concurrently on their own
 * streams, 8 packs better into the GPU's processing clusters.
 * autotune: 1 = at mgiga_assemble, pick per level the contraction engine of the
 * fast diagonalisation (batched SIMT tiles, tensor-core tiles, one CTA per
 * patch) and the row blocking of the FP32 cycle residual by timing the
 * candidates on the device, once per size bucket (a factor sqrt(2) in the
 * interior size / the level's rows) for the process; later handles of a known
 * bucket reuse the choice.  0 = the built-in rules.  The paper has no
 * counterpart; the choice changes only the FP32 summation order.
 * matrix_free: 1 = the residuals the cycle computes on the finest level
 * (before the smoothers and the restriction) evaluate the stiffness action
 * at the Gauss points by sum factorisation instead of reading a stored band
 * (Sec. 2, Eq. linear:system:0: the same bilinear form and quadrature, with
 * p + 1 points per element and direction), with the geometric factors
 * computed from the geometry's control points; the SIPG terms (Sec. 3) stay
 * stored.  In the FP32/TF32/BF16 modes this replaces the FP32 copy of the
 * finest band (which is then not allocated); its arithmetic is the mode's
 * (FP32, or FP64 in the FP64 mode).  The outer CG's product keeps the FP64
 * band.  Needs maximal smoothness and a geometry map that is one polynomial
 * piece of degree <= 2 per patch; else mgiga_assemble returns MGIGA_EINVAL.
 * 0 = stored bands everywhere. */
typedef struct {
  int levels, smoother, nu, mu, outer, precision, max_iter;
  double tau, delta;
  size_t hbm_budget;
  void* stream;
  int gs_cluster;
  int autotune;
  int matrix_free;
} mgiga_options;

/* Fill `opts` with: levels 0, SCMS, nu 1, mu 1, PCG, FP64, max_iter 1000,
 * tau 1, delta 0.12, no budget, default stream, automatic cluster size, no
 * autotuning, stored bands. */
void mgiga_default_options(mgiga_options* opts);

/* Validate the problem, build the DoF numbering, the piece decomposition and
 * the Gauss-Seidel colouring of every level (host only, no device work).
 * On success *out owns a copy of everything it needs.  On failure *out is
 * still set (unless out is NULL) so that mgiga_last_error() can be read; it
 * must be released with mgiga_destroy(). */
mgiga_status mgiga_create(const mgiga_problem* problem, const mgiga_options* opts,
                          mgiga_handle** out);

/* Assemble the finest-level matrix (Sec. 2 Eq. linear:system:0, Sec. 3
 * Eq. linear:system), the Galerkin coarse matrices A_{l-1} = P^T A_l P
 * (Sec. 4: I_l^{l-1} is the transpose of the canonical embedding), the
 * smoother data (Sec. 5: interior eigenbases, interface-piece factors;
 * Sec. 4: colouring) and the coarse factor, then upload them to the device. */
mgiga_status mgiga_assemble(mgiga_handle* h);

/* Load vector rhs_out[g] = (f, phi_g)_{L2(Omega)} on the finest level, g in
 * global DoF order, by Gauss quadrature with p + 1 points per element and
 * direction.  f(x, ctx) is called with physical points x[dim]. */
mgiga_status mgiga_load(mgiga_handle* h, double (*f)(const double* x, void* ctx), void* ctx,
                        double* rhs_out);

/* Built-in source: f(x) = dim pi^2 prod_a sin(pi x_a) (= -Laplace of
 * prod sin(pi x_a), the manufactured solution of Sec. 2).  ctx: const int*
 * pointing to dim. */
double mgiga_source_sinprod(const double* x, void* ctx);

/* z = B r: one cycle (Algorithm 1 or 2 per the smoother option) on the finest
 * level with zero initial guess -- the preconditioner of PCG (Sec. 4).
 * r, z: ndof doubles in global order. */
mgiga_status mgiga_vcycle(mgiga_handle* h, const double* r, double* z);
mgiga_status mgiga_vcycle_d(mgiga_handle* h, const double* r, double* z);

/* Solve A u = rhs to ||A u - rhs||_2 / ||rhs||_2 <= tol (the stopping rule of
 * Sec. 4) with PCG (outer = PCG) or the V-cycle as solver (outer = DIRECT).
 * u: initial guess on entry, solution on exit.  iters / final_relres may be
 * NULL.  Returns MGIGA_ENOCONV with the last iterate in u when max_iter
 * outer iterations do not suffice (max_iter = k yields the k-th iterate), and
 * MGIGA_EBREAKDOWN when rhs or the initial guess holds NaN/Inf or CG breaks
 * down (p^T A p <= 0, non-finite residual); a zero rhs gives u = 0. */
mgiga_status mgiga_solve(mgiga_handle* h, const double* rhs, double* u, double tol,
                         int* iters, double* final_relres);
mgiga_status mgiga_solve_d(mgiga_handle* h, const double* rhs, double* u, double tol,
                           int* iters, double* final_relres);

/* Batched solves (many independent problems of uneven sizes, Sec. 4 PCG each): n distinct handles,
 * rhs[i] / u[i] device vectors of handle i as in mgiga_solve_d (u[i]: initial guess in, solution
 * out), one tolerance.  With the outer PCG iteration every solve runs as one graph with conditional
 * nodes (no host round trip per iteration): all n are enqueued from the calling thread, on their
 * handles' streams, before any is awaited; with MGIGA_BATCH_ONE_GRAPH the n solve graphs are the
 * branches of a single graph launched once (rebuilt when the handles, vectors or tolerance change;
 * without that support, or for handles with the direct outer iteration, the solves run as without
 * the flag).  iters, final_relres, status (n entries each, may be NULL) receive each problem's
 * results.  Returns MGIGA_OK when every solve converged, else the first failing status.  The
 * handles must not be in use by other threads during the call. */
enum { MGIGA_BATCH_ONE_GRAPH = 1 };
mgiga_status mgiga_solve_batch_d(mgiga_handle* const* hs, int n, const double* const* rhs, double* const* u,
                                 double tol, int flags, int* iters, double* final_relres, int* status);

/* Single stages of the cycle on level `level` (0 = coarsest), for testing and
 * profiling.  Vectors are in the global DoF order of the level they live on.
 *   MGIGA_OP_RESIDUAL   out = a - A_l b                 (a = f, b = u)
 *   MGIGA_OP_MATVEC     out = A_l a
 *   MGIGA_OP_SMOOTH     out = b + tau sum_T P_T L_T^{-1} P_T^T (a - A_l b)  (Eq. Ldef)
 *   MGIGA_OP_GS_FWD     out = b + L^{-1}(a - A_l b)      (forward multicolour sweep)
 *   MGIGA_OP_GS_BWD     out = b + L^{-T}(a - A_l b)      (backward sweep)
 *   MGIGA_OP_RESTRICT   out = P_l^T a   (out on level l-1)
 *   MGIGA_OP_PROLONG    out = P_l a     (a on level l-1, out on level l)
 *   MGIGA_OP_COARSE     out = A_0^{-1} a  (level must be 0)
 *   MGIGA_OP_CYCLE_RESIDUAL  out = a - A_l b as the V-cycle computes it on
 *                       level >= 1: with the FP32 band coefficients and FP32
 *                       arithmetic (FP64 result) unless the precision is FP64;
 *                       the error is bounded by FP32 rounding of the band sum */
enum {
  MGIGA_OP_RESIDUAL = 0, MGIGA_OP_MATVEC = 1, MGIGA_OP_SMOOTH = 2, MGIGA_OP_GS_FWD = 3,
  MGIGA_OP_GS_BWD = 4, MGIGA_OP_RESTRICT = 5, MGIGA_OP_PROLONG = 6, MGIGA_OP_COARSE = 7,
  MGIGA_OP_CYCLE_RESIDUAL = 8
};
mgiga_status mgiga_apply(mgiga_handle* h, int op, int level, const double* a, const double* b,
                         double* out);
mgiga_status mgiga_apply_d(mgiga_handle* h, int op, int level, const double* a, const double* b,
                           double* out);

/* Allocation-free residual.  The paper has no counterpart: this is a service
 * of the library for callers that must not allocate device memory while they
 * run, for example a request loop that works inside a fixed HBM budget it has
 * already reserved, or code that cannot afford the device-wide
 * synchronisation that cudaMalloc and cudaFree may cause.  Such a caller
 * creates and assembles its handle up front (mgiga_assemble allocates) and
 * then calls this entry point as often as it likes.
 *   out = f - A_l u on `level`, exactly what mgiga_apply_d(h,
 *   MGIGA_OP_RESIDUAL, level, f, u, out) computes: f, u, out are device
 *   pointers to ndof(level) doubles in global order; inputs are only read.
 * Its scratch (local-layout copies of f and u with zero guards, and the
 * residual before it is gathered) lives in one fixed device array of
 * MGIGA_NOALLOC_SCRATCH_DOUBLES doubles (24 MiB) that every GPU loading the
 * library holds until the process exits; the call uses no cudaMalloc,
 * cudaFree or other allocating routine and does not touch the handle's own
 * level buffers.  A level needing more scratch than that (about 1M local
 * coefficients) is rejected with MGIGA_EINVAL and a message giving both sizes.
 * The call must run with the handle's device (the one current at
 * mgiga_assemble) current, else it returns MGIGA_EINVAL.  The first call on a
 * device looks up the array's device address on that device; make that first
 * call before any stream capture.  All calls share
 * the array and it keeps the last call's contents: the zero guards are
 * cleared on every call.  Calls whose work overlaps on the GPU (other
 * streams, other handles, other threads) race on the array; serialise them.
 * Runs on the handle's stream and returns when `out` is ready. */
#define MGIGA_NOALLOC_SCRATCH_DOUBLES 3145728
mgiga_status mgiga_residual_noalloc_d(mgiga_handle* h, int level, const double* f, const double* u,
                                      double* out);

/* Profiling.  mgiga_kernel_launches: kernels this handle has enqueued so far
 * (kernels replayed by a CUDA graph count once per replay).
 * mgiga_time_stage: average device time in milliseconds of one application of
 * a stage on `level`, measured with CUDA events on the handle's stream over
 * `reps` back-to-back applications after one warm-up, on the handle's own
 * device buffers (their contents are overwritten).
 * mgiga_stage_work: algorithmic flops and HBM bytes of one application
 * (BAND: 2 nnz(A_l) flops, 8 nnz(A_l) + 24 N_l bytes; FD: 4 d n per interior
 * DoF flops, 24 bytes per interior DoF; GS: as BAND, with 4 bytes per nonzero
 * when the smoothers run in FP32 (precision other than FP64); RESIDUAL: as
 * BAND, 4 bytes per nonzero on the mixed path); MGIGA_ESTATE before
 * mgiga_assemble (the operators are not yet built). */
enum {
  MGIGA_STAGE_BAND = 0,     /* band product A_l u (a1) */
  MGIGA_STAGE_FD = 1,       /* interior fast diagonalisation (a2) */
  MGIGA_STAGE_PIECES = 2,   /* interface-piece solves (a3) */
  MGIGA_STAGE_GS = 3,       /* forward multicolour Gauss-Seidel sweep (a4) */
  MGIGA_STAGE_RESTRICT = 4, /* a5 */
  MGIGA_STAGE_PROLONG = 5,  /* a6 */
  MGIGA_STAGE_COARSE = 6,   /* a7 (level 0) */
  MGIGA_STAGE_VCYCLE = 7,   /* a whole cycle from `level` down */
  MGIGA_STAGE_RESIDUAL = 8  /* residual f - A u inside the cycle (level >= 1): FP32 band
                               coefficients and arithmetic unless the precision is FP64 */
};
mgiga_status mgiga_kernel_launches(const mgiga_handle* h, long long* n);

/* Relative residuals ||f - A u|| / ||f|| of the last mgiga_solve[_d] on this
 * handle: the initial one, then one per outer iteration (PCG: the recursive
 * residual, the last entry the confirming true residual; direct: the true
 * residual); a zero right-hand side gives {0}; empty before the first solve.
 * *n receives the number of entries; min(cap, *n) are written to out (out may
 * be NULL when cap is 0). */
mgiga_status mgiga_residual_history(const mgiga_handle* h, double* out, int cap, int* n);

/* Diagnostics of the bounded device waits.  Every spin-wait of the kernels
 * (grid barrier, mbarrier of an asynchronous copy) gives up after a fixed
 * number of polls (2^18 for an mbarrier, ~1 s), records the expiry in a
 * device flag and lets the launch end; the host reads the flag after the
 * stream drains and the call returns MGIGA_ETIMEOUT, the handle staying
 * usable.  This call runs one such
 * wait on a barrier phase that nothing completes, with `iterations` polls
 * (1 .. 2^18), on the handle's stream (after mgiga_assemble): it returns
 * MGIGA_ETIMEOUT with the message of a real expiry when the wait gave up,
 * and *elapsed_ms (may be NULL) receives the wait's device duration. */
mgiga_status mgiga_check_wait_expiry(mgiga_handle* h, long long iterations, double* elapsed_ms);
mgiga_status mgiga_time_stage(mgiga_handle* h, int stage, int level, int reps, double* ms);
mgiga_status mgiga_stage_work(const mgiga_handle* h, int stage, int level, double* flops, double* bytes);

/* Sizes and integer maps (host only, valid after mgiga_create). */
mgiga_status mgiga_num_levels(const mgiga_handle* h, int* levels);
mgiga_status mgiga_ndof(const mgiga_handle* h, int level, long* n);
/* owner copy of every global DoF of the level: patch[g], local[g] (flat index) */
mgiga_status mgiga_dof_map(const mgiga_handle* h, int level, int* patch, int* local_index);
/* Gauss-Seidel colour of every global DoF of level `level` (level >= 1, when
 * the smoother uses Gauss-Seidel; MGIGA_ESTATE otherwise). */
mgiga_status mgiga_colours(const mgiga_handle* h, int level, int* colour);
/* Piece decomposition of level >= 1 (Sec. 5): piece_of[g] = piece id of
 * global DoF g; pieces are the patch interiors in patch order, then the
 * interface pieces ordered by their smallest global DoF.  *num_pieces may
 * be NULL.  Available with an SCMS or hybrid smoother (else MGIGA_ESTATE). */
mgiga_status mgiga_pieces(const mgiga_handle* h, int level, int* piece_of, int* num_pieces);

/* Device footprint in bytes of the assembled handle (0 before assemble). */
mgiga_status mgiga_device_bytes(const mgiga_handle* h, size_t* bytes);

/* Text of the last error on this handle ("" if none; never NULL). */
const char* mgiga_last_error(const mgiga_handle* h);
void mgiga_destroy(mgiga_handle* h);

#ifdef __cplusplus
}
#endif
#endif /* MGIGA_H */
