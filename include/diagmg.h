/*
 * diagmg.h -- C ABI of the GPU (sm_103a) diagonally oriented multigrid
 * V-cycle for Poisson's equation, Laplacian(u) = f, with zero Dirichlet data
 * on the unit square (dim 2) or unit cube (dim 3).
 *
 * Method: A.J. Roberts, "Fast and accurate multigrid solution of Poisson's
 * equation using diagonally oriented grids".  The problem statement is Eq.
 * Epois / Eq. Evpois (Section 1); the 2D cycle is Section 2, the 3D cycle
 * Section 3; the conventional 2^-l cycle the paper compares against is
 * described alongside (Sections 2.1, 2.2, 3.1, 3.2).
 *
 * Conventions shared by every call
 *   - Grids.  n = 2^m - 1 interior points per side, h = 1/(n+1).  A caller
 *     array is the full grid of (n+2)^dim doubles including the Dirichlet
 *     ring, x fastest: element (i,j) at [j*pitch + i], (i,j,k) at
 *     [(k*(n+2) + j)*pitch + i], 0 <= i,j,k <= n+1, pitch >= n+2 elements.
 *   - Memory.  Every array pointer is caller-owned DEVICE memory on the
 *     context's device unless the parameter says "host".  A grid pointer
 *     (f, u, r, a level grid) must be 8-byte aligned (an FP64 element
 *     boundary); a null or misaligned one gives MG_EINVAL.  The library never
 *     keeps a caller pointer after a call returns.  All workspace (level
 *     buffers, norms, control words) is allocated by mg_create and freed by
 *     mg_destroy; no other call allocates device memory, except the first
 *     mg_solve_host of a context (its device copies of f and u) and the
 *     first mg_set_gamma with gamma > 1 (its coarse-level work arrays).
 *   - Streams.  `stream` is a cudaStream_t passed as void* (NULL = the legacy
 *     default stream).  Calls are stream-ordered; a call that returns a value
 *     to a host pointer synchronises that stream before returning.
 *   - Boundary.  The ring of u must be zero (homogeneous Dirichlet data, the
 *     only case the paper treats).  The ring of f is read only by the
 *     fourth-order residuals (Eq. Efos2, Eq. Efos4), which reach it.
 *   - Errors.  Every call returns an mg_status; MG_EINVAL for a bad argument
 *     (nothing is launched), MG_ECUDA for a CUDA runtime error (the context
 *     may be unusable), MG_ENOCONV / MG_EDIVERGED from the solvers.  A context
 *     is not thread-safe: one host thread at a time.
 *   - Levels.  Level 0 is the finest grid.  Diagonal hierarchy, 2D: level 2k
 *     is the axis grid of side n_k = 2^(m-k) - 1 ("green"), level 2k+1 the 45
 *     degree grid ("red", points i+j even of that axis grid).  3D: level 3k
 *     green (cubic), 3k+1 red (i+j+k even), 3k+2 magenta (corners (e,e,e) and
 *     centres (o,o,o)).  Conventional hierarchy: level k is the axis grid of
 *     side n_k.  The coarsest level is the axis grid of side `coarsest`.
 */
#ifndef DIAGMG_H
#define DIAGMG_H

#ifdef __cplusplus
extern "C" {
#endif

typedef struct mg_ctx mg_ctx;

typedef enum {
    MG_OK = 0,
    MG_EINVAL = -1,     /* invalid argument; nothing was launched */
    MG_ENOMEM = -2,     /* device allocation failed in mg_create */
    MG_ECUDA = -3,      /* CUDA runtime error (message: mg_last_error) */
    MG_ENOCONV = -4,    /* max_cycles reached above rtol */
    MG_EDIVERGED = -5,  /* residual became non-finite or grew 1e3-fold */
    MG_ETIMEOUT = -6    /* reserved: no call returns it (no kernel waits on another block) */
} mg_status;

enum { MG_DIAG = 0, MG_USUAL = 1 };   /* hierarchy */
enum { MG_FP64 = 0, MG_MIXED = 1 };   /* precision of the level arithmetic */

/* Context description.
 *   dim        2 or 3
 *   n          interior points per side, 2^m - 1 with m >= 2
 *   pitch      elements per row of the caller's full-grid arrays, >= n+2
 *   hierarchy  MG_DIAG (Sections 2, 3) or MG_USUAL (the conventional cycle)
 *   order      2 (5/7-point residual) or 4 (Eq. Efos2 / Eq. Efos4)
 *   precision  MG_FP64: every level in FP64.  MG_MIXED: residual on the
 *              finest grid and the update u += v in FP64, all levels and
 *              sweeps in FP32, coarsest solve in FP64 (iterative refinement
 *              with one FP32 V-cycle per FP64 residual).  The residual norms
 *              square FP32 values, so MG_MIXED wants residual and right-hand
 *              side values between about 1e-18 and 1e18 in magnitude.
 *   coarsest   interior side of the coarsest axis grid: 1, 3 or 7, <= n.  It is
 *              solved exactly.  In 3D a 7^3 coarsest grid (the grid under
 *              which the paper's 17^3 convergence factors of the diagonal
 *              cycle are reproduced) runs every level with the per-stage
 *              kernels and a dense inverse in global memory, and its mixed
 *              solves take a direct residual every cycle.
 *   omega      over-relaxation weights multiplying the residual term of the
 *              Jacobi sweeps.  2D: {p} (Eq. Eajacr, Eq. Eajacb); 3D diagonal:
 *              {p_m, p_r1, p_r2, p_g} (Eq. Emprolm .. Eq. Egprolr);
 *              conventional: {p} (2D) or {p_g} (3D).  Unused entries ignored. */
typedef struct {
    int dim;
    int n;
    int pitch;
    int hierarchy;
    int order;
    int precision;
    int coarsest;
    double omega[4];
} mg_desc;

/* Create a context on the current CUDA device and allocate all of its
 * workspace.  *out receives the context (NULL on error).  Synchronous. */
mg_status mg_create(mg_ctx **out, const mg_desc *desc);

/* Free the context and its workspace.  Synchronises the device.  NULL is a no-op. */
mg_status mg_destroy(mg_ctx *ctx);

/* Number of levels (finest 0 .. coarsest), and for one level the side of the
 * axis grid its points are indexed on (n_k) and its kind: 0 green/axis,
 * 1 red (45 degree / FCC), 2 magenta (BCC).  Host-only; no device work. */
mg_status mg_num_levels(const mg_ctx *ctx, int *num_levels);
mg_status mg_level_info(const mg_ctx *ctx, int level, int *side, int *kind);

/* Residual on the finest grid (Eq. Evpois): r = f - L_h u with the 5/7-point
 * Laplacian (order 2), or the compact fourth-order forms Eq. Efos2 (2D) /
 * Eq. Efos4 (3D) (order 4).  h must equal 1/(n+1).  The result is stored in
 * the context as the level-0 residual (in the context's level precision) and,
 * when r is not NULL, also written in FP64 to r (caller pitch, interior points
 * only; r's extent must not overlap f's or u's, else MG_EINVAL).  norm2
 * (host, nullable) receives sum(r^2) over interior points; the call then
 * synchronises `stream`. */
mg_status mg_residual(mg_ctx *ctx, const double *f, const double *u, double h, int order, double *r,
                      double *norm2, void *stream);

/* One restriction stage on the context's level buffers: r^(level+1) from
 * r^(level).  Diagonal 2D: Eq. Erest2r (green -> red) or Eq. Erest2b (red ->
 * blue).  Diagonal 3D: Eq. Erred, Eq. Ermagc + Eq. Ermagm, Eq. Erblu.
 * Conventional: full weighting (9 / 27 points, Sections 2.1 and 3.1).
 * 0 <= level < num_levels - 1. */
mg_status mg_restrict_diag(mg_ctx *ctx, int level, void *stream);

/* Exact solve on the coarsest level: v = L_H^-1 r with the 5/7-point operator
 * of that grid's spacing H (the paper leaves the coarsest treatment open). */
mg_status mg_coarse_solve(mg_ctx *ctx, void *stream);

/* One prolongation stage: v^(level) from v^(level+1) and r^(level).
 * Diagonal 2D: Eq. Eajacr then Eq. Eajacb on a red level; the analogous
 * green-red sweep on a green level (Section 2.2, weight of Section 2.4).
 * Diagonal 3D: Eq. Emprolm + Eq. Emprolb (magenta), Eq. Erprolr + Eq. Erprolm
 * (red), Eq. Egprolg + Eq. Egprolr (green).  Conventional: bilinear /
 * trilinear interpolation then one red-black ordered Jacobi iteration with
 * residual weight p (Sections 2.2, 3.2).  omega (host, nullable) overrides
 * the context's weights for this call.  0 <= level < num_levels - 1. */
mg_status mg_jacobi_prolong(mg_ctx *ctx, int level, const double *omega, void *stream);

/* Copy a level buffer between the context and a caller full grid of side
 * n_k (mg_level_info), pitch n_k+2, indexed with that grid's subscripts as
 * the paper does.  which: 0 = residual r, 1 = correction v.  Only the
 * interior points of the level are read or written; other entries of the
 * caller grid are left untouched (get) or ignored (set).  FP64 on the caller
 * side, converted to the level precision. */
mg_status mg_level_get(mg_ctx *ctx, int level, int which, double *grid, void *stream);
mg_status mg_level_set(mg_ctx *ctx, int level, int which, const double *grid, void *stream);

/* One V-cycle in place: r = f - L u, restriction down every level, exact
 * coarsest solve, Jacobi prolongation up every level, u += v (Sections 2.3,
 * 3.3).  u: in/out (caller pitch, zero ring). */
mg_status mg_vcycle(mg_ctx *ctx, const double *f, double *u, void *stream);

/* V-cycles from the warm start u until ||r||_2 / ||r(u=0)||_2 <= rtol, where
 * r is the residual of the context's order, or until max_cycles cycles.  The
 * convergence test runs on the device; the host waits once at the end.  The
 * whole solve is one CUDA graph launch; the context keeps the graphs of its
 * four most recent argument sets (f, u, rtol, max_cycles, with its weights,
 * order and sweeps), so alternating between a few buffers does not rebuild
 * them (set DIAGMG_SOLVE_GRAPH=0 for a host-driven loop of the same kernels).
 * Single 2D problems launch their kernels with programmatic dependent
 * launch (in FP64, only the grids of at most 256 blocks), so that a kernel's
 * launch overlaps the tail of the one before.  DIAGMG_PDL=1 or 0 and
 * DIAGMG_PDL_MAX_BLOCKS=<blocks> (0: no limit), read at mg_create, override
 * that for any context.  The results are the same bit for bit.
 * DIAGMG_CLUSTER=1, read at mg_create, runs the 2D pairs whose green side
 * lies between 63 and 255 (127 with FP64 levels) and everything coarser in
 * one launch of a thread-block cluster of 8 blocks that keeps those levels in
 * distributed shared memory (the finest pair of a mixed solve stays outside
 * it), instead of the per-pair kernels and the single coarse thread block
 * (same arithmetic, term for term).  It is off by default: on GB300 it
 * measured slower; mg_tune tries both.
 *   cycles_out  (host, nullable) cycles applied
 *   relres_out  (host, nullable) final relative residual
 *   history     (host, nullable, length max_cycles) relative residual after
 *               each cycle
 * Returns MG_OK, MG_ENOCONV or MG_EDIVERGED (u holds the last iterate). */
mg_status mg_solve(mg_ctx *ctx, const double *f, double *u, double rtol, int max_cycles, int *cycles_out,
                   double *relres_out, double *history, void *stream);

/* mg_solve from u = 0: the same V-cycles (Sections 2.3, 3.3), but u (device,
 * full grid, caller layout) is output only -- its contents on entry are never
 * read, and it need not be zeroed.  On return it holds the same iterate, bit
 * for bit, as mg_solve from a zeroed u.  The call zeroes u's (n+2)^d points
 * itself (a 2D memset on `stream` that leaves the padding of a larger pitch
 * alone; inside the solve's graph on the fused mixed path, whose start
 * residual then is f itself and reads no u), which saves the caller's fill
 * and one read of u per solve.  u must not overlap f (MG_EINVAL).  Arguments
 * and returns as mg_solve; the graph cache keys a solve from zero apart from
 * a warm start on the same arrays. */
mg_status mg_solve_zero(mg_ctx *ctx, const double *f, double *u, double rtol, int max_cycles, int *cycles_out,
                        double *relres_out, double *history, void *stream);

/* mg_solve with HOST arrays, for callers whose data live in host memory:
 * f_host (the right-hand side), u0_host (the warm start, zero ring; NULL:
 * start from u = 0) and u_host (receives the result; may equal u0_host) are
 * full grids in the caller layout (pitch; only their (n+2)^d points are read
 * or written, never the padding of a larger pitch).  The call copies f and the warm
 * start to device copies owned by the context, runs mg_solve there (mg_solve_zero
 * when u0_host is NULL) and copies
 * u back, and returns once u_host holds the result.  The copy in runs on
 * `stream`; on the fused mixed path the copy back starts as soon as the last
 * cycle has written u (an event the solve's graph records) and runs on a
 * stream of the context beside the direct residual that closes the solve,
 * otherwise it follows the solve on `stream`.  For full copy bandwidth the
 * host arrays should be page-locked (cudaHostAlloc / cudaHostRegister).  The
 * first call allocates the two device copies and creates that stream
 * (MG_ENOMEM / MG_ECUDA if that fails); later calls allocate nothing.  Single-problem contexts only; u_host must not overlap
 * f_host.  Returns what mg_solve returns. */
mg_status mg_solve_host(mg_ctx *ctx, const double *f_host, const double *u0_host, double *u_host, double rtol,
                        int max_cycles, int *cycles_out, double *relres_out, void *stream);

/* mg_solve_host for a sequence of `count` problems of the context's size, each
 * solved from u = 0 (as mg_solve_zero): f_host[k] (host, full grid, caller
 * layout) in, u_host[k] out; no u_host may overlap any f_host (MG_EINVAL),
 * and outputs that share a buffer are written in the order of k.  The call
 * pipelines
 * the problems over two pairs of device copies: the copy in of problem k + 1
 * and the copy back of problem k run on a stream of the context while problem
 * k is solved on `stream`, so the host link and the solve overlap; every
 * result is the one mg_solve_host gives for that problem alone, bit for bit.
 * cycles_out, relres_out: host arrays of count entries (nullable).  Returns
 * MG_EDIVERGED if any problem diverged, else MG_ENOCONV if any did not
 * converge, else MG_OK (the per-problem outcome is in relres_out); returns
 * once every u_host[k] holds its result, and on an error only after every
 * copy it issued has finished.  The first call allocates a second
 * pair of device copies (MG_ENOMEM) and two page-locked control words; with
 * DIAGMG_SOLVE_GRAPH=0 the problems run one after the other. */
mg_status mg_solve_host_many(mg_ctx *ctx, int count, const double *const *f_host, double *const *u_host,
                             double rtol, int max_cycles, int *cycles_out, double *relres_out, void *stream);

/* Replace the context's over-relaxation weights (same meaning as
 * mg_desc.omega, host, 4 entries). */
mg_status mg_set_omega(mg_ctx *ctx, const double *omega);

/* Extra Jacobi sweeps at each level of the 2D diagonal hierarchy, the
 * extension the paper's conclusion (Section 5) leaves open: after a level's
 * prolongation (its two half-sweeps from the coarser values), `extra` more
 * sweeps repeat both half-sweeps from the level's own current values, with
 * the level's coefficients (red level 2 p h^2: not-blue points from their
 * four diagonal neighbours, then blue points; green level p h^2: green-only
 * points from their four axis neighbours, then red points).  0 (the default)
 * is the paper's cycle.  extra > 0 runs every level with per-stage kernels
 * (no fused pair kernels, no carried mixed residual) and applies to
 * mg_vcycle, mg_solve and mg_rho.  MG_EINVAL unless 0 <= extra <= 64 and,
 * for extra > 0, the context is a single 2D diagonal problem. */
mg_status mg_set_sweeps(mg_ctx *ctx, int extra);

/* Gamma-cycles (W-cycles for gamma = 2) of the 2D diagonal hierarchy, the
 * other extension the paper's conclusion (Section 5) leaves open.  In the
 * cycle of each pair the coarse problem on its blue grid -- the next pair's
 * green grid, an axis grid with the 5-point Laplacian at its spacing -- is
 * approximated by `gamma` cycles of the next pair from a zero correction,
 * each after the first on the residual of the corrections accumulated so far
 * (the coarsest grid is solved exactly).  gamma = 1 (the default) is the
 * paper's V-cycle.  gamma > 1 runs every level with per-stage kernels
 * (combined with mg_set_sweeps if set) and applies to mg_vcycle, mg_solve and
 * mg_rho; the number of visits of a level grows as gamma^depth.  The first
 * call with gamma > 1 allocates, per green level below the finest, a kept
 * residual and an accumulator (MG_ENOMEM if that fails).  MG_EINVAL unless
 * 1 <= gamma <= 4 and, for gamma > 1, the context is a single 2D diagonal
 * problem. */
mg_status mg_set_gamma(mg_ctx *ctx, int gamma);

/* Convergence factor of the context's V-cycle (the paper's rho, Tables 1-3:
 * the slowest decay of the error) by power iteration on its error
 * propagation: with f = 0 every V-cycle maps the error u to u + B(-L u); u is
 * renormalised after each cycle and rho_out (host) is the geometric mean of
 * the norm ratios of cycles skip..cycles-1.  zero_f: caller device array of
 * zeros (full grid, caller pitch; order 4 reads its ring too); u: caller
 * device array holding the start vector (zero ring), overwritten.
 * 2 <= cycles <= 4096, 0 <= skip < cycles.  Synchronous. */
mg_status mg_rho(mg_ctx *ctx, const double *zero_f, double *u, int cycles, int skip, double *rho_out,
                 void *stream);

/* Two-stage fourth-order solve (Section 2.4, and Section 3.4 for 3D: the
 * fourth-order solution is best reached by first converging with second-order
 * residuals, then refining with a few fourth-order V-cycles).  ctx must have
 * order 4.  Stage 1 runs the context's V-cycle on the second-order residual
 * r = f - L_h u with weights omega2 (host, 4 entries; NULL: the context's)
 * until its relative residual <= rtol2 (or max_cycles); stage 2 continues from
 * that u with the fourth-order residual (Eq. Efos2 / Eq. Efos4) and the
 * context's weights until ||f~ - L u|| / ||f~|| <= rtol.  Cycle counts of the
 * stages (host, nullable) and the final fourth-order relative residual. */
mg_status mg_solve_two_stage(mg_ctx *ctx, const double *f, double *u, const double *omega2, double rtol2,
                             double rtol, int max_cycles, int *cycles2_out, int *cycles4_out, double *relres_out,
                             void *stream);

/* Batches of independent problems (no paper counterpart: the paper solves
 * one problem at a time).  A batch holds nprob 2D or 3D problems of sides
 * n[0..nprob) (each 2^m - 1), all with the same hierarchy, order (2 only),
 * precision, coarsest side and omega[4] (host).  Problems of equal side are
 * grouped; every kernel of a group processes all of its problems in one
 * launch (grid z = problem), and one CUDA graph holds a device-driven loop
 * per group as parallel branches, so a batched solve is a single graph
 * launch.  Each problem stops on its own convergence test; a group's loop
 * ends when all of its problems are done.  mg_batch_create allocates all
 * workspace (synchronous).
 *   f, u        host arrays of nprob DEVICE pointers; problem p's full grid,
 *               pitch n[p]+2, zero ring of u; u is the warm start, in/out
 *   cycles_out  host, nullable, nprob entries; relres_out likewise
 * Returns MG_OK, MG_ENOCONV or MG_EDIVERGED if any problem did not converge
 * or diverged (the per-problem outputs say which), MG_EINVAL, MG_ECUDA.
 * max_cycles <= 256.  The graph is rebuilt when f, u, rtol or max_cycles
 * differ from the previous call. */
typedef struct mg_batch mg_batch;
mg_status mg_batch_create(mg_batch **out, int dim, int nprob, const int *n, int hierarchy, int order,
                          int precision, int coarsest, const double *omega);
mg_status mg_batch_destroy(mg_batch *batch);
mg_status mg_solve_batched(mg_batch *batch, const double *const *f, double *const *u, double rtol, int max_cycles,
                           int *cycles_out, double *relres_out, void *stream);
mg_status mg_batch_launch_count(const mg_batch *batch, long long *launches);
/* Per-problem outcome of the batch's last mg_solve_batched: status[p] (host,
 * nprob entries) is MG_OK, MG_ENOCONV (max_cycles reached above rtol) or
 * MG_EDIVERGED (its residual became non-finite, grew 1e3-fold, or its
 * right-hand side carried a NaN).  MG_EINVAL before the first solve. */
mg_status mg_batch_status(const mg_batch *batch, int *status);

/* Autotuning (no paper counterpart).  mg_tune times, on this context's own
 * buffers with the caller's f and u, the size cut-off below which whole
 * pairs/triples run in one thread block and, in 2D, whether the middle pairs
 * run in the thread-block cluster (whole V-cycles for each candidate; a
 * candidate whose launch fails is never chosen), then the tile shape of every
 * pair kernel outside them (each kernel alone, three shapes), and keeps the
 * fastest.  The choice is appended to the cache file
 * `cache_path` (NULL: the file named by the environment variable
 * DIAGMG_TUNE_CACHE; neither: no file) as one JSON object per line keyed by
 * device name, dim, n, hierarchy, precision and batch size; a later mg_tune
 * with a matching entry applies it without measuring.  u is scratch and is
 * left zero (interior and ring).  measured_out (host, nullable): 1 if timed,
 * 0 if taken from the cache or nothing is tunable.  Synchronous.
 * mg_tune_info reports the cut-off (0 = default) and the tile class of each
 * pair kernel outside the thread block and the cluster, npairs of them (FP64
 * levels: tiles of 0: 32x16 cells, 1: 16x8, 2: 8x8; FP32 levels: streaming
 * kernels with strips of 0: 32, 1: 16, 2: 8 cell rows for the prolongation
 * and 16, 8, 4 for the restriction, 3-5: the tiles of 0-2);
 * tiles_down / tiles_up need 32 entries.  mg_batch_tune does the same for
 * every size group of a batch (f, u as in mg_solve_batched).
 * Untuned contexts take defaults fitted to the tuner's choices on GB300 from
 * 255^2 to 4095^2 (within 2% of them there): the coarse thread block takes
 * pairs of green side <= 63 (FP64: 15) and triples <= 15 (FP64: 7); the
 * fused finest pair of the mixed path the longest strips that still fill the
 * device with warps (for a single problem with 2-12 warps' worth of strips
 * per SM it loads u and the residual's low part straight into registers),
 * the coarser FP32 pairs streaming kernels from 512 cells
 * and tiles below, FP64 pairs 16x8 tiles from 256 cells; a context of
 * several problems (a batch's size group) the largest FP64 tiles or the
 * FP32 streaming kernels at every level. */
mg_status mg_tune(mg_ctx *ctx, const double *f, double *u, const char *cache_path, int *measured_out,
                  void *stream);
mg_status mg_tune_info(const mg_ctx *ctx, int *cut_side, int *npairs, int *tiles_down, int *tiles_up);
mg_status mg_batch_tune(mg_batch *batch, const double *const *f, double *const *u, const char *cache_path,
                        void *stream);

/* Diagnostics (no paper counterpart).  mg_launch_count: kernels this context
 * has launched since creation (host counter).  mg_probe_set: when family >= 0,
 * every later launch of that kernel family is bracketed with CUDA events on
 * its stream (family 0: finest-grid residual / down pass, 1: finest-grid
 * prolongation and update, 2: all other level stages, 3: control kernels;
 * 4, 5, 6: the parts of family 2 -- restriction, prolongation of the coarser
 * levels, the coarse thread block; -1 turns the probe off).  mg_probe_read synchronises `stream` and returns
 * the probed launches and their summed device time in ms since the last
 * mg_probe_set.  Event objects are created by the first mg_probe_set. */
mg_status mg_launch_count(const mg_ctx *ctx, long long *launches);
mg_status mg_probe_set(mg_ctx *ctx, int family);
mg_status mg_probe_read(mg_ctx *ctx, long long *launches, double *ms, void *stream);
/* Measured FP64 pipe rate of this device (the roofline of the FP64 path's
 * arithmetic): a kernel of independent FP64 FMA chains on every SM, timed with
 * CUDA events on `stream`, best of three launches after a warm-up; *ops_per_s
 * (host) counts one FMA as one operation.  Synchronous. */
mg_status mg_fp64_rate(mg_ctx *ctx, double *ops_per_s, void *stream);

/* Residual and squared norm without any device allocation (the paper has no
 * counterpart; this serves callers that may not allocate device memory: code
 * inside another framework's allocator or fixed memory budget, latency-bound
 * loops where cudaMalloc/cudaFree could stall the device, plug-ins that keep
 * no workspace between calls).  No context is needed.
 *   r = f - L_h u exactly as mg_residual computes it for the same order (the
 *   5/7-point Laplacian, or with order 4 the compact fourth-order 9-point
 *   (2D) / 19-point (3D) forms that mg_residual uses); h must be 1/(n+1).
 *   f, u      caller device arrays, full grid (n+2)^dim, row pitch `pitch`
 *   r         caller device array (same layout) receiving r on the interior
 *             points, or NULL; its extent must not overlap f's or u's
 *             (MG_EINVAL)
 *   norm2     caller DEVICE pointer to one double receiving sum(r^2) over the
 *             interior, or NULL; written in stream order (no host sync)
 * Scratch: one partial sum per 256-thread block lives in a static device
 * array of 65536 doubles (512 KiB, resident on every GPU that loads this
 * library until the process exits).  Sizes needing more -- 2D n > 4095, 3D
 * n > 255 -- are rejected with MG_EINVAL before anything is launched, as are
 * other invalid arguments.  Every call overwrites the partial sums it uses
 * before reading them, so no state carries over between calls; but all calls
 * on one device share the array, so calls that may overlap on the GPU (other
 * streams, other host threads) race and must be serialised by the caller.
 * The first call on each device looks up the array's device address (with
 * that device current) and keeps it for the life of the process; make that
 * first call before any stream capture, and do not reset the device
 * (cudaDeviceReset) after it.  Allocates nothing: no cudaMalloc, cudaFree or allocating library
 * routine is called. */
mg_status mg_residual_noalloc(int dim, int n, int pitch, double h, int order, const double *f, const double *u,
                              double *r, double *norm2, void *stream);

/* Message for a status, and the last CUDA error text of this process. */
const char *mg_strerror(mg_status status);
const char *mg_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* DIAGMG_H */
