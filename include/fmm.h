/*
 * fmm.h -- C-ABI of libfmm: the 3D Laplace (1/r) fast multipole mat-vec on
 * one GB300 (sm_103a), and its Helmholtz (e^{i kappa r}/r) counterpart.
 *
 * Method (Yokota, Ibeid & Keyes, "Fast Multipole Method as a Matrix-Free
 * Hierarchical Low-Rank Approximation"): the analytic FMM is a matrix-free
 * H^2-matrix-vector product (§1, §2.4).  The paper separates the
 * precalculation (hierarchy) from the application of the mat-vec (§4.1) and
 * asks for a common interface between the hierarchical structure and the
 * inner kernels (§5); this header mirrors that split:
 *   fmm_plan_create  -- hierarchy: root cube, Morton keys (§3.1), radix sort,
 *                       adaptive octree, interaction lists (§2.2).
 *   fmm_eval         -- mat-vec: P2M, M2M, per-level M2L (§2.2: the dominant
 *                       translation), P2L, L2L, L2P, M2P and the near-field
 *                       direct sum (the dense diagonal blocks, §2.2).
 *   fmm_adjoint      -- the transpose mat-vec and the coordinate gradient.
 *   fmm_helmholtz_eval -- the same hierarchy with the Helmholtz kernel
 *                       e^{i kappa r}/r (the paper's second kernel, §1, §4.2).
 *
 * Computed quantities (no 1/(4 pi) factor):
 *   phi_i  = sum_{j != i} q_j / |x_i - x_j|
 *   grad_i = grad phi(x_i) = -sum_{j != i} q_j (x_i - x_j) / |x_i - x_j|^3
 * Pairs at zero distance contribute nothing.
 *
 * Conventions for every entry point:
 *   - Pointers named d_* are DEVICE pointers on the current CUDA device;
 *     h_* are host pointers.  The caller owns them.  Coordinates are FP64,
 *     row-major N x 3 (x0,y0,z0,x1,...); gradients likewise.  Outputs are in
 *     the caller's input order.
 *   - `stream` is a cudaStream_t passed as void* (NULL = legacy default).
 *     Work is stream-ordered and asynchronous unless stated otherwise.
 *   - Every function returns an fmm_status; nothing throws across the ABI.
 *     fmm_last_error_message() describes the last failure of this thread.
 *   - A plan is not thread-safe; distinct plans are independent.
 */
#ifndef FMM_H
#define FMM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct fmm_plan_s *fmm_plan_t; /* opaque; owned by the library */

typedef enum {
  FMM_OK = 0,
  FMM_ERR_INVALID_ARG = 1,     /* bad size, order, leaf size or NULL pointer  */
  FMM_ERR_CUDA = 2,            /* a CUDA runtime call failed                  */
  FMM_ERR_OOM = 3,             /* device allocation failed                    */
  FMM_ERR_TIMEOUT = 4,         /* a bounded device-side wait gave up          */
  FMM_ERR_NONFINITE_INPUT = 5, /* a coordinate is NaN or infinite             */
  FMM_ERR_UNSUPPORTED = 6      /* valid request the library does not provide  */
} fmm_status;

typedef enum {
  FMM_FP64 = 0,  /* every pass in FP64                                        */
  FMM_MIXED = 1  /* P2M/M2L/L2P/M2P/P2L/P2P in FP32 with FP32 accumulation;
                    M2M/L2L at the coarsest levels and the per-target
                    reduction in FP64                                         */
} fmm_precision;

/* Options; a zero-initialised struct gives the defaults. */
typedef struct {
  int precision;          /* fmm_precision (default FMM_FP64)                 */
  int coarse_fp64_levels; /* MIXED: M2M/L2L into levels <= this run in FP64;
                             0 = default (3), negative = none                 */
  int max_depth;          /* deepest level, 1..21; 0 = default (21)           */
  int m2l_path;           /* MIXED, order <= 10: 0 = default (tensor cores),
                             1 = FP32 CUDA cores, 2 = tensor cores (tcgen05,
                             three-product TF32 split);
                             3 = rotated operators, either precision, order
                             <= 12: rotate each multipole onto the offset
                             axis, translate along it, rotate back
                             (O(p^3) per pair instead of O(p^4)).
                             FP64, order <= 12: the default is 3 (0 and 3
                             both select it; 1 and 2 the dense operator)      */
  int interaction;        /* how boxes are paired (§2.1):
                             0 = U/V/W/X lists of the adaptive octree (default);
                             1 = dual-tree walk with the multipole acceptance
                                 criterion r_T + r_S < mac_theta |c_T - c_S|,
                                 r_B = max |x_j - c_B| over the box's points
                                 (Dehnen): M2L between cells of any sizes,
                                 P2P between the remaining leaf pairs          */
  int p2p_tile;           /* MIXED near field: staging shape of the FP32 P2P
                             kernel, 1..4 (pairs per shared-memory buffer,
                             buffers, resident warps); 0 = the default        */
  double mac_theta;       /* interaction 1: 0 < theta < 1 (0 = default, 0.5);
                             smaller is more accurate and slower              */
  int m2l_tile;           /* MIXED, tensor-core M2L: operand form, 1 = TF32
                             hi/lo split (kind::tf32), 2 = FP16 hi/lo split
                             with power-of-two scalings (kind::f16: half the
                             operand bytes, twice the MMA rate); 0 = default */
  int wx_direct;          /* interaction 0: 1 = a W-list pair of two leaves
                             whose W leaf holds at most (order+1)^2 points
                             (no more points than its expansion has
                             coefficients) is evaluated by the direct sum in
                             both directions instead of M2P and P2L: both
                             leaves join each other's U list.  More exact and,
                             on adaptive trees, faster.  0 = the lists as
                             defined (default)                                */
} fmm_opts;

/* Build a plan for n points (d_xyz: device, n x 3 FP64).
 *   leaf_size : a box holding more than leaf_size points splits (>= 1);
 *               a leaf exceeds it only at max_depth.  0 = autotune: time
 *               plan + mat-vec on these points for leaf sizes 16..512 and
 *               keep the fastest (cached per size bucket, order and
 *               precision for the life of the process; fmm_plan_rebuild of
 *               an autotuned plan reuses the cache).
 *   order     : expansion order p = largest harmonic degree, 0..20;
 *               (p+1)^2 real coefficients per box.
 * The plan copies what it needs from d_xyz; d_xyz may be freed afterwards.
 * n == 0 gives a valid empty plan.  Synchronises `stream` (box counts per
 * level are read back to size the lists).
 * Errors: INVALID_ARG (n < 0, n >= 2^31, leaf_size < 0, order outside 0..20,
 * bad opts, NULL out/d_xyz with n > 0), NONFINITE_INPUT, OOM, CUDA. */
fmm_status fmm_plan_create(const double *d_xyz, int64_t n, int leaf_size, int order,
                           const fmm_opts *opts, void *stream, fmm_plan_t *out);

/* A batch of independent problems in one plan: problem b owns points
 * [h_offsets[b], h_offsets[b+1]) of d_xyz (host offsets, nproblems + 1
 * entries, h_offsets[0] = 0, non-decreasing).  Each problem gets its own root
 * cube and octree (a forest); problems never interact.  fmm_eval /
 * fmm_adjoint then run every pass once over all problems' boxes, and each
 * problem's results equal those of its own single plan bit for bit (same
 * leaf size, order and options).  Charges and outputs are concatenated in the
 * same order as the points.  Errors as fmm_plan_create, plus INVALID_ARG for
 * bad offsets. */
fmm_status fmm_plan_create_batch(const double *d_xyz, const int64_t *h_offsets, int nproblems,
                                 int leaf_size, int order, const fmm_opts *opts, void *stream,
                                 fmm_plan_t *out);

/* Rebuild an existing plan for new points (n may change), keeping its leaf
 * size, order and options and reusing its device memory where it fits.
 * A batch plan rebuilds only for the same total size (same offsets).
 * Same errors and synchronisation as fmm_plan_create. */
fmm_status fmm_plan_rebuild(fmm_plan_t plan, const double *d_xyz, int64_t n, void *stream);

/* Move the points to d_xyz (same n, same input order) WITHOUT rebuilding
 * the tree: box membership, centres and lists stay frozen.  Used to
 * differentiate the frozen-plan FMM by finite differences.  Asynchronous. */
fmm_status fmm_plan_set_points(fmm_plan_t plan, const double *d_xyz, void *stream);

/* phi = A~ q, grad = grad phi.  d_q: n charges; d_phi: n outputs; d_grad:
 * n x 3 or NULL (then gradients are not computed).  Asynchronous. */
fmm_status fmm_eval(fmm_plan_t plan, const double *d_q, double *d_phi, double *d_grad,
                    void *stream);

/* Helmholtz mat-vec on the plan's tree and U/V/W/X lists (the paper's second
 * kernel, §1 and §4.2):
 *   phi_i = sum_{j : x_j != x_i} q_j e^{i kappa |x_i - x_j|} / |x_i - x_j|,
 * approximated by the low-frequency FMM of order `order` (0..12) in FP64:
 * expansions in spherical Bessel/Hankel functions times spherical harmonics,
 * translation operators per level (they depend on kappa times the box side).
 * d_q, d_phi: n complex values each, interleaved (re, im) doubles, in the
 * caller's point order, device memory owned by the caller.  kappa > 0 and
 * finite.  The expansions converge when kappa times the side of a level-2
 * box is of order one or less (e.g. kappa = 7 on [-1, 1]^3); the error falls
 * with `order` as for Laplace.  A plan of precision FMM_MIXED evaluates M2L
 * in FP32 (coefficients scaled per level by powers of min(kappa a, 1), a the
 * box side) and the near field in FP32 (sincos, reciprocal square root, FP64
 * totals per staged batch), the other passes in FP64: ~1e-6 relative.
 * The first call for a (kappa, order, tree
 * depth, root cube) builds that set of operators (synchronous); later calls
 * are asynchronous on `stream`.  Errors: FMM_ERR_INVALID_ARG for a NULL plan
 * or pointer (n > 0), an order outside 0..12, kappa <= 0 or not finite, a
 * dual-tree plan or a batch plan (one problem only); FMM_ERR_OOM, FMM_ERR_CUDA. */
fmm_status fmm_helmholtz_eval(fmm_plan_t plan, double kappa, int order, const double *d_q,
                              double *d_phi, void *stream);

/* Adjoint of L = sum_i w_i phi_i with respect to q and x (frozen plan):
 *   d_dq[k]      = dL/dq_k = (A~^T w)_k = (A~ w)_k   (A~ is symmetric)
 *   d_dx[3k+a]   = dL/dx_k = w_k grad phi^q_k + q_k grad phi^w_k.
 * d_grad_q: the forward's gradient of phi^q (n x 3) or NULL, in which case
 * it is recomputed (recompute instead of store).  d_dx may be NULL (then
 * only d_dq is produced).  Asynchronous. */
fmm_status fmm_adjoint(fmm_plan_t plan, const double *d_w, const double *d_q,
                       const double *d_grad_q, double *d_dq, double *d_dx, void *stream);

/* fmm_eval, and fmm_adjoint when d_w is not NULL (d_dq, d_dx as in
 * fmm_adjoint, with d_grad as the stored forward gradient), replayed as one
 * CUDA graph.  The first call with a given set of pointers runs the work once
 * eagerly (sizing buffers, building operators), captures it on `stream`, and
 * launches the graph; later calls with the same pointers only launch the
 * graph.  `stream` must not be the legacy default stream.  A rebuild of the
 * plan drops the graph.  Asynchronous. */
fmm_status fmm_eval_graph(fmm_plan_t plan, const double *d_q, double *d_phi, double *d_grad,
                          const double *d_w, double *d_dq, double *d_dx, void *stream);

/* End-to-end call on HOST buffers: copies h_xyz (n x 3) and h_q (n) to the
 * device, rebuilds `plan` for them, evaluates, and copies phi (n) and, if
 * h_grad is not NULL, grad (n x 3) back.  Pinned host memory is fastest.
 * Returns after the results are on the host. */
fmm_status fmm_solve_host(fmm_plan_t plan, const double *h_xyz, const double *h_q, int64_t n,
                          double *h_phi, double *h_grad, void *stream);

/* The forward and adjoint step on HOST buffers: copies h_xyz (n x 3), h_q
 * (n) and the loss weights h_w (n) to the device, rebuilds `plan` for the
 * points, evaluates phi and grad phi (fmm_eval), then the adjoint of
 * L = sum_i w_i phi_i with the forward gradient stored (fmm_adjoint), and
 * copies phi (n), grad (n x 3), dL/dq (n) and dL/dx (n x 3) back.  The
 * weights' upload overlaps the tree build, and phi and grad come down while
 * the adjoint runs, on a side stream of the plan ordered by events.  All
 * pointers are required; pinned host memory is fastest.  Returns after the
 * results are on the host.  Errors as fmm_solve_host. */
fmm_status fmm_solve_adjoint_host(fmm_plan_t plan, const double *h_xyz, const double *h_q,
                                  const double *h_w, int64_t n, double *h_phi, double *h_grad,
                                  double *h_dq, double *h_dx, void *stream);

/* Plan layout, for tests and inspection.  sizes[0..9] =
 *   n, nboxes, nlevels, |U|, |V|, |W|, |X|, order, leaf_size, precision.
 * For a dual-tree plan |U| counts P2P leaf pairs and |V| M2L pairs. */
fmm_status fmm_plan_sizes(fmm_plan_t plan, int64_t sizes[10]);

/* The kernel shapes a mixed-precision plan evaluates with: the staging shape
 * of the FP32 near field (1..4, see fmm_opts.p2p_tile) and the operand form
 * of the tensor-core M2L (1 TF32, 2 FP16) -- the caller's options, else the
 * autotuner's choice (leaf_size 0), else the defaults.  Either output may be
 * NULL.  FMM_ERR_INVALID_ARG for a NULL plan. */
fmm_status fmm_plan_tiles(fmm_plan_t plan, int *p2p_tile, int *m2l_tile);

/* Copy one plan array to host memory (synchronous).  Arrays (element type,
 * length in elements):
 *   0 keys      (uint64, n)         sorted Morton keys
 *   1 perm      (int32, n)          input index of the i-th sorted point
 *   2 level_off (int32, nlevels+1)  first box of each level
 *   3 box_key   (uint64, nboxes)    Morton key of the box's anchor at its level
 *   4 box_level (int32, nboxes)
 *   5 box_first (int32, nboxes)     first sorted point
 *   6 box_count (int32, nboxes)
 *   7 box_parent(int32, nboxes)     -1 for the root
 *   8 box_child (int32, nboxes)     first child, -1 for a leaf
 *   9 box_nchild(int32, nboxes)
 *  10/11 U offsets (int32, nboxes+1) / sources (int32, |U|)
 *  12/13 V, 14/15 W, 16/17 X likewise.
 *  18 root cubes (double, 4 per problem): lo_x, lo_y, lo_z, D.
 *  19 problem offsets (int64, nproblems + 1).
 *  20 cell radii (double, nboxes; dual-tree plans only, else 0 bytes).
 * A dual-tree plan (opts.interaction 1) keeps its P2P source leaves in U (per
 * leaf) and its M2L sources in V (per box of any level, sources of any
 * level); W and X are empty.
 * Boxes are numbered by (level, key); list sources ascend by box number.
 * `bytes` must equal the array's size in bytes (INVALID_ARG otherwise). */
fmm_status fmm_plan_export(fmm_plan_t plan, int which, void *h_dst, size_t bytes);

/* Diagnostics: per-pass device time.  When enabled, the plan records CUDA
 * events on its stream around each pass of fmm_plan_create/rebuild, fmm_eval
 * and fmm_adjoint.  fmm_profile_read synchronises the plan's stream, returns
 * the milliseconds and kernel launches accumulated per pass since the last
 * read, and resets them.  Pass order: 0 keys+sort, 1 boxes, 2 lists,
 * 3 P2M, 4 M2M, 5 M2L, 6 P2L, 7 L2L, 8 L2P, 9 M2P, 10 P2P, 11 reduce. */
#define FMM_NPASS 12
fmm_status fmm_profile(fmm_plan_t plan, int enable);
fmm_status fmm_profile_read(fmm_plan_t plan, double ms[FMM_NPASS], int64_t launches[FMM_NPASS]);

/* Diagnostic of the tensor-core path: one CTA computes D[128][n] =
 * A[128][k] B[n][k]^T with tcgen05.mma (kind::tf32).  mode 1: one TF32
 * product; mode 3: the three-product TF32 split with FP32-level accuracy.
 * Device pointers, row-major FP32; n a multiple of 16 in 16..256, k a
 * multiple of 8, and the four operand halves (2*128*kp + 2*n*k floats, kp = k
 * rounded up to a multiple of 32) at most 200 KB, else FMM_ERR_INVALID_ARG.
 * Synchronous.  FMM_ERR_TIMEOUT if the bounded wait for MMA
 * completion gave up. */
fmm_status fmm_tc_selftest(int n, int k, const float *d_a, const float *d_b, float *d_d, int mode,
                           void *stream);

/* Diagnostic of the bounded device-side wait used by the tensor-core kernels:
 * one thread waits on a shared-memory mbarrier that expects one arrival.
 * arrive != 0: the thread arrives first, the wait completes, FMM_OK.
 * arrive == 0: nothing arrives; the wait gives up after limit_cycles SM
 * cycles (1..2e9), the kernel records it and returns, and the call reports
 * FMM_ERR_TIMEOUT; the device stays usable.  Synchronous. */
fmm_status fmm_wait_selftest(int arrive, long long limit_cycles, void *stream);

/* Measured FP32 rate of the current device in TFLOP/s: every SM runs
 * independent chains of paired fused multiply-adds (fma.rn.f32x2, the
 * instruction form of the FP32 near field), timed with CUDA events on
 * `stream`, the best over four launch shapes (8 or 16 chains per thread,
 * 256 or 512 threads per block) of five launches each; 2 flop per FMA.  The
 * roofline denominator of the FP32-bound passes.  Synchronous; some tens of
 * milliseconds.  FMM_ERR_INVALID_ARG for a NULL output. */
fmm_status fmm_fp32_peak(double *tflops, void *stream);

/* Measured FP64 rate of the current GPU in TFLOP/s, the same way with plain
 * FP64 fused multiply-add chains (the roofline denominator of the FP64-bound
 * Helmholtz passes).  Synchronous.  FMM_ERR_INVALID_ARG for a NULL output. */
fmm_status fmm_fp64_peak(double *tflops, void *stream);

/* Synchronise `stream`, then report FMM_ERR_TIMEOUT (once) if a bounded
 * device-side wait of this plan's kernels gave up since the last call, else
 * FMM_OK.  Results of an evaluation that timed out are not valid. */
fmm_status fmm_sync(fmm_plan_t plan, void *stream);

/* Device memory held by this library's plans on the current device: bytes
 * in use now and the high-water mark since the last reset (reset_peak != 0
 * resets it after reading).  Either output may be NULL. */
fmm_status fmm_memory_usage(uint64_t *current, uint64_t *peak, int reset_peak);

/* Brute-force reference: for m targets t (d_tgt: device, m x 3 FP64)
 *   phi(t) = sum_j q_j / |t - x_j|,  grad(t) = -sum_j q_j (t - x_j) / |t - x_j|^3
 * over the n sources x_j (d_src: device, n x 3 FP64; d_q: n), skipping pairs
 * at zero distance -- the plain definition the FMM approximates (§2, Eq. 1,
 * kernel 1/r).  FP64, O(n m) work; the sum over sources is taken in a fixed
 * order (deterministic).  d_grad (m x 3) may be NULL.  Stream-ordered and
 * asynchronous; scratch comes from the library pool.  FMM_ERR_INVALID_ARG
 * for negative sizes or NULL required pointers; non-finite inputs give
 * non-finite outputs.  n = 0 gives zeros; m = 0 is a no-op. */
fmm_status fmm_direct(const double *d_src, const double *d_q, int64_t n, const double *d_tgt,
                      int64_t m, double *d_phi, double *d_grad, void *stream);

/* The 7-point discrete Laplacian with zero Dirichlet boundary values on an
 * m x m x m interior grid of spacing h (the PDE operator of the paper's
 * preconditioning experiment, §4.2):
 *   out_ijk = (6 u_ijk - sum of the 6 neighbours) / h^2, neighbours outside
 *   the grid taken as 0; index (k m + j) m + i.
 * d_u, d_out: device, m^3 FP64, not overlapping.  Stream-ordered, asynchronous.
 * FMM_ERR_INVALID_ARG for m < 0, h <= 0, m^3 beyond int64 range or NULL
 * pointers with m > 0. */
fmm_status fmm_laplace7_apply(const double *d_u, double *d_out, int64_t m, double h, void *stream);

/* The Helmholtz operator of the same experiment (§4.2, wave number kappa):
 *   out = (7-point Laplacian as above) u - kappa^2 u.
 * Same arguments, layout and errors as fmm_laplace7_apply, plus
 * FMM_ERR_INVALID_ARG for a kappa that is not finite. */
fmm_status fmm_helmholtz7_apply(const double *d_u, double *d_out, int64_t m, double h,
                                double kappa, void *stream);

/* Number of kernels this library has launched in this process so far. */
uint64_t fmm_kernel_launches(void);

/* Morton keys and their stable sort, allocating no device memory.
 * The paper has no counterpart: this serves callers that cannot let a
 * library call cudaMalloc -- e.g. a host application whose memory manager
 * already holds all free device memory in its own pool, or a
 * latency-critical loop that forbids cudaMalloc/cudaFree because they can
 * synchronise the device and take unbounded time.
 *   d_xyz  : device, n x 3 FP64 (input)
 *   d_keys : device, uint64[n] (output) sorted Morton keys, the same as
 *            fmm_plan_export array 0 of a plan built on d_xyz
 *   d_perm : device, int32[n] (output) input index of each sorted key
 *            (stable), the same as export array 1
 *   h_root : host double[4] (output, may be NULL): lo_x, lo_y, lo_z, D
 * Scratch comes from one fixed device array of this library (12,906,752
 * bytes: room for FMM_NOALLOC_MAX_POINTS points) that every GPU loading the
 * library holds until the process exits.  n above FMM_NOALLOC_MAX_POINTS is
 * rejected with FMM_ERR_INVALID_ARG, and so is a stream of another device
 * than the current one.  The first call on a device looks up the array's
 * device address (once per device; a cudaDeviceReset needs the library
 * reloaded).  Every call reads the root cube back and synchronises `stream`,
 * so no call can be part of a CUDA graph: a stream that is capturing is
 * rejected with FMM_ERR_INVALID_ARG (the caller's capture is left intact).
 * All calls share the array: calls that can
 * overlap on the GPU (different streams, or different host threads on one
 * device) race and must be serialised by the caller.  Synchronises `stream`
 * (the root cube and the finiteness check are read back).
 * Errors: INVALID_ARG, NONFINITE_INPUT, CUDA. */
#define FMM_NOALLOC_MAX_POINTS 1048576
fmm_status fmm_morton_sort_noalloc(const double *d_xyz, int64_t n, uint64_t *d_keys,
                                   int32_t *d_perm, double *h_root, void *stream);

/* Release the plan and all its device memory (synchronises its stream). */
fmm_status fmm_plan_destroy(fmm_plan_t plan);

const char *fmm_status_string(fmm_status s);
const char *fmm_last_error_message(void);

#ifdef __cplusplus
}
#endif
#endif /* FMM_H */
