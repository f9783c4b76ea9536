/*
 * dfmm.h — C ABI of the GB300 directional fast multipole matvec.
 *
 * The library computes, for N points p_i in R^3 and densities f_j,
 *
 *     u_i = sum_{j : p_j != p_i} G(p_i, p_j) f_j,   G(x, y) = exp(2 pi i |x-y|) / |x-y|
 *
 * (Eq. 1 of Benson, Poulson, Tran, Engquist, Ying, "A parallel directional
 * fast multipole method", arXiv:1311.4257; wavelength 1, |p_i| <= K/2).  The
 * self term G(p_i, p_i) is infinite; every source whose point is bitwise equal
 * to the target point is skipped.
 *
 * The method is the sequential directional FMM of Alg. 1 (Sec. 2.3): an
 * octree that is uniform in the high-frequency regime (box width w >= 1) and
 * adaptive below it (Sec. 2.2); directional low-rank representations
 * (Eq. 2, Sec. 2.1) with M2M / M2L / L2L translations over the directional
 * interaction lists for w >= 1 and kernel-independent FMM lists below; and a
 * direct near-field sum.
 *
 * Conventions
 *  - Every call returns a dfmm_status (0 on success).  On failure the message
 *    of the calling thread's last error is available from dfmm_last_error().
 *  - "device pointer" means memory of the current CUDA device, allocated by
 *    the caller (cudaMalloc, torch, ...).  "host pointer" means ordinary host
 *    memory.  The library never frees caller memory.
 *  - Complex numbers are interleaved (re, im) pairs of the stated float type.
 *  - A plan is immutable after dfmm_plan returns and is owned by the library
 *    until dfmm_destroy.  Applies on one plan may be issued from several host
 *    threads on different streams: each stream gets its own workspace.
 */
#ifndef DFMM_H
#define DFMM_H

#include <stdint.h>
#include <cuda_runtime_api.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct dfmm_plan_s* dfmm_plan_t;   /* opaque, owned by the library */

typedef enum {
  DFMM_OK = 0,
  DFMM_ERR_INVALID = -1,      /* bad argument (null pointer, N < 1, nrhs < 1, ...) */
  DFMM_ERR_DOMAIN = -2,       /* a point lies outside the root box |x|_inf <= K/2 */
  DFMM_ERR_OOM = -3,          /* device or host allocation failed */
  DFMM_ERR_CUDA = -4,         /* a CUDA runtime / cuBLAS call failed */
  DFMM_ERR_UNSUPPORTED = -5,  /* eps outside [1e-8, 1e-2], K outside (0, 4096] */
  DFMM_ERR_TIMEOUT = -6,      /* a device-side bounded wait gave up */
  DFMM_ERR_DEVICE = -7,       /* a device-side check failed (status word set) */
  DFMM_ERR_CANCELLED = -8     /* a queued server request was cancelled (dfmm_server_cancel) */
} dfmm_status;

/* Plan-time options.  Zero-initialise and set what you need; zero fields take
 * the defaults given in brackets. */
typedef struct {
  int32_t leaf_max;        /* [64] an LF box with more points is split (Sec. 2.2) */
  int32_t sample_box;      /* [1024] box samples per skeleton */
  int32_t sample_far;      /* [4096] far-region samples per skeleton */
  int32_t sketch_rows;     /* [0 = 400 if eps >= 1e-7, else 800] rows of the random sketch in the
                              pivoted QR (at least twice the largest rank) */
  double eps_op_factor;    /* [0 = 0.3 if eps >= 1e-7, else 0.1] skeleton tolerance = eps * factor */
  int32_t m2l_mode;        /* [0] translations on: 0 = automatic (tensor cores if eps >= 1e-5, else
                              FP32 CUDA cores), 1 = FP32 CUDA cores, 2 = tensor cores (tcgen05,
                              scaled FP16 hi/lo split; adds about 2e-6 relative error) */
  int32_t host_threads;    /* [0 = all cores] threads for the skeleton precompute */
  const char* cache_dir;   /* [NULL = no disk cache] directory for skeleton files */
  int32_t tc_stages;       /* [0 = all] with m2l_mode 2, the translation families that run on
                              the tensor cores, as a bit mask: 1 = HF M2L, 2 = LF M2L (V list),
                              4 = M2M, 8 = L2L, 16 = P2L projection; the others run on the FP32
                              CUDA cores.  For measuring the error each family's split adds. */
  int32_t wait_test;       /* [0] testing aid for the failure path: with 1, the first CTA of every
                              tensor-core translation launch waits on a barrier that nothing
                              arrives at.  Its bounded wait gives up after 0.2 s, the launch (and
                              the rest of the apply's tensor-core launches) stop early, and
                              dfmm_sync_status returns DFMM_ERR_TIMEOUT.  The potentials of such
                              an apply are undefined. */
  int32_t tile_order;      /* [0] order of a translation stage's work tiles: 0 = by block of
                              target rows when the stage's operators total at most 64 MB (they
                              stay in L2), else by operator (each read from DRAM once); 1 = always
                              by target block; 2 = always by operator.  The result is the same up
                              to the order of the floating-point additions. */
  int32_t p2p_mode;        /* [0] near-field form: 0 = automatic (2 if eps >= 1e-5, else 1);
                              1 = double-float box-local coordinates; 2 = FP32 coordinates, with
                              the pairs closer than min(0.5, 1e-6 / eps) wavelengths corrected
                              exactly (listed at plan time).  Form 2 falls back to 1 when two
                              distinct points round to the same FP32 coordinates, when N >= 2^25,
                              or when a leaf has more than 127 near leaves. */
  int32_t tc_layout;       /* [0] tensor-core translations (m2l_mode 2): 0 = split-complex form
                              (Re y = Tr xr - Ti xi, Im y = Ti xr + Tr xi as four real products;
                              ranks padded to 16) wherever the target rank is at most 128, the
                              real-block form elsewhere; 1 = the real-block form [[Tr, -Ti],
                              [Ti, Tr]] everywhere (ranks padded to 8). */
  int32_t tc_accumulate;   /* [0] split-complex form: 0 = automatic (1 if eps >= 1e-5, else 2);
                              1 = one tensor-memory accumulator per component, two buffers, so
                              that a tile's MMAs overlap the previous tile's epilogue (faster;
                              the cross terms take the large terms' accumulation truncation:
                              about 1e-6 more error against the FP32 form); 2 = the hi*hi terms
                              and the cross terms in separate accumulators (one tile at a time). */
  int32_t tc_precision;    /* [0] element type of the scaled hi / lo split of the tensor-core form:
                              0 = FP16 (11 + 11 significant bits, kind::f16); 1 = BF16 (8 + 8 bits,
                              "3xBF16"); 2 = TF32 (11 + 11 bits with an 8-bit exponent, kind::tf32
                              at half the FP16 rate, "3xTF32").  1 and 2 need tc_layout 0; stages
                              whose target rank exceeds 128 then run on the FP32 CUDA cores. */
  int32_t arith;           /* [0] arithmetic of the apply: 0 = automatic (32 if eps >= 1e-6, else
                              64); 32 = the FP32 forms above (complex64 f and u); 64 = FP64
                              throughout (translations, rows, check points and near field on
                              the CUDA cores; operators kept in complex128), for eps down to
                              1e-8.  With 64, f and u of every apply entry point are complex128
                              [nrhs][N], m2l_mode 2 is refused and the other m2l / p2p / tc
                              options are ignored; dfmm_solve takes arith 32 plans only. */
  int32_t skeleton_host;   /* [0] where the skeleton pivot selection (Sec. 2.1: pivoted QR of the
                              random sketch, then of the far samples) runs: 0 = on the GPU for all
                              representation types of the plan at once; 1 = host threads
                              (host_threads).  The samples, draws and pivot rule are the same. */
} dfmm_options;

/* Build a plan (Sec. 2.2 octree, lists, Eq. 2 representations and the
 * translation operators).
 *   points : device pointer, float64, row-major [N][3], caller order.  Read
 *            during the call only; the plan keeps its own copies.
 *   N      : number of points, >= 1.
 *   K      : domain size in wavelengths; every point must satisfy
 *            max_d |p_d| <= K/2 (else DFMM_ERR_DOMAIN).  0 < K <= 4096.
 *   eps    : requested relative accuracy, 1e-8 <= eps <= 1e-2.
 *   opts   : host pointer to options, or NULL for the defaults.
 *   out    : host pointer receiving the plan handle.
 * Runs on the current device and the legacy default stream; synchronises the
 * device before returning. */
int dfmm_plan(const double* points, int64_t N, double K, double eps,
              const dfmm_options* opts, dfmm_plan_t* out);

/* The matvec u = G f (Alg. 1 passes plus the near field).
 *   f      : device pointer, complex64 [nrhs][N] in the caller's point order
 *            (complex128 for a plan whose arith is 64: eps < 1e-6 by default).
 *   u      : device pointer, complex64 [nrhs][N] (complex128 likewise); overwritten, never
 *            accumulated.  Must not alias f.
 *   nrhs   : number of right-hand sides, 1 <= nrhs <= 64.
 *   stream : CUDA stream; the call only enqueues work (no host sync).
 * The workspace of (plan, stream) is allocated on the first call with that
 * stream and nrhs at least as large; it is reused afterwards. */
int dfmm_apply(dfmm_plan_t plan, const void* f, void* u, int nrhs, cudaStream_t stream);

/* Same as dfmm_apply with host (pageable or pinned) f and u: copies f to the
 * device, applies, copies u back, and synchronises the stream. */
int dfmm_apply_host(dfmm_plan_t plan, const void* f_host, void* u_host, int nrhs,
                    cudaStream_t stream);

/* Read back the device status word of the last apply on `stream`
 * (synchronises the stream), together with that of the last
 * dfmm_apply_noalloc on the current device if that call was issued on
 * `stream`.  Returns DFMM_OK, DFMM_ERR_TIMEOUT or DFMM_ERR_DEVICE. */
int dfmm_sync_status(dfmm_plan_t plan, cudaStream_t stream);

/* Device-side bounds check of every index table of the plan: translation
 * pairs against the rows of their source and target states, the work tiles of
 * every workspace laid out so far against operator and pair counts, the
 * per-point row maps and leaf jobs, the W- and X-list jobs, the near-field
 * leaves, offsets, sources and staging list, the close pairs and the
 * permutation.  The check kernels only read the tables.  Returns DFMM_OK, or
 * DFMM_ERR_DEVICE naming the first table with an entry out of range
 * (dfmm_last_error).  Synchronises `stream`.  A library built with
 * DFMM_CHECK=1 (paper_1311_4257_gb300/build.py) runs it at the end of every
 * dfmm_plan.
 *   flags: 0, or DFMM_VALIDATE_PLANT (testing aid): also check a scratch copy
 *          of one translation pair table whose first source row is set to
 *          its bound; the plan is not touched, and the call must fail. */
#define DFMM_VALIDATE_PLANT 1
int dfmm_validate(dfmm_plan_t plan, cudaStream_t stream, int flags);

/* Free every resource of the plan (waits for the device first).  NULL is a
 * no-op; a handle that is not a live plan, or a plan that a request server
 * still holds (queued or running requests), is refused with DFMM_ERR_INVALID. */
int dfmm_destroy(dfmm_plan_t plan);

/* Sizes and counts of a plan, for reports and tests. */
typedef struct {
  int64_t N;
  double K, W, eps, eps_op;
  int32_t n_levels;            /* octree levels (root = 0) */
  int32_t level_hf_top;        /* coarsest level with a non-empty HF list */
  int32_t level_w1;            /* level of width 1 */
  int64_t boxes[32];           /* non-empty boxes per level */
  int64_t leaves[32];          /* leaves per level */
  int64_t hf_pairs[32];        /* HF-M2L pairs per level */
  int64_t hf_offsets[32];      /* distinct HF-M2L offsets per level */
  int64_t slots_out[32];       /* active outgoing (box, direction) per level */
  int64_t slots_in[32];        /* active incoming (box, direction) per level */
  int32_t rank[32];            /* padded representation rank per level */
  int64_t v_pairs, u_pairs, w_pairs, x_pairs;
  int64_t p2p_interactions;    /* sum over U pairs of n_target * n_source */
  int64_t plan_bytes;          /* device bytes held by the plan */
  double plan_seconds;         /* wall time of dfmm_plan */
  double m2l_flops;            /* algorithmic M2L flops per RHS: 8 r_t r_s per pair */
  double other_translation_flops; /* M2M, L2L, LF-M2L, P2M/L2P GEMMs per RHS */
  int64_t hf_ops[32];          /* distinct HF-M2L operators per level (offsets up to cube symmetry) */
  int64_t p2p_close_pairs;     /* FP32 near field: pairs with a stored exact correction */
  int32_t arith;               /* 32 or 64: arithmetic of the apply (options.arith resolved) */
  int32_t reserved;
  double plan_phase_seconds[8];   /* wall time of dfmm_plan by phase: 0 = points, sort, octree, lists
                                     and active directions; 1 = skeletons (Eq. 2 representations,
                                     host, from the disk cache when present); 2 = their upload;
                                     3 = translation operators (M2M, M2L, L2L, P2L projections);
                                     4 = per-point rows (L2P, P2M, M2P); 5 = near-field lists and
                                     close pairs; 6 = tensor-core operator images; 7 = the part of
                                     phase 3 spent forming operators on the device */
  double skeleton_phase_seconds[4]; /* phase 1 in detail: 0 = disk cache and samples; 1 = sketch pivots
                                       (the whole host build in the host form); 2 = check-point
                                       pivots; 3 = least-squares factors */
  int64_t skeleton_types;           /* representation types built or loaded (canonical, up to the
                                       cube's symmetries) */
  int64_t plan_id;                  /* unique within the process (a destroyed plan's handle may be
                                       reused by a later plan; its id is not) */
} dfmm_stats;

int dfmm_plan_stats(dfmm_plan_t plan, dfmm_stats* out);

/* Device bytes of the workspace that one apply with nrhs right-hand sides
 * needs (sorted densities and potentials, translation states, staging buffers
 * and work tables; the plan itself is not included).  -1 on a bad argument. */
int64_t dfmm_apply_workspace_bytes(dfmm_plan_t plan, int nrhs);

/* Device bytes held by the plan (tree, lists, operators, evaluation rows);
 * the same value as dfmm_stats.plan_bytes.  -1 for a NULL plan. */
int64_t dfmm_plan_bytes(dfmm_plan_t plan);

/* Several independent matvecs in one call: u[k] = G_k f[k] for k < count,
 * where G_k is the operator of plans[k] (Eq. 1 on that plan's points) and
 * f[k], u[k] are device pointers laid out as in dfmm_apply with nrhs[k]
 * right-hand sides.  The paper treats one geometry at a time; this entry point
 * batches uneven geometries so that their stages overlap on the device: the
 * applies run on a library-owned pool of streams that wait for the work
 * already queued on `stream`, and `stream` waits for all of them.  Asynchronous
 * like dfmm_apply (no host sync); the caller keeps the buffers alive until
 * the batch has finished on `stream`.  Errors: DFMM_ERR_INVALID for a NULL
 * array or element, nrhs outside [1, 64], f[k] == u[k], or a plan of another
 * device (nothing is launched then); a failure during launch returns its code
 * and may leave earlier applies of the batch queued. */
int dfmm_apply_batched(const dfmm_plan_t* plans, const void* const* f, void* const* u, const int* nrhs, int count,
                       cudaStream_t stream);

/* The batched form with merged stages (the paper has no counterpart): the
 * plans of a batch run wave by wave, one wave being the same step of every
 * plan (by kind and box width), and the tensor-core translation stages of a
 * wave (split-complex form) run as one persistent launch over a table of the
 * plans' stages.  dfmm_batch_create fixes the device buffers f[k], u[k] (layout
 * as in dfmm_apply, nrhs[k] right-hand sides, plans[k] of the current device),
 * lays out one workspace per plan and the merged stage tables, and runs the
 * batch once on `stream` (u = G f).  flags:
 *   DFMM_BATCH_TUNE:  autotune: time every merged launch under each of three
 *                     tile orders (by block of 8 MB or 2 MB of target rows, or
 *                     by operator) and keep the fastest per launch;
 *   DFMM_BATCH_GRAPH: capture one run of the batch into a CUDA graph.
 * dfmm_batch_launch reruns the batch on `stream` (as one graph launch when
 * captured) with the contents f has then; runs of one batch must not overlap
 * (they share the workspaces).  Stages that the split-complex form does not
 * take (target rank above 128, FP32 CUDA-core plans) run per plan.  Plans must
 * stay alive while the batch exists.  dfmm_batch_destroy waits for the device
 * and frees the batch. */
typedef struct dfmm_batch_s* dfmm_batch_t;
#define DFMM_BATCH_GRAPH 1
#define DFMM_BATCH_TUNE 2
typedef struct {
  int64_t launches;            /* kernel launches of one run */
  int64_t waves;               /* waves of the batch */
  int64_t merged_launches;     /* merged translation launches of one run */
  int64_t merged_stages;       /* plan stages they cover */
  int32_t order_chosen[3];     /* merged launches per chosen tile order (8 MB, 2 MB blocks, operator) */
  int32_t graph;               /* 1 if captured */
  double tune_ms[3];           /* autotuning: summed merged-launch time under each order */
} dfmm_batch_report;

int dfmm_batch_create(const dfmm_plan_t* plans, const void* const* f, void* const* u, const int* nrhs, int count,
                      cudaStream_t stream, int flags, dfmm_batch_t* out);
int dfmm_batch_launch(dfmm_batch_t batch, cudaStream_t stream);
int dfmm_batch_stats(dfmm_batch_t batch, dfmm_batch_report* out);
int dfmm_batch_destroy(dfmm_batch_t batch);

/* Export of the plan's tree and lists for parity tests (host buffers).
 * Call with a NULL buffer to get the required element count in *count.
 *   what = 0: Morton permutation, int64 [N]
 *          1: sorted Morton keys, uint64 [N]
 *          2: boxes, int64 [n][5] = (level, key prefix, first, count, leaf)
 *          3: HF-M2L pairs, int64 [n][5] = (level, target box, source box,
 *             incoming direction, outgoing direction), box = index within level
 *          4: active outgoing slots, int64 [n][3] = (level, box, direction)
 *          5: active incoming slots, int64 [n][3]
 *          6: V pairs, int64 [n][3] = (level, target, source)
 *          7: U pairs, int64 [n][4] = (target level, target, source level, source)
 *          8: W pairs, int64 [n][4] (target leaf level, leaf, source level, box)
 *          9: X pairs, int64 [n][4] (target level, box, source level, leaf)
 *         10: ranks of every representation type, int64 [n][3] = (level, cell or -1, rank)
 */
int dfmm_export(dfmm_plan_t plan, int what, void* buffer, int64_t* count);

/* The matvec of dfmm_apply without allocating device memory.
 *
 * The paper has no counterpart: this entry point serves callers that must not
 * let a library call cudaMalloc or cudaFree, such as request paths of services
 * that forbid allocation after start-up (the allocator belongs to someone
 * else, or its latency and failures are not allowed there) and hosts whose
 * device memory is budgeted in advance.  Every per-apply buffer (the status
 * word, sorted densities and potentials, the translation states, the staging
 * buffers and the work tables) is laid out in one file-scope device array of
 * dfmm_noalloc_capacity() bytes (64 MiB), which every device that loads the
 * library holds until the process exits.
 *   plan, f, u, nrhs, stream : as for dfmm_apply (device pointers, complex64
 *            [nrhs][N], complex128 for an arith 64 plan; u overwritten).  The plan must belong to the current
 *            device.
 * An apply fits exactly when dfmm_apply_workspace_bytes(plan, nrhs) <=
 * dfmm_noalloc_capacity(); otherwise the call returns DFMM_ERR_UNSUPPORTED,
 * with the required size in the message, and enqueues nothing.
 * The first call on a device looks up the array's device address on that
 * device (make that first call before any stream capture).  All calls share
 * the one array and each overwrites what the previous left there: calls that
 * overlap on the GPU (other streams, other threads) race on it and must be
 * serialised by the caller.  The status word of the last such apply on the
 * current device is read back by dfmm_sync_status (with any plan and the
 * stream of that apply). */
int dfmm_apply_noalloc(dfmm_plan_t plan, const void* f, void* u, int nrhs, cudaStream_t stream);

/* Size in bytes of the scratch array of dfmm_apply_noalloc. */
int64_t dfmm_noalloc_capacity(void);

/* A captured apply (the paper has no counterpart): dfmm_graph_create lays out
 * a workspace that the graph object owns (dfmm_apply_workspace_bytes of device
 * memory), runs one ordinary apply of the plan on the device buffers f and u
 * (nrhs right-hand sides, layout as in dfmm_apply) on `stream`, then captures
 * the same apply into a CUDA graph.  dfmm_graph_launch replays it on any
 * stream of the device: u = G f with the contents f has when the replay runs,
 * as one graph launch instead of some thirty kernel launches and memsets.  f
 * and u must stay allocated while the graph exists; concurrent replays of one
 * graph must not overlap (they share the workspace).  dfmm_graph_destroy waits
 * for the device, then frees the graph and its workspace.  Errors: as
 * dfmm_apply; DFMM_ERR_CUDA if the capture fails. */
typedef struct dfmm_graph_s* dfmm_graph_t;
int dfmm_graph_create(dfmm_plan_t plan, const void* f, void* u, int nrhs, cudaStream_t stream, dfmm_graph_t* out);
int dfmm_graph_launch(dfmm_graph_t graph, cudaStream_t stream);
int dfmm_graph_destroy(dfmm_graph_t graph);

/* Iterative solution of (alpha I + beta G) x = b by restarted GMRES around the
 * plan's matvec: the use the paper's fast matvec serves (Sec. 1: the
 * discretised integral equation is solved by a Krylov method, one
 * application of G per iteration).  b and x are device complex64 vectors of
 * N values in the caller's point order; x holds the initial guess on entry
 * and the solution on return.  alpha and beta are complex (re, im).  GMRES
 * restarts every `restart` iterations (1..500) and stops once the estimated
 * relative residual |b - A x| / |b| is <= tol or after maxit matvecs.  On
 * return *iters (if not NULL) holds the number of matvecs of the Krylov
 * iterations, and *relres (if not NULL) the true relative residual of x
 * (one more matvec).  The accuracy of A is that of the plan (eps), so tol
 * below about eps is not meaningful.  The plan must compute in FP32 (arith
 * 32; else DFMM_ERR_UNSUPPORTED).  Allocates (restart + 2) N complex64 of
 * device workspace per call; synchronises `stream` at every iteration (the
 * small least-squares problem is solved on the host).  Returns DFMM_OK
 * whether or not tol was reached (compare *relres), or an error status. */
int dfmm_solve(dfmm_plan_t plan, double alpha_re, double alpha_im, double beta_re, double beta_im, const void* b,
               void* x, int restart, int maxit, double tol, cudaStream_t stream, int* iters, double* relres);

/* Request server (the paper has no counterpart): continuous batching of
 * matvec requests over plans that stay resident.
 *
 * dfmm_server_create starts a dispatcher thread that serves requests on
 * `streams` streams of the current device.  It allocates one device arena of
 * budget_bytes, and every running apply takes its staging buffers and
 * workspace from that arena; nothing else is allocated while serving.
 * Requests are admitted oldest first.  The dispatcher groups every pending
 * request on the same plan, up to max_rhs right-hand sides in total, into one
 * apply whose right-hand sides sit side by side.  A group starts when a
 * stream is free and its footprint fits in the arena: 2 N nrhs complex64
 * (complex128 for an arith 64 plan) staging plus dfmm_apply_workspace_bytes.  Requests that arrive while others
 * run are admitted as streams and memory free up.  A request that could never
 * fit fails with DFMM_ERR_OOM.
 *
 * dfmm_server_submit queues one request: nrhs right-hand sides of the plan's
 * N points, host buffers f_host (read) and u_host (written) of nrhs * N
 * complex64 each (complex128 for an arith 64 plan), laid out as in dfmm_apply (pinned memory makes the copies
 * asynchronous).  The caller keeps both buffers alive and untouched until
 * dfmm_server_wait has returned for the ticket written to *ticket.
 * dfmm_server_wait blocks until the request has finished or timeout_seconds
 * have passed (DFMM_ERR_TIMEOUT; the ticket stays valid), then returns the
 * request's status and, if latency_ms is not NULL, its submit-to-finish time.
 * A ticket can be collected once.
 * dfmm_server_cancel removes a request that has not started from the queue:
 * its wait returns DFMM_ERR_CANCELLED and u_host is not written.  A request
 * that has started or finished is not cancelled (DFMM_ERR_INVALID); it
 * completes normally.
 * dfmm_server_fail_next (testing aid for the failure path): the next group
 * the dispatcher starts fails on the host before anything is queued for it,
 * as a failed staging copy would; its requests finish with `status` (a
 * negative dfmm_status) and the server goes on with the others.
 * A submitted request holds its plan: dfmm_server_submit refuses a handle that
 * is not a live plan (never created, or destroyed: DFMM_ERR_INVALID), and
 * dfmm_destroy refuses a plan while requests on it are queued or running.
 * Cancelled and failed requests count in requests_failed.
 * dfmm_server_destroy finishes every queued request, then frees the server. */
typedef struct dfmm_server_s* dfmm_server_t;

typedef struct {
  int64_t requests_done;           /* finished without error */
  int64_t requests_failed;
  int64_t applies;                 /* grouped applies run */
  int64_t rhs_done;                /* right-hand sides of the finished requests */
  int64_t points_rhs_done;         /* sum over finished requests of N x nrhs */
  int64_t pending;                 /* queued, not started */
  int32_t max_concurrent_applies;  /* most groups running at once so far */
  int32_t reserved;
  double wall_seconds;             /* first submit to last finish */
  double latency_p50_ms;           /* over finished requests */
  double latency_p99_ms;
} dfmm_server_report;

int dfmm_server_create(int streams, int64_t budget_bytes, int max_rhs, dfmm_server_t* out);
int dfmm_server_submit(dfmm_server_t server, dfmm_plan_t plan, const void* f_host, void* u_host, int nrhs,
                       int64_t* ticket);
int dfmm_server_wait(dfmm_server_t server, int64_t ticket, double timeout_seconds, double* latency_ms);
int dfmm_server_cancel(dfmm_server_t server, int64_t ticket);
int dfmm_server_fail_next(dfmm_server_t server, int status);
int dfmm_server_stats(dfmm_server_t server, dfmm_server_report* out);
int dfmm_server_destroy(dfmm_server_t server);

/* Per-kernel timing of applies, measured with CUDA events that the library
 * records on the apply stream around each of its launches.
 *   enable != 0 : start recording on `stream` (out may be NULL).
 *   enable == 0 : stop, synchronise `stream`, and write the totals since
 *                 recording started into out[0 .. *n) (cap entries at most),
 *                 one entry per kernel family:
 *                 m2l_hf, m2l_lf, m2m, l2l, p2l_proj, p2m_eval, p2l_eval,
 *                 l2p, m2p, p2p, permute, zero, split.
 *   flops and bytes are algorithmic: 8 r_t r_s per (pair, right-hand side)
 *   for the translations with the unpadded ranks; every operator, source
 *   state and target state counted once per launch; for P2P 16 + 8 nrhs
 *   flops per interaction. */
typedef struct {
  char name[32];
  int64_t launches;
  double ms;
  double flops;
  double bytes;
} dfmm_kernel_time;

int dfmm_profile(dfmm_plan_t plan, cudaStream_t stream, int enable, dfmm_kernel_time* out, int cap, int* n);

/* Number of kernel launches one apply with nrhs right-hand sides makes. */
int64_t dfmm_apply_launches(dfmm_plan_t plan, int nrhs);

/* Host-only (no device work): build one representation type of Eq. 2 the
 * way dfmm_plan does, for inspection and tests.
 *   w       : box width (a power of two); cell: face-cell index (w >= 1) or
 *             -1 for the non-directional low-frequency type (w < 1).
 *   w_top   : coarsest width whose representations are evaluated.
 *   eps_op  : skeleton tolerance; sample_box, sample_far, sketch_rows as in
 *             dfmm_options (0 = default).
 *   r_out   : receives the rank r.
 *   b2, a2  : host buffers of at least 6*cap doubles, or NULL; on return they
 *             hold the 2r box check points (first r = equivalent points) and
 *             the 2r far check points, [2r][3] row-major, box-centred frame.
 *   cap     : capacity of b2/a2 in points; DFMM_ERR_INVALID if 2r > cap. */
int dfmm_representation(double w, int cell, double w_top, double eps_op, int sample_box, int sample_far,
                        int sketch_rows, int* r_out, double* b2, double* a2, int cap);

/* dfmm_representation with the two pivot selections (the column-pivoted QR of
 * the +-1 sketch and the two QRs that pick the far check points) on the
 * current GPU, the way dfmm_plan runs them unless options.skeleton_host is
 * set.  Samples and sketch draws are the host's; the FP64 rounding differs,
 * so pivots that nearly tie may differ from dfmm_representation's (either
 * result is a valid skeleton).  Synchronises the device; same arguments and
 * errors as dfmm_representation. */
int dfmm_representation_device(double w, int cell, double w_top, double eps_op, int sample_box, int sample_far,
                               int sketch_rows, int* r_out, double* b2, double* a2, int cap);

/* Measured peak rates of the current GPU, for roofline denominators (the
 * paper has no counterpart).  Each rate comes from a short probe kernel of
 * independent chains on all SMs, timed with CUDA events after one warm-up
 * launch: fused multiply-adds on the CUDA cores (FP32 and FP64, 2 flops
 * each), fast sine + cosine pairs and reciprocal square roots on the
 * special-function unit, and dense tcgen05 MMAs (M = 128, N = 256, one CTA
 * per SM, operands from shared memory) of kind::tf32 and kind::f16.  The
 * rates depend on the SM clock at the time; sample it beside the call.
 * Allocates 4 KB of device memory; synchronises the device. */
typedef struct {
  int32_t sm_count;
  int32_t reserved;
  double fp32_fma_tflops;
  double fp64_fma_tflops;
  double sincos_gops;        /* sine + cosine pairs per second, 1e9 */
  double rsqrt_gops;
  double tf32_mma_tflops;
  double f16_mma_tflops;
} dfmm_peaks;

int dfmm_measure_peaks(dfmm_peaks* out);

/* Thread-local message of the last failed call on this thread. */
const char* dfmm_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* DFMM_H */
