/*
 * vqnnf.h -- C ABI of the GB300 VQ-NNF template-matching hot path.
 *
 * The calls follow the problem statement of Gupta & Sintorn, "Efficient High-Resolution
 * Template Matching with Vector Quantized Nearest Neighbour Fields" (Sec. 3): a template
 * tau of w x h x c features and a query I of W x H x c features; a k-vector codebook of
 * the template (Sec. 3.1); the nearest-neighbour field of both images over that codebook
 * (Algorithm 1); coarse-filter responses on the integral image of the one-hot field
 * (Sec. 3.2, Eq. 1, Algorithm 2); and the similarity score of every query sub-window
 * (Sec. 3.3, Eq. 2) with its maximum (Sec. 4, "Target Localization").
 *
 * Conventions shared by every call
 * --------------------------------
 * Memory.    Every pointer named *device* is CUDA device memory owned by the caller; the
 *            library never allocates, frees or retains memory.  Scratch space is passed in
 *            as `ws` (device, at least vqnnf_workspace_bytes(...) bytes, 256-byte aligned);
 *            its contents on entry are ignored.  Filter banks are host memory, read during
 *            the call only.
 * Layout.    Feature maps are HWC row-major float32: element (y, x, i) of an H x W x D map
 *            is at [(y * W + x) * D + i].  Label images are row-major uint8 (k <= 256).
 *            Codebooks are k x D row-major float32.
 * Streams.   `stream` is a cudaStream_t (NULL = legacy default stream).  Calls only
 *            enqueue work on it and return; none synchronises the host, so a call can be
 *            captured into a CUDA graph.  Results are valid once the stream reaches them.
 * Errors.    Argument errors are detected on the host and returned before anything is
 *            enqueued (VQNNF_EINVAL, VQNNF_ENOMEM for a workspace that is too small,
 *            VQNNF_EUNSUPPORTED for shapes outside the supported range).  A failed launch
 *            returns VQNNF_ECUDA.  Bounded device-side waits that give up record
 *            VQNNF_ETIMEOUT in a device error word that vqnnf_last_device_error() reads.
 *            No call aborts the process or traps on the device.
 * Threads.   Calls from several host threads on different streams are independent, with
 *            three exceptions, all process-wide: the profiling events of
 *            vqnnf_set_kernel_events (set under a lock), the one device scratch area of
 *            vqnnf_assign_noalloc, which overlapping calls must not share, and the lanes of
 *            the batch calls (library streams shared per device: concurrent batch calls
 *            enqueue one at a time under a lock, and their work shares the lanes).
 * Ties.      Nearest-neighbour ties go to the lowest centroid index; the heatmap maximum
 *            goes to the lowest row-major (y, then x) window.
 */
#ifndef VQNNF_H
#define VQNNF_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum vqnnf_status {
    VQNNF_OK = 0,
    VQNNF_EINVAL = 1,        /* bad pointer, size or filter bank                         */
    VQNNF_ENOMEM = 2,        /* workspace smaller than vqnnf_workspace_bytes(...)          */
    VQNNF_ECUDA = 3,         /* a CUDA runtime call or kernel launch failed               */
    VQNNF_ETIMEOUT = 4,      /* a bounded device wait gave up (see last_device_error)     */
    VQNNF_EUNSUPPORTED = 5   /* valid request outside the implemented range              */
} vqnnf_status;

/* Arithmetic of the nearest-neighbour distance contraction (Sec. 4.2: exact L2 NN). */
typedef enum vqnnf_prec {
    VQNNF_PREC_FP32 = 0,     /* FP32 SIMT dot products                                   */
    VQNNF_PREC_BF16 = 1,     /* BF16 tensor cores (tcgen05), FP32 accumulation            */
    VQNNF_PREC_FP8 = 2       /* FP8 e4m3 tensor cores (tcgen05 kind::f8f6f4) with a power-of-
                              * two scale per feature row and per centroid, FP32
                              * accumulation; the features are quantised by the call itself
                              * (workspace: H*W*D bytes more).  D % 16 == 0 and
                              * ceil(k / 32) * 32 * D <= 131072 (the codebook stays in shared
                              * memory: k <= 256 at D <= 512, k <= 128 at D <= 1024) */
} vqnnf_prec;
/* Both precisions return the exact nearest neighbour of the FP32 inputs: every pixel
 * whose two best distances are closer than a proven bound on the contraction's error is
 * re-scored in compensated FP32 over its candidate centroids.  Labels therefore equal
 * an exact (FP64) evaluation except where that evaluation's own relative gap between
 * the two best distances is below about 1e-11. */

/* A rectangle of a coarse filter, relative to the window's top-left corner, half-open:
 * columns [x0, x1), rows [y0, y1), 0 <= x0 < x1 <= tw, 0 <= y0 < y1 <= th.  Its
 * response for cluster j is weight * (number of pixels labelled j inside it). */
typedef struct vqnnf_rect {
    int32_t x0, y0, x1, y1;
    int32_t weight;
} vqnnf_rect;

/* A filter f: the sum of its rectangles' responses (the integral-image form of a coarse
 * filter, Algorithm 2), its score weight w_f (Eq. 2) and its normaliser A_f (the
 * receptive-field area of Eq. 1).  The score uses w_f / A_f. */
typedef struct vqnnf_filter {
    int32_t n_rects;
    const vqnnf_rect *rects;
    float w_f;
    float area;
} vqnnf_filter;

/* Counters of the near-tie re-scoring, accumulated on the device by vqnnf_assign. */
typedef struct vqnnf_assign_stats {
    unsigned long long n_flagged;     /* pixels whose contraction result was ambiguous      */
    unsigned long long n_candidates;  /* candidate centroids re-scored over those pixels    */
    unsigned long long n_deep;        /* pixels that needed the double-float second stage   */
    unsigned long long reserved;
} vqnnf_assign_stats;

/* Operation codes for vqnnf_workspace_bytes. */
enum {
    VQNNF_OP_FIT = 0,
    VQNNF_OP_ASSIGN = 1,
    VQNNF_OP_FILTER_RESPONSES = 2,
    VQNNF_OP_SCORE = 3
};

/* Scratch bytes needed by one call.  Arguments not used by `op` are ignored:
 *   FIT:              H x W = template h x w, D, k, prec
 *   ASSIGN:           H x W pixels, D, k, prec
 *   FILTER_RESPONSES: nothing (returns a small constant)
 *   SCORE:            H x W query, k, th x tw template, F filters
 * Returns 0 for arguments that are out of range. */
size_t vqnnf_workspace_bytes(int op, int H, int W, int D, int k, int th, int tw, int F,
                             int prec);

/* k-means codebook of the template (Sec. 3.1; Sec. 4.2 uses plain k-means).
 *   T      device, h x w x D float32 template features
 *   k      1 <= k <= min(256, h*w) clusters;  iters >= 0 Lloyd steps (no early stop)
 *   seed   seeds the initial centroids: k distinct template pixels, the first k slots of
 *          a Fisher-Yates shuffle of 0..h*w-1 in which slot i swaps with slot
 *          i + (r mod (h*w - i)), r the i-th output of SplitMix64 started at `seed`
 *   C      device, k x D float32, written
 * Each Lloyd step assigns every template pixel to its exact nearest centroid (lowest
 * index on ties), then replaces each non-empty cluster's centroid by the FP64 mean of its
 * members, summed in pixel order and rounded to float32; an empty cluster keeps its
 * centroid.  D % 4 == 0.  `prec` selects the arithmetic of the assignment steps. */
vqnnf_status vqnnf_fit_codebook(const float *T, int h, int w, int D, int k, int iters,
                                uint64_t seed, vqnnf_prec prec, float *C,
                                void *ws, size_t ws_bytes, void *stream);

/* Nearest-neighbour field (Algorithm 1): labels[p] = argmin_j ||X[p] - C[j]||^2.
 *   X       device, H x W x D float32 features (query or template)
 *   C       device, k x D float32 codebook, 1 <= k <= 256
 *   prec    VQNNF_PREC_FP32 (D % 4 == 0), VQNNF_PREC_BF16 (D % 16 == 0) or VQNNF_PREC_FP8
 *           (see vqnnf_prec); every precision returns the exact nearest neighbour: pixels whose
 *           contraction result is ambiguous under its proven error bound are re-scored from
 *           the FP32 inputs
 *   labels  device, H x W uint8, written
 *   stats   device vqnnf_assign_stats, overwritten; may be NULL */
vqnnf_status vqnnf_assign(const float *X, int H, int W, int D, const float *C, int k,
                          vqnnf_prec prec, uint8_t *labels, vqnnf_assign_stats *stats,
                          void *ws, size_t ws_bytes, void *stream);

/* Allocation-free variant of vqnnf_assign.  The paper has no counterpart: this entry point
 * exists for callers that cannot allocate device memory themselves -- plug-ins whose host
 * application owns every device allocation, and loops that must never wait on the allocator
 * (cudaMalloc and cudaFree can synchronise the whole device).  Such callers cannot provide
 * the scratch workspace vqnnf_assign needs, so this call uses a fixed scratch area compiled
 * into the library instead:
 *   - the area is VQNNF_NOALLOC_SCRATCH_BYTES (16 MiB) of device memory, held on every GPU
 *     that loads the library until the process exits;
 *   - a request whose workspace (vqnnf_workspace_bytes(VQNNF_OP_ASSIGN, ...)) exceeds it is
 *     rejected with VQNNF_ENOMEM before anything is enqueued (about 450,000 pixels at D=512,
 *     k=128; use vqnnf_assign with a caller workspace for larger images);
 *   - the first call on a device looks up the area's device address (with that device
 *     current) and keeps it for the life of the process; make that first call before any
 *     stream capture begins.  A device reset (cudaDeviceReset) invalidates the kept address:
 *     do not call this entry point again in that process after one;
 *   - every call on a device shares the one area: calls whose work overlaps on the GPU (on
 *     different streams, or from different host threads) race and give wrong labels --
 *     order them on one stream.  The area keeps the last call's contents; the call clears
 *     what must start at zero itself.
 * Arguments, results and errors are those of vqnnf_assign without ws / ws_bytes; nothing is
 * allocated or freed. */
#define VQNNF_NOALLOC_SCRATCH_BYTES (16u << 20)
vqnnf_status vqnnf_assign_noalloc(const float *X, int H, int W, int D, const float *C, int k,
                                  vqnnf_prec prec, uint8_t *labels, vqnnf_assign_stats *stats,
                                  void *stream);

/* Template representation vectors (Sec. 3.3, R(tau)): for every filter f and cluster j,
 *   counts[f * k + j] = sum over rects of weight * #{pixels labelled j in the rect}
 * with the window placed at the template's origin.
 *   labels  device, h x w uint8 template NNF, every label < k;  bank: host, 1 <= F <= 32
 *           filters with at most 192 rectangles in total (else VQNNF_EUNSUPPORTED); the
 *           counts must fit int32 (|weight| * rectangle area summed over a filter)
 *   counts  device, F x k int32, written */
vqnnf_status vqnnf_filter_responses(const uint8_t *labels, int h, int w, int k,
                                    const vqnnf_filter *bank, int F, int32_t *counts,
                                    void *ws, size_t ws_bytes, void *stream);

/* Similarity heatmap (Eq. 2, |.| read as the L1 norm over clusters):
 *   heat[y][x] = - sum_f (w_f / A_f) * sum_j | t_counts[f][j] - q_f(y, x)[j] |
 * for every valid window top-left (y, x), 0 <= y <= H - th, 0 <= x <= W - tw, where
 * q_f(y, x) are the filter's counts over the query NNF with the window at (y, x), taken
 * from the per-cluster integral image of the one-hot query NNF.  The inner sums are exact
 * integers; the outer sum is float32 in bank order.
 *   q_labels  device, H x W uint8, every label < k;  t_counts: device, F x k int32
 *             (vqnnf_filter_responses)
 *   heatmap   device, (H - th + 1) x (W - tw + 1) float32, written
 *   argmax_yx device int32[2] (y, x) of the maximum, lowest row-major index on ties;
 *             may be NULL */
vqnnf_status vqnnf_score(const uint8_t *q_labels, int H, int W, int k, int th, int tw,
                         const vqnnf_filter *bank, int F, const int32_t *t_counts,
                         float *heatmap, int32_t *argmax_yx,
                         void *ws, size_t ws_bytes, void *stream);

/* ---------------------------------------------------------------------------------
 * Soft-VQ heatmap (training path): the differentiable reading of Algorithm 1, Eq. 1 and
 * Eq. 2.  Every pixel is soft-assigned, p_j(x) = softmax_j(-||x - c_j||^2 / tau); the soft
 * counts of cell f of a G x G grid over the template window (floor boundaries, Sec. 3.2.1)
 * are the sums of p over the cell, T_fj for the template and Q_fj(y, x) for the query window
 * at (y, x); the heatmap is Eq. 2 with the L1 norm over clusters,
 *     heat[b][y][x] = - sum_f (wf[f] / A_f) sum_j | T_fj - Q_fj(b, y, x) |,
 * A_f the cell area, wf learnable.  All FP32.
 *   Qf    device, B x H x W x D float32 (HWC per query);  Tf: device, th x tw x D;
 *   C     device, k x D;  tau > 0;  1 <= G <= 4;  wf: device, G*G float32
 *   heat  device, B x (H - th + 1) x (W - tw + 1) float32, written
 *   ws    device workspace of vqnnf_soft_workspace_bytes() bytes, 256-byte aligned; it keeps
 *         the soft assignments, the template soft counts, the query cell sums and the
 *         per-filter L1 maps for the backward call with the same arguments.
 * Limits: k <= 128, D <= 512, k * D <= 32768, B * k <= 65535, H <= 65535, W <= 12288,
 * B * k * H < 2^31, B * k * H * W < 2^40 (else VQNNF_EUNSUPPORTED). */
size_t vqnnf_soft_workspace_bytes(int B, int H, int W, int D, int k, int th, int tw, int G);
vqnnf_status vqnnf_soft_forward(const float *Qf, int B, int H, int W, const float *Tf, int th, int tw,
                                int D, const float *C, int k, float tau, int G, const float *wf,
                                float *heat, void *ws, size_t ws_bytes, void *stream);

/* Gradients of L = sum heat * dheat after vqnnf_soft_forward with the same arguments and
 * workspace: dQf (B x H x W x D), dC (k x D: query and template soft assignments both
 * contribute) and dwf (G*G), all device float32, written.  |.| has subgradient sign(0) = 0;
 * dL/dT accumulates with float atomics, so the centroid gradient may differ in the last bits
 * between runs. */
vqnnf_status vqnnf_soft_backward(const float *Qf, int B, int H, int W, const float *Tf, int th,
                                 int tw, int D, const float *C, int k, float tau, int G,
                                 const float *wf, const float *dheat, float *dQf, float *dC,
                                 float *dwf, void *ws, size_t ws_bytes, void *stream);

/* Profiling aid (the paper has no counterpart).  After
 * vqnnf_set_kernel_events(op, start, stop) with op = VQNNF_OP_ASSIGN or VQNNF_OP_SCORE and
 * two CUDA event handles (cudaEvent_t, created and owned by the caller, timing enabled),
 * every later call of that operation records `start` on its stream immediately before it
 * enqueues its main kernel (the distance contraction of vqnnf_assign, the score kernel of
 * vqnnf_score) and `stop` immediately after, so that cudaEventElapsedTime(start, stop) is
 * that kernel's duration.  Two NULL handles switch it off.  The setting is process-wide
 * (guarded by a lock) and applies to calls enqueued after it; the events must stay alive
 * while set.  Returns VQNNF_EINVAL for another op or when only one handle is NULL. */
vqnnf_status vqnnf_set_kernel_events(int op, void *start_event, void *stop_event);

/* Human-readable name of a status code (static string). */
const char *vqnnf_status_str(vqnnf_status s);

/* Synchronises `stream`, then returns and clears the device error word of the current
 * device: VQNNF_OK, or VQNNF_ETIMEOUT when a bounded device wait gave up since the last
 * call. */
vqnnf_status vqnnf_last_device_error(void *stream);

/* Self-test of the failure detection above (the paper has no counterpart).  Enqueues on
 * `stream` one single-thread kernel that waits on an mbarrier which nothing completes.  It
 * uses the score kernels' bounded wait, but with a limit of `limit_cycles` SM cycles
 * (1 .. 4,000,000,000, the kernels' own limit; else VQNNF_EINVAL, nothing enqueued).  The wait
 * gives up, records VQNNF_ETIMEOUT in the device error word, and the kernel returns.  No copy
 * is issued, so nothing is left in flight and the context stays usable.  The next
 * vqnnf_last_device_error() on that stream returns VQNNF_ETIMEOUT and clears the word. */
#define VQNNF_WAIT_LIMIT_CYCLES 4000000000LL
vqnnf_status vqnnf_selftest_bounded_wait(long long limit_cycles, void *stream);

/* ABI version of this header (major * 100 + minor). */
int vqnnf_version(void);

/* ---------------------------------------------------------------- whole path, host buffers
 * One template-query pair end to end with the features in host memory: the template's
 * codebook (vqnnf_fit_codebook with `iters`, `seed`), both NNFs, the template's responses,
 * the query's integral image, Eq. 2 heatmap and maximum; results copied back to the host.
 * The copies overlap the compute: the template goes first and its side runs while the query
 * arrives in row bands, each assigned as soon as it has landed.
 *   X_host      host, H x W x D float32 (HWC); pinned memory lets the copies run asynchronously
 *   T_host      host, th x tw x D float32
 *   bank, F     host filter bank, as for vqnnf_score
 *   heat_host   host, (H - th + 1) x (W - tw + 1) float32, written; NULL = maximum only
 *   argmax_host host, 2 int32 (y, x), written
 *   ws          device workspace of vqnnf_match_host_workspace_bytes(...) bytes, 256-byte
 *               aligned: it holds the device copies of X and T and every intermediate
 *   stream      the copies run on it, and it is the stream to synchronise on: when it reaches
 *               the end of this call's work, the host results are written
 *   stream2     a second stream for the compute, or NULL (everything on `stream`, no overlap)
 * Enqueues only; the events it uses are created and released inside the call, so the call is
 * not graph-capturable.  Errors as for the calls it is made of. */
size_t vqnnf_match_host_workspace_bytes(int H, int W, int D, int k, int th, int tw, int F, vqnnf_prec prec);
vqnnf_status vqnnf_match_host(const float *X_host, int H, int W, int D, const float *T_host, int th, int tw,
                              int k, int iters, uint64_t seed, vqnnf_prec prec, const vqnnf_filter *bank, int F,
                              float *heat_host, int32_t *argmax_host, void *ws, size_t ws_bytes, void *stream,
                              void *stream2);

/* ---------------------------------------------------------------- batched matching
 * Many templates against many queries: the template side of the method (codebook, NNF and
 * filter responses, Sec. 3.1-3.2) is computed once per template and reused for every query,
 * the reuse that the similarity measure allows across images (Sec. 4).  Template j gets its
 * own codebook of k_j centroids (seeded initialisation with seed + j, `iters` Lloyd steps,
 * BF16 contraction), its NNF and the responses of the grid bank: the full window plus the
 * G x G cells of the window (boundaries floor(i * side / G)), w_f = 1, A_f the pixel count.
 * Every query i is quantised against every template's codebook (Algorithm 1).  Templates whose
 * codebooks, each padded to a multiple of 32 centroids, fit one tensor-core contraction
 * together (plan->group_cols columns, at most 8 codebooks) share it, so a query's features are
 * read once per group rather than once per template; each codebook keeps its own exact
 * labels (interval test and re-scoring as in vqnnf_assign).  Then every pair (i, j) gets the
 * integral image of its NNF, the Eq. 2 heatmap and its maximum, as vqnnf_score computes them.
 *   q       host array of nq >= 1 images: X device, H x W x D float32 (HWC), 16-byte aligned
 *   t       host array of nt >= 1 templates: T device, h x w x D float32, 16-byte aligned;
 *           1 <= k <= 256 and k <= h w;  every template fits every query (h <= H, w <= W)
 *   D       feature length, a multiple of 16;  G: 1 <= G <= 4, G <= h and G <= w
 *   plan    tile choices from vqnnf_batch_tune, or NULL for the defaults
 *   heat    host array of nq * nt device pointers, pair (i, j) at [i * nt + j], each a
 *           (H_i - h_j + 1) x (W_i - w_j + 1) float32 heatmap, written; or NULL for the
 *           maxima only
 *   argmax  device, nq * nt * 2 int32: (y, x) of each pair's best window, pair (i, j) at
 *           [2 (i * nt + j)]
 *   ws      device workspace of vqnnf_batch_workspace_bytes(q, nq, t, nt, D, G) bytes,
 *           256-byte aligned
 * The call only enqueues work (graph-capturable).  Inside it the template sides, and each
 * query's pairs, run in eight lanes at once: `stream` and seven streams that the library
 * creates on its first call on a device (with the events that fork and join them) and keeps
 * for the process.  Every lane starts after the work enqueued on `stream` before the call,
 * and `stream` waits for every lane before the call returns, so ordering on `stream` is as if
 * all work ran on it.  Make the first call on a device outside stream capture (it creates the
 * streams; if that fails every lane runs on `stream`); a device reset invalidates them.  The
 * workspace holds an integral-image area per lane and two sets of query labels, so that a
 * query's assignment runs beside the previous query's pairs.  Limits: nq * nt <= 65536,
 * n = H W < 2^31 (else VQNNF_EUNSUPPORTED). */
typedef struct vqnnf_image {
    const float *X;
    int32_t H, W;
} vqnnf_image;

typedef struct vqnnf_batch_template {
    const float *T;
    int32_t h, w, k;
} vqnnf_batch_template;

typedef struct vqnnf_batch_plan {
    int32_t group_cols;   /* 128 or 256: columns of one shared contraction                 */
    int32_t sf;           /* FP32 feature boxes in flight per SM: 0 (default) or 2, 4, 6, 8 */
    int32_t pf;           /* L2 prefetch distance in 64-feature chunks, -1 = default       */
    int32_t stationary;   /* 1: where D <= 256, a query's features are read once per tile for
                             all its groups (the tile's operand stays in tensor memory while
                             every group's centroids stream past); 0: one launch per group  */
} vqnnf_batch_plan;

size_t vqnnf_batch_workspace_bytes(const vqnnf_image *q, int nq, const vqnnf_batch_template *t, int nt,
                                   int D, int G);
vqnnf_status vqnnf_match_batch(const vqnnf_image *q, int nq, const vqnnf_batch_template *t, int nt, int D,
                               int iters, uint64_t seed, int G, const vqnnf_batch_plan *plan,
                               float *const *heat, int32_t *argmax_yx, void *ws, size_t ws_bytes,
                               void *stream);

/* Autotuner: fits the templates as vqnnf_match_batch does, then times the assignment of the
 * largest query under each candidate plan (stationary where D <= 256, and one launch per group
 * with group_cols in {128, 256} x feature boxes in {4, 6, 8} x prefetch in {0, 8}) with CUDA
 * events and writes the fastest to *plan.  It
 * SYNCHRONISES `stream` (not graph-capturable); the workspace is the batch workspace. */
vqnnf_status vqnnf_batch_tune(const vqnnf_image *q, int nq, const vqnnf_batch_template *t, int nt, int D,
                              int iters, uint64_t seed, int G, vqnnf_batch_plan *plan, void *ws,
                              size_t ws_bytes, void *stream);

#ifdef __cplusplus
}
#endif
#endif /* VQNNF_H */
