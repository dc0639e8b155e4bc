// Internal declarations shared by the library's translation units.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/vqnnf.h"

namespace vqnnf {

constexpr int kMaxK = 256;          // labels are uint8
constexpr int kMaskWords = kMaxK / 32;

// Per-centroid terms of the assignment error bound and the centred codebook, written by
// prep_codebook (assign_fp32.cu) into the workspace.
struct CodebookPrep {
    float *mean;      // D       reference point m (the FP32 codebook mean)
    float *cc;        // k x D   FP32 rounding of c_j - m
    uint16_t *chi;    // k x D   BF16 rounding of c_j - m              (BF16 path)
    uint16_t *clo;    // k x D   BF16 rounding of the remainder        (BF16 path)
    float *nrm;       // k       FP32 rounding of ||c_j - m||^2
    float *a;         // k       bound coefficient of ||x'||
    float *v;         // k       bound coefficient of the per-pixel rounding residual
    float *b;         // k       bound constant (error of nrm)
    uint8_t *cq8;     // k x D   FP8 e4m3 of (c_j - m) / s_j                 (FP8 path)
    float *csc;       // k       the power-of-two scale s_j                  (FP8 path)
};

// FP8 path: the features quantised per row (x - m = s_x q + residual, s_x a power of two).
struct Fp8Feat {
    uint8_t *q;       // n x D   FP8 e4m3 of (x - m) / s_x
    float2 *rs;       // n       (s_x, upper bound of ||fl(x - m)||)
};

// List of pixels whose contraction result is ambiguous, with their candidate sets.
struct FlagList {
    unsigned int *count;      // device counter
    unsigned int *pix;        // capacity entries
    unsigned int *mask;       // capacity x kMaskWords candidate bit sets
    unsigned long long *stats;  // [n_flagged, n_candidates, n_deep, reserved]
};

// One codebook among several side by side in the columns of one tensor-core contraction:
// columns [col0, col0 + ncol) of the prepared codebook, ncol a multiple of 32, the first k of
// them real centroids; its labels and its flag list (candidate masks relative to col0).
constexpr int kMaxSeg = 8;
constexpr int kMaxSegStat = 64;     // segments of one stationary launch (all its groups)
constexpr int kMaxGroupsStat = 63;  // groups of one stationary launch
struct TcSeg {
    int col0, ncol, k;
    uint8_t *labels;
    FlagList fl;
};

// Host-side launchers (defined in the .cu files).
// zero64: if not null, 64 words zeroed by the first kernel (a flag list's counter and statistics).
// keep_mean: the reference point p.mean is left as it is (set by an earlier call on the same
// workspace) instead of recomputed as the codebook mean; any fixed m keeps the bound valid.
cudaError_t launch_prep_codebook(const float *C, int k, int D, int prec, CodebookPrep p,
                                 cudaStream_t s, unsigned *zero64 = nullptr, bool keep_mean = false);
cudaError_t launch_assign_fp32(const float *X, long long n, int D, int k,
                               const CodebookPrep &p, uint8_t *labels, FlagList fl,
                               cudaStream_t s);
cudaError_t launch_assign_bf16(const float *X, long long n, int D, int k,
                               const CodebookPrep &p, uint8_t *labels, FlagList fl,
                               cudaStream_t s);
// FP8 e4m3 contraction (quantisation of the features into f8, then tcgen05 kind::f8f6f4).
bool fp8_supported(int D, int k);
cudaError_t launch_assign_fp8(const float *X, long long n, int D, int k, const CodebookPrep &p, Fp8Feat f8,
                              uint8_t *labels, FlagList fl, cudaStream_t s);
// Several codebooks in one contraction: p holds krows prepared rows (the segments' columns,
// padding rows included); the sum of the segments' ncol is at most 256.
cudaError_t launch_assign_bf16_seg(const float *X, long long n, int D, const CodebookPrep &p, int krows,
                                   const TcSeg *seg, int nseg, int sf, int pf, cudaStream_t s);
// Several groups of codebooks against one tile of features read once (the tile's BF16 operand
// stays in tensor memory while every group's centroids stream past): p holds ngroup * gcols
// prepared rows, group g at rows g * gcols; seg[] lists every group's segments with absolute
// columns (group g's segments are seg[gs0[g] .. gs0[g + 1]), inside [g * gcols, (g + 1) * gcols)).
// D <= 256; gcols <= 128 (double-buffered accumulators) or 256 (single).
cudaError_t launch_assign_bf16_stat(const float *X, long long n, int D, const CodebookPrep &p, int ngroup,
                                    int gcols, const TcSeg *seg, const int *gs0, cudaStream_t s);
// Largest number of groups of gcols columns one stationary launch holds (shared memory).
int stat_max_groups(int D, int gcols);
cudaError_t launch_rescore(const float *X, long long n, int D, const float *C, int k,
                           uint8_t *labels, FlagList fl, cudaStream_t s);
cudaError_t launch_finish_stats(FlagList fl, vqnnf_assign_stats *out, cudaStream_t s);

// Launch with programmatic stream serialization: the kernel's blocks may be scheduled before the
// preceding kernel of the stream finishes; every kernel launched this way calls ptx::pdl_enter()
// before it touches global memory, so the order of effects is the stream order.  The launch
// latency and the tail of the previous kernel overlap instead of adding up.
bool pdl_enabled();
template <typename... KArgs, typename... Args>
inline cudaError_t launch_pdl(void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t s,
                              Args... args)
{
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[0].val.programmaticStreamSerializationAllowed = 1;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cfg.attrs = at;
    cfg.numAttrs = pdl_enabled() ? 1 : 0;
    return cudaLaunchKernelEx(&cfg, kernel, static_cast<KArgs>(args)...);
}

// Records the caller's profiling event `which` (0 = start, 1 = stop) of operation `op` on s,
// when vqnnf_set_kernel_events has set one; otherwise does nothing.
cudaError_t record_kernel_event(int op, int which, cudaStream_t s);

// Device error word of the tensor-core translation unit (bounded waits).
cudaError_t read_and_clear_tc_error(int *out);

// Initial centroid indices of the k-means (kernel parameter).
struct InitIdx {
    int32_t idx[kMaxK];
};
cudaError_t launch_gather_init(const float *T, int D, int k, const InitIdx &ii, float *C,
                               cudaStream_t s);
// Lloyd update workspace (fit.cu).  The members of each cluster are cut into
// chunks of kLloydRows rows; a cluster of more than one chunk combines its chunks' exact partial
// sums (one LloydPart per chunk and dimension) in the block that finishes last.
constexpr int kLloydRows = 128;
constexpr int kLloydSortBlocks = 32;  // most blocks of the counting sort
struct __align__(16) LloydPart {
    unsigned __int128 pos, neg, mag;   // sums of the positive parts, negative parts; a bound of sum |x|
    int low, hish, bad, pad;           // lowest set bit, largest shift, a value outside the range
};
struct LloydWs {
    int *cnt, *off, *members;          // cluster sizes, first slots, member pixels (any order)
    int *ordered;                      // member pixels in pixel order (the in-order FP64 route only)
    int4 *chunks;                      // (first member slot, rows | cluster << 8, first chunk, size)
    int *bh;                           // per sort block and cluster: label counts
    double *rcp;                       // per cluster: 1 / size, correctly rounded
    int *done;                         // per (cluster, 32 dimensions): chunks finished
    LloydPart *part;                   // per (chunk, dimension) partial sums
};
inline long long lloyd_max_chunks(long long l, int k) { return (l + kLloydRows - 1) / kLloydRows + k; }
cudaError_t launch_lloyd_update(const float *T, int l, int D, int k, const uint8_t *lab, const LloydWs &lw,
                                float *C, cudaStream_t s);

}  // namespace vqnnf

// Bump allocator over a caller-provided workspace (256-byte alignment).
struct WsCursor {
    char *base;
    size_t off;
    template <typename T>
    T *take(size_t count) {
        off = (off + 255) & ~size_t(255);
        T *p = base ? reinterpret_cast<T *>(base + off) : nullptr;
        off += count * sizeof(T);
        return p;
    }
};
