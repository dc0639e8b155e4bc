// Internal pieces of the call sequences shared by the C ABI translation units (api.cu, batch.cu):
// workspace layouts (the same code computes sizes with a null base), the assignment and
// codebook-fit sequences, and filter-bank compilation.
#pragma once

#include "common.cuh"
#include "score_spec.cuh"

namespace vqnnf {

struct AssignWs {
    CodebookPrep prep;
    FlagList fl;
    Fp8Feat f8;       // FP8 path only (null otherwise)
};

struct FitWs {
    AssignWs as;
    uint8_t *lab;
    LloydWs lw;
};

struct ScoreWs {
    void *S;          // integral image, uint16 (mod 2^16) or uint32, plus read slack
    bool u16;
    int *carry;
    int *bandsum;
    unsigned long long *amax;
};

cudaStream_t as_stream(void *s);
bool aligned(const void *p, size_t a);
vqnnf_status from_cuda(cudaError_t e);
bool check_prec(int prec, int D);
int device_smem_optin();

AssignWs carve_assign(WsCursor &c, long long n, int D, int k, int prec = VQNNF_PREC_FP32);
FitWs carve_fit(WsCursor &c, long long l, int D, int k, int prec = VQNNF_PREC_FP32);
ScoreWs carve_score(WsCursor &c, int H, int W, int k, int th, int tw);

// Enqueue the full assignment of n pixels (prep, contraction, re-scoring, stats).
// keep_mean: reuse the reference point of the previous call on w (the Lloyd steps after the first).
vqnnf_status run_assign(const float *X, long long n, int D, const float *C, int k, int prec,
                        uint8_t *labels, vqnnf_assign_stats *stats, AssignWs &w, cudaStream_t s,
                        bool keep_mean = false);
// Seeded initial centroids, then `iters` Lloyd steps.
vqnnf_status run_fit(const float *T, long long l, int D, int k, int iters, uint64_t seed, int prec,
                     float *C, FitWs &fw, cudaStream_t s);
// Host-side description of a filter bank for the score kernels (grid bank detected).
vqnnf_status compile_bank(const vqnnf_filter *bank, int F, int th, int tw, BankSpec &bs, GridSpec &gs);
void detect_wgrid(const vqnnf_filter *bank, int F, const BankSpec &bs, WGridSpec &ws);

}  // namespace vqnnf
