// Nearest-neighbour field (Algorithm 1) on the tcgen05 tensor cores.
//
// The distance contraction s_j = ||c_j - m||^2 - 2 (x - m).(c_j - m) runs as BF16 x BF16
// UMMAs with FP32 accumulation in tensor memory.  Both sides are split into two BF16 planes
// (v = hi + lo + rest, hi = bf16(v), lo = bf16(v - hi)) and three products are accumulated
// into the same result: x_hi.c_hi + x_hi.c_lo + x_lo.c_hi, so the rounding left in the
// contraction is about 2^-16 relative instead of 2^-8.  The epilogue applies the same proven
// interval test as the FP32 path (assign_fp32.cu) and flags ambiguous pixels for the
// shared re-scoring stage, so labels stay exact.
//
// One persistent CTA per SM, 128-pixel tiles, warp-specialised (23 warps):
//   warp 0      TMA producer of the FP32 feature boxes (128 rows x 32 floats, 128B swizzle),
//               up to eight boxes in flight (an optional L2 prefetch further ahead is off by
//               default: it measured slower)
//   warp 22     TMA producer of the two BF16 centroid planes (k rows x 64 elements, 128B
//               swizzle); separate from warp 0 so that feature loads never wait for MMAs
//   warp 1      TMEM allocation; lane 0 issues tcgen05.mma and tcgen05.commit
//   warps 2-17  converters: warp w writes TMEM lane group w % 4 (pixel rows 32 (w % 4) ..)
//               and the 16-column quarter (w - 2) / 4 of every 64-column chunk; FP32 ->
//               centred BF16 hi and lo planes stored with tcgen05.st straight into tensor
//               memory, where the MMA reads its A operand (row r in lane r, two K elements per
//               32-bit column), so the pixel planes never pass through shared memory;
//               accumulates its part of ||x'||^2
//   warps 18-21 epilogue: tcgen05.ld of the row's accumulators, interval test, label, flag
//               push; the TMEM accumulator is double-buffered when k <= 128
// The columns may hold several codebooks side by side (segments, each padded to 32 columns,
// at most 256 columns in all): the contraction is shared and the epilogue takes each
// segment's nearest centroid, interval test, labels and flag list on its own.  One codebook
// is the single-segment case.
// Every mbarrier wait is bounded: on timeout the CTA records VQNNF_ETIMEOUT in the device
// error word, all roles leave their loops, in-flight copies and MMAs are drained (bounded)
// and the tensor memory is released before the kernel returns.
#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_fp8.h>
#include <cudaTypedefs.h>

#include <cfloat>
#include <cstring>
#include <mutex>

#include "common.cuh"
#include "ptx.cuh"

namespace vqnnf {
namespace {

__device__ int g_tc_error = 0;

constexpr int TM = 128;            // pixels per tile (UMMA M)
constexpr int KC = 64;             // K elements per chunk (128 bytes of BF16)
constexpr int kMaxSF = 8;          // FP32 staging slots, one 16 KB box (32 columns) each
constexpr int kMaxSB = 4;          // centroid stages (hi and lo planes of one 64-column chunk)
constexpr int kMaxSA = 4;          // BF16 A-operand stages (tensor memory, 64 columns each)
constexpr int NT = 736;            // 23 warps
constexpr int F32_BOX = TM * 32 * 4;       // 16 KB: 128 rows x 32 floats
constexpr double kU = 5.9604644775390625e-08;
constexpr long long kWaitCycles = 4000000000ll;   // ~2 s at 2 GHz
constexpr int PF = 0;              // chunks prefetched into L2 ahead of the loads (none: measured best)

struct TcArgs {
    long long n;
    int D, krows, npad, nkc, sb, sf, nb, sa, pf;   // krows: rows of the prepared codebook
    long long ntiles;
    CodebookPrep p;
    int nseg;
    TcSeg seg[kMaxSegStat];          // the single and multi modes use the first kMaxSeg
    int ngroup;                      // stationary mode: groups of npad columns
    int gs0[kMaxGroupsStat + 1];     // stationary mode: group g's segments are seg[gs0[g] .. gs0[g + 1])
};

// ------------------------------------------------------------------ PTX helpers
__device__ __forceinline__ uint32_t smem_u32(const void *p)
{
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ void mbar_init(uint64_t *b, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(b)), "r"(count));
}
__device__ __forceinline__ void mbar_arrive(uint64_t *b)
{
    asm volatile("{\n .reg .b64 st;\n mbarrier.arrive.shared::cta.b64 st, [%0];\n}" ::"r"(smem_u32(b))
                 : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t *b, uint32_t bytes)
{
    asm volatile("{\n .reg .b64 st;\n mbarrier.arrive.expect_tx.shared::cta.b64 st, [%0], %1;\n}" ::"r"(
                     smem_u32(b)),
                 "r"(bytes)
                 : "memory");
}
__device__ __forceinline__ bool mbar_try(uint64_t *b, uint32_t parity)
{
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
        : "=r"(ok)
        : "r"(smem_u32(b)), "r"(parity)
        : "memory");
    return ok != 0;
}
// Bounded wait: false when this CTA gave up (timeout here or abort raised elsewhere).
__device__ __forceinline__ bool mbar_wait(uint64_t *b, uint32_t parity, volatile int *abort)
{
    if (mbar_try(b, parity)) return true;
    const long long t0 = clock64();
    for (uint32_t i = 1;; ++i) {
        if (mbar_try(b, parity)) return true;
        if ((i & 63) == 0) {
            if (*abort) return false;
            if (clock64() - t0 > kWaitCycles) {
                *abort = 1;
                atomicExch(&g_tc_error, (int)VQNNF_ETIMEOUT);
                return false;
            }
        }
    }
}
__device__ __forceinline__ void fence_barrier_init()
{
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ void fence_proxy_async()
{
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}
__device__ __forceinline__ void tma_load_2d(void *dst, const CUtensorMap *map, int x, int y, uint64_t *bar)
{
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::"r"(
            smem_u32(dst)),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(smem_u32(bar))
        : "memory");
}
__device__ __forceinline__ void tma_prefetch_2d(const CUtensorMap *map, int x, int y)
{
    asm volatile("cp.async.bulk.prefetch.tensor.2d.L2.global [%0, {%1, %2}];" ::"l"(reinterpret_cast<uint64_t>(map)),
                 "r"(x), "r"(y)
                 : "memory");
}
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_commit(uint64_t *bar)
{
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
                 : "memory");
}
// D (+)= A . B^T with A (128 rows x 16 BF16) in tensor memory, B in shared memory.  ACC = false
// overwrites D.  The issuing thread feeds the tensor pipe one MMA per 64 cycles at N = 128, so
// the issue path is kept to the instruction itself.
template <bool ACC>
__device__ __forceinline__ void tc_mma_ts(uint32_t d_tmem, uint32_t a_tmem, uint64_t bdesc, uint32_t idesc)
{
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
        " tcgen05.mma.cta_group::1.kind::f16 [%0], [%1], %2, %3, p;\n}" ::"r"(d_tmem),
        "r"(a_tmem), "l"(bdesc), "r"(idesc), "n"(ACC ? 1 : 0)
        : "memory");
}
// One 64-column chunk: for each K step ks (A columns + 8 ks, B start field + 2 ks) the three
// products x_hi.c_hi, x_hi.c_lo, x_lo.c_hi (A hi plane at a_hi, lo plane at a_hi + 32; B lo
// plane blo_off descriptor units after the hi plane).  The first MMA overwrites D when acc == 0.
// In the same instruction stream the next chunk's two barriers are tested without blocking,
// so the test latency overlaps the MMAs; returns whether both phases had completed.
__device__ __forceinline__ uint32_t tc_mma_chunk(uint32_t d, uint32_t a_hi, uint64_t bh, uint64_t blo_off,
                                                 uint32_t idesc, uint32_t acc, uint32_t nbar_a, uint32_t npar_a,
                                                 uint32_t nbar_b, uint32_t npar_b)
{
    uint32_t ready;
    asm volatile(
        "{\n"
        " .reg .pred pa, pb, pacc, pt;\n"
        " .reg .b32 a1, a2, a3, l0, l1, l2, l3;\n"
        " .reg .b64 h1, h2, h3, o0, o1, o2, o3;\n"
        " mbarrier.test_wait.parity.shared::cta.b64 pa, [%7], %8;\n"
        " mbarrier.test_wait.parity.shared::cta.b64 pb, [%9], %10;\n"
        " setp.ne.b32 pacc, %6, 0;\n"
        " setp.eq.b32 pt, %6, %6;\n"
        " add.u32 a1, %1, 8;\n add.u32 a2, %1, 16;\n add.u32 a3, %1, 24;\n"
        " add.u32 l0, %1, 32;\n add.u32 l1, %1, 40;\n add.u32 l2, %1, 48;\n add.u32 l3, %1, 56;\n"
        " add.u64 h1, %3, 2;\n add.u64 h2, %3, 4;\n add.u64 h3, %3, 6;\n"
        " add.u64 o0, %3, %4;\n add.u64 o1, o0, 2;\n add.u64 o2, o0, 4;\n add.u64 o3, o0, 6;\n"
        " tcgen05.mma.cta_group::1.kind::f16 [%2], [%1], %3, %5, pacc;\n"
        " tcgen05.mma.cta_group::1.kind::f16 [%2], [%1], o0, %5, pt;\n"
        " tcgen05.mma.cta_group::1.kind::f16 [%2], [l0], %3, %5, pt;\n"
        " tcgen05.mma.cta_group::1.kind::f16 [%2], [a1], h1, %5, pt;\n"
        " tcgen05.mma.cta_group::1.kind::f16 [%2], [a1], o1, %5, pt;\n"
        " tcgen05.mma.cta_group::1.kind::f16 [%2], [l1], h1, %5, pt;\n"
        " tcgen05.mma.cta_group::1.kind::f16 [%2], [a2], h2, %5, pt;\n"
        " tcgen05.mma.cta_group::1.kind::f16 [%2], [a2], o2, %5, pt;\n"
        " tcgen05.mma.cta_group::1.kind::f16 [%2], [l2], h2, %5, pt;\n"
        " tcgen05.mma.cta_group::1.kind::f16 [%2], [a3], h3, %5, pt;\n"
        " tcgen05.mma.cta_group::1.kind::f16 [%2], [a3], o3, %5, pt;\n"
        " tcgen05.mma.cta_group::1.kind::f16 [%2], [l3], h3, %5, pt;\n"
        " and.pred pa, pa, pb;\n"
        " selp.u32 %0, 1, 0, pa;\n"
        "}"
        : "=r"(ready)
        : "r"(a_hi), "r"(d), "l"(bh), "l"(blo_off), "r"(idesc), "r"(acc), "r"(nbar_a), "r"(npar_a), "r"(nbar_b),
          "r"(npar_b)
        : "memory");
    return ready;
}
// 8 consecutive 32-bit columns of this thread's TMEM lane.
__device__ __forceinline__ void tc_st8(uint32_t taddr, const uint32_t *v)
{
    asm volatile("tcgen05.st.sync.aligned.32x32b.x8.b32 [%0], {%1, %2, %3, %4, %5, %6, %7, %8};" ::"r"(taddr),
                 "r"(v[0]), "r"(v[1]), "r"(v[2]), "r"(v[3]), "r"(v[4]), "r"(v[5]), "r"(v[6]), "r"(v[7])
                 : "memory");
}
__device__ __forceinline__ void tc_wait_st() { asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory"); }
// 32 consecutive FP32 accumulator columns of this thread's TMEM lane.
__device__ __forceinline__ void tc_ld32(uint32_t taddr, float *v)
{
    uint32_t r[32];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, "
        "%14, %15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]),
          "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]),
          "=r"(r[22]), "=r"(r[23]), "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]),
          "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int i = 0; i < 32; ++i) v[i] = __uint_as_float(r[i]);
}

// UMMA shared-memory descriptor: K-major operand, 128-byte swizzle, 8-row atoms 1 KB apart.
__device__ __forceinline__ uint64_t sw128_desc(uint32_t saddr)
{
    uint64_t d = 0;
    d |= (uint64_t)((saddr >> 4) & 0x3FFF);
    d |= (uint64_t)1 << 16;                   // leading byte offset (unused for this layout)
    d |= (uint64_t)(1024 >> 4) << 32;          // stride byte offset: next 8-row group
    d |= (uint64_t)1 << 46;                    // descriptor version
    d |= (uint64_t)2 << 61;                    // 128-byte swizzle
    return d;
}
// Instruction descriptor: BF16 x BF16 -> F32, both K-major, M = 128, N = npad.
__host__ __device__ constexpr uint32_t bf16_idesc(int M, int N)
{
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ uint32_t pack_bf16(float a, float b, float &ra, float &rb)
{
    const __nv_bfloat162 h = __floats2bfloat162_rn(a, b);   // a -> low half
    ra = __low2float(h);
    rb = __high2float(h);
    return *reinterpret_cast<const uint32_t *>(&h);
}

// ------------------------------------------------------------------ the kernel
// MULTI: several codebook segments (batching); the single-codebook instantiation keeps the
// segment's bounds and bound maxima out of the tile loop.  STAT (with MULTI): several groups
// of npad columns per tile; the tile's A stages (all nkc chunks) stay in tensor memory until
// the last group's MMAs, and every group's centroid chunks stream through the B stages.
template <bool MULTI, bool STAT>
__global__ void __launch_bounds__(NT, 1) assign_tc_kernel(const __grid_constant__ CUtensorMap tmA,
                                                          const __grid_constant__ CUtensorMap tmBhi,
                                                          const __grid_constant__ CUtensorMap tmBlo,
                                                          const __grid_constant__ TcArgs g)
{
    ptx::pdl_enter();
    extern __shared__ uint8_t smem_raw[];
    uint8_t *base = reinterpret_cast<uint8_t *>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
    const int npad = g.npad, D = g.D, nkc = g.nkc, SB = g.sb, SF = g.sf, NB = g.nb, SA = g.sa;
    const int B_PLANE = npad * 128;
    const int ngroup = STAT ? g.ngroup : 1;
    const int ncols = ngroup * npad;                       // prepared columns of this launch
    const int nsegcap = STAT ? kMaxSegStat : kMaxSeg;
    uint8_t *f32s = base;                                  // SF x 16 KB
    uint8_t *bs = f32s + SF * F32_BOX;                     // SB x (hi, lo)
    // per column {||c*||^2, a, v, b}; cn[c * CS] = ||c*||^2 (the stationary mode keeps no
    // separate copy of it, to leave shared memory for centroid stages)
    constexpr int CS = STAT ? 4 : 1;
    float *cn0 = reinterpret_cast<float *>(bs + SB * 2 * B_PLANE);
    float4 *colc = reinterpret_cast<float4 *>(cn0 + (STAT ? 0 : ncols));
    const float *cn = STAT ? reinterpret_cast<const float *>(colc) : cn0;
    float *mean = reinterpret_cast<float *>(colc + ncols); // roundup(D, 64)
    float *norms = mean + nkc * KC;                        // [2 buf][4 quarters][128]
    uint32_t *maskbuf = reinterpret_cast<uint32_t *>(norms + 2 * 4 * TM);   // [128][8]
    float4 *segmx = reinterpret_cast<float4 *>(maskbuf + TM * kMaskWords);   // per segment maxima
    TcSeg *segt = reinterpret_cast<TcSeg *>(segmx + nsegcap);                // segment table
    uint64_t *bar = reinterpret_cast<uint64_t *>(segt + nsegcap);
    uint64_t *full_f = bar, *empty_f = bar + SF, *a_full = bar + 2 * SF, *a_empty = bar + 2 * SF + SA;
    uint64_t *full_b = bar + 2 * SF + 2 * SA, *empty_b = full_b + kMaxSB;
    uint64_t *acc_full = empty_b + kMaxSB, *acc_empty = acc_full + 2, *nrm_full = acc_empty + 2,
             *nrm_empty = nrm_full + 2, *drain = nrm_empty + 2;
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(drain + 1);
    volatile int *abort = reinterpret_cast<volatile int *>(tmem_slot + 1);

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    // tensor memory: NB accumulator buffers of npad columns, then SA A-operand stages of 64
    // columns (32 for the hi plane, 32 for the lo plane: two BF16 per 32-bit column)
    const int a_col0 = NB * npad;
    const int need = a_col0 + SA * 64;
    const uint32_t tmem_cols = need <= 32 ? 32 : need <= 64 ? 64 : need <= 128 ? 128 : need <= 256 ? 256 : 512;

    for (int j = tid; j < ncols; j += NT) {
        bool ok = false;                                  // a real centroid of some segment
        if constexpr (STAT) {
            const int gi = j / npad;
            for (int q = g.gs0[gi]; q < g.gs0[gi + 1]; ++q)
                ok |= j >= g.seg[q].col0 && j < g.seg[q].col0 + g.seg[q].k;
        } else {
#pragma unroll
            for (int q = 0; q < kMaxSeg; ++q)
                ok |= q < g.nseg && j >= g.seg[q].col0 && j < g.seg[q].col0 + g.seg[q].k;
        }
        const int jc = j < g.krows ? j : g.krows - 1;
        const float nrm = ok ? g.p.nrm[jc] : FLT_MAX;     // padding columns never win nor qualify
        if constexpr (!STAT) cn0[j] = nrm;
        colc[j] = make_float4(nrm, ok ? g.p.a[jc] : 0.f, ok ? g.p.v[jc] : 0.f, ok ? g.p.b[jc] : 0.f);
    }
    // segment table
    if constexpr (STAT) {
        for (int q = tid; q < g.nseg; q += NT) segt[q] = g.seg[q];
    } else {
#pragma unroll
        for (int q = 0; q < kMaxSeg; ++q)
            if (tid == q && q < g.nseg) segt[q] = g.seg[q];
    }
    for (int i = tid; i < nkc * KC; i += NT) mean[i] = g.p.mean[i < D ? i : D - 1];
    if (tid == 0) {
        for (int s = 0; s < SF; ++s) { mbar_init(&full_f[s], 1); mbar_init(&empty_f[s], 2 * TM); }
        for (int s = 0; s < SA; ++s) { mbar_init(&a_full[s], 4 * TM); mbar_init(&a_empty[s], 1); }
        for (int s = 0; s < SB; ++s) { mbar_init(&full_b[s], 1); mbar_init(&empty_b[s], 1); }
        for (int s = 0; s < 2; ++s) {
            mbar_init(&acc_full[s], 1); mbar_init(&acc_empty[s], TM);
            mbar_init(&nrm_full[s], 4 * TM); mbar_init(&nrm_empty[s], TM);
        }
        mbar_init(drain, 1);
        *abort = 0;
        fence_barrier_init();
        fence_proxy_async();
    }
    if (warp == 1) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                     "r"(tmem_cols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem_base = *tmem_slot;

    if (warp == 0) {
        // ---------------------------------------------------------- feature producer
        if (lane == 0) {
            uint32_t ib = 0, fs = 0, fp = 0;                  // box counter, its slot and phase parity
            bool ok = true;
            long long last[kMaxSF];
            for (int q = 0; q < kMaxSF; ++q) last[q] = -1;
            // optional L2 prefetch, g.pf chunks ahead of the shared-memory loads
            long long pf_tile = blockIdx.x;
            int pf_kc = 0;
            auto prefetch_next = [&]() {
                if (pf_tile >= g.ntiles) return;
                tma_prefetch_2d(&tmA, pf_kc * KC, (int)(pf_tile * TM));
                tma_prefetch_2d(&tmA, pf_kc * KC + 32, (int)(pf_tile * TM));
                if (++pf_kc == nkc) { pf_kc = 0; pf_tile += gridDim.x; }
            };
            for (int q = 0; q < g.pf; ++q) prefetch_next();
            for (long long tile = blockIdx.x; ok && tile < g.ntiles; tile += gridDim.x) {
                for (int kc = 0; ok && kc < nkc; ++kc) {
                    if (g.pf) prefetch_next();
                    for (int h = 0; h < 2; ++h, ++ib) {
                        if (!(ok = mbar_wait(&empty_f[fs], fp ^ 1, abort))) break;
                        mbar_expect_tx(&full_f[fs], F32_BOX);
                        tma_load_2d(f32s + fs * F32_BOX, &tmA, kc * KC + 32 * h, (int)(tile * TM), &full_f[fs]);
                        last[fs] = ib;
                        if (++fs == SF) { fs = 0; fp ^= 1; }
                    }
                }
            }
            if (!ok) {
                // drain: wait (bounded) for every copy this thread issued to land
                volatile int no_abort = 0;
                for (int q = 0; q < SF; ++q)
                    if (last[q] >= 0) mbar_wait(&full_f[q], (uint32_t)((last[q] / SF) & 1), &no_abort);
            }
        }
    } else if (warp == 22) {
        // ---------------------------------------------------------- centroid producer
        if (lane == 0) {
            uint32_t itb = 0, sb = 0, pb = 0;
            bool ok = true;
            long long last_b[kMaxSB] = {-1, -1, -1, -1};
            for (long long tile = blockIdx.x; ok && tile < g.ntiles; tile += gridDim.x) {
                for (int gi = 0; ok && gi < ngroup; ++gi) {      // one group unless stationary
                    for (int kc = 0; kc < nkc; ++kc, ++itb) {
                        if (!(ok = mbar_wait(&empty_b[sb], pb ^ 1, abort))) break;
                        mbar_expect_tx(&full_b[sb], 2 * B_PLANE);
                        uint8_t *bd = bs + sb * 2 * B_PLANE;
                        tma_load_2d(bd, &tmBhi, kc * KC, gi * npad, &full_b[sb]);
                        tma_load_2d(bd + B_PLANE, &tmBlo, kc * KC, gi * npad, &full_b[sb]);
                        last_b[sb] = itb;
                        if (++sb == (uint32_t)SB) { sb = 0; pb ^= 1; }
                    }
                }
            }
            if (!ok) {
                volatile int no_abort = 0;
                for (int q = 0; q < SB; ++q)
                    if (last_b[q] >= 0) mbar_wait(&full_b[q], (uint32_t)((last_b[q] / SB) & 1), &no_abort);
            }
        }
    } else if (warp == 1) {
        // ---------------------------------------------------------- MMA issuer
        if (lane == 0) {
            const uint32_t idesc = bf16_idesc(TM, npad);
            const uint32_t a_base = tmem_base + a_col0;
            const uint64_t bdesc0 = sw128_desc(smem_u32(bs)), bstep = (uint64_t)((2 * B_PLANE) >> 4);
            const uint64_t blo_off = (uint64_t)(B_PLANE >> 4);
            uint32_t sa = 0, pa = 0, sb = 0, pb = 0, tl = 0;   // stage indices and phase parities
            uint32_t ready = 0;                                // this chunk's barriers seen complete
            bool ok = true;
            if constexpr (STAT) {
                // SA == nkc: chunk kc of every tile sits in A stage kc; each tile's stages are
                // released after the last group's MMAs.  gl counts (tile, group) pairs for the
                // accumulator buffers.
                uint32_t gl = 0;
                for (long long tile = blockIdx.x; ok && tile < g.ntiles; tile += gridDim.x) {
                    for (int gi = 0; ok && gi < ngroup; ++gi, ++gl) {
                        const uint32_t buf = gl % NB;
                        if (!(ok = mbar_wait(&acc_empty[buf], ((gl / NB) & 1) ^ 1, abort))) break;
                        tc_fence_after();
                        const uint32_t d_tmem = tmem_base + buf * npad;
                        for (int kc = 0; kc < nkc; ++kc) {
                            if (gi == 0 && !(ok = mbar_wait(&a_full[kc], pa, abort))) break;
                            if (!(ok = mbar_wait(&full_b[sb], pb, abort))) break;
                            tc_fence_after();
                            const uint32_t nsb = sb + 1 == (uint32_t)SB ? 0 : sb + 1, npb = nsb ? pb : pb ^ 1;
                            tc_mma_chunk(d_tmem, a_base + kc * 64, bdesc0 + (uint64_t)sb * bstep, blo_off, idesc,
                                         kc != 0, smem_u32(&full_b[nsb]), npb, smem_u32(&full_b[nsb]), npb);
                            tc_commit(&empty_b[sb]);
                            if (gi == ngroup - 1) tc_commit(&a_empty[kc]);
                            sb = nsb; pb = npb;
                        }
                        if (ok) tc_commit(&acc_full[buf]);
                    }
                    pa ^= 1;
                }
            }
            for (long long tile = blockIdx.x; !STAT && ok && tile < g.ntiles; tile += gridDim.x, ++tl) {
                const uint32_t buf = tl % NB;
                if (!(ok = mbar_wait(&acc_empty[buf], ((tl / NB) & 1) ^ 1, abort))) break;
                tc_fence_after();
                const uint32_t d_tmem = tmem_base + buf * npad;
                for (int kc = 0; kc < nkc; ++kc) {
                    if (!ready) {
                        if (!(ok = mbar_wait(&a_full[sa], pa, abort))) break;
                        if (!(ok = mbar_wait(&full_b[sb], pb, abort))) break;
                    }
                    tc_fence_after();
                    const uint32_t nsa = sa + 1 == (uint32_t)SA ? 0 : sa + 1, npa = nsa ? pa : pa ^ 1;
                    const uint32_t nsb = sb + 1 == (uint32_t)SB ? 0 : sb + 1, npb = nsb ? pb : pb ^ 1;
                    ready = tc_mma_chunk(d_tmem, a_base + sa * 64, bdesc0 + (uint64_t)sb * bstep, blo_off, idesc,
                                         kc != 0, smem_u32(&a_full[nsa]), npa, smem_u32(&full_b[nsb]), npb);
                    tc_commit(&a_empty[sa]);
                    tc_commit(&empty_b[sb]);
                    sa = nsa; pa = npa; sb = nsb; pb = npb;
                }
                if (ok) tc_commit(&acc_full[buf]);
            }
            // drain every MMA issued before the tensor memory is released
            tc_commit(drain);
            volatile int no_abort = 0;
            mbar_wait(drain, 0, &no_abort);
        }
    } else if (warp >= 2 && warp < 18) {
        // ---------------------------------------------------------- converters
        const int grp = warp & 3;                 // TMEM lane group this warp may write
        const int r = grp * 32 + lane;            // pixel row of the tile
        const int qt = (warp - 2) >> 2;           // 16-column quarter of each chunk this thread converts
        const int h = qt >> 1;                    // its 32-column box
        const int sw = r & 7;
        const uint32_t lane_base = tmem_base + ((uint32_t)(grp * 32) << 16);
        // A stage and its parity; this thread's box is number 2 it + h of the feature producer,
        // so its slot advances by two per chunk
        uint32_t sa = 0, pa = 0, sf = h, pf = 0, tl = 0;
        bool ok = true;
        for (long long tile = blockIdx.x; ok && tile < g.ntiles; tile += gridDim.x, ++tl) {
            const uint32_t nb = tl & 1;
            float2 x2 = make_float2(0.f, 0.f);              // partial ||x'||^2 of this quarter (even, odd columns)
            for (int kc = 0; kc < nkc; ++kc) {
                ok = __all_sync(0xffffffffu, mbar_wait(&a_empty[sa], pa ^ 1, abort));
                ok = __all_sync(0xffffffffu, ok && mbar_wait(&full_f[sf], pf, abort));
                if (!ok) break;
                tc_fence_after();
                const uint8_t *box = f32s + sf * F32_BOX + r * 128;
                // the quarter's 16 floats of row r (two 8-column groups of the 128B-swizzled box)
                float4 v[4];
#pragma unroll
                for (int cc = 0; cc < 2; ++cc) {
                    const int cb = 2 * (qt & 1) + cc;
                    v[2 * cc] = *reinterpret_cast<const float4 *>(box + (((2 * cb) ^ sw) << 4));
                    v[2 * cc + 1] = *reinterpret_cast<const float4 *>(box + (((2 * cb + 1) ^ sw) << 4));
                }
                uint32_t hw[8], lw[8];
#pragma unroll
                for (int cc = 0; cc < 2; ++cc) {
                    const int d0 = kc * KC + 16 * qt + 8 * cc;
                    if (d0 < D) {                            // D % 16 == 0: all 8 columns valid
                        const float4 m0 = *reinterpret_cast<const float4 *>(mean + d0);
                        const float4 m1 = *reinterpret_cast<const float4 *>(mean + d0 + 4);
                        const float4 v0 = v[2 * cc], v1 = v[2 * cc + 1];
                        // pairs of columns on the packed FP32 lanes, each rounded as the scalar
                        // operation: x' = fma(m, -1, x) = fl(x - m), the residual x' - hi (exact)
                        // and the norm's FMA
                        const float2 xv[4] = {make_float2(v0.x, v0.y), make_float2(v0.z, v0.w),
                                              make_float2(v1.x, v1.y), make_float2(v1.z, v1.w)};
                        const float2 mv[4] = {make_float2(m0.x, m0.y), make_float2(m0.z, m0.w),
                                              make_float2(m1.x, m1.y), make_float2(m1.z, m1.w)};
                        const float2 neg1 = make_float2(-1.f, -1.f);
#pragma unroll
                        for (int q = 0; q < 4; ++q) {
                            const float2 xs = __ffma2_rn(mv[q], neg1, xv[q]);
                            float ha, hb, la, lb;
                            hw[4 * cc + q] = pack_bf16(xs.x, xs.y, ha, hb);
                            x2 = __ffma2_rn(xs, xs, x2);
                            const float2 rs = __ffma2_rn(make_float2(ha, hb), neg1, xs);
                            lw[4 * cc + q] = pack_bf16(rs.x, rs.y, la, lb);   // exact residuals
                        }
                    } else {
#pragma unroll
                        for (int q = 0; q < 4; ++q) hw[4 * cc + q] = lw[4 * cc + q] = 0u;
                    }
                }
                // the box is released only once its values have been consumed: an arrive issued
                // right after the shared-memory loads let the next TMA copy overwrite the box
                // before those loads had returned (wrong labels at full size)
                mbar_arrive(&empty_f[sf]);
                const uint32_t col = lane_base + a_col0 + sa * 64 + 8 * qt;
                tc_st8(col, hw);
                tc_st8(col + 32, lw);
                tc_wait_st();
                tc_fence_before();
                mbar_arrive(&a_full[sa]);
                if (++sa == (uint32_t)SA) { sa = 0; pa ^= 1; }
                sf += 2;
                if (sf >= (uint32_t)SF) { sf -= SF; pf ^= 1; }
            }
            if (!ok) break;
            ok = __all_sync(0xffffffffu, mbar_wait(&nrm_empty[nb], ((tl >> 1) & 1) ^ 1, abort));
            if (!ok) break;
            norms[(nb * 4 + qt) * TM + r] = x2.x + x2.y;
            mbar_arrive(&nrm_full[nb]);
        }
    } else if (warp >= 18 && warp < 22) {
        // ---------------------------------------------------------- epilogue
        const int grp = warp & 3;                 // TMEM lane group this warp may read
        const int r = grp * 32 + lane;
        const float u = (float)kU;
        const float u4 = 4.0f * u;
        const float infl = 1.0f + 0.00390625f;
        const int nseg = MULTI ? g.nseg : 1;
        // per segment the largest ||c_j*||^2, a_j, v_j and b_j over its centroids (lanes of the
        // first epilogue warp scan the segments): Bmax below bounds every B_j of a pixel within
        // the segment
        if (warp == 18) {
            for (int q = lane; q < nseg; q += 32) {
                float nm = 0.f, am = 0.f, vm = 0.f, bm = 0.f;
                for (int j = segt[q].col0; j < segt[q].col0 + segt[q].k; ++j) {
                    const float4 c = colc[j];
                    nm = fmaxf(nm, c.x);
                    am = fmaxf(am, c.y);
                    vm = fmaxf(vm, c.z);
                    bm = fmaxf(bm, c.w);
                }
                segmx[q] = make_float4(nm, am, vm, bm);
            }
        }
        asm volatile("bar.sync 1, 128;" ::: "memory");       // the four epilogue warps
        // one codebook: its bound maxima and output pointers are loop invariants
        const float4 mx0 = segmx[0];
        const float cnorm0 = sqrtf(mx0.x) * 1.0001f, nrm0 = mx0.x * 1.0001f;
        uint8_t *const labels0 = g.seg[0].labels;
        const FlagList fl0 = g.seg[0].fl;
        // One segment of this tile: prepared columns [cb, ce), whose accumulators sit at TMEM
        // column c - cshift of taddr; `release` frees the accumulator buffer after its last read.
        auto segment = [&](int sgi, uint32_t taddr, int cshift, float X, float Y, float nx, long long pix,
                           bool valid, bool release, uint32_t buf) {
            const int cb = MULTI ? segt[sgi].col0 : 0, ce = MULTI ? cb + segt[sgi].ncol : npad;
            const float4 mx = MULTI ? segmx[sgi] : mx0;
            // max ||c_j*|| (cn = ||c*||^2 in FP32) and max ||c_j*||^2, with margins
            const float cnorm_max = MULTI ? sqrtf(mx.x) * 1.0001f : cnorm0;
            const float nrm_max = MULTI ? mx.x * 1.0001f : nrm0;
            int cnt = 0, last = 0, amin = cb;
            if (STAT && ce - cb == 32) {
                // a one-block segment (k <= 32): both passes read the same registers, one
                // tensor-memory load instead of two
                float v[32];
                tc_ld32(taddr + (uint32_t)(cb - cshift), v);
                float sm[4] = {FLT_MAX, FLT_MAX, FLT_MAX, FLT_MAX};
                int am[4] = {cb, cb, cb, cb};
#pragma unroll
                for (int j = 0; j < 32; ++j) {
                    const float sc = fmaf(-2.0f, v[j], cn[(cb + j) * CS]);
                    if (sc < sm[j & 3]) { sm[j & 3] = sc; am[j & 3] = cb + j; }
                }
                float smin = sm[0];
                amin = am[0];
#pragma unroll
                for (int q = 1; q < 4; ++q)
                    if (sm[q] < smin || (sm[q] == smin && am[q] < amin)) { smin = sm[q]; amin = am[q]; }
                const float4 ca = colc[amin];
                const float U = smin + fmaf(X, ca.y, fmaf(Y, ca.z, fmaf(u4, fabsf(smin), ca.w))) * infl;
                const float smax_abs = fmaf(2.0f * nx * 1.02f, cnorm_max, nrm_max) + 1.0f;
                const float Bmax = fmaf(X, mx.y, fmaf(Y, mx.z, fmaf(u4, smax_abs, mx.w))) * infl;
                const float lim = U + 2.0f * Bmax;
                uint32_t maybe = 0;
#pragma unroll
                for (int j = 0; j < 32; ++j) maybe |= (uint32_t)(fmaf(-2.0f, v[j], cn[(cb + j) * CS]) <= lim) << j;
                const uint32_t own = 1u << (amin & 31);
                uint32_t word = own;
                if (__any_sync(0xffffffffu, (maybe & ~own) != 0u)) {
                    word = 0;
#pragma unroll
                    for (int j = 0; j < 32; ++j) {
                        const float4 c = colc[cb + j];
                        const float sc = fmaf(-2.0f, v[j], c.x);
                        const float B = fmaf(X, c.y, fmaf(Y, c.z, fmaf(u4, fabsf(sc), c.w))) * infl;
                        word |= (uint32_t)(sc - B <= U) << j;
                    }
                }
                cnt = __popc(word);
                last = word ? cb + 31 - __clz(word) : amin;
                maskbuf[r * kMaskWords] = word;
            } else {
                // pass 1: smallest score of the segment, lowest column on ties, as four
                // interleaved running minima.  Padding columns hold +inf in cn (never chosen).
                float sm[4] = {FLT_MAX, FLT_MAX, FLT_MAX, FLT_MAX};
                int am[4] = {cb, cb, cb, cb};
                for (int c0 = cb; c0 < ce; c0 += 32) {
                    float v[32];
                    tc_ld32(taddr + (uint32_t)(c0 - cshift), v);
#pragma unroll
                    for (int j = 0; j < 32; ++j) {
                        const float sc = fmaf(-2.0f, v[j], cn[(c0 + j) * CS]);
                        if (sc < sm[j & 3]) { sm[j & 3] = sc; am[j & 3] = c0 + j; }
                    }
                }
                float smin = sm[0];
                amin = am[0];
#pragma unroll
                for (int q = 1; q < 4; ++q)
                    if (sm[q] < smin || (sm[q] == smin && am[q] < amin)) { smin = sm[q]; amin = am[q]; }
                // U, the upper end of column amin's interval, bounds the smallest distance from
                // above, so the nearest column j has s_j - B_j <= U.
                const float4 ca = colc[amin];
                const float U = smin + fmaf(X, ca.y, fmaf(Y, ca.z, fmaf(u4, fabsf(smin), ca.w))) * infl;
                // |s_j| <= ||c_j*||^2 + 2 ||x'|| ||c_j*|| (1 + 2^-6) + 1, with margin for the
                // contraction's own error, so Bmax >= every B_j of this pixel in the segment (the
                // float evaluation is monotone).  The nearest column has s_j <= U + B_j <= U + Bmax;
                // the limit U + 2 Bmax also covers the rounding of that sum (u |U| < Bmax / 2
                // because Bmax >= 4u |smin|).  A 32-column block where no lane has a column under
                // the limit besides amin needs no per-column interval test: its only candidate is
                // amin.
                const float smax_abs = fmaf(2.0f * nx * 1.02f, cnorm_max, nrm_max) + 1.0f;
                const float Bmax = fmaf(X, mx.y, fmaf(Y, mx.z, fmaf(u4, smax_abs, mx.w))) * infl;
                const float lim = U + 2.0f * Bmax;
                last = amin;
                for (int c0 = cb; c0 < ce; c0 += 32) {
                    float v[32];
                    tc_ld32(taddr + (uint32_t)(c0 - cshift), v);
                    uint32_t maybe = 0;
#pragma unroll
                    for (int j = 0; j < 32; ++j) maybe |= (uint32_t)(fmaf(-2.0f, v[j], cn[(c0 + j) * CS]) <= lim) << j;
                    const uint32_t own = (amin >> 5) == (c0 >> 5) ? 1u << (amin & 31) : 0u;
                    uint32_t word = own;
                    if (__any_sync(0xffffffffu, (maybe & ~own) != 0u)) {
                        word = 0;
#pragma unroll
                        for (int j = 0; j < 32; ++j) {
                            const float4 c = colc[c0 + j];
                            const float sc = fmaf(-2.0f, v[j], c.x);
                            const float B = fmaf(X, c.y, fmaf(Y, c.z, fmaf(u4, fabsf(sc), c.w))) * infl;
                            word |= (uint32_t)(sc - B <= U) << j;
                        }
                    }
                    cnt += __popc(word);
                    if (word) last = c0 + 31 - __clz(word);
                    maskbuf[r * kMaskWords + ((c0 - cb) >> 5)] = word;
                }
            }
            for (int w = (ce - cb) >> 5; w < kMaskWords; ++w) maskbuf[r * kMaskWords + w] = 0u;
            if (release) {                               // every accumulator of the buffer read
                tc_fence_before();
                mbar_arrive(&acc_empty[buf]);
            }
            uint8_t *const labels = MULTI ? segt[sgi].labels : labels0;
            const FlagList fl = MULTI ? segt[sgi].fl : fl0;
            const int lab = (cnt == 1 ? last : amin) - cb;
            if (valid) labels[pix] = (uint8_t)lab;
            const bool flagged = valid && cnt > 1;
            const unsigned ballot = __ballot_sync(0xffffffffu, flagged);
            if (ballot) {
                const int leader = __ffs(ballot) - 1;
                unsigned basei = 0;
                if (lane == leader) basei = atomicAdd(fl.count, (unsigned)__popc(ballot));
                basei = __shfl_sync(0xffffffffu, basei, leader);
                if (flagged) {
                    const unsigned slot = basei + __popc(ballot & ((1u << lane) - 1u));
                    if (slot < (unsigned long long)g.n) {
                        fl.pix[slot] = (unsigned)pix;
#pragma unroll
                        for (int w = 0; w < kMaskWords; ++w)
                            fl.mask[(size_t)slot * kMaskWords + w] = maskbuf[r * kMaskWords + w];
                    }
                }
            }
        };
        uint32_t tl = 0, gl = 0;
        bool ok = true;
        for (long long tile = blockIdx.x; ok && tile < g.ntiles; tile += gridDim.x, ++tl) {
            const uint32_t nb = tl & 1, nph = (tl >> 1) & 1;
            if constexpr (!STAT) {
                const uint32_t buf = tl % NB, ph = (tl / NB) & 1;
                ok = mbar_wait(&acc_full[buf], ph, abort);
                ok = __all_sync(0xffffffffu, ok && mbar_wait(&nrm_full[nb], nph, abort));
            } else {
                ok = __all_sync(0xffffffffu, mbar_wait(&nrm_full[nb], nph, abort));
            }
            if (!ok) break;
            tc_fence_after();
            // ||x_hi|| <= (1 + 2^-8) ||x'||  and  ||x' - x_hi - x_lo|| <= 2^-16 ||x'||  (two
            // round-to-nearest BF16 roundings, each within 2^-8 relative)
            const float x2 = (norms[(nb * 4 + 0) * TM + r] + norms[(nb * 4 + 1) * TM + r]) +
                             (norms[(nb * 4 + 2) * TM + r] + norms[(nb * 4 + 3) * TM + r]);
            const float nx = sqrtf(x2) * (1.0f + (float)(D + 8) * u);
            const float X = nx * (1.0f + 0.00390625f);
            const float Dl = nx * 1.5318e-05f + 1e-30f;      // 2^-16 * 1.004
            mbar_arrive(&nrm_empty[nb]);
            const float Y = Dl + u * (X * 1.01f + Dl) * (1.0f + 4.0f * u);
            const long long pix = tile * TM + r;
            const bool valid = pix < g.n;
            const uint32_t lanes = tmem_base + ((uint32_t)(grp * 32) << 16);
            if constexpr (!STAT) {
                const uint32_t buf = tl % NB;
                for (int sgi = 0; sgi < nseg; ++sgi)
                    segment(sgi, lanes + buf * npad, 0, X, Y, nx, pix, valid, sgi == nseg - 1, buf);
            } else {
                for (int gi = 0; ok && gi < ngroup; ++gi, ++gl) {
                    const uint32_t buf = gl % NB, ph = (gl / NB) & 1;
                    ok = __all_sync(0xffffffffu, mbar_wait(&acc_full[buf], ph, abort));
                    if (!ok) break;
                    tc_fence_after();
                    const int s0 = g.gs0[gi], s1 = g.gs0[gi + 1];
                    for (int sgi = s0; sgi < s1; ++sgi)
                        segment(sgi, lanes + buf * npad, gi * npad, X, Y, nx, pix, valid, sgi == s1 - 1, buf);
                }
            }
        }
    }

    __syncwarp();
    tc_fence_before();
    __syncthreads();
    if (warp == 1) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem_base), "r"(tmem_cols)
                     : "memory");
    }
}

// ------------------------------------------------------------------ FP8 e4m3 path
// Feature quantisation: one warp per pixel row.  x' = fl(x - m) (as the BF16 converters form
// it), s_x = 2^ceil(log2(max |x'| / 448)) so that x' / s_x is exact and at most 448, and
// q = e4m3(x' / s_x) rounded to nearest; rs = (s_x, an upper bound of ||x'||).
__device__ __forceinline__ float pow2_scale_f8(float amax)
{
    const float t = amax * (1.0f / 448.0f);
    if (!(t > 0x1p-100f)) return 0x1p-100f;
    int e;
    frexpf(t, &e);
    float sc = ldexpf(1.0f, e);
    if (amax / sc > 448.0f) sc *= 2.0f;
    return sc;
}

__global__ void __launch_bounds__(256) fp8_quant_kernel(const float *__restrict__ X, long long n, int D,
                                                      const float *__restrict__ mean, uint8_t *__restrict__ q,
                                                      float2 *__restrict__ rs)
{
    ptx::pdl_enter();
    const int lane = threadIdx.x & 31;
    const long long nw = ((long long)gridDim.x * blockDim.x) >> 5;
    for (long long row = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5; row < n; row += nw) {
        const float *x = X + row * D;
        float am = 0.f, x2 = 0.f;
        for (int i0 = 4 * lane; i0 < D; i0 += 128) {   // D % 16 == 0: whole float4 groups
            const float4 v = __ldg(reinterpret_cast<const float4 *>(x + i0));
            const float4 m = __ldg(reinterpret_cast<const float4 *>(mean + i0));
            const float a = v.x - m.x, b = v.y - m.y, c = v.z - m.z, d = v.w - m.w;
            am = fmaxf(am, fmaxf(fmaxf(fabsf(a), fabsf(b)), fmaxf(fabsf(c), fabsf(d))));
            x2 = fmaf(a, a, fmaf(b, b, fmaf(c, c, fmaf(d, d, x2))));
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            am = fmaxf(am, __shfl_xor_sync(0xffffffffu, am, o));
            x2 += __shfl_xor_sync(0xffffffffu, x2, o);
        }
        const float sx = pow2_scale_f8(am);
        const float inv = 1.0f / sx;                         // a power of two: exact, and so is x' * inv
        for (int i0 = 4 * lane; i0 < D; i0 += 128) {
            const float4 v = __ldg(reinterpret_cast<const float4 *>(x + i0));
            const float4 m = __ldg(reinterpret_cast<const float4 *>(mean + i0));
            const __nv_fp8x2_storage_t lo =
                __nv_cvt_float2_to_fp8x2(make_float2((v.x - m.x) * inv, (v.y - m.y) * inv), __NV_SATFINITE, __NV_E4M3);
            const __nv_fp8x2_storage_t hi =
                __nv_cvt_float2_to_fp8x2(make_float2((v.z - m.z) * inv, (v.w - m.w) * inv), __NV_SATFINITE, __NV_E4M3);
            *reinterpret_cast<uint32_t *>(q + row * D + i0) = (uint32_t)lo | ((uint32_t)hi << 16);
        }
        // ||x'|| from an FP32 sum of D non-negative terms: within (D + 8) u of the exact norm
        if (lane == 0) rs[row] = make_float2(sx, sqrtf(x2) * (1.0f + (float)(D + 8) * (float)kU));
    }
}

constexpr int F8_NT = 256;             // 8 warps
constexpr int F8_KC = 128;             // K elements (= bytes) per chunk
constexpr int F8_BOX = TM * F8_KC;     // 16 KB: 128 rows x 128 bytes
constexpr int F8_SA = 4;               // A stages
constexpr int F8_BMAX = 131072;        // resident codebook bytes (npad x padded D)

struct F8Args {
    long long n;
    int D, k, npad, nkc;
    long long ntiles;
    CodebookPrep p;
    const float2 *rs;
    uint8_t *labels;
    FlagList fl;
};

// D (+)= A . B^T, A (128 rows x 32 e4m3) and B (npad rows x 32 e4m3) in shared memory.
__device__ __forceinline__ void tc_mma_f8(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                          uint32_t acc)
{
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
        " tcgen05.mma.cta_group::1.kind::f8f6f4 [%0], %1, %2, %3, p;\n}" ::"r"(d_tmem),
        "l"(adesc), "l"(bdesc), "r"(idesc), "r"(acc)
        : "memory");
}
// Instruction descriptor: E4M3 x E4M3 -> F32, both K-major, M = 128, N = npad.
__host__ __device__ constexpr uint32_t f8_idesc(int M, int N)
{
    return (1u << 4) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

// One CTA per SM over 128-pixel tiles.  The FP8 codebook (npad rows x D bytes) is loaded once
// and stays in shared memory; the FP8 features stream through F8_SA stages of 128 x 128 bytes.
//   warp 0   TMA producer (codebook once, then the feature boxes)
//   warp 1   TMEM allocation; lane 0 issues the MMAs (K = 32 per instruction)
//   warps 4-7  epilogue: accumulators times s_x s_j give the dot products; the interval test
//            of the BF16 path with the FP8 bound terms; labels and flags
// Every mbarrier wait is bounded, as in assign_tc_kernel.
__global__ void __launch_bounds__(F8_NT, 1) assign_fp8_kernel(const __grid_constant__ CUtensorMap tmA,
                                                              const __grid_constant__ CUtensorMap tmB,
                                                              const __grid_constant__ F8Args g)
{
    ptx::pdl_enter();
    extern __shared__ uint8_t smem_raw[];
    uint8_t *base = reinterpret_cast<uint8_t *>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
    const int npad = g.npad, D = g.D, nkc = g.nkc, k = g.k;
    uint8_t *as = base;                                            // F8_SA x 16 KB
    uint8_t *bsm = as + F8_SA * F8_BOX;                            // nkc chunks x npad rows x 128 B
    float4 *colc = reinterpret_cast<float4 *>(bsm + (size_t)nkc * npad * 128);   // {||c*||^2, a, v, b}
    float *cn = reinterpret_cast<float *>(colc + npad);            // ||c*||^2 (+inf for padding)
    float *csc = cn + npad;                                        // per-column scale s_j
    uint32_t *maskbuf = reinterpret_cast<uint32_t *>(csc + npad);  // [128][8]
    float4 *segmx = reinterpret_cast<float4 *>(maskbuf + TM * kMaskWords);
    uint64_t *bar = reinterpret_cast<uint64_t *>(segmx + 1);
    uint64_t *a_full = bar, *a_empty = bar + F8_SA, *b_full = bar + 2 * F8_SA;
    uint64_t *acc_full = b_full + 1, *acc_empty = acc_full + 2, *drain = acc_empty + 2;
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(drain + 1);
    volatile int *abort = reinterpret_cast<volatile int *>(tmem_slot + 1);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const uint32_t tmem_cols = 2 * npad <= 32 ? 32 : 2 * npad <= 64 ? 64 : 2 * npad <= 128 ? 128
                             : 2 * npad <= 256 ? 256 : 512;
    for (int j = tid; j < npad; j += F8_NT) {
        const bool ok = j < k;
        const int jc = ok ? j : k - 1;
        const float nrm = ok ? g.p.nrm[jc] : FLT_MAX;               // padding columns never win nor qualify
        cn[j] = nrm;
        colc[j] = make_float4(nrm, ok ? g.p.a[jc] : 0.f, ok ? g.p.v[jc] : 0.f, ok ? g.p.b[jc] : 0.f);
        csc[j] = ok ? g.p.csc[jc] : 0.f;
    }
    if (tid == 0) {
        for (int q = 0; q < F8_SA; ++q) { mbar_init(&a_full[q], 1); mbar_init(&a_empty[q], 1); }
        mbar_init(b_full, 1);
        for (int q = 0; q < 2; ++q) { mbar_init(&acc_full[q], 1); mbar_init(&acc_empty[q], TM); }
        mbar_init(drain, 1);
        *abort = 0;
        fence_barrier_init();
        fence_proxy_async();
    }
    if (warp == 1) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                     "r"(tmem_cols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem_base = *tmem_slot;

    if (warp == 0) {
        // ---------------------------------------------------------- TMA producer
        if (lane == 0) {
            mbar_expect_tx(b_full, (uint32_t)(nkc * npad * 128));
            for (int kc = 0; kc < nkc; ++kc) tma_load_2d(bsm + (size_t)kc * npad * 128, &tmB, kc * F8_KC, 0, b_full);
            uint32_t st = 0, ph = 0;
            bool ok = true;
            long long issued = 0, last[F8_SA] = {-1, -1, -1, -1};
            for (long long tile = blockIdx.x; ok && tile < g.ntiles; tile += gridDim.x)
                for (int kc = 0; kc < nkc; ++kc, ++issued) {
                    if (!(ok = mbar_wait(&a_empty[st], ph ^ 1, abort))) break;
                    mbar_expect_tx(&a_full[st], F8_BOX);
                    tma_load_2d(as + st * F8_BOX, &tmA, kc * F8_KC, (int)(tile * TM), &a_full[st]);
                    last[st] = issued;
                    if (++st == (uint32_t)F8_SA) { st = 0; ph ^= 1; }
                }
            // every copy issued has landed before the block can leave (bounded)
            volatile int no_abort = 0;
            mbar_wait(b_full, 0, &no_abort);
            if (!ok)
                for (int q = 0; q < F8_SA; ++q)
                    if (last[q] >= 0) mbar_wait(&a_full[q], (uint32_t)((last[q] / F8_SA) & 1), &no_abort);
        }
    } else if (warp == 1) {
        // ---------------------------------------------------------- MMA issuer
        if (lane == 0) {
            const uint32_t idesc = f8_idesc(TM, npad);
            const uint64_t adesc0 = sw128_desc(smem_u32(as)), bdesc0 = sw128_desc(smem_u32(bsm));
            uint32_t st = 0, ph = 0, tl = 0;
            bool ok = mbar_wait(b_full, 0, abort);
            tc_fence_after();
            for (long long tile = blockIdx.x; ok && tile < g.ntiles; tile += gridDim.x, ++tl) {
                const uint32_t buf = tl & 1;
                if (!(ok = mbar_wait(&acc_empty[buf], ((tl >> 1) & 1) ^ 1, abort))) break;
                tc_fence_after();
                const uint32_t d_tmem = tmem_base + buf * npad;
                for (int kc = 0; kc < nkc; ++kc) {
                    if (!(ok = mbar_wait(&a_full[st], ph, abort))) break;
                    tc_fence_after();
                    const uint64_t ad = adesc0 + (uint64_t)((st * F8_BOX) >> 4);
                    const uint64_t bd = bdesc0 + (uint64_t)(((size_t)kc * npad * 128) >> 4);
#pragma unroll
                    for (int ks = 0; ks < F8_KC / 32; ++ks)    // K = 32 bytes per MMA: +2 in 16-byte units
                        tc_mma_f8(d_tmem, ad + 2 * ks, bd + 2 * ks, idesc, (kc | ks) != 0);
                    tc_commit(&a_empty[st]);
                    if (++st == (uint32_t)F8_SA) { st = 0; ph ^= 1; }
                }
                if (ok) tc_commit(&acc_full[buf]);
            }
            tc_commit(drain);                                 // every MMA done before TMEM is released
            volatile int no_abort = 0;
            mbar_wait(drain, 0, &no_abort);
        }
    } else if (warp >= 4) {
        // ---------------------------------------------------------- epilogue
        const int grp = warp & 3;                 // TMEM lane group this warp may read
        const int r = grp * 32 + lane;
        const float u = (float)kU;
        const float u4 = 4.0f * u;
        const float infl = 1.0f + 0.00390625f;
        const float sqD = sqrtf((float)D) * 1.0001f;
        if (warp == 4) {
            float nm = 0.f, am = 0.f, vm = 0.f, bm = 0.f;
            for (int j = lane; j < k; j += 32) {
                const float4 c = colc[j];
                nm = fmaxf(nm, c.x); am = fmaxf(am, c.y); vm = fmaxf(vm, c.z); bm = fmaxf(bm, c.w);
            }
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                nm = fmaxf(nm, __shfl_xor_sync(0xffffffffu, nm, o));
                am = fmaxf(am, __shfl_xor_sync(0xffffffffu, am, o));
                vm = fmaxf(vm, __shfl_xor_sync(0xffffffffu, vm, o));
                bm = fmaxf(bm, __shfl_xor_sync(0xffffffffu, bm, o));
            }
            if (lane == 0) *segmx = make_float4(nm, am, vm, bm);
        }
        asm volatile("bar.sync 1, 128;" ::: "memory");       // the four epilogue warps
        const float4 mx = *segmx;
        const float cnorm_max = sqrtf(mx.x) * 1.0001f, nrm_max = mx.x * 1.0001f;
        uint32_t tl = 0;
        bool ok = true;
        for (long long tile = blockIdx.x; ok && tile < g.ntiles; tile += gridDim.x, ++tl) {
            const uint32_t buf = tl & 1;
            const long long pix = tile * TM + r;
            const bool valid = pix < g.n;
            const float2 rsv = valid ? g.rs[pix] : make_float2(1.0f, 0.0f);
            ok = __all_sync(0xffffffffu, mbar_wait(&acc_full[buf], (tl >> 1) & 1, abort));
            if (!ok) break;
            tc_fence_after();
            // pixel side: ||x' - s_x q_x|| <= 2^-4 ||x'|| + 2^-10 s_x sqrt(D) (= Dl) and
            // ||s_x q_x|| <= ||x'|| + Dl (= X); Y adds the rounding of x' = fl(x - m)
            const float sx = rsv.x, nx = rsv.y;
            const float Dl = (0.0625f * nx + 0.0009765625f * sx * sqD) * 1.0001f + 1e-30f;
            const float X = (nx + Dl) * infl;
            const float Y = Dl + u * (X * 1.01f + Dl) * (1.0f + 4.0f * u);
            const uint32_t taddr = tmem_base + ((uint32_t)(grp * 32) << 16) + buf * npad;
            // pass 1: smallest score, lowest column on ties (four interleaved running minima);
            // s_j = ||c*||^2 - 2 s_x s_j acc_j, the scales powers of two (exact products)
            float sm[4] = {FLT_MAX, FLT_MAX, FLT_MAX, FLT_MAX};
            int amv[4] = {0, 0, 0, 0};
            for (int c0 = 0; c0 < npad; c0 += 32) {
                float v[32];
                tc_ld32(taddr + (uint32_t)c0, v);
#pragma unroll
                for (int j = 0; j < 32; ++j) {
                    const float sc = fmaf(-2.0f, v[j] * (sx * csc[c0 + j]), cn[c0 + j]);
                    if (sc < sm[j & 3]) { sm[j & 3] = sc; amv[j & 3] = c0 + j; }
                }
            }
            float smin = sm[0];
            int amin = amv[0];
#pragma unroll
            for (int q = 1; q < 4; ++q)
                if (sm[q] < smin || (sm[q] == smin && amv[q] < amin)) { smin = sm[q]; amin = amv[q]; }
            const float4 ca = colc[amin];
            const float U = smin + fmaf(X, ca.y, fmaf(Y, ca.z, fmaf(u4, fabsf(smin), ca.w))) * infl;
            const float smax_abs = fmaf(2.0f * X * 1.02f, cnorm_max, nrm_max) + 1.0f;
            const float Bmax = fmaf(X, mx.y, fmaf(Y, mx.z, fmaf(u4, smax_abs, mx.w))) * infl;
            const float lim = U + 2.0f * Bmax;
            int cnt = 0, last = amin;
            for (int c0 = 0; c0 < npad; c0 += 32) {
                float v[32];
                tc_ld32(taddr + (uint32_t)c0, v);
                uint32_t maybe = 0;
#pragma unroll
                for (int j = 0; j < 32; ++j)
                    maybe |= (uint32_t)(fmaf(-2.0f, v[j] * (sx * csc[c0 + j]), cn[c0 + j]) <= lim) << j;
                const uint32_t own = (amin >> 5) == (c0 >> 5) ? 1u << (amin & 31) : 0u;
                uint32_t word = own;
                if (__any_sync(0xffffffffu, (maybe & ~own) != 0u)) {
                    word = 0;
#pragma unroll
                    for (int j = 0; j < 32; ++j) {
                        const float4 c = colc[c0 + j];
                        const float sc = fmaf(-2.0f, v[j] * (sx * csc[c0 + j]), c.x);
                        const float B = fmaf(X, c.y, fmaf(Y, c.z, fmaf(u4, fabsf(sc), c.w))) * infl;
                        word |= (uint32_t)(sc - B <= U) << j;
                    }
                }
                cnt += __popc(word);
                if (word) last = c0 + 31 - __clz(word);
                maskbuf[r * kMaskWords + (c0 >> 5)] = word;
            }
            for (int w = npad >> 5; w < kMaskWords; ++w) maskbuf[r * kMaskWords + w] = 0u;
            tc_fence_before();
            mbar_arrive(&acc_empty[buf]);                    // every accumulator of the buffer read
            const int lab = cnt == 1 ? last : amin;
            if (valid) g.labels[pix] = (uint8_t)lab;
            const bool flagged = valid && cnt > 1;
            const unsigned ballot = __ballot_sync(0xffffffffu, flagged);
            if (ballot) {
                const int leader = __ffs(ballot) - 1;
                unsigned basei = 0;
                if (lane == leader) basei = atomicAdd(g.fl.count, (unsigned)__popc(ballot));
                basei = __shfl_sync(0xffffffffu, basei, leader);
                if (flagged) {
                    const unsigned slot = basei + __popc(ballot & ((1u << lane) - 1u));
                    if (slot < (unsigned long long)g.n) {
                        g.fl.pix[slot] = (unsigned)pix;
#pragma unroll
                        for (int w = 0; w < kMaskWords; ++w)
                            g.fl.mask[(size_t)slot * kMaskWords + w] = maskbuf[r * kMaskWords + w];
                    }
                }
            }
        }
    }

    __syncwarp();
    tc_fence_before();
    __syncthreads();
    if (warp == 1) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem_base), "r"(tmem_cols)
                     : "memory");
    }
}

// ------------------------------------------------------------------ host side
PFN_cuTensorMapEncodeTiled_v12000 g_encode = nullptr;
std::once_flag g_encode_once;

cudaError_t get_encode()
{
    std::call_once(g_encode_once, [] {
        void *fn = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            g_encode = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(fn);
    });
    return g_encode ? cudaSuccess : cudaErrorNotSupported;
}

cudaError_t make_map(CUtensorMap *m, CUtensorMapDataType dt, const void *ptr, uint64_t cols, uint64_t rows,
                     uint64_t row_bytes, uint32_t box_cols, uint32_t box_rows)
{
    const cuuint64_t dims[2] = {cols, rows};
    const cuuint64_t strides[1] = {row_bytes};
    const cuuint32_t box[2] = {box_cols, box_rows};
    const cuuint32_t es[2] = {1, 1};
    const CUresult r = g_encode(m, dt, 2, const_cast<void *>(ptr), dims, strides, box, es,
                                CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                                CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorInvalidValue;
}

// ncols: prepared columns held per column (npad, or ngroup * npad when stationary); nsegcap:
// capacity of the segment table
size_t tc_smem_bytes(int npad, int D, int sb, int sf, int ncols = 0, int nsegcap = kMaxSeg, bool stat = false)
{
    const int nkc = (D + KC - 1) / KC;
    if (ncols == 0) ncols = npad;
    size_t b = 1024;                                       // alignment slack
    b += (size_t)sf * F32_BOX + (size_t)sb * 2 * npad * 128;
    b += sizeof(float) * ((stat ? 4 : 5) * (size_t)ncols + (size_t)nkc * KC + 8 * TM);
    b += sizeof(uint32_t) * TM * kMaskWords;
    b += (sizeof(float4) + sizeof(TcSeg)) * nsegcap;
    b += sizeof(uint64_t) * (2 * sf + 2 * kMaxSA + 2 * kMaxSB + 8 + 1) + 16;   // barriers, TMEM slot, abort flag
    return b;
}

}  // namespace

cudaError_t launch_assign_bf16_seg(const float *X, long long n, int D, const CodebookPrep &p, int krows,
                                   const TcSeg *seg, int nseg, int sf_req, int pf, cudaStream_t s)
{
    if (D % 16 != 0 || nseg < 1 || nseg > kMaxSeg || krows < 1 || n < 1) return cudaErrorNotSupported;
    int npad = 0;
    for (int q = 0; q < nseg; ++q) {
        if (seg[q].col0 != npad || seg[q].ncol % 32 != 0 || seg[q].k < 1 || seg[q].k > seg[q].ncol ||
            seg[q].col0 + seg[q].k > krows)
            return cudaErrorNotSupported;
        npad += seg[q].ncol;
    }
    if (npad > kMaxK) return cudaErrorNotSupported;
    cudaError_t e = get_encode();
    if (e != cudaSuccess) return e;
    int dev = 0, sms = 0, optin = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    // centroid stages (the codebook is streamed from L2 by every CTA) and feature boxes (HBM
    // latency): the first split that fits, or the requested feature-box count with as many
    // centroid stages as fit
    static const int kSplit[][2] = {{3, 6}, {2, 8}, {2, 6}, {2, 4}, {1, 4}};
    int sb = 0, sf = 0;
    size_t smem = 0;
    if (sf_req > 0) {
        if (sf_req < 2 || sf_req > kMaxSF || sf_req % 2) return cudaErrorNotSupported;
        for (int b = 3; b >= 1 && !sf; --b)
            if ((smem = tc_smem_bytes(npad, D, b, sf_req)) <= (size_t)optin) { sb = b; sf = sf_req; }
    } else {
        for (const auto &c : kSplit)
            if ((smem = tc_smem_bytes(npad, D, c[0], c[1])) <= (size_t)optin) { sb = c[0]; sf = c[1]; break; }
    }
    if (!sf) return cudaErrorNotSupported;
    // accumulators double-buffered when they fit beside two A stages in the 512 TMEM columns;
    // the remaining columns hold as many A stages as fit (at most four)
    const int nb = 2 * npad + 2 * 64 <= 512 ? 2 : 1;
    const int sa = (512 - nb * npad) / 64 < kMaxSA ? (512 - nb * npad) / 64 : kMaxSA;
    CUtensorMap tmA, tmBhi, tmBlo;
    if ((e = make_map(&tmA, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, X, (uint64_t)D, (uint64_t)n, (uint64_t)D * 4, 32,
                      TM)) != cudaSuccess)
        return e;
    if ((e = make_map(&tmBhi, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, p.chi, (uint64_t)D, (uint64_t)krows,
                      (uint64_t)D * 2, KC, (uint32_t)npad)) != cudaSuccess)
        return e;
    if ((e = make_map(&tmBlo, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, p.clo, (uint64_t)D, (uint64_t)krows,
                      (uint64_t)D * 2, KC, (uint32_t)npad)) != cudaSuccess)
        return e;
    TcArgs a;
    memset(&a, 0, sizeof(a));
    a.n = n;
    a.D = D;
    a.krows = krows;
    a.npad = npad;
    a.nkc = (D + KC - 1) / KC;
    a.sb = sb;
    a.sf = sf;
    a.nb = nb;
    a.sa = sa;
    a.pf = pf < 0 ? PF : pf;
    a.ntiles = (n + TM - 1) / TM;
    a.p = p;
    a.nseg = nseg;
    for (int q = 0; q < nseg; ++q) a.seg[q] = seg[q];
    const long long grid = a.ntiles < sms ? a.ntiles : sms;
    if (nseg == 1) {
        e = cudaFuncSetAttribute(assign_tc_kernel<false, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)smem);
        if (e != cudaSuccess) return e;
        {
        const cudaError_t le_ = launch_pdl(assign_tc_kernel<false, false>, dim3((unsigned)grid), dim3(NT), smem, s, tmA, tmBhi, tmBlo, a);
        if (le_ != cudaSuccess) return le_;
    }
    } else {
        e = cudaFuncSetAttribute(assign_tc_kernel<true, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)smem);
        if (e != cudaSuccess) return e;
        {
        const cudaError_t le_ = launch_pdl(assign_tc_kernel<true, false>, dim3((unsigned)grid), dim3(NT), smem, s, tmA, tmBhi, tmBlo, a);
        if (le_ != cudaSuccess) return le_;
    }
    }
    return cudaGetLastError();
}

// Stationary mode: two FP32 feature boxes in flight (the features are read once per tile, then
// every group's MMAs run on them); four centroid stages for groups of 128 columns, two for 256
// (twice the MMA work per stage).
constexpr int STAT_SF = 2;
int stat_sb(int gcols) { return gcols <= 128 ? 4 : 2; }

int stat_max_groups(int D, int gcols)
{
    int dev = 0, optin = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    int gmax = 0;
    for (int ng = 1; ng <= kMaxGroupsStat; ++ng)
        if (tc_smem_bytes(gcols, D, stat_sb(gcols), STAT_SF, ng * gcols, kMaxSegStat, true) <= (size_t)optin)
            gmax = ng;
    return gmax;
}

cudaError_t launch_assign_bf16_stat(const float *X, long long n, int D, const CodebookPrep &p, int ngroup,
                                    int gcols, const TcSeg *seg, const int *gs0, cudaStream_t s)
{
    const int nkc = (D + KC - 1) / KC;
    // all A stages resident: nkc * 64 columns beside one or two accumulators of gcols columns
    const int nb = 2 * gcols + nkc * 64 <= 512 ? 2 : 1;
    if (D % 16 != 0 || nkc > kMaxSA || gcols % 32 != 0 || gcols < 32 || gcols > kMaxK ||
        nb * gcols + nkc * 64 > 512 ||
        ngroup < 1 || ngroup > kMaxGroupsStat || n < 1 || gs0[0] != 0 || gs0[ngroup] > kMaxSegStat)
        return cudaErrorNotSupported;
    for (int gi = 0; gi < ngroup; ++gi) {
        if (gs0[gi + 1] <= gs0[gi]) return cudaErrorNotSupported;
        int col = gi * gcols;
        for (int q = gs0[gi]; q < gs0[gi + 1]; ++q) {
            if (seg[q].col0 != col || seg[q].ncol % 32 != 0 || seg[q].k < 1 || seg[q].k > seg[q].ncol)
                return cudaErrorNotSupported;
            col += seg[q].ncol;
        }
        if (col > (gi + 1) * gcols) return cudaErrorNotSupported;
    }
    cudaError_t e = get_encode();
    if (e != cudaSuccess) return e;
    int dev = 0, sms = 0, optin = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    const size_t smem = tc_smem_bytes(gcols, D, stat_sb(gcols), STAT_SF, ngroup * gcols, kMaxSegStat, true);
    if (smem > (size_t)optin) return cudaErrorNotSupported;
    const int krows = ngroup * gcols;
    CUtensorMap tmA, tmBhi, tmBlo;
    if ((e = make_map(&tmA, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, X, (uint64_t)D, (uint64_t)n, (uint64_t)D * 4, 32,
                      TM)) != cudaSuccess)
        return e;
    if ((e = make_map(&tmBhi, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, p.chi, (uint64_t)D, (uint64_t)krows,
                      (uint64_t)D * 2, KC, (uint32_t)gcols)) != cudaSuccess)
        return e;
    if ((e = make_map(&tmBlo, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, p.clo, (uint64_t)D, (uint64_t)krows,
                      (uint64_t)D * 2, KC, (uint32_t)gcols)) != cudaSuccess)
        return e;
    TcArgs a;
    memset(&a, 0, sizeof(a));
    a.n = n;
    a.D = D;
    a.krows = krows;
    a.npad = gcols;
    a.nkc = nkc;
    a.sb = stat_sb(gcols);
    a.sf = STAT_SF;
    a.nb = nb;
    a.sa = nkc;                                            // chunk kc in A stage kc
    a.pf = 0;
    a.ntiles = (n + TM - 1) / TM;
    a.p = p;
    a.nseg = gs0[ngroup];
    for (int q = 0; q < a.nseg; ++q) a.seg[q] = seg[q];
    a.ngroup = ngroup;
    for (int gi = 0; gi <= ngroup; ++gi) a.gs0[gi] = gs0[gi];
    const long long grid = a.ntiles < sms ? a.ntiles : sms;
    e = cudaFuncSetAttribute(assign_tc_kernel<true, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    {
        const cudaError_t le_ = launch_pdl(assign_tc_kernel<true, true>, dim3((unsigned)grid), dim3(NT), smem, s, tmA, tmBhi, tmBlo, a);
        if (le_ != cudaSuccess) return le_;
    }
    return cudaGetLastError();
}

cudaError_t launch_assign_bf16(const float *X, long long n, int D, int k, const CodebookPrep &p,
                               uint8_t *labels, FlagList fl, cudaStream_t s)
{
    if (k < 1 || k > kMaxK) return cudaErrorNotSupported;
    TcSeg one;
    one.col0 = 0;
    one.ncol = (k + 31) / 32 * 32;            // UMMA N (multiple of 16) and whole 32-column TMEM loads
    one.k = k;
    one.labels = labels;
    one.fl = fl;
    return launch_assign_bf16_seg(X, n, D, p, k, &one, 1, 0, -1, s);
}

bool fp8_supported(int D, int k)
{
    const int npad = (k + 31) / 32 * 32;
    const int dpad = (D + F8_KC - 1) / F8_KC * F8_KC;
    return D % 16 == 0 && k >= 1 && k <= kMaxK && (long long)npad * dpad <= F8_BMAX;
}

static size_t f8_smem_bytes(int npad, int D)
{
    const int nkc = (D + F8_KC - 1) / F8_KC;
    size_t b = 1024;                                       // alignment slack
    b += (size_t)F8_SA * F8_BOX + (size_t)nkc * npad * 128;
    b += sizeof(float4) * npad + sizeof(float) * 2 * npad + sizeof(uint32_t) * TM * kMaskWords + sizeof(float4);
    b += sizeof(uint64_t) * (2 * F8_SA + 1 + 4 + 1) + 16;
    return b;
}

cudaError_t launch_assign_fp8(const float *X, long long n, int D, int k, const CodebookPrep &p, Fp8Feat f8,
                              uint8_t *labels, FlagList fl, cudaStream_t s)
{
    if (!fp8_supported(D, k) || n < 1 || !f8.q || !f8.rs || !p.cq8 || !p.csc) return cudaErrorNotSupported;
    cudaError_t e = get_encode();
    if (e != cudaSuccess) return e;
    int dev = 0, sms = 0, optin = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    const int npad = (k + 31) / 32 * 32;
    const size_t smem = f8_smem_bytes(npad, D);
    if (smem > (size_t)optin) return cudaErrorNotSupported;
    {
        const cudaError_t le_ = launch_pdl(fp8_quant_kernel, dim3(sms * 16), dim3(256), 0, s, X, n, D,
                                           (const float *)p.mean, f8.q, f8.rs);
        if (le_ != cudaSuccess) return le_;
    }
    CUtensorMap tmA, tmB;
    if ((e = make_map(&tmA, CU_TENSOR_MAP_DATA_TYPE_UINT8, f8.q, (uint64_t)D, (uint64_t)n, (uint64_t)D, F8_KC,
                      TM)) != cudaSuccess)
        return e;
    if ((e = make_map(&tmB, CU_TENSOR_MAP_DATA_TYPE_UINT8, p.cq8, (uint64_t)D, (uint64_t)k, (uint64_t)D, F8_KC,
                      (uint32_t)npad)) != cudaSuccess)
        return e;
    F8Args a;
    memset(&a, 0, sizeof(a));
    a.n = n;
    a.D = D;
    a.k = k;
    a.npad = npad;
    a.nkc = (D + F8_KC - 1) / F8_KC;
    a.ntiles = (n + TM - 1) / TM;
    a.p = p;
    a.rs = f8.rs;
    a.labels = labels;
    a.fl = fl;
    e = cudaFuncSetAttribute(assign_fp8_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    if ((e = record_kernel_event(VQNNF_OP_ASSIGN, 0, s)) != cudaSuccess) return e;
    const long long grid = a.ntiles < sms ? a.ntiles : sms;
    {
        const cudaError_t le_ = launch_pdl(assign_fp8_kernel, dim3((unsigned)grid), dim3(F8_NT), smem, s, tmA, tmB, a);
        if (le_ != cudaSuccess) return le_;
    }
    return cudaGetLastError();
}

cudaError_t read_and_clear_tc_error(int *out)
{
    int zero = 0;
    cudaError_t e = cudaMemcpyFromSymbol(out, g_tc_error, sizeof(int));
    if (e == cudaSuccess) e = cudaMemcpyToSymbol(g_tc_error, &zero, sizeof(int));
    return e;
}

}  // namespace vqnnf
