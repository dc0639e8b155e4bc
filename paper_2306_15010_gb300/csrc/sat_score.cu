// Integral image of the one-hot NNF, coarse-filter responses and the Eq. 2 similarity.
//
// Integral image (Supp. "Integral Image"; exclusive-prefix reading): for cluster j,
//     S[y][j][x] = #{ (y', x') : y' < y, x' < x, label(y', x') = j },  0 <= y <= H, 0 <= x <= W
// stored channel-planar: element (y, j, x) at (y * k + j) * P + x, P = W + 1 rounded up to a
// multiple of 4 (16-byte rows for vector copies).  A half-open rectangle's count is the
// four-corner sum S(y1,x1) - S(y0,x1) - S(y1,x0) + S(y0,x0); a filter is a weighted sum of
// such boxes, i.e. the dilation filter that Algorithm 2 builds on the integral image.
//
// Build: (1) per row, the count of every cluster left of every 32-column strip; (2) one
// warp per (strip, 8 clusters) sweeps the rows, each lane one column: the row prefix
// inside the strip is a ballot + popcount, added to the running column sum.
//
// Score: one block per (window row, 256 windows); the corner rows of its windows are
// staged in shared memory 8 clusters at a time (cp.async double buffering), each thread
// owns two windows and accumulates exact integer L1 distances per filter over all
// clusters, then combines them in float32 in bank order.
#include <cuda_pipeline.h>

#include <cfloat>

#include "common.cuh"
#include "score_spec.cuh"

namespace vqnnf {
namespace {

constexpr int SW = 32;     // columns per strip = lanes
constexpr int CGW = 8;     // clusters per warp in the sweep

// carry[(y * nS + s) * k + j] = #{x' < 32 s : label(y, x') = j}
__global__ void row_carry_kernel(const uint8_t *__restrict__ lab, int W, int k, int nS,
                                 int *__restrict__ carry)
{
    extern __shared__ int hist[];     // [nS][k]
    const int y = blockIdx.x;
    for (int q = threadIdx.x; q < nS * k; q += blockDim.x) hist[q] = 0;
    __syncthreads();
    const uint8_t *row = lab + (size_t)y * W;
    for (int x = threadIdx.x; x < W; x += blockDim.x) {
        const int lb = row[x];
        if (lb < k) atomicAdd(&hist[(x / SW) * k + lb], 1);
    }
    __syncthreads();
    for (int j = threadIdx.x; j < k; j += blockDim.x) {
        int s = 0;
        for (int q = 0; q < nS; ++q) {
            const int c = hist[q * k + j];
            carry[((size_t)y * nS + q) * k + j] = s;
            s += c;
        }
    }
}

__global__ void __launch_bounds__(128) sat_sweep_kernel(const uint8_t *__restrict__ lab, int H,
                                                        int W, int k, int P, int nS,
                                                        const int *__restrict__ carry,
                                                        int *__restrict__ S)
{
    const int lane = threadIdx.x & 31;
    const int gw = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    const int ncg = (k + CGW - 1) / CGW;
    if (gw >= nS * ncg) return;
    const int s = gw / ncg, cg = gw % ncg;
    const int x = s * SW + lane;          // S column owned by this lane
    const bool xin = x < P;
    const unsigned lt = (1u << lane) - 1u;
    int acc[CGW];
#pragma unroll
    for (int q = 0; q < CGW; ++q) acc[q] = 0;
    // row 0 of S is all zero
#pragma unroll
    for (int q = 0; q < CGW; ++q) {
        const int j = cg * CGW + q;
        if (j < k && xin) S[(size_t)j * P + x] = 0;
    }
    for (int y = 0; y < H; ++y) {
        const int xl = s * SW + lane;      // label column tested by this lane
        const int l0 = (int)lab[(size_t)y * W + min(xl, W - 1)];   // clamped address
        const int lb = (xl < W) ? l0 : -1;
        const int jc = min(cg * CGW + (lane & (CGW - 1)), k - 1);
        const int c0 = carry[((size_t)y * nS + s) * k + jc];
        const int cj = (lane < CGW && cg * CGW + lane < k) ? c0 : 0;
#pragma unroll
        for (int q = 0; q < CGW; ++q) {
            const int j = cg * CGW + q;
            const unsigned b = __ballot_sync(0xffffffffu, lb == j);
            const int r = __shfl_sync(0xffffffffu, cj, q) + __popc(b & lt);
            acc[q] += r;
            if (j < k && xin) S[((size_t)(y + 1) * k + j) * P + x] = acc[q];
        }
    }
}

// ---------------------------------------------------------------------------------
// Template responses: one block per filter, shared-memory histogram (integer atomics).
// ---------------------------------------------------------------------------------
__global__ void filter_responses_kernel(const uint8_t *__restrict__ lab, int w, int k,
                                        BankSpec bs, int32_t *__restrict__ counts)
{
    __shared__ int hist[kMaxK];
    const int f = blockIdx.x;
    for (int j = threadIdx.x; j < k; j += blockDim.x) hist[j] = 0;
    __syncthreads();
    for (int r = bs.rect_begin[f]; r < bs.rect_begin[f + 1]; ++r) {
        const RectSpec rc = bs.rect[r];
        const int rw = rc.x1 - rc.x0, n = rw * (rc.y1 - rc.y0);
        for (int q = threadIdx.x; q < n; q += blockDim.x) {
            const int yy = rc.y0 + q / rw, xx = rc.x0 + q % rw;
            atomicAdd(&hist[lab[(size_t)yy * w + xx]], rc.weight);
        }
    }
    __syncthreads();
    for (int j = threadIdx.x; j < k; j += blockDim.x) counts[(size_t)f * k + j] = hist[j];
}

// ---------------------------------------------------------------------------------
// Score.
// ---------------------------------------------------------------------------------
constexpr int TXW = 256;          // windows per block along x
constexpr int STH = 128;          // threads (2 windows each)
constexpr int CH = 8;             // clusters per staged chunk

__device__ __forceinline__ unsigned long long pack_key(float v, unsigned idx)
{
    unsigned b = __float_as_uint(v);
    b = (b & 0x80000000u) ? ~b : (b | 0x80000000u);   // order-preserving
    return ((unsigned long long)b << 32) | (unsigned long long)(0xFFFFFFFFu - idx);
}

// Stage corner rows [nrow] x NCOL columns of CH clusters starting at cluster j0.
__device__ __forceinline__ void stage_chunk(int *dst, const int *__restrict__ S, int k, int P,
                                            int y, int x0, int j0, int ncol, const int *roff,
                                            int nrow)
{
    const int per_row = ncol / 4;                 // 16-byte pieces
    const int total = CH * nrow * per_row;
    for (int q = threadIdx.x; q < total; q += blockDim.x) {
        const int piece = q % per_row;
        const int rr = (q / per_row) % nrow;
        const int c = q / (per_row * nrow);
        const int j = j0 + c;
        int *d = dst + ((c * nrow + rr) * ncol + piece * 4);
        const int col = x0 + piece * 4;
        if (j < k && col < P) {
            const int *src = S + ((size_t)(y + roff[rr]) * k + j) * P + col;
            __pipeline_memcpy_async(d, src, 16);
        } else {
            d[0] = d[1] = d[2] = d[3] = 0;
        }
    }
    __pipeline_commit();
}

template <int G, bool FULL>
__global__ void __launch_bounds__(STH) score_grid_kernel(const int *__restrict__ S, int P, int k,
                                                         int HO, int WO, GridSpec gs,
                                                         const int32_t *__restrict__ tcounts,
                                                         float *__restrict__ heat,
                                                         unsigned long long *amax)
{
    constexpr int NR = G + 1;
    constexpr int NSLOT = G * G + (FULL ? 1 : 0);
    extern __shared__ __align__(16) int sm[];
    const int ncol = gs.ncol;
    int *buf0 = sm;
    int *buf1 = sm + CH * NR * ncol;
    int *tc = buf1 + CH * NR * ncol;      // [NSLOT][k]
    const int y = blockIdx.y;
    const int x0 = blockIdx.x * TXW;
    for (int q = threadIdx.x; q < NSLOT * k; q += blockDim.x) {
        const int slot = q / k, j = q % k;
        tc[q] = tcounts[(size_t)gs.slot_filter[slot] * k + j];
    }
    const int nchunk = (k + CH - 1) / CH;
    stage_chunk(buf0, S, k, P, y, x0, 0, ncol, gs.by, NR);
    int l1[2][NSLOT];
#pragma unroll
    for (int w = 0; w < 2; ++w)
#pragma unroll
        for (int q = 0; q < NSLOT; ++q) l1[w][q] = 0;
    const int xl = threadIdx.x * 2;
    for (int ch = 0; ch < nchunk; ++ch) {
        int *cur = (ch & 1) ? buf1 : buf0;
        if (ch + 1 < nchunk) {
            stage_chunk((ch & 1) ? buf0 : buf1, S, k, P, y, x0, (ch + 1) * CH, ncol, gs.by, NR);
            __pipeline_wait_prior(1);
        } else {
            __pipeline_wait_prior(0);
        }
        __syncthreads();
        const int cmax = min(CH, k - ch * CH);
        for (int c = 0; c < cmax; ++c) {
            const int j = ch * CH + c;
            const int *base = cur + c * NR * ncol;
            int t[NSLOT];
#pragma unroll
            for (int q = 0; q < NSLOT; ++q) t[q] = tc[q * k + j];
#pragma unroll
            for (int w = 0; w < 2; ++w) {
                int cr[NR][NR];
#pragma unroll
                for (int r = 0; r < NR; ++r)
#pragma unroll
                    for (int cc = 0; cc < NR; ++cc) cr[r][cc] = base[r * ncol + xl + w + gs.bx[cc]];
#pragma unroll
                for (int r = 0; r < G; ++r)
#pragma unroll
                    for (int cc = 0; cc < G; ++cc) {
                        const int v = cr[r + 1][cc + 1] - cr[r + 1][cc] - cr[r][cc + 1] + cr[r][cc];
                        l1[w][r * G + cc] += abs(t[r * G + cc] - v);
                    }
                if (FULL) {
                    const int v = cr[G][G] - cr[G][0] - cr[0][G] + cr[0][0];
                    l1[w][NSLOT - 1] += abs(t[NSLOT - 1] - v);
                }
            }
        }
        __syncthreads();
    }
    // combine in bank order: H = - sum_f coef_f * L1_f
    unsigned long long best = 0ull;
#pragma unroll
    for (int w = 0; w < 2; ++w) {
        const int x = x0 + xl + w;
        float acc = 0.f;
        for (int f = 0; f < gs.F; ++f) {
            int v = 0;
#pragma unroll
            for (int q = 0; q < NSLOT; ++q)
                if (gs.filter_slot[f] == q) v = l1[w][q];
            acc = fmaf(gs.coef[f], (float)v, acc);
        }
        const float h = -acc;
        if (x < WO) {
            heat[(size_t)y * WO + x] = h;
            const unsigned long long key = pack_key(h, (unsigned)(y * WO + x));
            best = key > best ? key : best;
        }
    }
    if (amax) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            const unsigned long long other = __shfl_xor_sync(0xffffffffu, best, o);
            best = other > best ? other : best;
        }
        if ((threadIdx.x & 31) == 0 && best) atomicMax(amax, best);
    }
}

// Generic bank: any weighted half-open rectangles.  Corner rows are the distinct row
// offsets of the bank; each rectangle reads its four corners from shared memory.
__global__ void __launch_bounds__(STH) score_generic_kernel(const int *__restrict__ S, int P,
                                                            int k, int HO, int WO, BankSpec bs,
                                                            const int32_t *__restrict__ tcounts,
                                                            float *__restrict__ heat,
                                                            unsigned long long *amax)
{
    extern __shared__ __align__(16) int sm[];
    const int ncol = bs.ncol, nrow = bs.nrow;
    int *buf0 = sm;
    int *buf1 = sm + CH * nrow * ncol;
    int *tc = buf1 + CH * nrow * ncol;    // [F][k]
    const int y = blockIdx.y;
    const int x0 = blockIdx.x * TXW;
    for (int q = threadIdx.x; q < bs.F * k; q += blockDim.x) tc[q] = tcounts[q];
    const int nchunk = (k + CH - 1) / CH;
    stage_chunk(buf0, S, k, P, y, x0, 0, ncol, bs.roff, nrow);
    long long l1[2][kMaxFilters];
    for (int w = 0; w < 2; ++w)
        for (int f = 0; f < kMaxFilters; ++f) l1[w][f] = 0;
    const int xl = threadIdx.x * 2;
    for (int ch = 0; ch < nchunk; ++ch) {
        int *cur = (ch & 1) ? buf1 : buf0;
        if (ch + 1 < nchunk) {
            stage_chunk((ch & 1) ? buf0 : buf1, S, k, P, y, x0, (ch + 1) * CH, ncol, bs.roff, nrow);
            __pipeline_wait_prior(1);
        } else {
            __pipeline_wait_prior(0);
        }
        __syncthreads();
        const int cmax = min(CH, k - ch * CH);
        for (int c = 0; c < cmax; ++c) {
            const int j = ch * CH + c;
            const int *base = cur + c * nrow * ncol;
            for (int f = 0; f < bs.F; ++f) {
                const int t = tc[f * k + j];
                for (int w = 0; w < 2; ++w) {
                    int v = 0;
                    for (int r = bs.rect_begin[f]; r < bs.rect_begin[f + 1]; ++r) {
                        const RectSpec rc = bs.rect[r];
                        const int *r0 = base + rc.ry0 * ncol + xl + w;
                        const int *r1 = base + rc.ry1 * ncol + xl + w;
                        v += rc.weight * (r1[rc.x1] - r1[rc.x0] - r0[rc.x1] + r0[rc.x0]);
                    }
                    l1[w][f] += abs(t - v);
                }
            }
        }
        __syncthreads();
    }
    unsigned long long best = 0ull;
    for (int w = 0; w < 2; ++w) {
        const int x = x0 + xl + w;
        float acc = 0.f;
        for (int f = 0; f < bs.F; ++f) acc = fmaf(bs.coef[f], (float)l1[w][f], acc);
        const float h = -acc;
        if (x < WO) {
            heat[(size_t)y * WO + x] = h;
            const unsigned long long key = pack_key(h, (unsigned)(y * WO + x));
            best = key > best ? key : best;
        }
    }
    if (amax) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            const unsigned long long other = __shfl_xor_sync(0xffffffffu, best, o);
            best = other > best ? other : best;
        }
        if ((threadIdx.x & 31) == 0 && best) atomicMax(amax, best);
    }
}

__global__ void argmax_finish_kernel(const unsigned long long *amax, int WO, int32_t *out)
{
    const unsigned idx = 0xFFFFFFFFu - (unsigned)(*amax & 0xFFFFFFFFull);
    out[0] = (int32_t)(idx / (unsigned)WO);
    out[1] = (int32_t)(idx % (unsigned)WO);
}

template <int G, bool FULL>
cudaError_t launch_grid(const int *S, int P, int k, int HO, int WO, const GridSpec &gs,
                        const int32_t *tc, float *heat, unsigned long long *amax, cudaStream_t s)
{
    constexpr int NR = G + 1;
    constexpr int NSLOT = G * G + (FULL ? 1 : 0);
    const size_t smem = sizeof(int) * ((size_t)2 * CH * NR * gs.ncol + (size_t)NSLOT * k);
    cudaError_t e = cudaFuncSetAttribute(score_grid_kernel<G, FULL>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    dim3 grid((WO + TXW - 1) / TXW, HO);
    score_grid_kernel<G, FULL><<<grid, STH, smem, s>>>(S, P, k, HO, WO, gs, tc, heat, amax);
    return cudaGetLastError();
}

}  // namespace

size_t score_smem_bytes(const BankSpec &bs, const GridSpec &gs, int k)
{
    if (gs.G > 0) {
        const int NR = gs.G + 1;
        const int NSLOT = gs.G * gs.G + (gs.full ? 1 : 0);
        return sizeof(int) * ((size_t)2 * CH * NR * gs.ncol + (size_t)NSLOT * k);
    }
    return sizeof(int) * ((size_t)2 * CH * bs.nrow * bs.ncol + (size_t)bs.F * k);
}

int sat_pitch(int W) { return (W + 1 + 3) / 4 * 4; }
int sat_strips(int W) { return (W + 1 + SW - 1) / SW; }
int score_ncol(int tw) { return (TXW + tw + 3) / 4 * 4; }

cudaError_t launch_sat(const uint8_t *lab, int H, int W, int k, int *carry, int *S, cudaStream_t s)
{
    const int nS = sat_strips(W);
    const int P = sat_pitch(W);
    const size_t hsmem = sizeof(int) * (size_t)nS * k;
    cudaError_t e = cudaFuncSetAttribute(row_carry_kernel,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)hsmem);
    if (e != cudaSuccess) return e;
    row_carry_kernel<<<H, 256, hsmem, s>>>(lab, W, k, nS, carry);
    const int nwarps = nS * ((k + CGW - 1) / CGW);
    sat_sweep_kernel<<<(nwarps + 3) / 4, 128, 0, s>>>(lab, H, W, k, P, nS, carry, S);
    return cudaGetLastError();
}

cudaError_t launch_filter_responses(const uint8_t *lab, int h, int w, int k, const BankSpec &bs,
                                    int32_t *counts, cudaStream_t s)
{
    (void)h;
    filter_responses_kernel<<<bs.F, 256, 0, s>>>(lab, w, k, bs, counts);
    return cudaGetLastError();
}

cudaError_t launch_score(const int *S, int W, int k, int HO, int WO, const BankSpec &bs,
                         const GridSpec &gs, const int32_t *tc, float *heat,
                         unsigned long long *amax, int32_t *argmax_yx, cudaStream_t s)
{
    const int P = sat_pitch(W);
    cudaError_t e = cudaSuccess;
    if (amax) {
        e = cudaMemsetAsync(amax, 0, sizeof(unsigned long long), s);
        if (e != cudaSuccess) return e;
    }
    bool done = false;
#define VQNNF_GRID_CASE(GG, FF)                                                         \
    if (!done && gs.G == GG && gs.full == FF) {                                         \
        e = launch_grid<GG, FF>(S, P, k, HO, WO, gs, tc, heat, amax, s);                 \
        done = true;                                                                    \
    }
    VQNNF_GRID_CASE(1, false) VQNNF_GRID_CASE(1, true) VQNNF_GRID_CASE(2, false)
    VQNNF_GRID_CASE(2, true) VQNNF_GRID_CASE(3, false) VQNNF_GRID_CASE(3, true)
    VQNNF_GRID_CASE(4, false) VQNNF_GRID_CASE(4, true)
#undef VQNNF_GRID_CASE
    if (!done) {
        const size_t smem = score_smem_bytes(bs, gs, k);
        e = cudaFuncSetAttribute(score_generic_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)smem);
        if (e != cudaSuccess) return e;
        dim3 grid((WO + TXW - 1) / TXW, HO);
        score_generic_kernel<<<grid, STH, smem, s>>>(S, P, k, HO, WO, bs, tc, heat, amax);
        e = cudaGetLastError();
    }
    if (e != cudaSuccess) return e;
    if (argmax_yx && amax) {
        argmax_finish_kernel<<<1, 1, 0, s>>>(amax, WO, argmax_yx);
        e = cudaGetLastError();
    }
    return e;
}

}  // namespace vqnnf
