// Soft-VQ backward contractions on the tensor cores (tcgen05, BF16 operands split three ways,
// FP32 accumulation in tensor memory).  For a pixel u with features x_u, the kept soft
// assignment p(u) and the adjoint g(u) = dL/dp(u) (Eq. 2 through the cell sums):
//   a_j(u)  = -(1/tau) p_j (g_j - sum_i p_i g_i)                       (softmax backward)
//   dX_u    = 2 (sum_j a_j(u)) x_u - 2 sum_j a_j(u) c_j                 (GEMM 1: A . C)
//   Y_j     = sum_u a_j(u) x_u,   S_j = sum_u a_j(u)                    (GEMM 2: A^T . X)
// and dL/dc_j = 2 S_j c_j - 2 Y_j, summed over the per-CTA partials afterwards.
//
// Each operand v is split v = hi + lo with hi = bf16(v), lo = bf16(v - hi); the products
// hi.hi + hi.lo + lo.hi leave out lo.lo and the rounding of lo, together at most ~3 * 2^-18 of
// |a| |c| (or |a| |x|) per term, far inside the 1e-3-of-largest-entry gradient tolerance.
//
// One CTA per SM over 128-pixel tiles; per tile, all 256 threads
//   1. form a for the tile (thread: one pixel, half of the centroids) and store it twice in
//      shared memory, as A [pixel][centroid] and A^T [centroid][pixel] (K-major, 128-byte
//      swizzle, hi and lo planes), and reduce it over the tile's pixels per centroid (S_j);
//   2. per 128-wide feature chunk m: store the chunk of X (thread: one feature, 64 pixels,
//      loaded into registers during the previous chunk) as X^T [feature][pixel] hi/lo; one
//      thread issues
//        GEMM 1  acc1[d][u]   = C^T_m (128 features x kp)  . A^T      (kp = k rounded up to 16)
//        GEMM 2  acc2_m[d][j] += X^T_m (128 features x 128 px) . (A^T)^T
//      and while they run the threads load the next chunk's features; then they read acc1 back
//      for dX = 2 (s_u x_u - acc1) (tensor-memory lane = feature), x_u = hi + lo from the
//      planes (within 2^-17 relative of x_u).
// C^T (hi and lo, every chunk) is loaded once per CTA from an image built by ct_image_kernel.
// acc2 stays in tensor memory across the CTA's tiles and is written out once at the end.
#include <cuda_bf16.h>

#include <algorithm>

#include "common.cuh"
#include "ptx.cuh"
#include "soft_spec.cuh"

namespace vqnnf {
namespace {

__device__ int g_soft_error = 0;

constexpr int UP = 128;                 // pixels per tile
constexpr int UNT = 256;                // threads per CTA (8 warps)
constexpr int ATOM = 128 * 128;         // bytes of a 128-row x 128-byte swizzled block
constexpr int kSmemLimit = 232448;      // opt-in shared memory per block

struct SoftTcArgs {
    const float *X;
    long long n, npi;
    int D, k, nd;
    float inv_tau;
    const float *P, *G;                 // planar: [(item * k + j) * npi + pixel]
    const uint8_t *ct;                  // C^T image: [hi, lo][nd][ATOM]
    float *dX;                          // null: no feature gradient (template pixels)
    float *part;                        // [gridDim.x][k D + k]: Y_j[d] at j D + d, S_j at k D + j
    int ntiles;
    uint32_t tmem_cols;
};

__host__ __device__ constexpr int smem_bytes_for(int kp, int nd)
{
    return 1024 + 2 * ATOM + 2 * 2 * kp * 128 + 4 * ATOM + 2 * nd * ATOM   // A, A^T, X^T, C^T
           + 4 * UP * 4 + 4 * kp * 4 + 64;                                   // sums, barriers
}

// Bounded wait on an mbarrier phase; on timeout the error word is set.
__device__ __forceinline__ bool wait_bounded(uint64_t *bar, uint32_t parity)
{
    return ptx::mbar_wait_for(bar, parity, &g_soft_error, (int)VQNNF_ETIMEOUT, ptx::kWaitCycles);
}

__device__ __forceinline__ uint32_t split_bf16(float v)      // hi | lo << 16
{
    const __nv_bfloat16 h = __float2bfloat16_rn(v);
    const __nv_bfloat16 l = __float2bfloat16_rn(v - __bfloat162float(h));
    return (uint32_t)__bfloat16_as_ushort(h) | ((uint32_t)__bfloat16_as_ushort(l) << 16);
}

// Byte offset of element (row, col) in a K-major 128-byte-swizzled block of 64 columns.
__device__ __forceinline__ uint32_t sw_off(int row, int col)
{
    return (uint32_t)((row >> 3) * 1024 + (row & 7) * 128 + ((((col >> 3) ^ row) & 7) << 4) + (col & 7) * 2);
}

template <int KP>
__global__ void __launch_bounds__(UNT, 1) soft_grad_tc_kernel(const __grid_constant__ SoftTcArgs g)
{
    constexpr int KH = KP / 2;                                   // centroids per thread in step 1
    extern __shared__ uint8_t smem_raw[];
    uint8_t *base = reinterpret_cast<uint8_t *>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
    const int nd = g.nd;
    uint8_t *sA = base;                                          // [hi, lo] x ATOM
    uint8_t *sAT = sA + 2 * ATOM;                                // [hi, lo] x 2 pixel atoms x KP rows
    uint8_t *sXT = sAT + 2 * 2 * KP * 128;                       // [hi, lo] x 2 pixel atoms x 128 rows
    uint8_t *sCT = sXT + 4 * ATOM;                               // [hi, lo] x nd x ATOM
    float *spg = reinterpret_cast<float *>(sCT + 2 * nd * ATOM); // [2][UP] partial sum_j p_j g_j
    float *sas = spg + 2 * UP;                                   // [2][UP] partial sum_j a_j
    float *scol = sas + 2 * UP;                                  // [4][KP] per-centroid sums
    uint64_t *bar = reinterpret_cast<uint64_t *>(scol + 4 * KP); // [0] C^T loaded, [1] MMAs done
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(bar + 2);

    const int t = threadIdx.x, warp = t >> 5, lane = t & 31;
    if (t == 0) {
        ptx::mbar_init(&bar[0], 1);
        ptx::mbar_init(&bar[1], 1);
        ptx::fence_barrier_init();
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(ptx::smem_u32(tmem_slot)),
                     "r"(g.tmem_cols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    ptx::tc_fence_before();
    __syncthreads();
    ptx::tc_fence_after();
    const uint32_t tmem = *tmem_slot;
    if (t == 0) {
        ptx::mbar_expect_tx(&bar[0], (uint32_t)(2 * nd * ATOM));
        for (int b = 0; b < 2 * nd; ++b) ptx::bulk_g2s(sCT + b * ATOM, g.ct + (size_t)b * ATOM, ATOM, &bar[0]);
    }
    bool ok = !__syncthreads_or(!wait_bounded(&bar[0], 0));

    const int pp = t & (UP - 1), hf = t >> 7;                   // step 1: pixel, centroid half
    const int q4 = warp & 3, pxh = warp >> 2;                   // step 2: lane quadrant, pixel half
    const int dl = 32 * q4 + lane;                              // feature row within a chunk
    const uint32_t id1 = ptx::bf16_idesc(128, UP), id2 = ptx::bf16_idesc(128, KP);
    // this thread's 64 pixels of feature column 128 m + dl of the tile at pixel p0n
    float xv[64];
    auto load_x = [&](long long p0n, int mn) {
        const int dc = 128 * mn + dl;
        const bool dvn = dc < g.D;
#pragma unroll
        for (int q = 0; q < 64; ++q) {
            const long long u = p0n + 64 * pxh + q;
            xv[q] = (dvn && u < g.n) ? g.X[u * g.D + dc] : 0.f;
        }
    };
    if (ok && (int)blockIdx.x < g.ntiles) load_x((long long)blockIdx.x * UP, 0);
    uint32_t phase = 0;
    float sacc = 0.f;                                           // S_j, j = hf KH + lane (lane < KH)
    bool first = true;
    for (int tile = blockIdx.x; ok && tile < g.ntiles; tile += gridDim.x) {
        const long long p0 = (long long)tile * UP;
        // ---- 1. softmax backward for pixel pp, centroids hf KH .. hf KH + KH - 1
        float pv[KH], gv[KH];
        {
            const long long u = p0 + pp;
            const bool in = u < g.n;
            const long long it = in ? u / g.npi : 0, pix = in ? u - it * g.npi : 0;
            const size_t b0 = (size_t)(it * g.k) * g.npi + pix;
            float s = 0.f;
#pragma unroll
            for (int i = 0; i < KH; ++i) {
                const int j = hf * KH + i;
                const bool v = in && j < g.k;
                pv[i] = v ? g.P[b0 + (size_t)j * g.npi] : 0.f;
                gv[i] = v ? g.G[b0 + (size_t)j * g.npi] : 0.f;
                s = fmaf(pv[i], gv[i], s);
            }
            spg[hf * UP + pp] = s;
        }
        __syncthreads();
        {
            const float s = spg[pp] + spg[UP + pp];
            float as = 0.f;
            uint32_t hw[KH];
#pragma unroll
            for (int i = 0; i < KH; ++i) {
                const float a = -g.inv_tau * pv[i] * (gv[i] - s);
                pv[i] = a;
                as += a;
                hw[i] = split_bf16(a);
            }
            sas[hf * UP + pp] = as;
            // A [pixel][centroid]: 8 centroids per 16-byte store, hi and lo planes
#pragma unroll
            for (int c = 0; c < KH / 8; ++c) {
                uint4 h4, l4;
                uint32_t *hp = &h4.x, *lp = &l4.x;
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    const uint32_t a0 = hw[8 * c + 2 * q], a1 = hw[8 * c + 2 * q + 1];
                    hp[q] = (a0 & 0xFFFFu) | (a1 << 16);
                    lp[q] = (a0 >> 16) | (a1 & 0xFFFF0000u);
                }
                const uint32_t o = sw_off(pp, hf * KH + 8 * c);
                *reinterpret_cast<uint4 *>(sA + o) = h4;
                *reinterpret_cast<uint4 *>(sA + ATOM + o) = l4;
            }
            // A^T [centroid][pixel]: lane pairs swap so that each stores two pixels of one row
            const int odd = pp & 1;
#pragma unroll
            for (int i = 0; i < KH; i += 2) {
                const uint32_t send = odd ? hw[i] : hw[i + 1];
                const uint32_t recv = __shfl_xor_sync(0xffffffffu, send, 1);
                uint32_t wh, wl;
                if (odd) {
                    wh = (recv & 0xFFFFu) | (hw[i + 1] << 16);
                    wl = (recv >> 16) | (hw[i + 1] & 0xFFFF0000u);
                } else {
                    wh = (hw[i] & 0xFFFFu) | (recv << 16);
                    wl = (hw[i] >> 16) | (recv & 0xFFFF0000u);
                }
                const int row = hf * KH + i + odd, col = pp - odd;
                const uint32_t o = (uint32_t)(col >> 6) * (KP * 128) + sw_off(row, col & 63);
                *reinterpret_cast<uint32_t *>(sAT + o) = wh;
                *reinterpret_cast<uint32_t *>(sAT + 2 * KP * 128 + o) = wl;
            }
            // S_j over the warp's 32 pixels: reduce-scatter, lane l ends with centroid hf KH + l
            float v[32];
#pragma unroll
            for (int i = 0; i < 32; ++i) v[i] = i < KH ? pv[i] : 0.f;
#pragma unroll
            for (int sh = 16; sh >= 1; sh >>= 1) {
                const bool up = lane & sh;
#pragma unroll
                for (int i = 0; i < sh; ++i) {
                    const float send = up ? v[i] : v[i + sh];
                    const float keep = up ? v[i + sh] : v[i];
                    v[i] = keep + __shfl_xor_sync(0xffffffffu, send, sh);
                }
            }
            sacc += v[0];
        }
        // ---- 2. feature chunks (this chunk's features were loaded during the previous one)
        for (int m = 0; m < nd; ++m) {
            const int dcol = 128 * m + dl;
            const bool dv = dcol < g.D;
#pragma unroll
            for (int c = 0; c < 8; ++c) {
                uint4 h4, l4;
                uint32_t *hp = &h4.x, *lp = &l4.x;
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    const uint32_t a0 = split_bf16(xv[8 * c + 2 * q]), a1 = split_bf16(xv[8 * c + 2 * q + 1]);
                    hp[q] = (a0 & 0xFFFFu) | (a1 << 16);
                    lp[q] = (a0 >> 16) | (a1 & 0xFFFF0000u);
                }
                const uint32_t o = (uint32_t)pxh * ATOM + sw_off(dl, 8 * c);
                *reinterpret_cast<uint4 *>(sXT + o) = h4;
                *reinterpret_cast<uint4 *>(sXT + 2 * ATOM + o) = l4;
            }
            ptx::fence_proxy_async();
            ptx::tc_fence_before();
            __syncthreads();
            if (t == 0) {
                ptx::tc_fence_after();
                if (g.dX) {                                     // GEMM 1: acc1 = C^T_m . A^T
                    const uint32_t ch = ptx::smem_u32(sCT) + m * ATOM, cl = ch + nd * ATOM;
                    const uint32_t ah = ptx::smem_u32(sA), al = ah + ATOM;
#pragma unroll
                    for (int kk = 0; kk < KP / 16; ++kk) {
                        const uint64_t dch = ptx::sw128_desc(ch) + 2 * kk, dcl = ptx::sw128_desc(cl) + 2 * kk;
                        const uint64_t dah = ptx::sw128_desc(ah) + 2 * kk, dal = ptx::sw128_desc(al) + 2 * kk;
                        ptx::tc_mma_bf16_ss(tmem, dch, dah, id1, kk > 0);
                        ptx::tc_mma_bf16_ss(tmem, dch, dal, id1, 1);
                        ptx::tc_mma_bf16_ss(tmem, dcl, dah, id1, 1);
                    }
                }
                {                                               // GEMM 2: acc2_m += X^T_m . A
                    const uint32_t xh = ptx::smem_u32(sXT), xl = xh + 2 * ATOM;
                    const uint32_t bh = ptx::smem_u32(sAT), bl = bh + 2 * KP * 128;
                    const uint32_t d2 = tmem + UP + m * KP;
#pragma unroll
                    for (int kk = 0; kk < UP / 16; ++kk) {
                        const int at = kk >> 2, sub = kk & 3;
                        const uint64_t dxh = ptx::sw128_desc(xh + at * ATOM) + 2 * sub;
                        const uint64_t dxl = ptx::sw128_desc(xl + at * ATOM) + 2 * sub;
                        const uint64_t dbh = ptx::sw128_desc(bh + at * KP * 128) + 2 * sub;
                        const uint64_t dbl = ptx::sw128_desc(bl + at * KP * 128) + 2 * sub;
                        ptx::tc_mma_bf16_ss(d2, dxh, dbh, id2, !(first && kk == 0));
                        ptx::tc_mma_bf16_ss(d2, dxh, dbl, id2, 1);
                        ptx::tc_mma_bf16_ss(d2, dxl, dbh, id2, 1);
                    }
                }
                ptx::tc_commit(&bar[1]);
            }
            // the next chunk's features (of this tile, else of the CTA's next tile) are loaded
            // while the MMAs run; the epilogue below takes x from the hi and lo planes
            if (m + 1 < nd) load_x(p0, m + 1);
            else if (tile + (int)gridDim.x < g.ntiles) load_x(p0 + (long long)gridDim.x * UP, 0);
            const bool w_ok = wait_bounded(&bar[1], phase);
            phase ^= 1;
            if (__syncthreads_or(!w_ok)) {
                ok = false;
                break;
            }
            ptx::tc_fence_after();
            if (g.dX) {                                         // dX = 2 (s_u x_u - acc1)
#pragma unroll
                for (int hh = 0; hh < 2; ++hh) {
                    float acc[32];
                    ptx::tc_ld32(tmem + ((uint32_t)(32 * q4) << 16) + 64 * pxh + 32 * hh, acc);
#pragma unroll
                    for (int c = 0; c < 4; ++c) {
                        const uint32_t o = (uint32_t)pxh * ATOM + sw_off(dl, 32 * hh + 8 * c);
                        const uint4 h4 = *reinterpret_cast<const uint4 *>(sXT + o);
                        const uint4 l4 = *reinterpret_cast<const uint4 *>(sXT + 2 * ATOM + o);
                        const uint32_t hw[4] = {h4.x, h4.y, h4.z, h4.w}, lw[4] = {l4.x, l4.y, l4.z, l4.w};
#pragma unroll
                        for (int e = 0; e < 8; ++e) {
                            const uint32_t hb = e & 1 ? hw[e >> 1] & 0xFFFF0000u : hw[e >> 1] << 16;
                            const uint32_t lb = e & 1 ? lw[e >> 1] & 0xFFFF0000u : lw[e >> 1] << 16;
                            const float x = __uint_as_float(hb) + __uint_as_float(lb);   // hi + lo
                            const int px = 64 * pxh + 32 * hh + 8 * c + e;
                            const long long u = p0 + px;
                            if (dv && u < g.n)
                                g.dX[u * g.D + dcol] = 2.0f * ((sas[px] + sas[UP + px]) * x - acc[8 * c + e]);
                        }
                    }
                }
            }
            ptx::tc_fence_before();
        }
        first = false;
    }
    __syncthreads();
    ptx::tc_fence_after();
    if (ok && !first) {
        float *part = g.part + (size_t)blockIdx.x * ((size_t)g.k * g.D + g.k);
        for (int m = pxh; m < nd; m += 2) {                     // Y: lane = feature, column = centroid
            const int dcol = 128 * m + dl;
#pragma unroll
            for (int c = 0; c < KP / 8; ++c) {
                float v[8];
                ptx::tc_ld8(tmem + ((uint32_t)(32 * q4) << 16) + UP + m * KP + 8 * c, v);
#pragma unroll
                for (int i = 0; i < 8; ++i) {
                    const int j = 8 * c + i;
                    if (j < g.k && dcol < g.D) part[(size_t)j * g.D + dcol] = v[i];
                }
            }
        }
        if (lane < KH) scol[q4 * KP + hf * KH + lane] = sacc;
        __syncthreads();
        if (t < g.k) part[(size_t)g.k * g.D + t] = scol[t] + scol[KP + t] + scol[2 * KP + t] + scol[3 * KP + t];
    }
    ptx::tc_fence_before();
    __syncthreads();
    if (warp == 0) {
        ptx::tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(g.tmem_cols)
                     : "memory");
    }
}

// C^T image in the kernel's shared-memory layout: element (d, j) of feature chunk m at
// [plane][m][sw_off(d, j)], hi plane then lo plane; one thread per 8 centroids of one feature.
__global__ void ct_image_kernel(const float *__restrict__ C, int k, int D, int nd, uint8_t *__restrict__ img)
{
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= nd * 128 * 8) return;
    const int jc = e & 7, d = (e >> 3) & 127, m = e >> 10;
    const int dg = 128 * m + d;
    uint4 h4, l4;
    uint32_t *hp = &h4.x, *lp = &l4.x;
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        const int j0 = 8 * jc + 2 * q;
        const float c0 = (j0 < k && dg < D) ? C[(size_t)j0 * D + dg] : 0.f;
        const float c1 = (j0 + 1 < k && dg < D) ? C[(size_t)(j0 + 1) * D + dg] : 0.f;
        const uint32_t a0 = split_bf16(c0), a1 = split_bf16(c1);
        hp[q] = (a0 & 0xFFFFu) | (a1 << 16);
        lp[q] = (a0 >> 16) | (a1 & 0xFFFF0000u);
    }
    const size_t o = (size_t)m * ATOM + sw_off(d, 8 * jc);
    *reinterpret_cast<uint4 *>(img + o) = h4;
    *reinterpret_cast<uint4 *>(img + (size_t)nd * ATOM + o) = l4;
}

int kp_of(int k) { return (k + 15) / 16 * 16; }

template <int KP>
cudaError_t launch_kp(const SoftTcArgs &a, int grid, cudaStream_t s)
{
    const int sm = smem_bytes_for(KP, a.nd);
    cudaError_t e = cudaFuncSetAttribute(soft_grad_tc_kernel<KP>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm);
    if (e != cudaSuccess) return e;
    soft_grad_tc_kernel<KP><<<grid, UNT, sm, s>>>(a);
    return cudaGetLastError();
}

}  // namespace

bool soft_tc_supported(int D, int k)
{
    if (k < 1 || k > 64 || D < 1) return false;
    const int kp = kp_of(k), nd = (D + 127) / 128;
    return smem_bytes_for(kp, nd) <= kSmemLimit && UP + nd * kp <= 512;
}

size_t soft_ct_image_bytes(int D) { return (size_t)2 * ((D + 127) / 128) * ATOM; }

cudaError_t launch_soft_ct_image(const float *C, int k, int D, uint8_t *img, cudaStream_t s)
{
    const int nd = (D + 127) / 128;
    ct_image_kernel<<<(nd * 1024 + 255) / 256, 256, 0, s>>>(C, k, D, nd, img);
    return cudaGetLastError();
}

cudaError_t launch_soft_grad_tc(const float *X, long long n, long long npi, int D, int k, float tau,
                                const float *P, const float *G, const uint8_t *ct_img, float *dX, float *part,
                                int max_slices, int *slices, cudaStream_t s)
{
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    SoftTcArgs a;
    a.X = X;
    a.n = n;
    a.npi = npi;
    a.D = D;
    a.k = k;
    a.nd = (D + 127) / 128;
    a.inv_tau = 1.0f / tau;
    a.P = P;
    a.G = G;
    a.ct = ct_img;
    a.dX = dX;
    a.part = part;
    a.ntiles = (int)((n + UP - 1) / UP);
    const int kp = kp_of(k);
    uint32_t cols = 32;
    while (cols < (uint32_t)(UP + a.nd * kp)) cols <<= 1;
    a.tmem_cols = cols;
    const int grid = std::max(1, std::min({a.ntiles, sms, max_slices}));
    *slices = grid;
    switch (kp) {
    case 16: return launch_kp<16>(a, grid, s);
    case 32: return launch_kp<32>(a, grid, s);
    case 48: return launch_kp<48>(a, grid, s);
    case 64: return launch_kp<64>(a, grid, s);
    default: return cudaErrorInvalidValue;
    }
}

cudaError_t read_and_clear_soft_error(int *out)
{
    int zero = 0;
    cudaError_t e = cudaMemcpyFromSymbol(out, g_soft_error, sizeof(int));
    if (e == cudaSuccess) e = cudaMemcpyToSymbol(g_soft_error, &zero, sizeof(int));
    return e;
}

}  // namespace vqnnf
