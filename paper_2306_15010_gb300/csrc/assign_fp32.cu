// Nearest-neighbour field (Algorithm 1) -- codebook preparation, the FP32 SIMT distance
// contraction with bound-driven near-tie flagging, and the compensated re-scoring stage
// shared by both precisions.
//
// Distances.  For a pixel x and centroid c_j the contraction computes
//     s_j = ||c_j - m||^2 - 2 (x - m) . (c_j - m)  =  ||x - c_j||^2 - ||x - m||^2
// with m the FP32 mean of the codebook (centring shrinks the norms that scale the
// rounding error; the argmin over j is unchanged).  A proven per-pixel bound B_j on
// |s_j - exact| gives an interval for every distance; the pixel's label is decided when
// exactly one interval reaches below the smallest upper end, otherwise the pixel and its
// candidate set go to the re-scoring stage, which decides them from the uncentred FP32
// inputs in compensated arithmetic.
//
// Bound (u = 2^-24, X = ||x'|| with x' = fl(x - m), Delta = ||x' - A-operand||):
//     B_j = X a_j + (Delta + u (X + Delta)(1 + 4u)) v_j + b_j + 4u |s_j|,  inflated by 2^-8
// with per-centroid a_j, v_j, b_j written by prep_codebook (derivation in the design
// notes: contraction accumulation error, rounding of the centred codebook and of x').
#include <cuda_bf16.h>
#include <cuda_fp8.h>

#include <cfloat>

#include <algorithm>

#include "common.cuh"
#include "ptx.cuh"

namespace vqnnf {
namespace {

constexpr double kU32 = 5.9604644775390625e-08;  // 2^-24

// ----------------------------------------------------------------------------------
// Codebook preparation: reference point, centred copies and bound terms.
// ----------------------------------------------------------------------------------
// The reference point m only has to be the same FP32 vector for every use (the bound holds
// for any m); the codebook mean keeps the centred norms small.  Four interleaved FP32 partial
// sums in a fixed order: deterministic and short.
__global__ void __launch_bounds__(256) prep_mean_kernel(const float *__restrict__ C, int k, int D,
                                                        float *mean, unsigned *zero64)
{
    ptx::pdl_enter();
    // the flag list's counter and statistics words start at zero (one launch fewer than a memset)
    if (zero64 && blockIdx.x == 0 && threadIdx.x < 64) zero64[threadIdx.x] = 0u;
    // block: 32 dimensions x 8 row groups; partial sums combined in a fixed order
    __shared__ float part[8][33];
    const int i = blockIdx.x * 32 + (threadIdx.x & 31);
    const int g = threadIdx.x >> 5;
    float s = 0.f;
    if (i < D)
        for (int j = g; j < k; j += 8) s += C[(size_t)j * D + i];
    part[g][threadIdx.x & 31] = s;
    __syncthreads();
    if (g == 0 && i < D) {
        float t = 0.f;
#pragma unroll
        for (int q = 0; q < 8; ++q) t += part[q][threadIdx.x];
        mean[i] = t / (float)k;
    }
}

// Error-free transformations in FP32 (Knuth's TwoSum; the FMA product error).
__device__ __forceinline__ void two_sum(float a, float b, float &s, float &e)
{
    s = __fadd_rn(a, b);
    const float bv = __fsub_rn(s, a);
    const float av = __fsub_rn(s, bv);
    e = __fadd_rn(__fsub_rn(a, av), __fsub_rn(b, bv));
}

// BF16 rounding (to nearest, ties to even) of the exact value v = f + e, where f = fl32(v):
// identical to rounding f except when f sits exactly halfway between two BF16 values and
// e != 0, where the exact value lies on the side of e.
__device__ __forceinline__ uint32_t bf16_round_exact(float f, float e)
{
    const uint32_t bits = __float_as_uint(f);
    if ((bits & 0xFFFFu) == 0x8000u && e != 0.0f) {
        const uint32_t down = bits & 0xFFFF0000u;          // toward zero
        const bool away = (e > 0.0f) == (f > 0.0f);
        return (away ? down + 0x10000u : down) >> 16;
    }
    return __bfloat16_as_ushort(__float2bfloat16_rn(f));
}

__device__ __forceinline__ float bf16_value(uint32_t h) { return __uint_as_float(h << 16); }

// The power of two s with s >= amax / 448 > s / 2 (at least 2^-100): dividing by s is exact in
// FP32 and brings every value of magnitude <= amax to at most 448, the largest e4m3 value.
__device__ __forceinline__ float pow2_scale(float amax)
{
    const float t = amax * (1.0f / 448.0f);           // correctly rounded; checked below
    if (!(t > 0x1p-100f)) return 0x1p-100f;
    int e;
    frexpf(t, &e);                                    // t = f 2^e, f in [0.5, 1)
    float s = ldexpf(1.0f, e);                        // s >= t
    if (amax / s > 448.0f) s *= 2.0f;                 // t rounded below amax / 448
    return s;
}

// One block per centroid, FP32 error-free arithmetic (the FP64 pipe of this GPU is narrow):
// c* = c - m exactly as cf + d32 (TwoSum), the BF16 splits hi = bf16(c*), lo = bf16(c* - hi)
// of the exact values, ||c*||^2 as a compensated sum of the exact squares (FMA products),
// and upper bounds of the other norms (sums of squares inflated by their summation bound).
// The block reduction has a fixed tree order (deterministic).
__global__ void __launch_bounds__(256) prep_centroid_kernel(const float *__restrict__ C, int k,
                                                            int D, int prec, CodebookPrep p, unsigned *zero64)
{
    ptx::pdl_enter();
    if (zero64 && blockIdx.x == 0 && threadIdx.x < 64) zero64[threadIdx.x] = 0u;   // see prep_mean_kernel
    const int j = blockIdx.x;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    __shared__ float red[8][8];
    __shared__ float s_amax[8];
    // FP8 path: the centroid's power-of-two scale s = 2^ceil(log2(max |fl32(c*)| / 448)), so
    // that every fl32(c*_i) / s is exact in FP32 and at most 448 (the largest e4m3 value)
    float csc = 1.0f;
    if (prec == VQNNF_PREC_FP8) {
        float am = 0.f;
        for (int i = threadIdx.x; i < D; i += blockDim.x) {
            float cf, d32;
            two_sum(C[(size_t)j * D + i], -p.mean[i], cf, d32);
            am = fmaxf(am, fabsf(cf));
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) am = fmaxf(am, __shfl_xor_sync(0xffffffffu, am, o));
        if (lane == 0) s_amax[w] = am;
        __syncthreads();
        am = s_amax[0];
        for (int q = 1; q < (int)(blockDim.x >> 5); ++q) am = fmaxf(am, s_amax[q]);
        csc = pow2_scale(am);
    }
    float S = 0.f, Sc = 0.f, Q = 0.f;                 // ||c*||^2: main sum, its compensation, small terms
    float s_cc2 = 0.f, s_d32 = 0.f, s_hi2 = 0.f, s_lo2 = 0.f, s_d16 = 0.f;
    for (int i = threadIdx.x; i < D; i += blockDim.x) {
        const float c = C[(size_t)j * D + i], m = p.mean[i];
        float cf, d32;
        two_sum(c, -m, cf, d32);                      // c - m = cf + d32 exactly
        p.cc[(size_t)j * D + i] = cf;
        const uint32_t hb = bf16_round_exact(cf, d32);
        const float hf = bf16_value(hb);
        float rf, rd;
        two_sum(__fsub_rn(cf, hf), d32, rf, rd);      // r = c* - hi = rf + rd (cf - hf is exact)
        const uint32_t lb = bf16_round_exact(rf, rd);
        const float lf = bf16_value(lb);
        const float d16 = fabsf(__fsub_rn(rf, lf)) + fabsf(rd);   // >= |r - lo| (rf - lf exact)
        p.chi[(size_t)j * D + i] = (uint16_t)hb;
        p.clo[(size_t)j * D + i] = (uint16_t)lb;
        if (prec == VQNNF_PREC_FP8)                   // cf / csc is exact (power-of-two scale)
            p.cq8[(size_t)j * D + i] = (uint8_t)__nv_cvt_float_to_fp8(cf / csc, __NV_SATFINITE, __NV_E4M3);
        // c*^2 = cf^2 + 2 cf d32 + d32^2, cf^2 = pp + pe exactly
        const float pp = __fmul_rn(cf, cf), pe = fmaf(cf, cf, -pp);
        float t, te;
        two_sum(S, pp, t, te);
        S = t;
        Sc += te;
        Q += pe + 2.0f * cf * d32 + d32 * d32;
        s_cc2 = fmaf(cf, cf, s_cc2);
        s_d32 = fmaf(d32, d32, s_d32);
        s_hi2 = fmaf(hf, hf, s_hi2);
        s_lo2 = fmaf(lf, lf, s_lo2);
        s_d16 = fmaf(d16, d16, s_d16);
    }
    // warp then block tree: (S, Sc) added as double-floats, the rest plainly
    float v8[8] = {S, Sc, Q, s_cc2, s_d32, s_hi2, s_lo2, s_d16};
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        float o8[8];
#pragma unroll
        for (int q = 0; q < 8; ++q) o8[q] = __shfl_xor_sync(0xffffffffu, v8[q], o);
        float t, te;
        two_sum(v8[0], o8[0], t, te);
        v8[0] = t;
        v8[1] = v8[1] + o8[1] + te;
#pragma unroll
        for (int q = 2; q < 8; ++q) v8[q] += o8[q];
    }
    if (lane == 0)
#pragma unroll
        for (int q = 0; q < 8; ++q) red[w][q] = v8[q];
    __syncthreads();
    if (threadIdx.x == 0) {
        const int nw = blockDim.x >> 5;
        float tot[8];
#pragma unroll
        for (int q = 0; q < 8; ++q) tot[q] = red[0][q];
        for (int u2 = 1; u2 < nw; ++u2) {
            float t, te;
            two_sum(tot[0], red[u2][0], t, te);
            tot[0] = t;
            tot[1] = tot[1] + red[u2][1] + te;
#pragma unroll
            for (int q = 2; q < 8; ++q) tot[q] += red[u2][q];
        }
        const double u = kU32;
        // ||c*||^2: the compensated sum is within (2u + 2 D u^2) of the exact value (plus the
        // small terms' own rounding, relative u^2 D); n32 rounds it once more
        const float n32 = __fadd_rn(tot[0], tot[1] + tot[2]);
        const double c2 = (double)n32;
        const double en = 4.0 * u * c2 + 1e-37;                 // >= |n32 - ||c*||^2|
        // other norms: sums of D non-negative terms are within gamma_D of the exact value
        const double up = 1.0 + (2.0 * D + 8.0) * u;
        const double margin = 1.0 + 4.0 * u;
        const double nc = sqrt((c2 + en) * up) * margin;        // ||c*||
        const double ncc = sqrt((double)tot[3] * up) * margin;  // ||fl32(c*)||
        const double nd32 = sqrt((double)tot[4] * up) * margin; // ||c* - fl32(c*)||
        const double nhi = sqrt((double)tot[5] * up) * margin;
        const double nlo = sqrt((double)tot[6] * up) * margin;
        const double nd16 = sqrt((double)tot[7] * up) * margin;
        double a, v;
        if (prec == VQNNF_PREC_FP32) {
            const double gD = (double)D * u / (1.0 - (double)D * u);
            a = 2.0 * gD * ncc + 2.0 * (1.0 + 2.0 * u) * nd32;
            v = 2.0 * (ncc > nc ? ncc : nc);
        } else if (prec == VQNNF_PREC_FP8) {
            // e4m3 of fl32(c*) / s, round to nearest: each element within 2^-4 of its value, or
            // within 2^-10 s absolute below the normal range; so with q the centroid's FP8 row,
            //   ||c* - s q|| <= 2^-4 ||fl32(c*)|| + 2^-10 s sqrt(D) + ||c* - fl32(c*)||  (= dc)
            //   ||s q||      <= (1 + 2^-4) ||fl32(c*)|| + 2^-10 s sqrt(D)              (= nq)
            // The products of two e4m3 values are exact in FP32; the accumulation order and
            // rounding of the tensor core are not documented: four times the sequential FP32
            // bound (gacc).  The dot product's error is then at most
            //   X (dc + gacc nq) + ||x' - s_x q_x|| ||c*||,  X >= ||s_x q_x||
            const double sub = 0.0009765625 * (double)csc * sqrt((double)D) * margin;
            const double dc = 0.0625 * ncc + sub + nd32;
            const double nq = (1.0 + 0.0625) * ncc + sub;
            const double gacc = (double)D * 4.0 * u;
            a = 2.0 * (dc + gacc * nq) * (1.0 + 4.0 * u);
            v = 2.0 * nc;
            p.csc[j] = csc;
        } else {
            // Three BF16 products x_hi.hi + x_hi.lo + x_lo.hi.  Tensor-core accumulation
            // order and rounding are not documented: take four times the sequential FP32
            // bound.  The x_lo terms (||x_lo|| <= 2^-8 ||x_hi||) are folded into a_j:
            //   |err| <= X [gacc (|hi| + |lo|) + |d|] + X_lo [gacc |hi| + |lo| + |d|] + ...
            const double gacc = (double)D * 4.0 * u;
            a = 2.0 * (gacc * (nhi + nlo) + nd16) + 2.0 * 0.00390625 * (gacc * nhi + nlo + nd16);
            v = 2.0 * nc;
        }
        p.nrm[j] = n32;
        p.a[j] = __double2float_ru(a);
        p.v[j] = __double2float_ru(v);
        p.b[j] = __double2float_ru(en);
    }
}

// ----------------------------------------------------------------------------------
// FP32 SIMT contraction: 128 pixels x 128 centroids per pass, 8 x 8 outputs per thread,
// sequential FMA accumulation over D (so the per-dot error is <= gamma_D sum |x c|).
// ----------------------------------------------------------------------------------
constexpr int BM = 128, BN = 128, BK = 16, NT = 256;

__device__ __forceinline__ void push_flag(bool flagged, unsigned int pix, const unsigned *mask,
                                          FlagList fl)
{
    const unsigned ballot = __ballot_sync(0xffffffffu, flagged);
    if (!ballot) return;
    const int lane = threadIdx.x & 31;
    const int leader = __ffs(ballot) - 1;
    unsigned base = 0;
    if (lane == leader) base = atomicAdd(fl.count, (unsigned)__popc(ballot));
    base = __shfl_sync(0xffffffffu, base, leader);
    if (flagged) {
        const unsigned slot = base + __popc(ballot & ((1u << lane) - 1u));
        fl.pix[slot] = pix;
#pragma unroll
        for (int w = 0; w < kMaskWords; ++w) fl.mask[(size_t)slot * kMaskWords + w] = mask[w];
    }
}

// Epilogue shared with the tensor-core path: decide or flag one pixel from its row of
// scores s_j (strided by `stride` floats), X = ||A-side vector||, Dl = rounding residual.
__device__ __forceinline__ int decide_pixel(const float *srow, int stride, int k, float X, float Dl,
                                            const float *ca, const float *cv, const float *cb,
                                            unsigned *mask, int *ncand)
{
    const float u = (float)kU32;
    const float Y = Dl + u * (X * 1.01f + Dl) * (1.0f + 4.0f * u);
    const float infl = 1.0f + 0.00390625f;
    float U = FLT_MAX, smin = FLT_MAX;
    int amin = 0;
    for (int j = 0; j < k; ++j) {
        const float s = srow[j * stride];
        const float B = fmaf(X, ca[j], fmaf(Y, cv[j], cb[j] + 4.0f * u * fabsf(s))) * infl;
        U = fminf(U, s + B);
        if (s < smin) { smin = s; amin = j; }
    }
#pragma unroll
    for (int w = 0; w < kMaskWords; ++w) mask[w] = 0u;
    int cnt = 0, last = amin;
    for (int j = 0; j < k; ++j) {
        const float s = srow[j * stride];
        const float B = fmaf(X, ca[j], fmaf(Y, cv[j], cb[j] + 4.0f * u * fabsf(s))) * infl;
        if (s - B <= U) {
            ++cnt;
            last = j;
            mask[j >> 5] |= 1u << (j & 31);
        }
    }
    *ncand = cnt;
    return cnt == 1 ? last : amin;
}

__global__ void __launch_bounds__(NT, 2) assign_fp32_kernel(const float *__restrict__ X, long long n,
                                                         int D, int k, CodebookPrep p,
                                                         uint8_t *__restrict__ labels, FlagList fl)
{
    ptx::pdl_enter();
    extern __shared__ __align__(16) float smem[];
    const int kp = (k + BN - 1) / BN * BN;
    const int sp = kp + 1;
    float *As = smem;                  // [2][BK][BM]
    float *Bs = As + 2 * BK * BM;      // [2][BK][BN]
    float *Sc = Bs + 2 * BK * BN;      // [BM][sp]
    float *ca = Sc + BM * sp;          // [kp]
    float *cv = ca + kp;
    float *cb = cv + kp;
    float *cn = cb + kp;
    float *xn = cn + kp;               // [2][BM]

    const int tid = threadIdx.x;
    const int tx = tid & 15, ty = tid >> 4;
    const long long p0 = (long long)blockIdx.x * BM;
    for (int j = tid; j < kp; j += NT) {
        const bool ok = j < k;
        const int jc = ok ? j : k - 1;
        ca[j] = ok ? p.a[jc] : 0.f;
        cv[j] = ok ? p.v[jc] : 0.f;
        cb[j] = ok ? p.b[jc] : 0.f;
        cn[j] = ok ? p.nrm[jc] : 0.f;
    }
    // loader mapping: row lp (pixel or centroid), dims lh*8 .. lh*8+7 of the k-step
    const int lp = tid >> 1, lh = tid & 1;
    const long long prow = p0 + lp;
    const bool prow_ok = prow < n;
    const float *xrow = X + (prow_ok ? prow : 0) * (long long)D;
    float xsq = 0.f;

    for (int nc = 0; nc < kp; nc += BN) {
        const int crow = nc + lp;
        const bool crow_ok = crow < k;
        const float *crw = p.cc + (size_t)(crow_ok ? crow : 0) * D;
        float acc[8][8];
#pragma unroll
        for (int a = 0; a < 8; ++a)
#pragma unroll
            for (int b = 0; b < 8; ++b) acc[a][b] = 0.f;

        float ra[8], rb[8];
        // Every load address is clamped into its buffer and out-of-range values are
        // zeroed afterwards: no address past a buffer is ever formed, even for loads the
        // compiler may issue ahead of their guard.
        auto gload = [&](int d0) {
#pragma unroll
            for (int q = 0; q < 2; ++q) {
                const int d = d0 + lh * 8 + q * 4;
                const bool din = d < D;
                const int dc = din ? d : D - 4;
                float4 xa = __ldg(reinterpret_cast<const float4 *>(xrow + dc));
                const float4 mm = __ldg(reinterpret_cast<const float4 *>(p.mean + dc));
                float4 cbv = __ldg(reinterpret_cast<const float4 *>(crw + dc));
                const bool xok = din && prow_ok, cok = din && crow_ok;
                xa.x = xok ? xa.x - mm.x : 0.f; xa.y = xok ? xa.y - mm.y : 0.f;
                xa.z = xok ? xa.z - mm.z : 0.f; xa.w = xok ? xa.w - mm.w : 0.f;
                cbv.x = cok ? cbv.x : 0.f; cbv.y = cok ? cbv.y : 0.f;
                cbv.z = cok ? cbv.z : 0.f; cbv.w = cok ? cbv.w : 0.f;
                ra[q * 4 + 0] = xa.x; ra[q * 4 + 1] = xa.y; ra[q * 4 + 2] = xa.z; ra[q * 4 + 3] = xa.w;
                rb[q * 4 + 0] = cbv.x; rb[q * 4 + 1] = cbv.y; rb[q * 4 + 2] = cbv.z; rb[q * 4 + 3] = cbv.w;
            }
        };
        auto sstore = [&](int buf) {
            float *a = As + buf * BK * BM;
            float *b = Bs + buf * BK * BN;
#pragma unroll
            for (int q = 0; q < 8; ++q) {
                a[(lh * 8 + q) * BM + lp] = ra[q];
                b[(lh * 8 + q) * BN + lp] = rb[q];
            }
        };
        gload(0);
        if (nc == 0)
#pragma unroll
            for (int q = 0; q < 8; ++q) xsq = fmaf(ra[q], ra[q], xsq);
        sstore(0);
        __syncthreads();
        int buf = 0;
        for (int d0 = 0; d0 < D; d0 += BK) {
            const bool more = d0 + BK < D;
            if (more) gload(d0 + BK);   // gload clamps its addresses
            const float *a = As + buf * BK * BM;
            const float *b = Bs + buf * BK * BN;
#pragma unroll
            for (int kk = 0; kk < BK; ++kk) {
                const float4 a0 = *reinterpret_cast<const float4 *>(a + kk * BM + ty * 4);
                const float4 a1 = *reinterpret_cast<const float4 *>(a + kk * BM + 64 + ty * 4);
                const float4 b0 = *reinterpret_cast<const float4 *>(b + kk * BN + tx * 4);
                const float4 b1 = *reinterpret_cast<const float4 *>(b + kk * BN + 64 + tx * 4);
                const float av[8] = {a0.x, a0.y, a0.z, a0.w, a1.x, a1.y, a1.z, a1.w};
                const float bv[8] = {b0.x, b0.y, b0.z, b0.w, b1.x, b1.y, b1.z, b1.w};
#pragma unroll
                for (int i = 0; i < 8; ++i)
#pragma unroll
                    for (int jj = 0; jj < 8; ++jj) acc[i][jj] = fmaf(av[i], bv[jj], acc[i][jj]);
            }
            if (more) {
                if (nc == 0)
#pragma unroll
                    for (int q = 0; q < 8; ++q) xsq = fmaf(ra[q], ra[q], xsq);
                sstore(buf ^ 1);
            }
            __syncthreads();
            buf ^= 1;
        }
#pragma unroll
        for (int i = 0; i < 8; ++i) {
            const int r = (i < 4) ? ty * 4 + i : 64 + ty * 4 + (i - 4);
#pragma unroll
            for (int jj = 0; jj < 8; ++jj) {
                const int c = nc + ((jj < 4) ? tx * 4 + jj : 64 + tx * 4 + (jj - 4));
                Sc[r * sp + c] = fmaf(-2.0f, acc[i][jj], cn[c]);
            }
        }
    }
    xn[lh * BM + lp] = xsq;
    __syncthreads();
    if (tid < BM) {
        const long long pix = p0 + tid;
        const bool valid = pix < n;
        const float xs = xn[tid] + xn[BM + tid];
        const float X = sqrtf(xs) * (1.0f + (float)(D + 8) * (float)kU32);
        unsigned mask[kMaskWords];
        int ncand = 1;
        int lab = 0;
        if (valid) lab = decide_pixel(Sc + tid * sp, 1, k, X, 0.0f, ca, cv, cb, mask, &ncand);
        if (valid) labels[pix] = (uint8_t)lab;
        push_flag(valid && ncand > 1, (unsigned)pix, mask, fl);
    }
}

// ----------------------------------------------------------------------------------
// Re-scoring of flagged pixels: one warp per pixel, uncentred FP32 inputs.
// Stage 1: plain FP32 direct form sum (x_i - c_i)^2, lane-sequential then a fixed
//          butterfly; every term is non-negative, so the relative error is at most
//          rho = (ceil(D/32) + 8) u.  Decided when the two smallest intervals separate.
// Stage 2: double-float direct form -- exact differences (TwoSum), exact squares
//          (FMA), compensated accumulation -- relative error about D u^2; ties between
//          equal values go to the lowest index.
// ----------------------------------------------------------------------------------
__device__ __forceinline__ float warp_sum(float v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

__device__ __forceinline__ void df_warp_sum(float &hi, float &lo)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const float h2 = __shfl_xor_sync(0xffffffffu, hi, o);
        const float l2 = __shfl_xor_sync(0xffffffffu, lo, o);
        float s, e;
        two_sum(hi, h2, s, e);
        hi = s;
        lo = lo + l2 + e;
    }
    float s, e;
    two_sum(hi, lo, s, e);   // renormalise
    hi = s;
    lo = e;
}

constexpr int RS_MAXC = 16;        // 32-feature chunks of a pixel held in registers by the re-scoring

__global__ void __launch_bounds__(256, 2) rescore_kernel(const float *__restrict__ X, int D,
                                                      const float *__restrict__ C, int k,
                                                      uint8_t *__restrict__ labels, FlagList fl,
                                                      unsigned cap)
{
    ptx::pdl_enter();
    const int lane = threadIdx.x & 31;
    const unsigned wid = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const unsigned nw = (gridDim.x * blockDim.x) >> 5;
    const unsigned n_entries = min(*fl.count, cap);     // the list holds at most cap entries
    const float u = (float)kU32;
    const float rho = ((float)((D + 31) / 32) + 8.0f) * u * 1.01f + 4.0f * u;
    unsigned long long my_cand = 0, my_deep = 0;
    // D <= 32 RS_MAXC: a pixel's features stay in registers and every candidate's loads are
    // issued together (the same per-lane order of additions as the general loop).  The warp's
    // next entry (pixel, candidate mask word, features) is loaded while this one is scored.
    const bool inreg = D <= 32 * RS_MAXC;
    unsigned pix_n = 0u, mw_n = 0u;
    float xn[RS_MAXC];
    auto fetch = [&](unsigned e2) {
        pix_n = fl.pix[e2];
        const unsigned m0 = fl.mask[(size_t)e2 * kMaskWords + (lane & (kMaskWords - 1))];
        mw_n = lane < kMaskWords ? m0 : 0u;
        const float *x2 = X + (size_t)pix_n * D;
#pragma unroll
        for (int t = 0; t < RS_MAXC; ++t) {
            const int i = 32 * t + lane;
            xn[t] = inreg && i < D ? x2[i] : 0.f;
        }
    };
    if (wid < n_entries) fetch(wid);
    for (unsigned e = wid; e < n_entries; e += nw) {
        const unsigned pix = pix_n;
        const unsigned mw = mw_n;
        const float *x = X + (size_t)pix * D;
        float r1 = FLT_MAX, r2 = FLT_MAX;
        int a = 0, nc = 0;
        float xv[RS_MAXC];
#pragma unroll
        for (int t = 0; t < RS_MAXC; ++t) xv[t] = xn[t];
        if (e + nw < n_entries) fetch(e + nw);
        auto keep = [&](float r, int j) {
            ++nc;
            if (r < r1) { r2 = r1; r1 = r; a = j; }
            else if (r < r2) { r2 = r; }
        };
        if (inreg) {
            // candidates in increasing index order, the next one's centroid loaded while the
            // current one is summed
            int cw = 0;
            unsigned cb = __shfl_sync(0xffffffffu, mw, 0);
            auto next = [&]() -> int {                       // uniform over the warp
                while (cb == 0u) {
                    if (++cw >= kMaskWords) return -1;
                    cb = __shfl_sync(0xffffffffu, mw, cw);
                }
                const int j = cw * 32 + __ffs(cb) - 1;
                cb &= cb - 1;
                return j;
            };
            auto load_c = [&](int j, float (&cv)[RS_MAXC]) {
                const float *c = C + (size_t)j * D;
#pragma unroll
                for (int t = 0; t < RS_MAXC; ++t) {
                    const int i = 32 * t + lane;
                    cv[t] = i < D ? c[i] : 0.f;
                }
            };
            auto sum_c = [&](const float (&cv)[RS_MAXC], int j) {
                float acc = 0.f;
#pragma unroll
                for (int t = 0; t < RS_MAXC; ++t) {
                    const float d = xv[t] - cv[t];
                    if (32 * t + lane < D) acc = fmaf(d, d, acc);
                }
                keep(warp_sum(acc), j);
            };
            float ca[RS_MAXC], cb2[RS_MAXC];                 // two buffers, used in turn
            int ja = next();
            if (ja >= 0) load_c(ja, ca);
            while (ja >= 0) {
                const int jb = next();
                if (jb >= 0) load_c(jb, cb2);
                sum_c(ca, ja);
                if (jb < 0) break;
                ja = next();
                if (ja >= 0) load_c(ja, ca);
                sum_c(cb2, jb);
            }
        } else {
            for (int w = 0; w < kMaskWords; ++w) {
                unsigned bits = __shfl_sync(0xffffffffu, mw, w);
                while (bits) {
                    const int j = w * 32 + __ffs(bits) - 1;
                    bits &= bits - 1;
                    const float *c = C + (size_t)j * D;
                    float acc = 0.f;
                    for (int i0 = 0; i0 < D; i0 += 32) {
                        const bool ok = i0 + lane < D;
                        const int i = ok ? i0 + lane : D - 1;
                        const float d = x[i] - c[i];
                        acc = ok ? fmaf(d, d, acc) : acc;
                    }
                    keep(warp_sum(acc), j);
                }
            }
        }
        const bool decided = r2 * (1.0f - rho) > r1 * (1.0f + rho);
        if (!decided) {
            float bh = FLT_MAX, bl = 0.f;
            int best = 0;
            for (int w = 0; w < kMaskWords; ++w) {
                unsigned bits = __shfl_sync(0xffffffffu, mw, w);
                while (bits) {
                    const int j = w * 32 + __ffs(bits) - 1;
                    bits &= bits - 1;
                    const float *c = C + (size_t)j * D;
                    float S = 0.f, E = 0.f;
                    for (int i0 = 0; i0 < D; i0 += 32) {
                        const bool ok = i0 + lane < D;
                        const int i = ok ? i0 + lane : D - 1;
                        const float xi = ok ? x[i] : 0.f, ci = ok ? c[i] : 0.f;
                        float h, l;
                        two_sum(xi, -ci, h, l);          // xi - ci = h + l exactly
                        const float p2 = h * h;
                        const float pe = fmaf(h, h, -p2);  // h^2 = p2 + pe exactly
                        float t, te;
                        two_sum(S, p2, t, te);
                        S = t;
                        E += te + pe + fmaf(2.0f * h, l, l * l);
                    }
                    df_warp_sum(S, E);
                    if (S < bh || (S == bh && E < bl)) { bh = S; bl = E; best = j; }
                }
            }
            a = best;
            ++my_deep;
        }
        my_cand += (unsigned long long)nc;
        if (lane == 0) labels[pix] = (uint8_t)a;
    }
    if (lane == 0 && (my_cand | my_deep)) {
        atomicAdd(&fl.stats[1], my_cand);
        if (my_deep) atomicAdd(&fl.stats[2], my_deep);
    }
}

__global__ void finish_stats_kernel(FlagList fl, vqnnf_assign_stats *out)
{
    ptx::pdl_enter();
    out->n_flagged = *fl.count;
    out->n_candidates = fl.stats[1];
    out->n_deep = fl.stats[2];
    out->reserved = 0;
}

}  // namespace

cudaError_t launch_prep_codebook(const float *C, int k, int D, int prec, CodebookPrep p,
                                 cudaStream_t s, unsigned *zero64, bool keep_mean)
{
    if (!keep_mean) {
        const cudaError_t le_ = launch_pdl(prep_mean_kernel, dim3((D + 31) / 32), dim3(256), 0, s, C, k, D, p.mean, zero64);
        if (le_ != cudaSuccess) return le_;
    }
    {
        const cudaError_t le_ = launch_pdl(prep_centroid_kernel, dim3(k), dim3(256), 0, s, C, k, D, prec, p,
                                           keep_mean ? zero64 : nullptr);
        if (le_ != cudaSuccess) return le_;
    }
    return cudaGetLastError();
}

static size_t fp32_smem_bytes(int k)
{
    const int kp = (k + BN - 1) / BN * BN;
    return sizeof(float) * (size_t)(2 * BK * BM + 2 * BK * BN + BM * (kp + 1) + 4 * kp + 2 * BM);
}

cudaError_t launch_assign_fp32(const float *X, long long n, int D, int k, const CodebookPrep &p,
                               uint8_t *labels, FlagList fl, cudaStream_t s)
{
    const size_t smem = fp32_smem_bytes(k);
    cudaError_t e = cudaFuncSetAttribute(assign_fp32_kernel,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    const long long blocks = (n + BM - 1) / BM;
    {
        const cudaError_t le_ = launch_pdl(assign_fp32_kernel, dim3((unsigned)blocks), dim3(NT), smem, s, X, n, D, k, p, labels, fl);
        if (le_ != cudaSuccess) return le_;
    }
    return cudaGetLastError();
}

cudaError_t launch_rescore(const float *X, long long n, int D, const float *C, int k,
                           uint8_t *labels, FlagList fl, cudaStream_t s)
{
    int dev = 0, sms = 148;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    // one warp per flagged pixel at a time; at most n pixels can be flagged, so small calls
    // (the Lloyd steps' template assignments) launch fewer blocks
    const long long blocks = std::min<long long>((long long)sms * 8, std::max<long long>(sms, (n + 63) / 64));
    {
        const cudaError_t le_ = launch_pdl(rescore_kernel, dim3((unsigned)blocks), dim3(256), 0, s, X, D, C, k, labels, fl, (unsigned)n);
        if (le_ != cudaSuccess) return le_;
    }
    return cudaGetLastError();
}

cudaError_t launch_finish_stats(FlagList fl, vqnnf_assign_stats *out, cudaStream_t s)
{
    {
        const cudaError_t le_ = launch_pdl(finish_stats_kernel, dim3(1), dim3(1), 0, s, fl, out);
        if (le_ != cudaSuccess) return le_;
    }
    return cudaGetLastError();
}

}  // namespace vqnnf
