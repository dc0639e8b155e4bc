// k-means codebook of the template (Sec. 3.1): seeded initial centroids, then Lloyd
// steps whose assignment is the exact nearest-neighbour field of assign_fp32.cu /
// assign_tc.cu and whose update sums every cluster's members in FP64 in pixel order.
//
// Determinism: the members of each cluster are listed in pixel order by a stable counting
// sort, and thread (j, i) adds member features one after another in that order, so every
// FP64 sum is the same sequence of additions as a plain loop over pixels -- the centroids
// do not depend on scheduling.
#include "common.cuh"
#include "ptx.cuh"

namespace vqnnf {

namespace {

__global__ void gather_init_kernel(const float *__restrict__ T, int D, int k, InitIdx ii,
                                   float *__restrict__ C)
{
    ptx::pdl_enter();
    const int j = blockIdx.x;
    const float *src = T + (size_t)ii.idx[j] * D;
    for (int i = threadIdx.x; i < D; i += blockDim.x) C[(size_t)j * D + i] = src[i];
}

// Stable counting sort of the labels by cluster (one block of 32 warps).
//   cnt[k], off[k+1], members[l] (pixel indices in increasing order within a cluster)
// Warp w owns the contiguous pixel range [w L, (w+1) L), L = ceil(l / 32) rounded up to 32.
// Pass 1 counts each cluster's pixels per warp (match_any: one leader per label value),
// then one exclusive prefix in (cluster, warp) order gives every warp's first slot per
// cluster; pass 2 repeats the walk and writes each pixel at its slot + rank.
__global__ void __launch_bounds__(1024) stable_sort_kernel(const uint8_t *__restrict__ lab,
                                                           int l, int k, int *cnt, int *off,
                                                           int *members)
{
    ptx::pdl_enter();
    __shared__ int wc[32][kMaxK];   // per-warp counts, then per-warp running slots
    __shared__ int tot[kMaxK];
    const int t = threadIdx.x, lane = t & 31, w = t >> 5;
    const unsigned lt = (1u << lane) - 1u;
    const int L = ((l + 31) / 32 + 31) / 32 * 32;
    const int p0 = w * L, p1 = min(l, p0 + L);
    for (int j = lane; j < k; j += 32) wc[w][j] = 0;
    __syncwarp();
    for (int pb = p0; pb < p1; pb += 32) {
        const int p = pb + lane;
        const bool in = p < p1;
        const int l0 = (int)lab[in ? p : p1 - 1];             // clamped address
        const int lb = in ? l0 : -1 - lane;                   // unique dummies never match
        const unsigned same = __match_any_sync(0xffffffffu, lb);
        if (in && __popc(same & lt) == 0) wc[w][lb] += __popc(same);
        __syncwarp();
    }
    __syncthreads();
    // totals per cluster, exclusive prefix over clusters (warp 0), then over warps per cluster
    for (int j = t; j < k; j += blockDim.x) {
        int s = 0;
        for (int q = 0; q < 32; ++q) s += wc[q][j];
        tot[j] = s;
    }
    __syncthreads();
    if (w == 0) {
        int carry = 0;
        for (int j0 = 0; j0 < k; j0 += 32) {
            const int j = j0 + lane;
            const int v = j < k ? tot[j] : 0;
            int x = v;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const int y = __shfl_up_sync(0xffffffffu, x, o);
                if (lane >= o) x += y;
            }
            if (j < k) {
                off[j] = carry + x - v;
                cnt[j] = v;
                tot[j] = carry + x - v;                       // first slot of cluster j
            }
            carry += __shfl_sync(0xffffffffu, x, 31);
        }
        if (lane == 0) off[k] = carry;
    }
    __syncthreads();
    for (int j = t; j < k; j += blockDim.x) {
        int s = tot[j];
        for (int q = 0; q < 32; ++q) {
            const int c = wc[q][j];
            wc[q][j] = s;
            s += c;
        }
    }
    __syncthreads();
    for (int pb = p0; pb < p1; pb += 32) {
        const int p = pb + lane;
        const bool in = p < p1;
        const int l0 = (int)lab[in ? p : p1 - 1];
        const int lb = in ? l0 : -1 - lane;
        const unsigned same = __match_any_sync(0xffffffffu, lb);
        const int rank = __popc(same & lt);
        if (in) members[wc[w][lb] + rank] = p;
        __syncwarp();
        if (in && rank == 0) wc[w][lb] += __popc(same);
        __syncwarp();
    }
}

// c_j[i] = fl32( (sum over members, pixel order, FP64) / count ); empty clusters keep c_j.
//
// The FP64 pipe of this GPU is narrow, so the in-order FP64 sum is not evaluated as such.
// Every member value is an FP32 number, i.e. an integer multiple of a power of two; in units
// of 2^-80 the values with 2^-57 <= |x| < 2^46 (and zero) are exact 128-bit integers, whose
// sum is exact and associative, so it is split over the 16 warps of the block.  If moreover
// every partial sum of the in-order FP64 evaluation fits in 53 significant bits, none of its
// additions rounds and its result IS the exact sum.  Sufficient: the top bit of sum |x| (a
// bound of every partial sum) and the lowest set bit over all members' values are at most 52
// positions apart.  A (cluster, dimension) pair that fails this, holds a value outside the
// range, or whose sums could exceed 128 bits is summed in FP64 in pixel order by its lane.
// Both branches therefore equal the in-order FP64 sum bit for bit.
//
// The common case takes a narrower route first: values with 2^-17 <= |x| < 2^5 (and zero) are
// integers below 2^45 in units of 2^-40, so with fewer than 2^18 members their signed sum and
// the sum of |x| are exact in 64 bits, at a quarter of the 128-bit route's instructions.  A
// block with any value outside that range (or a larger cluster) repeats the members in 128 bits.
constexpr int UW = 16;       // warps per (cluster, 32 dimensions)

struct Fixed64 {
    long long sum;                     // signed sum, units 2^-40
    unsigned long long mag;            // sum of |x|
    int low;                           // lowest set bit position over the values
    bool bad;                          // a value outside [2^-17, 2^5)
};

__device__ __forceinline__ void fixed64_add(Fixed64 &f, float x)
{
    const uint32_t b = __float_as_uint(x);
    const uint32_t E = (b >> 23) & 0xFFu;
    const uint32_t frac = b & 0x7FFFFFu;
    if (E == 0u && frac == 0u) return;                     // +-0 adds nothing
    if (E < 110u || E > 131u) { f.bad = true; return; }     // |x| < 2^-17 or >= 2^5 (inf, nan)
    const uint32_t M = frac | 0x800000u;
    const int sh = (int)E - 110;                          // x = M * 2^(sh - 40), M 2^sh < 2^45
    const unsigned long long X = (unsigned long long)M << sh;
    f.sum += (b >> 31) ? -(long long)X : (long long)X;
    f.mag += X;
    f.low = min(f.low, sh + __ffs((int)M) - 1);
}

struct Fixed {
    unsigned __int128 pos, neg, mag;   // sums of the positive and negative parts, of |x|
    int low;                           // lowest set bit position over the values (units 2^-80)
    int hish;                          // largest shift: every value is below 2^(hish + 24) units
    bool bad;                          // a value outside the exact range
};

__device__ __forceinline__ void fixed_add(Fixed &f, float x)
{
    const uint32_t b = __float_as_uint(x);
    const uint32_t E = (b >> 23) & 0xFFu;
    const uint32_t frac = b & 0x7FFFFFu;
    if (E == 0u && frac == 0u) return;                     // +-0 adds nothing
    if (E < 70u || E > 172u) { f.bad = true; return; }      // |x| < 2^-57 or >= 2^46 (inf, nan)
    const uint32_t M = frac | 0x800000u;
    const int sh = (int)E - 70;                           // x = M * 2^(sh - 80)
    const unsigned __int128 X = (unsigned __int128)M << sh;
    if (b >> 31) f.neg += X;
    else f.pos += X;
    f.mag += X;
    f.low = min(f.low, sh + __ffs((int)M) - 1);
    f.hish = max(f.hish, sh);
}

__device__ __forceinline__ int top_bit(unsigned __int128 v)
{
    const uint64_t hi = (uint64_t)(v >> 64), lo = (uint64_t)v;
    return hi ? 127 - __clzll((long long)hi) : (lo ? 63 - __clzll((long long)lo) : -1);
}

constexpr int FCH = 88;      // member rows per staged chunk of the in-order FP64 route
constexpr int COOP_MIN = 1024;   // clusters at least this large stage that route block-wide

__global__ void __launch_bounds__(32 * UW, 3) update_kernel(const float *__restrict__ T, int D, int k,
                                                         const int *__restrict__ cnt, const int *__restrict__ off,
                                                         const int *__restrict__ members, float *__restrict__ C)
{
    ptx::pdl_enter();
    // the 128-bit partial sums, later reused for the staged member values of the FP64 route
    __shared__ __align__(16) unsigned __int128 sacc[3][UW][32];
    __shared__ int slow[UW][32], shish[UW][32];
    __shared__ unsigned char sbad[UW][32];
    __shared__ unsigned s_need;
    static_assert(2 * FCH * 33 * sizeof(float) <= sizeof(sacc), "staging buffers exceed the reused space");
    auto spos = sacc[0], sneg = sacc[1], smag = sacc[2];
    const int j = blockIdx.y;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int i = blockIdx.x * 32 + lane;
    const int c = cnt[j];
    if (c == 0) return;                                  // uniform over the block
    const int *m = members + off[j];
    const int ic = i < D ? i : D - 1;                    // clamped column (every address in bounds)
    Fixed64 f6;
    f6.sum = 0;
    f6.mag = 0;
    f6.low = 1 << 30;
    f6.bad = false;
    int q = w;
    for (; q + 7 * UW < c; q += 8 * UW) {                // eight member rows in flight per warp
        float x[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) x[u] = __ldg(T + (size_t)m[q + u * UW] * D + ic);
#pragma unroll
        for (int u = 0; u < 8; ++u) fixed64_add(f6, x[u]);
    }
    for (; q < c; q += UW) fixed64_add(f6, __ldg(T + (size_t)m[q] * D + ic));
    // uniform over the block: the 128-bit route when a value is outside the 64-bit range
    const bool wide = __syncthreads_or(f6.bad || c >= (1 << 18));
    long long (*s64)[32] = reinterpret_cast<long long (*)[32]>(&sacc[0][0][0]);
    unsigned long long (*m64)[32] = reinterpret_cast<unsigned long long (*)[32]>(&sacc[1][0][0]);
    if (!wide) {
        s64[w][lane] = f6.sum;
        m64[w][lane] = f6.mag;
        slow[w][lane] = f6.low;
    } else {
        Fixed f;
        f.pos = f.neg = f.mag = 0;
        f.low = 1 << 30;
        f.hish = 0;
        f.bad = false;
        for (q = w; q + 7 * UW < c; q += 8 * UW) {
            float x[8];
#pragma unroll
            for (int u = 0; u < 8; ++u) x[u] = __ldg(T + (size_t)m[q + u * UW] * D + ic);
#pragma unroll
            for (int u = 0; u < 8; ++u) fixed_add(f, x[u]);
        }
        for (; q < c; q += UW) fixed_add(f, __ldg(T + (size_t)m[q] * D + ic));
        spos[w][lane] = f.pos;
        sneg[w][lane] = f.neg;
        smag[w][lane] = f.mag;
        slow[w][lane] = f.low;
        shish[w][lane] = f.hish;
        sbad[w][lane] = f.bad ? 1 : 0;
    }
    __syncthreads();
    // small clusters: warp 0 alone finishes (the other warps leave now, so the next block can
    // start); large clusters keep every warp for a staged in-order FP64 route
    const bool coop = c >= COOP_MIN;                    // uniform over the block
    if (!coop && w != 0) return;
    double s = 0.0;
    bool need = false;                                  // this lane's column takes the FP64 route
    if (w == 0 && !wide) {
        long long sum = 0;
        unsigned long long mag = 0;
        int low = 1 << 30;
#pragma unroll 4
        for (int u = 0; u < UW; ++u) {
            sum += s64[u][lane];
            mag += m64[u][lane];
            low = min(low, slow[u][lane]);
        }
        if (mag == 0) {
            s = 0.0;                                     // only zeros: the FP64 sum is +0
        } else if (63 - __clzll((long long)mag) - low <= 52) {
            // exact: |sum| >> low has at most 53 significant bits
            const unsigned long long a = sum < 0 ? (unsigned long long)(-sum) : (unsigned long long)sum;
            const double v = (double)(a >> low);
            s = ldexp(sum < 0 ? -v : v, low - 40);
        } else {
            need = true;                                 // a rounding could occur in order
        }
    } else if (w == 0) {
        unsigned __int128 pos = 0, neg = 0, mag = 0;
        int low = 1 << 30, hish = 0;
        bool bad = false;
#pragma unroll 2
        for (int u = 0; u < UW; ++u) {
            pos += spos[u][lane];
            neg += sneg[u][lane];
            mag += smag[u][lane];
            low = min(low, slow[u][lane]);
            hish = max(hish, shish[u][lane]);
            bad |= sbad[u][lane] != 0;
        }
        // the 128-bit sums cannot have wrapped while c values below 2^(hish + 24) units stay
        // below 2^128: hish + 24 + ceil(log2 c) <= 127
        const bool nowrap = hish + 24 + (32 - __clz(c)) <= 127;
        if (bad || !nowrap) {
            need = true;                                 // outside the exact route
        } else if (mag == 0) {
            s = 0.0;                                     // only zeros: the FP64 sum is +0
        } else if (top_bit(mag) - low <= 52) {
            // exact: |sum| >> low has at most 53 significant bits
            const bool negative = neg > pos;
            const unsigned __int128 d = negative ? neg - pos : pos - neg;
            const double v = (double)(uint64_t)(d >> low);
            s = ldexp(negative ? -v : v, low - 80);
        } else {
            need = true;                                 // a rounding could occur in order
        }
    }
    if (w == 0) {
        const unsigned nm = __ballot_sync(0xffffffffu, need && i < D);
        if (lane == 0) s_need = nm;
        if (!coop && need) {                             // the in-order FP64 sum, lane by lane
            s = 0.0;
            for (int q2 = 0; q2 < c; ++q2) s += (double)__ldg(T + (size_t)m[q2] * D + ic);
        }
    }
    if (!coop) {
        if (i < D) C[(size_t)j * D + i] = (float)(s / (double)c);
        return;
    }
    __syncthreads();                                     // partial sums read; s_need visible
    const unsigned nm = s_need;
    if (nm) {
        // the in-order FP64 sum of the flagged columns: the block's 32 columns of the members'
        // rows are staged in shared memory, FCH rows at a time and double-buffered; warps 1..15
        // load the next chunk while warp 0 adds the current one, row by row, in member order
        float (*vals)[FCH][33] = reinterpret_cast<float (*)[FCH][33]>(&sacc[0][0][0]);
        auto stage = [&](int q0, int buf, int w0, int nwarp) {
            const int nr = min(FCH, c - q0);
            for (int r = w - w0; r < nr; r += nwarp) vals[buf][r][lane] = __ldg(T + (size_t)m[q0 + r] * D + ic);
        };
        stage(0, 0, 0, UW);
        __syncthreads();
        const bool mine = w == 0 && ((nm >> lane) & 1u);
        double acc = 0.0;
        for (int q0 = 0, t = 0; q0 < c; q0 += FCH, ++t) {
            if (w != 0 && q0 + FCH < c) stage(q0 + FCH, (t + 1) & 1, 1, UW - 1);
            if (mine) {
                const int nr = min(FCH, c - q0);
                for (int r = 0; r < nr; ++r) acc += (double)vals[t & 1][r][lane];
            }
            __syncthreads();
        }
        if (mine) s = acc;
    }
    if (w == 0 && i < D) C[(size_t)j * D + i] = (float)(s / (double)c);
}

}  // namespace

cudaError_t launch_gather_init(const float *T, int D, int k, const InitIdx &ii, float *C,
                               cudaStream_t s)
{
    {
        const cudaError_t le_ = launch_pdl(gather_init_kernel, dim3(k), dim3(128), 0, s, T, D, k, ii, C);
        if (le_ != cudaSuccess) return le_;
    }
    return cudaGetLastError();
}

cudaError_t launch_lloyd_update(const float *T, int l, int D, int k, const uint8_t *lab, int *cnt,
                                int *off, int *members, float *C, cudaStream_t s)
{
    {
        const cudaError_t le_ = launch_pdl(stable_sort_kernel, dim3(1), dim3(1024), 0, s, lab, l, k, cnt, off, members);
        if (le_ != cudaSuccess) return le_;
    }
    // one block of UW warps per (32 dimensions, cluster)
    dim3 g((D + 31) / 32, k);
    {
        const cudaError_t le_ = launch_pdl(update_kernel, dim3(g), dim3(32 * UW), 0, s, T, D, k, cnt, off, members, C);
        if (le_ != cudaSuccess) return le_;
    }
    return cudaGetLastError();
}

}  // namespace vqnnf
