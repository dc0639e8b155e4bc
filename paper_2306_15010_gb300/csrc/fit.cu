// k-means codebook of the template (Sec. 3.1): seeded initial centroids, then Lloyd
// steps whose assignment is the exact nearest-neighbour field of assign_fp32.cu /
// assign_tc.cu and whose update is the mean of every cluster's members, summed in FP64 in
// pixel order.
//
// Determinism: the update's sums are exact integers (fixed point), so they do not depend on
// the order in which the members are listed or added; it certifies that the in-order FP64
// sum of a (cluster, dimension) has no rounding and then equals it, and otherwise adds the
// members in FP64 in pixel order.  The centroids do not depend on scheduling.
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

// Counting sort of the labels by cluster, over up to kSortBlocks blocks of 256 threads (one
// block's shared-memory atomics would serialise on one SM):
//   sort_count_kernel: block b counts the clusters of its label range [b LB, (b + 1) LB);
//   sort_scatter_kernel: every block adds up the counts (at most kSortBlocks x k values), takes
//     its own first slot per cluster, and writes its pixels there (shared-memory cursors);
//     block 0 also writes cnt[k], off[k+1], the chunk table of the update (every non-empty
//     cluster's member slots cut into chunks of kLloydRows, listed cluster by cluster, the
//     unused entries up to max_chunks zeroed) and zeroes the update's chunk counters.
// members[l] lists the pixels of each cluster in no particular order: the update's sums do
// not depend on it, and its in-order route rebuilds pixel order itself.
constexpr int kSortBlocks = kLloydSortBlocks;
constexpr int kSortThreads = 256;
static_assert(kMaxK <= kSortThreads, "one cluster per thread in the scatter's prefix");

__host__ __device__ inline int sort_block_labels(int l)
{
    // a multiple of 1024 (whole 32-bit words per thread), at most kSortBlocks blocks
    const int per = (l + kSortBlocks - 1) / kSortBlocks;
    return ((per > 1024 ? per : 1024) + 1023) / 1024 * 1024;
}

// The label range of block b as whole words [w0, w1) plus, for the last block, a byte tail.
__device__ __forceinline__ void sort_range(int l, int b, int &w0, int &w1, int &p_tail)
{
    const int LB = sort_block_labels(l);
    const int p0 = min(l, b * LB), p1 = min(l, p0 + LB);
    w0 = p0 >> 2;                                        // p0 is a multiple of 4
    w1 = p1 >> 2;
    p_tail = 4 * w1;                                     // bytes [p_tail, p1) remain (last block)
}

__global__ void __launch_bounds__(kSortThreads) sort_count_kernel(const uint8_t *__restrict__ lab, int l, int k,
                                                                  int *__restrict__ bh)
{
    ptx::pdl_enter();
    __shared__ int hist[kMaxK];
    const int t = threadIdx.x, b = blockIdx.x;
    for (int j = t; j < k; j += blockDim.x) hist[j] = 0;
    __syncthreads();
    int w0, w1, pt;
    sort_range(l, b, w0, w1, pt);
    const uint32_t *lab4 = reinterpret_cast<const uint32_t *>(lab);   // 256-byte aligned
    for (int q = w0 + t; q < w1; q += blockDim.x) {
        const uint32_t v = __ldg(lab4 + q);
#pragma unroll
        for (int c = 0; c < 4; ++c) atomicAdd(&hist[(v >> (8 * c)) & 0xFFu], 1);
    }
    const int pe = min(l, b * sort_block_labels(l) + sort_block_labels(l));
    for (int p = pt + t; p < pe; p += blockDim.x) atomicAdd(&hist[lab[p]], 1);
    __syncthreads();
    for (int j = t; j < k; j += blockDim.x) bh[b * k + j] = hist[j];
}

// exclusive block-wide prefix of one value per thread (kSortThreads threads); returns the
// total through *total
__device__ __forceinline__ int block_exclusive_scan(int v, int *warp_tot, int *total)
{
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    int x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) warp_tot[w] = x;
    __syncthreads();
    int before = 0, all = 0;
    for (int q = 0; q < kSortThreads / 32; ++q) {
        before += q < w ? warp_tot[q] : 0;
        all += warp_tot[q];
    }
    __syncthreads();
    *total = all;
    return before + x - v;
}

__global__ void __launch_bounds__(kSortThreads) sort_scatter_kernel(const uint8_t *__restrict__ lab, int l, int k,
                                                                    int D, int max_chunks,
                                                                    const int *__restrict__ bh, LloydWs lw)
{
    ptx::pdl_enter();
    __shared__ int cur[kMaxK];
    __shared__ int wt[kSortThreads / 32];
    const int t = threadIdx.x, b = blockIdx.x, nb = gridDim.x;
    // thread t: cluster t's size and this block's first slot in it
    int c = 0, mine = 0;
    if (t < k)
        for (int q = 0; q < nb; ++q) {
            const int n = __ldg(bh + q * k + t);
            mine += q < b ? n : 0;
            c += n;
        }
    int nslots, nch_all;
    const int first = block_exclusive_scan(c, wt, &nslots);
    const int nch = (c + kLloydRows - 1) / kLloydRows;
    const int f = block_exclusive_scan(nch, wt, &nch_all);
    if (t < k) cur[t] = first + mine;
    if (b == 0) {
        if (t < k) {
            lw.cnt[t] = c;
            lw.off[t] = first;
            lw.rcp[t] = c > 0 ? 1.0 / (double)c : 0.0;
            // chunk entries (first slot, rows | cluster << 8, cluster's first chunk, cluster size)
            for (int r = 0; r < nch; ++r)
                lw.chunks[f + r] = make_int4(first + r * kLloydRows, min(kLloydRows, c - r * kLloydRows) | t << 8, f, c);
        }
        if (t == 0) lw.off[k] = nslots;
        for (int q = nch_all + t; q < max_chunks; q += blockDim.x) lw.chunks[q] = make_int4(0, 0, 0, 0);
        const int nd = k * ((D + 31) / 32);
        for (int q = t; q < nd; q += blockDim.x) lw.done[q] = 0;
    }
    __syncthreads();
    int w0, w1, pt;
    sort_range(l, b, w0, w1, pt);
    const uint32_t *lab4 = reinterpret_cast<const uint32_t *>(lab);
    for (int q = w0 + t; q < w1; q += blockDim.x) {
        const uint32_t v = __ldg(lab4 + q);
#pragma unroll
        for (int cc = 0; cc < 4; ++cc) lw.members[atomicAdd(&cur[(v >> (8 * cc)) & 0xFFu], 1)] = 4 * q + cc;
    }
    const int pe = min(l, b * sort_block_labels(l) + sort_block_labels(l));
    for (int p = pt + t; p < pe; p += blockDim.x) lw.members[atomicAdd(&cur[lab[p]], 1)] = p;
}

// The pixels of cluster j in increasing order, written to out[0, cnt_j): a block-wide stable
// compaction of the labels (for the in-order FP64 route only).  scan: blockDim.x ints of
// shared memory.  Every thread of the block must call it.
__device__ void ordered_members(const uint8_t *__restrict__ lab, int l, int j, int *out, int *scan)
{
    const int nt = blockDim.x, t = threadIdx.x;
    const int seg = (l + nt - 1) / nt, p0 = min(l, t * seg), p1 = min(l, p0 + seg);
    int n = 0;
    for (int p = p0; p < p1; ++p) n += lab[p] == j;
    scan[t] = n;
    __syncthreads();
    for (int o = 1; o < nt; o <<= 1) {                   // inclusive scan (Hillis-Steele)
        const int v = t >= o ? scan[t - o] : 0;
        __syncthreads();
        scan[t] += v;
        __syncthreads();
    }
    int pos = scan[t] - n;
    for (int p = p0; p < p1; ++p)
        if (lab[p] == j) out[pos++] = p;
    __syncthreads();
}

// c_j[i] = fl32( (sum over members, pixel order, FP64) / count ); empty clusters keep c_j.
//
// The FP64 pipe of this GPU is narrow, so the in-order FP64 sum is not evaluated as such.
// Every member value is an FP32 number, i.e. an integer multiple of a power of two; in units
// of 2^-80 the values with 2^-57 <= |x| < 2^46 (and zero) are exact 128-bit integers, whose
// sum is exact and associative, so it is split over the warps of a block and over the chunks
// of a cluster.  If moreover every partial sum of the in-order FP64 evaluation fits in 53
// significant bits, none of its additions rounds and its result IS the exact sum.  Sufficient:
// the top bit of sum |x| (a bound of every partial sum) and the lowest set bit over all
// members' values are at most 52 positions apart.  A (cluster, dimension) pair that fails this,
// holds a value outside the range, or whose sums could exceed 128 bits is summed in FP64 in
// pixel order.  Both branches therefore equal the in-order FP64 sum bit for bit.
//
// The common case takes a narrower route first (Split32 below): values with 2^-17 <= |x| < 2^5
// (and zero) are multiples of 2^-40, summed exactly on the FP32 pipe at a fraction of the
// 128-bit route's instructions.  Its exactness test uses bounds: rows x max |x| for sum |x|,
// and the last mantissa bit of the smallest nonzero |x| for the lowest set bit.  A block with
// any value outside that range repeats its rows in 128 bits.
//
// Work split: one block per (chunk of at most kLloydRows member rows, 32 dimensions), so a
// large cluster is spread over many blocks.  A one-chunk cluster finishes in its block; the
// chunks of a larger cluster store their partial sums, and the block that finishes last (a
// counter per (cluster, 32 dimensions)) adds them in chunk order and finishes the cluster.
constexpr int UW = 8;        // warps per (chunk, 32 dimensions)
constexpr int UB = 16;       // member rows per warp (a short chunk is zero-padded)
static_assert(UW * UB == kLloydRows, "one batch of loads per warp covers a chunk");
static_assert(kLloydRows < 256, "a chunk's row count is packed in 8 bits");

// The narrow route, on the FP32 pipe: every value with 2^-17 <= |x| < 2^5 is a multiple of
// 2^-40.  t = fl(K1 + x), K1 = 1.5 * 2^6, lies in (64, 128), where the float spacing is 2^-17, so
// hi = t - K1 is x rounded to a multiple of 2^-17 and both hi and lo = x - hi are exact, with
// |lo| <= 2^-18.  u = fl(K2 + lo), K2 = 1.5 * 2^-17, lies in [2^-17, 2^-16], spacing 2^-40, and
// is exact.  Consecutive floats have consecutive bit patterns (also across the one binade step
// at 2^-16), so bits(t) - bits(K1) = hi / 2^-17 and bits(u) - bits(K2) = lo / 2^-40 exactly.  The
// patterns are summed mod 2^32 and the constants taken off once per added value: the true sums
// stay below 2^31 in magnitude, so the wrapped results equal them.  The largest |x| and the
// smallest nonzero |x| are kept for the range test and for the bounds of the exactness test.
constexpr float kSplitHi = 96.0f;                 // 1.5 * 2^6
constexpr float kSplitLo = 1.1444091796875e-05f;  // 1.5 * 2^-17
struct Split32 {
    uint32_t th, tl;                   // sums of bits(t) and of bits(u), mod 2^32
    uint32_t mx;                       // largest |x| (bit pattern)
    uint32_t mn;                       // smallest nonzero |x| pattern minus one (zero: 2^32 - 1)
};

__device__ __forceinline__ void split_add(Split32 &f, float x)
{
    const float t = __fadd_rn(kSplitHi, x);
    const float hi = __fsub_rn(t, kSplitHi);
    const float lo = __fsub_rn(x, hi);
    const float u = __fadd_rn(kSplitLo, lo);
    f.th += __float_as_uint(t);
    f.tl += __float_as_uint(u);
    const uint32_t a = __float_as_uint(x) & 0x7FFFFFFFu;
    f.mx = max(f.mx, a);
    f.mn = min(f.mn, a - 1u);
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

constexpr int FCH = 44;      // member rows per staged chunk of the in-order FP64 route

// RN(a / b) for finite a and b > 0 from y = RN(1 / b) (Markstein's theorem: if q is within one
// ulp of a / b, r = a - b q is exact and RN(q + r y) is the correctly rounded quotient).  The
// first correction brings q0 = RN(a y), within 1.5 ulp, to within one ulp.
__device__ __forceinline__ double div_rn(double a, double b, double y)
{
    double q = a * y;
    double r = fma(-q, b, a);
    q = fma(r, y, q);
    r = fma(-q, b, a);
    return fma(r, y, q);
}

__global__ void __launch_bounds__(32 * UW, 5) update_kernel(const float *__restrict__ T, int l, int D,
                                                         const uint8_t *__restrict__ lab, LloydWs lw,
                                                         float *__restrict__ C)
{
    ptx::pdl_enter();
    __shared__ int sscan[32 * UW];
    // the per-warp partial sums, later reused for the staged member values of the FP64 route
    __shared__ __align__(16) unsigned __int128 sacc[3][UW][32];
    __shared__ int slow[UW][32], shish[UW][32];
    __shared__ unsigned char sbad[UW][32];
    __shared__ unsigned s_need;
    __shared__ int s_last;
    static_assert(2 * FCH * 33 * sizeof(float) <= sizeof(sacc), "staging buffers exceed the reused space");
    auto spos = sacc[0], sneg = sacc[1], smag = sacc[2];
    // (first slot, rows | cluster << 8, cluster's first chunk, cluster size); rows = 0: unused
    const int4 ch = lw.chunks[blockIdx.x];
    const int nr = ch.y & 0xFF, j = ch.y >> 8, c = ch.w;
    if (nr == 0) return;                                 // uniform over the block
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int i = blockIdx.y * 32 + lane;
    const int *m = lw.members + ch.x;
    const int ic = i < D ? i : D - 1;                    // clamped column (every address in bounds)
    // rows w + u UW of the chunk, all loads issued before the adds; rows past the chunk read as
    // zero, which adds nothing on either route
    float x[UB];
#pragma unroll
    for (int u = 0; u < UB; ++u) {
        const int q = w + u * UW;
        x[u] = q < nr ? __ldg(T + (size_t)m[q] * D + ic) : 0.f;
    }
    Split32 f2;
    f2.th = f2.tl = 0u;
    f2.mx = 0u;
    f2.mn = 0xFFFFFFFFu;
#pragma unroll
    for (int u = 0; u < UB; ++u) split_add(f2, x[u]);
    // outside [2^-17, 2^5) (infinities and NaN included), zeros aside
    const bool out = f2.mx >= 0x42000000u || (f2.mn != 0xFFFFFFFFu && f2.mn + 1u < 0x37000000u);
    // uniform over the block: the 128-bit route when a value is outside the narrow route's range
    const bool wide = __syncthreads_or(out);
    int (*shi)[32] = slow, (*slo)[32] = shish;
    uint32_t (*smx)[32] = reinterpret_cast<uint32_t (*)[32]>(&sacc[0][0][0]);
    uint32_t (*smn)[32] = reinterpret_cast<uint32_t (*)[32]>(&sacc[1][0][0]);
    if (!wide) {
        shi[w][lane] = (int)(f2.th - (uint32_t)UB * __float_as_uint(kSplitHi));   // units 2^-17
        slo[w][lane] = (int)(f2.tl - (uint32_t)UB * __float_as_uint(kSplitLo));   // units 2^-40
        smx[w][lane] = f2.mx;
        smn[w][lane] = f2.mn;
    } else {
        Fixed f;
        f.pos = f.neg = f.mag = 0;
        f.low = 1 << 30;
        f.hish = 0;
        f.bad = false;
#pragma unroll
        for (int u = 0; u < UB; ++u) fixed_add(f, x[u]);
        spos[w][lane] = f.pos;
        sneg[w][lane] = f.neg;
        smag[w][lane] = f.mag;
        slow[w][lane] = f.low;
        shish[w][lane] = f.hish;
        sbad[w][lane] = f.bad ? 1 : 0;
    }
    __syncthreads();
    // the chunk's sums per dimension (warp 0), in 128 bits at units 2^-80
    unsigned __int128 pos = 0, neg = 0, mag = 0;
    int low = 1 << 30, hish = 0;
    bool bad = false;
    if (w == 0) {
        if (!wide) {
            int sh = 0, sl = 0;                          // |sums| <= 128 * 2^22: no overflow
            uint32_t mx = 0u, mn = 0xFFFFFFFFu;
#pragma unroll
            for (int u = 0; u < UW; ++u) {
                sh += shi[u][lane];
                sl += slo[u][lane];
                mx = max(mx, smx[u][lane]);
                mn = min(mn, smn[u][lane]);
            }
            // the exact sum in units 2^-40, then 2^-80
            const long long sum = (long long)sh * (1ll << 23) + sl;
            const unsigned long long a = sum < 0 ? 0ull - (unsigned long long)sum : (unsigned long long)sum;
            (sum < 0 ? neg : pos) = (unsigned __int128)a << 40;
            if (mx != 0u) {
                // bounds for the exactness test: sum |x| <= rows * max |x|, and no value has a
                // set bit below the last mantissa bit of the smallest nonzero |x|
                const uint32_t Mx = (mx & 0x7FFFFFu) | 0x800000u;
                mag = (unsigned __int128)(unsigned)nr * ((unsigned __int128)Mx << ((mx >> 23) - 70u));
                low = (int)((mn + 1u) >> 23) - 70;
            }
            hish = 61;                                   // every value is below 2^5
        } else {
#pragma unroll 2
            for (int u = 0; u < UW; ++u) {
                pos += spos[u][lane];
                neg += sneg[u][lane];
                mag += smag[u][lane];
                low = min(low, slow[u][lane]);
                hish = max(hish, shish[u][lane]);
                bad |= sbad[u][lane] != 0;
            }
        }
    }
    const bool single = nr == c;                         // uniform: a one-chunk cluster
    if (!single) {
        // store the chunk's sums; the last chunk of (cluster, 32 dimensions) to arrive adds them all
        if (w == 0) {
            if (i < D) {
                LloydPart pt;
                pt.pos = pos;
                pt.neg = neg;
                pt.mag = mag;
                pt.low = low;
                pt.hish = hish;
                pt.bad = bad ? 1 : 0;
                pt.pad = 0;
                lw.part[(size_t)blockIdx.x * D + i] = pt;
            }
            __threadfence();
            __syncwarp();
            if (lane == 0) {
                const int nch = (c + kLloydRows - 1) / kLloydRows;
                s_last = atomicAdd(&lw.done[j * gridDim.y + blockIdx.y], 1) == nch - 1;
            }
        }
        __syncthreads();
        if (!s_last) return;                             // uniform over the block
        __threadfence();
        if (w == 0) {
            const int f = ch.z, nch = (c + kLloydRows - 1) / kLloydRows;
            pos = neg = mag = 0;
            low = 1 << 30;
            hish = 0;
            bad = false;
            for (int q = 0; q < nch; ++q) {              // chunk order (the sums are exact anyway)
                const LloydPart *pp = lw.part + (size_t)(f + q) * D + ic;
                const uint4 *pv = reinterpret_cast<const uint4 *>(pp);
                const uint4 v0 = __ldcg(pv), v1 = __ldcg(pv + 1), v2 = __ldcg(pv + 2), v3 = __ldcg(pv + 3);
                auto u128 = [](const uint4 &v) {
                    return (unsigned __int128)v.x | (unsigned __int128)v.y << 32 | (unsigned __int128)v.z << 64 |
                           (unsigned __int128)v.w << 96;
                };
                pos += u128(v0);
                neg += u128(v1);
                mag += u128(v2);
                low = min(low, (int)v3.x);
                hish = max(hish, (int)v3.y);
                bad |= v3.z != 0u;
            }
        }
    }
    // warp 0: is the exact sum certified to be the in-order FP64 sum?
    bool need = false;                                  // this lane's column takes the FP64 route
    if (w == 0) {
        // the 128-bit sums cannot have wrapped while c values below 2^(hish + 24) units stay
        // below 2^128: hish + 24 + ceil(log2 c) <= 127
        const bool nowrap = hish + 24 + (32 - __clz(c)) <= 127;
        // exact when |sum| >> low has at most 53 significant bits (only zeros: the sum is +0)
        need = bad || !nowrap || (mag != 0 && top_bit(mag) - low > 52);
        const unsigned nm = __ballot_sync(0xffffffffu, need && i < D);
        if (lane == 0) s_need = nm;
    }
    __syncthreads();                                     // partial sums read; s_need visible
    const unsigned nm = s_need;
    if (nm == 0u && w != 0) return;                      // uniform over the warp
    double s = 0.0;
    if (w == 0 && !need && mag != 0) {
        const bool negative = neg > pos;
        const unsigned __int128 d = negative ? neg - pos : pos - neg;
        const double v = (double)(uint64_t)(d >> low);
        // times 2^(low - 80), a normal power of two (low - 80 lies in [-80, 45])
        s = (negative ? -v : v) * __longlong_as_double((long long)(low - 80 + 1023) << 52);
    }
    if (nm) {
        // the in-order FP64 sum of the flagged columns over all c members: the members are
        // listed in pixel order, then the block's 32 columns of their rows are staged in shared
        // memory, FCH rows at a time and double-buffered; warps 1..UW-1 load the next chunk
        // while warp 0 adds the current one, row by row, in pixel order
        int *mc = lw.ordered + lw.off[j];
        ordered_members(lab, l, j, mc, sscan);
        float (*vals)[FCH][33] = reinterpret_cast<float (*)[FCH][33]>(&sacc[0][0][0]);
        auto stage = [&](int q0, int buf, int w0, int nwarp) {
            const int nrow = min(FCH, c - q0);
            for (int r = w - w0; r < nrow; r += nwarp) vals[buf][r][lane] = __ldg(T + (size_t)mc[q0 + r] * D + ic);
        };
        stage(0, 0, 0, UW);
        __syncthreads();
        const bool mine = w == 0 && ((nm >> lane) & 1u);
        double acc = 0.0;
        for (int q0 = 0, t = 0; q0 < c; q0 += FCH, ++t) {
            if (w != 0 && q0 + FCH < c) stage(q0 + FCH, (t + 1) & 1, 1, UW - 1);
            if (mine) {
                const int nrow = min(FCH, c - q0);
                for (int r = 0; r < nrow; ++r) acc += (double)vals[t & 1][r][lane];
            }
            __syncthreads();
        }
        if (mine) s = acc;
    }
    if (w == 0 && i < D) C[(size_t)j * D + i] = (float)(isfinite(s) ? div_rn(s, (double)c, __ldg(lw.rcp + j)) : s / (double)c);
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

cudaError_t launch_lloyd_update(const float *T, int l, int D, int k, const uint8_t *lab, const LloydWs &lw,
                                float *C, cudaStream_t s)
{
    const int nb = (l + sort_block_labels(l) - 1) / sort_block_labels(l);
    {
        const cudaError_t le_ = launch_pdl(sort_count_kernel, dim3(nb), dim3(kSortThreads), 0, s, lab, l, k, lw.bh);
        if (le_ != cudaSuccess) return le_;
    }
    {
        const cudaError_t le_ = launch_pdl(sort_scatter_kernel, dim3(nb), dim3(kSortThreads), 0, s, lab, l, k, D,
                                           (int)lloyd_max_chunks(l, k), (const int *)lw.bh, lw);
        if (le_ != cudaSuccess) return le_;
    }
    // one block of UW warps per (chunk, 32 dimensions); blocks past the chunks in use return
    dim3 g((unsigned)lloyd_max_chunks(l, k), (D + 31) / 32);
    {
        const cudaError_t le_ = launch_pdl(update_kernel, dim3(g), dim3(32 * UW), 0, s, T, l, D, lab, lw, C);
        if (le_ != cudaSuccess) return le_;
    }
    return cudaGetLastError();
}

}  // namespace vqnnf
