// Integral image of the one-hot NNF, coarse-filter responses and the Eq. 2 similarity.
//
// Integral image (Supp. "Integral Image"; exclusive-prefix reading): for cluster j,
//     S[y][j][x] = #{ (y', x') : y' < y, x' < x, label(y', x') = j },  0 <= y <= H, 0 <= x <= W
// stored channel-planar: element (y, j, x) at (y * k + j) * P + x, P = W + 1 rounded up to a
// multiple of 64 (every 64-column strip of a row is whole, and a 16-bit strip row is one
// 128-byte line).  A half-open rectangle's count is the
// four-corner sum S(y1,x1) - S(y0,x1) - S(y1,x0) + S(y0,x0); a filter is a weighted sum of
// such boxes, i.e. the dilation filter that Algorithm 2 builds on the integral image.
//
// Element type: uint16_t holding S mod 2^16 when every rectangle of the bank is smaller than
// 65,536 pixels (template area <= 65,535) -- the four-corner sum taken mod 2^16 is then the
// exact count -- else uint32_t.
//
// Build, in bands of BH rows so that every warp sweeps few rows:
//   (1) row carries: per row, the count of every cluster left of every 64-column strip;
//   (2) band sums: per (band, strip), the column sums of the row prefixes (exact int32) =
//       the band's carries plus the prefix along x of the band's per-column label counts;
//   (3) exclusive prefix of the band sums over bands = S at every band's first row;
//   (4) one warp per (band, strip, 32 clusters) sweeps its band from there and writes S;
//       each lane owns one cluster and the strip's 64 columns of its plane (in registers),
//       and walks the strip's labels once per row.  Adjacent warps take adjacent strips, so
//       the rows they write are contiguous runs.
//
// Score: one block per (window row, 512 windows).  The corner rows of its windows are
// staged in shared memory one cluster at a time by bulk copies (one per row segment,
// completing on an mbarrier, four buffers in flight); each thread owns four windows and
// accumulates exact integer L1 distances per filter over all clusters, then combines them
// in float32 in a fixed filter order.
#include <cfloat>

#include "common.cuh"
#include "ptx.cuh"
#include "score_spec.cuh"

namespace vqnnf {
namespace {

__device__ int g_score_error = 0;

constexpr int SW = 64;     // columns per strip (two per lane)
constexpr int BH = 64;     // rows per band

// carry[(y * nS + s) * k + j] = #{x' < 64 s : label(y, x') = j}
__global__ void row_carry_kernel(const uint8_t *__restrict__ lab, int W, int k, int nS,
                                 int *__restrict__ carry)
{
    ptx::pdl_enter();
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

// Band sums: one block per (band, strip).  bandsum[(b * k + j) * P + x] for the strip's
// columns x = sum over the band's rows y of #{x' < x : label(y, x') = j}
//          = sum_y carry(y, strip, j) + #{(y, x') : y in band, strip start <= x' < x, label = j}.
__global__ void __launch_bounds__(256) band_sum_kernel(const uint8_t *__restrict__ lab, int H, int W,
                                                       int k, int P, int nS, const int *__restrict__ carry,
                                                       int *__restrict__ bandsum)
{
    ptx::pdl_enter();
    extern __shared__ int cc[];                          // [SW][k] label counts per column, then [k] carry sums
    int *csum_s = cc + SW * k;
    const int s = blockIdx.x, b = blockIdx.y;
    const int x0 = s * SW, y0 = b * BH, y1 = min(H, y0 + BH);
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    for (int q = threadIdx.x; q < SW * k; q += blockDim.x) cc[q] = 0;
    // the band's carry sums, cluster-major (consecutive threads read consecutive clusters),
    // sixteen rows' loads in flight at a time (integer sums: any order is exact)
    for (int j = threadIdx.x; j < k; j += blockDim.x) {
        const int *cp = carry + ((size_t)y0 * nS + s) * k + j;
        const size_t rs = (size_t)nS * k;                // one row further
        int cs = 0, y = y0;
        for (; y + 16 <= y1; y += 16, cp += 16 * rs) {
            int v[16];
#pragma unroll
            for (int u = 0; u < 16; ++u) v[u] = cp[u * rs];
#pragma unroll
            for (int u = 0; u < 16; ++u) cs += v[u];
        }
        for (; y < y1; ++y, cp += rs) cs += *cp;
        csum_s[j] = cs;
    }
    __syncthreads();
    for (int q = threadIdx.x; q < (y1 - y0) * SW; q += blockDim.x) {
        const int y = y0 + q / SW, xx = q % SW, x = x0 + xx;
        if (x < W) {
            const int lb = lab[(size_t)y * W + x];
            if (lb < k) atomicAdd(&cc[xx * k + lb], 1);
        }
    }
    __syncthreads();
    // per cluster: an inclusive warp scan of the 64 column counts (two per lane) shifted by
    // one column, on top of the band's carry sum
    for (int j = w; j < k; j += blockDim.x >> 5) {
        const int csum = csum_s[j];
        const int a0 = cc[(2 * lane) * k + j], a1 = cc[(2 * lane + 1) * k + j];
        int v = a0 + a1;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int t = __shfl_up_sync(0xffffffffu, v, o);
            if (lane >= o) v += t;
        }
        const int ex = v - a0 - a1;                      // counts of the columns left of 2 lane
        const int x = x0 + 2 * lane;
        if (x < P)
            *reinterpret_cast<int2 *>(&bandsum[((size_t)b * k + j) * P + x]) =
                make_int2(csum + ex, csum + ex + a0);
    }
}

// One warp per (band, strip, 32 clusters); lane l owns cluster j = 32 cg + l and keeps the
// band's running S values of the strip's 64 columns in registers.  Per row the strip's labels
// are staged in shared memory (two bytes per lane, double-buffered) and read back whole by
// every lane; the lane walks the 64 columns once, adding its row prefix (the carry plus one
// for every earlier column labelled j) to each column's value.  The finished row of its plane
// goes to a padded shared-memory row (conflict-free 16-byte stores) and from there to global
// memory as one bulk copy, double-buffered: stores of 32 lanes to 32 different planes would
// otherwise each touch a different line.  Columns past the image carry a label byte that no
// lane of the warp owns, so they repeat the value of column W.
template <typename T>
struct SatSweep {
    static constexpr int warps = sizeof(T) == 2 ? 4 : 2;        // warps per block
    static constexpr int pitch = SW * (int)sizeof(T) + 16;       // staged row bytes (padded)
};

template <typename T>
__device__ __forceinline__ void pack_row(uint8_t *dst, const int (&acc)[SW]);
template <>
__device__ __forceinline__ void pack_row<uint16_t>(uint8_t *dst, const int (&acc)[SW])
{
#pragma unroll
    for (int g = 0; g < SW / 8; ++g)
        reinterpret_cast<uint4 *>(dst)[g] = make_uint4(__byte_perm(acc[8 * g], acc[8 * g + 1], 0x5410),
                                                       __byte_perm(acc[8 * g + 2], acc[8 * g + 3], 0x5410),
                                                       __byte_perm(acc[8 * g + 4], acc[8 * g + 5], 0x5410),
                                                       __byte_perm(acc[8 * g + 6], acc[8 * g + 7], 0x5410));
}
template <>
__device__ __forceinline__ void pack_row<uint32_t>(uint8_t *dst, const int (&acc)[SW])
{
#pragma unroll
    for (int g = 0; g < SW / 4; ++g)
        reinterpret_cast<uint4 *>(dst)[g] = make_uint4((uint32_t)acc[4 * g], (uint32_t)acc[4 * g + 1],
                                                       (uint32_t)acc[4 * g + 2], (uint32_t)acc[4 * g + 3]);
}

template <typename T>
__global__ void __launch_bounds__(32 * SatSweep<T>::warps, 4) sat_write_kernel(
    const uint8_t *__restrict__ lab, int H, int W, int k, int P, int nS, int nB, const int *__restrict__ carry,
    const int *__restrict__ bandsum, T *__restrict__ S)
{
    ptx::pdl_enter();
    constexpr int NW = SatSweep<T>::warps, PITCH = SatSweep<T>::pitch;
    __shared__ __align__(16) uint8_t srow[NW][2][SW];
    __shared__ __align__(16) uint8_t sout[NW][2][32][PITCH];
    const int lane = threadIdx.x & 31, wi = threadIdx.x >> 5;
    const int ncg = (k + 31) >> 5;
    const long long gw = (long long)blockIdx.x * NW + wi;
    if (gw >= (long long)nB * nS * ncg) return;              // uniform over the warp
    const int s = (int)(gw % nS);                            // adjacent warps: adjacent strips
    const int cg = (int)((gw / nS) % ncg);
    const int b = (int)(gw / ((long long)ncg * nS));
    const int j = cg * 32 + lane;                            // < 256: k <= 256
    const bool jin = j < k;
    const int jc = jin ? j : k - 1;                          // clamped (every address in bounds)
    const int x0 = s * SW;
    const int ncolv = min(SW, P - x0);                       // S columns of the strip: a multiple of 8
    const uint32_t row_bytes = (uint32_t)(ncolv * (int)sizeof(T));   // a multiple of 16
    const int y0 = b * BH, y1 = min(H, y0 + BH);
    const uint32_t fill = (uint32_t)(((cg + 1) * 32) & 0xFF);   // outside [32 cg, 32 cg + 31]
    const uint32_t jj = (uint32_t)j * 0x01010101u;
    // S at the band's first row: the exclusive prefix of the band sums
    int acc[SW];
    {
        const int *src = bandsum + ((size_t)b * k + jc) * P + x0;
#pragma unroll
        for (int g = 0; g < SW / 4; ++g) {
            int4 v = make_int4(0, 0, 0, 0);
            if (4 * g < ncolv) v = *reinterpret_cast<const int4 *>(src + 4 * g);
            acc[4 * g] = v.x;
            acc[4 * g + 1] = v.y;
            acc[4 * g + 2] = v.z;
            acc[4 * g + 3] = v.w;
        }
    }
    // row yrow of this lane's plane, through staging buffer bsel; a buffer is rewritten only
    // once the copy committed two rows earlier has read it
    auto emit = [&](int yrow, int bsel) {
        if (!jin) return;
        uint8_t *st = &sout[wi][bsel][lane][0];
        ptx::bulk_wait_read<1>();
        pack_row<T>(st, acc);
        ptx::fence_proxy_async();
        ptx::bulk_s2g(S + ((size_t)yrow * k + j) * P + x0, st, row_bytes);
        ptx::bulk_commit();
    };
    if (b == 0) emit(0, 1);                                   // row 0 of S (all zero)
    // labels and carry of the next row are loaded one row ahead; lane l stages columns
    // x0 + 2l and x0 + 2l + 1
    const int xa = x0 + 2 * lane;
    uint32_t la_n = fill, lb_n = fill;
    int c_n = 0;
    if (y0 < y1) {
        const uint8_t *row = lab + (size_t)y0 * W;
        if (xa < W) la_n = row[xa];
        if (xa + 1 < W) lb_n = row[xa + 1];
        c_n = carry[((size_t)y0 * nS + s) * k + jc];
    }
    for (int y = y0; y < y1; ++y) {
        uint8_t *buf = srow[wi][y & 1];
        buf[2 * lane] = (uint8_t)la_n;
        buf[2 * lane + 1] = (uint8_t)lb_n;
        int rp = c_n;
        if (y + 1 < y1) {
            const uint8_t *row = lab + (size_t)(y + 1) * W;
            la_n = xa < W ? row[xa] : fill;
            lb_n = xa + 1 < W ? row[xa + 1] : fill;
            c_n = carry[((size_t)(y + 1) * nS + s) * k + jc];
        }
        __syncwarp();
        uint32_t wd[SW / 4];
#pragma unroll
        for (int q = 0; q < SW / 16; ++q) {
            const uint4 v = reinterpret_cast<const uint4 *>(buf)[q];
            wd[4 * q] = v.x;
            wd[4 * q + 1] = v.y;
            wd[4 * q + 2] = v.z;
            wd[4 * q + 3] = v.w;
        }
#pragma unroll
        for (int q = 0; q < SW / 4; ++q) {
            const uint32_t d = wd[q] ^ jj;                   // a zero byte: that column is labelled j
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                acc[4 * q + u] += rp;
                rp += (d & (0xFFu << (8 * u))) == 0u ? 1 : 0;
            }
        }
        emit(y + 1, y & 1);
    }
    ptx::bulk_wait_read<0>();                                 // staging rows read before the block exits
}

// Exclusive prefix of the band sums over bands, per (cluster, column), in place.
__global__ void band_prefix_kernel(int *__restrict__ bandsum, int nB, long long kP)
{
    ptx::pdl_enter();
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= kP) return;
    int run = 0;
    int b = 0;
    for (; b + 8 <= nB; b += 8) {            // eight independent loads in flight
        int t[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) t[u] = bandsum[(size_t)(b + u) * kP + i];
#pragma unroll
        for (int u = 0; u < 8; ++u) {
            bandsum[(size_t)(b + u) * kP + i] = run;
            run += t[u];
        }
    }
    for (; b < nB; ++b) {
        const int t = bandsum[(size_t)b * kP + i];
        bandsum[(size_t)b * kP + i] = run;
        run += t;
    }
}

// ---------------------------------------------------------------------------------
// Template responses: one block per filter, shared-memory histogram (integer atomics).
// ---------------------------------------------------------------------------------
__global__ void filter_responses_kernel(const uint8_t *__restrict__ lab, int w, int k,
                                        BankSpec bs, int32_t *__restrict__ counts)
{
    ptx::pdl_enter();
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
constexpr int STH = 128;          // threads per block
constexpr int WPT = 4;            // windows per thread
constexpr int TXW = STH * WPT;    // windows per block along x
constexpr int CH = 1;             // clusters per staged chunk
constexpr int NBUF = 4;           // staging buffers of the grid kernel

__device__ __forceinline__ unsigned long long pack_key(float v, unsigned idx)
{
    unsigned b = __float_as_uint(v);
    b = (b & 0x80000000u) ? ~b : (b | 0x80000000u);   // order-preserving
    return ((unsigned long long)b << 32) | (unsigned long long)(0xFFFFFFFFu - idx);
}

// Box count from four integral-image values; exact mod 2^16 for the 16-bit table.
template <typename T>
__device__ __forceinline__ int box(int s11, int s10, int s01, int s00)
{
    const int v = s11 - s10 - s01 + s00;
    return sizeof(T) == 2 ? (v & 0xFFFF) : v;
}

// Thread 0 issues the bulk copies of one chunk of corner rows: for cluster c of the chunk
// and corner row rr, the ncol elements of S starting at column x0, staged pitch elements apart.
template <typename T>
__device__ __forceinline__ void issue_chunk(T *dst, const T *__restrict__ S, int k, int P, int y, int x0,
                                            int j0, int ncol, int pitch, const int *roff, int nrow,
                                            uint64_t *bar)
{
    const int cmax = min(CH, k - j0);
    const uint32_t row_bytes = (uint32_t)(ncol * sizeof(T));
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");   // earlier reads before the refill
    ptx::mbar_expect_tx(bar, row_bytes * (uint32_t)(cmax * nrow));
    for (int c = 0; c < cmax; ++c)
        for (int rr = 0; rr < nrow; ++rr)
            ptx::bulk_g2s(dst + (size_t)(c * nrow + rr) * pitch,
                          S + ((size_t)(y + roff[rr]) * k + (j0 + c)) * P + x0, row_bytes, bar);
}

template <typename T, int G, bool FULL, int NCOLP>
__global__ void __launch_bounds__(STH, G <= 3 ? 8 : 6) score_grid_kernel(const T *__restrict__ S, int P, int k,
                                                         int HO, int WO, GridSpec gs,
                                                         const int32_t *__restrict__ tcounts,
                                                         float *__restrict__ heat,
                                                         unsigned long long *amax)
{
    ptx::pdl_enter();
    // For a single-rectangle filter q and clusters j, with t = template count and n = query
    // count (every pixel carries one label < k, so sum_j n_qj = area_q):
    //     L1_q = sum_j |t_qj - n_qj| = area_q + sum_{j : t_qj > 0} (|t_qj - n_qj| - n_qj)
    // so cluster j only costs work in the cells where the template holds it.
    constexpr int NR = G + 1;
    constexpr int NSLOT = G * G + (FULL ? 1 : 0);
    extern __shared__ __align__(128) uint8_t smem_raw[];
    // staged rows are NCOLP elements apart (a compile-time pitch >= ncol), so that every
    // corner load of the inner loop is a per-thread column pointer plus an immediate offset
    const int ncol = gs.ncol;
    constexpr int chunk_elems = CH * NR * NCOLP;
    T *bufs = reinterpret_cast<T *>(smem_raw);                               // [NBUF][chunk]
    int *tc = reinterpret_cast<int *>(bufs + NBUF * chunk_elems);           // [NSLOT][k]
    unsigned *cmask = reinterpret_cast<unsigned *>(tc + NSLOT * k);          // [k]
    uint64_t *full = reinterpret_cast<uint64_t *>(cmask + k + ((NSLOT * k + k) & 1));
    uint64_t *empty = full + NBUF;
    int *n_issued = reinterpret_cast<int *>(empty + NBUF);
    const int y = blockIdx.y;
    const int x0 = blockIdx.x * TXW;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int nchunk = (k + CH - 1) / CH;
    for (int q = threadIdx.x; q < NSLOT * k; q += blockDim.x) {
        const int slot = q / k, j = q % k;
        tc[q] = tcounts[(size_t)gs.slot_filter[slot] * k + j];
    }
    if (threadIdx.x == 0) {
        for (int b = 0; b < NBUF; ++b) {
            ptx::mbar_init(&full[b], 1);
            ptx::mbar_init(&empty[b], STH / 32);
        }
        ptx::fence_barrier_init();
        int c = 0;
        for (; c < NBUF - 1 && c < nchunk; ++c)
            issue_chunk<T>(bufs + c * chunk_elems, S, k, P, y, x0, c * CH, ncol, NCOLP, gs.by, NR, &full[c]);
        *n_issued = c;
    }
    __syncthreads();
    for (int j = threadIdx.x; j < k; j += blockDim.x) {
        unsigned m = 0;
#pragma unroll
        for (int q = 0; q < NSLOT; ++q) m |= (tc[q * k + j] > 0 ? 1u : 0u) << q;
        cmask[j] = m;
    }
    // per-window corner column offsets are the same for every cluster
    int off[NR];
#pragma unroll
    for (int cc = 0; cc < NR; ++cc) off[cc] = gs.bx[cc];
    int acc[WPT][NSLOT];
#pragma unroll
    for (int w = 0; w < WPT; ++w)
#pragma unroll
        for (int q = 0; q < NSLOT; ++q) acc[w][q] = gs.slot_area[q];
    __syncthreads();
    bool ok = true;
    for (int ch = 0; ch < nchunk; ++ch) {
        const int b = ch % NBUF;
        if (threadIdx.x == 0 && ch + NBUF - 1 < nchunk) {
            // refill the buffer that chunk ch - 1 used, once every warp has released it
            const int nb = (ch + NBUF - 1) % NBUF;
            const int use = (ch + NBUF - 1) / NBUF;          // how many times nb was filled before
            if (use > 0)
                ok = ptx::mbar_wait_bounded(&empty[nb], (use - 1) & 1, &g_score_error, (int)VQNNF_ETIMEOUT);
            if (ok) {
                issue_chunk<T>(bufs + nb * chunk_elems, S, k, P, y, x0, (ch + NBUF - 1) * CH, ncol, NCOLP,
                               gs.by, NR, &full[nb]);
                *n_issued = ch + NBUF;
            }
        }
        ok = __all_sync(0xffffffffu, ok && ptx::mbar_wait_bounded(&full[b], (ch / NBUF) & 1, &g_score_error,
                                                                  (int)VQNNF_ETIMEOUT));
        if (!ok) break;
        const T *cur = bufs + b * chunk_elems + threadIdx.x;
        const int cmax = min(CH, k - ch * CH);
        const T *pc[NR];                                  // this thread's column of each corner column
#pragma unroll
        for (int cc = 0; cc < NR; ++cc) pc[cc] = cur + off[cc];
#pragma unroll
        for (int c = 0; c < CH; ++c) {
            if (c >= cmax) break;
            const int j = ch * CH + c;
            const unsigned m = cmask[j];                    // same for every thread: uniform branches
#pragma unroll
            for (int q = 0; q < NSLOT; ++q) {
                if (!(m & (1u << q))) continue;
                const int t = tc[q * k + j];
                const int r0 = (FULL && q == NSLOT - 1) ? 0 : q / G;
                const int r1 = (FULL && q == NSLOT - 1) ? G : q / G + 1;
                const int c0 = (FULL && q == NSLOT - 1) ? 0 : q % G;
                const int c1 = (FULL && q == NSLOT - 1) ? G : q % G + 1;
#pragma unroll
                for (int w = 0; w < WPT; ++w) {
                    const int o0 = (c * NR + r0) * NCOLP + w * STH, o1 = (c * NR + r1) * NCOLP + w * STH;
                    const int n = box<T>((int)pc[c1][o1], (int)pc[c0][o1], (int)pc[c1][o0], (int)pc[c0][o0]);
                    acc[w][q] = (int)__sad(t, n, (unsigned)acc[w][q]) - n;
                }
            }
        }
        __syncwarp();
        if (lane == 0) asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(ptx::smem_u32(&empty[b]))
                                    : "memory");
    }
    if (!__syncthreads_and(ok) && threadIdx.x == 0) {
        // a wait gave up: let every bulk copy issued into shared memory land (bounded)
        // before the block exits
        const int issued = *n_issued;
        for (int c = max(0, issued - NBUF); c < issued; ++c)
            ptx::mbar_wait_bounded(&full[c % NBUF], (c / NBUF) & 1, &g_score_error, (int)VQNNF_ETIMEOUT);
    }
    (void)warp;
    // combine in a fixed (cell-major, full window last) order: H = - sum_q coef_q * L1_q
    unsigned long long best = 0ull;
#pragma unroll
    for (int w = 0; w < WPT; ++w) {
        const int x = x0 + threadIdx.x + w * STH;
        float accf = 0.f;
#pragma unroll
        for (int q = 0; q < NSLOT; ++q) accf = fmaf(gs.slot_coef[q], (float)acc[w][q], accf);
        const float h = -accf;
        if (ok && x < WO) {
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

// Weighted-grid bank (WGridSpec): grid by grid, one pass over the clusters stages that grid's
// four corner rows; per cluster and window the 16 corners give the 9 cell counts, each of the
// grid's filters is their integer weighting R, and |t - R| is summed exactly per filter.  The
// weights and coefficients are kernel parameters indexed at compile time.  After each grid's
// pass its filters' sums enter the float heatmap accumulator (fixed order).
template <typename T, int NG, int NCOLP>
__global__ void __launch_bounds__(STH, 6) score_wgrid_kernel(const T *__restrict__ S, int P, int k,
                                                          int HO, int WO, WGridSpec ws,
                                                          const int32_t *__restrict__ tcounts,
                                                          float *__restrict__ heat,
                                                          unsigned long long *amax)
{
    ptx::pdl_enter();
    extern __shared__ __align__(128) uint8_t smem_raw[];
    const int ncol = ws.ncol;
    constexpr int chunk_elems = 4 * NCOLP;                    // one cluster, four corner rows
    T *bufs = reinterpret_cast<T *>(smem_raw);                 // [NBUF][chunk]
    int *tc = reinterpret_cast<int *>(bufs + NBUF * chunk_elems);   // [NG][5][k]
    uint64_t *full = reinterpret_cast<uint64_t *>(tc + NG * kMaxWFilters * k + ((NG * kMaxWFilters * k) & 1));
    uint64_t *empty = full + NBUF;
    int *n_issued = reinterpret_cast<int *>(empty + NBUF);
    const int y = blockIdx.y;
    const int x0 = blockIdx.x * TXW;
    const int lane = threadIdx.x & 31;
    const int nchunk = NG * k;                                 // chunk ci: grid ci / k, cluster ci % k
    for (int q = threadIdx.x; q < NG * kMaxWFilters * k; q += blockDim.x) {
        const int gf = q / k, j = q % k, g = gf / kMaxWFilters, f = gf % kMaxWFilters;
        tc[q] = f < ws.nf[g] ? tcounts[(size_t)ws.filt[g][f] * k + j] : 0;
    }
    if (threadIdx.x == 0) {
        for (int b = 0; b < NBUF; ++b) {
            ptx::mbar_init(&full[b], 1);
            ptx::mbar_init(&empty[b], STH / 32);
        }
        ptx::fence_barrier_init();
        int c = 0;
        for (; c < NBUF - 1 && c < nchunk; ++c)
            issue_chunk<T>(bufs + c * chunk_elems, S, k, P, y, x0, c % k, ncol, NCOLP, ws.by[c / k], 4, &full[c]);
        *n_issued = c;
    }
    __syncthreads();
    float hs[WPT];
#pragma unroll
    for (int w = 0; w < WPT; ++w) hs[w] = 0.f;
    bool ok = true;
#pragma unroll
    for (int g = 0; g < NG; ++g) {
        const int nf = ws.nf[g];
        int acc[WPT][kMaxWFilters];
#pragma unroll
        for (int w = 0; w < WPT; ++w)
#pragma unroll
            for (int f = 0; f < kMaxWFilters; ++f) acc[w][f] = 0;
        int off[4];
#pragma unroll
        for (int cc = 0; cc < 4; ++cc) off[cc] = ws.bx[g][cc];
        for (int j = 0; ok && j < k; ++j) {
            const int ch = g * k + j;
            const int b = ch % NBUF;
            if (threadIdx.x == 0 && ch + NBUF - 1 < nchunk) {
                const int nb = (ch + NBUF - 1) % NBUF;
                const int use = (ch + NBUF - 1) / NBUF;
                if (use > 0)
                    ok = ptx::mbar_wait_bounded(&empty[nb], (use - 1) & 1, &g_score_error, (int)VQNNF_ETIMEOUT);
                if (ok) {
                    const int cn = ch + NBUF - 1;
                    issue_chunk<T>(bufs + nb * chunk_elems, S, k, P, y, x0, cn % k, ncol, NCOLP, ws.by[cn / k], 4,
                                   &full[nb]);
                    *n_issued = cn + 1;
                }
            }
            ok = __all_sync(0xffffffffu, ok && ptx::mbar_wait_bounded(&full[b], (ch / NBUF) & 1, &g_score_error,
                                                                      (int)VQNNF_ETIMEOUT));
            if (!ok) break;
            const T *cur = bufs + b * chunk_elems + threadIdx.x;
            int t[kMaxWFilters];
#pragma unroll
            for (int f = 0; f < kMaxWFilters; ++f) t[f] = tc[(g * kMaxWFilters + f) * k + j];
#pragma unroll
            for (int w = 0; w < WPT; ++w) {
                int cr[4][4];
#pragma unroll
                for (int r = 0; r < 4; ++r)
#pragma unroll
                    for (int cc = 0; cc < 4; ++cc) cr[r][cc] = (int)cur[off[cc] + r * NCOLP + w * STH];
                int n[9];
#pragma unroll
                for (int r = 0; r < 3; ++r)
#pragma unroll
                    for (int cc = 0; cc < 3; ++cc)
                        n[r * 3 + cc] = box<T>(cr[r + 1][cc + 1], cr[r + 1][cc], cr[r][cc + 1], cr[r][cc]);
#pragma unroll
                for (int f = 0; f < kMaxWFilters; ++f) {
                    if (f >= nf) break;
                    int R = 0;
#pragma unroll
                    for (int c = 0; c < 9; ++c) R += ws.w[g][f][c] * n[c];
                    acc[w][f] += abs(t[f] - R);
                }
            }
            __syncwarp();
            if (lane == 0) asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(ptx::smem_u32(&empty[b]))
                                        : "memory");
        }
#pragma unroll
        for (int f = 0; f < kMaxWFilters; ++f) {
            if (f >= nf) break;
#pragma unroll
            for (int w = 0; w < WPT; ++w) hs[w] = fmaf(ws.coef[g][f], (float)acc[w][f], hs[w]);
        }
    }
    if (!__syncthreads_and(ok) && threadIdx.x == 0) {
        const int issued = *n_issued;
        for (int c = max(0, issued - NBUF); c < issued; ++c)
            ptx::mbar_wait_bounded(&full[c % NBUF], (c / NBUF) & 1, &g_score_error, (int)VQNNF_ETIMEOUT);
    }
    unsigned long long best = 0ull;
#pragma unroll
    for (int w = 0; w < WPT; ++w) {
        const int x = x0 + threadIdx.x + w * STH;
        const float h = -hs[w];
        if (ok && x < WO) {
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
template <typename T>
__global__ void __launch_bounds__(STH) score_generic_kernel(const T *__restrict__ S, int P, int k,
                                                            int HO, int WO, BankSpec bs,
                                                            const int32_t *__restrict__ tcounts,
                                                            float *__restrict__ heat,
                                                            unsigned long long *amax)
{
    ptx::pdl_enter();
    extern __shared__ __align__(128) uint8_t smem_raw[];
    const int ncol = bs.ncol, nrow = bs.nrow;
    T *buf0 = reinterpret_cast<T *>(smem_raw);
    T *buf1 = buf0 + (size_t)CH * nrow * ncol;
    int *tc = reinterpret_cast<int *>(buf1 + (size_t)CH * nrow * ncol);      // [F][k]
    uint64_t *bar = reinterpret_cast<uint64_t *>(tc + bs.F * k + (bs.F * k & 1));
    const int y = blockIdx.y;
    const int x0 = blockIdx.x * TXW;
    const int nchunk = (k + CH - 1) / CH;
    for (int q = threadIdx.x; q < bs.F * k; q += blockDim.x) tc[q] = tcounts[q];
    if (threadIdx.x == 0) {
        ptx::mbar_init(&bar[0], 1);
        ptx::mbar_init(&bar[1], 1);
        ptx::fence_barrier_init();
        issue_chunk<T>(buf0, S, k, P, y, x0, 0, ncol, ncol, bs.roff, nrow, &bar[0]);
    }
    __syncthreads();
    long long l1[WPT][kMaxFilters];
    for (int w = 0; w < WPT; ++w)
        for (int f = 0; f < kMaxFilters; ++f) l1[w][f] = 0;
    bool ok = true;
    for (int ch = 0; ch < nchunk; ++ch) {
        T *cur = (ch & 1) ? buf1 : buf0;
        if (threadIdx.x == 0 && ch + 1 < nchunk)
            issue_chunk<T>((ch & 1) ? buf0 : buf1, S, k, P, y, x0, (ch + 1) * CH, ncol, ncol, bs.roff, nrow,
                           &bar[(ch + 1) & 1]);
        ok = ptx::mbar_wait_bounded(&bar[ch & 1], (ch >> 1) & 1, &g_score_error, (int)VQNNF_ETIMEOUT);
        if (!__syncthreads_and(ok)) { ok = false; break; }
        const int cmax = min(CH, k - ch * CH);
        for (int c = 0; c < cmax; ++c) {
            const int j = ch * CH + c;
            const T *base = cur + (size_t)c * nrow * ncol;
            for (int f = 0; f < bs.F; ++f) {
                const int t = tc[f * k + j];
                for (int w = 0; w < WPT; ++w) {
                    const int xl = threadIdx.x + w * STH;
                    int v = 0;
                    for (int r = bs.rect_begin[f]; r < bs.rect_begin[f + 1]; ++r) {
                        const RectSpec rc = bs.rect[r];
                        const T *r0 = base + rc.ry0 * ncol + xl;
                        const T *r1 = base + rc.ry1 * ncol + xl;
                        v += rc.weight * box<T>(r1[rc.x1], r1[rc.x0], r0[rc.x1], r0[rc.x0]);
                    }
                    l1[w][f] += abs(t - v);
                }
            }
        }
        __syncthreads();
    }
    unsigned long long best = 0ull;
    for (int w = 0; w < WPT; ++w) {
        const int x = x0 + threadIdx.x + w * STH;
        float acc = 0.f;
        for (int f = 0; f < bs.F; ++f) acc = fmaf(bs.coef[f], (float)l1[w][f], acc);
        const float h = -acc;
        if (ok && x < WO) {
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

// Self-test of the bounded waits: one thread waits on an mbarrier that nothing completes.  No
// copy is issued, so nothing is in flight when the wait gives up after `limit` SM cycles and
// records VQNNF_ETIMEOUT in the score kernels' error word.
__global__ void wait_selftest_kernel(long long limit)
{
    __shared__ __align__(8) uint64_t bar;
    ptx::mbar_init(&bar, 1);
    ptx::fence_barrier_init();
    (void)ptx::mbar_wait_for(&bar, 0, &g_score_error, (int)VQNNF_ETIMEOUT, limit);
}

__global__ void argmax_finish_kernel(const unsigned long long *amax, int WO, int32_t *out)
{
    ptx::pdl_enter();
    const unsigned idx = 0xFFFFFFFFu - (unsigned)(*amax & 0xFFFFFFFFull);
    out[0] = (int32_t)(idx / (unsigned)WO);
    out[1] = (int32_t)(idx % (unsigned)WO);
}

template <typename T, int G, bool FULL>
cudaError_t launch_grid(const T *S, int P, int k, int HO, int WO, const GridSpec &gs,
                        const int32_t *tc, float *heat, unsigned long long *amax, cudaStream_t s)
{
    BankSpec none;
    none.F = 0;
    const size_t smem = score_smem_bytes_for(sizeof(T), none, gs, k);
    dim3 grid((WO + TXW - 1) / TXW, HO);
    cudaError_t e;
    if (gs.ncol <= TXW + 128) {
        e = cudaFuncSetAttribute(score_grid_kernel<T, G, FULL, TXW + 128>,
                                 cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        {
        const cudaError_t le_ = launch_pdl(score_grid_kernel<T, G, FULL, TXW + 128>, dim3(grid), dim3(STH), smem, s, S, P, k, HO, WO, gs, tc, heat, amax);
        if (le_ != cudaSuccess) return le_;
    }
    } else {
        e = cudaFuncSetAttribute(score_grid_kernel<T, G, FULL, TXW + 256>,
                                 cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        {
        const cudaError_t le_ = launch_pdl(score_grid_kernel<T, G, FULL, TXW + 256>, dim3(grid), dim3(STH), smem, s, S, P, k, HO, WO, gs, tc, heat, amax);
        if (le_ != cudaSuccess) return le_;
    }
    }
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_sat_t(const uint8_t *lab, int H, int W, int k, int *carry, int *bandsum, T *S,
                         cudaStream_t s)
{
    const int nS = sat_strips(W);
    const int P = sat_pitch(W);
    const int nB = sat_bands(H);
    const size_t hsmem = sizeof(int) * (size_t)nS * k;
    cudaError_t e = cudaFuncSetAttribute(row_carry_kernel,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)hsmem);
    if (e != cudaSuccess) return e;
    {
        const cudaError_t le_ = launch_pdl(row_carry_kernel, dim3(H), dim3(256), hsmem, s, lab, W, k, nS, carry);
        if (le_ != cudaSuccess) return le_;
    }
    const size_t csmem = sizeof(int) * ((size_t)SW * k + k);
    e = cudaFuncSetAttribute(band_sum_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)csmem);
    if (e != cudaSuccess) return e;
    {
        const cudaError_t le_ = launch_pdl(band_sum_kernel, dim3(dim3(nS, nB)), dim3(256), csmem, s, lab, H, W, k, P, nS, carry, bandsum);
        if (le_ != cudaSuccess) return le_;
    }
    const long long kP = (long long)k * P;
    {
        const cudaError_t le_ = launch_pdl(band_prefix_kernel, dim3((unsigned)((kP + 255) / 256)), dim3(256), 0, s, bandsum, nB, kP);
        if (le_ != cudaSuccess) return le_;
    }
    const long long nwarps = (long long)nB * nS * ((k + 31) / 32);
    constexpr int NW = SatSweep<T>::warps;
    const unsigned blocks = (unsigned)((nwarps + NW - 1) / NW);
    {
        const cudaError_t le_ = launch_pdl(sat_write_kernel<T>, dim3(blocks), dim3(32 * NW), 0, s, lab, H, W, k, P, nS, nB, carry, bandsum, S);
        if (le_ != cudaSuccess) return le_;
    }
    return cudaGetLastError();
}

template <typename T, int NG>
cudaError_t launch_wgrid(const T *S, int P, int k, int HO, int WO, const WGridSpec &ws, const int32_t *tc,
                         float *heat, unsigned long long *amax, cudaStream_t s)
{
    const size_t smem = score_wgrid_smem_bytes(sizeof(T), ws, k);
    dim3 grid((WO + TXW - 1) / TXW, HO);
    cudaError_t e;
    if (ws.ncol <= TXW + 128) {
        e = cudaFuncSetAttribute(score_wgrid_kernel<T, NG, TXW + 128>,
                                 cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        {
        const cudaError_t le_ = launch_pdl(score_wgrid_kernel<T, NG, TXW + 128>, dim3(grid), dim3(STH), smem, s, S, P, k, HO, WO, ws, tc, heat, amax);
        if (le_ != cudaSuccess) return le_;
    }
    } else {
        e = cudaFuncSetAttribute(score_wgrid_kernel<T, NG, TXW + 256>,
                                 cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        {
        const cudaError_t le_ = launch_pdl(score_wgrid_kernel<T, NG, TXW + 256>, dim3(grid), dim3(STH), smem, s, S, P, k, HO, WO, ws, tc, heat, amax);
        if (le_ != cudaSuccess) return le_;
    }
    }
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_score_t(const T *S, int W, int k, int HO, int WO, const BankSpec &bs,
                           const GridSpec &gs, const WGridSpec &ws, const int32_t *tc, float *heat,
                           unsigned long long *amax, int32_t *argmax_yx, cudaStream_t s)
{
    const int P = sat_pitch(W);
    cudaError_t e = cudaSuccess;
    if (amax) {
        e = cudaMemsetAsync(amax, 0, sizeof(unsigned long long), s);
        if (e != cudaSuccess) return e;
    }
    if ((e = record_kernel_event(VQNNF_OP_SCORE, 0, s)) != cudaSuccess) return e;
    bool done = false;
#define VQNNF_GRID_CASE(GG, FF)                                                         \
    if (!done && gs.G == GG && gs.full == FF) {                                         \
        e = launch_grid<T, GG, FF>(S, P, k, HO, WO, gs, tc, heat, amax, s);              \
        done = true;                                                                    \
    }
    VQNNF_GRID_CASE(1, false) VQNNF_GRID_CASE(1, true) VQNNF_GRID_CASE(2, false)
    VQNNF_GRID_CASE(2, true) VQNNF_GRID_CASE(3, false) VQNNF_GRID_CASE(3, true)
    VQNNF_GRID_CASE(4, false) VQNNF_GRID_CASE(4, true)
#undef VQNNF_GRID_CASE
    if (!done && ws.NG > 0) {
        switch (ws.NG) {
        case 1: e = launch_wgrid<T, 1>(S, P, k, HO, WO, ws, tc, heat, amax, s); break;
        case 2: e = launch_wgrid<T, 2>(S, P, k, HO, WO, ws, tc, heat, amax, s); break;
        case 3: e = launch_wgrid<T, 3>(S, P, k, HO, WO, ws, tc, heat, amax, s); break;
        default: e = launch_wgrid<T, 4>(S, P, k, HO, WO, ws, tc, heat, amax, s); break;
        }
        done = true;
    }
    if (!done) {
        GridSpec none;
        none.G = 0;
        const size_t smem = score_smem_bytes_for(sizeof(T), bs, none, k);
        e = cudaFuncSetAttribute(score_generic_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)smem);
        if (e != cudaSuccess) return e;
        dim3 grid((WO + TXW - 1) / TXW, HO);
        {
        const cudaError_t le_ = launch_pdl(score_generic_kernel<T>, dim3(grid), dim3(STH), smem, s, S, P, k, HO, WO, bs, tc, heat, amax);
        if (le_ != cudaSuccess) return le_;
    }
        e = cudaGetLastError();
    }
    if (e != cudaSuccess) return e;
    if ((e = record_kernel_event(VQNNF_OP_SCORE, 1, s)) != cudaSuccess) return e;
    if (argmax_yx && amax) {
        {
        const cudaError_t le_ = launch_pdl(argmax_finish_kernel, dim3(1), dim3(1), 0, s, amax, WO, argmax_yx);
        if (le_ != cudaSuccess) return le_;
    }
        e = cudaGetLastError();
    }
    return e;
}

}  // namespace

// Staged row pitch of the grid kernel for a window strip of ncol columns (template width up
// to 256; wider templates take the generic kernel).
int score_grid_pitch(int ncol) { return ncol <= TXW + 128 ? TXW + 128 : TXW + 256; }
bool score_grid_fits(int ncol) { return ncol <= TXW + 256; }

size_t score_wgrid_smem_bytes(size_t elem, const WGridSpec &ws, int k)
{
    return elem * (size_t)NBUF * 4 * score_grid_pitch(ws.ncol) + sizeof(int) * ((size_t)ws.NG * kMaxWFilters * k + 1) +
           sizeof(uint64_t) * 2 * NBUF + 16 + 16;
}


size_t score_smem_bytes_for(size_t elem, const BankSpec &bs, const GridSpec &gs, int k)
{
    if (gs.G > 0) {
        const int NR = gs.G + 1;
        const int NSLOT = gs.G * gs.G + (gs.full ? 1 : 0);
        return elem * (size_t)NBUF * CH * NR * score_grid_pitch(gs.ncol) + sizeof(int) * ((size_t)NSLOT * k + k + 1) +
               sizeof(uint64_t) * 2 * NBUF + 16 + 16;
    }
    return elem * (size_t)2 * CH * bs.nrow * bs.ncol + sizeof(int) * ((size_t)bs.F * k + 1) + 32;
}

bool sat_is_u16(int th, int tw) { return (long long)th * tw <= 65535; }
int sat_pitch(int W) { return (W + 1 + 63) / 64 * 64; }
int sat_strips(int W) { return (W + 1 + SW - 1) / SW; }
int sat_bands(int H) { return (H + BH - 1) / BH; }
int score_ncol(int tw) { return (TXW + tw + 7) / 8 * 8; }
size_t sat_slack_elems(int tw) { return (size_t)score_ncol(tw) + 64; }

cudaError_t launch_sat(const uint8_t *lab, int H, int W, int k, bool u16, int *carry, int *bandsum,
                       void *S, cudaStream_t s)
{
    return u16 ? launch_sat_t<uint16_t>(lab, H, W, k, carry, bandsum, static_cast<uint16_t *>(S), s)
               : launch_sat_t<uint32_t>(lab, H, W, k, carry, bandsum, static_cast<uint32_t *>(S), s);
}

cudaError_t launch_filter_responses(const uint8_t *lab, int h, int w, int k, const BankSpec &bs,
                                    int32_t *counts, cudaStream_t s)
{
    (void)h;
    {
        const cudaError_t le_ = launch_pdl(filter_responses_kernel, dim3(bs.F), dim3(256), 0, s, lab, w, k, bs, counts);
        if (le_ != cudaSuccess) return le_;
    }
    return cudaGetLastError();
}

cudaError_t launch_score(const void *S, bool u16, int W, int k, int HO, int WO, const BankSpec &bs,
                         const GridSpec &gs, const WGridSpec &ws, const int32_t *tc, float *heat,
                         unsigned long long *amax, int32_t *argmax_yx, cudaStream_t s)
{
    return u16 ? launch_score_t<uint16_t>(static_cast<const uint16_t *>(S), W, k, HO, WO, bs, gs, ws, tc,
                                          heat, amax, argmax_yx, s)
               : launch_score_t<uint32_t>(static_cast<const uint32_t *>(S), W, k, HO, WO, bs, gs, ws, tc,
                                          heat, amax, argmax_yx, s);
}

cudaError_t launch_wait_selftest(long long limit_cycles, cudaStream_t s)
{
    wait_selftest_kernel<<<1, 1, 0, s>>>(limit_cycles);
    return cudaGetLastError();
}

cudaError_t read_and_clear_score_error(int *out)
{
    int zero = 0;
    cudaError_t e = cudaMemcpyFromSymbol(out, g_score_error, sizeof(int));
    if (e == cudaSuccess) e = cudaMemcpyToSymbol(g_score_error, &zero, sizeof(int));
    return e;
}

}  // namespace vqnnf
