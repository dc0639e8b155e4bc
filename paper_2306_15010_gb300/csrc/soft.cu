// Soft vector-quantised heatmap (the differentiable reading of Algorithm 1, Eq. 1 and Eq. 2)
// and its gradients.
//
//   p_j(x)    = softmax_j( -||x - c_j||^2 / tau )                      (soft NNF)
//   T_fj      = sum over template pixels v in cell f of p_j(v)          (soft counts, Eq. 1)
//   Q_fj(y,x) = sum over query pixels u in cell f + (y, x) of p_j(u)
//   H(y,x)    = - sum_f (w_f / A_f) sum_j | T_fj - Q_fj(y, x) |         (Eq. 2, L1 norm)
//
// The filters are the G x G cells of the template window (floor boundaries); the cells have
// at most two widths and two heights, so every query soft count is a read of one of at most
// four per-cluster box-sum maps BX_s (s = cell size), built by separable direct sums (no
// integral image: FP32 prefix sums would lose the counts to cancellation).
//
// Backward, for L = sum Gw * H:
//   dL/dw_f      = - sum_{y,x} Gw L1_f / A_f
//   m_fj(y,x)    = -(w_f / A_f) Gw(y,x) sign(Q_fj(y,x) - T_fj)          (dL/dQ_fj)
//   dL/dT_fj     = - sum_{y,x} m_fj(y,x)
//   g_j(u)       = sum_f sum_{windows whose cell f covers u} m_fj         (adjoint box sums)
//   a_j(u)       = -(1/tau) p_j (g_j - sum_i p_i g_i)                    (p kept from the forward)
//   dL/dx_u      = 2 (sum_j a_j) x_u - 2 sum_j a_j c_j
//   dL/dc_j      = -2 sum_u a_j(u) x_u + 2 (sum_u a_j(u)) c_j   (query and template pixels)
#include <cfloat>

#include "common.cuh"
#include "soft_spec.cuh"

namespace vqnnf {
namespace {

constexpr int PT = 64;             // pixels per tile of the soft-assignment kernels
constexpr int DCH = 32;            // feature dimensions staged per chunk
constexpr int PPT = 4;             // pixels per thread: pg * 4 .. pg * 4 + 3
// KI (template parameter): centroids per thread, thread (pg, cl) holds j = cl + 16 i, i < KI;
// 16 KI >= k (2, 4 or 8)

// Planar offset of pixel p0 + pp of cluster plane j, P[(item * k + j) * npi + pixel], from the
// tile's first item and offset (one 64-bit division per tile, not per element).
__device__ __forceinline__ long long planar_index(long long it0, long long of0, int pp, int j, int k, long long npi)
{
    long long it = it0, of = of0 + pp;
    if (of >= npi) {                                          // the tile straddles items
        it += of / npi;
        of %= npi;
    }
    return (it * k + j) * npi + of;
}

// Tile of the soft-assignment kernel: 16 pixel groups of PPT pixels.
template <int KI>
struct SoftTile {
    static constexpr int PPT = KI <= 4 ? 8 : 4;
    static constexpr int PT = 16 * PPT;
};

// Distances of a tile of 16 PPT pixels to all k centroids and the softmax over each pixel's k
// logits.  Thread t = 16 pg + cl owns pixels PPT pg .. PPT pg + PPT - 1 and centroids cl,
// cl + 16, ... (PPT = 8 pixels for k <= 64, else 4, so that the register tile stays within
// budget; the larger tile halves the shared-memory loads per (pixel, centroid) pair); the 16
// threads of a pixel group are consecutive lanes (half a warp).  X rows are pixels.  The
// direct differences run on packed pairs of pixels (two FP32 lanes per instruction, each
// rounded as the scalar subtraction and FMA would be): the centroid chunk is staged negated,
// cs[j][dd] = -c, and paired as (-c, -c) in registers, so one add and one FMA cover two
// (pixel, centroid) pairs.
template <int KI>
__device__ __forceinline__ void tile_softmax(const float *__restrict__ X, long long n, long long p0, int D,
                                             const float *__restrict__ C, int k, float tau, float (*xs)[DCH + 1],
                                             float (*cs)[DCH + 1], float (*pr)[KI])
{
    constexpr int PPTK = SoftTile<KI>::PPT, PTK = SoftTile<KI>::PT;
    const int t = threadIdx.x, pg = t >> 4, cl = t & 15;
    float2 acc[PPTK / 2][KI];
#pragma unroll
    for (int r = 0; r < PPTK / 2; ++r)
#pragma unroll
        for (int i = 0; i < KI; ++i) acc[r][i] = make_float2(0.f, 0.f);
    // the next chunk's features and centroids are loaded into registers while the current one
    // is consumed (256 threads: XE and CE elements each)
    constexpr int XE = PTK * DCH / 256, CE = 16 * KI * DCH / 256;
    float xr[XE], cr[CE];
    auto fetch = [&](int d0) {
#pragma unroll
        for (int q = 0; q < XE; ++q) {
            const int e = t + 256 * q, pp = e / DCH, dd = e % DCH;
            const long long g = p0 + pp;
            xr[q] = (g < n && d0 + dd < D) ? X[g * D + d0 + dd] : 0.f;
        }
#pragma unroll
        for (int q = 0; q < CE; ++q) {
            const int e = t + 256 * q, j = e / DCH, dd = e % DCH;
            cr[q] = (j < k && d0 + dd < D) ? -C[(size_t)j * D + d0 + dd] : 0.f;
        }
    };
    fetch(0);
    for (int d0 = 0; d0 < D; d0 += DCH) {
        __syncthreads();                                       // the previous chunk is consumed
#pragma unroll
        for (int q = 0; q < XE; ++q) {
            const int e = t + 256 * q;
            xs[e / DCH][e % DCH] = xr[q];
        }
#pragma unroll
        for (int q = 0; q < CE; ++q) {
            const int e = t + 256 * q;
            cs[e / DCH][e % DCH] = cr[q];
        }
        __syncthreads();
        if (d0 + DCH < D) fetch(d0 + DCH);
#pragma unroll 2
        for (int dd = 0; dd < DCH; ++dd) {
            float2 xv[PPTK / 2], cv[KI];
#pragma unroll
            for (int r = 0; r < PPTK / 2; ++r)
                xv[r] = make_float2(xs[pg * PPTK + 2 * r][dd], xs[pg * PPTK + 2 * r + 1][dd]);
#pragma unroll
            for (int i = 0; i < KI; ++i) {
                const float c = (cl + 16 * i < k) ? cs[cl + 16 * i][dd] : 0.f;
                cv[i] = make_float2(c, c);
            }
#pragma unroll
            for (int r = 0; r < PPTK / 2; ++r)
#pragma unroll
                for (int i = 0; i < KI; ++i) {
                    const float2 df = __fadd2_rn(xv[r], cv[i]);
                    acc[r][i] = __ffma2_rn(df, df, acc[r][i]);
                }
        }
    }
    const float it = 1.0f / tau;
#pragma unroll
    for (int r = 0; r < PPTK; ++r) {
        float dr[KI];
#pragma unroll
        for (int i = 0; i < KI; ++i) dr[i] = (r & 1) ? acc[r >> 1][i].y : acc[r >> 1][i].x;
        float dmin = FLT_MAX;
#pragma unroll
        for (int i = 0; i < KI; ++i)
            if (cl + 16 * i < k) dmin = fminf(dmin, dr[i]);
#pragma unroll
        for (int o = 1; o < 16; o <<= 1) dmin = fminf(dmin, __shfl_xor_sync(0xffffffffu, dmin, o));
        float s = 0.f;
#pragma unroll
        for (int i = 0; i < KI; ++i) {
            const float e = cl + 16 * i < k ? expf((dmin - dr[i]) * it) : 0.f;
            dr[i] = e;
            s += e;
        }
#pragma unroll
        for (int o = 1; o < 16; o <<= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
        const float inv = 1.0f / s;
#pragma unroll
        for (int i = 0; i < KI; ++i) pr[r][i] = dr[i] * inv;
    }
}

// p planar: P[(item * k + j) * npi + pixel], written through a shared-memory transpose so that
// consecutive threads store consecutive pixels of one plane.
template <int KI>
__global__ void __launch_bounds__(256, KI == 2 ? 3 : 2) soft_p_kernel(const float *__restrict__ X, long long n, long long npi,
                                                     int D, const float *__restrict__ C, int k, float tau,
                                                     float *__restrict__ P)
{
    constexpr int PPTK = SoftTile<KI>::PPT, PTK = SoftTile<KI>::PT;
    extern __shared__ __align__(16) float sm[];
    float (*xs)[DCH + 1] = reinterpret_cast<float (*)[DCH + 1]>(sm);
    float (*cs)[DCH + 1] = reinterpret_cast<float (*)[DCH + 1]>(sm + PTK * (DCH + 1));
    float *ps = sm + (PTK + 16 * KI) * (DCH + 1);             // [k][PTK + 1]
    const long long p0 = (long long)blockIdx.x * PTK;
    float pr[PPTK][KI];
    tile_softmax<KI>(X, n, p0, D, C, k, tau, xs, cs, pr);
    const int pg = threadIdx.x >> 4, cl = threadIdx.x & 15;
#pragma unroll
    for (int r = 0; r < PPTK; ++r)
#pragma unroll
        for (int i = 0; i < KI; ++i)
            if (cl + 16 * i < k) ps[(cl + 16 * i) * (PTK + 1) + pg * PPTK + r] = pr[r][i];
    __syncthreads();
    const long long it0 = p0 / npi, of0 = p0 - it0 * npi;
    for (int e = threadIdx.x; e < k * PTK; e += blockDim.x) {
        const int j = e / PTK, pp = e % PTK;
        if (p0 + pp < n) P[planar_index(it0, of0, pp, j, k, npi)] = ps[j * (PTK + 1) + pp];
    }
}

constexpr int SEG = 8;             // consecutive outputs per thread in the box passes

// Row sums of width w: RW[row][x] = sum_{dx < w} P[row][x + dx], x <= W - w.  A block of 128
// threads covers RBX = 128 SEG outputs of one row: the inputs it needs are staged in shared
// memory with coalesced loads, thread t forms outputs SEG t .. SEG t + SEG - 1 (the first summed
// directly, the next ones by sliding it), and the outputs leave through shared memory as
// coalesced stores.  The shared arrays are skewed by one word per 32 so that the threads'
// stride-SEG reads fall in distinct banks.
constexpr int RBX = 128 * SEG;
__device__ __forceinline__ int skew32(int i) { return i + (i >> 5); }
__host__ __device__ constexpr size_t row_box_smem(int w) { return sizeof(float) * ((RBX + w + (RBX + w) / 32 + 1) + (RBX + RBX / 32 + 1)); }
__global__ void __launch_bounds__(128) row_box_kernel(const float *__restrict__ P, int W, int w, float *__restrict__ RW)
{
    extern __shared__ float rb[];
    const long long row = blockIdx.x;                          // rows in grid.x (> 65535 of them)
    const int x0 = blockIdx.y * RBX, xm = W - w;
    if (x0 > xm) return;                                       // uniform over the block
    const int nout = min(RBX, xm - x0 + 1), nin = nout + w - 1;  // inputs x0 .. x0 + nin - 1 <= W - 1
    float *ins = rb, *outs = rb + (RBX + w + (RBX + w) / 32 + 1);
    const float *src = P + row * W + x0;
    for (int i = threadIdx.x; i < nin; i += blockDim.x) ins[skew32(i)] = src[i];
    __syncthreads();
    const int o0 = SEG * threadIdx.x;
    if (o0 < nout) {
        float s = 0.f;
        for (int dx = 0; dx < w; ++dx) s += ins[skew32(o0 + dx)];
        outs[skew32(o0)] = s;
        const int oe = min(o0 + SEG, nout);
        for (int o = o0 + 1; o < oe; ++o) {
            s += ins[skew32(o + w - 1)] - ins[skew32(o - 1)];
            outs[skew32(o)] = s;
        }
    }
    __syncthreads();
    float *dst = RW + row * W + x0;
    for (int i = threadIdx.x; i < nout; i += blockDim.x) dst[i] = outs[skew32(i)];
}

// Column sums of height h: BX[plane][y][x] = sum_{dy < h} RW[plane][y + dy][x], y <= H - h,
// x <= wlim; thread: SEG consecutive y.
__global__ void col_box_kernel(const float *__restrict__ RW, int H, int W, int h, int wlim,
                               float *__restrict__ BX)
{
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int y0 = blockIdx.y * SEG;
    const long long plane = blockIdx.z;
    if (x > wlim || y0 > H - h) return;
    const float *src = RW + plane * H * W + x;
    float s = 0.f;
    for (int dy = 0; dy < h; ++dy) s += src[(size_t)(y0 + dy) * W];
    const int ye = min(y0 + SEG, H - h + 1);
    BX[(plane * H + y0) * W + x] = s;
    for (int y = y0 + 1; y < ye; ++y) {
        s += src[(size_t)(y + h - 1) * W] - src[(size_t)(y - 1) * W];
        BX[(plane * H + y) * W + x] = s;
    }
}

// Template soft counts: T[f * k + j] = sum over cell f of Pt[j][v] (one block per (f, j)).
__global__ void cell_sum_kernel(const float *__restrict__ Pt, int th, int tw, int k, SoftGrid sg,
                                float *__restrict__ T)
{
    const int f = blockIdx.x / k, j = blockIdx.x % k;
    const SoftCell c = sg.cell[f];
    float s = 0.f;
    const int cw = c.x1 - c.x0, n = (c.y1 - c.y0) * cw;
    for (int e = threadIdx.x; e < n; e += blockDim.x) {
        const int y = c.y0 + e / cw, x = c.x0 + e % cw;
        s += Pt[(size_t)j * th * tw + (size_t)y * tw + x];
    }
    __shared__ float red[32];
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        float t = 0.f;
        for (int q = 0; q < (int)(blockDim.x >> 5); ++q) t += red[q];
        T[f * k + j] = t;
    }
}

// Heatmap: one thread per window; L1[(b * F + f) * HO * WO + y * WO + x] kept for dL/dw.
__global__ void __launch_bounds__(128) soft_heat_kernel(const float *__restrict__ BX, int H, int W, int k,
                                                        int HO, int WO, SoftGrid sg, const float *__restrict__ T,
                                                        const float *__restrict__ wf, float *__restrict__ L1,
                                                        float *__restrict__ heat)
{
    extern __shared__ float ts[];                             // [F][k]
    const int F = sg.F;
    for (int e = threadIdx.x; e < F * k; e += blockDim.x) ts[e] = T[e];
    __syncthreads();
    const int x = blockIdx.x * blockDim.x + threadIdx.x, y = blockIdx.y, b = blockIdx.z;
    if (x >= WO) return;
    float h = 0.f;
    for (int f = 0; f < F; ++f) {
        const SoftCell c = sg.cell[f];
        const float *bx = BX + ((size_t)(b * sg.ns + c.s) * k) * H * W + (size_t)(y + c.y0) * W + (x + c.x0);
        float l1 = 0.f;
        for (int j = 0; j < k; ++j) l1 += fabsf(ts[f * k + j] - bx[(size_t)j * H * W]);
        L1[((size_t)b * F + f) * HO * WO + (size_t)y * WO + x] = l1;
        h = fmaf(wf[f] / (float)((c.y1 - c.y0) * (c.x1 - c.x0)), l1, h);
    }
    heat[((size_t)b * HO + y) * WO + x] = -h;
}

// ---------------------------------------------------------------------------------- backward
// dL/dw_f = -(1/A_f) sum_{b,y,x} dheat L1_f   (64 blocks per filter, float atomics)
__global__ void soft_dw_kernel(const float *__restrict__ dheat, const float *__restrict__ L1, int B, int HO,
                               int WO, SoftGrid sg, float *__restrict__ dwf)
{
    const int f = blockIdx.x, F = sg.F;
    const long long per = (long long)HO * WO;
    float s = 0.f;
    for (long long e = (long long)blockIdx.y * blockDim.x + threadIdx.x; e < (long long)B * per;
         e += (long long)gridDim.y * blockDim.x) {
        const long long b = e / per, r = e % per;
        s = fmaf(dheat[e], L1[((size_t)b * F + f) * per + r], s);
    }
    __shared__ float red[32];
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        float t = 0.f;
        for (int q = 0; q < (int)(blockDim.x >> 5); ++q) t += red[q];
        const SoftCell c = sg.cell[f];
        atomicAdd(&dwf[f], -t / (float)((c.y1 - c.y0) * (c.x1 - c.x0)));
    }
}

// Size class s (cells of height h, width w), one block per (item b, J consecutive planes j,
// GR consecutive rows y' <= H - h):
//   Z_j[x'] = sum over cells f of class s with window (y' - y0_f, x' - x0_f) valid of
//             m_fj = -(w_f / A_f) dheat sign(Q_fj - T_fj), Q_fj(window) = BX_j[y'][x'], x' <= W - w,
// kept in shared memory (rows skewed by one word per 32, so that the threads' stride-SG reads
// fall in distinct banks), then the row pass of the adjoint box sum
//   R2_j[y'][ux] = sum over x' in [ux - w + 1, ux] within [0, W - w] of Z_j[x']
// by sliding sums over segments of SG outputs per thread.  The window weights
// -(w_f / A_f) dheat do not depend on j: each thread loads them once per pixel and applies them
// to its J planes.  Also dT_fj += -m_fj
// (block sums, then one atomic per block, filter and plane).  The class's cells (at most G * G)
// are staged in shared memory first, so the per-pixel loop has uniform guards.
constexpr int GR = 2;              // rows per block of the gradient gather
constexpr int SG = 32;             // outputs per thread segment of its row pass
__host__ __device__ constexpr int gather_pitch(int W) { return W + W / 32 + 1; }   // skewed row
template <int MC, int J>           // MC >= number of cells in class s; J planes per block
__global__ void __launch_bounds__(256, MC <= 4 ? 2 : 1) soft_gather_kernel(const float *__restrict__ BX, const float *__restrict__ dheat,
                                                          const float *__restrict__ T, const float *__restrict__ wf,
                                                          int H, int W, int k, int HO, int WO, SoftGrid sg, int s,
                                                          float *__restrict__ R2, float *__restrict__ dT)
{
    extern __shared__ float zrow[];                           // [J][GR][WS]: Z (skewed rows)
    __shared__ int c_y0[MC], c_x0[MC], c_f[MC];
    __shared__ float c_t[MC][J], c_coef[MC];
    __shared__ int n_cell;
    __shared__ float red[MC * J][8];
    const int h = sg.hgt[sg.size_h[s]], w = sg.wid[sg.size_w[s]];
    const int nrow = H - h + 1, nrb = (nrow + GR - 1) / GR, njg = (k + J - 1) / J;
    const int rb = (int)(blockIdx.x % nrb), jg = (int)((blockIdx.x / nrb) % njg), b = (int)(blockIdx.x / nrb / njg);
    const int yb = rb * GR, j0 = jg * J, nj = min(J, k - j0);
    if (threadIdx.x == 0) {
        int n = 0;
        for (int f = 0; f < sg.F && n < MC; ++f) {
            const SoftCell c = sg.cell[f];
            if (c.s != s) continue;
            c_y0[n] = c.y0;
            c_x0[n] = c.x0;
            c_f[n] = f;
            for (int jj = 0; jj < J; ++jj) c_t[n][jj] = jj < nj ? T[f * k + j0 + jj] : 0.f;
            c_coef[n] = -(wf[f] / (float)((c.y1 - c.y0) * (c.x1 - c.x0)));
            ++n;
        }
        n_cell = n;
    }
    __syncthreads();
    const int nc = n_cell;
    float dt[MC][J];
#pragma unroll
    for (int c = 0; c < MC; ++c)
#pragma unroll
        for (int jj = 0; jj < J; ++jj) dt[c][jj] = 0.f;
    const int xm = W - w, WS = gather_pitch(W);
    const int nr = min(GR, nrow - yb);
    const size_t plane = (size_t)H * W;
    const float *bxp = BX + ((size_t)(b * sg.ns + s) * k + j0) * plane + (size_t)yb * W;
    // per row: the planes' row pointers, and per cell a dheat row pointer with the valid x
    // range [xlo, xhi) of its windows; loads outside that range are clamped into the row (and
    // their value dropped), so every address formed stays inside the buffers
#pragma unroll
    for (int r = 0; r < GR; ++r) {
        if (r >= nr) break;                                   // uniform
        const int y = yb + r;
        const float *bq[J];
#pragma unroll
        for (int jj = 0; jj < J; ++jj) bq[jj] = bxp + (size_t)(jj < nj ? jj : 0) * plane + (size_t)r * W;
        const float *dp[MC];
        int xlo[MC], xhi[MC];
#pragma unroll
        for (int c = 0; c < MC; ++c) {
            const int wy = c < nc ? y - c_y0[c] : -1;
            const bool rowok = wy >= 0 && wy < HO;
            const int x0c = c < nc ? c_x0[c] : 0;
            dp[c] = dheat + ((size_t)b * HO + (rowok ? wy : 0)) * WO;
            xlo[c] = rowok ? x0c : 1 << 30;
            xhi[c] = rowok ? x0c + WO : 0;
        }
        float *zr = zrow + r * WS;
        for (int x = threadIdx.x; x <= xm; x += blockDim.x) {
            float q[J];
#pragma unroll
            for (int jj = 0; jj < J; ++jj) q[jj] = jj < nj ? bq[jj][x] : 0.f;
            float mc[MC];
#pragma unroll
            for (int c = 0; c < MC; ++c) {
                const bool ok = x >= xlo[c] && x < xhi[c];
                const float d = dp[c][ok ? x - xlo[c] : 0];
                mc[c] = ok ? c_coef[c] * d : 0.f;
            }
            const int sx = skew32(x);
#pragma unroll
            for (int jj = 0; jj < J; ++jj) {
                float z = 0.f;
#pragma unroll
                for (int c = 0; c < MC; ++c) {
                    if (c >= nc) break;                       // uniform
                    const float t = c_t[c][jj];
                    const float m = q[jj] > t ? mc[c] : (q[jj] < t ? -mc[c] : 0.f);
                    z += m;
                    dt[c][jj] -= m;
                }
                zr[jj * GR * WS + sx] = z;
            }
        }
    }
    __syncthreads();
    // row pass: thread segments of SG consecutive outputs, the first summed directly and the
    // next ones by sliding it; the outputs leave from registers as 16-byte stores.  Segments
    // whose adds and subtractions all fall inside [0, W - w] take an unguarded loop.
    const int lane = threadIdx.x & 31, wp = threadIdx.x >> 5;
    const int nseg = (W + SG - 1) / SG;
    const bool vec = (W & 3) == 0;
    for (int e = threadIdx.x; e < nj * GR * nseg; e += blockDim.x) {
        const int rr = e / nseg, u0 = (e - rr * nseg) * SG;
        const int jj = rr / GR, r = rr % GR;
        if (r >= nr) continue;
        const float *zr = zrow + rr * WS;
        const int n = min(SG, W - u0);
        float o[SG];
        float acc = 0.f;
        for (int x = max(0, u0 - w + 1); x <= min(u0, xm); ++x) acc += zr[skew32(x)];
        o[0] = acc;
        if (n == SG && u0 + SG - 1 <= xm && u0 + 1 - w >= 0) {
#pragma unroll
            for (int i = 1; i < SG; ++i) {
                acc += zr[skew32(u0 + i)];
                acc -= zr[skew32(u0 + i - w)];
                o[i] = acc;
            }
        } else {
#pragma unroll
            for (int i = 1; i < SG; ++i) {
                const int ux = u0 + i;
                if (i < n) {
                    if (ux <= xm) acc += zr[skew32(ux)];
                    if (ux - w >= 0) acc -= zr[skew32(ux - w)];
                }
                o[i] = acc;
            }
        }
        float *out = R2 + (((size_t)b * k + j0 + jj) * H + yb + r) * W + u0;
        if (vec && n == SG) {
#pragma unroll
            for (int i = 0; i < SG; i += 4)
                *reinterpret_cast<float4 *>(out + i) = make_float4(o[i], o[i + 1], o[i + 2], o[i + 3]);
        } else {
#pragma unroll
            for (int i = 0; i < SG; ++i)
                if (i < n) out[i] = o[i];
        }
    }
    if constexpr (MC * J <= 32) {
        // the warp's sums of all MC J values at once: a reduce-scatter over the lanes (31
        // exchanges), after which lane l holds the warp's sum of value l = c J + jj
        float v[32];
#pragma unroll
        for (int i = 0; i < 32; ++i) v[i] = i < MC * J ? dt[i / J][i % J] : 0.f;
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
        if (lane < MC * J) red[lane][wp] = v[0];
    } else {
#pragma unroll
        for (int c = 0; c < MC; ++c) {
            if (c >= nc) break;                               // uniform
#pragma unroll
            for (int jj = 0; jj < J; ++jj) {
                float v = dt[c][jj];
                for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
                if (lane == 0) red[c * J + jj][wp] = v;
            }
        }
    }
    __syncthreads();
    if ((int)threadIdx.x < nc * J) {
        const int c = threadIdx.x / J, jj = threadIdx.x % J;
        float v = 0.f;
        for (int q = 0; q < (int)(blockDim.x >> 5); ++q) v += red[c * J + jj][q];
        if (jj < nj && v != 0.f) atomicAdd(&dT[c_f[c] * k + j0 + jj], v);
    }
}

// G[plane][uy][ux] = sum over size classes s of the sum over y' in [uy - h_s + 1, uy] within
// [0, H - h_s] of R2_s[plane][y'][ux] (the column pass of every class's adjoint box sum, so G is
// written once); thread: SEG consecutive uy, one sliding window per class.
struct AdjCols {
    int ns;
    int h[4];
};
__global__ void adj_col_kernel(const float *__restrict__ R2, long long cls_stride, int H, int W, AdjCols ac,
                               float *__restrict__ Gp)
{
    const int ux = blockIdx.x * blockDim.x + threadIdx.x, v0 = blockIdx.y * SEG;
    const long long plane = blockIdx.z;
    if (ux >= W || v0 >= H) return;
    const int ve = min(v0 + SEG, H);
    float out[SEG];
#pragma unroll
    for (int i = 0; i < SEG; ++i) out[i] = 0.f;
    for (int is = 0; is < ac.ns; ++is) {
        const float *src = R2 + is * cls_stride + plane * H * W + ux;
        const int h = ac.h[is], ym = H - h;
        float s = 0.f;
        for (int yp = max(0, v0 - h + 1); yp <= min(v0, ym); ++yp) s += src[(size_t)yp * W];
        out[0] += s;
#pragma unroll
        for (int i = 1; i < SEG; ++i) {
            const int uy = v0 + i;
            if (uy < ve) {
                if (uy <= ym) s += src[(size_t)uy * W];
                if (uy - h >= 0 && uy - h <= ym) s -= src[(size_t)(uy - h) * W];
            }
            out[i] += s;
        }
    }
#pragma unroll
    for (int i = 0; i < SEG; ++i)
        if (v0 + i < ve) Gp[(plane * H + v0 + i) * W + ux] = out[i];
}

// Template pixel gradients: Gt[j][v] = sum over cells f containing v of dT_fj.
__global__ void tmpl_grad_kernel(const float *__restrict__ dT, int th, int tw, int k, SoftGrid sg,
                                 float *__restrict__ Gt)
{
    const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= (long long)k * th * tw) return;
    const int j = (int)(e / ((long long)th * tw)), v = (int)(e % ((long long)th * tw));
    const int y = v / tw, x = v % tw;
    float s = 0.f;
    for (int f = 0; f < sg.F; ++f) {
        const SoftCell c = sg.cell[f];
        if (y >= c.y0 && y < c.y1 && x >= c.x0 && x < c.x1) s += dT[f * k + j];
    }
    Gt[e] = s;
}

// Softmax backward from the forward's soft assignment P (planar, as soft_p_kernel wrote it):
// a_j = -(1/tau) p_j (g_j - sum_i p_i g_i), A pixel-major; dX = 2 (sum_j a_j) x - 2 sum_j a_j c_j
// (skipped when dX is null).
template <int KI>
__global__ void __launch_bounds__(256) soft_back_kernel(const float *__restrict__ X, long long n, long long npi,
                                                        int D, const float *__restrict__ C, int k, float tau,
                                                        const float *__restrict__ P, const float *__restrict__ Gp,
                                                        float *__restrict__ A, float *__restrict__ dX)
{
    extern __shared__ __align__(16) float sm[];
    float (*xs)[DCH + 1] = reinterpret_cast<float (*)[DCH + 1]>(sm);
    float (*cs)[DCH + 1] = reinterpret_cast<float (*)[DCH + 1]>(sm + PT * (DCH + 1));
    float *as = sm + (PT + 16 * KI) * (DCH + 1);             // [PT][k + 1]: g, then a
    float *asum_s = as + PT * (16 * KI + 1);                  // [PT]
    float *ps = asum_s + PT + 16 * KI * (PT + 4);             // [PT][k + 1]: p
    const long long p0 = (long long)blockIdx.x * PT;
    const int t = threadIdx.x, pg = t >> 4, cl = t & 15;
    // p and g of the tile's pixels, coalesced along pixels of each plane
    const long long it0 = p0 / npi, of0 = p0 - it0 * npi;
    for (int e = t; e < k * PT; e += blockDim.x) {
        const int j = e / PT, pp = e % PT;
        const bool in = p0 + pp < n;
        const long long o = in ? planar_index(it0, of0, pp, j, k, npi) : 0;
        as[pp * (k + 1) + j] = in ? Gp[o] : 0.f;
        ps[pp * (k + 1) + j] = in ? P[o] : 0.f;
    }
    __syncthreads();
    float pr[PPT][KI];
#pragma unroll
    for (int r = 0; r < PPT; ++r)
#pragma unroll
        for (int i = 0; i < KI; ++i)
            pr[r][i] = cl + 16 * i < k ? ps[(pg * PPT + r) * (k + 1) + cl + 16 * i] : 0.f;
    const float it = 1.0f / tau;
#pragma unroll
    for (int r = 0; r < PPT; ++r) {
        const int pp = pg * PPT + r;
        float gv[KI], s = 0.f;
#pragma unroll
        for (int i = 0; i < KI; ++i) {
            gv[i] = cl + 16 * i < k ? as[pp * (k + 1) + cl + 16 * i] : 0.f;
            s = fmaf(pr[r][i], gv[i], s);
        }
#pragma unroll
        for (int o = 1; o < 16; o <<= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
        float asum = 0.f;
        __syncwarp();
#pragma unroll
        for (int i = 0; i < KI; ++i)
            if (cl + 16 * i < k) {
                const float a = -it * pr[r][i] * (gv[i] - s);
                as[pp * (k + 1) + cl + 16 * i] = a;
                asum += a;
            }
#pragma unroll
        for (int o = 1; o < 16; o <<= 1) asum += __shfl_xor_sync(0xffffffffu, asum, o);
        if (cl == 0) asum_s[pp] = asum;
    }
    __syncthreads();
    for (int e = t; e < PT * k; e += blockDim.x) {
        const int pp = e / k, j = e % k;
        const long long g = p0 + pp;
        if (g < n) A[g * k + j] = as[pp * (k + 1) + j];
    }
    if (!dX) return;                                          // uniform over the block
    // a transposed, at[j][PT + 4], for float4 reads along pixels (rows 16-byte aligned)
    float *at = asum_s + PT;
    for (int e = t; e < k * PT; e += blockDim.x) {
        const int j = e / PT, pp = e % PT;
        at[j * (PT + 4) + pp] = as[pp * (k + 1) + j];
    }
    // dX tile per chunk: thread owns pixels 4 pq .. 4 pq + 3 and dims 2 dg, 2 dg + 1 of the chunk;
    // the chunk's centroid columns are restaged unpadded, cs2[j][DCH], for float2 reads
    float *cs2 = &cs[0][0];
    const int pq = t >> 4, dg = t & 15;
    for (int d0 = 0; d0 < D; d0 += DCH) {
        __syncthreads();
        for (int e = t; e < PT * DCH; e += blockDim.x) {
            const int pp = e / DCH, dd = e % DCH;
            const long long gg = p0 + pp;
            xs[pp][dd] = (gg < n && d0 + dd < D) ? X[gg * D + d0 + dd] : 0.f;
        }
        for (int e = t; e < k * DCH; e += blockDim.x) {
            const int j = e / DCH, dd = e % DCH;
            cs2[e] = d0 + dd < D ? C[(size_t)j * D + d0 + dd] : 0.f;
        }
        __syncthreads();
        float ac[4][2] = {{0.f, 0.f}, {0.f, 0.f}, {0.f, 0.f}, {0.f, 0.f}};
#pragma unroll 4
        for (int j = 0; j < k; ++j) {
            const float4 a4 = *reinterpret_cast<const float4 *>(at + j * (PT + 4) + 4 * pq);
            const float2 c2 = *reinterpret_cast<const float2 *>(cs2 + j * DCH + 2 * dg);
            ac[0][0] = fmaf(a4.x, c2.x, ac[0][0]);
            ac[0][1] = fmaf(a4.x, c2.y, ac[0][1]);
            ac[1][0] = fmaf(a4.y, c2.x, ac[1][0]);
            ac[1][1] = fmaf(a4.y, c2.y, ac[1][1]);
            ac[2][0] = fmaf(a4.z, c2.x, ac[2][0]);
            ac[2][1] = fmaf(a4.z, c2.y, ac[2][1]);
            ac[3][0] = fmaf(a4.w, c2.x, ac[3][0]);
            ac[3][1] = fmaf(a4.w, c2.y, ac[3][1]);
        }
#pragma unroll
        for (int r = 0; r < 4; ++r) {
            const int pp = 4 * pq + r;
            const long long g = p0 + pp;
#pragma unroll
            for (int c = 0; c < 2; ++c) {
                const int d = d0 + 2 * dg + c;
                if (g < n && d < D) dX[g * D + d] = 2.0f * (asum_s[pp] * xs[pp][2 * dg + c] - ac[r][c]);
            }
        }
    }
}

// Partial centroid gradients over a pixel slice, one output tile of 64 centroids x 64 dims per
// block (thread: 4 centroids x 4 dims in registers, float4 shared-memory reads):
// part[slice][j D + d] = sum_u a_j(u) x_u[d]; the j-tile's first d-tile also writes
// part[slice][k D + j] = sum_u a_j(u).
constexpr int DCU = 32;            // pixels staged per step of the centroid-gradient reduction
__global__ void __launch_bounds__(256) dc_partial_kernel(const float *__restrict__ A, const float *__restrict__ X,
                                                         long long n, int D, int k, int nslice,
                                                         float *__restrict__ part)
{
    __shared__ __align__(16) float at[DCU][64 + 4];
    __shared__ __align__(16) float xt[DCU][64 + 4];
    const int t = threadIdx.x, ty = t >> 4, tx = t & 15;        // centroids 4 ty.., dims 4 tx..
    const int j0 = blockIdx.x * 64, d0 = blockIdx.y * 64;
    const int slice = blockIdx.z;
    const long long per = (n + nslice - 1) / nslice;
    const long long u0 = (long long)slice * per, u1 = min(n, u0 + per);
    float acc[4][4] = {};
    float asum[4] = {0.f, 0.f, 0.f, 0.f};
    for (long long t0 = u0; t0 < u1; t0 += DCU) {
        const int m = (int)min((long long)DCU, u1 - t0);
        __syncthreads();
        for (int e = t; e < DCU * 64; e += blockDim.x) {
            const int uu = e >> 6, jj = e & 63;
            at[uu][jj] = (uu < m && j0 + jj < k) ? A[(t0 + uu) * k + j0 + jj] : 0.f;
        }
        for (int e = t; e < DCU * 64; e += blockDim.x) {
            const int uu = e >> 6, dd = e & 63;
            xt[uu][dd] = (uu < m && d0 + dd < D) ? X[(t0 + uu) * D + d0 + dd] : 0.f;
        }
        __syncthreads();
#pragma unroll 4
        for (int uu = 0; uu < DCU; ++uu) {
            const float4 a4 = *reinterpret_cast<const float4 *>(&at[uu][4 * ty]);
            const float4 x4 = *reinterpret_cast<const float4 *>(&xt[uu][4 * tx]);
            const float av[4] = {a4.x, a4.y, a4.z, a4.w}, xv[4] = {x4.x, x4.y, x4.z, x4.w};
#pragma unroll
            for (int r = 0; r < 4; ++r) {
                asum[r] += av[r];
#pragma unroll
                for (int c = 0; c < 4; ++c) acc[r][c] = fmaf(av[r], xv[c], acc[r][c]);
            }
        }
    }
    float *o = part + (size_t)slice * ((size_t)k * D + k);
#pragma unroll
    for (int r = 0; r < 4; ++r) {
        const int j = j0 + 4 * ty + r;
        if (j >= k) continue;
#pragma unroll
        for (int c = 0; c < 4; ++c) {
            const int d = d0 + 4 * tx + c;
            if (d < D) o[(size_t)j * D + d] = acc[r][c];
        }
        if (blockIdx.y == 0 && tx == 0) o[(size_t)k * D + j] = asum[r];
    }
}

// dC[j][d] = -2 sum_slices part[.][j D + d] + 2 (sum_slices part[.][k D + j]) C[j][d], over the
// query slices and then the template slices (fixed order).
__global__ void dc_reduce_kernel(const float *__restrict__ part, int nslice, int D, int k,
                                 const float *__restrict__ C, float *__restrict__ dC)
{
    const int o = blockIdx.x * blockDim.x + threadIdx.x;
    const int kD = k * D;
    if (o >= kD) return;
    const int j = o / D;
    float s = 0.f, a = 0.f;
    for (int q = 0; q < nslice; ++q) {
        s += part[(size_t)q * (kD + k) + o];
        a += part[(size_t)q * (kD + k) + kD + j];
    }
    dC[o] = 2.0f * (a * C[o] - s);
}

template <int KI>
cudaError_t launch_soft_p_ki(const float *X, long long n, long long npi, int D, const float *C, int k, float tau,
                             float *P, cudaStream_t s)
{
    constexpr int PTK = SoftTile<KI>::PT;
    const size_t sm = sizeof(float) * ((PTK + 16 * KI) * (DCH + 1) + 16 * KI * (PTK + 1));
    cudaError_t e = cudaFuncSetAttribute(soft_p_kernel<KI>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (e != cudaSuccess) return e;
    soft_p_kernel<KI><<<(unsigned)((n + PTK - 1) / PTK), 256, sm, s>>>(X, n, npi, D, C, k, tau, P);
    return cudaGetLastError();
}

cudaError_t launch_soft_p(const float *X, long long n, long long npi, int D, const float *C, int k, float tau,
                          float *P, cudaStream_t s)
{
    if (k <= 32) return launch_soft_p_ki<2>(X, n, npi, D, C, k, tau, P, s);
    if (k <= 64) return launch_soft_p_ki<4>(X, n, npi, D, C, k, tau, P, s);
    return launch_soft_p_ki<8>(X, n, npi, D, C, k, tau, P, s);
}

template <int KI>
cudaError_t launch_soft_back_ki(const float *X, long long n, long long npi, int D, const float *C, int k,
                                float tau, const float *P, const float *Gp, float *A, float *dX, cudaStream_t s)
{
    const size_t sm = sizeof(float) * ((PT + 16 * KI) * (DCH + 1) + 2 * PT * (16 * KI + 1) + PT + 16 * KI * (PT + 4));
    cudaError_t e = cudaFuncSetAttribute(soft_back_kernel<KI>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (e != cudaSuccess) return e;
    soft_back_kernel<KI><<<(unsigned)((n + PT - 1) / PT), 256, sm, s>>>(X, n, npi, D, C, k, tau, P, Gp, A, dX);
    return cudaGetLastError();
}

cudaError_t launch_soft_back(const float *X, long long n, long long npi, int D, const float *C, int k, float tau,
                             const float *P, const float *Gp, float *A, float *dX, cudaStream_t s)
{
    if (k <= 32) return launch_soft_back_ki<2>(X, n, npi, D, C, k, tau, P, Gp, A, dX, s);
    if (k <= 64) return launch_soft_back_ki<4>(X, n, npi, D, C, k, tau, P, Gp, A, dX, s);
    return launch_soft_back_ki<8>(X, n, npi, D, C, k, tau, P, Gp, A, dX, s);
}

template <int MC, int J>
cudaError_t launch_gather_j(const SoftWs &w, const float *dheat, const float *wf, int B, int H, int W, int k, int HO,
                            int WO, const SoftGrid &sg, int is, cudaStream_t s)
{
    const int h = sg.hgt[sg.size_h[is]];
    const size_t zs = sizeof(float) * J * GR * gather_pitch(W);   // up to ~198 KB
    cudaError_t e = cudaFuncSetAttribute(soft_gather_kernel<MC, J>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)zs);
    if (e != cudaSuccess) return e;
    const long long nblk = (long long)B * ((k + J - 1) / J) * ((H - h + GR) / GR);
    soft_gather_kernel<MC, J><<<(unsigned)nblk, 256, zs, s>>>(w.BX, dheat, w.T, wf, H, W, k, HO, WO, sg, is,
                                                              w.R2 + (size_t)is * B * k * H * W,
                                                              w.dT);
    return cudaGetLastError();
}

// Planes per block: the register budget (MC x J accumulators) and shared memory (J GR W floats).
template <int MC, int JMAX>
cudaError_t launch_gather(const SoftWs &w, const float *dheat, const float *wf, int B, int H, int W, int k, int HO,
                          int WO, const SoftGrid &sg, int is, cudaStream_t s)
{
    const long long room = 200704 / ((long long)sizeof(float) * GR * gather_pitch(W));   // planes that fit
    if constexpr (JMAX >= 8)
        if (room >= 8) return launch_gather_j<MC, 8>(w, dheat, wf, B, H, W, k, HO, WO, sg, is, s);
    if constexpr (JMAX >= 4)
        if (room >= 4) return launch_gather_j<MC, 4>(w, dheat, wf, B, H, W, k, HO, WO, sg, is, s);
    return launch_gather_j<MC, 2>(w, dheat, wf, B, H, W, k, HO, WO, sg, is, s);
}

}  // namespace

bool soft_grid(int th, int tw, int G, SoftGrid &sg)
{
    if (G < 1 || G > kSoftMaxG || th < G || tw < G) return false;
    sg = SoftGrid{};
    sg.G = G;
    sg.F = G * G;
    int bx[kSoftMaxG + 1], by[kSoftMaxG + 1];
    for (int i = 0; i <= G; ++i) {
        bx[i] = (i * tw) / G;
        by[i] = (i * th) / G;
    }
    auto index_of = [](int *arr, int &n, int v) {
        for (int q = 0; q < n; ++q)
            if (arr[q] == v) return q;
        arr[n] = v;
        return n++;
    };
    for (int r = 0; r < G; ++r)
        for (int c = 0; c < G; ++c) {
            SoftCell &cl = sg.cell[r * G + c];
            cl.y0 = by[r]; cl.y1 = by[r + 1]; cl.x0 = bx[c]; cl.x1 = bx[c + 1];
            const int iw = index_of(sg.wid, sg.nw, cl.x1 - cl.x0);
            const int ih = index_of(sg.hgt, sg.nh, cl.y1 - cl.y0);
            int s = 0;
            while (s < sg.ns && !(sg.size_w[s] == iw && sg.size_h[s] == ih)) ++s;
            if (s == sg.ns) {
                sg.size_w[s] = iw;
                sg.size_h[s] = ih;
                ++sg.ns;
            }
            cl.s = s;
        }
    return true;
}

size_t soft_workspace_bytes(int B, int H, int W, int D, int k, int th, int tw, const SoftGrid &sg)
{
    WsCursor c{nullptr, 0};
    carve_soft(c, B, H, W, D, k, th, tw, sg);
    return c.off + 256;
}

SoftWs carve_soft(WsCursor &c, int B, int H, int W, int D, int k, int th, int tw, const SoftGrid &sg)
{
    SoftWs w;
    const size_t plane = (size_t)H * W;
    w.P = c.take<float>((size_t)B * k * plane);
    w.RW = c.take<float>((size_t)B * sg.nw * k * plane);
    w.BX = c.take<float>((size_t)B * sg.ns * k * plane);
    w.Pt = c.take<float>((size_t)k * th * tw);
    w.T = c.take<float>((size_t)sg.F * k);
    w.L1 = c.take<float>((size_t)B * sg.F * (H - th + 1) * (W - tw + 1));
    w.R2 = c.take<float>((size_t)sg.ns * B * k * plane);    // one area per size class
    w.G = c.take<float>((size_t)B * k * plane);
    w.A = c.take<float>((size_t)B * k * plane);
    w.At = c.take<float>((size_t)k * th * tw);
    w.dT = c.take<float>((size_t)sg.F * k);
    w.part = c.take<float>((size_t)2 * kSoftSlices * ((size_t)k * D + k));
    w.ct = c.take<uint8_t>(soft_ct_image_bytes(D));
    return w;
}

cudaError_t soft_forward(const float *Qf, int B, int H, int W, const float *Tf, int th, int tw, int D,
                         const float *C, int k, float tau, const SoftGrid &sg, const float *wf, float *heat,
                         SoftWs &w, cudaStream_t s)
{
    const long long nq = (long long)B * H * W, nt = (long long)th * tw;
    cudaError_t e = launch_soft_p(Qf, nq, (long long)H * W, D, C, k, tau, w.P, s);
    if (e != cudaSuccess) return e;
    e = launch_soft_p(Tf, nt, nt, D, C, k, tau, w.Pt, s);
    if (e != cudaSuccess) return e;
    const long long planes = (long long)B * k;
    for (int iw = 0; iw < sg.nw; ++iw) {
        const int wd = sg.wid[iw];
        const size_t rs = row_box_smem(wd);                   // up to ~56 KB (W <= 12288)
        e = cudaFuncSetAttribute(row_box_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)rs);
        if (e != cudaSuccess) return e;
        dim3 g((unsigned)(planes * H), (W - wd + RBX) / RBX);
        row_box_kernel<<<g, 128, rs, s>>>(w.P, W, wd, w.RW + (size_t)iw * planes * H * W);
    }
    for (int is = 0; is < sg.ns; ++is) {
        const int iw = sg.size_w[is];
        for (int b = 0; b < B; ++b) {
            dim3 g((W + 127) / 128, (H + SEG - 1) / SEG, k);
            col_box_kernel<<<g, 128, 0, s>>>(w.RW + ((size_t)iw * planes + (size_t)b * k) * H * W, H, W,
                                             sg.hgt[sg.size_h[is]], W - sg.wid[iw],
                                             w.BX + ((size_t)b * sg.ns + is) * k * H * W);
        }
    }
    cell_sum_kernel<<<sg.F * k, 128, 0, s>>>(w.Pt, th, tw, k, sg, w.T);
    const int HO = H - th + 1, WO = W - tw + 1;
    dim3 g((WO + 127) / 128, HO, B);
    soft_heat_kernel<<<g, 128, sizeof(float) * sg.F * k, s>>>(w.BX, H, W, k, HO, WO, sg, w.T, wf, w.L1, heat);
    return cudaGetLastError();
}

cudaError_t soft_backward(const float *Qf, int B, int H, int W, const float *Tf, int th, int tw, int D,
                          const float *C, int k, float tau, const SoftGrid &sg, const float *wf,
                          const float *dheat, float *dQf, float *dC, float *dwf, SoftWs &w, cudaStream_t s)
{
    const int HO = H - th + 1, WO = W - tw + 1;
    const long long nq = (long long)B * H * W, nt = (long long)th * tw;
    cudaError_t e = cudaMemsetAsync(dwf, 0, sizeof(float) * sg.F, s);
    if (e != cudaSuccess) return e;
    soft_dw_kernel<<<dim3(sg.F, 64), 256, 0, s>>>(dheat, w.L1, B, HO, WO, sg, dwf);
    e = cudaMemsetAsync(w.dT, 0, sizeof(float) * sg.F * k, s);
    if (e != cudaSuccess) return e;
    const long long planes = (long long)B * k;
    AdjCols ac{sg.ns, {0, 0, 0, 0}};
    for (int is = 0; is < sg.ns; ++is) {
        const int h = sg.hgt[sg.size_h[is]];
        int ncell = 0;
        for (int f = 0; f < sg.F; ++f) ncell += sg.cell[f].s == is;
        e = ncell <= 4 ? launch_gather<4, 8>(w, dheat, wf, B, H, W, k, HO, WO, sg, is, s)
            : ncell <= 9 ? launch_gather<9, 4>(w, dheat, wf, B, H, W, k, HO, WO, sg, is, s)
                         : launch_gather<kSoftMaxG * kSoftMaxG, 2>(w, dheat, wf, B, H, W, k, HO, WO, sg, is, s);
        if (e != cudaSuccess) return e;
        ac.h[is] = h;
    }
    dim3 g3((W + 127) / 128, (H + SEG - 1) / SEG, (unsigned)planes);
    adj_col_kernel<<<g3, 128, 0, s>>>(w.R2, planes * H * W, H, W, ac, w.G);
    const size_t kDk = (size_t)k * D + k;
    if (soft_tc_supported(D, k)) {                            // tensor-core contractions
        int nqs = 0, nts = 0;
        e = launch_soft_ct_image(C, k, D, w.ct, s);
        if (e != cudaSuccess) return e;
        e = launch_soft_grad_tc(Qf, nq, (long long)H * W, D, k, tau, w.P, w.G, w.ct, dQf, w.part, kSoftSlices,
                                &nqs, s);
        if (e != cudaSuccess) return e;
        tmpl_grad_kernel<<<(unsigned)((k * nt + 255) / 256), 256, 0, s>>>(w.dT, th, tw, k, sg, w.G);
        e = launch_soft_grad_tc(Tf, nt, nt, D, k, tau, w.Pt, w.G, w.ct, nullptr, w.part + (size_t)nqs * kDk,
                                kSoftSlices, &nts, s);
        if (e != cudaSuccess) return e;
        dc_reduce_kernel<<<(k * D + 255) / 256, 256, 0, s>>>(w.part, nqs + nts, D, k, C, dC);
        return cudaGetLastError();
    }
    e = launch_soft_back(Qf, nq, (long long)H * W, D, C, k, tau, w.P, w.G, w.A, dQf, s);
    if (e != cudaSuccess) return e;
    // template side: pixel gradients from dT, then its softmax backward (no feature gradient)
    tmpl_grad_kernel<<<(unsigned)((k * nt + 255) / 256), 256, 0, s>>>(w.dT, th, tw, k, sg, w.G);
    e = launch_soft_back(Tf, nt, nt, D, C, k, tau, w.Pt, w.G, w.At, nullptr, s);
    if (e != cudaSuccess) return e;
    dim3 gp((k + 63) / 64, (D + 63) / 64, kSoftSlices);
    dc_partial_kernel<<<gp, 256, 0, s>>>(w.A, Qf, nq, D, k, kSoftSlices, w.part);
    dc_partial_kernel<<<gp, 256, 0, s>>>(w.At, Tf, nt, D, k, kSoftSlices, w.part + (size_t)kSoftSlices * (k * D + k));
    dc_reduce_kernel<<<(k * D + 255) / 256, 256, 0, s>>>(w.part, 2 * kSoftSlices, D, k, C, dC);
    return cudaGetLastError();
}

}  // namespace vqnnf
