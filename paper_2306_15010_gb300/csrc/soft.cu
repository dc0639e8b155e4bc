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
//   a_j(u)       = -(1/tau) p_j (g_j - sum_i p_i g_i)                    (softmax recomputed)
//   dL/dx_u      = 2 (sum_j a_j) x_u - 2 sum_j a_j c_j
//   dL/dc_j      = -2 sum_u a_j(u) x_u + 2 (sum_u a_j(u)) c_j   (query and template pixels)
#include <cfloat>

#include "common.cuh"
#include "soft_spec.cuh"

namespace vqnnf {
namespace {

constexpr int PT = 64;            // pixels per tile of the soft-assignment kernels
constexpr int DCH = 32;           // feature dimensions staged per chunk
constexpr int KQ = kSoftMaxK / 4; // centroids per thread (four threads per pixel)

// Distances of a 64-pixel tile to all k centroids, four threads per pixel (thread 4p + q holds
// centroids q, q + 4, ...), then the softmax over the pixel's k logits.  X rows are pixels.
__device__ __forceinline__ void tile_softmax(const float *__restrict__ X, long long n, long long p0, int D,
                                             const float *__restrict__ C, int k, float tau, float (*xs)[DCH + 1],
                                             float (*cs)[DCH + 1], float *pr)
{
    const int t = threadIdx.x, p = t >> 2, q = t & 3;
    float acc[KQ];
#pragma unroll
    for (int i = 0; i < KQ; ++i) acc[i] = 0.f;
    for (int d0 = 0; d0 < D; d0 += DCH) {
        __syncthreads();
        for (int e = t; e < PT * DCH; e += blockDim.x) {
            const int pp = e / DCH, dd = e % DCH;
            const long long g = p0 + pp;
            xs[pp][dd] = (g < n && d0 + dd < D) ? X[g * D + d0 + dd] : 0.f;
        }
        for (int e = t; e < k * DCH; e += blockDim.x) {
            const int j = e / DCH, dd = e % DCH;
            cs[j][dd] = d0 + dd < D ? C[(size_t)j * D + d0 + dd] : 0.f;
        }
        __syncthreads();
#pragma unroll 4
        for (int dd = 0; dd < DCH; ++dd) {
            const float x = xs[p][dd];
#pragma unroll
            for (int i = 0; i < KQ; ++i) {
                const int j = q + 4 * i;
                if (j < k) {
                    const float df = x - cs[j][dd];
                    acc[i] = fmaf(df, df, acc[i]);
                }
            }
        }
    }
    float dmin = FLT_MAX;
#pragma unroll
    for (int i = 0; i < KQ; ++i)
        if (q + 4 * i < k) dmin = fminf(dmin, acc[i]);
    dmin = fminf(dmin, __shfl_xor_sync(0xffffffffu, dmin, 1));
    dmin = fminf(dmin, __shfl_xor_sync(0xffffffffu, dmin, 2));
    float s = 0.f;
    const float it = 1.0f / tau;
#pragma unroll
    for (int i = 0; i < KQ; ++i) {
        const float e = q + 4 * i < k ? expf((dmin - acc[i]) * it) : 0.f;
        acc[i] = e;
        s += e;
    }
    s += __shfl_xor_sync(0xffffffffu, s, 1);
    s += __shfl_xor_sync(0xffffffffu, s, 2);
    const float inv = 1.0f / s;
#pragma unroll
    for (int i = 0; i < KQ; ++i) pr[i] = acc[i] * inv;
}

// p planar: P[(item * k + j) * npi + pixel]
__global__ void __launch_bounds__(256) soft_p_kernel(const float *__restrict__ X, long long n, long long npi,
                                                     int D, const float *__restrict__ C, int k, float tau,
                                                     float *__restrict__ P)
{
    __shared__ float xs[PT][DCH + 1];
    __shared__ float cs[kSoftMaxK][DCH + 1];
    const long long p0 = (long long)blockIdx.x * PT;
    float pr[KQ];
    tile_softmax(X, n, p0, D, C, k, tau, xs, cs, pr);
    const int p = threadIdx.x >> 2, q = threadIdx.x & 3;
    const long long g = p0 + p;
    if (g >= n) return;
    const long long item = g / npi, pix = g % npi;
#pragma unroll
    for (int i = 0; i < KQ; ++i) {
        const int j = q + 4 * i;
        if (j < k) P[(item * k + j) * npi + pix] = pr[i];
    }
}

// Row sums of width w: RW[row][x] = sum_{dx < w} P[row][x + dx], x <= W - w (one block per
// row of a plane).
__global__ void row_box_kernel(const float *__restrict__ P, int W, int w, float *__restrict__ RW)
{
    const long long row = blockIdx.x;
    const float *src = P + row * W;
    for (int x = threadIdx.x; x <= W - w; x += blockDim.x) {
        float s = 0.f;
        for (int dx = 0; dx < w; ++dx) s += src[x + dx];
        RW[row * W + x] = s;
    }
}

// Column sums of height h: BX[plane][y][x] = sum_{dy < h} RW[plane][y + dy][x], y <= H - h.
__global__ void col_box_kernel(const float *__restrict__ RW, int H, int W, int h, int wlim,
                               float *__restrict__ BX)
{
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = blockIdx.y;
    const long long plane = blockIdx.z;
    if (x > wlim || y > H - h) return;
    const float *src = RW + (plane * H + y) * W + x;
    float s = 0.f;
    for (int dy = 0; dy < h; ++dy) s += src[(size_t)dy * W];
    BX[(plane * H + y) * W + x] = s;
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
// dL/dw_f = -(1/A_f) sum_{b,y,x} dheat L1_f   (one block per filter, fixed-order tree)
__global__ void soft_dw_kernel(const float *__restrict__ dheat, const float *__restrict__ L1, int B, int HO,
                               int WO, SoftGrid sg, float *__restrict__ dwf)
{
    const int f = blockIdx.x, F = sg.F;
    const long long per = (long long)HO * WO;
    float s = 0.f;
    for (long long e = threadIdx.x; e < (long long)B * per; e += blockDim.x) {
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
        dwf[f] = -t / (float)((c.y1 - c.y0) * (c.x1 - c.x0));
    }
}

// Size class s: Z[(b k + j)][y'][x'] = sum over cells f of class s with window (y' - y0_f,
// x' - x0_f) valid of m_fj = -(w_f/A_f) dheat sign(Q_fj - T_fj); Q_fj(window) is BX at (y', x').
// Also dT_fj += -m_fj (block sums, then one atomic per block and filter).
__global__ void __launch_bounds__(128) soft_gather_kernel(const float *__restrict__ BX, const float *__restrict__ dheat,
                                                          const float *__restrict__ T, const float *__restrict__ wf,
                                                          int H, int W, int k, int HO, int WO, SoftGrid sg, int s,
                                                          float *__restrict__ Z, float *__restrict__ dT)
{
    const int x = blockIdx.x * blockDim.x + threadIdx.x, y = blockIdx.y;
    const int bj = blockIdx.z, b = bj / k, j = bj % k;
    const int h = sg.hgt[sg.size_h[s]], w = sg.wid[sg.size_w[s]];
    float dt[kSoftMaxG * kSoftMaxG];
#pragma unroll
    for (int f = 0; f < kSoftMaxG * kSoftMaxG; ++f) dt[f] = 0.f;
    const bool in = x <= W - w && y <= H - h;
    float z = 0.f;
    if (in) {
        const float q = BX[((size_t)(b * sg.ns + s) * k + j) * H * W + (size_t)y * W + x];
#pragma unroll
        for (int f = 0; f < kSoftMaxG * kSoftMaxG; ++f) {
            if (f >= sg.F) break;
            const SoftCell c = sg.cell[f];
            if (c.s != s) continue;
            const int wy = y - c.y0, wx = x - c.x0;
            if (wy < 0 || wy >= HO || wx < 0 || wx >= WO) continue;
            const float t = T[f * k + j];
            const float sg_ = q > t ? 1.f : (q < t ? -1.f : 0.f);
            const float m = -(wf[f] / (float)((c.y1 - c.y0) * (c.x1 - c.x0))) *
                            dheat[((size_t)b * HO + wy) * WO + wx] * sg_;
            z += m;
            dt[f] -= m;
        }
        Z[(size_t)bj * H * W + (size_t)y * W + x] = z;
    }
    __shared__ float red[kSoftMaxG * kSoftMaxG][4];
    const int lane = threadIdx.x & 31, wp = threadIdx.x >> 5;
#pragma unroll
    for (int f = 0; f < kSoftMaxG * kSoftMaxG; ++f) {
        float v = dt[f];
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        if (lane == 0) red[f][wp] = v;
    }
    __syncthreads();
    if (threadIdx.x < sg.F && sg.cell[threadIdx.x].s == s) {
        const int f = threadIdx.x;
        const float v = red[f][0] + red[f][1] + red[f][2] + red[f][3];
        if (v != 0.f) atomicAdd(&dT[f * k + j], v);
    }
}

// R2[row][ux] = sum over x' in [ux - w + 1, ux] within [0, W - w] of Z[row][x'] (rows y' <= H - h)
__global__ void adj_row_kernel(const float *__restrict__ Z, int H, int W, int h, int w, float *__restrict__ R2)
{
    const long long row = blockIdx.x;                         // plane * H + y'
    if ((int)(row % H) > H - h) return;
    const float *src = Z + row * W;
    for (int ux = threadIdx.x; ux < W; ux += blockDim.x) {
        const int lo = max(0, ux - w + 1), hi = min(ux, W - w);
        float s = 0.f;
        for (int xp = lo; xp <= hi; ++xp) s += src[xp];
        R2[row * W + ux] = s;
    }
}

// G[plane][uy][ux] (+)= sum over y' in [uy - h + 1, uy] within [0, H - h] of R2[plane][y'][ux]
__global__ void adj_col_kernel(const float *__restrict__ R2, int H, int W, int h, bool first, float *__restrict__ Gp)
{
    const int ux = blockIdx.x * blockDim.x + threadIdx.x, uy = blockIdx.y;
    const long long plane = blockIdx.z;
    if (ux >= W) return;
    const int lo = max(0, uy - h + 1), hi = min(uy, H - h);
    float s = 0.f;
    for (int yp = lo; yp <= hi; ++yp) s += R2[(plane * H + yp) * W + ux];
    const size_t o = (plane * H + uy) * W + ux;
    Gp[o] = first ? s : Gp[o] + s;
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

// Softmax backward with the softmax recomputed: a_j = -(1/tau) p_j (g_j - sum_i p_i g_i),
// A pixel-major; dX = 2 (sum_j a_j) x - 2 sum_j a_j c_j (skipped when dX is null).
__global__ void __launch_bounds__(256) soft_back_kernel(const float *__restrict__ X, long long n, long long npi,
                                                        int D, const float *__restrict__ C, int k, float tau,
                                                        const float *__restrict__ Gp, float *__restrict__ A,
                                                        float *__restrict__ dX)
{
    extern __shared__ float sm[];
    float (*xs)[DCH + 1] = reinterpret_cast<float (*)[DCH + 1]>(sm);
    float (*cs)[DCH + 1] = reinterpret_cast<float (*)[DCH + 1]>(sm + PT * (DCH + 1));
    float *as = sm + (PT + kSoftMaxK) * (DCH + 1);             // [PT][k + 1]
    const long long p0 = (long long)blockIdx.x * PT;
    float pr[KQ];
    tile_softmax(X, n, p0, D, C, k, tau, xs, cs, pr);
    const int p = threadIdx.x >> 2, q = threadIdx.x & 3;
    const long long g = p0 + p;
    const bool in = g < n;
    const long long item = in ? g / npi : 0, pix = in ? g % npi : 0;
    float gv[KQ];
    float s = 0.f;
#pragma unroll
    for (int i = 0; i < KQ; ++i) {
        const int j = q + 4 * i;
        gv[i] = (in && j < k) ? Gp[(item * k + j) * npi + pix] : 0.f;
        s = fmaf(pr[i], gv[i], s);
    }
    s += __shfl_xor_sync(0xffffffffu, s, 1);
    s += __shfl_xor_sync(0xffffffffu, s, 2);
    const float it = 1.0f / tau;
    float asum = 0.f;
#pragma unroll
    for (int i = 0; i < KQ; ++i) {
        const int j = q + 4 * i;
        if (j < k) {
            const float a = in ? -it * pr[i] * (gv[i] - s) : 0.f;
            as[p * (k + 1) + j] = a;
            asum += a;
            if (in) A[g * k + j] = a;
        }
    }
    asum += __shfl_xor_sync(0xffffffffu, asum, 1);
    asum += __shfl_xor_sync(0xffffffffu, asum, 2);
    if (!dX) return;                                          // uniform over the block
    for (int d0 = 0; d0 < D; d0 += DCH) {
        __syncthreads();
        for (int e = threadIdx.x; e < PT * DCH; e += blockDim.x) {
            const int pp = e / DCH, dd = e % DCH;
            const long long gg = p0 + pp;
            xs[pp][dd] = (gg < n && d0 + dd < D) ? X[gg * D + d0 + dd] : 0.f;
        }
        for (int e = threadIdx.x; e < k * DCH; e += blockDim.x) {
            const int j = e / DCH, dd = e % DCH;
            cs[j][dd] = d0 + dd < D ? C[(size_t)j * D + d0 + dd] : 0.f;
        }
        __syncthreads();
        for (int dd = q; dd < DCH; dd += 4) {
            float ac = 0.f;
            for (int j = 0; j < k; ++j) ac = fmaf(as[p * (k + 1) + j], cs[j][dd], ac);
            if (in && d0 + dd < D) dX[g * D + d0 + dd] = 2.0f * (asum * xs[p][dd] - ac);
        }
    }
}

// Partial centroid gradients over a pixel slice: part[slice][j D + d] = sum_u a_j(u) x_u[d],
// part[slice][k D + j] = sum_u a_j(u).
__global__ void __launch_bounds__(256) dc_partial_kernel(const float *__restrict__ A, const float *__restrict__ X,
                                                         long long n, int D, int k, int nslice,
                                                         float *__restrict__ part)
{
    extern __shared__ float sm[];
    float *acc = sm;                                          // [k D + k]
    float *at = acc + k * D + k;                              // [32][k]
    float *xt = at + 32 * k;                                  // [32][D]
    const int kD = k * D;
    for (int o = threadIdx.x; o < kD + k; o += blockDim.x) acc[o] = 0.f;
    const long long per = (n + nslice - 1) / nslice;
    const long long u0 = (long long)blockIdx.x * per, u1 = min(n, u0 + per);
    for (long long t0 = u0; t0 < u1; t0 += 32) {
        const int m = (int)min(32LL, u1 - t0);
        __syncthreads();
        for (int e = threadIdx.x; e < 32 * k; e += blockDim.x) at[e] = e / k < m ? A[(t0 + e / k) * k + e % k] : 0.f;
        for (int e = threadIdx.x; e < 32 * D; e += blockDim.x) xt[e] = e / D < m ? X[(t0 + e / D) * D + e % D] : 0.f;
        __syncthreads();
        for (int o = threadIdx.x; o < kD; o += blockDim.x) {
            const int j = o / D, d = o % D;
            float s = 0.f;
#pragma unroll 8
            for (int u = 0; u < 32; ++u) s = fmaf(at[u * k + j], xt[u * D + d], s);
            acc[o] += s;
        }
        for (int j = threadIdx.x; j < k; j += blockDim.x) {
            float s = 0.f;
            for (int u = 0; u < 32; ++u) s += at[u * k + j];
            acc[kD + j] += s;
        }
    }
    __syncthreads();
    for (int o = threadIdx.x; o < kD + k; o += blockDim.x) part[(size_t)blockIdx.x * (kD + k) + o] = acc[o];
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
    w.Z = w.RW;                                               // backward reuses the row-sum area
    w.R2 = w.P;                                               // and the soft-assignment area
    w.G = c.take<float>((size_t)B * k * plane);
    w.A = c.take<float>((size_t)B * k * plane);
    w.At = c.take<float>((size_t)k * th * tw);
    w.dT = c.take<float>((size_t)sg.F * k);
    w.part = c.take<float>((size_t)2 * kSoftSlices * ((size_t)k * D + k));
    return w;
}

cudaError_t soft_forward(const float *Qf, int B, int H, int W, const float *Tf, int th, int tw, int D,
                         const float *C, int k, float tau, const SoftGrid &sg, const float *wf, float *heat,
                         SoftWs &w, cudaStream_t s)
{
    const long long nq = (long long)B * H * W, nt = (long long)th * tw;
    soft_p_kernel<<<(unsigned)((nq + PT - 1) / PT), 256, 0, s>>>(Qf, nq, (long long)H * W, D, C, k, tau, w.P);
    soft_p_kernel<<<(unsigned)((nt + PT - 1) / PT), 256, 0, s>>>(Tf, nt, nt, D, C, k, tau, w.Pt);
    const long long planes = (long long)B * k;
    for (int iw = 0; iw < sg.nw; ++iw)
        row_box_kernel<<<(unsigned)(planes * H), 128, 0, s>>>(w.P, W, sg.wid[iw], w.RW + (size_t)iw * planes * H * W);
    for (int is = 0; is < sg.ns; ++is) {
        const int iw = sg.size_w[is];
        for (int b = 0; b < B; ++b) {
            dim3 g((W + 127) / 128, H, k);
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
    soft_dw_kernel<<<sg.F, 256, 0, s>>>(dheat, w.L1, B, HO, WO, sg, dwf);
    cudaError_t e = cudaMemsetAsync(w.dT, 0, sizeof(float) * sg.F * k, s);
    if (e != cudaSuccess) return e;
    const long long planes = (long long)B * k;
    for (int is = 0; is < sg.ns; ++is) {
        const int h = sg.hgt[sg.size_h[is]], wd = sg.wid[sg.size_w[is]];
        dim3 g1((W + 127) / 128, H, (unsigned)planes);
        soft_gather_kernel<<<g1, 128, 0, s>>>(w.BX, dheat, w.T, wf, H, W, k, HO, WO, sg, is, w.Z, w.dT);
        adj_row_kernel<<<(unsigned)(planes * H), 128, 0, s>>>(w.Z, H, W, h, wd, w.R2);
        dim3 g3((W + 127) / 128, H, (unsigned)planes);
        adj_col_kernel<<<g3, 128, 0, s>>>(w.R2, H, W, h, is == 0, w.G);
    }
    const size_t bsm = sizeof(float) * ((PT + kSoftMaxK) * (DCH + 1) + PT * (k + 1));
    e = cudaFuncSetAttribute(soft_back_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bsm);
    if (e != cudaSuccess) return e;
    soft_back_kernel<<<(unsigned)((nq + PT - 1) / PT), 256, bsm, s>>>(Qf, nq, (long long)H * W, D, C, k, tau, w.G,
                                                                       w.A, dQf);
    // template side: pixel gradients from dT, then its softmax backward (no feature gradient)
    tmpl_grad_kernel<<<(unsigned)((k * nt + 255) / 256), 256, 0, s>>>(w.dT, th, tw, k, sg, w.G);
    soft_back_kernel<<<(unsigned)((nt + PT - 1) / PT), 256, bsm, s>>>(Tf, nt, nt, D, C, k, tau, w.G, w.At, nullptr);
    const size_t psm = sizeof(float) * ((size_t)k * D + k + 32 * (size_t)k + 32 * (size_t)D);
    e = cudaFuncSetAttribute(dc_partial_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)psm);
    if (e != cudaSuccess) return e;
    dc_partial_kernel<<<kSoftSlices, 256, psm, s>>>(w.A, Qf, nq, D, k, kSoftSlices, w.part);
    dc_partial_kernel<<<kSoftSlices, 256, psm, s>>>(w.At, Tf, nt, D, k, kSoftSlices,
                                                    w.part + (size_t)kSoftSlices * (k * D + k));
    dc_reduce_kernel<<<(k * D + 255) / 256, 256, 0, s>>>(w.part, 2 * kSoftSlices, D, k, C, dC);
    return cudaGetLastError();
}

}  // namespace vqnnf
