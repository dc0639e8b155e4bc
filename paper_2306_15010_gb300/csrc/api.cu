// C ABI of the VQ-NNF hot path (include/vqnnf.h): argument checks, workspace layout and
// the launch sequence of every call.  All work is enqueued on the caller's stream.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <cstdlib>
#include <mutex>

#include "common.cuh"
#include "driver.cuh"
#include "score_spec.cuh"
#include "soft_spec.cuh"

using namespace vqnnf;

namespace vqnnf {

constexpr int kVersion = 100;

cudaStream_t as_stream(void *s) { return reinterpret_cast<cudaStream_t>(s); }

// ----------------------------------------------------------------------------------
// Workspace layouts (the same code computes sizes with a null base).
// ----------------------------------------------------------------------------------
AssignWs carve_assign(WsCursor &c, long long n, int D, int k, int prec)
{
    AssignWs w;
    memset(&w, 0, sizeof(w));
    w.prep.mean = c.take<float>((size_t)D);
    w.prep.cc = c.take<float>((size_t)k * D);
    w.prep.chi = c.take<uint16_t>((size_t)k * D);
    w.prep.clo = c.take<uint16_t>((size_t)k * D);
    w.prep.nrm = c.take<float>((size_t)k);
    w.prep.a = c.take<float>((size_t)k);
    w.prep.v = c.take<float>((size_t)k);
    w.prep.b = c.take<float>((size_t)k);
    w.fl.count = c.take<unsigned int>(64);     // count + stats, zeroed together
    w.fl.stats = c.base ? reinterpret_cast<unsigned long long *>(w.fl.count + 16) : nullptr;
    w.fl.pix = c.take<unsigned int>((size_t)n);
    w.fl.mask = c.take<unsigned int>((size_t)n * kMaskWords);
    if (prec == VQNNF_PREC_FP8) {
        w.prep.cq8 = c.take<uint8_t>((size_t)k * D);
        w.prep.csc = c.take<float>((size_t)k);
        w.f8.q = c.take<uint8_t>((size_t)n * D);
        w.f8.rs = c.take<float2>((size_t)n);
    }
    return w;
}

FitWs carve_fit(WsCursor &c, long long l, int D, int k, int prec)
{
    FitWs w;
    w.as = carve_assign(c, l, D, k, prec);
    w.lab = c.take<uint8_t>((size_t)l);
    w.lw.cnt = c.take<int>((size_t)k);
    w.lw.off = c.take<int>((size_t)k + 1);
    w.lw.members = c.take<int>((size_t)l);
    w.lw.ordered = c.take<int>((size_t)l);
    const long long mc = lloyd_max_chunks(l, k);
    w.lw.chunks = c.take<int4>((size_t)mc);
    w.lw.bh = c.take<int>((size_t)kLloydSortBlocks * k);
    w.lw.rcp = c.take<double>((size_t)k);
    w.lw.done = c.take<int>((size_t)k * ((D + 31) / 32));
    w.lw.part = c.take<LloydPart>((size_t)mc * D);
    return w;
}

ScoreWs carve_score(WsCursor &c, int H, int W, int k, int th, int tw)
{
    ScoreWs w;
    w.u16 = sat_is_u16(th, tw);
    const size_t elems = (size_t)(H + 1) * k * sat_pitch(W) + sat_slack_elems(tw);
    w.S = w.u16 ? (void *)c.take<uint16_t>(elems) : (void *)c.take<uint32_t>(elems);
    w.carry = c.take<int>((size_t)H * sat_strips(W) * k);
    w.bandsum = c.take<int>((size_t)sat_bands(H) * k * sat_pitch(W));
    w.amax = c.take<unsigned long long>(1);
    return w;
}

// Whole path with host buffers: device copies of both feature maps and every intermediate.
struct HostWs {
    float *X, *T, *C, *heat;
    uint8_t *tl, *ql;
    int32_t *tc, *am;
    FitWs fit;
    AssignWs as;
    ScoreWs sc;
};

HostWs carve_host(WsCursor &c, int H, int W, int D, int k, int th, int tw, int F, int prec)
{
    HostWs w;
    const long long n = (long long)H * W, l = (long long)th * tw;
    w.X = c.take<float>((size_t)n * D);
    w.T = c.take<float>((size_t)l * D);
    w.C = c.take<float>((size_t)k * D);
    w.heat = c.take<float>((size_t)(H - th + 1) * (W - tw + 1));
    w.tl = c.take<uint8_t>((size_t)l);
    w.ql = c.take<uint8_t>((size_t)n);
    w.tc = c.take<int32_t>((size_t)F * k);
    w.am = c.take<int32_t>(2);
    w.fit = carve_fit(c, l, D, k, prec);
    w.as = carve_assign(c, n, D, k, prec);
    w.sc = carve_score(c, H, W, k, th, tw);
    return w;
}

bool aligned(const void *p, size_t a) { return (reinterpret_cast<uintptr_t>(p) % a) == 0; }

vqnnf_status from_cuda(cudaError_t e)
{
    if (e == cudaSuccess) return VQNNF_OK;
    if (e == cudaErrorNotSupported) return VQNNF_EUNSUPPORTED;
    return VQNNF_ECUDA;
}

bool check_prec(int prec, int D)
{
    if (prec == VQNNF_PREC_FP32) return D % 4 == 0;
    if (prec == VQNNF_PREC_BF16 || prec == VQNNF_PREC_FP8) return D % 16 == 0;
    return false;
}

// Profiling events set by vqnnf_set_kernel_events, per operation: {start, stop}.
static std::mutex g_ev_mu;
static cudaEvent_t g_ev[4][2] = {};

}  // namespace vqnnf

bool vqnnf::pdl_enabled()
{
    // VQNNF_PDL=0 launches every kernel without programmatic stream serialization (for A/B timing)
    static const bool on = [] {
        const char *v = getenv("VQNNF_PDL");
        return !(v && v[0] == '0');
    }();
    return on;
}

cudaError_t vqnnf::record_kernel_event(int op, int which, cudaStream_t s)
{
    cudaEvent_t ev;
    {
        std::lock_guard<std::mutex> lk(g_ev_mu);
        ev = g_ev[op][which];
    }
    return ev ? cudaEventRecord(ev, s) : cudaSuccess;
}

namespace vqnnf {

// Enqueue the full assignment of n pixels (prep, contraction, re-scoring, stats).
vqnnf_status run_assign(const float *X, long long n, int D, const float *C, int k, int prec,
                        uint8_t *labels, vqnnf_assign_stats *stats, AssignWs &w, cudaStream_t s, bool keep_mean)
{
    cudaError_t e = launch_prep_codebook(C, k, D, prec, w.prep, s, w.fl.count, keep_mean);
    if (e == cudaSuccess) {
        e = record_kernel_event(VQNNF_OP_ASSIGN, 0, s);
        if (e == cudaSuccess)
            e = prec == VQNNF_PREC_BF16  ? launch_assign_bf16(X, n, D, k, w.prep, labels, w.fl, s)
                : prec == VQNNF_PREC_FP8 ? launch_assign_fp8(X, n, D, k, w.prep, w.f8, labels, w.fl, s)
                                         : launch_assign_fp32(X, n, D, k, w.prep, labels, w.fl, s);
        if (e == cudaSuccess) e = record_kernel_event(VQNNF_OP_ASSIGN, 1, s);
    }
    if (e == cudaSuccess) e = launch_rescore(X, n, D, C, k, labels, w.fl, s);
    if (e == cudaSuccess && stats) e = launch_finish_stats(w.fl, stats, s);
    return from_cuda(e);
}

// SplitMix64 (Steele, Lea & Flood 2014) and the partial Fisher-Yates initial indices,
// with the swapped slots kept in a small table instead of an l-element permutation.
uint64_t splitmix64(uint64_t &st)
{
    st += 0x9E3779B97F4A7C15ULL;
    uint64_t z = st;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}

void kmeans_init_indices(long long l, int k, uint64_t seed, int32_t *out)
{
    long long key[2 * kMaxK];
    long long val[2 * kMaxK];
    int nmap = 0;
    auto get = [&](long long p) {
        for (int q = 0; q < nmap; ++q)
            if (key[q] == p) return val[q];
        return p;
    };
    auto set = [&](long long p, long long v) {
        for (int q = 0; q < nmap; ++q)
            if (key[q] == p) { val[q] = v; return; }
        key[nmap] = p;
        val[nmap] = v;
        ++nmap;
    };
    uint64_t st = seed;
    for (int i = 0; i < k; ++i) {
        const uint64_t r = splitmix64(st);
        const long long j = (long long)i + (long long)(r % (uint64_t)(l - i));
        const long long vi = get(i), vj = get(j);
        set(i, vj);
        set(j, vi);
        out[i] = (int32_t)vj;
    }
}

// Seeded initial centroids, then `iters` Lloyd steps (assignment + exact centroid means).  The
// reference point of the assignment bound is the mean of the initial centroids, kept for every
// step (the bound holds for any fixed point; the labels are exact either way).
vqnnf_status run_fit(const float *T, long long l, int D, int k, int iters, uint64_t seed, int prec,
                     float *C, FitWs &fw, cudaStream_t s)
{
    InitIdx ii;
    memset(&ii, 0, sizeof(ii));
    kmeans_init_indices(l, k, seed, ii.idx);
    cudaError_t e = launch_gather_init(T, D, k, ii, C, s);
    if (e != cudaSuccess) return from_cuda(e);
    for (int it = 0; it < iters; ++it) {
        vqnnf_status st = run_assign(T, l, D, C, k, prec, fw.lab, nullptr, fw.as, s, it > 0);
        if (st != VQNNF_OK) return st;
        e = launch_lloyd_update(T, (int)l, D, k, fw.lab, fw.lw, C, s);
        if (e != cudaSuccess) return from_cuda(e);
    }
    return VQNNF_OK;
}

// ----------------------------------------------------------------------------------
// Filter banks.
// ----------------------------------------------------------------------------------
// Weighted-grid detection: the filters fall into at most four groups by bounding box; within
// a group, the distinct column and row boundaries of its rectangles (at most four each) cut
// the box into a 3 x 3 grid (repeated last boundaries give empty cells), every rectangle is a
// union of whole cells, and each filter becomes its cell weights.  Counts and per-window L1
// sums must stay inside int32.
void detect_wgrid(const vqnnf_filter *bank, int F, const BankSpec &bs, WGridSpec &ws)
{
    memset(&ws, 0, sizeof(ws));
    int gbox[kMaxWGrids][4];
    int ng = 0;
    for (int f = 0; f < F; ++f) {
        int bb[4] = {1 << 30, 1 << 30, -1, -1};
        for (int r = 0; r < bank[f].n_rects; ++r) {
            const vqnnf_rect &rc = bank[f].rects[r];
            bb[0] = std::min(bb[0], rc.x0); bb[1] = std::min(bb[1], rc.y0);
            bb[2] = std::max(bb[2], rc.x1); bb[3] = std::max(bb[3], rc.y1);
        }
        int g = 0;
        while (g < ng && !(gbox[g][0] == bb[0] && gbox[g][1] == bb[1] && gbox[g][2] == bb[2] && gbox[g][3] == bb[3]))
            ++g;
        if (g == ng) {
            if (ng == kMaxWGrids) return;
            for (int q = 0; q < 4; ++q) gbox[ng][q] = bb[q];
            ++ng;
        }
        if (ws.nf[g] == kMaxWFilters) { ws.nf[0] = 0; return; }
        ws.filt[g][ws.nf[g]++] = f;
    }
    for (int g = 0; g < ng; ++g) {
        int xs[2 * kMaxRects], ys[2 * kMaxRects], nx = 0, ny = 0;
        for (int q = 0; q < ws.nf[g]; ++q) {
            const vqnnf_filter &fl = bank[ws.filt[g][q]];
            for (int r = 0; r < fl.n_rects; ++r) {
                xs[nx++] = fl.rects[r].x0; xs[nx++] = fl.rects[r].x1;
                ys[ny++] = fl.rects[r].y0; ys[ny++] = fl.rects[r].y1;
            }
        }
        std::sort(xs, xs + nx);
        nx = int(std::unique(xs, xs + nx) - xs);
        std::sort(ys, ys + ny);
        ny = int(std::unique(ys, ys + ny) - ys);
        if (nx > 4 || ny > 4) { memset(&ws, 0, sizeof(ws)); return; }
        for (int q = 0; q < 4; ++q) {
            ws.bx[g][q] = xs[std::min(q, nx - 1)];
            ws.by[g][q] = ys[std::min(q, ny - 1)];
        }
        for (int q = 0; q < ws.nf[g]; ++q) {
            const int f = ws.filt[g][q];
            const vqnnf_filter &fl = bank[f];
            long long absw = 0;
            for (int r = 0; r < fl.n_rects; ++r) {
                const vqnnf_rect &rc = fl.rects[r];
                const int a = int(std::lower_bound(xs, xs + nx, rc.x0) - xs);
                const int b = int(std::lower_bound(xs, xs + nx, rc.x1) - xs);
                const int c = int(std::lower_bound(ys, ys + ny, rc.y0) - ys);
                const int d = int(std::lower_bound(ys, ys + ny, rc.y1) - ys);
                for (int rr = c; rr < d; ++rr)
                    for (int cc = a; cc < b; ++cc) ws.w[g][q][rr * 3 + cc] += rc.weight;
                absw += (long long)std::abs(rc.weight) * (rc.x1 - rc.x0) * (rc.y1 - rc.y0);
            }
            // |R| <= absw per cluster; sum_j |t - R| <= 2 absw (t and R are sums over the
            // same pixels with the same weights)
            if (2 * absw >= (1ll << 31)) { memset(&ws, 0, sizeof(ws)); return; }
            ws.coef[g][q] = bs.coef[f];
        }
    }
    ws.NG = ng;
    ws.ncol = bs.ncol;
    if (!score_grid_fits(bs.ncol)) ws.NG = 0;
}

vqnnf_status compile_bank(const vqnnf_filter *bank, int F, int th, int tw, BankSpec &bs,
                          GridSpec &gs)
{
    if (!bank || F < 1) return VQNNF_EINVAL;
    if (F > kMaxFilters) return VQNNF_EUNSUPPORTED;
    memset(&bs, 0, sizeof(bs));
    memset(&gs, 0, sizeof(gs));
    int nr = 0;
    int rows[kMaxRows];
    int nrect = 0;
    for (int f = 0; f < F; ++f) {
        const vqnnf_filter &fl = bank[f];
        if (fl.n_rects < 1 || !fl.rects || !(fl.area > 0.f) || !std::isfinite(fl.area) ||
            !std::isfinite(fl.w_f))
            return VQNNF_EINVAL;
        if (nrect + fl.n_rects > kMaxRects) return VQNNF_EUNSUPPORTED;
        bs.rect_begin[f] = nrect;
        for (int r = 0; r < fl.n_rects; ++r) {
            const vqnnf_rect &rc = fl.rects[r];
            if (rc.x0 < 0 || rc.y0 < 0 || rc.x1 > tw || rc.y1 > th || rc.x0 >= rc.x1 ||
                rc.y0 >= rc.y1)
                return VQNNF_EINVAL;
            RectSpec &o = bs.rect[nrect++];
            o.x0 = rc.x0; o.y0 = rc.y0; o.x1 = rc.x1; o.y1 = rc.y1; o.weight = rc.weight;
            for (int yy : {rc.y0, rc.y1}) {
                bool seen = false;
                for (int q = 0; q < nr; ++q) seen |= rows[q] == yy;
                if (!seen) rows[nr++] = yy;
            }
        }
        bs.coef[f] = (float)((double)fl.w_f / (double)fl.area);
    }
    bs.rect_begin[F] = nrect;
    bs.F = F;
    std::sort(rows, rows + nr);
    bs.nrow = nr;
    for (int q = 0; q < nr; ++q) bs.roff[q] = rows[q];
    for (int r = 0; r < nrect; ++r) {
        RectSpec &o = bs.rect[r];
        o.ry0 = int(std::lower_bound(rows, rows + nr, o.y0) - rows);
        o.ry1 = int(std::lower_bound(rows, rows + nr, o.y1) - rows);
    }
    bs.ncol = score_ncol(tw);

    // grid detection: single unit-weight rectangles forming a G x G cell grid (+ full)
    bool single = true;
    for (int f = 0; f < F; ++f)
        single &= bank[f].n_rects == 1 && bank[f].rects[0].weight == 1;
    if (!single) return VQNNF_OK;
    int xs[kMaxRects * 2], ys[kMaxRects * 2], nx = 0, ny = 0;
    int full_f = -1;
    for (int f = 0; f < F; ++f) {
        const vqnnf_rect &rc = bank[f].rects[0];
        if (rc.x0 == 0 && rc.y0 == 0 && rc.x1 == tw && rc.y1 == th && full_f < 0 && F > 1) {
            full_f = f;
            continue;
        }
        xs[nx++] = rc.x0; xs[nx++] = rc.x1;
        ys[ny++] = rc.y0; ys[ny++] = rc.y1;
    }
    std::sort(xs, xs + nx);
    nx = int(std::unique(xs, xs + nx) - xs);
    std::sort(ys, ys + ny);
    ny = int(std::unique(ys, ys + ny) - ys);
    const int G = nx - 1;
    if (G < 1 || G > 4 || ny - 1 != G || xs[0] != 0 || xs[G] != tw || ys[0] != 0 || ys[G] != th)
        return VQNNF_OK;
    const int ncell = F - (full_f >= 0 ? 1 : 0);
    if (ncell != G * G) return VQNNF_OK;
    if (!score_grid_fits(bs.ncol)) return VQNNF_OK;       // template wider than the grid kernel stages
    int seen[16] = {0};
    GridSpec g;
    memset(&g, 0, sizeof(g));
    for (int f = 0; f < F; ++f) {
        if (f == full_f) {
            g.filter_slot[f] = G * G;
            g.slot_filter[G * G] = f;
            continue;
        }
        const vqnnf_rect &rc = bank[f].rects[0];
        const int c = int(std::lower_bound(xs, xs + nx, rc.x0) - xs);
        const int r = int(std::lower_bound(ys, ys + ny, rc.y0) - ys);
        if (xs[c + 1] != rc.x1 || ys[r + 1] != rc.y1 || seen[r * G + c]) return VQNNF_OK;
        seen[r * G + c] = 1;
        g.filter_slot[f] = r * G + c;
        g.slot_filter[r * G + c] = f;
    }
    g.G = G;
    g.full = full_f >= 0;
    g.F = F;
    g.ncol = bs.ncol;
    for (int q = 0; q <= G; ++q) {
        g.bx[q] = xs[q];
        g.by[q] = ys[q];
    }
    for (int r = 0; r < G; ++r)
        for (int c = 0; c < G; ++c) g.slot_area[r * G + c] = (xs[c + 1] - xs[c]) * (ys[r + 1] - ys[r]);
    if (full_f >= 0) g.slot_area[G * G] = tw * th;
    for (int f = 0; f < F; ++f) {
        g.coef[f] = bs.coef[f];
        g.slot_coef[g.filter_slot[f]] = bs.coef[f];
    }
    gs = g;
    return VQNNF_OK;
}

int device_smem_optin()
{
    int dev = 0, v = 0;
    cudaGetDevice(&dev);
    if (cudaDeviceGetAttribute(&v, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess)
        return 0;
    return v;
}

}  // namespace vqnnf

extern "C" {

int vqnnf_version(void) { return kVersion; }

const char *vqnnf_status_str(vqnnf_status s)
{
    switch (s) {
    case VQNNF_OK: return "ok";
    case VQNNF_EINVAL: return "invalid argument";
    case VQNNF_ENOMEM: return "workspace too small";
    case VQNNF_ECUDA: return "CUDA error";
    case VQNNF_ETIMEOUT: return "device wait timed out";
    case VQNNF_EUNSUPPORTED: return "unsupported configuration";
    }
    return "unknown status";
}

size_t vqnnf_workspace_bytes(int op, int H, int W, int D, int k, int th, int tw, int F, int prec)
{
    (void)F;
    WsCursor c{nullptr, 0};
    switch (op) {
    case VQNNF_OP_FIT:
        if (H < 1 || W < 1 || D < 1 || k < 1 || k > kMaxK) return 0;
        carve_fit(c, (long long)H * W, D, k, prec);
        break;
    case VQNNF_OP_ASSIGN:
        if (H < 1 || W < 1 || D < 1 || k < 1 || k > kMaxK) return 0;
        carve_assign(c, (long long)H * W, D, k, prec);
        break;
    case VQNNF_OP_FILTER_RESPONSES:
        return 256;
    case VQNNF_OP_SCORE:
        if (H < 1 || W < 1 || k < 1 || k > kMaxK || th < 1 || tw < 1 || th > H || tw > W) return 0;
        carve_score(c, H, W, k, th, tw);
        break;
    default:
        return 0;
    }
    return (c.off + 255) & ~size_t(255);
}

vqnnf_status vqnnf_assign(const float *X, int H, int W, int D, const float *C, int k,
                          vqnnf_prec prec, uint8_t *labels, vqnnf_assign_stats *stats, void *ws,
                          size_t ws_bytes, void *stream)
{
    if (!X || !C || !labels || !ws || H < 1 || W < 1 || D < 1 || k < 1) return VQNNF_EINVAL;
    if (!aligned(X, 16) || !aligned(C, 16) || !aligned(ws, 256)) return VQNNF_EINVAL;
    if (k > kMaxK) return VQNNF_EUNSUPPORTED;
    if (!check_prec(prec, D)) return prec > VQNNF_PREC_FP8 ? VQNNF_EINVAL : VQNNF_EUNSUPPORTED;
    if (prec == VQNNF_PREC_FP8 && !fp8_supported(D, k)) return VQNNF_EUNSUPPORTED;
    const long long n = (long long)H * W;
    if (n >= (1ll << 32)) return VQNNF_EUNSUPPORTED;
    if (ws_bytes < vqnnf_workspace_bytes(VQNNF_OP_ASSIGN, H, W, D, k, 0, 0, 0, prec))
        return VQNNF_ENOMEM;
    WsCursor c{static_cast<char *>(ws), 0};
    AssignWs w = carve_assign(c, n, D, k, prec);
    return run_assign(X, n, D, C, k, prec, labels, stats, w, as_stream(stream));
}

vqnnf_status vqnnf_fit_codebook(const float *T, int h, int w, int D, int k, int iters,
                                uint64_t seed, vqnnf_prec prec, float *C, void *ws,
                                size_t ws_bytes, void *stream)
{
    if (!T || !C || !ws || h < 1 || w < 1 || D < 1 || k < 1 || iters < 0) return VQNNF_EINVAL;
    if (!aligned(T, 16) || !aligned(C, 16) || !aligned(ws, 256)) return VQNNF_EINVAL;
    const long long l = (long long)h * w;
    if (k > l) return VQNNF_EINVAL;
    if (k > kMaxK) return VQNNF_EUNSUPPORTED;
    if (!check_prec(prec, D)) return prec > VQNNF_PREC_FP8 ? VQNNF_EINVAL : VQNNF_EUNSUPPORTED;
    if (prec == VQNNF_PREC_FP8 && !fp8_supported(D, k)) return VQNNF_EUNSUPPORTED;
    if (l > (1ll << 30)) return VQNNF_EUNSUPPORTED;
    if (ws_bytes < vqnnf_workspace_bytes(VQNNF_OP_FIT, h, w, D, k, 0, 0, 0, prec))
        return VQNNF_ENOMEM;
    WsCursor c{static_cast<char *>(ws), 0};
    FitWs fw = carve_fit(c, l, D, k, prec);
    return run_fit(T, l, D, k, iters, seed, prec, C, fw, as_stream(stream));
}

vqnnf_status vqnnf_filter_responses(const uint8_t *labels, int h, int w, int k,
                                    const vqnnf_filter *bank, int F, int32_t *counts, void *ws,
                                    size_t ws_bytes, void *stream)
{
    (void)ws; (void)ws_bytes;
    if (!labels || !counts || h < 1 || w < 1 || k < 1) return VQNNF_EINVAL;
    if (k > kMaxK) return VQNNF_EUNSUPPORTED;
    BankSpec bs;
    GridSpec gs;
    vqnnf_status st = compile_bank(bank, F, h, w, bs, gs);
    if (st != VQNNF_OK) return st;
    return from_cuda(launch_filter_responses(labels, h, w, k, bs, counts, as_stream(stream)));
}

vqnnf_status vqnnf_score(const uint8_t *q_labels, int H, int W, int k, int th, int tw,
                         const vqnnf_filter *bank, int F, const int32_t *t_counts, float *heatmap,
                         int32_t *argmax_yx, void *ws, size_t ws_bytes, void *stream)
{
    if (!q_labels || !t_counts || !heatmap || !ws || H < 1 || W < 1 || k < 1 || th < 1 ||
        tw < 1 || th > H || tw > W)
        return VQNNF_EINVAL;
    if (!aligned(ws, 256)) return VQNNF_EINVAL;
    if (k > kMaxK) return VQNNF_EUNSUPPORTED;
    if ((long long)(H + 1) * (W + 1) >= (1ll << 31)) return VQNNF_EUNSUPPORTED;
    if (ws_bytes < vqnnf_workspace_bytes(VQNNF_OP_SCORE, H, W, 0, k, th, tw, F, 0))
        return VQNNF_ENOMEM;
    BankSpec bs;
    GridSpec gs;
    WGridSpec wg;
    vqnnf_status st = compile_bank(bank, F, th, tw, bs, gs);
    if (st != VQNNF_OK) return st;
    memset(&wg, 0, sizeof(wg));
    if (gs.G == 0) detect_wgrid(bank, F, bs, wg);
    const bool u16 = sat_is_u16(th, tw);
    const size_t smem = wg.NG > 0 ? score_wgrid_smem_bytes(u16 ? 2 : 4, wg, k)
                                  : score_smem_bytes_for(u16 ? 2 : 4, bs, gs, k);
    if (smem > (size_t)device_smem_optin()) return VQNNF_EUNSUPPORTED;
    cudaStream_t s = as_stream(stream);
    WsCursor c{static_cast<char *>(ws), 0};
    ScoreWs sw = carve_score(c, H, W, k, th, tw);
    cudaError_t e = launch_sat(q_labels, H, W, k, sw.u16, sw.carry, sw.bandsum, sw.S, s);
    if (e != cudaSuccess) return from_cuda(e);
    const int HO = H - th + 1, WO = W - tw + 1;
    return from_cuda(launch_score(sw.S, sw.u16, W, k, HO, WO, bs, gs, wg, t_counts, heatmap, sw.amax,
                                  argmax_yx, s));
}

// ------------------------------------------------------------------ whole path, host buffers
static vqnnf_status match_host_check(int H, int W, int D, int k, int th, int tw, int F, int prec)
{
    if (H < 1 || W < 1 || D < 1 || k < 1 || th < 1 || tw < 1 || th > H || tw > W || F < 1) return VQNNF_EINVAL;
    if ((long long)k > (long long)th * tw) return VQNNF_EINVAL;
    if (k > kMaxK) return VQNNF_EUNSUPPORTED;
    if (!check_prec(prec, D)) return prec > VQNNF_PREC_FP8 ? VQNNF_EINVAL : VQNNF_EUNSUPPORTED;
    if (prec == VQNNF_PREC_FP8 && !fp8_supported(D, k)) return VQNNF_EUNSUPPORTED;
    if ((long long)H * W >= (1ll << 32) || (long long)th * tw > (1ll << 30) ||
        (long long)(H + 1) * (W + 1) >= (1ll << 31))
        return VQNNF_EUNSUPPORTED;
    return VQNNF_OK;
}

size_t vqnnf_match_host_workspace_bytes(int H, int W, int D, int k, int th, int tw, int F, vqnnf_prec prec)
{
    if (match_host_check(H, W, D, k, th, tw, F, prec) != VQNNF_OK) return 0;
    WsCursor c{nullptr, 0};
    carve_host(c, H, W, D, k, th, tw, F, prec);
    return (c.off + 255) & ~size_t(255);
}

vqnnf_status vqnnf_match_host(const float *X_host, int H, int W, int D, const float *T_host, int th, int tw,
                              int k, int iters, uint64_t seed, vqnnf_prec prec, const vqnnf_filter *bank, int F,
                              float *heat_host, int32_t *argmax_host, void *ws, size_t ws_bytes, void *stream,
                              void *stream2)
{
    if (!X_host || !T_host || !argmax_host || !ws || iters < 0 || !aligned(ws, 256)) return VQNNF_EINVAL;
    vqnnf_status st = match_host_check(H, W, D, k, th, tw, F, prec);
    if (st != VQNNF_OK) return st;
    if (ws_bytes < vqnnf_match_host_workspace_bytes(H, W, D, k, th, tw, F, prec)) return VQNNF_ENOMEM;
    BankSpec bs;
    GridSpec gs;
    WGridSpec wg;
    if ((st = compile_bank(bank, F, th, tw, bs, gs)) != VQNNF_OK) return st;
    memset(&wg, 0, sizeof(wg));
    if (gs.G == 0) detect_wgrid(bank, F, bs, wg);
    const bool u16 = sat_is_u16(th, tw);
    const size_t smem = wg.NG > 0 ? score_wgrid_smem_bytes(u16 ? 2 : 4, wg, k)
                                  : score_smem_bytes_for(u16 ? 2 : 4, bs, gs, k);
    if (smem > (size_t)device_smem_optin()) return VQNNF_EUNSUPPORTED;
    WsCursor cur{static_cast<char *>(ws), 0};
    HostWs w = carve_host(cur, H, W, D, k, th, tw, F, prec);
    const cudaStream_t s = as_stream(stream), cs = stream2 ? as_stream(stream2) : s;
    const long long l = (long long)th * tw;
    constexpr int kBands = 8;
    const int nb = H < kBands ? H : kBands;
    cudaEvent_t evT = nullptr, evDone = nullptr, evB[kBands] = {};
    cudaError_t e = cudaEventCreateWithFlags(&evT, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&evDone, cudaEventDisableTiming);
    for (int b = 0; b < nb && e == cudaSuccess; ++b) e = cudaEventCreateWithFlags(&evB[b], cudaEventDisableTiming);
    // copies, in order: the template, then the query's row bands
    if (e == cudaSuccess) e = cudaMemcpyAsync(w.T, T_host, sizeof(float) * (size_t)l * D, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaEventRecord(evT, s);
    for (int b = 0; b < nb && e == cudaSuccess; ++b) {
        const long long y0 = (long long)H * b / nb, y1 = (long long)H * (b + 1) / nb;
        const size_t off = (size_t)y0 * W * D;
        e = cudaMemcpyAsync(w.X + off, X_host + off, sizeof(float) * (size_t)(y1 - y0) * W * D,
                            cudaMemcpyHostToDevice, s);
        if (e == cudaSuccess) e = cudaEventRecord(evB[b], s);
    }
    // compute: template side, then each band's assignment once it has landed, then the score
    if (e == cudaSuccess) e = cudaStreamWaitEvent(cs, evT, 0);
    if (e == cudaSuccess) {
        st = run_fit(w.T, l, D, k, iters, seed, prec, w.C, w.fit, cs);
        if (st == VQNNF_OK) st = run_assign(w.T, l, D, w.C, k, prec, w.tl, nullptr, w.fit.as, cs);
        if (st == VQNNF_OK) st = from_cuda(launch_filter_responses(w.tl, th, tw, k, bs, w.tc, cs));
        for (int b = 0; b < nb && st == VQNNF_OK; ++b) {
            const long long y0 = (long long)H * b / nb, y1 = (long long)H * (b + 1) / nb;
            st = from_cuda(cudaStreamWaitEvent(cs, evB[b], 0));
            if (st == VQNNF_OK)
                st = run_assign(w.X + (size_t)y0 * W * D, (y1 - y0) * W, D, w.C, k, prec, w.ql + (size_t)y0 * W,
                                nullptr, w.as, cs);
        }
        const int HO = H - th + 1, WO = W - tw + 1;
        if (st == VQNNF_OK) st = from_cuda(launch_sat(w.ql, H, W, k, w.sc.u16, w.sc.carry, w.sc.bandsum, w.sc.S, cs));
        if (st == VQNNF_OK)
            st = from_cuda(launch_score(w.sc.S, w.sc.u16, W, k, HO, WO, bs, gs, wg, w.tc, w.heat, w.sc.amax, w.am, cs));
        if (st == VQNNF_OK && heat_host)
            st = from_cuda(cudaMemcpyAsync(heat_host, w.heat, sizeof(float) * (size_t)HO * WO,
                                           cudaMemcpyDeviceToHost, cs));
        if (st == VQNNF_OK)
            st = from_cuda(cudaMemcpyAsync(argmax_host, w.am, 2 * sizeof(int32_t), cudaMemcpyDeviceToHost, cs));
        // the caller's stream reaches the end of this call's work only after the compute stream
        if (st == VQNNF_OK) st = from_cuda(cudaEventRecord(evDone, cs));
        if (st == VQNNF_OK) st = from_cuda(cudaStreamWaitEvent(s, evDone, 0));
    } else {
        st = from_cuda(e);
    }
    // events are released once their pending work completes
    if (evT) cudaEventDestroy(evT);
    if (evDone) cudaEventDestroy(evDone);
    for (int b = 0; b < nb; ++b)
        if (evB[b]) cudaEventDestroy(evB[b]);
    return st;
}

// ------------------------------------------------------------------ soft-VQ heatmap
static vqnnf_status soft_check(const void *Qf, int B, int H, int W, const void *Tf, int th, int tw, int D,
                               const void *C, int k, float tau, int G, SoftGrid &sg)
{
    if (!Qf || !Tf || !C || B < 1 || H < 1 || W < 1 || th < 1 || tw < 1 || th > H || tw > W || D < 1 ||
        k < 1 || !(tau > 0.f) || !std::isfinite(tau))
        return VQNNF_EINVAL;
    if (k > kSoftMaxK || D > 512 || (long long)k * D > 32768 || (long long)B * k > 65535 ||
        H > 65535 || W > 12288 || (long long)B * k * H >= (1ll << 31) || (long long)B * k * H * W >= (1ll << 40))
        return VQNNF_EUNSUPPORTED;
    if (!soft_grid(th, tw, G, sg)) return G < 1 || G > kSoftMaxG ? VQNNF_EUNSUPPORTED : VQNNF_EINVAL;
    return VQNNF_OK;
}

size_t vqnnf_soft_workspace_bytes(int B, int H, int W, int D, int k, int th, int tw, int G)
{
    SoftGrid sg;
    if (B < 1 || H < 1 || W < 1 || th < 1 || tw < 1 || th > H || tw > W || k < 1 || D < 1 ||
        !soft_grid(th, tw, G, sg))
        return 0;
    return soft_workspace_bytes(B, H, W, D, k, th, tw, sg);
}

vqnnf_status vqnnf_soft_forward(const float *Qf, int B, int H, int W, const float *Tf, int th, int tw, int D,
                                const float *C, int k, float tau, int G, const float *wf, float *heat,
                                void *ws, size_t ws_bytes, void *stream)
{
    SoftGrid sg;
    vqnnf_status st = soft_check(Qf, B, H, W, Tf, th, tw, D, C, k, tau, G, sg);
    if (st != VQNNF_OK) return st;
    if (!wf || !heat || !ws || !aligned(ws, 256)) return VQNNF_EINVAL;
    if (ws_bytes < soft_workspace_bytes(B, H, W, D, k, th, tw, sg)) return VQNNF_ENOMEM;
    WsCursor c{static_cast<char *>(ws), 0};
    SoftWs w = carve_soft(c, B, H, W, D, k, th, tw, sg);
    return from_cuda(soft_forward(Qf, B, H, W, Tf, th, tw, D, C, k, tau, sg, wf, heat, w, as_stream(stream)));
}

vqnnf_status vqnnf_soft_backward(const float *Qf, int B, int H, int W, const float *Tf, int th, int tw, int D,
                                 const float *C, int k, float tau, int G, const float *wf, const float *dheat,
                                 float *dQf, float *dC, float *dwf, void *ws, size_t ws_bytes, void *stream)
{
    SoftGrid sg;
    vqnnf_status st = soft_check(Qf, B, H, W, Tf, th, tw, D, C, k, tau, G, sg);
    if (st != VQNNF_OK) return st;
    if (!wf || !dheat || !dQf || !dC || !dwf || !ws || !aligned(ws, 256)) return VQNNF_EINVAL;
    if (ws_bytes < soft_workspace_bytes(B, H, W, D, k, th, tw, sg)) return VQNNF_ENOMEM;
    WsCursor c{static_cast<char *>(ws), 0};
    SoftWs w = carve_soft(c, B, H, W, D, k, th, tw, sg);
    return from_cuda(soft_backward(Qf, B, H, W, Tf, th, tw, D, C, k, tau, sg, wf, dheat, dQf, dC, dwf, w,
                                   as_stream(stream)));
}

vqnnf_status vqnnf_set_kernel_events(int op, void *start_event, void *stop_event)
{
    if (op != VQNNF_OP_ASSIGN && op != VQNNF_OP_SCORE) return VQNNF_EINVAL;
    if ((start_event == nullptr) != (stop_event == nullptr)) return VQNNF_EINVAL;
    std::lock_guard<std::mutex> lk(g_ev_mu);
    g_ev[op][0] = static_cast<cudaEvent_t>(start_event);
    g_ev[op][1] = static_cast<cudaEvent_t>(stop_event);
    return VQNNF_OK;
}

vqnnf_status vqnnf_last_device_error(void *stream)
{
    if (cudaStreamSynchronize(as_stream(stream)) != cudaSuccess) return VQNNF_ECUDA;
    int err = 0, err2 = 0, err3 = 0;
    if (read_and_clear_tc_error(&err) != cudaSuccess) return VQNNF_ECUDA;
    if (read_and_clear_score_error(&err2) != cudaSuccess) return VQNNF_ECUDA;
    if (read_and_clear_soft_error(&err3) != cudaSuccess) return VQNNF_ECUDA;
    return (err || err2 || err3) ? VQNNF_ETIMEOUT : VQNNF_OK;
}

vqnnf_status vqnnf_selftest_bounded_wait(long long limit_cycles, void *stream)
{
    if (limit_cycles < 1 || limit_cycles > VQNNF_WAIT_LIMIT_CYCLES) return VQNNF_EINVAL;
    return from_cuda(launch_wait_selftest(limit_cycles, as_stream(stream)));
}

}  // extern "C"

// ----------------------------------------------------------------------------------
// Allocation-free assignment: the scratch workspace is a fixed device array compiled into
// the library.  Host code may not pass the array's name to a kernel (on the host it is only
// a stand-in symbol); its device address is looked up once per device with
// cudaGetSymbolAddress, with that device current, and cached.
// ----------------------------------------------------------------------------------
namespace {

constexpr size_t kNoallocBytes = VQNNF_NOALLOC_SCRATCH_BYTES;
__device__ __align__(256) unsigned char g_noalloc_scratch[kNoallocBytes];

constexpr int kNoallocMaxDevices = 64;
std::mutex g_noalloc_mu;
void *g_noalloc_ptr[kNoallocMaxDevices];

// Device address of the scratch area on the current device (set up on first use).
cudaError_t noalloc_scratch(void **out)
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= kNoallocMaxDevices) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lock(g_noalloc_mu);
    if (!g_noalloc_ptr[dev]) {
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess) return e;
        g_noalloc_ptr[dev] = p;
    }
    *out = g_noalloc_ptr[dev];
    return cudaSuccess;
}

}  // namespace

extern "C" vqnnf_status vqnnf_assign_noalloc(const float *X, int H, int W, int D, const float *C,
                                             int k, vqnnf_prec prec, uint8_t *labels,
                                             vqnnf_assign_stats *stats, void *stream)
{
    if (!X || !C || !labels || H < 1 || W < 1 || D < 1 || k < 1) return VQNNF_EINVAL;
    if (!aligned(X, 16) || !aligned(C, 16)) return VQNNF_EINVAL;
    if (k > kMaxK) return VQNNF_EUNSUPPORTED;
    if (!check_prec(prec, D)) return prec > VQNNF_PREC_FP8 ? VQNNF_EINVAL : VQNNF_EUNSUPPORTED;
    if (prec == VQNNF_PREC_FP8 && !fp8_supported(D, k)) return VQNNF_EUNSUPPORTED;
    const long long n = (long long)H * W;
    if (n >= (1ll << 32)) return VQNNF_EUNSUPPORTED;
    const size_t need = vqnnf_workspace_bytes(VQNNF_OP_ASSIGN, H, W, D, k, 0, 0, 0, prec);
    if (need == 0 || need > kNoallocBytes) return VQNNF_ENOMEM;
    void *base = nullptr;
    if (noalloc_scratch(&base) != cudaSuccess) return VQNNF_ECUDA;
    WsCursor c{static_cast<char *>(base), 0};
    AssignWs w = carve_assign(c, n, D, k, prec);
    return run_assign(X, n, D, C, k, prec, labels, stats, w, as_stream(stream));
}
