// Batched matching (vqnnf_match_batch, vqnnf_batch_tune): many templates against many queries.
//
// The template side of the method (codebook by k-means, template NNF, filter responses;
// Sec. 3.1-3.2) runs once per template; every query is then quantised against every
// template's codebook (Algorithm 1) and every pair gets its integral image, Eq. 2 heatmap and
// maximum (Sec. 3.3).  Codebooks are packed into groups that share one tensor-core
// contraction: each codebook padded to a multiple of 32 columns, at most plan.group_cols
// columns (and eight codebooks) per group, first fit in template order.  The contraction
// kernel keeps every codebook's argmin, interval test, labels and flag list apart (segments),
// so a query's features are read from HBM once per group instead of once per template.
#include <algorithm>
#include <cstring>
#include <mutex>
#include <vector>

#include "common.cuh"
#include "driver.cuh"
#include "score_spec.cuh"

using namespace vqnnf;

namespace {

constexpr int kGroupRows = kMaxK;            // rows of one group codebook, at most
constexpr int kLanes = 8;                    // pairs of one query in flight at once (streams)

// The library's own streams and events for the lanes, created once per device on first use
// (outside any stream capture in the intended use: the first call is a warm-up) and kept for
// the process.  If they cannot be created, everything runs on the caller's stream.
struct LanePool {
    bool ok = false;
    cudaStream_t st[kLanes];
    cudaEvent_t fork, join[kLanes][2];
};

// The lanes and their events are shared by every call on a device, so the batch calls of
// several host threads take this lock while they enqueue (the work itself still overlaps).
std::recursive_mutex g_lane_mu;

bool lane_pool(LanePool *&out)
{
    static std::mutex mu;
    static LanePool pools[64];
    static bool tried[64];
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return false;
    std::lock_guard<std::mutex> lk(mu);
    LanePool &p = pools[dev];
    if (!tried[dev]) {
        tried[dev] = true;
        bool ok = cudaEventCreateWithFlags(&p.fork, cudaEventDisableTiming) == cudaSuccess;
        for (int l = 0; l < kLanes && ok; ++l)
            ok = cudaStreamCreateWithFlags(&p.st[l], cudaStreamNonBlocking) == cudaSuccess &&
                 cudaEventCreateWithFlags(&p.join[l][0], cudaEventDisableTiming) == cudaSuccess &&
                 cudaEventCreateWithFlags(&p.join[l][1], cudaEventDisableTiming) == cudaSuccess;
        p.ok = ok;
        if (!ok) cudaGetLastError();                 // clear the failed creation's error
    }
    out = &p;
    return p.ok;
}

struct GroupSrc {
    int nseg;
    int col0[kMaxSeg], ncol[kMaxSeg], k[kMaxSeg];
    const float *C[kMaxSeg];
};

// Group codebook: row r of segment q is centroid r - col0[q] of codebook q; its padding rows
// repeat centroid 0, and rows past the last segment are zero (the contraction kernel never
// picks a padding column).
__global__ void group_codebook_kernel(GroupSrc g, int D, float *__restrict__ Cg)
{
    const int r = blockIdx.x;
    const float *src = nullptr;
#pragma unroll
    for (int q = 0; q < kMaxSeg; ++q)
        if (q < g.nseg && r >= g.col0[q] && r < g.col0[q] + g.ncol[q]) {
            const int li = r - g.col0[q];
            src = g.C[q] + (size_t)(li < g.k[q] ? li : 0) * D;
        }
    for (int d = threadIdx.x; d < D; d += blockDim.x) Cg[(size_t)r * D + d] = src ? src[d] : 0.f;
}

struct Group {
    int nseg = 0, npad = 0;
    int tj[kMaxSeg];                          // template of each segment
};

struct BatchWs {
    std::vector<float *> C;                   // per template: codebook k x D
    std::vector<uint8_t *> tlab;              // per template: NNF h x w
    std::vector<int32_t *> tcnt;              // per template: responses F x k
    std::vector<float *> gC;                  // per group slot: group codebook
    std::vector<CodebookPrep> gprep;          // per group slot: its prepared planes
    std::vector<uint8_t *> qlab;              // per template: the current query's NNF (one of qset)
    std::vector<uint8_t *> qset[2];           // two sets, alternating between queries
    unsigned *flcount;                        // kMaxSegStat x 64 (counters and stats, one memset)
    FlagList fl[kMaxSegStat];
    float *sC;                                // stationary codebooks, every launch's groups in a row
    CodebookPrep sprep;                       // their prepared planes (one common centring mean)
    FitWs fit[kLanes];                        // per lane: the k-means and template-NNF workspace
    char *score_base[kLanes];                 // integral-image workspace of one pair per lane
    float *heat_scratch[kLanes];              // heatmap of one pair when the caller wants maxima only
};

int bank_size(int G) { return 1 + G * G; }

BatchWs carve_batch(WsCursor &c, const vqnnf_image *q, int nq, const vqnnf_batch_template *t, int nt, int D,
                    int G)
{
    BatchWs w;
    long long n_max = 0, l_max = 0, hw_max = 0;
    int k_max = 1, H_max = 1, W_max = 1;
    for (int i = 0; i < nq; ++i) {
        n_max = std::max(n_max, (long long)q[i].H * q[i].W);
        H_max = std::max(H_max, (int)q[i].H);
        W_max = std::max(W_max, (int)q[i].W);
    }
    for (int j = 0; j < nt; ++j) {
        l_max = std::max(l_max, (long long)t[j].h * t[j].w);
        k_max = std::max(k_max, (int)t[j].k);
    }
    for (int i = 0; i < nq; ++i)
        for (int j = 0; j < nt; ++j)
            hw_max = std::max(hw_max, (long long)(q[i].H - t[j].h + 1) * (q[i].W - t[j].w + 1));
    const int F = bank_size(G);
    for (int j = 0; j < nt; ++j) {
        w.C.push_back(c.take<float>((size_t)t[j].k * D));
        w.tlab.push_back(c.take<uint8_t>((size_t)t[j].h * t[j].w));
        w.tcnt.push_back(c.take<int32_t>((size_t)F * t[j].k));
    }
    for (int g = 0; g < nt; ++g) {            // at most one group per template
        w.gC.push_back(c.take<float>((size_t)kGroupRows * D));
        CodebookPrep p;
        p.mean = c.take<float>((size_t)D);
        p.cc = c.take<float>((size_t)kGroupRows * D);
        p.chi = c.take<uint16_t>((size_t)kGroupRows * D);
        p.clo = c.take<uint16_t>((size_t)kGroupRows * D);
        p.nrm = c.take<float>(kGroupRows);
        p.a = c.take<float>(kGroupRows);
        p.v = c.take<float>(kGroupRows);
        p.b = c.take<float>(kGroupRows);
        w.gprep.push_back(p);
    }
    for (int b = 0; b < 2; ++b)
        for (int j = 0; j < nt; ++j) w.qset[b].push_back(c.take<uint8_t>((size_t)n_max));
    w.qlab = w.qset[0];
    w.flcount = c.take<unsigned>((size_t)kMaxSegStat * 64);
    for (int s = 0; s < kMaxSegStat; ++s) {
        FlagList &f = w.fl[s];
        f.count = w.flcount ? w.flcount + 64 * s : nullptr;
        f.stats = w.flcount ? reinterpret_cast<unsigned long long *>(f.count + 16) : nullptr;
        f.pix = c.take<unsigned>((size_t)n_max);
        f.mask = c.take<unsigned>((size_t)n_max * kMaskWords);
    }
    // stationary codebooks: at most one 256-column group per template
    const size_t srows = (size_t)nt * kGroupRows;
    w.sC = c.take<float>(srows * D);
    w.sprep.mean = c.take<float>((size_t)D);
    w.sprep.cc = c.take<float>(srows * D);
    w.sprep.chi = c.take<uint16_t>(srows * D);
    w.sprep.clo = c.take<uint16_t>(srows * D);
    w.sprep.nrm = c.take<float>(srows);
    w.sprep.a = c.take<float>(srows);
    w.sprep.v = c.take<float>(srows);
    w.sprep.b = c.take<float>(srows);
    for (int l = 0; l < kLanes; ++l) w.fit[l] = carve_fit(c, l_max, D, k_max);
    // the largest integral-image layout over the templates (its size depends on the template)
    size_t sbytes = 0;
    for (int j = 0; j < nt; ++j) {
        WsCursor z{nullptr, 0};
        carve_score(z, H_max, W_max, k_max, t[j].h, t[j].w);
        sbytes = std::max(sbytes, z.off);
    }
    for (int l = 0; l < kLanes; ++l) {
        w.score_base[l] = c.take<char>(sbytes);
        w.heat_scratch[l] = c.take<float>((size_t)hw_max);
    }
    return w;
}

// Grid bank of a th x tw template: the full window, then the cells r * G + c.
void grid_bank(int th, int tw, int G, std::vector<vqnnf_rect> &rects, std::vector<vqnnf_filter> &bank)
{
    rects.clear();
    bank.clear();
    rects.push_back(vqnnf_rect{0, 0, tw, th, 1});
    for (int r = 0; r < G; ++r)
        for (int c = 0; c < G; ++c) {
            vqnnf_rect rc;
            rc.x0 = c * tw / G;
            rc.x1 = (c + 1) * tw / G;
            rc.y0 = r * th / G;
            rc.y1 = (r + 1) * th / G;
            rc.weight = 1;
            rects.push_back(rc);
        }
    for (size_t f = 0; f < rects.size(); ++f) {
        vqnnf_filter fl;
        fl.n_rects = 1;
        fl.rects = nullptr;                     // set below, once rects no longer moves
        fl.w_f = 1.0f;
        fl.area = (float)((rects[f].x1 - rects[f].x0) * (rects[f].y1 - rects[f].y0));
        bank.push_back(fl);
    }
    for (size_t f = 0; f < rects.size(); ++f) bank[f].rects = &rects[f];
}

// First-fit packing of the codebooks (padded to 32 columns) into groups of at most
// group_cols columns and kMaxSeg codebooks; a codebook wider than group_cols is a group of
// its own.
std::vector<Group> make_groups(const vqnnf_batch_template *t, int nt, int group_cols)
{
    std::vector<Group> gs;
    for (int j = 0; j < nt; ++j) {
        const int nc = (t[j].k + 31) / 32 * 32;
        size_t g = 0;
        while (g < gs.size() && (gs[g].nseg == kMaxSeg || gs[g].npad + nc > std::max(group_cols, nc))) ++g;
        if (g == gs.size()) gs.push_back(Group{});
        Group &G = gs[g];
        G.tj[G.nseg++] = j;
        G.npad += nc;
    }
    return gs;
}

vqnnf_status check_batch(const vqnnf_image *q, int nq, const vqnnf_batch_template *t, int nt, int D, int G)
{
    if (!q || !t || nq < 1 || nt < 1 || D < 1) return VQNNF_EINVAL;
    if (G < 1 || G > 4 || D % 16 != 0) return VQNNF_EUNSUPPORTED;
    if ((long long)nq * nt > 65536) return VQNNF_EUNSUPPORTED;
    for (int i = 0; i < nq; ++i) {
        if (!q[i].X || q[i].H < 1 || q[i].W < 1 || !aligned(q[i].X, 16)) return VQNNF_EINVAL;
        if ((long long)q[i].H * q[i].W >= (1ll << 31) || (long long)(q[i].H + 1) * (q[i].W + 1) >= (1ll << 31))
            return VQNNF_EUNSUPPORTED;
    }
    for (int j = 0; j < nt; ++j) {
        if (!t[j].T || t[j].h < 1 || t[j].w < 1 || t[j].k < 1 || !aligned(t[j].T, 16)) return VQNNF_EINVAL;
        if ((long long)t[j].k > (long long)t[j].h * t[j].w || t[j].h < G || t[j].w < G) return VQNNF_EINVAL;
        if (t[j].k > kMaxK) return VQNNF_EUNSUPPORTED;
        for (int i = 0; i < nq; ++i)
            if (t[j].h > q[i].H || t[j].w > q[i].W) return VQNNF_EINVAL;
    }
    return VQNNF_OK;
}

vqnnf_status check_plan(const vqnnf_batch_plan &p)
{
    if (p.group_cols != 128 && p.group_cols != 256) return VQNNF_EINVAL;
    if (p.sf != 0 && (p.sf < 2 || p.sf > 8 || p.sf % 2)) return VQNNF_EINVAL;
    if (p.pf < -1 || p.pf > 64) return VQNNF_EINVAL;
    if (p.stationary != 0 && p.stationary != 1) return VQNNF_EINVAL;
    return VQNNF_OK;
}

const vqnnf_batch_plan kDefaultPlan = {256, 0, -1, 1};

// ---------------------------------------------------------------- stationary launches
// Codebooks of at most 128 columns go to groups of 128 columns (first fit), wider ones to
// groups of 256; each launch holds as many groups as its shared memory allows (and at most
// kMaxSegStat codebooks); every launch's groups sit one after another in the concatenated
// stationary codebook.
struct StatLaunch {
    int gcols, ngroup, row0;                  // group width, groups, first row in the codebook
    std::vector<int> tj;                      // template of each segment, in group order
    std::vector<int> gs0;                     // group g's segments: [gs0[g], gs0[g + 1])
};

bool stat_possible(int D)
{
    return D % 16 == 0 && (D + 63) / 64 <= 4 && stat_max_groups(D, 128) >= 1 && stat_max_groups(D, 256) >= 1;
}

std::vector<StatLaunch> make_stat_plan(const vqnnf_batch_template *t, int nt, int D)
{
    std::vector<StatLaunch> out;
    int row = 0;
    for (int gcols : {128, 256}) {
        std::vector<int> js;
        for (int j = 0; j < nt; ++j) {
            const int nc = (t[j].k + 31) / 32 * 32;
            if ((gcols == 128) == (nc <= 128)) js.push_back(j);
        }
        if (js.empty()) continue;
        std::vector<Group> gs;                            // first fit into groups of gcols columns
        for (int j : js) {
            const int nc = (t[j].k + 31) / 32 * 32;
            size_t g = 0;
            while (g < gs.size() && (gs[g].nseg == kMaxSeg || gs[g].npad + nc > gcols)) ++g;
            if (g == gs.size()) gs.push_back(Group{});
            gs[g].tj[gs[g].nseg++] = j;
            gs[g].npad += nc;
        }
        const int gmax = std::min(stat_max_groups(D, gcols), kMaxGroupsStat);
        size_t gi = 0;
        while (gi < gs.size()) {
            StatLaunch L;
            L.gcols = gcols;
            L.row0 = row;
            L.gs0.push_back(0);
            while (gi < gs.size() && (int)L.gs0.size() - 1 < gmax &&
                   (int)L.tj.size() + gs[gi].nseg <= kMaxSegStat) {
                for (int q = 0; q < gs[gi].nseg; ++q) L.tj.push_back(gs[gi].tj[q]);
                L.gs0.push_back((int)L.tj.size());
                ++gi;
            }
            L.ngroup = (int)L.gs0.size() - 1;
            row += L.ngroup * gcols;
            out.push_back(L);
        }
    }
    return out;
}

// The concatenated stationary codebook (group g of launch L at rows L.row0 + g * L.gcols) and
// its prepared planes, centred on the mean of all its rows.
vqnnf_status build_stat(const std::vector<StatLaunch> &plan, const vqnnf_batch_template *t, int D, BatchWs &w,
                        cudaStream_t s)
{
    int rows = 0;
    for (const StatLaunch &L : plan) {
        for (int gi = 0; gi < L.ngroup; ++gi) {
            GroupSrc src;
            memset(&src, 0, sizeof(src));
            int col = 0;
            for (int q = L.gs0[gi]; q < L.gs0[gi + 1]; ++q) {
                const int j = L.tj[q], e = q - L.gs0[gi];
                src.col0[e] = col;
                src.ncol[e] = (t[j].k + 31) / 32 * 32;
                src.k[e] = t[j].k;
                src.C[e] = w.C[j];
                col += src.ncol[e];
            }
            src.nseg = L.gs0[gi + 1] - L.gs0[gi];
            group_codebook_kernel<<<L.gcols, 128, 0, s>>>(src, D, w.sC + (size_t)(L.row0 + gi * L.gcols) * D);
            cudaError_t e = cudaGetLastError();
            if (e != cudaSuccess) return from_cuda(e);
        }
        rows = L.row0 + L.ngroup * L.gcols;
    }
    if (rows == 0) return VQNNF_OK;
    return from_cuda(launch_prep_codebook(w.sC, rows, D, VQNNF_PREC_BF16, w.sprep, s));
}

CodebookPrep prep_rows(const CodebookPrep &p, int row0, int D)
{
    CodebookPrep v = p;                                   // same centring mean
    v.cc = p.cc + (size_t)row0 * D;
    v.chi = p.chi + (size_t)row0 * D;
    v.clo = p.clo + (size_t)row0 * D;
    v.nrm = p.nrm + row0;
    v.a = p.a + row0;
    v.v = p.v + row0;
    v.b = p.b + row0;
    return v;
}

// NNF of query i under every codebook, each stationary launch reading the features once.
vqnnf_status assign_query_stat(const vqnnf_image &qi, const std::vector<StatLaunch> &plan,
                               const vqnnf_batch_template *t, int D, BatchWs &w, cudaStream_t s)
{
    const long long n = (long long)qi.H * qi.W;
    for (const StatLaunch &L : plan) {
        cudaError_t e = cudaMemsetAsync(w.flcount, 0, sizeof(unsigned) * 64 * kMaxSegStat, s);
        if (e != cudaSuccess) return from_cuda(e);
        std::vector<TcSeg> seg(L.tj.size());
        for (int gi = 0; gi < L.ngroup; ++gi) {
            int col = gi * L.gcols;
            for (int q = L.gs0[gi]; q < L.gs0[gi + 1]; ++q) {
                const int j = L.tj[q];
                seg[q].col0 = col;
                seg[q].ncol = (t[j].k + 31) / 32 * 32;
                seg[q].k = t[j].k;
                seg[q].labels = w.qlab[j];
                seg[q].fl = w.fl[q];
                col += seg[q].ncol;
            }
        }
        e = launch_assign_bf16_stat(qi.X, n, D, prep_rows(w.sprep, L.row0, D), L.ngroup, L.gcols, seg.data(),
                                    L.gs0.data(), s);
        if (e != cudaSuccess) return from_cuda(e);
        for (size_t q = 0; q < L.tj.size(); ++q) {
            const int j = L.tj[q];
            e = launch_rescore(qi.X, n, D, w.C[j], t[j].k, w.qlab[j], w.fl[q], s);
            if (e != cudaSuccess) return from_cuda(e);
        }
    }
    return VQNNF_OK;
}

struct Banks {
    std::vector<BankSpec> bs;
    std::vector<GridSpec> gs;
};

vqnnf_status compile_banks(const vqnnf_batch_template *t, int nt, int G, Banks &b)
{
    b.bs.resize(nt);
    b.gs.resize(nt);
    std::vector<vqnnf_rect> rects;
    std::vector<vqnnf_filter> bank;
    const int optin = device_smem_optin();
    for (int j = 0; j < nt; ++j) {
        grid_bank(t[j].h, t[j].w, G, rects, bank);
        vqnnf_status st = compile_bank(bank.data(), (int)bank.size(), t[j].h, t[j].w, b.bs[j], b.gs[j]);
        if (st != VQNNF_OK) return st;
        const bool u16 = sat_is_u16(t[j].h, t[j].w);
        if (score_smem_bytes_for(u16 ? 2 : 4, b.bs[j], b.gs[j], t[j].k) > (size_t)optin) return VQNNF_EUNSUPPORTED;
    }
    return VQNNF_OK;
}

// Template side: codebook, NNF and filter responses of every template.
// Template sides in up to kLanes lanes at once (template j in lane j % nl, each lane with its
// own fit workspace): one template's Lloyd steps are a chain of small dependent launches that
// leave most of the GPU idle.  The lanes fork from s and join it again before returning.
vqnnf_status fit_templates(const vqnnf_batch_template *t, int nt, int D, int iters, uint64_t seed, const Banks &b,
                           BatchWs &w, cudaStream_t s)
{
    LanePool *lp = nullptr;
    const int nl = lane_pool(lp) ? std::min(kLanes, nt) : 1;
    cudaError_t e = cudaSuccess;
    if (nl > 1) {
        e = cudaEventRecord(lp->fork, s);
        for (int l = 1; l < nl && e == cudaSuccess; ++l) e = cudaStreamWaitEvent(lp->st[l], lp->fork, 0);
        if (e != cudaSuccess) return from_cuda(e);
    }
    for (int j = 0; j < nt; ++j) {
        const int l = j % nl;
        const cudaStream_t ls = l ? lp->st[l] : s;
        const long long n = (long long)t[j].h * t[j].w;
        vqnnf_status st = run_fit(t[j].T, n, D, t[j].k, iters, seed + (uint64_t)j, VQNNF_PREC_BF16, w.C[j], w.fit[l], ls);
        if (st != VQNNF_OK) return st;
        st = run_assign(t[j].T, n, D, w.C[j], t[j].k, VQNNF_PREC_BF16, w.tlab[j], nullptr, w.fit[l].as, ls);
        if (st != VQNNF_OK) return st;
        e = launch_filter_responses(w.tlab[j], t[j].h, t[j].w, t[j].k, b.bs[j], w.tcnt[j], ls);
        if (e != cudaSuccess) return from_cuda(e);
    }
    for (int l = 1; l < nl; ++l) {
        e = cudaEventRecord(lp->join[l][0], lp->st[l]);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(s, lp->join[l][0], 0);
        if (e != cudaSuccess) return from_cuda(e);
    }
    return VQNNF_OK;
}

// Group codebooks and their prepared BF16 planes.
vqnnf_status build_groups(const std::vector<Group> &groups, const vqnnf_batch_template *t, int D, BatchWs &w,
                          cudaStream_t s)
{
    for (size_t g = 0; g < groups.size(); ++g) {
        const Group &G = groups[g];
        GroupSrc src;
        memset(&src, 0, sizeof(src));
        src.nseg = G.nseg;
        int col = 0;
        for (int q = 0; q < G.nseg; ++q) {
            const int j = G.tj[q];
            src.col0[q] = col;
            src.ncol[q] = (t[j].k + 31) / 32 * 32;
            src.k[q] = t[j].k;
            src.C[q] = w.C[j];
            col += src.ncol[q];
        }
        group_codebook_kernel<<<G.npad, 128, 0, s>>>(src, D, w.gC[g]);
        cudaError_t e = cudaGetLastError();
        if (e == cudaSuccess) e = launch_prep_codebook(w.gC[g], G.npad, D, VQNNF_PREC_BF16, w.gprep[g], s);
        if (e != cudaSuccess) return from_cuda(e);
    }
    return VQNNF_OK;
}

// NNF of query i under every template's codebook: one contraction per group, then the
// re-scoring of each codebook's flagged pixels.
vqnnf_status assign_query(const vqnnf_image &qi, const std::vector<Group> &groups, const vqnnf_batch_template *t,
                          int D, const vqnnf_batch_plan &plan, BatchWs &w, cudaStream_t s)
{
    const long long n = (long long)qi.H * qi.W;
    for (size_t g = 0; g < groups.size(); ++g) {
        const Group &G = groups[g];
        cudaError_t e = cudaMemsetAsync(w.flcount, 0, sizeof(unsigned) * 64 * kMaxSeg, s);
        if (e != cudaSuccess) return from_cuda(e);
        TcSeg seg[kMaxSeg];
        int col = 0;
        for (int q = 0; q < G.nseg; ++q) {
            const int j = G.tj[q];
            seg[q].col0 = col;
            seg[q].ncol = (t[j].k + 31) / 32 * 32;
            seg[q].k = t[j].k;
            seg[q].labels = w.qlab[j];
            seg[q].fl = w.fl[q];
            col += seg[q].ncol;
        }
        e = launch_assign_bf16_seg(qi.X, n, D, w.gprep[g], G.npad, seg, G.nseg, plan.sf, plan.pf, s);
        if (e != cudaSuccess) return from_cuda(e);
        for (int q = 0; q < G.nseg; ++q) {
            const int j = G.tj[q];
            e = launch_rescore(qi.X, n, D, w.C[j], t[j].k, w.qlab[j], w.fl[q], s);
            if (e != cudaSuccess) return from_cuda(e);
        }
    }
    return VQNNF_OK;
}

size_t batch_bytes(const vqnnf_image *q, int nq, const vqnnf_batch_template *t, int nt, int D, int G)
{
    WsCursor c{nullptr, 0};
    carve_batch(c, q, nq, t, nt, D, G);
    return (c.off + 255) & ~size_t(255);
}

}  // namespace

extern "C" {

size_t vqnnf_batch_workspace_bytes(const vqnnf_image *q, int nq, const vqnnf_batch_template *t, int nt, int D,
                                   int G)
{
    if (check_batch(q, nq, t, nt, D, G) != VQNNF_OK) return 0;
    return batch_bytes(q, nq, t, nt, D, G);
}

vqnnf_status vqnnf_match_batch(const vqnnf_image *q, int nq, const vqnnf_batch_template *t, int nt, int D,
                               int iters, uint64_t seed, int G, const vqnnf_batch_plan *plan,
                               float *const *heat, int32_t *argmax_yx, void *ws, size_t ws_bytes, void *stream)
{
    vqnnf_status st = check_batch(q, nq, t, nt, D, G);
    if (st != VQNNF_OK) return st;
    if (!argmax_yx || !ws || iters < 0 || !aligned(ws, 256)) return VQNNF_EINVAL;
    const vqnnf_batch_plan p = plan ? *plan : kDefaultPlan;
    if ((st = check_plan(p)) != VQNNF_OK) return st;
    if (heat)
        for (int e = 0; e < nq * nt; ++e)
            if (!heat[e]) return VQNNF_EINVAL;
    if (ws_bytes < batch_bytes(q, nq, t, nt, D, G)) return VQNNF_ENOMEM;
    Banks banks;
    if ((st = compile_banks(t, nt, G, banks)) != VQNNF_OK) return st;
    cudaStream_t s = as_stream(stream);
    std::lock_guard<std::recursive_mutex> lane_lock(g_lane_mu);
    WsCursor c{static_cast<char *>(ws), 0};
    BatchWs w = carve_batch(c, q, nq, t, nt, D, G);
    if ((st = fit_templates(t, nt, D, iters, seed, banks, w, s)) != VQNNF_OK) return st;
    const bool stat = p.stationary && stat_possible(D);
    std::vector<Group> groups;
    std::vector<StatLaunch> splan;
    if (stat) {
        splan = make_stat_plan(t, nt, D);
        if ((st = build_stat(splan, t, D, w, s)) != VQNNF_OK) return st;
    } else {
        groups = make_groups(t, nt, p.group_cols);
        if ((st = build_groups(groups, t, D, w, s)) != VQNNF_OK) return st;
    }
    WGridSpec no_wgrid;
    memset(&no_wgrid, 0, sizeof(no_wgrid));
    // Each query's pairs (integral image + score) run in kLanes lanes at once, pair j in lane
    // j % kLanes with the lane's own integral-image workspace: small pairs leave most of the GPU
    // idle one at a time.  The lanes are library streams; the caller's stream runs the query
    // assignments.  The labels alternate between two sets, so query i + 1's assignment runs
    // beside query i's pairs and only waits for query i - 1's pairs, the last readers of its
    // set.  Everything joins the caller's stream before the call returns.
    LanePool *lp = nullptr;
    const int nl = lane_pool(lp) ? std::min(kLanes, nt) : 0;
    cudaError_t e = cudaSuccess;
    for (int i = 0; i < nq; ++i) {
        const int par = i & 1;
        w.qlab = w.qset[par];
        if (nl && i >= 2)
            for (int l = 0; l < nl && e == cudaSuccess; ++l) e = cudaStreamWaitEvent(s, lp->join[l][par], 0);
        if (e != cudaSuccess) return from_cuda(e);
        st = stat ? assign_query_stat(q[i], splan, t, D, w, s) : assign_query(q[i], groups, t, D, p, w, s);
        if (st != VQNNF_OK) return st;
        if (nl) {
            e = cudaEventRecord(lp->fork, s);
            for (int l = 0; l < nl && e == cudaSuccess; ++l) e = cudaStreamWaitEvent(lp->st[l], lp->fork, 0);
            if (e != cudaSuccess) return from_cuda(e);
        }
        for (int j = 0; j < nt; ++j) {
            const int l = nl ? j % nl : 0;
            const cudaStream_t ls = nl ? lp->st[l] : s;
            WsCursor sc{w.score_base[l], 0};
            ScoreWs sw = carve_score(sc, q[i].H, q[i].W, t[j].k, t[j].h, t[j].w);
            e = launch_sat(w.qlab[j], q[i].H, q[i].W, t[j].k, sw.u16, sw.carry, sw.bandsum, sw.S, ls);
            if (e != cudaSuccess) return from_cuda(e);
            const int HO = q[i].H - t[j].h + 1, WO = q[i].W - t[j].w + 1;
            float *hp = heat ? heat[(size_t)i * nt + j] : w.heat_scratch[l];
            e = launch_score(sw.S, sw.u16, q[i].W, t[j].k, HO, WO, banks.bs[j], banks.gs[j], no_wgrid, w.tcnt[j], hp,
                             sw.amax, argmax_yx + 2 * ((size_t)i * nt + j), ls);
            if (e != cudaSuccess) return from_cuda(e);
        }
        for (int l = 0; l < nl && e == cudaSuccess; ++l) e = cudaEventRecord(lp->join[l][par], lp->st[l]);
        if (e != cudaSuccess) return from_cuda(e);
    }
    // join: each lane's last record follows all of its work
    for (int l = 0; l < nl && e == cudaSuccess; ++l) e = cudaStreamWaitEvent(s, lp->join[l][(nq - 1) & 1], 0);
    return from_cuda(e);
}

vqnnf_status vqnnf_batch_tune(const vqnnf_image *q, int nq, const vqnnf_batch_template *t, int nt, int D,
                              int iters, uint64_t seed, int G, vqnnf_batch_plan *plan, void *ws, size_t ws_bytes,
                              void *stream)
{
    vqnnf_status st = check_batch(q, nq, t, nt, D, G);
    if (st != VQNNF_OK) return st;
    if (!plan || !ws || iters < 0 || !aligned(ws, 256)) return VQNNF_EINVAL;
    if (ws_bytes < batch_bytes(q, nq, t, nt, D, G)) return VQNNF_ENOMEM;
    Banks banks;
    if ((st = compile_banks(t, nt, G, banks)) != VQNNF_OK) return st;
    cudaStream_t s = as_stream(stream);
    std::lock_guard<std::recursive_mutex> lane_lock(g_lane_mu);
    WsCursor c{static_cast<char *>(ws), 0};
    BatchWs w = carve_batch(c, q, nq, t, nt, D, G);
    if ((st = fit_templates(t, nt, D, iters, seed, banks, w, s)) != VQNNF_OK) return st;
    int ib = 0;
    for (int i = 1; i < nq; ++i)
        if ((long long)q[i].H * q[i].W > (long long)q[ib].H * q[ib].W) ib = i;
    cudaEvent_t e0, e1;
    if (cudaEventCreate(&e0) != cudaSuccess) return VQNNF_ECUDA;
    if (cudaEventCreate(&e1) != cudaSuccess) {
        cudaEventDestroy(e0);
        return VQNNF_ECUDA;
    }
    float best = 0.f;
    vqnnf_batch_plan best_plan = kDefaultPlan;
    // time one candidate: assignment of the largest query, second of two runs
    auto time_plan = [&](const vqnnf_batch_plan &cand, float &ms) -> vqnnf_status {
        const bool stat = cand.stationary && stat_possible(D);
        std::vector<Group> groups;
        std::vector<StatLaunch> splan;
        vqnnf_status r;
        if (stat) {
            splan = make_stat_plan(t, nt, D);
            r = build_stat(splan, t, D, w, s);
        } else {
            groups = make_groups(t, nt, cand.group_cols);
            r = build_groups(groups, t, D, w, s);
        }
        for (int rep = 0; rep < 2 && r == VQNNF_OK; ++rep) {
            if (cudaEventRecord(e0, s) != cudaSuccess) return VQNNF_ECUDA;
            r = stat ? assign_query_stat(q[ib], splan, t, D, w, s) : assign_query(q[ib], groups, t, D, cand, w, s);
            if (r != VQNNF_OK) return r;
            if (cudaEventRecord(e1, s) != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess ||
                cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess)
                return VQNNF_ECUDA;
        }
        return r;
    };
    if (stat_possible(D)) {
        const vqnnf_batch_plan cand = {256, 0, -1, 1};
        float ms = 0.f;
        st = time_plan(cand, ms);
        if (st == VQNNF_EUNSUPPORTED) st = VQNNF_OK;
        else if (st == VQNNF_OK) { best = ms; best_plan = cand; }
    }
    for (int gc : {128, 256}) {
        if (st != VQNNF_OK) break;
        for (int sf : {4, 6, 8}) {
            for (int pf : {0, 8}) {
                const vqnnf_batch_plan cand = {gc, sf, pf, 0};
                float ms = 0.f;
                st = time_plan(cand, ms);
                if (st == VQNNF_EUNSUPPORTED) {               // this split does not fit shared memory
                    st = VQNNF_OK;
                    continue;
                }
                if (st != VQNNF_OK) break;
                if (best == 0.f || ms < best) { best = ms; best_plan = cand; }
            }
            if (st != VQNNF_OK) break;
        }
        if (st != VQNNF_OK) break;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (st != VQNNF_OK) return st;
    *plan = best_plan;
    return VQNNF_OK;
}

}  // extern "C"
