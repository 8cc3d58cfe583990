// Batched parameter search: many (block size, search radius, selection
// fraction) settings of the registration, on one or many volume pairs of
// different sizes, run as one unit of GPU work.
//
// The paper runs such sweeps as separate registrations spread over grid or
// cloud resources (Sec. 4.2, speculative execution with many parameter
// values; Sec. 5, the parameter pool of the learned predictor).  On one GPU
// the same sweep becomes a plan built once and replayed:
//   - box sums of the reference volume, once per distinct block size;
//   - one selection per distinct (block, stride, fraction), each on its own
//     preallocated scratch;
//   - settings that share (block, stride, radius) and differ only in the
//     fraction select nested sets of blocks (a smaller fraction takes a
//     prefix of the same selection order), and a block's match does not
//     depend on the fraction: only the largest fraction's blocks are
//     matched, and every other setting of that unit gathers its blocks'
//     results from them;
//   - per (block, stride), a unit whose search box lies inside a matched
//     unit's box and whose fraction is not larger is not matched either: the
//     larger unit's job reports the best shift within the smaller box too
//     (an extra radius level of the same search), and its settings gather
//     from those results;
//   - one persistent match launch per distinct (block, radius), whose job
//     table holds the matched selection of every unit of that variant, of
//     every volume pair (up to 16 per launch; each job carries its pair's
//     volumes, box sums, sizes and tensor maps, so one launch mixes
//     registrations of different sizes);
//   - with NRR_BATCH_NO_DEDUP every setting is selected and matched on its
//     own (no shared selections' prefixes, no radius levels): the same
//     results, for measuring what the sharing saves;
//   - all of it forked over internal streams with event dependencies and
//     captured as a single CUDA graph, so a run is one graph launch with no
//     host round trip.
// Results stay on the device; every setting's count, centres, displacements,
// NCC and valid flags are reachable through nrr_batch_view_get.
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <map>
#include <tuple>
#include <vector>

#include "nrr_internal.h"

namespace nrr {

namespace {
constexpr int NSTREAMS = 8;

struct PairEntry {
    const uint16_t *preop, *intraop;
    const uint8_t *mask;
    nrr_dims dims;
};
struct SelEntry {
    int pair, box;  // its volume pair and box sums
    int block, stride;
    double frac;
    SelectPlan plan;
    unsigned char *ws;
    int32_t *centers;
    int32_t *d_n;
    int32_t cap;
    cudaEvent_t done;
};
struct BoxEntry {
    int pair;
    int block;
    void *buf;
    cudaEvent_t done;
};
struct LevelOut {  // an extra radius a matched setting's job reports
    int r[3];
    int32_t *disp;
    double *ncc;
    uint8_t *valid;
};
struct SettingOut {
    int sel;
    int src;  // setting whose job holds this one's results (itself if matched)
    int lvl;  // -1: src's own radius; else src's extra radius level
    int32_t *disp;
    double *ncc;
    uint8_t *valid;
    std::vector<LevelOut> levels;  // matched settings only
};

// Results of a nested selection from those of the larger one it is part of:
// both centre lists are in raster order, so each centre is found by binary
// search on its raster index.
__global__ void gather_nested_kernel(const int32_t *__restrict__ centers, const int32_t *__restrict__ d_n,
                                     int32_t cap, const int32_t *__restrict__ big_centers,
                                     const int32_t *__restrict__ big_n, int32_t big_cap, int nx, int ny,
                                     const int32_t *__restrict__ big_disp, const double *__restrict__ big_ncc,
                                     const uint8_t *__restrict__ big_valid, int32_t *__restrict__ disp,
                                     double *__restrict__ ncc, uint8_t *__restrict__ valid, unsigned int *err)
{
    const int n = *d_n < cap ? *d_n : cap;
    const int nb = *big_n < big_cap ? *big_n : big_cap;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const long long key = ((long long)centers[3 * i + 2] * ny + centers[3 * i + 1]) * nx + centers[3 * i];
        int lo = 0, hi = nb;  // first index whose raster key is >= key
        while (lo < hi) {
            const int mid = (lo + hi) >> 1;
            const long long mk =
                ((long long)big_centers[3 * mid + 2] * ny + big_centers[3 * mid + 1]) * nx + big_centers[3 * mid];
            if (mk < key) lo = mid + 1;
            else hi = mid;
        }
        if (lo < nb && big_centers[3 * lo] == centers[3 * i] && big_centers[3 * lo + 1] == centers[3 * i + 1] &&
            big_centers[3 * lo + 2] == centers[3 * i + 2]) {
            disp[3 * i + 0] = big_disp[3 * lo + 0];
            disp[3 * i + 1] = big_disp[3 * lo + 1];
            disp[3 * i + 2] = big_disp[3 * lo + 2];
            ncc[i] = big_ncc[lo];
            valid[i] = big_valid[lo];
        } else {  // cannot happen for nested selections; reported, never silent
            disp[3 * i + 0] = disp[3 * i + 1] = disp[3 * i + 2] = 0;
            ncc[i] = 0.0;
            valid[i] = 0;
            atomicOr(err, DEV_ERR_INTERNAL);
        }
    }
}
struct Group {
    int block;
    int radius[3];
    std::vector<int> settings;
    CUtensorMap *maps;  // device [pair][2]: window and floating-block maps of this variant
};
}  // namespace

}  // namespace nrr

struct nrr_batch_s {
    int device = 0;
    std::vector<nrr::PairEntry> pairs;
    std::vector<int> pair_of;  // per setting
    int flags = 0;
    int64_t graph_launches = 0;
    int32_t *queues = nullptr;  // a work-queue head (128 bytes apart) per match launch
    std::vector<nrr_setting> settings;
    std::vector<nrr::SelEntry> sels;
    std::vector<nrr::BoxEntry> boxes;
    std::vector<nrr::SettingOut> outs;
    std::vector<nrr::Group> groups;
    cudaStream_t streams[nrr::NSTREAMS] = {};
    cudaStream_t launch = nullptr;
    cudaEvent_t ev_in = nullptr, ev_out = nullptr, fork = nullptr, join[nrr::NSTREAMS] = {};
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    std::vector<void *> allocs;
    unsigned int *err = nullptr;
};

namespace nrr {

static nrr_status batch_alloc(nrr_batch_s *b, size_t bytes, void **p)
{
    cudaError_t e = cudaMalloc(p, bytes);
    if (e != cudaSuccess) return cuda_fail(e, "cudaMalloc (batch plan)");
    b->allocs.push_back(*p);
    return NRR_OK;
}

// Enqueue the whole sweep on the plan's streams, ordered after `in` and
// joined back into `out` (the same stream in practice).
static nrr_status batch_enqueue(nrr_batch_s *b, cudaStream_t s)
{
    NRR_CUDA_TRY(cudaEventRecord(b->fork, s));
    for (int k = 0; k < NSTREAMS; ++k) NRR_CUDA_TRY(cudaStreamWaitEvent(b->streams[k], b->fork, 0));
    int rr = 0, nq = 0;
    for (auto &bx : b->boxes) {
        cudaStream_t st = b->streams[rr++ % NSTREAMS];
        const PairEntry &pe = b->pairs[bx.pair];
        nrr_status r = launch_boxsums(pe.intraop, NRR_U16, pe.dims, bx.block, bx.buf, st);
        if (r != NRR_OK) return r;
        NRR_CUDA_TRY(cudaEventRecord(bx.done, st));
    }
    for (auto &se : b->sels) {
        cudaStream_t st = b->streams[rr++ % NSTREAMS];
        const PairEntry &pe = b->pairs[se.pair];
        nrr_status r = enqueue_select(pe.preop, pe.mask, pe.dims, se.block, se.stride, se.frac, se.centers, se.cap,
                                      se.d_n, se.ws, se.plan, st);
        if (r != NRR_OK) return r;
        NRR_CUDA_TRY(cudaEventRecord(se.done, st));
    }
    // match launches, largest groups first so they start early
    std::vector<int> order(b->groups.size());
    for (size_t i = 0; i < order.size(); ++i) order[i] = (int)i;
    std::sort(order.begin(), order.end(), [&](int x, int y) {
        auto work = [&](int g) {
            const Group &G = b->groups[g];
            long long w = 0;
            for (int s_ : G.settings)
                if (b->outs[s_].src == s_) w += (long long)b->sels[b->outs[s_].sel].cap;
            return w * (2 * G.radius[0] + 1) * (2 * G.radius[1] + 1) * (2 * G.radius[2] + 1) * G.block * G.block *
                   G.block;
        };
        return work(x) > work(y);
    });
    for (int gi : order) {
        const Group &G = b->groups[gi];
        std::vector<int> matched;
        for (int s_ : G.settings)
            if (b->outs[s_].src == s_) matched.push_back(s_);
        cudaStream_t st = b->streams[rr++ % NSTREAMS];  // the group's launches, then its gathers
        for (size_t c0 = 0; c0 < matched.size(); c0 += MATCH_MAX_JOBS) {
            MatchLaunch a{};
            a.dtype = NRR_U16;
            a.block = G.block;
            for (int i = 0; i < 3; ++i) a.radius[i] = G.radius[i];
            a.err = b->err;
            apply_tuning(a, NRR_U16, G.block, G.radius);
            a.queue = b->queues + 32 * nq++;  // at most one launch per setting
            if (b->flags & NRR_BATCH_PLAIN_LAUNCH) {
                a.one_cta_per_block = 1;
                a.ctas_per_sm = 0;
            }
            for (size_t c = c0; c < matched.size() && c < c0 + MATCH_MAX_JOBS; ++c) {
                const SettingOut &o = b->outs[matched[c]];
                const SelEntry &se = b->sels[o.sel];
                const PairEntry &pe = b->pairs[se.pair];
                const BoxEntry *bx = &b->boxes[se.box];
                NRR_CUDA_TRY(cudaStreamWaitEvent(st, bx->done, 0));
                NRR_CUDA_TRY(cudaStreamWaitEvent(st, se.done, 0));
                MatchJob jb{se.centers, se.d_n, se.cap, o.disp, o.ncc, o.valid};
                jb.n_levels = (int32_t)o.levels.size();
                for (size_t l = 0; l < o.levels.size(); ++l)
                    jb.levels[l] = MatchLevel{{o.levels[l].r[0], o.levels[l].r[1], o.levels[l].r[2]}, o.levels[l].disp,
                                              o.levels[l].ncc, o.levels[l].valid};
                // this job's pair: volumes, box sums, sizes, tensor maps
                jb.preop = pe.preop;
                jb.intraop = pe.intraop;
                jb.s1 = bx->buf;
                jb.s2 = (const char *)bx->buf + boxsum_s2_offset(pe.dims, NRR_U16);
                jb.nx = pe.dims.nx;
                jb.ny = pe.dims.ny;
                jb.nz = pe.dims.nz;
                jb.mapJ = G.maps + 2 * se.pair;
                jb.mapI = G.maps + 2 * se.pair + 1;
                if (a.n_jobs == 0) {  // the launch's own maps: the first job's pair
                    a.preop = pe.preop;
                    a.intraop = pe.intraop;
                    a.s1 = jb.s1;
                    a.s2 = jb.s2;
                    a.dims = pe.dims;
                }
                a.jobs[a.n_jobs++] = jb;
            }
            nrr_status r = launch_match(a, st);
            if (r != NRR_OK) return r;
        }
        // settings served by this group's jobs: gathered after the launches
        for (size_t s_ = 0; s_ < b->outs.size(); ++s_) {
            const SettingOut &o = b->outs[s_];
            if (o.src == (int)s_ || std::find(matched.begin(), matched.end(), o.src) == matched.end()) continue;
            const SettingOut &m = b->outs[o.src];
            const SelEntry &se = b->sels[o.sel], &sm = b->sels[m.sel];
            const int32_t *md = o.lvl < 0 ? m.disp : m.levels[o.lvl].disp;
            const double *mn = o.lvl < 0 ? m.ncc : m.levels[o.lvl].ncc;
            const uint8_t *mv = o.lvl < 0 ? m.valid : m.levels[o.lvl].valid;
            NRR_CUDA_TRY(cudaStreamWaitEvent(st, se.done, 0));
            const int grid = (se.cap + 255) / 256;
            const nrr_dims &dd = b->pairs[se.pair].dims;
            gather_nested_kernel<<<grid < 1 ? 1 : grid, 256, 0, st>>>(
                se.centers, se.d_n, se.cap, sm.centers, sm.d_n, sm.cap, dd.nx, dd.ny, md, mn, mv, o.disp,
                o.ncc, o.valid, b->err);
            NRR_CUDA_TRY(cudaGetLastError());
            count_launches(1);
        }
    }
    for (int k = 0; k < NSTREAMS; ++k) {
        NRR_CUDA_TRY(cudaEventRecord(b->join[k], b->streams[k]));
        NRR_CUDA_TRY(cudaStreamWaitEvent(s, b->join[k], 0));
    }
    return NRR_OK;
}

static void batch_free(nrr_batch_s *b)
{
    if (b->exec) cudaGraphExecDestroy(b->exec);
    if (b->graph) cudaGraphDestroy(b->graph);
    for (auto &e : b->sels)
        if (e.done) cudaEventDestroy(e.done);
    for (auto &e : b->boxes)
        if (e.done) cudaEventDestroy(e.done);
    for (int k = 0; k < NSTREAMS; ++k) {
        if (b->join[k]) cudaEventDestroy(b->join[k]);
        if (b->streams[k]) cudaStreamDestroy(b->streams[k]);
    }
    if (b->fork) cudaEventDestroy(b->fork);
    if (b->ev_in) cudaEventDestroy(b->ev_in);
    if (b->ev_out) cudaEventDestroy(b->ev_out);
    if (b->launch) cudaStreamDestroy(b->launch);
    for (void *p : b->allocs) cudaFree(p);
    delete b;
}

}  // namespace nrr

using namespace nrr;

extern "C" {

nrr_status nrr_batch_create_pairs(const nrr_pair *pairs, int32_t n_pairs, const nrr_setting *settings,
                                  const int32_t *pair_of, int32_t n_settings, int32_t flags, nrr_batch *out)
{
    clear_error();
    if (!out) return fail(NRR_E_INVALID, "out is NULL");
    *out = nullptr;
    if (!pairs || n_pairs < 1 || !settings || n_settings < 1)
        return fail(NRR_E_INVALID, "NULL pairs/settings, no pairs or no settings");
    for (int p = 0; p < n_pairs; ++p) {
        const nrr_pair &pe = pairs[p];
        if (!pe.d_preop || !pe.d_intraop || !pe.d_mask) return fail(NRR_E_INVALID, "pair %d: NULL volume or mask", p);
        if (((uintptr_t)pe.d_preop & 15u) || ((uintptr_t)pe.d_intraop & 15u))
            return fail(NRR_E_INVALID, "pair %d: volumes must be 16-byte aligned", p);
    }
    for (int i = 0; i < n_settings; ++i) {
        const nrr_setting &s = settings[i];
        const int pi = pair_of ? pair_of[i] : 0;
        if (pi < 0 || pi >= n_pairs) return fail(NRR_E_INVALID, "setting %d: pair index %d outside 0..%d", i, pi, n_pairs - 1);
        nrr_status st = check_select_args(pairs[pi].dims, s.block, s.stride, s.frac);
        if (st != NRR_OK) {
            char why[256];
            snprintf(why, sizeof why, "%s", nrr_last_error());
            return fail(st, "setting %d: %s", i, why);
        }
        for (int k = 0; k < 3; ++k)
            if (s.radius[k] < 0 || s.radius[k] > MATCH_MAX_R)
                return fail(NRR_E_INVALID, "setting %d: radius outside 0..%d", i, MATCH_MAX_R);
    }
    const bool dedup = !(flags & NRR_BATCH_NO_DEDUP);
    nrr_batch_s *b = new nrr_batch_s();
    for (int p = 0; p < n_pairs; ++p)
        b->pairs.push_back(PairEntry{pairs[p].d_preop, pairs[p].d_intraop, pairs[p].d_mask, pairs[p].dims});
    for (int i = 0; i < n_settings; ++i) b->pair_of.push_back(pair_of ? pair_of[i] : 0);
    b->flags = flags;
    b->settings.assign(settings, settings + n_settings);
    cudaGetDevice(&b->device);
    nrr_status st = device_error_word(&b->err);
    auto bail = [&](nrr_status r) {
        batch_free(b);
        return r;
    };
    if (st != NRR_OK) return bail(st);
    // distinct box sums, selections and match variants; without dedup every
    // setting gets its own box sums, selection and match (uniq = its index)
    std::map<std::tuple<int, int, int>, int> box_of;
    std::map<std::tuple<int, int, int, double, int>, int> sel_of;
    std::map<std::tuple<int, int, int, int>, int> grp_of;
    for (int i = 0; i < n_settings; ++i) {
        const nrr_setting &s = settings[i];
        const int pi = b->pair_of[i], uniq = dedup ? -1 : i;
        const nrr_dims dims = b->pairs[pi].dims;
        auto bk = std::make_tuple(pi, s.block, uniq);
        if (!box_of.count(bk)) {
            box_of[bk] = (int)b->boxes.size();
            BoxEntry e{pi, s.block, nullptr, nullptr};
            if ((st = batch_alloc(b, boxsum_bytes(dims, NRR_U16), &e.buf)) != NRR_OK) return bail(st);
            if (cudaEventCreateWithFlags(&e.done, cudaEventDisableTiming) != cudaSuccess)
                return bail(fail(NRR_E_CUDA, "event"));
            b->boxes.push_back(e);
        }
        auto sk = std::make_tuple(pi, s.block, s.stride, s.frac, uniq);
        if (!sel_of.count(sk)) {
            sel_of[sk] = (int)b->sels.size();
            SelEntry e{};
            e.pair = pi;
            e.box = box_of[bk];
            e.block = s.block;
            e.stride = s.stride;
            e.frac = s.frac;
            e.plan = select_plan(dims, s.stride);
            const long long ng = e.plan.ng;
            long long cap = (long long)(0.5 + (double)ng * s.frac) + 1;
            if (cap > ng) cap = ng;
            e.cap = (int32_t)(cap < 1 ? 1 : cap);
            void *p;
            if ((st = batch_alloc(b, e.plan.bytes, &p)) != NRR_OK) return bail(st);
            e.ws = (unsigned char *)p;
            if ((st = batch_alloc(b, sizeof(int32_t) * 3 * (size_t)e.cap, &p)) != NRR_OK) return bail(st);
            e.centers = (int32_t *)p;
            if ((st = batch_alloc(b, 256, &p)) != NRR_OK) return bail(st);
            e.d_n = (int32_t *)p;
            if (cudaEventCreateWithFlags(&e.done, cudaEventDisableTiming) != cudaSuccess)
                return bail(fail(NRR_E_CUDA, "event"));
            b->sels.push_back(e);
        }
        SettingOut o{};
        o.sel = sel_of[sk];
        const int32_t cap = b->sels[o.sel].cap;
        void *p;
        if ((st = batch_alloc(b, (size_t)cap * (12 + 8 + 1) + 512, &p)) != NRR_OK) return bail(st);
        o.ncc = (double *)p;
        o.disp = (int32_t *)((char *)p + align_up((size_t)cap * 8, 256));
        o.valid = (uint8_t *)((char *)o.disp + align_up((size_t)cap * 12, 256));
        b->outs.push_back(o);
        auto gk = std::make_tuple(s.block, s.radius[0], s.radius[1], s.radius[2]);
        if (!grp_of.count(gk)) {
            grp_of[gk] = (int)b->groups.size();
            Group g;
            g.block = s.block;
            for (int k = 0; k < 3; ++k) g.radius[k] = s.radius[k];
            g.maps = nullptr;
            b->groups.push_back(g);
        }
        b->groups[grp_of[gk]].settings.push_back(i);
    }
    {
        void *p;
        if ((st = batch_alloc(b, 128 * (size_t)n_settings, &p)) != NRR_OK) return bail(st);
        b->queues = (int32_t *)p;
    }
    // each match variant's tensor maps for every pair (window and
    // floating-block boxes of that variant), encoded here once and kept on
    // the device: the jobs of one launch read them from there
    for (auto &G : b->groups) {
        std::vector<CUtensorMap> maps(2 * (size_t)n_pairs);
        memset(maps.data(), 0, maps.size() * sizeof(CUtensorMap));
        int wb[3], tb[3];
        match_boxes(NRR_U16, G.block, G.block, G.block, G.radius, wb, tb);
        for (int pi = 0; pi < n_pairs; ++pi) {
            bool used = false;
            for (int s_ : G.settings) used |= b->pair_of[s_] == pi;
            if (!used) continue;
            const PairEntry &pe = b->pairs[pi];
            if ((st = encode_volume_map(&maps[2 * pi], pe.intraop, NRR_U16, pe.dims, wb[0], wb[1], wb[2])) != NRR_OK ||
                (st = encode_volume_map(&maps[2 * pi + 1], pe.preop, NRR_U16, pe.dims, tb[0], tb[1], tb[2])) != NRR_OK)
                return bail(st);
        }
        void *p;
        if ((st = batch_alloc(b, maps.size() * sizeof(CUtensorMap), &p)) != NRR_OK) return bail(st);
        if (cudaMemcpy(p, maps.data(), maps.size() * sizeof(CUtensorMap), cudaMemcpyHostToDevice) != cudaSuccess)
            return bail(fail(NRR_E_CUDA, "tensor map copy"));
        G.maps = (CUtensorMap *)p;
    }
    // per (pair, block, stride, radius): the setting with the largest
    // fraction is matched, the others gather from it (their selections are
    // nested in it)
    std::map<std::tuple<int, int, int, int, int, int, int>, int> unit_of;
    auto unit_key = [&](int i) {
        const nrr_setting &s = settings[i];
        return std::make_tuple(b->pair_of[i], s.block, s.stride, s.radius[0], s.radius[1], s.radius[2],
                               dedup ? -1 : i);
    };
    for (int i = 0; i < n_settings; ++i) {
        auto uk = unit_key(i);
        auto it = unit_of.find(uk);
        if (it == unit_of.end() || settings[it->second].frac < settings[i].frac) unit_of[uk] = i;
    }
    // per (pair, block, stride): a unit whose radius box lies in a matched
    // unit's box and whose fraction is not larger is served by that unit's
    // job as an extra radius level (its blocks are among the larger unit's,
    // and the search over the larger box contains the smaller one); units
    // are taken largest box first
    std::vector<int> prim;
    for (auto &kv : unit_of) prim.push_back(kv.second);
    auto vol = [&](int i) {
        const nrr_setting &s = settings[i];
        return (2 * s.radius[0] + 1) * (2 * s.radius[1] + 1) * (2 * s.radius[2] + 1);
    };
    std::sort(prim.begin(), prim.end(), [&](int x, int y) {
        if (vol(x) != vol(y)) return vol(x) > vol(y);
        if (settings[x].frac != settings[y].frac) return settings[x].frac > settings[y].frac;
        return x < y;
    });
    std::map<int, std::pair<int, int>> served;  // unit primary -> (matched primary, level)
    std::vector<int> launched;
    for (int u : prim) {
        const nrr_setting &su = settings[u];
        int host = -1;
        for (int a_ : launched) {
            const nrr_setting &sa = settings[a_];
            // a search answers smaller boxes only while one window holds it
            const bool one_window = sa.radius[0] <= MATCH_WINDOW_R && sa.radius[1] <= MATCH_WINDOW_R &&
                                    sa.radius[2] <= MATCH_WINDOW_R;
            if (dedup && one_window && b->pair_of[a_] == b->pair_of[u] && sa.block == su.block &&
                sa.stride == su.stride && sa.frac >= su.frac && sa.radius[0] >= su.radius[0] &&
                sa.radius[1] >= su.radius[1] && sa.radius[2] >= su.radius[2] &&
                (int)b->outs[a_].levels.size() < MATCH_MAX_LEVELS) {
                host = a_;
                break;
            }
        }
        if (host < 0) {
            launched.push_back(u);
            continue;
        }
        LevelOut lv{};
        for (int k = 0; k < 3; ++k) lv.r[k] = su.radius[k];
        const int32_t hcap = b->sels[b->outs[host].sel].cap;
        void *p;
        if ((st = batch_alloc(b, (size_t)hcap * (12 + 8 + 1) + 512, &p)) != NRR_OK) return bail(st);
        lv.ncc = (double *)p;
        lv.disp = (int32_t *)((char *)p + align_up((size_t)hcap * 8, 256));
        lv.valid = (uint8_t *)((char *)lv.disp + align_up((size_t)hcap * 12, 256));
        b->outs[host].levels.push_back(lv);
        served[u] = std::make_pair(host, (int)b->outs[host].levels.size() - 1);
    }
    for (int i = 0; i < n_settings; ++i) {
        const int u = unit_of[unit_key(i)];
        auto it = served.find(u);
        b->outs[i].src = it == served.end() ? u : it->second.first;
        b->outs[i].lvl = it == served.end() ? -1 : it->second.second;
    }
    for (int k = 0; k < NSTREAMS; ++k) {
        if (cudaStreamCreateWithFlags(&b->streams[k], cudaStreamNonBlocking) != cudaSuccess ||
            cudaEventCreateWithFlags(&b->join[k], cudaEventDisableTiming) != cudaSuccess)
            return bail(fail(NRR_E_CUDA, "stream/event creation"));
    }
    if (cudaStreamCreateWithFlags(&b->launch, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&b->fork, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&b->ev_in, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&b->ev_out, cudaEventDisableTiming) != cudaSuccess)
        return bail(fail(NRR_E_CUDA, "stream/event creation"));

    if (flags & NRR_BATCH_AUTOTUNE) {
        // one eager run for real inputs, then tune every match variant on its
        // largest setting
        if ((st = batch_enqueue(b, b->launch)) != NRR_OK) return bail(st);
        if (cudaStreamSynchronize(b->launch) != cudaSuccess) return bail(fail(NRR_E_CUDA, "sync"));
        for (auto &G : b->groups) {
            int best_s = G.settings[0];
            for (int s_ : G.settings)
                if (b->sels[b->outs[s_].sel].cap > b->sels[b->outs[best_s].sel].cap) best_s = s_;
            const SettingOut &o = b->outs[best_s];
            const SelEntry &se = b->sels[o.sel];
            int32_t n = 0;
            if (cudaMemcpy(&n, se.d_n, sizeof(n), cudaMemcpyDeviceToHost) != cudaSuccess)
                return bail(fail(NRR_E_CUDA, "count copy"));
            if (n < 1) continue;
            const PairEntry &pe = b->pairs[se.pair];
            st = nrr_autotune_match(pe.preop, pe.intraop, b->boxes[se.box].buf, NRR_U16, pe.dims, se.centers, n,
                                    G.block, G.radius, o.disp, o.ncc, o.valid, nullptr, nullptr, b->launch);
            if (st != NRR_OK) return bail(st);
        }
    }
    if (flags & NRR_BATCH_GRAPH) {
        if (cudaStreamBeginCapture(b->launch, cudaStreamCaptureModeRelaxed) != cudaSuccess)
            return bail(fail(NRR_E_CUDA, "cudaStreamBeginCapture"));
        const int64_t before = nrr_kernel_launches();
        st = batch_enqueue(b, b->launch);
        b->graph_launches = nrr_kernel_launches() - before;  // kernels one replay runs
        cudaGraph_t g = nullptr;
        cudaError_t e = cudaStreamEndCapture(b->launch, &g);
        if (st != NRR_OK) {
            if (g) cudaGraphDestroy(g);
            return bail(st);
        }
        if (e != cudaSuccess) return bail(cuda_fail(e, "cudaStreamEndCapture"));
        b->graph = g;
        e = cudaGraphInstantiate(&b->exec, g, 0);
        if (e != cudaSuccess) return bail(cuda_fail(e, "cudaGraphInstantiate"));
    }
    *out = b;
    return NRR_OK;
}

nrr_status nrr_batch_create(const uint16_t *d_preop, const uint16_t *d_intraop, const uint8_t *d_mask, nrr_dims dims,
                            const nrr_setting *settings, int32_t n_settings, int32_t flags, nrr_batch *out)
{
    const nrr_pair one{d_preop, d_intraop, d_mask, dims};
    return nrr_batch_create_pairs(&one, 1, settings, nullptr, n_settings, flags, out);
}

nrr_status nrr_batch_run(nrr_batch b, void *stream)
{
    clear_error();
    if (!b) return fail(NRR_E_INVALID, "NULL plan");
    cudaStream_t s = (cudaStream_t)stream;
    NRR_CUDA_TRY(cudaEventRecord(b->ev_in, s));
    NRR_CUDA_TRY(cudaStreamWaitEvent(b->launch, b->ev_in, 0));
    if (b->exec) {
        NRR_CUDA_TRY(cudaGraphLaunch(b->exec, b->launch));
        count_launches((int)b->graph_launches);
    } else {
        nrr_status st = batch_enqueue(b, b->launch);
        if (st != NRR_OK) return st;
    }
    NRR_CUDA_TRY(cudaEventRecord(b->ev_out, b->launch));
    NRR_CUDA_TRY(cudaStreamWaitEvent(s, b->ev_out, 0));
    return NRR_OK;
}

nrr_status nrr_batch_view_get(nrr_batch b, int32_t setting, nrr_batch_view *view)
{
    clear_error();
    if (!b || !view || setting < 0 || setting >= (int32_t)b->outs.size())
        return fail(NRR_E_INVALID, "bad plan, setting index or view");
    const SettingOut &o = b->outs[setting];
    const SelEntry &se = b->sels[o.sel];
    view->centers = se.centers;
    view->n_blocks = se.d_n;
    view->disp = o.disp;
    view->ncc = o.ncc;
    view->valid = o.valid;
    view->capacity = se.cap;
    return NRR_OK;
}

nrr_status nrr_batch_destroy(nrr_batch b)
{
    clear_error();
    if (!b) return NRR_OK;
    cudaStreamSynchronize(b->launch);
    batch_free(b);
    return NRR_OK;
}

}  // extern "C"
