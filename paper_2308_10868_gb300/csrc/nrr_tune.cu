// Execution-configuration autotuner for the match kernel.
//
// The paper tunes its GPU block-matching kernel by an empirical search over
// the thread configuration (Sec. 4.3, GADAPT), reporting ~30x between tuned
// and untuned.  Here the free parameters of a launch's shape are
//   - the search lines each thread owns (uint16 cubic blocks: one, or two
//     sharing each converted window row; which is faster depends on how the
//     line units fill the CTA's last warp),
//   - how many persistent CTAs share an SM (fewer leave more shared-memory
//     bandwidth and L1 to each; more hide more latency),
//   - the window buffers, i.e. blocks in flight per CTA (two: the next
//     block's copy overlaps this block's search; one: less shared memory,
//     more CTAs),
//   - whether each thread's box sums are staged into shared memory by
//     asynchronous copies during the search (no load latency at the bounds,
//     more shared memory) or loaded at the bounds.
// The tuner times every feasible shape on real inputs and keeps the fastest
// in a per-process table keyed by (device, dtype, block, radius); every
// later launch of that variant, single or batched, uses it.  The table can
// be saved to and loaded from a small text file.
#include <stdio.h>

#include <map>
#include <mutex>
#include <tuple>

#include "nrr_internal.h"

namespace nrr {

typedef std::tuple<int, int, int, int, int, int> TuneKey;  // device, dtype, block, rx, ry, rz
static std::mutex g_tune_mu;
static std::map<TuneKey, nrr_match_shape> g_tune;

static TuneKey make_key(nrr_dtype dtype, int block, const int32_t *r)
{
    int dev = 0;
    cudaGetDevice(&dev);
    return TuneKey(dev, (int)dtype, block, r[0], r[1], r[2]);
}

static nrr_match_shape tuned_shape(nrr_dtype dtype, int block, const int32_t *radius)
{
    std::lock_guard<std::mutex> lk(g_tune_mu);
    auto it = g_tune.find(make_key(dtype, block, radius));
    return it == g_tune.end() ? nrr_match_shape{0, 0, 0, 0} : it->second;
}

void apply_tuning(MatchLaunch &a, nrr_dtype dtype, int block, const int32_t *radius)
{
    const nrr_match_shape sh = tuned_shape(dtype, block, radius);
    a.ctas_per_sm = sh.ctas_per_sm;
    a.windows = sh.windows;
    a.stage_boxsums = sh.stage;
    a.lines = sh.lines;
}

static bool shape_ok(const nrr_match_shape &s)
{
    return s.ctas_per_sm >= 0 && s.ctas_per_sm <= 64 && s.windows >= 0 && s.windows <= 2 && s.stage >= 0 &&
           s.stage <= 2 && s.lines >= 0 && s.lines <= 2;
}

static void set_tuned(nrr_dtype dtype, int block, const int32_t *radius, const nrr_match_shape &v)
{
    std::lock_guard<std::mutex> lk(g_tune_mu);
    g_tune[make_key(dtype, block, radius)] = v;
}

}  // namespace nrr

using namespace nrr;

extern "C" {

nrr_status nrr_tuning_get(nrr_dtype dtype, int32_t block, const int32_t radius[3], int32_t *ctas_per_sm)
{
    clear_error();
    if (!radius || !ctas_per_sm) return fail(NRR_E_INVALID, "NULL argument");
    *ctas_per_sm = tuned_shape(dtype, block, radius).ctas_per_sm;
    return NRR_OK;
}

nrr_status nrr_tuning_set(nrr_dtype dtype, int32_t block, const int32_t radius[3], int32_t ctas_per_sm)
{
    clear_error();
    if (!radius || ctas_per_sm < 0 || ctas_per_sm > 64) return fail(NRR_E_INVALID, "bad tuning entry");
    set_tuned(dtype, block, radius, nrr_match_shape{ctas_per_sm, 0, 0, 0});
    return NRR_OK;
}

nrr_status nrr_tuning_get_shape(nrr_dtype dtype, int32_t block, const int32_t radius[3], nrr_match_shape *shape)
{
    clear_error();
    if (!radius || !shape) return fail(NRR_E_INVALID, "NULL argument");
    *shape = tuned_shape(dtype, block, radius);
    return NRR_OK;
}

nrr_status nrr_tuning_set_shape(nrr_dtype dtype, int32_t block, const int32_t radius[3], const nrr_match_shape *shape)
{
    clear_error();
    if (!radius || !shape || !shape_ok(*shape)) return fail(NRR_E_INVALID, "bad tuning entry");
    set_tuned(dtype, block, radius, *shape);
    return NRR_OK;
}

nrr_status nrr_tuning_save(const char *path)
{
    clear_error();
    FILE *f = path ? fopen(path, "w") : nullptr;
    if (!f) return fail(NRR_E_INVALID, "cannot open tuning file for writing");
    {
        std::lock_guard<std::mutex> lk(g_tune_mu);
        fprintf(f, "# device dtype block rx ry rz ctas_per_sm windows stage lines\n");
        for (auto &kv : g_tune)
            fprintf(f, "%d %d %d %d %d %d %d %d %d %d\n", std::get<0>(kv.first), std::get<1>(kv.first),
                    std::get<2>(kv.first), std::get<3>(kv.first), std::get<4>(kv.first), std::get<5>(kv.first),
                    kv.second.ctas_per_sm, kv.second.windows, kv.second.stage, kv.second.lines);
    }
    fclose(f);
    return NRR_OK;
}

nrr_status nrr_tuning_load(const char *path)
{
    clear_error();
    FILE *f = path ? fopen(path, "r") : nullptr;
    if (!f) return fail(NRR_E_NOTFOUND, "cannot open tuning file");
    char line[256];
    int n = 0;
    while (fgets(line, sizeof line, f)) {
        int d, t, b, x, y, z;
        nrr_match_shape v{0, 0, 0, 0};
        if (line[0] == '#') continue;
        // a line of 7 fields (ctas per SM only) or 9 (no lines per thread)
        // leaves the missing ones at their defaults
        const int k = sscanf(line, "%d %d %d %d %d %d %d %d %d %d", &d, &t, &b, &x, &y, &z, &v.ctas_per_sm,
                             &v.windows, &v.stage, &v.lines);
        if ((k == 7 || k == 9 || k == 10) && shape_ok(v)) {
            std::lock_guard<std::mutex> lk(g_tune_mu);
            g_tune[TuneKey(d, t, b, x, y, z)] = v;
            ++n;
        }
    }
    fclose(f);
    return NRR_OK;
}

nrr_status nrr_autotune_match(const void *d_preop, const void *d_intraop, const void *d_boxsums, nrr_dtype dtype,
                              nrr_dims dims, const int32_t *d_centers, int32_t n_blocks, int32_t block,
                              const int32_t radius[3], int32_t *d_disp, double *d_ncc, uint8_t *d_valid,
                              int32_t *best_ctas_per_sm, float *best_ms, void *stream)
{
    clear_error();
    nrr_status st = check_dims(dims, dtype, block);
    if (st != NRR_OK) return st;
    if (!d_preop || !d_intraop || !d_boxsums || !d_centers || !d_disp || !d_ncc || !d_valid || !radius || n_blocks < 1)
        return fail(NRR_E_INVALID, "NULL buffer or no blocks to tune on");
    for (int i = 0; i < 3; ++i)
        if (radius[i] < 0 || radius[i] > MATCH_MAX_R) return fail(NRR_E_INVALID, "radius[%d] outside 0..%d", i, MATCH_MAX_R);
    cudaStream_t s = (cudaStream_t)stream;
    MatchLaunch a{};
    a.preop = d_preop;
    a.intraop = d_intraop;
    a.s1 = d_boxsums;
    a.s2 = (const char *)d_boxsums + boxsum_s2_offset(dims, dtype);
    a.dtype = dtype;
    a.dims = dims;
    a.block = block;
    for (int i = 0; i < 3; ++i) a.radius[i] = radius[i];
    a.n_jobs = 1;
    a.jobs[0] = MatchJob{d_centers, nullptr, n_blocks, d_disp, d_ncc, d_valid};
    st = device_error_word(&a.err);
    if (st != NRR_OK) return st;
    cudaEvent_t e0, e1;
    NRR_CUDA_TRY(cudaEventCreate(&e0));
    NRR_CUDA_TRY(cudaEventCreate(&e1));
    nrr_match_shape best{0, 0, 0, 0};
    float best_t = 1e30f;
    // two lines per thread exist for uint16 cubic blocks only
    const int max_lines = dtype == NRR_U16 ? 2 : 1;
    for (int lines = 1; lines <= max_lines && st == NRR_OK; ++lines)
        for (int stage = 1; stage <= 2 && st == NRR_OK; ++stage)
            for (int windows = 2; windows >= 1 && st == NRR_OK; --windows) {
                a.lines = lines;
                a.stage_boxsums = stage;
                a.windows = windows;
                a.ctas_per_sm = 0;
                int occ = 0;
                st = match_occupancy(a, &occ);
                for (int k = occ; k >= 1 && st == NRR_OK; --k) {
                    a.ctas_per_sm = k;
                    st = launch_match(a, s);  // warm-up
                    float tot = 0.f;
                    for (int rep = 0; rep < 3 && st == NRR_OK; ++rep) {
                        cudaEventRecord(e0, s);
                        st = launch_match(a, s);
                        cudaEventRecord(e1, s);
                        if (cudaEventSynchronize(e1) != cudaSuccess) st = fail(NRR_E_CUDA, "event sync during tuning");
                        float ms = 0.f;
                        cudaEventElapsedTime(&ms, e0, e1);
                        tot += ms;
                    }
                    if (st == NRR_OK && tot / 3 < best_t) {
                        best_t = tot / 3;
                        best = nrr_match_shape{k, windows, stage, max_lines > 1 ? lines : 0};
                    }
                }
            }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (st != NRR_OK) return st;
    set_tuned(dtype, block, radius, best);
    if (best_ctas_per_sm) *best_ctas_per_sm = best.ctas_per_sm;
    if (best_ms) *best_ms = best_t;
    return NRR_OK;
}

}  // extern "C"
