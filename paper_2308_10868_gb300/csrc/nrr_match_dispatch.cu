// Chooses the match-kernel variant for a call's element type, block size and
// search lines per thread.
#include "nrr_match.cuh"

namespace nrr {

static nrr_status dispatch(const MatchLaunch &m, cudaStream_t stream, int *occ)
{
    if (m.dtype == NRR_F32) {
        switch (m.block) {
        case 3: return launch_match_f32_b3(m, stream, occ);
        case 5: return launch_match_f32_b5(m, stream, occ);
        case 7: return launch_match_f32_b7(m, stream, occ);
        case 9: return launch_match_f32_b9(m, stream, occ);
        case 11: return launch_match_f32_b11(m, stream, occ);
        }
        return fail(NRR_E_INVALID, "block %d not supported", m.block);
    }
    const bool two = match_lines(m) == 2;
    switch (m.block) {
#define NRR_U16(b) \
    case b: return two ? launch_match_u16_b##b##_l2(m, stream, occ) : launch_match_u16_b##b##_l1(m, stream, occ);
        NRR_U16(3)
        NRR_U16(5)
        NRR_U16(7)
        NRR_U16(9)
        NRR_U16(11)
#undef NRR_U16
    }
    return fail(NRR_E_INVALID, "block %d not supported", m.block);
}

void plan_subwindows(int R, int *r, int *k, int *off)
{
    const int n = 2 * R + 1;
    int kk = (n + 2 * MATCH_WINDOW_R) / (2 * MATCH_WINDOW_R + 1);  // ceil(n / 15)
    if (kk < 1) kk = 1;
    int len = (n + kk - 1) / kk;
    if (!(len & 1)) ++len;
    const int rr = (len - 1) / 2;
    for (int i = 0; i < kk; ++i) {
        int o = -R + rr + i * len;
        if (o > R - rr) o = R - rr;
        off[i] = o;
    }
    *r = rr;
    *k = kk;
}

void match_boxes(nrr_dtype dtype, int block, int by, int bz, const int32_t radius[3], int wbox[3], int tbox[3])
{
    int r[3], k, off[MATCH_MAX_SUB];
    for (int a = 0; a < 3; ++a) plan_subwindows(radius[a], &r[a], &k, off);
    const int es = (int)elem_size(dtype), epc = 16 / es;
    const int P = 2 * r[0] + 1, py = 2 * r[1] + 1;
    int c = (block + P - 1 + 2 * epc - 2) / epc;  // as match_bx: chunks, made odd
    if (!(c & 1)) ++c;
    wbox[0] = epc * c;
    wbox[1] = match_wyp(by + 2 * r[1], py);
    wbox[2] = bz + 2 * r[2];
    tbox[0] = round_up_i(block + epc - 1, epc);
    tbox[1] = by;
    tbox[2] = bz;
}

static nrr_status with_subwindows(const MatchLaunch &m0, MatchLaunch &m)
{
    m = m0;
    for (int a = 0; a < 3; ++a) {
        if (m.radius[a] < 0 || m.radius[a] > MATCH_MAX_R)
            return fail(NRR_E_INVALID, "radius[%d]=%d outside 0..%d", a, m.radius[a], MATCH_MAX_R);
        plan_subwindows(m.radius[a], &m.sub_r[a], &m.nsub[a], m.soff[a]);
        if (m.nsub[a] > MATCH_MAX_SUB) return fail(NRR_E_INTERNAL, "too many sub-windows");
    }
    if (m.nsub[0] * m.nsub[1] * m.nsub[2] > 1)
        for (int j = 0; j < m.n_jobs; ++j)
            if (m.jobs[j].n_levels > 0)
                return fail(NRR_E_INVALID, "extra radius levels need a radius of at most %d per axis", MATCH_WINDOW_R);
    return NRR_OK;
}

nrr_status launch_match(const MatchLaunch &m0, cudaStream_t stream)
{
    if (m0.n_jobs < 1 || m0.n_jobs > MATCH_MAX_JOBS) return fail(NRR_E_INVALID, "1..%d jobs per launch", MATCH_MAX_JOBS);
    MatchLaunch m;
    nrr_status st = with_subwindows(m0, m);
    if (st != NRR_OK) return st;
    return dispatch(m, stream, nullptr);
}

nrr_status match_occupancy(const MatchLaunch &m0, int *ctas_per_sm)
{
    MatchLaunch m;
    nrr_status st = with_subwindows(m0, m);
    if (st != NRR_OK) return st;
    return dispatch(m, nullptr, ctas_per_sm);
}

}  // namespace nrr
