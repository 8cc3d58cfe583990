// Chooses the match-kernel variant for a call's element type and block size.
#include "nrr_match.cuh"

namespace nrr {

static nrr_status dispatch(const MatchLaunch &m, cudaStream_t stream, int *occ)
{
    const bool f = m.dtype == NRR_F32;
    switch (m.block) {
    case 3: return f ? launch_match_f32_b3(m, stream, occ) : launch_match_u16_b3(m, stream, occ);
    case 5: return f ? launch_match_f32_b5(m, stream, occ) : launch_match_u16_b5(m, stream, occ);
    case 7: return f ? launch_match_f32_b7(m, stream, occ) : launch_match_u16_b7(m, stream, occ);
    case 9: return f ? launch_match_f32_b9(m, stream, occ) : launch_match_u16_b9(m, stream, occ);
    case 11: return f ? launch_match_f32_b11(m, stream, occ) : launch_match_u16_b11(m, stream, occ);
    }
    return fail(NRR_E_INVALID, "block %d not supported", m.block);
}

nrr_status launch_match(const MatchLaunch &m, cudaStream_t stream)
{
    if (m.n_jobs < 1 || m.n_jobs > MATCH_MAX_JOBS) return fail(NRR_E_INVALID, "1..%d jobs per launch", MATCH_MAX_JOBS);
    return dispatch(m, stream, nullptr);
}

nrr_status match_occupancy(const MatchLaunch &m, int *ctas_per_sm) { return dispatch(m, nullptr, ctas_per_sm); }

}  // namespace nrr
