// Chooses the match-kernel variant for a call's element type and block size.
#include "nrr_match.cuh"

namespace nrr {

nrr_status launch_match(const MatchLaunch &m, cudaStream_t stream)
{
    const bool f = m.dtype == NRR_F32;
    switch (m.block) {
    case 3: return f ? launch_match_f32_b3(m, stream) : launch_match_u16_b3(m, stream);
    case 5: return f ? launch_match_f32_b5(m, stream) : launch_match_u16_b5(m, stream);
    case 7: return f ? launch_match_f32_b7(m, stream) : launch_match_u16_b7(m, stream);
    case 9: return f ? launch_match_f32_b9(m, stream) : launch_match_u16_b9(m, stream);
    case 11: return f ? launch_match_f32_b11(m, stream) : launch_match_u16_b11(m, stream);
    }
    return fail(NRR_E_INVALID, "block %d not supported", m.block);
}

}  // namespace nrr
