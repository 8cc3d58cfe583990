// Instantiates the match kernel for one (element type, block size) pair.
// The build compiles this file once per pair with NRR_INST_F32 (0 or 1) and
// NRR_INST_B (3, 5, 7, 9 or 11) defined, so the variants compile in
// parallel.
#include "nrr_match.cuh"

#if !defined(NRR_INST_F32) || !defined(NRR_INST_B)
#error "define NRR_INST_F32 and NRR_INST_B"
#endif

#define NRR_CAT3(a, b, c) a##b##c
#define NRR_NAME(t, b) NRR_CAT3(launch_match_, t, b)
#if NRR_INST_F32
#define NRR_T float
#define NRR_FN NRR_NAME(f32_b, NRR_INST_B)
#else
#define NRR_T uint16_t
#define NRR_FN NRR_NAME(u16_b, NRR_INST_B)
#endif

namespace nrr {
nrr_status NRR_FN(const MatchLaunch &m, cudaStream_t stream, int *occ)
{
    return launch_match_b<NRR_T, NRR_INST_B>(m, stream, occ);
}
}  // namespace nrr
