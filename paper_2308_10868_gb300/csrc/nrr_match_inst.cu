// Instantiates the match kernel for one (element type, block size, lines per
// thread) triple.  The build compiles this file once per triple with
// NRR_INST_F32 (0 or 1), NRR_INST_B (3, 5, 7, 9 or 11) and, for uint16,
// NRR_INST_LPT (1 or 2) defined, so the variants compile in parallel.
#include "nrr_match.cuh"

#if !defined(NRR_INST_F32) || !defined(NRR_INST_B)
#error "define NRR_INST_F32 and NRR_INST_B"
#endif

#define NRR_CAT3(a, b, c) a##b##c
#define NRR_CAT4(a, b, c, d) a##b##c##d
#if NRR_INST_F32
#define NRR_T float
#define NRR_LPT 1
#define NRR_FN_(b) NRR_CAT3(launch_match_, f32_b, b)
#define NRR_FN NRR_FN_(NRR_INST_B)
#else
#if !defined(NRR_INST_LPT) || (NRR_INST_LPT != 1 && NRR_INST_LPT != 2)
#error "define NRR_INST_LPT as 1 or 2 for uint16 variants"
#endif
#define NRR_T uint16_t
#define NRR_LPT NRR_INST_LPT
#define NRR_FN_(b, l) NRR_CAT4(launch_match_u16_b, b, _l, l)
#define NRR_FN NRR_FN_(NRR_INST_B, NRR_INST_LPT)
#endif

namespace nrr {
nrr_status NRR_FN(const MatchLaunch &m, cudaStream_t stream, int *occ)
{
    return launch_match_b<NRR_T, NRR_INST_B, NRR_LPT>(m, stream, occ);
}
}  // namespace nrr
