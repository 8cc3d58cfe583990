// Connectivity pattern of the block selection (Sec. 4.1): blocks too close
// to a better one are not selected.  The "face", "edge" and "vertex" simplex
// patterns are 6-, 18- and 26-connectivity on the candidate grid.
//
// The selection is the greedy walk in selection order (key descending,
// raster index ascending): a candidate is accepted unless an already
// accepted candidate is its pattern neighbour, until floor(0.5 + N_c F_s)
// are accepted.  Those are the first members, in selection order, of the
// greedy independent set of the whole candidate graph, so the kernel builds
// that whole set and the ordinary top-k selection then takes its first
// n_sel members (every other candidate's key is set to 0, which the top-k
// never selects, and the cap becomes the size of the set).
//
// The greedy set is found without a sequential walk.  A candidate's fate
// depends only on its higher-priority neighbours: it is rejected as soon as
// one of them is accepted and accepted once all of them are rejected.  Each
// round applies that rule to every undecided candidate, in place (states
// only ever move from undecided to final, and a final state is the greedy
// answer, so reading a neighbour's old or new state is equally safe); the
// rounds end when none is undecided.  Their number is the longest chain of
// decreasing priority that the decisions have to follow, tens on smooth
// variance fields.
//
// One cooperative launch runs all rounds: every CTA is resident, rounds are
// separated by a grid barrier on a monotone arrival counter, and every wait
// gives up after a time limit (the device error word records it).
#include <stddef.h>

#include "nrr_internal.h"
#include "nrr_ptx.cuh"

namespace nrr {
namespace {

constexpr int SP_THREADS = 256;
constexpr uint64_t SP_WAIT_NS = 2000000000ull;
constexpr int SP_MAX_ROUNDS = 1 << 20;
enum : unsigned char { SP_OUT_OF_PLAY = 0, SP_UNDECIDED = 1, SP_ACCEPTED = 2, SP_REJECTED = 3 };

// Grid offsets (di, dj, dk): the 6 face neighbours, then the 12 edge
// neighbours, then the 8 vertex neighbours, so pattern order n uses the
// first 6, 18 or 26 entries.
__constant__ signed char c_offs[26][3] = {
    {-1, 0, 0},  {1, 0, 0},  {0, -1, 0}, {0, 1, 0},  {0, 0, -1},  {0, 0, 1},                              // face
    {-1, -1, 0}, {1, -1, 0}, {-1, 1, 0}, {1, 1, 0},  {-1, 0, -1}, {1, 0, -1}, {-1, 0, 1}, {1, 0, 1},      // edge
    {0, -1, -1}, {0, 1, -1}, {0, -1, 1}, {0, 1, 1},                                                       // edge
    {-1, -1, -1}, {1, -1, -1}, {-1, 1, -1}, {1, 1, -1}, {-1, -1, 1}, {1, -1, 1}, {-1, 1, 1}, {1, 1, 1}};  // vertex

// Grid-wide barrier number `index` (0, 1, ...): every CTA adds one arrival
// and waits for (index + 1) * gridDim.x of them.  Returns false if the wait
// ran out of time.
__device__ bool grid_barrier(unsigned int *arrive, unsigned int index, uint64_t limit_ns)
{
    __shared__ int ok;
    __syncthreads();
    if (threadIdx.x == 0) {
        const unsigned int target = (index + 1u) * gridDim.x;
        __threadfence();
        atomicAdd(arrive, 1u);
        int good = 1;
        const uint64_t t0 = global_ns();
        while (*(volatile unsigned int *)arrive < target) {
            if (global_ns() - t0 > limit_ns) {
                good = 0;
                break;
            }
            __nanosleep(64);
        }
        __threadfence();
        ok = good;
    }
    __syncthreads();
    return ok != 0;
}

__device__ __forceinline__ unsigned char load_state(const unsigned char *p) { return (unsigned char)__ldcg(p); }
__device__ __forceinline__ void store_state(unsigned char *p, unsigned char v) { __stcg(p, v); }

template <int ORDER>
__global__ void __launch_bounds__(SP_THREADS) spacing_kernel(long long *__restrict__ keys, int gx, int gy, long long ng,
                                                           int slots, unsigned char *__restrict__ state,
                                                           unsigned int *__restrict__ hmask, SpacingSync *sync,
                                                           unsigned long long *npos, unsigned int *err)
{
    constexpr int NOFF = ORDER == 1 ? 6 : ORDER == 2 ? 18 : 26;
    const long long chunk = (long long)slots * SP_THREADS;
    const long long g0 = (long long)blockIdx.x * chunk + threadIdx.x;
    const long long gxy = (long long)gx * gy;
    const int gz = (int)(ng / gxy);

    // ---- the candidates in play and each one's higher-priority neighbours
    if (blockIdx.x == 0 && threadIdx.x == 0) *npos = 0;  // becomes the size of the greedy set
    for (int q = 0; q < slots; ++q) {
        const long long g = g0 + (long long)q * SP_THREADS;
        if (g >= ng) break;
        const long long key = keys[g];
        unsigned int m = 0;
        if (key > 0) {
            const int i = (int)(g % gx), j = (int)((g / gx) % gy), k = (int)(g / gxy);
#pragma unroll
            for (int b = 0; b < NOFF; ++b) {
                const int ii = i + c_offs[b][0], jj = j + c_offs[b][1], kk = k + c_offs[b][2];
                if (ii < 0 || jj < 0 || kk < 0 || ii >= gx || jj >= gy || kk >= gz) continue;
                const long long u = g + c_offs[b][0] + (long long)c_offs[b][1] * gx + (long long)c_offs[b][2] * gxy;
                const long long ku = keys[u];
                if (ku > 0 && (ku > key || (ku == key && u < g))) m |= 1u << b;
            }
        }
        hmask[g] = m;
        store_state(state + g, key > 0 ? SP_UNDECIDED : SP_OUT_OF_PLAY);
    }
    unsigned int nb = 0;  // grid barriers passed
    if (!grid_barrier(&sync->arrive, nb++, SP_WAIT_NS)) {
        if (threadIdx.x == 0) atomicOr(err, DEV_ERR_TIMEOUT);
        return;
    }

    // ---- rounds ----------------------------------------------------------------
    __shared__ unsigned long long s_pend, s_acc;
    for (int r = 0;; ++r) {
        if (threadIdx.x == 0) {
            s_pend = 0;
            s_acc = 0;
            if (blockIdx.x == 0) sync->undecided[(r + 1) % 3] = 0;  // its last reader finished two barriers ago
        }
        __syncthreads();
        unsigned int pend = 0, acc = 0;
        for (int q = 0; q < slots; ++q) {
            const long long g = g0 + (long long)q * SP_THREADS;
            if (g >= ng) break;
            if (load_state(state + g) != SP_UNDECIDED) continue;
            unsigned int m = hmask[g];
            bool waiting = false, blocked = false;
            while (m) {
                const int b = __ffs(m) - 1;
                m &= m - 1;
                const long long u = g + c_offs[b][0] + (long long)c_offs[b][1] * gx + (long long)c_offs[b][2] * gxy;
                const unsigned char su = load_state(state + u);
                if (su == SP_ACCEPTED) {
                    blocked = true;
                    break;
                }
                if (su == SP_UNDECIDED) waiting = true;
            }
            if (blocked) {
                store_state(state + g, SP_REJECTED);
            } else if (!waiting) {
                store_state(state + g, SP_ACCEPTED);
                ++acc;
            } else {
                ++pend;
            }
        }
        if (pend) atomicAdd(&s_pend, (unsigned long long)pend);
        if (acc) atomicAdd(&s_acc, (unsigned long long)acc);
        __syncthreads();
        if (threadIdx.x == 0) {
            if (s_pend) atomicAdd(&sync->undecided[r % 3], s_pend);
            if (s_acc) atomicAdd(npos, s_acc);
        }
        if (!grid_barrier(&sync->arrive, nb++, SP_WAIT_NS)) {
            if (threadIdx.x == 0) atomicOr(err, DEV_ERR_TIMEOUT);
            return;
        }
        const unsigned long long left = *(volatile unsigned long long *)&sync->undecided[r % 3];
        if (left == 0) break;
        if (r + 1 >= SP_MAX_ROUNDS) {  // cannot happen for a finite grid; kept as a bound
            if (blockIdx.x == 0 && threadIdx.x == 0) atomicOr(err, DEV_ERR_INTERNAL);
            return;
        }
    }

    // ---- only members of the greedy set stay selectable ----------------------
    for (int q = 0; q < slots; ++q) {
        const long long g = g0 + (long long)q * SP_THREADS;
        if (g >= ng) break;
        if (keys[g] > 0 && load_state(state + g) != SP_ACCEPTED) keys[g] = 0;
    }
}

template <int ORDER>
nrr_status launch_order(long long *keys, int gx, int gy, long long ng, unsigned char *state, unsigned int *hmask,
                        SpacingSync *sync, unsigned long long *npos, cudaStream_t s)
{
    auto kern = spacing_kernel<ORDER>;
    int occ = 0;
    NRR_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, SP_THREADS, 0));
    if (occ < 1) return fail(NRR_E_INTERNAL, "spacing kernel does not fit on an SM");
    long long maxb = (long long)occ * sm_count();
    long long need = (ng + SP_THREADS - 1) / SP_THREADS;
    int blocks = (int)(need < maxb ? need : maxb);
    if (blocks < 1) blocks = 1;
    int slots = (int)((ng + (long long)blocks * SP_THREADS - 1) / ((long long)blocks * SP_THREADS));
    if (slots < 1) slots = 1;
    unsigned int *err = nullptr;
    nrr_status st = device_error_word(&err);
    if (st != NRR_OK) return st;
    void *args[] = {&keys, &gx, &gy, &ng, &slots, &state, &hmask, &sync, &npos, &err};
    NRR_CUDA_TRY(cudaLaunchCooperativeKernel((const void *)kern, dim3(blocks), dim3(SP_THREADS), args, 0, s));
    count_launches(1);
    return NRR_OK;
}

}  // namespace

nrr_status launch_spacing(int connectivity, long long *keys, int gx, int gy, long long ng, unsigned char *state,
                          unsigned int *hmask, SpacingSync *sync, unsigned long long *npos, cudaStream_t s)
{
    if (ng <= 0) return NRR_OK;
    switch (connectivity) {
    case 6: return launch_order<1>(keys, gx, gy, ng, state, hmask, sync, npos, s);
    case 18: return launch_order<2>(keys, gx, gy, ng, state, hmask, sync, npos, s);
    case 26: return launch_order<3>(keys, gx, gy, ng, state, hmask, sync, npos, s);
    default: return fail(NRR_E_INVALID, "connectivity %d is not 0, 6, 18 or 26", connectivity);
    }
}

}  // namespace nrr
