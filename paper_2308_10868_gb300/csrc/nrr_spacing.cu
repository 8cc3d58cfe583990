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
// Only a prefix of the candidates in selection order matters: a decision
// depends only on higher-priority neighbours, so the greedy set restricted
// to any prefix is the greedy set of that prefix.  The kernel therefore puts
// in play the candidates whose key reaches a threshold chosen from a
// histogram of the keys so that about 4 * n_sel of them are in play, builds
// their greedy set, and widens the prefix (four times as many candidates)
// only while fewer than n_sel have been accepted and candidates are left.
//
// The greedy set of the candidates in play is found without a sequential
// walk.  A candidate is rejected as soon as one of its higher-priority
// neighbours is accepted and accepted once all of them are rejected.  States
// only ever move from undecided to final and a final state is the greedy
// answer, so applying that rule in place, in any order, reading a
// neighbour's old or new state, converges to the greedy set.  Decisions
// propagate along chains of decreasing priority, so the work is tiled: a CTA
// loads a 16 x 8 x 8 tile of the candidate grid with a one-point halo into
// shared memory and applies the rule there until the tile stops changing
// (chains inside the tile cost block barriers only), then writes the tile
// back.  A global round does this for every tile; rounds repeat until no
// candidate in play is undecided.  Halo states read at the start of a round
// may be stale, which only delays a decision to a later round.
//
// One cooperative launch runs all phases: every CTA is resident, phases and
// rounds are separated by a grid barrier on a monotone arrival counter, and
// every wait gives up after a time limit (the device error word records it).
#include <math.h>
#include <stddef.h>

#include "nrr_internal.h"
#include "nrr_ptx.cuh"

namespace nrr {
namespace {

constexpr int SP_THREADS = 256;
constexpr int TLX = SP_TILE_X, TLY = SP_TILE_Y, TLZ = SP_TILE_Z, TPTS = TLX * TLY * TLZ;  // tile of candidate grid points
constexpr int HX = TLX + 2, HY = TLY + 2, HZ = TLZ + 2, HPTS = HX * HY * HZ;  // with a one-point halo
constexpr int PPT = TPTS / SP_THREADS;  // tile points per thread
constexpr int SP_MAX_ROUNDS = 1 << 20;
constexpr int SP_BINS = 2048;  // histogram of the keys' top 11 bits
constexpr int SP_PREFIX = 4;   // candidates in play per selected block, and growth factor
enum : unsigned char { SP_OUT_OF_PLAY = 0, SP_UNDECIDED = 1, SP_ACCEPTED = 2, SP_REJECTED = 3 };

// Grid offsets (di, dj, dk): the 6 face neighbours, then the 12 edge
// neighbours, then the 8 vertex neighbours, so pattern order n uses the
// first 6, 18 or 26 entries.
__constant__ signed char c_offs[26][3] = {
    {-1, 0, 0},  {1, 0, 0},  {0, -1, 0}, {0, 1, 0},  {0, 0, -1},  {0, 0, 1},                              // face
    {-1, -1, 0}, {1, -1, 0}, {-1, 1, 0}, {1, 1, 0},  {-1, 0, -1}, {1, 0, -1}, {-1, 0, 1}, {1, 0, 1},      // edge
    {0, -1, -1}, {0, 1, -1}, {0, -1, 1}, {0, 1, 1},                                                       // edge
    {-1, -1, -1}, {1, -1, -1}, {-1, 1, -1}, {1, 1, -1}, {-1, -1, 1}, {1, -1, 1}, {-1, 1, 1}, {1, 1, 1}};  // vertex

__device__ __forceinline__ unsigned char load_state(const unsigned char *p) { return (unsigned char)__ldcg(p); }
__device__ __forceinline__ void store_state(unsigned char *p, unsigned char v) { __stcg(p, v); }

// Number selected without a pattern's cap: floor(0.5 + N_c * F_s) (Sec. 4.1).
__device__ __forceinline__ long long n_select_dev(unsigned long long nc, double frac)
{
    return (long long)floor(__dadd_rn(0.5, __dmul_rn((double)nc, frac)));
}

// Smallest histogram bin b such that the keys in bins >= b number at least
// `m` (0 if all of them are fewer); the keys >= b << sh are then a prefix of
// the selection order holding at least m candidates.  Every CTA computes the
// same value from the same global histogram.
__device__ int prefix_bin(const unsigned int *hist, unsigned long long m)
{
    __shared__ unsigned long long s_cnt[32];
    __shared__ int s_bin;
    const int lane = threadIdx.x & 31;
    if (threadIdx.x < 32) {  // lane l sums bins [64 l, 64 l + 64)
        unsigned long long c = 0;
        for (int q = 0; q < SP_BINS / 32; ++q) c += __ldcg(hist + lane * (SP_BINS / 32) + q);
        s_cnt[lane] = c;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned long long acc = 0;
        int bin = 0;
        for (int l = 31; l >= 0 && !bin; --l) {
            if (acc + s_cnt[l] < m) {
                acc += s_cnt[l];
                continue;
            }
            for (int b = l * (SP_BINS / 32) + SP_BINS / 32 - 1; b >= l * (SP_BINS / 32); --b) {
                acc += __ldcg(hist + b);
                if (acc >= m) {
                    bin = b;
                    break;
                }
            }
            if (!bin) break;  // reached m exactly at bin 0
        }
        s_bin = bin;
    }
    __syncthreads();
    return s_bin;
}

template <int ORDER>
__global__ void __launch_bounds__(SP_THREADS, 2)
    spacing_kernel(long long *__restrict__ keys, int gx, int gy, long long ng, int slots, double frac,
                   unsigned char *__restrict__ state, unsigned int *__restrict__ hmask, SpacingSync *sync,
                   const unsigned long long *nc, const unsigned long long *maxkey, unsigned long long *npos,
                   unsigned int *__restrict__ tile_pend, unsigned int *err, uint64_t wait_ns, unsigned int missing)
{
    constexpr int NOFF = ORDER == 1 ? 6 : ORDER == 2 ? 18 : 26;
    const long long chunk = (long long)slots * SP_THREADS;
    const long long g0 = (long long)blockIdx.x * chunk + threadIdx.x;
    const long long gxy = (long long)gx * gy;
    const int gz = (int)(ng / gxy);
    const unsigned long long mx = *maxkey;
    const int top = mx ? 64 - __clzll((long long)mx) : 0;  // bits of the largest key
    const int sh = top > 11 ? top - 11 : 0;
    const long long want = n_select_dev(*nc, frac);
    unsigned int nb = 0;  // grid barriers passed
    __shared__ unsigned int s_hist[SP_BINS];
    __shared__ unsigned char s_state[HPTS];
    __shared__ unsigned long long s_pend, s_acc;
    __shared__ unsigned int s_tp;

    // ---- each candidate's higher-priority neighbours; histogram of the keys
    for (int e = threadIdx.x; e < SP_BINS; e += SP_THREADS) s_hist[e] = 0;
    if (blockIdx.x == 0 && threadIdx.x == 0) *npos = 0;  // becomes the size of the greedy set
    __syncthreads();
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
            atomicAdd(&s_hist[(key >> sh) & (SP_BINS - 1)], 1u);
        }
        hmask[g] = m;
    }
    __syncthreads();
    for (int e = threadIdx.x; e < SP_BINS; e += SP_THREADS)
        if (s_hist[e]) atomicAdd(&sync->hist[e], s_hist[e]);
    if (!grid_barrier(&sync->arrive, nb++, wait_ns, missing)) {
        if (threadIdx.x == 0) atomicOr(err, DEV_ERR_TIMEOUT);
        return;
    }

    // ---- grow the prefix in play until n_sel are accepted or none is left --
    const int ntx = (gx + TLX - 1) / TLX, nty = (gy + TLY - 1) / TLY, ntz = (gz + TLZ - 1) / TLZ;
    const int ntiles = ntx * nty * ntz;
    unsigned long long m_play = (unsigned long long)(want > 0 ? want : 1) * SP_PREFIX;
    long long t_hi = 0x7fffffffffffffffll;  // keys >= t_hi are already in play
    int r = 0;                              // rounds so far
    for (;;) {
        const int bin = prefix_bin(sync->hist, m_play);
        const long long t_lo = bin ? ((long long)bin << sh) : 1;  // keys >= t_lo in play from now on
        for (int q = 0; q < slots; ++q) {
            const long long g = g0 + (long long)q * SP_THREADS;
            if (g >= ng) break;
            const long long key = keys[g];
            if (key >= t_lo && key < t_hi) store_state(state + g, SP_UNDECIDED);
            else if (t_hi == 0x7fffffffffffffffll && key < t_lo) store_state(state + g, SP_OUT_OF_PLAY);
        }
        // every tile may hold newly undecided points: all of this CTA's tiles
        // are visited in the next round (a CTA always takes the same tiles)
        for (int t = blockIdx.x + threadIdx.x * (int)gridDim.x; t < ntiles; t += SP_THREADS * (int)gridDim.x)
            tile_pend[t] = 1u;
        if (!grid_barrier(&sync->arrive, nb++, wait_ns, missing)) {
            if (threadIdx.x == 0) atomicOr(err, DEV_ERR_TIMEOUT);
            return;
        }
        t_hi = t_lo;

        // ---- rounds over tiles until no candidate in play is undecided ----
        for (;; ++r) {
            if (threadIdx.x == 0) {
                s_pend = 0;
                s_acc = 0;
                if (blockIdx.x == 0) sync->undecided[(r + 1) % 3] = 0;  // its last reader finished two barriers ago
            }
            unsigned int pend = 0, acc = 0;
            for (int t = blockIdx.x; t < ntiles; t += gridDim.x) {
                // a tile left with no undecided point has nothing more to
                // decide (states only move from undecided to final); the flag
                // was written by this CTA, before a barrier
                if (__ldcg(tile_pend + t) == 0u) continue;
                const int i0 = (t % ntx) * TLX, j0 = ((t / ntx) % nty) * TLY, k0 = (t / (ntx * nty)) * TLZ;
                __syncthreads();  // the previous tile's shared states are no longer read
                if (threadIdx.x == 0) s_tp = 0;
                for (int e = threadIdx.x; e < HPTS; e += SP_THREADS) {
                    const int i = i0 - 1 + e % HX, j = j0 - 1 + (e / HX) % HY, k = k0 - 1 + e / (HX * HY);
                    unsigned char v = SP_OUT_OF_PLAY;
                    if (i >= 0 && j >= 0 && k >= 0 && i < gx && j < gy && k < gz)
                        v = load_state(state + (long long)k * gxy + (long long)j * gx + i);
                    s_state[e] = v;
                }
                __syncthreads();
                // this thread's points of the tile: undecided ones and their masks
                unsigned int m[PPT];
                int sidx[PPT];
                unsigned int open = 0;  // bit q: point q still undecided
#pragma unroll
                for (int q = 0; q < PPT; ++q) {
                    const int p = threadIdx.x + q * SP_THREADS;
                    const int li = p % TLX, lj = (p / TLX) % TLY, lk = p / (TLX * TLY);
                    sidx[q] = ((lk + 1) * HY + (lj + 1)) * HX + (li + 1);
                    m[q] = 0;
                    if (s_state[sidx[q]] == SP_UNDECIDED) {  // in the grid by construction
                        m[q] = hmask[(long long)(k0 + lk) * gxy + (long long)(j0 + lj) * gx + (i0 + li)];
                        open |= 1u << q;
                    }
                }
                const unsigned int open0 = open;
                // apply the rule inside the tile until nothing changes; every
                // pass that changes something decides at least one point, so at
                // most TPTS + 1 passes.  A pass reads all masked neighbours at
                // once (independent shared loads); a state another thread
                // writes during the pass may be seen old or new, either is safe.
                for (int it = 0; it <= TPTS; ++it) {
                    bool changed = false;
#pragma unroll
                    for (int q = 0; q < PPT; ++q) {
                        if (!((open >> q) & 1u)) continue;
                        const unsigned int mm = m[q];
                        bool waiting = false, blocked = false;
#pragma unroll
                        for (int b = 0; b < NOFF; ++b) {
                            if ((mm >> b) & 1u) {
                                const unsigned char su =
                                    s_state[sidx[q] + c_offs[b][0] + c_offs[b][1] * HX + c_offs[b][2] * (HX * HY)];
                                blocked |= su == SP_ACCEPTED;
                                waiting |= su == SP_UNDECIDED;
                            }
                        }
                        if (blocked || !waiting) {
                            s_state[sidx[q]] = blocked ? SP_REJECTED : SP_ACCEPTED;
                            acc += blocked ? 0u : 1u;
                            open &= ~(1u << q);
                            changed = true;
                        }
                    }
                    if (!__syncthreads_or(changed)) break;
                }
                // write back the points decided in this tile pass (only this
                // CTA writes them, so nothing newer can be overwritten)
#pragma unroll
                for (int q = 0; q < PPT; ++q) {
                    if (((open0 & ~open) >> q) & 1u) {
                        const int p = threadIdx.x + q * SP_THREADS;
                        const int li = p % TLX, lj = (p / TLX) % TLY, lk = p / (TLX * TLY);
                        store_state(state + (long long)(k0 + lk) * gxy + (long long)(j0 + lj) * gx + (i0 + li),
                                    s_state[sidx[q]]);
                    }
                    pend += (open >> q) & 1u;
                }
                // this tile's points still undecided after the pass
                if (open) atomicAdd(&s_tp, (unsigned int)__popc(open));
                __syncthreads();
                if (threadIdx.x == 0) __stcg(tile_pend + t, s_tp);
            }
            if (pend) atomicAdd(&s_pend, (unsigned long long)pend);
            if (acc) atomicAdd(&s_acc, (unsigned long long)acc);
            __syncthreads();
            if (threadIdx.x == 0) {
                if (s_pend) atomicAdd(&sync->undecided[r % 3], s_pend);
                if (s_acc) atomicAdd(npos, s_acc);
            }
            if (!grid_barrier(&sync->arrive, nb++, wait_ns, missing)) {
                if (threadIdx.x == 0) atomicOr(err, DEV_ERR_TIMEOUT);
                return;
            }
            const unsigned long long left = *(volatile unsigned long long *)&sync->undecided[r % 3];
            if (r + 1 >= SP_MAX_ROUNDS) {  // cannot happen for a finite grid; kept as a bound
                if (blockIdx.x == 0 && threadIdx.x == 0) atomicOr(err, DEV_ERR_INTERNAL);
                return;
            }
            if (left == 0) {
                ++r;
                break;
            }
        }
        // every CTA reads the same count: all additions precede the barrier
        const unsigned long long accepted = *(volatile unsigned long long *)npos;
        if ((long long)accepted >= want || t_lo <= 1) break;
        m_play *= SP_PREFIX;
    }

    // ---- only members of the greedy set stay selectable ----------------------
    for (int q = 0; q < slots; ++q) {
        const long long g = g0 + (long long)q * SP_THREADS;
        if (g >= ng) break;
        if (keys[g] > 0 && load_state(state + g) != SP_ACCEPTED) keys[g] = 0;
    }
}

template <int ORDER>
nrr_status launch_order(long long *keys, int gx, int gy, long long ng, double frac, unsigned char *state,
                        unsigned int *hmask, SpacingSync *sync, const unsigned long long *nc,
                        const unsigned long long *maxkey, unsigned long long *npos, unsigned int *tile_pend,
                        cudaStream_t s)
{
    auto kern = spacing_kernel<ORDER>;
    int occ = 0;
    NRR_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, SP_THREADS, 0));
    if (occ < 1) return fail(NRR_E_INTERNAL, "spacing kernel does not fit on an SM");
    const long long gz = ng / ((long long)gx * gy);
    const long long ntiles = (long long)((gx + TLX - 1) / TLX) * ((gy + TLY - 1) / TLY) * ((gz + TLZ - 1) / TLZ);
    long long maxb = (long long)occ * sm_count();
    int blocks = (int)(ntiles < maxb ? ntiles : maxb);
    if (blocks < 1) blocks = 1;
    int slots = (int)((ng + (long long)blocks * SP_THREADS - 1) / ((long long)blocks * SP_THREADS));
    if (slots < 1) slots = 1;
    unsigned int *err = nullptr;
    nrr_status st = device_error_word(&err);
    if (st != NRR_OK) return st;
    uint64_t wait_ns = device_wait_ns();
    unsigned int missing = test_missing_arrivals();
    void *args[] = {&keys, &gx,   &gy,  &ng,  &slots,   &frac,    &state,  &hmask,
                    &sync, &nc,   &maxkey, &npos, &tile_pend, &err, &wait_ns, &missing};
    NRR_CUDA_TRY(cudaLaunchCooperativeKernel((const void *)kern, dim3(blocks), dim3(SP_THREADS), args, 0, s));
    count_launches(1);
    return NRR_OK;
}

}  // namespace

nrr_status launch_spacing(int connectivity, long long *keys, int gx, int gy, long long ng, double frac,
                          unsigned char *state, unsigned int *hmask, SpacingSync *sync,
                          const unsigned long long *nc, const unsigned long long *maxkey, unsigned long long *npos,
                          unsigned int *tile_pend, cudaStream_t s)
{
    if (ng <= 0) return NRR_OK;
    switch (connectivity) {
    case 6: return launch_order<1>(keys, gx, gy, ng, frac, state, hmask, sync, nc, maxkey, npos, tile_pend, s);
    case 18: return launch_order<2>(keys, gx, gy, ng, frac, state, hmask, sync, nc, maxkey, npos, tile_pend, s);
    case 26: return launch_order<3>(keys, gx, gy, ng, frac, state, hmask, sync, nc, maxkey, npos, tile_pend, s);
    default: return fail(NRR_E_INVALID, "connectivity %d is not 0, 6, 18 or 26", connectivity);
    }
}

}  // namespace nrr
