// Variance-based block selection (Sec. 4.1, "Parallel feature selection").
//
// The paper partitions the image among threads, computes a variance and an
// index per candidate, sorts the pairs in parallel, merges them and keeps
// 0.5 + N_c * F_s blocks.  Here that becomes:
//   K1 keys          exact key N*sum(I^2) - (sum I)^2 of the b^3 block at
//                    every stride grid point that is a candidate (centre in
//                    mask, block in volume), else -1; counts N_c and the
//                    number of keys > 0.  Strides up to 3 use the TMA-fed
//                    separable box-sum kernel (nrr_boxsum.cu); larger ones one
//                    thread per grid point.
//   K2 radix select  up to five histogram passes over 11-bit digits of the
//                    keys, starting at the top bit of the largest key, find
//                    the n_sel-th largest key K* and how many keys equal to
//                    K* are needed; no full sort.
//   K3 compaction    an order-preserving compaction writes every centre
//                    with key > K*, plus the first `need` with key == K*
//                    in raster order, to the output in raster order.
//   K2 and K3 are one cooperative launch: a grid barrier after each pass
//   (every CTA then fixes the same digit from the global histogram) and
//   one before the compaction's writes (each CTA's offset is the sum of
//   the counts of the CTAs before it).
// Ties are therefore ranked by raster index and the result is
// deterministic.
#include <math.h>

#include <mutex>

#include "nrr_internal.h"
#include "nrr_ptx.cuh"

namespace nrr {
namespace {

constexpr int KEY_THREADS = 256;
constexpr int HIST_BINS = 2048;
constexpr int CMP_ITEMS = 4;      // keys per thread per compaction sub-block
constexpr int CMP_CHUNK = 4096;   // keys per entry of the count scratch (at least one entry per rank CTA)
constexpr int NPASS = 5;

struct SelState {
    unsigned long long nc;    // candidates
    unsigned long long npos;  // candidates with key > 0
    long long prefix;         // digits fixed so far
    long long kth;            // rank still to find inside the current bucket (1-based)
    long long nsel;           // number selected
    long long thresh;         // key of the nsel-th largest (K*)
    long long need_ties;      // how many keys equal to K* are selected
    unsigned long long maxkey;  // largest key (sets the first digit)
    unsigned int arrived[NPASS + 1];  // [0]: the rank kernel's grid-barrier arrivals
    unsigned int nlist;       // keys collected from a small bucket
    int done;                 // nothing (more) to select
};

// B: block edge along x; by, bz: edges along y and z
template <int B>
__global__ void __launch_bounds__(KEY_THREADS) grid_keys_kernel(const uint16_t *__restrict__ preop,
                                                                const uint8_t *__restrict__ mask, int nx, int ny,
                                                                int nz, int by, int bz, int stride, int gx, int gy,
                                                                long long ng, long long *__restrict__ keys,
                                                                SelState *st)
{
    constexpr int H = (B - 1) / 2;
    const int HY = (by - 1) / 2, HZ = (bz - 1) / 2;
    const long long N = (long long)B * by * bz;
    const long long g = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    int cand = 0, pos = 0;
    unsigned long long kmax = 0;
    if (g < ng) {
        const int i = (int)(g % gx), j = (int)((g / gx) % gy), k = (int)(g / ((long long)gx * gy));
        const int x = i * stride, y = j * stride, z = k * stride;
        long long key = -1;
        if (x >= H && y >= HY && z >= HZ && x <= nx - 1 - H && y <= ny - 1 - HY && z <= nz - 1 - HZ &&
            mask[((size_t)z * ny + y) * nx + x] != 0) {
            unsigned int s = 0;
            unsigned long long q = 0;
            for (int kz = -HZ; kz <= HZ; ++kz)
                for (int ky = -HY; ky <= HY; ++ky) {
                    const uint16_t *row = preop + ((size_t)(z + kz) * ny + (y + ky)) * nx + (x - H);
                    unsigned int rs = 0;
                    unsigned long long rq = 0;
#pragma unroll
                    for (int kx = 0; kx < B; ++kx) {
                        unsigned int v = __ldg(row + kx);
                        rs += v;
                        rq += (unsigned long long)(v * v);
                    }
                    s += rs;
                    q += rq;
                }
            key = N * (long long)q - (long long)s * (long long)s;
            cand = 1;
            pos = key > 0;
            kmax = (unsigned long long)key;
        }
        keys[g] = key;
    }
    // block reduction of the two counts
    __shared__ int ws[KEY_THREADS / 32][2];
    __shared__ unsigned long long wmax[KEY_THREADS / 32];
    unsigned m = 0xffffffffu;
    for (int o = 16; o; o >>= 1) {
        cand += __shfl_xor_sync(m, cand, o);
        pos += __shfl_xor_sync(m, pos, o);
        const unsigned long long other = __shfl_xor_sync(m, kmax, o);
        kmax = other > kmax ? other : kmax;
    }
    if ((threadIdx.x & 31) == 0) {
        ws[threadIdx.x >> 5][0] = cand;
        ws[threadIdx.x >> 5][1] = pos;
        wmax[threadIdx.x >> 5] = kmax;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        int c = 0, p = 0;
        unsigned long long mx = 0;
        for (int w = 0; w < KEY_THREADS / 32; ++w) {
            c += ws[w][0];
            p += ws[w][1];
            mx = wmax[w] > mx ? wmax[w] : mx;
        }
        if (c) atomicAdd(&st->nc, (unsigned long long)c);
        if (p) atomicAdd(&st->npos, (unsigned long long)p);
        if (mx) atomicMax(&st->maxkey, mx);
    }
}

// Digit of pass `pass`: 11-bit digits from the top bit of the largest key
// down; the last one may be narrower.  Returns false if the pass is unused.
__device__ __forceinline__ bool digit_of_pass(const SelState *st, int pass, int *shift, int *width)
{
    const unsigned long long mx = st->maxkey;
    if (!mx) return false;
    const int top = 64 - __clzll((long long)mx);  // bits in the largest key
    int sh = top - 11 * (pass + 1), w = 11;
    if (sh < 0) {
        w += sh;
        sh = 0;
    }
    if (w <= 0) return false;
    *shift = sh;
    *width = w;
    return true;
}

// K2 + K3 in one cooperative launch (every CTA resident; waits bounded).
// Radix select: per pass, every CTA histograms this pass's digit over its
// share of the keys that match the digits fixed so far and adds its bins to
// the pass's global histogram; after a grid barrier every CTA reads the
// same histogram and fixes the same digit (the bucket holding the kth
// largest key), so a pass costs one barrier.  Compaction: CTA c owns one
// contiguous span of keys; it counts its keys > K* and == K*, and after a
// barrier its output offset is the sum of the counts of the CTAs before it;
// the keys selected are written in raster order with the ties quota.
constexpr int RK_THREADS = 512;
constexpr int RK_KPT = 8;  // keys per thread per sweep (RK_THREADS * RK_KPT = CMP_CHUNK)
constexpr int RK_SUB = RK_THREADS * CMP_ITEMS;     // keys per compaction sub-block
constexpr int RK_SMALL = 2048;  // a bucket this small is collected and finished inside every CTA

__device__ __forceinline__ unsigned long long block_excl_scan_rk(unsigned long long v, unsigned long long *tot)
{
    __shared__ unsigned long long ws[RK_THREADS / 32];
    const int lane = threadIdx.x & 31, wp = threadIdx.x >> 5;
    unsigned long long incl = v;
    for (int o = 1; o < 32; o <<= 1) {
        const unsigned long long n = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += n;
    }
    __syncthreads();  // ws is reused from the previous call
    if (lane == 31) ws[wp] = incl;
    __syncthreads();
    unsigned long long before = 0, all = 0;
    for (int i = 0; i < RK_THREADS / 32; ++i) {
        if (i < wp) before += ws[i];
        all += ws[i];
    }
    if (tot) *tot = all;
    return before + incl - v;
}

__global__ void __launch_bounds__(RK_THREADS) select_rank_kernel(const long long *__restrict__ keys, long long ng,
                                                                 long long span, double frac, SelState *st,
                                                                 unsigned int *__restrict__ hist,
                                                                 long long *__restrict__ list,
                                                                 unsigned long long *__restrict__ cnt, int gx, int gy,
                                                                 int stride, int32_t *__restrict__ centers,
                                                                 int max_blocks, int32_t *d_n_selected,
                                                                 unsigned int *err, uint64_t wait_ns,
                                                                 unsigned int missing)
{
    __shared__ unsigned int h[HIST_BINS];
    __shared__ long long wsum[RK_THREADS / 32];
    __shared__ long long lk[RK_SMALL];  // a small bucket's keys
    __shared__ long long s_prefix, s_kth, s_thresh, s_need, s_nsel, s_bcount;
    __shared__ int s_done;
    const int t = threadIdx.x, lane = t & 31, wp = t >> 5;
    unsigned int nb = 0;  // grid barriers passed
    auto barrier = [&]() {
        if (grid_barrier(&st->arrived[0], nb++, wait_ns, missing)) return true;
        if (t == 0) atomicOr(err, DEV_ERR_TIMEOUT);
        return false;
    };
    if (t == 0) {
        // n_sel = floor(0.5 + N_c * F_s), capped at the keys > 0 (Sec. 4.1)
        long long ns = (long long)floor(__dadd_rn(0.5, __dmul_rn((double)st->nc, frac)));
        if (ns > (long long)st->npos) ns = (long long)st->npos;
        if (ns < 0) ns = 0;
        s_nsel = ns;
        s_kth = ns;
        s_prefix = 0;
        s_done = ns == 0 || st->maxkey == 0;
        s_thresh = 0x7fffffffffffffffll;  // nothing selected unless a pass fixes it
        s_need = 0;
        s_bcount = 0;
    }
    __syncthreads();
    // every CTA finds the bucket of `src` (nbins bins of the digit at bit
    // sh) holding the kth largest key: thread t owns reversed bins r =
    // PER*t .. PER*t+PER-1 (bin b = nbins-1-r), an inclusive scan over r
    // counts the keys in bins >= b; the digit joins the prefix, kth becomes
    // the rank inside the bucket, and at bit 0 the threshold is fixed
    auto pick = [&](const unsigned int *src, bool global, int nbins, int sh) {
        constexpr int PER = HIST_BINS / RK_THREADS;
        const long long kth = s_kth, prefix = s_prefix;
        long long c[PER], v = 0;
#pragma unroll
        for (int q = 0; q < PER; ++q) {
            const int bin = nbins - 1 - (PER * t + q);
            c[q] = bin >= 0 ? (long long)(global ? __ldcg(src + bin) : src[bin]) : 0;
            v += c[q];
        }
        long long incl = v;
        for (int o = 1; o < 32; o <<= 1) {
            const long long n2 = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += n2;
        }
        if (lane == 31) wsum[wp] = incl;
        __syncthreads();  // every thread has read s_kth and s_prefix
        long long above = incl - v;  // keys in bins above this thread's first bin
        for (int i = 0; i < wp; ++i) above += wsum[i];
#pragma unroll
        for (int q = 0; q < PER; ++q) {
            const int bin = nbins - 1 - (PER * t + q);
            if (bin >= 0 && above < kth && above + c[q] >= kth) {
                const long long pre = prefix | ((long long)bin << sh);
                s_prefix = pre;
                s_kth = kth - above;
                s_bcount = c[q];
                if (sh == 0) {
                    s_thresh = pre;
                    s_need = kth - above;
                    s_done = 1;
                }
            }
            above += c[q];
        }
        __syncthreads();
    };
    int sh_fixed = 64;  // the digits at and above this bit are fixed
    for (int pass = 0; pass < NPASS && !s_done; ++pass) {
        int sh, w;
        if (!digit_of_pass(st, pass, &sh, &w)) break;
        for (int i = t; i < HIST_BINS; i += RK_THREADS) h[i] = 0;
        __syncthreads();
        const long long hi = s_prefix >> (sh + w);
        const long long dmask = (1ll << w) - 1;
        // RK_KPT keys per thread per sweep, all loads issued before any is used
        const long long sweep = (long long)gridDim.x * RK_THREADS * RK_KPT;
        for (long long g0 = (long long)blockIdx.x * RK_THREADS * RK_KPT + t; g0 < ng; g0 += sweep) {
            long long kv[RK_KPT];
#pragma unroll
            for (int q = 0; q < RK_KPT; ++q) {
                const long long g = g0 + (long long)q * RK_THREADS;
                kv[q] = g < ng ? __ldcg(keys + g) : -1;
            }
#pragma unroll
            for (int q = 0; q < RK_KPT; ++q) {
                const long long k = kv[q];
                if (k > 0 && (k >> (sh + w)) == hi) {
                    const unsigned bin = (unsigned)((k >> sh) & dmask);
                    // lanes of a warp with the same bin add once
                    const unsigned peers = __match_any_sync(__activemask(), bin);
                    if (lane == __ffs(peers) - 1) atomicAdd(&h[bin], (unsigned)__popc(peers));
                }
            }
        }
        __syncthreads();
        unsigned int *gh = hist + pass * HIST_BINS;
        for (int i = t; i < HIST_BINS; i += RK_THREADS)
            if (h[i]) atomicAdd(&gh[i], h[i]);
        if (!barrier()) return;
        pick(gh, true, 1 << w, sh);
        sh_fixed = sh;
        if (!s_done && s_bcount <= RK_SMALL) break;  // a small bucket: finished below
    }
    if (!s_done && sh_fixed < 64 && s_bcount <= RK_SMALL) {
        // collect the bucket's keys (every key > 0 whose digits above
        // sh_fixed are the prefix's), then every CTA finishes the radix
        // select on them in shared memory, with no more grid barriers
        const long long hi = s_prefix >> sh_fixed;
        const long long sweep = (long long)gridDim.x * RK_THREADS * RK_KPT;
        for (long long g0 = (long long)blockIdx.x * RK_THREADS * RK_KPT + t; g0 < ng; g0 += sweep) {
            long long kv[RK_KPT];
#pragma unroll
            for (int q = 0; q < RK_KPT; ++q) {
                const long long g = g0 + (long long)q * RK_THREADS;
                kv[q] = g < ng ? __ldcg(keys + g) : -1;
            }
#pragma unroll
            for (int q = 0; q < RK_KPT; ++q)
                if (kv[q] > 0 && (kv[q] >> sh_fixed) == hi) {
                    const unsigned pos = atomicAdd(&st->nlist, 1u);
                    if (pos < (unsigned)RK_SMALL) __stcg(list + pos, kv[q]);
                }
        }
        if (!barrier()) return;
        const int nl = (int)s_bcount;
        for (int i = t; i < nl; i += RK_THREADS) lk[i] = __ldcg(list + i);
        int shr = sh_fixed;
        while (!s_done && shr > 0) {
            const int w = shr < 11 ? shr : 11, shift = shr - w;
            for (int i = t; i < HIST_BINS; i += RK_THREADS) h[i] = 0;
            __syncthreads();  // and lk is loaded
            const long long hib = s_prefix >> shr;
            const long long dmask = (1ll << w) - 1;
            for (int i = t; i < nl; i += RK_THREADS)
                if ((lk[i] >> shr) == hib) atomicAdd(&h[(unsigned)((lk[i] >> shift) & dmask)], 1u);
            __syncthreads();
            pick(h, false, 1 << w, shift);
            shr = shift;
        }
    }
    const long long th = s_thresh, need = s_need;
    if (blockIdx.x == 0 && t == 0) {
        st->nsel = s_nsel;
        st->thresh = th;
        st->need_ties = need;
        if (d_n_selected) *d_n_selected = (int32_t)s_nsel;
    }
    // ---- compaction over this CTA's span [k0, k1) ----------------------------
    const long long k0 = (long long)blockIdx.x * span;
    const long long k1 = k0 + span < ng ? k0 + span : ng;
    unsigned long long v = 0;  // keys > K* (high word), == K* (low word)
    for (long long b0 = k0; b0 < k1; b0 += RK_SUB) {
#pragma unroll
        for (int i = 0; i < CMP_ITEMS; ++i) {
            const long long g = b0 + (long long)t * CMP_ITEMS + i;
            if (g < k1) {
                const long long k = __ldcg(keys + g);
                if (k > th) v += 1ull << 32;
                else if (k == th) v += 1ull;
            }
        }
    }
    unsigned long long tot;
    block_excl_scan_rk(v, &tot);
    if (t == 0) __stcg(cnt + blockIdx.x, tot);
    if (!barrier()) return;
    // this CTA's offset: the counts of the CTAs before it
    unsigned long long off = 0;
    for (int i = t; i < (int)blockIdx.x; i += RK_THREADS) off += __ldcg(cnt + i);
    unsigned long long offall;
    block_excl_scan_rk(off, &offall);
    unsigned long long carry = offall;
    for (long long b0 = k0; b0 < k1; b0 += RK_SUB) {
        long long k[CMP_ITEMS];
        unsigned long long u = 0;
#pragma unroll
        for (int i = 0; i < CMP_ITEMS; ++i) {
            const long long g = b0 + (long long)t * CMP_ITEMS + i;
            k[i] = g < k1 ? __ldcg(keys + g) : -1;
            if (k[i] > th) u += 1ull << 32;
            else if (k[i] == th) u += 1ull;
        }
        unsigned long long subtot;
        const unsigned long long ex = block_excl_scan_rk(u, &subtot) + carry;
        carry += subtot;
        long long sb = (long long)(ex >> 32), tb = (long long)(ex & 0xffffffffull);
#pragma unroll
        for (int i = 0; i < CMP_ITEMS; ++i) {
            const long long g = b0 + (long long)t * CMP_ITEMS + i;
            bool sel = false;
            long long pos = 0;
            if (k[i] > th) {
                sel = true;
                pos = sb + (tb < need ? tb : need);
                ++sb;
            } else if (k[i] == th) {
                if (tb < need) {
                    sel = true;
                    pos = sb + tb;
                }
                ++tb;
            }
            if (sel && pos < max_blocks) {
                const int x = (int)(g % gx), y = (int)((g / gx) % gy), z = (int)(g / ((long long)gx * gy));
                centers[3 * pos + 0] = x * stride;
                centers[3 * pos + 1] = y * stride;
                centers[3 * pos + 2] = z * stride;
            }
        }
    }
}

template <int B>
void launch_keys(const uint16_t *preop, const uint8_t *mask, nrr_dims d, int by, int bz, int stride, int gx, int gy,
                 long long ng, long long *keys, SelState *st, cudaStream_t s)
{
    const unsigned grid = (unsigned)((ng + KEY_THREADS - 1) / KEY_THREADS);
    grid_keys_kernel<B><<<grid, KEY_THREADS, 0, s>>>(preop, mask, d.nx, d.ny, d.nz, by, bz, stride, gx, gy, ng, keys,
                                                     st);
}

}  // namespace

SelectPlan select_plan(nrr_dims d, int stride, int connectivity)
{
    SelectPlan p;
    p.connectivity = connectivity;
    p.gx = (d.nx + stride - 1) / stride;
    p.gy = (d.ny + stride - 1) / stride;
    p.gz = (d.nz + stride - 1) / stride;
    p.ng = (long long)p.gx * p.gy * p.gz;
    p.nchunks = (int)((p.ng + CMP_CHUNK - 1) / CMP_CHUNK);
    size_t o = 0;
    p.off_keys = o;
    o += align_up((size_t)p.ng * 8, 256);
    p.off_hist = o;
    o += align_up(sizeof(unsigned int) * HIST_BINS * NPASS, 256);
    p.off_state = o;
    o += align_up(sizeof(SelState), 256);
    p.off_sync = o;  // zeroed together with the histograms and the state
    o += align_up(sizeof(SpacingSync), 256);
    p.off_cnt = o;
    o += align_up((size_t)p.nchunks * 8, 256);
    p.off_list = o;
    o += align_up(sizeof(long long) * RK_SMALL, 256);
    p.off_sp_state = p.off_sp_mask = p.off_sp_tiles = o;
    if (connectivity) {
        o += align_up((size_t)p.ng, 256);
        p.off_sp_mask = o;
        o += align_up((size_t)p.ng * 4, 256);
        p.off_sp_tiles = o;  // a pending flag per tile of the pattern kernel
        const size_t ntiles = (size_t)((p.gx + SP_TILE_X - 1) / SP_TILE_X) * ((p.gy + SP_TILE_Y - 1) / SP_TILE_Y) *
                              ((p.gz + SP_TILE_Z - 1) / SP_TILE_Z);
        o += align_up(ntiles * 4, 256);
    }
    p.bytes = o;
    return p;
}

// Enqueue the whole selection on `s` using the scratch buffer `ws` (at least
// select_plan().bytes, 256-byte aligned).  Reads nothing back.
nrr_status enqueue_select(const uint16_t *preop, const uint8_t *mask, nrr_dims d, int block, int stride,
                                 double frac, int32_t *centers, int32_t max_blocks, int32_t *d_n_selected,
                                 unsigned char *ws, const SelectPlan &p, cudaStream_t s, int block_y, int block_z)
{
    const int by = block_y > 0 ? block_y : block, bz = block_z > 0 ? block_z : block;
    long long *keys = (long long *)(ws + p.off_keys);
    unsigned int *hist = (unsigned int *)(ws + p.off_hist);
    SelState *st = (SelState *)(ws + p.off_state);
    unsigned long long *cnt = (unsigned long long *)(ws + p.off_cnt);
    NRR_CUDA_TRY(cudaMemsetAsync(ws + p.off_hist, 0, p.off_cnt - p.off_hist, s));
    if (by == block && bz == block && keys_box_supported(block, stride)) {
        nrr_status ks = launch_keys_box(preop, mask, d, block, stride, p.gx, p.gy, p.gz, keys, &st->nc, &st->npos,
                                        &st->maxkey, s);
        if (ks != NRR_OK) return ks;
    } else {
        switch (block) {
        case 3: launch_keys<3>(preop, mask, d, by, bz, stride, p.gx, p.gy, p.ng, keys, st, s); break;
        case 5: launch_keys<5>(preop, mask, d, by, bz, stride, p.gx, p.gy, p.ng, keys, st, s); break;
        case 7: launch_keys<7>(preop, mask, d, by, bz, stride, p.gx, p.gy, p.ng, keys, st, s); break;
        case 9: launch_keys<9>(preop, mask, d, by, bz, stride, p.gx, p.gy, p.ng, keys, st, s); break;
        default: launch_keys<11>(preop, mask, d, by, bz, stride, p.gx, p.gy, p.ng, keys, st, s); break;
        }
    }
    if (p.connectivity) {
        nrr_status ss = launch_spacing(p.connectivity, keys, p.gx, p.gy, p.ng, frac, ws + p.off_sp_state,
                                       (unsigned int *)(ws + p.off_sp_mask), (SpacingSync *)(ws + p.off_sync),
                                       &st->nc, &st->maxkey, &st->npos, (unsigned int *)(ws + p.off_sp_tiles), s);
        if (ss != NRR_OK) return ss;
    }
    // the rank kernel: at most two CTAs per SM (and as many as are resident),
    // one span of keys each
    static int occ = 0;
    if (!occ) {
        NRR_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, select_rank_kernel, RK_THREADS, 0));
        if (occ < 1) return fail(NRR_E_INTERNAL, "selection kernel does not fit on an SM");
    }
    long long grid = (p.ng + RK_THREADS * RK_KPT - 1) / (RK_THREADS * RK_KPT);
    const long long most = (long long)(occ < 2 ? occ : 2) * sm_count();
    if (grid > most) grid = most;
    if (grid < 1) grid = 1;
    long long span = (p.ng + grid - 1) / grid;
    span = (span + RK_SUB - 1) / RK_SUB * RK_SUB;
    unsigned int *err = nullptr;
    nrr_status es = device_error_word(&err);
    if (es != NRR_OK) return es;
    const uint64_t wait_ns = device_wait_ns();
    const unsigned int missing = test_missing_arrivals();
    cudaLaunchConfig_t cfg{};
    cfg.gridDim = dim3((unsigned)grid);
    cfg.blockDim = dim3(RK_THREADS);
    cfg.dynamicSmemBytes = 0;
    cfg.stream = s;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeCooperative;
    at[0].val.cooperative = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    NRR_CUDA_TRY(cudaLaunchKernelEx(&cfg, select_rank_kernel, (const long long *)keys, p.ng, span, frac, st, hist,
                                    (long long *)(ws + p.off_list), cnt, p.gx, p.gy, stride, centers, (int)max_blocks,
                                    d_n_selected, err, wait_ns, missing));
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "selection kernel launch");
    count_launches(2);
    return NRR_OK;
}

size_t select_count_offset(const SelectPlan &p) { return p.off_state + offsetof(SelState, nsel); }

nrr_status check_select_args(nrr_dims dims, int32_t block, int32_t stride, double frac)
{
    nrr_status st = check_dims(dims, NRR_U16, block);
    if (st != NRR_OK) return st;
    if (stride < 1 || stride > 64) return fail(NRR_E_INVALID, "stride %d outside 1..64", stride);
    if (!(frac > 0.0 && frac <= 1.0)) return fail(NRR_E_INVALID, "frac must be in (0, 1]");
    return NRR_OK;
}

}  // namespace nrr

using namespace nrr;

// Selection with the scratch from the stream-ordered allocator: block edges
// (x, y, z) and an optional connectivity pattern.
static nrr_status select_alloc(const uint16_t *d_preop, const uint8_t *d_mask, nrr_dims dims, const int32_t *block,
                               int32_t stride, double frac, int32_t connectivity, int32_t *d_centers,
                               int32_t max_blocks, int32_t *d_n_selected, int32_t *h_n_selected, void *stream)
{
    clear_error();
    nrr_status st = check_dims3(dims, NRR_U16, block);
    if (st != NRR_OK) return st;
    st = check_select_args(dims, block[0], stride, frac);
    if (st != NRR_OK) return st;
    if (connectivity != 0 && connectivity != 6 && connectivity != 18 && connectivity != 26)
        return fail(NRR_E_INVALID, "connectivity %d is not 0, 6, 18 or 26", connectivity);
    if (max_blocks < 0) return fail(NRR_E_INVALID, "max_blocks < 0");
    if (!d_preop || !d_mask) return fail(NRR_E_INVALID, "NULL volume or mask");
    if (max_blocks > 0 && !d_centers) return fail(NRR_E_INVALID, "NULL centre buffer");
    cudaStream_t s = (cudaStream_t)stream;
    const SelectPlan p = select_plan(dims, stride, connectivity);
    void *ws = nullptr;
    NRR_CUDA_TRY(cudaMallocAsync(&ws, p.bytes, s));
    st = enqueue_select(d_preop, d_mask, dims, block[0], stride, frac, d_centers, max_blocks, d_n_selected,
                        (unsigned char *)ws, p, s, block[1], block[2]);
    long long nsel = 0;
    if (st == NRR_OK && h_n_selected) {
        cudaError_t e = cudaMemcpyAsync(&nsel, (unsigned char *)ws + select_count_offset(p),
                                        sizeof(nsel), cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) st = cuda_fail(e, "reading the selection count");
    }
    cudaError_t e = cudaFreeAsync(ws, s);
    if (st != NRR_OK) return st;
    if (e != cudaSuccess) return cuda_fail(e, "cudaFreeAsync");
    if (h_n_selected) {
        *h_n_selected = (int32_t)nsel;
        if (nsel > max_blocks)
            return fail(NRR_E_CAPACITY, "%lld blocks selected but max_blocks is %d", nsel, max_blocks);
    }
    return NRR_OK;
}

extern "C" nrr_status nrr_select_blocks(const uint16_t *d_preop, const uint8_t *d_mask, nrr_dims dims, int32_t block,
                                        int32_t stride, double frac, int32_t *d_centers, int32_t max_blocks,
                                        int32_t *d_n_selected, int32_t *h_n_selected, void *stream)
{
    const int32_t b3[3] = {block, block, block};
    return select_alloc(d_preop, d_mask, dims, b3, stride, frac, 0, d_centers, max_blocks, d_n_selected,
                        h_n_selected, stream);
}

extern "C" nrr_status nrr_select_blocks_spaced(const uint16_t *d_preop, const uint8_t *d_mask, nrr_dims dims,
                                               int32_t block, int32_t stride, double frac, int32_t connectivity,
                                               int32_t *d_centers, int32_t max_blocks, int32_t *d_n_selected,
                                               int32_t *h_n_selected, void *stream)
{
    const int32_t b3[3] = {block, block, block};
    return select_alloc(d_preop, d_mask, dims, b3, stride, frac, connectivity, d_centers, max_blocks, d_n_selected,
                        h_n_selected, stream);
}

extern "C" nrr_status nrr_select_blocks_aniso(const uint16_t *d_preop, const uint8_t *d_mask, nrr_dims dims,
                                              const int32_t block[3], int32_t stride, double frac,
                                              int32_t *d_centers, int32_t max_blocks, int32_t *d_n_selected,
                                              int32_t *h_n_selected, void *stream)
{
    if (!block) return fail(NRR_E_INVALID, "block is NULL");
    return select_alloc(d_preop, d_mask, dims, block, stride, frac, 0, d_centers, max_blocks, d_n_selected,
                        h_n_selected, stream);
}

// ---------------------------------------------------------------------------
// Selection without any allocation at call time.
//
// The scratch lives in one file-scope device array of fixed size, so every
// GPU that loads the library holds it until the process exits.  Host code
// cannot use the array's name as a device address (it only stands in for
// the symbol on the host), so the address is looked up once per device with
// cudaGetSymbolAddress, with that device current.
// ---------------------------------------------------------------------------
namespace nrr {
namespace {
constexpr size_t SELECT_STATIC_SCRATCH_BYTES = (size_t)NRR_SELECT_STATIC_SCRATCH_BYTES;
__device__ __align__(256) unsigned char g_select_scratch[SELECT_STATIC_SCRATCH_BYTES];

nrr_status static_select_scratch(unsigned char **ptr)
{
    static std::mutex mu;
    static unsigned char *addr[64] = {};
    int dev = 0;
    NRR_CUDA_TRY(cudaGetDevice(&dev));
    if (dev < 0 || dev >= 64) return fail(NRR_E_INTERNAL, "device ordinal %d out of range", dev);
    std::lock_guard<std::mutex> lk(mu);
    if (!addr[dev]) {
        void *p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_select_scratch);
        if (e != cudaSuccess) return cuda_fail(e, "cudaGetSymbolAddress(selection scratch)");
        addr[dev] = (unsigned char *)p;
    }
    *ptr = addr[dev];
    return NRR_OK;
}
}  // namespace
}  // namespace nrr

extern "C" nrr_status nrr_select_blocks_noalloc(const uint16_t *d_preop, const uint8_t *d_mask, nrr_dims dims,
                                                int32_t block, int32_t stride, double frac, int32_t *d_centers,
                                                int32_t max_blocks, int32_t *d_n_selected, int32_t *h_n_selected,
                                                void *stream)
{
    clear_error();
    nrr_status st = check_select_args(dims, block, stride, frac);
    if (st != NRR_OK) return st;
    if (max_blocks < 0) return fail(NRR_E_INVALID, "max_blocks < 0");
    if (!d_preop || !d_mask) return fail(NRR_E_INVALID, "NULL volume or mask");
    if (max_blocks > 0 && !d_centers) return fail(NRR_E_INVALID, "NULL centre buffer");
    const SelectPlan p = select_plan(dims, stride);
    if (p.bytes > SELECT_STATIC_SCRATCH_BYTES)
        return fail(NRR_E_CAPACITY,
                    "%lld candidate grid points need %zu scratch bytes; the allocation-free selection holds %zu "
                    "(use nrr_select_blocks or a larger stride)",
                    p.ng, p.bytes, SELECT_STATIC_SCRATCH_BYTES);
    unsigned char *ws = nullptr;
    st = static_select_scratch(&ws);
    if (st != NRR_OK) return st;
    cudaStream_t s = (cudaStream_t)stream;
    // enqueue_select zeroes the histograms and counters it accumulates into
    // (the array keeps whatever the previous call left there).
    st = enqueue_select(d_preop, d_mask, dims, block, stride, frac, d_centers, max_blocks, d_n_selected, ws, p, s);
    if (st != NRR_OK) return st;
    if (h_n_selected) {
        long long nsel = 0;
        cudaError_t e = cudaMemcpyAsync(&nsel, ws + select_count_offset(p), sizeof(nsel), cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) return cuda_fail(e, "reading the selection count");
        *h_n_selected = (int32_t)nsel;
        if (nsel > max_blocks)
            return fail(NRR_E_CAPACITY, "%lld blocks selected but max_blocks is %d", nsel, max_blocks);
    }
    return NRR_OK;
}
