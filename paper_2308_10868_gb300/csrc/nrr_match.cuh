// NCC block-matching kernel (Sec. 3 NCC equation and O(B x W) bound;
// Sec. 4.3 block-matching loop), written for sm_103a.
//
// A persistent CTA walks its share of the registration blocks.  Per block:
//   1. TMA tiled loads bring the block's search window of the reference
//      image, [c-h-R, c+h+R] per axis, and the floating block [c-h, c+h]^3
//      into shared memory (x start rounded down to a 16-byte boundary;
//      out-of-volume voxels arrive as zeros and are excluded by coordinates).
//      The copy for the next block is issued as soon as the current one has
//      been unpacked, so it lands while the current block is searched.
//   2. Warp 0 reduces the floating block's sums; the other warps unpack the
//      window to float, shifted by a per-block constant c (J'_k = J_k - c).
//      The floating block is stored mean-shifted (T_k = I_k - m).
//   3. Search: thread t owns one (dz, dy) line of the window and all 2*rx+1
//      shifts along x; for every template row it loads one window row
//      (16-byte shared loads, conflict-free row pitch) and accumulates
//      A(d) = sum_k T_k J'_{k+d} with FP32 FFMA, fully unrolled over the row
//      and the x shifts.
//   4. Every shift gets an approximate NCC and a rigorous bound on its error
//      (recursive-summation bound gamma_N * sum|T||J'| for the FFMA chain,
//      Cauchy-Schwarz sum|T||J'| <= sqrt(sum T^2 * sum J'^2), plus the
//      rounding of the final operations; doubled for margin).
//   5. Shifts whose upper bound reaches the best lower bound survive (about
//      one per block on the phantoms) and are rescored by a warp each:
//      uint16 -> exact int64 sum, then the canonical FP64 ratio
//      num / sqrt(vI * vJ); float32 -> FP64 Pearson.  The best survivor
//      under the tie-break rule is the block's answer.
// The exhaustive maximum is therefore found exactly: the true arg-max can
// never be filtered out, because its upper bound is at least its value,
// which is at least every other shift's value, hence at least every lower
// bound.
#pragma once

#include <math.h>
#include <stdint.h>

#include <type_traits>

#include "nrr_internal.h"
#include "nrr_ptx.cuh"

namespace nrr {

struct MatchParams {
    const void *preop;
    const void *intraop;
    const void *s1;
    const void *s2;
    int nx, ny, nz;
    int ry, rz;
    int bx;   // TMA box extent along x of the window (elements)
    int btx;  // TMA box extent along x of the floating block (elements)
    int pf;   // row pitch of the float window (floats)
    int n_jobs;
    MatchJob jobs[MATCH_MAX_JOBS];
    unsigned int *err;
};

constexpr int MATCH_MAX_THREADS = 256;
constexpr int MATCH_MAX_WARPS = MATCH_MAX_THREADS / 32;
constexpr uint64_t WAIT_LIMIT_NS = 2000000000ull;  // 2 s

// Per-block constants produced by warp 0 and read by the whole CTA.
struct BlockConst {
    long long vI;   // uint16: N*S_II - S_I^2 (exact)
    long long rr;   // uint16: N*m - S_I
    double dvI;     // float32: sum (I - Ibar)^2
    double ibar;    // float32: mean of I
    float fvI;      // vI as float
    float kq;       // uint16: N*gamma_N*sqrt(sum T^2); float32: sqrt(sum T^2) (rounded up)
    float mu;       // float32: float mean used for T
    float emu;      // float32: Ibar - mu
    int m;          // uint16: integer mean used for T
    int flat;       // floating block has zero variance
};

struct MatchScratch {
    BlockConst bc;
    float wlb[MATCH_MAX_WARPS];
    double bs[MATCH_MAX_WARPS];
    int bn2[MATCH_MAX_WARPS];
    int bcode[MATCH_MAX_WARPS];
    int bok[MATCH_MAX_WARPS];
    int nsurv;
    int jstart[MATCH_MAX_JOBS + 1];  // first work item of each job
};

struct MatchLayout {
    int u, ut, f, t, surv, sc, bar, total;
};

__host__ __device__ inline int round_up_i(int v, int a) { return (v + a - 1) / a * a; }

// Shared-memory carve-up of one CTA (all offsets 128-byte aligned).
__host__ __device__ inline MatchLayout match_layout(int elem, int B, int P, int bx, int btx, int pf, int wy, int wz,
                                                   int py, int pz)
{
    MatchLayout L;
    int pt = round_up_i(B, 4);
    int o = 0;
    L.u = o;
    o += round_up_i(bx * wy * wz * elem, 128);
    L.ut = o;
    o += round_up_i(btx * B * B * elem, 128);
    L.f = o;
    o += round_up_i(pf * wy * wz * 4, 128);
    L.t = o;
    o += round_up_i(B * B * pt * 4, 128);
    L.surv = o;
    o += round_up_i(P * py * pz * 2, 128);
    L.sc = o;
    o += round_up_i((int)sizeof(MatchScratch), 128);
    L.bar = o;
    o += 128;
    L.total = o;
    return L;
}

// Row pitch of the float window: a multiple of 4 floats with an odd number
// of 16-byte chunks, so 8 consecutive rows fall in distinct bank groups.
__host__ __device__ inline int match_pitch(int wx)
{
    int q = (wx + 3) / 4;
    if ((q & 1) == 0) ++q;
    return 4 * q;
}

struct Cand {
    double s;
    int n2;
    int code;
    int ok;
};

// NCC descending, then |d|^2 ascending, then (dz, dy, dx) lexicographic
// ascending; `code` increases with (dz, dy, dx) lexicographically.
__device__ __forceinline__ bool cand_better(const Cand &a, const Cand &b)
{
    if (!a.ok) return false;
    if (!b.ok) return true;
    if (a.s != b.s) return a.s > b.s;
    if (a.n2 != b.n2) return a.n2 < b.n2;
    return a.code < b.code;
}

__device__ __forceinline__ float warp_max_f(float v)
{
#pragma unroll
    for (int o = 16; o; o >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}
__device__ __forceinline__ float warp_min_f(float v)
{
#pragma unroll
    for (int o = 16; o; o >>= 1) v = fminf(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}
template <typename V>
__device__ __forceinline__ V warp_sum(V v)
{
#pragma unroll
    for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Exact uint16 -> float of (u - c) for u, c < 2^16: 0x4B000000|u is the float
// 2^23 + u, so one integer OR and one float subtraction suffice.
__device__ __forceinline__ float u16_minus(uint32_t u, float c_plus_2p23)
{
    return __fsub_rn(__uint_as_float(0x4B000000u | u), c_plus_2p23);
}

__device__ __forceinline__ void write_result(const MatchJob &a, int blk, const Cand &b, int P, int py, int rx, int ry,
                                             int rz)
{
    if (b.ok) {
        int dxi = b.code % P, dyi = (b.code / P) % py, dzi = b.code / (P * py);
        a.disp[3 * blk + 0] = dxi - rx;
        a.disp[3 * blk + 1] = dyi - ry;
        a.disp[3 * blk + 2] = dzi - rz;
        a.ncc[blk] = b.s;
        a.valid[blk] = 1;
    } else {
        a.disp[3 * blk + 0] = 0;
        a.disp[3 * blk + 1] = 0;
        a.disp[3 * blk + 2] = 0;
        a.ncc[blk] = __longlong_as_double(0x7ff8000000000000ll);
        a.valid[blk] = 0;
    }
}

template <int H>
__device__ __forceinline__ bool center_inside(int cx, int cy, int cz, int nx, int ny, int nz)
{
    return cx >= H && cy >= H && cz >= H && cx <= nx - 1 - H && cy <= ny - 1 - H && cz <= nz - 1 - H;
}

// Register budget: at most 80 registers per thread for blocks up to 7^3 and
// up to 11 x-shifts (5-6 search CTAs of <= 128 threads per SM), 128 above.
template <int B, int P>
struct MatchMinBlocks {
    static constexpr int value = (P <= 11 && B <= 7) ? 3 : 2;
};

template <typename T, int B, int P>
__global__ void __launch_bounds__(MATCH_MAX_THREADS, MatchMinBlocks<B, P>::value) match_kernel(const MatchParams a,
                                                                  const __grid_constant__ CUtensorMap tmapJ,
                                                                  const __grid_constant__ CUtensorMap tmapI)
{
    constexpr bool F32 = std::is_same<T, float>::value;
    constexpr int H = (B - 1) / 2;
    constexpr int N = B * B * B;
    constexpr int PT = (B + 3) / 4 * 4;
    constexpr int RX = (P - 1) / 2;
    constexpr int WX = B + P - 1;
    constexpr int NJ4 = (WX + 3) / 4;
    constexpr int ALIGN = 16 / (int)sizeof(T);
    constexpr float U32 = 5.9604644775390625e-08f;  // 2^-24, unit roundoff of binary32
    constexpr double GAMMA_N = (double)N * 5.9604644775390625e-08 / (1.0 - (double)N * 5.9604644775390625e-08);

    const int ry = a.ry, rz = a.rz, py = 2 * ry + 1, pz = 2 * rz + 1, lines = py * pz;
    const int wy = B + 2 * ry, wz = B + 2 * rz, bx = a.bx, btx = a.btx, pf = a.pf;
    const int nx = a.nx, ny = a.ny, nz = a.nz;

    extern __shared__ __align__(128) unsigned char smem[];
    const MatchLayout L = match_layout((int)sizeof(T), B, P, bx, btx, pf, wy, wz, py, pz);
    T *U = reinterpret_cast<T *>(smem + L.u);
    T *Ut = reinterpret_cast<T *>(smem + L.ut);
    float *Fw = reinterpret_cast<float *>(smem + L.f);
    float *Tm = reinterpret_cast<float *>(smem + L.t);
    uint16_t *surv = reinterpret_cast<uint16_t *>(smem + L.surv);
    MatchScratch *sc = reinterpret_cast<MatchScratch *>(smem + L.sc);
    uint64_t *bar = reinterpret_cast<uint64_t *>(smem + L.bar);

    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nthr = blockDim.x, nwarp = nthr >> 5;
    if (tid == 0) {
        int w = 0;
        for (int j = 0; j < a.n_jobs; ++j) {
            sc->jstart[j] = w;
            int m = a.jobs[j].cap;
            if (a.jobs[j].d_n) {
                const int d = *a.jobs[j].d_n;
                m = d < 0 ? 0 : (d < m ? d : m);
            }
            w += m;
        }
        sc->jstart[a.n_jobs] = w;
    }
    __syncthreads();
    const int n = sc->jstart[a.n_jobs];  // work items over all jobs
    // work item -> (job, index within the job)
    auto locate = [&](int w, int &j, int &i) {
        j = 0;
        while (j + 1 < a.n_jobs && w >= sc->jstart[j + 1]) ++j;
        i = w - sc->jstart[j];
    };
    const uint32_t tx_bytes = (uint32_t)((bx * wy * wz + btx * B * B) * (int)sizeof(T));
    // Thread 0 issues both copies of block b (its centre must be inside).
    auto issue = [&](int b) {
        int j, i;
        locate(b, j, i);
        const int32_t *cc = a.jobs[j].centers + 3 * i;
        const int cx = cc[0], cy = cc[1], cz = cc[2];
        const int x0 = cx - H - RX, xt = cx - H;
        fence_proxy_async_smem();
        mbar_arrive_expect_tx(bar, tx_bytes);
        tma_load_3d(U, &tmapJ, bar, x0 & ~(ALIGN - 1), cy - H - ry, cz - H - rz);
        tma_load_3d(Ut, &tmapI, bar, xt & ~(ALIGN - 1), cy - H, cz - H);
    };
    if (tid == 0) {
        mbar_init(bar, 1);
        fence_mbar_init();
    }
    __syncthreads();
    uint32_t phase = 0;
    int inflight = -1;  // block whose copies are in flight (same value in every thread)

    for (int blk = blockIdx.x; blk < n; blk += gridDim.x) {
        int job, bi;
        locate(blk, job, bi);
        const MatchJob &J = a.jobs[job];
        const int cx = J.centers[3 * bi + 0], cy = J.centers[3 * bi + 1], cz = J.centers[3 * bi + 2];
        if (!center_inside<H>(cx, cy, cz, nx, ny, nz)) {
            if (tid == 0) write_result(J, bi, Cand{0.0, 0, 0, 0}, P, py, RX, ry, rz);
            continue;
        }
        if (inflight != blk) {
            if (tid == 0) issue(blk);
            inflight = blk;
        }
        const int x0 = cx - H - RX, xo = x0 - (x0 & ~(ALIGN - 1));
        const int xt = cx - H, xot = xt - (xt & ~(ALIGN - 1));
        const size_t cidx = ((size_t)cz * ny + cy) * nx + cx;
        // window centring constant from the box sum at the centre
        float cshift;  // value subtracted (with 2^23 folded in for uint16)
        int c_i = 0;
        float c_f = 0.f;
        if constexpr (F32) {
            c_f = __fdiv_rn(reinterpret_cast<const float *>(a.s1)[cidx], (float)N);
            cshift = c_f;
        } else {
            const long long s1c = reinterpret_cast<const int32_t *>(a.s1)[cidx];
            c_i = (int)((2 * s1c + N) / (2 * N));
            cshift = 8388608.0f + (float)c_i;
        }
        if (tid == 0) sc->nsurv = 0;

        // ---- wait for the window and the floating block ------------------
        const bool got = mbar_wait_bounded(bar, phase, WAIT_LIMIT_NS);
        if (!__syncthreads_and(got)) {
            if (tid == 0) {
                atomicOr(a.err, DEV_ERR_TIMEOUT);
                write_result(J, bi, Cand{0.0, 0, 0, 0}, P, py, RX, ry, rz);
            }
            mbar_wait_bounded(bar, phase, WAIT_LIMIT_NS);  // let an in-flight copy land before exiting
            return;
        }
        phase ^= 1u;

        // ---- phase A: warp 0 reduces the floating block, the rest unpack ---
        if (warp == 0) {
            if constexpr (F32) {
                constexpr int KPL = (N + 31) / 32;  // values per lane
                constexpr int CH = KPL < 6 ? KPL : 6;   // loads in flight per lane
                double s = 0.0;
                float lo = INFINITY, hi = -INFINITY;
#pragma unroll 1
                for (int i0 = 0; i0 < KPL; i0 += CH) {
                    float vals[CH];
#pragma unroll
                    for (int i = 0; i < CH; ++i) {
                        const int k = lane + 32 * (i0 + i);
                        const int kzy = k / B, kx = k - kzy * B;
                        vals[i] = k < N ? Ut[kzy * btx + xot + kx] : NAN;
                    }
#pragma unroll
                    for (int i = 0; i < CH; ++i) {
                        if (lane + 32 * (i0 + i) < N) {
                            s += (double)vals[i];
                            lo = fminf(lo, vals[i]);
                            hi = fmaxf(hi, vals[i]);
                        }
                    }
                }
                s = warp_sum(s);
                lo = warp_min_f(lo);
                hi = warp_max_f(hi);
                const double ibar = s / (double)N;
                const float mu = (float)ibar;
                double q = 0.0, dv = 0.0;
#pragma unroll 1
                for (int i0 = 0; i0 < KPL; i0 += CH) {
                    float vals[CH];
#pragma unroll
                    for (int i = 0; i < CH; ++i) {
                        const int k = lane + 32 * (i0 + i);
                        const int kzy = k / B, kx = k - kzy * B;
                        vals[i] = k < N ? Ut[kzy * btx + xot + kx] : 0.f;
                    }
#pragma unroll
                    for (int i = 0; i < CH; ++i) {
                        if (lane + 32 * (i0 + i) < N) {
                            const double t = (double)__fsub_rn(vals[i], mu);
                            q = fma(t, t, q);
                            const double d = (double)vals[i] - ibar;
                            dv = fma(d, d, dv);
                        }
                    }
                }
                q = warp_sum(q);
                dv = warp_sum(dv);
                if (lane == 0) {
                    BlockConst &c = sc->bc;
                    c.flat = !(lo < hi);
                    c.ibar = ibar;
                    c.mu = mu;
                    c.emu = (float)(ibar - (double)mu);
                    c.dvI = dv;
                    c.fvI = (float)dv;
                    c.kq = (float)(sqrt(q) * (1.0 + 1e-6));
                }
            } else {
                constexpr int KPL = (N + 31) / 32;  // values per lane
                constexpr int CH = KPL < 6 ? KPL : 6;   // loads in flight per lane
                long long s = 0;
                unsigned long long q = 0;
#pragma unroll 1
                for (int i0 = 0; i0 < KPL; i0 += CH) {
                    uint32_t vals[CH];
#pragma unroll
                    for (int i = 0; i < CH; ++i) {
                        const int k = lane + 32 * (i0 + i);
                        const int kzy = k / B, kx = k - kzy * B;
                        vals[i] = k < N ? (uint32_t)Ut[kzy * btx + xot + kx] : 0u;
                    }
#pragma unroll
                    for (int i = 0; i < CH; ++i) {
                        s += vals[i];
                        q += (unsigned long long)(vals[i] * vals[i]);
                    }
                }
                s = warp_sum(s);
                q = warp_sum(q);
                if (lane == 0) {
                    BlockConst &c = sc->bc;
                    const long long vI = (long long)N * (long long)q - s * s;
                    const long long m = (2 * s + N) / (2 * N);  // nearest integer to the block mean
                    const long long qt = (long long)q - 2 * m * s + (long long)N * m * m;  // sum (I-m)^2, exact
                    c.vI = vI;
                    c.flat = vI == 0;
                    c.m = (int)m;
                    c.rr = (long long)N * m - s;
                    c.fvI = (float)vI;
                    c.kq = (float)((double)N * GAMMA_N * sqrt((double)qt) * (1.0 + 1e-6));
                }
            }
        }
        {
            // Window rows: lanes along x, a warp takes RB rows at a time and
            // issues all their loads before any store, so the shared-memory
            // latency is paid once per batch rather than once per row.
            constexpr int RB = 8;
            const int rows = wz * wy;
            for (int r0 = warp * RB; r0 < rows; r0 += nwarp * RB) {
                float v[RB];
#pragma unroll
                for (int j = 0; j < RB; ++j) {
                    const int r = r0 + j;
                    v[j] = 0.f;
                    if (r < rows && lane < WX) {
                        const T u = U[r * bx + xo + lane];
                        if constexpr (F32)
                            v[j] = __fsub_rn(u, cshift);
                        else
                            v[j] = u16_minus(u, cshift);
                    }
                }
#pragma unroll
                for (int j = 0; j < RB; ++j) {
                    const int r = r0 + j;
                    if (r < rows && lane < pf) Fw[r * pf + lane] = v[j];
                }
            }
        }
        __syncthreads();
        const BlockConst bc = sc->bc;
        if (bc.flat) {  // flat floating block: NCC undefined for every shift
            if (tid == 0) write_result(J, bi, Cand{0.0, 0, 0, 0}, P, py, RX, ry, rz);
            __syncthreads();
            continue;
        }
        // ---- phase B: mean-shifted template ---------------------------------
        {
            const float tsh = F32 ? bc.mu : 8388608.0f + (float)bc.m;
            constexpr int TB = B * B * PT;
            constexpr int TPT = (TB + 63) / 64;  // items per thread at 64+ threads
            float v[TPT];
#pragma unroll
            for (int j = 0; j < TPT; ++j) {
                const int k = tid + j * nthr;
                const int kzy = k / PT, kx = k - kzy * PT;
                v[j] = 0.f;
                if (k < TB && kx < B) {
                    if constexpr (F32)
                        v[j] = __fsub_rn(Ut[kzy * btx + xot + kx], tsh);
                    else
                        v[j] = u16_minus(Ut[kzy * btx + xot + kx], tsh);
                }
            }
#pragma unroll
            for (int j = 0; j < TPT; ++j) {
                const int k = tid + j * nthr;
                if (k < TB) Tm[k] = v[j];
            }
            for (int k = tid + TPT * nthr; k < TB; k += nthr) {  // fewer than 64 threads
                const int kzy = k / PT, kx = k - kzy * PT;
                float w = 0.f;
                if (kx < B) {
                    if constexpr (F32)
                        w = __fsub_rn(Ut[kzy * btx + xot + kx], tsh);
                    else
                        w = u16_minus(Ut[kzy * btx + xot + kx], tsh);
                }
                Tm[k] = w;
            }
        }
        __syncthreads();
        // both staging buffers are free: start the next block's copies
        {
            int nb = blk + gridDim.x;
            if (nb < n) {
                int nj, ni;
                locate(nb, nj, ni);
                const int32_t *nc = a.jobs[nj].centers + 3 * ni;
                const int ncx = nc[0], ncy = nc[1], ncz = nc[2];
                if (center_inside<H>(ncx, ncy, ncz, nx, ny, nz)) {
                    if (tid == 0) issue(nb);
                    inflight = nb;
                }
            }
        }

        // ---- search: FP32 accumulation of A(d) over the whole window ------
        float ub[P];
        float lbm = -INFINITY;
        const int dyi = tid % py, dzi = tid / py;
        if (tid < lines) {
            const int dy = dyi - ry, dz = dzi - rz, Y = cy + dy, Z = cz + dz;
            const bool yz_ok = Y >= H && Y <= ny - 1 - H && Z >= H && Z <= nz - 1 - H;
            typedef typename std::conditional<F32, float, int32_t>::type S1T;
            typedef typename std::conditional<F32, float, long long>::type S2T;

            const float *fbase = Fw + (dzi * wy + dyi) * pf;
            float acc[P];
#pragma unroll
            for (int p = 0; p < P; ++p) acc[p] = 0.f;
#pragma unroll 1
            for (int kz = 0; kz < B; ++kz) {
#pragma unroll 1
                for (int ky = 0; ky < B; ++ky) {
                    const float *fr = fbase + (kz * wy + ky) * pf;
                    const float *tr = Tm + (kz * B + ky) * PT;
                    float j[4 * NJ4], t[PT];
#pragma unroll
                    for (int q = 0; q < NJ4; ++q) {
                        const float4 v = *reinterpret_cast<const float4 *>(fr + 4 * q);
                        j[4 * q + 0] = v.x;
                        j[4 * q + 1] = v.y;
                        j[4 * q + 2] = v.z;
                        j[4 * q + 3] = v.w;
                    }
#pragma unroll
                    for (int q = 0; q < PT / 4; ++q) {
                        const float4 v = *reinterpret_cast<const float4 *>(tr + 4 * q);
                        t[4 * q + 0] = v.x;
                        t[4 * q + 1] = v.y;
                        t[4 * q + 2] = v.z;
                        t[4 * q + 3] = v.w;
                    }
#pragma unroll
                    for (int kx = 0; kx < B; ++kx)
#pragma unroll
                        for (int p = 0; p < P; ++p) acc[p] = __fmaf_rn(t[kx], j[kx + p], acc[p]);
                }
            }

            // box sums of this thread's shifts (independent loads, issued together)
            S1T ps1[P];
            S2T ps2[P];
            uint32_t vmask = 0;
            const size_t rowbase = ((size_t)Z * ny + Y) * nx;
#pragma unroll
            for (int p = 0; p < P; ++p) {
                const int X = cx + p - RX;
                ps1[p] = 0;
                ps2[p] = 0;
                if (yz_ok && X >= H && X <= nx - 1 - H) {
                    vmask |= 1u << p;
                    ps1[p] = reinterpret_cast<const S1T *>(a.s1)[rowbase + X];
                    ps2[p] = reinterpret_cast<const S2T *>(a.s2)[rowbase + X];
                }
            }

            // ---- approximate NCC and its error bound per shift -----------
            const float fN = (float)N;
#pragma unroll
            for (int p = 0; p < P; ++p) {
                ub[p] = -INFINITY;
                if (!((vmask >> p) & 1u)) continue;
                if constexpr (!F32) {
                    const long long s1 = ps1[p];
                    const long long s2 = ps2[p];
                    const long long vJ = (long long)N * s2 - s1 * s1;
                    if (vJ <= 0) continue;  // flat reference block
                    const long long s1p = s1 - (long long)N * c_i;
                    const long long s2p = s2 - 2ll * c_i * s1 + (long long)N * c_i * c_i;  // sum (J-c)^2
                    const float inv = __frsqrt_rn(__fmul_rn(bc.fvI, (float)vJ));
                    const float na = __fmul_rn(fN, acc[p]);
                    const float rs = (float)(bc.rr * s1p);
                    const float v = __fmul_rn(__fadd_rn(na, rs), inv);
                    float e = bc.kq * __fsqrt_rn((float)s2p) * inv + 3.f * U32 * (fabsf(na) + fabsf(rs)) * inv +
                              6.f * U32 * fabsf(v);
                    e = 2.f * e + 1e-9f;
                    ub[p] = v + e;
                    lbm = fmaxf(lbm, v - e);
                } else {
                    constexpr float GS = (float)(3.0 * B * 5.9604644775390625e-08 /
                                                 (1.0 - 3.0 * B * 5.9604644775390625e-08));  // box-sum depth
                    constexpr float GN = (float)GAMMA_N;
                    const float s1 = ps1[p];
                    const float s2 = fmaxf(ps2[p], 0.f);
                    const float d1 = GS * __fsqrt_rn(fN * s2) * 1.01f;  // |S1 err| bound
                    const float s1sq_n = __fmul_rn(__fmul_rn(s1, s1), 1.0f / fN);
                    const float vJa = __fsub_rn(s2, s1sq_n);
                    const float dv = GS * s2 + (2.f * fabsf(s1) + d1) * d1 / fN + 4.f * U32 * (s2 + s1sq_n);
                    const float s1p = __fsub_rn(s1, __fmul_rn(fN, c_f));  // ~ sum (J - c)
                    const float m2 = s2 + 2.f * fabsf(c_f) * fabsf(s1) + fN * c_f * c_f;
                    const float e2 = __fadd_rn(__fsub_rn(s2, 2.f * c_f * s1), fN * c_f * c_f);
                    const float sj2 = (fmaxf(e2, 0.f) + (GS + 8.f * U32) * m2 * 1.01f) * (1.f + 4.f * U32);
                    if (!(vJa - dv > 0.f)) {  // spread of the reference block not resolved: rescore
                        ub[p] = INFINITY;
                        continue;
                    }
                    const float rho = dv / (vJa - dv);
                    if (!(rho <= 0.25f)) {
                        ub[p] = INFINITY;
                        continue;
                    }
                    const float inv = __frsqrt_rn(__fmul_rn(bc.fvI, vJa));
                    const float A = acc[p];
                    const float es = __fmul_rn(bc.emu, s1p);
                    const float num = __fsub_rn(A, es);
                    const float v = __fmul_rn(num, inv);
                    const float enum_ = (GN + 3.f * U32) * bc.kq * __fsqrt_rn(sj2) +
                                        fabsf(bc.emu) * (fabsf(s1p) + d1 + 2.f * U32 * fN * fabsf(c_f)) * 1.01f +
                                        U32 * (fabsf(A) + fabsf(es));
                    float e = enum_ * inv * (1.f + 0.7f * rho + 4.f * U32) +
                              fabsf(num) * inv * (0.7f * rho + 6.f * U32) + 3.f * U32 * fabsf(v);
                    e = 2.f * e + 1e-9f;
                    ub[p] = v + e;
                    lbm = fmaxf(lbm, v - e);
                }
            }
        }

        // ---- best lower bound over the window; survivors ------------------
        lbm = warp_max_f(lbm);
        if (lane == 0) sc->wlb[warp] = lbm;
        __syncthreads();
        float LB = -INFINITY;
        for (int w = 0; w < nwarp; ++w) LB = fmaxf(LB, sc->wlb[w]);
        if (tid < lines) {
#pragma unroll
            for (int p = 0; p < P; ++p) {
                if (ub[p] > -INFINITY && ub[p] >= LB) {
                    int s = atomicAdd(&sc->nsurv, 1);
                    surv[s] = (uint16_t)((dzi * py + dyi) * P + p);
                }
            }
        }
        __syncthreads();
        const int nsurv = sc->nsurv;

        // ---- exact rescoring of the survivors, one warp each -------------
        Cand wb{0.0, 0, 0, 0};
        for (int s = warp; s < nsurv; s += nwarp) {
            const int code = surv[s];
            const int sxi = code % P, syi = (code / P) % py, szi = code / (P * py);
            const int dx = sxi - RX, dy = syi - ry, dz = szi - rz;
            const size_t idx = ((size_t)(cz + dz) * ny + (cy + dy)) * nx + (cx + dx);
            Cand c{0.0, dx * dx + dy * dy + dz * dz, code, 0};
            if constexpr (!F32) {
                long long s1 = 0, s2 = 0;
                if (lane == 0) {  // issued first, consumed after the warp sum
                    s1 = reinterpret_cast<const int32_t *>(a.s1)[idx];
                    s2 = reinterpret_cast<const long long *>(a.s2)[idx];
                }
                constexpr int KPL = (N + 31) / 32;
                constexpr int CH = KPL < 6 ? KPL : 6;
                long long e = 0;
#pragma unroll 1
                for (int i0 = 0; i0 < KPL; i0 += CH) {
                    int tv[CH], jv[CH];
#pragma unroll
                    for (int i = 0; i < CH; ++i) {
                        const int k = lane + 32 * (i0 + i);
                        const int kz = k / (B * B), rem = k - kz * B * B, ky = rem / B, kx = rem - ky * B;
                        tv[i] = 0;
                        jv[i] = 0;
                        if (k < N) {
                            tv[i] = (int)Tm[(kz * B + ky) * PT + kx];
                            jv[i] = (int)Fw[((szi + kz) * wy + (syi + ky)) * pf + sxi + kx];
                        }
                    }
#pragma unroll
                    for (int i = 0; i < CH; ++i) e += (long long)tv[i] * jv[i];
                }
                e = warp_sum(e);
                if (lane == 0) {
                    const long long vJ = (long long)N * s2 - s1 * s1;
                    const long long num = (long long)N * e + bc.rr * (s1 - (long long)N * c_i);
                    if (vJ > 0) {
                        const double den = __dsqrt_rn(__dmul_rn((double)bc.vI, (double)vJ));
                        c.s = __ddiv_rn((double)num, den);
                        c.ok = 1;
                    }
                }
            } else {
                const float *pre = reinterpret_cast<const float *>(a.preop);
                const float *intra = reinterpret_cast<const float *>(a.intraop);
                double sij = 0.0, sj = 0.0, sjj = 0.0;
                float lo = INFINITY, hi = -INFINITY;
                for (int k = lane; k < N; k += 32) {
                    const int kz = k / (B * B), rem = k - kz * B * B, ky = rem / B, kx = rem - ky * B;
                    const double di =
                        (double)pre[((size_t)(cz - H + kz) * ny + (cy - H + ky)) * nx + (cx - H + kx)] - bc.ibar;
                    const float jf = intra[((size_t)(cz + dz - H + kz) * ny + (cy + dy - H + ky)) * nx + (cx + dx - H + kx)];
                    const double jd = (double)jf;
                    sij = fma(di, jd, sij);
                    sj += jd;
                    sjj = fma(jd, jd, sjj);
                    lo = fminf(lo, jf);
                    hi = fmaxf(hi, jf);
                }
                sij = warp_sum(sij);
                sj = warp_sum(sj);
                sjj = warp_sum(sjj);
                lo = warp_min_f(lo);
                hi = warp_max_f(hi);
                if (lane == 0 && lo < hi) {
                    const double vJ = sjj - sj * sj / (double)N;
                    if (vJ > 0.0) {
                        c.s = sij / sqrt(bc.dvI * vJ);
                        c.ok = 1;
                    }
                }
            }
            if (lane == 0 && cand_better(c, wb)) wb = c;
        }
        if (lane == 0) {
            sc->bs[warp] = wb.s;
            sc->bn2[warp] = wb.n2;
            sc->bcode[warp] = wb.code;
            sc->bok[warp] = wb.ok;
        }
        __syncthreads();
        if (tid == 0) {
            Cand best{0.0, 0, 0, 0};
            for (int w = 0; w < nwarp; ++w) {
                Cand c{sc->bs[w], sc->bn2[w], sc->bcode[w], sc->bok[w]};
                if (cand_better(c, best)) best = c;
            }
            write_result(J, bi, best, P, py, RX, ry, rz);
        }
        __syncthreads();
    }
    // a copy issued for a block this CTA never reached cannot exist: copies
    // are only issued for blocks < n that the loop visits next.
}

// Host side: launch one (element type, block size, x-shift count) variant.
template <typename T, int B, int P>
nrr_status launch_match_variant(const MatchLaunch &m, cudaStream_t stream)
{
    constexpr int ALIGN = 16 / (int)sizeof(T);
    constexpr int WX = B + P - 1;
    const int ry = m.radius[1], rz = m.radius[2], py = 2 * ry + 1, pz = 2 * rz + 1;
    const int wy = B + 2 * ry, wz = B + 2 * rz;
    const int bx = round_up_i(WX + ALIGN - 1, ALIGN);
    const int btx = round_up_i(B + ALIGN - 1, ALIGN);
    const int pf = match_pitch(WX);
    const MatchLayout L = match_layout((int)sizeof(T), B, P, bx, btx, pf, wy, wz, py, pz);
    const int lines = py * pz;
    const int threads = round_up_i(lines, 32);
    if (threads > MATCH_MAX_THREADS) return fail(NRR_E_INVALID, "search window too large");

    CUtensorMap mapJ, mapI;
    nrr_status st = encode_volume_map(&mapJ, m.intraop, m.dtype, m.dims, bx, wy, wz);
    if (st != NRR_OK) return st;
    st = encode_volume_map(&mapI, m.preop, m.dtype, m.dims, btx, B, B);
    if (st != NRR_OK) return st;

    auto kern = match_kernel<T, B, P>;
    static int smem_set = 0;  // largest dynamic shared memory opted in so far
    if (L.total > smem_set) {
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, L.total);
        if (e == cudaSuccess)
            e = cudaFuncSetAttribute(kern, cudaFuncAttributePreferredSharedMemoryCarveout, cudaSharedmemCarveoutMaxShared);
        if (e != cudaSuccess) return cuda_fail(e, "cudaFuncSetAttribute(match_kernel)");
        smem_set = L.total;
    }
    int occ = 0;
    cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, threads, L.total);
    if (e != cudaSuccess) return cuda_fail(e, "cudaOccupancyMaxActiveBlocksPerMultiprocessor");
    if (occ < 1) return fail(NRR_E_INVALID, "match kernel does not fit on an SM (%d B shared)", L.total);
    if (m.ctas_per_sm > 0 && m.ctas_per_sm < occ) occ = m.ctas_per_sm;
    long long cap = 0;
    for (int j = 0; j < m.n_jobs; ++j) cap += m.jobs[j].cap;
    long long grid = (long long)occ * sm_count();
    if (grid > cap) grid = cap;
    if (grid < 1) return NRR_OK;

    MatchParams p;
    p.preop = m.preop;
    p.intraop = m.intraop;
    p.s1 = m.s1;
    p.s2 = m.s2;
    p.nx = m.dims.nx;
    p.ny = m.dims.ny;
    p.nz = m.dims.nz;
    p.ry = ry;
    p.rz = rz;
    p.bx = bx;
    p.btx = btx;
    p.pf = pf;
    p.n_jobs = m.n_jobs;
    for (int j = 0; j < MATCH_MAX_JOBS; ++j) p.jobs[j] = j < m.n_jobs ? m.jobs[j] : MatchJob{};
    p.err = m.err;
    kern<<<(unsigned)grid, threads, L.total, stream>>>(p, mapJ, mapI);
    e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "match kernel launch");
    count_launches(1);
    return NRR_OK;
}

template <typename T, int B, int P>
nrr_status occupancy_variant(const MatchLaunch &m, int *occ)
{
    constexpr int ALIGN = 16 / (int)sizeof(T);
    constexpr int WX = B + P - 1;
    const int ry = m.radius[1], rz = m.radius[2], py = 2 * ry + 1, pz = 2 * rz + 1;
    const int bx = round_up_i(WX + ALIGN - 1, ALIGN), btx = round_up_i(B + ALIGN - 1, ALIGN);
    const MatchLayout L = match_layout((int)sizeof(T), B, P, bx, btx, match_pitch(WX), B + 2 * ry, B + 2 * rz, py, pz);
    auto kern = match_kernel<T, B, P>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, L.total);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(kern, cudaFuncAttributePreferredSharedMemoryCarveout, cudaSharedmemCarveoutMaxShared);
    if (e == cudaSuccess)
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(occ, kern, round_up_i(py * pz, 32), L.total);
    if (e != cudaSuccess) return cuda_fail(e, "match occupancy query");
    return NRR_OK;
}

template <typename T, int B>
nrr_status launch_match_b(const MatchLaunch &m, cudaStream_t stream, int *occ)
{
    switch (m.radius[0]) {
#define NRR_CASE(r, p) \
    case r: return occ ? occupancy_variant<T, B, p>(m, occ) : launch_match_variant<T, B, p>(m, stream);
        NRR_CASE(0, 1)
        NRR_CASE(1, 3)
        NRR_CASE(2, 5)
        NRR_CASE(3, 7)
        NRR_CASE(4, 9)
        NRR_CASE(5, 11)
        NRR_CASE(6, 13)
        NRR_CASE(7, 15)
#undef NRR_CASE
    }
    return fail(NRR_E_INVALID, "radius x %d outside 0..7", m.radius[0]);
}

// One entry per (element type, block size); defined in the instantiation
// translation units.
nrr_status launch_match_u16_b3(const MatchLaunch &, cudaStream_t, int *);
nrr_status launch_match_u16_b5(const MatchLaunch &, cudaStream_t, int *);
nrr_status launch_match_u16_b7(const MatchLaunch &, cudaStream_t, int *);
nrr_status launch_match_u16_b9(const MatchLaunch &, cudaStream_t, int *);
nrr_status launch_match_u16_b11(const MatchLaunch &, cudaStream_t, int *);
nrr_status launch_match_f32_b3(const MatchLaunch &, cudaStream_t, int *);
nrr_status launch_match_f32_b5(const MatchLaunch &, cudaStream_t, int *);
nrr_status launch_match_f32_b7(const MatchLaunch &, cudaStream_t, int *);
nrr_status launch_match_f32_b9(const MatchLaunch &, cudaStream_t, int *);
nrr_status launch_match_f32_b11(const MatchLaunch &, cudaStream_t, int *);

}  // namespace nrr
