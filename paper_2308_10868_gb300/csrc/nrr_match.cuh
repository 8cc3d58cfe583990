// NCC block-matching kernel (Sec. 3 NCC equation and O(B x W) bound;
// Sec. 4.3 block-matching loop), written for sm_103a.
//
// A persistent CTA walks its share of the registration blocks, two blocks in
// flight: while block i is processed, the TMA copies of block i+1 land in
// the other half of a double buffer.  Per block:
//   1. TMA tiled loads bring the block's search window of the reference
//      image, [c-h-R, c+h+R] per axis, and the floating block [c-h, c+h]^3
//      into shared memory.  The x start is rounded down to a 16-byte
//      boundary (offset xo); the box is widened so that its row and plane
//      pitches make every 16-byte load of 8 consecutive threads hit 8
//      distinct bank groups.  Out-of-volume voxels arrive as zeros and are
//      excluded by coordinates.
//   2. Every warp sums a share of the floating block; each thread combines
//      the partials into the shift m (cheap, identical everywhere) and
//      thread 0 alone derives the FP64 block constants (FP64 issue is
//      scarce on this part).  The CTA stores the block mean-shifted
//      (T_k = I_k - m) as float.
//   3. Search: thread t owns one (dz, dy) line of the window and all 2*rx+1
//      shifts along x.  For every template row it reads the window row
//      straight from the TMA buffer with 16-byte loads, turns the values it
//      needs into floats shifted by a per-block constant c (J'_k = J_k - c;
//      for uint16 one byte-permute per value, then the subtraction two
//      values at a time as packed f32x2, exact), and
//      accumulates A(d) = sum_k T_k J'_{k+d} with FP32 FFMA, fully unrolled
//      over the row and the x shifts.  The offset xo is a compile-time
//      parameter of the loop, so every register index is static.
//   4. Every shift gets an approximate NCC from A(d) and the box sums S_J,
//      S_JJ (precomputed, exact for uint16) together with a rigorous bound on
//      its error (recursive-summation bound gamma_N * sum|T||J'| for the FFMA
//      chain, Cauchy-Schwarz sum|T||J'| <= sqrt(sum T^2 * sum J'^2), plus the
//      rounding of the final operations; doubled for margin).
//   5. Shifts whose upper bound reaches the best lower bound survive (about
//      one per block on the phantoms) and are rescored: a warp per survivor
//      (float32 with fewer survivors than warps: each survivor's terms split
//      over several warps).  uint16 -> exact int64 sums, then the canonical
//      FP64 ratio num / sqrt(vI * vJ); float32 -> Pearson sums in
//      float-float pairs and one FP64 ratio.  The best survivor under the
//      tie-break rule is the block's answer.
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
    int wyp;  // rows per plane of the window box (>= window height)
    int n_jobs;
    int single_window;  // one window buffer: the next block's copy is issued once this block's window is read
    int by, bz;         // block edges along y and z (the x edge is the template parameter B)
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
    float ibh, ibl; // float32: the mean as a float pair (ibh + ibl)
    float fvI;      // vI as float
    float frr;      // uint16: rr as float (exact: |rr| <= N/2)
    float kq;       // uint16: N*gamma_N*sqrt(sum T^2); float32: sqrt(sum T^2) (rounded up)
    float mu;       // float32: float mean used for T
    float emu;      // float32: Ibar - mu
    int m;          // uint16: integer mean used for T
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
    // per-warp partial statistics of the floating block
    double pd1[MATCH_MAX_WARPS], pd2[MATCH_MAX_WARPS];
    float plo[MATCH_MAX_WARPS], phi[MATCH_MAX_WARPS];
    // float32: per-warp partial sums when few survivors are split across warps
    double rf[MATCH_MAX_WARPS][3];
    float rlo[MATCH_MAX_WARPS], rhi[MATCH_MAX_WARPS];
};

// Extra radius levels (level-aware kernel only): per-warp lower bounds and
// per-warp best survivors of each level.
struct MatchLevelScratch {
    float wlbl[MATCH_MAX_LEVELS][MATCH_MAX_WARPS];
    double lbs[MATCH_MAX_LEVELS][MATCH_MAX_WARPS];
    int lbn2[MATCH_MAX_LEVELS][MATCH_MAX_WARPS], lbcode[MATCH_MAX_LEVELS][MATCH_MAX_WARPS],
        lbok[MATCH_MAX_LEVELS][MATCH_MAX_WARPS];
};

__host__ __device__ constexpr int round_up_c(int v, int a) { return (v + a - 1) / a * a; }
__host__ __device__ inline int round_up_i(int v, int a) { return (v + a - 1) / a * a; }

// Row pitch (elements) of the window box: covers the WX needed values from
// any start offset below one 16-byte chunk, and is an odd number of 16-byte
// chunks, so 8 consecutive rows start in 8 distinct bank groups.
template <typename T, int B, int P>
__host__ __device__ constexpr int match_bx()
{
    constexpr int EPC = 16 / (int)sizeof(T);
    constexpr int c = (B + P - 1 + EPC - 1 + EPC - 1) / EPC;  // chunks
    return EPC * (c % 2 ? c : c + 1);
}

// Rows per plane of the window box.  Consecutive threads own consecutive
// (dz, dy) lines; their rows are 1 apart except at the wrap from dy = py-1
// to the next dz, where they are wyp - py + 1 apart.  With an odd number of
// chunks per row, both steps map to the same bank-group step iff
// wyp == py (mod 8).
__host__ __device__ inline int match_wyp(int wy, int py)
{
    int w = wy;
    while ((w - py) % 8 != 0) ++w;
    return w;
}

struct MatchLayout {
    int u[2], ut[2], t, surv, sc, lsc, bar, total;
};

// Shared-memory carve-up of one CTA (all offsets 128-byte aligned).  With
// single_window the two blocks in flight share one window buffer (their
// floating blocks stay double-buffered); `levels` adds the level scratch.
__host__ __device__ inline MatchLayout match_layout(int elem, int B, int P, int bx, int btx, int wyp, int wz, int py,
                                                   int pz, bool single_window, bool levels, int brows)
{
    // brows: rows of the floating block (by * bz)
    MatchLayout L;
    const int pt = round_up_i(B, 4);
    int o = 0;
    for (int b = 0; b < 2; ++b) {
        if (single_window && b == 1) {
            L.u[1] = L.u[0];
        } else {
            L.u[b] = o;
            o += round_up_i(bx * wyp * wz * elem, 128);
        }
        L.ut[b] = o;
        o += round_up_i(btx * brows * elem, 128);
    }
    L.t = o;
    o += round_up_i(brows * pt * 4, 128);
    L.surv = o;
    o += round_up_i(P * py * pz * 2, 128);
    L.sc = o;
    o += round_up_i((int)sizeof(MatchScratch), 128);
    L.lsc = o;
    if (levels) o += round_up_i((int)sizeof(MatchLevelScratch), 128);
    L.bar = o;
    o += 128;
    L.total = o;
    return L;
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

// Float-float sums (a value h + l with |l| <= ulp(h)/2): the float32 path's
// statistics and rescoring accumulate in pairs of floats on the FP32 pipe
// instead of in FP64 (narrow on this part).  Products of two floats are exact
// as p + fma(x, y, -p); a sum is Knuth's branch-free two-sum of the high
// parts, the low terms added, then renormalised (Dekker's fast two-sum), so
// each step errs by about 2^-48 relative and sums of integers below 2^48 are
// exact -- far below the 1e-6 NCC tolerance.
struct FF {
    float h, l;
};
__device__ __forceinline__ void two_sum(float a, float b, float &s, float &e)
{
    s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}
__device__ __forceinline__ FF ff_norm(float s, float e)  // |s| >= |e|
{
    const float h = __fadd_rn(s, e);
    return FF{h, __fsub_rn(e, __fsub_rn(h, s))};
}
__device__ __forceinline__ FF ff_add(FF a, float b)
{
    float s, e;
    two_sum(a.h, b, s, e);
    return ff_norm(s, __fadd_rn(e, a.l));
}
__device__ __forceinline__ FF ff_add2(FF a, float b, float c)  // a + b + c, |c| tiny next to b
{
    float s, e;
    two_sum(a.h, b, s, e);
    return ff_norm(s, __fadd_rn(__fadd_rn(e, a.l), c));
}
__device__ __forceinline__ FF ff_add_prod(FF a, float x, float y)  // a + x*y
{
    const float p = __fmul_rn(x, y);
    return ff_add2(a, p, __fmaf_rn(x, y, -p));
}
__device__ __forceinline__ FF ff_add_ff(FF a, FF b)
{
    float s, e;
    two_sum(a.h, b.h, s, e);
    return ff_norm(s, __fadd_rn(__fadd_rn(e, a.l), b.l));
}
__device__ __forceinline__ FF warp_sum_ff(FF v)
{
#pragma unroll
    for (int o = 16; o; o >>= 1) {
        FF w{__shfl_xor_sync(0xffffffffu, v.h, o), __shfl_xor_sync(0xffffffffu, v.l, o)};
        v = ff_add_ff(v, w);
    }
    return v;
}
__device__ __forceinline__ double ff_to_double(FF v) { return (double)v.h + (double)v.l; }

// Exact uint16 -> float of (u - c) for u, c < 2^16: 0x4B000000|u is the float
// 2^23 + u, so one integer OR and one float subtraction suffice.
__device__ __forceinline__ float u16_minus(uint32_t u, float c_plus_2p23)
{
    return __fsub_rn(__uint_as_float(0x4B000000u | u), c_plus_2p23);
}

__device__ __forceinline__ void write_out(int32_t *disp, double *ncc, uint8_t *valid, int blk, const Cand &b, int P,
                                          int py, int rx, int ry, int rz)
{
    if (b.ok) {
        int dxi = b.code % P, dyi = (b.code / P) % py, dzi = b.code / (P * py);
        disp[3 * blk + 0] = dxi - rx;
        disp[3 * blk + 1] = dyi - ry;
        disp[3 * blk + 2] = dzi - rz;
        ncc[blk] = b.s;
        valid[blk] = 1;
    } else {
        disp[3 * blk + 0] = 0;
        disp[3 * blk + 1] = 0;
        disp[3 * blk + 2] = 0;
        ncc[blk] = __longlong_as_double(0x7ff8000000000000ll);
        valid[blk] = 0;
    }
}
__device__ __forceinline__ void write_result(const MatchJob &a, int blk, const Cand &b, int P, int py, int rx, int ry,
                                             int rz)
{
    write_out(a.disp, a.ncc, a.valid, blk, b, P, py, rx, ry, rz);
}
// A block with no candidate shift: invalid in its own radius and every level.
__device__ __forceinline__ void write_invalid(const MatchJob &a, int blk, int P, int py, int rx, int ry, int rz)
{
    const Cand none{0.0, 0, 0, 0};
    write_out(a.disp, a.ncc, a.valid, blk, none, P, py, rx, ry, rz);
    for (int l = 0; l < a.n_levels; ++l)
        write_out(a.levels[l].disp, a.levels[l].ncc, a.levels[l].valid, blk, none, P, py, rx, ry, rz);
}
// Shift `code` (x fastest, P x-shifts, py y-shifts) lies in level box r.
__device__ __forceinline__ bool in_level(int code, const int32_t (&r)[3], int P, int py, int rx, int ry, int rz)
{
    const int dx = code % P - rx, dy = (code / P) % py - ry, dz = code / (P * py) - rz;
    return abs(dx) <= r[0] && abs(dy) <= r[1] && abs(dz) <= r[2];
}

__device__ __forceinline__ bool center_inside(int cx, int cy, int cz, int nx, int ny, int nz, int hx, int hy, int hz)
{
    return cx >= hx && cy >= hy && cz >= hz && cx <= nx - 1 - hx && cy <= ny - 1 - hy && cz <= nz - 1 - hz;
}

// The search of one thread's line for a window whose row data starts XO
// elements into each row of the box.  `row0` points at the thread's first
// row; rows of the next template row are one box row apart, template planes
// `zstride` elements apart.
template <typename T, int B, int P, int XO>
__device__ __forceinline__ void search_line(const T *row0, int zstride, const float *Tm, float csh, float (&acc)[P],
                                            int by, int bz)
{
    constexpr bool F32 = std::is_same<T, float>::value;
    constexpr int WX = B + P - 1;
    constexpr int EPC = 16 / (int)sizeof(T);
    constexpr int NC = (XO + WX - 1) / EPC + 1;  // 16-byte chunks covering [XO, XO + WX)
    constexpr int PT = (B + 3) / 4 * 4;
    constexpr int BX = match_bx<T, B, P>();
    unsigned long long negc2;  // (-csh, -csh) as one f32x2 operand
    asm("mov.b64 %0, {%1, %1};" : "=l"(negc2) : "f"(-csh));
#pragma unroll 1
    for (int kz = 0; kz < bz; ++kz) {
#pragma unroll 1
        for (int ky = 0; ky < by; ++ky) {
            const T *row = row0 + kz * zstride + ky * BX;
            const float *tr = Tm + (kz * by + ky) * PT;
            uint4 ch[NC];
#pragma unroll
            for (int c = 0; c < NC; ++c) ch[c] = *reinterpret_cast<const uint4 *>(row + c * EPC);
            float t[PT];
#pragma unroll
            for (int q = 0; q < PT / 4; ++q) {
                const float4 v = *reinterpret_cast<const float4 *>(tr + 4 * q);
                t[4 * q + 0] = v.x;
                t[4 * q + 1] = v.y;
                t[4 * q + 2] = v.z;
                t[4 * q + 3] = v.w;
            }
            // the raw bits of each value as a float: uint16 as 0x4B00|u, the
            // float 2^23 + u (one byte-permute), float32 as it is
            uint32_t raw[WX];
#pragma unroll
            for (int e = 0; e < WX; ++e) {
                const int E = XO + e;  // element within the loaded chunks (compile-time after unrolling)
                const uint4 &q = ch[E / EPC];
                if constexpr (F32) {
                    const int w = E % 4;
                    raw[e] = w == 0 ? q.x : w == 1 ? q.y : w == 2 ? q.z : q.w;
                } else {
                    const int w = (E % 8) / 2;
                    const uint32_t word = w == 0 ? q.x : w == 1 ? q.y : w == 2 ? q.z : q.w;
                    raw[e] = (E & 1) ? __byte_perm(word, 0x4B00u, 0x5432) : __byte_perm(word, 0x4B00u, 0x5410);
                }
            }
            // minus the centring constant (2^23 + c for uint16, so u - c
            // exactly), two values per packed f32x2 subtraction
            float j[WX];
#pragma unroll
            for (int e = 0; e + 1 < WX; e += 2) {
                unsigned long long d;
                asm("{\n\t.reg .b64 pa;\n\t"
                    "mov.b64 pa, {%1, %2};\n\t"
                    "add.rn.f32x2 %0, pa, %3;\n\t}"
                    : "=l"(d)
                    : "r"(raw[e]), "r"(raw[e + 1]), "l"(negc2));
                j[e] = __uint_as_float((uint32_t)d);
                j[e + 1] = __uint_as_float((uint32_t)(d >> 32));
            }
            if constexpr (WX & 1) j[WX - 1] = __fsub_rn(__uint_as_float(raw[WX - 1]), csh);
#pragma unroll
            for (int kx = 0; kx < B; ++kx)
#pragma unroll
                for (int p = 0; p < P; ++p) acc[p] = __fmaf_rn(t[kx], j[kx + p], acc[p]);
        }
    }
}

// The kernel body; the __global__ entries below differ only in their
// register budget.  `a`, `tmapJ` and `tmapI` live in kernel-parameter space.
// LEV: the jobs may report extra radius levels (batched search); without it
// that code is compiled out of the search's per-shift loops.  ANI: the block
// edges along y and z (a.by, a.bz) may differ from the x edge B; without it
// they are B and every size below is a compile-time constant.
template <typename T, int B, int P, bool LEV, bool ANI>
__device__ __forceinline__ void match_body(const MatchParams &a, const CUtensorMap *tmapJ, const CUtensorMap *tmapI)
{
    constexpr bool F32 = std::is_same<T, float>::value;
    constexpr int H = (B - 1) / 2;  // x half edge
    constexpr int N3 = B * B * B;   // terms of a cubic block
    const int BY = ANI ? a.by : B, BZ = ANI ? a.bz : B;
    const int HY = (BY - 1) / 2, HZ = (BZ - 1) / 2;
    const int N = ANI ? B * BY * BZ : N3;
    constexpr int PT = (B + 3) / 4 * 4;
    constexpr int RX = (P - 1) / 2;
    constexpr int ALIGN = 16 / (int)sizeof(T);
    constexpr int BX = match_bx<T, B, P>();
    constexpr int BTX = round_up_c(B + ALIGN - 1, ALIGN);
    constexpr float U32 = 5.9604644775390625e-08f;  // 2^-24, unit roundoff of binary32
    const double GAMMA_N = (double)N * 5.9604644775390625e-08 / (1.0 - (double)N * 5.9604644775390625e-08);

    const int ry = a.ry, rz = a.rz, py = 2 * ry + 1, pz = 2 * rz + 1, lines = py * pz;
    const int wz = BZ + 2 * rz, wyp = a.wyp;
    const int nx = a.nx, ny = a.ny, nz = a.nz;

    extern __shared__ __align__(128) unsigned char smem[];
    const MatchLayout L =
        match_layout((int)sizeof(T), B, P, BX, BTX, wyp, wz, py, pz, a.single_window != 0, LEV, BY * BZ);
    const bool single = a.single_window != 0;
    float *Tm = reinterpret_cast<float *>(smem + L.t);
    uint16_t *surv = reinterpret_cast<uint16_t *>(smem + L.surv);
    MatchScratch *sc = reinterpret_cast<MatchScratch *>(smem + L.sc);
    MatchLevelScratch *ls = reinterpret_cast<MatchLevelScratch *>(smem + L.lsc);  // LEV only
    uint64_t *bar = reinterpret_cast<uint64_t *>(smem + L.bar);  // [2]

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
        mbar_init(bar + 0, 1);
        mbar_init(bar + 1, 1);
        fence_mbar_init();
    }
    __syncthreads();
    const int n = sc->jstart[a.n_jobs];  // work items over all jobs
    auto locate = [&](int w, int &j, int &i) {
        j = 0;
        while (j + 1 < a.n_jobs && w >= sc->jstart[j + 1]) ++j;
        i = w - sc->jstart[j];
    };
    auto centre = [&](int w, int &cx, int &cy, int &cz) {
        int j, i;
        locate(w, j, i);
        const int32_t *c = a.jobs[j].centers + 3 * i;
        cx = c[0];
        cy = c[1];
        cz = c[2];
    };
    // next work item of this CTA at or after w whose centre is inside;
    // thread 0 reports the skipped ones as invalid
    auto next_inside = [&](int w) {
        for (; w < n; w += gridDim.x) {
            int cx, cy, cz;
            centre(w, cx, cy, cz);
            if (center_inside(cx, cy, cz, nx, ny, nz, H, HY, HZ)) return w;
            if (tid == 0) {
                int j, i;
                locate(w, j, i);
                write_invalid(a.jobs[j], i, P, py, RX, ry, rz);
            }
        }
        return n;
    };
    const uint32_t tx_bytes = (uint32_t)((BX * wyp * wz + BTX * BY * BZ) * (int)sizeof(T));
    // thread 0: both copies of block w into buffer b
    auto issue = [&](int w, int b) {
        int cx, cy, cz;
        centre(w, cx, cy, cz);
        const int x0 = cx - H - RX, xt = cx - H;
        fence_proxy_async_smem();
        mbar_arrive_expect_tx(bar + b, tx_bytes);
        tma_load_3d(smem + L.u[b], tmapJ, bar + b, x0 & ~(ALIGN - 1), cy - HY - ry, cz - HZ - rz);
        tma_load_3d(smem + L.ut[b], tmapI, bar + b, xt & ~(ALIGN - 1), cy - HY, cz - HZ);
    };

    uint32_t phase[2] = {0u, 0u};
    int i = 0;
    int blk = next_inside(blockIdx.x);
    if (blk < n && tid == 0) issue(blk, 0);
    while (blk < n) {
        const int b = i & 1;
        const T *U = reinterpret_cast<const T *>(smem + L.u[b]);
        const T *Ut = reinterpret_cast<const T *>(smem + L.ut[b]);
        int job, bi;
        locate(blk, job, bi);
        const MatchJob &J = a.jobs[job];
        const int cx = J.centers[3 * bi + 0], cy = J.centers[3 * bi + 1], cz = J.centers[3 * bi + 2];
        const int x0 = cx - H - RX, xo = x0 - (x0 & ~(ALIGN - 1));
        const int xt = cx - H, xot = xt - (xt & ~(ALIGN - 1));
        const size_t cidx = ((size_t)cz * ny + cy) * nx + cx;
        // window centring constant from the box sum at the centre
        float cshift;  // subtracted from the float of each window value (2^23 folded in for uint16)
        int c_i = 0;
        float c_f = 0.f;
        if constexpr (F32) {
            c_f = __fdiv_rn(reinterpret_cast<const float *>(a.s1)[cidx], (float)N);
            cshift = c_f;
        } else {
            const long long s1c = reinterpret_cast<const int32_t *>(a.s1)[cidx];
            c_i = (int)((2u * (uint32_t)s1c + (uint32_t)N) / (2u * (uint32_t)N));
            cshift = 8388608.0f + (float)c_i;
        }
        if (tid == 0) sc->nsurv = 0;

        // ---- wait for this block's copies; start the next block's --------
        const bool got = mbar_wait_bounded(bar + b, phase[b], WAIT_LIMIT_NS);
        if (!__syncthreads_and(got)) {
            if (tid == 0) {
                atomicOr(a.err, DEV_ERR_TIMEOUT);
                write_invalid(J, bi, P, py, RX, ry, rz);
            }
            mbar_wait_bounded(bar + b, phase[b], WAIT_LIMIT_NS);  // let an in-flight copy land before exiting
            return;
        }
        phase[b] ^= 1u;
        const int nb = next_inside(blk + gridDim.x);
        // buffer b^1 was released by the previous block's last barrier; a
        // shared window buffer is refilled only once this block has read it
        if (!single && nb < n && tid == 0) issue(nb, b ^ 1);

        // ---- floating block statistics.  Every warp sums a share (float32 in
        // float-float, uint16 in exact integers) and every thread combines the
        // per-warp partials after the barrier ----
        {
            constexpr int IPT = ANI ? 1 : (N3 + 63) / 64;  // values per thread at 64+ threads
            if constexpr (F32) {
                // sums of (I - I0) and (I - I0)^2 with I0 the block's first
                // value (shifted data: the spread loses no digits to
                // cancellation), in float-float; I - I0 is exact as dh + de
                const float i0 = Ut[xot];
                FF s1{0.f, 0.f}, s2{0.f, 0.f};
                float lo = INFINITY, hi = -INFINITY;
                for (int k0 = tid; k0 < N; k0 += IPT * nthr) {
                    float vals[IPT];
#pragma unroll
                    for (int q = 0; q < IPT; ++q) {
                        const int k = k0 + q * nthr;
                        const int kzy = k / B, kx = k - kzy * B;
                        vals[q] = k < N ? Ut[kzy * BTX + xot + kx] : 0.f;
                    }
#pragma unroll
                    for (int q = 0; q < IPT; ++q)
                        if (k0 + q * nthr < N) {
                            float dh, de;
                            two_sum(vals[q], -i0, dh, de);
                            s1 = ff_add2(s1, dh, de);
                            const float p = __fmul_rn(dh, dh);  // (dh + de)^2; de^2 is below the pair's precision
                            s2 = ff_add2(s2, p, __fmaf_rn(2.f * dh, de, __fmaf_rn(dh, dh, -p)));
                            lo = fminf(lo, vals[q]);
                            hi = fmaxf(hi, vals[q]);
                        }
                }
                s1 = warp_sum_ff(s1);
                s2 = warp_sum_ff(s2);
                lo = warp_min_f(lo);
                hi = warp_max_f(hi);
                if (lane == 0) {
                    sc->pd1[warp] = ff_to_double(s1);
                    sc->pd2[warp] = ff_to_double(s2);
                    sc->plo[warp] = lo;
                    sc->phi[warp] = hi;
                }
            } else {  // uint16: every warp sums a share (exact integer sums)
                constexpr int KPT = ANI ? 0 : (N3 + 63) / 64;
                long long s1 = 0;
                unsigned long long s2 = 0;
#pragma unroll
                for (int q = 0; q < KPT; ++q) {
                    const int k = tid + q * nthr;
                    const int kzy = k / B, kx = k - kzy * B;
                    const uint32_t v = k < N ? (uint32_t)Ut[kzy * BTX + xot + kx] : 0u;
                    s1 += v;
                    s2 += (unsigned long long)(v * v);
                }
                for (int k = tid + KPT * nthr; k < N; k += nthr) {  // fewer than 64 threads
                    const int kzy = k / B, kx = k - kzy * B;
                    const uint32_t v = (uint32_t)Ut[kzy * BTX + xot + kx];
                    s1 += v;
                    s2 += (unsigned long long)(v * v);
                }
                s1 = warp_sum(s1);
                s2 = warp_sum(s2);
                if (lane == 0) {
                    reinterpret_cast<long long *>(sc->pd1)[warp] = s1;
                    reinterpret_cast<long long *>(sc->pd2)[warp] = (long long)s2;
                }
            }
        }
        __syncthreads();
        // float32: every thread needs only the template shift and the flat
        // test, both cheap and computed identically everywhere; thread 0
        // alone derives the FP64 block constants (FP64 issue is scarce on
        // this part), read by all threads after the next barrier.
        float tsh;
        bool flat;
        if constexpr (F32) {
            float sf = 0.f, lo = INFINITY, hi = -INFINITY;
            for (int w = 0; w < nwarp; ++w) {
                sf += (float)sc->pd1[w];
                lo = fminf(lo, sc->plo[w]);
                hi = fmaxf(hi, sc->phi[w]);
            }
            // any float near the mean serves as the shift mu (the partials
            // are sums of I - I0)
            tsh = __fadd_rn(Ut[xot], __fmul_rn(sf, 1.0f / (float)N));
            flat = !(lo < hi);
            if (tid == 0 && !flat) {
                double s1 = 0.0, s2 = 0.0;  // sums of (I - I0) and (I - I0)^2
                for (int w = 0; w < nwarp; ++w) {
                    s1 += sc->pd1[w];
                    s2 += sc->pd2[w];
                }
                const double i0 = (double)Ut[xot];
                const double ibar = i0 + s1 / (double)N;
                double dv = s2 - s1 * (s1 / (double)N);  // sum (I - Ibar)^2
                if (dv < 0.0) dv = 0.0;
                sc->bc.ibh = (float)ibar;
                sc->bc.ibl = (float)(ibar - (double)sc->bc.ibh);
                const double em = ibar - (double)tsh;
                BlockConst &c = sc->bc;
                c.ibar = ibar;
                c.mu = tsh;
                c.emu = (float)em;
                c.dvI = dv;
                c.fvI = (float)dv;
                // sum of T^2 with T = fl(I - mu): at most (1+u)^2 sum (I - mu)^2
                // = (1+u)^2 (sum (I - Ibar)^2 + N (Ibar - mu)^2); the
                // float-float sums (about 2^-48 relative per step, tens of
                // steps) leave the spread inexact by well under 2048 ulp of s2
                c.kq = (float)(sqrt((dv + 2048.0 * 1.1102230246251565e-16 * s2 + (double)N * em * em) * (1.0 + 2.4e-7)) *
                               (1.0 + 1e-6));
            }
        } else {
            // uint16: every thread adds the per-warp partials (exact) and
            // derives the integer mean; thread 0 writes the block constants
            long long s1 = 0, s2 = 0;
            for (int w = 0; w < nwarp; ++w) {
                s1 += reinterpret_cast<const long long *>(sc->pd1)[w];
                s2 += reinterpret_cast<const long long *>(sc->pd2)[w];
            }
            const long long vI = (long long)N * s2 - s1 * s1;
            const long long m = (long long)((2u * (uint32_t)s1 + (uint32_t)N) / (2u * (uint32_t)N));  // nearest integer to the mean
            flat = vI == 0;
            tsh = 8388608.0f + (float)(int)m;
            if (tid == 0) {
                BlockConst &c = sc->bc;
                const long long qt = s2 - 2 * m * s1 + (long long)N * m * m;  // sum (I-m)^2, exact, below 2^48
                c.vI = vI;
                c.m = (int)m;
                c.rr = (long long)N * m - s1;
                c.frr = (float)(int)c.rr;
                c.fvI = (float)vI;
                // kq = N gamma_N sqrt(qt), rounded up in float (no FP64 on this
                // path): qt < 2^48 becomes a float through two exact 24-bit
                // halves and one rounding; the factor 1 + 4e-6 covers that
                // rounding and the rounding of N gamma_N
                const float qf = __fmaf_rn((float)(int)(qt >> 24), 16777216.f, (float)(int)(qt & 0xFFFFFF));
                c.kq = __fmul_ru(__fmul_ru((float)((double)N * GAMMA_N), __fsqrt_ru(qf)), 1.000004f);
            }
        }
        if (flat) {  // flat floating block: NCC undefined for every shift
            if (single && nb < n && tid == 0) issue(nb, b ^ 1);  // the window is not read
            if (tid == 0) write_invalid(J, bi, P, py, RX, ry, rz);
            __syncthreads();
            blk = nb;
            ++i;
            continue;
        }
        // ---- mean-shifted template (loads batched before stores) -----------
        {
            const int TB = BY * BZ * PT;
            constexpr int TPT = ANI ? 0 : (B * B * PT + 63) / 64;  // items per thread at 64+ threads
            float v[TPT > 0 ? TPT : 1];
#pragma unroll
            for (int j = 0; j < TPT; ++j) {
                const int k = tid + j * nthr;
                const int kzy = k / PT, kx = k - kzy * PT;
                v[j] = 0.f;
                if (k < TB && kx < B) {
                    if constexpr (F32)
                        v[j] = __fsub_rn(Ut[kzy * BTX + xot + kx], tsh);
                    else
                        v[j] = u16_minus(Ut[kzy * BTX + xot + kx], tsh);
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
                        w = __fsub_rn(Ut[kzy * BTX + xot + kx], tsh);
                    else
                        w = u16_minus(Ut[kzy * BTX + xot + kx], tsh);
                }
                Tm[k] = w;
            }
        }
        __syncthreads();
        const BlockConst bc = sc->bc;

        // ---- search: FP32 accumulation of A(d) over the whole window ------
        float ub[P];
        float lbm = -INFINITY;
        const int dyi = tid % py, dzi = tid / py;
        const int nl = LEV ? J.n_levels : 0;  // extra radius levels of this block's job
        float lbl[MATCH_MAX_LEVELS];
        unsigned int lvl_line = 0;  // bit l: this thread's (dz, dy) line lies in level l
        if constexpr (LEV) {
#pragma unroll
            for (int l = 0; l < MATCH_MAX_LEVELS; ++l) {
                lbl[l] = -INFINITY;
                if (l < nl && tid < lines && abs(dyi - ry) <= J.levels[l].r[1] && abs(dzi - rz) <= J.levels[l].r[2])
                    lvl_line |= 1u << l;
            }
        }
        if (tid < lines) {
            const int dy = dyi - ry, dz = dzi - rz, Y = cy + dy, Z = cz + dz;
            const bool yz_ok = Y >= HY && Y <= ny - 1 - HY && Z >= HZ && Z <= nz - 1 - HZ;
            typedef typename std::conditional<F32, float, int32_t>::type S1T;
            typedef float S2T;  // uint16: v_J = N S_JJ - S_J^2 rounded to float; float32: S_JJ
            float acc[P];
#pragma unroll
            for (int p = 0; p < P; ++p) acc[p] = 0.f;
            const T *row0 = U + (dzi * wyp + dyi) * BX;
            const int zs = wyp * BX;
            switch (xo) {
#define NRR_XO(k) \
    case k:       \
        if constexpr (k < ALIGN) search_line<T, B, P, k>(row0, zs, Tm, cshift, acc, BY, BZ); \
        break;
                NRR_XO(0)
                NRR_XO(1)
                NRR_XO(2)
                NRR_XO(3)
                NRR_XO(4)
                NRR_XO(5)
                NRR_XO(6)
                NRR_XO(7)
#undef NRR_XO
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
                    // 32-bit integer and float arithmetic only: a 64-bit
                    // integer to float conversion issues on the FP64 pipe,
                    // which is narrow on this part.  v_J arrives rounded once
                    // (zero only for a flat block); S'_J = S_J - N c is exact.
                    const float vjf = ps2[p];
                    if (!(vjf > 0.f)) continue;  // flat reference block
                    const int s1p = ps1[p] - N * c_i;
                    const float s1pf = (float)s1p;
                    // sum (J - c)^2 = (v_J + S'_J^2) / N, rounded up: the
                    // rounded v_J and S'_J and three operations stay below 6u
                    const float s2p = __fmul_rn(__fmul_rn(__fmaf_rn(s1pf, s1pf, vjf), 1.0f / fN), 1.f + 16.f * U32);
                    // rsqrt.approx and sqrt.approx (relative error below 2^-22
                    // over the whole range) instead of the correctly rounded
                    // forms: the factor 1 + 64u on the error terms and 40u|v|
                    // for the centre value absorb their error
                    float inv;
                    asm("rsqrt.approx.f32 %0, %1;" : "=f"(inv) : "f"(__fmul_rn(bc.fvI, vjf)));
                    const float na = __fmul_rn(fN, acc[p]);
                    const float rs = __fmul_rn(bc.frr, s1pf);  // rr exact in float (|rr| <= N/2)
                    const float v = __fmul_rn(__fadd_rn(na, rs), inv);
                    float sq;
                    asm("sqrt.approx.f32 %0, %1;" : "=f"(sq) : "f"(s2p));
                    float e = (bc.kq * sq * inv + 4.f * U32 * (fabsf(na) + fabsf(rs)) * inv) * (1.f + 64.f * U32) +
                              40.f * U32 * fabsf(v);
                    e = 2.f * e + 1e-9f;
                    ub[p] = v + e;
                    lbm = fmaxf(lbm, v - e);
                    if (LEV && lvl_line) {
#pragma unroll
                        for (int l = 0; l < MATCH_MAX_LEVELS; ++l)
                            if (((lvl_line >> l) & 1u) && abs(p - RX) <= J.levels[l].r[0]) lbl[l] = fmaxf(lbl[l], v - e);
                    }
                } else {
                    const float GS = (float)((B + BY + BZ) * 5.9604644775390625e-08 /
                                             (1.0 - (B + BY + BZ) * 5.9604644775390625e-08));  // box-sum depth
                    const float GN = (float)GAMMA_N;
                    const float s1 = ps1[p];
                    const float s2 = fmaxf(ps2[p], 0.f);
                    float d1;  // |S1 err| bound (the factor 1.01 covers sqrt.approx)
                    asm("sqrt.approx.f32 %0, %1;" : "=f"(d1) : "f"(fN * s2));
                    d1 = GS * d1 * 1.01f;
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
                    // approximate rsqrt / sqrt as for uint16: 1 + 64u on the
                    // error terms and 40u|v| absorb their error
                    float inv, sq;
                    asm("rsqrt.approx.f32 %0, %1;" : "=f"(inv) : "f"(__fmul_rn(bc.fvI, vJa)));
                    asm("sqrt.approx.f32 %0, %1;" : "=f"(sq) : "f"(sj2));
                    const float A = acc[p];
                    const float es = __fmul_rn(bc.emu, s1p);
                    const float num = __fsub_rn(A, es);
                    const float v = __fmul_rn(num, inv);
                    const float enum_ = (GN + 3.f * U32) * bc.kq * sq +
                                        fabsf(bc.emu) * (fabsf(s1p) + d1 + 2.f * U32 * fN * fabsf(c_f)) * 1.01f +
                                        U32 * (fabsf(A) + fabsf(es));
                    float e = (enum_ * inv * (1.f + 0.7f * rho + 4.f * U32) + fabsf(num) * inv * (0.7f * rho + 6.f * U32)) *
                                  (1.f + 64.f * U32) +
                              43.f * U32 * fabsf(v);
                    e = 2.f * e + 1e-9f;
                    ub[p] = v + e;
                    lbm = fmaxf(lbm, v - e);
                    if (LEV && lvl_line) {
#pragma unroll
                        for (int l = 0; l < MATCH_MAX_LEVELS; ++l)
                            if (((lvl_line >> l) & 1u) && abs(p - RX) <= J.levels[l].r[0]) lbl[l] = fmaxf(lbl[l], v - e);
                    }
                }
            }
        }

        // ---- best lower bound over the window; survivors ------------------
        lbm = warp_max_f(lbm);
        if (lane == 0) sc->wlb[warp] = lbm;
        if (LEV && nl) {
#pragma unroll
            for (int l = 0; l < MATCH_MAX_LEVELS; ++l) {
                const float v = warp_max_f(lbl[l]);
                if (lane == 0) {
                    ls->wlbl[l][warp] = v;
                    ls->lbok[l][warp] = 0;  // this warp's best survivor in level l: none yet
                }
            }
        }
        __syncthreads();
        // float32 reads the window only in the search (its rescoring reads
        // global memory): a shared window buffer is refilled from here
        if constexpr (F32)
            if (single && nb < n && tid == 0) issue(nb, b ^ 1);
        float LB = -INFINITY;
        for (int w = 0; w < nwarp; ++w) LB = fmaxf(LB, sc->wlb[w]);
        // a shift survives if it can be the best of the whole window or of
        // a level box holding it
        float LBl[MATCH_MAX_LEVELS];
        if constexpr (LEV) {
#pragma unroll
            for (int l = 0; l < MATCH_MAX_LEVELS; ++l) {
                LBl[l] = INFINITY;
                if (l < nl) {
                    LBl[l] = -INFINITY;
                    for (int w = 0; w < nwarp; ++w) LBl[l] = fmaxf(LBl[l], ls->wlbl[l][w]);
                }
            }
        }
        if (tid < lines) {
#pragma unroll
            for (int p = 0; p < P; ++p) {
                bool lv = false;
                if (LEV && lvl_line) {
#pragma unroll
                    for (int l = 0; l < MATCH_MAX_LEVELS; ++l)
                        lv |= ((lvl_line >> l) & 1u) && abs(p - RX) <= J.levels[l].r[0] && ub[p] >= LBl[l];
                }
                if (ub[p] > -INFINITY && (ub[p] >= LB || lv)) {
                    int s = atomicAdd(&sc->nsurv, 1);
                    surv[s] = (uint16_t)((dzi * py + dyi) * P + p);
                }
            }
        }
        __syncthreads();
        const int nsurv = sc->nsurv;

        // ---- exact rescoring of the survivors ---------------------------------
        // A warp rescores a whole survivor.  float32 (FP64 sums, slow on this
        // part): with fewer survivors than warps, each survivor's terms are
        // split over nwarp/nsurv warps whose partial sums thread 0 adds up.
        const int parts = (!F32 || nsurv >= nwarp) ? 1 : (nsurv > 0 ? nwarp / nsurv : 1);
        const int KS1 = N;  // terms of a whole survivor
        Cand wb{0.0, 0, 0, 0};
        const int ntask = parts == 1 ? nsurv : nsurv * parts;
        for (int task = warp; task < ntask; task += nwarp) {
            const int sidx = task / parts, part = task - sidx * parts;
            const int ks = (KS1 + parts - 1) / parts;
            const int kbeg = part * ks, kend = kbeg + ks < N ? kbeg + ks : N;
            const int code = surv[sidx];
            const int sxi = code % P, syi = (code / P) % py, szi = code / (P * py);
            const int dx = sxi - RX, dy = syi - ry, dz = szi - rz;
            const size_t idx = ((size_t)(cz + dz) * ny + (cy + dy)) * nx + (cx + dx);
            Cand c{0.0, dx * dx + dy * dy + dz * dz, code, 0};
            if constexpr (!F32) {  // one warp per survivor: parts == 1
                long long s1 = 0;
                if (lane == 0) s1 = reinterpret_cast<const int32_t *>(a.s1)[idx];  // issued first, used after the warp sums
                const int KPL = (N + 31) / 32;
                constexpr int CH = ANI ? 6 : ((N3 + 31) / 32 < 6 ? (N3 + 31) / 32 : 6);
                long long e = 0, q2 = 0;  // sum T (J - c), sum (J - c)^2: exact
#pragma unroll 1
                for (int i0 = 0; i0 < KPL; i0 += CH) {
                    int tv[CH], jv[CH];
#pragma unroll
                    for (int q = 0; q < CH; ++q) {
                        const int k = lane + 32 * (i0 + q);
                        const int kz = k / (B * BY), rem = k - kz * B * BY, ky = rem / B, kx = rem - ky * B;
                        tv[q] = 0;
                        jv[q] = 0;
                        if (k < N) {
                            tv[q] = (int)Tm[(kz * BY + ky) * PT + kx];
                            jv[q] = (int)U[((szi + kz) * wyp + (syi + ky)) * BX + xo + sxi + kx] - c_i;
                        }
                    }
#pragma unroll
                    for (int q = 0; q < CH; ++q) {
                        e += (long long)tv[q] * jv[q];
                        q2 += (long long)jv[q] * jv[q];
                    }
                }
                e = warp_sum(e);
                q2 = warp_sum(q2);
                if (lane == 0) {
                    const long long s1p = s1 - (long long)N * c_i;  // sum (J - c)
                    const long long vJ = (long long)N * q2 - s1p * s1p;  // = N S_JJ - S_J^2, exact
                    const long long num = (long long)N * e + bc.rr * s1p;
                    if (vJ > 0) {
                        const double den = __dsqrt_rn(__dmul_rn((double)bc.vI, (double)vJ));
                        c.s = __ddiv_rn((double)num, den);
                        c.ok = 1;
                    }
                }
            } else {
                const float *pre = reinterpret_cast<const float *>(a.preop);
                const float *intra = reinterpret_cast<const float *>(a.intraop);
                // float-float sums of (I - Ibar) J, J and J^2 (FP32 pipe)
                FF fij{0.f, 0.f}, fj{0.f, 0.f}, fjj{0.f, 0.f};
                float lo = INFINITY, hi = -INFINITY;
                for (int k = kbeg + lane; k < kend; k += 32) {
                    const int kz = k / (B * BY), rem = k - kz * B * BY, ky = rem / B, kx = rem - ky * B;
                    const float iv = pre[((size_t)(cz - HZ + kz) * ny + (cy - HY + ky)) * nx + (cx - H + kx)];
                    const float jf =
                        intra[((size_t)(cz + dz - HZ + kz) * ny + (cy + dy - HY + ky)) * nx + (cx + dx - H + kx)];
                    float dh, de;
                    two_sum(iv, -bc.ibh, dh, de);  // I - Ibar = dh + dl, nearly exact
                    const float dl = __fsub_rn(de, bc.ibl);
                    const float p = __fmul_rn(dh, jf);
                    fij = ff_add2(fij, p, __fmaf_rn(dl, jf, __fmaf_rn(dh, jf, -p)));
                    fj = ff_add(fj, jf);
                    fjj = ff_add_prod(fjj, jf, jf);
                    lo = fminf(lo, jf);
                    hi = fmaxf(hi, jf);
                }
                fij = warp_sum_ff(fij);
                fj = warp_sum_ff(fj);
                fjj = warp_sum_ff(fjj);
                const double sij = ff_to_double(fij), sj = ff_to_double(fj), sjj = ff_to_double(fjj);
                lo = warp_min_f(lo);
                hi = warp_max_f(hi);
                if (lane == 0) {
                    if (parts == 1) {
                        if (lo < hi) {
                            const double vJ = sjj - sj * sj / (double)N;
                            if (vJ > 0.0) {
                                c.s = sij / sqrt(bc.dvI * vJ);
                                c.ok = 1;
                            }
                        }
                    } else {
                        sc->rf[task][0] = sij;
                        sc->rf[task][1] = sj;
                        sc->rf[task][2] = sjj;
                        sc->rlo[task] = lo;
                        sc->rhi[task] = hi;
                    }
                }
            }
            if (lane == 0 && parts == 1) {
                if (cand_better(c, wb)) wb = c;
                if constexpr (LEV)
                    for (int l = 0; l < nl; ++l)
                    if (in_level(code, J.levels[l].r, P, py, RX, ry, rz)) {
                        const Cand cur{ls->lbs[l][warp], ls->lbn2[l][warp], ls->lbcode[l][warp], ls->lbok[l][warp]};
                        if (cand_better(c, cur)) {
                            ls->lbs[l][warp] = c.s;
                            ls->lbn2[l][warp] = c.n2;
                            ls->lbcode[l][warp] = c.code;
                            ls->lbok[l][warp] = c.ok;
                        }
                    }
            }
        }
        if (lane == 0) {
            sc->bs[warp] = wb.s;
            sc->bn2[warp] = wb.n2;
            sc->bcode[warp] = wb.code;
            sc->bok[warp] = wb.ok;
        }
        __syncthreads();
        if constexpr (!F32)  // uint16 rescoring read the window up to here
            if (single && nb < n && tid == 0) issue(nb, b ^ 1);
        if (tid == 0) {
            Cand best{0.0, 0, 0, 0};
            Cand bestl[MATCH_MAX_LEVELS];
            for (int w = 0; w < nwarp; ++w) {
                Cand c{sc->bs[w], sc->bn2[w], sc->bcode[w], sc->bok[w]};
                if (cand_better(c, best)) best = c;
            }
            for (int l = 0; l < nl; ++l) {
                bestl[l] = Cand{0.0, 0, 0, 0};
                for (int w = 0; w < nwarp; ++w) {
                    Cand c{ls->lbs[l][w], ls->lbn2[l][w], ls->lbcode[l][w], ls->lbok[l][w]};
                    if (cand_better(c, bestl[l])) bestl[l] = c;
                }
            }
            if (parts > 1) {
                for (int si = 0; si < nsurv; ++si) {
                    const int code = surv[si];
                    const int sxi = code % P, syi = (code / P) % py, szi = code / (P * py);
                    const int dx = sxi - RX, dy = syi - ry, dz = szi - rz;
                    Cand c{0.0, dx * dx + dy * dy + dz * dz, code, 0};
                    if constexpr (F32) {
                        double sij = 0.0, sj = 0.0, sjj = 0.0;
                        float lo = INFINITY, hi = -INFINITY;
                        for (int q = 0; q < parts; ++q) {
                            sij += sc->rf[si * parts + q][0];
                            sj += sc->rf[si * parts + q][1];
                            sjj += sc->rf[si * parts + q][2];
                            lo = fminf(lo, sc->rlo[si * parts + q]);
                            hi = fmaxf(hi, sc->rhi[si * parts + q]);
                        }
                        if (lo < hi) {
                            const double vJ = sjj - sj * sj / (double)N;
                            if (vJ > 0.0) {
                                c.s = sij / sqrt(bc.dvI * vJ);
                                c.ok = 1;
                            }
                        }
                    }
                    if (cand_better(c, best)) best = c;
                    for (int l = 0; l < nl; ++l)
                        if (in_level(code, J.levels[l].r, P, py, RX, ry, rz) && cand_better(c, bestl[l])) bestl[l] = c;
                }
            }
            write_result(J, bi, best, P, py, RX, ry, rz);
            for (int l = 0; l < nl; ++l)
                write_out(J.levels[l].disp, J.levels[l].ncc, J.levels[l].valid, bi, bestl[l], P, py, RX, ry, rz);
        }
        __syncthreads();  // releases buffer b for the copies of the block after next
        blk = nb;
        ++i;
    }
    // every copy issued was waited for: a block's copies are issued only
    // when the loop is certain to visit it next
}

// Host side: launch one (element type, block size, x-shift count) variant.
// Register budgets.  uint16: 96 per thread for blocks up to 7^3 with up to
// 11 x-shifts (5 CTAs per SM are limited by shared memory there anyway), 128
// above.  float32: the same limits expressed as resident CTAs per SM.
template <int B, int P>
struct MatchRegs {
    static constexpr int value = (P <= 11 && B <= 7) ? 96 : 128;
};
template <int B, int P>
struct MatchMinBlocks {
    static constexpr int value = (P <= 11 && B <= 7) ? 3 : 2;
};

template <int B, int P, bool LEV, bool ANI>
__global__ void __maxnreg__((MatchRegs<B, P>::value))
    match_kernel_u16(const __grid_constant__ MatchParams a, const __grid_constant__ CUtensorMap tmapJ,
                     const __grid_constant__ CUtensorMap tmapI)
{
    match_body<uint16_t, B, P, LEV, ANI>(a, &tmapJ, &tmapI);
}

template <int B, int P, bool ANI>
__global__ void __launch_bounds__(MATCH_MAX_THREADS, MatchMinBlocks<B, P>::value)
    match_kernel_f32(const __grid_constant__ MatchParams a, const __grid_constant__ CUtensorMap tmapJ,
                     const __grid_constant__ CUtensorMap tmapI)
{
    match_body<float, B, P, false, ANI>(a, &tmapJ, &tmapI);
}

template <typename T, int B, int P, bool LEV, bool ANI>
constexpr auto match_kernel_ptr()
{
    if constexpr (std::is_same<T, float>::value)
        return match_kernel_f32<B, P, ANI>;  // float32 jobs report no extra levels
    else
        return match_kernel_u16<B, P, LEV, ANI>;
}

// Shared-memory layout of a launch: double-buffered windows, unless that
// leaves three or fewer CTAs per SM and a single window buffer gives more
// (the other CTAs then hide the exposed copy latency; measured on float32
// windows: b = 9, R = 7 from 1 to 2 CTAs, 23% faster; b = 7, R = 5 from 3 to
// 6 CTAs, 16% faster).
// Block edges along y and z of a launch (0 in MatchLaunch: the x edge).
inline int launch_by(const MatchLaunch &m) { return m.block_y > 0 ? m.block_y : m.block; }
inline int launch_bz(const MatchLaunch &m) { return m.block_z > 0 ? m.block_z : m.block; }

template <typename T, int B, int P, bool LEV, bool ANI>
nrr_status choose_layout(const MatchLaunch &m, MatchLayout *L, bool *single, int *occ)
{
    constexpr int ALIGN = 16 / (int)sizeof(T);
    const int by = launch_by(m), bz = launch_bz(m);
    const int ry = m.radius[1], rz = m.radius[2], py = 2 * ry + 1, pz = 2 * rz + 1;
    const int wyp = match_wyp(by + 2 * ry, py), threads = round_up_i(py * pz, 32);
    const MatchLayout L2 = match_layout((int)sizeof(T), B, P, match_bx<T, B, P>(), round_up_c(B + ALIGN - 1, ALIGN),
                                        wyp, bz + 2 * rz, py, pz, false, LEV, by * bz);
    const MatchLayout L1 = match_layout((int)sizeof(T), B, P, match_bx<T, B, P>(), round_up_c(B + ALIGN - 1, ALIGN),
                                        wyp, bz + 2 * rz, py, pz, true, LEV, by * bz);
    auto kern = match_kernel_ptr<T, B, P, LEV, ANI>();
    static int smem_set = 0;  // largest dynamic shared memory opted in so far
    if (L2.total > smem_set) {
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, L2.total);
        if (e == cudaSuccess)
            e = cudaFuncSetAttribute(kern, cudaFuncAttributePreferredSharedMemoryCarveout, cudaSharedmemCarveoutMaxShared);
        if (e != cudaSuccess) return cuda_fail(e, "cudaFuncSetAttribute(match_kernel)");
        smem_set = L2.total;
    }
    int o2 = 0, o1 = 0;
    cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&o2, kern, threads, L2.total);
    if (e == cudaSuccess && o2 <= 3) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&o1, kern, threads, L1.total);
    if (e != cudaSuccess) return cuda_fail(e, "cudaOccupancyMaxActiveBlocksPerMultiprocessor");
    *single = o2 <= 3 && o1 > o2;
    *L = *single ? L1 : L2;
    *occ = *single ? o1 : o2;
    return NRR_OK;
}

template <typename T, int B, int P, bool LEV, bool ANI>
nrr_status launch_match_variant_l(const MatchLaunch &m, cudaStream_t stream)
{
    constexpr int ALIGN = 16 / (int)sizeof(T);
    constexpr int BX = match_bx<T, B, P>();
    constexpr int BTX = round_up_c(B + ALIGN - 1, ALIGN);
    const int by = launch_by(m), bz = launch_bz(m);
    const int ry = m.radius[1], rz = m.radius[2], py = 2 * ry + 1, pz = 2 * rz + 1;
    const int wy = by + 2 * ry, wz = bz + 2 * rz, wyp = match_wyp(wy, py);
    const int threads = round_up_i(py * pz, 32);
    if (threads > MATCH_MAX_THREADS) return fail(NRR_E_INVALID, "search window too large");
    if (wyp > 256) return fail(NRR_E_INVALID, "search window too large");

    CUtensorMap mapJ, mapI;
    nrr_status st = encode_volume_map(&mapJ, m.intraop, m.dtype, m.dims, BX, wyp, wz);
    if (st != NRR_OK) return st;
    st = encode_volume_map(&mapI, m.preop, m.dtype, m.dims, BTX, by, bz);
    if (st != NRR_OK) return st;

    auto kern = match_kernel_ptr<T, B, P, LEV, ANI>();
    MatchLayout L;
    bool single = false;
    int occ = 0;
    st = choose_layout<T, B, P, LEV, ANI>(m, &L, &single, &occ);
    if (st != NRR_OK) return st;
    if (occ < 1) return fail(NRR_E_INVALID, "match kernel does not fit on an SM (%d B shared)", L.total);
    if (m.ctas_per_sm > 0 && m.ctas_per_sm < occ) occ = m.ctas_per_sm;
    long long cap = 0;
    for (int j = 0; j < m.n_jobs; ++j) cap += m.jobs[j].cap;
    long long grid = m.one_cta_per_block ? cap : (long long)occ * sm_count();
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
    p.wyp = wyp;
    p.n_jobs = m.n_jobs;
    p.single_window = single ? 1 : 0;
    p.by = by;
    p.bz = bz;
    for (int j = 0; j < MATCH_MAX_JOBS; ++j) p.jobs[j] = j < m.n_jobs ? m.jobs[j] : MatchJob{};
    p.err = m.err;
    kern<<<(unsigned)grid, threads, L.total, stream>>>(p, mapJ, mapI);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "match kernel launch");
    count_launches(1);
    return NRR_OK;
}

// Launches whose jobs report extra radius levels use the level-aware kernel
// (uint16 only: the batched search runs on uint16 volumes).
// Launches whose blocks have other edges along y or z than along x use the
// variant with those edges at run time.
template <typename T, int B, int P>
nrr_status launch_match_variant(const MatchLaunch &m, cudaStream_t stream)
{
    bool lev = false;
    for (int j = 0; j < m.n_jobs; ++j) lev |= m.jobs[j].n_levels > 0;
    const bool ani = launch_by(m) != B || launch_bz(m) != B;
    if (ani) {
        if (lev) return fail(NRR_E_INTERNAL, "extra radius levels are not supported for anisotropic blocks");
        return launch_match_variant_l<T, B, P, false, true>(m, stream);
    }
    if (!lev) return launch_match_variant_l<T, B, P, false, false>(m, stream);
    if constexpr (std::is_same<T, float>::value)
        return fail(NRR_E_INTERNAL, "extra radius levels are not supported for float32 volumes");
    else
        return launch_match_variant_l<T, B, P, true, false>(m, stream);
}

template <typename T, int B, int P>
nrr_status occupancy_variant(const MatchLaunch &m, int *occ)
{
    MatchLayout L;
    bool single = false;
    if (launch_by(m) != B || launch_bz(m) != B) return choose_layout<T, B, P, false, true>(m, &L, &single, occ);
    return choose_layout<T, B, P, false, false>(m, &L, &single, occ);
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
