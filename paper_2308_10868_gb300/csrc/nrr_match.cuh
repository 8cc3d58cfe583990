// NCC block-matching kernel (Sec. 3 NCC equation and O(B x W) bound;
// Sec. 4.3 block-matching loop), written for sm_103a.
//
// Persistent CTAs take the registration blocks of up to 16 jobs (each job
// one registration, with its own volumes, sizes and box sums) from a work
// queue, the next item's index fetched a block ahead.  Two blocks are in
// flight: the TMA copies of block i+1 land while block i is processed, in
// the other half of a double window buffer, or, with one window buffer
// (more CTAs per SM), as soon as block i's window has been read.  A search
// radius above 7 on an axis is covered by sub-windows of one radius that
// tile [-R, R]; a block's sub-windows are consecutive items of the same
// CTA, which keeps the best over all of them.  Per block (or sub-window):
//   1. TMA tiled loads bring the block's search window of the reference
//      image, [c-h-R, c+h+R] per axis, and the floating block [c-h, c+h]^3
//      into shared memory.  The x start is rounded down to a 16-byte
//      boundary (offset xo); the CTA then shifts every window row left by xo
//      in place, so the search reads each row from element 0 with aligned
//      16-byte loads.  Out-of-volume voxels arrive as zeros and are excluded
//      by coordinates.
//   2. Every warp sums the whole floating block (uint16: exact integers;
//      float32: float-float pairs), so every thread holds the block's
//      statistics without a barrier; thread 0 stores the constants the later
//      phases need.  The CTA stores the mean-shifted block T_k = I_k - m as
//      float (uint16: scaled by 2^64, see 3).
//   3. Search: a thread owns two neighbouring (dz, dy) lines of the window
//      (one row apart along y, or along z for the lines left over) and all
//      2*rx+1 shifts along x of both.  It walks the window rows the pair
//      shares: each row is loaded once with 16-byte loads and converted once,
//      then multiplied with the template row of the first line and with the
//      previous template row for the second line.  float32 windows and
//      blocks with an edge per axis take one line per thread instead (their
//      rows need no conversion, or their short planes would leave paired
//      units idle).  Window values enter
//      centred by the floating block's mean: uint16 u becomes the subnormal
//      float (u - m) * 2^-149 by one byte-permute and a packed subtraction
//      of two values (exact); the template scaled by 2^64 brings the
//      products into the normal range, and every partial sum is a multiple
//      of 2^-85, so none underflows.  A(d) = sum_k T_k J_{k+d} accumulates
//      with FP32 FFMA, one chain of N terms per shift.
//   4. Every shift gets an approximate NCC from A(d) and the box sums S_J,
//      S_JJ (precomputed: exact for uint16; for float32 sums of J - c, c
//      the reference volume's centre value; read from global memory in the
//      bound's loop, or staged per thread into shared memory by
//      asynchronous copies during the search) and a rigorous bound on its
//      error (recursive-summation
//      bound gamma_N * sum|T||J - m| for the FMA chain, Cauchy-Schwarz
//      sum|T||J - m| <= sqrt(sum T^2 * sum (J - m)^2), plus the rounding of
//      the final operations, each written as a separately rounded operation;
//      doubled for margin).
//   5. Shifts whose upper bound reaches the best lower bound over the CTA
//      survive (about one per block on the phantoms); each warp rescores
//      the survivors of its own lines: uint16 -> exact int64 sums, then the
//      canonical FP64 ratio num / sqrt(vI * vJ); float32 -> Pearson sums of
//      the values less the block's first value, in float-float pairs, and
//      one FP64 ratio.  The best survivor under the
//      tie-break rule is the block's answer.
// Three CTA barriers per block: after the template, after the lower bounds,
// after the rescoring.
// The exhaustive maximum is therefore found exactly: the true arg-max can
// never be filtered out, because its upper bound is at least its value,
// which is at least every other shift's value, hence at least every lower
// bound.
#pragma once

#include <math.h>
#include <stdint.h>

#include <algorithm>
#include <type_traits>
#include <vector>

#include "nrr_internal.h"
#include "nrr_ptx.cuh"

namespace nrr {

constexpr int MATCH_MAX_THREADS_C = 256;
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
    uint64_t wait_ns;  // limit of the wait for a block's copies
    // Search radius above what one window holds: the jobs' full radii, and
    // the sub-windows (radius rx = (P-1)/2, ry, rz each) that tile
    // [-R, R] per axis, nsub[axis] of them centred at soff[axis][0..]
    int R[3];
    int nsub[3];
    int soff[3][MATCH_MAX_SUB];
    int nsubt;  // nsub[0] * nsub[1] * nsub[2]
    // Work queue: CTA k starts with item k; further items (gridDim.x, ...)
    // are taken from this head, zero when the launch starts.
    int32_t *queue;
    // box sums of each thread's lines staged in shared memory by
    // asynchronous copies issued at the block's start
    int stage;
    // thread k takes line unit unit_of[k] (255: none), an order of the units
    // in which the 16-byte window loads of every 8 consecutive threads fall
    // in distinct bank groups where possible
    uint8_t unit_of[MATCH_MAX_THREADS_C];
};

constexpr int MATCH_MAX_THREADS = MATCH_MAX_THREADS_C;
constexpr int MATCH_MAX_WARPS = MATCH_MAX_THREADS / 32;

struct Cand {
    double s;
    int n2;
    int code;
    int ok;
};

// float32 block constants, derived by thread 0 and read by the CTA after
// the template barrier.
struct BlockConstF {
    double dvI;      // sum (I - Ibar)^2
    float ibh, ibl;  // the mean as a float pair (ibh + ibl)
    float fvI;       // dvI as float
    float kq;        // sqrt(sum T^2), rounded up
    float emu;       // Ibar - mu (mu: the float mean used for T)
    float cv;        // c of the box sums (sums of J - c): the reference volume's centre value
    float eI;        // bound on emu's error beyond 2u |emu| (the float-float mean's), rounded up
};

// uint16 block constants: every thread derives them from the warp sums;
// thread 0 stores them for the phases after the search, so that they hold
// no registers through it.
struct BlockConstU {
    long long vI;  // N*S_II - S_I^2 (exact)
    long long rr;  // N*m - S_I
    float frr;     // rr as float (exact: |rr| <= N/2)
    float fvI;     // vI as float
    float kq;      // N*gamma_L*sqrt(sum (I-m)^2), rounded up
    int m;         // nearest integer to the block mean
};

struct MatchScratch {
    BlockConstF bc;
    BlockConstU bu;
    int cen[2][6];  // per window buffer: cx, cy, cz, job, index of the block in its job, sub-window
    Cand sbest;     // best candidate of the current block over its sub-windows so far
    int nb[2];      // per window buffer: the work item after that buffer's block
    int ns[2];      // and its sub-window
    float wlb[MATCH_MAX_WARPS];
    double bs[MATCH_MAX_WARPS];
    int bn2[MATCH_MAX_WARPS];
    int bcode[MATCH_MAX_WARPS];
    int bok[MATCH_MAX_WARPS];
    int jstart[MATCH_MAX_JOBS + 1];  // first work item of each job
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

// Template pairs per row: the B columns padded to an even count, so a
// 16-byte load brings two columns' (t, t) pairs.
__host__ __device__ constexpr int match_tpr(int B) { return (B + 1) / 2 * 2; }

// Rows per plane of the window box: the window's wy rows plus one (the pad
// line of a thread with a single line reads one row further), rounded up to
// an odd count.  Consecutive threads own lines one window plane apart; with
// an odd number of 16-byte chunks per row and an odd number of rows per
// plane, 8 consecutive planes start in 8 distinct bank groups.
__host__ __device__ inline int match_wyp(int wy, int py)
{
    (void)py;
    return (wy + 1) | 1;
}

struct MatchLayout {
    int u[2], ut[2], t, sc, lsc, bs, bar, total;
};

// Shared-memory carve-up of one CTA (all offsets 128-byte aligned).  With
// single_window the two blocks in flight share one window buffer (their
// floating blocks stay double-buffered); `levels` adds the level scratch;
// `stage` adds each thread's box sums of its two lines (4 P words a thread,
// interleaved over the `threads` threads).
__host__ __device__ inline MatchLayout match_layout(int elem, int B, int P, int bx, int btx, int wyp, int wz, int py,
                                                   int pz, bool single_window, bool levels, int brows, bool stage,
                                                   int threads)
{
    // brows: rows of the floating block (by * bz)
    (void)P;
    (void)py;
    (void)pz;
    MatchLayout L;
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
    o += round_up_i(brows * ((B + 3) / 4 * 4) * 4, 128);
    L.sc = o;
    o += round_up_i((int)sizeof(MatchScratch), 128);
    L.lsc = o;
    if (levels) o += round_up_i((int)sizeof(MatchLevelScratch), 128);
    L.bs = o;
    if (stage) o += round_up_i(4 * P * threads * 4, 128);
    L.bar = o;
    o += 128;
    L.total = o;
    return L;
}

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

// Two floats as one 64-bit register pair (the operand form of the packed
// f32x2 instructions), and the packed FMA itself (round to nearest, IEEE
// subnormals kept: no .ftz).
typedef unsigned long long f2_t;
__device__ __forceinline__ f2_t f2_bits(uint32_t lo, uint32_t hi)
{
    f2_t r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "r"(lo), "r"(hi));
    return r;
}
__device__ __forceinline__ float f2_lo(f2_t v) { return __uint_as_float((uint32_t)v); }
__device__ __forceinline__ float f2_hi(f2_t v) { return __uint_as_float((uint32_t)(v >> 32)); }
__device__ __forceinline__ f2_t f2_fma(f2_t a, f2_t b, f2_t c)
{
    f2_t d;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
    return d;
}

// Codes of candidate shifts run over the full search box [-R, R] per axis
// (x fastest: P = 2 Rx + 1 x-shifts, py = 2 Ry + 1 y-shifts).
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

// Bits of window element E (within the loaded 16-byte chunks) as the float
// the search multiplies: float32 as it is, uint16 u as the subnormal u * 2^-149
// (one byte-permute; elements past the loaded chunks are a zero pad).
template <typename T, int NC>
__device__ __forceinline__ uint32_t win_bits(const uint4 (&ch)[NC], int E)
{
    constexpr bool F32 = std::is_same<T, float>::value;
    constexpr int EPC = 16 / (int)sizeof(T);
    if (E < 0 || E >= NC * EPC) return 0u;
    const uint4 &q = ch[E / EPC];
    if constexpr (F32) {
        const int w = E % 4;
        return w == 0 ? q.x : w == 1 ? q.y : w == 2 ? q.z : q.w;
    } else {
        const int w = (E % 8) / 2;
        const uint32_t word = w == 0 ? q.x : w == 1 ? q.y : w == 2 ? q.z : q.w;
        return (E & 1) ? __byte_perm(word, 0u, 0x4432) : __byte_perm(word, 0u, 0x4410);
    }
}

// Line units.  Thread k of a CTA owns one or two (dz, dy) lines of the
// search window.  Two lines one row apart along y (type A) or z (type B)
// read the same window rows one template row apart, so each window row a
// thread loads and converts serves both lines' products.  Type A pairs
// (dy, dy+1) fill every plane dz (consecutive threads walk dz, so their
// rows are one window plane apart: distinct bank groups); with an odd
// number py of y-shifts the last line of each plane is left over, and those
// pair along z (type B); with pz odd too one line stays single, paired with
// a pad line one row further along y whose sums are discarded (the window
// box holds that extra row).
// With one line per thread (LPT = 1: float32 windows, whose rows need no
// conversion and whose values take twice the registers, and blocks with an
// edge per axis, whose short window planes leave paired units a third of a
// CTA idle), thread k owns line (dz, dy) = (k mod pz, k / pz) alone.
__host__ __device__ inline int match_units(int py, int pz, int lpt = 2)
{
    if (lpt == 1) return py * pz;
    return pz * (py / 2) + ((py & 1) ? pz / 2 + (pz & 1) : 0);
}
// Search lines per thread of a uint16 cubic-block launch when its shape asks
// for none, by x-shift count P of one (sub-)window.  Measured on the clinical
// pair (b = 5, 7, 9): one line is 20-30 % faster at P = 5 and 9, where two
// lines per thread leave a larger share of the CTA's last warp idle (15 units
// in 32 threads at R = 2, 45 in 64 at R = 4); even at P = 7; two are 10-30 %
// faster from P = 11 on.  At P = 1 and 3 a single warp holds every line, so
// one line per thread halves each thread's serial work.  Float32 windows and
// per-axis blocks always take one line per thread.
__host__ __device__ constexpr int match_default_lines(int P)
{
    return P <= 5 || P == 9 ? 1 : 2;
}
struct LineUnit {
    int dz0, dy0;  // first line (shift indices 0 .. pz-1, 0 .. py-1)
    int along_z;   // the second line is (dz0 + 1, dy0) instead of (dz0, dy0 + 1)
    int two;       // the second line is a real line (not the pad)
};
template <int LPT>
__device__ __forceinline__ bool line_unit(int k, int py, int pz, LineUnit &u)
{
    if constexpr (LPT == 1) {
        u.dz0 = k % pz;
        u.dy0 = k / pz;
        u.along_z = 0;
        u.two = 0;
        return k < py * pz;
    }
    const int hp = py / 2, nA = pz * hp;
    if (k < nA) {
        u.dz0 = k % pz;
        u.dy0 = 2 * (k / pz);
        u.along_z = 0;
        u.two = 1;
        return true;
    }
    if (!(py & 1)) return false;
    const int m = k - nA, nB = pz / 2;
    if (m < nB) {
        u.dz0 = 2 * m;
        u.dy0 = py - 1;
        u.along_z = 1;
        u.two = 1;
        return true;
    }
    if (m == nB && (pz & 1)) {
        u.dz0 = pz - 1;
        u.dy0 = py - 1;
        u.along_z = 0;
        u.two = 0;
        return true;
    }
    return false;
}

// Shift every row of the window box left by xo elements in place, so that
// each row's data starts at element 0 (rows 0 .. wy-1 of each of the wz
// planes; the rows past them are never used).  A thread moves whole rows:
// it loads a row's 16-byte chunks, shifts the words in registers by xo's
// word part with two select stages (by one, then by two words) and the
// uint16 half-word remainder with a funnel shift, and stores the row back.
template <typename T, int BX>
__device__ __forceinline__ void realign_window(T *U, int wyp, int wy, int wz, int xo, int tid, int nthr)
{
    constexpr bool F32 = std::is_same<T, float>::value;
    constexpr int NCH = BX * (int)sizeof(T) / 16;  // 16-byte chunks per row
    constexpr int RW = 4 * NCH;                    // words per row
    const int s = F32 ? xo : xo >> 1;              // whole words to drop (0..3)
    const uint32_t hs = F32 ? 0u : 16u * (uint32_t)(xo & 1);
    const int nrows = wy * wz;
    for (int row = tid; row < nrows; row += nthr) {
        const int z = row / wy, y = row - z * wy;
        uint4 *rp = reinterpret_cast<uint4 *>(U + (size_t)(z * wyp + y) * BX);
        uint32_t w[RW];
#pragma unroll
        for (int c = 0; c < NCH; ++c) {
            const uint4 v = rp[c];
            w[4 * c + 0] = v.x;
            w[4 * c + 1] = v.y;
            w[4 * c + 2] = v.z;
            w[4 * c + 3] = v.w;
        }
#pragma unroll
        for (int k = 0; k + 1 < RW; ++k) w[k] = (s & 1) ? w[k + 1] : w[k];
#pragma unroll
        for (int k = 0; k + 2 < RW; ++k) w[k] = (s & 2) ? w[k + 2] : w[k];
        if constexpr (!F32) {
#pragma unroll
            for (int k = 0; k + 1 < RW; ++k) w[k] = __funnelshift_r(w[k], w[k + 1], hs);
        }
#pragma unroll
        for (int c = 0; c < NCH; ++c) rp[c] = make_uint4(w[4 * c], w[4 * c + 1], w[4 * c + 2], w[4 * c + 3]);
    }
}

// One line (LPT = 1): for every template row, the window row below it is
// loaded, converted and multiplied with that template row only.
template <typename T, int B, int P>
__device__ __forceinline__ void search_line(const T *row0, int sO, const float *Ts, int bO, int bI, float csh,
                                            float (&acc)[P])
{
    constexpr int WX = B + P - 1;
    constexpr int EPC = 16 / (int)sizeof(T);
    constexpr int NC = (WX - 1) / EPC + 1;
    constexpr int PT = (B + 3) / 4 * 4;
    f2_t negc2;
    asm("mov.b64 %0, {%1, %1};" : "=l"(negc2) : "f"(-csh));
#pragma unroll
    for (int p = 0; p < P; ++p) acc[p] = 0.f;
#pragma unroll 1
    for (int o = 0; o < bO; ++o) {
        const float *tp = Ts + o * bI * PT;
#pragma unroll 1
        for (int i = 0; i < bI; ++i, tp += PT) {
            const T *wp = row0 + o * sO + i * match_bx<T, B, P>();
            uint4 ch[NC];
#pragma unroll
            for (int c = 0; c < NC; ++c) ch[c] = *reinterpret_cast<const uint4 *>(wp + c * EPC);
            float tc[PT];
#pragma unroll
            for (int q = 0; q < PT / 4; ++q) {
                const float4 v = *reinterpret_cast<const float4 *>(tp + 4 * q);
                tc[4 * q + 0] = v.x;
                tc[4 * q + 1] = v.y;
                tc[4 * q + 2] = v.z;
                tc[4 * q + 3] = v.w;
            }
            float j[WX];
#pragma unroll
            for (int e = 0; e + 1 < WX; e += 2) {
                f2_t d;
                asm("add.rn.f32x2 %0, %1, %2;"
                    : "=l"(d)
                    : "l"(f2_bits(win_bits<T, NC>(ch, e), win_bits<T, NC>(ch, e + 1))), "l"(negc2));
                j[e] = f2_lo(d);
                j[e + 1] = f2_hi(d);
            }
            if constexpr (WX & 1) j[WX - 1] = __fsub_rn(__uint_as_float(win_bits<T, NC>(ch, WX - 1)), csh);
#pragma unroll
            for (int kx = 0; kx < B; ++kx)
#pragma unroll
                for (int p = 0; p < P; ++p) acc[p] = __fmaf_rn(tc[kx], j[kx + p], acc[p]);
        }
    }
}

// The search of one thread's two lines.  `row0` points at the first line's
// first window row (rows realigned: data from element 0); the template is
// walked with its rows along the pair's direction ("inner", bI rows, window
// rows sI elements apart, template rows tI rows apart) innermost and the
// other direction ("outer", bO rows, sO, tO) outside.  Step i of an inner
// pass reads one window row: the first line multiplies it with template row
// i (i < bI), the second line, which sits one window row further on, with
// template row i - 1 (i >= 1).  Ts holds the template, PT floats per row.
// On return acc0[p] / acc1[p] = sum over the block of T_k * J_{k + p} for the
// two lines (uint16: in units of 2^-85), each a chain of N FMAs, with
// J_k = window value minus csh (uint16: csh = m * 2^-149, the floating
// block's integer mean, so the difference is exact; float32: the float mean,
// the difference rounded once).
template <typename T, int B, int P>
__device__ __forceinline__ void search_pair(const T *row0, int sI, int sO, const float *Ts, int tI, int tO, int bI, int bO,
                                            float csh, float (&acc0)[P], float (&acc1)[P])
{
    constexpr int WX = B + P - 1;
    constexpr int EPC = 16 / (int)sizeof(T);
    constexpr int NC = (WX - 1) / EPC + 1;  // 16-byte chunks covering [0, WX)
    constexpr int PT = (B + 3) / 4 * 4;
    constexpr int ROW_UNROLL = B >= 9 ? 2 : 1;
    f2_t negc2;  // (-csh, -csh): the centring subtraction, two values per packed add
    asm("mov.b64 %0, {%1, %1};" : "=l"(negc2) : "f"(-csh));
#pragma unroll
    for (int p = 0; p < P; ++p) {
        acc0[p] = 0.f;
        acc1[p] = 0.f;
    }
#pragma unroll 1
    for (int o = 0; o < bO; ++o) {
        const T *wp = row0 + o * sO;
        const float *tp = Ts + o * tO * PT;
        float tprev[B];
        // rows two at a time for the larger blocks (measured: high
        // resolution b = 9 2.8% faster; the clinical b = 7 1.8% slower)
#pragma unroll(ROW_UNROLL)
        for (int i = 0; i <= bI; ++i, wp += sI, tp += tI * PT) {
            uint4 ch[NC];
#pragma unroll
            for (int c = 0; c < NC; ++c) ch[c] = *reinterpret_cast<const uint4 *>(wp + c * EPC);
            float tc[PT];
            if (i < bI) {
#pragma unroll
                for (int q = 0; q < PT / 4; ++q) {
                    const float4 v = *reinterpret_cast<const float4 *>(tp + 4 * q);
                    tc[4 * q + 0] = v.x;
                    tc[4 * q + 1] = v.y;
                    tc[4 * q + 2] = v.z;
                    tc[4 * q + 3] = v.w;
                }
            }
            // window values minus the centring constant, two per packed add
            // (uint16: u * 2^-149 - m * 2^-149, exact on subnormals)
            float j[WX];
#pragma unroll
            for (int e = 0; e + 1 < WX; e += 2) {
                f2_t d;
                asm("add.rn.f32x2 %0, %1, %2;"
                    : "=l"(d)
                    : "l"(f2_bits(win_bits<T, NC>(ch, e), win_bits<T, NC>(ch, e + 1))), "l"(negc2));
                j[e] = f2_lo(d);
                j[e + 1] = f2_hi(d);
            }
            if constexpr (WX & 1) j[WX - 1] = __fsub_rn(__uint_as_float(win_bits<T, NC>(ch, WX - 1)), csh);
            if (i >= 1) {
#pragma unroll
                for (int kx = 0; kx < B; ++kx)
#pragma unroll
                    for (int p = 0; p < P; ++p) acc1[p] = __fmaf_rn(tprev[kx], j[kx + p], acc1[p]);
            }
            if (i < bI) {
#pragma unroll
                for (int kx = 0; kx < B; ++kx)
#pragma unroll
                    for (int p = 0; p < P; ++p) acc0[p] = __fmaf_rn(tc[kx], j[kx + p], acc0[p]);
            }
#pragma unroll
            for (int kx = 0; kx < B; ++kx) tprev[kx] = tc[kx];
        }
    }
}

// Box sums S_J and S_JJ (uint16: v_J) of every x-shift of one line, and
// the mask of the shifts whose block lies inside the volume.  The loads are
// independent and issued together.
template <typename T, int B, int P>
__device__ __forceinline__ uint32_t line_boxsums(const MatchParams &a, const MatchJob &J, int cx, int cy, int cz,
                                                 int dyi, int dzi, int HY, int HZ,
                                                 typename std::conditional<std::is_same<T, float>::value, float,
                                                                           int32_t>::type (&ps1)[P],
                                                 float (&ps2)[P])
{
    typedef typename std::conditional<std::is_same<T, float>::value, float, int32_t>::type S1T;
    constexpr int H = (B - 1) / 2;
    constexpr int RX = (P - 1) / 2;
    const int ny = J.ny, nz = J.nz, nx = J.nx;
    const int Y = cy + dyi - a.ry, Z = cz + dzi - a.rz;
    const bool yz_ok = Y >= HY && Y <= ny - 1 - HY && Z >= HZ && Z <= nz - 1 - HZ;
    uint32_t vmask = 0;
    const size_t rowbase = ((size_t)Z * ny + Y) * nx;
#pragma unroll
    for (int p = 0; p < P; ++p) {
        const int X = cx + p - RX;
        ps1[p] = 0;
        ps2[p] = 0.f;
        if (yz_ok && X >= H && X <= nx - 1 - H) {
            vmask |= 1u << p;
            ps1[p] = reinterpret_cast<const S1T *>(J.s1)[rowbase + X];
            ps2[p] = reinterpret_cast<const float *>(J.s2)[rowbase + X];
        }
    }
    return vmask;
}

// The same mask without the loads, and the loads as 4-byte asynchronous
// copies into this thread's staging words (s1 at dst1 + 4 p stride, s2 at
// dst2 + 4 p stride; shifts outside the volume are zero-filled without a
// read), issued as one group at the block's start and waited for before
// the bounds.
template <int B, int P>
__device__ __forceinline__ uint32_t line_vmask(const MatchParams &a, const MatchJob &J, int cx, int cy, int cz,
                                               int dyi, int dzi, int HY, int HZ)
{
    constexpr int H = (B - 1) / 2;
    constexpr int RX = (P - 1) / 2;
    const int Y = cy + dyi - a.ry, Z = cz + dzi - a.rz;
    if (!(Y >= HY && Y <= J.ny - 1 - HY && Z >= HZ && Z <= J.nz - 1 - HZ)) return 0u;
    uint32_t vmask = 0;
#pragma unroll
    for (int p = 0; p < P; ++p) {
        const int X = cx + p - RX;
        if (X >= H && X <= J.nx - 1 - H) vmask |= 1u << p;
    }
    return vmask;
}
// Index of the box sum of shift (x0 + p, cy + dy, cz + dz) less p.
__device__ __forceinline__ long long line_row(const MatchJob &J, int x0, int cy, int cz, int dy, int dz)
{
    return ((long long)(cz + dz) * J.ny + (cy + dy)) * J.nx + x0;
}
template <int B, int P>
__device__ __forceinline__ void line_boxsums_async(const MatchParams &a, const MatchJob &J, int cx, int cy, int cz,
                                                   int dyi, int dzi, int HY, int HZ, uint32_t dst1, uint32_t dst2,
                                                   uint32_t stride)
{
    constexpr int RX = (P - 1) / 2;
    const uint32_t vmask = line_vmask<B, P>(a, J, cx, cy, cz, dyi, dzi, HY, HZ);
    const int Y = cy + dyi - a.ry, Z = cz + dzi - a.rz;
    const long long rowbase = vmask ? ((long long)Z * J.ny + Y) * J.nx + cx - RX : 0;
    const uint32_t *s1 = reinterpret_cast<const uint32_t *>(J.s1), *s2 = reinterpret_cast<const uint32_t *>(J.s2);
#pragma unroll
    for (int p = 0; p < P; ++p) {
        const bool ok = (vmask >> p) & 1u;
        cp_async_4(dst1 + 4u * p * stride, ok ? s1 + rowbase + p : s1, ok ? 4u : 0u);
        cp_async_4(dst2 + 4u * p * stride, ok ? s2 + rowbase + p : s2, ok ? 4u : 0u);
    }
}

// Approximate NCC of every x-shift of one line, with a rigorous bound on its
// error (see the header comment); ub[p] = v + e and the best lower bound
// v - e of the line (and of each level box holding it).
template <typename T, int B, int P, bool LEV, class G1, class G2>
__device__ __forceinline__ void line_bounds(const MatchJob &J, int nl, int dyi, int dzi, int ry, int rz, int N, int BY,
                                            int BZ, const float (&acc)[P], G1 ps1, G2 ps2, uint32_t vmask, float kq,
                                            float fvI, float frr,
                                            int m, float c_f, const BlockConstF &bcf, double GAMMA_L, float (&ub)[P],
                                            float &lbm, float (&lbl)[MATCH_MAX_LEVELS])
{
    constexpr bool F32 = std::is_same<T, float>::value;
    constexpr int RX = (P - 1) / 2;
    constexpr float U32 = 5.9604644775390625e-08f;  // 2^-24, unit roundoff of binary32
    constexpr float ASCALE = 0x1p85f;
    const int dy = dyi - ry, dz = dzi - rz;
    unsigned int lvl_line = 0;  // bit l: this line lies in level l
    if constexpr (LEV) {
#pragma unroll
        for (int l = 0; l < MATCH_MAX_LEVELS; ++l)
            if (l < nl && abs(dy) <= J.levels[l].r[1] && abs(dz) <= J.levels[l].r[2]) lvl_line |= 1u << l;
    }
    const float fN = (float)N;
#pragma unroll
    for (int p = 0; p < P; ++p) {
        ub[p] = -INFINITY;
        if (!((vmask >> p) & 1u)) continue;
        float v, e;
        if constexpr (!F32) {
            // 32-bit integer and float arithmetic only: a 64-bit integer to
            // float conversion issues on the FP64 pipe, which is narrow on
            // this part.  v_J arrives rounded once (zero only for a flat
            // block); S_J rounds at most once.
            const float vjf = ps2(p);
            if (!(vjf > 0.f)) continue;  // flat reference block
            const float s1f = (float)(ps1(p) - N * m);  // S'_J = sum (J - m), exact before the rounding
            // sum (J - m)^2 = (v_J + S'_J^2) / N, rounded up: the rounded v_J
            // and S'_J and three operations stay below 6u
            const float s2u = __fmul_rn(__fmul_rn(__fmaf_rn(s1f, s1f, vjf), 1.0f / fN), 1.f + 16.f * U32);
            // rsqrt.approx and sqrt.approx (relative error below 2^-22 over
            // the whole range) instead of the correctly rounded forms: the
            // factor 1 + 64u on the error terms and 40u|v| for the centre
            // value absorb their error
            float inv, sq;
            asm("rsqrt.approx.f32 %0, %1;" : "=f"(inv) : "f"(__fmul_rn(fvI, vjf)));
            asm("sqrt.approx.f32 %0, %1;" : "=f"(sq) : "f"(s2u));
            const float na = __fmul_rn(acc[p], fN * ASCALE);  // N * A
            const float rs = __fmul_rn(frr, s1f);             // (N m - S_I) S'_J
            v = __fmul_rn(__fadd_rn(na, rs), inv);
            // e = (kq sq inv + 4u (|na| + |rs|) inv) (1 + 64u) + 40u |v|, each
            // operation rounded on its own (no contraction)
            const float t1 = __fmul_rn(__fmul_rn(kq, sq), inv);
            const float t2 = __fmul_rn(__fmul_rn(4.f * U32, __fadd_rn(fabsf(na), fabsf(rs))), inv);
            e = __fadd_rn(__fmul_rn(__fadd_rn(t1, t2), 1.f + 64.f * U32), __fmul_rn(40.f * U32, fabsf(v)));
        } else {
            // box-sum depth: the b-term levels, the rounding of J - c and of
            // its square
            const float GS = (float)((B + BY + BZ + 3) * 5.9604644775390625e-08 /
                                     (1.0 - (B + BY + BZ + 3) * 5.9604644775390625e-08));
            // the box sums are of J - cv; the window is centred by c_f:
            // dl = fl(c_f - cv), and c_f - (cv + dl) is at most 1.01 u |dl|
            const float GN = (float)GAMMA_L;
            const float s1 = ps1(p);
            const float s2 = fmaxf(ps2(p), 0.f);
            // every operation below is rounded on its own (no contraction)
            float d1;  // |S1 err| bound (the factor 1.01 covers sqrt.approx)
            asm("sqrt.approx.f32 %0, %1;" : "=f"(d1) : "f"(__fmul_rn(fN, s2)));
            d1 = __fmul_rn(__fmul_rn(GS, d1), 1.01f);
            const float s1sq_n = __fmul_rn(__fmul_rn(s1, s1), 1.0f / fN);
            const float vJa = __fsub_rn(s2, s1sq_n);
            const float dv = __fadd_rn(__fadd_rn(__fmul_rn(GS, s2),
                                                 __fdiv_rn(__fmul_rn(__fadd_rn(__fmul_rn(2.f, fabsf(s1)), d1), d1), fN)),
                                       __fmul_rn(4.f * U32, __fadd_rn(s2, s1sq_n)));
            // S'_J ~ sum (J - c_f), and sum (J - c_f)^2 <= its estimate e2
            // plus the error of the sums, of the dl terms and of c_f - (cv +
            // dl) (m2 bounds their size), rounded up
            const float dl = __fsub_rn(c_f, bcf.cv);
            const float s1p = __fsub_rn(s1, __fmul_rn(fN, dl));
            const float m2 = __fadd_rn(__fadd_rn(s2, __fmul_rn(__fmul_rn(2.f, fabsf(dl)), fabsf(s1))),
                                       __fmul_rn(__fmul_rn(fN, dl), dl));
            const float e2 = __fadd_rn(__fsub_rn(s2, __fmul_rn(__fmul_rn(2.f, dl), s1)), __fmul_rn(__fmul_rn(fN, dl), dl));
            const float sj2 = __fmul_rn(__fadd_rn(fmaxf(e2, 0.f), __fmul_rn(__fmul_rn(__fadd_rn(GS, 12.f * U32), m2), 1.01f)),
                                        1.f + 4.f * U32);
            if (!(vJa - dv > 0.f)) {  // spread of the reference block not resolved: rescore
                ub[p] = INFINITY;
                continue;
            }
            const float rho = __fdiv_rn(dv, __fsub_rn(vJa, dv));
            if (!(rho <= 0.25f)) {
                ub[p] = INFINITY;
                continue;
            }
            float inv, sq;
            asm("rsqrt.approx.f32 %0, %1;" : "=f"(inv) : "f"(__fmul_rn(bcf.fvI, vJa)));
            asm("sqrt.approx.f32 %0, %1;" : "=f"(sq) : "f"(sj2));
            const float A = acc[p];
            const float es = __fmul_rn(bcf.emu, s1p);  // (Ibar - mu) S'_J
            const float num = __fsub_rn(A, es);
            v = __fmul_rn(num, inv);
            // the numerator's error: the search sum's (GN, and 3u for the
            // roundings of T and of the window values), then es = emu S'_J:
            // emu errs by at most 2u |emu| + eI and s1p by d1 + 4uN|dl| +
            // 2u |s1p| (the box sums, N dl and c_f - (cv + dl), the
            // subtraction), with |S'_J| <= sb
            const float aem = fabsf(bcf.emu);
            const float ds = __fadd_rn(d1, __fmul_rn(4.f * U32, __fmul_rn(fN, fabsf(dl))));
            const float sb = __fadd_rn(fabsf(s1p), ds);
            const float tes = __fadd_rn(__fmul_rn(sb, __fadd_rn(__fmul_rn(2.f * U32, aem), bcf.eI)),
                                        __fmul_rn(aem, __fadd_rn(ds, __fmul_rn(2.f * U32, fabsf(s1p)))));
            const float enum_ = __fadd_rn(
                __fadd_rn(__fmul_rn(__fmul_rn(__fadd_rn(GN, 3.f * U32), bcf.kq), sq), __fmul_rn(tes, 1.01f)),
                __fmul_rn(U32, __fadd_rn(fabsf(A), fabsf(es))));
            const float r1 = __fadd_rn(__fadd_rn(1.f, __fmul_rn(0.7f, rho)), 4.f * U32);
            const float r2 = __fadd_rn(__fmul_rn(0.7f, rho), 6.f * U32);
            e = __fadd_rn(__fmul_rn(__fadd_rn(__fmul_rn(__fmul_rn(enum_, inv), r1), __fmul_rn(__fmul_rn(fabsf(num), inv), r2)),
                                    1.f + 64.f * U32),
                          __fmul_rn(43.f * U32, fabsf(v)));
        }
        e = __fadd_rn(__fmul_rn(2.f, e), 1e-9f);
        ub[p] = __fadd_rn(v, e);
        const float lo = __fsub_rn(v, e);
        lbm = fmaxf(lbm, lo);
        if (LEV && lvl_line) {
#pragma unroll
            for (int l = 0; l < MATCH_MAX_LEVELS; ++l)
                if (((lvl_line >> l) & 1u) && abs(p - RX) <= J.levels[l].r[0]) lbl[l] = fmaxf(lbl[l], lo);
        }
    }
}

// x-shifts of one line that survive: they can be the best of the whole
// window (ub >= LB) or of a level box holding them.
template <int P, bool LEV>
__device__ __forceinline__ uint32_t line_survivors(const MatchJob &J, int nl, int dyi, int dzi, int ry, int rz,
                                                   const float (&ub)[P], float LB, const float (&LBl)[MATCH_MAX_LEVELS])
{
    constexpr int RX = (P - 1) / 2;
    uint32_t lvl_line = 0;
    if constexpr (LEV) {
#pragma unroll
        for (int l = 0; l < MATCH_MAX_LEVELS; ++l)
            if (l < nl && abs(dyi - ry) <= J.levels[l].r[1] && abs(dzi - rz) <= J.levels[l].r[2]) lvl_line |= 1u << l;
    }
    uint32_t m = 0;
#pragma unroll
    for (int p = 0; p < P; ++p) {
        bool lv = false;
        if (LEV && lvl_line) {
#pragma unroll
            for (int l = 0; l < MATCH_MAX_LEVELS; ++l)
                lv |= ((lvl_line >> l) & 1u) && abs(p - RX) <= J.levels[l].r[0] && ub[p] >= LBl[l];
        }
        if (ub[p] > -INFINITY && (ub[p] >= LB || lv)) m |= 1u << p;
    }
    return m;
}

// The kernel body; the __global__ entries below differ only in their
// register budget.  `a`, `tmapJ` and `tmapI` live in kernel-parameter space.
// LEV: the jobs may report extra radius levels (batched search); without it
// that code is compiled out.  ANI: the block edges along y and z (a.by,
// a.bz) may differ from the x edge B; without it they are B and every size
// below is a compile-time constant.  LPT: search lines per thread (1 or 2;
// 2 for uint16 cubic blocks only).
template <typename T, int B, int P, bool LEV, bool ANI, int LPT>
__device__ __forceinline__ void match_body(const MatchParams &a, const CUtensorMap *tmapJ, const CUtensorMap *tmapI)
{
    constexpr bool F32 = std::is_same<T, float>::value;
    constexpr int H = (B - 1) / 2;  // x half edge
    constexpr int N3 = B * B * B;   // terms of a cubic block
    const int BY = ANI ? a.by : B, BZ = ANI ? a.bz : B;
    const int HY = (BY - 1) / 2, HZ = (BZ - 1) / 2;
    const int N = ANI ? B * BY * BZ : N3;
    const int NROW = BY * BZ;  // rows of the floating block
    constexpr int PT = (B + 3) / 4 * 4;
    constexpr int RX = (P - 1) / 2;
    constexpr int ALIGN = 16 / (int)sizeof(T);
    constexpr int BX = match_bx<T, B, P>();
    constexpr int BTX = round_up_c(B + ALIGN - 1, ALIGN);
    // rounding depth of the search sums: one chain of N FMAs per shift
    const double GAMMA_L = (double)N * 5.9604644775390625e-08 / (1.0 - (double)N * 5.9604644775390625e-08);
    // uint16: the template is scaled by 2^64 and the window values enter as
    // u * 2^-149, so a search sum is A * 2^-85
    constexpr float TSCALE = 0x1p64f;

    const int ry = a.ry, rz = a.rz, py = 2 * ry + 1, pz = 2 * rz + 1;  // one (sub-)window
    const int wz = BZ + 2 * rz, wyp = a.wyp;
    // the full search box: candidate codes, displacements and levels use it
    const int Rx = a.R[0], Ry = a.R[1], Rz = a.R[2], PxF = 2 * Rx + 1, PyF = 2 * Ry + 1;
    const int nsubt = a.nsubt;
    // offset of sub-window s (x fastest) from the block centre
    auto sub_off = [&](int s, int &ox, int &oy, int &oz) {
        ox = oy = oz = 0;
        if (nsubt > 1) {
            const int sx = s % a.nsub[0], sy = (s / a.nsub[0]) % a.nsub[1], sz = s / (a.nsub[0] * a.nsub[1]);
            ox = a.soff[0][sx];
            oy = a.soff[1][sy];
            oz = a.soff[2][sz];
        }
    };

    extern __shared__ __align__(128) unsigned char smem[];
    const MatchLayout L =
        match_layout((int)sizeof(T), B, P, BX, BTX, wyp, wz, py, pz, a.single_window != 0, LEV, NROW, a.stage != 0,
                     (int)blockDim.x);
    const bool single = a.single_window != 0;
    float *Ts = reinterpret_cast<float *>(smem + L.t);
    MatchScratch *sc = reinterpret_cast<MatchScratch *>(smem + L.sc);
    MatchLevelScratch *ls = reinterpret_cast<MatchLevelScratch *>(smem + L.lsc);  // LEV only
    uint64_t *bar = reinterpret_cast<uint64_t *>(smem + L.bar);  // [2]

    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nthr = blockDim.x, nwarp = nthr >> 5;
    const uint32_t tx_bytes = (uint32_t)((BX * wyp * wz + BTX * BY * BZ) * (int)sizeof(T));

    // this thread's lines
    LineUnit un;
    static_assert(LPT == 1 || (LPT == 2 && !ANI && !std::is_same<T, float>::value), "lines per thread");
    const bool has_unit = line_unit<LPT>(a.unit_of[tid], py, pz, un);
    const int dz1 = un.dz0 + (un.along_z ? 1 : 0), dy1 = un.dy0 + (un.along_z ? 0 : 1);

    // ---- thread 0's work-item bookkeeping ----------------------------------
    auto locate = [&](int w, int &j, int &i) {
        j = 0;
        while (j + 1 < a.n_jobs && w >= sc->jstart[j + 1]) ++j;
        i = w - sc->jstart[j];
    };
    // Work items come from a queue: the next candidate (pf) has its centre
    // loaded a block ahead (pfx..), and the one after it (qn) was taken from
    // the queue head a block before it is needed, so neither the atomic's
    // nor the load's latency is waited on.  A CTA takes increasing indices,
    // so once a candidate is past the end every later one is too.
    int pf = 0, pfx = 0, pfy = 0, pfz = 0, qn = 0;
    auto take = [&]() { return (int)gridDim.x + atomicAdd(a.queue, 1); };
    auto centre = [&](int w, int &c0, int &c1, int &c2) {
        int j, i;
        locate(w, j, i);
        const int32_t *c = a.jobs[j].centers + 3 * i;
        c0 = c[0];
        c1 = c[1];
        c2 = c[2];
    };
    // next work item whose centre is inside, from the candidate on (the
    // skipped ones are reported invalid).  Records its centre in cen[buf]
    // and moves the queue one item on.
    auto advance = [&](int n, int buf) {
        int w = pf;
        int c0 = pfx, c1 = pfy, c2 = pfz;
        while (w < n) {
            int j, i;
            locate(w, j, i);
            const MatchJob &Jw = a.jobs[j];
            if (center_inside(c0, c1, c2, Jw.nx, Jw.ny, Jw.nz, H, HY, HZ)) {
                sc->cen[buf][0] = c0;
                sc->cen[buf][1] = c1;
                sc->cen[buf][2] = c2;
                sc->cen[buf][3] = j;
                sc->cen[buf][4] = i;
                sc->cen[buf][5] = 0;
                break;
            }
            write_invalid(a.jobs[j], i, PxF, PyF, Rx, Ry, Rz);
            if (qn >= n) {
                w = n;
                break;
            }
            w = qn;  // skipped: the next candidate at once
            qn = take();
            centre(w, c0, c1, c2);
        }
        if (w >= n) return n;
        pf = qn;
        if (pf < n) {
            centre(pf, pfx, pfy, pfz);
            qn = take();
        }
        return w;
    };
    // the next item: the block's next sub-window, else the next block
    auto next_item = [&](int n, int buf, int cur_blk, int cur_s, int &ns) {
        if (cur_s + 1 < nsubt) {
            for (int q = 0; q < 5; ++q) sc->cen[buf ^ 1][q] = sc->cen[buf][q];
            sc->cen[buf ^ 1][5] = cur_s + 1;
            ns = cur_s + 1;
            return cur_blk;
        }
        ns = 0;
        return advance(n, buf ^ 1);
    };
    // both copies of the item recorded in cen[buf] into buffer buf
    auto issue = [&](int buf) {
        const int cx = sc->cen[buf][0], cy = sc->cen[buf][1], cz = sc->cen[buf][2];
        const MatchJob &Jb = a.jobs[sc->cen[buf][3]];
        const CUtensorMap *mJ = Jb.mapJ ? Jb.mapJ : tmapJ, *mI = Jb.mapI ? Jb.mapI : tmapI;
        int ox, oy, oz;
        sub_off(sc->cen[buf][5], ox, oy, oz);
        const int x0 = cx + ox - H - RX, xt = cx - H;
        fence_proxy_async_smem();
        mbar_arrive_expect_tx(bar + buf, tx_bytes);
        tma_load_3d(smem + L.u[buf], mJ, bar + buf, x0 & ~(ALIGN - 1), cy + oy - HY - ry, cz + oz - HZ - rz);
        tma_load_3d(smem + L.ut[buf], mI, bar + buf, xt & ~(ALIGN - 1), cy - HY, cz - HZ);
    };

    if (tid == 0) {
        int w = 0;
        for (int j = 0; j < a.n_jobs; ++j) {
            if (a.jobs[j].mapJ) tensormap_acquire(a.jobs[j].mapJ);
            if (a.jobs[j].mapI) tensormap_acquire(a.jobs[j].mapI);
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
        pf = blockIdx.x;
        if (pf < w) centre(pf, pfx, pfy, pfz);
        qn = take();
        const int first = advance(w, 0);
        sc->nb[1] = first;  // the loop starts with buffer 0 holding `first`
        sc->ns[1] = 0;
        if (first < w) issue(0);
    }
    __syncthreads();
    const int n = sc->jstart[a.n_jobs];  // blocks over all jobs
    int blk = sc->nb[1];

    uint32_t phase[2] = {0u, 0u};
    int i = 0;
    while (blk < n) {
        const int b = i & 1;
        const T *U = reinterpret_cast<const T *>(smem + L.u[b]);
        const T *Ut = reinterpret_cast<const T *>(smem + L.ut[b]);
        const int cx = sc->cen[b][0], cy = sc->cen[b][1], cz = sc->cen[b][2];
        const MatchJob &J = a.jobs[sc->cen[b][3]];
        const int bi = sc->cen[b][4];
        const int nx = J.nx, ny = J.ny, nz = J.nz;  // this block's volumes
        float cv_pre = 0.f;  // float32: c of the box sums, loaded ahead of the statistics
        if constexpr (F32)
            if (tid == 0) cv_pre = reinterpret_cast<const float *>(J.intraop)[volume_centre_index(nx, ny, nz)];
        const int si = sc->cen[b][5];  // sub-window of this item
        int x0;
        {
            int ox, oy, oz;
            sub_off(si, ox, oy, oz);
            x0 = cx + ox - H - RX;
        }
        const int xo = x0 - (x0 & ~(ALIGN - 1));
        const int xt = cx - H, xot = xt - (xt & ~(ALIGN - 1));
        // this thread's box sums of the item, copied while it searches
        const uint32_t bs_base = smem_addr(smem + L.bs) + 4u * (uint32_t)tid, bs_str = (uint32_t)nthr;
        if (a.stage && has_unit) {
            int ox, oy, oz;
            sub_off(si, ox, oy, oz);
            line_boxsums_async<B, P>(a, J, cx + ox, cy + oy, cz + oz, un.dy0, un.dz0, HY, HZ, bs_base,
                                     bs_base + 4u * P * bs_str, bs_str);
            if (un.two)
                line_boxsums_async<B, P>(a, J, cx + ox, cy + oy, cz + oz, dy1, dz1, HY, HZ, bs_base + 8u * P * bs_str,
                                         bs_base + 12u * P * bs_str, bs_str);
            cp_async_commit();
        }

        const bool got = mbar_wait_bounded(bar + b, phase[b], a.wait_ns);
        phase[b] ^= 1u;
        // window rows realigned to start at element 0 (read after barrier T)
        if (xo && got) realign_window<T, BX>(const_cast<T *>(U), wyp, BY + 2 * ry, wz, xo, tid, nthr);
        // thread 0: the next block (its centre goes to the other buffer's
        // record, read by every thread after this block's last barrier)
        if (tid == 0) {
            int ns;
            sc->nb[b] = next_item(n, b, blk, si, ns);
            sc->ns[b] = ns;
        }

        // ---- floating block statistics: every warp sums the whole block ----
        // uint16: exact integer sums; thread 0 stores the block constants.
        // float32: float-float sums of the values shifted by the block's
        // first value; thread 0 derives the FP64 constants.
        bool flat;
        int m = 0;        // uint16: nearest integer to the block mean
        float tsh = 0.f;  // float32: the float mean mu used for T
        if constexpr (F32) {
            const float i0 = Ut[xot];
            FF s1{0.f, 0.f}, s2{0.f, 0.f};
            float lo = INFINITY, hi = -INFINITY;
            for (int row = lane; row < NROW; row += 32) {
                float vals[B];
#pragma unroll
                for (int kx = 0; kx < B; ++kx) vals[kx] = Ut[row * BTX + xot + kx];
#pragma unroll
                for (int kx = 0; kx < B; ++kx) {
                    float dh, de;
                    two_sum(vals[kx], -i0, dh, de);
                    s1 = ff_add2(s1, dh, de);
                    const float p = __fmul_rn(dh, dh);  // (dh + de)^2; de^2 is below the pair's precision
                    s2 = ff_add2(s2, p, __fmaf_rn(2.f * dh, de, __fmaf_rn(dh, dh, -p)));
                    lo = fminf(lo, vals[kx]);
                    hi = fmaxf(hi, vals[kx]);
                }
            }
            s1 = warp_sum_ff(s1);
            s2 = warp_sum_ff(s2);
            lo = warp_min_f(lo);
            hi = warp_max_f(hi);
            // any float near the mean serves as the shift mu
            tsh = __fadd_rn(i0, __fmul_rn(s1.h, 1.0f / (float)N));
            flat = !(lo < hi);
            if (tid == 0 && !flat) {
                const double d1 = ff_to_double(s1), d2 = ff_to_double(s2);  // sums of (I - I0) and (I - I0)^2
                const double ibar = (double)i0 + d1 / (double)N;
                double dv = d2 - d1 * (d1 / (double)N);  // sum (I - Ibar)^2
                if (dv < 0.0) dv = 0.0;
                BlockConstF &c = sc->bc;
                c.ibh = (float)ibar;
                c.ibl = (float)(ibar - (double)c.ibh);
                const double em = ibar - (double)tsh;
                c.emu = (float)em;
                c.cv = cv_pre;
                // the mean's error: the float-float sum of the N terms I - I0
                // errs by at most 2^-36 sum |I - I0| <= 2^-36 sqrt(N d2), and
                // i0 + d1 / N rounds twice in FP64; emu's own rounding (and
                // that of em) stays within 2u |emu|
                c.eI = __double2float_ru((0x1p-36 * sqrt((double)N * d2) / (double)N +
                                          0x1p-52 * (fabs((double)i0) + fabs(d1) / (double)N)) * 1.01);
                c.dvI = dv;
                c.fvI = (float)dv;
                // sum of T^2 with T = fl(I - mu): at most (1+u)^2 sum (I - mu)^2
                // = (1+u)^2 (sum (I - Ibar)^2 + N (Ibar - mu)^2); the
                // float-float sums (about 2^-48 relative per step, tens of
                // steps) leave the spread inexact by well under 2048 ulp of d2
                c.kq = (float)(sqrt((dv + 2048.0 * 1.1102230246251565e-16 * d2 + (double)N * em * em) * (1.0 + 2.4e-7)) *
                               (1.0 + 1e-6));
            }
        } else {
            int s1 = 0;
            unsigned long long s2 = 0;
            for (int row = lane; row < NROW; row += 32) {
                uint32_t vals[B];
#pragma unroll
                for (int kx = 0; kx < B; ++kx) vals[kx] = Ut[row * BTX + xot + kx];
#pragma unroll
                for (int kx = 0; kx < B; ++kx) {
                    s1 += (int)vals[kx];
                    s2 += (unsigned long long)(vals[kx] * vals[kx]);  // below 2^32
                }
            }
            s1 = warp_sum(s1);
            s2 = warp_sum(s2);
            const long long vI = (long long)N * (long long)s2 - (long long)s1 * s1;
            m = (int)((2u * (uint32_t)s1 + (uint32_t)N) / (2u * (uint32_t)N));
            flat = vI == 0;
            if (tid == 0 && !flat) {
                BlockConstU &c = sc->bu;
                c.vI = vI;
                c.m = m;
                c.rr = (long long)N * m - s1;
                c.frr = (float)(int)c.rr;
                c.fvI = (float)vI;
                // kq = N gamma_L sqrt(qt), qt = sum (I - m)^2 exact below
                // 2^48, rounded up in float: qt becomes a float through two
                // exact 24-bit halves and one rounding; the factor 1 + 4e-6
                // covers that rounding and the rounding of N gamma_L
                const long long qt = (long long)s2 - 2ll * m * s1 + (long long)N * m * m;
                const float qf = __fmaf_rn((float)(int)(qt >> 24), 16777216.f, (float)(int)(qt & 0xFFFFFF));
                c.kq = __fmul_ru(__fmul_ru((float)((double)N * GAMMA_L), __fsqrt_ru(qf)), 1.000004f);
            }
        }

        // ---- template ---------------------------------------------------------
        if (!flat) {
            const int TB = NROW * PT;
            for (int k = tid; k < TB; k += nthr) {
                const int row = k / PT, kx = k - row * PT;
                float t = 0.f;
                if (kx < B) {
                    if constexpr (F32)
                        t = __fsub_rn(Ut[row * BTX + xot + kx], tsh);
                    else
                        t = __fmul_rn(u16_minus(Ut[row * BTX + xot + kx], 8388608.0f + (float)m), TSCALE);
                }
                Ts[k] = t;
            }
        }

        // ---- barrier T: template written, copies landed (or gave up) --------
        if (!__syncthreads_and(got)) {
            if (tid == 0) {
                atomicOr(a.err, DEV_ERR_TIMEOUT);
                write_invalid(J, bi, PxF, PyF, Rx, Ry, Rz);
            }
            // let an in-flight copy land before exiting (the full limit:
            // a copy into this CTA's shared memory must not outlive it)
            mbar_wait_bounded(bar + b, phase[b] ^ 1u, DEVICE_WAIT_NS);
            cp_async_wait_all();
            return;
        }
        const int nb = sc->nb[b];
        // buffer b^1 was last read before the previous block's last barrier
        if (!single && nb < n && tid == 0) issue(b ^ 1);
        if (flat) {  // flat floating block: NCC undefined for every shift
            if (single && nb < n && tid == 0) issue(b ^ 1);  // the window is not read
            if (tid == 0) write_invalid(J, bi, PxF, PyF, Rx, Ry, Rz);
            cp_async_wait_all();  // the next item's copies reuse the staging words
            blk = nb;
            ++i;
            continue;
        }
        BlockConstF bcf;
        if constexpr (F32) bcf = sc->bc;

        // ---- search: FP32 accumulation of A(d) over the window, two lines ----
        float ub0[P], ub1[P];
        float lbm = -INFINITY;
        const int nl = LEV ? J.n_levels : 0;  // extra radius levels of this block's job
        float lbl[MATCH_MAX_LEVELS];
#pragma unroll
        for (int l = 0; l < MATCH_MAX_LEVELS; ++l) lbl[l] = -INFINITY;
#pragma unroll
        for (int p = 0; p < P; ++p) {
            ub0[p] = -INFINITY;
            ub1[p] = -INFINITY;
        }
        if (has_unit) {
            float acc0[P], acc1[P];
            const T *row0 = U + (un.dz0 * wyp + un.dy0) * BX;
            const int sI = un.along_z ? wyp * BX : BX, sO = un.along_z ? BX : wyp * BX;
            const int tI = un.along_z ? BY : 1, tO = un.along_z ? 1 : BY;
            const int bI = un.along_z ? BZ : BY, bO = un.along_z ? BY : BZ;
            // centring constant: the floating block's mean (uint16: the
            // subnormal m * 2^-149, whose bits are m)
            const float csh = F32 ? tsh : __uint_as_float((uint32_t)m);
            if constexpr (LPT == 1)
                search_line<T, B, P>(row0, sO, Ts, bO, bI, csh, acc0);
            else
                search_pair<T, B, P>(row0, sI, sO, Ts, tI, tO, bI, bO, csh, acc0, acc1);
            // the sub-window offset is read again (no registers held across
            // the search)
            int ox, oy, oz;
            sub_off(sc->cen[b][5], ox, oy, oz);
            typedef typename std::conditional<F32, float, int32_t>::type S1T;
            const float kq = F32 ? 0.f : sc->bu.kq, fvI = F32 ? 0.f : sc->bu.fvI, frr = F32 ? 0.f : sc->bu.frr;
            if (a.stage) {
                // the staged box sums (this thread's own copies)
                const uint32_t va = line_vmask<B, P>(a, J, cx + ox, cy + oy, cz + oz, un.dy0, un.dz0, HY, HZ);
                const uint32_t vb = un.two ? line_vmask<B, P>(a, J, cx + ox, cy + oy, cz + oz, dy1, dz1, HY, HZ) : 0u;
                cp_async_wait_all();
                const S1T *st1 = reinterpret_cast<const S1T *>(smem + L.bs) + tid;
                const float *st2 = reinterpret_cast<const float *>(smem + L.bs) + tid;
                const int q = nthr * P;
                line_bounds<T, B, P, LEV>(
                    J, nl, un.dy0, un.dz0, ry, rz, N, BY, BZ, acc0, [&](int p) { return st1[p * nthr]; },
                    [&](int p) { return st2[q + p * nthr]; }, va, kq, fvI, frr, m, tsh, bcf, GAMMA_L, ub0, lbm, lbl);
                if (un.two)
                    line_bounds<T, B, P, LEV>(
                        J, nl, dy1, dz1, ry, rz, N, BY, BZ, acc1, [&](int p) { return st1[2 * q + p * nthr]; },
                        [&](int p) { return st2[3 * q + p * nthr]; }, vb, kq, fvI, frr, m, tsh, bcf,
                        GAMMA_L, ub1, lbm, lbl);
            } else {
                // the box sums straight from global memory, in the bounds loop
                const uint32_t va = line_vmask<B, P>(a, J, cx + ox, cy + oy, cz + oz, un.dy0, un.dz0, HY, HZ);
                const uint32_t vb = un.two ? line_vmask<B, P>(a, J, cx + ox, cy + oy, cz + oz, dy1, dz1, HY, HZ) : 0u;
                const S1T *g1 = reinterpret_cast<const S1T *>(J.s1);
                const float *g2 = reinterpret_cast<const float *>(J.s2);
                const long long ra = va ? line_row(J, cx + ox - RX, cy + oy, cz + oz, un.dy0 - ry, un.dz0 - rz) : 0;
                line_bounds<T, B, P, LEV>(J, nl, un.dy0, un.dz0, ry, rz, N, BY, BZ, acc0,
                                          [&](int p) { return g1[ra + p]; }, [&](int p) { return g2[ra + p]; }, va,
                                          kq, fvI, frr, m, tsh, bcf, GAMMA_L, ub0, lbm, lbl);
                if (un.two) {
                    const long long rb = vb ? line_row(J, cx + ox - RX, cy + oy, cz + oz, dy1 - ry, dz1 - rz) : 0;
                    line_bounds<T, B, P, LEV>(J, nl, dy1, dz1, ry, rz, N, BY, BZ, acc1,
                                              [&](int p) { return g1[rb + p]; }, [&](int p) { return g2[rb + p]; },
                                              vb, kq, fvI, frr, m, tsh, bcf, GAMMA_L, ub1, lbm, lbl);
                }
            }
        }

        // ---- best lower bound over the window ------------------------------
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
        // ---- barrier A: every warp's lower bounds ---------------------------
        __syncthreads();
        // float32 reads the window only in the search (its rescoring reads
        // global memory): a shared window buffer is refilled from here
        if constexpr (F32)
            if (single && nb < n && tid == 0) issue(b ^ 1);
        float LB = -INFINITY;
        for (int w = 0; w < nwarp; ++w) LB = fmaxf(LB, sc->wlb[w]);
        float LBl[MATCH_MAX_LEVELS];
#pragma unroll
        for (int l = 0; l < MATCH_MAX_LEVELS; ++l) {
            LBl[l] = INFINITY;
            if (LEV && l < nl) {
                LBl[l] = -INFINITY;
                for (int w = 0; w < nwarp; ++w) LBl[l] = fmaxf(LBl[l], ls->wlbl[l][w]);
            }
        }
        // surviving x-shifts of this thread's lines: bits 0..P-1 line 0,
        // bits 16.. line 1
        uint32_t smask = 0;
        if (has_unit) {
            smask = line_survivors<P, LEV>(J, nl, un.dy0, un.dz0, ry, rz, ub0, LB, LBl);
            if (un.two) smask |= line_survivors<P, LEV>(J, nl, dy1, dz1, ry, rz, ub1, LB, LBl) << 16;
        }

        // ---- exact rescoring of this warp's survivors -------------------------
        Cand wb{0.0, 0, 0, 0};
        int ox, oy, oz;
        sub_off(sc->cen[b][5], ox, oy, oz);
        uint32_t act = __ballot_sync(0xffffffffu, smask != 0);
        while (act) {
            const int src = __ffs(act) - 1;
            act &= act - 1;
            uint32_t mb = __shfl_sync(0xffffffffu, smask, src);
            LineUnit su;
            line_unit<LPT>(a.unit_of[warp * 32 + src], py, pz, su);
            while (mb) {
                const int bit = __ffs(mb) - 1;
                mb &= mb - 1;
                const int second = bit >> 4, sxi = bit & 15;
                const int syi = su.dy0 + (second && !su.along_z ? 1 : 0);
                const int szi = su.dz0 + (second && su.along_z ? 1 : 0);
                // the shift in the full search box (this sub-window's offset added)
                const int dx = sxi - RX + ox, dy = syi - ry + oy, dz = szi - rz + oz;
                const int code = ((dz + Rz) * PyF + (dy + Ry)) * PxF + (dx + Rx);
                Cand c{0.0, dx * dx + dy * dy + dz * dz, code, 0};
                if constexpr (!F32) {
                    const int mm = sc->bu.m;
                    // sums of T J, J^2 and J over the block, exact
                    const int KPL = (N + 31) / 32;
                    constexpr int CH = ANI ? 6 : ((N3 + 31) / 32 < 6 ? (N3 + 31) / 32 : 6);
                    long long e = 0;
                    unsigned long long q2 = 0;
                    int s1 = 0;
#pragma unroll 1
                    for (int i0 = 0; i0 < KPL; i0 += CH) {
                        int tv[CH];
                        uint32_t jv[CH];
#pragma unroll
                        for (int q = 0; q < CH; ++q) {
                            const int k = lane + 32 * (i0 + q);
                            const int kz = k / (B * BY), rem = k - kz * B * BY, ky = rem / B, kx = rem - ky * B;
                            tv[q] = 0;
                            jv[q] = 0;
                            if (k < N) {
                                tv[q] = (int)Ut[(kz * BY + ky) * BTX + xot + kx] - mm;
                                jv[q] = U[((szi + kz) * wyp + (syi + ky)) * BX + sxi + kx];
                            }
                        }
#pragma unroll
                        for (int q = 0; q < CH; ++q) {
                            e += (long long)tv[q] * (int)jv[q];
                            q2 += (unsigned long long)(jv[q] * jv[q]);
                            s1 += (int)jv[q];
                        }
                    }
                    e = warp_sum(e);
                    q2 = warp_sum(q2);
                    s1 = warp_sum(s1);
                    if (lane == 0) {
                        const long long vJ = (long long)N * (long long)q2 - (long long)s1 * s1;  // N S_JJ - S_J^2
                        const long long num = (long long)N * e + sc->bu.rr * s1;  // N S_IJ - S_I S_J
                        if (vJ > 0) {
                            const double den = __dsqrt_rn(__dmul_rn((double)sc->bu.vI, (double)vJ));
                            c.s = __ddiv_rn((double)num, den);
                            c.ok = 1;
                        }
                    }
                } else {
                    const float *pre = reinterpret_cast<const float *>(J.preop);
                    const float *intra = reinterpret_cast<const float *>(J.intraop);
                    // float-float sums of (I - Ibar) G, G and G^2 with
                    // G = J - J0, J0 the reference block's first value: the
                    // shifted values carry the block's spread, not its mean,
                    // so sum G^2 - (sum G)^2 / N does not cancel however large
                    // the intensities' offset (FP32 pipe; G exact as gh + ge)
                    const size_t jrow = ((size_t)(cz + dz - HZ) * ny + (cy + dy - HY)) * nx + (cx + dx - H);
                    const float j0 = intra[jrow];
                    FF fij{0.f, 0.f}, fj{0.f, 0.f}, fjj{0.f, 0.f};
                    float lo = INFINITY, hi = -INFINITY;
                    for (int k = lane; k < N; k += 32) {
                        const int kz = k / (B * BY), rem = k - kz * B * BY, ky = rem / B, kx = rem - ky * B;
                        const float iv = pre[((size_t)(cz - HZ + kz) * ny + (cy - HY + ky)) * nx + (cx - H + kx)];
                        const float jf = intra[jrow + ((size_t)kz * ny + ky) * nx + kx];
                        float dh, de;
                        two_sum(iv, -bcf.ibh, dh, de);  // I - Ibar = dh + dl, nearly exact
                        const float dl = __fsub_rn(de, bcf.ibl);
                        float gh, ge;
                        two_sum(jf, -j0, gh, ge);  // G = J - J0 = gh + ge, exact
                        // (dh + dl)(gh + ge): the product dh*gh exactly, the
                        // cross terms to float precision, dl*ge below it
                        const float p = __fmul_rn(dh, gh);
                        fij = ff_add2(fij, p, __fmaf_rn(dl, gh, __fmaf_rn(dh, ge, __fmaf_rn(dh, gh, -p))));
                        fj = ff_add2(fj, gh, ge);
                        const float q = __fmul_rn(gh, gh);
                        fjj = ff_add2(fjj, q, __fmaf_rn(2.f * gh, ge, __fmaf_rn(gh, gh, -q)));
                        lo = fminf(lo, jf);
                        hi = fmaxf(hi, jf);
                    }
                    fij = warp_sum_ff(fij);
                    fj = warp_sum_ff(fj);
                    fjj = warp_sum_ff(fjj);
                    lo = warp_min_f(lo);
                    hi = warp_max_f(hi);
                    if (lane == 0 && lo < hi) {
                        const double sij = ff_to_double(fij), sj = ff_to_double(fj), sjj = ff_to_double(fjj);
                        const double vJ = sjj - sj * sj / (double)N;
                        if (vJ > 0.0) {
                            c.s = sij / sqrt(bcf.dvI * vJ);
                            c.ok = 1;
                        }
                    }
                }
                if (lane == 0) {
                    if (cand_better(c, wb)) wb = c;
                    if constexpr (LEV)
                        for (int l = 0; l < nl; ++l)
                            if (in_level(code, J.levels[l].r, PxF, PyF, Rx, Ry, Rz)) {
                                const Cand cur{ls->lbs[l][warp], ls->lbn2[l][warp], ls->lbcode[l][warp],
                                               ls->lbok[l][warp]};
                                if (cand_better(c, cur)) {
                                    ls->lbs[l][warp] = c.s;
                                    ls->lbn2[l][warp] = c.n2;
                                    ls->lbcode[l][warp] = c.code;
                                    ls->lbok[l][warp] = c.ok;
                                }
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
        // ---- barrier C: every warp's best survivor -----------------------------
        __syncthreads();
        if constexpr (!F32)  // uint16 rescoring read the window up to here
            if (single && nb < n && tid == 0) issue(b ^ 1);
        if (tid == 0) {
            Cand best{0.0, 0, 0, 0};
            for (int w = 0; w < nwarp; ++w) {
                Cand c{sc->bs[w], sc->bn2[w], sc->bcode[w], sc->bok[w]};
                if (cand_better(c, best)) best = c;
            }
            // over the block's sub-windows (in order, in this CTA): the
            // best so far, written with the last one
            if (nsubt > 1) {
                if (si > 0 && !cand_better(best, sc->sbest)) best = sc->sbest;
                sc->sbest = best;
            }
            if (si == nsubt - 1) write_result(J, bi, best, PxF, PyF, Rx, Ry, Rz);
            if constexpr (LEV)
                for (int l = 0; l < nl; ++l) {
                    Cand bl{0.0, 0, 0, 0};
                    for (int w = 0; w < nwarp; ++w) {
                        Cand c{ls->lbs[l][w], ls->lbn2[l][w], ls->lbcode[l][w], ls->lbok[l][w]};
                        if (cand_better(c, bl)) bl = c;
                    }
                    write_out(J.levels[l].disp, J.levels[l].ncc, J.levels[l].valid, bi, bl, PxF, PyF, Rx, Ry, Rz);
                }
        }
        blk = nb;
        ++i;
    }
    // every copy issued was waited for: a block's copies are issued only
    // when the loop is certain to visit it next
}

// Host side: launch one (element type, block size, x-shift count) variant.
// Register budget per thread: what two lines of P x-shifts (search sums,
// then bounds) need without spilling, so that small CTAs (two warps for
// lines of 11 or fewer) fit nine or more to an SM: uint16 blocks up to 7
// take 104 up to 9 shifts and 112 for 11; everything else 128.
template <bool F32, int B, int P>
struct MatchRegs {
    static constexpr int value = !F32 && B <= 7 ? (P <= 9 ? 104 : P <= 11 ? 112 : 128) : 128;
};
template <int B, int P, bool LEV, bool ANI, int LPT>
__global__ void __maxnreg__((MatchRegs<false, B, P>::value))
    match_kernel_u16(const __grid_constant__ MatchParams a, const __grid_constant__ CUtensorMap tmapJ,
                     const __grid_constant__ CUtensorMap tmapI)
{
    match_body<uint16_t, B, P, LEV, ANI, LPT>(a, &tmapJ, &tmapI);
}

template <int B, int P, bool ANI>
__global__ void __maxnreg__((MatchRegs<true, B, P>::value))
    match_kernel_f32(const __grid_constant__ MatchParams a, const __grid_constant__ CUtensorMap tmapJ,
                     const __grid_constant__ CUtensorMap tmapI)
{
    match_body<float, B, P, false, ANI, 1>(a, &tmapJ, &tmapI);
}

template <typename T, int B, int P, bool LEV, bool ANI, int LPT>
constexpr auto match_kernel_ptr()
{
    if constexpr (std::is_same<T, float>::value)
        return match_kernel_f32<B, P, ANI>;  // float32 jobs report no extra levels
    else
        return match_kernel_u16<B, P, LEV, ANI, LPT>;
}

// Shared-memory layout of a launch: double-buffered windows, unless that
// leaves three or fewer CTAs per SM and a single window buffer gives more
// (the other CTAs then hide the exposed copy latency; measured on float32
// windows: b = 9, R = 7 from 1 to 2 CTAs, 23% faster; b = 7, R = 5 from 3 to
// 6 CTAs, 16% faster).
// Block edges along y and z of a launch (0 in MatchLaunch: the x edge).
inline int launch_by(const MatchLaunch &m) { return m.block_y > 0 ? m.block_y : m.block; }
inline int launch_bz(const MatchLaunch &m) { return m.block_z > 0 ? m.block_z : m.block; }

// Host: the order of line units over threads.  A type A unit's 16-byte
// window loads start at bank group ((dz * wyp + dy) * bxc) mod 8 (bxc =
// 16-byte chunks per window row) and move in step with every other type A
// unit's, so units are dealt to groups of 8 consecutive threads with
// distinct start groups as far as the counts allow; the type B and single
// units, whose loads move differently, follow.  One line per thread keeps
// the identity order (consecutive threads are a window plane apart).
inline void match_unit_order(int py, int pz, int wyp, int bxc, int lpt, int threads, uint8_t *unit_of)
{
    for (int k = 0; k < MATCH_MAX_THREADS_C; ++k) unit_of[k] = 255;
    const int nu = match_units(py, pz, lpt);
    if (lpt == 1) {
        for (int k = 0; k < nu && k < threads; ++k) unit_of[k] = (uint8_t)k;
        return;
    }
    const int nA = pz * (py / 2);
    std::vector<int> byg[8];
    for (int k = nA - 1; k >= 0; --k) {
        const int dz = k % pz, dy = 2 * (k / pz);
        byg[((dz * wyp + dy) * bxc) & 7].push_back(k);
    }
    // each group of 8 threads: one unit from each of the fullest start
    // groups, then, if fewer than 8 groups are left, further units anyway
    int t = 0, left = nA;
    while (left > 0) {
        int order[8];
        for (int g = 0; g < 8; ++g) order[g] = g;
        std::sort(order, order + 8, [&](int x, int y) { return byg[x].size() > byg[y].size(); });
        int n = 0;
        for (int q = 0; q < 8 && left > 0; ++q)
            if (!byg[order[q]].empty()) {
                unit_of[t++] = (uint8_t)byg[order[q]].back();
                byg[order[q]].pop_back();
                --left;
                ++n;
            }
        for (int q = 0; n < 8 && left > 0; q = (q + 1) & 7)
            if (!byg[order[q]].empty()) {
                unit_of[t++] = (uint8_t)byg[order[q]].back();
                byg[order[q]].pop_back();
                --left;
                ++n;
            }
    }
    for (int k = nA; k < nu; ++k) unit_of[t++] = (uint8_t)k;
}

template <typename T, int B, int P, bool LEV, bool ANI, int LPT>
nrr_status choose_layout(const MatchLaunch &m, MatchLayout *L, bool *single, bool *stage, int *occ)
{
    constexpr int ALIGN = 16 / (int)sizeof(T);
    const int by = launch_by(m), bz = launch_bz(m);
    const int ry = m.sub_r[1], rz = m.sub_r[2], py = 2 * ry + 1, pz = 2 * rz + 1;
    const int wyp = match_wyp(by + 2 * ry, py), threads = round_up_i(match_units(py, pz, LPT), 32);
    // [stage][single]: box sums staged or loaded at the bounds, two window
    // buffers or one
    MatchLayout Ls[2][2];
    int most = 0;
    for (int st = 0; st < 2; ++st)
        for (int sw = 0; sw < 2; ++sw) {
            Ls[st][sw] = match_layout((int)sizeof(T), B, P, match_bx<T, B, P>(), round_up_c(B + ALIGN - 1, ALIGN), wyp,
                                      bz + 2 * rz, py, pz, sw != 0, LEV, by * bz, st != 0, threads);
            most = Ls[st][sw].total > most ? Ls[st][sw].total : most;
        }
    auto kern = match_kernel_ptr<T, B, P, LEV, ANI, LPT>();
    static int smem_set = 0;  // largest dynamic shared memory opted in so far
    if (most > smem_set) {
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, most);
        if (e == cudaSuccess)
            e = cudaFuncSetAttribute(kern, cudaFuncAttributePreferredSharedMemoryCarveout, cudaSharedmemCarveoutMaxShared);
        if (e != cudaSuccess) return cuda_fail(e, "cudaFuncSetAttribute(match_kernel)");
        smem_set = most;
    }
    int o[2][2];
    for (int st = 0; st < 2; ++st)
        for (int sw = 0; sw < 2; ++sw) {
            cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&o[st][sw], kern, threads, Ls[st][sw].total);
            if (e != cudaSuccess) return cuda_fail(e, "cudaOccupancyMaxActiveBlocksPerMultiprocessor");
        }
    // one window buffer where it fits more CTAs on an SM than two (measured:
    // more resident CTAs beat the overlap of the next block's copy), or as
    // asked
    bool sw1[2];
    for (int st = 0; st < 2; ++st) {
        sw1[st] = o[st][1] > o[st][0];
        if (m.windows == 1) sw1[st] = true;
        if (m.windows == 2) sw1[st] = false;
    }
    // box sums loaded at the bounds unless staging is asked for (measured:
    // staging wins only at one or two CTAs per SM)
    const bool stg = m.stage_boxsums == 2;
    *stage = stg;
    *single = sw1[stg];
    *L = Ls[stg][sw1[stg]];
    *occ = o[stg][sw1[stg]];
    return NRR_OK;
}

template <typename T, int B, int P, bool LEV, bool ANI, int LPT>
nrr_status launch_match_variant_l(const MatchLaunch &m, cudaStream_t stream)
{
    constexpr int ALIGN = 16 / (int)sizeof(T);
    constexpr int BX = match_bx<T, B, P>();
    constexpr int BTX = round_up_c(B + ALIGN - 1, ALIGN);
    const int by = launch_by(m), bz = launch_bz(m);
    const int ry = m.sub_r[1], rz = m.sub_r[2], py = 2 * ry + 1, pz = 2 * rz + 1;
    const int wy = by + 2 * ry, wz = bz + 2 * rz, wyp = match_wyp(wy, py);
    const int threads = round_up_i(match_units(py, pz, LPT), 32);
    if (threads > MATCH_MAX_THREADS) return fail(NRR_E_INVALID, "search window too large");
    if (wyp > 256) return fail(NRR_E_INVALID, "search window too large");

    for (int j = 0; j < m.n_jobs; ++j)
        if (m.jobs[j].mapJ || m.jobs[j].mapI) {
            // maps a caller encoded must have this variant's boxes
            int wb[3], tb[3];
            match_boxes(m.dtype, m.block, by, bz, m.radius, wb, tb);
            if (wb[0] != BX || wb[1] != wyp || wb[2] != wz || tb[0] != BTX || tb[1] != by || tb[2] != bz)
                return fail(NRR_E_INTERNAL, "job tensor map boxes differ from the launch's");
            break;
        }
    CUtensorMap mapJ, mapI;
    nrr_status st = encode_volume_map(&mapJ, m.intraop, m.dtype, m.dims, BX, wyp, wz);
    if (st != NRR_OK) return st;
    st = encode_volume_map(&mapI, m.preop, m.dtype, m.dims, BTX, by, bz);
    if (st != NRR_OK) return st;

    auto kern = match_kernel_ptr<T, B, P, LEV, ANI, LPT>();
    MatchLayout L;
    bool single = false;
    int occ = 0;
    bool stage = false;
    st = choose_layout<T, B, P, LEV, ANI, LPT>(m, &L, &single, &stage, &occ);
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
    p.stage = stage ? 1 : 0;
    match_unit_order(py, pz, wyp, BX * (int)sizeof(T) / 16, LPT, threads, p.unit_of);
    p.by = by;
    p.bz = bz;
    for (int j = 0; j < MATCH_MAX_JOBS; ++j) {
        MatchJob jb = j < m.n_jobs ? m.jobs[j] : MatchJob{};
        if (!jb.preop) jb.preop = m.preop;
        if (!jb.intraop) jb.intraop = m.intraop;
        if (!jb.s1) jb.s1 = m.s1;
        if (!jb.s2) jb.s2 = m.s2;
        if (!jb.nx) {
            jb.nx = m.dims.nx;
            jb.ny = m.dims.ny;
            jb.nz = m.dims.nz;
        }
        p.jobs[j] = jb;
    }
    p.err = m.err;
    p.wait_ns = device_wait_ns();
    p.nsubt = 1;
    for (int a = 0; a < 3; ++a) {
        p.R[a] = m.radius[a];
        p.nsub[a] = m.nsub[a];
        p.nsubt *= m.nsub[a];
        for (int q = 0; q < MATCH_MAX_SUB; ++q) p.soff[a][q] = q < m.nsub[a] ? m.soff[a][q] : 0;
    }
    p.queue = m.queue;
    if (!p.queue) {
        cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
        NRR_CUDA_TRY(cudaStreamIsCapturing(stream, &cs));
        if ((st = match_queue_head(&p.queue, cs != cudaStreamCaptureStatusNone)) != NRR_OK) return st;
    }
    NRR_CUDA_TRY(cudaMemsetAsync(p.queue, 0, sizeof(int32_t), stream));
    kern<<<(unsigned)grid, threads, L.total, stream>>>(p, mapJ, mapI);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "match kernel launch");
    count_launches(1);
    return NRR_OK;
}

// Search lines per thread of a launch (sub-windows planned): two only for
// uint16 cubic blocks, as the launch's shape asks, else by the window's
// x-shift count.
inline int match_lines(const MatchLaunch &m)
{
    if (m.dtype != NRR_U16 || launch_by(m) != m.block || launch_bz(m) != m.block) return 1;
    if (m.lines == 1 || m.lines == 2) return m.lines;
    return match_default_lines(2 * m.sub_r[0] + 1);
}

// Launches whose jobs report extra radius levels use the level-aware kernel
// (uint16 only: the batched search runs on uint16 volumes).
// Launches whose blocks have other edges along y or z than along x use the
// variant with those edges at run time (one line per thread).
template <typename T, int B, int P, int LPT>
nrr_status launch_match_variant(const MatchLaunch &m, cudaStream_t stream)
{
    bool lev = false;
    for (int j = 0; j < m.n_jobs; ++j) lev |= m.jobs[j].n_levels > 0;
    const bool ani = launch_by(m) != B || launch_bz(m) != B;
    if constexpr (LPT == 2) {
        if (ani) return fail(NRR_E_INTERNAL, "two lines per thread need a cubic block");
        return lev ? launch_match_variant_l<T, B, P, true, false, 2>(m, stream)
                   : launch_match_variant_l<T, B, P, false, false, 2>(m, stream);
    } else {
        if (ani) {
            if (lev) return fail(NRR_E_INTERNAL, "extra radius levels are not supported for anisotropic blocks");
            return launch_match_variant_l<T, B, P, false, true, 1>(m, stream);
        }
        if (!lev) return launch_match_variant_l<T, B, P, false, false, 1>(m, stream);
        if constexpr (std::is_same<T, float>::value)
            return fail(NRR_E_INTERNAL, "extra radius levels are not supported for float32 volumes");
        else
            return launch_match_variant_l<T, B, P, true, false, 1>(m, stream);
    }
}

template <typename T, int B, int P, int LPT>
nrr_status occupancy_variant(const MatchLaunch &m, int *occ)
{
    MatchLayout L;
    bool single = false;
    bool stage = false;
    if constexpr (LPT == 2) {
        return choose_layout<T, B, P, false, false, 2>(m, &L, &single, &stage, occ);
    } else {
        if (launch_by(m) != B || launch_bz(m) != B)
            return choose_layout<T, B, P, false, true, 1>(m, &L, &single, &stage, occ);
        return choose_layout<T, B, P, false, false, 1>(m, &L, &single, &stage, occ);
    }
}

template <typename T, int B, int LPT>
nrr_status launch_match_b(const MatchLaunch &m, cudaStream_t stream, int *occ)
{
    switch (m.sub_r[0]) {
#define NRR_CASE(r, p) \
    case r: return occ ? occupancy_variant<T, B, p, LPT>(m, occ) : launch_match_variant<T, B, p, LPT>(m, stream);
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
    return fail(NRR_E_INVALID, "sub-window radius x %d outside 0..%d", m.sub_r[0], MATCH_WINDOW_R);
}

// One entry per (element type, block size, lines per thread); defined in the
// instantiation translation units.  Float32 variants take one line per
// thread.
#define NRR_DECL_U16(b)                                                        \
    nrr_status launch_match_u16_b##b##_l1(const MatchLaunch &, cudaStream_t, int *); \
    nrr_status launch_match_u16_b##b##_l2(const MatchLaunch &, cudaStream_t, int *);
NRR_DECL_U16(3)
NRR_DECL_U16(5)
NRR_DECL_U16(7)
NRR_DECL_U16(9)
NRR_DECL_U16(11)
#undef NRR_DECL_U16
nrr_status launch_match_f32_b3(const MatchLaunch &, cudaStream_t, int *);
nrr_status launch_match_f32_b5(const MatchLaunch &, cudaStream_t, int *);
nrr_status launch_match_f32_b7(const MatchLaunch &, cudaStream_t, int *);
nrr_status launch_match_f32_b9(const MatchLaunch &, cudaStream_t, int *);
nrr_status launch_match_f32_b11(const MatchLaunch &, cudaStream_t, int *);

}  // namespace nrr
