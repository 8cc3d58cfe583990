// The robust finite-element update that consumes the block matches (Sec. 3:
// "Estimation of brain deformation is based on the finite element analysis
// ..."; Sec. 5: N_rej approximation (outlier rejection) steps, N_int
// interpolation steps, the rejected fraction F_r):
//
//     F_i = K U_i,    U_{i+1} = [K + H^T S H]^{-1} [H^T S D + F_i].
//
// Mesh: a structured grid of 8-node hexahedra, vertices every g voxels; an
// element belongs to the model when the mask is set at its centre voxel.
// K: homogeneous isotropic linear elasticity (E, nu), 2x2x2 Gauss.  H:
// trilinear interpolation at the block centres.  S: the peak NCC of each
// valid match with positive NCC inside the model.  After each of the first
// N_rej solves, floor(0.5 + F_r n) of the n blocks still trusted -- those
// with the largest squared residual |D_k - H_k U|^2, ties to the lower block
// index, none at or below 1e-6 voxel^2 -- lose their confidence.
//
// One call runs every step on the device:
//   fem_elements / fem_nodes   model membership of elements and vertices;
//   fem_init_blocks            s_k, and -1 in the rejection record;
//   fem_assemble               H^T S H as a scalar 27-point stencil per
//                              vertex and H^T S D, accumulated as 64-bit
//                              fixed-point integers so that the sums do not
//                              depend on the order of the atomics;
//   fem_solve                  conjugate gradients preconditioned by the
//                              inverse 3x3 diagonal block of each vertex, in
//                              FP64 on K + H^T S H, matrix-free (K element by
//                              element around each vertex, the stencil for
//                              H^T S H; three lanes per vertex, one per
//                              neighbour plane), warm-started from U_i until the
//                              residual falls to tol times its start, as ONE
//                              cooperative launch with two bounded grid
//                              barriers per iteration; every CTA sums the
//                              per-CTA partial dot products in the same order,
//                              so all take the same decisions;
//   fem_residuals + fem_reject the squared residuals as order-preserving
//                              64-bit keys and a one-CTA radix select of the
//                              n_rej largest.
#include <math.h>
#include <string.h>

#include <vector>

#include "nrr_internal.h"
#include "nrr_ptx.cuh"

namespace nrr {
namespace {

constexpr int FEM_THREADS = 256;
constexpr int SOLVE_THREADS = 128;  // small CTAs spread a small mesh over every SM
constexpr int REJ_THREADS = 1024;
constexpr double FIX_M = 17592186044416.0;  // 2^44: fixed-point scale of the H^T S H terms (each in [0, 1])
constexpr double FIX_B = 1099511627776.0;   // 2^40: fixed-point scale of the H^T S D terms (|D| < 2^15)
constexpr double R2_MIN = 1e-6;             // squared residual at or below which a block is never rejected
constexpr int MAX_FEM_BLOCKS = 1 << 19;     // keeps every fixed-point sum below 2^63

struct FemGrid {
    int nx, ny, nz;  // volume
    int g;           // vertex spacing (voxels)
    int Nx, Ny, Nz;  // vertices per axis
    int Ex, Ey, Ez;  // elements per axis
    long long nv;    // vertices
};

// The element stiffness, row 3 a + c, column 3 b + d (local nodes a, b;
// components c, d), and the stiffness stencil of a vertex whose 8 elements
// all belong to the model (the 3x3 block coupling it to neighbour o, summed
// over the elements holding both), passed as a kernel parameter and copied
// into shared memory at the start of the solve (the three lanes of a vertex
// read different planes of them).
struct FemKe {
    double k[24 * 24];
    double st[27 * 9];
};

__host__ __device__ inline long long vidx(const FemGrid &G, int i, int j, int k)
{
    return (long long)i + (long long)G.Nx * ((long long)j + (long long)G.Ny * k);
}

// Element holding block centre (cx, cy, cz) and its 8 trilinear weights, in
// the same operations and order as the reading states (t = c / g - i, the
// weight of local node a = ax + 2 ay + 4 az the product over x, y, z of t or
// 1 - t).
__device__ __forceinline__ void block_weights(const FemGrid &G, int cx, int cy, int cz, int &i, int &j, int &k,
                                              double (&w)[8])
{
    const int c[3] = {cx, cy, cz};
    const int N[3] = {G.Nx, G.Ny, G.Nz};
    int e[3];
    double t[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        int v = c[a] / G.g;
        v = v < 0 ? 0 : (v > N[a] - 2 ? N[a] - 2 : v);
        e[a] = v;
        t[a] = __dsub_rn(__ddiv_rn((double)c[a], (double)G.g), (double)v);
    }
    i = e[0];
    j = e[1];
    k = e[2];
#pragma unroll
    for (int a = 0; a < 8; ++a) {
        const double wx = (a & 1) ? t[0] : __dsub_rn(1.0, t[0]);
        const double wy = (a & 2) ? t[1] : __dsub_rn(1.0, t[1]);
        const double wz = (a & 4) ? t[2] : __dsub_rn(1.0, t[2]);
        w[a] = __dmul_rn(__dmul_rn(wx, wy), wz);
    }
}

__global__ void fem_elements_kernel(const uint8_t *__restrict__ mask, FemGrid G, uint8_t *__restrict__ eact)
{
    const long long ne = (long long)G.Ex * G.Ey * G.Ez;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < ne; e += (long long)gridDim.x * blockDim.x) {
        const int i = (int)(e % G.Ex), j = (int)((e / G.Ex) % G.Ey), k = (int)(e / ((long long)G.Ex * G.Ey));
        const int x = min(i * G.g + G.g / 2, G.nx - 1), y = min(j * G.g + G.g / 2, G.ny - 1),
                  z = min(k * G.g + G.g / 2, G.nz - 1);
        eact[e] = mask[((long long)z * G.ny + y) * G.nx + x] != 0;
    }
}

__device__ __forceinline__ bool elem_on(const FemGrid &G, const uint8_t *eact, int i, int j, int k)
{
    if (i < 0 || j < 0 || k < 0 || i >= G.Ex || j >= G.Ey || k >= G.Ez) return false;
    return eact[(long long)i + (long long)G.Ex * ((long long)j + (long long)G.Ey * k)] != 0;
}

__global__ void fem_nodes_kernel(FemGrid G, const uint8_t *__restrict__ eact, uint8_t *__restrict__ nact)
{
    for (long long n = blockIdx.x * (long long)blockDim.x + threadIdx.x; n < G.nv; n += (long long)gridDim.x * blockDim.x) {
        const int i = (int)(n % G.Nx), j = (int)((n / G.Nx) % G.Ny), k = (int)(n / ((long long)G.Nx * G.Ny));
        bool on = false;
#pragma unroll
        for (int a = 0; a < 8; ++a) on |= elem_on(G, eact, i - (a & 1), j - ((a >> 1) & 1), k - ((a >> 2) & 1));
        nact[n] = on;
    }
}

// s_k = NCC_k for a valid match with positive NCC whose element is in the
// model, else 0; the rejection record starts at -1 (never).
__global__ void fem_init_blocks_kernel(FemGrid G, const uint8_t *__restrict__ eact, const int32_t *__restrict__ centers,
                                       const double *__restrict__ ncc, const uint8_t *__restrict__ valid, int n,
                                       double *__restrict__ s, int32_t *__restrict__ step)
{
    for (int b = blockIdx.x * blockDim.x + threadIdx.x; b < n; b += gridDim.x * blockDim.x) {
        int i, j, k;
        double w[8];
        block_weights(G, centers[3 * b], centers[3 * b + 1], centers[3 * b + 2], i, j, k, w);
        const double v = ncc[b];
        s[b] = (valid[b] != 0 && elem_on(G, eact, i, j, k) && v > 0.0) ? v : 0.0;
        step[b] = -1;
    }
}

// H^T S H as 27 stencil coefficients per vertex (neighbour offset o = (dx+1)
// + 3 (dy+1) + 9 (dz+1)) and H^T S D (3 per vertex), summed as fixed-point
// integers: each term s w_a w_b (in [0, 1]) times 2^44 and s w_a D_c times
// 2^40 is rounded to the nearest integer once, so the totals are the same in
// any order of the atomics.
__global__ void fem_assemble_kernel(FemGrid G, const int32_t *__restrict__ centers, const int32_t *__restrict__ disp,
                                    const double *__restrict__ s, int n, unsigned long long *__restrict__ mfix,
                                    unsigned long long *__restrict__ bfix)
{
    for (int b = blockIdx.x * blockDim.x + threadIdx.x; b < n; b += gridDim.x * blockDim.x) {
        const double sk = s[b];
        if (!(sk > 0.0)) continue;
        int i, j, k;
        double w[8];
        block_weights(G, centers[3 * b], centers[3 * b + 1], centers[3 * b + 2], i, j, k, w);
        const double D[3] = {(double)disp[3 * b], (double)disp[3 * b + 1], (double)disp[3 * b + 2]};
#pragma unroll
        for (int a = 0; a < 8; ++a) {
            const long long na = vidx(G, i + (a & 1), j + ((a >> 1) & 1), k + ((a >> 2) & 1));
            const double sw = __dmul_rn(sk, w[a]);
#pragma unroll
            for (int c = 0; c < 3; ++c)
                atomicAdd(bfix + 3 * na + c, (unsigned long long)__double2ll_rn(__dmul_rn(__dmul_rn(sw, D[c]), FIX_B)));
#pragma unroll
            for (int q = 0; q < 8; ++q) {
                const int o = ((q & 1) - (a & 1) + 1) + 3 * (((q >> 1) & 1) - ((a >> 1) & 1) + 1) +
                              9 * (((q >> 2) & 1) - ((a >> 2) & 1) + 1);
                atomicAdd(mfix + 27 * na + o, (unsigned long long)__double2ll_rn(__dmul_rn(__dmul_rn(sw, w[q]), FIX_M)));
            }
        }
    }
}

// The model's vertices in increasing order (one CTA: a block-wide scan per
// round of REJ_THREADS x 8 vertices), so that the solve deals them out
// evenly and in the same order on every run.
__global__ void __launch_bounds__(REJ_THREADS) fem_active_list_kernel(const uint8_t *__restrict__ nact, long long nv,
                                                                      int32_t *__restrict__ alist,
                                                                      int32_t *__restrict__ acount)
{
    constexpr int CH = 8;
    __shared__ int wsum[REJ_THREADS / 32];
    __shared__ int s_base;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nw = blockDim.x >> 5;
    if (tid == 0) s_base = 0;
    __syncthreads();
    for (long long start = 0; start < nv; start += (long long)blockDim.x * CH) {
        const long long v0 = start + (long long)tid * CH;
        int c = 0;
        for (int q = 0; q < CH; ++q) c += (v0 + q < nv && nact[v0 + q]) ? 1 : 0;
        int inc = c;  // inclusive scan over the CTA
        for (int o = 1; o < 32; o <<= 1) {
            const int u = __shfl_up_sync(0xffffffffu, inc, o);
            if (lane >= o) inc += u;
        }
        if (lane == 31) wsum[warp] = inc;
        __syncthreads();
        if (warp == 0) {
            int w = lane < nw ? wsum[lane] : 0;
            for (int o = 1; o < 32; o <<= 1) {
                const int u = __shfl_up_sync(0xffffffffu, w, o);
                if (lane >= o) w += u;
            }
            if (lane < nw) wsum[lane] = w;  // inclusive over warps
        }
        __syncthreads();
        int pos = s_base + (warp ? wsum[warp - 1] : 0) + inc - c;
        for (int q = 0; q < CH; ++q)
            if (v0 + q < nv && nact[v0 + q]) alist[pos++] = (int32_t)(v0 + q);
        __syncthreads();
        if (tid == 0) s_base += wsum[nw - 1];
        __syncthreads();
    }
    if (tid == 0) *acount = s_base;
}

// ---- the solve ------------------------------------------------------------

struct FemSolveArgs {
    FemGrid G;
    const uint8_t *eact, *nact;
    const unsigned long long *mfix, *bfix;
    double *m;     // [nv][27] H^T S H stencil
    double *binv;  // [nv][9] inverse of each vertex's 3x3 diagonal block of K + H^T S H (0 off the model)
    double *x;     // [nv][3] in: U_i, out: U_{i+1}
    double *r, *p0, *p1, *q;  // [nv][3]
    double *z;                // [nv][3] the preconditioned residual B^-1 r, written with r
    double *part;             // [4][gridDim.x] per-CTA partial dot products
    const int32_t *alist;     // the model's vertices in increasing order
    const int32_t *acount;    // their number
    unsigned int *arrive;     // grid-barrier arrivals (zero at launch)
    int32_t *iters;           // iterations taken (-1: a grid barrier gave up, -2: breakdown)
    double *relres;           // final |r| / |r_0|
    double tol;
    int max_iter;
    unsigned int *err;
    uint64_t wait_ns;
};

// Bits a of the elements around vertex (i, j, k) that are in the model:
// element (i - ax, j - ay, k - az), in which the vertex is local node a.
__device__ __forceinline__ unsigned elem_mask(const FemGrid &G, const uint8_t *eact, int i, int j, int k)
{
    unsigned em = 0;
#pragma unroll
    for (int a = 0; a < 8; ++a)
        if (elem_on(G, eact, i - (a & 1), j - ((a >> 1) & 1), k - ((a >> 2) & 1))) em |= 1u << a;
    return em;
}

// Local-node bits a for which neighbour offset o = (dx, dy, dz) stays inside
// the element that has the vertex as node a (compile-time).
__host__ __device__ constexpr unsigned couple_mask(int dx, int dy, int dz)
{
    unsigned cm = 0;
    for (int a = 0; a < 8; ++a) {
        const int bx = (a & 1) + dx, by = ((a >> 1) & 1) + dy, bz = ((a >> 2) & 1) + dz;
        if (bx >= 0 && bx <= 1 && by >= 0 && by <= 1 && bz >= 0 && bz <= 1) cm |= 1u << a;
    }
    return cm;
}

// The part of y = (K + H^T S H) v at vertex (i, j, k) that comes from the
// 9 neighbours in plane dz = pl - 1, with the stiffness stencil `st` (27 x 9)
// and the element stiffness `ke` (24 x 24) in shared memory (the three lanes
// of a vertex read different planes of them).
template <class Get>
__device__ __forceinline__ void apply_A_plane(const FemGrid &G, const double *st, const double *ke, const double *mrow,
                                              unsigned em, int i, int j, int k, int pl, Get get, double (&y)[3])
{
    y[0] = y[1] = y[2] = 0.0;
    const int dz = pl - 1;
    if (em == 0xFFu) {  // interior of the model: the precomputed stencil
        const double *sp = st + 81 * pl;
#pragma unroll
        for (int oo = 0; oo < 9; ++oo) {
            double v[3];
            get(vidx(G, i + oo % 3 - 1, j + oo / 3 - 1, k + dz), v);
            const double mo = mrow[oo + 9 * pl];
#pragma unroll
            for (int c = 0; c < 3; ++c) {
#pragma unroll
                for (int d = 0; d < 3; ++d) y[c] = fma(sp[oo * 9 + 3 * c + d], v[d], y[c]);
                y[c] = fma(mo, v[c], y[c]);
            }
        }
        return;
    }
#pragma unroll
    for (int oo = 0; oo < 9; ++oo) {
        const int dx = oo % 3 - 1, dy = oo / 3 - 1;
        const unsigned on = couple_mask(dx, dy, dz) & em;
        if (!on) continue;
        double v[3];
        get(vidx(G, i + dx, j + dy, k + dz), v);
        for (int a = 0; a < 8; ++a) {
            if (!((on >> a) & 1u)) continue;
            const int b = ((a & 1) + dx) + 2 * (((a >> 1) & 1) + dy) + 4 * (((a >> 2) & 1) + dz);
            const double *kr = ke + 3 * a * 24 + 3 * b;
#pragma unroll
            for (int c = 0; c < 3; ++c)
#pragma unroll
                for (int d = 0; d < 3; ++d) y[c] = fma(kr[c * 24 + d], v[d], y[c]);
        }
        const double mo = mrow[oo + 9 * pl];
#pragma unroll
        for (int c = 0; c < 3; ++c) y[c] = fma(mo, v[c], y[c]);
    }
}

// Inverse of a symmetric positive definite 3x3 matrix (cofactors over the
// determinant), row-major.
__device__ __forceinline__ void inverse3(const double (&B)[3][3], double (&I)[9])
{
    const double c00 = B[1][1] * B[2][2] - B[1][2] * B[2][1], c01 = B[1][2] * B[2][0] - B[1][0] * B[2][2],
                 c02 = B[1][0] * B[2][1] - B[1][1] * B[2][0];
    const double det = B[0][0] * c00 + B[0][1] * c01 + B[0][2] * c02;
    const double id = det > 0.0 ? 1.0 / det : 0.0;
    I[0] = c00 * id;
    I[1] = (B[0][2] * B[2][1] - B[0][1] * B[2][2]) * id;
    I[2] = (B[0][1] * B[1][2] - B[0][2] * B[1][1]) * id;
    I[3] = c01 * id;
    I[4] = (B[0][0] * B[2][2] - B[0][2] * B[2][0]) * id;
    I[5] = (B[0][2] * B[1][0] - B[0][0] * B[1][2]) * id;
    I[6] = c02 * id;
    I[7] = (B[0][1] * B[2][0] - B[0][0] * B[2][1]) * id;
    I[8] = (B[0][0] * B[1][1] - B[0][1] * B[1][0]) * id;
}

// Sum of v over the CTA, in a fixed order; every thread gets the result.
__device__ double cta_sum(double v, double *sh)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    __syncthreads();
    if (lane == 0) sh[warp] = v;
    __syncthreads();
    double t = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += sh[w];
    return t;
}

// Sum of the per-CTA partials of slot `slot`, in the same order in every CTA
// (after a grid barrier; read through L2).
__device__ double grid_total(const double *part, int slot, double *sh)
{
    const int lane = threadIdx.x & 31;
    __syncthreads();
    if (threadIdx.x < 32) {
        double v = 0.0;
        for (int j = lane; j < (int)gridDim.x; j += 32) v += __ldcg(part + (size_t)slot * gridDim.x + j);
        for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        if (lane == 0) sh[0] = v;
    }
    __syncthreads();
    return sh[0];
}

__global__ void __launch_bounds__(SOLVE_THREADS, 1) fem_solve_kernel(const __grid_constant__ FemSolveArgs a,
                                                                  const __grid_constant__ FemKe Ke)
{
    __shared__ double sh[SOLVE_THREADS / 32];
    __shared__ double s_st[27 * 9], s_ke[24 * 24];
    for (int e = threadIdx.x; e < 24 * 24; e += blockDim.x) s_ke[e] = Ke.k[e];
    for (int e = threadIdx.x; e < 27 * 9; e += blockDim.x) s_st[e] = Ke.st[e];
    __syncthreads();
    const FemGrid &G = a.G;
    const long long T = (long long)gridDim.x * blockDim.x, t0 = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    unsigned int bi = 0;  // grid barriers passed

    // ---- set-up: stencil, inverse diagonal, r_0 = H^T S D - H^T S H U_i ----
    double rz = 0.0, rr = 0.0;
    for (long long n = t0; n < G.nv; n += T) {
        double *mrow = a.m + 27 * n;
        for (int o = 0; o < 27; ++o) mrow[o] = (double)(long long)a.mfix[27 * n + o] / FIX_M;
        a.p0[3 * n] = a.p0[3 * n + 1] = a.p0[3 * n + 2] = 0.0;
        if (!a.nact[n]) {
            for (int e = 0; e < 9; ++e) a.binv[9 * n + e] = 0.0;
            for (int c = 0; c < 3; ++c) {
                a.r[3 * n + c] = 0.0;
                a.z[3 * n + c] = 0.0;
                a.x[3 * n + c] = 0.0;
            }
            continue;
        }
        const int i = (int)(n % G.Nx), j = (int)((n / G.Nx) % G.Ny), k = (int)(n / ((long long)G.Nx * G.Ny));
        const unsigned em = elem_mask(G, a.eact, i, j, k);
        double Mx[3] = {0.0, 0.0, 0.0};
        for (int o = 0; o < 27; ++o) {
            if (mrow[o] == 0.0) continue;
            const long long nb = vidx(G, i + o % 3 - 1, j + (o / 3) % 3 - 1, k + o / 9 - 1);
            for (int c = 0; c < 3; ++c) Mx[c] = fma(mrow[o], a.x[3 * nb + c], Mx[c]);
        }
        // the vertex's 3x3 diagonal block of K + H^T S H and its inverse
        // (the block preconditioner: it couples the three components,
        // which a nearly incompressible material ties closely)
        double Bd[3][3], Bi[9];
        for (int c = 0; c < 3; ++c)
            for (int d = 0; d < 3; ++d) {
                double v = c == d ? mrow[13] : 0.0;
                for (int q = 0; q < 8; ++q)
                    if ((em >> q) & 1u) v += Ke.k[(3 * q + c) * 24 + 3 * q + d];
                Bd[c][d] = v;
            }
        inverse3(Bd, Bi);
        double rc[3];
        for (int c = 0; c < 3; ++c) {
            // r_0 = H^T S D + K U_i - (K + H^T S H) U_i
            rc[c] = (double)(long long)a.bfix[3 * n + c] / FIX_B - Mx[c];
            a.r[3 * n + c] = rc[c];
            rr += rc[c] * rc[c];
        }
        for (int c = 0; c < 3; ++c) {
            const double zc = Bi[3 * c] * rc[0] + Bi[3 * c + 1] * rc[1] + Bi[3 * c + 2] * rc[2];
            a.z[3 * n + c] = zc;
            rz += rc[c] * zc;
        }
        for (int e = 0; e < 9; ++e) a.binv[9 * n + e] = Bi[e];
    }
    rr = cta_sum(rr, sh);
    rz = cta_sum(rz, sh);
    if (threadIdx.x == 0) {
        a.part[0 * gridDim.x + blockIdx.x] = rz;
        a.part[1 * gridDim.x + blockIdx.x] = rr;
    }
    if (!grid_barrier(a.arrive, bi++, a.wait_ns, 0)) goto timeout;
    {
        rz = grid_total(a.part, 0, sh);
        rr = grid_total(a.part, 1, sh);
        // stop once |r| <= tol |r_0|: the warm start's residual is what the
        // solve has to remove (|b| holds K U_i, which can dwarf it)
        const double rr0 = rr, thr = a.tol * a.tol * rr0;
        const long long na = *a.acount;  // the model's vertices
        // three lanes per vertex: lane 3 g + pl of a warp's first 30 serves
        // vertex slot g, with the neighbours of plane dz = pl - 1 in the
        // product and component pl in the updates; slot s of round rep is
        // list entry blockIdx + gridDim (s + slots rep), so that every CTA
        // gets the same share
        const int lane = threadIdx.x & 31, grp = lane / 3, pl = lane - 3 * (lane / 3), base = 3 * grp;
        const long long wslot0 = 10LL * (threadIdx.x >> 5), slots = 10LL * (blockDim.x >> 5);
        double rz_prev = 1.0;
        int it = 0;
        bool broke = false;
        while (rr > thr && it < a.max_iter) {
            const double beta = it == 0 ? 0.0 : rz / rz_prev;
            const double *pold = (it & 1) ? a.p1 : a.p0;
            double *pcur = (it & 1) ? a.p0 : a.p1;
            // p = z + beta p_old is formed where it is read
            auto getp = [&](long long nb, double(&v)[3]) {
#pragma unroll
                for (int c = 0; c < 3; ++c) v[c] = fma(beta, __ldcg(pold + 3 * nb + c), __ldcg(a.z + 3 * nb + c));
            };
            double pq = 0.0;
            for (long long rep = 0;; ++rep) {
                const long long qw = blockIdx.x + (long long)gridDim.x * (wslot0 + slots * rep);
                if (qw >= na) break;  // the warp's first slot holds its smallest entry
                const long long q = qw + (long long)gridDim.x * grp;
                const bool act = grp < 10 && q < na;
                double y[3] = {0.0, 0.0, 0.0};
                long long n = 0;
                if (act) {
                    n = a.alist[q];
                    const int i = (int)(n % G.Nx), j = (int)((n / G.Nx) % G.Ny), k = (int)(n / ((long long)G.Nx * G.Ny));
                    const unsigned em = elem_mask(G, a.eact, i, j, k);
                    apply_A_plane(G, s_st, s_ke, a.m + 27 * n, em, i, j, k, pl, getp, y);
                }
                double tot[3];
#pragma unroll
                for (int c = 0; c < 3; ++c) {
                    const double t0 = __shfl_sync(0xffffffffu, y[c], base), t1 = __shfl_sync(0xffffffffu, y[c], base + 1),
                                 t2 = __shfl_sync(0xffffffffu, y[c], base + 2);
                    tot[c] = (t0 + t1) + t2;
                }
                if (act) {
                    const double yc = pl == 0 ? tot[0] : (pl == 1 ? tot[1] : tot[2]);
                    const double pn = fma(beta, __ldcg(pold + 3 * n + pl), __ldcg(a.z + 3 * n + pl));
                    pcur[3 * n + pl] = pn;
                    a.q[3 * n + pl] = yc;
                    pq += pn * yc;
                }
            }
            pq = cta_sum(pq, sh);
            if (threadIdx.x == 0) a.part[3 * gridDim.x + blockIdx.x] = pq;
            if (!grid_barrier(a.arrive, bi++, a.wait_ns, 0)) goto timeout;
            pq = grid_total(a.part, 3, sh);
            if (!(pq > 0.0)) {  // not positive definite on this vector: stop
                broke = true;
                break;
            }
            const double alpha = rz / pq;
            double rz_l = 0.0, rr_l = 0.0;
            for (long long rep = 0;; ++rep) {
                const long long qw = blockIdx.x + (long long)gridDim.x * (wslot0 + slots * rep);
                if (qw >= na) break;
                const long long q = qw + (long long)gridDim.x * grp;
                const bool act = grp < 10 && q < na;
                double rp = 0.0;
                long long n = 0;
                if (act) {
                    n = a.alist[q];
                    a.x[3 * n + pl] = fma(alpha, pcur[3 * n + pl], a.x[3 * n + pl]);
                    rp = fma(-alpha, a.q[3 * n + pl], a.r[3 * n + pl]);
                    a.r[3 * n + pl] = rp;
                    rr_l += rp * rp;
                }
                const double r0 = __shfl_sync(0xffffffffu, rp, base), r1 = __shfl_sync(0xffffffffu, rp, base + 1),
                             r2 = __shfl_sync(0xffffffffu, rp, base + 2);
                if (act) {
                    const double *Bi = a.binv + 9 * n + 3 * pl;
                    const double zp = Bi[0] * r0 + Bi[1] * r1 + Bi[2] * r2;
                    a.z[3 * n + pl] = zp;
                    rz_l += rp * zp;
                }
            }
            rz_l = cta_sum(rz_l, sh);
            rr_l = cta_sum(rr_l, sh);
            if (threadIdx.x == 0) {
                a.part[0 * gridDim.x + blockIdx.x] = rz_l;
                a.part[1 * gridDim.x + blockIdx.x] = rr_l;
            }
            if (!grid_barrier(a.arrive, bi++, a.wait_ns, 0)) goto timeout;
            rz_prev = rz;
            rz = grid_total(a.part, 0, sh);
            rr = grid_total(a.part, 1, sh);
            ++it;
        }
        if (blockIdx.x == 0 && threadIdx.x == 0) {
            *a.iters = broke ? -2 : it;
            *a.relres = rr0 > 0.0 ? sqrt(rr / rr0) : 0.0;
        }
        return;
    }
timeout:
    if (threadIdx.x == 0) {
        atomicOr(a.err, DEV_ERR_TIMEOUT);
        *a.iters = -1;
    }
}

// ---- rejection --------------------------------------------------------------

// Squared residual |D_k - H_k U|^2 of every trusted block as a 64-bit key
// whose unsigned order is the order of the residuals (the bits of a
// non-negative double); 0 for untrusted blocks and residuals at or below
// R2_MIN.  counts[0] = trusted blocks, counts[1] = nonzero keys.
__global__ void fem_residuals_kernel(FemGrid G, const int32_t *__restrict__ centers, const int32_t *__restrict__ disp,
                                     const double *__restrict__ s, int n, const double *__restrict__ U,
                                     unsigned long long *__restrict__ keys, unsigned long long *__restrict__ counts)
{
    unsigned long long ntr = 0, npos = 0;
    for (int b = blockIdx.x * blockDim.x + threadIdx.x; b < n; b += gridDim.x * blockDim.x) {
        unsigned long long key = 0;
        if (s[b] > 0.0) {
            ++ntr;
            int i, j, k;
            double w[8];
            block_weights(G, centers[3 * b], centers[3 * b + 1], centers[3 * b + 2], i, j, k, w);
            double hu[3] = {0.0, 0.0, 0.0};
#pragma unroll
            for (int a = 0; a < 8; ++a) {
                const long long na = vidx(G, i + (a & 1), j + ((a >> 1) & 1), k + ((a >> 2) & 1));
#pragma unroll
                for (int c = 0; c < 3; ++c) hu[c] = __dadd_rn(hu[c], __dmul_rn(w[a], U[3 * na + c]));
            }
            double r2 = 0.0;
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                const double d = __dsub_rn((double)disp[3 * b + c], hu[c]);
                r2 = __dadd_rn(r2, __dmul_rn(d, d));
            }
            if (r2 > R2_MIN) {
                key = (unsigned long long)__double_as_longlong(r2);
                ++npos;
            }
        }
        keys[b] = key;
    }
    for (int o = 16; o; o >>= 1) {
        ntr += __shfl_xor_sync(0xffffffffu, ntr, o);
        npos += __shfl_xor_sync(0xffffffffu, npos, o);
    }
    if ((threadIdx.x & 31) == 0 && (ntr || npos)) {
        atomicAdd(counts, ntr);
        atomicAdd(counts + 1, npos);
    }
}

// One CTA: n_rej = min(floor(0.5 + F_r n_trusted), nonzero keys); find the
// n_rej-th largest key K* by eight 8-bit radix passes, then reject every key
// above K* and the first keys equal to K* in block order, up to n_rej.
__global__ void __launch_bounds__(REJ_THREADS) fem_reject_kernel(const unsigned long long *__restrict__ keys, int n,
                                                                 const unsigned long long *__restrict__ counts,
                                                                 double fr, int stepno, double *__restrict__ s,
                                                                 int32_t *__restrict__ step)
{
    __shared__ unsigned int hist[256];
    __shared__ unsigned long long s_prefix;
    __shared__ long long s_rem;
    __shared__ int s_before[REJ_THREADS];
    const int tid = threadIdx.x, T = blockDim.x;
    long long want = (long long)floor(__dadd_rn(0.5, __dmul_rn((double)counts[0], fr)));
    if (want > (long long)counts[1]) want = (long long)counts[1];
    if (want <= 0) return;
    unsigned long long prefix = 0, mask = 0;
    long long rem = want;  // rank still to find among the keys matching the prefix
    for (int sh = 56; sh >= 0; sh -= 8) {
        for (int q = tid; q < 256; q += T) hist[q] = 0;
        __syncthreads();
        for (int b = tid; b < n; b += T) {
            const unsigned long long key = keys[b];
            if ((key & mask) == prefix) atomicAdd(&hist[(key >> sh) & 255u], 1u);
        }
        __syncthreads();
        if (tid == 0) {
            long long cum = 0;
            for (int d = 255; d >= 0; --d) {
                if (cum + (long long)hist[d] >= rem) {
                    prefix |= (unsigned long long)d << sh;
                    rem -= cum;
                    break;
                }
                cum += hist[d];
            }
            s_prefix = prefix;
            s_rem = rem;
        }
        __syncthreads();
        prefix = s_prefix;
        rem = s_rem;
        mask |= 0xFFull << sh;
    }
    // K* = prefix; `rem` keys equal to it are taken, in block order
    const int chunk = (n + T - 1) / T, lo = tid * chunk, hi = min(lo + chunk, n);
    int eq = 0;
    for (int b = lo; b < hi; ++b) eq += keys[b] == prefix;
    s_before[tid] = eq;
    __syncthreads();
    if (tid == 0) {
        int acc = 0;
        for (int q = 0; q < T; ++q) {
            const int v = s_before[q];
            s_before[q] = acc;
            acc += v;
        }
    }
    __syncthreads();
    long long before = s_before[tid];
    for (int b = lo; b < hi; ++b) {
        const unsigned long long key = keys[b];
        bool out = key > prefix;
        if (key == prefix) out = before++ < rem;
        if (out) {
            s[b] = 0.0;
            step[b] = stepno;
        }
    }
}

// ---- host ---------------------------------------------------------------------

// 24x24 stiffness of a cube element of edge g (local node a = ax + 2 ay + 4 az
// at corner (ax, ay, az) g, dof 3 a + c): the integral of B^T C B over the
// element by the 2x2x2 Gauss rule, C the isotropic stress-strain matrix of
// (E, nu) in Voigt order (xx, yy, zz, xy, yz, zx) with engineering shears.
void element_stiffness(double g, double E, double nu, double *K)
{
    const double lam = E * nu / ((1.0 + nu) * (1.0 - 2.0 * nu)), mu = E / (2.0 * (1.0 + nu));
    double C[6][6] = {};
    for (int p = 0; p < 3; ++p) {
        for (int q = 0; q < 3; ++q) C[p][q] = lam;
        C[p][p] = lam + 2.0 * mu;
        C[3 + p][3 + p] = mu;
    }
    for (int e = 0; e < 576; ++e) K[e] = 0.0;
    const double gp = 1.0 / sqrt(3.0), jac = (g / 2.0) * (g / 2.0) * (g / 2.0);
    for (int qp = 0; qp < 8; ++qp) {
        const double xi[3] = {(qp & 1) ? gp : -gp, (qp & 2) ? gp : -gp, (qp & 4) ? gp : -gp};
        double Bm[6][24] = {};
        for (int a = 0; a < 8; ++a) {
            const double sg[3] = {(a & 1) ? 1.0 : -1.0, (a & 2) ? 1.0 : -1.0, (a & 4) ? 1.0 : -1.0};
            double grad[3];
            for (int d = 0; d < 3; ++d) {
                double v = sg[d] * 0.5 * (2.0 / g);
                for (int o = 0; o < 3; ++o)
                    if (o != d) v *= 0.5 * (1.0 + sg[o] * xi[o]);
                grad[d] = v;
            }
            Bm[0][3 * a] = grad[0];
            Bm[1][3 * a + 1] = grad[1];
            Bm[2][3 * a + 2] = grad[2];
            Bm[3][3 * a] = grad[1];
            Bm[3][3 * a + 1] = grad[0];
            Bm[4][3 * a + 1] = grad[2];
            Bm[4][3 * a + 2] = grad[1];
            Bm[5][3 * a] = grad[2];
            Bm[5][3 * a + 2] = grad[0];
        }
        double CB[6][24];
        for (int p = 0; p < 6; ++p)
            for (int col = 0; col < 24; ++col) {
                double v = 0.0;
                for (int q = 0; q < 6; ++q) v += C[p][q] * Bm[q][col];
                CB[p][col] = v;
            }
        for (int row = 0; row < 24; ++row)
            for (int col = 0; col < 24; ++col) {
                double v = 0.0;
                for (int p = 0; p < 6; ++p) v += Bm[p][row] * CB[p][col];
                K[row * 24 + col] += v * jac;
            }
    }
}

// The stiffness stencil of a vertex with all 8 elements in the model: the
// block coupling it (local node a of the element at offset -a) to neighbour
// o = (dx, dy, dz), summed over the elements holding both.
void interior_stencil(const double *K, double *st)
{
    for (int o = 0; o < 27; ++o) {
        const int dx = o % 3 - 1, dy = (o / 3) % 3 - 1, dz = o / 9 - 1;
        for (int e = 0; e < 9; ++e) st[o * 9 + e] = 0.0;
        for (int a = 0; a < 8; ++a) {
            const int bx = (a & 1) + dx, by = ((a >> 1) & 1) + dy, bz = ((a >> 2) & 1) + dz;
            if (bx < 0 || bx > 1 || by < 0 || by > 1 || bz < 0 || bz > 1) continue;
            const int b = bx + 2 * by + 4 * bz;
            for (int c = 0; c < 3; ++c)
                for (int d = 0; d < 3; ++d) st[o * 9 + 3 * c + d] += K[(3 * a + c) * 24 + 3 * b + d];
        }
    }
}

FemGrid make_grid(nrr_dims d, int g)
{
    FemGrid G;
    G.nx = d.nx;
    G.ny = d.ny;
    G.nz = d.nz;
    G.g = g;
    G.Nx = (d.nx - 1 + g - 1) / g + 1;
    G.Ny = (d.ny - 1 + g - 1) / g + 1;
    G.Nz = (d.nz - 1 + g - 1) / g + 1;
    G.Ex = G.Nx - 1;
    G.Ey = G.Ny - 1;
    G.Ez = G.Nz - 1;
    G.nv = (long long)G.Nx * G.Ny * G.Nz;
    return G;
}

int grid_for(long long items, int threads)
{
    long long b = (items + threads - 1) / threads, cap = 8LL * sm_count();
    if (b > cap) b = cap;
    return b < 1 ? 1 : (int)b;
}

}  // namespace
}  // namespace nrr

using namespace nrr;

extern "C" nrr_status nrr_fem_grid(nrr_dims dims, int32_t grid, int32_t n_vertices[3])
{
    clear_error();
    if (!n_vertices) return fail(NRR_E_INVALID, "n_vertices is NULL");
    if (grid < 2 || grid > 4096) return fail(NRR_E_INVALID, "grid spacing %d outside 2..4096", grid);
    if (dims.nx < 2 || dims.ny < 2 || dims.nz < 2) return fail(NRR_E_INVALID, "volume needs at least 2 voxels per axis");
    const FemGrid G = make_grid(dims, grid);
    n_vertices[0] = G.Nx;
    n_vertices[1] = G.Ny;
    n_vertices[2] = G.Nz;
    return NRR_OK;
}

extern "C" nrr_status nrr_fem_update(const uint8_t *d_mask, nrr_dims dims, const int32_t *d_centers,
                                     const int32_t *d_disp, const double *d_ncc, const uint8_t *d_valid,
                                     int32_t n_blocks, const nrr_fem_params *params, double *d_U, double *d_s,
                                     int32_t *d_rejected_step, int32_t *h_cg_iters, void *stream)
{
    clear_error();
    if (!params) return fail(NRR_E_INVALID, "params is NULL");
    const nrr_fem_params P = *params;
    if (P.grid < 2 || P.grid > 4096) return fail(NRR_E_INVALID, "grid spacing %d outside 2..4096", P.grid);
    if (!(P.young > 0.0) || !(P.poisson >= 0.0 && P.poisson < 0.5))
        return fail(NRR_E_INVALID, "material needs young > 0 and 0 <= poisson < 0.5");
    if (P.n_rej < 0 || P.n_int < 0 || P.n_rej > 1000 || P.n_int > 1000)
        return fail(NRR_E_INVALID, "n_rej and n_int must lie in 0..1000");
    if (!(P.reject_frac >= 0.0 && P.reject_frac <= 1.0)) return fail(NRR_E_INVALID, "reject_frac outside [0, 1]");
    if (!(P.cg_tol > 0.0) || P.cg_max_iter < 1) return fail(NRR_E_INVALID, "cg_tol must be > 0 and cg_max_iter >= 1");
    if (n_blocks < 0 || n_blocks > MAX_FEM_BLOCKS) return fail(NRR_E_INVALID, "n_blocks %d outside 0..%d", n_blocks, MAX_FEM_BLOCKS);
    if (dims.nx < 2 || dims.ny < 2 || dims.nz < 2) return fail(NRR_E_INVALID, "volume needs at least 2 voxels per axis");
    if (!d_mask || !d_U) return fail(NRR_E_INVALID, "d_mask and d_U must not be NULL");
    if (n_blocks > 0 && (!d_centers || !d_disp || !d_ncc || !d_valid || !d_s || !d_rejected_step))
        return fail(NRR_E_INVALID, "block arrays must not be NULL");
    const FemGrid G = make_grid(dims, P.grid);
    if (G.nv > (1LL << 31)) return fail(NRR_E_INVALID, "mesh of %lld vertices is too large", G.nv);
    cudaStream_t st = (cudaStream_t)stream;
    const int steps = P.n_rej + P.n_int;
    const size_t nv = (size_t)G.nv, ne = (size_t)G.Ex * G.Ey * G.Ez, nb = (size_t)(n_blocks > 0 ? n_blocks : 1);

    NRR_CUDA_TRY(cudaMemsetAsync(d_U, 0, nv * 3 * sizeof(double), st));
    if (steps == 0 && n_blocks == 0) return NRR_OK;

    auto kern = fem_solve_kernel;
    int occ = 0;
    NRR_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, SOLVE_THREADS, 0));
    if (occ < 1) return fail(NRR_E_INTERNAL, "solve kernel does not fit on an SM");
    // at most two CTAs per SM: the solve's time per iteration is its two grid
    // barriers plus an even share of the model's vertices per CTA
    // three lanes per vertex, 30 of each warp's 32 lanes in use
    long long cg_blocks = (3LL * (long long)nv + SOLVE_THREADS / 32 * 30 - 1) / (SOLVE_THREADS / 32 * 30);
    const long long cap_blocks = (long long)(occ < 2 ? occ : 2) * sm_count();
    if (cg_blocks > cap_blocks) cg_blocks = cap_blocks;
    if (cg_blocks < 1) cg_blocks = 1;

    // scratch, one allocation: offsets in bytes, each 256-aligned
    size_t off = 0;
    auto take = [&](size_t bytes) {
        const size_t o = off;
        off = align_up(off + bytes, 256);
        return o;
    };
    const size_t o_eact = take(ne), o_nact = take(nv), o_mfix = take(nv * 27 * 8), o_bfix = take(nv * 3 * 8),
                 o_m = take(nv * 27 * 8), o_binv = take(nv * 9 * 8), o_r = take(nv * 3 * 8), o_p0 = take(nv * 3 * 8),
                 o_p1 = take(nv * 3 * 8), o_q = take(nv * 3 * 8), o_part = take(4 * (size_t)cg_blocks * 8),
                 o_arr = take(8), o_keys = take(nb * 8), o_cnt = take(16), o_it = take((size_t)(steps + 1) * 4),
                 o_rel = take((size_t)(steps + 1) * 8), o_alist = take(nv * 4), o_acnt = take(4),
                 o_z = take(nv * 3 * 8);
    unsigned char *scr = nullptr;
    {
        const cudaError_t e = cudaMallocAsync((void **)&scr, off, st);
        if (e == cudaErrorMemoryAllocation) {
            cudaGetLastError();
            return fail(NRR_E_NOMEM, "no room for %zu bytes of finite-element scratch", off);
        }
        if (e != cudaSuccess) return cuda_fail(e, "cudaMallocAsync");
    }
    uint8_t *eact = scr + o_eact, *nact = scr + o_nact;
    unsigned long long *mfix = (unsigned long long *)(scr + o_mfix), *bfix = (unsigned long long *)(scr + o_bfix);
    unsigned long long *keys = (unsigned long long *)(scr + o_keys), *cnt = (unsigned long long *)(scr + o_cnt);
    int32_t *iters = (int32_t *)(scr + o_it);
    double *relres = (double *)(scr + o_rel);

    nrr_status rs = NRR_OK;
    auto run = [&]() -> nrr_status {
        unsigned int *err = nullptr;
        nrr_status s2 = device_error_word(&err);
        if (s2 != NRR_OK) return s2;
        fem_elements_kernel<<<grid_for((long long)ne, FEM_THREADS), FEM_THREADS, 0, st>>>(d_mask, G, eact);
        fem_nodes_kernel<<<grid_for((long long)nv, FEM_THREADS), FEM_THREADS, 0, st>>>(G, eact, nact);
        fem_active_list_kernel<<<1, REJ_THREADS, 0, st>>>(nact, (long long)nv, (int32_t *)(scr + o_alist),
                                                          (int32_t *)(scr + o_acnt));
        count_launches(3);
        if (n_blocks > 0) {
            fem_init_blocks_kernel<<<grid_for(n_blocks, FEM_THREADS), FEM_THREADS, 0, st>>>(G, eact, d_centers, d_ncc,
                                                                                         d_valid, n_blocks, d_s,
                                                                                         d_rejected_step);
            count_launches(1);
        }
        NRR_CUDA_TRY(cudaGetLastError());
        FemKe Ke;
        element_stiffness((double)P.grid, P.young, P.poisson, Ke.k);
        interior_stencil(Ke.k, Ke.st);
        FemSolveArgs A;
        A.G = G;
        A.eact = eact;
        A.nact = nact;
        A.mfix = mfix;
        A.bfix = bfix;
        A.m = (double *)(scr + o_m);
        A.binv = (double *)(scr + o_binv);
        A.x = d_U;
        A.r = (double *)(scr + o_r);
        A.p0 = (double *)(scr + o_p0);
        A.p1 = (double *)(scr + o_p1);
        A.q = (double *)(scr + o_q);
        A.z = (double *)(scr + o_z);
        A.part = (double *)(scr + o_part);
        A.alist = (const int32_t *)(scr + o_alist);
        A.acount = (const int32_t *)(scr + o_acnt);
        A.arrive = (unsigned int *)(scr + o_arr);
        A.tol = P.cg_tol;
        A.max_iter = P.cg_max_iter;
        A.err = err;
        A.wait_ns = device_wait_ns();
        for (int it = 0; it < steps; ++it) {
            NRR_CUDA_TRY(cudaMemsetAsync(mfix, 0, nv * 27 * 8, st));
            NRR_CUDA_TRY(cudaMemsetAsync(bfix, 0, nv * 3 * 8, st));
            NRR_CUDA_TRY(cudaMemsetAsync(A.arrive, 0, 8, st));
            if (n_blocks > 0) {
                fem_assemble_kernel<<<grid_for(n_blocks, FEM_THREADS), FEM_THREADS, 0, st>>>(G, d_centers, d_disp, d_s,
                                                                                          n_blocks, mfix, bfix);
                count_launches(1);
                NRR_CUDA_TRY(cudaGetLastError());
            }
            A.iters = iters + it;
            A.relres = relres + it;
            void *args[] = {(void *)&A, (void *)&Ke};
            NRR_CUDA_TRY(cudaLaunchCooperativeKernel((const void *)kern, dim3((unsigned)cg_blocks), dim3(SOLVE_THREADS),
                                                     args, 0, st));
            count_launches(1);
            if (it < P.n_rej && n_blocks > 0) {
                NRR_CUDA_TRY(cudaMemsetAsync(cnt, 0, 16, st));
                fem_residuals_kernel<<<grid_for(n_blocks, FEM_THREADS), FEM_THREADS, 0, st>>>(
                    G, d_centers, d_disp, d_s, n_blocks, d_U, keys, cnt);
                fem_reject_kernel<<<1, REJ_THREADS, 0, st>>>(keys, n_blocks, cnt, P.reject_frac, it, d_s,
                                                             d_rejected_step);
                count_launches(2);
                NRR_CUDA_TRY(cudaGetLastError());
            }
        }
        return NRR_OK;
    };
    rs = run();
    std::vector<int32_t> hi((size_t)steps + 1, 0);
    std::vector<double> hr((size_t)steps + 1, 0.0);
    if (rs == NRR_OK && steps > 0) {
        cudaError_t e = cudaMemcpyAsync(hi.data(), iters, (size_t)steps * 4, cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess) e = cudaMemcpyAsync(hr.data(), relres, (size_t)steps * 8, cudaMemcpyDeviceToHost, st);
        if (e != cudaSuccess) rs = cuda_fail(e, "cudaMemcpyAsync");
    }
    const cudaError_t ef = cudaFreeAsync(scr, st);
    if (rs == NRR_OK && ef != cudaSuccess) rs = cuda_fail(ef, "cudaFreeAsync");
    if (rs != NRR_OK) return rs;
    NRR_CUDA_TRY(cudaStreamSynchronize(st));
    for (int it = 0; it < steps; ++it) {
        if (h_cg_iters) h_cg_iters[it] = hi[it];
        if (hi[it] == -1) return fail(NRR_E_TIMEOUT, "a grid barrier of solve %d gave up", it);
        if (hi[it] == -2) return fail(NRR_E_INTERNAL, "solve %d met a direction of non-positive curvature", it);
        if (!(hr[it] <= P.cg_tol))
            return fail(NRR_E_INTERNAL, "solve %d stopped at relative residual %g after %d iterations (tolerance %g)", it,
                        hr[it], hi[it], P.cg_tol);
    }
    return NRR_OK;
}
