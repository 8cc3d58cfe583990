// Sums over b^3 blocks, for both steps of the path:
//  * matching (Sec. 3, NCC equation): S_J = sum J of the reference block at
//    every voxel and its spread, from S_JJ = sum J^2 -- the reference block's
//    mean and spread change with every shift -- computed once per (volume,
//    block size) because neighbouring blocks' search windows overlap heavily;
//  * selection (Sec. 4.1, "Parallel feature selection"): the variance key
//    N*sum I^2 - (sum I)^2 of the floating block at every stride grid point
//    whose centre lies in the mask and whose block lies in the volume.
//
// Both are separable box sums.  One CTA owns TX x TY x ZC outputs (spaced
// `stride` voxels apart; stride 1 for matching).  Its input brick, with the
// b-1 halo, is brought into shared memory by TMA in z-chunks of CZ planes,
// each completing its own mbarrier, so the first planes are summed while the
// later ones are still in flight.  Per phase of PP input planes: sums of b
// along x at the output columns, for every row of those planes, a few
// outputs per thread so that the whole CTA shares the work
// (double-buffered, so one barrier per phase suffices); then sums of b of
// those along y at the output rows, one thread per output column; the last
// b plane sums stay in registers and at every output plane their sum is the
// result.
//   uint16: exact (32-bit sums of J, 64-bit sums of J^2, running z sums);
//           stored as S_J (int32) and v_J = N*S_JJ - S_J^2 rounded once to
//           float (the match kernel's filter needs only an approximation
//           of v_J, and its exact rescoring recomputes the sums).
//   float32: float sums of J - c (c the volume's centre value; the
//            difference rounded once) whose every output is three levels
//            of b-term sums; the match kernel's error bound relies on that
//            shape.
#include <stddef.h>

#include "nrr_internal.h"
#include "nrr_ptx.cuh"

namespace nrr {
namespace {

constexpr int TX = 32, MAX_TY = 8, MAX_NT = TX * MAX_TY;
constexpr int CZ = 4;          // planes per TMA chunk
constexpr int PP = 2;          // planes per phase (x sums of PP planes, one barrier, their y sums); divides CZ
constexpr int MAX_CHUNKS = 8;  // so at most 32 input planes per CTA
constexpr uint64_t BOX_WAIT_NS = 2000000000ull;
constexpr size_t BOX_SMEM_TARGET = 112 * 1024;  // keeps two CTAs per SM

// Per-element quantities summed: uint16 -> J (32-bit) and J^2 (64-bit,
// exact); float32 -> J and J^2 in float.
template <typename T>
struct BoxQ;
template <>
struct BoxQ<uint16_t> {
    typedef uint32_t A1;
    typedef unsigned long long A2;
    static constexpr bool exact = true;
};
template <>
struct BoxQ<float> {
    typedef float A1;
    typedef float A2;
    static constexpr bool exact = false;
};

// Geometry of one CTA's brick; the same on host and device.
struct BoxGeom {
    int S, TY, ZC;         // output spacing, output rows and planes per CTA
    int xoff;              // x of the brick's first needed voxel inside the TMA box
    int bw, ih, iz;        // TMA box width (x), rows, input planes
    int nchunk;            // TMA chunks of CZ planes
    size_t chunk_pitch;    // bytes between chunks (128-byte multiple)
    size_t r_off;          // byte offset of the x-sum buffers
    size_t smem;           // dynamic shared memory
};

__host__ __device__ inline BoxGeom box_geom(int B, int S, int TY, int ZC, int es)
{
    BoxGeom g;
    const int H = (B - 1) / 2, A = 16 / es;  // TMA x coordinates are multiples of A elements
    g.S = S;
    g.TY = TY;
    g.ZC = ZC;
    g.xoff = (A - H % A) % A;
    const int iw = (TX - 1) * S + B;
    g.bw = (g.xoff + iw + A - 1) / A * A;
    g.ih = (TY - 1) * S + B;
    g.iz = (ZC - 1) * S + B;
    g.nchunk = (g.iz + CZ - 1) / CZ;
    g.chunk_pitch = ((size_t)g.bw * g.ih * CZ * es + 127) / 128 * 128;
    g.r_off = g.chunk_pitch * g.nchunk;
    const size_t a12 = es == 2 ? 12 : 8;  // bytes of (A1, A2) per x sum
    g.smem = g.r_off + 2 * PP * (size_t)g.ih * TX * a12;
    return g;
}

struct BoxArgs {
    BoxGeom g;
    int nx, ny, nz;
    int gx, gy, gz;  // outputs per axis (grid points for keys, voxels for box sums)
    // box sums
    void *out1, *out2;
    const float *centre;  // float32: the volume's centre voxel, c of the sums of J - c
    // keys
    const uint8_t *mask;
    long long *keys;
    unsigned long long *nc, *npos, *maxkey;
    unsigned int *err;
};

// Resident CTAs per SM to keep registers for, without spills (the keys
// epilogue's stride-spaced brick allows only two by shared memory).
template <int B, bool KEYS>
struct BoxMinBlocks {
    static constexpr int value = KEYS ? 2 : B <= 3 ? 6 : B <= 5 ? 5 : B <= 7 ? 4 : B <= 9 ? 3 : 2;
};

template <typename T, int B, bool KEYS, int S>
__global__ void __launch_bounds__(MAX_NT, (BoxMinBlocks<B, KEYS>::value)) box_kernel(const __grid_constant__ CUtensorMap map, const BoxArgs a)
{
    typedef typename BoxQ<T>::A1 A1;
    typedef typename BoxQ<T>::A2 A2;
    constexpr int H = (B - 1) / 2;
    constexpr long long N = (long long)B * B * B;
    extern __shared__ __align__(128) unsigned char smem[];
    __shared__ __align__(8) uint64_t bar[MAX_CHUNKS];
    const BoxGeom &g = a.g;
    const int IH = g.ih, IZ = g.iz, BW = g.bw, NT = TX * g.TY;
    A2 *rb2 = reinterpret_cast<A2 *>(smem + g.r_off);                                   // [2][PP][IH][TX]
    A1 *rb1 = reinterpret_cast<A1 *>(smem + g.r_off + 2 * PP * sizeof(A2) * IH * TX);  // [2][PP][IH][TX]

    const int tid = threadIdx.x, tx = tid % TX, ty = tid / TX;
    const int i0 = blockIdx.x * TX, j0 = blockIdx.y * g.TY, k0 = blockIdx.z * g.ZC;
    if (tid == 0) {
        for (int c = 0; c < g.nchunk; ++c) mbar_init(bar + c, 1);
        fence_mbar_init();
    }
    __syncthreads();
    if (tid == 0) {
        const uint32_t bytes = (uint32_t)((size_t)BW * IH * CZ * sizeof(T));
        const int xa = i0 * S - H - g.xoff, ya = j0 * S - H, za = k0 * S - H;
        for (int c = 0; c < g.nchunk; ++c) {
            mbar_arrive_expect_tx(bar + c, bytes);
            tma_load_3d(smem + c * g.chunk_pitch, &map, bar + c, xa, ya, za + c * CZ);
        }
    }

    const int i = i0 + tx, j = j0 + ty;  // this thread's output column
    float cval = 0.f;  // float32: the sums are of J - c
    if constexpr (!BoxQ<T>::exact) cval = *a.centre;
    A1 ring1[B];
    A2 ring2[B];
    A1 run1 = 0;  // exact path: running sums of the ring
    A2 run2 = 0;
#pragma unroll
    for (int k = 0; k < B; ++k) {
        ring1[k] = 0;
        ring2[k] = 0;
    }
    int cand = 0, pos = 0;
    unsigned long long kmax = 0;
    // keys: this column's mask bits, fetched while the brick is in flight
    uint32_t mbits = 0;
    if constexpr (KEYS) {
        const int x = i * S, y = j * S;
        if (i < a.gx && j < a.gy && x >= H && x <= a.nx - 1 - H && y >= H && y <= a.ny - 1 - H) {
#pragma unroll
            for (int kk = 0; kk < 16; ++kk) {
                const int z = (k0 + kk) * S;
                if (kk < g.ZC && z >= H && z <= a.nz - 1 - H && a.mask[((size_t)z * a.ny + y) * a.nx + x] != 0)
                    mbits |= 1u << kk;
            }
        }
    }

    // planes in groups of 2B, PP at a time, so that ring slot (u mod B)
    // always holds the plane sums of the planes congruent to u modulo B
    // (static register indices)
    for (int iz0 = 0; iz0 < IZ; iz0 += 2 * B) {
#pragma unroll
    for (int u = 0; u < 2 * B; u += PP) {
        const int iz = iz0 + u;  // first plane of this phase
        if (iz >= IZ) break;
        if (iz % CZ == 0) {  // PP divides CZ: a phase's planes share a chunk
            const bool got = mbar_wait_bounded(bar + iz / CZ, 0, BOX_WAIT_NS);
            if (!__syncthreads_and(got)) {
                if (tid == 0) {
                    atomicOr(a.err, DEV_ERR_TIMEOUT);
                    for (int c = iz / CZ; c < g.nchunk; ++c)  // let copies in flight land before exiting
                        mbar_wait_bounded(bar + c, 0, BOX_WAIT_NS);
                }
                __syncthreads();
                return;
            }
        }
        const int set = (iz / PP) & 1;
        A1 *const r1s = rb1 + set * PP * IH * TX;
        A2 *const r2s = rb2 + set * PP * IH * TX;
        // x sums at the output columns of every row of planes iz .. iz+PP-1
        if constexpr (BoxQ<T>::exact) {
            // a thread slides along SEG consecutive outputs of a row: the next
            // sum adds the S entering values and drops the S leaving ones
            // (modular 32/64-bit arithmetic, exact since the true sums fit)
            constexpr int SEG = 4, NSEG = TX / SEG, NV = (SEG - 1) * S + B;
            for (int it = tid; it < PP * IH * NSEG; it += NT) {
                const int pl = it / (IH * NSEG), rem = it - pl * (IH * NSEG);
                const int seg = rem % NSEG, iy = rem / NSEG;
                if (iz + pl >= IZ) continue;
                const T *plane = reinterpret_cast<const T *>(smem + ((iz + pl) / CZ) * g.chunk_pitch) +
                                 ((iz + pl) % CZ) * IH * BW;
                const T *src = plane + iy * BW + g.xoff + seg * SEG * S;
                uint32_t v[NV], sq[NV];
#pragma unroll
                for (int k = 0; k < NV; ++k) {
                    v[k] = src[k];
                    sq[k] = v[k] * v[k];  // < 2^32
                }
                uint32_t a1 = 0, o1[SEG];
                unsigned long long a2 = 0, o2[SEG];
#pragma unroll
                for (int k = 0; k < B; ++k) {
                    a1 += v[k];
                    a2 += sq[k];
                }
                o1[0] = a1;
                o2[0] = a2;
#pragma unroll
                for (int i = 1; i < SEG; ++i) {
#pragma unroll
                    for (int k = 0; k < S; ++k) {
                        a1 += v[(i - 1) * S + B + k] - v[(i - 1) * S + k];
                        a2 += (unsigned long long)sq[(i - 1) * S + B + k] - sq[(i - 1) * S + k];
                    }
                    o1[i] = a1;
                    o2[i] = a2;
                }
                const int o = (pl * IH + iy) * TX + seg * SEG;
                *reinterpret_cast<uint4 *>(r1s + o) = make_uint4(o1[0], o1[1], o1[2], o1[3]);  // 16-byte aligned
                ulonglong2 *d2 = reinterpret_cast<ulonglong2 *>(r2s + o);
                d2[0] = make_ulonglong2(o2[0], o2[1]);
                d2[1] = make_ulonglong2(o2[2], o2[3]);
            }
        } else {  // float: every x sum a direct b-term sum (fixed depth)
            for (int it = tid; it < PP * IH * TX; it += NT) {
                const int pl = it / (IH * TX), rem = it - pl * (IH * TX);
                const int ox = rem % TX, iy = rem / TX;
                if (iz + pl >= IZ) continue;
                const T *plane = reinterpret_cast<const T *>(smem + ((iz + pl) / CZ) * g.chunk_pitch) +
                                 ((iz + pl) % CZ) * IH * BW;
                const T *src = plane + iy * BW + g.xoff + ox * S;
                A1 a1 = 0;
                A2 a2 = 0;
#pragma unroll
                for (int k = 0; k < B; ++k) {
                    const float v = __fsub_rn((float)src[k], cval);
                    a1 += v;
                    a2 += __fmul_rn(v, v);
                }
                r1s[(pl * IH + iy) * TX + ox] = a1;
                r2s[(pl * IH + iy) * TX + ox] = a2;
            }
        }
        __syncthreads();  // x sums of this phase ready (and the phase before last's buffers are free)
#pragma unroll
        for (int pl = 0; pl < PP; ++pl) {
            const int izp = iz + pl;
            if (izp >= IZ) break;
            const int slot = (u + pl) % B;
            const A1 *r1 = r1s + pl * IH * TX;
            const A2 *r2 = r2s + pl * IH * TX;
            A1 p1 = 0;
            A2 p2 = 0;
#pragma unroll
            for (int k = 0; k < B; ++k) {
                p1 += r1[(ty * S + k) * TX + tx];
                p2 += r2[(ty * S + k) * TX + tx];
            }
            if constexpr (BoxQ<T>::exact) {  // the slot held plane izp - B
                run1 += p1 - ring1[slot];
                run2 += p2 - ring2[slot];
            }
            ring1[slot] = p1;
            ring2[slot] = p2;
            // the ring now holds input planes izp-B+1..izp: an output plane
            // when they are the planes of local output kk
            const int q = izp - (B - 1);
            if (q < 0 || q % S) continue;
            const int kk = q / S, k = k0 + kk;
            if (kk >= g.ZC || k >= a.gz || i >= a.gx || j >= a.gy) continue;
            A1 o1;
            A2 o2;
            if constexpr (BoxQ<T>::exact) {
                o1 = run1;
                o2 = run2;
            } else {  // a direct sum of the b plane sums (fixed depth b)
                o1 = 0;
                o2 = 0;
#pragma unroll
                for (int t = 0; t < B; ++t) {
                    o1 += ring1[t];
                    o2 += ring2[t];
                }
            }
            const int x = i * S, y = j * S, z = k * S;
            const bool in = x >= H && x <= a.nx - 1 - H && y >= H && y <= a.ny - 1 - H && z >= H && z <= a.nz - 1 - H;
            if constexpr (KEYS) {
                long long key = -1;
                if (in && ((mbits >> kk) & 1u)) {
                    key = N * (long long)o2 - (long long)o1 * (long long)o1;
                    cand += 1;
                    pos += key > 0;
                    kmax = (unsigned long long)key > kmax ? (unsigned long long)key : kmax;
                }
                a.keys[((long long)k * a.gy + j) * a.gx + i] = key;
            } else {
                const size_t idx = ((size_t)z * a.ny + y) * a.nx + x;
                if constexpr (BoxQ<T>::exact) {
                    reinterpret_cast<int32_t *>(a.out1)[idx] = in ? (int32_t)o1 : 0;
                    // v_J = N*S_JJ - S_J^2 (exact in 64 bits), rounded once to float
                    reinterpret_cast<float *>(a.out2)[idx] =
                        in ? __ll2float_rn(N * (long long)o2 - (long long)o1 * (long long)o1) : 0.f;
                } else {
                    reinterpret_cast<float *>(a.out1)[idx] = in ? (float)o1 : 0.f;
                    reinterpret_cast<float *>(a.out2)[idx] = in ? (float)o2 : 0.f;
                }
            }
        }
    }
    }

    if constexpr (KEYS) {  // candidate counts and the largest key of this CTA
        __shared__ int ws[MAX_NT / 32][2];
        __shared__ unsigned long long wmax[MAX_NT / 32];
        for (int o = 16; o; o >>= 1) {
            cand += __shfl_xor_sync(0xffffffffu, cand, o);
            pos += __shfl_xor_sync(0xffffffffu, pos, o);
            const unsigned long long other = __shfl_xor_sync(0xffffffffu, kmax, o);
            kmax = other > kmax ? other : kmax;
        }
        if ((tid & 31) == 0) {
            ws[tid >> 5][0] = cand;
            ws[tid >> 5][1] = pos;
            wmax[tid >> 5] = kmax;
        }
        __syncthreads();
        if (tid == 0) {
            int c = 0, p = 0;
            unsigned long long mx = 0;
            for (int w = 0; w < NT / 32; ++w) {
                c += ws[w][0];
                p += ws[w][1];
                mx = wmax[w] > mx ? wmax[w] : mx;
            }
            if (c) atomicAdd(a.nc, (unsigned long long)c);
            if (p) atomicAdd(a.npos, (unsigned long long)p);
            if (mx) atomicMax(a.maxkey, mx);
        }
    }
}

// The largest CTA tile (TY in {8, 4}, then ZC in {16, 8, 4}) whose brick fits
// the shared-memory target and the chunk count; ok = false if none does.
inline bool pick_geom(int B, int S, int es, BoxGeom *out)
{
    for (int ty = MAX_TY; ty >= 4; ty /= 2)
        for (int zc = 16; zc >= 4; zc /= 2) {
            const BoxGeom g = box_geom(B, S, ty, zc, es);
            if (g.nchunk <= MAX_CHUNKS && g.bw <= 256 && g.ih <= 256 && g.smem <= BOX_SMEM_TARGET) {
                *out = g;
                return true;
            }
        }
    return false;
}

template <typename T, int B, bool KEYS, int S>
cudaError_t launch_box_s(const CUtensorMap &map, BoxArgs &a, cudaStream_t st)
{
    auto kern = box_kernel<T, B, KEYS, S>;
    static size_t attr = 0;  // largest dynamic shared memory opted in so far
    if (a.g.smem > attr) {
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)a.g.smem);
        if (e != cudaSuccess) return e;
        attr = a.g.smem;
    }
    dim3 grid((a.gx + TX - 1) / TX, (a.gy + a.g.TY - 1) / a.g.TY, (a.gz + a.g.ZC - 1) / a.g.ZC);
    kern<<<grid, TX * a.g.TY, a.g.smem, st>>>(map, a);
    return cudaGetLastError();
}

template <typename T, int B, bool KEYS>
cudaError_t launch_box(const CUtensorMap &map, BoxArgs &a, cudaStream_t st)
{
    if constexpr (!KEYS) {
        return launch_box_s<T, B, KEYS, 1>(map, a, st);
    } else {
        switch (a.g.S) {
        case 1: return launch_box_s<T, B, KEYS, 1>(map, a, st);
        case 2: return launch_box_s<T, B, KEYS, 2>(map, a, st);
        default: return launch_box_s<T, B, KEYS, 3>(map, a, st);
        }
    }
}

template <typename T, bool KEYS>
cudaError_t launch_box_b(int b, const CUtensorMap &map, BoxArgs &a, cudaStream_t st)
{
    switch (b) {
    case 3: return launch_box<T, 3, KEYS>(map, a, st);
    case 5: return launch_box<T, 5, KEYS>(map, a, st);
    case 7: return launch_box<T, 7, KEYS>(map, a, st);
    case 9: return launch_box<T, 9, KEYS>(map, a, st);
    default: return launch_box<T, 11, KEYS>(map, a, st);
    }
}

}  // namespace

nrr_status launch_boxsums(const void *d_intraop, nrr_dtype dtype, nrr_dims dims, int32_t block, void *d_boxsums,
                          cudaStream_t stream)
{
    const int es = (int)elem_size(dtype);
    BoxArgs a{};
    if (!pick_geom(block, 1, es, &a.g)) return fail(NRR_E_INTERNAL, "box-sum brick does not fit shared memory");
    a.nx = a.gx = dims.nx;
    a.ny = a.gy = dims.ny;
    a.nz = a.gz = dims.nz;
    a.out1 = d_boxsums;
    a.out2 = (char *)d_boxsums + boxsum_s2_offset(dims, dtype);
    a.centre = (const float *)d_intraop + volume_centre_index(dims.nx, dims.ny, dims.nz);
    nrr_status s = device_error_word(&a.err);
    if (s != NRR_OK) return s;
    CUtensorMap map;
    s = encode_volume_map(&map, d_intraop, dtype, dims, a.g.bw, a.g.ih, CZ);
    if (s != NRR_OK) return s;
    cudaError_t e = dtype == NRR_F32 ? launch_box_b<float, false>(block, map, a, stream)
                                     : launch_box_b<uint16_t, false>(block, map, a, stream);
    if (e != cudaSuccess) return cuda_fail(e, "boxsum kernel launch");
    count_launches(1);
    return NRR_OK;
}

bool keys_box_supported(int32_t block, int32_t stride)
{
    BoxGeom g;
    return stride <= 3 && pick_geom(block, stride, 2, &g);
}

nrr_status launch_keys_box(const uint16_t *d_preop, const uint8_t *d_mask, nrr_dims dims, int32_t block,
                           int32_t stride, int gx, int gy, int gz, long long *keys, unsigned long long *nc,
                           unsigned long long *npos, unsigned long long *maxkey, cudaStream_t stream)
{
    BoxArgs a{};
    if (stride > 3 || !pick_geom(block, stride, 2, &a.g))
        return fail(NRR_E_INTERNAL, "key brick does not fit shared memory");
    a.nx = dims.nx;
    a.ny = dims.ny;
    a.nz = dims.nz;
    a.gx = gx;
    a.gy = gy;
    a.gz = gz;
    a.mask = d_mask;
    a.keys = keys;
    a.nc = nc;
    a.npos = npos;
    a.maxkey = maxkey;
    nrr_status s = device_error_word(&a.err);
    if (s != NRR_OK) return s;
    CUtensorMap map;
    s = encode_volume_map(&map, d_preop, NRR_U16, dims, a.g.bw, a.g.ih, CZ);
    if (s != NRR_OK) return s;
    cudaError_t e = launch_box_b<uint16_t, true>(block, map, a, stream);
    if (e != cudaSuccess) return cuda_fail(e, "key kernel launch");
    return NRR_OK;
}

}  // namespace nrr
