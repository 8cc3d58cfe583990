// Box sums of the reference volume for blocks with a different edge per axis
// (bx, by, bz): S_J = sum J and, for uint16, v_J = N S_JJ - S_J^2 (N =
// bx by bz, exact in 64-bit integers, rounded once to float), for float32
// the sums of J - c and (J - c)^2 in float (c the volume's centre value).  Same output layout as the cubic box kernel: the
// first array (int32 or float) at offset 0, the second (float) at
// boxsum_s2_offset.  Values are written where the whole block fits in the
// volume and are zero elsewhere (the match kernel reads only the former).
//
// Three separable passes over the volume (x, then y, then z), one thread per
// voxel, coalesced along x; the first two write their partial sums to a
// scratch buffer.  The summation along each axis is sequential, so a float32
// sum carries at most bx + by + bz roundings per term besides the rounding
// of J - c and of its square, the depth the match kernel's error bound
// assumes.
#include "nrr_internal.h"

namespace nrr {
namespace {

constexpr int P3_THREADS = 256;

// uint16: x pass from the volume (partial sums exact in 32 and 64 bits)
__global__ void __launch_bounds__(P3_THREADS) box3_u16_x(const uint16_t *__restrict__ vol, int nx, long long nvox,
                                                         int h, uint32_t *__restrict__ s, unsigned long long *__restrict__ q)
{
    for (long long v = (long long)blockIdx.x * blockDim.x + threadIdx.x; v < nvox; v += (long long)gridDim.x * blockDim.x) {
        const int x = (int)(v % nx);
        uint32_t a = 0;
        unsigned long long b = 0;
        if (x >= h && x <= nx - 1 - h)
            for (int k = -h; k <= h; ++k) {
                const uint32_t u = vol[v + k];
                a += u;
                b += (unsigned long long)(u * u);
            }
        s[v] = a;
        q[v] = b;
    }
}

// uint16: y or z pass over the previous partial sums (stride = nx or nx*ny);
// `fin` makes it the last pass, writing S_J and v_J
__global__ void __launch_bounds__(P3_THREADS) box3_u16_yz(const uint32_t *__restrict__ si,
                                                          const unsigned long long *__restrict__ qi, int n_axis,
                                                          long long stride, long long nvox, int h, int fin,
                                                          long long nblk, uint32_t *__restrict__ so,
                                                          unsigned long long *__restrict__ qo, int32_t *__restrict__ o1,
                                                          float *__restrict__ o2)
{
    for (long long v = (long long)blockIdx.x * blockDim.x + threadIdx.x; v < nvox; v += (long long)gridDim.x * blockDim.x) {
        const int c = (int)((v / stride) % n_axis);
        uint32_t a = 0;
        unsigned long long b = 0;
        if (c >= h && c <= n_axis - 1 - h)
            for (int k = -h; k <= h; ++k) {
                a += si[v + k * stride];
                b += qi[v + k * stride];
            }
        if (fin) {
            o1[v] = (int32_t)a;
            o2[v] = __ll2float_rn(nblk * (long long)b - (long long)a * (long long)a);
        } else {
            so[v] = a;
            qo[v] = b;
        }
    }
}

// float32: x pass from the volume
__global__ void __launch_bounds__(P3_THREADS) box3_f32_x(const float *__restrict__ vol, int nx, long long nvox, int h,
                                                         const float *__restrict__ centre, float *__restrict__ s,
                                                         float *__restrict__ q)
{
    const float c = *centre;  // the sums are of J - c
    for (long long v = (long long)blockIdx.x * blockDim.x + threadIdx.x; v < nvox; v += (long long)gridDim.x * blockDim.x) {
        const int x = (int)(v % nx);
        float a = 0.f, b = 0.f;
        if (x >= h && x <= nx - 1 - h)
            for (int k = -h; k <= h; ++k) {
                const float u = __fsub_rn(vol[v + k], c);
                a = __fadd_rn(a, u);
                b = __fadd_rn(b, __fmul_rn(u, u));
            }
        s[v] = a;
        q[v] = b;
    }
}

// float32: y or z pass; the last pass writes S_J and S_JJ
__global__ void __launch_bounds__(P3_THREADS) box3_f32_yz(const float *__restrict__ si, const float *__restrict__ qi,
                                                          int n_axis, long long stride, long long nvox, int h,
                                                          float *__restrict__ so, float *__restrict__ qo)
{
    for (long long v = (long long)blockIdx.x * blockDim.x + threadIdx.x; v < nvox; v += (long long)gridDim.x * blockDim.x) {
        const int c = (int)((v / stride) % n_axis);
        float a = 0.f, b = 0.f;
        if (c >= h && c <= n_axis - 1 - h)
            for (int k = -h; k <= h; ++k) {
                a = __fadd_rn(a, si[v + k * stride]);
                b = __fadd_rn(b, qi[v + k * stride]);
            }
        so[v] = a;
        qo[v] = b;
    }
}

}  // namespace

size_t boxsum3_scratch_bytes(nrr_dims dims, nrr_dtype dtype)
{
    const size_t v = (size_t)dims.nx * dims.ny * dims.nz;
    const size_t per = dtype == NRR_F32 ? 8 : 12;  // partial S and Q of one pass
    return 2 * align_up(v * per, 256);
}

nrr_status launch_boxsums3(const void *d_intraop, nrr_dtype dtype, nrr_dims dims, const int32_t block[3],
                           void *d_boxsums, void *d_scratch, cudaStream_t stream)
{
    const long long nvox = (long long)dims.nx * dims.ny * dims.nz;
    const size_t half = boxsum3_scratch_bytes(dims, dtype) / 2;
    unsigned char *A = (unsigned char *)d_scratch, *Bf = A + half;
    const int hx = (block[0] - 1) / 2, hy = (block[1] - 1) / 2, hz = (block[2] - 1) / 2;
    const long long sy = dims.nx, sz = (long long)dims.nx * dims.ny;
    long long grid = (nvox + P3_THREADS - 1) / P3_THREADS;
    if (grid > 32LL * sm_count()) grid = 32LL * sm_count();
    if (grid < 1) grid = 1;
    const unsigned g = (unsigned)grid;
    void *o1 = d_boxsums, *o2 = (char *)d_boxsums + boxsum_s2_offset(dims, dtype);
    if (dtype == NRR_U16) {
        const size_t off_q = align_up((size_t)nvox * 4, 256);
        uint32_t *sa = (uint32_t *)A, *sb = (uint32_t *)Bf;
        unsigned long long *qa = (unsigned long long *)(A + off_q), *qb = (unsigned long long *)(Bf + off_q);
        const long long nblk = (long long)block[0] * block[1] * block[2];
        box3_u16_x<<<g, P3_THREADS, 0, stream>>>((const uint16_t *)d_intraop, dims.nx, nvox, hx, sa, qa);
        box3_u16_yz<<<g, P3_THREADS, 0, stream>>>(sa, qa, dims.ny, sy, nvox, hy, 0, nblk, sb, qb, nullptr, nullptr);
        box3_u16_yz<<<g, P3_THREADS, 0, stream>>>(sb, qb, dims.nz, sz, nvox, hz, 1, nblk, nullptr, nullptr,
                                                  (int32_t *)o1, (float *)o2);
    } else {
        const size_t off_q = align_up((size_t)nvox * 4, 256);
        float *sa = (float *)A, *sb = (float *)Bf, *qa = (float *)(A + off_q), *qb = (float *)(Bf + off_q);
        box3_f32_x<<<g, P3_THREADS, 0, stream>>>((const float *)d_intraop, dims.nx, nvox, hx,
                                                 (const float *)d_intraop +
                                                     volume_centre_index(dims.nx, dims.ny, dims.nz),
                                                 sa, qa);
        box3_f32_yz<<<g, P3_THREADS, 0, stream>>>(sa, qa, dims.ny, sy, nvox, hy, sb, qb);
        box3_f32_yz<<<g, P3_THREADS, 0, stream>>>(sb, qb, dims.nz, sz, nvox, hz, (float *)o1, (float *)o2);
    }
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "box-sum pass launch");
    count_launches(3);
    return NRR_OK;
}

}  // namespace nrr
