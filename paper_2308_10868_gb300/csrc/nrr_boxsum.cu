// Box sums of the reference image: the per-shift sums S_J = sum J and
// S_JJ = sum J^2 over the b^3 block at every voxel (Sec. 3, NCC equation:
// the mean and spread of the reference block change with every shift).
//
// Computed once per (volume, block size) instead of once per registration
// block: neighbouring blocks' search windows overlap heavily, so the match
// kernel reads these sums rather than re-deriving them from its window.
//
// One CTA owns a 32 x 8 column of outputs and streams through z: for every
// input plane it stages the (32+b-1) x (8+b-1) tile in shared memory, sums
// rows of b along x, then b row sums along y (the plane sum of that
// column), keeps the last b plane sums in registers and emits their sum.
// uint16: int32 / uint64 arithmetic, exact.  float32: float32 arithmetic
// with every output formed by three levels of b-term sums (the match
// kernel's error bound relies on that shape).
#include "nrr_internal.h"

namespace nrr {
namespace {

constexpr int TX = 32, TY = 8, ZCHUNK = 32;

template <typename T>
struct Acc;
template <>
struct Acc<uint16_t> {
    typedef int32_t A1;
    typedef unsigned long long A2;
    static __device__ __forceinline__ A1 v1(uint16_t v) { return (A1)v; }
    static __device__ __forceinline__ A2 v2(uint16_t v) { return (A2)((uint32_t)v * (uint32_t)v); }
};
template <>
struct Acc<float> {
    typedef float A1;
    typedef float A2;
    static __device__ __forceinline__ A1 v1(float v) { return v; }
    static __device__ __forceinline__ A2 v2(float v) { return __fmul_rn(v, v); }
};

template <typename T, int B>
__global__ void __launch_bounds__(TX *TY) boxsum_kernel(const T *__restrict__ vol, int nx, int ny, int nz,
                                                        typename Acc<T>::A1 *__restrict__ s1,
                                                        typename Acc<T>::A2 *__restrict__ s2)
{
    typedef typename Acc<T>::A1 A1;
    typedef typename Acc<T>::A2 A2;
    constexpr int H = (B - 1) / 2;
    constexpr int IW = TX + B - 1, IH = TY + B - 1;
    __shared__ T tile[IH][IW];
    __shared__ A1 r1[IH][TX];
    __shared__ A2 r2[IH][TX];

    const int tx = threadIdx.x % TX, ty = threadIdx.x / TX;
    const int x0 = blockIdx.x * TX, y0 = blockIdx.y * TY;
    const int zo0 = blockIdx.z * ZCHUNK, zo1 = min(nz, zo0 + ZCHUNK);
    const int x = x0 + tx, y = y0 + ty;
    const bool xy_ok = x < nx && y < ny;
    const bool xy_in = x >= H && x <= nx - 1 - H && y >= H && y <= ny - 1 - H;

    A1 ring1[B];
    A2 ring2[B];
#pragma unroll
    for (int i = 0; i < B; ++i) {
        ring1[i] = 0;
        ring2[i] = 0;
    }
    // input planes zo0-H .. zo1-1+H; output plane z-H emitted after plane z
    for (int z = zo0 - H; z < zo1 + H; ++z) {
        __syncthreads();
        for (int i = threadIdx.x; i < IH * IW; i += TX * TY) {
            int iy = i / IW, ix = i % IW;
            int gx = x0 - H + ix, gy = y0 - H + iy;
            T v = 0;
            if (z >= 0 && z < nz && gx >= 0 && gx < nx && gy >= 0 && gy < ny)
                v = vol[((size_t)z * ny + gy) * nx + gx];
            tile[iy][ix] = v;
        }
        __syncthreads();
        for (int i = threadIdx.x; i < IH * TX; i += TX * TY) {
            int iy = i / TX, ix = i % TX;
            A1 a = 0;
            A2 q = 0;
#pragma unroll
            for (int k = 0; k < B; ++k) {
                T v = tile[iy][ix + k];
                a += Acc<T>::v1(v);
                q += Acc<T>::v2(v);
            }
            r1[iy][ix] = a;
            r2[iy][ix] = q;
        }
        __syncthreads();
        A1 p1 = 0;
        A2 p2 = 0;
#pragma unroll
        for (int k = 0; k < B; ++k) {
            p1 += r1[ty + k][tx];
            p2 += r2[ty + k][tx];
        }
#pragma unroll
        for (int i = 0; i < B - 1; ++i) {
            ring1[i] = ring1[i + 1];
            ring2[i] = ring2[i + 1];
        }
        ring1[B - 1] = p1;
        ring2[B - 1] = p2;
        const int zo = z - H;  // output plane whose block spans planes zo-H..zo+H == z-2H..z
        if (zo >= zo0 && zo < zo1 && xy_ok) {
            A1 o1 = 0;
            A2 o2 = 0;
            if (xy_in && zo >= H && zo <= nz - 1 - H) {
#pragma unroll
                for (int i = 0; i < B; ++i) {
                    o1 += ring1[i];
                    o2 += ring2[i];
                }
            }
            size_t idx = ((size_t)zo * ny + y) * nx + x;
            s1[idx] = o1;
            s2[idx] = o2;
        }
    }
}

template <typename T, int B>
void launch_one(const void *vol, nrr_dims d, void *bs, size_t off2, cudaStream_t st)
{
    typedef typename Acc<T>::A1 A1;
    typedef typename Acc<T>::A2 A2;
    dim3 grid((d.nx + TX - 1) / TX, (d.ny + TY - 1) / TY, (d.nz + ZCHUNK - 1) / ZCHUNK);
    boxsum_kernel<T, B><<<grid, TX * TY, 0, st>>>((const T *)vol, d.nx, d.ny, d.nz, (A1 *)bs,
                                                  (A2 *)((char *)bs + off2));
}

template <typename T>
void launch_t(const void *vol, nrr_dims d, int b, void *bs, size_t off2, cudaStream_t st)
{
    switch (b) {
    case 3: launch_one<T, 3>(vol, d, bs, off2, st); break;
    case 5: launch_one<T, 5>(vol, d, bs, off2, st); break;
    case 7: launch_one<T, 7>(vol, d, bs, off2, st); break;
    case 9: launch_one<T, 9>(vol, d, bs, off2, st); break;
    default: launch_one<T, 11>(vol, d, bs, off2, st); break;
    }
}

}  // namespace

nrr_status launch_boxsums(const void *d_intraop, nrr_dtype dtype, nrr_dims dims, int32_t block, void *d_boxsums,
                          cudaStream_t stream)
{
    size_t off2 = boxsum_s2_offset(dims, dtype);
    if (dtype == NRR_F32)
        launch_t<float>(d_intraop, dims, block, d_boxsums, off2, stream);
    else
        launch_t<uint16_t>(d_intraop, dims, block, d_boxsums, off2, stream);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "boxsum kernel launch");
    count_launches(1);
    return NRR_OK;
}

}  // namespace nrr
