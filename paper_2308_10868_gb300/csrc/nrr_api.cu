// Entry points of the C ABI (include/nrr.h) other than block selection:
// status strings, the device error word, tensor-map encoding, argument
// checks, box sums and block matching.
#include <stdarg.h>
#include <stdio.h>
#include <string.h>

#include <atomic>
#include <mutex>

#include "nrr_internal.h"

namespace nrr {

static thread_local char g_last_error[512];

void clear_error() { g_last_error[0] = 0; }

nrr_status fail(nrr_status s, const char *fmt, ...)
{
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_last_error, sizeof(g_last_error), fmt, ap);
    va_end(ap);
    return s;
}

nrr_status cuda_fail(cudaError_t e, const char *what)
{
    nrr_status s = (e == cudaErrorMemoryAllocation) ? NRR_E_NOMEM : NRR_E_CUDA;
    return fail(s, "%s: %s (%s)", what, cudaGetErrorName(e), cudaGetErrorString(e));
}

// One word per device; set by kernels, read and cleared by nrr_device_status.
static __device__ unsigned int g_device_error;

nrr_status device_error_word(unsigned int **ptr)
{
    static std::mutex mu;
    static unsigned int *addr[64] = {};
    int dev = 0;
    NRR_CUDA_TRY(cudaGetDevice(&dev));
    if (dev < 0 || dev >= 64) return fail(NRR_E_INTERNAL, "device ordinal %d out of range", dev);
    std::lock_guard<std::mutex> lk(mu);
    if (!addr[dev]) {
        void *p = nullptr;
        NRR_CUDA_TRY(cudaGetSymbolAddress(&p, g_device_error));
        addr[dev] = (unsigned int *)p;
    }
    *ptr = addr[dev];
    return NRR_OK;
}

// match work-queue heads, one 128-byte line each: the first half for
// eager launches, the second for launches captured into CUDA graphs
static __device__ int32_t g_match_queue[2 * MATCH_QUEUE_SLOTS * 32];

nrr_status match_queue_head(int32_t **ptr, bool captured)
{
    static std::mutex mu;
    static int32_t *addr[64] = {};
    static unsigned int next[64][2] = {};
    int dev = 0;
    NRR_CUDA_TRY(cudaGetDevice(&dev));
    if (dev < 0 || dev >= 64) return fail(NRR_E_INTERNAL, "device ordinal %d out of range", dev);
    std::lock_guard<std::mutex> lk(mu);
    if (!addr[dev]) {
        void *p = nullptr;
        NRR_CUDA_TRY(cudaGetSymbolAddress(&p, g_match_queue));
        addr[dev] = (int32_t *)p;
    }
    const int h = captured ? 1 : 0;
    *ptr = addr[dev] + 32 * ((size_t)h * MATCH_QUEUE_SLOTS + next[dev][h]++ % MATCH_QUEUE_SLOTS);
    return NRR_OK;
}

static std::atomic<long long> g_launches{0};
static std::atomic<unsigned long long> g_wait_ns{0};
static std::atomic<unsigned int> g_missing{0};

uint64_t device_wait_ns()
{
    const unsigned long long v = g_wait_ns.load(std::memory_order_relaxed);
    return v ? (uint64_t)v : DEVICE_WAIT_NS;
}
unsigned int test_missing_arrivals() { return g_missing.load(std::memory_order_relaxed); }

void count_launches(int n) { g_launches.fetch_add(n, std::memory_order_relaxed); }

int sm_count()
{
    static int cached[64] = {};
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return 148;
    if (!cached[dev]) {
        int n = 0;
        if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || n <= 0) n = 148;
        cached[dev] = n;
    }
    return cached[dev];
}

typedef CUresult (*EncodeTiledFn)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *, const cuuint64_t *,
                                  const cuuint64_t *, const cuuint32_t *, const cuuint32_t *, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

static EncodeTiledFn encode_fn(nrr_status *st)
{
    static std::once_flag once;
    static EncodeTiledFn fn = nullptr;
    static cudaError_t err = cudaSuccess;
    std::call_once(once, [] {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        err = cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q);
        if (err == cudaSuccess && q == cudaDriverEntryPointSuccess) fn = (EncodeTiledFn)p;
    });
    if (!fn) *st = fail(NRR_E_CUDA, "cuTensorMapEncodeTiled unavailable (%s)", cudaGetErrorName(err));
    return fn;
}

nrr_status encode_volume_map(CUtensorMap *map, const void *base, nrr_dtype dtype, nrr_dims dims, int bx, int by,
                             int bz)
{
    nrr_status st = NRR_OK;
    EncodeTiledFn fn = encode_fn(&st);
    if (!fn) return st;
    size_t es = elem_size(dtype);
    cuuint64_t gdim[3] = {(cuuint64_t)dims.nx, (cuuint64_t)dims.ny, (cuuint64_t)dims.nz};
    cuuint64_t gstride[2] = {(cuuint64_t)dims.nx * es, (cuuint64_t)dims.nx * dims.ny * es};
    cuuint32_t box[3] = {(cuuint32_t)bx, (cuuint32_t)by, (cuuint32_t)bz};
    cuuint32_t estr[3] = {1, 1, 1};
    CUresult r = fn(map, dtype == NRR_F32 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32 : CU_TENSOR_MAP_DATA_TYPE_UINT16, 3,
                    const_cast<void *>(base), gdim, gstride, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                    CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                    CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) return fail(NRR_E_CUDA, "cuTensorMapEncodeTiled failed (CUresult %d)", (int)r);
    return NRR_OK;
}

nrr_status check_dims(nrr_dims d, nrr_dtype dtype, int32_t block)
{
    if (dtype != NRR_U16 && dtype != NRR_F32) return fail(NRR_E_INVALID, "unknown dtype %d", (int)dtype);
    if (block < 3 || block > 11 || (block & 1) == 0)
        return fail(NRR_E_INVALID, "block must be odd and in 3..11 (got %d)", block);
    if (d.nx < block || d.ny < block || d.nz < block)
        return fail(NRR_E_INVALID, "volume %dx%dx%d smaller than block %d", d.nx, d.ny, d.nz, block);
    if ((int64_t)d.nx * d.ny * d.nz > ((int64_t)1 << 31) - 1)
        return fail(NRR_E_INVALID, "volume of %lld voxels exceeds 2^31-1", (long long)d.nx * d.ny * d.nz);
    if (((size_t)d.nx * elem_size(dtype)) % 16 != 0)
        return fail(NRR_E_INVALID, "nx*%zu bytes must be a multiple of 16 (nx=%d)", elem_size(dtype), d.nx);
    return NRR_OK;
}

nrr_status check_dims3(nrr_dims d, nrr_dtype dtype, const int32_t *block)
{
    if (!block) return fail(NRR_E_INVALID, "block is NULL");
    nrr_status st = check_dims(d, dtype, 3);  // dtype, size and pitch rules
    if (st != NRR_OK) return st;
    for (int i = 0; i < 3; ++i)
        if (block[i] < 3 || block[i] > 11 || (block[i] & 1) == 0)
            return fail(NRR_E_INVALID, "block[%d] must be odd and in 3..11 (got %d)", i, block[i]);
    if (d.nx < block[0] || d.ny < block[1] || d.nz < block[2])
        return fail(NRR_E_INVALID, "volume %dx%dx%d smaller than block %dx%dx%d", d.nx, d.ny, d.nz, block[0], block[1],
                    block[2]);
    return NRR_OK;
}

size_t boxsum_bytes(nrr_dims dims, nrr_dtype dtype)
{
    size_t v = (size_t)dims.nx * dims.ny * dims.nz;
    (void)dtype;
    return boxsum_s2_offset(dims, dtype) + align_up(v * 4, 256);  // second array: 4-byte elements
}

static bool aligned16(const void *p) { return ((uintptr_t)p & 15u) == 0; }

}  // namespace nrr

using namespace nrr;

extern "C" {

const char *nrr_status_string(nrr_status s)
{
    switch (s) {
    case NRR_OK: return "ok";
    case NRR_PENDING: return "pending";
    case NRR_E_INVALID: return "invalid argument";
    case NRR_E_NOMEM: return "out of device memory";
    case NRR_E_CUDA: return "CUDA error";
    case NRR_E_CAPACITY: return "capacity exceeded";
    case NRR_E_TIMEOUT: return "device wait timed out";
    case NRR_E_INTERNAL: return "internal error";
    case NRR_E_NOTFOUND: return "not found";
    }
    return "unknown status";
}

const char *nrr_last_error(void) { return g_last_error; }

int32_t nrr_version(void) { return 100; }

nrr_status nrr_test_set_wait(uint64_t limit_ns, int32_t missing_arrivals)
{
    clear_error();
    if (missing_arrivals < 0 || missing_arrivals > 1024) return fail(NRR_E_INVALID, "missing_arrivals outside 0..1024");
    if (limit_ns > 60000000000ull) return fail(NRR_E_INVALID, "limit_ns above 60 s");
    g_wait_ns.store(limit_ns, std::memory_order_relaxed);
    g_missing.store((unsigned int)missing_arrivals, std::memory_order_relaxed);
    return NRR_OK;
}

int64_t nrr_kernel_launches(void) { return nrr::g_launches.load(std::memory_order_relaxed); }

nrr_status nrr_device_status(void *stream)
{
    clear_error();
    unsigned int *w = nullptr;
    nrr_status st = device_error_word(&w);
    if (st != NRR_OK) return st;
    NRR_CUDA_TRY(cudaStreamSynchronize((cudaStream_t)stream));
    unsigned int v = 0;
    NRR_CUDA_TRY(cudaMemcpy(&v, w, sizeof(v), cudaMemcpyDeviceToHost));
    if (v) {
        unsigned int z = 0;
        NRR_CUDA_TRY(cudaMemcpy(w, &z, sizeof(z), cudaMemcpyHostToDevice));
        if (v & DEV_ERR_TIMEOUT) return fail(NRR_E_TIMEOUT, "a device-side wait gave up (error word 0x%x)", v);
        return fail(NRR_E_INTERNAL, "device-side check failed (error word 0x%x)", v);
    }
    return NRR_OK;
}

nrr_status nrr_boxsum_bytes(nrr_dims dims, nrr_dtype dtype, size_t *bytes)
{
    clear_error();
    if (!bytes) return fail(NRR_E_INVALID, "bytes is NULL");
    nrr_status st = check_dims(dims, dtype, 3);
    if (st != NRR_OK) return st;
    *bytes = boxsum_bytes(dims, dtype);
    return NRR_OK;
}

nrr_status nrr_boxsums(const void *d_intraop, nrr_dtype dtype, nrr_dims dims, int32_t block, void *d_boxsums,
                       void *stream)
{
    clear_error();
    nrr_status st = check_dims(dims, dtype, block);
    if (st != NRR_OK) return st;
    if (!d_intraop || !d_boxsums) return fail(NRR_E_INVALID, "NULL volume or box-sum buffer");
    if (((uintptr_t)d_boxsums & 255u) != 0) return fail(NRR_E_INVALID, "box-sum buffer must be 256-byte aligned");
    return launch_boxsums(d_intraop, dtype, dims, block, d_boxsums, (cudaStream_t)stream);
}

static nrr_status check_match_args(const void *d_preop, const void *d_intraop, nrr_dtype dtype, nrr_dims dims,
                                   const int32_t *d_centers, int32_t n_blocks, const int32_t *block3,
                                   const int32_t *radius, int32_t *d_disp, double *d_ncc, uint8_t *d_valid)
{
    nrr_status st = check_dims3(dims, dtype, block3);
    if (st != NRR_OK) return st;
    if (!radius) return fail(NRR_E_INVALID, "radius is NULL");
    for (int i = 0; i < 3; ++i)
        if (radius[i] < 0 || radius[i] > MATCH_MAX_R)
            return fail(NRR_E_INVALID, "radius[%d]=%d outside 0..%d", i, radius[i], MATCH_MAX_R);
    if (n_blocks < 0) return fail(NRR_E_INVALID, "n_blocks < 0");
    if (!d_preop || !d_intraop) return fail(NRR_E_INVALID, "NULL volume");
    if (!aligned16(d_preop) || !aligned16(d_intraop)) return fail(NRR_E_INVALID, "volumes must be 16-byte aligned");
    if (n_blocks > 0 && (!d_centers || !d_disp || !d_ncc || !d_valid))
        return fail(NRR_E_INVALID, "NULL centre or output buffer");
    return NRR_OK;
}

static nrr_status match_with_boxsums(const void *d_preop, const void *d_intraop, const void *d_boxsums,
                                     nrr_dtype dtype, nrr_dims dims, const int32_t *d_centers, int32_t n_blocks,
                                     const int32_t *d_n_blocks, const int32_t block[3], const int32_t radius[3],
                                     int32_t *d_disp, double *d_ncc, uint8_t *d_valid, void *stream, bool plain)
{
    clear_error();
    nrr_status st = check_match_args(d_preop, d_intraop, dtype, dims, d_centers, n_blocks, block, radius, d_disp,
                                     d_ncc, d_valid);
    if (st != NRR_OK) return st;
    if (!d_boxsums || ((uintptr_t)d_boxsums & 255u) != 0)
        return fail(NRR_E_INVALID, "box-sum buffer NULL or not 256-byte aligned");
    if (n_blocks == 0) return NRR_OK;
    MatchLaunch a{};
    a.preop = d_preop;
    a.intraop = d_intraop;
    a.s1 = d_boxsums;
    a.s2 = (const char *)d_boxsums + boxsum_s2_offset(dims, dtype);
    a.dtype = dtype;
    a.dims = dims;
    a.block = block[0];
    const bool cubic = block[1] == block[0] && block[2] == block[0];
    a.block_y = cubic ? 0 : block[1];
    a.block_z = cubic ? 0 : block[2];
    for (int i = 0; i < 3; ++i) a.radius[i] = radius[i];
    a.n_jobs = 1;
    a.jobs[0] = MatchJob{d_centers, d_n_blocks, n_blocks, d_disp, d_ncc, d_valid};
    if (cubic && !plain) apply_tuning(a, dtype, block[0], radius);
    a.one_cta_per_block = plain ? 1 : 0;
    st = device_error_word(&a.err);
    if (st != NRR_OK) return st;
    return launch_match(a, (cudaStream_t)stream);
}

nrr_status nrr_block_match_bs_aniso(const void *d_preop, const void *d_intraop, const void *d_boxsums,
                                    nrr_dtype dtype, nrr_dims dims, const int32_t *d_centers, int32_t n_blocks,
                                    const int32_t *d_n_blocks, const int32_t block[3], const int32_t radius[3],
                                    int32_t *d_disp, double *d_ncc, uint8_t *d_valid, void *stream)
{
    return match_with_boxsums(d_preop, d_intraop, d_boxsums, dtype, dims, d_centers, n_blocks, d_n_blocks, block,
                              radius, d_disp, d_ncc, d_valid, stream, false);
}

nrr_status nrr_block_match_plain(const void *d_preop, const void *d_intraop, const void *d_boxsums, nrr_dtype dtype,
                                 nrr_dims dims, const int32_t *d_centers, int32_t n_blocks, const int32_t *d_n_blocks,
                                 int32_t block, const int32_t radius[3], int32_t *d_disp, double *d_ncc,
                                 uint8_t *d_valid, void *stream)
{
    const int32_t b3[3] = {block, block, block};
    return match_with_boxsums(d_preop, d_intraop, d_boxsums, dtype, dims, d_centers, n_blocks, d_n_blocks, b3, radius,
                              d_disp, d_ncc, d_valid, stream, true);
}

nrr_status nrr_block_match_bs(const void *d_preop, const void *d_intraop, const void *d_boxsums, nrr_dtype dtype,
                              nrr_dims dims, const int32_t *d_centers, int32_t n_blocks, const int32_t *d_n_blocks,
                              int32_t block, const int32_t radius[3], int32_t *d_disp, double *d_ncc,
                              uint8_t *d_valid, void *stream)
{
    const int32_t b3[3] = {block, block, block};
    return nrr_block_match_bs_aniso(d_preop, d_intraop, d_boxsums, dtype, dims, d_centers, n_blocks, d_n_blocks, b3,
                                    radius, d_disp, d_ncc, d_valid, stream);
}

nrr_status nrr_boxsums_aniso(const void *d_intraop, nrr_dtype dtype, nrr_dims dims, const int32_t block[3],
                             void *d_boxsums, void *stream)
{
    clear_error();
    nrr_status st = check_dims3(dims, dtype, block);
    if (st != NRR_OK) return st;
    if (!d_intraop || !d_boxsums) return fail(NRR_E_INVALID, "NULL volume or box-sum buffer");
    if (((uintptr_t)d_boxsums & 255u) != 0) return fail(NRR_E_INVALID, "box-sum buffer must be 256-byte aligned");
    cudaStream_t s = (cudaStream_t)stream;
    if (block[1] == block[0] && block[2] == block[0])
        return launch_boxsums(d_intraop, dtype, dims, block[0], d_boxsums, s);
    void *scratch = nullptr;
    NRR_CUDA_TRY(cudaMallocAsync(&scratch, boxsum3_scratch_bytes(dims, dtype), s));
    st = launch_boxsums3(d_intraop, dtype, dims, block, d_boxsums, scratch, s);
    cudaError_t e = cudaFreeAsync(scratch, s);
    if (st == NRR_OK && e != cudaSuccess) return cuda_fail(e, "cudaFreeAsync");
    return st;
}

nrr_status nrr_block_match_aniso(const void *d_preop, const void *d_intraop, nrr_dtype dtype, nrr_dims dims,
                                 const int32_t *d_centers, int32_t n_blocks, const int32_t *d_n_blocks,
                                 const int32_t block[3], const int32_t radius[3], int32_t *d_disp, double *d_ncc,
                                 uint8_t *d_valid, void *stream)
{
    clear_error();
    nrr_status st = check_match_args(d_preop, d_intraop, dtype, dims, d_centers, n_blocks, block, radius, d_disp,
                                     d_ncc, d_valid);
    if (st != NRR_OK) return st;
    if (n_blocks == 0) return NRR_OK;
    cudaStream_t s = (cudaStream_t)stream;
    void *bs = nullptr;
    NRR_CUDA_TRY(cudaMallocAsync(&bs, boxsum_bytes(dims, dtype), s));
    st = nrr_boxsums_aniso(d_intraop, dtype, dims, block, bs, stream);
    if (st == NRR_OK)
        st = nrr_block_match_bs_aniso(d_preop, d_intraop, bs, dtype, dims, d_centers, n_blocks, d_n_blocks, block,
                                      radius, d_disp, d_ncc, d_valid, stream);
    cudaError_t e = cudaFreeAsync(bs, s);
    if (st == NRR_OK && e != cudaSuccess) return cuda_fail(e, "cudaFreeAsync");
    return st;
}

nrr_status nrr_block_match(const void *d_preop, const void *d_intraop, nrr_dtype dtype, nrr_dims dims,
                           const int32_t *d_centers, int32_t n_blocks, const int32_t *d_n_blocks, int32_t block,
                           const int32_t radius[3], int32_t *d_disp, double *d_ncc, uint8_t *d_valid, void *stream)
{
    const int32_t b3[3] = {block, block, block};
    return nrr_block_match_aniso(d_preop, d_intraop, dtype, dims, d_centers, n_blocks, d_n_blocks, b3, radius, d_disp,
                                 d_ncc, d_valid, stream);
}

}  // extern "C"
