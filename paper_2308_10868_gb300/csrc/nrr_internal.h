// Internal declarations shared by the library's translation units.
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "nrr.h"

namespace nrr {

// ---- host-side error reporting -------------------------------------------
nrr_status fail(nrr_status s, const char *fmt, ...);
nrr_status cuda_fail(cudaError_t e, const char *what);
void clear_error();

#define NRR_CUDA_TRY(call)                                  \
    do {                                                    \
        cudaError_t e_ = (call);                            \
        if (e_ != cudaSuccess) return nrr::cuda_fail(e_, #call); \
    } while (0)

// Device word the kernels set on a bounded-wait timeout or failed check.
// Returns its device address for the current device (no allocation: it is a
// file-scope __device__ variable of the library).
nrr_status device_error_word(unsigned int **ptr);
// Next match work-queue head of this device's eager or captured ring (see
// MatchLaunch::queue).
constexpr int MATCH_QUEUE_SLOTS = 4096;
nrr_status match_queue_head(int32_t **ptr, bool captured);

// Bits of the device error word.
enum : unsigned int { DEV_ERR_TIMEOUT = 1u, DEV_ERR_INTERNAL = 2u };

// Limit of the kernels' bounded device-side waits for later launches (2 s
// unless a test shortened it through nrr_test_set_wait), and the arrivals
// that never come which a test adds to the selection pattern's grid
// barrier (0 outside tests).
constexpr uint64_t DEVICE_WAIT_NS = 2000000000ull;
uint64_t device_wait_ns();
unsigned int test_missing_arrivals();

// Encode a 3-D tiled tensor map over a [nz][ny][nx] volume of `dtype` with a
// box of (bx, by, bz) elements; out-of-bounds reads fill zeros.
nrr_status encode_volume_map(CUtensorMap *map, const void *base, nrr_dtype dtype, nrr_dims dims, int bx, int by,
                             int bz);

int sm_count();

// Running count of kernel launches made by the library in this process.
void count_launches(int n);

// Common argument checks.
nrr_status check_dims(nrr_dims dims, nrr_dtype dtype, int32_t block);
// Per-axis block edges (x, y, z): each odd in 3..11 and no larger than the volume.
nrr_status check_dims3(nrr_dims dims, nrr_dtype dtype, const int32_t *block);
inline size_t elem_size(nrr_dtype t) { return t == NRR_F32 ? 4 : 2; }
// float32 box sums are sums of J - c with c the reference volume's value at
// its centre voxel (nx/2, ny/2, nz/2): with c near the data the sums keep
// a block's spread even when the intensities sit on a large offset.  This
// is that voxel's index; the box-sum kernels and the match kernel read c
// from it.
__host__ __device__ inline long long volume_centre_index(int nx, int ny, int nz)
{
    return ((long long)(nz / 2) * ny + ny / 2) * nx + nx / 2;
}
inline size_t align_up(size_t v, size_t a) { return (v + a - 1) / a * a; }

// Box sums: number of bytes and the two sub-arrays of a box-sum buffer.
size_t boxsum_bytes(nrr_dims dims, nrr_dtype dtype);
inline size_t boxsum_s2_offset(nrr_dims dims, nrr_dtype dtype)
{
    size_t v = (size_t)dims.nx * dims.ny * dims.nz;
    (void)dtype;
    return align_up(v * 4, 256);  // S1 is int32 or float: 4 bytes each
}
// Box sums for blocks with per-axis edges (nrr_boxsum3.cu): three separable
// passes through a scratch buffer of boxsum3_scratch_bytes.
size_t boxsum3_scratch_bytes(nrr_dims dims, nrr_dtype dtype);
nrr_status launch_boxsums3(const void *d_intraop, nrr_dtype dtype, nrr_dims dims, const int32_t block[3],
                           void *d_boxsums, void *d_scratch, cudaStream_t stream);
nrr_status launch_boxsums(const void *d_intraop, nrr_dtype dtype, nrr_dims dims, int32_t block, void *d_boxsums,
                          cudaStream_t stream);

// Selection keys N*sum(I^2) - (sum I)^2 at the stride grid points through the
// box-sum kernel (strides up to 3): keys[(k*gy + j)*gx + i] for the point
// (i, j, k)*stride, -1 for non-candidates; adds the candidate count, the count
// of keys > 0 and the largest key into *nc, *npos, *maxkey.
bool keys_box_supported(int32_t block, int32_t stride);
nrr_status launch_keys_box(const uint16_t *d_preop, const uint8_t *d_mask, nrr_dims dims, int32_t block,
                           int32_t stride, int gx, int gy, int gz, long long *keys, unsigned long long *nc,
                           unsigned long long *npos, unsigned long long *maxkey, cudaStream_t stream);

// Match kernel launch (box sums already computed).  One launch serves up to
// MATCH_MAX_JOBS lists of blocks that share the volume pair, block size and
// search radius (one job per registration or per parameter setting).
constexpr int MATCH_MAX_JOBS = 16;
// Extra search radii a job reports besides its own (batched search): the
// best shift within a smaller box [-r, r] per axis, from the same search.
constexpr int MATCH_MAX_LEVELS = 4;
// Largest search radius per axis one window holds, and the most sub-windows
// per axis a larger radius is split into (radius up to 15 needs three).
constexpr int MATCH_WINDOW_R = 7;
constexpr int MATCH_MAX_SUB = 4;
constexpr int MATCH_MAX_R = 15;
struct MatchLevel {
    int32_t r[3];
    int32_t *disp;
    double *ncc;
    uint8_t *valid;
};
struct MatchJob {
    const int32_t *centers;  // [cap][3]
    const int32_t *d_n;      // optional device count (<= cap)
    int32_t cap;
    int32_t *disp;
    double *ncc;
    uint8_t *valid;
    int32_t n_levels;  // 0 .. MATCH_MAX_LEVELS
    MatchLevel levels[MATCH_MAX_LEVELS];
    // The job's volume pair (jobs of one launch may come from different
    // registrations of different sizes): null / 0 fields take the launch's
    // volumes, box sums and dims; mapJ / mapI are device copies of the
    // job's tensor maps (window and floating block boxes of the launch's
    // variant), null for the launch's own maps.
    const void *preop, *intraop, *s1, *s2;
    int32_t nx, ny, nz;
    const CUtensorMap *mapJ, *mapI;
};
struct MatchLaunch {
    const void *preop;
    const void *intraop;
    const void *s1;
    const void *s2;
    nrr_dtype dtype;
    nrr_dims dims;
    int32_t block;             // block edge along x
    int32_t block_y, block_z;  // edges along y and z; 0 = the x edge (cubic block)
    int32_t radius[3];
    int n_jobs;
    MatchJob jobs[MATCH_MAX_JOBS];
    int ctas_per_sm;  // persistent CTAs per SM; 0 = as many as fit
    int one_cta_per_block;  // plain launch: one CTA per block instead of persistent CTAs
    int stage_boxsums;      // 0 or 1 = load the box sums at the bounds, 2 = stage them
    int windows;            // window buffers: 0 = by occupancy, 1 or 2
    int lines;              // search lines per thread: 0 = by x-shift count, 1 or 2 (uint16 cubic blocks only)
    unsigned int *err;
    // work-queue head (device int32) the launcher zeroes on the stream before
    // the kernel; null: the next head of a per-device ring, one ring for
    // eager launches (distinct while fewer than MATCH_QUEUE_SLOTS of them are
    // in flight at once) and one for launches captured into CUDA graphs
    // (distinct while fewer than MATCH_QUEUE_SLOTS captured launches live)
    int32_t *queue;
    // filled in by launch_match: sub-windows of radius sub_r per axis that
    // tile [-radius, radius] (one of radius `radius` when it is at most
    // MATCH_WINDOW_R), nsub per axis centred at soff
    int sub_r[3];
    int nsub[3];
    int soff[3][MATCH_MAX_SUB];
};
// Sub-windows for a search radius R on one axis: k = ceil((2R+1)/15) windows
// of one radius r (k(2r+1) >= 2R+1), centred at min(-R + r + i(2r+1),
// R - r): they cover [-R, R], may overlap (a shift searched twice gives the
// same exact score), and need one window of radius r in shared memory.
void plan_subwindows(int R, int *r, int *k, int *off);
// TMA boxes of a match launch's variant (dtype, block edges, search radius):
// the window box (wbox[3], x y z) and the floating-block box (tbox[3]), for
// tensor maps a caller encodes itself (jobs with their own volumes).
void match_boxes(nrr_dtype dtype, int block, int by, int bz, const int32_t radius[3], int wbox[3], int tbox[3]);
nrr_status launch_match(const MatchLaunch &a, cudaStream_t stream);

// Upper bound on resident match CTAs per SM for this launch's variant.
nrr_status match_occupancy(const MatchLaunch &a, int *ctas_per_sm);

// Autotuned persistent CTAs per SM for a match variant (0 = as many as fit).
// The tuned launch shape of a (dtype, block, radius) variant, written into
// a launch (CTAs per SM, window buffers, box-sum staging).
void apply_tuning(MatchLaunch &a, nrr_dtype dtype, int block, const int32_t *radius);

// Autotuner entry used by the batch plan (C ABI function).
// Block selection on caller-provided scratch (no allocation, no host sync).
struct SelectPlan {
    int gx, gy, gz;
    long long ng;
    int nchunks;
    int connectivity;  // 0, 6, 18 or 26
    size_t off_keys, off_hist, off_state, off_sync, off_cnt, off_list, off_sp_state, off_sp_mask, off_sp_tiles, bytes;
};
SelectPlan select_plan(nrr_dims d, int stride, int connectivity = 0);
nrr_status enqueue_select(const uint16_t *preop, const uint8_t *mask, nrr_dims d, int block, int stride, double frac,
                          int32_t *centers, int32_t max_blocks, int32_t *d_n_selected, unsigned char *ws,
                          const SelectPlan &p, cudaStream_t s, int block_y = 0, int block_z = 0);

// Connectivity pattern of the selection (6, 18 or 26 neighbours on the
// candidate grid): keeps selectable (key > 0) only the members of the greedy
// independent set, in selection order, of a prefix of the candidates that
// holds at least n_sel = floor(0.5 + *nc * frac) members if the whole set
// does, and sets *npos to the number kept.  `sync` must be zero on entry;
// state and hmask hold ng bytes and ng 32-bit words.
struct SpacingSync {
    unsigned int arrive;
    unsigned int pad;
    unsigned long long undecided[3];
    unsigned int hist[2048];
};
// Tile of the candidate grid the connectivity-pattern kernel works on.
constexpr int SP_TILE_X = 16, SP_TILE_Y = 8, SP_TILE_Z = 8;
nrr_status launch_spacing(int connectivity, long long *keys, int gx, int gy, long long ng, double frac,
                          unsigned char *state, unsigned int *hmask, SpacingSync *sync,
                          const unsigned long long *nc, const unsigned long long *maxkey, unsigned long long *npos,
                          unsigned int *tile_pend, cudaStream_t s);
// Offset of the selected count (int64) inside the selection scratch.
size_t select_count_offset(const SelectPlan &p);
nrr_status check_select_args(nrr_dims dims, int32_t block, int32_t stride, double frac);

}  // namespace nrr
