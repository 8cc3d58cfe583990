/*
 * nrr.h -- C ABI of the GB300 block-selection and block-matching library.
 *
 * The library implements the data-parallel hot path of physics-based
 * non-rigid registration (PBNRR) as described in Chrisochoides et al.,
 * "Advancing Intra-operative Precision: Dynamic Data-Driven Non-Rigid
 * Registration for Enhanced Brain Tumor Resection in Image-Guided
 * Neurosurgery" (arXiv 2308.10868):
 *
 *   1. variance-based selection of registration blocks inside the
 *      intracranial mask of the floating (pre-operative) image
 *      (Sec. 4.1, "Parallel feature selection");
 *   2. exhaustive block matching of each selected block against a search
 *      window of the reference (intra-operative) image, scored by the
 *      normalized cross-correlation, keeping the arg-max displacement and
 *      its NCC (Sec. 3, the NCC equation and the O(B x W) bound; Sec. 4.3,
 *      the block-matching loop).
 *
 * The finite-element solve and outlier rejection that consume the result
 * (Sec. 3, the iterative FEM equation) are not part of this library.
 *
 * Conventions shared by every call
 * --------------------------------
 *  - Volumes are C-contiguous [nz][ny][nx] arrays, x fastest, in device
 *    memory.  dims = {nx, ny, nz}.  nx * sizeof(element) must be a multiple
 *    of 16 bytes (the row pitch of the TMA tensor map) and the base
 *    pointer 16-byte aligned.
 *  - Block edge `block` is the full odd edge b (3, 5, 7, 9 or 11);
 *    h = (b-1)/2.  Search radius is given per axis {rx, ry, rz}, each 0..7;
 *    the candidate shifts are d in [-rx,rx] x [-ry,ry] x [-rz,rz].
 *  - Centres and displacements are int32 triples (x, y, z).
 *  - NCC is Pearson's correlation of the block of the floating image at c
 *    with the block of the reference image at c+d.  A shift whose block
 *    leaves the volume, or whose reference block is flat, is not a
 *    candidate.  The maximum NCC wins; ties go to the smaller |d|^2, then
 *    to the smaller (dz, dy, dx) in lexicographic order.
 *  - uint16 intensities: all sums are exact integers and the score is the
 *    single IEEE double expression num / sqrt(vI * vJ) with
 *    num = N*S_IJ - S_I*S_J, vI = N*S_II - S_I^2, vJ = N*S_JJ - S_J^2,
 *    N = b^3, so results are reproducible bit for bit.
 *    float32 intensities: the score is the FP64 Pearson value of the float
 *    inputs (within 1e-6 of an FP64 reference; see nrr_block_match).
 *  - Every call that takes `stream` (a cudaStream_t, NULL = legacy default
 *    stream) only enqueues work, unless stated otherwise, and returns
 *    without waiting for it.  The caller owns every buffer it passes and
 *    must keep it alive until that stream work has completed.
 *  - No call throws, aborts or traps.  Each returns an nrr_status; a
 *    human-readable reason for the last failure on the calling thread is
 *    available from nrr_last_error().
 */
#ifndef NRR_H
#define NRR_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    NRR_OK = 0,
    NRR_PENDING = 1,       /* nrr_poll: the request has not finished yet */
    NRR_E_INVALID = -1,    /* an argument is out of range or inconsistent */
    NRR_E_NOMEM = -2,      /* device memory could not be obtained */
    NRR_E_CUDA = -3,       /* a CUDA runtime or driver call failed */
    NRR_E_CAPACITY = -4,   /* an output buffer or queue is too small */
    NRR_E_TIMEOUT = -5,    /* a bounded device-side wait gave up */
    NRR_E_INTERNAL = -6,   /* an internal consistency check failed */
    NRR_E_NOTFOUND = -7    /* unknown ticket */
} nrr_status;

typedef enum { NRR_U16 = 0, NRR_F32 = 1 } nrr_dtype;

typedef struct {
    int32_t nx, ny, nz;
} nrr_dims;

/* Static description of a status code.  Never NULL. */
const char *nrr_status_string(nrr_status s);

/* Detail message of the last failing call on this thread ("" if none).
 * The pointer stays valid until the next library call on this thread. */
const char *nrr_last_error(void);

/* Library ABI version (major * 100 + minor). */
int32_t nrr_version(void);

/* Number of CUDA kernels this library has launched in this process so far
 * (instrumentation for benchmarks and tests). */
int64_t nrr_kernel_launches(void);

/* ------------------------------------------------------------------------
 * Block selection (Sec. 4.1, "Parallel feature selection").
 *
 * Candidates are the grid points p = (i*stride, j*stride, k*stride) whose
 * centre voxel has mask[p] != 0 and whose b^3 block lies inside the volume.
 * Each candidate is scored by the exact variance key
 *     key = N * sum(I^2) - (sum I)^2      (N = b^3; = N^2 * variance),
 * and the n_sel = floor(0.5 + N_c * frac) candidates with the largest keys
 * are kept (N_c = number of candidates), never one with key 0 (a flat
 * block), so n_sel is capped at the number of candidates with key > 0.
 * Equal keys are ranked by raster index (z, y, x ascending), which makes the
 * selection deterministic.  The chosen centres are written to d_centers in
 * raster order.
 *
 *   d_preop      device, uint16 [nz][ny][nx], floating (pre-operative) image
 *   d_mask       device, uint8  [nz][ny][nx], nonzero inside the ICC mask
 *   block        odd, 3..11
 *   stride       1..64
 *   frac         0 < frac <= 1
 *   d_centers    device, int32 [max_blocks][3] (x, y, z), written
 *   max_blocks   capacity of d_centers (>= 0)
 *   d_n_selected device int32, optional (may be NULL): receives n_sel
 *   h_n_selected host int32, optional (may be NULL): receives n_sel; when
 *                given, the call waits for the stream (its one host sync)
 *   stream       cudaStream_t
 *
 * Scratch memory (keys of every grid point plus small histograms) is taken
 * from the device's stream-ordered memory pool and returned on the same
 * stream.  If n_sel > max_blocks only the first max_blocks centres are
 * written; with h_n_selected the call then returns NRR_E_CAPACITY.
 * Errors: NRR_E_INVALID (arguments), NRR_E_NOMEM, NRR_E_CUDA.
 * ---------------------------------------------------------------------- */
nrr_status nrr_select_blocks(const uint16_t *d_preop, const uint8_t *d_mask, nrr_dims dims,
                             int32_t block, int32_t stride, double frac,
                             int32_t *d_centers, int32_t max_blocks,
                             int32_t *d_n_selected, int32_t *h_n_selected, void *stream);

/* ------------------------------------------------------------------------
 * Box sums of the reference image, the per-shift sums S_J and S_JJ of the
 * NCC (Sec. 3): for every voxel v whose b^3 block lies in the volume,
 *   S1[v] = sum of J over the block centred at v,
 *   S2[v] = sum of J^2 over the same block.
 * uint16: S1 is int32 and S2 int64, both exact.  float32: both float32.
 * Layout of d_boxsums: S1 as [nz][ny][nx] elements, then S2 as
 * [nz][ny][nx] elements starting at the next 256-byte boundary; size from
 * nrr_boxsum_bytes.  Voxels whose block leaves the volume hold 0.
 * ---------------------------------------------------------------------- */
nrr_status nrr_boxsum_bytes(nrr_dims dims, nrr_dtype dtype, size_t *bytes);
nrr_status nrr_boxsums(const void *d_intraop, nrr_dtype dtype, nrr_dims dims, int32_t block,
                       void *d_boxsums, void *stream);

/* ------------------------------------------------------------------------
 * Exhaustive NCC block matching (Sec. 3; Sec. 4.3 block-matching loop).
 *
 * For every block i < n (n = n_blocks, or *d_n_blocks when that pointer is
 * given, clamped to n_blocks), centred at d_centers[i] in the floating
 * image, every shift d of the search window is scored by NCC against the
 * reference image and the best one (rule above) is returned:
 *
 *   d_preop, d_intraop  device volumes of `dtype` (uint16 or float32)
 *   d_centers  device int32 [n_blocks][3]
 *   d_n_blocks device int32, optional: actual count, read on the device
 *   block      odd 3..11;  radius  host int32[3] = {rx, ry, rz}, each 0..7
 *   d_disp     device int32 [n_blocks][3], written: best d (x, y, z)
 *   d_ncc      device double [n_blocks], written: NCC at d (NaN if invalid)
 *   d_valid    device uint8 [n_blocks], written: 1 if the block had at
 *              least one candidate shift; a block whose centre is too close
 *              to the border or whose floating block is flat has valid = 0
 *              and d = (0,0,0)
 *
 * uint16: displacements and NCC are bit-identical to the exact-integer
 * definition above.  float32: the search accumulates in FP32 with a
 * rigorous error bound; the shifts the bound cannot rule out are rescored in
 * FP64, so the returned NCC is the FP64 Pearson value of the chosen shift
 * (the chosen shift can differ from an FP64 reference only between shifts
 * whose FP64 scores differ by rounding).
 *
 * nrr_block_match computes the box sums itself (scratch from the stream-
 * ordered pool); nrr_block_match_bs takes them precomputed by nrr_boxsums
 * for the same volume and block size.
 * Errors: NRR_E_INVALID, NRR_E_NOMEM, NRR_E_CUDA.  A device-side wait that
 * times out is reported by nrr_device_status.
 * ---------------------------------------------------------------------- */
nrr_status nrr_block_match(const void *d_preop, const void *d_intraop, nrr_dtype dtype, nrr_dims dims,
                           const int32_t *d_centers, int32_t n_blocks, const int32_t *d_n_blocks,
                           int32_t block, const int32_t radius[3],
                           int32_t *d_disp, double *d_ncc, uint8_t *d_valid, void *stream);

nrr_status nrr_block_match_bs(const void *d_preop, const void *d_intraop, const void *d_boxsums,
                              nrr_dtype dtype, nrr_dims dims,
                              const int32_t *d_centers, int32_t n_blocks, const int32_t *d_n_blocks,
                              int32_t block, const int32_t radius[3],
                              int32_t *d_disp, double *d_ncc, uint8_t *d_valid, void *stream);

/* Waits for `stream`, then reports and clears the device error word that
 * the kernels set when a bounded wait gives up (NRR_E_TIMEOUT) or an
 * internal check fails (NRR_E_INTERNAL).  NRR_OK if neither happened. */
nrr_status nrr_device_status(void *stream);

#ifdef __cplusplus
}
#endif

#endif /* NRR_H */
