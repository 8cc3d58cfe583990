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
 *    h = (b-1)/2.  Search radius is given per axis {rx, ry, rz}, each
 *    0..15; the candidate shifts are d in [-rx,rx] x [-ry,ry] x [-rz,rz].
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
 * Block selection with a connectivity pattern (Sec. 4.1, "Parallel feature
 * selection": a connectivity pattern keeps selected blocks from being too
 * close to each other; its "face", "edge" and "vertex" simplex patterns are
 * 6-, 18- and 26-connectivity, the face pattern giving the densest
 * selection).
 *
 * Same candidates, keys, count n_sel = floor(0.5 + N_c * frac) and order
 * (key descending, raster index ascending) as nrr_select_blocks.  The
 * candidates are taken greedily in that order: one is skipped when a
 * candidate taken before it is its neighbour on the candidate grid, i.e. its
 * grid offset (di, dj, dk) lies in {-1,0,1}^3 with |di|+|dj|+|dk| at most 1
 * (connectivity 6), 2 (18) or 3 (26); the walk stops after n_sel have been
 * taken, or earlier when the candidates run out.  Centres are written in
 * raster order.
 *
 *   connectivity  0 (no pattern: exactly nrr_select_blocks), 6, 18 or 26
 *   other arguments as nrr_select_blocks
 *
 * Scratch: as nrr_select_blocks plus 5 bytes per candidate grid point, from
 * the stream-ordered pool.  The pattern runs as one cooperative kernel (all
 * of its CTAs resident at once) whose rounds are separated by grid-wide
 * barriers; a barrier that waits longer than 2 s gives up and sets the
 * device error word (nrr_device_status then returns NRR_E_TIMEOUT).  Not for
 * use inside stream capture.
 * Errors: NRR_E_INVALID (arguments, connectivity), NRR_E_NOMEM, NRR_E_CUDA,
 * NRR_E_CAPACITY as nrr_select_blocks.
 * ---------------------------------------------------------------------- */
nrr_status nrr_select_blocks_spaced(const uint16_t *d_preop, const uint8_t *d_mask, nrr_dims dims,
                                    int32_t block, int32_t stride, double frac, int32_t connectivity,
                                    int32_t *d_centers, int32_t max_blocks,
                                    int32_t *d_n_selected, int32_t *h_n_selected, void *stream);

/* ------------------------------------------------------------------------
 * Block selection that allocates nothing.
 *
 * Some callers cannot allocate device memory when they call in: systems
 * whose whole device-memory budget is reserved at start-up (an
 * intra-operative workstation whose memory use must be fixed and verified in
 * advance), code that runs where an allocation is not allowed (a host
 * callback, a real-time thread that must not block in the allocator), or a
 * host application whose own pool owns all device memory.
 * nrr_select_blocks_noalloc does exactly what nrr_select_blocks does, with
 * the same arguments, results and errors, but takes its scratch from a
 * fixed array of NRR_SELECT_STATIC_SCRATCH_BYTES (32 MiB) built into the
 * library instead of from an allocator: it calls no cudaMalloc, cudaFree or
 * other allocating routine.  The array is reserved on a device when the
 * library's selection module is loaded there: with lazy module loading
 * (the CUDA default) that happens at the first selection call of any kind
 * on that device at the latest, and that call can then need the 32 MiB and
 * fail with NRR_E_CUDA (out of memory) if the process's own allocator
 * already holds all device memory.  Make a first selection call (this entry
 * point on a tiny volume will do) at start-up, while memory is still free
 * and before any stream capture; the array is then held until the process
 * exits.
 *
 *  - Limit: the scratch needs about 8 bytes per candidate grid point
 *    (ceil(nx/stride) * ceil(ny/stride) * ceil(nz/stride)), so up to about
 *    4 million grid points; a larger grid returns NRR_E_CAPACITY and writes
 *    nothing.
 *  - The first call on each device also looks up the array's device
 *    address (once); the start-up call above covers it.
 *  - All calls share the one array and each leaves its contents there (each
 *    call clears what it needs zeroed before use).  Calls whose work could
 *    overlap on the GPU (different streams without ordering between them,
 *    or several host threads) race on it: order them on one stream or
 *    serialise them.
 *  - The paper has no counterpart of this entry point.
 * ---------------------------------------------------------------------- */
#define NRR_SELECT_STATIC_SCRATCH_BYTES (32u * 1024u * 1024u)
nrr_status nrr_select_blocks_noalloc(const uint16_t *d_preop, const uint8_t *d_mask, nrr_dims dims,
                                     int32_t block, int32_t stride, double frac,
                                     int32_t *d_centers, int32_t max_blocks,
                                     int32_t *d_n_selected, int32_t *h_n_selected, void *stream);

/* ------------------------------------------------------------------------
 * Box sums of the reference image, from the per-shift sums S_J and S_JJ of
 * the NCC (Sec. 3): for every voxel v whose b^3 block lies in the volume,
 *   S1[v] = uint16:  sum of J over the block centred at v,
 *           float32: sum of (J - c) over the block, c = J at the volume's
 *                    centre voxel (nx/2, ny/2, nz/2), each J - c rounded
 *                    once (so that the sums keep a block's spread even on
 *                    a large intensity offset),
 *   A2[v] = uint16:  N * (sum of J^2) - S1[v]^2  (N = b^3; exact in 64 bits,
 *                    then rounded once to float32: N^2 times the block's
 *                    variance),
 *           float32: sum of (J - c)^2 over the block.
 * uint16: S1 is int32 (exact), A2 float32.  float32: both float32.
 * Layout of d_boxsums: S1 as [nz][ny][nx] elements, then A2 as [nz][ny][nx]
 * elements starting at the next 256-byte boundary (8 bytes per voxel in
 * all); size from nrr_boxsum_bytes.  Voxels whose block leaves the volume
 * hold 0.
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
 *   block      odd 3..11;  radius  host int32[3] = {rx, ry, rz}, each 0..15
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
 * A radius above 7 on an axis is searched as sub-windows of one smaller
 * radius that tile [-r, r] on that axis (two for r = 8..11, three for
 * r = 12..15; they may overlap), each block's sub-windows in turn within
 * the same launch; the result is the same best shift under the rule above.
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

/* ------------------------------------------------------------------------
 * nrr_block_match_plain: nrr_block_match_bs in the plain launch form, one CTA
 * per block, as the paper's GPU kernel maps its loop over blocks to thread
 * blocks (Sec. 4.3), instead of persistent CTAs that walk the blocks with the
 * next block's window copy in flight.  Arguments, results (identical to
 * nrr_block_match_bs), ownership and errors are those of nrr_block_match_bs;
 * it is there to measure what the persistent form gains.
 * ---------------------------------------------------------------------- */
nrr_status nrr_block_match_plain(const void *d_preop, const void *d_intraop, const void *d_boxsums,
                                 nrr_dtype dtype, nrr_dims dims,
                                 const int32_t *d_centers, int32_t n_blocks, const int32_t *d_n_blocks,
                                 int32_t block, const int32_t radius[3],
                                 int32_t *d_disp, double *d_ncc, uint8_t *d_valid, void *stream);

/* ------------------------------------------------------------------------
 * Blocks with a different edge per axis (Sec. 5 lists the half block size,
 * like the half window size, per anatomical axis).  block = {bx, by, bz},
 * host int32[3], each odd in 3..11; N = bx*by*bz; the block centred at c
 * covers c +- (bx-1)/2 along x, (by-1)/2 along y, (bz-1)/2 along z.
 * Otherwise each call is its cubic counterpart above, with the same
 * arguments, results, exactness, ownership and errors:
 *
 *   nrr_select_blocks_aniso  = nrr_select_blocks (keys over the bx*by*bz
 *                              block; a candidate's block must lie in the
 *                              volume along every axis)
 *   nrr_boxsums_aniso        = nrr_boxsums (for a non-cubic block the sums
 *                              run in three separable passes through a
 *                              scratch buffer from the stream-ordered pool,
 *                              12 bytes per voxel for uint16, 8 for float32)
 *   nrr_block_match_aniso    = nrr_block_match
 *   nrr_block_match_bs_aniso = nrr_block_match_bs, with box sums from
 *                              nrr_boxsums_aniso for the same block
 * A cubic triple {b, b, b} takes exactly the cubic path.
 * ---------------------------------------------------------------------- */
nrr_status nrr_select_blocks_aniso(const uint16_t *d_preop, const uint8_t *d_mask, nrr_dims dims,
                                   const int32_t block[3], int32_t stride, double frac,
                                   int32_t *d_centers, int32_t max_blocks,
                                   int32_t *d_n_selected, int32_t *h_n_selected, void *stream);
nrr_status nrr_boxsums_aniso(const void *d_intraop, nrr_dtype dtype, nrr_dims dims, const int32_t block[3],
                             void *d_boxsums, void *stream);
nrr_status nrr_block_match_aniso(const void *d_preop, const void *d_intraop, nrr_dtype dtype, nrr_dims dims,
                                 const int32_t *d_centers, int32_t n_blocks, const int32_t *d_n_blocks,
                                 const int32_t block[3], const int32_t radius[3],
                                 int32_t *d_disp, double *d_ncc, uint8_t *d_valid, void *stream);
nrr_status nrr_block_match_bs_aniso(const void *d_preop, const void *d_intraop, const void *d_boxsums,
                                    nrr_dtype dtype, nrr_dims dims,
                                    const int32_t *d_centers, int32_t n_blocks, const int32_t *d_n_blocks,
                                    const int32_t block[3], const int32_t radius[3],
                                    int32_t *d_disp, double *d_ncc, uint8_t *d_valid, void *stream);

/* ------------------------------------------------------------------------
 * Execution-configuration autotuning (Sec. 4.3: the paper tunes its GPU
 * block-matching kernel by an empirical search over thread configurations).
 *
 * A match launch's shape: persistent CTAs per SM (0 = as many as fit),
 * window buffers per CTA, i.e. blocks in flight (1: one window buffer and
 * more CTAs; 2: the next block's copy overlaps this block's search; 0 = the
 * one that fits more CTAs), and where each thread's box sums come from (0
 * or 1: loaded at the bounds; 2: staged into shared memory by asynchronous
 * copies while the block is searched), and the search lines each thread
 * owns (uint16 cubic blocks only: 1, or 2 sharing each converted window row;
 * 0 = by the x-shift count 2r+1 of one window: one line up to 5 and at 9,
 * else two; float32 and per-axis blocks always take one and ignore the
 * field).  No shape changes a result bit.
 *
 * nrr_autotune_match times the match kernel for one (dtype, block, radius)
 * at every feasible shape on the given inputs (arguments as
 * nrr_block_match_bs, with a host block count) and stores the fastest in a
 * per-process table that every later match launch of that variant uses.
 * It waits for `stream`.  best_ctas_per_sm and best_ms may be NULL.
 * nrr_tuning_get/set read and write one entry's CTAs per SM (set leaves the
 * other fields by occupancy), nrr_tuning_get_shape/set_shape the whole
 * shape (a shape whose layout does not fit makes the launches fail with
 * NRR_E_INVALID); nrr_tuning_save/load write and read the whole table as
 * text.
 * ---------------------------------------------------------------------- */
typedef struct {
    int32_t ctas_per_sm; /* 0..64 */
    int32_t windows;     /* 0..2 */
    int32_t stage;       /* 0..2 */
    int32_t lines;       /* 0..2 */
} nrr_match_shape;

nrr_status nrr_autotune_match(const void *d_preop, const void *d_intraop, const void *d_boxsums,
                              nrr_dtype dtype, nrr_dims dims, const int32_t *d_centers, int32_t n_blocks,
                              int32_t block, const int32_t radius[3],
                              int32_t *d_disp, double *d_ncc, uint8_t *d_valid,
                              int32_t *best_ctas_per_sm, float *best_ms, void *stream);
nrr_status nrr_tuning_get(nrr_dtype dtype, int32_t block, const int32_t radius[3], int32_t *ctas_per_sm);
nrr_status nrr_tuning_set(nrr_dtype dtype, int32_t block, const int32_t radius[3], int32_t ctas_per_sm);
nrr_status nrr_tuning_get_shape(nrr_dtype dtype, int32_t block, const int32_t radius[3], nrr_match_shape *shape);
nrr_status nrr_tuning_set_shape(nrr_dtype dtype, int32_t block, const int32_t radius[3],
                                const nrr_match_shape *shape);
nrr_status nrr_tuning_save(const char *path);
nrr_status nrr_tuning_load(const char *path);

/* ------------------------------------------------------------------------
 * Batched parameter search (the paper's sweep over registration parameters,
 * Sec. 4.2 speculative runs with many parameter values and Sec. 5 the
 * parameter pool of the learned predictor, both run there as separate
 * registrations).
 *
 * A plan binds one or more uint16 volume pairs with their masks (device
 * pointers that must stay valid and unchanged in place for the plan's life;
 * the pairs may differ in size) and n_settings settings, each on one pair;
 * each setting is a full registration's hot path: selection with (block,
 * stride, frac), then matching with (block, radius).  The plan owns all
 * scratch and result memory (allocated at creation, nothing is allocated
 * when it runs).  Work shared between settings is done once: box sums per
 * distinct (pair, block size), selection per distinct (pair, block, stride,
 * frac), one match of the largest fraction per (pair, block, stride,
 * radius) with smaller fractions gathered from it, and smaller radii
 * answered by a larger radius's search (up to radius 7 per axis).
 * Matching runs as one persistent launch per distinct (block, radius)
 * holding that variant's settings of every pair (up to 16 per launch).
 *
 * flags: NRR_BATCH_GRAPH captures the whole sweep into one CUDA graph at
 * creation, so nrr_batch_run is a single graph launch with no host round
 * trip; NRR_BATCH_AUTOTUNE runs the sweep once at creation and autotunes
 * every match variant on it (creation then waits for the device);
 * NRR_BATCH_NO_DEDUP selects and matches every setting by itself (no
 * shared selections, gathered fractions or radius levels; the results are
 * the same bit for bit), to measure what the sharing saves;
 * NRR_BATCH_PLAIN_LAUNCH makes every match launch one CTA per block instead
 * of persistent CTAs that take blocks from a work queue (same results).
 * nrr_batch_run enqueues one sweep on `stream` (asynchronous).  After it
 * completes, nrr_batch_view_get gives setting s's device arrays: the count
 * (device int32), centres, displacements, NCC and valid flags, each with
 * `capacity` entries of which the first count are meaningful.
 * Errors: NRR_E_INVALID (arguments), NRR_E_NOMEM, NRR_E_CUDA.
 * ---------------------------------------------------------------------- */
typedef struct {
    int32_t block;      /* odd 3..11 */
    int32_t stride;     /* 1..64 */
    int32_t radius[3];  /* 0..15 each; radius reuse across settings only up to 7 */
    double frac;        /* (0, 1] */
} nrr_setting;

typedef struct nrr_batch_s *nrr_batch;

typedef struct {
    const int32_t *centers;   /* device [capacity][3] */
    const int32_t *n_blocks;  /* device, one int32 */
    const int32_t *disp;      /* device [capacity][3] */
    const double *ncc;        /* device [capacity] */
    const uint8_t *valid;     /* device [capacity] */
    int32_t capacity;
} nrr_batch_view;

enum { NRR_BATCH_GRAPH = 1, NRR_BATCH_AUTOTUNE = 2, NRR_BATCH_NO_DEDUP = 4, NRR_BATCH_PLAIN_LAUNCH = 8 };

/* One volume pair of a plan: uint16 reference (pre-operative) and floating
 * (intra-operative) volumes and the mask, device, [nz][ny][nx] x-fastest,
 * volumes 16-byte aligned, nx * 2 a multiple of 16. */
typedef struct {
    const uint16_t *d_preop;
    const uint16_t *d_intraop;
    const uint8_t *d_mask;
    nrr_dims dims;
} nrr_pair;

/* A plan over one pair: nrr_batch_create_pairs with that single pair. */
nrr_status nrr_batch_create(const uint16_t *d_preop, const uint16_t *d_intraop, const uint8_t *d_mask,
                            nrr_dims dims, const nrr_setting *settings, int32_t n_settings, int32_t flags,
                            nrr_batch *plan);
/* pairs: n_pairs >= 1 entries (host, read during the call); pair_of: host
 * [n_settings], setting s runs on pairs[pair_of[s]] (NULL: all on pair 0).
 * Errors: NRR_E_INVALID for a bad pair, setting or pair index (the message
 * names it). */
nrr_status nrr_batch_create_pairs(const nrr_pair *pairs, int32_t n_pairs, const nrr_setting *settings,
                                  const int32_t *pair_of, int32_t n_settings, int32_t flags, nrr_batch *plan);
nrr_status nrr_batch_run(nrr_batch plan, void *stream);
nrr_status nrr_batch_view_get(nrr_batch plan, int32_t setting, nrr_batch_view *view);
nrr_status nrr_batch_destroy(nrr_batch plan);

/* ------------------------------------------------------------------------
 * Serving with continuous batching (the paper's client/server registration
 * service, Sec. 4.1 "Ease-of-use", on one GPU).
 *
 * nrr_server_start starts a scheduler thread on the current device with
 * `slots` CUDA streams.  nrr_submit queues one registration and returns a
 * ticket at once.  Queued requests are admitted in arrival order whenever
 * a slot is free and the memory available, less reserve_bytes, covers the
 * request's scratch and result buffers (available: the device's free memory
 * plus what the library's request pool holds mapped but unused; the pool
 * keeps the memory it maps for the rest of the process, for later requests
 * and servers); queued requests of the same dtype, block and radius as an
 * admitted one join it (up to 16: each runs its own selection and box sums,
 * one match launch holds all their jobs); admitted requests run
 * concurrently (their kernels overlap on the device) and a new one starts
 * as soon as an earlier one finishes.  Each request runs selection (on
 * d_select), box sums and matching exactly as the synchronous calls do, so
 * its result equals a lone call's bit for bit whatever else is running.
 *
 * The caller keeps the request's volumes and mask valid and unchanged until
 * nrr_poll has returned NRR_OK (or an error) for it.  nrr_poll returns
 * NRR_PENDING while the request is queued or running; afterwards it fills
 * `out` with the block count, device pointers to the results (owned by the
 * library until nrr_release), the time from submission to admission and
 * from submission to completion on the device.  nrr_release frees a
 * finished (or still queued) request's buffers and forgets its ticket.
 * A request whose allocation or launch fails is reported by nrr_poll with
 * that status; the server keeps serving the others.  nrr_server_stop waits
 * for running work and frees everything.  Only one server per process.
 * ---------------------------------------------------------------------- */
typedef struct {
    const void *d_preop;       /* floating volume, `dtype` */
    const void *d_intraop;     /* reference volume, `dtype` */
    const uint16_t *d_select;  /* uint16 floating volume used for selection
                                  (d_preop itself when dtype is NRR_U16) */
    const uint8_t *d_mask;
    nrr_dims dims;
    nrr_dtype dtype;
    int32_t block;
    int32_t stride;
    int32_t radius[3];
    double frac;
} nrr_request;

typedef struct {
    int32_t n_blocks;
    const int32_t *centers;  /* device [n_blocks][3] */
    const int32_t *disp;     /* device [n_blocks][3] */
    const double *ncc;       /* device [n_blocks] */
    const uint8_t *valid;    /* device [n_blocks] */
    double queued_s;         /* submission -> admission */
    double latency_s;        /* submission -> completion on the device */
} nrr_result;

nrr_status nrr_server_start(int32_t slots, size_t reserve_bytes);
/* As nrr_server_start with at most max_group (1..16) requests per match
 * launch (nrr_server_start: 16; 1: every request on its own). */
nrr_status nrr_server_start_ex(int32_t slots, size_t reserve_bytes, int32_t max_group);
nrr_status nrr_server_stop(void);
nrr_status nrr_submit(const nrr_request *req, uint64_t *ticket);
nrr_status nrr_poll(uint64_t ticket, nrr_result *out);
nrr_status nrr_release(uint64_t ticket);

/* ---- Robust finite-element update (Sec. 3 equation; Sec. 5 N_rej, N_int,
 * F_r) ------------------------------------------------------------------------
 * The step that consumes the block matches: mesh vertex displacements U
 * balance a linear elastic model against the matched displacements D,
 *     F_i = K U_i,   U_{i+1} = [K + H^T S H]^{-1} [H^T S D + F_i],
 * K the stiffness matrix, H the interpolation from mesh vertices to the
 * block centres, S the diagonal confidence of the matches.  The paper
 * leaves mesh, material, S and the rejection rule to its references; this
 * library reads them as:
 *   mesh      8-node hexahedra on a grid of vertices every `grid` voxels
 *             from the origin (Nx = ceil((nx - 1) / grid) + 1 per axis, the
 *             last vertex at or past the last voxel); an element is in the
 *             model when d_mask is set at its centre voxel (e * grid +
 *             grid / 2 per axis, clamped into the volume); vertices of no
 *             such element stay at U = 0;
 *   material  homogeneous isotropic linear elasticity (young, poisson),
 *             lengths in voxels, element stiffness by 2x2x2 Gauss points;
 *   H         trilinear interpolation in the element floor(c / grid)
 *             (clamped to the grid) of block centre c;
 *   S         s_k = ncc_k for a valid match with ncc_k > 0 whose element is
 *             in the model, else 0;
 *   steps     U_0 = 0; n_rej approximation steps, each a solve followed by
 *             the rejection (s_k = 0) of floor(0.5 + reject_frac * n) of
 *             the n blocks with s_k > 0: those with the largest squared
 *             residual |D_k - H_k U|^2, ties to the lower block index,
 *             never one at or below 1e-6 voxel^2; then n_int interpolation
 *             steps (solves without rejection); with no block left with
 *             s_k > 0 a step keeps U_i.
 * Each solve is conjugate gradients in FP64 preconditioned by the inverse of
 * each vertex's 3x3 diagonal block, warm-started from U_i, run until
 * |r| <= cg_tol |r_0| (r_0 = H^T S D + F_i - [K + H^T S H] U_i, the warm
 * start's residual), as one cooperative launch.  The sums of H^T S H and
 * H^T S D are accumulated in 64-bit fixed point (terms rounded to 2^-44 and
 * 2^-40), so results do not depend on the order of the device's atomics.
 *
 * nrr_fem_update arguments:
 *   d_mask [nz][ny][nx] u8, dims: the brain mask and the volume size;
 *   d_centers int32 [n][3] (x, y, z), d_disp int32 [n][3], d_ncc f64 [n],
 *     d_valid u8 [n]: the block matches (the outputs of nrr_block_match);
 *     n = n_blocks, 0 .. 2^19;
 *   params: grid >= 2, young > 0, 0 <= poisson < 0.5, n_rej >= 0,
 *     n_int >= 0, 0 <= reject_frac <= 1, cg_tol > 0, cg_max_iter >= 1;
 *   d_U f64 [Nz][Ny][Nx][3] (vertex (i, j, k) at x = i grid, ...): out;
 *   d_s f64 [n]: the confidence after the rejections (out);
 *   d_rejected_step int32 [n]: the approximation step that rejected each
 *     block, -1 if none (out);
 *   h_cg_iters: NULL, or a host array of n_rej + n_int ints receiving each
 *     solve's iteration count;
 *   stream: a cudaStream_t (NULL = legacy default stream).
 * Device buffers are the caller's; scratch (about 0.6 KB per vertex plus
 * 8 B per block) is allocated and freed on the stream.  The call waits for
 * the stream once at the end to read the solves' records.
 * Errors: NRR_E_INVALID for an argument out of range or a NULL pointer
 * (n_blocks > 0); NRR_E_INTERNAL if a solve stops short of cg_tol within
 * cg_max_iter iterations or meets a direction of non-positive curvature (a
 * model part no block pins); NRR_E_TIMEOUT if a grid barrier of the solve
 * gave up; NRR_E_CUDA / NRR_E_NOMEM from the runtime.
 *
 * nrr_fem_grid writes the vertex counts (Nx, Ny, Nz) of a volume and grid
 * spacing; no device work. */
typedef struct {
    int32_t grid;
    double young;
    double poisson;
    int32_t n_rej;
    int32_t n_int;
    double reject_frac;
    double cg_tol;
    int32_t cg_max_iter;
} nrr_fem_params;

nrr_status nrr_fem_grid(nrr_dims dims, int32_t grid, int32_t n_vertices[3]);
nrr_status nrr_fem_update(const uint8_t *d_mask, nrr_dims dims, const int32_t *d_centers, const int32_t *d_disp,
                          const double *d_ncc, const uint8_t *d_valid, int32_t n_blocks, const nrr_fem_params *params,
                          double *d_U, double *d_s, int32_t *d_rejected_step, int32_t *h_cg_iters, void *stream);

/* Waits for `stream`, then reports and clears the device error word that
 * the kernels set when a bounded wait gives up (NRR_E_TIMEOUT) or an
 * internal check fails (NRR_E_INTERNAL).  NRR_OK if neither happened. */
nrr_status nrr_device_status(void *stream);

/* Test hook for the bounded device-side waits (the paper has no counterpart:
 * it exists so that tests can make a wait run out without faulting or
 * hanging the GPU).  For kernels launched after the call:
 *   limit_ns          the limit of every bounded wait; 0 restores the
 *                     default of 2 s.  At most 60 s.
 *   missing_arrivals  arrivals, 0..1024, added to the target of every grid
 *                     barrier of the connectivity-pattern selection
 *                     (nrr_select_blocks_spaced) that never come: with one
 *                     or more, each barrier waits out its limit, the kernel
 *                     records NRR_E_TIMEOUT in the device error word and
 *                     returns.  0 restores normal barriers.
 * Process-wide; takes effect at launch (a captured graph keeps the values
 * it was captured with).  Returns NRR_E_INVALID for values out of range. */
nrr_status nrr_test_set_wait(uint64_t limit_ns, int32_t missing_arrivals);

#ifdef __cplusplus
}
#endif

#endif /* NRR_H */
