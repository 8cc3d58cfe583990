/*
 * CPU oracle for the block-selection and block-matching path of
 * physics-based non-rigid registration (Clatz et al. as used in
 * Chrisochoides et al., "Advancing Intra-operative Precision ...",
 * arXiv 2308.10868).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing on the product path may call, link or
 * load this file; only the tests, the smoke check and the benchmark's CPU
 * baseline do.  It shares no code, header, table or helper with the CUDA
 * library.
 *
 * It is written to be read against the paper, not to be fast: plain nested
 * loops in the order the method states them, FP64 for every real quantity,
 * exact 64-bit integer sums for uint16 intensities.  Build with
 * -O2 -fopenmp -ffp-contract=off (no FMA contraction, no fast-math), so the
 * one floating-point expression that decides the arg-max is evaluated with
 * IEEE round-to-nearest multiply, square root and divide.
 *
 * Readings of the paper that this file fixes (the paper's NCC formula is
 * garbled and several details are left open):
 *   - NCC is Pearson's correlation of the floating (pre-operative) block and
 *     the reference (intra-operative) block, each mean-centred over the
 *     block (Sec. 3, the NCC equation).  The signed value is maximised.
 *   - Block edge b is odd, h = (b-1)/2; the search radius is given per axis
 *     and the shifts are d in [-R,R]^3 (Sec. 3, complexity bound; Sec. 5
 *     gives the half window size per anatomical axis).  Sec. 5 counts twelve
 *     tunable parameters, which holds only if the half block size is also
 *     given per axis: the *_3 functions take the block edges (bx, by, bz),
 *     each odd, N = bx*by*bz; the cubic functions are the case bx=by=bz=b.
 *   - A shift whose block leaves the volume, or whose reference block is
 *     flat (zero variance), is not a candidate.
 *   - Ties in NCC are broken by smaller |d|^2, then by (dz,dy,dx)
 *     lexicographic order.
 *   - Candidates for selection are grid points whose coordinates are
 *     multiples of the stride, whose centre voxel lies in the mask and whose
 *     block lies inside the volume.  Each is scored by the exact variance key
 *     N*sum(I^2) - (sum I)^2 (N = b^3), which orders blocks as their variance
 *     does (Sec. 4.1, "Parallel feature selection").
 *   - The number selected is floor(0.5 + N_c * F_s) with N_c the number of
 *     candidates (Sec. 4.1), capped at the number of candidates with a
 *     nonzero key.  Order is key descending, raster index ascending; the
 *     selected centres are returned in raster order.
 *   - Connectivity pattern (Sec. 4.1, optional): greedy in selection order;
 *     a candidate is skipped if an already accepted candidate is its 6-, 18-
 *     or 26-neighbour on the candidate grid (offsets in {-1,0,1}^3 of L1
 *     norm at most 1, 2 or 3).
 *
 * Layout: volumes are C-contiguous [nz][ny][nx]; centres and displacements
 * are int32 triples (x, y, z).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

static int64_t lin(int64_t x, int64_t y, int64_t z, int64_t nx, int64_t ny)
{
    return (z * ny + y) * nx + x;
}

int oracle_num_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

void oracle_set_threads(int n)
{
#ifdef _OPENMP
    if (n > 0) omp_set_num_threads(n);
#else
    (void)n;
#endif
}

/* Block of edges (bx,by,bz) centred at (x,y,z) lies inside the volume. */
static int block_inside(int nx, int ny, int nz, const int bl[3], int64_t x, int64_t y, int64_t z)
{
    int hx = (bl[0] - 1) / 2, hy = (bl[1] - 1) / 2, hz = (bl[2] - 1) / 2;
    return x - hx >= 0 && y - hy >= 0 && z - hz >= 0 &&
           x + hx <= nx - 1 && y + hy <= ny - 1 && z + hz <= nz - 1;
}

/* Exact variance key of the bx*by*bz block at (x,y,z):
 * N*sum(I^2) - (sum I)^2, which equals N^2 times the population variance
 * (Sec. 4.1). */
int64_t oracle_block_key_3(const uint16_t *vol, int nx, int ny, int nz, int bx, int by, int bz, int x, int y,
                           int z)
{
    int hx = (bx - 1) / 2, hy = (by - 1) / 2, hz = (bz - 1) / 2;
    int64_t n = (int64_t)bx * by * bz, s = 0, q = 0;
    (void)nz;
    for (int k = -hz; k <= hz; ++k)
        for (int j = -hy; j <= hy; ++j)
            for (int i = -hx; i <= hx; ++i) {
                int64_t v = vol[lin(x + i, y + j, z + k, nx, ny)];
                s += v;
                q += v * v;
            }
    return n * q - s * s;
}

int64_t oracle_block_key(const uint16_t *vol, int nx, int ny, int nz, int b, int x, int y, int z)
{
    return oracle_block_key_3(vol, nx, ny, nz, b, b, b, x, y, z);
}

/* Keys of every stride grid point, in raster order of the grid
 * (gz, gy, gx ascending).  Non-candidates get -1.  Returns N_c. */
int64_t oracle_grid_keys_3(const uint16_t *preop, const uint8_t *mask, int nx, int ny, int nz, int bx, int by,
                           int bz, int stride, int64_t *keys)
{
    const int bl[3] = {bx, by, bz};
    int64_t gx = (nx + stride - 1) / stride, gy = (ny + stride - 1) / stride,
            gz = (nz + stride - 1) / stride, nc = 0;
#pragma omp parallel for reduction(+ : nc) schedule(static)
    for (int64_t k = 0; k < gz; ++k)
        for (int64_t j = 0; j < gy; ++j)
            for (int64_t i = 0; i < gx; ++i) {
                int64_t x = i * stride, y = j * stride, z = k * stride, g = (k * gy + j) * gx + i;
                if (block_inside(nx, ny, nz, bl, x, y, z) && mask[lin(x, y, z, nx, ny)] != 0) {
                    keys[g] = oracle_block_key_3(preop, nx, ny, nz, bx, by, bz, (int)x, (int)y, (int)z);
                    nc += 1;
                } else {
                    keys[g] = -1;
                }
            }
    return nc;
}

int64_t oracle_grid_keys(const uint16_t *preop, const uint8_t *mask, int nx, int ny, int nz,
                         int b, int stride, int64_t *keys)
{
    return oracle_grid_keys_3(preop, mask, nx, ny, nz, b, b, b, stride, keys);
}

typedef struct {
    int64_t key;
    int64_t idx;
} keyed;

static int by_key_desc_idx_asc(const void *pa, const void *pb)
{
    const keyed *a = (const keyed *)pa, *b = (const keyed *)pb;
    if (a->key != b->key) return a->key > b->key ? -1 : 1;
    return a->idx < b->idx ? -1 : (a->idx > b->idx ? 1 : 0);
}

static int by_idx_asc(const void *pa, const void *pb)
{
    const keyed *a = (const keyed *)pa, *b = (const keyed *)pb;
    return a->idx < b->idx ? -1 : (a->idx > b->idx ? 1 : 0);
}

/* Number of blocks to select from N_c candidates at fraction frac:
 * floor(0.5 + N_c * frac), i.e. N_c*frac rounded half up (Sec. 4.1). */
int64_t oracle_n_select(int64_t n_candidates, double frac)
{
    double x = (double)n_candidates * frac;
    double y = 0.5 + x;
    return (int64_t)floor(y);
}

/* Variance-based block selection (Sec. 4.1).  Writes up to `cap` centres
 * (x,y,z) in raster order; returns the number selected (may exceed cap).
 * *n_candidates receives N_c. */
int64_t oracle_select_blocks_3(const uint16_t *preop, const uint8_t *mask, int nx, int ny, int nz, int bx,
                               int by, int bz, int stride, double frac, int32_t *centers, int64_t cap,
                               int64_t *n_candidates)
{
    int64_t gx = (nx + stride - 1) / stride, gy = (ny + stride - 1) / stride,
            gz = (nz + stride - 1) / stride, ng = gx * gy * gz;
    int64_t *keys = (int64_t *)malloc(sizeof(int64_t) * (size_t)(ng > 0 ? ng : 1));
    int64_t nc = oracle_grid_keys_3(preop, mask, nx, ny, nz, bx, by, bz, stride, keys);
    keyed *pos = (keyed *)malloc(sizeof(keyed) * (size_t)(ng > 0 ? ng : 1));
    int64_t npos = 0;
    for (int64_t g = 0; g < ng; ++g)
        if (keys[g] > 0) {
            pos[npos].key = keys[g];
            pos[npos].idx = g;
            ++npos;
        }
    int64_t nsel = oracle_n_select(nc, frac);
    if (nsel > npos) nsel = npos;
    if (nsel < 0) nsel = 0;
    qsort(pos, (size_t)npos, sizeof(keyed), by_key_desc_idx_asc);
    qsort(pos, (size_t)nsel, sizeof(keyed), by_idx_asc);
    for (int64_t s = 0; s < nsel && s < cap; ++s) {
        int64_t g = pos[s].idx, i = g % gx, j = (g / gx) % gy, k = g / (gx * gy);
        centers[3 * s + 0] = (int32_t)(i * stride);
        centers[3 * s + 1] = (int32_t)(j * stride);
        centers[3 * s + 2] = (int32_t)(k * stride);
    }
    if (n_candidates) *n_candidates = nc;
    free(pos);
    free(keys);
    return nsel;
}

int64_t oracle_select_blocks(const uint16_t *preop, const uint8_t *mask, int nx, int ny, int nz,
                             int b, int stride, double frac, int32_t *centers, int64_t cap,
                             int64_t *n_candidates)
{
    return oracle_select_blocks_3(preop, mask, nx, ny, nz, b, b, b, stride, frac, centers, cap, n_candidates);
}

/* Variance-based selection with a connectivity pattern (Sec. 4.1: blocks
 * that are too close are not both selected; the "face", "edge" and "vertex"
 * simplex patterns mean 6-, 18- and 26-connectivity).  Reading: the
 * candidates are visited in selection order (key descending, raster index
 * ascending; flat blocks never); a candidate is accepted unless a candidate
 * accepted before it is its neighbour on the candidate grid, i.e. its grid
 * offset (di,dj,dk) lies in {-1,0,1}^3 with |di|+|dj|+|dk| at most 1 (6),
 * 2 (18) or 3 (26); the walk stops after floor(0.5 + N_c * F_s) accepted.
 * conn = 0 is selection without a pattern.  Writes up to `cap` centres in
 * raster order; returns the number selected. */
int64_t oracle_select_blocks_spaced(const uint16_t *preop, const uint8_t *mask, int nx, int ny, int nz,
                                    int b, int stride, double frac, int conn, int32_t *centers, int64_t cap,
                                    int64_t *n_candidates)
{
    int order = conn == 6 ? 1 : conn == 18 ? 2 : conn == 26 ? 3 : 0;
    int64_t gx = (nx + stride - 1) / stride, gy = (ny + stride - 1) / stride,
            gz = (nz + stride - 1) / stride, ng = gx * gy * gz;
    int64_t *keys = (int64_t *)malloc(sizeof(int64_t) * (size_t)(ng > 0 ? ng : 1));
    int64_t nc = oracle_grid_keys(preop, mask, nx, ny, nz, b, stride, keys);
    keyed *pos = (keyed *)malloc(sizeof(keyed) * (size_t)(ng > 0 ? ng : 1));
    unsigned char *taken = (unsigned char *)calloc((size_t)(ng > 0 ? ng : 1), 1);
    int64_t npos = 0;
    for (int64_t g = 0; g < ng; ++g)
        if (keys[g] > 0) {
            pos[npos].key = keys[g];
            pos[npos].idx = g;
            ++npos;
        }
    qsort(pos, (size_t)npos, sizeof(keyed), by_key_desc_idx_asc);
    int64_t want = oracle_n_select(nc, frac), nsel = 0;
    for (int64_t r = 0; r < npos && nsel < want; ++r) {
        int64_t g = pos[r].idx, i = g % gx, j = (g / gx) % gy, k = g / (gx * gy);
        int blocked = 0;
        for (int dk = -1; dk <= 1 && !blocked; ++dk)
            for (int dj = -1; dj <= 1 && !blocked; ++dj)
                for (int di = -1; di <= 1 && !blocked; ++di) {
                    int l1 = abs(di) + abs(dj) + abs(dk);
                    if (l1 == 0 || l1 > order) continue;
                    int64_t ii = i + di, jj = j + dj, kk = k + dk;
                    if (ii < 0 || jj < 0 || kk < 0 || ii >= gx || jj >= gy || kk >= gz) continue;
                    if (taken[(kk * gy + jj) * gx + ii]) blocked = 1;
                }
        if (!blocked) {
            taken[g] = 1;
            pos[nsel++] = pos[r];  /* accepted ones move to the front (r >= nsel) */
        }
    }
    qsort(pos, (size_t)nsel, sizeof(keyed), by_idx_asc);
    for (int64_t s = 0; s < nsel && s < cap; ++s) {
        int64_t g = pos[s].idx, i = g % gx, j = (g / gx) % gy, k = g / (gx * gy);
        centers[3 * s + 0] = (int32_t)(i * stride);
        centers[3 * s + 1] = (int32_t)(j * stride);
        centers[3 * s + 2] = (int32_t)(k * stride);
    }
    if (n_candidates) *n_candidates = nc;
    free(taken);
    free(pos);
    free(keys);
    return nsel;
}

/* ---------------------------------------------------------------------
 * NCC of one (block, shift) pair.
 * ------------------------------------------------------------------- */

/* uint16 path: exact int64 sums S_I, S_J, S_II, S_JJ, S_IJ over the block,
 * then  num = N*S_IJ - S_I*S_J,  vI = N*S_II - S_I^2,  vJ = N*S_JJ - S_J^2
 * (N^2 times covariance and variances: the common factor cancels) and the
 * single rounded expression  num / sqrt(vI * vJ).  Returns 0 and leaves
 * *ncc untouched when the shift is not a candidate. */
int oracle_ncc_u16_3(const uint16_t *preop, const uint16_t *intraop, int nx, int ny, int nz, int bx, int by,
                     int bz, int cx, int cy, int cz, int dx, int dy, int dz, double *ncc)
{
    const int bl[3] = {bx, by, bz};
    if (!block_inside(nx, ny, nz, bl, cx, cy, cz)) return 0;
    if (!block_inside(nx, ny, nz, bl, (int64_t)cx + dx, (int64_t)cy + dy, (int64_t)cz + dz)) return 0;
    int hx = (bx - 1) / 2, hy = (by - 1) / 2, hz = (bz - 1) / 2;
    int64_t n = (int64_t)bx * by * bz, si = 0, sj = 0, sii = 0, sjj = 0, sij = 0;
    for (int k = -hz; k <= hz; ++k)
        for (int j = -hy; j <= hy; ++j)
            for (int i = -hx; i <= hx; ++i) {
                int64_t a = preop[lin(cx + i, cy + j, cz + k, nx, ny)];
                int64_t c = intraop[lin(cx + dx + i, cy + dy + j, cz + dz + k, nx, ny)];
                si += a;
                sj += c;
                sii += a * a;
                sjj += c * c;
                sij += a * c;
            }
    int64_t vi = n * sii - si * si, vj = n * sjj - sj * sj, num = n * sij - si * sj;
    if (vi == 0 || vj == 0) return 0;
    double den2 = (double)vi * (double)vj;
    *ncc = (double)num / sqrt(den2);
    return 1;
}

int oracle_ncc_u16(const uint16_t *preop, const uint16_t *intraop, int nx, int ny, int nz, int b,
                   int cx, int cy, int cz, int dx, int dy, int dz, double *ncc)
{
    return oracle_ncc_u16_3(preop, intraop, nx, ny, nz, b, b, b, cx, cy, cz, dx, dy, dz, ncc);
}

/* Definition path (Sec. 3 NCC equation, read as Pearson): means first, then
 * the centred cross and squared sums, all in FP64.  Inputs widened from the
 * given element type.  Used for float32 intensities and as a check of the
 * integer path. */
static int pearson_generic(const void *preop, const void *intraop, int is_f32, int nx, int ny, int nz,
                           const int bl[3], int cx, int cy, int cz, int dx, int dy, int dz, double *ncc)
{
    if (!block_inside(nx, ny, nz, bl, cx, cy, cz)) return 0;
    if (!block_inside(nx, ny, nz, bl, (int64_t)cx + dx, (int64_t)cy + dy, (int64_t)cz + dz)) return 0;
    int hx = (bl[0] - 1) / 2, hy = (bl[1] - 1) / 2, hz = (bl[2] - 1) / 2;
    double n = (double)bl[0] * bl[1] * bl[2], mi = 0.0, mj = 0.0;
#define VAL(p, idx) (is_f32 ? (double)((const float *)(p))[idx] : (double)((const uint16_t *)(p))[idx])
    for (int k = -hz; k <= hz; ++k)
        for (int j = -hy; j <= hy; ++j)
            for (int i = -hx; i <= hx; ++i) {
                mi += VAL(preop, lin(cx + i, cy + j, cz + k, nx, ny));
                mj += VAL(intraop, lin(cx + dx + i, cy + dy + j, cz + dz + k, nx, ny));
            }
    mi /= n;
    mj /= n;
    double cov = 0.0, vi = 0.0, vj = 0.0;
    for (int k = -hz; k <= hz; ++k)
        for (int j = -hy; j <= hy; ++j)
            for (int i = -hx; i <= hx; ++i) {
                double a = VAL(preop, lin(cx + i, cy + j, cz + k, nx, ny)) - mi;
                double c = VAL(intraop, lin(cx + dx + i, cy + dy + j, cz + dz + k, nx, ny)) - mj;
                cov += a * c;
                vi += a * a;
                vj += c * c;
            }
#undef VAL
    if (vi == 0.0 || vj == 0.0) return 0;
    *ncc = cov / sqrt(vi * vj);
    return 1;
}

int oracle_pearson_u16_3(const uint16_t *preop, const uint16_t *intraop, int nx, int ny, int nz, int bx, int by,
                         int bz, int cx, int cy, int cz, int dx, int dy, int dz, double *ncc)
{
    const int bl[3] = {bx, by, bz};
    return pearson_generic(preop, intraop, 0, nx, ny, nz, bl, cx, cy, cz, dx, dy, dz, ncc);
}

int oracle_pearson_f32_3(const float *preop, const float *intraop, int nx, int ny, int nz, int bx, int by, int bz,
                         int cx, int cy, int cz, int dx, int dy, int dz, double *ncc)
{
    const int bl[3] = {bx, by, bz};
    return pearson_generic(preop, intraop, 1, nx, ny, nz, bl, cx, cy, cz, dx, dy, dz, ncc);
}

int oracle_pearson_u16(const uint16_t *preop, const uint16_t *intraop, int nx, int ny, int nz, int b,
                       int cx, int cy, int cz, int dx, int dy, int dz, double *ncc)
{
    return oracle_pearson_u16_3(preop, intraop, nx, ny, nz, b, b, b, cx, cy, cz, dx, dy, dz, ncc);
}

int oracle_pearson_f32(const float *preop, const float *intraop, int nx, int ny, int nz, int b,
                       int cx, int cy, int cz, int dx, int dy, int dz, double *ncc)
{
    return oracle_pearson_f32_3(preop, intraop, nx, ny, nz, b, b, b, cx, cy, cz, dx, dy, dz, ncc);
}

/* ---------------------------------------------------------------------
 * Exhaustive block matching (Sec. 3; the block-matching loop of Sec. 4.3):
 * for every block, score every shift of the search window and keep the
 * maximum.
 * ------------------------------------------------------------------- */

/* Is candidate (s, d) better than the current best (bs, bd)?  NCC
 * descending, then |d|^2 ascending, then (dz,dy,dx) lexicographic. */
static int better(double s, const int d[3], double bs, const int bd[3])
{
    if (s != bs) return s > bs;
    int64_t n1 = (int64_t)d[0] * d[0] + (int64_t)d[1] * d[1] + (int64_t)d[2] * d[2];
    int64_t n2 = (int64_t)bd[0] * bd[0] + (int64_t)bd[1] * bd[1] + (int64_t)bd[2] * bd[2];
    if (n1 != n2) return n1 < n2;
    if (d[2] != bd[2]) return d[2] < bd[2];
    if (d[1] != bd[1]) return d[1] < bd[1];
    return d[0] < bd[0];
}

static void match_generic(const void *preop, const void *intraop, int is_f32, int nx, int ny, int nz,
                          const int32_t *centers, int64_t n_blocks, const int32_t block[3], const int32_t radius[3],
                          int32_t *disp, double *ncc_out, uint8_t *valid)
{
    int bx = block[0], by = block[1], bz = block[2];
    int rx = radius[0], ry = radius[1], rz = radius[2];
#pragma omp parallel for schedule(dynamic, 1)
    for (int64_t blk = 0; blk < n_blocks; ++blk) {
        int cx = centers[3 * blk], cy = centers[3 * blk + 1], cz = centers[3 * blk + 2];
        int found = 0, best_d[3] = {0, 0, 0};
        double best = 0.0;
        for (int dz = -rz; dz <= rz; ++dz)
            for (int dy = -ry; dy <= ry; ++dy)
                for (int dx = -rx; dx <= rx; ++dx) {
                    double s;
                    int ok = is_f32 ? oracle_pearson_f32_3((const float *)preop, (const float *)intraop, nx, ny,
                                                           nz, bx, by, bz, cx, cy, cz, dx, dy, dz, &s)
                                    : oracle_ncc_u16_3((const uint16_t *)preop, (const uint16_t *)intraop, nx, ny,
                                                       nz, bx, by, bz, cx, cy, cz, dx, dy, dz, &s);
                    if (!ok) continue;
                    int d[3] = {dx, dy, dz};
                    if (!found || better(s, d, best, best_d)) {
                        found = 1;
                        best = s;
                        best_d[0] = dx;
                        best_d[1] = dy;
                        best_d[2] = dz;
                    }
                }
        disp[3 * blk + 0] = best_d[0];
        disp[3 * blk + 1] = best_d[1];
        disp[3 * blk + 2] = best_d[2];
        ncc_out[blk] = found ? best : NAN;
        valid[blk] = (uint8_t)found;
    }
}

/* uint16 intensities: exact integer sums, FP64 ratio (see oracle_ncc_u16);
 * block edges (bx, by, bz). */
void oracle_match_u16_3(const uint16_t *preop, const uint16_t *intraop, int nx, int ny, int nz,
                        const int32_t *centers, int64_t n_blocks, const int32_t block[3], const int32_t radius[3],
                        int32_t *disp, double *ncc, uint8_t *valid)
{
    match_generic(preop, intraop, 0, nx, ny, nz, centers, n_blocks, block, radius, disp, ncc, valid);
}

/* float32 intensities: FP64 two-pass Pearson (see pearson_generic). */
void oracle_match_f32_3(const float *preop, const float *intraop, int nx, int ny, int nz,
                        const int32_t *centers, int64_t n_blocks, const int32_t block[3], const int32_t radius[3],
                        int32_t *disp, double *ncc, uint8_t *valid)
{
    match_generic(preop, intraop, 1, nx, ny, nz, centers, n_blocks, block, radius, disp, ncc, valid);
}

void oracle_match_u16(const uint16_t *preop, const uint16_t *intraop, int nx, int ny, int nz,
                      const int32_t *centers, int64_t n_blocks, int b, const int32_t radius[3],
                      int32_t *disp, double *ncc, uint8_t *valid)
{
    const int32_t block[3] = {b, b, b};
    oracle_match_u16_3(preop, intraop, nx, ny, nz, centers, n_blocks, block, radius, disp, ncc, valid);
}

void oracle_match_f32(const float *preop, const float *intraop, int nx, int ny, int nz,
                      const int32_t *centers, int64_t n_blocks, int b, const int32_t radius[3],
                      int32_t *disp, double *ncc, uint8_t *valid)
{
    const int32_t block[3] = {b, b, b};
    oracle_match_f32_3(preop, intraop, nx, ny, nz, centers, n_blocks, block, radius, disp, ncc, valid);
}
