/*
 * Seeded synthetic proton pencil-beam dose-deposition matrices (input generator).
 *
 * The paper's matrices come from a clinical Monte Carlo engine and patient CT
 * (Sec. II-A, Table I) and are not available; this generator produces matrices
 * with the same structure: rows are voxels of a dose grid, columns are beam
 * spots on a lateral lattice seen in the beam's-eye view (Sec. II-A, Fig. 1),
 * most rows are empty and row lengths are strongly uneven (Sec. II-B, Fig. 2).
 *
 * Geometry.  Grid nx*ny*nz, beam along +z.  Row r = (iz*ny + iy)*nx + ix, voxel
 * centre (ix+0.5, iy+0.5, iz+0.5).  Spot j = b*sx + a sits at
 *   cx = nx/2 + (a - (sx-1)/2)*dx + shift_x,  cy = ny/2 + (b - (sy-1)/2)*dy + shift_y
 * and has a Bragg depth z_j = nz * U(0.4, 0.8), U the j-th splitmix64 output of
 * the beam seed.  Deposited value v = G * B with
 *   G = exp(-rho^2 / (2 sigma^2))               (lateral Gaussian)
 *   B = 0.3 + 0.7 (z/z_j)^4          z <= z_j  (entrance plateau, rise)
 *   B = exp(-(z - z_j)^2 / 2)        z >  z_j  (sharp distal falloff)
 * Entries with v >= tau are kept; columns inside a row are emitted ascending.
 *
 * This file holds input generation only: no decoding, no products, nothing of
 * the dose calculation itself.  Compile with -ffp-contract=off so that the
 * values do not depend on whether the host compiler fuses multiply-adds.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

typedef struct {
    int32_t nx, ny, nz;      /* voxel grid */
    int32_t sx, sy;          /* spot lattice */
    double dx, dy;           /* spot spacing in voxels */
    double sigma;            /* lateral Gaussian sigma in voxels */
    double tau;              /* truncation threshold (spot maximum is 1) */
    double shift_x, shift_y; /* setup-shift scenario: lateral shift of spot centres */
    uint64_t seed;           /* beam seed (Bragg depths) */
} pb_params;

static const uint64_t GOLDEN = 0x9E3779B97F4A7C15ull;

/* splitmix64 output function (Steele, Lea, Flood, "Fast splittable
 * pseudorandom number generators", OOPSLA 2014). */
static uint64_t sm64_mix(uint64_t z) {
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

/* k-th (0-based) output of a splitmix64 stream seeded with `seed`. */
uint64_t pb_splitmix64_at(uint64_t seed, uint64_t k) {
    return sm64_mix(seed + (k + 1) * GOLDEN);
}

/* n uniform FP32 values in [0,1): top 24 bits of the stream, exact in FP32. */
void pb_uniform_f32(uint64_t seed, uint64_t n, float* out) {
    for (uint64_t k = 0; k < n; ++k)
        out[k] = (float)(pb_splitmix64_at(seed, k) >> 40) * (1.0f / 16777216.0f);
}

/* n uniform FP64 values in [0,1): top 53 bits of the stream, exact in FP64. */
void pb_uniform_f64(uint64_t seed, uint64_t n, double* out) {
    for (uint64_t k = 0; k < n; ++k)
        out[k] = (double)(pb_splitmix64_at(seed, k) >> 11) * (1.0 / 9007199254740992.0);
}

static double bragg_depth(const pb_params* p, int32_t j) {
    double u = (double)(pb_splitmix64_at(p->seed, (uint64_t)j) >> 11) * (1.0 / 9007199254740992.0);
    return (double)p->nz * (0.4 + 0.4 * u);
}

static double depth_profile(double z, double zj) {
    if (z <= zj) {
        double t = z / zj;
        double t2 = t * t;
        return 0.3 + 0.7 * (t2 * t2);
    }
    double dz = z - zj;
    return exp(-0.5 * dz * dz);
}

/* Table B[j*nz + iz] of the depth profile at voxel centres. */
static double* depth_table(const pb_params* p) {
    int32_t ns = p->sx * p->sy;
    double* t = (double*)malloc(sizeof(double) * (size_t)ns * (size_t)p->nz);
    if (!t) return NULL;
    for (int32_t j = 0; j < ns; ++j) {
        double zj = bragg_depth(p, j);
        for (int32_t iz = 0; iz < p->nz; ++iz)
            t[(size_t)j * p->nz + iz] = depth_profile(iz + 0.5, zj);
    }
    return t;
}

/* Candidate spots of one lateral position, ascending j, with their G. */
static int32_t lateral_candidates(const pb_params* p, int32_t ix, int32_t iy,
                                  int32_t* cj, double* cg) {
    double x = ix + 0.5, y = iy + 0.5;
    double r2max = -2.0 * p->sigma * p->sigma * log(p->tau);
    if (!(r2max > 0.0)) return 0;
    double r = sqrt(r2max);
    double x0 = 0.5 * p->nx - 0.5 * (p->sx - 1) * p->dx + p->shift_x;
    double y0 = 0.5 * p->ny - 0.5 * (p->sy - 1) * p->dy + p->shift_y;
    int32_t a0 = (int32_t)ceil((x - r - x0) / p->dx), a1 = (int32_t)floor((x + r - x0) / p->dx);
    int32_t b0 = (int32_t)ceil((y - r - y0) / p->dy), b1 = (int32_t)floor((y + r - y0) / p->dy);
    if (a0 < 0) a0 = 0;
    if (b0 < 0) b0 = 0;
    if (a1 > p->sx - 1) a1 = p->sx - 1;
    if (b1 > p->sy - 1) b1 = p->sy - 1;
    int32_t n = 0;
    double inv2s2 = 1.0 / (2.0 * p->sigma * p->sigma);
    for (int32_t b = b0; b <= b1; ++b) {
        double ey = y - (y0 + b * p->dy);
        for (int32_t a = a0; a <= a1; ++a) {
            double ex = x - (x0 + a * p->dx);
            double rho2 = ex * ex + ey * ey;
            if (rho2 > r2max) continue;
            double g = exp(-rho2 * inv2s2);
            if (g < p->tau) continue;
            cj[n] = b * p->sx + a;
            cg[n] = g;
            ++n;
        }
    }
    return n;
}

static int32_t max_candidates(const pb_params* p) {
    double r = sqrt(fmax(0.0, -2.0 * p->sigma * p->sigma * log(p->tau)));
    int32_t na = (int32_t)(2.0 * r / p->dx) + 3, nb = (int32_t)(2.0 * r / p->dy) + 3;
    if (na > p->sx) na = p->sx;
    if (nb > p->sy) nb = p->sy;
    return na * nb;
}

static int check_params(const pb_params* p) {
    if (p->nx <= 0 || p->ny <= 0 || p->nz <= 0 || p->sx <= 0 || p->sy <= 0) return -1;
    if (!(p->dx > 0) || !(p->dy > 0) || !(p->sigma > 0) || !(p->tau > 0) || !(p->tau < 1)) return -1;
    return 0;
}

/* Row lengths (row_len[nr], may be NULL) and total nnz; -1 on bad params or OOM. */
int64_t pb_count(const pb_params* p, uint32_t* row_len) {
    if (check_params(p)) return -1;
    double* bt = depth_table(p);
    if (!bt) return -1;
    int64_t nr = (int64_t)p->nx * p->ny * p->nz;
    if (row_len) memset(row_len, 0, sizeof(uint32_t) * (size_t)nr);
    int32_t mc = max_candidates(p);
    int64_t total = 0;
    int failed = 0;
#pragma omp parallel reduction(+ : total)
    {
        int32_t* cj = (int32_t*)malloc(sizeof(int32_t) * (size_t)mc);
        double* cg = (double*)malloc(sizeof(double) * (size_t)mc);
        if (!cj || !cg) {
#pragma omp atomic write
            failed = 1;
        } else {
#pragma omp for schedule(dynamic, 4)
            for (int32_t iy = 0; iy < p->ny; ++iy)
                for (int32_t ix = 0; ix < p->nx; ++ix) {
                    int32_t nc = lateral_candidates(p, ix, iy, cj, cg);
                    if (nc == 0) continue;
                    for (int32_t iz = 0; iz < p->nz; ++iz) {
                        uint32_t len = 0;
                        for (int32_t c = 0; c < nc; ++c)
                            if (cg[c] * bt[(size_t)cj[c] * p->nz + iz] >= p->tau) ++len;
                        if (row_len) row_len[((int64_t)iz * p->ny + iy) * p->nx + ix] = len;
                        total += len;
                    }
                }
        }
        free(cj);
        free(cg);
    }
    free(bt);
    return failed ? -1 : total;
}

/* Fill col[] and val[] given row_ptr[nr+1] from pb_count's row lengths. 0 on success. */
int pb_fill(const pb_params* p, const uint32_t* row_ptr, uint32_t* col, double* val) {
    if (check_params(p)) return -1;
    double* bt = depth_table(p);
    if (!bt) return -1;
    int32_t mc = max_candidates(p);
    int failed = 0;
#pragma omp parallel
    {
        int32_t* cj = (int32_t*)malloc(sizeof(int32_t) * (size_t)mc);
        double* cg = (double*)malloc(sizeof(double) * (size_t)mc);
        if (!cj || !cg) {
#pragma omp atomic write
            failed = 1;
        } else {
#pragma omp for schedule(dynamic, 4)
            for (int32_t iy = 0; iy < p->ny; ++iy)
                for (int32_t ix = 0; ix < p->nx; ++ix) {
                    int32_t nc = lateral_candidates(p, ix, iy, cj, cg);
                    if (nc == 0) continue;
                    for (int32_t iz = 0; iz < p->nz; ++iz) {
                        int64_t r = ((int64_t)iz * p->ny + iy) * p->nx + ix;
                        uint64_t k = row_ptr[r], kend = row_ptr[r + 1];
                        for (int32_t c = 0; c < nc; ++c) {
                            double v = cg[c] * bt[(size_t)cj[c] * p->nz + iz];
                            if (v >= p->tau) {
                                if (k >= kend) { /* row_ptr does not match pb_count */
#pragma omp atomic write
                                    failed = 1;
                                    break;
                                }
                                col[k] = (uint32_t)cj[c];
                                val[k] = v;
                                ++k;
                            }
                        }
                    }
                }
        }
        free(cj);
        free(cg);
    }
    free(bt);
    return failed ? -1 : 0;
}
