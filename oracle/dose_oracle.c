/*
 * FP64 CPU oracle for the dose calculation -- TEST INFRASTRUCTURE ONLY.
 *
 * Plain, slow, obviously correct loops.  Only the tests, the smoke check and the
 * benchmark's CPU-baseline leg use this file; the CUDA library never links it
 * and shares no code with it.
 *
 * What it computes (paper: Sec. II-A "dose = dose-deposition matrix times spot
 * weights"; Sec. III, Listing 1: one output per row equal to the row's dot
 * product; Sec. II-C: CSR layout):
 *   decode   a_k  = dec(fmt, stored_k)                      (exact in FP64)
 *   spmv     d_i  = sum_{k=row_ptr[i]}^{row_ptr[i+1]-1} a_k x[col_k]   (ascending k)
 *   adjoint  g_j  = sum_i a_ij r_i                          (row-order scatter)
 *   spmm     D[i,v] = sum_k a_k X[col_k, v]
 *   objective f = sum_i w_i (d_i - p_i)^2,  r_i = 2 w_i (d_i - p_i)
 *   pg step  x <- max(0, x - eta * A^T r(Ax))
 * Empty rows produce d_i = 0 (the definition d = A x; the paper's listing
 * skips the store but its byte model in Sec. V counts a write for every row).
 *
 * Stored formats (the paper fixes 16-bit storage, Sec. II-D, but not the
 * format; these are the library's formats, each decoded from its definition):
 *   U16_SCALE : unsigned 16-bit fixed point, one FP32 scale s per matrix, a = s*q
 *   BF16      : bfloat16 (1 sign, 8 exponent, 7 fraction bits), a = bf16 value
 *   FP8E4M3   : OCP FP8 E4M3 (bias 7, no infinities, S.1111.111 = NaN,
 *               subnormals m/8 * 2^-6) with one FP32 scale per row, a = s_r*e4m3(q)
 *   F16       : IEEE 754 binary16 (1 sign, 5 exponent with bias 15, 10 fraction
 *               bits, subnormals m/1024 * 2^-14), a = half value (the paper's
 *               "Half" storage, Sec. IV)
 *   F32       : IEEE 754 binary32, a = float value (the paper's "Single"
 *               configuration, Sec. IV); encoded by C's double-to-float
 *               conversion (round to nearest, ties to even)
 * Encoders follow the readings: u16 s = fl32(max v / 65535), q = RNE(v/s)
 * clamped to [0,65535]; BF16 = round-to-nearest-even of the FP64 value; FP8
 * s_r = fl32(row max / 448) (1 for empty or all-zero rows), q = nearest E4M3
 * code of v/s_r (ties to even code), saturating at 448.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

/* ---------------------------------------------------------------- formats */

/* Value of an FP8 E4M3 code from its bit fields (OCP 8-bit FP spec). */
double oracle_fp8_e4m3_value(uint8_t code) {
    int sign = (code >> 7) & 1;
    int e = (code >> 3) & 0xF;
    int m = code & 0x7;
    double v;
    if (e == 0xF && m == 0x7) return NAN;
    if (e == 0)
        v = ldexp((double)m / 8.0, -6);            /* subnormal */
    else
        v = ldexp(1.0 + (double)m / 8.0, e - 7);   /* normal */
    return sign ? -v : v;
}

/* Value of a bfloat16 bit pattern: the upper half of an IEEE binary32. */
double oracle_bf16_value(uint16_t bits) {
    uint32_t u = (uint32_t)bits << 16;
    float f;
    memcpy(&f, &u, sizeof f);
    return (double)f;
}

/* Value of an IEEE binary16 bit pattern from its fields. */
double oracle_f16_value(uint16_t bits) {
    int sign = (bits >> 15) & 1;
    int e = (bits >> 10) & 0x1F;
    int m = bits & 0x3FF;
    double v;
    if (e == 0x1F) return m ? NAN : (sign ? -INFINITY : INFINITY);
    if (e == 0)
        v = ldexp((double)m / 1024.0, -14);          /* subnormal */
    else
        v = ldexp(1.0 + (double)m / 1024.0, e - 15); /* normal */
    return sign ? -v : v;
}

/* Round-to-nearest-even of v to binary16 (11 significant bits; quantum 2^-24
 * below 2^-14; magnitudes from 65520 up round to infinity). */
uint16_t oracle_f16_round(double v) {
    if (v != v) return 0x7E00;
    double a = fabs(v);
    uint16_t sign = (v < 0 || (v == 0 && signbit(v))) ? 0x8000 : 0;
    double q;
    if (a == 0) {
        q = 0;
    } else if (a < ldexp(1.0, -14)) {
        q = nearbyint(ldexp(a, 24)) * ldexp(1.0, -24);   /* subnormal quantum 2^-24 */
    } else {
        int ex;
        double m = frexp(a, &ex);                         /* a = m 2^ex, m in [0.5,1) */
        q = ldexp(nearbyint(ldexp(m, 11)), ex - 11);       /* 11 significant bits */
    }
    if (q >= 65536.0) return sign | 0x7C00;                /* overflow: infinity */
    if (q < ldexp(1.0, -14)) return sign | (uint16_t)(q * 16777216.0); /* subnormal or zero */
    int ex;
    double m = frexp(q, &ex);                              /* q = m 2^ex, m in [0.5,1) */
    uint16_t e = (uint16_t)(ex - 1 + 15);
    uint16_t f = (uint16_t)((m * 2.0 - 1.0) * 1024.0);
    return sign | (uint16_t)(e << 10) | f;
}

/* Nearest E4M3 code to a non-negative finite t, searched over every finite
 * non-negative code; ties go to the code with an even mantissa LSB; values
 * beyond 448 saturate to 448.  Returns the code. */
uint8_t oracle_fp8_e4m3_nearest(double t) {
    int best = 0;
    double bestd = INFINITY;
    for (int c = 0; c < 0x7F; ++c) { /* 0x7F is NaN */
        double v = oracle_fp8_e4m3_value((uint8_t)c);
        double dd = fabs(v - t);
        if (dd < bestd || (dd == bestd && (c & 1) == 0 && (best & 1) == 1)) {
            bestd = dd;
            best = c;
        }
    }
    return (uint8_t)best;
}

/* Round-to-nearest-even of v to bfloat16 (8 significant bits, binary32 range). */
uint16_t oracle_bf16_round(double v) {
    if (v != v) return 0x7FC0;
    double a = fabs(v);
    uint16_t sign = (v < 0 || (v == 0 && signbit(v))) ? 0x8000 : 0;
    double q;
    if (a == 0) {
        q = 0;
    } else if (a < ldexp(1.0, -126)) {
        q = nearbyint(ldexp(a, 133)) * ldexp(1.0, -133);   /* subnormal quantum 2^-133 */
    } else {
        int ex;
        double m = frexp(a, &ex);                          /* a = m 2^ex, m in [0.5,1) */
        q = ldexp(nearbyint(ldexp(m, 8)), ex - 8);          /* 8 significant bits */
    }
    float f = (float)q; /* exact when q is finite in binary32 */
    if (q > 3.3895313892515355e38) f = INFINITY;
    uint32_t u;
    memcpy(&u, &f, sizeof u);
    return (uint16_t)(sign | ((u >> 16) & 0x7FFF));
}

/* U16 fixed point with one scale: returns 0, or -1 for a negative/NaN value. */
int oracle_encode_u16(uint64_t nnz, const double* v, float* scale, uint16_t* q) {
    double vmax = 0.0;
    for (uint64_t k = 0; k < nnz; ++k) {
        if (!(v[k] >= 0.0)) return -1;
        if (v[k] > vmax) vmax = v[k];
    }
    float s = vmax > 0.0 ? (float)(vmax / 65535.0) : 1.0f;
    if (!(s > 0.0f)) s = 1.0f; /* vmax so small that the scale underflows */
    *scale = s;
    for (uint64_t k = 0; k < nnz; ++k) {
        double t = nearbyint(v[k] / (double)s);
        if (t > 65535.0) t = 65535.0;
        q[k] = (uint16_t)t;
    }
    return 0;
}

int oracle_encode_bf16(uint64_t nnz, const double* v, uint16_t* out) {
    for (uint64_t k = 0; k < nnz; ++k) out[k] = oracle_bf16_round(v[k]);
    return 0;
}

int oracle_encode_f32(uint64_t nnz, const double* v, float* out) {
    for (uint64_t k = 0; k < nnz; ++k) out[k] = (float)v[k];
    return 0;
}

void oracle_decode_f32(uint64_t nnz, const float* bits, double* a) {
    for (uint64_t k = 0; k < nnz; ++k) a[k] = (double)bits[k];
}

int oracle_encode_f16(uint64_t nnz, const double* v, uint16_t* out) {
    for (uint64_t k = 0; k < nnz; ++k) out[k] = oracle_f16_round(v[k]);
    return 0;
}

/* FP8 E4M3 with one FP32 scale per row: returns 0, or -1 for a negative/NaN value. */
int oracle_encode_fp8_rowscale(uint32_t nrows, const uint32_t* row_ptr, const double* v,
                               float* row_scale, uint8_t* q) {
    for (uint32_t i = 0; i < nrows; ++i) {
        double rmax = 0.0;
        for (uint32_t k = row_ptr[i]; k < row_ptr[i + 1]; ++k) {
            if (!(v[k] >= 0.0)) return -1;
            if (v[k] > rmax) rmax = v[k];
        }
        float s = rmax > 0.0 ? (float)(rmax / 448.0) : 1.0f;
        if (!(s > 0.0f)) s = 1.0f;
        row_scale[i] = s;
        for (uint32_t k = row_ptr[i]; k < row_ptr[i + 1]; ++k)
            q[k] = oracle_fp8_e4m3_nearest(v[k] / (double)s);
    }
    return 0;
}

void oracle_decode_u16(uint64_t nnz, const uint16_t* q, float scale, double* a) {
    for (uint64_t k = 0; k < nnz; ++k) a[k] = (double)scale * (double)q[k];
}

void oracle_decode_bf16(uint64_t nnz, const uint16_t* bits, double* a) {
    for (uint64_t k = 0; k < nnz; ++k) a[k] = oracle_bf16_value(bits[k]);
}

void oracle_decode_f16(uint64_t nnz, const uint16_t* bits, double* a) {
    for (uint64_t k = 0; k < nnz; ++k) a[k] = oracle_f16_value(bits[k]);
}

void oracle_decode_fp8_rowscale(uint32_t nrows, const uint32_t* row_ptr, const uint8_t* q,
                                const float* row_scale, double* a) {
    for (uint32_t i = 0; i < nrows; ++i)
        for (uint32_t k = row_ptr[i]; k < row_ptr[i + 1]; ++k)
            a[k] = (double)row_scale[i] * oracle_fp8_e4m3_value(q[k]);
}

/* ------------------------------------------------------------- products */

/* d = A x; rows in order, entries of a row in ascending storage order. */
void oracle_spmv(uint32_t nrows, const uint32_t* row_ptr, const uint32_t* col, const double* a,
                 const double* x, double* d) {
    for (uint32_t i = 0; i < nrows; ++i) {
        double s = 0.0;
        for (uint32_t k = row_ptr[i]; k < row_ptr[i + 1]; ++k) s += a[k] * x[col[k]];
        d[i] = s;
    }
}

/* Only the listed rows of d = A x (for sampled checks of very large matrices). */
void oracle_spmv_rows(uint64_t nsel, const uint32_t* rows, const uint32_t* row_ptr,
                      const uint32_t* col, const double* a, const double* x, double* d) {
    for (uint64_t t = 0; t < nsel; ++t) {
        uint32_t i = rows[t];
        double s = 0.0;
        for (uint32_t k = row_ptr[i]; k < row_ptr[i + 1]; ++k) s += a[k] * x[col[k]];
        d[t] = s;
    }
}

/* D = A X with X[ncols][nvec], D[nrows][nvec] row-major. */
void oracle_spmm(uint32_t nrows, uint32_t nvec, const uint32_t* row_ptr, const uint32_t* col,
                 const double* a, const double* X, double* D) {
    for (uint32_t i = 0; i < nrows; ++i)
        for (uint32_t v = 0; v < nvec; ++v) {
            double s = 0.0;
            for (uint32_t k = row_ptr[i]; k < row_ptr[i + 1]; ++k)
                s += a[k] * X[(uint64_t)col[k] * nvec + v];
            D[(uint64_t)i * nvec + v] = s;
        }
}

/* g = A^T r by scattering each row's entries, rows in order. */
void oracle_spmv_t(uint32_t nrows, uint32_t ncols, const uint32_t* row_ptr, const uint32_t* col,
                   const double* a, const double* r, double* g) {
    for (uint32_t j = 0; j < ncols; ++j) g[j] = 0.0;
    for (uint32_t i = 0; i < nrows; ++i)
        for (uint32_t k = row_ptr[i]; k < row_ptr[i + 1]; ++k) g[col[k]] += a[k] * r[i];
}

/* |A|^T |r| : the scale of the adjoint's rounding error per column. */
void oracle_abs_spmv_t(uint32_t nrows, uint32_t ncols, const uint32_t* row_ptr,
                       const uint32_t* col, const double* a, const double* r, double* g) {
    for (uint32_t j = 0; j < ncols; ++j) g[j] = 0.0;
    for (uint32_t i = 0; i < nrows; ++i)
        for (uint32_t k = row_ptr[i]; k < row_ptr[i + 1]; ++k) g[col[k]] += fabs(a[k]) * fabs(r[i]);
}

/* f = sum w_i (d_i - p_i)^2 and r_i = 2 w_i (d_i - p_i) (r may be NULL). */
double oracle_objective(uint32_t n, const double* d, const double* p, const double* w, double* r) {
    double f = 0.0;
    for (uint32_t i = 0; i < n; ++i) {
        double e = d[i] - p[i];
        f += w[i] * e * e;
        if (r) r[i] = 2.0 * w[i] * e;
    }
    return f;
}

/* f(x) and grad f(x) = A^T (2 W (A x - p)); work needs 2*nrows doubles. */
double oracle_fgrad(uint32_t nrows, uint32_t ncols, const uint32_t* row_ptr, const uint32_t* col,
                    const double* a, const double* x, const double* p, const double* w,
                    double* grad, double* work) {
    double* d = work;
    double* r = work + nrows;
    oracle_spmv(nrows, row_ptr, col, a, x, d);
    double f = oracle_objective(nrows, d, p, w, r);
    oracle_spmv_t(nrows, ncols, row_ptr, col, a, r, grad);
    return f;
}

/* Projected gradient: iters steps of x <- max(0, x - eta grad f(x)).  f_hist[k]
 * is f at the start of step k (f(x_k)); x is updated in place.  Returns 0, -1 on OOM. */
int oracle_pg(uint32_t nrows, uint32_t ncols, const uint32_t* row_ptr, const uint32_t* col,
              const double* a, const double* p, const double* w, double eta, uint32_t iters,
              double* x, double* f_hist) {
    double* work = (double*)malloc(sizeof(double) * (2 * (size_t)nrows + ncols));
    if (!work) return -1;
    double* grad = work + 2 * (size_t)nrows;
    for (uint32_t it = 0; it < iters; ++it) {
        f_hist[it] = oracle_fgrad(nrows, ncols, row_ptr, col, a, x, p, w, grad, work);
        for (uint32_t j = 0; j < ncols; ++j) {
            double t = x[j] - eta * grad[j];
            x[j] = t > 0.0 ? t : 0.0;
        }
    }
    free(work);
    return 0;
}

/* Robust quadratic objective over S dose scenarios (Sec. I: doses under several
 * realisations of the uncertainties in every optimisation iteration), from the
 * per-scenario values f_s = f(A_s x) and gradients g_s = grad f(A_s x) (g row s
 * of an S x ncols array):
 *   mode 0, expected:   F = sum_s prob_s f_s,  G = sum_s prob_s g_s;
 *   mode 1, worst case: s* = the first s with the largest f_s, F = f_s*, G = g_s*
 *                       (a subgradient of max_s f_s).
 * Returns F and writes G; returns s* through *arg (mode 0: -1). */
double oracle_robust_combine(uint32_t S, uint32_t ncols, int mode, const double* prob, const double* f_s,
                             const double* g_s, double* G, int32_t* arg) {
    if (mode == 0) {
        double F = 0.0;
        for (uint32_t s = 0; s < S; ++s) F += prob[s] * f_s[s];
        for (uint32_t j = 0; j < ncols; ++j) {
            double t = 0.0;
            for (uint32_t s = 0; s < S; ++s) t += prob[s] * g_s[(size_t)s * ncols + j];
            G[j] = t;
        }
        *arg = -1;
        return F;
    }
    uint32_t best = 0;
    for (uint32_t s = 1; s < S; ++s)
        if (f_s[s] > f_s[best]) best = s;
    for (uint32_t j = 0; j < ncols; ++j) G[j] = g_s[(size_t)best * ncols + j];
    *arg = (int32_t)best;
    return f_s[best];
}

/* Largest eigenvalue of A^T A by `iters` power iterations from the all-ones vector. */
double oracle_norm2_sq(uint32_t nrows, uint32_t ncols, const uint32_t* row_ptr,
                       const uint32_t* col, const double* a, uint32_t iters) {
    double* v = (double*)malloc(sizeof(double) * (2 * (size_t)ncols + nrows));
    if (!v) return -1.0;
    double* u = v + ncols;
    double* t = u + ncols;
    for (uint32_t j = 0; j < ncols; ++j) v[j] = 1.0;
    double lam = 0.0;
    for (uint32_t it = 0; it < iters; ++it) {
        double nv = 0.0;
        for (uint32_t j = 0; j < ncols; ++j) nv += v[j] * v[j];
        nv = sqrt(nv);
        if (nv == 0.0) break;
        for (uint32_t j = 0; j < ncols; ++j) v[j] /= nv;
        oracle_spmv(nrows, row_ptr, col, a, v, t);
        oracle_spmv_t(nrows, ncols, row_ptr, col, a, t, u);
        lam = 0.0;
        for (uint32_t j = 0; j < ncols; ++j) lam += v[j] * u[j]; /* Rayleigh quotient */
        memcpy(v, u, sizeof(double) * ncols);
    }
    free(v);
    return lam;
}
