/* A C client of include/dose.h, compiled by gcc against the header and linked
 * to libdose.so (test_c_client.py builds and runs it; no GPU is needed).
 *
 * It pins the header itself:
 *   - prints the size and field offsets of the ABI structs, which the Python
 *     test compares with the binding's ctypes declarations;
 *   - calls the host-only entry points: dose_version, dose_encode_host (U16
 *     codes of a tiny matrix, checked by value), and dose_create_matrix with
 *     descriptors that the library must reject on the host before touching a
 *     device (each must return DOSE_ERR_INVALID_ARG with a message from
 *     dose_last_error), and the NULL-tolerant calls.
 * Exit status 0 means every check passed; each failure prints a line. */
#define _POSIX_C_SOURCE 200809L /* mkstemp, close */
#include <stddef.h>
#include <stdint.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>
#include <unistd.h>

#include "dose.h"

static int failures = 0;

#define CHECK(cond, what)                                 \
    do {                                                  \
        if (!(cond)) {                                    \
            printf("FAIL %s (line %d)\n", what, __LINE__); \
            ++failures;                                   \
        }                                                 \
    } while (0)

#define LAYOUT(T, f) printf("offset %s.%s %zu\n", #T, #f, offsetof(T, f))

static void print_layouts(void) {
    printf("sizeof dose_csr_desc %zu\n", sizeof(dose_csr_desc));
    LAYOUT(dose_csr_desc, nrows);
    LAYOUT(dose_csr_desc, ncols);
    LAYOUT(dose_csr_desc, nnz);
    LAYOUT(dose_csr_desc, row_ptr);
    LAYOUT(dose_csr_desc, col_idx);
    LAYOUT(dose_csr_desc, fmt);
    LAYOUT(dose_csr_desc, values);
    LAYOUT(dose_csr_desc, scales);
    LAYOUT(dose_csr_desc, values_f64);
    LAYOUT(dose_csr_desc, on_device);
    printf("sizeof dose_tuning %zu\n", sizeof(dose_tuning));
    LAYOUT(dose_tuning, tile_nnz);
    LAYOUT(dose_tuning, l2_prefetch);
    LAYOUT(dose_tuning, adj_tile_nnz);
    LAYOUT(dose_tuning, adj_l2_prefetch);
    LAYOUT(dose_tuning, row_order);
    LAYOUT(dose_tuning, sell_sigma);
    LAYOUT(dose_tuning, adj_layout);
    LAYOUT(dose_tuning, rg_warps);
    LAYOUT(dose_tuning, rg_l2_prefetch);
    LAYOUT(dose_tuning, fwd_layout);
    printf("sizeof dose_info %zu\n", sizeof(dose_info));
    LAYOUT(dose_info, nnz);
    LAYOUT(dose_info, lanes_hist);
    LAYOUT(dose_info, device_bytes);
    LAYOUT(dose_info, fused_bytes);
    LAYOUT(dose_info, sell_entries);
    LAYOUT(dose_info, scale);
    LAYOUT(dose_info, tuning);
    LAYOUT(dose_info, adj_layout_fused);
    LAYOUT(dose_info, rg_groups);
    LAYOUT(dose_info, rg_union_entries);
    LAYOUT(dose_info, rg_window);
    LAYOUT(dose_info, rg_index_bytes);
    LAYOUT(dose_info, fingerprint);
    LAYOUT(dose_info, spmv_layout);
    LAYOUT(dose_info, rg_spmv_bytes);
}

/* create must refuse desc on the host: DOSE_ERR_INVALID_ARG, a message, no handle */
static void expect_rejected(const dose_csr_desc* desc, unsigned flags, const dose_tuning* t, const char* what) {
    dose_matrix* A = (dose_matrix*)0x1;
    const dose_status st = dose_create_matrix(desc, flags, t, NULL, &A);
    CHECK(st == DOSE_ERR_INVALID_ARG, what);
    CHECK(A == NULL, "handle cleared on failure");
    const char* msg = dose_last_error();
    CHECK(msg != NULL && msg[0] != '\0', "error message set");
    printf("rejected %s: %s\n", what, msg ? msg : "(null)");
}

int main(void) {
    print_layouts();

    const char* v = dose_version();
    CHECK(v != NULL && strncmp(v, "libdose", 7) == 0, "dose_version");

    /* a 3 x 4 matrix: rows {0: (0, 1.0), (2, 0.5)}, {1: empty}, {2: (3, 0.25)} */
    const uint32_t row_ptr[4] = {0, 2, 2, 3};
    const uint32_t col[3] = {0, 2, 3};
    const double val[3] = {1.0, 0.5, 0.25};
    uint16_t codes[3] = {0, 0, 0};
    float scale = 0.f;
    CHECK(dose_encode_host(DOSE_FMT_U16_SCALE, 3, row_ptr, 3, val, codes, &scale) == DOSE_OK, "encode u16");
    /* s = fl32(max / 65535), q = nearest code of v / s */
    CHECK(scale == (float)(1.0 / 65535.0), "u16 scale");
    CHECK(codes[0] == 65535 && codes[1] == 32768 && codes[2] == 16384, "u16 codes");
    CHECK(dose_encode_host(DOSE_FMT_U16_SCALE, 3, row_ptr, 3, val, codes, NULL) == DOSE_ERR_INVALID_ARG,
          "encode needs scales");

    dose_csr_desc d;
    memset(&d, 0, sizeof d);
    d.nrows = 3;
    d.ncols = 4;
    d.nnz = 3;
    d.row_ptr = row_ptr;
    d.col_idx = col;
    d.fmt = DOSE_FMT_U16_SCALE;
    d.values_f64 = val;
    d.on_device = 0;

    dose_csr_desc bad = d;
    const uint32_t rp_start[4] = {1, 2, 2, 3};
    bad.row_ptr = rp_start;
    expect_rejected(&bad, 0, NULL, "row_ptr[0] != 0");
    bad = d;
    const uint32_t rp_back[4] = {0, 2, 1, 3};
    bad.row_ptr = rp_back;
    expect_rejected(&bad, 0, NULL, "decreasing row_ptr");
    bad = d;
    bad.nnz = 2;
    expect_rejected(&bad, 0, NULL, "row_ptr[nrows] != nnz");
    bad = d;
    const uint32_t col_out[3] = {0, 2, 4};
    bad.col_idx = col_out;
    expect_rejected(&bad, 0, NULL, "column >= ncols");
    bad = d;
    const uint32_t rp_dup[4] = {0, 2, 2, 3};
    const uint32_t col_dup[3] = {2, 2, 3};
    bad.row_ptr = rp_dup;
    bad.col_idx = col_dup;
    expect_rejected(&bad, 0, NULL, "duplicate column in a row");
    bad = d;
    bad.fmt = (dose_format)9;
    expect_rejected(&bad, 0, NULL, "unknown format");
    bad = d;
    bad.values_f64 = NULL;
    expect_rejected(&bad, 0, NULL, "no values");
    bad = d;
    bad.row_ptr = NULL;
    expect_rejected(&bad, 0, NULL, "null row_ptr");
    expect_rejected(&d, 0x80u, NULL, "unknown flag");
    bad = d;
    bad.ncols = 70000;
    expect_rejected(&bad, DOSE_CREATE_U16_INDEX, NULL, "16-bit indices with ncols > 65536");
    dose_tuning t;
    memset(&t, 0, sizeof t);
    t.tile_nnz = 100;
    expect_rejected(&d, 0, &t, "tile_nnz below range");
    memset(&t, 0, sizeof t);
    t.adj_layout = 3;
    expect_rejected(&d, 0, &t, "adj_layout out of range");
    memset(&t, 0, sizeof t);
    t.rg_warps = 16;
    expect_rejected(&d, 0, &t, "rg_warps out of range");
    memset(&t, 0, sizeof t);
    t.fwd_layout = 3;
    expect_rejected(&d, 0, &t, "fwd_layout out of range");
    CHECK(dose_create_matrix(NULL, 0, NULL, NULL, NULL) == DOSE_ERR_INVALID_ARG, "null desc");

    {
        /* host-only calls of the autotuner: plan of no matrices, a fingerprint, a cache round trip */
        int layout = 7, launches = 7;
        CHECK(dose_spmv_batched_plan(NULL, 0, 16, &layout, &launches) == DOSE_OK && layout == 0 && launches == 0,
              "batched plan of no matrices");
        uint64_t fp1 = 0, fp2 = 0;
        CHECK(dose_fingerprint_host(&d, 0, &fp1) == DOSE_OK && fp1 != 0, "fingerprint");
        CHECK(dose_fingerprint_host(&d, DOSE_CREATE_U16_INDEX, &fp2) == DOSE_OK && fp2 != fp1,
              "fingerprint depends on the flags");
        char path[] = "/tmp/dose_c_client_cache_XXXXXX";
        int fd = mkstemp(path);
        CHECK(fd >= 0, "temporary cache file");
        if (fd >= 0) {
            close(fd);
            remove(path); /* a missing file reads as an empty cache */
            dose_tuning in, out;
            memset(&in, 0, sizeof in);
            in.tile_nnz = 4096;
            in.rg_tile_union = 3072;
            in.fwd_layout = 1;
            double ms[3] = {0.1, 0.2, 0.3}, got_ms[3] = {0, 0, 0};
            int found = 1;
            CHECK(dose_autotune_cache_lookup(path, "GPU", fp1, 3, &out, got_ms, &found) == DOSE_OK && !found,
                  "lookup in a missing cache");
            CHECK(dose_autotune_cache_store(path, "GPU", fp1, 3, &in, ms) == DOSE_OK, "cache store");
            CHECK(dose_autotune_cache_lookup(path, "GPU", fp1, 3, &out, got_ms, &found) == DOSE_OK && found &&
                      out.tile_nnz == 4096 && out.rg_tile_union == 3072 && out.fwd_layout == 1 && got_ms[2] == 0.3,
                  "cache round trip");
            CHECK(dose_autotune_cache_lookup(path, "GPU", fp2, 3, &out, got_ms, &found) == DOSE_OK && !found,
                  "cache miss on another fingerprint");
            remove(path);
        }
    }
    CHECK(dose_destroy(NULL) == DOSE_OK, "destroy NULL");
    CHECK(dose_destroy_scenarios(NULL) == DOSE_OK, "destroy_scenarios NULL");
    dose_info info;
    CHECK(dose_matrix_info(NULL, &info) == DOSE_ERR_INVALID_ARG, "info of NULL");
    CHECK(dose_spmv(NULL, NULL, NULL, NULL) == DOSE_ERR_INVALID_ARG, "spmv of NULL");
    CHECK(dose_adjoint_noalloc(1, 4, 0, NULL, NULL, (dose_format)9, NULL, NULL, 1.f, NULL, NULL, NULL) ==
              DOSE_ERR_INVALID_ARG,
          "noalloc unknown format");

    printf("%s\n", failures ? "FAILED" : "ALL OK");
    return failures ? 1 : 0;
}
