// Host side of libdose: the C ABI declared in include/dose.h.
//
// dose_create_matrix validates the CSR (Sec. II-C layout), encodes FP64 values
// into the stored format if asked, builds the row-binned pipeline schedule and
// uploads everything once: the dose-deposition matrix does not change during
// the optimisation, only the spot weights do (Sec. II-A).  Compute calls only
// enqueue kernels on the caller's stream.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <memory>
#include <string>
#include <vector>

#include "dose_internal.cuh"
#include "nvtx_range.cuh"

namespace dose {

static thread_local std::string g_last_error;

void set_error(const std::string& msg) { g_last_error = msg; }

dose_status cuda_fail(cudaError_t e, const char* what) {
    if (e == cudaErrorMemoryAllocation) {
        set_error(std::string(what) + ": out of device memory");
        return DOSE_ERR_OOM;
    }
    set_error(std::string(what) + ": " + cudaGetErrorName(e) + " (" + cudaGetErrorString(e) + ")");
    return DOSE_ERR_CUDA;
}

cudaError_t dev_malloc(void** p, size_t bytes) {
    *p = nullptr;
    if (const char* lim = std::getenv("DOSE_TEST_ALLOC_LIMIT")) {
        const unsigned long long n = std::strtoull(lim, nullptr, 10);
        if (n && bytes > n) return cudaErrorMemoryAllocation;
    }
    return cudaMalloc(p, bytes);
}

static dose_status invalid(const std::string& msg) {
    set_error(msg);
    return DOSE_ERR_INVALID_ARG;
}

// ------------------------------------------------------------- encoders
// Library encoders of the stored formats (same definitions as the format
// comments in dose.h; written independently of any checker).

// Round-to-nearest-even of a double to 8 significant bits (bfloat16), by
// rounding the binary64 significand at bit 45.
static uint16_t encode_bf16(double v) {
    if (std::isnan(v)) return 0x7FC0;
    const uint16_t sign = std::signbit(v) ? 0x8000 : 0;
    const double a = std::fabs(v);
    float f;
    if (a < 0x1p-126) {
        f = (float)(std::rint(a * 0x1p133) * 0x1p-133);  // bf16 subnormal quantum 2^-133
    } else {
        uint64_t u;
        std::memcpy(&u, &a, 8);
        const uint64_t lsb = (u >> 45) & 1u;
        u += 0x0FFFFFFFFFFFull + lsb;  // half of the dropped 45 bits, minus one, plus the kept LSB
        u &= ~0x1FFFFFFFFFFFull;
        double r;
        std::memcpy(&r, &u, 8);
        f = r > 0x1.FEp127 ? INFINITY : (float)r;
    }
    uint32_t b;
    std::memcpy(&b, &f, 4);
    return (uint16_t)(sign | (b >> 16));
}

// Nearest OCP E4M3 code of a non-negative finite t, ties to the even code,
// saturating at 448 (code 0x7E).
static uint8_t encode_e4m3(double t) {
    if (!(t > 0)) return 0;
    if (t >= 448.0) return 0x7E;
    if (t < 0x1p-6) {  // subnormal range: quantum 2^-9 (q = 8 is the smallest normal)
        return (uint8_t)std::rint(t * 0x1p9);
    }
    int ex;
    const double f = std::frexp(t, &ex);  // t = f 2^ex, f in [0.5, 1)
    int e = ex - 1;                       // t = (2f) 2^e, 2f in [1, 2)
    double m = std::rint((2.0 * f - 1.0) * 8.0);
    if (m == 8.0) {
        m = 0.0;
        ++e;
    }
    const int code = ((e + 7) << 3) | (int)m;
    return code > 0x7E ? (uint8_t)0x7E : (uint8_t)code;
}

// IEEE binary16 bits of v, rounded to nearest with ties to even, from the
// binary64 fields of v: the 53-bit significand is shifted down to the half's
// quantum (2^(E-10) for normal halves, 2^-24 below 2^-14) and the dropped bits
// decide the rounding; a carry out of the significand moves to the next
// exponent, and past the largest finite half (65504) to infinity.
static uint16_t encode_f16(double v) {
    uint64_t b;
    std::memcpy(&b, &v, 8);
    const uint16_t sign = (uint16_t)((b >> 48) & 0x8000u);
    const int e = (int)((b >> 52) & 0x7FF);
    const uint64_t frac = b & ((1ull << 52) - 1);
    if (e == 0x7FF) return sign | (frac ? 0x7E00 : 0x7C00);
    if (e == 0) return sign;  // below 2^-1022: far under half the smallest half
    const int E = e - 1023;
    if (E > 15) return sign | 0x7C00;
    const uint64_t sig = frac | (1ull << 52);                 // v = sig * 2^(E - 52)
    const int qexp = E >= -14 ? E - 10 : -24;                  // exponent of the half's quantum
    const int shift = qexp - (E - 52);                         // 42 for normal halves
    if (shift > 63) return sign;
    uint64_t keep = sig >> shift;
    const uint64_t rem = sig & ((1ull << shift) - 1), halfway = 1ull << (shift - 1);
    if (rem > halfway || (rem == halfway && (keep & 1))) ++keep;
    if (E < -14) return sign | (uint16_t)keep;                 // subnormal (1024 = smallest normal)
    const uint32_t bits = ((uint32_t)(E + 15) << 10) + (uint32_t)(keep - 1024);  // carry moves the exponent
    return sign | (uint16_t)(bits >= 0x7C00u ? 0x7C00u : bits);
}

static dose_status encode(dose_format fmt, uint32_t nrows, const uint32_t* row_ptr, uint64_t nnz,
                          const double* v, void* codes, float* scales) {
    for (uint64_t k = 0; k < nnz; ++k)
        if (!(v[k] >= 0.0) || std::isinf(v[k])) return invalid("values_f64 must be finite and non-negative");
    if (fmt == DOSE_FMT_U16_SCALE) {
        double vmax = 0.0;
        for (uint64_t k = 0; k < nnz; ++k) vmax = std::max(vmax, v[k]);
        float s = vmax > 0.0 ? (float)(vmax / 65535.0) : 1.0f;
        if (!(s > 0.0f)) s = 1.0f;
        scales[0] = s;
        uint16_t* q = static_cast<uint16_t*>(codes);
        const double sd = s;
        for (uint64_t k = 0; k < nnz; ++k) {
            const double t = std::rint(v[k] / sd);
            q[k] = (uint16_t)(t > 65535.0 ? 65535.0 : t);
        }
        return DOSE_OK;
    }
    if (fmt == DOSE_FMT_BF16) {
        uint16_t* q = static_cast<uint16_t*>(codes);
        for (uint64_t k = 0; k < nnz; ++k) q[k] = encode_bf16(v[k]);
        return DOSE_OK;
    }
    if (fmt == DOSE_FMT_F16) {
        uint16_t* q = static_cast<uint16_t*>(codes);
        for (uint64_t k = 0; k < nnz; ++k) q[k] = encode_f16(v[k]);
        return DOSE_OK;
    }
    if (fmt == DOSE_FMT_F32) {
        float* q = static_cast<float*>(codes);
        for (uint64_t k = 0; k < nnz; ++k) {
            q[k] = (float)v[k];  // IEEE conversion: round to nearest, ties to even
            if (std::isinf(q[k])) return invalid("values_f64 exceed the FP32 range");
        }
        return DOSE_OK;
    }
    if (fmt == DOSE_FMT_FP8E4M3_ROWSCALE) {
        uint8_t* q = static_cast<uint8_t*>(codes);
        for (uint32_t i = 0; i < nrows; ++i) {
            double rmax = 0.0;
            for (uint64_t k = row_ptr[i]; k < row_ptr[i + 1]; ++k) rmax = std::max(rmax, v[k]);
            float s = rmax > 0.0 ? (float)(rmax / 448.0) : 1.0f;
            if (!(s > 0.0f)) s = 1.0f;
            scales[i] = s;
            const double sd = s;
            for (uint64_t k = row_ptr[i]; k < row_ptr[i + 1]; ++k) q[k] = encode_e4m3(v[k] / sd);
        }
        return DOSE_OK;
    }
    return invalid("unknown format");
}

// ------------------------------------------------------------ schedule

static uint32_t nearest_pow2_log2(double v) {
    if (!(v > 1.0)) return 0;
    int lg = (int)std::lround(std::log2(v));
    return (uint32_t)std::min(5, std::max(0, lg));
}

// Deal work items (ranges of S.desc) to the grid's CTAs and store the
// descriptors CTA by CTA.  Without windows: round-robin in matrix order.  With
// windows: items with entries are sorted by lowest column and cut into G groups
// of equal estimated cost; group g is dealt round-robin, in matrix order, to
// its own grid/G CTAs.  A CTA's window then spans one group's columns (for a
// pencil beam: one lateral band plus the spot footprint), while round-robin
// inside the group mixes long and short rows as evenly as dealing over the
// whole matrix does.  Items without entries (blocks of empty rows: cheap in
// bytes, but each costs a ring round trip) are dealt round-robin over all CTAs.
// Each CTA runs its items in matrix order, so the blocks in flight at any time
// lie close together in HBM.  align_wlo: windows start on a multiple of 32
// columns (a column then falls in shared-memory bank c mod 32 in every CTA).
void deal_items(Schedule& S, const std::vector<DealItem>& items, uint32_t grid, uint32_t ncols, bool windowed,
                bool align_wlo) {
    const uint32_t n = (uint32_t)S.desc.size();
    std::vector<std::vector<uint32_t>> per(grid);
    S.wlo.assign(grid, 0);
    const uint32_t ncols_pad = (ncols + 31) / 32 * 32;
    S.wwidth = ncols_pad;
    if (!windowed) {
        for (size_t i = 0; i < items.size(); ++i)
            for (uint32_t k = items[i].s; k < items[i].e; ++k) per[i % grid].push_back(k);
    } else {
        std::vector<uint32_t> order, empties;
        for (uint32_t i = 0; i < items.size(); ++i) (items[i].lo <= items[i].hi ? order : empties).push_back(i);
        std::stable_sort(order.begin(), order.end(),
                         [&](uint32_t a, uint32_t b) { return items[a].lo < items[b].lo; });
        uint64_t total = 0;
        for (uint32_t i : order) total += items[i].cost;
        const uint32_t G = std::max<uint32_t>(1, std::min<uint32_t>(kAdjColumnGroups, grid));
        std::vector<std::vector<uint32_t>> group(G);
        uint64_t acc = 0;
        uint32_t gi = 0;
        for (uint32_t i : order) {
            while (gi + 1 < G && acc * G >= total * (gi + 1)) ++gi;  // group gi holds its share
            group[gi].push_back(i);
            acc += items[i].cost;
        }
        std::vector<uint32_t> lo(grid, 0xFFFFFFFFu), hi(grid, 0);
        std::vector<std::vector<uint32_t>> mine(grid);
        for (uint32_t g = 0; g < G; ++g) {
            const uint32_t c0 = (uint32_t)((uint64_t)grid * g / G), c1 = (uint32_t)((uint64_t)grid * (g + 1) / G);
            std::sort(group[g].begin(), group[g].end());
            for (size_t k = 0; k < group[g].size(); ++k) {
                const uint32_t c = c0 + (uint32_t)(k % (c1 - c0)), i = group[g][k];
                mine[c].push_back(i);
                lo[c] = std::min(lo[c], items[i].lo);
                hi[c] = std::max(hi[c], items[i].hi);
            }
        }
        for (size_t k = 0; k < empties.size(); ++k) mine[k % grid].push_back(empties[k]);
        if (align_wlo)
            for (uint32_t k = 0; k < grid; ++k)
                if (lo[k] <= hi[k]) lo[k] &= ~31u;
        uint32_t width = 0;
        for (uint32_t k = 0; k < grid; ++k) {
            std::sort(mine[k].begin(), mine[k].end());
            for (uint32_t i : mine[k])
                for (uint32_t d = items[i].s; d < items[i].e; ++d) per[k].push_back(d);
            if (lo[k] <= hi[k]) width = std::max(width, hi[k] - lo[k] + 1);
        }
        S.wwidth = std::max<uint32_t>(32, std::min(ncols_pad, (width + 31) / 32 * 32));
        for (uint32_t k = 0; k < grid; ++k) S.wlo[k] = lo[k] <= hi[k] ? lo[k] : 0;
    }
    // Store the descriptors CTA by CTA, so each CTA reads one contiguous range.
    std::vector<StageDesc> sorted;
    sorted.reserve(n);
    S.cta_begin.assign(grid + 1, 0);
    for (uint32_t c = 0; c < grid; ++c) {
        S.cta_begin[c] = (uint32_t)sorted.size();
        for (uint32_t k : per[c]) sorted.push_back(S.desc[k]);
    }
    S.cta_begin[grid] = (uint32_t)sorted.size();
    S.desc.swap(sorted);
}

// Column windows: rcmin / rcmax give each row's lowest and highest column (null
// for a schedule without windows, which deals round-robin).  vbytes: stored bytes per
// entry (value + column index), used to balance the CTAs' HBM traffic.  tight:
// also end a block where its column range would more than double below the cap
// (narrower windows; more blocks).
static Schedule build_schedule(const std::vector<uint32_t>& rp, uint32_t nrows, const Tuning& t, uint32_t grid,
                               const uint32_t* rcmin, const uint32_t* rcmax, uint32_t ncols, uint32_t vbytes,
                               bool tight = false) {
    Schedule S;
    uint32_t r = 0;
    // Widest single row: a block wider than 1.5 times it can only come from rows
    // far apart in the spot numbering (see the cut below).
    uint32_t row_span_max = 0;
    if (rcmin)
        for (uint32_t i = 0; i < nrows; ++i)
            if (rcmin[i] <= rcmax[i]) row_span_max = std::max(row_span_max, rcmax[i] - rcmin[i]);
    const uint64_t span_cap = (uint64_t)row_span_max * 3 / 2;
    while (r < nrows) {
        const uint32_t len = rp[r + 1] - rp[r];
        if (len > t.coop_nnz) {
            const uint32_t nch = (len + t.tile_nnz - 1) / t.tile_nnz;
            const uint32_t ne = (uint32_t)S.ne.size();
            for (uint32_t c = 0; c < nch; ++c) {
                StageDesc D{};
                D.row0 = r;
                D.row1 = r + 1;
                D.nz0 = rp[r] + c * t.tile_nnz;
                D.nz1 = std::min(rp[r + 1], D.nz0 + t.tile_nnz);
                D.ne0 = D.ne1 = ne;
                D.meta = STAGE_COOP | (c == 0 ? STAGE_FIRST : 0u) | (c + 1 == nch ? STAGE_LAST : 0u);
                S.desc.push_back(D);
            }
            ++S.n_coop_rows;
            ++r;
            continue;
        }
        StageDesc D{};
        D.row0 = r;
        D.nz0 = rp[r];
        D.ne0 = (uint32_t)S.ne.size();
        uint64_t nz = 0;
        uint32_t slo = 0xFFFFFFFFu, shi = 0;  // columns of the block's rows so far (windowed schedules)
        while (r < nrows && r - D.row0 < t.tile_rows) {
            const uint32_t l = rp[r + 1] - rp[r];
            if (l > t.coop_nnz || nz + l > t.tile_nnz) break;
            if (rcmin && l) {
                // A block whose column range would more than double with this row,
                // and grow wider than 1.5 times any single row (the voxel order
                // wrapping to the far side of the beam), ends here: one wide block
                // would widen every CTA's window.  Rows of a multi-beam plan
                // already span all beams' spots, so their blocks are never cut.
                const uint32_t nlo = std::min(slo, rcmin[r]), nhi = std::max(shi, rcmax[r]);
                if (slo <= shi && nhi - nlo > 2 * std::max(shi - slo, rcmax[r] - rcmin[r]) + 64 &&
                    (tight || nhi - nlo > span_cap))
                    break;
                slo = nlo;
                shi = nhi;
            }
            nz += l;
            if (l) S.ne.push_back((uint16_t)(r - D.row0));
            ++r;
        }
        D.row1 = r;
        D.nz1 = rp[r];
        D.ne1 = (uint32_t)S.ne.size();
        if (t.row_order == 2) {
            // Longest rows first (counted in the 4-entry groups a lane loads), so the
            // rows that one warp reduces together have similar trip counts.
            const uint32_t row0 = D.row0;
            auto groups = [&](uint16_t o) { return (rp[row0 + o + 1] - (rp[row0 + o] & ~3u) + 3) / 4; };
            std::stable_sort(S.ne.begin() + D.ne0, S.ne.end(),
                             [&](uint16_t a, uint16_t b) { return groups(a) > groups(b); });
        }
        const uint32_t nonempty = D.ne1 - D.ne0;
        const double mean = nonempty ? (double)nz / nonempty : 0.0;
        const uint32_t lg = nonempty ? nearest_pow2_log2(mean / t.lane_target) : 5;
        D.meta = lg;
        S.desc.push_back(D);
        ++S.lanes_hist[lg];
    }

    // Work items: a NORMAL stage, or the consecutive chunks of one long row.
    const uint32_t n = (uint32_t)S.desc.size();
    std::vector<DealItem> items;
    for (uint32_t s = 0; s < n;) {
        uint32_t e = s + 1;
        if (S.desc[s].meta & STAGE_COOP)
            while (e < n && (S.desc[e].meta & STAGE_COOP) && !(S.desc[e].meta & STAGE_FIRST)) ++e;
        DealItem it{s, e, 0xFFFFFFFFu, 0u, 0};
        const uint32_t r0 = S.desc[s].row0, r1 = S.desc[e - 1].row1;
        // HBM bytes (entries, row pointers, two per-row vectors) + for the
        // adjoint, a share per 128-entry step of each row
        it.cost = (uint64_t)vbytes * (rp[r1] - rp[r0]) + 12ull * (r1 - r0);
        if (rcmin)
            for (uint32_t r = r0; r < r1; ++r)
                if (rcmin[r] <= rcmax[r]) {
                    it.lo = std::min(it.lo, rcmin[r]);
                    it.hi = std::max(it.hi, rcmax[r]);
                    // a scatter warp takes a row in steps of 128 entries, whatever its length
                    it.cost += 512ull * ((rp[r + 1] - rp[r] + 2 + 127) / 128);
                }
        items.push_back(it);
        s = e;
    }
    deal_items(S, items, grid, ncols, rcmin != nullptr, false);
    return S;
}

// ------------------------------------------------------------ handle state

static void free_dev_schedule(DevSchedule& D) {
    cudaFree(D.desc);
    cudaFree(D.ne);
    cudaFree(D.cta_begin);
    cudaFree(D.wlo);
    D.desc = nullptr;
    D.ne = nullptr;
    D.cta_begin = nullptr;
    D.wlo = nullptr;
    D.wwidth = 0;
    D.n_stages = 0;
}

static void free_all(dose_matrix* A) {
    free_row_groups(A);
    free_dev_schedule(A->fwd);
    free_dev_schedule(A->fwd64);
    free_dev_schedule(A->adj);
    cudaFree(A->row_ptr);
    cudaFree(A->col);
    cudaFree(A->col16);
    cudaFree(A->val);
    cudaFree(A->row_scale);
    cudaFree(A->x64);
    free_sell(A);
    cudaFree(A->g_part);
    cudaFree(A->f_part);
    cudaFree(A->err);
}

// Ranges of the forward knobs (no handle needed).
static dose_status check_tuning_ranges(const Tuning& t) {
    if (t.tile_nnz < 256 || t.tile_nnz > 16384) return invalid("tuning.tile_nnz must be in [256, 16384]");
    if (t.tile_rows < 32 || t.tile_rows > 8192) return invalid("tuning.tile_rows must be in [32, 8192]");
    if (t.coop_nnz < 32 || t.coop_nnz > t.tile_nnz) return invalid("tuning.coop_nnz must be in [32, tile_nnz]");
    if (t.lane_target < 1 || t.lane_target > 64) return invalid("tuning.lane_target must be in [1, 64]");
    if (t.stages < 2 || t.stages > 8) return invalid("tuning.stages must be in [2, 8]");
    if (t.consumer_warps != 4 && t.consumer_warps != 8 && t.consumer_warps != 16)
        return invalid("tuning.consumer_warps must be 4, 8 or 16");
    if (t.row_order < 1 || t.row_order > 2) return invalid("tuning.row_order must be 1 or 2");
    if (t.layout > 2) return invalid("tuning.fwd_layout must be 0, 1 or 2");
    return DOSE_OK;
}

dose_status check_tuning(const dose_matrix* A, Tuning& t) {
    if (t.tile_nnz < 256 || t.tile_nnz > 16384) return invalid("tuning.tile_nnz must be in [256, 16384]");
    if (t.tile_rows < 32 || t.tile_rows > 8192) return invalid("tuning.tile_rows must be in [32, 8192]");
    if (t.coop_nnz < 32 || t.coop_nnz > t.tile_nnz) return invalid("tuning.coop_nnz must be in [32, tile_nnz]");
    if (t.lane_target < 1 || t.lane_target > 64) return invalid("tuning.lane_target must be in [1, 64]");
    if (t.stages < 2 || t.stages > 8) return invalid("tuning.stages must be in [2, 8]");
    if (t.consumer_warps != 4 && t.consumer_warps != 8 && t.consumer_warps != 16)
        return invalid("tuning.consumer_warps must be 4, 8 or 16");
    if (t.row_order < 1 || t.row_order > 2) return invalid("tuning.row_order must be 1 or 2");
    if (t.layout > 2) return invalid("tuning.fwd_layout must be 0, 1 or 2");
    if (spmv_smem_bytes(A, t, spmv_x_in_smem(A, t)) > kMaxSmemPerBlock)
        return invalid("tuning needs more shared memory than a CTA has");
    return DOSE_OK;
}

// Knobs the caller left at 0 shrink until the forward pipeline fits beside x:
// first the tile (down to 1024 entries), then the depth (down to 2).
static void fit_default_tuning(const dose_matrix* A, Tuning& t, const dose_tuning* in) {
    const bool user_tile = in && in->tile_nnz, user_stages = in && in->stages;
    while (spmv_smem_bytes(A, t, spmv_x_in_smem(A, t)) > kMaxSmemPerBlock) {
        if (!user_tile && t.tile_nnz > 1024) {
            t.tile_nnz /= 2;
            if (!(in && in->coop_nnz)) t.coop_nnz = std::min(t.coop_nnz, t.tile_nnz);
        } else if (!user_stages && t.stages > 2) {
            --t.stages;
        } else {
            break;
        }
    }
}

dose_status check_adj_tuning(const AdjTuning& t) {
    if (t.tile_nnz < 256 || t.tile_nnz > 16384) return invalid("tuning.adj_tile_nnz must be in [256, 16384]");
    if (t.tile_rows < 32 || t.tile_rows > 8192) return invalid("tuning.adj_tile_rows must be in [32, 8192]");
    if (t.stages < 2 || t.stages > 8) return invalid("tuning.adj_stages must be in [2, 8]");
    if (t.forward_warps < 1 || t.forward_warps > 15) return invalid("tuning.adj_forward_warps must be in [1, 15]");
    if (t.row_order < 1 || t.row_order > 2) return invalid("tuning.adj_row_order must be 1 or 2");
    if (t.scatter_warps > kMaxAdjWarps - 2)
        return invalid("tuning.adj_scatter_warps must be in [0, " + std::to_string(kMaxAdjWarps - 2) + "]");
    if (t.layout > 2) return invalid("tuning.adj_layout must be 0, 1 or 2");
    if (t.rg_tile_u && (t.rg_tile_u < 256 || t.rg_tile_u > 8192))
        return invalid("tuning.rg_tile_union must be in [256, 8192]");
    if (t.rg_tile_rows < 256 || t.rg_tile_rows > 8192) return invalid("tuning.rg_tile_rows must be in [256, 8192]");
    if (t.rg_stages < 2 || t.rg_stages > 8) return invalid("tuning.rg_stages must be in [2, 8]");
    if (t.rg_warps > kRgMaxWarps) return invalid("tuning.rg_warps must be in [0, " + std::to_string(kRgMaxWarps) + "]");
    return DOSE_OK;
}

void merge_tuning(Tuning& t, AdjTuning& a, const dose_tuning* in) {
    if (!in) return;
    if (in->tile_nnz) t.tile_nnz = in->tile_nnz;
    if (in->tile_rows) t.tile_rows = in->tile_rows;
    if (in->coop_nnz) t.coop_nnz = in->coop_nnz;
    if (in->lane_target) t.lane_target = in->lane_target;
    if (in->stages) t.stages = in->stages;
    if (in->consumer_warps) t.consumer_warps = in->consumer_warps;
    if (in->l2_prefetch) t.l2_prefetch = in->l2_prefetch >= 32 ? 0 : in->l2_prefetch;
    if (in->adj_tile_nnz) a.tile_nnz = in->adj_tile_nnz;
    if (in->adj_tile_rows) a.tile_rows = in->adj_tile_rows;
    if (in->adj_stages) a.stages = in->adj_stages;
    if (in->adj_forward_warps) a.forward_warps = in->adj_forward_warps;
    if (in->adj_scatter_warps) a.scatter_warps = in->adj_scatter_warps;
    if (in->adj_l2_prefetch) a.l2_prefetch = in->adj_l2_prefetch >= 32 ? 0 : in->adj_l2_prefetch;
    if (in->row_order) t.row_order = in->row_order;
    if (in->adj_row_order) a.row_order = in->adj_row_order;
    if (in->adj_layout) a.layout = in->adj_layout;
    if (in->rg_tile_union) a.rg_tile_u = in->rg_tile_union;
    if (in->rg_tile_rows) a.rg_tile_rows = in->rg_tile_rows;
    if (in->rg_stages) a.rg_stages = in->rg_stages;
    if (in->rg_warps) a.rg_warps = in->rg_warps;
    if (in->rg_l2_prefetch) a.rg_l2_prefetch = in->rg_l2_prefetch >= 32 ? 0 : in->rg_l2_prefetch;
    if (in->fwd_layout) t.layout = in->fwd_layout;
    if (!in->coop_nnz) t.coop_nnz = std::min(t.coop_nnz, t.tile_nnz);  // the default follows a smaller tile
}

void export_tuning(const Tuning& t, const AdjTuning& a, dose_tuning* out) {
    out->tile_nnz = t.tile_nnz;
    out->tile_rows = t.tile_rows;
    out->coop_nnz = t.coop_nnz;
    out->lane_target = t.lane_target;
    out->stages = t.stages;
    out->consumer_warps = t.consumer_warps;
    out->l2_prefetch = t.l2_prefetch ? t.l2_prefetch : 32;
    out->adj_tile_nnz = a.tile_nnz;
    out->adj_tile_rows = a.tile_rows;
    out->adj_stages = a.stages;
    out->adj_forward_warps = a.forward_warps;
    out->adj_scatter_warps = a.scatter_warps;
    out->adj_l2_prefetch = a.l2_prefetch ? a.l2_prefetch : 32;
    out->row_order = t.row_order;
    out->adj_row_order = a.row_order;
    out->adj_layout = a.layout;
    out->rg_tile_union = a.rg_tile_u;
    out->rg_tile_rows = a.rg_tile_rows;
    out->rg_stages = a.rg_stages;
    out->rg_warps = a.rg_warps;
    out->rg_l2_prefetch = a.rg_l2_prefetch ? a.rg_l2_prefetch : 32;
    out->fwd_layout = t.layout;
}

template <class T>
static cudaError_t upload(T** dst, const T* src, size_t n, size_t alloc_n) {
    cudaError_t e = dev_malloc(dst, std::max<size_t>(alloc_n, 1) * sizeof(T));
    if (e != cudaSuccess) return e;
    e = cudaMemset(*dst, 0, std::max<size_t>(alloc_n, 1) * sizeof(T));
    if (e != cudaSuccess) return e;
    if (n) e = cudaMemcpy(*dst, src, n * sizeof(T), cudaMemcpyHostToDevice);
    return e;
}

// Build one schedule on the host and replace `D` with its device copy.  The
// adjoint schedule (`windowed`) gets per-CTA column windows.
dose_status apply_schedule(dose_matrix* A, DevSchedule& D, const Tuning& t, bool windowed) {
    const bool win = windowed && !A->host_row_cmin.empty();
    const uint32_t vbytes = value_bytes(A->fmt) + 4;
    Schedule S = build_schedule(A->host_row_ptr, A->nrows, t, D.grid, win ? A->host_row_cmin.data() : nullptr,
                                win ? A->host_row_cmax.data() : nullptr, A->ncols, vbytes);
    if (win) {
        // Cutting blocks at every doubling of their column range narrows the
        // windows of a single beam (one more scatter warp fits on the clinical
        // beam) but only fragments a multi-beam plan, whose rows already span
        // every beam: keep it where it narrows the window.
        Schedule T = build_schedule(A->host_row_ptr, A->nrows, t, D.grid, A->host_row_cmin.data(),
                                    A->host_row_cmax.data(), A->ncols, vbytes, true);
        if (T.wwidth < S.wwidth) S = std::move(T);
    }
    free_dev_schedule(D);
    cudaError_t e;
    if ((e = upload(&D.desc, S.desc.data(), S.desc.size(), S.desc.size() + 1)) != cudaSuccess ||
        (e = upload(&D.ne, S.ne.data(), S.ne.size(), (S.ne.size() + 7) / 8 * 8 + 16)) != cudaSuccess ||
        (e = upload(&D.cta_begin, S.cta_begin.data(), S.cta_begin.size(), S.cta_begin.size())) != cudaSuccess ||
        (e = upload(&D.wlo, S.wlo.data(), S.wlo.size(), S.wlo.size())) != cudaSuccess)
        return cuda_fail(e, "uploading the schedule");
    D.wwidth = S.wwidth;
    D.n_stages = (uint32_t)S.desc.size();
    D.n_coop_rows = S.n_coop_rows;
    std::memcpy(D.lanes_hist, S.lanes_hist, sizeof(D.lanes_hist));
    D.tuning = t;
    return DOSE_OK;
}

// The adjoint schedule: its own tile sizes, the forward's lane binning.
Tuning adj_schedule_tuning(const Tuning& fwd, const AdjTuning& a) {
    Tuning t = fwd;
    t.tile_nnz = a.tile_nnz;
    t.tile_rows = a.tile_rows;
    t.coop_nnz = std::min({fwd.coop_nnz, a.tile_nnz, kAdjCoopNnz});
    t.stages = a.stages;
    t.row_order = a.row_order;
    return t;
}

static uint64_t schedule_bytes(const DevSchedule& D) {
    return (uint64_t)(D.n_stages + 1) * sizeof(StageDesc) + (D.grid + 1) * 4 + D.grid * 4;
}

static cudaStream_t as_stream(void* s) { return static_cast<cudaStream_t>(s); }

}  // namespace dose

using namespace dose;

namespace {
// Time `reps` launches of fn after 3 warm-up launches; returns ms per launch or
// a negative value on error.

// Self-test of the bounded waits: one thread waits on a phase of an mbarrier
// that nothing arrives at; the wait gives up after limit_ns and the kernel
// records whether it did, then returns.
__device__ int g_selftest_timed_out;

__global__ void selftest_wait_kernel(uint64_t limit_ns) {
    __shared__ uint64_t bar;
    dev::mbar_init(&bar, 1);
    dev::fence_mbar_init();
    g_selftest_timed_out = dev::mbar_wait_limit(&bar, 0, limit_ns) ? 0 : 1;
}

}  // namespace

extern "C" {

dose_status dose_selftest_bounded_wait(uint32_t limit_us, void* stream) {
    if (limit_us == 0 || limit_us > 1000000u) return invalid("dose_selftest_bounded_wait: limit_us must be in [1, 1e6]");
    cudaStream_t s = as_stream(stream);
    selftest_wait_kernel<<<1, 1, 0, s>>>((uint64_t)limit_us * 1000ull);
    cudaError_t e = cudaGetLastError();
    int flag = 0;
    if (e == cudaSuccess) e = cudaMemcpyFromSymbolAsync(&flag, g_selftest_timed_out, sizeof(int), 0,
                                                        cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cuda_fail(e, "dose_selftest_bounded_wait");
    if (!flag) {
        set_error("dose_selftest_bounded_wait: the wait on a phase that never completes returned as completed");
        return DOSE_OK;
    }
    set_error("dose_selftest_bounded_wait: the bounded wait ran out as designed");
    return DOSE_ERR_TIMEOUT;
}

const char* dose_last_error(void) { return g_last_error.c_str(); }

const char* dose_version(void) { return "libdose 0.1 (sm_103a)"; }

dose_status dose_encode_host(dose_format fmt, uint32_t nrows, const uint32_t* row_ptr, uint64_t nnz,
                             const double* values_f64, void* codes, float* scales) {
    if ((nnz && (!values_f64 || !codes)) || !row_ptr) return invalid("dose_encode_host: null pointer");
    if ((fmt == DOSE_FMT_U16_SCALE || fmt == DOSE_FMT_FP8E4M3_ROWSCALE) && !scales)
        return invalid("dose_encode_host: scales needed for this format");
    return encode(fmt, nrows, row_ptr, nnz, values_f64, codes, scales);
}

dose_status dose_create_matrix(const dose_csr_desc* desc, unsigned flags, const dose_tuning* tuning, void* stream,
                               dose_matrix** out) {
    NvtxRange nvtx_range("dose_create_matrix");
    if (!desc || !out) return invalid("dose_create_matrix: null desc or out");
    *out = nullptr;
    if (flags & ~(DOSE_CREATE_COMPENSATED | DOSE_CREATE_U16_INDEX | DOSE_CREATE_SELL))
        return invalid("dose_create_matrix: unknown flags");
    const uint32_t sell_sigma = (tuning && tuning->sell_sigma) ? tuning->sell_sigma : kSellDefaultSigma;
    if ((flags & DOSE_CREATE_SELL) && sell_sigma > (1u << 24))
        return invalid("tuning.sell_sigma must be in [1, 2^24]");
    if ((flags & DOSE_CREATE_U16_INDEX) && desc->ncols > 65536u)
        return invalid("DOSE_CREATE_U16_INDEX needs ncols <= 65536 (16-bit column indices)");
    const dose_format fmt = desc->fmt;
    if (fmt != DOSE_FMT_U16_SCALE && fmt != DOSE_FMT_BF16 && fmt != DOSE_FMT_FP8E4M3_ROWSCALE &&
        fmt != DOSE_FMT_F16 && fmt != DOSE_FMT_F32)
        return invalid("dose_create_matrix: unknown format");
    if (desc->nnz >= (1ull << 32)) return invalid("nnz must be < 2^32 (uint32 row pointers)");
    if (desc->nrows == 0xFFFFFFFFu) return invalid("nrows must be < 2^32 - 1");
    if (!desc->row_ptr) return invalid("row_ptr is NULL");
    if (desc->nnz && !desc->col_idx) return invalid("col_idx is NULL");
    if (desc->on_device && desc->values_f64) return invalid("values_f64 must be host memory (on_device=0)");
    if (!desc->values && !desc->values_f64 && desc->nnz) return invalid("neither values nor values_f64 given");
    if (desc->values && (fmt == DOSE_FMT_U16_SCALE || fmt == DOSE_FMT_FP8E4M3_ROWSCALE) && !desc->scales)
        return invalid("scales are NULL for this format");
    {
        // knob ranges first: a bad tuning is refused before any CUDA call
        Tuning t0;
        AdjTuning a0;
        merge_tuning(t0, a0, tuning);
        dose_status st = check_tuning_ranges(t0);
        if (st == DOSE_OK) st = check_adj_tuning(a0);
        if (st != DOSE_OK) return st;
    }
    const uint32_t nrows = desc->nrows, ncols = desc->ncols;
    const uint64_t nnz = desc->nnz;
    const size_t esize = value_bytes(fmt);
    cudaStream_t s = as_stream(stream);

    // Bring the structure to the host (validation and scheduling need it).
    std::vector<uint32_t> rp(nrows + 1), col(nnz);
    std::vector<unsigned char> vals;
    std::vector<float> scl;
    cudaError_t e;
    if (desc->on_device) {
        if ((e = cudaMemcpyAsync(rp.data(), desc->row_ptr, rp.size() * 4, cudaMemcpyDeviceToHost, s)) != cudaSuccess)
            return cuda_fail(e, "reading row_ptr");
        if (nnz && (e = cudaMemcpyAsync(col.data(), desc->col_idx, nnz * 4, cudaMemcpyDeviceToHost, s)) != cudaSuccess)
            return cuda_fail(e, "reading col_idx");
        if ((e = cudaStreamSynchronize(s)) != cudaSuccess) return cuda_fail(e, "reading the CSR");
    } else {
        std::memcpy(rp.data(), desc->row_ptr, rp.size() * 4);
        if (nnz) std::memcpy(col.data(), desc->col_idx, nnz * 4);
    }
    if (rp[0] != 0) return invalid("row_ptr[0] must be 0");
    if (rp[nrows] != nnz) return invalid("row_ptr[nrows] must equal nnz");
    uint32_t max_len = 0;
    for (uint32_t i = 0; i < nrows; ++i) {
        if (rp[i + 1] < rp[i]) return invalid("row_ptr must be non-decreasing (row " + std::to_string(i) + ")");
        max_len = std::max(max_len, rp[i + 1] - rp[i]);
    }
    std::vector<uint32_t> rcmin(nrows, 0xFFFFFFFFu), rcmax(nrows, 0);
    {
        std::vector<uint32_t> stamp(ncols, 0xFFFFFFFFu);
        for (uint32_t i = 0; i < nrows; ++i) {
            uint32_t lo = 0xFFFFFFFFu, hi = 0;
            for (uint32_t k = rp[i]; k < rp[i + 1]; ++k) {
                const uint32_t c = col[k];
                if (c >= ncols)
                    return invalid("col_idx[" + std::to_string(k) + "] = " + std::to_string(c) + " >= ncols");
                if (stamp[c] == i)
                    return invalid("duplicate column " + std::to_string(c) + " in row " + std::to_string(i));
                stamp[c] = i;
                lo = std::min(lo, c);
                hi = std::max(hi, c);
            }
            rcmin[i] = lo;
            rcmax[i] = hi;
        }
    }
    // Values: encode FP64 on the host, or take the given codes.
    float scale = 1.0f;
    if (!desc->values) {
        vals.resize(nnz * esize);
        scl.resize(fmt == DOSE_FMT_FP8E4M3_ROWSCALE ? std::max<uint32_t>(nrows, 1) : 1);
        dose_status st = encode(fmt, nrows, rp.data(), nnz, desc->values_f64, vals.data(), scl.data());
        if (st != DOSE_OK) return st;
    } else {
        vals.resize(nnz * esize);
        scl.resize(fmt == DOSE_FMT_FP8E4M3_ROWSCALE ? nrows : (fmt == DOSE_FMT_U16_SCALE ? 1 : 0));
        if (desc->on_device) {
            if (nnz && (e = cudaMemcpyAsync(vals.data(), desc->values, nnz * esize, cudaMemcpyDeviceToHost, s)) !=
                           cudaSuccess)
                return cuda_fail(e, "reading values");
            if (!scl.empty() && (e = cudaMemcpyAsync(scl.data(), desc->scales, scl.size() * 4,
                                                     cudaMemcpyDeviceToHost, s)) != cudaSuccess)
                return cuda_fail(e, "reading scales");
            if ((e = cudaStreamSynchronize(s)) != cudaSuccess) return cuda_fail(e, "reading values");
        } else {
            if (nnz) std::memcpy(vals.data(), desc->values, nnz * esize);
            if (!scl.empty()) std::memcpy(scl.data(), desc->scales, scl.size() * 4);
        }
        for (float v : scl)
            if (!(v > 0.0f) || std::isinf(v)) return invalid("scales must be finite and positive");
        if (fmt == DOSE_FMT_FP8E4M3_ROWSCALE)
            for (uint64_t k = 0; k < nnz; ++k)
                if ((vals[k] & 0x7F) == 0x7F) return invalid("FP8 code is NaN at entry " + std::to_string(k));
        if (fmt == DOSE_FMT_F16)
            for (uint64_t k = 0; k < nnz; ++k) {
                uint16_t h;
                std::memcpy(&h, vals.data() + 2 * k, 2);
                if ((h & 0x7C00u) == 0x7C00u) return invalid("F16 value is infinite or NaN at entry " + std::to_string(k));
            }
        if (fmt == DOSE_FMT_BF16)
            for (uint64_t k = 0; k < nnz; ++k) {
                uint16_t b;
                std::memcpy(&b, vals.data() + 2 * k, 2);
                if ((b & 0x7F80u) == 0x7F80u)
                    return invalid("BF16 value is infinite or NaN at entry " + std::to_string(k));
            }
        if (fmt == DOSE_FMT_F32)
            for (uint64_t k = 0; k < nnz; ++k) {
                uint32_t w;
                std::memcpy(&w, vals.data() + 4 * k, 4);
                if ((w & 0x7F800000u) == 0x7F800000u)
                    return invalid("F32 value is infinite or NaN at entry " + std::to_string(k));
            }
    }
    if (fmt == DOSE_FMT_U16_SCALE) scale = scl.empty() ? 1.0f : scl[0];

    std::unique_ptr<dose_matrix> A(new dose_matrix());
    A->nrows = nrows;
    A->ncols = ncols;
    A->nnz = nnz;
    A->fmt = fmt;
    A->flags = flags;
    A->scale = scale;
    A->max_row_len = max_len;
    if ((e = cudaGetDevice(&A->device)) != cudaSuccess) return cuda_fail(e, "cudaGetDevice");
    if ((e = cudaDeviceGetAttribute(&A->sm_count, cudaDevAttrMultiProcessorCount, A->device)) != cudaSuccess)
        return cuda_fail(e, "cudaDeviceGetAttribute");
    A->fwd.grid = A->adj.grid = (uint32_t)std::max(1, A->sm_count);
    A->host_row_ptr = std::move(rp);
    A->host_row_cmin = std::move(rcmin);
    A->host_row_cmax = std::move(rcmax);
    // Too many columns for all of x in shared memory: the forward schedule gets
    // column windows (a row block of a pencil beam touches a narrow band of
    // spots) and the kernels stage each CTA's window of x.
    A->fwd_windowed = ncols > kXSmemMaxCols;
    Tuning t;
    AdjTuning at;
    merge_tuning(t, at, tuning);
    fit_default_tuning(A.get(), t, tuning);
    {
        dose_status st = check_tuning(A.get(), t);
        if (st == DOSE_OK) st = check_adj_tuning(at);
        if (st != DOSE_OK) return st;
    }
    A->adj_tuning = at;
    auto fail = [&](cudaError_t err, const char* what) {
        free_all(A.get());
        return err == cudaErrorMemoryAllocation ? (set_error(std::string(what) + ": out of device memory"),
                                                   DOSE_ERR_OOM)
                                                : cuda_fail(err, what);
    };
    const size_t rp_alloc = ((size_t)nrows + 1 + 3) / 4 * 4 + 16;
    const size_t col_alloc = ((size_t)nnz + 3) / 4 * 4 + 16;
    const size_t val_alloc = ((size_t)nnz * esize + 15) / 16 * 16 + 64;
    if ((e = upload(&A->row_ptr, A->host_row_ptr.data(), (size_t)nrows + 1, rp_alloc)) != cudaSuccess)
        return fail(e, "row_ptr");
    if ((e = upload(&A->col, col.data(), (size_t)nnz, col_alloc)) != cudaSuccess) return fail(e, "col_idx");
    const size_t col16_alloc = ((size_t)nnz + 7) / 8 * 8 + 32;  // copy windows reach round_up(nz1, 8)
    if (flags & DOSE_CREATE_U16_INDEX) {
        std::vector<uint16_t> c16(nnz);
        for (uint64_t k = 0; k < nnz; ++k) c16[k] = (uint16_t)col[k];
        if ((e = upload(&A->col16, c16.data(), (size_t)nnz, col16_alloc)) != cudaSuccess)
            return fail(e, "16-bit col_idx");
    }
    if ((e = upload((unsigned char**)&A->val, vals.data(), vals.size(), val_alloc)) != cudaSuccess)
        return fail(e, "values");
    if (fmt == DOSE_FMT_FP8E4M3_ROWSCALE &&
        (e = upload(&A->row_scale, scl.data(), (size_t)nrows, (size_t)nrows + 16)) != cudaSuccess)
        return fail(e, "row scales");
    const size_t x64_alloc = ((size_t)ncols + 2) / 2 * 2;  // ncols + 1 elements, even count (16 B multiple)
    if ((e = dev_malloc(&A->x64, x64_alloc * 8)) != cudaSuccess) return fail(e, "FP64 vector scratch");
    const size_t ncols_pad = ((size_t)ncols + 31) / 32 * 32;  // a CTA's window is at most this wide
    if ((e = dev_malloc(&A->g_part, std::max<size_t>((size_t)A->adj.grid * ncols_pad, 1) * 4)) != cudaSuccess)
        return fail(e, "adjoint partials");
    if ((e = dev_malloc(&A->f_part, (size_t)A->adj.grid * 8)) != cudaSuccess) return fail(e, "objective partials");
    if ((e = dev_malloc(&A->err, sizeof(int))) != cudaSuccess) return fail(e, "error word");
    if ((e = cudaMemset(A->err, 0, sizeof(int))) != cudaSuccess) return fail(e, "error word");
    {
        const Tuning t_full = t;
        dose_status st = apply_schedule(A.get(), A->fwd, t, A->fwd_windowed);
        // Default tiles shrink (down to 1024 entries) until the window of x fits
        // beside the ring; past that the kernels gather x from global memory.
        while (st == DOSE_OK && A->fwd_windowed && !(tuning && tuning->tile_nnz) && !spmv_x_in_smem(A.get(), t) &&
               t.tile_nnz > 1024) {
            t.tile_nnz /= 2;
            if (!(tuning && tuning->coop_nnz)) t.coop_nnz = std::min(t.coop_nnz, t.tile_nnz);
            st = apply_schedule(A.get(), A->fwd, t, A->fwd_windowed);
        }
        if (st == DOSE_OK) st = apply_schedule(A.get(), A->adj, adj_schedule_tuning(t, at), true);
        // dose_spmv_f64 stages 8 bytes per column: if even that window does not
        // fit, it reads x from L2 and gets its own schedule with the full tiles.
        if (st == DOSE_OK && A->fwd_windowed && !spmv_f64_x_in_smem(A.get())) {
            A->fwd64.grid = A->fwd.grid;
            A->fwd64_own = true;
            st = apply_schedule(A.get(), A->fwd64, t_full, false);
        }
        // A wide column window (e.g. a multi-beam plan, whose rows span every
        // beam's spots) leaves few scatter warps beside 5120-entry tiles; the
        // default then takes 4096-entry tiles (measured on a three-beam plan with
        // a 3008-column window: 5 -> 7 scatter warps, fused pass 15 % faster).
        AdjTuning sh;
        if (st == DOSE_OK && !(tuning && tuning->adj_tile_nnz) &&
            adjoint_shape(A.get(), at, true, &sh, nullptr) && sh.scatter_warps < kAdjMinScatterWarps) {
            at.tile_nnz = 4096;
            A->adj_tuning = at;
            st = apply_schedule(A.get(), A->adj, adj_schedule_tuning(t, at), true);
        }
        if (st != DOSE_OK) {
            free_all(A.get());
            return st;
        }
    }
    if (flags & DOSE_CREATE_SELL) {
        std::string why;
        if ((e = build_sell(A.get(), col, vals.data(), sell_sigma, &why)) != cudaSuccess) {
            if (!why.empty()) {
                free_all(A.get());
                return invalid(why);
            }
            return fail(e, "SELL copy");
        }
    }
    // Row-group layout of the adjoint and fused passes (unless the caller asked for CSR).
    if (A->adj_tuning.layout != 1) {
        std::string why;
        A->rg.sched.grid = A->adj.grid;
        bool ok = build_row_groups(A.get(), A->host_row_ptr.data(), col.data(), vals.data(), &why, &e);
        if (!ok && e != cudaSuccess) {
            // the layout is optional by default: without the memory for it the
            // handle keeps the CSR passes (asked for explicitly, it is an error)
            if (e != cudaErrorMemoryAllocation || A->adj_tuning.layout == 2) return fail(e, "row-group layout");
            cudaGetLastError();
            why = "its arrays do not fit in device memory";
        }
        if (ok) {
            e = rg_schedule(A.get(), A->adj_tuning);
            if (e == cudaErrorMemoryAllocation && A->adj_tuning.layout != 2) {
                cudaGetLastError();
                free_row_groups(A.get());
                ok = false;
            } else if (e == cudaErrorInvalidValue) {
                why = "tuning.rg_tile_union is smaller than a group's union of columns";
                free_row_groups(A.get());
                ok = false;
                if (A->adj_tuning.layout == 2) {
                    free_all(A.get());
                    return invalid(why);
                }
            } else if (e != cudaSuccess) {
                return fail(e, "row-group schedule");
            }
        }
        if (A->adj_tuning.layout == 2 && !(ok && rg_active(A.get(), false))) {
            free_all(A.get());
            set_error("adj_layout = 2: the row-group layout does not apply" + (why.empty() ? std::string() : ": " + why));
            return DOSE_ERR_UNSUPPORTED;
        }
    }
    if (A->fwd.tuning.layout == 2 && !spmv_on_row_groups(A.get())) {
        free_all(A.get());
        set_error("fwd_layout = 2: dose_spmv cannot run on the row-group layout of this handle" +
                  std::string((flags & DOSE_CREATE_COMPENSATED) ? " (DOSE_CREATE_COMPENSATED sums on CSR)" : ""));
        return DOSE_ERR_UNSUPPORTED;
    }
    A->device_bytes = A->rg.bytes + (A->rg.built ? (A->rg.host.size() + 1) * 16 + schedule_bytes(A->rg.sched) : 0) +
                      A->sell.bytes + rp_alloc * 4 + col_alloc * 4 + ((flags & DOSE_CREATE_U16_INDEX) ? col16_alloc * 2 : 0) + val_alloc +
                      (fmt == DOSE_FMT_FP8E4M3_ROWSCALE ? ((size_t)nrows + 16) * 4 : 0) + x64_alloc * 8 +
                      (size_t)A->adj.grid * ncols_pad * 4 + (size_t)A->adj.grid * 8 + 4 + schedule_bytes(A->fwd) +
                      schedule_bytes(A->adj) + (A->fwd64_own ? schedule_bytes(A->fwd64) : 0);
    A->fingerprint = matrix_fingerprint(A.get());
    if ((e = cudaDeviceSynchronize()) != cudaSuccess) return fail(e, "create");
    dose_matrix* H = A.release();
    // DOSE_AUTOTUNE=cached|full in the environment tunes a handle created with
    // default knobs (dose_autotune_cached with its environment defaults)
    const char* env = std::getenv("DOSE_AUTOTUNE");
    if (!tuning && env && *env && std::strcmp(env, "off") && std::strcmp(env, "0")) {
        const dose_status st = dose_autotune_cached(H, nullptr, DOSE_AUTOTUNE_ENV, 0, nullptr, stream, nullptr, nullptr);
        if (st != DOSE_OK) {
            cudaDeviceSynchronize();
            free_all(H);
            delete H;
            return st;
        }
    }
    *out = H;
    return DOSE_OK;
}

dose_status dose_create_multibeam(const dose_csr_desc* beams, int nbeams, unsigned flags, const dose_tuning* tuning,
                                  void* stream, dose_matrix** out) {
    NvtxRange nvtx_range("dose_create_multibeam");
    if (!out) return invalid("dose_create_multibeam: out is NULL");
    *out = nullptr;
    if (!beams || nbeams < 1 || nbeams > 64) return invalid("dose_create_multibeam: nbeams must be in [1, 64]");
    const dose_csr_desc& b0 = beams[0];
    const bool f64 = b0.values == nullptr;
    uint64_t ncols = 0, nnz = 0;
    for (int b = 0; b < nbeams; ++b) {
        const dose_csr_desc& d = beams[b];
        const std::string tag = "dose_create_multibeam: beam " + std::to_string(b) + ": ";
        if (d.on_device) return invalid(tag + "beams must be host CSR arrays (on_device = 0)");
        if (d.nrows != b0.nrows) return invalid(tag + "every beam needs the same voxel grid (nrows)");
        if (d.fmt != b0.fmt) return invalid(tag + "every beam needs the same format");
        if ((d.values == nullptr) != f64) return invalid(tag + "give values_f64 for every beam, or codes for every beam");
        if (!d.row_ptr || (d.nnz && !d.col_idx) || (d.nnz && f64 && !d.values_f64))
            return invalid(tag + "null array");
        if (d.row_ptr[0] != 0 || d.row_ptr[d.nrows] != d.nnz) return invalid(tag + "row_ptr must run from 0 to nnz");
        for (uint32_t i = 0; i < d.nrows; ++i)
            if (d.row_ptr[i + 1] < d.row_ptr[i]) return invalid(tag + "row_ptr must be non-decreasing");
        for (uint64_t k = 0; k < d.nnz; ++k)
            if (d.col_idx[k] >= d.ncols) return invalid(tag + "col_idx out of range");
        if (!f64) {
            if (d.fmt == DOSE_FMT_FP8E4M3_ROWSCALE)
                return invalid(tag + "FP8 row scales of different beams cannot share a row: give values_f64");
            if (d.fmt == DOSE_FMT_U16_SCALE && (!d.scales || !b0.scales || d.scales[0] != b0.scales[0]))
                return invalid(tag + "U16 codes of beams with different scales cannot be merged: give values_f64");
        }
        ncols += d.ncols;
        nnz += d.nnz;
    }
    if (ncols > 0xFFFFFFFFull || nnz >= (1ull << 32)) return invalid("dose_create_multibeam: merged matrix too large");
    // Row i of the plan = row i of beam 0, then of beam 1, ... with beam b's
    // columns moved up by the spots of the beams before it.
    const uint32_t nrows = b0.nrows;
    const size_t es = f64 ? 8 : value_bytes(b0.fmt);
    std::vector<uint32_t> rp(nrows + 1, 0), col(nnz), off(nbeams, 0);
    std::vector<unsigned char> val(nnz * es);
    for (int b = 1; b < nbeams; ++b) off[b] = off[b - 1] + beams[b - 1].ncols;
    for (uint32_t i = 0; i < nrows; ++i) {
        uint32_t len = 0;
        for (int b = 0; b < nbeams; ++b) len += beams[b].row_ptr[i + 1] - beams[b].row_ptr[i];
        rp[i + 1] = rp[i] + len;
    }
    for (uint32_t i = 0; i < nrows; ++i) {
        uint32_t k = rp[i];
        for (int b = 0; b < nbeams; ++b) {
            const dose_csr_desc& d = beams[b];
            for (uint32_t q = d.row_ptr[i]; q < d.row_ptr[i + 1]; ++q, ++k) {
                col[k] = d.col_idx[q] + off[b];
                const unsigned char* src = f64 ? reinterpret_cast<const unsigned char*>(d.values_f64)
                                               : static_cast<const unsigned char*>(d.values);
                std::memcpy(val.data() + (size_t)k * es, src + (size_t)q * es, es);
            }
        }
    }
    dose_csr_desc m{};
    m.nrows = nrows;
    m.ncols = (uint32_t)ncols;
    m.nnz = nnz;
    m.row_ptr = rp.data();
    m.col_idx = col.data();
    m.fmt = b0.fmt;
    m.on_device = 0;
    if (f64) {
        m.values_f64 = reinterpret_cast<const double*>(val.data());
    } else {
        m.values = val.data();
        m.scales = b0.scales;
    }
    return dose_create_matrix(&m, flags, tuning, stream, out);
}

dose_status dose_destroy(dose_matrix* A) {
    if (!A) return DOSE_OK;
    cudaDeviceSynchronize();
    free_all(A);
    delete A;
    return DOSE_OK;
}

dose_status dose_spmv(const dose_matrix* A, const float* x, float* d, void* stream) {
    NvtxRange nvtx_range("dose_spmv");
    if (!A) return invalid("dose_spmv: null matrix");
    if (A->nrows && !d) return invalid("dose_spmv: d is NULL");
    if (A->ncols && !x) return invalid("dose_spmv: x is NULL");
    cudaError_t e = (A->flags & DOSE_CREATE_SELL) ? launch_spmv_sell(A, x, d, as_stream(stream))
                    : spmv_on_row_groups(A)      ? launch_rg_spmv(A, x, d, as_stream(stream))
                                                 : launch_spmv(A, x, d, as_stream(stream));
    return e == cudaSuccess ? DOSE_OK : cuda_fail(e, "dose_spmv launch");
}

dose_status dose_spmv_f64(const dose_matrix* A, const double* x, double* d, unsigned flags, void* stream) {
    NvtxRange nvtx_range("dose_spmv_f64");
    if (!A) return invalid("dose_spmv_f64: null matrix");
    if (flags & ~DOSE_SPMV_F64_NATIVE) return invalid("dose_spmv_f64: unknown flags");
    if (A->nrows && !d) return invalid("dose_spmv_f64: d is NULL");
    if (A->ncols && !x) return invalid("dose_spmv_f64: x is NULL");
    if ((reinterpret_cast<uintptr_t>(x) | reinterpret_cast<uintptr_t>(d)) & 7u)
        return invalid("dose_spmv_f64: x and d must be 8-byte aligned");
    cudaError_t e = launch_spmv_f64(A, x, d, (flags & DOSE_SPMV_F64_NATIVE) != 0, as_stream(stream));
    return e == cudaSuccess ? DOSE_OK : cuda_fail(e, "dose_spmv_f64 launch");
}

}  // extern "C"

namespace dose {
// dose_spmv runs on the row-group layout unless the caller asked for CSR
// (fwd_layout = 1), the handle sums long rows with compensation (a CSR path),
// or the layout is missing or its ring does not fit beside the window of x.
bool spmv_on_row_groups(const dose_matrix* A) {
    return A->fwd.tuning.layout != 1 && !(A->flags & DOSE_CREATE_COMPENSATED) && rg_spmv_applies(A, nullptr, nullptr);
}

dose_status adjoint_supported(const dose_matrix* A, bool quad, const float* const* vecs, int nvec) {
    for (int k = 0; k < nvec; ++k)
        if (vecs[k] && (reinterpret_cast<uintptr_t>(vecs[k]) & 15u))
            return invalid("per-row vectors (p, w, r) must be 16-byte aligned");
    if (rg_active(A, quad)) return DOSE_OK;
    if (quad && A->adj.wwidth > kXSmemMaxCols) {
        set_error("the fused objective pass keeps each CTA's window of x in shared memory: the column window (" +
                  std::to_string(A->adj.wwidth) + ") must be <= 16384");
        return DOSE_ERR_UNSUPPORTED;
    }
    if (!adjoint_shape(A, A->adj_tuning, quad, nullptr, nullptr)) {
        set_error("per-warp gradient accumulators of the column window (" + std::to_string(A->adj.wwidth) +
                  " floats) do not fit in shared memory");
        return DOSE_ERR_UNSUPPORTED;
    }
    for (int k = 0; k < nvec; ++k)
        if (vecs[k] && (reinterpret_cast<uintptr_t>(vecs[k]) & 15u))
            return invalid("per-row vectors (p, w, r) must be 16-byte aligned");
    return DOSE_OK;
}
}  // namespace dose

extern "C" {

dose_status dose_adjoint(const dose_matrix* A, const float* r, float* g, void* stream) {
    NvtxRange nvtx_range("dose_adjoint");
    if (!A) return invalid("dose_adjoint: null matrix");
    if (A->nrows && !r) return invalid("dose_adjoint: r is NULL");
    if (A->ncols && !g) return invalid("dose_adjoint: g is NULL");
    const float* vv[1] = {r};
    dose_status st = adjoint_supported(A, false, vv, 1);
    if (st != DOSE_OK) return st;
    cudaError_t e = launch_adjoint(A, ADJ_MODE_ADJOINT, nullptr, nullptr, nullptr, r, nullptr, nullptr, g, nullptr,
                                   0.f, as_stream(stream));
    return e == cudaSuccess ? DOSE_OK : cuda_fail(e, "dose_adjoint launch");
}

dose_status dose_fwd_adj_quadratic(const dose_matrix* A, const float* x, const float* p, const float* w, float* d,
                                   double* f, float* g, void* stream) {
    NvtxRange nvtx_range("dose_fwd_adj_quadratic");
    if (!A) return invalid("dose_fwd_adj_quadratic: null matrix");
    if (!f || (A->ncols && (!x || !g)) || (A->nrows && (!p || !w)))
        return invalid("dose_fwd_adj_quadratic: null pointer argument");
    const float* vv[2] = {p, w};
    dose_status st = adjoint_supported(A, true, vv, 2);
    if (st != DOSE_OK) return st;
    cudaError_t e = launch_adjoint(A, ADJ_MODE_QUADRATIC, x, p, w, nullptr, d, f, g, nullptr, 0.f, as_stream(stream));
    return e == cudaSuccess ? DOSE_OK : cuda_fail(e, "dose_fwd_adj_quadratic launch");
}

dose_status dose_pg_step(const dose_matrix* A, float* x, const float* p, const float* w, float eta, double* f,
                         float* g, void* stream) {
    NvtxRange nvtx_range("dose_pg_step");
    if (!A) return invalid("dose_pg_step: null matrix");
    if (!f || (A->ncols && !x) || (A->nrows && (!p || !w))) return invalid("dose_pg_step: null pointer argument");
    if (!(eta >= 0.0f) || std::isinf(eta)) return invalid("dose_pg_step: eta must be finite and >= 0");
    const float* vv[2] = {p, w};
    dose_status st = adjoint_supported(A, true, vv, 2);
    if (st != DOSE_OK) return st;
    cudaError_t e = launch_adjoint(A, ADJ_MODE_QUADRATIC, x, p, w, nullptr, nullptr, f, g, x, eta, as_stream(stream));
    return e == cudaSuccess ? DOSE_OK : cuda_fail(e, "dose_pg_step launch");
}

dose_status dose_spmv_batched(const dose_matrix* const* A, int count, const float* const* X, float* const* D,
                              int nvec, void* stream) {
    NvtxRange nvtx_range("dose_spmv_batched");
    if (count < 0 || count > 4096) return invalid("dose_spmv_batched: count must be in [0, 4096]");
    if (count == 0) return DOSE_OK;
    if (!A || !X || !D) return invalid("dose_spmv_batched: null array");
    if (nvec < 1 || nvec > 16) return invalid("dose_spmv_batched: nvec must be in [1, 16]");
    for (int m = 0; m < count; ++m) {
        if (!A[m]) return invalid("dose_spmv_batched: null matrix " + std::to_string(m));
        if ((A[m]->ncols && !X[m]) || (A[m]->nrows && !D[m]))
            return invalid("dose_spmv_batched: null vector for matrix " + std::to_string(m));
    }
    std::string why;
    cudaError_t e = launch_spmm_batched(A, count, X, D, nvec, as_stream(stream), &why);
    if (!why.empty()) {
        set_error(why);
        return DOSE_ERR_UNSUPPORTED;
    }
    return e == cudaSuccess ? DOSE_OK : cuda_fail(e, "dose_spmv_batched launch");
}

dose_status dose_spmv_batched_plan(const dose_matrix* const* A, int count, int nvec, int* layout, int* launches) {
    if (!layout || !launches) return invalid("dose_spmv_batched_plan: null output");
    if (count < 0 || count > 4096) return invalid("dose_spmv_batched_plan: count must be in [0, 4096]");
    if (nvec < 1 || nvec > 16) return invalid("dose_spmv_batched_plan: nvec must be in [1, 16]");
    if (count && !A) return invalid("dose_spmv_batched_plan: null array");
    for (int m = 0; m < count; ++m)
        if (!A[m]) return invalid("dose_spmv_batched_plan: null matrix " + std::to_string(m));
    *layout = 0;
    *launches = 0;
    if (count) spmm_batched_plan(A, count, layout, launches);
    return DOSE_OK;
}

dose_status dose_matrix_info(const dose_matrix* A, dose_info* out) {
    if (!A || !out) return invalid("dose_matrix_info: null argument");
    std::memset(out, 0, sizeof(*out));
    out->nrows = A->nrows;
    out->ncols = A->ncols;
    out->nnz = A->nnz;
    out->fmt = A->fmt;
    out->flags = A->flags;
    out->fingerprint = A->fingerprint;
    out->spmv_layout = (A->flags & DOSE_CREATE_SELL) ? 3u : spmv_on_row_groups(A) ? 2u : 1u;
    out->rg_spmv_bytes = out->spmv_layout == 2 ? rg_spmv_bytes(A) : 0;
    out->n_stages = A->fwd.n_stages;
    out->n_coop_rows = A->fwd.n_coop_rows;
    std::memcpy(out->lanes_hist, A->fwd.lanes_hist, sizeof(out->lanes_hist));
    out->grid = A->fwd.grid;
    out->block = 32 * (A->fwd.tuning.consumer_warps + 1);
    out->adj_n_stages = A->adj.n_stages;
    AdjTuning sh;
    if (adjoint_shape(A, A->adj_tuning, true, &sh, nullptr) && A->adj.wwidth <= kXSmemMaxCols)
        out->adj_block_fused = 32 * (1 + sh.forward_warps + sh.scatter_warps);
    if (adjoint_shape(A, A->adj_tuning, false, &sh, nullptr)) out->adj_block_adjoint = 32 * (1 + sh.scatter_warps);
    out->adj_window = A->adj.wwidth;
    out->fwd_window = A->fwd_windowed ? A->fwd.wwidth : 0;
    out->max_row_len = A->max_row_len;
    out->device_bytes = A->device_bytes;
    const uint64_t vb = value_bytes(A->fmt);
    const uint64_t nz = A->nnz, nr = A->nrows, nc = A->ncols;
    const uint64_t rs = A->fmt == DOSE_FMT_FP8E4M3_ROWSCALE ? 4 * nr : 0;  // row scales
    // Algorithmic bytes: every stored byte of A once, the vectors once.
    const uint64_t ib = (A->flags & DOSE_CREATE_U16_INDEX) ? 2 : 4;  // column index bytes read by dose_spmv
    out->spmv_bytes = (vb + ib) * nz + 4 * (nr + 1) + rs + 4 * nr + 4 * nc;
    if (A->flags & DOSE_CREATE_SELL) {
        // padded entries, one perm word per chunk slot, 8 bytes per chunk descriptor
        out->sell_entries = A->sell.entries;
        out->spmv_bytes = (vb + ib) * A->sell.entries + 4ull * 32 * A->sell.nchunks + 8ull * A->sell.nchunks + rs +
                          4 * nr + 4 * nc;
    }
    out->adjoint_bytes = (vb + 4) * nz + 4 * (nr + 1) + rs + 4 * nr + 4 * nc;
    out->fused_bytes = (vb + 4) * nz + 4 * (nr + 1) + rs + 8 * nr + 4 * nc + 4 * nc + 8;
    // FP64 vectors: 8-byte x read once, 8-byte d written once (for F16 values and
    // 32-bit indices this is 6 nnz + 12 nr + 8 nc + 4, the traffic model of Sec. V)
    out->spmv_f64_bytes = (vb + ib) * nz + 4 * (nr + 1) + rs + 8 * nr + 8 * nc;
    out->scale = A->fmt == DOSE_FMT_U16_SCALE ? A->scale : 0.f;
    export_tuning(A->fwd.tuning, A->adj_tuning, &out->tuning);
    out->tuning.sell_sigma = A->sell.sigma;
    out->adj_layout_fused = out->adj_block_fused ? 1 : 0;
    out->adj_layout_adjoint = out->adj_block_adjoint ? 1 : 0;
    if (A->rg.built) {
        out->rg_groups = A->rg.host.size();
        out->rg_union_entries = A->rg.n_union;
        out->rg_window = A->rg.sched.wwidth;
        out->rg_index_bytes = A->rg.iw;
        out->tuning.rg_tile_union = A->rg.tile_u;
        size_t smem = 0;
        out->rg_warps_fused = rg_shape(A, A->adj_tuning, true, &smem);
        if (rg_active(A, true)) {
            out->adj_layout_fused = 2;
            out->adj_block_fused = 32 * (1 + out->rg_warps_fused);
            out->fused_bytes = rg_fused_bytes(A, false);
        }
        if (rg_active(A, false)) {
            out->adj_layout_adjoint = 2;
            out->adj_block_adjoint = 32 * (1 + rg_shape(A, A->adj_tuning, false, &smem));
            out->adjoint_bytes = rg_adjoint_bytes(A);
        }
    }
    return DOSE_OK;
}

dose_status dose_set_tuning(dose_matrix* A, const dose_tuning* tuning) {
    NvtxRange nvtx_range("dose_set_tuning");
    if (!A) return invalid("dose_set_tuning: null matrix");
    Tuning t = A->fwd.tuning;
    AdjTuning at = A->adj_tuning;
    merge_tuning(t, at, tuning);
    dose_status st = check_tuning(A, t);
    if (st == DOSE_OK) st = check_adj_tuning(at);
    if (st != DOSE_OK) return st;
    cudaError_t e = cudaDeviceSynchronize();
    if (e != cudaSuccess) return cuda_fail(e, "dose_set_tuning");
    st = apply_schedule(A, A->fwd, t, A->fwd_windowed);
    if (st == DOSE_OK && A->fwd64_own) st = apply_schedule(A, A->fwd64, t, false);
    if (st != DOSE_OK) return st;
    if (at.layout == 2 && !A->rg.built) return invalid("adj_layout = 2: the handle has no row-group layout");
    if (t.layout == 2 && (!A->rg.built || (A->flags & DOSE_CREATE_COMPENSATED)))
        return invalid("fwd_layout = 2: dose_spmv cannot run on the row-group layout of this handle");
    const AdjTuning old_at = A->adj_tuning;
    A->adj_tuning = at;
    if (A->rg.built && (at.rg_tile_u != old_at.rg_tile_u || at.rg_tile_rows != old_at.rg_tile_rows)) {
        e = rg_schedule(A, at);
        if (e == cudaErrorInvalidValue) {
            A->adj_tuning = old_at;
            rg_schedule(A, old_at);
            return invalid("tuning.rg_tile_union is smaller than a group's union of columns");
        }
        if (e != cudaSuccess) return cuda_fail(e, "row-group schedule");
    }
    return apply_schedule(A, A->adj, adj_schedule_tuning(t, at), true);
}

dose_status dose_device_status(const dose_matrix* A, void* stream) {
    if (!A) return invalid("dose_device_status: null matrix");
    int h = 0;
    cudaError_t e = cudaMemcpyAsync(&h, A->err, sizeof(int), cudaMemcpyDeviceToHost, as_stream(stream));
    if (e == cudaSuccess) e = cudaStreamSynchronize(as_stream(stream));
    if (e != cudaSuccess) return cuda_fail(e, "dose_device_status");
    if (h != 0) {
        cudaMemsetAsync(A->err, 0, sizeof(int), as_stream(stream));
        cudaStreamSynchronize(as_stream(stream));
        if (h == kErrBounds) {
            set_error("a kernel met an index outside its buffer and skipped that work (debug-checked build)");
            return DOSE_ERR_BOUNDS;
        }
        set_error(h == kErrTimeoutFull ? "a consumer warp timed out waiting for staged data"
                                       : "the producer timed out waiting for a free stage slot");
        return DOSE_ERR_TIMEOUT;
    }
    return DOSE_OK;
}


}  // extern "C"
