// Host side of the row-group layout of the adjoint and fused objective passes
// (the kernels are in rg_kernel.cu).
//
// The gradient of the dose objective needs g = A^T r every iteration (Sec. I;
// Sec. II-A: A fixed, x changing).  Scattering a_ij r_i entry by entry costs a
// shared-memory read-modify-write per entry.  Neighbouring voxels of a dose
// matrix see almost the same spots, so the library groups up to four
// consecutive non-empty rows and stores, for the union of their columns, the
// four rows' values side by side (stored zeros where a row has no entry).  On
// the clinical pencil beam the union holds 1.17 times the entries of its rows,
// so the layout takes 3.5 instead of 6 bytes per entry (u16 values, 32-bit
// indices) and one gradient update serves four entries.
//
// Built once at create from the validated host CSR and the stored codes; the
// stage cut and the dealing to CTAs are redone when the tuning changes.
#include <algorithm>
#include <cstring>
#include <string>
#include <vector>

#include "dose_internal.cuh"

namespace dose {
namespace {

constexpr uint32_t kRgTileGroups = 64;    // groups per stage (slot's record area)
constexpr uint32_t kRgGroupSpan = 255;    // rows of one group lie within this distance
constexpr uint64_t kRgGroupCost = 256;    // dealing cost of a group beyond its bytes

cudaError_t rg_upload(void** dst, const void* src, size_t bytes, size_t alloc_bytes) {
    alloc_bytes = std::max<size_t>(alloc_bytes, 16);
    cudaError_t e = dev_malloc(dst, alloc_bytes);
    if (e != cudaSuccess) return e;
    e = cudaMemset(*dst, 0, alloc_bytes);
    if (e != cudaSuccess) return e;
    if (bytes) e = cudaMemcpy(*dst, src, bytes, cudaMemcpyHostToDevice);
    return e;
}

void free_rg_schedule(DevSchedule& D) {
    cudaFree(D.desc);
    cudaFree(D.cta_begin);
    cudaFree(D.wlo);
    D.desc = nullptr;
    D.cta_begin = nullptr;
    D.wlo = nullptr;
    D.n_stages = 0;
    D.wwidth = 0;
}

// Order the union columns of one group for the kernel: position p = 32 it + l
// is read by lane l in step it.  The gather of x and the update of the
// gradient accumulator of step it touch shared-memory bank c mod 32 of each of
// the 32 columns (every window starts on a multiple of 32 columns), so the
// columns of one step should have distinct residues mod 32.  Greedy: residues
// with the most columns first; each column goes to the step with the most free
// positions among those that do not hold its residue yet (a step that holds it
// only when all do).  The order changes only the rounding order of the
// forward sum, never which values are added.
void bank_order(std::vector<uint32_t>& cols, std::vector<uint32_t>& perm) {
    const uint32_t nu = (uint32_t)cols.size();
    perm.resize(nu);
    if (nu <= 1) {
        for (uint32_t i = 0; i < nu; ++i) perm[i] = i;
        return;
    }
    const uint32_t steps = (nu + 31) / 32;
    std::vector<uint32_t> cap(steps, 32), has(steps, 0);
    cap[steps - 1] = nu - 32 * (steps - 1);
    std::vector<std::vector<uint32_t>> bucket(32);
    for (uint32_t i = 0; i < nu; ++i) bucket[cols[i] & 31u].push_back(i);
    uint32_t bank[32];
    for (uint32_t b = 0; b < 32; ++b) bank[b] = b;
    std::stable_sort(bank, bank + 32, [&](uint32_t a, uint32_t b) { return bucket[a].size() > bucket[b].size(); });
    std::vector<std::vector<uint32_t>> slot(steps);
    for (uint32_t bi = 0; bi < 32; ++bi) {
        const uint32_t b = bank[bi];
        std::sort(bucket[b].begin(), bucket[b].end(), [&](uint32_t x, uint32_t y) { return cols[x] < cols[y]; });
        for (uint32_t i : bucket[b]) {
            int best = -1;
            for (uint32_t s = 0; s < steps; ++s)
                if (cap[s] && !((has[s] >> b) & 1u) && (best < 0 || cap[s] > cap[best])) best = (int)s;
            if (best < 0)
                for (uint32_t s = 0; s < steps; ++s)
                    if (cap[s] && (best < 0 || cap[s] > cap[best])) best = (int)s;
            slot[best].push_back(i);
            --cap[best];
            has[best] |= 1u << b;
        }
    }
    uint32_t p = 0;
    for (uint32_t s = 0; s < steps; ++s) {
        std::sort(slot[s].begin(), slot[s].end(), [&](uint32_t x, uint32_t y) { return cols[x] < cols[y]; });
        for (uint32_t i : slot[s]) perm[p++] = i;
    }
}

}  // namespace

// Union entries one stage holds by default: about 40 KB of union columns and
// values (each stage costs a ring round trip, so stages carry as many bytes as
// two ring slots beside the accumulators allow).
static uint32_t rg_default_tile_u(uint32_t esize, uint32_t iw) {
    const uint32_t per = iw + 4 * esize;
    uint32_t t = 40960 / per / 32 * 32;
    return std::max<uint32_t>(512, std::min<uint32_t>(8192, t));
}

void free_row_groups(dose_matrix* A) {
    RowGroups& R = A->rg;
    cudaFree(R.ucol);
    cudaFree(R.uval);
    cudaFree(R.grp);
    cudaFree(R.mask);
    cudaFree(R.f_rows);
    cudaFree(R.ticket);
    R.f_rows = nullptr;
    R.ticket = nullptr;
    free_rg_schedule(R.sched);
    R.ucol = R.uval = nullptr;
    R.grp = nullptr;
    R.mask = nullptr;
    R.built = false;
    R.bytes = 0;
    R.n_union = 0;
    R.host.clear();
    R.host.shrink_to_fit();
}

bool build_row_groups(dose_matrix* A, const uint32_t* rp, const uint32_t* col, const unsigned char* vals,
                      std::string* why, cudaError_t* err) {
    *err = cudaSuccess;
    RowGroups& R = A->rg;
    const uint32_t nrows = A->nrows, ncols = A->ncols;
    const uint32_t es = value_bytes(A->fmt);
    R.iw = ncols <= 65536u ? 2u : 4u;
    // A single row must fit one stage at the largest union tile a caller may set.
    const uint32_t umax = 4096;
    if (A->max_row_len > umax) {
        *why = "a row has " + std::to_string(A->max_row_len) + " entries; row groups hold at most " +
               std::to_string(umax) + " columns";
        return false;
    }
    std::vector<RgHostGroup> G;
    std::vector<uint32_t> ucol;
    std::vector<unsigned char> uval;
    ucol.reserve((size_t)(A->nnz / 3 + 64));
    uval.reserve((size_t)(A->nnz / 3 + 64) * 4 * es);
    std::vector<uint32_t> stamp(std::max<uint32_t>(ncols, 1), 0xFFFFFFFFu), pos(std::max<uint32_t>(ncols, 1), 0);
    std::vector<uint32_t> U, perm;           // union of the open group, in order of first appearance
    std::vector<unsigned char> V, Vp;        // its values: 4 per union column
    RgHostGroup cur{};
    uint32_t nrow_in = 0, gid = 0;
    auto close = [&]() {
        if (!nrow_in) return;
        bank_order(U, perm);
        const uint32_t nu = (uint32_t)U.size();
        cur.uoff = (uint32_t)ucol.size();
        cur.nu = nu;
        cur.lo = 0xFFFFFFFFu;
        cur.hi = 0;
        const size_t rec = 4 * (size_t)es;
        Vp.resize(V.size());
        for (uint32_t k = 0; k < nu; ++k) {
            const uint32_t c = U[perm[k]];
            ucol.push_back(c);
            cur.lo = std::min(cur.lo, c);
            cur.hi = std::max(cur.hi, c);
            std::memcpy(Vp.data() + k * rec, V.data() + (size_t)perm[k] * rec, rec);
        }
        uval.insert(uval.end(), Vp.begin(), Vp.begin() + (size_t)nu * rec);
        for (uint32_t s = nrow_in; s < 4; ++s) cur.row[s] = 0xFFFFFFFFu;
        G.push_back(cur);
        nrow_in = 0;
        U.clear();
        V.clear();
        ++gid;
    };
    for (uint32_t r = 0; r < nrows; ++r) {
        const uint32_t kb = rp[r], ke = rp[r + 1], len = ke - kb;
        if (!len) continue;
        if (nrow_in) {
            bool join = nrow_in < 4 && r - cur.row[0] <= kRgGroupSpan;
            if (join) {
                uint32_t fresh = 0;
                for (uint32_t k = kb; k < ke; ++k) fresh += stamp[col[k]] != gid;
                const uint32_t nu = (uint32_t)U.size() + fresh;
                // the union stays in registers, and grows by at most half of the
                // larger of the group and the row (rows that see other spots, e.g.
                // across the end of a voxel line, start a new group)
                join = nu <= kRgMaxUnionReg && 2 * (uint64_t)nu <= 3 * (uint64_t)std::max<size_t>(U.size(), len);
            }
            if (!join) close();
        }
        const uint32_t slot = nrow_in++;
        cur.row[slot] = r;
        for (uint32_t k = kb; k < ke; ++k) {
            const uint32_t c = col[k];
            if (stamp[c] != gid) {
                stamp[c] = gid;
                pos[c] = (uint32_t)U.size();
                U.push_back(c);
                V.resize(V.size() + 4 * (size_t)es, 0);
            }
            std::memcpy(V.data() + ((size_t)pos[c] * 4 + slot) * es, vals + (size_t)k * es, es);
        }
    }
    close();

    // device arrays that do not depend on the stage cut
    R.n_union = ucol.size();
    cudaError_t e;
    const size_t nu_pad = (R.n_union + 7) / 8 * 8 + 16;  // copy windows reach whole 16-byte pieces
    if (R.iw == 2) {
        std::vector<uint16_t> c16(ucol.size());
        for (size_t k = 0; k < ucol.size(); ++k) c16[k] = (uint16_t)ucol[k];
        e = rg_upload(&R.ucol, c16.data(), c16.size() * 2, nu_pad * 2);
    } else {
        e = rg_upload(&R.ucol, ucol.data(), ucol.size() * 4, nu_pad * 4);
    }
    if (e == cudaSuccess) e = rg_upload(&R.uval, uval.data(), uval.size(), nu_pad * 4 * es);
    const size_t nwords = ((size_t)nrows + 31) / 32;
    std::vector<uint32_t> mask((nwords + 3) / 4 * 4 + 4, 0);
    for (uint32_t r = 0; r < nrows; ++r)
        if (rp[r + 1] > rp[r]) mask[r >> 5] |= 1u << (r & 31);
    if (e == cudaSuccess)
        e = rg_upload(reinterpret_cast<void**>(&R.mask), mask.data(), mask.size() * 4, mask.size() * 4);
    // finalize blocks of the fused pass: four 256-thread blocks per SM (one wave)
    R.nblk_rows = 4 * std::max<uint32_t>(R.sched.grid, 1);
    if (e == cudaSuccess)
        e = rg_upload(reinterpret_cast<void**>(&R.f_rows), nullptr, 0, (size_t)R.nblk_rows * 8);
    if (e == cudaSuccess) e = rg_upload(reinterpret_cast<void**>(&R.ticket), nullptr, 0, 16);
    if (e != cudaSuccess) {
        *err = e;
        free_row_groups(A);
        return false;
    }
    R.bytes = nu_pad * (R.iw + 4 * es) + mask.size() * 4 + (size_t)R.nblk_rows * 8 + 16;
    R.host = std::move(G);
    R.built = true;
    return true;
}

// Cut the groups into stages and deal them to CTAs (windowed); upload the
// stage descriptors and the group records (their row offsets are relative to
// each stage's first row).
cudaError_t rg_schedule(dose_matrix* A, const AdjTuning& t) {
    RowGroups& R = A->rg;
    const std::vector<RgHostGroup>& G = R.host;
    const uint32_t ng = (uint32_t)G.size();
    const uint32_t es = value_bytes(A->fmt);
    const uint32_t tile_rows = t.rg_tile_rows;
    uint32_t span_max = 0, nu_max = 0;
    for (const RgHostGroup& g : G) {
        span_max = std::max(span_max, g.hi - g.lo);
        nu_max = std::max(nu_max, g.nu);
    }
    // the default grows to the largest group's union; a caller's tile must hold it
    const uint32_t tile_u = t.rg_tile_u ? t.rg_tile_u : std::max(rg_default_tile_u(es, R.iw), (nu_max + 31) / 32 * 32);
    if (nu_max > tile_u) return cudaErrorInvalidValue;
    const uint64_t span_cap = (uint64_t)span_max * 3 / 2;
    const uint32_t nvec_bytes = 8 + (A->fmt == DOSE_FMT_FP8E4M3_ROWSCALE ? 4 : 0);
    // Stages hold runs of consecutive groups; rows without entries are not staged
    // (the finalize kernel handles them), so a stage's rows run from its first
    // group's first row to its last group's last row.
    auto last_row = [&](const RgHostGroup& q) {
        uint32_t last = q.row[0];
        for (int s = 1; s < 4; ++s)
            if (q.row[s] != 0xFFFFFFFFu) last = q.row[s];
        return last;
    };
    auto cut = [&](bool tight, Schedule& S, std::vector<DealItem>& items) {
        uint32_t g = 0;
        while (g < ng) {
            StageDesc D{};
            D.row0 = G[g].row[0];
            D.ne0 = g;
            D.nz0 = G[g].uoff;
            uint32_t u = 0, lo = 0xFFFFFFFFu, hi = 0, row1 = D.row0 + 1;
            while (g < ng) {
                const RgHostGroup& q = G[g];
                const uint32_t last = last_row(q);
                if (last >= D.row0 + tile_rows || u + q.nu > tile_u || g - D.ne0 >= kRgTileGroups) break;
                if (g > D.ne0) {
                    // as the CSR adjoint schedule: a stage whose column range would
                    // more than double (the voxel order wrapping across the beam)
                    // ends here, so that one wide stage cannot widen every window
                    const uint32_t nlo = std::min(lo, q.lo), nhi = std::max(hi, q.hi);
                    if (nhi - nlo > 2 * std::max(hi - lo, q.hi - q.lo) + 64 && (tight || nhi - nlo > span_cap))
                        break;
                }
                lo = std::min(lo, q.lo);
                hi = std::max(hi, q.hi);
                u += q.nu;
                row1 = last + 1;
                ++g;
            }
            D.row1 = row1;
            D.ne1 = g;
            D.nz1 = D.nz0 + u;
            const uint32_t rows = D.row1 - D.row0;
            DealItem it{(uint32_t)S.desc.size(), (uint32_t)S.desc.size() + 1, lo, hi,
                        (uint64_t)u * (R.iw + 4 * es) + 16ull * (D.ne1 - D.ne0) + (uint64_t)rows * nvec_bytes +
                            kRgGroupCost * (D.ne1 - D.ne0)};
            S.desc.push_back(D);
            items.push_back(it);
        }
    };
    Schedule S;
    {
        Schedule S1, S2;
        std::vector<DealItem> i1, i2;
        cut(false, S1, i1);
        cut(true, S2, i2);
        deal_items(S1, i1, R.sched.grid, A->ncols, true, true);
        deal_items(S2, i2, R.sched.grid, A->ncols, true, true);
        S = S2.wwidth < S1.wwidth ? std::move(S2) : std::move(S1);
    }
    std::vector<uint4> rec(std::max<uint32_t>(ng, 1) + 1, make_uint4(0, 0, 0, 0));
    for (const StageDesc& D : S.desc)
        for (uint32_t g = D.ne0; g < D.ne1; ++g) {
            uint32_t off[4];
            for (int s = 0; s < 4; ++s) off[s] = G[g].row[s] == 0xFFFFFFFFu ? 0xFFFFu : G[g].row[s] - D.row0;
            rec[g] = make_uint4(G[g].uoff, G[g].nu, off[0] | (off[1] << 16), off[2] | (off[3] << 16));
        }
    free_rg_schedule(R.sched);
    cudaFree(R.grp);
    R.grp = nullptr;
    cudaError_t e;
    if ((e = rg_upload(reinterpret_cast<void**>(&R.grp), rec.data(), rec.size() * sizeof(uint4),
                       rec.size() * sizeof(uint4))) != cudaSuccess ||
        (e = rg_upload(reinterpret_cast<void**>(&R.sched.desc), S.desc.data(), S.desc.size() * sizeof(StageDesc),
                       (S.desc.size() + 1) * sizeof(StageDesc))) != cudaSuccess ||
        (e = rg_upload(reinterpret_cast<void**>(&R.sched.cta_begin), S.cta_begin.data(), S.cta_begin.size() * 4,
                       S.cta_begin.size() * 4)) != cudaSuccess ||
        (e = rg_upload(reinterpret_cast<void**>(&R.sched.wlo), S.wlo.data(), S.wlo.size() * 4, S.wlo.size() * 4)) !=
            cudaSuccess)
        return e;
    R.sched.wwidth = S.wwidth;
    R.sched.n_stages = (uint32_t)S.desc.size();
    R.tile_u = tile_u;
    R.tile_g = kRgTileGroups;
    R.tile_rows = tile_rows;
    return cudaSuccess;
}

}  // namespace dose
