// Autotuner of the schedule knobs and its on-disk cache.
//
// The paper picks its kernels' execution configuration by sweeping it on the
// target GPU (Sec. V-A, Fig. 4).  This file does the same for the knobs of
// dose_tuning: it times candidate schedules of the calls a handle is used for
// (dose_spmv; dose_fwd_adj_quadratic on either adjoint layout; dose_spmv_batched
// with 16 vectors), keeps the fastest and stores the result in a JSON file keyed
// by a fingerprint of the matrix's structure and the GPU's name, so that a
// later process with the same matrix on the same kind of GPU applies the knobs
// without timing anything.  Knobs never change which rows an output depends on;
// they may change the last bits of FP32 sums.
#include <cuda_runtime.h>

#include <sys/stat.h>
#include <unistd.h>

#include <algorithm>
#include <cerrno>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <string>
#include <utility>
#include <vector>

#include "dose_internal.cuh"
#include "nvtx_range.cuh"

namespace dose {
namespace {

dose_status bad(const std::string& msg, dose_status st = DOSE_ERR_INVALID_ARG) {
    set_error(msg);
    return st;
}

// ------------------------------------------------------------ fingerprint
// FNV-1a (64-bit) over the matrix's shape, format and creation flags, its row
// pointers and each non-empty row's lowest and highest column: the inputs the
// schedules are cut from.  Values do not enter (no knob depends on them).
struct Fnv {
    uint64_t h = 0xcbf29ce484222325ull;
    void bytes(const void* p, size_t n) {
        const unsigned char* c = static_cast<const unsigned char*>(p);
        for (size_t i = 0; i < n; ++i) {
            h ^= c[i];
            h *= 0x100000001b3ull;
        }
    }
    void u32(uint32_t v) { bytes(&v, 4); }
    void u64(uint64_t v) { bytes(&v, 8); }
};

uint64_t fingerprint_of(uint32_t nrows, uint32_t ncols, uint64_t nnz, uint32_t fmt, uint32_t flags,
                        const uint32_t* rp, const uint32_t* cmin, const uint32_t* cmax) {
    Fnv f;
    f.bytes("dose-fp1", 8);
    f.u32(nrows);
    f.u32(ncols);
    f.u64(nnz);
    f.u32(fmt);
    f.u32(flags);
    f.bytes(rp, (size_t)(nrows + 1) * 4);
    for (uint32_t i = 0; i < nrows; ++i)
        if (rp[i + 1] > rp[i]) {
            f.u32(cmin[i]);
            f.u32(cmax[i]);
        }
    return f.h;
}

std::string hex64(uint64_t v) {
    char b[17];
    std::snprintf(b, sizeof(b), "%016llx", (unsigned long long)v);
    return b;
}

std::string gpu_name(int device) {
    cudaDeviceProp p;
    if (cudaGetDeviceProperties(&p, device) != cudaSuccess) return "unknown GPU";
    return std::string(p.name) + " (" + std::to_string(p.multiProcessorCount) + " SMs, sm_" +
           std::to_string(p.major) + std::to_string(p.minor) + ")";
}

// The cache file: the caller's path, else $DOSE_AUTOTUNE_CACHE, else
// $XDG_CACHE_HOME/dose/autotune.json, else $HOME/.cache/dose/autotune.json.
std::string cache_path(const char* given) {
    if (given && *given) return given;
    if (const char* e = std::getenv("DOSE_AUTOTUNE_CACHE"); e && *e) return e;
    if (const char* x = std::getenv("XDG_CACHE_HOME"); x && *x) return std::string(x) + "/dose/autotune.json";
    if (const char* h = std::getenv("HOME"); h && *h) return std::string(h) + "/.cache/dose/autotune.json";
    return "dose_autotune.json";
}

// mode < 0: $DOSE_AUTOTUNE (off | cached | full, or 0 | 1 | 2; unset = off).
bool resolve_mode(int mode, int* out) {
    if (mode >= 0) {
        if (mode > 2) return false;
        *out = mode;
        return true;
    }
    const char* e = std::getenv("DOSE_AUTOTUNE");
    if (!e || !*e || !std::strcmp(e, "off") || !std::strcmp(e, "0")) {
        *out = DOSE_AUTOTUNE_OFF;
    } else if (!std::strcmp(e, "cached") || !std::strcmp(e, "1")) {
        *out = DOSE_AUTOTUNE_CACHED;
    } else if (!std::strcmp(e, "full") || !std::strcmp(e, "2")) {
        *out = DOSE_AUTOTUNE_FULL;
    } else {
        return false;
    }
    return true;
}

// ------------------------------------------------------------ JSON
// A small reader for the cache file (objects, arrays, strings with the
// escapes \" \\ \/ \n \t, numbers, true, false, null) and a writer of the
// one layout the cache uses.
struct JVal {
    enum Kind { NUL, BOOL, NUM, STR, ARR, OBJ } kind = NUL;
    double num = 0;
    bool b = false;
    std::string str;
    std::vector<JVal> arr;
    std::vector<std::pair<std::string, JVal>> obj;
    const JVal* get(const char* key) const {
        if (kind != OBJ) return nullptr;
        for (const auto& kv : obj)
            if (kv.first == key) return &kv.second;
        return nullptr;
    }
};

class JReader {
  public:
    JReader(const char* p, const char* e) : p_(p), e_(e) {}
    bool parse(JVal* out) {
        if (!value(out, 0)) return false;
        ws();
        return p_ == e_;
    }

  private:
    const char* p_;
    const char* e_;
    void ws() {
        while (p_ < e_ && (*p_ == ' ' || *p_ == '\n' || *p_ == '\r' || *p_ == '\t')) ++p_;
    }
    bool lit(const char* w) {
        const size_t n = std::strlen(w);
        if ((size_t)(e_ - p_) < n || std::strncmp(p_, w, n)) return false;
        p_ += n;
        return true;
    }
    bool string(std::string* s) {
        if (p_ >= e_ || *p_ != '"') return false;
        ++p_;
        while (p_ < e_ && *p_ != '"') {
            char c = *p_++;
            if (c == '\\') {
                if (p_ >= e_) return false;
                const char q = *p_++;
                c = q == 'n' ? '\n' : q == 't' ? '\t' : q;
                if (q != '"' && q != '\\' && q != '/' && q != 'n' && q != 't') return false;
            }
            s->push_back(c);
        }
        if (p_ >= e_) return false;
        ++p_;
        return true;
    }
    bool value(JVal* v, int depth) {
        if (depth > 16) return false;
        ws();
        if (p_ >= e_) return false;
        const char c = *p_;
        if (c == '{') {
            ++p_;
            v->kind = JVal::OBJ;
            ws();
            if (p_ < e_ && *p_ == '}') return ++p_, true;
            for (;;) {
                ws();
                std::string k;
                if (!string(&k)) return false;
                ws();
                if (p_ >= e_ || *p_ != ':') return false;
                ++p_;
                v->obj.emplace_back(std::move(k), JVal());
                if (!value(&v->obj.back().second, depth + 1)) return false;
                ws();
                if (p_ < e_ && *p_ == ',') {
                    ++p_;
                    continue;
                }
                if (p_ < e_ && *p_ == '}') return ++p_, true;
                return false;
            }
        }
        if (c == '[') {
            ++p_;
            v->kind = JVal::ARR;
            ws();
            if (p_ < e_ && *p_ == ']') return ++p_, true;
            for (;;) {
                v->arr.emplace_back();
                if (!value(&v->arr.back(), depth + 1)) return false;
                ws();
                if (p_ < e_ && *p_ == ',') {
                    ++p_;
                    continue;
                }
                if (p_ < e_ && *p_ == ']') return ++p_, true;
                return false;
            }
        }
        if (c == '"') {
            v->kind = JVal::STR;
            return string(&v->str);
        }
        if (lit("true")) return v->kind = JVal::BOOL, v->b = true, true;
        if (lit("false")) return v->kind = JVal::BOOL, v->b = false, true;
        if (lit("null")) return v->kind = JVal::NUL, true;
        char* end = nullptr;
        const std::string tok(p_, (size_t)std::min<ptrdiff_t>(e_ - p_, 64));
        const double d = std::strtod(tok.c_str(), &end);
        if (end == tok.c_str()) return false;
        p_ += end - tok.c_str();
        v->kind = JVal::NUM;
        v->num = d;
        return true;
    }
};

std::string json_str(const std::string& s) {
    std::string o = "\"";
    for (char c : s) {
        if (c == '"' || c == '\\') o.push_back('\\');
        if (c == '\n') {
            o += "\\n";
            continue;
        }
        if (c == '\t') {
            o += "\\t";
            continue;
        }
        o.push_back(c);
    }
    return o + "\"";
}

// ------------------------------------------------------------ cache file
// {"format": "dose-autotune-1", "entries": [{"gpu": ..., "fingerprint": ...,
//   "purposes": ..., "nrows": ..., "ncols": ..., "nnz": ..., "fmt": ...,
//   "flags": ..., "tuning": {<dose_tuning field>: value, ...},
//   "ms": {"forward": ..., "fused": ..., "batched": ...}}, ...]}
constexpr const char* kFormat = "dose-autotune-1";
constexpr const char* kTuneNames[] = {
    "tile_nnz",      "tile_rows",         "coop_nnz",          "lane_target",     "stages",
    "consumer_warps", "l2_prefetch",      "adj_tile_nnz",      "adj_tile_rows",   "adj_stages",
    "adj_forward_warps", "adj_scatter_warps", "adj_l2_prefetch", "row_order",     "adj_row_order",
    "sell_sigma",    "adj_layout",        "rg_tile_union",     "rg_tile_rows",    "rg_stages",
    "rg_warps",      "rg_l2_prefetch",    "fwd_layout"};
constexpr size_t kTuneFields = sizeof(kTuneNames) / sizeof(kTuneNames[0]);
static_assert(sizeof(dose_tuning) == kTuneFields * sizeof(uint32_t), "dose_tuning is a list of uint32_t knobs");

struct CacheEntry {
    std::string gpu, fp;
    uint32_t purposes = 0, nrows = 0, ncols = 0, fmt = 0, flags = 0;
    uint64_t nnz = 0;
    dose_tuning t{};
    double ms[3] = {0, 0, 0};
};
constexpr const char* kPurposeNames[3] = {"forward", "fused", "batched"};

bool entry_from(const JVal& v, CacheEntry* e) {
    const JVal *g = v.get("gpu"), *f = v.get("fingerprint"), *p = v.get("purposes"), *t = v.get("tuning");
    if (!g || g->kind != JVal::STR || !f || f->kind != JVal::STR || !p || p->kind != JVal::NUM || !t ||
        t->kind != JVal::OBJ)
        return false;
    e->gpu = g->str;
    e->fp = f->str;
    e->purposes = (uint32_t)p->num;
    auto num = [&](const char* k, double dflt) {
        const JVal* x = v.get(k);
        return x && x->kind == JVal::NUM ? x->num : dflt;
    };
    e->nrows = (uint32_t)num("nrows", 0);
    e->ncols = (uint32_t)num("ncols", 0);
    e->nnz = (uint64_t)num("nnz", 0);
    e->fmt = (uint32_t)num("fmt", 0);
    e->flags = (uint32_t)num("flags", 0);
    uint32_t* knobs = reinterpret_cast<uint32_t*>(&e->t);
    for (size_t i = 0; i < kTuneFields; ++i) {
        const JVal* x = t->get(kTuneNames[i]);
        if (x && x->kind != JVal::NUM) return false;
        if (x && (x->num < 0 || x->num > 4294967295.0 || x->num != std::floor(x->num))) return false;
        knobs[i] = x ? (uint32_t)x->num : 0u;
    }
    if (const JVal* m = v.get("ms"))
        for (int i = 0; i < 3; ++i)
            if (const JVal* x = m->get(kPurposeNames[i]); x && x->kind == JVal::NUM) e->ms[i] = x->num;
    return true;
}

// Entries of the file at `path` (a missing file has none).  A file that is
// not a cache of this format is an error, so that it is never overwritten.
dose_status load_entries(const std::string& path, std::vector<CacheEntry>* out) {
    out->clear();
    FILE* fh = std::fopen(path.c_str(), "rb");
    if (!fh) {
        if (errno == ENOENT) return DOSE_OK;
        return bad("autotune cache " + path + ": " + std::strerror(errno), DOSE_ERR_IO);
    }
    std::string text;
    char buf[65536];
    size_t n;
    while ((n = std::fread(buf, 1, sizeof(buf), fh)) > 0) text.append(buf, n);
    const bool err = std::ferror(fh);
    std::fclose(fh);
    if (err) return bad("autotune cache " + path + ": read error", DOSE_ERR_IO);
    JVal root;
    JReader rd(text.data(), text.data() + text.size());
    if (!rd.parse(&root) || root.kind != JVal::OBJ)
        return bad("autotune cache " + path + " is not JSON", DOSE_ERR_IO);
    const JVal *fmt = root.get("format"), *ents = root.get("entries");
    if (!fmt || fmt->kind != JVal::STR || fmt->str != kFormat || !ents || ents->kind != JVal::ARR)
        return bad("autotune cache " + path + " is not a " + kFormat + " file", DOSE_ERR_IO);
    for (const JVal& v : ents->arr) {
        CacheEntry e;
        if (entry_from(v, &e)) out->push_back(std::move(e));
    }
    return DOSE_OK;
}

dose_status make_parents(const std::string& path) {
    for (size_t i = 1; i < path.size(); ++i) {
        if (path[i] != '/') continue;
        const std::string dir = path.substr(0, i);
        if (::mkdir(dir.c_str(), 0755) != 0 && errno != EEXIST)
            return bad("autotune cache directory " + dir + ": " + std::strerror(errno), DOSE_ERR_IO);
    }
    return DOSE_OK;
}

// Write all entries to a temporary file beside `path`, then rename it over
// `path` (readers see the old or the new file, never a part of one).
dose_status save_entries(const std::string& path, const std::vector<CacheEntry>& es) {
    dose_status st = make_parents(path);
    if (st != DOSE_OK) return st;
    std::string o = "{\"format\": " + json_str(kFormat) + ", \"entries\": [";
    for (size_t k = 0; k < es.size(); ++k) {
        const CacheEntry& e = es[k];
        char num[64];
        o += k ? ",\n  {" : "\n  {";
        o += "\"gpu\": " + json_str(e.gpu) + ", \"fingerprint\": " + json_str(e.fp);
        o += ", \"purposes\": " + std::to_string(e.purposes) + ", \"nrows\": " + std::to_string(e.nrows);
        o += ", \"ncols\": " + std::to_string(e.ncols) + ", \"nnz\": " + std::to_string(e.nnz);
        o += ", \"fmt\": " + std::to_string(e.fmt) + ", \"flags\": " + std::to_string(e.flags);
        o += ",\n   \"tuning\": {";
        const uint32_t* knobs = reinterpret_cast<const uint32_t*>(&e.t);
        for (size_t i = 0; i < kTuneFields; ++i)
            o += (i ? ", " : "") + json_str(kTuneNames[i]) + ": " + std::to_string(knobs[i]);
        o += "},\n   \"ms\": {";
        for (int i = 0; i < 3; ++i) {
            std::snprintf(num, sizeof(num), "%.6g", e.ms[i]);
            o += (i ? ", " : "") + json_str(kPurposeNames[i]) + ": " + num;
        }
        o += "}}";
    }
    o += "\n]}\n";
    const std::string tmp = path + ".tmp." + std::to_string((long)::getpid());
    FILE* fh = std::fopen(tmp.c_str(), "wb");
    if (!fh) return bad("autotune cache " + tmp + ": " + std::strerror(errno), DOSE_ERR_IO);
    const bool ok = std::fwrite(o.data(), 1, o.size(), fh) == o.size();
    if (std::fclose(fh) != 0 || !ok) {
        std::remove(tmp.c_str());
        return bad("autotune cache " + tmp + ": write error", DOSE_ERR_IO);
    }
    if (std::rename(tmp.c_str(), path.c_str()) != 0) {
        const std::string why = std::strerror(errno);
        std::remove(tmp.c_str());
        return bad("autotune cache " + path + ": " + why, DOSE_ERR_IO);
    }
    return DOSE_OK;
}

const CacheEntry* find_entry(const std::vector<CacheEntry>& es, const std::string& gpu, const std::string& fp,
                             uint32_t purposes) {
    for (const CacheEntry& e : es)
        if (e.gpu == gpu && e.fp == fp && e.purposes == purposes) return &e;
    return nullptr;
}

// ------------------------------------------------------------ the sweep
// Mean time of `reps` calls after 3 untimed ones, with CUDA events on `s`;
// -1 with *st set when a call fails.
template <class F>
float time_calls(cudaStream_t s, cudaEvent_t e0, cudaEvent_t e1, int reps, dose_status* st, F&& fn) {
    for (int i = 0; i < 3; ++i)
        if ((*st = fn()) != DOSE_OK) return -1.f;
    cudaEventRecord(e0, s);
    for (int i = 0; i < reps; ++i)
        if ((*st = fn()) != DOSE_OK) return -1.f;
    cudaEventRecord(e1, s);
    cudaError_t e = cudaEventSynchronize(e1);
    if (e != cudaSuccess) {
        *st = cuda_fail(e, "autotune timing");
        return -1.f;
    }
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    return ms / reps;
}

struct Scratch {
    float *x1 = nullptr, *d = nullptr, *pw = nullptr, *g = nullptr, *X16 = nullptr, *D16 = nullptr;
    double* f = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    ~Scratch() {
        cudaFree(x1);
        cudaFree(d);
        cudaFree(pw);
        cudaFree(g);
        cudaFree(X16);
        cudaFree(D16);
        cudaFree(f);
        if (e0) cudaEventDestroy(e0);
        if (e1) cudaEventDestroy(e1);
    }
};

cudaError_t upload_fill(float** p, size_t n, float v) {
    cudaError_t e = dev_malloc(p, std::max<size_t>(n, 1) * 4);
    if (e != cudaSuccess) return e;
    std::vector<float> h(std::max<size_t>(n, 1), v);
    return cudaMemcpy(*p, h.data(), h.size() * 4, cudaMemcpyHostToDevice);
}

// Time candidate knobs of the purposes asked for and keep the fastest on A.
// ms[0..2]: the chosen knobs' times of dose_spmv, of the fused objective pass
// and of a 16-vector dose_spmv_batched on A alone (0 where not asked for).
dose_status sweep(dose_matrix* A, const float* x, unsigned purposes, cudaStream_t s, double ms[3]) {
    ms[0] = ms[1] = ms[2] = 0;
    Scratch S;
    const size_t nr = std::max<size_t>(A->nrows, 1), nrp = (nr + 3) / 4 * 4, nc = std::max<uint32_t>(A->ncols, 1);
    cudaError_t e = cudaSuccess;
    if (!x) {
        e = upload_fill(&S.x1, nc, 1.0f);
        x = S.x1;
    }
    if (e == cudaSuccess) e = dev_malloc(&S.d, nr * 4);
    if (e == cudaSuccess) e = upload_fill(&S.pw, 2 * nrp, 1.0f);  // p = 1, w = 1 on every row
    if (e == cudaSuccess) e = dev_malloc(&S.g, nc * 4);
    if (e == cudaSuccess) e = dev_malloc(&S.f, 8);
    if (e == cudaSuccess) e = cudaEventCreate(&S.e0);
    if (e == cudaSuccess) e = cudaEventCreate(&S.e1);
    if (e != cudaSuccess) return cuda_fail(e, "autotune scratch");
    if (purposes & DOSE_TUNE_BATCHED) {
        // 16 vectors of X and D; without room for them the batched call is not timed
        if (upload_fill(&S.X16, (size_t)nc * 16, 0.5f) != cudaSuccess ||
            dev_malloc(&S.D16, nr * 16 * 4) != cudaSuccess) {
            cudaGetLastError();
            cudaFree(S.X16);
            cudaFree(S.D16);
            S.X16 = S.D16 = nullptr;
        }
    }
    const float* p = S.pw;
    const float* w = S.pw + nrp;
    dose_status st = DOSE_OK;
    auto spmv = [&] { return dose_spmv(A, x, S.d, s); };
    auto fused = [&] { return dose_fwd_adj_quadratic(A, x, p, w, nullptr, S.f, S.g, s); };
    const dose_matrix* one[1] = {A};
    const float* X1[1] = {S.X16};
    float* D1[1] = {S.D16};
    auto batched = [&] { return dose_spmv_batched(one, 1, X1, D1, 16, s); };

    // 1. dose_spmv: the CSR form's stage tiles, lanes-per-row target and
    //    pipeline depth, then the row-group form against the best of them
    if ((purposes & DOSE_TUNE_FORWARD) && !(A->flags & DOSE_CREATE_SELL)) {
        const Tuning orig = A->fwd.tuning;
        Tuning base = orig;
        base.layout = 1;  // time the CSR form
        if ((st = apply_schedule(A, A->fwd, base, A->fwd_windowed)) != DOSE_OK) return st;
        Tuning best = base;
        float best_ms = time_calls(s, S.e0, S.e1, 10, &st, spmv);
        if (best_ms < 0.f) return st;
        for (uint32_t tn : {4096u, 8192u})
            for (uint32_t tr : {1024u, 2048u, 4096u})
                for (uint32_t lt : {8u, 16u, 24u})
                    for (uint32_t sd : {3u, 4u}) {
                        Tuning t = base;
                        t.tile_nnz = tn;
                        t.tile_rows = tr;
                        t.coop_nnz = std::min(base.coop_nnz, tn);
                        t.lane_target = lt;
                        t.stages = sd;
                        if (!std::memcmp(&t, &base, sizeof(t)) || check_tuning(A, t) != DOSE_OK) continue;
                        if ((st = apply_schedule(A, A->fwd, t, A->fwd_windowed)) != DOSE_OK) return st;
                        const float m = time_calls(s, S.e0, S.e1, 10, &st, spmv);
                        if (m < 0.f) return st;
                        if (m < best_ms) {
                            best_ms = m;
                            best = t;
                        }
                    }
        if ((st = apply_schedule(A, A->fwd, best, A->fwd_windowed)) != DOSE_OK) return st;
        if (orig.layout != 1) {
            A->fwd.tuning.layout = orig.layout;
            if (spmv_on_row_groups(A)) {
                const float m = time_calls(s, S.e0, S.e1, 10, &st, spmv);
                if (m < 0.f) return st;
                if (m < best_ms || orig.layout == 2) {
                    best_ms = m;
                    best.layout = orig.layout;
                }
            }
            A->fwd.tuning.layout = best.layout;
        }
        if (A->fwd64_own && (st = apply_schedule(A, A->fwd64, best, false)) != DOSE_OK) return st;
        // the adjoint schedule takes the forward's lane binning
        if ((st = apply_schedule(A, A->adj, adj_schedule_tuning(best, A->adj_tuning), true)) != DOSE_OK) return st;
        ms[0] = best_ms;
    } else if (purposes & DOSE_TUNE_FORWARD) {
        const float m = time_calls(s, S.e0, S.e1, 10, &st, spmv);
        if (m < 0.f) return st;
        ms[0] = m;
    }

    // 2. the fused objective pass (p = w = 1 on every row, so the objective
    //    terms of rows without entries are paid as in use) and the batched SpMM:
    //    the adjoint layout and its knobs, scored by the sum of their times
    if (purposes & (DOSE_TUNE_FUSED | DOSE_TUNE_BATCHED)) {
        const bool time_b = (purposes & DOSE_TUNE_BATCHED) && S.X16;
        // a row-group dose_spmv shares the layout's stages: its time joins the score
        const bool time_v = (purposes & DOSE_TUNE_FORWARD) && !(A->flags & DOSE_CREATE_SELL) && A->rg.built &&
                            A->fwd.tuning.layout != 1;
        const AdjTuning base = A->adj_tuning;
        AdjTuning rg_cut = base, csr_cut = base;  // knobs the two adjoint schedules are cut with
        std::vector<AdjTuning> cands{base};
        if (A->rg.built) {
            for (uint32_t tu : {0u, 2048u, 3072u, 4096u, 6144u})
                for (uint32_t tr : {512u, 1024u})
                    for (uint32_t wn : {0u, 12u})
                        for (uint32_t sd : {2u, 3u}) {
                            AdjTuning a = base;
                            a.layout = 0;
                            a.rg_tile_u = tu;
                            a.rg_tile_rows = tr;
                            a.rg_warps = wn;
                            a.rg_stages = sd;
                            cands.push_back(a);
                        }
            AdjTuning a = base;
            a.layout = 1;  // the CSR layout, for comparison
            cands.push_back(a);
        } else {
            for (uint32_t tn : {4096u, 5120u, 8192u})
                for (uint32_t tr : {1024u, 2048u})
                    for (uint32_t sd : {3u, 4u}) {
                        AdjTuning a = base;
                        a.tile_nnz = tn;
                        a.tile_rows = tr;
                        a.stages = sd;
                        cands.push_back(a);
                    }
        }
        // Re-cut what a candidate changes; *usable = false when its stage cannot
        // hold a group's union (the previous cut is then restored).
        auto cut = [&](const AdjTuning& a, bool* usable) -> dose_status {
            *usable = true;
            if (check_adj_tuning(a) != DOSE_OK) {
                *usable = false;
                return DOSE_OK;
            }
            if (A->rg.built && (a.rg_tile_u != rg_cut.rg_tile_u || a.rg_tile_rows != rg_cut.rg_tile_rows)) {
                cudaError_t e2 = rg_schedule(A, a);
                if (e2 == cudaErrorInvalidValue) {
                    *usable = false;
                    e2 = rg_schedule(A, rg_cut);
                }
                if (e2 != cudaSuccess) return cuda_fail(e2, "row-group schedule");
                if (!*usable) return DOSE_OK;
                rg_cut = a;
            }
            if (a.tile_nnz != csr_cut.tile_nnz || a.tile_rows != csr_cut.tile_rows || a.stages != csr_cut.stages ||
                a.row_order != csr_cut.row_order) {
                const dose_status s2 = apply_schedule(A, A->adj, adj_schedule_tuning(A->fwd.tuning, a), true);
                if (s2 != DOSE_OK) return s2;
                csr_cut = a;
            }
            A->adj_tuning = a;
            return DOSE_OK;
        };
        float best = 3e38f;
        AdjTuning best_a = base;
        double bf = 0, bb = 0, bv = ms[0];
        for (const AdjTuning& a : cands) {
            bool usable = true;
            if ((st = cut(a, &usable)) != DOSE_OK) return st;
            if (!usable) continue;
            float tf = 0.f, tb = 0.f, tv = 0.f;
            if (purposes & DOSE_TUNE_FUSED) {
                tf = time_calls(s, S.e0, S.e1, 10, &st, fused);
                if (tf < 0.f) {
                    if (st == DOSE_ERR_UNSUPPORTED) continue;
                    return st;
                }
            }
            if (time_b) {
                tb = time_calls(s, S.e0, S.e1, 5, &st, batched);
                if (tb < 0.f) {
                    if (st == DOSE_ERR_UNSUPPORTED) continue;
                    return st;
                }
            }
            if (time_v && spmv_on_row_groups(A)) {
                tv = time_calls(s, S.e0, S.e1, 10, &st, spmv);
                if (tv < 0.f) return st;
            }
            if (tf + tb + tv < best) {
                best = tf + tb + tv;
                best_a = a;
                bf = tf;
                bb = tb;
                if (tv > 0.f) bv = tv;
            }
        }
        bool usable = true;
        if ((st = cut(best_a, &usable)) != DOSE_OK) return st;
        ms[0] = bv;
        ms[1] = bf;
        ms[2] = bb;
    }
    set_error("");
    return DOSE_OK;
}

}  // namespace

uint64_t matrix_fingerprint(const dose_matrix* A) {
    return fingerprint_of(A->nrows, A->ncols, A->nnz, (uint32_t)A->fmt, A->flags, A->host_row_ptr.data(),
                          A->host_row_cmin.data(), A->host_row_cmax.data());
}

}  // namespace dose

using namespace dose;

extern "C" {

dose_status dose_autotune(dose_matrix* A, const float* x, void* stream, dose_tuning* best) {
    NvtxRange nvtx_range("dose_autotune");
    if (!A) return bad("dose_autotune: null matrix");
    double ms[3];
    const dose_status st = sweep(A, x, DOSE_TUNE_FORWARD | DOSE_TUNE_FUSED, static_cast<cudaStream_t>(stream), ms);
    if (st != DOSE_OK) return st;
    if (best) {
        dose_info inf;
        dose_matrix_info(A, &inf);
        *best = inf.tuning;  // the knobs in effect, as dose_matrix_info reports them
    }
    return DOSE_OK;
}

dose_status dose_autotune_cached(dose_matrix* A, const float* x, int mode, unsigned purposes, const char* path,
                                 void* stream, dose_tuning* best, dose_autotune_report* report) {
    NvtxRange nvtx_range("dose_autotune_cached");
    if (!A) return bad("dose_autotune_cached: null matrix");
    if (purposes & ~(unsigned)(DOSE_TUNE_FORWARD | DOSE_TUNE_FUSED | DOSE_TUNE_BATCHED))
        return bad("dose_autotune_cached: unknown purposes");
    if (!purposes) purposes = DOSE_TUNE_FORWARD | DOSE_TUNE_FUSED;
    int m = 0;
    if (!resolve_mode(mode, &m))
        return bad(mode < 0 ? "DOSE_AUTOTUNE must be off, cached or full" : "dose_autotune_cached: mode must be 0, 1 or 2");
    dose_autotune_report rep{};
    rep.purposes = purposes;
    rep.fingerprint = A->fingerprint;
    dose_status st = DOSE_OK;
    if (m != DOSE_AUTOTUNE_OFF) {
        const std::string file = cache_path(path), gpu = gpu_name(A->device), fp = hex64(A->fingerprint);
        std::vector<CacheEntry> es;
        if ((st = load_entries(file, &es)) != DOSE_OK) return st;
        const CacheEntry* hit = m == DOSE_AUTOTUNE_CACHED ? find_entry(es, gpu, fp, purposes) : nullptr;
        if (hit && dose_set_tuning(A, &hit->t) == DOSE_OK) {
            rep.source = 1;
            for (int i = 0; i < 3; ++i) rep.ms[i] = hit->ms[i];
        } else {
            // no entry (or one this handle cannot take): time the candidates and store the result
            if ((st = sweep(A, x, purposes, static_cast<cudaStream_t>(stream), rep.ms)) != DOSE_OK) return st;
            CacheEntry e;
            e.gpu = gpu;
            e.fp = fp;
            e.purposes = purposes;
            e.nrows = A->nrows;
            e.ncols = A->ncols;
            e.nnz = A->nnz;
            e.fmt = (uint32_t)A->fmt;
            e.flags = A->flags;
            dose_info inf;
            dose_matrix_info(A, &inf);
            e.t = inf.tuning;
            for (int i = 0; i < 3; ++i) e.ms[i] = rep.ms[i];
            bool replaced = false;
            for (CacheEntry& o : es)
                if (o.gpu == gpu && o.fp == fp && o.purposes == purposes) {
                    o = e;
                    replaced = true;
                }
            if (!replaced) es.push_back(e);
            if ((st = save_entries(file, es)) != DOSE_OK) return st;  // the swept knobs stay applied
            rep.source = 2;
        }
    }
    if (best) {
        dose_info inf;
        dose_matrix_info(A, &inf);
        *best = inf.tuning;
    }
    if (report) *report = rep;
    return DOSE_OK;
}

dose_status dose_fingerprint_host(const dose_csr_desc* desc, unsigned flags, uint64_t* out) {
    if (!desc || !out) return bad("dose_fingerprint_host: null argument");
    if (desc->on_device) return bad("dose_fingerprint_host: needs host arrays (on_device = 0)");
    if (!desc->row_ptr || (desc->nnz && !desc->col_idx)) return bad("dose_fingerprint_host: null array");
    const uint32_t n = desc->nrows;
    const uint32_t* rp = desc->row_ptr;
    if (rp[0] != 0 || rp[n] != desc->nnz) return bad("dose_fingerprint_host: row_ptr must run from 0 to nnz");
    std::vector<uint32_t> lo(n, 0xFFFFFFFFu), hi(n, 0);
    for (uint32_t i = 0; i < n; ++i) {
        if (rp[i + 1] < rp[i]) return bad("dose_fingerprint_host: row_ptr must be non-decreasing");
        for (uint32_t k = rp[i]; k < rp[i + 1]; ++k) {
            lo[i] = std::min(lo[i], desc->col_idx[k]);
            hi[i] = std::max(hi[i], desc->col_idx[k]);
        }
    }
    *out = fingerprint_of(n, desc->ncols, desc->nnz, (uint32_t)desc->fmt, flags, rp, lo.data(), hi.data());
    return DOSE_OK;
}

dose_status dose_autotune_cache_lookup(const char* path, const char* gpu, uint64_t fingerprint, unsigned purposes,
                                       dose_tuning* out, double* ms, int* found) {
    if (!path || !gpu || !found) return bad("dose_autotune_cache_lookup: null argument");
    *found = 0;
    std::vector<CacheEntry> es;
    const dose_status st = load_entries(path, &es);
    if (st != DOSE_OK) return st;
    const CacheEntry* e = find_entry(es, gpu, hex64(fingerprint), purposes);
    if (!e) return DOSE_OK;
    *found = 1;
    if (out) *out = e->t;
    if (ms)
        for (int i = 0; i < 3; ++i) ms[i] = e->ms[i];
    return DOSE_OK;
}

dose_status dose_autotune_cache_store(const char* path, const char* gpu, uint64_t fingerprint, unsigned purposes,
                                      const dose_tuning* t, const double* ms) {
    if (!path || !gpu || !t) return bad("dose_autotune_cache_store: null argument");
    std::vector<CacheEntry> es;
    dose_status st = load_entries(path, &es);
    if (st != DOSE_OK) return st;
    CacheEntry e;
    e.gpu = gpu;
    e.fp = hex64(fingerprint);
    e.purposes = purposes;
    e.t = *t;
    if (ms)
        for (int i = 0; i < 3; ++i) e.ms[i] = ms[i];
    bool replaced = false;
    for (CacheEntry& o : es)
        if (o.gpu == e.gpu && o.fp == e.fp && o.purposes == purposes) {
            o = e;
            replaced = true;
        }
    if (!replaced) es.push_back(e);
    return save_entries(path, es);
}

const char* dose_gpu_name(int device, char* buf, int len) {
    if (!buf || len < 1) return nullptr;
    const std::string s = gpu_name(device);
    std::snprintf(buf, (size_t)len, "%s", s.c_str());
    return buf;
}

}  // extern "C"
