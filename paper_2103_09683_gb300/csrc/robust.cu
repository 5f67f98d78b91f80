// Multi-beam plans and robust scenario objectives (Sec. I: in every iteration
// the optimiser needs the doses of several beams, possibly under several
// realisations of the uncertainties, with function values and gradients).
//
//   * dose_create_multibeam: a plan's total dose is d = sum_b A_b x_b over its
//     beams on one voxel grid.  The beams are merged on the host into one matrix
//     whose columns are the beams' spots in beam order, so x = [x_1; ...; x_B]
//     and one pass over the merged rows gives the total dose (and A^T r gives
//     every beam's gradient at once) with the single-matrix kernels: no
//     cross-beam reduction, nothing extra to make deterministic.
//   * dose_scenarios: S scenario matrices of one shape (the same plan under S
//     setup shifts).  dose_robust_quadratic runs the fused objective pass of
//     each scenario (f_s and g_s = A_s^T r_s into the set's scratch) and one
//     combine kernel: the expected value sum_s prob_s f_s (gradient
//     sum_s prob_s g_s), or the worst case max_s f_s (gradient g_s* of the first
//     scenario with the largest f_s, a subgradient of the max).  Every sum runs
//     in scenario order, so results are bitwise reproducible.
#include <cmath>
#include <cstring>
#include <memory>
#include <string>
#include <vector>

#include "dose_internal.cuh"
#include "nvtx_range.cuh"

using namespace dose;

struct dose_scenarios {
    std::vector<const dose_matrix*> A;
    uint32_t nrows = 0, ncols = 0;
    double* prob = nullptr;  // device, S
    double* f_s = nullptr;   // device, S: objective of each scenario
    float* g_s = nullptr;    // device, S x ncols: gradient of each scenario
};

namespace dose {
namespace {

constexpr int kMaxScenarios = 64;

// F and G (and optionally the projected-gradient update of x) from the
// per-scenario f_s, g_s.  Every thread finds s* itself (S <= 64 values): the
// first scenario with the largest f_s, a NaN counting as larger than every
// number (a diverged scenario is reported, whatever its position).
__global__ void __launch_bounds__(256) robust_combine(uint32_t S, uint32_t ncols, int mode,
                                                      const double* __restrict__ prob,
                                                      const double* __restrict__ f_s, const float* __restrict__ g_s,
                                                      double* F, double* f_out, float* G, float* x_update,
                                                      float eta) {
    uint32_t best = 0;
    if (mode == DOSE_ROBUST_WORST_CASE)
        for (uint32_t s = 1; s < S; ++s)
            if (!isnan(f_s[best]) && (isnan(f_s[s]) || f_s[s] > f_s[best])) best = s;
    const uint32_t j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j == 0) {
        double t = 0.0;
        if (mode == DOSE_ROBUST_EXPECTED)
            for (uint32_t s = 0; s < S; ++s) t = __fma_rn(prob[s], f_s[s], t);
        else
            t = f_s[best];
        *F = t;
        if (f_out)
            for (uint32_t s = 0; s < S; ++s) f_out[s] = f_s[s];
    }
    if (j >= ncols) return;
    float g;
    if (mode == DOSE_ROBUST_EXPECTED) {
        double t = 0.0;
        for (uint32_t s = 0; s < S; ++s) t = __fma_rn(prob[s], (double)g_s[(size_t)s * ncols + j], t);
        g = __double2float_rn(t);
    } else {
        g = g_s[(size_t)best * ncols + j];
    }
    if (G) G[j] = g;
    if (x_update) {
        const float xn = __fsub_rn(x_update[j], __fmul_rn(eta, g));
        x_update[j] = xn > 0.f ? xn : 0.f;
    }
}

dose_status invalid(const std::string& m) {
    set_error(m);
    return DOSE_ERR_INVALID_ARG;
}

dose_status robust_run(const dose_scenarios* S, int mode, const float* x, const float* p, const float* w,
                       double* f, double* f_scen, float* g, float* x_update, float eta, void* stream) {
    if (!S) return invalid("robust: null scenario set");
    if (mode != DOSE_ROBUST_EXPECTED && mode != DOSE_ROBUST_WORST_CASE) return invalid("robust: unknown mode");
    if (!f || (S->ncols && !x) || (S->nrows && (!p || !w))) return invalid("robust: null pointer argument");
    const float* vv[2] = {p, w};
    for (const dose_matrix* A : S->A) {
        dose_status st = adjoint_supported(A, true, vv, 2);
        if (st != DOSE_OK) return st;
    }
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const uint32_t n = (uint32_t)S->A.size();
    for (uint32_t k = 0; k < n; ++k) {
        cudaError_t e = launch_adjoint(S->A[k], ADJ_MODE_QUADRATIC, x, p, w, nullptr, nullptr, S->f_s + k,
                                       S->g_s + (size_t)k * S->ncols, nullptr, 0.f, s);
        if (e != cudaSuccess) return cuda_fail(e, "robust: scenario pass");
    }
    const uint32_t blocks = S->ncols ? (S->ncols + 255) / 256 : 1;
    robust_combine<<<blocks, 256, 0, s>>>(n, S->ncols, mode, S->prob, S->f_s, S->g_s, f, f_scen, g, x_update, eta);
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? DOSE_OK : cuda_fail(e, "robust: combine");
}

}  // namespace
}  // namespace dose

extern "C" {

dose_status dose_create_scenarios(const dose_matrix* const* A, int count, const double* prob, dose_scenarios** out) {
    if (!out) return invalid("dose_create_scenarios: out is NULL");
    *out = nullptr;
    if (!A || count < 1 || count > kMaxScenarios)
        return invalid("dose_create_scenarios: count must be in [1, " + std::to_string(kMaxScenarios) + "]");
    for (int k = 0; k < count; ++k) {
        if (!A[k]) return invalid("dose_create_scenarios: null matrix " + std::to_string(k));
        if (A[k]->nrows != A[0]->nrows || A[k]->ncols != A[0]->ncols)
            return invalid("dose_create_scenarios: scenario " + std::to_string(k) + " has another shape");
        if (A[k]->device != A[0]->device) return invalid("dose_create_scenarios: matrices on different devices");
    }
    std::vector<double> pr(count, 1.0 / count);
    if (prob) {
        double sum = 0.0;
        for (int k = 0; k < count; ++k) {
            if (!(prob[k] >= 0.0) || std::isinf(prob[k]))
                return invalid("dose_create_scenarios: probabilities must be finite and >= 0");
            pr[k] = prob[k];
            sum += prob[k];
        }
        if (!(std::fabs(sum - 1.0) <= 1e-9)) return invalid("dose_create_scenarios: probabilities must sum to 1");
    }
    std::unique_ptr<dose_scenarios> S(new dose_scenarios());
    S->A.assign(A, A + count);
    S->nrows = A[0]->nrows;
    S->ncols = A[0]->ncols;
    int dev_prev = 0;
    cudaGetDevice(&dev_prev);
    cudaSetDevice(A[0]->device);
    cudaError_t e = dev_malloc(&S->prob, count * sizeof(double));
    if (e == cudaSuccess) e = dev_malloc(&S->f_s, count * sizeof(double));
    if (e == cudaSuccess) e = dev_malloc(&S->g_s, std::max<size_t>((size_t)count * S->ncols, 1) * sizeof(float));
    if (e == cudaSuccess) e = cudaMemcpy(S->prob, pr.data(), count * sizeof(double), cudaMemcpyHostToDevice);
    cudaSetDevice(dev_prev);
    if (e != cudaSuccess) {
        cudaFree(S->prob);
        cudaFree(S->f_s);
        cudaFree(S->g_s);
        if (e == cudaErrorMemoryAllocation) {
            set_error("dose_create_scenarios: out of device memory");
            return DOSE_ERR_OOM;
        }
        return cuda_fail(e, "dose_create_scenarios");
    }
    *out = S.release();
    return DOSE_OK;
}

dose_status dose_destroy_scenarios(dose_scenarios* S) {
    if (!S) return DOSE_OK;
    cudaDeviceSynchronize();
    cudaFree(S->prob);
    cudaFree(S->f_s);
    cudaFree(S->g_s);
    delete S;
    return DOSE_OK;
}

dose_status dose_robust_quadratic(const dose_scenarios* S, int mode, const float* x, const float* p, const float* w,
                                  double* f, double* f_scen, float* g, void* stream) {
    NvtxRange nvtx_range("dose_robust_quadratic");
    if (S && S->ncols && !g) return invalid("dose_robust_quadratic: g is NULL");
    return robust_run(S, mode, x, p, w, f, f_scen, g, nullptr, 0.f, stream);
}

dose_status dose_robust_pg_step(const dose_scenarios* S, int mode, float* x, const float* p, const float* w,
                                float eta, double* f, float* g, void* stream) {
    NvtxRange nvtx_range("dose_robust_pg_step");
    if (!(eta >= 0.0f) || std::isinf(eta)) return invalid("dose_robust_pg_step: eta must be finite and >= 0");
    return robust_run(S, mode, x, p, w, f, nullptr, g, x, eta, stream);
}

}  // extern "C"
