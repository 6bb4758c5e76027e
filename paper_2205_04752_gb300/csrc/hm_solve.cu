// hm_solve.cu -- solution of V_h t = g with the assembled H-matrix:
// restarted GMRES on a packed (low-precision) product form, wrapped in
// iterative refinement whose residual r = g - V_h t is computed with the FP64
// form.  The FP64 residual is what the tolerance refers to.
//
// The GMRES vector operations are this file's own kernels: Gram-Schmidt in
// two classical passes (CGS2), each a fused multi-dot and a multi-axpy over
// the Krylov basis, with deterministic two-stage reductions.  The small
// Hessenberg least-squares problem (Givens rotations) lives on the host; one
// device-to-host copy of the new Hessenberg column per iteration.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include "hm_internal.h"

namespace hm {
namespace {

constexpr int kRedThreads = 256;
constexpr int kRedBlocks = 256;  // partial sums per dot (fixed: deterministic order)
constexpr int kMaxBasis = 128;   // largest restart length + 1

// partial[b][q] = sum over this block's slice of V[q] . w, q < nq
__global__ void __launch_bounds__(kRedThreads) multidot_kernel(const double* __restrict__ V, int64_t ldv,
                                                               int nq, const double* __restrict__ w,
                                                               int64_t n, double* __restrict__ partial)
{
    __shared__ double red[kRedThreads / 32];
    const int64_t per = (n + gridDim.x - 1) / gridDim.x;
    const int64_t lo = (int64_t)blockIdx.x * per, hi = min(n, lo + per);
    for (int q = 0; q < nq; ++q) {
        const double* v = V + (size_t)q * ldv;
        double s = 0.0;
        for (int64_t i = lo + threadIdx.x; i < hi; i += blockDim.x) s += v[i] * w[i];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
        if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
        __syncthreads();
        if (threadIdx.x == 0) {
            double t = 0.0;
            for (int k = 0; k < kRedThreads / 32; ++k) t += red[k];
            partial[(size_t)blockIdx.x * kMaxBasis + q] = t;
        }
        __syncthreads();
    }
}

// out[q] = sum_b partial[b][q]
__global__ void finish_dot_kernel(const double* __restrict__ partial, int nb, int nq, double* __restrict__ out)
{
    const int q = threadIdx.x;
    if (q >= nq) return;
    double s = 0.0;
    for (int b = 0; b < nb; ++b) s += partial[(size_t)b * kMaxBasis + q];
    out[q] = s;
}

// w -= sum_q h[q] V[q]   (h on the device)
__global__ void multiaxpy_kernel(const double* __restrict__ V, int64_t ldv, int nq, const double* __restrict__ h,
                                 double* __restrict__ w, int64_t n)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        double s = w[i];
        for (int q = 0; q < nq; ++q) s -= h[q] * V[(size_t)q * ldv + i];
        w[i] = s;
    }
}

// y = sum_q c[q] V[q] + beta * y   (c on the device)
__global__ void combine_kernel(const double* __restrict__ V, int64_t ldv, int nq, const double* __restrict__ c,
                               double beta, double* __restrict__ y, int64_t n)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        double s = beta == 0.0 ? 0.0 : beta * y[i];
        for (int q = 0; q < nq; ++q) s += c[q] * V[(size_t)q * ldv + i];
        y[i] = s;
    }
}

// y = a * x + b * y
__global__ void axpby_kernel(double a, const double* __restrict__ x, double b, double* __restrict__ y, int64_t n)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        y[i] = a * x[i] + (b == 0.0 ? 0.0 : b * y[i]);
}

struct Solver {
    const hm_matrix& H;
    cudaStream_t s;
    int64_t n;
    double* basis;   // (restart + 1) x n
    double* w;       // n
    double* r;       // n, FP64 residual
    double* d;       // n, correction
    double* partial; // kRedBlocks x kMaxBasis
    double* dots;    // kMaxBasis (device)
    double* coef;    // kMaxBasis (device)
    std::vector<double> hdots;

    int dot(const double* V, int nq, const double* x, double* out_host)
    {
        multidot_kernel<<<kRedBlocks, kRedThreads, 0, s>>>(V, n, nq, x, n, partial);
        HM_CUDA(cudaGetLastError());
        finish_dot_kernel<<<1, kMaxBasis, 0, s>>>(partial, kRedBlocks, nq, dots);
        HM_CUDA(cudaGetLastError());
        HM_CUDA(cudaMemcpyAsync(out_host, dots, (size_t)nq * 8, cudaMemcpyDeviceToHost, s));
        HM_CUDA(cudaStreamSynchronize(s));
        return HM_OK;
    }
    int norm(const double* x, double* out)
    {
        int rc = dot(x, 1, x, out);
        *out = std::sqrt(std::max(*out, 0.0));
        return rc;
    }
    int axpby(double a, const double* x, double b, double* y)
    {
        axpby_kernel<<<592, 256, 0, s>>>(a, x, b, y, n);
        return cuda_check(cudaGetLastError(), "axpby");
    }
};

}  // namespace
}  // namespace hm

namespace hm {

size_t solve_workspace_bytes(int64_t n, int32_t restart)
{
    return ((size_t)(restart + 1) * n + 3 * (size_t)n + (size_t)kRedBlocks * kMaxBasis + 2 * kMaxBasis) * 8;
}

int solve_check_params(const hm_matrix* H, hm_solve_params& p)
{
    if (p.restart <= 0) p.restart = 50;
    if (p.restart > kMaxBasis - 1) return fail(HM_EINVAL, "hm_solve: restart above %d", kMaxBasis - 1);
    if (!(p.tol > 0.0)) return fail(HM_EINVAL, "hm_solve: tol must be > 0");
    if (p.inner_tol <= 0.0) p.inner_tol = 1e-3;
    if (p.max_inner <= 0) p.max_inner = 1000;
    if (p.max_refine <= 0) p.max_refine = 20;
    if (p.residual_form < HM_FP64 || p.residual_form >= HM_NFORMS || !H->packed[p.residual_form])
        return fail(HM_EINVAL, "hm_solve: residual form %d not available (FP64 released by hm_compact, or not packed)",
                    p.residual_form);
    if (p.inner_form < HM_FP64 || p.inner_form >= HM_NFORMS || !H->packed[p.inner_form])
        return fail(HM_EINVAL, "hm_solve: inner form %d not available (hm_pack first)", p.inner_form);
    return HM_OK;
}

// The solve on caller-provided memory: `ws` of solve_workspace_bytes(3M,
// restart) bytes; products use `scratch` (matvec_scratch_bytes(H, 1, form)
// bytes for the larger of the two forms) or, if null, the matrix's own
// workspace.  `p` must have passed solve_check_params.
int solve_device(const hm_matrix& Hm, const double* g, double* t, const hm_solve_params& p, hm_solve_info* info,
                 cudaStream_t s, void* ws, void* scratch)
{
    const hm_matrix* H = &Hm;
    if (info) std::memset(info, 0, sizeof *info);
    const int64_t n = 3 * H->M;
    const int m = p.restart;
    auto mv = [&](const double* x, double* y, int32_t form) -> int {
        if (!scratch) return matvec_device(*H, x, y, 1, n, form, s);
        return matvec_device_scratch(*H, x, y, 1, n, form, s, make_scratch(*H, 1, form, scratch));
    };
    double* base = static_cast<double*>(ws);
    Solver S{*H, s, n, base, base + (size_t)(m + 1) * n, base + (size_t)(m + 2) * n,
             base + (size_t)(m + 3) * n, base + (size_t)(m + 4) * n,
             base + (size_t)(m + 4) * n + (size_t)kRedBlocks * kMaxBasis,
             base + (size_t)(m + 4) * n + (size_t)kRedBlocks * kMaxBasis + kMaxBasis, {}};
    S.hdots.resize(kMaxBasis);
    int rc;
    // t = initial guess (zero unless asked to keep it), r = g - V t
    double gnorm = 0.0;
    if ((rc = S.norm(g, &gnorm))) return rc;
    if (gnorm == 0.0) {
        HM_CUDA(cudaMemsetAsync(t, 0, (size_t)n * 8, s));
        HM_CUDA(cudaStreamSynchronize(s));
        return HM_OK;
    }
    if (!p.use_initial_guess) HM_CUDA(cudaMemsetAsync(t, 0, (size_t)n * 8, s));
    auto residual = [&]() -> int {
        // r = g - V_h t with the residual form (FP64 unless asked otherwise)
        int e = mv(t, S.r, p.residual_form);
        if (e) return e;
        return S.axpby(1.0, g, -1.0, S.r);
    };
    if ((rc = residual())) return rc;
    double rnorm = 0.0;
    if ((rc = S.norm(S.r, &rnorm))) return rc;
    int total_inner = 0, restarts = 0, refine = 0;
    std::vector<double> Hh((size_t)(m + 1) * m), cs(m), sn(m), gv(m + 1), y(m);
    while (rnorm > p.tol * gnorm && refine < p.max_refine && total_inner < p.max_inner) {
        ++refine;
        // ---- GMRES(m) on V~ d = r with the inner form, d from 0
        HM_CUDA(cudaMemsetAsync(S.d, 0, (size_t)n * 8, s));
        const double target = p.inner_tol * rnorm;
        double beta = rnorm;  // residual of the inner system for d = 0
        const double* rhs = S.r;
        bool first_cycle = true;
        while (total_inner < p.max_inner) {
            // v0 = (r - V~ d) / beta
            if (first_cycle) {
                if ((rc = S.axpby(1.0 / beta, rhs, 0.0, S.basis))) return rc;
            } else {
                if ((rc = mv(S.d, S.w, p.inner_form))) return rc;
                if ((rc = S.axpby(1.0, rhs, -1.0, S.w))) return rc;
                if ((rc = S.norm(S.w, &beta))) return rc;
                if (beta <= target) break;
                if ((rc = S.axpby(1.0 / beta, S.w, 0.0, S.basis))) return rc;
            }
            first_cycle = false;
            std::fill(gv.begin(), gv.end(), 0.0);
            gv[0] = beta;
            int k = 0;
            double res = beta;
            for (; k < m && total_inner < p.max_inner; ++k) {
                double* vk = S.basis + (size_t)k * n;
                double* vk1 = S.basis + (size_t)(k + 1) * n;
                if ((rc = mv(vk, vk1, p.inner_form))) return rc;
                ++total_inner;
                // classical Gram-Schmidt, two passes
                std::vector<double> h(k + 2, 0.0);
                for (int pass = 0; pass < 2; ++pass) {
                    if ((rc = S.dot(S.basis, k + 1, vk1, S.hdots.data()))) return rc;
                    HM_CUDA(cudaMemcpyAsync(S.coef, S.hdots.data(), (size_t)(k + 1) * 8, cudaMemcpyHostToDevice, s));
                    multiaxpy_kernel<<<592, 256, 0, s>>>(S.basis, n, k + 1, S.coef, vk1, n);
                    HM_CUDA(cudaGetLastError());
                    for (int q = 0; q <= k; ++q) h[q] += S.hdots[q];
                }
                double hn = 0.0;
                if ((rc = S.norm(vk1, &hn))) return rc;
                h[k + 1] = hn;
                if (hn > 0.0)
                    if ((rc = S.axpby(1.0 / hn, vk1, 0.0, vk1))) return rc;
                // apply the previous rotations, then a new one
                for (int q = 0; q < k; ++q) {
                    const double a = cs[q] * h[q] + sn[q] * h[q + 1];
                    const double b = -sn[q] * h[q] + cs[q] * h[q + 1];
                    h[q] = a;
                    h[q + 1] = b;
                }
                const double den = std::hypot(h[k], h[k + 1]);
                cs[k] = den > 0.0 ? h[k] / den : 1.0;
                sn[k] = den > 0.0 ? h[k + 1] / den : 0.0;
                h[k] = den;
                h[k + 1] = 0.0;
                gv[k + 1] = -sn[k] * gv[k];
                gv[k] = cs[k] * gv[k];
                for (int q = 0; q <= k; ++q) Hh[(size_t)q * m + k] = h[q];
                res = std::fabs(gv[k + 1]);
                if (res <= target || hn == 0.0) {
                    ++k;
                    break;
                }
            }
            // y = R^{-1} g, d += V y
            for (int q = k - 1; q >= 0; --q) {
                double sum = gv[q];
                for (int c = q + 1; c < k; ++c) sum -= Hh[(size_t)q * m + c] * y[c];
                y[q] = Hh[(size_t)q * m + q] != 0.0 ? sum / Hh[(size_t)q * m + q] : 0.0;
            }
            HM_CUDA(cudaMemcpyAsync(S.coef, y.data(), (size_t)k * 8, cudaMemcpyHostToDevice, s));
            combine_kernel<<<592, 256, 0, s>>>(S.basis, n, k, S.coef, 1.0, S.d, n);
            HM_CUDA(cudaGetLastError());
            HM_CUDA(cudaStreamSynchronize(s));
            if (res <= target) break;
            ++restarts;
        }
        // ---- refinement: t += d, r = g - V_h t (FP64)
        if ((rc = S.axpby(1.0, S.d, 1.0, t))) return rc;
        if ((rc = residual())) return rc;
        if ((rc = S.norm(S.r, &rnorm))) return rc;
    }
    HM_CUDA(cudaStreamSynchronize(s));
    if (info) {
        info->iterations = total_inner;
        info->restarts = restarts;
        info->refinements = refine;
        info->rel_residual = rnorm / gnorm;
    }
    if (rnorm > p.tol * gnorm)
        return fail(HM_ENOTCONV, "hm_solve: relative residual %.3e above tol %.3e after %d inner iterations",
                    rnorm / gnorm, p.tol, total_inner);
    return HM_OK;
}

}  // namespace hm

using namespace hm;

extern "C" int hm_solve(const hm_matrix* H, const double* g, double* t, const hm_solve_params* sp,
                        hm_solve_info* info, void* stream)
{
    if (!H || !g || !t || !sp) return fail(HM_EINVAL, "hm_solve: NULL argument");
    if (H->rect) return fail(HM_EINVAL, "hm_solve: an evaluation operator (hm_build_point_tree) has only hm_eval_points and hm_amvm");
    hm_solve_params p = *sp;
    int rc = solve_check_params(H, p);
    if (rc) return rc;
    cudaStream_t s = (cudaStream_t)stream;
    // workspace, through the matrix's allocator
    Allocator al = H->alloc;
    al.stream = s;
    const size_t bytes = solve_workspace_bytes(3 * H->M, p.restart);
    void* ws = al.alloc(bytes);
    if (!ws) return fail(HM_ENOMEM, "hm_solve: workspace of %zu bytes", bytes);
    rc = solve_device(*H, g, t, p, info, s, ws, nullptr);
    cudaStreamSynchronize(s);
    al.release(ws, bytes);
    return rc;
}
