// hm_baca.cu -- block-adaptive ACA (Algorithm 3, Section 5) restricted to
// the single layer: restarted GMRES on A_k (the evaluation operator's product
// passes of hm_parts.cuh with the prefix ranks r_b of every block-kernel), the
// look-ahead parts by the adaptive product's part kernel, Doerfler marking
// of the blocks with the fewest blocks, refinement by `look` crosses, and
// Algorithm 1 on demand where asked.  Vectors live in cluster order (3 values
// per position) during the solve.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <map>
#include <numeric>
#include <vector>

#include "hm_parts.cuh"

namespace hm {
namespace {
constexpr int kBacaDotCtas = 296;  // partial sums of a dot product (2 per SM)

__global__ void baca_soa_kernel(const double* __restrict__ x, double* __restrict__ xs, int64_t M)
{
    const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= M) return;
#pragma unroll
    for (int a = 0; a < 3; ++a) xs[a * M + p] = x[3 * p + a];
}

__device__ __forceinline__ double baca_block_sum(double v, double* red)
{
    v = ev_sum32<double>(v);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
    __syncthreads();
    double s = 0.0;
    if (threadIdx.x == 0)
        for (int i = 0; i < (int)(blockDim.x >> 5); ++i) s += red[i];
    __syncthreads();
    return s;
}

// partial[i * gridDim.x + cta] = this CTA's share of Q_i . w, i < k (grid-stride
// slices, fixed order)
__global__ void __launch_bounds__(256) baca_mdot_kernel(const double* __restrict__ Q, int k, int64_t N,
                                                        const double* __restrict__ w, double* __restrict__ partial)
{
    __shared__ double red[8];
    for (int i = 0; i < k; ++i) {
        const double* q = Q + (int64_t)i * N;
        double s = 0.0;
        for (int64_t n = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; n < N; n += (int64_t)gridDim.x * blockDim.x)
            s += q[n] * w[n];
        const double t = baca_block_sum(s, red);
        if (threadIdx.x == 0) partial[(int64_t)i * gridDim.x + blockIdx.x] = t;
    }
}

// out[i] = the sum of row i of partial (G values), one CTA per i
__global__ void __launch_bounds__(256) baca_msum_kernel(const double* __restrict__ partial, int G,
                                                        double* __restrict__ out)
{
    __shared__ double red[8];
    double s = 0.0;
    for (int j = threadIdx.x; j < G; j += blockDim.x) s += partial[(int64_t)blockIdx.x * G + j];
    const double t = baca_block_sum(s, red);
    if (threadIdx.x == 0) out[blockIdx.x] = t;
}

// w += sgn sum_{i<k} h_i Q_i
__global__ void baca_maxpy_kernel(const double* __restrict__ Q, int k, int64_t N, const double* __restrict__ h,
                                  double sgn, double* __restrict__ w)
{
    const int64_t n = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (n >= N) return;
    double s = 0.0;
    for (int i = 0; i < k; ++i) s += h[i] * Q[(int64_t)i * N + n];
    w[n] += sgn * s;
}

// out = a x + b y (out may be x or y)
__global__ void baca_axpby_kernel(double a, const double* x, double b, const double* y, double* out, int64_t N)
{
    const int64_t n = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (n < N) out[n] = a * x[n] + b * y[n];
}

// bn[b] = ||D_b||^2 over the block's 3|t| part values (one CTA per block)
__global__ void __launch_bounds__(256) baca_blocknorm_kernel(const int64_t* __restrict__ doff,
                                                             const double* __restrict__ D, double* __restrict__ bn)
{
    __shared__ double red[8];
    const double* d = D + doff[blockIdx.x];
    const int64_t n = doff[blockIdx.x + 1] - doff[blockIdx.x];
    double s = 0.0;
    for (int64_t i = threadIdx.x; i < n; i += blockDim.x) s += d[i] * d[i];
    const double t = baca_block_sum(s, red);
    if (threadIdx.x == 0) bn[blockIdx.x] = t;
}
}  // namespace
}  // namespace hm

using namespace hm;

extern "C" int hm_baca(hm_matrix* H, const double* b, double* x, const hm_baca_params* prm, hm_baca_info* info,
                       hm_baca_step* hist, int32_t hist_cap, int32_t* block_ranks, void* stream)
{
    if (!H || !b || !x || !prm) return fail(HM_EINVAL, "hm_baca: NULL argument");
    if (H->rect) return fail(HM_EINVAL, "hm_baca: an evaluation operator is not a system matrix");
    if (prm->flags & ~HM_BACA_ACA_ON_DEMAND) return fail(HM_EINVAL, "hm_baca: unknown flags 0x%x", prm->flags);
    const bool lazy = (prm->flags & HM_BACA_ACA_ON_DEMAND) != 0;
    if (H->compacted) return fail(HM_EINVAL, "hm_baca: the FP64 data were released (hm_compact)");
    if (!lazy && (H->aca_deferred || !H->U64.p))
        return fail(HM_EINVAL, "hm_baca: no assembled ACA factors (HM_DEFER_ACA): use HM_BACA_ACA_ON_DEMAND");
    const double theta = prm->theta == 0.0 ? 0.8 : prm->theta;
    const double alpha = prm->alpha == 0.0 ? 10.0 : prm->alpha;
    const double tol0 = prm->tol0 == 0.0 ? 0.1 : prm->tol0;
    const double eps = prm->eps;
    const int r0 = prm->r0 == 0 ? 8 : prm->r0, look = prm->look == 0 ? 2 : prm->look;
    const int m = prm->restart == 0 ? 50 : prm->restart;
    const int64_t max_it = prm->max_iter == 0 ? 100000 : prm->max_iter;
    const int max_steps = prm->max_steps == 0 ? 1000 : prm->max_steps;
    if (!(theta > 0.0 && theta < 1.0)) return fail(HM_EINVAL, "hm_baca: theta %g outside (0, 1)", theta);
    if (!(alpha > 0.0) || !(tol0 > 0.0) || !(eps >= 0.0))
        return fail(HM_EINVAL, "hm_baca: alpha %g, tol0 %g must be > 0 and eps %g >= 0", alpha, tol0, eps);
    if (r0 < 1 || look < 1 || look > kAmvmMaxCross || m < 1 || m > 200 || max_it < 1 || max_steps < 0)
        return fail(HM_EINVAL, "hm_baca: r0 %d, look %d (1..%d), restart %d (1..200), max_iter or max_steps out of range",
                    r0, look, kAmvmMaxCross, m);
    if (hist_cap < 0) return fail(HM_EINVAL, "hm_baca: hist_cap < 0");
    cudaStream_t s = (cudaStream_t)stream;
    hm_matrix& Hm = *H;  // the product tables are built once and kept
    const cudaStream_t saved_stream = Hm.alloc.stream;
    Hm.alloc.stream = s;
    struct Restore {
        hm_matrix& h;
        cudaStream_t st;
        std::vector<DevBuf> arenas;  // factors of ACA on demand
        ~Restore()
        {
            for (DevBuf& a : arenas) h.alloc.release(a.p, a.bytes);
            h.alloc.stream = st;
        }
    } restore{Hm, saved_stream, {}};
    int rc;
    if (!Hm.ev[kEvXc].p && (rc = eval_prepare(Hm))) return rc;
    const int64_t M = H->M, N = 3 * M, nb = H->nadm;
    const double c1 = (1.0 + H->nu) * (3.0 - 4.0 * H->nu) / (2.0 * H->E * (1.0 - H->nu));
    const double c2 = (1.0 + H->nu) / (2.0 * H->E * (1.0 - H->nu));
    const DevBuf* ev = H->ev;

    Pool pool;
    pool.al = H->alloc;
    pool.al.stream = s;
    const int G = kBacaDotCtas;
    double* Q = pool.get<double>((size_t)(m + 1) * N);
    double* bc = pool.get<double>((size_t)N);
    double* xc = pool.get<double>((size_t)N);
    double* rv = pool.get<double>((size_t)N);
    double* yv = pool.get<double>((size_t)N);
    double* ev_e = pool.get<double>((size_t)N);
    double* Dl = pool.get<double>((size_t)std::max<int64_t>(H->ev_parts, 1));
    double* bn = pool.get<double>((size_t)nb);
    double* partial = pool.get<double>((size_t)(m + 1) * G);
    double* dots = pool.get<double>((size_t)(m + 1));
    double* coef = pool.get<double>((size_t)(m + 1));
    int32_t* rk = pool.get<int32_t>((size_t)nb * 7);
    AmvmItem* items = pool.get<AmvmItem>((size_t)nb);
    const double** uptr = pool.get<const double*>((size_t)nb * 7);
    const double** vptr = pool.get<const double*>((size_t)nb * 7);
    if (!Q || !bc || !xc || !rv || !yv || !ev_e || !Dl || !bn || !partial || !dots || !coef || !rk || !items ||
        !uptr || !vptr)
        return fail(HM_ENOMEM, "hm_baca: workspace (%d Krylov vectors of %lld)", m + 1, (long long)N);
    // the crosses of every block-kernel: pointers to U (k x m) and V (k x n)
    // and how many there are (krank): the assembled factors, or, on demand,
    // the arenas of the ACA runs so far (with the w slot offsets coff)
    std::vector<const double*> up((size_t)nb * 7, nullptr), vp((size_t)nb * 7, nullptr);
    std::vector<int32_t> krank((size_t)nb * 7, 0), kflags((size_t)nb * 7, 0);
    std::vector<int64_t> hcoff((size_t)nb * 7, 0);
    int32_t* d_krank = pool.get<int32_t>((size_t)nb * 7);
    int64_t* d_coff = pool.get<int64_t>((size_t)nb * 7);
    double* w_od = nullptr;  // w of the on-demand factors
    int64_t w_od_cap = 0;
    if (!d_krank || !d_coff) return fail(HM_ENOMEM, "hm_baca: rank tables");
    const int kcap = std::max(1, (int)H->prm.kmax);
    AcaResume rs{};
    std::vector<const double*> prev((size_t)nb * 7, nullptr);
    const double** d_prev = nullptr;
    if (lazy) {
        std::vector<int64_t> zoff((size_t)nb * 7 + 1, 0);
        for (int64_t q = 0; q < nb * 7; ++q) zoff[(size_t)q + 1] = zoff[(size_t)q] + H->adm_h[(size_t)(q / 7)].m;
        rs.k = pool.get<int32_t>((size_t)nb * 7);
        rs.nz = pool.get<int32_t>((size_t)nb * 7);
        rs.irow = pool.get<int32_t>((size_t)nb * 7);
        rs.flags = pool.get<int32_t>((size_t)nb * 7);
        rs.S2 = pool.get<double>((size_t)nb * 7);
        rs.Z = pool.get<unsigned char>((size_t)zoff[(size_t)nb * 7]);
        int64_t* d_zoff = pool.get<int64_t>(zoff.size());
        d_prev = pool.get<const double*>((size_t)nb * 7);
        if (!rs.k || !rs.nz || !rs.irow || !rs.flags || !rs.S2 || !rs.Z || !d_zoff || !d_prev)
            return fail(HM_ENOMEM, "hm_baca: ACA state");
        if ((rc = put(d_zoff, zoff, s))) return rc;
        HM_CUDA(cudaMemsetAsync(rs.flags, 0, (size_t)nb * 7 * 4, s));
        rs.zoff = d_zoff;
        rs.prevU = d_prev;
    } else {
        for (int64_t q = 0; q < nb * 7; ++q) {
            up[(size_t)q] = H->U64.as<double>() + H->uoff_h[(size_t)q];
            vp[(size_t)q] = H->V64.as<double>() + H->voff_h[(size_t)q];
            krank[(size_t)q] = H->rank_h[(size_t)q];
        }
    }
    // Algorithm 1 on demand for the tasks bkl to kmax crosses, resumed where a
    // task ran before (prev), then the tables of the product
    auto run_aca = [&](const std::vector<int32_t>& bkl, int kmax) -> int {
        if (bkl.empty()) return HM_OK;
        std::vector<int32_t> rr;
        std::vector<int64_t> oo;
        DevBuf arena;
        int rc2 = put(d_prev, prev, s);
        if (rc2) return rc2;
        rc2 = aca_on_demand(Hm, bkl, kmax, s, arena, rr, oo, &rs);
        if (arena.p) restore.arenas.push_back(arena);
        if (rc2) return rc2;
        for (size_t q = 0; q < bkl.size(); ++q) {
            const int32_t v = bkl[q];
            up[(size_t)v] = arena.as<double>() + oo[q];
            vp[(size_t)v] = up[(size_t)v] + (int64_t)rr[q] * H->adm_h[(size_t)(v / 7)].m;
            krank[(size_t)v] = rr[q];
        }
        HM_CUDA(cudaMemcpyAsync(kflags.data(), rs.flags, kflags.size() * 4, cudaMemcpyDeviceToHost, s));
        HM_CUDA(cudaStreamSynchronize(s));
        return HM_OK;
    };
    auto upload_factors = [&]() -> int {
        int64_t c = 0;
        for (int64_t q = 0; q < nb * 7; ++q) {
            hcoff[(size_t)q] = c;
            c += krank[(size_t)q];
        }
        if (lazy && c > w_od_cap) {
            w_od_cap = c + c / 2 + 1;
            w_od = pool.get<double>((size_t)(3 * w_od_cap));
            if (!w_od) return fail(HM_ENOMEM, "hm_baca: w of %lld crosses", (long long)w_od_cap);
        }
        int rc2;
        if ((rc2 = put(uptr, up, s)) || (rc2 = put(vptr, vp, s)) || (rc2 = put(d_krank, krank, s)) ||
            (rc2 = put(d_coff, hcoff, s)))
            return rc2;
        return HM_OK;
    };
    if (lazy) {
        std::vector<int32_t> all;
        for (int64_t q = 0; q < nb * 7; ++q)
            if (!(H->flags_h[(size_t)q] & 32)) all.push_back((int32_t)q);  // 32: identically zero kernel
        if ((rc = run_aca(all, std::min(r0 + look, kcap)))) return rc;
    }
    if ((rc = upload_factors())) return rc;
    const unsigned gM = (unsigned)((M + 255) / 256), gN = (unsigned)((N + 255) / 256);
    auto grid = [&](int64_t warps) {
        return (unsigned)std::max<int64_t>(1, std::min<int64_t>(H->ev_grid, (warps + kEvWarps - 1) / kEvWarps));
    };
    // A_k xin -> yout (cluster order): the evaluation passes with ranks rk
    auto apply = [&](const double* xin, double* yout) -> int {
        double* xs = ev[kEvXc].as<double>();
        baca_soa_kernel<<<gM, 256, 0, s>>>(xin, xs, M);
        HM_CUDA(cudaGetLastError());
        if (H->ev_nnear > 0) {
            ev_near_kernel<double><<<grid(H->ev_nnear), kEvThreads, 0, s>>>(
                ev[kEvNear].as<int2>(), H->ev_nnear, H->d_near.as<Blk>(), H->d_noff.as<int64_t>(),
                H->N64.as<double>(), xs, M, c1, c2, ev[kEvNdoff].as<int64_t>(), ev[kEvDn].as<double>());
            HM_CUDA(cudaGetLastError());
        }
        if (nb > 0) {
            double* w = lazy ? w_od : ev[kEvW].as<double>();
            ev_fwd_kernel<double><<<grid(nb * 7), kEvThreads, 0, s>>>(H->d_adm.as<Blk>(), rk, H->d_voff.as<int64_t>(),
                                                                      d_coff, H->V64.as<double>(), vptr, xs, M,
                                                                      nb * 7, w);
            HM_CUDA(cudaGetLastError());
            ev_back_kernel<double><<<grid(H->ev_nback), kEvThreads, 0, s>>>(
                ev[kEvBack].as<int2>(), H->ev_nback, H->d_adm.as<Blk>(), rk, H->d_uoff.as<int64_t>(), d_coff,
                H->U64.as<double>(), uptr, w, c1, c2, ev[kEvDoff].as<int64_t>(), ev[kEvD].as<double>());
            HM_CUDA(cudaGetLastError());
        }
        ev_rowsum_kernel<double><<<gM, 256, 0, s>>>(ev[kEvIpos].as<int32_t>(), ev[kEvAptr].as<int32_t>(),
                                                   ev[kEvAidx].as<int32_t>(), H->d_adm.as<Blk>(),
                                                   ev[kEvDoff].as<int64_t>(), ev[kEvD].as<double>(),
                                                   ev[kEvNptr].as<int32_t>(), ev[kEvNidx].as<int32_t>(),
                                                   H->d_near.as<Blk>(), ev[kEvNdoff].as<int64_t>(),
                                                   ev[kEvDn].as<double>(), yout, M);
        HM_CUDA(cudaGetLastError());
        return HM_OK;
    };
    // dot products Q_i . w for i < k, into host out (deterministic)
    std::vector<double> hdots((size_t)(m + 1));
    auto mdot = [&](const double* Qb, int k, const double* w, double* out) -> int {
        baca_mdot_kernel<<<G, 256, 0, s>>>(Qb, k, N, w, partial);
        HM_CUDA(cudaGetLastError());
        baca_msum_kernel<<<(unsigned)k, 256, 0, s>>>(partial, G, dots);
        HM_CUDA(cudaGetLastError());
        HM_CUDA(cudaMemcpyAsync(out, dots, (size_t)k * sizeof(double), cudaMemcpyDeviceToHost, s));
        HM_CUDA(cudaStreamSynchronize(s));
        return HM_OK;
    };
    auto norm = [&](const double* v, double& out) -> int {
        double t = 0.0;
        int rc2 = mdot(v, 1, v, &t);
        out = std::sqrt(std::max(t, 0.0));
        return rc2;
    };
    // the look-ahead parts (A^_k - A_k)_b xin into Dl, their sum e, ||e||,
    // and (optionally) the squared part norms of the blocks
    std::vector<int32_t> r((size_t)nb, r0);
    std::vector<AmvmItem> hitems((size_t)nb);
    std::vector<double> hbn((size_t)nb);
    auto lookahead = [&](const double* xin, bool norms, double& enorm) -> int {
        if (nb == 0) {
            enorm = 0.0;
            if (norms) std::fill(hbn.begin(), hbn.end(), 0.0);
            return HM_OK;
        }
        amvm_part_kernel<<<(unsigned)nb, kAmvmThreads, 0, s>>>(items, H->d_adm.as<Blk>(), d_krank, uptr, vptr, xin,
                                                              c1, c2, ev[kEvDoff].as<int64_t>(), Dl);
        HM_CUDA(cudaGetLastError());
        amvm_rowsum_kernel<<<gM, 256, 0, s>>>(ev[kEvIpos].as<int32_t>(), ev[kEvAptr].as<int32_t>(),
                                             ev[kEvAidx].as<int32_t>(), H->d_adm.as<Blk>(), ev[kEvDoff].as<int64_t>(),
                                             Dl, nullptr, 0, ev_e, M);
        HM_CUDA(cudaGetLastError());
        int rc2 = norm(ev_e, enorm);
        if (rc2) return rc2;
        if (norms) {
            baca_blocknorm_kernel<<<(unsigned)nb, 256, 0, s>>>(ev[kEvDoff].as<int64_t>(), Dl, bn);
            HM_CUDA(cudaGetLastError());
            HM_CUDA(cudaMemcpyAsync(hbn.data(), bn, (size_t)nb * sizeof(double), cudaMemcpyDeviceToHost, s));
            HM_CUDA(cudaStreamSynchronize(s));
        }
        return HM_OK;
    };
    auto upload_ranks = [&]() -> int {
        std::vector<int32_t> hrk((size_t)nb * 7);
        for (int64_t bb = 0; bb < nb; ++bb) {
            for (int k = 0; k < 7; ++k)
                hrk[(size_t)(bb * 7 + k)] = std::min(r[(size_t)bb], krank[(size_t)(bb * 7 + k)]);
            hitems[(size_t)bb] = AmvmItem{(int32_t)bb, r[(size_t)bb], r[(size_t)bb] + look, 0};
        }
        int rc2;
        if ((rc2 = put(rk, hrk, s)) || (rc2 = put(items, hitems, s))) return rc2;
        return HM_OK;
    };
    if ((rc = upload_ranks())) return rc;

    amvm_gather_kernel<<<gM, 256, 0, s>>>(H->d_perm.as<int32_t>(), b, bc, M);
    HM_CUDA(cudaGetLastError());
    HM_CUDA(cudaMemsetAsync(xc, 0, (size_t)N * sizeof(double), s));
    double bnorm = 0.0;
    if ((rc = norm(bc, bnorm))) return rc;
    const double floor_res = 1e-13 * bnorm;
    bool x_zero = true;
    int64_t its_total = 0;

    // step 2: restarted GMRES(m) from the current x (classical Gram-Schmidt
    // applied twice, Givens rotations on the host)
    double last_res = 0.0;
    auto solve = [&](int64_t& its_step) -> int {
        its_step = 0;
        std::vector<double> Hh((size_t)(m + 1) * m), cs((size_t)m), sn((size_t)m), g((size_t)(m + 1)),
            h((size_t)(m + 1)), h2((size_t)(m + 1)), y((size_t)m);
        for (;;) {
            int rc2;
            if ((rc2 = apply(xc, yv))) return rc2;
            baca_axpby_kernel<<<gN, 256, 0, s>>>(1.0, bc, -1.0, yv, rv, N);
            HM_CUDA(cudaGetLastError());
            double beta = 0.0;
            if ((rc2 = norm(rv, beta))) return rc2;
            last_res = beta;
            double tol = tol0 * bnorm;
            if (!x_zero) {
                double en = 0.0;
                if ((rc2 = lookahead(xc, false, en))) return rc2;
                tol = alpha * en;
            }
            if (beta <= tol || beta <= floor_res || its_total >= max_it) return HM_OK;
            baca_axpby_kernel<<<gN, 256, 0, s>>>(1.0 / beta, rv, 0.0, rv, Q, N);
            HM_CUDA(cudaGetLastError());
            std::fill(g.begin(), g.end(), 0.0);
            g[0] = beta;
            int jend = 0;
            for (int j = 0; j < m; ++j) {
                double* w = Q + (int64_t)(j + 1) * N;
                if ((rc2 = apply(Q + (int64_t)j * N, w))) return rc2;
                if ((rc2 = mdot(Q, j + 1, w, h.data()))) return rc2;
                baca_maxpy_kernel<<<gN, 256, 0, s>>>(Q, j + 1, N, dots, -1.0, w);
                HM_CUDA(cudaGetLastError());
                if ((rc2 = mdot(Q, j + 1, w, h2.data()))) return rc2;
                baca_maxpy_kernel<<<gN, 256, 0, s>>>(Q, j + 1, N, dots, -1.0, w);
                HM_CUDA(cudaGetLastError());
                double hn = 0.0;
                if ((rc2 = norm(w, hn))) return rc2;
                ++its_step;
                ++its_total;
                for (int i = 0; i <= j; ++i) Hh[(size_t)i * m + j] = h[(size_t)i] + h2[(size_t)i];
                Hh[(size_t)(j + 1) * m + j] = hn;
                for (int i = 0; i < j; ++i) {
                    const double a = Hh[(size_t)i * m + j], c = Hh[(size_t)(i + 1) * m + j];
                    Hh[(size_t)i * m + j] = cs[(size_t)i] * a + sn[(size_t)i] * c;
                    Hh[(size_t)(i + 1) * m + j] = -sn[(size_t)i] * a + cs[(size_t)i] * c;
                }
                const double a = Hh[(size_t)j * m + j], c = Hh[(size_t)(j + 1) * m + j];
                const double rr = std::hypot(a, c);
                cs[(size_t)j] = rr > 0.0 ? a / rr : 1.0;
                sn[(size_t)j] = rr > 0.0 ? c / rr : 0.0;
                Hh[(size_t)j * m + j] = rr;
                Hh[(size_t)(j + 1) * m + j] = 0.0;
                g[(size_t)j + 1] = -sn[(size_t)j] * g[(size_t)j];
                g[(size_t)j] = cs[(size_t)j] * g[(size_t)j];
                jend = j + 1;
                if (std::fabs(g[(size_t)j + 1]) <= tol || hn <= 1e-300 || its_total >= max_it) break;
                baca_axpby_kernel<<<gN, 256, 0, s>>>(1.0 / hn, w, 0.0, w, w, N);
                HM_CUDA(cudaGetLastError());
            }
            for (int i = jend - 1; i >= 0; --i) {
                double t = g[(size_t)i];
                for (int l = i + 1; l < jend; ++l) t -= Hh[(size_t)i * m + l] * y[(size_t)l];
                y[(size_t)i] = Hh[(size_t)i * m + i] != 0.0 ? t / Hh[(size_t)i * m + i] : 0.0;
            }
            HM_CUDA(cudaMemcpyAsync(coef, y.data(), (size_t)jend * sizeof(double), cudaMemcpyHostToDevice, s));
            baca_maxpy_kernel<<<gN, 256, 0, s>>>(Q, jend, N, coef, 1.0, xc);
            HM_CUDA(cudaGetLastError());
            x_zero = false;
        }
    };

    int k = 0;
    int64_t marked_total = 0;
    double Ek = 0.0, en = 0.0;
    for (;;) {
        int64_t its_step = 0;
        if ((rc = solve(its_step))) return rc;
        if ((rc = lookahead(xc, true, en))) return rc;
        double E2 = 0.0;
        for (int64_t bb = 0; bb < nb; ++bb) E2 += hbn[(size_t)bb];
        Ek = std::sqrt(E2);
        std::vector<int64_t> ord;
        bool stop = Ek <= eps * bnorm || k >= max_steps;
        int32_t nmarked = 0;
        if (!stop) {
            // step 3: the fewest blocks with E_k(M_k) >= theta E_k: the largest
            // parts first (ties: lower block index)
            ord.resize((size_t)nb);
            std::iota(ord.begin(), ord.end(), 0);
            std::sort(ord.begin(), ord.end(), [&](int64_t p1, int64_t p2) {
                return hbn[(size_t)p1] > hbn[(size_t)p2] || (hbn[(size_t)p1] == hbn[(size_t)p2] && p1 < p2);
            });
            const double target = theta * Ek * theta * Ek;
            double acc = 0.0;
            std::map<int, std::vector<int32_t>> rerun;  // on demand: tasks to extend, by their new kmax
            for (int64_t bb : ord) {
                if (acc >= target || hbn[(size_t)bb] == 0.0) break;
                acc += hbn[(size_t)bb];
                r[(size_t)bb] += look;  // step 4: A_{k+1} = A^_k on the block
                ++nmarked;
                if (lazy)
                    for (int kk = 0; kk < 7; ++kk) {
                        const size_t q = (size_t)bb * 7 + (size_t)kk;
                        const int want = std::min(r[(size_t)bb] + look, kcap);
                        // only a run that stopped at its kmax has more crosses to give
                        if (!(H->flags_h[q] & 32) && (kflags[q] & 1) && want > krank[q])
                            rerun[want].push_back((int32_t)q);
                    }
            }
            if (!rerun.empty()) {
                std::fill(prev.begin(), prev.end(), nullptr);
                for (auto& kv : rerun)
                    for (int32_t q : kv.second) prev[(size_t)q] = up[(size_t)q];
                for (auto& kv : rerun)
                    if ((rc = run_aca(kv.second, kv.first))) return rc;
                if ((rc = upload_factors())) return rc;
            }
        }
        if (k < hist_cap && hist)
            hist[k] = hm_baca_step{Ek, last_res, en, (int32_t)its_step, nmarked};
        if (stop || nmarked == 0) break;
        marked_total += nmarked;
        if ((rc = upload_ranks())) return rc;
        ++k;
    }
    amvm_scatter_kernel<<<gM, 256, 0, s>>>(H->d_perm.as<int32_t>(), xc, x, M);
    HM_CUDA(cudaGetLastError());
    HM_CUDA(cudaStreamSynchronize(s));
    if (info) {
        info->steps = k;
        info->gmres_iterations = its_total;
        info->E = Ek;
        info->rel_residual = bnorm > 0.0 ? last_res / bnorm : 0.0;
        info->b_norm = bnorm;
        int64_t used = 0, full = 0;
        for (int64_t bb = 0; bb < nb; ++bb)
            for (int kk = 0; kk < 7; ++kk) {
                const int32_t K = krank[(size_t)(bb * 7 + kk)];  // on demand: the crosses computed
                used += std::min<int64_t>(K, r[(size_t)bb]);
                full += K;
            }
        info->crosses_used = used;
        info->crosses_full = full;
        info->marked_total = marked_total;
    }
    if (block_ranks)
        for (int64_t bb = 0; bb < nb; ++bb) block_ranks[bb] = r[(size_t)bb];
    return HM_OK;
}

