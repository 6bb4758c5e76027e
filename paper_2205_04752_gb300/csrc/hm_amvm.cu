// hm_amvm.cu -- adaptive matrix-vector multiplication (Algorithm 2, Section
// 3) on the device, FP64, from the assembled ACA factors.
//
// A_k keeps the first r_b crosses of each of the seven ACA sequences of every
// admissible block (the whole sequence when it is shorter), the look-ahead
// A^_k the first r_b + L; near blocks are exact in both.  With b_k = A_k x
// and the look-ahead parts D_b = (A^_k - A_k)_b x, the estimator is gamma_k =
// ||sum_b D_b|| = ||b^_k - b_k||.  Marking (step 3) goes through the rows in
// decreasing |(b^_k - b_k)_i| and adds every block t x s with i in t and
// |(D_b)_i| >= (1 - theta)(c_sp N_r N_c)^{-1/2} gamma_k (N_r rows, N_c
// columns: 3M each, or 3 points x 3M for the evaluation operator) until
// gamma_k - gamma_k(P_k) >= theta gamma_k; a marked block takes the
// look-ahead ranks (step 4).  The loop ends when gamma_k <= eps ||b^_k||.
//
// Device work per iteration (kernels shared with the other block products in
// hm_parts.cuh): the look-ahead parts of the blocks refined in the previous
// step (one CTA per block: V^T x of the new crosses by warp reductions, then
// U times them row by row), the row sums of all parts (each
// position adds the parts of the blocks whose row cluster holds it, in block
// order: deterministic), and the update of b_k by the marked blocks' parts.
// The marking runs on the device too: the rows sorted by their error, the
// row at which each block joins the marked set, and a bisection for the row
// at which the Doerfler condition holds (see step 3 below).
//
// The crosses come either from the assembled ACA (prefixes of its sequences)
// or, with HM_AMVM_ACA_ON_DEMAND, from Algorithm 1 run on demand: every
// block-kernel to r0 + look crosses first, a refined block's kernels on to
// its new r_b + look, resumed from the state their last run ended in (its
// crosses, Z, the next row and ||S_k||), so that only the crosses the
// refinement reaches are ever computed -- the combination of assembly and
// product of Section 3.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <map>
#include <numeric>
#include <vector>

#include "hm_parts.cuh"

namespace hm {
namespace {
// ---- step 3 on the device
// the rows in decreasing |e_i| (ties: increasing i): a bitonic sort of (key,
// row) over P = a power of two >= N (padding keys -1 sort last)
__global__ void amvm_sort_init_kernel(const double* __restrict__ e, int64_t N, int64_t P, double* __restrict__ key,
                                      int32_t* __restrict__ idx)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= P) return;
    key[i] = i < N ? fabs(e[i]) : -1.0;
    idx[i] = (int32_t)i;
}

__global__ void amvm_bitonic_kernel(double* __restrict__ key, int32_t* __restrict__ idx, int64_t P, int64_t j,
                                    int64_t k)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= P) return;
    const int64_t l = i ^ j;
    if (l <= i) return;
    const double ka = key[i], kb = key[l];
    const int32_t ia = idx[i], ib = idx[l];
    const bool a_first = ka > kb || (ka == kb && ia < ib);
    const bool up = (i & k) == 0;
    if (a_first != up) {
        key[i] = kb;
        key[l] = ka;
        idx[i] = ib;
        idx[l] = ia;
    }
}

__global__ void amvm_rowpos_kernel(const int32_t* __restrict__ idx, int64_t N, int32_t* __restrict__ rowpos)
{
    const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p < N) rowpos[idx[p]] = (int32_t)p;
}

// first[b]: the earliest position (in the sorted rows) of a row of block b
// whose part reaches thr, INT_MAX if none; one CTA per block
__global__ void __launch_bounds__(256) amvm_first_kernel(const Blk* __restrict__ adm,
                                                         const int64_t* __restrict__ doff,
                                                         const double* __restrict__ D,
                                                         const int32_t* __restrict__ rowpos, double thr,
                                                         int32_t* __restrict__ first)
{
    __shared__ int32_t red[8];
    const int b = blockIdx.x;
    const Blk bk = adm[b];
    const double* d = D + doff[b];
    const int64_t r0 = 3 * (int64_t)bk.t0;
    int32_t best = INT_MAX;
    for (int z = threadIdx.x; z < 3 * bk.m; z += blockDim.x)
        if (fabs(d[z]) >= thr) best = min(best, rowpos[r0 + z]);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) best = min(best, __shfl_xor_sync(0xffffffffu, best, o));
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = best;
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int w = 1; w < (int)(blockDim.x >> 5); ++w) best = min(best, red[w]);
        first[b] = best;
    }
}

__global__ void amvm_cut_kernel(const int32_t* __restrict__ first, int64_t nb, int32_t j, uint8_t* __restrict__ flags)
{
    const int64_t b = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (b < nb) flags[b] = first[b] <= j ? 1 : 0;
}

// the squares of e - (the flagged parts), summed per CTA (fixed order)
__global__ void __launch_bounds__(256) amvm_rest_kernel(const int32_t* __restrict__ ipos,
                                                        const int32_t* __restrict__ aptr,
                                                        const int32_t* __restrict__ aidx,
                                                        const Blk* __restrict__ adm,
                                                        const int64_t* __restrict__ doff,
                                                        const double* __restrict__ D,
                                                        const uint8_t* __restrict__ flags,
                                                        const double* __restrict__ e, int64_t M,
                                                        double* __restrict__ partial)
{
    __shared__ double red[8];
    const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    double v = 0.0;
    if (p < M) {
        const int I = ipos[p];
        double s0 = 0.0, s1 = 0.0, s2 = 0.0;
        for (int q = aptr[I]; q < aptr[I + 1]; ++q) {
            const int b = aidx[q];
            if (!flags[b]) continue;
            const double* d = D + doff[b] + 3 * (p - adm[b].t0);
            s0 += d[0];
            s1 += d[1];
            s2 += d[2];
        }
        const double r0 = e[3 * p] - s0, r1 = e[3 * p + 1] - s1, r2 = e[3 * p + 2] - s2;
        v = r0 * r0 + r1 * r1 + r2 * r2;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int w = 1; w < (int)(blockDim.x >> 5); ++w) v += red[w];
        partial[blockIdx.x] = v;
    }
}

// out = the sum of n partial sums, in a fixed order (one CTA)
__global__ void __launch_bounds__(256) amvm_sum_kernel(const double* __restrict__ partial, int64_t n,
                                                       double* __restrict__ out)
{
    __shared__ double red[8];
    double v = 0.0;
    for (int64_t i = threadIdx.x; i < n; i += blockDim.x) v += partial[i];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int w = 1; w < (int)(blockDim.x >> 5); ++w) v += red[w];
        out[0] = v;
    }
}

}  // namespace
}  // namespace hm

using namespace hm;

using namespace hm;

extern "C" int hm_amvm(hm_matrix* H, const double* x, double* y, const hm_amvm_params* prm,
                       hm_amvm_info* info, double* gamma_hist, double* gamma_rest_hist, int32_t hist_cap,
                       int32_t* block_ranks, void* stream)
{
    if (!H || !x || !y || !prm) return fail(HM_EINVAL, "hm_amvm: NULL argument");
    if (H->dl) return fail(HM_EINVAL, "hm_amvm: the double layer's K_Delta is applied by hm_double_layer_matvec");
    if (prm->flags & ~HM_AMVM_ACA_ON_DEMAND) return fail(HM_EINVAL, "hm_amvm: unknown flags 0x%x", prm->flags);
    const bool lazy = (prm->flags & HM_AMVM_ACA_ON_DEMAND) != 0;
    if (H->compacted) return fail(HM_EINVAL, "hm_amvm: the FP64 data were released (hm_compact)");
    if (!lazy && (H->aca_deferred || !H->U64.p))
        return fail(HM_EINVAL, "hm_amvm: no assembled ACA factors (HM_DEFER_ACA): use HM_AMVM_ACA_ON_DEMAND");
    const double theta = prm->theta == 0.0 ? 0.7 : prm->theta;
    const double eps = prm->eps;
    const int r0 = prm->r0 == 0 ? 2 : prm->r0, look = prm->look == 0 ? 2 : prm->look;
    const int max_iter = prm->max_iter == 0 ? 1000 : prm->max_iter;
    if (!(theta > 0.0 && theta < 1.0)) return fail(HM_EINVAL, "hm_amvm: theta %g outside (0, 1)", theta);
    if (!(eps >= 0.0)) return fail(HM_EINVAL, "hm_amvm: eps %g < 0", eps);
    if (r0 < 1 || look < 1 || r0 > kAmvmMaxCross || look > kAmvmMaxCross || max_iter < 0)
        return fail(HM_EINVAL, "hm_amvm: r0 %d / look %d outside 1..%d or max_iter %d < 0", r0, look, kAmvmMaxCross,
                    max_iter);
    if (hist_cap < 0) return fail(HM_EINVAL, "hm_amvm: hist_cap < 0");
    cudaStream_t s = (cudaStream_t)stream;
    hm_matrix& Hm = *H;  // on-demand ACA allocates through the matrix's allocator
    const cudaStream_t saved_stream = Hm.alloc.stream;
    Hm.alloc.stream = s;
    struct Restore {
        hm_matrix& h;
        cudaStream_t st;
        std::vector<DevBuf> arenas;
        ~Restore()
        {
            for (DevBuf& a : arenas) h.alloc.release(a.p, a.bytes);
            h.alloc.stream = st;
        }
    } restore{Hm, saved_stream, {}};
    // rows: the 3 Mr dofs of the row points (Mr = M unless H is the
    // evaluation operator); columns: the 3M dofs of the triangles
    const int64_t M = H->M, Mr = H->Mr, nb = H->nadm, N = 3 * Mr, Ncol = 3 * M;
    if (M > INT32_MAX / 3 || Mr > INT32_MAX / 3) return fail(HM_EINVAL, "hm_amvm: mesh too large");
    const double c1 = (1.0 + H->nu) * (3.0 - 4.0 * H->nu) / (2.0 * H->E * (1.0 - H->nu));
    const double c2 = (1.0 + H->nu) / (2.0 * H->E * (1.0 - H->nu));

    // ---- host tables: row intervals, block lists, part offsets, c_sp
    std::vector<int64_t> bounds = {0, Mr};
    for (const Blk& b : H->adm_h) {
        bounds.push_back(b.t0);
        bounds.push_back(b.t0 + b.m);
    }
    for (const Blk& b : H->near_h) {
        bounds.push_back(b.t0);
        bounds.push_back(b.t0 + b.m);
    }
    std::sort(bounds.begin(), bounds.end());
    bounds.erase(std::unique(bounds.begin(), bounds.end()), bounds.end());
    const RowLists ra = row_lists(Mr, bounds, H->adm_h), rn = row_lists(Mr, bounds, H->near_h);
    std::vector<int64_t> doff((size_t)nb + 1, 0);
    for (int64_t b = 0; b < nb; ++b) doff[(size_t)b + 1] = doff[(size_t)b] + 3 * (int64_t)H->adm_h[(size_t)b].m;
    int csp = 0;
    {
        // Section 2.1: the most blocks of P that share a row or a column cluster
        std::map<std::pair<int32_t, int32_t>, int> rows, cols;
        for (const auto* L : {&H->adm_h, &H->near_h})
            for (const Blk& b : *L) {
                csp = std::max(csp, ++rows[{b.t0, b.m}]);
                csp = std::max(csp, ++cols[{b.s0, b.n}]);
            }
    }

    // ---- device buffers
    Pool pool;
    pool.al = H->alloc;
    pool.al.stream = s;
    double* xc = pool.get<double>((size_t)Ncol);
    double* bk = pool.get<double>((size_t)N);
    double* e = pool.get<double>((size_t)N);
    double* D = pool.get<double>((size_t)doff[(size_t)nb]);
    int32_t* d_ipos = pool.get<int32_t>((size_t)Mr);
    int32_t* d_aptr = pool.get<int32_t>(ra.ptr.size());
    int32_t* d_aidx = pool.get<int32_t>(ra.idx.size());
    int32_t* d_nptr = pool.get<int32_t>(rn.ptr.size());
    int32_t* d_nidx = pool.get<int32_t>(rn.idx.size());
    int64_t* d_doff = pool.get<int64_t>(doff.size());
    AmvmItem* d_items = pool.get<AmvmItem>((size_t)nb);
    uint8_t* d_flags = pool.get<uint8_t>((size_t)nb);
    int64_t P = 1;
    while (P < N) P <<= 1;
    double* d_key = pool.get<double>((size_t)P);
    int32_t* d_sidx = pool.get<int32_t>((size_t)P);
    int32_t* d_rowpos = pool.get<int32_t>((size_t)N);
    int32_t* d_first = pool.get<int32_t>((size_t)nb);
    double* d_part = pool.get<double>((size_t)(Mr + 255) / 256 + 1);
    double* d_norm = pool.get<double>(1);
    if (!d_key || !d_sidx || !d_rowpos || !d_first || !d_part || !d_norm)
        return fail(HM_ENOMEM, "hm_amvm: marking workspace");
    const double** d_uptr = pool.get<const double*>((size_t)nb * 7);
    const double** d_vptr = pool.get<const double*>((size_t)nb * 7);
    int32_t* d_krank = pool.get<int32_t>((size_t)nb * 7);
    if (!xc || !bk || !e || !D || !d_ipos || !d_aptr || !d_aidx || !d_nptr || !d_nidx || !d_doff || !d_items ||
        !d_flags || !d_uptr || !d_vptr || !d_krank)
        return fail(HM_ENOMEM, "hm_amvm: workspace (%lld parts)", (long long)doff[(size_t)nb]);
    int rc;
    if ((rc = put(d_ipos, ra.ipos, s)) || (rc = put(d_aptr, ra.ptr, s)) || (rc = put(d_aidx, ra.idx, s)) ||
        (rc = put(d_nptr, rn.ptr, s)) || (rc = put(d_nidx, rn.idx, s)) || (rc = put(d_doff, doff, s)))
        return rc;
    const unsigned gM = (unsigned)((Mr + 255) / 256), gMc = (unsigned)((M + 255) / 256);
    const Blk* d_adm = H->d_adm.as<Blk>();
    // the crosses of every block-kernel: pointers to U (k x m) and V (k x n),
    // and how many there are (krank); on demand, also the kmax of the run
    // that produced them
    std::vector<const double*> uptr((size_t)nb * 7, nullptr), vptr((size_t)nb * 7, nullptr);
    std::vector<int32_t> krank((size_t)nb * 7, 0), kflags((size_t)nb * 7, 0);
    const int kcap = std::max(1, (int)H->prm.kmax);
    // resumable ACA state (on demand)
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
            return fail(HM_ENOMEM, "hm_amvm: ACA state");
        if ((rc = put(d_zoff, zoff, s))) return rc;
        HM_CUDA(cudaMemsetAsync(rs.flags, 0, (size_t)nb * 7 * 4, s));
        rs.zoff = d_zoff;
        rs.prevU = d_prev;
    }
    auto run_aca = [&](const std::vector<int32_t>& bkl, int kmax) -> int {
        if (bkl.empty()) return HM_OK;
        std::vector<int32_t> rr;
        std::vector<int64_t> oo;
        DevBuf arena;
        int rc2 = put(d_prev, prev, s);  // resume from these (null: afresh)
        if (rc2) return rc2;
        rc2 = aca_on_demand(Hm, bkl, kmax, s, arena, rr, oo, &rs);
        if (arena.p) restore.arenas.push_back(arena);
        if (rc2) return rc2;
        for (size_t q = 0; q < bkl.size(); ++q) {
            const int32_t v = bkl[q];
            const Blk& bb = H->adm_h[(size_t)(v / 7)];
            uptr[(size_t)v] = arena.as<double>() + oo[q];
            vptr[(size_t)v] = uptr[(size_t)v] + (int64_t)rr[q] * bb.m;
            krank[(size_t)v] = rr[q];
        }
        // the exit flags: bit 0 = stopped at kmax (the sequence goes on)
        HM_CUDA(cudaMemcpyAsync(kflags.data(), rs.flags, kflags.size() * 4, cudaMemcpyDeviceToHost, s));
        HM_CUDA(cudaStreamSynchronize(s));
        return HM_OK;
    };
    auto upload_factors = [&]() -> int {
        int rc2;
        if ((rc2 = put(d_uptr, uptr, s)) || (rc2 = put(d_vptr, vptr, s)) || (rc2 = put(d_krank, krank, s)))
            return rc2;
        return HM_OK;
    };
    if (lazy) {
        std::vector<int32_t> all;
        for (int64_t q = 0; q < nb * 7; ++q)
            if (!(H->flags_h[(size_t)q] & 32)) all.push_back((int32_t)q);  // 32: identically zero kernel
        if ((rc = run_aca(all, std::min(r0 + look, kcap)))) return rc;
    } else {
        for (int64_t q = 0; q < nb * 7; ++q) {
            const Blk& bb = H->adm_h[(size_t)(q / 7)];
            uptr[(size_t)q] = H->U64.as<double>() + H->uoff_h[(size_t)q];
            vptr[(size_t)q] = H->V64.as<double>() + H->voff_h[(size_t)q];
            krank[(size_t)q] = H->rank_h[(size_t)q];
            (void)bb;
        }
    }
    if ((rc = upload_factors())) return rc;
    auto parts = [&](const std::vector<AmvmItem>& items) -> int {
        if (items.empty()) return HM_OK;
        int rc2 = put(d_items, items, s);
        if (rc2) return rc2;
        amvm_part_kernel<<<(unsigned)items.size(), kAmvmThreads, 0, s>>>(d_items, d_adm, d_krank, d_uptr, d_vptr, xc,
                                                                        c1, c2, d_doff, D);
        HM_CUDA(cudaGetLastError());
        return HM_OK;
    };

    // ---- b_0 = near field + every admissible block at rank r0
    amvm_gather_kernel<<<gMc, 256, 0, s>>>(H->d_perm.as<int32_t>(), x, xc, M);
    HM_CUDA(cudaGetLastError());
    amvm_near_kernel<<<gM, 256, 0, s>>>(d_ipos, d_nptr, d_nidx, H->d_near.as<Blk>(), H->d_noff.as<int64_t>(),
                                       H->N64.as<double>(), xc, c1, c2, bk, Mr);
    HM_CUDA(cudaGetLastError());
    std::vector<int32_t> r((size_t)nb, r0);
    std::vector<AmvmItem> items((size_t)nb);
    for (int64_t b = 0; b < nb; ++b) items[(size_t)b] = AmvmItem{(int32_t)b, 0, r0, 0};
    if ((rc = parts(items))) return rc;
    if (nb > 0) {
        amvm_rowsum_kernel<<<gM, 256, 0, s>>>(d_ipos, d_aptr, d_aidx, d_adm, d_doff, D, nullptr, 1, bk, Mr);
        HM_CUDA(cudaGetLastError());
    }
    // look-ahead parts at the current ranks
    for (int64_t b = 0; b < nb; ++b) items[(size_t)b] = AmvmItem{(int32_t)b, r0, r0 + look, 0};
    if ((rc = parts(items))) return rc;

    std::vector<double> he((size_t)N), hb((size_t)N);
    std::vector<uint8_t> marked((size_t)nb);
    int it = 0;
    int64_t marked_total = 0;
    double gamma = 0.0, bhat = 0.0;
    for (;;) {
        // e = b^_k - b_k
        if (nb > 0) {
            amvm_rowsum_kernel<<<gM, 256, 0, s>>>(d_ipos, d_aptr, d_aidx, d_adm, d_doff, D, nullptr, 0, e, Mr);
            HM_CUDA(cudaGetLastError());
        } else {
            HM_CUDA(cudaMemsetAsync(e, 0, (size_t)N * sizeof(double), s));
        }
        HM_CUDA(cudaMemcpyAsync(he.data(), e, (size_t)N * sizeof(double), cudaMemcpyDeviceToHost, s));
        HM_CUDA(cudaMemcpyAsync(hb.data(), bk, (size_t)N * sizeof(double), cudaMemcpyDeviceToHost, s));
        HM_CUDA(cudaStreamSynchronize(s));
        double g2 = 0.0, b2 = 0.0;
        for (int64_t i = 0; i < N; ++i) {
            g2 += he[(size_t)i] * he[(size_t)i];
            const double v = hb[(size_t)i] + he[(size_t)i];
            b2 += v * v;
        }
        gamma = std::sqrt(g2);
        bhat = std::sqrt(b2);
        if (it < hist_cap && gamma_hist) gamma_hist[it] = gamma;
        if (gamma <= eps * bhat || it >= max_iter) break;
        // step 3: Doerfler marking through the rows in decreasing error, on the
        // device: first[b] = the earliest sorted row at which block b joins P_k;
        // the marked set after row j is {b : first[b] <= j}, and the stopping row
        // is found by bisection on ||rest(j)|| <= (1 - theta) gamma_k (the first
        // such row when ||rest|| decreases along the scan, as it does when parts
        // remove error; otherwise a row where the condition holds)
        // (c_sp M N)^{-1/2} of step 3 with the paper's M x N = 3 Mr x 3M
        const double thr = (1.0 - theta) * gamma / std::sqrt((double)csp * (double)N * (double)Ncol);
        const unsigned gP = (unsigned)((P + 255) / 256), gB = (unsigned)((nb + 255) / 256);
        amvm_sort_init_kernel<<<gP, 256, 0, s>>>(e, N, P, d_key, d_sidx);
        HM_CUDA(cudaGetLastError());
        for (int64_t kk2 = 2; kk2 <= P; kk2 <<= 1)
            for (int64_t jj = kk2 >> 1; jj > 0; jj >>= 1) {
                amvm_bitonic_kernel<<<gP, 256, 0, s>>>(d_key, d_sidx, P, jj, kk2);
                HM_CUDA(cudaGetLastError());
            }
        amvm_rowpos_kernel<<<(unsigned)((N + 255) / 256), 256, 0, s>>>(d_sidx, N, d_rowpos);
        HM_CUDA(cudaGetLastError());
        amvm_first_kernel<<<(unsigned)nb, 256, 0, s>>>(d_adm, d_doff, D, d_rowpos, thr, d_first);
        HM_CUDA(cudaGetLastError());
        const int64_t npart = (Mr + 255) / 256;
        auto rest2 = [&](int32_t j, double& out) -> int {
            amvm_cut_kernel<<<gB, 256, 0, s>>>(d_first, nb, j, d_flags);
            HM_CUDA(cudaGetLastError());
            amvm_rest_kernel<<<(unsigned)npart, 256, 0, s>>>(d_ipos, d_aptr, d_aidx, d_adm, d_doff, D, d_flags, e,
                                                            Mr, d_part);
            HM_CUDA(cudaGetLastError());
            amvm_sum_kernel<<<1, 256, 0, s>>>(d_part, npart, d_norm);
            HM_CUDA(cudaGetLastError());
            HM_CUDA(cudaMemcpyAsync(&out, d_norm, sizeof(double), cudaMemcpyDeviceToHost, s));
            HM_CUDA(cudaStreamSynchronize(s));
            return HM_OK;
        };
        const double target2 = (1.0 - theta) * gamma * (1.0 - theta) * gamma;
        int32_t lo = 0, hi = (int32_t)(N - 1);
        double f_hi = 0.0;
        if ((rc = rest2(hi, f_hi))) return rc;
        if (f_hi <= target2) {
            while (lo < hi) {
                const int32_t mid = lo + (hi - lo) / 2;
                double f_mid = 0.0;
                if ((rc = rest2(mid, f_mid))) return rc;
                if (f_mid <= target2) {
                    hi = mid;
                    f_hi = f_mid;
                } else {
                    lo = mid + 1;
                }
            }
            if ((rc = rest2(hi, f_hi))) return rc;  // the flags of the cut
        }
        double g_rest = std::sqrt(std::max(f_hi, 0.0));
        HM_CUDA(cudaMemcpyAsync(marked.data(), d_flags, (size_t)nb, cudaMemcpyDeviceToHost, s));
        HM_CUDA(cudaStreamSynchronize(s));
        std::vector<int32_t> newly;
        for (int64_t b = 0; b < nb; ++b)
            if (marked[(size_t)b]) newly.push_back((int32_t)b);
        if (it < hist_cap && gamma_rest_hist) gamma_rest_hist[it] = g_rest;
        if (newly.empty()) break;
        marked_total += (int64_t)newly.size();
        // step 4: A_{k+1} = A^_k on the marked blocks (d_flags), and their next look-ahead
        amvm_rowsum_kernel<<<gM, 256, 0, s>>>(d_ipos, d_aptr, d_aidx, d_adm, d_doff, D, d_flags, 1, bk, Mr);
        HM_CUDA(cudaGetLastError());
        items.clear();
        std::map<int, std::vector<int32_t>> rerun;  // on demand: tasks to extend, by their new kmax
        for (int32_t b : newly) {
            r[(size_t)b] += look;
            items.push_back(AmvmItem{b, r[(size_t)b], r[(size_t)b] + look, 0});
            if (lazy)
                for (int k = 0; k < 7; ++k) {
                    const size_t q = (size_t)b * 7 + (size_t)k;
                    const int want = std::min(r[(size_t)b] + look, kcap);
                    // only a run that stopped at its kmax has more crosses to give
                    // (an identically zero kernel never ran: flag 32)
                    if (!(H->flags_h[q] & 32) && (kflags[q] & 1) && want > krank[q])
                        rerun[want].push_back((int32_t)q);
                }
        }
        if (!rerun.empty()) {
            std::fill(prev.begin(), prev.end(), nullptr);
            for (auto& kv : rerun)
                for (int32_t q : kv.second) prev[(size_t)q] = uptr[(size_t)q];
            for (auto& kv : rerun)
                if ((rc = run_aca(kv.second, kv.first))) return rc;
            if ((rc = upload_factors())) return rc;
        }
        if ((rc = parts(items))) return rc;
        ++it;
    }
    amvm_scatter_kernel<<<gM, 256, 0, s>>>(H->row_perm(), bk, y, Mr);
    HM_CUDA(cudaGetLastError());
    HM_CUDA(cudaStreamSynchronize(s));
    if (info) {
        info->iterations = it;
        info->csp = csp;
        info->gamma = gamma;
        info->bhat_norm = bhat;
        int64_t used = 0, full = 0;
        for (int64_t b = 0; b < nb; ++b)
            for (int k = 0; k < 7; ++k) {
                const int32_t K = lazy ? krank[(size_t)(b * 7 + k)] : H->rank_h[(size_t)(b * 7 + k)];
                used += std::min<int64_t>(K, r[(size_t)b]);
                full += K;
            }
        info->crosses_used = used;
        info->crosses_full = full;
        info->marked_total = marked_total;
    }
    if (block_ranks)
        for (int64_t b = 0; b < nb; ++b) block_ranks[b] = r[(size_t)b];
    return HM_OK;
}
