// hm_eval.cu -- the evaluation operator ~V_h of Section 5, Eq. (vector_eq)
// (the displacement at points of the domain): the tables of its product, its
// FP32 form and hm_eval_points.  The product's kernels (ev_*) are in
// hm_parts.cuh.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <map>
#include <numeric>
#include <vector>

#include "hm_parts.cuh"

namespace hm {

int eval_prepare(hm_matrix& H)
{
    const int64_t M = H.M, Mr = H.Mr, nb = H.nadm, nn = H.nnear;
    std::vector<int64_t> bounds = {0, Mr};
    for (const auto* L : {&H.adm_h, &H.near_h})
        for (const Blk& b : *L) {
            bounds.push_back(b.t0);
            bounds.push_back(b.t0 + b.m);
        }
    std::sort(bounds.begin(), bounds.end());
    bounds.erase(std::unique(bounds.begin(), bounds.end()), bounds.end());
    const RowLists ra = row_lists(Mr, bounds, H.adm_h), rn = row_lists(Mr, bounds, H.near_h);
    // parts: 3 values per row of every admissible block (doff) and of every
    // near block (ndoff); work items (block, 32-row chunk)
    std::vector<int64_t> doff((size_t)nb + 1, 0), ndoff((size_t)nn + 1, 0);
    std::vector<int2> back, nearit;
    for (int64_t b = 0; b < nb; ++b) {
        const Blk& bk = H.adm_h[(size_t)b];
        doff[(size_t)b + 1] = doff[(size_t)b] + 3 * (int64_t)bk.m;
        for (int c = 0; 32 * c < bk.m; ++c) back.push_back(int2{(int)b, c});
    }
    for (int64_t b = 0; b < nn; ++b) {
        const Blk& bk = H.near_h[(size_t)b];
        ndoff[(size_t)b + 1] = ndoff[(size_t)b] + 3 * (int64_t)bk.m;
        for (int c = 0; 32 * c < bk.m; ++c) nearit.push_back(int2{(int)b, c});
    }
    int dev = 0, nsm = 0;
    HM_CUDA(cudaGetDevice(&dev));
    HM_CUDA(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
    H.ev_parts = doff[(size_t)nb];
    H.ev_nback = (int64_t)back.size();
    H.ev_nnear = (int64_t)nearit.size();
    H.ev_grid = std::max(1, nsm) * 8;  // 8 CTAs of 256 threads per SM
    int rc;
    const std::vector<double> none;
    if ((rc = ev_put(H, kEvIpos, ra.ipos, ra.ipos.size())) || (rc = ev_put(H, kEvAptr, ra.ptr, ra.ptr.size())) ||
        (rc = ev_put(H, kEvAidx, ra.idx, ra.idx.size())) || (rc = ev_put(H, kEvNptr, rn.ptr, rn.ptr.size())) ||
        (rc = ev_put(H, kEvNidx, rn.idx, rn.idx.size())) || (rc = ev_put(H, kEvDoff, doff, doff.size())) ||
        (rc = ev_put(H, kEvBack, back, back.size())) || (rc = ev_put(H, kEvNear, nearit, nearit.size())) ||
        (rc = ev_put(H, kEvNdoff, ndoff, ndoff.size())) ||
        (rc = ev_put(H, kEvW, none, (size_t)(3 * std::max<int64_t>(H.c_total, 1)))) ||
        (rc = ev_put(H, kEvXc, none, (size_t)(3 * M))) || (rc = ev_put(H, kEvYc, none, (size_t)(3 * Mr))) ||
        (rc = ev_put(H, kEvD, none, (size_t)doff[(size_t)nb])) || (rc = ev_put(H, kEvDn, none, (size_t)ndoff[(size_t)nn]))) {
        // all or nothing: a later call must not find half of the tables
        for (DevBuf& b : H.ev) {
            H.alloc.release(b.p, b.bytes);
            b = DevBuf{};
        }
        return rc;
    }
    return HM_OK;
}
int eval_pack_fp32(hm_matrix& H, cudaStream_t s)
{
    // FP32 copies of the block-ordered arenas, same offsets: factors U, V and
    // the near field (the FP32 form of the evaluation operator)
    struct Pair {
        const DevBuf* src;
        DevBuf* dst;
        int64_t n;
    } pairs[3] = {{&H.U64, &H.Ul[HM_FP32], H.u_total}, {&H.V64, &H.Vr[HM_FP32], H.v_total},
                  {&H.N64, &H.Nl32, H.n_total}};
    for (Pair& pr : pairs) {
        pr.dst->bytes = (size_t)std::max<int64_t>(pr.n, 1) * sizeof(float);
        pr.dst->p = H.alloc.alloc(pr.dst->bytes);
        if (!pr.dst->p) return fail(HM_ENOMEM, "hm_pack: FP32 evaluation arenas (%zu bytes)", pr.dst->bytes);
        if (pr.n > 0) {
            ev_to_fp32_kernel<<<(unsigned)std::min<int64_t>((pr.n + 255) / 256, 4096), 256, 0, s>>>(
                pr.src->as<double>(), pr.dst->as<float>(), pr.n);
            HM_CUDA(cudaGetLastError());
        }
    }
    return HM_OK;
}

namespace {
template <class T>
int eval_run(const hm_matrix& H, const double* t, double* u, int32_t nrhs, const T* Uf, const T* Vf, const T* Nf,
             cudaStream_t s, bool accumulate = false)
{
    const int64_t M = H.M, Mr = H.Mr, nb = H.nadm;
    // the double layer's K_Delta is one scalar kernel in slot 0, applied to
    // each component: c1 = 1, c2 = 0
    const T c1 = H.dl ? (T)1 : (T)((1.0 + H.nu) * (3.0 - 4.0 * H.nu) / (2.0 * H.E * (1.0 - H.nu)));
    const T c2 = H.dl ? (T)0 : (T)((1.0 + H.nu) / (2.0 * H.E * (1.0 - H.nu)));
    const DevBuf* ev = H.ev;
    T* xc = ev[kEvXc].as<T>();
    T* yc = ev[kEvYc].as<T>();
    T* w = ev[kEvW].as<T>();
    T* D = ev[kEvD].as<T>();
    T* Dn = ev[kEvDn].as<T>();
    const unsigned gM = (unsigned)((Mr + 255) / 256), gMc = (unsigned)((M + 255) / 256);
    auto grid = [&](int64_t warps) {
        return (unsigned)std::max<int64_t>(1, std::min<int64_t>(H.ev_grid, (warps + kEvWarps - 1) / kEvWarps));
    };
    for (int32_t r = 0; r < nrhs; ++r) {
        ev_gather_kernel<T><<<gMc, 256, 0, s>>>(H.d_perm.as<int32_t>(), t + (int64_t)r * 3 * M, xc, M);
        HM_CUDA(cudaGetLastError());
        if (nb > 0) {
            ev_fwd_kernel<T><<<grid(nb * 7), kEvThreads, 0, s>>>(H.d_adm.as<Blk>(), H.d_rank.as<int32_t>(),
                                                                 H.d_voff.as<int64_t>(), H.d_coff.as<int64_t>(), Vf,
                                                                 nullptr, xc, M, nb * 7, w);
            HM_CUDA(cudaGetLastError());
            ev_back_kernel<T><<<grid(H.ev_nback), kEvThreads, 0, s>>>(
                ev[kEvBack].as<int2>(), H.ev_nback, H.d_adm.as<Blk>(), H.d_rank.as<int32_t>(), H.d_uoff.as<int64_t>(),
                H.d_coff.as<int64_t>(), Uf, nullptr, w, c1, c2, ev[kEvDoff].as<int64_t>(), D);
            HM_CUDA(cudaGetLastError());
        }
        if (H.ev_nnear > 0) {
            ev_near_kernel<T><<<grid(H.ev_nnear), kEvThreads, 0, s>>>(
                ev[kEvNear].as<int2>(), H.ev_nnear, H.d_near.as<Blk>(), H.d_noff.as<int64_t>(), Nf, xc, M, c1, c2,
                ev[kEvNdoff].as<int64_t>(), Dn);
            HM_CUDA(cudaGetLastError());
        }
        ev_rowsum_kernel<T><<<gM, 256, 0, s>>>(ev[kEvIpos].as<int32_t>(), ev[kEvAptr].as<int32_t>(),
                                              ev[kEvAidx].as<int32_t>(), H.d_adm.as<Blk>(), ev[kEvDoff].as<int64_t>(),
                                              D, ev[kEvNptr].as<int32_t>(), ev[kEvNidx].as<int32_t>(),
                                              H.d_near.as<Blk>(), ev[kEvNdoff].as<int64_t>(), Dn, yc, Mr);
        HM_CUDA(cudaGetLastError());
        if (accumulate)
            ev_scatter_add_kernel<T><<<gM, 256, 0, s>>>(H.d_rperm.as<int32_t>(), yc, u + (int64_t)r * 3 * Mr, Mr);
        else
            ev_scatter_kernel<T><<<gM, 256, 0, s>>>(H.d_rperm.as<int32_t>(), yc, u + (int64_t)r * 3 * Mr, Mr);
        HM_CUDA(cudaGetLastError());
    }
    return HM_OK;
}
}  // namespace

int eval_apply(const hm_matrix& H, const double* t, double* u, int32_t nrhs, int32_t form, bool accumulate,
               cudaStream_t s)
{
    if (form == HM_FP32)
        return eval_run<float>(H, t, u, nrhs, H.Ul[HM_FP32].as<float>(), H.Vr[HM_FP32].as<float>(),
                               H.Nl32.as<float>(), s, accumulate);
    return eval_run<double>(H, t, u, nrhs, H.U64.as<double>(), H.V64.as<double>(), H.N64.as<double>(), s,
                            accumulate);
}
}  // namespace hm

using namespace hm;

extern "C" int hm_eval_points(const hm_matrix* H, const double* t, double* u, int32_t nrhs, int32_t form,
                              void* stream)
{
    if (!H || !t || !u) return fail(HM_EINVAL, "hm_eval_points: NULL argument");
    if (!H->rect) return fail(HM_EINVAL, "hm_eval_points: not an evaluation operator (use hm_matvec)");
    if (H->aca_deferred)
        return fail(HM_EINVAL, "hm_eval_points: assembled with HM_DEFER_ACA (use hm_amvm with HM_AMVM_ACA_ON_DEMAND)");
    if (nrhs < 1) return fail(HM_EINVAL, "hm_eval_points: nrhs %d < 1", nrhs);
    if (!H->ev[kEvXc].p) return fail(HM_EINVAL, "hm_eval_points: the operator has no product tables");
    cudaStream_t s = (cudaStream_t)stream;
    if (form == HM_FP64)
        return eval_run<double>(*H, t, u, nrhs, H->U64.as<double>(), H->V64.as<double>(), H->N64.as<double>(), s);
    if (form == HM_FP32) {
        if (!H->packed[HM_FP32]) return fail(HM_EINVAL, "hm_eval_points: FP32 form not packed (hm_pack)");
        return eval_run<float>(*H, t, u, nrhs, H->Ul[HM_FP32].as<float>(), H->Vr[HM_FP32].as<float>(),
                               H->Nl32.as<float>(), s);
    }
    return fail(HM_EINVAL, "hm_eval_points: form %d (an evaluation operator has HM_FP64 and HM_FP32)", form);
}
