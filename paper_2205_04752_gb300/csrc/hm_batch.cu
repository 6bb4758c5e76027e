// hm_batch.cu -- one H-matrix-vector product over many resident matrices.
//
// Every member keeps its own factor streams and tables; the batch only adds
// a plan over all of them (a mesh table, the forward-pass records of all
// admissible blocks tagged with their mesh, one (mesh, leaf) work list) and
// a workspace sized for the concatenated vectors.  A product is then the same
// three phases as for one matrix, each one launch over every block of every
// member: gather, forward pass (one kernel for the large blocks of all
// members, one for the small blocks), and the persistent streamed leaf kernel
// that takes (mesh, leaf) items from one counter.
//
// The schedule knobs (CTAs per SM of the leaf kernel, order of the work list,
// forward kernels on one or two streams) change only when and where work
// runs, never the order of any sum, so every member's part of a batched
// product is bitwise equal to that member's own hm_matvec.
#include <algorithm>
#include <cstring>
#include <numeric>
#include <vector>

#include "hm_internal.h"

struct hm_batch {
    std::vector<const hm_matrix*> mats;
    int32_t form = 0, max_rhs = 0;
    int64_t npos = 0, w_total = 0, ngroups = 0, nunits = 0, nmulti = 0, zcols = 0, nwork = 0, nbig = 0, nsmall = 0;
    int32_t max_leaf = 0;
    int ctas_max = 1;  // CTAs per SM of the streamed kernel that fit
    std::vector<int64_t> pos_prefix;  // nmat + 1 cluster positions
    std::vector<hm::MeshDev> mesh_h;
    hm::Allocator alloc;
    hm::DevBuf d_mesh, d_pos_prefix, d_fwd, d_groups, d_units, d_tcunits, d_multi, d_big, d_small, d_work[2], xg, w, z, counters,
        err;
    hm_schedule sched{};
    cudaStream_t side = nullptr, cap = nullptr;
    cudaEvent_t fork = nullptr, join = nullptr;
    // cached graph of one product
    cudaGraphExec_t gexec = nullptr;
    const double* gx = nullptr;
    double* gy = nullptr;
    int32_t gnrhs = 0;
    int64_t gld = 0;
    hm_schedule gsched{};
};

namespace {

using namespace hm;

int balloc(hm_batch& B, DevBuf& d, size_t bytes)
{
    d.bytes = std::max<size_t>(bytes, 256);
    d.p = B.alloc.alloc(d.bytes);
    if (!d.p) return fail(HM_ENOMEM, "hm_batch: device allocation of %zu bytes failed", d.bytes);
    return HM_OK;
}

int bupload(hm_batch& B, DevBuf& d, const void* src, size_t bytes)
{
    int rc = balloc(B, d, bytes);
    if (rc) return rc;
    if (bytes) HM_CUDA(cudaMemcpy(d.p, src, bytes, cudaMemcpyHostToDevice));
    return HM_OK;
}

void batch_free(hm_batch* B)
{
    if (!B) return;
    if (B->gexec) cudaGraphExecDestroy(B->gexec);
    for (DevBuf* b : {&B->d_mesh, &B->d_pos_prefix, &B->d_fwd, &B->d_groups, &B->d_units, &B->d_tcunits, &B->d_multi, &B->d_big,
                      &B->d_small, &B->d_work[0],
                      &B->d_work[1], &B->xg, &B->w, &B->z,
                      &B->counters, &B->err})
        if (b->p) B->alloc.release(b->p, b->bytes);
    if (B->side) cudaStreamDestroy(B->side);
    if (B->cap) cudaStreamDestroy(B->cap);
    if (B->fork) cudaEventDestroy(B->fork);
    if (B->join) cudaEventDestroy(B->join);
    delete B;
}

Plan make_plan(const hm_batch& B)
{
    Plan P{};
    P.meshes = B.d_mesh.as<MeshDev>();
    if (B.mesh_h.size() == 1) P.mesh0 = B.mesh_h[0];
    P.nmesh = (int32_t)B.mesh_h.size();
    P.pos_prefix = B.d_pos_prefix.as<int64_t>();
    P.npos = B.npos;
    P.fwd = B.d_fwd.as<FwdRec>();
    P.groups = B.d_groups.as<FwdGroup>();
    P.units = B.d_units.as<FwdUnit>();
    P.tcu = B.d_tcunits.as<FwdTcUnit>();
    P.nunits = B.nunits;
    P.multi = B.d_multi.as<FwdMulti>();
    P.nmulti = B.nmulti;
    P.zcols = B.zcols;
    P.z = B.z.p;
    P.big = B.d_big.as<int32_t>();
    P.nbig = B.nbig;
    P.small = B.d_small.as<int32_t>();
    P.nsmall = B.nsmall;
    P.work = B.d_work[B.sched.work_order ? 1 : 0].as<int2>();
    P.nwork = B.nwork;
    P.max_leaf = B.max_leaf;
    P.counters = B.counters.as<int>();
    P.err = B.err.as<int>();
    return P;
}

Sched make_sched(const hm_batch& B)
{
    Sched sc;
    sc.ctas_per_sm = B.sched.leaf_ctas_per_sm;
    if (B.sched.fork_forward) {
        sc.side = B.side;
        sc.fork = B.fork;
        sc.join = B.join;
    }
    return sc;
}

int run(hm_batch& B, const double* x, double* y, int32_t nrhs, int64_t ld, cudaStream_t s)
{
    const Plan P = make_plan(B);
    const Sched sc = make_sched(B);
    return run_product(P, B.form, x, y, nrhs, ld, B.xg.p, B.w.p, s, nullptr, &sc);
}

bool same_sched(const hm_schedule& a, const hm_schedule& b)
{
    return a.leaf_ctas_per_sm == b.leaf_ctas_per_sm && a.work_order == b.work_order &&
           a.fork_forward == b.fork_forward;
}

int check_sched(const hm_batch& B, const hm_schedule* s)
{
    if (!s) return fail(HM_EINVAL, "hm_batch: NULL schedule");
    if (s->leaf_ctas_per_sm < 0 || s->leaf_ctas_per_sm > 32)
        return fail(HM_EINVAL, "hm_batch: leaf_ctas_per_sm=%d outside 0..32", s->leaf_ctas_per_sm);
    if (s->work_order != 0 && s->work_order != 1)
        return fail(HM_EINVAL, "hm_batch: work_order must be 0 or 1");
    if (s->fork_forward != 0 && s->fork_forward != 1)
        return fail(HM_EINVAL, "hm_batch: fork_forward must be 0 or 1");
    (void)B;
    return HM_OK;
}

}  // namespace

extern "C" {

int hm_batch_create(const hm_matrix* const* mats, int32_t nmat, int32_t form, int32_t max_rhs, hm_batch** out)
{
    if (!out) return fail(HM_EINVAL, "hm_batch_create: NULL out");
    *out = nullptr;
    if (!mats || nmat < 1) return fail(HM_EINVAL, "hm_batch_create: need at least one matrix");
    if (nmat > 65535) return fail(HM_EINVAL, "hm_batch_create: at most 65535 matrices");
    if (form < HM_FP64 || form >= HM_NFORMS) return fail(HM_EINVAL, "hm_batch_create: unknown form %d", form);
    if (max_rhs < 1) return fail(HM_EINVAL, "hm_batch_create: max_rhs must be >= 1");
    for (int32_t m = 0; m < nmat; ++m) {
        if (!mats[m]) return fail(HM_EINVAL, "hm_batch_create: matrix %d is NULL", m);
        if (mats[m]->rect) return fail(HM_EINVAL, "hm_batch_create: matrix %d: an evaluation operator (hm_build_point_tree) has only hm_eval_points and hm_amvm", m);
        if (!mats[m]->packed[form])
            return fail(HM_EINVAL, "hm_batch_create: matrix %d has form %d not packed (call hm_pack)", m, form);
        for (int32_t q = 0; q < m; ++q)
            if (mats[q] == mats[m]) return fail(HM_EINVAL, "hm_batch_create: matrix %d listed twice", m);
    }
    hm_batch* B = new (std::nothrow) hm_batch;
    if (!B) return fail(HM_ENOMEM, "hm_batch_create: out of host memory");
    B->mats.assign(mats, mats + nmat);
    B->form = form;
    B->max_rhs = max_rhs;
    B->alloc = mats[0]->alloc;
    B->alloc.stream = nullptr;
    int rc = product_prepare(form, &B->ctas_max);
    if (rc) {
        batch_free(B);
        return rc;
    }

    // offsets of every member in the concatenated vectors
    B->pos_prefix.assign((size_t)nmat + 1, 0);
    std::vector<int64_t> woff((size_t)nmat + 1, 0);
    for (int32_t m = 0; m < nmat; ++m) {
        B->pos_prefix[(size_t)m + 1] = B->pos_prefix[(size_t)m] + mats[m]->M;
        woff[(size_t)m + 1] = woff[(size_t)m] + mats[m]->w_total;
        B->max_leaf = std::max(B->max_leaf, mats[m]->max_leaf);
    }
    B->npos = B->pos_prefix.back();
    B->w_total = woff.back();
    for (int32_t m = 0; m < nmat; ++m) {
        MeshDev d = mesh_desc(*mats[m], form);
        d.xoff = 3 * B->pos_prefix[(size_t)m];
        d.xgoff = B->pos_prefix[(size_t)m];
        d.woff = woff[(size_t)m] / 4;  // in factor columns
        B->mesh_h.push_back(d);
    }

    // forward groups, units and tall groups of every member (indices shifted
    // into the concatenated lists; a block's group and its arithmetic are its
    // own matrix's), the units with the most data first across members
    std::vector<FwdRec> fwd;
    std::vector<FwdGroup> groups;
    std::vector<FwdUnit> units;
    std::vector<FwdMulti> multi;
    std::vector<int32_t> bigv, smallv;
    int64_t zc = 0;
    for (int32_t m = 0; m < nmat; ++m) {
        const hm_matrix& H = *mats[m];
        const int32_t rbase = (int32_t)fwd.size(), gbase = (int32_t)groups.size();
        for (FwdRec r : H.fwd_h) {
            r.mesh = (uint16_t)m;
            r.grp += gbase;
            fwd.push_back(r);
        }
        for (int32_t q : H.big_h) bigv.push_back(q + rbase);
        for (int32_t q : H.small_h) smallv.push_back(q + rbase);
        for (FwdGroup g : H.grp_h) {
            g.first += rbase;
            g.mesh = (uint16_t)m;
            groups.push_back(g);
        }
        for (FwdUnit u : H.unit_h) {
            u.group += gbase;
            if (u.zcol0 >= 0) u.zcol0 += zc;
            units.push_back(u);
        }
        for (FwdMulti mu : H.multi_h) {
            mu.group += gbase;
            mu.zcol0 += zc;
            multi.push_back(mu);
        }
        zc += H.zcols;
    }
    std::stable_sort(units.begin(), units.end(), [&](const FwdUnit& a, const FwdUnit& b) {
        return (int64_t)a.nrows * groups[(size_t)a.group].Cs > (int64_t)b.nrows * groups[(size_t)b.group].Cs;
    });
    auto by_work = [&](int32_t a, int32_t b) {
        return (int64_t)fwd[(size_t)a].n * fwd[(size_t)a].C > (int64_t)fwd[(size_t)b].n * fwd[(size_t)b].C;
    };
    std::stable_sort(bigv.begin(), bigv.end(), by_work);
    std::stable_sort(smallv.begin(), smallv.end(), by_work);
    B->nbig = (int64_t)bigv.size();
    B->nsmall = (int64_t)smallv.size();
    B->ngroups = (int64_t)groups.size();
    B->nunits = (int64_t)units.size();
    const std::vector<FwdTcUnit> tcu = tc_units(units, groups);
    B->nmulti = (int64_t)multi.size();
    B->zcols = zc;

    // work lists: 0 = every (mesh, leaf) by decreasing streamed elements (a
    // longest-processing-time order over the whole batch); 1 = member by
    // member, each in its own order
    std::vector<int2> w1;
    std::vector<std::pair<int64_t, int2>> all;
    for (int32_t m = 0; m < nmat; ++m) {
        const hm_matrix& H = *mats[m];
        for (int32_t lf : H.leaf_order_h) {
            w1.push_back(make_int2(m, lf));
            all.push_back({H.leaf_bytes_h[(size_t)lf], make_int2(m, lf)});
        }
    }
    std::stable_sort(all.begin(), all.end(),
                     [](const std::pair<int64_t, int2>& a, const std::pair<int64_t, int2>& b) {
                         return a.first > b.first;
                     });
    std::vector<int2> w0(all.size());
    for (size_t q = 0; q < all.size(); ++q) w0[q] = all[q].second;
    B->nwork = (int64_t)w0.size();
    if (B->nwork > INT32_MAX) {
        batch_free(B);
        return fail(HM_EINVAL, "hm_batch_create: more than 2^31 leaves");
    }

    const size_t ta = form == HM_FP64 ? 8 : 4;
    if ((rc = bupload(*B, B->d_mesh, B->mesh_h.data(), B->mesh_h.size() * sizeof(MeshDev))) ||
        (rc = bupload(*B, B->d_pos_prefix, B->pos_prefix.data(), B->pos_prefix.size() * 8)) ||
        (rc = bupload(*B, B->d_fwd, fwd.data(), fwd.size() * sizeof(FwdRec))) ||
        (rc = bupload(*B, B->d_groups, groups.data(), groups.size() * sizeof(FwdGroup))) ||
        (rc = bupload(*B, B->d_units, units.data(), units.size() * sizeof(FwdUnit))) ||
        (rc = bupload(*B, B->d_tcunits, tcu.data(), tcu.size() * sizeof(FwdTcUnit))) ||
        (rc = bupload(*B, B->d_multi, multi.data(), multi.size() * sizeof(FwdMulti))) ||
        (rc = bupload(*B, B->d_big, bigv.data(), bigv.size() * 4)) ||
        (rc = bupload(*B, B->d_small, smallv.data(), smallv.size() * 4)) ||
        (rc = balloc(*B, B->z, (size_t)max_rhs * (size_t)std::max<int64_t>(B->zcols, 1) * 4 * ta)) ||
        (rc = bupload(*B, B->d_work[0], w0.data(), w0.size() * sizeof(int2))) ||
        (rc = bupload(*B, B->d_work[1], w1.data(), w1.size() * sizeof(int2))) ||
        (rc = balloc(*B, B->xg, (size_t)max_rhs * 4 * (size_t)B->npos * ta)) ||
        (rc = balloc(*B, B->w, (size_t)max_rhs * (size_t)std::max<int64_t>(B->w_total, 1) * ta)) ||
        (rc = balloc(*B, B->counters, (size_t)kCounterInts * sizeof(int))) || (rc = balloc(*B, B->err, 64))) {
        batch_free(B);
        return rc;
    }
    cudaError_t e = cudaMemset(B->err.p, 0, 64);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&B->side, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&B->cap, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&B->fork, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&B->join, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaDeviceSynchronize();
    if (e != cudaSuccess) {
        rc = cuda_check(e, "hm_batch_create");
        batch_free(B);
        return rc;
    }
    *out = B;
    return HM_OK;
}

int hm_batch_layout(const hm_batch* B, int64_t* dof_offsets, int64_t* sizes)
{
    if (!B) return fail(HM_EINVAL, "hm_batch_layout: NULL batch");
    if (dof_offsets)
        for (size_t m = 0; m < B->pos_prefix.size(); ++m) dof_offsets[m] = 3 * B->pos_prefix[m];
    if (sizes) {
        sizes[0] = (int64_t)B->mats.size();
        sizes[1] = 3 * B->npos;
        sizes[2] = B->ngroups;
        sizes[3] = B->nwork;
    }
    return HM_OK;
}

int hm_batch_set_schedule(hm_batch* B, const hm_schedule* s)
{
    if (!B) return fail(HM_EINVAL, "hm_batch_set_schedule: NULL batch");
    int rc = check_sched(*B, s);
    if (rc) return rc;
    B->sched = *s;
    return HM_OK;
}

int hm_batch_get_schedule(const hm_batch* B, hm_schedule* s)
{
    if (!B || !s) return fail(HM_EINVAL, "hm_batch_get_schedule: NULL argument");
    *s = B->sched;
    return HM_OK;
}

int hm_batch_matvec(hm_batch* B, const double* x, double* y, int32_t nrhs, int64_t ld, int32_t use_graph,
                    void* stream)
{
    if (!B || !x || !y) return fail(HM_EINVAL, "hm_batch_matvec: NULL argument");
    if (nrhs < 1 || nrhs > B->max_rhs)
        return fail(HM_EINVAL, "hm_batch_matvec: nrhs=%d outside 1..%d", nrhs, B->max_rhs);
    const int64_t n = 3 * B->npos;
    if (ld < n) return fail(HM_EINVAL, "hm_batch_matvec: ld=%lld < %lld", (long long)ld, (long long)n);
    const char* xb = (const char*)x;
    const char* yb = (const char*)y;
    const size_t span = ((size_t)(nrhs - 1) * ld + (size_t)n) * sizeof(double);
    if (xb < yb + span && yb < xb + span) return fail(HM_EINVAL, "hm_batch_matvec: x and y overlap");
    cudaStream_t s = (cudaStream_t)stream;
    if (!use_graph) return run(*B, x, y, nrhs, ld, s);
    if (!B->gexec || B->gx != x || B->gy != y || B->gnrhs != nrhs || B->gld != ld ||
        !same_sched(B->gsched, B->sched)) {
        if (B->gexec) {
            HM_CUDA(cudaStreamSynchronize(s));
            HM_CUDA(cudaGraphExecDestroy(B->gexec));
            B->gexec = nullptr;
        }
        HM_CUDA(cudaStreamBeginCapture(B->cap, cudaStreamCaptureModeThreadLocal));
        const int rc = run(*B, x, y, nrhs, ld, B->cap);
        cudaGraph_t g = nullptr;
        const cudaError_t e = cudaStreamEndCapture(B->cap, &g);
        if (rc) {
            if (g) cudaGraphDestroy(g);
            return rc;
        }
        HM_CUDA(e);
        const cudaError_t ei = cudaGraphInstantiate(&B->gexec, g, 0);
        cudaGraphDestroy(g);
        HM_CUDA(ei);
        B->gx = x;
        B->gy = y;
        B->gnrhs = nrhs;
        B->gld = ld;
        B->gsched = B->sched;
    }
    HM_CUDA(cudaGraphLaunch(B->gexec, s));
    return HM_OK;
}

int hm_batch_autotune(hm_batch* B, int32_t nrhs, int32_t reps, hm_schedule* chosen, double* ms_best, void* stream)
{
    if (!B) return fail(HM_EINVAL, "hm_batch_autotune: NULL batch");
    if (nrhs < 1 || nrhs > B->max_rhs)
        return fail(HM_EINVAL, "hm_batch_autotune: nrhs=%d outside 1..%d", nrhs, B->max_rhs);
    if (reps < 1) reps = 3;
    cudaStream_t s = (cudaStream_t)stream;
    const int64_t n = 3 * B->npos;
    const size_t bytes = (size_t)nrhs * (size_t)n * sizeof(double);
    Allocator al = B->alloc;
    al.stream = s;
    void* x = al.alloc(bytes);
    void* y = al.alloc(bytes);
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    int rc = HM_OK;
    const hm_schedule saved = B->sched;
    hm_schedule best = saved;
    double tbest = -1.0;
    if (!x || !y) rc = fail(HM_ENOMEM, "hm_batch_autotune: could not allocate %zu bytes", 2 * bytes);
    if (!rc) rc = cuda_check(cudaEventCreate(&e0), "hm_batch_autotune");
    if (!rc) rc = cuda_check(cudaEventCreate(&e1), "hm_batch_autotune");
    // the values do not change the work: every product does the same loads
    // and operations whatever x holds
    if (!rc) rc = cuda_check(cudaMemsetAsync(x, 0, bytes, s), "hm_batch_autotune");
    std::vector<hm_schedule> cand;
    for (int ctas : {0, 1}) {
        if (ctas == 1 && B->ctas_max <= 1) continue;
        for (int order = 0; order < 2; ++order)
            for (int fork = 0; fork < 2; ++fork) {
                hm_schedule c{};
                c.leaf_ctas_per_sm = ctas;
                c.work_order = order;
                c.fork_forward = fork;
                cand.push_back(c);
            }
    }
    for (size_t i = 0; i < cand.size() && !rc; ++i) {
        B->sched = cand[i];
        if ((rc = run(*B, (const double*)x, (double*)y, nrhs, n, s))) break;  // warm-up
        if ((rc = cuda_check(cudaEventRecord(e0, s), "hm_batch_autotune"))) break;
        for (int r = 0; r < reps && !rc; ++r) rc = run(*B, (const double*)x, (double*)y, nrhs, n, s);
        if (rc) break;
        if ((rc = cuda_check(cudaEventRecord(e1, s), "hm_batch_autotune"))) break;
        if ((rc = cuda_check(cudaEventSynchronize(e1), "hm_batch_autotune"))) break;
        float ms = 0.f;
        if ((rc = cuda_check(cudaEventElapsedTime(&ms, e0, e1), "hm_batch_autotune"))) break;
        const double t = (double)ms / reps;
        if (tbest < 0.0 || t < tbest) {
            tbest = t;
            best = cand[i];
        }
    }
    B->sched = rc ? saved : best;
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (x) al.release(x, bytes);
    if (y) al.release(y, bytes);
    if (!rc) rc = cuda_check(cudaStreamSynchronize(s), "hm_batch_autotune");
    if (rc) return rc;
    if (chosen) *chosen = best;
    if (ms_best) *ms_best = tbest;
    return HM_OK;
}

int hm_batch_check(const hm_batch* B)
{
    if (!B) return fail(HM_EINVAL, "hm_batch_check: NULL batch");
    int e[4] = {0, 0, 0, 0};
    HM_CUDA(cudaMemcpy(e, B->err.p, sizeof e, cudaMemcpyDeviceToHost));
    if (e[0]) {
        const int zero[4] = {0, 0, 0, 0};
        HM_CUDA(cudaMemcpy(B->err.p, zero, sizeof zero, cudaMemcpyHostToDevice));
        return fail(HM_ETIMEOUT,
                    "hm_batch_check: a bounded device wait ran out in an earlier product (site %d, stage %d, CTA %d)",
                    e[1], e[2], e[3]);
    }
    return HM_OK;
}

void hm_batch_destroy(hm_batch* B)
{
    if (!B) return;
    cudaDeviceSynchronize();
    batch_free(B);
}

}  // extern "C"
