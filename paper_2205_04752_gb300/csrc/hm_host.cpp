// hm_host.cpp -- host side of the H-matrix library: error reporting, device
// allocation, cluster tree and block partition (Section 2.1), and the ABI
// entry points that need no kernel.
//
// Compiled with -ffp-contract=off: the geometric decisions (split axis,
// admissibility) are made with separately rounded operations so that they
// are reproducible on any host.
#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <new>

#include "hm_internal.h"

namespace hm {

static thread_local std::string g_err;

void set_error(const char* fmt, ...)
{
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    g_err = buf;
}

int fail(int code, const char* fmt, ...)
{
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    g_err = buf;
    return code;
}

int cuda_check(cudaError_t e, const char* what)
{
    if (e == cudaSuccess) return HM_OK;
    set_error("%s: %s", what, cudaGetErrorString(e));
    return e == cudaErrorMemoryAllocation ? HM_ENOMEM : HM_EDEVICE;
}

void* Allocator::alloc(size_t bytes)
{
    if (bytes == 0) bytes = 256;
    void* p = nullptr;
    if (has_user) {
        p = user.alloc(bytes, (void*)stream, user.user);
    } else if (cudaMallocAsync(&p, bytes, stream) != cudaSuccess) {
        cudaGetLastError();
        p = nullptr;
    }
    return p;
}

void Allocator::release(void* p, size_t bytes)
{
    if (!p) return;
    if (has_user)
        user.free(p, bytes, (void*)stream, user.user);
    else
        cudaFreeAsync(p, stream);
}

void prof_mark(const hm_matrix& H, int which, cudaStream_t s)
{
    if (!H.prof_on) return;
    if (which == 0 && H.prof_calls >= 4096) return;
    int64_t c = which == 0 ? H.prof_calls : H.prof_calls - 1;
    if (which == 0) {
        if ((size_t)(4 * (c + 1)) > H.prof_ev.size()) {
            for (int k = 0; k < 4; ++k) {
                cudaEvent_t e;
                if (cudaEventCreate(&e) != cudaSuccess) return;
                H.prof_ev.push_back(e);
            }
        }
        ++H.prof_calls;
    }
    if (c < 0 || (size_t)(4 * c + which) >= H.prof_ev.size()) return;
    cudaEventRecord(H.prof_ev[(size_t)(4 * c + which)], s);
}

// ---------------------------------------------------------------- tree
namespace {

struct TreeBuilder {
    hm_tree& tr;
    std::vector<std::pair<double, int64_t>> keys;

    int64_t build(int64_t lo, int64_t hi, int32_t level)
    {
        int64_t id = (int64_t)tr.nodes.size();
        tr.nodes.emplace_back();
        {
            Node& nd = tr.nodes.back();
            nd.lo = lo;
            nd.hi = hi;
            nd.level = level;
            nd.son[0] = nd.son[1] = -1;
            for (int k = 0; k < 3; ++k) {
                nd.bmin[k] = INFINITY;
                nd.bmax[k] = -INFINITY;
            }
            for (int64_t p = lo; p < hi; ++p) {
                if (tr.T.empty()) {
                    // a tree of points: the box of the points themselves; of
                    // vertices: the union of their stars
                    for (int k = 0; k < 3; ++k) {
                        const bool star = !tr.ibox.empty();
                        double lo = star ? tr.ibox[6 * tr.perm[p] + k] : tr.coll[3 * tr.perm[p] + k];
                        double hi = star ? tr.ibox[6 * tr.perm[p] + 3 + k] : tr.coll[3 * tr.perm[p] + k];
                        nd.bmin[k] = std::min(nd.bmin[k], lo);
                        nd.bmax[k] = std::max(nd.bmax[k], hi);
                    }
                    continue;
                }
                const int32_t* t = &tr.T[3 * tr.perm[p]];
                for (int c = 0; c < 3; ++c)
                    for (int k = 0; k < 3; ++k) {
                        double v = tr.V[3 * (int64_t)t[c] + k];
                        nd.bmin[k] = std::min(nd.bmin[k], v);
                        nd.bmax[k] = std::max(nd.bmax[k], v);
                    }
            }
        }
        if (level > tr.depth) tr.depth = level;
        if (hi - lo <= tr.leaf) return id;
        double cmin[3] = {INFINITY, INFINITY, INFINITY};
        double cmax[3] = {-INFINITY, -INFINITY, -INFINITY};
        for (int64_t p = lo; p < hi; ++p)
            for (int k = 0; k < 3; ++k) {
                double v = tr.coll[3 * tr.perm[p] + k];
                cmin[k] = std::min(cmin[k], v);
                cmax[k] = std::max(cmax[k], v);
            }
        // longest extent of the collocation-point box; lowest axis on ties
        int ax = 0;
        double ext = cmax[0] - cmin[0];
        for (int k = 1; k < 3; ++k) {
            double e = cmax[k] - cmin[k];
            if (e > ext) {
                ext = e;
                ax = k;
            }
        }
        keys.resize((size_t)(hi - lo));
        for (int64_t p = lo; p < hi; ++p)
            keys[(size_t)(p - lo)] = {tr.coll[3 * tr.perm[p] + ax], tr.perm[p]};
        std::sort(keys.begin(), keys.end());  // (coordinate, id): unique keys
        for (int64_t p = lo; p < hi; ++p) tr.perm[p] = keys[(size_t)(p - lo)].second;
        int64_t mid = lo + (hi - lo) / 2;
        int64_t s0 = build(lo, mid, level + 1);
        int64_t s1 = build(mid, hi, level + 1);
        tr.nodes[id].son[0] = s0;
        tr.nodes[id].son[1] = s1;
        return id;
    }
};

double box_diam2(const Node& a)
{
    double s = 0.0;
    for (int k = 0; k < 3; ++k) {
        double e = a.bmax[k] - a.bmin[k];
        s += e * e;
    }
    return s;
}

double box_dist2(const Node& a, const Node& b)
{
    double s = 0.0;
    for (int k = 0; k < 3; ++k) {
        double g = std::max(a.bmin[k] - b.bmax[k], b.bmin[k] - a.bmax[k]);
        if (g < 0.0) g = 0.0;
        s += g * g;
    }
    return s;
}

// block-cluster recursion (Section 2.1) with an explicit stack; the visiting
// order is the recursive pre-order (sons in order (0,0), (0,1), (1,0), (1,1));
// rows come from `rows` (the tree itself, or a tree of points) and columns
// from `cols`
void build_partition(hm_tree& tr, const std::vector<Node>& rows, const std::vector<Node>& cols)
{
    const double eta2 = tr.eta * tr.eta;
    std::vector<std::array<int64_t, 2>> st;
    st.push_back({0, 0});
    while (!st.empty()) {
        auto [t, s] = st.back();
        st.pop_back();
        const Node& a = rows[(size_t)t];
        const Node& b = cols[(size_t)s];
        double dmin = std::min(box_diam2(a), box_diam2(b));
        if (dmin < eta2 * box_dist2(a, b)) {
            tr.adm.push_back({t, s});
            continue;
        }
        bool tl = a.son[0] < 0, sl = b.son[0] < 0;
        if (!tl && !sl) {
            st.push_back({a.son[1], b.son[1]});
            st.push_back({a.son[1], b.son[0]});
            st.push_back({a.son[0], b.son[1]});
            st.push_back({a.son[0], b.son[0]});
        } else if (!tl) {
            st.push_back({a.son[1], s});
            st.push_back({a.son[0], s});
        } else if (!sl) {
            st.push_back({t, b.son[1]});
            st.push_back({t, b.son[0]});
        } else {
            tr.near_blocks.push_back({t, s});
        }
    }
}

}  // namespace
}  // namespace hm

using namespace hm;

extern "C" {

const char* hm_last_error(void) { return hm::g_err.c_str(); }

int hm_build_cluster_tree(const double* verts, int64_t nv, const int32_t* tris, int64_t nt,
                          int32_t leaf, double eta, hm_tree** out)
{
    if (!out) return fail(HM_EINVAL, "hm_build_cluster_tree: out is NULL");
    *out = nullptr;
    if (!verts || !tris) return fail(HM_EINVAL, "hm_build_cluster_tree: NULL mesh array");
    if (nv < 3 || nt < 1) return fail(HM_EINVAL, "hm_build_cluster_tree: empty mesh (nv=%lld, nt=%lld)",
                                      (long long)nv, (long long)nt);
    if (nt > (int64_t)INT32_MAX / 4)
        return fail(HM_EINVAL, "hm_build_cluster_tree: too many triangles (%lld)", (long long)nt);
    if (leaf < 1 || leaf > HM_MAX_LEAF)
        return fail(HM_EINVAL, "hm_build_cluster_tree: leaf must lie in 1..%d", HM_MAX_LEAF);
    if (!(eta > 0.0) || !std::isfinite(eta)) return fail(HM_EINVAL, "hm_build_cluster_tree: eta must be > 0");
    for (int64_t i = 0; i < 3 * nv; ++i)
        if (!std::isfinite(verts[i]))
            return fail(HM_EINVAL, "hm_build_cluster_tree: non-finite vertex coordinate");
    hm_tree* tr = new (std::nothrow) hm_tree();
    if (!tr) return fail(HM_ENOMEM, "hm_build_cluster_tree: out of host memory");
    try {
        tr->M = nt;
        tr->nv = nv;
        tr->leaf = leaf;
        tr->eta = eta;
        tr->V.assign(verts, verts + 3 * nv);
        tr->T.assign(tris, tris + 3 * nt);
        tr->coll.resize((size_t)(3 * nt));
        for (int64_t i = 0; i < nt; ++i) {
            const int32_t* t = &tr->T[(size_t)(3 * i)];
            for (int c = 0; c < 3; ++c)
                if (t[c] < 0 || t[c] >= nv) {
                    delete tr;
                    return fail(HM_EINVAL, "hm_build_cluster_tree: triangle %lld has vertex id %d out of range",
                                (long long)i, t[c]);
                }
            const double* a = &tr->V[3 * (size_t)t[0]];
            const double* b = &tr->V[3 * (size_t)t[1]];
            const double* c = &tr->V[3 * (size_t)t[2]];
            double u[3], v[3];
            for (int k = 0; k < 3; ++k) {
                u[k] = b[k] - a[k];
                v[k] = c[k] - a[k];
                tr->coll[(size_t)(3 * i + k)] = (a[k] + b[k] + c[k]) / 3.0;
            }
            double n0 = u[1] * v[2] - u[2] * v[1], n1 = u[2] * v[0] - u[0] * v[2],
                   n2 = u[0] * v[1] - u[1] * v[0];
            if (!(n0 * n0 + n1 * n1 + n2 * n2 > 0.0)) {
                delete tr;
                return fail(HM_EINVAL, "hm_build_cluster_tree: triangle %lld is degenerate", (long long)i);
            }
        }
        tr->perm.resize((size_t)nt);
        for (int64_t i = 0; i < nt; ++i) tr->perm[(size_t)i] = i;
        tr->nodes.reserve((size_t)(2 * nt));
        TreeBuilder tb{*tr, {}};
        tb.build(0, nt, 0);
        build_partition(*tr, tr->nodes, tr->nodes);
        for (size_t n = 0; n < tr->nodes.size(); ++n)
            if (tr->nodes[n].son[0] < 0) tr->leaves.push_back((int64_t)n);
        std::sort(tr->leaves.begin(), tr->leaves.end(), [&](int64_t a, int64_t b) {
            return tr->nodes[(size_t)a].lo < tr->nodes[(size_t)b].lo;
        });
    } catch (const std::bad_alloc&) {
        delete tr;
        return fail(HM_ENOMEM, "hm_build_cluster_tree: out of host memory");
    }
    *out = tr;
    return HM_OK;
}

int hm_build_point_tree(const hm_tree* surface, const double* pts, int64_t npts, int32_t leaf, hm_tree** out)
{
    if (!out) return fail(HM_EINVAL, "hm_build_point_tree: out is NULL");
    *out = nullptr;
    if (!surface || !pts) return fail(HM_EINVAL, "hm_build_point_tree: NULL argument");
    if (surface->kind != 0) return fail(HM_EINVAL, "hm_build_point_tree: `surface` must be a triangle tree");
    if (npts < 1) return fail(HM_EINVAL, "hm_build_point_tree: no points");
    if (npts > (int64_t)INT32_MAX / 4) return fail(HM_EINVAL, "hm_build_point_tree: too many points");
    if (leaf < 1 || leaf > HM_MAX_LEAF)
        return fail(HM_EINVAL, "hm_build_point_tree: leaf must lie in 1..%d", HM_MAX_LEAF);
    for (int64_t i = 0; i < 3 * npts; ++i)
        if (!std::isfinite(pts[i])) return fail(HM_EINVAL, "hm_build_point_tree: non-finite point coordinate");
    hm_tree* tr = new (std::nothrow) hm_tree();
    if (!tr) return fail(HM_ENOMEM, "hm_build_point_tree: out of host memory");
    try {
        auto src = std::make_shared<hm_tree>(*surface);
        src->adm.clear();
        src->near_blocks.clear();
        tr->M = npts;
        tr->kind = 1;
        tr->leaf = leaf;
        tr->eta = surface->eta;
        tr->coll.assign(pts, pts + 3 * npts);
        tr->perm.resize((size_t)npts);
        for (int64_t i = 0; i < npts; ++i) tr->perm[(size_t)i] = i;
        tr->nodes.reserve((size_t)(2 * npts));
        TreeBuilder tb{*tr, {}};
        tb.build(0, npts, 0);
        build_partition(*tr, tr->nodes, src->nodes);
        for (size_t n = 0; n < tr->nodes.size(); ++n)
            if (tr->nodes[n].son[0] < 0) tr->leaves.push_back((int64_t)n);
        std::sort(tr->leaves.begin(), tr->leaves.end(), [&](int64_t a, int64_t b) {
            return tr->nodes[(size_t)a].lo < tr->nodes[(size_t)b].lo;
        });
        tr->src = std::move(src);
    } catch (const std::bad_alloc&) {
        delete tr;
        return fail(HM_ENOMEM, "hm_build_point_tree: out of host memory");
    }
    *out = tr;
    return HM_OK;
}

int hm_build_vertex_tree(const hm_tree* surface, int32_t leaf, hm_tree** out)
{
    if (!out) return fail(HM_EINVAL, "hm_build_vertex_tree: out is NULL");
    *out = nullptr;
    if (!surface) return fail(HM_EINVAL, "hm_build_vertex_tree: NULL surface");
    if (surface->kind != 0) return fail(HM_EINVAL, "hm_build_vertex_tree: `surface` must be a triangle tree");
    if (leaf < 1 || leaf > HM_MAX_LEAF)
        return fail(HM_EINVAL, "hm_build_vertex_tree: leaf must lie in 1..%d", HM_MAX_LEAF);
    hm_tree* tr = new (std::nothrow) hm_tree();
    if (!tr) return fail(HM_ENOMEM, "hm_build_vertex_tree: out of host memory");
    try {
        const int64_t nv = surface->nv, M = surface->M;
        auto src = std::make_shared<hm_tree>(*surface);
        src->adm.clear();
        src->near_blocks.clear();
        tr->M = nv;
        tr->kind = 2;
        tr->leaf = leaf;
        tr->eta = surface->eta;
        tr->coll = surface->V;
        // stars: the box of every triangle merged into its three vertices
        tr->ibox.resize((size_t)(6 * nv));
        for (int64_t p = 0; p < nv; ++p)
            for (int k = 0; k < 3; ++k) {
                tr->ibox[(size_t)(6 * p + k)] = INFINITY;
                tr->ibox[(size_t)(6 * p + 3 + k)] = -INFINITY;
            }
        for (int64_t i = 0; i < M; ++i) {
            double lo[3] = {INFINITY, INFINITY, INFINITY}, hi[3] = {-INFINITY, -INFINITY, -INFINITY};
            for (int c = 0; c < 3; ++c)
                for (int k = 0; k < 3; ++k) {
                    const double v = surface->V[3 * (size_t)surface->T[(size_t)(3 * i + c)] + k];
                    lo[k] = std::min(lo[k], v);
                    hi[k] = std::max(hi[k], v);
                }
            for (int c = 0; c < 3; ++c) {
                const int64_t p = surface->T[(size_t)(3 * i + c)];
                for (int k = 0; k < 3; ++k) {
                    tr->ibox[(size_t)(6 * p + k)] = std::min(tr->ibox[(size_t)(6 * p + k)], lo[k]);
                    tr->ibox[(size_t)(6 * p + 3 + k)] = std::max(tr->ibox[(size_t)(6 * p + 3 + k)], hi[k]);
                }
            }
        }
        for (int64_t p = 0; p < nv; ++p)
            if (!(tr->ibox[(size_t)(6 * p)] <= tr->ibox[(size_t)(6 * p + 3)])) {
                delete tr;
                return fail(HM_EINVAL, "hm_build_vertex_tree: vertex %lld belongs to no triangle", (long long)p);
            }
        tr->perm.resize((size_t)nv);
        for (int64_t p = 0; p < nv; ++p) tr->perm[(size_t)p] = p;
        tr->nodes.reserve((size_t)(2 * nv));
        TreeBuilder tb{*tr, {}};
        tb.build(0, nv, 0);
        build_partition(*tr, src->nodes, tr->nodes);
        for (size_t n = 0; n < tr->nodes.size(); ++n)
            if (tr->nodes[n].son[0] < 0) tr->leaves.push_back((int64_t)n);
        std::sort(tr->leaves.begin(), tr->leaves.end(), [&](int64_t a, int64_t b) {
            return tr->nodes[(size_t)a].lo < tr->nodes[(size_t)b].lo;
        });
        tr->src = std::move(src);
    } catch (const std::bad_alloc&) {
        delete tr;
        return fail(HM_ENOMEM, "hm_build_vertex_tree: out of host memory");
    }
    *out = tr;
    return HM_OK;
}

int hm_tree_sizes(const hm_tree* tr, int64_t counts[6])
{
    if (!tr || !counts) return fail(HM_EINVAL, "hm_tree_sizes: NULL argument");
    counts[0] = tr->M;
    counts[1] = (int64_t)tr->nodes.size();
    counts[2] = (int64_t)tr->adm.size();
    counts[3] = (int64_t)tr->near_blocks.size();
    counts[4] = (int64_t)tr->leaves.size();
    counts[5] = tr->depth;
    return HM_OK;
}

int hm_tree_export(const hm_tree* tr, int64_t* perm, int64_t* nodes, int64_t* adm,
                   int64_t* near_blocks)
{
    if (!tr) return fail(HM_EINVAL, "hm_tree_export: NULL tree");
    if (perm) std::memcpy(perm, tr->perm.data(), (size_t)tr->M * sizeof(int64_t));
    if (nodes)
        for (size_t n = 0; n < tr->nodes.size(); ++n) {
            const Node& nd = tr->nodes[n];
            nodes[5 * n + 0] = nd.lo;
            nodes[5 * n + 1] = nd.hi;
            nodes[5 * n + 2] = nd.son[0];
            nodes[5 * n + 3] = nd.son[1];
            nodes[5 * n + 4] = nd.level;
        }
    if (adm)
        for (size_t b = 0; b < tr->adm.size(); ++b) {
            adm[2 * b] = tr->adm[b][0];
            adm[2 * b + 1] = tr->adm[b][1];
        }
    if (near_blocks)
        for (size_t b = 0; b < tr->near_blocks.size(); ++b) {
            near_blocks[2 * b] = tr->near_blocks[b][0];
            near_blocks[2 * b + 1] = tr->near_blocks[b][1];
        }
    return HM_OK;
}

void hm_tree_destroy(hm_tree* tr) { delete tr; }

int hm_set_material(hm_matrix* H, double E, double nu)
{
    if (!H) return fail(HM_EINVAL, "hm_set_material: NULL matrix");
    if (!(E > 0.0) || !std::isfinite(E)) return fail(HM_EINVAL, "hm_set_material: E must be > 0");
    if (!(nu > 0.0 && nu < 0.5)) return fail(HM_EINVAL, "hm_set_material: nu must lie in (0, 1/2)");
    H->E = E;
    H->nu = nu;
    // an evaluation operator reads E and nu at each call; the square matrix's
    // packed forms keep c1, c2 in their device tables
    for (int f = 0; f < HM_NFORMS && !H->rect; ++f)
        if (H->packed[f]) {
            int rc = write_mesh_table(*H, f, nullptr);
            if (rc) return rc;
        }
    return cuda_check(cudaDeviceSynchronize(), "hm_set_material");
}

int hm_get_stats(const hm_matrix* H, hm_stats* st)
{
    if (!H || !st) return fail(HM_EINVAL, "hm_get_stats: NULL argument");
    std::memset(st, 0, sizeof *st);
    st->M = H->M;
    st->nadm = H->nadm;
    st->nnear = H->nnear;
    st->nleaves = H->nleaves;
    for (const Blk& b : H->near_h) st->near_pairs += (int64_t)b.m * b.n;
    int64_t far_cols = 0;
    for (int64_t b = 0; b < H->nadm; ++b) {
        const Blk& bk = H->adm_h[(size_t)b];
        for (int k = 0; k < 7; ++k) {
            int32_t r = H->rank_h[(size_t)(b * 7 + k)];
            st->far_entries += (int64_t)r * (bk.m + bk.n);
            st->far_entries_kern[k] += (int64_t)r * (bk.m + bk.n);
            st->far_u_entries += (int64_t)r * bk.m;
            st->far_v_entries += (int64_t)r * bk.n;
            st->rank_sum[k] += r;
            st->rank_max[k] = std::max(st->rank_max[k], r);
            far_cols += r;
            if (H->flags_h[(size_t)(b * 7 + k)] & 1) st->rank_cap_hits++;
        }
    }
    st->factor_columns = far_cols;
    st->csp = H->csp;
    int64_t near_vals = st->near_pairs * 6;
    st->bytes_fp64 = (st->far_entries + near_vals) * 8;
    // bytes one product streams in each packed form (padded layouts; the
    // 16-bit forms add one float scale per factor column of U)
    const int64_t stream_elems = H->ul_total + H->vr_total;
    if (H->rect) {
        // the evaluation operator reads its block-ordered arenas (FP64, and
        // the FP32 copies once packed)
        const int64_t elems = H->u_total + H->v_total + H->n_total;
        st->bytes_form[HM_FP64] = elems * 8;
        if (H->packed[HM_FP32]) st->bytes_form[HM_FP32] = elems * 4;
    }
    for (int f = 0; f < HM_NFORMS && !H->rect; ++f) {
        if (!H->packed[f]) continue;
        int64_t wf = f == HM_FP64 ? 8 : (f == HM_FP32 ? 4 : 2);
        int64_t wn = f == HM_FP64 ? 8 : 4;
        st->bytes_form[f] = stream_elems * wf + H->nl_total * wn + (wf == 2 ? far_cols * 4 : 0);
        // INT16: the diagonal blocks from the FP32 near stream, the rest INT16
        if (f == HM_I16) st->bytes_form[f] = stream_elems * 2 + far_cols * 4 + H->nl_diag_total * 4 + H->nl16_bytes;
    }
    for (int i = 0; i < 3; ++i) st->assemble_ms[i] = H->asm_ms[i];
    for (int i = 0; i < 3; ++i) st->near_points[i] = H->asm_count[i];
    for (int i = 0; i < 2; ++i) st->aca_entries[i] = H->asm_count[3 + i];
    // FP64 operations the formulas state (header of hm_stats): near field
    const double whole = (double)H->asm_count[0], leaves = (double)H->asm_count[1],
                 self = (double)H->asm_count[2];
    const double split_pairs = std::max(0.0, (double)st->near_pairs - whole - self);
    const double steps = std::max(0.0, (leaves - split_pairs) / 3.0);  // a step turns 1 leaf into 4
    st->assembly_flops[0] = whole * 7 * 31 + leaves * (7 * 46 + 36) + steps * 63 + self * (96 * 35 + 63 + 7) +
                            split_pairs * 7;
    // ACA: the entries, then per block-kernel task of rank k the updates
    double upd = 0.0;
    if (H->asm_count[3] + H->asm_count[4] > 0)
        for (int64_t b = 0; b < H->nadm; ++b) {
            const hm::Blk& bk = H->adm_h[(size_t)b];
            for (int k = 0; k < 7; ++k) {
                const double r = (double)H->rank_h[(size_t)(b * 7 + k)];
                upd += 2.0 * r * (r - 1.0) * (bk.m + bk.n) + r * (3.0 * bk.n + 2.0 * bk.m);
            }
        }
    st->assembly_flops[1] = (double)H->asm_count[3] * 86 + (double)H->asm_count[4] * 114 + upd;
    return HM_OK;
}

int hm_export_factors(const hm_matrix* H, int64_t blk, int32_t kern, int32_t* rank, double* U,
                      double* V)
{
    if (!H || !rank) return fail(HM_EINVAL, "hm_export_factors: NULL argument");
    if (H->compacted && (U || V)) return fail(HM_EINVAL, "hm_export_factors: FP64 factors released (hm_compact)");
    if (blk < 0 || blk >= H->nadm || kern < 0 || kern > 6)
        return fail(HM_EINVAL, "hm_export_factors: block %lld kernel %d out of range",
                    (long long)blk, kern);
    size_t q = (size_t)(blk * 7 + kern);
    int32_t k = H->rank_h[q];
    *rank = k;
    const Blk& b = H->adm_h[(size_t)blk];
    if (U && k > 0)
        HM_CUDA(cudaMemcpy(U, H->U64.as<double>() + H->uoff_h[q], (size_t)k * b.m * sizeof(double),
                           cudaMemcpyDeviceToHost));
    if (V && k > 0)
        HM_CUDA(cudaMemcpy(V, H->V64.as<double>() + H->voff_h[q], (size_t)k * b.n * sizeof(double),
                           cudaMemcpyDeviceToHost));
    return HM_OK;
}

int hm_export_near(const hm_matrix* H, int64_t blk, double* out)
{
    if (!H || !out) return fail(HM_EINVAL, "hm_export_near: NULL argument");
    if (H->compacted) return fail(HM_EINVAL, "hm_export_near: FP64 near field released (hm_compact)");
    if (blk < 0 || blk >= H->nnear) return fail(HM_EINVAL, "hm_export_near: block out of range");
    const Blk& b = H->near_h[(size_t)blk];
    // device layout per block: [v][j][i] (i fastest); exported as [v][i][j]
    std::vector<double> tmp((size_t)6 * b.m * b.n);
    HM_CUDA(cudaMemcpy(tmp.data(), H->N64.as<double>() + H->noff_h[(size_t)blk],
                       tmp.size() * sizeof(double), cudaMemcpyDeviceToHost));
    for (int v = 0; v < 6; ++v)
        for (int i = 0; i < b.m; ++i)
            for (int j = 0; j < b.n; ++j)
                out[((size_t)v * b.m + i) * b.n + j] = tmp[((size_t)v * b.n + j) * b.m + i];
    return HM_OK;
}

int hm_check(const hm_matrix* H)
{
    if (!H) return fail(HM_EINVAL, "hm_check: NULL matrix");
    int e[4] = {0, 0, 0, 0};
    HM_CUDA(cudaMemcpy(e, H->d_err.p, sizeof e, cudaMemcpyDeviceToHost));
    if (e[0]) {
        const int zero[4] = {0, 0, 0, 0};
        HM_CUDA(cudaMemcpy(H->d_err.p, zero, sizeof zero, cudaMemcpyHostToDevice));
        if (e[0] == 2) return fail(HM_EINVAL, "hm_check: an earlier product met a leaf larger than a stage");
        return fail(HM_ETIMEOUT,
                    "hm_check: a bounded device wait ran out in an earlier product (site %d, stage %d, CTA %d)",
                    e[1], e[2], e[3]);
    }
    return HM_OK;
}

int hm_profile_enable(hm_matrix* H, int32_t on)
{
    if (!H) return fail(HM_EINVAL, "hm_profile_enable: NULL matrix");
    H->prof_on = on != 0;
    return HM_OK;
}

int hm_profile_read(hm_matrix* H, double ms[4], int64_t* calls)
{
    if (!H || !ms) return fail(HM_EINVAL, "hm_profile_read: NULL argument");
    for (int i = 0; i < 4; ++i) ms[i] = 0.0;
    int64_t n = H->prof_calls;
    for (int64_t c = 0; c < n; ++c) {
        cudaEvent_t* e = &H->prof_ev[(size_t)(4 * c)];
        HM_CUDA(cudaEventSynchronize(e[3]));
        for (int k = 0; k < 3; ++k) {
            float t = 0.0f;
            HM_CUDA(cudaEventElapsedTime(&t, e[k], e[k + 1]));
            ms[k] += t;
        }
    }
    if (calls) *calls = n;
    H->prof_calls = 0;
    return HM_OK;
}

// every device buffer a matrix may hold (its footprint; released at destroy)
static std::vector<hm::DevBuf*> matrix_bufs(hm_matrix* H)
{
    std::vector<hm::DevBuf*> v = {
        &H->d_perm, &H->d_adm, &H->d_near, &H->d_rank, &H->d_uoff, &H->d_voff, &H->d_coff, &H->d_noff,
        &H->d_leaf, &H->d_lf_base, &H->d_lf_ptr, &H->d_lf_items, &H->d_lf_src, &H->d_lr_ptr, &H->d_lr_items, &H->d_ln_base, &H->d_ln_ptr,
        &H->d_ln_items, &H->d_ln_src, &H->d_vb_base, &H->d_vb_ld, &H->d_vb_coff, &H->fdesc, &H->d_groups,
        &H->d_units, &H->d_tcunits, &H->d_multi, &H->d_big, &H->d_small, &H->d_fwd_all, &H->d_work,
        &H->d_pos_prefix, &H->d_counters, &H->d_err, &H->U64, &H->V64, &H->N64, &H->Nl64, &H->Nl32, &H->SU,
        &H->SV, &H->SW16, &H->fdesc16, &H->xg, &H->wb, &H->zb, &H->xh, &H->yh, &H->g_coll, &H->g_tri, &H->g_qp, &H->g_qw,
        &H->Nl16, &H->d_ln16_base, &H->d_ln16_diag,
        &H->g_diam, &H->d_rperm, &H->g_rows, &H->g_nrm, &H->d_star_ptr, &H->d_star, &H->d_tris, &H->d_mesh_k,
        &H->dl_w};
    for (int f = 0; f < HM_NFORMS; ++f) {
        v.push_back(&H->d_mesh[f]);
        v.push_back(&H->Ul[f]);
        v.push_back(&H->Vr[f]);
    }
    return v;
}

int hm_compact(hm_matrix* H)
{
    if (!H) return fail(HM_EINVAL, "hm_compact: NULL matrix");
    if (H->rect) return fail(HM_EINVAL, "hm_compact: an evaluation operator has no packed form");
    if (H->compacted) return HM_OK;
    if (!H->packed[HM_FP32] && !H->packed[HM_BF16] && !H->packed[HM_FP16] && !H->packed[HM_I16])
        return fail(HM_EINVAL, "hm_compact: pack a reduced form first (hm_pack)");
    HM_CUDA(cudaDeviceSynchronize());
    hm::DevBuf* bufs[] = {&H->U64, &H->V64, &H->N64, &H->SV, &H->Ul[HM_FP64], &H->Vr[HM_FP64], &H->Nl64,
                          &H->d_lf_src, &H->d_ln_src, &H->d_mesh[HM_FP64]};
    cudaStream_t saved = H->alloc.stream;
    H->alloc.stream = nullptr;
    for (hm::DevBuf* b : bufs) {
        H->alloc.release(b->p, b->bytes);
        b->p = nullptr;
        b->bytes = 0;
    }
    H->alloc.stream = saved;
    H->packed[HM_FP64] = false;
    H->compacted = true;
    return cuda_check(cudaDeviceSynchronize(), "hm_compact");
}

int hm_footprint(const hm_matrix* H, int64_t* bytes)
{
    if (!H || !bytes) return fail(HM_EINVAL, "hm_footprint: NULL argument");
    int64_t t = 0;
    for (const hm::DevBuf* b : matrix_bufs(const_cast<hm_matrix*>(H)))
        if (b->p) t += (int64_t)b->bytes;
    for (const hm::DevBuf& b : H->ev)
        if (b.p) t += (int64_t)b.bytes;
    *bytes = t;
    return HM_OK;
}

void hm_matrix_destroy(hm_matrix* H)
{
    if (!H) return;
    for (cudaEvent_t e : H->prof_ev) cudaEventDestroy(e);

    // the assembly stream may be gone by now: drain the device and release
    // on the legacy default stream
    cudaDeviceSynchronize();
    H->alloc.stream = nullptr;
    for (hm::DevBuf* b : matrix_bufs(H)) {
        H->alloc.release(b->p, b->bytes);
        b->p = nullptr;
    }
    for (hm::DevBuf& b : H->ev) {
        H->alloc.release(b.p, b.bytes);
        b.p = nullptr;
    }
    cudaDeviceSynchronize();
    delete H;
}

}  // extern "C"
