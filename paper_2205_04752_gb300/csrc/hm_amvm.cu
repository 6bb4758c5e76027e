// hm_amvm.cu -- adaptive matrix-vector multiplication (Algorithm 2, Section
// 3) on the device, FP64, from the assembled ACA factors.
//
// A_k keeps the first r_b crosses of each of the seven ACA sequences of every
// admissible block (the whole sequence when it is shorter), the look-ahead
// A^_k the first r_b + L; near blocks are exact in both.  With b_k = A_k x
// and the look-ahead parts D_b = (A^_k - A_k)_b x, the estimator is gamma_k =
// ||sum_b D_b|| = ||b^_k - b_k||.  Marking (step 3) goes through the rows in
// decreasing |(b^_k - b_k)_i| and adds every block t x s with i in t and
// |(D_b)_i| >= (1 - theta)(c_sp N N)^{-1/2} gamma_k until gamma_k -
// gamma_k(P_k) >= theta gamma_k; a marked block takes the look-ahead ranks
// (step 4).  The loop ends when gamma_k <= eps ||b^_k||.
//
// Device work per iteration: the look-ahead parts of the blocks refined in
// the previous step (one CTA per block: V^T x of the new crosses by warp
// reductions, then U times them row by row), the row sums of all parts (each
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

#include "hm_internal.h"

namespace hm {
namespace {

constexpr int kAmvmThreads = 256;
constexpr int kAmvmMaxCross = 32;  // crosses of one block part (r0 and the look-ahead)

struct AmvmItem {
    int32_t b, l0, l1, pad;
};

__global__ void amvm_gather_kernel(const int32_t* __restrict__ perm, const double* __restrict__ x,
                                   double* __restrict__ xc, int64_t M)
{
    const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= M) return;
    const int64_t o = 3 * (int64_t)perm[p];
#pragma unroll
    for (int a = 0; a < 3; ++a) xc[3 * p + a] = x[o + a];
}

__global__ void amvm_scatter_kernel(const int32_t* __restrict__ perm, const double* __restrict__ bc,
                                    double* __restrict__ y, int64_t M)
{
    const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= M) return;
    const int64_t o = 3 * (int64_t)perm[p];
#pragma unroll
    for (int a = 0; a < 3; ++a) y[o + a] = bc[3 * p + a];
}

// near field, exact: position p adds its near blocks (row cluster = its leaf)
// in block order; the six stored kernels V_11..V_33 give V_Delta as their
// trace
__global__ void amvm_near_kernel(const int32_t* __restrict__ ipos, const int32_t* __restrict__ nptr,
                                 const int32_t* __restrict__ nidx, const Blk* __restrict__ near,
                                 const int64_t* __restrict__ noff, const double* __restrict__ N64,
                                 const double* __restrict__ xc, double c1, double c2, double* __restrict__ out,
                                 int64_t M)
{
    const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= M) return;
    const int I = ipos[p];
    double s0 = 0.0, s1 = 0.0, s2 = 0.0;
    for (int q = nptr[I]; q < nptr[I + 1]; ++q) {
        const int b = nidx[q];
        const Blk bk = near[b];
        const int64_t i = p - bk.t0, pairs = (int64_t)bk.m * bk.n;
        const double* Nb = N64 + noff[b];
        for (int j = 0; j < bk.n; ++j) {
            const double* xj = xc + 3 * (int64_t)(bk.s0 + j);
            const int64_t e = (int64_t)j * bk.m + i;
            const double v11 = Nb[e], v12 = Nb[pairs + e], v13 = Nb[2 * pairs + e];
            const double v22 = Nb[3 * pairs + e], v23 = Nb[4 * pairs + e], v33 = Nb[5 * pairs + e];
            const double vd = v11 + v22 + v33;
            s0 += c1 * vd * xj[0] + c2 * (v11 * xj[0] + v12 * xj[1] + v13 * xj[2]);
            s1 += c1 * vd * xj[1] + c2 * (v12 * xj[0] + v22 * xj[1] + v23 * xj[2]);
            s2 += c1 * vd * xj[2] + c2 * (v13 * xj[0] + v23 * xj[1] + v33 * xj[2]);
        }
    }
    out[3 * p] = s0;
    out[3 * p + 1] = s1;
    out[3 * p + 2] = s2;
}

// the crosses l0 .. l1 - 1 of admissible block b applied to x(s): |t| x 3
// values at D + doff[b] (component fastest).  Kernel k = 0 (V_Delta) acts on
// each component with c1; V_pq (k = 1..6) adds c2 U (V^T x_q) to y_p and, p !=
// q, c2 U (V^T x_p) to y_q.  The crosses go kAmvmMaxCross at a time: the
// first chunk writes the block's values, later ones add theirs (a fixed
// order, so the result is deterministic).
__global__ void __launch_bounds__(kAmvmThreads) amvm_part_kernel(
    const AmvmItem* __restrict__ items, const Blk* __restrict__ adm, const int32_t* __restrict__ rank,
    const double* const* __restrict__ uptr, const double* const* __restrict__ vptr, const double* __restrict__ xc,
    double c1, double c2, const int64_t* __restrict__ doff, double* __restrict__ D)
{
    __shared__ double W[7][kAmvmMaxCross][3];
    __shared__ int kk[7];
    const AmvmItem it = items[blockIdx.x];
    const Blk bk = adm[it.b];
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31, nw = kAmvmThreads / 32;
    int rmax = 0;
#pragma unroll
    for (int k = 0; k < 7; ++k) rmax = max(rmax, rank[it.b * 7 + k]);
    // at least one chunk, so that a block without crosses in range writes zeros
    const int lend = max(it.l0 + 1, min(it.l1, rmax));
    double* out = D + doff[it.b];
    for (int l0 = it.l0; l0 < lend; l0 += kAmvmMaxCross) {
    const int l1 = min(it.l1, l0 + kAmvmMaxCross);
    __syncthreads();  // the previous chunk's W has been read
    if (tid < 7) kk[tid] = max(0, min(l1, rank[it.b * 7 + tid]) - l0);
    __syncthreads();
    // V^T x(s) of every (kernel, cross): one warp each, fixed reduction order
    for (int pr = warp; pr < 7 * kAmvmMaxCross; pr += nw) {
        const int k = pr / kAmvmMaxCross, l = pr - k * kAmvmMaxCross;
        if (l >= kk[k]) continue;
        const double* v = vptr[it.b * 7 + k] + (int64_t)(l0 + l) * bk.n;
        double a0 = 0.0, a1 = 0.0, a2 = 0.0;
        for (int j = lane; j < bk.n; j += 32) {
            const double* xj = xc + 3 * (int64_t)(bk.s0 + j);
            a0 += v[j] * xj[0];
            a1 += v[j] * xj[1];
            a2 += v[j] * xj[2];
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            a0 += __shfl_xor_sync(0xffffffffu, a0, o);
            a1 += __shfl_xor_sync(0xffffffffu, a1, o);
            a2 += __shfl_xor_sync(0xffffffffu, a2, o);
        }
        if (lane == 0) {
            W[k][l][0] = a0;
            W[k][l][1] = a1;
            W[k][l][2] = a2;
        }
    }
    __syncthreads();
    for (int i = tid; i < bk.m; i += kAmvmThreads) {
        double y[3] = {0.0, 0.0, 0.0};
#pragma unroll
        for (int k = 0; k < 7; ++k) {
            const double* u = uptr[it.b * 7 + k] + (int64_t)l0 * bk.m + i;
            double s[3] = {0.0, 0.0, 0.0};
            for (int l = 0; l < kk[k]; ++l) {
                const double ul = u[(int64_t)l * bk.m];
                s[0] += ul * W[k][l][0];
                s[1] += ul * W[k][l][1];
                s[2] += ul * W[k][l][2];
            }
            if (k == 0) {
                y[0] += c1 * s[0];
                y[1] += c1 * s[1];
                y[2] += c1 * s[2];
            } else {
                const int p = k <= 3 ? 0 : (k <= 5 ? 1 : 2);
                const int q = k <= 3 ? k - 1 : (k <= 5 ? k - 3 : 2);
                y[p] += c2 * s[q];
                if (p != q) y[q] += c2 * s[p];
            }
        }
        if (l0 == it.l0) {
            out[3 * i] = y[0];
            out[3 * i + 1] = y[1];
            out[3 * i + 2] = y[2];
        } else {
            out[3 * i] += y[0];
            out[3 * i + 1] += y[1];
            out[3 * i + 2] += y[2];
        }
    }
    }
}

// out[p] = (or +=) sum of the parts of the admissible blocks whose row
// cluster holds position p, in block order; with flags, the flagged blocks
// only
__global__ void amvm_rowsum_kernel(const int32_t* __restrict__ ipos, const int32_t* __restrict__ aptr,
                                   const int32_t* __restrict__ aidx, const Blk* __restrict__ adm,
                                   const int64_t* __restrict__ doff, const double* __restrict__ D,
                                   const uint8_t* __restrict__ flags, int add, double* __restrict__ out,
                                   int64_t M)
{
    const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= M) return;
    const int I = ipos[p];
    double s0 = 0.0, s1 = 0.0, s2 = 0.0;
    for (int q = aptr[I]; q < aptr[I + 1]; ++q) {
        const int b = aidx[q];
        if (flags && !flags[b]) continue;
        const double* d = D + doff[b] + 3 * (p - adm[b].t0);
        s0 += d[0];
        s1 += d[1];
        s2 += d[2];
    }
    if (add) {
        out[3 * p] += s0;
        out[3 * p + 1] += s1;
        out[3 * p + 2] += s2;
    } else {
        out[3 * p] = s0;
        out[3 * p + 1] = s1;
        out[3 * p + 2] = s2;
    }
}

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

// elementary intervals of cluster positions (between consecutive block row
// boundaries) and, per interval, the blocks whose row range covers it, in
// block order
struct RowLists {
    std::vector<int32_t> ipos;  // M: interval of each position
    std::vector<int32_t> ptr, idx;
};

RowLists row_lists(int64_t M, const std::vector<int64_t>& bounds, const std::vector<Blk>& blks)
{
    RowLists r;
    const int nI = (int)bounds.size() - 1;
    r.ipos.resize((size_t)M);
    for (int I = 0; I < nI; ++I)
        for (int64_t p = bounds[(size_t)I]; p < bounds[(size_t)I + 1]; ++p) r.ipos[(size_t)p] = I;
    std::vector<int32_t> cnt((size_t)nI + 1, 0);
    for (const Blk& b : blks)
        for (int I = r.ipos[(size_t)b.t0]; I < nI && bounds[(size_t)I] < b.t0 + b.m; ++I) cnt[(size_t)I + 1]++;
    r.ptr.assign((size_t)nI + 1, 0);
    for (int I = 0; I < nI; ++I) r.ptr[(size_t)I + 1] = r.ptr[(size_t)I] + cnt[(size_t)I + 1];
    r.idx.resize((size_t)r.ptr[(size_t)nI]);
    std::vector<int32_t> fill(r.ptr.begin(), r.ptr.end() - 1);
    for (size_t b = 0; b < blks.size(); ++b)
        for (int I = r.ipos[(size_t)blks[b].t0]; I < nI && bounds[(size_t)I] < blks[b].t0 + blks[b].m; ++I)
            r.idx[(size_t)fill[(size_t)I]++] = (int32_t)b;
    return r;
}

// device buffers of one call, from the matrix's allocator
struct Pool {
    Allocator al;
    std::vector<std::pair<void*, size_t>> held;
    ~Pool()
    {
        for (auto& h : held) al.release(h.first, h.second);
    }
    template <class T>
    T* get(size_t n)
    {
        const size_t bytes = std::max<size_t>(n, 1) * sizeof(T);
        void* p = al.alloc(bytes);
        if (p) held.emplace_back(p, bytes);
        return static_cast<T*>(p);
    }
};

template <class T>
int put(T* d, const std::vector<T>& h, cudaStream_t s)
{
    if (!h.empty()) HM_CUDA(cudaMemcpyAsync(d, h.data(), h.size() * sizeof(T), cudaMemcpyHostToDevice, s));
    return HM_OK;
}

}  // namespace
}  // namespace hm

using namespace hm;

extern "C" int hm_amvm(const hm_matrix* H, const double* x, double* y, const hm_amvm_params* prm,
                       hm_amvm_info* info, double* gamma_hist, double* gamma_rest_hist, int32_t hist_cap,
                       int32_t* block_ranks, void* stream)
{
    if (!H || !x || !y || !prm) return fail(HM_EINVAL, "hm_amvm: NULL argument");
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
    hm_matrix& Hm = const_cast<hm_matrix&>(*H);  // on-demand ACA allocates through the matrix's allocator
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

// ------------------------------------------------------------------------
// The evaluation operator ~V_h (Section 5, Eq. (vector_eq)): its product --
// every admissible block with all its crosses, the near field exact, per row
// position a fixed summation order -- in FP64 (the exact form) or, after
// hm_pack(HM_FP32), from FP32 copies of the same block-ordered arenas with
// FP32 arithmetic (T = double or float below), in four passes, each
// spread over warps so that the factor and near-field streams are read with
// many loads in flight:
//   ev_fwd   one warp per (block, kernel): w_c = V_c^T x(s) for its crosses c
//            (3 components of x gathered component-major; lane-strided sums,
//            fixed butterfly);
//   ev_back  one warp per (block, 32 rows): the block's part of the rows,
//            U w with c1 / c2 as in the adaptive product's part kernel;
//   ev_near  one warp per (near block, 32 rows): the near block's part;
//   ev_rowsum  one thread per row position: its admissible parts in block
//            order, then its near parts in block order.
namespace hm {
namespace {
enum { kEvIpos, kEvAptr, kEvAidx, kEvNptr, kEvNidx, kEvDoff, kEvBack, kEvNear, kEvNdoff, kEvW, kEvXc, kEvYc,
       kEvD, kEvDn };
static_assert(kEvDn + 1 == hm_matrix::kEvBufs, "evaluation buffers");
constexpr int kEvThreads = 256;
constexpr int kEvWarps = kEvThreads / 32;

template <class T>
__device__ __forceinline__ T ev_sum32(T v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// x gathered to cluster order, component-major (xs[a M + p]), so that a
// warp reading 32 consecutive positions of one component is coalesced
template <class T>
__global__ void ev_gather_kernel(const int32_t* __restrict__ perm, const double* __restrict__ x,
                                 T* __restrict__ xs, int64_t M)
{
    const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= M) return;
    const int64_t o = 3 * (int64_t)perm[p];
#pragma unroll
    for (int a = 0; a < 3; ++a) xs[a * M + p] = (T)x[o + a];
}

template <class T>
__global__ void ev_scatter_kernel(const int32_t* __restrict__ perm, const T* __restrict__ yc,
                                  double* __restrict__ y, int64_t M)
{
    const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= M) return;
    const int64_t o = 3 * (int64_t)perm[p];
#pragma unroll
    for (int a = 0; a < 3; ++a) y[o + a] = (double)yc[3 * p + a];
}

// the FP32 form: element-wise copies of the block-ordered FP64 arenas
__global__ void ev_to_fp32_kernel(const double* __restrict__ src, float* __restrict__ dst, int64_t n)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        dst[i] = (float)src[i];
}

// Butterfly sums of 2 or 4 values at once: at the first levels each half (or
// quarter) of the warp keeps one value and sends the other, so that later
// levels reduce all of them together.  Every value meets the same partners in
// the same order as in ev_sum32 (the bits agree); the totals end in lane 0
// (a), 16 (b), 8 (c) and 24 (d).
template <class T>
__device__ __forceinline__ T ev_sum32x2(T a, T b, int lane)
{
    const bool h = lane & 16;
    T k = h ? b : a;
    k += __shfl_xor_sync(0xffffffffu, h ? a : b, 16);
#pragma unroll
    for (int o = 8; o > 0; o >>= 1) k += __shfl_xor_sync(0xffffffffu, k, o);
    return k;
}

template <class T>
__device__ __forceinline__ T ev_sum32x4(T a, T b, T c, T d, int lane)
{
    const bool h = lane & 16, g = lane & 8;
    T k0 = h ? b : a, k1 = h ? d : c;
    k0 += __shfl_xor_sync(0xffffffffu, h ? a : b, 16);
    k1 += __shfl_xor_sync(0xffffffffu, h ? c : d, 16);
    T k = g ? k1 : k0;
    k += __shfl_xor_sync(0xffffffffu, g ? k0 : k1, 8);
#pragma unroll
    for (int o = 4; o > 0; o >>= 1) k += __shfl_xor_sync(0xffffffffu, k, o);
    return k;
}

// the sums of G crosses l .. l + G - 1 (G = 4, 2 or 1): V_l^T x_a for the
// components a the kernel needs -- all three for V_Delta, p for V_pp, p and
// q for V_pq (p != q) -- each lane-strided over the columns, then the
// butterfly; the other slots of w are not written (nor read)
template <class T, bool A0, bool A1, bool A2, int G>
__device__ __forceinline__ void ev_fwd_group(const T* __restrict__ v, int l, int n, const T* __restrict__ x0,
                                             const T* __restrict__ x1, const T* __restrict__ x2,
                                             T* __restrict__ wq, int lane)
{
    const T* vl = v + (int64_t)l * n;
    T acc[3][G];
#pragma unroll
    for (int c = 0; c < 3; ++c)
#pragma unroll
        for (int g = 0; g < G; ++g) acc[c][g] = T(0);
#pragma unroll 2
    for (int j = lane; j < n; j += 32) {
        T vg[G];
#pragma unroll
        for (int g = 0; g < G; ++g) vg[g] = vl[(int64_t)g * n + j];
        if (A0) {
            const T x = x0[j];
#pragma unroll
            for (int g = 0; g < G; ++g) acc[0][g] += vg[g] * x;
        }
        if (A1) {
            const T x = x1[j];
#pragma unroll
            for (int g = 0; g < G; ++g) acc[1][g] += vg[g] * x;
        }
        if (A2) {
            const T x = x2[j];
#pragma unroll
            for (int g = 0; g < G; ++g) acc[2][g] += vg[g] * x;
        }
    }
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        if ((c == 0 && !A0) || (c == 1 && !A1) || (c == 2 && !A2)) continue;
        T* wc = wq + 3 * l + c;
        if (G == 4) {
            const T t = ev_sum32x4<T>(acc[c][0], acc[c][G > 1 ? 1 : 0], acc[c][G > 2 ? 2 : 0],
                                        acc[c][G > 3 ? 3 : 0], lane);
            if (lane == 0) wc[0] = t;
            if (lane == 16) wc[3] = t;
            if (lane == 8) wc[6] = t;
            if (lane == 24) wc[9] = t;
        } else if (G == 2) {
            const T t = ev_sum32x2<T>(acc[c][0], acc[c][G > 1 ? 1 : 0], lane);
            if (lane == 0) wc[0] = t;
            if (lane == 16) wc[3] = t;
        } else {
            const T t = ev_sum32<T>(acc[c][0]);
            if (lane == 0) wc[0] = t;
        }
    }
}

template <class T, bool A0, bool A1, bool A2>
__device__ __forceinline__ void ev_fwd_task(const T* __restrict__ v, int r, int n, const T* __restrict__ x0,
                                            const T* __restrict__ x1, const T* __restrict__ x2,
                                            T* __restrict__ wq, int lane)
{
    int l = 0;
    for (; l + 4 <= r; l += 4) ev_fwd_group<T, A0, A1, A2, 4>(v, l, n, x0, x1, x2, wq, lane);
    if (l + 2 <= r) {
        ev_fwd_group<T, A0, A1, A2, 2>(v, l, n, x0, x1, x2, wq, lane);
        l += 2;
    }
    if (l < r) ev_fwd_group<T, A0, A1, A2, 1>(v, l, n, x0, x1, x2, wq, lane);
}

template <class T>
__global__ void __launch_bounds__(kEvThreads) ev_fwd_kernel(const Blk* __restrict__ adm,
                                                            const int32_t* __restrict__ rank,
                                                            const int64_t* __restrict__ voff,
                                                            const int64_t* __restrict__ coff,
                                                            const T* __restrict__ Vf,
                                                            const T* const* __restrict__ vptr,
                                                            const T* __restrict__ xs, int64_t M, int64_t ntask,
                                                            T* __restrict__ w)
{
    const int lane = threadIdx.x & 31;
    const int64_t nwarp = (int64_t)gridDim.x * kEvWarps;
    for (int64_t q = (int64_t)blockIdx.x * kEvWarps + (threadIdx.x >> 5); q < ntask; q += nwarp) {
        const int r = rank[q];
        if (r == 0) continue;
        const Blk b = adm[q / 7];
        const T* v = vptr ? vptr[q] : Vf + voff[q];  // per-task pointers: factors of ACA on demand
        const T* x0 = xs + b.s0;
        const T* x1 = x0 + M;
        const T* x2 = x1 + M;
        T* wq = w + 3 * coff[q];
        switch ((int)(q % 7)) {  // V_Delta, V_11, V_12, V_13, V_22, V_23, V_33
            case 0: ev_fwd_task<T, true, true, true>(v, r, b.n, x0, x1, x2, wq, lane); break;
            case 1: ev_fwd_task<T, true, false, false>(v, r, b.n, x0, x1, x2, wq, lane); break;
            case 2: ev_fwd_task<T, true, true, false>(v, r, b.n, x0, x1, x2, wq, lane); break;
            case 3: ev_fwd_task<T, true, false, true>(v, r, b.n, x0, x1, x2, wq, lane); break;
            case 4: ev_fwd_task<T, false, true, false>(v, r, b.n, x0, x1, x2, wq, lane); break;
            case 5: ev_fwd_task<T, false, true, true>(v, r, b.n, x0, x1, x2, wq, lane); break;
            default: ev_fwd_task<T, false, false, true>(v, r, b.n, x0, x1, x2, wq, lane); break;
        }
    }
}

template <class T>
__global__ void __launch_bounds__(kEvThreads) ev_back_kernel(const int2* __restrict__ items, int64_t nitems,
                                                             const Blk* __restrict__ adm,
                                                             const int32_t* __restrict__ rank,
                                                             const int64_t* __restrict__ uoff,
                                                             const int64_t* __restrict__ coff,
                                                             const T* __restrict__ Uf,
                                                             const T* const* __restrict__ uptr,
                                                             const T* __restrict__ w,
                                                             T c1, T c2, const int64_t* __restrict__ doff,
                                                             T* __restrict__ D)
{
    const int lane = threadIdx.x & 31;
    const int64_t nwarp = (int64_t)gridDim.x * kEvWarps;
    for (int64_t it = (int64_t)blockIdx.x * kEvWarps + (threadIdx.x >> 5); it < nitems; it += nwarp) {
        const int2 item = items[it];
        const Blk bk = adm[item.x];
        const int i = item.y * 32 + lane;
        if (i >= bk.m) continue;
        T y[3] = {T(0), T(0), T(0)};
#pragma unroll
        for (int k = 0; k < 7; ++k) {
            const int64_t q = (int64_t)item.x * 7 + k;
            const int r = rank[q];
            const T* u = (uptr ? uptr[q] : Uf + uoff[q]) + i;
            const T* wq = w + 3 * coff[q];
            // the components this kernel uses (the slots ev_fwd wrote)
            const bool u0 = k <= 3, u1 = k == 0 || k == 2 || k == 4 || k == 5, u2 = k == 0 || k == 3 || k >= 5;
            T s[3] = {T(0), T(0), T(0)};
            // loads in flight: eight crosses deep in FP64, four in FP32 (measured best)
            if (sizeof(T) == 8) {
#pragma unroll 8
                for (int l = 0; l < r; ++l) {
                    const T ul = u[(int64_t)l * bk.m];
                    if (u0) s[0] += ul * wq[3 * l];
                    if (u1) s[1] += ul * wq[3 * l + 1];
                    if (u2) s[2] += ul * wq[3 * l + 2];
                }
            } else {
#pragma unroll 4
                for (int l = 0; l < r; ++l) {
                    const T ul = u[(int64_t)l * bk.m];
                    if (u0) s[0] += ul * wq[3 * l];
                    if (u1) s[1] += ul * wq[3 * l + 1];
                    if (u2) s[2] += ul * wq[3 * l + 2];
                }
            }
            if (k == 0) {
                y[0] += c1 * s[0];
                y[1] += c1 * s[1];
                y[2] += c1 * s[2];
            } else {
                const int p = k <= 3 ? 0 : (k <= 5 ? 1 : 2);
                const int qq = k <= 3 ? k - 1 : (k <= 5 ? k - 3 : 2);
                y[p] += c2 * s[qq];
                if (p != qq) y[qq] += c2 * s[p];
            }
        }
        T* out = D + doff[item.x] + 3 * (int64_t)i;
        out[0] = y[0];
        out[1] = y[1];
        out[2] = y[2];
    }
}

template <class T>
__global__ void __launch_bounds__(kEvThreads) ev_near_kernel(const int2* __restrict__ items, int64_t nitems,
                                                             const Blk* __restrict__ near,
                                                             const int64_t* __restrict__ noff,
                                                             const T* __restrict__ Nf, const T* __restrict__ xs,
                                                             int64_t M, T c1, T c2,
                                                             const int64_t* __restrict__ ndoff, T* __restrict__ Dn)
{
    const int lane = threadIdx.x & 31;
    const int64_t nwarp = (int64_t)gridDim.x * kEvWarps;
    for (int64_t it = (int64_t)blockIdx.x * kEvWarps + (threadIdx.x >> 5); it < nitems; it += nwarp) {
        const int2 item = items[it];
        const Blk bk = near[item.x];
        const int i = item.y * 32 + lane;
        if (i >= bk.m) continue;
        const int64_t pairs = (int64_t)bk.m * bk.n;
        const T* Nb = Nf + noff[item.x];
        // y_a = c1 sum_j V_Delta x_a + c2 sum_j sum_b V_ab x_b: the two sums
        // apart, c1 and c2 applied once per row (14 operations a pair)
        T d0 = T(0), d1 = T(0), d2 = T(0), s0 = T(0), s1 = T(0), s2 = T(0);
        const T* x0 = xs + bk.s0;
#pragma unroll 4
        for (int j = 0; j < bk.n; ++j) {
            const T xa = x0[j], xb = x0[M + j], xc = x0[2 * M + j];
            const int64_t e = (int64_t)j * bk.m + i;
            const T v11 = Nb[e], v12 = Nb[pairs + e], v13 = Nb[2 * pairs + e];
            const T v22 = Nb[3 * pairs + e], v23 = Nb[4 * pairs + e], v33 = Nb[5 * pairs + e];
            const T vd = v11 + v22 + v33;
            d0 += vd * xa;
            d1 += vd * xb;
            d2 += vd * xc;
            s0 += v11 * xa;
            s0 += v12 * xb;
            s0 += v13 * xc;
            s1 += v12 * xa;
            s1 += v22 * xb;
            s1 += v23 * xc;
            s2 += v13 * xa;
            s2 += v23 * xb;
            s2 += v33 * xc;
        }
        T* out = Dn + ndoff[item.x] + 3 * (int64_t)i;
        out[0] = c1 * d0 + c2 * s0;
        out[1] = c1 * d1 + c2 * s1;
        out[2] = c1 * d2 + c2 * s2;
    }
}

template <class T>
__global__ void ev_rowsum_kernel(const int32_t* __restrict__ ipos, const int32_t* __restrict__ aptr,
                                 const int32_t* __restrict__ aidx, const Blk* __restrict__ adm,
                                 const int64_t* __restrict__ doff, const T* __restrict__ D,
                                 const int32_t* __restrict__ nptr, const int32_t* __restrict__ nidx,
                                 const Blk* __restrict__ near, const int64_t* __restrict__ ndoff,
                                 const T* __restrict__ Dn, T* __restrict__ out, int64_t Mr)
{
    const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= Mr) return;
    const int I = ipos[p];
    T s0 = T(0), s1 = T(0), s2 = T(0);
    for (int q = aptr[I]; q < aptr[I + 1]; ++q) {
        const int b = aidx[q];
        const T* d = D + doff[b] + 3 * (p - adm[b].t0);
        s0 += d[0];
        s1 += d[1];
        s2 += d[2];
    }
    for (int q = nptr[I]; q < nptr[I + 1]; ++q) {
        const int b = nidx[q];
        const T* d = Dn + ndoff[b] + 3 * (p - near[b].t0);
        s0 += d[0];
        s1 += d[1];
        s2 += d[2];
    }
    out[3 * p] = s0;
    out[3 * p + 1] = s1;
    out[3 * p + 2] = s2;
}

template <class T>
int ev_put(hm_matrix& H, int which, const std::vector<T>& h, size_t n)
{
    DevBuf& d = H.ev[which];
    d.bytes = std::max<size_t>(n, 1) * sizeof(T);
    d.p = H.alloc.alloc(d.bytes);
    if (!d.p) return fail(HM_ENOMEM, "evaluation operator: device allocation of %zu bytes failed", d.bytes);
    if (!h.empty())
        HM_CUDA(cudaMemcpyAsync(d.p, h.data(), h.size() * sizeof(T), cudaMemcpyHostToDevice, H.alloc.stream));
    return HM_OK;
}
}  // namespace

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
        (rc = ev_put(H, kEvD, none, (size_t)doff[(size_t)nb])) || (rc = ev_put(H, kEvDn, none, (size_t)ndoff[(size_t)nn])))
        return rc;
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
             cudaStream_t s)
{
    const int64_t M = H.M, Mr = H.Mr, nb = H.nadm;
    const T c1 = (T)((1.0 + H.nu) * (3.0 - 4.0 * H.nu) / (2.0 * H.E * (1.0 - H.nu)));
    const T c2 = (T)((1.0 + H.nu) / (2.0 * H.E * (1.0 - H.nu)));
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
        ev_scatter_kernel<T><<<gM, 256, 0, s>>>(H.d_rperm.as<int32_t>(), yc, u + (int64_t)r * 3 * Mr, Mr);
        HM_CUDA(cudaGetLastError());
    }
    return HM_OK;
}
}  // namespace
}  // namespace hm

extern "C" int hm_eval_points(const hm_matrix* H, const double* t, double* u, int32_t nrhs, int32_t form,
                              void* stream)
{
    if (!H || !t || !u) return fail(HM_EINVAL, "hm_eval_points: NULL argument");
    if (!H->rect) return fail(HM_EINVAL, "hm_eval_points: not an evaluation operator (use hm_matvec)");
    if (H->aca_deferred)
        return fail(HM_EINVAL, "hm_eval_points: assembled with HM_DEFER_ACA (use hm_amvm with HM_AMVM_ACA_ON_DEMAND)");
    if (nrhs < 1) return fail(HM_EINVAL, "hm_eval_points: nrhs %d < 1", nrhs);
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

// ------------------------------------------------------------------------
// Algorithm 3 (block-adaptive ACA, Section 5) restricted to the single
// layer: restarted GMRES on A_k (a product of the passes above with the
// prefix ranks r_b of every block-kernel), the look-ahead parts by the
// adaptive product's part kernel, Doerfler marking of the blocks with the
// fewest blocks, refinement by `look` crosses.  Vectors live in cluster
// order (3 values per position) during the solve.
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

extern "C" int hm_baca(const hm_matrix* H, const double* b, double* x, const hm_baca_params* prm, hm_baca_info* info,
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
    hm_matrix& Hm = const_cast<hm_matrix&>(*H);  // the product tables are built once and kept
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
