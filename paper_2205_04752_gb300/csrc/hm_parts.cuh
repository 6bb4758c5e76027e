// hm_parts.cuh -- device kernels and host helpers shared by the FP64 block
// products outside the streamed H-matrix-vector product: the adaptive product
// (hm_amvm.cu), the evaluation operator (hm_eval.cu) and block-adaptive ACA
// (hm_baca.cu).  Everything sits in an unnamed namespace: each translation
// unit that includes this header compiles its own copy of what it uses.
//
// Block parts: the crosses l0 .. l1 - 1 of an admissible block applied to
// x(s) give |t| x 3 values (component fastest) at an offset of a part arena;
// the row sums add, for every row position, the parts of the blocks whose row
// cluster holds it, in block order (deterministic).
#pragma once

#include <algorithm>
#include <cmath>
#include <cstring>
#include <map>
#include <numeric>
#include <vector>

#include "hm_internal.h"

#if defined(__CUDACC__)
#pragma nv_diag_suppress 177  // a unit need not launch every shared kernel
#endif

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

template <class T>
__global__ void ev_scatter_add_kernel(const int32_t* __restrict__ perm, const T* __restrict__ yc,
                                      double* __restrict__ y, int64_t M)
{
    const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= M) return;
    const int64_t o = 3 * (int64_t)perm[p];
#pragma unroll
    for (int a = 0; a < 3; ++a) y[o + a] += (double)yc[3 * p + a];
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
    if (!d.p) {
        d.bytes = 0;
        return fail(HM_ENOMEM, "evaluation operator: device allocation of %zu bytes failed",
                    std::max<size_t>(n, 1) * sizeof(T));
    }
    if (!h.empty())
        HM_CUDA(cudaMemcpyAsync(d.p, h.data(), h.size() * sizeof(T), cudaMemcpyHostToDevice, H.alloc.stream));
    return HM_OK;
}
}  // namespace
}  // namespace hm
