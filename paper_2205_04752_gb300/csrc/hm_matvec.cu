// hm_matvec.cu -- H-matrix-vector product y = V_h x on the device.
//
// Section 2: an admissible block t x s stored as U V^T is applied as U (V^T x_s)
// at O(k(|t|+|s|)) cost, a near block by its dense entries; the results of all
// blocks of a row are summed into y.  With Eq. (Vh),
//   y_a(t) += c1 U_Delta (V_Delta^T x_a(s)) + c2 sum_b U_ab (V_ab^T x_b(s)).
//
// Three launches, all stream ordered and deterministic (fixed summation order,
// no atomics):
//   1. gather   x (original dof order) -> xg[r][a][p] (cluster order, SoA)
//   2. far_fwd  one CTA per admissible block: w = coefficient * V^T xg, i.e.
//               for every kernel and column l the three values that multiply
//               column l of U for the outputs a = 0, 1, 2
//   3. leaf     one CTA per leaf row cluster tau: for every row i of tau,
//               sum over all admissible blocks t x s with t containing tau of
//               U[i, :] . w(a) plus its near blocks' dense rows, then the
//               scatter to the original dof order.
// Forms: FP64 (factors, near field, accumulation); FP32; BF16 / FP16 factors
// with one FP32 scale per factor column (folded into w) and an FP32 near field.
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include <algorithm>
#include <cmath>

#include "hm_internal.h"

namespace hm {
namespace {

template <class T>
__device__ __forceinline__ float to_f(T v);
template <>
__device__ __forceinline__ float to_f<float>(float v) { return v; }
template <>
__device__ __forceinline__ float to_f<__nv_bfloat16>(__nv_bfloat16 v) { return __bfloat162float(v); }
template <>
__device__ __forceinline__ float to_f<__half>(__half v) { return __half2float(v); }

template <class TF, class TA>
__device__ __forceinline__ TA load_f(const TF* p)
{
    return (TA)to_f<TF>(*p);
}
template <>
__device__ __forceinline__ double load_f<double, double>(const double* p) { return __ldg(p); }

// kernel -> (p, q) component pair; kernel 0 is V_Delta
__device__ __forceinline__ void kern_pq(int kern, int& p, int& q)
{
    p = kern == 0 ? -1 : (kern <= 3 ? 0 : (kern <= 5 ? 1 : 2));
    q = kern == 0 ? -1 : (kern <= 3 ? kern - 1 : (kern <= 5 ? kern - 3 : 2));
}

template <class TA>
__global__ void gather_kernel(int M, int nrhs, const double* __restrict__ x, int64_t ld,
                              const int32_t* __restrict__ perm, TA* __restrict__ xg)
{
    int p = blockIdx.x * blockDim.x + threadIdx.x;
    int r = blockIdx.y;
    if (p >= M || r >= nrhs) return;
    size_t src = (size_t)r * ld + 3 * (size_t)perm[p];
#pragma unroll
    for (int a = 0; a < 3; ++a) xg[((size_t)r * 3 + a) * M + p] = (TA)x[src + a];
}

template <class TA>
__device__ __forceinline__ TA warp_sum(TA v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

constexpr int kFwdThreads = 128;

// Phase 1: one CTA per admissible block (largest first); warp w takes the
// block's factor columns c = w, w + 4, ... (all seven kernels concatenated).
template <class TF, class TA, int RC>
__global__ void __launch_bounds__(kFwdThreads) far_fwd_kernel(
    const int32_t* __restrict__ order, const Blk* __restrict__ blks, const int32_t* __restrict__ rank,
    const int64_t* __restrict__ voff, const int64_t* __restrict__ woff,
    const int64_t* __restrict__ coff, const TF* __restrict__ V, const float* __restrict__ SU,
    const float* __restrict__ SV, const TA* __restrict__ xg, TA* __restrict__ w, int M, int nrhs,
    int64_t wtot, TA c1, TA c2)
{
    const int b = order[blockIdx.x];
    const Blk bk = blks[b];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int nw = blockDim.x >> 5;
    int kk[7];
    int ctot = 0;
#pragma unroll
    for (int k = 0; k < 7; ++k) {
        kk[k] = rank[(size_t)b * 7 + k];
        ctot += kk[k];
    }
    for (int c = warp; c < ctot; c += nw) {
        int kern = 0, l = c;
        while (l >= kk[kern]) {
            l -= kk[kern];
            ++kern;
        }
        const size_t q = (size_t)b * 7 + kern;
        const int k = kk[kern];
        const TF* v = V + voff[q] + (size_t)l * bk.n;
        const TA sv = SV ? (TA)SV[coff[q] + l] : (TA)1;
        const TA su = SU ? (TA)SU[coff[q] + l] : (TA)1;
        int p, pq;
        kern_pq(kern, p, pq);
        for (int r0 = 0; r0 < nrhs; r0 += RC) {
            TA z[RC][3];
#pragma unroll
            for (int rr = 0; rr < RC; ++rr) z[rr][0] = z[rr][1] = z[rr][2] = (TA)0;
            for (int j = lane; j < bk.n; j += 32) {
                TA vj = load_f<TF, TA>(v + j);
#pragma unroll
                for (int rr = 0; rr < RC; ++rr) {
                    if (r0 + rr < nrhs) {
                        const TA* xr = xg + (size_t)(r0 + rr) * 3 * M + bk.s0 + j;
                        z[rr][0] += vj * xr[0];
                        z[rr][1] += vj * xr[M];
                        z[rr][2] += vj * xr[2 * (size_t)M];
                    }
                }
            }
#pragma unroll
            for (int rr = 0; rr < RC; ++rr) {
                if (r0 + rr >= nrhs) break;
                TA z0 = warp_sum(z[rr][0]) * sv, z1 = warp_sum(z[rr][1]) * sv,
                   z2 = warp_sum(z[rr][2]) * sv;
                if (lane == 0) {
                    TA* wo = w + (size_t)(r0 + rr) * wtot + woff[q];
                    TA o[3];
                    if (kern == 0) {
                        o[0] = c1 * su * z0;
                        o[1] = c1 * su * z1;
                        o[2] = c1 * su * z2;
                    } else {
                        TA zz[3] = {z0, z1, z2};
                        o[0] = o[1] = o[2] = (TA)0;
                        o[p] = c2 * su * zz[pq];
                        if (p != pq) o[pq] = c2 * su * zz[p];
                    }
                    wo[l] = o[0];
                    wo[k + l] = o[1];
                    wo[2 * k + l] = o[2];
                }
            }
        }
    }
}

// Phase 2 (+ near field): one CTA per leaf.  Thread (i, h): row i of the leaf,
// group h of H = blockDim / |tau| groups; the groups split the factor columns
// and near-block columns round robin and are summed at the end.
template <class TF, class TN, class TA, int RC>
__global__ void leaf_kernel(const int32_t* __restrict__ leaf, const int32_t* __restrict__ far_ptr,
                            const FarItem* __restrict__ far_items, const int32_t* __restrict__ near_ptr,
                            const int32_t* __restrict__ near_items, const Blk* __restrict__ adm,
                            const Blk* __restrict__ nearb, const int32_t* __restrict__ rank,
                            const int64_t* __restrict__ uoff, const int64_t* __restrict__ woff,
                            const int64_t* __restrict__ noff, const TF* __restrict__ U,
                            const TN* __restrict__ N, const TA* __restrict__ xg,
                            const TA* __restrict__ w, const int32_t* __restrict__ perm,
                            double* __restrict__ y, int64_t ld, int M, int nrhs, int64_t wtot,
                            TA c1, TA c2)
{
    extern __shared__ unsigned char smem_raw[];
    TA* red = reinterpret_cast<TA*>(smem_raw);
    const int lf = blockIdx.x;
    const int t0 = leaf[2 * lf], mt = leaf[2 * lf + 1];
    const int H = blockDim.x / mt;
    const int i = threadIdx.x % mt, h = threadIdx.x / mt;
    const bool active = h < H;
    const int f0 = far_ptr[lf], f1 = far_ptr[lf + 1];
    const int n0 = near_ptr[lf], n1 = near_ptr[lf + 1];
    for (int r0 = 0; r0 < nrhs; r0 += RC) {
        const int rc = min(RC, nrhs - r0);
        TA acc[RC][3];
#pragma unroll
        for (int rr = 0; rr < RC; ++rr) acc[rr][0] = acc[rr][1] = acc[rr][2] = (TA)0;
        if (active) {
            int rot = 0;  // global column counter mod H
            for (int it = f0; it < f1; ++it) {
                const FarItem fi = far_items[it];
                const int m = adm[fi.b].m;
#pragma unroll 1
                for (int kern = 0; kern < 7; ++kern) {
                    const size_t q = (size_t)fi.b * 7 + kern;
                    const int k = rank[q];
                    if (k == 0) continue;
                    const TF* ub = U + uoff[q] + fi.off + i;
                    const TA* wb = w + woff[q];
                    int l = h - rot;
                    l = ((l % H) + H) % H;
                    for (; l < k; l += H) {
                        const TA u = load_f<TF, TA>(ub + (size_t)l * m);
#pragma unroll
                        for (int rr = 0; rr < RC; ++rr) {
                            if (rr < rc) {
                                const TA* wr = wb + (size_t)(r0 + rr) * wtot;
                                acc[rr][0] += u * wr[l];
                                acc[rr][1] += u * wr[k + l];
                                acc[rr][2] += u * wr[2 * k + l];
                            }
                        }
                    }
                    rot = (rot + k) % H;
                }
            }
            for (int it = n0; it < n1; ++it) {
                const int nb = near_items[it];
                const Blk bk = nearb[nb];
                const int n = bk.n;
                const size_t pairs = (size_t)mt * n;
                const TN* Nb = N + noff[nb] + i;
                int j = h - rot;
                j = ((j % H) + H) % H;
                for (; j < n; j += H) {
                    const TN* e = Nb + (size_t)j * mt;
                    const TA v11 = (TA)e[0], v12 = (TA)e[pairs], v13 = (TA)e[2 * pairs];
                    const TA v22 = (TA)e[3 * pairs], v23 = (TA)e[4 * pairs], v33 = (TA)e[5 * pairs];
                    const TA vd = c1 * (v11 + v22 + v33);
#pragma unroll
                    for (int rr = 0; rr < RC; ++rr) {
                        if (rr < rc) {
                            const TA* xr = xg + (size_t)(r0 + rr) * 3 * M + bk.s0 + j;
                            const TA x0 = xr[0], x1 = xr[M], x2 = xr[2 * (size_t)M];
                            acc[rr][0] += vd * x0 + c2 * (v11 * x0 + v12 * x1 + v13 * x2);
                            acc[rr][1] += vd * x1 + c2 * (v12 * x0 + v22 * x1 + v23 * x2);
                            acc[rr][2] += vd * x2 + c2 * (v13 * x0 + v23 * x1 + v33 * x2);
                        }
                    }
                }
                rot = (rot + n) % H;
            }
        }
        // sum the H partial results of every row in a fixed order
        __syncthreads();
        if (active) {
#pragma unroll
            for (int rr = 0; rr < RC; ++rr)
#pragma unroll
                for (int a = 0; a < 3; ++a) red[((size_t)(rr * 3 + a) * H + h) * mt + i] = acc[rr][a];
        }
        __syncthreads();
        if (active && h == 0) {
            const size_t dst = 3 * (size_t)perm[t0 + i];
            for (int rr = 0; rr < rc; ++rr)
#pragma unroll
                for (int a = 0; a < 3; ++a) {
                    TA s = (TA)0;
                    for (int g = 0; g < H; ++g) s += red[((size_t)(rr * 3 + a) * H + g) * mt + i];
                    y[(size_t)(r0 + rr) * ld + dst + a] = (double)s;
                }
        }
    }
}

// ---------------------------------------------------------------- packing
template <class TO>
__global__ void convert_kernel(const double* __restrict__ src, TO* __restrict__ dst, size_t n)
{
    for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < n;
         e += (size_t)gridDim.x * blockDim.x)
        dst[e] = (TO)src[e];
}

template <class T16>
__device__ __forceinline__ T16 from_f(float v);
template <>
__device__ __forceinline__ __nv_bfloat16 from_f<__nv_bfloat16>(float v) { return __float2bfloat16_rn(v); }
template <>
__device__ __forceinline__ __half from_f<__half>(float v) { return __float2half_rn(v); }

// 16-bit factors with one scale per column: column / max|column|
template <class T16>
__global__ void pack16_kernel(int ntask, const Blk* __restrict__ blks, const int32_t* __restrict__ rank,
                              const int64_t* __restrict__ off, const int64_t* __restrict__ coff,
                              int rows_is_m, const double* __restrict__ src, T16* __restrict__ dst,
                              float* __restrict__ scale)
{
    const int q = blockIdx.x;
    if (q >= ntask) return;
    const int k = rank[q];
    const Blk bk = blks[q / 7];
    const int len = rows_is_m ? bk.m : bk.n;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
    for (int l = warp; l < k; l += nw) {
        const double* c = src + off[q] + (size_t)l * len;
        double mx = 0.0;
        for (int e = lane; e < len; e += 32) mx = fmax(mx, fabs(c[e]));
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
        const float sc = mx > 0.0 ? (float)mx : 1.0f;
        const double inv = 1.0 / (double)sc;
        T16* d = dst + off[q] + (size_t)l * len;
        for (int e = lane; e < len; e += 32) d[e] = from_f<T16>((float)(c[e] * inv));
        if (lane == 0) scale[coff[q] + l] = sc;
    }
}

int dalloc(hm_matrix& H, DevBuf& d, size_t bytes)
{
    d.bytes = bytes;
    d.p = H.alloc.alloc(bytes);
    if (!d.p) return fail(HM_ENOMEM, "device allocation of %zu bytes failed", bytes);
    return HM_OK;
}

template <class TF, class TN, class TA>
int run_matvec(const hm_matrix& H, const TF* U, const TF* V, const TN* N, const float* SU,
               const float* SV, const double* x, double* y, int nrhs, int64_t ld, cudaStream_t s,
               const Scratch& scr)
{
    const int M = (int)H.M;
    TA* xg = static_cast<TA*>(scr.xg);
    TA* w = static_cast<TA*>(scr.w);
    const TA c1 = (TA)((1.0 + H.nu) * (3.0 - 4.0 * H.nu) / (2.0 * H.E * (1.0 - H.nu)));
    const TA c2 = (TA)((1.0 + H.nu) / (2.0 * H.E * (1.0 - H.nu)));
    dim3 gg((unsigned)((M + 255) / 256), (unsigned)nrhs);
    if (scr.profile) prof_mark(H, 0, s);
    gather_kernel<TA><<<gg, 256, 0, s>>>(M, nrhs, x, ld, H.d_perm.as<int32_t>(), xg);
    HM_CUDA(cudaGetLastError());
    const bool multi = nrhs > 1;
    if (scr.profile) prof_mark(H, 1, s);
    if (H.nadm > 0) {
        if (multi)
            far_fwd_kernel<TF, TA, 4><<<(unsigned)H.nadm, kFwdThreads, 0, s>>>(
                H.d_p1_order.as<int32_t>(), H.d_adm.as<Blk>(), H.d_rank.as<int32_t>(),
                H.d_voff.as<int64_t>(), H.d_woff.as<int64_t>(), H.d_coff.as<int64_t>(), V, SU, SV, xg, w,
                M, nrhs, H.w_total, c1, c2);
        else
            far_fwd_kernel<TF, TA, 1><<<(unsigned)H.nadm, kFwdThreads, 0, s>>>(
                H.d_p1_order.as<int32_t>(), H.d_adm.as<Blk>(), H.d_rank.as<int32_t>(),
                H.d_voff.as<int64_t>(), H.d_woff.as<int64_t>(), H.d_coff.as<int64_t>(), V, SU, SV, xg, w,
                M, nrhs, H.w_total, c1, c2);
        HM_CUDA(cudaGetLastError());
    }
    if (scr.profile) prof_mark(H, 2, s);
    int bdim = H.max_leaf <= 128 ? 128 : ((H.max_leaf + 31) / 32) * 32;
    const int RCm = multi ? 4 : 1;
    size_t smem = (size_t)RCm * 3 * bdim * sizeof(TA);
    if (multi)
        leaf_kernel<TF, TN, TA, 4><<<(unsigned)H.nleaves, bdim, smem, s>>>(
            H.d_leaf.as<int32_t>(), H.d_far_ptr.as<int32_t>(), H.d_far_items.as<FarItem>(),
            H.d_near_ptr.as<int32_t>(), H.d_near_items.as<int32_t>(), H.d_adm.as<Blk>(),
            H.d_near.as<Blk>(), H.d_rank.as<int32_t>(), H.d_uoff.as<int64_t>(), H.d_woff.as<int64_t>(),
            H.d_noff.as<int64_t>(), U, N, xg, w, H.d_perm.as<int32_t>(), y, ld, M, nrhs, H.w_total, c1, c2);
    else
        leaf_kernel<TF, TN, TA, 1><<<(unsigned)H.nleaves, bdim, smem, s>>>(
            H.d_leaf.as<int32_t>(), H.d_far_ptr.as<int32_t>(), H.d_far_items.as<FarItem>(),
            H.d_near_ptr.as<int32_t>(), H.d_near_items.as<int32_t>(), H.d_adm.as<Blk>(),
            H.d_near.as<Blk>(), H.d_rank.as<int32_t>(), H.d_uoff.as<int64_t>(), H.d_woff.as<int64_t>(),
            H.d_noff.as<int64_t>(), U, N, xg, w, H.d_perm.as<int32_t>(), y, ld, M, nrhs, H.w_total, c1, c2);
    HM_CUDA(cudaGetLastError());
    if (scr.profile) prof_mark(H, 3, s);
    return HM_OK;
}

}  // namespace

int matvec_device_scratch(const hm_matrix& H, const double* x, double* y, int32_t nrhs, int64_t ld,
                          int32_t form, cudaStream_t s, const Scratch& scr)
{
    switch (form) {
        case HM_FP64:
            return run_matvec<double, double, double>(H, H.U64.as<double>(), H.V64.as<double>(),
                                                      H.N64.as<double>(), nullptr, nullptr, x, y,
                                                      nrhs, ld, s, scr);
        case HM_FP32:
            return run_matvec<float, float, float>(H, H.U32.as<float>(), H.V32.as<float>(),
                                                   H.N32.as<float>(), nullptr, nullptr, x, y, nrhs,
                                                   ld, s, scr);
        case HM_BF16:
            return run_matvec<__nv_bfloat16, float, float>(
                H, H.U16b.as<__nv_bfloat16>(), H.V16b.as<__nv_bfloat16>(), H.N32.as<float>(),
                H.SUb.as<float>(), H.SVb.as<float>(), x, y, nrhs, ld, s, scr);
        case HM_FP16:
            return run_matvec<__half, float, float>(H, H.U16h.as<__half>(), H.V16h.as<__half>(),
                                                    H.N32.as<float>(), H.SUh.as<float>(),
                                                    H.SVh.as<float>(), x, y, nrhs, ld, s, scr);
        default:
            return fail(HM_EINVAL, "hm_matvec: unknown form %d", form);
    }
}

int matvec_device(const hm_matrix& H, const double* x, double* y, int32_t nrhs, int64_t ld,
                  int32_t form, cudaStream_t s)
{
    Scratch scr{H.xg.p, H.wb.p, true};
    return matvec_device_scratch(H, x, y, nrhs, ld, form, s, scr);
}

size_t matvec_scratch_bytes(const hm_matrix& H, int32_t nrhs, int32_t form)
{
    size_t ta = form == HM_FP64 ? 8 : 4;
    size_t xg = ((size_t)nrhs * 3 * (size_t)H.M * ta + 255) & ~(size_t)255;
    size_t w = (size_t)nrhs * (size_t)std::max<int64_t>(H.w_total, 1) * ta;
    return xg + w;
}

int pack_device(hm_matrix& H, int32_t form, cudaStream_t s)
{
    int rc;
    const int ntask = (int)(H.nadm * 7);
    auto convert = [&](const DevBuf& src, DevBuf& dst, int64_t n) -> int {
        if ((rc = dalloc(H, dst, (size_t)std::max<int64_t>(n, 1) * 4))) return rc;
        if (n > 0) {
            convert_kernel<float><<<1216, 256, 0, s>>>(src.as<double>(), dst.as<float>(), (size_t)n);
            HM_CUDA(cudaGetLastError());
        }
        return HM_OK;
    };
    if (!H.N32.p && form != HM_FP64)
        if ((rc = convert(H.N64, H.N32, H.n_total))) return rc;
    if (form == HM_FP32) {
        if ((rc = convert(H.U64, H.U32, H.u_total))) return rc;
        if ((rc = convert(H.V64, H.V32, H.v_total))) return rc;
    } else if (form == HM_BF16 || form == HM_FP16) {
        DevBuf &Ud = form == HM_BF16 ? H.U16b : H.U16h, &Vd = form == HM_BF16 ? H.V16b : H.V16h;
        DevBuf &Su = form == HM_BF16 ? H.SUb : H.SUh, &Sv = form == HM_BF16 ? H.SVb : H.SVh;
        if ((rc = dalloc(H, Ud, (size_t)std::max<int64_t>(H.u_total, 1) * 2))) return rc;
        if ((rc = dalloc(H, Vd, (size_t)std::max<int64_t>(H.v_total, 1) * 2))) return rc;
        if ((rc = dalloc(H, Su, (size_t)std::max<int64_t>(H.c_total, 1) * 4))) return rc;
        if ((rc = dalloc(H, Sv, (size_t)std::max<int64_t>(H.c_total, 1) * 4))) return rc;
        if (ntask > 0) {
            if (form == HM_BF16) {
                pack16_kernel<__nv_bfloat16><<<ntask, 128, 0, s>>>(
                    ntask, H.d_adm.as<Blk>(), H.d_rank.as<int32_t>(), H.d_uoff.as<int64_t>(),
                    H.d_coff.as<int64_t>(), 1, H.U64.as<double>(), Ud.as<__nv_bfloat16>(), Su.as<float>());
                pack16_kernel<__nv_bfloat16><<<ntask, 128, 0, s>>>(
                    ntask, H.d_adm.as<Blk>(), H.d_rank.as<int32_t>(), H.d_voff.as<int64_t>(),
                    H.d_coff.as<int64_t>(), 0, H.V64.as<double>(), Vd.as<__nv_bfloat16>(), Sv.as<float>());
            } else {
                pack16_kernel<__half><<<ntask, 128, 0, s>>>(
                    ntask, H.d_adm.as<Blk>(), H.d_rank.as<int32_t>(), H.d_uoff.as<int64_t>(),
                    H.d_coff.as<int64_t>(), 1, H.U64.as<double>(), Ud.as<__half>(), Su.as<float>());
                pack16_kernel<__half><<<ntask, 128, 0, s>>>(
                    ntask, H.d_adm.as<Blk>(), H.d_rank.as<int32_t>(), H.d_voff.as<int64_t>(),
                    H.d_coff.as<int64_t>(), 0, H.V64.as<double>(), Vd.as<__half>(), Sv.as<float>());
            }
            HM_CUDA(cudaGetLastError());
        }
    }
    return HM_OK;
}

}  // namespace hm

using namespace hm;

extern "C" {

int hm_pack(hm_matrix* H, int32_t form, void* stream)
{
    if (!H) return fail(HM_EINVAL, "hm_pack: NULL matrix");
    if (form < HM_FP64 || form > HM_FP16) return fail(HM_EINVAL, "hm_pack: unknown form %d", form);
    if (H->packed[form]) return HM_OK;
    cudaStream_t s = (cudaStream_t)stream;
    cudaStream_t saved = H->alloc.stream;
    H->alloc.stream = s;
    cudaEvent_t e0, e1;
    HM_CUDA(cudaEventCreate(&e0));
    HM_CUDA(cudaEventCreate(&e1));
    cudaEventRecord(e0, s);
    int rc = pack_device(*H, form, s);
    cudaEventRecord(e1, s);
    H->alloc.stream = saved;
    if (rc == HM_OK) rc = cuda_check(cudaStreamSynchronize(s), "hm_pack");
    float ms = 0;
    if (rc == HM_OK) cudaEventElapsedTime(&ms, e0, e1);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (rc) return rc;
    H->asm_ms[2] += ms;
    H->packed[form] = true;
    return HM_OK;
}

int hm_matvec(const hm_matrix* H, const double* x, double* y, int32_t nrhs, int64_t ld, int32_t form,
              void* stream)
{
    if (!H || !x || !y) return fail(HM_EINVAL, "hm_matvec: NULL argument");
    if (nrhs < 1 || nrhs > H->max_rhs)
        return fail(HM_EINVAL, "hm_matvec: nrhs=%d outside 1..%d", nrhs, H->max_rhs);
    if (ld < 3 * H->M) return fail(HM_EINVAL, "hm_matvec: ld=%lld < 3M=%lld", (long long)ld, (long long)(3 * H->M));
    if (form < HM_FP64 || form > HM_FP16) return fail(HM_EINVAL, "hm_matvec: unknown form %d", form);
    if (!H->packed[form]) return fail(HM_EINVAL, "hm_matvec: form %d not packed (call hm_pack)", form);
    const char* xb = (const char*)x;
    const char* yb = (const char*)y;
    size_t span = ((size_t)(nrhs - 1) * ld + 3 * H->M) * sizeof(double);
    if (xb < yb + span && yb < xb + span) return fail(HM_EINVAL, "hm_matvec: x and y overlap");
    return matvec_device(*H, x, y, nrhs, ld, form, (cudaStream_t)stream);
}

int hm_matvec_host(const hm_matrix* H, const double* x_host, double* y_host, int32_t nrhs, int64_t ld,
                   int32_t form, void* stream)
{
    if (!H || !x_host || !y_host) return fail(HM_EINVAL, "hm_matvec_host: NULL argument");
    if (nrhs < 1 || nrhs > H->max_rhs)
        return fail(HM_EINVAL, "hm_matvec_host: nrhs=%d outside 1..%d", nrhs, H->max_rhs);
    if (ld < 3 * H->M) return fail(HM_EINVAL, "hm_matvec_host: ld too small");
    if (!H->xh.p || !H->yh.p) return fail(HM_EINVAL, "hm_matvec_host: no staging buffers");
    cudaStream_t s = (cudaStream_t)stream;
    const int64_t n3 = 3 * H->M;
    HM_CUDA(cudaMemcpy2DAsync(H->xh.p, (size_t)n3 * 8, x_host, (size_t)ld * 8, (size_t)n3 * 8, (size_t)nrhs,
                              cudaMemcpyHostToDevice, s));
    int rc = hm_matvec(H, H->xh.as<double>(), H->yh.as<double>(), nrhs, n3, form, stream);
    if (rc) return rc;
    HM_CUDA(cudaMemcpy2DAsync(y_host, (size_t)ld * 8, H->yh.p, (size_t)n3 * 8, (size_t)n3 * 8, (size_t)nrhs,
                              cudaMemcpyDeviceToHost, s));
    HM_CUDA(cudaStreamSynchronize(s));
    return HM_OK;
}

}  // extern "C"
