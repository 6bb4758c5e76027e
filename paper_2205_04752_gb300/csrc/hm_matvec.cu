// hm_matvec.cu -- H-matrix-vector product y = V_h x on the device.
//
// Section 2: an admissible block t x s stored as U V^T is applied as U (V^T x_s)
// at O(k(|t|+|s|)) cost, a near block by its dense entries; the results of all
// blocks of a row are summed into y.  With Eq. (Vh),
//   y_a(t) += c1 U_Delta (V_Delta^T x_a(s)) + c2 sum_b U_ab (V_ab^T x_b(s)).
//
// The product is memory bound: every stored factor and near-field value is
// read once per product.  The factors are therefore stored in the order the
// kernels stream them (built once by pack_device):
//   V  per admissible block, row-major |s| x Cp (all seven kernels' columns
//      side by side, Cp = sum k rounded up to 8): 16-byte loads along a row;
//   U  per leaf row cluster tau, one contiguous stream of segments (a segment
//      is one column of U restricted to the rows of tau, padded to a multiple
//      of 8) over all admissible blocks t x s with t containing tau;
//   near field per leaf, one contiguous stream: for each near block and
//      column j, six segments (V_11, V_12, V_13, V_22, V_23, V_33).
// The product runs over a Plan: one or more meshes (a single matrix is a plan
// over one mesh), each with its own streams, tables and material
// coefficients, whose vectors sit side by side in shared x / y rows.  Three
// phases, stream ordered and deterministic (fixed summation order, no
// floating-point atomics):
//   1. gather   x (original dof order) -> xg[r][p][a] (cluster order of every
//               mesh, a padded to 4)
//   2. fwd      one CTA per admissible block with |s| > 128, one warp per
//               smaller block: z = V^T xg, and for every factor column c the
//               three values w[c][a] that multiply column c of U for output
//               component a (c1, c2 and the column scale folded in)
//   3. leaf     persistent CTAs take (mesh, leaf) items from a counter and
//               stream the leaf's U and near field through shared memory
//               (hm_stream.cuh), sum U w and the dense near rows in a fixed
//               order and scatter y to the original dof order.
// Forms: FP64 (factors, near field, accumulation); FP32; BF16 / FP16 factors
// with one FP32 scale per factor column (folded into w) and an FP32 near field.
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include <algorithm>
#include <cstring>
#include <cmath>

#include <type_traits>

#include "hm_internal.h"
#include "hm_stream.cuh"
#include "hm_leaf_tc.cuh"

namespace hm {
namespace {



// ---------------------------------------------------------------- 16-byte loads
// load N = 16 / sizeof(T) consecutive values (16-byte aligned, streaming) as TA
template <class T, class TA>
struct Vec16;

template <class TA>
struct Vec16<double, TA> {
    static constexpr int N = 2;
    __device__ __forceinline__ static void load(const double* p, TA* o)
    {
        double2 v = __ldcs(reinterpret_cast<const double2*>(p));
        o[0] = (TA)v.x;
        o[1] = (TA)v.y;
    }
};
template <class TA>
struct Vec16<float, TA> {
    static constexpr int N = 4;
    __device__ __forceinline__ static void load(const float* p, TA* o)
    {
        float4 v = __ldcs(reinterpret_cast<const float4*>(p));
        o[0] = (TA)v.x;
        o[1] = (TA)v.y;
        o[2] = (TA)v.z;
        o[3] = (TA)v.w;
    }
};
template <class TA>
struct Vec16<__half, TA> {
    static constexpr int N = 8;
    __device__ __forceinline__ static void load(const __half* p, TA* o)
    {
        uint4 v = __ldcs(reinterpret_cast<const uint4*>(p));
        const __half2* h = reinterpret_cast<const __half2*>(&v);
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            float2 f = __half22float2(h[q]);
            o[2 * q] = (TA)f.x;
            o[2 * q + 1] = (TA)f.y;
        }
    }
};
template <class TA>
struct Vec16<__nv_bfloat16, TA> {
    static constexpr int N = 8;
    __device__ __forceinline__ static void load(const __nv_bfloat16* p, TA* o)
    {
        uint4 v = __ldcs(reinterpret_cast<const uint4*>(p));
        const __nv_bfloat162* h = reinterpret_cast<const __nv_bfloat162*>(&v);
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            float2 f = __bfloat1622float2(h[q]);
            o[2 * q] = (TA)f.x;
            o[2 * q + 1] = (TA)f.y;
        }
    }
};

template <class TA>
struct Vec16<int16_t, TA> {
    static constexpr int N = 8;
    __device__ __forceinline__ static void load(const int16_t* p, TA* o)
    {
        uint4 v = __ldcs(reinterpret_cast<const uint4*>(p));
        const uint32_t wv[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            float2 f = stream::i16x2_to_float2(wv[q]);
            o[2 * q] = (TA)f.x;
            o[2 * q + 1] = (TA)f.y;
        }
    }
};

// forms whose several-vector launches run on the tensor cores (tcgen05
// kind::f16 operands): FP16 and BF16 factors as stored, INT16 factors split
// in shared memory into two exact FP16 operands
template <class TF>
constexpr bool tc_form()
{
    return sizeof(TF) == 2;
}

// element offset of V[j, c] (c a multiple of 8 for the vector loads) in a
// forward group of n rows and Cs columns: row-major for FP64 / FP32; for the
// 16-bit forms the group is cut into the units of the forward pass (rows
// 256 k .., columns 256 m ..), each unit stored contiguously in 8 x 8 tiles
// (row j / 8, column c / 8 of the unit), the units of a row chunk side by
// side: one stage of 32 rows of a unit is one contiguous range, the operand
// layout of the tensor cores
template <class TF>
__device__ __forceinline__ size_t vel(int j, int c, int Cs, int n)
{
    if constexpr (sizeof(TF) == 2) {
        const int k = j >> 8, jl = j & 255, c0 = c & ~255, cl = c & 255;
        const int cu = min(256, Cs - c0), n16 = (min(256, n - (k << 8)) + 15) & ~15;
        return (size_t)k * 256 * (size_t)Cs + (size_t)n16 * c0 +
               ((size_t)(jl >> 3) * (size_t)(cu >> 3) + (size_t)(cl >> 3)) * 64 + (size_t)(jl & 7) * 8 + (cl & 7);
    } else {
        return (size_t)j * (size_t)Cs + (size_t)c;
    }
}

// R consecutive values of type T (R * sizeof(T) a multiple of 16)
template <class T, class TA, int R>
__device__ __forceinline__ void load_rows(const T* p, TA* o)
{
    constexpr int N = Vec16<T, TA>::N;
#pragma unroll
    for (int q = 0; q < R / N; ++q) Vec16<T, TA>::load(p + q * N, o + q * N);
}

// x and w are stored as 4-vectors (the 4th entry is zero): one position of x
// (components 0..2) or one factor column of w (outputs 0..2) per 16 bytes
// (FP32) or 32 bytes (FP64)
__device__ __forceinline__ void load3(const float* p, float& a, float& b, float& c)
{
    const float4 v = *reinterpret_cast<const float4*>(p);
    a = v.x;
    b = v.y;
    c = v.z;
}
__device__ __forceinline__ void load3(const double* p, double& a, double& b, double& c)
{
    const double2 v = *reinterpret_cast<const double2*>(p);
    a = v.x;
    b = v.y;
    c = p[2];
}

// kernel -> (p, q) component pair; kernel 0 is V_Delta
__device__ __forceinline__ void kern_pq(int kern, int& p, int& q)
{
    p = kern == 0 ? -1 : (kern <= 3 ? 0 : (kern <= 5 ? 1 : 2));
    q = kern == 0 ? -1 : (kern <= 3 ? kern - 1 : (kern <= 5 ? kern - 3 : 2));
}

// mesh of cluster position p of the product: the largest m with pos_prefix[m] <= p
__device__ __forceinline__ int mesh_of(const int64_t* __restrict__ pos_prefix, int nmesh, int64_t p)
{
    int lo = 0, hi = nmesh - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (pos_prefix[mid] <= p) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

// x (original dof order of every mesh) -> xg[p][r][a] (cluster order, G
// right-hand sides interleaved, a padded to 4).  With xmax (G <= 32), also
// max |xg| of each vector, as the bits of a non-negative float (ordered like
// the values), for the power-of-two scales of the tensor-core kernels.
template <class TA>
__global__ void gather_kernel(const MeshDev* __restrict__ meshes, int nmesh, const int64_t* __restrict__ pos_prefix,
                              int64_t npos, const double* __restrict__ x, int64_t ld, TA* __restrict__ xg, int G,
                              int* __restrict__ xmax)
{
    const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const bool in = idx < npos * G;
    const int64_t p = idx / G;
    const int r = (int)(idx - p * G);
    float mx = 0.0f;
    if (in) {
        const int m = mesh_of(pos_prefix, nmesh, p);
        const MeshDev& md = meshes[m];
        const size_t src = (size_t)r * ld + md.xoff + 3 * (size_t)md.perm[p - pos_prefix[m]];
        TA* d = xg + (size_t)idx * 4;
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            const TA v = (TA)x[src + a];
            d[a] = v;
            mx = fmaxf(mx, fabsf((float)v));
        }
        d[3] = (TA)0;
    }
    if (xmax == nullptr) return;
    __shared__ int smx[32];
    if (threadIdx.x < 32) smx[threadIdx.x] = 0;
    __syncthreads();
    if (in && mx > 0.0f) atomicMax(&smx[r], __float_as_int(mx));
    __syncthreads();
    if ((int)threadIdx.x < G && smx[threadIdx.x] > 0) atomicMax(xmax + threadIdx.x, smx[threadIdx.x]);
}

// ---------------------------------------------------------------- phase 1
// w for every factor column c of block `rec` from its reduced z = V^T x
// (three components), with c1 / c2 and the column scale of U folded in
template <class TA>
__device__ __forceinline__ void write_w(const FwdRec& rec, int c, TA z0, TA z1, TA z2, const float* __restrict__ SU,
                                        TA* __restrict__ wr, TA c1, TA c2, int G, int r)
{
    int kern = 0, l = c;
    for (;;) {
        const int k = (int)((rec.kpack >> (8 * kern)) & 0xff);
        if (l < k) break;
        l -= k;
        ++kern;
    }
    const int64_t col = (int64_t)rec.col0 + c;
    const TA su = SU ? (TA)SU[col] : (TA)1;
    TA o[3];
    if (kern == 0) {
        const TA f = c1 * su;
        o[0] = f * z0;
        o[1] = f * z1;
        o[2] = f * z2;
    } else {
        // V_pq enters y_p with x_q and (p != q) y_q with x_p; selects keep
        // everything in registers
        int p, pq;
        kern_pq(kern, p, pq);
        const TA f = c2 * su;
        const TA zp = p == 0 ? z0 : (p == 1 ? z1 : z2);
        const TA zq = pq == 0 ? z0 : (pq == 1 ? z1 : z2);
#pragma unroll
        for (int a = 0; a < 3; ++a) o[a] = a == p ? f * zq : (a == pq ? f * zp : (TA)0);
    }
    TA* d = wr + ((size_t)col * G + r) * 4;
    d[0] = o[0];
    d[1] = o[1];
    d[2] = o[2];
    d[3] = (TA)0;
}

// ---------------------------------------------------------------- forward groups
// z = V^T x for every admissible block, a group of blocks that share the
// column cluster s at a time (their V side by side, one n x Cs row-major
// matrix), so that x(s) is read once per group.  One CTA per group.  The work
// is the pairs (column vector q = VEC consecutive columns, RHS chunk c of RC
// vectors); the T threads split the rows into GG groups and take the pairs in
// rounds of PR = T / GG (GG = T / pairs when the pairs are fewer than the
// threads).  x(s) is staged in shared memory kFwdRows rows at a time; V is
// read once, 16 bytes per row and column vector.  The GG partial sums are
// added in a fixed order through shared memory, then w is written for every
// column (c1 / c2 and the U column scale folded in).  Deterministic.
constexpr int kFwdThreads = 128;
constexpr int kFwdXsBytes = 8192;

template <class TF, class TA, int RC, bool ONE>
__global__ void __launch_bounds__(kFwdThreads) fwd_group_kernel(
    const FwdUnit* __restrict__ units, const FwdGroup* __restrict__ groups, const FwdRec* __restrict__ recs,
    const __grid_constant__ MeshDev m0, const MeshDev* __restrict__ meshes, const TA* __restrict__ xg,
    TA* __restrict__ w, TA* __restrict__ z, int G)
{
    constexpr int VEC = Vec16<TF, TA>::N;
    constexpr int T = kFwdThreads;
    constexpr int kPer = VEC * RC * 3;
    __shared__ __align__(16) TA xs[kFwdXsBytes / sizeof(TA)];
    __shared__ __align__(16) TA red[T * kPer];
    __shared__ FwdRec srec[kMaxGroupRecs];
    const FwdUnit un = units[blockIdx.x];
    const FwdGroup gp = groups[un.group];
    const MeshDev& md = ONE ? m0 : meshes[gp.mesh];
    const int tid = threadIdx.x;
    for (int i = tid; i < gp.nrec; i += T) srec[i] = recs[gp.first + i];
    const TF* Vg = static_cast<const TF*>(md.Vr) + gp.vbase;
    const TA* x0 = xg + ((size_t)md.xgoff + gp.s0 + un.j0) * G * 4;
    TA* wr = w + (size_t)md.woff * G * 4;
    const float* SU = md.SU;
    const TA c1 = (TA)md.c1, c2 = (TA)md.c2;
    const int Cs = gp.Cs, n = un.nrows;
    const int Q = un.ncols / VEC;  // column vectors of this unit (from column un.c0)
    const int NRC = (G + RC - 1) / RC;
    const int pairs = Q * NRC;
    const int rows = max(1, (int)(kFwdXsBytes / sizeof(TA)) / (G * 4));  // x rows per staged chunk
    const int GG = pairs >= T ? 1 : min(T / pairs, rows);
    const int PR = T / GG;
    const int pl = tid % PR, g = tid / PR;
    __syncthreads();
    for (int pr0 = 0; pr0 < pairs; pr0 += PR) {
        const int nr = min(PR, pairs - pr0);
        const bool active = g < GG && pl < nr;
        const int pr = pr0 + pl;
        const int q = pr % Q, c = pr / Q;
        const int nq = min(RC, G - c * RC);
        TA acc[VEC][RC][3];
#pragma unroll
        for (int e = 0; e < VEC; ++e)
#pragma unroll
            for (int k = 0; k < RC; ++k) acc[e][k][0] = acc[e][k][1] = acc[e][k][2] = (TA)0;
        const int cq = un.c0 + q * VEC;
        for (int j0 = 0; j0 < n; j0 += rows) {
            const int nrows = min(rows, n - j0);
            __syncthreads();  // the previous chunk is consumed
            // stage x rows j0 .. j0 + nrows (4-vectors, G per row), 16 bytes a thread
            {
                constexpr int E16 = 16 / sizeof(TA);
                const int nv = nrows * G * 4 / E16;
                const uint4* src = reinterpret_cast<const uint4*>(x0 + (size_t)j0 * G * 4);
                uint4* dst = reinterpret_cast<uint4*>(xs);
                for (int e = tid; e < nv; e += T) dst[e] = src[e];
            }
            __syncthreads();
            if (active) {
#pragma unroll 4
                for (int jj = g; jj < nrows; jj += GG) {
                    TA v[VEC];
                    Vec16<TF, TA>::load(Vg + vel<TF>(un.j0 + j0 + jj, cq, Cs, gp.n), v);
                    const TA* xr = xs + ((size_t)jj * G + c * RC) * 4;
#pragma unroll
                    for (int k = 0; k < RC; ++k) {
                        if (RC > 1 && k >= nq) break;
                        TA xa, xb, xc;
                        load3(xr + k * 4, xa, xb, xc);
#pragma unroll
                        for (int e = 0; e < VEC; ++e) {
                            acc[e][k][0] += v[e] * xa;
                            acc[e][k][1] += v[e] * xb;
                            acc[e][k][2] += v[e] * xc;
                        }
                    }
                }
            }
        }
        // the partial sums of the GG row groups, in a fixed order
        if (GG > 1) {
            __syncthreads();
            if (active) {
                TA* rp = red + (size_t)(g * PR + pl) * kPer;
#pragma unroll
                for (int e = 0; e < VEC; ++e)
#pragma unroll
                    for (int k = 0; k < RC; ++k)
#pragma unroll
                        for (int a = 0; a < 3; ++a) rp[(e * RC + k) * 3 + a] = acc[e][k][a];
            }
            __syncthreads();
        }
        for (int idx = (GG > 1 ? tid : (active ? 0 : 1 << 30)); idx < (GG > 1 ? nr * VEC * RC : 1);
             idx += (GG > 1 ? T : 1)) {
            // GG == 1: this thread's own pair; GG > 1: (pair, column, vector) items
            const int pp = GG > 1 ? idx / (VEC * RC) : pl;
            const int q2 = (pr0 + pp) % Q + un.c0 / VEC, c2i = (pr0 + pp) / Q;
            // the block of column vector q2: the last record with offset <= q2 VEC
            int lo = 0, hi = gp.nrec - 1;
            while (lo < hi) {
                const int mid = (lo + hi + 1) >> 1;
                if (srec[mid].coff <= q2 * VEC) lo = mid;
                else hi = mid - 1;
            }
            const FwdRec& rec = srec[lo];
            const int cb0 = q2 * VEC - rec.coff;  // first column of the vector in the block
            // one-unit groups write w; the units of taller groups write their
            // partial sums for the second pass
            TA* zp = un.zcol0 >= 0 ? z + ((size_t)(un.zcol0 + (int64_t)un.chunk * Cs) * G) * 4 : nullptr;
            if (GG > 1) {
                const int rem = idx - pp * (VEC * RC);
                const int e = rem / RC, k = rem - e * RC;
                const int r = c2i * RC + k;
                if (cb0 + e >= rec.C || r >= G) continue;
                TA zz[3] = {(TA)0, (TA)0, (TA)0};
                for (int gg = 0; gg < GG; ++gg)
#pragma unroll
                    for (int a = 0; a < 3; ++a) zz[a] += red[(size_t)(gg * PR + pp) * kPer + (e * RC + k) * 3 + a];
                if (zp) {
                    TA* d = zp + ((size_t)(q2 * VEC + e) * G + r) * 4;
                    d[0] = zz[0];
                    d[1] = zz[1];
                    d[2] = zz[2];
                } else {
                    write_w<TA>(rec, cb0 + e, zz[0], zz[1], zz[2], SU, wr, c1, c2, G, r);
                }
            } else {
#pragma unroll
                for (int e = 0; e < VEC; ++e) {
                    if (cb0 + e >= rec.C) continue;
#pragma unroll
                    for (int k = 0; k < RC; ++k) {
                        if (k >= nq) break;
                        if (zp) {
                            TA* d = zp + ((size_t)(q2 * VEC + e) * G + c * RC + k) * 4;
                            d[0] = acc[e][k][0];
                            d[1] = acc[e][k][1];
                            d[2] = acc[e][k][2];
                        } else {
                            write_w<TA>(rec, cb0 + e, acc[e][k][0], acc[e][k][1], acc[e][k][2], SU, wr, c1, c2, G,
                                        c * RC + k);
                        }
                    }
                }
            }
        }
    }
}

constexpr int kThreads = 128;  // per-block forward kernels

// One vector, 16-bit forms: the forward pass of a unit on the CUDA cores.
// The unit's tiles are contiguous, so thread 0 streams them into shared
// memory in stages of 32 rows by bulk copies (two stages in flight per CTA,
// several CTAs per SM).  Lane (jr, qq) of warp w takes row jr of every 8-row
// core row of column vector q = 4 w + qq, so a warp reads four whole tiles
// (512 contiguous bytes); the eight partial sums of a column are added by a
// fixed butterfly and lane jr writes column 8 q + jr.  x of the unit's rows
// is staged in shared memory once.  Every wait is bounded; a CTA that gives
// up drains its copies in flight before it returns.
constexpr int kTile1Threads = 256;
constexpr int kTile1Rows = 32;
constexpr int kTile1Stage = kTile1Rows * kFwdUnitCols * 2;  // bytes of a stage (16-bit V)

template <class TF, bool ONE>
__global__ void __launch_bounds__(kTile1Threads) fwd_tile1_kernel(
    const FwdUnit* __restrict__ units, const FwdTcUnit* __restrict__ tcu, const FwdGroup* __restrict__ groups,
    const FwdRec* __restrict__ recs, const __grid_constant__ MeshDev m0, const MeshDev* __restrict__ meshes,
    const float* __restrict__ xg, float* __restrict__ w, float* __restrict__ z, int* __restrict__ err, int G, int r)
{
    __shared__ __align__(128) unsigned char vs[2][kTile1Stage];
    __shared__ float4 xs[kFwdUnitRows];
    __shared__ FwdRec srec[kMaxGroupRecs];
    __shared__ __align__(8) uint64_t vbar[2];
    const FwdTcUnit tu = tcu[blockIdx.x];
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31, jr = lane & 7;
    const int nrows = tu.nrows, n16 = (nrows + 15) & ~15, cu = tu.ncols, nq = cu >> 3;
    const int nst = (n16 + kTile1Rows - 1) / kTile1Rows;
    const MeshDev& md = ONE ? m0 : meshes[tu.mesh];
    const TF* Vu = static_cast<const TF*>(md.Vr) + tu.v0;
    // V is read once per product: evict it from L2 first (x and w stay)
    const uint64_t pol = stream::l2_evict_first_policy();
    auto issue = [&](int q) {
        const uint32_t bytes = (uint32_t)(min(kTile1Rows, n16 - q * kTile1Rows) * cu * 2);
        stream::mbar_arrive_expect_tx(&vbar[q & 1], bytes);
        stream::bulk_g2s_hint(vs[q & 1], Vu + (size_t)q * kTile1Rows * cu, bytes, &vbar[q & 1], pol);
    };
    if (tid == 0) {
        stream::mbar_init(&vbar[0], 1);
        stream::mbar_init(&vbar[1], 1);
        stream::mbar_fence_init();
        issue(0);
        if (nst > 1) issue(1);
    }
    const FwdUnit un = units[blockIdx.x];
    const FwdGroup gp = groups[un.group];
    for (int i = tid; i < gp.nrec; i += kTile1Threads) srec[i] = recs[gp.first + i];
    // vector r of the G interleaved ones: position p's 4-vector at p G + r
    const float4* xsrc = reinterpret_cast<const float4*>(xg) + (size_t)(md.xgoff + tu.x0) * G + r;
    for (int j = tid; j < n16; j += kTile1Threads)
        xs[j] = j < nrows ? xsrc[(size_t)j * G] : make_float4(0.f, 0.f, 0.f, 0.f);
    __syncthreads();
    const int q = 4 * warp + (lane >> 3);  // this lane's column vector
    float acc[8][3];
#pragma unroll
    for (int c = 0; c < 8; ++c) acc[c][0] = acc[c][1] = acc[c][2] = 0.0f;
    int failed = -1;  // the stage whose wait ran out
    for (int st = 0; st < nst; ++st) {
        const bool got = stream::mbar_wait(&vbar[st & 1], (uint32_t)(st >> 1) & 1u, err, 20, st);
        if (!__syncthreads_and(got ? 1 : 0)) {
            failed = st;
            break;
        }
        if (q < nq) {
            const int nkr = min(kTile1Rows, n16 - st * kTile1Rows) >> 3;
            const unsigned char* base = vs[st & 1];
#pragma unroll
            for (int kr = 0; kr < kTile1Rows / 8; ++kr) {
                if (kr >= nkr) break;
                float v[8];
                stream::Smem16<TF, float>::load(
                    reinterpret_cast<const TF*>(base) + ((size_t)(kr * nq + q) * 64 + jr * 8), v);
                const float4 x = xs[st * kTile1Rows + kr * 8 + jr];
#pragma unroll
                for (int c = 0; c < 8; ++c) {
                    acc[c][0] += v[c] * x.x;
                    acc[c][1] += v[c] * x.y;
                    acc[c][2] += v[c] * x.z;
                }
            }
        }
        __syncthreads();  // the stage is consumed
        if (tid == 0 && st + 2 < nst) issue(st + 2);
    }
    if (failed >= 0) {
        // the copies in flight (stages failed and failed + 1) land before the
        // CTA returns (bounded)
        if (tid == 0)
            for (int st = failed; st < min(nst, failed + 2); ++st)
                stream::mbar_wait(&vbar[st & 1], (uint32_t)(st >> 1) & 1u, err, 21, st);
        return;
    }
#pragma unroll
    for (int o = 1; o < 8; o <<= 1)
#pragma unroll
        for (int c = 0; c < 8; ++c)
#pragma unroll
            for (int a = 0; a < 3; ++a) acc[c][a] += __shfl_xor_sync(0xffffffffu, acc[c][a], o);
    if (q >= nq) return;
    float z0 = 0.0f, z1 = 0.0f, z2 = 0.0f;
#pragma unroll
    for (int c = 0; c < 8; ++c)
        if (c == jr) {
            z0 = acc[c][0];
            z1 = acc[c][1];
            z2 = acc[c][2];
        }
    const int col = un.c0 + q * 8 + jr;  // column of the group
    if (un.zcol0 >= 0) {
        float* d = z + ((size_t)(un.zcol0 + (int64_t)un.chunk * gp.Cs + col) * G + r) * 4;
        d[0] = z0;
        d[1] = z1;
        d[2] = z2;
    } else {
        int lo = 0, hi = gp.nrec - 1;
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (srec[mid].coff <= col) lo = mid;
            else hi = mid - 1;
        }
        const FwdRec& rec = srec[lo];
        float* wr = w + (size_t)md.woff * 4 * G;
        if (col - rec.coff < rec.C)
            write_w<float>(rec, col - rec.coff, z0, z1, z2, md.SU, wr, (float)md.c1, (float)md.c2, G, r);
    }
}

}  // namespace
}  // namespace hm

#include "hm_fwd_tc.cuh"

namespace hm {
namespace {

// pointers of block `rec` of its mesh.  ONE: the plan
// has a single mesh, passed by value as a kernel parameter (no dependent load
// of the mesh table before the first load of V).
template <class TF, class TA, bool ONE>
struct FwdArgs {
    const TF* Vb;  // V of the block's group
    int coff;      // first column of the block in the group
    int ld;        // columns of the group (Cs)
    const TA* x0;
    TA* wr;
    const float* SU;
    TA c1, c2;
    __device__ __forceinline__ FwdArgs(const FwdRec& rec, const FwdGroup* __restrict__ groups, const MeshDev& m0,
                                       const MeshDev* __restrict__ meshes, const TA* xg, TA* w, int G)
    {
        const MeshDev& md = ONE ? m0 : meshes[rec.mesh];
        const FwdGroup gp = groups[rec.grp];
        Vb = static_cast<const TF*>(md.Vr) + gp.vbase;
        coff = rec.coff;
        ld = gp.Cs;
        x0 = xg + ((size_t)md.xgoff + rec.s0) * G * 4;
        wr = w + (size_t)md.woff * G * 4;
        SU = md.SU;
        c1 = (TA)md.c1;
        c2 = (TA)md.c2;
    }
};

// Several (G) interleaved right-hand sides.  A block's work is the pairs
// (column vector q, RHS chunk c of RC vectors).  T threads (a warp, or the CTA
// for a large block) split the rows into GG groups and take the pairs in
// rounds of PR = T / GG; the GG partial sums are added in a fixed order
// through shared memory.  A warp uses GG = 32 / pairs when the pairs fit a
// warp (else GG = 1, rounds of 32); a CTA keeps at most 32 pairs per round so
// that every large block has at least 4 row groups.
template <class TF, class TA, int RC, int T>
__device__ __forceinline__ void fwd_multi_block(const FwdRec& rec, const FwdArgs<TF, TA, true>& fa, int G, int tid,
                                                TA* red)
{
    constexpr int VEC = Vec16<TF, TA>::N;
    constexpr int kPer = VEC * RC * 3;
    const int Cp = (rec.C + 7) & ~7, Q = Cp / VEC;
    const int NRC = (G + RC - 1) / RC;
    const int pairs = Q * NRC;
    const int GG = T == 32 ? max(1, 32 / pairs) : max(1, T / min(pairs, T / 4));
    const int PR = T / GG;
    const int pl = tid % PR, g = tid / PR;
    for (int pr0 = 0; pr0 < pairs; pr0 += PR) {
        const int nr = min(PR, pairs - pr0);
        const bool active = g < GG && pl < nr;
        const int pr = pr0 + pl;
        const int q = pr % Q, c = pr / Q;
        const int nq = min(RC, G - c * RC);
        TA acc[VEC][RC][3];
#pragma unroll
        for (int e = 0; e < VEC; ++e)
#pragma unroll
            for (int k = 0; k < RC; ++k) acc[e][k][0] = acc[e][k][1] = acc[e][k][2] = (TA)0;
        if (active) {
            const int cq = fa.coff + q * VEC;
            const TA* xp = fa.x0 + (size_t)c * RC * 4;
#pragma unroll 2
            for (int j = g; j < rec.n; j += GG) {
                TA v[VEC];
                Vec16<TF, TA>::load(fa.Vb + vel<TF>(j, cq, fa.ld, rec.n), v);
                const TA* xr = xp + (size_t)j * G * 4;
#pragma unroll
                for (int k = 0; k < RC; ++k) {
                    if (k >= nq) break;
                    TA xa, xb, xc;
                    load3(xr + k * 4, xa, xb, xc);
#pragma unroll
                    for (int e = 0; e < VEC; ++e) {
                        acc[e][k][0] += v[e] * xa;
                        acc[e][k][1] += v[e] * xb;
                        acc[e][k][2] += v[e] * xc;
                    }
                }
            }
        }
        if (GG == 1) {
            if (active) {
#pragma unroll
                for (int e = 0; e < VEC; ++e) {
                    const int col = q * VEC + e;
                    if (col >= rec.C) continue;
#pragma unroll
                    for (int k = 0; k < RC; ++k) {
                        if (k >= nq) break;
                        write_w<TA>(rec, col, acc[e][k][0], acc[e][k][1], acc[e][k][2], fa.SU, fa.wr, fa.c1, fa.c2, G,
                                    c * RC + k);
                    }
                }
            }
        } else {
            if (active) {
                TA* rp = red + (size_t)(g * PR + pl) * kPer;
#pragma unroll
                for (int e = 0; e < VEC; ++e)
#pragma unroll
                    for (int k = 0; k < RC; ++k)
#pragma unroll
                        for (int a = 0; a < 3; ++a) rp[(e * RC + k) * 3 + a] = acc[e][k][a];
            }
            if (T == 32) __syncwarp();
            else __syncthreads();
            for (int idx = tid; idx < nr * VEC * RC; idx += T) {
                const int pp = idx / (VEC * RC), rem = idx - pp * (VEC * RC);
                const int e = rem / RC, k = rem - e * RC;
                const int qq = (pr0 + pp) % Q, cc = (pr0 + pp) / Q;
                const int col = qq * VEC + e, r = cc * RC + k;
                if (col >= rec.C || r >= G) continue;
                TA z[3] = {(TA)0, (TA)0, (TA)0};
                for (int gg = 0; gg < GG; ++gg)
#pragma unroll
                    for (int a = 0; a < 3; ++a) z[a] += red[(size_t)(gg * PR + pp) * kPer + (e * RC + k) * 3 + a];
                write_w<TA>(rec, col, z[0], z[1], z[2], fa.SU, fa.wr, fa.c1, fa.c2, G, r);
            }
            if (T == 32) __syncwarp();
            else __syncthreads();
        }
    }
}

template <class TF, class TA, bool ONE, int RC>
__global__ void __launch_bounds__(kThreads) fwd_small_multi_kernel(
    const int32_t* __restrict__ ids, int64_t nrec, const FwdRec* __restrict__ recs, const FwdGroup* __restrict__ groups,
    const __grid_constant__ MeshDev m0, const MeshDev* __restrict__ meshes, const TA* __restrict__ xg,
    TA* __restrict__ w, int G)
{
    constexpr int kPer = Vec16<TF, TA>::N * RC * 3;
    __shared__ TA red[kThreads / 32][32 * kPer];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t bi = (int64_t)blockIdx.x * (kThreads / 32) + warp;
    if (bi >= nrec) return;
    const FwdRec rec = recs[ids[bi]];
    const FwdArgs<TF, TA, ONE> fa0(rec, groups, m0, meshes, xg, w, G);
    const FwdArgs<TF, TA, true>& fa = reinterpret_cast<const FwdArgs<TF, TA, true>&>(fa0);
    fwd_multi_block<TF, TA, RC, 32>(rec, fa, G, lane, red[warp]);
}

template <class TF, class TA, bool ONE, int RC>
__global__ void __launch_bounds__(kThreads) fwd_big_multi_kernel(
    const int32_t* __restrict__ ids, const FwdRec* __restrict__ recs, const FwdGroup* __restrict__ groups,
    const __grid_constant__ MeshDev m0, const MeshDev* __restrict__ meshes, const TA* __restrict__ xg,
    TA* __restrict__ w, int G)
{
    constexpr int kPer = Vec16<TF, TA>::N * RC * 3;
    __shared__ TA red[kThreads * kPer];
    const FwdRec rec = recs[ids[blockIdx.x]];
    const FwdArgs<TF, TA, ONE> fa0(rec, groups, m0, meshes, xg, w, G);
    const FwdArgs<TF, TA, true>& fa = reinterpret_cast<const FwdArgs<TF, TA, true>&>(fa0);
    fwd_multi_block<TF, TA, RC, kThreads>(rec, fa, G, threadIdx.x, red);
}

// Second pass for the groups taller than one unit: z of every (column,
// vector) as the sum of the units' partial sums in chunk order, then w; one
// CTA per chunk of kReduceCols columns of a group.
template <class TA, bool ONE>
__global__ void __launch_bounds__(kFwdThreads) fwd_reduce_kernel(
    const FwdMulti* __restrict__ multi, const FwdGroup* __restrict__ groups, const FwdRec* __restrict__ recs,
    const __grid_constant__ MeshDev m0, const MeshDev* __restrict__ meshes, const TA* __restrict__ z,
    TA* __restrict__ w, int G)
{
    __shared__ FwdRec srec[kMaxGroupRecs];
    const FwdMulti mu = multi[blockIdx.x];
    const FwdGroup gp = groups[mu.group];
    const MeshDev& md = ONE ? m0 : meshes[gp.mesh];
    for (int i = threadIdx.x; i < gp.nrec; i += blockDim.x) srec[i] = recs[gp.first + i];
    __syncthreads();
    TA* wr = w + (size_t)md.woff * G * 4;
    const TA c1 = (TA)md.c1, c2 = (TA)md.c2;
    const int Cs = gp.Cs;
    for (int idx = threadIdx.x; idx < mu.ncols * G; idx += blockDim.x) {
        const int col = mu.c0 + idx / G, r = idx % G;
        int lo = 0, hi = gp.nrec - 1;
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (srec[mid].coff <= col) lo = mid;
            else hi = mid - 1;
        }
        const FwdRec& rec = srec[lo];
        const int cb = col - rec.coff;
        if (cb >= rec.C) continue;
        // the chunks' partial sums in chunk order, one 4-vector load each
        TA zz[3] = {(TA)0, (TA)0, (TA)0};
#pragma unroll 4
        for (int k = 0; k < mu.nchunk; ++k) {
            TA d0, d1, d2;
            stream::load3(z + ((size_t)(mu.zcol0 + (int64_t)k * Cs + col) * G + r) * 4, d0, d1, d2);
            zz[0] += d0;
            zz[1] += d1;
            zz[2] += d2;
        }
        write_w<TA>(rec, cb, zz[0], zz[1], zz[2], md.SU, wr, c1, c2, G, r);
    }
}

// max over the factor columns of (column scale of U) x |s| of the column's block
__global__ void wbound_kernel(const FwdRec* __restrict__ recs, int64_t nrec, const float* __restrict__ SU,
                              int* __restrict__ out)
{
    float mx = 0.0f;
    for (int64_t b = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; b < nrec; b += (int64_t)gridDim.x * blockDim.x) {
        const FwdRec rec = recs[b];
        float s = 0.0f;
        for (int c = 0; c < rec.C; ++c) s = fmaxf(s, SU[rec.col0 + c]);
        mx = fmaxf(mx, s * (float)rec.n);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    if ((threadIdx.x & 31) == 0) atomicMax(out, __float_as_int(mx));
}

// Column descriptors of the tensor-core forward pass (one warp per block
// record): for every column of a forward group the factor column it feeds,
// the components of z its kernel takes (as write_w) and the factor c su;
// padding columns are marked kFdSkip
__global__ void fdesc_kernel(const FwdRec* __restrict__ recs, int64_t nrec, const FwdGroup* __restrict__ groups,
                             const float* __restrict__ SU, float c1, float c2, uint2* __restrict__ desc)
{
    const int64_t b = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (b >= nrec) return;
    const FwdRec rec = recs[b];
    const int64_t base = (int64_t)groups[rec.grp].dbase + rec.coff;
    const int Cp = (rec.C + 7) & ~7;
    for (int c = lane; c < Cp; c += 32) {
        uint2 d = make_uint2(kFdSkip, 0u);
        if (c < rec.C) {
            int kern = 0, l = c;
            for (;;) {
                const int k = (int)((rec.kpack >> (8 * kern)) & 0xff);
                if (l < k) break;
                l -= k;
                ++kern;
            }
            const int64_t col = (int64_t)rec.col0 + c;
            int p, pq;
            kern_pq(kern, p, pq);
            const float f = (kern == 0 ? c1 : c2) * SU[col];
            const uint32_t pp = kern == 0 ? 3u : (uint32_t)p, qq = kern == 0 ? 3u : (uint32_t)pq;
            d = make_uint2((uint32_t)col | (pp << 28) | (qq << 30), __float_as_uint(f));
        }
        desc[base + c] = d;
    }
}

// ---------------------------------------------------------------- packing
template <class T>
__device__ __forceinline__ T cvt(double v);
template <>
__device__ __forceinline__ double cvt<double>(double v) { return v; }
template <>
__device__ __forceinline__ float cvt<float>(double v) { return (float)v; }
template <>
__device__ __forceinline__ __half cvt<__half>(double v) { return __float2half_rn((float)v); }
template <>
__device__ __forceinline__ __nv_bfloat16 cvt<__nv_bfloat16>(double v) { return __float2bfloat16_rn((float)v); }
// INT16 form: v is already divided by its column's max |v| (|v| <= 1);
// q = round(32767 v) is stored in offset binary, q + 32768 as an unsigned
// 16-bit pattern (see stream::i16x2_to_float2)
__device__ __forceinline__ int16_t i16_store(int q)
{
    return (int16_t)(uint16_t)(max(-32767, min(32767, q)) + 32768);
}
template <>
__device__ __forceinline__ int16_t cvt<int16_t>(double v)
{
    return i16_store(__double2int_rn(v * 32767.0));
}

// per-column scale of the 16-bit forms: max |column| (1 for a zero column)
__global__ void colscale_kernel(int ntask, const Blk* __restrict__ blks, const int32_t* __restrict__ rank,
                                const int64_t* __restrict__ uoff, const int64_t* __restrict__ voff,
                                const int64_t* __restrict__ coff, const double* __restrict__ U,
                                const double* __restrict__ V, float* __restrict__ SU,
                                float* __restrict__ SV)
{
    const int q = blockIdx.x;
    if (q >= ntask) return;
    const int k = rank[q];
    const Blk bk = blks[q / 7];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
    for (int task = warp; task < 2 * k; task += nw) {
        const int l = task % k;
        const bool isu = task < k;
        const int len = isu ? bk.m : bk.n;
        const double* c = (isu ? U + uoff[q] : V + voff[q]) + (size_t)l * len;
        double mx = 0.0;
        for (int e = lane; e < len; e += 32) mx = fmax(mx, fabs(c[e]));
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
        if (lane == 0) (isu ? SU : SV)[coff[q] + l] = mx > 0.0 ? (float)mx : 1.0f;
    }
}

// INT16 form: the factor of w per column, (max|u| / 32767) (max|v| / 32767)
__global__ void sw16_kernel(int64_t n, const float* __restrict__ SU, const float* __restrict__ SV,
                            float* __restrict__ SW)
{
    const int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (c < n) SW[c] = (float)((double)SU[c] * (double)SV[c] / (32767.0 * 32767.0));
}

// U leaf-major: one CTA per leaf.  The 16-bit forms store each leaf's stream
// in 8 x 8 tiles, segment group g = s / 8 and row block b = i / 8 at
// ((g * mp / 8 + b) * 64 + (s % 8) * 8 + i % 8): eight rows of one segment
// stay 16 contiguous bytes, and the tiles are the core matrices of an
// MN-major tensor-core operand.  Other forms: segment-major, s * mp + i.
template <class T>
__global__ void pack_ul_kernel(const int32_t* __restrict__ leaf, const int64_t* __restrict__ lf_base,
                               const int32_t* __restrict__ lf_ptr, const LeafFarItem* __restrict__ items,
                               const PackSrc* __restrict__ src, const double* __restrict__ U,
                               const float* __restrict__ SU, T* __restrict__ Ul)
{
    const int lf = blockIdx.x;
    const int mt = leaf[2 * lf + 1], mp = (mt + 7) & ~7;
    T* dst = Ul + lf_base[lf];
    for (int q = lf_ptr[lf]; q < lf_ptr[lf + 1] - 1; ++q) {
        const PackSrc ps = src[q];
        const LeafFarItem it = items[q];
        const int n = ps.k * mp;
        for (int e = threadIdx.x; e < n; e += blockDim.x) {
            const int l = e / mp, i = e - l * mp;
            double v = 0.0;
            if (i < mt) {
                v = U[ps.src + (size_t)l * ps.ld + i];
                if (SU) v /= (double)SU[it.col + l];
            }
            const size_t sg = (size_t)it.seg_start + l;
            const size_t o = sizeof(T) == 2 ? ((sg / 8) * (size_t)(mp / 8) + (size_t)(i / 8)) * 64 + (sg % 8) * 8 + i % 8
                                            : sg * mp + i;
            dst[o] = cvt<T>(v);
        }
    }
}

// V in its forward group (ld[b] = the group's Cs columns, the block at
// column vb_coff[b]; the layout of vel: unit-contiguous 8 x 8 tiles for the
// 16-bit forms, row-major otherwise): one CTA per block.
template <class T>
__global__ void pack_vr_kernel(const Blk* __restrict__ blks, const int32_t* __restrict__ rank,
                               const int64_t* __restrict__ voff, const int64_t* __restrict__ coff,
                               const int64_t* __restrict__ vb_base, const int64_t* __restrict__ vb_ld,
                               const int64_t* __restrict__ vb_coff, const double* __restrict__ V,
                               const float* __restrict__ SV, T* __restrict__ Vr)
{
    const int b = blockIdx.x;
    const Blk bk = blks[b];
    int kk[7], kp[8];
    kp[0] = 0;
    for (int k = 0; k < 7; ++k) {
        kk[k] = rank[(size_t)b * 7 + k];
        kp[k + 1] = kp[k] + kk[k];
    }
    const int C = kp[7], Cp = (C + 7) & ~7;
    if (C == 0) return;
    T* dst = Vr + vb_base[b];
    const int64_t ld = vb_ld[b], cb = vb_coff[b];
    const int64_t col0 = coff[(size_t)b * 7];
    for (int64_t e = threadIdx.x; e < (int64_t)bk.n * Cp; e += blockDim.x) {
        const int j = (int)(e / Cp), c = (int)(e - (int64_t)j * Cp);
        double v = 0.0;
        if (c < C) {
            int kern = 0;
            while (c >= kp[kern + 1]) ++kern;
            const int l = c - kp[kern];
            v = V[voff[(size_t)b * 7 + kern] + (size_t)l * bk.n + j];
            if (SV) v /= (double)SV[col0 + c];
        }
        const int64_t cc = cb + c;
        dst[vel<T>(j, (int)cc, (int)ld, bk.n)] = cvt<T>(v);
    }
}

// near field leaf-major: one CTA per leaf
template <class T>
__global__ void pack_nl_kernel(const int32_t* __restrict__ leaf, const int64_t* __restrict__ ln_base,
                               const int32_t* __restrict__ ln_ptr, const LeafNearItem* __restrict__ items,
                               const NearSrc* __restrict__ src, const double* __restrict__ N,
                               T* __restrict__ Nl)
{
    const int lf = blockIdx.x;
    const int mt = leaf[2 * lf + 1], mp = (mt + 7) & ~7;
    T* dst = Nl + ln_base[lf];
    for (int q = ln_ptr[lf]; q < ln_ptr[lf + 1] - 1; ++q) {
        const NearSrc ns = src[q];
        const int c0 = items[q].col_start;
        const int n = ns.n * 6 * mp;
        for (int e = threadIdx.x; e < n; e += blockDim.x) {
            const int jv = e / mp, i = e - jv * mp;
            const int j = jv / 6, v = jv - 6 * j;
            double val = 0.0;
            if (i < mt) val = N[ns.src + ((size_t)v * ns.n + j) * mt + i];
            dst[((size_t)(c0 + j) * 6 + v) * mp + i] = cvt<T>(val);
        }
    }
}

// INT16 near stream of the INT16 form: one CTA per leaf, one thread per
// (column, value) segment of the columns after the leaf's diagonal block.
// Header float v of a column = max |V_v| over the leaf's rows / 32767 (0 for
// a zero segment); the segment stores round(32767 V_v / max |V_v|).
__global__ void pack_nl16_kernel(const int32_t* __restrict__ leaf, const int64_t* __restrict__ ln16_base,
                                 const int32_t* __restrict__ ln16_diag, const int32_t* __restrict__ ln_ptr,
                                 const LeafNearItem* __restrict__ items, const NearSrc* __restrict__ src,
                                 const double* __restrict__ N, unsigned char* __restrict__ out)
{
    const int lf = blockIdx.x;
    const int mt = leaf[2 * lf + 1], mp = (mt + 7) & ~7;
    const int ndiag = ln16_diag[lf];
    const size_t colB = (size_t)kNear16Head + 12 * (size_t)mp;
    unsigned char* base = out + ln16_base[lf];
    for (int q = ln_ptr[lf]; q < ln_ptr[lf + 1] - 1; ++q) {
        const NearSrc ns = src[q];
        const int c0 = items[q].col_start;
        if (c0 < ndiag) continue;  // the diagonal block streams from the FP32 near stream
        for (int e = threadIdx.x; e < ns.n * 6; e += blockDim.x) {
            const int j = e / 6, v = e - 6 * j;
            const double* seg = N + ns.src + ((size_t)v * ns.n + j) * mt;
            double mx = 0.0;
            for (int i = 0; i < mt; ++i) mx = fmax(mx, fabs(seg[i]));
            unsigned char* col = base + (size_t)(c0 + j - ndiag) * colB;
            reinterpret_cast<float*>(col)[v] = (float)(mx / 32767.0);
            if (v == 0)
                for (int z = 6; z < kNear16Head / 4; ++z) reinterpret_cast<float*>(col)[z] = 0.0f;
            int16_t* d = reinterpret_cast<int16_t*>(col + kNear16Head) + (size_t)v * mp;
            for (int i = 0; i < mp; ++i) {
                int qv = 0;
                if (i < mt && mx > 0.0) qv = __double2int_rn(seg[i] / mx * 32767.0);
                d[i] = i16_store(qv);
            }
        }
    }
}

int dalloc(hm_matrix& H, DevBuf& d, size_t bytes)
{
    d.bytes = std::max<size_t>(bytes, 256);
    d.p = H.alloc.alloc(d.bytes);
    if (!d.p) return fail(HM_ENOMEM, "device allocation of %zu bytes failed", d.bytes);
    return HM_OK;
}

// right-hand sides per consumer thread of the multi-vector kernels (the
// fwd kernels use the same chunk): 16 accumulated rows x vectors for FP32
// accumulation, 8 for FP64
template <class TF, class TA>
constexpr int multi_rc()
{
    return (sizeof(TA) == 8 ? 8 : 16) / Vec16<TF, TA>::N;
}

// per-device launch data of the streamed leaf kernel of one form
struct StreamLaunch {
    int ctas_per_sm = 0;
    int nsm = 0;
};

template <class TF, class TN, class TA, int RC>
int stream_launch(StreamLaunch& out)
{
    constexpr int kMaxDevices = 64;
    static StreamLaunch cache[kMaxDevices];  // per template instance and device
    int dev = 0;
    HM_CUDA(cudaGetDevice(&dev));
    if (dev < kMaxDevices && cache[dev].nsm > 0) {
        out = cache[dev];
        return HM_OK;
    }
    auto kern = stream::leaf_stream_kernel<TF, TN, TA, RC>;
    const size_t smem = stream::LeafCfg<TF, TA, RC>::smem();
    HM_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    StreamLaunch l;
    HM_CUDA(cudaDeviceGetAttribute(&l.nsm, cudaDevAttrMultiProcessorCount, dev));
    HM_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&l.ctas_per_sm, kern, stream::kThreads, smem));
    l.ctas_per_sm = std::max(l.ctas_per_sm, 1);
    if (dev < kMaxDevices) cache[dev] = l;
    out = l;
    return HM_OK;
}

// a launch of several vectors of a 16-bit form takes its forward pass to
// the tensor cores (and needs max |x| of each vector)
template <class TF>
constexpr bool fwd_on_tc(int G)
{
    // the INT16 split costs two warps' pass over every stage: with 2 vectors
    // the per-vector CUDA-core kernel is faster (level 6: 1.00 against
    // 1.45 ms), with 3 the two tie, with 4 the tensor cores win (1.57 against
    // 2.10 ms)
    return tc_form<TF>() && G >= (std::is_same<TF, int16_t>::value ? 3 : 2);
}

// The forward pass of the 16-bit forms on the tensor cores: one persistent
// launch over every unit for up to 16 vectors, then the second pass of the
// tall groups.  xmax holds max |xg| of each vector (from the gather).
template <class TF>
int run_forward_tc(const Plan& P, const float* xg, float* w, float* z, int G, const int* xmax, cudaStream_t s)
{
    constexpr int kMaxDevices = 64;
    static int nsm_cache[kMaxDevices][2];
    int dev = 0;
    HM_CUDA(cudaGetDevice(&dev));
    const bool one = P.nmesh == 1;
    auto kern = one ? stream::fwd_tc_kernel<TF, true> : stream::fwd_tc_kernel<TF, false>;
    int nsm = dev < kMaxDevices ? nsm_cache[dev][one] : 0;
    if (nsm == 0) {
        HM_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)stream::fp_smem<TF>()));
        HM_CUDA(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
        if (dev < kMaxDevices) nsm_cache[dev][one] = nsm;
    }
    if (P.nunits > INT32_MAX) return fail(HM_EINVAL, "forward pass: too many units");
    if (G > stream::kTcMaxG) return fail(HM_EINVAL, "forward pass: %d vectors in one tensor-core launch", G);
    const MeshDev m0 = one ? P.mesh0 : MeshDev{};
    const unsigned grid = (unsigned)std::min<int64_t>(P.nunits, nsm);  // one CTA per SM (all of its TMEM)
    kern<<<grid, stream::kFpThreads, stream::fp_smem<TF>(), s>>>(P.tcu, (int)P.nunits, m0, P.meshes, P.nmesh, xg, w, z,
                                                             G, xmax, P.err);
    HM_CUDA(cudaGetLastError());
    if (P.nmulti > 0) {
        auto red = one ? fwd_reduce_kernel<float, true> : fwd_reduce_kernel<float, false>;
        red<<<(unsigned)P.nmulti, kFwdThreads, 0, s>>>(P.multi, P.groups, P.fwd, m0, P.meshes, z, w, G);
        HM_CUDA(cudaGetLastError());
    }
    return HM_OK;
}

// One vector of a 16-bit form on the CUDA cores: one CTA per unit (with a
// fork schedule the unit list is split in two halves on two streams), then
// the second pass of the tall groups.
// Several vectors of the INT16 form take the same kernel once per vector
// (vector r of the G interleaved ones), each launch reading the tiles again.
template <class TF>
int run_forward_tile1(const Plan& P, const float* xg, float* w, float* z, cudaStream_t s, const Sched& sc,
                      int G = 1)
{
    const bool one = P.nmesh == 1;
    const MeshDev m0 = one ? P.mesh0 : MeshDev{};
    const bool fork = sc.side && P.nunits > 1;
    const int64_t half = fork ? P.nunits / 2 : P.nunits;
    auto launch = [&](int64_t first, int64_t n, cudaStream_t st) -> int {
        if (n <= 0) return HM_OK;
        auto kt = one ? fwd_tile1_kernel<TF, true> : fwd_tile1_kernel<TF, false>;
        for (int r = 0; r < G; ++r) {
            kt<<<(unsigned)n, kTile1Threads, 0, st>>>(P.units + first, P.tcu + first, P.groups, P.fwd, m0, P.meshes,
                                                      xg, w, z, P.err, G, r);
            HM_CUDA(cudaGetLastError());
        }
        return HM_OK;
    };
    if (fork) {
        HM_CUDA(cudaEventRecord(sc.fork, s));
        HM_CUDA(cudaStreamWaitEvent(sc.side, sc.fork, 0));
        int rc = launch(half, P.nunits - half, sc.side);
        if (rc) return rc;
    }
    {
        int rc = launch(0, half, s);
        if (rc) return rc;
    }
    if (fork) {
        HM_CUDA(cudaEventRecord(sc.join, sc.side));
        HM_CUDA(cudaStreamWaitEvent(s, sc.join, 0));
    }
    if (P.nmulti > 0) {
        auto red = one ? fwd_reduce_kernel<float, true> : fwd_reduce_kernel<float, false>;
        red<<<(unsigned)P.nmulti, kFwdThreads, 0, s>>>(P.multi, P.groups, P.fwd, m0, P.meshes, z, w, G);
        HM_CUDA(cudaGetLastError());
    }
    return HM_OK;
}

// The forward pass over every unit of the plan (with a fork schedule the
// unit list is split in two halves on two streams), then the second pass of
// the tall groups.  The 16-bit forms read their tiles (CUDA or tensor cores).
template <class TF, class TA, int RC>
int run_forward(const Plan& P, TA* xg, TA* w, TA* z, int G, const int* xmax, cudaStream_t s, const Sched& sc)
{
    if (P.nunits <= 0) return HM_OK;
    if constexpr (sizeof(TF) == 2 && std::is_same<TA, float>::value) {
        // the tiles of V: one vector on the CUDA cores, several (up to 16 a
        // launch; INT16 from 3) on the tensor cores
        if (!fwd_on_tc<TF>(G)) return run_forward_tile1<TF>(P, xg, w, z, s, sc, G);
        if constexpr (tc_form<TF>()) return run_forward_tc<TF>(P, xg, w, z, G, xmax, s);
    }
    const bool one = P.nmesh == 1;
    const MeshDev m0 = one ? P.mesh0 : MeshDev{};
    if (RC > 1) {
        // several vectors: one CTA per tall block, one warp per other block
        const bool fork = sc.side && P.nbig > 0 && P.nsmall > 0;
        if (fork) {
            HM_CUDA(cudaEventRecord(sc.fork, s));
            HM_CUDA(cudaStreamWaitEvent(sc.side, sc.fork, 0));
        }
        if (P.nbig > 0) {
            auto kb = one ? fwd_big_multi_kernel<TF, TA, true, RC> : fwd_big_multi_kernel<TF, TA, false, RC>;
            kb<<<(unsigned)P.nbig, kThreads, 0, fork ? sc.side : s>>>(P.big, P.fwd, P.groups, m0, P.meshes, xg, w, G);
            HM_CUDA(cudaGetLastError());
        }
        if (P.nsmall > 0) {
            const unsigned nb = (unsigned)((P.nsmall + kThreads / 32 - 1) / (kThreads / 32));
            auto ks = one ? fwd_small_multi_kernel<TF, TA, true, RC> : fwd_small_multi_kernel<TF, TA, false, RC>;
            ks<<<nb, kThreads, 0, s>>>(P.small, P.nsmall, P.fwd, P.groups, m0, P.meshes, xg, w, G);
            HM_CUDA(cudaGetLastError());
        }
        if (fork) {
            HM_CUDA(cudaEventRecord(sc.join, sc.side));
            HM_CUDA(cudaStreamWaitEvent(s, sc.join, 0));
        }
        return HM_OK;
    }
    const bool fork = sc.side && P.nunits > 1;
    const int64_t half = fork ? P.nunits / 2 : P.nunits;
    if (fork) {
        HM_CUDA(cudaEventRecord(sc.fork, s));
        HM_CUDA(cudaStreamWaitEvent(sc.side, sc.fork, 0));
    }
    // the unit lists [0, half) on s and [half, nunits) on the side stream
    auto launch = [&](int64_t first, int64_t n, cudaStream_t st) -> int {
        if (n <= 0) return HM_OK;
        auto kern = one ? fwd_group_kernel<TF, TA, RC, true> : fwd_group_kernel<TF, TA, RC, false>;
        kern<<<(unsigned)n, kFwdThreads, 0, st>>>(P.units + first, P.groups, P.fwd, m0, P.meshes, xg, w, z, G);
        HM_CUDA(cudaGetLastError());
        return HM_OK;
    };
    if (fork) {
        int rc = launch(half, P.nunits - half, sc.side);
        if (rc) return rc;
    }
    {
        int rc = launch(0, half, s);
        if (rc) return rc;
    }
    if (fork) {
        HM_CUDA(cudaEventRecord(sc.join, sc.side));
        HM_CUDA(cudaStreamWaitEvent(s, sc.join, 0));
    }
    if (P.nmulti > 0) {
        auto red = one ? fwd_reduce_kernel<TA, true> : fwd_reduce_kernel<TA, false>;
        red<<<(unsigned)P.nmulti, kFwdThreads, 0, s>>>(P.multi, P.groups, P.fwd, m0, P.meshes, z, w, G);
        HM_CUDA(cudaGetLastError());
    }
    return HM_OK;
}

// One launch of each phase for G right-hand sides (rows of x and y at
// stride ld), with RC vectors per thread chunk.
template <class TF, class TN, class TA, int RC>
int run_phases(const Plan& P, const double* x, double* y, int G, int64_t ld, TA* xg, TA* w, int* counter,
               cudaStream_t s, const hm_matrix* prof, const Sched& sc)
{
    if (prof) prof_mark(*prof, 0, s);
    int* xmax = fwd_on_tc<TF>(G) ? P.counters + 64 : nullptr;
    if (xmax) HM_CUDA(cudaMemsetAsync(xmax, 0, (size_t)G * sizeof(int), s));
    if (P.npos > 0) {
        const int64_t n = P.npos * G;
        gather_kernel<TA><<<(unsigned)((n + 255) / 256), 256, 0, s>>>(P.meshes, P.nmesh, P.pos_prefix, P.npos, x,
                                                                      ld, xg, G, xmax);
        HM_CUDA(cudaGetLastError());
    }
    if (prof) prof_mark(*prof, 1, s);
    {
        int rc = run_forward<TF, TA, RC>(P, xg, w, static_cast<TA*>(P.z), G, xmax, s, sc);
        if (rc) return rc;
    }
    if (prof) prof_mark(*prof, 2, s);
    if (P.nwork > 0) {
        StreamLaunch l;
        int rc = stream_launch<TF, TN, TA, RC>(l);
        if (rc) return rc;
        const size_t smem = stream::LeafCfg<TF, TA, RC>::smem();
        const int per_sm = sc.ctas_per_sm > 0 ? std::min(sc.ctas_per_sm, l.ctas_per_sm) : l.ctas_per_sm;
        const int64_t ncta = std::min<int64_t>(P.nwork, (int64_t)l.nsm * per_sm);
        stream::leaf_stream_kernel<TF, TN, TA, RC><<<(unsigned)ncta, stream::kThreads, smem, s>>>(
            P.work, (int)P.nwork, P.meshes, counter, P.err, xg, w, G, y, ld);
        HM_CUDA(cudaGetLastError());
    }
    if (prof) prof_mark(*prof, 3, s);
    return HM_OK;
}

// fewest vectors of a launch that takes the far field to the tensor cores
// (leaf product at level 6, CUDA against tensor cores: INT16 8 vectors 3.35
// against 3.72 ms, 10 vectors 4.42 against 4.04 ms; FP16 3.04 against 3.15
// and 3.88 against 3.23 ms; the two meet near 9 in both 16-bit forms)
constexpr int kTcMinG = 9;

// per-device launch data of the tensor-core leaf kernel
template <class TF>
int tc_launch(StreamLaunch& out)
{
    constexpr int kMaxDevices = 64;
    static StreamLaunch cache[kMaxDevices];
    int dev = 0;
    HM_CUDA(cudaGetDevice(&dev));
    if (dev < kMaxDevices && cache[dev].nsm > 0) {
        out = cache[dev];
        return HM_OK;
    }
    auto kern = stream::leaf_tc_kernel<TF>;
    const size_t smem = stream::tc_smem<TF>();
    HM_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    StreamLaunch l;
    HM_CUDA(cudaDeviceGetAttribute(&l.nsm, cudaDevAttrMultiProcessorCount, dev));
    HM_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&l.ctas_per_sm, kern, stream::kThreads, smem));
    l.ctas_per_sm = std::max(l.ctas_per_sm, 1);
    if (dev < kMaxDevices) cache[dev] = l;
    out = l;
    return HM_OK;
}

// One launch of each phase for G <= 16 vectors with the tensor-core leaf kernel.
template <class TF>
int run_phases_tc(const Plan& P, const double* x, double* y, int G, int64_t ld, float* xg, float* w, int* counter,
                  int* xmax, cudaStream_t s, const hm_matrix* prof, const Sched& sc)
{
    constexpr int RC = multi_rc<TF, float>();
    if (prof) prof_mark(*prof, 0, s);
    HM_CUDA(cudaMemsetAsync(xmax, 0, (size_t)G * sizeof(int), s));
    if (P.npos > 0) {
        const int64_t n = P.npos * G;
        gather_kernel<float><<<(unsigned)((n + 255) / 256), 256, 0, s>>>(P.meshes, P.nmesh, P.pos_prefix, P.npos, x,
                                                                         ld, xg, G, xmax);
        HM_CUDA(cudaGetLastError());
    }
    if (prof) prof_mark(*prof, 1, s);
    {
        int rc = run_forward<TF, float, RC>(P, xg, w, static_cast<float*>(P.z), G, xmax, s, sc);
        if (rc) return rc;
    }
    if (prof) prof_mark(*prof, 2, s);
    if (P.nwork > 0) {
        StreamLaunch l;
        int rc = tc_launch<TF>(l);
        if (rc) return rc;
        // tensor memory: the leaf's rows (rounded up to 16) as FP32 columns
        const int mp16 = (std::max(P.max_leaf, 1) + 15) & ~15;
        uint32_t cols = 32;
        while ((int)cols < mp16) cols <<= 1;
        // two CTAs per SM fit by registers and shared memory (a persistent CTA
        // that does not become resident at once finds the work taken and exits)
        int per_sm = sc.ctas_per_sm > 0 ? std::min(sc.ctas_per_sm, 2) : 2;
        per_sm = std::min(per_sm, (int)(512 / cols));  // never wait for another CTA's columns
        const int64_t ncta = std::min<int64_t>(P.nwork, (int64_t)l.nsm * std::max(per_sm, 1));
        stream::leaf_tc_kernel<TF><<<(unsigned)ncta, stream::kThreads, stream::tc_smem<TF>(), s>>>(
            P.work, (int)P.nwork, P.meshes, counter, P.err, xg, w, G, xmax, cols, y, ld);
        HM_CUDA(cudaGetLastError());
    }
    if (prof) prof_mark(*prof, 3, s);
    return HM_OK;
}

// The product over every mesh of the plan: one vector with the single-vector
// kernels, several in launches of up to Gmax interleaved vectors each.
template <class TF, class TN, class TA>
int run_product_t(const Plan& P, const double* x, double* y, int nrhs, int64_t ld, TA* xg, TA* w,
                  cudaStream_t s, const hm_matrix* prof, const Sched& sc)
{
    constexpr int Rr = stream::Smem16<TF, TA>::N;
    constexpr int RC = multi_rc<TF, TA>();
    const int mpmax = std::max((P.max_leaf + 7) & ~7, 8);
    if (mpmax / Rr > stream::kConsumers || 6 * mpmax * (int)sizeof(TN) > stream::kStageBytes)
        return fail(HM_EINVAL, "product: a leaf of %d rows does not fit the streamed kernel", P.max_leaf);
    if (P.nwork > 0) HM_CUDA(cudaMemsetAsync(P.counters, 0, 64 * sizeof(int), s));
    if (nrhs == 1) return run_phases<TF, TN, TA, 1>(P, x, y, 1, ld, xg, w, P.counters, s, prof, sc);
    int k = 0, r0 = 0;
    if constexpr (tc_form<TF>() && std::is_same<TA, float>::value) {
        // 16-bit factors: launches of 16 vectors (at least kTcMinG) take the
        // far field to the tensor cores; fewer vectors stay on the CUDA cores,
        // where the per-stage latency of the tensor-core pipeline does not pay
        for (; nrhs - r0 >= kTcMinG; r0 += std::min(stream::kTcMaxG, nrhs - r0), ++k) {
            const int G = std::min(stream::kTcMaxG, nrhs - r0);
            int rc = run_phases_tc<TF>(P, x + (size_t)r0 * ld, y + (size_t)r0 * ld, G, ld, reinterpret_cast<float*>(xg),
                                       reinterpret_cast<float*>(w), P.counters + k, P.counters + 64, s,
                                       k == 0 ? prof : nullptr, sc);
            if (rc) return rc;
        }
        if (r0 == nrhs) return HM_OK;
        if (nrhs - r0 == 1)
            return run_phases<TF, TN, TA, 1>(P, x + (size_t)r0 * ld, y + (size_t)r0 * ld, 1, ld, xg, w,
                                             P.counters + k, s, k == 0 ? prof : nullptr, sc);
    }
    // every (row block, RHS chunk) pair of the largest leaf needs a consumer
    // thread; at most 32 vectors keep at least 16 segments per slot (16 where
    // the forward pass takes them to the tensor cores)
    int Gmax = std::min(32, RC * (stream::kConsumers / (mpmax / Rr)));
    if (tc_form<TF>() && std::is_same<TA, float>::value) Gmax = std::min(Gmax, stream::kTcMaxG);
    for (; r0 < nrhs; r0 += Gmax, ++k) {
        const int G = std::min(Gmax, nrhs - r0);
        int rc = run_phases<TF, TN, TA, RC>(P, x + (size_t)r0 * ld, y + (size_t)r0 * ld, G, ld, xg, w,
                                            P.counters + k, s, k == 0 ? prof : nullptr, sc);
        if (rc) return rc;
    }
    return HM_OK;
}

template <class T>
int pack_form(hm_matrix& H, int form, const float* SU, const float* SV, cudaStream_t s)
{
    int rc;
    if ((rc = dalloc(H, H.Ul[form], (size_t)H.ul_total * sizeof(T)))) return rc;
    if ((rc = dalloc(H, H.Vr[form], (size_t)H.vr_total * sizeof(T)))) return rc;
    HM_CUDA(cudaMemsetAsync(H.Vr[form].p, 0, (size_t)H.vr_total * sizeof(T), s));  // padding rows and columns
    // padding segments are zero
    HM_CUDA(cudaMemsetAsync(H.Ul[form].p, 0, (size_t)H.ul_total * sizeof(T), s));
    if (H.nleaves > 0) {
        pack_ul_kernel<T><<<(unsigned)H.nleaves, 256, 0, s>>>(
            H.d_leaf.as<int32_t>(), H.d_lf_base.as<int64_t>(), H.d_lf_ptr.as<int32_t>(),
            H.d_lf_items.as<LeafFarItem>(), H.d_lf_src.as<PackSrc>(), H.U64.as<double>(), SU,
            H.Ul[form].as<T>());
        HM_CUDA(cudaGetLastError());
    }
    if (H.nadm > 0) {
        pack_vr_kernel<T><<<(unsigned)H.nadm, 256, 0, s>>>(
            H.d_adm.as<Blk>(), H.d_rank.as<int32_t>(), H.d_voff.as<int64_t>(), H.d_coff.as<int64_t>(),
            H.d_vb_base.as<int64_t>(), H.d_vb_ld.as<int64_t>(), H.d_vb_coff.as<int64_t>(), H.V64.as<double>(), SV,
            H.Vr[form].as<T>());
        HM_CUDA(cudaGetLastError());
    }
    return HM_OK;
}

template <class T>
int pack_near(hm_matrix& H, DevBuf& dst, cudaStream_t s)
{
    int rc;
    if ((rc = dalloc(H, dst, (size_t)H.nl_total * sizeof(T)))) return rc;
    if (H.nleaves > 0) {
        pack_nl_kernel<T><<<(unsigned)H.nleaves, 256, 0, s>>>(
            H.d_leaf.as<int32_t>(), H.d_ln_base.as<int64_t>(), H.d_ln_ptr.as<int32_t>(),
            H.d_ln_items.as<LeafNearItem>(), H.d_ln_src.as<NearSrc>(), H.N64.as<double>(),
            dst.as<T>());
        HM_CUDA(cudaGetLastError());
    }
    return HM_OK;
}

}  // namespace

template <class TF, class TN, class TA>
int prepare_t(int* ctas_per_sm)
{
    StreamLaunch l1, lm;
    int rc = stream_launch<TF, TN, TA, 1>(l1);
    if (!rc) rc = stream_launch<TF, TN, TA, multi_rc<TF, TA>()>(lm);
    if (!rc && ctas_per_sm) *ctas_per_sm = std::max(l1.ctas_per_sm, lm.ctas_per_sm);
    return rc;
}

int product_prepare(int32_t form, int* ctas_per_sm)
{
    switch (form) {
        case HM_FP64: return prepare_t<double, double, double>(ctas_per_sm);
        case HM_FP32: return prepare_t<float, float, float>(ctas_per_sm);
        case HM_BF16: return prepare_t<__nv_bfloat16, float, float>(ctas_per_sm);
        case HM_FP16: return prepare_t<__half, float, float>(ctas_per_sm);
        case HM_I16: return prepare_t<int16_t, float, float>(ctas_per_sm);
        default: return fail(HM_EINVAL, "product: unknown form %d", form);
    }
}

int run_product(const Plan& P, int32_t form, const double* x, double* y, int32_t nrhs, int64_t ld, void* xg,
                void* w, cudaStream_t s, const hm_matrix* prof, const Sched* sched)
{
    const Sched sc = sched ? *sched : Sched{};
    switch (form) {
        case HM_FP64:
            return run_product_t<double, double, double>(P, x, y, nrhs, ld, static_cast<double*>(xg),
                                                         static_cast<double*>(w), s, prof, sc);
        case HM_FP32:
            return run_product_t<float, float, float>(P, x, y, nrhs, ld, static_cast<float*>(xg),
                                                      static_cast<float*>(w), s, prof, sc);
        case HM_BF16:
            return run_product_t<__nv_bfloat16, float, float>(P, x, y, nrhs, ld, static_cast<float*>(xg),
                                                              static_cast<float*>(w), s, prof, sc);
        case HM_FP16:
            return run_product_t<__half, float, float>(P, x, y, nrhs, ld, static_cast<float*>(xg),
                                                       static_cast<float*>(w), s, prof, sc);
        case HM_I16:
            return run_product_t<int16_t, float, float>(P, x, y, nrhs, ld, static_cast<float*>(xg),
                                                        static_cast<float*>(w), s, prof, sc);
        default:
            return fail(HM_EINVAL, "product: unknown form %d", form);
    }
}

MeshDev mesh_desc(const hm_matrix& H, int32_t form)
{
    MeshDev m{};
    m.Ul = H.Ul[form].p;
    m.Vr = H.Vr[form].p;
    m.Nl = form == HM_FP64 ? H.Nl64.p : H.Nl32.p;
    m.SU = (form == HM_BF16 || form == HM_FP16) ? H.SU.as<float>() : (form == HM_I16 ? H.SW16.as<float>() : nullptr);
    m.fdesc = (form == HM_BF16 || form == HM_FP16) ? H.fdesc.as<uint2>()
                                                   : (form == HM_I16 ? H.fdesc16.as<uint2>() : nullptr);
    m.leaf = H.d_leaf.as<int32_t>();
    m.lf_base = H.d_lf_base.as<int64_t>();
    m.lf_ptr = H.d_lf_ptr.as<int32_t>();
    m.lf_items = H.d_lf_items.as<LeafFarItem>();
    m.lr_ptr = H.d_lr_ptr.as<int32_t>();
    m.lr_items = H.d_lr_items.as<LeafFarItem>();
    m.ln_base = H.d_ln_base.as<int64_t>();
    m.ln_ptr = H.d_ln_ptr.as<int32_t>();
    m.ln_items = H.d_ln_items.as<LeafNearItem>();
    if (form == HM_I16) {
        m.Nl16 = H.Nl16.as<unsigned char>();
        m.ln16_base = H.d_ln16_base.as<int64_t>();
        m.ln16_diag = H.d_ln16_diag.as<int32_t>();
    }
    m.perm = H.d_perm.as<int32_t>();
    m.xoff = m.xgoff = m.woff = 0;
    m.M = (int32_t)H.M;
    m.max_leaf = H.max_leaf;
    m.c1 = (1.0 + H.nu) * (3.0 - 4.0 * H.nu) / (2.0 * H.E * (1.0 - H.nu));
    m.c2 = (1.0 + H.nu) / (2.0 * H.E * (1.0 - H.nu));
    // |w| <= max(c1, c2) x column scale x |s| x max|x| (|v| <= 1); rounded up
    m.wbound = (form == HM_BF16 || form == HM_FP16) ? (float)(std::max(m.c1, m.c2) * (double)H.wbound_su) * 1.0001f
               : form == HM_I16 ? (float)(std::max(m.c1, m.c2) * 32767.0 * (double)H.wbound_sw16) * 1.0001f
                                : 0.0f;
    return m;
}

int write_mesh_table(hm_matrix& H, int32_t form, cudaStream_t s)
{
    int rc;
    if (!H.d_mesh[form].p)
        if ((rc = dalloc(H, H.d_mesh[form], sizeof(MeshDev)))) return rc;
    // a product in flight may still read the old table
    HM_CUDA(cudaDeviceSynchronize());
    const MeshDev m = mesh_desc(H, form);
    HM_CUDA(cudaMemcpy(H.d_mesh[form].p, &m, sizeof m, cudaMemcpyHostToDevice));
    (void)s;
    return HM_OK;
}

int matvec_device_scratch(const hm_matrix& H, const double* x, double* y, int32_t nrhs, int64_t ld,
                          int32_t form, cudaStream_t s, const Scratch& scr)
{
    Plan P{};
    P.meshes = H.d_mesh[form].as<MeshDev>();
    P.mesh0 = mesh_desc(H, form);
    P.nmesh = 1;
    P.pos_prefix = H.d_pos_prefix.as<int64_t>();
    P.npos = H.M;
    P.fwd = H.d_fwd_all.as<FwdRec>();
    P.groups = H.d_groups.as<FwdGroup>();
    P.units = H.d_units.as<FwdUnit>();
    P.tcu = H.d_tcunits.as<FwdTcUnit>();
    P.nunits = (int64_t)H.unit_h.size();
    P.multi = H.d_multi.as<FwdMulti>();
    P.nmulti = (int64_t)H.multi_h.size();
    P.zcols = H.zcols;
    P.z = scr.z;
    P.big = H.d_big.as<int32_t>();
    P.nbig = (int64_t)H.big_h.size();
    P.small = H.d_small.as<int32_t>();
    P.nsmall = (int64_t)H.small_h.size();
    P.work = H.d_work.as<int2>();
    P.nwork = H.nleaves;
    P.max_leaf = H.max_leaf;
    P.counters = scr.counters;
    P.err = H.d_err.as<int>();
    return run_product(P, form, x, y, nrhs, ld, scr.xg, scr.w, s, scr.profile ? &H : nullptr);
}

int matvec_device_coeffs(hm_matrix& H, const double* x, double* y, int32_t form, double c1, double c2,
                         cudaStream_t s)
{
    int rc;
    if (!H.d_mesh_k.p)
        if ((rc = dalloc(H, H.d_mesh_k, sizeof(MeshDev)))) return rc;
    MeshDev m = mesh_desc(H, form);
    m.c1 = c1;
    m.c2 = c2;
    // a pageable source: the copy is staged before the call returns
    HM_CUDA(cudaMemcpyAsync(H.d_mesh_k.p, &m, sizeof m, cudaMemcpyHostToDevice, s));
    Plan P{};
    P.meshes = H.d_mesh_k.as<MeshDev>();
    P.mesh0 = m;
    P.nmesh = 1;
    P.pos_prefix = H.d_pos_prefix.as<int64_t>();
    P.npos = H.M;
    P.fwd = H.d_fwd_all.as<FwdRec>();
    P.groups = H.d_groups.as<FwdGroup>();
    P.units = H.d_units.as<FwdUnit>();
    P.tcu = H.d_tcunits.as<FwdTcUnit>();
    P.nunits = (int64_t)H.unit_h.size();
    P.multi = H.d_multi.as<FwdMulti>();
    P.nmulti = (int64_t)H.multi_h.size();
    P.zcols = H.zcols;
    P.z = H.zb.p;
    P.big = H.d_big.as<int32_t>();
    P.nbig = (int64_t)H.big_h.size();
    P.small = H.d_small.as<int32_t>();
    P.nsmall = (int64_t)H.small_h.size();
    P.work = H.d_work.as<int2>();
    P.nwork = H.nleaves;
    P.max_leaf = H.max_leaf;
    P.counters = H.d_counters.as<int>();
    P.err = H.d_err.as<int>();
    return run_product(P, form, x, y, 1, 3 * H.M, H.xg.p, H.wb.p, s, nullptr);
}

int matvec_device(const hm_matrix& H, const double* x, double* y, int32_t nrhs, int64_t ld,
                  int32_t form, cudaStream_t s)
{
    Scratch scr{H.xg.p, H.wb.p, H.d_counters.as<int>(), true, H.zb.p};
    return matvec_device_scratch(H, x, y, nrhs, ld, form, s, scr);
}

Scratch make_scratch(const hm_matrix& H, int32_t nrhs, int32_t form, void* base)
{
    // the layout matvec_scratch_bytes counts: xg, w, counters
    const size_t ta = form == HM_FP64 ? 8 : 4;
    auto up = [](size_t v) { return (v + 255) & ~(size_t)255; };
    const size_t vec = up((size_t)nrhs * 4 * (size_t)H.M * ta);
    const size_t wb = up((size_t)nrhs * (size_t)std::max<int64_t>(H.w_total, 1) * ta);
    unsigned char* b = static_cast<unsigned char*>(base);
    const size_t cnt = up((size_t)kCounterInts * sizeof(int));
    return Scratch{b, b + vec, reinterpret_cast<int*>(b + vec + wb), false, b + vec + wb + cnt};
}

size_t matvec_scratch_bytes(const hm_matrix& H, int32_t nrhs, int32_t form)
{
    const size_t ta = form == HM_FP64 ? 8 : 4;
    auto up = [](size_t b) { return (b + 255) & ~(size_t)255; };
    return up((size_t)nrhs * 4 * (size_t)H.M * ta) + up((size_t)nrhs * (size_t)std::max<int64_t>(H.w_total, 1) * ta) +
           up((size_t)kCounterInts * sizeof(int)) + up((size_t)nrhs * (size_t)std::max<int64_t>(H.zcols, 1) * 4 * ta);
}

// max over the factor columns of S[column] x |s| of the column's block (the
// bound of |w| / max|x| of the tensor-core far field, before the coefficients)
static int column_bound(hm_matrix& H, const float* S, float& out, cudaStream_t s)
{
    int rc;
    DevBuf wb;
    if ((rc = dalloc(H, wb, 256))) return rc;
    HM_CUDA(cudaMemsetAsync(wb.p, 0, 4, s));
    const int64_t nrec = (int64_t)H.fwd_h.size();
    if (nrec > 0) {
        wbound_kernel<<<256, 256, 0, s>>>(H.d_fwd_all.as<FwdRec>(), nrec, S, wb.as<int>());
        HM_CUDA(cudaGetLastError());
    }
    int bits = 0;
    HM_CUDA(cudaMemcpyAsync(&bits, wb.p, 4, cudaMemcpyDeviceToHost, s));
    HM_CUDA(cudaStreamSynchronize(s));
    H.alloc.release(wb.p, wb.bytes);
    std::memcpy(&out, &bits, 4);
    return HM_OK;
}

// the streaming layouts of one form (and the FP32 near field and the column
// scales it shares with the other reduced forms), then the form's mesh table
int pack_device(hm_matrix& H, int32_t form, cudaStream_t s)
{
    int rc;
    const int ntask = (int)(H.nadm * 7);
    if (form == HM_FP64) {
        if ((rc = pack_form<double>(H, HM_FP64, nullptr, nullptr, s))) return rc;
        if ((rc = pack_near<double>(H, H.Nl64, s))) return rc;
        if ((rc = write_mesh_table(H, HM_FP64, s))) return rc;
        H.packed[HM_FP64] = true;
        return HM_OK;
    }
    if (!H.Nl32.p)
        if ((rc = pack_near<float>(H, H.Nl32, s))) return rc;
    if (form == HM_FP32) {
        if ((rc = pack_form<float>(H, HM_FP32, nullptr, nullptr, s))) return rc;
    } else {
        if (!H.SU.p) {
            if ((rc = dalloc(H, H.SU, (size_t)std::max<int64_t>(H.c_total, 1) * 4))) return rc;
            if ((rc = dalloc(H, H.SV, (size_t)std::max<int64_t>(H.c_total, 1) * 4))) return rc;
            if (ntask > 0) {
                colscale_kernel<<<ntask, 128, 0, s>>>(
                    ntask, H.d_adm.as<Blk>(), H.d_rank.as<int32_t>(), H.d_uoff.as<int64_t>(),
                    H.d_voff.as<int64_t>(), H.d_coff.as<int64_t>(), H.U64.as<double>(),
                    H.V64.as<double>(), H.SU.as<float>(), H.SV.as<float>());
                HM_CUDA(cudaGetLastError());
            }
        }
        if (form == HM_I16) {
            // block floating point: U and V each divided by their column's
            // max |value| and stored as round(32767 v); w carries the product
            // of the two scales and 1 / 32767^2
            if (!H.SW16.p) {
                if ((rc = dalloc(H, H.SW16, (size_t)std::max<int64_t>(H.c_total, 1) * 4))) return rc;
                if (H.c_total > 0) {
                    sw16_kernel<<<(unsigned)((H.c_total + 255) / 256), 256, 0, s>>>(H.c_total, H.SU.as<float>(),
                                                                                    H.SV.as<float>(), H.SW16.as<float>());
                    HM_CUDA(cudaGetLastError());
                }
            }
            if ((rc = pack_form<int16_t>(H, HM_I16, H.SU.as<float>(), H.SV.as<float>(), s))) return rc;
            if (H.wbound_sw16 == 0.0f)
                if ((rc = column_bound(H, H.SW16.as<float>(), H.wbound_sw16, s))) return rc;
            // the column descriptors of the tensor-core forward pass, with
            // c1 or c2 times the column's SU SV / 32767^2
            if (!H.fdesc16.p) {
                if (H.c_total > kFdMaxCol)
                    return fail(HM_EINVAL, "16-bit forms: more than %lld factor columns", (long long)kFdMaxCol);
                if ((rc = dalloc(H, H.fdesc16, (size_t)std::max<int64_t>(H.dcols, 1) * sizeof(uint2)))) return rc;
                const int64_t nrec = (int64_t)H.fwd_h.size();
                if (nrec > 0) {
                    const MeshDev m = mesh_desc(H, HM_FP64);
                    fdesc_kernel<<<(unsigned)((nrec + 7) / 8), 256, 0, s>>>(H.d_fwd_all.as<FwdRec>(), nrec,
                                                                            H.d_groups.as<FwdGroup>(),
                                                                            H.SW16.as<float>(), (float)m.c1,
                                                                            (float)m.c2, H.fdesc16.as<uint2>());
                    HM_CUDA(cudaGetLastError());
                }
            }
            if (!H.Nl16.p) {
                if ((rc = dalloc(H, H.Nl16, (size_t)std::max<int64_t>(H.nl16_bytes, 16)))) return rc;
                if (H.nleaves > 0) {
                    pack_nl16_kernel<<<(unsigned)H.nleaves, 256, 0, s>>>(
                        H.d_leaf.as<int32_t>(), H.d_ln16_base.as<int64_t>(), H.d_ln16_diag.as<int32_t>(),
                        H.d_ln_ptr.as<int32_t>(), H.d_ln_items.as<LeafNearItem>(), H.d_ln_src.as<NearSrc>(),
                        H.N64.as<double>(), H.Nl16.as<unsigned char>());
                    HM_CUDA(cudaGetLastError());
                }
            }
            if ((rc = write_mesh_table(H, form, s))) return rc;
            H.packed[form] = true;
            return HM_OK;
        }
        if (!H.fdesc.p) {
            if (H.c_total > kFdMaxCol) return fail(HM_EINVAL, "16-bit forms: more than %lld factor columns", (long long)kFdMaxCol);
            if ((rc = dalloc(H, H.fdesc, (size_t)std::max<int64_t>(H.dcols, 1) * sizeof(uint2)))) return rc;
            const int64_t nrec = (int64_t)H.fwd_h.size();
            if (nrec > 0) {
                const MeshDev m = mesh_desc(H, HM_FP64);
                fdesc_kernel<<<(unsigned)((nrec + 7) / 8), 256, 0, s>>>(H.d_fwd_all.as<FwdRec>(), nrec,
                                                                        H.d_groups.as<FwdGroup>(), H.SU.as<float>(),
                                                                        (float)m.c1, (float)m.c2,
                                                                        H.fdesc.as<uint2>());
                HM_CUDA(cudaGetLastError());
            }
        }
        if (H.wbound_su == 0.0f)
            if ((rc = column_bound(H, H.SU.as<float>(), H.wbound_su, s))) return rc;
        // V columns are normalised by their ACA pivot (max |v| = 1), so V is
        // stored without a scale; U carries the magnitudes and gets one scale
        // per column
        if (form == HM_BF16)
            rc = pack_form<__nv_bfloat16>(H, HM_BF16, H.SU.as<float>(), nullptr, s);
        else
            rc = pack_form<__half>(H, HM_FP16, H.SU.as<float>(), nullptr, s);
        if (rc) return rc;
    }
    if ((rc = write_mesh_table(H, form, s))) return rc;
    H.packed[form] = true;
    return HM_OK;
}

}  // namespace hm

using namespace hm;

extern "C" {

int hm_pack(hm_matrix* H, int32_t form, void* stream)
{
    if (!H) return fail(HM_EINVAL, "hm_pack: NULL matrix");
    if (form < HM_FP64 || form >= HM_NFORMS) return fail(HM_EINVAL, "hm_pack: unknown form %d", form);
    if (H->rect && form != HM_FP64 && form != HM_FP32)
        return fail(HM_EINVAL, "hm_pack: an evaluation operator has the forms HM_FP64 and HM_FP32");
    if (H->rect && form == HM_FP64) return HM_OK;  // its FP64 arenas are the FP64 form
    if (H->packed[form]) return HM_OK;
    if (H->compacted) return fail(HM_EINVAL, "hm_pack: FP64 data released (hm_compact); pack before compacting");
    if (H->aca_deferred)
        return fail(HM_EINVAL, "hm_pack: ACA deferred (HM_DEFER_ACA): the matrix serves hm_amvm with ACA on demand only");
    cudaStream_t s = (cudaStream_t)stream;
    cudaStream_t saved = H->alloc.stream;
    H->alloc.stream = s;
    cudaEvent_t e0, e1;
    HM_CUDA(cudaEventCreate(&e0));
    HM_CUDA(cudaEventCreate(&e1));
    cudaEventRecord(e0, s);
    int rc = H->rect ? eval_pack_fp32(*H, s) : pack_device(*H, form, s);
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
    if (H->rect) return fail(HM_EINVAL, "hm_matvec: an evaluation operator (hm_build_point_tree) has only hm_eval_points and hm_amvm");
    if (nrhs < 1 || nrhs > H->max_rhs)
        return fail(HM_EINVAL, "hm_matvec: nrhs=%d outside 1..%d", nrhs, H->max_rhs);
    if (ld < 3 * H->M) return fail(HM_EINVAL, "hm_matvec: ld=%lld < 3M=%lld", (long long)ld, (long long)(3 * H->M));
    if (form < HM_FP64 || form >= HM_NFORMS) return fail(HM_EINVAL, "hm_matvec: unknown form %d", form);
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
    if (H->rect) return fail(HM_EINVAL, "hm_matvec_host: an evaluation operator (hm_build_point_tree) has only hm_eval_points and hm_amvm");
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
