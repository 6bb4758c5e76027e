// hm_leaf_tc.cuh -- per-leaf product for several right-hand sides with the
// far field on the tensor cores (tcgen05), for the FP16 / BF16 / INT16 forms.
//
// For a leaf tau and G <= 16 right-hand sides the far field is
//   Y[i, (r, a)] = sum_s U[i, s] W[s, (r, a)]
// over the leaf's U segments s (Section 2: the U factors of every admissible
// block whose row cluster contains tau, with w = c V^T x of the block).  One
// tcgen05.mma computes D[m, i] += A[m, k] B[k, i] for M = 128, K = 16 and N =
// the leaf's rows (rounded up to 16), accumulating in tensor memory:
//   B = U of 16 segments, straight from the stage (the stream is stored in
//       8 x 8 core-matrix tiles, an MN-major operand).  INT16 stages (offset
//       binary q = v + 32768) are split into two exact FP16 operands of the
//       same layout, 256 (q / 256 - 128) in place and q mod 256 right after
//       the stage's U when both fit the stage region (split by a second warp
//       while the builder builds A), otherwise in the slot's 4-vector region
//       (free once A is built); their MMAs accumulate into the same D;
//   A = 128 rows 64 split + 16 a + r: W scaled by a power of two t_r and
//       split into hi = fp16(W t_r) (split 0) and lo = fp16(W t_r - hi)
//       (split 1), so that D[(0, a, r)] + D[(1, a, r)] = t_r (U W) to about
//       2^-22 relative; the rows of vectors r >= G and of the padding
//       component a = 3 are zero (never written).  The consumer warps build it
//       in a K-major core-matrix layout from the staged FP32 w: a lane takes
//       vector r and eight segments, so that the eight lanes of a shared-memory
//       phase read 128 contiguous bytes and write the eight rows of one core.
// t_r = 2^floor(log2(2^15 / (wbound x max|x_r|))): wbound bounds |w| / max|x|
// for the mesh (|v| <= 1 after pivot normalisation, so |V^T x| <= |s| max|x|;
// INT16: |v| <= 32767 and w carries the scales SU SV / 32767^2), which keeps
// every scaled value inside the FP16 range.
// The three builder warps take the far stages round-robin, each into its own
// A buffer, so that the builds of consecutive stages overlap; INT16: warp
// 5 + k splits the stages that builder 2 + k builds.  One thread
// (lane 0 of warp 1) issues every stage's MMAs in stage order, once its
// builder has announced the A tile, and commits them to the barriers that
// release the builder's A buffer and the stage (one issuing thread: the
// accumulation order is fixed, and every commit tracks all far MMAs).  The near field stays on the CUDA cores
// (as in the multi-vector kernel) and is added to the far result at the end of
// the leaf, in a fixed order.  Every wait is bounded.
#pragma once

#include <type_traits>

#include "hm_stream.cuh"

namespace hm {
namespace stream {

constexpr int kTcStage = 12288;  // bytes of stream data per slot
constexpr int kTcAux = 12288;    // bytes of staged 4-vectors per slot
constexpr int kTcSlots = 3;
constexpr int kTcSlotBytes = kTcStage + kTcAux;
constexpr int kTcK = 48;                   // segments per far stage at most (three K steps)
constexpr int kTcABytes = 128 * kTcK * 2;  // one A tile
constexpr int kTcSbo = (kTcK / 8) * 128;   // M-direction core stride of an A tile
constexpr int kTcMaxG = 16;
constexpr int kTcBuildW = 3;  // builder warps, one A buffer each
template <class TF>
constexpr size_t tc_smem()
{
    return (size_t)kTcSlots * kTcSlotBytes + kTcBuildW * (size_t)kTcABytes;
}

// the low half of an INT16 far stage's split (at most a stage) fits the
// slot's 4-vector region; an MMA of N = rows rounded up to 16 reads up to
// 128 bytes past it, still inside shared memory (the next slot or A tiles)
static_assert(kTcStage <= kTcAux, "the split of a far stage must fit the 4-vector region");
static_assert(kConsumers * 8 * 3 * 4 <= kTcSlotBytes, "the near reduction must fit a slot");
static_assert(64 * 64 * 4 <= kTcSlotBytes, "the far epilogue exchange must fit a slot");
static_assert(2 + 2 * kTcBuildW <= kThreads / 32, "an INT16 splitter warp for every builder warp");

__device__ __forceinline__ uint64_t tc_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo)
{
    // SWIZZLE_NONE shared-memory matrix descriptor: start, leading (K-direction)
    // and stride (M/N-direction) core-matrix offsets in 16-byte units, version 1
    return (uint64_t)((saddr >> 4) & 0x3fff) | ((uint64_t)((lbo >> 4) & 0x3fff) << 16) |
           ((uint64_t)((sbo >> 4) & 0x3fff) << 32) | ((uint64_t)1 << 46);
}

// kind::f16, D FP32, A K-major, B MN-major, M = 128
__device__ __forceinline__ uint32_t tc_idesc(int n, bool bf16)
{
    const uint32_t f = bf16 ? 1u : 0u;
    return (1u << 4) | (f << 7) | (f << 10) | (0u << 15) | (1u << 16) | ((uint32_t)(n >> 3) << 17) |
           ((uint32_t)(128 >> 4) << 24);
}

__device__ __forceinline__ void tc_mma(uint32_t d, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc)
{
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(d),
        "l"(a), "l"(b), "r"(idesc), "r"(acc)
        : "memory");
}

__device__ __forceinline__ void tc_commit(uint64_t* bar)
{
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                     smem_addr(bar))
                 : "memory");
}

__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// 8 consecutive FP32 columns of this thread's TMEM lane
__device__ __forceinline__ void tc_ld8(uint32_t addr, float* v)
{
    uint32_t r[8];
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7])
                 : "r"(addr)
                 : "memory");
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int q = 0; q < 8; ++q) v[q] = __uint_as_float(r[q]);
}

// two FP32 values -> their hi = rn(v) and lo = rn(v - hi) in the operand type,
// packed (v0 in the low half); each conversion rounds as the scalar one does
template <class T>
__device__ __forceinline__ void tc_split2(float v0, float v1, uint32_t& hi, uint32_t& lo);
template <>
__device__ __forceinline__ void tc_split2<__half>(float v0, float v1, uint32_t& hi, uint32_t& lo)
{
    const __half2 h = __floats2half2_rn(v0, v1);
    const float2 b = __half22float2(h);
    const __half2 l = __floats2half2_rn(v0 - b.x, v1 - b.y);
    hi = *reinterpret_cast<const uint32_t*>(&h);
    lo = *reinterpret_cast<const uint32_t*>(&l);
}
template <>
__device__ __forceinline__ void tc_split2<__nv_bfloat16>(float v0, float v1, uint32_t& hi, uint32_t& lo)
{
    const __nv_bfloat162 h = __floats2bfloat162_rn(v0, v1);
    const float2 b = __bfloat1622float2(h);
    const __nv_bfloat162 l = __floats2bfloat162_rn(v0 - b.x, v1 - b.y);
    hi = *reinterpret_cast<const uint32_t*>(&h);
    lo = *reinterpret_cast<const uint32_t*>(&l);
}

// two offset-binary int16 values q (one word) -> the exact FP16 pairs
// 256 (q / 256 - 128) (hi) and q mod 256 (lo): a byte b becomes the FP16
// number 1024 + b by its bits 0x6400 | b, from which 1024 (or 1024 + 128) is
// subtracted exactly (one byte permute per half: bytes b0, 0x64, b2, 0x64
// and b1, 0x64, b3, 0x64)
__device__ __forceinline__ void i16_split_word(uint32_t q, uint32_t& hi, uint32_t& lo)
{
    const uint32_t lb = __byte_perm(q, 0x64646464u, 0x4240);
    const uint32_t hb = __byte_perm(q, 0x64646464u, 0x4341);
    __half2 l2 = *reinterpret_cast<const __half2*>(&lb);
    __half2 h2 = *reinterpret_cast<const __half2*>(&hb);
    l2 = __hsub2(l2, __float2half2_rn(1024.0f));
    h2 = __hmul2(__hsub2(h2, __float2half2_rn(1152.0f)), __float2half2_rn(256.0f));
    hi = *reinterpret_cast<const uint32_t*>(&h2);
    lo = *reinterpret_cast<const uint32_t*>(&l2);
}

// the power-of-two scale of vector r's far-field values on a mesh
__device__ __forceinline__ float tc_scale(float wbound, const int* xmax, int r)
{
    const float xm = __int_as_float(xmax[r]);
    const float b = wbound * xm;
    if (!(b > 0.0f) || !isfinite(b)) return 1.0f;
    return exp2f(floorf(log2f(32768.0f / b)));
}

// where the low bytes of an INT16 far stage's split go: right after its U in
// the stage region when both halves fit there (then a warp other than the
// builder splits the stage while the builder builds A), otherwise into the
// 4-vector region once the builder has read w from it
__device__ __forceinline__ uint32_t tc_lo_offset(int count, int mp)
{
    const int ub = count * mp * 2;  // bytes of the stage's U (a multiple of 256)
    return 2 * ub <= kTcStage ? (uint32_t)ub : (uint32_t)kTcStage;
}

// split an INT16 stage of nch 16-byte chunks: 256 x high bytes in place, the
// low bytes lo16 chunks further on
__device__ __forceinline__ void tc_split_stage(uint4* Us, int nch, int lo16, int lane)
{
    for (int e = lane; e < nch; e += 32) {
        const uint4 v = Us[e];
        uint4 hv, lv;
        i16_split_word(v.x, hv.x, lv.x);
        i16_split_word(v.y, hv.y, lv.y);
        i16_split_word(v.z, hv.z, lv.z);
        i16_split_word(v.w, hv.w, lv.w);
        Us[e] = hv;
        Us[e + lo16] = lv;
    }
}

template <class TF>
__global__ void __launch_bounds__(kThreads) leaf_tc_kernel(
    const int2* __restrict__ work, int nwork, const MeshDev* __restrict__ meshes, int* __restrict__ counter,
    int* __restrict__ err, const float* __restrict__ xg_base, const float* __restrict__ w_base, int G,
    const int* __restrict__ xmax, uint32_t tmem_cols, double* __restrict__ y, int64_t ld)
{
    using TA = float;
    using TN = float;
    constexpr int Rr = 8;  // rows per consumer thread in the near field (as for 16-bit U)
    constexpr int RC = 2;
    constexpr bool kI16 = std::is_same<TF, int16_t>::value;
    constexpr bool kBf16 = std::is_same<TF, __nv_bfloat16>::value;
    using TO = typename std::conditional<kBf16, __nv_bfloat16, __half>::type;  // the operand type
    extern __shared__ __align__(128) unsigned char smem[];
    auto sdata = [&](int q) { return smem + (size_t)q * kTcSlotBytes; };
    auto saux = [&](int q) { return smem + (size_t)q * kTcSlotBytes + kTcStage; };
    unsigned char* abuf = smem + (size_t)kTcSlots * kTcSlotBytes;  // one A tile per builder warp
    __shared__ __align__(8) uint64_t full[kTcSlots];
    __shared__ __align__(8) uint64_t empty[kTcSlots];      // every stage: one arrival per consumer warp
    __shared__ __align__(8) uint64_t empty_far[kTcSlots];  // far stages, also: the MMA commit
    __shared__ __align__(8) uint64_t afull[kTcBuildW];     // a builder's A tile is built
    __shared__ __align__(8) uint64_t aempty[kTcBuildW];    // a builder's A tile is read by its MMAs
    __shared__ __align__(8) uint64_t dbar;                 // a leaf's far MMAs are done
    __shared__ __align__(8) uint64_t fbar;                 // drain
    __shared__ StageMeta meta[kTcSlots];
    __shared__ uint32_t tmem_slot;

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (threadIdx.x == 0) {
        for (int s = 0; s < kTcSlots; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], kConsumers / 32);
            mbar_init(&empty_far[s], 1);
        }
        for (int b = 0; b < kTcBuildW; ++b) {
            mbar_init(&afull[b], kI16 ? 2 : 1);  // INT16: the builder and the splitter
            mbar_init(&aempty[b], 1);
        }
        mbar_init(&dbar, 1);
        mbar_init(&fbar, 1);
        mbar_fence_init();
    }
    if (warp == 1) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                         smem_addr(&tmem_slot)),
                     "r"(tmem_cols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    // the rows of the A tiles that no builder writes stay zero
    for (int e = threadIdx.x; e < kTcBuildW * kTcABytes / 16; e += kThreads)
        reinterpret_cast<uint4*>(abuf)[e] = make_uint4(0u, 0u, 0u, 0u);
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = tmem_slot;

    if (warp == 0) {
        leaf_producer<TF, TN, TA, kTcSlots, kTcStage, kTcAux, 16, kTcK, true>(
            work, nwork, meshes, counter, err, xg_base, w_base, G, smem, full, empty, meta, empty_far);
        return;
    }

    // ---------------------------------------------------------------- consumers
    // warps 2..4 build the A tiles of the far stages (far stage f by warp
    // 2 + f mod 3), lane 0 of warp 1 issues the MMAs; the other warps go on to
    // the near stages meanwhile, and warps 4..7 read the accumulators (TMEM
    // lane quarters 0..3) in the epilogue
    const int ctid = threadIdx.x - 32;
    const bool builder = warp >= 2 && warp < 2 + kTcBuildW;
    const int NRC = (G + RC - 1) / RC;
    int cur = -1, cur_mesh = -1, P = 1, H = 0, p = 0, c = 0, h = 0, t0 = 0, mt = 0, mp = 8, mp16 = 16;
    const int32_t* perm = nullptr;
    int64_t xoff = 0;
    TA c1 = 0.f, c2 = 0.f;
    float wbound = 0.f;
    float tl = 0.f;  // a builder lane's t_r, r = lane mod 16 (0: a vector beyond G)
    int fs = 0;   // far stages seen (the builder, the use of its A tile, the MMA turn)
    int nfl = 0;  // leaves with a far field finished (phase of dbar)
    bool far_started = false;
    TA acc[Rr][RC][3];
    for (int it = 0;; ++it) {
        const int slot = it % kTcSlots;
        if (!mbar_wait(&full[slot], (uint32_t)(it / kTcSlots) & 1u, err, 3, it)) break;
        const StageMeta m = meta[slot];
        if (m.kind == 2) break;
        if (m.leaf != cur || m.pad[0] != cur_mesh) {
            cur = m.leaf;
            cur_mesh = m.pad[0];
            const MeshDev& md = meshes[cur_mesh];
            t0 = md.leaf[2 * cur];
            mt = md.leaf[2 * cur + 1];
            perm = md.perm;
            xoff = md.xoff;
            c1 = (TA)md.c1;
            c2 = (TA)md.c2;
            wbound = md.wbound;
            if (builder) tl = (lane & 15) < G ? tc_scale(wbound, xmax, lane & 15) : 0.0f;
            mp = (mt + 7) & ~7;
            mp16 = (mt + 15) & ~15;
            P = mp / Rr;
            H = kConsumers / (P * NRC);
            p = ctid % P;
            c = (ctid / P) % NRC;
            h = ctid / (P * NRC);
            far_started = false;
#pragma unroll
            for (int e = 0; e < Rr; ++e)
#pragma unroll
                for (int q = 0; q < RC; ++q) acc[e][q][0] = acc[e][q][1] = acc[e][q][2] = (TA)0;
        }
        if (m.kind == 0) {
            // ---- far stage on the tensor cores
            const int f = fs++;
            const bool first_far = !far_started;
            far_started = true;
            const int own = f % kTcBuildW;  // its builder: warp 2 + own
            const int use = f / kTcBuildW;  // that builder's use of its A tile
            unsigned char* A = abuf + (size_t)own * kTcABytes;
            if (warp == 1) {
                // the issuer: the stage's MMAs once its A tile is built
                int ok = 1;
                if (lane == 0) {
                    ok = mbar_wait(&afull[own], (uint32_t)use & 1u, err, 4, it) ? 1 : 0;
                    if (ok) {
                        tc_fence_after();
                        const uint32_t a0 = smem_addr(A), b0 = smem_addr(sdata(slot));
                        const uint32_t kstride = (uint32_t)(mp >> 3) * 128;  // K-direction core stride of U
                        const uint32_t bl0 = b0 + (kI16 ? tc_lo_offset(m.count, mp) : 0u);  // INT16 low bytes
                        for (int ks = 0; ks < (m.count >> 4); ++ks) {
                            for (int n0 = 0; n0 < mp16; n0 += 256) {
                                const int n = min(256, mp16 - n0);
                                const uint64_t ad = tc_desc(a0 + (uint32_t)ks * 256, 128, kTcSbo);
                                const uint64_t bd = tc_desc(b0 + (uint32_t)ks * 2 * kstride + (uint32_t)(n0 >> 3) * 128,
                                                            kstride, 128);
                                tc_mma(tmem + (uint32_t)n0, ad, bd, tc_idesc(n, kBf16),
                                       (!first_far || ks > 0) ? 1u : 0u);
                                if (kI16) {
                                    const uint64_t bl = tc_desc(bl0 + (uint32_t)ks * 2 * kstride + (uint32_t)(n0 >> 3) * 128,
                                                                kstride, 128);
                                    tc_mma(tmem + (uint32_t)n0, ad, bl, tc_idesc(n, kBf16), 1u);
                                }
                            }
                        }
                        tc_commit(&aempty[own]);
                        tc_commit(&empty_far[slot]);
                        if (m.pad[1]) tc_commit(&dbar);
                    }
                }
                if (!__shfl_sync(0xffffffffu, ok, 0)) break;
                __syncwarp();
                if (lane == 0) mbar_arrive(&empty[slot]);  // the warp has passed the stage
                continue;
            }
            if (!builder || warp - 2 != own) {
                if (kI16 && warp == 2 + kTcBuildW + own) {
                    // the splitter of this stage (warps 5..7): the split, where
                    // it goes into the stage region, while the builder builds A
                    const uint32_t lo = tc_lo_offset(m.count, mp);
                    if (lo < (uint32_t)kTcStage)
                        tc_split_stage(reinterpret_cast<uint4*>(sdata(slot)), m.count * (mp >> 3), (int)(lo >> 4),
                                       lane);
                    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                    __syncwarp();
                    if (lane == 0) mbar_arrive(&afull[own]);
                }
                __syncwarp();
                if (lane == 0) mbar_arrive(&empty[slot]);
                continue;
            }
            // the builder of this stage: its A tile is free once the MMAs of its
            // previous use are done
            if (use > 0 && !mbar_wait(&aempty[own], (uint32_t)(use - 1) & 1u, err, 8, it)) break;
            const float* av = reinterpret_cast<const float*>(saux(slot));
            const int nkb = m.count >> 3;  // core columns of this stage
            // item (r, kb): vector r = lane mod 16, segments 8 kb .. 8 kb + 7;
            // its rows 16 a + r (hi) and 64 + 16 a + r (lo) are row r mod 8 of
            // the cores 2 a + r / 8 and 8 + 2 a + r / 8 of core column kb
            const int r = lane & 15;
            if (r < G) {
                for (int kb = lane >> 4; kb < nkb; kb += 2) {
                    uint32_t hw[3][4], lw[3][4];
#pragma unroll
                    for (int s2 = 0; s2 < 4; ++s2) {
                        const float4 x0 = *reinterpret_cast<const float4*>(av + ((size_t)(kb * 8 + 2 * s2) * G + r) * 4);
                        const float4 x1 =
                            *reinterpret_cast<const float4*>(av + ((size_t)(kb * 8 + 2 * s2 + 1) * G + r) * 4);
                        tc_split2<TO>(x0.x * tl, x1.x * tl, hw[0][s2], lw[0][s2]);
                        tc_split2<TO>(x0.y * tl, x1.y * tl, hw[1][s2], lw[1][s2]);
                        tc_split2<TO>(x0.z * tl, x1.z * tl, hw[2][s2], lw[2][s2]);
                    }
#pragma unroll
                    for (int a = 0; a < 3; ++a) {
                        const size_t o = (size_t)((2 * a + (r >> 3)) * (kTcK / 8) + kb) * 128 + (r & 7) * 16;
                        *reinterpret_cast<uint4*>(A + o) = make_uint4(hw[a][0], hw[a][1], hw[a][2], hw[a][3]);
                        *reinterpret_cast<uint4*>(A + o + (size_t)8 * (kTcK / 8) * 128) =
                            make_uint4(lw[a][0], lw[a][1], lw[a][2], lw[a][3]);
                    }
                }
            }
            if constexpr (kI16) {
                // a stage whose split does not fit its region: the low bytes go
                // into the 4-vector region right after it, once the warp is done
                // reading w from it
                if (tc_lo_offset(m.count, mp) == (uint32_t)kTcStage) {
                    __syncwarp();
                    tc_split_stage(reinterpret_cast<uint4*>(sdata(slot)), m.count * (mp >> 3), kTcStage / 16, lane);
                }
            }
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            tc_fence_before();
            __syncwarp();
            if (lane == 0) {
                mbar_arrive(&afull[own]);
                mbar_arrive(&empty[slot]);  // the warp has passed the stage
            }
            continue;
        }
        // ---- near stage on the CUDA cores (as in the multi-vector kernel)
        const TA* av = reinterpret_cast<const TA*>(saux(slot)) + (size_t)c * RC * 4;
        if (kI16 && m.kind == 3 && h < H) {
            // INT16 near columns: six FP32 scales, then six segments of int16;
            // the scales are folded into the coefficients of x (V_aa enters y_a
            // with (c1 + c2) x_a and the other components with c1 x_b; V_ab,
            // a != b, enters y_a with c2 x_b and y_b with c2 x_a)
            const unsigned char* sb3 = sdata(slot);
            const int colB16 = kNear16Head + 12 * mp;
            const TA c12 = c1 + c2;
            for (int s = h; s < m.count; s += H) {
                const unsigned char* col = sb3 + (size_t)s * colB16;
                const float4 sa = *reinterpret_cast<const float4*>(col);       // s11 s12 s13 s22
                const float2 sz = *reinterpret_cast<const float2*>(col + 16);  // s23 s33
                const TA sc[6] = {sa.x, sa.y, sa.z, sa.w, sz.x, sz.y};
                const int16_t* e0 = reinterpret_cast<const int16_t*>(col + kNear16Head) + p * Rr;
                TA xs[RC][3];
#pragma unroll
                for (int q = 0; q < RC; ++q) {
                    if (c * RC + q < G) load3(av + ((size_t)s * G + q) * 4, xs[q][0], xs[q][1], xs[q][2]);
                    else xs[q][0] = xs[q][1] = xs[q][2] = (TA)0;
                }
#pragma unroll
                for (int v = 0; v < 6; ++v) {
                    const int va = v < 3 ? 0 : (v < 5 ? 1 : 2);
                    const int vb = v < 3 ? v : (v < 5 ? v - 2 : 2);
                    TA val[Rr];
                    smem_rows<int16_t, TA, Rr>(e0 + v * mp, val);
#pragma unroll
                    for (int q = 0; q < RC; ++q) {
                        if (va == vb) {
                            const TA f0 = (va == 0 ? c12 : c1) * sc[v] * xs[q][0];
                            const TA f1 = (va == 1 ? c12 : c1) * sc[v] * xs[q][1];
                            const TA f2 = (va == 2 ? c12 : c1) * sc[v] * xs[q][2];
#pragma unroll
                            for (int e = 0; e < Rr; ++e) {
                                acc[e][q][0] += f0 * val[e];
                                acc[e][q][1] += f1 * val[e];
                                acc[e][q][2] += f2 * val[e];
                            }
                        } else {
                            const TA fa = c2 * sc[v] * xs[q][vb], fb = c2 * sc[v] * xs[q][va];
#pragma unroll
                            for (int e = 0; e < Rr; ++e) {
                                acc[e][q][va] += fa * val[e];
                                acc[e][q][vb] += fb * val[e];
                            }
                        }
                    }
                }
            }
        } else if (h < H) {
            const TN* sb = reinterpret_cast<const TN*>(sdata(slot)) + p * Rr;
            const TA c12 = c1 + c2;
            for (int s = h; s < m.count; s += H) {
                const TN* e0 = sb + (size_t)s * 6 * mp;
                TA xs[RC][3];
#pragma unroll
                for (int q = 0; q < RC; ++q) {
                    if (c * RC + q < G) load3(av + ((size_t)s * G + q) * 4, xs[q][0], xs[q][1], xs[q][2]);
                    else xs[q][0] = xs[q][1] = xs[q][2] = (TA)0;
                }
#pragma unroll
                for (int v = 0; v < 6; ++v) {
                    const int va = v < 3 ? 0 : (v < 5 ? 1 : 2);
                    const int vb = v < 3 ? v : (v < 5 ? v - 2 : 2);
                    TA val[Rr];
                    smem_rows<TN, TA, Rr>(e0 + v * mp, val);
#pragma unroll
                    for (int q = 0; q < RC; ++q) {
                        if (va == vb) {
                            const TA f0 = (va == 0 ? c12 : c1) * xs[q][0];
                            const TA f1 = (va == 1 ? c12 : c1) * xs[q][1];
                            const TA f2 = (va == 2 ? c12 : c1) * xs[q][2];
#pragma unroll
                            for (int e = 0; e < Rr; ++e) {
                                acc[e][q][0] += f0 * val[e];
                                acc[e][q][1] += f1 * val[e];
                                acc[e][q][2] += f2 * val[e];
                            }
                        } else {
                            const TA fa = c2 * xs[q][vb], fb = c2 * xs[q][va];
#pragma unroll
                            for (int e = 0; e < Rr; ++e) {
                                acc[e][q][va] += fa * val[e];
                                acc[e][q][vb] += fb * val[e];
                            }
                        }
                    }
                }
            }
        }
        if (m.last) {
            named_barrier_consumers();  // everyone is done reading the slot
            const bool has_far = far_started;
            if (has_far) {
                // ---- far epilogue: D (TMEM) -> y, hi + lo rows added, t_r removed
                if (!mbar_wait(&dbar, (uint32_t)nfl & 1u, err, 5, it)) break;
                ++nfl;
                tc_fence_after();
                float* X = reinterpret_cast<float*>(sdata(slot));  // lo rows [64][64 columns]
                const int q4 = warp & 3;                          // TMEM lane quarter of this warp
                const bool reader = warp >= 4;                    // warps 4..7 cover lanes 0..127
                for (int c0 = 0; c0 < mp16; c0 += 64) {
                    const int nc = min(64, mp16 - c0);
                    if (reader && q4 >= 2) {
                        const int row = 32 * q4 + lane - 64;
                        for (int cc = 0; cc < nc; cc += 8) {
                            float v[8];
                            tc_ld8(tmem + ((uint32_t)(32 * q4) << 16) + (uint32_t)(c0 + cc), v);
#pragma unroll
                            for (int q = 0; q < 8; ++q) X[row * 64 + cc + q] = v[q];
                        }
                    }
                    named_barrier_consumers();
                    if (reader && q4 < 2) {
                        const int row = 32 * q4 + lane;
                        const int r = row & 15, a = row >> 4;
                        const float inv = 1.0f / tc_scale(wbound, xmax, r);
                        for (int cc = 0; cc < nc; cc += 8) {
                            float v[8];
                            tc_ld8(tmem + ((uint32_t)(32 * q4) << 16) + (uint32_t)(c0 + cc), v);
                            if (a < 3 && r < G) {
#pragma unroll
                                for (int q = 0; q < 8; ++q) {
                                    const int i = c0 + cc + q;
                                    if (i < mt)
                                        y[(size_t)r * ld + xoff + 3 * (size_t)perm[t0 + i] + a] =
                                            (double)((v[q] + X[row * 64 + cc + q]) * inv);
                                }
                            }
                        }
                    }
                    __threadfence_block();
                    tc_fence_before();
                    named_barrier_consumers();
                }
                tc_fence_after();
            }
            // ---- near field: the H partial sums, added to the far result
            TA* red = reinterpret_cast<TA*>(sdata(slot));
            constexpr int kPer = Rr * 3;
#pragma unroll
            for (int q = 0; q < RC; ++q) {
                if (h < H) {
                    TA* rp = red + (size_t)((h * P + p) * NRC + c) * kPer;
#pragma unroll
                    for (int e = 0; e < Rr; ++e)
#pragma unroll
                        for (int a = 0; a < 3; ++a) rp[e * 3 + a] = acc[e][q][a];
                }
                named_barrier_consumers();
                const int nvec = (G - q + RC - 1) / RC;
                const int per_row = 3 * nvec;
                for (int idx = ctid; idx < mt * per_row; idx += kConsumers) {
                    const int i = idx / per_row, rem = idx - i * per_row;
                    const int cc = rem / 3, a = rem - 3 * cc;
                    const int pp = i / Rr, e = i - pp * Rr;
                    TA sum = (TA)0;
                    for (int g = 0; g < H; ++g) sum += red[(size_t)((g * P + pp) * NRC + cc) * kPer + e * 3 + a];
                    const int r = cc * RC + q;
                    double* yp = y + (size_t)r * ld + xoff + 3 * (size_t)perm[t0 + i] + a;
                    *yp = has_far ? *yp + (double)sum : (double)sum;
                }
                named_barrier_consumers();
            }
        }
        // the slot may be refilled once every consumer warp is done with it
        __syncwarp();
        if (lane == 0) mbar_arrive(&empty[slot]);
    }
    // ---- drain: no MMA may still run when the tensor memory is released
    tc_fence_before();
    named_barrier_consumers();
    if (ctid == 0 && fs > 0) {
        tc_fence_after();
        tc_commit(&fbar);
        mbar_wait(&fbar, 0u, err, 6, 0);
    }
    tc_fence_before();
    named_barrier_consumers();
    tc_fence_after();
    if (warp == 1)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(tmem_cols) : "memory");
}

}  // namespace stream
}  // namespace hm
