// hm_fwd_tc.cuh -- the far-field forward pass z = V^T x on the tensor cores
// (tcgen05), for the FP16 / BF16 / INT16 forms and up to 16 right-hand sides
// a launch.
//
// A forward group holds the V of the admissible blocks that share a column
// cluster s, side by side (Section 2: each block contributes w = c V^T x(s)).
// A unit is rows j0 .. j0 + 255 and columns c0 .. c0 + 255 of a group; for
// it the kernel computes
//   D[m, c] = sum_j A[m, j] V[j, c]
// with M = 128, N = the unit's columns (rounded up to 16), K = 16 rows per
// MMA, accumulating in tensor memory:
//   B = V, streamed 32 rows (a stage) at a time by one bulk copy each
//       straight into the MN-major core-matrix layout (the 16-bit V of a
//       unit is stored contiguously in 8 x 8 tiles).  INT16 values (offset
//       binary q = v + 32768) are split in shared memory into two FP16
//       operands of the same layout, 256 (q / 256 - 128) and q mod 256, both
//       exact, whose MMAs accumulate into the same rows;
// Every ring is used in stage order by each of its waiting threads, or (the
// A ring, filled by the builder warps round-robin) has a multiple of their
// number of slots, so that no wait can see a barrier's parity of two phases
// before.
//   A = x(s) of the G vectors, scaled by a power of two t_r per vector (from
//       max|x_r|, so that every value fits FP16) and split into hi = fp16(x
//       t_r) and lo = fp16(x t_r - hi): two K-major core-matrix tiles whose
//       MMAs accumulate into the same rows (hi and lo stacked along K), so a
//       TMEM row holds t_r times the result.  A lane quarter q (32 rows) holds
//       eight vectors: row 32 q + 4 k + a is component a of vector
//       8 (q mod nq) + k (nq = ceil(G / 8) distinct quarters; the quarters
//       repeat, and the warps that read copies of the same vectors split the
//       columns).
// Persistent CTAs (one per SM) take the units round-robin (largest first)
// with specialised warps:
//   warp 0      producer: the V of every stage of every unit through a ring
//               of slots (bulk copies);
//   warps 2-5   build the A tiles from the gathered x into a second ring, a
//               stage each round-robin, ahead of the V stream (INT16 form
//               with at most 8 vectors: warps 2-3 only);
//   warps 14-15 (and 4-5 where they build nothing) INT16 form: split every
//               stage's V once it has landed, in stage order, each its share
//               of the 16-byte chunks (256 x high bytes in place, the low
//               bytes into a ring of two buffers that the MMA commits
//               release);
//   warp 1      one thread issues the MMAs of a stage and commits them to the
//               release barriers of its V and A slots, and after a unit's last
//               stage to its accumulator barrier; two accumulators (2 x 256
//               TMEM columns) let a unit's epilogue overlap the next unit's
//               MMAs;
//   warps 6-13  epilogue, four warps (one per lane quarter) per accumulator:
//               add the hi and lo rows, remove t_r and write w through the
//               precomputed column descriptors (factor column, kernel
//               components, c1 su or c2 su), or the unit's partial sums for
//               the second pass of a tall group; the TMEM read of the next 32
//               columns overlaps the writes of the current ones.
// Every wait is bounded.  A thread whose wait runs out raises a shared abort
// flag that ends every other wait; before the tensor memory is freed the CTA
// waits (bounded) for its copies and MMAs in flight.
#pragma once

#include "hm_leaf_tc.cuh"

namespace hm {
namespace stream {

constexpr int kFpThreads = 512;
constexpr int kFpRows = 32;                          // rows (K) per stage: two MMA K steps
constexpr int kFpCols = 256;                         // columns per unit at most (one N tile)
constexpr int kFpVBytes = kFpRows * kFpCols * 2;     // V of a stage
constexpr int kFpAHalf = 128 * kFpRows * 2;          // the hi (or lo) tile of a stage
constexpr int kFpABytes = 2 * kFpAHalf;              // A of a stage: hi tile, lo tile
constexpr int kFpVSlots = 7;                         // slots of the ring of V (16-bit floats)
constexpr int kFpASlots = 4;
constexpr int kFpSbo = (kFpRows / 8) * 128;          // M-direction core stride of an A tile
constexpr int kFpBld = 33;                           // row stride of an epilogue warp's buffer
constexpr int kFpBBytes = 32 * kFpBld * 4;           // one epilogue warp's buffer: 32 columns x 32 rows
// the rings of a form: INT16 takes fewer V slots (the 256 x high bytes of
// the split replace the stage) and a ring of LS buffers for the low bytes
template <class TF>
struct FpCfg {
    static constexpr bool kI16 = std::is_same<TF, int16_t>::value;
    static constexpr int VS = kI16 ? 5 : kFpVSlots;
    static constexpr int LS = kI16 ? 2 : 0;
    static constexpr int AS = kFpASlots;
    static constexpr size_t smem()
    {
        return (size_t)(VS + LS) * kFpVBytes + (size_t)AS * kFpABytes + 8 * (size_t)kFpBBytes;
    }
};
static_assert(kFpASlots % 4 == 0, "four (or two) builder warps take the A slots round-robin");

// A-builder warps of a launch (warps 2 .. 1 + nb); the INT16 form splits V
// on the other warps of 2-5 and on 14-15.  The builds grow with the vectors,
// the split does not: level 6, INT16, four builders and two converters
// against two and four: 4 vectors 1.57 against 1.38 ms, 8 vectors 1.83
// against 1.64 ms, 16 vectors 2.08 against 2.11 ms (one builder and five
// converters: 2.02, 2.42, 3.19 ms)
template <class TF>
__host__ __device__ constexpr int fp_builders(int ng)
{
    return std::is_same<TF, int16_t>::value && ng <= 8 ? 2 : 4;
}
template <class TF>
constexpr size_t fp_smem()
{
    return FpCfg<TF>::smem();
}

constexpr int kFpMeshes = 64;                        // meshes whose pointers are kept in shared memory
static_assert(kFpCols == kFwdUnitCols, "a unit is one N tile");
static_assert(kFwdUnitRows % kFpRows == 0, "a unit is whole stages, but its last one");

// what the roles need of a unit's mesh
struct FpMesh {
    const void* Vr;
    const uint2* fdesc;
    int64_t xgoff, woff;
};

// bounded wait that also ends when another thread has raised the abort
// flag; between polls the thread sleeps (32 ns doubling to 512 ns), so that
// the waiting warps leave the issue slots and the shared-memory pipe to the
// working ones
__device__ __forceinline__ bool fp_wait(uint64_t* bar, uint32_t parity, volatile int* abort_flag, int* err, int site,
                                        int stage)
{
    if (mbar_try_wait(bar, parity)) return true;
    const long long t0 = clock64();
    uint32_t ns = 32;
    for (;;) {
        __nanosleep(ns);
        if (mbar_try_wait(bar, parity)) return true;
        if (ns < 512) ns <<= 1;
        if (*abort_flag) return false;
        if (clock64() - t0 > kWaitCycles) {
            if (atomicCAS(err + 1, 0, site) == 0) {
                err[2] = stage;
                err[3] = (int)blockIdx.x;
            }
            atomicExch(err, 1);
            *abort_flag = 1;
            return false;
        }
    }
}

// 32 consecutive FP32 columns of this thread's TMEM lane: the load is issued
// by fp_ld32_issue and its registers are complete after fp_ld32_wait (which
// names them, so that no use moves above it)
__device__ __forceinline__ void fp_ld32_issue(uint32_t addr, uint32_t* r)
{
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
        "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
          "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
          "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
        : "r"(addr)
        : "memory");
}
__device__ __forceinline__ void fp_ld32_wait(uint32_t* r)
{
    asm volatile("tcgen05.wait::ld.sync.aligned;"
                 : "+r"(r[0]), "+r"(r[1]), "+r"(r[2]), "+r"(r[3]), "+r"(r[4]), "+r"(r[5]), "+r"(r[6]), "+r"(r[7]),
                   "+r"(r[8]), "+r"(r[9]), "+r"(r[10]), "+r"(r[11]), "+r"(r[12]), "+r"(r[13]), "+r"(r[14]),
                   "+r"(r[15]), "+r"(r[16]), "+r"(r[17]), "+r"(r[18]), "+r"(r[19]), "+r"(r[20]), "+r"(r[21]),
                   "+r"(r[22]), "+r"(r[23]), "+r"(r[24]), "+r"(r[25]), "+r"(r[26]), "+r"(r[27]), "+r"(r[28]),
                   "+r"(r[29]), "+r"(r[30]), "+r"(r[31])
                 :
                 : "memory");
}

template <class TF, bool ONE>
__global__ void __launch_bounds__(kFpThreads, 1) fwd_tc_kernel(
    const FwdTcUnit* __restrict__ units, int nunits, const __grid_constant__ MeshDev m0,
    const MeshDev* __restrict__ meshes, int nmesh, const float* __restrict__ xg, float* __restrict__ w,
    float* __restrict__ z, int G, const int* __restrict__ xmax, int* __restrict__ err)
{
    using Cfg = FpCfg<TF>;
    constexpr bool kI16 = Cfg::kI16;
    constexpr int VS = Cfg::VS, AS = Cfg::AS, LS = Cfg::LS;
    constexpr bool kBf16 = std::is_same<TF, __nv_bfloat16>::value;
    using TO = typename std::conditional<kBf16, __nv_bfloat16, __half>::type;  // the operand type
    extern __shared__ __align__(128) unsigned char smem[];
    __shared__ __align__(8) uint64_t vfull[kFpVSlots];   // the V of a stage has landed
    __shared__ __align__(8) uint64_t vconv[kFpVSlots];   // INT16: the V of a stage is split
    __shared__ __align__(8) uint64_t lempty[2];          // INT16: the MMAs that read a low-byte buffer are done
    __shared__ __align__(8) uint64_t vempty[kFpVSlots];  // the MMAs that read a V slot are done
    __shared__ __align__(8) uint64_t afull[kFpASlots];   // the A of a stage is built
    __shared__ __align__(8) uint64_t aempty[kFpASlots];  // the MMAs that read an A slot are done
    __shared__ __align__(8) uint64_t accf[2];            // an accumulator holds a finished unit
    __shared__ __align__(8) uint64_t acce[2];            // an accumulator is read out (4 warps)
    __shared__ __align__(8) uint64_t fbar;               // drain after an abort
    __shared__ float tsc[kTcMaxG];
    __shared__ float tinv[kTcMaxG];  // 1 / tsc (powers of two)
    __shared__ FpMesh smesh[kFpMeshes];
    __shared__ uint32_t tmem_slot;
    __shared__ int abort_sh;
    volatile int* abort_flag = &abort_sh;

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int ng = min(kTcMaxG, G);  // vectors of this launch
    const int nq = (ng + 7) >> 3;    // distinct quarter contents
    const int rep = 4 / nq;          // copies of each (4 or 2)
    const int nb = fp_builders<TF>(ng);  // A-builder warps (a power of two dividing AS)
    const int ncv = kI16 ? 6 - nb : 0;   // INT16 converter warps
    auto slot_v = [&](int s) { return smem + (size_t)s * kFpVBytes; };
    auto slot_l = [&](int s) { return smem + (size_t)(VS + s) * kFpVBytes; };
    auto slot_a = [&](int s) { return smem + (size_t)(VS + LS) * kFpVBytes + (size_t)s * kFpABytes; };
    if (tid == 0) {
        for (int s = 0; s < VS; ++s) {
            mbar_init(&vfull[s], 1);
            mbar_init(&vconv[s], ncv > 0 ? ncv : 1);  // one arrival per converter warp
            mbar_init(&vempty[s], 1);
        }
        for (int s = 0; s < LS; ++s) mbar_init(&lempty[s], 1);
        for (int s = 0; s < AS; ++s) {
            mbar_init(&afull[s], 1);
            mbar_init(&aempty[s], 1);
        }
        for (int b = 0; b < 2; ++b) {
            mbar_init(&accf[b], 1);
            mbar_init(&acce[b], 4);
        }
        mbar_init(&fbar, 1);
        abort_sh = 0;
        mbar_fence_init();
    }
    if (tid < kTcMaxG) {
        float t = 1.0f;
        if (tid < ng) {
            const float xm = __int_as_float(xmax[tid]);
            if (xm > 0.0f && isfinite(xm)) t = exp2f(floorf(log2f(32768.0f / xm)));
        }
        tsc[tid] = t;
        tinv[tid] = 1.0f / t;
    }
    for (int m = tid; m < (ONE ? 1 : min(nmesh, kFpMeshes)); m += kFpThreads) {
        const MeshDev& md = ONE ? m0 : meshes[m];
        smesh[m] = FpMesh{md.Vr, md.fdesc, md.xgoff, md.woff};
    }
    // A rows that no stage writes (vectors >= G, the fourth component) stay zero
    for (int e = tid; e < AS * kFpABytes / 16; e += kFpThreads)
        reinterpret_cast<uint4*>(slot_a(0))[e] = make_uint4(0u, 0u, 0u, 0u);
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                         smem_addr(&tmem_slot)),
                     "r"(512)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = tmem_slot;
    int issued = 0;  // stages whose V copy was issued (producer thread)
    auto mesh_of_unit = [&](int m) -> FpMesh {
        if (ONE) return smesh[0];
        if (m < kFpMeshes) return smesh[m];
        const MeshDev& md = meshes[m];
        return FpMesh{md.Vr, md.fdesc, md.xgoff, md.woff};
    };

    if (warp == 0) {
        // ---- producer
        if (lane == 0) {
            int it = 0;
            bool run = true;
            FwdTcUnit nx{};
            if ((int)blockIdx.x < nunits) nx = units[blockIdx.x];
            for (int u = blockIdx.x; u < nunits && run; u += gridDim.x) {
                const FwdTcUnit un = nx;
                if (u + (int)gridDim.x < nunits) nx = units[u + gridDim.x];  // the next unit, ahead of its use
                const TF* Vg = static_cast<const TF*>(mesh_of_unit(un.mesh).Vr) + un.v0;
                const int n16 = (un.nrows + 15) & ~15, cu = un.ncols;
                for (int q = 0; q * kFpRows < n16; ++q, ++it) {
                    const int slot = it % VS;
                    if (it >= VS &&
                        !fp_wait(&vempty[slot], (uint32_t)((it / VS) - 1) & 1u, abort_flag, err, 7, it)) {
                        run = false;
                        break;
                    }
                    // the stage's tiles are contiguous: one bulk copy
                    const int kr0 = q * (kFpRows / 8);
                    const int nkr = min(kFpRows / 8, (n16 >> 3) - kr0);
                    const uint32_t bytes = (uint32_t)(nkr * cu * 16);
                    mbar_arrive_expect_tx(&vfull[slot], bytes);
                    bulk_g2s(slot_v(slot), Vg + (size_t)kr0 * (size_t)un.ld8, bytes, &vfull[slot]);
                    issued = it + 1;
                }
            }
        }
    } else if (warp == 1) {
        // ---- MMA issue
        if (lane == 0) {
            int it = 0, i = 0;
            bool run = true;
            FwdTcUnit nx{};
            if ((int)blockIdx.x < nunits) nx = units[blockIdx.x];
            for (int u = blockIdx.x; u < nunits && run; u += gridDim.x, ++i) {
                const FwdTcUnit un = nx;
                if (u + (int)gridDim.x < nunits) nx = units[u + gridDim.x];
                const int n16 = (un.nrows + 15) & ~15, cu = un.ncols, nN = (cu + 15) & ~15;
                const int ab = i & 1;
                if (i >= 2 && !fp_wait(&acce[ab], (uint32_t)((i >> 1) - 1) & 1u, abort_flag, err, 8, i)) break;
                tc_fence_after();
                const uint32_t d = tmem + (uint32_t)(ab * kFpCols);
                const uint32_t idesc = tc_idesc(nN, kBf16);
                const uint32_t kstride = (uint32_t)cu * 16;  // K-direction core stride of V
                for (int q = 0; q * kFpRows < n16; ++q, ++it) {
                    const int vs = it % VS, as = it % AS;
                    if (!fp_wait(kI16 ? &vconv[vs] : &vfull[vs], (uint32_t)(it / VS) & 1u, abort_flag, err, 9, it) ||
                        !fp_wait(&afull[as], (uint32_t)(it / AS) & 1u, abort_flag, err, 10, it)) {
                        run = false;
                        break;
                    }
                    tc_fence_after();
                    const uint32_t a0 = smem_addr(slot_a(as)), b0 = smem_addr(slot_v(vs));
                    const int steps = min(kFpRows / 16, (n16 >> 4) - q * (kFpRows / 16));
                    for (int ks = 0; ks < steps; ++ks) {
                        const uint64_t ah = tc_desc(a0 + (uint32_t)ks * 256, 128, kFpSbo);
                        const uint64_t al = tc_desc(a0 + kFpAHalf + (uint32_t)ks * 256, 128, kFpSbo);
                        const uint64_t bd = tc_desc(b0 + (uint32_t)ks * 2 * kstride, kstride, 128);
                        tc_mma(d, ah, bd, idesc, (q > 0 || ks > 0) ? 1u : 0u);
                        tc_mma(d, al, bd, idesc, 1u);
                        if (kI16) {
                            // the low bytes of the split, in the stage's buffer
                            const uint64_t bl = tc_desc(smem_addr(slot_l(it % 2)) + (uint32_t)ks * 2 * kstride,
                                                        kstride, 128);
                            tc_mma(d, ah, bl, idesc, 1u);
                            tc_mma(d, al, bl, idesc, 1u);
                        }
                    }
                    tc_commit(&vempty[vs]);
                    tc_commit(&aempty[as]);
                    if (kI16) tc_commit(&lempty[it % 2]);
                }
                if (run) tc_commit(&accf[ab]);
            }
        }
    } else if (warp < 2 + nb) {
        // ---- A builders: warp bw builds the stages it with it % nb == bw; an
        // item is (8-row K block kb, vector r): 8 rows of x_r -> three hi and
        // three lo rows of 8 K values in every quarter that holds r
        const int bw = warp - 2;
        int it = 0;
        bool run = true;
        FwdTcUnit nx{};
        if ((int)blockIdx.x < nunits) nx = units[blockIdx.x];
        for (int u = blockIdx.x; u < nunits && run; u += gridDim.x) {
            const FwdTcUnit un = nx;
            if (u + (int)gridDim.x < nunits) nx = units[u + gridDim.x];
            const int n16 = (un.nrows + 15) & ~15;
            const int nst = (n16 + kFpRows - 1) / kFpRows;
            if (((bw - it) & (nb - 1)) >= nst) {  // no stage of this unit is ours
                it += nst;
                continue;
            }
            const float* x0 = xg + ((size_t)mesh_of_unit(un.mesh).xgoff + un.x0) * G * 4;
            for (int q = 0; q < nst; ++q, ++it) {
                if ((it & (nb - 1)) != bw) continue;
                const int as = it % AS;
                // the lanes of a warp decide together (they meet at __syncwarp)
                const bool got = it < AS ||
                                 fp_wait(&aempty[as], (uint32_t)((it / AS) - 1) & 1u, abort_flag, err, 11, it);
                if (!__all_sync(0xffffffffu, got)) {
                    run = false;
                    break;
                }
                unsigned char* A = slot_a(as);
                for (int itm = lane; itm < 4 * ng; itm += 32) {
                    const int kb = itm / ng, r = itm - kb * ng;
                    const float t = tsc[r];
                    float4 xv[8];
#pragma unroll
                    for (int i = 0; i < 8; ++i) {
                        const int j = q * kFpRows + kb * 8 + i;
                        xv[i] = make_float4(0.f, 0.f, 0.f, 0.f);
                        if (j < un.nrows) xv[i] = *reinterpret_cast<const float4*>(x0 + ((size_t)j * G + r) * 4);
                    }
                    uint32_t hw[3][4], lw[3][4];
#pragma unroll
                    for (int i = 0; i < 8; i += 2) {
                        const float va[2][3] = {{xv[i].x * t, xv[i].y * t, xv[i].z * t},
                                                {xv[i + 1].x * t, xv[i + 1].y * t, xv[i + 1].z * t}};
#pragma unroll
                        for (int a = 0; a < 3; ++a) tc_split2<TO>(va[0][a], va[1][a], hw[a][i >> 1], lw[a][i >> 1]);
                    }
                    const int k = r & 7;
                    for (int qq = r >> 3; qq < rep * nq; qq += nq)
#pragma unroll
                        for (int a = 0; a < 3; ++a) {
                            const int m = 32 * qq + 4 * k + a;
                            const size_t o = (size_t)((m >> 3) * (kFpRows / 8) + kb) * 128 + (m & 7) * 16;
                            *reinterpret_cast<uint4*>(A + o) = make_uint4(hw[a][0], hw[a][1], hw[a][2], hw[a][3]);
                            *reinterpret_cast<uint4*>(A + kFpAHalf + o) =
                                make_uint4(lw[a][0], lw[a][1], lw[a][2], lw[a][3]);
                        }
                }
                asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                __syncwarp();
                if (lane == 0) mbar_arrive(&afull[as]);
            }
        }
    } else if (warp < 6 || warp >= 14) {
        // ---- INT16: split every stage's V in stage order once it has landed
        // (and its low-byte buffer is free): 256 x high bytes in place, the
        // low bytes into the buffer; converter h (warps 2 + nb .. 5, then 14
        // and 15) takes the groups of 32 16-byte chunks h, h + ncv, ...
        const int cw = warp < 6 ? warp - 2 - nb : warp - 14 + (4 - nb);
        if constexpr (kI16) {
            int it = 0;
            bool run = true;
            FwdTcUnit nx{};
            if ((int)blockIdx.x < nunits) nx = units[blockIdx.x];
            for (int u = blockIdx.x; u < nunits && run; u += gridDim.x) {
                const FwdTcUnit un = nx;
                if (u + (int)gridDim.x < nunits) nx = units[u + gridDim.x];
                const int n16 = (un.nrows + 15) & ~15;
                for (int q = 0; q * kFpRows < n16; ++q, ++it) {
                    const int vs = it % VS, ls = it % 2;
                    bool got = fp_wait(&vfull[vs], (uint32_t)(it / VS) & 1u, abort_flag, err, 15, it);
                    if (got && it >= 2)
                        got = fp_wait(&lempty[ls], (uint32_t)((it / 2) - 1) & 1u, abort_flag, err, 16, it);
                    if (!__all_sync(0xffffffffu, got)) {
                        run = false;
                        break;
                    }
                    uint4* V = reinterpret_cast<uint4*>(slot_v(vs));
                    uint4* L = reinterpret_cast<uint4*>(slot_l(ls));
                    const int nkr = min(kFpRows / 8, (n16 >> 3) - q * (kFpRows / 8));
                    const int nch = nkr * un.ncols;  // 16-byte chunks of the stage
                    for (int e = 32 * cw + lane; e < nch; e += 32 * ncv) {
                        const uint4 v = V[e];
                        uint4 h, l;
                        i16_split_word(v.x, h.x, l.x);
                        i16_split_word(v.y, h.y, l.y);
                        i16_split_word(v.z, h.z, l.z);
                        i16_split_word(v.w, h.w, l.w);
                        V[e] = h;
                        L[e] = l;
                    }
                    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                    __syncwarp();
                    if (lane == 0) mbar_arrive(&vconv[vs]);
                }
            }
        }
    } else {
        // ---- epilogue: warps 6-9 take the units with an even local index
        // (accumulator 0), warps 10-13 the odd ones (accumulator 1).  The warp
        // of quarter q reads vectors 8 (q mod nq) + k (lane l holds component
        // l % 4 of k = l / 4) and, of the 32-column rounds of the unit, those
        // with index = q / nq mod rep.
        const int e = (warp - 6) >> 2, quarter = warp & 3;
        float* B = reinterpret_cast<float*>(smem + (size_t)(VS + LS) * kFpVBytes + (size_t)AS * kFpABytes +
                                            (size_t)(warp - 6) * kFpBBytes);
        const int vb = 8 * (quarter % nq);                                // first vector of the quarter
        const int nk = quarter < rep * nq ? max(0, min(8, ng - vb)) : 0;  // vectors of the quarter
        const int sub = quarter / nq;                                     // this warp's share of the rounds
        // the descriptors of this lane's columns of a unit, loaded one unit
        // ahead (when the previous unit is done with the registers)
        uint2 dsc[kFpCols / 32];
        auto load_dsc = [&](const FwdTcUnit& un) {
            const FpMesh md = mesh_of_unit(un.mesh);
#pragma unroll
            for (int jj = 0; jj < kFpCols / 32; ++jj) {
                dsc[jj] = make_uint2(kFdSkip, 0u);
                if (un.z0 < 0 && nk > 0 && jj % rep == sub && jj * 32 + lane < un.ncols)
                    dsc[jj] = md.fdesc[(size_t)un.d0 + jj * 32 + lane];
            }
        };
        int i = e;
        const int u0 = blockIdx.x + e * gridDim.x;
        FwdTcUnit nx{};
        if (u0 < nunits) {
            nx = units[u0];
            load_dsc(nx);
        }
        for (int u = u0; u < nunits; u += 2 * gridDim.x, i += 2) {
            const FwdTcUnit un = nx;
            const bool more = u + 2 * (int)gridDim.x < nunits;
            if (more) nx = units[u + 2 * gridDim.x];
            const FpMesh md = mesh_of_unit(un.mesh);
            const int cu = un.ncols, nround = (cu + 31) >> 5;
            const bool got = fp_wait(&accf[e], (uint32_t)(i >> 1) & 1u, abort_flag, err, 12, i);
            if (!__all_sync(0xffffffffu, got)) break;
            tc_fence_after();
            float* wr = w + (size_t)md.woff * G * 4;
            float* zb = un.z0 >= 0 ? z + (size_t)un.z0 * G * 4 : nullptr;
            const uint32_t ta = tmem + ((uint32_t)(32 * quarter) << 16) + (uint32_t)(e * kFpCols);
            if (nk == 0 || sub >= nround) {
                // nothing of this unit to read
                tc_fence_before();
                __syncwarp();
                if (lane == 0) mbar_arrive(&acce[e]);
                if (more) load_dsc(nx);
                continue;
            }
            uint32_t rv[32];
            fp_ld32_issue(ta + (uint32_t)(sub * 32), rv);
#pragma unroll
            for (int jj = 0; jj < kFpCols / 32; ++jj) {
                if (jj >= nround) break;
                if (jj % rep != sub) continue;
                fp_ld32_wait(rv);
#pragma unroll
                for (int c = 0; c < 32; ++c) B[c * kFpBld + lane] = __uint_as_float(rv[c]);
                if (jj + rep >= nround) {
                    // this warp's last read of the accumulator
                    tc_fence_before();
                    __syncwarp();
                    if (lane == 0) mbar_arrive(&acce[e]);
                } else {
                    // the next round's columns, read while this round is written
                    fp_ld32_issue(ta + (uint32_t)((jj + rep) * 32), rv);
                }
                __syncwarp();
                const int c = jj * 32 + lane;  // this lane's column of the unit
                const float* bp = B + lane * kFpBld;
                if (c < cu && (zb || dsc[jj].x != kFdSkip)) {
                    // the column, decoded once for the quarter's vectors: output
                    // component a takes component s_a of z times f_a (V_pq enters
                    // y_p with x_q and, p != q, y_q with x_p; the third is zero)
                    int s0 = 0, s1 = 1, s2 = 2;
                    bool m0 = true, m1 = true, m2 = true;
                    float f = 1.0f;
                    float* d;
                    if (zb) {
                        d = zb + ((size_t)c * G + vb) * 4;
                    } else {
                        const uint32_t x = dsc[jj].x;
                        const int p = (int)((x >> 28) & 3u), pq = (int)(x >> 30);
                        f = __uint_as_float(dsc[jj].y);
                        if (p != 3) {
                            m0 = p == 0 || pq == 0;
                            m1 = p == 1 || pq == 1;
                            m2 = p == 2 || pq == 2;
                            s0 = p == 0 ? pq : p;
                            s1 = p == 1 ? pq : p;
                            s2 = p == 2 ? pq : p;
                        }
                        d = wr + ((size_t)(x & 0x0fffffffu) * G + vb) * 4;
                    }
#pragma unroll
                    for (int k = 0; k < 8; ++k) {
                        if (k >= nk) break;
                        const float fk = f * tinv[vb + k];  // a power of two times f: exact
                        const float* bk = bp + 4 * k;
                        *reinterpret_cast<float4*>(d + 4 * k) =
                            make_float4(m0 ? fk * bk[s0] : 0.0f, m1 ? fk * bk[s1] : 0.0f, m2 ? fk * bk[s2] : 0.0f, 0.0f);
                    }
                }
                __syncwarp();
            }
            if (more) load_dsc(nx);
        }
    }
    __syncthreads();
    if (*abort_flag) {
        // no copy may still write into shared memory and no MMA may still run
        // when the CTA frees its tensor memory and exits
        if (tid == 0)
            for (int q = max(0, issued - VS); q < issued; ++q)
                mbar_wait(&vfull[q % VS], (uint32_t)(q / VS) & 1u, err, 13, q);
        if (tid == 32) {
            tc_fence_after();
            tc_commit(&fbar);
            mbar_wait(&fbar, 0u, err, 14, 0);
        }
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(512) : "memory");
}

}  // namespace stream
}  // namespace hm
