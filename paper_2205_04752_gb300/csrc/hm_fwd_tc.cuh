// hm_fwd_tc.cuh -- the far-field forward pass z = V^T x on the tensor cores
// (tcgen05), for the FP16 / BF16 forms and up to 16 right-hand sides a launch.
//
// A forward group holds the V of the admissible blocks that share a column
// cluster s, side by side (Section 2: each block contributes w = c V^T x(s)).
// A unit is rows j0 .. j0 + 255 and columns c0 .. c0 + 255 of a group; for
// it the kernel computes
//   D[m, c] = sum_j A[m, j] V[j, c]
// with M = 128, N = the unit's columns (rounded up to 16), K = 16 rows per
// MMA, accumulating in tensor memory:
//   B = V, streamed 32 rows (a stage) at a time by bulk copies straight into
//       the MN-major core-matrix layout (the 16-bit V is stored in 8 x 8
//       tiles);
//   A = x(s) of the vectors r0 .. r0 + 15 of the launch, scaled by a power of
//       two t_r per vector (from max|x_r|, so that every value fits FP16) and
//       split into hi = fp16(x t_r) and lo = fp16(x t_r - hi), in a K-major
//       core-matrix layout.  Row m = 32 q + 16 h + 4 k + a holds component a
//       of vector r = q + 4 k, h = 0 for hi and 1 for lo: the hi and lo rows
//       of a value sit 16 TMEM lanes apart in the same lane quarter, so each
//       epilogue warp finishes its vectors alone.
// Persistent CTAs (one per SM) take the units round-robin (largest first)
// with specialised warps:
//   warp 0      producer: the V stages of every unit through a ring of slots;
//   warp 1      one thread issues the MMAs of a stage and commits them to the
//               slot's release barrier, and after a unit's last stage to its
//               accumulator barrier; two accumulators (2 x 256 TMEM columns)
//               let a unit's epilogue overlap the next unit's MMAs;
//   warps 2-5   build the A tile of a stage each, stages round-robin;
//   warps 6-13  epilogue, four warps (one per lane quarter) per accumulator:
//               add the hi and lo rows, remove t_r and write w through the
//               precomputed column descriptors (factor column, kernel
//               components, c1 su or c2 su), or the unit's partial sums for
//               the second pass of a tall group.
// Every wait is bounded.  A thread whose wait runs out raises a shared abort
// flag that ends every other wait; before the tensor memory is freed the CTA
// waits (bounded) for its copies and MMAs in flight.
#pragma once

#include "hm_leaf_tc.cuh"

namespace hm {
namespace stream {

constexpr int kFpThreads = 448;
constexpr int kFpRows = 32;                          // rows (K) per stage: two MMA K steps
constexpr int kFpCols = 256;                         // columns per unit at most (one N tile)
constexpr int kFpVBytes = kFpRows * kFpCols * 2;     // V of a stage
constexpr int kFpABytes = 128 * kFpRows * 2;         // A of a stage
constexpr int kFpSlotBytes = kFpVBytes + kFpABytes;
constexpr int kFpSlots = 7;
constexpr int kFpSbo = (kFpRows / 8) * 128;          // M-direction core stride of an A tile
constexpr int kFpBld = 33;                           // row stride of an epilogue warp's buffer
constexpr int kFpBBytes = 32 * kFpBld * 4;           // one epilogue warp's buffer
constexpr size_t fp_smem() { return (size_t)kFpSlots * kFpSlotBytes + 8 * (size_t)kFpBBytes; }
static_assert(kFpCols == kFwdUnitCols, "a unit is one N tile");
static_assert(kFwdUnitRows % kFpRows == 0, "a unit is whole stages, but its last one");

// bounded wait that also ends when another thread has raised the abort flag
__device__ __forceinline__ bool fp_wait(uint64_t* bar, uint32_t parity, volatile int* abort_flag, int* err, int site,
                                        int stage)
{
    if (mbar_try_wait(bar, parity)) return true;
    const long long t0 = clock64();
    for (;;) {
        if (mbar_try_wait(bar, parity)) return true;
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

// 32 consecutive FP32 columns of this thread's TMEM lane
__device__ __forceinline__ void fp_ld32(uint32_t addr, float* v)
{
    uint32_t r[32];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
        "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
          "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
          "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
        : "r"(addr)
        : "memory");
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int q = 0; q < 32; ++q) v[q] = __uint_as_float(r[q]);
}

template <class TF, bool ONE>
__global__ void __launch_bounds__(kFpThreads, 1) fwd_tc_kernel(
    const FwdUnit* __restrict__ units, int nunits, const FwdGroup* __restrict__ groups,
    const __grid_constant__ MeshDev m0, const MeshDev* __restrict__ meshes, const float* __restrict__ xg,
    float* __restrict__ w, float* __restrict__ z, int G, int r0, const int* __restrict__ xmax, int* __restrict__ err)
{
    constexpr bool kBf16 = !std::is_same<TF, __half>::value;
    extern __shared__ __align__(128) unsigned char smem[];
    __shared__ __align__(8) uint64_t vfull[kFpSlots];  // the V of a stage has landed
    __shared__ __align__(8) uint64_t afull[kFpSlots];  // the A of a stage is built
    __shared__ __align__(8) uint64_t empty[kFpSlots];  // the MMAs of a stage are done
    __shared__ __align__(8) uint64_t accf[2];          // an accumulator holds a finished unit
    __shared__ __align__(8) uint64_t acce[2];          // an accumulator is read out (4 warps)
    __shared__ __align__(8) uint64_t fbar;             // drain after an abort
    __shared__ float tsc[kTcMaxG];
    __shared__ uint32_t tmem_slot;
    __shared__ int abort_sh;
    volatile int* abort_flag = &abort_sh;

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int ng = min(kTcMaxG, G - r0);  // vectors of this launch
    auto slot_v = [&](int s) { return smem + (size_t)s * kFpSlotBytes; };
    auto slot_a = [&](int s) { return smem + (size_t)s * kFpSlotBytes + kFpVBytes; };
    if (tid == 0) {
        for (int s = 0; s < kFpSlots; ++s) {
            mbar_init(&vfull[s], 1);
            mbar_init(&afull[s], 1);
            mbar_init(&empty[s], 1);
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
            const float xm = __int_as_float(xmax[r0 + tid]);
            if (xm > 0.0f && isfinite(xm)) t = exp2f(floorf(log2f(32768.0f / xm)));
        }
        tsc[tid] = t;
    }
    // A rows that no stage writes (vectors >= ng, the fourth component) stay zero
    for (int s = 0; s < kFpSlots; ++s)
        for (int e = tid; e < kFpABytes / 16; e += kFpThreads)
            reinterpret_cast<uint4*>(slot_a(s))[e] = make_uint4(0u, 0u, 0u, 0u);
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

    if (warp == 0) {
        // ---- producer
        if (lane == 0) {
            int it = 0;
            bool run = true;
            for (int u = blockIdx.x; u < nunits && run; u += gridDim.x) {
                const FwdUnit un = units[u];
                const FwdGroup gp = groups[un.group];
                const TF* Vg = static_cast<const TF*>(ONE ? m0.Vr : meshes[gp.mesh].Vr) + gp.vbase;
                const int n16 = (un.nrows + 15) & ~15, cu = un.ncols, Cs8 = gp.Cs >> 3;
                for (int q = 0; q * kFpRows < n16; ++q, ++it) {
                    const int slot = it % kFpSlots;
                    if (it >= kFpSlots &&
                        !fp_wait(&empty[slot], (uint32_t)((it / kFpSlots) - 1) & 1u, abort_flag, err, 7, it)) {
                        run = false;
                        break;
                    }
                    // one bulk copy per 8-row core row: cu * 16 contiguous bytes of the tiles
                    const int kr0 = (un.j0 >> 3) + q * (kFpRows / 8);
                    const int nkr = min(kFpRows / 8, (n16 >> 3) - q * (kFpRows / 8));
                    mbar_arrive_expect_tx(&vfull[slot], (uint32_t)(nkr * cu * 16));
                    for (int kr = 0; kr < nkr; ++kr)
                        bulk_g2s(slot_v(slot) + (size_t)kr * cu * 16,
                                 Vg + ((size_t)(kr0 + kr) * (size_t)Cs8 + (size_t)(un.c0 >> 3)) * 64,
                                 (uint32_t)(cu * 16), &vfull[slot]);
                    issued = it + 1;
                }
            }
        }
    } else if (warp == 1) {
        // ---- MMA issue
        if (lane == 0) {
            int it = 0, i = 0;
            bool run = true;
            for (int u = blockIdx.x; u < nunits && run; u += gridDim.x, ++i) {
                const FwdUnit un = units[u];
                const int n16 = (un.nrows + 15) & ~15, cu = un.ncols, nN = (cu + 15) & ~15;
                const int ab = i & 1;
                if (i >= 2 && !fp_wait(&acce[ab], (uint32_t)((i >> 1) - 1) & 1u, abort_flag, err, 8, i)) break;
                tc_fence_after();
                const uint32_t d = tmem + (uint32_t)(ab * kFpCols);
                const uint32_t idesc = tc_idesc(nN, kBf16);
                const uint32_t kstride = (uint32_t)cu * 16;  // K-direction core stride of V
                for (int q = 0; q * kFpRows < n16; ++q, ++it) {
                    const int slot = it % kFpSlots;
                    const uint32_t par = (uint32_t)(it / kFpSlots) & 1u;
                    if (!fp_wait(&vfull[slot], par, abort_flag, err, 9, it) ||
                        !fp_wait(&afull[slot], par, abort_flag, err, 10, it)) {
                        run = false;
                        break;
                    }
                    tc_fence_after();
                    const uint32_t a0 = smem_addr(slot_a(slot)), b0 = smem_addr(slot_v(slot));
                    const int steps = min(kFpRows / 16, (n16 >> 4) - q * (kFpRows / 16));
                    for (int ks = 0; ks < steps; ++ks) {
                        const uint64_t ad = tc_desc(a0 + (uint32_t)ks * 256, 128, kFpSbo);
                        const uint64_t bd = tc_desc(b0 + (uint32_t)ks * 2 * kstride, kstride, 128);
                        tc_mma(d, ad, bd, idesc, (q > 0 || ks > 0) ? 1u : 0u);
                    }
                    tc_commit(&empty[slot]);
                }
                if (run) tc_commit(&accf[ab]);
            }
        }
    } else if (warp < 6) {
        // ---- A builders: warp bw builds the stages it with it % 4 == bw; an
        // item is (8-row K block kb, vector r): 8 rows of x_r -> three hi and
        // three lo rows of 8 K values
        const int bw = warp - 2;
        int it = 0;
        bool run = true;
        for (int u = blockIdx.x; u < nunits && run; u += gridDim.x) {
            const FwdUnit un = units[u];
            const int n16 = (un.nrows + 15) & ~15;
            const int nst = (n16 + kFpRows - 1) / kFpRows;
            if (it + ((bw - it) & 3) >= it + nst) {  // no stage of this unit is ours
                it += nst;
                continue;
            }
            const FwdGroup gp = groups[un.group];
            const int64_t xgoff = ONE ? m0.xgoff : meshes[gp.mesh].xgoff;
            const float* x0 = xg + ((size_t)xgoff + gp.s0 + un.j0) * G * 4;
            for (int q = 0; q < nst; ++q, ++it) {
                if ((it & 3) != bw) continue;
                const int slot = it % kFpSlots;
                // the lanes of a warp decide together (they meet at __syncwarp)
                const bool got = it < kFpSlots ||
                                 fp_wait(&empty[slot], (uint32_t)((it / kFpSlots) - 1) & 1u, abort_flag, err, 11, it);
                if (!__all_sync(0xffffffffu, got)) {
                    run = false;
                    break;
                }
                unsigned char* A = slot_a(slot);
                for (int itm = lane; itm < 4 * ng; itm += 32) {
                    const int kb = itm / ng, r = itm - kb * ng;
                    const float t = tsc[r];
                    uint32_t hw[3][4], lw[3][4];
#pragma unroll
                    for (int i = 0; i < 8; i += 2) {
                        float va[2][3];
#pragma unroll
                        for (int e = 0; e < 2; ++e) {
                            const int j = q * kFpRows + kb * 8 + i + e;
                            float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
                            if (j < un.nrows) v = *reinterpret_cast<const float4*>(x0 + ((size_t)j * G + r0 + r) * 4);
                            va[e][0] = v.x * t;
                            va[e][1] = v.y * t;
                            va[e][2] = v.z * t;
                        }
#pragma unroll
                        for (int a = 0; a < 3; ++a) {
                            const uint32_t h0 = tc_bits<TF>(va[0][a]), h1 = tc_bits<TF>(va[1][a]);
                            const uint32_t l0 = tc_bits<TF>(va[0][a] - tc_back<TF>((unsigned short)h0));
                            const uint32_t l1 = tc_bits<TF>(va[1][a] - tc_back<TF>((unsigned short)h1));
                            hw[a][i >> 1] = h0 | (h1 << 16);
                            lw[a][i >> 1] = l0 | (l1 << 16);
                        }
                    }
                    const int qq = r & 3, k = r >> 2;
#pragma unroll
                    for (int a = 0; a < 3; ++a) {
                        const int mh = 32 * qq + 4 * k + a, ml = mh + 16;
                        *reinterpret_cast<uint4*>(A + (size_t)((mh >> 3) * (kFpRows / 8) + kb) * 128 + (mh & 7) * 16) =
                            make_uint4(hw[a][0], hw[a][1], hw[a][2], hw[a][3]);
                        *reinterpret_cast<uint4*>(A + (size_t)((ml >> 3) * (kFpRows / 8) + kb) * 128 + (ml & 7) * 16) =
                            make_uint4(lw[a][0], lw[a][1], lw[a][2], lw[a][3]);
                    }
                }
                asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                __syncwarp();
                if (lane == 0) mbar_arrive(&afull[slot]);
            }
        }
    } else {
        // ---- epilogue: warps 6-9 take the units with an even local index
        // (accumulator 0), warps 10-13 the odd ones (accumulator 1).  Lane l
        // of the warp of quarter q holds row 32 q + l: hi (l < 16) or lo (l >=
        // 16) of component l % 4 of vector q + 4 ((l / 4) % 4).
        const int e = (warp - 6) >> 2, quarter = warp & 3;
        float* B = reinterpret_cast<float*>(smem + (size_t)kFpSlots * kFpSlotBytes + (size_t)(warp - 6) * kFpBBytes);
        const int nk = ng > quarter ? (ng - quarter + 3) >> 2 : 0;  // vectors of this quarter
        int i = e;
        for (int u = blockIdx.x + e * gridDim.x; u < nunits; u += 2 * gridDim.x, i += 2) {
            const FwdUnit un = units[u];
            const FwdGroup gp = groups[un.group];
            const MeshDev& md = ONE ? m0 : meshes[gp.mesh];
            const int cu = un.ncols;
            // the descriptors of this lane's columns, loaded while the MMAs run
            uint2 dsc[kFpCols / 32];
#pragma unroll
            for (int jj = 0; jj < kFpCols / 32; ++jj) {
                dsc[jj] = make_uint2(kFdSkip, 0u);
                if (un.zcol0 < 0 && jj * 32 + lane < cu && nk > 0)
                    dsc[jj] = md.fdesc[(size_t)gp.dbase + un.c0 + jj * 32 + lane];
            }
            const bool got = fp_wait(&accf[e], (uint32_t)(i >> 1) & 1u, abort_flag, err, 12, i);
            if (!__all_sync(0xffffffffu, got)) break;
            tc_fence_after();
            float* wr = w + (size_t)md.woff * G * 4;
            float* zb = un.zcol0 >= 0 ? z + (size_t)(un.zcol0 + (int64_t)un.chunk * gp.Cs + un.c0) * G * 4 : nullptr;
            const uint32_t ta = tmem + ((uint32_t)(32 * quarter) << 16) + (uint32_t)(e * kFpCols);
#pragma unroll
            for (int jj = 0; jj < kFpCols / 32; ++jj) {
                if (jj * 32 >= cu) break;
                float v[32];
                if (nk > 0) fp_ld32(ta + (uint32_t)(jj * 32), v);
                if (jj * 32 + 32 >= cu) {
                    // the last read of the accumulator
                    tc_fence_before();
                    __syncwarp();
                    if (lane == 0) mbar_arrive(&acce[e]);
                }
                if (nk == 0) continue;
#pragma unroll
                for (int c = 0; c < 32; ++c) B[c * kFpBld + lane] = v[c];
                __syncwarp();
                const int c = jj * 32 + lane;  // this lane's column of the unit
                if (c < cu)
                    for (int k = 0; k < nk; ++k) {
                        const int r = quarter + 4 * k;
                        const float inv = 1.0f / tsc[r];
                        const float* bp = B + lane * kFpBld + 4 * k;
                        const float z0 = (bp[0] + bp[16]) * inv, z1 = (bp[1] + bp[17]) * inv,
                                    z2 = (bp[2] + bp[18]) * inv;
                        if (zb) {
                            *reinterpret_cast<float4*>(zb + ((size_t)c * G + r0 + r) * 4) =
                                make_float4(z0, z1, z2, 0.0f);
                        } else if (dsc[jj].x != kFdSkip) {
                            const uint32_t x = dsc[jj].x;
                            const int p = (int)((x >> 28) & 3u), pq = (int)(x >> 30);
                            const float f = __uint_as_float(dsc[jj].y);
                            float o0, o1, o2;
                            if (p == 3) {
                                o0 = f * z0;
                                o1 = f * z1;
                                o2 = f * z2;
                            } else {
                                // V_pq enters y_p with x_q and (p != q) y_q with x_p
                                const float zp = p == 0 ? z0 : (p == 1 ? z1 : z2);
                                const float zq = pq == 0 ? z0 : (pq == 1 ? z1 : z2);
                                o0 = p == 0 ? f * zq : (pq == 0 ? f * zp : 0.0f);
                                o1 = p == 1 ? f * zq : (pq == 1 ? f * zp : 0.0f);
                                o2 = p == 2 ? f * zq : (pq == 2 ? f * zp : 0.0f);
                            }
                            *reinterpret_cast<float4*>(wr + ((size_t)(x & 0x0fffffffu) * G + r0 + r) * 4) =
                                make_float4(o0, o1, o2, 0.0f);
                        }
                    }
                __syncwarp();
            }
        }
    }
    __syncthreads();
    if (*abort_flag) {
        // no copy may still write into shared memory and no MMA may still run
        // when the CTA frees its tensor memory and exits
        if (tid == 0)
            for (int q = max(0, issued - kFpSlots); q < issued; ++q)
                mbar_wait(&vfull[q % kFpSlots], (uint32_t)(q / kFpSlots) & 1u, err, 13, q);
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
