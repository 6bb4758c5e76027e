// hm_stream.cuh -- per-leaf product of the far and near field streamed through
// shared memory with bulk asynchronous copies (cp.async.bulk + mbarrier).
//
// For every leaf row cluster tau the factor segments (columns of U restricted
// to the rows of tau) and the near-field columns are contiguous in memory
// (see hm_matvec.cu).  A persistent CTA takes (mesh, leaf) work items from a
// global counter (largest first, over every mesh of the product).  Warp 0 is
// the producer: for every slot of a ring of shared-memory slots (LeafCfg::kS)
// it copies up to kStage bytes of the current leaf's stream and, next to it,
// the 4-vector each segment needs: w of the segment's factor column (far
// field) or x at the segment's source position (near field).  The far items
// of a leaf are merged into runs of consecutive factor columns (the kernels
// of a block, often consecutive blocks), and one near block's columns are
// consecutive positions, so these are a few contiguous copies per slot, one
// per run and lane.
// Warps 1..7 consume the slots from shared memory only: thread (p, c, h) owns
// Rr rows (16 bytes of U), a chunk of RC right-hand sides and every H-th
// segment of a slot; at the end of a leaf the H partial sums of each row are
// added in a fixed order and y is written in the original dof order.
// Deterministic for a given number G of right-hand sides per launch (H, the
// segment split, depends on G, so the same vector applied in launches of
// different width agrees to the rounding of the accumulation type).
//
// Every mbarrier wait is bounded (kWaitCycles); on expiry the thread records
// an error in *err, the producer drains its own copies in flight (again
// bounded) and the CTA returns.
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include <climits>
#include <cstdint>

namespace hm {
namespace stream {

constexpr int kThreads = 256;             // warp 0 producer + 7 consumer warps
constexpr int kConsumers = kThreads - 32;
constexpr int kStages = 5;
constexpr int kStageBytes = 16384;        // stream bytes of a slot at least (LeafCfg::kStage)
constexpr int kMaxSeg = 256;              // segments / columns per stage at most
constexpr long long kWaitCycles = 4000000000LL;  // ~2 s at 2 GHz

struct StageMeta {
    int32_t leaf;   // leaf index (into its mesh's leaf table)
    int32_t kind;   // 0 far segments, 1 near columns, 2 no more work, 3 INT16 near columns
    int32_t first;  // first segment / column of the stage within the leaf's stream
    int32_t count;  // segments / columns in the stage
    int32_t last;   // 1 if this is the last stage of the leaf
    int32_t pad[3]; // pad[0]: mesh of the leaf
};

__device__ __forceinline__ uint32_t smem_addr(const void* p)
{
    return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_fence_init()
{
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)),
                 "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ void mbar_arrive(uint64_t* bar)
{
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_addr(bar)) : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity)
{
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_addr(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

// bounded wait for the phase with the given parity; false on expiry, with
// err[0] = 1 and the first expiry's site, stage and CTA in err[1..3]
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity, int* err, int site = 0, int stage = 0)
{
    if (mbar_try_wait(bar, parity)) return true;
    const long long t0 = clock64();
    for (;;) {
        if (mbar_try_wait(bar, parity)) return true;
        if (clock64() - t0 > kWaitCycles) {
            if (atomicCAS(err + 1, 0, site) == 0) {
                err[2] = stage;
                err[3] = (int)blockIdx.x;
            }
            atomicExch(err, 1);
            return false;
        }
    }
}

// bulk copy global -> shared (16-byte aligned, size a multiple of 16), with
// completion counted on the mbarrier
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* bar)
{
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            smem_addr(dst)),
        "l"(src), "r"(bytes), "r"(smem_addr(bar))
        : "memory");
}

// the same with an L2 cache policy (the streamed factors and near field are
// read once per product: evict them first, so that the vectors and tables the
// kernels read repeatedly stay in L2)
__device__ __forceinline__ void bulk_g2s_hint(void* dst, const void* src, uint32_t bytes, uint64_t* bar,
                                              uint64_t policy)
{
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes.L2::cache_hint [%0], [%1], %2, [%3], %4;" ::"r"(
            smem_addr(dst)),
        "l"(src), "r"(bytes), "r"(smem_addr(bar)), "l"(policy)
        : "memory");
}

__device__ __forceinline__ uint64_t l2_evict_first_policy()
{
    uint64_t pol;
    asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(pol));
    return pol;
}

// prefetch [p, p + bytes) into L2: only the 16-byte-aligned interior, so that
// nothing outside the range is touched
__device__ __forceinline__ void prefetch_l2(const void* p, size_t bytes)
{
    const uintptr_t a = (uintptr_t)p, b = a + bytes;
    const uintptr_t a16 = (a + 15) & ~(uintptr_t)15, b16 = b & ~(uintptr_t)15;
    for (uintptr_t q = a16; q < b16; q += 65536) {
        const uint32_t n = (uint32_t)min((uintptr_t)65536, b16 - q);
        asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(q), "r"(n) : "memory");
    }
}

// 16-byte asynchronous copy global -> shared through the load/store path
__device__ __forceinline__ void cp_async16(void* dst, const void* src)
{
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(smem_addr(dst)), "l"(src) : "memory");
}

// the mbarrier's current phase also waits for this thread's cp.async copies
// (its pending count is raised now and lowered when they have landed)
__device__ __forceinline__ void cp_async_arrive(uint64_t* bar)
{
    asm volatile("cp.async.mbarrier.arrive.shared::cta.b64 [%0];" ::"r"(smem_addr(bar)) : "memory");
}

// aux ranges up to this many bytes go through cp.async, larger ones through
// the bulk copy engine
constexpr int kSmallCopy = 256;

// 16 KB of zeros: the staged w of the padding segments of a 16-bit U stream
__device__ __align__(128) unsigned char g_zeros[16384] = {};

// element offset of rows [Rr p, Rr p + Rr) of segment s in a stage whose
// first segment is a multiple of 8 (tiled 16-bit streams) or any segment
template <class TF>
__device__ __forceinline__ size_t useg(int s, int p, int mp)
{
    if (sizeof(TF) == 2) return ((size_t)(s >> 3) * (size_t)(mp >> 3) + (size_t)p) * 64 + (size_t)(s & 7) * 8;
    return (size_t)s * mp + (size_t)p * (16 / sizeof(TF));
}

__device__ __forceinline__ void named_barrier_consumers()
{
    asm volatile("bar.sync 1, %0;" ::"n"(kConsumers) : "memory");
}

// 16 bytes from shared memory as N values
template <class T, class TA>
struct Smem16;
template <class TA>
struct Smem16<double, TA> {
    static constexpr int N = 2;
    __device__ __forceinline__ static void load(const double* p, TA* o)
    {
        double2 v = *reinterpret_cast<const double2*>(p);
        o[0] = (TA)v.x;
        o[1] = (TA)v.y;
    }
};
template <class TA>
struct Smem16<float, TA> {
    static constexpr int N = 4;
    __device__ __forceinline__ static void load(const float* p, TA* o)
    {
        float4 v = *reinterpret_cast<const float4*>(p);
        o[0] = (TA)v.x;
        o[1] = (TA)v.y;
        o[2] = (TA)v.z;
        o[3] = (TA)v.w;
    }
};
template <class TA>
struct Smem16<__half, TA> {
    static constexpr int N = 8;
    __device__ __forceinline__ static void load(const __half* p, TA* o)
    {
        uint4 v = *reinterpret_cast<const uint4*>(p);
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
struct Smem16<__nv_bfloat16, TA> {
    static constexpr int N = 8;
    __device__ __forceinline__ static void load(const __nv_bfloat16* p, TA* o)
    {
        uint4 v = *reinterpret_cast<const uint4*>(p);
        const __nv_bfloat162* h = reinterpret_cast<const __nv_bfloat162*>(&v);
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            float2 f = __bfloat1622float2(h[q]);
            o[2 * q] = (TA)f.x;
            o[2 * q + 1] = (TA)f.y;
        }
    }
};

// Two values of the INT16 form from a 32-bit word (low half first) as exact
// FP32 values.  The form stores q in [-32767, 32767] in offset binary,
// u = q + 32768 as an unsigned 16-bit integer; placed under the exponent of
// 2^23 (bytes u_lo, u_hi, 0x00, 0x4B) it is the float 2^23 + u, and
// subtracting 2^23 + 2^15 leaves q exactly.  One byte permute and one FP32
// add per value, no int-to-float conversion instruction.
__device__ __forceinline__ float2 i16x2_to_float2(uint32_t word)
{
    const float lo = __uint_as_float(__byte_perm(word, 0x4B000000u, 0x7410)) - 8421376.0f;
    const float hi = __uint_as_float(__byte_perm(word, 0x4B000000u, 0x7432)) - 8421376.0f;
    return make_float2(lo, hi);
}

template <class TA>
struct Smem16<int16_t, TA> {
    static constexpr int N = 8;
    __device__ __forceinline__ static void load(const int16_t* p, TA* o)
    {
        uint4 v = *reinterpret_cast<const uint4*>(p);
        const uint32_t wv[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            float2 f = i16x2_to_float2(wv[q]);
            o[2 * q] = (TA)f.x;
            o[2 * q + 1] = (TA)f.y;
        }
    }
};

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

// R consecutive values (R * sizeof(T) a multiple of 16) from shared memory
template <class T, class TA, int R>
__device__ __forceinline__ void smem_rows(const T* p, TA* o)
{
    constexpr int N = Smem16<T, TA>::N;
#pragma unroll
    for (int q = 0; q < R / N; ++q) Smem16<T, TA>::load(p + q * N, o + q * N);
}

// Right-hand sides: a launch serves G of them at once (the vectors are
// interleaved, 4-vector (position or column, r) at index pos * G + r).  A
// consumer thread holds Rr rows (16 bytes of U) for RC right-hand sides.
// RC = 1 is the single-vector kernel; RC * Rr = 16 otherwise.
// A slot is kStage bytes of stream data followed by kAuxBytes of staged 4-vectors.
// A finished leaf is reduced inside the slot of its last stage (released
// afterwards): the single-vector kernel one output component at a time, the
// multi-vector kernel one RHS-chunk position at a time.  The single-vector
// kernel keeps 3 slots of 20 KB stages (16 KB in FP64, whose 4-vectors take
// twice the room) at three CTAs per SM (at most 85 registers a thread): nine
// stages in flight per SM and 21 consumer warps.  Measured at level 6
// (INT16): 5 slots of 16 KB at two CTAs per SM 0.887 ms, 3 of 16 KB at three
// CTAs 0.793 ms, 3 of 20 KB 0.708 ms -- the kernel issues about half of the
// SM's instruction slots, and the extra warps and longer stages hide latency
// (four CTAs of 2 slots, at 64 registers, were no faster; 6 slots of 12 KB
// at two CTAs took 1.15 ms).  The multi-vector kernels keep 3 slots of 20 KB
// stages and 16 KB of 4-vectors at two CTAs per SM (at most 128 registers;
// at one CTA per SM the 4-vector leaf product took 2.52 ms at level 6
// against 1.85 ms).
template <class TF, class TA, int RC>
struct LeafCfg {
    static constexpr int Rr = Smem16<TF, TA>::N;
    static constexpr int kMinCtas = RC == 1 ? 3 : 2;  // CTAs per SM the registers must allow
    static constexpr int kS = 3;
    static constexpr int kStage = (RC == 1 && sizeof(TA) == 8) ? kStageBytes : 20480;
    static_assert(kStage >= kStageBytes, "the host admits leaves by the smallest stage");
    static constexpr int kAuxBytes = RC == 1 ? kMaxSeg * 4 * (int)sizeof(TA) : 16384;
    static constexpr int kSlotBytes = kStage + kAuxBytes;
    static_assert(kS <= kStages, "the barrier arrays hold kStages slots");
    static_assert(kConsumers * Rr * (RC == 1 ? 1 : 3) * (int)sizeof(TA) <= kSlotBytes,
                  "one pass of the leaf reduction must fit a slot");
    static constexpr size_t smem() { return (size_t)kS * kSlotBytes; }
};

// ---------------------------------------------------------------- producer
// Warp 0 of a leaf kernel: takes (mesh, leaf) items from the counter and
// fills the NS slots (stream data + staged 4-vectors) with bulk copies; each
// slot is handed over through full[slot] and taken back through empty[slot]
// (whatever count that barrier was initialised with).  kGran: stage
// granularity of a tiled 16-bit U stream (8 for the single-vector kernel,
// 16, the tensor-core K step, otherwise).
// empty_far (optional): a far stage is taken back once its barrier in this
// second set completes too (the tensor-core kernel's MMA commit); every stage
// is taken back through empty[slot] as well, once every consumer warp has
// passed it, so that no warp can find a full barrier two phases on.
template <class TF, class TN, class TA, int NS, int kStage, int kAuxBytes, int kGran, int kFarCap = 1 << 20,
          bool kTwoRelease = false>
__device__ __forceinline__ void leaf_producer(const int2* __restrict__ work, int nwork,
                                              const MeshDev* __restrict__ meshes, int* __restrict__ counter,
                                              int* __restrict__ err, const TA* __restrict__ xg_base,
                                              const TA* __restrict__ w_base, int G, unsigned char* smem,
                                              uint64_t* full, uint64_t* empty, StageMeta* meta,
                                              uint64_t* empty_far = nullptr)
{
    // per slot (two release barriers only): kind of its last stage and the
    // uses of each release barrier, as bit fields of registers
    uint32_t far_mask = 0u;      // bit q: slot q last held a far stage
    uint32_t far_parity = 0u;    // bit q: parity of the next far release of slot q
    constexpr int kSlotBytes = kStage + kAuxBytes;
    const int lane = threadIdx.x & 31;
    const uint64_t stream_policy = l2_evict_first_policy();
    const int vecG = 4 * G;
    auto sdata = [&](int q) { return smem + (size_t)q * kSlotBytes; };
    auto saux = [&](int q) { return smem + (size_t)q * kSlotBytes + kStage; };
        // ------------------------------------------------------------ producer
        int it = 0;
        bool ok = true;
        // One stage: [first, first + count) of the current stream.  `items`
        // are the stream's (start, vector index) records (sentinel last, ni
        // records); *cur is the item containing `first` and is advanced to
        // the item containing first + count.  vec: the 4-vectors the stream
        // reads (w for the far field, x for the near field), G per index.
        int sreal = 0;  // real segments of the current leaf's U stream
        // the items of the next stage's scan, loaded at the end of the previous
        // one so that their latency overlaps the wait for a free slot
        const int2* pre_items = nullptr;
        int pre_q0 = -1, pre_b31 = INT_MAX;
        int2 pre_a = make_int2(INT_MAX, 0);
        // lastfar: the stage ends the leaf's far stream (meta pad[1])
        auto emit = [&](int mesh, int lf, int kind, int first, int count, int last, const void* src,
                        uint32_t bytes, const int2* items, int ni, int* cur, const TA* vec, int lastfar) -> bool {
            const int slot = it % NS;
            if (it >= NS) {
                bool got;
                // every consumer warp has taken the slot's previous stage (so that
                // none can miss a phase of its full barrier)...
                got = mbar_wait(&empty[slot], (uint32_t)((it / NS) - 1) & 1u, err, 1, it);
                if (got && kTwoRelease) {
                    // ...and, for a far stage, its MMAs are done; then flip that
                    // barrier's expected parity
                    const uint32_t bit = 1u << slot;
                    if (far_mask & bit) {
                        got = mbar_wait(&empty_far[slot], (far_parity & bit) ? 1u : 0u, err, 1, it);
                        far_parity ^= bit;
                    }
                }
                if (!got) return false;
            }
            if (kTwoRelease) {
                const uint32_t bit = 1u << slot;
                far_mask = kind == 0 ? (far_mask | bit) : (far_mask & ~bit);
            }
            if (lane == 0) {
                StageMeta m;
                m.leaf = lf;
                m.kind = kind;
                m.first = first;
                m.count = count;
                m.last = last;
                m.pad[0] = mesh;
                m.pad[1] = lastfar;
                meta[slot] = m;
            }
            __syncwarp();
            if (kind != 2) {
                // bytes of this lane's copies that go through the bulk engine
                uint32_t bulk = 0;
                auto copy = [&](TA* dst, const TA* srcp, uint32_t nb) {
                    if (nb <= (uint32_t)kSmallCopy) {
                        for (uint32_t o = 0; o < nb; o += 16)
                            cp_async16(reinterpret_cast<unsigned char*>(dst) + o,
                                       reinterpret_cast<const unsigned char*>(srcp) + o);
                    } else {
                        bulk_g2s(dst, srcp, nb, &full[slot]);
                        bulk += nb;
                    }
                };
                TA* av = reinterpret_cast<TA*>(saux(slot));
                const int end = first + count;
                int q0 = *cur;
                for (;;) {
                    // lane l looks at item q0 + l; its end is the next item's start
                    // (the sentinel's start for the last real item)
                    const int q = q0 + lane;
                    int2 a = make_int2(INT_MAX, 0);
                    int b31 = INT_MAX;
                    if (pre_items == items && pre_q0 == q0) {
                        a = pre_a;
                        b31 = pre_b31;
                    } else {
                        if (q < ni) a = items[q];
                        if (lane == 31 && q + 1 < ni) b31 = items[q + 1].x;
                    }
                    int b = __shfl_down_sync(0xffffffffu, a.x, 1);
                    if (lane == 31) b = b31;
                    const bool overlap = q < ni - 1 && a.x < end;  // items are sorted by start
                    if (overlap) {
                        const int g0 = max(a.x, first), g1 = min(b, end);
                        if (g0 < g1)
                            copy(av + (size_t)(g0 - first) * vecG, vec + (size_t)(a.y + (g0 - a.x)) * vecG,
                                 (uint32_t)((g1 - g0) * vecG * sizeof(TA)));
                    }
                    const unsigned ov = __ballot_sync(0xffffffffu, overlap);
                    const int nov = __popc(ov);  // overlapping items are a prefix of the lanes
                    const int lastq = q0 + nov - 1;
                    const int lastb = __shfl_sync(0xffffffffu, b, (nov - 1) & 31);
                    if (nov < 32 || lastb >= end) {
                        *cur = lastb > end ? lastq : lastq + 1;
                        break;
                    }
                    q0 += 32;
                }
                {
                    // issue the next scan's loads now
                    const int qn = *cur + lane;
                    pre_items = items;
                    pre_q0 = *cur;
                    pre_a = qn < ni ? items[qn] : make_int2(INT_MAX, 0);
                    pre_b31 = (lane == 31 && qn + 1 < ni) ? items[qn + 1].x : INT_MAX;
                }
                // padding segments of a 16-bit U stream: zero w
                if (lane == 0 && kind == 0 && end > sreal) {
                    const int z0 = max(first, sreal);
                    copy(av + (size_t)(z0 - first) * vecG, reinterpret_cast<const TA*>(g_zeros),
                         (uint32_t)((end - z0) * vecG * sizeof(TA)));
                }
                // the phase waits for every lane's cp.async copies, then for the
                // bulk bytes that lane 0 announces with its arrival
                cp_async_arrive(&full[slot]);
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) bulk += __shfl_xor_sync(0xffffffffu, bulk, o);
                __syncwarp();
                if (lane == 0) {
                    mbar_arrive_expect_tx(&full[slot], bytes + bulk);
                    bulk_g2s_hint(sdata(slot), src, bytes, &full[slot], stream_policy);
                }
            } else if (lane == 0) {
                mbar_arrive(&full[slot]);
            }
            ++it;
            return true;
        };
        const int perV = min(kMaxSeg, kAuxBytes / (vecG * (int)sizeof(TA)));
        for (;;) {
            int idx = 0;
            if (lane == 0) idx = atomicAdd(counter, 1);
            idx = __shfl_sync(0xffffffffu, idx, 0);
            if (idx >= nwork || !ok) break;
            const int2 wk = work[idx];
            const MeshDev& md = meshes[wk.x];
            const int lf = wk.y;
            const int mt = md.leaf[2 * lf + 1];
            const int mp = (mt + 7) & ~7;
            const int fi0 = md.lr_ptr[lf], fi1 = md.lr_ptr[lf + 1];
            const int ni0 = md.ln_ptr[lf], ni1 = md.ln_ptr[lf + 1];
            sreal = md.lr_items[fi1 - 1].seg_start;
            // 16-bit streams are tiled in groups of 8 segments (and stored padded
            // to 16, the tensor-core K step); the single-vector kernel takes
            // stages in whole tiles, the multi-vector one in K steps
            constexpr bool kTiled = sizeof(TF) == 2;
            const int S = kTiled ? (sreal + kGran - 1) & ~(kGran - 1) : sreal;
            const int Sn = md.ln_items[ni1 - 1].col_start;
            const TF* Ul = static_cast<const TF*>(md.Ul);
            const TN* Nl = static_cast<const TN*>(md.Nl);
            const TA* wvec = w_base + (size_t)md.woff * vecG;
            const TA* xvec = xg_base + (size_t)md.xgoff * vecG;
            const int segB = mp * (int)sizeof(TF);
            const int perF = kTiled ? min(min(kStage / segB, perV), kFarCap) & ~(kGran - 1) : min(kStage / segB, perV);
            const int colB = 6 * mp * (int)sizeof(TN);
            const int perN = min(kStage / colB, perV);
            if (perF < 1 || perN < 1) {
                // a segment or a near column larger than a stage (the host
                // rejects such leaves before the launch): stop producing
                if (lane == 0) atomicExch(err, 2);
                break;
            }
            const int2* fitems = reinterpret_cast<const int2*>(md.lr_items + fi0);
            const int2* nitems = reinterpret_cast<const int2*>(md.ln_items + ni0);
            // the leaf's item tables, read by every stage's scan, into L2 now
            if (lane == 0) {
                prefetch_l2(fitems, (size_t)(fi1 - fi0) * sizeof(int2));
                prefetch_l2(nitems, (size_t)(ni1 - ni0) * sizeof(int2));
            }
            int cur = 0;
            for (int g = 0; g < S && ok; g += perF) {
                const int cnt = min(perF, S - g);
                const TF* src = Ul + md.lf_base[lf] + (size_t)g * mp;
                ok = emit(wk.x, lf, 0, g, cnt, (g + cnt == S && Sn == 0) ? 1 : 0, src, (uint32_t)(cnt * segB),
                          fitems, fi1 - fi0, &cur, wvec, g + cnt == S ? 1 : 0);
            }
            cur = 0;
            // the INT16 form streams the leaf's diagonal block from the FP32
            // near stream and its other columns from the INT16 one (kind 3)
            const int nd = md.Nl16 ? min(md.ln16_diag[lf], Sn) : Sn;
            for (int g = 0; g < nd && ok; g += perN) {
                const int cnt = min(perN, nd - g);
                const TN* src = Nl + md.ln_base[lf] + (size_t)g * 6 * mp;
                ok = emit(wk.x, lf, 1, g, cnt, (g + cnt == Sn) ? 1 : 0, src, (uint32_t)(cnt * colB), nitems,
                          ni1 - ni0, &cur, xvec, 0);
            }
            if (md.Nl16 && nd < Sn && ok) {
                const int colB16 = kNear16Head + 12 * mp;
                const int perN16 = min(kStage / colB16, perV);
                const unsigned char* n16 = md.Nl16 + md.ln16_base[lf];
                for (int g = nd; g < Sn && ok; g += perN16) {
                    const int cnt = min(perN16, Sn - g);
                    ok = emit(wk.x, lf, 3, g, cnt, (g + cnt == Sn) ? 1 : 0, n16 + (size_t)(g - nd) * colB16,
                              (uint32_t)(cnt * colB16), nitems, ni1 - ni0, &cur, xvec, 0);
                }
            }
        }
        if (ok) ok = emit(0, -1, 2, 0, 0, 0, nullptr, 0, nullptr, 0, nullptr, nullptr, 0);
        if (!ok) {
            // drain this CTA's own copies in flight before returning (bounded)
            for (int k = 1; k <= NS && k <= it; ++k) {
                const int j = it - k;
                mbar_wait(&full[j % NS], (uint32_t)(j / NS) & 1u, err, 2, j);
            }
        }
}

template <class TF, class TN, class TA, int RC>
__global__ void __launch_bounds__(kThreads, LeafCfg<TF, TA, RC>::kMinCtas) leaf_stream_kernel(
    const int2* __restrict__ work, int nwork, const MeshDev* __restrict__ meshes, int* __restrict__ counter,
    int* __restrict__ err, const TA* __restrict__ xg_base, const TA* __restrict__ w_base, int G,
    double* __restrict__ y, int64_t ld)
{
    using Cfg = LeafCfg<TF, TA, RC>;
    constexpr int Rr = Cfg::Rr;
    constexpr int NS = Cfg::kS;
    extern __shared__ __align__(128) unsigned char smem[];
    // slot q: stream data at smem + q * kSlotBytes, its 4-vectors kStage bytes later
    auto sdata = [&](int q) { return smem + (size_t)q * Cfg::kSlotBytes; };
    auto saux = [&](int q) { return smem + (size_t)q * Cfg::kSlotBytes + Cfg::kStage; };
    __shared__ __align__(8) uint64_t full[kStages];
    __shared__ __align__(8) uint64_t empty[kStages];
    __shared__ StageMeta meta[kStages];

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (threadIdx.x == 0) {
        for (int s = 0; s < NS; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], kConsumers / 32);
        }
        mbar_fence_init();
    }
    __syncthreads();

    if (warp == 0) {
        leaf_producer<TF, TN, TA, NS, Cfg::kStage, Cfg::kAuxBytes, RC == 1 ? 8 : 16>(
            work, nwork, meshes, counter, err, xg_base, w_base, G, smem, full, empty, meta);
        return;
    }

    // ---------------------------------------------------------------- consumers
    // thread (p, c, h): row block p (Rr rows), RHS chunk c (RC vectors),
    // segment group h (every H-th segment / column of each slot)
    const int ctid = threadIdx.x - 32;
    const int NRC = (G + RC - 1) / RC;
    int cur = -1, cur_mesh = -1, P = 1, H = 0, p = 0, c = 0, h = 0, t0 = 0, mt = 0, mp = 8;
    const int32_t* perm = nullptr;
    int64_t xoff = 0;
    TA c1 = (TA)0, c2 = (TA)0;
    TA acc[Rr][RC][3];
    for (int it = 0;; ++it) {
        const int slot = it % NS;
        if (!mbar_wait(&full[slot], (uint32_t)(it / NS) & 1u, err, 3, it)) break;
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
            mp = (mt + 7) & ~7;
            P = mp / Rr;
            H = kConsumers / (P * NRC);
            if (std::is_same<TF, int16_t>::value && RC == 1) {
                // INT16 form, one vector: segments fastest, so that the eight
                // threads of a shared-memory phase read eight consecutive
                // segments (columns) of one row block -- distinct 16-byte
                // positions of a tile, or columns an odd number of 16-byte
                // chunks apart -- and no two of them share a bank
                h = ctid % H;
                p = ctid / H;
                c = 0;
                if (p >= P) h = H;  // idle
            } else {
                p = ctid % P;
                c = (ctid / P) % NRC;
                h = ctid / (P * NRC);
            }
#pragma unroll
            for (int e = 0; e < Rr; ++e)
#pragma unroll
                for (int q = 0; q < RC; ++q) acc[e][q][0] = acc[e][q][1] = acc[e][q][2] = (TA)0;
        }
        const TA* av = reinterpret_cast<const TA*>(saux(slot)) + (size_t)c * RC * 4;
        if (h < H) {
            if (m.kind == 0) {
                const TF* sb = reinterpret_cast<const TF*>(sdata(slot));
                if (RC == 1 && G == 1) {
                    // single vector: two segments per iteration
                    int s = h;
                    for (; s + H < m.count; s += 2 * H) {
                        TA wa0, wa1, wa2, wb0, wb1, wb2;
                        load3(av + (size_t)s * 4, wa0, wa1, wa2);
                        load3(av + (size_t)(s + H) * 4, wb0, wb1, wb2);
                        TA ua[Rr], ub[Rr];
                        smem_rows<TF, TA, Rr>(sb + useg<TF>(s, p, mp), ua);
                        smem_rows<TF, TA, Rr>(sb + useg<TF>(s + H, p, mp), ub);
#pragma unroll
                        for (int e = 0; e < Rr; ++e) {
                            acc[e][0][0] += ua[e] * wa0 + ub[e] * wb0;
                            acc[e][0][1] += ua[e] * wa1 + ub[e] * wb1;
                            acc[e][0][2] += ua[e] * wa2 + ub[e] * wb2;
                        }
                    }
                    if (s < m.count) {
                        TA wa0, wa1, wa2;
                        load3(av + (size_t)s * 4, wa0, wa1, wa2);
                        TA ua[Rr];
                        smem_rows<TF, TA, Rr>(sb + useg<TF>(s, p, mp), ua);
#pragma unroll
                        for (int e = 0; e < Rr; ++e) {
                            acc[e][0][0] += ua[e] * wa0;
                            acc[e][0][1] += ua[e] * wa1;
                            acc[e][0][2] += ua[e] * wa2;
                        }
                    }
                } else {
                    for (int s = h; s < m.count; s += H) {
                        TA ua[Rr];
                        smem_rows<TF, TA, Rr>(sb + useg<TF>(s, p, mp), ua);
#pragma unroll
                        for (int q = 0; q < RC; ++q) {
                            if (RC > 1 && c * RC + q >= G) break;
                            TA w0, w1, w2;
                            load3(av + ((size_t)s * G + q) * 4, w0, w1, w2);
#pragma unroll
                            for (int e = 0; e < Rr; ++e) {
                                acc[e][q][0] += ua[e] * w0;
                                acc[e][q][1] += ua[e] * w1;
                                acc[e][q][2] += ua[e] * w2;
                            }
                        }
                    }
                }
            } else if (m.kind == 3) {
                // INT16 near columns: header of six scales, then six segments
                // of int16; the scales are folded into the coefficients of x,
                // so that each row costs the 15 FMAs of the FP32 columns:
                // V_aa enters y_a with (c1 + c2) x_a and the other two
                // components with c1 x_b; V_ab (a != b) enters y_a with c2 x_b
                // and y_b with c2 x_a
                const unsigned char* sb3 = sdata(slot);
                const int colB16 = kNear16Head + 12 * mp;
                const TA c12 = c1 + c2;
                for (int s = h; s < m.count; s += H) {
                    const unsigned char* col = sb3 + (size_t)s * colB16;
                    const float4 sa = *reinterpret_cast<const float4*>(col);        // s11 s12 s13 s22
                    const float2 sz = *reinterpret_cast<const float2*>(col + 16);   // s23 s33
                    const TA sc[6] = {(TA)sa.x, (TA)sa.y, (TA)sa.z, (TA)sa.w, (TA)sz.x, (TA)sz.y};
                    const int16_t* e0 = reinterpret_cast<const int16_t*>(col + kNear16Head) + p * Rr;
#pragma unroll
                    for (int q = 0; q < RC; ++q) {
                        if (RC > 1 && c * RC + q >= G) break;
                        TA x0, x1, x2;
                        load3(av + ((size_t)s * G + q) * 4, x0, x1, x2);
                        const TA xs3[3] = {x0, x1, x2};
#pragma unroll
                        for (int v = 0; v < 6; ++v) {
                            // (a, b) of value v: 11, 12, 13, 22, 23, 33
                            const int va = v < 3 ? 0 : (v < 5 ? 1 : 2);
                            const int vb = v < 3 ? v : (v < 5 ? v - 2 : 2);
                            TA val[Rr];
                            smem_rows<int16_t, TA, Rr>(e0 + v * mp, val);
                            if (va == vb) {
                                const TA f0 = (va == 0 ? c12 : c1) * sc[v] * xs3[0];
                                const TA f1 = (va == 1 ? c12 : c1) * sc[v] * xs3[1];
                                const TA f2 = (va == 2 ? c12 : c1) * sc[v] * xs3[2];
#pragma unroll
                                for (int e = 0; e < Rr; ++e) {
                                    acc[e][q][0] += f0 * val[e];
                                    acc[e][q][1] += f1 * val[e];
                                    acc[e][q][2] += f2 * val[e];
                                }
                            } else {
                                const TA fa = c2 * sc[v] * xs3[vb], fb = c2 * sc[v] * xs3[va];
#pragma unroll
                                for (int e = 0; e < Rr; ++e) {
                                    acc[e][q][va] += fa * val[e];
                                    acc[e][q][vb] += fb * val[e];
                                }
                            }
                        }
                    }
                }
            } else if (RC == 1) {
                const TN* sb = reinterpret_cast<const TN*>(sdata(slot)) + p * Rr;
                for (int s = h; s < m.count; s += H) {
                    const TN* e0 = sb + (size_t)s * 6 * mp;
                    TA v11[Rr], v12[Rr], v13[Rr], v22[Rr], v23[Rr], v33[Rr];
                    smem_rows<TN, TA, Rr>(e0, v11);
                    smem_rows<TN, TA, Rr>(e0 + mp, v12);
                    smem_rows<TN, TA, Rr>(e0 + 2 * mp, v13);
                    smem_rows<TN, TA, Rr>(e0 + 3 * mp, v22);
                    smem_rows<TN, TA, Rr>(e0 + 4 * mp, v23);
                    smem_rows<TN, TA, Rr>(e0 + 5 * mp, v33);
                    TA x0, x1, x2;
                    load3(av + (size_t)s * G * 4, x0, x1, x2);
#pragma unroll
                    for (int e = 0; e < Rr; ++e) {
                        const TA vd = c1 * (v11[e] + v22[e] + v33[e]);
                        acc[e][0][0] += vd * x0 + c2 * (v11[e] * x0 + v12[e] * x1 + v13[e] * x2);
                        acc[e][0][1] += vd * x1 + c2 * (v12[e] * x0 + v22[e] * x1 + v23[e] * x2);
                        acc[e][0][2] += vd * x2 + c2 * (v13[e] * x0 + v23[e] * x1 + v33[e] * x2);
                    }
                }
            } else {
                // several vectors: the six values of a column one at a time
                // (few live registers); per vector the products c x_b that
                // multiply each value: V_aa enters y_a with (c1 + c2) x_a and the
                // other two components with c1 x_b; V_ab (a != b) enters y_a with
                // c2 x_b and y_b with c2 x_a
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
                        // (a, b) of value v: 11, 12, 13, 22, 23, 33
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
        }
        if (!m.last) {
            // the slot may be refilled once every consumer warp is done with it
            __syncwarp();
            if (lane == 0) mbar_arrive(&empty[slot]);
        } else {
            // the H partial sums of every (row, vector, component), added in a
            // fixed order inside the slot of this last stage (released
            // afterwards): one output component at a time for one vector,
            // red[(h * P + p) * Rr + e]; one position q of the RHS chunk at a
            // time for several, red[((h * P + p) * NRC + c)][e][a]
            TA* red = reinterpret_cast<TA*>(sdata(slot));
            named_barrier_consumers();  // everyone is done reading the slot
            if (RC == 1) {
#pragma unroll
                for (int a = 0; a < 3; ++a) {
                    if (h < H) {
                        TA* rp = red + (size_t)(h * P + p) * Rr;
#pragma unroll
                        for (int e = 0; e < Rr; ++e) rp[e] = acc[e][0][a];
                    }
                    named_barrier_consumers();
                    for (int i = ctid; i < mt; i += kConsumers) {
                        const int pp = i / Rr, e = i - pp * Rr;
                        TA sum = (TA)0;
                        for (int g = 0; g < H; ++g) sum += red[(size_t)(g * P + pp) * Rr + e];
                        y[xoff + 3 * (size_t)perm[t0 + i] + a] = (double)sum;
                    }
                    named_barrier_consumers();
                }
            } else {
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
                    const int nvec = (G - q + RC - 1) / RC;  // vectors r = cc * RC + q < G
                    const int per_row = 3 * nvec;
                    for (int idx = ctid; idx < mt * per_row; idx += kConsumers) {
                        const int i = idx / per_row, rem = idx - i * per_row;
                        const int cc = rem / 3, a = rem - 3 * cc;
                        const int pp = i / Rr, e = i - pp * Rr;
                        TA sum = (TA)0;
                        for (int g = 0; g < H; ++g) sum += red[(size_t)((g * P + pp) * NRC + cc) * kPer + e * 3 + a];
                        const int r = cc * RC + q;
                        y[(size_t)r * ld + xoff + 3 * (size_t)perm[t0 + i] + a] = (double)sum;
                    }
                    named_barrier_consumers();
                }
            }
            __syncwarp();
            if (lane == 0) mbar_arrive(&empty[slot]);
        }
    }
}

}  // namespace stream
}  // namespace hm
