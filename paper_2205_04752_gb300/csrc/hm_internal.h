// hm_internal.h -- internal structures of the H-matrix library (host side).
// Not part of the ABI; shared by the library's own translation units only.
#pragma once

#include <cuda_runtime.h>

#include <array>
#include <cstdint>
#include <string>
#include <vector>

#include "../../include/hmat.h"

namespace hm {

// ---------------------------------------------------------------- errors
void set_error(const char* fmt, ...);
int fail(int code, const char* fmt, ...);
// check a CUDA call; on failure records the error text and returns HM_EDEVICE
int cuda_check(cudaError_t e, const char* what);
#define HM_CUDA(call)                                 \
    do {                                              \
        int hm_rc_ = ::hm::cuda_check((call), #call); \
        if (hm_rc_) return hm_rc_;                    \
    } while (0)

// ---------------------------------------------------------------- tree
struct Node {
    int64_t lo, hi;      // [lo, hi) in cluster order
    int64_t son[2];      // -1 for a leaf
    int32_t level;
    double bmin[3], bmax[3];  // box of all triangle vertices of the cluster
};

}  // namespace hm

struct hm_tree {
    int64_t M = 0, nv = 0;
    int32_t leaf = 0;
    double eta = 0.0;
    int32_t depth = 0;
    std::vector<double> V;        // nv x 3
    std::vector<int32_t> T;       // M x 3
    std::vector<double> coll;     // M x 3, original order (centroids)
    std::vector<int64_t> perm;    // cluster position -> original id
    std::vector<hm::Node> nodes;  // pre-order
    std::vector<std::array<int64_t, 2>> adm, near_blocks;  // (row node, col node)
    std::vector<int64_t> leaves;  // leaf node ids in cluster order
};

namespace hm {

// ---------------------------------------------------------------- device memory
struct Allocator {
    hm_allocator user{};
    bool has_user = false;
    cudaStream_t stream = nullptr;
    void* alloc(size_t bytes);
    void release(void* p, size_t bytes);
};

struct DevBuf {
    void* p = nullptr;
    size_t bytes = 0;
    template <class T>
    T* as() const { return static_cast<T*>(p); }
};

// block descriptor shared with the kernels: rows [t0, t0+m), cols [s0, s0+n)
struct Blk {
    int32_t t0, m, s0, n;
};

// far-field stream of a leaf: item = one (admissible block, kernel) with its
// first segment in the leaf's stream and its first global factor column; each
// leaf's list ends with a sentinel whose seg_start is the segment count
struct LeafFarItem {
    int32_t seg_start, col;
};
// source of a far item in the block-ordered FP64 U arena (used by packing):
// element offset of (first row of the leaf, column 0), leading dimension, rank
struct PackSrc {
    int64_t src;
    int32_t ld, k;
};
// near-field stream of a leaf: item = one near block with its first column in
// the stream and its first column cluster position; sentinel as above
struct LeafNearItem {
    int32_t col_start, s0;
};
struct NearSrc {
    int64_t src;  // element offset of the block in the block-ordered FP64 near arena
    int32_t n, pad;
};
// one admissible block of the far-field forward pass (32 bytes): column
// cluster start and size, first global factor column, total rank, offset of
// its row-major V, and the rank of each of the seven kernels
struct FwdRec {
    int32_t s0, n, col0, C;
    int64_t vbase;
    uint64_t kpack;  // rank of kernel q in bits 8q .. 8q+7
};


}  // namespace hm

struct hm_matrix {
    // geometry / partition
    int64_t M = 0;
    int64_t nadm = 0, nnear = 0, nleaves = 0;
    double E = 1.0, nu = 0.3;
    hm_params prm{};
    hm::Allocator alloc;
    std::vector<hm::Blk> adm_h, near_h;   // cluster-order ranges
    std::vector<int32_t> rank_h;          // nadm * 7
    std::vector<int32_t> flags_h;         // nadm * 7
    std::vector<int64_t> uoff_h, voff_h;  // element offsets in the U / V arenas (nadm*7)
    std::vector<int64_t> coff_h;          // column offsets (per-column scales), nadm*7
    std::vector<int64_t> noff_h;          // element offsets in the near arena (nnear)
    int64_t u_total = 0, v_total = 0, c_total = 0, w_total = 0, n_total = 0;
    int32_t csp = 0;
    int32_t max_leaf = 0;
    double asm_ms[3] = {0, 0, 0};

    // device arrays
    hm::DevBuf d_perm;   // int32 M: cluster position -> original id
    hm::DevBuf d_adm;    // Blk nadm
    hm::DevBuf d_near;   // Blk nnear
    hm::DevBuf d_rank;   // int32 nadm*7
    hm::DevBuf d_uoff, d_voff, d_coff;  // int64 nadm*7
    hm::DevBuf d_noff;   // int64 nnear
    hm::DevBuf d_leaf;   // int32 2*nleaves (t0, m)
    hm::DevBuf d_lf_base, d_lf_ptr, d_lf_items, d_lf_src;  // far stream per leaf
    hm::DevBuf d_ln_base, d_ln_ptr, d_ln_items, d_ln_src;  // near stream per leaf
    hm::DevBuf d_vb_base;                 // int64 nadm+1: row-major V of each block
    hm::DevBuf d_fwd_all;                // FwdRec in stream order: |s| > 128 first, then the rest
    std::vector<hm::FwdRec> fwd_h;       // host copy of d_fwd_all

    hm::DevBuf d_leaf_order;             // int32 nleaves: leaves by decreasing streamed bytes
    hm::DevBuf d_counters;               // int32 max_rhs: work counters of the streamed kernel
    hm::DevBuf d_err;                    // int32: set by a device wait that ran out
    int64_t n_fwd_small = 0, n_fwd_big = 0;
    int64_t ul_total = 0, nl_total = 0, vr_total = 0;
    // the near field runs on a second stream, concurrently with the far field
    cudaStream_t side = nullptr;
    cudaEvent_t ev_fork = nullptr, ev_join = nullptr;

    // FP64 factor and near arenas in block order (ACA output, export)
    hm::DevBuf U64, V64, N64;
    // streaming arenas of each form (index = form): U leaf-major, V row-major
    hm::DevBuf Ul[4], Vr[4];
    hm::DevBuf Nl64, Nl32;  // near field leaf-major: FP64 form / all other forms
    hm::DevBuf SU, SV;      // per-column scales of the 16-bit forms (float, c_total)
    bool packed[4] = {false, false, false, false};

    // workspace
    int32_t max_rhs = 32;
    hm::DevBuf xg;  // max_rhs x M x 4 doubles (gathered x, cluster order, padded 4-vectors)
    hm::DevBuf wb;  // max_rhs x w_total doubles (one 4-vector per factor column)
    hm::DevBuf yn;  // max_rhs x 3 x M doubles (near-field part of y, cluster order)
    hm::DevBuf xh, yh;  // device staging for hm_matvec_host (max_rhs x 3M doubles)

    // measurement hook (hm_profile_enable / hm_profile_read)
    bool prof_on = false;
    mutable std::vector<cudaEvent_t> prof_ev;  // 4 per profiled call
    mutable int64_t prof_calls = 0;
};

namespace hm {
// workspace of one product: gathered x (nrhs x M x 4), the far-field w
// vectors (nrhs x c_total x 4) and the near-field part of y (nrhs x 3 x M),
// all in the form's accumulation type
struct Scratch {
    void* xg;
    void* w;
    void* yn;
    bool profile;  // record the measurement-hook events
};
int matvec_device_scratch(const hm_matrix& H, const double* x, double* y, int32_t nrhs,
                          int64_t ld, int32_t form, cudaStream_t s, const Scratch& scr);
// bytes of Scratch a product of nrhs vectors in `form` needs (xg, yn, w; each
// part 256-byte aligned)
size_t matvec_scratch_bytes(const hm_matrix& H, int32_t nrhs, int32_t form);
// record event `which` (0..3) of the current profiled call, if profiling
void prof_mark(const hm_matrix& H, int which, cudaStream_t s);
// kernels launchers (implemented in the .cu files)
int assemble_device(const hm_tree& tr, hm_matrix& H);
int matvec_device(const hm_matrix& H, const double* x, double* y, int32_t nrhs, int64_t ld,
                  int32_t form, cudaStream_t s);
int pack_device(hm_matrix& H, int32_t form, cudaStream_t s);
}  // namespace hm
