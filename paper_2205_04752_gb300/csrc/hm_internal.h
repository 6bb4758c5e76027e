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

// matvec work item of a leaf: admissible block b, row offset of the leaf in t
struct FarItem {
    int32_t b, off;
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
    std::vector<int64_t> woff_h;          // offsets in the w workspace (nadm*7), 3k each
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
    hm::DevBuf d_uoff, d_voff, d_coff, d_woff;  // int64 nadm*7
    hm::DevBuf d_noff;   // int64 nnear
    hm::DevBuf d_leaf;   // int32 2*nleaves (t0, m)
    hm::DevBuf d_far_ptr, d_far_items;    // CSR per leaf
    hm::DevBuf d_near_ptr, d_near_items;  // CSR per leaf (near block ids)
    hm::DevBuf d_p1_order;                // int32 nadm: phase-1 block order (largest first)

    // FP64 arenas
    hm::DevBuf U64, V64, N64;
    // packed arenas
    hm::DevBuf U32, V32, N32;          // FP32 (N32 also serves BF16/FP16 forms)
    hm::DevBuf U16b, V16b, U16h, V16h;  // BF16 / FP16 factors
    hm::DevBuf SUb, SVb, SUh, SVh;     // per-column scales (float) for BF16 / FP16
    bool packed[4] = {true, false, false, false};

    // workspace
    int32_t max_rhs = 32;
    hm::DevBuf xg;  // max_rhs x 3 x M doubles (gathered x, cluster order)
    hm::DevBuf wb;  // max_rhs x w_total doubles
    hm::DevBuf xh, yh;  // device staging for hm_matvec_host (max_rhs x 3M doubles)

    // measurement hook (hm_profile_enable / hm_profile_read)
    bool prof_on = false;
    mutable std::vector<cudaEvent_t> prof_ev;  // 4 per profiled call
    mutable int64_t prof_calls = 0;
};

namespace hm {
// workspace of one product: gathered x (nrhs x 3 x M) and the far-field w
// vectors (nrhs x w_total), both in the form's accumulation type
struct Scratch {
    void* xg;
    void* w;
    bool profile;  // record the measurement-hook events
};
int matvec_device_scratch(const hm_matrix& H, const double* x, double* y, int32_t nrhs,
                          int64_t ld, int32_t form, cudaStream_t s, const Scratch& scr);
// bytes of Scratch a product of nrhs vectors in `form` needs (xg 256-aligned, then w)
size_t matvec_scratch_bytes(const hm_matrix& H, int32_t nrhs, int32_t form);
// record event `which` (0..3) of the current profiled call, if profiling
void prof_mark(const hm_matrix& H, int which, cudaStream_t s);
// kernels launchers (implemented in the .cu files)
int assemble_device(const hm_tree& tr, hm_matrix& H);
int matvec_device(const hm_matrix& H, const double* x, double* y, int32_t nrhs, int64_t ld,
                  int32_t form, cudaStream_t s);
int pack_device(hm_matrix& H, int32_t form, cudaStream_t s);
}  // namespace hm
