// hm_internal.h -- internal structures of the H-matrix library (host side).
// Not part of the ABI; shared by the library's own translation units only.
#pragma once

#include <cuda_runtime.h>

#include <array>
#include <cstdint>
#include <memory>
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
    double bmin[3], bmax[3];  // box of all triangle vertices of the cluster (of the points in a point tree)
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
    // kind 0: a triangle tree (rows and columns the triangles);
    // kind 1, a tree of points (hm_build_point_tree): `coll` holds the points,
    //   V and T are empty, and the partition pairs its nodes (rows) with the
    //   nodes of the triangle tree `src` (columns) -- the evaluation operator
    //   of Section 5, Eq. (vector_eq);
    // kind 2, a tree of vertices (hm_build_vertex_tree): `coll` holds the
    //   vertex coordinates, `ibox` each vertex's star box (6 values), and the
    //   partition pairs the nodes of the triangle tree `src` (rows) with its
    //   nodes (columns) -- the double layer's K_Delta of Eq. (Kh)
    int32_t kind = 0;
    std::vector<double> ibox;
    std::shared_ptr<const hm_tree> src;
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
// INT16 near stream (the INT16 form): a column is a header of kNear16Head
// bytes (six FP32 scales, max |value| / 32767 of V_11 .. V_33 over the
// leaf's rows, then padding) and six segments of mp 16-bit values (offset
// binary, see cvt<int16_t>), 48 + 12 mp bytes: an odd number of 16-byte
// chunks, so that the columns read by eight consecutive consumer threads
// start in different shared-memory banks
constexpr int kNear16Head = 48;
// one admissible block of the far-field forward pass (32 bytes): column
// cluster start and size, first factor column, total rank, mesh, column offset
// of its V inside its group's row-major matrix, the group, and the rank of
// each of the seven kernels
struct FwdRec {
    int32_t s0, n, col0;
    int16_t C;
    uint16_t mesh;
    int32_t coff, grp;
    uint64_t kpack;  // rank of kernel q in bits 8q .. 8q+7
};
// the blocks that share a column cluster: V of all of them as one n x Cs
// matrix at element offset vbase (row-major, or unit-contiguous 8 x 8 tiles
// for the 16-bit forms); records first .. first + nrec - 1; the column descriptors of the
// 16-bit tensor-core forward pass at dbase .. dbase + Cs - 1
struct FwdGroup {
    int64_t vbase;
    int32_t s0, n, Cs, first;
    int16_t nrec;
    uint16_t mesh;
    int32_t dbase;
};
// column descriptor (x, y) of a forward-group column for the tensor-core
// forward pass: x = factor column | p << 28 | q << 30 with the block's kernel
// V_pq (p = q = 3: the c1 kernel), y = the bits of c1 su or c2 su; kFdSkip
// marks a padding column
constexpr uint32_t kFdSkip = 0xffffffffu;
constexpr int64_t kFdMaxCol = (1 << 28) - 1;
constexpr int kMaxGroupRecs = 64;
// a CTA's share of a forward group: rows j0 .. j0 + nrows of group `group`;
// a group taller than kFwdUnitRows has several units whose partial sums go
// to the z workspace (column zcol0 + chunk * Cs of the group's slice) and are
// added by a second pass in chunk order; zcol0 < 0 for a one-unit group
struct FwdUnit {
    int32_t group, j0, nrows, chunk;
    int32_t c0, ncols;  // the unit's columns of the group (at most kFwdUnitCols)
    int64_t zcol0;
};
// the second pass of the groups with several units, in column chunks (one
// CTA each): group, units, first z column of the group, the chunk's columns
struct FwdMulti {
    int32_t group, nchunk;
    int64_t zcol0;
    int32_t c0, ncols;
};
constexpr int kReduceCols = 128;  // columns of a second-pass chunk
constexpr int kFwdUnitRows = 256;
constexpr int kFwdUnitCols = 256;
// a unit as the tensor-core forward pass reads it: one load, no dependent
// load of its group (the fields are mesh relative but z0)
struct FwdTcUnit {
    int64_t v0;   // element offset in the mesh's V of the unit's contiguous 8 x 8 tiles
    int64_t z0;   // z column of the unit's first column, -1 for a one-unit group
    int32_t x0;   // first gathered-x position (group s0 + j0)
    int32_t d0;   // first column descriptor (group dbase + c0)
    int32_t ld8;  // elements from one 8-row core row of the unit to the next (ncols * 8)
    int16_t nrows, ncols;
    int32_t mesh, pad;
};
std::vector<FwdTcUnit> tc_units(const std::vector<FwdUnit>& units, const std::vector<FwdGroup>& groups);

// Device-side description of one mesh taking part in a product (a single
// matrix is a product over one mesh; a batch concatenates several).  Stream
// and table pointers are the mesh's own; the vectors live in shared arrays:
// x and y rows hold the mesh's dofs at element offset xoff; the gathered x
// and w hold G interleaved 4-vectors per cluster position / factor column,
// the mesh's first position at xgoff and first column at woff.
struct MeshDev {
    const void* Ul;   // leaf-major U stream (factor type of the form)
    const void* Vr;   // row-major V of every block
    const void* Nl;   // leaf-major near-field stream
    const float* SU;  // per-column U scales (16-bit forms) or null
    const uint2* fdesc;  // 16-bit forms: column descriptors of the forward groups
    const int32_t* leaf;
    const int64_t* lf_base;
    const int32_t* lf_ptr;
    const LeafFarItem* lf_items;
    // the far items merged into runs whose w columns are contiguous (the
    // kernels of a block, and blocks with consecutive columns): the w copies
    // of a stage, lr_items[lr_ptr[leaf] .. lr_ptr[leaf + 1]) with a sentinel
    const int32_t* lr_ptr;
    const LeafFarItem* lr_items;
    const int64_t* ln_base;
    const int32_t* ln_ptr;
    const LeafNearItem* ln_items;
    // INT16 form: the near columns after each leaf's diagonal block in the
    // INT16 near stream (null for the other forms, which stream every
    // column from Nl); the diagonal block's columns still come from Nl (FP32)
    const unsigned char* Nl16;
    const int64_t* ln16_base;   // byte offset of each leaf's INT16 columns
    const int32_t* ln16_diag;   // columns of each leaf's diagonal block
    const int32_t* perm;
    int64_t xoff, xgoff, woff;
    int32_t M, max_leaf;
    double c1, c2;
    float wbound;  // 16-bit forms: bound of |w| / max|x| over the factor columns
    float pad;
};

// A product over one or more meshes: device tables and work lists.
struct Plan {
    const MeshDev* meshes;      // nmesh entries (form specific)
    MeshDev mesh0;              // host copy of the only mesh when nmesh == 1
    int32_t nmesh;
    const int64_t* pos_prefix;  // nmesh + 1: cluster positions before each mesh
    int64_t npos;
    const FwdRec* fwd;          // the block records of every group
    const FwdGroup* groups;     // forward groups (records indexed over all meshes)
    const FwdUnit* units;       // nunits CTAs of the forward pass
    const FwdTcUnit* tcu;       // the same units for the tensor-core forward pass
    int64_t nunits;
    const FwdMulti* multi;      // nmulti groups added by the second pass
    int64_t nmulti;
    const int32_t* big;         // records of the blocks with |s| > 128 (several vectors: CTA per block)
    int64_t nbig;
    const int32_t* small;       // the other records (several vectors: warp per block)
    int64_t nsmall;
    int64_t zcols;              // z workspace columns (4-vectors per vector)
    const int2* work;           // (mesh, leaf) in processing order
    int64_t nwork;
    int32_t max_leaf;
    int* counters;              // kCounterInts ints of device memory (work counters, max|x| per vector)
    int* err;
    void* z;                    // forward partial sums: nrhs x zcols 4-vectors
};
// device ints of the counter region of a product: one work counter per
// launch (at most 64) and the max|x| words of a launch at offset 64
constexpr int kCounterInts = 128;


}  // namespace hm

struct hm_matrix {
    // geometry / partition
    int64_t M = 0;   // columns: triangles (and rows of a square matrix)
    int64_t Mr = 0;  // rows: M, or the points of an evaluation operator
    bool rect = false;  // evaluation operator ~V_h (Section 5, Eq. (vector_eq)): rows are points
    // the double layer's K_Delta (Section 4.2, Eq. (Kh)), a rectangular
    // operator too: rows the collocation points (triangles), columns the hat
    // functions of the vertices; one scalar kernel (slot 0), c1 = 1, c2 = 0
    bool dl = false;
    uint64_t mesh_fp = 0;  // fingerprint of the mesh (vertices and triangles) the matrix was built on
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
    // assembly work counted by the kernels: near-field pairs on the whole-
    // triangle rule, subdivision leaves, self pairs; ACA entries V_Delta, V_kl
    int64_t asm_count[5] = {0, 0, 0, 0, 0};

    // device arrays
    hm::DevBuf d_perm;   // int32 M: cluster position -> original id
    hm::DevBuf d_adm;    // Blk nadm
    hm::DevBuf d_near;   // Blk nnear
    hm::DevBuf d_rank;   // int32 nadm*7
    hm::DevBuf d_uoff, d_voff, d_coff;  // int64 nadm*7
    hm::DevBuf d_noff;   // int64 nnear
    hm::DevBuf d_leaf;   // int32 2*nleaves (t0, m)
    hm::DevBuf d_lf_base, d_lf_ptr, d_lf_items, d_lf_src;  // far stream per leaf
    hm::DevBuf d_lr_ptr, d_lr_items;                        // its w runs (MeshDev::lr_items)
    hm::DevBuf d_ln_base, d_ln_ptr, d_ln_items, d_ln_src;  // near stream per leaf
    hm::DevBuf d_ln16_base, d_ln16_diag;                   // INT16 near stream per leaf
    hm::DevBuf d_vb_base;                 // int64 nadm+1: V of each block (first row) in its group
    hm::DevBuf d_vb_ld;                   // int64 nadm+1: row stride of that V (its group's Cs)
    hm::DevBuf d_vb_coff;                 // int64 nadm+1: column offset of the block in its group
    hm::DevBuf fdesc;                     // uint2 per forward-group column (16-bit forms)
    int64_t dcols = 0;                    // forward-group columns (sum of Cs)
    hm::DevBuf d_fwd_all;                // FwdRec of every block, group by group
    hm::DevBuf d_groups;                 // FwdGroup
    hm::DevBuf d_units, d_multi;         // FwdUnit (the most data first), FwdMulti
    hm::DevBuf d_tcunits;                // FwdTcUnit of d_units
    hm::DevBuf d_big, d_small;           // record indices by block height, the most data first
    std::vector<int32_t> big_h, small_h;
    std::vector<hm::FwdUnit> unit_h;
    std::vector<hm::FwdMulti> multi_h;
    int64_t zcols = 0;
    std::vector<hm::FwdRec> fwd_h;       // host copies
    std::vector<hm::FwdGroup> grp_h;

    hm::DevBuf d_work;                   // int2 (0, leaf): leaves by decreasing streamed bytes
    std::vector<int32_t> leaf_order_h;   // host copy of the order
    std::vector<int64_t> leaf_bytes_h;   // streamed elements per leaf (U + near)
    hm::DevBuf d_pos_prefix;             // int64 {0, M}
    hm::DevBuf d_mesh[HM_NFORMS];        // MeshDev of this matrix, per packed form
    hm::DevBuf d_counters;               // int32 2*max_rhs: work counters of the streamed kernel
    hm::DevBuf d_err;                    // int32: set by a device wait that ran out
    int64_t ul_total = 0, nl_total = 0, vr_total = 0;
    int64_t nl16_bytes = 0;  // bytes of the INT16 near stream
    int64_t nl_diag_total = 0;  // elements of the leaves' diagonal blocks in the near stream

    // FP64 factor and near arenas in block order (ACA output, export)
    hm::DevBuf U64, V64, N64;
    // streaming arenas of each form (index = form): U leaf-major, V row-major
    hm::DevBuf Ul[HM_NFORMS], Vr[HM_NFORMS];
    hm::DevBuf Nl64, Nl32;  // near field leaf-major: FP64 form / all other forms
    hm::DevBuf SU, SV;      // per-column scales of the 16-bit forms (float, c_total)
    hm::DevBuf SW16;        // HM_I16: per-column factor of w, SU SV / 32767^2 (float, c_total)
    hm::DevBuf fdesc16;     // HM_I16: the forward column descriptors (as fdesc, with SW16)
    hm::DevBuf Nl16;        // HM_I16: INT16 near stream (nl16_bytes)
    bool packed[HM_NFORMS] = {false, false, false, false, false};
    float wbound_su = 0.0f;  // max over factor columns of (U column scale x |s| of its block)
    float wbound_sw16 = 0.0f;  // the same with the INT16 factor SU SV / 32767^2
    bool compacted = false;  // FP64 data released (hm_compact)
    bool aca_deferred = false;  // HM_DEFER_ACA: no ACA at assembly (adaptive product only)
    hm::DevBuf g_coll, g_tri, g_qp, g_qw, g_diam;  // cluster-order geometry of the entries (ACA on demand)
    hm::DevBuf d_rperm;  // evaluation operator: int32 Mr, point cluster position -> original point
    hm::DevBuf g_rows;   // evaluation operator: Mr x 3 points in cluster order
    // double layer: per triangle (cluster order) the unit normal and twice the
    // area; per vertex (cluster order) its star as (triangle position * 4 +
    // local vertex index), CSR; the triangles' vertex ids (original order)
    hm::DevBuf g_nrm, d_star_ptr, d_star, d_tris;
    hm::DevBuf d_mesh_k;  // square matrix: the mesh table with the double layer's coefficients
    hm::DevBuf dl_w;      // double layer: T_h u (3 x rows doubles)
    // evaluation operator: tables and workspace of its exact product
    // (hm_eval.cu; index names in hm_parts.cuh)
    static constexpr int kEvBufs = 14;
    hm::DevBuf ev[kEvBufs];
    int64_t ev_parts = 0;              // 3 sum |t| over the admissible blocks
    int64_t ev_nback = 0, ev_nnear = 0;  // work items (block, 32 rows) of the far and near passes
    int32_t ev_grid = 0;               // CTAs of the warp-per-item passes
    // rows of an entry: the collocation points, or the points of ~V_h
    const int32_t* row_perm() const { return rect ? d_rperm.as<int32_t>() : d_perm.as<int32_t>(); }

    // workspace
    int32_t max_rhs = 32;
    hm::DevBuf xg;  // max_rhs x M x 4 doubles (gathered x, cluster order, padded 4-vectors)
    hm::DevBuf wb;  // max_rhs x w_total doubles (one 4-vector per factor column)
    hm::DevBuf zb;  // max_rhs x zcols x 4 doubles (forward partial sums of the tall groups)
    hm::DevBuf xh, yh;  // device staging for hm_matvec_host (max_rhs x 3M doubles)

    // measurement hook (hm_profile_enable / hm_profile_read)
    bool prof_on = false;
    mutable std::vector<cudaEvent_t> prof_ev;  // 4 per profiled call
    mutable int64_t prof_calls = 0;
};

namespace hm {
// workspace of one product: gathered x (nrhs x M x 4), the far-field w
// vectors (nrhs x c_total x 4) and the forward partial sums (nrhs x zcols x
// 4), in the form's accumulation type, and the counters of the launches
struct Scratch {
    void* xg;
    void* w;
    int* counters;
    bool profile;  // record the measurement-hook events
    void* z = nullptr;
};
int matvec_device_scratch(const hm_matrix& H, const double* x, double* y, int32_t nrhs,
                          int64_t ld, int32_t form, cudaStream_t s, const Scratch& scr);
// bytes of Scratch a product of nrhs vectors in `form` needs (xg, w and the
// counters, each part 256-byte aligned)
size_t matvec_scratch_bytes(const hm_matrix& H, int32_t nrhs, int32_t form);
// a Scratch laid out in the matvec_scratch_bytes(H, nrhs, form) bytes at base
Scratch make_scratch(const hm_matrix& H, int32_t nrhs, int32_t form, void* base);
// Launch schedule of a product.  None of these change the arithmetic: every
// output element is summed in the same order under every schedule.
struct Sched {
    int32_t ctas_per_sm = 0;        // streamed leaf kernel: CTAs per SM (0 = as many as fit)
    cudaStream_t side = nullptr;    // non-null: the large-block forward kernel runs on `side`
    cudaEvent_t fork = nullptr, join = nullptr;  // (with these two events) beside the small-block one
};
// the product over the meshes of a plan: x, y rows of length >= total dofs
// with leading dimension ld; xg / w workspace with the plan's strides
int run_product(const Plan& P, int32_t form, const double* x, double* y, int32_t nrhs, int64_t ld,
                void* xg, void* w, cudaStream_t s, const hm_matrix* prof, const Sched* sched = nullptr);
// (re)write the single-mesh table of a packed form (after packing or a
// change of material)
int write_mesh_table(hm_matrix& H, int32_t form, cudaStream_t s);
MeshDev mesh_desc(const hm_matrix& H, int32_t form);
// record event `which` (0..3) of the current profiled call, if profiling
void prof_mark(const hm_matrix& H, int which, cudaStream_t s);
// kernels launchers (implemented in the .cu files)
int assemble_device(const hm_tree& tr, hm_matrix& H);
// Algorithm 1 on demand: the (block, kernel) tasks bk[q] = block * 7 + kernel,
// each stopped after kmax crosses at most (or earlier by its stop test), into
// a new arena `out` from the matrix's allocator; per task its rank and the
// element offset of its U (k x m) with V (k x n) right after it.  The same
// task gives the same first crosses for any kmax (the kernel is
// deterministic).
// State of resumable ACA tasks (device arrays indexed by block * 7 + kernel):
// the crosses so far, the rows in Z, the next row, the exit flags of the last
// run (bit 0: stopped at kmax, so it can go on), ||S_k||_F^2, Z itself (m
// bytes per task at zoff), and the previous run's U (k x m, V right after) or
// null to start afresh.  A resumed task takes exactly the steps a fresh run to
// the same kmax would take after its first k crosses.  cap_hint (elements,
// 0 = the exact bound kmax (m + n) per task) sizes a first arena for runs
// without resume; the batch runs again into an exact arena if it overflows.
struct AcaResume {
    int32_t *k, *nz, *irow, *flags;
    double* S2;
    unsigned char* Z;
    const int64_t* zoff;
    const double* const* prevU;
};
int aca_on_demand(hm_matrix& H, const std::vector<int32_t>& bk, int kmax, cudaStream_t s, DevBuf& out,
                  std::vector<int32_t>& rank, std::vector<int64_t>& off, const AcaResume* resume = nullptr,
                  std::vector<int32_t>* flags = nullptr, size_t cap_hint = 0);
// the evaluation operator (a matrix assembled from a point tree): tables and
// workspace of its product (hm_eval.cu), built once at assembly (and by
// hm_baca for a square matrix at its first call)
int eval_prepare(hm_matrix& H);
// the FP32 form of an evaluation operator: FP32 copies of its block-ordered
// U, V and near arenas (in Ul[HM_FP32], Vr[HM_FP32] and Nl32), same offsets
int eval_pack_fp32(hm_matrix& H, cudaStream_t s);
// the product of a rectangular operator (evaluation operator or the double
// layer's K_Delta) in HM_FP64 or a packed HM_FP32; accumulate: u += instead of u =
int eval_apply(const hm_matrix& H, const double* t, double* u, int32_t nrhs, int32_t form, bool accumulate,
               cudaStream_t s);
// the single-layer product of a square matrix with the coefficients of
// Eq. (Vh) replaced by (c1, c2) (one vector; its mesh table in d_mesh_k)
int matvec_device_coeffs(hm_matrix& H, const double* x, double* y, int32_t form, double c1, double c2,
                         cudaStream_t s);
int matvec_device(const hm_matrix& H, const double* x, double* y, int32_t nrhs, int64_t ld,
                  int32_t form, cudaStream_t s);
int pack_device(hm_matrix& H, int32_t form, cudaStream_t s);
// fill the launch caches of a form's kernels (call before capture or threads)
int product_prepare(int32_t form, int* ctas_per_sm);
// the solver on caller-provided memory (hm_solve.cu)
size_t solve_workspace_bytes(int64_t n, int32_t restart);
int solve_check_params(const hm_matrix* H, hm_solve_params& p);
int solve_device(const hm_matrix& H, const double* g, double* t, const hm_solve_params& p, hm_solve_info* info,
                 cudaStream_t s, void* ws, void* scratch);
}  // namespace hm
