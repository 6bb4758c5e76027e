/*
 * hmat.h -- C ABI of the GB300 (sm_103a) H-matrix library for the collocation
 * Lame single-layer operator (Bauer & Bebendorf, "Adaptive H-Matrix
 * Computations in Linear Elasticity").
 *
 * Conventions for every entry point:
 *   - Plain C types only.  A "device pointer" is memory of the current CUDA
 *     device; a "host pointer" is ordinary (preferably pinned) host memory.
 *   - `stream` is a cudaStream_t passed as void* (NULL = legacy default stream).
 *     Device work is stream ordered and asynchronous unless stated otherwise;
 *     results are valid once the stream has been synchronised.
 *   - Return value 0 (HM_OK) on success, a negative HM_E* code otherwise; the
 *     text of the last error of the calling thread is hm_last_error().
 *     Nothing throws across this boundary.
 *   - Degrees of freedom are ordered dof = 3*i + a (triangle i in the mesh's
 *     original order, component a in {0,1,2}).  Multi-RHS vectors are nrhs
 *     rows of length >= 3M with leading dimension ld (elements).
 *   - Objects (hm_tree, hm_matrix) are owned by the library; destroy them with
 *     the matching *_destroy call.  Input arrays are copied and never retained.
 */
#ifndef HMAT_H
#define HMAT_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* status codes */
#define HM_OK 0
#define HM_EINVAL (-1)    /* invalid argument: bad mesh, E <= 0, nu outside (0, 1/2), ... */
#define HM_ENOMEM (-2)    /* device or host allocation failed */
#define HM_ENOTCONV (-3)  /* iterative solve stopped before reaching the tolerance */
#define HM_ETIMEOUT (-4)  /* a bounded device wait ran out; the context stays usable */
#define HM_EDEVICE (-5)   /* a CUDA call failed */
#define HM_ERANK (-6)     /* an ACA block reached the rank cap (result kept, flagged) */
#define HM_EBUSY (-7)     /* request rejected by admission (queue full or footprint too large) */

/* storage / arithmetic forms of the H-matrix-vector product */
#define HM_FP64 0 /* factors and near field FP64, FP64 accumulation ("plain form") */
#define HM_FP32 1 /* factors and near field FP32, FP32 accumulation */
#define HM_BF16 2 /* factors BF16 with per-column FP32 scales, near field FP32, FP32 acc. */
#define HM_FP16 3 /* factors FP16 with per-column FP32 scales, near field FP32, FP32 acc. */
#define HM_I16 4  /* factors INT16 with per-column FP32 scales on U and V (block floating
                   * point: a column is stored as round(32767 v / max|v|)); near field:
                   * the leaves' diagonal blocks FP32, every other near column INT16
                   * with six FP32 scales; FP32 acc.  Same factor bytes as FP16; a
                   * column keeps 15 significant bits at its largest entries instead
                   * of FP16's 11, which makes the product's error against HM_FP64
                   * about 10 times smaller */
#define HM_NFORMS 5

/* largest leaf size b_min of a cluster tree (see hm_build_cluster_tree) */
#define HM_MAX_LEAF 336

typedef struct hm_tree hm_tree;     /* cluster tree + block partition (host) */
typedef struct hm_matrix hm_matrix; /* assembled H-matrix resident on the device */

/* Optional device allocator.  alloc returns a device pointer of at least
 * `bytes` (NULL on failure) usable on `stream`; free releases it.  When no
 * allocator is given the library uses cudaMallocAsync / cudaFreeAsync. */
typedef struct {
    void* (*alloc)(size_t bytes, void* stream, void* user);
    void (*free)(void* ptr, size_t bytes, void* stream, void* user);
    void* user;
} hm_allocator;

/* ---------------------------------------------------------------------------
 * hm_build_cluster_tree -- cluster tree T_I and block partition P (Section
 * 2.1: binary tree of index sets, leaves of at most b_min = leaf indices;
 * Eq. (adm): a block t x s is admissible iff
 *     min(diam X_t, diam X_s) < eta * dist(X_t, X_s),
 * evaluated on the bounding boxes of the clusters' triangle vertices).
 * Host-only: touches no GPU.
 *   verts  host, nv x 3 float64, row-major vertex coordinates
 *   tris   host, nt x 3 int32, vertex ids of each flat triangle tau_i
 *          (Section 4.2); the collocation point of tau_i is its centroid
 *   leaf   b_min, 1 <= b_min <= HM_MAX_LEAF (the streamed product keeps the
 *          rows of one leaf in one CTA and one near-field column of a leaf,
 *          6 x 336 FP64 values, in one 16 KB shared-memory stage); eta > 0
 *   out    receives a new tree (NULL on error)
 * Split rule: longest axis of the box of the collocation points, median of a
 * stable sort by (coordinate, triangle id), first son floor(n/2).
 * Errors: HM_EINVAL (nv < 3, nt < 1, vertex id out of range, degenerate
 * triangle, leaf outside 1..HM_MAX_LEAF, eta <= 0, non-finite coordinate),
 * HM_ENOMEM.
 * ------------------------------------------------------------------------- */
int hm_build_cluster_tree(const double* verts, int64_t nv, const int32_t* tris, int64_t nt,
                          int32_t leaf, double eta, hm_tree** out);

/* sizes of a tree: counts[0..5] = M, nodes, admissible blocks, near blocks,
 * leaves, depth */
int hm_tree_sizes(const hm_tree* tree, int64_t counts[6]);

/* Export for inspection and tests (host arrays sized from hm_tree_sizes):
 *   perm[M]          cluster position -> original triangle id
 *   nodes[nodes*5]   (lo, hi, son0, son1, level) per node, pre-order, sons -1
 *                    for a leaf; [lo, hi) are cluster positions
 *   adm[nadm*2]      (row node, column node) of each admissible block
 *   near[nnear*2]    (row node, column node) of each near (dense) block
 * Any pointer may be NULL to skip that array. */
int hm_tree_export(const hm_tree* tree, int64_t* perm, int64_t* nodes, int64_t* adm,
                   int64_t* near_blocks);

void hm_tree_destroy(hm_tree* tree);

/* ---------------------------------------------------------------------------
 * hm_build_point_tree -- the rows of the evaluation operator ~V_h of
 * Section 5, Eq. (vector_eq): the displacement
 *     u_h(x_i) = sum_j int_{tau_j} S(x_i - y) ds_y t_j
 * at points x_1 .. x_l of the domain; ~V_h[i, j] is the collocation entry of
 * hm_aca_assemble with x_i in place of the centroid c_i (never a self pair).
 * Builds the cluster tree of the points (the split rule of
 * hm_build_cluster_tree; boxes of the points) and the block partition of
 * (point tree) x (triangle tree of `surface`) under Eq. (adm) with the
 * surface tree's eta.  Host only.
 *   surface  a triangle tree (copied; may be destroyed afterwards)
 *   pts      host, npts x 3 float64 points off the surface (a point on a
 *            triangle gives non-finite or inaccurate entries: the 7-point rule
 *            and its subdivision assume x outside tau_j)
 *   leaf     b_min of the point tree, 1..HM_MAX_LEAF
 *   out      new tree: hm_tree_sizes / hm_tree_export describe the point tree
 *            (perm over the points, nodes) and the partition (row node of the
 *            point tree, column node of the surface tree)
 * hm_aca_assemble on this tree assembles ~V_h (FP64 factors and near field;
 * hm_pack(H, HM_FP32) adds FP32 copies, the only other form); apply it with
 * hm_eval_points, or adaptively with hm_amvm.
 * Errors: HM_EINVAL (NULL argument, `surface` itself a point tree, npts < 1,
 * leaf outside 1..HM_MAX_LEAF, non-finite coordinate), HM_ENOMEM.
 * ------------------------------------------------------------------------- */
int hm_build_point_tree(const hm_tree* surface, const double* pts, int64_t npts, int32_t leaf,
                        hm_tree** out);

/* ---------------------------------------------------------------------------
 * hm_build_vertex_tree -- the column side of the double layer's K_Delta
 * (Section 4.2, Eq. (Kh): rows the collocation points, columns the hat
 * functions psi_p of the mesh vertices).  Builds the cluster tree of the
 * vertices (the split rule of hm_build_cluster_tree on the vertex
 * coordinates) whose boxes are the unions of the vertices' stars (the boxes
 * of all triangles holding the vertex, the support of psi_p), and the block
 * partition of (triangle tree of `surface`) x (vertex tree) under Eq. (adm)
 * with the surface tree's eta.  Host only.
 *   surface  a triangle tree (copied)
 *   leaf     b_min of the vertex tree, 1..HM_MAX_LEAF
 *   out      new tree: hm_tree_sizes / hm_tree_export describe the vertex
 *            tree (perm over the vertices, nodes) and the partition (row node
 *            of the surface tree, column node of the vertex tree)
 * hm_aca_assemble on this tree assembles K_Delta (Eq. (Kh) in collocation
 * form, the collocation point's own flat panel contributing 0):
 *   K_Delta[i, p] = 1/(4 pi) sum over the triangles tau_j holding vertex p of
 *                   int_{tau_j} (c_i - y).n_j / |c_i - y|^3 psi_p(y) ds_y,
 * near blocks entry by entry and one ACA (Algorithm 1) per admissible block,
 * with the quadrature of the single layer (the 7-point rule, subdivided
 * near c_i).  The matrix is a rectangular operator (rows the triangles,
 * columns the vertices): hm_eval_points applies K_Delta to each component
 * (u of 3 nv values, dof 3p + b), hm_double_layer_matvec the whole K_h.
 * A block whose triangles all lie in one plane has K_Delta = 0 in exact
 * arithmetic; its computed entries are rounding noise (not special-cased).
 * Errors: HM_EINVAL (NULL, `surface` not a triangle tree, leaf out of range,
 * a vertex in no triangle), HM_ENOMEM.
 * ------------------------------------------------------------------------- */
int hm_build_vertex_tree(const hm_tree* surface, int32_t leaf, hm_tree** out);

/* ---------------------------------------------------------------------------
 * hm_eval_points -- u = ~V_h t (Section 5, Eq. (vector_eq) with W_h u = 0):
 * the displacement at the points of an evaluation operator for densities t.
 *   t      device, nrhs rows of 3M float64 (dof 3j + b, original triangle order)
 *   u      device, nrhs rows of 3 npts float64 (3i + a, original point
 *          order), overwritten; t and u must not overlap
 *   form   HM_FP64: the exact product of the assembled H-matrix in FP64;
 *          HM_FP32 (after hm_pack(H, HM_FP32)): the same product from FP32
 *          copies of the factors and near field with FP32 arithmetic
 * Every admissible block applies all its crosses, every near block its
 * entries, and each output element is summed in a fixed order (repeated
 * calls agree bitwise).
 * Asynchronous on `stream`; allocates nothing (its workspace was reserved at
 * assembly); calls on the same operator must not overlap on the device.
 * Errors: HM_EINVAL (NULL argument, not an evaluation operator, assembled
 * with HM_DEFER_ACA, nrhs < 1, a form other than HM_FP64 or a packed
 * HM_FP32), HM_EDEVICE.
 * ------------------------------------------------------------------------- */
int hm_eval_points(const hm_matrix* H, const double* t, double* u, int32_t nrhs, int32_t form, void* stream);

/* Assembly parameters. */
typedef struct {
    double E;            /* Young modulus > 0 (Section 1) */
    double nu;           /* Poisson ratio in (0, 1/2) */
    double aca_eps;      /* eps_ACA > 0 (Algorithm 1) */
    double aca_eta_stop; /* beta of Algorithm 1's stop factor eps(1-beta)/(1+eps); 0 = plain eps */
    int32_t kmax;        /* rank cap per block and kernel, 1..256 (0 = 128) */
    int32_t max_rhs;     /* largest nrhs a later hm_matvec may use, 1..64 (0 = 32) */
    int32_t flags;       /* HM_DEFER_FP64: do not build the FP64 product form at assembly */
    int32_t pad;
} hm_params;

/* hm_params.flags: build the FP64 product form only on hm_pack(H, HM_FP64)
 * (saves its memory while a matrix is assembled only to be packed into a
 * reduced form and compacted) */
#define HM_DEFER_FP64 1
/* hm_params.flags: run no ACA at assembly (tree, partition, near field and
 * product tables only); such a matrix cannot be packed and serves the
 * adaptive product with ACA on demand (hm_amvm, HM_AMVM_ACA_ON_DEMAND) */
#define HM_DEFER_ACA 2

/* ---------------------------------------------------------------------------
 * hm_aca_assemble -- assemble the H-matrix of V_h on the device.
 * Eq. (Vh) in collocation form with the prefactor read as 1/(4 pi):
 *   V_h = c1 diag(V_Delta, V_Delta, V_Delta) + c2 [V_kl],
 *   c1 = (1+nu)(3-4nu) / (2E(1-nu)),  c2 = (1+nu) / (2E(1-nu)),
 *   V_Delta[i,j] = 1/(4pi) int_{tau_j} 1/|c_i - y| ds_y,
 *   V_kl[i,j]    = 1/(4pi) int_{tau_j} (c_i-y)_k (c_i-y)_l / |c_i - y|^3 ds_y.
 * Near (non-admissible) blocks are computed entry by entry (Section 2.2);
 * every admissible block gets one ACA (Algorithm 1) per scalar kernel
 * (V_Delta, V_11, V_12, V_13, V_22, V_23, V_33), in FP64.  The factors do not
 * depend on E, nu; c1 and c2 are applied in the product.
 *   tree   from hm_build_cluster_tree (not retained)
 *   prm    parameters (validated; HM_EINVAL on a bad value)
 *   alloc  optional device allocator (NULL: cudaMallocAsync)
 *   stream stream for all device work; the call synchronises it before return
 *   out    receives the matrix
 * The FP64 product form is built too unless prm->flags has HM_DEFER_FP64.
 * A tree from hm_build_point_tree gives the evaluation operator ~V_h instead
 * (rows are its points; HM_DEFER_FP64 has no effect there).
 * Returns HM_ERANK (matrix still valid) if a block hit the rank cap below
 * min(|t|, |s|).
 * ------------------------------------------------------------------------- */
int hm_aca_assemble(const hm_tree* tree, const hm_params* prm, const hm_allocator* alloc,
                    void* stream, hm_matrix** out);

/* Change E, nu of an assembled matrix (the factors are material-free). */
int hm_set_material(hm_matrix* H, double E, double nu);

/* Build the streaming copy used by a product form (HM_FP64 is built at
 * assembly unless deferred).  Idempotent; synchronises `stream`. */
int hm_pack(hm_matrix* H, int32_t form, void* stream);

/* ---------------------------------------------------------------------------
 * hm_matvec -- y = V_h x (H-matrix-vector product, Section 2: each admissible
 * block applies U (V^T x) at O(k(|t|+|s|)) cost, each near block its dense
 * entries; the contributions of all blocks of a row are summed into y).
 *   x, y    device pointers, nrhs rows of length 3M, leading dimension ld
 *           (>= 3M); y is overwritten; x and y must not overlap
 *   nrhs    1 .. max_rhs of the assembly
 *   form    HM_FP64 or a packed form (hm_pack first)
 * Deterministic: every output element is summed in a fixed order, so repeated
 * calls give bitwise-identical results.  Asynchronous on `stream`; allocates
 * nothing.  Calls on the same matrix must not overlap in time on the device
 * (they share the matrix's workspace).
 * ------------------------------------------------------------------------- */
int hm_matvec(const hm_matrix* H, const double* x, double* y, int32_t nrhs, int64_t ld,
              int32_t form, void* stream);

/* ---------------------------------------------------------------------------
 * hm_matvec_noalloc -- the product of hm_matvec for callers that cannot
 * allocate device memory when they need it (a fixed, pre-reserved memory
 * budget such as a real-time or embedded loop, or a host framework that owns
 * all allocation).  The paper has no counterpart; this is a library service.
 * Same arguments, result and determinism as hm_matvec, but the workspace
 * comes from one static device array of 32 MiB inside the library instead of
 * the matrix's own workspace.
 *   - Allocates nothing and calls no allocating routine.
 *   - The array is held by every GPU on which the library is loaded, until
 *     the process exits.
 *   - The workspace of a product is the sum of four parts, each rounded up
 *     to a multiple of 256 bytes, with ta = 8 bytes for HM_FP64 and 4 for
 *     the other forms:
 *       gathered x:            nrhs * 4M * ta
 *       w = V^T x per factor:  nrhs * 4 * (sum of ACA ranks) * ta
 *       forward partial sums:  nrhs * 4 * zcols * ta, where zcols sums, over
 *                              the column clusters taller than 256 rows,
 *                              (number of 256-row chunks) x (their factor
 *                              columns)
 *       counters:              512 bytes
 *     Products needing more than 32 MiB are rejected with HM_EINVAL, and
 *     the message states the exact need.
 *   - The address of the array is looked up (cudaGetSymbolAddress) on every
 *     call; the first call on a device may load the library's device code
 *     on that device, so make that first call before any stream capture.
 *   - All calls share the array: calls whose kernels overlap in time on the
 *     device race and give wrong results.  Nothing in it needs to start at
 *     zero (every call writes each element before reading it).
 * ------------------------------------------------------------------------- */
int hm_matvec_noalloc(const hm_matrix* H, const double* x, double* y, int32_t nrhs, int64_t ld,
                      int32_t form, void* stream);

/* ---------------------------------------------------------------------------
 * hm_double_layer_matvec -- y = K_h u, the double-layer operator of Section
 * 4.2, Eq. (Kh), in collocation form:
 *   K_h = diag(K_Delta) - diag(V_Delta) T_h + E/(1+nu) V_h T_h,
 * T_h the surface curls T_kl = n_l d_k - n_k d_l of the hat functions
 * (constant on each flat triangle; the tangential derivative, antisymmetric
 * in (k, l), T_h = [[0, T12, T13], [-T12, 0, T23], [-T13, -T23, 0]]).  The
 * last two terms are one single-layer product of w = T_h u with the
 * coefficients ((1 - 2nu) / (2(1 - nu)), 1 / (2(1 - nu))) in place of
 * (c1, c2): E cancels.  Rigid motions u (translations, rotations) give
 * K_h u = -u/2 up to the discretisation error.
 *   V     the single layer of the mesh (hm_aca_assemble on its triangle
 *         tree), with `form` packed; its material nu is used.  The first call
 *         allocates a small mesh table in V (hence non-const).
 *   K     K_Delta (hm_aca_assemble on hm_build_vertex_tree of the same
 *         triangle tree); FP64 factors
 *   u     device, nrhs rows of 3 nv doubles (vertex p, component b at 3p + b,
 *         original vertex order)
 *   y     device, nrhs rows of 3M doubles (3i + a, original triangle order),
 *         overwritten; must not overlap u
 *   form  the product form of the V_h part (K_Delta is applied in FP64)
 * Asynchronous on `stream`; calls on the same V or K must not overlap.
 * Errors: HM_EINVAL (NULL, V not a triangle tree's matrix or K not a vertex
 * tree's, different meshes, nrhs < 1, form not packed, K without factors),
 * HM_ENOMEM, HM_EDEVICE.
 * ------------------------------------------------------------------------- */
int hm_double_layer_matvec(hm_matrix* V, const hm_matrix* K, const double* u, double* y, int32_t nrhs,
                           int32_t form, void* stream);

/* Same product with HOST x and y: copies x in, runs hm_matvec, copies y back
 * and synchronises `stream`.  Pinned host memory gives the fastest copies. */
int hm_matvec_host(const hm_matrix* H, const double* x_host, double* y_host, int32_t nrhs,
                   int64_t ld, int32_t form, void* stream);

/* ---------------------------------------------------------------------------
 * hm_batch -- the product of hm_matvec over many resident matrices at once
 * (meshes of different sizes and materials).  The paper treats one mesh at
 * a time; the batch is a library service for many independent problems: it
 * runs each phase of the product (Section 2: V^T x per admissible block, then
 * U w and the near field per row cluster) as ONE launch over every block of
 * every member, with one work list of (mesh, leaf) items for the persistent
 * per-leaf kernel.
 *   mats     nmat (1..65535) distinct assembled matrices, each with `form`
 *            packed.  The batch refers to their device data: they must
 *            outlive it and must not change (hm_set_material on a member
 *            after hm_batch_create is not seen by the batch; create a new one).
 *   max_rhs  largest nrhs of hm_batch_matvec (sizes the batch's workspace)
 * Vector layout: member m's dofs (3 M_m, dof 3i + a in its own original
 * order) sit at offsets dof_offsets[m] .. dof_offsets[m+1] of each row of x
 * and y; hm_batch_layout returns the nmat + 1 offsets and sizes[0..3] =
 * members, total dofs, forward groups (admissible blocks sharing a column
 * cluster), leaves.
 * Result: member m's part of y is bitwise equal to hm_matvec(mats[m], ...)
 * on its part of x, under every schedule.
 * Allocates its workspace through the first member's allocator.
 * ------------------------------------------------------------------------- */
typedef struct hm_batch hm_batch;

/* Launch schedule of a batched product.  No knob changes any result. */
typedef struct {
    int32_t leaf_ctas_per_sm; /* CTAs per SM of the per-leaf kernel (0 = as many as fit) */
    int32_t work_order;       /* 0: all (mesh, leaf) items by decreasing bytes; 1: member by member */
    int32_t fork_forward;     /* 1: large- and small-block forward kernels on two streams */
    int32_t pad;
} hm_schedule;

int hm_batch_create(const hm_matrix* const* mats, int32_t nmat, int32_t form, int32_t max_rhs,
                    hm_batch** out);
int hm_batch_layout(const hm_batch* B, int64_t* dof_offsets, int64_t sizes[4]);

/* y = V_h x for every member: x, y device pointers, nrhs (1..max_rhs) rows
 * of length >= total dofs, leading dimension ld; must not overlap.
 * use_graph != 0: the product is captured once into a CUDA graph (per x, y,
 * nrhs, ld and schedule; a change of any of them captures a new one) and
 * replayed with one cudaGraphLaunch on `stream`.  Asynchronous; calls on the
 * same batch must not overlap on the device (shared workspace). */
int hm_batch_matvec(hm_batch* B, const double* x, double* y, int32_t nrhs, int64_t ld,
                    int32_t use_graph, void* stream);

/* Time every candidate schedule (CTAs per SM in {max, 1}, both work orders,
 * forward on one or two streams) over `reps` products of nrhs right-hand
 * sides on `stream` and keep the fastest; returns it and its ms per product.
 * Allocates two temporary vectors; synchronises `stream`. */
int hm_batch_autotune(hm_batch* B, int32_t nrhs, int32_t reps, hm_schedule* chosen, double* ms,
                      void* stream);
int hm_batch_set_schedule(hm_batch* B, const hm_schedule* s);
int hm_batch_get_schedule(const hm_batch* B, hm_schedule* s);
/* as hm_check, for the batch's own products */
int hm_batch_check(const hm_batch* B);
void hm_batch_destroy(hm_batch* B);

/* ---------------------------------------------------------------------------
 * hm_server -- a request loop over resident H-matrices (a library service;
 * the paper solves one problem at a time).  Matvec requests (y = V_h x for
 * 1..32 vectors, Section 2's product) and solve requests (hm_solve's GMRES
 * with iterative refinement) on any of the server's matrices arrive over
 * time.  A request is admitted, in arrival order, as soon as one of `slots`
 * worker streams is free AND its device footprint fits in the free part of
 * a fixed arena of budget_bytes (its vectors, the product workspace and, for
 * a solve, the Krylov basis); admitted requests run concurrently on their
 * own streams, so their kernels overlap on the device while later arrivals
 * keep being admitted.  Requests of one kind are admitted in arrival order;
 * a solve that waits for one of its solve_slots does not hold back the
 * matvec requests behind it, and matvec requests run on streams of the
 * device's greatest priority (solves on its least), so that their kernels'
 * CTAs are started first.  Arrivals that find queue_cap requests waiting,
 * or whose footprint exceeds the arena, are rejected (HM_EBUSY).
 * Every request runs the kernels it would run alone, with its own
 * workspace: its result is bitwise the same alone and in any mix.
 * The matrices must stay alive and unchanged while the server exists; the
 * arena is allocated once through the first matrix's allocator.
 * ------------------------------------------------------------------------- */
typedef struct hm_server hm_server;

#define HM_REQ_MATVEC 0
#define HM_REQ_SOLVE 1

typedef struct {
    int32_t slots;          /* requests in flight at most (1..64 worker streams) */
    int32_t queue_cap;      /* waiting requests at most; later arrivals are rejected */
    int64_t budget_bytes;   /* device arena for the footprints of requests in flight */
    int32_t matvec_form;    /* packed form of matvec requests */
    int32_t inner_form;     /* solve: GMRES product form */
    int32_t residual_form;  /* solve: refinement residual form */
    int32_t restart;        /* solve: GMRES restart (0 = 30) */
    double inner_tol;       /* solve: residual reduction per GMRES solve (0 = 1e-3) */
    int32_t max_inner;      /* solve: cap on inner products (0 = 1000) */
    int32_t solve_slots;    /* at most this many slots run solves at once (0 = any slot); the
                               other slots are kept for matvec requests, so that long solves
                               cannot hold every slot */
} hm_server_params;

typedef struct {
    double arrival_s;      /* seconds after the start of hm_server_run */
    int32_t mesh;          /* index into the server's matrices */
    int32_t kind;          /* HM_REQ_MATVEC or HM_REQ_SOLVE */
    int32_t nrhs;          /* matvec: 1..32 vectors; solve: ignored (1) */
    int32_t seed;          /* inputs drawn on the device when x_host is NULL */
    double tol;            /* solve: relative residual target (0 = 1e-6) */
    const double* x_host;  /* nrhs x 3M inputs (matvec x, solve g) or NULL */
    double* y_host;        /* nrhs x 3M results (matvec y, solve t) or NULL */
} hm_request;

typedef struct {
    int32_t status;        /* HM_OK, HM_ENOTCONV (solve), HM_EBUSY (rejected), other errors */
    int32_t iterations;    /* solve: inner GMRES iterations */
    double arrival_s;      /* request arrival (0 when not replayed in real time) */
    double start_s;        /* admission */
    double done_s;         /* completion, results copied back */
    double rel_residual;   /* solve: final relative residual in residual_form */
} hm_result;

int hm_server_create(const hm_matrix* const* mats, int32_t nmat, const hm_server_params* p,
                     hm_server** out);
/* device bytes request q would hold while in flight */
int hm_server_footprint(const hm_server* S, const hm_request* q, int64_t* bytes);
/* Serve n requests and return when all are finished or rejected.
 * realtime != 0: request i arrives at reqs[i].arrival_s (sorted); otherwise
 * all arrive at once.  Inputs with x_host == NULL are uniform[-1, 1) values
 * from a counter-based generator (splitmix64 of the seed and the index).
 * Blocks the calling thread (which schedules); one worker thread per slot. */
int hm_server_run(hm_server* S, const hm_request* reqs, int32_t n, int32_t realtime, hm_result* out);
void hm_server_destroy(hm_server* S);

/* ---------------------------------------------------------------------------
 * hm_solve -- solve V_h t = g (one right-hand side) for the single-layer
 * density t.  Restarted GMRES(m) runs on the product form `inner_form` (for
 * speed), inside iterative refinement whose residual r = g - V_h t is
 * computed with `residual_form` (FP64 by default): the result satisfies
 *     ||g - V_h t||_2 <= tol ||g||_2
 * for the H-matrix operator in that form (FP64 by default) (the paper solves with the assembled
 * approximation of the operator as well; the solver choice is this library's).
 *   g, t    device vectors of 3M doubles (dof 3i + a); t is overwritten (or
 *           used as the initial guess if use_initial_guess)
 *   info    optional: iterations, restarts, refinements, final relative residual
 * Synchronises `stream`.  Allocates (restart + 5) vectors of workspace through
 * the matrix's allocator for the duration of the call.  Returns HM_ENOTCONV
 * (info filled, t = best iterate) if the caps are reached first.
 * ------------------------------------------------------------------------- */
typedef struct {
    double tol;                /* relative FP64 residual target (> 0) */
    double inner_tol;          /* residual reduction asked of each GMRES solve (0 = 1e-3) */
    int32_t inner_form;        /* HM_FP16, HM_BF16, HM_FP32 or HM_FP64 (must be packed) */
    int32_t restart;           /* GMRES restart length m (0 = 50, at most 127) */
    int32_t max_inner;         /* cap on the total number of inner products (0 = 1000) */
    int32_t max_refine;        /* cap on refinement steps (0 = 20) */
    int32_t use_initial_guess; /* nonzero: start from the given t */
    int32_t residual_form;     /* form of the refinement residual: HM_FP64 (0, the default) or,
                                  on a compacted matrix, a packed reduced form */
} hm_solve_params;

typedef struct {
    int32_t iterations;   /* inner products (GMRES iterations) */
    int32_t restarts;
    int32_t refinements;  /* FP64 residual evaluations after the first */
    int32_t pad;
    double rel_residual;  /* ||g - V_h t|| / ||g|| with the FP64 form */
} hm_solve_info;

int hm_solve(const hm_matrix* H, const double* g, double* t, const hm_solve_params* p,
             hm_solve_info* info, void* stream);

/* ---------------------------------------------------------------------------
 * Adaptive matrix-vector multiplication (Section 3, Algorithm 2), FP64.
 *
 * Computes b_k = A_k x for a sequence of approximations A_k of the assembled
 * H-matrix: A_k keeps, on each admissible block t x s, the first r_b crosses
 * of every one of its seven ACA sequences (a shorter sequence is used whole),
 * A_0 has r_b = r0; the look-ahead A^_k has r_b + look crosses; near blocks
 * are exact in both.  gamma_k = ||A_k x - A^_k x||_2 is the error estimator.
 * Step 3 marks blocks through the dof rows in decreasing |(A_k x - A^_k x)_i|
 * (ties: increasing row), adding every block t x s with i in t whose part
 * satisfies |[(A_k - A^_k)_ts x_s]_i| >= (1 - theta)(c_sp N_r N_c)^{-1/2}
 * gamma_k (N_r = N_c = 3M dofs; for an evaluation operator N_r = 3 npts rows;
 * c_sp the sparsity constant of Section 2.1), until gamma_k - gamma_k(P_k) >=
 * theta gamma_k (the stopping row found by bisection over the sorted rows);
 * marked blocks take the look-ahead ranks.  The loop ends when gamma_k <= eps
 * ||A^_k x||_2, when no block can be refined, or after max_iter refinements.
 * On an evaluation operator (hm_build_point_tree) this is the adaptive
 * evaluation of the displacement at the points that Section 5 proposes.
 *   x, y      device, original dof order: x 3M doubles, y 3M (3 npts for an
 *             evaluation operator) doubles; y = A_k x at exit
 *   info      optional: iterations, c_sp, last gamma, ||A^_k x||, crosses
 *             used by A_k and by the assembled ACA, blocks marked in all
 *   gamma_hist, gamma_rest_hist   optional host arrays of hist_cap entries:
 *             gamma_k per iteration, gamma_k(P_k) per refinement
 *   block_ranks  optional host array of nadm ints: r_b at exit
 * Needs the FP64 factors (or HM_AMVM_ACA_ON_DEMAND) and the near field
 * (HM_EINVAL after hm_compact).
 * Allocates about 40 (3M) + 24 sum|t| bytes of workspace (with ACA on demand
 * also the factors it computes and about 7 sum|t| bytes of ACA state)
 * through the matrix's allocator for the duration of the call; synchronises
 * `stream`.
 * ------------------------------------------------------------------------- */
typedef struct {
    double theta;      /* Doerfler parameter in (0, 1) (0 = 0.7) */
    double eps;        /* stop when gamma_k <= eps ||A^_k x|| (>= 0) */
    int32_t r0;        /* crosses per block and kernel in A_0 (0 = 2), at most 32 */
    int32_t look;      /* look-ahead ACA steps (0 = 2), at most 32 */
    int32_t max_iter;  /* cap on refinement steps (0 = 1000) */
    int32_t flags;     /* HM_AMVM_ACA_ON_DEMAND */
} hm_amvm_params;

/* hm_amvm_params.flags: run Algorithm 1 on demand (every block-kernel to
 * r0 + look crosses, a refined block's kernels on to r_b + look) instead of
 * taking prefixes of the assembled factors; the matrix may be assembled with
 * HM_DEFER_ACA.  info->crosses_full then counts the crosses computed. */
#define HM_AMVM_ACA_ON_DEMAND 1

typedef struct {
    int32_t iterations;    /* refinement steps taken */
    int32_t csp;           /* sparsity constant of the partition */
    double gamma;          /* gamma_k at exit */
    double bhat_norm;      /* ||A^_k x|| at exit */
    int64_t crosses_used;  /* sum over block-kernels of the crosses in A_k */
    int64_t crosses_full;  /* the same for the assembled ACA */
    int64_t marked_total;  /* blocks marked over all steps */
} hm_amvm_info;

int hm_amvm(hm_matrix* H, const double* x, double* y, const hm_amvm_params* p, hm_amvm_info* info,
            double* gamma_hist, double* gamma_rest_hist, int32_t hist_cap, int32_t* block_ranks, void* stream);

/* ---------------------------------------------------------------------------
 * Block-adaptive ACA for the single layer (Section 5, Algorithm 3 with only
 * the V blocks, branch (iii)), FP64: solves V_h t = b while the H-matrix
 * approximation A_k is refined block by block.
 *
 * A_k keeps, on each admissible block, the first r_b crosses of all seven ACA
 * sequences (A_0: r_b = r0; a shorter sequence is used whole); the look-ahead
 * A^_k has r_b + look; near blocks are exact in both.  Each step k:
 *   2. restarted GMRES(restart) on A_k t = b from the previous t (0 at
 *      first): a cycle ends early when its residual estimate reaches
 *      tau = alpha ||(A_k - A^_k) t|| at the cycle's start (tau = tol0 ||b||
 *      while t = 0); the solve ends when ||b - A_k t|| <= alpha ||(A_k - A^_k)
 *      t|| (Eq. (solvCond)) or below 1e-13 ||b|| (or after max_iter GMRES
 *      iterations in all);
 *   3. E_k^2 = sum_b ||(A_k - A^_k)_b t||^2; if E_k <= eps ||b|| stop;
 *      otherwise mark the fewest blocks with E_k(M_k) >= theta E_k (the
 *      largest parts first, ties by block index) and set A_{k+1} = A^_k on
 *      them (r_b += look).
 *   b, t     device, 3M doubles each, original dof order; t is overwritten
 *   info     optional: steps, GMRES iterations, final E, ||b - A_k t|| / ||b||,
 *            ||b||, crosses used by A_k and held by the assembled ACA, blocks
 *            marked in all
 *   hist     optional host array of hist_cap steps (E_k, ||b - A_k t||,
 *            ||(A_k - A^_k) t||, GMRES iterations, blocks marked)
 *   block_ranks  optional host array of nadm ints: r_b at exit
 * Needs the FP64 near field and either the assembled factors or
 * HM_BACA_ACA_ON_DEMAND (not after hm_compact); not for an evaluation
 * operator.  Allocates
 * (restart + 6) 3M doubles and about 24 sum|t| bytes of workspace through
 * the matrix's allocator for the call (and, at the first call, the product
 * tables and workspace it keeps with the matrix, so that calls on the same
 * matrix must not overlap); synchronises `stream`.
 * ------------------------------------------------------------------------- */
typedef struct {
    double theta;      /* Doerfler parameter in (0, 1) (0 = 0.8) */
    double alpha;      /* solve accuracy factor of Eq. (solvCond), > 0 (0 = 10) */
    double eps;        /* stop when E_k <= eps ||b|| (>= 0) */
    double tol0;       /* first solve: relative residual tol0 (0 = 0.1) */
    int32_t r0;        /* crosses per block and kernel in A_0 (0 = 8) */
    int32_t look;      /* look-ahead ACA steps, 1..32 (0 = 2) */
    int32_t restart;   /* GMRES restart length, 1..200 (0 = 50) */
    int32_t max_iter;  /* GMRES iterations in all (0 = 100000) */
    int32_t max_steps; /* refinement steps (0 = 1000) */
    int32_t flags;     /* HM_BACA_ACA_ON_DEMAND */
} hm_baca_params;

/* hm_baca_params.flags: run Algorithm 1 on demand -- every block-kernel to
 * r0 + look crosses, a refined block's kernels on to r_b + look, resumed from
 * their saved state -- instead of taking prefixes of the assembled factors
 * (the adaptive construction of A_k together with the solve); the matrix may
 * be assembled with HM_DEFER_ACA.  info->crosses_full then counts the
 * crosses computed. */
#define HM_BACA_ACA_ON_DEMAND 1

typedef struct {
    int32_t steps;             /* refinement steps taken */
    int32_t pad;
    int64_t gmres_iterations;  /* in all */
    double E;                  /* E_k at exit */
    double rel_residual;       /* ||b - A_k t|| / ||b|| at exit */
    double b_norm;
    int64_t crosses_used;      /* sum over block-kernels of the crosses in A_k */
    int64_t crosses_full;      /* the same for the assembled ACA */
    int64_t marked_total;      /* blocks marked over all steps */
} hm_baca_info;

typedef struct {
    double E;           /* E_k after the solve of step k */
    double residual;    /* ||b - A_k t_k|| */
    double lookahead;   /* ||(A_k - A^_k) t_k|| */
    int32_t iterations; /* GMRES iterations of the step */
    int32_t marked;     /* blocks refined after it */
} hm_baca_step;

int hm_baca(hm_matrix* H, const double* b, double* t, const hm_baca_params* p, hm_baca_info* info,
            hm_baca_step* hist, int32_t hist_cap, int32_t* block_ranks, void* stream);

/* Status of the asynchronous products of H: HM_ETIMEOUT if a bounded device
 * wait inside an earlier hm_matvec ran out (its result is then invalid; the
 * flag is cleared), HM_OK otherwise.  Synchronises the device. */
int hm_check(const hm_matrix* H);

/* Statistics of an assembled matrix. */
typedef struct {
    int64_t M, nadm, nnear, nleaves;
    int64_t near_pairs;         /* sum over near blocks of |t||s| */
    int64_t far_entries;        /* sum over admissible blocks and kernels of k(|t|+|s|) */
    int64_t far_u_entries;      /* sum of k|t| (U factors) */
    int64_t far_v_entries;      /* sum of k|s| (V factors) */
    int64_t factor_columns;     /* sum of k over admissible blocks and kernels */
    int64_t rank_sum[7];        /* per scalar kernel */
    int32_t rank_max[7];
    int32_t rank_cap_hits;      /* block-kernel pairs that hit kmax */
    int32_t csp;                /* sparsity constant: max blocks per row cluster */
    int64_t bytes_fp64;         /* far + near bytes read by one FP64 product */
    int64_t bytes_form[HM_NFORMS]; /* same for each form (0 if not packed) */
    double assemble_ms[3];      /* near-field quadrature, ACA, packing (device time) */
    int64_t far_entries_kern[7]; /* sum over admissible blocks of k(|t|+|s|), per scalar kernel */
    /* Assembly work, counted by the kernels at assembly (0 for a matrix
     * assembled before these counters or with HM_DEFER_ACA):
     *   near_points  near-field pairs on the 7-point rule over the whole
     *                triangle, 7-point-rule applications on subdivision
     *                leaves, and self pairs (3 x 32 Duffy points each)
     *   aca_entries  entries Algorithm 1 evaluated (every row it tried times
     *                |s|, every cross's column times |t|): V_Delta, V_kl */
    int64_t near_points[3];
    int64_t aca_entries[2];
    /* FP64 operations of the near-field quadrature and of ACA, from the
     * operations the formulas state (an FMA is 2, a square root or reciprocal
     * square root 1): per quadrature point of all seven kernels 31 (35 on the
     * self term, 46 on a subdivision leaf, whose rule also forms the points
     * and the leaf's area: 36 per leaf, and 63 per subdivision step); per ACA
     * entry 86 (V_Delta) or 114 (V_kl) with its 7-point rule; per ACA task of
     * rank k the residual, scaling and Frobenius updates
     * 2k(k-1)(|t|+|s|) + k(3|s|+2|t|). */
    double assembly_flops[2];
} hm_stats;

int hm_get_stats(const hm_matrix* H, hm_stats* st);

/* Measurement hook.  While enabled, hm_matvec records CUDA events around each
 * of its kernels on the launching stream (no synchronisation is added);
 * hm_profile_read synchronises on those events, returns the summed device
 * time per kernel in ms (ms[0] gather, ms[1] far-field forward, ms[2]
 * per-leaf product with the near field, ms[3] unused), the number of
 * profiled calls, and resets the sums.  At most 4096 calls are kept between
 * two reads (later ones are not profiled).  Not thread safe. */
int hm_profile_enable(hm_matrix* H, int32_t on);
int hm_profile_read(hm_matrix* H, double ms[4], int64_t* calls);

/* Export one admissible block's FP64 factors for inspection: blk indexes the
 * admissible list of hm_tree_export; kern 0..6 as above.  *rank receives k;
 * U (|t| x k) and V (|s| x k) are host arrays in column-major order, cluster
 * order within the block; pass NULL to query the rank only. */
int hm_export_factors(const hm_matrix* H, int64_t blk, int32_t kern, int32_t* rank, double* U,
                      double* V);

/* Export one near block's FP64 entries: host array of 6 x |t| x |s|, values
 * (V_11, V_12, V_13, V_22, V_23, V_33) row-major per value; V_Delta is their
 * trace. */
int hm_export_near(const hm_matrix* H, int64_t blk, double* out);

/* Release the FP64 data of H (the block-ordered FP64 factors and near field,
 * the FP64 product form and the pack sources) once the reduced forms it will
 * serve are packed: it keeps only what the packed forms read, typically a
 * third of the assembled footprint or less.  Afterwards hm_matvec in
 * HM_FP64, hm_solve, hm_pack and the exports return HM_EINVAL.  At least one
 * of HM_FP32 / HM_BF16 / HM_FP16 must be packed.  Synchronises the device. */
int hm_compact(hm_matrix* H);

/* Device bytes H currently holds (all its buffers and workspace). */
int hm_footprint(const hm_matrix* H, int64_t* bytes);

void hm_matrix_destroy(hm_matrix* H);

/* text of the calling thread's last error ("" if none) */
const char* hm_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* HMAT_H */
