"""Thin ctypes binding of the C ABI in ``include/hmat.h`` (argument marshalling
only: every step of the hot path runs in the CUDA library).

PyTorch supplies device memory (through the library's allocator hook, wired
to the caching allocator) and streams.  If the compiled library is missing
the import fails loudly: there is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_lib", "libhmat.so")

HM_OK, HM_EINVAL, HM_ENOMEM, HM_ENOTCONV, HM_ETIMEOUT, HM_EDEVICE, HM_ERANK, HM_EBUSY = \
    0, -1, -2, -3, -4, -5, -6, -7
HM_REQ_MATVEC, HM_REQ_SOLVE = 0, 1
FP64, FP32, BF16, FP16, I16 = 0, 1, 2, 3, 4
FORMS = {"fp64": FP64, "fp32": FP32, "bf16": BF16, "fp16": FP16, "i16": I16}
MAX_LEAF = 336  # HM_MAX_LEAF

# every symbol the header declares
SYMBOLS = (
    "hm_build_cluster_tree", "hm_tree_sizes", "hm_tree_export", "hm_tree_destroy",
    "hm_aca_assemble", "hm_set_material", "hm_pack", "hm_matvec", "hm_matvec_host",
    "hm_get_stats", "hm_export_factors", "hm_export_near", "hm_matrix_destroy",
    "hm_last_error", "hm_profile_enable", "hm_profile_read", "hm_matvec_noalloc", "hm_check",
    "hm_solve", "hm_batch_create", "hm_batch_layout", "hm_batch_matvec", "hm_batch_autotune",
    "hm_batch_set_schedule", "hm_batch_get_schedule", "hm_batch_check", "hm_batch_destroy",
    "hm_compact", "hm_footprint", "hm_server_create", "hm_server_footprint", "hm_server_run",
    "hm_server_destroy", "hm_amvm", "hm_build_point_tree", "hm_eval_points", "hm_baca",
    "hm_build_vertex_tree", "hm_double_layer_matvec",
)


class HMError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"hmat error {code}: {msg}")
        self.code = code


class _Params(ctypes.Structure):
    _fields_ = [("E", ctypes.c_double), ("nu", ctypes.c_double), ("aca_eps", ctypes.c_double),
                ("aca_eta_stop", ctypes.c_double), ("kmax", ctypes.c_int32),
                ("max_rhs", ctypes.c_int32), ("flags", ctypes.c_int32), ("pad", ctypes.c_int32)]


_ALLOC_T = ctypes.CFUNCTYPE(ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p, ctypes.c_void_p)
_FREE_T = ctypes.CFUNCTYPE(None, ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p, ctypes.c_void_p)


class _Allocator(ctypes.Structure):
    _fields_ = [("alloc", _ALLOC_T), ("free", _FREE_T), ("user", ctypes.c_void_p)]


class _SolveParams(ctypes.Structure):
    _fields_ = [("tol", ctypes.c_double), ("inner_tol", ctypes.c_double),
                ("inner_form", ctypes.c_int32), ("restart", ctypes.c_int32),
                ("max_inner", ctypes.c_int32), ("max_refine", ctypes.c_int32),
                ("use_initial_guess", ctypes.c_int32), ("residual_form", ctypes.c_int32)]


class _SolveInfo(ctypes.Structure):
    _fields_ = [("iterations", ctypes.c_int32), ("restarts", ctypes.c_int32),
                ("refinements", ctypes.c_int32), ("pad", ctypes.c_int32),
                ("rel_residual", ctypes.c_double)]


class _AmvmParams(ctypes.Structure):
    _fields_ = [("theta", ctypes.c_double), ("eps", ctypes.c_double), ("r0", ctypes.c_int32),
                ("look", ctypes.c_int32), ("max_iter", ctypes.c_int32), ("flags", ctypes.c_int32)]


class _AmvmInfo(ctypes.Structure):
    _fields_ = [("iterations", ctypes.c_int32), ("csp", ctypes.c_int32), ("gamma", ctypes.c_double),
                ("bhat_norm", ctypes.c_double), ("crosses_used", ctypes.c_int64),
                ("crosses_full", ctypes.c_int64), ("marked_total", ctypes.c_int64)]


class _BacaParams(ctypes.Structure):
    _fields_ = [("theta", ctypes.c_double), ("alpha", ctypes.c_double), ("eps", ctypes.c_double),
                ("tol0", ctypes.c_double), ("r0", ctypes.c_int32), ("look", ctypes.c_int32),
                ("restart", ctypes.c_int32), ("max_iter", ctypes.c_int32), ("max_steps", ctypes.c_int32),
                ("flags", ctypes.c_int32)]


class _BacaInfo(ctypes.Structure):
    _fields_ = [("steps", ctypes.c_int32), ("pad", ctypes.c_int32), ("gmres_iterations", ctypes.c_int64),
                ("E", ctypes.c_double), ("rel_residual", ctypes.c_double), ("b_norm", ctypes.c_double),
                ("crosses_used", ctypes.c_int64), ("crosses_full", ctypes.c_int64),
                ("marked_total", ctypes.c_int64)]


class _BacaStep(ctypes.Structure):
    _fields_ = [("E", ctypes.c_double), ("residual", ctypes.c_double), ("lookahead", ctypes.c_double),
                ("iterations", ctypes.c_int32), ("marked", ctypes.c_int32)]


class _Schedule(ctypes.Structure):
    _fields_ = [("leaf_ctas_per_sm", ctypes.c_int32), ("work_order", ctypes.c_int32),
                ("fork_forward", ctypes.c_int32), ("pad", ctypes.c_int32)]


class _ServerParams(ctypes.Structure):
    _fields_ = [("slots", ctypes.c_int32), ("queue_cap", ctypes.c_int32),
                ("budget_bytes", ctypes.c_int64), ("matvec_form", ctypes.c_int32),
                ("inner_form", ctypes.c_int32), ("residual_form", ctypes.c_int32),
                ("restart", ctypes.c_int32), ("inner_tol", ctypes.c_double),
                ("max_inner", ctypes.c_int32), ("solve_slots", ctypes.c_int32)]


class _Request(ctypes.Structure):
    _fields_ = [("arrival_s", ctypes.c_double), ("mesh", ctypes.c_int32), ("kind", ctypes.c_int32),
                ("nrhs", ctypes.c_int32), ("seed", ctypes.c_int32), ("tol", ctypes.c_double),
                ("x_host", ctypes.c_void_p), ("y_host", ctypes.c_void_p)]


class _Result(ctypes.Structure):
    _fields_ = [("status", ctypes.c_int32), ("iterations", ctypes.c_int32),
                ("arrival_s", ctypes.c_double), ("start_s", ctypes.c_double),
                ("done_s", ctypes.c_double), ("rel_residual", ctypes.c_double)]


class _Stats(ctypes.Structure):
    _fields_ = [("M", ctypes.c_int64), ("nadm", ctypes.c_int64), ("nnear", ctypes.c_int64),
                ("nleaves", ctypes.c_int64), ("near_pairs", ctypes.c_int64),
                ("far_entries", ctypes.c_int64), ("far_u_entries", ctypes.c_int64),
                ("far_v_entries", ctypes.c_int64), ("factor_columns", ctypes.c_int64),
                ("rank_sum", ctypes.c_int64 * 7),
                ("rank_max", ctypes.c_int32 * 7), ("rank_cap_hits", ctypes.c_int32),
                ("csp", ctypes.c_int32), ("bytes_fp64", ctypes.c_int64),
                ("bytes_form", ctypes.c_int64 * 5), ("assemble_ms", ctypes.c_double * 3),
                ("far_entries_kern", ctypes.c_int64 * 7), ("near_points", ctypes.c_int64 * 3),
                ("aca_entries", ctypes.c_int64 * 2), ("assembly_flops", ctypes.c_double * 2)]


_lib = None


def load():
    """Load the in-tree library (build it with ``__graft_entry__.build()``)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"CUDA library not built: {LIB_PATH} is missing "
                          "(run __graft_entry__.build()); there is no CPU fallback")
    lib = ctypes.CDLL(LIB_PATH)
    P, I64, I32, D = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int32, ctypes.c_double
    sig = {
        "hm_build_cluster_tree": (ctypes.c_int, [P, I64, P, I64, I32, D, ctypes.POINTER(P)]),
        "hm_tree_sizes": (ctypes.c_int, [P, P]),
        "hm_tree_export": (ctypes.c_int, [P, P, P, P, P]),
        "hm_tree_destroy": (None, [P]),
        "hm_build_point_tree": (ctypes.c_int, [P, P, I64, I32, ctypes.POINTER(P)]),
        "hm_build_vertex_tree": (ctypes.c_int, [P, I32, ctypes.POINTER(P)]),
        "hm_eval_points": (ctypes.c_int, [P, P, P, I32, I32, P]),
        "hm_double_layer_matvec": (ctypes.c_int, [P, P, P, P, I32, I32, P]),
        "hm_aca_assemble": (ctypes.c_int, [P, ctypes.POINTER(_Params), ctypes.POINTER(_Allocator),
                                           P, ctypes.POINTER(P)]),
        "hm_set_material": (ctypes.c_int, [P, D, D]),
        "hm_pack": (ctypes.c_int, [P, I32, P]),
        "hm_matvec": (ctypes.c_int, [P, P, P, I32, I64, I32, P]),
        "hm_matvec_host": (ctypes.c_int, [P, P, P, I32, I64, I32, P]),
        "hm_matvec_noalloc": (ctypes.c_int, [P, P, P, I32, I64, I32, P]),
        "hm_check": (ctypes.c_int, [P]),
        "hm_solve": (ctypes.c_int, [P, P, P, ctypes.POINTER(_SolveParams),
                                    ctypes.POINTER(_SolveInfo), P]),
        "hm_get_stats": (ctypes.c_int, [P, ctypes.POINTER(_Stats)]),
        "hm_amvm": (ctypes.c_int, [P, P, P, ctypes.POINTER(_AmvmParams), ctypes.POINTER(_AmvmInfo), P, P,
                                   I32, P, P]),
        "hm_baca": (ctypes.c_int, [P, P, P, ctypes.POINTER(_BacaParams), ctypes.POINTER(_BacaInfo), P, I32, P,
                                   P]),
        "hm_export_factors": (ctypes.c_int, [P, I64, I32, ctypes.POINTER(I32), P, P]),
        "hm_export_near": (ctypes.c_int, [P, I64, P]),
        "hm_matrix_destroy": (None, [P]),
        "hm_last_error": (ctypes.c_char_p, []),
        "hm_profile_enable": (ctypes.c_int, [P, I32]),
        "hm_profile_read": (ctypes.c_int, [P, P, ctypes.POINTER(I64)]),
        "hm_batch_create": (ctypes.c_int, [P, I32, I32, I32, ctypes.POINTER(P)]),
        "hm_batch_layout": (ctypes.c_int, [P, P, P]),
        "hm_batch_matvec": (ctypes.c_int, [P, P, P, I32, I64, I32, P]),
        "hm_batch_autotune": (ctypes.c_int, [P, I32, I32, ctypes.POINTER(_Schedule),
                                             ctypes.POINTER(D), P]),
        "hm_batch_set_schedule": (ctypes.c_int, [P, ctypes.POINTER(_Schedule)]),
        "hm_batch_get_schedule": (ctypes.c_int, [P, ctypes.POINTER(_Schedule)]),
        "hm_batch_check": (ctypes.c_int, [P]),
        "hm_batch_destroy": (None, [P]),
        "hm_compact": (ctypes.c_int, [P]),
        "hm_footprint": (ctypes.c_int, [P, ctypes.POINTER(I64)]),
        "hm_server_create": (ctypes.c_int, [P, I32, ctypes.POINTER(_ServerParams), ctypes.POINTER(P)]),
        "hm_server_footprint": (ctypes.c_int, [P, ctypes.POINTER(_Request), ctypes.POINTER(I64)]),
        "hm_server_run": (ctypes.c_int, [P, P, I32, I32, P]),
        "hm_server_destroy": (None, [P]),
    }
    for name, (res, args) in sig.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    _lib = lib
    return lib


def _check(rc: int, ok=(HM_OK,)):
    if rc not in ok:
        raise HMError(rc, load().hm_last_error().decode())
    return rc


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def _stream_handle(stream):
    if stream is None:
        import torch
        return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    if isinstance(stream, int):
        return ctypes.c_void_p(stream)
    return ctypes.c_void_p(stream.cuda_stream)


class ClusterTree:
    """Cluster tree and block partition (host), ``hm_build_cluster_tree``."""

    def __init__(self, verts, tris, leaf: int, eta: float):
        lib = load()
        self.verts = np.ascontiguousarray(verts, dtype=np.float64)
        self.tris = np.ascontiguousarray(tris, dtype=np.int32)
        h = ctypes.c_void_p()
        _check(lib.hm_build_cluster_tree(_ptr(self.verts), self.verts.shape[0], _ptr(self.tris),
                                         self.tris.shape[0], int(leaf), float(eta),
                                         ctypes.byref(h)))
        self._h = h
        c = np.zeros(6, dtype=np.int64)
        _check(lib.hm_tree_sizes(self._h, _ptr(c)))
        self.M, self.nnodes, self.nadm, self.nnear, self.nleaves, self.depth = map(int, c)
        self.leaf, self.eta = int(leaf), float(eta)

    def export(self):
        perm = np.zeros(self.M, dtype=np.int64)
        nodes = np.zeros((self.nnodes, 5), dtype=np.int64)
        adm = np.zeros((max(self.nadm, 1), 2), dtype=np.int64)
        near = np.zeros((max(self.nnear, 1), 2), dtype=np.int64)
        _check(load().hm_tree_export(self._h, _ptr(perm), _ptr(nodes), _ptr(adm), _ptr(near)))
        return perm, nodes, adm[:self.nadm], near[:self.nnear]

    def __del__(self):
        h = getattr(self, "_h", None)
        if h and _lib is not None:
            _lib.hm_tree_destroy(h)
            self._h = None


def build_cluster_tree(verts, tris, leaf: int, eta: float) -> ClusterTree:
    return ClusterTree(verts, tris, leaf, eta)


class PointTree(ClusterTree):
    """Rows of the evaluation operator ~V_h (Section 5, Eq. (vector_eq)):
    the cluster tree of points of the domain and the partition (point tree) x
    (triangle tree of ``surface``), ``hm_build_point_tree``.  ``M`` counts
    the points, ``M_src`` the triangles."""

    def __init__(self, surface: ClusterTree, points, leaf: int):
        lib = load()
        self.points = np.ascontiguousarray(points, dtype=np.float64).reshape(-1, 3)
        h = ctypes.c_void_p()
        _check(lib.hm_build_point_tree(surface._h, _ptr(self.points), self.points.shape[0], int(leaf),
                                       ctypes.byref(h)))
        self._h = h
        c = np.zeros(6, dtype=np.int64)
        _check(lib.hm_tree_sizes(self._h, _ptr(c)))
        self.M, self.nnodes, self.nadm, self.nnear, self.nleaves, self.depth = map(int, c)
        self.leaf, self.eta = int(leaf), surface.eta
        self.M_src = surface.M


def build_point_tree(surface: ClusterTree, points, leaf: int) -> PointTree:
    return PointTree(surface, points, leaf)


class VertexTree(ClusterTree):
    """Columns of the double layer's K_Delta (Eq. (Kh)): the cluster tree of
    the mesh vertices with star boxes and the partition (triangle tree of
    ``surface``) x (vertex tree), ``hm_build_vertex_tree``.  ``M`` counts the
    vertices, ``M_src`` the triangles.  ``HMatrix`` on it assembles K_Delta."""

    def __init__(self, surface: ClusterTree, leaf: int):
        lib = load()
        h = ctypes.c_void_p()
        _check(lib.hm_build_vertex_tree(surface._h, int(leaf), ctypes.byref(h)))
        self._h = h
        c = np.zeros(6, dtype=np.int64)
        _check(lib.hm_tree_sizes(self._h, _ptr(c)))
        self.M, self.nnodes, self.nadm, self.nnear, self.nleaves, self.depth = map(int, c)
        self.leaf, self.eta = int(leaf), surface.eta
        self.M_src = surface.M


def build_vertex_tree(surface: ClusterTree, leaf: int) -> VertexTree:
    return VertexTree(surface, leaf)


def _torch_allocator(device: int):
    import torch

    def _a(nbytes, stream, user):
        try:
            return torch.cuda.caching_allocator_alloc(int(nbytes), device, int(stream or 0))
        except Exception:  # reported to the library as a NULL allocation
            return None

    def _f(ptr, nbytes, stream, user):
        if ptr:
            torch.cuda.caching_allocator_delete(int(ptr))

    fa, ff = _ALLOC_T(_a), _FREE_T(_f)
    return _Allocator(fa, ff, None), (fa, ff)


@dataclass
class Stats:
    M: int
    nadm: int
    nnear: int
    nleaves: int
    near_pairs: int
    far_entries: int
    far_u_entries: int
    far_v_entries: int
    factor_columns: int
    rank_sum: list
    rank_max: list
    rank_cap_hits: int
    csp: int
    bytes_fp64: int
    bytes_form: list
    assemble_ms: list
    far_entries_kern: list
    near_points: list
    aca_entries: list
    assembly_flops: list


class HMatrix:
    """Assembled H-matrix resident on the device (``hm_aca_assemble``)."""

    def __init__(self, tree: ClusterTree, E: float, nu: float, aca_eps: float,
                 aca_eta_stop: float = 0.8, kmax: int = 128, max_rhs: int = 32, stream=None,
                 torch_memory: bool = True, defer_fp64: bool = False, defer_aca: bool = False):
        import torch
        lib = load()
        # columns are triangles (the vertices for the double layer's K_Delta);
        # rows are the triangles (the points of an evaluation operator)
        self.dl = isinstance(tree, VertexTree)
        self.rect = isinstance(tree, (PointTree, VertexTree))
        if self.dl:
            self.M, self.Mr = tree.M, tree.M_src
        else:
            self.M = tree.M_src if self.rect else tree.M
            self.Mr = tree.M
        self.device = torch.cuda.current_device()
        prm = _Params(float(E), float(nu), float(aca_eps), float(aca_eta_stop), int(kmax),
                      int(max_rhs), (1 if defer_fp64 else 0) | (2 if defer_aca else 0), 0)
        self._alloc_keep = None
        ap = None
        if torch_memory:
            al, keep = _torch_allocator(self.device)
            self._alloc_struct = al
            self._alloc_keep = keep
            ap = ctypes.byref(al)
        h = ctypes.c_void_p()
        rc = lib.hm_aca_assemble(tree._h, ctypes.byref(prm), ap, _stream_handle(stream),
                                 ctypes.byref(h))
        _check(rc, ok=(HM_OK, HM_ERANK))
        self.rank_cap_hit = rc == HM_ERANK
        self._h = h
        self.max_rhs = int(max_rhs) if max_rhs else 32

    def __del__(self):
        h = getattr(self, "_h", None)
        if h and _lib is not None:
            _lib.hm_matrix_destroy(h)
            self._h = None

    def set_material(self, E: float, nu: float):
        _check(load().hm_set_material(self._h, float(E), float(nu)))

    def pack(self, form, stream=None):
        f = FORMS[form] if isinstance(form, str) else int(form)
        _check(load().hm_pack(self._h, f, _stream_handle(stream)))

    def stats(self) -> Stats:
        st = _Stats()
        _check(load().hm_get_stats(self._h, ctypes.byref(st)))
        return Stats(st.M, st.nadm, st.nnear, st.nleaves, st.near_pairs, st.far_entries,
                     st.far_u_entries, st.far_v_entries, st.factor_columns, list(st.rank_sum), list(st.rank_max), st.rank_cap_hits, st.csp,
                     st.bytes_fp64, list(st.bytes_form), list(st.assemble_ms), list(st.far_entries_kern),
                     list(st.near_points), list(st.aca_entries), list(st.assembly_flops))

    def check(self):
        """Raise if a bounded device wait in an earlier product ran out."""
        _check(load().hm_check(self._h))

    def compact(self):
        """``hm_compact``: release the FP64 data, keep the packed reduced forms."""
        _check(load().hm_compact(self._h))

    def footprint(self) -> int:
        """Device bytes held by the matrix (``hm_footprint``)."""
        b = ctypes.c_int64(0)
        _check(load().hm_footprint(self._h, ctypes.byref(b)))
        return int(b.value)

    def profile(self, on: bool):
        _check(load().hm_profile_enable(self._h, 1 if on else 0))

    def profile_read(self):
        """(ms per kernel [gather, far forward, leaf product, -], calls)."""
        ms = np.zeros(4)
        n = ctypes.c_int64(0)
        _check(load().hm_profile_read(self._h, _ptr(ms), ctypes.byref(n)))
        return ms, int(n.value)

    def export_factors(self, blk: int, kern: int):
        lib = load()
        k = ctypes.c_int32(0)
        _check(lib.hm_export_factors(self._h, int(blk), int(kern), ctypes.byref(k), None, None))
        return int(k.value)

    def factors(self, blk: int, kern: int, m: int, n: int):
        lib = load()
        k = self.export_factors(blk, kern)
        U = np.zeros((max(k, 1), m))
        V = np.zeros((max(k, 1), n))
        kk = ctypes.c_int32(0)
        _check(lib.hm_export_factors(self._h, int(blk), int(kern), ctypes.byref(kk), _ptr(U),
                                     _ptr(V)))
        return U[:k].T.copy(), V[:k].T.copy()

    def near_block(self, blk: int, m: int, n: int):
        out = np.zeros((6, m, n))
        _check(load().hm_export_near(self._h, int(blk), _ptr(out)))
        return out


def aca_assemble(tree: ClusterTree, E: float, nu: float, aca_eps: float, **kw) -> HMatrix:
    return HMatrix(tree, E, nu, aca_eps, **kw)


def hmatvec(H: HMatrix, x, y, form="fp64", stream=None):
    """y = V_h x on the device.  x, y: CUDA float64 tensors of shape (3M,) or
    (nrhs, 3M) (row stride = ld)."""
    import torch
    f = FORMS[form] if isinstance(form, str) else int(form)
    if not (x.is_cuda and y.is_cuda and x.dtype == torch.float64 and y.dtype == torch.float64):
        raise TypeError("hmatvec: x and y must be CUDA float64 tensors")
    nrhs = 1 if x.dim() == 1 else x.shape[0]
    # the stride of a single row is irrelevant (and may be anything)
    ld = x.shape[-1] if nrhs == 1 else x.stride(0)
    if (y.dim() == 1 and nrhs != 1) or (y.dim() == 2 and (y.shape[0] != nrhs or
                                                          (nrhs > 1 and y.stride(0) != ld))):
        raise ValueError("hmatvec: y must have the shape and row stride of x")
    if x.shape[-1] != 3 * H.M or x.stride(-1) != 1 or y.stride(-1) != 1:
        raise ValueError("hmatvec: rows must be contiguous of length 3M")
    _check(load().hm_matvec(H._h, ctypes.c_void_p(x.data_ptr()), ctypes.c_void_p(y.data_ptr()),
                            nrhs, ld, f, _stream_handle(stream)))
    return y


def solve(H: HMatrix, g, t, tol: float = 1e-8, inner_form="fp16", inner_tol: float = 0.0,
          restart: int = 50, max_inner: int = 0, max_refine: int = 0, initial_guess=False,
          stream=None, raise_on_fail: bool = True, residual_form="fp64"):
    """``hm_solve``: V_h t = g with GMRES on ``inner_form`` and FP64-residual
    iterative refinement.  g, t: CUDA float64 tensors of 3M.  Returns a dict
    with iterations, restarts, refinements and the relative FP64 residual."""
    import torch
    if not (g.is_cuda and t.is_cuda and g.dtype == torch.float64 and t.dtype == torch.float64):
        raise TypeError("solve: g and t must be CUDA float64 tensors")
    if g.numel() != 3 * H.M or t.numel() != 3 * H.M or not g.is_contiguous() or not t.is_contiguous():
        raise ValueError("solve: g and t must be contiguous vectors of 3M")
    f = FORMS[inner_form] if isinstance(inner_form, str) else int(inner_form)
    fr = FORMS[residual_form] if isinstance(residual_form, str) else int(residual_form)
    p = _SolveParams(float(tol), float(inner_tol), f, int(restart), int(max_inner), int(max_refine),
                     1 if initial_guess else 0, fr)
    info = _SolveInfo()
    rc = load().hm_solve(H._h, ctypes.c_void_p(g.data_ptr()), ctypes.c_void_p(t.data_ptr()),
                         ctypes.byref(p), ctypes.byref(info), _stream_handle(stream))
    out = dict(iterations=info.iterations, restarts=info.restarts, refinements=info.refinements,
               rel_residual=info.rel_residual, converged=rc == HM_OK)
    if raise_on_fail:
        _check(rc)
    elif rc not in (HM_OK, HM_ENOTCONV):
        _check(rc)
    return out


def amvm(H: HMatrix, x, y, theta: float = 0.7, eps: float = 1e-6, r0: int = 2, look: int = 2,
         max_iter: int = 0, on_demand: bool = False, stream=None):
    """``hm_amvm``: adaptive matrix-vector multiplication (Algorithm 2), FP64.
    x, y: CUDA float64 vectors of 3M (original dof order); y = A_k x at exit.
    Returns a dict with the iterations, the estimator history (gamma per
    iteration, gamma_rest per refinement), the final block ranks and the
    crosses used against the assembled ACA (``on_demand``: Algorithm 1 run on
    demand, HM_AMVM_ACA_ON_DEMAND; crosses_full then counts the crosses
    computed)."""
    import torch
    if not (x.is_cuda and y.is_cuda and x.dtype == torch.float64 and y.dtype == torch.float64):
        raise TypeError("amvm: x and y must be CUDA float64 tensors")
    if x.numel() != 3 * H.M or y.numel() != 3 * H.Mr or not x.is_contiguous() or not y.is_contiguous():
        raise ValueError("amvm: x must be a contiguous vector of 3M and y of 3 rows (3M, or 3 points)")
    p = _AmvmParams(float(theta), float(eps), int(r0), int(look), int(max_iter), 1 if on_demand else 0)
    info = _AmvmInfo()
    cap = 4096
    g = np.zeros(cap)
    gr = np.zeros(cap)
    ranks = np.zeros(max(H.stats().nadm, 1), dtype=np.int32)
    _check(load().hm_amvm(H._h, ctypes.c_void_p(x.data_ptr()), ctypes.c_void_p(y.data_ptr()),
                          ctypes.byref(p), ctypes.byref(info), _ptr(g), _ptr(gr), cap, _ptr(ranks),
                          _stream_handle(stream)))
    k = info.iterations
    return dict(iterations=k, csp=info.csp, gamma=list(g[:min(k + 1, cap)]),
                gamma_rest=list(gr[:min(k, cap)]), bhat_norm=info.bhat_norm,
                crosses_used=int(info.crosses_used), crosses_full=int(info.crosses_full),
                marked_total=int(info.marked_total), block_ranks=ranks[:H.stats().nadm].copy())


def double_layer_matvec(V: HMatrix, K: HMatrix, u, y, form="fp64", stream=None):
    """``hm_double_layer_matvec``: y = K_h u, the double layer of Eq. (Kh) in
    collocation form.  V: the single layer of the mesh (``form`` packed), K:
    K_Delta (an ``HMatrix`` of a ``VertexTree`` of the same triangle tree).
    u: CUDA float64 (3 nv,) or (nrhs, 3 nv) in the original vertex order; y:
    (3M,) or (nrhs, 3M); both contiguous."""
    import torch
    f = FORMS[form] if isinstance(form, str) else int(form)
    if not (u.is_cuda and y.is_cuda and u.dtype == torch.float64 and y.dtype == torch.float64):
        raise TypeError("double_layer_matvec: u and y must be CUDA float64 tensors")
    nrhs = 1 if u.dim() == 1 else u.shape[0]
    if (u.shape[-1] != 3 * K.M or y.shape[-1] != 3 * V.M or (u.dim() == 2) != (y.dim() == 2)
            or (u.dim() == 2 and y.shape[0] != nrhs) or not u.is_contiguous() or not y.is_contiguous()):
        raise ValueError("double_layer_matvec: u must be contiguous rows of 3 nv, y rows of 3M")
    _check(load().hm_double_layer_matvec(V._h, K._h, ctypes.c_void_p(u.data_ptr()), ctypes.c_void_p(y.data_ptr()),
                                         nrhs, f, _stream_handle(stream)))
    return y


def eval_points(H: HMatrix, t, u, form="fp64", stream=None):
    """``hm_eval_points``: u = ~V_h t, the displacement at the points of an
    evaluation operator (an ``HMatrix`` assembled from a ``PointTree``) for
    densities t.  t: CUDA float64 (3M,) or (nrhs, 3M); u: (3 npts,) or
    (nrhs, 3 npts); both contiguous.  ``form``: "fp64" (exact) or "fp32"
    (after ``H.pack("fp32")``)."""
    f = FORMS[form] if isinstance(form, str) else int(form)
    import torch
    if not (t.is_cuda and u.is_cuda and t.dtype == torch.float64 and u.dtype == torch.float64):
        raise TypeError("eval_points: t and u must be CUDA float64 tensors")
    nrhs = 1 if t.dim() == 1 else t.shape[0]
    if (t.shape[-1] != 3 * H.M or u.shape[-1] != 3 * H.Mr or (u.dim() == 2) != (t.dim() == 2)
            or (t.dim() == 2 and u.shape[0] != nrhs) or not t.is_contiguous() or not u.is_contiguous()):
        raise ValueError("eval_points: t must be contiguous rows of 3M, u rows of 3 npts")
    _check(load().hm_eval_points(H._h, ctypes.c_void_p(t.data_ptr()), ctypes.c_void_p(u.data_ptr()), nrhs, f,
                                 _stream_handle(stream)))
    return u


def baca(H: HMatrix, b, t, theta: float = 0.8, alpha: float = 10.0, eps: float = 1e-4, tol0: float = 0.1,
         r0: int = 8, look: int = 2, restart: int = 50, max_iter: int = 0, max_steps: int = 0,
         on_demand: bool = False, stream=None):
    """``hm_baca``: solve V_h t = b with block-adaptive ACA (Algorithm 3,
    single layer), FP64.  b, t: contiguous CUDA float64 vectors of 3M.
    Returns a dict with steps, GMRES iterations, the final estimator and
    residual, the crosses used against the assembled ACA (``on_demand``:
    Algorithm 1 run on demand, HM_BACA_ACA_ON_DEMAND; crosses_full then counts
    the crosses computed), per-step history (E, residual, lookahead,
    iterations, marked) and the final block ranks."""
    import torch
    if not (b.is_cuda and t.is_cuda and b.dtype == torch.float64 and t.dtype == torch.float64):
        raise TypeError("baca: b and t must be CUDA float64 tensors")
    if b.numel() != 3 * H.M or t.numel() != 3 * H.M or not b.is_contiguous() or not t.is_contiguous():
        raise ValueError("baca: b and t must be contiguous vectors of 3M")
    p = _BacaParams(float(theta), float(alpha), float(eps), float(tol0), int(r0), int(look), int(restart),
                    int(max_iter), int(max_steps), 1 if on_demand else 0)
    info = _BacaInfo()
    cap = 4096
    hist = (_BacaStep * cap)()
    ranks = np.zeros(max(H.stats().nadm, 1), dtype=np.int32)
    _check(load().hm_baca(H._h, ctypes.c_void_p(b.data_ptr()), ctypes.c_void_p(t.data_ptr()), ctypes.byref(p),
                          ctypes.byref(info), ctypes.cast(hist, ctypes.c_void_p), cap, _ptr(ranks),
                          _stream_handle(stream)))
    n = min(info.steps + 1, cap)
    steps = [dict(E=hist[i].E, residual=hist[i].residual, lookahead=hist[i].lookahead,
                  iterations=hist[i].iterations, marked=hist[i].marked) for i in range(n)]
    return dict(steps=info.steps, gmres_iterations=int(info.gmres_iterations), E=info.E,
                rel_residual=info.rel_residual, b_norm=info.b_norm, crosses_used=int(info.crosses_used),
                crosses_full=int(info.crosses_full), marked_total=int(info.marked_total), history=steps,
                block_ranks=ranks[:H.stats().nadm].copy())


def hmatvec_noalloc(H: HMatrix, x, y, form="fp64", stream=None):
    """``hm_matvec_noalloc``: the product of ``hmatvec`` with its workspace
    taken from the library's fixed 32 MiB static device array, for callers
    that cannot allocate device memory; it allocates nothing.  Calls must not
    overlap on the device (they share that array)."""
    import torch
    f = FORMS[form] if isinstance(form, str) else int(form)
    if not (x.is_cuda and y.is_cuda and x.dtype == torch.float64 and y.dtype == torch.float64):
        raise TypeError("hmatvec_noalloc: x and y must be CUDA float64 tensors")
    nrhs = 1 if x.dim() == 1 else x.shape[0]
    ld = x.shape[-1] if nrhs == 1 else x.stride(0)
    if y.shape != x.shape or (nrhs > 1 and y.stride(0) != ld):
        raise ValueError("hmatvec_noalloc: y must have the shape and row stride of x")
    _check(load().hm_matvec_noalloc(H._h, ctypes.c_void_p(x.data_ptr()),
                                    ctypes.c_void_p(y.data_ptr()), nrhs, ld, f,
                                    _stream_handle(stream)))
    return y


def hmatvec_host(H: HMatrix, x: np.ndarray, y: np.ndarray, form="fp64", stream=None):
    """Same product with host arrays (copies inside the call; synchronous)."""
    f = FORMS[form] if isinstance(form, str) else int(form)
    if x.dtype != np.float64 or y.dtype != np.float64:
        raise TypeError("hmatvec_host: float64 arrays required")
    nrhs = 1 if x.ndim == 1 else x.shape[0]
    ld = x.shape[-1] if nrhs == 1 else x.strides[0] // 8
    if nrhs > 1 and (y.shape != x.shape or y.strides != x.strides):
        raise ValueError("hmatvec_host: y must have the shape and strides of x")
    if x.strides[-1] != 8 or y.strides[-1] != 8:
        raise ValueError("hmatvec_host: rows must be contiguous")
    _check(load().hm_matvec_host(H._h, _ptr(x), _ptr(y), nrhs, ld, f, _stream_handle(stream)))
    return y


class Batch:
    """``hm_batch``: one product over several resident matrices (each with
    ``form`` packed).  Rows of x and y hold every member's dofs side by side
    at ``offsets[m] .. offsets[m+1]``.  The members must stay alive and
    unchanged while the batch exists."""

    def __init__(self, mats, form="fp16", max_rhs: int = 16):
        lib = load()
        self.mats = list(mats)  # keeps the members alive
        self.form = FORMS[form] if isinstance(form, str) else int(form)
        arr = (ctypes.c_void_p * len(self.mats))(*[m._h.value for m in self.mats])
        h = ctypes.c_void_p()
        _check(lib.hm_batch_create(arr, len(self.mats), self.form, int(max_rhs), ctypes.byref(h)))
        self._h = h
        self.max_rhs = int(max_rhs)
        off = np.zeros(len(self.mats) + 1, dtype=np.int64)
        sz = np.zeros(4, dtype=np.int64)
        _check(lib.hm_batch_layout(self._h, _ptr(off), _ptr(sz)))
        self.offsets = off
        self.ndof = int(sz[1])
        self.ngroups, self.nleaves = int(sz[2]), int(sz[3])

    def __del__(self):
        h = getattr(self, "_h", None)
        if h and _lib is not None:
            _lib.hm_batch_destroy(h)
            self._h = None

    def matvec(self, x, y, graph: bool = False, stream=None):
        """y = V_h x for every member; x, y CUDA float64 tensors (ndof,) or
        (nrhs, ndof) with the same row stride."""
        import torch
        if not (x.is_cuda and y.is_cuda and x.dtype == torch.float64 and y.dtype == torch.float64):
            raise TypeError("Batch.matvec: x and y must be CUDA float64 tensors")
        nrhs = 1 if x.dim() == 1 else x.shape[0]
        ld = x.shape[-1] if nrhs == 1 else x.stride(0)
        if y.shape != x.shape or (nrhs > 1 and y.stride(0) != ld):
            raise ValueError("Batch.matvec: y must have the shape and row stride of x")
        if x.shape[-1] < self.ndof or x.stride(-1) != 1 or y.stride(-1) != 1:
            raise ValueError("Batch.matvec: rows must be contiguous of length >= ndof")
        _check(load().hm_batch_matvec(self._h, ctypes.c_void_p(x.data_ptr()),
                                      ctypes.c_void_p(y.data_ptr()), nrhs, ld, 1 if graph else 0,
                                      _stream_handle(stream)))
        return y

    def autotune(self, nrhs: int = 1, reps: int = 3, stream=None):
        """Time every schedule, keep the fastest; returns (schedule dict, ms)."""
        sc = _Schedule()
        ms = ctypes.c_double(0.0)
        _check(load().hm_batch_autotune(self._h, int(nrhs), int(reps), ctypes.byref(sc),
                                        ctypes.byref(ms), _stream_handle(stream)))
        return self._sched_dict(sc), float(ms.value)

    @staticmethod
    def _sched_dict(sc):
        return dict(leaf_ctas_per_sm=sc.leaf_ctas_per_sm, work_order=sc.work_order,
                    fork_forward=sc.fork_forward)

    def schedule(self):
        sc = _Schedule()
        _check(load().hm_batch_get_schedule(self._h, ctypes.byref(sc)))
        return self._sched_dict(sc)

    def set_schedule(self, leaf_ctas_per_sm=0, work_order=0, fork_forward=0):
        sc = _Schedule(int(leaf_ctas_per_sm), int(work_order), int(fork_forward), 0)
        _check(load().hm_batch_set_schedule(self._h, ctypes.byref(sc)))

    def check(self):
        _check(load().hm_batch_check(self._h))


class Server:
    """``hm_server``: a request loop over resident matrices (each with the
    forms it serves packed).  ``run`` replays a list of requests (dicts with
    arrival_s, mesh, kind 'matvec' / 'solve', nrhs, seed, tol and optional
    host arrays x / y) and returns one result dict per request."""

    def __init__(self, mats, slots=8, queue_cap=1024, budget_bytes=8 << 30, matvec_form="fp16",
                 inner_form="fp16", residual_form="fp32", restart=30, inner_tol=1e-3, max_inner=0,
                 solve_slots=0):
        lib = load()
        self.mats = list(mats)
        f = lambda v: FORMS[v] if isinstance(v, str) else int(v)
        p = _ServerParams(int(slots), int(queue_cap), int(budget_bytes), f(matvec_form), f(inner_form),
                          f(residual_form), int(restart), float(inner_tol), int(max_inner), int(solve_slots))
        arr = (ctypes.c_void_p * len(self.mats))(*[m._h.value for m in self.mats])
        h = ctypes.c_void_p()
        _check(lib.hm_server_create(arr, len(self.mats), ctypes.byref(p), ctypes.byref(h)))
        self._h = h

    def __del__(self):
        h = getattr(self, "_h", None)
        if h and _lib is not None:
            _lib.hm_server_destroy(h)
            self._h = None

    @staticmethod
    def _request(r):
        x = r.get("x")
        y = r.get("y")
        for a in (x, y):
            if a is not None and (a.dtype != np.float64 or not a.flags.c_contiguous):
                raise TypeError("Server: x / y must be C-contiguous float64 arrays")
        kind = r.get("kind", "matvec")
        kind = HM_REQ_SOLVE if kind in ("solve", HM_REQ_SOLVE) else HM_REQ_MATVEC
        return _Request(float(r.get("arrival_s", 0.0)), int(r["mesh"]), kind, int(r.get("nrhs", 1)),
                        int(r.get("seed", 0)), float(r.get("tol", 0.0)),
                        x.ctypes.data if x is not None else None, y.ctypes.data if y is not None else None)

    def footprint(self, r) -> int:
        b = ctypes.c_int64(0)
        q = self._request(r)
        _check(load().hm_server_footprint(self._h, ctypes.byref(q), ctypes.byref(b)))
        return int(b.value)

    def run(self, requests, realtime=True):
        n = len(requests)
        reqs = (_Request * max(n, 1))(*[self._request(r) for r in requests])
        res = (_Result * max(n, 1))()
        _check(load().hm_server_run(self._h, reqs, n, 1 if realtime else 0, res))
        return [dict(status=r.status, iterations=r.iterations, arrival_s=r.arrival_s,
                     start_s=r.start_s, done_s=r.done_s, rel_residual=r.rel_residual)
                for r in res[:n]]
