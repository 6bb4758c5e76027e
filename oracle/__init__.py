"""FP64 CPU oracle for the collocation Lame single-layer H-matrix.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and
the CPU-baseline leg of ``bench.py`` may import this package.  It shares no
code with the CUDA library in ``paper_2205_04752_gb300`` and never imports it.

The C part (``hm_oracle.c``) follows the paper step by step (see its header
for the passage behind each function); this module only marshals arguments and
adds the pieces for which a library routine is the plain definition:

* ``svd_rank`` / ``svd_truncate`` -- the truncated singular value
  decomposition, the best rank-k approximation (Section 2, Eckart-Young),
  computed with ``numpy.linalg.svd``;
* ``dense_matvec`` -- y = A x with ``numpy`` on the dense Kelvin matrix;
* ``amvm`` -- Algorithm 2 (adaptive matrix-vector multiplication, Section 3)
  step by step on the oracle's own ACA factors, with the readings stated in
  its docstring (per-block products are ``numpy`` matrix products);
* ``baca`` -- Algorithm 3 (Section 5) restricted to the single layer: the
  solve interleaved with block refinement, on a dense A_k formed from the
  oracle's factors, with a plain restarted GMRES (``numpy.linalg.lstsq`` for
  its small least-squares problems);
* the double-layer operator K_h of Eq. (Kh) in collocation form
  (``double_layer_dense``: K_Delta with hat functions, the surface curls T_h,
  V_Delta T_h and E/(1+nu) V_h T_h; matrix products by numpy);
* the evaluation operator ~V_h of Section 5, Eq. (vector_eq) (the displacement at points of
  the domain): ``points_matvec`` by its definition, and ``HMatrix`` with
  ``points=`` (a tree of the points for the rows, the same ACA).

Accuracy of the quadrature contract on badly shaped triangles (pinned in
``tests/test_oracle_pins.py``): the near-singular rule stays within 5e-6 up to
aspect ratio 30; the self term is within 5e-5 up to aspect ratio 4 (the
workloads' meshes) and degrades on slivers (1e-2 at 10:1), a limit of the
contract's 32-point angular rule.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "hm_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "libhm_oracle.so")
_lib = None
_lock = threading.Lock()

ND = 32          # Gauss-Legendre points of the self term
KERNELS = ("V_Delta", "V_11", "V_12", "V_13", "V_22", "V_23", "V_33")


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (OpenMP if available, no FMA contraction)."""
    os.makedirs(_BUILD, exist_ok=True)
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    base = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-ffp-contract=off",
            "-fno-fast-math", "-o", tmp, _SRC, "-lm"]
    try:
        subprocess.run(base[:1] + ["-fopenmp"] + base[1:], check=True,
                       capture_output=True)
    except subprocess.CalledProcessError:
        subprocess.run(base, check=True, capture_output=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _L():
    global _lib
    with _lock:
        if _lib is None:
            build()
            lib = ctypes.CDLL(_LIB_PATH)
            P = ctypes.c_void_p
            I64 = ctypes.c_int64
            I32 = ctypes.c_int32
            D = ctypes.c_double
            sig = {
                "or_radon7": (None, [P, P]),
                "or_gauss_legendre01": (None, [ctypes.c_int, P, P]),
                "or_centroids": (None, [P, P, I64, P]),
                "or_scalar_entry": (None, [P, P, P, ctypes.c_int, ctypes.c_int, P]),
                "or_kelvin_entry": (None, [P, P, P, ctypes.c_int, ctypes.c_int, D, D, P]),
                "or_scalar_rows": (None, [P, P, I64, P, I64, P]),
                "or_kelvin_rows_matvec": (None, [P, P, I64, D, D, P, I64, P, I64, P]),
                "or_kelvin_dense": (None, [P, P, I64, D, D, P]),
                "or_aca_dense": (I32, [P, I64, I64, D, D, I32, P, P, P, P, P, P]),
                "or_hmat_create": (P, [P, I64, P, I64, I64, D, D, D, I32]),
                "or_hmat_points_create": (P, [P, I64, P, I64, I64, P, I64, I64, D, D, D, I32]),
                "or_hmat_rsizes": (None, [P, P]),
                "or_hmat_rtree": (None, [P, P, P, P]),
                "or_kelvin_points_matvec": (None, [P, P, I64, D, D, P, I64, P, I64, P]),
                "or_scalar_points": (None, [P, P, I64, P, I64, P]),
                "or_dl_entry": (None, [P, P, P, ctypes.c_int, P]),
                "or_vpart_create": (P, [P, I64, P, I64, I64, I64, D]),
                "or_vpart_sizes": (None, [P, P]),
                "or_vpart_tree": (None, [P, P, P, P]),
                "or_vpart_blocks": (None, [P, P, P]),
                "or_vpart_free": (None, [P]),
                "or_dl_dense": (None, [P, I64, P, I64, P]),
                "or_hmat_free": (None, [P]),
                "or_hmat_sizes": (None, [P, P]),
                "or_hmat_tree": (None, [P, P, P, P]),
                "or_hmat_blocks": (None, [P, P, P]),
                "or_hmat_assemble": (None, [P, P, I64, P, I64]),
                "or_hmat_rank": (I32, [P, I64, ctypes.c_int]),
                "or_hmat_aca_flags": (I32, [P, I64, ctypes.c_int]),
                "or_hmat_factors": (None, [P, I64, ctypes.c_int, P, P]),
                "or_hmat_near_block": (None, [P, I64, P]),
                "or_hmat_matvec": (None, [P, D, D, P, P, I64, P, I64, P, I64]),
                "or_hmat_matvec_c": (None, [P, D, D, P, P, I64, P, I64, P, I64]),
                "or_num_threads": (I32, []),
                "or_set_num_threads": (None, [I32]),
            }
            for name, (res, args) in sig.items():
                f = getattr(lib, name)
                f.restype = res
                f.argtypes = args
            _lib = lib
    return _lib


def _p(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def _i32(a):
    return np.ascontiguousarray(a, dtype=np.int32)


def _i64(a):
    return np.ascontiguousarray(a, dtype=np.int64)


def num_threads() -> int:
    return int(_L().or_num_threads())


def set_num_threads(n: int) -> None:
    """OpenMP threads of the oracle's later calls from this thread (the
    results do not depend on it)."""
    _L().or_set_num_threads(int(n))


# --------------------------------------------------------------------------
# quadrature and entries
# --------------------------------------------------------------------------

def radon7():
    lam = np.zeros(21)
    w = np.zeros(7)
    _L().or_radon7(_p(lam), _p(w))
    return lam.reshape(7, 3), w


def gauss_legendre01(n: int):
    x = np.zeros(n)
    w = np.zeros(n)
    _L().or_gauss_legendre01(n, _p(x), _p(w))
    return x, w


def centroids(V, T) -> np.ndarray:
    V, T = _f64(V), _i32(T)
    C = np.zeros((T.shape[0], 3))
    _L().or_centroids(_p(V), _p(T), T.shape[0], _p(C))
    return C


def scalar_entry(x, V, tri, self_pair: bool, nd: int = ND) -> np.ndarray:
    """Seven scalar kernels (Eq. (Vh), collocation, 1/(4 pi) prefactor) of
    point x against triangle ``tri`` (3 vertex ids into V); the self term
    takes 1 <= nd <= 64 Gauss-Legendre points."""
    if not 1 <= nd <= 64:
        raise ValueError("nd must lie in 1..64")
    x, V, tri = _f64(x), _f64(V), _i32(tri)
    out = np.zeros(7)
    _L().or_scalar_entry(_p(x), _p(V), _p(tri), int(self_pair), nd, _p(out))
    return out


def kelvin_entry(x, V, tri, self_pair: bool, E: float, nu: float, nd: int = ND) -> np.ndarray:
    """int_tau S_K(x - y) ds_y from Kelvin's tensor directly, 3 x 3 (the
    self term with 1 <= nd <= 64 Gauss-Legendre points)."""
    if not 1 <= nd <= 64:
        raise ValueError("nd must lie in 1..64")
    x, V, tri = _f64(x), _f64(V), _i32(tri)
    out = np.zeros(9)
    _L().or_kelvin_entry(_p(x), _p(V), _p(tri), int(self_pair), nd, E, nu, _p(out))
    return out.reshape(3, 3)


def scalar_rows(V, T, rows) -> np.ndarray:
    """(7, len(rows), M) scalar-kernel matrix rows at the collocation points."""
    V, T, rows = _f64(V), _i32(T), _i64(rows)
    M = T.shape[0]
    out = np.zeros((7, rows.shape[0], M))
    _L().or_scalar_rows(_p(V), _p(T), M, _p(rows), rows.shape[0], _p(out))
    return out


def scalar_points(V, T, P) -> np.ndarray:
    """(7, len(P), M) scalar-kernel matrix at arbitrary points P (no self pair)."""
    V, T, P = _f64(V), _i32(T), _f64(P).reshape(-1, 3)
    M = T.shape[0]
    out = np.zeros((7, P.shape[0], M))
    _L().or_scalar_points(_p(V), _p(T), M, _p(P), P.shape[0], _p(out))
    return out


def points_matvec(V, T, E: float, nu: float, P, x) -> np.ndarray:
    """The evaluation operator of Section 5, Eq. (vector_eq) by its definition: u(x_r) =
    sum_j int_{tau_j} S_K(x_r - y) ds_y t_j at the points P (np x 3), from
    Kelvin's tensor.  x: (nrhs, 3M) densities; returns (nrhs, 3 np)."""
    V, T, P = _f64(V), _i32(T), _f64(P).reshape(-1, 3)
    x = _f64(np.atleast_2d(x))
    M = T.shape[0]
    y = np.zeros((x.shape[0], 3 * P.shape[0]))
    _L().or_kelvin_points_matvec(_p(V), _p(T), M, E, nu, _p(P), P.shape[0], _p(x), x.shape[0], _p(y))
    return y


def kelvin_dense(V, T, E: float, nu: float) -> np.ndarray:
    """Dense 3M x 3M collocation matrix of the Lame single layer, dof 3 i + a."""
    V, T = _f64(V), _i32(T)
    M = T.shape[0]
    A = np.zeros((3 * M, 3 * M))
    _L().or_kelvin_dense(_p(V), _p(T), M, E, nu, _p(A))
    return A


def dense_matvec(A: np.ndarray, x: np.ndarray) -> np.ndarray:
    """y = A x for x of shape (nrhs, 3M) (library matmul)."""
    return (A @ np.atleast_2d(x).T).T


def kelvin_rows_matvec(V, T, E: float, nu: float, rows, x) -> np.ndarray:
    """Exact rows (dofs 3 i + a, i in rows) of y = A x without forming A.
    x: (nrhs, 3M).  Returns (nrhs, 3 * len(rows))."""
    V, T, rows = _f64(V), _i32(T), _i64(rows)
    x = _f64(np.atleast_2d(x))
    M = T.shape[0]
    y = np.zeros((x.shape[0], 3 * rows.shape[0]))
    _L().or_kelvin_rows_matvec(_p(V), _p(T), M, E, nu, _p(rows), rows.shape[0], _p(x),
                               x.shape[0], _p(y))
    return y


def lame_coefficients(E: float, nu: float):
    """c1, c2 of Eq. (Vh) in collocation form: V_h = c1 diag(V_Delta) + c2 [V_kl]."""
    c1 = (1.0 + nu) * (3.0 - 4.0 * nu) / (2.0 * E * (1.0 - nu))
    c2 = (1.0 + nu) / (2.0 * E * (1.0 - nu))
    return c1, c2


# --------------------------------------------------------------------------
# ACA (Algorithm 1) and SVD truncation
# --------------------------------------------------------------------------

def aca_dense(A, eps: float, eta_stop: float = 0.8, kmax: int = 256):
    """Algorithm 1 on an explicit matrix.  Returns dict(U, V, rank, piv_i,
    piv_j, steps, flags) with U (m x k), V (n x k) so that A ~ U V^T."""
    A = _f64(A)
    m, n = A.shape
    kmax = int(kmax)
    U = np.zeros((kmax, m))
    Vv = np.zeros((kmax, n))
    pi = np.zeros(kmax, dtype=np.int64)
    pj = np.zeros(kmax, dtype=np.int64)
    steps = ctypes.c_int32(0)
    flags = ctypes.c_int32(0)
    k = _L().or_aca_dense(_p(A), m, n, eps, eta_stop, kmax, _p(U), _p(Vv), _p(pi), _p(pj),
                          ctypes.byref(steps), ctypes.byref(flags))
    return dict(U=U[:k].T.copy(), V=Vv[:k].T.copy(), rank=int(k), piv_i=pi[:k].copy(),
                piv_j=pj[:k].copy(), steps=int(steps.value), flags=int(flags.value))


def svd_rank(A: np.ndarray, eps: float) -> int:
    """Smallest r with ||A - A_r||_F <= eps ||A||_F (truncated SVD is the best
    rank-r approximation, Section 2)."""
    s = np.linalg.svd(A, compute_uv=False)
    tot = float(np.sum(s * s))
    if tot == 0.0:
        return 0
    tail = np.concatenate([np.cumsum((s * s)[::-1])[::-1], [0.0]])
    for r in range(len(s) + 1):
        if tail[r] <= eps * eps * tot:
            return r
    return len(s)


def svd_truncate(U: np.ndarray, V: np.ndarray, eps: float):
    """Recompress U V^T to the smallest rank r with relative Frobenius error
    <= eps via QR of both factors and an SVD of the small core."""
    if U.shape[1] == 0:
        return U, V
    qu, ru = np.linalg.qr(U)
    qv, rv = np.linalg.qr(V)
    w, s, zt = np.linalg.svd(ru @ rv.T)
    tot = float(np.sum(s * s))
    r = len(s)
    tail = np.concatenate([np.cumsum((s * s)[::-1])[::-1], [0.0]])
    for rr in range(len(s) + 1):
        if tail[rr] <= eps * eps * tot:
            r = rr
            break
    return (qu @ (w[:, :r] * s[:r])), (qv @ zt[:r].T)


# --------------------------------------------------------------------------
# the oracle's own H-matrix
# --------------------------------------------------------------------------

class HMatrix:
    """Cluster tree, partition, ACA factors and near blocks built by the
    oracle (FP64), and its H-matrix-vector product.

    With ``points`` (np x 3) the rows are those points instead of the
    collocation points: the evaluation operator ~V_h of Section 5, Eq. (vector_eq), rows
    clustered by a tree of the points (leaves of ``leaf_points``)."""

    def __init__(self, V, T, leaf: int, eta: float, eps: float, eta_stop: float = 0.8,
                 kmax: int = 256, points=None, leaf_points: int | None = None):
        self.V, self.T = _f64(V), _i32(T)
        self.M = self.T.shape[0]
        self.leaf, self.eta, self.eps, self.eta_stop, self.kmax = leaf, eta, eps, eta_stop, kmax
        if points is None:
            self.points = None
            self._h = _L().or_hmat_create(_p(self.V), self.V.shape[0], _p(self.T), self.M, leaf,
                                          eta, eps, eta_stop, kmax)
        else:
            self.points = _f64(points).reshape(-1, 3)
            lp = leaf if leaf_points is None else leaf_points
            self._h = _L().or_hmat_points_create(_p(self.V), self.V.shape[0], _p(self.T), self.M, leaf,
                                                 _p(self.points), self.points.shape[0], lp, eta, eps,
                                                 eta_stop, kmax)
        s = np.zeros(4, dtype=np.int64)
        _L().or_hmat_sizes(self._h, _p(s))
        self.nnodes, self.nadm, self.nnear = int(s[0]), int(s[1]), int(s[2])
        self.perm = np.zeros(self.M, dtype=np.int64)
        self.nodes = np.zeros((self.nnodes, 5), dtype=np.int64)
        self.boxes = np.zeros((self.nnodes, 6))
        _L().or_hmat_tree(self._h, _p(self.perm), _p(self.nodes), _p(self.boxes))
        self.adm = np.zeros((self.nadm, 2), dtype=np.int64)
        self.near = np.zeros((self.nnear, 2), dtype=np.int64)
        _L().or_hmat_blocks(self._h, _p(self.adm), _p(self.near))
        # the row tree (the point tree of ~V_h, else the triangle tree)
        r = np.zeros(2, dtype=np.int64)
        _L().or_hmat_rsizes(self._h, _p(r))
        self.nrnodes, self.Mr = int(r[0]), int(r[1])
        self.rperm = np.zeros(self.Mr, dtype=np.int64)
        self.rnodes = np.zeros((self.nrnodes, 5), dtype=np.int64)
        self.rboxes = np.zeros((self.nrnodes, 6))
        _L().or_hmat_rtree(self._h, _p(self.rperm), _p(self.rnodes), _p(self.rboxes))

    def __del__(self):
        h = getattr(self, "_h", None)
        if h:
            _L().or_hmat_free(h)
            self._h = None

    # block ranges in cluster order (rows in the row tree)
    def ranges(self, blocks: np.ndarray) -> np.ndarray:
        t, s = blocks[:, 0], blocks[:, 1]
        return np.stack([self.rnodes[t, 0], self.rnodes[t, 1], self.nodes[s, 0],
                         self.nodes[s, 1]], 1)

    @staticmethod
    def _ids(ids):
        """(pointer, count) with count -1 meaning 'all blocks'."""
        if ids is None:
            return None, -1, None
        a = _i64(ids)
        if a.size == 0:
            a = np.zeros(1, dtype=np.int64)
            return _p(a), 0, a
        return _p(a), a.size, a

    def assemble(self, adm_ids=None, near_ids=None):
        """Assemble the listed blocks (all of a kind when its list is None)."""
        pa, na, ka = self._ids(adm_ids)
        pn, nn, kn = self._ids(near_ids)
        _L().or_hmat_assemble(self._h, pa, na, pn, nn)

    def rank(self, b: int, kern: int) -> int:
        return int(_L().or_hmat_rank(self._h, b, kern))

    def ranks(self) -> np.ndarray:
        r = np.zeros((self.nadm, 7), dtype=np.int64)
        for b in range(self.nadm):
            for k in range(7):
                r[b, k] = _L().or_hmat_rank(self._h, b, k)
        return r

    def aca_flags(self, b: int, kern: int) -> int:
        return int(_L().or_hmat_aca_flags(self._h, b, kern))

    def factors(self, b: int, kern: int):
        t, s = self.adm[b]
        m = int(self.rnodes[t, 1] - self.rnodes[t, 0])
        n = int(self.nodes[s, 1] - self.nodes[s, 0])
        k = self.rank(b, kern)
        U = np.zeros((max(k, 0), m))
        Vv = np.zeros((max(k, 0), n))
        if k > 0:
            _L().or_hmat_factors(self._h, b, kern, _p(U), _p(Vv))
        return U.T.copy(), Vv.T.copy()

    def near_block(self, b: int) -> np.ndarray:
        t, s = self.near[b]
        m = int(self.rnodes[t, 1] - self.rnodes[t, 0])
        n = int(self.nodes[s, 1] - self.nodes[s, 0])
        out = np.zeros((7, m, n))
        _L().or_hmat_near_block(self._h, b, _p(out))
        return out

    def matvec(self, E: float, nu: float, x, adm_ids=None, near_ids=None) -> np.ndarray:
        x = _f64(np.atleast_2d(x))
        y = np.zeros((x.shape[0], 3 * self.Mr))
        pa, na, ka = self._ids(adm_ids)
        pn, nn, kn = self._ids(near_ids)
        _L().or_hmat_matvec(self._h, E, nu, _p(x), _p(y), x.shape[0], pa, na, pn, nn)
        return y

    def matvec_coeffs(self, c1: float, c2: float, x) -> np.ndarray:
        """The H-matrix product with the coefficients of Eq. (Vh) given
        directly: y_a = c1 V_Delta x_a + c2 sum_b V_ab x_b (the double layer
        of Eq. (Kh) applies the single layer's blocks with its own c1, c2)."""
        x = _f64(np.atleast_2d(x))
        y = np.zeros((x.shape[0], 3 * self.Mr))
        _L().or_hmat_matvec_c(self._h, float(c1), float(c2), _p(x), _p(y), x.shape[0], None, -1, None, -1)
        return y

    def dense_block(self, b: int, kern: int) -> np.ndarray:
        """The exact (quadrature-contract) scalar-kernel block of admissible
        block b, computed entry by entry."""
        t, s = self.adm[b]
        lo_t, hi_t = self.rnodes[t, :2]
        lo_s, hi_s = self.nodes[s, :2]
        rows = self.rperm[lo_t:hi_t]
        cols = self.perm[lo_s:hi_s]
        if self.points is not None:
            R = scalar_points(self.V, self.T, self.points[rows])[kern]
        else:
            R = scalar_rows(self.V, self.T, rows)[kern]
        return R[:, cols]


# --------------------------------------------------------------------------
# Adaptive matrix-vector multiplication (Algorithm 2)
# --------------------------------------------------------------------------

# kernel index of the component pair (p, q) of V_pq (V_11, V_12, V_13, V_22, V_23, V_33)
_KPQ = {1: (0, 0), 2: (0, 1), 3: (0, 2), 4: (1, 1), 5: (1, 2), 6: (2, 2)}


def sparsity_constant(Ho: "HMatrix") -> int:
    """c_sp of the block partition (Section 2.1): the largest number of
    blocks of P that share a row cluster, or a column cluster."""
    blocks = np.concatenate([Ho.adm, Ho.near]) if Ho.nnear else Ho.adm
    rows = np.bincount(blocks[:, 0], minlength=Ho.nrnodes)
    cols = np.bincount(blocks[:, 1], minlength=Ho.nnodes)
    return int(max(rows.max(), cols.max()))


def amvm(Ho: "HMatrix", E: float, nu: float, x, theta: float = 0.7, eps: float = 1e-6,
         r0: int = 2, look: int = 2, max_iter: int = 1000, record_scan: bool = False):
    """Algorithm 2 (adaptive matrix-vector multiplication, Section 3) on the
    oracle's own H-matrix, FP64, for one vector x (3M dofs, original order);
    the rows are the 3 Mr dofs of the row points (Mr = M unless Ho is the
    evaluation operator of Section 5, Eq. (vector_eq)).

    Readings (the paper leaves these open):
    * A_k keeps, on every admissible block t x s, the first r_b crosses of
      each of the block's seven ACA sequences (Algorithm 1 as assembled with
      the matrix's ACA epsilon; a sequence shorter than r_b is used whole);
      A_0 has r_b = r0 = 2.  The look-ahead A^_k has r_b + look crosses
      (look = 2, "two steps of ACA ahead").  Near blocks are exact in both.
    * Marking is per block t x s: a marked block moves all seven kernels to
      the look-ahead ranks, A_{k+1} = A^_k on it.
    * Rows are the 3 Mr dofs (component a of row cluster position p is row
      3p + a); the threshold (1 - theta)(c_sp M N)^{-1/2} gamma_k takes the
      paper's M x N as 3 Mr x 3M; rows of equal error are taken in increasing
      row order.
    * Step 4 stops when gamma_k <= eps * ||b^_k|| (a relative epsilon) and
      returns b_k; it also stops when no block can be refined any more.

    Returns a dict: b (A_k x at the last k, original order), b_hat, gamma
    (gamma_k per iteration), gamma_rest (gamma_k(P_k) per iteration), marked
    (|P_k| per iteration), ranks (min(r_b, full rank) per block and kernel at
    the end), r (r_b per block at the end), csp, iterations; with
    ``record_scan`` also scans: per refinement, gamma_k(P_k) after each row
    of the step-3 scan up to the stopping row."""
    x = _f64(x).reshape(-1)
    M, Mr = Ho.M, Ho.Mr
    c1, c2 = lame_coefficients(E, nu)
    perm, rperm = Ho.perm, Ho.rperm
    Xc = x.reshape(M, 3)[perm]                                  # cluster order
    rng = Ho.ranges(Ho.adm)                                     # lo_t, hi_t, lo_s, hi_s
    nb = Ho.nadm
    F = [[Ho.factors(b, k) for k in range(7)] for b in range(nb)]
    full = np.array([[F[b][k][0].shape[1] for k in range(7)] for b in range(nb)], dtype=np.int64)

    def part(b: int, l0: int, l1: int) -> np.ndarray:
        """The crosses l0 .. l1 - 1 of block b applied to x(s): (|t|, 3)."""
        lo_t, hi_t, lo_s, hi_s = rng[b]
        xs = Xc[lo_s:hi_s]
        out = np.zeros((hi_t - lo_t, 3))
        for k in range(7):
            U, Vv = F[b][k]
            a, z = min(l0, U.shape[1]), min(l1, U.shape[1])
            if a >= z:
                continue
            W = Vv[:, a:z].T @ xs                               # (z - a, 3)
            if k == 0:
                out += c1 * (U[:, a:z] @ W)
            else:
                p, q = _KPQ[k]
                out[:, p] += c2 * (U[:, a:z] @ W[:, q])
                if p != q:
                    out[:, q] += c2 * (U[:, a:z] @ W[:, p])
        return out

    # b_0: near field exactly, every admissible block at rank r0
    near = Ho.matvec(E, nu, x, adm_ids=[])[0].reshape(Mr, 3)[rperm]
    r = np.full(nb, int(r0), dtype=np.int64)
    bk = near.copy()
    for b in range(nb):
        bk[rng[b, 0]:rng[b, 1]] += part(b, 0, r0)
    csp = sparsity_constant(Ho)
    N, Ncol = 3 * Mr, 3 * M
    # blocks whose row cluster holds cluster position p, in block order
    blocks_of_pos = [[] for _ in range(Mr)]
    for b in range(nb):
        for p in range(rng[b, 0], rng[b, 1]):
            blocks_of_pos[p].append(b)
    hist = dict(gamma=[], gamma_rest=[], marked=[])
    scans = []
    delta = [part(b, r[b], r[b] + look) for b in range(nb)]
    it = 0
    while True:
        e = np.zeros((Mr, 3))
        for b in range(nb):
            e[rng[b, 0]:rng[b, 1]] += delta[b]
        bhat = bk + e
        gamma = float(np.linalg.norm(e))
        hist["gamma"].append(gamma)
        if gamma <= eps * float(np.linalg.norm(bhat)) or it >= max_iter:
            break
        # step 3: Doerfler marking through the rows in decreasing error
        thr = (1.0 - theta) * gamma / np.sqrt(csp * float(N) * float(Ncol))
        err = np.abs(e).reshape(-1)
        order = np.lexsort((np.arange(N), -err))              # decreasing error, then row
        rest = e.copy()
        marked = []
        is_marked = np.zeros(nb, dtype=bool)
        g_rest = gamma
        scan = []
        for i in order:
            p, a = divmod(int(i), 3)
            for b in blocks_of_pos[p]:
                if is_marked[b]:
                    continue
                if abs(delta[b][p - rng[b, 0], a]) >= thr:
                    is_marked[b] = True
                    marked.append(b)
                    rest[rng[b, 0]:rng[b, 1]] -= delta[b]
            g_rest = float(np.linalg.norm(rest))
            if record_scan:
                scan.append(g_rest)
            if gamma - g_rest >= theta * gamma:
                break
        if record_scan:
            scans.append(np.array(scan))
        hist["gamma_rest"].append(g_rest)
        hist["marked"].append(len(marked))
        if not marked:
            break
        # step 4: A_{k+1} = A^_k on the marked blocks
        for b in marked:
            bk[rng[b, 0]:rng[b, 1]] += delta[b]
            r[b] += look
            delta[b] = part(b, r[b], r[b] + look)
        it += 1
    out = np.zeros(3 * Mr)
    out.reshape(Mr, 3)[rperm] = bk
    outh = np.zeros(3 * Mr)
    outh.reshape(Mr, 3)[rperm] = bhat
    res = dict(b=out, b_hat=outh, ranks=np.minimum(r[:, None], full), full_ranks=full, r=r.copy(),
               csp=csp, iterations=it, **hist)
    if record_scan:
        res["scans"] = scans
    return res


# --------------------------------------------------------------------------
# Block-adaptive ACA for the single layer (Algorithm 3, branch (iii))
# --------------------------------------------------------------------------

def _dense_block(Ho: "HMatrix", F, rng, b: int, l0: int, l1: int, c1: float, c2: float) -> np.ndarray:
    """The crosses l0 .. l1 - 1 of admissible block b as a dense (3|t|, 3|s|)
    block of V_h, rows 3i + a and columns 3j + c in cluster order:
    c1 U V^T on the diagonal components for V_Delta, c2 U V^T at (p, q) and
    (q, p) for V_pq (Eq. (Vh))."""
    lo_t, hi_t, lo_s, hi_s = rng[b]
    m, n = hi_t - lo_t, hi_s - lo_s
    out = np.zeros((3 * m, 3 * n))
    for k in range(7):
        U, Vv = F[b][k]
        a, z = min(l0, U.shape[1]), min(l1, U.shape[1])
        if a >= z:
            continue
        S = U[:, a:z] @ Vv[:, a:z].T
        if k == 0:
            for p in range(3):
                out[p::3, p::3] += c1 * S
        else:
            p, q = _KPQ[k]
            out[p::3, q::3] += c2 * S
            if p != q:
                out[q::3, p::3] += c2 * S
    return out


def _gmres(A, b, x, tol_of, restart: int, max_it: int, floor: float):
    """Restarted GMRES(m) on the dense matrix A (plain: Arnoldi with
    modified Gram-Schmidt, the small least-squares problem by
    numpy.linalg.lstsq).  A cycle ends early when its residual estimate is
    <= tol, tol = tol_of(x) at the cycle's start; after each cycle the solve
    ends when ||b - A x|| <= tol_of(x) (or <= floor, or at max_it
    iterations).  Returns (x, iterations)."""
    its = 0
    while True:
        r = b - A @ x
        beta = float(np.linalg.norm(r))
        tol = tol_of(x)
        if beta <= tol or beta <= floor or its >= max_it:
            return x, its
        Q = [r / beta]
        Hh = np.zeros((restart + 1, restart))
        j_end = 0
        for j in range(restart):
            w = A @ Q[j]
            for i in range(j + 1):
                Hh[i, j] = float(Q[i] @ w)
                w = w - Hh[i, j] * Q[i]
            Hh[j + 1, j] = float(np.linalg.norm(w))
            its += 1
            j_end = j + 1
            e1 = np.zeros(j + 2)
            e1[0] = beta
            y, *_ = np.linalg.lstsq(Hh[:j + 2, :j + 1], e1, rcond=None)
            est = float(np.linalg.norm(e1 - Hh[:j + 2, :j + 1] @ y))
            if est <= tol or Hh[j + 1, j] <= 1e-300 or its >= max_it:
                break
            Q.append(w / Hh[j + 1, j])
        x = x + np.stack(Q[:j_end], 1) @ y


def baca(Ho: "HMatrix", E: float, nu: float, b, theta: float = 0.8, alpha: float = 10.0,
         eps: float = 1e-4, r0: int = 8, look: int = 2, tol0: float = 0.1, restart: int = 50,
         max_it: int = 100000, max_steps: int = 1000):
    """Algorithm 3 of Section 5 restricted to the single layer (branch (iii)):
    solve V_h t = b while the H-matrix approximation is refined block by
    block, FP64, on the oracle's own ACA factors.

    Readings (the paper leaves these open; it runs Bramble-Pasciak CG on the
    saddle system):
    * A_k keeps the first r_b crosses of each of the seven ACA sequences of
      block b (A_0: r_b = r0); the look-ahead A^_k has r_b + look; near blocks
      exact in both.  A block of P_adm is a block t x s of V_h (all seven
      kernels); refining it sets A_{k+1} = A^_k on it.
    * Step 2 is restarted GMRES(m) from x_{k-1} (x_{-1} = 0): a cycle ends
      early when its residual estimate falls to tau = alpha ||(A_k - A^_k) x||
      at the cycle's start (tau = tol0 ||b|| while x = 0); after each cycle the
      solve ends when ||b - A_k x|| <= alpha ||(A_k - A^_k) x|| (Eq. (solvCond))
      or the residual is below 1e-13 ||b||.
    * E_k^2 = sum_b ||(A_k - A^_k)_b x_k||^2; step 3 marks the fewest blocks
      with E_k(M_k) >= theta E_k: blocks in decreasing ||(A_k - A^_k)_b x_k||
      (ties: lower block index first) until the condition holds.
    * The loop stops when E_k <= eps ||b|| (a relative epsilon) after a
      solve, returning x_k, or when no block can be refined.

    Returns a dict: x (original order), E (per step), iterations (GMRES per
    step), marked (per step), ranks (r_b at the end, capped by the sequences),
    steps, and per step the final residual ||b - A_k x_k||, ||(A_k - A^_k)
    x_k||, the squared block parts and the marked blocks."""
    b = _f64(b).reshape(-1)
    M = Ho.M
    N = 3 * M
    c1, c2 = lame_coefficients(E, nu)
    perm = Ho.perm
    rng = Ho.ranges(Ho.adm)
    nrng = Ho.ranges(Ho.near) if Ho.nnear else np.zeros((0, 4), dtype=np.int64)
    nb = Ho.nadm
    F = [[Ho.factors(bb, k) for k in range(7)] for bb in range(nb)]
    full = np.array([[F[bb][k][0].shape[1] for k in range(7)] for bb in range(nb)], dtype=np.int64)
    # cluster order, component fastest: row 3p + a
    bc = b.reshape(M, 3)[perm].reshape(-1)
    A0 = np.zeros((N, N))
    for q in range(Ho.nnear):
        lo_t, hi_t, lo_s, hi_s = nrng[q]
        Nb = Ho.near_block(q)
        blk = np.zeros((3 * (hi_t - lo_t), 3 * (hi_s - lo_s)))
        for p in range(3):
            blk[p::3, p::3] += c1 * Nb[0]
        for k in range(1, 7):
            p, qq = _KPQ[k]
            blk[p::3, qq::3] += c2 * Nb[k]
            if p != qq:
                blk[qq::3, p::3] += c2 * Nb[k]
        A0[3 * lo_t:3 * hi_t, 3 * lo_s:3 * hi_s] += blk
    r = np.full(nb, int(r0), dtype=np.int64)
    Ak = A0.copy()
    for bb in range(nb):
        lo_t, hi_t, lo_s, hi_s = rng[bb]
        Ak[3 * lo_t:3 * hi_t, 3 * lo_s:3 * hi_s] += _dense_block(Ho, F, rng, bb, 0, r0, c1, c2)
    look_blk = [_dense_block(Ho, F, rng, bb, r0, r0 + look, c1, c2) for bb in range(nb)]

    def parts(x):
        """(A^_k - A_k)_b x for every block, and their sum."""
        P = []
        e = np.zeros(N)
        for bb in range(nb):
            lo_t, hi_t, lo_s, hi_s = rng[bb]
            d = look_blk[bb] @ x[3 * lo_s:3 * hi_s]
            P.append(d)
            e[3 * lo_t:3 * hi_t] += d
        return P, e

    bnorm = float(np.linalg.norm(bc))
    x = np.zeros(N)
    hist = dict(E=[], iterations=[], marked=[], residual=[], lookahead=[], parts=[], marked_sets=[])
    k = 0
    while True:
        def tol_of(xx):
            if not np.any(xx):
                return tol0 * bnorm
            return alpha * float(np.linalg.norm(parts(xx)[1]))
        x, its = _gmres(Ak, bc, x, tol_of, restart, max_it, 1e-13 * bnorm)
        hist["iterations"].append(its)
        P, e = parts(x)
        hist["residual"].append(float(np.linalg.norm(bc - Ak @ x)))
        hist["lookahead"].append(float(np.linalg.norm(e)))
        bn2 = np.array([float(d @ d) for d in P])
        hist["parts"].append(bn2)
        Ek = float(np.sqrt(bn2.sum()))
        hist["E"].append(Ek)
        if Ek <= eps * bnorm or k >= max_steps:
            break
        order = np.lexsort((np.arange(nb), -bn2))
        acc, marked = 0.0, []
        target = (theta * Ek) ** 2
        for bb in order:
            if acc >= target:
                break
            if bn2[bb] == 0.0:
                break
            marked.append(int(bb))
            acc += bn2[bb]
        hist["marked"].append(len(marked))
        hist["marked_sets"].append(marked)
        if not marked:
            break
        for bb in marked:
            lo_t, hi_t, lo_s, hi_s = rng[bb]
            Ak[3 * lo_t:3 * hi_t, 3 * lo_s:3 * hi_s] += look_blk[bb]
            r[bb] += look
            look_blk[bb] = _dense_block(Ho, F, rng, bb, r[bb], r[bb] + look, c1, c2)
        k += 1
    out = np.zeros(N)
    out.reshape(M, 3)[perm] = x.reshape(M, 3)
    return dict(x=out, ranks=np.minimum(r[:, None], full), full_ranks=full, steps=k, **hist)


# --------------------------------------------------------------------------
# The double-layer operator K_h (Section 4.2, Eq. (Kh)), collocation form
# --------------------------------------------------------------------------

def dl_dense(V, T) -> np.ndarray:
    """K_Delta of Eq. (Kh) at the centroids: (M, nv), column p the hat
    function of vertex p, (1/(4 pi)) int (c_i - y).n / |c_i - y|^3 psi_p(y) ds_y
    (the triangle's own flat panel gives 0)."""
    V, T = _f64(V), _i32(T)
    out = np.zeros((T.shape[0], V.shape[0]))
    _L().or_dl_dense(_p(V), V.shape[0], _p(T), T.shape[0], _p(out))
    return out


def surface_curls(V, T) -> np.ndarray:
    """T_kl,h of Eq. (Kh): (3, 3, M, nv) with T[k, l][i, p] = n_l d_k psi_p -
    n_k d_l psi_p on triangle i (constant there; psi_p the hat function of
    vertex p, n the unit normal from the vertex order).  Reading of the
    boundary operators T_kl: the tangential (Guenter) derivative n_l d_k -
    n_k d_l, antisymmetric in (k, l) as the block structure of T_h requires.
    d psi_a on (p0, p1, p2) is n x (p_{a+2} - p_{a+1}) / (2 area)."""
    V, T = _f64(V), _i32(T)
    M, nv = T.shape[0], V.shape[0]
    out = np.zeros((3, 3, M, nv))
    for i in range(M):
        P = V[T[i]]
        c = np.cross(P[1] - P[0], P[2] - P[0])
        A2 = float(np.linalg.norm(c))
        n = c / A2
        for a in range(3):
            g = np.cross(n, P[(a + 2) % 3] - P[(a + 1) % 3]) / A2
            for k in range(3):
                for l in range(3):
                    out[k, l, i, T[i, a]] += n[l] * g[k] - n[k] * g[l]
    return out


def double_layer_dense(V, T, E: float, nu: float) -> np.ndarray:
    """K_h of Eq. (Kh) in collocation form, (3M, 3 nv), rows 3i + a (centroid
    i, component a), columns 3p + b (vertex p, component b):
        K_h = diag(K_Delta) - diag(V_Delta) T_h + E / (1 + nu) V_h T_h,
    with T_h the 3 x 3 block matrix [[0, T12, T13], [-T12, 0, T23],
    [-T13, -T23, 0]] of the surface curls (matrix products by numpy)."""
    V, T = _f64(V), _i32(T)
    M, nv = T.shape[0], V.shape[0]
    KD = dl_dense(V, T)
    S = surface_curls(V, T)
    Th = np.zeros((3 * M, 3 * nv))
    for a, b in ((0, 1), (0, 2), (1, 2)):
        Th[a::3, b::3] = S[a, b]
        Th[b::3, a::3] = -S[a, b]
    VD = scalar_rows(V, T, np.arange(M))[0]
    Vh = kelvin_dense(V, T, E, nu)
    K = np.zeros((3 * M, 3 * nv))
    for a in range(3):
        K[a::3, a::3] = KD
    VDT = np.zeros((3 * M, 3 * nv))
    for a in range(3):
        VDT[a::3, :] = VD @ Th[a::3, :]
    return K - VDT + (E / (1.0 + nu)) * (Vh @ Th)


class VertexPartition:
    """The block partition of the double layer's K_Delta (Eq. (Kh)): rows the
    triangle tree (``HMatrix``'s), columns a tree of the vertices whose boxes
    are the unions of the vertices' stars (the supports of their hat
    functions), Eq. (adm) with eta."""

    def __init__(self, V, T, leaf: int, leaf_v: int, eta: float):
        self.V, self.T = _f64(V), _i32(T)
        self._h = _L().or_vpart_create(_p(self.V), self.V.shape[0], _p(self.T), self.T.shape[0], leaf, leaf_v, eta)
        s = np.zeros(4, dtype=np.int64)
        _L().or_vpart_sizes(self._h, _p(s))
        self.nnodes, self.nadm, self.nnear, self.nv = map(int, s)
        self.perm = np.zeros(self.nv, dtype=np.int64)
        self.nodes = np.zeros((self.nnodes, 5), dtype=np.int64)
        self.boxes = np.zeros((self.nnodes, 6))
        _L().or_vpart_tree(self._h, _p(self.perm), _p(self.nodes), _p(self.boxes))
        self.adm = np.zeros((self.nadm, 2), dtype=np.int64)
        self.near = np.zeros((self.nnear, 2), dtype=np.int64)
        _L().or_vpart_blocks(self._h, _p(self.adm), _p(self.near))

    def __del__(self):
        h = getattr(self, "_h", None)
        if h:
            _L().or_vpart_free(h)
            self._h = None


class DoubleLayerHMatrix:
    """The H-matrix of the double layer's K_Delta (Eq. (Kh)) on the partition
    of ``VertexPartition``: Algorithm 1 (``aca_dense``) on every admissible
    block of the dense K_Delta (``dl_dense``; small meshes), near blocks
    dense.  Rows and columns in cluster order (the triangle tree of
    ``HMatrix`` and the vertex tree)."""

    def __init__(self, V, T, leaf: int, leaf_v: int, eta: float, eps: float, eta_stop: float = 0.8):
        self.V, self.T = _f64(V), _i32(T)
        self.vp = VertexPartition(self.V, self.T, leaf, leaf_v, eta)
        self.tri = HMatrix(self.V, self.T, leaf, eta, eps)  # its triangle tree (rows)
        KD = dl_dense(self.V, self.T)
        tn, tp = self.tri.nodes, self.tri.perm
        vn, vperm = self.vp.nodes, self.vp.perm
        self.KDc = KD[tp][:, vperm]  # cluster order
        self.factors = []
        for (t, s) in self.vp.adm:
            blk = self.KDc[tn[t, 0]:tn[t, 1], vn[s, 0]:vn[s, 1]]
            self.factors.append(aca_dense(blk, eps, eta_stop))
        self.near = [self.KDc[tn[t, 0]:tn[t, 1], vn[s, 0]:vn[s, 1]].copy() for (t, s) in self.vp.near]

    def matvec(self, u) -> np.ndarray:
        """y = K_Delta u (u over the vertices, y over the triangles, original
        order): U (V^T u_s) per admissible block, dense near blocks."""
        u = _f64(u).reshape(-1)
        tn, tp = self.tri.nodes, self.tri.perm
        vn, vperm = self.vp.nodes, self.vp.perm
        uc = u[vperm]
        yc = np.zeros(self.T.shape[0])
        for (t, s), f in zip(self.vp.adm, self.factors):
            yc[tn[t, 0]:tn[t, 1]] += f["U"] @ (f["V"].T @ uc[vn[s, 0]:vn[s, 1]])
        for (t, s), Nb in zip(self.vp.near, self.near):
            yc[tn[t, 0]:tn[t, 1]] += Nb @ uc[vn[s, 0]:vn[s, 1]]
        y = np.zeros_like(yc)
        y[tp] = yc
        return y
