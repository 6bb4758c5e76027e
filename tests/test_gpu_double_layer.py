"""The double-layer operator K_h of Section 4.2, Eq. (Kh), on the GPU (through
the C ABI) against the oracle: K_Delta's near entries and every admissible
block's ACA on the vertex partition, its H-matrix product, the whole K_h
product against the oracle's H-matrix form (1e-12) and its dense matrix
(the ACA accuracy), and rigid motions mapped to -1/2 of themselves."""
import numpy as np
import pytest

import oracle
from paper_2205_04752_gb300 import binding, inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

E, NU = 1.0, 0.3
LEAF, LEAF_V, ETA = 32, 24, 0.8
_cache = {}


def _rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def case(eps=1e-4):
    """Level-3 icosphere (1280 triangles, 642 vertices): the single layer V,
    K_Delta on the vertex partition, and the oracle's counterparts."""
    if eps not in _cache:
        V, T = inputs.icosphere(3)
        tree = binding.build_cluster_tree(V, T, LEAF, ETA)
        vt = binding.build_vertex_tree(tree, LEAF_V)
        Hv = binding.aca_assemble(tree, E, NU, eps, max_rhs=2)
        Kd = binding.aca_assemble(vt, E, NU, eps, max_rhs=2)
        Ho = oracle.HMatrix(V, T, LEAF, ETA, eps)
        Ho.assemble()
        Hd = oracle.DoubleLayerHMatrix(V, T, LEAF, LEAF_V, ETA, eps)
        _cache[eps] = (V, T, tree, vt, Hv, Kd, Ho, Hd)
    return _cache[eps]


def curl_matrix(V, T):
    """T_h of Eq. (Kh) as a dense (3M, 3 nv) matrix from the oracle's surface curls."""
    S = oracle.surface_curls(V, T)
    M, nv = len(T), len(V)
    Th = np.zeros((3 * M, 3 * nv))
    for a, b in ((0, 1), (0, 2), (1, 2)):
        Th[a::3, b::3] = S[a, b]
        Th[b::3, a::3] = -S[a, b]
    return Th


def oracle_h_form(Ho, Hd, V, T, u):
    """K_h u from the oracle's H-matrices: K_Delta per component plus the
    single layer applied to T_h u with ((1-2nu)/(2(1-nu)), 1/(2(1-nu)))."""
    M, nv = len(T), len(V)
    y = np.zeros(3 * M)
    ur = u.reshape(nv, 3)
    for b in range(3):
        y[b::3] = Hd.matvec(ur[:, b])
    w = curl_matrix(V, T) @ u
    c1, c2 = (1 - 2 * NU) / (2 * (1 - NU)), 1 / (2 * (1 - NU))
    return y + Ho.matvec_coeffs(c1, c2, w)[0]


def gpu_dl(Hv, Kd, u, form="fp64"):
    ud = torch.tensor(np.ascontiguousarray(u), device="cuda")
    yd = torch.full((3 * Hv.M,), float("nan"), dtype=torch.float64, device="cuda")
    binding.double_layer_matvec(Hv, Kd, ud, yd, form)
    torch.cuda.synchronize()
    return yd.cpu().numpy()


def test_k_delta_near_entries_and_aca_match_oracle():
    """Every near block of K_Delta to 1e-12 of the block's scale, and every
    admissible block: the same rank and U V^T within 1e-12 of the oracle's."""
    V, T, tree, vt, Hv, Kd, Ho, Hd = case()
    perm, nodes, adm, near = vt.export()
    tn, vn = Hd.tri.nodes, Hd.vp.nodes
    np.testing.assert_array_equal(adm, Hd.vp.adm)
    np.testing.assert_array_equal(near, Hd.vp.near)
    for b, (t, s) in enumerate(Hd.vp.near):
        m, n = tn[t, 1] - tn[t, 0], vn[s, 1] - vn[s, 0]
        g = Kd.near_block(b, m, n)
        o = Hd.near[b]
        scale = max(np.abs(o).max(), 1e-300)
        assert np.abs(g[0] - o).max() <= 1e-12 * scale, b
        assert not np.any(g[1:]), b
    worst = 0.0
    for b, ((t, s), f) in enumerate(zip(Hd.vp.adm, Hd.factors)):
        m, n = tn[t, 1] - tn[t, 0], vn[s, 1] - vn[s, 0]
        Ug, Vg = Kd.factors(b, 0, m, n)
        assert Ug.shape[1] == f["rank"], b
        for k in range(1, 7):
            assert Kd.factors(b, k, m, n)[0].shape[1] == 0
        So = f["U"] @ f["V"].T
        if np.linalg.norm(So) > 0:
            worst = max(worst, np.linalg.norm(Ug @ Vg.T - So) / np.linalg.norm(So))
    assert worst <= 1e-12


def test_k_delta_product_matches_oracle():
    """hm_eval_points on K_Delta applies it to each component of u: equal to
    the oracle's H-matrix of K_Delta to 1e-12; the rows of K_Delta sum to
    -1/2 (the solid angle) within the ACA accuracy."""
    V, T, tree, vt, Hv, Kd, Ho, Hd = case()
    nv = len(V)
    u = inputs.uniform_rhs(3 * nv, 5)[0]
    ud = torch.tensor(u, device="cuda")
    yd = torch.empty(3 * len(T), dtype=torch.float64, device="cuda")
    binding.eval_points(Kd, ud, yd)
    torch.cuda.synchronize()
    y = yd.cpu().numpy()
    for b in range(3):
        yo = Hd.matvec(u.reshape(nv, 3)[:, b])
        assert _rel(y[b::3], yo) <= 1e-12, b
    binding.eval_points(Kd, torch.ones(3 * nv, dtype=torch.float64, device="cuda"), yd)
    torch.cuda.synchronize()
    assert np.abs(yd.cpu().numpy() + 0.5).max() <= 1e-6 + 10 * 1e-4


def test_double_layer_product_matches_oracle_h_form_and_dense():
    """y = K_h u in the FP64 form: the oracle's H-matrix form to 1e-12, the
    oracle's dense K_h (every entry from its definition) to the ACA accuracy."""
    V, T, tree, vt, Hv, Kd, Ho, Hd = case()
    u = inputs.uniform_rhs(3 * len(V), 6)[0]
    y = gpu_dl(Hv, Kd, u)
    assert _rel(y, oracle_h_form(Ho, Hd, V, T, u)) <= 1e-12
    Kdense = oracle.double_layer_dense(V, T, E, NU)
    assert _rel(y, Kdense @ u) <= 1e-4


def test_rigid_motions_are_mapped_to_minus_half():
    """Translations and rotations u(y) = omega x y give K_h u = -u/2 at the
    centroids (the jump relation of the double layer for rigid motions),
    through the GPU path at ACA eps 1e-8."""
    V, T, tree, vt, Hv, Kd, Ho, Hd = case(1e-8)
    M, nv = len(T), len(V)
    C = oracle.centroids(V, T)
    c = np.array([1.0, -2.0, 0.5])
    y = gpu_dl(Hv, Kd, np.tile(c, nv)).reshape(M, 3)
    assert np.abs(y + 0.5 * c).max() <= 1e-5 * np.abs(c).max()
    om = np.array([0.3, -0.5, 0.8])
    ref = -0.5 * np.cross(om, C)
    y = gpu_dl(Hv, Kd, np.cross(om, V).reshape(-1)).reshape(M, 3)
    assert np.abs(y - ref).max() <= 1e-5 * np.abs(ref).max()


@pytest.mark.parametrize("form,tol", [("fp32", 1e-6), ("i16", 6e-5), ("fp16", 2e-4)])
def test_double_layer_reduced_forms(form, tol):
    """The single-layer part of K_h in a packed form, against the FP64 form."""
    V, T, tree, vt, Hv, Kd, Ho, Hd = case()
    Hv.pack(form)
    u = inputs.uniform_rhs(3 * len(V), 7, nrhs=2)
    y64 = np.stack([gpu_dl(Hv, Kd, u[r]) for r in range(2)])
    ud = torch.tensor(u, device="cuda")
    yd = torch.empty((2, 3 * len(T)), dtype=torch.float64, device="cuda")
    binding.double_layer_matvec(Hv, Kd, ud, yd, form)
    torch.cuda.synchronize()
    y = yd.cpu().numpy()
    for r in range(2):
        assert _rel(y[r], y64[r]) <= tol, r


def test_double_layer_argument_errors():
    """Refusals of the C ABI (called directly, past the binding's own shape
    checks): V must be a single layer, K a K_Delta of the same mesh."""
    import ctypes
    V, T, tree, vt, Hv, Kd, Ho, Hd = case()
    lib = binding.load()
    u = torch.zeros(3 * max(len(V), len(T)), dtype=torch.float64, device="cuda")
    y = torch.zeros_like(u)

    def call(A, B):
        return lib.hm_double_layer_matvec(A._h, B._h, ctypes.c_void_p(u.data_ptr()), ctypes.c_void_p(y.data_ptr()),
                                          1, binding.FP64, None)
    assert call(Kd, Kd) == binding.HM_EINVAL          # V must be the single layer
    assert call(Hv, Hv) == binding.HM_EINVAL          # K must be K_Delta
    V2, T2 = inputs.icosphere(3)
    tr2 = binding.build_cluster_tree(V2 * 1.5, T2, LEAF, ETA)
    H2 = binding.aca_assemble(tr2, E, NU, 1e-4, max_rhs=1)
    assert call(H2, Kd) == binding.HM_EINVAL          # another mesh
    assert b"different meshes" in lib.hm_last_error()
    with pytest.raises(binding.HMError):
        binding.amvm(Kd, u[:3 * len(V)], y[:3 * len(T)])   # not for K_Delta
