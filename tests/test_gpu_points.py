"""GPU parity of the evaluation operator ~V_h (Section 5, Eq. (vector_eq):
the displacement at points of the domain) through the C ABI
(``hm_build_point_tree``, ``hm_aca_assemble``, ``hm_eval_points``,
``hm_amvm``) against the FP64 CPU oracle on the same seeded inputs.

Tolerances: near-field entries and ACA reconstructions against the oracle's
same blocks 1e-12 (relative); the product against the oracle's H-matrix
product 1e-12 and against the operator's definition within the ACA accuracy;
the adaptive product as for the square matrix."""
import numpy as np
import pytest

import oracle
from paper_2205_04752_gb300 import binding, inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

E, NU = 1.0, 0.3


def _rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


class PCase:
    def __init__(self, level, npts, leaf, leaf_pts, eps, r_in=0.0, r_out=0.95, seed=3, eta=0.8,
                 defer_aca=False, oracle_h=True):
        self.V, self.T = inputs.icosphere(level)
        self.M = len(self.T)
        self.P = inputs.shell_points(npts, r_in, r_out, seed)
        self.tree = binding.build_cluster_tree(self.V, self.T, leaf, eta)
        self.pt = binding.build_point_tree(self.tree, self.P, leaf_pts)
        self.H = binding.aca_assemble(self.pt, E, NU, eps, max_rhs=1, defer_aca=defer_aca)
        self.perm, self.nodes, self.adm, self.near = self.pt.export()
        _, self.snodes, _, _ = self.tree.export()
        self.Ho = None
        if oracle_h:
            self.Ho = oracle.HMatrix(self.V, self.T, leaf, eta, eps, points=self.P, leaf_points=leaf_pts)
            self.Ho.assemble()

    def rows(self, b, blocks):
        t, s = blocks[b]
        return int(self.nodes[t, 1] - self.nodes[t, 0]), int(self.snodes[s, 1] - self.snodes[s, 0])

    def eval(self, x, form="fp64"):
        td = torch.tensor(np.ascontiguousarray(np.atleast_2d(x)), device="cuda")
        ud = torch.full((td.shape[0], 3 * len(self.P)), np.nan, dtype=torch.float64, device="cuda")
        binding.eval_points(self.H, td, ud, form)
        torch.cuda.synchronize()
        return ud.cpu().numpy()

    def amvm(self, x, **kw):
        xd = torch.tensor(x, device="cuda")
        yd = torch.full((3 * len(self.P),), np.nan, dtype=torch.float64, device="cuda")
        info = binding.amvm(self.H, xd, yd, **kw)
        torch.cuda.synchronize()
        return yd.cpu().numpy(), info


_cache = {}


def small():
    if "s" not in _cache:
        _cache["s"] = PCase(3, 700, 32, 24, 1e-8)
    return _cache["s"]


def test_point_blocks_match_oracle():
    """The same partition, near-field entries to 1e-12 and every admissible
    block's ACA with the same rank and U V^T to 1e-12."""
    c = small()
    np.testing.assert_array_equal(c.perm, c.Ho.rperm)
    np.testing.assert_array_equal(c.adm, c.Ho.adm)
    np.testing.assert_array_equal(c.near, c.Ho.near)
    rng = np.random.default_rng(0)
    for b in sorted(rng.choice(len(c.near), 80, replace=False).tolist()):
        m, n = c.rows(b, c.near)
        g = c.H.near_block(b, m, n)
        o = c.Ho.near_block(b)
        scale = np.abs(o[0]).max()
        assert np.abs(g - o[1:]).max() <= 1e-12 * scale, b
    worst = 0.0
    for b in range(len(c.adm)):
        m, n = c.rows(b, c.adm)
        for kern in range(7):
            Uo, Vo = c.Ho.factors(b, kern)
            Ug, Vg = c.H.factors(b, kern, m, n)
            assert Ug.shape[1] == Uo.shape[1], (b, kern)
            if Uo.shape[1] == 0:
                continue
            So = Uo @ Vo.T
            worst = max(worst, np.linalg.norm(Ug @ Vg.T - So) / np.linalg.norm(So))
    assert worst <= 1e-12


def test_eval_points_matches_oracle_and_definition():
    """u = ~V_h t for three densities: the oracle's H-matrix product to 1e-12
    and the operator's definition (Kelvin's tensor entry by entry) to the ACA
    accuracy; repeated calls agree bitwise."""
    c = small()
    x = inputs.uniform_rhs(3 * c.M, 0, nrhs=3)
    u = c.eval(x)
    uo = c.Ho.matvec(E, NU, x)
    ud = oracle.points_matvec(c.V, c.T, E, NU, c.P, x)
    for r in range(3):
        assert _rel(u[r], uo[r]) <= 1e-12, r
        assert _rel(u[r], ud[r]) <= 1e-7, r
    assert np.array_equal(c.eval(x), u)


def test_eval_points_fp32_form():
    """The FP32 form (FP32 copies of the same factors and near field, FP32
    arithmetic): refused before hm_pack(HM_FP32), then within 1e-5 of the
    FP64 form, deterministic; the 16-bit forms do not exist for ~V_h."""
    c = small()
    x = inputs.uniform_rhs(3 * c.M, 6, nrhs=2)
    with pytest.raises(binding.HMError):
        c.eval(x, "fp32")
    with pytest.raises(binding.HMError):
        c.H.pack("bf16")
    c.H.pack("fp32")
    u32 = c.eval(x, "fp32")
    u64 = c.eval(x)
    for r in range(2):
        assert _rel(u32[r], u64[r]) <= 1e-5, r
    assert np.array_equal(c.eval(x, "fp32"), u32)
    st = c.H.stats()
    assert st.bytes_form[1] * 2 == st.bytes_form[0] > 0


def test_eval_points_with_more_than_32_crosses():
    """Blocks whose ACA sequences exceed one chunk of crosses (level 4, leaf
    64, eps 1e-12: ranks up to about 60) are applied chunk by chunk."""
    c = PCase(4, 2000, 64, 64, 1e-12, r_out=0.97, seed=4)
    assert c.H.stats().rank_max[1] > 32
    x = inputs.uniform_rhs(3 * c.M, 1)[0]
    u = c.eval(x)[0]
    uo = c.Ho.matvec(E, NU, x)[0]
    assert _rel(u, uo) <= 1e-12
    c.H.pack("fp32")
    assert _rel(c.eval(x, "fp32")[0], uo) <= 1e-5


@pytest.mark.parametrize("npts,leaf_pts,r_in,r_out", [(1, 8, 0.0, 0.5), (333, 7, 0.0, 0.9),
                                                      (257, 32, 1.2, 3.0), (96, 336, 0.0, 0.8)])
def test_eval_points_ragged_and_exterior(npts, leaf_pts, r_in, r_out):
    """One point, a ragged count with many small leaves, points outside the
    surface, and one leaf holding every point: the product equals the
    oracle's H-matrix product and the definition."""
    c = PCase(2, npts, 16, leaf_pts, 1e-8, r_in=r_in, r_out=r_out, seed=5)
    x = inputs.uniform_rhs(3 * c.M, 2)[0]
    u = c.eval(x)[0]
    assert _rel(u, c.Ho.matvec(E, NU, x)[0]) <= 1e-12
    assert _rel(u, oracle.points_matvec(c.V, c.T, E, NU, c.P, x)[0]) <= 1e-6


def test_eval_points_closed_form_and_material():
    """A uniform density on the level-4 icosphere gives the interior value
    (1+nu)(5-6nu)R/(3E(1-nu)) f at every interior point to the mesh's O(h^2)
    accuracy; hm_set_material rescales it to the new (E, nu)."""
    c = PCase(4, 300, 64, 32, 1e-6, r_out=0.8, seed=6, oracle_h=False)
    f = np.array([0.2, -0.7, 0.4])
    x = np.tile(f, c.M)
    u = c.eval(x)[0].reshape(-1, 3)
    exact = (1 + NU) * (5 - 6 * NU) / (3 * E * (1 - NU)) * f
    assert np.abs(u - exact).max() <= 1.5e-3 * np.abs(exact).max()
    c.H.pack("fp32")
    c.H.set_material(2.0, 0.25)
    u2 = c.eval(x)[0].reshape(-1, 3)
    exact2 = (1.25) * (5 - 1.5) / (3 * 2.0 * 0.75) * f
    assert np.abs(u2 - exact2).max() <= 1.5e-3 * np.abs(exact2).max()
    u3 = c.eval(x, "fp32")[0].reshape(-1, 3)
    assert np.abs(u3 - exact2).max() <= 1.5e-3 * np.abs(exact2).max()


def test_point_amvm_follows_the_oracle():
    """Algorithm 2 on ~V_h: the GPU follows the oracle's refinement, meets
    the Doerfler condition at every step and the relative stop; with eps = 0
    it returns the exact product of hm_eval_points."""
    c = small()
    x = inputs.uniform_rhs(3 * c.M, 3)[0]
    y, info = c.amvm(x, theta=0.7, eps=1e-5)
    ro = oracle.amvm(c.Ho, E, NU, x, theta=0.7, eps=1e-5)
    assert info["csp"] == ro["csp"]
    assert abs(info["iterations"] - ro["iterations"]) <= 1
    for k in range(min(3, len(info["gamma"]), len(ro["gamma"]))):
        assert abs(info["gamma"][k] - ro["gamma"][k]) <= 1e-6 * ro["gamma"][k], k
    assert np.linalg.norm(y - ro["b"]) <= 4e-5 * np.linalg.norm(ro["b"])
    g, rest = info["gamma"], info["gamma_rest"]
    for k in range(len(rest)):
        assert g[k] - rest[k] >= 0.7 * g[k] * (1 - 1e-12), k
    assert g[-1] <= 1e-5 * info["bhat_norm"]
    yf, inf = c.amvm(x, theta=0.7, eps=0.0)
    assert inf["crosses_used"] == inf["crosses_full"]
    ue = c.eval(x)[0]
    assert np.linalg.norm(yf - ue) <= 1e-13 * np.linalg.norm(ue)


def test_point_operator_with_aca_on_demand():
    """Assembled without ACA (HM_DEFER_ACA): hm_eval_points refuses, and the
    adaptive product with ACA on demand gives the same bits as on the fully
    assembled operator."""
    c = small()
    d = PCase(3, 700, 32, 24, 1e-8, defer_aca=True, oracle_h=False)
    x = inputs.uniform_rhs(3 * c.M, 4)[0]
    with pytest.raises(binding.HMError):
        d.eval(x)
    y1, i1 = c.amvm(x, theta=0.7, eps=1e-5, on_demand=True)
    y2, i2 = d.amvm(x, theta=0.7, eps=1e-5, on_demand=True)
    assert np.array_equal(y1, y2)
    assert i1["crosses_full"] == i2["crosses_full"]
    y3, i3 = c.amvm(x, theta=0.7, eps=1e-5)
    assert np.array_equal(y1, y3)


def test_point_operator_refuses_square_calls():
    c = small()
    x = torch.zeros(3 * c.M, dtype=torch.float64, device="cuda")
    with pytest.raises(binding.HMError):
        binding.hmatvec(c.H, x, torch.zeros_like(x))
    with pytest.raises(binding.HMError):
        c.H.pack("fp16")
    with pytest.raises(binding.HMError):
        binding.solve(c.H, x, torch.zeros_like(x))
    sq = binding.aca_assemble(c.tree, E, NU, 1e-4, max_rhs=1)
    with pytest.raises(binding.HMError):
        binding.eval_points(sq, x, torch.zeros_like(x))


def test_level6_points_sampled():
    """Level-6 icosphere (81,920 triangles) and 65,536 points in the ball of
    radius 0.95 at eps 1e-4: sampled points against the operator's
    definition (the oracle computes those rows one by one)."""
    c = PCase(6, 65536, 64, 64, 1e-4, seed=7, oracle_h=False)
    x = inputs.uniform_rhs(3 * c.M, 5)[0]
    u = c.eval(x)[0].reshape(-1, 3)
    idx = inputs.sample_rows(len(c.P), 48, 8)
    uo = oracle.points_matvec(c.V, c.T, E, NU, c.P[idx], x)[0].reshape(-1, 3)
    assert np.linalg.norm(u[idx] - uo) <= 1e-4 * np.linalg.norm(uo)
    c.H.pack("fp32")
    u32 = c.eval(x, "fp32")[0].reshape(-1, 3)
    assert np.linalg.norm(u32[idx] - uo) <= 1e-4 * np.linalg.norm(uo)
    assert np.linalg.norm(u32 - u) <= 1e-5 * np.linalg.norm(u)
