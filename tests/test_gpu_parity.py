"""GPU parity: the CUDA path (through the C ABI) against the FP64 CPU oracle
on the same seeded inputs.

Tolerances: FP64 kernels against the oracle's same blocks 1e-12 (relative);
the H-matrix product against the dense product 1e-4 (relative 2-norm); packed
product forms against the FP64 form as stated per form.
"""
import numpy as np
import pytest

import oracle
from paper_2205_04752_gb300 import binding, inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

E, NU = 1.0, 0.3


def _rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


class Case:
    def __init__(self, V, T, leaf, eta=0.8, eps=1e-4, max_rhs=8):
        self.V, self.T, self.leaf, self.eta, self.eps = V, T, leaf, eta, eps
        self.M = len(T)
        self.tree = binding.build_cluster_tree(V, T, leaf, eta)
        self.H = binding.aca_assemble(self.tree, E, NU, eps, max_rhs=max_rhs)
        self.Ho = oracle.HMatrix(V, T, leaf, eta, eps)
        self.perm, self.nodes, self.adm, self.near = self.tree.export()

    def matvec(self, x, form="fp64"):
        xd = torch.tensor(np.ascontiguousarray(np.atleast_2d(x)), device="cuda")
        yd = torch.full_like(xd, np.nan)
        binding.hmatvec(self.H, xd, yd, form)
        torch.cuda.synchronize()
        return yd.cpu().numpy()

    def size(self, node):
        return int(self.nodes[node, 1] - self.nodes[node, 0])


_cache = {}


def c1():
    if "c1" not in _cache:
        V, T = inputs.icosphere(3)
        _cache["c1"] = Case(V, T, 32)
        _cache["c1"].Ho.assemble()
    return _cache["c1"]


def test_near_field_entries_match_oracle():
    c = c1()
    rng = np.random.default_rng(0)
    ids = sorted(set(rng.choice(c.Ho.nnear, 60, replace=False).tolist()) |
                 {b for b in range(c.Ho.nnear) if c.near[b, 0] == c.near[b, 1]})
    for b in ids:
        m, n = c.size(c.near[b, 0]), c.size(c.near[b, 1])
        g = c.H.near_block(b, m, n)
        o = c.Ho.near_block(b)
        scale = np.abs(o[0]).max()
        assert np.abs(g - o[1:]).max() <= 1e-12 * scale, b
        assert np.abs(g[0] + g[3] + g[5] - o[0]).max() <= 1e-12 * scale, b


def test_aca_factors_match_oracle_blocks():
    """Every admissible block and scalar kernel of C1: same rank, and the
    reconstructions U V^T agree to 1e-12 of the block's norm."""
    c = c1()
    worst = 0.0
    for b in range(c.Ho.nadm):
        m, n = c.size(c.adm[b, 0]), c.size(c.adm[b, 1])
        for kern in range(7):
            Uo, Vo = c.Ho.factors(b, kern)
            Ug, Vg = c.H.factors(b, kern, m, n)
            assert Ug.shape[1] == Uo.shape[1], (b, kern)
            So = Uo @ Vo.T
            d = np.linalg.norm(Ug @ Vg.T - So) / np.linalg.norm(So)
            worst = max(worst, d)
    assert worst <= 1e-12


def test_hmatvec_fp64_matches_oracle_and_dense():
    c = c1()
    x = inputs.uniform_rhs(3 * c.M, 0, nrhs=3)
    y = c.matvec(x)
    yo = c.Ho.matvec(E, NU, x)
    for r in range(3):
        assert _rel(y[r], yo[r]) <= 1e-12
    A = oracle.kelvin_dense(c.V, c.T, E, NU)
    yd = oracle.dense_matvec(A, x)
    for r in range(3):
        assert _rel(y[r], yd[r]) <= 1e-4


# Relative error of each packed form against the FP64 form at C1, bounded at
# about twice what the forms reach there (measured on GB300 with these
# inputs: FP32 3.2e-7, BF16 3.3e-4, FP16 4.1e-5, INT16 9.5e-6); the errors
# follow each storage type's rounding of the factors (unit roundoff 2^-24,
# 2^-8, 2^-11, and 2^-16 of each column's largest entry; INT16 also stores
# the near field outside the leaves' diagonal blocks in INT16)
C1_BOUNDS = {"fp32": 6e-7, "bf16": 7e-4, "fp16": 8e-5, "i16": 2e-5}


@pytest.mark.parametrize("form", ["fp32", "bf16", "fp16", "i16"])
def test_packed_forms_against_fp64_form(form):
    c = c1()
    c.H.pack(form)
    x = inputs.uniform_rhs(3 * c.M, 1, nrhs=2)
    y64 = c.matvec(x)
    y = c.matvec(x, form)
    errs = [_rel(y[r], y64[r]) for r in range(2)]
    print(f"C1 {form}: {max(errs):.3e}")
    assert max(errs) <= C1_BOUNDS[form]


def test_deterministic_and_multi_rhs_consistent():
    c = c1()
    x = inputs.uniform_rhs(3 * c.M, 7, nrhs=5)
    y1 = c.matvec(x)
    y2 = c.matvec(x)
    np.testing.assert_array_equal(y1, y2)
    for r in (0, 4):
        ys = c.matvec(x[r])
        np.testing.assert_allclose(ys[0], y1[r], rtol=0, atol=1e-14 * np.abs(y1[r]).max())


@pytest.mark.parametrize("form", ["fp16", "fp32", "bf16", "i16", "fp64"])
def test_multi_rhs_launches_match_single_vector_products(form):
    """Several right-hand sides share one pass over the factors (interleaved
    vectors, up to 32 per launch): each row agrees with the single-vector
    product to the rounding of the accumulation type, and repeats are bitwise
    equal."""
    if "c32" not in _cache:
        V, T = inputs.icosphere(3)
        _cache["c32"] = Case(V, T, 32, max_rhs=32)
    c = _cache["c32"]
    if form != "fp64":
        c.H.pack(form)
    tol = 1e-13 if form == "fp64" else 2e-6
    # 16-bit forms: 32 = two tensor-core launches of 16; 20 = one of 16 and
    # one of 4 vectors with the leaf product on the CUDA cores; 2 and 7: the
    # forward pass on the tensor cores, the leaf product on the CUDA cores
    for nrhs in (2, 7, 20, 32):
        x = inputs.uniform_rhs(3 * c.M, 40 + nrhs, nrhs=nrhs)
        y = c.matvec(x, form)
        np.testing.assert_array_equal(y, c.matvec(x, form))
        for r in sorted({0, nrhs // 2, nrhs - 1}):
            ys = c.matvec(x[r], form)[0]
            assert _rel(y[r], ys) <= tol, (nrhs, r)


@pytest.mark.parametrize("form,nrhs", [("fp16", 16), ("bf16", 16), ("fp16", 3), ("bf16", 6), ("fp16", 11),
                                       ("i16", 16), ("i16", 9), ("i16", 6)])
def test_tensor_core_far_field_scales_exactly(form, nrhs):
    """The tensor-core forward pass (2-16 vectors; INT16 V split into two
    exact FP16 operands) and far field (9-16) scale x and W by a power of
    two chosen from max|x| of each vector:
    scaling x by 2^40 or 2^-40 scales y exactly, a zero vector gives zero,
    and vectors of very different size share a launch.  3, 6 and 11 vectors
    cover the lane quarters holding four, two and one copy of the vectors;
    9 is the fewest that take the far field to the tensor cores."""
    if "c32" not in _cache:
        V, T = inputs.icosphere(3)
        _cache["c32"] = Case(V, T, 32, max_rhs=32)
    c = _cache["c32"]
    c.H.pack(form)
    x = inputs.uniform_rhs(3 * c.M, 91, nrhs=nrhs)
    y = c.matvec(x, form)
    for k in (40, -40):
        f = 2.0 ** k
        np.testing.assert_array_equal(c.matvec(x * f, form), y * f)
    xm = x.copy()
    xm[1] = 0.0
    xm[nrhs - 1] *= 2.0 ** 30
    ym = c.matvec(xm, form)
    assert np.all(ym[1] == 0.0)
    for r in sorted({0, nrhs // 2, nrhs - 1} - {1}):
        ref = c.matvec(xm[r], form)[0]
        assert _rel(ym[r], ref) <= 2e-6, r


@pytest.mark.parametrize("nrhs", [9, 16])
def test_tensor_core_far_field_large_leaves(nrhs):
    """Leaves of more than 64 rows (leaf size 128 on the level-4 icosphere:
    up to 80): a far stage of 48 segments then holds more U than half the
    stage region, so the INT16 split goes into the staged-vector region after
    the A build (leaves of up to 64 rows split beside U, on a second warp).
    Every vector of the launch matches its own single-vector product within
    1e-5 (both accumulate the same INT16 product in FP32 and the far field's
    W carries the 2^-22 of its hi/lo split; the 80-row leaves sum more
    segments per leaf than the 32-row ones of the 2e-6 tests: 2.5e-6
    measured), and scaling x by 2^40 scales y exactly."""
    if "c128" not in _cache:
        V, T = inputs.icosphere(4)
        _cache["c128"] = Case(V, T, 128, max_rhs=16)
    c = _cache["c128"]
    assert max(c.size(n) for n in range(len(c.nodes)) if c.nodes[n, 2] < 0) > 64
    c.H.pack("i16")
    x = inputs.uniform_rhs(3 * c.M, 77, nrhs=nrhs)
    y = c.matvec(x, "i16")
    assert np.all(np.isfinite(y))
    np.testing.assert_array_equal(c.matvec(x * 2.0 ** 40, "i16"), y * 2.0 ** 40)
    for r in range(nrhs):
        ys = c.matvec(x[r], "i16")[0]
        assert _rel(y[r], ys) <= 1e-5, r


def test_multi_rhs_split_into_several_launches():
    """Leaves of 300 rows in FP64 leave room for only 4 vectors per launch:
    10 right-hand sides run as launches of 4, 4 and 2; every row matches the
    oracle's H-matrix product."""
    V, T = inputs.ellipsoid(10, 0.6, 1.7, 1.1)
    c = Case(V, T, 336, max_rhs=10)
    c.Ho.assemble()
    x = inputs.uniform_rhs(3 * c.M, 9, nrhs=10)
    y = c.matvec(x)
    yo = c.Ho.matvec(E, NU, x)
    for r in range(10):
        assert _rel(y[r], yo[r]) <= 1e-12, r


def test_host_entry_point_equals_device_entry_point():
    c = c1()
    x = inputs.uniform_rhs(3 * c.M, 3, nrhs=2)
    y = np.zeros_like(x)
    binding.hmatvec_host(c.H, x, y, "fp64")
    np.testing.assert_array_equal(y, c.matvec(x))


def test_set_material():
    c = c1()
    E2, nu2 = 2.5, 0.41
    x = inputs.uniform_rhs(3 * c.M, 9)
    c.H.set_material(E2, nu2)
    try:
        y = c.matvec(x)
    finally:
        c.H.set_material(E, NU)
    yo = c.Ho.matvec(E2, nu2, x)
    assert _rel(y[0], yo[0]) <= 1e-12


@pytest.mark.parametrize("mesh,leaf", [("ico0", 3), ("ico1", 7), ("ico2", 336), ("cube4", 12),
                                       ("ell", 20), ("ell10", 336)])
def test_small_and_ragged_meshes(mesh, leaf):
    """Tiny meshes, leaves of ragged size, a single dense leaf (leaf >= M), a
    cube surface whose planar faces make some kernels vanish identically
    (rank 0 blocks), an ellipsoid, and leaves of 300 rows near the largest
    leaf the library takes (336): one FP64 near-field column per stage."""
    if mesh.startswith("ico"):
        V, T = inputs.icosphere(int(mesh[3:]))
    elif mesh == "cube4":
        V, T = inputs.cube_surface(4)
    elif mesh == "ell10":
        V, T = inputs.ellipsoid(10, 0.6, 1.7, 1.1)
    else:
        V, T = inputs.ellipsoid(7, 0.6, 1.7, 1.1)
    c = Case(V, T, leaf, max_rhs=2)
    c.Ho.assemble()
    x = inputs.uniform_rhs(3 * c.M, 2, nrhs=2)
    y = c.matvec(x)
    yo = c.Ho.matvec(E, NU, x)
    A = oracle.kelvin_dense(V, T, E, NU)
    yd = oracle.dense_matvec(A, x)
    for r in range(2):
        assert _rel(y[r], yo[r]) <= 1e-12
        assert _rel(y[r], yd[r]) <= 1e-4
    if mesh == "cube4" and c.Ho.nadm:
        assert (c.Ho.ranks() == 0).any()


def l6():
    """The benchmark workload: level-6 icosphere (81,920 triangles, 245,760
    dofs), leaf 64, eta 0.8, eps 1e-4, assembled with room for 32 vectors
    per call as bench.py does."""
    if "l6" not in _cache:
        V, T = inputs.icosphere(6)
        tree = binding.build_cluster_tree(V, T, 64, 0.8)
        H = binding.aca_assemble(tree, E, NU, 1e-4, max_rhs=32)
        _cache["l6"] = (V, T, tree, H)
    return _cache["l6"]


def _l6_products(H, M, form, nrhs, seed):
    x = torch.tensor(inputs.uniform_rhs(3 * M, seed, nrhs=nrhs), device="cuda")
    y64 = torch.empty_like(x)
    y = torch.full_like(x, float("nan"))
    binding.hmatvec(H, x, y64, "fp64")
    binding.hmatvec(H, x, y, form)
    torch.cuda.synchronize()
    d = torch.linalg.norm(y - y64, dim=1) / torch.linalg.norm(y64, dim=1)
    return d.cpu().numpy()


# E_mixed = ||y_form - y_fp64|| / ||y_fp64|| over the full 245,760-dof vector
# of every right-hand side, at the benchmark workload, one vector and 32 in
# one call.  INT16 (the form the benchmark times) is gated at the metric's
# 1e-4.  FP16 does not meet it at this size (8.2e-5 for seed 0 alone but up to
# 1.21e-4 over 32 vectors): it is kept, bounded at its own measured level, as
# the form of the tensor-core kernels.  BF16 keeps three fewer mantissa bits
# than FP16 (unit roundoff 2^-8 against 2^-11), about 8x FP16's error, and
# serves as an inner form of the refined solve.  FP32 is gated far below
# (measured on GB300 over 32 vectors: INT16 1.28e-5, FP16 1.21e-4, BF16 9.7e-4,
# FP32 1.7e-6).
L6_BOUNDS = {"i16": 1e-4, "fp16": 1.5e-4, "bf16": 1.5e-3, "fp32": 3e-6}


@pytest.mark.slow
@pytest.mark.parametrize("form", ["i16", "fp16", "bf16", "fp32"])
def test_level6_mixed_form_error_against_fp64_form(form):
    V, T, tree, H = l6()
    H.pack(form)
    M = len(T)
    e1 = _l6_products(H, M, form, 1, 0)
    e32 = _l6_products(H, M, form, 32, 0)
    print(f"E_mixed {form}: R=1 {e1.max():.3e}, R=32 max {e32.max():.3e} mean {e32.mean():.3e}")
    assert e1.max() <= L6_BOUNDS[form]
    assert e32.max() <= L6_BOUNDS[form]


@pytest.mark.slow
def test_level6_sampled_rows_and_blocks():
    """The benchmark workload (level-6 icosphere, 245,760 dofs, leaf 64,
    eta 0.8, eps 1e-4) in the configuration the benchmark times: the FP64
    product against exact rows of the dense product at 384 sampled triangles
    (relative error <= 1e-4), and ACA parity on 60 sampled admissible
    blocks."""
    V, T, tree, H = l6()
    M = len(T)
    x = inputs.uniform_rhs(3 * M, 0)
    xd = torch.tensor(x, device="cuda")
    y64 = torch.empty_like(xd)
    binding.hmatvec(H, xd[0], y64[0], "fp64")
    torch.cuda.synchronize()
    y64 = y64.cpu().numpy()
    rows = inputs.sample_rows(M, 384, 11)
    yr = oracle.kelvin_rows_matvec(V, T, E, NU, rows, x)[0]
    dofs = (3 * rows[:, None] + np.arange(3)[None, :]).ravel()
    assert _rel(y64[0][dofs], yr) <= 1e-4
    # ACA parity on sampled blocks
    Ho = oracle.HMatrix(V, T, 64, 0.8, 1e-4)
    perm, nodes, adm, near = tree.export()
    rng = np.random.default_rng(4)
    sizes = nodes[adm[:, 0], 1] - nodes[adm[:, 0], 0]
    pick = list(rng.choice(len(adm), 50, replace=False)) + list(np.argsort(-sizes)[:10])
    Ho.assemble(adm_ids=pick, near_ids=[])
    for b in pick:
        m = int(nodes[adm[b, 0], 1] - nodes[adm[b, 0], 0])
        n = int(nodes[adm[b, 1], 1] - nodes[adm[b, 1], 0])
        for kern in range(7):
            Uo, Vo = Ho.factors(b, kern)
            Ug, Vg = H.factors(b, kern, m, n)
            assert Ug.shape[1] == Uo.shape[1], (b, kern)
            So = Uo @ Vo.T
            assert np.linalg.norm(Ug @ Vg.T - So) <= 1e-12 * np.linalg.norm(So), (b, kern)
    _cache.pop("l6", None)  # release the level-6 matrix (tens of GB) for the later tests
