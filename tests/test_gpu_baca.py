"""GPU block-adaptive ACA for the single layer (Algorithm 3, ``hm_baca``)
against the oracle's Algorithm 3 on the same mesh and partition, and against
what the algorithm guarantees by construction."""
import numpy as np
import pytest

import oracle
from paper_2205_04752_gb300 import binding, inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

E, NU = 1.0, 0.3
_cache = {}


def case():
    if "c" not in _cache:
        V, T = inputs.icosphere(3)
        tree = binding.build_cluster_tree(V, T, 32, 0.8)
        H = binding.aca_assemble(tree, E, NU, 1e-8, max_rhs=1)
        Ho = oracle.HMatrix(V, T, 32, 0.8, 1e-8)
        Ho.assemble()
        _cache["c"] = (V, T, tree, H, Ho)
    return _cache["c"]


def rhs(M, seed=2):
    return np.tile([1.0, 0.0, 0.0], M) + 0.1 * inputs.uniform_rhs(3 * M, seed)[0]


def run(H, b, **kw):
    bd = torch.tensor(b, device="cuda")
    td = torch.full_like(bd, np.nan)
    info = binding.baca(H, bd, td, **kw)
    torch.cuda.synchronize()
    return td.cpu().numpy(), info


def product(H, x):
    xd = torch.tensor(x, device="cuda")
    yd = torch.empty_like(xd)
    binding.hmatvec(H, xd, yd, "fp64")
    torch.cuda.synchronize()
    return yd.cpu().numpy()


def test_baca_follows_the_oracle():
    """Same partition and ACA: the GPU takes the oracle's steps (same
    estimator sequence to the rounding of the two GMRES runs, same marked
    counts) and ends at the same solution."""
    V, T, tree, H, Ho = case()
    b = rhs(Ho.M)
    kw = dict(theta=0.8, alpha=10.0, eps=1e-4, r0=2, look=2)
    t, info = run(H, b, **kw)
    ro = oracle.baca(Ho, E, NU, b, **kw)
    assert info["steps"] == ro["steps"]
    for k in range(info["steps"] + 1):
        assert abs(info["history"][k]["E"] - ro["E"][k]) <= 1e-6 * ro["E"][k], k
        assert info["history"][k]["iterations"] == ro["iterations"][k], k
    for k in range(info["steps"]):
        assert info["history"][k]["marked"] == ro["marked"][k], k
    assert np.linalg.norm(t - ro["x"]) <= 1e-6 * np.linalg.norm(ro["x"])
    assert np.array_equal(np.minimum(info["block_ranks"][:, None], ro["full_ranks"]), ro["ranks"])


def test_baca_conditions_and_stop():
    """Every step meets Eq. (solvCond) (or the residual floor); the loop ends
    at E <= eps ||b|| with fewer crosses than the assembled ACA; the returned
    residual is the FP64 product's with A_k."""
    V, T, tree, H, Ho = case()
    b = rhs(Ho.M, 5)
    alpha, eps = 10.0, 1e-4
    t, info = run(H, b, theta=0.8, alpha=alpha, eps=eps, r0=2, look=2)
    for k, st in enumerate(info["history"]):
        assert st["residual"] <= alpha * st["lookahead"] * (1 + 1e-12) or \
            st["residual"] <= 1e-13 * info["b_norm"], k
    assert info["E"] <= eps * info["b_norm"]
    assert info["crosses_used"] < info["crosses_full"]
    assert info["steps"] >= 2
    # reliability against the full H-matrix (c_sat <= 1/2)
    y = product(H, t)
    assert np.linalg.norm(b - y) <= (1 + alpha * 1.5) / 0.5 * info["history"][-1]["lookahead"]


def test_baca_full_refinement_solves_the_full_system():
    """eps = 0: every block is refined to its whole ACA sequence, and the last
    solve runs to the residual floor, so t solves the FP64 H-matrix system."""
    V, T, tree, H, Ho = case()
    b = rhs(Ho.M, 7)
    t, info = run(H, b, theta=0.8, alpha=10.0, eps=0.0, r0=2, look=4)
    assert info["crosses_used"] == info["crosses_full"]
    assert info["E"] == 0.0
    y = product(H, t)
    assert np.linalg.norm(b - y) <= 1e-11 * np.linalg.norm(b)


def test_baca_with_aca_on_demand():
    """HM_BACA_ACA_ON_DEMAND: Algorithm 1 runs only to the crosses the
    refinement reaches (resumed tasks); the solve is bitwise the prefix mode's,
    on the fully assembled matrix and on one assembled without ACA, with fewer
    crosses computed than the full ACA holds."""
    V, T, tree, H, Ho = case()
    b = rhs(Ho.M, 3)
    kw = dict(theta=0.8, alpha=10.0, eps=1e-4, r0=2, look=2)
    t1, i1 = run(H, b, **kw)
    t2, i2 = run(H, b, on_demand=True, **kw)
    assert np.array_equal(t1, t2)
    assert i1["steps"] == i2["steps"] and np.array_equal(i1["block_ranks"], i2["block_ranks"])
    assert i2["crosses_used"] == i1["crosses_used"]
    assert i2["crosses_full"] < i1["crosses_full"]
    Hd = binding.aca_assemble(tree, E, NU, 1e-8, max_rhs=1, defer_aca=True)
    t3, i3 = run(Hd, b, on_demand=True, **kw)
    assert np.array_equal(t1, t3)
    assert i3["crosses_full"] == i2["crosses_full"]


def test_baca_zero_rhs_and_errors():
    V, T, tree, H, Ho = case()
    t, info = run(H, np.zeros(3 * Ho.M))
    assert info["steps"] == 0 and not np.any(t) and info["E"] == 0.0
    x = torch.zeros(3 * Ho.M, dtype=torch.float64, device="cuda")
    for kw in (dict(theta=1.2), dict(alpha=-1.0), dict(eps=-1.0), dict(look=40), dict(restart=500)):
        with pytest.raises(binding.HMError):
            binding.baca(H, x, torch.zeros_like(x), **kw)
    Hd = binding.aca_assemble(tree, E, NU, 1e-8, max_rhs=1, defer_aca=True)
    with pytest.raises(binding.HMError):
        binding.baca(Hd, x, torch.zeros_like(x))
