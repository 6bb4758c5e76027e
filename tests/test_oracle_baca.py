"""Pins of the oracle's block-adaptive ACA for the single layer (Algorithm 3,
branch (iii), Section 5) against what the algorithm and the mathematics fix
(CPU only)."""
import numpy as np
import pytest

import oracle
from paper_2205_04752_gb300 import inputs

E, NU = 1.0, 0.3
_cache = {}


def _case():
    if "h" not in _cache:
        V, T = inputs.icosphere(3)
        Ho = oracle.HMatrix(V, T, 32, 0.8, 1e-8)
        Ho.assemble()
        _cache["h"] = Ho
    return _cache["h"]


def _rhs(Ho, seed=2):
    return np.tile([1.0, 0.0, 0.0], Ho.M) + 0.1 * inputs.uniform_rhs(3 * Ho.M, seed)[0]


def test_zero_rhs_needs_nothing():
    """b = 0: x = 0 solves every A_k, the estimator is 0 and nothing is refined."""
    Ho = _case()
    res = oracle.baca(Ho, E, NU, np.zeros(3 * Ho.M))
    assert res["steps"] == 0 and res["E"] == [0.0] and not np.any(res["x"])
    assert np.all(res["ranks"] == np.minimum(8, res["full_ranks"]))


def test_unreachable_eps_refines_to_the_full_solve():
    """With eps = 0 every block is refined until its ACA sequence is used up
    (E = 0), and the last solve runs to the residual floor: x solves the full
    H-matrix system, checked with the oracle's C H-matrix product (an
    independent code path from the dense A_k)."""
    Ho = _case()
    b = _rhs(Ho)
    res = oracle.baca(Ho, E, NU, b, eps=0.0, r0=2, look=4)
    assert np.all(res["ranks"] == res["full_ranks"])
    assert res["E"][-1] == 0.0
    y = Ho.matvec(E, NU, res["x"])[0]
    assert np.linalg.norm(b - y) <= 1e-11 * np.linalg.norm(b)


@pytest.mark.parametrize("theta", [0.5, 0.8])
def test_each_step_meets_the_solve_and_marking_conditions(theta):
    """Step 2: ||b - A_k x_k|| <= alpha ||(A_k - A^_k) x_k|| (Eq. (solvCond));
    step 3: the marked blocks carry E_k(M_k) >= theta E_k and no smaller
    set of blocks does (the marked ones are the largest parts, and dropping
    the smallest of them breaks the condition); the loop ends at E <= eps ||b||."""
    Ho = _case()
    b = _rhs(Ho)
    alpha, eps = 10.0, 1e-4
    res = oracle.baca(Ho, E, NU, b, theta=theta, alpha=alpha, eps=eps, r0=2, look=2)
    for k in range(len(res["E"])):
        assert res["residual"][k] <= alpha * res["lookahead"][k] * (1 + 1e-12) or \
            res["residual"][k] <= 1e-13 * np.linalg.norm(b), k
    for k, Mk in enumerate(res["marked_sets"]):
        bn2 = res["parts"][k]
        Ek2 = bn2.sum()
        assert bn2[Mk].sum() >= theta ** 2 * Ek2 * (1 - 1e-12)
        assert bn2[Mk[:-1]].sum() < theta ** 2 * Ek2
        rest = np.delete(bn2, Mk)
        assert rest.size == 0 or rest.max() <= bn2[Mk].min()
    assert res["E"][-1] <= eps * np.linalg.norm(b)
    assert res["steps"] >= 2


def test_estimator_bounds_the_error_of_the_solve():
    """Reliability (the estimate after Algorithm 3): with the fully refined
    H-matrix standing in for A, ||b - A x_k|| stays within a small multiple of
    ||(A_k - A^_k) x_k|| (1 + alpha (1 + c_sat)) / (1 - c_sat) with c_sat <= 1/2,
    and far fewer crosses than the full ACA are used."""
    Ho = _case()
    b = _rhs(Ho, 5)
    res = oracle.baca(Ho, E, NU, b, theta=0.8, alpha=10.0, eps=1e-4, r0=2, look=2)
    y = Ho.matvec(E, NU, res["x"])[0]
    assert np.linalg.norm(b - y) <= (1 + 10.0 * 1.5) / 0.5 * res["lookahead"][-1]
    assert res["ranks"].sum() < 0.5 * res["full_ranks"].sum()
