"""Pins of the oracle's adaptive matrix-vector multiplication (Algorithm 2,
Section 3) against what the paper and the mathematics fix (CPU only)."""
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


def test_sparsity_constant_counts_blocks_per_cluster():
    """c_sp (Section 2.1): the most blocks of P sharing a row or a column
    cluster, counted here by brute force over the partition."""
    Ho = _case()
    worst = 0
    for nd in range(Ho.nnodes):
        worst = max(worst, int(np.sum(Ho.adm[:, 0] == nd)) + int(np.sum(Ho.near[:, 0] == nd)),
                    int(np.sum(Ho.adm[:, 1] == nd)) + int(np.sum(Ho.near[:, 1] == nd)))
    assert oracle.sparsity_constant(Ho) == worst


def test_zero_vector_needs_no_refinement():
    """x = 0: b_0 = b^_0 = 0, gamma_0 = 0, and the iteration stops at once
    without approximating any block further (Section 3: the adaptive approach
    detects that no accuracy is needed)."""
    Ho = _case()
    res = oracle.amvm(Ho, E, NU, np.zeros(3 * Ho.M))
    assert res["iterations"] == 0
    assert res["gamma"] == [0.0]
    assert not np.any(res["b"])
    assert np.all(res["ranks"] == np.minimum(2, res["full_ranks"]))


def test_full_refinement_gives_the_aca_product():
    """With an unreachable epsilon every block is refined until its ACA
    sequence is used up; b_k then equals the H-matrix product A x computed by
    the oracle's C code (same factors, independent summation)."""
    Ho = _case()
    x = inputs.uniform_rhs(3 * Ho.M, 4)[0]
    res = oracle.amvm(Ho, E, NU, x, theta=0.7, eps=0.0)
    assert np.all(res["ranks"] == res["full_ranks"])
    y = Ho.matvec(E, NU, x)[0]
    assert np.linalg.norm(res["b"] - y) <= 1e-13 * np.linalg.norm(y)
    assert res["gamma"][-1] == 0.0


@pytest.mark.parametrize("theta", [0.3, 0.7, 0.9])
def test_marking_meets_the_doerfler_condition(theta):
    """Step 3: the marked set satisfies gamma_k - gamma_k(P_k) >= theta gamma_k
    in every iteration (the Remark after Algorithm 2 guarantees it even when
    every row has been visited), and the estimator shrinks from one step to
    the next."""
    Ho = _case()
    x = inputs.uniform_rhs(3 * Ho.M, 5)[0]
    res = oracle.amvm(Ho, E, NU, x, theta=theta, eps=1e-6)
    g, rest = res["gamma"], res["gamma_rest"]
    assert len(rest) == len(g) - 1 == res["iterations"]
    for k in range(len(rest)):
        assert g[k] - rest[k] >= theta * g[k] * (1 - 1e-12), (k, g[k], rest[k])
    assert g[-1] < g[0]


def test_estimator_tracks_the_error_and_stops_at_epsilon():
    """gamma_k = ||b_k - b^_k|| is, for the look-ahead approximation, a
    reliable and efficient estimate of ||b_k - b|| (Lemma after Algorithm 2,
    with b the H-matrix product at full ACA rank): the ratio stays within
    [1/(1+c), 1/(1-c)] for the observed saturation c = ||b^_k - b|| / ||b_k -
    b||, and the loop ends with gamma <= eps ||b^||, using fewer crosses than
    the full ACA."""
    Ho = _case()
    x = inputs.uniform_rhs(3 * Ho.M, 6)[0]
    eps = 1e-6
    res = oracle.amvm(Ho, E, NU, x, theta=0.7, eps=eps)
    y = Ho.matvec(E, NU, x)[0]
    err = np.linalg.norm(res["b"] - y)
    c = np.linalg.norm(res["b_hat"] - y) / err
    assert c < 1.0
    gam = res["gamma"][-1]
    assert err / (1 + c) <= gam * (1 + 1e-12) and gam <= err / (1 - c) * (1 + 1e-12)
    assert gam <= eps * np.linalg.norm(res["b_hat"])
    assert err <= 10 * eps * np.linalg.norm(y)
    assert res["ranks"].sum() < res["full_ranks"].sum()


def test_blocks_over_a_zero_region_are_not_refined():
    """x zero on a cluster (Section 3: clusters of zero entries need no
    approximation): every block whose column cluster lies in the zero region
    keeps its starting rank."""
    Ho = _case()
    x = inputs.uniform_rhs(3 * Ho.M, 7)[0]
    root = int(np.argmax(Ho.nodes[:, 1] - Ho.nodes[:, 0]))
    lo, hi = Ho.nodes[root, 0], Ho.nodes[root, 1]
    half = (lo + hi) // 2
    zero_pos = Ho.perm[half:hi]                       # the second half in cluster order
    xz = x.reshape(-1, 3).copy()
    xz[zero_pos] = 0.0
    res = oracle.amvm(Ho, E, NU, xz.reshape(-1), theta=0.7, eps=1e-6)
    rng = Ho.ranges(Ho.adm)
    inside = (rng[:, 2] >= half) & (rng[:, 3] <= hi)
    assert inside.any()
    start = np.minimum(2, res["full_ranks"])
    assert np.all(res["ranks"][inside] == start[inside])
    assert np.any(res["ranks"][~inside] > start[~inside])
