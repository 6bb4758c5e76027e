"""Pins of the oracle's evaluation operator ~V_h (Section 5, Eq. (vector_eq): the
displacement u_h(x) = sum_j int_{tau_j} S(x - y) ds_y t_j at points x of the
domain) against what the mathematics fixes (CPU only).

Closed forms (derived from Kelvin's tensor of Section 4.1, not printed in the
paper): for a uniform density f on the sphere |y| = R,
  int 1/|x-y| dS = 4 pi R            (|x| < R),  4 pi R^2 / |x|          (|x| > R),
  int d_k d_l / |d|^3 dS = (4 pi R / 3) delta_kl                          (|x| < R),
                         = 4 pi R^2 [x^_k x^_l / rho - R^2 (3 x^_k x^_l - delta_kl) / (3 rho^3)]
                                                                          (rho = |x| > R),
with d = x - y (from d_k d_l / r^3 = delta_kl / r - d_k d_l r and the sphere
means of 1/r and r).  Inside, u = (1+nu)(5-6nu) R / (3E(1-nu)) f, constant.
On the icosphere the discrete values approach these at O(h^2): the error
shrinks about 4x per subdivision level."""
import numpy as np
import pytest

import oracle
from paper_2205_04752_gb300 import inputs

E, NU = 1.0, 0.3


def _closed_form(P, f, E=E, nu=NU, R=1.0):
    out = []
    for x in np.atleast_2d(P):
        rho = float(np.linalg.norm(x))
        if rho < R:
            I0, I = 4 * np.pi * R, (4 * np.pi * R / 3) * np.eye(3)
        else:
            xh = x / rho
            xx = np.outer(xh, xh)
            I0 = 4 * np.pi * R * R / rho
            I = 4 * np.pi * R * R * (xx / rho - (R * R / 3) * (3 * xx - np.eye(3)) / rho ** 3)
        S = (1 / (8 * np.pi * E)) * ((1 + nu) / (1 - nu)) * ((3 - 4 * nu) * I0 * np.eye(3) + I)
        out.append(S @ f)
    return np.array(out)


def _errors(P, f):
    ex = _closed_form(P, f)
    errs = []
    for lev in (2, 3, 4):
        V, T = inputs.icosphere(lev)
        y = oracle.points_matvec(V, T, E, NU, P, np.tile(f, T.shape[0]))[0].reshape(-1, 3)
        errs.append(np.abs(y - ex).max() / np.abs(ex).max())
    return errs


def test_interior_value_is_the_closed_form():
    """Inside the sphere the displacement of a uniform density is constant,
    (1+nu)(5-6nu)R/(3E(1-nu)) f = 1.98095... f at E = 1, nu = 0.3; the values at
    interior points (the centre included) converge to it at O(h^2)."""
    assert abs((1 + NU) * (5 - 6 * NU) / (3 * E * (1 - NU)) - 1.9809523809523) < 1e-12
    P = np.array([[0.0, 0.0, 0.0], [0.3, -0.2, 0.1], [0.5, 0.0, 0.0], [-0.1, 0.6, -0.3]])
    f = np.array([1.0, 0.0, 0.0])
    e2, e3, e4 = _errors(P, f)
    assert 3.5 < e2 / e3 < 4.6 and 3.5 < e3 / e4 < 4.6, (e2, e3, e4)
    assert e4 < 1.5e-3


def test_exterior_value_is_the_closed_form():
    """Outside the sphere the field of a uniform density is anisotropic (the
    x^ x^ terms): a general f at points 1.5 .. 5 radii away converges to the
    closed form at O(h^2); a dropped or transposed term of V_kl fails it."""
    rng = np.random.default_rng(1)
    d = rng.normal(size=(4, 3))
    d /= np.linalg.norm(d, axis=1)[:, None]
    P = d * np.array([1.5, 2.0, 3.0, 5.0])[:, None]
    f = np.array([0.3, -0.5, 0.8])
    e2, e3, e4 = _errors(P, f)
    assert 3.5 < e2 / e3 < 4.6 and 3.5 < e3 / e4 < 4.6, (e2, e3, e4)
    assert e4 < 2e-3


def test_point_entries_satisfy_the_kernel_identities():
    """At points off the surface: V_11 + V_22 + V_33 = V_Delta (trace of
    d d^T / r^3 is 1/r) and Kelvin's tensor integrated directly equals
    c1 delta V_Delta + c2 V_kl (Eq. (Vh) with the prefactor 1/(4 pi))."""
    V, T = inputs.icosphere(2)
    P = inputs.shell_points(6, 0.2, 1.6, 11)
    S = oracle.scalar_points(V, T, P)
    assert np.abs(S[1] + S[4] + S[6] - S[0]).max() <= 1e-14 * np.abs(S[0]).max()
    c1, c2 = oracle.lame_coefficients(E, NU)
    kab = [[1, 2, 3], [2, 4, 5], [3, 5, 6]]
    for r in range(P.shape[0]):
        for j in (0, 17, 200):
            K = oracle.kelvin_entry(P[r], V, T[j], False, E, NU)
            ref = np.array([[c1 * (a == b) * S[0, r, j] + c2 * S[kab[a][b], r, j] for b in range(3)]
                            for a in range(3)])
            assert np.abs(K - ref).max() <= 1e-13 * np.abs(ref).max()
            assert np.array_equal(K, K.T)


def _rect(eps=1e-4, np_=700, leaf_points=24, eta=0.8, seed=3, level=3):
    V, T = inputs.icosphere(level)
    P = inputs.ball_points(np_, 0.95, seed)
    Ho = oracle.HMatrix(V, T, 32, eta, eps, points=P, leaf_points=leaf_points)
    return V, T, P, Ho


def test_point_tree_and_rectangular_partition():
    """The point tree (same split rule, boxes of the points) and the
    partition of points x triangles: a permutation, leaves of at most b_min
    points, every box the exact box of its points, sons splitting their
    father at floor(n/2), blocks tiling the Mr x M rectangle exactly, every
    admissible block satisfying Eq. (adm) on the boxes and every near block a
    pair of leaves."""
    V, T, P, Ho = _rect()
    assert np.array_equal(np.sort(Ho.rperm), np.arange(Ho.Mr))
    for n in range(Ho.nrnodes):
        lo, hi, s0, s1, _ = Ho.rnodes[n]
        pts = P[Ho.rperm[lo:hi]]
        assert np.array_equal(Ho.rboxes[n, :3], pts.min(0)) and np.array_equal(Ho.rboxes[n, 3:], pts.max(0))
        if s0 < 0:
            assert hi - lo <= 24
        else:
            assert Ho.rnodes[s0, 0] == lo and Ho.rnodes[s0, 1] == lo + (hi - lo) // 2
            assert Ho.rnodes[s1, 0] == Ho.rnodes[s0, 1] and Ho.rnodes[s1, 1] == hi
            assert hi - lo > 24
    cover = np.zeros((Ho.Mr, Ho.M), dtype=np.int32)
    for (t, s) in np.concatenate([Ho.adm, Ho.near]):
        cover[Ho.rnodes[t, 0]:Ho.rnodes[t, 1], Ho.nodes[s, 0]:Ho.nodes[s, 1]] += 1
    assert np.all(cover == 1)

    def diam2(b):
        return float(np.sum((b[3:] - b[:3]) ** 2))

    def dist2(a, b):
        g = np.maximum(np.maximum(a[:3] - b[3:], b[:3] - a[3:]), 0.0)
        return float(np.sum(g * g))

    for (t, s) in Ho.adm:
        a, b = Ho.rboxes[t], Ho.boxes[s]
        assert min(diam2(a), diam2(b)) < 0.8 ** 2 * dist2(a, b)
    for (t, s) in Ho.near:
        assert Ho.rnodes[t, 2] < 0 and Ho.nodes[s, 2] < 0


def test_point_aca_meets_its_bound_on_every_block():
    """Algorithm 1 on the blocks of ~V_h: ||A_b - U V^T||_F <= 2 eps ||A_b||_F
    on every admissible block and kernel (the stop test estimates the
    remainder), A_b computed entry by entry."""
    V, T, P, Ho = _rect(eps=1e-4, np_=300)
    Ho.assemble()
    worst = 0.0
    for b in range(Ho.nadm):
        for k in range(7):
            A = Ho.dense_block(b, k)
            U, W = Ho.factors(b, k)
            nA = np.linalg.norm(A)
            if nA == 0.0:
                continue
            worst = max(worst, np.linalg.norm(A - U @ W.T) / nA)
    assert worst <= 2e-4


@pytest.mark.parametrize("eps,tol", [(1e-4, 1e-4), (1e-8, 1e-7)])
def test_point_hmatrix_product_approaches_the_definition(eps, tol):
    """The H-matrix of ~V_h applied to a density equals the operator applied
    by its definition (Kelvin's tensor, entry by entry) within the ACA
    accuracy."""
    V, T, P, Ho = _rect(eps=eps)
    Ho.assemble()
    x = inputs.uniform_rhs(3 * Ho.M, 7)[0]
    y = Ho.matvec(E, NU, x)[0]
    yd = oracle.points_matvec(V, T, E, NU, P, x)[0]
    assert np.linalg.norm(y - yd) <= tol * np.linalg.norm(yd)


def test_point_near_field_alone_is_the_definition():
    """With eta so small that no block is admissible, the H-matrix is its
    near field: the product equals the definition to rounding."""
    V, T, P, Ho = _rect(eps=1e-4, np_=200, eta=1e-9)
    assert Ho.nadm == 0
    Ho.assemble()
    x = inputs.uniform_rhs(3 * Ho.M, 8)[0]
    y = Ho.matvec(E, NU, x)[0]
    yd = oracle.points_matvec(V, T, E, NU, P, x)[0]
    assert np.linalg.norm(y - yd) <= 1e-13 * np.linalg.norm(yd)


def test_point_amvm_refines_to_the_product_and_stops_at_eps():
    """Algorithm 2 on ~V_h (Section 5, Eq. (vector_eq) applies the adaptive product to the
    evaluation): with eps = 0 it refines every block to its whole ACA
    sequence and returns the H-matrix product; with eps = 1e-3 it stops with
    gamma_k <= eps ||b^_k|| and an error of that size."""
    V, T, P, Ho = _rect(eps=1e-8)
    Ho.assemble()
    x = inputs.uniform_rhs(3 * Ho.M, 9)[0]
    y = Ho.matvec(E, NU, x)[0]
    full = oracle.amvm(Ho, E, NU, x, eps=0.0)
    assert np.all(full["ranks"] == full["full_ranks"])
    assert np.linalg.norm(full["b"] - y) <= 1e-13 * np.linalg.norm(y)
    res = oracle.amvm(Ho, E, NU, x, eps=1e-3)
    assert res["gamma"][-1] <= 1e-3 * np.linalg.norm(res["b_hat"])
    assert np.linalg.norm(res["b"] - y) <= 3e-3 * np.linalg.norm(y)
    assert res["iterations"] >= 1
