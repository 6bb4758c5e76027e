"""GPU adaptive matrix-vector multiplication (Algorithm 2, ``hm_amvm``)
against the oracle's Algorithm 2 on the same mesh and partition, and against
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


def run(H, x, **kw):
    xd = torch.tensor(x, device="cuda")
    yd = torch.full_like(xd, np.nan)
    info = binding.amvm(H, xd, yd, **kw)
    torch.cuda.synchronize()
    return yd.cpu().numpy(), info


def product(H, x):
    xd = torch.tensor(x, device="cuda")
    yd = torch.empty_like(xd)
    binding.hmatvec(H, xd, yd, "fp64")
    torch.cuda.synchronize()
    return yd.cpu().numpy()


@pytest.mark.parametrize("seed,theta", [(0, 0.7), (3, 0.5)])
def test_amvm_follows_the_oracle(seed, theta):
    """Same mesh, partition and ACA epsilon: the GPU and the oracle take the
    same refinement steps.  The GPU finds step 3's stopping row by bisection
    over the sorted rows; the oracle scans them one by one.  The two rows
    coincide when the remaining error gamma_k(P_k) does not grow along the
    scan, which is asserted on the oracle's scan for these inputs.  Then
    every step marks the same blocks (the same final ranks and marked
    counts), the estimators agree to the rounding of the two ACA runs, and
    the products agree to 1e-12."""
    V, T, tree, H, Ho = case()
    x = inputs.uniform_rhs(3 * Ho.M, seed)[0]
    ro = oracle.amvm(Ho, E, NU, x, theta=theta, eps=1e-6, record_scan=True)
    for k, sc in enumerate(ro["scans"]):
        assert np.all(np.diff(sc) <= 0), k  # the case the bisection must reproduce
    y, info = run(H, x, theta=theta, eps=1e-6)
    assert info["csp"] == ro["csp"]
    assert info["iterations"] == ro["iterations"]
    assert info["marked_total"] == sum(ro["marked"])
    np.testing.assert_array_equal(info["block_ranks"], ro["r"])
    assert len(info["gamma"]) == len(ro["gamma"])
    for k, (g, go) in enumerate(zip(info["gamma"], ro["gamma"])):
        assert abs(g - go) <= 1e-10 * go, k
    for k, (g, go) in enumerate(zip(info["gamma_rest"], ro["gamma_rest"])):
        assert abs(g - go) <= 1e-10 * ro["gamma"][k], k
    assert np.linalg.norm(y - ro["b"]) <= 1e-12 * np.linalg.norm(ro["b"])
    yf = Ho.matvec(E, NU, x)[0]
    assert np.linalg.norm(y - yf) <= 1e-5 * np.linalg.norm(yf)


def test_amvm_full_refinement_is_the_fp64_product():
    """With eps = 0 every block is refined until its ACA sequence is used up:
    the result is the FP64 H-matrix product (independent kernels, same
    factors) to rounding."""
    V, T, tree, H, Ho = case()
    x = inputs.uniform_rhs(3 * Ho.M, 2)[0]
    y, info = run(H, x, theta=0.7, eps=0.0)
    assert info["crosses_used"] == info["crosses_full"]
    assert info["gamma"][-1] == 0.0
    yp = product(H, x)
    assert np.linalg.norm(y - yp) <= 1e-13 * np.linalg.norm(yp)


@pytest.mark.parametrize("theta", [0.3, 0.7, 0.9])
def test_amvm_doerfler_condition_and_stop(theta):
    """Every refinement meets gamma_k - gamma_k(P_k) >= theta gamma_k, and the
    loop ends with gamma <= eps ||A^_k x|| using fewer crosses than the ACA."""
    V, T, tree, H, Ho = case()
    x = inputs.uniform_rhs(3 * Ho.M, 3)[0]
    eps = 1e-6
    y, info = run(H, x, theta=theta, eps=eps)
    g, rest = info["gamma"], info["gamma_rest"]
    assert len(rest) == info["iterations"] == len(g) - 1
    for k in range(len(rest)):
        assert g[k] - rest[k] >= theta * g[k] * (1 - 1e-12), k
    assert g[-1] <= eps * info["bhat_norm"]
    assert info["crosses_used"] < info["crosses_full"]


def test_amvm_zero_vector_and_zero_region():
    """x = 0 needs no refinement and gives 0; with x zero on the second half
    of the cluster order, the blocks whose columns lie there keep the
    starting rank (Section 3)."""
    V, T, tree, H, Ho = case()
    y, info = run(H, np.zeros(3 * Ho.M))
    assert info["iterations"] == 0 and not np.any(y)
    assert np.all(info["block_ranks"] == 2)
    x = inputs.uniform_rhs(3 * Ho.M, 7)[0]
    root = int(np.argmax(Ho.nodes[:, 1] - Ho.nodes[:, 0]))
    lo, hi = Ho.nodes[root, 0], Ho.nodes[root, 1]
    half = (lo + hi) // 2
    xz = x.reshape(-1, 3).copy()
    xz[Ho.perm[half:hi]] = 0.0
    y, info = run(H, xz.reshape(-1), theta=0.7, eps=1e-6)
    rng = Ho.ranges(Ho.adm)
    inside = (rng[:, 2] >= half) & (rng[:, 3] <= hi)
    assert inside.any()
    assert np.all(info["block_ranks"][inside] == 2)
    assert np.any(info["block_ranks"][~inside] > 2)


def test_amvm_argument_errors():
    V, T, tree, H, Ho = case()
    x = torch.zeros(3 * Ho.M, dtype=torch.float64, device="cuda")
    y = torch.zeros_like(x)
    with pytest.raises(binding.HMError):
        binding.amvm(H, x, y, theta=1.5)
    with pytest.raises(binding.HMError):
        binding.amvm(H, x, y, eps=-1.0)
    with pytest.raises(binding.HMError):
        binding.amvm(H, x, y, r0=64)
    Hc = binding.aca_assemble(tree, E, NU, 1e-4, max_rhs=1)
    Hc.pack("fp16")
    Hc.compact()
    with pytest.raises(binding.HMError):
        binding.amvm(Hc, x, y)


def test_aca_on_demand_repeats_the_assembled_crosses():
    """Algorithm 1 run on demand (every block-kernel to r0 + look crosses,
    refined ones further) computes the same first crosses as the full
    assembly, so the adaptive product is bitwise the same, with fewer crosses
    computed than the full ACA holds."""
    V, T, tree, H, Ho = case()
    x = inputs.uniform_rhs(3 * Ho.M, 8)[0]
    y1, i1 = run(H, x, theta=0.7, eps=1e-6)
    y2, i2 = run(H, x, theta=0.7, eps=1e-6, on_demand=True)
    assert np.array_equal(y1, y2)
    assert i1["iterations"] == i2["iterations"] and i1["gamma"] == i2["gamma"]
    assert np.array_equal(i1["block_ranks"], i2["block_ranks"])
    assert i2["crosses_used"] == i1["crosses_used"]
    assert i2["crosses_full"] < i1["crosses_full"]


def test_deferred_aca_matrix_serves_the_adaptive_product_only():
    """HM_DEFER_ACA: no ACA at assembly; the matrix cannot be packed, the
    prefix mode is refused, and the on-demand adaptive product gives the same
    bits as on the fully assembled matrix."""
    V, T, tree, H, Ho = case()
    Hd = binding.aca_assemble(tree, E, NU, 1e-8, max_rhs=1, defer_aca=True)
    with pytest.raises(binding.HMError):
        Hd.pack("fp16")
    x = inputs.uniform_rhs(3 * Ho.M, 9)[0]
    xd = torch.tensor(x, device="cuda")
    with pytest.raises(binding.HMError):
        binding.amvm(Hd, xd, torch.empty_like(xd))
    y1, i1 = run(H, x, theta=0.7, eps=1e-6, on_demand=True)
    y2, i2 = run(Hd, x, theta=0.7, eps=1e-6, on_demand=True)
    assert np.array_equal(y1, y2)
    assert i1["crosses_full"] == i2["crosses_full"]
