"""hm_solve: GMRES on a packed product form with FP64-residual iterative
refinement.  The residual is checked with the oracle's own H-matrix product
(independent of the CUDA path), and the solution of the sphere problem with
constant data against the closed form of the single layer of a uniform
density on a sphere."""
import numpy as np
import pytest

import oracle
from paper_2205_04752_gb300 import binding, inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

E, NU = 1.0, 0.3


@pytest.fixture(scope="module")
def c1():
    V, T = inputs.icosphere(3)
    tree = binding.build_cluster_tree(V, T, 32, 0.8)
    H = binding.aca_assemble(tree, E, NU, 1e-4, max_rhs=2)
    for form in ("fp16", "bf16", "i16", "fp32"):
        H.pack(form)
    Ho = oracle.HMatrix(V, T, 32, 0.8, 1e-4)
    Ho.assemble()
    return V, T, H, Ho


@pytest.mark.parametrize("form", ["fp16", "bf16", "i16", "fp32", "fp64"])
def test_solve_reaches_fp64_tolerance(c1, form):
    V, T, H, Ho = c1
    g = inputs.uniform_rhs(3 * len(T), 2)[0]
    gd = torch.tensor(g, device="cuda")
    td = torch.zeros_like(gd)
    info = binding.solve(H, gd, td, tol=1e-8, inner_form=form)
    t = td.cpu().numpy()
    r = g - Ho.matvec(E, NU, t)[0]
    assert np.linalg.norm(r) <= 1.5e-8 * np.linalg.norm(g)
    assert info["rel_residual"] <= 1e-8 and info["converged"]
    assert info["refinements"] >= 1


def test_solve_sphere_constant_data(c1):
    """Constant data on the sphere: the single layer of a uniform density f
    is (1+nu)(5-6nu)R/(3E(1-nu)) f on the surface, so the density solving
    V t = e_1 is nearly constant, e_1 / 1.98095 (discretisation error ~1%)."""
    V, T, H, Ho = c1
    g = np.tile([1.0, 0.0, 0.0], len(T))
    gd = torch.tensor(g, device="cuda")
    td = torch.zeros_like(gd)
    binding.solve(H, gd, td, tol=1e-8, inner_form="fp16")
    t = td.cpu().numpy().reshape(-1, 3)
    ref = 3 * E * (1 - NU) / ((1 + NU) * (5 - 6 * NU))
    assert abs(np.mean(t[:, 0]) / ref - 1) < 1e-2
    assert np.abs(t[:, 1:]).max() < 2e-2 * ref


def test_solve_reports_nonconvergence(c1):
    V, T, H, Ho = c1
    g = inputs.uniform_rhs(3 * len(T), 3)[0]
    gd = torch.tensor(g, device="cuda")
    td = torch.zeros_like(gd)
    info = binding.solve(H, gd, td, tol=1e-12, inner_form="fp16", max_inner=3, raise_on_fail=False)
    assert not info["converged"] and info["iterations"] <= 3


def test_solve_cube_dirichlet_bf16_inner_form():
    """The cube solve of the benchmark at reduced size: the surface of
    [-1,1]^3 with 16 x 16 squares per face (3,072 triangles, 9,216 dofs),
    leaf 64, g = (1,0,0) + U[-1,1] per dof (seed 2), GMRES(50) on the BF16
    form inside refinement with the FP64 residual to 1e-8.  The residual is
    checked with the oracle's own H-matrix product (independent code)."""
    V, T = inputs.cube_surface(16)
    M = len(T)
    tree = binding.build_cluster_tree(V, T, 64, 0.8)
    H = binding.aca_assemble(tree, E, NU, 1e-4, max_rhs=1)
    H.pack("bf16")
    g = np.tile([1.0, 0.0, 0.0], M) + inputs.uniform_rhs(3 * M, 2)[0]
    gd = torch.tensor(g, device="cuda")
    td = torch.zeros_like(gd)
    info = binding.solve(H, gd, td, tol=1e-8, inner_form="bf16", restart=50)
    assert info["converged"] and info["rel_residual"] <= 1e-8
    Ho = oracle.HMatrix(V, T, 64, 0.8, 1e-4)
    Ho.assemble()
    r = g - Ho.matvec(E, NU, td.cpu().numpy())[0]
    assert np.linalg.norm(r) <= 1.5e-8 * np.linalg.norm(g)
