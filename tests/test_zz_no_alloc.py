"""The allocation-free product hm_matvec_noalloc, for callers that cannot
allocate device memory when they need a product (a fixed memory budget, or a
host framework that owns all allocation).  It is checked through the C ABI
against hm_matvec on two calls in a row, in the tolerance of the other
parity tests.  This file is collected last so that a run that stops at the
first failure has run every other test before it."""
import ctypes

import numpy as np
import pytest

from paper_2205_04752_gb300 import binding, inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _call(lib, H, x, y, form):
    nrhs = 1 if x.dim() == 1 else x.shape[0]
    ld = x.shape[-1] if nrhs == 1 else x.stride(0)
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    return lib.hm_matvec_noalloc(H._h, ctypes.c_void_p(x.data_ptr()), ctypes.c_void_p(y.data_ptr()),
                                 nrhs, ld, binding.FORMS[form], stream)


def test_noalloc_matches_matvec_on_two_calls():
    lib = binding.load()
    V, T = inputs.icosphere(3)
    M = len(T)
    tree = binding.build_cluster_tree(V, T, 32, 0.8)
    H = binding.aca_assemble(tree, 1.0, 0.3, 1e-4, max_rhs=32)
    H.pack("fp32")
    for form, tol in (("fp64", 1e-12), ("fp32", 1e-12)):
        for seed in (0, 1):  # two calls in a row; different data each time
            x = torch.tensor(inputs.uniform_rhs(3 * M, seed, nrhs=2), device="cuda")
            y_ref = torch.empty_like(x)
            y = torch.full_like(x, float("nan"))
            binding.hmatvec(H, x, y_ref, form)
            assert _call(lib, H, x, y, form) == binding.HM_OK, lib.hm_last_error()
            torch.cuda.synchronize()
            a, b = y.cpu().numpy(), y_ref.cpu().numpy()
            for r in range(2):
                assert np.linalg.norm(a[r] - b[r]) <= tol * np.linalg.norm(b[r])


def test_noalloc_rejects_oversized_products():
    lib = binding.load()
    V, T = inputs.icosphere(3)
    tree = binding.build_cluster_tree(V, T, 32, 0.8)
    H = binding.aca_assemble(tree, 1.0, 0.3, 1e-4, max_rhs=32)
    x = torch.zeros((32, 3 * len(T)), dtype=torch.float64, device="cuda")
    y = torch.zeros_like(x)
    rc = _call(lib, H, x, y, "fp64")
    assert rc == binding.HM_EINVAL
    assert b"static scratch" in lib.hm_last_error()
