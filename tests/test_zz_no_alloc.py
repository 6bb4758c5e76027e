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


def _check(lib, H, M, form, nrhs, seed, tol):
    x = torch.tensor(inputs.uniform_rhs(3 * M, seed, nrhs=nrhs), device="cuda")
    if nrhs == 1:
        x = x[0]
    y_ref = torch.empty_like(x)
    y = torch.full_like(x, float("nan"))
    binding.hmatvec(H, x, y_ref, form)
    assert _call(lib, H, x, y, form) == binding.HM_OK, lib.hm_last_error()
    torch.cuda.synchronize()
    a, b = np.atleast_2d(y.cpu().numpy()), np.atleast_2d(y_ref.cpu().numpy())
    for r in range(nrhs):
        assert np.linalg.norm(a[r] - b[r]) <= tol * np.linalg.norm(b[r]), (form, nrhs, r)


_mats = {}


def _c1():
    if "c1" not in _mats:
        V, T = inputs.icosphere(3)
        tree = binding.build_cluster_tree(V, T, 32, 0.8)
        H = binding.aca_assemble(tree, 1.0, 0.3, 1e-4, max_rhs=32)
        _mats["c1"] = (H, len(T))
    return _mats["c1"]


def test_noalloc_matches_matvec_on_two_calls():
    lib = binding.load()
    H, M = _c1()
    H.pack("fp32")
    for form, tol in (("fp64", 1e-12), ("fp32", 1e-12)):
        for seed in (0, 1):  # two calls in a row; different data each time
            _check(lib, H, M, form, 2, seed, tol)


@pytest.mark.parametrize("form", ["fp16", "bf16", "i16"])
def test_noalloc_16bit_forms_one_and_sixteen_vectors(form):
    """The 16-bit forms: one vector (the CUDA-core forward pass) and 16
    vectors (FP16 / BF16: the tensor-core forward pass and far field, whose
    per-vector max|x| words live beside the counters in the static array;
    INT16: the CUDA-core kernels), two calls in a row each.  The kernels are those of hm_matvec, so the results agree to
    the same 1e-12 as the other forms."""
    lib = binding.load()
    H, M = _c1()
    H.pack(form)
    for nrhs in (1, 16):
        for seed in (3, 4):
            _check(lib, H, M, form, nrhs, seed, 1e-12)


def test_noalloc_smaller_matrix_after_a_larger_one():
    """A product of a smaller matrix after one that filled more of the static
    array: nothing of the earlier call's contents leaks into the result."""
    lib = binding.load()
    H, M = _c1()
    H.pack("fp16")
    _check(lib, H, M, "fp16", 16, 5, 1e-12)
    V, T = inputs.icosphere(2)
    tree = binding.build_cluster_tree(V, T, 16, 0.8)
    Hs = binding.aca_assemble(tree, 1.0, 0.3, 1e-4, max_rhs=4)
    Hs.pack("fp16")
    for form in ("fp16", "fp64"):
        _check(lib, Hs, len(T), form, 3, 6, 1e-12)


def test_noalloc_rejects_oversized_products():
    lib = binding.load()
    H, M = _c1()
    x = torch.zeros((32, 3 * M), dtype=torch.float64, device="cuda")
    y = torch.zeros_like(x)
    rc = _call(lib, H, x, y, "fp64")
    assert rc == binding.HM_EINVAL
    assert b"static scratch" in lib.hm_last_error()
