"""Batched product over several resident matrices (``hm_batch``): every
member's part of the batched product equals that member's own product
bitwise, under every schedule, with and without CUDA-graph replay, and the
FP64 batch matches the oracle's H-matrix product of each member (1e-12).
"""
import numpy as np
import pytest

import oracle
from paper_2205_04752_gb300 import binding, inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

# (mesh, leaf, E, nu): sizes, leaves and materials all differ
MEMBERS = [("ico2", 16, 1.0, 0.3), ("ell6", 20, 2.0, 0.25), ("ico3", 32, 1.0, 0.45),
           ("cube4", 12, 0.5, 0.2), ("ico1", 7, 1.0, 0.3)]


def _mesh(name):
    if name.startswith("ico"):
        return inputs.icosphere(int(name[3:]))
    if name == "cube4":
        return inputs.cube_surface(4)
    return inputs.ellipsoid(6, 0.7, 1.6, 1.1)


_cache = {}


def members():
    if "m" not in _cache:
        out = []
        for name, leaf, E, nu in MEMBERS:
            V, T = _mesh(name)
            tr = binding.build_cluster_tree(V, T, leaf, 0.8)
            H = binding.aca_assemble(tr, E, nu, 1e-4, max_rhs=4)
            for form in ("fp16", "fp32", "i16"):
                H.pack(form)
            out.append((name, V, T, leaf, E, nu, tr, H))
        _cache["m"] = out
    return _cache["m"]


def _alone(H, x, form):
    y = torch.empty_like(x)
    binding.hmatvec(H, x.contiguous(), y, form)
    return y


@pytest.mark.parametrize("form,nrhs", [("fp64", 3), ("fp16", 3), ("fp32", 3), ("fp16", 1), ("fp32", 1), ("i16", 1),
                                       ("i16", 3)])
def test_batch_equals_each_member_alone_bitwise(form, nrhs):
    """One launch per phase over all members gives each member's own bits:
    the FP16 form with one vector (forward pass from the tiles on the CUDA
    cores) and with three (on the tensor cores), the INT16 form (CUDA cores),
    FP32 and FP64 (row-major)."""
    ms = members()
    B = binding.Batch([m[-1] for m in ms], form, max_rhs=3)
    assert B.ndof == sum(3 * len(m[2]) for m in ms)
    x = torch.tensor(inputs.uniform_rhs(B.ndof, 11, nrhs=nrhs), device="cuda")
    y = torch.full_like(x, np.nan)
    B.matvec(x, y)
    torch.cuda.synchronize()
    B.check()
    for i, m in enumerate(ms):
        a, b = int(B.offsets[i]), int(B.offsets[i + 1])
        ya = _alone(m[-1], x[:, a:b], form)
        torch.cuda.synchronize()
        assert torch.equal(y[:, a:b], ya), (m[0], form)


@pytest.mark.parametrize("nrhs", [1, 2])
def test_every_schedule_and_graph_replay_give_the_same_bits(nrhs):
    ms = members()
    B = binding.Batch([m[-1] for m in ms], "fp16", max_rhs=2)
    x = torch.tensor(inputs.uniform_rhs(B.ndof, 5, nrhs=nrhs), device="cuda")
    ref = torch.empty_like(x)
    B.set_schedule(0, 0, 0)
    B.matvec(x, ref)
    for ctas in (0, 1):
        for order in (0, 1):
            for fork in (0, 1):
                B.set_schedule(ctas, order, fork)
                y = torch.full_like(x, np.nan)
                B.matvec(x, y)
                yg = torch.full_like(x, np.nan)
                B.matvec(x, yg, graph=True)
                B.matvec(x, yg, graph=True)  # replay of the captured graph
                torch.cuda.synchronize()
                assert torch.equal(y, ref), (ctas, order, fork)
                assert torch.equal(yg, ref), (ctas, order, fork)
    # the replayed graph reads x at call time: new values, same buffers
    B.set_schedule(0, 0, 1)
    yg = torch.empty_like(x)
    B.matvec(x, yg, graph=True)
    x.mul_(-0.5)
    B.matvec(x, yg, graph=True)
    y = torch.empty_like(x)
    B.matvec(x, y)
    torch.cuda.synchronize()
    assert torch.equal(yg, y)
    B.check()


def test_autotune_keeps_a_valid_schedule_and_the_result():
    ms = members()
    B = binding.Batch([m[-1] for m in ms], "fp16", max_rhs=2)
    x = torch.tensor(inputs.uniform_rhs(B.ndof, 8, nrhs=2), device="cuda")
    y0 = torch.empty_like(x)
    B.matvec(x, y0)
    sc, t = B.autotune(nrhs=2, reps=2)
    assert t > 0.0
    assert sc == B.schedule()
    assert sc["work_order"] in (0, 1) and sc["fork_forward"] in (0, 1)
    y1 = torch.empty_like(x)
    B.matvec(x, y1, graph=True)
    torch.cuda.synchronize()
    assert torch.equal(y0, y1)


def test_fp64_batch_matches_the_oracle_per_member():
    ms = members()
    B = binding.Batch([m[-1] for m in ms], "fp64", max_rhs=1)
    # padded rows: ld > ndof
    xb = torch.tensor(np.pad(inputs.uniform_rhs(B.ndof, 3, nrhs=1), ((0, 0), (0, 5))), device="cuda")
    x = xb[:, :B.ndof]
    yb = torch.full_like(xb, np.nan)
    y = yb[:, :B.ndof]
    # one row: pass 1-D views
    B.matvec(x[0], y[0])
    torch.cuda.synchronize()
    assert torch.isnan(yb[0, B.ndof:]).all()
    xn, yn = x.cpu().numpy()[0], y.cpu().numpy()[0]
    for i, (name, V, T, leaf, E, nu, tr, H) in enumerate(ms):
        a, b = int(B.offsets[i]), int(B.offsets[i + 1])
        Ho = oracle.HMatrix(V, T, leaf, 0.8, 1e-4)
        Ho.assemble()
        yo = Ho.matvec(E, nu, xn[a:b][None, :])[0]
        rel = np.linalg.norm(yn[a:b] - yo) / np.linalg.norm(yo)
        assert rel <= 1e-12, (name, rel)


def test_batch_argument_errors():
    ms = members()
    mats = [m[-1] for m in ms]
    with pytest.raises(binding.HMError):
        binding.Batch(mats + [mats[0]], "fp16")  # a member twice
    with pytest.raises(binding.HMError):
        binding.Batch(mats, "bf16")  # not packed
    B = binding.Batch(mats[:2], "fp64", max_rhs=1)
    x = torch.zeros((2, B.ndof), dtype=torch.float64, device="cuda")
    with pytest.raises(binding.HMError):
        B.matvec(x, torch.zeros_like(x))  # nrhs above max_rhs
    with pytest.raises(binding.HMError):
        B.set_schedule(work_order=2)


def test_compact_keeps_the_packed_form_and_releases_fp64():
    V, T = inputs.icosphere(3)
    tr = binding.build_cluster_tree(V, T, 32, 0.8)
    H = binding.aca_assemble(tr, 1.0, 0.3, 1e-4, max_rhs=1)
    H.pack("fp16")
    x = torch.tensor(inputs.uniform_rhs(3 * len(T), 4), device="cuda")[0]
    y0 = _alone(H, x, "fp16")
    torch.cuda.synchronize()
    before = H.footprint()
    H.compact()
    after = H.footprint()
    assert after < 0.6 * before, (before, after)
    y1 = _alone(H, x, "fp16")
    torch.cuda.synchronize()
    assert torch.equal(y0, y1)
    with pytest.raises(binding.HMError):
        _alone(H, x, "fp64")
    with pytest.raises(binding.HMError):
        H.pack("fp32")
    with pytest.raises(binding.HMError):
        H.near_block(0, 1, 1)
    with pytest.raises(binding.HMError):
        binding.solve(H, x, torch.zeros_like(x))
    # a compacted matrix still joins a batch in its packed form
    B = binding.Batch([H], "fp16", max_rhs=1)
    y2 = torch.empty_like(x)
    B.matvec(x, y2)
    torch.cuda.synchronize()
    assert torch.equal(y0, y2)


def test_deferred_fp64_form_is_built_on_request():
    V, T = inputs.icosphere(2)
    tr = binding.build_cluster_tree(V, T, 16, 0.8)
    Hd = binding.aca_assemble(tr, 1.0, 0.3, 1e-4, max_rhs=1, defer_fp64=True)
    H = binding.aca_assemble(tr, 1.0, 0.3, 1e-4, max_rhs=1)
    x = torch.tensor(inputs.uniform_rhs(3 * len(T), 6), device="cuda")[0]
    with pytest.raises(binding.HMError):
        _alone(Hd, x, "fp64")
    Hd.pack("fp64")
    a, b = _alone(Hd, x, "fp64"), _alone(H, x, "fp64")
    torch.cuda.synchronize()
    assert torch.equal(a, b)
