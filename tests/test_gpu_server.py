"""Request loop (``hm_server``): continuous admission by slot and device
footprint, overlapping execution, and every result bitwise the same alone
and in the mix."""
import numpy as np
import pytest

from paper_2205_04752_gb300 import binding, inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

_cache = {}


def pool():
    if "p" not in _cache:
        mats = []
        for (V, T), leaf, nu, compact in [(inputs.icosphere(2), 16, 0.3, False),
                                          (inputs.ellipsoid(6, 0.7, 1.6, 1.1), 20, 0.25, True),
                                          (inputs.icosphere(3), 32, 0.3, False)]:
            tr = binding.build_cluster_tree(V, T, leaf, 0.8)
            H = binding.aca_assemble(tr, 1.0, nu, 1e-4, max_rhs=4)
            H.pack("fp16")
            H.pack("fp32")
            if compact:
                H.compact()
            mats.append(H)
        _cache["p"] = mats
    return _cache["p"]


def _trace(n, rate, seed, mats):
    rng = np.random.default_rng(seed)
    t = np.cumsum(rng.exponential(1.0 / rate, n))
    reqs = []
    for i in range(n):
        m = int(rng.integers(len(mats)))
        solve = rng.random() < 0.2
        nrhs = 1 if solve else int(rng.integers(1, 5))
        y = np.full((nrhs, 3 * mats[m].M), np.nan)
        reqs.append(dict(arrival_s=float(t[i]), mesh=m, kind="solve" if solve else "matvec", nrhs=nrhs,
                         seed=1000 + i, tol=1e-6, y=y))
    return reqs


def test_results_are_the_same_alone_and_in_the_mix():
    mats = pool()
    srv = binding.Server(mats, slots=6, budget_bytes=1 << 30)
    reqs = _trace(48, 3000.0, 5, mats)
    res = srv.run(reqs, realtime=True)
    assert all(r["status"] == binding.HM_OK for r in res), [r["status"] for r in res]
    # the work of different requests overlapped on the device
    iv = sorted((r["start_s"], r["done_s"]) for r in res)
    assert any(iv[i + 1][0] < iv[i][1] for i in range(len(iv) - 1))
    for q, r in zip(reqs, res):
        assert r["done_s"] >= r["start_s"] >= r["arrival_s"] - 1e-6
        if q["kind"] == "solve":
            assert r["rel_residual"] <= 1e-6 and r["iterations"] > 0
        alone = dict(q, arrival_s=0.0, y=np.full_like(q["y"], np.nan))
        ra = srv.run([alone], realtime=True)[0]
        assert ra["status"] == binding.HM_OK
        assert np.array_equal(alone["y"], q["y"]), (q["kind"], q["mesh"], q["nrhs"])


def test_matvec_request_equals_the_library_product():
    mats = pool()
    srv = binding.Server(mats, slots=2, budget_bytes=1 << 28)
    H = mats[2]
    x = inputs.uniform_rhs(3 * H.M, 77, nrhs=3)
    y = np.zeros_like(x)
    res = srv.run([dict(mesh=2, kind="matvec", nrhs=3, x=x, y=y)], realtime=False)
    assert res[0]["status"] == binding.HM_OK
    xd = torch.tensor(x, device="cuda")
    yd = torch.empty_like(xd)
    binding.hmatvec(H, xd, yd, "fp16")
    torch.cuda.synchronize()
    assert np.array_equal(yd.cpu().numpy(), y)


def test_admission_by_footprint_and_queue_cap():
    mats = pool()
    big = dict(mesh=2, kind="matvec", nrhs=4, seed=1)
    small = dict(mesh=0, kind="matvec", nrhs=1, seed=2)
    probe = binding.Server(mats, slots=1, budget_bytes=1 << 30)
    fb, fs = probe.footprint(big), probe.footprint(small)
    assert fb > fs > 0
    # an arena that holds the small requests but never the big one
    srv = binding.Server(mats, slots=4, queue_cap=64, budget_bytes=(fs + fb) // 2)
    res = srv.run([small, big, small], realtime=False)
    assert [r["status"] for r in res] == [binding.HM_OK, binding.HM_EBUSY, binding.HM_OK]
    # everything arrives at once: a queue of 3 behind 1 slot rejects the rest
    srv = binding.Server(mats, slots=1, queue_cap=3, budget_bytes=1 << 30)
    res = srv.run([dict(small, seed=i) for i in range(10)], realtime=False)
    st = [r["status"] for r in res]
    assert st.count(binding.HM_OK) == 3 and st.count(binding.HM_EBUSY) == 7
    # memory-limited: two slots but room for one request at a time; all finish
    srv = binding.Server(mats, slots=2, queue_cap=64, budget_bytes=fb + fs // 2)
    res = srv.run([dict(big, seed=i) for i in range(4)], realtime=False)
    assert all(r["status"] == binding.HM_OK for r in res)
    iv = sorted((r["start_s"], r["done_s"]) for r in res)
    assert all(iv[i + 1][0] >= iv[i][1] - 1e-9 for i in range(3))


def test_solve_slots_keep_a_lane_for_matvecs():
    """With solve_slots = 1 of 2 slots, solves run one at a time and the
    matvec requests queued behind them are admitted while they wait; every
    result still equals the same request run alone."""
    mats = pool()
    srv = binding.Server(mats, slots=2, queue_cap=64, budget_bytes=1 << 30, solve_slots=1)
    solves = [dict(mesh=2, kind="solve", nrhs=1, seed=10 + i, tol=1e-6, y=np.full((1, 3 * mats[2].M), np.nan))
              for i in range(3)]
    mvs = [dict(mesh=1, kind="matvec", nrhs=2, seed=20 + i, y=np.full((2, 3 * mats[1].M), np.nan))
           for i in range(3)]
    reqs = solves + mvs
    res = srv.run(reqs, realtime=False)
    assert all(r["status"] == binding.HM_OK for r in res), [r["status"] for r in res]
    sv = sorted((r["start_s"], r["done_s"]) for r in res[:3])
    assert all(sv[i + 1][0] >= sv[i][1] - 1e-9 for i in range(2))   # one solve at a time
    assert min(r["start_s"] for r in res[3:]) < sv[1][0]            # matvecs did not wait for the solves
    for q, r in zip(reqs, res):
        alone = dict(q, y=np.full_like(q["y"], np.nan))
        assert srv.run([alone], realtime=False)[0]["status"] == binding.HM_OK
        assert np.array_equal(alone["y"], q["y"]), q["kind"]
    with pytest.raises(binding.HMError):
        binding.Server(mats, slots=2, solve_slots=3)


def test_concurrent_tensor_core_matvecs():
    """Many INT16 requests of 14-20 vectors (the forward pass and the far field
    of their first 16 on the tensor cores) on two meshes, admitted all at
    once on 8 slots so that their kernels share the SMs: every request
    completes (no bounded device wait runs out) and equals the library's
    product of the same vectors bitwise."""
    mats = []
    for (V, T), leaf in [(inputs.icosphere(4), 32), (inputs.ellipsoid(16, 0.7, 1.6, 1.1), 32)]:
        tr = binding.build_cluster_tree(V, T, leaf, 0.8)
        H = binding.aca_assemble(tr, 1.0, 0.3, 1e-4, max_rhs=20)
        H.pack("i16")
        mats.append(H)
    srv = binding.Server(mats, slots=8, queue_cap=256, budget_bytes=1 << 31, matvec_form="i16",
                         inner_form="i16", residual_form="i16")
    rng = np.random.default_rng(11)
    reqs = []
    for i in range(48):
        m = int(rng.integers(2))
        nrhs = int(rng.integers(14, 21))
        x = inputs.uniform_rhs(3 * mats[m].M, 300 + i, nrhs=nrhs)
        reqs.append(dict(mesh=m, kind="matvec", nrhs=nrhs, x=x, y=np.full_like(x, np.nan)))
    res = srv.run(reqs, realtime=False)
    assert all(r["status"] == binding.HM_OK for r in res), [r["status"] for r in res]
    for q in reqs[:12]:
        xd = torch.tensor(q["x"], device="cuda")
        yd = torch.empty_like(xd)
        binding.hmatvec(mats[q["mesh"]], xd, yd, "i16")
        torch.cuda.synchronize()
        assert np.array_equal(yd.cpu().numpy(), q["y"]), (q["mesh"], q["nrhs"])
