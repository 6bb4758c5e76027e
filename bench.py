"""Benchmark: H-matrix-vector products per second of the collocation Lame
single layer on a level-6 icosphere (81,920 flat triangles, 245,760 dofs,
E = 1, nu = 0.3, leaf 64, eta = 0.8, ACA eps = 1e-4), at <= 1e-4 relative
error against the FP64 form.

One step = one H-matrix-vector product y = V_h x (gather, far-field forward,
per-leaf product with the near field).  The H-matrix (GBs) is far larger than
L2, so every step streams it from HBM; no L2 flush is needed.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--form i16|fp16|fp32|...]
  python bench.py --impl reference     # the FP64 CPU oracle on the host cores

Besides the headline the JSON line carries, as context: the FP64 form, 32
right-hand sides, end-to-end products with host buffers, "batch64" (batched
products over 64 ellipsoid meshes with 1 and 16 right-hand sides), "solve"
(GMRES with FP64-residual refinement to 1e-8 on a 196,608-triangle cube),
"serving" (the request loop over 16 resident meshes at swept Poisson rates,
p50 / p99 latency), "amvm" (Algorithm 2 on the level-6 matrix, FP64, theta
0.7, eps 1e-4), "points" (the evaluation operator of Section 5, Eq.
(vector_eq): the displacement at 65,536 points inside the level-6 sphere,
its exact FP64 product and Algorithm 2 on it) and "baca" (Algorithm 3 on the
single layer: the level-6 solve with block-adaptive refinement); --no-batch /
--no-solve / --no-serve / --no-amvm / --no-points / --no-baca skip them.

Under torchrun (N > 1) every rank runs its own replica (the product shards
into independent problems; no collective on the data path): weak scaling,
value = all ranks' products / the slowest rank's time.
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

WORKLOAD = dict(workload="lame-single-layer-icosphere-L6", mesh="icosphere level 6",
                triangles=81920, dofs=245760, E=1.0, nu=0.3, leaf=64, eta=0.8, aca_eps=1e-4,
                nrhs=1)
# DRAM bytes per launch of the dominant kernel, from one ncu capture
# (dram__bytes_read.sum + dram__bytes_write.sum) on the benchmark workload.
# Reported only while every source file of the library is the one that was
# measured (sha256 over csrc/ in name order): any change to a kernel or to
# the layout code nulls it until it is measured again.
MEASURED_TRAFFIC = {"kernel": "leaf_near", "form": "i16", "level": 6,
                    "sources_sha256": "c578ec3bb6fe24b9fe4f66dc370281caf52d3d84ef662ccd8c5da61d5bec7098",
                    "bytes": 3925656832 + 1554432}
METRIC = "H-matvecs/s"
UNIT = "matvec/s"
MEAS_PEAKS = os.path.join(ROOT, "MEASURED_PEAKS.json")


def _sources_sha256():
    """sha256 over the library's source files (csrc/, in name order)."""
    import hashlib
    d = os.path.join(ROOT, "paper_2205_04752_gb300", "csrc")
    h = hashlib.sha256()
    for f in sorted(os.listdir(d)):
        if f.endswith((".cu", ".cuh", ".h", ".cpp")):
            h.update(f.encode())
            with open(os.path.join(d, f), "rb") as fh:
                h.update(fh.read())
    return h.hexdigest()


def _peaks():
    try:
        with open(MEAS_PEAKS) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi clock / throttle samples during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.Q}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, smax, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            p = [s.strip() for s in ln.split(",")]
            if len(p) < 9:
                continue
            try:
                sm.append(float(p[1]))
                smax = float(p[2])
            except ValueError:
                continue
            for k, nm in enumerate(names):
                if p[5 + k].lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": smax,
                "reasons": sorted(reasons), "samples": len(sm)}


# --------------------------------------------------------------------------
# CPU baseline: the oracle on a bounded sample of the same workload
# --------------------------------------------------------------------------

def _cpu_model():
    """Host CPU model name and logical CPU count, for the baseline's record."""
    name = None
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for ln in out.splitlines():
            if ln.lower().startswith("model name:"):
                name = ln.split(":", 1)[1].strip()
                break
    except (OSError, subprocess.SubprocessError):
        pass
    if not name:
        try:
            with open("/proc/cpuinfo") as f:
                for ln in f:
                    if ln.lower().startswith("model name"):
                        name = ln.split(":", 1)[1].strip()
                        break
        except OSError:
            pass
    import platform
    return name or platform.machine(), os.cpu_count()


class OracleFull:
    """The oracle's H-matrix of the whole workload -- its own cluster tree,
    partition, near-field quadrature and ACA (FP64, OpenMP over blocks) --
    assembled once, and its full FP64 H-matrix-vector product.  Nothing is
    sampled or scaled: one step is one complete product."""

    def __init__(self, V, T):
        import oracle
        w = WORKLOAD
        self.oracle = oracle
        self.threads = oracle.num_threads()
        t0 = time.perf_counter()
        self.H = oracle.HMatrix(V, T, w["leaf"], w["eta"], w["aca_eps"])
        self.H.assemble()
        self.t_asm = time.perf_counter() - t0
        from paper_2205_04752_gb300 import inputs
        self.x = inputs.uniform_rhs(3 * len(T), 0)

    def step(self):
        """Seconds of one full product."""
        t0 = time.perf_counter()
        self.H.matvec(WORKLOAD["E"], WORKLOAD["nu"], self.x)
        return time.perf_counter() - t0

    def median(self, reps, threads=None):
        if threads:
            self.oracle.set_num_threads(threads)
        try:
            return float(np.median([self.step() for _ in range(reps)]))
        finally:
            if threads:
                self.oracle.set_num_threads(self.threads)

    def describe(self, reps):
        model, ncpu = _cpu_model()
        return (f"the whole level-6 workload, no sampling: the oracle's own tree, partition, near field and "
                f"ACA (FP64) assembled once in {self.t_asm:.1f} s on {self.threads} threads (not timed), then "
                f"its full FP64 H-matrix-vector product, median of {reps}; host {model}, {ncpu} CPUs")


def cpu_baseline(V, T, reps=5):
    s = OracleFull(V, T)
    s.step()  # warm-up (first touch of the factors)
    t = s.median(reps)
    t1 = s.median(reps, threads=1)
    model, ncpu = _cpu_model()
    return {"value": 1.0 / t, "unit": UNIT, "cores": s.threads, "kind": "oracle", "sample": s.describe(reps),
            "one_core": {"value": 1.0 / t1, "unit": UNIT, "cores": 1, "ms_per_matvec": round(t1 * 1e3, 1)},
            "ms_per_matvec": round(t * 1e3, 1), "assembly_s": round(s.t_asm, 1), "cpu_model": model,
            "nproc": ncpu}


# --------------------------------------------------------------------------

def _dist():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def _slowest(ms, ws, device):
    """The job's time of a timed region: the slowest rank's (max over the ws
    ranks of the process group; every rank gets it)."""
    if ws == 1:
        return ms
    import torch
    import torch.distributed as dist
    t = torch.tensor([ms], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def run_reference(args):
    ws, rank, local = _dist()
    if rank != 0:
        return 0
    from paper_2205_04752_gb300 import inputs
    V, T = inputs.icosphere(6)
    ref = OracleFull(V, T)
    for _ in range(args.warmup):
        ref.step()
    ts = [ref.step() for _ in range(args.steps)]
    t = float(np.median(ts))
    v = 1.0 / t
    model, ncpu = _cpu_model()
    info = {"value": v, "unit": UNIT, "cores": ref.threads, "kind": "oracle", "sample": ref.describe(args.steps),
            "assembly_s": round(ref.t_asm, 1), "cpu_model": model, "nproc": ncpu}
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": ws,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * t,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": dict(WORKLOAD, form="fp64-cpu"),
            "cpu_baseline": info,
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def run_ours(args):
    import torch
    import torch.distributed as dist
    from paper_2205_04752_gb300 import binding, inputs

    ws, rank, local = _dist()
    torch.cuda.set_device(local)
    if ws > 1:
        dist.init_process_group("nccl" if dist.is_nccl_available() else "gloo")
    w = dict(WORKLOAD)
    if args.level != 6:
        w.update(workload=f"lame-single-layer-icosphere-L{args.level}",
                 mesh=f"icosphere level {args.level}", triangles=20 * 4 ** args.level,
                 dofs=60 * 4 ** args.level)
    V, T = inputs.icosphere(args.level)
    M = len(T)
    stream = torch.cuda.current_stream()
    t0 = time.perf_counter()
    tree = binding.build_cluster_tree(V, T, w["leaf"], w["eta"])
    t_tree = time.perf_counter() - t0
    if args.points_minimal:
        # profiling runs of the evaluation operator alone
        xp = torch.tensor(inputs.uniform_rhs(3 * M, 0)[0], device="cuda")

        def timed_p(fn, steps, warmup):
            for _ in range(warmup):
                fn()
            torch.cuda.synchronize()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            for _ in range(steps):
                fn()
            e1.record(stream)
            torch.cuda.synchronize()
            return e0.elapsed_time(e1)
        ctx = bench_points(args, tree, w, xp, timed_p, eval_only=True)
        print(json.dumps({"points_minimal": True, "level": args.level, **ctx}), flush=True)
        return 0
    t0 = time.perf_counter()
    H = binding.aca_assemble(tree, w["E"], w["nu"], w["aca_eps"], max_rhs=32)
    torch.cuda.synchronize()
    t_asm = time.perf_counter() - t0
    form = args.form
    H.pack(form)
    st = H.stats()
    x = torch.tensor(inputs.uniform_rhs(3 * M, 0, nrhs=args.nrhs), device="cuda")
    if args.nrhs == 1:
        x = x[0]
    y = torch.empty_like(x)
    y64 = torch.empty_like(x)
    binding.hmatvec(H, x, y64, "fp64")
    binding.hmatvec(H, x, y, form)
    torch.cuda.synchronize()
    err_mixed = float(torch.linalg.norm(y - y64) / torch.linalg.norm(y64))

    def timed(fn, steps, warmup):
        for _ in range(warmup):
            fn()
        torch.cuda.synchronize()
        if ws > 1:
            dist.barrier()
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(steps):
            fn()
        e1.record(stream)
        torch.cuda.synchronize()
        return _slowest(e0.elapsed_time(e1), ws, "cuda")

    # ---- headline: device-resident product in the chosen form
    clk = ClockSampler(local)
    if not args.minimal:
        clk.start()
    ms_total = timed(lambda: binding.hmatvec(H, x, y, form), args.steps, args.warmup)
    clocks = clk.stop() if not args.minimal else None
    ms_step = ms_total / args.steps
    value = ws * 1e3 / ms_step
    if args.minimal:
        if rank == 0:
            print(json.dumps({"metric": METRIC, "value": round(value, 3), "unit": UNIT,
                              "ms_per_step": round(ms_step, 4), "steps": args.steps,
                              "warmup": args.warmup, "config": dict(w, form=form, nrhs=args.nrhs),
                              "vectors_per_s": round(value * args.nrhs, 2),
                              "minimal": True, "rel_err_vs_fp64_form": err_mixed}), flush=True)
        if ws > 1:
            dist.barrier()
            dist.destroy_process_group()
        return 0

    # ---- per-kernel device times (CUDA events on the launching stream)
    H.profile(True)
    for _ in range(args.steps):
        binding.hmatvec(H, x, y, form)
    kms, calls = H.profile_read()
    H.profile(False)
    kms = kms[:3] / max(calls, 1)
    names = ["gather", "far_fwd", "leaf_near"]
    dom = int(np.argmax(kms))
    wf = {"fp64": 8, "fp32": 4, "bf16": 2, "fp16": 2, "i16": 2}[form]
    wn = 8 if form == "fp64" else 4
    wa = 8 if form == "fp64" else 4
    # algorithmic bytes: every stored value once, the vectors once; U column
    # scales (16-bit forms) are read by the forward pass; x and w are 4-vectors
    scales = 0 if wf >= 4 else st.factor_columns * 4
    nvals = st.near_pairs * 6
    xvec = 4 * M * wa
    wvec = 4 * st.factor_columns * wa
    near_bytes = nvals * wn
    if form == "i16":
        # the leaves' diagonal blocks stay FP32; every other near column is
        # six INT16 segments and six FP32 scales
        _, nodes, _, near = tree.export()
        nsz = nodes[:, 1] - nodes[:, 0]
        diag = near[:, 0] == near[:, 1]
        pairs = nsz[near[:, 0]] * nsz[near[:, 1]]
        near_bytes = int(pairs[diag].sum()) * 6 * 4 + int(pairs[~diag].sum()) * 6 * 2 + \
            int(nsz[near[~diag, 1]].sum()) * 6 * 4
    alg = {
        "gather": 3 * M * 8 + M * 4 + xvec,
        "far_fwd": st.far_v_entries * wf + scales + xvec + wvec,
        "leaf_near": st.far_u_entries * wf + near_bytes + wvec + xvec + 3 * M * 8,
    }
    peak, peak_kind = _peaks()
    achieved = alg[names[dom]] / (kms[dom] * 1e-3) / 1e9
    traffic = None
    mt = MEASURED_TRAFFIC
    if (mt["bytes"] and names[dom] == mt["kernel"] and form == mt["form"] and args.level == mt["level"]
            and _sources_sha256() == mt["sources_sha256"]):
        traffic = mt["bytes"]
    roofline = {"bound": "hbm", "achieved": round(achieved, 1), "peak": peak, "unit": "GB/s",
                "frac": round(achieved / peak, 4), "traffic": traffic, "kernel": names[dom],
                "peak_kind": peak_kind,
                "kernel_ms": {n: round(float(k), 4) for n, k in zip(names, kms)},
                "alg_bytes": {n: int(b) for n, b in alg.items()}}
    total_alg = sum(alg.values())

    # ---- end to end through the public API with host buffers
    xh = torch.empty(3 * M, dtype=torch.float64, pin_memory=True)
    xh.copy_(x.cpu())
    yh = torch.empty(3 * M, dtype=torch.float64, pin_memory=True)
    xn, yn = xh.numpy(), yh.numpy()
    ms_e2e = timed(lambda: binding.hmatvec_host(H, xn, yn, form), args.steps, args.warmup)
    e2e = {"value": ws * 1e3 * args.steps / ms_e2e, "unit": UNIT,
           "h2d_bytes_per_step": 3 * M * 8, "d2h_bytes_per_step": 3 * M * 8}

    failed = []  # contexts that ended in a device failure
    # ---- context: FP64 plain form and 32 right-hand sides
    ms64 = timed(lambda: binding.hmatvec(H, x, y64, "fp64"), max(2, args.steps // 4), 1) \
        / max(2, args.steps // 4)
    X = torch.tensor(inputs.uniform_rhs(3 * M, 0, nrhs=32), device="cuda")
    Y = torch.empty_like(X)
    ms32 = timed(lambda: binding.hmatvec(H, X, Y, form), max(2, args.steps // 4), 1) \
        / max(2, args.steps // 4)
    Y64 = torch.empty_like(X)
    binding.hmatvec(H, X, Y64, "fp64")
    torch.cuda.synchronize()

    def e_mixed(Yf):
        d = torch.linalg.norm(Yf - Y64, dim=1) / torch.linalg.norm(Y64, dim=1)
        return {"max": float(d.max()), "mean": float(d.mean())}
    err32 = e_mixed(Y)

    # ---- context: the other reduced forms on the same matrix (one vector,
    # and their error against the FP64 form over the same 32 vectors)
    forms_ctx = {}
    for f in ("fp16", "bf16", "fp32"):
        if f == form or args.minimal:
            continue
        try:
            H.pack(f)
            msf = timed(lambda: binding.hmatvec(H, x, y, f), max(4, args.steps // 4), 2) / max(4, args.steps // 4)
            binding.hmatvec(H, X, Y, f)
            torch.cuda.synchronize()
            forms_ctx[f] = {"ms_per_matvec": round(msf, 4), "value": round(1e3 / msf, 2),
                            "rel_err_vs_fp64_form_32_vectors": e_mixed(Y)}
        except Exception as e:  # reported, the headline still prints
            forms_ctx[f] = _context_error(e, "forms", failed)

    # ---- context: adaptive matrix-vector multiplication (Algorithm 2, FP64)
    amvm_ctx = None
    if not args.no_amvm:
        try:
            ya = torch.empty_like(x)
            binding.amvm(H, x, ya, theta=0.7, eps=1e-4)  # warm-up (host tables, allocations)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            ai = binding.amvm(H, x, ya, theta=0.7, eps=1e-4)
            torch.cuda.synchronize()
            amvm_ms = (time.perf_counter() - t0) * 1e3
            amvm_ctx = {"theta": 0.7, "eps": 1e-4, "ms": round(amvm_ms, 1), "iterations": ai["iterations"],
                        "crosses_used_fraction": round(ai["crosses_used"] / max(ai["crosses_full"], 1), 4),
                        "rel_err_vs_fp64_product": float(torch.linalg.norm(ya - y64) / torch.linalg.norm(y64)),
                        "gamma_over_bhat": ai["gamma"][-1] / ai["bhat_norm"]}
            # Section 3's combination of assembly and product: no ACA at assembly,
            # Algorithm 1 on demand inside the adaptive product
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            Hd = binding.aca_assemble(tree, w["E"], w["nu"], w["aca_eps"], max_rhs=1, defer_aca=True)
            torch.cuda.synchronize()
            t_def = time.perf_counter() - t0
            t0 = time.perf_counter()
            ad = binding.amvm(Hd, x, ya, theta=0.7, eps=1e-4, on_demand=True)
            torch.cuda.synchronize()
            t_od = time.perf_counter() - t0
            amvm_ctx["aca_on_demand"] = {
                "assemble_without_aca_s": round(t_def, 3), "amvm_s": round(t_od, 3),
                "total_s": round(t_def + t_od, 3), "full_assembly_s": round(t_asm, 3),
                "crosses_computed_fraction": round(ad["crosses_full"] / max(ai["crosses_full"], 1), 4),
                "iterations": ad["iterations"],
                "rel_err_vs_fp64_product": float(torch.linalg.norm(ya - y64) / torch.linalg.norm(y64))}
            del Hd
        except Exception as e:  # reported, the headline still prints
            amvm_ctx = _context_error(e, "amvm", failed)

    # ---- context: block-adaptive ACA solve of the single layer (Algorithm 3,
    # the paper's parameters theta 0.8, alpha 10, eps 1e-4, 8 starting ACA steps)
    baca_ctx = None
    if not args.no_baca:
        try:
            g = np.tile([1.0, 0.0, 0.0], M) + inputs.uniform_rhs(3 * M, 2)[0]
            gd = torch.tensor(g, device="cuda")
            td = torch.empty_like(gd)
            yv = torch.empty_like(gd)
            baca_ctx = {"rhs": "(1,0,0) + U[-1,1] per dof (seed 2)", "theta": 0.8, "alpha": 10.0, "eps": 1e-4,
                        "look": 2}
            for r0 in (8, 2):  # the paper's starting rank, and a coarse start that the refinement must lift
                torch.cuda.synchronize()
                t0 = time.perf_counter()
                bi = binding.baca(H, gd, td, theta=0.8, alpha=10.0, eps=1e-4, r0=r0, look=2)
                torch.cuda.synchronize()
                t_baca = time.perf_counter() - t0
                binding.hmatvec(H, td, yv, "fp64")
                torch.cuda.synchronize()
                baca_ctx[f"r0_{r0}"] = {
                    "s": round(t_baca, 3), "steps": bi["steps"], "gmres_iterations": bi["gmres_iterations"],
                    "marked_total": bi["marked_total"],
                    "crosses_used_fraction": round(bi["crosses_used"] / max(bi["crosses_full"], 1), 4),
                    "E_over_b": bi["E"] / max(bi["b_norm"], 1e-300), "rel_residual_A_k": bi["rel_residual"],
                    "rel_residual_full_fp64": float(torch.linalg.norm(gd - yv) / torch.linalg.norm(gd))}
            # the adaptive construction with the solve: no ACA at assembly, Algorithm 1
            # on demand inside Algorithm 3 (coarse start), against the full assembly
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            Hd = binding.aca_assemble(tree, w["E"], w["nu"], w["aca_eps"], max_rhs=1, defer_aca=True)
            torch.cuda.synchronize()
            t_def = time.perf_counter() - t0
            t0 = time.perf_counter()
            bd = binding.baca(Hd, gd, td, theta=0.8, alpha=10.0, eps=1e-4, r0=2, look=2, on_demand=True)
            torch.cuda.synchronize()
            t_od = time.perf_counter() - t0
            binding.hmatvec(H, td, yv, "fp64")
            torch.cuda.synchronize()
            baca_ctx["r0_2_aca_on_demand"] = {
                "assemble_without_aca_s": round(t_def, 3), "baca_s": round(t_od, 3),
                "total_s": round(t_def + t_od, 3), "full_assembly_s": round(t_asm, 3), "steps": bd["steps"],
                "crosses_computed_fraction": round(bd["crosses_full"] / max(sum(st.rank_sum), 1), 4),
                "rel_residual_full_fp64": float(torch.linalg.norm(gd - yv) / torch.linalg.norm(gd))}
            del Hd
        except Exception as e:  # reported, the headline still prints
            baca_ctx = _context_error(e, "baca", failed)

    points_ctx = None
    if not args.no_points and rank == 0 and ws == 1:
        try:
            points_ctx = bench_points(args, tree, w, x, timed)
        except Exception as e:  # reported, the headline still prints
            points_ctx = _context_error(e, "points", failed)

    line = {"metric": METRIC, "value": round(value, 3), "unit": UNIT, "n_gpus": ws,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(ms_step, 4),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": {"fp64": "f64", "fp32": "f32", "bf16": "bf16+f32", "fp16": "f16+f32", "i16": "i16+f32"}[form],
            "data": "synthetic",
            "config": dict(w, form=form, l2="inputs larger than L2 (H-matrix "
                           f"{total_alg/1e9:.2f} GB per product)", parallelism=f"replicas{ws}"),
            "roofline": roofline, "clocks": clocks, "e2e": e2e,
            "gpu_launches": 4 * args.steps,
            "rel_err_vs_fp64_form": err_mixed,
            "rel_err_vs_fp64_form_32_vectors": err32,
            "fp64_form": {"ms_per_matvec": round(ms64, 4), "value": round(1e3 / ms64, 3)},
            "other_forms": forms_ctx,
            "nrhs32": {"ms_per_call": round(ms32, 4), "vectors_per_s": round(32e3 / ms32, 2)},
            "amvm": amvm_ctx,
            "points": points_ctx,
            "baca": baca_ctx,
            "assembly": assembly_context(st, t_tree, t_asm)}
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(V, T)
    elif rank == 0:
        line["cpu_baseline"] = None
    # ---- batched and served workloads (their own matrices; free this one first)
    del H, X, Y
    torch.cuda.empty_cache()
    for key, skip, fn in (("batch64", args.no_batch, bench_batch), ("solve", args.no_solve, bench_solve),
                          ("serving", args.no_serve, bench_serving)):
        if skip or rank != 0 or ws != 1:
            continue
        try:
            line[key] = fn(args)
        except Exception as e:  # reported, the headline still prints
            line[key] = _context_error(e, key, failed)
    line["context_failed"] = failed
    if rank == 0:
        print(json.dumps(line), flush=True)
    if ws > 1:
        dist.barrier()
        dist.destroy_process_group()
    # a device failure may leave the CUDA context unusable: the headline was
    # measured before it, but the run is not clean
    return 3 if failed else 0


def assembly_context(st, t_tree, t_asm):
    """Assembly times and their roofline: the near-field quadrature and ACA
    are bound by the FP64 units; their FP64 operations are counted by the
    kernels (quadrature points, ACA entries) with the per-rule operation
    counts of the library's statistics."""
    fp64_peak, fp64_src = _fp64_peak()
    out = {"tree_s": round(t_tree, 3), "assemble_s": round(t_asm, 3),
           "near_ms": round(st.assemble_ms[0], 1), "aca_ms": round(st.assemble_ms[1], 1),
           "rank_mean": [round(r / max(st.nadm, 1), 2) for r in st.rank_sum],
           "bytes_per_form": st.bytes_form,
           "near_points": {"whole_triangle_pairs": st.near_points[0], "subdivision_leaves": st.near_points[1],
                           "self_pairs": st.near_points[2]},
           "aca_entries": {"V_Delta": st.aca_entries[0], "V_kl": st.aca_entries[1]}}
    rl = {}
    for key, fl, ms in (("near", st.assembly_flops[0], st.assemble_ms[0]),
                        ("aca", st.assembly_flops[1], st.assemble_ms[1])):
        if fl > 0 and ms > 0:
            tf = fl / (ms * 1e-3) / 1e12
            rl[key] = {"bound": "alu", "flops": fl, "achieved": round(tf, 4), "peak": fp64_peak,
                       "unit": "TFLOP/s (FP64)", "frac": round(tf / fp64_peak, 4)}
    out["roofline"] = rl
    out["fp64_peak_from"] = fp64_src
    return out


def _context_error(e, key, failed):
    """Record a context section's exception.  A failed bounded wait or CUDA
    call of the library (HM_ETIMEOUT, HM_EDEVICE) or a CUDA error raised by
    torch marks the run as failed on the device."""
    from paper_2205_04752_gb300 import binding
    if isinstance(e, binding.HMError):
        device = e.code in (binding.HM_ETIMEOUT, binding.HM_EDEVICE)
    else:
        device = "CUDA" in str(e) or "cuda" in type(e).__name__.lower()
    if device:
        failed.append(key)
    return {"error": f"{type(e).__name__}: {e}", "device_failure": device}


def _fp64_peak():
    """FP64 (CUDA-core) peak of this GPU: 2 FMA per SM per clock (4 flops),
    the rate behind NVIDIA's 1.25 TFLOP/s for GB300 (152 SMs at 2.07 GHz),
    scaled by this device's SM count and maximum SM clock."""
    import torch
    nsm = torch.cuda.get_device_properties(0).multi_processor_count
    mhz = 2070.0
    try:
        out = subprocess.run(["nvidia-smi", "--query-gpu=clocks.max.sm", "--format=csv,noheader,nounits",
                              "-i", "0"], capture_output=True, text=True, timeout=10).stdout.split()
        mhz = float(out[0]) if out else mhz
    except (OSError, ValueError, subprocess.SubprocessError):
        pass
    return round(nsm * 4 * mhz * 1e6 / 1e12, 4), f"{nsm} SMs x 4 FP64 flops/clk x {mhz:.0f} MHz"


def bench_points(args, tree, w, x, timed, eval_only=False):
    """The evaluation operator ~V_h (Section 5, Eq. (vector_eq)) for 65,536
    points uniform in the ball of radius 0.95 inside the level-6 sphere (leaf
    64): assembly, the exact FP64 product u = ~V_h t (device time, the bytes
    it must read: every factor and near value once, the parts and vectors),
    and Algorithm 2 on it (theta 0.7, eps 1e-4) with the assembled ACA and
    with ACA on demand."""
    import torch
    from paper_2205_04752_gb300 import binding, inputs
    npts = 65536 if args.level == 6 else 65536 >> (2 * (6 - args.level))
    P = inputs.ball_points(npts, 0.95, 7)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    pt = binding.build_point_tree(tree, P, 64)
    t_tree = time.perf_counter() - t0
    t0 = time.perf_counter()
    Hp = binding.aca_assemble(pt, w["E"], w["nu"], w["aca_eps"], max_rhs=1)
    torch.cuda.synchronize()
    t_asm = time.perf_counter() - t0
    st = Hp.stats()
    _, nodes, adm, _ = pt.export()
    rows_far = int(np.sum(nodes[adm[:, 0], 1] - nodes[adm[:, 0], 0])) if len(adm) else 0
    M = pt.M_src
    t = x if x.dim() == 1 else x[0]
    u = torch.empty(3 * npts, dtype=torch.float64, device="cuda")
    steps = max(5, min(50, args.steps // 8))
    ms = timed(lambda: binding.eval_points(Hp, t, u), steps, 2) / steps
    # algorithmic bytes: every factor and near value once, the block parts
    # written and read once, the densities gathered and the result scattered
    alg = (st.far_entries + 6 * st.near_pairs) * 8 + 2 * 3 * rows_far * 8 + 2 * 3 * M * 8 + 2 * 3 * npts * 8
    peak, peak_kind = _peaks()
    gbs = alg / (ms * 1e-3) / 1e9
    # FP64 operations the product must execute: per factor entry of kernel k
    # one FMA per component it needs (V_Delta 3, V_pp 1, V_pq 2) in V^T x and
    # again in U w; per near pair 12 FMA and 2 additions; an FMA counts 2
    need = (3, 1, 2, 2, 1, 2, 1)
    flops = 2 * sum(c * e for c, e in zip(need, st.far_entries_kern)) + 26 * st.near_pairs
    fp64_peak, fp64_src = _fp64_peak()
    tf = flops / (ms * 1e-3) / 1e12
    ev = {"ms": round(ms, 3), "evals_per_s": round(1e3 / ms, 2), "alg_bytes": int(alg),
          "achieved_GBps": round(gbs, 1), "hbm_peak": peak, "hbm_peak_kind": peak_kind,
          "hbm_frac": round(gbs / peak, 4), "steps": steps,
          "roofline": {"bound": "alu", "achieved": round(tf, 4), "peak": fp64_peak, "unit": "TFLOP/s",
                       "frac": round(tf / fp64_peak, 4), "flops": int(flops), "peak_from": fp64_src}}
    # the FP32 form: the same passes on FP32 copies, bound by HBM
    Hp.pack("fp32")
    u32 = torch.empty_like(u)
    ms32 = timed(lambda: binding.eval_points(Hp, t, u32, "fp32"), steps, 2) / steps
    alg32 = (st.far_entries + 6 * st.near_pairs) * 4 + 2 * 3 * rows_far * 4 + 2 * 3 * M * 8 + 2 * 3 * npts * 8
    gbs32 = alg32 / (ms32 * 1e-3) / 1e9
    ev32 = {"ms": round(ms32, 3), "evals_per_s": round(1e3 / ms32, 2),
            "rel_err_vs_fp64_form": float(torch.linalg.norm(u32 - u) / torch.linalg.norm(u)),
            "roofline": {"bound": "hbm", "achieved": round(gbs32, 1), "peak": peak, "unit": "GB/s",
                         "frac": round(gbs32 / peak, 4), "alg_bytes": int(alg32), "peak_kind": peak_kind}}
    if eval_only:
        return {"points": npts, "nadm": st.nadm, "nnear": st.nnear, "assemble_s": round(t_asm, 3), "eval": ev,
                "eval_fp32": ev32}
    ya = torch.empty_like(u)
    binding.amvm(Hp, t, ya, theta=0.7, eps=1e-4)  # warm-up
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    ai = binding.amvm(Hp, t, ya, theta=0.7, eps=1e-4)
    torch.cuda.synchronize()
    amvm_ms = (time.perf_counter() - t0) * 1e3
    err = float(torch.linalg.norm(ya - u) / torch.linalg.norm(u))
    del Hp
    torch.cuda.empty_cache()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    Hd = binding.aca_assemble(pt, w["E"], w["nu"], w["aca_eps"], max_rhs=1, defer_aca=True)
    torch.cuda.synchronize()
    t_def = time.perf_counter() - t0
    t0 = time.perf_counter()
    ad = binding.amvm(Hd, t, ya, theta=0.7, eps=1e-4, on_demand=True)
    torch.cuda.synchronize()
    t_od = time.perf_counter() - t0
    err_od = float(torch.linalg.norm(ya - u) / torch.linalg.norm(u))
    del Hd
    torch.cuda.empty_cache()
    return {"points": npts, "region": "ball r <= 0.95 (seed 7)", "leaf": 64, "nadm": st.nadm,
            "nnear": st.nnear, "tree_s": round(t_tree, 3), "assemble_s": round(t_asm, 3),
            "rank_mean": [round(r / max(st.nadm, 1), 2) for r in st.rank_sum],
            "eval": ev,
            "eval_fp32": ev32,
            "amvm": {"theta": 0.7, "eps": 1e-4, "ms": round(amvm_ms, 1), "iterations": ai["iterations"],
                     "crosses_used_fraction": round(ai["crosses_used"] / max(ai["crosses_full"], 1), 4),
                     "rel_err_vs_exact_product": err,
                     "gamma_over_bhat": ai["gamma"][-1] / max(ai["bhat_norm"], 1e-300)},
            "amvm_aca_on_demand": {"assemble_without_aca_s": round(t_def, 3), "amvm_s": round(t_od, 3),
                                   "total_s": round(t_def + t_od, 3), "full_assembly_s": round(t_asm, 3),
                                   "crosses_computed_fraction":
                                       round(ad["crosses_full"] / max(ai["crosses_full"], 1), 4),
                                   "rel_err_vs_exact_product": err_od}}


def bench_batch(args):
    """Batched products over 64 ellipsoid meshes (2k-40k triangles each, leaf
    32, nu uniform[0.2, 0.45]): one launch per phase over all members, the
    schedule chosen by the autotuner, replayed as a CUDA graph; FP16 form."""
    import torch
    from paper_2205_04752_gb300 import binding, inputs
    specs = inputs.ellipsoid_batch_specs(64, 3, 2000.0, 40000.0)
    mats, t0, resident, tri = [], time.perf_counter(), 0, 0
    for sp in specs:
        V, T = inputs.ellipsoid(sp["n"], sp["a"], sp["b"], sp["c"])
        tr = binding.build_cluster_tree(V, T, 32, 0.8)
        H = binding.aca_assemble(tr, sp["E"], sp["nu"], 1e-4, max_rhs=1, defer_fp64=True)
        H.pack("fp16")
        H.compact()
        resident += H.footprint()
        tri += len(T)
        mats.append(H)
    torch.cuda.synchronize()
    t_asm = time.perf_counter() - t0
    R = 16
    B = binding.Batch(mats, "fp16", max_rhs=R)
    out = {"workload": "64 ellipsoids, 2k-40k triangles (log-uniform), leaf 32, eta 0.8, eps 1e-4",
           "meshes": len(mats), "triangles": tri, "dofs": B.ndof, "forward_groups": B.ngroups,
           "leaves": B.nleaves, "assemble_s": round(t_asm, 2), "resident_gb": round(resident / 1e9, 2)}
    bytes_prod = sum(m.stats().bytes_form[3] for m in mats)
    stream = torch.cuda.current_stream()
    for nrhs in (1, R):
        sched, _ = B.autotune(nrhs=nrhs, reps=3)
        x = torch.tensor(inputs.uniform_rhs(B.ndof, 1000, nrhs=nrhs), device="cuda")
        y = torch.empty_like(x)
        for _ in range(3):
            B.matvec(x, y, graph=True)
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        n = 10
        e0.record(stream)
        for _ in range(n):
            B.matvec(x, y, graph=True)
        e1.record(stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / n
        out[f"nrhs{nrhs}"] = {"ms_per_batch_product": round(ms, 3),
                              "mesh_vector_products_per_s": round(len(mats) * nrhs * 1e3 / ms, 1),
                              "factor_gb_per_s": round(bytes_prod / (ms * 1e-3) / 1e9, 1),
                              "schedule": sched}
    B.check()
    out["bytes_per_product_gb"] = round(bytes_prod / 1e9, 2)
    del B, mats
    torch.cuda.empty_cache()
    return out


def bench_solve(args):
    """The Dirichlet solve on the cube surface [-1,1]^3 with 128 x 128
    squares per face (196,608 triangles, 589,824 dofs), nu = 0.3, leaf 64:
    GMRES(50) on the BF16 form inside FP64-residual iterative refinement to
    ||g - V_h t|| <= 1e-8 ||g||; g = (1, 0, 0) + uniform[-1, 1] per dof."""
    import torch
    from paper_2205_04752_gb300 import binding, inputs
    V, T = inputs.cube_surface(128)
    M = len(T)
    t0 = time.perf_counter()
    tr = binding.build_cluster_tree(V, T, 64, 0.8)
    H = binding.aca_assemble(tr, 1.0, 0.3, 1e-4, max_rhs=1)
    H.pack("bf16")
    torch.cuda.synchronize()
    t_asm = time.perf_counter() - t0
    g = (np.array([1.0, 0.0, 0.0])[None, :] + np.random.default_rng(2).uniform(-1, 1, (M, 3))).ravel()
    gd = torch.tensor(g, device="cuda")
    td = torch.zeros_like(gd)
    out = {"workload": "cube surface 6x128x128x2 = 196,608 triangles, 589,824 dofs, nu 0.3, leaf 64",
           "assemble_s": round(t_asm, 2)}
    stream = torch.cuda.current_stream()
    for f in ("bf16", "fp64"):
        binding.hmatvec(H, gd, td, f)
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(5):
            binding.hmatvec(H, gd, td, f)
        e1.record(stream)
        torch.cuda.synchronize()
        out[f"{f}_matvec_ms"] = round(e0.elapsed_time(e1) / 5, 3)
    td.zero_()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    info = binding.solve(H, gd, td, tol=1e-8, inner_form="bf16", restart=50, max_inner=5000,
                         raise_on_fail=False)
    torch.cuda.synchronize()
    out["solve_s"] = round(time.perf_counter() - t0, 3)
    out.update({k: info[k] for k in ("iterations", "restarts", "refinements", "rel_residual", "converged")})
    # what the same iteration count would cost on the plain FP64 form
    out["fp64_inner_estimate_s"] = round(info["iterations"] * out["fp64_matvec_ms"] * 1e-3, 2)
    del H
    torch.cuda.empty_cache()
    return out


def bench_serving(args):
    """Request loop over a pool of 16 resident meshes (icospheres of levels
    3-6 and 12 ellipsoids of 1k-200k triangles): Poisson arrivals at swept
    rates, 80% matvec (1-32 vectors, INT16 form, within 1e-4 of the FP64
    form) / 20% solve (tol 1e-6, GMRES on FP16 with FP32-residual
    refinement), mesh uniform over the pool; 8 slots of which solves may take
    --serve-solve-slots, so that matvec requests always find a lane.  Latency
    percentiles per request kind."""
    import torch
    from paper_2205_04752_gb300 import binding, inputs
    meshes = [(inputs.icosphere(l), 64, 0.3) for l in (3, 4, 5, 6)]
    for sp in inputs.ellipsoid_batch_specs(12, 5, 1000.0, 200000.0):
        meshes.append((inputs.ellipsoid(sp["n"], sp["a"], sp["b"], sp["c"]), 64, sp["nu"]))
    mats, t0, resident, tri = [], time.perf_counter(), 0, []
    for (V, T), leaf, nu in meshes:
        tr = binding.build_cluster_tree(V, T, leaf, 0.8)
        H = binding.aca_assemble(tr, 1.0, nu, 1e-4, max_rhs=1, defer_fp64=True)
        for f in ("i16", "fp16", "fp32"):
            H.pack(f)
        H.compact()
        resident += H.footprint()
        tri.append(len(T))
        mats.append(H)
    torch.cuda.synchronize()
    t_asm = time.perf_counter() - t0
    srv = binding.Server(mats, slots=8, queue_cap=256, budget_bytes=24 << 30, matvec_form="i16",
                         inner_form="fp16", residual_form="fp32", restart=30, solve_slots=args.serve_solve_slots)
    out = {"workload": "16 resident meshes (icosphere L3-L6, 12 ellipsoids 1k-200k triangles), "
                       "Poisson arrivals, 80% matvec (1-32 RHS, i16) / 20% solve (tol 1e-6)",
           "triangles": tri, "assemble_s": round(t_asm, 2), "resident_gb": round(resident / 1e9, 2),
           "slots": 8, "solve_slots": args.serve_solve_slots, "budget_gb": 24, "rates": []}
    # warm the kernels of every form once
    srv.run([dict(mesh=m, kind="matvec", nrhs=1, seed=m) for m in range(len(mats))], realtime=False)
    rng = np.random.default_rng(5)
    for rate in args.serve_rates:
        n = max(20, int(rate * args.serve_seconds))
        t = np.cumsum(rng.exponential(1.0 / rate, n))
        reqs = []
        for i in range(n):
            solve = rng.random() < 0.2
            reqs.append(dict(arrival_s=float(t[i]), mesh=int(rng.integers(len(mats))),
                             kind="solve" if solve else "matvec",
                             nrhs=1 if solve else int(rng.integers(1, 33)), seed=i, tol=1e-6))
        w0 = time.perf_counter()
        res = srv.run(reqs, realtime=True)
        wall = time.perf_counter() - w0
        ok = [r for r in res if r["status"] in (binding.HM_OK, binding.HM_ENOTCONV)]
        lat = np.array([r["done_s"] - r["arrival_s"] for r in ok]) * 1e3

        def pct(kind):
            v = np.array([r["done_s"] - r["arrival_s"] for q, r in zip(reqs, res)
                          if q["kind"] == kind and r["status"] in (binding.HM_OK, binding.HM_ENOTCONV)]) * 1e3
            return ({"p50_ms": round(float(np.percentile(v, 50)), 2), "p99_ms": round(float(np.percentile(v, 99)), 2),
                     "completed": int(len(v))} if len(v) else None)
        vec = sum(q["nrhs"] for q, r in zip(reqs, res) if r["status"] == binding.HM_OK and q["kind"] == "matvec")
        sres = [r["rel_residual"] for q, r in zip(reqs, res) if q["kind"] == "solve" and r["status"] == binding.HM_OK]
        out["rates"].append({
            "rate_rps": rate, "requests": n, "completed": len(ok),
            "rejected": sum(r["status"] == binding.HM_EBUSY for r in res),
            "not_converged": sum(r["status"] == binding.HM_ENOTCONV for r in res),
            "p50_ms": round(float(np.percentile(lat, 50)), 2) if len(lat) else None,
            "p99_ms": round(float(np.percentile(lat, 99)), 2) if len(lat) else None,
            "matvec": pct("matvec"), "solve": pct("solve"),
            "throughput_rps": round(len(ok) / wall, 1),
            "matvec_vectors_per_s": round(vec / wall, 1),
            "solve_max_rel_residual": float(max(sres)) if sres else None})
    del srv, mats
    torch.cuda.empty_cache()
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=400)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--form", default="i16", choices=["fp64", "fp32", "bf16", "fp16", "i16"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-batch", action="store_true", help="skip the 64-mesh batched products")
    ap.add_argument("--no-serve", action="store_true", help="skip the request-loop measurement")
    ap.add_argument("--no-solve", action="store_true", help="skip the 196,608-triangle cube solve")
    ap.add_argument("--no-amvm", action="store_true", help="skip the adaptive matrix-vector multiplication")
    ap.add_argument("--no-baca", action="store_true",
                    help="skip the block-adaptive ACA solve (Algorithm 3 on the single layer)")
    ap.add_argument("--no-points", action="store_true",
                    help="skip the evaluation operator (displacement at 65,536 interior points)")
    ap.add_argument("--serve-rates", type=float, nargs="+", default=[10.0, 30.0, 100.0, 300.0, 1000.0])
    ap.add_argument("--serve-solve-slots", type=int, default=2,
                    help="of the 8 request slots, how many solves may hold at once")
    ap.add_argument("--serve-seconds", type=float, default=4.0)
    ap.add_argument("--minimal", action="store_true",
                    help="profiling runs: assemble, pack and time the headline product only "
                         "(no e2e, context forms, clock sampling or CPU baseline)")
    ap.add_argument("--nrhs", type=int, default=1,
                    help="with --minimal: right-hand sides per timed product (profiling the several-vector "
                         "kernels)")
    ap.add_argument("--points-minimal", action="store_true",
                    help="profiling runs of the evaluation operator: assemble it for 65,536 points "
                         "(4^(level-6) x 65,536 below level 6) and time its exact product only")
    ap.add_argument("--level", type=int, default=6,
                    help="icosphere level; 6 is the benchmark workload, smaller levels are for "
                         "profiling captures")
    args = ap.parse_args()
    if args.nrhs != 1 and not args.minimal:
        ap.error("--nrhs applies to --minimal profiling runs only")
    if not 1 <= args.nrhs <= 32:
        ap.error("--nrhs must be in 1..32")
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        return run_reference(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
