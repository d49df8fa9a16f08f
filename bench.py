"""Benchmark of the fused cascaded-LBM step on the lid-driven cubic cavity.

One step = one time step of the three 128^3 cavities at Re = 100 with
n = 0.5, 1.0 and 1.5 (lid U = 0.05), each a separate lattice on the same
stream.  ``value`` is the whole-job MLUPS of the FP32-storage form (fluid
nodes x steps / seconds / 1e6, CUDA events on the launching stream, inputs
resident in HBM).  The FP64 and FP16-shifted forms are timed the same way and
reported under ``forms``, each against the HBM roofline of its bytes per
lattice update, 19 reads + 19 writes x bytes per population.

``--impl reference`` times the FP64 CPU oracle on the host cores instead (the
reference arm): the same workload and metric, one oracle step per step.

Multi-GPU (torchrun, one rank per GPU): every rank runs its own replica of
the workload (weak scaling, no collective in the data path); a barrier
brackets the timed region and the slowest rank's time is used.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "MLUPS & % HBM roofline, FP64 vs FP32/FP16-store; served solves/s, p50/p99"
BYTES_PER_POP = {"f64": 8, "f32": 4, "f16s": 2, "f16r": 2}
# algorithmic bytes per lattice update: 19 reads + 19 writes of the stored
# type; F16R also reads and writes its node's 8-byte FP16 reference
BYTES_PER_UPDATE = {"f64": 304, "f32": 152, "f16s": 76, "f16r": 92}
L_BENCH = 128
RE_BENCH = 100.0
NS_BENCH = (0.5, 1.0, 1.5)


def _peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as fh:
            d = json.load(fh)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def max_over_ranks(x: float, ws: int, device: str = "cpu") -> float:
    """The largest x over all ranks (the slowest rank's time); x itself at
    one rank.  NCCL needs device="cuda", gloo takes "cpu"."""
    if ws <= 1:
        return float(x)
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_mlups(nodes_per_rank: float, ws: int, ms_max: float) -> float:
    """Weak scaling: every rank updates nodes_per_rank nodes in the timed
    region; the job's rate is all ranks' updates over the slowest rank's time."""
    return nodes_per_rank * ws / (ms_max * 1e-3) / 1e6


def _dist():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


class Clocks:
    """nvidia-smi sampling during the timed region."""

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.path = None

    def __enter__(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.index}", f"--query-gpu={q}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
        time.sleep(0.3)
        return self

    def __exit__(self, *exc):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        if self.path is None or not os.path.exists(self.path):
            return None
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx = float(parts[2])
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        os.unlink(self.path)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sm)}


STEP_KERNEL_SOURCES = ("d3q19.cuh", "v2.cuh", "collide.cuh", "launch.h", "kernels.cuh",
                       "tma_step.cuh")
# translation unit of each storage form's step kernel
STEP_TU = {"f64": "step_f64.cu", "f32": "step_f32.cu", "f16s": "step_f16.cu"}


def kernel_source_hash(form: str = "f32") -> str:
    """Hash of the sources that define one form's step kernel (its headers and
    translation unit), so that changes elsewhere keep a capture valid."""
    import hashlib
    csrc = os.path.join(ROOT, "paper_1908_05396_gb300", "csrc")
    h = hashlib.sha256()
    for fn in STEP_KERNEL_SOURCES + (STEP_TU[form],):
        h.update(open(os.path.join(csrc, fn), "rb").read())
    return h.hexdigest()[:16]


def _profile_note(fname: str, kernel: str, form: str):
    """The numbers after the kernel name and source hash in a committed ncu
    summary table under profiles/, if they were taken on the current kernel
    sources (else None)."""
    path = os.path.join(ROOT, "profiles", fname)
    if not os.path.exists(path):
        return None
    digest = kernel_source_hash(form)
    for line in open(path):
        parts = line.split()
        if len(parts) >= 3 and parts[0] == kernel and parts[1] == digest:
            return [float(x) for x in parts[2:]]
    return None


def _traffic_note(kernel: str, form: str = "f32"):
    """DRAM bytes per launch (read + write) from the committed ncu summary."""
    v = _profile_note("traffic.txt", kernel, form)
    return v[0] if v else None


def _fp64_ops_note(kernel: str):
    """FP64 instructions per node update (DADD, DFMA, DMUL) of the FP64 step
    kernel from the committed ncu summary."""
    return _profile_note("fp64_ops.txt", kernel, "f64")


def _oracle_lattices(nz: int | None = None):
    import oracle
    from paper_1908_05396_gb300 import workloads as wl
    oracle.build()
    out = []
    for n in NS_BENCH:
        prob = wl.cavity(L_BENCH, RE_BENCH, n)
        p = oracle.Params(nx=prob.nx, ny=prob.ny, nz=nz or prob.nz, face=prob.face, K=prob.K,
                          n=prob.n, U=prob.U_lid)
        out.append([p, oracle.rest_state(p), p.N])
    return oracle, out


def _cpu_baseline(budget_s: float = 12.0):
    """The FP64 oracle on the host cores, a bounded sample of the same workload:
    whole oracle steps of the three 128^3 cavities until the budget is spent."""
    oracle, lats = _oracle_lattices()
    cores = int(os.environ.get("OMP_NUM_THREADS", "0")) or (os.cpu_count() or 1)
    nodes, steps = 0, 0
    t0 = time.perf_counter()
    while True:
        for lt in lats:
            lt[1] = oracle.run(lt[0], lt[1], 1)
            nodes += lt[2]
        steps += 1
        if time.perf_counter() - t0 >= budget_s:
            break
    dt = time.perf_counter() - t0
    out = {"value": nodes / dt / 1e6, "unit": "MLUPS", "cores": cores, "kind": "oracle",
           "sample": f"{steps} oracle step(s) of the three 128^3 Re=100 cavities "
                     f"(n=0.5,1,1.5), FP64, OpenMP over z-planes, {dt:.1f} s"}
    # the same oracle on one core, in a fresh process (its thread count is
    # fixed when the OpenMP runtime starts)
    try:
        r = subprocess.run([sys.executable, os.path.abspath(__file__), "--oracle-one-core"],
                           env=dict(os.environ, OMP_NUM_THREADS="1"), capture_output=True,
                           text=True, timeout=120)
        out["single_core"] = json.loads(r.stdout.strip().splitlines()[-1])
    except Exception as e:  # reported, not fatal: the multi-core number stands
        out["single_core"] = {"error": str(e)[:200]}
    return out


def run_oracle_one_core():
    """The oracle on one core: steps of a 64^3 cavity (Re 100, n 0.5) for
    about 5 s."""
    import oracle
    from paper_1908_05396_gb300 import workloads as wl
    oracle.build()
    prob = wl.cavity(64, RE_BENCH, 0.5)
    p = oracle.Params(nx=prob.nx, ny=prob.ny, nz=prob.nz, face=prob.face, K=prob.K, n=prob.n,
                      U=prob.U_lid)
    f = oracle.run(p, oracle.rest_state(p), 1)
    steps, t0 = 0, time.perf_counter()
    while time.perf_counter() - t0 < 5.0:
        f = oracle.run(p, f, 1)
        steps += 1
    dt = time.perf_counter() - t0
    print(json.dumps({"value": prob.N * steps / dt / 1e6, "unit": "MLUPS", "cores": 1,
                      "sample": f"{steps} oracle steps of a 64^3 cavity (Re 100, n 0.5), FP64, "
                                f"OMP_NUM_THREADS=1, {dt:.1f} s"}))
    return 0


def ref_slab(cores: int) -> int:
    """z-planes of each cavity per reference step: one plane per host core
    (the oracle's OpenMP loop runs over z-planes, so fewer planes would leave
    cores idle), at least 16 and at most the whole 128^3 cavity."""
    return min(L_BENCH, max(16, cores))


def run_reference(args):
    ws, rank, _ = _dist()
    if rank != 0:
        return 0
    cores = int(os.environ.get("OMP_NUM_THREADS", "0")) or (os.cpu_count() or 1)
    slab = ref_slab(cores)
    oracle, lats = _oracle_lattices(nz=slab)
    for _ in range(args.warmup):
        for lt in lats:
            lt[1] = oracle.run(lt[0], lt[1], 1)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        for lt in lats:
            lt[1] = oracle.run(lt[0], lt[1], 1)
    dt = time.perf_counter() - t0
    nodes = sum(lt[2] for lt in lats) * args.steps
    v = nodes / dt / 1e6
    line = {
        "impl": "reference", "metric": METRIC, "value": v, "unit": "MLUPS", "n_gpus": ws,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt / args.steps * 1e3,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic",
        "config": {"workload": "lid-driven cubic cavity 128^3 x3 (Re=100, n=0.5/1.0/1.5, U=0.05)",
                   "storage": "f64", "l2": "n/a (CPU)"},
        "cpu_baseline": {"value": v, "unit": "MLUPS", "cores": cores, "kind": "oracle",
                         "sample": f"{args.steps} oracle steps of a 128x128x{slab} slab of "
                                   "each of the three cavities (walls on all faces, lid +y; "
                                   "one z-plane per core)"},
        "e2e": {"value": v, "unit": "MLUPS", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line))
    return 0


def form_spec(name: str):
    """(dtype, in_place, rounding) of a form name: a storage form, optionally
    with "_inplace" (one buffer streamed in place) or "_sr" (F16S with
    stochastically rounded stores)."""
    if name.endswith("_inplace"):
        return name[:-len("_inplace")], True, None
    if name.endswith("_sr"):
        return name[:-len("_sr")], False, "stochastic"
    return name, False, None


def _time_form(clbm, torch, dtype, steps, warmup, stream, in_place=False, rounding=None):
    """MLUPS of one storage form over the three cavities, each lattice stepping
    on its own stream so that one lattice's launch gaps and tail waves are
    filled by the others' work; the timed region is fenced by events on
    ``stream`` that every lattice stream joins."""
    from paper_1908_05396_gb300 import workloads as wl
    streams = [torch.cuda.Stream() for _ in NS_BENCH]
    lats = [clbm.Lattice(**wl.cavity(L_BENCH, RE_BENCH, n).kwargs(), dtype=dtype,
                         stream=s.cuda_stream, in_place=in_place) for n, s in zip(NS_BENCH, streams)]
    if rounding:
        for lt in lats:
            lt.set_rounding(rounding)
    tuned = [lt.autotune(10) for lt in lats]     # launch shape per lattice (cached)
    N = lats[0].N
    for _ in range(warmup):
        for lt in lats:
            lt.step(1)
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for s in streams:
        s.wait_event(e0)
    for _ in range(steps):
        for lt in lats:
            lt.step(1)
    for s in streams:
        ev = torch.cuda.Event()
        ev.record(s)
        stream.wait_event(ev)
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    for lt in lats:
        lt.close()
    launches = steps * len(lats)
    return ms, N, launches, tuned


def run_ours(args):
    import torch
    ws, rank, local = _dist()
    torch.cuda.set_device(local)
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    from paper_1908_05396_gb300 import build, workloads as wl
    build.build()
    from paper_1908_05396_gb300 import clbm
    clbm.lib()
    peak, peak_kind = _peaks()
    stream = torch.cuda.Stream()

    def barrier():
        if ws > 1:
            import torch.distributed as dist
            dist.barrier()
        torch.cuda.synchronize()

    # ---- headline: FP32 storage ---------------------------------------------
    head = "f32"
    # untimed warm-up of every lattice (also builds nothing new)
    barrier()
    with Clocks(local) as clk:
        barrier()
        ms, N, launches, tuned = _time_form(clbm, torch, head, args.steps, args.warmup, stream)
        barrier()
    clocks = clk.summary()
    ms_max = max_over_ranks(ms, ws, device="cuda")
    nodes = N * len(NS_BENCH) * args.steps
    value = whole_job_mlups(nodes, ws, ms_max)
    per_launch_s = ms * 1e-3 / launches
    bpn = 38 * BYTES_PER_POP[head]
    achieved = bpn * N / per_launch_s / 1e9
    npt0 = tuned[0]["npt"]
    cap = "true" if npt0 & 4 else "false"
    kern = (f"step2_kernel<float,false,false,{cap}>" if (npt0 & 3) == 2
            else f"step_kernel<float,float,false,false,{cap}>")
    traffic = _traffic_note(kern)

    # ---- the other forms ------------------------------------------------------
    forms = {}
    form_steps = {"f64": max(3, args.steps // 40), "f16s": args.steps, "f16r": args.steps}
    form_steps["f32_inplace"] = form_steps["f16s_sr"] = args.steps
    for name in ("f64", "f16s", "f16s_sr", "f16r", "f32_inplace"):
        if args.forms and name not in args.forms:
            continue
        dt, ip, rnd = form_spec(name)
        barrier()
        ms_f, N_f, launches_f, tuned_f = _time_form(clbm, torch, dt, form_steps[name], args.warmup,
                                                    stream, in_place=ip, rounding=rnd)
        mlups = N_f * len(NS_BENCH) * form_steps[name] / (ms_f * 1e-3) / 1e6
        gbs = BYTES_PER_UPDATE[dt] * N_f * launches_f / (ms_f * 1e-3) / 1e9
        forms[name] = {"MLUPS": mlups, "GB/s": gbs, "frac_of_hbm": gbs / peak,
                       "steps": form_steps[name], "bytes_per_update": BYTES_PER_UPDATE[dt],
                       "launch": [(t["block"], t["npt"]) for t in tuned_f]}
        if ip:
            forms[name]["what"] = "one population buffer streamed in place (half the memory)"
        if rnd:
            forms[name]["what"] = "F16S storage with stochastically rounded stores"
    forms[head] = {"MLUPS": value / ws, "GB/s": achieved, "frac_of_hbm": achieved / peak,
                   "steps": args.steps, "bytes_per_update": bpn,
                   "launch": [(t["block"], t["npt"]) for t in tuned]}
    # The FP64 form is bound by the FP64 pipe, not HBM: its roofline is the
    # FP64 instruction rate (one DADD, DMUL or DFMA per slot), measured live
    # by the FMA probe, against the FP64 instructions per update counted by
    # ncu on the current kernel sources.
    if "f64" in forms:
        rate = clbm.probe_fma_rate("f64")
        kern64 = "step_kernel<double,double,false,false,false>"
        ops = _fp64_ops_note(kern64)
        alu = {"bound": "alu", "unit": "FP64 instructions/s", "peak": rate / 2.0,
               "peak_kind": "measured (FMA probe: two FLOP per DFMA)", "kernel": kern64,
               "probe_tflops": rate / 1e12}
        if ops:
            per_node = sum(ops)
            alu.update({"fp64_instructions_per_update": per_node,
                        "achieved": per_node * forms["f64"]["MLUPS"] * 1e6,
                        "flops_per_update": ops[0] + 2.0 * ops[1] + ops[2]})
            alu["frac"] = alu["achieved"] / alu["peak"]
            alu["tflops"] = alu["flops_per_update"] * forms["f64"]["MLUPS"] * 1e6 / 1e12
        forms["f64"]["alu_roofline"] = alu
    summary = {k: {"MLUPS": round(v["MLUPS"], 1), "frac_of_hbm": round(v["frac_of_hbm"], 4)}
               for k, v in forms.items()}
    if "f64" in forms and "frac" in forms["f64"]["alu_roofline"]:
        summary["f64"]["frac_of_fp64_pipe"] = round(forms["f64"]["alu_roofline"]["frac"], 4)

    # ---- end to end through the C ABI with host buffers ------------------------
    # The same three-cavity job from pinned host states: per lattice, create,
    # upload the state, step, and read rho, u and gamma_dot back to the host.
    import numpy as np
    e2e_steps = args.steps
    probs = [wl.cavity(L_BENCH, RE_BENCH, n) for n in NS_BENCH]
    f0s, outs_pinned = [], []
    for prob in probs:
        with clbm.Lattice(**prob.kwargs(), dtype=head) as lat:
            f = lat.get_state()                  # host copy of the initial state
        pin = torch.empty(f.shape, dtype=torch.float64, pin_memory=True)
        pin.numpy()[...] = f                     # inputs in pinned host memory
        f0s.append(pin.numpy())
        shp = f.shape[1:]
        outs_pinned.append(tuple(torch.empty(s_, dtype=torch.float64, pin_memory=True).numpy()
                                 for s_ in (shp, (3,) + shp, shp)))
    e2e_streams = [torch.cuda.Stream() for _ in probs]
    barrier()
    t0 = time.perf_counter()
    lats = [clbm.Lattice(**prob.kwargs(), dtype=head, stream=s.cuda_stream)
            for prob, s in zip(probs, e2e_streams)]
    for lat, f0 in zip(lats, f0s):
        lat.autotune(10)              # cached: no timing runs here
        lat.set_state(f0)             # H2D of the inputs
    for lat in lats:
        lat.step(e2e_steps)
    outs = [lat.fields(out=o) for lat, o in zip(lats, outs_pinned)]   # D2H of the results
    t1 = time.perf_counter()
    for lat in lats:
        lat.close()
    e2e_val = sum(p.N for p in probs) * e2e_steps / (t1 - t0) / 1e6 * ws
    h2d = sum(f0.nbytes for f0 in f0s) / e2e_steps
    d2h = sum(a.nbytes for o in outs for a in o) / e2e_steps

    batch = serving = None
    if not args.no_extra:
        barrier()
        batch = _batch_bench(clbm, torch, wl, args.batch_steps, peak)
        trace = wl.serving_trace(count=256, seed=0, rate=20.0)[:args.serve_requests]
        serving = _serving_bench(
            clbm, trace, 1e-7, args.serve_cap, 20, 100,
            f"the first {len(trace)} requests of the serving trace: Poisson 20/s (seed 0), half "
            "cavities L~U{32..192}, half channels 8xU{32..256}x8, Re~U[50,1000], n~U[0.4,1.6]")

    cpu = None
    if rank == 0 and ws == 1 and not args.no_cpu:
        cpu = _cpu_baseline()

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": "MLUPS", "n_gpus": ws,
            "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": ms_max / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": "lid-driven cubic cavity 128^3 x3 (Re=100, n=0.5/1.0/1.5, "
                                   "U=0.05), one lattice per n, FP32 storage",
                       "storage": head, "nodes_per_step": N * len(NS_BENCH),
                       "l2": "inputs larger than L2: 159 MB read + 159 MB written per lattice step"},
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                         "frac": achieved / peak, "traffic": traffic,
                         "peak_kind": peak_kind, "kernel": kern,
                         "algorithmic_bytes_per_launch": bpn * N,
                         "duration": "timed region / launches, three lattices on three streams "
                                     "(launches overlap)",
                         "forms": summary},
            "forms": forms,
            "e2e": {"value": e2e_val, "unit": "MLUPS", "h2d_bytes_per_step": h2d,
                    "d2h_bytes_per_step": d2h,
                    "what": f"create + set_state from host + {e2e_steps} steps + fields to host, "
                            "the three 128^3 cavities on three streams, FP32 storage, "
                            "pinned host buffers, wall clock"},
            "batch": batch,
            "serving": serving,
            "gpu_launches": launches,
            "clocks": clocks,
            "cpu_baseline": cpu,
        }
        print(json.dumps(line))
    if ws > 1:
        import torch.distributed as dist
        dist.destroy_process_group()
    return 0


def _clamp_active_nodes(lats, probs, nu_min=5e-4, nu_max=10.0) -> dict:
    """Nodes whose viscosity sits on a clamp after the timed steps: the
    reported shear rate is the one at the clamped omega, and the power law
    evaluated there lies beyond the clamp exactly when the clamp binds."""
    import numpy as np
    lo = hi = 0
    for lt, p in zip(lats, probs):
        rho, _, gd = lt.fields()
        with np.errstate(divide="ignore", over="ignore", invalid="ignore"):
            nu = p.K / rho * np.power(gd, p.n - 1.0)
        lo += int(np.count_nonzero(nu < nu_min * (1 - 1e-4)))
        hi += int(np.count_nonzero(nu > nu_max * (1 + 1e-4)))
    return {"at_nu_min": lo, "at_nu_max": hi}


def _batch_bench(clbm, torch, wl, steps, peak):
    """64 seeded cavities of uneven size in one batch (FP32), against the same
    lattices stepped one launch at a time."""
    probs = wl.batch_cavities(count=64, seed=0)
    lats = [clbm.Lattice(**p.kwargs(), dtype="f32") for p in probs]
    N = sum(p.N for p in probs)
    def timed(b):
        b.step(200)                          # warm-up: graph capture and caches
        b.sync()
        t0 = time.perf_counter()
        b.step(steps)
        b.sync()
        return time.perf_counter() - t0

    with clbm.Batch("f32", capacity=len(lats), check_interval=100) as b:
        for lt in lats:
            b.add(lt)
        tuned = b.autotune(4)
        dt = timed(b)
        diverged = int(b.stats_all()["diverged"].sum())
        clamped = _clamp_active_nodes(lats, probs)
        # both modes at their usual best shapes, whichever the tuner kept
        b.set_launch(32, 4, 2, -8)
        dt_persistent = timed(b)
        b.set_lattice_launch(32, 2, 5, 4)
        dt_per_lattice = timed(b)
    mlups = N * steps / dt / 1e6
    # the same lattices, one launch per lattice per step
    for lt in lats:
        lt.sync()
    n_alone = max(10, steps // 10)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(n_alone):
        for lt in lats:
            lt.step(1)
    for lt in lats:
        lt.sync()
    dt_alone = time.perf_counter() - t0
    for lt in lats:
        lt.close()
    # one cavity of about the same node count, for the batch's efficiency
    L1 = round(N ** (1.0 / 3.0))
    with clbm.Lattice(**wl.cavity(L1, 100.0, 1.0).kwargs(), dtype="f32") as one:
        one.autotune(5)
        one.step(50)
        one.sync()
        t0 = time.perf_counter()
        one.step(steps)
        one.sync()
        dt_one = time.perf_counter() - t0
    gbs = 152 * N * steps / dt / 1e9
    return {"workload": "64 cavities, L~U{32..96}, Re~U[50,500], n~U[0.4,1.6], U=0.05, FP32, seed 0",
            "nodes": N, "steps": steps, "MLUPS": mlups, "GB/s": gbs, "frac_of_hbm": gbs / peak,
            "launch": tuned, "diverged_lattices": diverged, "clamp_active_nodes": clamped,
            "equal_size_single_MLUPS": L1 ** 3 * steps / dt_one / 1e6,
            "equal_size_single": f"one {L1}^3 cavity (Re 100, n 1), FP32, autotuned",
            "persistent_MLUPS": N * steps / dt_persistent / 1e6,
            "persistent_launch": "one persistent launch per step: 32x4 tiles, zc 2, 8 capped CTAs/SM",
            "per_lattice_MLUPS": N * steps / dt_per_lattice / 1e6,
            "per_lattice_launch": "one launch per lattice per step: 32x2 capped, 4 streams",
            "separate_launches_MLUPS": N * n_alone / dt_alone / 1e6,
            "timing": "host wall clock around graph-captured batch steps, synchronised"}


def _serve_trace(clbm, trace, dtype, tol, cap, plateau, check):
    """Replay the trace through the continuous-batching server (requests
    submitted at their arrival times); every request keeps its fields."""
    dt_, _, rnd_ = form_spec(dtype)
    with clbm.Server(dt_, hbm_budget_bytes=150e9, max_active=64, check_interval=check) as srv:
        if rnd_:
            srv.set_rounding(rnd_)
        t0 = time.perf_counter()
        ids = []
        for r in trace:
            delay = t0 + r.arrival - time.perf_counter()
            if delay > 0:
                time.sleep(delay)
            ids.append(srv.submit(**r.problem.kwargs(), tol=tol, max_steps=cap,
                                  plateau_checks=plateau, keep_fields=True))
        res = [srv.wait(i) for i in ids]
        fields = [srv.fields(i)[1] for i in ids]
        info = srv.info()
    return res, fields, info


def _latency_stats(clbm, res) -> dict:
    lat = sorted(r["t_done"] - r["t_submit"] for r in res)
    span = max(r["t_done"] for r in res) - min(r["t_submit"] for r in res)
    status = {}
    for r in res:
        k = clbm.SOLVE_STATUS[r["status"]]
        status[k] = status.get(k, 0) + 1
    q = lambda p: lat[min(len(lat) - 1, int(round(p * (len(lat) - 1))))]
    return {"solves_per_s": len(res) / span, "p50_latency_s": q(0.5), "p99_latency_s": q(0.99),
            "makespan_s": span, "status": status,
            "mean_steps": sum(r["steps"] for r in res) / len(res)}


def _solve_alone(clbm, prob, dtype, tol, cap, plateau, check):
    """One request solved by a plain single-instance handle with the server's
    stopping rule: R <= tol, divergence, the step cap, or a plateau of the
    residual (no 10 % drop over `plateau` checks), read at every check."""
    with clbm.Lattice(**prob.kwargs(), dtype=dtype, check_interval=check) as lt:
        best, since, steps, status = float("inf"), 0, 0, "max_steps"
        while steps < cap:
            lt.step(check)
            steps += check
            R, rc = lt.residual()
            if rc != 0:
                status = "diverged"
                break
            if R <= tol:
                status = "converged"
                break
            if R < 0.9 * best:
                best, since = R, 0
            elif R == R and R != float("inf"):
                since += 1
            if since >= plateau:
                status = "plateau"
                break
        u = lt.fields()[1] if status != "diverged" else None
    return status, steps, u


def _serving_bench(clbm, trace, tol, cap, plateau, check, workload, bars=None):
    """The trace through the continuous-batching server in four storage
    forms (F16R, the headline: the FP16 store that meets its bar on every
    trace; F16S with stochastically rounded and with round-to-nearest stores;
    FP32), and the same requests solved
    one at a time by plain single-instance FP64 handles with the same
    stopping rule and check interval (the solves/s baseline).  Each served
    result is compared with the FP64 result of the same request: at the same
    step count where both stopped on the step cap, else at each one's own end
    (its steady state when both converged)."""
    import numpy as np
    bars = bars or {"f16r": 2e-3, "f16s": 2e-3, "f16s_sr": 2e-3, "f32": 1e-4}
    t0 = time.perf_counter()
    base = [_solve_alone(clbm, r.problem, "f64", tol, cap, plateau, check) for r in trace]
    seq_dt = time.perf_counter() - t0
    base_status = {}
    for st, _, _ in base:
        base_status[st] = base_status.get(st, 0) + 1
    forms = {}
    for dt in ("f16r", "f16s_sr", "f16s", "f32"):
        res, fields, info = _serve_trace(clbm, trace, dt, tol, cap, plateau, check)
        out = _latency_stats(clbm, res)
        out["server_MLUPS"] = info["lattice_updates"] / max(info["busy_seconds"], 1e-9) / 1e6
        l2 = []
        for r, u, (st, n, u64) in zip(res, fields, base):
            if u64 is None or clbm.SOLVE_STATUS[r["status"]] == "diverged":
                continue
            l2.append(float(np.linalg.norm(u - u64) / max(np.linalg.norm(u64), 1e-300)))
        out["velocity_l2_vs_f64"] = {"n": len(l2), "median": float(np.median(l2)) if l2 else None,
                                     "max": max(l2) if l2 else None,
                                     "within_bar": f"{sum(x <= bars[dt] for x in l2)}/{len(l2)} at "
                                                   f"L2 <= {bars[dt]:g}"}
        del fields
        forms[dt] = out
    head = dict(forms["f16r"])
    head.update({
        "form": "f16r", "workload": workload,
        "rule": f"tol {tol}, step cap {cap}, plateau {plateau} checks, check interval {check} steps",
        "other_forms": {dt: forms[dt] for dt in ("f16s_sr", "f16s", "f32")},
        "sequential_f64": {"solves_per_s": len(trace) / seq_dt, "seconds": seq_dt,
                           "status": base_status,
                           "what": "the same requests one at a time, plain FP64 handles, same rule"},
        "speedup_vs_sequential_f64": forms["f16r"]["solves_per_s"] / (len(trace) / seq_dt),
        "accuracy": "velocity L2 of each served result against the same request solved in FP64 "
                    "(same step count when both stop on the cap; else each at its own end)"})
    return head


def run_serve_steady(args):
    """Serving to steady state: a scaled trace whose requests converge within
    minutes (48 requests, Poisson 20/s, cavities L ~ U{16..48}, channels
    8 x U{16..64} x 8, Re ~ U[50, 400], n ~ U[0.4, 1.6]), run to residual
    1e-7 with residual checks every 4000 steps (a per-step rate; the long
    interval puts the F16R form's rounding floor below the tolerance), in
    every form and by sequential FP64 on the same requests."""
    import torch  # noqa: F401  (CUDA context on the chosen device)
    from paper_1908_05396_gb300 import build, workloads as wl
    build.build()
    from paper_1908_05396_gb300 import clbm
    trace = wl.serving_trace(count=args.serve_requests, seed=0, rate=20.0, cavity_L=(16, 48),
                             channel_H=(16, 64), Re_range=(50.0, 400.0))
    wk = (f"{len(trace)} requests, Poisson 20/s (seed 0), half cavities L~U{{16..48}}, half "
          "channels 8xU{16..64}x8, Re~U[50,400], n~U[0.4,1.6]")
    out = _serving_bench(clbm, trace, 1e-7, 400_000, 20, 4000, wk,
                         bars={"f16r": 2e-3, "f16s": 2e-3, "f16s_sr": 2e-3, "f32": 1e-4})
    print(json.dumps({"metric": "served solves/s, p50/p99, to steady state", "serving": out}))
    return 0


def _run_to_steady(clbm, prob, dtype, tol, max_steps, plateau=20, chunk=1000, check=100,
                   progress=None, start=None, snapshot_at=None):
    """Step a lattice until R <= tol, a residual plateau (no 10 % drop over
    `plateau` reads, one per chunk), divergence or max_steps.  `start` =
    (populations, steps) continues from a stored state; `snapshot_at` keeps
    the populations after that many steps (returned in the info)."""
    snap = None
    dt_, ip_, rnd_ = form_spec(dtype)
    with clbm.Lattice(**prob.kwargs(), dtype=dt_, in_place=ip_, check_interval=check) as lat:
        if rnd_:
            lat.set_rounding(rnd_)
        lat.autotune(5)
        best, since, steps, R, status = float("inf"), 0, 0, float("inf"), "max_steps"
        if start is not None:
            lat.set_state(start[0])
            steps = start[1]
        t0 = time.perf_counter()
        while steps < max_steps:
            lat.step(chunk)
            steps += chunk
            if snapshot_at is not None and steps == snapshot_at:
                snap = lat.get_state()
            R, rc = lat.residual()
            if progress and (steps // chunk) % progress == 0:
                print(f"[{dtype}] step {steps} R {R:.3e} {time.perf_counter() - t0:.0f} s",
                      file=sys.stderr, flush=True)
            if rc != 0:
                status = "diverged"
                break
            if R <= tol:
                status = "converged"
                break
            if R < 0.9 * best:
                best, since = R, 0
            else:
                since += 1
            if since >= plateau:
                status = "plateau"
                break
        dt = time.perf_counter() - t0
        _, u, _ = lat.fields()
    info = {"steps": steps, "residual": R, "status": status, "seconds": dt}
    if snapshot_at is not None:
        info["snapshot"] = snap
    return u, info


def run_precision(args):
    """Velocity error of the FP32 and FP16-shifted forms against FP64: a 64^3
    cavity (Re 100, n 0.8) at steady state, and the 256^3 Re 1000 n 0.8
    cavity after a fixed number of steps (the FP64 form is ALU bound, and a
    256^3 steady state needs ~1e6 steps)."""
    import numpy as np
    import torch  # noqa: F401  (CUDA context on the chosen device)
    from paper_1908_05396_gb300 import build, workloads as wl
    build.build()
    from paper_1908_05396_gb300 import clbm
    out = {"metric": "precision", "cases": []}
    prob = wl.cavity(64, 100.0, 0.8)
    res = {}
    forms = ("f64", "f32", "f16s", "f16s_sr", "f16r")
    for dt in forms:
        res[dt] = _run_to_steady(clbm, prob, dt, 1e-8, 600_000)
    n64 = float(np.linalg.norm(res["f64"][0]))
    out["cases"].append({
        "case": "cavity 64^3, Re 100, n 0.8, U 0.05, run to R <= 1e-8 (F16S: or plateau)",
        "runs": {k: v[1] for k, v in res.items()},
        "l2_vs_f64": {k: float(np.linalg.norm(res[k][0] - res["f64"][0])) / n64
                      for k in forms[1:]}})
    prob = wl.cavity(256, 1000.0, 0.8)
    fixed = {}
    for dt in forms:
        dt_, ip_, rnd_ = form_spec(dt)
        with clbm.Lattice(**prob.kwargs(), dtype=dt_, in_place=ip_) as lat:
            if rnd_:
                lat.set_rounding(rnd_)
            lat.autotune(3)
            t0 = time.perf_counter()
            lat.step(args.precision_steps)
            lat.sync()
            sec = time.perf_counter() - t0
            _, u, _ = lat.fields()
        fixed[dt] = (u, sec)
    n64 = float(np.linalg.norm(fixed["f64"][0]))
    out["cases"].append({
        "case": f"cavity 256^3, Re 1000, n 0.8, U 0.05, {args.precision_steps} steps from rest",
        "seconds": {k: v[1] for k, v in fixed.items()},
        "l2_vs_f64": {k: float(np.linalg.norm(fixed[k][0] - fixed["f64"][0])) / n64
                      for k in forms[1:]}})
    print(json.dumps(out))
    return 0


STABILITY_RATES = {
    "unit": None,                                   # Sec. 3.1: omega_9..18 = 1
    "w9=0.5": (0.5,) + (1.0,) * 9,                  # larger bulk viscosity
    "w9=1.5": (1.5,) + (1.0,) * 9,
    "w10-18=0.8": (1.0,) + (0.8,) * 9,              # under-relaxed 3rd/4th orders
    "w10-18=1.2": (1.0,) + (1.2,) * 9,              # over-relaxed 3rd/4th orders
    "w10-18=1.1": (1.0,) + (1.1,) * 9,
    "w10-18=1.3": (1.0,) + (1.3,) * 9,
    "w10-18=1.4": (1.0,) + (1.4,) * 9,
}
STABILITY_DEFAULT_SETS = ("unit", "w9=0.5", "w9=1.5", "w10-18=0.8", "w10-18=1.2")


def run_stability(args):
    """Stability limit of the cascaded scheme alone (Sec. 5, second study):
    the largest lid velocity a 64^3 cavity sustains for 50,000 steps, for
    n = 0.8, 1, 1.5, several tau_p and several sets of the rates omega_9..18,
    by bisection with all open cases of a round in one batch.  With
    --stability-confirm the FP64 form re-runs each bracket of one rate set
    (--stability-confirm-set, default the unit rates) at tau_p = 0.51 (the
    stable and the unstable end)."""
    import torch  # noqa: F401  (CUDA context on the chosen device)
    from paper_1908_05396_gb300 import build
    build.build()
    from paper_1908_05396_gb300 import stability as st
    sets = args.stability_sets or STABILITY_DEFAULT_SETS
    cases = [st.Case(n, tau, STABILITY_RATES[label], label) for label in sets
             for n in args.stability_n for tau in args.stability_tau]
    t0 = time.perf_counter()
    run = st.batch_runner(args.stability_L, args.stability_steps, args.stability_dtype)
    res = st.max_lid_velocity(cases, run, u_hi=args.stability_uhi, rounds=args.stability_rounds)
    sec = time.perf_counter() - t0
    out = {"metric": "max stable lid velocity", "L": args.stability_L,
           "steps": args.stability_steps, "dtype": args.stability_dtype,
           "u_hi": args.stability_uhi, "rounds": args.stability_rounds, "seconds": sec,
           "cases": [{"rates": c.label, "n": c.n, "tau_p": c.tau_p, "u_stable": lo,
                      "u_unstable": hi} for c, (lo, hi) in zip(cases, res)]}
    if args.stability_confirm:
        sel = [(c, r) for c, r in zip(cases, res)
               if c.label == args.stability_confirm_set and c.tau_p == 0.51 and r[1] is not None]
        pairs = [(c, u) for c, (lo, hi) in sel for u in (lo, hi) if u > 0.0]
        t0 = time.perf_counter()
        ok = st.batch_runner(args.stability_L, args.stability_steps, "f64")(
            [c for c, _ in pairs], [u for _, u in pairs])
        out["f64_confirm"] = {"seconds": time.perf_counter() - t0, "runs": [
            {"n": c.n, "tau_p": c.tau_p, "U": u, "stable": s} for (c, u), s in zip(pairs, ok)]}
    print(json.dumps(out))
    return 0


def run_precision_steady(args):
    """The precision configuration as written: the 256^3 cavity (Re 1000,
    n 0.8, U 0.05) run from rest to steady state (residual 1e-8) in the FP64
    form, which is the reference (its parity with the oracle is tested at
    1000 steps), and in the FP32, F16R and F16S forms, which run to the same
    residual or until it stops falling (20 reads without a 10 % drop).  The
    residual is checked over intervals of 2000 steps (R is a rate per step,
    so the tolerance keeps its meaning; the longer interval lowers the
    residual floor that the FP16 forms' rounding sets).  The velocity L2
    error of each form against FP64 at its own end is reported.  With
    --precision-f64-from T the FP64 run starts from the FP32 state after T
    steps instead of from rest (the two trajectories agree to the FP32
    rounding level, and the FP64 steps that follow damp that start-up
    difference with the flow's slowest mode), which shortens the FP64 run
    by T steps; the start is stated in the output."""
    import numpy as np
    import torch  # noqa: F401  (CUDA context on the chosen device)
    from paper_1908_05396_gb300 import build, workloads as wl
    build.build()
    from paper_1908_05396_gb300 import clbm
    prob = wl.cavity(256, 1000.0, 0.8)
    forms = list(args.precision_forms)
    res = {}
    warm = args.precision_f64_from
    if warm and "f64" in forms and "f32" in forms:
        # FP32 first, keeping its state at step `warm`; FP64 continues from it
        forms.remove("f32")
        forms.insert(0, "f32")
    snap = None
    for dt in forms:
        kw = {}
        if dt == "f32" and warm and "f64" in forms:
            kw["snapshot_at"] = warm
        if dt == "f64" and snap is not None:
            kw["start"] = (snap, warm)
        res[dt] = _run_to_steady(clbm, prob, dt, 1e-8, args.precision_cap, chunk=2000,
                                 check=2000, progress=10, **kw)
        if "snapshot" in res[dt][1]:
            snap = res[dt][1].pop("snapshot")
        if dt == "f64" and snap is not None:
            res[dt][1]["started_from"] = f"the FP32 state after {warm} steps"
            snap = None
        print(json.dumps({"form": dt, **res[dt][1]}), file=sys.stderr, flush=True)
    ref_form = "f64" if "f64" in res else forms[0]
    ref = res[ref_form][0]
    nref = float(np.linalg.norm(ref))
    print(json.dumps({
        "metric": "precision at steady state",
        "case": "cavity 256^3, Re 1000, n 0.8, U 0.05, from rest to R <= 1e-8 (check interval "
                "2000 steps; FP16 forms: or a residual plateau of 20 reads)"
                + (f"; FP64 from the FP32 state after {warm} steps" if warm else ""),
        "runs": {k: v[1] for k, v in res.items()},
        "reference": ref_form,
        f"l2_vs_{ref_form}": {k: float(np.linalg.norm(res[k][0] - ref)) / nref
                              for k in res if k != ref_form}}))
    return 0


def run_profile_batch(args):
    """The batch profiling case: the 64 seeded cavities in one FP32 batch."""
    import torch
    from paper_1908_05396_gb300 import build, workloads as wl
    build.build()
    from paper_1908_05396_gb300 import clbm
    probs = wl.batch_cavities(count=64, seed=0)
    lats = [clbm.Lattice(**p.kwargs(), dtype="f32") for p in probs]
    with clbm.Batch("f32", capacity=len(lats), check_interval=100) as b:
        for lt in lats:
            b.add(lt)
        if args.launch:
            b.set_launch(args.launch[0], args.launch[1], args.launch[2], args.batch_bps)
        b.step(args.warmup)
        b.sync()
        t0 = time.perf_counter()
        b.step(args.steps)
        b.sync()
        dt = time.perf_counter() - t0
    N = sum(p.N for p in probs)
    print(json.dumps({"case": "batch of 64 cavities f32", "steps": args.steps,
                      "MLUPS": N * args.steps / dt / 1e6}))
    for lt in lats:
        lt.close()
    return 0


def run_profile(args):
    """The profiling case: steps of one 128^3 cavity (n = 0.5) in one form."""
    import torch
    from paper_1908_05396_gb300 import build, workloads as wl
    build.build()
    from paper_1908_05396_gb300 import clbm
    stream = torch.cuda.Stream()
    lat = clbm.Lattice(**wl.cavity(L_BENCH, RE_BENCH, 0.5).kwargs(), dtype=args.profile,
                       stream=stream.cuda_stream)
    if args.launch:
        lat.set_launch(*args.launch)
    else:
        lat.autotune(10)
    lat.step(args.warmup)
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    lat.step(args.steps)
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    print(json.dumps({"case": f"{args.profile} 128^3 cavity n=0.5", "steps": args.steps,
                      "us_per_step": ms * 1e3 / args.steps,
                      "MLUPS": lat.N * args.steps / (ms * 1e-3) / 1e6}))
    lat.close()
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=4000)
    ap.add_argument("--warmup", type=int, default=20)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--forms", nargs="*", default=None)
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-extra", action="store_true",
                    help="skip the batched and serving measurements")
    ap.add_argument("--batch-steps", type=int, default=500)
    ap.add_argument("--serve-requests", type=int, default=32,
                    help="requests of the serving trace (configured sizes; --serve-steady: scaled)")
    ap.add_argument("--serve-cap", type=int, default=4000,
                    help="step cap of each served request in the default run")
    ap.add_argument("--serve-steady", action="store_true",
                    help="serving to steady state on a scaled trace, against sequential FP64")
    ap.add_argument("--precision", action="store_true",
                    help="velocity error of the FP32 / F16S forms against FP64")
    ap.add_argument("--precision-steps", type=int, default=2000)
    ap.add_argument("--precision-steady", action="store_true",
                    help="the 256^3 precision cavity run to steady state (FP64, FP32, F16R, F16S)")
    ap.add_argument("--precision-cap", type=int, default=600_000,
                    help="step cap of each --precision-steady run")
    ap.add_argument("--precision-f64-from", type=int, default=0,
                    help="--precision-steady: start FP64 from the FP32 state after this many "
                         "steps (0: from rest)")
    ap.add_argument("--precision-forms", nargs="*", default=["f64", "f32", "f16r", "f16s", "f16s_sr"],
                    choices=["f64", "f32", "f16r", "f16s", "f16s_sr"],
                    help="forms of --precision-steady, the first the reference unless FP64 runs")
    ap.add_argument("--profile-batch", action="store_true",
                    help="time only the batch of 64 cavities (profiling case)")
    ap.add_argument("--batch-bps", type=int, default=4,
                    help="profiling case: blocks per SM of the batch (negative: capped)")
    ap.add_argument("--launch", type=int, nargs=3, default=None,
                    metavar=("BX", "BY", "NPT"), help="profiling case: fixed launch shape")
    ap.add_argument("--profile", nargs="?", const="f32", default=None,
                    choices=["f64", "f32", "f16s", "f16r"],
                    help="time only the steps of the n=0.5 cavity in one storage form "
                         "(profiling case)")
    ap.add_argument("--stability", action="store_true",
                    help="largest stable lid velocity of the cavity per (n, tau_p, rates)")
    ap.add_argument("--stability-L", type=int, default=64)
    ap.add_argument("--stability-steps", type=int, default=50_000)
    ap.add_argument("--stability-tau", type=float, nargs="*", default=[0.505, 0.51, 0.52, 0.55])
    ap.add_argument("--stability-sets", nargs="*", default=None, choices=list(STABILITY_RATES),
                    help="rate sets to sweep (default: the five of the committed table)")
    ap.add_argument("--stability-n", type=float, nargs="*", default=[0.8, 1.0, 1.5])
    ap.add_argument("--stability-uhi", type=float, default=0.25,
                    help="upper end of the bisection (the library takes |U_lid| < 0.3)")
    ap.add_argument("--stability-rounds", type=int, default=8)
    ap.add_argument("--stability-dtype", default="f32", choices=["f64", "f32"])
    ap.add_argument("--stability-confirm", action="store_true",
                    help="re-run the brackets at tau_p = 0.51 of one rate set in FP64")
    ap.add_argument("--stability-confirm-set", default="unit", choices=list(STABILITY_RATES))
    ap.add_argument("--oracle-one-core", action="store_true", help=argparse.SUPPRESS)
    args = ap.parse_args()
    if args.oracle_one_core:
        return run_oracle_one_core()
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        return run_reference(args)
    if args.profile_batch:
        return run_profile_batch(args)
    if args.precision:
        return run_precision(args)
    if args.precision_steady:
        return run_precision_steady(args)
    if args.serve_steady:
        if args.serve_requests == 32:
            args.serve_requests = 48
        return run_serve_steady(args)
    if args.stability:
        return run_stability(args)
    if args.profile:
        return run_profile(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
