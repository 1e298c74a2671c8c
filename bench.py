#!/usr/bin/env python
"""Benchmark of the GB300-native ASUCA-style RK3 step.

Metric: grid-cell updates per second per RK3 step (one step = three RK stage
sweeps + the column pass + FP64 budgets), on the 1024x1024x58, 8-tracer
workload with FP32 fields and stencils and an FP64 Thomas solve and sums; the
all-FP64 path is timed on the same workload beside it.  Inputs are seeded
synthetic fields (gen/), resident in HBM when the timed region starts; the
2.4 GB state is larger than L2, so no flush is needed between steps.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

--impl reference times the FP64 CPU oracle (test infrastructure) on the host
cores, each step a bounded sample of the same workload.  Under torchrun
(N > 1) every rank advances its own replica (no data-path collective; weak
scaling) and rank 0 prints one JSON line.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "cell-updates/s per RK3 step (FP32 vs FP64), % HBM roofline; adjoint/fwd cost"
UNIT = "cell-updates/s"
WORKLOAD = "large_1024x1024x58"


def _peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as fh:
            d = json.load(fh)
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


def _recorded(kernel, key, cells):
    """A per-cell figure (`key`) of `kernel` from the recorded ncu captures
    (profiles/traffic.json), scaled to `cells`; None when the record is missing
    or the kernel's sources changed since."""
    import hashlib
    p = os.path.join(ROOT, "profiles", "traffic.json")
    try:
        with open(p) as fh:
            rec = json.load(fh)[kernel]
        h = hashlib.sha256()
        for f in rec["sources"]:
            with open(os.path.join(ROOT, "paper_1710_08616_gb300", "csrc", f), "rb") as fh:
                h.update(fh.read())
        if h.hexdigest()[:16] != rec["source_sha256_16"]:
            return None
        return rec[key] * cells
    except (OSError, KeyError, ValueError):
        return None


def _recorded_traffic(kernel, cells):
    """DRAM bytes per launch of `kernel` (dram__bytes_read.sum + dram__bytes_write.sum)."""
    return _recorded(kernel, "bytes_per_cell", cells)


def _floor_and_dram(kern, F, s, C, ms, steps, peak):
    """Two more fractions of the measured HBM peak over the timed region (ms for
    `steps` steps of C cells): the compulsory floor (read the state and M once,
    write the state once: 2F+3 values per cell and step), and the DRAM rate the
    recorded ncu traffic of the timed launches implies (kern: the per-kernel
    report, each with its launches and recorded bytes per launch; None when a
    kernel that moves algorithmic bytes has no current record)."""
    out = {"floor_bytes_per_cell": (2 * F + 3) * s, "floor_frac": None, "dram_gbs_ncu": None,
           "dram_frac_ncu": None}
    try:
        out["floor_frac"] = (2 * F + 3) * s * C * steps / (ms * 1e-3) / 1e9 / peak
        total = 0.0
        for v in kern.values():
            if v.get("algo_bytes_per_launch", 0.0) > 0.0:
                t = v.get("traffic_bytes_per_launch")
                if t is None:
                    return out
                total += t * v["launches"]
        if total > 0.0:
            out["dram_gbs_ncu"] = total / (ms * 1e-3) / 1e9
            out["dram_frac_ncu"] = out["dram_gbs_ncu"] / peak
    except (ArithmeticError, KeyError, TypeError, ValueError):
        pass
    return out


# FP64 pipe: 2 DFMA/DADD/DMUL per clock per SM (ncu's
# sm__sass_thread_inst_executed_op_dfma_pred_on peak), 152 SMs, 2070 MHz maximum clock
FP64_INST_PEAK = 2 * 152 * 2.07e9


# ---------------------------------------------------------------- clocks

class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_id: str):
        self.gpu_id = gpu_id
        self.proc = None
        self.path = None

    def start(self):
        try:
            import tempfile
            fd, self.path = tempfile.mkstemp(prefix="asuca_clocks_", suffix=".csv")
            self.fh = os.fdopen(fd, "w")
            self.proc = subprocess.Popen(["nvidia-smi", "-i", self.gpu_id, f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=self.fh, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
        time.sleep(0.3)

    def stop(self):
        if self.proc is None:
            if self.path:
                try:
                    self.fh.close()
                    os.remove(self.path)
                except OSError:
                    pass
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.3)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.fh.close()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        with open(self.path) as fh:
            for line in fh:
                parts = [x.strip() for x in line.split(",")]
                if len(parts) < 9:
                    continue
                try:
                    sm.append(float(parts[1]))
                    smax.append(float(parts[2]))
                except ValueError:
                    continue
                for nm, v in zip(names, parts[5:9]):
                    if v.lower().startswith("active"):
                        reasons.add(nm)
        try:
            os.remove(self.path)
        except OSError:
            pass
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "samples": len(sm), "reasons": sorted(reasons)}


# ---------------------------------------------------------------- helpers

def _dist():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def _barrier(ws):
    if ws > 1:
        import torch.distributed as dist
        dist.barrier()


def _max_over_ranks(ws, v):
    if ws == 1:
        return v
    import torch
    import torch.distributed as dist
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([v], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def _gpu_local_cpus(gpu_id: str):
    """The CPUs of the GPU's host NUMA node (its PCI function's local_cpulist),
    or None when nvidia-smi or sysfs do not say."""
    try:
        out = subprocess.run(["nvidia-smi", "-i", gpu_id, "--query-gpu=pci.bus_id", "--format=csv,noheader"],
                             capture_output=True, text=True, timeout=20).stdout.strip().splitlines()[0].lower()
        dom, rest = out.split(":", 1)
        with open(f"/sys/bus/pci/devices/{int(dom, 16):04x}:{rest}/local_cpulist") as fh:
            txt = fh.read().strip()
        cpus = set()
        for part in txt.split(","):
            a, _, b = part.partition("-")
            cpus.update(range(int(a), int(b or a) + 1))
        return cpus & os.sched_getaffinity(0) or None
    except Exception:
        return None


def _link_gbs(dev, nbytes=1 << 30, reps=3):
    """Pinned host <-> device copy rates (GB/s): host to device, device to
    host, and each direction while both run at once (two streams)."""
    import torch
    h = torch.empty(nbytes, dtype=torch.uint8).pin_memory()
    h2 = torch.empty(nbytes, dtype=torch.uint8).pin_memory()
    d = torch.empty(nbytes, dtype=torch.uint8, device=dev)
    d2 = torch.empty(nbytes, dtype=torch.uint8, device=dev)
    sa, sb = torch.cuda.Stream(), torch.cuda.Stream()

    def run(pairs):
        best = None
        for _ in range(reps):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            for (dst, src), sx in zip(pairs, (sa, sb)):
                with torch.cuda.stream(sx):
                    dst.copy_(src, non_blocking=True)
            torch.cuda.synchronize()
            el = time.perf_counter() - t0
            best = el if best is None else min(best, el)
        return nbytes / best / 1e9

    out = {"h2d": run([(d, h)]), "d2h": run([(h, d)])}
    out["each_way_concurrent"] = run([(d, h), (h2, d2)])
    del h, h2, d, d2
    return out


def cpu_oracle_rate(min_seconds=10.0, nx=256, ny=256, steps_cap=50):
    """The FP64 oracle as it stands on the host cores: 256x256x58, 8 tracers."""
    import gen
    import oracle
    case = gen.make_case(nx, ny, 58, 8, seed=gen.SEED_BASE + 4)
    g = oracle.Grid.from_case(case)
    Y = case.state()
    oracle.step(g, Y, case.mu, case.mv, case.mw, case.dt, 1)       # warm, builds the library
    t0 = time.perf_counter()
    n = 0
    while True:
        Y, _ = oracle.step(g, Y, case.mu, case.mv, case.mw, case.dt, 1)
        n += 1
        el = time.perf_counter() - t0
        if el >= min_seconds or n >= steps_cap:
            break
    out = {"value": case.cells * n / el, "unit": UNIT, "cores": oracle.get_threads(),
           "kind": "oracle",
           "sample": f"{n} step(s) of a {nx}x{ny}x58 periodic domain with 8 tracers (same per-cell "
                     f"work as the 1024x1024x58 workload), {el:.1f} s, FP64, OpenMP over j"}
    out["single_thread"] = _cpu_oracle_rate_one_thread(min_seconds / 2, steps_cap)
    out["host"] = _host_cpu()
    return out


def _host_cpu():
    """The host's processor model (lscpu, where present), architecture and
    logical CPU count."""
    import platform
    import subprocess
    model = None
    try:
        r = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10)
        for line in r.stdout.splitlines():
            if line.lower().startswith("model name"):
                model = line.split(":", 1)[1].strip()
                break
    except (OSError, subprocess.SubprocessError):
        pass
    return {"cpu_model": model, "arch": platform.machine(), "logical_cpus": os.cpu_count()}


def _cpu_oracle_rate_one_thread(min_seconds, steps_cap, n=128):
    """The same oracle step on one host thread, on an n x n x 58 sample (None
    if it cannot be timed); the thread count is restored afterwards."""
    import gen
    import oracle
    threads = oracle.get_threads()
    try:
        oracle.set_threads(1)
        case = gen.make_case(n, n, 58, 8, seed=gen.SEED_BASE + 4)
        g = oracle.Grid.from_case(case)
        Y = case.state()
        t0 = time.perf_counter()
        k = 0
        while True:
            Y, _ = oracle.step(g, Y, case.mu, case.mv, case.mw, case.dt, 1)
            k += 1
            el = time.perf_counter() - t0
            if el >= min_seconds or k >= steps_cap:
                break
        return {"value": case.cells * k / el, "unit": UNIT, "cores": 1,
                "sample": f"{k} step(s) of a {n}x{n}x58 periodic domain with 8 tracers, {el:.1f} s, FP64"}
    except (OSError, RuntimeError, ValueError, ArithmeticError):
        return None
    finally:
        oracle.set_threads(threads)


# ---------------------------------------------------------------- reference arm

def run_reference(args):
    ws, rank, _ = _dist()
    if rank != 0:
        return 0
    import gen
    import oracle
    nx = ny = args.ref_n
    case = gen.make_case(nx, ny, 58, 8, seed=gen.SEED_BASE + 4)
    g = oracle.Grid.from_case(case)
    Y = case.state()
    for _ in range(args.warmup):
        Y, _b = oracle.step(g, Y, case.mu, case.mv, case.mw, case.dt, 1)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        Y, _b = oracle.step(g, Y, case.mu, case.mv, case.mw, case.dt, 1)
    el = time.perf_counter() - t0
    value = case.cells * args.steps / el
    cores = oracle.get_threads()
    sample = (f"each step: one oracle RK3 step of a {nx}x{ny}x58 periodic domain with 8 tracers "
              f"(the 1024x1024x58 workload's per-cell work on a bounded sample), FP64")
    out = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": el / args.steps * 1e3, "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
           "impl": "reference",
           "config": {"workload": WORKLOAD, "sample": f"{nx}x{ny}x58", "ntracers": 8,
                      "precision": "fp64 (CPU oracle)"},
           "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                            "sample": sample},
           "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out), flush=True)
    return 0


# ---------------------------------------------------------------- our arm

def _time_steps(asuca, g, st, dt, ws_t, bud, steps, warmup, world, profile=False):
    import torch
    for _ in range(warmup):
        asuca.step(g, st, dt, 1, workspace=ws_t, budgets=bud)
    torch.cuda.synchronize()
    if profile:
        asuca.profile_enable(g, True)
    stream = torch.cuda.current_stream()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    _barrier(world)
    torch.cuda.synchronize()
    e0.record(stream)
    for _ in range(steps):
        asuca.step(g, st, dt, 1, workspace=ws_t, budgets=bud)
    e1.record(stream)
    torch.cuda.synchronize()
    _barrier(world)
    ms = e0.elapsed_time(e1)
    prof = asuca.profile_read(g) if profile else None
    if profile:
        asuca.profile_enable(g, False)
    assert asuca.get_status(g) == asuca.OK
    return ms, prof


def adjoint_cost(asuca, dev, reps=3):
    """Adjoint cost on the 128x128x58, 4-tracer workload, 50 steps, checkpoints
    every 10 steps, FP64 and FP32, against the wall time of asuca_step for the
    same 50 steps:
      * backward: asuca_adjoint_from_checkpoints (what AdjointFn.backward runs:
        each segment recomputed from the checkpoints AdjointFn.forward kept,
        then reversed); adjoint_over_forward = backward / forward;
      * the forward with checkpoints (asuca_forward_checkpointed, AdjointFn.forward);
      * standalone asuca_adjoint_step, which also runs the checkpointing forward pass."""
    import torch
    import gen
    case = gen.make_config_case("adjoint_128x128x58")
    nsteps, K = gen.CONFIGS["adjoint_128x128x58"]["nsteps"], 10
    out = {"workload": "adjoint_128x128x58", "nsteps": nsteps, "checkpoint_every": K}
    from paper_1710_08616_gb300 import autotune
    for name, prec in (("fp64", asuca.FP64), ("fp32", asuca.FP32_MIXED)):
        g = asuca.Grid.from_case(case, prec=prec)
        st0 = asuca.State.from_case(case, prec=prec, device=dev)
        # the forward it is compared with runs in its fastest launch configuration
        tuned = autotune.tune_step(g, st0, case.dt, steps=2, reps=2, save=False)["best"]
        ws = g.workspace(device=dev)
        nadj = asuca.adjoint_workspace_bytes(g, nsteps, K)
        wsa = torch.empty(nadj, dtype=torch.uint8, device=dev)
        ckb = torch.empty(max(asuca.checkpoint_bytes(g, nsteps, K), 256), dtype=torch.uint8, device=dev)
        lam = torch.randn((case.nfields,) + tuple(st0.rho.shape), dtype=g.torch_dtype, device=dev).contiguous()

        def timed(fn):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            fn()
            e1.record()
            torch.cuda.synchronize()
            return e0.elapsed_time(e1)

        s_ = st0.clone()

        def reset():
            for a_, b_ in zip((s_.rho, s_.rhotheta, s_.rhoq), (st0.rho, st0.rhotheta, st0.rhoq)):
                a_.copy_(b_)

        fwd = lambda: asuca.step(g, s_, case.dt, nsteps, workspace=ws)
        fwd_ck = lambda: asuca.forward_checkpointed(g, s_, case.dt, nsteps, checkpoint_every=K, workspace=ws,
                                                     checkpoints=ckb)
        bwd = lambda: asuca.adjoint_from_checkpoints(g, ckb, st0, case.dt, nsteps, lam, checkpoint_every=K,
                                                     workspace=wsa)
        alone = lambda: asuca.adjoint_step(g, st0, case.dt, nsteps, lam, checkpoint_every=K, workspace=wsa)

        def best(fn):
            r = []
            for _ in range(reps):
                reset()
                torch.cuda.synchronize()
                r.append(timed(fn))
            return min(r)

        for fn in (fwd, fwd_ck, bwd, alone):
            reset()
            fn()
        torch.cuda.synchronize()
        tf, tfc = best(fwd), best(fwd_ck)
        reset()
        fwd_ck()
        torch.cuda.synchronize()
        asuca.profile_enable(g, True)
        tb = min(timed(bwd) for _ in range(reps))
        prof = asuca.profile_read(g)
        asuca.profile_enable(g, False)
        ta = min(timed(alone) for _ in range(reps))
        assert asuca.get_status(g) == asuca.OK
        names = {0: "stage", 1: "column", 2: "budget_reduce", 3: "adj_stage", 4: "adj_column"}
        out[name] = {"forward_config": tuned, "forward_ms": tf, "forward_checkpointed_ms": tfc, "backward_ms": tb,
                     "adjoint_over_forward": tb / tf,
                     "forward_plus_backward_over_forward": (tfc + tb) / tf,
                     "standalone_adjoint_step_ms": ta, "standalone_over_forward": ta / tf,
                     "backward_kernels_ms_per_call": {names.get(k, str(k)): v[0] / reps for k, v in prof.items()}}
        del st0, ws, wsa, lam, ckb, s_
        torch.cuda.empty_cache()
    return out


PRECISION = "precision_256x256x58"


def _oracle_precision_job(path, threads):
    """Child process: the oracle's 100 steps of the precision workload, saved to path (.npy)."""
    import gen
    import oracle
    if threads:
        oracle.set_threads(threads)
    case = gen.make_config_case(PRECISION)
    g = oracle.Grid.from_case(case)
    Y, _ = oracle.step(g, case.state(), case.mu, case.mv, case.mw, case.dt, gen.CONFIGS[PRECISION]["nsteps"])
    np.save(path, Y)


def start_oracle_precision():
    """Start the oracle's run of the precision workload in a spawned process
    (the host cores are otherwise idle while the GPU reports run); returns a
    handle for precision_report."""
    import multiprocessing as mp
    import tempfile
    fd, path = tempfile.mkstemp(prefix="asuca_oracle_precision_", suffix=".npy")
    os.close(fd)
    threads = max(1, (os.cpu_count() or 2) - 2)     # leave the launching thread a core
    proc = mp.get_context("spawn").Process(target=_oracle_precision_job, args=(path, threads))
    proc.start()
    return {"proc": proc, "path": path, "threads": threads, "t0": time.perf_counter()}


def _field_errors(a, b, names):
    out = {}
    for f, nm in enumerate(names):
        d = a[f] - b[f]
        out[nm] = {"rel_l2": float(np.linalg.norm(d) / np.linalg.norm(b[f])),
                   "rel_max": float(np.abs(d).max() / np.abs(b[f]).max())}
    return out


def precision_report(asuca, dev, oracle_job=None):
    """256x256x58, 6 tracers, 100 steps from the same initial state in FP32-mixed
    and in FP64 on the GPU and in the FP64 oracle: per-field relative L2 and max
    error of both GPU paths against the oracle (rho, rho*theta, each rho*q_n and
    theta' = theta - theta_ref, the perturbation that rho*theta's magnitude
    hides), FP32 against the GPU FP64 path, and the drift of the FP64 budgets
    over the run (mass; each tracer plus its precipitation for the sedimenting
    one) in both precisions."""
    import torch
    import gen
    name = PRECISION
    case = gen.make_config_case(name)
    nsteps = gen.CONFIGS[name]["nsteps"]
    res, buds, times = {}, {}, {}
    for label, prec in (("fp64", asuca.FP64), ("fp32", asuca.FP32_MIXED)):
        g = asuca.Grid.from_case(case, prec=prec)
        st = asuca.State.from_case(case, prec=prec, device=dev)
        b0 = asuca.step(g, st, case.dt, 0, budgets=True).cpu().numpy()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        b1 = asuca.step(g, st, case.dt, nsteps, budgets=True)
        e1.record()
        torch.cuda.synchronize()
        assert asuca.get_status(g) == asuca.OK
        times[label] = e0.elapsed_time(e1) / nsteps
        res[label] = st.fields().double().cpu().numpy()
        buds[label] = (b0, b1.cpu().numpy())
    names = ["rho", "rhotheta"] + [f"rhoq{n + 1}" for n in range(case.ntracers)]
    errs = _field_errors(res["fp32"], res["fp64"], names)
    drift = {}
    F = case.nfields
    for label, (b0, b1) in buds.items():
        tr = b1[2:F].copy()
        tr[-1] += b1[F]      # the sedimenting (last) tracer: mass aloft + precipitation
        drift[label] = {"mass": float((b1[0] - b0[0]) / b0[0]),
                        "tracers_plus_precip": [float(v) for v in (tr - b0[2:F]) / b0[2:F]]}
    out = {"workload": name, "nsteps": nsteps, "fp32_vs_fp64_gpu": errs, "budget_drift": drift,
           "ms_per_step": times, "fp32_over_fp64_speedup": times["fp64"] / times["fp32"]}
    if oracle_job is not None:
        oracle_job["proc"].join()
        if oracle_job["proc"].exitcode == 0:
            ref = np.load(oracle_job["path"])
            zf = np.concatenate([[0.0], np.cumsum(case.dz)])
            thref = (300.0 + 0.004 * (zf[:-1] + 0.5 * case.dz))[:, None, None]
            prime = lambda Y: Y[1] / Y[0] - thref

            def vs_oracle(Y):
                e = _field_errors(Y, ref, names)
                d = prime(Y) - prime(ref)
                e["theta_prime"] = {"rel_l2": float(np.linalg.norm(d) / np.linalg.norm(prime(ref))),
                                    "rel_max": float(np.abs(d).max() / np.abs(prime(ref)).max())}
                return e

            out["fp32_vs_oracle"] = vs_oracle(res["fp32"])
            out["fp64_vs_oracle"] = vs_oracle(res["fp64"])
            out["oracle"] = {"threads": oracle_job["threads"],
                             "wall_s_incl_waiting": time.perf_counter() - oracle_job["t0"]}
        else:
            out["oracle"] = {"failed": f"exit code {oracle_job['proc'].exitcode}"}
        try:
            os.remove(oracle_job["path"])
        except OSError:
            pass
    return out


def layout_ablation(asuca, dev, reps=10):
    """The reduced weather application's 7-point diffusion step (Sec. 4) on the
    1024x1024x58 rho*theta field, same kernel and thread mapping in IJK (i fastest)
    and KIJ (k fastest) storage (Sec. 1.3: KIJ 7.7x slower on GPU), FP32 and FP64.
    Reported against the paper's two bandwidth models at the measured HBM peak:
    perfect cache (read and write each value once) and no cache (7 reads + 1
    write per cell).  The 243 MB (FP32) field is larger than L2."""
    import torch
    import gen
    case = gen.make_config_case(WORKLOAD)
    peak, _ = _peaks()
    C = case.cells
    out = {"workload": "stencil7_1024x1024x58", "paper_kij_over_ijk": 7.7}
    for name, dt in (("fp32", torch.float32), ("fp64", torch.float64)):
        s = dt.itemsize
        f = torch.tensor(case.rhotheta, dtype=dt, device=dev).contiguous()
        res = {}
        for lname, layout in (("ijk", asuca.LAYOUT_IJK), ("kij", asuca.LAYOUT_KIJ)):
            x = f if layout == asuca.LAYOUT_IJK else f.permute(1, 2, 0).contiguous()
            y = torch.empty_like(x)
            for _ in range(3):
                asuca.stencil7(x, y, 0.1, layout)
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            for _ in range(reps):
                asuca.stencil7(x, y, 0.1, layout)
            e1.record()
            torch.cuda.synchronize()
            ms = e0.elapsed_time(e1) / reps
            t_perfect = 2 * s * C / (peak * 1e9) * 1e3
            t_nocache = 8 * s * C / (peak * 1e9) * 1e3
            res[lname] = {"ms": ms, "achieved_gbs_perfect_cache_bytes": 2 * s * C / (ms * 1e-3) / 1e9,
                          "frac_of_perfect_cache_model": t_perfect / ms,
                          "speedup_over_no_cache_model": t_nocache / ms}
            del x, y
        res["kij_over_ijk"] = res["kij"]["ms"] / res["ijk"]["ms"]
        out[name] = res
        del f
    torch.cuda.empty_cache()
    return out


def damping_report(asuca, dev, reps=10, nx=None, precs=("fp32", "fp64")):
    """Lateral and upper damping toward boundary data (asuca_damping) on the
    1024x1024x58, 8-tracer state with the workload's zone (16 edge cells, top 8
    levels), FP32 and FP64.  The kernel streams ref, bnd0, bnd1 and the state in
    and the state out for every zone cell: 5 F values per zone cell, against the
    measured HBM peak.  Its inputs (1.7 GB FP32 per launch) exceed L2."""
    import torch
    import gen
    case = gen.make_config_case(WORKLOAD, nx=nx, ny=nx)
    D = gen.DAMPING
    peak, _ = _peaks()
    nx, ny, nz, W, ntop, F = case.nx, case.ny, case.nz, D["width"], D["ntop"], case.nfields
    zone = ntop * nx * ny + (nz - ntop) * (nx * ny - (nx - 2 * W) * (ny - 2 * W))
    Y = case.state()
    bnd = [torch.from_numpy(a).to(dev) for a in gen.make_boundary_data(Y, case.seed + 17)]
    out = {"workload": f"damping_{nx}x{ny}x{nz}_width{W}_top{ntop}", "zone_cells": zone,
           "zone_fraction": zone / case.cells, "algorithmic_bytes": "5 F values per zone cell"}
    for name, prec, dt in (("fp32", asuca.FP32_MIXED, torch.float32), ("fp64", asuca.FP64, torch.float64)):
        if name not in precs:
            continue
        g = asuca.Grid.from_case(case, prec=prec)
        st = asuca.State.from_case(case, prec=prec, device=dev)
        ref, b0, b1 = (b.to(dt) for b in bnd)
        call = lambda: asuca.damping(g, st, ref, b0, b1, D["tratio"], case.dt, width=W, ntop=ntop,
                                     nu_lat=D["nu_lat"], nu_top=D["nu_top"])
        for _ in range(3):
            call()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(reps):
            call()
        e1.record()
        torch.cuda.synchronize()
        assert asuca.get_status(g) == asuca.OK
        ms = e0.elapsed_time(e1) / reps
        algo = 5 * F * dt.itemsize * zone
        out[name] = {"ms": ms, "launches": reps, "achieved_gbs": algo / (ms * 1e-3) / 1e9,
                     "frac": algo / (ms * 1e-3) / 1e9 / peak, "peak_gbs": peak}
        del st, ref, b0, b1
    del bnd
    torch.cuda.empty_cache()
    return out


def open_report(asuca, dev, case, reps=3):
    """Open lateral boundaries on the 1024x1024x58, 8-tracer state, FP32, against
    the periodic step on the same state:
      * limited area (asuca_step_open): every stage's ghosts filled from two
        boundary datasets interpolated in time (gen.make_open_boundary), the
        outer faces' own fluxes; per step three ghost fills and a prepare
        launch more than the periodic step;
      * decomposed: the domain as 2 x 2 blocks of 512 x 512 on this GPU, halos
        of width 2 exchanged by device copies before every stage
        (distributed.step_decomposed: pack, copy, unpack); the time a
        multi-GPU run would add for the exchange is the copies' time here plus
        the link's."""
    import torch
    import gen
    from paper_1710_08616_gb300.distributed import Block, Decomposition, step_decomposed
    prec, dt_ = asuca.FP32_MIXED, torch.float32
    t = lambda a: torch.as_tensor(np.array(a, copy=True)).to(device=dev, dtype=dt_).contiguous()

    def best(fn, nsteps):
        fn(1)
        torch.cuda.synchronize()
        r = []
        for _ in range(reps):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            fn(nsteps)
            e1.record()
            torch.cuda.synchronize()
            r.append(e0.elapsed_time(e1) / nsteps)
        return min(r)

    g = asuca.Grid.from_case(case, prec=prec)
    st = asuca.State.from_case(case, prec=prec, device=dev)
    ws = g.workspace(device=dev)
    t_per = best(lambda n: asuca.step(g, st, case.dt, n, workspace=ws), 5)
    del ws
    mu_x, mv_x = gen.extend_fluxes(case.mu, case.mv)
    sto = asuca.State(st.rho, st.rhotheta, st.rhoq, t(mu_x), t(mv_x), st.mw)
    b0, b1 = (t(b) for b in gen.make_open_boundary(case, seed=case.seed + 1))
    wso = asuca.open_workspace(g, device=dev)
    t_open = best(lambda n: asuca.step_open(g, sto, case.dt, n, b0, bnd1=b1, tratio=0.3, workspace=wso), 5)
    assert asuca.get_status(g) == asuca.OK
    del sto, wso, b0, b1, mu_x, mv_x
    torch.cuda.empty_cache()
    d = Decomposition(case.nx, case.ny, 2, 2)
    blocks = {}
    for r in range(d.nblocks):
        rx, ry = d.coords(r)
        sd = gen.subdomain(case, 2, 2, rx, ry)
        gb = asuca.Grid(sd["nx"], sd["ny"], case.nz, case.ntracers, case.dz, case.dx, case.dy, prec=prec)
        Y = sd["Y"]
        blocks[r] = Block(gb, asuca.State(t(Y[0]), t(Y[1]), t(Y[2:]), t(sd["mu_x"]), t(sd["mv_x"]), t(sd["mw"])))
    t_dec = best(lambda n: step_decomposed(blocks, d, case.dt, n), 3)
    for b in blocks.values():
        assert asuca.get_status(b.grid) == asuca.OK
    halo = sum(asuca.halo_count(b.grid) for b in blocks.values()) * 4
    del blocks
    torch.cuda.empty_cache()
    C = case.cells
    return {"workload": "large_1024x1024x58 fp32", "periodic_ms_per_step": t_per,
            "limited_area": {"ms_per_step": t_open, "cell_updates_per_s": C / (t_open * 1e-3),
                             "over_periodic": t_open / t_per},
            "decomposed_2x2_one_gpu": {"ms_per_step": t_dec, "cell_updates_per_s": C / (t_dec * 1e-3),
                                       "over_periodic": t_dec / t_per,
                                       "halo_bytes_per_stage": halo,
                                       "exchange": "device copies between the blocks' halo buffers"}}


def hevi_report(asuca, dev, case, reps=3):
    """The long step with nested acoustic short steps (asuca_step_hevi) on the
    1024x1024x58 grid with 8 tracers: 12 s long step, 6 short steps (2, 3 and 6
    per RK stage: 11 short steps per long step), FP32 and FP64.  Algorithmic
    values per cell and long step: the stage model (10 F + 8) plus, per short
    step, the 18 of the acoustic kernels and 8 of the mean-flux accumulation,
    plus 2 for the acoustic density perturbation at the start: 396 at F = 10."""
    import torch
    import gen
    peak, _ = _peaks()
    Y, U, V, W, r0c, r0f, dt, ns = gen.make_hevi_state(case)
    A = gen.ACOUSTIC
    nshort_total = sum(max(1, int(np.floor(fr * ns + 0.5))) for fr in (1 / 3, 1 / 2, 1.0))
    F = case.nfields
    values = (10 * F + 8) + 26 * nshort_total + 2
    out = {"workload": "hevi_1024x1024x58", "dt_s": dt, "short_steps_per_long_step": nshort_total,
           "algorithmic_values_per_cell": values}
    names = {asuca.KERNEL_STAGE: "stage", asuca.KERNEL_COLUMN: "column", asuca.KERNEL_REDUCE: "budget_reduce",
             asuca.KERNEL_STAGE_COLUMN: "stage3_column", asuca.KERNEL_ACOUSTIC: "acoustic"}
    for name, prec, dt_ in (("fp32", asuca.FP32_MIXED, torch.float32), ("fp64", asuca.FP64, torch.float64)):
        t = lambda a: torch.as_tensor(np.array(a, copy=True)).to(device=dev, dtype=dt_).contiguous()
        g = asuca.Grid.from_case(case, prec=prec)
        st = asuca.State(t(Y[0]), t(Y[1]), t(Y[2:]), t(U), t(V), t(W))
        ws = torch.empty(asuca.hevi_workspace_bytes(g), dtype=torch.uint8, device=dev)
        nsteps = 3 if name == "fp32" else 1
        asuca.step_hevi(g, st, dt, 1, r0c, r0f, A["cs2"], A["beta"], ns, workspace=ws)
        torch.cuda.synchronize()
        best, prof = None, None
        for _ in range(reps):
            asuca.profile_enable(g, True)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            asuca.step_hevi(g, st, dt, nsteps, r0c, r0f, A["cs2"], A["beta"], ns, workspace=ws)
            e1.record()
            torch.cuda.synchronize()
            ms = e0.elapsed_time(e1) / nsteps
            p_ = asuca.profile_read(g)
            asuca.profile_enable(g, False)
            if best is None or ms < best:
                best, prof = ms, p_
        assert asuca.get_status(g) == asuca.OK
        s = dt_.itemsize
        out[name] = {"ms_per_step": best, "cell_updates_per_s": case.cells / (best * 1e-3),
                     "frac": values * s * case.cells / (best * 1e-3) / 1e9 / peak,
                     "kernels_ms_per_step": {names.get(k, str(k)): v[0] / nsteps for k, v in prof.items()}}
        del st, ws
        torch.cuda.empty_cache()
    return out


def acoustic_report(asuca, dev, reps=5, nx=None, precs=("fp32", "fp64")):
    """HEVI acoustic short steps (asuca_acoustic_steps) on the 1024x1024x58 grid,
    6 short steps of 2 s per call, FP32 and FP64.  A short step is two launches,
    one thread per column each; the algorithmic bytes count every array once per
    launch: stage 1 reads S, U, V, W and writes U*, V*, s* (7 values per cell),
    stage 2 reads S, W, U, V, s*, U*, V* and writes U, V, W, S (11): 18 values
    per cell and short step, against the measured HBM peak.  The 4 fields
    (1 GB in FP32) exceed L2."""
    import torch
    import gen
    case = gen.make_config_case(WORKLOAD, nx=nx, ny=nx, ntracers=1)
    A = gen.ACOUSTIC
    peak, _ = _peaks()
    C = case.cells
    arrays = gen.make_acoustic_state(case)
    out = {"workload": f"acoustic_{case.nx}x{case.ny}x{case.nz}", "nshort_per_call": A["nshort"],
           "dtau_s": A["dtau"], "beta": A["beta"], "algorithmic_bytes": "18 values per cell and short step"}
    for name, prec, dt in (("fp32", asuca.FP32_MIXED, torch.float32), ("fp64", asuca.FP64, torch.float64)):
        if name not in precs:
            continue
        g = asuca.Grid.from_case(case, prec=prec)
        U, V, W, S = (torch.from_numpy(np.ascontiguousarray(a)).to(device=dev, dtype=dt) for a in arrays[:4])
        ws = torch.empty(asuca.acoustic_workspace_bytes(g), dtype=torch.uint8, device=dev)
        call = lambda: asuca.acoustic_steps(g, U, V, W, S, arrays[4], arrays[5], A["cs2"], A["beta"], A["dtau"],
                                            A["nshort"], workspace=ws)
        for _ in range(3):
            call()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(reps):
            call()
        e1.record()
        torch.cuda.synchronize()
        assert asuca.get_status(g) == asuca.OK
        ms = e0.elapsed_time(e1) / (reps * A["nshort"])
        algo = 18 * dt.itemsize * C
        out[name] = {"ms_per_short_step": ms, "launches": 2 * reps * A["nshort"],
                     "cell_updates_per_s": C / (ms * 1e-3), "achieved_gbs": algo / (ms * 1e-3) / 1e9,
                     "frac": algo / (ms * 1e-3) / 1e9 / peak, "peak_gbs": peak}
        del U, V, W, S, ws
    torch.cuda.empty_cache()
    return out


def ensemble_throughput(asuca, dev, nsteps=10, reps=3):
    """32 members with nx = ny drawn from U{64..320}, 58 levels, 4 tracers, FP32:
    cell-updates/s of one persistent launch per call (graph-replayed) against the
    same members advanced one after another with asuca_step."""
    import torch
    import gen
    from paper_1710_08616_gb300 import autotune
    cases = gen.make_ensemble_cases()
    grids = [asuca.Grid.from_case(c) for c in cases]
    states = [asuca.State.from_case(c, device=dev) for c in cases]
    dts = [c.dt for c in cases]
    cells = sum(c.cells for c in cases)
    tune = autotune.tune_ensemble(grids, states, dts, steps=2, reps=2, save=False)
    ws = torch.empty(asuca.ensemble_workspace_bytes(grids), dtype=torch.uint8, device=dev)
    asuca.ensemble_step(grids, states, dts, nsteps, workspace=ws)     # capture + warm
    asuca.ensemble_step(grids, states, dts, nsteps, workspace=ws)
    torch.cuda.synchronize()

    def ens():
        asuca.ensemble_step(grids, states, dts, nsteps, workspace=ws)

    wss = [g.workspace(device=dev) for g in grids]

    def seq():
        for g, s, d, w in zip(grids, states, dts, wss):
            asuca.step(g, s, d, nsteps, workspace=w)

    def timed(fn):
        best = None
        for _ in range(reps):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            fn()
            e1.record()
            torch.cuda.synchronize()
            best = e0.elapsed_time(e1) if best is None else min(best, e0.elapsed_time(e1))
        return best

    seq()
    t_ens, t_seq = timed(ens), timed(seq)
    assert asuca.get_status(grids[0]) == asuca.OK
    peak, _ = _peaks()
    F = cases[0].nfields
    frac = (10 * F + 8) * 4 * cells * nsteps / (t_ens * 1e-3) / 1e9 / peak
    return {"workload": "ensemble_32x_64to320x58", "members": len(cases), "cells": cells, "nsteps_per_call": nsteps,
            "frac": frac, "frac_model": f"(10 F + 8) x 4 B = {(10 * F + 8) * 4} B per member cell and step "
                                        "over the measured HBM peak",
            "sizes": [c.nx for c in cases], "ensemble_tile_rows": tune["best"]["ensemble_tile_rows"],
            "ensemble_cell_updates_per_s": cells * nsteps / (t_ens * 1e-3),
            "sequential_members_cell_updates_per_s": cells * nsteps / (t_seq * 1e-3),
            "ensemble_ms_per_step": t_ens / nsteps, "sequential_ms_per_step": t_seq / nsteps,
            "speedup_over_sequential": t_seq / t_ens}


def adjoint_probe(prec_name):
    """One adjoint step (K = 1) of the 128x128x58, 4-tracer workload, twice: per call
    3 recording stage launches, 1 column launch, 1 column transpose and 3 stage
    transposes."""
    import torch
    from paper_1710_08616_gb300 import build as _b
    _b.build()
    import paper_1710_08616_gb300 as asuca
    import gen
    torch.cuda.set_device(0)
    prec = asuca.FP64 if prec_name == "fp64" else asuca.FP32_MIXED
    case = gen.make_config_case("adjoint_128x128x58")
    g = asuca.Grid.from_case(case, prec=prec)
    st = asuca.State.from_case(case, prec=prec)
    lam = torch.randn((case.nfields,) + tuple(st.rho.shape), dtype=g.torch_dtype, device=st.rho.device)
    for _ in range(2):
        asuca.adjoint_step(g, st, case.dt, 1, lam.contiguous(), checkpoint_every=1)
    torch.cuda.synchronize()
    assert asuca.get_status(g) == asuca.OK
    return 0


def run_ours(args):
    import numpy as np
    import torch

    world, rank, local = _dist()
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    else:
        torch.cuda.set_device(0)
    from paper_1710_08616_gb300 import build as _b
    _b.build()
    import paper_1710_08616_gb300 as asuca
    import gen

    if args.nx == 1024:
        case = gen.make_config_case(WORKLOAD)
        workload = WORKLOAD
    else:   # a smaller case of the same workload, for profiler captures
        case = gen.make_config_case(WORKLOAD, nx=args.nx, ny=args.nx)
        workload = f"profile_{args.nx}x{args.nx}x58"
    F = case.nfields
    C = case.cells
    dev = torch.device("cuda", torch.cuda.current_device())

    # ---- FP32-mixed, device-resident (headline)
    g = asuca.Grid.from_case(case, prec=asuca.FP32_MIXED)
    st = asuca.State.from_case(case, prec=asuca.FP32_MIXED, device=dev)
    ws_t = g.workspace(device=dev)
    bud = torch.empty(F + 1, dtype=torch.float64, device=dev)
    props = torch.cuda.get_device_properties(dev)
    gpu_id = str(getattr(props, "uuid", "")) or str(local)
    if gpu_id and not gpu_id.startswith("GPU-") and len(gpu_id) > 8:
        gpu_id = "GPU-" + gpu_id
    sampler = ClockSampler(gpu_id if rank == 0 else str(local))
    if rank == 0:
        sampler.start()
    ms, prof = _time_steps(asuca, g, st, case.dt, ws_t, bud, args.steps, args.warmup, world, profile=True)
    clocks = sampler.stop() if rank == 0 else None
    ms = _max_over_ranks(world, ms)
    value = world * C * args.steps / (ms * 1e-3)

    # ---- roofline of the dominant kernel, from the live per-kernel events
    hbm_peak, peak_kind = _peaks()
    s = 4
    kinds = {asuca.KERNEL_STAGE: "stage", asuca.KERNEL_COLUMN: "column", asuca.KERNEL_REDUCE: "budget_reduce",
             asuca.KERNEL_STAGE_COLUMN: "stage3_column", asuca.KERNEL_STAGE_FACTOR: "stage2_factor"}
    fused = asuca.get_tuning(g, asuca.TUNE_FUSED_COLUMN) == 1
    split = bool(prof) and asuca.KERNEL_STAGE_FACTOR in prof
    # algorithmic bytes per launch.  Stage 1 reads Yn and M and writes Y* (2F+3 values);
    # stage 2 reads Y*, Yn and M and writes Y** (3F+3).  With the fused path, stage 3
    # with the top-down column pass reads Y**, Yn and M and writes rho plus the
    # elimination values (m, gamma, e_f: F+1 doubles), and the bottom-up pass reads
    # those and rho and writes the F-1 other fields; without it, stage 3 is a stage
    # launch (3F+3) and the column pass reads F and writes F-1 values.
    # With the column pass split over the stages (the plain step), stage 2 also
    # writes m, gamma and alpha (3 doubles) and stage 3 reads alpha and writes rho
    # and the nine e_f (F-1 doubles).
    if fused and split:
        algo = {asuca.KERNEL_STAGE: (2 * F + 3) * C * s,
                asuca.KERNEL_STAGE_FACTOR: ((3 * F + 3) * s + 3 * 8) * C,
                asuca.KERNEL_STAGE_COLUMN: ((2 * F + 3 + 1) * s + F * 8) * C,
                asuca.KERNEL_COLUMN: ((F + 1) * 8 + F * s) * C,
                asuca.KERNEL_REDUCE: 0.0}
    elif fused:
        algo = {asuca.KERNEL_STAGE: ((2 * F + 3) + (3 * F + 3)) / 2.0 * C * s,
                asuca.KERNEL_STAGE_COLUMN: ((2 * F + 3 + 1) * s + (F + 1) * 8) * C,
                asuca.KERNEL_COLUMN: ((F + 1) * 8 + F * s) * C,
                asuca.KERNEL_REDUCE: 0.0}
    else:
        algo = {asuca.KERNEL_STAGE: ((2 * F + 3) + 2 * (3 * F + 3)) / 3.0 * C * s,
                asuca.KERNEL_COLUMN: (2 * F - 1) * C * s,
                asuca.KERNEL_REDUCE: 0.0}
    kern = {}
    for k, (tot, n) in (prof or {}).items():
        avg = tot / n
        kname = kinds.get(k, str(k))
        kern[kname] = {"launches": n, "total_ms": tot, "avg_ms": avg,
                       "share": tot / max(sum(v[0] for v in prof.values()), 1e-30),
                       "algo_bytes_per_launch": algo.get(k, 0.0),
                       "achieved_gbs": algo.get(k, 0.0) / (avg * 1e-3) / 1e9 if avg else None,
                       "traffic_bytes_per_launch": _recorded_traffic(kname, C)}
    dom = max(prof.items(), key=lambda kv: kv[1][0])[0] if prof else asuca.KERNEL_STAGE
    dname = kinds.get(dom, str(dom))
    ach = kern[dname]["achieved_gbs"] if dname in kern else None
    roofline = {"kernel": dname, "bound": "hbm", "achieved": ach, "peak": hbm_peak, "unit": "GB/s",
                "frac": (ach / hbm_peak) if ach else None, "peak_source": peak_kind,
                "traffic": _recorded_traffic(dname, C),
                "step_frac": (10 * F + 8) * s * C / (ms / args.steps * 1e-3) / 1e9 / hbm_peak,
                "step_model_bytes_per_cell": (10 * F + 8) * s, "kernels": kern}
    roofline.update(_floor_and_dram(kern, F, s, C, ms, args.steps, hbm_peak))

    # ---- e2e through the C ABI with pinned host buffers, copies inside the timed region
    e2e = None
    if not args.no_e2e:
        # End to end: every step copies its inputs (state and mass fluxes) from pinned
        # host memory, advances them through the C ABI and copies the state and the
        # budgets back.  Copies in, the step and copies out run on separate streams
        # with NB device buffer sets, so step n's copies overlap the neighbouring
        # steps' work (with two sets the copy in of step n waits for the copy out
        # of step n - 2, which chains copy in, step and copy out); the timed
        # region spans the first copy in to the last copy out.
        names = ("rho", "rhotheta", "rhoq", "mu", "mv", "mw")
        # pinned buffers on the GPU's own host NUMA node: the allocating thread
        # runs on that node's CPUs, so the pages land there
        aff0 = os.sched_getaffinity(0)
        local_cpus = _gpu_local_cpus(gpu_id if rank == 0 else str(local))
        if local_cpus:
            os.sched_setaffinity(0, local_cpus)
        link = _link_gbs(dev)
        host = {k: getattr(st, k).cpu().pin_memory() for k in names}
        hout = {k: torch.empty_like(host[k]).pin_memory() for k in ("rho", "rhotheta", "rhoq")}
        hbud = torch.empty(F + 1, dtype=torch.float64).pin_memory()
        h2d = sum(t.numel() * t.element_size() for t in host.values())
        d2h = sum(t.numel() * t.element_size() for t in hout.values()) + hbud.numel() * 8
        ne = max(1, min(args.steps, args.e2e_steps))
        NB = max(2, args.e2e_buffers)
        bufs = [st] + [asuca.State(*[torch.empty_like(getattr(st, k)) for k in names]) for _ in range(NB - 1)]
        buds = [bud] + [torch.empty_like(bud) for _ in range(NB - 1)]
        # copies may be split over several streams per direction (one was the
        # fastest: the host link, not the copy engines, is the bound)
        NCOPY = max(1, args.e2e_copy_streams)
        s_in = [torch.cuda.Stream() for _ in range(NCOPY)]
        s_out = [torch.cuda.Stream() for _ in range(NCOPY)]
        s_run = torch.cuda.Stream()
        ev_in = [[torch.cuda.Event() for _ in range(NCOPY)] for _ in range(NB)]
        ev_out = [[torch.cuda.Event() for _ in range(NCOPY)] for _ in range(NB)]
        ev_run = [torch.cuda.Event() for _ in range(NB)]
        # pieces of about equal size: every tensor cut along its slowest dimension
        def pieces(tensors):
            if NCOPY == 1:
                return list(tensors)
            out = []
            for dst, src in tensors:
                n = dst.shape[0]
                step = max(1, -(-n // NCOPY))
                for a in range(0, n, step):
                    out.append((dst[a:a + step], src[a:a + step]))
            return out

        def e2e_steps(n):
            for q in range(n):
                b = q % NB
                ins = pieces([(getattr(bufs[b], k), host[k]) for k in names])
                for c, sx in enumerate(s_in):
                    if q >= NB:
                        for c2 in range(NCOPY):       # buffer set b has been read back
                            sx.wait_event(ev_out[b][c2])
                    with torch.cuda.stream(sx):
                        for dst, src in ins[c::NCOPY]:
                            dst.copy_(src, non_blocking=True)
                    ev_in[b][c].record(sx)
                for c in range(NCOPY):
                    s_run.wait_event(ev_in[b][c])
                asuca.step(g, bufs[b], case.dt, 1, workspace=ws_t, budgets=buds[b], stream=s_run)
                ev_run[b].record(s_run)
                outs = pieces([(hout[k], getattr(bufs[b], k)) for k in hout]) + [(hbud, buds[b])]
                for c, sx in enumerate(s_out):
                    sx.wait_event(ev_run[b])
                    with torch.cuda.stream(sx):
                        for dst, src in outs[c::NCOPY]:
                            dst.copy_(src, non_blocking=True)
                    ev_out[b][c].record(sx)

        cur = torch.cuda.current_stream()
        streams = s_in + [s_run] + s_out

        def join():
            for sx in streams:
                cur.wait_stream(sx)

        for sx in streams:
            sx.wait_stream(cur)
        e2e_steps(2)
        join()
        torch.cuda.synchronize()
        _barrier(world)
        a0 = torch.cuda.Event(enable_timing=True)
        a1 = torch.cuda.Event(enable_timing=True)
        a0.record(cur)
        for sx in streams:
            sx.wait_stream(cur)
        e2e_steps(ne)
        join()
        a1.record(cur)
        torch.cuda.synchronize()
        _barrier(world)
        assert asuca.get_status(g) == asuca.OK
        ems = _max_over_ranks(world, a0.elapsed_time(a1))
        e2e = {"value": world * C * ne / (ems * 1e-3), "unit": UNIT, "h2d_bytes_per_step": h2d,
               "d2h_bytes_per_step": d2h, "steps": ne, "ms_per_step": ems / ne,
               "overlap": f"copies in ({NCOPY} stream(s)), the step, copies out ({NCOPY} stream(s)); "
                          f"{NB} device buffer sets",
               "link_gbs": link,
               "link_bound_ms_per_step": max(h2d, d2h) / (link["each_way_concurrent"] * 1e9) * 1e3,
               "host_numa": ({"bound_to_gpu_local_cpus": len(local_cpus)} if local_cpus
                             else {"bound_to_gpu_local_cpus": None, "why": "GPU's local CPUs not found"})}
        os.sched_setaffinity(0, aff0)
        del host, hout, bufs
    del st, ws_t
    torch.cuda.empty_cache()

    # ---- all-FP64 path on the same workload
    fp64 = None
    if not args.no_fp64:
        g64 = asuca.Grid.from_case(case, prec=asuca.FP64)
        st64 = asuca.State.from_case(case, prec=asuca.FP64, device=dev)
        ws64 = g64.workspace(device=dev)
        bud64 = torch.empty(F + 1, dtype=torch.float64, device=dev)
        n64 = max(1, min(args.steps, args.fp64_steps))
        ms64, prof64 = _time_steps(asuca, g64, st64, case.dt, ws64, bud64, n64, 1, world, profile=True)
        ms64 = _max_over_ranks(world, ms64)
        fp64 = {"value": world * C * n64 / (ms64 * 1e-3), "ms_per_step": ms64 / n64, "steps": n64,
                "kernels": {kinds.get(k, str(k)): {"launches": n, "avg_ms": t / n} for k, (t, n) in prof64.items()}}
        # the FP64 stage launches are bound by the FP64 pipe: its instruction rate
        # (FP64 instructions per cell from the recorded capture) against the pipe's peak
        st64k = fp64["kernels"].get("stage")
        inst = _recorded("stage_fp64", "fp64_inst_per_cell", C)
        fp64["roofline"] = {"kernel": "stage", "bound": "fp64", "unit": "FP64 inst/s", "peak": FP64_INST_PEAK,
                            "achieved": (inst / (st64k["avg_ms"] * 1e-3)) if (inst and st64k) else None,
                            "frac": (inst / (st64k["avg_ms"] * 1e-3) / FP64_INST_PEAK) if (inst and st64k) else None,
                            "peak_source": "recipe unit counts and maximum SM clock"}
        del st64, ws64

    # the oracle's run of the precision workload, on the host cores while the
    # GPU reports below run (started after the headline and end-to-end timings)
    ojob = None
    if not args.no_precision and rank == 0 and world == 1:
        ojob = start_oracle_precision()
    open_rep = None
    if not args.no_open:
        open_rep = open_report(asuca, dev, case)
    hevi = None
    if not args.no_hevi:
        hevi = hevi_report(asuca, dev, case)
    adjoint = None
    if not args.no_adjoint:
        adjoint = adjoint_cost(asuca, dev)
    ensemble = None
    if not args.no_ensemble:
        ensemble = ensemble_throughput(asuca, dev, args.ens_steps)
    layout = None
    if not args.no_layout:
        layout = layout_ablation(asuca, dev)
    damping = None
    if not args.no_damping:
        damping = damping_report(asuca, dev)
    acoustic = None
    if not args.no_acoustic:
        acoustic = acoustic_report(asuca, dev)
    precision = None
    if not args.no_precision:
        precision = precision_report(asuca, dev, ojob)

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu:
        cpu = cpu_oracle_rate()

    if rank == 0:
        out = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
               "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True,
               "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
               "config": {"workload": workload, "nx": case.nx, "ny": case.ny, "nz": case.nz,
                          "ntracers": case.ntracers, "cells": C, "dt_s": case.dt,
                          "precision": "fp32 fields/stencils/physics, fp64 Thomas solve and budget sums",
                          "limiter": "koren", "l2": "inputs larger than L2 (2.4 GB state), no flush",
                          "parallelism": f"{world} independent replica(s), one per GPU"},
               "clocks": clocks, "gpu_launches": sum(n for _t, n in (prof or {}).values()), "roofline": roofline,
               "e2e": e2e, "fp64": fp64, "precision": precision, "adjoint": adjoint, "ensemble": ensemble,
               "layout_ablation": layout, "damping": damping, "acoustic": acoustic, "open": open_rep,
               "hevi": hevi,
               "fp32_over_fp64_speedup": (value / fp64["value"]) if fp64 else None,
               "cpu_baseline": cpu}
        print(json.dumps(out), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()
    return 0


def main():
    ap = argparse.ArgumentParser(description=__doc__, formatter_class=argparse.RawDescriptionHelpFormatter)
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=100)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--fp64-steps", type=int, default=5)
    ap.add_argument("--e2e-steps", type=int, default=10)
    ap.add_argument("--e2e-copy-streams", type=int, default=1,
                    help="streams per copy direction in the end-to-end measurement (1 was fastest on GB300)")
    ap.add_argument("--e2e-buffers", type=int, default=4,
                    help="device buffer sets the end-to-end pipeline rotates through (>= 2)")
    ap.add_argument("--ref-n", type=int, default=128, help="reference arm sample size (n x n x 58)")
    ap.add_argument("--no-fp64", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-adjoint", action="store_true")
    ap.add_argument("--no-precision", action="store_true")
    ap.add_argument("--no-ensemble", action="store_true")
    ap.add_argument("--no-layout", action="store_true")
    ap.add_argument("--no-damping", action="store_true")
    ap.add_argument("--no-acoustic", action="store_true")
    ap.add_argument("--no-open", action="store_true")
    ap.add_argument("--no-hevi", action="store_true")
    ap.add_argument("--acoustic-probe", choices=["fp32", "fp64"], default=None,
                    help="time the acoustic short steps alone on the nx x nx x 58 grid in one precision and "
                         "exit (a small launch sequence for profiler captures)")
    ap.add_argument("--ens-steps", type=int, default=10)
    ap.add_argument("--nx", type=int, default=1024,
                    help="nx = ny of the timed case; anything but 1024 is a smaller case of the same "
                         "workload for profiler captures, not a bench line")
    ap.add_argument("--adjoint-probe", choices=["fp32", "fp64"], default=None,
                    help="run one adjoint step of the 128x128x58 workload twice (recomputed from one "
                         "checkpoint) and exit: a small fixed launch sequence for profiler captures")
    ap.add_argument("--damping-probe", choices=["fp32", "fp64"], default=None,
                    help="time the damping alone on the nx x nx x 58 case in one precision and exit "
                         "(a small launch sequence for profiler captures)")
    args = ap.parse_args()
    if args.warmup < 3:
        ap.error("--warmup must be >= 3")
    if args.adjoint_probe:
        return adjoint_probe(args.adjoint_probe)
    if args.acoustic_probe:
        import torch
        from paper_1710_08616_gb300 import build as _b
        _b.build()
        import paper_1710_08616_gb300 as asuca
        torch.cuda.set_device(0)
        print(json.dumps(acoustic_report(asuca, torch.device("cuda", 0), reps=1, nx=args.nx,
                                         precs=(args.acoustic_probe,))), flush=True)
        return 0
    if args.damping_probe:
        import torch
        from paper_1710_08616_gb300 import build as _b
        _b.build()
        import paper_1710_08616_gb300 as asuca
        torch.cuda.set_device(0)
        print(json.dumps(damping_report(asuca, torch.device("cuda", 0), reps=3, nx=args.nx,
                                        precs=(args.damping_probe,))), flush=True)
        return 0
    if args.impl == "reference":
        return run_reference(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
