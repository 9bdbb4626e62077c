"""Benchmark: cell-ordinate-group updates per second of the SHDOM time step.

Workload (one GPU): the relativistic jet problem, 64^3 nodes, 16 log-spaced
groups over 1e-3..1e1 m_e c^2, L = 7 (64 harmonics), 16 x 32 ordinates,
Thomson scattering with radial optical depth 10, bulk Lorentz factor 10 in the
jet core; one source iteration per time step (project -> source -> sh2lab ->
sweep -> sums), c dt = half a node spacing.  Synthetic seeded inputs; the
state (8.6 GB in FP32) is far larger than L2, so no flush is needed between
steps.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--precision fp32|mixed|fp64]
  python bench.py --impl reference ...   (the FP64 CPU oracle on a bounded sample)

Under torchrun each rank runs its own replica of the problem (the problems
are independent: weak scaling, no collective in the data path); rank 0
prints one JSON line.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "cell-ordinate-group updates/s"
UNIT = "updates/s"
WORKLOAD = "relativistic jet 64^3, 16 groups (1e-3..1e1 m_e c^2), L=7, 16x32 ordinates, Thomson tau_r=10, Gamma<=10"
# algorithmic bytes per update of the sweep: its own work is to read I^n and
# write I^{n+1} (8 B in FP32).  The laboratory eta and chi it also reads are
# the materialised output of the SH -> ordinate stage, traffic a fused design
# avoids: they are reported apart (operand_bytes_per_update), not counted as
# algorithmic.
SWEEP_BYTES_PER_UPDATE = {"fp32": 8, "mixed": 8, "fp64": 16}
SWEEP_OPERAND_BYTES_PER_UPDATE = {"fp32": 8, "mixed": 8, "fp64": 16}
# floor of the whole step's traffic per update: the intensity read and written
# once plus the SH state, about 2 B at L = 7 with 512 ordinates
STEP_FLOOR_BYTES_PER_UPDATE = {"fp32": 10, "mixed": 10, "fp64": 20}


def _sha256(path):
    import hashlib
    with open(path, "rb") as f:
        return hashlib.sha256(f.read()).hexdigest()


def sweep_traffic(prec, spec):
    """DRAM bytes (read + write) of one sweep launch from the committed ncu
    summary of this workload and precision, or None when there is none or the
    sweep's source has changed since it was captured."""
    if spec.grid != (64, 64, 64):
        return None
    path = os.path.join(ROOT, "profiles", f"sweep_jet64_{prec}.md")
    if not os.path.exists(path):
        return None
    fields = {}
    with open(path) as f:
        for ln in f:
            if ":" in ln and ln.startswith("- "):
                k, v = ln[2:].split(":", 1)
                fields[k.strip()] = v.strip().strip("`")
    csrc = os.path.join(ROOT, "paper_1507_05141_gb300", "csrc")
    try:
        if fields.get("shd_kernels.cu sha256") != _sha256(os.path.join(csrc, "shd_kernels.cu")):
            return None
        if fields.get("shd_internal.cuh sha256") != _sha256(os.path.join(csrc, "shd_internal.cuh")):
            return None
        return int(fields["dram bytes per launch"])
    except (KeyError, ValueError, OSError):
        return None


def _dist():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def max_over_ranks(x, device=None):
    """The largest of the ranks' values of x (x itself in a single process).
    Timing only: the replicas exchange nothing else."""
    ws, _, _ = _dist()
    if ws <= 1:
        return float(x)
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_rate(updates_per_step, steps, ws, seconds):
    """Whole-job updates/s: every rank's steps over the slowest rank's time."""
    return updates_per_step * steps * ws / seconds


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            p = json.load(f)
        return float(p["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.rows = []
        self._stop = threading.Event()
        self._t = None

    def _run(self):
        while not self._stop.is_set():
            try:
                out = subprocess.run(["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.Q}",
                                      "--format=csv,noheader,nounits"], capture_output=True, text=True, timeout=5)
                if out.returncode == 0 and out.stdout.strip():
                    self.rows.append([x.strip() for x in out.stdout.strip().split(",")])
            except Exception:
                pass
            self._stop.wait(0.2)

    def __enter__(self):
        self._t = threading.Thread(target=self._run, daemon=True)
        self._t.start()
        return self

    def __exit__(self, *a):
        self._stop.set()
        self._t.join(timeout=10)

    def summary(self):
        if not self.rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        sm = [float(r[1]) for r in self.rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in self.rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in self.rows for i in range(4) if len(r) > 5 + i and r[5 + i] == "Active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(self.rows)}


def cpu_sample_spec(n=24):
    """Bounded CPU sample: the same recipe (groups, harmonics, ordinates, flow,
    opacities) on an n^3 grid."""
    from paper_1507_05141_gb300 import inputs
    return inputs.jet(n=n)


def run_oracle_steps(spec, steps):
    """Time `steps` oracle steps of spec on the host cores; returns (updates/s, seconds)."""
    from oracle import oracle as O
    from paper_1507_05141_gb300 import inputs
    K, so = O.thomson_table(spec.G, spec.L)
    P = O.OracleProblem(grid=spec.grid, L=spec.L, nmu=spec.nmu, nphi=spec.nphi, edges=spec.edges,
                        alpha0=spec.alpha0, ne=spec.ne, u=spec.u, emis0=spec.emis0, K=K, sigma_out=so,
                        kappa=spec.kappa, box=spec.box)
    I = inputs.random_state(spec, seed=1)
    t0 = time.perf_counter()
    P.step(I, steps)
    dt = time.perf_counter() - t0
    return spec.updates_per_step * steps / dt, dt


def cpu_baseline(steps=6):
    spec = cpu_sample_spec()
    v, dt = run_oracle_steps(spec, steps)
    cores = int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1))
    return {"value": v, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": f"{steps} FP64 oracle steps of the jet recipe on a {spec.grid[0]}^3 grid "
                      f"({spec.updates_per_step:.3g} updates/step, {dt:.1f} s)"}


def bench_reference(args):
    ws, rank, _ = _dist()
    if rank != 0:
        return 0
    spec = cpu_sample_spec()
    run_oracle_steps(spec, max(0, min(args.warmup, 1)))
    times = []
    for _ in range(args.steps):
        _, dt = run_oracle_steps(spec, 1)
        times.append(dt)
    tot = sum(times)
    v = spec.updates_per_step * args.steps / tot
    cores = int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1))
    line = {"metric": METRIC, "value": v, "unit": UNIT, "impl": "reference", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * tot / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic",
            "config": {"workload": WORKLOAD + f" (CPU sample: {spec.grid[0]}^3 grid, same recipe)", "grid": spec.grid,
                       "groups": spec.G, "L": spec.L, "ordinates": spec.N},
            "cpu_baseline": {"value": v, "unit": UNIT, "cores": cores, "kind": "oracle",
                             "sample": f"one FP64 oracle step of the jet recipe on a {spec.grid[0]}^3 grid per step"},
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))
    return 0


def field_errors(precision, device, n=16, steps=3):
    """Per-field error of a GPU precision against the FP64 oracle on the jet
    recipe at a reduced grid (same groups, harmonics and ordinates), after
    `steps` steps from a seeded state: J and I_lm relative to their maxima
    per (node, group), H and K relative to J, f_ij absolute."""
    import numpy as np

    from oracle import oracle as O
    from paper_1507_05141_gb300 import inputs, native
    spec = inputs.jet(n=n)
    I0 = inputs.random_state(spec, seed=11)
    s = native.Solver.from_spec(spec, device=device, precision=precision)
    s.set_state(I0)
    s.step(steps)
    J, H, K, Ish = s.moments(with_sh=True)
    s.close()
    Kt, so = O.thomson_table(spec.G, spec.L)
    P = O.OracleProblem(grid=spec.grid, L=spec.L, nmu=spec.nmu, nphi=spec.nphi, edges=spec.edges,
                        alpha0=spec.alpha0, ne=spec.ne, u=spec.u, emis0=spec.emis0, K=Kt, sigma_out=so,
                        kappa=spec.kappa, box=spec.box)
    Ir, _, _ = P.step(I0, steps)
    Ish_r, J_r, H_r, K_r = P.project(Ir)
    Jd = np.maximum(np.abs(J_r), 1e-300)
    f, f_r = O.moments_to_eddington(J, K), O.moments_to_eddington(J_r, K_r)
    return {"J": float(np.max(np.abs(J - J_r) / Jd)),
            "H": float(np.max(np.abs(H - H_r) / Jd[..., None])),
            "K": float(np.max(np.abs(K - K_r) / Jd[..., None])),
            "f_ij": float(np.max(np.abs(f - f_r))),
            "I_lm": float(np.max(np.abs(Ish - Ish_r)) / np.max(np.abs(Ish_r))),
            "case": f"jet recipe {n}^3, G={spec.G}, L={spec.L}, {spec.N} ordinates, {steps} steps"}


def time_steps(solver, spec, steps, warmup, stream, dev, barrier, with_timing=True):
    """Warm-up, then `steps` device-timed steps on `stream`; returns
    (ms, per-stage ms per step, clock summary, kernels the library launched
    in the timed region)."""
    import torch
    sptr = stream.cuda_stream
    solver.step(warmup, sptr)
    torch.cuda.synchronize(dev)
    if with_timing:
        solver.set_timing(True)
    barrier()
    torch.cuda.synchronize(dev)
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    from paper_1507_05141_gb300 import native
    with ClockSampler(dev.index) as clk:
        n0 = native.launch_count()
        ev0.record(stream)
        solver.step(steps, sptr)
        ev1.record(stream)
        launches = native.launch_count() - n0
        torch.cuda.synchronize(dev)
    barrier()
    ms = ev0.elapsed_time(ev1)
    stage = {}
    if with_timing:
        stage_ms, nrec = solver.timing()
        solver.set_timing(False)
        stage = {k: v / max(1, nrec) for k, v in stage_ms.items()}
    return ms, stage, clk.summary(), launches


def bench_ours(args):
    import numpy as np
    import torch

    from paper_1507_05141_gb300 import inputs, native

    ws, rank, local = _dist()
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)

    spec = inputs.jet(n=args.grid)
    prec = args.precision
    solver = native.Solver.from_spec(spec, device=local, precision=prec)
    solver.zero_state()
    stream = torch.cuda.Stream(dev)  # a real stream: its handle is never 0
    torch.cuda.set_stream(stream)
    sptr = stream.cuda_stream

    def barrier():
        if ws > 1:
            import torch.distributed as dist
            dist.barrier()

    # warm-up (also fills the state with a physical solution), then the
    # device-resident timed region
    ms, stage, clk_summary, launches = time_steps(solver, spec, args.steps, args.warmup, stream, dev, barrier)
    ms = max_over_ranks(ms, dev)
    (sw_C, sw_NT), sw_rows = solver.sweep_schedule()
    sweep_sched = {"cluster_ctas": sw_C, "threads": sw_NT,
                   "timed": [{"cluster_ctas": c, "threads": nt, "ms_sample": round(t, 4)} for c, nt, t in sw_rows]}
    upd = spec.updates_per_step
    value = job_rate(upd, args.steps, ws, ms / 1e3)

    # end to end through the C ABI with host buffers: per step the fields
    # are uploaded from pinned host memory, one step runs, and the FP64 sums
    # are read back.
    def pinned(a):
        t = torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64)).pin_memory()
        return t, t.numpy()
    hold = [pinned(x) for x in (spec.alpha0, spec.ne, spec.u, spec.emis0)]
    arrs = [h[1] for h in hold]
    h2d = sum(a.nbytes for a in arrs)
    d2h = 3 * 8
    e2e_steps = max(1, min(args.steps, 10))
    barrier()
    torch.cuda.synchronize(dev)
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        solver.set_fields(*arrs)
        solver.step(1, sptr)
        solver.sums()
    torch.cuda.synchronize(dev)
    e2e_s = max_over_ranks(time.perf_counter() - t0, dev)
    e2e_value = job_rate(upd, e2e_steps, ws, e2e_s)

    peak, peak_kind = _peaks()
    do_gb = upd * (8 if prec == "fp64" else 4) / 1e9
    sweep_ms = stage["sweep"]
    sweep_bytes = upd * SWEEP_BYTES_PER_UPDATE[prec]
    achieved = sweep_bytes / (sweep_ms / 1e3) / 1e9
    traffic = sweep_traffic(prec, spec)
    # the whole step against the floor of its own traffic: I^n read and
    # I^{n+1} written once (8 B at FP32) plus the SH state (I_lm, S_lm, S_prev,
    # about 2 B per update at L = 7 and 512 ordinates)
    step_floor = STEP_FLOOR_BYTES_PER_UPDATE[prec]
    step_achieved = upd * step_floor / (ms / args.steps / 1e3) / 1e9

    # the plain-FP32 arm on the same GPU, same workload and timing
    plain = None
    if prec == "mixed" and not args.no_compare:
        solver.close()
        torch.cuda.empty_cache()
        s32 = native.Solver.from_spec(spec, device=local, precision="fp32")
        s32.zero_state()
        ms32, stage32, _, _ = time_steps(s32, spec, args.steps, args.warmup, stream, dev, barrier)
        ms32 = max_over_ranks(ms32, dev)
        s32.close()
        solver = None
        plain = {"value": job_rate(upd, args.steps, ws, ms32 / 1e3), "unit": UNIT, "ms_per_step": ms32 / args.steps,
                 "stage_ms": stage32}
    errors = None
    if rank == 0 and not args.no_errors:
        errors = {p: field_errors(p, local) for p in ([prec, "fp32"] if prec == "mixed" else [prec])}

    if rank == 0:
        cpu = cpu_baseline() if (ws == 1 and not args.no_cpu) else None
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None,
            "dtype": {"fp32": "f32", "mixed": "f32", "fp64": "f64"}[prec], "data": "synthetic",
            "config": {"workload": WORKLOAD if args.grid == 64 else WORKLOAD.replace("64^3", f"{args.grid}^3"),
                       "grid": list(spec.grid), "groups": spec.G, "L": spec.L,
                       "ordinates": spec.N, "precision": prec, "updates_per_step": upd,
                       "l2": f"no flush: the {do_gb:.1f} GB intensity state is far larger than L2",
                       "parallelism": f"replicas x{ws}"},
            "stage_ms": stage,
            "sweep_schedule": sweep_sched,
            "plain_fp32": plain,
            "err_vs_fp64_oracle": errors,
            "roofline": {"kernel": "k_sweep_pp", "bound": "hbm", "achieved": achieved, "peak": peak,
                         "unit": "GB/s", "frac": achieved / peak, "traffic": traffic,
                         "traffic_ratio": (traffic / sweep_bytes) if traffic else None,
                         "peak_kind": peak_kind,
                         "algorithmic_bytes": f"{SWEEP_BYTES_PER_UPDATE[prec]} B/update x {upd} updates "
                                              f"(I^n read, I^n+1 written)",
                         "operand_bytes_per_update": SWEEP_OPERAND_BYTES_PER_UPDATE[prec],
                         "operand_bytes_note": "laboratory eta, chi read from HBM (materialised by sh2lab; "
                                               "chi only where a node moves)"},
            "step_roofline": {"bound": "hbm", "floor_bytes_per_update": step_floor, "achieved": step_achieved,
                              "peak": peak, "unit": "GB/s", "frac": step_achieved / peak},
            "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
                    "steps": e2e_steps},
            "gpu_launches": launches,
            "clocks": clk_summary,
            "cpu_baseline": cpu,
        }
        print(json.dumps(line))
    if solver is not None:
        solver.close()
    if ws > 1:
        import torch.distributed as dist
        dist.destroy_process_group()
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--precision", default="mixed", choices=["fp32", "mixed", "fp64"])
    ap.add_argument("--no-compare", action="store_true", help="skip the plain-FP32 arm of a mixed run")
    ap.add_argument("--no-errors", action="store_true", help="skip the per-field error check against the oracle")
    ap.add_argument("--no-cpu", action="store_true", help="skip the CPU-baseline sample")
    ap.add_argument("--grid", type=int, default=64,
                    help="nodes per axis of the jet workload (64 is the benchmark; smaller for profiling)")
    args = ap.parse_args()
    if args.warmup < 3 and args.impl == "ours":
        print("warning: fewer than 3 warm-up steps", file=sys.stderr)
    if args.impl == "reference":
        return bench_reference(args)
    return bench_ours(args)


if __name__ == "__main__":
    sys.exit(main())
