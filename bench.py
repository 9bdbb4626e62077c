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
    if args.sweep_schedule:
        sc, snt = (int(v) for v in args.sweep_schedule.split(","))
        solver.set_sweep_schedule(sc, snt)
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
    # the production path: every timed step replays the captured step graph
    # (shd_step without per-stage events); then the same number of steps as
    # direct launches with per-stage CUDA events for the stage times and the
    # sweep's roofline (--no-e2e, used for profiling, keeps to direct launches)
    if args.no_e2e:
        ms, stage, clk_summary, launches = time_steps(solver, spec, args.steps, args.warmup, stream, dev, barrier)
        ms_direct = ms
    else:
        ms, _, clk_summary, launches = time_steps(solver, spec, args.steps, args.warmup, stream, dev, barrier,
                                                  with_timing=False)
        ms_direct, stage, _, _ = time_steps(solver, spec, args.steps, 1, stream, dev, barrier)
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
    e2e_value = None
    if not args.no_e2e:
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
            "timing": {"value_from": "graph replays of the captured step (shd_step's production path)"
                                     if not args.no_e2e else "direct launches with per-stage events",
                       "ms_per_step_direct_launches": ms_direct / args.steps,
                       "stage_ms_from": "direct launches with per-stage CUDA events"},
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


# ---------------------------------------------------------------------------
# the other workloads (python bench.py --config N): each prints one JSON line
# with the same keys; the default run (--config 2) is the jet above
# ---------------------------------------------------------------------------

def _do_bytes(spec, esize=4):
    """Device bytes a problem holds: three intensity-sized arrays (state,
    laboratory eta and chi), three node-major remap arrays for the moving
    nodes, three SH arrays and the remap tables."""
    import numpy as np
    nmov = int(np.count_nonzero(np.any(spec.u != 0, axis=1)))
    per_node = spec.G * spec.N * esize
    return (3 * spec.Nc * per_node + 3 * nmov * per_node + 3 * spec.Nc * spec.G * spec.NLM * esize
            + 2 * nmov * spec.N * 16 + 64 * spec.Nc * spec.G)


def _fit_groups(make, G_full, free_bytes, frac=0.9, esize=4):
    """The largest group count (G_full, then 3/4, 1/2, 3/8, 1/4, 3/16, 1/8 of it) whose
    problem fits in frac of the free device memory; returns (spec, G)."""
    for G in [G_full, (3 * G_full) // 4, G_full // 2, (3 * G_full) // 8, G_full // 4, (3 * G_full) // 16,
              G_full // 8]:
        spec = make(G)
        if _do_bytes(spec, esize) <= frac * free_bytes:
            return spec, G
    return None, 0


def _errors_vs_oracle(spec_small, precision, device, steps=3, scattering=None):
    """Per-field errors of a GPU precision against the FP64 oracle on a
    reduced copy of a workload's recipe (same generator)."""
    import numpy as np

    from oracle import oracle as O
    from paper_1507_05141_gb300 import inputs, native
    spec = spec_small
    kind = scattering or spec.scattering
    I0 = inputs.random_state(spec, seed=11)
    s = native.Solver.from_spec(spec, device=device, precision=precision, scattering=kind)
    s.set_state(I0)
    s.step(steps)
    J, H, K, Ish = s.moments(with_sh=True)
    s.close()
    P = _oracle_problem(spec, kind)
    Ir, _, _ = P.step(I0, steps)
    Ish_r, J_r, H_r, K_r = P.project(Ir)
    Jd = np.maximum(np.abs(J_r), 1e-300)
    f, f_r = O.moments_to_eddington(J, K), O.moments_to_eddington(J_r, K_r)
    return {"J": float(np.max(np.abs(J - J_r) / Jd)),
            "H": float(np.max(np.abs(H - H_r) / Jd[..., None])),
            "f_ij": float(np.max(np.abs(f - f_r))),
            "I_lm": float(np.max(np.abs(Ish - Ish_r)) / np.max(np.abs(Ish_r))),
            "case": f"{spec.name} {spec.grid[0]}x{spec.grid[1]}x{spec.grid[2]}, G={spec.G}, L={spec.L}, "
                    f"{spec.N} ordinates, {steps} steps"}


def _oracle_problem(spec, kind):
    """The FP64 oracle's problem for spec with scattering `kind` (thermal
    electrons: the kernels on the library's temperature grid and the
    recipe's temperature field)."""
    from oracle import oracle as O
    if kind == "kn_thermal":
        Kth, soth = O.thermal_tables(spec.edges, spec.L)
        th = {"theta_e": spec.extra["theta_e"], "K_th": Kth, "so_th": soth, "lg0": O.THERMAL_LG0,
              "dlg": O.THERMAL_DLG}
        return O.OracleProblem(grid=spec.grid, L=spec.L, nmu=spec.nmu, nphi=spec.nphi, edges=spec.edges,
                               alpha0=spec.alpha0, ne=spec.ne, u=spec.u, emis0=spec.emis0, K=Kth[0],
                               sigma_out=soth[0], kappa=spec.kappa, box=spec.box, thermal=th)
    Kt, so = {"thomson": lambda: O.thomson_table(spec.G, spec.L), "iso": lambda: O.iso_table(spec.G, spec.L),
              "kn": lambda: O.kn_table(spec.edges, spec.L)}[kind]()
    return O.OracleProblem(grid=spec.grid, L=spec.L, nmu=spec.nmu, nphi=spec.nphi, edges=spec.edges,
                           alpha0=spec.alpha0, ne=spec.ne, u=spec.u, emis0=spec.emis0, K=Kt, sigma_out=so,
                           kappa=spec.kappa, box=spec.box)


def _oracle_rate(spec, steps, scattering=None):
    """The FP64 oracle's updates/s on `spec` over `steps` steps (host cores;
    the scattering tables are set up before the clock starts)."""
    from paper_1507_05141_gb300 import inputs
    P = _oracle_problem(spec, scattering or spec.scattering)
    I = inputs.random_state(spec, seed=1)
    t0 = time.perf_counter()
    P.step(I, steps)
    dt = time.perf_counter() - t0
    return spec.updates_per_step * steps / dt, dt


def _line(args, *, workload, spec, prec, value, ms_step, stage, sched, extra_config, errors, e2e, launches, clk,
          cpu, sweep_ms, plain=None, notes=None):
    peak, peak_kind = _peaks()
    upd = spec.updates_per_step
    byt = SWEEP_BYTES_PER_UPDATE[prec]
    ach = upd * byt / (sweep_ms / 1e3) / 1e9 if sweep_ms else None
    step_ach = upd * STEP_FLOOR_BYTES_PER_UPDATE[prec] / (ms_step / 1e3) / 1e9
    cfg = {"workload": workload, "grid": list(spec.grid), "groups": spec.G, "L": spec.L, "ordinates": spec.N,
           "precision": prec, "updates_per_step": upd, "parallelism": "replicas x1"}
    cfg.update(extra_config)
    return {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": 1, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": ms_step, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": {"fp32": "f32", "mixed": "f32", "fp64": "f64"}[prec], "data": "synthetic",
            "config": cfg, "stage_ms": stage, "sweep_schedule": sched, "plain_fp32": plain,
            "err_vs_fp64_oracle": errors,
            "roofline": {"kernel": "sweep", "bound": "hbm", "achieved": ach, "peak": peak, "unit": "GB/s",
                         "frac": (ach / peak) if ach else None, "traffic": None, "peak_kind": peak_kind,
                         "algorithmic_bytes": f"{byt} B/update x {upd} updates (I^n read, I^n+1 written)"},
            "step_roofline": {"bound": "hbm", "floor_bytes_per_update": STEP_FLOOR_BYTES_PER_UPDATE[prec],
                              "achieved": step_ach, "peak": peak, "unit": "GB/s", "frac": step_ach / peak},
            "e2e": e2e, "gpu_launches": launches, "clocks": clk, "cpu_baseline": cpu, "notes": notes}


def _sched(solver):
    (c, nt), rows = solver.sweep_schedule()
    return {"cluster_ctas": c, "threads": nt,
            "timed": [{"cluster_ctas": a, "threads": b, "ms_sample": round(t, 4)} for a, b, t in rows]}


def bench_config1(args, dev):
    """Static relaxation box in FP64: Lambda iteration to 1e-6, then 10 time
    steps at c dt = half a node spacing (the whole problem is timed, the
    oracle runs the same problem in full)."""
    import numpy as np
    import torch

    from oracle import oracle as O
    from paper_1507_05141_gb300 import inputs, native
    spec = inputs.relax_box()
    prec = "fp64"
    s = native.Solver.from_spec(spec, device=dev.index, precision=prec)
    stream = torch.cuda.Stream(dev)
    sptr = stream.cuda_stream

    def run(timing=False):
        s.zero_state()
        it, r = s.solve_static(1e-6, 500)
        s.set_timing(timing)
        s.step(10, sptr)
        torch.cuda.synchronize(dev)
        return it
    for _ in range(max(1, args.warmup)):
        it = run()
    n0 = native.launch_count()
    with ClockSampler(dev.index) as clk:
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize(dev)
        t0 = time.perf_counter()
        reps = max(1, args.steps)
        for _ in range(reps):
            it = run()
        wall = (time.perf_counter() - t0) / reps
    launches = (native.launch_count() - n0) // reps
    # per-stage times of the 10 steps
    s.zero_state()
    s.solve_static(1e-6, 500)
    s.set_timing(True)
    s.step(10, sptr)
    stage_ms, nrec = s.timing()
    s.set_timing(False)
    stage = {k: v / max(1, nrec) for k, v in stage_ms.items()}
    upd_total = spec.updates_per_step * (it + 10)
    value = upd_total / wall
    # end to end with host buffers: the zero state uploaded, the solve and the
    # steps, the moments read back
    Iz = np.zeros((spec.Nc, spec.G, spec.N))
    t0 = time.perf_counter()
    s.set_state(Iz)
    s.solve_static(1e-6, 500)
    s.step(10, sptr)
    J, H, K = s.moments()
    e2e_s = time.perf_counter() - t0
    # errors against the oracle on the full problem
    Kt, so = O.iso_table(spec.G, spec.L)
    P = O.OracleProblem(grid=spec.grid, L=spec.L, nmu=spec.nmu, nphi=spec.nphi, edges=spec.edges,
                        alpha0=spec.alpha0, ne=spec.ne, u=spec.u, emis0=spec.emis0, K=Kt, sigma_out=so,
                        kappa=spec.kappa, box=spec.box)
    t0 = time.perf_counter()
    Ir, it_r, _ = P.solve_static(tol=1e-6, max_iter=500)
    Ir, _, _ = P.step(Ir, 10)
    cpu_s = time.perf_counter() - t0
    _, J_r, _, K_r = P.project(Ir)
    f, f_r = O.moments_to_eddington(J, K), O.moments_to_eddington(J_r, K_r)
    errors = {"fp64": {"J": float(np.max(np.abs(J - J_r) / np.abs(J_r))), "f_ij": float(np.max(np.abs(f - f_r))),
                       "iterations": [int(it), int(it_r)], "case": "the full problem"}}
    cores = int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1))
    cpu = {"value": spec.updates_per_step * (it_r + 10) / cpu_s, "unit": UNIT, "cores": cores, "kind": "oracle",
           "sample": f"the whole problem ({it_r} static iterations + 10 steps, {cpu_s:.2f} s)"}
    e2e = {"value": upd_total / e2e_s, "unit": UNIT, "h2d_bytes_per_step": Iz.nbytes,
           "d2h_bytes_per_step": spec.Nc * spec.G * 10 * 8, "steps": 1}
    s.close()
    return _line(args, workload=f"static relaxation box 16^3, G=1, L=3, 8x16 ordinates, FP64: Lambda iteration to "
                                f"1e-6 ({it} iterations) then 10 steps at c dt = h/2",
                 spec=spec, prec=prec, value=value, ms_step=1e3 * wall / (it + 10), stage=stage,
                 sched=None, extra_config={"config": 1, "l2": "the whole problem (4 MB) is L2-resident",
                                           "static_iterations": int(it)},
                 errors=errors, e2e=e2e, launches=launches, clk=clk.summary(), cpu=cpu,
                 sweep_ms=stage.get("sweep"),
                 notes="launch- and latency-bound: 5.2e5 updates per step, the residual read after every "
                       "iteration synchronises")


def bench_single(args, dev, *, spec, prec, workload, extra, errors_spec, cpu_spec, plain_prec=None,
                 scattering=None, notes=None, report_every=None):
    """Device-timed steps of one problem, its end-to-end leg (fields
    uploaded, one step, the FP64 sums read back every step, as in the
    benchmark's own leg; with report_every, that many steps and then the
    moments J, H, K read back, the workload's Eddington-tensor report) and
    the oracle's rate on a sample."""
    import numpy as np
    import torch

    from paper_1507_05141_gb300 import native
    stream = torch.cuda.Stream(dev)
    torch.cuda.set_stream(stream)
    s = native.Solver.from_spec(spec, device=dev.index, precision=prec, scattering=scattering)
    if args.source_path != "auto":
        s.set_source_path(args.source_path)
    if args.sweep_schedule:
        sc, snt = (int(v) for v in args.sweep_schedule.split(","))
        s.set_sweep_schedule(sc, snt)
    s.zero_state()
    ms, stage, clk, launches = time_steps(s, spec, args.steps, args.warmup, stream, dev, lambda: None)
    sched = _sched(s)
    src_path = s.source_path()
    upd = spec.updates_per_step
    value = upd * args.steps / (ms / 1e3)

    def pinned(a):
        t = torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64)).pin_memory()
        return t, t.numpy()
    fields = [spec.alpha0, spec.ne, spec.u, spec.emis0]
    if spec.extra.get("theta_e") is not None:
        fields.append(spec.extra["theta_e"])
    hold = [pinned(x) for x in fields]
    arrs = [h[1] for h in hold]
    h2d = sum(a.nbytes for a in arrs)
    d2h = 3 * 8
    e2e_steps = report_every or max(1, min(args.steps, 3))
    torch.cuda.synchronize(dev)
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        s.set_fields(*arrs)
        s.step(1, stream.cuda_stream)
        s.sums()
    if report_every:
        J, H, K = s.moments()  # the report: f_ij = K_ij / J on the host
        d2h += (J.nbytes + H.nbytes + K.nbytes) / report_every
    torch.cuda.synchronize(dev)
    e2e_s = time.perf_counter() - t0
    s.close()
    del s
    torch.cuda.empty_cache()
    plain = None
    if plain_prec:
        p = native.Solver.from_spec(spec, device=dev.index, precision=plain_prec, scattering=scattering)
        p.zero_state()
        ms32, stage32, _, _ = time_steps(p, spec, args.steps, args.warmup, stream, dev, lambda: None)
        p.close()
        del p
        torch.cuda.empty_cache()
        plain = {"value": upd * args.steps / (ms32 / 1e3), "unit": UNIT, "ms_per_step": ms32 / args.steps,
                 "stage_ms": stage32}
    errors = None
    if not args.no_errors and errors_spec is not None:
        errors = {q: _errors_vs_oracle(errors_spec, q, dev.index, scattering=scattering)
                  for q in ([prec, plain_prec] if plain_prec else [prec])}
    cpu = None
    if not args.no_cpu and cpu_spec is not None:
        v, dt = _oracle_rate(cpu_spec, 1, scattering=scattering)
        cores = int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1))
        cpu = {"value": v, "unit": UNIT, "cores": cores, "kind": "oracle",
               "sample": f"one FP64 oracle step of the same recipe on a {cpu_spec.grid[0]}^3 grid with G = "
                         f"{cpu_spec.G} ({cpu_spec.updates_per_step:.3g} updates, {dt:.1f} s)"}
    e2e = {"value": upd * e2e_steps / e2e_s, "unit": UNIT, "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
           "steps": e2e_steps}
    if report_every:
        e2e["report"] = f"J, H, K read back after the {report_every} steps (the Eddington tensor report)"
    extra = dict(extra)
    extra["source_pass"] = {"path": {0: "untimed", 1: "CUDA cores", 2: "tensor cores"}[src_path[0]],
                            "ms_cuda_cores": src_path[1], "ms_tensor_cores": src_path[2]}
    return _line(args, workload=workload, spec=spec, prec=prec, value=value, ms_step=ms / args.steps, stage=stage,
                 sched=sched, extra_config=extra, errors=errors, e2e=e2e, launches=launches, clk=clk, cpu=cpu,
                 sweep_ms=stage.get("sweep"), plain=plain, notes=notes)


def bench_config3(args, dev):
    import torch

    from paper_1507_05141_gb300 import inputs
    free, _ = torch.cuda.mem_get_info(dev)
    n = args.grid or 96
    L = args.order or 7
    spec, G = _fit_groups(lambda g: inputs.compton_shell(n=n, G=g, L=L), args.groups or 32, free)
    note = None if G == 32 else (f"G = {G} by --groups (a profiling case, not the workload)" if args.groups
                                 else f"G reduced from 32 to {G} to fit the device memory (stated deviation)")
    kind = "kn_thermal" if args.thermal else "kn"
    what = ("Compton scattering off thermal electrons at the recipe's temperature field" if args.thermal
            else "cold Klein-Nishina")
    return bench_single(args, dev, spec=spec, prec="mixed",
                        workload=f"Compton shell {n}^3, {G} groups (1e-4..1e2 m_e c^2), L={L}, "
                                 f"{spec.nmu}x{spec.nphi} ordinates, {what}, shell flow Gamma 2..5",
                        extra={"config": 3, "scattering": kind,
                               "l2": "no flush: the intensity state is far larger than L2"},
                        errors_spec=inputs.compton_shell(n=16, G=8),
                        cpu_spec=inputs.compton_shell(n=20, G=8 if args.thermal else G),
                        plain_prec=None if args.no_compare else "fp32", scattering=kind, notes=note)


def bench_config5(args, dev):
    import torch

    from paper_1507_05141_gb300 import inputs
    free, _ = torch.cuda.mem_get_info(dev)
    n = args.grid or 128
    spec, G = _fit_groups(lambda g: inputs.jet_cocoon(n=n, G=g), 64, free)
    note = (f"G reduced from 64 to {G}: with the laboratory eta, chi materialised in FP32 the 64-group state "
            f"needs about {_do_bytes(inputs.jet_cocoon(n=16, G=64)) * 512 / 1e9:.0f} GB (stated deviation)")
    return bench_single(args, dev, spec=spec, prec="mixed",
                        workload=f"jet in a cocoon {n}^3, {G} groups (1e-4..1e2 m_e c^2), L=7, 16x32 ordinates, "
                                 f"Gamma=30 core, cold Klein-Nishina",
                        extra={"config": 5, "l2": "no flush: the intensity state is far larger than L2"},
                        errors_spec=inputs.jet_cocoon(n=16, G=8), cpu_spec=inputs.jet_cocoon(n=20, G=G),
                        plain_prec=None, notes=note, report_every=50)


def bench_config4(args, dev):
    """The largest seeded prefix of the 256-problem batch that fits in 85 %
    of the free device memory, stepped as one CUDA graph launch per step; the
    same problems stepped one by one for comparison."""
    import torch

    from paper_1507_05141_gb300 import inputs, native
    free, _ = torch.cuda.mem_get_info(dev)
    budget = 0.85 * free
    specs, used = [], 0
    for i in range(256):
        sp = inputs.batch_problem(i)
        b = _do_bytes(sp)
        if used + b > budget:
            break
        specs.append(sp)
        used += b
    stream = torch.cuda.Stream(dev)
    sptr = stream.cuda_stream
    t0 = time.perf_counter()
    solvers = [native.Solver.from_spec(sp, device=dev.index, precision="mixed") for sp in specs]
    for s in solvers:
        s.zero_state()
    setup_s = time.perf_counter() - t0
    upd = sum(sp.updates_per_step for sp in specs)
    batch = native.Batch(solvers)
    batch.step(args.warmup, sptr)
    torch.cuda.synchronize(dev)
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with ClockSampler(dev.index) as clk:
        n0 = native.launch_count()
        ev0.record(stream)
        batch.step(args.steps, sptr)
        ev1.record(stream)
        launches = native.launch_count() - n0
        torch.cuda.synchronize(dev)
    ms = ev0.elapsed_time(ev1)
    # the same batch with the plane sweeps of each kernel variant in one
    # persistent launch
    batch.set_sweep_mode(1)
    batch.step(2, sptr)
    torch.cuda.synchronize(dev)
    ev0.record(stream)
    batch.step(args.steps, sptr)
    ev1.record(stream)
    torch.cuda.synchronize(dev)
    ms_one = ev0.elapsed_time(ev1)
    batch.set_sweep_mode(0)
    batch.step(2, sptr)
    # one by one
    for s in solvers:
        s.step(1, sptr)
    torch.cuda.synchronize(dev)
    ev0.record(stream)
    for _ in range(args.steps):
        for s in solvers:
            s.step(1, sptr)
    ev1.record(stream)
    torch.cuda.synchronize(dev)
    ms_seq = ev0.elapsed_time(ev1)
    # end to end: the batch step plus every problem's sums read back
    t0 = time.perf_counter()
    for _ in range(max(1, min(args.steps, 3))):
        batch.step(1, sptr)
        for s in solvers:
            s.sums()
    e2e_s = (time.perf_counter() - t0) / max(1, min(args.steps, 3))
    batch.close()
    cpu = None
    if not args.no_cpu:
        sp = inputs.batch_problem(0)
        v, dt = _oracle_rate(sp, 1)
        cores = int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1))
        cpu = {"value": v, "unit": UNIT, "cores": cores, "kind": "oracle",
               "sample": f"one FP64 oracle step of batch problem 0 ({sp.grid[0]}^3, G={sp.G}, L={sp.L}, {dt:.1f} s)"}
    for s in solvers:
        s.close()
    peak, peak_kind = _peaks()
    return {"metric": METRIC, "value": upd * args.steps / (ms / 1e3), "unit": UNIT, "n_gpus": 1,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": f"batch of independent problems: the first {len(specs)} of 256 seeded problems "
                                   f"(n 16..64 cubic, G 8..32, L 3/5/7, random jet axis, Gamma 1..20, "
                                   f"Thomson or KN), mixed precision, one graph launch per step",
                       "config": 4, "problems": len(specs), "updates_per_step": upd,
                       "device_bytes_estimate": used, "setup_s": setup_s,
                       "l2": "no flush: the states are far larger than L2", "parallelism": "replicas x1"},
            "one_by_one": {"value": upd * args.steps / (ms_seq / 1e3), "unit": UNIT,
                           "ms_per_step": ms_seq / args.steps},
            "batch_one_sweep_launch": {"value": upd * args.steps / (ms_one / 1e3), "unit": UNIT,
                                       "ms_per_step": ms_one / args.steps,
                                       "note": "sweep mode 1: the plane sweeps of each kernel variant in one "
                                               "persistent launch after every member's other stages"},
            "roofline": {"kernel": "whole batch step", "bound": "hbm",
                         "achieved": upd * STEP_FLOOR_BYTES_PER_UPDATE["mixed"] / (ms / args.steps / 1e3) / 1e9,
                         "peak": peak, "unit": "GB/s", "peak_kind": peak_kind,
                         "frac": upd * STEP_FLOOR_BYTES_PER_UPDATE["mixed"] / (ms / args.steps / 1e3) / 1e9 / peak,
                         "traffic": None, "algorithmic_bytes": "10 B/update (the step's floor)"},
            "e2e": {"value": upd / e2e_s, "unit": UNIT, "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 24 * len(specs), "steps": max(1, min(args.steps, 3))},
            "gpu_launches": launches, "clocks": clk.summary(), "cpu_baseline": cpu,
            "notes": f"the 256 problems need about {sum(_do_bytes(inputs.batch_problem(i)) for i in range(256)) / 1e9:.0f} "
                     f"GB; the prefix that fits is stepped (stated deviation)"}


def bench_other(args):
    import torch
    torch.cuda.set_device(0)
    dev = torch.device("cuda", 0)
    fn = {1: bench_config1, 3: bench_config3, 4: bench_config4, 5: bench_config5}[args.config]
    line = fn(args, dev)
    print(json.dumps(line))
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=None,
                    help="timed steps (default: 100, the jet workload's run length, for config 2; 20 otherwise)")
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--precision", default="mixed", choices=["fp32", "mixed", "fp64"])
    ap.add_argument("--no-compare", action="store_true", help="skip the plain-FP32 arm of a mixed run")
    ap.add_argument("--no-errors", action="store_true", help="skip the per-field error check against the oracle")
    ap.add_argument("--no-cpu", action="store_true", help="skip the CPU-baseline sample")
    ap.add_argument("--thermal", action="store_true",
                    help="config 3 with Compton scattering off thermal electrons (the temperature field's kernel)")
    ap.add_argument("--no-e2e", action="store_true",
                    help="skip the end-to-end leg (profiling: every launch then is a direct launch)")
    ap.add_argument("--config", type=int, default=2, choices=[1, 2, 3, 4, 5],
                    help="workload: 2 = the relativistic jet (the benchmark); 1 static FP64 box, 3 Compton shell, "
                         "4 batch of independent problems, 5 jet in a cocoon")
    ap.add_argument("--groups", type=int, default=None,
                    help="config 3: groups (default 32; fewer for small profiling captures)")
    ap.add_argument("--order", type=int, default=None,
                    help="config 3: angular order L (default 7; lower for small profiling captures)")
    ap.add_argument("--grid", type=int, default=None,
                    help="nodes per axis (defaults: 64 for the jet, 96 for config 3, 128 for config 5; smaller "
                         "for profiling)")
    ap.add_argument("--sweep-schedule", default=None, metavar="C,NT",
                    help="force the FP32 sweep schedule (cluster CTAs, threads) instead of timing the candidates")
    ap.add_argument("--source-path", default="auto", choices=["auto", "cuda", "tensor"],
                    help="source pass of group-mixing kernels in MIXED (configs 3, 5): timed choice or forced")
    args = ap.parse_args()
    if args.steps is None:
        args.steps = 100 if (args.config == 2 and args.impl == "ours") else 20
    if args.warmup < 3 and args.impl == "ours":
        print("warning: fewer than 3 warm-up steps", file=sys.stderr)
    if args.impl == "reference":
        return bench_reference(args)
    if args.config != 2:
        return bench_other(args)
    if args.grid is None:
        args.grid = 64
    return bench_ours(args)


if __name__ == "__main__":
    sys.exit(main())
