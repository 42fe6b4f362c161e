"""Throughput of the GB300 ADER-AFE-DG step: DOF-updates/s on the density-wave workload.

Workload (one GPU): the smooth density wave rho = 1 + 0.2 sin(2 pi (x+y+z)), u = (1,1,1),
p = 1 on the periodic unit cube, jittered-lattice Voronoi mesh with 32^3 cells and fan
subgrids, AFE degree N = 3, Euler, at the largest CFL at which these meshes run the workload
stably (0.15 at N = 3; the paper's 0.3 diverges on them at N >= 2 and is timed beside it as
``fp32_paper_cfl``).  A DOF-update is one conserved variable at one
AFE node advanced by one full ADER step (limiter check, time step, predictor, face fluxes,
corrector).  ``value`` is the reduced-precision form (FP32 arithmetic, FP64 master state,
FP64 time step and conservative cell totals); the plain FP64 form is timed beside it.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
  python bench.py --serve      (continuous-batching serving run alone; see run_serving())

N > 1 (torchrun): every rank runs an independent simulation (mesh seed = rank); there is
no data-path collective and ``value`` is the sum over ranks of DOF-updates over the max
over ranks of the timed wall.  ``--impl reference`` times the CPU oracle (the plain FP64
restatement of the paper's scheme) on a bounded sample of the same workload.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "DOF-updates/s per ADER-DG step"

# Largest CFL numbers at which the fan-subgrid Voronoi meshes of inputs.voronoi run the
# density wave stably to t = 0.1 (measured on 16^3 and 32^3 meshes, both forms): the
# paper's 0.3 holds for N = 1; at N = 2 a 32^3 mesh diverges after ~200 steps at 0.3, and at
# N = 3 within 8 steps at 0.3 and after ~30 at 0.2.
STABLE_CFL = {1: 0.3, 2: 0.2, 3: 0.15}
PAPER_CFL = 0.3

# DRAM bytes (read + write) of one predictor_f32_kernel<3> launch per cell of the density-wave
# workload, from one ncu capture (dram__bytes_read.sum + dram__bytes_write.sum) of a 12^3 launch
# of the current kernel; None until that capture exists.  The fixed-point iterations re-read
# M_i^-1 from L2, so the traffic grows with the cells, not with the iterations.
PREDICTOR_N3_DRAM_BYTES_PER_CELL = (812361984 + 40285696) / 1728
UNIT = "DOF-updates/s"


def _args():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--n", type=int, default=32, help="cells per direction of the jittered lattice")
    ap.add_argument("--order", type=int, default=3)
    ap.add_argument("--fp64-steps", type=int, default=2, help="timed steps of the plain FP64 form (0: skip)")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cfl", type=float, default=None,
                    help="CFL number (default: the largest stable one of STABLE_CFL; the paper's is 0.3)")
    ap.add_argument("--visc-dt", default="subtet", choices=["subtet", "cell"],
                    help="shock/tgv: length in the viscous term of the time step (the smallest "
                         "sub-tet length, or the cell length as printed; see the stokes study)")
    ap.add_argument("--no-autotune", dest="autotune", action="store_false",
                    help="keep the default predictor schedule instead of the autotuned one")
    ap.add_argument("--variant", type=int, default=0, choices=[0, 1],
                    help="FP32 predictor's M_i^-1 apply: 0 mma.sync, 1 tcgen05 with tensor memory")
    ap.add_argument("--serve", action="store_true", help="serving run: Poisson requests on small meshes")
    ap.add_argument("--study", choices=["convergence", "stokes", "vortex", "shock", "tgv"],
                    help="accuracy study instead of the throughput run")
    ap.add_argument("--workload", default="density", choices=["density", "shock", "tgv"],
                    help="density: density wave, periodic unit cube, Euler; shock: spherical explosion on "
                         "[-1,1]^3, transmissive, limiter on; tgv: Navier-Stokes Taylor-Green vortex on "
                         "[0,2pi)^3, mu 0.01")
    ap.add_argument("--serve-requests", type=int, default=64)
    ap.add_argument("--serve-rate", type=float, default=50.0, help="offered load, requests per second")
    ap.add_argument("--serve-steps", type=int, default=100, help="CFL steps per request")
    ap.add_argument("--serve-slots", type=int, default=4, help="slots per catalogue entry (mesh, N)")
    ap.add_argument("--serve-elastic", type=float, default=None, metavar="BYTES",
                    help="admit by device footprint within BYTES instead of fixed slot pools")
    ap.add_argument("--serve-no-limiter", dest="serve_limiter", action="store_false",
                    help="explosion requests without the limiter (they may end non-finite)")
    ap.add_argument("--no-serving", action="store_true", help="skip the serving record of the throughput run")
    return ap.parse_args()


def workload_name(n, N, workload="density"):
    if workload == "shock":
        return (f"spherical explosion (smoothed over 1.5 lattice spacings) on [-1,1]^3 (transmissive), {n}^3 "
                f"jittered-Voronoi cells (fan subgrid), AFE N={N}, Euler with the artificial-viscosity limiter")
    if workload == "tgv":
        return (f"Taylor-Green vortex on [0,2pi)^3 (periodic), {n}^3 jittered-Voronoi cells (fan subgrid), "
                f"AFE N={N}, Navier-Stokes mu 0.01 Pr 0.71")
    return f"density-wave periodic unit cube, {n}^3 jittered-Voronoi cells (fan subgrid), AFE N={N}, Euler"


# ----------------------------------------------------------------------------------------
# CPU oracle (reference arm and cpu_baseline)

_ORACLE_SNIPPET = r"""
import json, sys, time
sys.path.insert(0, {root!r})
from inputs import states
from inputs.voronoi import periodic_voronoi
from oracle.mesh import from_polymesh
from oracle import scheme
pm = periodic_voronoi({n})
m = from_polymesh(pm, {N})
prm = scheme.Params(cfl={cfl})
uc = m.split(states.density_wave(m.node_coords()))
dt = scheme.cfl_dt(m, uc, [0.0] * m.n_cells, prm) * {dt_scale}
out = []
wall0 = time.time()
for s in range({steps}):
    t0 = time.perf_counter()
    uc, info = scheme.step(m, uc, prm, dt=dt)
    out.append(time.perf_counter() - t0)
print(json.dumps(dict(times=out, dofs=5 * m.n_nodes, cells=m.n_cells, iters=float(info.iterations.mean()),
                      wall=[wall0, time.time()])))
"""


def run_oracle(n_sample, N, steps, dt_scale, cfl):
    """Run the oracle in a fresh single-threaded process; returns its JSON record."""
    env = dict(os.environ, OMP_NUM_THREADS="1", OPENBLAS_NUM_THREADS="1", MKL_NUM_THREADS="1")
    code = _ORACLE_SNIPPET.format(root=ROOT, n=n_sample, N=N, steps=steps, dt_scale=dt_scale, cfl=float(cfl))
    r = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, env=env)
    if r.returncode != 0:
        raise RuntimeError("oracle run failed: " + r.stderr[-2000:])
    return json.loads(r.stdout.strip().splitlines()[-1])


def oracle_all_cores(N, cfl, procs=None):
    """The same one-step oracle sample run by ``procs`` single-threaded processes at once
    (default: every host core), each on its own copy of the 6^3 mesh: the host's aggregate
    oracle throughput over independent problems, all DOF-updates over the span from the
    first step's start to the last step's end.  Returns (DOF-updates/s, processes)."""
    procs = procs or os.cpu_count() or 1
    env = dict(os.environ, OMP_NUM_THREADS="1", OPENBLAS_NUM_THREADS="1", MKL_NUM_THREADS="1")
    code = _ORACLE_SNIPPET.format(root=ROOT, n=6, N=N, steps=1, dt_scale=1.0, cfl=float(cfl))
    runs = [subprocess.Popen([sys.executable, "-c", code], stdout=subprocess.PIPE, stderr=subprocess.PIPE, text=True,
                             env=env) for _ in range(procs)]
    dofs, starts, ends = 0, [], []
    for r in runs:
        out, err = r.communicate()
        if r.returncode != 0:
            raise RuntimeError("oracle run failed: " + err[-2000:])
        rec = json.loads(out.strip().splitlines()[-1])
        dofs += rec["dofs"]
        starts.append(rec["wall"][0])
        ends.append(rec["wall"][1])
    return dofs / (max(ends) - min(starts)), procs


def oracle_sample(N, steps, cfl):
    """A bounded sample of the workload for the oracle: full steps of the same generator,
    order and CFL on the 6^3 periodic mesh."""
    n_s = 6
    return n_s, run_oracle(n_s, N, steps, 1.0, cfl)


def reference_arm(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    n_s = 6
    cfl = args.cfl if args.cfl is not None else STABLE_CFL[args.order]
    rec = run_oracle(n_s, args.order, args.warmup + args.steps, 1.0, cfl)
    times = rec["times"][args.warmup:]
    t = sum(times)
    value = rec["dofs"] * len(times) / t
    sample = (f"oracle (numpy FP64, 1 thread) full steps on the {n_s}^3 periodic mesh of the same generator, "
              f"N={args.order}, CFL {cfl:g} ({rec['cells']} cells, {rec['dofs']} DOFs per step)")
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": len(times), "warmup": args.warmup, "ms_per_step": 1e3 * t / len(times), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": workload_name(args.n, args.order), "sample_mesh": f"{n_s}^3"},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle", "sample": sample},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }), flush=True)


# ----------------------------------------------------------------------------------------
# clocks during the timed region


class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index):
        self.idx = device_index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.idx}", f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except OSError:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx.append(float(parts[2]))
            except ValueError:
                continue
            for name, val in zip(names, parts[5:9]):
                if val.lower() == "active":
                    reasons.add(name)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        sm.sort()
        return {"sm_mhz": sm[len(sm) // 2], "sm_max_mhz": max(mx), "reasons": sorted(reasons), "samples": len(sm)}


# ----------------------------------------------------------------------------------------


def predictor_model(node_ptr, sub_ptr, iters, N, real_bytes):
    """Algorithmic work of one predictor launch (the dominant kernel), split by the pipe the
    design puts it on.

    Per cell and fixed-point iteration, with Np = (N+1)(N+2)(N+3)/6, Nt = N+1, S sub-tets,
    N_i nodes.  Dense contractions (tensor cores): the reference-stiffness contraction,
    2 * 3 Np flop per (sub-tet, time, node, variable), and the inverse-mass apply
    2 N_i^2 (5 Nt); the epilogue's volume-term contraction once per step.  Pointwise work
    (FP32 FMA pipe): flux and 3x3 pre-contraction 150 flop per (sub-tet, time, node), the
    agglomeration 1 flop per incidence and variable, the update 2 Nt per (node, time,
    variable), and the epilogue's flux pass.  Bytes (the method's minimum): M_i^-1 once per
    step (N_i^2 words; row padding is storage, not work), the state, the sub-tet records and
    the outputs once; the variant that streams M_i^-1 from HBM in every fixed-point
    iteration is returned beside it.  Returns (contraction flops, pointwise flops, bytes,
    streamed bytes).
    """
    import numpy as np
    Np = (N + 1) * (N + 2) * (N + 3) // 6
    Nt = N + 1
    Ni = np.diff(node_ptr).astype(np.float64)
    S = np.diff(sub_ptr).astype(np.float64)
    it = iters.astype(np.float64)
    con_it = S * Nt * Np * 5 * 6 * Np + 2 * Ni * Ni * 5 * Nt
    pw_it = S * Nt * Np * (150 + 5) + Ni * Nt * 5 * 2 * Nt
    con_epi = S * Np * 5 * 6 * Np
    pw_epi = S * Np * Nt * 150 + S * Np * 5
    f_con = float(np.sum(it * con_it + con_epi))
    f_pw = float(np.sum(it * pw_it + pw_epi))
    once = Ni * 5 * 8 + S * (10 * 4 + Np * 2) + Ni * 5 * real_bytes
    bytes_min = float(np.sum(Ni * Ni * real_bytes + once))
    bytes_streamed = float(np.sum(it * Ni * Ni * real_bytes + once))
    return f_con, f_pw, bytes_min, bytes_streamed


def predictor_roofline(f_con, f_pw, abytes, ms, peaks):
    """Time-based roofline of one predictor launch against the pipes the design assigns:
    contractions on the tensor cores as 3xTF32 (the TF32 dense peak, taken as half the
    measured BF16 burst peak by the nominal 1:2 ratio, divided by the three products of
    the split), pointwise work on the FP32 FMA pipe (152 SMs x 128 lanes x 2 flop x the
    maximum SM clock), bytes at the measured HBM copy bandwidth.  The roofline time is
    max(t_hbm, t_tensor + t_fma); the main fields follow the bound that sets it."""
    hbm = peaks.get("hbm_gbs") or 6800.0
    bf16 = peaks.get("bf16_tflops") or 1900.0
    sm_max = peaks.get("sm_max_mhz") or 2070.0
    tf32 = bf16 / 2.0
    tensor_eff = tf32 / 3.0
    fma = 152 * 128 * 2 * sm_max * 1e6 / 1e12
    t = ms / 1e3
    t_hbm = abytes / (hbm * 1e9)
    t_ten = f_con / (tensor_eff * 1e12)
    t_fma = f_pw / (fma * 1e12)
    t_roof = max(t_hbm, t_ten + t_fma)
    if t_hbm >= t_ten + t_fma:
        ach = abytes / t / 1e9
        out = {"bound": "hbm", "achieved": ach, "peak": hbm, "unit": "GB/s", "frac": ach / hbm,
               "peak_note": "of measured (HBM copy bandwidth)"}
    else:
        ach = f_con / t / 1e12
        out = {"bound": "tensor", "achieved": ach, "peak": tensor_eff, "unit": "TFLOP/s", "frac": ach / tensor_eff,
               "peak_note": "3xTF32 effective: half the measured BF16 burst peak (nominal TF32:BF16 ratio) / 3"}
    out.update({"frac_roofline_time": t_roof / t, "roofline_ms": t_roof * 1e3, "measured_ms": ms,
                "pipes_ms": {"hbm": t_hbm * 1e3, "tensor_3xtf32": t_ten * 1e3, "fp32_fma": t_fma * 1e3},
                "peaks": {"hbm_gbs": hbm, "tf32_tflops": tf32, "tensor_3xtf32_tflops": tensor_eff,
                          "fp32_fma_tflops": fma},
                "algorithmic_flops_contraction": f_con, "algorithmic_flops_pointwise": f_pw,
                "algorithmic_bytes": abytes})
    return out


class RankReducer:
    """Max / sum of one float over the ranks of a process group (identity without one).

    ``device`` is where the reduction tensor lives: "cuda" under NCCL, "cpu" under gloo."""

    def __init__(self, dist=None, device="cpu"):
        self.dist = dist
        self.device = device

    def _reduce(self, x, op):
        if self.dist is None:
            return float(x)
        import torch
        t = torch.tensor([float(x)], dtype=torch.float64, device=self.device)
        self.dist.all_reduce(t, op=op)
        return float(t.item())

    def max(self, x):
        return self._reduce(x, None if self.dist is None else self.dist.ReduceOp.MAX)

    def sum(self, x):
        return self._reduce(x, None if self.dist is None else self.dist.ReduceOp.SUM)


def throughput(red, dofs_per_step, steps, ms):
    """Whole-job DOF-updates/s: DOF-updates of all ranks over the slowest rank's time."""
    ms_max = red.max(ms)
    return red.sum(dofs_per_step * steps) / (ms_max / 1e3), ms_max


def equal_steps_accuracy(N, cfl, n=8, t_end=0.1):
    """Both forms on the density wave of the throughput workload's order and CFL, on the
    n^3 mesh of the same generator, to t_end with the same steps: the L2 error of rho against
    the exact solution (volume-weighted nodal norm) of each form and their relative
    difference.  The ratio of the throughput line compares the forms at equal steps, so it
    holds at equal error when these two errors agree."""
    import numpy as np

    from inputs import states
    from inputs.voronoi import periodic_voronoi
    from paper_2605_00619_gb300 import afe
    pm = periodic_voronoi(n)
    sub = pm.subtet_coords()
    vol = np.bincount(np.repeat(np.arange(pm.n_cells), np.diff(pm.cell_subtet_ptr)),
                      weights=np.abs(np.linalg.det(sub[:, 1:] - sub[:, :1])) / 6.0, minlength=pm.n_cells)
    out = {"mesh": f"{n}^3", "N": N, "cfl": cfl, "t": t_end}
    rho = {}
    for name, prec in (("fp32", afe.AFE_FP32), ("fp64", afe.AFE_FP64)):
        fp32 = prec == afe.AFE_FP32
        p = afe.afe_default_params(N, precision=prec, picard_tol=1e-6 if fp32 else 1e-12,
                                   picard_max=128 if fp32 else 64, cfl=cfl)
        h = afe.create_from_polymesh(pm, p)
        x = afe.afe_get_node_coords(h)
        ptr = afe.afe_node_ptr(h, pm.n_cells)
        afe.afe_set_state(h, states.density_wave(x))
        if name == "fp32":
            nsteps = int(math.ceil(t_end / afe.afe_compute_dt(h) - 1e-9))
            dt = t_end / nsteps
        afe.afe_step_async(h, dt, nsteps)
        st = afe.afe_sync(h, check=False)
        q = afe.afe_get_state(h)
        afe.afe_mesh_destroy(h)
        e2 = (q[:, 0] - states.density_wave(x, t=t_end)[:, 0]) ** 2
        out[f"l2_rho_{name}"] = float(np.sqrt(np.sum(vol * np.add.reduceat(e2, ptr[:-1]) / np.diff(ptr))))
        out[f"status_{name}"] = int(st)
        rho[name] = q[:, 0]
    out["steps"] = nsteps
    out["rel_l2_fp32_vs_fp64"] = float(np.linalg.norm(rho["fp32"] - rho["fp64"]) / np.linalg.norm(rho["fp64"]))
    out["note"] = ("the throughput ratio is at equal steps; on this smaller mesh of the same generator both forms "
                   "reach the same L2 error of rho against the exact solution (CFL below the paper's 0.3, at "
                   "which these meshes diverge for N >= 2)")
    return out


def ours(args):
    import numpy as np
    import torch

    from inputs import states
    from inputs.voronoi import periodic_voronoi
    from paper_2605_00619_gb300 import afe

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    afe.lib()

    def barrier():
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()

    red = RankReducer(dist, "cuda")
    max_over_ranks, sum_over_ranks = red.max, red.sum

    from inputs.voronoi import box_voronoi
    if args.workload == "shock":
        pm = box_voronoi(args.n, seed=rank)
    elif args.workload == "tgv":
        pm = periodic_voronoi(args.n, L=2 * math.pi, seed=rank)
    else:
        pm = periodic_voronoi(args.n, seed=rank)
    stream = torch.cuda.Stream()
    sid = stream.cuda_stream
    peaks = {}
    try:
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except (OSError, ValueError):
        pass

    def run_form(prec, steps, warmup, e2e, cfl):
        fp32 = prec == afe.AFE_FP32
        extra = {}
        if args.workload == "shock":
            extra = dict(limiter=1)
        elif args.workload == "tgv":
            extra = dict(equations=afe.AFE_NAVIER_STOKES, mu=0.01, Pr=0.71, kappa=-1.0,
                         visc_dt_subtet=int(args.visc_dt == "subtet"))
        if args.workload == "shock":
            extra["visc_dt_subtet"] = int(args.visc_dt == "subtet")
        p = afe.afe_default_params(args.order, precision=prec, picard_tol=1e-6 if fp32 else 1e-12,
                                   picard_max=128 if fp32 else 64, cfl=cfl, **extra)
        h = afe.create_from_polymesh(pm, p, stream=sid)
        tune = None
        if prec == afe.AFE_FP32:
            afe.afe_set_predictor_variant(h, args.variant)
        n_nodes = afe.afe_num_nodes(h)
        node_ptr = afe.afe_node_ptr(h, pm.n_cells)
        x = afe.afe_get_node_coords(h)
        if args.workload == "shock":  # smoothed over 1.5 lattice spacings
            u0 = states.spherical_riemann(x, alpha0=1.5 * 2.0 / args.n)
        elif args.workload == "tgv":
            u0 = states.taylor_green_3d(x, p0=100.0)
        else:
            u0 = states.density_wave(x)
        afe.afe_set_state(h, u0)
        if fp32 and args.autotune:
            sched, best_ms, default_ms = afe.afe_autotune(h, 3)
            tune = {"cost_order": sched.cost_order, "variant": sched.variant, "ring_cap": sched.ring_cap,
                    "narrow": sched.narrow, "predictor_ms": best_ms, "default_schedule_ms": default_ms}
        afe.afe_step_async(h, 0.0, warmup)
        st = afe.afe_sync(h, check=False)
        barrier()
        afe.afe_set_profiling(h, True)
        afe.afe_stage_times(h, reset=True)
        launches0 = afe.afe_get_stats(h).kernel_launches
        clocks = ClockSampler(local)
        clocks.start()
        ev0 = torch.cuda.Event(enable_timing=True)
        ev1 = torch.cuda.Event(enable_timing=True)
        barrier()
        t0 = time.perf_counter()
        ev0.record(stream)
        afe.afe_step_async(h, 0.0, steps)
        ev1.record(stream)
        stream.synchronize()
        barrier()
        wall = time.perf_counter() - t0
        clk = clocks.stop()
        ms = ev0.elapsed_time(ev1)
        st2 = afe.afe_sync(h, check=False)
        stage_ms, nst = afe.afe_stage_times(h, reset=True)
        afe.afe_set_profiling(h, False)
        stats = afe.afe_get_stats(h)
        launches = stats.kernel_launches - launches0
        _, iters, _, _ = afe.afe_get_diagnostics(h, pm.n_cells, qbar=False)
        rec = dict(status=[st, st2], ms=ms, wall=wall, stage_ms=(stage_ms / max(nst, 1)).tolist(), clocks=clk,
                   n_nodes=n_nodes, launches=launches, iters_mean=float(iters.mean()), iters_max=int(iters.max()),
                   nonconverged=int(stats.nonconverged), dt=stats.dt, bytes=afe.afe_device_bytes(h), schedule=tune)
        rec["f_con"], rec["f_pw"], rec["abytes"], rec["abytes_streamed"] = predictor_model(
            node_ptr, pm.cell_subtet_ptr, iters, args.order, 4 if prec == afe.AFE_FP32 else 8)
        if e2e:
            # end to end through the public API, host buffers: per step the state goes up from
            # pinned host memory, one step runs, the new state comes back
            hin = torch.empty((n_nodes, 5), dtype=torch.float64, pin_memory=True).numpy()
            hin[:] = u0
            barrier()
            t1 = time.perf_counter()
            for _ in range(steps):
                afe.afe_set_state(h, hin)
                afe.afe_step(h, 0.0, check=False)
                afe.afe_get_state(h, out=hin)
            barrier()
            rec["e2e_wall"] = time.perf_counter() - t1
        afe.afe_mesh_destroy(h)
        return rec

    cfl = args.cfl if args.cfl is not None else STABLE_CFL[args.order]
    r32 = run_form(afe.AFE_FP32, args.steps, args.warmup, not args.no_e2e, cfl)
    r64 = run_form(afe.AFE_FP64, args.fp64_steps, 1, False, cfl) if args.fp64_steps > 0 else None
    # the same FP32 step at the paper's CFL, which these meshes do not sustain at N >= 2
    rst = run_form(afe.AFE_FP32, args.steps, args.warmup, False, PAPER_CFL) if cfl != PAPER_CFL else None

    K = args.steps
    dofs = 5 * r32["n_nodes"]
    value, ms_max = throughput(red, dofs, K, r32["ms"])
    total_dofs = sum_over_ranks(dofs * K)
    out = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": K, "warmup": args.warmup,
        "ms_per_step": ms_max / K, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f32", "data": "synthetic",
        "config": {"workload": workload_name(args.n, args.order, args.workload)
                   + (f", viscous time step from the {args.visc_dt} length" if args.workload != "density" else ""),
                   "cells": pm.n_cells, "nodes": r32["n_nodes"],
                   "dofs": dofs, "precision": "FP32 arithmetic, FP64 master state / dt / cell totals",
                   "picard_tol": 1e-6, "l2": "inputs larger than L2 (M_i^-1 alone is "
                   f"{r32['bytes'] / 1e9:.1f} GB of device state)",
                   "parallelism": f"{world} independent replica" + ("s" if world > 1 else "")},
        "clocks": r32["clocks"],
        "gpu_launches": int(r32["launches"]),
        "status": {"fp32": r32["status"], "picard_iters_mean": r32["iters_mean"], "picard_iters_max": r32["iters_max"],
                   "nonconverged_cells": r32["nonconverged"]},
        "stage_ms_per_step": dict(zip(["limiter_dt", "predictor", "face", "corrector"], r32["stage_ms"])),
        "predictor_schedule": r32["schedule"],
    }
    if "e2e_wall" in r32:
        e2e_wall = max_over_ranks(r32["e2e_wall"])
        out["e2e"] = {"value": total_dofs / e2e_wall, "unit": UNIT, "h2d_bytes_per_step": r32["n_nodes"] * 5 * 8,
                      "d2h_bytes_per_step": r32["n_nodes"] * 5 * 8}
    # roofline of the dominant kernel (the predictor), by the pipes the design assigns
    pred_ms = r32["stage_ms"][1]
    out["roofline"] = predictor_roofline(r32["f_con"], r32["f_pw"], r32["abytes"], pred_ms, peaks)
    out["roofline"]["kernel"] = f"predictor_f32_kernel<{args.order}>"
    out["roofline"]["traffic"] = None
    out["roofline"]["algorithmic_bytes_streamed_per_iteration"] = r32["abytes_streamed"]
    if args.order == 3 and args.workload == "density" and PREDICTOR_N3_DRAM_BYTES_PER_CELL:
        out["roofline"]["traffic"] = PREDICTOR_N3_DRAM_BYTES_PER_CELL * pm.n_cells
        out["roofline"]["traffic_note"] = "ncu dram__bytes_read+write of a 12^3 launch, scaled by cells"
    out["config"]["cfl"] = cfl
    if rst is not None:
        v_st, ms_st = throughput(red, 5 * rst["n_nodes"], K, rst["ms"])
        finite = all(st == 0 for st in rst["status"])
        note = ("the paper's CFL; finite over the steps timed here, but on these meshes runs at N >= 2 "
                "diverge later at this CFL, so it is not a valid throughput over a full run" if finite else
                "the paper's CFL; on these meshes it diverges at N >= 2 (non-finite status within the "
                "timed steps), so this timing is not a valid throughput there")
        out["fp32_paper_cfl"] = {"cfl": PAPER_CFL, "value": v_st, "unit": UNIT, "ms_per_step": ms_st / K,
                                 "picard_iters_mean": rst["iters_mean"], "status": rst["status"], "note": note}
    if r64 is not None:
        ms64 = max_over_ranks(r64["ms"])
        out["fp64_plain"] = {"value": sum_over_ranks(5 * r64["n_nodes"] * args.fp64_steps) / (ms64 / 1e3),
                             "unit": UNIT, "ms_per_step": ms64 / args.fp64_steps, "status": r64["status"],
                             "picard_iters_mean": r64["iters_mean"],
                             "stage_ms_per_step": dict(zip(["limiter_dt", "predictor", "face", "corrector"],
                                                           r64["stage_ms"]))}
        out["fp32_over_fp64"] = value / out["fp64_plain"]["value"]
        if args.workload == "density":
            out["fp32_over_fp64_accuracy"] = equal_steps_accuracy(args.order, cfl)
    if rank == 0 and world == 1 and not args.no_serving and args.workload == "density":
        # bounded serving record: 64 requests of 100 steps on 8^3 - 16^3 meshes; the serial
        # FP64 comparison runs the first 16 of them
        try:
            out["serving"] = run_serving(64, 50.0, 100, serial_requests=16)
            out["serving"].pop("clocks", None)
        except Exception as e:  # the serving record never hides the throughput line
            out["serving"] = {"error": str(e)[:300]}
    if rank == 0 and not args.no_cpu_baseline:
        try:
            n_s, rec = oracle_sample(args.order, 1, cfl)
            cb = rec["dofs"] / rec["times"][0]
            out["cpu_baseline"] = {"value": cb, "unit": UNIT, "cores": 1, "kind": "oracle",
                                   "sample": f"one oracle step (numpy FP64, 1 thread) on the {n_s}^3 periodic mesh of "
                                             f"the same generator, N={args.order}, CFL {cfl:g} ({rec['cells']} cells, "
                                             f"{rec['dofs']} DOFs, {rec['iters']:.1f} mean fixed-point "
                                             f"iterations)"}
        except Exception as e:  # the baseline never hides the GPU number
            out["cpu_baseline"] = {"value": None, "unit": UNIT, "cores": 1, "kind": "oracle", "sample": str(e)[:200]}
        try:
            v_all, procs = oracle_all_cores(args.order, cfl)
            out["cpu_baseline_all_cores"] = {
                "value": v_all, "unit": UNIT, "cores": procs, "kind": "oracle",
                "sample": f"{procs} single-threaded oracle processes at once, each one step on its own 6^3 mesh, "
                          f"N={args.order}, CFL {cfl:g} (span from the first step's start to the last step's end)"}
        except Exception as e:
            out["cpu_baseline_all_cores"] = {"value": None, "unit": UNIT, "kind": "oracle", "sample": str(e)[:200]}
    if rank == 0:
        print(json.dumps(out), flush=True)
    if dist is not None:
        dist.destroy_process_group()


def run_serving(n_req, rate, steps, sizes=(8, 12, 16), limiter=True, slots_per_key=4, elastic_bytes=None,
                serial_requests=None, ratio=(2.0, 20.0), seed=12345):
    """Continuous batching of many independent simulations on one GPU; returns one record.

    Requests follow the serving workload of the method's evaluation, scaled to resident
    meshes: a mesh drawn uniformly from a catalogue of jittered-Voronoi meshes -- the periodic
    unit cube and the box [-1,1]^3 with ``sizes`` seeds per direction -- with N uniform in
    {1, 2, 3}; periodic meshes carry the density wave, box meshes a spherical explosion
    smoothed over 1.5 lattice spacings with a random centre in [-0.5,0.5]^3 and a pressure
    ratio uniform in ``ratio`` (with the limiter and the sub-tet viscous time step when
    ``limiter``); each request runs ``steps`` CFL steps.  Arrivals: a Poisson process of
    ``rate`` per second (seeded).  The catalogue's meshes and slots are built before the
    arrival clock starts.  The batched server (FP32 form; every occupied slot advanced together,
    one launch per stage and order, a CUDA graph per batch) runs every request; the serial
    server runs the first ``serial_requests`` (all by default) one at a time in the plain FP64
    form, so that its DOF-updates/s compare rate with rate.  ``elastic_bytes`` admits by device
    footprint within that budget instead of fixed pools of ``slots_per_key`` slots.
    """
    import numpy as np
    import torch

    from inputs import states
    from inputs.voronoi import box_voronoi, periodic_voronoi
    from paper_2605_00619_gb300 import afe
    from paper_2605_00619_gb300.serving import GpuEngine, Request, Server

    afe.lib()
    meshes = {}
    for n in sizes:
        meshes[f"p{n}"] = periodic_voronoi(n, seed=100 + n)
        meshes[f"b{n}"] = box_voronoi(n, seed=200 + n)

    def params(kind, N, prec):
        fp32 = prec == afe.AFE_FP32
        extra = dict(limiter=1, visc_dt_subtet=1) if kind == "b" and limiter else {}
        return afe.afe_default_params(N, precision=prec, picard_tol=1e-6 if fp32 else 1e-12,
                                      picard_max=128 if fp32 else 64, cfl=STABLE_CFL[N], **extra)

    keys = [f"{mk}_N{N}" for mk in sorted(meshes) for N in (1, 2, 3)]
    cat32 = {k: (meshes[k.split("_")[0]], params(k[0], int(k[-1]), afe.AFE_FP32)) for k in keys}
    cat64 = {k: (meshes[k.split("_")[0]], params(k[0], int(k[-1]), afe.AFE_FP64)) for k in keys}
    elastic = elastic_bytes is not None
    t_setup = time.perf_counter()
    eng = (GpuEngine(cat32, {}, budget_bytes=int(elastic_bytes)) if elastic
           else GpuEngine(cat32, {k: slots_per_key for k in keys}))
    ser = GpuEngine(cat64, {k: 1 for k in keys})
    t_setup = time.perf_counter() - t_setup
    rng = np.random.default_rng(seed)

    def make_requests(count, r):
        out, t = [], 0.0
        for i in range(count):
            t += rng.exponential(1.0 / r) if r > 0 else 0.0
            k = keys[int(rng.integers(len(keys)))]
            if k.startswith("p"):
                ic = states.density_wave
            else:
                c = rng.uniform(-0.5, 0.5, 3)
                pr = rng.uniform(*ratio)
                a0 = 1.5 * 2.0 / int(k.split("_")[0][1:])  # smoothing width: 1.5 lattice spacings
                ic = (lambda c_, r_, a_: lambda x: states.spherical_riemann(x, centre=tuple(c_), p_in=0.1 * r_,
                                                                             alpha0=a_))(c, pr, a0)
            out.append(Request(i, k, steps, t, q0=ic))
        return out

    Server(eng, elastic=elastic).run(make_requests(len(keys) if elastic else len(eng.slots), 0.0))  # warm-up
    Server(ser, mode="serial").run(make_requests(len(keys), 0.0))
    reqs = make_requests(n_req, rate)
    clocks = ClockSampler(torch.cuda.current_device())
    clocks.start()
    srv = Server(eng, max_chunk=8, elastic=elastic)
    sb = srv.run([Request(r.rid, r.mesh, r.nsteps, r.arrival, q0=r.q0) for r in reqs])
    clk = clocks.stop()
    sub = reqs[:serial_requests] if serial_requests else reqs
    ss = Server(ser, mode="serial").run([Request(r.rid, r.mesh, r.nsteps, r.arrival, q0=r.q0) for r in sub])
    out = {
        "metric": "serving throughput, continuous batching (FP32) vs serial plain FP64", "value": sb.throughput,
        "unit": UNIT, "higher_is_better": True, "n_gpus": 1, "dtype": "f32", "data": "synthetic",
        "requests": sb.requests, "p50_ms": 1e3 * sb.p50_s, "p99_ms": 1e3 * sb.p99_s, "mean_ms": 1e3 * sb.mean_s,
        "mean_batch_members": sb.mean_batch, "batch_steps": sb.steps_launched, "failed": sb.failed,
        "makespan_s": sb.makespan_s,
        "serial_fp64": {"value": ss.throughput, "unit": UNIT, "requests": ss.requests, "p50_ms": 1e3 * ss.p50_s,
                        "p99_ms": 1e3 * ss.p99_s, "makespan_s": ss.makespan_s, "failed": ss.failed,
                        "note": "the same requests one at a time in the plain FP64 form"
                                + (f" (the first {len(sub)} of {len(reqs)}: DOF-updates/s compare as rates)"
                                   if len(sub) < len(reqs) else "")},
        "batched_over_serial": sb.throughput / ss.throughput,
        "clocks": clk,
        "config": {"workload": f"{n_req} requests, Poisson arrivals at {rate:g}/s, {steps} CFL steps each; meshes "
                               f"periodic/box {', '.join(f'{n}^3' for n in sizes)}, N in {{1,2,3}}; density wave "
                               f"(periodic) or smoothed spherical explosion, pressure ratio {ratio[0]:g}-{ratio[1]:g} "
                               f"(box)", "catalogue_keys": len(keys),
                   "slots": len(eng.slots), "pool_device_bytes": eng.device_bytes, "setup_s": t_setup,
                   "admission": (f"elastic within {int(elastic_bytes)} bytes: {srv.slots_added} slots made, "
                                 f"{srv.slots_evicted} evicted") if elastic else "fixed slot pools",
                   "limiter_on_explosions": bool(limiter)},
    }
    eng.close()
    ser.close()
    return out


def serve(args):
    """``--serve``: the serving run alone (see run_serving) with the command-line settings."""
    import torch
    torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
    print(json.dumps(run_serving(args.serve_requests, args.serve_rate, args.serve_steps,
                                 limiter=args.serve_limiter, slots_per_key=args.serve_slots,
                                 elastic_bytes=args.serve_elastic)), flush=True)


def convergence(args):
    """Accuracy of both forms on the density wave (periodic unit cube, Euler, CFL 0.3).

    For N = 2, 3 and jittered-Voronoi meshes of 8^3 and 16^3 cells (and 32^3 for the FP32
    form), integrate to t = 0.1 with equal steps (the CFL step of the initial state at the
    stable CFL of STABLE_CFL, shortened to land on t = 0.1) and report the error in rho against the exact solution
    rho(x - (1,1,1) t): a volume-weighted nodal L2 norm, sqrt(sum_i |P_i| mean_{n in P_i} e_n^2),
    and the max norm; the observed order between consecutive meshes (h ~ 1/n); and the
    relative L2 difference between the FP32 and FP64 forms.
    """
    import numpy as np
    import torch

    from inputs import states
    from inputs.voronoi import periodic_voronoi
    from paper_2605_00619_gb300 import afe

    torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
    afe.lib()
    t_end = 0.1
    rows = []
    meshes = {n: periodic_voronoi(n) for n in (8, 16, 32)}
    for N in (2, 3):
        for n, pm in meshes.items():
            sub = pm.subtet_coords()
            d = sub[:, 1:] - sub[:, :1]
            vol_t = np.abs(np.linalg.det(d)) / 6.0
            cell_of = np.repeat(np.arange(pm.n_cells), np.diff(pm.cell_subtet_ptr))
            vol = np.bincount(cell_of, weights=vol_t, minlength=pm.n_cells)
            finals = {}
            for prec in (afe.AFE_FP32, afe.AFE_FP64):
                if n == 32 and (prec == afe.AFE_FP64 or N > 1):
                    continue  # the FP64 form at 32^3 takes seconds per step
                fp32 = prec == afe.AFE_FP32
                p = afe.afe_default_params(N, precision=prec, picard_tol=1e-6 if fp32 else 1e-12,
                                           picard_max=128 if fp32 else 64, cfl=STABLE_CFL[N])
                h = afe.create_from_polymesh(pm, p)
                x = afe.afe_get_node_coords(h)
                ptr = afe.afe_node_ptr(h, pm.n_cells)
                afe.afe_set_state(h, states.density_wave(x))
                dt0 = afe.afe_compute_dt(h)
                nsteps = int(math.ceil(t_end / dt0 - 1e-9))
                dt = t_end / nsteps
                torch.cuda.synchronize()
                t0 = time.perf_counter()
                afe.afe_step_async(h, dt, nsteps)
                st = afe.afe_sync(h, check=False)
                wall = time.perf_counter() - t0
                q = afe.afe_get_state(h)
                afe.afe_mesh_destroy(h)
                rho_ex = states.density_wave(x, t=t_end)[:, 0]
                e2 = (q[:, 0] - rho_ex) ** 2
                cnt = np.diff(ptr)
                per_cell = np.add.reduceat(e2, ptr[:-1]) / cnt
                l2 = float(np.sqrt(np.sum(vol * per_cell)))
                finals[prec] = q
                rows.append({"N": N, "n": n, "precision": "fp32" if fp32 else "fp64", "cfl": STABLE_CFL[N],
                             "steps": nsteps, "dt": dt,
                             "l2_rho": l2, "linf_rho": float(np.sqrt(e2.max())), "status": int(st),
                             "ms_per_step": 1e3 * wall / nsteps, "dofs": int(5 * len(x))})
            if len(finals) == 2:
                a, b = finals[afe.AFE_FP32][:, 0], finals[afe.AFE_FP64][:, 0]
                rows[-2]["rel_l2_fp32_vs_fp64"] = float(np.linalg.norm(a - b) / np.linalg.norm(b))
    orders = {}
    for N in (2, 3):
        for prec in ("fp32", "fp64"):
            rs = [r for r in rows if r["N"] == N and r["precision"] == prec]
            orders[f"N{N}_{prec}"] = [math.log(r0["l2_rho"] / r1["l2_rho"]) / math.log(r1["n"] / r0["n"])
                                      for r0, r1 in zip(rs, rs[1:])]
    print(json.dumps({"study": "convergence", "workload": "density wave to t=0.1, periodic unit cube, "
                                                         "CFL 0.2 (N=2) / 0.15 (N=3)",
                      "rows": rows, "observed_order": orders}), flush=True)


def vortex(args):
    """Space and space-time accuracy on the isentropic vortex (Sec. 5.1): its steady form and
    its travelling form (background velocity (1, 1, 0)) on the periodic box [0, 10)^3, to
    t = 1 with equal steps at the stable CFL, FP32 form, N = 1, 2, 3 on jittered-Voronoi
    meshes of 8^3, 16^3 and 32^3 cells.  Reported per run (one JSON line each, then a
    summary line with the observed orders between consecutive meshes): the L1 and L2 errors
    in rho against the exact solution (the initial state, shifted by (1, 1, 0) t for the
    travelling form), volume-weighted nodal norms as in the convergence study.
    """
    import numpy as np
    import torch

    from inputs import states
    from inputs.voronoi import periodic_voronoi
    from paper_2605_00619_gb300 import afe

    torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
    afe.lib()
    t_end, L = 1.0, 10.0
    rows = []
    for n in (8, 16, 32):
        pm = periodic_voronoi(n, L=L)
        sub = pm.subtet_coords()
        vol_t = np.abs(np.linalg.det(sub[:, 1:] - sub[:, :1])) / 6.0
        cell_of = np.repeat(np.arange(pm.n_cells), np.diff(pm.cell_subtet_ptr))
        vol = np.bincount(cell_of, weights=vol_t, minlength=pm.n_cells)
        for flow, vel in (("steady", (0.0, 0.0, 0.0)), ("travelling", (1.0, 1.0, 0.0))):
            for N in (1, 2, 3):
                p = afe.afe_default_params(N, precision=afe.AFE_FP32, picard_tol=1e-6, picard_max=128,
                                           cfl=STABLE_CFL[N])
                h = afe.create_from_polymesh(pm, p)
                x = afe.afe_get_node_coords(h)
                ptr = afe.afe_node_ptr(h, pm.n_cells)
                afe.afe_set_state(h, states.isentropic_vortex(x, vel=vel, period=L))
                nsteps = int(math.ceil(t_end / afe.afe_compute_dt(h) - 1e-9))
                torch.cuda.synchronize()
                t0 = time.perf_counter()
                afe.afe_step_async(h, t_end / nsteps, nsteps)
                st = afe.afe_sync(h, check=False)
                wall = time.perf_counter() - t0
                q = afe.afe_get_state(h)
                afe.afe_mesh_destroy(h)
                e = np.abs(q[:, 0] - states.isentropic_vortex(x, t=t_end, vel=vel, period=L)[:, 0])
                cnt = np.diff(ptr)
                l1 = float(np.sum(vol * np.add.reduceat(e, ptr[:-1]) / cnt))
                l2 = float(np.sqrt(np.sum(vol * np.add.reduceat(e * e, ptr[:-1]) / cnt)))
                rows.append({"flow": flow, "n": n, "N": N, "steps": nsteps, "l1_rho": l1, "l2_rho": l2,
                             "status": int(st), "ms_per_step": 1e3 * wall / nsteps})
                print(json.dumps({"study": "vortex", "row": rows[-1]}), flush=True)
    orders = {}
    for flow in ("steady", "travelling"):
        for N in (1, 2, 3):
            rs = [r for r in rows if r["flow"] == flow and r["N"] == N]
            orders[f"{flow}_N{N}"] = [math.log(r0["l2_rho"] / r1["l2_rho"]) / math.log(r1["n"] / r0["n"])
                                      for r0, r1 in zip(rs, rs[1:])]
    print(json.dumps({"study": "vortex", "workload": "isentropic vortex, eps 5, periodic [0,10)^3, to t = 1, FP32",
                      "rows": rows, "observed_order_l2": orders}), flush=True)


def shock_study(args):
    """The spherical explosion (Sec. 5.4) against its one-dimensional radial reference.

    The ``--workload shock`` problem (box [-1,1]^3, transmissive, limiter on, erf-smoothed
    over 1.5 lattice spacings, viscous time step from the sub-tet length unless
    ``--visc-dt cell``) on the ``--n``^3 mesh at order ``--order``, FP32 form, integrated with
    CFL steps to t = 0.25 (the last step shortened).  The reference is the radial MUSCL
    solution of ``inputs.radial`` from the same smoothed data on 15,000 cells of
    r in [0, 1.75].  Reported: volume-weighted nodal L1 errors of rho, |u| and p over the
    nodes with r < 0.95 (the transmissive faces of the box are at distance 1), and the
    radius where the shell-averaged density falls across the shock, against the reference's.
    """
    import numpy as np
    import torch

    from inputs import radial, states
    from inputs.voronoi import box_voronoi
    from paper_2605_00619_gb300 import afe

    torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
    afe.lib()
    t_end, N, n = 0.25, args.order, args.n
    alpha0 = 1.5 * 2.0 / n
    pm = box_voronoi(n)
    sub = pm.subtet_coords()
    vol_t = np.abs(np.linalg.det(sub[:, 1:] - sub[:, :1])) / 6.0
    cell_of = np.repeat(np.arange(pm.n_cells), np.diff(pm.cell_subtet_ptr))
    vol = np.bincount(cell_of, weights=vol_t, minlength=pm.n_cells)
    p = afe.afe_default_params(N, precision=afe.AFE_FP32, picard_tol=1e-6, picard_max=128, cfl=STABLE_CFL[N],
                               limiter=1, visc_dt_subtet=int(args.visc_dt == "subtet"))
    h = afe.create_from_polymesh(pm, p)
    x = afe.afe_get_node_coords(h)
    ptr = afe.afe_node_ptr(h, pm.n_cells)
    afe.afe_set_state(h, states.spherical_riemann(x, alpha0=alpha0))
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    status, steps = 0, 0
    while True:
        s = afe.afe_get_stats(h)
        rem = t_end - s.t
        if rem <= 1e-12 * t_end:
            break
        if steps == 0 or rem > 25.0 * s.dt:
            k, dt = 20, 0.0
        elif rem > s.dt:
            k, dt = 1, 0.0
        else:
            k, dt = 1, rem
        afe.afe_step_async(h, dt, k)
        st = afe.afe_sync(h, check=False)
        steps += k
        if st not in (0, afe.AFE_ENOCONV):
            status = st
            break
        status = status or st
    wall = time.perf_counter() - t0
    q = afe.afe_get_state(h)
    t_reached = afe.afe_get_stats(h).t
    afe.afe_mesh_destroy(h)
    rref, wref = radial.explosion_reference(t_end=t_end, n=15000, R=1.75, alpha0=alpha0)
    cmp = compare_with_radial(x, q, ptr, vol, rref, wref)
    print(json.dumps({"study": "shock", "workload": workload_name(n, N, "shock") + ", to t = 0.25, FP32",
                      "status": int(status), "t": t_reached, "steps": steps, "ms_per_step": 1e3 * wall / max(steps, 1),
                      **cmp, "reference": "radial MUSCL, Rusanov flux, 15000 cells on r in [0, 1.75]"}), flush=True)


def tgv_study(args):
    """The compressible Navier-Stokes Taylor-Green vortex (the fourth configuration of the
    method's evaluation: mu 0.01, Pr 0.71, kappa from Pr, p0 100) on the periodic [0, 2pi)^3
    mesh of ``--n``^3 cells at order ``--order``, FP32 form, CFL steps of ``--cfl`` (default
    the stable CFL) to t = 1, viscous time step from the sub-tet length unless ``--visc-dt
    cell``.  Reported: the status, the time reached, steps, ms per step and the kinetic energy
    (volume-weighted nodal sum of rho |v|^2 / 2) every 0.1 time units; a run that ends
    non-finite reports where.
    """
    import numpy as np
    import torch

    from inputs import states
    from inputs.voronoi import periodic_voronoi
    from paper_2605_00619_gb300 import afe

    torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
    afe.lib()
    t_end, N, n = 1.0, args.order, args.n
    cfl = args.cfl if args.cfl is not None else STABLE_CFL[N]
    pm = periodic_voronoi(n, L=2 * math.pi)
    sub = pm.subtet_coords()
    vol = np.bincount(np.repeat(np.arange(pm.n_cells), np.diff(pm.cell_subtet_ptr)),
                      weights=np.abs(np.linalg.det(sub[:, 1:] - sub[:, :1])) / 6.0, minlength=pm.n_cells)
    p = afe.afe_default_params(N, precision=afe.AFE_FP32, picard_tol=1e-6, picard_max=128, cfl=cfl,
                               equations=afe.AFE_NAVIER_STOKES, mu=0.01, Pr=0.71, kappa=-1.0,
                               visc_dt_subtet=int(args.visc_dt == "subtet"))
    h = afe.create_from_polymesh(pm, p)
    x = afe.afe_get_node_coords(h)
    ptr = afe.afe_node_ptr(h, pm.n_cells)
    wn = np.repeat(vol / np.diff(ptr), np.diff(ptr))

    def kinetic(q):
        return float(np.sum(wn * 0.5 * (q[:, 1] ** 2 + q[:, 2] ** 2 + q[:, 3] ** 2) / q[:, 0]))

    afe.afe_set_state(h, states.taylor_green_3d(x, p0=100.0))
    history = [(0.0, kinetic(afe.afe_get_state(h)))]
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    status, steps, t_mark = 0, 0, 0.1
    while True:
        s = afe.afe_get_stats(h)
        if s.t >= t_end - 1e-12:
            break
        k = 1 if steps == 0 else max(1, min(50, int((t_mark - s.t) / max(s.dt, 1e-30))))
        afe.afe_step_async(h, 0.0, k)
        st = afe.afe_sync(h, check=False)
        steps += k
        if st not in (0, afe.AFE_ENOCONV):
            status = st
            break
        t = afe.afe_get_stats(h).t
        if t >= t_mark - 1e-12:
            history.append((t, kinetic(afe.afe_get_state(h))))
            t_mark += 0.1
    wall = time.perf_counter() - t0
    s = afe.afe_get_stats(h)
    afe.afe_mesh_destroy(h)
    print(json.dumps({"study": "tgv", "workload": workload_name(n, N, "tgv") + ", to t = 1, FP32", "cfl": cfl,
                      "visc_dt": args.visc_dt, "status": int(status), "t": s.t, "steps": steps,
                      "ms_per_step": 1e3 * wall / max(steps, 1), "kinetic_energy": history,
                      "cells": pm.n_cells}), flush=True)


def compare_with_radial(x, q, ptr, vol, rref, wref, r_max=0.95, ambient=0.125, gamma=1.4):
    """Nodal state q [n_nodes, 5] at positions x against a radial profile (rref, wref = rho, u,
    p): volume-weighted nodal L1 errors of rho, |u| and p over the nodes with r < r_max (each
    cell's volume shared equally by its nodes ptr), and the shock radius of both: the
    outermost radius below r_max where the (shell-averaged) density exceeds the ambient value
    by half the reference's jump across its outermost front."""
    import numpy as np

    r = np.linalg.norm(x, axis=1)
    rho = q[:, 0]
    speed = np.linalg.norm(q[:, 1:4], axis=1) / rho
    pres = (gamma - 1.0) * (q[:, 4] - 0.5 * rho * speed ** 2)
    ref = [np.interp(r, rref, wref[:, j]) for j in range(3)]
    cnt = np.diff(ptr)
    w_node = np.repeat(np.asarray(vol) / cnt, cnt) * (r < r_max)
    err = {name: float(np.sum(w_node * np.abs(v - rv)) / np.sum(w_node))
           for name, v, rv in (("rho", rho, ref[0]), ("speed", speed, np.abs(ref[1])), ("p", pres, ref[2]))}
    bins = np.linspace(0.0, r_max, 96)
    idx = np.digitize(r, bins) - 1
    shell = np.array([rho[idx == b].mean() if np.any(idx == b) else np.nan for b in range(len(bins) - 1)])
    mid = 0.5 * (bins[1:] + bins[:-1])
    inside = rref < r_max
    front = rref[np.nonzero(inside & (np.abs(wref[:, 0] - ambient) > 1e-3 * ambient))[0].max()]
    behind = inside & (rref > front - 0.05)
    jump = ambient + 0.5 * (wref[behind, 0].max() - ambient)
    hit = np.nonzero(shell > jump)[0]
    r_sh = float(mid[hit.max()]) if len(hit) else None
    r_sh_ref = float(rref[np.nonzero((wref[:, 0] > jump) & inside)[0].max()])
    return {"l1_vs_radial_reference": err, "shock_radius": r_sh, "shock_radius_reference": r_sh_ref}


def stokes(args):
    """Viscous check: periodic form of the first problem of Stokes (two shear layers, nu = mu =
    1e-3 with rho = 1, p = 1/gamma, Navier-Stokes, kappa from Pr 0.71), integrated to t = 0.25
    on periodic meshes of 8^3 and 16^3 cells (N = 1, 2; FP32 and FP64 forms) and 32^3 cells
    (N = 1, FP32) at the stable CFL, with the viscous term of the time step bounded by the
    smallest sub-tet length (with the cell length, as printed, these runs go non-finite
    within 20 steps).  One JSON line per run, then a summary line.
    Reported: the volume-weighted nodal L2 error of the shear velocity v against the closed
    form v = erf profiles of width 2 sqrt(nu (t + 0.05)), and the status.
    """
    import numpy as np
    import torch

    from inputs import states
    from inputs.voronoi import periodic_voronoi
    from paper_2605_00619_gb300 import afe

    torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
    afe.lib()
    nu, t_end = 1e-3, 0.25
    rows = []
    for n in (8, 16, 32):
        pm = periodic_voronoi(n)
        sub = pm.subtet_coords()
        vol_t = np.abs(np.linalg.det(sub[:, 1:] - sub[:, :1])) / 6.0
        cell_of = np.repeat(np.arange(pm.n_cells), np.diff(pm.cell_subtet_ptr))
        vol = np.bincount(cell_of, weights=vol_t, minlength=pm.n_cells)
        for N in (1, 2):
            for prec in (afe.AFE_FP32, afe.AFE_FP64):
                if n == 32 and (prec == afe.AFE_FP64 or N > 1):
                    continue
                fp32 = prec == afe.AFE_FP32
                p = afe.afe_default_params(N, precision=prec, picard_tol=1e-6 if fp32 else 1e-12,
                                           picard_max=128 if fp32 else 64, cfl=STABLE_CFL[N],
                                           equations=afe.AFE_NAVIER_STOKES, mu=nu, Pr=0.71, kappa=-1.0,
                                           visc_dt_subtet=1)
                h = afe.create_from_polymesh(pm, p)
                x = afe.afe_get_node_coords(h)
                ptr = afe.afe_node_ptr(h, pm.n_cells)
                afe.afe_set_state(h, states.shear_layers(x, nu))
                dt0 = afe.afe_compute_dt(h)
                nsteps = int(math.ceil(t_end / dt0 - 1e-9))
                dt = t_end / nsteps
                t0 = time.perf_counter()
                afe.afe_step_async(h, dt, nsteps)
                st = afe.afe_sync(h, check=False)
                wall = time.perf_counter() - t0
                q = afe.afe_get_state(h)
                afe.afe_mesh_destroy(h)
                v = q[:, 2] / q[:, 0]
                v_ex = states.shear_layers(x, nu, t=t_end)[:, 2]
                e2 = (v - v_ex) ** 2
                per_cell = np.add.reduceat(e2, ptr[:-1]) / np.diff(ptr)
                rows.append({"n": n, "N": N, "precision": "fp32" if fp32 else "fp64", "steps": nsteps, "dt": dt,
                             "l2_v": float(np.sqrt(np.sum(vol * per_cell))), "linf_v": float(np.sqrt(e2.max())),
                             "status": int(st), "ms_per_step": 1e3 * wall / nsteps})
                print(json.dumps({"study": "stokes", "row": rows[-1]}), flush=True)
    print(json.dumps({"study": "stokes", "workload": "two periodic shear layers, nu = 1e-3, to t = 0.25, "
                                                     "viscous time step from the smallest sub-tet length",
                      "rows": rows}), flush=True)


def main():
    args = _args()
    if args.study == "convergence":
        convergence(args)
        return
    if args.study == "stokes":
        stokes(args)
        return
    if args.study == "vortex":
        vortex(args)
        return
    if args.study == "shock":
        shock_study(args)
        return
    if args.study == "tgv":
        tgv_study(args)
        return
    if args.serve:
        serve(args)
        return
    if args.impl == "reference":
        reference_arm(args)
    else:
        ours(args)


if __name__ == "__main__":
    main()
