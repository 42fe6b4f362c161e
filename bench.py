"""Throughput of the GB300 ADER-AFE-DG step: DOF-updates/s on the density-wave workload.

Workload (one GPU): the smooth density wave rho = 1 + 0.2 sin(2 pi (x+y+z)), u = (1,1,1),
p = 1 on the periodic unit cube, jittered-lattice Voronoi mesh with 32^3 cells and fan
subgrids, AFE degree N = 3, CFL 0.3, Euler.  A DOF-update is one conserved variable at one
AFE node advanced by one full ADER step (limiter check, time step, predictor, face fluxes,
corrector).  ``value`` is the reduced-precision form (FP32 arithmetic, FP64 master state,
FP64 time step and conservative cell totals); the plain FP64 form is timed beside it.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
  python bench.py --serve      (continuous-batching serving run; see serve())

N > 1 (torchrun): every rank runs an independent simulation (mesh seed = rank); there is
no data-path collective and ``value`` is the sum over ranks of DOF-updates over the max
over ranks of the timed wall.  ``--impl reference`` times the CPU oracle (the plain FP64
restatement of the paper's scheme) on a bounded sample of the same workload.
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "DOF-updates/s per ADER-DG step"
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
    ap.add_argument("--serve", action="store_true", help="serving run: Poisson requests on small meshes")
    ap.add_argument("--serve-requests", type=int, default=300)
    ap.add_argument("--serve-rate", type=float, default=200.0, help="offered load, requests per second")
    ap.add_argument("--serve-slots", type=int, default=16, help="slots per catalogue mesh")
    return ap.parse_args()


def workload_name(n, N):
    return f"density-wave periodic unit cube, {n}^3 jittered-Voronoi cells (fan subgrid), AFE N={N}, Euler, CFL 0.3"


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
prm = scheme.Params(cfl=0.3)
uc = m.split(states.density_wave(m.node_coords()))
dt = scheme.cfl_dt(m, uc, [0.0] * m.n_cells, prm) * {dt_scale}
out = []
for s in range({steps}):
    t0 = time.perf_counter()
    uc, info = scheme.step(m, uc, prm, dt=dt)
    out.append(time.perf_counter() - t0)
print(json.dumps(dict(times=out, dofs=5 * m.n_nodes, cells=m.n_cells, iters=float(info.iterations.mean()))))
"""


def run_oracle(n_sample, N, steps, dt_scale):
    """Run the oracle in a fresh single-threaded process; returns its JSON record."""
    env = dict(os.environ, OMP_NUM_THREADS="1", OPENBLAS_NUM_THREADS="1", MKL_NUM_THREADS="1")
    code = _ORACLE_SNIPPET.format(root=ROOT, n=n_sample, N=N, steps=steps, dt_scale=dt_scale)
    r = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, env=env)
    if r.returncode != 0:
        raise RuntimeError("oracle run failed: " + r.stderr[-2000:])
    return json.loads(r.stdout.strip().splitlines()[-1])


def oracle_sample(N, steps):
    """A bounded sample of the workload for the oracle: full steps of the same generator,
    order and CFL on the 6^3 periodic mesh."""
    n_s = 6
    return n_s, run_oracle(n_s, N, steps, dt_scale=1.0)


def reference_arm(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    n_s = 6
    rec = run_oracle(n_s, args.order, args.warmup + args.steps, 1.0)
    times = rec["times"][args.warmup:]
    t = sum(times)
    value = rec["dofs"] * len(times) / t
    sample = (f"oracle (numpy FP64, 1 thread) full steps on the {n_s}^3 periodic mesh of the same generator, "
              f"N={args.order}, CFL 0.3 ({rec['cells']} cells, {rec['dofs']} DOFs per step)")
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
    """Algorithmic flops and bytes of one predictor launch (the dominant kernel).

    Per cell and fixed-point iteration, with Np = (N+1)(N+2)(N+3)/6, Nt = N+1, S sub-tets,
    N_i nodes: flux + 3x3 pre-contraction 150 flop per (sub-tet, time, node); the reference
    stiffness contraction 2*3*Np flop per (sub-tet, time, node, variable); the agglomeration
    1 flop per incidence and variable; the inverse-mass apply 2 N_i^2 (5 Nt); the update
    2 Nt per (node, time, variable).  Epilogue: one more flux pass and the volume term.
    Bytes: the dense M_i^-1 is read once per iteration (it does not stay on chip), plus the
    state, the sub-tet geometry and the outputs once.
    """
    import numpy as np
    Np = (N + 1) * (N + 2) * (N + 3) // 6
    Nt = N + 1
    Ni = np.diff(node_ptr).astype(np.float64)
    S = np.diff(sub_ptr).astype(np.float64)
    it = iters.astype(np.float64)
    per_it = S * Nt * Np * (150 + 5 * 6 * Np + 5) + 2 * Ni * Ni * 5 * Nt + Ni * Nt * 5 * 2 * Nt
    epi = S * Np * Nt * 150 + S * Np * 5 * 6 * Np + S * Np * 5
    flops = float(np.sum(it * per_it + epi))
    bytes_ = float(np.sum(it * Ni * Ni * real_bytes + Ni * 5 * 8 + S * (10 * 8 + Np * 2) + Ni * 5 * real_bytes))
    return flops, bytes_


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

    def max_over_ranks(x):
        if dist is None:
            return x
        t = torch.tensor([x], dtype=torch.float64, device="cuda")
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        return float(t.item())

    def sum_over_ranks(x):
        if dist is None:
            return x
        t = torch.tensor([x], dtype=torch.float64, device="cuda")
        dist.all_reduce(t, op=dist.ReduceOp.SUM)
        return float(t.item())

    pm = periodic_voronoi(args.n, seed=rank)
    stream = torch.cuda.Stream()
    sid = stream.cuda_stream
    peaks = {}
    try:
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except (OSError, ValueError):
        pass

    def run_form(prec, steps, warmup, e2e):
        fp32 = prec == afe.AFE_FP32
        p = afe.afe_default_params(args.order, precision=prec, picard_tol=1e-6 if fp32 else 1e-12,
                                   picard_max=128 if fp32 else 64)
        h = afe.create_from_polymesh(pm, p, stream=sid)
        n_nodes = afe.afe_num_nodes(h)
        node_ptr = afe.afe_node_ptr(h, pm.n_cells)
        x = afe.afe_get_node_coords(h)
        u0 = states.density_wave(x)
        afe.afe_set_state(h, u0)
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
                   nonconverged=int(stats.nonconverged), dt=stats.dt, bytes=afe.afe_device_bytes(h))
        rec["flops"], rec["abytes"] = predictor_model(node_ptr, pm.cell_subtet_ptr, iters, args.order,
                                                      4 if prec == afe.AFE_FP32 else 8)
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
                hin[:] = afe.afe_get_state(h)
            barrier()
            rec["e2e_wall"] = time.perf_counter() - t1
        afe.afe_mesh_destroy(h)
        return rec

    r32 = run_form(afe.AFE_FP32, args.steps, args.warmup, not args.no_e2e)
    r64 = run_form(afe.AFE_FP64, args.fp64_steps, 1, False) if args.fp64_steps > 0 else None

    K = args.steps
    dofs = 5 * r32["n_nodes"]
    ms_max = max_over_ranks(r32["ms"])
    total_dofs = sum_over_ranks(dofs * K)
    value = total_dofs / (ms_max / 1e3)
    out = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": K, "warmup": args.warmup,
        "ms_per_step": ms_max / K, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f32", "data": "synthetic",
        "config": {"workload": workload_name(args.n, args.order), "cells": pm.n_cells, "nodes": r32["n_nodes"],
                   "dofs": dofs, "precision": "FP32 arithmetic, FP64 master state / dt / cell totals",
                   "picard_tol": 1e-6, "l2": "inputs larger than L2 (M_i^-1 alone is "
                   f"{r32['bytes'] / 1e9:.1f} GB of device state)", "parallelism": f"{world} independent replicas"},
        "clocks": r32["clocks"],
        "gpu_launches": int(r32["launches"]),
        "status": {"fp32": r32["status"], "picard_iters_mean": r32["iters_mean"], "picard_iters_max": r32["iters_max"],
                   "nonconverged_cells": r32["nonconverged"]},
        "stage_ms_per_step": dict(zip(["limiter_dt", "predictor", "face", "corrector"], r32["stage_ms"])),
    }
    if "e2e_wall" in r32:
        e2e_wall = max_over_ranks(r32["e2e_wall"])
        out["e2e"] = {"value": total_dofs / e2e_wall, "unit": UNIT, "h2d_bytes_per_step": r32["n_nodes"] * 5 * 8,
                      "d2h_bytes_per_step": r32["n_nodes"] * 5 * 8}
    # roofline of the dominant kernel (the predictor), FP32 CUDA-core arithmetic vs HBM
    pred_ms = r32["stage_ms"][1]
    sm_max = (peaks.get("sm_max_mhz") or 2070.0)
    fp32_peak = 152 * 128 * 2 * sm_max * 1e6 / 1e12          # TFLOP/s, FMA units x clock
    hbm = peaks.get("hbm_gbs") or 6800.0
    t_alu = r32["flops"] / (fp32_peak * 1e12)
    t_hbm = r32["abytes"] / (hbm * 1e9)
    if t_alu >= t_hbm:
        ach = r32["flops"] / (pred_ms / 1e3) / 1e12
        out["roofline"] = {"bound": "alu", "achieved": ach, "peak": fp32_peak, "unit": "TFLOP/s",
                           "frac": ach / fp32_peak, "traffic": None,
                           "kernel": f"predictor_f32_kernel<{args.order}>",
                           "peak_note": "FP32 FMA: 152 SMs x 128 lanes x 2 flop x max SM clock (derived)"}
    else:
        ach = r32["abytes"] / (pred_ms / 1e3) / 1e9
        out["roofline"] = {"bound": "hbm", "achieved": ach, "peak": hbm, "unit": "GB/s", "frac": ach / hbm,
                           "traffic": None, "kernel": f"predictor_f32_kernel<{args.order}>", "peak_note": "of measured"}
    out["roofline"]["algorithmic_flops"] = r32["flops"]
    out["roofline"]["algorithmic_bytes"] = r32["abytes"]
    if r64 is not None:
        ms64 = max_over_ranks(r64["ms"])
        out["fp64_plain"] = {"value": sum_over_ranks(5 * r64["n_nodes"] * args.fp64_steps) / (ms64 / 1e3),
                             "unit": UNIT, "ms_per_step": ms64 / args.fp64_steps, "status": r64["status"],
                             "picard_iters_mean": r64["iters_mean"],
                             "stage_ms_per_step": dict(zip(["limiter_dt", "predictor", "face", "corrector"],
                                                           r64["stage_ms"]))}
        out["fp32_over_fp64"] = value / out["fp64_plain"]["value"]
    if rank == 0 and not args.no_cpu_baseline:
        try:
            n_s, rec = oracle_sample(args.order, 1)
            cb = rec["dofs"] / rec["times"][0]
            out["cpu_baseline"] = {"value": cb, "unit": UNIT, "cores": 1, "kind": "oracle",
                                   "sample": f"one oracle step (numpy FP64, 1 thread) on the {n_s}^3 periodic mesh of "
                                             f"the same generator, N={args.order} ({rec['cells']} cells, "
                                             f"{rec['dofs']} DOFs, {rec['iters']:.1f} mean fixed-point "
                                             f"iterations)"}
        except Exception as e:  # the baseline never hides the GPU number
            out["cpu_baseline"] = {"value": None, "unit": UNIT, "cores": 1, "kind": "oracle", "sample": str(e)[:200]}
    if rank == 0:
        print(json.dumps(out), flush=True)
    if dist is not None:
        dist.destroy_process_group()


def serve(args):
    """Continuous batching of many small simulations (one GPU).

    Catalogue: periodic jittered-Voronoi meshes with 4^3, 5^3 and 6^3 cells, AFE N (default
    3), FP32 form, Euler, CFL 0.3, density-wave initial data; ``--serve-slots`` resident
    handles per mesh.  Requests arrive as a Poisson process of ``--serve-rate`` per second,
    each for a mesh drawn uniformly and 5, 10 or 20 CFL steps.  The batched server (all
    occupied slots advanced together, one launch per stage, CUDA graph per batch) is timed
    against the serial server (one request at a time, alone) on the same requests.  Reported:
    DOF-updates/s over the run, p50/p99 request latency (arrival to completion).
    """
    import torch

    from inputs import states
    from inputs.voronoi import periodic_voronoi
    from paper_2605_00619_gb300 import afe
    from paper_2605_00619_gb300.serving import GpuEngine, Server, poisson_requests

    torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
    afe.lib()
    cat = {f"{n}^3": periodic_voronoi(n, seed=10 + n) for n in (4, 5, 6)}
    p = afe.afe_default_params(args.order, precision=afe.AFE_FP32, picard_tol=1e-6, picard_max=128)
    stream = torch.cuda.Stream()
    eng = GpuEngine(cat, {k: args.serve_slots for k in cat}, p, stream=stream.cuda_stream)
    for sl in eng.slots:
        if sl.mesh not in eng.default_state:
            eng.default_state[sl.mesh] = states.density_wave(afe.afe_get_node_coords(sl.handle))
    keys = sorted(cat)
    warm = poisson_requests(0.0, 2 * len(eng.slots), keys, [3], seed=99)
    Server(eng).run(warm)
    Server(eng, mode="serial").run(warm[:len(keys)])
    reqs = lambda: poisson_requests(args.serve_rate, args.serve_requests, keys, [5, 10, 20], seed=1)  # noqa: E731
    clocks = ClockSampler(torch.cuda.current_device())
    clocks.start()
    sb = Server(eng, max_chunk=4).run(reqs())
    clk = clocks.stop()
    ss = Server(eng, mode="serial").run(reqs())
    nodes = {k: next(s.n_nodes for s in eng.slots if s.mesh == k) for k in keys}
    out = {
        "metric": "serving throughput, continuous batching", "value": sb.throughput, "unit": UNIT,
        "higher_is_better": True, "n_gpus": 1, "dtype": "f32", "data": "synthetic",
        "p50_ms": 1e3 * sb.p50_s, "p99_ms": 1e3 * sb.p99_s, "mean_ms": 1e3 * sb.mean_s,
        "mean_batch_members": sb.mean_batch, "batch_steps": sb.steps_launched, "failed": sb.failed,
        "makespan_s": sb.makespan_s,
        "serial": {"value": ss.throughput, "unit": UNIT, "p50_ms": 1e3 * ss.p50_s, "p99_ms": 1e3 * ss.p99_s,
                   "makespan_s": ss.makespan_s, "failed": ss.failed},
        "batched_over_serial": sb.throughput / ss.throughput,
        "clocks": clk,
        "config": {"workload": f"Poisson arrivals at {args.serve_rate:g}/s, {args.serve_requests} requests of 5/10/20 "
                               f"CFL steps on periodic Voronoi meshes {', '.join(keys)} (nodes "
                               f"{', '.join(str(nodes[k]) for k in keys)}), AFE N={args.order}, FP32 form, Euler",
                   "slots": len(eng.slots), "pool_device_bytes": eng.device_bytes},
    }
    eng.close()
    print(json.dumps(out), flush=True)


def main():
    args = _args()
    if args.serve:
        serve(args)
        return
    if args.impl == "reference":
        reference_arm(args)
    else:
        ours(args)


if __name__ == "__main__":
    main()
