#!/usr/bin/env python
"""Benchmark of the GB300 MLS-MPM sand substep and its adjoint.

Metric: particle-substeps per second, forward + backward, on 1,048,576
particles (8 per cell, 64 x 32 x 64-cell bed) on a 128^3 grid with the
digging skill driving a box shovel (E 3e5, nu 0.25, rho 1800, phi 35 deg,
dt 5e-5). One step = restore the rollout start state (shovel inserting),
a recorded forward of S substeps with checkpoints every K, the MSE loss
against a target cloud and the checkpointed backward to
dL/d{E, nu, rho, phi, theta}. ``value`` counts N * S particle-substeps per
step. The forward-only rate is reported beside it.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Under torchrun (N > 1) every rank runs an independent replica of the
workload (the instances shard with no data exchange): weak scaling.
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

# the timed workload (both arms)
WORKLOAD = "bed1m_grid128: 1,048,576 particles, 128^3 grid, skill-driven box shovel"

# Algorithmic bytes per particle and launch: what the method must read and
# write with FP32 state (96 B per particle for x, v, C, F; the same for their
# adjoints), plus the grid at 8 particles per cell with a 1.3x halo (about
# 9 B per particle for a grid pass). A forward substep moves about 200 B per
# particle (state read and written once, 192 B, and the grid); a backward
# substep about 306 B (state k read, adjoint of k+1 read, adjoint of k
# written: 288 B, and two grid-adjoint passes). The recorded SVD of the trial
# F (written by a recorded forward, read by the adjoint) and the fused
# kernels' savings (adjoints kept in registers between two substeps) are
# implementation choices: they show in the measured DRAM traffic, not here.
FWD_BYTES = 200          # per particle-substep, forward
BWD_BYTES = 306          # per particle-substep, backward
ALGO_BYTES = {
    "k_p2g": 96 + 36,           # read x, v, C, F; write F
    "k_g2p": 12 + 60,           # read x; write x, v, C
    "k_g2p_bwd": 12 + 60 + 12,  # read x, adj x/v/C; write adj x
    "k_p2g_bwd": 96 + 48 + 96,  # read state and adj x/F; write adj x/v/C/F
    # one launch reverses one substep's worth (the P2G adjoint of substep k
    # and the G2P adjoint of k-1): the backward's bytes per particle-substep
    "k_p2g_g2p_bwd": BWD_BYTES,
}


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--substeps", type=int, default=100)
    ap.add_argument("--checkpoint", type=int, default=0,
                    help="checkpoint interval K (0: mpm.checkpoint_interval for the free HBM)")
    ap.add_argument("--start", type=int, default=600, help="substep of the rollout start state")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--tile", type=int, default=0, help="shared-memory tile scatter (1) or global atomics (0)")
    ap.add_argument("--sort", type=int, default=0, help="sort particles by cell every n substeps (0: never)")
    ap.add_argument("--tune-substeps", type=int, default=20,
                    help="trial substeps of mpm_autotune before timing (0: keep the default launch shape)")
    ap.add_argument("--batch", type=int, default=64, help="instances of the batched-vs-serial leg (0: skip)")
    ap.add_argument("--sysid", type=int, default=8,
                    help="candidates of the system-identification leg (0: skip; 32 x 1500 substeps takes minutes)")
    ap.add_argument("--sysid-substeps", type=int, default=300)
    ap.add_argument("--sysid-iters", type=int, default=30)
    ap.add_argument("--full-substeps", type=int, default=2000,
                    help="substeps of the whole-rollout leg (0: skip); the 1M bed's rollout is 2,000")
    ap.add_argument("--full-steps", type=int, default=2)
    ap.add_argument("--rollout-250k", type=int, default=1,
                    help="the 250k-particle differentiable rollout leg, 1,000 substeps (0: skip)")
    ap.add_argument("--batch-substeps", type=int, default=500, help="substeps of each fwd+bwd loop of the batched leg (the uneven-batch workload runs 500)")
    return ap.parse_args()


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def max_over_ranks(dist, values, device):
    """Each value's maximum over the ranks (the slowest rank sets the job's
    time); the values themselves with no process group."""
    import torch
    t = torch.tensor([float(v) for v in values], dtype=torch.float64, device=device)
    if dist is not None:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return [float(x) for x in t]


def job_rate(world_size: int, units_per_rank: float, seconds: float) -> float:
    """Whole-job throughput: the units all ranks processed (each rank runs
    its own replica) over the slowest rank's time."""
    return world_size * units_per_rank / seconds


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


# --------------------------------------------------------------------------
# clocks during the timed region
# --------------------------------------------------------------------------
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, bus_id):
        self.bus_id = bus_id
        self.proc = None
        self.lines = []

    def start(self):
        cmd = ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits", "-lms", "200"]
        if self.bus_id:
            cmd += ["-i", self.bus_id]
        try:
            self.proc = subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
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
        self.t.join(timeout=2)
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax.append(float(f[2]))
            except ValueError:
                continue
            for nm, val in zip(names, f[5:9]):
                if val.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# --------------------------------------------------------------------------
# CPU baseline: the FP64 oracle, as it stands, on a bounded sample
# --------------------------------------------------------------------------
def host_cores() -> int:
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


def oracle_sample(w, cells: int, nsub: int, start_substep: int, threads: int = 1):
    """fwd+bwd of the oracle on the particles of a cells^3 block of the bed,
    on the workload's own grid, with `threads` OpenMP threads (1: its plain
    serial loops); returns (particle-substeps/s, seconds, description)."""
    import numpy as np

    import oracle
    oracle.set_threads(threads)

    x0 = w.x0.astype(np.float64)
    lo = x0.min(0)
    sel = np.all((x0 - lo) < cells * w.dx, axis=1)
    x = x0[sel]
    n = x.shape[0]
    p = oracle.Params(res=tuple(w.res), dx=w.dx, dt=w.dt, gravity=tuple(w.gravity), bound=w.bound, E=w.E, nu=w.nu,
                      rho=w.rho, phi_deg=w.phi_deg, vol=w.vol, friction=w.friction, shovel_half=tuple(w.shovel_half))
    acts, T, _ = oracle.skill_actions(w.traj.theta, w.traj.v_lin, w.traj.v_ang, w.traj.substeps_per_action * w.dt)
    poses = oracle.pose_table(w.traj.start_pose, acts, w.traj.substeps_per_action, w.dt,
                              start_substep + nsub)[start_substep:]
    v, C, F = np.zeros((n, 3)), np.zeros((n, 9)), np.tile(np.eye(3).ravel(), (n, 1))
    gx = np.full((n, 3), 1.0 / n)
    t0 = time.perf_counter()
    st, g = oracle.rollout_adjoint(p, x, v, C, F, poses, gx=gx)
    dt = time.perf_counter() - t0
    oracle.set_threads(1)
    desc = (f"oracle fwd+bwd (FP64 C, {threads} thread{'s' if threads > 1 else ''}): {n} particles ({cells}^3-cell "
            f"block of the bed) x {nsub} substeps on the {w.res[0]}^3 grid")
    return n * nsub / dt, dt, desc


def oracle_small_workload(threads: int):
    """fwd+bwd of the oracle over the whole small parity workload (8,000
    particles, 32^3 grid, 200 substeps with the scripted shovel); returns
    (particle-substeps/s, seconds)."""
    import numpy as np

    import oracle
    from paper_2510_17335_gb300 import workloads as W
    w = W.cfg_small()
    oracle.set_threads(threads)
    p = oracle.Params(res=tuple(w.res), dx=w.dx, dt=w.dt, gravity=tuple(w.gravity), bound=w.bound, E=w.E, nu=w.nu,
                      rho=w.rho, phi_deg=w.phi_deg, vol=w.vol, friction=w.friction, shovel_half=tuple(w.shovel_half))
    acts = np.asarray(w.traj.actions, np.float64)
    poses = oracle.pose_table(w.traj.start_pose, acts, w.traj.substeps_per_action, w.dt, w.n_substeps)
    n = w.n
    x = w.x0.astype(np.float64)
    v, C, F = np.zeros((n, 3)), np.zeros((n, 9)), np.tile(np.eye(3).ravel(), (n, 1))
    t0 = time.perf_counter()
    oracle.rollout_adjoint(p, x, v, C, F, poses, gx=np.full((n, 3), 1.0 / n))
    dt = time.perf_counter() - t0
    oracle.set_threads(1)
    return n * w.n_substeps / dt, dt


def run_reference(args):
    ws, rank, _ = dist_env()
    if rank != 0:
        return
    from paper_2510_17335_gb300 import workloads as W
    w = W.cfg_1m()
    cores = host_cores()
    for _ in range(args.warmup):
        oracle_sample(w, 16, 10, args.start, cores)
    rates, secs = [], 0.0
    desc = ""
    for _ in range(args.steps):
        r, s, desc = oracle_sample(w, 16, 10, args.start, cores)
        rates.append(r)
        secs += s
    value = sum(rates) / len(rates)
    line = {"metric": "particle-substeps/s (fwd+bwd)", "value": value, "unit": "particle-substeps/s",
            "impl": "reference", "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * secs / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD, "substeps_per_step": args.substeps, "start_substep": args.start,
                       "sampled": "each step times the oracle on a bounded block of the bed (cpu_baseline.sample)"},
            "cpu_baseline": {"value": value, "unit": "particle-substeps/s", "cores": cores, "kind": "oracle",
                             "sample": desc},
            "e2e": {"value": value, "unit": "particle-substeps/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# --------------------------------------------------------------------------
# batched vs serial: uneven instances in one handle vs one handle each
# --------------------------------------------------------------------------
def batched_vs_serial(n_inst: int, nsub: int, steps: int, sort_every: int):
    import numpy as np
    import torch

    from paper_2510_17335_gb300 import mpm
    from paper_2510_17335_gb300 import workloads as W

    ws = W.batch_uneven(n_inst, n_substeps=nsub)
    n_total = sum(w.n for w in ws)
    # the same checkpoint policy as the main leg, for the whole batch (each
    # instance alone then fits too): both arms use the same interval
    nodes = sum(mpm.blocked_nodes(w.res) for w in ws)
    K = mpm.checkpoint_interval(nsub, n_total, nodes, torch.cuda.mem_get_info()[0])
    opts = mpm.make_options(checkpoint_every=K, sort_every=sort_every)

    def device_io(groups):
        # per handle: the target cloud and the dL/dx buffer, on the device as
        # an identification loop keeps them (made before the timed loops)
        out = []
        for g in groups:
            tgt = torch.from_numpy(np.concatenate([w.x0 for w in g]) + np.float32(0.002)).cuda()
            out.append((tgt, torch.empty_like(tgt)))
        return out

    def run(sims, io):
        for sim, (tgt, dl) in zip(sims, io):
            sim.reset()
            sim.forward(nsub, record=True)
            sim.loss_mse(tgt, grad_out=dl)
            sim.backward(dL_dx=dl)

    def timed(sims, groups):
        io = device_io(groups)
        # warm-up: the first loop allocates, the second captures the CUDA
        # graphs; the timed loops replay them, as an optimisation loop does
        run(sims, io)
        run(sims, io)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(steps):
            run(sims, io)
        torch.cuda.synchronize()
        return (time.perf_counter() - t0) / steps

    sim = mpm.simulation_from_workloads(ws, opts)
    tb = timed([sim], [ws])
    launches_b = sim.info()["kernel_launches"]
    sim.close()
    sims = [mpm.simulation_from_workloads([w], opts) for w in ws]
    ts = timed(sims, [[w] for w in ws])
    for s_ in sims:
        s_.close()
    return {"instances": n_inst, "particles_total": n_total, "particles_min": min(w.n for w in ws),
            "particles_max": max(w.n for w in ws), "grids": f"{min(w.res[0] for w in ws)}^3-{max(w.res[0] for w in ws)}^3",
            "substeps": nsub, "checkpoint_every": K,
            "timing": f"{steps} loops (reset, recorded forward, MSE loss, backward; target and dL/dx on the "
                      "device) after 2 warm-up loops (allocation, CUDA-graph capture), wall clock",
            "batched_particle_substeps_per_s": n_total * nsub / tb,
            "serial_particle_substeps_per_s": n_total * nsub / ts, "speedup": ts / tb,
            "batched_s_per_step": tb, "serial_s_per_step": ts}


# --------------------------------------------------------------------------
# whole recorded rollouts fwd+bwd with checkpoint recomputation
# --------------------------------------------------------------------------
def rollout_leg(w, nsub: int, steps: int, K: int, target, material=None):
    """fwd+bwd of a whole rollout of workload w from its initial state: a
    recorded forward of nsub substeps with checkpoint interval K, the MSE
    loss against target (host, [n, 3]) and the backward, which reverses the
    last segment from the record and recomputes every earlier one from its
    checkpoint. material: the (E, nu, rho, phi) the rollout runs with (None:
    the workload's). Timed with CUDA events on the library's stream after two
    warm-up steps (allocation, CUDA-graph capture)."""
    import numpy as np
    import torch

    from paper_2510_17335_gb300 import mpm

    N = w.n
    slot_state, slot_grid = mpm.record_bytes(N, mpm.blocked_nodes(w.res))
    n_seg = -(-nsub // K)
    record = (K + 1) * slot_state + K * slot_grid + n_seg * slot_state
    last = nsub - (n_seg - 1) * K
    stream = torch.cuda.Stream()
    sim = mpm.simulation_from_workloads([w], mpm.make_options(checkpoint_every=K))
    if material is not None:
        sim.set_material(0, material)
    sim.set_stream(stream.cuda_stream)
    dev = torch.device("cuda", torch.cuda.current_device())
    with torch.cuda.stream(stream):
        tgt = torch.from_numpy(np.ascontiguousarray(target, np.float32)).to(dev)
        dldx = torch.empty((N, 3), device=dev)

        def step():
            sim.reset()
            sim.forward(nsub, record=True)
            sim.loss_mse(tgt, grad_out=dldx)
            return sim.backward(dL_dx=dldx)

        for _ in range(2):
            step()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(steps):
            gm, gt = step()
        e1.record(stream)
        torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / steps
    sim.close()
    peak, peak_kind = measured_peaks()
    gbs = (FWD_BYTES + BWD_BYTES) * N * nsub / (ms / 1e3) / 1e9
    return {"roofline": {"bound": "hbm", "bytes_per_particle_substep": FWD_BYTES + BWD_BYTES,
                         "achieved": round(gbs, 1), "peak": peak, "unit": "GB/s", "frac": round(gbs / peak, 4),
                         "peak_kind": f"{peak_kind} hbm_gbs",
                         "note": "the method's bytes only: the recomputed substeps count as overhead"},
            "substeps": nsub, "checkpoint_every": K, "segments": n_seg, "recomputed_substeps": nsub - last,
            "record_bytes": record,
            "value": N * nsub / (ms / 1e3), "unit": "particle-substeps/s", "ms_per_step": ms, "steps": steps,
            "finite_gradient": bool(np.isfinite(gm).all() and (gt is None or np.isfinite(gt).all())),
            "timing": "CUDA events on the library's stream, after 2 warm-up steps (allocation, graph capture)"}


def full_rollout(nsub: int, steps: int):
    """The skill's whole rollout of the 1M bed (2,000 substeps) with the
    checkpoint interval the free memory allows, against a shifted copy of
    the initial bed."""
    import numpy as np
    import torch

    from paper_2510_17335_gb300 import mpm
    from paper_2510_17335_gb300 import workloads as W

    w = W.cfg_1m()
    K = mpm.checkpoint_interval(nsub, w.n, mpm.blocked_nodes(w.res), torch.cuda.mem_get_info()[0])
    target = w.x0 + np.array([0.003, -0.002, 0.001], np.float32)
    return {"workload": "bed1m_grid128, the skill's whole rollout from the initial bed",
            **rollout_leg(w, nsub, steps, K, target)}


def rollout_250k(steps: int):
    """The differentiable-rollout workload: 250,000 particles on 96^3, 1,000
    substeps from the initial bed with the start material, MSE of the final
    positions against the final positions of the ground-truth material (an
    untimed forward), gradients of (E, nu, rho, phi) and the six skill
    parameters; checkpoint every 50 substeps as the workload states, and
    again with the interval the free memory allows."""
    import torch

    from paper_2510_17335_gb300 import mpm
    from paper_2510_17335_gb300 import workloads as W

    w = W.cfg_250k()
    nsub = w.n_substeps
    with mpm.simulation_from_workloads([w]) as ref:
        ref.forward(nsub)
        target = ref.get_state()["x"]
    start = w.extra["start_material"]
    k_work = int(w.extra["checkpoint_every"])
    k_mem = mpm.checkpoint_interval(nsub, w.n, mpm.blocked_nodes(w.res), torch.cuda.mem_get_info()[0])
    out = {"workload": "bed250k_grid96: 250,000 particles, 96^3 grid, 1,000 substeps, MSE against the "
                       "ground-truth material's final positions, start material +20%",
           **rollout_leg(w, nsub, steps, k_work, target, start)}
    if k_mem != k_work:
        m = rollout_leg(w, nsub, steps, k_mem, target, start)
        out["memory_interval"] = {k: m[k] for k in ("checkpoint_every", "recomputed_substeps", "value",
                                                     "ms_per_step", "record_bytes")}
    return out


# --------------------------------------------------------------------------
# system identification: wall clock to 5% parameter error, batched vs serial
# --------------------------------------------------------------------------
def sysid_leg(n_cand: int, nsub: int, iters: int):
    import numpy as np

    from paper_2510_17335_gb300 import mpm, sysid
    from paper_2510_17335_gb300 import workloads as W

    w = W.cfg_sysid(n_substeps=nsub)
    rng = np.random.default_rng(W.SEED_BASE + 6)
    truth = (w.E, w.nu, w.rho, w.phi_deg)
    free = (True, True, False, True)                # E, nu and phi; rho known (only E/rho moves the bed)
    starts = [(rng.uniform(*sysid.RANGES[0]), rng.uniform(0.2, 0.4), w.rho, rng.uniform(*sysid.RANGES[3]))
              for _ in range(n_cand)]
    grid = mpm.make_obs_grid((0.5, 0.5), 0.5, 40)
    names, _ = sysid.identifiable(np.asarray(truth)[None, :], free)
    out = {"candidates": n_cand, "particles_per_candidate": w.n, "grid": "64^3", "substeps": nsub,
           "iterations": iters, "free": ["E", "nu", "phi"], "identified": names, "truth": list(truth),
           "line_search": "hmd (5 multiples, Sec. III-F)",
           "optimiser": "RMSprop beta 0.9, step sizes E 1e4, nu 0.01, phi 1; adjoint clipping 1e4",
           "criterion": "every candidate within 5% on the identified quantities (K = E / (3 (1 - 2 nu)), phi)"}
    # serial: one handle per candidate, its line-search multiples together;
    # serial_per_instance: every instance (candidate gradient, each
    # candidate's multiple) launched alone
    for mode in ("batched", "serial", "serial_per_instance"):
        r = sysid.identify(w, truth, starts, nsub, iters, grid, free=free, batched=(mode == "batched"),
                           per_instance=(mode == "serial_per_instance"))
        fin = r.params[-1]
        out[mode] = {"iterations_to_5pct": r.converged_at, "seconds_to_5pct": r.seconds_to_converge,
                     "seconds_per_iteration": r.seconds[-1] / len(r.seconds),
                     "final_max_rel_error": float(np.max(r.errors[-1])),
                     "final_rel_error_E_nu": [float(np.max(np.abs(fin[:, 0] / w.E - 1))),
                                              float(np.max(np.abs(fin[:, 1] / w.nu - 1)))],
                     "final_params": np.round(fin, 4).tolist()}
    b = out["batched"]["seconds_per_iteration"]
    out["speedup_per_iteration"] = out["serial"]["seconds_per_iteration"] / b
    out["speedup_per_iteration_vs_per_instance"] = out["serial_per_instance"]["seconds_per_iteration"] / b
    return out


# --------------------------------------------------------------------------
# our implementation
# --------------------------------------------------------------------------
def run_ours(args):
    import numpy as np
    import torch

    from paper_2510_17335_gb300 import mpm
    from paper_2510_17335_gb300 import workloads as W

    ws, rank, local = dist_env()
    torch.cuda.set_device(local)
    dist = None
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    def barrier():
        if dist is not None:
            dist.barrier()

    w = W.cfg_1m()
    N, S = w.n, args.substeps
    # per recorded substep: a state, the grids (acc + vout + flags) and the
    # SVD record of the trial F (the library's layout)
    slot_state, slot_grid = mpm.record_bytes(N, mpm.blocked_nodes(w.res))
    K = args.checkpoint or mpm.checkpoint_interval(S, N, mpm.blocked_nodes(w.res), torch.cuda.mem_get_info(local)[0])
    record_bytes = (K + 1) * slot_state + K * slot_grid
    stream = torch.cuda.Stream()
    opts = mpm.make_options(checkpoint_every=K, tile_scatter=args.tile, sort_every=args.sort)
    sim = mpm.simulation_from_workloads([w], opts)
    sim.set_stream(stream.cuda_stream)
    dev = torch.device("cuda", local)
    with torch.cuda.stream(stream):
        # rollout start state: the skill at substep `start` (shovel inserting)
        sim.forward(args.start)
        # register caps of the particle kernels and the sort interval, timed
        # from that state (which the tuner restores)
        tuned = sim.autotune(args.tune_substeps) if args.tune_substeps > 0 else None
        st0 = {k: torch.empty((N, 3) if k in "xv" else (N, 3, 3), device=dev) for k in "xvCF"}
        sim.get_state(device_out=st0)
        target = (torch.from_numpy(w.x0).to(dev) + torch.tensor([0.003, -0.002, 0.001], device=dev)).contiguous()
        dldx = torch.empty((N, 3), device=dev)
    stream.synchronize()

    def step():
        sim.set_substep(args.start)
        sim.set_state(st0["x"], st0["v"], st0["C"], st0["F"])
        sim.forward(S, record=True)
        sim.loss_mse(target, grad_out=dldx)
        return sim.backward(dL_dx=dldx)

    def fwd_step():
        sim.set_substep(args.start)
        sim.set_state(st0["x"], st0["v"], st0["C"], st0["F"])
        sim.forward(S)

    bus = None
    try:
        pr = torch.cuda.get_device_properties(local)
        bus = f"{pr.pci_domain_id:08X}:{pr.pci_bus_id:02X}:{pr.pci_device_id:02X}.0"
    except Exception:
        bus = None

    with torch.cuda.stream(stream):
        for _ in range(args.warmup):
            step()
            fwd_step()
        # ---- timed: forward + backward ----
        launches0 = sim.info()["kernel_launches"]
        clocks = ClockSampler(bus)
        clocks.start()
        barrier()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(args.steps):
            grads = step()
        e1.record(stream)
        torch.cuda.synchronize()
        barrier()
        clk = clocks.stop()
        launches = sim.info()["kernel_launches"] - launches0
        ms = e0.elapsed_time(e1)
        # ---- the same steps again with a CUDA event pair around every kernel
        # (on the library's stream) for the per-kernel times and the roofline;
        # kept out of the timed region above, which the events slow by ~4% ----
        sim.profile(True)
        for _ in range(args.steps):
            step()
        torch.cuda.synchronize()
        prof = sim.profile_read()
        sim.profile(False)
        # ---- forward only ----
        torch.cuda.synchronize()
        f0, f1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        f0.record(stream)
        for _ in range(args.steps):
            fwd_step()
        f1.record(stream)
        torch.cuda.synchronize()
        fms = f0.elapsed_time(f1)

    ms, fms = max_over_ranks(dist, [ms, fms], dev)
    value = job_rate(ws, N * S * args.steps, ms / 1e3)
    fwd_value = job_rate(ws, N * S * args.steps, fms / 1e3)

    # ---- end to end through the C ABI with host buffers ----
    e2e = None
    if not args.no_e2e:
        xh = torch.empty((N, 3), dtype=torch.float32, pin_memory=True)
        xh.copy_(st0["x"].cpu())
        vh = torch.empty((N, 3), dtype=torch.float32, pin_memory=True); vh.copy_(st0["v"].cpu())
        Ch = torch.empty((N, 3, 3), dtype=torch.float32, pin_memory=True); Ch.copy_(st0["C"].cpu())
        Fh = torch.empty((N, 3, 3), dtype=torch.float32, pin_memory=True); Fh.copy_(st0["F"].cpu())
        th = torch.empty((N, 3), dtype=torch.float32, pin_memory=True); th.copy_(target.cpu())
        arrs = [a.numpy() for a in (xh, vh, Ch, Fh, th)]

        def e2e_step():
            sim.set_substep(args.start)
            sim.set_state(*arrs[:4])
            sim.forward(S, record=True)
            L, g = sim.loss_mse(arrs[4])
            return sim.backward(dL_dx=g)

        with torch.cuda.stream(stream):
            e2e_step()
            torch.cuda.synchronize()
            barrier()
            t0 = time.perf_counter()
            for _ in range(args.steps):
                gm, gt = e2e_step()
            torch.cuda.synchronize()
            barrier()
            es = time.perf_counter() - t0
        (es,) = max_over_ranks(dist, [es], dev)
        h2d = N * 4 * (3 + 3 + 9 + 9) + 2 * N * 3 * 4      # state, target and dL/dx in
        d2h = N * 3 * 4 + 8 * (1 + 4 + 6)                   # dL/dx, loss and gradients out
        e2e = {"value": job_rate(ws, N * S * args.steps, es), "unit": "particle-substeps/s",
               "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h}

    if rank != 0:
        if dist is not None:
            dist.destroy_process_group()
        return

    # roofline of the dominant kernel (largest summed device time)
    peak, peak_kind = measured_peaks()
    name = max(prof, key=lambda k: prof[k][0])
    tot_ms, nl = prof[name]
    avg_s = tot_ms / 1e3 / max(nl, 1)
    kernels = {k: {"ms_total": round(v[0], 3), "launches": v[1],
                   "share": round(v[0] / max(sum(x[0] for x in prof.values()), 1e-12), 4)} for k, v in prof.items()}
    roof = alu = None
    if name in ALGO_BYTES:
        algo = ALGO_BYTES[name] * N
        ach = algo / avg_s / 1e9
        cnt = kernel_counters(name)
        roof = {"bound": "hbm", "achieved": round(ach, 1), "peak": peak, "unit": "GB/s", "frac": round(ach / peak, 4),
                "traffic": cnt["dram_bytes"] if cnt else None, "kernel": name, "algo_bytes_per_launch": algo,
                "avg_launch_us": round(avg_s * 1e6, 2), "peak_kind": f"{peak_kind} hbm_gbs",
                "timing": "CUDA events around every launch, repetition of the timed steps"}
        if cnt:
            # the second limit: FP32 arithmetic and instruction issue, from the
            # executed counts of one ncu capture and the live duration
            fl = cnt["fp32_flops"] / avg_s / 1e12
            ins = cnt["warp_insts"] / avg_s
            alu = {"kernel": name, "fp32_tflops": round(fl, 2), "fp32_peak_tflops": round(FP32_PEAK_TFLOPS, 1),
                   "fp32_frac": round(fl / FP32_PEAK_TFLOPS, 4), "warp_insts_per_s": round(ins, -6),
                   "issue_peak_per_s": ISSUE_PEAK, "issue_frac": round(ins / ISSUE_PEAK, 4),
                   "counts": "executed per launch (ncu, profiles/kernel_counters.txt)",
                   "peaks": "152 SMs x 128 FP32 lanes x 2 flop, 152 x 4 schedulers x 1 warp-instruction, at 2.07 GHz"}
    # the whole step against the same peak: the method's bytes per
    # particle-substep (forward + backward, and forward alone) over the
    # measured step times
    step_bytes = (FWD_BYTES + BWD_BYTES) * N * S
    roof_step = {"bound": "hbm", "bytes_per_particle_substep": FWD_BYTES + BWD_BYTES,
                 "achieved": round(step_bytes * args.steps / (ms / 1e3) / 1e9, 1), "peak": peak, "unit": "GB/s",
                 "frac": round(step_bytes * args.steps / (ms / 1e3) / 1e9 / peak, 4),
                 "fwd_bytes_per_particle_substep": FWD_BYTES,
                 "fwd_frac": round(FWD_BYTES * N * S * args.steps / (fms / 1e3) / 1e9 / peak, 4),
                 "peak_kind": f"{peak_kind} hbm_gbs"}
    # the other legs need the main leg's memory; they characterise one GPU,
    # so a multi-rank run (replicas) skips them
    sim.close()
    one = ws == 1
    full = full_rollout(args.full_substeps, args.full_steps) if one and args.full_substeps > 0 else None
    r250 = rollout_250k(args.full_steps) if one and args.rollout_250k else None
    batch = None
    if one and args.batch > 0:
        batch = batched_vs_serial(args.batch, args.batch_substeps, 3, args.sort)
    sid = sysid_leg(args.sysid, args.sysid_substeps, args.sysid_iters) if one and args.sysid > 0 else None
    cpu = None
    if not args.no_cpu_baseline and ws == 1:
        # the oracle on every host core (OpenMP), and its plain serial loops
        # on one core (about 14 s), on the same bounded sample
        cores = host_cores()
        r, secs, desc = oracle_sample(w, 24, 40, args.start, cores)
        r1, secs1, desc1 = oracle_sample(w, 24, 40, args.start, 1)
        rs, ss = oracle_small_workload(cores)
        w250 = W.cfg_250k()
        r250c, s250c, _ = oracle_sample(w250, max(w250.res), 20, 0, cores)
        cpu = {"value": r, "unit": "particle-substeps/s", "cores": cores, "kind": "oracle", "sample": desc,
               "seconds": round(secs, 2),
               "single_thread": {"value": r1, "cores": 1, "seconds": round(secs1, 2), "sample": desc1},
               "small_workload": {"value": rs, "cores": cores, "seconds": round(ss, 2),
                                  "sample": "the whole 8,000-particle parity workload on its 32^3 grid, "
                                            "200 substeps fwd+bwd"},
               "rollout_250k": {"value": r250c, "cores": cores, "seconds": round(s250c, 2),
                                "sample": f"the whole {w250.n}-particle bed of the differentiable-rollout "
                                          "workload on its 96^3 grid, its first 20 substeps fwd+bwd"}}
    line = {
        "metric": "particle-substeps/s (fwd+bwd)", "value": value, "unit": "particle-substeps/s",
        "n_gpus": ws, "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": WORKLOAD,
                   "substeps_per_step": S, "checkpoint_every": K, "start_substep": args.start,
                   "tile_scatter": args.tile, "sort_every": tuned["sort_every"] if tuned else args.sort,
                   "autotune": ({"trial_substeps": args.tune_substeps, **tuned} if tuned else None),
                   "record_bytes": record_bytes,
                   "l2": f"inputs larger than L2 (96 MB state, {record_bytes / 1e9:.1f} GB of recorded states and grids per step)",
                   "parallelism": f"replicas x{ws}"},
        "fwd_value": fwd_value, "fwd_ms_per_step": fms / args.steps,
        "roofline": roof, "roofline_step": roof_step, "alu": alu, "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": launches,
        "full_rollout": full,
        "rollout_250k": r250,
        "batched_vs_serial": batch,
        **({"sysid": sid} if sid is not None else {}),
        "kernels": kernels, "clocks": clk,
    }
    print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()


SM_CLOCK_HZ = 2.07e9
FP32_PEAK_TFLOPS = 152 * 128 * 2 * SM_CLOCK_HZ / 1e12     # 80.5
ISSUE_PEAK = 152 * 4 * SM_CLOCK_HZ                        # warp-instructions/s


def kernel_counters(name: str):
    """Per-launch DRAM bytes, executed FP32 flops and warp instructions of a
    kernel from profiles/kernel_counters.txt, while its sources still hash to
    the recorded sha (else None: the counters are stale)."""
    tf = os.path.join(ROOT, "profiles", "kernel_counters.txt")
    if not os.path.exists(tf):
        return None
    sha = kernel_source_sha()
    for line in open(tf):
        f = line.split()
        if len(f) >= 5 and not line.startswith("#") and f[0] == name and f[1] == sha:
            return {"dram_bytes": int(f[2]), "fp32_flops": int(f[3]), "warp_insts": int(f[4])}
    return None


def _code_only(text: str) -> str:
    """C/CUDA source without comments, trailing blanks and empty lines: what
    the compiler sees of it (comment edits leave the kernels, and so their
    counters, unchanged)."""
    import re
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    out = []
    for line in text.splitlines():
        cut = None
        i = line.find("//")
        while i >= 0:
            if line.count('"', 0, i) % 2 == 0:   # not inside a string literal
                cut = i
                break
            i = line.find("//", i + 2)
        line = (line if cut is None else line[:cut]).rstrip()
        if line:
            out.append(line)
    return "\n".join(out)


def kernel_source_sha() -> str:
    """Hash of what the profiled kernels are built from: the code (comments
    stripped) of their sources, including the launch constants, and the
    nvcc architecture and flags."""
    import hashlib

    from paper_2510_17335_gb300 import build
    h = hashlib.sha256()
    for f in ("mpm_kernels.cu", "mpm_device.cuh", "mpm_types.h", "mpm_reg.h", "mpm_launch.h"):
        h.update(_code_only(open(os.path.join(ROOT, "paper_2510_17335_gb300", "csrc", f)).read()).encode())
    flags = [f for f in build.FLAGS if not f.startswith("/") and ROOT not in f]
    h.update(" ".join(build.ARCH + flags).encode())
    return h.hexdigest()[:16]


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
        return
    from paper_2510_17335_gb300 import build
    build.build()
    run_ours(args)


if __name__ == "__main__":
    main()
