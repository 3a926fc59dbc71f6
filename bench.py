#!/usr/bin/env python3
"""Benchmark of the explicit PDN impact step on GB300.

A step is one explicit time step of the whole hot path (striker update,
contact detection/projection, hex8 + damage, interface + cohesive law, CSR
gather + lumped-mass update, reaction sum).  The default workload is the
largest single-GPU plate: 100x150x4.4 mm refined to 400x600x32 hex8
(7,680,000 elements, two per ply), 16 seeded quasi-isotropic plies with
interfaces, FP32 element arithmetic, FP64 integration, 5.5 kg striker at
4 m/s.  Before the warm-up and the timed steps, an untimed pre-roll advances
the impact past first contact into the contact phase (the workload's
``preroll``: 2,700 steps, about half way to the peak contact force), so that
the timed steps carry a contact set, damaged elements and a non-zero contact
force; the line's config states the window's state.

value  = element-updates/s = n_hex * K / (device time of the K timed steps),
         max over ranks; inputs already resident in HBM.
e2e    = the same metric through the C ABI from host buffers, a user's whole
         run: mesh upload and set-up, the pre-roll and the K steps, and the
         read-back of the force history, the final nodal state and a damage
         field, all inside the timed region; rate = n_hex * (pre-roll + K) /
         wall time.
roofline = the hex8 kernel's algorithmic bytes per launch in the window's
         state (connectivity, ply and pristine flag per element, the
         Gauss-point history read and written only for elements that left
         the initial state, reference coordinates and displacement per node)
         / its mean launch time (CUDA events on the library's stream, over a
         window of the same run right after the timed region) against the
         measured HBM copy bandwidth; beside it the kernel's instruction-issue
         bound from a stored ncu count of its warp instructions.
cpu_baseline = the FP64 oracle (oracle/) continuing from the GPU's committed
         state at the end of the timed window (displacement, velocity,
         acceleration, history, contact set, striker installed in it), timed
         for a bounded number of steps on this host's cores; the GPU advances
         the same steps from the same state and the line states the FP32 path's
         measured error against the oracle over them ("f32_vs_oracle").

--impl reference times the oracle alone on the same workload from rest
(bounded sample) and prints its own line.  Multi-GPU: one process per GPU,
each rank runs an independent replica (weak scaling, no data-path
collective).

--workload plate runs the same measurement on the 100x150x4.4 mm plate,
128x192x16 hex8 (393,216 elements, 3 m/s).

--workload batch64 measures the batched persistent launch instead: 64 seeded
plates of 8k-400k hex8 (6.2M in total) advanced together by pdn_batch_step,
against the same plates advanced one after another by the plain pdn_step
(speedup at identical peak contact forces).

--workload as4 runs the AS4/8552 coupon of Sec. 3.2: 150x100 mm, 207x138x8
hex8 (228,528 elements, 0.725 mm, one per ply cluster), interfaces between
clusters, frame and clamp supports, Table 1 material, 5 kg striker R = 8 mm at
2.78 m/s, gravity, Tchamwa-Wielgosz phi = 1.033; by default the paper's whole
5 ms of simulated time (214,000 steps).

--workload mmu divides the AS4/8552 coupon once on the device (Algorithm 3:
228,528 hexes and 171,396 interfaces become the paper's 0.3625 mm mesh of
1,828,224 hexes and 685,584 interfaces) and runs the impact on the divided
mesh: the division's device time and rate go in "mesh_multiply", the line's
value is the step rate on the divided mesh, and the end-to-end leg starts
from the coarse mesh on the host.

--workload surrogate trains the learned intralaminar law (generation and
training times reported), measures its held-out accuracy, and runs the
100x150 mm plate with the learned law against the exact law (step time and
peak contact force).
"""
from __future__ import annotations

import argparse
import json
import os
import re
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "element-updates/sec and HBM-roofline fraction at stated peak-contact-force error"
UNIT = "element-updates/s"
F32_PEAK_TOL = 5e-3     # peak contact force vs the FP64 oracle, asserted by tests/test_gpu_parity.py
F32_DISP_TOL = 1e-4


def hex_alg_bytes(n_hex: int, n_nodes: int) -> int:
    """Algorithmic bytes of one hex8 launch: per element the connectivity
    (32 B), the ply id (1 B) and the Gauss-point history read and written
    (2 x 8 points x 7 fields x 4 B = 448 B); per node the FP32 reference
    coordinates and displacement (12 + 12 B), each read once."""
    return n_hex * (32 + 1 + 448) + n_nodes * 24


def coh_alg_bytes(n_coh: int) -> int:
    """Algorithmic bytes of the interface elements of one pass: connectivity
    (32 B) and the four thresholds read and written (2 x 16 B)."""
    return n_coh * (32 + 2 * 4 * 4)


def step_alg_bytes(n_hex, n_coh, n_nodes, n_surf) -> int:
    """Algorithmic bytes of one whole step (every datum moved once):
    hexes as above; interface elements connectivity + 4 thresholds read and
    written; nodes: X and FP32 mirror read, mirror written, FP64 d and v read
    and written, mass, flag; surface nodes: FP64 reference position."""
    return (n_hex * (32 + 1 + 448) + n_coh * (32 + 2 * 4 * 4)
            + n_nodes * (12 + 12 + 12 + 48 + 48 + 8 + 1) + n_surf * 48)


def hex_alg_bytes_state(n_hex: int, n_nodes: int, n_hex_hist: int) -> int:
    """Algorithmic bytes of one hex8 launch in a given state: per element the
    connectivity (32 B), the ply id (1 B) and its pristine flag read and
    written (2 B); the Gauss-point history read and written (448 B) only for
    the n_hex_hist elements that have left the initial state; per node the
    FP32 reference coordinates and displacement (12 + 12 B), each read once."""
    return n_hex * (32 + 1 + 2) + n_hex_hist * 448 + n_nodes * 24


def step_alg_bytes_state(n_hex, n_hex_hist, n_coh, n_coh_hist, n_nodes, n_surf) -> int:
    """Algorithmic bytes of one whole step in a given state: hexes as in
    hex_alg_bytes_state; interface elements their connectivity and flag
    (32 + 2 B) and their four thresholds read and written (32 B) only when
    damaged; nodes and surface nodes as in step_alg_bytes."""
    return (n_hex * (32 + 1 + 2) + n_hex_hist * 448 + n_coh * (32 + 2) + n_coh_hist * 32
            + n_nodes * (12 + 12 + 12 + 48 + 48 + 8 + 1) + n_surf * 48)


def kernels_per_pass(info: dict, n_coh: int) -> int:
    """Kernels one pass launches: contact, hex, gather and tail, plus the
    interface kernel where interface elements are evaluated on their own
    (not as node pairs inside the gather, nor inside the mixed kernel)."""
    separate_coh = n_coh > 0 and not info.get("coh_pairs", 0) and info["hex_variant"] < 4
    return 5 if separate_coh else 4


def issue_bound_ms(warp_instructions: float, sm_mhz: float, n_sm: int = 152) -> float:
    """Time to issue a launch's warp instructions at one instruction per
    cycle on each of the four schedulers of every SM."""
    return warp_instructions / (n_sm * 4 * sm_mhz * 1e6) * 1e3


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(p) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi sampling of SM clocks and throttle reasons during a region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def __enter__(self):
        fd, self.path = tempfile.mkstemp(prefix="clocks_", suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
            time.sleep(0.3)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *a):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        if not self.path or not os.path.exists(self.path):
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for nm, val in zip(names, parts[5:9]):
                if val.lower() in ("active", "1"):
                    reasons.add(nm)
        os.unlink(self.path)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(smax), "reasons": sorted(reasons),
                "samples": len(sm)}


def max_over_ranks(dist, values, device):
    """Element-wise maximum over the ranks of a list of local timings (the
    job's time is its slowest replica's); identity on one process."""
    if dist is None:
        return [float(v) for v in values]
    import torch
    t = torch.tensor([float(v) for v in values], device=device, dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return [float(v) for v in t.tolist()]


def whole_job_rate(world_size: int, units_per_rank: float, ms: float) -> float:
    """Units processed by all ranks (each rank one replica of the workload)
    per second of the slowest rank's time."""
    return world_size * units_per_rank / (ms * 1e-3)


def dist_setup():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def divided_name(w) -> str:
    """Name of the AS4 coupon divided once (the mesh-multiplication workload)."""
    return w.name.replace("207x138x8", "414x276x16") + "_divided_on_device"


def reference_workload(args):
    """The workload the reference arm times for --workload: the oracle runs the
    same plate as the GPU arm (for the divided coupon, divided by the oracle's
    own mesh multiplication; for the learned law, the exact law it stands in
    for), under the GPU arm's workload name."""
    import dataclasses

    import pdn_inputs as pi
    if args.workload == "mmu":
        import oracle.mesh_multiply as omm
        w = pi.as4_frame_plate(steps=args.steps, seed=args.seed)
        g = omm.multiply_plate(w.plate, 1)
        nx, ny, nz = w.plate.grid
        fine = pi.Plate(X=g["X"], hex=g["hex"], coh=g["coh"], ply_of_hex=g["ply_of_hex"],
                        ply_of_coh=g["ply_of_coh"], ply_angle_deg=w.plate.ply_angle_deg, fixed=g["fixed"],
                        surf=g["surf"], dims=w.plate.dims, grid=(2 * nx, 2 * ny, 2 * nz))
        return dataclasses.replace(w, plate=fine), divided_name(w)
    w = workload_for(args)
    return w, (w.name + "_learned_law" if args.workload == "surrogate" else w.name)


def workload_for(args):
    import dataclasses

    import pdn_inputs as pi
    wl = getattr(args, "workload", "large")
    if wl == "large":
        w = pi.large_fp32_plate(steps=args.steps)
    elif wl == "as4":
        w = pi.as4_frame_plate(steps=args.steps, seed=args.seed)
    else:
        w = pi.damage_fp32_plate(seed=args.seed)
    if getattr(args, "preroll", None) is not None:
        w = dataclasses.replace(w, preroll=int(args.preroll))
    return w


def oracle_rate(w, seconds: float, max_steps: int, threads: int):
    """Oracle element-updates/s on a bounded sample of the workload's steps."""
    import oracle
    M = oracle.model_for(w, n_threads=threads)
    M.step(1)  # first step outside the timing (thread pool start)
    n = 0
    t0 = time.perf_counter()
    while n < max_steps:
        M.step(1)
        n += 1
        if time.perf_counter() - t0 > seconds:
            break
    dt = time.perf_counter() - t0
    M.close()
    return w.plate.n_hex * n / dt, n, dt


def run_reference(args, ws, rank):
    if rank != 0:
        return 0
    cores = len(os.sched_getaffinity(0))
    budget = max(10.0, min(120.0, args.ref_seconds))
    if args.workload == "batch64":
        return run_reference_batch(args, cores, budget)
    w, name = reference_workload(args)
    # warm-up steps are part of the bounded sample's set-up
    rate, n, dt = oracle_rate(w, budget, max(1, args.steps), cores)
    line = {
        "impl": "reference", "metric": METRIC, "value": rate, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * dt / n, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": name, "n_hex": w.plate.n_hex, "n_coh": w.plate.n_coh,
                   "n_nodes": w.plate.n_nodes, "l2": "inputs larger than L2"},
        "cpu_baseline": {"value": rate, "unit": UNIT, "cores": cores, "kind": "oracle",
                         "sample": f"{n} of the workload's explicit steps from rest, FP64 oracle, {cores} threads"},
        "e2e": {"value": rate, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


def run_reference_batch(args, cores, budget):
    """The oracle on the 64-plate cases, plate after plate, within the time
    budget (each plate gets an equal share of it)."""
    import pdn_inputs as pi
    cases = pi.batch_plates(n=64, seed=args.seed)
    share = budget / len(cases)
    upd, secs, steps = 0.0, 0.0, 0
    for w in cases:
        rate, n, dt = oracle_rate(w, share, max(1, args.steps), cores)
        upd += w.plate.n_hex * n
        secs += dt
        steps += n
    rate = upd / secs
    line = {
        "impl": "reference", "metric": METRIC, "value": rate, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": None, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": f"batch64_seed{args.seed}_8k-400k_hex8", "n_plates": len(cases),
                   "n_hex": sum(w.plate.n_hex for w in cases), "l2": "inputs larger than L2"},
        "cpu_baseline": {"value": rate, "unit": UNIT, "cores": cores, "kind": "oracle",
                         "sample": f"{steps} explicit steps over the 64 plates ({secs:.1f} s), FP64 oracle"},
        "e2e": {"value": rate, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


def end_to_end(pkg, torch, w, stream, K, ws, dist):
    """The same metric through the C ABI from host buffers, a user's whole
    run: mesh upload and set-up, the pre-roll and the K steps, and the
    read-back of the force history, the final nodal state and the matrix
    damage field, all inside the timed region."""
    plate = w.plate
    n = w.preroll + K
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    with torch.cuda.stream(stream):
        s2 = pkg.Solver(w, stream=stream.cuda_stream)
        pkg.pdn_step(s2.ctx, n)
        f_now, f_peak, hist = pkg.pdn_contact_force(s2.ctx)
        d_fin, v_fin, imp = pkg.pdn_get_state(s2.ctx)
        dmg = pkg.pdn_damage_field(s2.ctx, "D2")
    t_e2e = time.perf_counter() - t0
    s2.close()
    h2d = (plate.X.nbytes + plate.hex.nbytes + plate.coh.nbytes + plate.ply_of_hex.nbytes + plate.fixed.nbytes
           + plate.surf.nbytes + plate.ply_angle_deg.nbytes)
    d2h = hist.nbytes + d_fin.nbytes + v_fin.nbytes + dmg.nbytes + 24 + 80
    t_e2e = max_over_ranks(dist, [t_e2e], "cuda")[0]
    e2e_value = whole_job_rate(ws, plate.n_hex * n, t_e2e * 1e3)
    return {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": h2d / n, "d2h_bytes_per_step": d2h / n,
            "seconds": t_e2e, "steps": n}


def window_state(pkg, ctx):
    """State of the plate at the end of a window: elements whose history left
    the initial state (these move their history every step), damaged
    elements, damaged interface elements, contact nodes."""
    import numpy as np
    h, r = pkg.pdn_get_history(ctx)
    moved = (h[:4] != 1).any(axis=(0, 1)) | (h[4:] != 0).any(axis=(0, 1))
    damaged = (h[:4] > 1).any(axis=(0, 1))
    coh_moved = (r > 0).any(axis=0) if r.size else np.zeros(0, dtype=bool)
    info = pkg.pdn_get_info(ctx)
    return {"hex_with_history": int(moved.sum()), "hex_damaged": int(damaged.sum()),
            "coh_damaged": int(coh_moved.sum()), "n_active": int(info["n_active"]), "step": int(info["step"])}


def oracle_continuation(pkg, w, ctx, seconds: float, cores: int):
    """The FP64 oracle continuing from the GPU's committed state: the state
    (displacement, velocity, acceleration, Gauss-point and interface history,
    contact set, striker) is installed in the oracle, which is then timed
    step by step for about `seconds`; the GPU advances the same steps from
    the same state, and the FP32 path's errors against the oracle over those
    steps are returned beside the oracle's rate."""
    import numpy as np

    import oracle
    d0, v0, imp = pkg.pdn_get_state(ctx)
    a0 = pkg.pdn_get_acceleration(ctx)
    act, _ = pkg.pdn_get_contact(ctx)
    hist, rD = pkg.pdn_get_history(ctx)
    step0 = pkg.pdn_get_info(ctx)["step"]
    o = oracle.model_for(w, n_threads=cores)
    o.set_history(hist.astype(np.float64).transpose(2, 1, 0), rD.astype(np.float64).T)
    del hist, rD
    o.install_state(d0, v0, a0, act, imp, step0)
    n = 0
    t0 = time.perf_counter()
    while True:
        if o.step(1) != 0:
            raise RuntimeError("oracle step failed")
        n += 1
        if time.perf_counter() - t0 > seconds:
            break
    dt = time.perf_counter() - t0
    pkg.pdn_step(ctx, n)
    fg = pkg.pdn_contact_force(ctx)[2][-n:]
    fo = o.force_history()
    dg, vg, _ = pkg.pdn_get_state(ctx)
    do, vo, _ = o.state()
    ag, _ = pkg.pdn_get_contact(ctx)
    ao, _ = o.active()
    o.close()
    fmax = max(float(np.abs(fo).max()), 1e-300)
    err = {
        "from_step": int(step0), "steps": n,
        "f_rel_err_max": float(np.abs(fg - fo).max() / fmax),
        "f_peak_rel_err": float(abs(fg.max() - fo.max()) / fmax),
        "f_oracle_N": [float(fo.min()), float(fo.max())],
        "disp_rel_err": float(np.abs(dg - do).max() / max(np.abs(do).max(), 1e-300)),
        "dv_rel_err": float(np.abs((vg - v0) - (vo - v0)).max() / max(np.abs(vo - v0).max(), 1e-300)),
        "contact_set_differences": int(np.count_nonzero(ag != ao)), "contact_nodes_oracle": int(ao.sum()),
        "bounds": {"f_peak_rel": F32_PEAK_TOL, "disp_rel": F32_DISP_TOL},
    }
    return w.plate.n_hex * n / dt, n, dt, err


def hex_counters(w):
    """The stored ncu counters of one k_hex launch for this workload (DRAM
    bytes, warp instructions), valid only while the kernel's sources hash to
    the value stored with them."""
    tpath = os.path.join(ROOT, "profiles", "k_hex_counters.json")
    try:
        with open(tpath) as f:
            recs = json.load(f)
    except Exception:
        return None
    h = kernel_source_hash()
    for r in recs:
        if r.get("kernel_source_hash") == h and r.get("workload") == w.name:
            return r
    return None


def run_gpu(args, ws, rank, local):
    import numpy as np
    import torch

    import paper_2301_05552_gb300 as pkg

    if not torch.cuda.is_available():
        raise SystemExit("bench.py needs a CUDA device")
    torch.cuda.set_device(local)
    dist = None
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    pkg.lib()
    w = workload_for(args)
    plate = w.plate
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        solver = pkg.Solver(w, stream=stream.cuda_stream)
    ctx = solver.ctx
    K, W = args.steps, args.warmup
    pkg.pdn_step(ctx, w.preroll)  # untimed: into the contact phase
    pkg.pdn_step(ctx, W)
    rep0 = pkg.pdn_get_info(ctx)["n_repeats"]
    f_before = pkg.pdn_contact_force(ctx)[2]
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    if dist is not None:
        dist.barrier()
    torch.cuda.synchronize()
    with ClockSampler(local) as clocks:
        ev0.record(stream)
        pkg.pdn_step(ctx, K)
        ev1.record(stream)
        torch.cuda.synchronize()
    if dist is not None:
        dist.barrier()
    ms = ev0.elapsed_time(ev1)
    info = pkg.pdn_get_info(ctx)
    repeats = info["n_repeats"] - rep0
    ms = max_over_ranks(dist, [ms], "cuda")[0]
    # one kernel for hexes and interface elements (never with node pairs)
    mixed = info["hex_variant"] >= 4 and not info["coh_pairs"]
    gpu_launches = (K + repeats) * kernels_per_pass(info, plate.n_coh) + 1  # + the target/mode kernel
    value = whole_job_rate(ws, plate.n_hex * K, ms)
    fh = pkg.pdn_contact_force(ctx)[2]
    f_window = fh[len(f_before):]
    state = window_state(pkg, ctx)
    clock_summary = clocks.summary()

    # per-kernel device times over a window of the same run right after the
    # timed steps (CUDA events on the library's stream around every launch)
    prof = pkg.pdn_profile_kernels(ctx, args.profile_steps)
    # a repeated pass evaluates only the elements of released nodes: the
    # element kernel's time per step (all its launches over the steps) is
    # the time of one full launch, counted conservatively
    hex_ms = prof["hex"][0] * prof["hex"][1] / max(args.profile_steps, 1)
    peak_gbs, peak_kind = measured_peaks()
    alg = hex_alg_bytes_state(plate.n_hex, plate.n_nodes, state["hex_with_history"])
    kname = "k_hex<float>"
    if mixed:
        alg += plate.n_coh * (32 + 2) + state["coh_damaged"] * 32
        kname = "k_elem<float> (hex + interface)"
    achieved = alg / (hex_ms * 1e-3) / 1e9
    rec = None if mixed else hex_counters(w)
    sm_mhz = clock_summary.get("sm_mhz") or 2070.0
    roofline = {"bound": "hbm", "achieved": achieved, "peak": peak_gbs, "unit": "GB/s",
                "frac": achieved / peak_gbs, "traffic": rec["dram_bytes"] if rec else None, "kernel": kname,
                "alg_bytes_per_launch": alg, "launch_ms": hex_ms, "peak_kind": peak_kind,
                "alg_bytes_rule": "n_hex*35 + hex_with_history*448 + n_nodes*24 (window state)"}
    if rec:
        ib = issue_bound_ms(rec["warp_instructions"], sm_mhz)
        roofline["issue"] = {"warp_instructions": rec["warp_instructions"], "issue_bound_ms": ib,
                             "frac": ib / hex_ms, "sm_mhz": sm_mhz, "counters_from": rec["captured"]}
    solver_step = pkg.pdn_get_info(ctx)["step"]

    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": K, "warmup": W,
        "ms_per_step": ms / K, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f32+f64", "data": "synthetic",
        "config": {
            "workload": w.name, "n_hex": plate.n_hex, "n_coh": plate.n_coh, "n_nodes": plate.n_nodes,
            "n_surf": plate.n_surf, "dt_s": info["dt"], "preroll_steps": w.preroll,
            "window_first_step": w.preroll + W + 1, "simulated_us": info["time"] * 1e6,
            "precision": "FP32 element forces/damage/cohesive, FP64 integration, striker and gap test",
            "l2": "inputs larger than L2 (working set %.0f MB)" % (info["device_bytes"] / 1e6),
            "f_peak_N": float(fh.max()) if len(fh) else 0.0,
            "f_window_N": [float(f_window.min()), float(f_window.max())] if len(f_window) else None,
            "n_active": state["n_active"], "hex_with_history": state["hex_with_history"],
            "hex_with_history_frac": state["hex_with_history"] / plate.n_hex,
            "hex_damaged": state["hex_damaged"], "coh_damaged": state["coh_damaged"],
            "step_repeats": int(repeats),
            "step_alg_bytes": step_alg_bytes_state(plate.n_hex, state["hex_with_history"], plate.n_coh,
                                                   state["coh_damaged"], plate.n_nodes, plate.n_surf),
            "parallelism": f"replicas x{ws}",
        },
        "roofline": roofline,
        "kernel_ms": {k: v[0] for k, v in prof.items()},
        "kernel_launches": {k: v[1] for k, v in prof.items()}, "profile_steps": args.profile_steps,
        "autotune": {"element_variant": info["hex_variant"], "force_pass_ms_per_variant": info["tune_ms"],
                     "interfaces": ("node pairs in the gather" if info["coh_pairs"] else "interface elements")},
        "gpu_launches": gpu_launches,
        "clocks": clock_summary,
    }
    if rank == 0 and not args.no_cpu_baseline and ws == 1:
        cores = len(os.sched_getaffinity(0))
        rate, n, dt, err = oracle_continuation(pkg, w, ctx, args.cpu_seconds, cores)
        line["cpu_baseline"] = {"value": rate, "unit": UNIT, "cores": cores, "kind": "oracle",
                                "sample": f"{n} explicit steps of the same workload continuing from the GPU's "
                                          f"committed state at step {solver_step} ({dt:.1f} s)"}
        line["config"]["f32_vs_oracle"] = err
    solver.close()
    line["e2e"] = end_to_end(pkg, torch, w, stream, K, ws, dist)
    if rank == 0:
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()
    return 0


def run_batch(args, ws, rank, local):
    """64 independent plates: pdn_batch_step against pdn_step plate after
    plate, same steps, same stream."""
    import numpy as np
    import torch

    import paper_2301_05552_gb300 as pkg
    import pdn_inputs as pi

    if not torch.cuda.is_available():
        raise SystemExit("bench.py needs a CUDA device")
    torch.cuda.set_device(local)
    dist = None
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    pkg.lib()
    cases = pi.batch_plates(n=64, seed=args.seed)
    K, W = args.steps, args.warmup
    n_hex = sum(w.plate.n_hex for w in cases)
    stream = torch.cuda.Stream()
    prec = pkg.PDN_FP32_FORCE
    b = pkg.pdn_batch_init([w.plate for w in cases], [w.material for w in cases], precision=prec,
                           damage_on=True, plasticity_on=True, stream=stream.cuda_stream)
    for c, w in zip(b.plates, cases):
        pkg.pdn_set_impactor(c, *w.impactor())
    pkg.pdn_batch_step(b, W)  # the first call also runs the schedule autotuner
    info0 = pkg.pdn_batch_get_info(b)
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    if dist is not None:
        dist.barrier()
    torch.cuda.synchronize()
    with ClockSampler(local) as clocks:
        ev0.record(stream)
        pkg.pdn_batch_step(b, K)
        ev1.record(stream)
        torch.cuda.synchronize()
    ms_batch = ev0.elapsed_time(ev1)
    info = pkg.pdn_batch_get_info(b)
    peaks_b = np.array([pkg.pdn_contact_force(c)[1] for c in b.plates])
    repeats_b = sum(pkg.pdn_get_info(c)["n_repeats"] for c in b.plates)
    hist_b = {}
    if rank == 0 and not args.no_cpu_baseline:
        # the force histories of the smallest plates in contact, for the
        # comparison with the oracle below
        order = sorted(range(len(cases)), key=lambda k: cases[k].plate.n_hex)
        for k in order:
            if peaks_b[k] > 0.0:
                hist_b[k] = pkg.pdn_contact_force(b.plates[k])[2].copy()
            if len(hist_b) == 3:
                break
    b.close()

    # the plain step: one context per plate, stepped one after another
    ctxs = []
    for w in cases:
        c = pkg.pdn_init_mesh(w.plate, w.material, precision=prec, damage_on=True, plasticity_on=True,
                              stream=stream.cuda_stream)
        pkg.pdn_set_impactor(c, *w.impactor())
        pkg.pdn_step(c, W)
        ctxs.append(c)
    torch.cuda.synchronize()
    ev0.record(stream)
    for c in ctxs:
        pkg.pdn_step(c, K)
    ev1.record(stream)
    torch.cuda.synchronize()
    ms_plain = ev0.elapsed_time(ev1)
    peaks_p = np.array([pkg.pdn_contact_force(c)[1] for c in ctxs])
    for c in ctxs:
        c.close()
    ms_batch, ms_plain = max_over_ranks(dist, [ms_batch, ms_plain], "cuda")
    value = whole_job_rate(ws, n_hex * K, ms_batch)
    alg = sum(step_alg_bytes(w.plate.n_hex, w.plate.n_coh, w.plate.n_nodes, w.plate.n_surf) for w in cases)
    peak_gbs, peak_kind = measured_peaks()
    achieved = alg * K / (ms_batch * 1e-3) / 1e9
    scale = np.maximum(np.abs(peaks_p), 1e-300)
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": K, "warmup": W,
        "ms_per_step": ms_batch / K, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f32+f64", "data": "synthetic",
        "config": {
            "workload": f"batch64_seed{args.seed}_8k-400k_hex8", "n_plates": len(cases), "n_hex": n_hex,
            "n_coh": sum(w.plate.n_coh for w in cases), "n_nodes": sum(w.plate.n_nodes for w in cases),
            "hex_per_plate_min_max": [min(w.plate.n_hex for w in cases), max(w.plate.n_hex for w in cases)],
            "precision": "FP32 element forces/damage/cohesive, FP64 integration, striker and gap test",
            "l2": "inputs larger than L2", "step_alg_bytes": alg, "parallelism": f"replicas x{ws}",
        },
        "batch": {
            "speedup_vs_plain_step": ms_plain / ms_batch,
            "plain_value": ws * n_hex * K / (ms_plain * 1e-3), "plain_ms_per_step": ms_plain / K,
            "f_peak_max_rel_diff_vs_plain": float(np.max(np.abs(peaks_b - peaks_p) / scale)),
            "f_peak_N_range": [float(peaks_b.min()), float(peaks_b.max())],
            "step_repeats": int(repeats_b),
            "schedule": {k: info[k] for k in ("dataflow", "blocks_per_sm", "tile_items", "reg_variant", "grid", "graph")},
            "autotune_candidates": info0["candidates"],
            "passes": info["passes"] - info0["passes"], "launches": info["launches"] - info0["launches"],
        },
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak_gbs, "unit": "GB/s",
                     "frac": achieved / peak_gbs, "traffic": None, "kernel": "k_batch (whole step)",
                     "alg_bytes_per_step": alg, "peak_kind": peak_kind},
        "gpu_launches": int(info["launches"] - info0["launches"]),
        "clocks": clocks.summary(),
    }
    if hist_b:
        # the same plates through the FP64 oracle over the same steps from rest
        import oracle
        cores = len(os.sched_getaffinity(0))
        errs = []
        for k, fb in hist_b.items():
            o = oracle.model_for(cases[k], n_threads=cores)
            if o.step(len(fb)) != 0:
                raise RuntimeError("oracle step failed")
            fo = o.force_history()
            o.close()
            pk = max(float(fo.max()), 1e-300)
            errs.append({"plate": k, "n_hex": cases[k].plate.n_hex, "steps": len(fb), "f_peak_N_oracle": pk,
                         "f_peak_rel_err": abs(float(fb.max()) - pk) / pk,
                         "f_hist_rel_err_max": float(np.abs(fb - fo).max()) / pk})
        line["batch"]["vs_oracle"] = errs
        line["batch"]["f_peak_max_rel_err_vs_oracle"] = max(e["f_peak_rel_err"] for e in errs)
    if rank == 0:
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()
    return 0


def mmu_alg_bytes(nn, nh, nc, ns, nn1, ns1) -> int:
    """Algorithmic bytes of one division level: the coarse mesh read once and
    the divided mesh written once; per node 24 B of coordinates and 1 B of
    constraint bits, per hex 32 B of connectivity and 1 B of ply, per
    interface 32 B, per surface node 4 B."""
    return (nn * 25 + nh * 33 + nc * 32 + ns * 4) + (nn1 * 25 + 8 * nh * 33 + 4 * nc * 32 + ns1 * 4)


def run_mmu(args, ws, rank, local):
    """Device mesh multiplication of the AS4/8552 coupon and the impact on
    the divided mesh."""
    import numpy as np
    import torch

    import paper_2301_05552_gb300 as pkg
    import pdn_inputs as pi

    if not torch.cuda.is_available():
        raise SystemExit("bench.py needs a CUDA device")
    torch.cuda.set_device(local)
    dist = None
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    pkg.lib()
    w = pi.as4_frame_plate(steps=args.steps, seed=args.seed)
    coarse = w.plate
    stream = torch.cuda.Stream()
    opts = dict(precision=pkg.PDN_FP32_FORCE, damage_on=w.damage_on, plasticity_on=w.plasticity_on, phi=w.phi,
                dt_safety=w.dt_safety, gravity=w.gravity, stream=stream.cuda_stream)
    # division: one untimed call, then the device time of three calls
    with torch.cuda.stream(stream):
        pkg.pdn_mesh_multiply(coarse, 1, stream=stream.cuda_stream).close()
        div_ms = []
        for k in range(3):
            r = pkg.pdn_mesh_multiply(coarse, 1, stream=stream.cuda_stream)
            div_ms.append(pkg.pdn_refined_get_info(r)["device_ms"])
            if k < 2:
                r.close()
        ri = pkg.pdn_refined_get_info(r)
        ctx = pkg.pdn_init_refined(r, w.material, **opts)
        r.close()
    nh1, nc1, nn1, ns1 = ri["n_hex"], ri["n_coh"], ri["n_nodes"], ri["n_surf"]
    pkg.pdn_set_impactor(ctx, *w.impactor())
    K, W = args.steps, args.warmup
    pkg.pdn_step(ctx, W)
    rep0 = pkg.pdn_get_info(ctx)["n_repeats"]
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    if dist is not None:
        dist.barrier()
    torch.cuda.synchronize()
    with ClockSampler(local) as clocks:
        ev0.record(stream)
        pkg.pdn_step(ctx, K)
        ev1.record(stream)
        torch.cuda.synchronize()
    if dist is not None:
        dist.barrier()
    ms = max_over_ranks(dist, [ev0.elapsed_time(ev1)], "cuda")[0]
    info = pkg.pdn_get_info(ctx)
    repeats = info["n_repeats"] - rep0
    value = whole_job_rate(ws, nh1 * K, ms)
    prof = pkg.pdn_profile_kernels(ctx, args.profile_steps)
    hex_ms = prof["hex"][0]
    peak_gbs, peak_kind = measured_peaks()
    # the hex kernel's algorithmic bytes in the state of the window (history
    # traffic only for the elements that left the initial state)
    state = window_state(pkg, ctx)
    alg = hex_alg_bytes_state(nh1, nn1, state["hex_with_history"])
    achieved = alg / (hex_ms * 1e-3) / 1e9
    fh = pkg.pdn_contact_force(ctx)[2]
    ctx.close()

    # end to end: the coarse mesh from the host, division, solver set-up, K
    # steps, read-back of the force history and the final state
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    with torch.cuda.stream(stream):
        r2 = pkg.pdn_mesh_multiply(coarse, 1, stream=stream.cuda_stream)
        c2 = pkg.pdn_init_refined(r2, w.material, **opts)
        r2.close()
        pkg.pdn_set_impactor(c2, *w.impactor())
        pkg.pdn_step(c2, K)
        _, _, hist = pkg.pdn_contact_force(c2)
        d_fin, v_fin, _ = pkg.pdn_get_state(c2)
    t_e2e = max_over_ranks(dist, [time.perf_counter() - t0], "cuda")[0]
    c2.close()
    h2d = (coarse.X.nbytes + coarse.hex.nbytes + coarse.coh.nbytes + coarse.ply_of_hex.nbytes
           + coarse.fixed.nbytes + coarse.surf.nbytes + coarse.ply_angle_deg.nbytes)
    d2h = hist.nbytes + d_fin.nbytes + v_fin.nbytes + 104
    div = float(statistics.median(div_ms))
    div_alg = mmu_alg_bytes(coarse.n_nodes, coarse.n_hex, coarse.n_coh, coarse.n_surf, nn1, ns1)
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": K, "warmup": W,
        "ms_per_step": ms / K, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f32+f64", "data": "synthetic",
        "config": {
            "workload": divided_name(w),
            "n_hex": nh1, "n_coh": nc1, "n_nodes": nn1, "n_surf": ns1, "dt_s": info["dt"],
            "simulated_us": info["time"] * 1e6, "f_peak_N": float(fh.max()) if len(fh) else 0.0,
            "step_repeats": int(repeats), "l2": "inputs larger than L2 (working set %.0f MB)"
            % (info["device_bytes"] / 1e6), "parallelism": f"replicas x{ws}",
        },
        "mesh_multiply": {
            "levels": 1, "coarse": {"n_hex": coarse.n_hex, "n_coh": coarse.n_coh, "n_nodes": coarse.n_nodes},
            "divided_edges": ri["n_edges"], "divided_faces": ri["n_faces"], "device_ms": div,
            "device_ms_each": div_ms, "divided_elements_per_s": (nh1 + nc1) / (div * 1e-3),
            "roofline": {"bound": "hbm", "achieved": div_alg / (div * 1e-3) / 1e9, "peak": peak_gbs,
                         "unit": "GB/s", "frac": div_alg / (div * 1e-3) / 1e9 / peak_gbs,
                         "alg_bytes": div_alg, "peak_kind": peak_kind},
        },
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak_gbs, "unit": "GB/s",
                     "frac": achieved / peak_gbs, "traffic": None, "kernel": "k_hex<float>",
                     "alg_bytes_per_launch": alg, "launch_ms": hex_ms, "peak_kind": peak_kind,
                     "alg_bytes_rule": "n_hex*35 + hex_with_history*448 + n_nodes*24 (window state)",
                     "hex_with_history": state["hex_with_history"]},
        "kernel_ms": {k: v[0] for k, v in prof.items()},
        "e2e": {"value": whole_job_rate(ws, nh1 * K, t_e2e * 1e3), "unit": UNIT,
                "h2d_bytes_per_step": h2d / K, "d2h_bytes_per_step": d2h / K, "seconds": t_e2e},
        "gpu_launches": (K + repeats) * kernels_per_pass(info, nc1) + 1,
        "clocks": clocks.summary(),
    }
    if rank == 0 and not args.no_cpu_baseline and ws == 1:
        import oracle.mesh_multiply as omm
        # the oracle's division on a bounded sample: the cut-down coupon
        cut = pi.reduced_as4_frame_plate(nx=80, ny=56).plate
        t0 = time.perf_counter()
        omm.divide_once(cut.X, cut.hex, cut.coh, cut.ply_of_hex, cut.fixed, cut.surf)
        t_div = time.perf_counter() - t0
        line["mesh_multiply"]["cpu_baseline"] = {
            "value": (8 * cut.n_hex + 4 * cut.n_coh) / t_div, "unit": "divided elements/s", "cores": 1,
            "kind": "oracle", "sample": f"one level of the 80x56 cut-down coupon ({cut.n_hex} hexes, {t_div:.1f} s)"}
    if rank == 0:
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()
    return 0


def run_surrogate(args, ws, rank, local):
    """The learned law on the 128x192x16 plate against the exact law."""
    import numpy as np
    import torch

    import paper_2301_05552_gb300 as pkg

    if not torch.cuda.is_available():
        raise SystemExit("bench.py needs a CUDA device")
    torch.cuda.set_device(local)
    pkg.lib()
    w = workload_for(args)
    plate = w.plate
    K, W = args.steps, args.warmup
    Lx, Ly, H = plate.dims
    nx, ny = plate.grid[:2]
    plies = len(plate.ply_angle_deg)
    lc = (Lx / nx * Ly / ny * H / plies) ** (1.0 / 3.0)
    stream = torch.cuda.Stream()
    s = pkg.pdn_sur_create(w.material, lc, seed=args.seed + 1, stream=stream.cuda_stream)
    n_paths, steps_pp, iters, batch = 1_000_000, 8, 40000, 8192
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    n_kept = pkg.pdn_sur_generate(s, n_paths, steps_pp, 0.01, 0.4, 0.9, seed=args.seed + 11)
    t_gen = time.perf_counter() - t0
    t0 = time.perf_counter()
    loss = pkg.pdn_sur_train(s, iters, batch, 2e-3, seed=args.seed + 3)
    t_train = time.perf_counter() - t0
    h = pkg.pdn_sur_create(w.material, lc, seed=0, stream=stream.cuda_stream)
    n_hold = pkg.pdn_sur_generate(h, 20000, steps_pp, 0.01, 0.4, 0.9, seed=args.seed + 99)
    xh, yh = pkg.pdn_sur_get_data(h, 0, n_hold)
    h.close()
    yp = pkg.pdn_sur_forward(s, xh)
    rms = np.sqrt(np.mean(yh[:, :6].astype(np.float64) ** 2, axis=0))
    rel_rms = np.sqrt(np.mean((yp[:, :6] - yh[:, :6]).astype(np.float64) ** 2, axis=0)) / rms
    rel_max = np.max(np.abs(yp[:, :6] - yh[:, :6]), axis=0) / rms
    r_err = float(np.max(np.abs(yp[:, 6:] - yh[:, 6:])))
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    runs = {}
    clock_summary = None
    for mode in ("exact", "learned"):
        with torch.cuda.stream(stream):
            g = pkg.Solver(w, stream=stream.cuda_stream)
        if mode == "learned":
            pkg.pdn_set_surrogate(g.ctx, s, 0.9)
        pkg.pdn_step(g.ctx, W)
        torch.cuda.synchronize()
        with ClockSampler(local) as clocks:
            ev0.record(stream)
            pkg.pdn_step(g.ctx, K)
            ev1.record(stream)
            torch.cuda.synchronize()
        if mode == "learned":
            clock_summary = clocks.summary()
        ms = ev0.elapsed_time(ev1)
        prof = pkg.pdn_profile_kernels(g.ctx, args.profile_steps)
        fh = pkg.pdn_contact_force(g.ctx)[2]
        runs[mode] = dict(ms=ms, hex_ms=prof["hex"][0], f_peak=float(fh.max()) if len(fh) else 0.0,
                          kernel_ms={k: v[0] for k, v in prof.items()})
        g.close()
    s.close()
    ex, le = runs["exact"], runs["learned"]
    # tensor-core work of the learned-law hex kernel, counted as if every
    # Gauss point ran the network (padded 16-wide input and output layers):
    # 2 * (16*64 + 2*64*64 + 64*16) flops per point; a CTA runs it for its
    # 128 points whenever one of them needs it
    flops = plate.n_hex * 8 * 2 * (16 * 64 + 2 * 64 * 64 + 64 * 16)
    peak_tf = 1900.8
    try:
        peak_tf = float(json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))["bf16_tflops"])
    except Exception:
        pass
    ach = flops / (le["hex_ms"] * 1e-3) / 1e12
    line = {
        "metric": METRIC, "value": plate.n_hex * K / (le["ms"] * 1e-3), "unit": UNIT, "n_gpus": 1, "steps": K,
        "warmup": W, "ms_per_step": le["ms"] / K, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "bf16 (network) + f32 + f64", "data": "synthetic",
        "config": {"workload": w.name + "_learned_law", "n_hex": plate.n_hex, "n_coh": plate.n_coh,
                   "n_nodes": plate.n_nodes, "l2": "inputs larger than L2", "onset_ratio": 0.9,
                   "network": "10-64-64-64-10 ReLU, BF16 weights, FP32 accumulation (tcgen05.mma, TMEM "
                              "accumulators, 128 points per CTA)"},
        "surrogate": {
            "speedup_vs_exact_law": ex["ms"] / le["ms"], "exact_ms_per_step": ex["ms"] / K,
            "exact_value": plate.n_hex * K / (ex["ms"] * 1e-3),
            "f_peak_N_exact": ex["f_peak"], "f_peak_N_learned": le["f_peak"],
            "f_peak_rel_diff": abs(le["f_peak"] - ex["f_peak"]) / max(ex["f_peak"], 1e-300),
            "hex_ms_exact": ex["hex_ms"], "hex_ms_learned": le["hex_ms"],
            "kernel_ms_learned": le["kernel_ms"],
            "held_out_points": n_hold, "held_out_rel_rms_stress_err": [float(v) for v in rel_rms],
            "held_out_rel_max_stress_err": [float(v) for v in rel_max], "held_out_max_abs_threshold_err": r_err,
            "train": {"paths": n_paths, "steps_per_path": steps_pp, "points_kept": n_kept, "iters": iters,
                      "batch": batch, "seconds": t_train, "generate_seconds": t_gen,
                      "loss_first": float(loss[0]), "loss_last": float(loss[-1])},
        },
        "roofline": {"bound": "tensor", "achieved": ach, "peak": peak_tf, "unit": "TFLOP/s", "frac": ach / peak_tf,
                     "traffic": None, "kernel": "k_hex_sur (learned law)", "flops_per_launch": flops,
                     "launch_ms": le["hex_ms"], "peak_kind": "measured bf16 (dense GEMM, burst)"},
        "gpu_launches": None,
        "clocks": clock_summary,
    }
    if rank == 0:
        print(json.dumps(line), flush=True)
    return 0


# Sections of pdn_items.cuh (delimited by "// ----" rule lines) that k_hex is
# not compiled from: the contact, interface, tail and gather bodies.
NOT_HEX_SECTIONS = ("// Kernel 1:", "// Kernel 3:", "// Tail of a pass", "// Kernel 4:")


def hex_sections(text: str) -> str:
    """pdn_items.cuh without the sections in NOT_HEX_SECTIONS."""
    parts = re.split(r"^// -{20,}\n", text, flags=re.M)
    return "".join(p for p in parts if not p.startswith(NOT_HEX_SECTIONS))


def kernel_source_hash() -> str:
    """Hash of the source k_hex is compiled from: the kernel file, the device
    helpers and records, and the element sections of the item bodies.  A
    stored DRAM-traffic record of k_hex counts only while this matches."""
    import hashlib
    h = hashlib.sha256()
    for name in ("pdn_kernels.cu", "pdn_items.cuh", "pdn_device.cuh", "pdn_internal.h"):
        with open(os.path.join(ROOT, "paper_2301_05552_gb300", "csrc", name), encoding="utf-8") as f:
            text = f.read()
        if name == "pdn_items.cuh":
            text = hex_sections(text)
        h.update(text.encode("utf-8"))
    return h.hexdigest()[:16]


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=None,
                    help="timed steps (default: 5000 large, 20000 plate, 214000 as4, 500 batch64)")
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["gpu", "reference"], default="gpu")
    ap.add_argument("--seed", type=int, default=0)
    ap.add_argument("--profile-steps", type=int, default=200)
    ap.add_argument("--cpu-seconds", type=float, default=20.0)
    ap.add_argument("--ref-seconds", type=float, default=60.0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--workload", choices=["plate", "large", "as4", "mmu", "batch64", "surrogate"], default="large")
    ap.add_argument("--preroll", type=int, default=None,
                    help="untimed steps before the warm-up (default: the workload's pre-roll into contact)")
    args = ap.parse_args()
    if args.steps is None:
        args.steps = {"batch64": 500, "large": 5000, "as4": 214000}.get(args.workload, 20000)
    if args.warmup < 3 and args.impl == "gpu":
        args.warmup = 3
    ws, rank, local = dist_setup()
    if args.impl == "reference":
        return run_reference(args, ws, rank)
    if args.workload == "batch64":
        return run_batch(args, ws, rank, local)
    if args.workload == "surrogate":
        return run_surrogate(args, ws, rank, local)
    if args.workload == "mmu":
        return run_mmu(args, ws, rank, local)
    return run_gpu(args, ws, rank, local)


if __name__ == "__main__":
    sys.exit(main())
