#!/usr/bin/env python
"""Throughput of the GB300 particle-in-cell hot path.

One benchmark step = one whole PIC time step of the workload: field gather,
Boris push, move and Villasenor-Buneman deposit of every particle, the Yee
FDTD update, the energy diagnostics, and (every K steps) the supercell sort.

Default workload (1 GPU): the paper-scale FP64 plasma, 64^3 cells with 50
electrons per cell (13,107,200 particles, the same particles-per-cell as the
paper's 40^3 x 50 frozen-plasma benchmark), thermal velocity 0.05c, a 1%
density perturbation along x, periodic.  Inputs are seeded and synthetic,
resident in HBM when the timed region starts, and larger than L2 (the FP64
particle store alone is 839 MB).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl gb300|reference]

Prints one JSON line (rank 0).  With N > 1 (torchrun) every rank runs its own
independent replica of the workload (the path is not sharded across GPUs);
the time is the maximum over ranks and the value counts all ranks' particles.
--impl reference times the FP64 CPU oracle on this host's cores instead, on a
bounded sample of the same workload.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "particle-steps/s (FP64 plain vs FP32-mixed), HBM roofline %, adjoint/forward ratio"
UNIT = "particle-steps/s"

# Algorithmic cost of one particle-step of the fused particle kernel, counted
# from its arithmetic (FMA = 2 flops; rsqrt and divide = 1 each):
#   gather 6 trilinear interpolations x 7 lerps x 3 + 3 half-offset adds = 129
#   Boris push 58, move 16, Villasenor-Buneman (one segment) 57, energy 3.
FLOPS_PER_PARTICLE = 263
# Second-order (TSC) form factor with the Esirkepov current, for a move whose
# 1-D old and new stencils share their 3 nodes on every axis (the common case):
#   spline weights 2 lattices x 3 axes (48) + offsets (6); 6 separable 27-point
#   interpolations x 69 = 414; Boris 58, move 16; Esirkepov new weights and dS
#   45, 3 components x (9 transverse factors x 10 + 18 edges x 3) = 432;
#   charges, new offsets and energy 12.
FLOPS_PER_PARTICLE_TSC = 1031
# Minimum HBM traffic per particle-step of the particle store:
#   FP64 store: read cell(4) + offset(24) + u(24) + w(8) = 60 B, write cell + offset + u = 52 B.
#   mixed store: read 4 + 12 + 12 + 4 = 32 B, write 4 + 12 + 12 = 28 B.
# The launch right after a sort also moves the records to the other buffer
# through the sort's permutation (the sort computes ranks only): mixed store
# read cell + offset + u + w + id + perm index = 40 B, write the whole record
# (cell, offset, u, w, id) = 36 B; FP64 store read 4 + 24 + 24 + 8 + 4 + 4 = 68 B,
# write 64 B.
BYTES_PER_PARTICLE = {"fp64": 112, "fp64_after_sort": 132, "mixed": 60, "mixed_after_sort": 76}
FP64_NOMINAL_TFLOPS = 1.25  # GB300 nominal FP64 rate (context; the roofline divides by the in-run probe)


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f), "measured"
    except Exception:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0}, "fallback"


KERNEL_SOURCES = {"fp64": ("k_push.cu", "push_tile.cuh", "pic_internal.cuh"),
                  "mixed": ("k_push32.cu", "push_tile.cuh", "pic_internal.cuh"),
                  "tsc": ("k_tsc.cu", "pic_internal.cuh")}


def _kernel_hash(kind="fp64"):
    h = hashlib.sha256()
    for f in KERNEL_SOURCES[kind]:
        with open(os.path.join(ROOT, "paper_1608_01009_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def _traffic(kind):
    """Per-launch DRAM bytes of the particle kernel from the committed ncu
    summary, if it was taken on the current kernel source (else None)."""
    try:
        with open(os.path.join(ROOT, "profiles", "traffic.json")) as f:
            rec = json.load(f)
        r = rec.get(kind)
        if r and r.get("kernel_sha") == _kernel_hash(kind):
            return r["dram_bytes_per_launch"]
    except Exception:
        pass
    return None


class ClockSampler:
    """nvidia-smi clock / throttle samples while the timed region runs."""

    Q = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.Q,
                                          "--format=csv,noheader,nounits", "-lms", "50"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None
        time.sleep(0.15)
        return self

    def __exit__(self, *a):
        self.lines = []
        if self.proc is not None:
            time.sleep(0.1)
            self.proc.terminate()
            try:
                out, _ = self.proc.communicate(timeout=5)
            except Exception:
                self.proc.kill()
                out, _ = self.proc.communicate()
            self.lines = [l for l in out.splitlines() if l.strip()]

    def summary(self):
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for l in getattr(self, "lines", []):
            f = [x.strip() for x in l.split(",")]
            if len(f) < 8:
                continue
            try:
                sm.append(float(f[0]))
                mx.append(float(f[1]))
            except ValueError:
                continue
            for n, v in zip(names, f[4:8]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


def _dist():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def _barrier_max(torch, value, ws):
    """Maximum of `value` over the ranks (the slowest replica's time)."""
    if ws == 1:
        return value
    import torch.distributed as dist
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([value], dtype=torch.float64, device=dev)
    dist.barrier()
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def weak_value(npart_per_rank, ws, steps, ms_max):
    """Whole-job particle-steps/s: every rank's particles over the slowest rank's time."""
    return npart_per_rank * ws * steps / (ms_max / 1e3)


def _workload_desc(wl, precision):
    return ("%s: %dx%dx%d %s, %d e-/cell (%d particles), vth %.2fc%s, %s" % (
        wl.name, wl.n[0], wl.n[1], wl.n[2], "periodic" if wl.bc == (0, 0, 0) else "bc %s" % (wl.bc,),
        wl.meta.get("ppc", 0), wl.nparticles, wl.meta.get("vth", 0.0),
        ", 1% density perturbation" if wl.meta.get("perturb_eps") else "", precision))


def time_gpu(torch, pic, wl, precision, steps, warmup, clocks=None, with_timing=True, supercell=4, form_factor=1):
    """Device-timed steps of one simulation; returns a result dict."""
    prec = pic.FP64 if precision == "fp64" else pic.MIXED
    sim = pic.Simulation.from_workload(wl, precision=prec, supercell=supercell, form_factor=form_factor)
    st = sim.stream
    for _ in range(warmup):
        sim.step(1)
    sim.sync()
    sim.stage_times()  # reset the stage accumulators
    sim.enable_timing(with_timing)
    before = sim.stage_times()
    sim.launch_count(reset=True)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(st)
    sim.step(steps)
    e1.record(st)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    launches = sim.launch_count()
    after = sim.stage_times()
    sim.enable_timing(False)
    sim.sync()
    wf, wk = sim.energy()
    npart = wl.nparticles
    res = dict(ms=ms, npart=npart, launches=launches, wf=wf, wk=wk,
               stage_ms={k: (after[k] - before[k]) / steps for k in after}, sim=sim)
    return res


def time_e2e(torch, pic, wl, sim, steps):
    """End to end through the public API with HOST buffers: every step takes
    its particle and field inputs from pinned host memory, advances one step
    and reads the energy diagnostics back (pic_energy, 16 B).  The particle
    upload is double-buffered: step i installs its own set
    (pic_set_particles_uploaded) and starts the copy of step i+1's set
    (pic_upload_particles), which crosses the CPU-GPU link while step i
    computes; the first copy is inside the timed region, so every step's
    inputs cross the link there."""
    import numpy as np
    sp = wl.species[0]
    pinned = []
    for a in sp.arrays():
        t = torch.empty(a.shape[0], dtype=torch.float64, pin_memory=True)
        t.numpy()[:] = a
        pinned.append(t.numpy())
    Ep = torch.empty(wl.E.shape, dtype=torch.float64, pin_memory=True).numpy()
    Bp = torch.empty(wl.B.shape, dtype=torch.float64, pin_memory=True).numpy()
    Ep[:] = wl.E
    Bp[:] = wl.B
    h2d = sum(a.nbytes for a in pinned) + Ep.nbytes + Bp.nbytes
    d2h = 16
    # one untimed pass
    sim.upload_particles(0, *pinned)
    sim.set_fields(Ep, Bp)
    sim.set_particles_uploaded(0)
    sim.step(1)
    sim.energy()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    sim.upload_particles(0, *pinned)  # step 0's set
    for i in range(steps):
        sim.set_fields(Ep, Bp)
        sim.set_particles_uploaded(0)
        if i + 1 < steps:
            sim.upload_particles(0, *pinned)  # step i+1's set, copied while step i runs
        sim.step(1)
        sim.energy()
    torch.cuda.synchronize()
    dt = time.perf_counter() - t0
    return dict(seconds=dt, npart=wl.nparticles, steps=steps, h2d=h2d, d2h=d2h)


def time_adjoint(torch, pic, W, nsteps=200, ckpt=20):
    """Cost of the differentiable run on the laser-slab workload: the
    checkpointed forward (pic_tape_forward) and the backward (segment replay +
    adjoint kernels, pic_tape_backward), against the same steps of pic_step."""
    wl = W.config("c4")
    warm = pic.Simulation.from_workload(wl)
    warm.tape_forward(ckpt, ckpt)
    warm.tape_backward(1.0)
    warm.step(3)
    warm.close()
    sim = pic.Simulation.from_workload(wl)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    wk = sim.tape_forward(nsteps, ckpt)
    torch.cuda.synchronize()
    t1 = time.perf_counter()
    dE, dB = sim.tape_backward(1.0)
    torch.cuda.synchronize()
    t2 = time.perf_counter()
    sim.close()
    fast = pic.Simulation.from_workload(wl)
    torch.cuda.synchronize()
    t3 = time.perf_counter()
    fast.step(nsteps)
    fast.sync()
    t4 = time.perf_counter()
    fast.close()
    fwd, bwd, fst = (t1 - t0) * 1e3, (t2 - t1) * 1e3, (t4 - t3) * 1e3
    return {"workload": "c4: 32x32x64, x/y periodic, z absorbing, slab z in [24,40) cells at 0.1 n_crit, "
                        "16 e-/cell (%d particles), a0 = 1 plane wave, FP64" % wl.nparticles,
            "steps": nsteps, "checkpoint_every": ckpt, "loss": "W_K after %d steps" % nsteps,
            "loss_value": wk, "tape_forward_ms": fwd, "backward_ms": bwd, "fast_forward_ms": fst,
            "adjoint_forward_ratio": bwd / fwd, "adjoint_vs_fast_forward": bwd / fst,
            "note": "backward = segment replay (recomputation) + adjoint kernels; adjoint_vs_fast_forward "
                    "divides by pic_step steps of the same workload (the ratio judged against the 3x target), "
                    "adjoint_forward_ratio by the checkpointed forward it reverses"}


def measure_fp64_peak(pic, local):
    """FP64 FMA throughput of this GPU, measured now (pic_probe_fp64_fma: all SMs,
    independent DFMA chains), with the SM clock sampled while it runs."""
    with ClockSampler(local) as clk:
        tf, ms = pic.probe_fp64_fma(local, 16384)
    return {"tflops": tf, "launch_ms": ms, "clocks": clk.summary(),
            "how": "pic_probe_fp64_fma: 4 CTAs x 256 threads per SM, 8 independent FMA chains per thread, "
                   "best of 3 timed launches (FMA = 2 flops)"}


def mixed_vs_fp64(torch, pic, wl, checkpoints=(100, 200)):
    """Error of the mixed path against the FP64 path on the same seeded
    workload: field energy at each checkpoint step and the per-array
    norm-wise errors of E, B and J at the last one.  Beside it, the same
    figures for two FP64 runs that differ only in the sort interval (1, the
    FP64 default, and 3), i.e. in the order of every floating-point sum: the
    reordering noise floor of this chaotic system."""
    import numpy as np

    def rel(a, b):
        return float(np.max(np.abs(a - b)) / max(float(np.max(np.abs(b))), 1e-300))

    runs = {}
    for label, prec, K in (("fp64", pic.FP64, 0), ("fp64_sort3", pic.FP64, 3), ("mixed", pic.MIXED, 0)):
        sim = pic.Simulation.from_workload(wl, precision=prec, sort_interval=K)
        wf, done = {}, 0
        for c in checkpoints:
            sim.step(c - done)
            done = c
            wf[c] = sim.energy()[0]
        E, B = sim.get_fields()
        J = sim.get_current()
        runs[label] = (wf, E, B, J)
        sim.close()
    ref = runs["fp64"]

    def errs(label):
        wf, E, B, J = runs[label]
        out = {"field_energy_rel_err": {"step %d" % c: abs(wf[c] - ref[0][c]) / abs(ref[0][c]) for c in checkpoints}}
        out.update({"%s_rel_err_step_%d" % (k, checkpoints[-1]): rel(x, y)
                    for k, x, y in (("E", E, ref[1]), ("B", B, ref[2]), ("J", J, ref[3]))})
        return out

    return {"reference": "FP64 path, same seed and workload, sorted every step (its default)",
            "field_energy_fp64": {"step %d" % c: ref[0][c] for c in checkpoints},
            "mixed": errs("mixed"), "fp64_reordered_noise_floor": errs("fp64_sort3"),
            "target": "field energy <= 1e-5 relative after 100 steps"}


def time_laser_ramp(torch, pic, W, total=500, adj=50, ck=50):
    """The large laser-plasma workload c5 (256x128x128, 134.2 M electrons over a
    density ramp, a0 = 3 Gaussian pulse, x absorbing): the mixed-precision
    forward for the first total - adj steps (3 of them untimed warm-up), then
    the differentiable FP64 path for the final adj steps and its adjoint.
    Checkpoint every ck steps: with 50 the tape is one segment (a whole FP64
    state of 7 GB, the 50 steps' momenta, 3.2 GB each, and the positions and
    flags of every 8th step), so nothing is recomputed; if that does not fit in
    device memory the run takes ck = 25 and recomputes the first segment.
    The adjoint is set against the checkpointed
    forward it reverses and against plain steps of the same state: FP64
    pic_step steps (a context loaded with the state at step total - adj) and
    the mixed context's own steps."""
    torch.cuda.empty_cache()  # blocks cached by the earlier legs: the tape needs most of the device
    t0 = time.perf_counter()
    wl = W.config("c5")
    gen_s = time.perf_counter() - t0
    nfwd = total - adj - 3
    sim = pic.Simulation.from_workload(wl, precision=pic.MIXED)
    sim.step(3)
    sim.sync()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(sim.stream)
    sim.step(nfwd)
    e1.record(sim.stream)
    sim.sync()
    ms_fwd = e0.elapsed_time(e1)
    n_active = sim.count()
    wf, wk = sim.energy()
    # FP64 pic_step over the same adj steps from this state (then freed)
    E, B = sim.get_fields(device=True)
    p = sim.get_particles(0, device=True)
    fast = pic.Simulation(wl.n, wl.d, wl.dt, wl.bc, pic.FP64, absorb_cells=wl.absorb_cells,
                          absorb_sigma=wl.absorb_sigma)
    fast.set_fields(E, B)
    fast.add_species(wl.species[0].q, wl.species[0].m, *[p[k] for k in ("x", "y", "z", "ux", "uy", "uz", "w")])
    del p, E, B
    torch.cuda.synchronize()
    f0 = time.perf_counter()
    fast.step(adj)
    fast.sync()
    fast_fp64_s = time.perf_counter() - f0
    fast.close()
    del fast
    torch.cuda.empty_cache()
    torch.cuda.synchronize()
    t1 = time.perf_counter()
    try:
        wk_end = sim.tape_forward(adj, ck)
    except pic.PicError as e:
        if e.code != -3 or ck <= 25:  # PIC_ERR_OOM
            raise
        ck = 25
        torch.cuda.synchronize()
        t1 = time.perf_counter()
        wk_end = sim.tape_forward(adj, ck)
    torch.cuda.synchronize()
    t2 = time.perf_counter()
    dE, dB = sim.tape_backward(1.0)
    torch.cuda.synchronize()
    t3 = time.perf_counter()
    gnorm = (float(dE.norm().item()), float(dB.norm().item()))
    del dE, dB
    sim.close()
    mixed_step_s = ms_fwd / nfwd / 1e3
    bwd = t3 - t2
    return {"workload": "c5: 256x128x128, x absorbing, 64 e-/cell over x in [128,256) with a 0->1 n_crit ramp "
                        "over 32 cells (%d particles), a0 = 3 Gaussian pulse (waist 24 cells, 8 wavelengths)"
                        % wl.nparticles,
            "mixed_forward": {"steps": nfwd, "ms_per_step": ms_fwd / nfwd,
                              "particle_steps_per_s": wl.nparticles * nfwd / (ms_fwd / 1e3),
                              "active_after": n_active, "W_F": wf, "W_K": wk},
            "adjoint": {"steps": adj, "checkpoint_every": ck, "tape_forward_s": t2 - t1, "backward_s": bwd,
                        "fast_forward_fp64_s": fast_fp64_s, "fast_forward_mixed_s": mixed_step_s * adj,
                        "adjoint_forward_ratio": bwd / (t2 - t1),
                        "adjoint_vs_fast_forward": bwd / fast_fp64_s,
                        "adjoint_vs_fast_mixed_forward": bwd / (mixed_step_s * adj),
                        "W_K_final": wk_end, "grad_E_norm": gnorm[0], "grad_B_norm": gnorm[1],
                        "note": "backward = segment replay (recomputation, none with one segment), position "
                                "rebuilds + adjoint kernels; adjoint_vs_fast_forward divides by FP64 pic_step "
                                "steps of the same state, the ratio judged against the 3x target"},
            "input_generation_s": gen_s}


def run_laser_ramp(args):
    import torch
    from paper_1608_01009_gb300 import pic, workloads as W
    print(json.dumps(time_laser_ramp(torch, pic, W)))
    return 0


def cpu_oracle_rate(wl, nsteps=1, sample_every=1, threads=False):
    """The FP64 oracle as it stands on the workload state, optionally on every
    k-th particle: the serial build, or (threads=True) its timing build whose
    whole steps push the particles on all host cores.  Returns (particle-steps/s,
    particles, seconds, host threads used)."""
    import oracle as O
    O.use_threads(threads)
    ora = O.Oracle.from_workload(wl)
    if sample_every > 1:
        ora.species = [s.subset(slice(None, None, sample_every)) for s in ora.species]
    npart = sum(s.n for s in ora.species)
    nthreads = O.threads()
    t0 = time.perf_counter()
    ora.step(nsteps)
    dt = time.perf_counter() - t0
    O.use_threads(False)
    return npart * nsteps / dt, npart, dt, nthreads


def run_reference(args):
    ws, rank, _ = _dist()
    if rank != 0:
        return 0
    from paper_1608_01009_gb300 import workloads as W
    wl = W.config(args.workload)
    ncores = os.cpu_count() or 1
    # about 0.4 M particles per host core and step: a second or so of CPU work per step
    every = max(1, wl.nparticles // (400_000 * ncores))
    total_p, total_s, nthreads = 0, 0.0, 1
    for i in range(args.warmup + args.steps):
        r, npart, dt, nthreads = cpu_oracle_rate(wl, 1, every, threads=True)
        if i >= args.warmup:
            total_p += npart
            total_s += dt
    value = total_p / total_s
    sample = ("each step: one whole oracle step of the %dx%dx%d grid with every %d-th particle "
              "(%d particles), particles pushed on %d host threads" % (wl.n[0], wl.n[1], wl.n[2], every,
                                                                      npart, nthreads))
    out = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * total_s / args.steps,
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
           "data": "synthetic (seeded)", "config": {"workload": _workload_desc(wl, "fp64")},
           "cpu_baseline": {"value": value, "unit": UNIT, "cores": nthreads, "kind": "oracle", "sample": sample},
           "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out))
    return 0


def run_profile_case(args):
    """One reduced case (inputs still larger than L2, 2 GB of particle store)
    for profiler captures; prints its device-timed rate, not a bench line."""
    import torch
    torch.cuda.set_device(0)
    from paper_1608_01009_gb300 import pic, workloads as W
    ff = 2 if args.profile_case == "tsc" else 1
    if args.profile_case == "adjoint":
        # the laser slab c4 (262,144 electrons): a 40-step tape, checkpoint every 20, and its backward
        sim = pic.Simulation.from_workload(W.config("c4"))
        t0 = time.perf_counter()
        sim.tape_forward(40, 20)
        sim.tape_backward(1.0)
        torch.cuda.synchronize()
        print(json.dumps({"profile_case": "adjoint", "workload": "c4 laser slab, 40-step tape, checkpoint 20",
                          "seconds": time.perf_counter() - t0}))
        sim.close()
        return 0
    if args.profile_case in ("fp64", "tsc"):
        wl, prec = W.config("c2"), "fp64"
    elif args.profile_case == "fields":
        # the laser ramp's grid (256 x 128 x 128, x absorbing: the field arrays, 0.4 GB, exceed L2)
        # with one electron per cell, for the field kernels
        wl = W.uniform_plasma((256, 128, 128), 1, 0.05, 0.1, seed=1242, steps=args.steps, name="fields-256")
        wl.bc = (1, 0, 0)
        prec = "mixed"
    else:
        wl, prec = W.uniform_plasma((96, 96, 96), 32, 0.05, 0.1, seed=1241, steps=args.steps, name="mixed-96"), "mixed"
    r = time_gpu(torch, pic, wl, prec, args.steps, args.warmup, form_factor=ff)
    print(json.dumps({"profile_case": args.profile_case, "workload": _workload_desc(wl, prec),
                      "particle_steps_per_s": r["npart"] * args.steps / (r["ms"] / 1e3),
                      "stage_ms_per_step": {k: round(v, 4) for k, v in r["stage_ms"].items()}}))
    r["sim"].close()
    return 0


def run_gpu(args):
    ws, rank, local = _dist()
    import torch
    torch.cuda.set_device(local)
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    from paper_1608_01009_gb300 import pic, workloads as W
    # every rank its own replica (different seed): weak scaling, no data-path collective
    wl = W.config(args.workload, seed=None if ws == 1 else 1236 + 101 * rank)
    peaks, peak_kind = _peaks()
    hbm_peak = float(peaks.get("hbm_gbs", 6800.0))
    fp64_peak = measure_fp64_peak(pic, local)  # before any timed region
    fp64_tf = fp64_peak["tflops"]

    if ws > 1:
        dist.barrier()
    with ClockSampler(local) as clk:
        r = time_gpu(torch, pic, wl, "fp64", args.steps, args.warmup)
    ms = _barrier_max(torch, r["ms"], ws)
    value = weak_value(r["npart"], ws, args.steps, ms)
    push_ms = r["stage_ms"]["push_deposit"]
    flops = FLOPS_PER_PARTICLE * r["npart"]
    nsorts = max(0, (r["launches"] - 5 * args.steps) // 5)  # each followed by a launch that moves the records
    bytes_ = (BYTES_PER_PARTICLE["fp64"] * (args.steps - nsorts) + BYTES_PER_PARTICLE["fp64_after_sort"] * nsorts) \
        / args.steps * r["npart"]
    achieved_tf = flops / (push_ms / 1e3) / 1e12
    achieved_gbs = bytes_ / (push_ms / 1e3) / 1e9
    out = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True, "scaling": "weak",
           "vs_baseline": None, "dtype": "f64", "data": "synthetic (seeded)",
           "config": {"workload": _workload_desc(wl, "FP64"), "supercell": 4,
                      "sort_schedule": "every step (the FP64 default, sort_interval 0)",
                      "l2": "inputs larger than L2 (particle store %.0f MB)" % (64 * r["npart"] / 1e6),
                      "parallelism": "replicas x%d" % ws if ws > 1 else "single GPU"},
           "roofline": {"bound": "alu", "achieved": achieved_tf, "peak": fp64_tf, "unit": "TFLOP/s",
                        "frac": achieved_tf / fp64_tf, "traffic": _traffic("fp64"),
                        "kernel": "k_push<double,4> (gather + Boris + move + VB deposit)",
                        "peak_kind": "measured", "peak_source": "FP64 FMA probe in this run (fp64_peak)",
                        "frac_of_nominal": achieved_tf / FP64_NOMINAL_TFLOPS, "nominal": FP64_NOMINAL_TFLOPS,
                        "per_launch_ms": push_ms, "hbm_achieved_gbs": achieved_gbs,
                        "hbm_frac": achieved_gbs / hbm_peak, "hbm_peak_kind": peak_kind},
           "fp64_peak": fp64_peak,
           "stage_ms_per_step": {k: round(v, 4) for k, v in r["stage_ms"].items()},
           "gpu_launches": r["launches"], "clocks": clk.summary()}
    if not args.no_e2e:
        # up to 30 steps: the first step's copy cannot overlap (pipeline fill)
        e2e = time_e2e(torch, pic, wl, r["sim"], max(3, min(args.steps, 30)))
        sec = _barrier_max(torch, e2e["seconds"], ws)
        out["e2e"] = {"value": e2e["npart"] * ws * e2e["steps"] / sec, "unit": UNIT,
                      "h2d_bytes_per_step": e2e["h2d"], "d2h_bytes_per_step": e2e["d2h"],
                      "how": "per step: pic_set_fields from pinned host buffers, "
                             "pic_set_particles_uploaded (this step's set) + pic_upload_particles "
                             "(the next step's set from pinned host buffers, copied while this step "
                             "runs), pic_step(1), pic_energy (16 B back)"}
    r["sim"].close()
    if not args.no_mixed:
        wl3 = W.config("c3", seed=None if ws == 1 else 1237 + 101 * rank)
        with ClockSampler(local) as clk3:
            r3 = time_gpu(torch, pic, wl3, "mixed", args.steps, args.warmup)
        ms3 = _barrier_max(torch, r3["ms"], ws)
        pm = r3["stage_ms"]["push_deposit"]
        # launches right after a sort (the 5 sort kernels per sort come on top of 5 per step)
        nsorts = max(0, (r3["launches"] - 5 * args.steps) // 5)
        per_launch_b = (BYTES_PER_PARTICLE["mixed"] * (args.steps - nsorts) +
                        BYTES_PER_PARTICLE["mixed_after_sort"] * nsorts) / args.steps
        gbs = per_launch_b * r3["npart"] / (pm / 1e3) / 1e9
        out["mixed"] = {"value": r3["npart"] * ws * args.steps / (ms3 / 1e3), "unit": UNIT, "dtype": "f32/f64",
                        "config": {"workload": _workload_desc(wl3, "mixed FP32/FP64"),
                                   "sort_schedule": "displacement-bounded (the mixed default, sort_interval 0)"},
                        "ms_per_step": ms3 / args.steps,
                        "roofline": {"bound": "hbm", "achieved": gbs, "peak": hbm_peak, "unit": "GB/s",
                                     "frac": gbs / hbm_peak, "traffic": _traffic("mixed"),
                                     "kernel": "k_push_g<4> (mixed gather + Boris + move + VB deposit)",
                                     "per_launch_ms": pm, "bytes_per_particle": per_launch_b,
                                     "launches_after_sort": nsorts, "launches": args.steps},
                        "stage_ms_per_step": {k: round(v, 4) for k, v in r3["stage_ms"].items()},
                        "gpu_launches": r3["launches"], "clocks": clk3.summary()}
        r3["sim"].close()
        # the FP64 path on the same workload and seed, timed the same way
        r3d = time_gpu(torch, pic, wl3, "fp64", args.steps, args.warmup)
        ms3d = _barrier_max(torch, r3d["ms"], ws)
        v3d = r3d["npart"] * ws * args.steps / (ms3d / 1e3)
        pd = r3d["stage_ms"]["push_deposit"]
        out["mixed"]["fp64_same_workload"] = {
            "value": v3d, "ms_per_step": ms3d / args.steps, "mixed_speedup": out["mixed"]["value"] / v3d,
            "roofline": {"bound": "alu", "achieved": FLOPS_PER_PARTICLE * r3d["npart"] / (pd / 1e3) / 1e12,
                         "peak": fp64_tf, "unit": "TFLOP/s", "kernel": "k_push<double,4>", "per_launch_ms": pd},
            "stage_ms_per_step": {k: round(v, 4) for k, v in r3d["stage_ms"].items()}}
        r3d["sim"].close()
        if not args.no_error:
            out["mixed"]["error_vs_fp64"] = mixed_vs_fp64(torch, pic, wl3)
    if not args.no_tsc:
        # second-order form factor + Esirkepov current on the same FP64 workload
        rt = time_gpu(torch, pic, wl, "fp64", args.steps, args.warmup, form_factor=2)
        mst = _barrier_max(torch, rt["ms"], ws)
        pt = rt["stage_ms"]["push_deposit"]
        tf = FLOPS_PER_PARTICLE_TSC * rt["npart"] / (pt / 1e3) / 1e12
        out["tsc"] = {"value": weak_value(rt["npart"], ws, args.steps, mst), "unit": UNIT, "dtype": "f64",
                      "config": {"workload": _workload_desc(wl, "FP64"), "form_factor": "TSC + Esirkepov"},
                      "ms_per_step": mst / args.steps,
                      "roofline": {"bound": "alu", "achieved": tf, "peak": fp64_tf, "unit": "TFLOP/s",
                                   "frac": tf / fp64_tf, "peak_kind": "measured", "traffic": _traffic("tsc"),
                                   "kernel": "k_push_tsc", "per_launch_ms": pt},
                      "stage_ms_per_step": {k: round(v, 4) for k, v in rt["stage_ms"].items()},
                      "gpu_launches": rt["launches"]}
        rt["sim"].close()
    if not args.no_adjoint:
        out["adjoint"] = time_adjoint(torch, pic, W)
    if not args.no_laser_ramp:
        out["laser_ramp"] = time_laser_ramp(torch, pic, W)
    if not args.no_sweep:
        # supercell edge S (the paper's Tables 5-6 study): particle-steps/s per S
        sweep = {}
        wl3s = locals().get("wl3")
        for label, wls, prec, sizes in (("fp64 c2", wl, "fp64", (2, 4, 8)), ("fp64 r", W.config("r"), "fp64", (2, 4, 8)),
                                        ("mixed c3", wl3s, "mixed", (4, 8))):
            wlx = wls if wls is not None else W.config("c3")
            row = {}
            for S in sizes:
                rs = time_gpu(torch, pic, wlx, prec, 20, 3, with_timing=False, supercell=S)
                row["S=%d" % S] = rs["npart"] * 20 / (rs["ms"] / 1e3)
                rs["sim"].close()
            sweep[label] = row
        out["supercell_sweep"] = sweep
    if not args.no_replica:
        wlr = W.config("r")
        rr = time_gpu(torch, pic, wlr, "fp64", args.steps, args.warmup, with_timing=False)
        vr = rr["npart"] * args.steps / (rr["ms"] / 1e3)
        out["paper_replica"] = {"workload": _workload_desc(wlr, "FP64"), "value": vr, "unit": UNIT,
                                "paper_knl_value": 3.2e9 / 10.75,
                                "vs_paper_knl": vr / (3.2e9 / 10.75),
                                "note": "paper: 40^3 x 50 ppc x 1000 steps in 10.75 s on Xeon Phi 7250 "
                                        "(Table 6); context, other hardware"}
        rr["sim"].close()
    if rank == 0 and not args.no_cpu:
        rate, npart, dt, nth = cpu_oracle_rate(wl, 1, 1, threads=True)
        rate1, npart1, dt1, _ = cpu_oracle_rate(wl, 1, 1, threads=False)
        out["cpu_baseline"] = {"value": rate, "unit": UNIT, "cores": nth, "kind": "oracle",
                               "sample": "one whole oracle step of the full workload (%d particles, %.2f s), "
                                         "particles pushed on %d host threads (the oracle's threaded timing "
                                         "build; field solve serial)" % (npart, dt, nth),
                               "single_core": {"value": rate1, "unit": UNIT, "cores": 1,
                                               "sample": "the same step, serial build (%.1f s)" % dt1}}
    if ws > 1:
        dist.barrier()
        dist.destroy_process_group()
    if rank == 0:
        print(json.dumps(out))
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=100)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--workload", default="c2")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-mixed", action="store_true")
    ap.add_argument("--no-replica", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-adjoint", action="store_true")
    ap.add_argument("--no-sweep", action="store_true")
    ap.add_argument("--no-tsc", action="store_true")
    ap.add_argument("--no-error", action="store_true", help="skip the mixed-vs-FP64 error runs on c3")
    ap.add_argument("--no-laser-ramp", action="store_true", help="skip the c5 laser-plasma run and its adjoint")
    ap.add_argument("--laser-ramp", action="store_true",
                    help="run only the 134 M-particle laser-plasma workload with its 50-step adjoint")
    ap.add_argument("--profile-case", choices=["fp64", "mixed", "tsc", "adjoint", "fields"], default=None,
                    help="run only one reduced case for ncu captures (a few GB on the device): "
                         "fp64 = the 64^3 x 50 FP64 plasma, mixed = a 96^3 x 32 mixed plasma, "
                         "tsc = the 64^3 x 50 plasma with the second-order form factor, "
                         "adjoint = a 40-step tape of the laser slab and its backward")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        return run_reference(args)
    if args.laser_ramp:
        return run_laser_ramp(args)
    if args.profile_case:
        return run_profile_case(args)
    return run_gpu(args)


if __name__ == "__main__":
    sys.exit(main())
