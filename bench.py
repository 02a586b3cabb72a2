#!/usr/bin/env python
"""Throughput of the TDSLDA step (AB4AM5, Alg. 2) on B300.

Metric: state-site updates per second = states x lattice sites x steps / time,
one update being one quasiparticle state at one lattice site advanced by one
full predictor + corrector step. The workload is a 32^3 periodic lattice in a
harmonic trap V = 1/2 w^2 r^2 (w = 0.05) with 32768 quasiparticle states.

Default run (N = 1): the mixed-precision step (complex float states and FFTs,
double reductions) is timed with CUDA events on the library's stream over K
steps after W warm-up steps; the plain FP64 step on the same states is timed
the same way and reported beside it, with the relative density difference
between the two. Per-kernel CUDA events give the stage-X kernel's duration for
the roofline. The end-to-end number goes through the public API with pinned
host buffers: load_states (host -> device), start, K steps each followed by a
density read (device -> host) and a final get_states (device -> host).
`--impl reference` times the CPU oracle on the host cores instead.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "TD step state-site updates/s, mixed FP32 vs plain FP64 at ≤1e-5 rel density err"
UNIT = "state-site updates/s"
FALLBACK_HBM_GBS = 6400.0
FP64_PEAK_TFLOPS = 1.25   # nominal B300 FP64 rate (SM count x FP64 units x clock)
RHO_SIGMA = 1.0 / (6 * math.pi ** 2)


def _omega(text):
    v = [float(x) for x in text.split(",")]
    return v[0] if len(v) == 1 else tuple(v)


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=10)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", default="ours", choices=["ours", "reference"])
    p.add_argument("--shape", default="32,32,32")
    p.add_argument("--nstates", type=int, default=32768)
    p.add_argument("--omega", type=_omega, default=0.05,
                   help="trap frequency, or wx,wy,wz for an anisotropic trap")
    p.add_argument("--dt", type=float, default=0.007)
    p.add_argument("--precision", default="both", choices=["both", "mixed", "fp64"])
    p.add_argument("--no-e2e", action="store_true")
    p.add_argument("--no-cpu", action="store_true")
    p.add_argument("--cpu-seconds", type=float, default=15.0)
    p.add_argument("--batched", action="store_true",
                   help="also time the batched workload: 64 cubic boxes 12^3..24^3, BdG, one graph per 4 steps")
    p.add_argument("--integrator", default="AB4AM5", choices=["AB4AM5", "AB3AM4", "AB5AM5"],
                   help="predictor-corrector scheme of Sec. 3.3 (AB4AM5 is Alg. 2)")
    p.add_argument("--init", default="quench", choices=["quench", "scf"],
                   help="quench: uniform plane-wave states in the trap (default); scf: states of a static "
                        "self-consistent solve with nstates = M (slow: minutes at 32^3)")
    p.add_argument("--scf-n", type=float, default=200.0, help="particle-number target per spin for --init scf")
    p.add_argument("--scf-iters", type=int, default=40)
    p.add_argument("--scf-fp32-iters", type=int, default=30)
    p.add_argument("--friction", default=None,
                   help="alpha,beta,gamma of the quantum-friction terms (Sec. 5.2.4), e.g. 5,5,0")
    p.add_argument("--streams", type=int, default=4, help="forked streams of the batched workload")
    p.add_argument("--A", type=float, default=1.0,
                   help="inverse effective mass of the SLDA functional; != 1 adds the current terms "
                        "(1.094 = A_a(0) of the ASLDA functional)")
    p.add_argument("--stationary", action="store_true",
                   help="stationary start instead of the Taylor start (short profiling runs)")
    return p.parse_args()


def dist_env():
    return int(os.environ.get("RANK", 0)), int(os.environ.get("WORLD_SIZE", 1)), int(os.environ.get("LOCAL_RANK", 0))


def max_over_ranks(x: float, world: int, device) -> float:
    """The largest of the ranks' values of x (every rank gets it); x itself on one rank."""
    if world == 1:
        return float(x)
    import torch
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
    return float(t.item())


def job_rate(units_per_rank: float, world: int, seconds: float) -> float:
    """Whole-job throughput of independent replicas: every rank processes
    units_per_rank, and the job takes as long as its slowest rank."""
    return world * units_per_rank / seconds


def stage_source_hash() -> str:
    """git blob hash of the stage-kernel source (computed without git)."""
    import hashlib
    data = open(os.path.join(ROOT, "paper_2602_08982_b300", "csrc", "stage.cuh"), "rb").read()
    return hashlib.sha1(b"blob %d\0" % len(data) + data).hexdigest()


def profiled_traffic():
    """DRAM bytes per state-site of stage X from the committed ncu summary, if
    that capture was taken on the current stage-kernel source; else None."""
    path = os.path.join(ROOT, "profiles", "stage_x_traffic.txt")
    if not os.path.exists(path):
        return None
    kv = dict(line.split("=", 1) for line in open(path).read().split() if "=" in line)
    if kv.get("stage_cuh_blob") != stage_source_hash():
        return None
    return float(kv["mixed_bytes_per_state_site"])


def measured_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        d = json.load(open(path))
        return float(d["hbm_gbs"]), "of measured"
    return FALLBACK_HBM_GBS, "of fallback"


# ------------------------------------------------------------------ clocks
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device: int):
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        try:
            self.p = subprocess.Popen(["nvidia-smi", "-i", str(device), f"--query-gpu={self.FIELDS}",
                                       "--format=csv,noheader,nounits", "-lms", "200"],
                                      stdout=self.f, stderr=subprocess.DEVNULL)
        except OSError:
            self.p = None

    def stop(self) -> dict:
        if self.p is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.p.terminate()
        self.p.wait()
        self.f.flush()
        rows = [r.split(",") for r in open(self.f.name).read().strip().splitlines() if r.strip()]
        os.unlink(self.f.name)
        sm = [float(r[1]) for r in rows if len(r) >= 9 and r[1].strip().replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if len(r) >= 9 and r[2].strip().replace(".", "").isdigit()]
        names = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")
        reasons = sorted({names[i] for r in rows if len(r) >= 9 for i in range(4) if r[5 + i].strip() == "Active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows)}


# ------------------------------------------------------------------ GPU arms
def make_box(W, prec, shape, nstates, omega, stream, scheme="AB4AM5", mu=None, A=1.0):
    """A != 1: the SLDA functional with its current terms (same B, C, mu and
    uniform seed as the A = 1 workload)."""
    from paper_2602_08982_b300 import inputs
    u = W.uniform_solve(shape, kind=W.SLDA_A1, B=W.B_SLDA, rho_sigma=RHO_SIGMA, delta0=0.25)
    ctx = W.Context(prec, stream=stream)
    ctx.set_integrator(scheme)
    box = ctx.add_box(shape, kind=W.SLDA if A != 1.0 else W.SLDA_A1, B=W.B_SLDA, C=u["C"],
                      mu=u["mu"] if mu is None else mu, A=A, nstates=nstates)
    ctx.set_vext(box, inputs.harmonic_trap(shape, omega))
    return ctx, box, u


HISTORY_READS = {"AB3AM4": 2, "AB4AM5": 3, "AB5AM5": 4}


def stage_x_algorithmic(prec, shape, scheme="AB4AM5", cur=False):
    """Algorithmic traffic / work of one stage-X launch per state-site.
    Bytes: reads phi and the history (AB4AM5: f_{k-2}, f_{k-3}, f_{k-4});
    writes f_{k-1}, phi_p, c (AB4AM5: 7 state passes of two complex numbers);
    with the current terms (A != 1) it also reads the current term of H phi.
    Flops (FP64 path): forward and inverse 3D FFT of both components at
    5 M log2 M each, plus the pointwise H, <H>_n, f, predictor, corrector
    partial, norm and scaling (128)."""
    M = shape[0] * shape[1] * shape[2]
    csize = 8 if prec == 1 else 16
    bytes_per = (1 + HISTORY_READS[scheme] + 3 + (1 if cur else 0)) * 2 * csize
    flops_per = 2 * 2 * 5 * math.log2(M) + 128
    return bytes_per, flops_per


SCF_START = {}


def scf_start(W, args, shape):
    """Trapped start from a static self-consistent solve (Alg. 1) of the
    workload's SLDA system with a particle-number target (Eq. update-mu),
    modified Broyden mixing and single-precision leading iterations; the
    states are kept in host memory for every arm."""
    if "phi" in SCF_START:
        return SCF_START
    from paper_2602_08982_b300 import inputs
    M = shape[0] * shape[1] * shape[2]
    u = W.uniform_solve(shape, kind=W.SLDA_A1, B=W.B_SLDA, rho_sigma=RHO_SIGMA, delta0=0.25)
    ctx = W.Context(W.FP64)
    b = ctx.add_box(shape, kind=W.SLDA_A1, B=W.B_SLDA, C=u["C"], mu=u["mu"], nstates=M)
    ctx.set_vext(b, inputs.harmonic_trap(shape, args.omega))
    t0 = time.perf_counter()
    res, _ = ctx.static_solve(b, np.full(M, u["U"]), np.full(M, u["delta"]), method="broyden", mixing=0.5,
                              eps_energy=1e-6, max_iters=args.scf_iters, n_target=args.scf_n, a_mu=0.5,
                              eps_npart=1e-3, fp32_iters=args.scf_fp32_iters)
    sec = time.perf_counter() - t0
    SCF_START["phi"] = ctx.get_states(b)
    ctx.close()
    SCF_START["info"] = {"iters": res["iters"], "converged": res["converged"], "mu": res["mu"],
                         "n_sigma": res["n_sigma"], "max_rel_change": res["max_rel_change"], "seconds": sec,
                         "fp32_iters": args.scf_fp32_iters, "n_target": args.scf_n}
    return SCF_START


def run_arm(W, torch, prec, args, shape, rank, world, dev):
    stream = torch.cuda.current_stream()
    if args.init == "scf":
        start = scf_start(W, args, shape)
        ctx, box, u = make_box(W, prec, shape, args.nstates, args.omega, stream.cuda_stream, args.integrator,
                               mu=start["info"]["mu"], A=args.A)
        ctx.load_states(box, start["phi"])
        ctx.start(True, args.dt)               # a static solution: stationary start
    else:
        ctx, box, u = make_box(W, prec, shape, args.nstates, args.omega, stream.cuda_stream, args.integrator,
                               A=args.A)
        ctx.fill_uniform_states(box, u["mu_eff"], u["delta"])
        if args.friction:
            fa, fb, fg = (float(x) for x in args.friction.split(","))
            M = shape[0] * shape[1] * shape[2]
            ctx.set_friction(box, fa, fb, fg, RHO_SIGMA, 2.0 * RHO_SIGMA * M)
        ctx.start(args.stationary, args.dt)  # Taylor start: the trapped plane waves are not stationary
    variant = ctx.get_variant(box)
    if args.warmup:
        ctx.step(args.dt, args.warmup)
    torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    ctx.set_profiling(True)
    clocks = ClockSampler(dev)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    l0 = ctx.launch_count()
    e0.record(stream)
    ctx.step(args.dt, args.steps)
    e1.record(stream)
    torch.cuda.synchronize()
    launches = ctx.launch_count() - l0
    ms = e0.elapsed_time(e1)
    ck = clocks.stop()
    # "aux": the current-term passes of A != 1 (nothing in the A = 1 step)
    kt = {k: ctx.get_kernel_time(k) for k in ("stage_x", "stage_y", "density", "potentials", "aux")}
    ms = max_over_ranks(ms, world, "cuda")
    if world > 1:
        torch.distributed.barrier()
    rho, nu = ctx.get_densities(box)
    ctx.close()
    M = shape[0] * shape[1] * shape[2]
    units = float(args.nstates) * M * args.steps
    value = job_rate(units, world, ms * 1e-3)
    bx, fx = stage_x_algorithmic(prec, shape, args.integrator, args.A != 1.0)
    x_ms, x_n = kt["stage_x"]
    x_avg = x_ms / max(x_n, 1)
    per_launch = float(args.nstates) * M
    if prec == 1:
        peak, which = measured_peaks()
        achieved = bx * per_launch / (x_avg * 1e-3) / 1e9
        tb = profiled_traffic() if args.integrator == "AB4AM5" and args.A == 1.0 else None  # captured on A = 1
        roof = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                "traffic": None if tb is None else tb * per_launch,
                "kernel": "stage_x (f + AB4 predictor + AM5 partial + normalisation)",
                "peak_source": which, "algorithmic_bytes_per_state_site": bx}
    else:
        achieved = fx * per_launch / (x_avg * 1e-3) / 1e12
        roof = {"bound": "alu", "achieved": achieved, "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s",
                "frac": achieved / FP64_PEAK_TFLOPS, "traffic": None,
                "kernel": "stage_x (f + AB4 predictor + AM5 partial + normalisation), FP64",
                "peak_source": "nominal FP64 rate", "algorithmic_flops_per_state_site": fx}
    share = {k: kt[k][0] / ms for k in kt}
    roof["launch_variant"] = variant
    return dict(value=value, ms_per_step=ms / args.steps, roofline=roof, clocks=ck, launches=launches,
                kernel_ms=kt, kernel_share=share, rho=rho, nu=nu)


def run_e2e(W, torch, args, shape, world):
    """Mixed path end to end through the ABI with pinned host buffers: the
    states travel as complex64, the precision the mixed path stores them in."""
    stream = torch.cuda.current_stream()
    ctx, box, u = make_box(W, W.MIXED, shape, args.nstates, args.omega, stream.cuda_stream, args.integrator,
                           A=args.A)
    ctx.fill_uniform_states(box, u["mu_eff"], u["delta"])
    M = shape[0] * shape[1] * shape[2]
    host = torch.empty((args.nstates, 2, M), dtype=torch.complex64, pin_memory=True)
    host_np = host.numpy()
    ctx.get_states_f32(box, host_np)  # untimed: the job's input now lives in pinned host memory
    ctx.close()
    torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    t0 = time.perf_counter()
    ctx, box, _ = make_box(W, W.MIXED, shape, args.nstates, args.omega, stream.cuda_stream, args.integrator,
                           A=args.A)
    ctx.load_states_f32(box, host_np)
    ctx.start(False, args.dt)
    for _ in range(args.steps):
        ctx.step(args.dt, 1)
        r, n = ctx.get_densities(box)
    ctx.get_states_f32(box, host_np)
    torch.cuda.synchronize()
    sec = time.perf_counter() - t0
    ctx.close()
    sec = max_over_ranks(sec, world, "cuda")
    units = float(args.nstates) * M * args.steps
    nbytes = host.numel() * 8
    del host
    return {"value": job_rate(units, world, sec), "unit": UNIT,
            "h2d_bytes_per_step": nbytes / args.steps,
            "d2h_bytes_per_step": (nbytes + args.steps * 24 * M) / args.steps,
            "includes": "box creation, load_states_f32 from pinned host (complex64), Taylor start, K steps each "
                        "with a density read, final get_states_f32",
            "seconds": sec}


def batched_boxes(max_gb=240.0, first_seed=4):
    """Box sides for the batched workload: 64 cubic boxes drawn from
    {12, 16, 18, 20, 24}; a draw whose five complex64 buffers exceed max_gb is
    rejected and redrawn with the next seed."""
    from paper_2602_08982_b300 import inputs
    seed = first_seed
    while True:
        sides = inputs.draw_box_sides(64, seed)
        if sum(n ** 6 for n in sides) * 80 / 1e9 <= max_gb:
            return seed, sides
        seed += 1


def run_batched(W, torch, args):
    from paper_2602_08982_b300 import inputs
    seed, sides = batched_boxes()
    inv_kfa = inputs.draw_inv_kfa(64, 1004)
    stream = torch.cuda.current_stream()
    ctx = W.Context(W.MIXED, stream=stream.cuda_stream)
    units = 0.0
    for i, (n, ik) in enumerate(zip(sides, inv_kfa)):
        shape = (n, n, n)
        ia = float(ik) / (4 * math.pi)
        u = W.uniform_solve(shape, kind=W.BDG, inv_4pi_a=ia, rho_sigma=RHO_SIGMA)
        b = ctx.add_box(shape, kind=W.BDG, inv_4pi_a=ia, mu=u["mu"], nstates=n ** 3)
        ctx.set_dext(b, inputs.pairing_kick(shape, 5000 + i, 1e-3 * u["delta"]))
        ctx.fill_uniform_states(b, u["mu_eff"], u["delta"])
        units += float(n ** 3) ** 2
    ctx.set_graph(True, args.streams)
    ctx.start(False, args.dt)
    steps = max(4, 4 * (args.steps // 4))
    ctx.step(args.dt, 4)                      # warm-up (also captures the graphs)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    l0 = ctx.launch_count()
    e0.record(stream)
    ctx.step(args.dt, steps)
    e1.record(stream)
    torch.cuda.synchronize()
    launches = ctx.launch_count() - l0
    ms = e0.elapsed_time(e1)
    ctx.close()
    value = units * steps / (ms * 1e-3)
    peak, which = measured_peaks()
    step_gbs = 160.0 * units / (ms / steps * 1e-3) / 1e9
    return {"value": value, "unit": UNIT, "ms_per_step": ms / steps, "steps": steps, "boxes": 64,
            "gpu_launches": launches,
            "box_sides_seed": seed, "box_sides": sides, "state_sites_per_step": units,
            "config": "64 cubic boxes 12^3..24^3 (all states), BdG 1/(kF a) uniform in [-1, 1), 1e-3 pairing "
                      f"kick per box, complex64, boxes on {args.streams} forked streams, 4 steps per CUDA graph",
            "step_roofline": {"bound": "hbm", "achieved": step_gbs, "peak": peak, "unit": "GB/s",
                              "frac": step_gbs / peak, "peak_source": which,
                              "algorithmic_bytes_per_state_site": 160, "scope": "whole step (10 state passes)"}}


# ------------------------------------------------------------------ oracle (CPU)
def oracle_sample(shape, omega, n, A=1.0):
    """CPU-oracle system for the workload's lattice and trap, with n of its
    uniform plane-wave states (seeded choice of momenta)."""
    from oracle import tdslda as o
    from paper_2602_08982_b300 import inputs
    lat = o.Lattice(*shape)
    seed = o.uniform_slda_seed(lat, 0.25, RHO_SIGMA)
    fn = o.Functional("slda", B=o.B_SLDA, C=seed.C, mu=seed.mu, A=float(A))
    r = inputs.uniform01(77, lat.M)
    idx = np.sort(np.argsort(r)[:n])
    kx, ky, kz = (lat.kaxis(a) for a in range(3))
    ix, rem = np.divmod(idx, lat.ny * lat.nz)
    iy, iz = np.divmod(rem, lat.nz)
    e = [np.exp(1j * np.outer(k[i], np.arange(nn))) for k, i, nn in ((kx, ix, lat.nx), (ky, iy, lat.ny),
                                                                      (kz, iz, lat.nz))]
    pw = np.einsum("ni,nj,nk->nijk", *e).reshape(n, lat.M) / np.sqrt(lat.volume)
    Uk, Vk, _ = o.bcs_amplitudes(0.5 * (kx[ix] ** 2 + ky[iy] ** 2 + kz[iz] ** 2) - seed.mu_eff, seed.delta)
    phi = np.stack([Uk[:, None] * pw, Vk[:, None] * pw], axis=1)
    return o, o.TDSystem(lat, fn, vext=inputs.harmonic_trap(lat.shape, omega)), phi, lat


def oracle_stepper(o, scheme):
    """(start, step) of the oracle for the scheme: Alg. 2 itself for AB4AM5."""
    if scheme == "AB4AM5":
        return (lambda sysm, phi, dt: o.start(sysm, phi, dt, stationary=True)), o.ab4am5_step
    return ((lambda sysm, phi, dt: o.start_scheme(sysm, phi, dt, True, scheme)),
            (lambda sysm, st, dt: o.abm_step(sysm, st, dt, scheme)))


def cpu_oracle_rate(shape, omega, dt, seconds, max_states=2048, scheme="AB4AM5", A=1.0):
    """The oracle as it stands, on a bounded sample of the workload: the same
    lattice and trap with a subset of the uniform plane-wave states, timed over
    whole ABM steps after a stationary start."""
    max_states = min(max_states, shape[0] * shape[1] * shape[2])
    n = min(64, max_states)
    while True:
        o, sysm, phi, lat = oracle_sample(shape, omega, n, A)
        start, step = oracle_stepper(o, scheme)
        st = start(sysm, phi, dt)
        t0 = time.perf_counter()
        st = step(sysm, st, dt)
        one = time.perf_counter() - t0
        if one * 4 > seconds or n >= max_states:
            break
        n = min(max_states, n * 2)
    k = max(1, int(seconds / max(one, 1e-3)))
    t0 = time.perf_counter()
    for _ in range(k):
        st = step(sysm, st, dt)
    sec = time.perf_counter() - t0
    return {"value": n * lat.M * k / sec, "unit": UNIT, "cores": os.cpu_count(), "kind": "oracle", "n": n,
            "sample": f"{n} of the workload's states on the same {shape[0]}x{shape[1]}x{shape[2]} trap, {k} {scheme} "
                      f"steps after a stationary start, {sec:.1f} s"}


def reference_arm(args, shape):
    rank, world, _ = dist_env()
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("gloo")
        if rank != 0:
            dist.barrier()
            return
    # each step: one oracle step of the scheme over a bounded sample of the
    # states, sized so that one step takes about a second
    n = cpu_oracle_rate(shape, args.omega, args.dt, args.cpu_seconds / 4, scheme=args.integrator, A=args.A)["n"]
    o, sysm, phi, lat = oracle_sample(shape, args.omega, n, args.A)
    start, step = oracle_stepper(o, args.integrator)
    st = start(sysm, phi, args.dt)
    for _ in range(args.warmup):
        st = step(sysm, st, args.dt)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        st = step(sysm, st, args.dt)
    sec = time.perf_counter() - t0
    value = n * lat.M * args.steps / sec
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1e3 * sec / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic", "impl": "reference",
            "config": workload_config(args, shape, "fp64 oracle (CPU)"),
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": os.cpu_count(), "kind": "oracle",
                             "sample": f"{n} states of the workload per step, {args.steps} steps, {sec:.1f} s"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def workload_config(args, shape, precision):
    return {"workload": f"TDSLDA {args.integrator} step, {shape[0]}x{shape[1]}x{shape[2]} periodic lattice, harmonic trap "
                        f"w={args.omega}, {args.nstates} quasiparticle states",
            "lattice": list(shape), "nstates": args.nstates, "trap_omega": args.omega, "dt": args.dt,
            "functional": (f"SLDA with current terms (A={args.A}), " if args.A != 1.0 else "SLDA (A=1), ")
                          + "B=B_ASLDA(0), C from the uniform 16^3-style seed on this lattice",
            "init": ("states of a static self-consistent solve (fixed N, Broyden), stationary start"
                     if args.init == "scf" else
                     "uniform plane-wave BCS states (Delta0 = 0.5 eF) quenched into the trap, Taylor start"),
            "friction": args.friction, "precision": precision, "l2": "inputs larger than L2 (state buffers >> 126 MB), no flush needed",
            "parallelism": "replicas" if args.gpus > 1 else "single GPU"}


def main():
    args = parse()
    shape = tuple(int(v) for v in args.shape.split(","))
    if args.impl == "reference":
        reference_arm(args, shape)
        return
    rank, world, local = dist_env()
    import torch
    if world > 1:
        torch.distributed.init_process_group("nccl")
    torch.cuda.set_device(local)
    from paper_2602_08982_b300 import wslda as W

    cpu = None
    if rank == 0 and not args.no_cpu and world == 1:
        cpu = cpu_oracle_rate(shape, args.omega, args.dt, args.cpu_seconds, scheme=args.integrator, A=args.A)
    arms = {}
    if args.precision in ("both", "mixed"):
        arms["mixed"] = run_arm(W, torch, W.MIXED, args, shape, rank, world, local)
    if args.precision in ("both", "fp64"):
        arms["fp64"] = run_arm(W, torch, W.FP64, args, shape, rank, world, local)
    e2e = None if args.no_e2e else run_e2e(W, torch, args, shape, world)
    batched = run_batched(W, torch, args) if args.batched else None
    main_arm = arms.get("mixed") or arms["fp64"]
    line = {"metric": METRIC, "value": main_arm["value"], "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": main_arm["ms_per_step"], "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32" if "mixed" in arms else "f64",
            "data": "synthetic",
            "config": workload_config(args, shape, "mixed: complex64 states and FFTs, f64 accumulation"
                                      if "mixed" in arms else "fp64"),
            "roofline": main_arm["roofline"], "gpu_launches": main_arm["launches"], "clocks": main_arm["clocks"],
            "kernel_share": main_arm["kernel_share"]}
    if "fp64" in arms and "mixed" in arms:
        a = arms["fp64"]
        line["fp64"] = {"value": a["value"], "ms_per_step": a["ms_per_step"], "roofline": a["roofline"],
                        "gpu_launches": a["launches"], "clocks": a["clocks"], "kernel_share": a["kernel_share"]}
        m = arms["mixed"]
        line["mixed_vs_fp64"] = {
            "rel_density_err_rho": float(np.abs(m["rho"] - a["rho"]).max() / np.abs(a["rho"]).max()),
            "rel_density_err_nu": float(np.abs(m["nu"] - a["nu"]).max() / np.abs(a["nu"]).max()),
            "after_steps": 3 + args.warmup + args.steps}
    if e2e:
        line["e2e"] = e2e
    if "info" in SCF_START:
        line["scf_start"] = SCF_START["info"]
    if batched:
        line["batched"] = batched
    if cpu:
        line["cpu_baseline"] = cpu
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        torch.distributed.barrier()
        torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
