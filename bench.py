#!/usr/bin/env python
"""Throughput of the TDSLDA step (AB4AM5, Alg. 2) on B300.

Metric: state-site updates per second = states x lattice sites x steps / time,
one update being one quasiparticle state at one lattice site advanced by one
full predictor + corrector step.

Default run (N = 1):
  * value: the mixed-precision step (complex float states and FFTs, double
    reductions) on the elongated-trap workload: a 24 x 24 x 96 lattice in a
    harmonic trap w = (0.064, 0.064, 0.016), all 55296 quasiparticle states,
    a vortex line imprinted on Delta, Taylor start; K steps timed with CUDA
    events on the library's stream after W warm-up steps. Per-kernel CUDA
    events give the stage-X kernel's duration for its roofline; the whole
    step's algorithmic traffic (10 state passes) gives the step roofline.
  * fp64: the plain FP64 step on the 32^3 trap (w = 0.05, 32768 states),
    against the FP64 FMA rate measured on the same GPU in the same run.
  * batched: 64 independent cubic boxes 12^3..24^3 (BdG, all states), four
    steps per CUDA graph, boxes on forked streams.
  * mixed_vs_oracle: the mixed path against the CPU oracle on a bounded
    sample of the main workload (same lattice, trap and vortex, a subset of
    the states as the whole system), after 200 steps (the elongated-trap
    configuration's horizon), with the energy drift.
  * energy_drift: drift of E_tot - mu N over the timed run.
  * cufft: the kinetic-term transforms of one stage (forward 3D FFT of u and
    v, multiply by k^2/2, inverse) done with cuFFT (through torch.fft) on the
    main workload, timed as a comparison only.
  * e2e: the mixed job end to end through the ABI with pinned host buffers:
    load_states_f32 (host -> device), start, K steps each followed by a
    density read (device -> host) and a final get_states_f32.
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
FP64_NOMINAL_TFLOPS = 1.25   # nominal B300 FP64 rate, used only if the measurement fails
RHO_SIGMA = 1.0 / (6 * math.pi ** 2)
# workloads: (lattice, states, trap frequencies, vortex imprint)
WORKLOADS = {
    "elongated": dict(shape=(24, 24, 96), nstates=55296, omega=(0.064, 0.064, 0.016), vortex=True,
                      text="24x24x96 elongated harmonic trap w=(0.064, 0.064, 0.016) with a vortex line "
                           "imprinted on Delta, all 55296 quasiparticle states"),
    "cube32": dict(shape=(32, 32, 32), nstates=32768, omega=0.05, vortex=False,
                   text="32x32x32 periodic lattice, harmonic trap w=0.05, all 32768 quasiparticle states"),
}


def _omega(text):
    v = [float(x) for x in text.split(",")]
    return v[0] if len(v) == 1 else tuple(v)


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=10)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", default="ours", choices=["ours", "reference"])
    p.add_argument("--workload", default="elongated", choices=sorted(WORKLOADS),
                   help="main (mixed) workload; --shape / --nstates / --omega override its fields")
    p.add_argument("--fp64-workload", default="cube32", choices=sorted(WORKLOADS),
                   help="workload of the plain FP64 arm")
    p.add_argument("--shape", default=None)
    p.add_argument("--nstates", type=int, default=None)
    p.add_argument("--omega", type=_omega, default=None,
                   help="trap frequency, or wx,wy,wz for an anisotropic trap")
    p.add_argument("--vortex", type=int, default=None, help="1/0: imprint a vortex line on Delta")
    p.add_argument("--dt", type=float, default=0.007)
    p.add_argument("--precision", default="both", choices=["both", "mixed", "fp64"])
    p.add_argument("--no-e2e", action="store_true")
    p.add_argument("--no-cpu", action="store_true")
    p.add_argument("--cpu-seconds", type=float, default=15.0)
    p.add_argument("--no-batched", action="store_true",
                   help="skip the batched workload (64 cubic boxes 12^3..24^3, BdG, one graph per 4 steps)")
    p.add_argument("--no-oracle-check", action="store_true", help="skip the mixed-vs-oracle sample")
    p.add_argument("--oracle-states", type=int, default=32)
    p.add_argument("--oracle-steps", type=int, default=200)
    p.add_argument("--no-cufft", action="store_true")
    p.add_argument("--integrator", default="AB4AM5", choices=["AB4AM5", "AB3AM4", "AB5AM5"],
                   help="predictor-corrector scheme of Sec. 3.3 (AB4AM5 is Alg. 2)")
    p.add_argument("--init", default="quench", choices=["quench", "scf"],
                   help="quench: uniform plane-wave states in the trap (default); scf: states of a static "
                        "self-consistent solve with nstates = M (slow: minutes at 32^3)")
    p.add_argument("--scf-n", type=float, default=30.0,
                   help="particle-number target per spin for --init scf (30: a Thomas-Fermi radius of about 11 "
                        "sites in the w = 0.05 trap, central kF near 1)")
    p.add_argument("--scf-iters", type=int, default=60)
    p.add_argument("--scf-fp32-iters", type=int, default=30)
    p.add_argument("--friction", default=None,
                   help="alpha,beta,gamma of the quantum-friction terms (Sec. 5.2.4), e.g. 5,5,0")
    p.add_argument("--streams", type=int, default=4, help="forked streams of the batched workload")
    p.add_argument("--A", type=float, default=1.0,
                   help="inverse effective mass of the SLDA functional; != 1 adds the current terms "
                        "(1.094 = A_a(0) of the ASLDA functional)")
    p.add_argument("--stationary", action="store_true",
                   help="stationary start instead of the Taylor start (short profiling runs)")
    p.add_argument("--aslda", action="store_true",
                   help="spin-imbalanced ASLDA (Secs. 2.3-2.4): half the states and their partners (whole "
                        "spectrum), mu_a != mu_b, v weights halved (polarised); FP64 arm off by default")
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


def profiled_traffic(shape):
    """DRAM bytes per state-site of stage X from the committed ncu summary, if
    that capture was taken on the current stage-kernel source and on this
    lattice; else None."""
    path = os.path.join(ROOT, "profiles", "stage_x_traffic.txt")
    if not os.path.exists(path):
        return None
    kv = dict(line.split("=", 1) for line in open(path).read().split() if "=" in line)
    if kv.get("stage_cuh_blob") != stage_source_hash():
        return None
    if kv.get("lattice") != "x".join(str(n) for n in shape):
        return None
    return float(kv["mixed_bytes_per_state_site"])


def host_ram_gb():
    """Physical memory of the host in GB (None where the platform does not say)."""
    try:
        return os.sysconf("SC_PAGE_SIZE") * os.sysconf("SC_PHYS_PAGES") / 1e9
    except (ValueError, OSError, AttributeError):
        return None


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


# ------------------------------------------------------------------ workloads
def resolve(args, name):
    """The workload `name` with the command-line overrides applied."""
    w = dict(WORKLOADS[name])
    if name == args.workload:
        if args.shape:
            w["shape"] = tuple(int(v) for v in args.shape.split(","))
        if args.nstates:
            w["nstates"] = args.nstates
        if args.omega is not None:
            w["omega"] = args.omega
        if args.vortex is not None:
            w["vortex"] = bool(args.vortex)
        if args.shape or args.nstates or args.omega is not None or args.vortex is not None:
            s = w["shape"]
            w["text"] = (f"{s[0]}x{s[1]}x{s[2]} periodic lattice, harmonic trap w={w['omega']}"
                         f"{', vortex line imprinted on Delta' if w['vortex'] else ''}, {w['nstates']} quasiparticle states")
    return w


# ------------------------------------------------------------------ GPU arms
ASLDA_DMU = (0.02, -0.02)  # mu_a - mu, mu_b - mu of the spin-imbalanced workload


def make_box(W, prec, wl, stream, scheme="AB4AM5", mu=None, A=1.0, aslda=False, C=None):
    """A context with one box of the workload (SLDA with the uniform seed's
    B, C, mu unless C or mu are given; A != 1 adds the current terms; aslda:
    the spin-imbalanced functional with C = -11.11 and mu_a, mu_b around the
    seed's mu)."""
    from paper_2602_08982_b300 import inputs
    shape = wl["shape"]
    u = W.uniform_solve(shape, kind=W.SLDA_A1, B=W.B_SLDA, rho_sigma=RHO_SIGMA, delta0=0.25)
    ctx = W.Context(prec, stream=stream)
    ctx.set_integrator(scheme)
    m = u["mu"] if mu is None else mu
    if aslda:
        box = ctx.add_box(shape, kind=W.ASLDA, C=-11.11, mu=m + ASLDA_DMU[0], mu_b=m + ASLDA_DMU[1],
                          nstates=wl["nstates"])
    else:
        box = ctx.add_box(shape, kind=W.SLDA if A != 1.0 else W.SLDA_A1, B=W.B_SLDA, C=u["C"] if C is None else C,
                          mu=m, A=A, nstates=wl["nstates"])
    ctx.set_vext(box, inputs.harmonic_trap(shape, wl["omega"]))
    return ctx, box, u


def fill_workload(W, ctx, box, u, wl, aslda=False):
    """Uniform plane-wave BCS states of the lattice (Delta0 = 0.5 eF), with the
    vortex phase imprinted when the workload has one (reading P2: u e^{i theta/2},
    v e^{-i theta/2}, a gauge transform that keeps the state set and its
    partners complete and orthonormal, so the energy stays conserved). An
    ASLDA box gets half the states and their partners, and the weights of its
    v rows halved (a polarised start)."""
    from paper_2602_08982_b300 import inputs
    ctx.fill_uniform_states(box, u["mu_eff"], u["delta"])
    if aslda:
        n = wl["nstates"]
        h = n // 2
        wm = np.concatenate([np.full(h, 0.5), np.zeros(n - h)])
        wp = np.concatenate([np.zeros(h), np.ones(n - h)])
        ctx.set_weights(box, wm, wp)
    if wl["vortex"]:  # reading P2: u e^{i theta/2}, v e^{-i theta/2}
        half = inputs.vortex_phase(wl["shape"], winding=0.5)
        ctx.imprint_phase(box, 0, half)
        ctx.imprint_phase(box, 1, np.conj(half))


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


def step_algorithmic_bytes(prec, scheme="AB4AM5"):
    """State passes of a whole step per state-site: stage X (1 + D reads, 3
    writes) and stage Y (2 reads, 1 write); AB4AM5: 10 passes, 160 B mixed."""
    csize = 8 if prec == 1 else 16
    return (1 + HISTORY_READS[scheme] + 3 + 3) * 2 * csize


SCF_START = {}


def scf_start(W, args, wl):
    """Trapped start from a static self-consistent solve (Alg. 1) of the
    workload's SLDA system with the printed C (a trapped solve needs C < 0,
    the seed's backed-out C is positive), a particle-number target (Eq.
    update-mu), modified Broyden mixing and single-precision leading
    iterations; the states are kept in host memory for every arm."""
    if "phi" in SCF_START:
        return SCF_START
    from paper_2602_08982_b300 import inputs
    shape = wl["shape"]
    M = shape[0] * shape[1] * shape[2]
    u = W.uniform_solve(shape, kind=W.SLDA_A1, B=W.B_SLDA, rho_sigma=RHO_SIGMA, delta0=0.25)
    ctx = W.Context(W.FP64)
    b = ctx.add_box(shape, kind=W.SLDA_A1, B=W.B_SLDA, C=W.C_ASLDA, mu=u["mu"], nstates=M)
    ctx.set_vext(b, inputs.harmonic_trap(shape, wl["omega"]))
    t0 = time.perf_counter()
    res, _ = ctx.static_solve(b, np.full(M, u["U"]), np.full(M, u["delta"]), method="broyden", mixing=0.3,
                              eps_energy=1e-6, max_iters=args.scf_iters, n_target=args.scf_n, a_mu=0.5,
                              eps_npart=1e-3, fp32_iters=args.scf_fp32_iters)
    sec = time.perf_counter() - t0
    SCF_START["phi"] = ctx.get_states(b)
    ctx.close()
    SCF_START["info"] = {"iters": res["iters"], "converged": res["converged"], "mu": res["mu"],
                         "n_sigma": res["n_sigma"], "max_rel_change": res["max_rel_change"], "seconds": sec,
                         "fp32_iters": args.scf_fp32_iters, "n_target": args.scf_n}
    return SCF_START


def run_arm(W, torch, prec, args, wl, rank, world, dev):
    stream = torch.cuda.current_stream()
    shape, nstates = wl["shape"], wl["nstates"]
    if args.init == "scf":
        start = scf_start(W, args, wl)
        ctx, box, u = make_box(W, prec, wl, stream.cuda_stream, args.integrator, mu=start["info"]["mu"], A=args.A,
                               C=W.C_ASLDA)
        ctx.load_states(box, start["phi"])
        ctx.start(True, args.dt)               # a static solution: stationary start
    else:
        ctx, box, u = make_box(W, prec, wl, stream.cuda_stream, args.integrator, A=args.A, aslda=args.aslda)
        fill_workload(W, ctx, box, u, wl, args.aslda)
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
    de, dn = ctx.check_conservation(box, float("inf"), float("inf"))
    _, steps_done = ctx.get_time()
    rho, nu = ctx.get_densities(box)
    ctx.close()
    M = shape[0] * shape[1] * shape[2]
    units = float(nstates) * M * args.steps
    value = job_rate(units, world, ms * 1e-3)
    bx, fx = stage_x_algorithmic(prec, shape, args.integrator, args.A != 1.0 or args.aslda)
    x_ms, x_n = kt["stage_x"]
    x_avg = x_ms / max(x_n, 1)
    y_ms, y_n = kt["stage_y"]
    y_avg = y_ms / max(y_n, 1)
    per_launch = float(nstates) * M
    hbm, which = measured_peaks()
    if prec == 1:
        achieved = bx * per_launch / (x_avg * 1e-3) / 1e9
        tb = profiled_traffic(shape) if args.integrator == "AB4AM5" and args.A == 1.0 else None  # captured on A = 1
        roof = {"bound": "hbm", "achieved": achieved, "peak": hbm, "unit": "GB/s", "frac": achieved / hbm,
                "traffic": None if tb is None else tb * per_launch,
                "kernel": "stage_x (f + AB4 predictor + AM5 partial + normalisation)",
                "peak_source": which, "algorithmic_bytes_per_state_site": bx,
                "stage_y": {"achieved": 48.0 * per_launch / (y_avg * 1e-3) / 1e9,
                            "frac": 48.0 * per_launch / (y_avg * 1e-3) / 1e9 / hbm,
                            "algorithmic_bytes_per_state_site": 48}}
    else:
        try:
            peak, src = W.measure_fp64_rate(5), "of measured (FP64 FMA microbenchmark on this GPU, this run)"
        except W.WsldaError:
            peak, src = FP64_NOMINAL_TFLOPS, "nominal FP64 rate (measurement failed)"
        achieved = fx * per_launch / (x_avg * 1e-3) / 1e12
        roof = {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                "frac": achieved / peak, "traffic": None,
                "kernel": "stage_x (f + AB4 predictor + AM5 partial + normalisation), FP64",
                "peak_source": src, "algorithmic_flops_per_state_site": fx}
        try:
            # the count takes additions and multiplications as one operation each and the
            # butterflies are mostly unfused, so the FP64 addition issue rate also bounds them
            add = W.measure_fp64_add_rate(5)
            roof["unfused"] = {"peak": add, "unit": "Tops/s", "frac": achieved / add,
                               "peak_source": "of measured (FP64 addition microbenchmark on this GPU, this run)"}
        except W.WsldaError:
            pass
    sb = step_algorithmic_bytes(prec, args.integrator)
    step_gbs = sb * per_launch / (ms / args.steps * 1e-3) / 1e9
    share = {k: kt[k][0] / ms for k in kt}
    roof["launch_variant"] = variant
    return dict(value=value, ms_per_step=ms / args.steps, roofline=roof, clocks=ck, launches=launches,
                kernel_ms=kt, kernel_share=share, rho=rho, nu=nu,
                step_roofline={"bound": "hbm", "achieved": step_gbs, "peak": hbm, "unit": "GB/s",
                               "frac": step_gbs / hbm, "peak_source": which,
                               "algorithmic_bytes_per_state_site": sb,
                               "scope": "whole step: stage X + stage Y state passes (density and potential "
                                        "kernels add traffic the algorithmic figure does not count)"},
                energy_drift={"rel_e_tot_minus_mu_n": de, "rel_n": dn, "after_steps": steps_done,
                              "since": "wslda_start (t = 0 states)"})


def run_e2e(W, torch, args, wl, world):
    """Mixed path end to end through the ABI with pinned host buffers: the
    states travel as complex64, the precision the mixed path stores them in."""
    stream = torch.cuda.current_stream()
    shape, nstates = wl["shape"], wl["nstates"]
    ctx, box, u = make_box(W, W.MIXED, wl, stream.cuda_stream, args.integrator, A=args.A)
    fill_workload(W, ctx, box, u, wl)
    M = shape[0] * shape[1] * shape[2]
    host = torch.empty((nstates, 2, M), dtype=torch.complex64, pin_memory=True)
    host_np = host.numpy()
    ctx.get_states_f32(box, host_np)  # untimed: the job's input now lives in pinned host memory
    ctx.close()
    torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    t0 = time.perf_counter()
    ctx, box, _ = make_box(W, W.MIXED, wl, stream.cuda_stream, args.integrator, A=args.A)
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
    units = float(nstates) * M * args.steps
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


def run_cufft(torch, wl, args, our_stage_ms):
    """The kinetic-term transforms of one stage on the main workload with
    cuFFT (torch.fft): for chunks of states, forward 3D FFT of u and v,
    multiplication by k^2/2 (1/M folded in), inverse 3D FFT. A library
    comparison only; the product path never calls it."""
    shape, nstates = wl["shape"], wl["nstates"]
    M = shape[0] * shape[1] * shape[2]
    chunk = min(nstates, 2048)
    dev = torch.device("cuda")
    ks = [torch.fft.fftfreq(n, d=1.0 / (2 * math.pi), device=dev, dtype=torch.float64) for n in shape]
    k2 = (ks[0][:, None, None] ** 2 + ks[1][None, :, None] ** 2 + ks[2][None, None, :] ** 2)
    sym = (0.5 * k2).to(torch.float32)
    x = torch.randn((chunk, 2) + tuple(shape), dtype=torch.complex64, device=dev)
    stream = torch.cuda.current_stream()

    def once():
        y = torch.fft.fftn(x, dim=(-3, -2, -1))
        y.mul_(sym)
        return torch.fft.ifftn(y, dim=(-3, -2, -1))
    for _ in range(3):
        once()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    reps = 5
    e0.record(stream)
    for _ in range(reps):
        once()
    e1.record(stream)
    torch.cuda.synchronize()
    per_chunk = e0.elapsed_time(e1) / reps
    stage_ms = per_chunk * nstates / chunk
    del x
    torch.cuda.empty_cache()
    return {"ms_per_stage": stage_ms, "chunk_states": chunk,
            "what": "forward 3D FFT of u and v, times k^2/2, inverse 3D FFT (cuFFT plans via torch.fft, "
                    "complex64), states in chunks; the transform work of one stage, nothing else",
            "our_stage_x_ms": our_stage_ms[0], "our_stage_y_ms": our_stage_ms[1],
            "our_stage_y_over_cufft_transforms": our_stage_ms[1] / stage_ms}


def run_oracle_check(W, torch, args, wl):
    """The mixed path against the FP64 CPU oracle on a bounded sample of the
    main workload: the same lattice, trap and vortex imprint with a seeded
    subset of the uniform plane-wave states as the whole system, both started
    from the same double states (Taylor start), args.oracle_steps steps in all.
    Errors are N1's: max-norm relative differences of rho and nu, and of the
    energy; the drift is that of E_tot - mu N from t = 0."""
    n, nsteps = args.oracle_states, args.oracle_steps
    t0 = time.perf_counter()
    o, sysm, phi, lat = oracle_sample(wl, n, args.A)
    sysm.init_regulator(phi)
    e0 = sysm.energy(phi)
    st = o.start(sysm, phi, args.dt, False)
    st = o.evolve(sysm, st, args.dt, nsteps - st.steps)
    rho_r, nu_r = o.densities(st.phi, np.ones(n), np.zeros(n))
    e_r = sysm.energy(st.phi)
    cpu_sec = time.perf_counter() - t0
    ctx = W.Context(W.MIXED, stream=torch.cuda.current_stream().cuda_stream)
    box = ctx.add_box(lat.shape, kind=W.SLDA if args.A != 1.0 else W.SLDA_A1, B=sysm.fn.B, C=sysm.fn.C,
                      mu=sysm.fn.mu, A=args.A, nstates=n)
    ctx.set_vext(box, sysm.vext)
    ctx.load_states(box, phi)
    ctx.start(False, args.dt)
    ctx.step(args.dt, nsteps - ctx.get_time()[1])
    rho, nu = ctx.get_densities(box)
    e = ctx.get_energy(box)
    ctx.close()
    mu = sysm.fn.mu
    rel = lambda a, b: float(np.abs(a - b).max() / np.abs(b).max())
    ec0 = e0["e_total"] - mu * e0["n_part"]
    return {"rel_err_rho": rel(rho, rho_r), "rel_err_nu": rel(nu, nu_r),
            "rel_err_e_total": abs(e["e_total"] - e_r["e_total"]) / abs(e_r["e_total"]),
            "energy_drift_mixed": abs(e["e_total"] - mu * e["n_part"] - ec0) / abs(ec0),
            "energy_drift_oracle": abs(e_r["e_total"] - mu * e_r["n_part"] - ec0) / abs(ec0),
            "after_steps": nsteps, "states": n, "tolerance": 1e-5, "oracle_seconds": cpu_sec,
            "sample": f"{n} seeded plane-wave states of the {lat.nx}x{lat.ny}x{lat.nz} workload lattice (same trap"
                      f"{' and vortex' if wl['vortex'] else ''}) as the whole system, Taylor start, dt={args.dt}"}


# ------------------------------------------------------------------ oracle (CPU)
def oracle_sample(wl, n, A=1.0):
    """CPU-oracle system for the workload's lattice and trap, with n of its
    uniform plane-wave states (seeded choice of momenta), vortex imprinted on
    u when the workload has one."""
    from oracle import tdslda as o
    from paper_2602_08982_b300 import inputs
    shape = wl["shape"]
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
    if wl["vortex"]:
        half = inputs.vortex_phase(shape, winding=0.5)
        phi[:, 0, :] *= half[None, :]
        phi[:, 1, :] *= np.conj(half)[None, :]
    return o, o.TDSystem(lat, fn, vext=inputs.harmonic_trap(lat.shape, wl["omega"])), phi, lat


def oracle_sample_aslda(wl, n):
    """Spin-imbalanced oracle system of the ASLDA workload: n/2 of the uniform
    states and their partners, weights as fill_workload sets them; returns
    (start, step) closures over it and the lattice."""
    from oracle import aslda as a
    o, sysm, phi, lat = oracle_sample(wl, max(1, n // 2))
    h = phi.shape[0]
    u, v = phi[:, 0], phi[:, 1]
    phi2 = np.concatenate([phi, np.stack([np.conj(v), -np.conj(u)], axis=1)])
    fm = np.concatenate([np.full(h, 0.5), np.zeros(h)])
    fp = np.concatenate([np.zeros(h), np.ones(h)])
    m = sysm.fn.mu
    sys_i = a.ImbalancedSystem(lat, a.ASLDA(mu_a=m + ASLDA_DMU[0], mu_b=m + ASLDA_DMU[1]), sysm.vext, sysm.vext, fp, fm)
    start = lambda dt: a.start(sys_i, phi2, dt, True)
    step = lambda st, dt: o.abm_step(sys_i, st, dt, "AB4AM5")
    return start, step, lat, 2 * h


def oracle_stepper(o, scheme):
    """(start, step) of the oracle for the scheme: Alg. 2 itself for AB4AM5."""
    if scheme == "AB4AM5":
        return (lambda sysm, phi, dt: o.start(sysm, phi, dt, stationary=True)), o.ab4am5_step
    return ((lambda sysm, phi, dt: o.start_scheme(sysm, phi, dt, True, scheme)),
            (lambda sysm, st, dt: o.abm_step(sysm, st, dt, scheme)))


def sample_stepper(wl, n, dt, scheme, A, aslda):
    """(state, step, lattice, states) of the oracle on n states of the workload."""
    if aslda:
        start, step, lat, n = oracle_sample_aslda(wl, n)
        return start(dt), (lambda st: step(st, dt)), lat, n
    o, sysm, phi, lat = oracle_sample(wl, n, A)
    start, step = oracle_stepper(o, scheme)
    return start(sysm, phi, dt), (lambda st: step(sysm, st, dt)), lat, n


def cpu_oracle_rate(wl, dt, seconds, max_states=2048, scheme="AB4AM5", A=1.0, aslda=False):
    """The oracle as it stands, on a bounded sample of the workload: the same
    lattice and trap with a subset of the uniform plane-wave states, timed over
    whole ABM steps after a stationary start."""
    shape = wl["shape"]
    max_states = min(max_states, shape[0] * shape[1] * shape[2])
    n = min(64, max_states)
    while True:
        st, step, lat, n = sample_stepper(wl, n, dt, scheme, A, aslda)
        t0 = time.perf_counter()
        st = step(st)
        one = time.perf_counter() - t0
        if one * 4 > seconds or n >= max_states:
            break
        n = min(max_states, n * 2)
    k = max(1, int(seconds / max(one, 1e-3)))
    t0 = time.perf_counter()
    for _ in range(k):
        st = step(st)
    sec = time.perf_counter() - t0
    return {"value": n * lat.M * k / sec, "unit": UNIT, "cores": os.cpu_count(), "ram_gb": host_ram_gb(),
            "kind": "oracle", "n": n,
            "sample": f"{n} of the workload's states on the same {shape[0]}x{shape[1]}x{shape[2]} trap, {k} {scheme} "
                      f"steps after a stationary start, {sec:.1f} s"}


def reference_arm(args, wl):
    rank, world, _ = dist_env()
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("gloo")
        if rank != 0:
            dist.barrier()
            return
    # each step: one oracle step of the scheme over a bounded sample of the
    # states, sized so that one step takes about a second
    n = cpu_oracle_rate(wl, args.dt, args.cpu_seconds / 4, scheme=args.integrator, A=args.A,
                        aslda=args.aslda)["n"]
    st, step, lat, n = sample_stepper(wl, n, args.dt, args.integrator, args.A, args.aslda)
    for _ in range(args.warmup):
        st = step(st)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        st = step(st)
    sec = time.perf_counter() - t0
    value = n * lat.M * args.steps / sec
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1e3 * sec / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic", "impl": "reference",
            "config": workload_config(args, wl, "fp64 oracle (CPU)"),
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": os.cpu_count(), "ram_gb": host_ram_gb(),
                             "kind": "oracle",
                             "sample": f"{n} states of the workload per step, {args.steps} steps, {sec:.1f} s"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def workload_config(args, wl, precision):
    shape = wl["shape"]
    if args.aslda:
        return {"workload": f"spin-imbalanced ASLDA TDSLDA {args.integrator} step, {wl['text']} "
                            f"({wl['nstates'] // 2} plane-wave states and their partners)",
                "lattice": list(shape), "nstates": wl["nstates"], "trap_omega": wl["omega"], "vortex": wl["vortex"],
                "dt": args.dt, "functional": "ASLDA: A(p), B(p) as printed, C = -11.11, "
                                             f"mu_a - mu = {ASLDA_DMU[0]}, mu_b - mu = {ASLDA_DMU[1]}",
                "init": "uniform plane-wave BCS states with partners, v weights halved (polarised), Taylor start",
                "precision": precision, "l2": "inputs larger than L2 (state buffers >> 126 MB), no flush needed",
                "parallelism": "replicas" if args.gpus > 1 else "single GPU"}
    return {"workload": f"TDSLDA {args.integrator} step, {wl['text']}",
            "lattice": list(shape), "nstates": wl["nstates"], "trap_omega": wl["omega"], "vortex": wl["vortex"],
            "dt": args.dt,
            "functional": (f"SLDA with current terms (A={args.A}), " if args.A != 1.0 else "SLDA (A=1), ")
                          + "B=B_ASLDA(0), C from the uniform 16^3-style seed on this lattice",
            "init": ("states of a static self-consistent solve with C = -11.11 (fixed N, Broyden), stationary start"
                     if args.init == "scf" else
                     "uniform plane-wave BCS states (Delta0 = 0.5 eF) quenched into the trap, Taylor start"),
            "friction": args.friction, "precision": precision,
            "l2": "inputs larger than L2 (state buffers >> 126 MB), no flush needed",
            "parallelism": "replicas" if args.gpus > 1 else "single GPU"}


def main():
    args = parse()
    if args.aslda:  # the spin-imbalanced line: its own workload, the mixed arm and its CPU baseline
        if args.workload == "elongated" and not args.shape:
            args.workload = "cube32"
        args.no_e2e = args.no_batched = args.no_oracle_check = args.no_cufft = True
        if args.precision == "both":
            args.precision = "mixed"
    wl = resolve(args, args.workload)
    if args.impl == "reference":
        reference_arm(args, wl)
        return
    rank, world, local = dist_env()
    import torch
    if world > 1:
        torch.distributed.init_process_group("nccl")
    torch.cuda.set_device(local)
    from paper_2602_08982_b300 import wslda as W

    solo = rank == 0 and world == 1
    cpu = None
    if solo and not args.no_cpu:
        cpu = cpu_oracle_rate(wl, args.dt, args.cpu_seconds, scheme=args.integrator, A=args.A, aslda=args.aslda)
    arms = {}
    if args.precision in ("both", "mixed"):
        arms["mixed"] = run_arm(W, torch, W.MIXED, args, wl, rank, world, local)
    cufft = None
    if "mixed" in arms and not args.no_cufft and solo:
        xm, xn = arms["mixed"]["kernel_ms"]["stage_x"]
        ym, yn = arms["mixed"]["kernel_ms"]["stage_y"]
        cufft = run_cufft(torch, wl, args, (xm / max(xn, 1), ym / max(yn, 1)))
    wl64 = resolve(args, args.fp64_workload) if args.precision == "both" else wl
    if args.precision in ("both", "fp64"):
        arms["fp64"] = run_arm(W, torch, W.FP64, args, wl64, rank, world, local)
    e2e = None if args.no_e2e else run_e2e(W, torch, args, wl, world)
    batched = None if args.no_batched else run_batched(W, torch, args)
    check = None
    if solo and not args.no_oracle_check and "mixed" in arms:
        check = run_oracle_check(W, torch, args, wl)
    main_arm = arms.get("mixed") or arms["fp64"]
    line = {"metric": METRIC, "value": main_arm["value"], "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": main_arm["ms_per_step"], "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32" if "mixed" in arms else "f64",
            "data": "synthetic",
            "config": workload_config(args, wl, "mixed: complex64 states and FFTs, f64 accumulation"
                                      if "mixed" in arms else "fp64"),
            "roofline": main_arm["roofline"], "step_roofline": main_arm["step_roofline"],
            "gpu_launches": main_arm["launches"], "clocks": main_arm["clocks"],
            "kernel_share": main_arm["kernel_share"], "energy_drift": main_arm["energy_drift"]}
    if "fp64" in arms and "mixed" in arms:
        a = arms["fp64"]
        line["fp64"] = {"value": a["value"], "ms_per_step": a["ms_per_step"], "roofline": a["roofline"],
                        "step_roofline": a["step_roofline"], "gpu_launches": a["launches"], "clocks": a["clocks"],
                        "kernel_share": a["kernel_share"], "energy_drift": a["energy_drift"],
                        "config": workload_config(args, wl64, "fp64: complex128 states and FFTs")}
    if check:
        line["mixed_vs_oracle"] = check
    if cufft:
        line["cufft"] = cufft
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
