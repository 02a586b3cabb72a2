"""Thin ctypes binding of libwslda_td.so (include/wslda_td.h).

Argument marshalling only: every step of the TDSLDA path runs in the CUDA
library. Methods of `Context` carry the names of the C calls without the
`wslda_` prefix. Arrays may be numpy arrays (host) or torch CUDA tensors
(device, borrowed for the duration of the call). The library must have been
built (`python -m paper_2602_08982_b300.build`); importing this module without
it raises, there is no fallback.
"""
from __future__ import annotations

import ctypes as ct
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "_lib", "libwslda_td.so")

FP64, MIXED = 0, 1
SLDA_A1, BDG, SLDA, ASLDA = 0, 1, 2, 3
A_ASLDA = 1.094  # A_a(0) of the ASLDA functional (Sec. 2.4)
SCHEMES = {"AB4AM5": 0, "AB3AM4": 1, "AB5AM5": 2}
# B of the spin-symmetric ASLDA functional (Sec. 2.4): 2^(2/3) [0.357 - 2 A(0) 2^(-5/3)], A(0) = 1.094
B_SLDA = 2.0 ** (2.0 / 3.0) * (0.357 - 2.0 * 1.094 * 2.0 ** (-5.0 / 3.0))
C_ASLDA = -11.11  # C of the ASLDA functional as printed (Sec. 2.4)
STATUS = {0: "OK", 1: "EINVAL", 2: "ENOMEM", 3: "ECUDA", 4: "ENAN", 5: "EDRIFT", 6: "ETIMEOUT", 7: "ESTATE",
          8: "EUNSUPPORTED"}
KERNEL_KINDS = {"stage_x": 0, "stage_y": 1, "density": 2, "potentials": 3, "aux": 4}


class WsldaError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS.get(status, status)}: {msg}")
        self.status = status


class Lattice(ct.Structure):
    _fields_ = [("nx", ct.c_int), ("ny", ct.c_int), ("nz", ct.c_int),
                ("dx", ct.c_double), ("dy", ct.c_double), ("dz", ct.c_double)]


class Functional(ct.Structure):
    _fields_ = [("kind", ct.c_int), ("B", ct.c_double), ("C", ct.c_double), ("inv_4pi_a", ct.c_double),
                ("mu", ct.c_double), ("ec", ct.c_double), ("rho_floor", ct.c_double), ("A", ct.c_double),
                ("mu_b", ct.c_double)]


class Uniform(ct.Structure):
    _fields_ = [(k, ct.c_double) for k in ("mu_eff", "delta", "mu", "U", "C", "lam", "inv_g")]


class Energy(ct.Structure):
    _fields_ = [(k, ct.c_double) for k in ("e_kin", "e_pot", "e_pair", "e_ext", "e_pair_ext", "e_total", "n_part",
                                           "e_cur")]


class ScfParams(ct.Structure):
    _fields_ = [("mixing", ct.c_double), ("eps_energy", ct.c_double), ("e_ref", ct.c_double),
                ("max_iters", ct.c_int), ("n_target", ct.c_double), ("a_mu", ct.c_double),
                ("eps_npart", ct.c_double), ("method", ct.c_int), ("broyden_memory", ct.c_int),
                ("broyden_w0", ct.c_double), ("fp32_iters", ct.c_int)]


class ScfResult(ct.Structure):
    _fields_ = [("iters", ct.c_int), ("converged", ct.c_int), ("mu", ct.c_double), ("max_rel_change", ct.c_double),
                ("n_sigma", ct.c_double), ("energy", Energy)]


def _load():
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"{LIB_PATH} is missing: build it with `python -m paper_2602_08982_b300.build`")
    lib = ct.CDLL(LIB_PATH)
    P, I, D, I64 = ct.c_void_p, ct.c_int, ct.c_double, ct.c_int64
    DP = ct.POINTER(ct.c_double)
    sig = {
        "wslda_create": (I, [I, P, ct.POINTER(P)]),
        "wslda_destroy": (None, [P]),
        "wslda_last_error": (ct.c_char_p, [P]),
        "wslda_lattice_supported": (I, [I, I, I, I]),
        "wslda_lattice_variants": (I, [I, I, I, I]),
        "wslda_add_box": (I, [P, ct.POINTER(Lattice), ct.POINTER(Functional), I64]),
        "wslda_set_vext": (I, [P, I, P, I]),
        "wslda_set_dext": (I, [P, I, P, I]),
        "wslda_load_states": (I, [P, I, P, P, P, I]),
        "wslda_start": (I, [P, I, D]),
        "wslda_step": (I, [P, D, I]),
        "wslda_get_states": (I, [P, I, P, I]),
        "wslda_get_densities": (I, [P, I, P, P, P, P]),
        "wslda_get_fields": (I, [P, I, P, P]),
        "wslda_get_spin_densities": (I, [P, I, P, P, P, P, P, P, P]),
        "wslda_get_spin_fields": (I, [P, I, P, P, P]),
        "wslda_get_energy": (I, [P, I, ct.POINTER(Energy)]),
        "wslda_eval_f": (I, [P, I, P]),
        "wslda_save": (I, [P, ct.c_char_p]),
        "wslda_load": (I, [P, ct.c_char_p]),
        "wslda_get_time": (I, [P, DP, ct.POINTER(I64)]),
        "wslda_memory_bytes": (I64, [P]),
        "wslda_launch_count": (I64, [P]),
        "wslda_set_profiling": (I, [P, I]),
        "wslda_uniform_solve": (I, [ct.POINTER(Lattice), ct.POINTER(Functional), D, D, ct.POINTER(Uniform)]),
        "wslda_fill_uniform_states": (I, [P, I, D, D, P]),
        "wslda_set_weights": (I, [P, I, P, P]),
        "wslda_get_kernel_time": (I, [P, I, DP, ct.POINTER(I64)]),
        "wslda_get_variant": (I, [P, I, ct.c_char_p, I]),
        "wslda_set_graph": (I, [P, I, I]),
        "wslda_check_conservation": (I, [P, I, D, D, DP, DP]),
        "wslda_densities_noalloc": (I, [I, P, P, P, I64, I, I, I, P, P, P]),
        "wslda_set_integrator": (I, [P, I]),
        "wslda_set_friction": (I, [P, I, D, D, D, D, D]),
        "wslda_load_states_f32": (I, [P, I, P, P, P, I]),
        "wslda_get_states_f32": (I, [P, I, P, I]),
        "wslda_net_create": (I, [I, I, I, I, I, ct.POINTER(P)]),
        "wslda_net_destroy": (None, [P]),
        "wslda_net_last_error": (ct.c_char_p, [P]),
        "wslda_net_param_count": (I64, [P]),
        "wslda_net_set_params": (I, [P, P]),
        "wslda_net_get_params": (I, [P, P]),
        "wslda_net_forward": (I, [P, P, I, P, P]),
        "wslda_net_loss_grad": (I, [P, P, P, I, DP, P, P]),
        "wslda_net_adam": (I, [P, D, P]),
        "wslda_net_symmetrize": (I, [P, I64, I, I, I, P, P]),
        "wslda_net_get_activation": (I, [P, I, I, P, P]),
        "wslda_static_solve": (I, [P, I, P, P, ct.POINTER(ScfParams), P, ct.POINTER(ScfResult)]),
        "wslda_imprint_phase": (I, [P, I, I, P, I]),
        "wslda_measure_fp64_rate": (I, [I, DP]),
        "wslda_measure_fp64_add_rate": (I, [I, DP]),
    }
    for name, (res, args) in sig.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    return lib


lib = _load()


def lattice_supported(precision: int, nx: int, ny: int, nz: int) -> bool:
    return bool(lib.wslda_lattice_supported(precision, nx, ny, nz))


def lattice_variants(precision: int, nx: int, ny: int, nz: int) -> int:
    return int(lib.wslda_lattice_variants(precision, nx, ny, nz))


def uniform_solve(shape, spacing=(1.0, 1.0, 1.0), *, kind=SLDA_A1, B=0.0, inv_4pi_a=0.0, ec=-1.0,
                  rho_sigma=1.0 / (6 * np.pi ** 2), delta0=0.0) -> dict:
    """Uniform plane-wave BCS solution on the lattice (wslda_uniform_solve)."""
    lat = Lattice(*[int(v) for v in shape], *[float(v) for v in spacing])
    fn = Functional(int(kind), float(B), 0.0, float(inv_4pi_a), 0.0, float(ec), 1e-12, 1.0, 0.0)
    out = Uniform()
    st = lib.wslda_uniform_solve(ct.byref(lat), ct.byref(fn), float(rho_sigma), float(delta0), ct.byref(out))
    if st:
        raise WsldaError(st, "uniform_solve found no solution or got bad arguments")
    return {k: getattr(out, k) for k, _ in Uniform._fields_}


def measure_fp64_rate(reps: int = 5) -> float:
    """FP64 FMA throughput of the current device in TFLOP/s (wslda_measure_fp64_rate)."""
    out = ct.c_double()
    st = lib.wslda_measure_fp64_rate(int(reps), ct.byref(out))
    if st:
        raise WsldaError(st, "wslda_measure_fp64_rate failed")
    return out.value


def measure_fp64_add_rate(reps: int = 5) -> float:
    """FP64 addition throughput of the current device in tera-operations per
    second (wslda_measure_fp64_add_rate)."""
    out = ct.c_double()
    st = lib.wslda_measure_fp64_add_rate(int(reps), ct.byref(out))
    if st:
        raise WsldaError(st, "wslda_measure_fp64_add_rate failed")
    return out.value


def densities_noalloc(precision: int, uv, rho, nu, shape, w_minus=None, w_plus=None, stream: int = 0):
    """rho and nu of device states into device outputs without any device
    allocation (wslda_densities_noalloc). All arguments are torch CUDA tensors
    on the current device: uv [n][2][M] complex64 (MIXED) or complex128 (FP64),
    rho >= M and nu >= 2 M float64 elements, weights >= n float64 elements.
    They are checked here, because the C call takes raw device pointers and
    cannot see their sizes. The work is queued on `stream` and not waited for."""
    import torch
    M = int(shape[0]) * int(shape[1]) * int(shape[2])
    want = torch.complex64 if precision == MIXED else torch.complex128
    if precision not in (FP64, MIXED):
        raise ValueError("precision must be FP64 or MIXED")
    dev = torch.device("cuda", torch.cuda.current_device())
    named = [("uv", uv), ("rho", rho), ("nu", nu), ("w_minus", w_minus), ("w_plus", w_plus)]
    for name, t in named:
        if t is None:
            continue
        if not (hasattr(t, "is_cuda") and t.is_cuda and t.device == dev):
            raise ValueError(f"{name} must be a CUDA tensor on the current device")
        if not t.is_contiguous():
            raise ValueError(f"{name} must be contiguous")
    if uv.dtype != want or uv.dim() != 3 or uv.shape[1] != 2 or uv.shape[2] != M:
        raise ValueError(f"uv must be a {want} tensor of shape (n, 2, {M})")
    n = int(uv.shape[0])
    for name, t, need in (("rho", rho, M), ("nu", nu, 2 * M), ("w_minus", w_minus, n), ("w_plus", w_plus, n)):
        if t is not None and (t.dtype != torch.float64 or t.numel() < need):
            raise ValueError(f"{name} must hold at least {need} float64 values")
    ptr = lambda t: ct.c_void_p(t.data_ptr()) if t is not None else None
    st = lib.wslda_densities_noalloc(int(precision), ptr(uv), ptr(w_minus), ptr(w_plus), n,
                                     int(shape[0]), int(shape[1]), int(shape[2]), ptr(rho), ptr(nu),
                                     ct.c_void_p(stream))
    if st:
        raise WsldaError(st, "wslda_densities_noalloc failed")


def _ptr(a, dtype, on_device: bool):
    """(pointer, keep-alive) of a numpy array or a torch tensor."""
    if a is None:
        return None, None
    if hasattr(a, "data_ptr"):  # torch tensor
        if not a.is_contiguous():
            raise ValueError("tensor must be contiguous")
        return ct.c_void_p(a.data_ptr()), a
    arr = np.ascontiguousarray(a, dtype=dtype)
    return arr.ctypes.data_as(ct.c_void_p), arr


def _is_device(a) -> bool:
    return hasattr(a, "is_cuda") and a.is_cuda


class Context:
    def __init__(self, precision: int = MIXED, stream: int | None = None):
        self._h = ct.c_void_p()
        st = lib.wslda_create(precision, ct.c_void_p(stream or 0), ct.byref(self._h))
        if st:
            raise WsldaError(st, "wslda_create failed")
        self.precision = precision
        self.boxes: list[tuple] = []

    # ------------------------------------------------------------------ helpers
    def _check(self, st: int):
        if st:
            raise WsldaError(st, lib.wslda_last_error(self._h).decode())

    def close(self):
        if self._h:
            lib.wslda_destroy(self._h)
            self._h = ct.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    # ------------------------------------------------------------------ ABI
    def set_friction(self, box: int, alpha=0.0, beta=0.0, gamma=0.0, rho0=1.0 / (6.0 * np.pi ** 2), n_req=1.0):
        """Quantum-friction terms (Sec. 5.2.4) for one box."""
        self._check(lib.wslda_set_friction(self._h, box, float(alpha), float(beta), float(gamma), float(rho0),
                                           float(n_req)))

    def set_integrator(self, scheme: str):
        """'AB4AM5' (default), 'AB3AM4' or 'AB5AM5' for boxes added afterwards."""
        self._check(lib.wslda_set_integrator(self._h, SCHEMES[scheme]))

    def add_box(self, shape, spacing=(1.0, 1.0, 1.0), *, kind=SLDA_A1, B=0.0, C=-1.0, inv_4pi_a=0.0, mu=0.0,
                ec=-1.0, rho_floor=1e-12, A=1.0, mu_b=None, nstates: int) -> int:
        """kind SLDA with A != 1 carries the current terms (inverse effective mass A);
        kind ASLDA is the spin-imbalanced functional with mu (species a) and mu_b."""
        lat = Lattice(*[int(v) for v in shape], *[float(v) for v in spacing])
        fn = Functional(int(kind), float(B), float(C), float(inv_4pi_a), float(mu), float(ec), float(rho_floor),
                        float(A), float(mu if mu_b is None else mu_b))
        r = lib.wslda_add_box(self._h, ct.byref(lat), ct.byref(fn), int(nstates))
        if r < 0:
            self._check(-r)
        self.boxes.append((tuple(int(v) for v in shape), int(nstates)))
        return r

    def _M(self, box):
        s = self.boxes[box][0]
        return s[0] * s[1] * s[2]

    def set_vext(self, box: int, vext):
        p, keep = _ptr(vext, np.float64, _is_device(vext))
        self._check(lib.wslda_set_vext(self._h, box, p, int(_is_device(vext))))

    def set_dext(self, box: int, dext):
        if not _is_device(dext):
            dext = np.ascontiguousarray(dext, dtype=np.complex128)
        p, keep = _ptr(dext, np.complex128, _is_device(dext))
        self._check(lib.wslda_set_dext(self._h, box, p, int(_is_device(dext))))

    def load_states(self, box: int, uv, w_minus=None, w_plus=None):
        dev = _is_device(uv)
        if not dev:
            uv = np.ascontiguousarray(uv, dtype=np.complex128)
        p, keep = _ptr(uv, np.complex128, dev)
        pm, km = _ptr(w_minus, np.float64, False)
        pp, kp = _ptr(w_plus, np.float64, False)
        self._check(lib.wslda_load_states(self._h, box, p, pm, pp, int(dev)))

    def load_states_f32(self, box: int, uv, w_minus=None, w_plus=None):
        """load_states with complex64 states (host numpy or device tensor)."""
        dev = _is_device(uv)
        p, keep = _ptr(uv, np.complex64, dev)
        pm, km = _ptr(w_minus, np.float64, False)
        pp, kp = _ptr(w_plus, np.float64, False)
        self._check(lib.wslda_load_states_f32(self._h, box, p, pm, pp, int(dev)))

    def get_states_f32(self, box: int, out=None):
        """get_states as complex64 (host numpy unless `out` is a device tensor)."""
        n = self.boxes[box][1]
        if out is None:
            out = np.empty((n, 2, self._M(box)), dtype=np.complex64)
        p, keep = _ptr(out, np.complex64, _is_device(out))
        self._check(lib.wslda_get_states_f32(self._h, box, p, int(_is_device(out))))
        return out

    def set_weights(self, box: int, w_minus=None, w_plus=None):
        """Frozen weights f(-E_n), f(E_n) of the loaded states (None: T = 0)."""
        pm, km = _ptr(w_minus, np.float64, False)
        pp, kp = _ptr(w_plus, np.float64, False)
        self._check(lib.wslda_set_weights(self._h, box, pm, pp))

    def imprint_phase(self, box: int, comp: int, phase):
        """Multiply component comp (0 = u, 1 = v) of every state by phase[r]."""
        dev = _is_device(phase)
        if not dev:
            phase = np.ascontiguousarray(phase, dtype=np.complex128)
        p, keep = _ptr(phase, np.complex128, dev)
        self._check(lib.wslda_imprint_phase(self._h, box, int(comp), p, int(dev)))

    def fill_uniform_states(self, box: int, mu_eff: float, delta: float, kidx=None):
        p, keep = _ptr(kidx, np.int64, False)
        self._check(lib.wslda_fill_uniform_states(self._h, box, float(mu_eff), float(delta), p))

    def static_solve(self, box: int, U0, delta0, *, mixing: float = 0.5, eps_energy: float = 1e-6,
                     e_ref: float = 0.5, max_iters: int = 200, n_target: float = 0.0, a_mu: float = 0.0,
                     eps_npart: float = 1e-6, method: str = "linear", broyden_memory: int = 7,
                     broyden_w0: float = 0.01, fp32_iters: int = 0):
        """Static self-consistent solve (Alg. 1); the box's states become the
        positive-energy eigenstates. Returns (result dict, quasiparticle energies)."""
        M = self._M(box)
        U0 = np.ascontiguousarray(U0, dtype=np.float64)
        d0 = np.ascontiguousarray(delta0, dtype=np.float64)
        if U0.size != M or d0.size != M:
            raise ValueError("U0 and delta0 need M real values")
        E = np.empty(M)
        if method not in ("linear", "broyden"):
            raise ValueError("method is 'linear' or 'broyden'")
        prm = ScfParams(float(mixing), float(eps_energy), float(e_ref), int(max_iters), float(n_target),
                        float(a_mu), float(eps_npart), int(method == "broyden"), int(broyden_memory),
                        float(broyden_w0), int(fp32_iters))
        out = ScfResult()
        self._check(lib.wslda_static_solve(self._h, box, U0.ctypes.data_as(ct.c_void_p),
                                           d0.ctypes.data_as(ct.c_void_p), ct.byref(prm),
                                           E.ctypes.data_as(ct.c_void_p), ct.byref(out)))
        res = {k: getattr(out, k) for k, _ in ScfResult._fields_ if k != "energy"}
        res["converged"] = bool(res["converged"])
        res["energy"] = {k: getattr(out.energy, k) for k, _ in Energy._fields_}
        return res, E

    def start(self, stationary: bool, dt: float):
        self._check(lib.wslda_start(self._h, int(bool(stationary)), float(dt)))

    def step(self, dt: float, nsteps: int = 1):
        self._check(lib.wslda_step(self._h, float(dt), int(nsteps)))

    def get_states(self, box: int, out=None):
        n = self.boxes[box][1]
        if out is None:
            out = np.empty((n, 2, self._M(box)), dtype=np.complex128)
        p, keep = _ptr(out, np.complex128, _is_device(out))
        self._check(lib.wslda_get_states(self._h, box, p, int(_is_device(out))))
        return out

    def get_densities(self, box: int, tau: bool = False, current: bool = False):
        M = self._M(box)
        rho = np.empty(M)
        nu = np.empty(M, dtype=np.complex128)
        t = np.empty(M) if tau else None
        j = np.empty((3, M)) if current else None
        self._check(lib.wslda_get_densities(self._h, box, rho.ctypes.data_as(ct.c_void_p),
                                            nu.ctypes.data_as(ct.c_void_p),
                                            t.ctypes.data_as(ct.c_void_p) if tau else None,
                                            j.ctypes.data_as(ct.c_void_p) if current else None))
        return (rho, nu) if not (tau or current) else (rho, nu, t, j)

    def get_spin_densities(self, box: int) -> dict:
        """Per-species densities of an ASLDA box: rho_a, rho_b, nu, tau_a, tau_b, j_a, j_b."""
        M = self._M(box)
        out = {"rho_a": np.empty(M), "rho_b": np.empty(M), "nu": np.empty(M, dtype=np.complex128),
               "tau_a": np.empty(M), "tau_b": np.empty(M), "j_a": np.empty((3, M)), "j_b": np.empty((3, M))}
        p = lambda k: out[k].ctypes.data_as(ct.c_void_p)
        self._check(lib.wslda_get_spin_densities(self._h, box, p("rho_a"), p("rho_b"), p("nu"), p("tau_a"),
                                                 p("tau_b"), p("j_a"), p("j_b")))
        return out

    def get_spin_fields(self, box: int):
        """(V_a, V_b, Delta) of an ASLDA box."""
        M = self._M(box)
        Va, Vb, D = np.empty(M), np.empty(M), np.empty(M, dtype=np.complex128)
        self._check(lib.wslda_get_spin_fields(self._h, box, Va.ctypes.data_as(ct.c_void_p),
                                              Vb.ctypes.data_as(ct.c_void_p), D.ctypes.data_as(ct.c_void_p)))
        return Va, Vb, D

    def get_fields(self, box: int):
        M = self._M(box)
        U = np.empty(M)
        delta = np.empty(M, dtype=np.complex128)
        self._check(lib.wslda_get_fields(self._h, box, U.ctypes.data_as(ct.c_void_p),
                                         delta.ctypes.data_as(ct.c_void_p)))
        return U, delta

    def get_energy(self, box: int) -> dict:
        e = Energy()
        self._check(lib.wslda_get_energy(self._h, box, ct.byref(e)))
        return {k: getattr(e, k) for k, _ in Energy._fields_}

    def eval_f(self, box: int):
        n = self.boxes[box][1]
        out = np.empty((n, 2, self._M(box)), dtype=np.complex128)
        self._check(lib.wslda_eval_f(self._h, box, out.ctypes.data_as(ct.c_void_p)))
        return out

    def save(self, path: str):
        self._check(lib.wslda_save(self._h, path.encode()))

    def load(self, path: str):
        self._check(lib.wslda_load(self._h, path.encode()))

    def get_time(self):
        t = ct.c_double()
        s = ct.c_int64()
        self._check(lib.wslda_get_time(self._h, ct.byref(t), ct.byref(s)))
        return t.value, s.value

    def check_conservation(self, box: int, e_tol: float, n_tol: float):
        de, dn = ct.c_double(), ct.c_double()
        self._check(lib.wslda_check_conservation(self._h, box, float(e_tol), float(n_tol), ct.byref(de),
                                                 ct.byref(dn)))
        return de.value, dn.value

    def set_graph(self, enable: bool, nstreams: int = 4):
        self._check(lib.wslda_set_graph(self._h, int(bool(enable)), int(nstreams)))

    def get_variant(self, box: int) -> str:
        buf = ct.create_string_buffer(256)
        self._check(lib.wslda_get_variant(self._h, box, buf, 256))
        return buf.value.decode()

    def launch_count(self) -> int:
        return int(lib.wslda_launch_count(self._h))

    def memory_bytes(self) -> int:
        return int(lib.wslda_memory_bytes(self._h))

    def set_profiling(self, enable: bool):
        self._check(lib.wslda_set_profiling(self._h, int(bool(enable))))

    def get_kernel_time(self, kind) -> tuple[float, int]:
        k = KERNEL_KINDS[kind] if isinstance(kind, str) else int(kind)
        ms = ct.c_double()
        n = ct.c_int64()
        self._check(lib.wslda_get_kernel_time(self._h, k, ct.byref(ms), ct.byref(n)))
        return ms.value, n.value


class Net:
    """The learned starting-field network (wslda_net_*): four periodic 3x3x3
    convolutions 2 -> hidden -> hidden -> hidden -> 2 with tanh, bfloat16
    weights. Activations are device float32 arrays [batch][2][M] given as
    torch tensors (or raw device pointers)."""

    def __init__(self, shape, hidden: int = 32, max_batch: int = 16):
        h = ct.c_void_p()
        st = lib.wslda_net_create(int(shape[0]), int(shape[1]), int(shape[2]), int(hidden), int(max_batch),
                                  ct.byref(h))
        if st:
            raise WsldaError(st, "wslda_net_create failed")
        self._h = h
        self.shape = tuple(int(v) for v in shape)
        self.hidden = hidden
        self.max_batch = max_batch

    def _check(self, st: int):
        if st:
            raise WsldaError(st, lib.wslda_net_last_error(self._h).decode())

    def close(self):
        if self._h:
            lib.wslda_net_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def nparams(self) -> int:
        return int(lib.wslda_net_param_count(self._h))

    def set_params(self, theta):
        t = np.ascontiguousarray(theta, dtype=np.float32)
        if t.size != self.nparams:
            raise ValueError("wrong parameter count")
        self._check(lib.wslda_net_set_params(self._h, t.ctypes.data_as(ct.c_void_p)))

    def get_params(self):
        t = np.empty(self.nparams, dtype=np.float32)
        self._check(lib.wslda_net_get_params(self._h, t.ctypes.data_as(ct.c_void_p)))
        return t

    @staticmethod
    def _dev(x):
        return ct.c_void_p(x.data_ptr()) if hasattr(x, "data_ptr") else ct.c_void_p(int(x))

    @staticmethod
    def _stream(stream):
        return ct.c_void_p(0 if stream is None else int(stream))

    def forward(self, x, y, batch: int, stream=None):
        self._check(lib.wslda_net_forward(self._h, self._dev(x), int(batch), self._dev(y), self._stream(stream)))

    def loss_grad(self, x, target, batch: int, want_grad: bool = False, stream=None):
        loss = ct.c_double()
        g = np.empty(self.nparams, dtype=np.float32) if want_grad else None
        self._check(lib.wslda_net_loss_grad(self._h, self._dev(x), self._dev(target), int(batch), ct.byref(loss),
                                            g.ctypes.data_as(ct.c_void_p) if want_grad else None,
                                            self._stream(stream)))
        return (loss.value, g) if want_grad else loss.value

    def adam(self, lr: float, stream=None):
        self._check(lib.wslda_net_adam(self._h, float(lr), self._stream(stream)))

    def get_activation(self, layer: int, batch: int, stream=None):
        """Output of hidden layer `layer` (0..2) of the last forward pass, as a
        host array [batch][hidden][M]."""
        out = np.empty((batch, self.hidden, int(np.prod(self.shape))), dtype=np.float32)
        self._check(lib.wslda_net_get_activation(self._h, int(layer), int(batch), out.ctypes.data_as(ct.c_void_p),
                                                 self._stream(stream)))
        return out

    def symmetrize(self, y, out, nfields: int, stream=None):
        st = lib.wslda_net_symmetrize(self._dev(y), int(nfields), *self.shape, self._dev(out), self._stream(stream))
        if st:
            raise WsldaError(st, "wslda_net_symmetrize failed")
