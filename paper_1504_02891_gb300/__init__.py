"""Python binding of libgpe: the regularized Newton ground-state method of
Wu, Wen & Bao (arXiv:1504.02891) on GB300 (sm_103a).

Argument marshalling only: every step runs in the CUDA library behind the C
ABI declared in include/gpe.h.  Device buffers are passed as torch CUDA
tensors (their data pointers); torch is used for device memory and streams.
Importing this package loads ``libgpe.so`` and fails loudly if it is missing:
there is no CPU fallback.
"""
from __future__ import annotations

import ctypes as C
import math
import os

import numpy as np

__all__ = ["lib", "Problem", "Plan", "SolveOpts", "SolveReport", "GPEError",
           "FOURIER", "SINE", "FD", "F32", "F64", "load", "LIB_PATH"]

LIB_PATH = os.path.join(os.path.dirname(os.path.abspath(__file__)), "libgpe.so")

FOURIER, SINE, FD = 0, 1, 2
F32, F64 = 0, 1
V_HARMONIC, V_LATTICE, V_STIRRER, V_ARRAY = 0, 1, 2, 3
_DISC = {"fourier": FOURIER, "sine": SINE, "fd": FD}

OK, EINVAL, ECUDA, ENOMEM, ENONFINITE, ENOCONV, ETIMEOUT = 0, 1, 2, 3, 4, 5, 6
STATUS = {0: "GPE_OK", 1: "GPE_EINVAL", 2: "GPE_ECUDA", 3: "GPE_ENOMEM",
          4: "GPE_ENONFINITE", 5: "GPE_ENOCONV", 6: "GPE_ETIMEOUT"}


class GPEError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{STATUS.get(status, status)}: {msg}")
        self.status = status


class Problem(C.Structure):
    _fields_ = [("dim", C.c_int), ("n", C.c_int * 3), ("lo", C.c_double * 3), ("hi", C.c_double * 3),
                ("disc", C.c_int), ("beta", C.c_double), ("omega", C.c_double), ("is_complex", C.c_int),
                ("v_kind", C.c_int), ("v_param", C.c_double * 8), ("v_host", C.POINTER(C.c_double))]

    @classmethod
    def from_params(cls, p):
        """From a workload parameter dict (see workloads.problem)."""
        pr = cls()
        pr.dim = p["dim"]
        for a in range(3):
            pr.n[a] = p["n"][a] if a < p["dim"] else 1
            pr.lo[a] = p["lo"][a] if a < p["dim"] else 0.0
            pr.hi[a] = p["hi"][a] if a < p["dim"] else 1.0
        pr.disc = _DISC[p["disc"]]
        pr.beta = p["beta"]
        pr.omega = p["omega"]
        pr.is_complex = 1 if p["is_complex"] else 0
        pot = p["potential"]
        g = pot.get("gamma", (1.0, 1.0, 1.0))
        for a in range(3):
            pr.v_param[a] = g[a] if a < len(g) else 1.0
        kind = pot["kind"]
        if kind == "harmonic":
            pr.v_kind = V_HARMONIC
        elif kind == "lattice":
            pr.v_kind = V_LATTICE
            pr.v_param[3] = pot["depth"]
            pr.v_param[4] = pot["k"]
        elif kind == "stirrer":
            pr.v_kind = V_STIRRER
            pr.v_param[3] = pot["w0"]
            pr.v_param[4] = pot["delta"]
            pr.v_param[5] = pot["r0"]
        else:
            raise ValueError(kind)
        return pr


class SolveOpts(C.Structure):
    _fields_ = [("levels", C.c_int), ("mode", C.c_int), ("method", C.c_int), ("k_init", C.c_int),
                ("k_sub", C.c_int), ("max_outer", C.c_int), ("max_iter", C.c_int), ("eps0", C.c_double),
                ("delta_stop", C.c_double), ("res_tol", C.c_double), ("delta0", C.c_double),
                ("switch_rel", C.c_double), ("chunk", C.c_int), ("use_graphs", C.c_int), ("persistent", C.c_int),
                ("cluster", C.c_int), ("search", C.c_int), ("alpha_hat", C.c_double), ("eta", C.c_double)]


class SolveReport(C.Structure):
    _fields_ = [("E", C.c_double), ("mu", C.c_double), ("res", C.c_double), ("status", C.c_int),
                ("outer_f32", C.c_int), ("outer_f64", C.c_int), ("inner_f32", C.c_int), ("inner_f64", C.c_int),
                ("nfe", C.c_int), ("ms_f32", C.c_double), ("ms_f64", C.c_double)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


_lib = None


def load():
    """Load libgpe.so (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"libgpe.so not built at {LIB_PATH}; run "
                          "`python -m paper_1504_02891_gb300.build`")
    L = C.CDLL(LIB_PATH)
    vp, dp, ip = C.c_void_p, C.POINTER(C.c_double), C.c_int
    sig = {
        "gpe_plan_create": ([C.POINTER(Problem), ip, ip, vp, C.POINTER(vp)], ip),
        "gpe_plan_destroy": ([vp], ip),
        "gpe_last_error": ([], C.c_char_p),
        "gpe_plan_size": ([vp, C.POINTER(C.c_int64), dp], ip),
        "gpe_energy": ([vp, vp, dp, dp, dp], ip),
        "gpe_grad": ([vp, vp, vp, dp, dp], ip),
        "gpe_hessvec": ([vp, vp, vp, C.c_double, vp], ip),
        "gpe_feasible_step": ([vp, vp, vp, C.c_double, vp, dp], ip),
        "gpe_prolong": ([vp, vp, vp, vp], ip),
        "gpe_solve_opts_default": ([C.POINTER(SolveOpts)], ip),
        "gpe_plan_autotune": ([vp, ip], ip),
        "gpe_autotune_report": ([C.c_char_p, C.c_size_t], ip),
        "gpe_rnewton_solve": ([vp, vp, C.POINTER(SolveOpts), C.POINTER(SolveReport)], ip),
        "gpe_hess_min_eig": ([vp, vp, ip, C.c_double, dp, dp, C.POINTER(C.c_int)], ip),
        "gpe_solve_batch": ([C.POINTER(Problem), ip, C.POINTER(vp), C.POINTER(SolveOpts), C.POINTER(SolveReport),
                             vp], ip),
        "gpe_kernel_launches": ([], C.c_int64),
        "gpe_profile_enable": ([ip], ip),
        "gpe_profile_summary": ([C.c_char_p, ip], ip),
        "gpe_probe_peak": ([ip, vp, dp], ip),
        "gpe_set_wait_limit": ([C.c_int64], ip),
        "gpe_set_operator_path": ([ip], ip),
    }
    missing = [name for name in sig if not hasattr(L, name)]
    if missing:
        # a stale build: release it so that a rebuilt library can be loaded
        import _ctypes
        _ctypes.dlclose(L._handle)
        raise ImportError(f"{LIB_PATH} lacks {', '.join(missing)}; rebuild with "
                          "`python -m paper_1504_02891_gb300.build`")
    for name, (args, res) in sig.items():
        f = getattr(L, name)
        f.argtypes = args
        f.restype = res
    _lib = L
    return L


lib = None
try:
    lib = load()
except (ImportError, OSError):
    # Not built yet, or a stale build that lacks a newer entry point: the
    # module stays importable for build(); every call below raises.
    lib = None


def _check(st, allow=()):
    if st != 0 and st not in allow:
        raise GPEError(st, load().gpe_last_error().decode())
    return st


def _ptr(t):
    return C.c_void_p(t.data_ptr()) if t is not None else None


def _dbuf(n):
    return (C.c_double * n)()


class Plan:
    """Owns a gpe_plan.  ``params`` is a workload parameter dict."""

    def __init__(self, params, nbatch=1, prec=F64, stream=None):
        import torch
        L = load()
        self.params = params
        self.nbatch = nbatch
        self.prec = prec
        self.problem = Problem.from_params(params)
        if stream is None:
            stream = torch.cuda.current_stream()
        self.stream = stream
        h = C.c_void_p()
        _check(L.gpe_plan_create(C.byref(self.problem), nbatch, prec, C.c_void_p(stream.cuda_stream), C.byref(h)))
        self.handle = h
        n = C.c_int64()
        hv = C.c_double()
        _check(L.gpe_plan_size(h, C.byref(n), C.byref(hv)))
        self.M = n.value
        self.h_vol = hv.value
        ext = []
        for a in range(params["dim"]):
            N = params["n"][a]
            ext.append(N if params["disc"] == "fourier" else N - 1)
        self.shape = tuple(reversed(ext))
        self.is_complex = bool(params["is_complex"])

    @property
    def dtype(self):
        import torch
        if self.is_complex:
            return torch.complex64 if self.prec == F32 else torch.complex128
        return torch.float32 if self.prec == F32 else torch.float64

    def empty(self):
        import torch
        shape = (self.nbatch,) + self.shape if self.nbatch > 1 else self.shape
        return torch.empty(shape, dtype=self.dtype, device="cuda")

    def _chk(self, t):
        if t.dtype != self.dtype or not t.is_cuda or not t.is_contiguous() or t.numel() != self.M * self.nbatch:
            raise ValueError(f"expected contiguous CUDA {self.dtype} tensor with {self.M * self.nbatch} elements")

    def close(self):
        if getattr(self, "handle", None):
            load().gpe_plan_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    # -- entry points --------------------------------------------------------
    def energy(self, psi):
        self._chk(psi)
        E, mu, n2 = _dbuf(self.nbatch), _dbuf(self.nbatch), _dbuf(self.nbatch)
        _check(load().gpe_energy(self.handle, _ptr(psi), E, mu, n2))
        if self.nbatch == 1:
            return E[0], mu[0], n2[0]
        return list(E), list(mu), list(n2)

    def grad(self, psi, out=None, with_energy=False):
        self._chk(psi)
        out = self.empty() if out is None else out
        self._chk(out)
        if with_energy:
            E, mu = _dbuf(self.nbatch), _dbuf(self.nbatch)
            _check(load().gpe_grad(self.handle, _ptr(psi), _ptr(out), E, mu))
            return out, (E[0], mu[0]) if self.nbatch == 1 else (list(E), list(mu))
        _check(load().gpe_grad(self.handle, _ptr(psi), _ptr(out), None, None))
        return out

    def hessvec(self, psi, d, shift=0.0, out=None):
        self._chk(psi)
        self._chk(d)
        out = self.empty() if out is None else out
        self._chk(out)
        _check(load().gpe_hessvec(self.handle, _ptr(psi), _ptr(d), float(shift), _ptr(out)))
        return out

    def hess_min_eig(self, psi, max_iter=200, tol=1e-10):
        """gpe_hess_min_eig: the second-order certificate of Lemma 3.2 at psi,
        as (value, residual, Lanczos steps)."""
        self._chk(psi)
        lam, res, it = C.c_double(), C.c_double(), C.c_int()
        _check(load().gpe_hess_min_eig(self.handle, _ptr(psi), int(max_iter), float(tol), C.byref(lam),
                                       C.byref(res), C.byref(it)))
        return lam.value, res.value, it.value

    def feasible_step(self, psi, hpsi, tau, out=None, with_energy=False):
        self._chk(psi)
        self._chk(hpsi)
        out = self.empty() if out is None else out
        self._chk(out)
        if with_energy:
            E = _dbuf(self.nbatch)
            _check(load().gpe_feasible_step(self.handle, _ptr(psi), _ptr(hpsi), float(tau), _ptr(out), E))
            return out, (E[0] if self.nbatch == 1 else list(E))
        _check(load().gpe_feasible_step(self.handle, _ptr(psi), _ptr(hpsi), float(tau), _ptr(out), None))
        return out

    def prolong_to(self, fine, psi_c, out=None):
        self._chk(psi_c)
        out = fine.empty() if out is None else out
        fine._chk(out)
        _check(load().gpe_prolong(self.handle, fine.handle, _ptr(psi_c), _ptr(out)))
        return out

    def autotune(self, levels=1):
        """gpe_plan_autotune: measure and record the launch shapes for this
        plan's grid (and `levels` - 1 coarser cascade grids)."""
        _check(load().gpe_plan_autotune(self.handle, levels))

    def solve(self, psi, **opts):
        """gpe_rnewton_solve in place on psi; returns the report as a dict."""
        self._chk(psi)
        o = SolveOpts()
        _check(load().gpe_solve_opts_default(C.byref(o)))
        for k, v in opts.items():
            if not hasattr(o, k):
                raise KeyError(k)
            setattr(o, k, v)
        r = SolveReport()
        _check(load().gpe_rnewton_solve(self.handle, _ptr(psi), C.byref(o), C.byref(r)), allow=(5,))
        return r.as_dict()


def autotune_report():
    """The choices recorded by gpe_plan_autotune in this process (text)."""
    buf = C.create_string_buffer(4096)
    _check(load().gpe_autotune_report(buf, len(buf)))
    return buf.value.decode()


def solve_batch(params_list, psis, stream=None, **opts):
    """gpe_solve_batch: float32 Algorithm 1 for many independent problems in
    one call.  params_list[i] is a workload parameter dict (2D Fourier, up to
    256^2), psis[i] a contiguous CUDA tensor of its grid (complex64 or float32),
    updated in place.  Returns the reports as a list of dicts."""
    import torch
    n = len(params_list)
    if n != len(psis) or n == 0:
        raise ValueError("need one psi per problem")
    probs = (Problem * n)(*[Problem.from_params(p) for p in params_list])
    for t in psis:
        if not t.is_cuda or not t.is_contiguous() or t.dtype not in (torch.complex64, torch.float32):
            raise ValueError("psi tensors must be contiguous CUDA complex64/float32")
    ptrs = (C.c_void_p * n)(*[t.data_ptr() for t in psis])
    o = SolveOpts()
    _check(load().gpe_solve_opts_default(C.byref(o)))
    for k, v in opts.items():
        if not hasattr(o, k):
            raise KeyError(k)
        setattr(o, k, v)
    reps = (SolveReport * n)()
    if stream is None:
        stream = torch.cuda.current_stream()
    _check(load().gpe_solve_batch(probs, n, ptrs, C.byref(o), reps, C.c_void_p(stream.cuda_stream)))
    return [r.as_dict() for r in reps]


def kernel_launches():
    """Kernels launched through libgpe by this process so far."""
    return int(load().gpe_kernel_launches())


def set_operator_path(path=0):
    """gpe_set_operator_path: 0 automatic, 1 fused 2D kernel, 2 two line kernels."""
    _check(load().gpe_set_operator_path(int(path)))


def set_wait_limit(polls=0):
    """gpe_set_wait_limit: polls after which a bounded device wait gives up
    (0 restores the defaults)."""
    _check(load().gpe_set_wait_limit(int(polls)))


def probe_peak(kind, stream=None):
    """gpe_probe_peak: measured multiply-add rate of the current device in
    TFLOP/s; kind 0 float32, 1 packed two-lane float32, 2 float64."""
    import torch
    if stream is None:
        stream = torch.cuda.current_stream()
    out = C.c_double()
    _check(load().gpe_probe_peak(int(kind), C.c_void_p(stream.cuda_stream), C.byref(out)))
    return float(out.value)


def profile_enable(on=True):
    _check(load().gpe_profile_enable(1 if on else 0))


def profile_summary():
    """{kernel-name: (launches, total_ms)} of the launches recorded since
    profile_enable(True)."""
    import json
    buf = C.create_string_buffer(1 << 16)
    _check(load().gpe_profile_summary(buf, len(buf)))
    return {k: (int(v[0]), float(v[1])) for k, v in json.loads(buf.value.decode()).items()}


def default_opts():
    o = SolveOpts()
    _check(load().gpe_solve_opts_default(C.byref(o)))
    return {k: getattr(o, k) for k, _ in o._fields_}


def to_device(arr, prec=F64):
    """numpy grid function -> contiguous CUDA tensor of the plan dtype."""
    import torch
    a = np.ascontiguousarray(arr)
    if np.iscomplexobj(a):
        t = torch.from_numpy(a.astype(np.complex64 if prec == F32 else np.complex128))
    else:
        t = torch.from_numpy(a.astype(np.float32 if prec == F32 else np.float64))
    return t.cuda()


def unit_scale(h_vol):
    return math.sqrt(h_vol)
