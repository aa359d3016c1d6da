"""ctypes binding of libsplitctmrg.so (names follow include/splitctmrg.h)."""
from __future__ import annotations

import ctypes
import os

import numpy as np
import torch

__all__ = [
    "load_library", "Config", "sctm_create", "sctm_destroy", "split_ctmrg_init", "split_ctmrg_move",
    "split_ctmrg_sweeps", "split_ctmrg_run", "ctmrg_projectors", "energy_2x2", "energy_grad", "energy_grad_host",
    "energy_grad_implicit", "sctm_get_env", "sctm_workspace_high_water", "sctm_set_limits", "sctm_autotune", "sctm_autotune_table", "sctm_profile", "sctm_svd", "sctm_svd_noalloc", "sctm_einsum", "SplitCTMRG", "ENV_KEYS", "SctmError",
]

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libsplitctmrg.so")
ENV_KEYS = ("C1", "T1k", "T1b", "C2", "T2k", "T2b", "C3", "T3b", "T3k", "C4", "T4b", "T4k")
CONV_KEYS = ("C1", "T1", "C2", "T2", "C3", "T3", "C4", "T4")
_ERRORS = {-1: "ERR_ARG", -2: "ERR_CUDA", -3: "ERR_SVD_NOCONV", -4: "ERR_NONFINITE", -5: "ERR_OOM",
           -6: "ERR_STATE", -7: "ERR_NOT_FIXED_POINT", -8: "ERR_NO_CONVERGENCE"}


class SctmError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"{_ERRORS.get(code, code)}: {msg}")
        self.code = code


class Config(ctypes.Structure):
    _fields_ = [("Lx", ctypes.c_int), ("Ly", ctypes.c_int), ("p", ctypes.c_int), ("D", ctypes.c_int),
                ("chi", ctypes.c_int), ("precision", ctypes.c_int), ("svd_cutoff", ctypes.c_double),
                ("lorentz_eps", ctypes.c_double), ("workspace_bytes", ctypes.c_size_t),
                ("power_steps", ctypes.c_int), ("randomized_min", ctypes.c_int),
                ("adjoint_cg_steps", ctypes.c_int), ("adjoint_band", ctypes.c_int),
                ("rank_extra", ctypes.c_int), ("algorithm", ctypes.c_int), ("chi_I", ctypes.c_int),
                ("projector_order", ctypes.c_int)]


_lib = None
_ip = ctypes.POINTER(ctypes.c_int)
_dp = ctypes.POINTER(ctypes.c_double)


def load_library(path: str = LIB_PATH):
    """Load the in-tree library (build it with ``paper_2502_10298_gb300.build``)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError(f"libsplitctmrg.so not found at {path}; run paper_2502_10298_gb300/build.py")
    lib = ctypes.CDLL(path)
    vp, i, d = ctypes.c_void_p, ctypes.c_int, ctypes.c_double
    sig = {
        "sctm_create": (i, [ctypes.POINTER(Config), vp, ctypes.POINTER(vp)]),
        "sctm_destroy": (i, [vp]),
        "sctm_last_error": (ctypes.c_char_p, [vp]),
        "split_ctmrg_init": (i, [vp, vp]),
        "split_ctmrg_move": (i, [vp, i]),
        "split_ctmrg_sweeps": (i, [vp, i]),
        "split_ctmrg_run": (i, [vp, i, d, _ip, _dp]),
        "ctmrg_projectors": (i, [vp, i, i, i, i, vp, vp, _dp]),
        "energy_2x2": (i, [vp, _dp, _dp, _dp]),
        "energy_grad": (i, [vp, vp, i, _dp, _dp, _dp, vp]),
        "energy_grad_host": (i, [vp, _dp, i, _dp, _dp, _dp, _dp]),
        "energy_grad_implicit": (i, [vp, vp, i, d, _dp, _dp, d, d, i, i, _dp, vp, _ip, _ip, _ip, _dp]),
        "sctm_get_env": (i, [vp, i, i, vp]),
        "sctm_workspace_high_water": (i, [vp, ctypes.POINTER(ctypes.c_size_t)]),
        "sctm_profile": (i, [vp, i, _dp]),
        "sctm_svd": (i, [vp, i, i, vp, vp, vp, vp]),
        "sctm_einsum": (i, [vp, ctypes.c_char_p, vp, _ip, vp, _ip, vp, _ip, d, d]),
        "sctm_svd_noalloc": (i, [i, i, vp, vp, vp, vp, vp]),
        "sctm_set_limits": (i, [vp, i, d]),
        "sctm_autotune": (i, [vp, i]),
        "sctm_autotune_table": (i, [vp, _dp, i, _ip]),
    }
    for name, (res, args) in sig.items():
        f = getattr(lib, name)
        f.restype, f.argtypes = res, args
    _lib = lib
    return lib


def _check(h, rc):
    if rc != 0:
        msg = _lib.sctm_last_error(h).decode() if h else "create failed"
        raise SctmError(rc, msg)


def _hp(a):
    """host float64 array -> (keep-alive array, pointer)"""
    if a is None:
        return None, None
    arr = np.ascontiguousarray(np.asarray(a, dtype=np.float64))
    return arr, arr.ctypes.data_as(_dp)


def sctm_create(Lx, Ly, p, D, chi, precision=0, svd_cutoff=0.0, lorentz_eps=0.0, workspace_bytes=0,
                stream=None, power_steps=0, randomized_min=0, adjoint_cg_steps=0, adjoint_band=0, algorithm=0,
                rank_extra=0, projector_order=0, chi_I=0):
    lib = load_library()
    cfg = Config(Lx, Ly, p, D, chi, precision, svd_cutoff, lorentz_eps, workspace_bytes, power_steps,
                 randomized_min, adjoint_cg_steps, adjoint_band, rank_extra, algorithm, chi_I, projector_order)
    if stream is None:
        stream = torch.cuda.current_stream().cuda_stream
    h = ctypes.c_void_p()
    rc = lib.sctm_create(ctypes.byref(cfg), ctypes.c_void_p(stream), ctypes.byref(h))
    if rc != 0:
        raise SctmError(rc, "sctm_create failed")
    return h


def sctm_destroy(h):
    _check(h, _lib.sctm_destroy(h))


def _dev(t: torch.Tensor):
    assert t.is_cuda and t.dtype == torch.float64 and t.is_contiguous(), "need a contiguous CUDA float64 tensor"
    return ctypes.c_void_p(t.data_ptr())


def split_ctmrg_init(h, A_cell: torch.Tensor):
    _check(h, _lib.split_ctmrg_init(h, _dev(A_cell)))


def split_ctmrg_move(h, direction: int):
    _check(h, _lib.split_ctmrg_move(h, int(direction)))


def split_ctmrg_sweeps(h, n: int):
    _check(h, _lib.split_ctmrg_sweeps(h, int(n)))


def split_ctmrg_run(h, max_sweeps: int, tol: float = 0.0):
    """Steps until the corner spectra change by less than tol (0: the default
    of the precision); returns (steps done, last delta)."""
    n, dl = ctypes.c_int(), ctypes.c_double()
    _check(h, _lib.split_ctmrg_run(h, int(max_sweeps), float(tol), ctypes.byref(n), ctypes.byref(dl)))
    return n.value, dl.value


def ctmrg_projectors(h, direction, x, y, colour, chi, alpha):
    """P_up [chi][alpha], P_dn [alpha][chi] and the chi kept singular values
    (chi: chi_E for green and teal, chi_I for yellow and red)."""
    up = torch.empty((chi, alpha), dtype=torch.float64, device="cuda")
    dn = torch.empty((alpha, chi), dtype=torch.float64, device="cuda")
    s = np.zeros(chi)
    _check(h, _lib.ctmrg_projectors(h, direction, x, y, colour, _dev(up), _dev(dn), s.ctypes.data_as(_dp)))
    return up, dn, s


def energy_2x2(h, h_nn, h_diag=None) -> float:
    a, pa = _hp(h_nn)
    b, pb = _hp(h_diag)
    e = ctypes.c_double()
    _check(h, _lib.energy_2x2(h, pa, pb, ctypes.byref(e)))
    return e.value


def energy_grad(h, A_cell: torch.Tensor, sweeps: int, h_nn, h_diag=None):
    a, pa = _hp(h_nn)
    b, pb = _hp(h_diag)
    g = torch.empty_like(A_cell)
    e = ctypes.c_double()
    _check(h, _lib.energy_grad(h, _dev(A_cell), int(sweeps), pa, pb, ctypes.byref(e), _dev(g)))
    return e.value, g


def energy_grad_host(h, A_cell: np.ndarray, sweeps: int, h_nn, h_diag=None, grad_out: np.ndarray = None):
    A_cell = np.ascontiguousarray(A_cell, dtype=np.float64)
    if grad_out is None:
        grad_out = np.empty_like(A_cell)
    a, pa = _hp(h_nn)
    b, pb = _hp(h_diag)
    e = ctypes.c_double()
    _check(h, _lib.energy_grad_host(h, A_cell.ctypes.data_as(_dp), int(sweeps), pa, pb, ctypes.byref(e),
                                    grad_out.ctypes.data_as(_dp)))
    return e.value, grad_out


def energy_grad_implicit(h, A_cell: torch.Tensor, h_nn, h_diag=None, max_sweeps: int = 300, tol: float = 0.0,
                         fixed_point_tol: float = 0.0, solve_tol: float = 0.0, max_iter: int = 500,
                         max_period: int = 4):
    """(E, grad, info) by implicit differentiation of the converged environment
    as a fixed point of `period` full steps; info = dict(sweeps, period,
    solver_iterations, fixed_point_change).  Zero tolerances take the library
    defaults."""
    a, pa = _hp(h_nn)
    b, pb = _hp(h_diag)
    g = torch.empty_like(A_cell)
    e = ctypes.c_double()
    n, per, it, fp = ctypes.c_int(), ctypes.c_int(), ctypes.c_int(), ctypes.c_double()
    _check(h, _lib.energy_grad_implicit(h, _dev(A_cell), int(max_sweeps), float(tol), pa, pb, float(fixed_point_tol),
                                        float(solve_tol), int(max_iter), int(max_period), ctypes.byref(e), _dev(g),
                                        ctypes.byref(n), ctypes.byref(per), ctypes.byref(it), ctypes.byref(fp)))
    return e.value, g, {"sweeps": n.value, "period": per.value, "solver_iterations": it.value,
                        "fixed_point_change": fp.value}


def sctm_get_env(h, x, y, chi, D, conventional=False, chi_I=None):
    """Environment of site (x, y): split keys (C1, T1k, T1b, ...) or, for the
    conventional algorithm, C1, T1, C2, T2, C3, T3, C4, T4 with fused edges.
    chi is chi_E; chi_I (default chi) the interlayer bond of the split edges."""
    keys = CONV_KEYS if conventional else ENV_KEYS
    ci = chi if not chi_I else chi_I
    def shape(k):
        if k[0] == "C":
            return (chi, chi)
        if conventional:
            return (chi, D, D, chi)
        return (chi, D, ci) if k in ("T1k", "T2k", "T3b", "T4b") else (ci, D, chi)
    sizes = [int(np.prod(shape(k))) for k in keys]
    buf = torch.empty(sum(sizes), dtype=torch.float64, device="cuda")
    _check(h, _lib.sctm_get_env(h, x, y, _dev(buf)))
    out, off = {}, 0
    for k, n in zip(keys, sizes):
        out[k] = buf[off:off + n].view(shape(k))
        off += n
    return out


PROFILE_FAMILIES = ("contract", "svd", "other", "tensor")


def sctm_profile(h, enable: bool):
    """enable=True starts per-family event timing; enable=False returns
    {family: dict(ms, launches, flops, bytes)} and stops it."""
    out = np.zeros(4 * len(PROFILE_FAMILIES))
    _check(h, _lib.sctm_profile(h, 1 if enable else 0, out.ctypes.data_as(_dp)))
    if enable:
        return None
    return {f: dict(ms=out[4 * i], launches=int(out[4 * i + 1]), flops=out[4 * i + 2], bytes=out[4 * i + 3])
            for i, f in enumerate(PROFILE_FAMILIES)}


def sctm_svd(h, M: torch.Tensor):
    """(U, S, V) of a CUDA float64 matrix with rows >= columns (one-sided Jacobi)."""
    m, n = M.shape
    M = M.contiguous()
    U = torch.empty((m, n), dtype=torch.float64, device=M.device)
    S = torch.empty((n,), dtype=torch.float64, device=M.device)
    V = torch.empty((n, n), dtype=torch.float64, device=M.device)
    _check(h, _lib.sctm_svd(h, m, n, _dev(M), _dev(U), _dev(S), _dev(V)))
    return U, S, V


def sctm_einsum(h, spec: str, A: torch.Tensor, B: torch.Tensor, C: torch.Tensor = None, alpha=1.0, beta=0.0,
                out_shape=None):
    """C = alpha * einsum(spec, A, B) + beta * C on CUDA float64 tensors, in the
    handle's precision (3xTF32 tensor cores for large contractions when mixed)."""
    A, B = A.contiguous(), B.contiguous()
    if C is None:
        ins, out = spec.split("->")
        la, lb = ins.split(",")
        size = dict(zip(la, A.shape))
        size.update(zip(lb, B.shape))
        C = torch.empty([size[ch] for ch in out], dtype=torch.float64, device=A.device)
    assert C.is_contiguous()
    def shp(t):
        return (ctypes.c_int * t.dim())(*t.shape)
    sa, sb, sc = shp(A), shp(B), shp(C)
    _check(h, _lib.sctm_einsum(h, spec.encode(), _dev(A), sa, _dev(B), sb, _dev(C), sc, float(alpha), float(beta)))
    return C


def sctm_svd_noalloc(M: torch.Tensor, U=None, S=None, V=None):
    """(U, S, V) of a CUDA float64 matrix (rows >= columns, (m + n) n <= 2^21)
    through the handle-free entry point that allocates no device memory; the
    output buffers may be passed in (allocated beforehand by the caller)."""
    load_library()
    m, n = M.shape
    assert M.is_contiguous()
    U = torch.empty((m, n), dtype=torch.float64, device=M.device) if U is None else U
    S = torch.empty((n,), dtype=torch.float64, device=M.device) if S is None else S
    V = torch.empty((n, n), dtype=torch.float64, device=M.device) if V is None else V
    # the library takes the scratch of the current device: make M's device current
    with torch.cuda.device(M.device):
        rc = _lib.sctm_svd_noalloc(m, n, _dev(M), _dev(U), _dev(S), _dev(V),
                                   ctypes.c_void_p(torch.cuda.current_stream(M.device).cuda_stream))
    if rc != 0:
        raise SctmError(rc, "sctm_svd_noalloc failed")
    return U, S, V


def sctm_set_limits(h, svd_max_sweeps: int = 0, pipeline_wait_s: float = -1.0):
    """Bounded-loop limits of the handle (fault-injection hook): Jacobi sweeps
    (<= 0: default) and the tensor-core main-loop wait (< 0: default 2 s)."""
    _check(h, _lib.sctm_set_limits(h, int(svd_max_sweeps), float(pipeline_wait_s)))


def sctm_autotune(h, enable: bool):
    """Explore K-split counts of small-output contractions from now on (True),
    or stop exploring (False); tuned shapes keep their choice."""
    _check(h, _lib.sctm_autotune(h, 1 if enable else 0))


TUNE_KERNELS = ("fp64_cuda_cores", "fp32_cuda_cores", "tf32x3_tensor_cores", "bf16_slices_tensor_cores")


def sctm_autotune_table(h):
    """The tuner's choices: one dict per tuned shape."""
    n = ctypes.c_int()
    _check(h, _lib.sctm_autotune_table(h, None, 0, ctypes.byref(n)))
    out = np.zeros(9 * max(1, n.value))
    _check(h, _lib.sctm_autotune_table(h, out.ctypes.data_as(_dp), n.value, ctypes.byref(n)))
    rows = []
    for r in out[:9 * n.value].reshape(-1, 9):
        rows.append(dict(kernel=TUNE_KERNELS[int(r[0])], batch=int(r[1]), M=int(r[2]), N=int(r[3]), K=int(r[4]),
                         rule_splits=int(r[5]), rule_ms=float(r[6]), chosen_splits=int(r[7]), chosen_ms=float(r[8])))
    return rows


def sctm_workspace_high_water(h) -> int:
    v = ctypes.c_size_t()
    _check(h, _lib.sctm_workspace_high_water(h, ctypes.byref(v)))
    return v.value


class SplitCTMRG:
    """Owning wrapper: ``with SplitCTMRG(Lx, Ly, p, D, chi) as s: ...``"""

    def __init__(self, Lx, Ly, p, D, chi, **kw):
        self.Lx, self.Ly, self.p, self.D, self.chi = Lx, Ly, p, D, chi
        self.conventional = kw.get("algorithm", 0) == 1
        self.order = kw.get("projector_order", 0)
        self.chiI = kw.get("chi_I", 0) or chi
        self.h = sctm_create(Lx, Ly, p, D, chi, **kw)

    def close(self):
        if self.h is not None:
            sctm_destroy(self.h)
            self.h = None

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def init(self, A):
        split_ctmrg_init(self.h, A)

    def move(self, d):
        split_ctmrg_move(self.h, d)

    def sweeps(self, n):
        split_ctmrg_sweeps(self.h, n)

    def run(self, max_sweeps, tol=0.0):
        return split_ctmrg_run(self.h, max_sweeps, tol)

    def env(self, x, y):
        return sctm_get_env(self.h, x, y, self.chi, self.D, self.conventional, self.chiI)

    def energy(self, h_nn, h_diag=None):
        return energy_2x2(self.h, h_nn, h_diag)

    def energy_grad(self, A, sweeps, h_nn, h_diag=None):
        return energy_grad(self.h, A, sweeps, h_nn, h_diag)

    def energy_grad_implicit(self, A, h_nn, h_diag=None, **kw):
        return energy_grad_implicit(self.h, A, h_nn, h_diag, **kw)

    def projectors(self, direction, x, y, colour):
        # the colour that carries the physical leg: red (order 0) or yellow (order 1)
        phys = (colour == 3) if self.order == 0 else (colour == 2)
        k = self.chi if colour in (0, 1) else self.chiI      # green, teal: chi_E; yellow, red: chi_I
        alpha = k * self.D * (self.p if phys else 1)
        return ctmrg_projectors(self.h, direction, x, y, colour, k, alpha)
