"""Python binding of the GB300 gDC library (libgdc.so, C ABI declared in include/gdc.h).

Argument marshalling only: every step of the method runs in the library's CUDA
kernels.  PyTorch supplies device memory (the workspace and the state arrays)
and the stream.  There is no CPU fallback: importing works without a GPU, but
creating a Context without the built library or without a CUDA device raises.
"""
from __future__ import annotations

import ctypes
import dataclasses
import os
from typing import List, Optional, Sequence

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libgdc.so")

FP64 = 0
FP32_MIXED = 1
DIV_RFD = 0
DIV_FD = 1
SCHEME_GDC = 0
SCHEME_EM = 1
POT_SOFT = 0
POT_REPEL_ATTRACT = 1
POT_REPEL_ATTRACT_REPEL = 2
FORCES_CHOOSE = 0
FORCES_ALL_PAIRS = 1
FORCES_CELL_LIST = 2
MOB_RPY = 0
MOB_FCM = 1

STATUS = {0: "OK", 1: "INVALID_ARG", 2: "CUDA", 3: "NOT_CONVERGED", 4: "NONFINITE", 5: "TIMEOUT", 6: "WORKSPACE"}

# every entry point the header declares
EXPORTS = [
    "gdc_workspace_bytes", "gdc_init", "gdc_destroy", "gdc_last_error", "gdc_set_params",
    "gdc_mobility_solve", "gdc_step", "gdc_set_trace", "gdc_get_state", "gdc_set_state",
    "gdc_blob_positions", "gdc_rpy_apply", "gdc_saddle_apply", "gdc_precond_apply",
    "gdc_brownian_slip", "gdc_lsq_velocity", "gdc_forces", "gdc_draw_normals", "gdc_saddle_offsets",
    "gdc_profile", "gdc_profile_read", "gdc_rpy_apply_noalloc", "gdc_debug_wait_polls",
    "gdc_fcm_workspace_bytes", "gdc_fcm_init", "gdc_fcm_apply", "gdc_fcm_brownian", "gdc_fcm_average",
    "gdc_fcm_last_error", "gdc_fcm_launches", "gdc_fcm_destroy", "gdc_fma_probe",
]

NOALLOC_MAX_BLOBS = 16384   # GDC_NOALLOC_MAX_BLOBS of include/gdc.h


class GdcError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"gdc {STATUS.get(status, status)}: {msg}")
        self.status = status


class _Params(ctypes.Structure):
    _fields_ = [("eta", ctypes.c_double), ("kT", ctypes.c_double), ("a", ctypes.c_double), ("dt", ctypes.c_double),
                ("gmres_tol", ctypes.c_double), ("gmres_max_iter", ctypes.c_int), ("gmres_restart", ctypes.c_int),
                ("lanczos_tol", ctypes.c_double), ("lanczos_max_iter", ctypes.c_int), ("rfd_delta", ctypes.c_double),
                ("precision", ctypes.c_int), ("divmode", ctypes.c_int), ("scheme", ctypes.c_int),
                ("rep_A", ctypes.c_double), ("rep_b", ctypes.c_double), ("shear_rate", ctypes.c_double),
                ("seed", ctypes.c_ulonglong), ("autotune", ctypes.c_int), ("graph", ctypes.c_int),
                ("pair_kernel", ctypes.c_int), ("potential", ctypes.c_int), ("well_A", ctypes.c_double),
                ("well_lambda", ctypes.c_double), ("force_method", ctypes.c_int), ("mobility", ctypes.c_int),
                ("box_L", ctypes.c_double), ("fcm_N", ctypes.c_int), ("fcm_sigma", ctypes.c_double),
                ("fcm_R_t", ctypes.c_double), ("lanczos_precond", ctypes.c_int), ("wall", ctypes.c_int),
                ("wall_V0", ctypes.c_double), ("wall_b", ctypes.c_double), ("body_weight", ctypes.c_double),
                ("df_kernel", ctypes.c_int)]


class _FcmParams(ctypes.Structure):
    _fields_ = [("N", ctypes.c_int), ("L", ctypes.c_double), ("sigma", ctypes.c_double), ("R_t", ctypes.c_double),
                ("eta", ctypes.c_double), ("max_blobs", ctypes.c_int)]


class _SolveInfo(ctypes.Structure):
    _fields_ = [("iterations", ctypes.c_int), ("cycles", ctypes.c_int), ("matvecs_fp32", ctypes.c_int),
                ("matvecs_fp64", ctypes.c_int), ("residual", ctypes.c_double), ("converged", ctypes.c_int)]


class _StepInfo(ctypes.Structure):
    _fields_ = [("step", ctypes.c_ulonglong), ("lanczos_iters", ctypes.c_int * 3), ("lanczos_err", ctypes.c_double),
                ("solve", _SolveInfo), ("nu_min", ctypes.c_double), ("nu_max", ctypes.c_double),
                ("pair_evals", ctypes.c_double)]


class _Profile(ctypes.Structure):
    _fields_ = [("launches", ctypes.c_ulonglong), ("rpy32_launches", ctypes.c_ulonglong),
                ("rpy64_launches", ctypes.c_ulonglong), ("force_launches", ctypes.c_ulonglong),
                ("rpy32_ms", ctypes.c_double), ("rpy64_ms", ctypes.c_double), ("force_ms", ctypes.c_double),
                ("pairs_per_product", ctypes.c_double), ("targets_per_thread", ctypes.c_int),
                ("work_waves", ctypes.c_double), ("autotune_ms", ctypes.c_double),
                ("rpydf_launches", ctypes.c_ulonglong), ("rpydf_ms", ctypes.c_double),
                ("pair_kernel", ctypes.c_int), ("sym_width", ctypes.c_int),
                ("unique_pairs_per_product", ctypes.c_double), ("min_blocks_per_sm", ctypes.c_int),
                ("df_kernel", ctypes.c_int)]


class _Trace(ctypes.Structure):
    _fields_ = [(n, ctypes.c_void_p) for n in ("calV", "nu", "Ym", "qm", "Vm", "vb_n", "vb_m", "FTm")]


@dataclasses.dataclass
class Params:
    eta: float = 1.0
    kT: float = 1.0
    a: float = 1.0
    dt: float = 0.01
    gmres_tol: float = 1e-6
    gmres_max_iter: int = 500
    gmres_restart: int = 50
    lanczos_tol: float = 1e-4
    lanczos_max_iter: int = 64
    rfd_delta: float = 1e-6
    precision: int = FP64
    divmode: int = DIV_RFD
    scheme: int = SCHEME_GDC
    rep_A: float = 0.0
    rep_b: float = 0.1
    shear_rate: float = 0.0
    seed: int = 0
    autotune: int = 1
    graph: int = 1
    pair_kernel: int = 0
    potential: int = 0
    well_A: float = 0.0
    well_lambda: float = 0.5
    force_method: int = 0
    mobility: int = 0        # 0 unbounded RPY, 1 fluctuating FCM in a periodic cube
    box_L: float = 0.0
    fcm_N: int = 0
    fcm_sigma: float = 0.0   # 0: a / sqrt(pi)
    fcm_R_t: float = 0.0     # 0: 3a
    lanczos_precond: int = 1  # 1: block-preconditioned Lanczos (root L (L^-1 M L^-T)^(1/2)), 0: M^(1/2)
    wall: int = 0            # 1: blobs above a no-slip wall at z = 0 (wall-corrected RPY)
    wall_V0: float = 0.0     # wall repulsion strength (Sec. 6.2: 23 kT)
    wall_b: float = 0.5      # its range (Sec. 6.2: 0.5 a)
    body_weight: float = 0.0  # mg per body along -z (Sec. 6.2: 0.18 kT/a)
    df_kernel: int = 0       # double-float residual kernel: 0 as pair_kernel, 1 ordered, 3/4 symmetric

    def _c(self) -> _Params:
        return _Params(**{f.name: getattr(self, f.name) for f in dataclasses.fields(self)})


_lib = None


def load_library() -> ctypes.CDLL:
    """Load libgdc.so; raises if it has not been built (no fallback)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"{LIB_PATH} is missing: build it with python -m paper_2106_00449_gb300.build")
    lib = ctypes.CDLL(LIB_PATH)
    vp, cp, dp, ip, llp = ctypes.c_void_p, ctypes.c_char_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p
    lib.gdc_workspace_bytes.restype = ctypes.c_size_t
    lib.gdc_workspace_bytes.argtypes = [ctypes.POINTER(_Params), ctypes.c_int, ip, ctypes.c_int, llp, ip]
    lib.gdc_init.restype = ctypes.c_int
    lib.gdc_init.argtypes = [ctypes.POINTER(vp), ctypes.POINTER(_Params), ctypes.c_int, ip, dp, ctypes.c_int, llp, ip,
                             dp, dp, vp, ctypes.c_size_t, vp]
    lib.gdc_destroy.restype = None
    lib.gdc_fma_probe.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, vp, vp]
    lib.gdc_destroy.argtypes = [vp]
    lib.gdc_last_error.restype = cp
    lib.gdc_last_error.argtypes = [vp]
    lib.gdc_set_params.argtypes = [vp, ctypes.POINTER(_Params)]
    lib.gdc_mobility_solve.argtypes = [vp, dp, dp, dp, dp, ctypes.POINTER(_SolveInfo)]
    lib.gdc_step.argtypes = [vp, ctypes.c_int, ctypes.POINTER(_StepInfo)]
    lib.gdc_set_trace.argtypes = [vp, ctypes.POINTER(_Trace)]
    lib.gdc_get_state.argtypes = [vp, dp, dp, ctypes.POINTER(ctypes.c_ulonglong)]
    lib.gdc_set_state.argtypes = [vp, dp, dp, ctypes.c_ulonglong]
    lib.gdc_blob_positions.argtypes = [vp, dp]
    lib.gdc_rpy_apply.argtypes = [vp, ctypes.c_int, dp, dp]
    lib.gdc_saddle_apply.argtypes = [vp, ctypes.c_int, dp, dp]
    lib.gdc_precond_apply.argtypes = [vp, dp, dp]
    lib.gdc_brownian_slip.argtypes = [vp, dp, dp, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_double)]
    lib.gdc_lsq_velocity.argtypes = [vp, dp, dp]
    lib.gdc_forces.argtypes = [vp, dp]
    lib.gdc_draw_normals.argtypes = [vp, ctypes.c_ulonglong, ctypes.c_int, dp]
    lib.gdc_saddle_offsets.argtypes = [vp, llp]
    lib.gdc_profile.argtypes = [vp, ctypes.c_int]
    lib.gdc_profile_read.argtypes = [vp, ctypes.POINTER(_Profile)]
    lib.gdc_rpy_apply_noalloc.argtypes = [dp, dp, dp, ctypes.c_int, ctypes.c_double, ctypes.c_double, vp]
    lib.gdc_debug_wait_polls.restype = None
    lib.gdc_debug_wait_polls.argtypes = [ctypes.c_int]
    lib.gdc_fcm_workspace_bytes.restype = ctypes.c_size_t
    lib.gdc_fcm_workspace_bytes.argtypes = [ctypes.POINTER(_FcmParams)]
    lib.gdc_fcm_init.argtypes = [ctypes.POINTER(vp), ctypes.POINTER(_FcmParams), vp, ctypes.c_size_t, vp]
    lib.gdc_fcm_apply.argtypes = [vp, ctypes.c_int, dp, dp, dp]
    lib.gdc_fcm_brownian.argtypes = [vp, ctypes.c_ulonglong, ctypes.c_uint, ctypes.c_ulonglong, ctypes.c_double,
                                     ctypes.c_double, ctypes.c_int, dp, dp]
    lib.gdc_fcm_average.argtypes = [vp, ctypes.c_int, dp, dp]
    lib.gdc_fcm_last_error.restype = cp
    lib.gdc_fcm_last_error.argtypes = [vp]
    lib.gdc_fcm_launches.restype = ctypes.c_ulonglong
    lib.gdc_fcm_launches.argtypes = [vp]
    lib.gdc_fcm_destroy.restype = None
    lib.gdc_fcm_destroy.argtypes = [vp]
    for name in EXPORTS:
        if name not in ("gdc_workspace_bytes", "gdc_destroy", "gdc_last_error", "gdc_fcm_workspace_bytes",
                        "gdc_fcm_last_error", "gdc_fcm_launches", "gdc_fcm_destroy", "gdc_debug_wait_polls"):
            getattr(lib, name).restype = ctypes.c_int
    _lib = lib
    return lib


def _np_ptr(a: np.ndarray):
    return ctypes.c_void_p(a.ctypes.data)


def _dptr(t) -> ctypes.c_void_p:
    if t is None:
        return ctypes.c_void_p(0)
    if not (t.is_cuda and t.is_contiguous()):
        raise ValueError("expected a contiguous CUDA tensor")
    return ctypes.c_void_p(t.data_ptr())


def solve_info_dict(s: _SolveInfo) -> dict:
    return dict(iterations=s.iterations, cycles=s.cycles, matvecs_fp32=s.matvecs_fp32, matvecs_fp64=s.matvecs_fp64,
                residual=s.residual, converged=bool(s.converged))


def step_info_dict(s: _StepInfo) -> dict:
    return dict(step=s.step, lanczos_iters=list(s.lanczos_iters), lanczos_err=s.lanczos_err,
                solve=solve_info_dict(s.solve), nu_min=s.nu_min, nu_max=s.nu_max, pair_evals=s.pair_evals)


class Context:
    """One gDC context: S suspensions of rigid multiblob bodies on the current CUDA device.

    templates: list of (n_t, 3) body-frame blob coordinates; body_tmpl: template of each
    body; susp_body_off: (S+1,) body offsets; Y (N, 3), q (N, 4) initial state (host or device).
    """

    def __init__(self, params: Params, templates: Sequence[np.ndarray], body_tmpl, susp_body_off, Y, q,
                 device: int = 0, stream=None):
        import torch
        if not torch.cuda.is_available():
            raise RuntimeError("the gDC library needs a CUDA device")
        self.torch = torch
        self.lib = load_library()
        self.device = torch.device("cuda", device)
        self.stream = stream if stream is not None else torch.cuda.current_stream(self.device)
        self.params = dataclasses.replace(params)
        self.tmpl_n = np.ascontiguousarray([len(t) for t in templates], dtype=np.int32)
        self.tmpl_xyz = np.ascontiguousarray(np.concatenate([np.asarray(t, dtype=np.float64).reshape(-1) for t in templates]))
        self.body_tmpl = np.ascontiguousarray(body_tmpl, dtype=np.int32)
        self.susp_body_off = np.ascontiguousarray(susp_body_off, dtype=np.int64)
        self.n_susp = len(self.susp_body_off) - 1
        self.n_bodies = int(self.body_tmpl.shape[0])
        self.n_blobs = int(self.tmpl_n[self.body_tmpl].sum())
        cp = self.params._c()
        nbytes = self.lib.gdc_workspace_bytes(ctypes.byref(cp), len(templates), _np_ptr(self.tmpl_n), self.n_susp,
                                              _np_ptr(self.susp_body_off), _np_ptr(self.body_tmpl))
        if nbytes == 0:
            raise GdcError(1, "invalid sizes or parameters")
        self.workspace_bytes = int(nbytes)
        with torch.cuda.device(self.device):
            self.workspace = torch.empty(self.workspace_bytes + 256, dtype=torch.uint8, device=self.device)
            off = (-self.workspace.data_ptr()) % 256
            self._ws_ptr = self.workspace.data_ptr() + off
            self.Y = torch.as_tensor(np.asarray(Y, dtype=np.float64).reshape(-1, 3) if not hasattr(Y, "is_cuda") else Y,
                                     dtype=torch.float64, device=self.device).contiguous().clone()
            self.q = torch.as_tensor(np.asarray(q, dtype=np.float64).reshape(-1, 4) if not hasattr(q, "is_cuda") else q,
                                     dtype=torch.float64, device=self.device).contiguous().clone()
        h = ctypes.c_void_p(0)
        st = self.lib.gdc_init(ctypes.byref(h), ctypes.byref(cp), len(templates), _np_ptr(self.tmpl_n),
                               _np_ptr(self.tmpl_xyz), self.n_susp, _np_ptr(self.susp_body_off),
                               _np_ptr(self.body_tmpl), _dptr(self.Y), _dptr(self.q), ctypes.c_void_p(self._ws_ptr),
                               ctypes.c_size_t(self.workspace_bytes), ctypes.c_void_p(self.stream.cuda_stream))
        self._h = h
        if st != 0:
            msg = self.lib.gdc_last_error(h).decode()
            self.close()
            raise GdcError(st, msg)
        self._trace_keep = None
        off = np.zeros(self.n_susp + 1, dtype=np.int64)
        self._check(self.lib.gdc_saddle_offsets(self._h, _np_ptr(off)))
        self.saddle_off = off

    # -- lifetime --
    def close(self):
        if getattr(self, "_h", None) and self._h.value:
            self.lib.gdc_destroy(self._h)
        self._h = ctypes.c_void_p(0)

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _check(self, st: int):
        if st != 0:
            raise GdcError(st, self.lib.gdc_last_error(self._h).decode())

    def _dev(self, n, dtype=None):
        return self.torch.zeros(n, dtype=dtype or self.torch.float64, device=self.device)

    def _in(self, x, n):
        t = self.torch.as_tensor(x, dtype=self.torch.float64, device=self.device).reshape(-1).contiguous()
        if t.numel() != n:
            raise ValueError(f"expected {n} values, got {t.numel()}")
        return t

    # -- parameters / state --
    def set_params(self, params: Params):
        cp = params._c()
        self._check(self.lib.gdc_set_params(self._h, ctypes.byref(cp)))
        self.params = dataclasses.replace(params)

    def get_state(self):
        Y = np.zeros((self.n_bodies, 3))
        q = np.zeros((self.n_bodies, 4))
        step = ctypes.c_ulonglong(0)
        self._check(self.lib.gdc_get_state(self._h, _np_ptr(Y), _np_ptr(q), ctypes.byref(step)))
        return Y, q, int(step.value)

    def set_state(self, Y, q, step: int = 0):
        Yh = np.ascontiguousarray(Y, dtype=np.float64)
        qh = np.ascontiguousarray(q, dtype=np.float64)
        self._check(self.lib.gdc_set_state(self._h, _np_ptr(Yh), _np_ptr(qh), ctypes.c_ulonglong(step)))

    def set_state_host_ptr(self, Y_ptr: int, q_ptr: int, step: int):
        self._check(self.lib.gdc_set_state(self._h, ctypes.c_void_p(Y_ptr), ctypes.c_void_p(q_ptr),
                                           ctypes.c_ulonglong(step)))

    def get_state_host_ptr(self, Y_ptr: int, q_ptr: int) -> int:
        step = ctypes.c_ulonglong(0)
        self._check(self.lib.gdc_get_state(self._h, ctypes.c_void_p(Y_ptr), ctypes.c_void_p(q_ptr), ctypes.byref(step)))
        return int(step.value)

    # -- the method --
    def step(self, nsteps: int = 1, info: bool = True) -> List[dict]:
        if not info:
            self._check(self.lib.gdc_step(self._h, nsteps, None))
            return []
        arr = (_StepInfo * max(nsteps, 1))()
        self._check(self.lib.gdc_step(self._h, nsteps, arr))
        return [step_info_dict(arr[k]) for k in range(nsteps)]

    def mobility_solve(self, FT, vbrev=None, want_lambda: bool = False):
        FTt = self._in(FT, 6 * self.n_bodies)
        vbt = None if vbrev is None else self._in(vbrev, 3 * self.n_blobs)
        V = self._dev(6 * self.n_bodies)
        lam = self._dev(3 * self.n_blobs) if want_lambda else None
        inf = _SolveInfo()
        self._check(self.lib.gdc_mobility_solve(self._h, _dptr(FTt), _dptr(vbt), _dptr(V), _dptr(lam), ctypes.byref(inf)))
        return V, lam, solve_info_dict(inf)

    def set_trace(self, enable: bool = True) -> Optional[dict]:
        if not enable:
            self._check(self.lib.gdc_set_trace(self._h, None))
            self._trace_keep = None
            return None
        bufs = dict(calV=self._dev(6 * self.n_bodies), nu=self._dev(self.n_susp), Ym=self._dev(3 * self.n_bodies),
                    qm=self._dev(4 * self.n_bodies), Vm=self._dev(6 * self.n_bodies), vb_n=self._dev(3 * self.n_blobs),
                    vb_m=self._dev(3 * self.n_blobs), FTm=self._dev(6 * self.n_bodies))
        tr = _Trace(**{k: v.data_ptr() for k, v in bufs.items()})
        self._check(self.lib.gdc_set_trace(self._h, ctypes.byref(tr)))
        self._trace_keep = bufs
        return bufs

    # -- instrumentation --
    def profile(self, enable: bool = True):
        self._check(self.lib.gdc_profile(self._h, 1 if enable else 0))

    def profile_read(self) -> dict:
        p = _Profile()
        self._check(self.lib.gdc_profile_read(self._h, ctypes.byref(p)))
        return {f[0]: getattr(p, f[0]) for f in _Profile._fields_}

    # -- building blocks --
    def blob_positions(self):
        r = self._dev(3 * self.n_blobs)
        self._check(self.lib.gdc_blob_positions(self._h, _dptr(r)))
        return r

    def rpy_apply(self, lam, precision: int = FP64):
        lt = self._in(lam, 3 * self.n_blobs)
        u = self._dev(3 * self.n_blobs)
        self._check(self.lib.gdc_rpy_apply(self._h, precision, _dptr(lt), _dptr(u)))
        return u

    def saddle_apply(self, x, precision: int = FP64):
        xt = self._in(x, int(self.saddle_off[-1]))
        y = self._dev(int(self.saddle_off[-1]))
        self._check(self.lib.gdc_saddle_apply(self._h, precision, _dptr(xt), _dptr(y)))
        return y

    def precond_apply(self, r):
        rt = self._in(r, int(self.saddle_off[-1]))
        z = self._dev(int(self.saddle_off[-1]))
        self._check(self.lib.gdc_precond_apply(self._h, _dptr(rt), _dptr(z)))
        return z

    def brownian_slip(self, W):
        Wt = self._in(W, 3 * self.n_blobs)
        out = self._dev(3 * self.n_blobs)
        it = ctypes.c_int(0)
        err = ctypes.c_double(0)
        self._check(self.lib.gdc_brownian_slip(self._h, _dptr(Wt), _dptr(out), ctypes.byref(it), ctypes.byref(err)))
        return out, int(it.value), float(err.value)

    def lsq_velocity(self, vbrev):
        vt = self._in(vbrev, 3 * self.n_blobs)
        out = self._dev(6 * self.n_bodies)
        self._check(self.lib.gdc_lsq_velocity(self._h, _dptr(vt), _dptr(out)))
        return out

    def forces(self):
        out = self._dev(6 * self.n_bodies)
        self._check(self.lib.gdc_forces(self._h, _dptr(out)))
        return out

    def draw_normals(self, step: int, stream: int):
        n = 3 * self.n_blobs if stream == 0 else 6 * self.n_bodies
        out = self._dev(n)
        self._check(self.lib.gdc_draw_normals(self._h, ctypes.c_ulonglong(step), stream, _dptr(out)))
        return out


class Fcm:
    """Fluctuating FCM in a periodic cube of side L on an N^3 grid (C ABI gdc_fcm_*).

    sigma: envelope width (a / sqrt(pi) matches the RPY self-mobility); R_t: envelope
    truncation radius (3a in Sec. 6.1).  Positions and forces are (n, 3) float64 tensors on
    the context's device; every call returns a new (n, 3) tensor.
    """

    def __init__(self, N: int, L: float, sigma: float, R_t: float, eta: float = 1.0, max_blobs: int = 1,
                 device: int = 0, stream=None):
        import torch
        if not torch.cuda.is_available():
            raise RuntimeError("the gDC library needs a CUDA device")
        self.torch = torch
        self.lib = load_library()
        self.device = torch.device("cuda", device)
        self.stream = stream if stream is not None else torch.cuda.current_stream(self.device)
        self.params = _FcmParams(int(N), float(L), float(sigma), float(R_t), float(eta), int(max_blobs))
        nbytes = int(self.lib.gdc_fcm_workspace_bytes(ctypes.byref(self.params)))
        if nbytes == 0:
            raise GdcError(1, "invalid FCM parameters")
        self.workspace = torch.empty(nbytes + 256, dtype=torch.uint8, device=self.device)
        ptr = self.workspace.data_ptr() + (-self.workspace.data_ptr()) % 256
        h = ctypes.c_void_p(0)
        st = self.lib.gdc_fcm_init(ctypes.byref(h), ctypes.byref(self.params), ctypes.c_void_p(ptr),
                                   ctypes.c_size_t(nbytes), ctypes.c_void_p(self.stream.cuda_stream))
        if st != 0:
            raise GdcError(st, "gdc_fcm_init failed")
        self._h = h

    def _vec(self, x):
        t = self.torch.as_tensor(x, dtype=self.torch.float64, device=self.device).reshape(-1, 3).contiguous()
        return t

    def _check(self, st):
        if st != 0:
            raise GdcError(st, self.lib.gdc_fcm_last_error(self._h).decode())

    def apply(self, r, lam):
        """u = M_FCM lambda (Sec. 4.2)."""
        r, lam = self._vec(r), self._vec(lam)
        u = self.torch.empty_like(r)
        self._check(self.lib.gdc_fcm_apply(self._h, r.shape[0], _dptr(r), _dptr(lam), _dptr(u)))
        return u

    def brownian(self, r, seed: int, owner: int, step: int, kT: float, dt: float):
        """v-breve = J L^-1 D W for the stress of (seed, owner, step); keeps u-breve for average()."""
        r = self._vec(r)
        v = self.torch.empty_like(r)
        self._check(self.lib.gdc_fcm_brownian(self._h, int(seed), int(owner), int(step), float(kT), float(dt),
                                              r.shape[0], _dptr(r), _dptr(v)))
        return v

    def average(self, r):
        """J u-breve of the last brownian() at positions r."""
        r = self._vec(r)
        v = self.torch.empty_like(r)
        self._check(self.lib.gdc_fcm_average(self._h, r.shape[0], _dptr(r), _dptr(v)))
        return v

    @property
    def launches(self) -> int:
        return int(self.lib.gdc_fcm_launches(self._h))

    def close(self):
        if getattr(self, "_h", None) and self._h.value:
            self.lib.gdc_fcm_destroy(self._h)
        self._h = ctypes.c_void_p(0)

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def rpy_apply_noalloc(r, lam, a: float = 1.0, eta: float = 1.0, out=None, stream=None):
    """u = M lambda for one suspension of free blobs through gdc_rpy_apply_noalloc.

    For callers that must not allocate device memory on the library's behalf: the
    library uses only its fixed internal scratch array.  r, lam: contiguous float64 CUDA
    tensors of the same length, 3 values per blob, on one device; out (optional, same
    kind) receives u.  Returns out.  A pair-kernel timeout shows as NaN in out.
    """
    import torch
    lib = load_library()
    tensors = [r, lam] + ([out] if out is not None else [])
    for t in tensors:
        if not (t.is_cuda and t.dtype == torch.float64 and t.is_contiguous()):
            raise ValueError("r, lam and out must be contiguous float64 CUDA tensors")
        if t.numel() != r.numel() or t.device != r.device:
            raise ValueError("r, lam and out must have the same length and device")
    if r.numel() % 3 != 0 or r.numel() == 0:
        raise ValueError("r holds 3 values per blob")
    n = r.numel() // 3
    with torch.cuda.device(r.device):
        if out is None:
            out = torch.empty_like(lam)
        s = stream if stream is not None else torch.cuda.current_stream(r.device)
        st = lib.gdc_rpy_apply_noalloc(_dptr(r), _dptr(lam), _dptr(out), n, a, eta, ctypes.c_void_p(s.cuda_stream))
    if st != 0:
        raise GdcError(st, lib.gdc_last_error(None).decode())
    return out


def fma_probe(out, mode: int = 1, iters: int = 2048, stream=None) -> float:
    """Launch the FP32 FMA throughput probe (gdc_fma_probe) over out.numel() // 256 blocks of
    256 threads on `stream` (a torch.cuda.Stream or None for the current one): mode 0 scalar,
    1 packed f32x2, 2 half and half.  Returns the flops the launch performs.  out: a float32
    CUDA tensor the kernel writes."""
    import torch
    if out.dtype != torch.float32 or not out.is_cuda or out.numel() < 256:
        raise ValueError("out must be a float32 CUDA tensor of at least 256 elements")
    blocks = out.numel() // 256
    st = (stream or torch.cuda.current_stream(out.device)).cuda_stream
    with torch.cuda.device(out.device):
        rc = load_library().gdc_fma_probe(int(mode), blocks, int(iters), ctypes.c_void_p(out.data_ptr()),
                                          ctypes.c_void_p(st))
    if rc != 0:
        raise RuntimeError(f"gdc_fma_probe failed with status {rc}")
    return float(blocks) * 256 * iters * 32


def debug_wait_polls(polls: int) -> None:
    """Bound of the pair kernels' waits for a tile copy (gdc_debug_wait_polls): 0 restores
    the default; a negative value makes every first wait give up (tests of the timeout path)."""
    load_library().gdc_debug_wait_polls(int(polls))


def context_from_workload(wl, **overrides) -> Context:
    """Context for a synthetic workload (synthetic.workloads.Workload) with its physical parameters."""
    pp = wl.params
    kw = dict(eta=pp["eta"], kT=pp["kT"], a=pp["a"], dt=pp["dt"], gmres_tol=pp.get("gmres_tol", 1e-6),
              lanczos_tol=pp.get("lanczos_tol", 1e-4), rfd_delta=pp.get("rfd_delta", 1e-6), rep_A=pp.get("rep_A", 0.0),
              rep_b=pp.get("rep_b", 0.1), shear_rate=pp.get("shear_rate", 0.0), seed=int(pp.get("seed", 0)),
              potential=int(pp.get("potential", 0)), well_A=pp.get("well_A", 0.0), well_lambda=pp.get("well_lambda", 0.5),
              wall=int(pp.get("wall", 0)), wall_V0=pp.get("wall_V0", 0.0), wall_b=pp.get("wall_b", 0.5),
              body_weight=pp.get("body_weight", 0.0))
    kw.update(overrides)
    return Context(Params(**kw), wl.templates, wl.body_tmpl, wl.susp_body_off, wl.Y, wl.q)
