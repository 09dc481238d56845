"""ctypes binding of libgks.so (include/gks.h).

Argument marshalling only: PyTorch supplies device memory and the CUDA
stream, every step of the hot path runs in the library's sm_103a kernels.
There is no CPU fallback: without a built library ``lib()`` raises.
"""
from __future__ import annotations

import ctypes
import math
import os
from dataclasses import dataclass

import numpy as np

from . import build as _build

GKS_OK = 0
GKS_ERR_ARG = -1
GKS_ERR_CUDA = -2
GKS_ERR_NONPHYSICAL = -3
GKS_ERR_TIMEOUT = -4
GKS_ERR_STATE = -5
GKS_ERR_NOMEM = -6

SCHEMES = {"gks2": 0, "cgks5": 1}
PRECISIONS = {"fp64": 0, "mixed": 1}


class GksError(RuntimeError):
    def __init__(self, code, what):
        self.code = code
        msg = lib().gks_strerror(code).decode() if _LIB is not None else str(code)
        super().__init__(f"{what}: {msg} ({code})")


class Options(ctypes.Structure):
    """Mirror of gks_options."""

    _fields_ = [
        ("scheme", ctypes.c_int), ("nonlinear", ctypes.c_int),
        ("precision", ctypes.c_int), ("indicator", ctypes.c_int),
        ("mu_law", ctypes.c_int), ("inviscid", ctypes.c_int),
        ("C_tau", ctypes.c_double), ("eps_tau", ctypes.c_double),
        ("T_ref", ctypes.c_double), ("theta", ctypes.c_double),
        ("slab_planes", ctypes.c_int), ("reserved", ctypes.c_int),
        ("bc", ctypes.c_int * 3), ("reserved2", ctypes.c_int),
        ("h", ctypes.POINTER(ctypes.c_double) * 3),
    ]


BC = {"periodic": 0, "symmetry": 1, "outflow": 2}


_LIB = None
_VP = ctypes.c_void_p
_D = ctypes.c_double
_I = ctypes.c_int

SIGNATURES = {
    "gks_default_options": (None, [ctypes.POINTER(Options)]),
    "gks_init": (_I, [ctypes.POINTER(_VP), _D, _D, _D, _D, _I, _I, _I, _D, _D, _D,
                      ctypes.POINTER(Options), _VP]),
    "gks_destroy": (None, [_VP]),
    "gks_strerror": (ctypes.c_char_p, [_I]),
    "gks_face_state_bytes": (ctypes.c_size_t, [_VP]),
    "gks_face_flux_bytes": (ctypes.c_size_t, [_VP]),
    "gks_slab_planes": (_I, [_VP]),
    "gks_compute_dt": (_I, [_VP, _VP, _VP]),
    "gks_reconstruct": (_I, [_VP, _VP, _VP, _VP]),
    "gks_flux": (_I, [_VP, _VP, _VP, _VP, _VP]),
    "gks_flux_points": (_I, [_VP, _VP, _VP, _I, _VP, _VP]),
    "gks_step": (_I, [_VP, _VP, _VP, _I, _D, _VP, ctypes.POINTER(_D)]),
    "gks_step_host": (_I, [_VP, _VP, _VP, _I, _D, ctypes.POINTER(_D)]),
    "gks_diagnostics": (_I, [_VP, _VP, _VP, ctypes.POINTER(_D)]),
    "gks_status": (_I, [_VP, ctypes.POINTER(_I)]),
    "gks_recon_matrix": (_I, [ctypes.POINTER(_D)]),
    "gks_recon_matrix_lines": (_I, [ctypes.POINTER(_D)]),
    "gks_diagnostics_noalloc": (_I, [_VP, _VP, _I, _I, _I, _D, _D, _D, _D, _D, _I, _D, _VP, _VP]),
    "gks_fma_rate": (_I, [_I, _VP, ctypes.POINTER(_D), ctypes.POINTER(_D)]),
    "gks_kernel_timing": (_I, [_VP, _I]),
    "gks_kernel_times": (_I, [_VP, ctypes.POINTER(_D), ctypes.POINTER(ctypes.c_longlong)]),
    "gks_mlp_nparams": (_I, []),
    "gks_indicator_dump": (_I, [_VP, _VP, _VP, ctypes.c_float, _VP, _VP, _VP]),
    "gks_mlp_loss_grad": (_I, [_VP, _VP, _VP, _I, ctypes.c_longlong, ctypes.c_float, _VP, _VP, _VP]),
    "gks_mlp_train": (_I, [_VP, _VP, _VP, _I, ctypes.c_longlong, _I, _I, ctypes.c_float,
                           ctypes.c_float, ctypes.c_uint, _VP, _VP]),
    "gks_set_indicator": (_I, [_VP, ctypes.POINTER(ctypes.c_float), ctypes.c_float]),
    "gks_indicator_skips": (_I, [_VP, ctypes.POINTER(ctypes.c_ulonglong)]),
    "gks_ensemble_create": (_I, [ctypes.POINTER(_VP), _I, _VP, _VP, _VP, ctypes.POINTER(Options), _VP]),
    "gks_ensemble_destroy": (None, [_VP]),
    "gks_ensemble_offset": (ctypes.c_longlong, [_VP, _I]),
    "gks_ensemble_set_tile": (_I, [_VP, _I]),
    "gks_ensemble_step": (_I, [_VP, _VP, _VP, _I, _D, _I]),
    "gks_ensemble_times": (_I, [_VP, ctypes.POINTER(_D), ctypes.POINTER(_I)]),
    "gks_ensemble_autotune": (_I, [_VP, _VP, _VP, ctypes.POINTER(_I), ctypes.POINTER(ctypes.c_float)]),
    "gks_ensemble_dump": (_I, [_VP, _VP, _VP, ctypes.c_float, _VP, _VP, _VP]),
    "gks_ensemble_set_indicator": (_I, [_VP, ctypes.POINTER(ctypes.c_float), ctypes.c_float]),
    "gks_ensemble_set_mode": (_I, [_VP, _I]),
    "gks_ensemble_mode": (_I, [_VP]),
    "gks_barrier_timeout_check": (_I, [_D, _VP]),
    "gks_reconstruct_lines": (_I, [_VP, _VP, _VP, _VP]),
    "gks_step_lines": (_I, [_VP, _VP, _VP, _I, _D, _VP, ctypes.POINTER(_D)]),
    "gks_lines_gradients": (_I, [_VP, _VP, _VP]),
}


def lib_path() -> str:
    return _build.LIB


def lib(build_if_missing: bool = True):
    """Load libgks.so (building it first if asked); raises if unavailable."""
    global _LIB
    if _LIB is None:
        path = _build.LIB
        if build_if_missing and not _build.up_to_date():
            _build.build()
        if not os.path.exists(path):
            raise RuntimeError(f"libgks.so not built ({path}); run "
                               "python -m paper_2508_19911_gb300.build")
        L = ctypes.CDLL(path)
        for name, (res, args) in SIGNATURES.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _LIB = L
    return _LIB


def _check(rc, what):
    if rc != GKS_OK:
        raise GksError(rc, what)


def fma_rate(precision="fp64", stream=None):
    """Measured FMA throughput of the current device (FLOP/s, launch ms):
    precision "fp64" (double FMAs) or "fp32" (float FMAs)."""
    import torch
    st = stream if stream is not None else torch.cuda.current_stream()
    flops, ms = _D(0.0), _D(0.0)
    _check(lib().gks_fma_rate(0 if precision == "fp64" else 1, _VP(st.cuda_stream),
                              ctypes.byref(flops), ctypes.byref(ms)), "gks_fma_rate")
    return flops.value, ms.value


def mlp_nparams() -> int:
    return int(lib().gks_mlp_nparams())


def mlp_loss_grad(params, x, y, neg_weight=1.0, stream=None):
    """Loss and gradient of the indicator network (device tensors)."""
    import torch
    n = int(y.shape[0])
    loss = torch.zeros(1, dtype=torch.float32, device=params.device)
    grad = torch.zeros(mlp_nparams(), dtype=torch.float32, device=params.device)
    st = stream if stream is not None else torch.cuda.current_stream(params.device)
    _check(lib().gks_mlp_loss_grad(_ptr(params, torch.float32), _ptr(x, torch.float32),
                                   _ptr(y, torch.float32), n, int(x.shape[1]), float(neg_weight),
                                   _ptr(loss, torch.float32), _ptr(grad, torch.float32),
                                   _VP(st.cuda_stream)), "gks_mlp_loss_grad")
    return float(loss.item()), grad


def mlp_train(params, x, y, epochs=10, batch=4096, lr=3e-3, neg_weight=1.0, seed=0, stream=None):
    """Train in place; returns the per-epoch mean loss (numpy)."""
    import torch
    n = int(y.shape[0])
    hist = torch.zeros(max(epochs, 1), dtype=torch.float32, device=params.device)
    st = stream if stream is not None else torch.cuda.current_stream(params.device)
    _check(lib().gks_mlp_train(_ptr(params, torch.float32), _ptr(x, torch.float32),
                               _ptr(y, torch.float32), n, int(x.shape[1]), int(epochs), int(batch),
                               float(lr), float(neg_weight), int(seed) & 0xFFFFFFFF,
                               _ptr(hist, torch.float32), _VP(st.cuda_stream)), "gks_mlp_train")
    return hist.cpu().numpy()[:epochs]


def recon_matrix_lines() -> np.ndarray:
    """The library's line-form reconstruction matrix (34 x 72), host-built."""
    R = np.zeros((34, 72))
    _check(lib().gks_recon_matrix_lines(R.ctypes.data_as(ctypes.POINTER(_D))),
           "gks_recon_matrix_lines")
    return R


def recon_matrix() -> np.ndarray:
    """The library's CGKS-5th reconstruction matrix (34 x 63), host-built."""
    R = np.zeros((34, 63))
    _check(lib().gks_recon_matrix(R.ctypes.data_as(ctypes.POINTER(_D))), "gks_recon_matrix")
    return R


def _ptr(t, dtype=None):
    if t is None:
        return None
    import torch
    want = torch.float64 if dtype is None else dtype
    if not (isinstance(t, torch.Tensor) and t.is_cuda and t.dtype == want and t.is_contiguous()):
        raise TypeError(f"expected a contiguous {want} CUDA tensor")
    return ctypes.c_void_p(t.data_ptr())


@dataclass
class Config:
    n: tuple
    L: tuple
    gamma: float = 1.4
    Pr: float = 0.72
    mu: float = 1.0 / 1600
    cfl: float = 0.3
    scheme: str = "cgks5"
    nonlinear: bool = True
    precision: str = "fp64"
    indicator: bool = False
    mu_law: int = 0
    inviscid: bool = False
    C_tau: float = 10.0
    eps_tau: float = 0.05
    T_ref: float = 1.0
    theta: float = 0.9
    slab_planes: int = 0
    # boundary per axis ("periodic", "symmetry", "outflow") and, for a
    # stretched mesh, the cell sizes of each axis (None: uniform L/n)
    bc: tuple = ("periodic", "periodic", "periodic")
    spacing: tuple = (None, None, None)


class Solver:
    """One gks_ctx: a grid with its workspace on the current device."""

    def __init__(self, cfg: Config, stream=None):
        import torch
        self.cfg = cfg
        self.torch = torch
        L = lib()
        opt = Options()
        L.gks_default_options(ctypes.byref(opt))
        opt.scheme = SCHEMES[cfg.scheme]
        opt.nonlinear = int(bool(cfg.nonlinear))
        opt.precision = PRECISIONS[cfg.precision]
        opt.indicator = int(bool(cfg.indicator))
        opt.mu_law = int(cfg.mu_law)
        opt.inviscid = int(bool(cfg.inviscid))
        opt.C_tau, opt.eps_tau, opt.T_ref, opt.theta = cfg.C_tau, cfg.eps_tau, cfg.T_ref, cfg.theta
        opt.slab_planes = int(cfg.slab_planes)
        keep = []
        for a in range(3):
            b = cfg.bc[a]
            opt.bc[a] = BC[b] if isinstance(b, str) else int(b)
            if cfg.spacing[a] is not None:
                h = np.ascontiguousarray(cfg.spacing[a], dtype=np.float64)
                if h.shape != (int(cfg.n[a]),):
                    raise ValueError(f"spacing[{a}] needs {cfg.n[a]} cell sizes")
                keep.append(h)
                opt.h[a] = h.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        self.device = self.stream.device
        ctx = _VP()
        with torch.cuda.device(self.device):
            _check(L.gks_init(ctypes.byref(ctx), cfg.gamma, cfg.Pr, cfg.mu, cfg.cfl,
                              int(cfg.n[0]), int(cfg.n[1]), int(cfg.n[2]),
                              float(cfg.L[0]), float(cfg.L[1]), float(cfg.L[2]),
                              ctypes.byref(opt), _VP(self.stream.cuda_stream)), "gks_init")
        del keep  # gks_init copied the cell sizes
        self.ctx = ctx
        self.ncells = int(cfg.n[0]) * int(cfg.n[1]) * int(cfg.n[2])
        self.K = 4 if cfg.scheme == "cgks5" else 1
        self.fs_dtype = torch.float32 if cfg.precision == "mixed" else torch.float64

    def close(self):
        if getattr(self, "ctx", None):
            lib().gks_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # -- tensors -------------------------------------------------------------
    def zeros(self, *shape):
        return self.torch.zeros(*shape, dtype=self.torch.float64, device=self.device)

    def state_shape(self):
        nx, ny, nz = self.cfg.n
        return (5, nz, ny, nx), (5, 3, nz, ny, nx)

    # -- entry points ----------------------------------------------------------
    def compute_dt(self, Q, dt=None):
        dt = self.zeros(1) if dt is None else dt
        _check(lib().gks_compute_dt(self.ctx, _ptr(Q), _ptr(dt)), "gks_compute_dt")
        return dt

    @property
    def slab_planes(self):
        """z-planes per slab of step()'s reconstruction + flux (0: whole grid)."""
        return int(lib().gks_slab_planes(self.ctx))

    def reconstruct(self, Q, G=None, out=None):
        if out is None:
            out = self.torch.zeros(6, self.K, 20, self.ncells, dtype=self.fs_dtype, device=self.device)
        _check(lib().gks_reconstruct(self.ctx, _ptr(Q), _ptr(G), _ptr(out, self.fs_dtype)),
               "gks_reconstruct")
        return out

    def flux_bytes(self):
        """Bytes of gks_flux's records (boundary faces included)."""
        return int(lib().gks_face_flux_bytes(self.ctx))

    def flux(self, face_states, dt, out=None, Q=None):
        """Face records; on a grid with a non-periodic or stretched axis the
        returned buffer is flat: [3][30][cells] then the high-boundary
        records [3][30][np]."""
        if out is None:
            words = self.flux_bytes() // 8
            out = self.zeros(words) if words != 90 * self.ncells else self.zeros(3, 30, self.ncells)
        _check(lib().gks_flux(self.ctx, _ptr(Q), _ptr(face_states, self.fs_dtype), _ptr(dt),
                              _ptr(out)), "gks_flux")
        return out

    def flux_points(self, s_l, s_r, dt, out=None):
        n = s_l.shape[1]
        if out is None:
            out = self.zeros(30, n)
        _check(lib().gks_flux_points(self.ctx, _ptr(s_l), _ptr(s_r), n, _ptr(dt), _ptr(out)),
               "gks_flux_points")
        return out

    def step(self, Q, G=None, nsteps=1, t_stop=math.inf, t=None, sync=True):
        """Advance in place. Returns the last dt (sync=True) or None."""
        last = _D(0.0)
        rc = lib().gks_step(self.ctx, _ptr(Q), _ptr(G), int(nsteps), float(t_stop), _ptr(t),
                            ctypes.byref(last) if sync else None)
        _check(rc, "gks_step")
        return last.value if sync else None

    def step_host(self, Q, G=None, nsteps=1, t_stop=math.inf, t=None):
        """Advance a state held in host memory (contiguous float64 CPU
        tensors, pinned for full copy speed) in place; the library copies
        it to the device and back. t: None or a float (simulation time);
        returns the new time."""
        cg = self.cfg.scheme == "cgks5"
        for x in (Q, G) if cg else (Q,):
            if not (isinstance(x, self.torch.Tensor) and not x.is_cuda and
                    x.dtype == self.torch.float64 and x.is_contiguous()):
                raise TypeError("expected a contiguous float64 CPU tensor")
        tt = _D(0.0 if t is None else float(t))
        rc = lib().gks_step_host(self.ctx, ctypes.c_void_p(Q.data_ptr()),
                                 ctypes.c_void_p(G.data_ptr()) if cg else None, int(nsteps),
                                 float(t_stop), ctypes.byref(tt) if t is not None else None)
        _check(rc, "gks_step_host")
        return tt.value if t is not None else None

    # -- the line-averaged derivatives as the cell's own data ------------------
    def lines_shape(self):
        nx, ny, nz = self.cfg.n
        return (5, 12, nz, ny, nx)

    def reconstruct_lines(self, Q, L, out=None):
        """Face states (FP64, layout of reconstruct) from the averages Q and
        the 12 line-averaged derivatives L [5][12] per cell."""
        if out is None:
            out = self.zeros(6, 4, 20, self.ncells)
        _check(lib().gks_reconstruct_lines(self.ctx, _ptr(Q), _ptr(L), _ptr(out)),
               "gks_reconstruct_lines")
        return out

    def step_lines(self, Q, L, nsteps=1, t_stop=math.inf, t=None, sync=True):
        """Advance (Q, L) in place. Returns the last dt (sync=True) or None."""
        last = _D(0.0)
        rc = lib().gks_step_lines(self.ctx, _ptr(Q), _ptr(L), int(nsteps), float(t_stop), _ptr(t),
                                  ctypes.byref(last) if sync else None)
        _check(rc, "gks_step_lines")
        return last.value if sync else None

    def lines_gradients(self, L, out=None):
        """Averaged gradients [5][3] per cell: the mean of each axis' lines."""
        if out is None:
            out = self.zeros(*self.state_shape()[1])
        _check(lib().gks_lines_gradients(self.ctx, _ptr(L), _ptr(out)), "gks_lines_gradients")
        return out

    def diagnostics(self, Q, G=None):
        out = (_D * 12)()
        _check(lib().gks_diagnostics(self.ctx, _ptr(Q), _ptr(G), out), "gks_diagnostics")
        return np.array(out[:], dtype=np.float64)

    # -- learned indicator ----------------------------------------------------
    def indicator_dump(self, Q, G, label_eps=1e-4):
        """(x [63][5 cells], chi [5 cells], y [5 cells]) float32 CUDA tensors."""
        t = self.torch
        m = 5 * self.ncells
        x = t.empty(63, m, dtype=t.float32, device=self.device)
        chi = t.empty(m, dtype=t.float32, device=self.device)
        y = t.empty(m, dtype=t.float32, device=self.device)
        _check(lib().gks_indicator_dump(self.ctx, _ptr(Q), _ptr(G), float(label_eps),
                                        _ptr(x, t.float32), _ptr(chi, t.float32),
                                        _ptr(y, t.float32)), "gks_indicator_dump")
        return x, chi, y

    def set_indicator(self, params, theta=0.9):
        p = np.ascontiguousarray(np.asarray(params, dtype=np.float32))
        _check(lib().gks_set_indicator(self.ctx, p.ctypes.data_as(ctypes.POINTER(ctypes.c_float)),
                                       float(theta)), "gks_set_indicator")

    def indicator_skips(self):
        n = ctypes.c_ulonglong(0)
        _check(lib().gks_indicator_skips(self.ctx, ctypes.byref(n)), "gks_indicator_skips")
        return n.value

    def status(self):
        st = _I(0)
        _check(lib().gks_status(self.ctx, ctypes.byref(st)), "gks_status")
        return st.value

    KERNEL_KINDS = ("recon", "flux", "update", "dt")

    def kernel_timing(self, on=True):
        """Start (discarding earlier records) or stop recording the device
        time of every launch gks_step makes."""
        _check(lib().gks_kernel_timing(self.ctx, 1 if on else 0), "gks_kernel_timing")

    def kernel_times(self):
        """{kind: (summed ms, launches)} of the recorded launches."""
        ms = (_D * 4)()
        n = (ctypes.c_longlong * 4)()
        _check(lib().gks_kernel_times(self.ctx, ms, n), "gks_kernel_times")
        return {k: (ms[i], n[i]) for i, k in enumerate(self.KERNEL_KINDS)}


class Ensemble:
    """A batch of independent CGKS-5th instances advanced together.

    ``instances``: list of dicts with keys n (nx, ny, nz), L (Lx, Ly, Lz) and
    the physics gamma, Pr, mu, cfl, mu_law, inviscid, C_tau, eps_tau (defaults
    as in Config). The states live in two arenas owned by this object:
    ``Q`` [5 * total] and ``G`` [15 * total] (float64 CUDA tensors); use
    ``views(i)`` for instance i's [5][nz][ny][nx] and [5][3][nz][ny][nx] views.
    """

    def __init__(self, instances, *, precision="fp64", nonlinear=True, T_ref=1.0, stream=None):
        import torch
        self.torch = torch
        n = len(instances)
        dims = np.zeros(3 * n, dtype=np.int32)
        lens = np.zeros(3 * n, dtype=np.float64)
        phys = np.zeros(8 * n, dtype=np.float64)
        for i, ins in enumerate(instances):
            dims[3 * i: 3 * i + 3] = ins["n"]
            lens[3 * i: 3 * i + 3] = ins["L"]
            phys[8 * i: 8 * i + 8] = [ins.get("gamma", 1.4), ins.get("Pr", 0.72),
                                      ins.get("mu", 1.0 / 1600), ins.get("cfl", 0.3),
                                      ins.get("mu_law", 0), float(bool(ins.get("inviscid", False))),
                                      ins.get("C_tau", 10.0), ins.get("eps_tau", 0.05)]
        opt = Options()
        lib().gks_default_options(ctypes.byref(opt))
        opt.scheme = SCHEMES["cgks5"]
        opt.precision = PRECISIONS[precision]
        opt.nonlinear = int(bool(nonlinear))
        opt.indicator = 0
        opt.T_ref = T_ref
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        self.device = self.stream.device
        self.instances = instances
        ctx = _VP()
        with torch.cuda.device(self.device):
            _check(lib().gks_ensemble_create(ctypes.byref(ctx), n, dims.ctypes.data_as(_VP),
                                             lens.ctypes.data_as(_VP), phys.ctypes.data_as(_VP),
                                             ctypes.byref(opt), _VP(self.stream.cuda_stream)),
                   "gks_ensemble_create")
        self.e = ctx
        self.n = n
        self.offsets = [int(lib().gks_ensemble_offset(ctx, i)) for i in range(n + 1)]
        self.total = self.offsets[-1]
        self.Q = torch.zeros(5 * self.total, dtype=torch.float64, device=self.device)
        self.G = torch.zeros(15 * self.total, dtype=torch.float64, device=self.device)

    def close(self):
        if getattr(self, "e", None):
            lib().gks_ensemble_destroy(self.e)
            self.e = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def views(self, i):
        nx, ny, nz = self.instances[i]["n"]
        o, c = self.offsets[i], self.offsets[i + 1] - self.offsets[i]
        return (self.Q[5 * o: 5 * (o + c)].view(5, nz, ny, nx),
                self.G[15 * o: 15 * (o + c)].view(5, 3, nz, ny, nx))

    def set_tile(self, tile):
        _check(lib().gks_ensemble_set_tile(self.e, int(tile)), "gks_ensemble_set_tile")

    def set_mode(self, mode):
        """1: a step is one persistent launch (default); 0: one per phase."""
        _check(lib().gks_ensemble_set_mode(self.e, int(mode)), "gks_ensemble_set_mode")

    @property
    def mode(self):
        return int(lib().gks_ensemble_mode(self.e))

    def step(self, nsteps=1, t_stop=math.inf, graph=True):
        _check(lib().gks_ensemble_step(self.e, _ptr(self.Q), _ptr(self.G), int(nsteps),
                                       float(t_stop), int(bool(graph))), "gks_ensemble_step")

    def times(self):
        t = (_D * self.n)()
        st = _I(0)
        rc = lib().gks_ensemble_times(self.e, t, ctypes.byref(st))
        _check(rc, "gks_ensemble_times")
        return np.array(t[:])

    def autotune(self):
        tile = _I(0)
        ms = ctypes.c_float(0)
        _check(lib().gks_ensemble_autotune(self.e, _ptr(self.Q), _ptr(self.G), ctypes.byref(tile),
                                           ctypes.byref(ms)), "gks_ensemble_autotune")
        return tile.value, ms.value

    def dump(self, label_eps=1e-4):
        t = self.torch
        m = 5 * self.total
        x = t.empty(63, m, dtype=t.float32, device=self.device)
        chi = t.empty(m, dtype=t.float32, device=self.device)
        y = t.empty(m, dtype=t.float32, device=self.device)
        _check(lib().gks_ensemble_dump(self.e, _ptr(self.Q), _ptr(self.G), float(label_eps),
                                       _ptr(x, t.float32), _ptr(chi, t.float32), _ptr(y, t.float32)),
               "gks_ensemble_dump")
        return x, chi, y

    def set_indicator(self, params, theta=0.9):
        p = np.ascontiguousarray(np.asarray(params, dtype=np.float32))
        _check(lib().gks_ensemble_set_indicator(self.e, p.ctypes.data_as(ctypes.POINTER(ctypes.c_float)),
                                                float(theta)), "gks_ensemble_set_indicator")


def barrier_timeout_check(limit_s=0.2, stream=None):
    """The single-launch ensemble step's bounded barrier wait, made to run
    out: returns the C-ABI code (GKS_ERR_TIMEOUT = -4 expected)."""
    import torch
    st = stream if stream is not None else torch.cuda.current_stream()
    return int(lib().gks_barrier_timeout_check(float(limit_s), _VP(st.cuda_stream)))
