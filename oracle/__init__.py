"""FP64 CPU oracle of the CGKS-5th / GKS-2nd hot path.

TEST INFRASTRUCTURE ONLY: the tests, the package smoke check and the
benchmark's CPU-baseline leg load it; the product path never does. The C++
sources in this directory restate the paper's method step by step (Sec. 2
kinetic flux, Sec. 3.2/3.3 reconstructions, Sec. 3.4 time stepping, Sec. 4
time step and collision time) and share no code with the CUDA library.

``build()`` compiles ``liboracle.so`` with g++ (``-O2 -ffp-contract=off``,
OpenMP for the cell loops only); ``lib()`` loads it through ctypes.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_BUILD = os.path.join(_HERE, "_build")
_SO = os.path.join(_BUILD, "liboracle.so")
_SOURCES = ["moments.cpp", "flux.cpp", "recon.cpp", "scheme.cpp", "scheme_b.cpp", "mlp.cpp"]
_LOCK = threading.Lock()
_LIB = None


class Params(ctypes.Structure):
    """Mirror of ``orc_params`` (oracle.h)."""

    _fields_ = [
        ("gamma", ctypes.c_double), ("Pr", ctypes.c_double),
        ("mu0", ctypes.c_double), ("cfl", ctypes.c_double),
        ("C_tau", ctypes.c_double), ("eps_tau", ctypes.c_double),
        ("T_ref", ctypes.c_double),
        ("Lx", ctypes.c_double), ("Ly", ctypes.c_double), ("Lz", ctypes.c_double),
        ("nx", ctypes.c_int), ("ny", ctypes.c_int), ("nz", ctypes.c_int),
        ("scheme", ctypes.c_int), ("nonlinear", ctypes.c_int),
        ("mu_law", ctypes.c_int), ("inviscid", ctypes.c_int),
        ("threads", ctypes.c_int),
        ("bc", ctypes.c_int * 3), ("pad_", ctypes.c_int),
        ("hx", ctypes.POINTER(ctypes.c_double)), ("hy", ctypes.POINTER(ctypes.c_double)),
        ("hz", ctypes.POINTER(ctypes.c_double)),
    ]


BC_PERIODIC, BC_SYMMETRY, BC_OUTFLOW = 0, 1, 2


def params(*, gamma=1.4, Pr=0.72, mu0=1.0 / 1600, cfl=0.3, C_tau=10.0,
           eps_tau=0.05, T_ref=1.0, L=(2 * np.pi,) * 3, n=(16, 16, 16),
           scheme=1, nonlinear=1, mu_law=0, inviscid=0, threads=None,
           bc=(0, 0, 0), spacing=(None, None, None)):
    """bc[a]: BC_PERIODIC, BC_SYMMETRY (mirror, normal momentum negated) or
    BC_OUTFLOW (mirror) on axis a; spacing[a]: the n[a] cell sizes of axis a
    (None: uniform L[a]/n[a])."""
    if threads is None:
        threads = os.cpu_count() or 1
    P = Params(gamma, Pr, mu0, cfl, C_tau, eps_tau, T_ref, L[0], L[1], L[2],
               n[0], n[1], n[2], scheme, nonlinear, mu_law, inviscid, threads)
    for a in range(3):
        P.bc[a] = int(bc[a])
    keep = []
    for a, name in enumerate(("hx", "hy", "hz")):
        if spacing[a] is not None:
            h = np.ascontiguousarray(spacing[a], dtype=np.float64)
            assert h.shape == (n[a],) and np.all(h > 0)
            keep.append(h)
            setattr(P, name, h.ctypes.data_as(ctypes.POINTER(ctypes.c_double)))
    P._keep = keep  # the spacing arrays live as long as the parameters
    return P


def _sources():
    return [os.path.join(_HERE, s) for s in _SOURCES]


def build(force: bool = False) -> str:
    """Compile the oracle into oracle/_build/liboracle.so (idempotent)."""
    os.makedirs(_BUILD, exist_ok=True)
    deps = _sources() + [os.path.join(_HERE, h) for h in ("oracle.h", "oracle_internal.h")]
    if not force and os.path.exists(_SO):
        so_t = os.path.getmtime(_SO)
        if all(os.path.getmtime(d) <= so_t for d in deps):
            return _SO
    tmp = _SO + f".tmp{os.getpid()}"
    cmd = ["g++", "-std=c++17", "-O2", "-ffp-contract=off", "-fopenmp", "-fPIC",
           "-shared", "-o", tmp] + _sources()
    subprocess.run(cmd, check=True)
    os.replace(tmp, _SO)
    return _SO


_D = ctypes.POINTER(ctypes.c_double)
_P = ctypes.POINTER(Params)


def lib():
    global _LIB
    with _LOCK:
        if _LIB is None:
            build()
            L = ctypes.CDLL(_SO)
            sig = {
                "orc_moment_matrix": [ctypes.c_double] * 5 + [ctypes.c_int, ctypes.c_int, _D],
                "orc_slope": [_D, _D, ctypes.c_double, _D],
                "orc_flux_gp": [_P, _D, _D, ctypes.c_double, _D],
                "orc_fbar": [_P, _D, _D, ctypes.c_double, ctypes.c_double, _D],
                "orc_recon5_matrix": [_D],
                "orc_recon5b_matrix": [_D],
                "orc_recon5b_cell": [_D, _D, ctypes.c_double, ctypes.c_double,
                                     ctypes.c_double, ctypes.c_int, _D, _D],
                "orc_run_b": [_P, _D, _D, ctypes.c_int, ctypes.c_double, _D, _D],
                "orc_face_states_b": [_P, _D, _D, _D],
                "orc_geno_misfit": [_D, _D, _D],
                "orc_chi_field": [_P, _D, _D, _D],
                "orc_recon5_cell": [_D, _D, ctypes.c_double, ctypes.c_double,
                                    ctypes.c_double, ctypes.c_int, _D, _D],
                "orc_recon2_cell": [_D, ctypes.c_double, ctypes.c_double,
                                    ctypes.c_double, ctypes.c_int, _D, _D],
                "orc_dt": [_P, _D, _D],
                "orc_run": [_P, _D, _D, ctypes.c_int, ctypes.c_double, _D, _D],
                "orc_stage": [_P, _D, _D, ctypes.c_double, _D, _D, _D, _D],
                "orc_face_states": [_P, _D, _D, _D],
                "orc_face_states_at": [_P, _D, _D, ctypes.POINTER(ctypes.c_longlong),
                                       ctypes.c_longlong, _D],
                "orc_face_record": [_P, ctypes.c_int, _D, _D, ctypes.c_double, _D],
                "orc_diagnostics": [_P, _D, _D, _D],
                "orc_mlp_nparams": [],
                "orc_mlp_loss_grad": [_D, _D, _D, ctypes.c_int, ctypes.c_longlong,
                                      ctypes.c_double, _D, _D],
            }
            for name, args in sig.items():
                f = getattr(L, name)
                f.argtypes = args
                f.restype = ctypes.c_int
            _LIB = L
    return _LIB


def _ptr(a):
    if a is None:
        return None
    assert a.dtype == np.float64 and a.flags["C_CONTIGUOUS"]
    return a.ctypes.data_as(_D)


def _check(rc, what):
    if rc != 0:
        raise RuntimeError(f"oracle {what} failed with code {rc}")


# ---- thin numpy wrappers -------------------------------------------------

def moment_matrix(U, V, W, lam, Nint, half, which):
    out = np.zeros(25)
    _check(lib().orc_moment_matrix(U, V, W, lam, Nint, half, which, _ptr(out)), "moment_matrix")
    return out.reshape(5, 5)


def slope(Wc, dW, gamma=1.4):
    a = np.zeros(5)
    _check(lib().orc_slope(_ptr(np.ascontiguousarray(Wc, float)),
                           _ptr(np.ascontiguousarray(dW, float)), gamma, _ptr(a)), "slope")
    return a


def flux_gp(P, sl, sr, dt):
    out = np.zeros(30)
    _check(lib().orc_flux_gp(ctypes.byref(P), _ptr(np.ascontiguousarray(sl, float)),
                             _ptr(np.ascontiguousarray(sr, float)), dt, _ptr(out)), "flux_gp")
    return out


def fbar(P, sl, sr, dt, T):
    out = np.zeros(20)
    _check(lib().orc_fbar(ctypes.byref(P), _ptr(np.ascontiguousarray(sl, float)),
                          _ptr(np.ascontiguousarray(sr, float)), dt, T, _ptr(out)), "fbar")
    return out


def recon5_matrix():
    R = np.zeros((34, 63))
    _check(lib().orc_recon5_matrix(_ptr(R)), "recon5_matrix")
    return R


def recon5b_matrix():
    """Reading B's least-squares matrix (34 x 72)."""
    R = np.zeros((34, 72))
    _check(lib().orc_recon5b_matrix(_ptr(R)), "recon5b_matrix")
    return R


def recon5b_cell(q0, dvec, h=(1.0, 1.0, 1.0), nonlinear=1):
    out = np.zeros(480)
    chi = np.zeros(5)
    _check(lib().orc_recon5b_cell(_ptr(np.ascontiguousarray(q0, float)),
                                  _ptr(np.ascontiguousarray(dvec, float)),
                                  h[0], h[1], h[2], nonlinear, _ptr(out), _ptr(chi)),
           "recon5b_cell")
    return out.reshape(6, 4, 20), chi


def run_b(P, Q, L, nsteps=1, t_stop=np.inf, t=0.0):
    """CGKS-5th with reading B: advance Q [5][cells...] and the line-averaged
    derivatives L [5][12][cells...] in place (any of the boundaries of
    params(bc=...), uniform or stretched); returns (t, dt_last)."""
    tt = np.array([t], float)
    dl = np.zeros(1)
    _check(lib().orc_run_b(ctypes.byref(P), _ptr(Q), _ptr(L), nsteps, t_stop,
                           _ptr(tt), _ptr(dl)), "run_b")
    return float(tt[0]), float(dl[0])


def face_states_b(P, Q, L):
    n = P.nx * P.ny * P.nz
    fs = np.zeros((6, 4, 20, n))
    _check(lib().orc_face_states_b(ctypes.byref(P), _ptr(Q), _ptr(L), _ptr(fs)), "face_states_b")
    return fs


def geno_misfit(q0, dvec):
    """GENO's misfit sigma (reading R5) of one cell's five variables."""
    out = np.zeros(5)
    _check(lib().orc_geno_misfit(_ptr(np.ascontiguousarray(q0, float)),
                                 _ptr(np.ascontiguousarray(dvec, float)), _ptr(out)), "geno_misfit")
    return out


def chi_field(P, Q, G):
    """GENO's chi of every (variable, cell) of a CGKS-5th state: [5][cells]."""
    n = P.nx * P.ny * P.nz
    chi = np.zeros((5, n))
    _check(lib().orc_chi_field(ctypes.byref(P), _ptr(Q), _ptr(G), _ptr(chi)), "chi_field")
    return chi


def recon5_cell(q0, dvec, h=(1.0, 1.0, 1.0), nonlinear=1):
    out = np.zeros(480)
    chi = np.zeros(5)
    _check(lib().orc_recon5_cell(_ptr(np.ascontiguousarray(q0, float)),
                                 _ptr(np.ascontiguousarray(dvec, float)),
                                 h[0], h[1], h[2], nonlinear, _ptr(out), _ptr(chi)), "recon5_cell")
    return out.reshape(6, 4, 20), chi


def recon2_cell(q7, h=(1.0, 1.0, 1.0), nonlinear=1):
    out = np.zeros(120)
    phi = np.zeros(5)
    _check(lib().orc_recon2_cell(_ptr(np.ascontiguousarray(q7, float)), h[0], h[1], h[2],
                                 nonlinear, _ptr(out), _ptr(phi)), "recon2_cell")
    return out.reshape(6, 20), phi


def dt(P, Q):
    out = np.zeros(1)
    _check(lib().orc_dt(ctypes.byref(P), _ptr(Q), _ptr(out)), "dt")
    return float(out[0])


def run(P, Q, G=None, nsteps=1, t_stop=np.inf, t=0.0):
    """Advance in place; returns (t, dt_last)."""
    tt = np.array([t], float)
    dl = np.zeros(1)
    _check(lib().orc_run(ctypes.byref(P), _ptr(Q), _ptr(G), nsteps, t_stop,
                         _ptr(tt), _ptr(dl)), "run")
    return float(tt[0]), float(dl[0])


def n_plane(P):
    """Size of the boundary-face planes: max(ny nz, nx nz, nx ny)."""
    return max(P.ny * P.nz, P.nx * P.nz, P.nx * P.ny)


def stage(P, Q, G, dt_, boundary=False):
    """L, Lt [5][cells] and the face records [3][30][cells]; with
    boundary=True also the high-boundary records [3][30][n_plane]."""
    n = P.nx * P.ny * P.nz
    L = np.zeros((5, n))
    Lt = np.zeros((5, n))
    faces = np.zeros((3, 30, n))
    fhi = np.zeros((3, 30, n_plane(P)))
    _check(lib().orc_stage(ctypes.byref(P), _ptr(Q), _ptr(G), dt_, _ptr(L), _ptr(Lt),
                           _ptr(faces), _ptr(fhi)), "stage")
    return (L, Lt, faces, fhi) if boundary else (L, Lt, faces)


def face_states(P, Q, G):
    n = P.nx * P.ny * P.nz
    ngp = 4 if P.scheme else 1
    fs = np.zeros((6, ngp, 20, n))
    _check(lib().orc_face_states(ctypes.byref(P), _ptr(Q), _ptr(G), _ptr(fs)), "face_states")
    return fs


def face_states_at(P, Q, G, cells):
    """Face states of the listed cells: [m][6][ngp][20]."""
    cells = np.ascontiguousarray(cells, dtype=np.int64)
    ngp = 4 if P.scheme else 1
    out = np.zeros((cells.size, 6, ngp, 20))
    _check(lib().orc_face_states_at(ctypes.byref(P), _ptr(Q), _ptr(G),
                                    cells.ctypes.data_as(ctypes.POINTER(ctypes.c_longlong)),
                                    cells.size, _ptr(out)), "face_states_at")
    return out


def face_record(P, d, sl, sr, dt_):
    """Record of one face normal to axis d from sl, sr [ngp][20] (face
    frame): 30 values, global frame."""
    out = np.zeros(30)
    _check(lib().orc_face_record(ctypes.byref(P), int(d),
                                 _ptr(np.ascontiguousarray(sl, float)),
                                 _ptr(np.ascontiguousarray(sr, float)), dt_, _ptr(out)),
           "face_record")
    return out


def diagnostics(P, Q, G=None):
    out = np.zeros(12)
    _check(lib().orc_diagnostics(ctypes.byref(P), _ptr(Q), _ptr(G), _ptr(out)), "diagnostics")
    return out


def mlp_loss_grad(params, x, y, neg_weight=1.0):
    """Indicator network loss and gradient in FP64 (x: [63][n] samples)."""
    params = np.ascontiguousarray(params, dtype=np.float64)
    x = np.ascontiguousarray(x, dtype=np.float64)
    y = np.ascontiguousarray(y, dtype=np.float64)
    n = y.shape[0]
    loss = np.zeros(1)
    grad = np.zeros(lib().orc_mlp_nparams())
    _check(lib().orc_mlp_loss_grad(_ptr(params), _ptr(x), _ptr(y), n, x.shape[1], neg_weight,
                                   _ptr(loss), _ptr(grad)), "mlp_loss_grad")
    return float(loss[0]), grad
