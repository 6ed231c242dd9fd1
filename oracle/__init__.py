"""Reference oracle for the SACRA-2D hot path (Lam & Shibata, arXiv:2502.03223).

TEST INFRASTRUCTURE ONLY.  A plain FP64 CPU restatement of the method (C
sources in this directory, compiled with gcc, loaded through ctypes).  It
shares no code with the CUDA library in ``paper_2502_03223_gb300``; only the
tests, ``__graft_entry__.smoke()`` and the CPU-baseline leg of ``bench.py``
may import it.

Functions without an independent pin say so in their docstring ("parity
unpinned").
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_BUILD = os.path.join(_HERE, "_build")
_SOURCES = ["eos_c2p.c", "stencil.c", "riemann.c", "z4c.c", "grid.c"]
_LIBNAME = "liboracle.so"
_lock = threading.Lock()
_lib = None

G = 8
NMET, NCONS, NPRIM = 25, 5, 6
NSTATE = NMET + NCONS


def build(force: bool = False) -> str:
    """Compile the oracle into oracle/_build/liboracle.so (no FMA contraction,
    so x86 and Arm hosts round the same way)."""
    os.makedirs(_BUILD, exist_ok=True)
    out = os.path.join(_BUILD, _LIBNAME)
    srcs = [os.path.join(_HERE, s) for s in _SOURCES] + [os.path.join(_HERE, "orc.h")]
    if not force and os.path.exists(out):
        t = os.path.getmtime(out)
        if all(os.path.getmtime(s) <= t for s in srcs):
            return out
    tmp = out + ".tmp%d" % os.getpid()
    cmd = ["gcc", "-std=c11", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fopenmp", "-fPIC", "-shared", "-o", tmp]
    cmd += [os.path.join(_HERE, s) for s in _SOURCES] + ["-lm"]
    subprocess.check_call(cmd)
    os.replace(tmp, out)
    return out


def build_opcount(force: bool = False) -> str:
    """Compile the op-counting build of the oracle (oracle/opcount.cpp)."""
    os.makedirs(_BUILD, exist_ok=True)
    out = os.path.join(_BUILD, "opcount")
    srcs = [os.path.join(_HERE, s) for s in _SOURCES + ["orc.h", "opcount.cpp"]]
    if force or not os.path.exists(out) or any(os.path.getmtime(s) > os.path.getmtime(out) for s in srcs):
        tmp = out + ".tmp%d" % os.getpid()
        subprocess.check_call(["g++", "-std=c++17", "-O1", "-ffp-contract=off", "-w", "-o", tmp,
                               os.path.join(_HERE, "opcount.cpp")], cwd=_HERE)
        os.replace(tmp, out)
    return out


def opcount(cfg, level_data) -> dict:
    """Floating-point operations of one RK stage, per face or cell and per
    phase, counted on the oracle's plain restatement (see opcount.cpp)."""
    import json
    import tempfile
    exe = build_opcount()
    with tempfile.TemporaryDirectory() as td:
        files = []
        for l, d in enumerate(level_data):
            fn = os.path.join(td, "l%d.bin" % l)
            np.ascontiguousarray(d, dtype=np.float64).tofile(fn)
            files.append(fn)
        args = [exe, str(cfg.n_levels), str(cfg.nx), repr(cfg.dx0), repr(cfg.K), repr(cfg.Gamma), repr(cfg.Gamma_th),
                repr(cfg.rho_atm), repr(cfg.kappa), repr(cfg.eta_B), repr(cfg.r_z4)] + files
        out = subprocess.check_output(args, text=True)
    return json.loads(out)


class Params(C.Structure):
    _fields_ = [
        ("n_levels", C.c_int), ("nx", C.c_int), ("nz", C.c_int), ("geometry", C.c_int),
        ("evolve_spacetime", C.c_int), ("solver", C.c_int), ("rk", C.c_int), ("c2p_maxit", C.c_int),
        ("subcycle_from", C.c_int), ("hydro_outer", C.c_int), ("eos_adiabatic", C.c_int), ("n_pieces", C.c_int),
        ("bssn", C.c_int),
        ("dx0", C.c_double), ("dz0", C.c_double),
        ("kappa", C.c_double), ("eta_B", C.c_double), ("eps_ko", C.c_double), ("r_z4", C.c_double),
        ("K", C.c_double), ("Gamma", C.c_double), ("Gamma_th", C.c_double),
        ("rho_atm", C.c_double), ("w_max", C.c_double), ("c2p_tol", C.c_double), ("r_hold", C.c_double),
        ("pwp_rho", C.c_double * 7), ("pwp_Gamma", C.c_double * 7),
    ]


def make_params(cfg) -> Params:
    """Oracle parameter struct from any object carrying the run configuration
    attributes (see paper_2502_03223_gb300.workloads.RunConfig)."""
    p = Params()
    p.n_levels = int(cfg.n_levels); p.nx = int(cfg.nx); p.nz = int(cfg.nz)
    p.geometry = int(cfg.geometry); p.evolve_spacetime = int(cfg.evolve_spacetime)
    p.solver = int(cfg.solver); p.rk = int(cfg.rk); p.c2p_maxit = int(cfg.c2p_maxit)
    p.subcycle_from = int(getattr(cfg, "subcycle_from", 0))
    p.dx0 = float(cfg.dx0); p.dz0 = float(cfg.dz0)
    p.kappa = float(cfg.kappa); p.eta_B = float(cfg.eta_B); p.eps_ko = float(cfg.eps_ko); p.r_z4 = float(cfg.r_z4)
    p.K = float(cfg.K); p.Gamma = float(cfg.Gamma); p.Gamma_th = float(cfg.Gamma_th)
    p.rho_atm = float(cfg.rho_atm); p.w_max = float(cfg.w_max); p.c2p_tol = float(cfg.c2p_tol)
    p.hydro_outer = int(getattr(cfg, "hydro_outer", 0)); p.r_hold = float(getattr(cfg, "r_hold", 0.0))
    p.eos_adiabatic = int(getattr(cfg, "eos_adiabatic", 0))
    p.bssn = int(getattr(cfg, "bssn", 0))
    pieces = list(getattr(cfg, "pwp", ()) or ())       # [(rho_i, Gamma_(i+1)), ...]
    p.n_pieces = 1 + len(pieces)
    for i, (rt, gi) in enumerate(pieces):
        p.pwp_rho[i] = float(rt); p.pwp_Gamma[i] = float(gi)
    return p


_dp = C.POINTER(C.c_double)


def _ptr(a: np.ndarray):
    assert a.dtype == np.float64 and a.flags.c_contiguous
    return a.ctypes.data_as(_dp)


def lib():
    global _lib
    with _lock:
        if _lib is None:
            path = build()
            L = C.CDLL(path)
            P = C.POINTER(Params)
            L.orc_create.restype = C.c_void_p
            L.orc_set_threads.argtypes = [C.c_int]
            L.orc_get_threads.restype = C.c_int
            L.orc_create.argtypes = [P]
            L.orc_destroy.argtypes = [C.c_void_p]
            L.orc_set_level.argtypes = [C.c_void_p, C.c_int, C.c_int, _dp]
            L.orc_fill.argtypes = [C.c_void_p, C.c_int, C.c_double]
            L.orc_stage.argtypes = [C.c_void_p, C.c_int, C.c_double]
            L.orc_restrict_reflux.argtypes = [C.c_void_p]
            L.orc_step.argtypes = [C.c_void_p, C.c_double, C.c_int]
            L.orc_read.argtypes = [C.c_void_p, C.c_int, C.c_int, C.c_int, _dp]
            L.orc_diag.argtypes = [C.c_void_p, _dp]
            L.orc_fallbacks.argtypes = [C.c_void_p]
            L.orc_derivs_batch.argtypes = [C.c_void_p, C.c_int, C.c_int, C.POINTER(C.c_int), C.POINTER(C.c_int),
                                           _dp, _dp, _dp]
            L.orc_time_interp_probe.argtypes = [C.c_void_p, C.c_int, C.c_double, C.c_int, _dp, _dp]
            L.orc_stencil_init.argtypes = []
            L.orc_fd_weights.argtypes = [C.c_int, _dp, C.c_double, C.c_int, _dp]
            L.orc_lagrange.argtypes = [C.c_int, _dp, C.c_double, _dp]
            L.orc_eos_press.restype = C.c_double
            L.orc_eos_press.argtypes = [P, C.c_double, C.c_double]
            L.orc_eos_eps.restype = C.c_double
            L.orc_eos_eps.argtypes = [P, C.c_double, C.c_double]
            L.orc_eos_cs2.restype = C.c_double
            L.orc_eos_cs2.argtypes = [P, C.c_double, C.c_double, C.c_double]
            for nm in ("orc_eos_pcold", "orc_eos_ecold", "orc_eos_gamma_cold"):
                getattr(L, nm).restype = C.c_double
                getattr(L, nm).argtypes = [P, C.c_double]
            L.orc_prim2cons.argtypes = [P, _dp, C.c_double, _dp, C.c_double, _dp]
            L.orc_con2prim.restype = C.c_int
            L.orc_con2prim.argtypes = [P, _dp, C.c_double, _dp, C.c_double, _dp, C.POINTER(C.c_int)]
            L.orc_ppm_face.argtypes = [_dp, _dp, _dp]
            L.orc_riemann_flux.restype = C.c_int
            L.orc_riemann_flux.argtypes = [P, C.c_int, _dp, _dp, C.c_double, _dp, C.c_double, _dp, _dp]
            L.orc_z4c_point.argtypes = [P, _dp, _dp, _dp, _dp, C.c_double, _dp, _dp, C.c_double, _dp]
            L.orc_ricci_point.argtypes = [_dp, _dp, _dp, _dp]
            L.orc_constraints_point.argtypes = [_dp, _dp, _dp, C.c_double, _dp, _dp, _dp]
            L.orc_matter_point.argtypes = [P, _dp, C.c_double, _dp, _dp, _dp, _dp]
            L.orc_hydro_source.argtypes = [P, _dp, C.c_double, C.c_double, C.c_double, _dp, _dp, C.c_double, _dp,
                                           _dp, _dp, _dp, C.c_double, _dp]
            L.orc_stencil_init()
            _lib = L
    return _lib


# ---------------------------------------------------------------- point functions

def stencils() -> dict:
    """The weights the oracle derived from their definitions at start-up."""
    L = lib()
    out = {}
    for name, n in (("orc_c1", 7), ("orc_c2", 7), ("orc_lop", 7), ("orc_ko", 9), ("orc_face6", 6),
                    ("orc_prol8", 8), ("orc_rest8", 8)):
        arr = (C.c_double * n).in_dll(L, name)
        out[name[4:]] = np.array(arr[:], dtype=np.float64)
    return out


def fd_weights(nodes, x, deriv):
    nodes = np.ascontiguousarray(nodes, dtype=np.float64)
    w = np.zeros(len(nodes))
    lib().orc_fd_weights(len(nodes), _ptr(nodes), float(x), int(deriv), _ptr(w))
    return w


def lagrange(nodes, x):
    nodes = np.ascontiguousarray(nodes, dtype=np.float64)
    w = np.zeros(len(nodes))
    lib().orc_lagrange(len(nodes), _ptr(nodes), float(x), _ptr(w))
    return w


def eos_press(cfg, rho, eps):
    return lib().orc_eos_press(C.byref(make_params(cfg)), rho, eps)


def eos_eps(cfg, rho, press):
    return lib().orc_eos_eps(C.byref(make_params(cfg)), rho, press)


def eos_cs2(cfg, rho, eps, press):
    return lib().orc_eos_cs2(C.byref(make_params(cfg)), rho, eps, press)


def eos_pcold(cfg, rho):
    return lib().orc_eos_pcold(C.byref(make_params(cfg)), rho)


def eos_ecold(cfg, rho):
    return lib().orc_eos_ecold(C.byref(make_params(cfg)), rho)


def eos_gamma_cold(cfg, rho):
    return lib().orc_eos_gamma_cold(C.byref(make_params(cfg)), rho)


def set_threads(n):
    """Worker threads of the oracle's parallel loops (0: all processors)."""
    lib().orc_set_threads(int(n))


def get_threads():
    return lib().orc_get_threads()


def prim2cons(cfg, prim, W, h, x=1.0):
    """prim: (rho, u_x, u_y, u_z, P, eps); h: h_ij (xx,xy,xz,yy,yz,zz)."""
    pr = np.ascontiguousarray(prim, dtype=np.float64)
    hh = np.ascontiguousarray(h, dtype=np.float64)
    q = np.zeros(5)
    lib().orc_prim2cons(C.byref(make_params(cfg)), _ptr(pr), float(W), _ptr(hh), float(x), _ptr(q))
    return q


def con2prim(cfg, q, W, h, x=1.0):
    """Returns (prim[6], q_after[5], status, iterations)."""
    qq = np.array(q, dtype=np.float64)
    hh = np.ascontiguousarray(h, dtype=np.float64)
    pr = np.zeros(6)
    it = C.c_int(0)
    st = lib().orc_con2prim(C.byref(make_params(cfg)), _ptr(qq), float(W), _ptr(hh), float(x), _ptr(pr), C.byref(it))
    return pr, qq, st, it.value


def ppm_face(a6):
    a = np.ascontiguousarray(a6, dtype=np.float64)
    l = np.zeros(1); r = np.zeros(1)
    lib().orc_ppm_face(_ptr(a), _ptr(l), _ptr(r))
    return l[0], r[0]


def riemann_flux(cfg, direction, pl, pr, alpha, beta, W, h):
    """pl/pr: (rho, u_x, u_y, u_z, P).  Returns (flux[5], fallback)."""
    a = np.ascontiguousarray(pl, dtype=np.float64)
    b = np.ascontiguousarray(pr, dtype=np.float64)
    be = np.ascontiguousarray(beta, dtype=np.float64)
    hh = np.ascontiguousarray(h, dtype=np.float64)
    f = np.zeros(5)
    fb = lib().orc_riemann_flux(C.byref(make_params(cfg)), int(direction), _ptr(a), _ptr(b), float(alpha),
                                _ptr(be), float(W), _ptr(hh), _ptr(f))
    return f, fb


def z4c_point(cfg, Q, dQ, ddQ, adv, E, Si, Sij, fz=1.0):
    Q = np.ascontiguousarray(Q, dtype=np.float64)
    dQ = np.ascontiguousarray(dQ, dtype=np.float64).reshape(NMET, 3)
    ddQ = np.ascontiguousarray(ddQ, dtype=np.float64).reshape(NMET, 6)
    adv = np.ascontiguousarray(adv, dtype=np.float64)
    Si = np.ascontiguousarray(Si, dtype=np.float64)
    Sij = np.ascontiguousarray(Sij, dtype=np.float64)
    r = np.zeros(NMET)
    lib().orc_z4c_point(C.byref(make_params(cfg)), _ptr(Q), _ptr(dQ), _ptr(ddQ), _ptr(adv), float(E), _ptr(Si),
                        _ptr(Sij), float(fz), _ptr(r))
    return r


def hydro_source(cfg, prim, alpha, betay, W, h, A, K, dal, db, dW, dh, x=0.0):
    """Pointwise hydro sources (x > 0 adds the cylindrical geometric term).
    dal, dW: [2] (x, z); db: [2, 3]; dh: [2, 6]."""
    arr = lambda a: np.ascontiguousarray(a, dtype=np.float64)
    out = np.zeros(5)
    pr, hh, AA, da, dbb, dw, dhh = map(arr, (prim, h, A, dal, db, dW, dh))
    lib().orc_hydro_source(C.byref(make_params(cfg)), _ptr(pr), float(alpha), float(betay), float(W), _ptr(hh),
                           _ptr(AA), float(K), _ptr(da), _ptr(dbb), _ptr(dw), _ptr(dhh), float(x), _ptr(out))
    return out


def ricci_point(Q, dQ, ddQ):
    Q = np.ascontiguousarray(Q, dtype=np.float64)
    dQ = np.ascontiguousarray(dQ, dtype=np.float64).reshape(NMET, 3)
    ddQ = np.ascontiguousarray(ddQ, dtype=np.float64).reshape(NMET, 6)
    r = np.zeros(6)
    lib().orc_ricci_point(_ptr(Q), _ptr(dQ), _ptr(ddQ), _ptr(r))
    return r


def constraints_point(Q, dQ, ddQ, E, Si):
    Q = np.ascontiguousarray(Q, dtype=np.float64)
    dQ = np.ascontiguousarray(dQ, dtype=np.float64).reshape(NMET, 3)
    ddQ = np.ascontiguousarray(ddQ, dtype=np.float64).reshape(NMET, 6)
    Si = np.ascontiguousarray(Si, dtype=np.float64)
    H = np.zeros(1); M = np.zeros(3)
    lib().orc_constraints_point(_ptr(Q), _ptr(dQ), _ptr(ddQ), float(E), _ptr(Si), _ptr(H), _ptr(M))
    return H[0], M


def matter_point(cfg, prim, W, h):
    pr = np.ascontiguousarray(prim, dtype=np.float64)
    hh = np.ascontiguousarray(h, dtype=np.float64)
    E = np.zeros(1); Si = np.zeros(3); Sij = np.zeros(6)
    lib().orc_matter_point(C.byref(make_params(cfg)), _ptr(pr), float(W), _ptr(hh), _ptr(E), _ptr(Si), _ptr(Sij))
    return E[0], Si, Sij


# ---------------------------------------------------------------- hierarchy

class Oracle:
    """The whole level hierarchy on the CPU, with the same call sequence as
    the C ABI of the CUDA library: set_level -> (fill, stage)* -> restrict_reflux."""

    def __init__(self, cfg):
        self.cfg = cfg
        self._p = make_params(cfg)
        self._L = lib()
        self._c = self._L.orc_create(C.byref(self._p))
        if not self._c:
            raise ValueError("oracle rejected the configuration")
        self.px = cfg.nx + 2 * G
        self.pz = cfg.nz + 2 * G

    def close(self):
        if self._c:
            self._L.orc_destroy(self._c)
            self._c = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_level(self, level, kind, data):
        a = np.ascontiguousarray(data, dtype=np.float64)
        nf = 30 if kind == 0 else NSTATE
        assert a.size == nf * self.px * self.pz
        self._L.orc_set_level(self._c, level, kind, _ptr(a))

    def fill(self, stage, dt):
        self._L.orc_fill(self._c, stage, dt)

    def stage(self, stage, dt):
        self._L.orc_stage(self._c, stage, dt)

    def restrict_reflux(self):
        self._L.orc_restrict_reflux(self._c)

    def step(self, dt, n=1):
        self._L.orc_step(self._c, dt, n)

    def read(self, level, which, field):
        """which: 0 step-start state, 1 stage state, 2 primitives, 3 rhs, 4 status.
        Returns the padded (pz, px) plane."""
        out = np.zeros(self.px * self.pz)
        self._L.orc_read(self._c, level, which, field, _ptr(out))
        return out.reshape(self.pz, self.px)

    def diag(self):
        out = np.zeros(8)
        self._L.orc_diag(self._c, _ptr(out))
        return out

    def derivs(self, level, js, ks):
        """Derivatives of all metric fields of the step-start state at cells
        (js[i], ks[i]): (dQ[n,25,3], ddQ[n,25,6] in xx,xy,xz,yy,yz,zz, adv[n,25])."""
        js = np.ascontiguousarray(js, dtype=np.int32)
        ks = np.ascontiguousarray(ks, dtype=np.int32)
        n = len(js)
        dQ = np.zeros((n, NMET, 3)); ddQ = np.zeros((n, NMET, 6)); adv = np.zeros((n, NMET))
        ip = C.POINTER(C.c_int)
        self._L.orc_derivs_batch(self._c, level, n, js.ctypes.data_as(ip), ks.ctypes.data_as(ip),
                                 _ptr(dQ), _ptr(ddQ), _ptr(adv))
        return dQ, ddQ, adv

    def fallbacks(self):
        return self._L.orc_fallbacks(self._c)

    def time_interp(self, level, theta, have_old, old, now, new, p_old, p_now, p_new):
        """The parent data a sub-cycled child sees at t^n + theta (t^{n+1} - t^n)
        from the level's time slices (metric planes [25, pz, px] and primitive
        planes [6, pz, px] at t^{n-1}, t^n, t^{n+1}).  Returns (metric, prims)."""
        n = self.px * self.pz
        s = np.ascontiguousarray(np.concatenate([np.asarray(a, dtype=np.float64).ravel()
                                                 for a in (old, now, new, p_old, p_now, p_new)]))
        assert s.size == 3 * (NMET + 6) * n
        out = np.zeros((NMET + 6) * n)
        self._L.orc_time_interp_probe(self._c, level, float(theta), int(have_old), _ptr(s), _ptr(out))
        out = out.reshape(NMET + 6, self.pz, self.px)
        return out[:NMET], out[NMET:]

    @property
    def n_stages(self):
        return 4 if self.cfg.rk == 0 else 3
