"""ctypes binding of the C ABI in include/sacra2d.h (argument marshalling only).

The compiled library (paper_2502_03223_gb300/_build/libsacra2d.so, built by
``paper_2502_03223_gb300.build.build()``) does all the arithmetic on the GPU.
There is no CPU fallback: if the library is missing, importing it fails.
PyTorch, when present, provides the device arena and the CUDA stream.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "_build", "libsacra2d.so")

SACRA_OK = 0
PLANAR, CYLINDRICAL = 0, 1
HLLC, TVDLF = 0, 1
RK4, SSPRK3 = 0, 1
FP64, MIXED_FLUX, MIXED_SOURCES, MIXED_Z4C, MIXED = 0, 1, 2, 4, 7
PRIM_METRIC, RAW = 0, 1
FILL, RESTRICT_REFLUX = 0, 1
STATE_STEP, STATE_STAGE, PRIMS, RHS, STATUS = 0, 1, 2, 3, 4

EXPORTS = ["sacra_arena_bytes", "sacra_init_grid", "sacra_set_initial_data", "sacra_regrid_ghosts",
           "sacra_rk_stage", "sacra_step", "sacra_step_constraints", "sacra_read_state", "sacra_read_level",
           "sacra_constraints", "sacra_sync", "sacra_launch_count", "sacra_profile", "sacra_profile_get", "sacra_hydro_rhs_noalloc", "sacra_tune",
           "sacra_get_tuning", "sacra_set_tuning", "sacra_destroy", "sacra_last_error",
           "sacra_batch_arena_bytes", "sacra_init_batch", "sacra_batch_set_initial_data", "sacra_batch_step",
           "sacra_batch_read_state", "sacra_batch_constraints", "sacra_batch_tune", "sacra_batch_get_tuning",
           "sacra_batch_set_tuning", "sacra_batch_sync", "sacra_batch_launch_count", "sacra_batch_profile", "sacra_batch_profile_get",
           "sacra_batch_destroy", "sacra_batch_last_error", "sacra_mlp_bytes", "sacra_mlp_collect",
           "sacra_mlp_train", "sacra_mlp_grad", "sacra_set_mlp", "sacra_c2p_counting", "sacra_c2p_counts",
           "sacra_batch_set_mlp", "sacra_batch_mlp_collect"]
EXPORTS = sorted(EXPORTS)
MLP_NPARAM = 4865
KIND_NAMES = ["flux_x", "flux_z", "hydro_rhs", "cartoon", "z4c_derivs", "z4c_point", "rk_update"]


class SacraParams(C.Structure):
    _fields_ = [
        ("n_levels", C.c_int), ("nx", C.c_int), ("nz", C.c_int), ("geometry", C.c_int),
        ("evolve_spacetime", C.c_int), ("solver", C.c_int), ("rk", C.c_int), ("c2p_maxit", C.c_int),
        ("precision", C.c_int), ("subcycle_from", C.c_int), ("hydro_outer", C.c_int),
        ("eos_adiabatic", C.c_int), ("n_pieces", C.c_int), ("bssn", C.c_int),
        ("dx0", C.c_double), ("dz0", C.c_double),
        ("kappa", C.c_double), ("eta_B", C.c_double), ("eps_ko", C.c_double), ("r_z4", C.c_double),
        ("K", C.c_double), ("Gamma", C.c_double), ("Gamma_th", C.c_double),
        ("rho_atm", C.c_double), ("w_max", C.c_double), ("c2p_tol", C.c_double), ("r_hold", C.c_double),
        ("pwp_rho", C.c_double * 7), ("pwp_Gamma", C.c_double * 7),
    ]


class SacraDiag(C.Structure):
    _fields_ = [("H_L2", C.c_double), ("M_L2", C.c_double * 3), ("Mb", C.c_double), ("J", C.c_double),
                ("rho_max", C.c_double), ("n_c2p_fail", C.c_double), ("n_fallback", C.c_double)]


_lib = None


def load(path: str = LIB_PATH):
    """Load the compiled library; raises if it has not been built."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError("libsacra2d.so not built (run paper_2502_03223_gb300.build.build()): " + path)
    L = C.CDLL(path)
    vp, dp = C.c_void_p, C.POINTER(C.c_double)
    L.sacra_arena_bytes.argtypes = [C.POINTER(SacraParams), C.POINTER(C.c_size_t)]
    L.sacra_init_grid.argtypes = [C.POINTER(SacraParams), vp, vp, C.c_size_t, C.POINTER(vp)]
    L.sacra_set_initial_data.argtypes = [vp, C.c_int, C.c_int, dp, C.c_int]
    L.sacra_regrid_ghosts.argtypes = [vp, C.c_int, C.c_int, C.c_double]
    L.sacra_rk_stage.argtypes = [vp, C.c_int, C.c_double]
    L.sacra_step.argtypes = [vp, C.c_double, C.c_int, C.c_int]
    L.sacra_step_constraints.argtypes = [vp, C.c_double, C.c_int, C.c_int, C.POINTER(SacraDiag)]
    L.sacra_read_state.argtypes = [vp, C.c_int, C.c_int, C.c_int, dp, C.c_size_t]
    L.sacra_read_level.argtypes = [vp, C.c_int, C.c_int, vp, C.c_int]
    L.sacra_constraints.argtypes = [vp, C.POINTER(SacraDiag)]
    L.sacra_sync.argtypes = [vp]
    L.sacra_launch_count.argtypes = [vp]
    L.sacra_launch_count.restype = C.c_longlong
    L.sacra_profile.argtypes = [vp, C.c_int]
    L.sacra_profile.restype = C.c_int
    L.sacra_profile_get.argtypes = [vp, C.c_int, C.c_char_p, C.c_size_t, dp, C.POINTER(C.c_longlong),
                                    C.POINTER(C.c_longlong)]
    L.sacra_profile_get.restype = C.c_int
    L.sacra_hydro_rhs_noalloc.argtypes = [C.POINTER(SacraParams), C.c_int, vp, vp, vp, vp]
    L.sacra_hydro_rhs_noalloc.restype = C.c_int
    ip = C.POINTER(C.c_int)
    L.sacra_tune.argtypes = [vp, C.c_int]
    L.sacra_tune.restype = C.c_int
    L.sacra_get_tuning.argtypes = [vp, C.c_int, ip, ip, ip]
    L.sacra_get_tuning.restype = C.c_int
    L.sacra_set_tuning.argtypes = [vp, C.c_int, C.c_int, C.c_int, C.c_int]
    L.sacra_set_tuning.restype = C.c_int
    L.sacra_destroy.argtypes = [vp]
    L.sacra_last_error.argtypes = [vp]
    L.sacra_last_error.restype = C.c_char_p
    # batches
    PP = C.POINTER(SacraParams)
    L.sacra_batch_arena_bytes.argtypes = [PP, C.c_int, C.POINTER(C.c_size_t)]
    L.sacra_init_batch.argtypes = [PP, C.c_int, vp, vp, C.c_size_t, C.POINTER(vp)]
    L.sacra_batch_set_initial_data.argtypes = [vp, C.c_int, C.c_int, C.c_int, dp, C.c_int]
    L.sacra_batch_step.argtypes = [vp, C.c_double, C.c_int, C.c_int]
    L.sacra_batch_read_state.argtypes = [vp, C.c_int, C.c_int, C.c_int, C.c_int, dp, C.c_size_t]
    L.sacra_batch_constraints.argtypes = [vp, C.c_int, C.POINTER(SacraDiag)]
    L.sacra_batch_tune.argtypes = [vp, C.c_int]
    L.sacra_batch_get_tuning.argtypes = [vp, C.c_int, ip, ip, ip]
    L.sacra_batch_set_tuning.argtypes = [vp, C.c_int, C.c_int, C.c_int, C.c_int]
    L.sacra_batch_sync.argtypes = [vp]
    L.sacra_batch_launch_count.argtypes = [vp]
    L.sacra_batch_launch_count.restype = C.c_longlong
    L.sacra_batch_profile.argtypes = [vp, C.c_int]
    L.sacra_batch_profile_get.argtypes = [vp, C.c_int, C.c_char_p, C.c_size_t, dp, C.POINTER(C.c_longlong),
                                          C.POINTER(C.c_longlong)]
    L.sacra_batch_destroy.argtypes = [vp]
    L.sacra_batch_last_error.argtypes = [vp]
    L.sacra_batch_last_error.restype = C.c_char_p
    fp = C.POINTER(C.c_float)
    L.sacra_mlp_bytes.argtypes = []
    L.sacra_mlp_bytes.restype = C.c_size_t
    L.sacra_mlp_collect.argtypes = [vp, vp, C.c_longlong, C.POINTER(C.c_longlong)]
    L.sacra_mlp_train.argtypes = [vp, C.c_longlong, C.c_int, C.c_int, C.c_float, C.c_ulonglong, C.c_float, vp, fp, fp, vp]
    L.sacra_mlp_grad.argtypes = [vp, C.c_longlong, vp, fp, fp, vp]
    L.sacra_set_mlp.argtypes = [vp, vp]
    L.sacra_c2p_counting.argtypes = [vp, C.c_int]
    L.sacra_c2p_counts.argtypes = [vp, C.POINTER(C.c_longlong), C.c_int]
    L.sacra_batch_set_mlp.argtypes = [vp, vp]
    L.sacra_batch_mlp_collect.argtypes = [vp, vp, C.c_longlong, C.POINTER(C.c_longlong)]
    for name in ("sacra_mlp_collect", "sacra_mlp_train", "sacra_mlp_grad", "sacra_set_mlp", "sacra_c2p_counting",
                 "sacra_c2p_counts", "sacra_batch_set_mlp", "sacra_batch_mlp_collect"):
        getattr(L, name).restype = C.c_int
    for name in ("sacra_batch_arena_bytes", "sacra_init_batch", "sacra_batch_set_initial_data", "sacra_batch_step",
                 "sacra_batch_read_state", "sacra_batch_constraints", "sacra_batch_tune", "sacra_batch_get_tuning",
                 "sacra_batch_set_tuning", "sacra_batch_sync", "sacra_batch_profile", "sacra_batch_profile_get"):
        getattr(L, name).restype = C.c_int
    for name in ("sacra_arena_bytes", "sacra_init_grid", "sacra_set_initial_data", "sacra_regrid_ghosts",
                 "sacra_rk_stage", "sacra_step", "sacra_step_constraints", "sacra_read_state", "sacra_read_level",
                 "sacra_constraints", "sacra_sync"):
        getattr(L, name).restype = C.c_int
    _lib = L
    return L


def make_params(cfg) -> SacraParams:
    p = SacraParams()
    p.n_levels = int(cfg.n_levels); p.nx = int(cfg.nx); p.nz = int(cfg.nz)
    p.geometry = int(cfg.geometry); p.evolve_spacetime = int(cfg.evolve_spacetime)
    p.solver = int(cfg.solver); p.rk = int(cfg.rk); p.c2p_maxit = int(cfg.c2p_maxit)
    p.precision = int(getattr(cfg, "precision", 0))
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


def hydro_rhs_noalloc(cfg, level, state_ptr, prims_ptr, rhs_ptr, stream_ptr=0):
    """sacra_hydro_rhs_noalloc on device pointers (integers); returns the status."""
    L = load()
    p = make_params(cfg)
    return L.sacra_hydro_rhs_noalloc(C.byref(p), int(level), C.c_void_p(state_ptr), C.c_void_p(prims_ptr),
                                     C.c_void_p(rhs_ptr), C.c_void_p(stream_ptr))


class SacraError(RuntimeError):
    pass


class Sacra:
    """One level hierarchy on the GPU.  The arena is a torch uint8 tensor on
    the current CUDA device and the work runs on ``stream`` (a
    torch.cuda.Stream; default: a new non-default stream, so that whole steps
    can be captured in CUDA graphs)."""

    def __init__(self, cfg, stream=None):
        import torch
        self.cfg = cfg
        self._L = load()
        self._p = make_params(cfg)
        nbytes = C.c_size_t(0)
        if self._L.sacra_arena_bytes(C.byref(self._p), C.byref(nbytes)) != SACRA_OK:
            raise SacraError("configuration rejected by sacra_arena_bytes")
        self.arena_bytes = nbytes.value
        self.stream = stream if stream is not None else torch.cuda.Stream()
        self._arena = torch.empty(self.arena_bytes, dtype=torch.uint8, device="cuda")
        ctx = C.c_void_p()
        rc = self._L.sacra_init_grid(C.byref(self._p), C.c_void_p(self.stream.cuda_stream),
                                     C.c_void_p(self._arena.data_ptr()), nbytes, C.byref(ctx))
        if rc != SACRA_OK:
            raise SacraError("sacra_init_grid failed with status %d" % rc)
        self._c = ctx
        self.px, self.pz = cfg.nx + 16, cfg.nz + 16

    def _chk(self, rc, what):
        if rc != SACRA_OK:
            msg = self._L.sacra_last_error(self._c).decode()
            raise SacraError("%s failed (%d): %s" % (what, rc, msg))

    def close(self):
        if getattr(self, "_c", None):
            self._L.sacra_destroy(self._c)
            self._c = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_initial_data(self, level, kind, planes):
        a = np.ascontiguousarray(planes, dtype=np.float64)
        assert a.size == 30 * self.px * self.pz
        self._chk(self._L.sacra_set_initial_data(self._c, level, kind, a.ctypes.data_as(C.POINTER(C.c_double)), 30),
                  "set_initial_data")

    def regrid_ghosts(self, what, stage=0, dt=0.0):
        self._chk(self._L.sacra_regrid_ghosts(self._c, what, stage, dt), "regrid_ghosts")

    def fill(self, stage, dt):
        self.regrid_ghosts(FILL, stage, dt)

    def restrict_reflux(self):
        self.regrid_ghosts(RESTRICT_REFLUX)

    def rk_stage(self, stage, dt):
        self._chk(self._L.sacra_rk_stage(self._c, stage, dt), "rk_stage")

    def step(self, dt, n=1, use_graph=False):
        self._chk(self._L.sacra_step(self._c, dt, n, 1 if use_graph else 0), "step")

    def step_constraints(self, dt, n=1, use_graph=False):
        """n steps; row i holds the diagnostics of the state at the start of
        step i (formed inside its first stage), in the order of constraints()."""
        d = (SacraDiag * max(n, 1))()
        self._chk(self._L.sacra_step_constraints(self._c, dt, n, 1 if use_graph else 0, d), "step_constraints")
        return np.array([[x.H_L2, x.M_L2[0], x.M_L2[1], x.M_L2[2], x.Mb, x.J, x.rho_max, x.n_c2p_fail, x.n_fallback]
                         for x in d[:n]]).reshape(n, 9)

    def sync(self):
        self._chk(self._L.sacra_sync(self._c), "sync")

    def read(self, level, which, field, padded=True):
        n = self.px * self.pz if padded else self.cfg.nx * self.cfg.nz
        out = np.zeros(n)
        self._chk(self._L.sacra_read_state(self._c, level, which, field, out.ctypes.data_as(C.POINTER(C.c_double)), n),
                  "read_state")
        return out.reshape((self.pz, self.px) if padded else (self.cfg.nz, self.cfg.nx))

    def read_level(self, level, out, which=STATE_STEP):
        """All 30 padded state planes of `level` into `out` (a contiguous
        float64 array of 30 * pz * px elements, e.g. pinned torch memory as
        numpy), the layout set_initial_data(RAW) takes."""
        assert out.dtype == np.float64 and out.flags["C_CONTIGUOUS"] and out.size == 30 * self.px * self.pz
        self._chk(self._L.sacra_read_level(self._c, level, which, out.ctypes.data, 30), "read_level")
        return out

    def constraints(self):
        d = SacraDiag()
        self._chk(self._L.sacra_constraints(self._c, C.byref(d)), "constraints")
        return np.array([d.H_L2, d.M_L2[0], d.M_L2[1], d.M_L2[2], d.Mb, d.J, d.rho_max, d.n_c2p_fail, d.n_fallback])

    def profile(self, enable=True):
        self._chk(self._L.sacra_profile(self._c, 1 if enable else 0), "profile")

    def profile_report(self):
        """{kernel name: (total ms, launches, cells)} of the launches recorded since profile(True)."""
        out = {}
        idx = 0
        buf = C.create_string_buffer(64)
        while True:
            ms = C.c_double(0.0); n = C.c_longlong(0); cells = C.c_longlong(0)
            rc = self._L.sacra_profile_get(self._c, idx, buf, 64, C.byref(ms), C.byref(n), C.byref(cells))
            if rc != SACRA_OK:
                break
            if n.value:
                out[buf.value.decode()] = (ms.value, n.value, cells.value)
            idx += 1
        return out

    @property
    def launch_count(self):
        return self._L.sacra_launch_count(self._c)

    @property
    def n_stages(self):
        return 4 if self.cfg.rk == 0 else 3

    def mlp_collect(self, out):
        """Append-free dump of recovery tuples into `out` (CUDA float32 (cap, 10)); returns the count."""
        n = C.c_longlong(0)
        self._chk(self._L.sacra_mlp_collect(self._c, C.c_void_p(out.data_ptr()), out.shape[0], C.byref(n)),
                  "mlp_collect")
        return n.value

    def set_mlp(self, net):
        """Use a trained seed network (CUDA uint8 tensor, kept alive by the caller); None disables."""
        self._net = net
        self._chk(self._L.sacra_set_mlp(self._c, C.c_void_p(net.data_ptr()) if net is not None else None), "set_mlp")

    def c2p_counting(self, enable=True):
        self._chk(self._L.sacra_c2p_counting(self._c, 1 if enable else 0), "c2p_counting")

    def c2p_counts(self, reset=False):
        """(Illinois evaluations, seeded tries, seeded brackets that held, recoveries)."""
        out = (C.c_longlong * 4)()
        self._chk(self._L.sacra_c2p_counts(self._c, out, 1 if reset else 0), "c2p_counts")
        return tuple(out)

    def tune(self, reps=3):
        """Run the autotuner of the batched launches; returns {kind: (tile_x, tile_y, blocks_per_sm)}."""
        self._chk(self._L.sacra_tune(self._c, reps), "tune")
        return self.tuning()

    def tuning(self):
        out = {}
        for k, name in enumerate(KIND_NAMES):
            x, y, m = C.c_int(0), C.c_int(0), C.c_int(0)
            self._chk(self._L.sacra_get_tuning(self._c, k, C.byref(x), C.byref(y), C.byref(m)), "get_tuning")
            out[name] = (x.value, y.value, m.value)
        return out

    def set_tuning(self, kind, tile_x, tile_y, blocks_per_sm):
        """Pin one kernel kind's tile shape and persistent grid size (kind: index or name)."""
        k = KIND_NAMES.index(kind) if isinstance(kind, str) else int(kind)
        self._chk(self._L.sacra_set_tuning(self._c, k, tile_x, tile_y, blocks_per_sm), "set_tuning")


def mlp_train(tuples, steps=2000, batch_blocks=32, lr=3e-3, seed=1, record_loss=False, stream=None, kmin=0.0):
    """Train the recovery seed on the GPU.  tuples: a CUDA float32 tensor of
    shape (n, 10).  Returns (net: CUDA uint8 tensor, report: dict, loss history)."""
    import torch
    L = load()
    assert tuples.is_cuda and tuples.dtype == torch.float32 and tuples.shape[1] == 10
    net = torch.zeros(L.sacra_mlp_bytes(), dtype=torch.uint8, device="cuda")
    hist = np.zeros(max(steps, 1), dtype=np.float32) if record_loss else None
    rep = np.zeros(3, dtype=np.float32)
    st = stream if stream is not None else torch.cuda.current_stream()
    fpp = C.POINTER(C.c_float)
    rc = L.sacra_mlp_train(C.c_void_p(tuples.data_ptr()), tuples.shape[0], steps, batch_blocks, lr, seed, kmin,
                           C.c_void_p(net.data_ptr()), hist.ctypes.data_as(fpp) if record_loss else None,
                           rep.ctypes.data_as(fpp), C.c_void_p(st.cuda_stream))
    if rc != SACRA_OK:
        raise SacraError("sacra_mlp_train failed with status %d" % rc)
    return net, {"val_rms_log10": float(rep[0]), "z_err_q999": float(rep[1]), "delta": float(rep[2])}, hist


def mlp_grad(tuples, net, stream=None):
    """Full-batch gradient (4865 floats, the oracle's flat order) and loss."""
    import torch
    L = load()
    g = np.zeros(MLP_NPARAM, dtype=np.float32)
    loss = C.c_float(0.0)
    st = stream if stream is not None else torch.cuda.current_stream()
    rc = L.sacra_mlp_grad(C.c_void_p(tuples.data_ptr()), tuples.shape[0], C.c_void_p(net.data_ptr()),
                          g.ctypes.data_as(C.POINTER(C.c_float)), C.byref(loss), C.c_void_p(st.cuda_stream))
    if rc != SACRA_OK:
        raise SacraError("sacra_mlp_grad failed with status %d" % rc)
    return g, float(loss.value)


def mlp_unpack(net_bytes):
    """Host view of a packed network (numpy uint8 array): dict of float64 arrays."""
    b = np.asarray(net_bytes, dtype=np.uint8)
    def bf(o, n):
        u = b[o:o + 2 * n].view(np.uint16).astype(np.uint32) << 16
        return u.view(np.float32).astype(np.float64)
    def f(o, n):
        return b[o:o + 4 * n].view(np.float32).astype(np.float64)
    o = 0
    w1 = bf(o, 576).reshape(64, 9); o += 1152
    w2 = bf(o, 4096).reshape(64, 64); o += 8192
    w3 = bf(o, 64); o += 128 + 8
    b1 = f(o, 64); o += 256
    b2 = f(o, 64); o += 256
    b3 = f(o, 1)[0]; o += 4
    in_mu = f(o, 9); o += 36
    in_sd = f(o, 9); o += 36
    out_mu, out_sd, delta, kmin = f(o, 4)
    return {"w1": w1, "b1": b1, "w2": w2, "b2": b2, "w3": w3, "b3": b3, "in_mu": in_mu, "in_sd": in_sd,
            "out_mu": out_mu, "out_sd": out_sd, "delta": delta, "kmin": kmin}


class SacraBatch:
    """Many independent stars advanced together (one persistent launch per
    kernel kind and RK stage over all of them).  cfgs: one RunConfig per star;
    they must agree in geometry, evolve_spacetime, solver, rk and precision
    and may differ in everything else (grid, EOS, gauge, atmosphere, ...)."""

    def __init__(self, cfgs, stream=None):
        import torch
        self.cfgs = list(cfgs)
        self._L = load()
        n = len(self.cfgs)
        self._p = (SacraParams * n)(*[make_params(c) for c in self.cfgs])
        nbytes = C.c_size_t(0)
        if self._L.sacra_batch_arena_bytes(self._p, n, C.byref(nbytes)) != SACRA_OK:
            raise SacraError("configuration rejected by sacra_batch_arena_bytes")
        self.arena_bytes = nbytes.value
        self.stream = stream if stream is not None else torch.cuda.Stream()
        self._arena = torch.empty(self.arena_bytes, dtype=torch.uint8, device="cuda")
        b = C.c_void_p()
        rc = self._L.sacra_init_batch(self._p, n, C.c_void_p(self.stream.cuda_stream),
                                      C.c_void_p(self._arena.data_ptr()), nbytes, C.byref(b))
        if rc != SACRA_OK:
            raise SacraError("sacra_init_batch failed with status %d" % rc)
        self._b = b

    def _chk(self, rc, what):
        if rc != SACRA_OK:
            raise SacraError("%s failed (%d): %s" % (what, rc, self._L.sacra_batch_last_error(self._b).decode()))

    def close(self):
        if getattr(self, "_b", None):
            self._L.sacra_batch_destroy(self._b)
            self._b = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_initial_data(self, star, level, kind, planes):
        a = np.ascontiguousarray(planes, dtype=np.float64)
        c = self.cfgs[star]
        assert a.size == 30 * (c.nx + 16) * (c.nz + 16)
        self._chk(self._L.sacra_batch_set_initial_data(self._b, star, level, kind,
                                                       a.ctypes.data_as(C.POINTER(C.c_double)), 30),
                  "batch_set_initial_data")

    def step(self, dt, n=1, use_graph=False):
        self._chk(self._L.sacra_batch_step(self._b, dt, n, 1 if use_graph else 0), "batch_step")

    def sync(self):
        self._chk(self._L.sacra_batch_sync(self._b), "batch_sync")

    def read(self, star, level, which, field):
        c = self.cfgs[star]
        px, pz = c.nx + 16, c.nz + 16
        out = np.zeros(px * pz)
        self._chk(self._L.sacra_batch_read_state(self._b, star, level, which, field,
                                                 out.ctypes.data_as(C.POINTER(C.c_double)), px * pz),
                  "batch_read_state")
        return out.reshape(pz, px)

    def constraints(self, star):
        d = SacraDiag()
        self._chk(self._L.sacra_batch_constraints(self._b, star, C.byref(d)), "batch_constraints")
        return np.array([d.H_L2, d.M_L2[0], d.M_L2[1], d.M_L2[2], d.Mb, d.J, d.rho_max, d.n_c2p_fail, d.n_fallback])

    def tune(self, reps=3):
        self._chk(self._L.sacra_batch_tune(self._b, reps), "batch_tune")
        return self.tuning()

    def mlp_collect(self, out):
        n = C.c_longlong(0)
        self._chk(self._L.sacra_batch_mlp_collect(self._b, C.c_void_p(out.data_ptr()), out.shape[0], C.byref(n)),
                  "batch_mlp_collect")
        return n.value

    def set_mlp(self, net):
        self._net = net
        self._chk(self._L.sacra_batch_set_mlp(self._b, C.c_void_p(net.data_ptr()) if net is not None else None),
                  "batch_set_mlp")

    def tuning(self):
        out = {}
        for k, name in enumerate(KIND_NAMES):
            x, y, m = C.c_int(0), C.c_int(0), C.c_int(0)
            self._chk(self._L.sacra_batch_get_tuning(self._b, k, C.byref(x), C.byref(y), C.byref(m)), "get_tuning")
            out[name] = (x.value, y.value, m.value)
        return out

    def set_tuning(self, kind, tile_x, tile_y, blocks_per_sm):
        """Pin one kernel kind's tile shape and persistent grid size (kind: index or name)."""
        k = KIND_NAMES.index(kind) if isinstance(kind, str) else int(kind)
        self._chk(self._L.sacra_batch_set_tuning(self._b, k, tile_x, tile_y, blocks_per_sm), "batch_set_tuning")

    def profile(self, enable=True):
        self._chk(self._L.sacra_batch_profile(self._b, 1 if enable else 0), "batch_profile")

    def profile_report(self):
        out = {}
        idx = 0
        buf = C.create_string_buffer(64)
        while True:
            ms = C.c_double(0.0); n = C.c_longlong(0); cells = C.c_longlong(0)
            rc = self._L.sacra_batch_profile_get(self._b, idx, buf, 64, C.byref(ms), C.byref(n), C.byref(cells))
            if rc != SACRA_OK:
                break
            if n.value:
                out[buf.value.decode()] = (ms.value, n.value, cells.value)
            idx += 1
        return out

    @property
    def launch_count(self):
        return self._L.sacra_batch_launch_count(self._b)
