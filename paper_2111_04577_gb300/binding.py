"""ctypes binding of the C ABI in include/dualpf.h (argument marshalling only).

Every step of the solver runs in the CUDA library; this module converts
NumPy arrays / torch tensors to pointers and sizes and raises on error codes.
There is no fallback: if the library is missing or no GPU is present the calls
fail loudly.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

from . import workloads as wl

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "_lib", "libdualpf.so")

PF_FP64, PF_MIXED, PF_MIXED_Z64, PF_MIXED_Z2F = 0, 1, 2, 3
PF_STEP_CH_ONLY, PF_STEP_NO_GRAPH = 1, 2

ERRORS = {-1: "PF_ERR_ARG", -2: "PF_ERR_DISCRIMINANT", -3: "PF_ERR_UNSUPPORTED", -4: "PF_ERR_NONFINITE",
          -5: "PF_ERR_TIMEOUT", -6: "PF_ERR_CUDA", -7: "PF_ERR_NOMEM"}

EXPORTS = ["pf_init_grid", "pf_set_params", "pf_field_info", "pf_set_fields", "pf_step", "pf_step_ex",
           "pf_get_fields", "pf_diagnostics", "pf_profile", "pf_diagnostics_noalloc", "pf_last_error",
           "pf_destroy", "pf_batch_create", "pf_batch_field_info", "pf_batch_set_fields", "pf_batch_get_fields",
           "pf_batch_step", "pf_batch_diagnostics", "pf_batch_last_error", "pf_batch_destroy", "pf_set_tuning",
           "pf_get_tuning", "pf_adjoint", "pf_batch_adjoint", "pf_tangent", "pf_tangent_ex", "pf_batch_tangent",
           "pf_adjoint_ex", "pf_batch_adjoint_ex"]
PF_OBJ_WETTED, PF_OBJ_CENTROID_Z = 0, 1
PF_ADJ_COUPLED = 1
PF_PARAM_WI, PF_PARAM_THETA_BOT, PF_PARAM_PHI0, PF_PARAM_MOBILITY = 0, 1, 2, 3
PROFILE_NAME = 48


class GridDesc(C.Structure):
    _fields_ = [("nx", C.c_int), ("ny", C.c_int), ("nz", C.c_int), ("lx", C.c_double), ("ly", C.c_double),
                ("lz", C.c_double), ("precision", C.c_int), ("dual", C.c_int)]


class ParamsC(C.Structure):
    _fields_ = [(n, C.c_double) for n in
                ("rho1", "rho2", "mu1", "mu2", "sigma", "eta", "mobility", "theta_bot_deg", "theta_top_deg",
                 "dw", "wi", "beta", "alpha_giesekus", "dt", "S", "nu_m", "uw_bot", "uw_top", "gx", "gy", "gz",
                 "mu_p2", "wi2", "alpha_giesekus2")] + [("polymer_approach", C.c_int), ("advection", C.c_int)]


class PFError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"{ERRORS.get(code, code)}: {msg}")
        self.code = code


_lib = None


def load(path: str = LIB_PATH):
    global _lib
    if _lib is None:
        if not os.path.exists(path):
            raise RuntimeError(f"CUDA library not built: {path} (run paper_2111_04577_gb300.build)")
        lib = C.CDLL(path)
        vp = C.c_void_p
        lib.pf_init_grid.argtypes = [C.POINTER(vp), C.POINTER(GridDesc), vp]
        lib.pf_set_params.argtypes = [vp, C.POINTER(ParamsC)]
        lib.pf_field_info.argtypes = [vp, C.c_int, C.POINTER(C.c_size_t), C.POINTER(C.c_size_t)]
        lib.pf_set_fields.argtypes = [vp, C.c_int, vp, C.c_size_t, C.c_int]
        lib.pf_get_fields.argtypes = [vp, C.c_int, vp, C.c_size_t, C.c_int]
        lib.pf_step.argtypes = [vp, C.c_int]
        lib.pf_step_ex.argtypes = [vp, C.c_int, C.c_int]
        lib.pf_diagnostics.argtypes = [vp, C.POINTER(C.c_double)]
        lib.pf_profile.argtypes = [vp, C.c_int, C.c_int, C.c_int, C.c_char_p, C.POINTER(C.c_double),
                                   C.POINTER(C.c_int), C.POINTER(C.c_int), C.POINTER(C.c_int)]
        lib.pf_diagnostics_noalloc.argtypes = [C.POINTER(GridDesc), C.POINTER(ParamsC), vp,
                                               C.POINTER(C.c_double), vp]
        lib.pf_diagnostics_noalloc.restype = C.c_int
        lib.pf_batch_create.argtypes = [C.POINTER(vp), C.c_int, C.POINTER(GridDesc), C.POINTER(ParamsC), vp]
        lib.pf_batch_field_info.argtypes = [vp, C.c_int, C.c_int, C.POINTER(C.c_size_t), C.POINTER(C.c_size_t)]
        lib.pf_batch_set_fields.argtypes = [vp, C.c_int, C.c_int, vp, C.c_size_t, C.c_int]
        lib.pf_batch_get_fields.argtypes = [vp, C.c_int, C.c_int, vp, C.c_size_t, C.c_int]
        lib.pf_batch_step.argtypes = [vp, C.c_int]
        lib.pf_batch_diagnostics.argtypes = [vp, C.c_int, C.POINTER(C.c_double)]
        lib.pf_batch_last_error.argtypes = [vp]
        lib.pf_batch_last_error.restype = C.c_char_p
        lib.pf_batch_destroy.argtypes = [vp]
        lib.pf_batch_destroy.restype = None
        for f in ("pf_batch_create", "pf_batch_field_info", "pf_batch_set_fields", "pf_batch_get_fields",
                  "pf_batch_step", "pf_batch_diagnostics"):
            getattr(lib, f).restype = C.c_int
        lib.pf_adjoint.argtypes = [vp, C.c_int, C.c_int, C.c_int, C.POINTER(C.c_double), vp, C.c_int]
        lib.pf_adjoint.restype = C.c_int
        lib.pf_adjoint_ex.argtypes = [vp, C.c_int, C.c_int, C.c_int, C.c_int, C.POINTER(C.c_double), vp, C.c_int]
        lib.pf_adjoint_ex.restype = C.c_int
        lib.pf_batch_adjoint_ex.argtypes = [vp, C.c_int, C.c_int, C.c_int, C.c_int, C.c_int, C.POINTER(C.c_double),
                                            vp, C.c_int]
        lib.pf_batch_adjoint_ex.restype = C.c_int
        lib.pf_batch_adjoint.argtypes = [vp, C.c_int, C.c_int, C.c_int, C.c_int, C.POINTER(C.c_double), vp, C.c_int]
        lib.pf_batch_adjoint.restype = C.c_int
        lib.pf_tangent.argtypes = [vp, C.c_int, C.c_int, C.c_int, C.POINTER(C.c_double)]
        lib.pf_tangent.restype = C.c_int
        lib.pf_tangent_ex.argtypes = [vp, C.c_int, C.c_int, C.c_int, C.c_int, vp, C.c_int, C.POINTER(C.c_double)]
        lib.pf_tangent_ex.restype = C.c_int
        lib.pf_batch_tangent.argtypes = [vp, C.c_int, C.c_int, C.c_int, C.c_int, C.c_int, vp, C.c_int,
                                         C.POINTER(C.c_double)]
        lib.pf_batch_tangent.restype = C.c_int
        lib.pf_set_tuning.argtypes = [vp, C.c_int, C.c_int]
        lib.pf_get_tuning.argtypes = [vp, C.c_int, C.POINTER(C.c_int)]
        lib.pf_set_tuning.restype = C.c_int
        lib.pf_get_tuning.restype = C.c_int
        lib.pf_last_error.argtypes = [vp]
        lib.pf_last_error.restype = C.c_char_p
        lib.pf_destroy.argtypes = [vp]
        lib.pf_destroy.restype = None
        for f in ("pf_init_grid", "pf_set_params", "pf_field_info", "pf_set_fields", "pf_get_fields",
                  "pf_step", "pf_step_ex", "pf_diagnostics", "pf_profile"):
            getattr(lib, f).restype = C.c_int
        _lib = lib
    return _lib


FIELD = {"phi": wl.PHI, "phi_old": wl.PHI_OLD, "u": wl.U, "u_old": wl.U_OLD, "v": wl.V, "v_old": wl.V_OLD,
         "w": wl.W, "w_old": wl.W_OLD, "p": wl.P, "p_old": wl.P_OLD, "theta": wl.THETA, "tau": wl.TAU,
         "tau_old": wl.TAU_OLD, "G": wl.G_FINE, "phi_rem": wl.PHI_REM}


class Solver:
    """One GPU context: grid + parameters + fields."""

    def __init__(self, grid: wl.Grid, params: wl.Params, precision=PF_FP64, stream=None):
        self.lib = load()
        self.grid = grid
        self.precision = precision
        self.dtype = np.float64 if precision == PF_FP64 else np.float32
        gd = GridDesc(grid.nx, grid.ny, grid.nz, grid.lx, grid.ly, grid.lz, precision, grid.dual)
        h = C.c_void_p()
        rc = self.lib.pf_init_grid(C.byref(h), C.byref(gd), C.c_void_p(stream or 0))
        if rc != 0:
            raise PFError(rc, self.lib.pf_last_error(None).decode())
        self.h = h
        self.set_params(params)

    def _chk(self, rc):
        if rc != 0:
            raise PFError(rc, self.lib.pf_last_error(self.h).decode())

    def set_params(self, params: wl.Params):
        self._chk(self.lib.pf_set_params(self.h, C.byref(ParamsC(**params.as_dict()))))

    def info(self, name):
        cnt, eb = C.c_size_t(), C.c_size_t()
        self._chk(self.lib.pf_field_info(self.h, FIELD[name], C.byref(cnt), C.byref(eb)))
        return cnt.value, eb.value

    def set(self, name, arr):
        """arr: NumPy array (host) or torch tensor (host or CUDA) of the field."""
        cnt, eb = self.info(name)
        try:
            import torch
            if isinstance(arr, torch.Tensor):
                t = arr.contiguous()
                want = torch.float64 if eb == 8 else torch.float32
                if t.dtype != want:
                    t = t.to(want)
                if t.numel() != cnt:
                    raise ValueError(f"{name}: {t.numel()} elements, expected {cnt}")
                self._chk(self.lib.pf_set_fields(self.h, FIELD[name], C.c_void_p(t.data_ptr()), cnt * eb,
                                                 1 if t.is_cuda else 0))
                return
        except ImportError:
            pass
        a = np.ascontiguousarray(arr, dtype=self.dtype)
        if a.size != cnt:
            raise ValueError(f"{name}: {a.size} elements, expected {cnt}")
        self._chk(self.lib.pf_set_fields(self.h, FIELD[name], a.ctypes.data_as(C.c_void_p), cnt * eb, 0))

    def get(self, name, out=None):
        cnt, eb = self.info(name)
        if out is not None:  # torch tensor on the device
            self._chk(self.lib.pf_get_fields(self.h, FIELD[name], C.c_void_p(out.data_ptr()), cnt * eb,
                                             1 if out.is_cuda else 0))
            return out
        a = np.empty(cnt, dtype=self.dtype)
        self._chk(self.lib.pf_get_fields(self.h, FIELD[name], a.ctypes.data_as(C.c_void_p), cnt * eb, 0))
        return a

    def step(self, n=1, flags=0):
        self._chk(self.lib.pf_step_ex(self.h, int(n), int(flags)))

    def diagnostics(self):
        out = (C.c_double * 6)()
        self._chk(self.lib.pf_diagnostics(self.h, out))
        return dict(mass=out[0], energy=out[1], wetted=out[2], centroid=(out[3], out[4], out[5]))

    def profile(self, nsteps=3, flags=0, max_entries=64):
        """Per-kernel device ms per step (direct launches, CUDA events).
        Returns (list of (name, ms_per_step, launches_per_step), total launches
        per step).  Advances the state by nsteps."""
        names = C.create_string_buffer(max_entries * PROFILE_NAME)
        ms = (C.c_double * max_entries)()
        cnt = (C.c_int * max_entries)()
        n, per = C.c_int(), C.c_int()
        self._chk(self.lib.pf_profile(self.h, int(nsteps), int(flags), max_entries, names, ms, cnt, C.byref(n),
                                      C.byref(per)))
        out = []
        for i in range(n.value):
            raw = names.raw[i * PROFILE_NAME:(i + 1) * PROFILE_NAME]
            out.append((raw.split(b"\0", 1)[0].decode(), ms[i], cnt[i]))
        return out, per.value

    def adjoint(self, nsteps, ckpt_every=50, objective=PF_OBJ_WETTED, want_phi=True):
        """(J, dJ/dtheta_bot [per degree], dJ/dmobility, dJ/dphi0 or None) of the CH
        step with the velocity fixed, from the current state; leaves phi^N."""
        out = (C.c_double * 3)()
        g = None
        ptr = None
        if want_phi:
            cnt, _ = self.info("phi")
            g = np.empty(cnt, dtype=self.dtype)
            ptr = g.ctypes.data_as(C.c_void_p)
        self._chk(self.lib.pf_adjoint(self.h, int(nsteps), int(ckpt_every), int(objective), out, ptr, 0))
        if g is not None:
            g = g.reshape(self.grid.fine_shape)
        return out[0], out[1], out[2], g

    def adjoint_coupled(self, nsteps, ckpt_every=50, objective=PF_OBJ_WETTED, want_phi=True):
        """(J, dJ/dtheta_bot [per degree], dJ/dmobility, dJ/dWi, dJ/dphi0 or None)
        through the whole coupled step (2D), by one reverse sweep from the
        current state; leaves the context at step N."""
        out = (C.c_double * 4)()
        g = None
        ptr = None
        if want_phi:
            cnt, _ = self.info("phi")
            g = np.empty(cnt, dtype=self.dtype)
            ptr = g.ctypes.data_as(C.c_void_p)
        self._chk(self.lib.pf_adjoint_ex(self.h, int(nsteps), int(ckpt_every), int(objective), PF_ADJ_COUPLED, out,
                                         ptr, 0))
        if g is not None:
            g = g.reshape(self.grid.fine_shape)
        return out[0], out[1], out[2], out[3], g

    def tangent(self, nsteps, param=PF_PARAM_WI, objective=PF_OBJ_WETTED, flags=0, direction=None):
        """(J, dJ/dparam) after nsteps steps from the current state, by forward-mode
        derivatives (pf_tangent_ex); the solver is not advanced.  dJ/dtheta_bot is
        per degree; with param=PF_PARAM_PHI0, dJ/dparam is <dJ/dphi^0, direction>
        (direction: a fine-mesh array).  flags=PF_STEP_CH_ONLY holds the velocity."""
        out = (C.c_double * 2)()
        ptr = None
        if direction is not None:
            direction = np.ascontiguousarray(direction, dtype=np.float64).ravel()
            ptr = direction.ctypes.data_as(C.c_void_p)
        self._chk(self.lib.pf_tangent_ex(self.h, int(nsteps), int(param), int(objective), int(flags), ptr, 0, out))
        return out[0], out[1]

    def set_tuning(self, knob, value):
        self._chk(self.lib.pf_set_tuning(self.h, int(knob), int(value)))

    def get_tuning(self, knob):
        v = C.c_int()
        self._chk(self.lib.pf_get_tuning(self.h, int(knob), C.byref(v)))
        return v.value

    def close(self):
        if getattr(self, "h", None):
            self.lib.pf_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # ---- conveniences in the oracle's array shapes ----
    def load_state(self, phi, vel=None, p=None, phi_old=None, vel_old=None):
        self.set("phi", phi)
        if phi_old is not None:
            self.set("phi_old", phi_old)
        if vel is not None:
            u, v, w = vel
            self.set("u", u)
            if self.grid.dim == 3:
                self.set("v", v)
            self.set("w", w)
            if vel_old is not None:
                uo, vo, wo = vel_old
                self.set("u_old", uo)
                if self.grid.dim == 3:
                    self.set("v_old", vo)
                self.set("w_old", wo)
        if p is not None:
            self.set("p", p)

    def fine(self, name="phi"):
        return self.get(name).reshape(self.grid.fine_shape).astype(np.float64)

    def coarse(self, name):
        g = self.grid
        nz, ny, nx = g.coarse_shape
        a = self.get(name).astype(np.float64)
        if name in ("w", "w_old"):
            return a.reshape(nz + 1, ny, nx)
        if name in ("theta", "tau", "tau_old"):
            nc = 3 if g.dim == 2 else 6
            return a.reshape(nc, nz, ny, nx)
        return a.reshape(nz, ny, nx)


class Batch:
    """Many independent 2D problems advanced by one persistent launch per step."""

    def __init__(self, grids, params, precision=PF_MIXED, stream=None):
        self.lib = load()
        n = len(grids)
        self.grids = list(grids)
        self.dtype = np.float64 if precision == PF_FP64 else np.float32
        gd = (GridDesc * n)(*[GridDesc(g.nx, g.ny, g.nz, g.lx, g.ly, g.lz, precision, g.dual) for g in grids])
        pr = (ParamsC * n)(*[ParamsC(**p.as_dict()) for p in params])
        h = C.c_void_p()
        rc = self.lib.pf_batch_create(C.byref(h), n, gd, pr, C.c_void_p(stream or 0))
        if rc != 0:
            raise PFError(rc, self.lib.pf_batch_last_error(None).decode())
        self.h = h

    def _chk(self, rc):
        if rc != 0:
            raise PFError(rc, self.lib.pf_batch_last_error(self.h).decode())

    def info(self, b, name):
        cnt, eb = C.c_size_t(), C.c_size_t()
        self._chk(self.lib.pf_batch_field_info(self.h, b, FIELD[name], C.byref(cnt), C.byref(eb)))
        return cnt.value, eb.value

    def set(self, b, name, arr):
        cnt, eb = self.info(b, name)
        a = np.ascontiguousarray(arr, dtype=self.dtype)
        if a.size != cnt:
            raise ValueError(f"{name}: {a.size} elements, expected {cnt}")
        self._chk(self.lib.pf_batch_set_fields(self.h, b, FIELD[name], a.ctypes.data_as(C.c_void_p), cnt * eb, 0))

    def get(self, b, name):
        cnt, eb = self.info(b, name)
        a = np.empty(cnt, dtype=self.dtype)
        self._chk(self.lib.pf_batch_get_fields(self.h, b, FIELD[name], a.ctypes.data_as(C.c_void_p), cnt * eb, 0))
        return a

    def step(self, n=1):
        self._chk(self.lib.pf_batch_step(self.h, int(n)))

    def tangent(self, b, nsteps, param=PF_PARAM_WI, objective=PF_OBJ_WETTED, flags=0, direction=None):
        """Solver.tangent for problem b of the batch (not advanced)."""
        out = (C.c_double * 2)()
        ptr = None
        if direction is not None:
            direction = np.ascontiguousarray(direction, dtype=np.float64).ravel()
            ptr = direction.ctypes.data_as(C.c_void_p)
        self._chk(self.lib.pf_batch_tangent(self.h, int(b), int(nsteps), int(param), int(objective), int(flags),
                                            ptr, 0, out))
        return out[0], out[1]

    def adjoint(self, b, nsteps, ckpt_every=50, objective=PF_OBJ_WETTED, want_phi=True):
        """Solver.adjoint for problem b of the batch; leaves that problem at phi^N."""
        out = (C.c_double * 3)()
        g = None
        ptr = None
        if want_phi:
            cnt, _ = self.info(b, "phi")
            g = np.empty(cnt, dtype=self.dtype)
            ptr = g.ctypes.data_as(C.c_void_p)
        self._chk(self.lib.pf_batch_adjoint(self.h, int(b), int(nsteps), int(ckpt_every), int(objective), out, ptr, 0))
        if g is not None:
            g = g.reshape(self.grids[b].fine_shape)
        return out[0], out[1], out[2], g

    def adjoint_coupled(self, b, nsteps, ckpt_every=50, objective=PF_OBJ_WETTED, want_phi=True):
        """Solver.adjoint_coupled for problem b of the batch; leaves it at step N."""
        out = (C.c_double * 4)()
        g = None
        ptr = None
        if want_phi:
            cnt, _ = self.info(b, "phi")
            g = np.empty(cnt, dtype=self.dtype)
            ptr = g.ctypes.data_as(C.c_void_p)
        self._chk(self.lib.pf_batch_adjoint_ex(self.h, int(b), int(nsteps), int(ckpt_every), int(objective),
                                               PF_ADJ_COUPLED, out, ptr, 0))
        if g is not None:
            g = g.reshape(self.grids[b].fine_shape)
        return out[0], out[1], out[2], out[3], g

    def diagnostics(self, b):
        out = (C.c_double * 6)()
        self._chk(self.lib.pf_batch_diagnostics(self.h, b, out))
        return dict(mass=out[0], energy=out[1], wetted=out[2], centroid=(out[3], out[4], out[5]))

    def close(self):
        if getattr(self, "h", None):
            self.lib.pf_batch_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
