"""Python binding of libsfrd.so, the sm_103a compact-MTT ETDRK4-P13 solver.

Argument marshalling only: every step of the solver runs in the library's CUDA
kernels.  PyTorch supplies device memory (the workspace and the fields) and the
CUDA stream; nothing here computes any part of the method.  If the shared
library has not been built this module raises ImportError instead of falling
back to anything else.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libsfrd.so")

if not os.path.exists(LIB_PATH):
    raise ImportError("libsfrd.so is not built: run `python -c 'import __graft_entry__ as g; g.build()'` "
                      "(nvcc for sm_103a) before importing paper_2003_13569_gb300")

_lib = ctypes.CDLL(LIB_PATH)

SFRD_OK = 0
ERRORS = {-1: "EINVAL", -2: "EUNSUPPORTED", -3: "ENOWS", -4: "ECUDA", -5: "ENONFINITE", -6: "ESTATE"}
BC = {"periodic": 0, "dirichlet": 1, "neumann": 2}
DTYPE = {"f64": 0, "f32": 1}
REACTION = {"none": 0, "linear": 1, "fhn": 2, "gray_scott": 3, "schnakenberg": 4,
            "gierer_meinhardt": 5, "huxley_mms": 6, "fisher_mms": 7}
COEFFICIENTS = ("R13", "Q13", "phi", "phi1", "phi2", "phi3")
COEF_MODE = {"stored": 0, "rational": 1}
SCHEME = {"p13": 0, "cox_matthews": 1}
EXPORTS = ("sfrd_plan", "sfrd_set_coefficients", "sfrd_set_scheme", "sfrd_check_finite", "sfrd_autotune", "sfrd_batch_autotune", "sfrd_workspace_bytes", "sfrd_get_info", "sfrd_bind", "sfrd_load", "sfrd_advance",
           "sfrd_store", "sfrd_run", "sfrd_step", "sfrd_run_host", "sfrd_forward", "sfrd_forward_noalloc", "sfrd_inverse",
           "sfrd_coefficients", "sfrd_profile_step", "sfrd_adjoint_workspace_bytes", "sfrd_run_checkpointed",
           "sfrd_adjoint", "sfrd_batch_plan", "sfrd_batch_workspace_bytes", "sfrd_batch_bind", "sfrd_batch_load",
           "sfrd_batch_advance", "sfrd_batch_store", "sfrd_batch_info", "sfrd_batch_destroy", "sfrd_destroy",
           "sfrd_strerror", "sfrd_last_error")


class Grid(ctypes.Structure):
    _fields_ = [("dim", ctypes.c_int32), ("N", ctypes.c_int64 * 3), ("lo", ctypes.c_double * 3),
                ("hi", ctypes.c_double * 3)]


class Reaction(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int32), ("nspecies", ctypes.c_int32), ("p", ctypes.c_double * 8),
                ("offset", ctypes.c_double * 2)]


class Info(ctypes.Structure):
    _fields_ = [("dim", ctypes.c_int32), ("bc", ctypes.c_int32), ("dtype", ctypes.c_int32),
                ("nspecies", ctypes.c_int32), ("n", ctypes.c_int64 * 3), ("fft_len", ctypes.c_int64 * 3),
                ("dof", ctypes.c_int64), ("kernels_per_step", ctypes.c_int64),
                ("workspace_bytes", ctypes.c_size_t)]


_P = ctypes.c_void_p
_D = ctypes.c_double
_lib.sfrd_plan.argtypes = [ctypes.POINTER(_P), ctypes.POINTER(Grid), ctypes.c_int32, ctypes.POINTER(_D),
                           ctypes.POINTER(_D), _D, ctypes.c_int32, ctypes.POINTER(Reaction)]
_lib.sfrd_set_coefficients.argtypes = [_P, ctypes.c_int32]
_lib.sfrd_set_scheme.argtypes = [_P, ctypes.c_int32]
_lib.sfrd_check_finite.argtypes = [_P]
_lib.sfrd_autotune.argtypes = [_P, ctypes.c_int32, ctypes.POINTER(ctypes.c_int32)]
_lib.sfrd_batch_autotune.argtypes = [_P, ctypes.c_int32, ctypes.POINTER(ctypes.c_int32)]
_lib.sfrd_workspace_bytes.argtypes = [_P, ctypes.POINTER(ctypes.c_size_t)]
_lib.sfrd_get_info.argtypes = [_P, ctypes.POINTER(Info)]
_lib.sfrd_bind.argtypes = [_P, _P, ctypes.c_size_t, _P]
_lib.sfrd_load.argtypes = [_P, _P, _D]
_lib.sfrd_advance.argtypes = [_P, ctypes.c_int64]
_lib.sfrd_store.argtypes = [_P, _P]
_lib.sfrd_run.argtypes = [_P, _P, _D, ctypes.c_int64]
_lib.sfrd_step.argtypes = [_P, _P, _D]
_lib.sfrd_run_host.argtypes = [_P, _P, _P, _D, ctypes.c_int64]
_lib.sfrd_forward.argtypes = [_P, _P, _P]
_lib.sfrd_inverse.argtypes = [_P, _P, _P]
_lib.sfrd_forward_noalloc.argtypes = [_P, _P, _P, _P]
_lib.sfrd_coefficients.argtypes = [_P, ctypes.c_int32, _P]
_lib.sfrd_profile_step.argtypes = [_P, ctypes.c_int32, ctypes.POINTER(ctypes.c_float),
                                   ctypes.POINTER(ctypes.c_int32)]
_lib.sfrd_adjoint_workspace_bytes.argtypes = [_P, ctypes.c_int64, ctypes.c_int64, ctypes.POINTER(ctypes.c_size_t)]
_lib.sfrd_run_checkpointed.argtypes = [_P, _P, _D, ctypes.c_int64, ctypes.c_int64, _P, ctypes.c_size_t]
_lib.sfrd_adjoint.argtypes = [_P, _D, ctypes.c_int64, ctypes.c_int64, _P, ctypes.c_size_t, _P, _P,
                              ctypes.POINTER(_D), ctypes.POINTER(_D), ctypes.POINTER(_D)]
_lib.sfrd_destroy.argtypes = [_P]
_lib.sfrd_destroy.restype = None
_lib.sfrd_strerror.argtypes = [ctypes.c_int]
_lib.sfrd_strerror.restype = ctypes.c_char_p
_lib.sfrd_last_error.argtypes = []
_lib.sfrd_last_error.restype = ctypes.c_char_p
_lib.sfrd_batch_plan.argtypes = [ctypes.POINTER(_P), ctypes.c_int64, ctypes.POINTER(Grid), ctypes.POINTER(ctypes.c_int32),
                                 ctypes.POINTER(_D), ctypes.POINTER(_D), _D, ctypes.c_int32, ctypes.POINTER(Reaction)]
_lib.sfrd_batch_workspace_bytes.argtypes = [_P, ctypes.POINTER(ctypes.c_size_t)]
_lib.sfrd_batch_bind.argtypes = [_P, _P, ctypes.c_size_t, _P]
_lib.sfrd_batch_load.argtypes = [_P, ctypes.POINTER(_P), _D]
_lib.sfrd_batch_advance.argtypes = [_P, ctypes.c_int64]
_lib.sfrd_batch_store.argtypes = [_P, ctypes.POINTER(_P)]
_lib.sfrd_batch_info.argtypes = [_P, ctypes.POINTER(ctypes.c_int64), ctypes.POINTER(ctypes.c_int64),
                                 ctypes.POINTER(ctypes.c_int64)]
_lib.sfrd_batch_destroy.argtypes = [_P]
_lib.sfrd_batch_destroy.restype = None
for _name in EXPORTS:
    if _name not in ("sfrd_destroy", "sfrd_batch_destroy", "sfrd_strerror", "sfrd_last_error"):
        getattr(_lib, _name).restype = ctypes.c_int


class SfrdError(RuntimeError):
    def __init__(self, code, where):
        msg = "%s: %s (%s)" % (where, ERRORS.get(code, code), _lib.sfrd_strerror(code).decode())
        if code == -4:
            msg += ": " + _lib.sfrd_last_error().decode()
        super().__init__(msg)
        self.code = code


def _check(code, where):
    if code != SFRD_OK:
        raise SfrdError(code, where)


def lib():
    """The loaded ctypes library (for tests of the raw C ABI)."""
    return _lib


def _ptr(t):
    return ctypes.c_void_p(t.data_ptr())


def make_plan(dim, N, lo, hi, bc, alpha, kappa, dt, dtype, reaction, params=(), offset=(0.0, 0.0),
              nspecies=None):
    """Create a raw plan handle (ctypes c_void_p); raises SfrdError on a negative code."""
    g = Grid()
    g.dim = dim
    for d in range(3):
        g.N[d] = int(N[d]) if d < dim else 1
        g.lo[d] = float(lo[d]) if d < dim else 0.0
        g.hi[d] = float(hi[d]) if d < dim else 1.0
    r = Reaction()
    r.kind = REACTION[reaction] if isinstance(reaction, str) else int(reaction)
    S = nspecies if nspecies is not None else len(alpha)
    r.nspecies = S
    for i, v in enumerate(params):
        r.p[i] = float(v)
    r.offset[0], r.offset[1] = float(offset[0]), float(offset[1])
    a = (ctypes.c_double * 2)(*[float(x) for x in alpha], *([0.0] * (2 - len(alpha))))
    k = (ctypes.c_double * 2)(*[float(x) for x in kappa], *([0.0] * (2 - len(kappa))))
    h = ctypes.c_void_p()
    bcv = BC[bc] if isinstance(bc, str) else int(bc)
    dtv = DTYPE[dtype] if isinstance(dtype, str) else int(dtype)
    _check(_lib.sfrd_plan(ctypes.byref(h), ctypes.byref(g), bcv, a, k, float(dt), dtv, ctypes.byref(r)),
           "sfrd_plan")
    return h


class Solver:
    """One plan bound to a torch-allocated workspace on the current CUDA device and stream."""

    def __init__(self, cfg: dict, dtype: str | None = None, device=None, coefficients: str = "stored",
                 scheme: str | None = None):
        """coefficients: "stored" (FP64-computed coefficient arrays) or "rational" (L stored, the
        Padé(1,3) rationals evaluated in FP32 by the passes; FP32 plans on power-of-two grids).
        scheme: "p13" (the paper's ETDRK4-P13, default) or "cox_matthews" (exact exponentials);
        defaults to cfg.get("scheme", "p13")."""
        import torch
        self.torch = torch
        self.cfg = cfg
        self.dtype = dtype or cfg["dtype"]
        self.tdtype = torch.float32 if self.dtype == "f32" else torch.float64
        r = cfg["reaction"]
        self.S = len(cfg["alpha"])
        self.handle = make_plan(cfg["dim"], cfg["N"], cfg["lo"], cfg["hi"], cfg["bc"], cfg["alpha"],
                                cfg["kappa"], cfg["dt"], self.dtype, r["kind"], r.get("p", ()),
                                r.get("offset", (0.0, 0.0)), nspecies=self.S)
        self.scheme = scheme or cfg.get("scheme", "p13")
        if self.scheme != "p13":
            _check(_lib.sfrd_set_scheme(self.handle, SCHEME[self.scheme]), "sfrd_set_scheme")
        if coefficients != "stored":
            _check(_lib.sfrd_set_coefficients(self.handle, COEF_MODE[coefficients]), "sfrd_set_coefficients")
        self.coef_mode = coefficients
        info = Info()
        _check(_lib.sfrd_get_info(self.handle, ctypes.byref(info)), "sfrd_get_info")
        self.info = info
        self.shape = tuple([self.S] + [int(info.n[d]) for d in reversed(range(cfg["dim"]))])
        self.device = torch.device("cuda") if device is None else torch.device(device)
        self.ws = torch.empty(int(info.workspace_bytes) + 256, dtype=torch.uint8, device=self.device)
        base = self.ws.data_ptr()
        self._ws_ptr = (base + 255) // 256 * 256
        self.stream = torch.cuda.current_stream(self.device)
        _check(_lib.sfrd_bind(self.handle, ctypes.c_void_p(self._ws_ptr), int(info.workspace_bytes),
                              ctypes.c_void_p(self.stream.cuda_stream)), "sfrd_bind")

    # -- helpers -------------------------------------------------------------
    def _field(self, u):
        t = self.torch
        if isinstance(u, np.ndarray) or isinstance(u, (list, tuple)):
            u = t.as_tensor(np.stack([np.asarray(x) for x in u]) if isinstance(u, (list, tuple)) else u)
        u = u.to(device=self.device, dtype=self.tdtype).contiguous()
        if tuple(u.shape) != self.shape:
            raise ValueError("field shape %s, expected %s" % (tuple(u.shape), self.shape))
        return u

    def empty(self):
        return self.torch.empty(self.shape, dtype=self.tdtype, device=self.device)

    @property
    def dof(self):
        return int(self.info.dof)

    @property
    def kernels_per_step(self):
        return int(self.info.kernels_per_step)

    # -- the C ABI -----------------------------------------------------------
    def load(self, u0, t0=0.0):
        u0 = self._field(u0)
        self._keep = u0
        _check(_lib.sfrd_load(self.handle, _ptr(u0), float(t0)), "sfrd_load")

    def advance(self, nsteps):
        _check(_lib.sfrd_advance(self.handle, int(nsteps)), "sfrd_advance")

    def store(self, out=None):
        out = self.empty() if out is None else out
        _check(_lib.sfrd_store(self.handle, _ptr(out)), "sfrd_store")
        return out

    def run(self, u, t0=0.0, nsteps=1):
        """Returns u(t0 + nsteps dt) as a new device tensor (the input is not modified)."""
        w = self._field(u).clone()
        _check(_lib.sfrd_run(self.handle, _ptr(w), float(t0), int(nsteps)), "sfrd_run")
        return w

    def step(self, u, t=0.0):
        w = self._field(u).clone()
        _check(_lib.sfrd_step(self.handle, _ptr(w), float(t)), "sfrd_step")
        return w

    def run_host(self, u_in: np.ndarray, t0=0.0, nsteps=1, out: np.ndarray | None = None):
        """End-to-end through host memory (numpy arrays, ideally pinned); synchronises."""
        npdt = np.float32 if self.dtype == "f32" else np.float64
        if u_in.dtype != npdt or not u_in.flags.c_contiguous or tuple(u_in.shape) != self.shape:
            raise ValueError("u_in must be a C-contiguous %s array of shape %s" % (npdt.__name__, self.shape))
        out = np.empty_like(u_in) if out is None else out
        _check(_lib.sfrd_run_host(self.handle, ctypes.c_void_p(u_in.ctypes.data), ctypes.c_void_p(out.ctypes.data),
                                  float(t0), int(nsteps)), "sfrd_run_host")
        return out

    def run_host_ptr(self, src_ptr: int, dst_ptr: int, t0=0.0, nsteps=1):
        _check(_lib.sfrd_run_host(self.handle, ctypes.c_void_p(src_ptr), ctypes.c_void_p(dst_ptr), float(t0),
                                  int(nsteps)), "sfrd_run_host")

    def forward(self, u):
        u = self._field(u)
        out = self.empty()
        _check(_lib.sfrd_forward(self.handle, _ptr(u), _ptr(out)), "sfrd_forward")
        return out

    def inverse(self, uhat):
        uhat = self._field(uhat)
        out = self.empty()
        _check(_lib.sfrd_inverse(self.handle, _ptr(uhat), _ptr(out)), "sfrd_inverse")
        return out

    def check_finite(self):
        """True when the resident state holds only finite values (False: SFRD_ENONFINITE)."""
        code = _lib.sfrd_check_finite(self.handle)
        if code == -5:
            return False
        _check(code, "sfrd_check_finite")
        return True

    def autotune(self, steps=3):
        """Pick the fastest radix/tile schedule of the shared-memory engine's axes (the resident state
        is lost: load afterwards).  Returns (tile width, radix-order rule)."""
        ch = (ctypes.c_int32 * 2)()
        _check(_lib.sfrd_autotune(self.handle, int(steps), ch), "sfrd_autotune")
        return int(ch[0]), int(ch[1])

    def coefficients(self, which):
        w = COEFFICIENTS.index(which) if isinstance(which, str) else int(which)
        out = self.empty()
        _check(_lib.sfrd_coefficients(self.handle, w, _ptr(out)), "sfrd_coefficients")
        return out

    def profile_step(self):
        """[(kind, ms)] for each kernel of one step (advances the resident state by one step)."""
        n = self.kernels_per_step
        ms = (ctypes.c_float * n)()
        kd = (ctypes.c_int32 * n)()
        _check(_lib.sfrd_profile_step(self.handle, n, ms, kd), "sfrd_profile_step")
        return [(int(kd[i]), float(ms[i])) for i in range(n)]

    # -- discrete adjoint ----------------------------------------------------
    def _adj_ws(self, nsteps, K):
        nb = ctypes.c_size_t()
        _check(_lib.sfrd_adjoint_workspace_bytes(self.handle, int(nsteps), int(K), ctypes.byref(nb)),
               "sfrd_adjoint_workspace_bytes")
        key = (int(nsteps), int(K))
        if getattr(self, "_adj_key", None) != key:
            self._adj_buf = self.torch.empty(int(nb.value) + 256, dtype=self.torch.uint8, device=self.device)
            self._adj_key = key
        base = self._adj_buf.data_ptr()
        return (base + 255) // 256 * 256, int(nb.value)

    def run_checkpointed(self, u0, t0=0.0, nsteps=1, ckpt_every=50):
        """u(t0 + nsteps dt), keeping the checkpoints that adjoint() needs."""
        w = self._field(u0).clone()
        ptr, nb = self._adj_ws(nsteps, ckpt_every)
        _check(_lib.sfrd_run_checkpointed(self.handle, _ptr(w), float(t0), int(nsteps), int(ckpt_every),
                                          ctypes.c_void_p(ptr), nb), "sfrd_run_checkpointed")
        return w

    def adjoint(self, dLduT, t0=0.0, nsteps=1, ckpt_every=50):
        """(dL/du0, dL/dalpha[S], dL/dkappa[S], dL/dparams[8]) after run_checkpointed(u0, t0, nsteps, ckpt_every)."""
        g = self._field(dLduT)
        out = self.empty()
        ptr, nb = self._adj_ws(nsteps, ckpt_every)
        da = (ctypes.c_double * 2)()
        dk = (ctypes.c_double * 2)()
        dp = (ctypes.c_double * 8)()
        _check(_lib.sfrd_adjoint(self.handle, float(t0), int(nsteps), int(ckpt_every), ctypes.c_void_p(ptr), nb,
                                 _ptr(g), _ptr(out), da, dk, dp), "sfrd_adjoint")
        return out, list(da)[:self.S], list(dk)[:self.S], list(dp)

    def close(self):
        if getattr(self, "handle", None):
            _lib.sfrd_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# ---- batched instances -----------------------------------------------------------

class Batch:
    """Many independent instances (same dim, species, reaction, dt, dtype; own grid, BC, alpha,
    kappa) stepped together, one persistent launch per pass and axis-length group."""

    def __init__(self, cfgs: list, dtype: str | None = None, device=None):
        import torch
        self.torch = torch
        self.cfgs = cfgs
        self.dtype = dtype or cfgs[0]["dtype"]
        self.tdtype = torch.float32 if self.dtype == "f32" else torch.float64
        n = len(cfgs)
        S = len(cfgs[0]["alpha"])
        self.S = S
        grids = (Grid * n)()
        bcs = (ctypes.c_int32 * n)()
        al = (ctypes.c_double * (n * S))()
        ka = (ctypes.c_double * (n * S))()
        self.shapes = []
        for i, c in enumerate(cfgs):
            g = grids[i]
            g.dim = c["dim"]
            for d in range(3):
                g.N[d] = int(c["N"][d]) if d < c["dim"] else 1
                g.lo[d] = float(c["lo"][d]) if d < c["dim"] else 0.0
                g.hi[d] = float(c["hi"][d]) if d < c["dim"] else 1.0
            bcs[i] = BC[c["bc"]]
            for s in range(S):
                al[i * S + s] = float(c["alpha"][s])
                ka[i * S + s] = float(c["kappa"][s])
            unk = {"periodic": 0, "dirichlet": -1, "neumann": 1}[c["bc"]]
            self.shapes.append(tuple([S] + [int(c["N"][d]) + unk for d in reversed(range(c["dim"]))]))
        r0 = cfgs[0]["reaction"]
        r = Reaction()
        r.kind = REACTION[r0["kind"]]
        r.nspecies = S
        for i, v in enumerate(r0.get("p", [])):
            r.p[i] = float(v)
        off = r0.get("offset", (0.0, 0.0))
        r.offset[0], r.offset[1] = float(off[0]), float(off[1])
        h = ctypes.c_void_p()
        _check(_lib.sfrd_batch_plan(ctypes.byref(h), n, grids, bcs, al, ka, float(cfgs[0]["dt"]),
                                    DTYPE[self.dtype], ctypes.byref(r)), "sfrd_batch_plan")
        self.handle = h
        nb = ctypes.c_size_t()
        _check(_lib.sfrd_batch_workspace_bytes(h, ctypes.byref(nb)), "sfrd_batch_workspace_bytes")
        self.device = torch.device("cuda") if device is None else torch.device(device)
        self.ws = torch.empty(int(nb.value) + 256, dtype=torch.uint8, device=self.device)
        ptr = (self.ws.data_ptr() + 255) // 256 * 256
        self.stream = torch.cuda.current_stream(self.device)
        _check(_lib.sfrd_batch_bind(h, ctypes.c_void_p(ptr), int(nb.value), ctypes.c_void_p(self.stream.cuda_stream)),
               "sfrd_batch_bind")
        cnt, dof, lps = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int64()
        _check(_lib.sfrd_batch_info(h, ctypes.byref(cnt), ctypes.byref(dof), ctypes.byref(lps)), "sfrd_batch_info")
        self.count, self.dof, self.launches_per_step = cnt.value, dof.value, lps.value

    def _ptrs(self, fields):
        arr = (_P * self.count)()
        for i, f in enumerate(fields):
            arr[i] = f.data_ptr()
        return arr

    def autotune(self, steps=2):
        """Pick the fastest blocks-per-SM of the persistent launches and radix order of the instances
        on the shared-memory engine (instances must be loaded afterwards).  Returns (blocks per SM, rule)."""
        ch = (ctypes.c_int32 * 2)()
        _check(_lib.sfrd_batch_autotune(self.handle, int(steps), ch), "sfrd_batch_autotune")
        return int(ch[0]), int(ch[1])

    def load(self, fields, t0=0.0):
        t = self.torch
        self._keep = [t.as_tensor(np.asarray(f) if not isinstance(f, t.Tensor) else f).to(
            device=self.device, dtype=self.tdtype).contiguous() for f in fields]
        for f, shp in zip(self._keep, self.shapes):
            if tuple(f.shape) != shp:
                raise ValueError("field shape %s, expected %s" % (tuple(f.shape), shp))
        _check(_lib.sfrd_batch_load(self.handle, self._ptrs(self._keep), float(t0)), "sfrd_batch_load")

    def advance(self, nsteps):
        _check(_lib.sfrd_batch_advance(self.handle, int(nsteps)), "sfrd_batch_advance")

    def store(self):
        outs = [self.torch.empty(shp, dtype=self.tdtype, device=self.device) for shp in self.shapes]
        _check(_lib.sfrd_batch_store(self.handle, self._ptrs(outs)), "sfrd_batch_store")
        return outs

    def close(self):
        if getattr(self, "handle", None):
            _lib.sfrd_batch_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# ---- autograd ----------------------------------------------------------------------

def _with_params(cfg, alpha, kappa, params):
    c = dict(cfg)
    c["alpha"] = tuple(float(x) for x in alpha)
    c["kappa"] = tuple(float(x) for x in kappa)
    r = dict(cfg["reaction"])
    p = list(r.get("p", []))
    for i, v in enumerate(params):
        p[i] = float(v)
    r["p"] = p
    c["reaction"] = r
    return c


def _make_function():
    import torch

    class SfrdRun(torch.autograd.Function):
        """u_T = ETDRK4-P13^nsteps(u0; alpha, kappa, reaction params), differentiated by the
        library's discrete adjoint with checkpoints every ckpt_every steps."""

        @staticmethod
        def forward(ctx, u0, alpha, kappa, params, cfg, dtype, nsteps, ckpt_every, t0):
            c = _with_params(cfg, alpha.detach().cpu().tolist(), kappa.detach().cpu().tolist(),
                             params.detach().cpu().tolist())
            s = Solver(c, dtype=dtype, device=u0.device)
            uT = s.run_checkpointed(u0.detach(), t0=t0, nsteps=nsteps, ckpt_every=ckpt_every)
            ctx.solver, ctx.meta = s, (t0, nsteps, ckpt_every, len(params))
            return uT.to(u0.dtype)

        @staticmethod
        def backward(ctx, g):
            t0, nsteps, K, npar = ctx.meta
            du0, da, dk, dp = ctx.solver.adjoint(g.contiguous(), t0=t0, nsteps=nsteps, ckpt_every=K)
            f64 = torch.float64
            return (du0.to(g.dtype), torch.tensor(da, dtype=f64), torch.tensor(dk, dtype=f64),
                    torch.tensor(dp[:npar], dtype=f64), None, None, None, None, None)

    return SfrdRun


_SFRD_RUN = None


def run(u0, alpha, kappa, params, cfg, nsteps, ckpt_every=50, dtype=None, t0=0.0):
    """Differentiable run: u0 [S][...] device tensor; alpha, kappa [S] and params (the reaction
    parameter vector, in the order documented in sfrd.h) as float64 CPU tensors."""
    global _SFRD_RUN
    if _SFRD_RUN is None:
        _SFRD_RUN = _make_function()
    return _SFRD_RUN.apply(u0, alpha, kappa, params, cfg, dtype or cfg["dtype"], int(nsteps), int(ckpt_every),
                           float(t0))
