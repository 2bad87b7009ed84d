"""Thin Python binding of librism3d (include/rism3d.h).

Argument marshalling only: every value of the initialization grids is
computed by the CUDA kernels behind the C ABI.  PyTorch provides the device
memory of the outputs and the current CUDA stream.  If the compiled library
is missing, the first call raises: there is no CPU fallback.
"""
from __future__ import annotations

import ctypes as C
import os
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "lib", "librism3d.so")

OK, E_INVALID, E_STATE, E_NOMEM, E_CUDA, E_TIMEOUT, E_UNSUPPORTED = range(7)
METHOD_DIRECT, METHOD_TREECODE = 0, 1
PREC_FP64, PREC_FP32 = 0, 1
LJ_NONE, LJ_RCUT, LJ_TOL = 0, 1, 2
APPROX_BARYCENTRIC, APPROX_TAYLOR = 0, 1
MAX_SITES = 8

_STATUS = {0: "RISM_OK", 1: "RISM_E_INVALID", 2: "RISM_E_STATE", 3: "RISM_E_NOMEM", 4: "RISM_E_CUDA",
           5: "RISM_E_TIMEOUT", 6: "RISM_E_UNSUPPORTED"}


class RismError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{_STATUS.get(status, status)}: {msg}")
        self.status = status


class GridDesc(C.Structure):
    _fields_ = [("nx", C.c_int32), ("ny", C.c_int32), ("nz", C.c_int32), ("h", C.c_double),
                ("origin", C.c_double * 3)]


class Options(C.Structure):
    _fields_ = [("method", C.c_int32), ("precision", C.c_int32), ("degree", C.c_int32), ("theta", C.c_double),
                ("leaf", C.c_int32), ("batch", C.c_int32 * 3), ("lj_mode", C.c_int32), ("lj_rcut", C.c_double),
                ("lj_tol", C.c_double), ("eta", C.c_double), ("T", C.c_double), ("eps_r", C.c_double),
                ("kappa", C.c_double), ("k_e", C.c_double), ("k_B", C.c_double), ("r_short", C.c_double),
                ("autotune", C.c_int32), ("wait_limit", C.c_int64),
                ("debug_flags", C.c_int32), ("target_proxies", C.c_int32), ("approx", C.c_int32)]


class Info(C.Structure):
    _fields_ = [("beta", C.c_double), ("kappa", C.c_double), ("r_short", C.c_double), ("natoms", C.c_int64),
                ("nsite", C.c_int32), ("tree_nodes", C.c_int32), ("tree_proxied", C.c_int32),
                ("tree_leaves", C.c_int32), ("direct_pairs", C.c_int64), ("proxy_pairs", C.c_int64),
                ("near_pairs", C.c_int64), ("batch", C.c_int32 * 3), ("kernel_variant", C.c_int32),
                ("launches", C.c_int32), ("eval_ms", C.c_float), ("far_ms", C.c_float), ("near_ms", C.c_float),
                ("box_ms", C.c_float), ("tree_boxes", C.c_int32), ("cp_pairs", C.c_int64),
                ("near_tested", C.c_int64), ("lj_pairs", C.c_int64), ("sr_pairs", C.c_int64)]


class Guide(C.Structure):
    _fields_ = [("p_tcf", C.c_int32), ("p_dcf", C.c_int32), ("p_coulomb", C.c_int32), ("mac", C.c_double),
                ("n0", C.c_int32), ("k_tol", C.c_double), ("lj_tol", C.c_double)]


EXPORTS = ["rism_default_options", "rism_grid_create", "rism_set_solute", "rism_set_solvent", "rism_potential",
           "rism_asymptotics", "rism_init", "rism_potential_backward", "rism_potential_batched", "rism_get_info",
           "rism_destroy", "rism_last_error", "rism_init_noalloc", "rism_lra_integral",
           "rism_asymptotics_k", "rism_parameter_guide"]
NOALLOC_MAX_ATOMS = 8192

_lib = None
_lock = threading.Lock()


def load(path: str = LIB_PATH):
    """Load librism3d.so (raises if it has not been built)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        if not os.path.exists(path):
            raise RuntimeError(f"librism3d.so is not built ({path}); run __graft_entry__.build()")
        lib = C.CDLL(path)
        P, I32, I64 = C.c_void_p, C.c_int32, C.c_int64
        lib.rism_default_options.restype = None
        lib.rism_default_options.argtypes = [C.POINTER(Options)]
        lib.rism_grid_create.restype = C.c_int
        lib.rism_grid_create.argtypes = [C.POINTER(GridDesc), C.POINTER(Options), P, C.POINTER(P)]
        lib.rism_set_solute.restype = C.c_int
        lib.rism_set_solute.argtypes = [P, I64, P, P, P, P]
        lib.rism_set_solvent.restype = C.c_int
        lib.rism_set_solvent.argtypes = [P, I32, P, P, P, P, P]
        lib.rism_potential.restype = C.c_int
        lib.rism_potential.argtypes = [P, P, P]
        lib.rism_asymptotics.restype = C.c_int
        lib.rism_asymptotics.argtypes = [P, P, P]
        lib.rism_init.restype = C.c_int
        lib.rism_init.argtypes = [P, P, P, P, P]
        lib.rism_potential_backward.restype = C.c_int
        lib.rism_potential_backward.argtypes = [P, P, P, P, P, P, P, P]
        lib.rism_potential_batched.restype = C.c_int
        lib.rism_potential_batched.argtypes = [P, I32, P, P, P]
        lib.rism_get_info.restype = C.c_int
        lib.rism_get_info.argtypes = [P, C.POINTER(Info)]
        lib.rism_destroy.restype = None
        lib.rism_destroy.argtypes = [P]
        lib.rism_last_error.restype = C.c_char_p
        lib.rism_last_error.argtypes = [P]
        lib.rism_asymptotics_k.restype = C.c_int
        lib.rism_asymptotics_k.argtypes = [P, C.c_double, P, P, P]
        lib.rism_lra_integral.restype = C.c_int
        lib.rism_lra_integral.argtypes = [P, P, P]
        lib.rism_init_noalloc.restype = C.c_int
        lib.rism_init_noalloc.argtypes = [C.POINTER(GridDesc), C.POINTER(Options), I64, P, P, P, P, I32, P, P, P, P,
                                          P, P, P, P, P, C.c_char_p, C.c_size_t]
        lib.rism_parameter_guide.restype = C.c_int
        lib.rism_parameter_guide.argtypes = [C.c_double, C.POINTER(Guide)]
        _lib = lib
        return lib


def default_options(**over) -> Options:
    o = Options()
    load().rism_default_options(C.byref(o))
    for k, v in over.items():
        if k == "batch":
            for i in range(3):
                o.batch[i] = int(v[i])
        else:
            setattr(o, k, v)
    return o


def _host_f64(a, n=None):
    a = np.ascontiguousarray(np.asarray(a, dtype=np.float64))
    if n is not None and a.size != n:
        raise ValueError("array size mismatch")
    return a


def _ptr(t):
    return None if t is None else C.c_void_p(t.data_ptr())


class Rism:
    """One grid context.  Outputs are torch tensors on the current CUDA device."""

    def __init__(self, n, h, origin, stream=None, **opts):
        import torch

        self._torch = torch
        self.lib = load()
        self.n = tuple(int(v) for v in n)
        self.h = float(h)
        self.origin = tuple(float(v) for v in origin)
        self.opts = default_options(**opts)
        g = GridDesc(self.n[0], self.n[1], self.n[2], self.h, (C.c_double * 3)(*self.origin))
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        self.device = self.stream.device
        ctx = C.c_void_p()
        st = self.lib.rism_grid_create(C.byref(g), C.byref(self.opts), C.c_void_p(self.stream.cuda_stream),
                                       C.byref(ctx))
        if st != OK:
            raise RismError(st, "rism_grid_create")
        self.ctx = ctx
        self.S = 0
        self.natoms = 0

    def _check(self, st, what):
        if st != OK:
            msg = self.lib.rism_last_error(self.ctx).decode(errors="replace")
            raise RismError(st, f"{what}: {msg}")

    def close(self):
        if getattr(self, "ctx", None):
            self.lib.rism_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def npts(self):
        return self.n[0] * self.n[1] * self.n[2]

    def set_solute(self, xyz, q, sigma, eps):
        q = _host_f64(q)
        n = q.size
        xyz, sigma, eps = _host_f64(xyz, 3 * n), _host_f64(sigma, n), _host_f64(eps, n)
        self._check(self.lib.rism_set_solute(self.ctx, n, xyz.ctypes.data, q.ctypes.data, sigma.ctypes.data,
                                             eps.ctypes.data), "rism_set_solute")
        self.natoms = n

    def set_solvent(self, q, sigma, eps, rho=None, is_ion=None):
        q = _host_f64(q)
        S = q.size
        sigma, eps = _host_f64(sigma, S), _host_f64(eps, S)
        rho_ = None if rho is None else _host_f64(rho, S)
        ion_ = None if is_ion is None else np.ascontiguousarray(np.asarray(is_ion, dtype=np.int32))
        self._check(self.lib.rism_set_solvent(self.ctx, S, q.ctypes.data, sigma.ctypes.data, eps.ctypes.data,
                                              None if rho_ is None else rho_.ctypes.data,
                                              None if ion_ is None else ion_.ctypes.data), "rism_set_solvent")
        self.S = S

    def empty_grid(self):
        nx, ny, nz = self.n
        return self._torch.empty((self.S, nz, ny, nx), dtype=self._torch.float64, device=self.device)

    def init(self, u=True, c=True, h=True, lj_tail=False, out=None):
        """Fused u / c / h (+ LJ tail integrals).  Returns a dict of tensors."""
        out = dict(out or {})
        for k, want in (("u", u), ("c", c), ("h", h)):
            if want and k not in out:
                out[k] = self.empty_grid()
        tail = np.zeros(max(self.S, 1)) if lj_tail else None
        st = self.lib.rism_init(self.ctx, _ptr(out.get("u")), _ptr(out.get("c")), _ptr(out.get("h")),
                                None if tail is None else tail.ctypes.data)
        self._check(st, "rism_init")
        if tail is not None:
            out["lj_tail"] = tail[: self.S].copy()
        return out

    def init_host(self, u=None, c=None, h=None, lj_tail=None):
        """Same call with HOST numpy outputs (the library stages and copies back)."""
        P = lambda a: None if a is None else a.ctypes.data
        self._check(self.lib.rism_init(self.ctx, P(u), P(c), P(h), P(lj_tail)), "rism_init")

    def potential(self, lj_tail=False):
        u = self.empty_grid()
        tail = np.zeros(max(self.S, 1)) if lj_tail else None
        self._check(self.lib.rism_potential(self.ctx, _ptr(u), None if tail is None else tail.ctypes.data),
                    "rism_potential")
        return (u, tail[: self.S].copy()) if lj_tail else u

    def asymptotics(self, c=True, h=True):
        cc = self.empty_grid() if c else None
        hh = self.empty_grid() if h else None
        self._check(self.lib.rism_asymptotics(self.ctx, _ptr(cc), _ptr(hh)), "rism_asymptotics")
        return cc, hh

    def backward(self, g_u=None, g_c=None, g_h=None, want=("xyz", "q", "sigma", "eps")):
        torch = self._torch
        n = self.natoms
        dev = self.device
        outs = {k: (torch.empty((n, 3) if k == "xyz" else (n,), dtype=torch.float64, device=dev)
                    if k in want else None) for k in ("xyz", "q", "sigma", "eps")}
        gs = [None if g is None else g.contiguous() for g in (g_u, g_c, g_h)]
        st = self.lib.rism_potential_backward(self.ctx, _ptr(gs[0]), _ptr(gs[1]), _ptr(gs[2]), _ptr(outs["xyz"]),
                                              _ptr(outs["q"]), _ptr(outs["sigma"]), _ptr(outs["eps"]))
        self._check(st, "rism_potential_backward")
        return {k: v for k, v in outs.items() if v is not None}

    def asymptotics_k(self, k_tol=0.0, c=True, h=True):
        """c_s(k), h_s(k) of eqs. (dcf-k)/(tcf-k) on the half spectrum (rism_asymptotics_k) as complex128
        device tensors [S, nz, ny, nx//2+1], and the cut-off wave number used (0 = none)."""
        torch = self._torch
        nx, ny, nz = self.n
        shape = (self.S, nz, ny, nx // 2 + 1)
        cc = torch.empty(shape, dtype=torch.complex128, device=self.device) if c else None
        hh = torch.empty(shape, dtype=torch.complex128, device=self.device) if h else None
        kc = C.c_double(0.0)
        self._check(self.lib.rism_asymptotics_k(self.ctx, float(k_tol), _ptr(cc), _ptr(hh), C.byref(kc)),
                    "rism_asymptotics_k")
        return cc, hh, kc.value

    def lra_integral(self, atom_sums=False):
        """The all-space long-range integral T_s (A^3) of every site (rism_lra_integral); with atom_sums also
        the per-atom overlap sums (P_hc, P_hh) as an [n, 2] device tensor."""
        T = np.zeros(max(self.S, 1))
        a = self._torch.empty((self.natoms, 2), dtype=self._torch.float64, device=self.device) if atom_sums else None
        self._check(self.lib.rism_lra_integral(self.ctx, T.ctypes.data, _ptr(a)), "rism_lra_integral")
        return (T[: self.S].copy(), a) if atom_sums else T[: self.S].copy()

    def info(self):
        inf = Info()
        self._check(self.lib.rism_get_info(self.ctx, C.byref(inf)), "rism_get_info")
        return {f: (list(getattr(inf, f)) if f == "batch" else getattr(inf, f)) for f, _ in Info._fields_}


def init_noalloc(grid_n, h, origin, xyz, q, sigma, eps, solvent, u=None, c=None, hh=None, stream=None, **opts):
    """rism_init_noalloc: direct-sum u / c / h into caller-provided device tensors, no device allocation by
    the library (for callers that cannot allocate device memory themselves).  xyz, q, sigma, eps: device (or
    host) float64 tensors; solvent: (q, sigma, eps, rho, is_ion) host arrays; u, c, hh: device tensors.
    Raises RismError with the library's message on failure."""
    import torch

    lib = load()
    o = default_options(**opts)
    g = GridDesc(int(grid_n[0]), int(grid_n[1]), int(grid_n[2]), float(h), (C.c_double * 3)(*origin))
    qs, sg, ep = (_host_f64(a) for a in solvent[:3])
    rho = None if solvent[3] is None else _host_f64(solvent[3])
    ion = None if solvent[4] is None else np.ascontiguousarray(np.asarray(solvent[4], dtype=np.int32))
    st = stream if stream is not None else torch.cuda.current_stream()
    buf = C.create_string_buffer(256)
    n = int(q.numel())
    rc = lib.rism_init_noalloc(C.byref(g), C.byref(o), n, _ptr(xyz), _ptr(q), _ptr(sigma), _ptr(eps), qs.size,
                               qs.ctypes.data, sg.ctypes.data, ep.ctypes.data,
                               None if rho is None else rho.ctypes.data, None if ion is None else ion.ctypes.data,
                               _ptr(u), _ptr(c), _ptr(hh), C.c_void_p(st.cuda_stream), buf, 256)
    if rc != OK:
        raise RismError(rc, "rism_init_noalloc: " + buf.value.decode(errors="replace"))


def parameter_guide(tolerance):
    """rism_parameter_guide: the paper's accuracy parameters for a residual tolerance of the 3D-RISM solution,
    as a dict: the Taylor orders p_tcf (h_lr), p_dcf (c_lr), p_coulomb (u), the acceptance parameter mac and
    the leaf size n0 (Table 3), the reciprocal-space cut-off tolerance k_tol (Sec. 4.3.1) and the LJ cut-off
    tolerance lj_tol (Sec. 4.4.1).  Raises RismError(E_INVALID) unless 0 < tolerance < 1.  Host arithmetic only
    (no GPU)."""
    lib = load()
    g = Guide()
    st = lib.rism_parameter_guide(float(tolerance), C.byref(g))
    if st != OK:
        raise RismError(st, f"rism_parameter_guide: tolerance {tolerance!r} is not in (0, 1)")
    return {k: getattr(g, k) for k, _ in Guide._fields_}


def potential_batched(rs, u=True, c=True, h=True, out=None):
    """One batched launch over several contexts; returns a list of dicts.  Passing the previous call's list as
    `out` reuses its tensors, which lets the library replay its captured launch sequence (the capture is keyed
    by the output addresses among others)."""
    lib = load()
    n = len(rs)
    if out is not None:
        outs = out
    else:
        outs = [{k: r.empty_grid() for k, w in (("u", u), ("c", c), ("h", h)) if w} for r in rs]
    arr = lambda k: (C.c_void_p * n)(*[o[k].data_ptr() if k in o else None for o in outs])
    ctxs = (C.c_void_p * n)(*[r.ctx.value for r in rs])
    st = lib.rism_potential_batched(ctxs, n, arr("u") if u else None, arr("c") if c else None,
                                    arr("h") if h else None)
    if st != OK:
        raise RismError(st, "rism_potential_batched: " + lib.rism_last_error(rs[0].ctx).decode(errors="replace"))
    return outs


def from_workload(w, **opts):
    """A context for a seeded workload: grid, solute, solvent and physical options set."""
    o = dict(w.opts)
    kw = {k: o[k] for k in ("eta", "T", "eps_r", "k_e", "k_B") if k in o}
    if "degree" in o:
        kw["degree"] = int(o["degree"])
    if "theta" in o:
        kw["theta"] = float(o["theta"])
    if o.get("lj_rcut", 0.0) > 0.0:
        kw["lj_mode"], kw["lj_rcut"] = LJ_RCUT, float(o["lj_rcut"])
    elif o.get("lj_tol", 0.0) > 0.0:
        kw["lj_mode"], kw["lj_tol"] = LJ_TOL, float(o["lj_tol"])
    else:
        kw["lj_mode"] = LJ_NONE
    kw.update(opts)
    r = Rism(w.grid.n, w.grid.h, w.grid.origin, **kw)
    r.set_solvent(w.solvent.q, w.solvent.sigma, w.solvent.eps, w.solvent.rho, w.solvent.is_ion)
    r.set_solute(w.solute.xyz, w.solute.q, w.solute.sigma, w.solute.eps)
    return r


class _Fields:
    """torch.autograd.Function whose forward is rism_init and whose backward is
    rism_potential_backward (created lazily so that importing this module
    does not need torch)."""

    fn = None

    @classmethod
    def get(cls):
        if cls.fn is None:
            import torch

            class RismFields(torch.autograd.Function):
                @staticmethod
                def forward(ctx, xyz, q, sigma, eps, rism):
                    rism.set_solute(xyz.detach().cpu().numpy(), q.detach().cpu().numpy(),
                                    sigma.detach().cpu().numpy(), eps.detach().cpu().numpy())
                    kap = rism.info()["kappa"]
                    out = rism.init(u=True, c=True, h=True) if kap > 0 else rism.init(u=True, c=True, h=False)
                    ctx.rism = rism
                    ctx.has_h = "h" in out
                    hh = out.get("h")
                    if hh is None:
                        hh = torch.zeros_like(out["u"])
                    return out["u"], out["c"], hh

                @staticmethod
                def backward(ctx, gu, gc, gh):
                    r = ctx.rism
                    g = r.backward(gu, gc, gh if ctx.has_h else None)
                    dev = r.device
                    return (g["xyz"].reshape(-1, 3).to("cpu"), g["q"].to("cpu"), g["sigma"].to("cpu"),
                            g["eps"].to("cpu"), None)

            cls.fn = RismFields
        return cls.fn


def fields(xyz, q, sigma, eps, rism):
    """(u, c, h) as differentiable functions of the solute parameters (CPU float64 tensors)."""
    return _Fields.get().apply(xyz, q, sigma, eps, rism)
