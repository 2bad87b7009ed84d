"""ctypes front end of the FP64 CPU oracle (rism_oracle.c).

TEST INFRASTRUCTURE ONLY: imported by the tests, by the package smoke check
and by the CPU-baseline leg of the benchmark; never by the product path.

The oracle takes plain arrays.  ``Problem.from_workload`` accepts any object
with ``solute``/``solvent``/``grid``/``opts`` attributes (the seeded workloads
of the input generator) without importing it.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "rism_oracle.c")
_LIBDIR = os.path.join(_HERE, "lib")
_LIB = os.path.join(_LIBDIR, "liboracle.so")
_lock = threading.Lock()
_lib = None

CFLAGS = ["-O2", "-fopenmp", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared", "-std=c11"]


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (plain C11 + OpenMP)."""
    os.makedirs(_LIBDIR, exist_ok=True)
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", *CFLAGS, "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = C.CDLL(build())
            D, I64, I32 = C.c_double, C.c_int64, C.c_int32
            P = C.c_void_p
            lib.orc_beta.restype = D
            lib.orc_beta.argtypes = [D, D]
            lib.orc_kappa.restype = D
            lib.orc_kappa.argtypes = [I32, P, P, P, D, D, D]
            lib.orc_lj_rcut_tol.restype = D
            lib.orc_lj_rcut_tol.argtypes = [D, D, D]
            lib.orc_lj_tail.restype = None
            lib.orc_lj_tail.argtypes = [I64, P, P, I32, P, P, P, P]
            lib.orc_kernels.restype = None
            lib.orc_kernels.argtypes = [D, D, I64, P, P, P, P, P]
            lib.orc_fields.restype = C.c_int
            lib.orc_fields.argtypes = [I64, P, P, P, P, I32, P, P, P, P, D, D, D, D, D,
                                       I32, I32, I32, D, P, I64, P, P, P, P, I32]
            lib.orc_grad.restype = C.c_int
            lib.orc_grad.argtypes = [I64, P, P, P, P, I32, P, P, P, P, D, D, D, D, D,
                                     I32, I32, I32, D, P, P, P, P, I64, P, P, I32]
            lib.orc_lra_pair.restype = None
            lib.orc_lra_pair.argtypes = [D, D, I64, P, P, P]
            lib.orc_lra_atom_sums.restype = C.c_int
            lib.orc_lra_atom_sums.argtypes = [I64, P, P, D, D, I64, P, P, P, I32]
            lib.orc_lra_integral.restype = C.c_int
            lib.orc_lra_integral.argtypes = [I64, P, P, I32, P, D, D, D, D, D, P, P, I32]
            lib.orc_kspace.restype = C.c_int
            lib.orc_kspace.argtypes = [I64, P, P, I32, P, D, D, D, D, D, I32, I32, I32, D, P, D, I64, P, P, P, I32]
            lib.orc_kspace_bound.restype = D
            lib.orc_kspace_bound.argtypes = [D, D, D, D, D, D]
            lib.orc_kspace_kcut.restype = D
            lib.orc_kspace_kcut.argtypes = [D, D, D, D, D, D]
            lib.orc_taylor_coeffs.restype = C.c_int
            lib.orc_taylor_coeffs.argtypes = [I32, I32, D, D, D, D, D, P]
            lib.orc_taylor_eval.restype = C.c_int
            lib.orc_taylor_eval.argtypes = [I32, I32, P, I64, P, P, D, D, I64, P, P]
            _lib = lib
    return _lib


def _p(a):
    return None if a is None else a.ctypes.data


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


@dataclass
class Problem:
    xyz: np.ndarray
    q: np.ndarray
    sigma: np.ndarray
    eps: np.ndarray
    qs: np.ndarray
    sigs: np.ndarray
    epss: np.ndarray
    rho: np.ndarray
    is_ion: np.ndarray
    n: tuple
    h: float
    origin: tuple
    eta: float = 1.0
    T: float = 298.0
    eps_r: float = 78.44
    k_e: float = 332.0522173
    k_B: float = 0.0019872041
    lj_rcut: float = 0.0  # > 0: one cut-off for every pair
    lj_tol: float = 0.0  # > 0 (and lj_rcut == 0): per-pair cut-off from this tolerance
    kappa: float = -1.0  # < 0: derive from the ionic sites

    @classmethod
    def from_workload(cls, w, **over):
        o = dict(w.opts)
        kw = dict(xyz=_f64(w.solute.xyz), q=_f64(w.solute.q), sigma=_f64(w.solute.sigma), eps=_f64(w.solute.eps),
                  qs=_f64(w.solvent.q), sigs=_f64(w.solvent.sigma), epss=_f64(w.solvent.eps),
                  rho=_f64(w.solvent.rho), is_ion=np.ascontiguousarray(w.solvent.is_ion, dtype=np.int32),
                  n=tuple(int(v) for v in w.grid.n), h=float(w.grid.h), origin=tuple(float(v) for v in w.grid.origin))
        for k in ("eta", "T", "eps_r", "k_e", "k_B", "lj_rcut", "lj_tol", "kappa"):
            if k in o:
                kw[k] = float(o[k])
        kw.update(over)
        return cls(**kw)

    @property
    def natoms(self):
        return int(self.q.shape[0])

    @property
    def nsite(self):
        return int(self.qs.shape[0])

    @property
    def npts(self):
        return int(self.n[0]) * int(self.n[1]) * int(self.n[2])


def beta(p: Problem) -> float:
    return _load().orc_beta(p.k_B, p.T)


def kappa(p: Problem) -> float:
    if p.kappa >= 0.0:
        return float(p.kappa)
    lib = _load()
    qs, rho, ion = _f64(p.qs), _f64(p.rho), np.ascontiguousarray(p.is_ion, dtype=np.int32)
    return lib.orc_kappa(p.nsite, _p(qs), _p(rho), _p(ion), beta(p), p.k_e, p.eps_r)


def rcut(p: Problem) -> np.ndarray:
    """[S, n] per-pair cut-offs (0 = no cut-off)."""
    S, n = p.nsite, p.natoms
    if p.lj_rcut > 0.0:
        return np.full((S, n), float(p.lj_rcut))
    if p.lj_tol > 0.0:
        lib = _load()
        out = np.empty((S, n))
        for s in range(S):
            for i in range(n):
                sg = 0.5 * (p.sigma[i] + p.sigs[s])
                ep = float(np.sqrt(p.eps[i] * p.epss[s]))
                out[s, i] = lib.orc_lj_rcut_tol(sg, ep, p.lj_tol)
        return out
    return np.zeros((S, n))


def lj_rcut_tol(sig_is, eps_is, tol):
    return _load().orc_lj_rcut_tol(float(sig_is), float(eps_is), float(tol))


def lj_tail(p: Problem) -> np.ndarray:
    lib = _load()
    rc = _f64(rcut(p))
    out = np.zeros(p.nsite)
    lib.orc_lj_tail(p.natoms, _p(p.sigma), _p(p.eps), p.nsite, _p(p.sigs), _p(p.epss), _p(rc), _p(out))
    return out


def kernels(eta, kappa_, d):
    """phi_c, phi_h (with the e^{a^2} prefactor), phi_c'/d and phi_h'/d at distances d."""
    lib = _load()
    d = _f64(np.atleast_1d(d))
    pc, ph, gc, gh = (np.empty_like(d) for _ in range(4))
    lib.orc_kernels(float(eta), float(kappa_), d.size, _p(d), _p(pc), _p(ph), _p(gc), _p(gh))
    return pc, ph, gc, gh


def fields(p: Problem, idx=None, want=("u", "c", "h"), nthreads: int = 0):
    """u, c, h as [S, npts] arrays (npts = len(idx) or the full grid).

    ``h`` is only computed when kappa > 0 (it is reported as zeros otherwise).
    """
    lib = _load()
    S = p.nsite
    if idx is not None:
        idx = np.ascontiguousarray(idx, dtype=np.int64)
        m = int(idx.size)
    else:
        m = p.npts
    out = {k: (np.empty((S, m)) if k in want else None) for k in ("u", "c", "h")}
    rc = _f64(rcut(p))
    org = _f64(p.origin)
    rc_ = lib.orc_fields(p.natoms, _p(_f64(p.xyz)), _p(p.q), _p(p.sigma), _p(p.eps), S, _p(p.qs), _p(p.sigs),
                         _p(p.epss), _p(rc), beta(p), p.k_e, p.eps_r, p.eta, kappa(p),
                         int(p.n[0]), int(p.n[1]), int(p.n[2]), p.h, _p(org), m, _p(idx),
                         _p(out["u"]), _p(out["c"]), _p(out["h"]), int(nthreads))
    if rc_ != 0:
        raise MemoryError("oracle allocation failed")
    return {k: v for k, v in out.items() if v is not None}


def grad(p: Problem, atoms, gu=None, gc=None, gh=None, nthreads: int = 0):
    """[len(atoms), 6]: dL/dx, dL/dy, dL/dz, dL/dq, dL/dsigma, dL/deps."""
    lib = _load()
    atoms = np.ascontiguousarray(atoms, dtype=np.int64)
    out = np.zeros((atoms.size, 8))
    rc = _f64(rcut(p))
    org = _f64(p.origin)
    g = [None if a is None else _f64(a).reshape(-1) for a in (gu, gc, gh)]
    rc_ = lib.orc_grad(p.natoms, _p(_f64(p.xyz)), _p(p.q), _p(p.sigma), _p(p.eps), p.nsite, _p(p.qs), _p(p.sigs),
                       _p(p.epss), _p(rc), beta(p), p.k_e, p.eps_r, p.eta, kappa(p),
                       int(p.n[0]), int(p.n[1]), int(p.n[2]), p.h, _p(org), _p(g[0]), _p(g[1]), _p(g[2]),
                       atoms.size, _p(atoms), _p(out), int(nthreads))
    if rc_ != 0:
        raise MemoryError("oracle allocation failed")
    return out[:, :6]


def lra_pair(eta, kappa_, R):
    """I_hc(R), I_hh(R): the all-space overlap integrals of the TCF kernel with the DCF kernel and with itself,
    for two unit charges R apart (1D quadrature over the wave number)."""
    lib = _load()
    R = _f64(np.atleast_1d(R))
    a, b = np.empty_like(R), np.empty_like(R)
    lib.orc_lra_pair(float(eta), float(kappa_), R.size, _p(R), _p(a), _p(b))
    return a, b


def lra_atom_sums(p: Problem, atoms, nthreads: int = 0):
    """[len(atoms), 2]: P_hc[a] = sum_b Q_b I_hc(R_ab), P_hh[a] = sum_b Q_b I_hh(R_ab) (b over every atom)."""
    lib = _load()
    atoms = np.ascontiguousarray(atoms, dtype=np.int64)
    phc, phh = np.empty(atoms.size), np.empty(atoms.size)
    lib.orc_lra_atom_sums(p.natoms, _p(_f64(p.xyz)), _p(_f64(p.q)), p.eta, kappa(p), atoms.size, _p(atoms),
                          _p(phc), _p(phh), int(nthreads))
    return np.stack([phc, phh], 1)


def lra_integral(p: Problem, nthreads: int = 0):
    """(T [S], (S_hh, S_hc)): the all-space integral of eq. (excess-chemical-potential-LRA) per site (A^3) and
    the two atom-pair sums it is assembled from."""
    lib = _load()
    T = np.empty(p.nsite)
    S2 = np.empty(2)
    rc = lib.orc_lra_integral(p.natoms, _p(_f64(p.xyz)), _p(_f64(p.q)), p.nsite, _p(_f64(p.qs)), beta(p), p.k_e,
                              p.eps_r, p.eta, kappa(p), _p(T), _p(S2), int(nthreads))
    if rc != 0:
        raise MemoryError("oracle allocation failed")
    return T, (float(S2[0]), float(S2[1]))


def kspace_kcut(p: Problem, tol):
    """Cut-off wave number (1/A) where the bound of eq. (k-space-dcf-err) equals tol (0: no cut-off)."""
    return _load().orc_kspace_kcut(p.eta, float(np.max(np.abs(p.qs))), float(np.sum(np.abs(p.q))), beta(p), p.k_e,
                                   float(tol))


def kspace_bound(p: Problem, k):
    return _load().orc_kspace_bound(float(k), p.eta, float(np.max(np.abs(p.qs))), float(np.sum(np.abs(p.q))),
                                    beta(p), p.k_e)


def kspace(p: Problem, kcut=0.0, idx=None, want=("c", "h"), nthreads: int = 0):
    """c_s(k), h_s(k) of eqs. (dcf-k)/(tcf-k) on the half spectrum [S, nz*ny*(nx//2+1)] (complex128), or at the
    listed flat indices of it; entries with k > kcut are 0 (kcut <= 0: none)."""
    lib = _load()
    nx, ny, nz = (int(v) for v in p.n)
    m = (nx // 2 + 1) * ny * nz if idx is None else int(len(idx))
    if idx is not None:
        idx = np.ascontiguousarray(idx, dtype=np.int64)
    out = {k: (np.zeros((p.nsite, m), dtype=np.complex128) if k in want else None) for k in ("c", "h")}
    org = _f64(p.origin)
    lib.orc_kspace(p.natoms, _p(_f64(p.xyz)), _p(_f64(p.q)), p.nsite, _p(_f64(p.qs)), beta(p), p.k_e, p.eps_r,
                   p.eta, kappa(p), nx, ny, nz, p.h, _p(org), float(kcut), m, _p(idx), _p(out["c"]), _p(out["h"]),
                   int(nthreads))
    return {k: v for k, v in out.items() if v is not None}


TAYLOR_KINDS = {"coulomb": 0, "erf": 1, "yukawa": 2}


def taylor_index(k1, k2, k3):
    """Graded position of multi-index k in the coefficient arrays of taylor_coeffs."""
    n = k1 + k2 + k3
    i = n - k1
    return n * (n + 1) * (n + 2) // 6 + i * (i + 1) // 2 + (i - k2)


def taylor_coeffs(kind, p, r, eta=1.0, kappa_=0.0):
    """a_k = (1/k!) d^k/dy^k phi at x - y = r, |k| <= p, by the paper's recurrences (graded order)."""
    a = np.empty((p + 1) * (p + 2) * (p + 3) // 6)
    _load().orc_taylor_coeffs(TAYLOR_KINDS[kind], int(p), float(r[0]), float(r[1]), float(r[2]), float(eta),
                              float(kappa_), _p(a))
    return a


def taylor_eval(kind, p, center, xyz, q, pts, eta=1.0, kappa_=0.0):
    """The order-p Taylor approximation about `center` of sum_j q_j phi(x, y_j) at the points."""
    xyz, q, pts, c = _f64(xyz), _f64(q), _f64(pts), _f64(center)
    out = np.empty(len(pts))
    _load().orc_taylor_eval(TAYLOR_KINDS[kind], int(p), _p(c), len(q), _p(xyz), _p(q), float(eta), float(kappa_),
                            len(pts), _p(pts), _p(out))
    return out


def parameter_guide(tolerance):
    """The paper's accuracy parameters for a residual tolerance of the 3D-RISM solution.  Table 3 (Sec. 4.2.1):
    MAC 0.3, leaf size N0 = 500 and the Taylor order of each kernel, the least integer p >= 2 that is at least
    (log10 tolerance + 5.7) / -0.7 for the TCF, (log10 tolerance + 1.9) / -0.8 for the DCF and
    (log10 tolerance + 1.4) / -0.8 for the Coulomb potential (counted up from 2; a value the expression hits
    exactly, up to the rounding of log10, is kept).  Sec. 4.3.1: the reciprocal-space cut-off tolerance
    0.04 tolerance^0.9.  Sec. 4.4.1: the LJ cut-off tolerance, one tenth of the residual tolerance."""
    import math

    if not (0.0 < tolerance < 1.0) or not math.isfinite(tolerance):
        raise ValueError("tolerance must lie in (0, 1)")
    lt = math.log10(tolerance)

    def least_order(intercept, slope):
        bound = (lt + intercept) / slope
        p = 2
        while p < bound - 1e-9:
            p += 1
        return p

    return {"p_tcf": least_order(5.7, -0.7), "p_dcf": least_order(1.9, -0.8), "p_coulomb": least_order(1.4, -0.8),
            "mac": 0.3, "n0": 500, "k_tol": 0.04 * tolerance ** 0.9, "lj_tol": 0.1 * tolerance}
