"""Seeded synthetic workloads for the 3D-RISM initialization path.

This module only draws inputs: solute atoms (positions, partial charges and
Lennard-Jones sigma/epsilon), solvent site tables, grid descriptors, upstream
cotangent fields and point samples.  It holds none of the method's
arithmetic (no potentials, no mixing rules, no Debye length), so the CUDA
path and the CPU oracle can both consume its output without sharing any of
the computation they are compared on.

The paper's solutes (Table 1: phenol ... microtubule) come from PDB
structures and Amber force fields that are not available here; the
generators below stand in for them with globules of the same atom counts,
net charges and protein-like atom density (Sec. 3.1 describes the real
systems).  The solvent is the one of Sec. 3.2: water (55.2 M) with 0.1 M
NaCl, dielectric constant 78.44.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

AVOGADRO = 6.02214076e23
# number density (1/A^3) of a 1 mol/L species
MOLAR_TO_PER_A3 = AVOGADRO * 1e-27

# Solvent sites: charge (e), sigma (A), epsilon (kcal/mol), bulk number
# density of the site (1/A^3) and whether the site is an ionic co-solvent.
# Water site values are those of the workload definitions (SPC/E-like
# oxygen, a small hydrogen core); the ions use the Na+/Cl- parameters the
# workloads name.  The H density counts both hydrogens of each water.
SOLVENT_SITES = {
    "O": dict(q=-0.8476, sigma=3.166, eps=0.1553, rho=55.2 * MOLAR_TO_PER_A3, is_ion=0),
    "H": dict(q=+0.4238, sigma=1.0, eps=0.01, rho=2 * 55.2 * MOLAR_TO_PER_A3, is_ion=0),
    "Na+": dict(q=+1.0, sigma=2.16, eps=0.35, rho=0.1 * MOLAR_TO_PER_A3, is_ion=1),
    "Cl-": dict(q=-1.0, sigma=4.83, eps=0.01, rho=0.1 * MOLAR_TO_PER_A3, is_ion=1),
}

PROTEIN_DENSITY = 0.116  # atoms / A^3


@dataclass
class Solute:
    xyz: np.ndarray  # [n, 3] float64, A
    q: np.ndarray  # [n] float64, e
    sigma: np.ndarray  # [n] float64, A
    eps: np.ndarray  # [n] float64, kcal/mol

    @property
    def n(self) -> int:
        return int(self.q.shape[0])


@dataclass
class Solvent:
    names: list
    q: np.ndarray
    sigma: np.ndarray
    eps: np.ndarray
    rho: np.ndarray
    is_ion: np.ndarray  # int32

    @property
    def nsite(self) -> int:
        return int(self.q.shape[0])


@dataclass
class Grid:
    n: tuple  # (nx, ny, nz)
    h: float
    origin: tuple  # (ox, oy, oz)

    @property
    def npts(self) -> int:
        return int(self.n[0]) * int(self.n[1]) * int(self.n[2])


@dataclass
class Workload:
    name: str
    solute: Solute
    solvent: Solvent
    grid: Grid
    # physical / method options (see include/rism3d.h for their meaning)
    opts: dict = field(default_factory=dict)


def solvent(names) -> Solvent:
    rows = [SOLVENT_SITES[n] for n in names]
    return Solvent(
        names=list(names),
        q=np.array([r["q"] for r in rows], dtype=np.float64),
        sigma=np.array([r["sigma"] for r in rows], dtype=np.float64),
        eps=np.array([r["eps"] for r in rows], dtype=np.float64),
        rho=np.array([r["rho"] for r in rows], dtype=np.float64),
        is_ion=np.array([r["is_ion"] for r in rows], dtype=np.int32),
    )


def _rsa(n, inside, box_lo, box_hi, min_spacing, rng, max_tries=400):
    """Random sequential addition: uniform candidates inside the body,
    rejected when closer than ``min_spacing`` to an accepted point."""
    cell = float(min_spacing)
    grid = {}
    pts = np.empty((n, 3), dtype=np.float64)
    k = 0
    ms2 = min_spacing * min_spacing
    tries = 0
    batch = 4096
    while k < n:
        cand = rng.uniform(box_lo, box_hi, size=(batch, 3))
        cand = cand[inside(cand)]
        for p in cand:
            tries += 1
            if tries > max_tries * n:
                raise RuntimeError("random sequential addition did not converge")
            ci = (int(math.floor(p[0] / cell)), int(math.floor(p[1] / cell)),
                  int(math.floor(p[2] / cell)))
            ok = True
            for dx in (-1, 0, 1):
                for dy in (-1, 0, 1):
                    for dz in (-1, 0, 1):
                        lst = grid.get((ci[0] + dx, ci[1] + dy, ci[2] + dz))
                        if lst is None:
                            continue
                        for j in lst:
                            d = pts[j] - p
                            if d[0] * d[0] + d[1] * d[1] + d[2] * d[2] < ms2:
                                ok = False
                                break
                        if not ok:
                            break
                    if not ok:
                        break
                if not ok:
                    break
            if ok:
                pts[k] = p
                grid.setdefault(ci, []).append(k)
                k += 1
                if k == n:
                    break
    return pts


def _params(n, net_charge, rng):
    q = rng.normal(0.0, 0.35, size=n)
    q = q - q.mean() + net_charge / n
    sigma = rng.uniform(1.0, 3.8, size=n)
    eps = rng.uniform(0.01, 0.2, size=n)
    return q, sigma, eps


def sphere_solute(n, radius, net_charge, seed, min_spacing=1.2, center=(0.0, 0.0, 0.0)) -> Solute:
    rng = np.random.default_rng(seed)
    c = np.asarray(center, dtype=np.float64)
    r2 = radius * radius

    def inside(p):
        return ((p - c) ** 2).sum(axis=1) < r2

    xyz = _rsa(n, inside, c - radius, c + radius, min_spacing, rng)
    q, s, e = _params(n, net_charge, rng)
    return Solute(xyz, q, s, e)


def ellipsoid_solute(n, semi_axes, net_charge, seed, min_spacing=1.2, center=(0.0, 0.0, 0.0)) -> Solute:
    rng = np.random.default_rng(seed)
    c = np.asarray(center, dtype=np.float64)
    ax = np.asarray(semi_axes, dtype=np.float64)

    def inside(p):
        return (((p - c) / ax) ** 2).sum(axis=1) < 1.0

    xyz = _rsa(n, inside, c - ax, c + ax, min_spacing, rng)
    q, s, e = _params(n, net_charge, rng)
    return Solute(xyz, q, s, e)


def globule_radius(n, density=PROTEIN_DENSITY):
    return (3.0 * n / (4.0 * math.pi * density)) ** (1.0 / 3.0)


def centred_grid(n, h) -> Grid:
    n = tuple(int(v) for v in n)
    origin = tuple(-h * (v - 1) / 2.0 for v in n)
    return Grid(n=n, h=float(h), origin=origin)


BASE_OPTS = dict(eta=1.0, T=298.0, eps_r=78.44, k_e=332.0522173, k_B=0.0019872041)


def workload(idx: int, seed: int = 0) -> Workload:
    """The five workload definitions of the benchmark plan.

    0: 200 atoms in a 12 A sphere, 64^3 grid, water O/H, FP64 direct, no LJ cut-off, no ions.
    1: 2,000-atom globule (net +8), 128^3 grid, water + 0.1 M NaCl, LJ cut-off 9 A.
    2: 13,600-atom prolate ellipsoid 80x65x45 A (net -24), 224x192x160 grid.
    4: 55,000 atoms, four config-2-shaped ellipsoids stacked along z, 320x320x384 grid.
    (3, the batch of 32 solutes, is built by ``batch_workloads``.)
    """
    if idx == 0:
        sol = sphere_solute(200, 12.0, 0.0, seed=1000 + seed)
        return Workload("sphere200_64cubed", sol, solvent(["O", "H"]), centred_grid((64, 64, 64), 0.5),
                        dict(BASE_OPTS, lj_rcut=0.0))
    if idx == 1:
        sol = sphere_solute(2000, globule_radius(2000), 8.0, seed=1100 + seed)
        return Workload("globule2000_128cubed", sol, solvent(["O", "H", "Na+", "Cl-"]),
                        centred_grid((128, 128, 128), 0.5), dict(BASE_OPTS, lj_rcut=9.0, degree=8, theta=0.7))
    if idx == 2:
        sol = ellipsoid_solute(13600, (40.0, 32.5, 22.5), -24.0, seed=1200 + seed)
        return Workload("ellipsoid13600_224x192x160", sol, solvent(["O", "H", "Na+", "Cl-"]),
                        centred_grid((224, 192, 160), 0.5), dict(BASE_OPTS, lj_rcut=9.0, degree=8, theta=0.7))
    if idx == 4:
        parts = []
        for k, zc in enumerate((-67.5, -22.5, 22.5, 67.5)):
            parts.append(ellipsoid_solute(13750, (40.0, 32.5, 22.5), -24.0, seed=1400 + 10 * seed + k,
                                          center=(0.0, 0.0, zc)))
        sol = Solute(np.concatenate([p.xyz for p in parts]), np.concatenate([p.q for p in parts]),
                     np.concatenate([p.sigma for p in parts]), np.concatenate([p.eps for p in parts]))
        return Workload("stack55000_320x320x384", sol, solvent(["O", "H", "Na+", "Cl-"]),
                        centred_grid((320, 320, 384), 0.5), dict(BASE_OPTS, lj_rcut=9.0))
    raise ValueError("workload index must be 0, 1, 2 or 4 (3 is batch_workloads)")


def batch_workloads(count=32, seed=0, lo=500, hi=8000, buffer=12.0, h=0.5, multiple=16):
    """Uneven batch: atom counts log-uniform in [lo, hi], each a globule at
    protein density with its own centred grid (extent 2R + 2*buffer, rounded
    up to a multiple of ``multiple`` points)."""
    rng = np.random.default_rng(3000 + seed)
    ns = np.exp(rng.uniform(math.log(lo), math.log(hi), size=count)).astype(int)
    out = []
    for k, n in enumerate(ns):
        R = globule_radius(int(n))
        net = float(round(-24.0 * n / 13600.0))
        sol = sphere_solute(int(n), R, net, seed=3100 + 100 * seed + k)
        pts = int(math.ceil((2 * R + 2 * buffer) / h))
        pts = ((pts + multiple - 1) // multiple) * multiple
        out.append(Workload(f"globule{n}_{pts}cubed", sol, solvent(["O", "H", "Na+", "Cl-"]),
                            centred_grid((pts, pts, pts), h), dict(BASE_OPTS, lj_rcut=9.0, degree=8, theta=0.7)))
    return out


def small_workload(n_atoms=37, n=(19, 13, 11), h=0.5, seed=7, ions=True, lj_rcut=0.0, net=1.0,
                   radius=None) -> Workload:
    """A small ragged case (odd grid dims, a few atom tiles) for fast parity tests."""
    R = radius if radius is not None else max(2.0, globule_radius(n_atoms))
    sol = sphere_solute(n_atoms, R, net, seed=seed)
    names = ["O", "H", "Na+", "Cl-"] if ions else ["O", "H"]
    return Workload(f"small{n_atoms}", sol, solvent(names), centred_grid(n, h), dict(BASE_OPTS, lj_rcut=lj_rcut))


def gaussian_random_field(shape_zyx, h, seed, corr_len=3.0, amplitude=0.5):
    """Smooth seeded field: white noise convolved with a Gaussian of width
    ``corr_len`` (A), rescaled to standard deviation ``amplitude``."""
    from scipy.ndimage import gaussian_filter

    rng = np.random.default_rng(seed)
    w = rng.standard_normal(shape_zyx)
    f = gaussian_filter(w, sigma=corr_len / h, mode="wrap")
    f *= amplitude / f.std()
    return f


def sample_indices(npts, count, seed):
    rng = np.random.default_rng(seed)
    count = min(int(count), int(npts))
    return np.sort(rng.choice(npts, size=count, replace=False)).astype(np.int64)
