"""Shared helpers of the GPU parity tests (not collected by pytest)."""
import numpy as np


def rel_l2(a, b):
    a = np.asarray(a, dtype=np.float64).ravel()
    b = np.asarray(b, dtype=np.float64).ravel()
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def grid_points(grid, idx=None):
    nx, ny, nz = grid.n
    f = np.arange(nx * ny * nz, dtype=np.int64) if idx is None else np.asarray(idx, dtype=np.int64)
    i, j, k = f % nx, (f // nx) % ny, f // (nx * ny)
    o = np.asarray(grid.origin)
    return np.stack([o[0] + grid.h * i, o[1] + grid.h * j, o[2] + grid.h * k], 1)


def far_mask(grid, xyz, rmin=1.0, idx=None):
    """True at grid points at least ``rmin`` from every atom."""
    from scipy.spatial import cKDTree

    pts = grid_points(grid, idx)
    if len(xyz) == 0:
        return np.ones(len(pts), dtype=bool)
    d, _ = cKDTree(xyz).query(pts, k=1)
    return d >= rmin


def nearest_points(grid, xyz, count=None):
    """Flat indices of the grid point nearest to each atom (the largest |u| values)."""
    nx, ny, nz = grid.n
    o = np.asarray(grid.origin)
    ijk = np.rint((np.asarray(xyz) - o) / grid.h).astype(np.int64)
    ijk[:, 0] = np.clip(ijk[:, 0], 0, nx - 1)
    ijk[:, 1] = np.clip(ijk[:, 1], 0, ny - 1)
    ijk[:, 2] = np.clip(ijk[:, 2], 0, nz - 1)
    f = (ijk[:, 2] * ny + ijk[:, 1]) * nx + ijk[:, 0]
    f = np.unique(f)
    return f if count is None else f[:count]


def max_abs_rel(a, b):
    """max |a - b| over max |b|: the max-abs error of a grid, in units of the grid's largest value."""
    a = np.asarray(a, dtype=np.float64).ravel()
    b = np.asarray(b, dtype=np.float64).ravel()
    return float(np.abs(a - b).max() / max(np.abs(b).max(), 1e-300)) if b.size else 0.0


# Max-abs error / max |ref| allowed per tolerance class (rel L2 tolerance -> max-abs tolerance).  FP64 direct
# sums: the same 1e-12.  FP32 pairs: 4e-6, because the exact split erf(x)/d = 1/d - erfc(x)/d cancels at grid
# points much closer to an atom than eta (at d = 0.05 A the two terms are 20x the result), so the largest
# |c| and |h| values, found next to atoms, carry a few 1e-7 relative of FP32 rounding times that factor; the
# rel L2 over the grid stays at 1e-7.  Treecode at degree 8, theta 0.7: the same 1e-5 as its rel L2.
MAX_ABS_TOL = {1e-12: 1e-12, 1e-6: 4e-6, 1e-5: 1e-5}


def check_fields(gpu, ref, keys, tol, grid=None, xyz=None, idx=None, label="", max_tol=None):
    """Per output grid: rel L2 <= tol and max-abs error / max |ref| <= max_tol (default: the class's
    MAX_ABS_TOL), over all points and over the points >= 1 A from every atom.  Non-finite reference values (a
    point on an atom) must be matched exactly and are left out of both norms."""
    max_tol = MAX_ABS_TOL.get(tol, tol) if max_tol is None else max_tol
    mask = far_mask(grid, xyz, 1.0, idx) if grid is not None else None
    for k in keys:
        g = np.asarray(gpu[k]).reshape(ref[k].shape)
        r = ref[k]
        fin = np.isfinite(r)
        if not fin.all():
            assert np.array_equal(g[~fin], r[~fin]), f"{label} {k}: non-finite values differ"
        sel = fin.all(axis=0) if r.ndim == 2 else fin
        gg, rr = (g[:, sel], r[:, sel]) if r.ndim == 2 else (g[sel], r[sel])
        e = rel_l2(gg, rr)
        assert e <= tol, f"{label} {k}: rel L2 {e:.3e} > {tol:g}"
        m = max_abs_rel(gg, rr)
        assert m <= max_tol, f"{label} {k}: max-abs error / max |ref| {m:.3e} > {max_tol:g}"
        if mask is not None:
            mk = mask & sel
            if mk.any():
                gm, rm = (g[:, mk], r[:, mk]) if r.ndim == 2 else (g[mk], r[mk])
                em = rel_l2(gm, rm)
                assert em <= tol, f"{label} {k} (>= 1 A from atoms): rel L2 {em:.3e} > {tol:g}"
                mm = max_abs_rel(gm, rm)
                assert mm <= max_tol, f"{label} {k} (>= 1 A from atoms): max-abs / max {mm:.3e} > {max_tol:g}"


def lj_boundary_pairs(grid, xyz, rcut, rel=2.0 ** -20):
    """(point, atom) pairs whose LJ cut-off membership FP32 rounding of d^2 can flip: |d^2 - rc^2| <= rel rc^2
    (rel covers the rounding of an FP32 distance square, a few ulp).  Columns (i, j) of the disc around each
    atom are scanned and the k range of the thin shell solved for directly.  Returns flat point indices and
    atom indices (one entry per pair)."""
    nx, ny, nz = grid.n
    h = grid.h
    o = np.asarray(grid.origin, dtype=np.float64)
    lo2, hi2 = rcut * rcut * (1.0 - rel), rcut * rcut * (1.0 + rel)
    r = int(np.ceil(rcut * np.sqrt(1.0 + rel) / h)) + 1
    di, dj = np.meshgrid(np.arange(-r, r + 1), np.arange(-r, r + 1), indexing="ij")
    di, dj = di.ravel(), dj.ravel()
    pts, ats = [], []
    for a, R in enumerate(np.asarray(xyz, dtype=np.float64)):
        c = np.floor((R - o) / h).astype(np.int64)
        i, j = c[0] + di, c[1] + dj
        ok = (i >= 0) & (i < nx) & (j >= 0) & (j < ny)
        i, j = i[ok], j[ok]
        dx, dy = o[0] + h * i - R[0], o[1] + h * j - R[1]
        rem_lo, rem_hi = lo2 - dx * dx - dy * dy, hi2 - dx * dx - dy * dy
        keep = rem_hi >= 0.0
        i, j, rem_lo, rem_hi = i[keep], j[keep], rem_lo[keep], rem_hi[keep]
        zlo = np.sqrt(np.maximum(rem_lo, 0.0))
        zhi = np.sqrt(rem_hi)
        for sgn in (1.0, -1.0):
            # dz in [zlo, zhi] (or its mirror): k with o_z + h k - R_z in that interval
            a0, a1 = (zlo, zhi) if sgn > 0 else (-zhi, -zlo)
            k0 = np.ceil((R[2] + a0 - o[2]) / h - 1e-9).astype(np.int64)
            k1 = np.floor((R[2] + a1 - o[2]) / h + 1e-9).astype(np.int64)
            for t in np.nonzero(k1 >= k0)[0]:
                for k in range(max(k0[t], 0), min(k1[t], nz - 1) + 1):
                    d2 = (o[0] + h * i[t] - R[0]) ** 2 + (o[1] + h * j[t] - R[1]) ** 2 + (o[2] + h * k - R[2]) ** 2
                    if lo2 <= d2 <= hi2 and not (sgn < 0 and zlo[t] == 0.0 and o[2] + h * k - R[2] >= 0.0):
                        pts.append((k * ny + j[t]) * nx + i[t])
                        ats.append(a)
    return np.asarray(pts, dtype=np.int64), np.asarray(ats, dtype=np.int64)
