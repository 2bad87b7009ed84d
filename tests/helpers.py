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


def check_fields(gpu, ref, keys, tol, grid=None, xyz=None, idx=None, label=""):
    """rel L2 per output grid <= tol, over all points and over points >= 1 A from every atom."""
    mask = far_mask(grid, xyz, 1.0, idx) if grid is not None else None
    for k in keys:
        g = np.asarray(gpu[k]).reshape(ref[k].shape)
        e = rel_l2(g, ref[k])
        assert e <= tol, f"{label} {k}: rel L2 {e:.3e} > {tol:g}"
        if mask is not None and mask.any():
            em = rel_l2(g[:, mask], ref[k][:, mask])
            assert em <= tol, f"{label} {k} (>= 1 A from atoms): rel L2 {em:.3e} > {tol:g}"
