"""Pins of the FP64 oracle against the paper and against mathematics.

None of these compares the oracle with itself: each check uses a closed form,
a limit, an independent transform, a symmetry/invariant, a textbook value or
high-precision brute force, chosen so that a dropped term, a wrong sign, a
wrong prefactor or a transposed index in the oracle fails at least one.
"""
import math

import mpmath as mp
import numpy as np
import pytest
from scipy import integrate

from oracle import oracle as O
from paper_2109_09772_gb300 import inputs as I

ETA = 1.0
KAPPA = 0.10401606295269093  # 0.1 M NaCl, 298 K (pinned separately below)


def _one_atom_problem(pos, q=1.0, sigma=2.0, eps=0.0, site=(1.0, 2.0, 0.0), n=(5, 4, 3), h=0.5,
                      origin=(0.0, 0.0, 0.0), **kw):
    return O.Problem(xyz=np.array([pos], dtype=float), q=np.array([q]), sigma=np.array([sigma]),
                     eps=np.array([eps]), qs=np.array([site[0]]), sigs=np.array([site[1]]),
                     epss=np.array([site[2]]), rho=np.array([0.03]), is_ion=np.array([0], dtype=np.int32),
                     n=n, h=h, origin=origin, **kw)


# ---------------------------------------------------------------- kernels
def test_dcf_kernel_limits():
    """eq. (dcf-r): erf(d/eta)/d -> 2/(eta sqrt(pi)) at d = 0 and -> 1/d for d >> eta."""
    for eta in (0.7, 1.0, 1.6):
        pc, _, _, _ = O.kernels(eta, 0.0, [0.0, 1e-9])
        assert pc[0] == pytest.approx(2 / (eta * math.sqrt(math.pi)), rel=1e-15)
        assert pc[1] == pytest.approx(2 / (eta * math.sqrt(math.pi)), rel=1e-15)
        d = np.array([10.0, 20.0, 50.0]) * eta
        pc, _, _, _ = O.kernels(eta, 0.0, d)
        np.testing.assert_allclose(pc, 1.0 / d, rtol=1e-15)


def test_series_and_formula_agree_at_switch():
    """The small-d series and the closed forms must meet continuously."""
    for kappa in (0.0, KAPPA, 0.5):
        x0 = 0.02
        d = np.array([np.nextafter(x0, 0.0), np.nextafter(x0, 1.0)])
        pc, ph, gc, gh = O.kernels(ETA, kappa, d)
        assert abs(pc[0] - pc[1]) < 1e-13 * abs(pc[0])
        assert abs(ph[0] - ph[1]) < 1e-13 * abs(ph[0])
        assert abs(gc[0] - gc[1]) < 1e-9 * abs(gc[0])
        assert abs(gh[0] - gh[1]) < 1e-9 * abs(gh[0])


def _phi_h_mp(d, eta, kappa):
    mp.mp.dps = 60
    d, eta, kappa = mp.mpf(d), mp.mpf(eta), mp.mpf(kappa)
    a = kappa * eta / 2
    x = d / eta
    return mp.exp(a * a) * (mp.exp(-kappa * d) * mp.erfc(a - x) - mp.exp(kappa * d) * mp.erfc(a + x)) / d


def test_tcf_kernel_vs_high_precision():
    """eq. (tcf-r) bracket at small, medium and large d against 60-digit mpmath."""
    for kappa in (KAPPA, 0.35):
        d = np.array([1e-7, 1e-4, 5e-3, 0.0199, 0.0201, 0.05, 0.3, 1.0, 2.5, 6.0, 15.0, 40.0])
        _, ph, _, _ = O.kernels(ETA, kappa, d)
        ref = np.array([float(_phi_h_mp(v, ETA, kappa)) for v in d])
        np.testing.assert_allclose(ph, ref, rtol=2e-14)


def test_tcf_kernel_limits():
    """d -> 0 limit 2[2/(eta sqrt pi) - kappa erfcx(a)]; d >> eta gives eq. (tcfexp) times e^{a^2}."""
    a = KAPPA * ETA / 2
    lim = 2 * (2 / (ETA * math.sqrt(math.pi)) - KAPPA * float(mp.exp(a * a) * mp.erfc(a)))
    _, ph, _, _ = O.kernels(ETA, KAPPA, [0.0])
    assert ph[0] == pytest.approx(lim, rel=1e-14)
    d = np.array([8.0, 12.0, 30.0])
    _, ph, _, _ = O.kernels(ETA, KAPPA, d)
    far = 2 * math.exp(a * a) * np.exp(-KAPPA * d) / d
    np.testing.assert_allclose(ph, far, rtol=1e-14)


def test_tcf_reduces_to_dcf_without_ions():
    """kappa -> 0: the TCF kernel of eq. (tcf-r) becomes 2 erf(d/eta)/d, i.e. twice eq. (dcf-r)."""
    d = np.array([0.0, 0.01, 0.1, 0.5, 1.0, 3.0, 9.0])
    pc, ph, gc, gh = O.kernels(ETA, 0.0, d)
    np.testing.assert_allclose(ph, 2 * pc, rtol=1e-14)
    np.testing.assert_allclose(gh, 2 * gc, rtol=1e-9, atol=1e-14)


def _radial_inverse_ft(kF, r, kmax):
    """f(r) = 1/(2 pi^2 r) int_0^inf sin(kr) [k F(k)] dk (3D radial inverse Fourier transform);
    ``kF`` is k F(k), written so that it is finite at k = 0."""
    val, _ = integrate.quad(lambda k: math.sin(k * r) * kF(k), 0.0, kmax, limit=800, epsabs=0, epsrel=1e-12)
    return val / (2 * math.pi ** 2 * r)


def test_hankel_pairs_with_k_space_forms():
    """The real-space kernels are the inverse transforms of the k-space forms eq. (dcf-k) and eq. (tcf-k):
    4 pi/k^2 e^{-k^2 eta^2/4} <-> erf(r/eta)/r and 4 pi/(k^2+kappa^2) e^{-k^2 eta^2/4} <-> phi_h(r)/2.
    This pins the factor 2, the sign and the e^{kappa^2 eta^2/4} prefactor of eq. (tcf-r)."""
    kmax = 14.0 / ETA
    r = np.array([0.3, 1.0, 3.0, 10.0])
    pc, ph, _, _ = O.kernels(ETA, KAPPA, r)
    g = lambda k: math.exp(-k * k * ETA * ETA / 4)
    for i, rv in enumerate(r):
        # k * 4 pi / k^2 = 4 pi / k, and sin(kr)/k -> r at k = 0
        val_c, _ = integrate.quad(lambda k: 4 * math.pi * (rv if k == 0 else math.sin(k * rv) / k) * g(k),
                                  0.0, kmax, limit=800, epsabs=0, epsrel=1e-12)
        fc = val_c / (2 * math.pi ** 2 * rv)
        fh = _radial_inverse_ft(lambda k: 4 * math.pi * k / (k * k + KAPPA ** 2) * g(k), rv, kmax)
        assert pc[i] == pytest.approx(fc, rel=1e-9)
        assert ph[i] / 2 == pytest.approx(fh, rel=1e-9)


def test_kernel_derivatives_against_finite_differences():
    d = np.array([0.03, 0.2, 0.9, 2.0, 5.0])
    hstep = 1e-6
    for kappa in (0.0, KAPPA):
        pp, hp, _, _ = O.kernels(ETA, kappa, d + hstep)
        pm, hm, _, _ = O.kernels(ETA, kappa, d - hstep)
        _, _, gc, gh = O.kernels(ETA, kappa, d)
        np.testing.assert_allclose(gc * d, (pp - pm) / (2 * hstep), rtol=1e-7, atol=1e-9)
        np.testing.assert_allclose(gh * d, (hp - hm) / (2 * hstep), rtol=1e-7, atol=1e-9)


# ---------------------------------------------------------------- physics
def test_debye_kappa_textbook():
    """0.1 M 1:1 salt in water at 298 K: Debye length 0.304 nm / sqrt(0.1) = 9.61 A."""
    w = I.workload(1)
    p = O.Problem.from_workload(w)
    k = O.kappa(p)
    assert 1.0 / k == pytest.approx(9.61, abs=0.02)
    assert k == pytest.approx(KAPPA, rel=1e-12)


def test_single_charge_closed_form():
    """One unit charge, LJ off: u = k_e q_s q / d, c = -beta k_e q_s q erf(d/eta)/d at every grid point."""
    pos = (0.13, 0.41, 0.27)
    p = _one_atom_problem(pos, q=0.7, eps=0.0, site=(-0.8, 3.0, 0.1), n=(6, 5, 4), h=0.5,
                          origin=(-1.0, -0.7, -0.4), kappa=KAPPA)
    f = O.fields(p)
    ii, jj, kk = np.meshgrid(np.arange(6), np.arange(5), np.arange(4), indexing="ij")
    pts = np.stack([(-1.0 + 0.5 * ii).transpose(2, 1, 0).ravel(), (-0.7 + 0.5 * jj).transpose(2, 1, 0).ravel(),
                    (-0.4 + 0.5 * kk).transpose(2, 1, 0).ravel()], 1)
    d = np.linalg.norm(pts - np.array(pos), axis=1)
    beta = 1.0 / (p.k_B * p.T)
    np.testing.assert_allclose(f["u"][0], p.k_e * -0.8 * 0.7 / d, rtol=1e-14)
    erf = np.array([math.erf(v / ETA) for v in d])
    np.testing.assert_allclose(f["c"][0], -beta * p.k_e * -0.8 * 0.7 * erf / d, rtol=1e-14)


def test_grid_index_order():
    """Flat index (k ny + j) nx + i, x fastest: the nearest grid point to an atom holds the largest |u|."""
    p = _one_atom_problem((1.0, 0.5, 1.5), q=1.0, eps=0.0, n=(7, 5, 6), h=0.5, origin=(0.0, 0.0, 0.0))
    f = O.fields(p, want=("u",))
    k = int(np.argmax(np.abs(f["u"][0])))
    assert k == (3 * 5 + 1) * 7 + 2


def test_lj_minimum_and_zero():
    """Lorentz-Berthelot with sigma_i = sigma_s: u_LJ = -eps_is at 2^(1/6) sigma and 0 at sigma."""
    sig, ei, es = 3.0, 0.16, 0.09
    rmin = 2 ** (1 / 6) * sig
    for dist, expect in ((rmin, -math.sqrt(ei * es)), (sig, 0.0)):
        # grid point at origin, atom at distance `dist` along x
        p = _one_atom_problem((dist, 0.0, 0.0), q=0.0, sigma=sig, eps=ei, site=(0.0, sig, es), n=(1, 1, 1))
        u = O.fields(p, want=("u",))["u"][0, 0]
        assert u == pytest.approx(expect, abs=1e-14)


def test_lj_cutoff_membership():
    """eq. (ulj-trunc): pairs with d < r_cut are kept; d >= r_cut (equality included) are dropped."""
    rc = 4.0
    for dist, kept in ((rc - 1e-9, True), (rc, False), (rc + 1e-9, False)):
        p = _one_atom_problem((dist, 0.0, 0.0), q=0.0, sigma=3.0, eps=0.2, site=(0.0, 3.0, 0.2), n=(1, 1, 1),
                              lj_rcut=rc)
        u = O.fields(p, want=("u",))["u"][0, 0]
        assert (u != 0.0) == kept


def test_lj_tail_correction_quadrature():
    """Sec. 2.6: I = 4 pi int_rc^inf u_LJ(r) r^2 dr for each pair, summed over atoms."""
    w = I.small_workload(n_atoms=5, ions=True, lj_rcut=7.5)
    p = O.Problem.from_workload(w)
    I_s = O.lj_tail(p)
    for s in range(p.nsite):
        tot = 0.0
        for i in range(p.natoms):
            sg = 0.5 * (p.sigma[i] + p.sigs[s])
            ep = math.sqrt(p.eps[i] * p.epss[s])
            val, _ = integrate.quad(lambda r: 4 * math.pi * r * r * 4 * ep * ((sg / r) ** 12 - (sg / r) ** 6),
                                    7.5, np.inf, epsabs=0, epsrel=1e-13)
            tot += val
        assert I_s[s] == pytest.approx(tot, rel=1e-10)


def test_lj_tail_sign_by_grid_sum():
    """The correction is what the cut-off removes: sum_r (u_full - u_cut) h^3 -> I_s (sign and magnitude)."""
    rc, h = 3.0, 0.25
    n = 97
    org = (-h * (n - 1) / 2,) * 3
    base = dict(q=0.0, sigma=2.5, eps=0.2, site=(0.0, 2.5, 0.2), n=(n, n, n), h=h, origin=org)
    pos = (0.0375, -0.0125, 0.0875)
    full = O.fields(_one_atom_problem(pos, **base), want=("u",))["u"][0]
    cut_p = _one_atom_problem(pos, lj_rcut=rc, **base)
    cut = O.fields(cut_p, want=("u",))["u"][0]
    s = np.sum(full - cut) * h ** 3
    # the grid extends to ~12 A: add the analytic remainder beyond it only as a tolerance
    I_s = O.lj_tail(cut_p)[0]
    assert I_s < 0
    assert s == pytest.approx(I_s, rel=0.03)


def test_lj_rcut_from_tolerance():
    """Per-pair cut-off of Sec. 2.6: |u(r_cut)| = tol on the attractive tail (tol < eps) or the wall."""
    sg, ep = 3.2, 0.15
    for tol in (1e-3, 1e-6, 1e-9):
        rc = O.lj_rcut_tol(sg, ep, tol)
        u = 4 * ep * ((sg / rc) ** 12 - (sg / rc) ** 6)
        assert abs(u) == pytest.approx(tol, rel=1e-9)
        assert rc > 2 ** (1 / 6) * sg
    rc = O.lj_rcut_tol(sg, ep, 0.5)  # above the well depth: the repulsive wall
    u = 4 * ep * ((sg / rc) ** 12 - (sg / rc) ** 6)
    assert u == pytest.approx(0.5, rel=1e-9) and rc < sg


# ------------------------------------------------------------ invariants
def _random_problem(n_atoms, seed, **kw):
    w = I.small_workload(n_atoms=n_atoms, seed=seed, n=(9, 7, 5), ions=True)
    return O.Problem.from_workload(w, **kw)


def test_linearity_in_charges_and_superposition():
    p = _random_problem(11, seed=3, lj_rcut=0.0)
    rng = np.random.default_rng(0)
    q1, q2 = rng.normal(size=p.natoms), rng.normal(size=p.natoms)
    kap = O.kappa(p)

    def run(q, eps_on=True, atoms=None):
        sel = np.arange(p.natoms) if atoms is None else atoms
        pp = O.Problem(**{**p.__dict__, "q": q[sel], "xyz": p.xyz[sel], "sigma": p.sigma[sel],
                          "eps": (p.eps[sel] if eps_on else np.zeros(sel.size)), "kappa": kap})
        return O.fields(pp)

    a, b, ab = run(q1, False), run(q2, False), run(q1 + 2 * q2, False)
    for k in ("u", "c", "h"):
        np.testing.assert_allclose(ab[k], a[k] + 2 * b[k], rtol=1e-12, atol=1e-12 * np.abs(ab[k]).max())
    half1, half2 = np.arange(0, 5), np.arange(5, p.natoms)
    x, y, xy = run(q1, True, half1), run(q1, True, half2), run(q1, True)
    for k in ("u", "c", "h"):
        np.testing.assert_allclose(xy[k], x[k] + y[k], rtol=1e-12, atol=1e-12 * np.abs(xy[k]).max())


def test_on_atom_point_limits():
    """A grid point exactly on an atom: u = +inf, c and h take the finite d -> 0 limits."""
    p = _one_atom_problem((0.5, 0.5, 0.5), q=0.6, eps=0.1, site=(-0.8, 3.0, 0.15), n=(3, 3, 3), h=0.5,
                          origin=(0.0, 0.0, 0.0), kappa=KAPPA)
    f = O.fields(p)
    centre = (1 * 3 + 1) * 3 + 1
    assert np.isposinf(f["u"][0, centre])
    beta = 1.0 / (p.k_B * p.T)
    lim_c = -beta * p.k_e * -0.8 * 0.6 * 2 / (ETA * math.sqrt(math.pi))
    assert f["c"][0, centre] == pytest.approx(lim_c, rel=1e-14)
    assert np.all(np.isfinite(f["h"]))


def _mp_fields(p, kap):
    """Brute force at 40 digits straight from eqs. (dcf-r), (tcf-r) and the LJ + Coulomb potential."""
    mp.mp.dps = 40
    beta = 1 / (mp.mpf(p.k_B) * mp.mpf(p.T))
    ke, eta, kap = mp.mpf(p.k_e), mp.mpf(p.eta), mp.mpf(kap)
    a = kap * eta / 2
    nx, ny, nz = p.n
    S = p.nsite
    out = {k: np.zeros((S, nx * ny * nz)) for k in ("u", "c", "h")}
    for kk in range(nz):
        for jj in range(ny):
            for ii in range(nx):
                f = (kk * ny + jj) * nx + ii
                r = [mp.mpf(p.origin[0]) + mp.mpf(p.h) * ii, mp.mpf(p.origin[1]) + mp.mpf(p.h) * jj,
                     mp.mpf(p.origin[2]) + mp.mpf(p.h) * kk]
                for s in range(S):
                    u = c = hh = mp.mpf(0)
                    for i in range(p.natoms):
                        d = mp.sqrt(sum((r[t] - mp.mpf(p.xyz[i, t])) ** 2 for t in range(3)))
                        x = d / eta
                        qi, qs = mp.mpf(p.q[i]), mp.mpf(p.qs[s])
                        sg = (mp.mpf(p.sigma[i]) + mp.mpf(p.sigs[s])) / 2
                        ep = mp.sqrt(mp.mpf(p.eps[i]) * mp.mpf(p.epss[s]))
                        u += ke * qs * qi / d + 4 * ep * ((sg / d) ** 12 - (sg / d) ** 6)
                        c += -beta * ke * qs * qi * mp.erf(x) / d
                        hh += -beta * ke * qs * qi / (2 * mp.mpf(p.eps_r)) * mp.exp(a * a) * (
                            mp.exp(-kap * d) * mp.erfc(a - x) - mp.exp(kap * d) * mp.erfc(a + x)) / d
                    out["u"][s, f], out["c"][s, f], out["h"][s, f] = float(u), float(c), float(hh)
    return out


def test_brute_force_tiny_grid_mpmath():
    """4x3x3 grid, 3 atoms, 4 sites: every value to ~1e-14 of the 40-digit result."""
    w = I.small_workload(n_atoms=3, seed=11, n=(4, 3, 3), h=0.7, ions=True, radius=2.5)
    p = O.Problem.from_workload(w)
    kap = O.kappa(p)
    f = O.fields(p)
    ref = _mp_fields(p, kap)
    for k in ("u", "c", "h"):
        np.testing.assert_allclose(f[k], ref[k], rtol=5e-14, atol=0)


def test_threads_bitwise_deterministic():
    p = _random_problem(23, seed=5, lj_rcut=4.0)
    a = O.fields(p, nthreads=1)
    b = O.fields(p, nthreads=4)
    for k in a:
        assert np.array_equal(a[k], b[k])


# ------------------------------------------------------------- gradients
def _loss(p, G):
    f = O.fields(p)
    return sum(float(np.sum(G[k] * f[k])) for k in ("u", "c", "h"))


def test_gradient_against_finite_differences():
    """dL/dR, dL/dq, dL/dsigma, dL/deps of the oracle's gradient against central differences of its own
    fields (LJ cut-off off, so L is smooth).  Fields are sums over atoms, so atom i's derivative is taken
    on a problem holding atom i alone, which keeps the differenced totals small."""
    w = I.small_workload(n_atoms=6, seed=21, n=(8, 7, 6), h=0.6, ions=True)
    p = O.Problem.from_workload(w)
    p.kappa = O.kappa(p)
    rng = np.random.default_rng(1)
    M = p.npts
    G = {k: rng.normal(size=(p.nsite, M)) for k in ("u", "c", "h")}
    for i in (0, 3, 5):
        one = O.Problem(**{**p.__dict__, "xyz": p.xyz[i:i + 1].copy(), "q": p.q[i:i + 1].copy(),
                           "sigma": p.sigma[i:i + 1].copy(), "eps": p.eps[i:i + 1].copy()})
        # the charge derivative does not involve LJ: switch LJ off so L is not dominated by the r^-12 wall
        one_q = O.Problem(**{**one.__dict__, "eps": np.zeros(1)})
        g = O.grad(one, [0], G["u"], G["c"], G["h"])[0]
        gq = O.grad(one_q, [0], G["u"], G["c"], G["h"])[0]
        for t, (field, comp) in enumerate([("xyz", 0), ("xyz", 1), ("xyz", 2), ("q", None), ("sigma", None),
                                           ("eps", None)]):
            base = one_q if field == "q" else one
            want = gq[t] if field == "q" else g[t]
            step = 1e-6 if field != "eps" else 1e-8
            vals = []
            for sgn in (+1, -1):
                pp = O.Problem(**{**base.__dict__})
                arr = getattr(base, field).copy()
                if comp is None:
                    arr[0] += sgn * step
                else:
                    arr[0, comp] += sgn * step
                setattr(pp, field, arr)
                vals.append(_loss(pp, G))
            fd = (vals[0] - vals[1]) / (2 * step)
            assert want == pytest.approx(fd, rel=1e-5, abs=1e-9 * max(abs(v) for v in vals)), (i, field, comp)


# ------------------------------------------------- all-space LRA integral
def _lra_closed_forms(R, eta, kappa):
    """I_hc(R), I_hh(R) in closed form at 30 digits.  With sigma^2 = eta^2/2, b = kappa sigma, s = R/(2 sigma),
    P = e^{-kappa R} erfc(b - s), M = e^{kappa R} erfc(b + s) (the Gaussian-screened Yukawa transform evaluated
    with sigma), partial fractions of 1/(k^2 (k^2 + kappa^2)) and d/d(kappa^2) of the Yukawa transform give
    I_hc = (4 pi/kappa^2) [2 erf(s)/R - e^{b^2}(P - M)/R],
    I_hh = (4 pi e^{b^2}/(kappa R)) [R (P + M) - 2 kappa sigma^2 (P - M)],
    and at R = 0: I_hc = 8 pi erfcx(b)/kappa, I_hh = 32 [J + kappa J'/2], J(kappa) = (pi/(2 kappa)) erfcx(b)."""
    mp.mp.dps = 30
    k = mp.mpf(kappa)
    s2 = mp.mpf(eta) ** 2 / 2
    sig = mp.sqrt(s2)
    R = mp.mpf(R)
    E = mp.e ** ((k * sig) ** 2)
    if R == 0:
        J = lambda kk: mp.pi / (2 * kk) * mp.e ** ((kk * sig) ** 2) * mp.erfc(kk * sig)
        return float(8 * mp.pi * E * mp.erfc(k * sig) / k), float(32 * (J(k) + k * mp.diff(J, k) / 2))
    s = R / (2 * sig)
    P = mp.e ** (-k * R) * mp.erfc(k * sig - s)
    M = mp.e ** (k * R) * mp.erfc(k * sig + s)
    ihc = 4 * mp.pi / k ** 2 * (2 * mp.erf(s) / R - E * (P - M) / R)
    ihh = 4 * mp.pi * E / (k * R) * (R * (P + M) - 2 * k * s2 * (P - M))
    return float(ihc), float(ihh)


@pytest.mark.parametrize("eta,kappa", [(1.0, KAPPA), (0.7, 0.35)])
def test_lra_pair_integrals_against_closed_forms(eta, kappa):
    """The oracle's 1D quadratures of the overlap integrals against their closed forms."""
    R = np.array([0.0, 0.3, 1.2, 3.0, 10.0, 40.0, 100.0])
    ihc, ihh = O.lra_pair(eta, kappa, R)
    for i, r in enumerate(R):
        chc, chh = _lra_closed_forms(r, eta, kappa)
        assert ihc[i] == pytest.approx(chc, rel=1e-11), r
        assert ihh[i] == pytest.approx(chh, rel=1e-9, abs=1e-12 * abs(ihh[0])), r


def test_lra_pair_integrals_in_real_space():
    """The same overlaps from the real-space kernels of eqs. (tcf-r) and (dcf-r) (independent of the Fourier
    constants 8 pi, 4 pi and 1/(2 pi^2)): at R = 0 the radial integrals 4 pi int r^2 phi_h phi_c dr and
    4 pi int r^2 phi_h^2 dr; at R > 0 the radial convolution (2 pi/R) int r f(r) [G(R + r) - G(|R - r|)] dr
    with G(s) = int_0^s t g(t) dt (closed form for g = phi_c, nested quadrature for g = phi_h)."""
    from scipy.special import erf

    ph = lambda r: float(O.kernels(ETA, KAPPA, [r])[1][0])
    pc = lambda r: float(O.kernels(ETA, KAPPA, [r])[0][0])
    rmax = 420.0
    i0hc, _ = integrate.quad(lambda r: 4 * math.pi * r * r * ph(r) * pc(r), 0, rmax, limit=2000, epsrel=1e-12)
    i0hh, _ = integrate.quad(lambda r: 4 * math.pi * r * r * ph(r) ** 2, 0, rmax, limit=2000, epsrel=1e-12)
    ihc, ihh = O.lra_pair(ETA, KAPPA, [0.0, 4.0])
    assert ihc[0] == pytest.approx(i0hc, rel=1e-8)
    assert ihh[0] == pytest.approx(i0hh, rel=1e-8)
    R = 4.0
    Gc = lambda s: s * erf(s / ETA) + ETA / math.sqrt(math.pi) * (math.exp(-(s / ETA) ** 2) - 1.0)
    val, _ = integrate.quad(lambda r: r * ph(r) * (Gc(R + r) - Gc(abs(R - r))), 0, rmax, limit=2000,
                            epsrel=1e-11, points=[R])
    assert ihc[1] == pytest.approx(2 * math.pi / R * val, rel=1e-8)
    Gh = lambda s: integrate.quad(lambda t: t * ph(t), 0, s, epsrel=1e-12, limit=400)[0]
    val, _ = integrate.quad(lambda r: r * ph(r) * (Gh(R + r) - Gh(abs(R - r))), 0, 300.0, limit=400,
                            epsrel=1e-9, points=[R])
    assert ihh[1] == pytest.approx(2 * math.pi / R * val, rel=1e-7)


def _two_charge_problem(kappa, q=(0.7, -0.3), sep=(2.0, 1.0, -1.5), qs=(0.8, -0.5)):
    return O.Problem(xyz=np.array([[0.0, 0.0, 0.0], list(sep)]), q=np.array(q), sigma=np.array([2.0, 2.0]),
                     eps=np.array([0.1, 0.1]), qs=np.array(qs), sigs=np.array([3.0, 1.0]),
                     epss=np.array([0.1, 0.01]), rho=np.array([0.03, 0.06]), is_ion=np.array([0, 0], dtype=np.int32),
                     n=(4, 4, 4), h=0.5, origin=(0.0, 0.0, 0.0), kappa=kappa)


def test_lra_integral_against_grid_integration():
    """T_s, the all-space integral of [1/2 (h^lr)^2 Theta(Q q_s) - 1/2 h^lr c^lr], against a direct 3D grid
    sum of that integrand built from the oracle's real-space fields (eqs. (tcf-r), (dcf-r)), for two charges
    with a strong screening (kappa = 0.6 / A) so that a 64 A box holds the integrand; the integrand is smooth,
    so the grid sum converges spectrally.  One site has Q q_s > 0 (the squared term counts), one has Q q_s < 0."""
    kap = 0.6
    p = _two_charge_problem(kap)
    T, _ = O.lra_integral(p)
    h, L = 0.4, 32.0
    n = int(2 * L / h)
    origin = (-L + 1.0, -L + 0.5, -L)
    g = O.Problem(**{**p.__dict__, "n": (n, n, n), "h": h, "origin": origin})
    f = O.fields(g, want=("c", "h"))
    Q = float(np.sum(p.q))
    for s in range(p.nsite):
        theta = 1.0 if Q * p.qs[s] > 0 else 0.0
        integrand = 0.5 * theta * f["h"][s] ** 2 - 0.5 * f["h"][s] * f["c"][s]
        assert T[s] == pytest.approx(float(integrand.sum()) * h ** 3, rel=2e-6), s
    assert (Q * p.qs[0] > 0) != (Q * p.qs[1] > 0)


def test_lra_integral_invariants():
    """T is quadratic in the solute charges, invariant under a rigid motion of the solute, zero without
    ionic screening, and its squared term switches with the sign of Q q_s."""
    p = _two_charge_problem(KAPPA)
    T, (shh, shc) = O.lra_integral(p)
    T2, _ = O.lra_integral(O.Problem(**{**p.__dict__, "q": 3.0 * p.q}))
    np.testing.assert_allclose(T2, 9.0 * T, rtol=1e-13)
    rot = np.array([[0.0, -1.0, 0.0], [1.0, 0.0, 0.0], [0.0, 0.0, 1.0]])
    T3, _ = O.lra_integral(O.Problem(**{**p.__dict__, "xyz": p.xyz @ rot.T + np.array([5.0, -3.0, 7.0])}))
    np.testing.assert_allclose(T3, T, rtol=1e-12)
    T0, _ = O.lra_integral(O.Problem(**{**p.__dict__, "kappa": 0.0}))
    assert np.all(T0 == 0.0)
    Tneg, _ = O.lra_integral(O.Problem(**{**p.__dict__, "qs": -p.qs}))
    beta = O.beta(p)
    for s in range(p.nsite):
        A = -beta * p.k_e * p.qs[s] / (2 * p.eps_r)
        # flipping q_s flips Theta(Q q_s): the difference is the squared term
        sq = 0.5 * A * A * shh
        assert abs(T[s] - Tneg[s]) == pytest.approx(sq, rel=1e-12)


# ---------------------------------------------- reciprocal-space asymptotics
def _kspace_problem(kappa, n=(40, 37, 36), h=0.5, eta=2.0):
    """Two opposite charges off-lattice, an ionic and a water-like site, an odd and an even grid axis."""
    return O.Problem(xyz=np.array([[0.37, -0.81, 0.55], [2.13, 1.02, -1.44]]), q=np.array([0.9, -0.6]),
                     sigma=np.array([2.0, 2.0]), eps=np.array([0.1, 0.1]), qs=np.array([1.0, -0.4]),
                     sigs=np.array([2.0, 1.0]), epss=np.array([0.1, 0.01]), rho=np.array([0.03, 0.06]),
                     is_ion=np.array([1, 0], dtype=np.int32), n=n, h=h,
                     origin=tuple(-h * (v - 1) / 2.0 + 0.11 * (i + 1) for i, v in enumerate(n)), eta=eta, kappa=kappa)


def test_kspace_tcf_is_the_transform_of_the_real_space_tcf():
    """h_s(k) of eq. (tcf-k) on the grid's reciprocal lattice equals h^3 sum_j h_s^lr(o + h j) e^{+i k.(h j)}
    over the real-space samples of eq. (tcf-r) (the complex conjugate of numpy's forward rfftn, whose frequency
    layout the half spectrum follows): this fixes the sign of the phase, the origin, the lattice, the FFT order
    (one odd axis) and the 4 pi / (eps_r (k^2 + kappa^2)) Gaussian factor.  Strong screening and eta = 2 A make
    the truncated, sampled sum converge to the continuous transform."""
    p = _kspace_problem(kappa=0.6, n=(128, 121, 120))
    nx, ny, nz = p.n
    real = O.fields(p, want=("h",))["h"]
    ks = O.kspace(p, want=("c", "h"))
    for s in range(p.nsite):
        dft = np.conj(np.fft.rfftn(real[s].reshape(nz, ny, nx))) * p.h ** 3
        got = ks["h"][s].reshape(nz, ny, nx // 2 + 1)
        scale = np.abs(got).max()
        assert np.abs(got - dft).max() <= 2e-7 * scale, (s, np.abs(got - dft).max() / scale)


def test_kspace_dcf_against_tcf_and_at_k0():
    """c_s(k)/h_s(k) = eps_r (k^2 + kappa^2)/k^2 at every k != 0 (eq. (dcf-k) vs eq. (tcf-k)); c_s(0) = 0,
    h_s(0) = -(4 pi beta k_e q_s / (eps_r kappa^2)) sum_a Q_a."""
    p = _kspace_problem(kappa=0.3)
    nx, ny, nz = p.n
    ks = O.kspace(p)
    jx, jy, jz = np.meshgrid(np.arange(nx // 2 + 1), np.arange(ny), np.arange(nz), indexing="xy")
    f = np.fft.fftfreq
    kx = 2 * np.pi * np.arange(nx // 2 + 1) / (nx * p.h)
    ky = 2 * np.pi * f(ny, d=p.h)
    kz = 2 * np.pi * f(nz, d=p.h)
    k2 = (kz[:, None, None] ** 2 + ky[None, :, None] ** 2 + kx[None, None, :] ** 2).ravel()
    nz0 = k2 > 0
    for s in range(p.nsite):
        c, hh = ks["c"][s], ks["h"][s]
        np.testing.assert_allclose(c[nz0], hh[nz0] * p.eps_r * (k2[nz0] + 0.09) / k2[nz0], rtol=1e-12, atol=0)
        assert c[0] == 0.0
        h0 = -4 * np.pi * O.beta(p) * p.k_e * p.qs[s] / (p.eps_r * 0.09) * p.q.sum()
        assert hh[0] == pytest.approx(h0, rel=1e-13)


def test_kspace_translation_phase():
    """Moving the solute by a lattice vector t multiplies every entry by e^{i k.t}."""
    p = _kspace_problem(kappa=0.3, eta=1.0)
    t = np.array([3, -2, 5]) * p.h
    a = O.kspace(p)["c"][0]
    b = O.kspace(O.Problem(**{**p.__dict__, "xyz": p.xyz + t}))["c"][0]
    nx, ny, nz = p.n
    kx = 2 * np.pi * np.arange(nx // 2 + 1) / (nx * p.h)
    ky = 2 * np.pi * np.fft.fftfreq(ny, d=p.h)
    kz = 2 * np.pi * np.fft.fftfreq(nz, d=p.h)
    kt = (kz[:, None, None] * t[2] + ky[None, :, None] * t[1] + kx[None, None, :] * t[0]).ravel()
    np.testing.assert_allclose(b, a * np.exp(1j * kt), rtol=1e-12, atol=1e-12 * np.abs(a).max())


def test_kspace_cutoff_bound_and_root():
    """The cut-off wave number solves eq. (k-space-dcf-err) = tol (the bound decreases in k), every kept entry
    lies within it, every dropped entry is zero, and no dropped entry of the full sum exceeds the bound."""
    p = _kspace_problem(kappa=0.3, eta=1.0, n=(32, 30, 28))
    ks_full = O.kspace(p)
    tol = 1e-2 * float(np.abs(ks_full["c"]).max())
    kc = O.kspace_kcut(p, tol)
    assert O.kspace_bound(p, kc) == pytest.approx(tol, rel=1e-12)
    ks = np.linspace(0.2, 8.0, 50)
    b = np.array([O.kspace_bound(p, k) for k in ks])
    assert np.all(np.diff(b) < 0)
    cut = O.kspace(p, kcut=kc)
    nx, ny, nz = p.n
    kx = 2 * np.pi * np.arange(nx // 2 + 1) / (nx * p.h)
    ky = 2 * np.pi * np.fft.fftfreq(ny, d=p.h)
    kz = 2 * np.pi * np.fft.fftfreq(nz, d=p.h)
    k2 = (kz[:, None, None] ** 2 + ky[None, :, None] ** 2 + kx[None, None, :] ** 2).ravel()
    keep = k2 <= kc * kc
    assert 0 < keep.sum() < keep.size
    for key in ("c", "h"):
        np.testing.assert_array_equal(cut[key][:, keep], ks_full[key][:, keep])
        assert np.all(cut[key][:, ~keep] == 0)
        assert np.abs(ks_full[key][:, ~keep]).max() <= tol


# --------------------------------------------------- Taylor recurrences
@pytest.mark.parametrize("kind", ["coulomb", "erf", "yukawa"])
def test_taylor_recurrences_against_exact_derivatives(kind):
    """The recurrence coefficients against (1/k!) d^k/dy^k phi by 30-digit numerical differentiation, for every
    |k| <= 5 at two separations (a wrong factor, sign, index shift or auxiliary normalization fails)."""
    mp.mp.dps = 30
    eta, kap = 1.3, 0.35
    phi = {"coulomb": lambda r: 1 / r, "erf": lambda r: mp.erf(r / eta) / r,
           "yukawa": lambda r: mp.e ** (-kap * r) / r}[kind]
    P = 5
    for x, y in (((3.1, -1.7, 2.3), (0.4, 0.9, -0.6)), ((0.5, 4.0, -1.0), (-1.2, 0.3, 0.8))):
        a = O.taylor_coeffs(kind, P, [x[i] - y[i] for i in range(3)], eta, kap)
        X = [mp.mpf(v) for v in x]
        for n in range(P + 1):
            for k1 in range(n + 1):
                for k2 in range(n - k1 + 1):
                    k3 = n - k1 - k2
                    f = lambda y1, y2, y3: phi(mp.sqrt((X[0] - y1) ** 2 + (X[1] - y2) ** 2 + (X[2] - y3) ** 2))
                    d = mp.diff(f, tuple(mp.mpf(v) for v in y), (k1, k2, k3))
                    ex = float(d / (mp.factorial(k1) * mp.factorial(k2) * mp.factorial(k3)))
                    got = a[O.taylor_index(k1, k2, k3)]
                    assert got == pytest.approx(ex, rel=1e-10, abs=1e-13 * abs(a[0])), (kind, k1, k2, k3)


@pytest.mark.parametrize("kind", ["coulomb", "erf", "yukawa"])
def test_taylor_approximation_converges_to_direct_sum(kind):
    """Eq. (taylor_approximation) for a cluster of targets and well-separated sources: the error against the
    direct sum falls geometrically with the order, at the rate of the separation ratio."""
    rng = np.random.default_rng(3)
    eta, kap = 1.0, 0.3
    center = np.array([0.0, 0.0, 0.0])
    pts = rng.uniform(-1.0, 1.0, size=(40, 3))            # targets within r = sqrt(3) of the centre
    src = rng.uniform(-1.5, 1.5, size=(25, 3)) + np.array([9.0, -4.0, 3.0])
    q = rng.normal(0, 1, 25)
    d = np.linalg.norm(pts[:, None, :] - src[None, :, :], axis=2)
    from scipy.special import erf
    phi = {"coulomb": 1 / d, "erf": erf(d / eta) / d, "yukawa": np.exp(-kap * d) / d}[kind]
    direct = phi @ q
    errs = [np.abs(O.taylor_eval(kind, p, center, src, q, pts, eta, kap) - direct).max() / np.abs(direct).max()
            for p in (2, 4, 6, 8, 10)]
    assert all(b < a for a, b in zip(errs, errs[1:])), errs
    assert errs[-1] < 1e-8 and errs[0] / errs[-1] > 1e4, errs
