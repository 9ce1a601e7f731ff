"""Pins of the FP64 oracle against what the paper and the mathematics fix.

Each test checks the oracle against something other than itself: values the
paper prints, closed forms, brute-force Ewald summation, a dense
pseudo-inverse, finite differences and conservation laws.  None needs a GPU.
"""
import math

import numpy as np
import pytest

from oracle import p3maze_oracle as O
from paper_2606_31379_b300 import synth as S
from tests.golden_io import read_golden


# ---------------------------------------------------------------- parameters
def test_sigma_alpha_pair_printed_in_paper():
    g = read_golden("screening_width.txt")
    assert O.sigma_of_alpha(g["beta"]) == pytest.approx(g["sigma"], abs=5e-4)


def test_spcfw_table_matches_table_s1():
    g = read_golden("spcfw_table_s1.txt")
    p = S.spcfw_params()
    for k in ("eps_oo", "sigma_oo", "q_o", "q_h", "r0", "kb", "ka"):
        assert p[k] == g[k]
    assert math.degrees(p["theta0"]) == pytest.approx(g["theta0_deg"], abs=1e-12)


def test_smoothing_schedule_values():
    # alpha = 0.30 -> sigma^2 = 1/(2 alpha^2) = 5.5556; L = 25.2, N = 32 -> h = 0.7875
    K, c = O.smoothing_schedule(O.sigma_of_alpha(0.30), 25.2 / 32)
    assert K == 25 and 0.0 < c <= 1.0 / 6.0
    # total added per-axis variance equals sigma^2 - 4 h^2/6
    h = 25.2 / 32
    assert 2 * K * c * h * h == pytest.approx(1 / (2 * 0.09) - 4 * h * h / 6, rel=1e-14)
    assert O.smoothing_schedule(0.1, 1.0) == (0, 0.0)


# ---------------------------------------------------------------- B-splines
def _cardinal_bspline(x, order):
    """Cox-de Boor recursion for the cardinal B-spline M_order on [0, order)."""
    if order == 1:
        return np.where((x >= 0) & (x < 1), 1.0, 0.0)
    return (x * _cardinal_bspline(x, order - 1)
            + (order - x) * _cardinal_bspline(x - 1, order - 1)) / (order - 1)


def test_bspline_weights_match_recursion_and_moments():
    t = np.random.default_rng(0).uniform(0, 1, 1000)
    w = O.bspline4_weights(t)
    for k in range(4):
        # node floor(u)-1+k sits at distance t+1-k below u; M_4 centred at 2
        np.testing.assert_allclose(w[:, k], _cardinal_bspline(t + 3 - k, 4), atol=1e-15)
    offs = np.arange(4)[None, :] - 1 - t[:, None]
    np.testing.assert_allclose(w.sum(1), 1.0, atol=1e-15)
    np.testing.assert_allclose((w * offs).sum(1), 0.0, atol=1e-15)
    np.testing.assert_allclose((w * offs ** 2).sum(1), 1.0 / 3.0, atol=1e-14)


def test_assignment_moments_single_charge():
    n, box = 16, 16.0
    pos = np.array([[7.3, 8.91, 6.02]])
    q = O.assign_charges(pos, np.array([0.7]), box, n)
    assert q.sum() == pytest.approx(0.7, abs=1e-15)
    idx = np.arange(n, dtype=float)
    for ax in range(3):
        marg = q.sum(axis=tuple(a for a in range(3) if a != ax))
        m1 = (marg * idx).sum() / 0.7
        assert m1 == pytest.approx(pos[0, ax], abs=1e-13)
        assert ((marg * (idx - m1) ** 2).sum() / 0.7) == pytest.approx(1.0 / 3.0, abs=1e-13)


# ---------------------------------------------------------------- smoothing
def test_smoothing_conserves_charge_and_adds_closed_form_variance():
    # box wide enough (> 20 sigma) that the periodic tails do not overlap
    n, box = 64, 50.4
    h = box / n
    sigma = O.sigma_of_alpha(0.30)
    K, c = O.smoothing_schedule(sigma, h)
    pos = np.array([[24.1, 23.7, 26.05]])
    q = O.assign_charges(pos, np.array([1.0]), box, n)
    qs = O.smooth(q, K, c)
    assert qs.sum() == pytest.approx(1.0, abs=1e-13)
    assert qs.min() >= 0.0                     # c <= 1/6: positivity preserved
    x = np.arange(n) * h
    for ax in range(3):
        marg = qs.sum(axis=tuple(a for a in range(3) if a != ax))
        m1 = (marg * x).sum()
        var = (marg * (x - m1) ** 2).sum()
        assert m1 == pytest.approx(pos[0, ax], abs=1e-9)
        # assignment h^2/3 plus diffusion sigma^2 - 4h^2/6  =  sigma^2 - h^2/3
        assert var == pytest.approx(sigma * sigma - h * h / 3.0, rel=1e-9)
    np.testing.assert_array_equal(O.smooth(q, 0, 0.1), q)


# ---------------------------------------------------------------- Laplacian / solve
def test_laplacian_acts_on_fourier_modes_with_closed_form_eigenvalue():
    n = 12
    g = np.indices((n, n, n))
    for k in [(1, 0, 0), (2, 3, 5), (6, 6, 6), (0, 0, 0)]:
        mode = np.cos(2 * np.pi * (k[0] * g[0] + k[1] * g[1] + k[2] * g[2]) / n)
        lam = sum(2 * math.cos(2 * math.pi * ki / n) - 2 for ki in k)
        np.testing.assert_allclose(O.laplacian7(mode), lam * mode, atol=1e-12)


def _dense_M(n):
    size = n ** 3
    M = np.zeros((size, size))
    lin = lambda x, y, z: ((x % n) * n + (y % n)) * n + (z % n)
    for x in range(n):
        for y in range(n):
            for z in range(n):
                i = lin(x, y, z)
                M[i, i] -= 6
                for dx, dy, dz in ((1, 0, 0), (-1, 0, 0), (0, 1, 0), (0, -1, 0), (0, 0, 1), (0, 0, -1)):
                    M[i, lin(x + dx, y + dy, z + dz)] += 1
    return M


@pytest.mark.parametrize("n", [4, 6])
def test_fft_solve_matches_dense_pseudo_inverse(n):
    rng = np.random.default_rng(n)
    qs = rng.standard_normal((n, n, n))
    qs -= qs.mean()
    h = 0.8
    phi = O.solve_constraint_fft(qs, h)
    ref = -(4 * np.pi / h) * (np.linalg.pinv(_dense_M(n)) @ qs.reshape(-1))
    np.testing.assert_allclose(phi.reshape(-1), ref, atol=1e-11 * np.abs(ref).max())
    # and it satisfies the constraint of Eq. 13 with the stencil operator
    np.testing.assert_allclose(h / (4 * np.pi) * O.laplacian7(phi) + qs, 0.0, atol=1e-13)
    assert abs(phi.mean()) < 1e-13


# ---------------------------------------------------------------- Madelung / Ewald
def test_ewald_reproduces_madelung_constant():
    M = read_golden("madelung_nacl.txt")["madelung"]
    cr = S.rocksalt_crystal(5.64, 1)
    e, F = O.ewald(cr.pos, cr.charge, cr.box, 1.0, ke=1.0)
    assert -e * (5.64 / 2) / (cr.n / 2) == pytest.approx(M, abs=1e-6)
    assert np.abs(F).max() < 1e-10


def test_p3maze_energy_converges_to_madelung_as_h_squared():
    """Narrow screening (sigma = 0.7 A) so the mesh part carries a large share
    of the crystal's energy; real-space cutoff where erfc < 1e-12."""
    M = read_golden("madelung_nacl.txt")["madelung"]
    cr = S.rocksalt_crystal(5.64, 1)
    alpha = 1.0 / (math.sqrt(2) * 0.7)
    errs = []
    for n in (16, 32, 64):
        out = O.forces_and_energies(cr, alpha, 5.5, n, ke=1.0)
        m = -out["v_coul"] * (5.64 / 2) / (cr.n / 2)
        errs.append(abs(m - M) / M)
        assert out["v_lr"] > 0.5 * abs(out["v_coul"])       # the mesh term matters here
    assert errs[2] < 1.2e-3
    assert errs[0] / errs[1] > 2.5 and errs[1] / errs[2] > 3.0
    # Eq. 14 taken literally (1/2 phi^T q^s) double counts the smear: rejected
    lit = O.forces_and_energies(cr, alpha, 5.5, 32, ke=1.0, lr_energy="smoothed")
    assert abs(-lit["v_coul"] * (5.64 / 2) / (cr.n / 2) - M) / M > 0.1


def test_p3maze_forces_converge_to_brute_force_ewald():
    sysr = S.random_neutral(8, 12.0, seed=11, dmin=1.5)
    alpha = 0.5
    e_ref, F_ref = O.ewald(sysr.pos, sysr.charge, sysr.box, alpha, ke=1.0)
    # the Ewald reference does not depend on its splitting parameter
    e2, F2 = O.ewald(sysr.pos, sysr.charge, sysr.box, 0.8, ke=1.0)
    assert e2 == pytest.approx(e_ref, rel=1e-12)
    ferr, eerr = [], []
    for n in (16, 32, 64):
        out = O.forces_and_energies(sysr, alpha, 10.5, n, ke=1.0)
        ferr.append(np.sqrt(((out["F"] - F_ref) ** 2).sum() / (F_ref ** 2).sum()))
        eerr.append(abs(out["v_coul"] - e_ref) / abs(e_ref))
        # Newton III for both parts (momentum conservation, Sec. 2)
        assert np.abs(out["F_sr"].sum(0)).max() < 1e-14
        assert np.abs(out["F_lr"].sum(0)).max() < 1e-14
    assert ferr[2] < 2e-3 and eerr[2] < 1e-3
    assert ferr[0] / ferr[1] > 3.0 and ferr[1] / ferr[2] > 3.0


# ---------------------------------------------------------------- short range
def _fd_check(system, energy_fn, force, h=1e-5, rtol=1e-7, atol=1e-9):
    rng = np.random.default_rng(5)
    for i in rng.choice(system.n, 4, replace=False):
        for d in range(3):
            p0 = system.pos[i, d]
            system.pos[i, d] = p0 + h
            ep = energy_fn(system)
            system.pos[i, d] = p0 - h
            em = energy_fn(system)
            system.pos[i, d] = p0
            fd = -(ep - em) / (2 * h)
            assert fd == pytest.approx(force[i, d], rel=rtol, abs=atol)


def test_sr_forces_are_minus_gradient_of_sr_energy():
    s = S.nacl_melt(24, 11.0, seed=3, dmin=2.0)
    sigma = O.sigma_of_alpha(0.30)
    rc = 9.0                                  # > L/2: several images contribute

    def energy(sys_):
        _, ec, ev = O.sr_forces(sys_, sigma, rc)
        return ec.sum() + ev.sum()

    F, _, _ = O.sr_forces(s, sigma, rc)
    assert np.abs(F.sum(0)).max() < 1e-9 * np.abs(F).max()
    _fd_check(s, energy, F)


def test_sr_virial_is_the_scaling_derivative_of_the_sr_energy():
    """The short-range pair virial W = sum_{i<j} r_ij . F_ij.  For one pair it
    is -r dU/dr, with dU/dr by a central difference of the pair energy.  For
    a melt with the shifted-force cutoff (energy and force continuous at R_c)
    it is -dV/dlambda at lambda = 1, every position and the box scaled by
    lambda.  A wrong sign, a lost factor 1/2 (the double count) or a missing
    term fails both."""
    import dataclasses
    sigma = O.sigma_of_alpha(0.30)
    rc = 9.0
    pair = S.nacl_melt(2, 30.0, seed=0)
    r0 = 3.1

    def u(r):
        sys_ = dataclasses.replace(pair, pos=np.array([[5.0, 5.0, 5.0], [5.0 + r, 5.0, 5.0]]))
        _, ec, ev = O.sr_forces(sys_, sigma, rc)
        return ec.sum() + ev.sum()

    one = dataclasses.replace(pair, pos=np.array([[5.0, 5.0, 5.0], [5.0 + r0, 5.0, 5.0]]))
    _, _, _, w = O.sr_forces(one, sigma, rc, virial=True)
    dudr = (u(r0 + 1e-5) - u(r0 - 1e-5)) / 2e-5
    assert w.sum() == pytest.approx(-r0 * dudr, rel=1e-7)
    assert w[0] == pytest.approx(w[1], rel=1e-12)           # each particle carries half
    m = S.nacl_melt(24, 11.0, seed=3, dmin=2.0)

    def v(lam):
        sys_ = dataclasses.replace(m, pos=m.pos * lam, box=m.box * lam)
        _, ec, ev = O.sr_forces(sys_, sigma, rc, shift="force")
        return ec.sum() + ev.sum()

    _, _, _, w = O.sr_forces(m, sigma, rc, shift="force", virial=True)
    dv = (v(1.0 + 1e-6) - v(1.0 - 1e-6)) / 2e-6
    assert w.sum() == pytest.approx(-dv, rel=1e-6)
    ref = O.forces_and_energies(m, 0.30, rc, 16, sr_shift="force")
    assert ref["w_sr"] == pytest.approx(w.sum(), rel=1e-12)


def test_lj_pair_closed_form_zero_minimum_and_force():
    """Lennard-Jones (SPC/Fw O-O term, Table S1): U(sigma) = 0, the minimum sits
    at r = 2^(1/6) sigma with depth -eps (textbook values), and the returned
    force is -dU/dr (central differences of the energy, step 1e-6 A)."""
    eps, sig = 0.1554253, 3.165492
    e0, f0 = O.lj_pair(np.array([sig]), eps, sig)
    assert e0[0] == pytest.approx(0.0, abs=1e-15)
    rmin = 2.0 ** (1.0 / 6.0) * sig
    e1, f1 = O.lj_pair(np.array([rmin]), eps, sig)
    assert e1[0] == pytest.approx(-eps, rel=1e-14)
    assert abs(f1[0]) < 1e-12
    r = np.linspace(2.8, 9.0, 23)
    h = 1e-6
    _, fr = O.lj_pair(r, eps, sig)
    fd = -(O.lj_pair(r + h, eps, sig)[0] - O.lj_pair(r - h, eps, sig)[0]) / (2 * h)
    np.testing.assert_allclose(fr * r, fd, rtol=1e-7, atol=1e-12)


def test_bmh_pair_force_is_minus_derivative():
    t = S.nacl_melt(2, 10.0, seed=0).sr_table
    r = np.linspace(2.0, 9.0, 15)
    h = 1e-6
    for i, j in ((0, 0), (0, 1), (1, 1)):
        args = (t["A"][i, j], t["rho"][i, j], t["sigma"][i, j], t["C"][i, j], t["D"][i, j])
        _, fr = O.bmh_pair(r, *args)
        fd = -(O.bmh_pair(r + h, *args)[0] - O.bmh_pair(r - h, *args)[0]) / (2 * h)
        np.testing.assert_allclose(fr * r, fd, rtol=1e-7, atol=1e-10)


def test_sr_forces_with_lj_pairs_are_minus_gradient():
    """Two SPC/Fw molecules in a small box with their oxygens within R_c: the
    short-range force (erfc Coulomb + O-O Lennard-Jones, intramolecular pairs
    excluded) is minus the gradient of the short-range energy."""
    w = S.spcfw_water(2, 8.0, seed=4)
    o = np.nonzero(w.charge < 0)[0]
    d = w.pos[o[0]] - w.pos[o[1]]
    d -= w.box * np.round(d / w.box)
    assert np.linalg.norm(d) < 6.0
    sigma = O.sigma_of_alpha(0.30)
    rc = 6.0

    def energy(sys_):
        _, ec, ev = O.sr_forces(sys_, sigma, rc)
        return ec.sum() + ev.sum()

    F, _, ev = O.sr_forces(w, sigma, rc)
    assert abs(ev.sum()) > 1e-4                 # the LJ term is present
    assert np.abs(F.sum(0)).max() < 1e-9 * np.abs(F).max()
    _fd_check(w, energy, F, rtol=1e-6)


def test_shifted_force_cutoff_is_continuous_and_conservative():
    """The shifted-force option: every term and its force vanish at R_c, the
    energy approaches zero quadratically (a wrong linear term would leave a
    first-order step), and the summed forces are minus the gradient of the
    summed shifted energies (BMH melt and SPC/Fw with LJ)."""
    sigma = O.sigma_of_alpha(0.30)
    rc = 9.0
    t = S.nacl_melt(2, 10.0, seed=0).sr_table
    w = S.spcfw_params()
    cases = [(O.sr_coulomb_pair, (np.float64(-1.0), sigma, 332.0637)),
             (O.bmh_pair, (t["A"][0, 1], t["rho"][0, 1], t["sigma"][0, 1], t["C"][0, 1], t["D"][0, 1])),
             (O.lj_pair, (w["eps_oo"], w["sigma_oo"]))]
    for fn, args in cases:
        e, fr = O.shift_force(fn, np.array([rc]), rc, *args)
        assert e[0] == 0.0 and fr[0] == 0.0
        d = np.array([1e-2, 1e-3])
        e, _ = O.shift_force(fn, rc - d, rc, *args)
        scale = abs(fn(np.array([rc]), *args)[1][0]) * rc   # |F(r_c)|
        assert np.all(np.abs(e) < 10 * scale * d)              # no first-order step ...
        assert abs(e[1]) < 0.02 * abs(e[0]) + 1e-18           # ... it falls as d^2
        e_plain, _ = fn(rc - d, *args)
        assert np.any(np.abs(e_plain - e) > 0)                 # the shift is applied
    s = S.nacl_melt(24, 11.0, seed=3, dmin=2.0)

    def energy(sys_):
        _, ec, ev = O.sr_forces(sys_, sigma, rc, shift="force")
        return ec.sum() + ev.sum()

    F, _, _ = O.sr_forces(s, sigma, rc, shift="force")
    F0, _, _ = O.sr_forces(s, sigma, rc)
    assert np.abs(F - F0).max() > 1e-8 * np.abs(F0).max()
    assert np.abs(F.sum(0)).max() < 1e-9 * np.abs(F).max()
    _fd_check(s, energy, F)
    ww = S.spcfw_water(2, 8.0, seed=4)

    def energy_w(sys_):
        _, ec, ev = O.sr_forces(sys_, sigma, 6.0, shift="force")
        return ec.sum() + ev.sum()

    Fw, _, _ = O.sr_forces(ww, sigma, 6.0, shift="force")
    _fd_check(ww, energy_w, Fw, rtol=1e-6)


def test_spcfw_intramolecular_forces_are_minus_gradient():
    w = S.spcfw_water(8, 9.0, seed=2)
    sigma = O.sigma_of_alpha(0.30)

    def energy(sys_):
        _, eb, ea, ex = O.intramolecular_terms(sys_, sigma)
        return eb + ea + ex

    F, _, _, _ = O.intramolecular_terms(w, sigma)
    assert np.abs(F.sum(0)).max() < 1e-9 * np.abs(F).max()
    _fd_check(w, energy, F, rtol=1e-6)


def test_spcfw_exclusion_cancels_intramolecular_coulomb():
    """One water molecule alone in a large box, with no screening cutoff issue:
    the mesh pair kernel erf(r/sqrt2 sigma)/r minus the exclusion must leave no
    intramolecular Coulomb, so V_SR(intra) = 0 and V_excl = -sum QQ erf/r."""
    w = S.spcfw_water(1, 30.0, seed=0)
    sigma = 1.0
    _, _, _, ex = O.intramolecular_terms(w, sigma, ke=1.0)
    p, q = w.pos, w.charge
    ref = 0.0
    for i, j in ((0, 1), (0, 2), (1, 2)):
        r = np.linalg.norm(p[i] - p[j])
        ref -= q[i] * q[j] * math.erf(r / (math.sqrt(2) * sigma)) / r
    assert ex == pytest.approx(ref, rel=1e-14)
    F, ec, ev = O.sr_forces(w, sigma, 9.0, ke=1.0)
    assert np.abs(F).max() == 0.0 and ec.sum() == 0.0


# ---------------------------------------------------------------- cell list
def test_cell_list_covers_every_pair_within_cutoff():
    s = S.nacl_melt(400, 25.2, seed=1)
    rc = 9.0
    nc, cell, start, order = O.cell_list(s.pos, s.box, rc)
    assert nc == 5 and s.box / nc >= rc / 2
    # order sorted by (cell, index) and start offsets consistent
    assert np.all(np.diff(cell[order].astype(np.int64) * s.n + order) > 0)
    for c in range(nc ** 3):
        members = order[start[c]:start[c + 1]]
        assert np.all(cell[members] == c)
    # every pair within R_c sits in cells at most 2 apart along each axis (mod nc)
    c3 = np.stack([cell % nc, (cell // nc) % nc, cell // (nc * nc)], 1)
    d = s.pos[:, None, :] - s.pos[None, :, :]
    d -= s.box * np.round(d / s.box)
    close = (d ** 2).sum(-1) < rc * rc
    i, j = np.nonzero(close)
    dc = np.abs(c3[i] - c3[j])
    dc = np.minimum(dc, nc - dc)
    assert dc.max() <= 2


# ---------------------------------------------------------------- integrator
def test_velocity_verlet_is_second_order():
    """Energy error of velocity Verlet shrinks as dt^2 (SI Sec. 1).  Screened
    Coulomb only, cutoff where erfc(alpha r) < 1e-15 so the force is the exact
    gradient of the energy."""
    def run(dt):
        s = S.random_neutral(6, 10.0, seed=4, dmin=2.5)
        sigma, rc = O.sigma_of_alpha(1.0), 6.0

        def ff(sys_):
            F, ec, _ = O.sr_forces(sys_, sigma, rc, vdw=False)
            return {"F": F, "v_pot": ec.sum()}

        out = ff(s)
        e0 = out["v_pot"] + O.kinetic_energy(s.vel, s.mass)
        F = out["F"]
        err = 0.0
        for _ in range(int(round(40 / dt))):
            out = O.velocity_verlet_step(s, F, dt, ff)
            F = out["F"]
            err = max(err, abs(out["v_pot"] + O.kinetic_energy(s.vel, s.mass) - e0))
        assert np.all((s.pos >= 0) & (s.pos < s.box))
        return err

    e1, e2 = run(2.0), run(1.0)
    assert 3.0 < e1 / e2 < 5.0


# ------------------------------------------------------------------ multigrid
def test_multigrid_converges_to_the_pseudo_inverse():
    """The oracle's V-cycle iteration (red-black Gauss-Seidel 2+2, full
    weighting x4, trilinear, exact coarse level) reaches the FFT
    pseudo-inverse solution, and each V-cycle reduces the max-norm residual
    by at least 5x on a random zero-mean right-hand side (textbook multigrid
    for the 7-point Poisson operator reduces by about 10x)."""
    rng = np.random.default_rng(0)
    for n, cmax in ((32, 16), (64, 16), (24, 8)):
        b = rng.standard_normal((n, n, n))
        b -= b.mean()
        y, it, hist = O.mg_correction_solve(b, np.zeros_like(b), 1e-10, O.mg_levels(n, cmax))
        assert hist[-1] <= 1e-10 and it <= 15
        assert all(hist[k + 1] <= 0.2 * hist[k] for k in range(len(hist) - 1))
        ex = O.pseudo_inverse_solve(b)
        assert np.abs(O.laplacian7(ex) - b).max() < 1e-12        # the pseudo-inverse itself
        assert np.abs((y - y.mean()) - ex).max() < 1e-9


def test_multigrid_levels_and_exact_coarse_level():
    assert O.mg_levels(128, 64) == [128, 64]
    assert O.mg_levels(128, 16) == [128, 64, 32, 16]
    assert O.mg_levels(384, 64) == [384, 192, 96, 48]
    assert O.mg_levels(60, 64) == [60]
    assert O.mg_levels(36, 8) == [36, 18, 9]
    # a single exact level solves in one cycle
    rng = np.random.default_rng(1)
    b = rng.standard_normal((12, 12, 12))
    b -= b.mean()
    _, it, hist = O.mg_correction_solve(b, np.zeros_like(b), 1e-11, O.mg_levels(12, 64))
    assert it == 1 and hist[-1] < 1e-11


def test_restriction_is_the_scaled_adjoint_of_prolongation():
    """Full weighting is 1/8 of the transpose of trilinear interpolation:
    8 <R r, v> = <r, P v> (R without its factor 4)."""
    rng = np.random.default_rng(2)
    r = rng.standard_normal((16, 16, 16))
    v = rng.standard_normal((8, 8, 8))
    lhs = 8.0 * np.sum(O.restrict_full_weighting(r) / 4.0 * v)
    rhs = np.sum(r * O.prolong_trilinear(v))
    assert lhs == pytest.approx(rhs, rel=1e-13)
    # constants are reproduced: P 1 = 1, R 1 = 4 (the x4 rescaling)
    assert np.allclose(O.prolong_trilinear(np.ones((8, 8, 8))), 1.0)
    assert np.allclose(O.restrict_full_weighting(np.ones((16, 16, 16))), 4.0)


# ------------------------------------------------------------------ analytic-gradient force option
def test_analytic_mesh_force_is_the_energy_gradient():
    """The analytic B-spline-gradient force equals -dV_LR/dr (central finite
    differences of V_LR = 1/2 ke phi*^T q, step 1e-5 A) to 1e-6 relative; the
    paper's finite-difference force (Eq. 21) is not the gradient of that
    energy (a few per cent off at this coarse mesh), which is why it does not
    conserve energy exactly."""
    s = S.random_neutral(8, 12.0, seed=3)
    n, alpha = 16, 0.6
    mf = O.mesh_fields(s, alpha, n)
    Fa = O.interpolate_lr_forces_analytic(s.pos, s.charge, s.box, n, mf["phi"])
    Ff = O.interpolate_lr_forces(s.pos, s.charge, s.box, n, mf["phi"])
    eps = 1e-5
    g = np.zeros((3, 3))
    for i in range(3):
        for d in range(3):
            p1, p2 = s.pos.copy(), s.pos.copy()
            p1[i, d] += eps
            p2[i, d] -= eps
            g[i, d] = -(O.lr_energy_at(p1, s.charge, s.box, alpha, n)
                        - O.lr_energy_at(p2, s.charge, s.box, alpha, n)) / (2 * eps)
    scale = np.abs(g).max()
    assert np.abs(Fa[:3] - g).max() < 1e-6 * scale
    assert np.abs(Ff[:3] - g).max() > 1e-2 * scale
    # Eq. 21's force sums to zero exactly (Newton III on the mesh)
    assert np.abs(Ff.sum(0)).max() < 1e-10 * np.abs(Ff).max()


def test_bspline_derivative_weights():
    t = np.linspace(0.0, 1.0, 11)
    d = O.bspline4_derivatives(t)
    assert np.allclose(d.sum(-1), 0.0, atol=1e-15)
    h = 1e-6
    fd = (O.bspline4_weights(t + h) - O.bspline4_weights(t - h)) / (2 * h)
    assert np.allclose(d, fd, atol=1e-8)


# ---------------------------------------------------------------- PMaZe
def test_pmaze_forces_converge_to_full_coulomb_ewald():
    """PMaZe puts the whole Coulomb problem on the mesh (Sec. 2): with no
    screening, the Eq. 21 force of the constrained full-charge potential must
    approach the brute-force Ewald force of the point charges as h^2, sum to
    zero (Newton III on the mesh), and its mesh energy must exceed the Ewald
    energy by a grid self-energy that scales as 1/h."""
    s = S.random_neutral(8, 12.0, seed=11, dmin=1.5)
    e_ref, F_ref = O.ewald(s.pos, s.charge, s.box, 0.5, ke=1.0)
    ferr, self_h = [], []
    for n in (32, 64, 128):
        out = O.pmaze_forces_and_energies(s, 6.0, n, ke=1.0)
        ferr.append(np.sqrt(((out["F"] - F_ref) ** 2).sum() / (F_ref ** 2).sum()))
        assert np.abs(out["F"].sum(0)).max() < 1e-12 * np.abs(out["F"]).max()
        self_h.append((out["v_mesh"] - e_ref) * (s.box / n))
    assert ferr[2] < 2e-3
    assert 3.0 < ferr[0] / ferr[1] < 5.0 and 3.0 < ferr[1] / ferr[2] < 5.0
    assert self_h[0] > 0.0 and abs(self_h[2] - self_h[1]) < 0.01 * self_h[2]


def test_pmaze_source_is_the_unsmoothed_assigned_charge():
    """The PMaZe potential solves the constraint with q itself: applying
    (h/4pi) M to it returns -(q - mean q) (Eq. 13 with q in place of q^s)."""
    s = S.random_neutral(6, 10.0, seed=4, dmin=1.5)
    n = 24
    f = O.pmaze_mesh_fields(s, n)
    q = O.assign_charges(s.pos, s.charge, s.box, n)
    back = (f["h"] / (4.0 * np.pi)) * O.laplacian7(f["phi"])
    assert np.abs(back + (q - q.mean())).max() < 1e-12 * np.abs(q).max()


def test_pmaze_rejects_molecules():
    w = S.spcfw_water(8, 6.3, seed=2)
    with pytest.raises(ValueError):
        O.pmaze_forces_and_energies(w, 3.0, 16)


# ---------------------------------------------------------------- O(N) forms used for timing
@pytest.mark.parametrize("kind", ["nacl", "nacl_small_box", "water", "nacl_shift"])
def test_cell_list_sr_sum_equals_all_pairs(kind):
    """sr_forces_cells finds the same pairs and images as the all-pairs
    definition sr_forces: forces and per-particle energies agree to rounding
    (a box below 2 R_c, molecules with excluded partners, the shifted form)."""
    sigma = O.sigma_of_alpha(0.30)
    shift = "none"
    if kind == "nacl":
        s, rc = S.nacl_melt(200, 25.2, seed=2), 9.0
    elif kind == "nacl_small_box":
        s, rc = S.nacl_melt(40, 11.5, seed=3), 9.0          # 2 cells per axis, L < 2 R_c
    elif kind == "water":
        s, rc = S.spcfw_water(27, 9.4, seed=5), 6.0
    else:
        s, rc, shift = S.nacl_melt(120, 21.0, seed=4), 9.0, "force"
    F, ec, ev = O.sr_forces(s, sigma, rc, shift=shift)
    Fc, ecc, evc = O.sr_forces_cells(s, sigma, rc, shift=shift)
    np.testing.assert_allclose(Fc, F, rtol=0, atol=1e-10 * np.abs(F).max())
    np.testing.assert_allclose(ecc, ec, rtol=0, atol=1e-10 * np.abs(ec).max())
    np.testing.assert_allclose(evc, ev, rtol=0, atol=1e-10 * max(np.abs(ev).max(), 1e-30))


def test_mass_zero_stepper_tracks_the_exactly_constrained_field():
    """maze_md_step (the plain FP64 Mass-Zero MD step) keeps the field on the
    constraint: after every step max|(h/4pi) M phi + q^s| <= tol at the new
    positions, and the trajectory equals velocity Verlet driven by the exact
    (FFT-constrained) forces up to the solver tolerance's effect."""
    s = S.nacl_melt(64, 14.0, seed=6)
    n, alpha, rc, dt, tol = 16, 0.45, 6.5, 1.0, 1e-10
    a = S.System(pos=O.wrap(s.pos, s.box), vel=s.vel.copy(), charge=s.charge, mass=s.mass, types=s.types,
                 box=s.box, sr_kind=s.sr_kind, sr_table=s.sr_table)
    b = S.System(pos=a.pos.copy(), vel=a.vel.copy(), charge=s.charge, mass=s.mass, types=s.types,
                 box=s.box, sr_kind=s.sr_kind, sr_table=s.sr_table)
    state = O.maze_initial_state(a, alpha, rc, n)

    def exact(sys_):
        return O.forces_and_energies(sys_, alpha, rc, n)

    Fb = exact(b)["F"]
    iters = []
    for _ in range(5):
        iters.append(O.maze_md_step(a, state, alpha, rc, n, dt, tol))
        out = O.velocity_verlet_step(b, Fb, dt, exact)
        Fb = out["F"]
        mf = O.mesh_fields(a, alpha, n)
        res = np.abs(mf["h"] / (4 * np.pi) * O.laplacian7(state["phi"]) + mf["qs"]).max()
        assert res <= tol * (1 + 1e-6)
    np.testing.assert_allclose(a.pos, b.pos, rtol=0, atol=1e-9)
    np.testing.assert_allclose(state["F"], Fb, rtol=0, atol=1e-6 * np.abs(Fb).max())
    assert max(iters) >= 1
