"""FP64 CPU oracle for the P3MaZe long-range electrostatics hot path.

TEST INFRASTRUCTURE ONLY.  This module is the plain, slow, obviously correct
statement of what the CUDA path computes.  It may be imported only by the
tests, by __graft_entry__.smoke() and by bench.py's CPU-baseline leg; the
product path never imports, links or runs it.  It shares no code with the
CUDA library (no kernels, helpers, tables or constants): inputs come from the
seeded generators, every formula is written out here from the paper.

Units: lengths in A, charges in e, energies in kcal/mol when ke = 332.0637
(ke = 1 gives Gaussian units e^2/A, used by the Madelung and Ewald pins).

What the method reaches, and what this oracle therefore computes, at a given
particle configuration (Sec. 2):
  q      = A(r) Q                        cubic B-spline assignment (Sec. 2, "Charge
                                         assignment and smoothing")
  q^s    = (I + c M)^K q - mean         diffusion smoothing; gauge fix
  phi*   = -(4 pi / h) M^+ q^s           the exactly constrained mesh potential,
                                         i.e. the solution of the constraint Eq. 13
                                         (equivalently the discrete Poisson Eq. 9),
                                         which the Mass-Zero prediction/correction
                                         (Eqs. 16-17) reaches to within tol
  F^LR   = -Q W . D phi*                 Eq. 21
  F^SR   = erfc-screened pair force      Eq. 19, plus the non-Coulomb term V-bar
  V      = V_SR + V_LR + V_self          Eqs. 5, 6, 14 (reading below)

Readings of the paper (each is also listed with its reason in the design notes):
  * Screening: the Ewald splitting alpha and the Gaussian width sigma are tied by
    alpha = 1/(sqrt(2) sigma) (Eq. 5 erfc argument; Sec. 3.1.1 prints
    sigma = 1.39 A <-> beta = 0.5087 A^-1).
  * Smoothing: K explicit diffusion steps q <- q + c M q on the 7-point stencil.
    One step adds per-axis variance 2 c h^2.  The total smear between a charge
    and the force on another charge must be sigma^2 per axis; assignment and
    interpolation (the same cubic B-spline, variance h^2/3 each) supply
    2 * p h^2/12, so the diffusion supplies sigma^2 - p h^2/6:
        kappa = (sigma^2 - p h^2 / 6) / (2 h^2),  K = ceil(6 kappa),  c = kappa/K
    (c <= 1/6 keeps the step positivity preserving).
  * Energy: with that smoothing, the long-range energy consistent with the
    force of Eq. 21 and with V_SR (Eq. 5) and V_self (Eq. 6) is
        V_LR = 1/2 phi*^T q   (q = assigned charge BEFORE smoothing).
    Taking Eq. 14 literally with q^s counts the diffusion smear twice; the
    Madelung and brute-force Ewald pins reject that reading.
  * Gauge: M is singular under periodicity; q^s has its mean removed and
    phi* has zero mean (Eq. 16 is solvable only for zero-mean right-hand sides).
  * Short range: pair terms are truncated at R_c without shifting; all
    periodic images within R_c are included (boxes with R_c <= L < 2 R_c).

The comparison method PMaZe (Secs. 1-2) is here too: the assigned charge q
itself is the source of the same constraint, Eq. 21 on that potential is the
whole electrostatic force, and pairs keep only the non-Coulomb term.

Parity pins: see tests/test_oracle_*.py (Madelung constant, brute-force Ewald,
dense pseudo-inverse, B-spline and smoothing moments, finite-difference forces,
Newton III).  Functions without an independent pin say so in their docstring.
"""
from __future__ import annotations

import math
import time

import numpy as np
from scipy.special import erfc as _erfc, erf as _erf

COULOMB_K = 332.0637          # kcal A / (mol e^2)
ACCEL = 4.184e-4              # (kcal/mol/A)/(g/mol) in A/fs^2


# ---------------------------------------------------------------------------
# Parameters
# ---------------------------------------------------------------------------
def sigma_of_alpha(alpha: float) -> float:
    """Gaussian width sigma for Ewald splitting alpha: alpha = 1/(sqrt(2) sigma).

    Eq. 5 writes the short-range kernel as erfc(r / (sqrt(2) sigma)); the
    paper's NaCl setup (Sec. 3.1.1) pairs sigma = 1.39 A with 0.5087 A^-1."""
    return 1.0 / (math.sqrt(2.0) * alpha)


def smoothing_schedule(sigma: float, h: float, order: int = 4) -> tuple[int, float]:
    """Number of diffusion steps K and coefficient c (reading of Sec. 2 /
    Sec. 3.1.1 "diffusion-based smoothing"): per-axis variance added by the
    diffusion is sigma^2 - order h^2/6, split into K steps of 2 c h^2 with
    c <= 1/6."""
    kappa = (sigma * sigma - order * h * h / 6.0) / (2.0 * h * h)
    if kappa <= 0.0:
        return 0, 0.0
    K = int(math.ceil(6.0 * kappa))
    return K, kappa / K


# ---------------------------------------------------------------------------
# Mesh operators
# ---------------------------------------------------------------------------
def bspline4_weights(t: np.ndarray) -> np.ndarray:
    """Cubic (order-4) B-spline weights for the four nodes floor(u)-1 .. floor(u)+2
    of a particle at fractional mesh coordinate u, t = u - floor(u) (Sec. 2,
    cubic B-spline charge assignment).  Returns array (..., 4)."""
    t = np.asarray(t, dtype=np.float64)
    s = 1.0 - t
    w0 = s * s * s / 6.0
    w1 = (3.0 * t ** 3 - 6.0 * t ** 2 + 4.0) / 6.0
    w2 = (-3.0 * t ** 3 + 3.0 * t ** 2 + 3.0 * t + 1.0) / 6.0
    w3 = t ** 3 / 6.0
    return np.stack([w0, w1, w2, w3], axis=-1)


def bspline4_derivatives(t: np.ndarray) -> np.ndarray:
    """d/dt of the four cubic B-spline weights (the derivative of each
    polynomial above); they sum to zero.  Returns array (..., 4)."""
    t = np.asarray(t, dtype=np.float64)
    s = 1.0 - t
    d0 = -0.5 * s * s
    d1 = 1.5 * t * t - 2.0 * t
    d2 = -1.5 * t * t + t + 0.5
    d3 = 0.5 * t * t
    return np.stack([d0, d1, d2, d3], axis=-1)


def assignment_stencil(pos: np.ndarray, box: float, n: int):
    """Base node index (floor(u) - 1) and per-axis weights for each particle.

    u = r * (n / L); returns base (np,3) int64 and w (np,3,4)."""
    inv_h = n / box
    u = pos * inv_h
    fl = np.floor(u)
    base = fl.astype(np.int64) - 1
    return base, bspline4_weights(u - fl)


def assign_charges(pos: np.ndarray, charge: np.ndarray, box: float, n: int) -> np.ndarray:
    """q_n = sum_a Q_a W(u_a - n): cubic B-spline assignment to the periodic
    mesh, array indexed [ix, iy, iz] (Sec. 2)."""
    base, w = assignment_stencil(pos, box, n)
    q = np.zeros((n, n, n))
    for a in range(4):
        ix = (base[:, 0] + a) % n
        for b in range(4):
            iy = (base[:, 1] + b) % n
            for c in range(4):
                iz = (base[:, 2] + c) % n
                np.add.at(q, (ix, iy, iz), charge * w[:, 0, a] * w[:, 1, b] * w[:, 2, c])
    return q


def laplacian7(f: np.ndarray) -> np.ndarray:
    """(M f)_n = sum of the six periodic nearest neighbours - 6 f_n: the
    dimensionless 7-point stencil (M/h^2 is the discrete Laplacian, Sec. 2)."""
    out = -6.0 * f
    for ax in range(3):
        out = out + np.roll(f, 1, axis=ax) + np.roll(f, -1, axis=ax)
    return out


def smooth(q: np.ndarray, K: int, c: float) -> np.ndarray:
    """q^s = (I + c M)^K q: K explicit diffusion steps (reading of Sec. 2)."""
    s = q.copy()
    for _ in range(K):
        s = s + c * laplacian7(s)
    return s


def laplacian_eigenvalues(n: int) -> np.ndarray:
    """Eigenvalues of M on the periodic n^3 mesh for the Fourier modes
    exp(2 pi i k.m/n): -4 sum_axes sin^2(pi k_axis / n)."""
    s = np.sin(np.pi * np.arange(n) / n) ** 2
    return -4.0 * (s[:, None, None] + s[None, :, None] + s[None, None, :])


def solve_constraint_fft(qs: np.ndarray, h: float) -> np.ndarray:
    """phi* with (h/4pi) M phi* + (q^s - mean q^s) = 0 and mean(phi*) = 0:
    the exact solution of the constraint Eq. 13 (the discrete Poisson Eq. 9)
    by diagonalising the circulant M with a library FFT."""
    n = qs.shape[0]
    lam = laplacian_eigenvalues(n)
    qhat = np.fft.fftn(qs)
    phihat = np.zeros_like(qhat)
    nz = lam != 0.0
    phihat[nz] = -(4.0 * np.pi / h) * qhat[nz] / lam[nz]
    return np.fft.ifftn(phihat).real


# ---------------------------------------------------------------- multigrid
# The correction solve of Eq. 20 as the paper's method runs it: a multigrid
# V-cycle iteration on M y = sigma_p until max|sigma_p - M y| <= tol.  The
# paper does not give the smoother, transfer operators, depth or coarse solve
# (Sec. 3.3 footnote); this follows the reading taken for the GPU path:
# rediscretised dimensionless M on every level, red-black Gauss-Seidel (red =
# points with x + y + z even), full-weighting restriction scaled by 4 (the
# spacing doubles), trilinear prolongation, and the exact pseudo-inverse on
# the coarse level.  Levels are n, n/2, ... halved while even and larger than
# 16; the first of size <= coarse_max (else the deepest) is the coarse level.

def mg_levels(n: int, coarse_max: int) -> list[int]:
    levels = [n]
    while levels[-1] > 16 and levels[-1] % 2 == 0:
        levels.append(levels[-1] // 2)
    for i, m in enumerate(levels):
        if m <= coarse_max:
            return levels[: i + 1]
    return levels


def _red_mask(n: int) -> np.ndarray:
    i = np.arange(n)
    return ((i[:, None, None] + i[None, :, None] + i[None, None, :]) % 2) == 0


def gauss_seidel_half(e: np.ndarray, b: np.ndarray, mask: np.ndarray) -> np.ndarray:
    """One red-black Gauss-Seidel half sweep on M e = b: every point of one
    colour takes e = (sum of its six neighbours - b)/6; its neighbours all
    have the other colour, so updating them together is Gauss-Seidel."""
    nb = laplacian7(e) + 6.0 * e
    return np.where(mask, (nb - b) / 6.0, e)


def restrict_full_weighting(r: np.ndarray) -> np.ndarray:
    """Coarse right-hand side 4 R r: R weights the fine points around 2I by the
    tensor product of (1/4, 1/2, 1/4); the 4 rescales the dimensionless M to
    the doubled spacing."""
    out = r
    for ax in range(3):
        out = 0.25 * np.roll(out, 1, axis=ax) + 0.5 * out + 0.25 * np.roll(out, -1, axis=ax)
    return 4.0 * out[::2, ::2, ::2]


def prolong_trilinear(ec: np.ndarray) -> np.ndarray:
    """Trilinear interpolation from the coarse points (fine 2I) to the fine mesh."""
    out = ec
    for ax in range(3):
        shape = list(out.shape)
        shape[ax] *= 2
        f = np.zeros(shape)
        even = [slice(None)] * 3
        odd = [slice(None)] * 3
        even[ax] = slice(0, None, 2)
        odd[ax] = slice(1, None, 2)
        f[tuple(even)] = out
        f[tuple(odd)] = 0.5 * (out + np.roll(out, -1, axis=ax))
        out = f
    return out


def pseudo_inverse_solve(b: np.ndarray) -> np.ndarray:
    """e = M^+ b (the zero-mean solution; the mean of b is dropped), by FFT."""
    lam = laplacian_eigenvalues(b.shape[0])
    bh = np.fft.fftn(b)
    eh = np.zeros_like(bh)
    nz = lam != 0.0
    eh[nz] = bh[nz] / lam[nz]
    return np.fft.ifftn(eh).real


def v_cycle(b: np.ndarray, levels: list[int], nu1: int = 2, nu2: int = 2, level: int = 0) -> np.ndarray:
    """One V-cycle from e = 0 on M e = b: nu1 sweeps (red then black), the
    coarse correction, nu2 sweeps (black then red)."""
    if level == len(levels) - 1:
        return pseudo_inverse_solve(b)
    red = _red_mask(b.shape[0])
    black = ~red
    e = np.zeros_like(b)
    for _ in range(nu1):
        e = gauss_seidel_half(e, b, red)
        e = gauss_seidel_half(e, b, black)
    bc = restrict_full_weighting(b - laplacian7(e))
    e = e + prolong_trilinear(v_cycle(bc, levels, nu1, nu2, level + 1))
    for _ in range(nu2):
        e = gauss_seidel_half(e, b, black)
        e = gauss_seidel_half(e, b, red)
    return e


def mg_correction_solve(sigma: np.ndarray, y0: np.ndarray, tol: float, levels: list[int], nu1: int = 2,
                        nu2: int = 2, itmax: int = 50):
    """Eq. 20's correction solve: V-cycles on M e = sigma - M y, y += e, until
    max|sigma - M y| <= tol.  Returns y, the V-cycles run and the residual
    max-norm before and after each of them."""
    y = np.array(y0, dtype=np.float64, copy=True)
    r = sigma - laplacian7(y)
    hist = [float(np.abs(r).max())]
    it = 0
    while hist[-1] > tol and it < itmax:
        y = y + v_cycle(r, levels, nu1, nu2)
        r = sigma - laplacian7(y)
        hist.append(float(np.abs(r).max()))
        it += 1
    return y, it, hist


def mesh_gradient(phi: np.ndarray, h: float) -> list[np.ndarray]:
    """Central finite-difference gradient D phi (Eq. 21's D_x, D_y, D_z)."""
    return [(np.roll(phi, -1, axis=ax) - np.roll(phi, 1, axis=ax)) / (2.0 * h) for ax in range(3)]


def interpolate_lr_forces(pos, charge, box, n, phi, ke=COULOMB_K) -> np.ndarray:
    """F_a = -ke Q_a sum_n W(r_a - r_n) (D phi)_n (Eq. 21), W the same cubic
    B-spline as the assignment."""
    h = box / n
    grad = mesh_gradient(phi, h)
    base, w = assignment_stencil(pos, box, n)
    F = np.zeros((pos.shape[0], 3))
    for a in range(4):
        ix = (base[:, 0] + a) % n
        for b in range(4):
            iy = (base[:, 1] + b) % n
            for c in range(4):
                iz = (base[:, 2] + c) % n
                wt = w[:, 0, a] * w[:, 1, b] * w[:, 2, c]
                for d in range(3):
                    F[:, d] -= ke * charge * wt * grad[d][ix, iy, iz]
    return F


# ---------------------------------------------------------------------------
# Short range
# ---------------------------------------------------------------------------
def _image_shifts(box: float, r_cut: float) -> np.ndarray:
    m = int(math.ceil(r_cut / box))
    r = np.arange(-m, m + 1)
    return np.array([[i, j, k] for i in r for j in r for k in r], float) * box


def sr_coulomb_pair(r: np.ndarray, qq: np.ndarray, sigma: float, ke: float):
    """Energy and force magnitude/r of the screened Coulomb pair term:
    U = ke QQ erfc(r/(sqrt2 sigma))/r (Eq. 5);
    F/r = ke QQ [erfc(r/sqrt2 sigma)/r^3 + sqrt(2/pi) exp(-r^2/2sigma^2)/(sigma r^2)] (Eq. 19)."""
    x = r / (math.sqrt(2.0) * sigma)
    e = ke * qq * _erfc(x) / r
    f_over_r = ke * qq * (_erfc(x) / r ** 3
                          + math.sqrt(2.0 / math.pi) * np.exp(-r * r / (2.0 * sigma * sigma))
                          / (sigma * r * r))
    return e, f_over_r


def bmh_pair(r, A, rho, s, C, D):
    """Born-Huggins-Mayer: U = A exp((s - r)/rho) - C/r^6 - D/r^8 and -dU/dr / r."""
    ex = A * np.exp((s - r) / rho)
    e = ex - C / r ** 6 - D / r ** 8
    f_over_r = (ex / rho - 6.0 * C / r ** 7 - 8.0 * D / r ** 9) / r
    return e, f_over_r


def lj_pair(r, eps, sig):
    """Lennard-Jones: U = 4 eps [(s/r)^12 - (s/r)^6] and -dU/dr / r."""
    sr6 = (sig / r) ** 6
    e = 4.0 * eps * (sr6 * sr6 - sr6)
    f_over_r = 24.0 * eps * (2.0 * sr6 * sr6 - sr6) / (r * r)
    return e, f_over_r


def shift_force(pair_fn, r, r_cut, *args):
    """A pair term made continuous at the cutoff, the shifted-force form:
    U_sf(r) = U(r) - U(r_c) + (r - r_c) F(r_c) and F_sf(r) = F(r) - F(r_c),
    with F = -dU/dr the term's force magnitude (pair_fn returns U and F/r).
    This is an option for energy-conservation studies; the paper leaves the
    treatment of the cutoff open and the default truncates without a shift.
    Returns (U_sf, F_sf / r)."""
    e, f_over_r = pair_fn(r, *args)
    e_c, fr_c = pair_fn(np.full_like(r, r_cut), *args)
    f_c = fr_c * r_cut
    return e - e_c + (r - r_cut) * f_c, f_over_r - f_c / r


def sr_forces(system, sigma: float, r_cut: float, ke: float = COULOMB_K,
              subset: np.ndarray | None = None, coulomb: bool = True, vdw: bool = True,
              shift: str = "none", virial: bool = False):
    """Short-range forces and per-particle energies by explicit summation over
    every particle j and every periodic image within R_c (Eq. 19 plus the
    non-Coulomb term).  Pairs inside one molecule (nearest image) are skipped.
    shift='force' applies the shifted-force cutoff (shift_force) to every
    term; 'none' truncates at R_c.

    Returns (F (m,3), e_coul (m,), e_vdw (m,)) for the particles in `subset`
    (default all); per-particle energies carry the factor 1/2 of Eq. 5.  With
    virial=True also w (m,): half of sum_j r_ij . F_ij over the particle's
    pairs (r_ij = r_i - r_j, F_ij the pair force on i), so that w.sum() is the
    short-range pair virial sum_{i<j} r_ij . F_ij."""
    if shift not in ("none", "force"):
        raise ValueError(shift)

    def term(fn, r, *args):
        return shift_force(fn, r, r_cut, *args) if shift == "force" else fn(r, *args)

    pos, q, types, box = system.pos, system.charge, system.types, system.box
    idx = np.arange(system.n) if subset is None else np.asarray(subset)
    shifts = _image_shifts(box, r_cut)
    mol = system.molecule
    F = np.zeros((idx.size, 3))
    ec = np.zeros(idx.size)
    ev = np.zeros(idx.size)
    w = np.zeros(idx.size)
    for row, i in enumerate(idx):
        d0 = pos[i][None, :] - pos                      # r_i - r_j
        for s in shifts:
            d = d0 + s[None, :]
            r2 = (d * d).sum(1)
            mask = r2 < r_cut * r_cut
            if not s.any():
                mask[i] = False
            if mol is not None:
                # the nearest image of an intramolecular partner is excluded;
                # farther images of it are ordinary interactions
                same = mask & (mol == mol[i])
                if same.any():
                    dn = d0[same] - box * np.round(d0[same] / box)
                    nearest = np.all(np.abs(d[same] - dn) < 1e-9 * box, axis=1)
                    mask[np.nonzero(same)[0][nearest]] = False
            if not mask.any():
                continue
            dj = d[mask]
            r = np.sqrt(r2[mask])
            fr = np.zeros_like(r)
            if coulomb:
                e, f = term(sr_coulomb_pair, r, q[i] * q[mask], sigma, ke)
                ec[row] += 0.5 * e.sum()
                fr += f
            if vdw and system.sr_kind == "bmh":
                t = system.sr_table
                ti, tj = types[i], types[mask]
                e, f = term(bmh_pair, r, t["A"][ti, tj], t["rho"][ti, tj], t["sigma"][ti, tj],
                            t["C"][ti, tj], t["D"][ti, tj])
                ev[row] += 0.5 * e.sum()
                fr += f
            elif vdw and system.sr_kind == "lj":
                t = system.sr_table
                ti, tj = types[i], types[mask]
                eps = t["eps"][ti, tj]
                live = eps != 0.0
                if live.any():
                    e, f = term(lj_pair, r[live], eps[live], t["sigma"][ti, tj][live])
                    ev[row] += 0.5 * e.sum()
                    fr[live] += f
            F[row] += (fr[:, None] * dj).sum(0)
            w[row] += 0.5 * (fr * r * r).sum()              # r_ij . F_ij = (F/r) r^2
    if virial:
        return F, ec, ev, w
    return F, ec, ev


def sr_forces_cells(system, sigma: float, r_cut: float, ke: float = COULOMB_K, shift: str = "none"):
    """The short-range sum of sr_forces found through the oracle's own cell
    list instead of all pairs, O(N): cells have edge >= R_c/2, so every
    periodic image within R_c of a particle lies in the 5 x 5 x 5 block of
    cells around its own, each taken once with its explicit image shift (for
    fewer than 5 cells per axis the block wraps onto other images of the same
    cells).  Same terms, exclusions and per-particle energies as sr_forces
    (pinned against it on small systems); used where the all-pairs loop is
    too slow, e.g. to time the oracle's MD step."""
    pos, q, types, box = system.pos, system.charge, system.types, system.box
    mol = system.molecule
    nc, cell, start, order = cell_list(pos, box, r_cut)
    N = system.n
    F = np.zeros((N, 3))
    ec = np.zeros(N)
    ev = np.zeros(N)

    def term(fn, r, *args):
        return shift_force(fn, r, r_cut, *args) if shift == "force" else fn(r, *args)

    rc2 = r_cut * r_cut
    for cz in range(nc):
        for cy in range(nc):
            for cx in range(nc):
                c = (cz * nc + cy) * nc + cx
                home = order[start[c]:start[c + 1]]
                if home.size == 0:
                    continue
                js, shifts = [], []
                for dz in range(-2, 3):
                    for dy in range(-2, 3):
                        for dx in range(-2, 3):
                            u = (cx + dx, cy + dy, cz + dz)
                            w = [ui % nc for ui in u]
                            cc = (w[2] * nc + w[1]) * nc + w[0]
                            j = order[start[cc]:start[cc + 1]]
                            if j.size:
                                js.append(j)
                                img = np.array([(ui // nc) * box for ui in u])  # image of cell u
                                shifts.append(np.broadcast_to(img, (j.size, 3)))
                J = np.concatenate(js)
                Sft = np.concatenate(shifts)
                for i in home:
                    d = pos[i][None, :] - (pos[J] + Sft)            # r_i - image of r_j
                    r2 = (d * d).sum(1)
                    mask = (r2 < rc2) & ~((J == i) & ~Sft.any(1))
                    if mol is not None:
                        same = mask & (mol[J] == mol[i])
                        if same.any():
                            d0 = pos[i][None, :] - pos[J[same]]
                            dn = d0 - box * np.round(d0 / box)
                            nearest = np.all(np.abs(d[same] - dn) < 1e-9 * box, axis=1)
                            mask[np.nonzero(same)[0][nearest]] = False
                    if not mask.any():
                        continue
                    Jm = J[mask]
                    dj = d[mask]
                    r = np.sqrt(r2[mask])
                    fr = np.zeros_like(r)
                    e, f = term(sr_coulomb_pair, r, q[i] * q[Jm], sigma, ke)
                    ec[i] += 0.5 * e.sum()
                    fr += f
                    if system.sr_kind == "bmh":
                        t = system.sr_table
                        ti, tj = types[i], types[Jm]
                        e, f = term(bmh_pair, r, t["A"][ti, tj], t["rho"][ti, tj], t["sigma"][ti, tj],
                                    t["C"][ti, tj], t["D"][ti, tj])
                        ev[i] += 0.5 * e.sum()
                        fr += f
                    elif system.sr_kind == "lj":
                        t = system.sr_table
                        ti, tj = types[i], types[Jm]
                        eps = t["eps"][ti, tj]
                        live = eps != 0.0
                        if live.any():
                            e, f = term(lj_pair, r[live], eps[live], t["sigma"][ti, tj][live])
                            ev[i] += 0.5 * e.sum()
                            fr[live] += f
                    F[i] += (fr[:, None] * dj).sum(0)
    return F, ec, ev


def intramolecular_terms(system, sigma: float, ke: float = COULOMB_K):
    """SPC/Fw bonded terms and the intramolecular Coulomb exclusion.

    Bonds (k_b/2)(r - r0)^2 and angles (k_a/2)(theta - theta0)^2 (Table S1).
    Intramolecular pairs are left out of the short-range sum but are present
    in the mesh potential, whose pair kernel is ke QQ erf(r/(sqrt2 sigma))/r; that
    part is subtracted here so intramolecular Coulomb is excluded in total.
    Parity unpinned beyond finite differences (the paper gives no formula for
    the exclusion)."""
    pos, box, q = system.pos, system.box, system.charge
    F = np.zeros_like(pos)
    e_bond = e_angle = e_excl = 0.0
    b = system.bonded
    for i, j in system.bonds:
        d = pos[i] - pos[j]
        d -= box * np.round(d / box)
        r = np.linalg.norm(d)
        e_bond += 0.5 * b["kb"] * (r - b["r0"]) ** 2
        f = -b["kb"] * (r - b["r0"]) * d / r
        F[i] += f
        F[j] -= f
    for h1, o, h2 in system.angles:
        a = pos[h1] - pos[o]
        a -= box * np.round(a / box)
        c = pos[h2] - pos[o]
        c -= box * np.round(c / box)
        ra, rc = np.linalg.norm(a), np.linalg.norm(c)
        cos_t = np.clip(a @ c / (ra * rc), -1.0, 1.0)
        th = math.acos(cos_t)
        e_angle += 0.5 * b["ka"] * (th - b["theta0"]) ** 2
        dE = b["ka"] * (th - b["theta0"])
        sin_t = max(math.sqrt(1.0 - cos_t * cos_t), 1e-12)
        # dtheta/da = -(c/(ra rc) - cos a/ra^2) / sin
        ga = -(c / (ra * rc) - cos_t * a / ra ** 2) / sin_t
        gc = -(a / (ra * rc) - cos_t * c / rc ** 2) / sin_t
        F[h1] -= dE * ga
        F[h2] -= dE * gc
        F[o] += dE * (ga + gc)
    if system.molecule is not None:
        mol = system.molecule
        n_mol = int(mol.max()) + 1 if mol.size else 0
        for m in range(n_mol):
            atoms = np.nonzero(mol == m)[0]
            for x in range(atoms.size):
                for y in range(x + 1, atoms.size):
                    i, j = atoms[x], atoms[y]
                    d = pos[i] - pos[j]
                    d -= box * np.round(d / box)
                    r = np.linalg.norm(d)
                    qq = q[i] * q[j]
                    u = r / (math.sqrt(2.0) * sigma)
                    e_excl -= ke * qq * _erf(u) / r
                    # -d/dr [ -erf(u)/r ] = -(erf(u)/r^2 - sqrt(2/pi)/sigma exp(-u^2)/r)
                    f_over_r = -ke * qq * (_erf(u) / r ** 3
                                           - math.sqrt(2.0 / math.pi) * np.exp(-u * u) / (sigma * r * r))
                    F[i] += f_over_r * d
                    F[j] -= f_over_r * d
    return F, e_bond, e_angle, e_excl


# ---------------------------------------------------------------------------
# The whole force evaluation at one configuration
# ---------------------------------------------------------------------------
def self_energy(charge: np.ndarray, sigma: float, ke: float = COULOMB_K) -> float:
    """V_self = -(1/(sqrt(2 pi) sigma)) sum Q^2 (Eq. 6)."""
    return -ke * float((charge * charge).sum()) / (math.sqrt(2.0 * math.pi) * sigma)


def mesh_fields(system, alpha: float, n: int, order: int = 4):
    """q, q^s (mean removed), phi* and the smoothing schedule at the current
    positions."""
    if order != 4:
        raise ValueError("only cubic (order-4) assignment is defined here")
    box = system.box
    h = box / n
    sigma = sigma_of_alpha(alpha)
    K, c = smoothing_schedule(sigma, h, order)
    q = assign_charges(system.pos, system.charge, box, n)
    qs = smooth(q, K, c)
    qs = qs - qs.mean()
    phi = solve_constraint_fft(qs, h)
    return {"q": q, "qs": qs, "phi": phi, "K": K, "c": c, "h": h, "sigma": sigma}


def interpolate_lr_forces_analytic(pos, charge, box, n, phi, ke=COULOMB_K) -> np.ndarray:
    """F_a = -ke Q_a sum_n grad W(r_a - r_n) phi_n: the exact gradient of
    V_LR = 1/2 ke phi^T q with q = A(r)Q and phi = G q (G symmetric), the
    energy-conserving alternative to Eq. 21's finite differences (an option,
    not the paper's force)."""
    inv_h = n / box
    u = pos * inv_h
    fl = np.floor(u)
    base = fl.astype(np.int64) - 1
    w = bspline4_weights(u - fl)
    dw = bspline4_derivatives(u - fl) * inv_h
    F = np.zeros((pos.shape[0], 3))
    for a in range(4):
        ix = (base[:, 0] + a) % n
        for b in range(4):
            iy = (base[:, 1] + b) % n
            for c in range(4):
                iz = (base[:, 2] + c) % n
                p = phi[ix, iy, iz]
                F[:, 0] -= ke * charge * dw[:, 0, a] * w[:, 1, b] * w[:, 2, c] * p
                F[:, 1] -= ke * charge * w[:, 0, a] * dw[:, 1, b] * w[:, 2, c] * p
                F[:, 2] -= ke * charge * w[:, 0, a] * w[:, 1, b] * dw[:, 2, c] * p
    return F


def lr_energy_at(pos, charge, box, alpha, n, ke=COULOMB_K) -> float:
    """V_LR = 1/2 ke phi*^T q at the given positions (the adopted reading)."""
    h = box / n
    K, c = smoothing_schedule(sigma_of_alpha(alpha), h)
    q = assign_charges(pos, charge, box, n)
    qs = smooth(q, K, c)
    qs = qs - qs.mean()
    return 0.5 * ke * float((solve_constraint_fft(qs, h) * q).sum())


def forces_and_energies(system, alpha: float, r_cut: float, n: int, ke: float = COULOMB_K,
                        order: int = 4, lr_energy: str = "assigned", lr_force: str = "fd",
                        sr_shift: str = "none"):
    """Total force and energy terms of the P3MaZe decomposition at the exactly
    constrained field phi* (Eqs. 5, 6, 14, 19, 21).

    lr_energy='assigned' uses V_LR = 1/2 phi^T q (the reading adopted here);
    'smoothed' evaluates Eq. 14 literally, 1/2 phi^T q^s (kept so that a test
    can show the Madelung pin rejects it).  sr_shift as sr_forces' shift."""
    mf = mesh_fields(system, alpha, n, order)
    sigma = mf["sigma"]
    if lr_force == "analytic":
        F_lr = interpolate_lr_forces_analytic(system.pos, system.charge, system.box, n, mf["phi"], ke)
    else:
        F_lr = interpolate_lr_forces(system.pos, system.charge, system.box, n, mf["phi"], ke)
    F_sr, ec, ev, w = sr_forces(system, sigma, r_cut, ke, shift=sr_shift, virial=True)
    src = mf["q"] if lr_energy == "assigned" else mf["qs"]
    v_lr = 0.5 * ke * float((mf["phi"] * src).sum())
    out = {
        "F_lr": F_lr, "F_sr": F_sr, "F": F_lr + F_sr,
        "v_sr": float(ec.sum()), "v_vdw": float(ev.sum()), "v_lr": v_lr,
        "w_sr": float(w.sum()),
        "v_self": self_energy(system.charge, sigma, ke),
        "fields": mf,
    }
    if system.bonds.size or system.molecule is not None:
        Fb, eb, ea, ex = intramolecular_terms(system, sigma, ke)
        out["F"] = out["F"] + Fb
        out["v_bond"], out["v_angle"], out["v_excl"] = eb, ea, ex
    else:
        out["v_bond"] = out["v_angle"] = out["v_excl"] = 0.0
    out["v_coul"] = out["v_sr"] + out["v_lr"] + out["v_self"] + out["v_excl"]
    out["v_pot"] = out["v_coul"] + out["v_vdw"] + out["v_bond"] + out["v_angle"]
    return out


# ---------------------------------------------------------------------------
# PMaZe: the whole Coulomb problem on the mesh (the comparison method, Secs. 1-2)
# ---------------------------------------------------------------------------
def pmaze_mesh_fields(system, n: int) -> dict:
    """PMaZe's exactly constrained potential: the assigned charge q = A(r)Q
    itself is the source (Sec. 2, "charge assignment and smoothing": no
    Gaussian screening and no smoothing), its mean removed for the gauge, and
    phi* = -(4 pi / h) M^+ q solves (h/4pi) M phi + q = 0 (Eq. 13 with q in
    place of q^s)."""
    h = system.box / n
    q = assign_charges(system.pos, system.charge, system.box, n)
    phi = solve_constraint_fft(q - q.mean(), h)
    return {"q": q, "phi": phi, "h": h}


def pmaze_forces_and_energies(system, r_cut: float, n: int, ke: float = COULOMB_K) -> dict:
    """PMaZe forces at the exactly constrained field: Eq. 21 applied to the
    full-Coulomb mesh potential gives the whole electrostatic force; pairs
    within R_c carry only the non-Coulomb term.  v_mesh = 1/2 ke phi*^T q
    contains the grid self-energy of every charge (Sec. 2, "electrostatic
    energy"); the work-based energy the paper uses for PMaZe is not formed.
    Systems with molecules are not defined here (their exclusions would need
    the mesh pair interaction).  Only the finite-difference force of Eq. 21:
    with the whole charge on the mesh, the exact gradient of v_mesh is
    dominated by the gradient of the grid self-energy."""
    if system.molecule is not None:
        raise ValueError("PMaZe is defined here for systems without molecules")
    mf = pmaze_mesh_fields(system, n)
    F_mesh = interpolate_lr_forces(system.pos, system.charge, system.box, n, mf["phi"], ke)
    F_vdw, _, ev = sr_forces(system, 1.0, r_cut, ke, coulomb=False)
    return {"F_mesh": F_mesh, "F_vdw": F_vdw, "F": F_mesh + F_vdw, "v_vdw": float(ev.sum()),
            "v_mesh": 0.5 * ke * float((mf["phi"] * mf["q"]).sum()), "fields": mf}


def kinetic_energy(vel: np.ndarray, mass: np.ndarray) -> float:
    """sum 1/2 m v^2 in kcal/mol (v in A/fs, m in g/mol)."""
    return 0.5 * float((mass[:, None] * vel * vel).sum()) / ACCEL


def wrap(pos: np.ndarray, box: float) -> np.ndarray:
    """Map positions into [0, L): r - L floor(r/L), a result equal to L -> 0."""
    w = pos - box * np.floor(pos / box)
    return np.where(w >= box, 0.0, w)


def velocity_verlet_step(system, force, dt: float, force_fn):
    """One velocity-Verlet step (Sec. 2; SI Sec. 1 "Numerical integration"):
    kick, drift, wrap, new forces, kick.  Returns (new force, force_fn output)."""
    acc = ACCEL / system.mass[:, None]
    system.vel = system.vel + 0.5 * dt * force * acc
    system.pos = wrap(system.pos + dt * system.vel, system.box)
    out = force_fn(system)
    system.vel = system.vel + 0.5 * dt * out["F"] * acc
    return out


def maze_md_step(system, state: dict, alpha: float, r_cut: float, n: int, dt: float, tol: float,
                 predictor: int = 1, coarse_max: int = 64, ke: float = COULOMB_K,
                 timings: dict | None = None) -> int:
    """One velocity-Verlet MD step with the Mass-Zero field, the plain FP64
    stepper (Sec. 2; SI Sec. 1 "Numerical integration"; Eqs. 16-17, 20, 21):
      kick v += dt/2 F/m, drift r += dt v, wrap;
      q = A(r)Q, q^s = (I + cM)^K q - mean;
      phi_p = 2 phi^k - phi^{k-1}, sigma_p = (h/4pi) M phi_p + q^s (Eq. 17);
      y0 from the multiplier history (order `predictor`, fewer while the
      history is short), V-cycles on M y = sigma_p to max|M y - sigma_p| <= tol
      (Eq. 20, the plain multigrid of mg_correction_solve);
      phi^{k+1} = phi_p - (4pi/h) y*;
      F = -ke Q W . D phi^{k+1} (Eq. 21) + short-range forces (cell list);
      kick.
    state holds 'F', 'phi' (phi^k), 'phi_prev' (phi^{k-1}) and 'y' (the
    multiplier history, newest first); it is updated in place, and the
    system's positions and velocities advance.  Systems without molecules.
    If `timings` is given, the seconds spent in the short-range sum are
    stored under 'sr'.  Returns the V-cycles of the solve."""
    box = system.box
    h = box / n
    acc = ACCEL / system.mass[:, None]
    system.vel = system.vel + 0.5 * dt * state["F"] * acc
    system.pos = wrap(system.pos + dt * system.vel, box)
    sigma = sigma_of_alpha(alpha)
    K, c = smoothing_schedule(sigma, h)
    q = assign_charges(system.pos, system.charge, box, n)
    qs = smooth(q, K, c)
    qs = qs - qs.mean()
    phi_p = 2.0 * state["phi"] - state["phi_prev"]
    sigma_p = h / (4.0 * math.pi) * laplacian7(phi_p) + qs
    hist = state["y"]
    order = min(predictor, len(hist))
    if order == 0:
        y0 = np.zeros_like(sigma_p)
    elif order == 1:
        y0 = hist[0]
    elif order == 2:
        y0 = 2.0 * hist[0] - hist[1]
    else:
        y0 = 3.0 * hist[0] - 3.0 * hist[1] + hist[2]
    y, iters, _ = mg_correction_solve(sigma_p, y0, tol, mg_levels(n, coarse_max))
    phi = phi_p - (4.0 * math.pi / h) * y
    F_lr = interpolate_lr_forces(system.pos, system.charge, box, n, phi, ke)
    t_sr = time.perf_counter()
    F_sr, _, _ = sr_forces_cells(system, sigma, r_cut, ke)
    if timings is not None:
        timings["sr"] = time.perf_counter() - t_sr
    state["F"] = F_lr + F_sr
    state["phi_prev"], state["phi"] = state["phi"], phi
    state["y"] = [y] + hist[:2]
    system.vel = system.vel + 0.5 * dt * state["F"] * acc
    return iters


def maze_initial_state(system, alpha: float, r_cut: float, n: int, ke: float = COULOMB_K) -> dict:
    """Stepper state at the start (reading A7): the exactly constrained field
    at the initial positions as both phi^0 and phi^{-1}, an empty multiplier
    history, and the forces there."""
    mf = mesh_fields(system, alpha, n)
    F = interpolate_lr_forces(system.pos, system.charge, system.box, n, mf["phi"], ke)
    F = F + sr_forces_cells(system, mf["sigma"], r_cut, ke)[0]
    return {"F": F, "phi": mf["phi"], "phi_prev": mf["phi"].copy(), "y": []}


# ---------------------------------------------------------------------------
# Cell list (integer work: the CUDA path must match it bit for bit)
# ---------------------------------------------------------------------------
def cell_grid(box: float, r_cut: float) -> int:
    """Cells per axis: floor(L / (R_c/2)) sub-cells of edge >= R_c/2."""
    return max(1, int(math.floor(box / (0.5 * r_cut))))


def cell_list(pos: np.ndarray, box: float, r_cut: float):
    """Cell index of each particle (x fastest: (cz*nc + cy)*nc + cx, with
    c = floor(r * (nc/L)) clamped to nc-1), the cell start offsets, and the
    particle order sorted by (cell, particle index)."""
    nc = cell_grid(box, r_cut)
    inv = nc / box
    c3 = np.minimum(np.floor(pos * inv).astype(np.int64), nc - 1)
    cell = (c3[:, 2] * nc + c3[:, 1]) * nc + c3[:, 0]
    order = np.lexsort((np.arange(pos.shape[0]), cell))
    counts = np.bincount(cell, minlength=nc ** 3)
    start = np.concatenate([[0], np.cumsum(counts)])
    return nc, cell.astype(np.int32), start.astype(np.int32), order.astype(np.int32)


# ---------------------------------------------------------------------------
# Brute-force Ewald summation (independent reference for the pins)
# ---------------------------------------------------------------------------
def ewald(pos: np.ndarray, charge: np.ndarray, box: float, alpha: float, ke: float = 1.0,
          tol: float = 1e-16, forces: bool = True):
    """Classical Ewald sum of Eq. 2 for a cubic box: real-space erfc sum over
    all images within the cutoff where erfc(alpha r) < tol, reciprocal sum over
    all k with exp(-k^2/4alpha^2) < tol, and the self term.  Returns
    (energy, forces)."""
    n = pos.shape[0]
    # erfc(x) < tol for x > ~ sqrt(-ln tol)
    xc = math.sqrt(-math.log(tol)) + 0.5
    rc = xc / alpha
    shifts = _image_shifts(box, rc)
    e_real = 0.0
    F = np.zeros((n, 3))
    for i in range(n):
        d0 = pos[i][None, :] - pos
        for s in shifts:
            d = d0 + s[None, :]
            r = np.sqrt((d * d).sum(1))
            m = r < rc
            if not s.any():
                m[i] = False
            if not m.any():
                continue
            rr = r[m]
            qq = charge[i] * charge[m]
            e_real += 0.5 * float((qq * _erfc(alpha * rr) / rr).sum())
            if forces:
                fr = qq * (_erfc(alpha * rr) / rr + 2.0 * alpha / math.sqrt(math.pi)
                           * np.exp(-(alpha * rr) ** 2)) / (rr * rr)
                F[i] += (fr[:, None] * d[m]).sum(0)
    kc = 2.0 * alpha * xc
    mmax = int(math.ceil(kc * box / (2.0 * math.pi)))
    rng = np.arange(-mmax, mmax + 1)
    mvec = np.array([[a, b, c] for a in rng for b in rng for c in rng], float)
    mvec = mvec[np.any(mvec != 0, axis=1)]
    kvec = mvec * (2.0 * math.pi / box)
    k2 = (kvec * kvec).sum(1)
    keep = k2 <= kc * kc
    kvec, k2 = kvec[keep], k2[keep]
    vol = box ** 3
    e_rec = 0.0
    for start in range(0, kvec.shape[0], 4096):
        kv = kvec[start:start + 4096]
        kk = k2[start:start + 4096]
        phase = pos @ kv.T                                # (n, nk)
        eikr = np.exp(1j * phase)
        S = (charge[:, None] * eikr).sum(0)               # (nk,)
        g = np.exp(-kk / (4.0 * alpha * alpha)) / kk
        e_rec += (2.0 * math.pi / vol) * float((g * np.abs(S) ** 2).sum())
        if forces:
            im = np.imag(eikr * np.conj(S)[None, :])      # (n, nk)
            F += (4.0 * math.pi / vol) * charge[:, None] * ((im * g[None, :]) @ kv)
    e_self = -alpha / math.sqrt(math.pi) * float((charge * charge).sum())
    return ke * (e_real + e_rec + e_self), ke * F
