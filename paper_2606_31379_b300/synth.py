"""Seeded synthetic inputs for the P3MaZe electrostatics path.

This module holds input generation only: particle configurations, force-field
parameter tables and the unit constants needed to draw thermal velocities.  It
contains none of the method's arithmetic (no assignment, smoothing, solve or
force code), so both the CUDA path and the FP64 oracle can be fed from it.

Workload shapes follow the paper's two test systems (molten NaCl with a
Born-Huggins-Mayer short-range term, Sec. 3.1.1; flexible SPC/Fw water,
Sec. 3.2.1 and Table S1) at the sizes used in this project's configurations:
uniform random ion positions with a minimum pair distance, Maxwell-Boltzmann
velocities and net momentum removed.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

# ---------------------------------------------------------------------------
# Units: lengths in Angstrom, time in fs, mass in g/mol, charge in e,
# energy in kcal/mol.  Only what the generators need lives here.
# ---------------------------------------------------------------------------
KB_KCAL = 0.0019872043          # Boltzmann constant, kcal/(mol K)
ACCEL_CONV = 4.184e-4           # (kcal/mol/A)/(g/mol) -> A/fs^2
EV_TO_KCAL = 23.060548          # kcal/mol per eV
ERG_CM6_E60_TO_EV_A6 = 0.6241509074   # 1e-60 erg cm^6 in eV A^6 (same factor for 1e-76 erg cm^8 -> eV A^8)

MASS_NA = 22.98977
MASS_CL = 35.453
MASS_O = 15.9994
MASS_H = 1.008

# Species ids used by the short-range table.
NA, CL = 0, 1
OW, HW = 0, 1


@dataclass
class System:
    """One periodic system: SoA particle arrays plus its parameters."""
    pos: np.ndarray          # (n,3) float64, A, inside [0, L)
    vel: np.ndarray          # (n,3) float64, A/fs
    charge: np.ndarray       # (n,) float64, e
    mass: np.ndarray         # (n,) float64, g/mol
    types: np.ndarray        # (n,) int32 species id
    box: float               # cubic box edge, A
    # short-range table: kind 'bmh' or 'lj'; arrays indexed [ti, tj]
    sr_kind: str = "bmh"
    sr_table: dict = field(default_factory=dict)
    # SPC/Fw topology (empty for ionic systems)
    bonds: np.ndarray = field(default_factory=lambda: np.zeros((0, 2), np.int32))
    angles: np.ndarray = field(default_factory=lambda: np.zeros((0, 3), np.int32))
    bonded: dict = field(default_factory=dict)
    # molecule id per particle (for intramolecular exclusions); -1 = none
    molecule: np.ndarray | None = None

    @property
    def n(self) -> int:
        return int(self.pos.shape[0])


# ---------------------------------------------------------------------------
# Force-field tables
# ---------------------------------------------------------------------------
def tosi_fumi_nacl() -> dict:
    """Born-Huggins-Mayer table for NaCl (Tosi-Fumi form, Sec. 3.1.1).

    U_ij(r) = A_ij exp((s_ij - r)/rho) - C_ij/r^6 - D_ij/r^8, with
    A_ij = beta_ij * b (Pauling factors 1.25 / 1.00 / 0.75), b = 0.338e-19 J,
    rho = 0.317 A, s_ij = s_i + s_j (s_Na = 1.170, s_Cl = 1.585 A) and the
    dispersion coefficients C (1e-60 erg cm^6) = 1.68 / 11.2 / 116 and
    D (1e-76 erg cm^8) = 0.8 / 13.9 / 233 for ++ / +- / --.
    These values are the commonly quoted Fumi-Tosi 1964 set, written here from
    memory and not verified against the original table; the CUDA path and the
    oracle read the same table, so parity does not depend on them.
    """
    b_ev = 0.338e-19 / 1.602176634e-19
    pauling = np.array([[1.25, 1.00], [1.00, 0.75]])
    s_ion = np.array([1.170, 1.585])
    c6 = np.array([[1.68, 11.2], [11.2, 116.0]]) * ERG_CM6_E60_TO_EV_A6
    d8 = np.array([[0.8, 13.9], [13.9, 233.0]]) * ERG_CM6_E60_TO_EV_A6
    return {
        "A": pauling * b_ev * EV_TO_KCAL,
        "rho": np.full((2, 2), 0.317),
        "sigma": s_ion[:, None] + s_ion[None, :],
        "C": c6 * EV_TO_KCAL,
        "D": d8 * EV_TO_KCAL,
    }


def spcfw_params() -> dict:
    """SPC/Fw parameters as listed in Table S1 (Wu, Tepper, Voth 2006).

    Bond and angle energies are read as (k/2)(x - x0)^2 with the tabulated k.
    """
    return {
        "eps_oo": 0.1554253, "sigma_oo": 3.165492,
        "q_o": -0.82, "q_h": 0.41,
        "r0": 1.012, "theta0": math.radians(113.24),
        "kb": 1059.162, "ka": 75.90,
    }


def spcfw_lj_table() -> dict:
    p = spcfw_params()
    eps = np.zeros((2, 2))
    sig = np.ones((2, 2))
    eps[OW, OW] = p["eps_oo"]
    sig[OW, OW] = p["sigma_oo"]
    return {"eps": eps, "sigma": sig}


# ---------------------------------------------------------------------------
# Position generators
# ---------------------------------------------------------------------------
def _rsa_positions(n: int, box: float, dmin: float, rng: np.random.Generator) -> np.ndarray:
    """Uniform random points in a periodic cube with a minimum image distance.

    Batched random sequential addition: candidates too close to an accepted
    point are dropped, and of two candidates too close to each other the later
    one is dropped.  Deterministic for a given generator state.
    """
    from scipy.spatial import cKDTree

    acc = np.zeros((0, 3))
    while acc.shape[0] < n:
        need = n - acc.shape[0]
        cand = rng.uniform(0.0, box, size=(max(64, int(need * 1.3)), 3))
        cand = np.minimum(cand, np.nextafter(box, 0.0))
        if acc.shape[0]:
            d, _ = cKDTree(acc, boxsize=box).query(cand, k=1)
            cand = cand[d >= dmin]
        if cand.shape[0] > 1:
            pairs = cKDTree(cand, boxsize=box).query_pairs(dmin, output_type="ndarray")
            if pairs.size:
                keep = np.ones(cand.shape[0], bool)
                # greedily keep the lower index of a conflicting pair
                for i, j in pairs[np.lexsort((pairs[:, 1], pairs[:, 0]))]:
                    if keep[i] and keep[j]:
                        keep[j] = False
                cand = cand[keep]
        acc = np.vstack([acc, cand[:need]])
    return acc


def maxwell_boltzmann(mass: np.ndarray, temperature: float, rng: np.random.Generator) -> np.ndarray:
    """Velocities (A/fs) at temperature T with zero net momentum."""
    sd = np.sqrt(KB_KCAL * temperature * ACCEL_CONV / mass)
    v = rng.standard_normal((mass.shape[0], 3)) * sd[:, None]
    p = (mass[:, None] * v).sum(0) / mass.sum()
    return v - p[None, :]


def nacl_melt(n_ions: int, box: float, seed: int, temperature: float = 1200.0,
              dmin: float = 2.0) -> System:
    """Molten NaCl: n_ions/2 Na+ and n_ions/2 Cl-, uniform random positions
    with minimum pair distance dmin, Maxwell-Boltzmann velocities."""
    if n_ions % 2:
        raise ValueError("n_ions must be even for a neutral NaCl melt")
    rng = np.random.default_rng(seed)
    pos = _rsa_positions(n_ions, box, dmin, rng)
    types = (np.arange(n_ions) % 2).astype(np.int32)
    charge = np.where(types == NA, 1.0, -1.0)
    mass = np.where(types == NA, MASS_NA, MASS_CL)
    vel = maxwell_boltzmann(mass, temperature, rng)
    return System(pos=pos, vel=vel, charge=charge, mass=mass, types=types, box=float(box),
                  sr_kind="bmh", sr_table=tosi_fumi_nacl())


def rocksalt_crystal(a: float, reps: int) -> System:
    """Perfect NaCl rock-salt crystal: conventional 8-ion cell of edge a,
    replicated reps^3 times (zero velocities)."""
    base = np.array([[0, 0, 0], [0, .5, .5], [.5, 0, .5], [.5, .5, 0]])
    na = base
    cl = base + np.array([.5, 0, 0])
    cell = np.vstack([na, cl])
    q = np.r_[np.ones(4), -np.ones(4)]
    shifts = np.array([[i, j, k] for i in range(reps) for j in range(reps) for k in range(reps)], float)
    pos = (cell[None, :, :] + shifts[:, None, :]).reshape(-1, 3) * a
    charge = np.tile(q, reps ** 3)
    types = np.where(charge > 0, NA, CL).astype(np.int32)
    mass = np.where(types == NA, MASS_NA, MASS_CL)
    return System(pos=pos, vel=np.zeros_like(pos), charge=charge, mass=mass, types=types,
                  box=float(a * reps), sr_kind="bmh", sr_table=tosi_fumi_nacl())


def random_neutral(n: int, box: float, seed: int, dmin: float = 1.0,
                   charge_scale: float = 1.0) -> System:
    """Small random neutral system with unequal random charges (sum exactly 0)."""
    rng = np.random.default_rng(seed)
    pos = _rsa_positions(n, box, dmin, rng)
    q = rng.uniform(-1.0, 1.0, n) * charge_scale
    q -= q.mean()
    # make the sum exactly zero in floating point
    q[-1] = -q[:-1].sum()
    mass = rng.uniform(10.0, 40.0, n)
    types = (np.arange(n) % 2).astype(np.int32)
    return System(pos=pos, vel=maxwell_boltzmann(mass, 300.0, rng), charge=q, mass=mass,
                  types=types, box=float(box), sr_kind="none", sr_table={})


def _random_rotations(n: int, rng: np.random.Generator) -> np.ndarray:
    """n uniformly random rotation matrices from unit quaternions."""
    qv = rng.standard_normal((n, 4))
    qv /= np.linalg.norm(qv, axis=1, keepdims=True)
    w, x, y, z = qv.T
    return np.stack([
        np.stack([1 - 2 * (y * y + z * z), 2 * (x * y - z * w), 2 * (x * z + y * w)], -1),
        np.stack([2 * (x * y + z * w), 1 - 2 * (x * x + z * z), 2 * (y * z - x * w)], -1),
        np.stack([2 * (x * z - y * w), 2 * (y * z + x * w), 1 - 2 * (x * x + y * y)], -1),
    ], 1)


def spcfw_water(n_mol: int, box: float, seed: int, temperature: float = 298.15,
                jitter: float = 0.2) -> System:
    """Flexible SPC/Fw water: molecules at the equilibrium geometry, centred on
    randomly chosen sites of a jittered cubic lattice, random orientations.
    Atom order per molecule is O, H, H."""
    rng = np.random.default_rng(seed)
    p = spcfw_params()
    m = int(math.ceil(n_mol ** (1.0 / 3.0) - 1e-9))
    sites = np.array([[i, j, k] for i in range(m) for j in range(m) for k in range(m)], float)
    sites = (sites + 0.5) * (box / m)
    sites = sites[rng.permutation(sites.shape[0])[:n_mol]]
    sites += rng.uniform(-jitter, jitter, sites.shape)
    half = 0.5 * p["theta0"]
    # molecule frame: O at origin, H in the xz plane
    local = np.array([[0.0, 0.0, 0.0],
                      [p["r0"] * math.sin(half), 0.0, p["r0"] * math.cos(half)],
                      [-p["r0"] * math.sin(half), 0.0, p["r0"] * math.cos(half)]])
    rot = _random_rotations(n_mol, rng)
    pos = sites[:, None, :] + np.einsum("mij,aj->mai", rot, local)
    pos = np.mod(pos.reshape(-1, 3), box)
    pos = np.where(pos >= box, 0.0, pos)
    types = np.tile(np.array([OW, HW, HW], np.int32), n_mol)
    charge = np.where(types == OW, p["q_o"], p["q_h"])
    mass = np.where(types == OW, MASS_O, MASS_H)
    vel = maxwell_boltzmann(mass, temperature, rng)
    base = 3 * np.arange(n_mol, dtype=np.int32)
    bonds = np.concatenate([np.stack([base, base + 1], 1), np.stack([base, base + 2], 1)])
    angles = np.stack([base + 1, base, base + 2], 1).astype(np.int32)
    return System(pos=pos, vel=vel, charge=charge, mass=mass, types=types, box=float(box),
                  sr_kind="lj", sr_table=spcfw_lj_table(), bonds=bonds.astype(np.int32),
                  angles=angles, bonded={"kb": p["kb"], "r0": p["r0"], "ka": p["ka"],
                                         "theta0": p["theta0"]},
                  molecule=np.repeat(np.arange(n_mol, dtype=np.int32), 3))


# ---------------------------------------------------------------------------
# Named workloads (sizes of this project's configurations)
# ---------------------------------------------------------------------------
WORKLOADS = {
    # molten NaCl, 512 ions, L = 25.2 A, mesh 32^3
    "nacl_512": dict(kind="nacl", n=512, box=25.2, mesh=32, seed=1, dt=1.0),
    # molten NaCl, 32768 ions, L = 100.9 A, mesh 128^3
    "nacl_32k": dict(kind="nacl", n=32768, box=100.9, mesh=128, seed=2, dt=1.0),
    # SPC/Fw water, 30000 molecules, L = 96.4 A, mesh 128^3
    "spcfw_30k": dict(kind="water", n=30000, box=96.4, mesh=128, seed=3, dt=0.5),
    # molten NaCl sweep at the melt density
    "nacl_4k": dict(kind="nacl", n=4096, box=50.45, mesh=64, seed=5, dt=1.0),
    "nacl_262k": dict(kind="nacl", n=262144, box=201.8, mesh=256, seed=6, dt=1.0),
    "nacl_1m": dict(kind="nacl", n=1000000, box=315.4, mesh=384, seed=7, dt=1.0),
}

EWALD_ALPHA = 0.30      # A^-1
R_CUT = 9.0             # A
TOL = 1e-6              # e per mesh point, max-norm constraint residual
ORDER = 4               # cubic B-spline assignment


def make_workload(name: str) -> tuple[System, dict]:
    w = WORKLOADS[name]
    if w["kind"] == "nacl":
        s = nacl_melt(w["n"], w["box"], w["seed"])
    else:
        s = spcfw_water(w["n"], w["box"], w["seed"])
    params = dict(alpha=EWALD_ALPHA, r_cut=R_CUT, mesh=w["mesh"], order=ORDER, tol=TOL,
                  dt=w["dt"])
    return s, params
