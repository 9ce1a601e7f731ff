"""Shared helpers of the GPU parity tests: run the oracle at the GPU's own
state and compare."""
import copy

import numpy as np

from oracle import p3maze_oracle as O


def rel_rms(a, b):
    return float(np.sqrt(((a - b) ** 2).sum() / max((b ** 2).sum(), 1e-300)))


def at_positions(system, pos):
    s = copy.copy(system)
    s.pos = np.array(pos, dtype=np.float64)
    return s


def oracle_full(system, pos, alpha, r_cut, mesh):
    """Oracle forces and energies at the given positions (all particles)."""
    return O.forces_and_energies(at_positions(system, pos), alpha, r_cut, mesh)


def oracle_sampled(system, pos, alpha, r_cut, mesh, sample):
    """Oracle total force for the particles in `sample` and the full mesh
    fields; the short-range part is summed only for the sampled particles."""
    s = at_positions(system, pos)
    mf = O.mesh_fields(s, alpha, mesh)
    F_lr = O.interpolate_lr_forces(s.pos, s.charge, s.box, mesh, mf["phi"])
    F_sr, _, _ = O.sr_forces(s, mf["sigma"], r_cut, subset=sample)
    F = F_lr[sample] + F_sr
    if s.molecule is not None:
        Fb, _, _, _ = O.intramolecular_terms(s, mf["sigma"])
        F = F + Fb[sample]
    return F, mf, F_lr


def constraint_residual(phi, qs, h):
    """max_n |(h/4pi) (M phi)_n + q^s_n|: the constraint of Eq. 13 evaluated
    with the oracle's stencil."""
    return float(np.abs(h / (4 * np.pi) * O.laplacian7(phi) + qs).max())
