"""PMaZe, the comparison method with the whole Coulomb problem on the mesh
(Secs. 1-2), through the C ABI against the oracle's PMaZe at the GPU's own
positions.  Tolerances as in the P3MaZe parity tests: forces 1e-5 relative
RMS in FP64 and 1e-4 in mixed mode; the constraint (h/4pi) M phi + q = 0 to
tol with the oracle's stencil and the unsmoothed assigned charge."""
import numpy as np
import pytest

from oracle import p3maze_oracle as O
from paper_2606_31379_b300 import synth as S
from tests.parity_helpers import at_positions, constraint_residual, rel_rms

pytestmark = pytest.mark.gpu

MESH = 64          # h = 0.39 A: the full charge needs a finer mesh than P3MaZe's 32^3


@pytest.fixture(scope="module")
def P():
    from paper_2606_31379_b300 import p3maze
    return p3maze


@pytest.fixture(scope="module")
def nacl512():
    return S.nacl_melt(512, 25.2, seed=1)


def _ctx(P, system, **kw):
    args = dict(alpha=0.0, r_cut=9.0, mesh=MESH, tol=1e-10, dt=1.0, method="pmaze")
    args.update(kw)
    return P.Context.from_system(system, **args)


@pytest.mark.parametrize("precision, ftol", [("fp64", 1e-5), ("mixed", 1e-4)])
def test_pmaze_forces_and_energies_match_oracle(P, nacl512, precision, ftol):
    s = nacl512
    with _ctx(P, s, precision=precision) as ctx:
        pos = ctx.positions()
        ref = O.pmaze_forces_and_energies(at_positions(s, pos), 9.0, MESH)
        assert rel_rms(ctx.forces(), ref["F"]) < ftol
        assert rel_rms(ctx.forces("lr"), ref["F_mesh"]) < ftol
        assert rel_rms(ctx.forces("sr"), ref["F_vdw"]) < ftol
        st = ctx.stats()
        assert st["smooth_steps"] == 0 and st["sigma"] == 0.0
        e = ctx.energy()
        assert e["v_sr"] == 0.0 and e["v_self"] == 0.0
        etol = 1e-9 if precision == "fp64" else 1e-5
        assert e["v_vdw"] == pytest.approx(ref["v_vdw"], rel=etol)
        # 1/2 phi^T q: first order in the field error (tol 1e-10 against |q| ~ 0.1)
        assert e["v_lr"] == pytest.approx(ref["v_mesh"], rel=max(etol, 1e-7))
        q_ref = O.assign_charges(pos, s.charge, s.box, MESH)
        q = ctx.mesh("q")
        assert np.abs(q - q_ref).max() <= (1e-12 if precision == "fp64" else 1e-6) * np.abs(q_ref).max()
        # no smoothing: the source is q itself (reported with its mean removed)
        qtol = (1e-12 if precision == "fp64" else 1e-6) * np.abs(q).max()
        assert np.abs(ctx.mesh("qs") - (q - q.mean())).max() <= qtol
        # the constraint with the oracle's stencil and the GPU's own charge.
        # Mixed mode forms the charge term (4pi/h)(q - mean) in FP32 (two
        # roundings of 2^-24 each); with the whole charge on the mesh that is
        # far above tol, unlike P3MaZe's smoothed q^s (~1e-3 e per point)
        qc = q - q.mean()
        slack = 1e-11 if precision == "fp64" else 4.0 * 2.0 ** -24 * np.abs(qc).max()
        res = constraint_residual(ctx.mesh("phi"), qc, s.box / MESH)
        assert res <= 1e-10 * (1 + 1e-6) + slack


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_pmaze_steps_follow_velocity_verlet_and_conserve_momentum(P, nacl512, precision):
    s = nacl512
    acc = O.ACCEL / s.mass[:, None]
    # the net mesh force vanishes for the exact field; a field solved to tol
    # leaves q^T D (phi - phi*) (bound as in the P3MaZe momentum test)
    mom = 1e-7 if precision == "fp64" else 1e-5
    with _ctx(P, s, precision=precision) as ctx:
        for _ in range(3):
            r0, v0, F0 = ctx.positions(), ctx.velocities(), ctx.forces()
            ctx.step(1)
            r1, v1, F1 = ctx.positions(), ctx.velocities(), ctx.forces()
            vh = v0 + 0.5 * F0 * acc
            np.testing.assert_allclose(r1, O.wrap(r0 + vh, s.box), rtol=0, atol=1e-11)
            np.testing.assert_allclose(v1, vh + 0.5 * F1 * acc, rtol=1e-12, atol=1e-15)
            assert np.abs(ctx.forces("lr").sum(0)).max() < mom * np.abs(ctx.forces("lr")).max()
        ref = O.pmaze_forces_and_energies(at_positions(s, ctx.positions()), 9.0, MESH)
        assert rel_rms(ctx.forces(), ref["F"]) < (1e-5 if precision == "fp64" else 1e-4)
        st = ctx.stats()
        assert st["steps"] == 3 and st["last_residual"] <= 1e-10


def test_pmaze_rejects_molecules_and_the_analytic_force(P, nacl512):
    w = S.spcfw_water(27, 9.4, seed=3)
    with pytest.raises(P.P3MaZeError, match="topology"):
        P.Context.from_system(w, alpha=0.0, r_cut=4.5, mesh=32, tol=1e-6, dt=0.5, method="pmaze")
    with pytest.raises(P.P3MaZeError, match="finite-difference"):
        _ctx(P, nacl512, lr_force="analytic")
