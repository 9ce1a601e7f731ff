"""Checkpoint/resume of the full stepping state and contexts that borrow
caller-owned device arrays, through the C ABI."""
import numpy as np
import pytest

from paper_2606_31379_b300 import synth as S

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def P():
    from paper_2606_31379_b300 import p3maze
    return p3maze


@pytest.fixture(scope="module")
def nacl512():
    return S.nacl_melt(512, 25.2, seed=1)


def _ctx(P, system, **kw):
    args = dict(alpha=0.30, r_cut=9.0, mesh=32, tol=1e-9, dt=1.0)
    args.update(kw)
    return P.Context.from_system(system, **args)


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_checkpoint_resume(P, nacl512, precision):
    """A context restored from a checkpoint reports exactly the saved state
    and continues like the original: positions, velocities, forces, energies
    and the field agree bit for bit right after the load, and after five more
    steps (every kernel of a step is deterministic)."""
    with _ctx(P, nacl512, precision=precision) as a, _ctx(P, nacl512, precision=precision, mesh=32) as b:
        a.step(8)
        blob = a.save_state()
        e_a, x_a, f_a, phi_a = a.energy(), a.positions(), a.forces(), a.mesh("phi")
        b.step(3)                                  # b is elsewhere before the load
        b.load_state(blob)
        assert b.stats()["steps"] == a.stats()["steps"] == 8
        np.testing.assert_array_equal(b.positions(), x_a)
        np.testing.assert_array_equal(b.velocities(), a.velocities())
        np.testing.assert_array_equal(b.forces(), f_a)
        np.testing.assert_array_equal(b.mesh("phi"), phi_a)
        e_b = b.energy()
        for k in ("total", "kinetic", "v_lr", "v_sr", "v_vdw"):
            assert e_b[k] == e_a[k], k
        a.step(5)
        b.step(5)
        np.testing.assert_array_equal(b.positions(), a.positions())
        np.testing.assert_array_equal(b.forces(), a.forces())
        assert b.stats()["steps"] == 13


def test_checkpoint_rejects_other_parameters(P, nacl512):
    with _ctx(P, nacl512, precision="fp64") as a, _ctx(P, nacl512, precision="fp64", mesh=24) as b:
        blob = a.save_state()
        with pytest.raises(P.P3MaZeError, match="other parameters|smaller"):
            b.load_state(blob)


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_borrowed_device_arrays(P, nacl512, precision):
    """p3maze_init_device: the context steps caller-owned device arrays in
    place; the result equals a context that owns copies of the same data."""
    import torch

    pos = torch.tensor(nacl512.pos, dtype=torch.float64, device="cuda")
    vel = torch.tensor(nacl512.vel, dtype=torch.float64, device="cuda")
    kw = dict(alpha=0.30, r_cut=9.0, mesh=32, tol=1e-9, dt=1.0, precision=precision,
              **P.system_kwargs(nacl512))
    with P.Context(nacl512.pos, nacl512.charge, nacl512.mass, nacl512.box, device_pos=pos.data_ptr(),
                   device_vel=vel.data_ptr(), **kw) as b, \
            P.Context(nacl512.pos, nacl512.charge, nacl512.mass, nacl512.box, **kw) as a:
        a.step(4)
        b.step(4)
        torch.cuda.synchronize()
        xb = pos.cpu().numpy()
        np.testing.assert_array_equal(xb, b.positions())       # the borrowed array is the state
        np.testing.assert_array_equal(vel.cpu().numpy(), b.velocities())
        np.testing.assert_array_equal(xb, a.positions())
    # the arrays outlive the context and keep the last state
    assert torch.isfinite(pos).all()


def test_borrowed_arrays_reject_nonfinite(P, nacl512):
    import torch

    pos = torch.tensor(nacl512.pos, dtype=torch.float64, device="cuda")
    vel = torch.tensor(nacl512.vel, dtype=torch.float64, device="cuda")
    vel[5, 2] = float("inf")
    with pytest.raises(P.P3MaZeError, match="non-finite"):
        P.Context(nacl512.pos, nacl512.charge, nacl512.mass, nacl512.box, device_pos=pos.data_ptr(),
                  device_vel=vel.data_ptr(), alpha=0.30, r_cut=9.0, mesh=32, tol=1e-6, dt=1.0,
                  **P.system_kwargs(nacl512))


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_programmatic_dependent_launch_switch(P, nacl512, precision, monkeypatch):
    """P3MAZE_PDL=0 (read at context creation) launches the chained mesh
    kernels plainly; both launch modes do the same arithmetic in the same
    order, so ten steps agree bit for bit, and so do the multigrid iteration
    counts."""
    monkeypatch.setenv("P3MAZE_PDL", "0")
    plain = _ctx(P, nacl512, precision=precision)
    monkeypatch.setenv("P3MAZE_PDL", "1")
    overlapped = _ctx(P, nacl512, precision=precision)
    try:
        plain.step(10)
        overlapped.step(10)
        np.testing.assert_array_equal(overlapped.positions(), plain.positions())
        assert overlapped.stats()["total_iters"] == plain.stats()["total_iters"]
    finally:
        plain.close()
        overlapped.close()
