"""Batched stepping (one graph launch advances every member by one MD step)
and the device-memory estimate used for admission."""
import numpy as np
import pytest

from paper_2606_31379_b300 import synth as S

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def P():
    from paper_2606_31379_b300 import p3maze
    return p3maze


def _systems():
    return [
        (S.nacl_melt(512, 25.2, seed=1), dict(mesh=32, r_cut=9.0, dt=1.0)),
        (S.nacl_melt(216, 18.9, seed=8), dict(mesh=24, r_cut=9.0, dt=1.0)),
        (S.spcfw_water(64, 12.42, seed=3), dict(mesh=16, r_cut=6.0, dt=0.5)),
    ]


def _cluster(P, c):
    """Select the cluster smoothing (mode 5; meshes of at most 64^3 default to
    the spectral mode); skip where the device runs no such clusters."""
    try:
        c.set_tuning(diffusion_fuse=5)
    except P.P3MaZeError:
        c.close()
        pytest.skip("the device does not run clusters of the smoothing kernel")
    return c


def _ctx(P, system, precision, **kw):
    return P.Context.from_system(system, alpha=0.30, tol=1e-9, precision=precision, **kw)


@pytest.mark.parametrize("precision, mode", [("fp64", "shared"), ("mixed", "shared"), ("fp64", "per_member"),
                                             ("mixed", "per_member")])
def test_each_result_is_the_same_alone_and_in_the_batch(P, precision, mode):
    """A member of a batch follows the same trajectory as the same system
    stepped alone, bit for bit: every kernel is deterministic and a member's
    kernels read only its own arrays."""
    total = 12
    alone = []
    for system, kw in _systems():
        with _ctx(P, system, precision, **kw) as c:
            c.step(total)
            alone.append((c.positions(), c.forces(), c.stats()["steps"]))
    ctxs = [_ctx(P, system, precision, **kw) for system, kw in _systems()]
    batch = P.Batch(mode=mode)
    try:
        for c in ctxs:
            batch.add(c)                      # each joins after its 3 warm-up steps
        assert len(batch) == 3
        batch.step(total - 3)
        batch.wait()
        for c, (pos, F, steps) in zip(ctxs, alone):
            assert c.stats()["steps"] == steps == total
            np.testing.assert_array_equal(c.positions(), pos)
            np.testing.assert_array_equal(c.forces(), F)
        # membership change: drop one, keep stepping, it can still step alone
        batch.remove(ctxs[1])
        batch.step(2)
        batch.wait()
        ctxs[1].step(1)
        assert ctxs[0].stats()["steps"] == total + 2 and ctxs[1].stats()["steps"] == total + 1
    finally:
        batch.close()
        for c in ctxs:
            c.close()


@pytest.mark.parametrize("mode, fused", [("shared", True), ("shared", False), ("per_member", True),
                                         ("per_member", False)])
def test_many_small_members_with_smaller_clusters_match_alone(P, mode, fused):
    """Twelve members of 16^3-24^3 meshes plus one 48^3 member smoothed per
    step: with the smoothing fused across members the batch smooths the
    small ones with 8-CTA clusters (at most one CTA per SM over the launch)
    where each alone uses 16; the neutrality sum is formed per plane in z
    order, so the trajectories are still those of each member alone, bit for
    bit, fused or not."""
    boxes = [12.8 + 3.2 * (i % 3) for i in range(12)]       # meshes 16, 20, 24 at 0.8 A
    systems = [(S.nacl_melt(2 * int(round(0.031899 * b ** 3 / 2)), b, seed=70 + i),
                dict(mesh=int(round(b / 0.8)), r_cut=6.0, dt=1.0)) for i, b in enumerate(boxes)]
    systems.append((S.nacl_melt(300, 21.1, seed=31), dict(mesh=48, r_cut=9.0, dt=1.0)))
    per_step = {len(systems) - 1}
    total = 9

    def make(i):
        system, kw = systems[i]
        c = _ctx(P, system, "mixed", **kw)
        if i in per_step:
            c.set_tuning(diffusion_fuse=2, diffusion_zc=2)
        else:
            _cluster(P, c)
        return c

    alone = []
    for i in range(len(systems)):
        with make(i) as c:
            c.step(total)
            alone.append(c.positions())
    ctxs = [make(i) for i in range(len(systems))]
    batch = P.Batch(mode=mode, fused_smoothing=fused)
    try:
        for c in ctxs:
            batch.add(c)
        batch.step(total - 3)
        batch.wait()
        for c, pos in zip(ctxs, alone):
            np.testing.assert_array_equal(c.positions(), pos)
    finally:
        batch.close()
        for c in ctxs:
            c.close()


@pytest.mark.parametrize("mode", ["shared", "per_member"])
def test_a_setting_changed_inside_the_batch_takes_effect(P, mode):
    """A member's smoothing mode changed while it is in the batch applies
    from the next batch step on: the trajectory equals the member stepped
    alone with the same change at the same step."""
    system, kw = _systems()[0]
    switch = dict(diffusion_fuse=2, diffusion_zc=2)
    with _cluster(P, _ctx(P, system, "mixed", **kw)) as c:
        c.step(6)
        c.set_tuning(**switch)
        c.step(4)
        ref = c.positions()
    others = [_ctx(P, s, "mixed", **k) for s, k in _systems()[1:]]
    ctx = _cluster(P, _ctx(P, system, "mixed", **kw))
    batch = P.Batch(mode=mode)
    try:
        for c in [ctx] + others:
            batch.add(c)
        batch.step(3)
        ctx.set_tuning(**switch)
        ctx.set_timing(True)
        batch.step(4)
        batch.wait()
        np.testing.assert_array_equal(ctx.positions(), ref)
        assert ctx.timing()["launches"]["smooth"] > 4          # per-step launches again
    finally:
        batch.close()
        for c in [ctx] + others:
            c.close()


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_device_bytes_estimate_matches_allocation(P, precision):
    for system, kw in _systems():
        est = P.device_bytes(system, alpha=0.30, tol=1e-6, precision=precision, **kw)
        with _ctx(P, system, precision, **kw) as c:
            assert c.stats()["device_bytes"] == est


def test_contexts_with_different_shared_memory_needs_coexist(P):
    """The coarse-solve kernels' shared-memory limit is per process: a context
    with a small need created after one with a large need must not lower it
    (an FP64 exact coarse solve on 48^3 stages 55 KB, above the 48 KB default;
    24^3 needs 14 KB)."""
    big = S.nacl_melt(300, 21.1, seed=31)
    small = S.nacl_melt(216, 18.9, seed=32)
    a = P.Context.from_system(big, alpha=0.30, r_cut=9.0, mesh=48, tol=1e-8, dt=1.0, precision="fp64",
                              coarse_max=64)
    b = P.Context.from_system(small, alpha=0.30, r_cut=9.0, mesh=24, tol=1e-8, dt=1.0, precision="fp64",
                              coarse_max=64)
    try:
        assert a.stats()["coarse_n"] == 48 and b.stats()["coarse_n"] == 24
        a.step(6)                      # graph steps of the 48^3 context after the 24^3 set-up
        b.step(6)
        assert a.stats()["steps"] == 6 and b.stats()["steps"] == 6
    finally:
        a.close()
        b.close()


def test_setup_is_ordered_on_the_context_stream(P):
    """A context created while the legacy default stream is busy starts from
    the same state as one created on an idle device: its setup copies and the
    clearing of the per-cell counts run on the context's own stream.  (A plain
    cudaMemset or pageable cudaMemcpy runs on the legacy default stream, which
    the context's non-blocking streams are not ordered after: the first cell
    list could be built from counts not yet cleared.)  4096 ions, so the cell
    list takes the multi-kernel builder with its count array."""
    import torch

    s = S.nacl_melt(4096, 50.45, seed=23)
    kw = dict(alpha=0.30, r_cut=9.0, mesh=64, tol=1e-8, dt=1.0, precision="mixed")
    with P.Context.from_system(s, **kw) as a:
        a.step(3)
        ref = a.forces()
    torch.cuda.synchronize()
    x = torch.randn(4096, 4096, device="cuda")
    for _ in range(40):                     # some tens of ms queued on the legacy default stream
        x = x @ x
        x = x / x.norm()
    with P.Context.from_system(s, **kw) as b:
        b.step(3)
        got = b.forces()
    torch.cuda.synchronize()
    assert np.array_equal(got, ref)
