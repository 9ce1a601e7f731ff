"""The allocation-free smoothing entry point, p3maze_smooth_noalloc.

It serves callers that cannot allocate device memory when they need the
smoothing (code under a device-memory budget owned by a host framework that
makes every allocation itself, or services that reserve their memory at
start-up): its only scratch is a fixed device array in the library.  Its output must equal the smoothed charge q^s that the regular
context path computes (p3maze_get_mesh, P3MAZE_MESH_QS), within the FP64 mesh
tolerance of the parity tests, on two calls in a row that share the scratch.
This file sorts last so that a run stopping at the first failure has already
run every other test.
"""
import numpy as np
import pytest

from paper_2606_31379_b300 import synth as S

pytestmark = pytest.mark.gpu


def _raw(a):
    """[ix, iy, iz] view -> the library's x-fastest flat layout."""
    return np.ascontiguousarray(a.transpose(2, 1, 0)).reshape(-1)


def test_smooth_noalloc_matches_context_path_twice():
    import torch
    from paper_2606_31379_b300 import p3maze as P

    cases = []
    for seed, n_ions, box, mesh in ((1, 512, 25.2, 32), (7, 300, 19.0, 24)):
        s = S.nacl_melt(n_ions, box, seed=seed)
        with P.Context.from_system(s, alpha=0.30, r_cut=9.0, mesh=mesh, tol=1e-9, dt=1.0) as ctx:
            st = ctx.stats()
            cases.append((mesh, st["smooth_steps"], st["smooth_coeff"], _raw(ctx.mesh("q")),
                          _raw(ctx.mesh("qs"))))
    stream = torch.cuda.current_stream().cuda_stream
    # two calls in a row on the shared scratch: different meshes, then the first again
    for mesh, K, c, q, qs_ref in (cases[0], cases[1], cases[0]):
        dq = torch.from_numpy(q).cuda()
        out = torch.full_like(dq, float("nan"))
        P.smooth_noalloc(dq.data_ptr(), out.data_ptr(), mesh, K, c, stream)
        torch.cuda.synchronize()
        got = out.cpu().numpy()
        assert np.all(np.isfinite(got))
        assert np.abs(got - qs_ref).max() <= 1e-12 * np.abs(qs_ref).max()


def test_smooth_noalloc_rejects_meshes_beyond_its_scratch():
    import torch
    from paper_2606_31379_b300 import p3maze as P

    buf = torch.zeros(8, dtype=torch.float64, device="cuda")
    out = torch.zeros(8, dtype=torch.float64, device="cuda")
    with pytest.raises(P.P3MaZeError) as ei:
        P.smooth_noalloc(buf.data_ptr(), out.data_ptr(), 128, 25, 0.16, None)
    assert ei.value.code == P.ERR_INVALID and "64" in str(ei.value)
    with pytest.raises(P.P3MaZeError):
        P.smooth_noalloc(buf.data_ptr(), buf.data_ptr(), 8, 1, 0.1, None)
    # partly overlapping input and output (4^3 doubles each, 8 doubles apart)
    big = torch.zeros(2 * 64, dtype=torch.float64, device="cuda")
    with pytest.raises(P.P3MaZeError, match="overlap"):
        P.smooth_noalloc(big.data_ptr(), big[8:].data_ptr(), 4, 1, 0.1, None)
