"""Serving on the GPU: requests that arrive while others run are prepared on
the admission thread and join the batch, their work overlaps on the device,
and each result is the same alone and in the mix, bit for bit."""
import numpy as np
import pytest

from paper_2606_31379_b300.serve import GpuBackend, Request, Server, request_system

pytestmark = pytest.mark.gpu


def test_served_results_equal_results_alone():
    from paper_2606_31379_b300 import p3maze as P

    reqs = [Request(0, "nacl", 512, 11, 400, 0.00), Request(1, "water", 450, 12, 400, 0.00),
            Request(2, "nacl", 1200, 13, 400, 0.01), Request(3, "water", 900, 14, 400, 0.02),
            Request(4, "nacl", 300, 15, 400, 0.03)]
    be = GpuBackend(precision="fp64")
    try:
        m = Server(be, budget_bytes=8 << 30, max_slots=3).run(reqs)
    finally:
        be.shutdown()
    assert m["done"] == 5 and m["failed"] == 0 and m["rejected"] == 0
    assert m["peak_resident"] >= 2                    # several systems stepped together on the device
    for r in reqs:
        system, prm = request_system(r)
        with P.Context.from_system(system, precision="fp64", **prm) as ctx:
            ctx.step(r.steps)
            alone = ctx.positions()
        assert r.result["steps"] == r.steps
        np.testing.assert_array_equal(r.result["positions"], alone)   # deterministic kernels
    assert m["admission_host_s_p50"] > 0.0


def test_memory_budget_limits_admission():
    reqs = [Request(i, "nacl", 2000, 20 + i, 8, 0.0) for i in range(4)]
    be = GpuBackend(precision="mixed")
    try:
        need = Server(be, 1, 1)._need(reqs[0])
        srv = Server(be, budget_bytes=2 * need + need // 2, max_slots=8)
        m = srv.run(reqs)
    finally:
        be.shutdown()
    # two systems' memory reserved at a time (resident or being prepared), never three
    assert m["done"] == 4 and srv.peak_slots == 2 and srv.peak_used <= 2 * need + need // 2
