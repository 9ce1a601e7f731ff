"""Host logic of the continuous-batching server, with a fake backend (no GPU):
admission by slots and memory, backfill, retirement after exactly the
requested steps, rejection of requests larger than the budget, metrics."""
import pytest

from paper_2606_31379_b300.serve import Request, Server, allowed_mesh, poisson_requests


class FakeBackend:
    """Virtual clock; a batch step costs 1 ms + 0.1 ms per member; preparing
    a new member (its context and 3 first steps) takes 1.5 ms on the
    admission worker, beside the stepping loop, and it joins when ready."""

    PREP = 1.5e-3

    def __init__(self, bytes_per_atom=1000):
        self.t = 0.0
        self.members = []
        self.steps = {}
        self.bpa = bytes_per_atom
        self.log = []
        self.inflight = []                     # (ready time, request)

    def clock(self):
        return self.t

    def estimate(self, req):
        return req.n_atoms * self.bpa

    def submit(self, req):
        # one admission worker: preparations run one after another
        start = max([self.t] + [t for t, _ in self.inflight])
        self.inflight.append((start + self.PREP, req))

    def poll(self, block=False):
        if block and self.inflight and all(t > self.t for t, _ in self.inflight):
            self.t = min(t for t, _ in self.inflight)
        ready = [(t, r) for t, r in self.inflight if t <= self.t]
        self.inflight = [(t, r) for t, r in self.inflight if t > self.t]
        return [(r, ("ctx", r.rid), self.PREP, None) for _, r in sorted(ready, key=lambda x: x[0])]

    def attach(self, h):
        self.members.append(h)
        self.steps[h] = 3
        self.log.append(("open", h[1], len(self.members)))

    def steps_done(self, h):
        return self.steps[h]

    def step(self):
        self.t += 1e-3 + 1e-4 * len(self.members)
        for h in self.members:
            self.steps[h] += 1
        return []

    def result(self, h):
        return {"steps": self.steps[h]}

    def close(self, h):
        self.members.remove(h)
        self.log.append(("close", h[1], len(self.members)))

    def sleep_until(self, t):
        self.t = max(self.t, t)


def test_every_request_finishes_with_exact_steps_within_budget_and_slots():
    reqs = poisson_requests(40, rate=400.0, seed=3, lo=216, hi=4000, steps=50)
    be = FakeBackend()
    srv = Server(be, budget_bytes=12_000_000, max_slots=6, margin=1.0, margin_bytes=0)
    m = srv.run(reqs)
    assert m["done"] == 40 and m["failed"] == 0 and m["rejected"] == 0
    for r in reqs:
        assert r.result["steps"] == 50
        assert len(r.step_latencies) == 50 - 3
        assert r.admitted >= r.arrival - 1e-12 and r.finished > r.admitted
    assert srv.peak_used <= 12_000_000 and srv.peak_slots <= 6 and srv.peak_resident <= 6
    assert m["step_latency_ms_p50"] <= m["step_latency_ms_p99"]
    assert m["steps_per_s"] > 0 and m["atom_steps_per_s"] > 0
    # systems overlap: at some point several were resident
    assert max(n for kind, _, n in be.log if kind == "open") > 1


def test_backfill_and_rejection():
    reqs = [Request(0, "nacl", 9000, 1, 20, 0.0),     # fits alone
            Request(1, "nacl", 8000, 2, 20, 0.0001),  # does not fit beside 0
            Request(2, "nacl", 500, 3, 20, 0.0002),   # backfills beside 0
            Request(3, "nacl", 50000, 4, 20, 0.0003)]  # larger than the budget
    be = FakeBackend()
    srv = Server(be, budget_bytes=10_000_000, max_slots=4, margin=1.0, margin_bytes=0)
    m = srv.run(reqs)
    assert reqs[3].status == "rejected" and m["rejected"] == 1
    assert all(r.status == "done" for r in reqs[:3])
    assert reqs[2].admitted < reqs[1].admitted          # passed the head that did not fit
    assert reqs[1].admitted >= reqs[0].finished - 1e-12  # waited for memory


def test_admission_overlaps_stepping():
    """While a newcomer is being prepared the resident systems keep stepping:
    a request arriving at t = 0.5 ms beside a running one joins 1.5 ms of
    preparation later, and the running system took steps in between."""
    reqs = [Request(0, "nacl", 1000, 1, 40, 0.0), Request(1, "nacl", 1000, 2, 20, 0.0005)]
    be = FakeBackend()
    srv = Server(be, budget_bytes=10_000_000, max_slots=4, margin=1.0, margin_bytes=0)
    m = srv.run(reqs)
    assert m["done"] == 2
    # request 1 was admitted about PREP after it was submitted, not after a stall of the loop
    assert reqs[1].admitted - reqs[1].arrival < FakeBackend.PREP + 3e-3
    # request 0 stepped while request 1 was being prepared
    steps_before = sum(1 for _ in reqs[0].step_latencies[:5])
    assert steps_before >= 1 and reqs[0].admitted < reqs[1].admitted
    assert m["admission_host_s_p50"] == pytest.approx(FakeBackend.PREP)


@pytest.mark.parametrize("target, n", [(15.2, 16), (16.0, 16), (23.6, 24), (33.0, 36), (126.0, 128), (300.0, 128)])
def test_allowed_mesh_sizes(target, n):
    assert allowed_mesh(target) == n
