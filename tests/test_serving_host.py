"""The serving loop's scheduling on CPU, with the GPU work replaced by a
timed stand-in: admission by arrival and by the device-memory budget, every
request finished once, a failing request reported without stopping its slot."""
import threading
import time
from types import SimpleNamespace

import pytest

pytest.importorskip("torch")
from paper_2601_23002_gb300.serving import Server, summarize


class FakeServer(Server):
    """Plans of `cell.nbytes` bytes, `cell.work` seconds of service; a cell
    with `fail` set raises the way a failed allocation would."""

    def __init__(self, free_bytes, **kw):
        super().__init__(autotune=False, **kw)
        self.free = free_bytes
        self.peak = 0
        self.active = 0
        self.peak_active = 0
        self._probe = threading.Lock()

    def _slot_stream(self):
        return None

    def _free_bytes(self):
        return self.free

    def _plan_bytes(self, cell):
        return cell.nbytes

    def _serve_one(self, req, stream):
        with self._probe:
            self.peak = max(self.peak, self._committed)
            self.active += 1
            self.peak_active = max(self.peak_active, self.active)
        try:
            time.sleep(req.cell.work)
            if req.cell.fail:
                raise RuntimeError("out of memory (stand-in)")
            req.result = {"converged": True}
        finally:
            with self._probe:
                self.active -= 1


def _cells(sizes, work=0.01, fail=()):
    return [SimpleNamespace(n=32, nbytes=b, work=work, fail=(i in fail)) for i, b in enumerate(sizes)]


def test_admission_keeps_admitted_plans_within_the_memory_budget():
    sizes = [3, 5, 2, 6, 4, 1, 5, 3, 2, 6, 4, 3] * 2
    srv = FakeServer(free_bytes=10 + 100, reserve_bytes=100, slots=6)
    arrivals = [0.002 * i for i in range(len(sizes))]
    done = srv.run(arrivals, _cells(sizes))
    assert sorted(r.rid for r in done) == list(range(len(sizes)))
    assert srv.peak <= 10                          # never more than the budget admitted at once
    assert srv.peak_active >= 2                    # but requests did overlap
    for r in done:
        assert r.arrival <= r.admitted <= r.finished and not r.error
    s = summarize(done, srv.wall)
    assert s["requests"] == s["converged"] == len(sizes) and s["errors"] == 0
    assert s["p50_s"] <= s["p99_s"]


def test_requests_are_admitted_in_arrival_order():
    srv = FakeServer(free_bytes=1 << 40, reserve_bytes=0, slots=1)
    arrivals = [0.03, 0.0, 0.01, 0.02]
    done = srv.run(arrivals, _cells([1, 1, 1, 1], work=0.005))
    adm = sorted(done, key=lambda r: r.admitted)
    assert [r.arrival for r in adm] == sorted(arrivals)


@pytest.mark.timeout(120)       # before the fix a failed request stopped its slot and the run waited forever
def test_a_failing_request_is_reported_and_the_rest_complete():
    srv = FakeServer(free_bytes=1 << 40, reserve_bytes=0, slots=2)
    done = srv.run([0.0] * 6, _cells([1] * 6, fail=(2,)))
    assert len(done) == 6
    bad = [r for r in done if r.error]
    assert [r.rid for r in bad] == [2] and "RuntimeError" in bad[0].error
    assert summarize(done, srv.wall)["errors"] == 1


def test_a_request_larger_than_the_device_is_refused_up_front():
    srv = FakeServer(free_bytes=10, reserve_bytes=0, slots=2)
    with pytest.raises(ValueError):
        srv.run([0.0, 0.0], _cells([4, 11]))
