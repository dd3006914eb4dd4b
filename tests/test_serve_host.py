"""Host logic of the request loop (paper_2003_11679_gb300/serve.py) with a fake
backend: slots run requests at the same time, operators stay resident and
are reused, least recently used ones are released when device memory runs
short, and a request that can never fit is rejected.  No GPU is used.
"""
import threading
import time

import numpy as np
import pytest

from paper_2003_11679_gb300.serve import Request, Server


class Device:
    """One device's memory, shared by the fake backends of all slots."""

    def __init__(self, total):
        self.total, self.used, self.lock = total, 0, threading.Lock()


class FakeBackend:
    def __init__(self, dev, run_s=0.0):
        self.dev, self.run_s = dev, run_s

    def build(self, req):
        with self.dev.lock:
            self.dev.used += req.ne  # one byte per unknown
        return {"size": req.ne, "key": req.key()}

    def run(self, handle, req):
        time.sleep(self.run_s)
        return {"rcs": np.array([req.freq, req.sigma]), "iters": 1, "relres": 0.0}

    def release(self, handle):
        with self.dev.lock:
            self.dev.used -= handle["size"]

    def memory(self):
        with self.dev.lock:
            return self.dev.total - self.dev.used, self.dev.total

    def close(self):
        pass


def _req(ne, freq=1e9, sigma=0.0):
    V = np.zeros((3, 3))
    T = np.zeros((2, 3), np.int32)
    r = Request(V, T, freq, 1.0, sigma, [0, 0, -1], [1, 0, 0], [[0, 0, 1]])
    r.ne = ne
    return r


def test_slots_overlap_and_latency_stats():
    dev = Device(10 ** 9)
    with Server(slots=2, backend_factory=lambda s: FakeBackend(dev, run_s=0.2), bytes_per_unknown=1) as srv:
        t0 = time.perf_counter()
        futs = [srv.submit(_req(10, freq=1e9 * (i + 1))) for i in range(4)]
        outs = [f.result(timeout=30) for f in futs]
        wall = time.perf_counter() - t0
        st = srv.stats()
    assert wall < 0.75  # 4 requests of 0.2 s on 2 slots: two rounds, not four
    assert [o["rcs"][0] for o in outs] == [1e9, 2e9, 3e9, 4e9]
    assert {o["slot"] for o in outs} == {0, 1}
    assert st["completed"] == 4 and st["p99_s"] >= st["p50_s"] > 0


def test_resident_operator_is_reused():
    dev = Device(10 ** 9)
    with Server(slots=1, backend_factory=lambda s: FakeBackend(dev), bytes_per_unknown=1) as srv:
        srv.submit(_req(100)).result(timeout=30)
        srv.submit(_req(100)).result(timeout=30)
        srv.submit(_req(100, sigma=1.0)).result(timeout=30)
        st = srv.stats()
    assert st["built"] == 2 and st["reused"] == 1
    assert dev.used == 0  # close() released everything


def test_least_recently_used_operator_is_released():
    dev = Device(1000)  # reserve 10%: 900 usable
    with Server(slots=1, backend_factory=lambda s: FakeBackend(dev), bytes_per_unknown=1) as srv:
        srv.submit(_req(400, freq=1e9)).result(timeout=30)
        srv.submit(_req(400, freq=2e9)).result(timeout=30)
        srv.submit(_req(400, freq=1e9)).result(timeout=30)  # reuse: 1e9 becomes most recent
        srv.submit(_req(400, freq=3e9)).result(timeout=30)  # needs room: releases 2e9
        assert dev.used == 800
        srv.submit(_req(400, freq=1e9)).result(timeout=30)  # still resident
        st = srv.stats()
    assert st["evicted"] == 1 and st["reused"] == 2 and st["built"] == 3


def test_request_that_cannot_fit_is_rejected():
    dev = Device(1000)
    with Server(slots=2, backend_factory=lambda s: FakeBackend(dev), bytes_per_unknown=1) as srv:
        with pytest.raises(MemoryError):
            srv.submit(_req(950)).result(timeout=30)
        assert srv.submit(_req(100)).result(timeout=30)["iters"] == 1
        st = srv.stats()
    assert st["rejected"] == 1


def test_backend_failure_is_reported():
    def factory(slot):
        raise RuntimeError("no device")
    with pytest.raises(RuntimeError, match="no device"):
        Server(slots=2, backend_factory=factory)


def test_operator_is_shared_across_slots():
    """Two slots, many requests of one key: the operator is built once and used
    by both slots in turn (one cache; its context's lock keeps calls apart)."""
    dev = Device(10 ** 9)
    with Server(slots=2, backend_factory=lambda s: FakeBackend(dev, run_s=0.05), bytes_per_unknown=1) as srv:
        futs = [srv.submit(_req(100)) for _ in range(6)]
        outs = [f.result(timeout=30) for f in futs]
        st = srv.stats()
    # requests queued while the operator is in use join that solve (batched)
    assert st["built"] == 1 and st.get("reused", 0) + st.get("batched", 0) == 5
    assert all(o["iters"] == 1 for o in outs)
    assert dev.used == 0


def test_size_estimate_is_the_median():
    """Per-unknown operator sizes: the median of the measured builds, so one
    inflated sample does not raise the estimate."""
    dev = Device(10 ** 9)

    class Inflating(FakeBackend):
        n = 0

        def build(self, req):
            Inflating.n += 1
            with self.dev.lock:
                self.dev.used += req.ne * (50 if Inflating.n == 2 else 2)
            return {"size": req.ne * (50 if Inflating.n == 2 else 2), "key": req.key()}

    with Server(slots=1, backend_factory=lambda s: Inflating(dev), bytes_per_unknown=1) as srv:
        for f in (1e9, 2e9, 3e9):
            srv.submit(_req(100, freq=f)).result(timeout=30)
        assert srv.stats()["bytes_per_unknown"] == 2.0


class BatchingBackend(FakeBackend):
    """Records each batch it is given; answers per request."""

    def __init__(self, dev, run_s=0.0):
        super().__init__(dev, run_s)
        self.batches = []

    def run(self, handle, req):
        return self.run_batch(handle, [req])[0]

    def run_batch(self, handle, reqs):
        time.sleep(self.run_s)
        self.batches.append([r.khat[0, 0] for r in reqs])
        return [{"rcs": np.array([r.khat[0, 0], r.nrhs]), "iters": 1, "relres": 0.0} for r in reqs]


def _req_k(ne, freq, kx, nrhs=1):
    V = np.zeros((3, 3))
    T = np.zeros((2, 3), np.int32)
    kh = [[kx, 0.0, -1.0]] * nrhs if nrhs > 1 else [kx, 0.0, -1.0]
    ep = [[1.0, 0.0, 0.0]] * nrhs if nrhs > 1 else [1.0, 0.0, 0.0]
    r = Request(V, T, freq, 1.0, 0.0, kh, ep, [[0, 0, 1]])
    r.ne = ne
    return r


def test_queued_requests_of_one_operator_are_batched():
    """One slot busy on another operator: the three requests queued meanwhile
    for one operator are solved as one batch, each answered on its own; a
    request of a third operator is not mixed in."""
    dev = Device(10_000)
    be = []

    def factory(slot):
        b = BatchingBackend(dev, run_s=0.2)
        be.append(b)
        return b

    with Server(slots=1, backend_factory=factory, bytes_per_unknown=1) as srv:
        first = srv.submit(_req_k(10, 1e9, 0.5))
        time.sleep(0.05)
        same = [srv.submit(_req_k(10, 2e9, 0.1 * (i + 1))) for i in range(3)]
        other = srv.submit(_req_k(10, 3e9, 0.9))
        out = [f.result(timeout=10) for f in same]
        o = other.result(timeout=10)
        first.result(timeout=10)
        st = srv.stats()
    for i, r in enumerate(out):
        assert r["rcs"][0] == pytest.approx(0.1 * (i + 1))
    assert o["rcs"][0] == pytest.approx(0.9)
    assert st["batched"] == 2 and st["completed"] == 5
    assert sorted(len(b) for b in be[0].batches) == [1, 1, 3]


def test_batches_respect_the_right_hand_side_budget():
    """Requests of 3 plane waves each with max_batch_rhs = 8: two per batch."""
    dev = Device(10_000)
    be = []

    def factory(slot):
        b = BatchingBackend(dev, run_s=0.1)
        be.append(b)
        return b

    with Server(slots=1, backend_factory=factory, max_batch_rhs=8, bytes_per_unknown=1) as srv:
        block = srv.submit(_req_k(10, 1e9, 0.5))
        time.sleep(0.03)
        futs = [srv.submit(_req_k(10, 2e9, 0.1 * (i + 1), nrhs=3)) for i in range(4)]
        for f in futs:
            f.result(timeout=10)
        block.result(timeout=10)
    assert sorted(len(b) for b in be[0].batches) == [1, 2, 2]


def test_request_with_several_plane_waves():
    r = _req_k(10, 1e9, 0.3, nrhs=4)
    assert r.nrhs == 4 and not r.single
    with pytest.raises(ValueError):
        Request(np.zeros((3, 3)), np.zeros((2, 3), np.int32), 1e9, 1.0, 0.0, [[0, 0, 1], [0, 1, 0]], [1, 0, 0],
                [[0, 0, 1]])
