"""The request loop on the GPU: every request gets the same answer when it runs
alone (one slot) and when it runs in a mix with others (three slots whose
work overlaps on the device, operators kept resident).  The only differences
are rounding (the grid projection accumulates with atomics), so with the
outer tolerance at 1e-8 the RCS agree to 1e-6 of their peak and the iteration
counts to within one.
"""
import numpy as np
import pytest

from synth import icosphere

pytestmark = pytest.mark.gpu


def _requests():
    from paper_2003_11679_gb300.serve import Request
    th = np.linspace(0.2, np.pi, 7)
    dirs = np.stack([np.sin(th), 0 * th, -np.cos(th)], 1)
    Vd, Td = icosphere(2, 0.01, equal_volume=True)
    Vl, Tl = icosphere(2, 1e-3, equal_volume=True)
    tight = {"tol_outer": 1e-8}
    return [
        Request(Vd, Td, 3e9, 4.0, 0.0, [0, 0, -1], [1, 0, 0], dirs, tight),   # dielectric: AIM interior
        Request(Vl, Tl, 10e9, 1.0, 1e4, [0, 0, -1], [1, 0, 0], dirs, tight),  # conductor: near-only interior
        Request(Vd, Td, 2e9, 2.5, 0.0, [1, 0, 0], [0, 0, 1], dirs, tight),    # other frequency and material
    ]


def test_results_same_alone_and_in_the_mix(lib):
    from paper_2003_11679_gb300.serve import Server
    reqs = _requests()
    with Server(slots=1) as srv:
        alone = [srv.submit(r).result(timeout=900) for r in reqs]
    with Server(slots=3) as srv:
        futs = [srv.submit(r) for r in reqs + reqs[1:2]]  # the conductor twice
        mixed = [f.result(timeout=900) for f in futs]
        st = srv.stats()
    for a, m in zip(alone + alone[1:2], mixed):
        print("iters", a["iters"], m["iters"], "slot", m["slot"])
        assert abs(a["iters"] - m["iters"]) <= 1
        assert np.abs(m["rcs"] - a["rcs"]).max() <= 1e-6 * np.abs(a["rcs"]).max()
    assert st["completed"] == 4 and st["p99_s"] >= st["p50_s"] > 0
    assert st.get("built", 0) + st.get("reused", 0) + st.get("batched", 0) == 4
    print(st)


def test_requests_of_one_operator_batched_same_as_alone(lib):
    """Cross-request batching: four requests of one operator (different plane
    waves, one of them with two) queued while the slot is busy are solved as
    one several-right-hand-side solve; each answer equals the one it gets
    alone, to the solver tolerance (1e-8) amplified by the conditioning."""
    from paper_2003_11679_gb300.serve import Request, Server
    reqs = _requests()
    Vl, Tl = icosphere(2, 1e-3, equal_volume=True)
    th = np.linspace(0.2, np.pi, 5)
    dirs = np.stack([np.sin(th), 0 * th, -np.cos(th)], 1)
    tight = {"tol_outer": 1e-8}
    waves = [([0, 0, -1], [1, 0, 0]), ([1, 0, 0], [0, 0, 1]), ([0, 1, 0], [1, 0, 0])]
    same = [Request(Vl, Tl, 10e9, 1.0, 1e4, kh, ep, dirs, tight) for kh, ep in waves]
    same.append(Request(Vl, Tl, 10e9, 1.0, 1e4, [[0, 0, 1], [0, -1, 0]], [[0, 1, 0], [0, 0, 1]], dirs, tight))
    with Server(slots=1) as srv:
        alone = [srv.submit(r).result(timeout=900) for r in same]
    with Server(slots=1) as srv:
        block = srv.submit(reqs[0])                     # keeps the slot busy meanwhile
        futs = [srv.submit(r) for r in same]
        mixed = [f.result(timeout=900) for f in futs]
        block.result(timeout=900)
        st = srv.stats()
    assert st.get("batched", 0) == 3 and mixed[0]["batch_rhs"] == 5
    for a, m in zip(alone, mixed):
        assert np.abs(np.asarray(m["rcs"]) - np.asarray(a["rcs"])).max() <= 1e-6 * np.abs(a["rcs"]).max()
        assert np.max(m["relres"]) < 1e-8
