"""bench.py's ports leg on CPU with a stand-in backend (no GPU).

The leg's bookkeeping: one row per (structure, interior model, frequency),
S from Y by the oracle's formula, the time per admittance matrix counted
over the solves that reached the tolerance only, the others counted as
stalled, and a line that JSON serialises.
"""
import json
import types

import numpy as np

import bench
from oracle import ports

Y = np.array([[1e-9 + 1e-4j, 2e-10 + 2e-5j], [2e-10 + 2e-5j, 1e-9 + 1e-4j]])


def _backend():
    be = types.SimpleNamespace(SIE_GIBC=0, SIE_SIBC=1)

    class Mesh:
        def __init__(self, ctx, V, T, obj=None):
            self.nobj = 1 if obj is None else int(np.max(obj)) + 1
            self.materials = []

        def set_material(self, o, eps_r, mu_r, sigma):
            self.materials.append((o, sigma))

        def close(self):
            pass

    class Operator:
        def __init__(self, mesh, f, eps_r, mu_r, sigma, prm):
            self.model, self.maxit = prm.interior_model, prm.maxit

        def port_admittance(self, pts, check=True):
            assert len(pts) == 2 and not check
            rr = np.array([5e-5, 6e-5]) if self.model == 1 else np.array([1e-2, 1e-2])
            return Y, np.array([12, 12], np.int32), rr

        def info(self):
            a = np.zeros(20)
            a[9] = 1.0
            return a

        def close(self):
            pass

    be.Mesh, be.Operator = Mesh, Operator
    be.params = lambda **kw: types.SimpleNamespace(tol_outer=1e-4, **{"maxit": 800, **kw})
    be.port_sparams = lambda y, z: ports.sparams(y, z)
    return be


def test_ports_leg_bookkeeping():
    out = bench.ports_stats(_backend(), None, types.SimpleNamespace(port_freqs=[50.0, 100.0]))
    rows = out["rows"]
    assert len(rows) == 2 * 2 * 2                      # structures x models x frequencies
    assert out["converged"] == 4 and out["stalled_at_maxit"] == 4   # the stand-in's GIBC never converges
    assert all(r["converged"] == (r["interior"] == "sibc") for r in rows)
    S = ports.sparams(Y, 50.0)
    assert np.allclose(rows[0]["S21"], [S[1, 0].real, S[1, 0].imag])
    assert rows[0]["reciprocity"] == 0.0
    json.dumps(out)
