"""Several objects with their own materials (sie_mesh_create_objects,
sie_set_material; Sec. II: N_obj homogeneous objects, each interior problem
coupling only its own triangles).  Two spheres of different conductivity:

* Z' and the system product of Eq. (sys) against the oracle's several-object
  system (exterior AIM over both, block-diagonal near-only Z' by a sparse LU
  per object; and the SIBC variant), within 1e-10 (nested solve to 1e-13);
* Z' of the pair restricted to one sphere equals the one-object operator of
  that sphere alone (the other object does not enter its interior problem);
* host-side errors: an edge between objects, an object index out of range, a
  several-object operator whose interior needs an AIM grid.
"""
import numpy as np
import pytest

from oracle import aim, system
from oracle.rwg import Mesh
from synth import cn_vector, icosphere

pytestmark = pytest.mark.gpu

F = 10e9
MATS = [(1.0, 5.8e7), (1.0, 1e5)]


def _pair():
    Va, Ta = icosphere(1, 1e-3, equal_volume=True)
    Vb, Tb = icosphere(1, 0.7e-3, equal_volume=True)
    Vb = Vb + np.array([3e-3, 0.0, 0.0])
    V = np.vstack([Va, Vb])
    T = np.vstack([Ta, Tb + len(Va)])
    obj = np.concatenate([np.zeros(len(Ta), np.int32), np.ones(len(Tb), np.int32)])
    return V, T, obj, (Va, Ta)


@pytest.fixture(scope="module")
def pair(lib, ctx):
    V, T, obj, A = _pair()
    m = Mesh(V, T)
    gm = lib.Mesh(ctx, V, T, obj=obj)
    assert gm.nobj == 2
    for o, (er, sg) in enumerate(MATS):
        gm.set_material(o, er, 1.0, sg)
    ops = {model: lib.Operator(gm, F, 1.0, 1.0, 0.0, lib.params(tol_inner=1e-13, interior_model=code))
           for model, code in (("near", lib.SIE_GIBC), ("sibc", lib.SIE_SIBC))}
    g = aim.grid_params(m, M=2)
    yield m, gm, ops, obj, A, g
    for op in ops.values():
        op.close()
    gm.close()


@pytest.mark.parametrize("model", ["near", "sibc"])
def test_objects_impedance_and_system(lib, pair, model):
    m, gm, ops, obj, A, g = pair
    S = system.ObjectsGIBC(m, obj, MATS, F, g, interior=model)
    op = ops[model]
    H, rho = cn_vector(m.ne, 401), cn_vector(m.nt, 402)
    z = op.matvec(lib.SIE_OP_ZI, H)
    ref = S.Z(H)
    assert np.linalg.norm(z - ref) <= 1e-10 * np.linalg.norm(ref)
    y = op.matvec(lib.SIE_OP_SYS, np.concatenate([H, rho]))
    r1, r2 = S.apply(H, rho)
    assert np.linalg.norm(y[:m.ne] - r1) <= 1e-10 * np.linalg.norm(r1)
    assert np.linalg.norm(y[m.ne:] - r2) <= 1e-13 * np.linalg.norm(r2)


def test_objects_interior_is_per_object(lib, ctx, pair):
    m, gm, ops, obj, (Va, Ta), g = pair
    ga = lib.Mesh(ctx, Va, Ta)
    opa = lib.Operator(ga, F, MATS[0][0], 1.0, MATS[0][1], lib.params(tol_inner=1e-13))
    try:
        nea = ga.ne
        H = cn_vector(m.ne, 403)
        z = ops["near"].matvec(lib.SIE_OP_ZI, H)
        za = opa.matvec(lib.SIE_OP_ZI, np.ascontiguousarray(H[:nea]))
        assert np.linalg.norm(z[:nea] - za) <= 1e-10 * np.linalg.norm(za)
    finally:
        opa.close()
        ga.close()


def test_objects_errors(lib, ctx):
    V, T, obj, _ = _pair()
    bad = obj.copy()
    bad[0] = 1  # one triangle of sphere A assigned to B: its edges join two objects
    with pytest.raises(lib.SieError) as e:
        lib.Mesh(ctx, V, T, obj=bad)
    assert e.value.code == 2
    gm = lib.Mesh(ctx, V, T, obj=obj)
    try:
        with pytest.raises(lib.SieError) as e:
            gm.set_material(2, 1.0, 1.0, 0.0)
        assert e.value.code == 1
        gm.set_material(0, 4.0, 1.0, 0.0)  # a dielectric: its interior needs an AIM grid
        gm.set_material(1, 1.0, 1.0, 5.8e7)
        with pytest.raises(lib.SieError) as e:
            lib.Operator(gm, F, 1.0, 1.0, 0.0)
        assert e.value.code == 8
    finally:
        gm.close()
