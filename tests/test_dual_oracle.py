"""Pins of the oracle's dual (Buffa-Christiansen) basis (oracle/dual.py), CPU.

* The barycentric refinement is a closed, consistently oriented mesh of six
  triangles per coarse triangle with the coarse area and normals.
* Coarse RWG functions are fine Raviart-Thomas functions: the fine Gram
  matrix mapped back gives the coarse Gram matrix (closed forms on both
  meshes), and the divergence on every fine triangle is the coarse one.
* Each dual function lives on the dual cells of its edge's two vertices; all
  of its flux leaves the first cell and enters the second through the two
  fine edges of the dual edge, half a coefficient each.
* The property that defines the dual basis: paired with rotated RWG
  functions it gives a well-conditioned matrix, while the RWG / rotated-RWG
  pairing I_x of Eqs. (MFIE1dis), (EFIE01dis) is singular.
"""
import numpy as np
import pytest

from oracle import dual, mom
from oracle.rwg import Mesh
from synth import box, icosphere


def _scaled_cond(A):
    r = 1.0 / np.sqrt(np.einsum("ij,ij->i", A, A))
    c = 1.0 / np.sqrt(np.einsum("ij,ij->j", A, A))
    s = np.linalg.svd(r[:, None] * A * c[None, :], compute_uv=False)
    return s[0] / s[-1]


MESHES = {"sphere80": lambda: icosphere(1, 1.0), "sphere320": lambda: icosphere(2, 1.0),
          "cube54": lambda: box((1.0, 1.0, 1.0), (3, 3, 3)), "bar48": lambda: box((2.0, 1.0, 1.0), (4, 2, 2))}


@pytest.fixture(scope="module", params=list(MESHES))
def refined(request):
    m = Mesh(*MESHES[request.param]())
    fine, parent = dual.barycentric_refine(m)
    return request.param, m, fine, parent, dual.bc_matrix(m, fine), dual.rwg_in_fine(m, fine, parent)


def test_refinement(refined):
    _, m, fine, parent, _, _ = refined
    assert fine.nt == 6 * m.nt and fine.ne == 2 * m.ne + 6 * m.nt
    assert np.allclose(np.bincount(parent, weights=fine.area), m.area, rtol=1e-13)
    assert np.abs(fine.normal - m.normal[parent]).max() <= 1e-12


def test_coarse_rwg_exact_on_the_fine_mesh(refined):
    _, m, fine, parent, _, D = refined
    Gc = mom.gram(m)
    assert np.abs(D @ mom.gram(fine) @ D.T - Gc).max() <= 1e-13 * np.abs(Gc).max()
    div_f = (fine.incidence() @ D.T) / fine.area[:, None]      # fine triangle x coarse edge
    div_c = (m.incidence() / m.area[:, None])[parent]
    assert np.abs(div_f - div_c).max() <= 1e-12 * np.abs(div_c).max()


def test_dual_functions_flow_between_the_two_dual_cells(refined):
    _, m, fine, parent, C, _ = refined
    nv, ne = len(m.V), m.ne
    ev = dual.edge_vertices(m)
    out = fine.incidence() @ C.T                               # net outflow per fine triangle
    fl = fine.edge_len
    for e in range(ne):
        lo, hi = ev[e]
        around_lo = (fine.T == lo).any(1)
        around_hi = (fine.T == hi).any(1)
        # the two fine edges (m_e, c_T) of the dual edge
        half = 0.0
        for t in m.edge_tri[e]:
            f = np.nonzero((fine.T == nv + e).any(1) & (fine.T == nv + ne + t).any(1))[0][0]
            half += 0.5 * fl[dual._fine_edge_of(fine, f, nv + e, nv + ne + t)]
        assert abs(out[around_lo, e].sum() - half) <= 1e-12 * half
        assert abs(out[around_hi, e].sum() + half) <= 1e-12 * half
        assert np.abs(out[~(around_lo | around_hi), e]).max() == 0.0


def test_pairing_with_rotated_rwg_is_well_conditioned(refined):
    name, m, fine, parent, C, D = refined
    stable = -D @ mom.Ix(fine) @ C.T        # I (n x f_m) . g_n dS
    c_dual = _scaled_cond(stable)
    c_ix = _scaled_cond(mom.Ix(m))
    print(name, "cond <n x RWG, dual>", c_dual, "cond I_x", c_ix)
    assert c_dual < 5.0
    assert c_ix > 1e12
