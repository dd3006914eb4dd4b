"""Parity of the CUDA AIM operators (through the C ABI) with the CPU oracle.

Tolerances:
  * grid geometry: N exact, spacing and origin to 1e-14 relative;
  * near-region CSR and AIM products vs the oracle's FP64 AIM product
    (same definitions, independent code): 1e-10 relative (FP64 rounding of
    different summation orders, FMA contraction, 2^k vs 2N FFT sizes);
  * AIM product vs the dense direct-integration oracle: 1e-3 relative 2-norm
    (the AIM approximation error the method accepts, Sec. IV).
"""
import numpy as np
import pytest

from oracle import aim, mom
from oracle.rwg import Mesh
from synth import cn_vector, icosphere

pytestmark = pytest.mark.gpu

C0 = 299792458.0
MU0 = 4e-7 * np.pi
EPS0 = 1.0 / (MU0 * C0 ** 2)


def k_medium(f, eps_r, sigma, mu_r=1.0):
    w = 2 * np.pi * f
    k = np.sqrt(w * MU0 * mu_r * (w * EPS0 * eps_r - 1j * sigma) + 0j)
    return -k if k.imag > 0 else k


def _csr_dense(rp, col, val, n):
    A = np.zeros((n, n), complex)
    for r in range(n):
        A[r, col[rp[r]:rp[r + 1]]] = val[rp[r]:rp[r + 1]]
    return A


class Case:
    def __init__(self, lib, ctx, level, radius, f, eps_r, sigma):
        V, T = icosphere(level, radius)
        self.m = Mesh(V, T)
        self.gm = lib.Mesh(ctx, V, T)
        self.op = lib.Operator(self.gm, f, eps_r, 1.0, sigma)
        self.k0 = 2 * np.pi * f / C0
        self.ki = k_medium(f, eps_r, sigma)
        self.g = aim.grid_params(self.m, M=2)


@pytest.fixture(scope="module")
def dielectric(lib, ctx):
    """Dielectric sphere, radius 1 cm, eps_r = 4, 3 GHz (config-1 material) on
    a 320-triangle icosphere: exterior and interior AIM operators."""
    c = Case(lib, ctx, 2, 0.01, 3e9, 4.0, 0.0)
    c.ext = aim.AIM(c.m, c.k0, c.g)
    c.inn = aim.AIM(c.m, c.ki, c.g)
    return c


def test_library_loaded(lib):
    import ctypes
    L = lib.lib()
    for s in lib.SYMBOLS:
        assert isinstance(getattr(L, s), ctypes._CFuncPtr)


def test_grid_matches_oracle(dielectric):
    o, h, N = dielectric.op.grid()
    g = dielectric.g
    assert np.array_equal(N, g.N)
    assert abs(h - g.h) <= 1e-14 * g.h
    assert np.abs(o - g.origin).max() <= 1e-14 * np.abs(g.origin).max()
    info = dielectric.op.info()
    assert info[7] == len(dielectric.ext.pairs)
    assert info[9] == 0.0  # dielectric interior uses the AIM grid


@pytest.mark.parametrize("which,attr,mat", [(0, "ext", "NL"), (1, "ext", "NK"), (2, "inn", "NL"), (3, "inn", "NK")])
def test_near_csr_matches_oracle(dielectric, which, attr, mat):
    c = dielectric
    rp, col, val = c.op.near_csr(which)
    ref = getattr(getattr(c, attr), mat).toarray()
    got = _csr_dense(rp, col, val, c.m.ne)
    assert np.array_equal(got != 0, ref != 0) or np.abs(got[ref == 0]).max() < 1e-300
    assert np.abs(got - ref).max() <= 1e-10 * np.abs(ref).max()


@pytest.mark.parametrize("which", [0, 1, 2, 3])
def test_aim_matvec_matches_oracle(dielectric, which):
    c = dielectric
    x = cn_vector(c.m.ne, 7 + which)
    y = c.op.matvec(which, x)
    A = c.ext if which < 2 else c.inn
    ref = A.L(x) if which % 2 == 0 else A.K(x)
    assert np.linalg.norm(y - ref) / np.linalg.norm(ref) <= 1e-10


def test_aim_matvec_device_pointers(lib, dielectric):
    import torch
    c = dielectric
    x = cn_vector(c.m.ne, 3)
    xd = torch.from_numpy(x).cuda()
    yd = torch.zeros_like(xd)
    c.op.matvec(0, xd, yd)
    torch.cuda.synchronize()
    assert np.array_equal(yd.cpu().numpy(), c.op.matvec(0, x)) or \
        np.linalg.norm(yd.cpu().numpy() - c.op.matvec(0, x)) <= 1e-13 * np.linalg.norm(yd.cpu().numpy())


def test_aim_matvec_vs_dense(dielectric):
    c = dielectric
    LA, Lp, K = mom.dense(c.m, c.k0)
    L = mom.L_full(c.m, LA, Lp, c.k0)
    x = cn_vector(c.m.ne, 21)
    for which, A in ((0, L), (1, K)):
        y = c.op.matvec(which, x)
        ref = A @ x
        assert np.linalg.norm(y - ref) / np.linalg.norm(ref) <= 1e-3


def test_multi_rhs(dielectric):
    c = dielectric
    X = cn_vector(c.m.ne, 5, nrhs=3)
    Y = c.op.matvec(0, X, nrhs=3)
    for r in range(3):
        y1 = c.op.matvec(0, np.ascontiguousarray(X[r]))
        assert np.linalg.norm(Y[r] - y1) <= 1e-13 * np.linalg.norm(y1)


@pytest.fixture(scope="module")
def lossy(lib, ctx):
    """Conductive sphere (sigma = 1e4 S/m, 10 GHz, radius 1 mm): 5 skin depths fit
    inside the near region, so the interior operator is near-region only."""
    c = Case(lib, ctx, 2, 1e-3, 10e9, 1.0, 1e4)
    delta = -1.0 / c.ki.imag
    c.inn = aim.NearOnly(c.m, c.ki, 5 * delta)
    return c


def test_near_only_interior(lossy):
    c = lossy
    assert c.op.info()[9] == 1.0
    assert c.op.info()[10] == len(c.inn.pairs)
    for which, mat in ((2, "NL"), (3, "NK")):
        rp, col, val = c.op.near_csr(which)
        got = _csr_dense(rp, col, val, c.m.ne)
        ref = getattr(c.inn, mat).toarray()
        assert np.abs(got - ref).max() <= 1e-10 * np.abs(ref).max()
        x = cn_vector(c.m.ne, 40 + which)
        y = c.op.matvec(which, x)
        r = c.inn.L(x) if which == 2 else c.inn.K(x)
        assert np.linalg.norm(y - r) / np.linalg.norm(r) <= 1e-10
