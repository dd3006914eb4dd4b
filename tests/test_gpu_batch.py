"""Multi-right-hand-side AIM products (sie_matvec with nrhs > 1 on L0, K0, LI,
KI): blocks of up to 8 vectors that read the kernel spectra, the stencil
weights and the near-region values once per block.  Column by column against
the oracle's AIM products (1e-10, as for one vector) and against the
one-vector products (1e-13: only the order of the lane sums differs); 11
vectors make one full block and a ragged one."""
import numpy as np
import pytest

from oracle import aim, system
from oracle.rwg import Mesh
from synth import cn_vector, icosphere

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def diel(lib, ctx):
    V, T = icosphere(2, 0.01)
    m = Mesh(V, T)
    gm = lib.Mesh(ctx, V, T)
    op = lib.Operator(gm, 3e9, 4.0, 1.0, 0.0)
    g = aim.grid_params(m, M=2)
    k0 = 2 * np.pi * 3e9 / system.C0
    yield m, op, aim.AIM(m, k0, g), aim.AIM(m, system.k_medium(3e9, 4.0, 0.0), g)
    op.close()
    gm.close()


@pytest.mark.parametrize("which", [0, 1, 2, 3])
def test_block_products_match_oracle(lib, diel, which):
    m, op, ext, inn = diel
    R = 11
    X = cn_vector(m.ne, 300 + which, nrhs=R)
    Y = op.matvec(which, X, nrhs=R)
    A = ext if which < 2 else inn
    for r in range(R):
        ref = A.L(X[r]) if which % 2 == 0 else A.K(X[r])
        assert np.linalg.norm(Y[r] - ref) <= 1e-10 * np.linalg.norm(ref)
        one = op.matvec(which, np.ascontiguousarray(X[r]))
        assert np.linalg.norm(Y[r] - one) <= 1e-13 * np.linalg.norm(one)


def test_block_products_device_pointers(lib, diel):
    import torch
    m, op, ext, inn = diel
    X = cn_vector(m.ne, 310, nrhs=8)
    Xd = torch.from_numpy(X).cuda()
    Yd = torch.zeros_like(Xd)
    op.matvec(lib.SIE_OP_K0, Xd, Yd, nrhs=8)
    torch.cuda.synchronize()
    Yh = op.matvec(lib.SIE_OP_K0, X, nrhs=8)
    # the block projection scatters with atomics: the summation order of a grid
    # node's contributions differs between runs, each ~1e-16 relative
    Yd = Yd.cpu().numpy()
    for r in range(8):
        assert np.linalg.norm(Yd[r] - Yh[r]) <= 1e-13 * np.linalg.norm(Yh[r])


def test_block_products_near_only(lib, ctx):
    """Near-region-only interior operators (no grid): the CSR x panel product."""
    V, T = icosphere(1, 1e-3)
    m = Mesh(V, T)
    gm = lib.Mesh(ctx, V, T)
    op = lib.Operator(gm, 10e9, 1.0, 1.0, 1e4)
    try:
        assert op.info()[9] == 1.0
        ki = system.k_medium(10e9, 1.0, 1e4)
        no = aim.NearOnly(m, ki, 5.0 / abs(ki.imag))
        X = cn_vector(m.ne, 320, nrhs=5)
        for which, N in ((lib.SIE_OP_LI, no.NL), (lib.SIE_OP_KI, no.NK)):
            Y = op.matvec(which, X, nrhs=5)
            for r in range(5):
                ref = N @ X[r]
                assert np.linalg.norm(Y[r] - ref) <= 1e-10 * np.linalg.norm(ref)
    finally:
        op.close()
        gm.close()
