"""sie_rcs_static, the allocation-free variant of sie_rcs, through the C ABI.

Both entry points run the same nested interior solve and far-field kernel.
With the near-region-only interior every product of that solve is
reproducible to the bit, so the cross sections agree up to the rounding of
the last step (host vs device evaluation of |N_perp(H) + rhat x N(E')|^2):
1e-12 of the largest value.  With the interior on the AIM grid (the
dielectric sphere) the interior L and K products project with FP64 atomic
additions, whose order varies from call to call; each call's nested solve
(tol_inner 1e-6) then ends on an iterate that differs at the rounding level
amplified by the solve (2e-11 of the largest value measured): 1e-9.  Two calls in a row with different direction sets check that nothing
left in the shared device array leaks into the next call.  The file is
collected last so that it also runs after every other GPU test.
"""
import ctypes

import numpy as np
import pytest

from synth import icosphere

pytestmark = pytest.mark.gpu

TOL = {"dielectric": 1e-9, "lossy": 1e-12}


def _dirs(n, seed):
    v = np.random.default_rng(seed).normal(size=(n, 3))
    return np.ascontiguousarray(v / np.linalg.norm(v, axis=1, keepdims=True))


def _static(lib, op, x, rhat):
    """sie_rcs_static called directly through ctypes (host x, host rhat, host out)."""
    out = np.zeros(len(rhat))
    code = lib.lib().sie_rcs_static(op.h, x.ctypes.data, rhat.ctypes.data, len(rhat), out.ctypes.data, 0)
    return code, out


class Solved:
    def __init__(self, lib, ctx, level, radius, f, eps_r, sigma):
        V, T = icosphere(level, radius, equal_volume=True)
        self.gm = lib.Mesh(ctx, V, T)
        self.op = lib.Operator(self.gm, f, eps_r, 1.0, sigma)
        # before any solve the interior workspace does not exist: refused, nothing launched
        code, _ = _static(lib, self.op, np.zeros(self.gm.ne + self.gm.nt, complex), _dirs(2, 0))
        self.code_before_solve = code
        b = self.op.rhs_planewave([0.0, 0.0, -1.0], [1.0, 0.0, 0.0])
        self.x, _, _ = self.op.solve(b)


@pytest.fixture(scope="module", params=["dielectric", "lossy"])
def solved(request, lib, ctx):
    """Dielectric sphere (eps_r 4, r 1 cm, 3 GHz; interior on the AIM grid with
    the nested constraint solver) and conductive sphere (1e4 S/m, r 1 mm,
    10 GHz; near-region-only interior), 320 triangles each."""
    if request.param == "dielectric":
        s = Solved(lib, ctx, 2, 0.01, 3e9, 4.0, 0.0)
    else:
        s = Solved(lib, ctx, 2, 1e-3, 10e9, 1.0, 1e4)
    s.tol = TOL[request.param]
    yield s
    s.op.close()
    s.gm.close()


def test_refused_before_workspace_exists(lib, solved):
    assert solved.code_before_solve == 7  # SIE_ERR_STATE
    assert "sie_solve" in lib.lib().sie_last_error().decode()


def test_two_calls_in_a_row_match_sie_rcs(lib, solved):
    op, x = solved.op, solved.x
    d1, d2 = _dirs(37, 1), _dirs(181, 2)
    c1, r1 = _static(lib, op, x, d1)
    c2, r2 = _static(lib, op, x, d2)
    assert c1 == 0 and c2 == 0
    ref1, ref2 = op.rcs(x, d1), op.rcs(x, d2)
    assert np.all(ref1 > 0) and np.all(ref2 > 0)
    assert np.abs(r1 - ref1).max() <= solved.tol * ref1.max()
    assert np.abs(r2 - ref2).max() <= solved.tol * ref2.max()
    # and once more through the binding, back to the first set
    r3 = op.rcs_static(x, d1)
    assert np.abs(r3 - ref1).max() <= solved.tol * ref1.max()


def test_maximum_direction_count(lib, solved):
    op, x = solved.op, solved.x
    n = lib.SIE_RCS_STATIC_MAX_DIR
    d = _dirs(n, 3)
    r = op.rcs_static(x, d)
    ref = op.rcs(x, d)
    assert np.abs(r - ref).max() <= solved.tol * ref.max()


def test_too_many_directions_is_an_error(lib, solved):
    op, x = solved.op, solved.x
    d = _dirs(lib.SIE_RCS_STATIC_MAX_DIR + 1, 4)
    code, _ = _static(lib, op, x, d)
    assert code == 1  # SIE_ERR_ARG
    assert "SIE_RCS_STATIC_MAX_DIR" in lib.lib().sie_last_error().decode()
    # the array is untouched by the refused call: the next call is still exact
    d1 = _dirs(5, 5)
    assert np.abs(op.rcs_static(x, d1) - op.rcs(x, d1)).max() <= solved.tol * op.rcs(x, d1).max()


def test_profiling_on_is_refused(lib, ctx, solved):
    op, x = solved.op, solved.x
    ctx.profile(True)
    try:
        code, _ = _static(lib, op, x, _dirs(3, 6))
    finally:
        ctx.profile(False)
    assert code == 7  # SIE_ERR_STATE


def _pool_bytes():
    """(used, reserved, used high-water mark) of device 0's default stream-ordered
    memory pool, read through the driver API (the pool every cudaMallocAsync of
    the library draws from), after the high-water mark is reset to the current
    use."""
    cu = ctypes.CDLL("libcuda.so.1")
    dev = ctypes.c_int()
    assert cu.cuDeviceGet(ctypes.byref(dev), 0) == 0
    pool = ctypes.c_void_p()
    assert cu.cuDeviceGetDefaultMemPool(ctypes.byref(pool), dev) == 0
    RESERVED_CURRENT, USED_CURRENT, USED_HIGH = 5, 7, 8

    def get(attr):
        v = ctypes.c_uint64()
        assert cu.cuMemPoolGetAttribute(pool, attr, ctypes.byref(v)) == 0
        return v.value

    def reset_high():
        z = ctypes.c_uint64(0)
        assert cu.cuMemPoolSetAttribute(pool, USED_HIGH, ctypes.byref(z)) == 0

    return get, reset_high, (RESERVED_CURRENT, USED_CURRENT, USED_HIGH)


def test_calls_allocate_no_device_memory(lib, solved):
    """Repeated calls leave the device allocations as they were: the pool's
    used and reserved bytes and its high-water mark do not move (a stream-ordered
    allocation and free inside a call would raise the mark), and neither does
    the device's free memory (plain cudaMalloc)."""
    import torch
    op, x = solved.op, solved.x
    d = _dirs(64, 9)
    op.rcs_static(x, d)  # first call on the device: symbol lookup done
    torch.cuda.synchronize()
    get, reset_high, (RES, USED, HIGH) = _pool_bytes()
    reset_high()
    used0, res0 = get(USED), get(RES)
    free0 = torch.cuda.mem_get_info()[0]
    for s in range(3):
        op.rcs_static(x, _dirs(64 + s, 10 + s))
    torch.cuda.synchronize()
    assert get(HIGH) == used0
    assert get(USED) == used0 and get(RES) == res0
    assert torch.cuda.mem_get_info()[0] == free0
