"""Seeded complex Gaussian vectors (circularly symmetric CN(0, 1))."""
import numpy as np


def cn_vector(n, seed, nrhs=1):
    """Return a complex128 array of shape (n,) or (nrhs, n) drawn from CN(0,1).

    Real and imaginary parts are independent N(0, 1/2) draws from numpy's PCG64
    generator seeded with ``seed``; the same seed always gives the same vector.
    """
    rng = np.random.Generator(np.random.PCG64(seed))
    shape = (n,) if nrhs == 1 else (nrhs, n)
    re = rng.standard_normal(shape)
    im = rng.standard_normal(shape)
    return ((re + 1j * im) / np.sqrt(2.0)).astype(np.complex128)
