"""Host logic of the nested preconditioner for near-region-only interiors: the
sparse approximate inverse built at operator set-up (csrc/spai.cpp).

Each column j of M minimises ||A m_j - e_j||_2 over the sparsity pattern of
column j of A; the reference solves the same small least-squares problems with
numpy.  The matrix has the pattern of an RWG near region (edges sharing a
triangle or a vertex) and complex values with a dominant diagonal.
"""
import ctypes
import os
import shutil
import subprocess

import numpy as np
import pytest
import scipy.sparse as sp

from oracle.rwg import Mesh
from synth import icosphere

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CUDA = "/usr/local/cuda"


@pytest.fixture(scope="module")
def probe(tmp_path_factory):
    if shutil.which("g++") is None or not os.path.exists(os.path.join(CUDA, "include", "cuda_runtime.h")):
        pytest.skip("g++ or the CUDA headers are missing")
    so = str(tmp_path_factory.mktemp("spai") / "libspai_probe.so")
    cmd = ["g++", "-O2", "-std=c++17", "-fPIC", "-shared", "-I", os.path.join(CUDA, "include"),
           os.path.join(ROOT, "tests", "spai_probe.cpp"),
           os.path.join(ROOT, "paper_2003_11679_gb300", "csrc", "spai.cpp"),
           "-o", so, "-L", os.path.join(CUDA, "lib64"), "-lcudart", "-lpthread",
           "-Wl,-rpath," + os.path.join(CUDA, "lib64")]
    subprocess.run(cmd, check=True, capture_output=True)
    L = ctypes.CDLL(so)
    L.spai_probe.restype = ctypes.c_longlong
    L.spai_probe.argtypes = [ctypes.c_longlong] + [ctypes.c_void_p] * 4
    return L


def _near_matrix(seed):
    V, T = icosphere(2, 1.0)
    m = Mesh(V, T)
    # edges are neighbours when their supports share a vertex
    inc = sp.lil_matrix((m.ne, len(V)))
    for t in range(len(T)):
        for i in range(3):
            for v in T[t]:
                inc[m.tri_edge[t, i], v] = 1
    P = (inc.tocsr() @ inc.tocsr().T).tocsr()
    P.data[:] = 1
    rng = np.random.default_rng(seed)
    A = P.astype(complex)
    A.data = rng.normal(size=A.nnz) + 1j * rng.normal(size=A.nnz)
    A = ((A + A.T) * 0.05 + sp.diags(4.0 + 2.0j + rng.normal(size=m.ne))).tocsr()
    A.sort_indices()
    return A


def _reference(A):
    n = A.shape[0]
    Ac = A.tocsc()
    M = sp.lil_matrix(A.shape, dtype=complex)
    for j in range(n):
        J = A.indices[A.indptr[j]:A.indptr[j + 1]]
        sub = Ac[:, J]
        I = np.unique(sub.indices)
        mj = np.linalg.lstsq(sub[I, :].toarray(), (I == j).astype(complex), rcond=None)[0]
        for i, v in zip(J, mj):
            M[i, j] = v
    return M.tocsr()


def _run(probe, A):
    n = A.shape[0]
    rp = A.indptr.astype(np.int64)
    col = A.indices.astype(np.int32)
    val = np.ascontiguousarray(A.data.astype(complex))
    out = np.zeros_like(val)
    nbad = probe.spai_probe(n, rp.ctypes.data, col.ctypes.data, val.ctypes.data, out.ctypes.data)
    return nbad, sp.csr_matrix((out, col, rp), shape=A.shape)


def test_spai_matches_least_squares(probe):
    A = _near_matrix(3)
    nbad, M = _run(probe, A)
    assert nbad == 0
    ref = _reference(A)
    assert abs(M - ref).max() <= 1e-12 * abs(ref).max()
    # it is an approximate inverse: ||A M - I||_F well below ||I||_F
    R = (A @ M - sp.eye(A.shape[0])).toarray()
    assert np.linalg.norm(R) < 0.2 * np.sqrt(A.shape[0])


def test_spai_rejects_unsymmetric_pattern(probe):
    A = _near_matrix(4).tolil()
    A[0, A.shape[0] - 1] = 1.0  # (0, n-1) without (n-1, 0)
    A = A.tocsr()
    A.sort_indices()
    nbad, _ = _run(probe, A)
    assert nbad == -1
