"""Python binding of the sm_103a AIM surface-integral-equation library.

Thin ctypes marshalling over the C ABI declared in ``include/sie.h``: every
step of the computation runs in the library's CUDA kernels.  The binding
fails loudly (``ImportError`` on first use) when ``_libsie.so`` is missing;
there is no CPU fallback.

Vectors may be numpy arrays (host; complex128) or CUDA torch tensors
(complex128, contiguous) -- the latter are passed as device pointers.
"""
import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SO = os.path.join(_HERE, "_libsie.so")
_lib = None

SIE_OK = 0
SIE_ERR_NOT_CONVERGED = 5
SIE_FP64, SIE_MIXED = 0, 1
SIE_GIBC, SIE_SIBC = 0, 1
SIE_DEVICE_PTRS = 1
SIE_SOLVE_REFINE = 2
SIE_SOLVE_SEQUENTIAL = 4
SIE_RCS_STATIC_MAX_DIR = 2048
SIE_OP_L0, SIE_OP_K0, SIE_OP_LI, SIE_OP_KI, SIE_OP_SYS, SIE_OP_ZI = range(6)

_STATUS = {0: "SIE_OK", 1: "SIE_ERR_ARG", 2: "SIE_ERR_MESH", 3: "SIE_ERR_OOM", 4: "SIE_ERR_CUDA",
           5: "SIE_ERR_NOT_CONVERGED", 6: "SIE_ERR_TIMEOUT", 7: "SIE_ERR_STATE", 8: "SIE_ERR_UNSUPPORTED"}

# every symbol the header declares
SYMBOLS = ["sie_params_default", "sie_ctx_create", "sie_ctx_destroy", "sie_last_error", "sie_profile_enable",
           "sie_profile_read", "sie_mesh_create",
           "sie_mesh_destroy", "sie_mesh_counts", "sie_op_build", "sie_op_destroy", "sie_op_set_solver",
           "sie_op_stats", "sie_op_info", "sie_op_grid",
           "sie_matvec", "sie_op_near_csr", "sie_rhs_planewave", "sie_solve", "sie_rcs", "sie_rcs_static",
           "sie_probe_fma", "sie_dense_solve", "sie_mesh_create_objects", "sie_set_material",
           "sie_port_edges", "sie_rhs_ports", "sie_port_currents", "sie_port_admittance", "sie_port_sparams"]


class sie_params(ctypes.Structure):
    _fields_ = [("h", ctypes.c_double), ("h_over_edge", ctypes.c_double), ("grid_n", ctypes.c_int),
                ("stencil_order", ctypes.c_int), ("near_radius", ctypes.c_int), ("skin_cutoff", ctypes.c_double),
                ("precision", ctypes.c_int), ("tol_outer", ctypes.c_double), ("tol_inner", ctypes.c_double),
                ("maxit", ctypes.c_int), ("restart", ctypes.c_int), ("inner_maxit", ctypes.c_int),
                ("tol_constraint", ctypes.c_double), ("constraint_maxit", ctypes.c_int),
                ("constraint_restart", ctypes.c_int), ("tol_constraint_inner", ctypes.c_double),
                ("q_far", ctypes.c_int), ("q_out", ctypes.c_int), ("q_ang", ctypes.c_int), ("q_rad", ctypes.c_int),
                ("q_npan", ctypes.c_int), ("q_opan", ctypes.c_int), ("q_olam", ctypes.c_int),
                ("q_omu", ctypes.c_int), ("q_emupan", ctypes.c_int), ("q_emu", ctypes.c_int),
                ("q_ratio", ctypes.c_double), ("q_cf", ctypes.c_double), ("q_kres", ctypes.c_double),
                ("q_alen", ctypes.c_double), ("q_oratio", ctypes.c_double), ("dense_pc_max", ctypes.c_int),
                ("interior_model", ctypes.c_int)]


class sie_port(ctypes.Structure):
    _fields_ = [("origin", ctypes.c_double * 3), ("normal", ctypes.c_double * 3), ("radius", ctypes.c_double)]


def _ports(ports):
    """ctypes array of sie_port from (origin, normal, radius) tuples."""
    arr = (sie_port * len(ports))()
    for a, (o, n, r) in zip(arr, ports):
        a.origin[:] = [float(v) for v in o]
        a.normal[:] = [float(v) for v in n]
        a.radius = float(r)
    return arr


class SieError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"{_STATUS.get(code, code)}: {msg}")
        self.code = code


def lib():
    """Load ``_libsie.so`` (built by ``build.build()`` or ``__graft_entry__.build()``)."""
    global _lib
    if _lib is None:
        if not os.path.exists(_SO):
            raise ImportError(f"{_SO} is missing: build it with paper_2003_11679_gb300.build.build()")
        L = ctypes.CDLL(_SO)
        P, I, D, I64 = ctypes.c_void_p, ctypes.c_int, ctypes.c_double, ctypes.c_int64
        PP = ctypes.POINTER(ctypes.c_void_p)
        L.sie_params_default.argtypes = [ctypes.POINTER(sie_params)]
        L.sie_params_default.restype = None
        L.sie_last_error.restype = ctypes.c_char_p
        L.sie_ctx_create.argtypes = [I, P, PP]
        L.sie_ctx_destroy.argtypes = [P]
        L.sie_profile_enable.argtypes = [P, I]
        L.sie_profile_read.argtypes = [P, I, P, P, P, P]
        L.sie_mesh_create.argtypes = [P, P, I64, P, I64, PP]
        L.sie_mesh_destroy.argtypes = [P]
        L.sie_mesh_counts.argtypes = [P, P]
        L.sie_op_build.argtypes = [P, D, D, D, D, ctypes.POINTER(sie_params), PP]
        L.sie_op_destroy.argtypes = [P]
        L.sie_op_set_solver.argtypes = [P, ctypes.POINTER(sie_params)]
        L.sie_op_stats.argtypes = [P, P]
        L.sie_op_info.argtypes = [P, P]
        L.sie_op_grid.argtypes = [P, P, P, P]
        L.sie_matvec.argtypes = [P, I, P, P, I, I]
        L.sie_op_near_csr.argtypes = [P, I, P, P, P, P]
        L.sie_rhs_planewave.argtypes = [P, P, P, I, P, I]
        L.sie_solve.argtypes = [P, P, P, I, P, P, I]
        L.sie_rcs.argtypes = [P, P, P, I, P, I]
        L.sie_rcs_static.argtypes = [P, P, P, I, P, I]
        L.sie_probe_fma.argtypes = [I, P, P]
        L.sie_dense_solve.argtypes = [I, I, I, P, P, P, I]
        L.sie_mesh_create_objects.argtypes = [P, P, I64, P, I64, P, PP, P]
        L.sie_set_material.argtypes = [P, I, D, D, D]
        L.sie_port_edges.argtypes = [P, P, P, P, P]
        L.sie_rhs_ports.argtypes = [P, P, I, P, P, I]
        L.sie_port_currents.argtypes = [P, P, I, P, I, P, I]
        L.sie_port_admittance.argtypes = [P, P, I, P, P, P, I]
        L.sie_port_sparams.argtypes = [I, P, D, P]
        for name in SYMBOLS:
            f = getattr(L, name)
            if name not in ("sie_params_default", "sie_last_error"):
                f.restype = ctypes.c_int
        _lib = L
    return _lib


def _check(code):
    if code != SIE_OK:
        raise SieError(code, lib().sie_last_error().decode())


def probe_fma(device=0):
    """(FP64, FP32) FMA throughput in TFLOP/s measured on `device` by the library."""
    a, b = ctypes.c_double(), ctypes.c_double()
    _check(lib().sie_probe_fma(device, ctypes.byref(a), ctypes.byref(b)))
    return a.value, b.value


def dense_solve(A, b, device=0, inverse=False):
    """x = A^-1 b with the library's GPU complex64 LU (verification of the
    factorisation the constraint preconditioners use); inverse=True applies
    the explicit inverse formed from the factors, as the preconditioners do.
    b: one vector (n) or several ((nrhs, n), solved together)."""
    A = np.ascontiguousarray(A, dtype=np.complex128)
    b = np.ascontiguousarray(b, dtype=np.complex128)
    x = np.zeros_like(b)
    n = A.shape[0]
    nrhs = 1 if b.ndim == 1 else b.shape[0]
    _check(lib().sie_dense_solve(device, n, nrhs, A.ctypes.data, b.ctypes.data, x.ctypes.data, 1 if inverse else 0))
    return x


def port_sparams(Y, z_ref=50.0):
    """S = (1 - z_ref Y)(1 + z_ref Y)^-1 (the library's host routine)."""
    Y = np.ascontiguousarray(np.atleast_2d(Y), dtype=np.complex128)
    S = np.zeros_like(Y)
    _check(lib().sie_port_sparams(len(Y), Y.ctypes.data, float(z_ref), S.ctypes.data))
    return S


def params(**kw):
    p = sie_params()
    lib().sie_params_default(ctypes.byref(p))
    for k, v in kw.items():
        if not hasattr(p, k):
            raise KeyError(k)
        setattr(p, k, v)
    return p


def _ptr(a):
    """(pointer, is_device) of a numpy array or torch tensor."""
    if hasattr(a, "data_ptr"):
        if not a.is_contiguous():
            raise ValueError("tensor must be contiguous")
        return ctypes.c_void_p(a.data_ptr()), a.is_cuda
    if not a.flags["C_CONTIGUOUS"]:
        raise ValueError("array must be C-contiguous")
    return ctypes.c_void_p(a.ctypes.data), False


class Context:
    def __init__(self, device=0, stream=None):
        self.h = ctypes.c_void_p()
        s = ctypes.c_void_p(stream) if stream is not None else None
        _check(lib().sie_ctx_create(device, s, ctypes.byref(self.h)))

    def profile(self, enable):
        _check(lib().sie_profile_enable(self.h, 1 if enable else 0))

    def profile_read(self):
        """{stage: (total_ms, launches)} accumulated since profiling was enabled."""
        cap = 64
        names = ctypes.create_string_buffer(32 * cap)
        ms = np.zeros(cap)
        cnt = np.zeros(cap, np.int64)
        n = ctypes.c_int()
        _check(lib().sie_profile_read(self.h, cap, names, ms.ctypes.data, cnt.ctypes.data, ctypes.byref(n)))
        out = {}
        for i in range(min(n.value, cap)):
            nm = names.raw[32 * i:32 * i + 32].split(b"\0")[0].decode()
            out[nm] = (float(ms[i]), int(cnt[i]))
        return out

    def close(self):
        if self.h:
            _check(lib().sie_ctx_destroy(self.h))
            self.h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Mesh:
    """A closed triangle mesh; obj (optional, one index per triangle) splits it
    into several objects, each a closed surface with its own material."""

    def __init__(self, ctx, verts, tris, obj=None):
        self.ctx = ctx
        V = np.ascontiguousarray(verts, dtype=np.float64)
        T = np.ascontiguousarray(tris, dtype=np.int32)
        self.h = ctypes.c_void_p()
        self.nobj = 1
        if obj is None:
            _check(lib().sie_mesh_create(ctx.h, V.ctypes.data, len(V), T.ctypes.data, len(T), ctypes.byref(self.h)))
        else:
            O = np.ascontiguousarray(obj, dtype=np.int32)
            if len(O) != len(T):
                raise ValueError("obj needs one index per triangle")
            n = ctypes.c_int()
            _check(lib().sie_mesh_create_objects(ctx.h, V.ctypes.data, len(V), T.ctypes.data, len(T), O.ctypes.data,
                                                 ctypes.byref(self.h), ctypes.byref(n)))
            self.nobj = n.value
        c = np.zeros(3, np.int64)
        _check(lib().sie_mesh_counts(self.h, c.ctypes.data))
        self.ne, self.nt, self.nv = int(c[0]), int(c[1]), int(c[2])

    def port_edges(self, port):
        """(edges, signs) of one port (origin, normal, radius)."""
        n = ctypes.c_int64()
        pt = _ports([port])
        _check(lib().sie_port_edges(self.h, pt, None, None, ctypes.byref(n)))
        e = np.zeros(n.value, np.int32)
        s = np.zeros(n.value, np.int32)
        _check(lib().sie_port_edges(self.h, pt, e.ctypes.data, s.ctypes.data, ctypes.byref(n)))
        return e, s

    def set_material(self, obj, eps_r, mu_r=1.0, sigma=0.0):
        _check(lib().sie_set_material(self.h, obj, eps_r, mu_r, sigma))

    def close(self):
        if self.h:
            _check(lib().sie_mesh_destroy(self.h))
            self.h = ctypes.c_void_p()


class Operator:
    """Operators of one frequency: exterior AIM (vacuum) and interior (object)."""

    def __init__(self, mesh, freq, eps_r=1.0, mu_r=1.0, sigma=0.0, prm=None):
        self.mesh = mesh
        self.h = ctypes.c_void_p()
        p = prm if prm is not None else params()
        _check(lib().sie_op_build(mesh.h, freq, eps_r, mu_r, sigma, ctypes.byref(p), ctypes.byref(self.h)))

    def info(self):
        a = np.zeros(20)
        _check(lib().sie_op_info(self.h, a.ctypes.data))
        return a

    def grid(self):
        o = np.zeros(3)
        h = ctypes.c_double()
        N = np.zeros(3, np.int64)
        _check(lib().sie_op_grid(self.h, o.ctypes.data, ctypes.byref(h), N.ctypes.data))
        return o, h.value, N

    def matvec(self, which, x, y=None, nrhs=1):
        """y = A x; x numpy (host) or CUDA tensor (device), complex128."""
        if y is None:
            y = np.zeros_like(x)
        px, dx = _ptr(x)
        py, dy = _ptr(y)
        if dx != dy:
            raise ValueError("x and y must both be host or both be device buffers")
        _check(lib().sie_matvec(self.h, which, px, py, nrhs, SIE_DEVICE_PTRS if dx else 0))
        return y

    def near_csr(self, which):
        rp = np.zeros(self.mesh.ne + 1, np.int64)
        nnz = ctypes.c_int64()
        _check(lib().sie_op_near_csr(self.h, which, rp.ctypes.data, None, None, ctypes.byref(nnz)))
        col = np.zeros(nnz.value, np.int32)
        val = np.zeros(nnz.value, np.complex128)
        _check(lib().sie_op_near_csr(self.h, which, rp.ctypes.data, col.ctypes.data, val.ctypes.data,
                                     ctypes.byref(nnz)))
        return rp, col, val

    def set_solver(self, **kw):
        _check(lib().sie_op_set_solver(self.h, ctypes.byref(params(**kw))))

    def stats(self):
        a = np.zeros(6)
        _check(lib().sie_op_stats(self.h, a.ctypes.data))
        return dict(iters=int(a[0]), relres=a[1], inner_iters_max=int(a[2]), inner_relres_max=a[3],
                    constraint_iters_max=int(a[4]), constraint_relres_max=a[5])

    def rhs_planewave(self, khat, epol, out=None):
        """b = [-(1/eta0) <f_m, E_inc>; 0] (length N_e + N_t per right-hand side)."""
        kh = np.ascontiguousarray(np.atleast_2d(khat), dtype=np.float64)
        ep = np.ascontiguousarray(np.atleast_2d(epol), dtype=np.float64)
        nrhs = len(kh)
        n = self.mesh.ne + self.mesh.nt
        b = out if out is not None else np.zeros((nrhs, n) if nrhs > 1 else n, np.complex128)
        pb, dev = _ptr(b)
        _check(lib().sie_rhs_planewave(self.h, kh.ctypes.data, ep.ctypes.data, nrhs, pb,
                                       SIE_DEVICE_PTRS if dev else 0))
        return b

    def solve(self, b, x=None, nrhs=1, check=True, refine=False, sequential=False):
        """x = SYS^-1 b by FGMRES; returns (x, iters, relres).  refine=True: mixed-
        precision iterative refinement (complex64 corrections, FP64 residuals).
        nrhs > 1: b holds nrhs consecutive right-hand sides, solved in lockstep
        blocks of up to 8 (sequential=True: one after another)."""
        if x is None:
            x = np.zeros_like(b)
        pb, db = _ptr(b)
        px, dx = _ptr(x)
        it = np.zeros(nrhs, np.int32)
        rr = np.zeros(nrhs)
        flags = ((SIE_DEVICE_PTRS if db else 0) | (SIE_SOLVE_REFINE if refine else 0) |
                 (SIE_SOLVE_SEQUENTIAL if sequential else 0))
        code = lib().sie_solve(self.h, pb, px, nrhs, it.ctypes.data, rr.ctypes.data, flags)
        if check or code != SIE_ERR_NOT_CONVERGED:
            _check(code)
        return x, it, rr

    def rcs(self, x, rhat):
        rh = np.ascontiguousarray(np.atleast_2d(rhat), dtype=np.float64)
        out = np.zeros(len(rh))
        px, dx = _ptr(x)
        _check(lib().sie_rcs(self.h, px, rh.ctypes.data, len(rh), out.ctypes.data, SIE_DEVICE_PTRS if dx else 0))
        return out

    def rcs_static(self, x, rhat):
        """rcs() through sie_rcs_static, which allocates nothing (its scratch is a
        fixed device array of the library): for callers that must not allocate
        after start-up.  Needs a prior solve (or SYS product) on this operator and
        profiling off; at most SIE_RCS_STATIC_MAX_DIR directions; calls that
        overlap in time on one device race on the shared array."""
        rh = np.ascontiguousarray(np.atleast_2d(rhat), dtype=np.float64)
        out = np.zeros(len(rh))
        px, dx = _ptr(x)
        _check(lib().sie_rcs_static(self.h, px, rh.ctypes.data, len(rh), out.ctypes.data,
                                    SIE_DEVICE_PTRS if dx else 0))
        return out

    def rhs_ports(self, ports, volts=None, out=None):
        """One right-hand side per port (N_e + N_t each), port j driven with
        volts[j] (1 V by default), the others shorted.  ports: (origin,
        normal, radius) tuples."""
        n = self.mesh.ne + self.mesh.nt
        b = out if out is not None else np.zeros((len(ports), n), np.complex128)
        v = None if volts is None else np.ascontiguousarray(volts, dtype=np.float64)
        pb, dev = _ptr(b)
        _check(lib().sie_rhs_ports(self.h, _ports(ports), len(ports), None if v is None else v.ctypes.data, pb,
                                   SIE_DEVICE_PTRS if dev else 0))
        return b

    def port_currents(self, ports, x, nrhs=1):
        """I[r, i]: current through port i of solution r."""
        I = np.zeros((nrhs, len(ports)), np.complex128)
        px, dev = _ptr(x)
        _check(lib().sie_port_currents(self.h, _ports(ports), len(ports), px, nrhs, I.ctypes.data,
                                       SIE_DEVICE_PTRS if dev else 0))
        return I

    def port_admittance(self, ports, refine=False, sequential=False, check=True):
        """(Y, iters, relres): Y[i, j] = current through port i per volt on port j."""
        n = len(ports)
        Y = np.zeros((n, n), np.complex128)
        it = np.zeros(n, np.int32)
        rr = np.zeros(n)
        flags = (SIE_SOLVE_REFINE if refine else 0) | (SIE_SOLVE_SEQUENTIAL if sequential else 0)
        code = lib().sie_port_admittance(self.h, _ports(ports), n, Y.ctypes.data, it.ctypes.data, rr.ctypes.data,
                                         flags)
        if check or code != SIE_ERR_NOT_CONVERGED:
            _check(code)
        return Y, it, rr

    def close(self):
        if self.h:
            _check(lib().sie_op_destroy(self.h))
            self.h = ctypes.c_void_p()
