"""ctypes front end of the FP64 CPU oracle (oracle/lbm_oracle.c).

TEST INFRASTRUCTURE ONLY: the tests, the smoke check and the CPU-baseline
leg of the benchmark may use this module; the library never does.

Conventions: fields are C-order [z][y][x] flattened (x fastest); vectors are
component-major [3][N] (the third component is zero in 2D); populations are
[Q][N] in the oracle's own velocity order, given by ``velocities(lattice)``.
"""
import ctypes
import os

import numpy as np

from . import build as _build

D2Q21, D3Q59 = 0, 1
EOS_VDW, EOS_PSI_SINE = 0, 1
ST_D1, ST_LAP, ST_TRACELESS, ST_D3 = 0, 1, 2, 3

_lib = None


def lib():
    global _lib
    if _lib is None:
        path = _build.build()
        L = ctypes.CDLL(path)
        dp = ctypes.POINTER(ctypes.c_double)
        ip = ctypes.POINTER(ctypes.c_int)
        vp = ctypes.c_void_p
        L.orc_lattice_info.argtypes = [ctypes.c_int, ip, ip]
        L.orc_lattice_info.restype = ctypes.c_int
        L.orc_weights.argtypes = [ctypes.c_int, ctypes.c_double, dp]
        L.orc_weight_shell.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_double]
        L.orc_weight_shell.restype = ctypes.c_double
        L.orc_eos_eval.argtypes = [ctypes.c_int, dp, ctypes.c_double, dp]
        L.orc_stencil_info.argtypes = [ctypes.c_int, ctypes.c_int, ip, dp]
        L.orc_stencil_info.restype = ctypes.c_int
        L.orc_create.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int, dp,
                                 ctypes.c_double, ctypes.c_double, ctypes.c_double, ctypes.c_double,
                                 ctypes.c_int, ctypes.c_int]
        L.orc_create.restype = vp
        L.orc_destroy.argtypes = [vp]
        L.orc_Q.argtypes = [vp]
        L.orc_Q.restype = ctypes.c_int
        L.orc_cs0.argtypes = [vp]
        L.orc_cs0.restype = ctypes.c_double
        L.orc_init.argtypes = [vp, dp, dp]
        L.orc_step.argtypes = [vp, ctypes.c_int]
        L.orc_step.restype = ctypes.c_int
        L.orc_fields.argtypes = [vp, dp, dp]
        L.orc_fields.restype = ctypes.c_int
        L.orc_get_pops.argtypes = [vp, dp]
        L.orc_set_pops.argtypes = [vp, dp]
        L.orc_get_jt.argtypes = [vp, dp]
        L.orc_last_iters.argtypes = [vp]
        L.orc_last_iters.restype = ctypes.c_int
        L.orc_last_resid.argtypes = [vp]
        L.orc_last_resid.restype = ctypes.c_double
        L.orc_field.argtypes = [vp, ctypes.c_char_p, dp]
        L.orc_field.restype = ctypes.c_int
        L.orc_prepare.argtypes = [vp]
        L.orc_prepare.restype = ctypes.c_int
        L.orc_collision_parts.argtypes = [vp, ctypes.c_long, dp, dp]
        L.orc_apply_stencil.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int, dp, dp]
        L.orc_neq.argtypes = [ctypes.c_int, ctypes.c_double, ctypes.c_double, dp, dp]
        L.orc_num_threads.restype = ctypes.c_int
        L.orc_set_num_threads.argtypes = [ctypes.c_int]
        # one thread unless asked: the tests run many tiny lattices
        L.orc_set_num_threads(int(os.environ.get("ORACLE_THREADS", "1")))
        _lib = L
    return _lib


def _p(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _ip(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_int))


def velocities(lattice):
    """(c [Q,3] int, shell [Q] int) in the oracle's velocity order."""
    c = np.zeros((59, 3), dtype=np.int32)
    sh = np.zeros(59, dtype=np.int32)
    q = lib().orc_lattice_info(lattice, _ip(c), _ip(sh))
    return c[:q].copy(), sh[:q].copy()


def weights(lattice, cs2):
    q = velocities(lattice)[0].shape[0]
    w = np.zeros(q)
    lib().orc_weights(lattice, float(cs2), _p(w))
    return w


def weight_shell(lattice, shell, cs2):
    return lib().orc_weight_shell(lattice, shell, float(cs2))


def eos_params(kind, a=0.0, b=0.0, T=0.0, rho1=0.0, rho2=0.0, A=0.0, cs2_rho1=0.0):
    return np.array([a, b, T, rho1, rho2, A, cs2_rho1], dtype=np.float64)


def eos_eval(kind, prm, rho):
    """(p, dp/drho, p - rho dp/drho, rho d2p/drho2) at rho."""
    out = np.zeros(4)
    lib().orc_eos_eval(kind, _p(np.ascontiguousarray(prm, dtype=np.float64)), float(rho), _p(out))
    return out


def stencil(d, which):
    dv = np.zeros((32, 3), dtype=np.int32)
    tau = np.zeros(32)
    n = lib().orc_stencil_info(d, which, _ip(dv), _p(tau))
    return dv[:n].copy(), tau[:n].copy()


def apply_stencil(d, which, g):
    """Apply a Table III operator to a periodic field g of shape (nz, ny, nx) or (ny, nx)."""
    g = np.ascontiguousarray(g, dtype=np.float64)
    if d == 2:
        ny, nx = g.shape
        nz = 1
    else:
        nz, ny, nx = g.shape
    N = nx * ny * nz
    ncomp = {ST_D1: 3, ST_LAP: 1, ST_TRACELESS: 9, ST_D3: 3}[which]
    out = np.zeros(ncomp * N)
    lib().orc_apply_stencil(d, which, nx, ny, nz, _p(g), _p(out))
    return out.reshape((ncomp,) + g.shape) if ncomp > 1 else out.reshape(g.shape)


def neq(lattice, rho, cs2, u):
    q = velocities(lattice)[0].shape[0]
    u3 = np.zeros(3)
    u3[: len(u)] = u
    out = np.zeros(q)
    lib().orc_neq(lattice, float(rho), float(cs2), _p(u3), _p(out))
    return out


def num_threads():
    return lib().orc_num_threads()


def set_num_threads(n):
    lib().orc_set_num_threads(int(n))


class Sim:
    """The oracle's simulation: FP64 populations stepped by S1-S12."""

    def __init__(self, lattice, dims, eos_kind, eos_prm, gamma, kappa, rho0,
                 tol=1e-14, maxit=2000, warm=True):
        self.lattice = lattice
        self.d = 3 if lattice == D3Q59 else 2
        nx, ny = int(dims[0]), int(dims[1])
        nz = int(dims[2]) if self.d == 3 else 1
        self.dims = (nx, ny, nz)
        self.N = nx * ny * nz
        self.shape = (nz, ny, nx) if self.d == 3 else (ny, nx)
        prm = np.ascontiguousarray(eos_prm, dtype=np.float64)
        self._h = lib().orc_create(lattice, nx, ny, nz, eos_kind, _p(prm), float(gamma), float(kappa),
                                   float(rho0), float(tol), int(maxit), int(bool(warm)))
        if not self._h:
            raise MemoryError("oracle allocation failed")
        self.Q = lib().orc_Q(self._h)
        self.cs0 = lib().orc_cs0(self._h)

    def close(self):
        if getattr(self, "_h", None):
            lib().orc_destroy(self._h)
            self._h = None

    def __del__(self):
        self.close()

    def init(self, rho, u=None):
        rho = np.ascontiguousarray(rho, dtype=np.float64).reshape(-1)
        assert rho.size == self.N
        if u is None:
            lib().orc_init(self._h, _p(rho), None)
        else:
            u3 = np.zeros((3, self.N))
            uu = np.asarray(u, dtype=np.float64).reshape(len(u), -1)
            u3[: uu.shape[0]] = uu
            lib().orc_init(self._h, _p(rho), _p(u3))

    def step(self, n=1):
        return lib().orc_step(self._h, int(n))

    def fields(self):
        rho = np.zeros(self.N)
        u = np.zeros((3, self.N))
        st = lib().orc_fields(self._h, _p(rho), _p(u))
        return rho.reshape(self.shape), u[: self.d].reshape((self.d,) + self.shape), st

    def pops(self):
        out = np.zeros((self.Q, self.N))
        lib().orc_get_pops(self._h, _p(out))
        return out

    def set_pops(self, arr):
        arr = np.ascontiguousarray(arr, dtype=np.float64).reshape(self.Q, self.N)
        lib().orc_set_pops(self._h, _p(arr))

    def jt(self):
        out = np.zeros((3, self.N))
        lib().orc_get_jt(self._h, _p(out))
        return out

    def last_iters(self):
        return lib().orc_last_iters(self._h)

    def last_resid(self):
        return lib().orc_last_resid(self._h)

    _NCOMP = {"rho": 1, "j0": 3, "p": 1, "dp": 1, "pm": 1, "rpp": 1, "f": 3, "j0p": 3, "jt": 3, "u": 3,
              "j": 3, "du": 9, "dj": 9, "dp_grad": 3, "dpuu": 27, "dpr": 3, "Sigma": 9, "Xi": 27, "q": 9}

    def field(self, name):
        n = self._NCOMP[name]
        out = np.zeros(n * self.N)
        got = lib().orc_field(self._h, name.encode(), _p(out))
        assert got == n
        return out.reshape(n, self.N) if n > 1 else out

    def prepare(self):
        return lib().orc_prepare(self._h)

    def collision_parts(self, r):
        parts = np.zeros(3 * self.Q)
        nstar = np.zeros(self.Q)
        lib().orc_collision_parts(self._h, int(r), _p(parts), _p(nstar))
        return parts.reshape(3, self.Q), nstar
