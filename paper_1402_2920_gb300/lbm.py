"""Python binding of the C ABI in include/lbm.h (ctypes; argument marshalling only).

Every function here forwards to the function of the same name in liblbm.so;
all of the method's steps run in that library's CUDA kernels.  Arrays may be
numpy arrays (host memory) or torch tensors on the simulation's CUDA device;
both must be float64 and C-contiguous.  There is no CPU fallback: if the
library is missing, or no CUDA device is usable, the calls raise.
"""
import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "liblbm.so")

LBM_D2Q21, LBM_D3Q59 = 0, 1
LBM_EOS_VDW, LBM_EOS_PSI_SINE = 0, 1
LBM_STORE_F32, LBM_STORE_F32_DEV, LBM_STORE_F16_DEV, LBM_STORE_BF16_DEV, LBM_STORE_F64 = 0, 1, 2, 3, 4
LBM_STORE_F32_LOC, LBM_STORE_F16_LOC, LBM_STORE_BF16_LOC = 5, 6, 7
LBM_USOLVE_NATIVE, LBM_USOLVE_F64 = 0, 1
LBM_OK = 0
LBM_E_INVALID_ARG, LBM_E_WEIGHTS, LBM_E_BULKVISC, LBM_E_USOLVE_DIVERGED = -1, -2, -3, -4
LBM_E_OOM, LBM_E_CUDA, LBM_E_TIMEOUT, LBM_E_IO = -5, -6, -7, -8

#: every entry point the header declares (checked against the library's exports by the tests)
ENTRY_POINTS = ("lbm_create", "lbm_footprint_bytes", "lbm_init", "lbm_step", "lbm_fields", "lbm_populations",
                "lbm_set_populations", "lbm_velocities", "lbm_stats_get", "lbm_sync", "lbm_save", "lbm_load",
                "lbm_step_batch", "lbm_error_string", "lbm_destroy", "lbm_profile", "lbm_moment_sums_noalloc",
                "lbm_serve", "lbm_collision_map_bench")

#: kernel order of lbm_profile
PROFILE_STAGES = ("moments", "force", "usolve_sweep", "derivs", "collide")


class lbm_eos(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int), ("a", ctypes.c_double), ("b", ctypes.c_double), ("T", ctypes.c_double),
                ("rho1", ctypes.c_double), ("rho2", ctypes.c_double), ("A", ctypes.c_double),
                ("cs2_rho1", ctypes.c_double)]


class lbm_params(ctypes.Structure):
    _fields_ = [("gamma", ctypes.c_double), ("kappa", ctypes.c_double), ("rho0", ctypes.c_double),
                ("storage", ctypes.c_int), ("usolve_precision", ctypes.c_int), ("usolve_tol", ctypes.c_double),
                ("usolve_rtol", ctypes.c_double), ("usolve_max_iter", ctypes.c_int),
                ("usolve_warm_start", ctypes.c_int), ("rho_check_min", ctypes.c_double),
                ("rho_check_max", ctypes.c_double), ("usolve_omega", ctypes.c_double),
                ("usolve_chebyshev", ctypes.c_int)]


class lbm_stats(ctypes.Structure):
    _fields_ = [("mass", ctypes.c_double), ("mom", ctypes.c_double * 3), ("steps", ctypes.c_int64),
                ("usolve_iters_last", ctypes.c_int), ("usolve_iters_max", ctypes.c_int),
                ("usolve_resid", ctypes.c_double), ("status", ctypes.c_int),
                ("usolve_sweeps_total", ctypes.c_int64), ("usolve_tensor_copies", ctypes.c_int)]


class lbm_request(ctypes.Structure):
    _fields_ = [("lattice", ctypes.c_int), ("dims", ctypes.c_int64 * 3), ("eos", lbm_eos), ("params", lbm_params),
                ("steps", ctypes.c_int64), ("arrival_s", ctypes.c_double), ("rho_init", ctypes.c_void_p),
                ("u_init", ctypes.c_void_p), ("rho_out", ctypes.c_void_p), ("u_out", ctypes.c_void_p)]


class lbm_request_result(ctypes.Structure):
    _fields_ = [("admit_s", ctypes.c_double), ("finish_s", ctypes.c_double), ("status", ctypes.c_int),
                ("steps_done", ctypes.c_int64), ("footprint", ctypes.c_size_t)]


class lbm_serve_config(ctypes.Structure):
    _fields_ = [("memory_budget", ctypes.c_size_t), ("max_active", ctypes.c_int), ("chunk_steps", ctypes.c_int),
                ("batched", ctypes.c_int)]


class LbmError(RuntimeError):
    def __init__(self, code, where):
        self.code = code
        super().__init__("%s failed: %s (%d)" % (where, lbm_error_string(code), code))


_lib = None


def load_library(path=LIB_PATH):
    """Load liblbm.so (built by paper_1402_2920_gb300.build); raises if it is missing."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError("liblbm.so is not built (%s); run __graft_entry__.build()" % path)
    L = ctypes.CDLL(path)
    vp, i64p = ctypes.c_void_p, ctypes.POINTER(ctypes.c_int64)
    L.lbm_create.argtypes = [ctypes.c_int, i64p, ctypes.POINTER(lbm_eos), ctypes.POINTER(lbm_params), vp,
                             ctypes.POINTER(vp)]
    L.lbm_footprint_bytes.argtypes = [ctypes.c_int, i64p, ctypes.c_int]
    L.lbm_footprint_bytes.restype = ctypes.c_size_t
    L.lbm_init.argtypes = [vp, vp, vp, ctypes.c_int]
    L.lbm_step.argtypes = [vp, ctypes.c_int64]
    L.lbm_fields.argtypes = [vp, vp, vp, ctypes.c_int]
    L.lbm_populations.argtypes = [vp, vp, ctypes.c_int]
    L.lbm_set_populations.argtypes = [vp, vp, ctypes.c_int]
    L.lbm_velocities.argtypes = [ctypes.c_int, ctypes.POINTER(ctypes.c_int)]
    L.lbm_stats_get.argtypes = [vp, ctypes.POINTER(lbm_stats)]
    L.lbm_sync.argtypes = [vp]
    L.lbm_save.argtypes = [vp, ctypes.c_char_p]
    L.lbm_load.argtypes = [vp, ctypes.c_char_p]
    L.lbm_step_batch.argtypes = [ctypes.POINTER(vp), ctypes.c_int, i64p]
    L.lbm_error_string.argtypes = [ctypes.c_int]
    L.lbm_error_string.restype = ctypes.c_char_p
    L.lbm_profile.argtypes = [vp, ctypes.c_int, ctypes.POINTER(ctypes.c_double), ctypes.c_int]
    dp = ctypes.POINTER(ctypes.c_double)
    L.lbm_collision_map_bench.argtypes = [ctypes.c_int64, ctypes.c_int, dp, dp, dp, dp]
    L.lbm_destroy.argtypes = [vp]
    L.lbm_destroy.restype = None
    for name in ENTRY_POINTS:
        if name not in ("lbm_footprint_bytes", "lbm_error_string", "lbm_destroy"):
            getattr(L, name).restype = ctypes.c_int
    _lib = L
    return L


def _check(code, where):
    if code != LBM_OK:
        raise LbmError(code, where)


def _ptr(a, n=None, what="array"):
    """(address, on_device) of a float64 C-contiguous numpy array or CUDA torch tensor."""
    if a is None:
        return None, 0
    if isinstance(a, np.ndarray):
        if a.dtype != np.float64 or not a.flags.c_contiguous:
            raise TypeError("%s must be a C-contiguous float64 array" % what)
        if n is not None and a.size != n:
            raise ValueError("%s has %d elements, expected %d" % (what, a.size, n))
        return a.ctypes.data, 0
    import torch

    if isinstance(a, torch.Tensor):
        if a.dtype != torch.float64 or not a.is_contiguous() or not a.is_cuda:
            raise TypeError("%s must be a contiguous float64 CUDA tensor" % what)
        if n is not None and a.numel() != n:
            raise ValueError("%s has %d elements, expected %d" % (what, a.numel(), n))
        return a.data_ptr(), 1
    raise TypeError("%s must be a numpy array or a torch tensor" % what)


def _dims(dims):
    d = list(int(v) for v in dims)
    if len(d) == 2:
        d.append(1)
    return (ctypes.c_int64 * 3)(*d)


def lbm_error_string(code):
    return load_library().lbm_error_string(int(code)).decode()


def lbm_velocities(lattice):
    L = load_library()
    q = L.lbm_velocities(int(lattice), None)
    if q < 0:
        raise LbmError(q, "lbm_velocities")
    buf = (ctypes.c_int * (3 * q))()
    L.lbm_velocities(int(lattice), buf)
    return np.array(buf, dtype=np.int64).reshape(q, 3)


def lbm_footprint_bytes(lattice, dims, storage):
    return int(load_library().lbm_footprint_bytes(int(lattice), _dims(dims), int(storage)))


def lbm_create(lattice, dims, eos, params, stream=None):
    """Create a simulation; returns the opaque handle (an int)."""
    L = load_library()
    out = ctypes.c_void_p()
    rc = L.lbm_create(int(lattice), _dims(dims), ctypes.byref(eos), ctypes.byref(params),
                      ctypes.c_void_p(int(stream) if stream else 0), ctypes.byref(out))
    _check(rc, "lbm_create")
    return out.value


def lbm_destroy(sim):
    if sim:
        load_library().lbm_destroy(ctypes.c_void_p(sim))


def lbm_init(sim, rho, u=None, N=None, d=None):
    pr, on_r = _ptr(rho, N, "rho")
    pu, on_u = _ptr(u, None if N is None else d * N, "u")
    if u is not None and on_u != on_r:
        raise TypeError("rho and u must both live on the host or both on the device")
    _check(load_library().lbm_init(ctypes.c_void_p(sim), pr, pu, on_r), "lbm_init")


def lbm_step(sim, nsteps):
    _check(load_library().lbm_step(ctypes.c_void_p(sim), int(nsteps)), "lbm_step")


def lbm_fields(sim, rho, u, N=None, d=None):
    pr, on_r = _ptr(rho, N, "rho")
    pu, on_u = _ptr(u, None if N is None else d * N, "u")
    on = on_r if rho is not None else on_u
    _check(load_library().lbm_fields(ctypes.c_void_p(sim), pr, pu, on), "lbm_fields")


def lbm_populations(sim, out, n=None):
    p, on = _ptr(out, n, "out")
    _check(load_library().lbm_populations(ctypes.c_void_p(sim), p, on), "lbm_populations")


def lbm_set_populations(sim, arr, n=None):
    p, on = _ptr(arr, n, "in")
    _check(load_library().lbm_set_populations(ctypes.c_void_p(sim), p, on), "lbm_set_populations")


def lbm_stats_get(sim):
    st = lbm_stats()
    _check(load_library().lbm_stats_get(ctypes.c_void_p(sim), ctypes.byref(st)), "lbm_stats_get")
    return st


def lbm_sync(sim):
    return load_library().lbm_sync(ctypes.c_void_p(sim))


def lbm_save(sim, path):
    _check(load_library().lbm_save(ctypes.c_void_p(sim), os.fsencode(path)), "lbm_save")


def lbm_load(sim, path):
    _check(load_library().lbm_load(ctypes.c_void_p(sim), os.fsencode(path)), "lbm_load")


def lbm_moment_sums_noalloc(lattice, pops, n_sites, sums, stream=None):
    """(mass, j_x, j_y, j_z) of FP64 device populations [Q][n_sites] into the 4-element
    device tensor `sums`, on `stream`, without any allocation (does not synchronise)."""
    def addr(a):
        return a.data_ptr() if hasattr(a, "data_ptr") else int(a)

    rc = load_library().lbm_moment_sums_noalloc(int(lattice), ctypes.c_void_p(addr(pops)), ctypes.c_int64(n_sites),
                                                ctypes.c_void_p(addr(sums)),
                                                ctypes.c_void_p(int(stream) if stream else 0))
    _check(rc, "lbm_moment_sums_noalloc")


def lbm_serve(requests, memory_budget=0, max_active=16, chunk_steps=50, batched=0):
    """Run request dicts to completion (continuous batching); returns lbm_request_result[n].

    batched = 0: one stream per simulation (the faster on the seeded serving workload);
    1: batched launches per kernel combination and size class.

    Each dict has lattice, dims, eos (lbm_eos), params (lbm_params), steps, arrival_s,
    rho_init (C-contiguous float64 host array) and optionally u_init, rho_out, u_out
    (float64 host arrays the results are written to)."""
    n = len(requests)
    reqs = (lbm_request * max(n, 1))()
    keep = []
    for k, r in enumerate(requests):
        q = reqs[k]
        q.lattice = int(r["lattice"])
        q.dims = _dims(r["dims"])
        q.eos = r["eos"]
        q.params = r["params"]
        q.steps = int(r["steps"])
        q.arrival_s = float(r["arrival_s"])
        for name in ("rho_init", "u_init", "rho_out", "u_out"):
            a = r.get(name)
            if a is not None:
                ptr, on = _ptr(a, None, name)
                if on:
                    raise TypeError("%s must be a host array" % name)
                keep.append(a)
                setattr(q, name, ptr)
    out = (lbm_request_result * max(n, 1))()
    cfg = lbm_serve_config(int(memory_budget), int(max_active), int(chunk_steps), int(batched))
    _check(load_library().lbm_serve(reqs, n, ctypes.byref(cfg), out), "lbm_serve")
    return list(out)[:n]


def lbm_profile(sim, reps=10):
    """Average milliseconds per launch of each kernel, keyed by PROFILE_STAGES."""
    out = (ctypes.c_double * len(PROFILE_STAGES))()
    _check(load_library().lbm_profile(ctypes.c_void_p(sim), int(reps), out, len(PROFILE_STAGES)), "lbm_profile")
    return dict(zip(PROFILE_STAGES, list(out)))


def lbm_collision_map_bench(n_sites, reps=5):
    """(ms scalar, ms tensor, max |difference|, max |value|) of the collision's polynomial map."""
    v = [ctypes.c_double() for _ in range(4)]
    _check(load_library().lbm_collision_map_bench(int(n_sites), int(reps), *[ctypes.byref(x) for x in v]),
           "lbm_collision_map_bench")
    return tuple(x.value for x in v)


def lbm_step_batch(sims, nsteps):
    n = len(sims)
    arr = (ctypes.c_void_p * n)(*sims)
    st = (ctypes.c_int64 * n)(*[int(v) for v in nsteps])
    _check(load_library().lbm_step_batch(arr, n, st), "lbm_step_batch")


class Sim:
    """Owning wrapper of one simulation (same calls, numpy or torch buffers)."""

    def __init__(self, lattice, dims, eos, params, stream=None):
        self.lattice = int(lattice)
        self.d = 3 if self.lattice == LBM_D3Q59 else 2
        dd = list(int(v) for v in dims) + ([1] if len(dims) == 2 else [])
        self.dims = tuple(dd)
        self.N = dd[0] * dd[1] * dd[2]
        self.shape = (dd[2], dd[1], dd[0]) if self.d == 3 else (dd[1], dd[0])
        self.Q = 59 if self.d == 3 else 21
        self.handle = lbm_create(lattice, self.dims, eos, params, stream)

    def close(self):
        if getattr(self, "handle", None):
            lbm_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def init(self, rho, u=None):
        lbm_init(self.handle, rho, u, self.N, self.d)

    def step(self, n=1):
        lbm_step(self.handle, n)

    def fields(self):
        rho = np.zeros(self.shape)
        u = np.zeros((self.d,) + self.shape)
        lbm_fields(self.handle, rho, u, self.N, self.d)
        return rho, u

    def populations(self):
        out = np.zeros((self.Q, self.N))
        lbm_populations(self.handle, out, self.Q * self.N)
        return out

    def set_populations(self, arr):
        lbm_set_populations(self.handle, np.ascontiguousarray(arr, dtype=np.float64), self.Q * self.N)

    def stats(self):
        return lbm_stats_get(self.handle)

    def sync(self):
        rc = lbm_sync(self.handle)
        if rc != LBM_OK:
            raise LbmError(rc, "lbm_sync")

    def save(self, path):
        lbm_save(self.handle, path)

    def load(self, path):
        lbm_load(self.handle, path)


def make_eos(kind=LBM_EOS_VDW, a=0.0, b=0.0, T=0.0, rho1=0.0, rho2=0.0, A=0.0, cs2_rho1=0.0):
    return lbm_eos(kind, a, b, T, rho1, rho2, A, cs2_rho1)


def make_params(gamma=0.0, kappa=0.0, rho0=1.0, storage=LBM_STORE_F32, usolve_precision=LBM_USOLVE_NATIVE,
                usolve_tol=0.0, usolve_rtol=0.0, usolve_max_iter=0, usolve_warm_start=1,
                rho_check_min=0.0, rho_check_max=0.0, usolve_omega=1.0, usolve_chebyshev=0):
    return lbm_params(gamma, kappa, rho0, storage, usolve_precision, usolve_tol, usolve_rtol, usolve_max_iter,
                      usolve_warm_start, rho_check_min, rho_check_max, usolve_omega, usolve_chebyshev)
