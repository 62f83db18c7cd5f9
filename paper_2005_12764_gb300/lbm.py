"""ctypes binding of liblbm.so (include/lbm.h): argument marshalling only.

Every step of the method runs in the CUDA library; this module converts NumPy /
PyTorch arrays to pointers and status codes to exceptions. There is no CPU
fallback: if the library is not built, or no CUDA device is present, calls raise.

Arrays are float64 and indexed [z, y, x] (vector fields [3, z, y, x]). Device
tensors (``torch.Tensor`` on CUDA) are passed by pointer (``on_device=1``); NumPy
arrays are host memory. ``Lattice`` wraps one context.
"""
from __future__ import annotations

import ctypes as C
import os
import threading

import numpy as np

from . import build_lib

Q = 19
STORAGE = {"fp32": 0, "fp16": 1, "bf16": 2, "fp32_q5": 3, "fp16_q5": 4}
MODELS = {"colour": 0, "shan_chen": 1}
_STATUS = {0: "LBM_OK", -1: "LBM_EINVAL", -2: "LBM_ENOMEM", -3: "LBM_ECUDA", -4: "LBM_ESTATE",
           -5: "LBM_ETIMEOUT"}

# Exported symbols of include/lbm.h (checked by the test-suite).
SYMBOLS = ["lbm_velocity_set", "lbm_create", "lbm_set_fields", "lbm_set_pin_mask", "lbm_step",
           "lbm_step_timed", "lbm_launches_per_step",
           "lbm_get_fields", "lbm_get_pops", "lbm_set_pops", "lbm_observables", "lbm_laplace",
           "lbm_state_bytes", "lbm_save_state", "lbm_load_state", "lbm_sync",
           "lbm_footprint_bytes", "lbm_work_split", "lbm_steps_taken", "lbm_destroy",
           "lbm_last_error",
           "lbm_totals_noalloc", "lbm_get_nc_field", "lbm_get_window",
           "lbm_planes_bytes", "lbm_get_planes", "lbm_set_planes",
           "lbm_droplets", "lbm_structure_factor", "lbm_selftest_timeout",
           "lbm_engine_create", "lbm_engine_submit", "lbm_engine_tick", "lbm_engine_state",
           "lbm_engine_result", "lbm_engine_stats", "lbm_engine_destroy", "lbm_engine_cancel",
           "lbm_engine_last_error"]


class EngineParams(C.Structure):
    _fields_ = [("hbm_budget_bytes", C.c_size_t), ("max_slots", C.c_int),
                ("chunk_steps", C.c_int), ("autotune", C.c_int), ("policy", C.c_int),
                ("cuda_stream", C.c_void_p)]


class LbmError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{_STATUS.get(status, status)}: {msg}")
        self.status = status


class Params(C.Structure):
    _fields_ = [("nx", C.c_int), ("ny", C.c_int), ("nz", C.c_int),
                ("wall_y", C.c_int), ("wall_z", C.c_int),
                ("tau_r", C.c_double), ("tau_b", C.c_double),
                ("sigma", C.c_double), ("beta", C.c_double),
                ("A_nc", C.c_double), ("h_min", C.c_double), ("h_cut", C.c_double),
                ("g", C.c_double * 3), ("kolmogorov_amp", C.c_double), ("wall_u", C.c_double),
                ("rho0", C.c_double), ("model", C.c_int), ("G_sc", C.c_double),
                ("storage", C.c_int), ("cuda_stream", C.c_void_p), ("inplace", C.c_int)]


_lib = None
_lock = threading.Lock()
_P = C.c_void_p
_D = C.c_void_p   # pointers are passed as integers (host or device)


def library_path() -> str:
    return build_lib.LIB


def load():
    """Load liblbm.so; raises if it has not been built (see build_lib.build())."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        path = library_path()
        if not os.path.exists(path):
            raise RuntimeError(f"liblbm.so not built ({path}); run "
                               "paper_2005_12764_gb300.build_lib.build()")
        lib = C.CDLL(path)
        PP = C.POINTER(Params)
        sig = {
            "lbm_velocity_set": (None, [C.POINTER(C.c_int)]),
            "lbm_create": (C.c_int, [PP, C.POINTER(C.c_void_p)]),
            "lbm_set_fields": (C.c_int, [_P, _D, _D, _D, C.c_int]),
            "lbm_set_pin_mask": (C.c_int, [_P, _D, C.c_int]),
            "lbm_step": (C.c_int, [_P, C.c_int]),
            "lbm_step_timed": (C.c_int, [_P, C.c_int, C.POINTER(C.c_double)]),
            "lbm_launches_per_step": (C.c_int, [_P]),
            "lbm_get_fields": (C.c_int, [_P, _D, _D, _D, _D, C.c_int]),
            "lbm_get_pops": (C.c_int, [_P, _D, _D, _D, C.c_int]),
            "lbm_set_pops": (C.c_int, [_P, _D, _D, _D, C.c_int]),
            "lbm_observables": (C.c_int, [_P, C.POINTER(C.c_double)]),
            "lbm_laplace": (C.c_int, [_P, C.POINTER(C.c_double), C.POINTER(C.c_double)]),
            "lbm_state_bytes": (C.c_size_t, [_P]),
            "lbm_save_state": (C.c_int, [_P, C.c_void_p]),
            "lbm_load_state": (C.c_int, [_P, C.c_void_p]),
            "lbm_sync": (C.c_int, [_P]),
            "lbm_footprint_bytes": (C.c_size_t, [PP]),
            "lbm_work_split": (C.c_int, [PP, C.c_int, C.POINTER(C.c_longlong)]),
            "lbm_steps_taken": (C.c_longlong, [_P]),
            "lbm_destroy": (None, [_P]),
            "lbm_last_error": (C.c_char_p, [_P]),
            "lbm_totals_noalloc": (C.c_int, [_D, C.c_longlong, _D, C.c_void_p]),
            "lbm_get_nc_field": (C.c_int, [_P, _D, C.c_int]),
            "lbm_planes_bytes": (C.c_size_t, [_P, C.c_int]),
            "lbm_get_planes": (C.c_int, [_P, C.c_int, C.c_int, _D]),
            "lbm_set_planes": (C.c_int, [_P, C.c_int, C.c_int, _D]),
            "lbm_droplets": (C.c_int, [_P, C.POINTER(C.c_longlong), _D, C.c_longlong]),
            "lbm_selftest_timeout": (C.c_int, [_P]),
            "lbm_structure_factor": (C.c_int, [_P, C.c_int, _D, _D, _D]),
            "lbm_get_window": (C.c_int, [_P] + [C.c_int] * 6 + [_D, _D, _D, C.c_int]),
            "lbm_engine_create": (C.c_int, [C.POINTER(EngineParams), C.POINTER(C.c_void_p)]),
            "lbm_engine_submit": (C.c_int, [_P, PP, _D, _D, _D, C.c_longlong,
                                            C.POINTER(C.c_longlong)]),
            "lbm_engine_tick": (C.c_int, [_P] + [C.POINTER(C.c_int)] * 4),
            "lbm_engine_state": (C.c_int, [_P, C.c_longlong]),
            "lbm_engine_cancel": (C.c_int, [_P, C.c_longlong]),
            "lbm_engine_result": (C.c_int, [_P, C.c_longlong, _D, _D, _D, _D,
                                            C.POINTER(C.c_longlong)]),
            "lbm_engine_stats": (None, [_P, C.POINTER(C.c_longlong)]),
            "lbm_engine_destroy": (None, [_P]),
            "lbm_engine_last_error": (C.c_char_p, [_P]),
        }
        for name, (res, args) in sig.items():
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        _lib = lib
        return lib


def velocity_set() -> np.ndarray:
    c = (C.c_int * (3 * Q))()
    load().lbm_velocity_set(c)
    return np.array(list(c), dtype=np.int64).reshape(Q, 3)


def make_params(nx, ny, nz, *, wall_y=0, wall_z=0, tau_r=1.0, tau_b=None, sigma=0.0, beta=0.7,
                A_nc=0.0, h_min=3.0, h_cut=None, g=(0.0, 0.0, 0.0), kolmogorov_amp=0.0, rho0=1.0,
                storage="fp32", stream=None, wall_u=0.0, model="colour", G_sc=0.0,
                inplace=0) -> Params:
    p = Params()
    p.nx, p.ny, p.nz = int(nx), int(ny), int(nz)
    p.wall_y, p.wall_z = int(wall_y), int(wall_z)
    p.tau_r = float(tau_r)
    p.tau_b = float(tau_r if tau_b is None else tau_b)
    p.sigma, p.beta = float(sigma), float(beta)
    p.A_nc, p.h_min = float(A_nc), float(h_min)
    p.h_cut = float(2.0 * h_min if h_cut is None else h_cut)
    for a in range(3):
        p.g[a] = float(g[a])
    p.kolmogorov_amp = float(kolmogorov_amp)
    p.wall_u = float(wall_u)
    p.rho0 = float(rho0)
    p.model = MODELS[model] if isinstance(model, str) else int(model)
    p.G_sc = float(G_sc)
    p.storage = STORAGE[storage] if isinstance(storage, str) else int(storage)
    p.cuda_stream = stream
    p.inplace = int(inplace)
    return p


def totals_noalloc(pops_ptr: int, n_nodes: int, out_ptr: int, stream=None) -> None:
    """Conserved totals of a float32 device population array [2][19][n] into the
    device array out (5 doubles), without any allocation (see include/lbm.h)."""
    lib = load()
    rc = lib.lbm_totals_noalloc(pops_ptr, int(n_nodes), out_ptr, stream)
    if rc != 0:
        raise LbmError(rc, lib.lbm_last_error(None).decode())


def footprint_bytes(params: Params) -> int:
    return int(load().lbm_footprint_bytes(C.byref(params)))


def work_split(params: Params, num_sms: int) -> dict:
    """The step kernel's work split on a GPU of num_sms SMs (include/lbm.h,
    lbm_work_split): zparts, chain, band_k, band_h, grid."""
    out = (C.c_longlong * 5)()
    rc = load().lbm_work_split(C.byref(params), int(num_sms), out)
    if rc != 0:
        raise LbmError(rc, load().lbm_last_error(None).decode())
    return dict(zip(("zparts", "chain", "band_k", "band_h", "grid"), (int(v) for v in out)))


def _is_torch(a):
    return type(a).__module__.startswith("torch")


class Lattice:
    """One lattice context of liblbm.so (device memory owned by the library)."""

    def __init__(self, params: Params):
        self._lib = load()
        self.params = params
        self.shape = (params.nz, params.ny, params.nx)
        self.N = params.nx * params.ny * params.nz
        h = C.c_void_p()
        rc = self._lib.lbm_create(C.byref(params), C.byref(h))
        if rc != 0:
            raise LbmError(rc, self._lib.lbm_last_error(None).decode())
        self._h = h

    # -- plumbing
    def _check(self, rc):
        if rc != 0:
            raise LbmError(rc, self._lib.lbm_last_error(self._h).decode())

    def close(self):
        if getattr(self, "_h", None):
            self._lib.lbm_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @staticmethod
    def _ptr(a, n, keep):
        """pointer of a float64 array with n elements; returns (ptr, on_device)."""
        if a is None:
            return None, None
        if _is_torch(a):
            import torch
            assert a.dtype == torch.float64 and a.is_contiguous() and a.numel() == n
            return a.data_ptr(), a.is_cuda
        arr = np.ascontiguousarray(a, dtype=np.float64).reshape(-1)
        assert arr.size == n, (arr.size, n)
        keep.append(arr)
        return arr.ctypes.data, False

    def _ptrs(self, arrays, sizes):
        keep, ptrs, dev = [], [], set()
        for a, n in zip(arrays, sizes):
            p, d = self._ptr(a, n, keep)
            ptrs.append(p)
            if d is not None:
                dev.add(d)
        if len(dev) > 1:
            raise ValueError("mix of host and device arrays")
        return ptrs, int(dev.pop()) if dev else 0, keep

    # -- API
    def set_fields(self, rho_r, rho_b, u=None):
        (pr, pb, pu), dev, keep = self._ptrs([rho_r, rho_b, u], [self.N, self.N, 3 * self.N])
        self._check(self._lib.lbm_set_fields(self._h, pr, pb, pu, dev))

    def set_pin_mask(self, mask):
        if mask is None:
            self._check(self._lib.lbm_set_pin_mask(self._h, None, 0))
            return
        if _is_torch(mask):
            self._check(self._lib.lbm_set_pin_mask(self._h, mask.data_ptr(), int(mask.is_cuda)))
            return
        m = np.ascontiguousarray(mask, dtype=np.uint8).reshape(-1)
        self._check(self._lib.lbm_set_pin_mask(self._h, m.ctypes.data, 0))

    def step(self, n=1):
        self._check(self._lib.lbm_step(self._h, int(n)))

    def step_timed(self, n=1):
        """Advance n steps, returning (ms in the near-contact pass, ms in the step
        kernel, ms in the ghost fill) summed over the steps, from CUDA events inside
        the library."""
        out = (C.c_double * 3)()
        self._check(self._lib.lbm_step_timed(self._h, int(n), out))
        return float(out[0]), float(out[1]), float(out[2])

    @property
    def launches_per_step(self):
        return int(self._lib.lbm_launches_per_step(self._h))

    def sync(self):
        self._check(self._lib.lbm_sync(self._h))

    @property
    def steps_taken(self):
        return int(self._lib.lbm_steps_taken(self._h))

    def get_fields(self, out=None):
        """dict rho_r, rho_b, u [3,...], phi as NumPy (or into the given tensors)."""
        s = self.shape
        if out is None:
            res = {"rho_r": np.empty(s), "rho_b": np.empty(s), "u": np.empty((3,) + s),
                   "phi": np.empty(s)}
        else:
            res = out
        (pr, pb, pu, pp), dev, keep = self._ptrs(
            [res.get("rho_r"), res.get("rho_b"), res.get("u"), res.get("phi")],
            [self.N, self.N, 3 * self.N, self.N])
        if out is None:
            pr, pb = res["rho_r"].ctypes.data, res["rho_b"].ctypes.data
            pu, pp = res["u"].ctypes.data, res["phi"].ctypes.data
        self._check(self._lib.lbm_get_fields(self._h, pr, pb, pu, pp, dev))
        return res

    def get_pops(self):
        """(f_r [19, z, y, x], f_b, phi_lag [z, y, x]) in the library's velocity order."""
        fr = np.empty((Q,) + self.shape)
        fb = np.empty((Q,) + self.shape)
        lag = np.empty(self.shape)
        self._check(self._lib.lbm_get_pops(self._h, fr.ctypes.data, fb.ctypes.data,
                                           lag.ctypes.data, 0))
        return fr, fb, lag

    def set_pops(self, fr, fb, phi_lag=None):
        (pr, pb, pl), dev, keep = self._ptrs([fr, fb, phi_lag], [Q * self.N, Q * self.N, self.N])
        self._check(self._lib.lbm_set_pops(self._h, pr, pb, pl, dev))

    def get_window(self, x0, y0, z0, wx, wy, wz):
        """(f_r [19, wz, wy, wx], f_b, phi_lag [wz, wy, wx]) of a sub-box, wrapped on
        periodic axes (host copies)."""
        fr = np.empty((Q, wz, wy, wx))
        fb = np.empty((Q, wz, wy, wx))
        lag = np.empty((wz, wy, wx))
        self._check(self._lib.lbm_get_window(self._h, int(x0), int(y0), int(z0), int(wx), int(wy),
                                             int(wz), fr.ctypes.data, fb.ctypes.data,
                                             lag.ctypes.data, 0))
        return fr, fb, lag

    def get_nc_field(self):
        """A_h [z, y, x] on the current colour field (what the next step will use)."""
        ah = np.empty(self.shape)
        self._check(self._lib.lbm_get_nc_field(self._h, ah.ctypes.data, 0))
        return ah

    def planes_bytes(self, h):
        """Bytes of h z-planes of the stored state (populations as stored, lagged colour
        field)."""
        return int(self._lib.lbm_planes_bytes(self._h, int(h)))

    def get_planes(self, z0, h, buf):
        """Planes z0 .. z0+h-1 of the stored state into buf (a CUDA uint8 tensor of
        planes_bytes(h) bytes); queued on the lattice's stream."""
        assert _is_torch(buf) and buf.is_cuda and buf.numel() * buf.element_size() >= self.planes_bytes(h)
        self._check(self._lib.lbm_get_planes(self._h, int(z0), int(h), buf.data_ptr()))

    def set_planes(self, z0, h, buf):
        assert _is_torch(buf) and buf.is_cuda and buf.numel() * buf.element_size() >= self.planes_bytes(h)
        self._check(self._lib.lbm_set_planes(self._h, int(z0), int(h), buf.data_ptr()))

    def selftest_timeout(self) -> int:
        """Status of the bounded-wait self-test: LBM_ETIMEOUT (-5) when a wait that
        cannot complete gave up as designed (the context stays usable)."""
        return int(self._lib.lbm_selftest_timeout(self._h))

    def droplets(self):
        """(number of droplets, their node counts in descending order): the
        26-connected components of {phi > 0} of the current colour field."""
        n = C.c_longlong()
        self._check(self._lib.lbm_droplets(self._h, C.byref(n), None, 0))
        sizes = np.zeros(n.value, dtype=np.int64)
        if n.value:
            self._check(self._lib.lbm_droplets(self._h, C.byref(n), sizes.ctypes.data, sizes.size))
        return int(n.value), sizes

    def structure_factor(self, nbins):
        """(k, S(k), modes per shell) of the current colour field."""
        k, S = np.zeros(nbins), np.zeros(nbins)
        m = np.zeros(nbins, dtype=np.int64)
        self._check(self._lib.lbm_structure_factor(self._h, int(nbins), k.ctypes.data,
                                                   S.ctypes.data, m.ctypes.data))
        return k, S, m

    def observables(self):
        out = (C.c_double * 8)()
        self._check(self._lib.lbm_observables(self._h, out))
        return np.array(list(out))

    def laplace(self, centre):
        c = (C.c_double * 3)(*[float(v) for v in centre])
        out = (C.c_double * 5)()
        self._check(self._lib.lbm_laplace(self._h, c, out))
        o = list(out)
        return {"dp": o[0], "R_eff": o[1], "p_in": o[2], "p_out": o[3], "V": o[4]}

    def save_state(self) -> bytes:
        n = int(self._lib.lbm_state_bytes(self._h))
        buf = (C.c_char * n)()
        self._check(self._lib.lbm_save_state(self._h, buf))
        return bytes(buf)

    def load_state(self, blob: bytes):
        buf = C.create_string_buffer(blob, len(blob))
        self._check(self._lib.lbm_load_state(self._h, buf))


class Engine:
    """Serving engine of liblbm.so (lbm_engine_* in include/lbm.h): requests are
    queued, admitted by device memory, advanced together in batched launches and
    retired with their fields copied to host memory."""

    STATES = {0: "queued", 1: "resident", 2: "finished", 3: "taken", 4: "failed", 5: "cancelled",
              -1: "unknown"}

    POLICIES = {"fcfs": 0, "sjf": 1}

    def __init__(self, budget_bytes, max_slots=64, chunk_steps=50, autotune=True, policy="fcfs",
                 stream=None):
        self._lib = load()
        ep = EngineParams()
        ep.hbm_budget_bytes = int(budget_bytes)
        ep.max_slots, ep.chunk_steps, ep.autotune = int(max_slots), int(chunk_steps), int(autotune)
        ep.policy = self.POLICIES[policy]
        ep.cuda_stream = stream
        h = C.c_void_p()
        rc = self._lib.lbm_engine_create(C.byref(ep), C.byref(h))
        if rc != 0:
            raise LbmError(rc, self._lib.lbm_last_error(None).decode())
        self._h = h
        self.shapes = {}

    def _check(self, rc):
        if rc != 0:
            raise LbmError(rc, self._lib.lbm_engine_last_error(self._h).decode())

    def submit(self, params: Params, rho_r, rho_b, steps, u=None) -> int:
        n = params.nx * params.ny * params.nz
        rr = np.ascontiguousarray(rho_r, dtype=np.float64).reshape(-1)
        rb = np.ascontiguousarray(rho_b, dtype=np.float64).reshape(-1)
        assert rr.size == n and rb.size == n
        uu = None if u is None else np.ascontiguousarray(u, dtype=np.float64).reshape(-1)
        t = C.c_longlong()
        self._check(self._lib.lbm_engine_submit(self._h, C.byref(params), rr.ctypes.data,
                                                rb.ctypes.data,
                                                None if uu is None else uu.ctypes.data,
                                                int(steps), C.byref(t)))
        self.shapes[t.value] = (params.nz, params.ny, params.nx)
        return t.value

    def tick(self):
        """One round; returns (resident, queued, retired, steps advanced)."""
        v = [C.c_int() for _ in range(4)]
        self._check(self._lib.lbm_engine_tick(self._h, *[C.byref(x) for x in v]))
        return tuple(x.value for x in v)

    def cancel(self, ticket):
        """Withdraw a queued, resident or finished request (its state becomes
        'cancelled'); the other requests go on unchanged."""
        self._check(self._lib.lbm_engine_cancel(self._h, int(ticket)))

    def state(self, ticket) -> str:
        return self.STATES[self._lib.lbm_engine_state(self._h, int(ticket))]

    def result(self, ticket):
        """Fields of a finished request (dict as Lattice.get_fields) plus 'info' =
        (steps, tick submitted, tick admitted, tick retired); releases the result."""
        shape = self.shapes[ticket]
        out = {"rho_r": np.empty(shape), "rho_b": np.empty(shape), "u": np.empty((3,) + shape),
               "phi": np.empty(shape)}
        info = (C.c_longlong * 4)()
        self._check(self._lib.lbm_engine_result(self._h, int(ticket), out["rho_r"].ctypes.data,
                                                out["rho_b"].ctypes.data, out["u"].ctypes.data,
                                                out["phi"].ctypes.data, info))
        out["info"] = tuple(info)
        return out

    def stats(self):
        v = (C.c_longlong * 7)()
        self._lib.lbm_engine_stats(self._h, v)
        keys = ("ticks", "resident", "queued", "bytes", "peak_bytes", "planes_per_cta", "groups")
        return dict(zip(keys, list(v)))

    def close(self):
        if getattr(self, "_h", None):
            self._lib.lbm_engine_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
