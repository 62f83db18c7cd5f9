"""Plain FP64 CPU oracle of the two-component colour-gradient LB step (D3Q19).

TEST INFRASTRUCTURE ONLY. Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import this package. It shares no code with
the GPU library (``paper_2005_12764_gb300``) and never imports it.

``lbm_oracle.c`` holds the method (one plain loop per phase, in the paper's order);
this module compiles it with gcc on first use (or via :func:`build`) and wraps it
with ctypes. ``mini.py`` is a second, independently written NumPy version used to
cross-check the C code on tiny lattices.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "lbm_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB = os.path.join(_BUILD, "liboracle.so")
_lock = threading.Lock()
_lib = None

Q = 19


def build(force: bool = False) -> str:
    """Compile ``lbm_oracle.c`` into ``oracle/_build/liboracle.so`` (gcc, OpenMP).

    ``-ffp-contract=off`` keeps FP64 results identical on x86 and Arm.
    """
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        cmd = ["gcc", "-std=c11", "-O2", "-fopenmp", "-ffp-contract=off", "-fno-fast-math",
               "-fPIC", "-shared", "-o", tmp, _SRC, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB)
    return _LIB


class Params(C.Structure):
    _fields_ = [("nx", C.c_int), ("ny", C.c_int), ("nz", C.c_int),
                ("wall_y", C.c_int), ("wall_z", C.c_int),
                ("tau_r", C.c_double), ("tau_b", C.c_double),
                ("sigma", C.c_double), ("beta", C.c_double),
                ("A_nc", C.c_double), ("h_min", C.c_double), ("h_cut", C.c_double),
                ("g", C.c_double * 3), ("kolmogorov_amp", C.c_double),
                ("nc_lag", C.c_int), ("wall_u", C.c_double),
                ("model", C.c_int), ("G_sc", C.c_double)]


_D = C.POINTER(C.c_double)
_U8 = C.POINTER(C.c_uint8)
_L = C.POINTER(C.c_long)


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = C.CDLL(build())
            P = C.POINTER(Params)
            sig = {
                "or_lattice": (None, [C.POINTER(C.c_int), _D, C.POINTER(C.c_int), _D]),
                "or_feq": (None, [C.c_double, _D, _D]),
                "or_edm_source": (None, [C.c_double, _D, _D, _D]),
                "or_omega_eff": (C.c_double, [C.c_double] * 4),
                "or_bgk_edm": (None, [_D, C.c_double, _D, _D]),
                "or_perturb": (None, [_D, C.c_double, C.c_double, _D, _D]),
                "or_recolour": (None, [_D, C.c_double, C.c_double, C.c_double, _D, _D, _D]),
                "or_A_h": (C.c_double, [C.c_double] * 4),
                "or_nc_strength_node": (C.c_double, [P, _D, _U8, C.c_long, C.c_long, C.c_long]),
                "or_nc_strength_node_thr": (C.c_double, [P, _D, _U8, C.c_long, C.c_long,
                                                         C.c_long, C.c_double, C.c_double]),
                "or_nc_strength_node_g": (C.c_double, [P, _D, _U8, C.c_long, C.c_long, C.c_long,
                                                       C.c_double, C.c_double, _D]),
                "or_gradient": (None, [P, _D, _D, _D, _D]),
                "or_create": (C.c_void_p, [P]),
                "or_destroy": (None, [C.c_void_p]),
                "or_set_fields": (None, [C.c_void_p, _D, _D, _D]),
                "or_set_pins": (None, [C.c_void_p, _U8]),
                "or_get_pops": (None, [C.c_void_p, _D, _D]),
                "or_set_pops": (None, [C.c_void_p, _D, _D, _D]),
                "or_get_phi_lag": (None, [C.c_void_p, _D]),
                "or_stream_only": (None, [C.c_void_p, C.c_int]),
                "or_step": (None, [C.c_void_p, C.c_int]),
                "or_get_fields": (None, [C.c_void_p, _D, _D, _D, _D]),
                "or_get_forces": (None, [C.c_void_p, _D]),
                "or_totals": (None, [C.c_void_p, _D]),
                "or_step_nodes": (C.c_int, [P, _D, _D, _D, _U8, C.c_long, _L, _D, _D, _D]),
                "or_step_nodes_given_ah": (C.c_int, [P, _D, _D, _D, _U8, C.c_long, _L, _D, _D,
                                                     _D, _D]),
                "or_laplace": (None, [C.c_void_p, _D, _D]),
            }
            for name, (res, args) in sig.items():
                fn = getattr(lib, name)
                fn.restype = res
                fn.argtypes = args
            _lib = lib
    return _lib


def _d(a):
    return a.ctypes.data_as(_D)


def _f64(a, shape=None):
    a = np.ascontiguousarray(a, dtype=np.float64)
    if shape is not None:
        a = a.reshape(shape)
    return a


def make_params(nx, ny, nz, *, wall_y=0, wall_z=0, tau_r=1.0, tau_b=None, sigma=0.0,
                beta=0.7, A_nc=0.0, h_min=3.0, h_cut=None, g=(0.0, 0.0, 0.0),
                kolmogorov_amp=0.0, nc_lag=1, wall_u=0.0, model="colour", G_sc=0.0) -> Params:
    """Parameter block with the defaults of the method (h_cut = 2 h_min)."""
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
    p.nc_lag = int(nc_lag)
    p.wall_u = float(wall_u)
    p.model = {"colour": 0, "shan_chen": 1}[model] if isinstance(model, str) else int(model)
    p.G_sc = float(G_sc)
    return p


# ---------------------------------------------------------------- per-node routines
def lattice():
    """(c [19,3] int, w [19], opp [19] int, B [19]) of the D3Q19 set."""
    lib = _load()
    c = np.zeros((Q, 3), dtype=np.int32)
    w = np.zeros(Q)
    opp = np.zeros(Q, dtype=np.int32)
    b = np.zeros(Q)
    lib.or_lattice(c.ctypes.data_as(C.POINTER(C.c_int)), _d(w),
                   opp.ctypes.data_as(C.POINTER(C.c_int)), _d(b))
    return c, w, opp, b


def feq(rho, u):
    out = np.zeros(Q)
    _load().or_feq(float(rho), _d(_f64(u)), _d(out))
    return out


def edm_source(rho, u, F):
    out = np.zeros(Q)
    _load().or_edm_source(float(rho), _d(_f64(u)), _d(_f64(F)), _d(out))
    return out


def omega_eff(rho_r, rho_b, tau_r, tau_b):
    return _load().or_omega_eff(float(rho_r), float(rho_b), float(tau_r), float(tau_b))


def bgk_edm(f, omega, F):
    out = np.zeros(Q)
    _load().or_bgk_edm(_d(_f64(f)), float(omega), _d(_f64(F)), _d(out))
    return out


def perturb(f, omega, sigma, G):
    out = np.zeros(Q)
    _load().or_perturb(_d(_f64(f)), float(omega), float(sigma), _d(_f64(G)), _d(out))
    return out


def recolour(f, rho_r, rho_b, beta, G):
    a, b = np.zeros(Q), np.zeros(Q)
    _load().or_recolour(_d(_f64(f)), float(rho_r), float(rho_b), float(beta),
                        _d(_f64(G)), _d(a), _d(b))
    return a, b


def A_h(h, A, h_min, h_cut):
    return _load().or_A_h(float(h), float(A), float(h_min), float(h_cut))


def gradient(params: Params, phi):
    """Colour gradient of a node field phi [nz, ny, nx] -> G [3, nz, ny, nx]."""
    phi = _f64(phi)
    N = phi.size
    G = np.zeros((3, N))
    _load().or_gradient(C.byref(params), _d(phi), _d(G[0]), _d(G[1]), _d(G[2]))
    return G.reshape((3,) + phi.shape)


def nc_strength_node(params: Params, phi_ray, x, y, z, pin=None):
    """Near-contact strength A_h at one node, measured on the field phi_ray."""
    phi_ray = _f64(phi_ray)
    pin_p = None
    if pin is not None:
        pin = np.ascontiguousarray(pin, dtype=np.uint8)
        pin_p = pin.ctypes.data_as(_U8)
    return _load().or_nc_strength_node(C.byref(params), _d(phi_ray), pin_p, int(x), int(y),
                                       int(z))


def nc_strength_node_thr(params: Params, phi_ray, x, y, z, band, g_min, pin=None):
    """nc_strength_node with the reading's two thresholds given: the sign band of a
    ray sample (1e-5) and the least lagged gradient (1e-3)."""
    phi_ray = _f64(phi_ray)
    pin_p = None
    if pin is not None:
        pin = np.ascontiguousarray(pin, dtype=np.uint8)
        pin_p = pin.ctypes.data_as(_U8)
    return _load().or_nc_strength_node_thr(C.byref(params), _d(phi_ray), pin_p, int(x), int(y),
                                           int(z), float(band), float(g_min))


def nc_strength_node_g(params: Params, phi_ray, x, y, z, G, band=1e-5, g_min=1e-3, pin=None):
    """nc_strength_node_thr with the lagged gradient G' = (Gx, Gy, Gz) at the node given
    instead of evaluated from phi_ray."""
    phi_ray = _f64(phi_ray)
    g = np.ascontiguousarray(G, dtype=np.float64)
    pin_p = None
    if pin is not None:
        pin = np.ascontiguousarray(pin, dtype=np.uint8)
        pin_p = pin.ctypes.data_as(_U8)
    return _load().or_nc_strength_node_g(C.byref(params), _d(phi_ray), pin_p, int(x), int(y),
                                         int(z), float(band), float(g_min), _d(g))


def step_nodes(params: Params, fr, fb, phi_lag, nodes, pin=None, ah=None):
    """One step evaluated at the listed flat node indices from a given state.

    fr, fb: [19, N] post-collision populations; phi_lag: [N] lagged colour field.
    ah: optional near-contact strength of each listed node, used instead of the
    measured one. Returns (fr_new [n,19], fb_new [n,19], F [n,3]).
    """
    fr = _f64(fr)
    fb = _f64(fb)
    phi_lag = _f64(phi_lag)
    nodes = np.ascontiguousarray(nodes, dtype=np.int64)
    n = nodes.size
    oa, ob, F = np.zeros((n, Q)), np.zeros((n, Q)), np.zeros((n, 3))
    pin_p = None
    if pin is not None:
        pin = np.ascontiguousarray(pin, dtype=np.uint8)
        pin_p = pin.ctypes.data_as(_U8)
    if ah is None:
        rc = _load().or_step_nodes(C.byref(params), _d(fr), _d(fb), _d(phi_lag), pin_p, n,
                                   nodes.ctypes.data_as(_L), _d(oa), _d(ob), _d(F))
    else:
        ah = _f64(ah).reshape(-1)
        assert ah.size == n
        rc = _load().or_step_nodes_given_ah(C.byref(params), _d(fr), _d(fb), _d(phi_lag), pin_p,
                                            n, nodes.ctypes.data_as(_L), _d(ah), _d(oa),
                                            _d(ob), _d(F))
    if rc != 0:
        raise ValueError("or_step_nodes needs the lagged near-contact reading")
    return oa, ob, F


# ---------------------------------------------------------------- whole-lattice state
class Lattice:
    """FP64 lattice state advanced by the oracle; arrays are [.., nz, ny, nx]."""

    def __init__(self, params: Params):
        self.params = params
        self.shape = (params.nz, params.ny, params.nx)
        self.N = params.nx * params.ny * params.nz
        self._lib = _load()
        self._s = self._lib.or_create(C.byref(params))
        if not self._s:
            raise MemoryError("oracle allocation failed")

    def close(self):
        if getattr(self, "_s", None):
            self._lib.or_destroy(self._s)
            self._s = None

    def __del__(self):
        self.close()

    def set_fields(self, rho_r, rho_b, u=None):
        rr = _f64(rho_r).reshape(-1)
        rb = _f64(rho_b).reshape(-1)
        up = None
        if u is not None:
            uu = _f64(u).reshape(3, -1)
            up = _d(uu)
        self._lib.or_set_fields(self._s, _d(rr), _d(rb), up)

    def set_pins(self, mask):
        if mask is None:
            self._lib.or_set_pins(self._s, None)
            return
        m = np.ascontiguousarray(mask, dtype=np.uint8).reshape(-1)
        self._lib.or_set_pins(self._s, m.ctypes.data_as(_U8))

    def step(self, n=1):
        self._lib.or_step(self._s, int(n))

    def stream_only(self, n=1):
        self._lib.or_stream_only(self._s, int(n))

    def get_pops(self):
        fr, fb = np.zeros((Q, self.N)), np.zeros((Q, self.N))
        self._lib.or_get_pops(self._s, _d(fr), _d(fb))
        return fr.reshape((Q,) + self.shape), fb.reshape((Q,) + self.shape)

    def set_pops(self, fr, fb, phi_lag=None):
        fr = _f64(fr).reshape(Q, -1)
        fb = _f64(fb).reshape(Q, -1)
        pl = None if phi_lag is None else _d(_f64(phi_lag).reshape(-1))
        self._lib.or_set_pops(self._s, _d(fr), _d(fb), pl)

    def get_phi_lag(self):
        out = np.zeros(self.N)
        self._lib.or_get_phi_lag(self._s, _d(out))
        return out.reshape(self.shape)

    def get_fields(self):
        """dict of rho_r, rho_b, u [3,...], phi (u is the physical velocity)."""
        rr, rb, u, phi = (np.zeros(self.N), np.zeros(self.N), np.zeros((3, self.N)),
                          np.zeros(self.N))
        self._lib.or_get_fields(self._s, _d(rr), _d(rb), _d(u), _d(phi))
        s = self.shape
        return {"rho_r": rr.reshape(s), "rho_b": rb.reshape(s), "u": u.reshape((3,) + s),
                "phi": phi.reshape(s)}

    def get_forces(self):
        F = np.zeros((3, self.N))
        self._lib.or_get_forces(self._s, _d(F))
        return F.reshape((3,) + self.shape)

    def totals(self):
        out = np.zeros(5)
        self._lib.or_totals(self._s, _d(out))
        return out

    def laplace(self, centre):
        out = np.zeros(5)
        self._lib.or_laplace(self._s, _d(_f64(centre)), _d(out))
        return {"dp": out[0], "R_eff": out[1], "p_in": out[2], "p_out": out[3], "V": out[4]}
