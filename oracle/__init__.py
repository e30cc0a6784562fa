"""ctypes wrapper around the plain FP64 CPU oracle (kerr_oracle.c).

TEST INFRASTRUCTURE ONLY.  Only the test suite, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import this package.  The product library never
links, loads or calls it, and it shares no code with the product.

Scenes are plain dicts (see ``paper_1601_02063_gb300.workloads``); this module marshals
them into the oracle's own C struct.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "kerr_oracle.c")
_LIB_PATH = os.path.join(_HERE, "liboracle.so")
MAX_FREQ = 8

STATUS = {"running": 0, "escaped": 1, "captured": 2, "disk_hit": 3, "maxsteps": 4, "numerr": 5}
EMITTERS = {"none": 0, "thin_disk": 1, "torus": 2, "const": 3, "nt_disk": 4, "synch": 5, "spot": 6}
CONVENTIONS = {"physical": 0, "literal": 1}
RT_CONTROL = {"controlled": 0, "ride": 1}


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (IEEE FP64, no FMA contraction, OpenMP)."""
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= max(os.path.getmtime(_SRC),
                                                   os.path.getmtime(_SRC[:-1] + "h"))):
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math", "-fopenmp",
           "-fPIC", "-shared", "-o", tmp, _SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


class Scene(C.Structure):
    _fields_ = [
        ("a", C.c_double), ("r_obs", C.c_double), ("theta_obs", C.c_double),
        ("phi_obs", C.c_double),
        ("alpha_min", C.c_double), ("alpha_max", C.c_double),
        ("beta_min", C.c_double), ("beta_max", C.c_double),
        ("n_alpha", C.c_int32), ("n_beta", C.c_int32),
        ("emitter", C.c_int32), ("n_freq", C.c_int32),
        ("freqs", C.c_double * MAX_FREQ),
        ("r_in", C.c_double), ("r_out", C.c_double), ("q_emis", C.c_double),
        ("ne_index", C.c_double), ("theta_width", C.c_double),
        ("T0", C.c_double), ("T_index", C.c_double), ("C_norm", C.c_double),
        ("rtol", C.c_double), ("h0", C.c_double), ("hmax_frac", C.c_double),
        ("horizon_factor", C.c_double),
        ("max_steps", C.c_int32), ("convention", C.c_int32),
        ("n_e0", C.c_double), ("beta_B", C.c_double), ("mass", C.c_double),
        ("spot_r", C.c_double), ("spot_size", C.c_double), ("spot_phase", C.c_double),
        ("t_obs", C.c_double),
        ("rt_control", C.c_int32), ("pad_", C.c_int32),
    ]


class Result(C.Structure):
    _fields_ = [
        ("status", C.c_int32), ("n_acc", C.c_int32), ("n_rej", C.c_int32),
        ("n_cross", C.c_int32),
        ("r_cross", C.c_double), ("phi_cross", C.c_double),
        ("r_hit", C.c_double), ("phi_hit", C.c_double), ("g", C.c_double),
        ("intensity", C.c_double), ("H_end", C.c_double), ("Q_drift", C.c_double),
        ("s_end", C.c_double), ("L", C.c_double), ("Q0", C.c_double),
        ("y_end", C.c_double * 6),
        ("I_nu", C.c_double * MAX_FREQ), ("tau_nu", C.c_double * MAX_FREQ),
    ]


RESULT_DTYPE = np.dtype([
    ("status", np.int32), ("n_acc", np.int32), ("n_rej", np.int32), ("n_cross", np.int32),
    ("r_cross", np.float64), ("phi_cross", np.float64), ("r_hit", np.float64),
    ("phi_hit", np.float64), ("g", np.float64), ("intensity", np.float64),
    ("H_end", np.float64), ("Q_drift", np.float64), ("s_end", np.float64),
    ("L", np.float64), ("Q0", np.float64), ("y_end", np.float64, (6,)),
    ("I_nu", np.float64, (MAX_FREQ,)), ("tau_nu", np.float64, (MAX_FREQ,)),
])
assert RESULT_DTYPE.itemsize == C.sizeof(Result)

_lib = None


def lib():
    global _lib
    if _lib is None:
        _lib = C.CDLL(build())
        D, I32, I64, P = C.c_double, C.c_int32, C.c_int64, C.POINTER
        sigs = {
            "orc_horizon": (D, [D]),
            "orc_isco": (D, [D]),
            "orc_nt_flux": (D, [D, D]),
            "orc_circ_E": (D, [D, D]),
            "orc_circ_L": (D, [D, D]),
            "orc_bessel_k2": (D, [D]),
            "orc_spot_region": (D, [P(Scene), D, P(D), P(D)]),
            "orc_spot_omega": (D, [P(Scene)]),
            "orc_r_g": (D, [D]),
            "orc_synch_coeffs": (None, [P(Scene), D, D, D, P(D), P(D)]),
            "orc_ck_tableau": (None, [P(D), P(D), P(D), P(D)]),
            "orc_pixel_center": (None, [P(Scene), I32, I32, P(D), P(D)]),
            "orc_observer_point": (None, [P(Scene), D, D, P(D)]),
            "orc_init_ray": (None, [P(Scene), D, D, P(D), P(D), P(D), P(D)]),
            "orc_geodesic_rhs": (None, [D, D, P(D), P(D)]),
            "orc_disk_redshift": (D, [D, D, D]),
            "orc_torus_norm": (D, [D, D, D, D, D, D]),
            "orc_trace_ray": (C.c_int, [P(Scene), D, D, P(Result)]),
            "orc_trace_path": (C.c_int, [P(Scene), D, D, I32, P(D), P(D), P(I32),
                                         P(Result)]),
            "orc_render": (C.c_int, [P(Scene), C.c_void_p, I64, C.c_void_p, I32]),
            "orc_trace_list": (C.c_int, [P(Scene), C.c_void_p, I64, C.c_void_p, I32]),
            "orc_max_threads": (C.c_int, []),
        }
        for name, (res, args) in sigs.items():
            fn = getattr(_lib, name)
            fn.restype = res
            fn.argtypes = args
    return _lib


def torus_norm(a, nu=1.0, ne_index=1.5, T0=10.0, T_index=0.84, r_outer=1000.0) -> float:
    return lib().orc_torus_norm(a, nu, ne_index, T0, T_index, r_outer)


def make_scene(d: dict) -> Scene:
    """Marshal a scene dict into the oracle's struct.  A torus without an explicit
    C_norm is normalised by the oracle's own quadrature."""
    sc = Scene()
    for k in ("a", "r_obs", "theta_obs", "phi_obs", "alpha_min", "alpha_max", "beta_min",
              "beta_max", "r_in", "r_out", "q_emis", "ne_index", "theta_width", "T0",
              "T_index", "rtol", "h0", "hmax_frac", "horizon_factor"):
        setattr(sc, k, float(d[k]))
    sc.n_alpha, sc.n_beta = int(d["n_alpha"]), int(d["n_beta"])
    sc.emitter = EMITTERS[d["emitter"]]
    freqs = list(d.get("freqs", []))
    assert len(freqs) <= MAX_FREQ
    sc.n_freq = len(freqs)
    for i, f in enumerate(freqs):
        sc.freqs[i] = float(f)
    sc.max_steps = int(d["max_steps"])
    sc.convention = CONVENTIONS[d.get("convention", "physical")]
    sc.rt_control = RT_CONTROL[d.get("rt_control", "controlled")]
    sc.n_e0 = float(d.get("n_e0", 0.0))
    sc.beta_B = float(d.get("beta_B", 0.0))
    sc.mass = float(d.get("mass", 0.0))
    for k in ("spot_r", "spot_size", "spot_phase", "t_obs"):
        setattr(sc, k, float(d.get(k, 0.0)))
    cn = d.get("C_norm")
    if cn is None:
        cn = torus_norm(d["a"], d.get("nu_norm", 1.0), d["ne_index"], d["T0"], d["T_index"],
                        d.get("r_norm_outer", 1000.0)) if d["emitter"] == "torus" else 0.0
    sc.C_norm = float(cn)
    return sc


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(C.c_void_p)


def default_threads() -> int:
    return max(1, len(os.sched_getaffinity(0)))


def trace_ray(scene: dict, alpha: float, beta: float) -> Result:
    sc = make_scene(scene)
    out = Result()
    lib().orc_trace_ray(C.byref(sc), float(alpha), float(beta), C.byref(out))
    return out


def render(scene: dict, pixels=None, threads: int = 0) -> np.ndarray:
    """Trace every pixel (or the given flat pixel indices j*n_alpha+i); structured array."""
    sc = make_scene(scene)
    n = sc.n_alpha * sc.n_beta if pixels is None else len(pixels)
    out = np.zeros(n, dtype=RESULT_DTYPE)
    pix = None if pixels is None else np.ascontiguousarray(pixels, dtype=np.int64)
    lib().orc_render(C.byref(sc), None if pix is None else _ptr(pix), n, _ptr(out),
                     threads or default_threads())
    return out


def trace_list(scene: dict, rays: np.ndarray, threads: int = 0) -> np.ndarray:
    """rays[n,4] = (alpha, beta, a, cos i); other parameters from ``scene``."""
    sc = make_scene(scene)
    rays = np.ascontiguousarray(rays, dtype=np.float64)
    out = np.zeros(len(rays), dtype=RESULT_DTYPE)
    lib().orc_trace_list(C.byref(sc), _ptr(rays), len(rays), _ptr(out),
                         threads or default_threads())
    return out


def init_ray(scene: dict, alpha: float, beta: float):
    sc = make_scene(scene)
    y0 = (C.c_double * 6)()
    L, Q = C.c_double(), C.c_double()
    vin = (C.c_double * 3)()
    lib().orc_init_ray(C.byref(sc), alpha, beta, y0, C.byref(L), C.byref(Q), vin)
    return np.array(y0[:]), L.value, Q.value, np.array(vin[:])


def observer_point(scene: dict, alpha: float, beta: float) -> np.ndarray:
    sc = make_scene(scene)
    xyz = (C.c_double * 3)()
    lib().orc_observer_point(C.byref(sc), alpha, beta, xyz)
    return np.array(xyz[:])


def geodesic_rhs(a: float, L: float, y) -> np.ndarray:
    yy = (C.c_double * 6)(*[float(v) for v in y])
    f = (C.c_double * 6)()
    lib().orc_geodesic_rhs(a, L, yy, f)
    return np.array(f[:])


def trace_path(scene: dict, alpha: float, beta: float, max_pts: int = 200000):
    sc = make_scene(scene)
    n_comp = 6 + (2 * sc.n_freq if sc.emitter in (2, 3, 5) else 0)
    s = np.zeros(max_pts)
    y = np.zeros((max_pts, n_comp))
    npts = C.c_int32()
    out = Result()
    lib().orc_trace_path(C.byref(sc), alpha, beta, max_pts,
                         s.ctypes.data_as(C.POINTER(C.c_double)),
                         y.ctypes.data_as(C.POINTER(C.c_double)), C.byref(npts), C.byref(out))
    return s[:npts.value], y[:npts.value], out


def ck_tableau():
    c, a, b5, b4 = (C.c_double * 6)(), (C.c_double * 36)(), (C.c_double * 6)(), (C.c_double * 6)()
    lib().orc_ck_tableau(c, a, b5, b4)
    return np.array(c[:]), np.array(a[:]).reshape(6, 6), np.array(b5[:]), np.array(b4[:])


def horizon(a: float) -> float:
    return lib().orc_horizon(a)


def isco(a: float) -> float:
    return lib().orc_isco(a)


def nt_flux(a: float, r: float) -> float:
    """8 pi F(r) / 3 of the Novikov-Thorne disk (Page-Thorne integral by quadrature)."""
    return lib().orc_nt_flux(float(a), float(r))


def bessel_k2(x: float) -> float:
    """K_2(x) by quadrature of its integral definition."""
    return lib().orc_bessel_k2(float(x))


def spot_omega(scene: dict) -> float:
    """Angular velocity of the hot spot's circular orbit."""
    return lib().orc_spot_omega(C.byref(make_scene(scene)))


def spot_region(scene: dict, y, sgn: float = -1.0) -> tuple[float, float]:
    """(max(d - 4 r_spot, -z), d) of the hot spot at state y (r, theta, phi, t, ...)."""
    yy = (C.c_double * 6)(*[float(v) for v in list(y)[:6]])
    d = C.c_double()
    v = lib().orc_spot_region(C.byref(make_scene(scene)), float(sgn), yy, C.byref(d))
    return v, d.value


def r_g(mass: float) -> float:
    """G M / c^2 in cm for a mass in solar masses."""
    return lib().orc_r_g(float(mass))


def synch_coeffs(scene: dict, r: float, cost: float, nu0: float) -> tuple[float, float]:
    """(j_nu, alpha_nu) of the synchrotron shell in the fluid frame, CGS."""
    sc = make_scene(scene)
    j, al = C.c_double(), C.c_double()
    lib().orc_synch_coeffs(C.byref(sc), float(r), float(cost), float(nu0), C.byref(j),
                           C.byref(al))
    return j.value, al.value


def circ_E(a: float, r: float) -> float:
    return lib().orc_circ_E(float(a), float(r))


def circ_L(a: float, r: float) -> float:
    return lib().orc_circ_L(float(a), float(r))


def disk_redshift(a: float, r: float, L: float) -> float:
    return lib().orc_disk_redshift(a, r, L)
