"""Thin ctypes binding of the C ABI in include/odyssey.h (argument marshalling only).

Every function of the header is exposed under the same name.  PyTorch provides device
memory and streams: tensors are passed as raw device pointers.  Loading fails loudly if
the CUDA library has not been built; there is no CPU fallback.
"""
from __future__ import annotations

import ctypes as C
import functools
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libodyssey_gb300.so")
MAX_FREQ = 8

(OK, ERR_INVALID_ARG, ERR_CUDA, ERR_TIMEOUT, ERR_DEVICE_FLAG, ERR_NO_DEVICE, ERR_UNSUPPORTED,
 ERR_TOO_LARGE) = range(8)
STATIC_MAX_SCENES = 64
RUNNING, ESCAPED, CAPTURED, DISK_HIT, MAXSTEPS, NUMERR = range(6)
EMITTERS = {"none": 0, "thin_disk": 1, "torus": 2, "nt_disk": 3, "synch": 4, "spot": 5}
PRECISIONS = {"fp64": 0, "mixed": 1}
CONVENTIONS = {"physical": 0, "literal": 1}
RT_CONTROL = {"controlled": 0, "ride": 1}


class odx_scene(C.Structure):
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
        ("precision", C.c_int32), ("rt_control", C.c_int32),
        ("rtol_fp32", C.c_double), ("r_switch", C.c_double),
        ("n_e0", C.c_double), ("beta_B", C.c_double), ("mass", C.c_double),
        ("spot_r", C.c_double), ("spot_size", C.c_double), ("spot_phase", C.c_double),
        ("t_obs", C.c_double),
    ]


class odx_ray_record(C.Structure):
    _fields_ = [
        ("status", C.c_int32), ("n_acc", C.c_int32), ("n_rej", C.c_int32),
        ("n_cross", C.c_int32),
        ("r_cross", C.c_double), ("phi_cross", C.c_double),
        ("r_hit", C.c_double), ("phi_hit", C.c_double), ("g", C.c_double),
        ("intensity", C.c_double), ("H_end", C.c_double), ("Q_drift", C.c_double),
    ]


class odx_launch(C.Structure):
    _fields_ = [("block", C.c_int32), ("blocks_per_sm", C.c_int32), ("chunk", C.c_int32),
                ("persistent", C.c_int32), ("fp64_batch", C.c_int32)]


class odx_stats(C.Structure):
    _fields_ = [("rays", C.c_int64), ("steps_accepted", C.c_int64),
                ("steps_rejected", C.c_int64), ("steps_fp64", C.c_int64),
                ("lane_slots", C.c_int64), ("lane_active", C.c_int64),
                ("error_flag", C.c_int32), ("reserved", C.c_int32),
                ("trace_launches", C.c_int64), ("trace_ms", C.c_double)]


RECORD_DTYPE = np.dtype([
    ("status", np.int32), ("n_acc", np.int32), ("n_rej", np.int32), ("n_cross", np.int32),
    ("r_cross", np.float64), ("phi_cross", np.float64), ("r_hit", np.float64),
    ("phi_hit", np.float64), ("g", np.float64), ("intensity", np.float64),
    ("H_end", np.float64), ("Q_drift", np.float64),
])
RECORD_BYTES = 80
assert C.sizeof(odx_ray_record) == RECORD_BYTES == RECORD_DTYPE.itemsize
assert C.sizeof(odx_scene) == 328

# (name, restype, argtypes) of every entry point in include/odyssey.h
_P = C.c_void_p
_SIGNATURES = [
    ("odx_version", C.c_char_p, []),
    ("odx_error_string", C.c_char_p, [C.c_int32]),
    ("odx_last_error", C.c_char_p, [_P]),
    ("odx_create", C.c_int32, [C.POINTER(_P), C.c_int32]),
    ("odx_destroy", C.c_int32, [_P]),
    ("odx_set_launch", C.c_int32, [_P, C.POINTER(odx_launch)]),
    ("odx_get_launch", C.c_int32, [_P, C.POINTER(odx_launch)]),
    ("odx_render", C.c_int32, [_P, C.POINTER(odx_scene), C.c_int32, _P, _P, _P]),
    ("odx_trace_rays", C.c_int32, [_P, C.POINTER(odx_scene), _P, C.c_int64, _P, _P, _P]),
    ("odx_render_host", C.c_int32, [_P, C.POINTER(odx_scene), C.c_int32, _P, _P]),
    ("odx_get_stats", C.c_int32, [_P, _P, C.POINTER(odx_stats), C.c_int32]),
    ("odx_sync", C.c_int32, [_P, _P, C.c_double]),
    ("odx_image_flux", C.c_int32, [_P, C.POINTER(odx_scene), C.c_int32, _P, _P, _P, _P]),
    ("odx_set_kernel_timing", C.c_int32, [_P, C.c_int32]),
    ("odx_torus_norm", C.c_double, [C.c_double] * 6),
    ("odx_fma_peak", C.c_int32, [_P, C.c_int32, C.POINTER(C.c_double)]),
    ("odx_render_static", C.c_int32, [C.POINTER(odx_scene), C.c_int32, _P, _P, _P]),
    ("odx_graph_create", C.c_int32, [_P, C.POINTER(odx_scene), C.c_int32, _P, _P,
                                     C.POINTER(_P)]),
    ("odx_graph_launch", C.c_int32, [_P, _P]),
    ("odx_graph_destroy", C.c_int32, [_P]),
    ("odx_autotune", C.c_int32, [_P, C.POINTER(odx_scene), C.c_int32, _P,
                                 C.POINTER(odx_launch)]),
    ("odx_mlp_create", C.c_int32, [_P, C.c_int64, C.c_uint64, C.POINTER(_P)]),
    ("odx_mlp_destroy", C.c_int32, [_P]),
    ("odx_mlp_get_params", C.c_int32, [_P, _P]),
    ("odx_mlp_set_params", C.c_int32, [_P, _P]),
    ("odx_mlp_forward", C.c_int32, [_P, _P, C.c_int64, _P, _P]),
    ("odx_mlp_set_wait_limit", C.c_int32, [_P, C.c_uint32]),
    ("odx_mlp_gradients", C.c_int32, [_P, _P, _P, C.c_int64, _P, _P]),
    ("odx_mlp_train_step", C.c_int32, [_P, _P, _P, C.c_int64, C.c_float, _P, _P]),
    ("odx_mlp_targets", C.c_int32, [_P, _P, _P, C.c_int64, C.c_double, _P, _P, _P]),
    ("odx_surrogate_render", C.c_int32, [_P, C.POINTER(odx_scene), C.c_double, C.c_double,
                                         C.c_double, _P, _P, _P, C.POINTER(C.c_int64), _P]),
]
MLP_PARAMS = 199684
SYMBOLS = [s[0] for s in _SIGNATURES]

_lib = None


def lib() -> C.CDLL:
    """Load the CUDA library (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(
                f"{LIB_PATH} is missing: build it with `python -m paper_1601_02063_gb300.build` "
                "(there is no CPU fallback)")
        L = C.CDLL(LIB_PATH)
        for name, res, args in _SIGNATURES:
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _lib = L
    return _lib


class OdxError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"odx error {code} ({error_string(code)}): {msg}")
        self.code = code


def error_string(code: int) -> str:
    return lib().odx_error_string(code).decode()


# ---- same-name wrappers --------------------------------------------------------------------
def odx_version() -> str:
    return lib().odx_version().decode()


def odx_create(device: int = 0):
    h = C.c_void_p()
    rc = lib().odx_create(C.byref(h), device)
    if rc != OK:
        raise OdxError(rc, f"odx_create(device={device})")
    return h


def odx_destroy(ctx) -> None:
    lib().odx_destroy(ctx)


def odx_last_error(ctx) -> str:
    return lib().odx_last_error(ctx).decode()


def _check(ctx, rc: int, what: str) -> int:
    if rc != OK:
        raise OdxError(rc, f"{what}: {odx_last_error(ctx)}")
    return rc


def odx_set_launch(ctx, block=128, blocks_per_sm=3, chunk=0, persistent=2,
                   fp64_batch=16) -> None:
    L = odx_launch(block, blocks_per_sm, chunk, persistent, fp64_batch)
    _check(ctx, lib().odx_set_launch(ctx, C.byref(L)), "odx_set_launch")


def odx_get_launch(ctx) -> dict:
    L = odx_launch()
    _check(ctx, lib().odx_get_launch(ctx, C.byref(L)), "odx_get_launch")
    return {f: getattr(L, f) for f, _ in odx_launch._fields_}


def odx_render(ctx, scenes, records_ptr: int, image_ptr: int | None, stream: int | None = None,
               check: bool = True) -> int:
    arr = scene_array(scenes)
    rc = lib().odx_render(ctx, arr, len(arr), records_ptr, image_ptr or None, stream or None)
    return _check(ctx, rc, "odx_render") if check else rc


def odx_trace_rays(ctx, proto, rays_ptr: int, n: int, records_ptr: int, image_ptr: int | None,
                   stream: int | None = None, check: bool = True) -> int:
    arr = scene_array([proto])
    rc = lib().odx_trace_rays(ctx, arr, rays_ptr or None, n, records_ptr, image_ptr or None,
                              stream or None)
    return _check(ctx, rc, "odx_trace_rays") if check else rc


def odx_render_host(ctx, scenes, records_host: np.ndarray, image_host: np.ndarray | None):
    arr = scene_array(scenes)
    rc = lib().odx_render_host(ctx, arr, len(arr), records_host.ctypes.data,
                               None if image_host is None else image_host.ctypes.data)
    return _check(ctx, rc, "odx_render_host")


def odx_get_stats(ctx, stream: int | None = None, reset: bool = False) -> dict:
    s = odx_stats()
    _check(ctx, lib().odx_get_stats(ctx, stream or None, C.byref(s), int(reset)), "odx_get_stats")
    return {f: getattr(s, f) for f, _ in odx_stats._fields_}


def odx_image_flux(ctx, scenes, image_ptr: int, flux_ptr: int, lum_ptr: int | None = None,
                   stream: int | None = None) -> None:
    arr = scene_array(scenes)
    _check(ctx, lib().odx_image_flux(ctx, arr, len(arr), image_ptr, flux_ptr, lum_ptr or None,
                                     stream or None), "odx_image_flux")


def odx_set_kernel_timing(ctx, on: bool) -> None:
    _check(ctx, lib().odx_set_kernel_timing(ctx, int(bool(on))), "odx_set_kernel_timing")


def odx_sync(ctx, stream: int | None = None, timeout_s: float = 600.0) -> None:
    _check(ctx, lib().odx_sync(ctx, stream or None, timeout_s), "odx_sync")


@functools.lru_cache(maxsize=256)
def _torus_norm(a, nu, ne_index, T0, T_index, r_outer) -> float:
    return lib().odx_torus_norm(a, nu, ne_index, T0, T_index, r_outer)


def odx_torus_norm(a, nu=1.0, ne_index=1.5, T0=10.0, T_index=0.84, r_outer=1000.0) -> float:
    """Emissivity normalisation (a pure function of its arguments: memoised, so that
    scene structs built per call cost no quadrature)."""
    return _torus_norm(float(a), float(nu), float(ne_index), float(T0), float(T_index),
                       float(r_outer))


def odx_fma_peak(ctx, precision: str) -> float:
    v = C.c_double()
    _check(ctx, lib().odx_fma_peak(ctx, PRECISIONS[precision], C.byref(v)), "odx_fma_peak")
    return v.value


def odx_render_static(scenes, records_ptr: int, image_ptr: int | None,
                      stream: int | None = None) -> int:
    """Render without any device allocation by the library (fixed static scratch); returns
    the status code (no context, so no error text)."""
    arr = scene_array(scenes)
    return lib().odx_render_static(arr, len(arr), records_ptr, image_ptr or None, stream or None)


def odx_graph_create(ctx, scenes, records_ptr: int, image_ptr: int | None):
    arr = scene_array(scenes)
    g = C.c_void_p()
    _check(ctx, lib().odx_graph_create(ctx, arr, len(arr), records_ptr, image_ptr or None,
                                       C.byref(g)), "odx_graph_create")
    return g


def odx_graph_launch(ctx, graph, stream: int | None = None) -> None:
    _check(ctx, lib().odx_graph_launch(graph, stream or None), "odx_graph_launch")


def odx_graph_destroy(graph) -> None:
    lib().odx_graph_destroy(graph)


def odx_autotune(ctx, scenes, stream: int | None = None) -> dict:
    arr = scene_array(scenes)
    L = odx_launch()
    _check(ctx, lib().odx_autotune(ctx, arr, len(arr), stream or None, C.byref(L)),
           "odx_autotune")
    return {f: getattr(L, f) for f, _ in odx_launch._fields_}


def _ok(rc: int, what: str) -> None:
    if rc != OK:
        raise OdxError(rc, what)


def odx_mlp_create(ctx, max_batch: int, seed: int):
    h = C.c_void_p()
    _ok(lib().odx_mlp_create(ctx, max_batch, seed, C.byref(h)), "odx_mlp_create")
    return h


def odx_mlp_destroy(mlp) -> None:
    lib().odx_mlp_destroy(mlp)


def odx_mlp_get_params(mlp) -> np.ndarray:
    out = np.empty(MLP_PARAMS, dtype=np.float32)
    _ok(lib().odx_mlp_get_params(mlp, out.ctypes.data), "odx_mlp_get_params")
    return out


def odx_mlp_set_params(mlp, params: np.ndarray) -> None:
    p = np.ascontiguousarray(params, dtype=np.float32)
    assert p.size == MLP_PARAMS
    _ok(lib().odx_mlp_set_params(mlp, p.ctypes.data), "odx_mlp_set_params")


def odx_mlp_set_wait_limit(mlp, tries: int) -> None:
    _ok(lib().odx_mlp_set_wait_limit(mlp, int(tries)), "odx_mlp_set_wait_limit")


def odx_mlp_forward(mlp, x_ptr: int, n: int, y_ptr: int, stream: int | None = None) -> None:
    _ok(lib().odx_mlp_forward(mlp, x_ptr, n, y_ptr, stream or None), "odx_mlp_forward")


def odx_mlp_gradients(mlp, x_ptr: int, t_ptr: int, n: int):
    g = np.empty(MLP_PARAMS, dtype=np.float32)
    loss = np.zeros(1, dtype=np.float32)
    _ok(lib().odx_mlp_gradients(mlp, x_ptr, t_ptr, n, g.ctypes.data, loss.ctypes.data),
        "odx_mlp_gradients")
    return g, float(loss[0])


def odx_mlp_train_step(mlp, x_ptr: int, t_ptr: int, n: int, lr: float, loss_ptr: int | None,
                       stream: int | None = None) -> None:
    _ok(lib().odx_mlp_train_step(mlp, x_ptr, t_ptr, n, lr, loss_ptr or None, stream or None),
        "odx_mlp_train_step")


def odx_mlp_targets(ctx, rec_ptr: int, rays_ptr: int, n: int, r_max: float, x_ptr: int,
                    t_ptr: int, stream: int | None = None) -> None:
    _check(ctx, lib().odx_mlp_targets(ctx, rec_ptr, rays_ptr, n, r_max, x_ptr, t_ptr,
                                      stream or None), "odx_mlp_targets")


def odx_surrogate_render(mlp, scene, band: float, p_lo: float, p_hi: float, fb_rec_ptr: int,
                         fb_pix_ptr: int | None, image_ptr: int, stream: int | None = None) -> int:
    arr = scene_array([scene])
    n_fb = C.c_int64()
    _ok(lib().odx_surrogate_render(mlp, arr, band, p_lo, p_hi, fb_rec_ptr, fb_pix_ptr or None,
                                   image_ptr, C.byref(n_fb), stream or None),
        "odx_surrogate_render")
    return n_fb.value


# ---- marshalling helpers ----------------------------------------------------------------------
def scene_struct(d: dict) -> odx_scene:
    """A scene dict (see workloads.scene) as the C struct.  A torus without C_norm is
    normalised with odx_torus_norm."""
    s = odx_scene()
    for k in ("a", "r_obs", "theta_obs", "phi_obs", "alpha_min", "alpha_max", "beta_min",
              "beta_max", "r_in", "r_out", "q_emis", "ne_index", "theta_width", "T0",
              "T_index", "rtol", "h0", "hmax_frac", "horizon_factor", "rtol_fp32", "r_switch",
              "n_e0", "beta_B", "mass", "spot_r", "spot_size", "spot_phase", "t_obs"):
        setattr(s, k, float(d[k]))
    s.n_alpha, s.n_beta = int(d["n_alpha"]), int(d["n_beta"])
    s.emitter = EMITTERS[d["emitter"]]
    freqs = list(d.get("freqs", []))
    if len(freqs) > MAX_FREQ:
        raise ValueError(f"at most {MAX_FREQ} frequencies")
    s.n_freq = len(freqs)
    for i, f in enumerate(freqs):
        s.freqs[i] = float(f)
    s.max_steps = int(d["max_steps"])
    s.convention = CONVENTIONS[d.get("convention", "physical")]
    s.precision = PRECISIONS[d.get("precision", "fp64")]
    s.rt_control = RT_CONTROL[d.get("rt_control", "controlled")]
    cn = d.get("C_norm")
    if cn is None:
        cn = odx_torus_norm(d["a"], d.get("nu_norm", 1.0), d["ne_index"], d["T0"],
                            d["T_index"], d.get("r_norm_outer", 1000.0)) \
            if d["emitter"] == "torus" else 0.0
    s.C_norm = float(cn)
    return s


def scene_array(scenes):
    scenes = list(scenes) if isinstance(scenes, (list, tuple)) else [scenes]
    arr = (odx_scene * len(scenes))()
    for i, d in enumerate(scenes):
        arr[i] = d if isinstance(d, odx_scene) else scene_struct(d)
    return arr


def n_rays(scenes) -> int:
    scenes = scenes if isinstance(scenes, (list, tuple)) else [scenes]
    return sum(int(d["n_alpha"]) * int(d["n_beta"]) for d in scenes)


def image_planes(d: dict) -> int:
    return len(d["freqs"]) if d["emitter"] in ("torus", "nt_disk", "synch", "spot") else 1


def n_image(scenes) -> int:
    scenes = scenes if isinstance(scenes, (list, tuple)) else [scenes]
    return sum(image_planes(d) * int(d["n_alpha"]) * int(d["n_beta"]) for d in scenes)


def records_to_numpy(rec_tensor) -> np.ndarray:
    """Device or host tensor of n*80 bytes (any dtype) -> numpy structured records."""
    raw = rec_tensor.detach().cpu().contiguous().view(-1).numpy().view(np.uint8)
    return raw.view(RECORD_DTYPE)


class Tracer:
    """Owns one odx context; allocates outputs as torch tensors (plumbing only)."""

    def __init__(self, device: int = 0):
        import torch
        self.torch = torch
        self.device = device
        self.ctx = odx_create(device)

    def close(self):
        if self.ctx is not None:
            odx_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def alloc(self, n_rec: int, n_img: int):
        t = self.torch
        dev = f"cuda:{self.device}"
        rec = t.empty((max(n_rec, 1), RECORD_BYTES // 8), dtype=t.float64, device=dev)
        img = t.empty(max(n_img, 1), dtype=t.float64, device=dev)
        return rec, img

    def render(self, scenes, stream=None, out=None):
        scenes = scenes if isinstance(scenes, (list, tuple)) else [scenes]
        rec, img = out if out is not None else self.alloc(n_rays(scenes), n_image(scenes))
        st = stream if stream is not None else self.torch.cuda.current_stream(self.device)
        odx_render(self.ctx, scenes, rec.data_ptr(), img.data_ptr(), st.cuda_stream)
        return rec, img

    def trace_rays(self, proto: dict, rays, stream=None, out=None):
        """rays: float64 device tensor [n, 4] = (alpha, beta, a, cos i)."""
        n = int(rays.shape[0])
        planes = image_planes(proto)
        rec, img = out if out is not None else self.alloc(n, planes * n)
        st = stream if stream is not None else self.torch.cuda.current_stream(self.device)
        odx_trace_rays(self.ctx, proto, rays.data_ptr() if n else None, n, rec.data_ptr(),
                       img.data_ptr(), st.cuda_stream)
        return rec, img

    def stats(self, reset=False, stream=None):
        st = stream if stream is not None else self.torch.cuda.current_stream(self.device)
        return odx_get_stats(self.ctx, st.cuda_stream, reset)

    def set_launch(self, **kw):
        cur = odx_get_launch(self.ctx)
        cur.update(kw)
        odx_set_launch(self.ctx, **cur)
