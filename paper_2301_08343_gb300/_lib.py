"""ctypes declarations of the C ABI in include/tacchi.h (argument marshalling
only; every step of the computation runs in libtacchi.so's CUDA kernels)."""
from __future__ import annotations

import ctypes as C
import os
import threading

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libtacchi.so")

OK = 0
STATUS = {0: "OK", -1: "INVALID_ARG", -2: "OOM", -3: "CUDA", -4: "NUMERICAL",
          -5: "OUT_OF_GRID", -6: "TIMEOUT", -7: "STATE", -8: "CFL"}


class TacchiError(RuntimeError):
    def __init__(self, status: int, what: str = ""):
        self.status = status
        self.name = STATUS.get(status, str(status))
        super().__init__(f"{what}: TACCHI_ERR_{self.name} ({status})" if what else self.name)


class ElastomerDesc(C.Structure):
    _fields_ = [("extent_m", C.c_double * 3), ("dx_m", C.c_double), ("E_pa", C.c_double),
                ("nu", C.c_double), ("density", C.c_double), ("seed", C.c_uint64),
                ("jitter", C.c_int), ("pad_side", C.c_int), ("pad_bottom", C.c_int),
                ("pad_top", C.c_int), ("gravity", C.c_double * 3), ("free_base", C.c_int),
                ("block", C.c_int * 3), ("threads_per_cell", C.c_int), ("contact_mode", C.c_int)]


class IndenterDesc(C.Structure):
    _fields_ = [("kind", C.c_int), ("params", C.c_double * 8), ("hm_w", C.c_int),
                ("hm_h", C.c_int), ("hm_pixel_m", C.c_double), ("hm", C.POINTER(C.c_float))]


class RenderParams(C.Structure):
    _fields_ = [("n_lights", C.c_int), ("dir", (C.c_float * 3) * 8),
                ("diffuse", (C.c_float * 3) * 8), ("specular", (C.c_float * 3) * 8),
                ("ambient", C.c_float * 3), ("ka", C.c_float), ("kd", C.c_float),
                ("ks", C.c_float), ("alpha", C.c_float)]


class Info(C.Structure):
    _fields_ = [("n_particles", C.c_int64), ("n_surface", C.c_int64), ("grid", C.c_int * 3),
                ("n_nodes", C.c_int64), ("origin_m", C.c_double * 3), ("dx_m", C.c_double),
                ("z_top_m", C.c_double), ("block", C.c_int * 3), ("n_blocks", C.c_int64),
                ("device_bytes", C.c_size_t), ("threads_per_cell", C.c_int), ("pipelined", C.c_int)]


class Profile(C.Structure):
    _fields_ = [("grid_ms", C.c_double), ("fused_ms", C.c_double), ("edge_ms", C.c_double),
                ("sort_ms", C.c_double), ("grid_launches", C.c_int64),
                ("fused_launches", C.c_int64), ("edge_launches", C.c_int64),
                ("sort_launches", C.c_int64), ("sort_runs", C.c_int64)]


_lock = threading.Lock()
_lib = None

# name -> (restype, argtypes)
_vp, _fp, _dp, _u8p = C.c_void_p, C.POINTER(C.c_float), C.POINTER(C.c_double), C.POINTER(C.c_uint8)
SIGNATURES = {
    "tacchi_create": (C.c_int, [C.POINTER(ElastomerDesc), _vp, C.POINTER(_vp)]),
    "tacchi_destroy": (None, [_vp]),
    "tacchi_info": (C.c_int, [_vp, C.POINTER(Info)]),
    "tacchi_set_indenter": (C.c_int, [_vp, C.POINTER(IndenterDesc), _dp, _dp]),
    "tacchi_get_indenter_pose": (C.c_int, [_vp, _dp]),
    "tacchi_step": (C.c_int, [_vp, C.c_int, C.c_double]),
    "tacchi_heightmap": (C.c_int, [_vp, C.c_int, C.c_int, _dp, C.c_int, _vp]),
    "tacchi_render": (C.c_int, [_vp, C.POINTER(RenderParams), C.c_int, C.c_int, _dp, C.c_int, _vp, _vp]),
    "tacchi_shade": (C.c_int, [C.POINTER(RenderParams), _vp, C.c_int, C.c_int, C.c_double,
                               C.c_double, C.c_double, _vp, _vp]),
    "tacchi_get_state": (C.c_int, [_vp, _vp, _vp, _vp, _vp, _vp]),
    "tacchi_set_state": (C.c_int, [_vp, _vp, _vp, _vp, _vp]),
    "tacchi_get_grid": (C.c_int, [_vp, _vp]),
    "tacchi_sync": (C.c_int, [_vp]),
    "tacchi_set_profiling": (C.c_int, [_vp, C.c_int]),
    "tacchi_get_profile": (C.c_int, [_vp, C.POINTER(Profile), C.c_int]),
    "tacchi_clear_error": (C.c_int, [_vp]),
    "tacchi_init_lattice": (C.c_int, [C.c_int] * 5 + [C.c_uint64, C.c_int, _fp, _u8p]),
    "tacchi_status_string": (C.c_char_p, [C.c_int]),
    "tacchi_version": (C.c_int, []),
    "tacchi_measure_fp32_peak": (C.c_int, [_dp, C.POINTER(C.c_int), C.POINTER(C.c_int)]),
}
EXTRA_SIGNATURES = {
    "tacchi_batch_create": (C.c_int, [C.c_int, C.POINTER(ElastomerDesc), _vp, C.POINTER(_vp)]),
    "tacchi_batch_size": (C.c_int, [_vp, C.POINTER(C.c_int)]),
    "tacchi_batch_info": (C.c_int, [_vp, C.c_int, C.POINTER(Info)]),
    "tacchi_batch_set_indenter": (C.c_int, [_vp, C.c_int, C.POINTER(IndenterDesc), _dp, _dp]),
    "tacchi_batch_get_indenter_pose": (C.c_int, [_vp, C.c_int, _dp]),
    "tacchi_batch_heightmap": (C.c_int, [_vp, C.c_int, C.c_int, C.c_int, _dp, C.c_int, _vp]),
    "tacchi_batch_render": (C.c_int, [_vp, C.c_int, C.POINTER(RenderParams), C.c_int, C.c_int, _dp,
                                      C.c_int, _vp, _vp]),
    "tacchi_batch_get_state": (C.c_int, [_vp, C.c_int, _vp, _vp, _vp, _vp, _vp]),
    "tacchi_batch_set_state": (C.c_int, [_vp, C.c_int, _vp, _vp, _vp, _vp]),
    "tacchi_set_block": (C.c_int, [_vp, C.c_int, C.c_int, C.c_int]),
    "tacchi_set_transfer": (C.c_int, [_vp, C.c_int, C.c_int, C.c_int, C.c_int]),
    "tacchi_set_launch": (C.c_int, [_vp, C.c_int]),
    "tacchi_set_barrier_wait": (C.c_int, [_vp, C.c_int64, C.c_int]),
    "tacchi_set_pipeline": (C.c_int, [_vp, C.c_int]),
    "tacchi_batch_reset": (C.c_int, [_vp]),
    "tacchi_batch_displacement_map": (C.c_int, [_vp, C.c_int, C.c_int, C.c_int, _dp, _vp]),
    "tacchi_batch_markers": (C.c_int, [_vp, C.c_int, C.c_int, _vp, _vp]),
    "tacchi_batch_set_indenter_particles": (C.c_int, [_vp, C.c_int, C.c_int, _fp, C.c_double]),
    "tacchi_set_indenter_particles": (C.c_int, [_vp, C.c_int, _fp, C.c_double]),
    "tacchi_batch_penetration_map": (C.c_int, [_vp, C.c_int, C.c_int, C.c_int, _dp, _vp]),
    "tacchi_batch_render_smoothed": (C.c_int, [_vp, C.c_int, C.POINTER(RenderParams), C.c_int, C.c_int, _dp,
                                               C.c_double, _vp, _vp]),
    "tacchi_render_smoothed": (C.c_int, [_vp, C.POINTER(RenderParams), C.c_int, C.c_int, _dp, C.c_double, _vp,
                                         _vp]),
    "tacchi_autotune": (C.c_int, [_vp, C.c_int, C.c_double, C.POINTER(C.c_int), _dp]),
    "tacchi_nn_create": (C.c_int, [C.c_int, C.POINTER(C.c_int), C.c_int, C.c_int, C.c_int, C.c_int, C.c_int,
                                   C.c_uint64, _vp, C.POINTER(_vp)]),
    "tacchi_nn_destroy": (None, [_vp]),
    "tacchi_nn_num_params": (C.c_int, [_vp, C.POINTER(C.c_int64)]),
    "tacchi_nn_get_params": (C.c_int, [_vp, C.c_int, _fp]),
    "tacchi_nn_set_params": (C.c_int, [_vp, _fp]),
    "tacchi_nn_forward": (C.c_int, [_vp, C.c_int, _vp, _vp]),
    "tacchi_nn_gradients": (C.c_int, [_vp, C.c_int, _vp, _vp, C.POINTER(C.c_float)]),
    "tacchi_nn_train_step": (C.c_int, [_vp, C.c_int, _vp, _vp, C.c_float, C.POINTER(C.c_float)]),
    "tacchi_heightmap_static": (C.c_int, [_vp, C.c_int64, _vp, _vp, C.c_int, C.c_double, _dp,
                                          C.c_double, C.c_int, C.c_int, _dp, C.c_int, _vp, _vp]),
}


def lib():
    """Load libtacchi.so (fails loudly if it has not been built)."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(LIB_PATH):
                raise RuntimeError(f"{LIB_PATH} is missing: build it with "
                                   "paper_2301_08343_gb300.build.build() (needs nvcc)")
            L = C.CDLL(LIB_PATH)
            for name, (res, args) in {**SIGNATURES, **EXTRA_SIGNATURES}.items():
                fn = getattr(L, name)
                fn.restype = res
                fn.argtypes = args
            _lib = L
    return _lib


def check(status: int, what: str = "") -> None:
    if status != OK:
        raise TacchiError(status, what)


def ptr(t):
    """Device (or host) address of a tensor/ndarray, or None."""
    if t is None:
        return None
    if hasattr(t, "data_ptr"):
        return C.c_void_p(t.data_ptr())
    return C.c_void_p(t.ctypes.data)
