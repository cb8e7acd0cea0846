"""Thin ctypes binding of the C ABI in include/rflbm.h (argument marshalling only).

Every function has the C name and forwards to librflbm.so; all work runs in the CUDA
library. Arrays are numpy arrays (host memory, on_device = 0) or objects exposing
`data_ptr()` (torch CUDA tensors, on_device = 1). A negative status raises RflbmError
with the library's message. There is no fallback: if the library cannot be loaded the
import of this module fails.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

_LIB_PATH = os.path.join(os.path.dirname(os.path.abspath(__file__)), "_lib", "librflbm.so")

RFLBM_OK = 0
RFLBM_EINVAL = -1
RFLBM_ENOMEM = -2
RFLBM_ECUDA = -3
RFLBM_EUNSTABLE = -4
RFLBM_ETIMEOUT = -5
RFLBM_ESTATE = -6
RFLBM_MODEL_REG = 0
RFLBM_MODEL_BGK = 1
RFLBM_STORE_F32 = 0
RFLBM_STORE_F16 = 1
RFLBM_STORE_BF16 = 2
RFLBM_PHI_LOCAL_RHO = 0
RFLBM_PHI_RHO0 = 1
RFLBM_KERNEL_AUTO = 0
RFLBM_KERNEL_GATHER = 1
RFLBM_KERNEL_TMA = 2
RFLBM_PATTERN_PINGPONG = 0
RFLBM_PATTERN_AA = 1
FIELDS = ("rho", "jx", "jy", "jz", "pxx", "pyy", "pzz", "pxy", "pxz", "pyz")


class RflbmError(RuntimeError):
    def __init__(self, status, message):
        super().__init__(f"rflbm error {status}: {message}")
        self.status = status


class rflbm_config_t(C.Structure):
    _fields_ = [
        ("nx", C.c_int), ("ny", C.c_int), ("nz", C.c_int),
        ("tau", C.c_double), ("kT", C.c_double), ("rho0", C.c_double),
        ("seed", C.c_uint64), ("omega_g", C.c_double),
        ("model", C.c_int), ("storage", C.c_int), ("phi_rho", C.c_int),
        ("replica", C.c_uint32), ("stream", C.c_void_p),
        ("buffers", C.c_void_p * 2), ("device", C.c_int), ("kernel", C.c_int),
        ("pattern", C.c_int), ("z0", C.c_int), ("nz_global", C.c_int),
    ]


class rflbm_face_t(C.Structure):
    _fields_ = [("run", C.c_void_p * 3), ("plane_pitch", C.c_int64), ("row_bytes", C.c_int64)]


class rflbm_replica_t(C.Structure):
    _fields_ = [("nx", C.c_int), ("ny", C.c_int), ("nz", C.c_int),
                ("tau", C.c_double), ("kT", C.c_double), ("seed", C.c_uint64)]


class rflbm_stats_t(C.Structure):
    _fields_ = [
        ("step", C.c_int64), ("mass", C.c_double), ("momentum", C.c_double * 3),
        ("max_speed", C.c_double), ("nonfinite", C.c_int64),
    ]


def _load():
    if not os.path.exists(_LIB_PATH):
        raise ImportError(
            f"{_LIB_PATH} is missing: build it with `python -m paper_2507_08820_gb300.build`")
    return C.CDLL(_LIB_PATH)


lib = _load()
_H = C.c_void_p
_P = C.c_void_p
_sig = {
    "rflbm_config_default": (None, [C.POINTER(rflbm_config_t)]),
    "rflbm_config_size": (C.c_int64, []),
    "rflbm_buffer_bytes": (C.c_int64, [C.POINTER(rflbm_config_t)]),
    "rflbm_create": (_H, [C.c_int, C.c_int, C.c_int, C.c_double, C.c_double, C.c_double, C.c_uint64]),
    "rflbm_create_ex": (_H, [C.POINTER(rflbm_config_t)]),
    "rflbm_destroy": (None, [_H]),
    "rflbm_last_error": (C.c_char_p, []),
    "rflbm_init_rest": (C.c_int, [_H]),
    "rflbm_init_field": (C.c_int, [_H, _P, _P, C.c_int]),
    "rflbm_init_thermal": (C.c_int, [_H]),
    "rflbm_step": (C.c_int, [_H, C.c_int64]),
    "rflbm_moments": (C.c_int, [_H, _P, _P, _P, C.c_int]),
    "rflbm_stats": (C.c_int, [_H, C.POINTER(rflbm_stats_t)]),
    "rflbm_get_populations": (C.c_int, [_H, _P, C.c_int]),
    "rflbm_get_populations_f32": (C.c_int, [_H, _P, C.c_int]),
    "rflbm_set_populations": (C.c_int, [_H, _P, C.c_int]),
    "rflbm_set_populations_f32": (C.c_int, [_H, _P, C.c_int]),
    "rflbm_get_sites": (C.c_int, [_H, _P, C.c_int64, _P]),
    "rflbm_state_bytes": (C.c_int64, [_H]),
    "rflbm_save_state": (C.c_int, [_H, _P, C.c_int]),
    "rflbm_load_state": (C.c_int, [_H, _P, C.c_int]),
    "rflbm_get_step": (C.c_int64, [_H]),
    "rflbm_set_step": (C.c_int, [_H, C.c_int64]),
    "rflbm_set_stream": (C.c_int, [_H, _P]),
    "rflbm_synchronize": (C.c_int, [_H]),
    "rflbm_get_dims": (C.c_int, [_H, C.POINTER(C.c_int), C.POINTER(C.c_int), C.POINTER(C.c_int)]),
    "rflbm_launches_per_step": (C.c_int, [_H]),
    "rflbm_step_path": (C.c_int, [_H, C.POINTER(C.c_int)]),
    "rflbm_step_sites_per_thread": (C.c_int, [_H]),
    "rflbm_philox4x32_10": (C.c_int, [_P, C.c_uint32, C.c_uint32, _P, C.c_int64]),
    "rflbm_site_normals": (C.c_int, [C.c_uint64, C.c_int64, C.c_uint32, _P, C.c_int64, _P]),
    "rflbm_stats_f32_noalloc": (C.c_int, [_P, C.c_int64, _P, C.POINTER(rflbm_stats_t)]),
    "rflbm_mode_sums": (C.c_int, [_H, _P, _P]),
    "rflbm_batch_create": (_H, [_P, C.c_int, C.c_double, C.c_int, C.c_int]),
    "rflbm_batch_destroy": (None, [_H]),
    "rflbm_batch_tuning": (C.c_int, [_H, C.POINTER(C.c_int), C.POINTER(C.c_int), C.POINTER(C.c_int64)]),
    "rflbm_batch_launches_per_step": (C.c_int, [_H]),
    "rflbm_batch_replica_tiling": (C.c_int, [_H, C.c_int, C.POINTER(C.c_int), C.POINTER(C.c_int)]),
    "rflbm_batch_replica_dims": (C.c_int, [_H, C.c_int, C.POINTER(C.c_int), C.POINTER(C.c_int),
                                           C.POINTER(C.c_int)]),
    "rflbm_batch_init_rest": (C.c_int, [_H]),
    "rflbm_batch_run": (C.c_int, [_H, C.c_int64]),
    "rflbm_batch_prepare": (C.c_int, [_H, C.c_int64]),
    "rflbm_batch_synchronize": (C.c_int, [_H]),
    "rflbm_batch_get_populations": (C.c_int, [_H, C.c_int, _P]),
    "rflbm_batch_stats": (C.c_int, [_H, C.c_int, C.POINTER(rflbm_stats_t)]),
    "rflbm_structure_factor": (C.c_int, [_H, C.c_int, C.c_int, _P, _P]),
    "rflbm_shell_count": (C.c_int, [_H]),
    "rflbm_testing_expect_extra_bytes": (C.c_int, [_H, C.c_uint32]),
    "rflbm_testing_slab_copy_pitch_limit": (C.c_int, [C.c_int64]),
    "rflbm_testing_backtransform": (C.c_int, [C.c_int, _P, C.c_int64, _P]),
    "rflbm_testing_backtransform_time": (C.c_int, [C.c_int, C.c_int64, C.c_int, C.POINTER(C.c_float)]),
    "rflbm_testing_forward": (C.c_int, [C.c_int, _P, C.c_int64, _P]),
    "rflbm_testing_forward_time": (C.c_int, [C.c_int, C.c_int64, C.c_int, C.POINTER(C.c_float)]),
    "rflbm_testing_noise_time": (C.c_int, [C.c_int64, C.POINTER(C.c_float)]),
    "rflbm_slab_faces": (C.c_int, [_H] + [C.POINTER(rflbm_face_t)] * 4),
    "rflbm_slab_faces_ready": (C.c_int, [_H, _P]),
    "rflbm_slab_exchange_done": (C.c_int, [_H, _P]),
    "rflbm_slab_exchange": (C.c_int, [_P, C.c_int]),
}
for _name, (_res, _args) in _sig.items():
    _fn = getattr(lib, _name)
    _fn.restype = _res
    _fn.argtypes = _args


def _check(status):
    if status < 0:
        raise RflbmError(status, lib.rflbm_last_error().decode())
    return status


_TORCH_DTYPE = {np.dtype(np.float32): "torch.float32", np.dtype(np.float64): "torch.float64"}


def _ptr(a, dtype=None, count=None):
    """(pointer, on_device) of a numpy array or a CUDA tensor; None -> (None, 0).

    dtype: the element type the C function reads or writes (numpy dtype); count: the
    number of elements it touches. Both are checked before any pointer reaches the
    library, so a wrong element type or a short buffer raises ValueError here instead of
    letting a kernel run past the end of the allocation."""
    if a is None:
        return None, 0
    if hasattr(a, "data_ptr"):
        if not a.is_contiguous():
            raise ValueError("tensor must be contiguous")
        if dtype is not None and str(a.dtype) != _TORCH_DTYPE[np.dtype(dtype)]:
            raise ValueError(f"expected a tensor of {_TORCH_DTYPE[np.dtype(dtype)]}, got {a.dtype}")
        if count is not None and a.numel() < count:
            raise ValueError(f"tensor holds {a.numel()} elements, the call needs {count}")
        return a.data_ptr(), 1 if a.is_cuda else 0
    if not isinstance(a, np.ndarray) or not a.flags.c_contiguous:
        raise ValueError("expected a C-contiguous numpy array or a torch tensor")
    if dtype is not None and a.dtype != dtype:
        raise ValueError(f"expected dtype {np.dtype(dtype)}, got {a.dtype}")
    if count is not None and a.size < count:
        raise ValueError(f"array holds {a.size} elements, the call needs {count}")
    return a.ctypes.data, 0


def _sites(h):
    nx, ny, nz = rflbm_get_dims(h)
    return nx * ny * nz


def _same_side(*pairs):
    sides = {d for p, d in pairs if p is not None}
    if len(sides) > 1:
        raise ValueError("all arrays of one call must be on the same side (host or device)")
    return sides.pop() if sides else 0


# ------------------------------------------------------------------ C ABI, same names
def rflbm_config_default():
    cfg = rflbm_config_t()
    lib.rflbm_config_default(C.byref(cfg))
    return cfg


def rflbm_config_size():
    return lib.rflbm_config_size()


def rflbm_buffer_bytes(cfg):
    return _check(lib.rflbm_buffer_bytes(C.byref(cfg)))


def rflbm_create(nx, ny, nz, tau, kT, rho0, seed):
    h = lib.rflbm_create(nx, ny, nz, tau, kT, rho0, seed)
    if not h:
        raise RflbmError(-1, lib.rflbm_last_error().decode())
    return h


def rflbm_create_ex(cfg):
    h = lib.rflbm_create_ex(C.byref(cfg))
    if not h:
        raise RflbmError(-1, lib.rflbm_last_error().decode())
    return h


def rflbm_destroy(h):
    lib.rflbm_destroy(h)


def rflbm_last_error():
    return lib.rflbm_last_error().decode()


def rflbm_init_rest(h):
    return _check(lib.rflbm_init_rest(h))


def rflbm_init_thermal(h):
    return _check(lib.rflbm_init_thermal(h))


def rflbm_init_field(h, rho=None, u=None):
    n = _sites(h)
    pr, pu = _ptr(rho, np.float64, n), _ptr(u, np.float64, 3 * n)
    return _check(lib.rflbm_init_field(h, pr[0], pu[0], _same_side(pr, pu)))


def rflbm_step(h, n=1):
    return _check(lib.rflbm_step(h, int(n)))


def rflbm_moments(h, rho=None, u=None, pi=None):
    n = _sites(h)
    ps = [_ptr(a, np.float64, k * n) for a, k in ((rho, 1), (u, 3), (pi, 6))]
    return _check(lib.rflbm_moments(h, ps[0][0], ps[1][0], ps[2][0], _same_side(*ps)))


def rflbm_stats(h):
    st = rflbm_stats_t()
    status = lib.rflbm_stats(h, C.byref(st))
    if status < 0 and status != RFLBM_EUNSTABLE:
        _check(status)
    return st, status


def rflbm_get_populations(h, f):
    p, d = _ptr(f, np.float64, 27 * _sites(h))
    return _check(lib.rflbm_get_populations(h, p, d))


def rflbm_get_populations_f32(h, f):
    p, d = _ptr(f, np.float32, 27 * _sites(h))
    return _check(lib.rflbm_get_populations_f32(h, p, d))


def rflbm_set_populations(h, f):
    p, d = _ptr(f, np.float64, 27 * _sites(h))
    return _check(lib.rflbm_set_populations(h, p, d))


def rflbm_set_populations_f32(h, f):
    p, d = _ptr(f, np.float32, 27 * _sites(h))
    return _check(lib.rflbm_set_populations_f32(h, p, d))


def rflbm_get_sites(h, sites, out):
    sites = np.ascontiguousarray(sites, dtype=np.int64)
    p, _ = _ptr(out, np.float64, 27 * sites.size)
    return _check(lib.rflbm_get_sites(h, sites.ctypes.data, sites.size, p))


def rflbm_state_bytes(h):
    return _check(lib.rflbm_state_bytes(h))


def _image_bytes(image):
    return image.numel() * image.element_size() if hasattr(image, "data_ptr") else image.nbytes


def rflbm_save_state(h, image):
    if _image_bytes(image) < rflbm_state_bytes(h):
        raise ValueError("the image buffer is smaller than rflbm_state_bytes")
    p, d = _ptr(image)
    return _check(lib.rflbm_save_state(h, p, d))


def rflbm_load_state(h, image):
    if _image_bytes(image) < rflbm_state_bytes(h):
        raise ValueError("the image buffer is smaller than rflbm_state_bytes")
    p, d = _ptr(image)
    return _check(lib.rflbm_load_state(h, p, d))


def rflbm_get_step(h):
    return _check(lib.rflbm_get_step(h))


def rflbm_set_step(h, step):
    return _check(lib.rflbm_set_step(h, int(step)))


def rflbm_set_stream(h, stream):
    return _check(lib.rflbm_set_stream(h, stream))


def rflbm_synchronize(h):
    return _check(lib.rflbm_synchronize(h))


def rflbm_get_dims(h):
    nx, ny, nz = C.c_int(), C.c_int(), C.c_int()
    _check(lib.rflbm_get_dims(h, C.byref(nx), C.byref(ny), C.byref(nz)))
    return nx.value, ny.value, nz.value


def rflbm_launches_per_step(h):
    return _check(lib.rflbm_launches_per_step(h))


def rflbm_testing_expect_extra_bytes(h, nbytes):
    """Testing hook (include/rflbm_testing.h): later TMA steps wait for bytes that never
    arrive, so their bounded waits run out and the next synchronising call raises
    RFLBM_ETIMEOUT; 0 restores normal operation."""
    return _check(lib.rflbm_testing_expect_extra_bytes(h, int(nbytes)))


def rflbm_testing_slab_copy_pitch_limit(nbytes):
    """Testing hook (include/rflbm_testing.h): faces whose plane pitch exceeds nbytes move one
    plane row per copy in rflbm_slab_exchange; 0 restores the default."""
    return _check(lib.rflbm_testing_slab_copy_pitch_limit(int(nbytes)))


def rflbm_testing_backtransform(method, m):
    """Testing (include/rflbm_testing.h): the back transform of Eq. 11 alone; m: (27, n)
    float32 scaled moments in exponent order, n a multiple of 128. Returns (27, n) populations.
    method 0: float32 FMAs as in the step kernels, 1: tcgen05 MMA with split-bfloat16 moments."""
    m = np.ascontiguousarray(m, dtype=np.float32)
    f = np.empty_like(m)
    _check(lib.rflbm_testing_backtransform(int(method), m.ctypes.data, m.shape[1], f.ctypes.data))
    return f


def rflbm_testing_backtransform_time(method, tiles, reps):
    """Testing: milliseconds of one launch over `tiles` tiles of 128 sites, `reps` synthetic
    transforms per site."""
    ms = C.c_float()
    _check(lib.rflbm_testing_backtransform_time(int(method), int(tiles), int(reps), C.byref(ms)))
    return ms.value


def rflbm_testing_forward(method, f):
    """Testing (include/rflbm_testing.h): the forward projection alone; f: (27, n) float32
    populations, n a multiple of 128. Returns the (10, n) raw moments of order <= 2.
    method 0: float32 FMAs as in the step kernels, 1: tcgen05 MMA with float16 operands."""
    f = np.ascontiguousarray(f, dtype=np.float32)
    m = np.empty((10, f.shape[1]), dtype=np.float32)
    _check(lib.rflbm_testing_forward(int(method), f.ctypes.data, f.shape[1], m.ctypes.data))
    return m


def rflbm_testing_forward_time(method, tiles, reps):
    """Testing: milliseconds of one launch over `tiles` tiles of 128 sites, `reps` synthetic
    projections per site."""
    ms = C.c_float()
    _check(lib.rflbm_testing_forward_time(int(method), int(tiles), int(reps), C.byref(ms)))
    return ms.value


def rflbm_testing_noise_time(nsites):
    """Testing: milliseconds of one launch drawing the 24 normals of nsites sites."""
    ms = C.c_float()
    _check(lib.rflbm_testing_noise_time(int(nsites), C.byref(ms)))
    return ms.value


def rflbm_step_path(h):
    """(kernel, row-segment width) of the step kernel the handle runs."""
    w = C.c_int()
    k = _check(lib.rflbm_step_path(h, C.byref(w)))
    return k, w.value


def rflbm_step_sites_per_thread(h):
    """Sites one thread of the step kernel updates (2: the two-site TMA form)."""
    return _check(lib.rflbm_step_sites_per_thread(h))


def rflbm_mode_sums(h):
    """(sum, sumsq): 27 doubles each, see include/rflbm.h."""
    s1, s2 = np.zeros(27), np.zeros(27)
    _check(lib.rflbm_mode_sums(h, s1.ctypes.data, s2.ctypes.data))
    return s1, s2


def rflbm_shell_count(h):
    return _check(lib.rflbm_shell_count(h))


def rflbm_structure_factor(h, field, nshell=None):
    """(s_sum, count) per shell for field (index or name in FIELDS)."""
    if isinstance(field, str):
        field = FIELDS.index(field)
    nshell = rflbm_shell_count(h) if nshell is None else nshell
    s, c = np.zeros(nshell), np.zeros(nshell)
    _check(lib.rflbm_structure_factor(h, int(field), int(nshell), s.ctypes.data, c.ctypes.data))
    return s, c


def rflbm_philox4x32_10(ctr, k0, k1):
    ctr = np.ascontiguousarray(ctr, dtype=np.uint32).reshape(-1, 4)
    out = np.empty_like(ctr)
    _check(lib.rflbm_philox4x32_10(ctr.ctypes.data, k0, k1, out.ctypes.data, ctr.shape[0]))
    return out


def rflbm_site_normals(seed, step, replica, sites):
    sites = np.ascontiguousarray(sites, dtype=np.uint32)
    out = np.empty((sites.size, 24), dtype=np.float32)
    _check(lib.rflbm_site_normals(seed, step, replica, sites.ctypes.data, sites.size,
                                  out.ctypes.data))
    return out


def rflbm_slab_faces(h):
    """(send_up, send_down, recv_below, recv_above) faces of the pending exchange, each an
    rflbm_face_t (three runs of three plane rows, see include/rflbm.h)."""
    f = [rflbm_face_t() for _ in range(4)]
    _check(lib.rflbm_slab_faces(h, *[C.byref(x) for x in f]))
    return tuple(f)


def rflbm_slab_faces_ready(h, stream):
    return _check(lib.rflbm_slab_faces_ready(h, stream))


def rflbm_slab_exchange_done(h, stream):
    return _check(lib.rflbm_slab_exchange_done(h, stream))


def rflbm_slab_exchange(slabs):
    """The face exchange of slabs of one box on one device, in z order."""
    arr = (C.c_void_p * len(slabs))(*slabs)
    return _check(lib.rflbm_slab_exchange(C.cast(arr, C.c_void_p), len(slabs)))


RFLBM_STATS_NOALLOC_MAX_SITES = 134217728


def rflbm_stats_f32_noalloc(f, n_sites, stream=None):
    """Diagnostics of caller-owned float32 populations (a CUDA tensor of 27 * n_sites
    values, public layout) with the library's fixed scratch area: nothing is allocated.
    Returns (stats, status) like rflbm_stats."""
    n_sites = int(n_sites)
    if n_sites > RFLBM_STATS_NOALLOC_MAX_SITES:  # the library rejects it before any launch
        p, d = _ptr(f, np.float32)
    else:
        p, d = _ptr(f, np.float32, 27 * max(n_sites, 0))
    if not d:
        raise ValueError("populations must be in device memory")
    st = rflbm_stats_t()
    status = lib.rflbm_stats_f32_noalloc(p, n_sites, stream, C.byref(st))
    if status < 0 and status != RFLBM_EUNSTABLE:
        _check(status)
    return st, status


def rflbm_batch_create(replicas, rho0=1.0, storage=RFLBM_STORE_F32, tile=0):
    """replicas: list of dicts with nx, ny, nz, tau, kT, seed."""
    arr = (rflbm_replica_t * len(replicas))()
    for a, r in zip(arr, replicas):
        a.nx, a.ny, a.nz = r["nx"], r["ny"], r["nz"]
        a.tau, a.kT, a.seed = r["tau"], r["kT"], r["seed"]
    h = lib.rflbm_batch_create(C.cast(arr, C.c_void_p), len(replicas), rho0, storage, tile)
    if not h:
        raise RflbmError(-1, lib.rflbm_last_error().decode())
    return h


def rflbm_batch_destroy(b):
    lib.rflbm_batch_destroy(b)


def rflbm_batch_launches_per_step(b):
    return _check(lib.rflbm_batch_launches_per_step(b))


def rflbm_batch_tuning(b):
    t, c, n = C.c_int(), C.c_int(), C.c_int64()
    _check(lib.rflbm_batch_tuning(b, C.byref(t), C.byref(c), C.byref(n)))
    return t.value, c.value, n.value


def rflbm_batch_replica_tiling(b, r):
    """(tile size, rows per tile; 0 for tiles of consecutive sites) of replica r."""
    t, rows = C.c_int(), C.c_int()
    _check(lib.rflbm_batch_replica_tiling(b, int(r), C.byref(t), C.byref(rows)))
    return t.value, rows.value


def rflbm_batch_replica_dims(b, r):
    nx, ny, nz = C.c_int(), C.c_int(), C.c_int()
    _check(lib.rflbm_batch_replica_dims(b, int(r), C.byref(nx), C.byref(ny), C.byref(nz)))
    return nx.value, ny.value, nz.value


def _batch_sites(b, r):
    nx, ny, nz = rflbm_batch_replica_dims(b, r)
    return nx * ny * nz


def rflbm_batch_init_rest(b):
    return _check(lib.rflbm_batch_init_rest(b))


def rflbm_batch_run(b, n):
    return _check(lib.rflbm_batch_run(b, int(n)))


def rflbm_batch_prepare(b, n):
    """Builds the CUDA graph of an n-step run without running it."""
    return _check(lib.rflbm_batch_prepare(b, int(n)))


def rflbm_batch_synchronize(b):
    return _check(lib.rflbm_batch_synchronize(b))


def rflbm_batch_get_populations(b, r, f):
    p, _ = _ptr(f, np.float64, 27 * _batch_sites(b, r))
    return _check(lib.rflbm_batch_get_populations(b, int(r), p))


def rflbm_batch_stats(b, r):
    st = rflbm_stats_t()
    status = lib.rflbm_batch_stats(b, int(r), C.byref(st))
    if status < 0 and status != RFLBM_EUNSTABLE:
        _check(status)
    return st, status


# ------------------------------------------------------------------ convenience
class Box:
    """One periodic box (owns a handle), or with nz_global > 0 the z-slab of rows
    z0 .. z0 + nz - 1 of a box of nz_global rows. Population buffers are allocated by
    PyTorch when `torch_buffers` is true, else by the library."""

    def __init__(self, nx, ny, nz, tau, kT=0.0, rho0=1.0, seed=1, omega_g=1.0,
                 model=RFLBM_MODEL_REG, phi_rho=RFLBM_PHI_LOCAL_RHO, replica=0,
                 stream=None, torch_buffers=False, device=-1, kernel=RFLBM_KERNEL_AUTO,
                 storage=RFLBM_STORE_F32, pattern=RFLBM_PATTERN_PINGPONG, z0=0, nz_global=0):
        cfg = rflbm_config_default()
        cfg.nx, cfg.ny, cfg.nz = nx, ny, nz
        cfg.tau, cfg.kT, cfg.rho0, cfg.seed = tau, kT, rho0, seed
        cfg.omega_g, cfg.model, cfg.phi_rho, cfg.replica = omega_g, model, phi_rho, replica
        cfg.device = device
        cfg.kernel = kernel
        cfg.storage = storage
        cfg.pattern = pattern
        cfg.z0, cfg.nz_global = z0, nz_global
        if stream is not None:
            cfg.stream = stream
        self._buffers = None
        if torch_buffers:
            import torch
            nbytes = rflbm_buffer_bytes(cfg)
            dev = torch.device("cuda", device if device >= 0 else torch.cuda.current_device())
            nbuf = 1 if pattern == RFLBM_PATTERN_AA else 2
            self._buffers = [torch.empty(nbytes, dtype=torch.uint8, device=dev)
                             for _ in range(nbuf)]
            for b, t in enumerate(self._buffers):
                cfg.buffers[b] = t.data_ptr()
        self.cfg = cfg
        self.shape = (nx, ny, nz)
        self.n = nx * ny * nz
        self.h = rflbm_create_ex(cfg)

    def close(self):
        if self.h:
            rflbm_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def populations(self):
        f = np.empty((27, self.n))
        rflbm_get_populations(self.h, f)
        return f

    def macroscopic(self):
        rho, u, pi = np.empty(self.n), np.empty((3, self.n)), np.empty((6, self.n))
        rflbm_moments(self.h, rho, u, pi)
        return rho, u, pi
