"""Python binding of the C ABI in include/lbmd.h (argument marshalling only).

Every function here has the name of the C entry point it calls and does nothing
but convert arguments (numpy arrays, Python scalars, CUDA stream handles) and
turn negative return codes into :class:`LbmdError`.  All computation runs in
``liblbmd.so`` (hand-written sm_103a CUDA).  There is no fallback: if the
library is missing, importing the binding fails loudly.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "liblbmd.so")

LBMD_OK = 0
LBMD_E_INVALID_ARG = -1
LBMD_E_NOMEM = -2
LBMD_E_CUDA = -3
LBMD_E_NEGATIVE_DENSITY = -4
LBMD_E_NONFINITE = -5
LBMD_E_TIMEOUT = -6
LBMD_E_UNIMPLEMENTED = -7
LBMD_E_BOND_BROKEN = -8
LBMD_E_STATE = -9
LBMD_E_PARTICLE_TOO_FAST = -10
LBMD_E_DRIFT = -11

LBMD_STORAGE_FP32 = 0
LBMD_STORAGE_FP16_SHIFTED = 1
LBMD_STORAGE_BF16_SHIFTED = 2
LBMD_BOND_FENE = 2
LBMD_BOND_HARMONIC = 3
LBMD_WARN_GAMMA_DT = 1 << 0
LBMD_WARN_VISCOSITY = 1 << 1
LBMD_WARN_BOLTZMANN = 1 << 2
LBMD_WARN_ASYMMETRIC_G = 1 << 3
LBMD_MAX_TYPES = 8
LBMD_COLLISION_BGK = 0
LBMD_COLLISION_MRT = 1
LBMD_SLOT_EMPTY = 0
LBMD_SLOT_ACTIVE = 1
LBMD_SLOT_DONE = 2
LBMD_SLOT_FAILED = 3

# every symbol include/lbmd.h declares
EXPORTS = ("lbmd_create", "lbmd_destroy", "lbmd_set_types", "lbmd_set_debye_hueckel", "lbmd_init_fluid",
           "lbmd_set_populations", "lbmd_get_populations", "lbmd_set_particles", "lbmd_set_bonds",
           "lbmd_step", "lbmd_set_graphs", "lbmd_set_lattice_passes", "lbmd_get_lattice_passes", "lbmd_sync", "lbmd_clear_error", "lbmd_get_fields", "lbmd_get_particles",
           "lbmd_get_fields_dev", "lbmd_get_populations_dev", "lbmd_get_particles_dev",
           "lbmd_diagnostics", "lbmd_set_drift_reference", "lbmd_get_drift", "lbmd_step_count", "lbmd_profile_enable", "lbmd_profile_read",
           "lbmd_launch_count", "lbmd_last_error", "lbmd_fluid_moments_static",
           "lbmd_batch_create", "lbmd_batch_destroy", "lbmd_batch_add", "lbmd_batch_remove",
           "lbmd_batch_set_types", "lbmd_batch_set_debye_hueckel", "lbmd_batch_init_fluid",
           "lbmd_batch_set_particles", "lbmd_batch_step", "lbmd_batch_poll", "lbmd_batch_slot_error",
           "lbmd_batch_step_count", "lbmd_batch_get_populations", "lbmd_batch_get_fields",
           "lbmd_batch_get_particles", "lbmd_batch_diagnostics", "lbmd_batch_get_drift", "lbmd_batch_set_config",
           "lbmd_batch_get_config", "lbmd_batch_tune", "lbmd_batch_info", "lbmd_batch_launch_count",
           "lbmd_batch_last_error")


class LbmdError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__("lbmd error %d: %s" % (code, msg))
        self.code = code


class lbmd_params(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int), ("ny", ctypes.c_int), ("nz", ctypes.c_int),
                ("tau_r", ctypes.c_double), ("g_AB", ctypes.c_double), ("g_BA", ctypes.c_double),
                ("kT", ctypes.c_double), ("dt", ctypes.c_double), ("storage", ctypes.c_int),
                ("rho0_A", ctypes.c_double), ("rho0_B", ctypes.c_double), ("seed", ctypes.c_uint64),
                ("collision", ctypes.c_int), ("lambda_bulk", ctypes.c_double), ("lambda_mom", ctypes.c_double),
                ("lambda_ghost", ctypes.c_double), ("md_substeps", ctypes.c_int), ("diag_every", ctypes.c_int),
                ("drift_tol", ctypes.c_double)]


class lbmd_ptype(ctypes.Structure):
    _fields_ = [(n, ctypes.c_double) for n in ("kappa_A", "kappa_B", "lambda_A", "lambda_B", "gamma", "mass")]


class lbmd_pair(ctypes.Structure):
    _fields_ = [("type_i", ctypes.c_int), ("type_j", ctypes.c_int), ("wca_eps", ctypes.c_double),
                ("wca_sigma", ctypes.c_double)]


def _load():
    if not os.path.exists(LIB_PATH):
        raise ImportError("liblbmd.so is not built (run paper_1306_0788_gb300/build.py or "
                          "__graft_entry__.build()); there is no CPU fallback")
    lib = ctypes.CDLL(LIB_PATH)
    P = ctypes.c_void_p
    I = ctypes.c_int
    D = ctypes.c_double
    sig = {
        "lbmd_create": (I, [ctypes.POINTER(lbmd_params), P, ctypes.POINTER(P), ctypes.POINTER(ctypes.c_uint)]),
        "lbmd_destroy": (None, [P]),
        "lbmd_set_types": (I, [P, I, P, I, P, ctypes.POINTER(ctypes.c_uint)]),
        "lbmd_set_debye_hueckel": (I, [P, D, D, D]),
        "lbmd_init_fluid": (I, [P, P, P, P]),
        "lbmd_set_populations": (I, [P, I, P]),
        "lbmd_get_populations": (I, [P, I, P]),
        "lbmd_set_particles": (I, [P, I, P, P, P, P]),
        "lbmd_set_bonds": (I, [P, I, P, I, D, D]),
        "lbmd_step": (I, [P, I]),
        "lbmd_set_graphs": (I, [P, I]),
        "lbmd_set_lattice_passes": (I, [P, I]),
        "lbmd_get_lattice_passes": (I, [P]),
        "lbmd_sync": (I, [P]),
        "lbmd_clear_error": (I, [P]),
        "lbmd_get_fields": (I, [P, P, P, P]),
        "lbmd_get_particles": (I, [P, P, P, P]),
        "lbmd_get_fields_dev": (I, [P, P, P, P, P]),
        "lbmd_get_populations_dev": (I, [P, I, P, P]),
        "lbmd_get_particles_dev": (I, [P, P, P, P, P]),
        "lbmd_diagnostics": (I, [P, P]),
        "lbmd_set_drift_reference": (I, [P]),
        "lbmd_get_drift": (I, [P, P]),
        "lbmd_step_count": (ctypes.c_int64, [P]),
        "lbmd_profile_enable": (I, [P, I]),
        "lbmd_profile_read": (I, [P, ctypes.POINTER(D), ctypes.POINTER(ctypes.c_int64), I]),
        "lbmd_launch_count": (ctypes.c_int64, [P]),
        "lbmd_last_error": (ctypes.c_char_p, [P]),
        "lbmd_fluid_moments_static": (I, [P, I, I, I, P, P]),
        "lbmd_batch_create": (I, [ctypes.c_size_t, I, I, P, ctypes.POINTER(P)]),
        "lbmd_batch_destroy": (None, [P]),
        "lbmd_batch_add": (I, [P, ctypes.POINTER(lbmd_params), I, ctypes.c_int64, ctypes.POINTER(I),
                               ctypes.POINTER(ctypes.c_uint)]),
        "lbmd_batch_remove": (I, [P, I]),
        "lbmd_batch_set_types": (I, [P, I, I, P, I, P, ctypes.POINTER(ctypes.c_uint)]),
        "lbmd_batch_set_debye_hueckel": (I, [P, I, D, D, D]),
        "lbmd_batch_init_fluid": (I, [P, I, P, P, P]),
        "lbmd_batch_set_particles": (I, [P, I, I, P, P, P, P]),
        "lbmd_batch_step": (I, [P, I]),
        "lbmd_batch_poll": (I, [P, P]),
        "lbmd_batch_slot_error": (I, [P, I]),
        "lbmd_batch_step_count": (ctypes.c_int64, [P, I]),
        "lbmd_batch_get_populations": (I, [P, I, I, P]),
        "lbmd_batch_get_fields": (I, [P, I, P, P, P]),
        "lbmd_batch_get_particles": (I, [P, I, P, P, P]),
        "lbmd_batch_diagnostics": (I, [P, I, P]),
        "lbmd_batch_get_drift": (I, [P, I, P]),
        "lbmd_batch_set_config": (I, [P, I, I, I, I]),
        "lbmd_batch_get_config": (I, [P, P]),
        "lbmd_batch_tune": (I, [P, P, P]),
        "lbmd_batch_info": (I, [P, ctypes.POINTER(ctypes.c_size_t), ctypes.POINTER(ctypes.c_size_t),
                                ctypes.POINTER(I), ctypes.POINTER(I)]),
        "lbmd_batch_launch_count": (ctypes.c_int64, [P]),
        "lbmd_batch_last_error": (ctypes.c_char_p, [P]),
    }
    for name, (res, args) in sig.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    return lib


_lib = _load()


def _check(ctx, code: int):
    if code != LBMD_OK:
        raise LbmdError(code, _lib.lbmd_last_error(ctx).decode(errors="replace"))
    return code


def _p(a: np.ndarray | None):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


def _f32(a):
    return None if a is None else np.ascontiguousarray(a, dtype=np.float32)


def _f64(a):
    return None if a is None else np.ascontiguousarray(a, dtype=np.float64)


def stream_handle(stream) -> int | None:
    """Accept a raw cudaStream_t (int), a torch.cuda.Stream, or None."""
    if stream is None:
        return None
    if isinstance(stream, int):
        return stream
    return int(stream.cuda_stream)


# ------------------------------------------------------------------ entry points
def lbmd_create(params: lbmd_params, stream=None):
    """Returns (ctx, warnings)."""
    ctx = ctypes.c_void_p()
    w = ctypes.c_uint(0)
    _check(None, _lib.lbmd_create(ctypes.byref(params), stream_handle(stream), ctypes.byref(ctx), ctypes.byref(w)))
    return ctx, w.value


def lbmd_destroy(ctx) -> None:
    _lib.lbmd_destroy(ctx)


def lbmd_set_types(ctx, types, pairs=()) -> int:
    t = (lbmd_ptype * len(types))(*types)
    pr = (lbmd_pair * max(1, len(pairs)))(*pairs)
    w = ctypes.c_uint(0)
    _check(ctx, _lib.lbmd_set_types(ctx, len(types), t, len(pairs), pr, ctypes.byref(w)))
    return w.value


def lbmd_set_debye_hueckel(ctx, lB: float, kappa_D: float, rc: float) -> None:
    _check(ctx, _lib.lbmd_set_debye_hueckel(ctx, lB, kappa_D, rc))


def lbmd_init_fluid(ctx, rhoA, rhoB, u=None) -> None:
    a, b, c = _f32(rhoA), _f32(rhoB), _f32(u)
    _check(ctx, _lib.lbmd_init_fluid(ctx, _p(a), _p(b), _p(c)))


def lbmd_set_populations(ctx, comp: int, f) -> None:
    a = _f32(f)
    _check(ctx, _lib.lbmd_set_populations(ctx, comp, _p(a)))


def lbmd_get_populations(ctx, comp: int, shape) -> np.ndarray:
    """shape = (nz, ny, nx); returns [19, nz, ny, nx] float32."""
    out = np.empty((19,) + tuple(shape), dtype=np.float32)
    _check(ctx, _lib.lbmd_get_populations(ctx, comp, _p(out)))
    return out


def lbmd_set_particles(ctx, x, v, type_, q=None) -> None:
    x, v = _f64(x).reshape(-1, 3), _f64(v).reshape(-1, 3)
    t = np.ascontiguousarray(type_, dtype=np.int32)
    qq = _f64(q)
    _check(ctx, _lib.lbmd_set_particles(ctx, len(t), _p(x), _p(v), _p(t), _p(qq)))


def lbmd_set_bonds(ctx, pairs, kind: int, k: float, r: float) -> None:
    b = np.ascontiguousarray(pairs, dtype=np.int32).reshape(-1, 2)
    _check(ctx, _lib.lbmd_set_bonds(ctx, len(b), _p(b), kind, k, r))


def lbmd_step(ctx, nsteps: int) -> None:
    _check(ctx, _lib.lbmd_step(ctx, nsteps))


def lbmd_set_graphs(ctx, on: bool) -> None:
    _check(ctx, _lib.lbmd_set_graphs(ctx, int(bool(on))))


def lbmd_set_lattice_passes(ctx, passes: int) -> None:
    """0: chosen by the lattice size, 1: one-pass update, 2: density pass + update."""
    _check(ctx, _lib.lbmd_set_lattice_passes(ctx, passes))


def lbmd_get_lattice_passes(ctx) -> int:
    r = _lib.lbmd_get_lattice_passes(ctx)
    if r < 0:
        _check(ctx, r)
    return int(r)


def lbmd_sync(ctx) -> None:
    _check(ctx, _lib.lbmd_sync(ctx))


def lbmd_clear_error(ctx) -> None:
    _check(ctx, _lib.lbmd_clear_error(ctx))


def lbmd_get_fields(ctx, shape, want_u: bool = True):
    """Returns rhoA, rhoB [nz, ny, nx] and u [nz, ny, nx, 3] (or None)."""
    a = np.empty(tuple(shape), dtype=np.float32)
    b = np.empty(tuple(shape), dtype=np.float32)
    u = np.empty(tuple(shape) + (3,), dtype=np.float32) if want_u else None
    _check(ctx, _lib.lbmd_get_fields(ctx, _p(a), _p(b), _p(u)))
    return a, b, u


def lbmd_get_particles(ctx, n: int):
    """Returns x, v, f, each [n, 3] float64 in the caller's particle order."""
    x, v, f = np.empty((n, 3)), np.empty((n, 3)), np.empty((n, 3))
    _check(ctx, _lib.lbmd_get_particles(ctx, _p(x), _p(v), _p(f)))
    return x, v, f


def lbmd_get_fields_dev(ctx, rhoA_dev_ptr, rhoB_dev_ptr, u_dev_ptr, stream=None) -> None:
    """Device pointers (ints, e.g. tensor.data_ptr(); 0 or None to skip one) of rhoA, rhoB
    [nz, ny, nx] and u [nz, ny, nx, 3] FP32, written in the order of stream."""
    _check(ctx, _lib.lbmd_get_fields_dev(ctx, rhoA_dev_ptr or None, rhoB_dev_ptr or None, u_dev_ptr or None,
                                         stream_handle(stream)))


def lbmd_get_populations_dev(ctx, comp: int, f_dev_ptr: int, stream=None) -> None:
    """Device pointer of f [19, nz, ny, nx] FP32 of component comp, written in the order of stream."""
    _check(ctx, _lib.lbmd_get_populations_dev(ctx, comp, f_dev_ptr, stream_handle(stream)))


def lbmd_get_particles_dev(ctx, x_dev_ptr, v_dev_ptr, f_dev_ptr, stream=None) -> None:
    """Device pointers (or 0 / None) of x, v, f [n, 3] FP64 in the caller's particle order."""
    _check(ctx, _lib.lbmd_get_particles_dev(ctx, x_dev_ptr or None, v_dev_ptr or None, f_dev_ptr or None,
                                            stream_handle(stream)))


def lbmd_diagnostics(ctx) -> np.ndarray:
    out = np.zeros(8)
    _check(ctx, _lib.lbmd_diagnostics(ctx, _p(out)))
    return out


def lbmd_set_drift_reference(ctx) -> None:
    _check(ctx, _lib.lbmd_set_drift_reference(ctx))


def lbmd_get_drift(ctx) -> np.ndarray:
    """[step of the last check (-1: none), mass drift A, mass drift B, momentum drift per unit
    mass, checks since the reference]."""
    out = np.zeros(5)
    _check(ctx, _lib.lbmd_get_drift(ctx, _p(out)))
    return out


def lbmd_step_count(ctx) -> int:
    return int(_lib.lbmd_step_count(ctx))


def lbmd_launch_count(ctx) -> int:
    return int(_lib.lbmd_launch_count(ctx))


def lbmd_profile_enable(ctx, on: bool) -> None:
    _check(ctx, _lib.lbmd_profile_enable(ctx, int(bool(on))))


def lbmd_profile_read(ctx, reset: bool = True):
    ms = ctypes.c_double(0.0)
    n = ctypes.c_int64(0)
    _check(ctx, _lib.lbmd_profile_read(ctx, ctypes.byref(ms), ctypes.byref(n), int(bool(reset))))
    return ms.value, n.value


def lbmd_fluid_moments_static(f_dev_ptr: int, dims, out_dev_ptr: int, stream=None) -> None:
    """Device pointers in, device pointer out (no allocation); dims = (nx, ny, nz)."""
    nx, ny, nz = dims
    _check(None, _lib.lbmd_fluid_moments_static(f_dev_ptr, nx, ny, nz, out_dev_ptr, stream_handle(stream)))


def lbmd_last_error(ctx) -> str:
    return _lib.lbmd_last_error(ctx).decode(errors="replace")


# ------------------------------------------------------------------ batches
def _bcheck(b, code: int):
    if code != LBMD_OK:
        raise LbmdError(code, _lib.lbmd_batch_last_error(b).decode(errors="replace"))
    return code


def lbmd_batch_create(mem_budget: int = 0, storage: int = LBMD_STORAGE_FP32, max_slots: int = 1024, stream=None):
    b = ctypes.c_void_p()
    _bcheck(None, _lib.lbmd_batch_create(mem_budget, storage, max_slots, stream_handle(stream), ctypes.byref(b)))
    return b


def lbmd_batch_destroy(b) -> None:
    _lib.lbmd_batch_destroy(b)


def lbmd_batch_add(b, params: lbmd_params, np_max: int, total_steps: int):
    """Returns (slot, warnings); raises LbmdError(LBMD_E_NOMEM) when the replica does not fit."""
    slot = ctypes.c_int(-1)
    w = ctypes.c_uint(0)
    _bcheck(b, _lib.lbmd_batch_add(b, ctypes.byref(params), np_max, total_steps, ctypes.byref(slot), ctypes.byref(w)))
    return slot.value, w.value


def lbmd_batch_remove(b, slot: int) -> None:
    _bcheck(b, _lib.lbmd_batch_remove(b, slot))


def lbmd_batch_set_types(b, slot: int, types, pairs=()) -> int:
    t = (lbmd_ptype * len(types))(*types)
    pr = (lbmd_pair * max(1, len(pairs)))(*pairs)
    w = ctypes.c_uint(0)
    _bcheck(b, _lib.lbmd_batch_set_types(b, slot, len(types), t, len(pairs), pr, ctypes.byref(w)))
    return w.value


def lbmd_batch_set_debye_hueckel(b, slot: int, lB: float, kappa_D: float, rc: float) -> None:
    _bcheck(b, _lib.lbmd_batch_set_debye_hueckel(b, slot, lB, kappa_D, rc))


def lbmd_batch_init_fluid(b, slot: int, rhoA, rhoB, u=None) -> None:
    x, y, z = _f32(rhoA), _f32(rhoB), _f32(u)
    _bcheck(b, _lib.lbmd_batch_init_fluid(b, slot, _p(x), _p(y), _p(z)))


def lbmd_batch_set_particles(b, slot: int, x, v, type_, q=None) -> None:
    x, v = _f64(x).reshape(-1, 3), _f64(v).reshape(-1, 3)
    t = np.ascontiguousarray(type_, dtype=np.int32)
    qq = _f64(q)
    _bcheck(b, _lib.lbmd_batch_set_particles(b, slot, len(t), _p(x), _p(v), _p(t), _p(qq)))


def lbmd_batch_step(b, nsteps: int) -> None:
    _bcheck(b, _lib.lbmd_batch_step(b, nsteps))


def lbmd_batch_poll(b, max_slots: int) -> np.ndarray:
    st = np.zeros(max_slots, dtype=np.int32)
    _bcheck(b, _lib.lbmd_batch_poll(b, _p(st)))
    return st


def lbmd_batch_slot_error(b, slot: int) -> int:
    return int(_lib.lbmd_batch_slot_error(b, slot))


def lbmd_batch_step_count(b, slot: int) -> int:
    return int(_lib.lbmd_batch_step_count(b, slot))


def lbmd_batch_get_populations(b, slot: int, comp: int, shape) -> np.ndarray:
    out = np.empty((19,) + tuple(shape), dtype=np.float32)
    _bcheck(b, _lib.lbmd_batch_get_populations(b, slot, comp, _p(out)))
    return out


def lbmd_batch_get_fields(b, slot: int, shape, want_u: bool = True):
    a = np.empty(tuple(shape), dtype=np.float32)
    c = np.empty(tuple(shape), dtype=np.float32)
    u = np.empty(tuple(shape) + (3,), dtype=np.float32) if want_u else None
    _bcheck(b, _lib.lbmd_batch_get_fields(b, slot, _p(a), _p(c), _p(u)))
    return a, c, u


def lbmd_batch_get_particles(b, slot: int, n: int):
    x, v, f = np.empty((n, 3)), np.empty((n, 3)), np.empty((n, 3))
    _bcheck(b, _lib.lbmd_batch_get_particles(b, slot, _p(x), _p(v), _p(f)))
    return x, v, f


def lbmd_batch_diagnostics(b, slot: int) -> np.ndarray:
    out = np.zeros(8)
    _bcheck(b, _lib.lbmd_batch_diagnostics(b, slot, _p(out)))
    return out


def lbmd_batch_get_drift(b, slot: int) -> np.ndarray:
    out = np.zeros(5)
    _bcheck(b, _lib.lbmd_batch_get_drift(b, slot, _p(out)))
    return out


def lbmd_batch_set_config(b, tile_sites: int, grid_moments: int, grid_collide: int, collide_blocks: int) -> None:
    _bcheck(b, _lib.lbmd_batch_set_config(b, tile_sites, grid_moments, grid_collide, collide_blocks))


def lbmd_batch_get_config(b) -> dict:
    cfg = np.zeros(5, dtype=np.int32)
    _bcheck(b, _lib.lbmd_batch_get_config(b, _p(cfg)))
    return dict(zip(("tile_sites", "grid_moments", "grid_collide", "collide_blocks", "grid_particles"),
                    (int(v) for v in cfg)))


def lbmd_batch_tune(b):
    """Returns (config dict, (moments_ms, collide_ms))."""
    cfg = np.zeros(5, dtype=np.int32)
    ms = np.zeros(2)
    _bcheck(b, _lib.lbmd_batch_tune(b, _p(cfg), _p(ms)))
    keys = ("tile_sites", "grid_moments", "grid_collide", "collide_blocks", "grid_particles")
    return dict(zip(keys, (int(v) for v in cfg))), (float(ms[0]), float(ms[1]))


def lbmd_batch_info(b) -> dict:
    bud, used = ctypes.c_size_t(0), ctypes.c_size_t(0)
    occ, mx = ctypes.c_int(0), ctypes.c_int(0)
    _bcheck(b, _lib.lbmd_batch_info(b, ctypes.byref(bud), ctypes.byref(used), ctypes.byref(occ), ctypes.byref(mx)))
    return dict(budget=bud.value, used=used.value, occupied=occ.value, max_slots=mx.value)


def lbmd_batch_launch_count(b) -> int:
    return int(_lib.lbmd_batch_launch_count(b))


def lbmd_batch_last_error(b) -> str:
    return _lib.lbmd_batch_last_error(b).decode(errors="replace")


def params(dims, tau_r=1.0, g_AB=0.0, g_BA=None, kT=0.0, seed=0, storage=LBMD_STORAGE_FP32,
           rho0=(0.0, 0.0), collision=LBMD_COLLISION_BGK, lambda_bulk=None, lambda_mom=None,
           lambda_ghost=None, md_substeps=1, diag_every=0, drift_tol=0.0) -> lbmd_params:
    """Convenience constructor of lbmd_params (dims = (nx, ny, nz)); MRT eigenvalues left as
    None take the shear value -1/tau_r.  diag_every > 0 switches the FP64 drift check on."""
    nx, ny, nz = dims
    ls = -1.0 / tau_r
    pick = lambda v: ls if v is None else v  # noqa: E731
    return lbmd_params(nx, ny, nz, tau_r, g_AB, g_AB if g_BA is None else g_BA, kT, 1.0, storage,
                       rho0[0], rho0[1], seed, collision, pick(lambda_bulk), pick(lambda_mom), pick(lambda_ghost),
                       md_substeps, diag_every, drift_tol)
