"""FP64 CPU oracle of the coupled Shan-Chen LB / MD step (arXiv:1306.0788).

TEST INFRASTRUCTURE ONLY: the test-suite, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` are the only callers.  The oracle is plain C
(``lbmd_oracle.c``) compiled with gcc without FMA contraction, plus this ctypes
marshalling layer.  It shares no code with the CUDA library.

Every function follows one passage of the paper (cited in the C source):
  * ``feq``           Eq. (feq)
  * ``forcing``       forcing source term of the appendix (Delta^g, G)
  * ``sc_force``      Eq. (SCforce)
  * ``fs_geometry``   geometric factor of Eq. (solvation_lambda)
  * ``pair_energy`` / ``pair_force``  WCA, Debye-Hueckel, FENE, harmonic
  * ``step``          one full coupled step (Sec. 2 and the appendix)
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from dataclasses import dataclass, field

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "lbmd_oracle.c")
_LIB = os.path.join(_HERE, "liblbmd_oracle.so")
_lib = None

Q = 19
CS2 = 1.0 / 3.0


def build(force: bool = False) -> str:
    """Compile the oracle shared library with gcc (IEEE double, no FMA contraction)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + ".tmp%d" % os.getpid()
        subprocess.check_call(["gcc", "-O3", "-ffp-contract=off", "-fno-fast-math", "-fopenmp", "-fPIC",
                               "-shared", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    if _lib is None:
        build()
        _lib = ctypes.CDLL(_LIB)
        _lib.orc_step.restype = ctypes.c_int
        _lib.orc_pair_energy.restype = ctypes.c_double
        _lib.orc_pair_force.restype = ctypes.c_double
        for name in ("orc_pair_energy", "orc_pair_force"):
            getattr(_lib, name).argtypes = [ctypes.c_int, ctypes.c_double, ctypes.c_double,
                                            ctypes.c_double, ctypes.c_double]
        _lib.orc_feq.argtypes = [ctypes.c_double, ctypes.c_void_p, ctypes.c_void_p]
        _lib.orc_forcing.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_double,
                                     ctypes.c_double, ctypes.c_double, ctypes.c_void_p]
        _lib.orc_sc_force.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                      ctypes.c_double, ctypes.c_double] + [ctypes.c_void_p] * 4
        _lib.orc_normals.argtypes = [ctypes.c_uint64, ctypes.c_uint64, ctypes.c_uint32,
                                     ctypes.c_void_p]
        _lib.orc_fluid_normals.argtypes = [ctypes.c_uint64, ctypes.c_uint64, ctypes.c_uint32, ctypes.c_void_p]
        _lib.orc_mode_basis.argtypes = [ctypes.c_void_p, ctypes.c_void_p]
        _lib.orc_set_threads.argtypes = [ctypes.c_int]
    return _lib


def set_threads(n: int) -> None:
    """Host threads of the oracle's per-site loops (1 by default); results do not depend on it."""
    _load().orc_set_threads(int(n))


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def _f64(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.float64)


# ----------------------------------------------------------------- pieces
def lattice():
    """D3Q19 velocities (19, 3) and weights (19,), Eqs. (velo), (weights)."""
    c = np.zeros((Q, 3), dtype=np.int32)
    w = np.zeros(Q, dtype=np.float64)
    _load().orc_lattice(_ptr(c), _ptr(w))
    return c, w


def feq(rho: float, u) -> np.ndarray:
    out = np.zeros(Q)
    _load().orc_feq(float(rho), _ptr(_f64(u)), _ptr(out))
    return out


def forcing(g, u, lam_M: float, lam_s: float, lam_b: float) -> np.ndarray:
    out = np.zeros(Q)
    _load().orc_forcing(_ptr(_f64(g)), _ptr(_f64(u)), lam_M, lam_s, lam_b, _ptr(out))
    return out


def sc_force(rhoA: np.ndarray, rhoB: np.ndarray, gAB: float, gBA: float):
    """Shan-Chen force per component on a periodic [nz, ny, nx] lattice.
    Returns (gA, gB, SA, SB), each [nz, ny, nx, 3]."""
    rA, rB = _f64(rhoA), _f64(rhoB)
    nz, ny, nx = rA.shape
    dim = np.array([nx, ny, nz], dtype=np.int32)
    out = [np.zeros(rA.shape + (3,)) for _ in range(4)]
    _load().orc_sc_force(_ptr(dim), _ptr(rA), _ptr(rB), gAB, gBA, *[_ptr(o) for o in out])
    return tuple(out)


def philox4x32_10(ctr, key) -> np.ndarray:
    c = np.ascontiguousarray(ctr, dtype=np.uint32)
    k = np.ascontiguousarray(key, dtype=np.uint32)
    out = np.zeros(4, dtype=np.uint32)
    _load().orc_philox4x32_10(_ptr(c), _ptr(k), _ptr(out))
    return out


def normals(seed: int, step: int, pid: int) -> np.ndarray:
    out = np.zeros(3)
    _load().orc_normals(seed, step, pid, _ptr(out))
    return out


def mode_basis():
    """(e [19, 19] with e[k, i] = e_k(c_i), b [19] = sum_i w_i e_ki^2): the MRT mode basis."""
    e, b = np.zeros((Q, Q)), np.zeros(Q)
    _load().orc_mode_basis(_ptr(e), _ptr(b))
    return e, b


def fluid_normals(seed: int, step: int, site: int) -> np.ndarray:
    """The 36 unit normals of one node and step of the fluctuating MRT collision."""
    out = np.zeros(36)
    _load().orc_fluid_normals(seed, step, site, _ptr(out))
    return out


def fs_geometry(d) -> np.ndarray:
    out = np.zeros(3)
    _load().orc_fs_geometry(_ptr(_f64(d)), _ptr(out))
    return out


PAIR_WCA, PAIR_DH, BOND_FENE, BOND_HARMONIC = 0, 1, 2, 3
COLLISION_BGK, COLLISION_MRT = 0, 1


def pair_energy(kind: int, p0: float, p1: float, p2: float, r: float) -> float:
    return _load().orc_pair_energy(kind, p0, p1, p2, r)


def pair_force(kind: int, p0: float, p1: float, p2: float, r: float) -> float:
    return _load().orc_pair_force(kind, p0, p1, p2, r)


def init_equilibrium(rhoA: np.ndarray, rhoB: np.ndarray, u=None) -> np.ndarray:
    """f_zi = f^eq_i(rho_z, u) with layout [2, 19, nz, ny, nx]."""
    rA, rB = _f64(rhoA), _f64(rhoB)
    nz, ny, nx = rA.shape
    dim = np.array([nx, ny, nz], dtype=np.int32)
    f = np.zeros((2, Q, nz, ny, nx))
    up = None if u is None else _ptr(_f64(u))
    _load().orc_init_equilibrium(_ptr(dim), _ptr(rA), _ptr(rB), up, _ptr(f))
    return f


def fluid_moments(f: np.ndarray) -> np.ndarray:
    """[M_A, M_B, Px, Py, Pz] of populations [2, 19, nz, ny, nx]."""
    f = _f64(f)
    nz, ny, nx = f.shape[2:]
    dim = np.array([nx, ny, nz], dtype=np.int32)
    out = np.zeros(5)
    _load().orc_fluid_moments(_ptr(dim), _ptr(f), _ptr(out))
    return out


# ----------------------------------------------------------------- the step
class _OrcSystem(ctypes.Structure):
    _fields_ = [("dim", ctypes.c_int * 3), ("tau_r", ctypes.c_double), ("g_AB", ctypes.c_double),
                ("g_BA", ctypes.c_double), ("kT", ctypes.c_double), ("dt", ctypes.c_double),
                ("seed", ctypes.c_uint64), ("ntypes", ctypes.c_int),
                ("kappa", ctypes.c_void_p), ("lam", ctypes.c_void_p), ("gamma", ctypes.c_void_p),
                ("mass", ctypes.c_void_p), ("wca_eps", ctypes.c_void_p), ("wca_sig", ctypes.c_void_p),
                ("dh_lB", ctypes.c_double), ("dh_kappa", ctypes.c_double), ("dh_rc", ctypes.c_double),
                ("np", ctypes.c_int), ("type", ctypes.c_void_p), ("q", ctypes.c_void_p),
                ("pid", ctypes.c_void_p), ("nbonds", ctypes.c_int), ("bonds", ctypes.c_void_p),
                ("bond_kind", ctypes.c_int), ("bond_k", ctypes.c_double), ("bond_r", ctypes.c_double),
                ("collision", ctypes.c_int), ("lam_bulk", ctypes.c_double), ("lam_mom", ctypes.c_double),
                ("lam_ghost", ctypes.c_double), ("md_substeps", ctypes.c_int)]


class _OrcTrace(ctypes.Structure):
    _fields_ = [(n, ctypes.c_void_p) for n in
                ("rho", "u_cpl", "g", "f_fric", "f_ps", "f_fs", "f_pair", "f_bond", "f_total")]


@dataclass
class System:
    """Parameters of the coupled model (oracle side).

    Per-type arrays: kappa[t] = (kappa_A, kappa_B), lam[t] = (lambda_A, lambda_B),
    gamma[t], mass[t]; wca_eps / wca_sig are [ntypes, ntypes]."""
    dims: tuple  # (nx, ny, nz)
    tau_r: float = 1.0
    g_AB: float = 0.0
    g_BA: float = 0.0
    kT: float = 0.0
    dt: float = 1.0
    seed: int = 0
    kappa: np.ndarray = field(default_factory=lambda: np.zeros((1, 2)))
    lam: np.ndarray = field(default_factory=lambda: np.zeros((1, 2)))
    gamma: np.ndarray = field(default_factory=lambda: np.ones(1))
    mass: np.ndarray = field(default_factory=lambda: np.ones(1))
    wca_eps: np.ndarray = field(default_factory=lambda: np.zeros((1, 1)))
    wca_sig: np.ndarray = field(default_factory=lambda: np.ones((1, 1)))
    dh_lB: float = 0.0
    dh_kappa: float = 0.0
    dh_rc: float = 0.0
    type: np.ndarray = field(default_factory=lambda: np.zeros(0, dtype=np.int32))
    q: np.ndarray = field(default_factory=lambda: np.zeros(0))
    pid: np.ndarray = None
    bonds: np.ndarray = field(default_factory=lambda: np.zeros((0, 2), dtype=np.int32))
    bond_kind: int = BOND_FENE
    bond_k: float = 0.0
    bond_r: float = 1.0
    # collision: COLLISION_BGK, or COLLISION_MRT (fluctuating when kT > 0) with the bulk,
    # component-momentum and kinetic eigenvalues (None: -1/tau_r, the shear one)
    collision: int = 0
    lam_bulk: float = None
    lam_mom: float = None
    lam_ghost: float = None
    md_substeps: int = 1  # particle substeps per lattice step (reading R15)

    def _struct(self):
        keep = []

        def arr(a, dt):
            a = np.ascontiguousarray(a, dtype=dt)
            keep.append(a)
            return _ptr(a)

        n = len(self.type)
        pid = np.arange(n, dtype=np.int32) if self.pid is None else self.pid
        q = self.q if len(self.q) == n else np.zeros(n)
        s = _OrcSystem()
        s.dim[:] = [int(v) for v in self.dims]
        s.tau_r, s.g_AB, s.g_BA, s.kT, s.dt = self.tau_r, self.g_AB, self.g_BA, self.kT, self.dt
        s.seed = int(self.seed)
        s.ntypes = int(np.asarray(self.gamma).shape[0])
        s.kappa, s.lam = arr(self.kappa, np.float64), arr(self.lam, np.float64)
        s.gamma, s.mass = arr(self.gamma, np.float64), arr(self.mass, np.float64)
        s.wca_eps, s.wca_sig = arr(self.wca_eps, np.float64), arr(self.wca_sig, np.float64)
        s.dh_lB, s.dh_kappa, s.dh_rc = self.dh_lB, self.dh_kappa, self.dh_rc
        s.np = n
        s.type, s.q, s.pid = arr(self.type, np.int32), arr(q, np.float64), arr(pid, np.int32)
        s.nbonds = int(len(self.bonds))
        s.bonds = arr(self.bonds, np.int32)
        s.bond_kind, s.bond_k, s.bond_r = int(self.bond_kind), float(self.bond_k), float(self.bond_r)
        ls = -1.0 / self.tau_r
        s.collision = int(self.collision)
        s.lam_bulk = ls if self.lam_bulk is None else float(self.lam_bulk)
        s.lam_mom = ls if self.lam_mom is None else float(self.lam_mom)
        s.lam_ghost = ls if self.lam_ghost is None else float(self.lam_ghost)
        s.md_substeps = int(self.md_substeps)
        return s, keep


TRACE_KEYS = ("rho", "u_cpl", "g", "f_fric", "f_ps", "f_fs", "f_pair", "f_bond", "f_total")


def step(system: System, f: np.ndarray, x: np.ndarray, v: np.ndarray, step_index: int,
         trace: bool = False):
    """Advance f [2,19,nz,ny,nx], x [np,3], v [np,3] (float64, C order) by one step in
    place.  Returns (status, trace_dict or None)."""
    for a in (f, x, v):
        assert a.dtype == np.float64 and a.flags.c_contiguous
    nx, ny, nz = system.dims
    N = nx * ny * nz
    n = len(system.type)
    s, keep = system._struct()
    tr = None
    out = None
    if trace:
        out = {"rho": np.zeros((2, nz, ny, nx)), "u_cpl": np.zeros((nz, ny, nx, 3)),
               "g": np.zeros((2, nz, ny, nx, 3))}
        for k in TRACE_KEYS[3:]:
            out[k] = np.zeros((n, 3))
        tr = _OrcTrace(*[_ptr(out[k]) for k in TRACE_KEYS])
    del N
    st = _load().orc_step(ctypes.byref(s), _ptr(f), _ptr(x), _ptr(v), ctypes.c_uint64(step_index),
                          ctypes.byref(tr) if tr is not None else None)
    del keep
    return st, out


def run(system: System, f, x, v, nsteps: int, first_step: int = 0):
    """nsteps oracle steps; raises if a step reports an invalid state."""
    for k in range(nsteps):
        st, _ = step(system, f, x, v, first_step + k)
        if st != 0:
            raise FloatingPointError("oracle step %d returned status %d" % (first_step + k, st))
