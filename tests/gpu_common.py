"""Helpers that set up one system on both sides -- the CUDA library through the C ABI and
the FP64 oracle -- from the same seeded inputs."""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

import oracle
from paper_1306_0788_gb300 import inputs


@dataclass
class Case:
    dims: tuple
    tau_r: float = 1.0
    g: float = 0.0
    kT: float = 0.0
    seed: int = 7
    rhoA: np.ndarray = None
    rhoB: np.ndarray = None
    u: np.ndarray = None
    # per type: (kappa_A, kappa_B, lambda_A, lambda_B, gamma, mass)
    types: list = field(default_factory=lambda: [(0.0, 0.0, 0.0, 0.0, 1.0, 1.0)])
    wca: dict = field(default_factory=dict)  # (ti, tj) -> (eps, sigma)
    dh: tuple = (0.0, 0.0, 0.0)  # lB, kappa_D, rc
    x: np.ndarray = field(default_factory=lambda: np.zeros((0, 3)))
    v: np.ndarray = field(default_factory=lambda: np.zeros((0, 3)))
    ptype: np.ndarray = field(default_factory=lambda: np.zeros(0, dtype=np.int32))
    q: np.ndarray = None
    bonds: np.ndarray = field(default_factory=lambda: np.zeros((0, 2), dtype=np.int32))
    bond_kind: int = 2
    bond_k: float = 0.0
    bond_r: float = 1.0
    collision: int = 0  # 0 BGK, 1 fluctuating MRT
    lam_bulk: float = None
    lam_mom: float = None
    lam_ghost: float = None
    md_substeps: int = 1
    storage: int = 0  # LBMD_STORAGE_* (the CUDA path only)
    rho0: tuple = (0.0, 0.0)  # shift reference of the 16-bit storages

    def fields32(self):
        return (self.rhoA.astype(np.float32), self.rhoB.astype(np.float32),
                None if self.u is None else self.u.astype(np.float32))

    @property
    def shape(self):
        return self.dims[::-1]

    @property
    def n(self):
        return len(self.ptype)


def noisy_fluid(dims, amp=0.01, seed=7, rho0=1.0):
    return inputs.uniform_noise(dims, rho0, amp, seed=seed)


def oracle_system(c: Case) -> oracle.System:
    nt = len(c.types)
    kappa = np.array([[t[0], t[1]] for t in c.types])
    lam = np.array([[t[2], t[3]] for t in c.types])
    gamma = np.array([t[4] for t in c.types])
    mass = np.array([t[5] for t in c.types])
    eps = np.zeros((nt, nt))
    sig = np.ones((nt, nt))
    for (i, j), (e, s) in c.wca.items():
        eps[i, j] = eps[j, i] = e
        sig[i, j] = sig[j, i] = s
    q = np.zeros(c.n) if c.q is None else np.asarray(c.q, dtype=np.float64)
    return oracle.System(dims=c.dims, tau_r=c.tau_r, g_AB=c.g, g_BA=c.g, kT=c.kT, seed=c.seed, kappa=kappa,
                         lam=lam, gamma=gamma, mass=mass, wca_eps=eps, wca_sig=sig, dh_lB=c.dh[0],
                         dh_kappa=c.dh[1], dh_rc=c.dh[2], type=np.asarray(c.ptype, dtype=np.int32), q=q,
                         bonds=np.asarray(c.bonds, dtype=np.int32).reshape(-1, 2), bond_kind=c.bond_kind,
                         bond_k=c.bond_k, bond_r=c.bond_r, collision=c.collision, lam_bulk=c.lam_bulk,
                         lam_mom=c.lam_mom, lam_ghost=c.lam_ghost, md_substeps=c.md_substeps)


def run_oracle(c: Case, nsteps: int, trace_last: bool = False):
    a, b, u = c.fields32()
    f = oracle.init_equilibrium(a.astype(np.float64), b.astype(np.float64),
                                None if u is None else u.astype(np.float64))
    x = np.ascontiguousarray(c.x, dtype=np.float64).copy()
    v = np.ascontiguousarray(c.v, dtype=np.float64).copy()
    s = oracle_system(c)
    tr = None
    for k in range(nsteps):
        st, tr = oracle.step(s, f, x, v, k, trace=trace_last and k == nsteps - 1)
        assert st == 0, "oracle step %d status %d" % (k, st)
    return f, x, v, tr


def make_gpu(c: Case, stream=None, passes=None, **params):
    """A context holding case c (passes: the lattice update, lbmd_set_lattice_passes; params:
    further lbmd_params fields, e.g. the drift check)."""
    from paper_1306_0788_gb300 import lbmd as L
    ctx, _ = L.lbmd_create(L.params(c.dims, tau_r=c.tau_r, g_AB=c.g, kT=c.kT, seed=c.seed, collision=c.collision,
                                    lambda_bulk=c.lam_bulk, lambda_mom=c.lam_mom, lambda_ghost=c.lam_ghost,
                                    md_substeps=c.md_substeps, storage=c.storage, rho0=c.rho0, **params), stream)
    if passes is not None:
        L.lbmd_set_lattice_passes(ctx, passes)
    types = [L.lbmd_ptype(*t) for t in c.types]
    pairs = [L.lbmd_pair(i, j, e, s) for (i, j), (e, s) in c.wca.items()]
    L.lbmd_set_types(ctx, types, pairs)
    if c.dh[0] != 0.0:
        L.lbmd_set_debye_hueckel(ctx, *c.dh)
    a, b, u = c.fields32()
    L.lbmd_init_fluid(ctx, a, b, u)
    L.lbmd_set_particles(ctx, c.x, c.v, c.ptype, c.q)
    if len(c.bonds):
        L.lbmd_set_bonds(ctx, c.bonds, c.bond_kind, c.bond_k, c.bond_r)
    return ctx


def run_gpu(c: Case, nsteps: int, passes=None):
    from paper_1306_0788_gb300 import lbmd as L
    ctx = make_gpu(c, passes=passes)
    try:
        L.lbmd_step(ctx, nsteps)
        L.lbmd_sync(ctx)
        f = np.stack([L.lbmd_get_populations(ctx, 0, c.shape), L.lbmd_get_populations(ctx, 1, c.shape)])
        x, v, F = L.lbmd_get_particles(ctx, c.n)
    finally:
        L.lbmd_destroy(ctx)
    return f, x, v, F


def pop_error(fg, fo):
    """||f_gpu - f_ref||_inf / ||f_ref||_inf (the stated population tolerance)."""
    return float(np.abs(fg.astype(np.float64) - fo).max() / np.abs(fo).max())


def position_error(xg, xo, x0, dims):
    """Minimum-image |dx| over max(rms displacement, 1 lattice unit)."""
    L = np.asarray(dims, dtype=np.float64)

    def mi(d):
        return d - L * np.round(d / L)

    if len(xo) == 0:
        return 0.0
    err = np.sqrt((mi(xg - xo) ** 2).sum(1)).max()
    rms = np.sqrt((mi(xo - x0) ** 2).sum(1).mean())
    return float(err / max(rms, 1.0))
