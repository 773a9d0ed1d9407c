"""Reproductions of the paper's solvation-force examples on the CUDA path.

- Free-energy profile (Sec. 3, Eq. solvation_density and the figure beside it): a particle
  held at heights across a flat A/B interface; the work of the holding force is Delta E(z),
  whose bulk-to-bulk difference is -sum_z kappa_z Delta rho_z.
- Contact angle (Sec. 4.1): particles repelled by both components (kappa_A, kappa_B > 0)
  adsorb at the interface; their equilibrium distance d from it depends on the relative
  coupling difference 2 (kappa_A - kappa_B) / (kappa_A + kappa_B); the largest holding force
  across the interface is the detachment force F_D; with the interfacial tension gamma_AB
  (Laplace's law, Sec. 4.3) the effective radius is R_eff = F_D / (pi gamma_AB) and the
  effective contact angle cos(theta) = d / R_eff.
- Particle-fluid demixing (Sec. 3, the single-fluid example): particles that deplete the
  fluid around them (Eq. solvation_lambda) and are pushed down density gradients (Eq.
  solvation_kappa) gather into particle-rich, fluid-poor domains.

Every lattice and particle step runs in the library's kernels through the C ABI; the host
sets inputs up and reduces what it reads back (profiles, crossings, cluster statistics).
"""
from __future__ import annotations

import time

import numpy as np

from . import inputs
from . import lbmd as L

CS2 = 1.0 / 3.0
HELD_MASS = 1e12  # a held particle: no friction, and a mass that no force of a step moves


def _ctx(dims, g, kT=0.0, seed=0, tau_r=1.0):
    ctx, _ = L.lbmd_create(L.params(dims, tau_r=tau_r, g_AB=g, kT=kT, seed=seed))
    return ctx


def _pops(ctx, dims):
    shape = tuple(dims[::-1])
    return np.stack([L.lbmd_get_populations(ctx, 0, shape), L.lbmd_get_populations(ctx, 1, shape)])


def relax(rhoA, rhoB, g: float, steps: int, tau_r: float = 1.0):
    """Fluid started at equilibrium from rho_A, rho_B [nz, ny, nx] and run `steps` steps without
    particles.  Returns the populations [2, 19, nz, ny, nx] and the densities rho_A, rho_B."""
    dims = rhoA.shape[::-1]
    ctx = _ctx(dims, g, tau_r=tau_r)
    try:
        L.lbmd_init_fluid(ctx, rhoA, rhoB)
        L.lbmd_step(ctx, steps)
        f = _pops(ctx, dims)
        a, b, _ = L.lbmd_get_fields(ctx, dims[::-1], want_u=False)
    finally:
        L.lbmd_destroy(ctx)
    return f, a, b


def relaxed_interface(dims, g: float, rho_hi: float, rho_lo: float, width: float = 2.0, steps: int = 3000):
    """The flat-slab fluid of inputs.flat_slab relaxed for `steps` steps."""
    rA, rB = inputs.flat_slab(dims, rho_hi, rho_lo, width)
    return relax(rA.astype(np.float32), rB.astype(np.float32), g, steps)


def tile_lateral(f, nx: int, ny: int):
    """Populations of a state that is uniform in x and y, repeated to nx by ny columns."""
    f = np.asarray(f)
    assert nx % f.shape[-1] == 0 and ny % f.shape[-2] == 0
    return np.tile(f, (1, 1, 1, ny // f.shape[-2], nx // f.shape[-1]))


def holding_forces(f, g: float, kappa, probes, lam=(0.0, 0.0)):
    """Force on particles held at `probes` [n, 3] in the fluid state f [2, 19, nz, ny, nx]:
    one step from that state with the probes in place, no friction, no pair forces.  The force
    is that of Eq. solvation_kappa (plus the reaction of Eq. solvation_lambda when lam != 0),
    evaluated on the state before the step; the force needed to hold each probe is minus it."""
    dims = f.shape[-1], f.shape[-2], f.shape[-3]
    probes = np.ascontiguousarray(probes, dtype=np.float64).reshape(-1, 3)
    n = len(probes)
    ctx = _ctx(dims, g)
    try:
        L.lbmd_set_types(ctx, [L.lbmd_ptype(kappa[0], kappa[1], lam[0], lam[1], 0.0, HELD_MASS)])
        L.lbmd_set_populations(ctx, 0, f[0])
        L.lbmd_set_populations(ctx, 1, f[1])
        L.lbmd_set_particles(ctx, probes, np.zeros_like(probes), np.zeros(n, dtype=np.int32))
        L.lbmd_step(ctx, 1)
        _, _, F = L.lbmd_get_particles(ctx, n)
    finally:
        L.lbmd_destroy(ctx)
    return F


def free_energy_profile(zs, Fz):
    """Delta E(z) = -int_{z_0}^{z} F_z dz' (trapezoid rule): the work done by the force that
    holds the particle, zero at the first height."""
    zs, Fz = np.asarray(zs, dtype=np.float64), np.asarray(Fz, dtype=np.float64)
    steps = 0.5 * (Fz[1:] + Fz[:-1]) * np.diff(zs)
    return -np.concatenate([[0.0], np.cumsum(steps)])


def interface_height(rhoA, rhoB, z_lo: float, z_hi: float):
    """Height of the crossing rho_A = rho_B of the x-y averaged profiles between the nodes
    z_lo and z_hi (linear interpolation between the two nodes that bracket it)."""
    d = (np.asarray(rhoA, dtype=np.float64) - rhoB).mean(axis=(1, 2))
    for z in range(int(np.floor(z_lo)), int(np.ceil(z_hi))):
        a, b = d[z % len(d)], d[(z + 1) % len(d)]
        if a == 0.0:
            return float(z)
        if a * b < 0.0:
            return z + a / (a - b)
    raise ValueError("no crossing of rho_A = rho_B in [%g, %g]" % (z_lo, z_hi))


def coupling_pairs(kappa_sum: float, ratios):
    """(kappa_A, kappa_B) with kappa_A + kappa_B = kappa_sum and 2 (kappa_A - kappa_B) /
    (kappa_A + kappa_B) = ratio, for each ratio."""
    return [(0.5 * kappa_sum * (1 + 0.5 * r), 0.5 * kappa_sum * (1 - 0.5 * r)) for r in ratios]


def adsorption_heights(f, g: float, kappas, z0: float, steps: int, gamma: float = 1.0, mass: float = 10.0,
                       spacing: int = 4):
    """Free particles at k_BT = 0, one type per (kappa_A, kappa_B) pair, each alone in its own
    column (spacing apart in x and y), started at height z0 in the fluid f and run `steps`
    coupled steps.  Returns their final heights and the fluid densities at the end."""
    dims = f.shape[-1], f.shape[-2], f.shape[-3]
    nx, ny, _ = dims
    cols = [(spacing * (i % (nx // spacing)) + 0.5 * spacing, spacing * (i // (nx // spacing)) + 0.5 * spacing)
            for i in range(len(kappas))]
    if len(kappas) > (nx // spacing) * (ny // spacing) or len(kappas) > L.LBMD_MAX_TYPES:
        raise ValueError("too many coupling pairs for the lattice or the type table")
    x = np.array([[cx, cy, z0] for cx, cy in cols], dtype=np.float64)
    ctx = _ctx(dims, g)
    try:
        L.lbmd_set_types(ctx, [L.lbmd_ptype(ka, kb, 0.0, 0.0, gamma, mass) for ka, kb in kappas])
        L.lbmd_set_populations(ctx, 0, f[0])
        L.lbmd_set_populations(ctx, 1, f[1])
        L.lbmd_set_particles(ctx, x, np.zeros_like(x), np.arange(len(kappas), dtype=np.int32))
        L.lbmd_step(ctx, steps)
        xs, _, _ = L.lbmd_get_particles(ctx, len(kappas))
        a, b, _ = L.lbmd_get_fields(ctx, dims[::-1], want_u=False)
    finally:
        L.lbmd_destroy(ctx)
    return xs[:, 2], a, b


def laplace_tension(g: float, rho_hi: float, rho_lo: float, radii=(5.0, 7.0, 9.0), edge: int = 32,
                    steps: int = 3000, width: float = 1.0):
    """Interfacial tension from Laplace's law for A-rich cylinders in an edge x edge x 1 box
    (a flat interface has the tension of this lattice model's cylinder walls): after `steps`
    steps, Delta p = p(centre) - p(corner) with the bulk pressure of F_bulk, p = c_s^2 (rho_A +
    rho_B) + c_s^2 g rho_A rho_B; R from the A excess area.  Returns gamma (least-squares slope
    of Delta p against 1/R through the origin), the radii and the pressure jumps."""
    Rs, dps = [], []
    for R in radii:
        dims = (edge, edge, 1)
        rA, rB = inputs.disk(dims, R, rho_hi, rho_lo, width=width)
        _, A, B = relax(rA.astype(np.float32), rB.astype(np.float32), g, steps)
        A, B = A[0].astype(np.float64), B[0].astype(np.float64)
        p = CS2 * (A + B) + CS2 * g * A * B
        c = edge // 2
        dps.append(p[c, c] - p[0, 0])
        Rs.append(np.sqrt(((A - A[0, 0]) / (A[c, c] - A[0, 0])).sum() / np.pi))
    Rs, dps = np.array(Rs), np.array(dps)
    inv = 1.0 / Rs
    return float((inv @ dps) / (inv @ inv)), Rs, dps


def stable_zeros(zs, Fz):
    """Heights where F_z passes from positive to non-positive with increasing z: the stable
    equilibria of a particle free to move along z (linear interpolation)."""
    zs, Fz = np.asarray(zs, dtype=np.float64), np.asarray(Fz, dtype=np.float64)
    i = np.nonzero((Fz[:-1] > 0.0) & (Fz[1:] <= 0.0))[0]
    return zs[i] + Fz[i] / (Fz[i] - Fz[i + 1]) * (zs[i + 1] - zs[i])


def contact_angle(g: float, rho_hi: float, rho_lo: float, kappa_sum: float, ratios, lz: int = 32,
                  relax_steps: int = 3000, dz: float = 0.02, fluid=None, tension=None):
    """The analysis of Sec. 4.1 on the upper interface of a relaxed slab (A below, B above,
    at z_int near 3 lz / 4 - 1/2).  For each relative coupling difference r = 2 (kappa_A -
    kappa_B) / (kappa_A + kappa_B) the holding force is sampled every dz across the interface
    and its stable zero nearest z_int gives the equilibrium distance d = z_eq - z_int (d > 0
    into B; None: no zero within the interface, the particle detaches into its preferred bulk).
    F_D is the largest holding force at kappa_A = kappa_B = kappa_sum / 2 (the theta = pi / 2
    reference), gamma_AB that of laplace_tension at the same g and densities, R_eff = F_D /
    (pi gamma_AB) and cos(theta) = d / R_eff.  `fluid` = (f, rho_A, rho_B) and `tension`
    reuse a relaxed interface and a measured tension."""
    t0 = time.perf_counter()
    f, a, b = fluid if fluid is not None else relaxed_interface((2, 2, lz), g, rho_hi, rho_lo, steps=relax_steps)
    z_int = interface_height(a, b, 3 * lz / 4 - 4, 3 * lz / 4 + 3)
    zs = np.arange(lz / 2, lz - 0.5 * dz, dz)
    probes = np.column_stack([np.full_like(zs, 0.5), np.full_like(zs, 0.5), zs])
    near = np.abs(zs - z_int) < lz / 8
    d, profiles = [], {}
    for r, kap in zip(ratios, coupling_pairs(kappa_sum, ratios)):
        Fz = holding_forces(f, g, kap, probes)[:, 2]
        profiles[r] = Fz
        roots = [z for z in stable_zeros(zs, Fz) if abs(z - z_int) < lz / 8]
        d.append(min(roots, key=lambda z: abs(z - z_int)) - z_int if roots else None)
    F0 = holding_forces(f, g, (0.5 * kappa_sum, 0.5 * kappa_sum), probes)[:, 2]
    F_D = float(np.abs(F0[near]).max())
    if tension is None:
        tension = laplace_tension(g, rho_hi, rho_lo)[0]
    R_eff = F_D / (np.pi * tension)
    cos = [None if x is None else x / R_eff for x in d]
    return dict(z_int=z_int, zs=zs, profiles=profiles, ratios=list(ratios), d=d, F_D=F_D, gamma_AB=tension,
                R_eff=R_eff, cos_theta=cos, seconds=time.perf_counter() - t0)


def dispersion_index(x, dims, block: int = 8):
    """Variance over mean of the particle counts in block x block columns of the x-y plane: 1 for
    particles placed independently, growing as they gather into domains."""
    nx, ny = dims[0], dims[1]
    c, _, _ = np.histogram2d(np.mod(x[:, 0], nx), np.mod(x[:, 1], ny), bins=(nx // block, ny // block),
                             range=[[0, nx], [0, ny]])
    return float(c.var() / c.mean())


def block_correlation(x, rho, dims, block: int = 8):
    """Pearson correlation, over block x block columns, between the particle count and the mean
    fluid density: negative when particle-rich domains are fluid-poor."""
    nx, ny = dims[0], dims[1]
    c, _, _ = np.histogram2d(np.mod(x[:, 1], ny), np.mod(x[:, 0], nx), bins=(ny // block, nx // block),
                             range=[[0, ny], [0, nx]])
    r = np.asarray(rho, dtype=np.float64).mean(axis=0).reshape(ny // block, block, nx // block, block).mean(axis=(1, 3))
    if c.std() == 0.0 or r.std() == 0.0:
        return float("nan")  # a uniform field has no correlation
    return float(np.corrcoef(c.ravel(), r.ravel())[0, 1])


def particle_fluid_demixing(dims, rho0: float, n: int, kappa: float, lam: float, kT: float, steps: int,
                            every: int, eps: float, sigma: float, gamma: float = 1.0, mass: float = 10.0,
                            seed: int = 0):
    """The single-fluid example of Sec. 3: a uniform fluid (both components identical and
    uncoupled, g = 0, so that they act as one fluid of density 2 rho0) and n particles with
    kappa_A = kappa_B = kappa and lambda_A = lambda_B = lam, WCA (eps, sigma) between them,
    friction gamma and noise at k_BT.  Every `every` steps the dispersion index of the particle
    counts and their block correlation with the fluid density are recorded.  Returns
    {"step", "dispersion", "correlation", "rho_min", "x", "rho"} and the wall time."""
    t0 = time.perf_counter()
    nx, ny, nz = dims
    x = inputs.random_particles(n, dims, sigma, seed=seed)
    if nz == 1:
        x[:, 2] = 0.5
    ctx = _ctx(dims, 0.0, kT=kT, seed=seed + 1)
    out = dict(step=[], dispersion=[], correlation=[], rho_min=[])
    try:
        L.lbmd_set_types(ctx, [L.lbmd_ptype(kappa, kappa, lam, lam, gamma, mass)],
                         [L.lbmd_pair(0, 0, eps, sigma)])
        L.lbmd_init_fluid(ctx, np.full((nz, ny, nx), rho0, np.float32), np.full((nz, ny, nx), rho0, np.float32))
        L.lbmd_set_particles(ctx, x, np.zeros_like(x), np.zeros(n, dtype=np.int32))
        for k in range(0, steps + 1, every):
            if k:
                L.lbmd_step(ctx, every)
            xs, _, _ = L.lbmd_get_particles(ctx, n)
            a, b, _ = L.lbmd_get_fields(ctx, (nz, ny, nx), want_u=False)
            rho = a.astype(np.float64) + b
            out["step"].append(k)
            out["dispersion"].append(dispersion_index(xs, dims))
            out["correlation"].append(block_correlation(xs, rho, dims))
            out["rho_min"].append(float(rho.min()))
        out["x"], out["rho"] = xs, rho
    finally:
        L.lbmd_destroy(ctx)
    out["seconds"] = time.perf_counter() - t0
    return out
