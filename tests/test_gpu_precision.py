"""Reduced-precision population storage against the FP64 oracle.

Populations stored as FP16 or BF16 values shifted by w_i rho0_z (rho0 = mean density), the
rest population in FP32 absorbing each node's rounding, all arithmetic in FP32.  The
systems use the density scale of the paper's examples (rho ~ 78 per component,
g rho = 1.2-1.68).  The bounds are the stated errors of each storage (measured values in
the design notes), not parity: 16-bit rounding is far above the FP32 tolerance.
"""
import functools

import numpy as np
import pytest

from paper_1306_0788_gb300 import inputs

from gpu_common import Case, pop_error, run_oracle

pytestmark = pytest.mark.gpu

CS2 = 1.0 / 3.0
SCALE = 78.4
STORAGES = {"fp32": 0, "fp16": 1, "bf16": 2}
# stated bounds per storage: 10-step population error, 3000-step mass drift, Laplace dp error.
# The 16-bit rounding is systematic near a steady state, so its Laplace error depends on where
# the droplet's values fall between representable numbers: measured over R = 6, 7, 8, 9 it is
# 1.3-1.6e-4 (FP32), 0.4-1.2 % (FP16) and 1.6-19 % (BF16, 8 significant bits).  The FP32 rest
# population closes each node's mass, so the 16-bit drift (7e-7 to 8e-5) stays within FP32's.
# Particle MSD over 1000 steps (the particles' noise is the same on both sides, so the fluid's
# rounding is all that separates them): measured 7.5e-8 (FP32), 7.1e-8 (FP16), 9.2e-7 (BF16).
BOUNDS = {
    "fp32": dict(pop10=1e-5, drift=2e-4, dp=1e-3, msd=1e-6),
    "fp16": dict(pop10=2e-5, drift=3e-4, dp=0.04, msd=1e-6),
    "bf16": dict(pop10=1e-4, drift=3e-4, dp=0.25, msd=1e-5),
}


def _gpu(c, nsteps, storage, rho0):
    from paper_1306_0788_gb300 import lbmd as L
    ctx, _ = L.lbmd_create(L.params(c.dims, tau_r=c.tau_r, g_AB=c.g, storage=STORAGES[storage], rho0=rho0))
    try:
        L.lbmd_set_types(ctx, [L.lbmd_ptype(0, 0, 0, 0, 1, 1)], [])
        a, b, u = c.fields32()
        L.lbmd_init_fluid(ctx, a, b, u)
        d0 = L.lbmd_diagnostics(ctx)
        L.lbmd_step(ctx, nsteps)
        L.lbmd_sync(ctx)
        d1 = L.lbmd_diagnostics(ctx)
        f = np.stack([L.lbmd_get_populations(ctx, 0, c.shape), L.lbmd_get_populations(ctx, 1, c.shape)])
    finally:
        L.lbmd_destroy(ctx)
    return f.astype(np.float64), max(abs(d1[0] / d0[0] - 1), abs(d1[1] / d0[1] - 1))


@pytest.mark.parametrize("storage", sorted(STORAGES))
def test_ten_step_populations(storage):
    dims = (16, 12, 10)
    rA, rB = inputs.uniform_noise(dims, SCALE, 0.01 * SCALE, seed=3)
    c = Case(dims=dims, g=1.68 / SCALE, rhoA=rA, rhoB=rB)
    fo, *_ = run_oracle(c, 10)
    fg, _ = _gpu(c, 10, storage, (SCALE, SCALE))
    err = pop_error(fg, fo)
    print("populations 10 steps", storage, err)
    assert err <= BOUNDS[storage]["pop10"]


@functools.lru_cache(maxsize=None)
def _oracle_droplet(radius):
    """The oracle's droplet after 3000 steps (shared by the three storages)."""
    dims = (32, 32, 1)
    rA, rB = inputs.disk(dims, radius, 1.8 * SCALE, 0.2 * SCALE, width=1.0)
    fo, *_ = run_oracle(Case(dims=dims, g=1.68 / SCALE, rhoA=rA, rhoB=rB), 3000)
    return fo


@pytest.mark.parametrize("radius", [6.0, 7.0, 8.0, 9.0])
@pytest.mark.parametrize("storage", sorted(STORAGES))
def test_laplace_pressure_and_mass_drift(storage, radius):
    """Quasi-2D A-rich droplet (R = 6-9, 32 x 32 x 1) relaxed for 3000 steps: the Laplace
    pressure jump p(centre) - p(far) with p = c_s^2 (rho_A + rho_B) + c_s^2 g rho_A rho_B,
    against the FP64 oracle; mass drift of each component from the FP64 diagnostics."""
    g = 1.68 / SCALE
    dims = (32, 32, 1)
    rA, rB = inputs.disk(dims, radius, 1.8 * SCALE, 0.2 * SCALE, width=1.0)
    c = Case(dims=dims, g=g, rhoA=rA, rhoB=rB)
    fo = _oracle_droplet(radius)

    def dp(f):
        A, B = f[0].sum(0)[0], f[1].sum(0)[0]
        p = CS2 * (A + B) + CS2 * g * A * B
        return p[16, 16] - p[0, 0]

    fg, drift = _gpu(c, 3000, storage, (float(rA.mean()), float(rB.mean())))
    print("laplace quasi-2d", storage, radius, "dp error", abs(dp(fg) - dp(fo)) / abs(dp(fo)), "mass drift", drift)
    assert abs(dp(fg) - dp(fo)) <= BOUNDS[storage]["dp"] * abs(dp(fo))
    assert drift <= BOUNDS[storage]["drift"]


MSD_TIMES = (100, 200, 500, 1000)


def _unwrapped_track(step_fn, x0, dims, times):
    """Positions read after each interval, unwrapped by the minimum image of each interval's
    displacement (intervals of 100 steps move a particle far less than half the box)."""
    L = np.asarray(dims, dtype=np.float64)
    prev, disp, out, t = x0.copy(), np.zeros_like(x0), {}, 0
    for T in times:
        while t < T:
            x = step_fn(100)
            d = x - prev
            disp += d - L * np.round(d / L)
            prev, t = x, t + 100
        out[T] = float((disp ** 2).sum(1).mean())
    return out


def _msd_case():
    dims = (16, 16, 16)
    rA, rB = inputs.uniform_noise(dims, SCALE, 0.01 * SCALE, seed=5)
    x = inputs.random_particles(100, dims, 2 ** (1 / 6), seed=6)
    return Case(dims=dims, g=0.5 / SCALE, kT=0.01, seed=11, rhoA=rA, rhoB=rB, x=x, v=np.zeros_like(x),
                ptype=np.zeros(len(x), dtype=np.int32), types=[(0.0, 0.0, 0.0, 0.0, 1.0, 200.0)])


@functools.lru_cache(maxsize=None)
def _oracle_msd():
    import oracle
    from gpu_common import oracle_system
    c = _msd_case()
    a, b, _ = c.fields32()
    f = oracle.init_equilibrium(a.astype(np.float64), b.astype(np.float64))
    x, v = c.x.copy(), c.v.copy()
    s = oracle_system(c)
    state = {"k": 0}

    def step(n):
        for _ in range(n):
            assert oracle.step(s, f, x, v, state["k"])[0] == 0
            state["k"] += 1
        return x.copy()

    return _unwrapped_track(step, c.x, c.dims, MSD_TIMES)


@pytest.mark.parametrize("storage", sorted(STORAGES))
def test_particle_msd(storage):
    """Mean-square displacement of 100 thermal particles (k_BT = 0.01, gamma = 1, m = 200, friction
    noise from the same counter-based generator on both sides) in a stable mixture at the paper's
    density scale, 16^3, over 1000 steps: each storage against the FP64 oracle."""
    from paper_1306_0788_gb300 import lbmd as L
    c = _msd_case()
    rA, rB, _ = c.fields32()
    ctx, _ = L.lbmd_create(L.params(c.dims, tau_r=c.tau_r, g_AB=c.g, kT=c.kT, seed=c.seed,
                                    storage=STORAGES[storage], rho0=(float(rA.mean()), float(rB.mean()))))
    try:
        L.lbmd_set_types(ctx, [L.lbmd_ptype(*t) for t in c.types], [])
        L.lbmd_init_fluid(ctx, rA, rB)
        L.lbmd_set_particles(ctx, c.x, c.v, c.ptype)

        def step(n):
            L.lbmd_step(ctx, n)
            return L.lbmd_get_particles(ctx, c.n)[0]

        msd_g = _unwrapped_track(step, c.x, c.dims, MSD_TIMES)
    finally:
        L.lbmd_destroy(ctx)
    msd_o = _oracle_msd()
    errs = {t: abs(msd_g[t] / msd_o[t] - 1) for t in MSD_TIMES}
    print("MSD", storage, {t: (round(msd_o[t], 4), float("%.3e" % errs[t])) for t in MSD_TIMES})
    assert max(errs.values()) <= BOUNDS[storage]["msd"]


# ------------------------------------------------------------------ interface position, 3-D Laplace

def _crossings(rhoA, rhoB):
    """Zero crossings of rho_A - rho_B along z (reading 12: the interface is the locus rho_A =
    rho_B), the profile averaged over x and y, linearly interpolated between nodes (node k at
    z = k); sorted."""
    d = (rhoA - rhoB).mean(axis=(1, 2))
    n = len(d)
    out = []
    for k in range(n):
        a, b = d[k], d[(k + 1) % n]
        if (a < 0 <= b) or (a >= 0 > b):
            out.append(k + a / (a - b))
    return np.array(sorted(out))


IFACE_DIMS = (8, 8, 64)
IFACE_TIMES = (500, 1000, 2000)
# stated interface-position errors (lattice units) against the FP64 oracle.  BF16's 8
# significant bits round the shifted populations at this density scale (values up to ~60 w_i)
# by ~0.4 %, systematically near a steady state: while the bulk densities relax the error of its
# interfaces grows to 0.27 (500 steps), 0.50 (1000) and 1.6 lattice units (2000 steps, one GB300
# run) -- BF16 storage does not resolve this slow relaxation.  FP16's grows the same way, to
# 0.001, 0.03 and 0.18 lattice units: the rounding of a 16-bit population is the same from step
# to step near a steady state, so it biases the slow diffusive relaxation of the bulk densities.
IFACE_BOUNDS = {"fp32": 1e-3, "fp16": 0.5, "bf16": 2.5}


def _iface_fields():
    # an A-rich slab off coexistence (1.6 / 0.25 of the density scale instead of 1.9103 /
    # 0.0897): the bulk densities relax and both interfaces travel by ~0.2 lattice units and
    # back over 3000 steps, so the positions compared are the dynamics' result
    return inputs.slab_between(IFACE_DIMS, 15.3, 43.8, 1.6 * SCALE, 0.25 * SCALE, 2.0)


@functools.lru_cache(maxsize=None)
def _oracle_interfaces():
    import oracle
    from gpu_common import oracle_system
    rA, rB = _iface_fields()
    c = Case(dims=IFACE_DIMS, g=1.68 / SCALE, rhoA=rA, rhoB=rB)
    a, b, _ = c.fields32()
    f = oracle.init_equilibrium(a.astype(np.float64), b.astype(np.float64))
    s = oracle_system(c)
    x = np.zeros((0, 3))
    out, k = {}, 0
    for T in IFACE_TIMES:
        while k < T:
            assert oracle.step(s, f, x, x.copy(), k)[0] == 0
            k += 1
        out[T] = _crossings(f[0].sum(0), f[1].sum(0))
    return out


@pytest.mark.parametrize("storage", sorted(STORAGES))
def test_interface_position(storage):
    """Flat interfaces of an A-rich slab relaxing from off-coexistence densities (8 x 8 x 64,
    g rho = 1.68 at the paper's density scale): the two zero crossings of rho_A - rho_B after
    500, 1000 and 2000 steps against the FP64 oracle's."""
    from paper_1306_0788_gb300 import lbmd as L
    rA, rB = _iface_fields()
    c = Case(dims=IFACE_DIMS, g=1.68 / SCALE, rhoA=rA, rhoB=rB)
    a, b, _ = c.fields32()
    want = _oracle_interfaces()
    ctx, _ = L.lbmd_create(L.params(c.dims, tau_r=1.0, g_AB=c.g, storage=STORAGES[storage],
                                    rho0=(float(a.mean()), float(b.mean()))))
    errs = {}
    try:
        L.lbmd_init_fluid(ctx, a, b)
        k = 0
        for T in IFACE_TIMES:
            L.lbmd_step(ctx, T - k)
            k = T
            gA, gB, _ = L.lbmd_get_fields(ctx, c.shape, want_u=False)
            got = _crossings(gA.astype(np.float64), gB.astype(np.float64))
            assert len(got) == len(want[T]) == 2
            errs[T] = float(np.abs(got - want[T]).max())
    finally:
        L.lbmd_destroy(ctx)
    moved = float(np.abs(want[1000] - np.array([15.3, 43.8])).max())
    print("interface", storage, "oracle", {T: want[T].round(4).tolist() for T in IFACE_TIMES}, "errors", errs)
    assert moved > 0.05  # the interfaces did travel
    assert max(errs.values()) <= IFACE_BOUNDS[storage]


def _laplace_golden():
    import json
    import os
    p = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "laplace_droplets_64.json")
    return json.load(open(p))


# stated Laplace pressure-jump errors of 3-D droplets (relative) against the FP64 oracle: the
# jump of each droplet and the fitted 2 gamma.  BF16 (one GB300 run): 20 %, 15 %, 13 % for R = 8,
# 12, 16 and 45 % on 2 gamma -- its 8 significant bits do not resolve pressure jumps at this
# density scale.
LAPLACE3D_BOUNDS = {"fp32": dict(dp=1e-3, gamma=1e-3), "fp16": dict(dp=0.05, gamma=0.1),
                    "bf16": dict(dp=0.3, gamma=0.6)}


@pytest.mark.parametrize("storage", sorted(STORAGES))
def test_laplace_pressure_of_3d_droplets(storage):
    """A-rich spheres of R = 8, 12, 16 on 64^3 at the paper's density scale, 1000 steps: the
    pressure jump (reading 13) of each storage against the FP64 oracle's (stored by
    tests/golden/make_laplace_droplets_64.py, which calls only the oracle), and the fitted
    2 gamma of dp = 2 gamma / R (Laplace law, Sec. 4.3) against the oracle's fit."""
    from paper_1306_0788_gb300 import lbmd as L
    gold = _laplace_golden()
    n, scale, g = gold["lattice"], gold["scale"], gold["g"]
    dims = (n, n, n)
    dps = []
    for R in gold["radii"]:
        rA, rB = inputs.sphere(dims, R, 1.9103 * scale, 0.0897 * scale, gold["width"])
        a, b = rA.astype(np.float32), rB.astype(np.float32)
        ctx, _ = L.lbmd_create(L.params(dims, tau_r=1.0, g_AB=g, storage=STORAGES[storage],
                                        rho0=(float(a.mean()), float(b.mean()))))
        try:
            L.lbmd_init_fluid(ctx, a, b)
            L.lbmd_step(ctx, gold["steps"])
            A, B, _ = L.lbmd_get_fields(ctx, dims[::-1], want_u=False)
        finally:
            L.lbmd_destroy(ctx)
        A, B = A.astype(np.float64), B.astype(np.float64)
        p = CS2 * (A + B) + CS2 * g * A * B
        dps.append(p[n // 2, n // 2, n // 2] - p[0, 0, 0])
    dps, want = np.array(dps), np.array(gold["dp"])
    errs = np.abs(dps / want - 1)
    slope = np.polyfit(1.0 / np.array(gold["radii"]), dps, 1)[0]
    slope_err = abs(slope / gold["fit"]["two_gamma"] - 1)
    print("laplace 3d", storage, "dp", dps.round(5).tolist(), "oracle", want.round(5).tolist(), "errors",
          errs.tolist(), "2 gamma error", slope_err)
    assert errs.max() <= LAPLACE3D_BOUNDS[storage]["dp"]
    assert slope_err <= LAPLACE3D_BOUNDS[storage]["gamma"]
