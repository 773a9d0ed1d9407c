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
BOUNDS = {
    "fp32": dict(pop10=1e-5, drift=2e-4, dp=1e-3),
    "fp16": dict(pop10=2e-5, drift=3e-4, dp=0.04),
    "bf16": dict(pop10=1e-4, drift=3e-4, dp=0.25),
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
    assert pop_error(fg, fo) <= BOUNDS[storage]["pop10"]


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
    assert abs(dp(fg) - dp(fo)) <= BOUNDS[storage]["dp"] * abs(dp(fo))
    assert drift <= BOUNDS[storage]["drift"]
