"""Parity of the CUDA path (through the C ABI) with the FP64 oracle.

Tolerances: populations ||f_gpu - f_ref||_inf / ||f_ref||_inf <= 1e-5 after 10 steps;
particle positions: minimum-image |dx| / max(rms displacement, 1) <= 1e-4 after 100 steps.
"""
import numpy as np
import pytest

import oracle
from paper_1306_0788_gb300 import inputs

from gpu_common import Case, make_gpu, noisy_fluid, pop_error, position_error, run_gpu, run_oracle

pytestmark = pytest.mark.gpu

POP_TOL = 1e-5
POS_TOL = 1e-4


def L():
    from paper_1306_0788_gb300 import lbmd
    return lbmd


# ------------------------------------------------------------------ fluid only
@pytest.mark.parametrize("nsteps", [1, 10])
def test_fluid_4cubed_every_population(nsteps):
    dims = (4, 4, 4)
    rA, rB = noisy_fluid(dims, amp=0.05, seed=3)
    c = Case(dims=dims, g=1.68, rhoA=rA, rhoB=rB)
    fg, *_ = run_gpu(c, nsteps)
    fo, *_ = run_oracle(c, nsteps)
    assert pop_error(fg, fo) <= POP_TOL


@pytest.mark.parametrize("dims,tau", [((5, 7, 9), 0.8), ((33, 17, 6), 1.3), ((1, 16, 12), 1.0), ((2, 3, 5), 0.7)])
def test_fluid_ragged_sizes(dims, tau):
    rA, rB = noisy_fluid(dims, amp=0.03, seed=11)
    u = np.random.default_rng(2).uniform(-0.02, 0.02, size=dims[::-1] + (3,))
    c = Case(dims=dims, tau_r=tau, g=1.4, rhoA=rA, rhoB=rB, u=u)
    fg, *_ = run_gpu(c, 10)
    fo, *_ = run_oracle(c, 10)
    assert pop_error(fg, fo) <= POP_TOL


def test_fields_readback():
    dims = (6, 5, 7)
    rA, rB = noisy_fluid(dims, amp=0.05, seed=4)
    c = Case(dims=dims, g=1.5, rhoA=rA, rhoB=rB)
    fo, *_ = run_oracle(c, 3)
    ctx = make_gpu(c)
    try:
        L().lbmd_step(ctx, 3)
        a, b, u = L().lbmd_get_fields(ctx, c.shape)
    finally:
        L().lbmd_destroy(ctx)
    ra, rb = fo[0].sum(0), fo[1].sum(0)
    assert np.abs(a - ra).max() < 1e-5 and np.abs(b - rb).max() < 1e-5
    cvec, _ = oracle.lattice()
    j = np.einsum("zinyx,ia->nyxa", fo, cvec.astype(float))
    gA, gB, _, _ = oracle.sc_force(ra, rb, 1.5, 1.5)
    uo = (j + 0.5 * (gA + gB)) / (ra + rb)[..., None]
    assert np.abs(u - uo).max() < 1e-6


# ------------------------------------------------------------------ coupled
def config1_case(npart=64, kT=0.0, steps_seed=1):
    """32^3, rho_A, rho_B = 1 +- 0.01, tau = 1, g = 1.68 (above the demixing threshold),
    point particles friction-coupled (gamma = 1) with WCA (eps = 1, sigma = 1)."""
    dims = (32, 32, 32)
    rA, rB = noisy_fluid(dims, amp=0.01, seed=1234 + steps_seed)
    x = inputs.random_particles(npart, dims, 1.5, seed=99)
    return Case(dims=dims, g=1.68, kT=kT, rhoA=rA, rhoB=rB, x=x, v=np.zeros((npart, 3)),
                ptype=np.zeros(npart, dtype=np.int32), wca={(0, 0): (1.0, 1.0)})


def test_config1_populations_10_steps():
    c = config1_case()
    fg, xg, _, _ = run_gpu(c, 10)
    fo, xo, _, _ = run_oracle(c, 10)
    assert pop_error(fg, fo) <= POP_TOL
    assert position_error(xg, xo, c.x, c.dims) <= POS_TOL


def coupled_case(dims, npart, seed, g=0.8, kT=0.0, min_dist=2.0):
    """All couplings on, gentle enough for long parity runs: g below the threshold keeps the
    fluid stable; two particle types with opposite solvation preferences."""
    rA, rB = noisy_fluid(dims, amp=0.02, seed=seed)
    x = inputs.random_particles(npart, dims, min_dist, seed=seed + 1)
    v = np.random.default_rng(seed).normal(scale=0.02, size=(npart, 3))
    ptype = (np.arange(npart) % 2).astype(np.int32)
    q = np.where(np.arange(npart) % 4 < 2, 1.0, -1.0)
    types = [(-0.05, 0.02, 0.004, -0.002, 0.5, 1.0), (0.03, -0.04, 0.0, 0.003, 0.8, 2.0)]
    return Case(dims=dims, g=g, kT=kT, seed=seed, rhoA=rA, rhoB=rB, x=x, v=v, ptype=ptype, q=q, types=types,
                wca={(0, 0): (0.01, 1.0), (0, 1): (0.01, 0.9), (1, 1): (0.01, 0.8)}, dh=(0.02, 0.25, 2.5))


@pytest.mark.parametrize("kT", [0.0, 0.002])
def test_particles_100_steps(kT):
    """100 coupled steps, positions within 1e-4 of the oracle's.  The thermal case runs at kT =
    0.002 with particles at least 2.5 apart: at kT = 0.005 and 2.0 apart two particles meet in a
    WCA contact near step 68, the explicit update (dt = 1, m = 1) throws one of them at 10.7 lattice
    units per step, and the FP64 oracle's own densities go negative at step 72 -- the system
    leaves the model's stability range (Sec. 3: gamma dt / m << 1), after which FP32 and FP64
    trajectories part by chaos, not by error."""
    c = coupled_case((20, 18, 16), 30, seed=21, kT=kT, min_dist=2.5)
    fg, xg, vg, _ = run_gpu(c, 100)
    fo, xo, vo, _ = run_oracle(c, 100)
    assert position_error(xg, xo, c.x, c.dims) <= POS_TOL
    assert pop_error(fg, fo) <= 1e-4  # 100 steps: looser than the 10-step population bar


def test_coupled_10_steps_populations_and_forces():
    c = coupled_case((12, 10, 14), 24, seed=5, g=1.3, kT=0.01)
    fg, xg, vg, Fg = run_gpu(c, 10)
    fo, xo, vo, tr = run_oracle(c, 10, trace_last=True)
    assert pop_error(fg, fo) <= POP_TOL
    assert position_error(xg, xo, c.x, c.dims) <= POS_TOL
    Fo = tr["f_total"]
    assert np.abs(Fg - Fo).max() <= 1e-4 * max(np.abs(Fo).max(), 1e-3)


def test_dense_pairs_bonds_and_cell_list():
    """Short-range forces through the GPU cell list against the oracle's brute-force sum:
    WCA and screened Coulomb in a crowded box, FENE chains."""
    dims = (10, 9, 8)
    rA = np.ones(dims[::-1])
    rB = np.ones(dims[::-1])
    n_chains, length = 12, 8
    pos, bonds, q = inputs.bead_spring_chains(n_chains, length, dims, bond=0.97, seed=3)
    n = len(pos)
    c = Case(dims=dims, rhoA=rA, rhoB=rB, x=pos, v=np.zeros((n, 3)), ptype=np.zeros(n, dtype=np.int32), q=q,
             types=[(0.0, 0.0, 0.0, 0.0, 0.0, 1.0)], wca={(0, 0): (1.0, 1.0)}, dh=(1.0, 0.25, 3.0),
             bonds=bonds, bond_kind=2, bond_k=30.0, bond_r=1.5)
    fg, xg, vg, Fg = run_gpu(c, 1)
    fo, xo, vo, tr = run_oracle(c, 1, trace_last=True)
    Fo = tr["f_total"]
    assert np.abs(Fg - Fo).max() <= 1e-5 * np.abs(Fo).max()
    assert np.abs(Fg.sum(0)).max() <= 1e-4 * np.abs(Fo).max()


def test_noise_stream_matches_oracle():
    """Counter-based noise: the same Philox4x32-10 stream on both sides.  Fluid at rest,
    particles at rest, gamma = 1: the first-step force is the noise itself."""
    dims = (8, 8, 8)
    n = 50
    x = inputs.random_particles(n, dims, 0.5, seed=4)
    c = Case(dims=dims, kT=0.7, seed=123456789012345, rhoA=np.ones(dims[::-1]), rhoB=np.ones(dims[::-1]), x=x,
             v=np.zeros((n, 3)), ptype=np.zeros(n, dtype=np.int32))
    _, _, _, Fg = run_gpu(c, 1)
    _, _, _, tr = run_oracle(c, 1, trace_last=True)
    assert np.abs(Fg - tr["f_total"]).max() <= 1e-5 * np.abs(tr["f_total"]).max()


@pytest.mark.parametrize("pos", [
    [[2.5, 3.0, 4.0]],            # on a face and on lattice lines (exact Theta cases)
    [[0.0, 0.0, 0.0]],            # on a node at the box corner
    [[3.25, 3.25, 3.25]],         # on a body diagonal of its cell corner
    [[5.999999, 0.0000001, 2.5]],  # next to the upper box edge
])
def test_degenerate_positions(pos):
    dims = (6, 6, 6)
    rA, rB = noisy_fluid(dims, amp=0.02, seed=8)
    x = np.array(pos, dtype=np.float64)
    n = len(x)
    c = Case(dims=dims, g=1.1, rhoA=rA, rhoB=rB, x=x, v=np.full((n, 3), 0.01), ptype=np.zeros(n, dtype=np.int32),
             types=[(0.1, -0.1, 0.05, -0.03, 0.7, 1.0)])
    fg, xg, _, _ = run_gpu(c, 3)
    fo, xo, _, _ = run_oracle(c, 3)
    assert pop_error(fg, fo) <= POP_TOL
    assert position_error(xg, xo, c.x, c.dims) <= POS_TOL


def test_thin_lattices_with_particles():
    """nx = 1 and 2-wide lattices: a node is several corners of the same cell."""
    for dims in [(1, 12, 10), (2, 6, 5)]:
        rA, rB = noisy_fluid(dims, amp=0.02, seed=9)
        n = 5
        x = inputs.random_particles(n, dims, 0.0, seed=10)
        c = Case(dims=dims, g=1.2, rhoA=rA, rhoB=rB, x=x, v=np.zeros((n, 3)), ptype=np.zeros(n, dtype=np.int32),
                 types=[(0.05, -0.05, 0.01, 0.02, 0.6, 1.0)])
        fg, xg, _, _ = run_gpu(c, 5)
        fo, xo, _, _ = run_oracle(c, 5)
        assert pop_error(fg, fo) <= POP_TOL, dims
        assert position_error(xg, xo, c.x, c.dims) <= POS_TOL, dims


# ------------------------------------------------------------------ invariants on device
def test_fp64_diagnostics_conservation():
    c = coupled_case((24, 24, 24), 60, seed=31, g=1.3, kT=0.01)
    ctx = make_gpu(c)
    try:
        d0 = L().lbmd_diagnostics(ctx)
        L().lbmd_step(ctx, 50)
        d1 = L().lbmd_diagnostics(ctx)
    finally:
        L().lbmd_destroy(ctx)
    fo = oracle.init_equilibrium(*[a.astype(np.float32).astype(np.float64) for a in (c.rhoA, c.rhoB)])
    mo = oracle.fluid_moments(fo)
    assert np.allclose(d0[:2], mo[:2], rtol=1e-6)
    assert abs(d1[0] / d0[0] - 1) < 1e-6 and abs(d1[1] / d0[1] - 1) < 1e-6
    P0 = d0[2:5] + d0[5:8]
    P1 = d1[2:5] + d1[5:8]
    assert np.abs(P1 - P0).max() < 1e-3 * max(np.abs(d1[5:8]).max(), np.abs(d1[2:5] - d0[2:5]).max(), 1e-3)


def test_negative_density_is_reported_not_faulted():
    """Sec. 3: large lambda depletes the nodes next to a particle until densities turn
    negative.  The kernel records it in the device error word; the host reports it."""
    dims = (6, 6, 6)
    c = Case(dims=dims, rhoA=np.ones(dims[::-1]), rhoB=np.ones(dims[::-1]), x=np.array([[2.3, 2.6, 2.4]]),
             v=np.zeros((1, 3)), ptype=np.zeros(1, dtype=np.int32), types=[(0.0, 0.0, 50.0, 50.0, 0.0, 1.0)])
    ctx = make_gpu(c)
    try:
        L().lbmd_step(ctx, 3)
        with pytest.raises(L().LbmdError) as e:
            L().lbmd_sync(ctx)
        assert e.value.code in (L().LBMD_E_NEGATIVE_DENSITY, L().LBMD_E_NONFINITE)
        L().lbmd_clear_error(ctx)
        L().lbmd_sync(ctx)
    finally:
        L().lbmd_destroy(ctx)


def test_particles_can_be_removed_and_resized():
    c = config1_case(npart=16)
    ctx = make_gpu(c)
    try:
        L().lbmd_step(ctx, 2)
        L().lbmd_set_particles(ctx, np.zeros((0, 3)), np.zeros((0, 3)), np.zeros(0, dtype=np.int32))
        L().lbmd_step(ctx, 2)
        x = inputs.random_particles(40, c.dims, 1.5, seed=3)
        L().lbmd_set_particles(ctx, x, np.zeros((40, 3)), np.zeros(40, dtype=np.int32))
        L().lbmd_step(ctx, 2)
        xg, _, _ = L().lbmd_get_particles(ctx, 40)
        assert np.isfinite(xg).all()
    finally:
        L().lbmd_destroy(ctx)


# ------------------------------------------------------------------ full size
def test_full_size_256_tiled_against_16_oracle():
    """At the 256^3 size the bench runs, in the same launch configuration (the one-pass update,
    replayed step graphs): a state that is
    periodic with period 16 in every direction (a 16^3 system tiled 16 times per axis, its
    particles replicated -- 16384 particles) evolves exactly like the 16^3 system.  Sampled
    tiles of the GPU result are compared with the 16^3 oracle."""
    small = (16, 16, 16)
    rA, rB = noisy_fluid(small, amp=0.02, seed=77)
    n0 = 4
    x0 = inputs.random_particles(n0, small, 3.0, seed=78)
    types = [(-0.1, 0.05, 0.002, 0.0, 1.0, 1.0)]
    cs = Case(dims=small, g=1.68, rhoA=rA, rhoB=rB, x=x0, v=np.zeros((n0, 3)), ptype=np.zeros(n0, dtype=np.int32),
              types=types, wca={(0, 0): (1.0, 1.0)})
    fo, xo, _, _ = run_oracle(cs, 2)
    R = 16
    big = (256, 256, 256)
    shifts = np.array([(i, j, k) for k in range(R) for j in range(R) for i in range(R)], dtype=np.float64) * 16
    xb = (x0[None, :, :] + shifts[:, None, :]).reshape(-1, 3)
    nb = len(xb)
    cb = Case(dims=big, g=1.68, rhoA=np.tile(rA, (R, R, R)), rhoB=np.tile(rB, (R, R, R)), x=xb,
              v=np.zeros((nb, 3)), ptype=np.zeros(nb, dtype=np.int32), types=types, wca={(0, 0): (1.0, 1.0)})
    ctx = make_gpu(cb)
    try:
        assert L().lbmd_get_lattice_passes(ctx) == 1  # the bench's update at this size
        L().lbmd_step(ctx, 2)
        L().lbmd_sync(ctx)
        fa = L().lbmd_get_populations(ctx, 0, cb.shape)
        fbb = L().lbmd_get_populations(ctx, 1, cb.shape)
        xg, _, _ = L().lbmd_get_particles(ctx, nb)
    finally:
        L().lbmd_destroy(ctx)
    rng = np.random.default_rng(0)
    for (i, j, k) in [(0, 0, 0), (15, 15, 15)] + [tuple(t) for t in rng.integers(0, R, size=(6, 3))]:
        sl = (slice(None), slice(16 * k, 16 * k + 16), slice(16 * j, 16 * j + 16), slice(16 * i, 16 * i + 16))
        tile = np.stack([fa[sl], fbb[sl]])
        assert pop_error(tile, fo) <= POP_TOL, (i, j, k)
    xg = xg.reshape(R ** 3, n0, 3) - shifts[:, None, :]
    for t in range(0, R ** 3, 997):
        assert position_error(xg[t], xo, x0, small) <= POS_TOL


def test_single_solvation_force_variant():
    """kappa = 0, lambda != 0 (the per-node momentum-conserving scheme with one solvation
    force): populations and positions against the oracle after 30 steps in an interface."""
    dims = (8, 8, 24)
    rA, rB, _ = inputs.slab_and_droplets(dims, 1.9, 0.1, n_drops=0, width=3.0, seed=1)
    x = inputs.random_particles(12, dims, 2.0, seed=4)
    c = Case(dims=dims, g=1.68, rhoA=rA, rhoB=rB, x=x, v=np.zeros((12, 3)), ptype=np.zeros(12, dtype=np.int32),
             types=[(0.0, 0.0, 0.02, -0.01, 0.2, 5.0)])
    fg, xg, _, _ = run_gpu(c, 30)
    fo, xo, _, _ = run_oracle(c, 30)
    assert pop_error(fg, fo) <= 3e-5
    assert position_error(xg, xo, c.x, c.dims) <= POS_TOL


@pytest.mark.parametrize("bad", [0.0, -1.0, np.inf, -np.inf, np.nan])
def test_invalid_densities_are_refused(bad):
    """A density that is not finite and positive, at any site of either field, is refused with
    LBMD_E_INVALID_ARG by single contexts and batches alike; a valid field is accepted after."""
    from paper_1306_0788_gb300 import lbmd as L
    dims = (9, 7, 5)
    rA, rB = noisy_fluid(dims, amp=0.02, seed=4)
    ctx, _ = L.lbmd_create(L.params(dims))
    b = L.lbmd_batch_create(0, 0, 2)
    try:
        slot, _ = L.lbmd_batch_add(b, L.params(dims), 0, 10)
        for field, site in ((0, 0), (1, dims[0] * dims[1] * dims[2] - 1), (0, 123)):
            a, c = rA.astype(np.float32).copy(), rB.astype(np.float32).copy()
            (a if field == 0 else c).reshape(-1)[site] = bad
            with pytest.raises(L.LbmdError) as e:
                L.lbmd_init_fluid(ctx, a, c)
            assert e.value.code == L.LBMD_E_INVALID_ARG
            with pytest.raises(L.LbmdError) as e:
                L.lbmd_batch_init_fluid(b, slot, a, c)
            assert e.value.code == L.LBMD_E_INVALID_ARG
        L.lbmd_init_fluid(ctx, rA, rB)
        L.lbmd_batch_init_fluid(b, slot, rA, rB)
        L.lbmd_step(ctx, 2)
        L.lbmd_sync(ctx)
    finally:
        L.lbmd_batch_destroy(b)
        L.lbmd_destroy(ctx)
