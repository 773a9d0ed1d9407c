"""The one-pass lattice update (lbmd_set_lattice_passes(ctx, 1)) against the FP64 oracle.

The update of step t also forms the densities of step t + 1 from the post-collision values it
has just computed (streaming carries f*_i(r) to r + c_i), instead of a density pass pulling every
population again; a second kernel finishes the nodes whose sources lie in another block.  These
tests force the one-pass update at sizes the oracle runs in seconds -- ragged tiles along x (32
columns per warp) and y (8 rows per block), lattices narrower than a tile, one-column tiles, tiles
whose edge rows are pulled and tiles whose edge rows come from partial sums -- and hold it to the
same tolerances as the two-pass update:
populations within 1e-5 after 10 steps, positions within 1e-4 after 100 steps; the densities it
forms are checked node by node against the sum of the populations; the two updates agree to
rounding order; graphs replay it bit for bit.  At 256^3 the bench's launch (one pass, chosen by
the size) is covered by test_full_size_256_tiled_against_16_oracle.
"""
import numpy as np
import pytest

from paper_1306_0788_gb300 import inputs

from gpu_common import Case, make_gpu, noisy_fluid, pop_error, position_error, run_gpu, run_oracle

pytestmark = pytest.mark.gpu

POP_TOL = 1e-5
POS_TOL = 1e-4

# tiles of 32 x 8 columns: ragged along x and y, narrower than a tile, one-column tiles (33), tiles
# of 1 or 2 rows (edge rows pulled) and of >= 3 rows and >= 2 columns (edge rows from partial sums:
# (2, 3, 5), (64, 20, 24), (40, 11, 18), (34, 24, 20), (64, 16, 40), (40, 16, 3)); one z-chunk, two
# (24, 30) and three (40); chunk-edge planes from partial sums (nz >= 2: the two planes of nz = 2
# are both chunk-edge planes, each with parts from both ends of the one chunk) or pulled (nz = 1)
SIZES = [(20, 18, 16), (31, 9, 13), (33, 17, 12), (1, 16, 12), (2, 3, 5), (64, 20, 24), (7, 25, 30), (40, 11, 18),
         (34, 24, 20), (64, 16, 40), (20, 9, 2), (33, 11, 1), (40, 16, 3)]


def L():
    from paper_1306_0788_gb300 import lbmd
    return lbmd


@pytest.mark.parametrize("dims", SIZES)
def test_fluid_populations_10_steps(dims):
    rA, rB = noisy_fluid(dims, amp=0.03, seed=11)
    u = np.random.default_rng(2).uniform(-0.02, 0.02, size=dims[::-1] + (3,))
    c = Case(dims=dims, tau_r=0.9, g=1.4, rhoA=rA, rhoB=rB, u=u)
    fg, *_ = run_gpu(c, 10, passes=1)
    fo, *_ = run_oracle(c, 10)
    assert pop_error(fg, fo) <= POP_TOL


@pytest.mark.parametrize("dims", SIZES)
def test_formed_densities_are_the_population_sums(dims):
    """After steps of the one-pass update the densities it keeps (lbmd_get_fields reads them
    without a density pass) equal, node by node, the sums of the populations read back."""
    rA, rB = noisy_fluid(dims, amp=0.05, seed=4)
    c = Case(dims=dims, g=1.5, rhoA=rA, rhoB=rB)
    ctx = make_gpu(c, passes=1)
    try:
        assert L().lbmd_get_lattice_passes(ctx) == 1
        for n in (1, 4):
            L().lbmd_step(ctx, n)
            a, b, _ = L().lbmd_get_fields(ctx, c.shape, want_u=False)
            fA = L().lbmd_get_populations(ctx, 0, c.shape).astype(np.float64).sum(0)
            fB = L().lbmd_get_populations(ctx, 1, c.shape).astype(np.float64).sum(0)
            assert np.abs(a - fA).max() <= 2e-6 * np.abs(fA).max()
            assert np.abs(b - fB).max() <= 2e-6 * np.abs(fB).max()
    finally:
        L().lbmd_destroy(ctx)


def _coupled(dims, npart, seed, kT):
    from test_gpu_parity import coupled_case
    return coupled_case(dims, npart, seed=seed, kT=kT, min_dist=2.5)


def test_coupled_10_steps_populations_forces():
    c = _coupled((20, 18, 16), 30, 21, 0.01)
    fg, xg, _, Fg = run_gpu(c, 10, passes=1)
    fo, xo, _, tr = run_oracle(c, 10, trace_last=True)
    assert pop_error(fg, fo) <= POP_TOL
    assert position_error(xg, xo, c.x, c.dims) <= POS_TOL
    Fo = tr["f_total"]
    assert np.abs(Fg - Fo).max() <= 1e-4 * max(np.abs(Fo).max(), 1e-3)


def test_coupled_across_chunks_and_tile_edges():
    """Three z-chunks (nz = 40), edge rows and chunk-edge planes from partial sums, and 80
    particles: the corner j' of the coupling and the momentum return land on tile edges, chunk-edge
    planes and their corners; 20 coupled steps against the oracle."""
    c = _coupled((40, 16, 40), 80, 31, 0.002)
    fg, xg, _, _ = run_gpu(c, 20, passes=1)
    fo, xo, _, _ = run_oracle(c, 20)
    assert pop_error(fg, fo) <= POP_TOL
    assert position_error(xg, xo, c.x, c.dims) <= POS_TOL


def test_switching_the_lattice_form_mid_run():
    """One pass, then two, then one again on the same context (each switch drops the graphs and the
    one-pass buffers; the densities and corner j' are formed again where needed): the run equals
    the oracle's within the 10-step tolerance after 12 steps."""
    c = _coupled((34, 24, 20), 40, 33, 0.002)
    ctx = make_gpu(c, passes=1)
    try:
        for passes, n in ((1, 4), (2, 4), (1, 4)):
            L().lbmd_set_lattice_passes(ctx, passes)
            L().lbmd_step(ctx, n)
        L().lbmd_sync(ctx)
        fg = np.stack([L().lbmd_get_populations(ctx, 0, c.shape), L().lbmd_get_populations(ctx, 1, c.shape)])
        xg, _, _ = L().lbmd_get_particles(ctx, c.n)
    finally:
        L().lbmd_destroy(ctx)
    fo, xo, _, _ = run_oracle(c, 12)
    assert pop_error(fg, fo) <= POP_TOL
    assert position_error(xg, xo, c.x, c.dims) <= POS_TOL


@pytest.mark.parametrize("kT", [0.0, 0.002])
def test_particles_100_steps(kT):
    c = _coupled((20, 18, 16), 30, 21, kT)
    fg, xg, _, _ = run_gpu(c, 100, passes=1)
    fo, xo, _, _ = run_oracle(c, 100)
    assert position_error(xg, xo, c.x, c.dims) <= POS_TOL
    assert pop_error(fg, fo) <= 1e-4


@pytest.mark.parametrize("storage,tol", [(1, 2e-5), (2, 1e-4)])
def test_16bit_storage_10_steps(storage, tol):
    """FP16 / BF16 shifted storage (rest populations in FP32) at the paper's density scale, within
    the stated 10-step bounds of the two-pass update; with particles."""
    scale = 78.4
    dims = (33, 17, 12)
    rA, rB = inputs.uniform_noise(dims, scale, 0.01 * scale, seed=3)
    x = inputs.random_particles(20, dims, 2.0, seed=4)
    c = Case(dims=dims, g=1.68 / scale, rhoA=rA, rhoB=rB, x=x, v=np.zeros_like(x),
             ptype=np.zeros(len(x), dtype=np.int32), types=[(-0.001, -0.002, 0.0, 0.0, 1.0, 200.0)],
             wca={(0, 0): (1.0, 1.0)}, storage=storage, rho0=(float(rA.mean()), float(rB.mean())))
    fg, *_ = run_gpu(c, 10, passes=1)
    fo, *_ = run_oracle(c, 10)
    assert pop_error(fg, fo) <= tol


def test_one_and_two_passes_agree_and_graphs_replay_bit_for_bit():
    """The two updates give the same step up to rounding order (within 1e-6 after 20 coupled
    steps); the one-pass update replayed as graphs gives the bits of its launches one by one."""
    c = _coupled((33, 17, 12), 24, 5, 0.01)
    out = {}
    for name, passes, graphs in (("two", 2, True), ("one", 1, True), ("one_stream", 1, False)):
        ctx = make_gpu(c, passes=passes)
        try:
            L().lbmd_set_graphs(ctx, graphs)
            L().lbmd_step(ctx, 20)
            f = np.stack([L().lbmd_get_populations(ctx, 0, c.shape), L().lbmd_get_populations(ctx, 1, c.shape)])
            x, v, _ = L().lbmd_get_particles(ctx, c.n)
            out[name] = (f, x, v)
        finally:
            L().lbmd_destroy(ctx)
    for a, b in zip(out["one"], out["one_stream"]):
        assert np.array_equal(a, b)
    assert pop_error(out["one"][0], out["two"][0].astype(np.float64)) <= 1e-6
    assert np.abs(out["one"][1] - out["two"][1]).max() <= 1e-5


def test_setup_allocates_once():
    """The one-pass update's buffers (partial sums, plane table, run list -- empty on this lattice,
    whose every node is finished from partial sums) are set up once per context: many steps, as
    graph replays and as single launches, leave the device's free memory where the first step
    left it."""
    import torch
    c = _coupled((128, 64, 48), 40, 7, 0.0)
    ctx = make_gpu(c, passes=1)
    try:
        L().lbmd_step(ctx, 3)  # set-up, graphs recorded, one single launch
        L().lbmd_sync(ctx)
        free0, _ = torch.cuda.mem_get_info()
        for _ in range(40):
            L().lbmd_step(ctx, 3)
        L().lbmd_sync(ctx)
        free1, _ = torch.cuda.mem_get_info()
        assert free0 - free1 < 4 << 20, (free0, free1)
    finally:
        L().lbmd_destroy(ctx)


def test_mode_choice_and_limits():
    """Small lattices take two passes by default; the one-pass update refuses the fluctuating
    MRT collision and MD sub-stepping."""
    from paper_1306_0788_gb300 import lbmd as Lb
    ctx, _ = Lb.lbmd_create(Lb.params((16, 16, 16), g_AB=1.2))
    try:
        assert Lb.lbmd_get_lattice_passes(ctx) == 2
        Lb.lbmd_set_lattice_passes(ctx, 1)
        assert Lb.lbmd_get_lattice_passes(ctx) == 1
        with pytest.raises(Lb.LbmdError):
            Lb.lbmd_set_lattice_passes(ctx, 3)
    finally:
        Lb.lbmd_destroy(ctx)
    for prm in (Lb.params((16, 16, 16), collision=Lb.LBMD_COLLISION_MRT), Lb.params((16, 16, 16), md_substeps=2)):
        ctx, _ = Lb.lbmd_create(prm)
        try:
            with pytest.raises(Lb.LbmdError) as e:
                Lb.lbmd_set_lattice_passes(ctx, 1)
            assert e.value.code == Lb.LBMD_E_INVALID_ARG
            assert Lb.lbmd_get_lattice_passes(ctx) == 2
        finally:
            Lb.lbmd_destroy(ctx)
