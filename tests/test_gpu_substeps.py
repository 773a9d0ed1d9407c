"""MD sub-stepping (K particle substeps per lattice step, the fluid frozen within the step)
of the CUDA path against the FP64 oracle, with the parity tolerances (populations 1e-5 after
10 steps, positions 1e-4 after 100 steps)."""
import numpy as np
import pytest

from gpu_common import Case, make_gpu, pop_error, position_error, run_gpu, run_oracle

from test_gpu_parity import coupled_case

pytestmark = pytest.mark.gpu

POP_TOL = 1e-5
POS_TOL = 1e-4


def L():
    from paper_1306_0788_gb300 import lbmd
    return lbmd


@pytest.mark.parametrize("K,collision", [(4, 0), (3, 1)])
def test_substeps_coupled_10_steps(K, collision):
    c = coupled_case((12, 10, 14), 24, seed=5, g=1.3, kT=0.01)
    c.md_substeps, c.collision = K, collision
    fg, xg, vg, Fg = run_gpu(c, 10)
    fo, xo, vo, tr = run_oracle(c, 10, trace_last=True)
    assert pop_error(fg, fo) <= POP_TOL
    assert position_error(xg, xo, c.x, c.dims) <= POS_TOL
    Fo = tr["f_total"]
    assert np.abs(Fg - Fo).max() <= 1e-4 * max(np.abs(Fo).max(), 1e-3)


def test_substeps_100_steps_positions():
    c = coupled_case((20, 18, 16), 30, seed=21, kT=0.002, min_dist=2.5)
    c.md_substeps = 3
    fg, xg, _, _ = run_gpu(c, 100)
    fo, xo, _, _ = run_oracle(c, 100)
    assert position_error(xg, xo, c.x, c.dims) <= POS_TOL
    assert pop_error(fg, fo) <= 1e-4


def _pair_case(K):
    dims = (16, 16, 16)
    return Case(dims=dims, rhoA=np.ones(dims[::-1]), rhoB=np.ones(dims[::-1]),
                x=np.array([[7.0, 8.0, 8.0], [8.0, 8.0, 8.0]]), v=np.zeros((2, 3)), ptype=np.zeros(2, dtype=np.int32),
                types=[(0.0, 0.0, 0.0, 0.0, 0.0, 1.0)], wca={(0, 0): (1.0, 1.0)}, md_substeps=K)


def test_stiff_contact_with_200_substeps_matches_oracle():
    """Two m = 1 particles released at sigma: 200 substeps per lattice step follow the oracle
    and push the pair apart with the energy the WCA force does (about 1 = eps)."""
    c = _pair_case(200)
    _, xg, vg, _ = run_gpu(c, 3)
    _, xo, vo, _ = run_oracle(c, 3)
    assert np.abs(xg - xo).max() < 1e-4
    assert np.abs(vg - vo).max() < 1e-4 * np.abs(vo).max()
    ke = 0.5 * (vg * vg).sum()
    assert abs(ke - 1.0) < 0.03


def test_particle_leaving_its_neighbourhood_is_reported():
    """With substeps the cell list of the step assumes that no particle moves more than one
    cell: a particle at 2.5 cells per step is reported, and the state stays readable."""
    dims = (16, 16, 16)
    c = Case(dims=dims, rhoA=np.ones(dims[::-1]), rhoB=np.ones(dims[::-1]), x=np.array([[4.5, 8.0, 8.0]]),
             v=np.array([[2.5, 0.0, 0.0]]), ptype=np.zeros(1, dtype=np.int32),
             types=[(0.0, 0.0, 0.0, 0.0, 0.0, 1.0)], md_substeps=2)
    ctx = make_gpu(c)
    try:
        L().lbmd_step(ctx, 2)
        with pytest.raises(L().LbmdError) as e:
            L().lbmd_sync(ctx)
        assert e.value.code == L().LBMD_E_PARTICLE_TOO_FAST
        L().lbmd_clear_error(ctx)
        x, _, _ = L().lbmd_get_particles(ctx, 1)
        assert np.isfinite(x).all() and (x >= 0).all() and (x < 16).all()
    finally:
        L().lbmd_destroy(ctx)


def test_batches_take_one_substep_only():
    lb = L()
    b = lb.lbmd_batch_create(0, 0, 2)
    try:
        with pytest.raises(lb.LbmdError) as e:
            lb.lbmd_batch_add(b, lb.params((8, 8, 8), md_substeps=2), 0, 5)
        assert e.value.code == lb.LBMD_E_INVALID_ARG
    finally:
        lb.lbmd_batch_destroy(b)
