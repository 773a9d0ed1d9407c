"""Batches: many independent replicas advanced in shared launches (continuous batching).

Stated tolerances:
  * a replica's results (populations, positions, velocities, forces, step count) are
    BIT-IDENTICAL alone and in any mix of other replicas, slot positions, join / leave order,
    step chunking and launch shape: the kernels are the same, every site and particle does the
    same arithmetic, and a replica's particles keep their relative order in the shared sort;
  * against the FP64 oracle, the single-lattice tolerances (populations 1e-5 after 10 steps,
    positions 1e-4);
  * against a single context (lbmd_create) running the same system, 1e-6 relative.
"""
import numpy as np
import pytest

from gpu_common import Case, noisy_fluid, pop_error, position_error, run_oracle

from test_gpu_parity import coupled_case, config1_case

pytestmark = pytest.mark.gpu

POP_TOL = 1e-5
POS_TOL = 1e-4


def L():
    from paper_1306_0788_gb300 import lbmd
    return lbmd


def add_case(b, c: Case, total: int, np_max=None, storage=0, rho0=(0.0, 0.0)):
    lb = L()
    slot, _ = lb.lbmd_batch_add(b, lb.params(c.dims, tau_r=c.tau_r, g_AB=c.g, kT=c.kT, seed=c.seed, storage=storage,
                                             rho0=rho0, collision=c.collision, lambda_bulk=c.lam_bulk,
                                             lambda_mom=c.lam_mom, lambda_ghost=c.lam_ghost),
                                c.n if np_max is None else np_max, total)
    lb.lbmd_batch_set_types(b, slot, [lb.lbmd_ptype(*t) for t in c.types],
                            [lb.lbmd_pair(i, j, e, s) for (i, j), (e, s) in c.wca.items()])
    if c.dh[0] != 0.0:
        lb.lbmd_batch_set_debye_hueckel(b, slot, *c.dh)
    a, bb, u = c.fields32()
    lb.lbmd_batch_init_fluid(b, slot, a, bb, u)
    lb.lbmd_batch_set_particles(b, slot, c.x, c.v, c.ptype, c.q)
    return slot


def read(b, slot, c: Case):
    lb = L()
    f = np.stack([lb.lbmd_batch_get_populations(b, slot, 0, c.shape), lb.lbmd_batch_get_populations(b, slot, 1, c.shape)])
    x, v, F = lb.lbmd_batch_get_particles(b, slot, c.n)
    return f, x, v, F


def run_alone(c: Case, total: int, chunks=None, config=None, storage=0, rho0=(0.0, 0.0)):
    lb = L()
    b = lb.lbmd_batch_create(0, storage, 4)
    try:
        if config:
            lb.lbmd_batch_set_config(b, *config)
        s = add_case(b, c, total, storage=storage, rho0=rho0)
        for k in chunks or [total]:
            lb.lbmd_batch_step(b, k)
        st = lb.lbmd_batch_poll(b, 4)
        assert st[s] == lb.LBMD_SLOT_DONE
        assert lb.lbmd_batch_step_count(b, s) == total
        return read(b, s, c)
    finally:
        lb.lbmd_batch_destroy(b)


def fluid_case(dims, seed, g=1.3, tau=1.0):
    rA, rB = noisy_fluid(dims, amp=0.03, seed=seed)
    return Case(dims=dims, tau_r=tau, g=g, seed=seed, rhoA=rA, rhoB=rB)


def same(r1, r2):
    return all(np.array_equal(a, b) for a, b in zip(r1, r2))


# ------------------------------------------------------------------ against the oracle
def test_mixed_batch_matches_oracle():
    lb = L()
    cases = [coupled_case((12, 10, 14), 24, seed=5, g=1.3, kT=0.01), fluid_case((9, 7, 5), seed=8, tau=0.8),
             config1_case(npart=20), coupled_case((7, 11, 6), 6, seed=9, g=0.9)]
    b = lb.lbmd_batch_create(0, 0, 8)
    try:
        slots = [add_case(b, c, 10) for c in cases]
        lb.lbmd_batch_step(b, 4)
        lb.lbmd_batch_step(b, 6)
        st = lb.lbmd_batch_poll(b, 8)
        for c, s in zip(cases, slots):
            assert st[s] == lb.LBMD_SLOT_DONE
            fg, xg, _, _ = read(b, s, c)
            fo, xo, _, _ = run_oracle(c, 10)
            assert pop_error(fg, fo) <= POP_TOL
            assert position_error(xg, xo, c.x, c.dims) <= POS_TOL
    finally:
        lb.lbmd_batch_destroy(b)


def test_batch_100_steps_positions_match_oracle():
    c = coupled_case((20, 18, 16), 30, seed=21, kT=0.002, min_dist=2.5)
    fg, xg, _, _ = run_alone(c, 100, chunks=[33, 67])
    fo, xo, _, _ = run_oracle(c, 100)
    assert position_error(xg, xo, c.x, c.dims) <= POS_TOL
    assert pop_error(fg, fo) <= 1e-4


def test_batch_matches_single_context():
    from gpu_common import run_gpu
    c = coupled_case((14, 12, 10), 20, seed=31, g=1.2, kT=0.005)
    fb, xb, vb, Fb = run_alone(c, 30)
    fs, xs, vs, Fs = run_gpu(c, 30)
    assert pop_error(fb, fs.astype(np.float64)) <= 1e-6
    assert np.abs(xb - xs).max() <= 1e-6 * max(c.dims)
    assert np.abs(Fb - Fs).max() <= 1e-6 * max(np.abs(Fs).max(), 1e-3)


# ------------------------------------------------------------------ alone == in the mix
def test_replica_is_bit_identical_alone_and_in_a_changing_mix():
    lb = L()
    X = coupled_case((20, 18, 16), 30, seed=21, kT=0.002, min_dist=2.5)
    total = 60
    alone = run_alone(X, total, chunks=[25, 35])

    A = fluid_case((24, 24, 24), seed=40)
    B = coupled_case((14, 14, 14), 12, seed=41, g=1.1, kT=0.003)
    C = config1_case(npart=40)
    b = lb.lbmd_batch_create(0, 0, 16)
    try:
        lb.lbmd_batch_set_config(b, 256, 2 * 152, 2 * 152, 2)  # another launch shape than alone
        sa = add_case(b, A, 100)
        sb = add_case(b, B, 30)
        lb.lbmd_batch_step(b, 10)  # A and B run ahead
        sx = add_case(b, X, total)
        assert sx not in (sa, sb)
        lb.lbmd_batch_step(b, 7)
        lb.lbmd_batch_step(b, 13)  # B reaches its 30 steps and freezes while X goes on
        st = lb.lbmd_batch_poll(b, 16)
        assert st[sb] == lb.LBMD_SLOT_DONE and lb.lbmd_batch_step_count(b, sb) == 30
        lb.lbmd_batch_remove(b, sb)  # leaves mid-run: particles and rows repacked
        sc = add_case(b, C, 50)  # joins mid-run, possibly in B's old slot
        lb.lbmd_batch_step(b, 11)
        lb.lbmd_batch_set_config(b, 4096, 8 * 152, 3 * 152, 3)
        lb.lbmd_batch_step(b, 40)
        st = lb.lbmd_batch_poll(b, 16)
        assert st[sx] == lb.LBMD_SLOT_DONE and lb.lbmd_batch_step_count(b, sx) == total
        mixed = read(b, sx, X)
        assert same(alone, mixed), "replica differs between alone and in the mix"
        # the others are unharmed too
        assert lb.lbmd_batch_step_count(b, sa) == 81 and lb.lbmd_batch_step_count(b, sc) == 50
    finally:
        lb.lbmd_batch_destroy(b)


def test_step_budgets_freeze_finished_replicas():
    lb = L()
    cases = [coupled_case((10, 9, 8), 8, seed=50 + k, g=1.0, kT=0.002) for k in range(3)]
    totals = [5, 12, 20]
    b = lb.lbmd_batch_create(0, 0, 4)
    try:
        slots = [add_case(b, c, t) for c, t in zip(cases, totals)]
        lb.lbmd_batch_step(b, 8)
        st = lb.lbmd_batch_poll(b, 4)
        assert [lb.lbmd_batch_step_count(b, s) for s in slots] == [5, 8, 8]
        assert [st[s] for s in slots] == [lb.LBMD_SLOT_DONE, lb.LBMD_SLOT_ACTIVE, lb.LBMD_SLOT_ACTIVE]
        frozen = read(b, slots[0], cases[0])
        lb.lbmd_batch_step(b, 8)
        lb.lbmd_batch_step(b, 8)
        st = lb.lbmd_batch_poll(b, 4)
        assert [lb.lbmd_batch_step_count(b, s) for s in slots] == [5, 12, 20]
        assert all(st[s] == lb.LBMD_SLOT_DONE for s in slots)
        assert same(frozen, read(b, slots[0], cases[0]))
        for c, s, t in zip(cases, slots, totals):
            assert same(read(b, s, c), run_alone(c, t))
    finally:
        lb.lbmd_batch_destroy(b)


def test_failed_replica_stops_alone():
    lb = L()
    dims = (6, 6, 6)
    bad = Case(dims=dims, rhoA=np.ones(dims[::-1]), rhoB=np.ones(dims[::-1]), x=np.array([[2.3, 2.6, 2.4]]),
               v=np.zeros((1, 3)), ptype=np.zeros(1, dtype=np.int32), types=[(0.0, 0.0, 50.0, 50.0, 0.0, 1.0)])
    good = coupled_case((12, 10, 14), 24, seed=5, g=1.3, kT=0.01)
    b = lb.lbmd_batch_create(0, 0, 4)
    try:
        s_bad = add_case(b, bad, 20)
        s_good = add_case(b, good, 20)
        lb.lbmd_batch_step(b, 20)
        st = lb.lbmd_batch_poll(b, 4)
        assert st[s_bad] == lb.LBMD_SLOT_FAILED
        assert lb.lbmd_batch_slot_error(b, s_bad) in (lb.LBMD_E_NEGATIVE_DENSITY, lb.LBMD_E_NONFINITE)
        assert lb.lbmd_batch_step_count(b, s_bad) < 20
        assert st[s_good] == lb.LBMD_SLOT_DONE
        assert same(read(b, s_good, good), run_alone(good, 20))
    finally:
        lb.lbmd_batch_destroy(b)


# ------------------------------------------------------------------ admission, tuning, storage
def test_admission_by_device_memory():
    lb = L()
    c = fluid_case((32, 32, 32), seed=60)
    probe = lb.lbmd_batch_create(1 << 40, 0, 4)
    try:
        add_case(probe, c, 1)
        need = lb.lbmd_batch_info(probe)["used"]
    finally:
        lb.lbmd_batch_destroy(probe)
    b = lb.lbmd_batch_create(2 * need + need // 2, 0, 8)
    try:
        s0 = add_case(b, c, 3)
        s1 = add_case(b, c, 3)
        with pytest.raises(lb.LbmdError) as e:
            add_case(b, c, 3)
        assert e.value.code == lb.LBMD_E_NOMEM
        assert lb.lbmd_batch_info(b)["occupied"] == 2
        lb.lbmd_batch_step(b, 3)
        assert all(lb.lbmd_batch_poll(b, 8)[[s0, s1]] == lb.LBMD_SLOT_DONE)
        lb.lbmd_batch_remove(b, s0)
        s2 = add_case(b, c, 3)  # fits again
        lb.lbmd_batch_step(b, 3)
        assert lb.lbmd_batch_poll(b, 8)[s2] == lb.LBMD_SLOT_DONE
        assert lb.lbmd_batch_info(b)["used"] == 2 * need
    finally:
        lb.lbmd_batch_destroy(b)


def test_autotuner_keeps_state_and_results():
    lb = L()
    cases = [coupled_case((16, 16, 16), 20, seed=70, g=1.1, kT=0.002), fluid_case((20, 12, 9), seed=71)]
    b = lb.lbmd_batch_create(0, 0, 4)
    try:
        slots = [add_case(b, c, 12) for c in cases]
        lb.lbmd_batch_step(b, 5)
        cfg, ms = lb.lbmd_batch_tune(b)
        assert cfg["tile_sites"] in (256, 1024, 4096) and cfg["collide_blocks"] in (2, 3)
        assert ms[0] > 0 and ms[1] > 0
        assert lb.lbmd_batch_get_config(b) == cfg
        lb.lbmd_batch_step(b, 7)
        lb.lbmd_batch_poll(b, 4)
        for c, s in zip(cases, slots):
            assert same(read(b, s, c), run_alone(c, 12))
    finally:
        lb.lbmd_batch_destroy(b)


@pytest.mark.parametrize("storage", [1, 2])
def test_16bit_batch_matches_16bit_context(storage):
    lb = L()
    from gpu_common import make_gpu
    c = coupled_case((12, 10, 14), 16, seed=80, g=1.2, kT=0.002)
    rho0 = (float(c.rhoA.mean()), float(c.rhoB.mean()))
    fb, xb, _, _ = run_alone(c, 10, storage=storage, rho0=rho0)
    ctx, _ = lb.lbmd_create(lb.params(c.dims, tau_r=c.tau_r, g_AB=c.g, kT=c.kT, seed=c.seed, storage=storage,
                                      rho0=rho0))
    try:
        lb.lbmd_set_types(ctx, [lb.lbmd_ptype(*t) for t in c.types],
                          [lb.lbmd_pair(i, j, e, s) for (i, j), (e, s) in c.wca.items()])
        lb.lbmd_set_debye_hueckel(ctx, *c.dh)
        lb.lbmd_init_fluid(ctx, *c.fields32())
        lb.lbmd_set_particles(ctx, c.x, c.v, c.ptype, c.q)
        lb.lbmd_step(ctx, 10)
        fs = np.stack([lb.lbmd_get_populations(ctx, k, c.shape) for k in (0, 1)])
        xs, _, _ = lb.lbmd_get_particles(ctx, c.n)
    finally:
        lb.lbmd_destroy(ctx)
    assert pop_error(fb, fs.astype(np.float64)) <= 1e-6
    assert np.abs(xb - xs).max() <= 1e-6 * max(c.dims)


def test_batch_argument_errors():
    lb = L()
    c = fluid_case((8, 8, 8), seed=90)
    b = lb.lbmd_batch_create(0, 0, 2)
    try:
        with pytest.raises(lb.LbmdError):
            lb.lbmd_batch_remove(b, 1)  # free slot
        with pytest.raises(lb.LbmdError) as e:
            lb.lbmd_batch_add(b, lb.params(c.dims, storage=1), 0, 5)  # storage differs from the batch's
        assert e.value.code == lb.LBMD_E_INVALID_ARG
        s = add_case(b, c, 5, np_max=2)
        x = np.array([[1.0, 1.0, 1.0], [3.0, 3.0, 3.0], [5.0, 5.0, 5.0]])
        with pytest.raises(lb.LbmdError):
            lb.lbmd_batch_set_particles(b, s, x, np.zeros((3, 3)), np.zeros(3, dtype=np.int32))  # > np_max
        with pytest.raises(lb.LbmdError):
            lb.lbmd_batch_set_config(b, 300, 152, 152, 3)
        add_case(b, c, 5)
        with pytest.raises(lb.LbmdError) as e:
            add_case(b, c, 5)  # both slots taken
        assert e.value.code == lb.LBMD_E_NOMEM
    finally:
        lb.lbmd_batch_destroy(b)


def test_batch_mixing_bgk_and_fluctuating_mrt_replicas():
    """MRT replicas (with fluid noise) and BGK replicas in one batch: each matches the oracle,
    and the MRT one is bit-identical alone and in the mix."""
    lb = L()
    eigs = dict(collision=1, lam_bulk=-1.5, lam_mom=-0.7, lam_ghost=-1.2)
    m1 = coupled_case((12, 10, 14), 24, seed=5, g=1.3, kT=0.002)
    for k, v in eigs.items():
        setattr(m1, k, v)
    m2 = fluid_case((9, 7, 5), seed=8, tau=0.8)
    m2.kT, m2.seed = 1e-4, 44
    for k, v in eigs.items():
        setattr(m2, k, v)
    bg = coupled_case((7, 11, 6), 6, seed=9, g=0.9)
    b = lb.lbmd_batch_create(0, 0, 8)
    try:
        slots = [add_case(b, c, 10) for c in (bg, m1, m2)]
        lb.lbmd_batch_step(b, 3)
        lb.lbmd_batch_step(b, 7)
        st = lb.lbmd_batch_poll(b, 8)
        for c, s in zip((bg, m1, m2), slots):
            assert st[s] == lb.LBMD_SLOT_DONE
            fg, xg, _, _ = read(b, s, c)
            fo, xo, _, _ = run_oracle(c, 10)
            assert pop_error(fg, fo) <= POP_TOL
            assert position_error(xg, xo, c.x, c.dims) <= POS_TOL
        assert same(read(b, slots[1], m1), run_alone(m1, 10))
    finally:
        lb.lbmd_batch_destroy(b)
