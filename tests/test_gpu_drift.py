"""The FP64 drift check (lbmd_params.diag_every / drift_tol; LBMD_E_DRIFT).

The model conserves each component's mass (the collision and the forcing term of the appendix
have no zeroth moment) and the total momentum of fluid and particles (Sec. 2: forces on the
particles are returned to the fluid; Shan-Chen forces cancel pairwise when g_AB = g_BA).  The
check reduces both on the device every diag_every steps and compares them with the reference
taken when the state was set.  These tests show it quiet on a clean coupled run, raising on
states that break a conservation law -- populations changed by hand between steps (mass, then
momentum alone), and the asymmetric coupling g_AB != g_BA, whose momentum drift the FP64 oracle
predicts -- in single contexts and in batches.  Nothing here faults the device: every failure is
a value the check computes and reports through the error word.
"""
import numpy as np
import pytest

from paper_1306_0788_gb300 import inputs

from gpu_common import make_gpu

pytestmark = pytest.mark.gpu


def _coupled_case():
    from test_gpu_parity import coupled_case
    return coupled_case((20, 18, 16), 30, seed=21, kT=0.002, min_dist=2.5)


def _drifts(d0, d1):
    """Relative mass drift of A and B and the total momentum drift per unit mass between two
    lbmd_diagnostics outputs (the check's definitions, recomputed on the host)."""
    M = d0[0] + d0[1]
    P0, P1 = d0[2:5] + d0[5:8], d1[2:5] + d1[5:8]
    return abs(d1[0] - d0[0]) / abs(d0[0]), abs(d1[1] - d0[1]) / abs(d0[1]), float(np.linalg.norm(P1 - P0) / M)


def test_clean_coupled_run_is_quiet_and_reports_the_diagnostics_drift():
    """50 coupled steps (friction, solvation, WCA, thermal noise) with a check every 10 steps:
    no LBMD_E_DRIFT at a tolerance of 1e-5 (FP32 rounding moves each component's mass by about
    1.3e-8 per step: 6.6e-7 after these 50 steps on one GB300 run), five checks, and the drifts
    the check reports are the ones recomputed on the host from lbmd_diagnostics at the same
    step."""
    from paper_1306_0788_gb300 import lbmd as L
    c = _coupled_case()
    ctx = make_gpu(c, diag_every=10, drift_tol=1e-5)
    try:
        d0 = L.lbmd_diagnostics(ctx)
        assert L.lbmd_get_drift(ctx)[0] == -1  # reference taken, no check yet
        L.lbmd_step(ctx, 23)
        L.lbmd_step(ctx, 27)  # checks at 10, 20 (first call), 30, 40, 50 (second)
        L.lbmd_sync(ctx)  # raises on LBMD_E_DRIFT
        d1 = L.lbmd_diagnostics(ctx)
        got = L.lbmd_get_drift(ctx)
        want = _drifts(d0, d1)
        print("drift after 50 steps", got)
        assert got[0] == 50 and got[4] == 5
        assert np.allclose(got[1:4], want, rtol=1e-9, atol=1e-18)
        assert max(got[1:4]) < 1e-5
    finally:
        L.lbmd_destroy(ctx)


def _fluid_ctx(dims, rA, rB, g_AB, g_BA, diag_every, tol):
    from paper_1306_0788_gb300 import lbmd as L
    ctx, _ = L.lbmd_create(L.params(dims, tau_r=1.0, g_AB=g_AB, g_BA=g_BA, diag_every=diag_every, drift_tol=tol))
    L.lbmd_init_fluid(ctx, rA.astype(np.float32), rB.astype(np.float32))
    return ctx


def test_populations_changed_by_hand_raise_the_mass_drift():
    """A's populations scaled by 1 + 1e-3 between steps (lbmd_set_populations keeps the
    reference): the next check reports a mass drift of A of 1e-3 and the next synchronising call
    returns LBMD_E_DRIFT, sticky until lbmd_clear_error; B's mass and the momentum stay clean."""
    from paper_1306_0788_gb300 import lbmd as L
    dims = (16, 12, 10)
    rA, rB = inputs.uniform_noise(dims, 1.0, 0.01, seed=5)
    ctx = _fluid_ctx(dims, rA, rB, 1.2, 1.2, 5, 1e-5)
    try:
        L.lbmd_step(ctx, 5)
        L.lbmd_sync(ctx)
        fA = L.lbmd_get_populations(ctx, 0, dims[::-1])
        L.lbmd_set_populations(ctx, 0, fA * np.float32(1.001))
        L.lbmd_step(ctx, 5)
        with pytest.raises(L.LbmdError) as e:
            L.lbmd_sync(ctx)
        assert e.value.code == L.LBMD_E_DRIFT
        assert "drift" in L.lbmd_last_error(ctx)
        d = L.lbmd_get_drift(ctx)
        assert d[0] == 10 and d[4] == 2
        assert abs(d[1] - 1e-3) < 1e-6
        assert d[2] < 1e-6
        with pytest.raises(L.LbmdError):  # sticky
            L.lbmd_sync(ctx)
        L.lbmd_clear_error(ctx)
        L.lbmd_set_drift_reference(ctx)  # the changed state is the new reference
        L.lbmd_step(ctx, 5)
        L.lbmd_sync(ctx)
        assert L.lbmd_get_drift(ctx)[1] < 1e-6
    finally:
        L.lbmd_destroy(ctx)


def test_momentum_changed_by_hand_raises_the_momentum_drift():
    """+x and -x populations of B shifted by +d and -d at every node: mass unchanged, momentum
    changed by 2 d N along x; the check reports exactly that drift per unit mass."""
    from paper_1306_0788_gb300 import lbmd as L
    dims = (16, 12, 10)
    N = 16 * 12 * 10
    rA, rB = inputs.uniform_noise(dims, 1.0, 0.01, seed=6)
    ctx = _fluid_ctx(dims, rA, rB, 1.2, 1.2, 4, 1e-5)
    try:
        L.lbmd_step(ctx, 4)
        m0 = L.lbmd_diagnostics(ctx)
        fB = L.lbmd_get_populations(ctx, 1, dims[::-1])
        delta = np.float32(1e-4)
        fB[1] += delta
        fB[2] -= delta
        L.lbmd_set_populations(ctx, 1, fB)
        L.lbmd_step(ctx, 4)
        with pytest.raises(L.LbmdError) as e:
            L.lbmd_sync(ctx)
        assert e.value.code == L.LBMD_E_DRIFT
        d = L.lbmd_get_drift(ctx)
        want = 2 * float(delta) * N / (m0[0] + m0[1])
        assert d[1] < 1e-6 and d[2] < 1e-6
        assert abs(d[3] / want - 1) < 1e-3
    finally:
        L.lbmd_destroy(ctx)


def _asymmetric_oracle_drift(dims, rA, rB, g_AB, g_BA, steps):
    """Momentum drift per unit mass of the FP64 oracle after `steps` steps (no particles)."""
    import oracle
    s = oracle.System(dims=dims, tau_r=1.0, g_AB=g_AB, g_BA=g_BA)
    f = oracle.init_equilibrium(rA.astype(np.float32).astype(np.float64), rB.astype(np.float32).astype(np.float64))
    m0 = oracle.fluid_moments(f)
    x = np.zeros((0, 3))
    for k in range(steps):
        assert oracle.step(s, f, x, x.copy(), k)[0] == 0
    m = oracle.fluid_moments(f)
    return float(np.linalg.norm(m[2:] - m0[2:]) / (m0[0] + m0[1]))


ASYM_DIMS = (16, 14, 12)


def _asym_fields():
    return inputs.uniform_noise(ASYM_DIMS, 1.0, 0.1, seed=3)


def test_asymmetric_coupling_breaks_momentum_as_the_oracle_predicts():
    """g_AB = 1.2, g_BA = 0: the Shan-Chen forces no longer cancel pairwise (Sec. 2 gives the
    momentum guarantee for g_AB = g_BA only) and the total momentum moves by ~7e-6 per unit
    mass in 5 steps in the FP64 oracle; the GPU's check reports the same drift (FP32 path, 1 %)
    and raises at a tolerance of 1e-6, which the symmetric coupling stays below (its FP32
    rounding drift is ~1e-8 per step)."""
    from paper_1306_0788_gb300 import lbmd as L
    rA, rB = _asym_fields()
    want = _asymmetric_oracle_drift(ASYM_DIMS, rA, rB, 1.2, 0.0, 5)
    assert want > 5e-6
    ctx = _fluid_ctx(ASYM_DIMS, rA, rB, 1.2, 0.0, 5, 1e-6)
    try:
        L.lbmd_step(ctx, 5)
        with pytest.raises(L.LbmdError) as e:
            L.lbmd_sync(ctx)
        assert e.value.code == L.LBMD_E_DRIFT
        got = L.lbmd_get_drift(ctx)
        print("asymmetric drift", got[3], "oracle", want)
        assert abs(got[3] / want - 1) < 0.01
    finally:
        L.lbmd_destroy(ctx)
    ctx = _fluid_ctx(ASYM_DIMS, rA, rB, 1.2, 1.2, 5, 1e-6)
    try:
        L.lbmd_step(ctx, 20)
        L.lbmd_sync(ctx)
        got = L.lbmd_get_drift(ctx)
        print("symmetric drift", got)
        assert got[4] == 4 and max(got[1:4]) < 1e-6
    finally:
        L.lbmd_destroy(ctx)


def test_batch_replica_with_broken_momentum_stops_alone():
    """Two replicas in one batch with a check every 5 steps at 1e-6: the asymmetric one fails
    with LBMD_E_DRIFT at its first check (the same drift as the oracle's) and stops there, the
    symmetric one takes all its 20 steps; the reference is the state at admission."""
    from paper_1306_0788_gb300 import lbmd as L
    rA, rB = _asym_fields()
    want = _asymmetric_oracle_drift(ASYM_DIMS, rA, rB, 1.2, 0.0, 5)
    b = L.lbmd_batch_create(0, L.LBMD_STORAGE_FP32, 8)
    try:
        slots = []
        for g_BA in (1.2, 0.0):
            s, _ = L.lbmd_batch_add(b, L.params(ASYM_DIMS, g_AB=1.2, g_BA=g_BA, diag_every=5, drift_tol=1e-6), 0, 20)
            L.lbmd_batch_init_fluid(b, s, rA.astype(np.float32), rB.astype(np.float32))
            slots.append(s)
        L.lbmd_batch_step(b, 20)
        st = L.lbmd_batch_poll(b, 8)
        assert st[slots[0]] == L.LBMD_SLOT_DONE
        assert st[slots[1]] == L.LBMD_SLOT_FAILED
        assert L.lbmd_batch_slot_error(b, slots[1]) == L.LBMD_E_DRIFT
        assert L.lbmd_batch_step_count(b, slots[1]) == 5
        good, bad = L.lbmd_batch_get_drift(b, slots[0]), L.lbmd_batch_get_drift(b, slots[1])
        print("batch drifts", good, bad, "oracle", want)
        assert good[0] == 20 and good[4] == 4 and max(good[1:4]) < 1e-6
        assert bad[0] == 5 and abs(bad[3] / want - 1) < 0.01
    finally:
        L.lbmd_batch_destroy(b)


def test_no_check_without_diag_every():
    """diag_every = 0 (the default): no check runs and none is reported (step -1, no checks), with
    no reference taken by lbmd_init_fluid or lbmd_set_particles; lbmd_set_drift_reference still
    takes one on request."""
    from paper_1306_0788_gb300 import lbmd as L
    c = _coupled_case()
    ctx = make_gpu(c)
    try:
        L.lbmd_step(ctx, 12)
        L.lbmd_sync(ctx)
        d = L.lbmd_get_drift(ctx)
        assert d[0] == -1 and d[4] == 0 and max(d[1:4]) == 0
        L.lbmd_set_drift_reference(ctx)
        assert L.lbmd_get_drift(ctx)[0] == -1
    finally:
        L.lbmd_destroy(ctx)
