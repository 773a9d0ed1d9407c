"""Pins of the oracle's MD sub-stepping (reading R15: K particle substeps of dt / K per
lattice step, the fluid fields frozen, the momentum return averaged over the substeps)."""
import numpy as np

import oracle

from test_oracle_pins import _busy_system


def _uniform(dims, rho):
    return oracle.init_equilibrium(np.full(dims[::-1], rho), np.full(dims[::-1], rho))


def test_friction_decay_over_substeps_has_its_discrete_closed_form():
    """Fluid in uniform motion u0, one particle, friction only: the frozen coupling velocity
    is u0 at every substep, so K substeps give v = u0 + (v0 - u0) a^K with a = 1 - gamma dt /
    (K m) and x = x0 + sum_k v_k dt / K; the fluid receives exactly the momentum the particle
    loses."""
    dims = (6, 6, 6)
    u0 = np.array([0.02, 0.0, -0.01])
    u = np.broadcast_to(u0, dims[::-1] + (3,)).copy()
    f = oracle.init_equilibrium(np.full(dims[::-1], 1.0), np.full(dims[::-1], 1.0), u)
    P0 = oracle.fluid_moments(f)[2:]
    x0 = np.array([[2.3, 2.6, 2.4]])
    v0 = np.array([[0.05, -0.02, 0.01]])
    x, v = x0.copy(), v0.copy()
    m, gam, K = 3.0, 0.8, 4
    s = oracle.System(dims=dims, gamma=np.array([gam]), mass=np.array([m]), type=np.zeros(1, dtype=np.int32),
                      md_substeps=K)
    assert oracle.step(s, f, x, v, 0)[0] == 0
    a = 1.0 - gam / (K * m)
    vk = u0 + (v0 - u0) * a ** np.arange(1, K + 1)[:, None]
    assert np.allclose(v, vk[-1], rtol=1e-13, atol=1e-16)
    assert np.allclose(x, x0 + vk.sum(0) / K, rtol=0, atol=1e-14)
    P = oracle.fluid_moments(f)[2:]
    assert np.allclose(P - P0, m * (v0 - v)[0], rtol=1e-10, atol=1e-15)


def test_one_substep_is_the_plain_step():
    dims = (7, 6, 5)
    s1, f1, x1, v1 = _busy_system(dims, 6, seed=4)
    s2, f2, x2, v2 = _busy_system(dims, 6, seed=4)
    s2.md_substeps = 1
    for t in range(3):
        oracle.step(s1, f1, x1, v1, t)
        oracle.step(s2, f2, x2, v2, t)
    assert np.array_equal(f1, f2) and np.array_equal(x1, x2) and np.array_equal(v1, v2)


def test_substeps_conserve_mass_and_total_momentum():
    """Every coupling, noise, bonds, BGK and MRT: the fluid receives the averaged reactions,
    the particles the forces of every substep times dt / K -- fluid + particle momentum and
    each component's mass are conserved to rounding."""
    dims = (7, 6, 5)
    for collision in (0, 1):
        s, f, x, v = _busy_system(dims, 6, seed=4, kT=0.01)
        s.md_substeps, s.collision = 5, collision
        m = np.asarray(s.mass)[s.type][:, None]
        m0 = oracle.fluid_moments(f)
        P0 = m0[2:] + (m * v).sum(0)
        for t in range(6):
            assert oracle.step(s, f, x, v, t)[0] == 0
        m1 = oracle.fluid_moments(f)
        assert np.allclose(m1[:2], m0[:2], rtol=1e-13, atol=0)
        assert np.abs(m1[2:] + (m * v).sum(0) - P0).max() < 1e-12
        assert np.abs(m1[2:] - m0[2:]).max() > 1e-6


def _wca_energy(x, v, m, L):
    """Kinetic energy plus the WCA potential shifted by +eps below the cut-off (the force the
    particles feel is the unshifted one's, continuous at the cut-off; the shift makes the
    energy continuous too, so that it is the conserved quantity of the exact motion)."""
    d = x[0] - x[1]
    d -= L * np.round(d / L)
    r = np.sqrt(d @ d)
    u = oracle.pair_energy(oracle.PAIR_WCA, 1.0, 1.0, 0.0, r)
    if r < 2 ** (1 / 6):
        u += 1.0
    return 0.5 * m * (v * v).sum() + u


def test_substeps_keep_a_stiff_contact_stable():
    """Sec. 3 asks for a particle time step well below the stiffest interaction's: two light
    particles (m = 1) released at sigma = 1, inside the WCA range, no friction.  One update of
    dt = 1 throws them apart with hundreds of times the energy they had; 200 substeps conserve
    it to 3 %."""
    dims = (16, 16, 16)
    L = np.array(dims, dtype=float)
    out = {}
    for K in (1, 200):
        f = _uniform(dims, 1.0)
        x = np.array([[7.0, 8.0, 8.0], [8.0, 8.0, 8.0]])
        v = np.zeros((2, 3))
        s = oracle.System(dims=dims, gamma=np.array([0.0]), mass=np.array([1.0]), type=np.zeros(2, dtype=np.int32),
                          wca_eps=np.array([[1.0]]), wca_sig=np.array([[1.0]]), md_substeps=K)
        e0 = _wca_energy(x, v, 1.0, L)
        for t in range(3):
            oracle.step(s, f, x, v, t)
        out[K] = _wca_energy(x, v, 1.0, L) / e0
    assert out[1] > 100.0
    assert abs(out[200] - 1.0) < 0.03


def test_substep_noise_gives_the_discrete_langevin_variance():
    """Friction noise of substep k: sqrt(2 kT gamma K / dt) N(0,1) with its own counter.  A
    heavy bath (rho = 20 per component) at rest and one particle: the stationary velocity
    variance of v' = (1 - a) v + noise, a = gamma dt / (K m), is kT / (m (1 - a / 2)) -- a
    wrong factor K in the amplitude would be off by K."""
    dims = (10, 10, 10)
    kT, m, gam, K = 1e-3, 5.0, 1.0, 4
    f = _uniform(dims, 20.0)
    x = np.array([[4.3, 5.1, 4.7]])
    v = np.zeros((1, 3))
    s = oracle.System(dims=dims, kT=kT, seed=7, gamma=np.array([gam]), mass=np.array([m]),
                      type=np.zeros(1, dtype=np.int32), md_substeps=K)
    samples = []
    for t in range(2500):
        assert oracle.step(s, f, x, v, t)[0] == 0
        if t >= 100:
            samples.append(v[0].copy())
    var = np.mean(np.square(samples))
    a = gam / (K * m)
    assert abs(var / (kT / (m * (1 - a / 2))) - 1) < 0.12
