"""Pins of the oracle's fluctuating MRT collision (Eq. MODES and the appendix): the mode
basis, the reduction to BGK, the transport coefficients of Eq. (TRANSPORTCOEFF) for each
eigenvalue separately, exact conservation with noise, and the equilibrium fluctuations
(equipartition) that the noise amplitudes must produce for any set of eigenvalues."""
import numpy as np
import pytest

import oracle

from test_oracle_pins import CS2, _busy_system, _no_particles, _phi_mode

MRT = oracle.COLLISION_MRT


def _lattice():
    c, w = oracle.lattice()
    return c.astype(float), w


# ---------------------------------------------------------------- the mode basis
def test_mode_basis_is_orthogonal_and_splits_hydrodynamic_from_kinetic_modes():
    """Modes are orthogonal in the weighted inner product (b_k on the diagonal); the first
    ten span exactly the polynomials of degree <= 2 in c (density, momentum, stress), the
    other nine are orthogonal to all of them (kinetic modes)."""
    c, w = _lattice()
    e, b = oracle.mode_basis()
    G = (e * w) @ e.T
    assert np.abs(G - np.diag(b)).max() < 1e-14
    assert (b > 0).all()
    x, y, z = c.T
    mono = np.array([np.ones(19), x, y, z, x * x, y * y, z * z, x * y, y * z, z * x])
    # same span: projecting the monomials on e_0..e_9 (weighted) reproduces them
    coef = (mono * w) @ e[:10].T / b[:10]
    assert np.abs(coef @ e[:10] - mono).max() < 1e-13
    assert np.abs((mono * w) @ e[10:].T).max() < 1e-14
    assert e[0].tolist() == [1.0] * 19 and np.array_equal(e[1:4], c.T)


def test_equilibrium_and_forcing_have_no_kinetic_moments():
    """The quadratic f^eq (Eq. feq) and the forcing term carry no kinetic modes, and their
    stress moments are rho u u and G (appendix)."""
    c, w = _lattice()
    e, _ = oracle.mode_basis()
    u = np.array([0.03, -0.02, 0.05])
    g = np.array([0.01, 0.004, -0.007])
    m_eq = e @ oracle.feq(1.3, u)
    m_g = e @ oracle.forcing(g, u, -0.7, -1.25, -1.6)
    assert np.abs(m_eq[10:]).max() < 1e-15 and np.abs(m_g[10:]).max() < 1e-15
    assert abs(m_eq[7] - 1.3 * u[0] * u[1]) < 1e-15 and abs(m_eq[4] - 1.3 * u @ u) < 1e-15
    assert np.allclose(m_g[1:4], (2 - 0.7) / 2 * g, rtol=1e-13)
    assert abs(m_g[4] - (2 - 1.6) * (u @ g)) < 1e-15


# ---------------------------------------------------------------- deterministic part
def test_mrt_with_equal_eigenvalues_is_bgk():
    """With every eigenvalue -1/tau_r and no noise, Eq. MODES is the BGK update (R3)."""
    dims = (7, 6, 5)
    s, f, x, v = _busy_system(dims, 6, seed=4, kT=0.0)
    s2, f2, x2, v2 = _busy_system(dims, 6, seed=4, kT=0.0)
    s2.collision = MRT
    for t in range(5):
        assert oracle.step(s, f, x, v, t)[0] == 0
        assert oracle.step(s2, f2, x2, v2, t)[0] == 0
    assert np.abs(f2 - f).max() <= 1e-13 * np.abs(f).max()
    assert np.abs(x2 - x).max() <= 1e-12


@pytest.mark.parametrize("tau,others,axes", [(0.8, (-1.6, -0.7, -1.1), (0, 1)), (1.4, (-0.5, -1.9, -1.3), (1, 2)),
                                              (1.2, (-0.6, -1.5, -1.8), (2, 0))])
def test_mrt_shear_viscosity_follows_lambda_s_only(tau, others, axes):
    """Eq. (TRANSPORTCOEFF): eta_s / rho = -c_s^2 (1/lambda_s + 1/2) with lambda_s = -1/tau_r,
    whatever the bulk, momentum and kinetic eigenvalues; flow along axes[0] varying along
    axes[1] (the xy, yz and zx shear modes in turn)."""
    L = 64
    k = 2 * np.pi / L
    a, b = axes
    dims = [1, 1, 1]
    dims[b] = L
    shape = tuple(dims[::-1])
    prof = np.sin(k * np.arange(L)).reshape([L if ax == b else 1 for ax in (2, 1, 0)])
    u = np.zeros(shape + (3,))
    u[..., a] = 1e-3 * prof
    f = oracle.init_equilibrium(np.full(shape, 0.6), np.full(shape, 0.4), u)
    c, _ = _lattice()
    lb, lm, lg = others
    s = oracle.System(dims=tuple(dims), tau_r=tau, collision=MRT, lam_bulk=lb, lam_mom=lm, lam_ghost=lg)

    def amp():
        j = np.einsum("zinyx,i->nyx", f, c[:, a])
        return (j * prof).sum() * 2 / L

    oracle.run(s, f, *_no_particles(), 50)
    a0 = amp()
    oracle.run(s, f, *_no_particles(), 250, first_step=50)
    rate = -np.log(amp() / a0) / 250
    assert abs(rate / (CS2 * (tau - 0.5) * k * k) - 1) < 0.01


def test_mrt_conserves_mass_and_total_momentum_with_every_term():
    """With distinct eigenvalues, fluid noise and every coupling on, the forcing moments
    (built with lambda_M, lambda_s, lambda_b) hand the fluid exactly the impulse of the
    forces: per-component mass and fluid + particle momentum are conserved to rounding."""
    dims = (7, 6, 5)
    s, f, x, v = _busy_system(dims, 6, seed=4, kT=0.002)
    s.collision, s.lam_bulk, s.lam_mom, s.lam_ghost = MRT, -1.5, -0.6, -1.3
    m = np.asarray(s.mass)[s.type][:, None]
    m0 = oracle.fluid_moments(f)
    P0 = m0[2:] + (m * v).sum(0)
    for t in range(10):
        assert oracle.step(s, f, x, v, t)[0] == 0
    m1 = oracle.fluid_moments(f)
    assert np.allclose(m1[:2], m0[:2], rtol=1e-13, atol=0)
    assert np.abs(m1[2:] + (m * v).sum(0) - P0).max() < 1e-12
    assert np.abs(m1[2:] - m0[2:]).max() > 1e-6


@pytest.mark.parametrize("lam_mom", [-0.6, -1.7])
def test_mrt_interdiffusion_follows_lambda_M(lam_mom):
    """Eqs. (MERGING1), (TRANSPORTCOEFF), (comp_D): at g = 0 a composition wave decays at
    D k^2, D = c_s^2 mu, mu = -(1/lambda_M + 1/2), independent of lambda_s."""
    L = 64
    k = 2 * np.pi / L
    x = np.arange(L)
    rA = (1 + 1e-3 * np.sin(k * x))[None, None, :]
    rB = (1 - 1e-3 * np.sin(k * x))[None, None, :]
    f = oracle.init_equilibrium(rA, rB)
    s = oracle.System(dims=(L, 1, 1), tau_r=1.0, collision=MRT, lam_mom=lam_mom, lam_bulk=-1.3, lam_ghost=-0.9)
    oracle.run(s, f, *_no_particles(), 50)
    a0 = _phi_mode(f, L, k, np.sin)
    oracle.run(s, f, *_no_particles(), 250, first_step=50)
    rate = -np.log(_phi_mode(f, L, k, np.sin) / a0) / 250
    D = -CS2 * (1 / lam_mom + 0.5)
    assert abs(rate / (D * k * k) - 1) < 0.015


@pytest.mark.parametrize("lam_bulk", [-0.5, -1.5])
def test_mrt_sound_damping_follows_lambda_b(lam_bulk):
    """Linearised Navier-Stokes with the stress of Eq. (comp_Pi): a sound wave's energy
    decays at 2 Gamma with Gamma = k^2 (4/3 nu_s + nu_b) / 2.  Bulk viscosity (reading R14):
    the trace equation of the Chapman-Enskog expansion (first order, Pi_aa with lambda_b)
    with the traceless shear stress of Eq. (comp_Pi) gives nu_b = -(2/3) c_s^2 (1/lambda_b + 1/2)
    -- 2/3 nu_s at BGK, the known D3Q19 value; Eq. (TRANSPORTCOEFF) prints it without 2/3."""
    L = 40
    k = 2 * np.pi / L
    x = np.arange(L)
    tau = 0.9
    rA = (1 + 1e-4 * np.cos(k * x))[None, None, :]
    rB = (1 + 1e-4 * np.cos(k * x))[None, None, :]
    f = oracle.init_equilibrium(rA, rB)
    c, _ = _lattice()
    s = oracle.System(dims=(L, 1, 1), tau_r=tau, collision=MRT, lam_bulk=lam_bulk, lam_mom=-1.2, lam_ghost=-1.0)

    def energy():
        rho = f.sum(axis=(0, 1))[0, 0]
        j = np.einsum("zinyx,i->x", f, c[:, 0])
        dr = (rho * np.exp(-1j * k * x)).sum()
        dj = (j * np.exp(-1j * k * x)).sum()
        return CS2 * abs(dr) ** 2 + abs(dj) ** 2

    oracle.run(s, f, *_no_particles(), 20)
    t0, e0 = 20, energy()
    # average over whole periods of the exchange between the two terms
    period = L / np.sqrt(CS2)
    n = int(round(4 * period))
    es = []
    for t in range(n):
        oracle.run(s, f, *_no_particles(), 1, first_step=t0 + t)
        es.append(energy())
    es = np.array(es)
    ts = t0 + 1 + np.arange(n)
    slope = np.polyfit(ts, np.log(es), 1)[0]
    nu_s = CS2 * (tau - 0.5)
    nu_b = -2.0 / 3.0 * CS2 * (1 / lam_bulk + 0.5)
    gamma = k * k * (4 * nu_s / 3 + nu_b) / 2
    assert abs(-slope / (2 * gamma) - 1) < 0.02


# ---------------------------------------------------------------- the noise
def test_mrt_noise_conserves_mass_and_momentum():
    """The noise sits in the stress and kinetic modes and, with opposite signs, in the two
    components' momenta: per-component mass and total momentum are conserved exactly."""
    dims = (6, 5, 4)
    rA = np.full(dims[::-1], 1.2)
    rB = np.full(dims[::-1], 0.8)
    f = oracle.init_equilibrium(rA, rB)
    s = oracle.System(dims=dims, tau_r=0.9, collision=MRT, kT=1e-3, seed=5, lam_bulk=-1.4, lam_mom=-0.8,
                      lam_ghost=-1.1)
    m0 = oracle.fluid_moments(f)
    oracle.run(s, f, *_no_particles(), 30)
    m1 = oracle.fluid_moments(f)
    assert np.allclose(m1[:2], m0[:2], rtol=1e-13, atol=0)
    assert np.abs(m1[2:]).max() < 1e-12
    assert np.abs(f - oracle.init_equilibrium(rA, rB)).max() > 1e-3  # it does fluctuate


@pytest.mark.parametrize("rhoA,rhoB,tau,others", [(1.0, 1.0, 1.0, (-1.0, -1.0, -1.0)),
                                                  (1.5, 0.5, 0.8, (-1.5, -0.8, -1.2))])
def test_mrt_fluctuations_follow_equipartition(rhoA, rhoB, tau, others):
    """Fluctuation-dissipation: in equilibrium every node's populations fluctuate
    independently with variance (kT/c_s^2) rho_z w_i, so the component densities have
    variance (kT/c_s^2) rho_z and no cross-correlation, and the total momentum per direction
    kT rho -- for any set of eigenvalues (the amplitudes carry the 1 - (1+lambda)^2 factors)."""
    dims = (8, 8, 8)
    kT = 1e-4
    f = oracle.init_equilibrium(np.full(dims, rhoA), np.full(dims, rhoB))
    lb, lm, lg = others
    s = oracle.System(dims=dims, tau_r=tau, collision=MRT, kT=kT, seed=9, lam_bulk=lb, lam_mom=lm, lam_ghost=lg)
    oracle.run(s, f, *_no_particles(), 60)
    c, _ = _lattice()
    va, vb, cab, vj = [], [], [], []
    for t in range(40):
        oracle.run(s, f, *_no_particles(), 5, first_step=60 + 5 * t)
        a = f[0].sum(0) - rhoA
        b = f[1].sum(0) - rhoB
        j = np.einsum("zinyx,ia->nyxa", f, c)
        va.append((a * a).mean())
        vb.append((b * b).mean())
        cab.append((a * b).mean())
        vj.append((j * j).mean())
    ea, eb = kT / CS2 * rhoA, kT / CS2 * rhoB
    assert abs(np.mean(va) / ea - 1) < 0.05
    assert abs(np.mean(vb) / eb - 1) < 0.05
    assert abs(np.mean(cab)) < 0.05 * np.sqrt(ea * eb)
    assert abs(np.mean(vj) / (kT * (rhoA + rhoB)) - 1) < 0.05
