"""Pins of the oracle on the paper's solvation-force examples: the free-energy profile across a
flat interface (Sec. 3, Eq. solvation_density) and the adsorption analysis of the contact-angle
example (Sec. 4.1).

For a profile that varies along z only, the stencil gradient of Eq. SCforce's weights is the
central difference: S_z / c_s^2 = sum_i w_i c_iz rho(z + c_iz) / c_s^2 = (rho(z+1) - rho(z-1)) / 2
(1/18 from the axis link and 4 x 1/36 from the diagonals, over 1/3).  The particle force of Eq.
solvation_kappa interpolates it linearly between the nodes, so the holding force and its zeros
are fixed exactly by the node densities; these tests compute them that way, independently of the
oracle's stencil and interpolation.
"""
import numpy as np
import pytest

import oracle
from paper_1306_0788_gb300 import inputs

G = 1.68
RHO_HI, RHO_LO = 1.9103, 0.0897  # F_bulk coexistence pair for g = 1.68 at rho_A + rho_B = 2
LZ = 32


def _no_particles():
    return np.zeros((0, 3)), np.zeros((0, 3))


@pytest.fixture(scope="module")
def slab():
    rA, rB = inputs.flat_slab((2, 2, LZ), RHO_HI, RHO_LO, 2.0)
    f = oracle.init_equilibrium(rA.astype(np.float32).astype(np.float64), rB.astype(np.float32).astype(np.float64))
    oracle.run(oracle.System(dims=(2, 2, LZ), tau_r=1.0, g_AB=G, g_BA=G), f, *_no_particles(), 3000)
    return f


def probe_forces(f, kappa, zs):
    """z-force on a particle held at (0.5, 0.5, z) for each z, from one traced oracle step."""
    s = oracle.System(dims=(2, 2, LZ), tau_r=1.0, g_AB=G, g_BA=G, kappa=np.array([kappa]), lam=np.zeros((1, 2)),
                      gamma=np.zeros(1), mass=np.array([1e12]), type=np.zeros(1, dtype=np.int32), q=np.zeros(1))
    out = []
    for z in zs:
        _, tr = oracle.step(s, f.copy(), np.array([[0.5, 0.5, z]]), np.zeros((1, 3)), 0, trace=True)
        out.append(tr["f_total"][0, 2])
    return np.array(out)


def central_difference_force(rho, kappa, zs):
    """-sum_z kappa_z times the central difference of the node densities, interpolated linearly
    in z (periodic)."""
    F = np.zeros(len(zs))
    for k, r in zip(kappa, rho):
        grad = 0.5 * (np.roll(r, -1) - np.roll(r, 1))
        z0 = np.floor(zs).astype(int)
        t = zs - z0
        F -= k * ((1 - t) * grad[z0 % LZ] + t * grad[(z0 + 1) % LZ])
    return F


def crossing(d, lo, hi):
    for z in range(lo, hi):
        if d[z] * d[z + 1] < 0:
            return z + d[z] / (d[z] - d[z + 1])
    raise AssertionError("no crossing")


def stable_zero(zs, F, near):
    i = np.nonzero((F[:-1] > 0) & (F[1:] <= 0))[0]
    roots = zs[i] + F[i] / (F[i] - F[i + 1]) * (zs[i + 1] - zs[i])
    roots = roots[np.abs(roots - near) < 4]
    return roots[np.argmin(np.abs(roots - near))] if len(roots) else None


def test_relaxed_slab_is_symmetric_with_the_crossing_between_nodes(slab):
    """The slab of inputs.flat_slab is symmetric under A <-> B with z -> 2 z_int - z about its
    interfaces; the dynamics keep that symmetry, so rho_A = rho_B exactly at z_int = 3 LZ/4 - 1/2."""
    rho = slab.sum(1)[:, :, 0, 0]
    A, B = rho
    zi = 3 * LZ // 4 - 1  # nodes zi and zi + 1 bracket the upper interface
    for k in range(6):
        assert abs(A[zi - k] - B[zi + 1 + k]) < 1e-12
    assert abs(crossing(A - B, zi - 2, zi + 2) - (zi + 0.5)) < 1e-12


@pytest.mark.parametrize("kappa", [(-1.0, -2.0), (0.5, 0.5), (0.7, 0.3)])
def test_holding_force_is_the_interpolated_central_difference(slab, kappa):
    zs = np.arange(16.0, 31.99, 0.125)
    F = probe_forces(slab, kappa, zs)
    rho = slab.sum(1)[:, :, 0, 0]
    ref = central_difference_force(rho, kappa, zs)
    assert np.abs(F - ref).max() < 1e-12 * np.abs(ref).max()


def test_equal_positive_kappa_has_its_free_energy_minimum_at_the_interface(slab):
    """kappa_A = kappa_B = k > 0: Delta E(z) follows the total density (Sec. 3), so a particle
    repelled by both components is trapped at the interface, where the total density is lowest.
    On the lattice the identity is exact with the (1, 2, 1)/4-smoothed node density: the
    integral of the interpolated central difference from node a to node b is s(b) - s(a), s(z) =
    rho(z-1)/4 + rho(z)/2 + rho(z+1)/4, so Delta E at the nodes is k (s(z) - s(z_0)) to
    rounding, and the well depth is k (s_bulk - s_interface)."""
    k = 0.5
    zs = np.arange(16.0, 31.99, 0.05)
    F = probe_forces(slab, (k, k), zs)
    dE = -np.concatenate([[0.0], np.cumsum(0.5 * (F[1:] + F[:-1]) * np.diff(zs))])
    tot = slab.sum(1)[:, :, 0, 0].sum(0)
    smooth = 0.25 * np.roll(tot, 1) + 0.5 * tot + 0.25 * np.roll(tot, -1)
    nodes = np.arange(16, 32)
    at = np.rint((nodes - 16) / 0.05).astype(int)
    assert np.abs(dE[at] - k * (smooth[nodes] - smooth[16])).max() < 1e-11
    z_int = 3 * LZ / 4 - 0.5
    assert abs(zs[np.argmin(dE)] - z_int) <= 0.05
    depth = dE[0] - dE.min()
    assert depth > 0.1 * k * (tot[16] - tot.min())


def test_adsorption_distance_symmetry_and_closed_form(slab):
    """Equilibrium of a particle free to move along z: the stable zero of the holding force.
    At the symmetric interface d(0) = 0 and d(-r) = -d(r); d grows with r and moves into the
    component that repels the particle less; each zero equals that of the central-difference
    closed form."""
    rho = slab.sum(1)[:, :, 0, 0]
    z_int = 3 * LZ / 4 - 0.5
    zs = np.arange(16.0, 31.99, 0.02)
    d = {}
    for r in (-1.0, -0.5, 0.0, 0.5, 1.0):
        kap = (0.5 * (1 + r / 2), 0.5 * (1 - r / 2))
        F = probe_forces(slab, kap, zs)
        z0 = stable_zero(zs, F, z_int)
        zc = stable_zero(zs, central_difference_force(rho, kap, zs), z_int)
        assert z0 is not None and abs(z0 - zc) < 1e-9
        d[r] = z0 - z_int
    assert abs(d[0.0]) < 1e-9
    for r in (0.5, 1.0):
        assert abs(d[r] + d[-r]) < 1e-9
    assert 0 < d[0.5] < d[1.0]


def test_strong_preference_detaches_from_the_interface(slab):
    """Complete wetting: for r = 2 (kappa_B = 0) the force points into B at every height between
    the bulks, so the particle has no equilibrium at the interface."""
    zs = np.arange(17.0, 30.0, 0.05)
    F = probe_forces(slab, (1.0, 0.0), zs)
    assert stable_zero(zs, F, 3 * LZ / 4 - 0.5) is None
    assert (F >= -1e-15).all()


def _demixing_run(lam, steps, dims=(32, 32, 2), n=100, seed=3):
    """The single-fluid example of Sec. 3 on the oracle: two identical uncoupled components at
    rho = 1 each, particles with kappa = 0.05, the given lambda on both components, WCA with
    eps = 0.1 k_BT and sigma = 0.7, gamma = 1, m = 10, k_BT = 1e-5."""
    kT = 1e-5
    nx, ny, nz = dims
    x = inputs.random_particles(n, dims, 0.7, seed=seed)
    v = np.zeros_like(x)
    f = oracle.init_equilibrium(np.ones((nz, ny, nx)), np.ones((nz, ny, nx)))
    s = oracle.System(dims=dims, tau_r=1.0, kT=kT, seed=seed + 1, kappa=np.array([[0.05, 0.05]]),
                      lam=np.array([[lam, lam]]), gamma=np.ones(1), mass=np.array([10.0]),
                      wca_eps=np.full((1, 1), 0.1 * kT), wca_sig=np.full((1, 1), 0.7),
                      type=np.zeros(n, dtype=np.int32), q=np.zeros(n))
    for k in range(steps):
        assert oracle.step(s, f, x, v, k)[0] == 0
    return x, f.sum(1).sum(0)


def _block_stats(x, rho, dims, block=8):
    nx, ny, _ = dims
    c, _, _ = np.histogram2d(np.mod(x[:, 1], ny), np.mod(x[:, 0], nx), bins=(ny // block, nx // block),
                             range=[[0, ny], [0, nx]])
    r = rho.mean(0).reshape(ny // block, block, nx // block, block).mean(axis=(1, 3))
    return c, r


def test_depleting_particles_gather_in_fluid_poor_domains():
    """Sec. 3, single-fluid example: particles that push the fluid away (lambda > 0 in Eq.
    solvation_lambda as printed) and move down density gradients (kappa > 0) gather where the
    fluid is thin -- block particle counts anti-correlate with the fluid density and spread
    beyond independent placement -- while the fluid stays positive there; with kappa alone
    (lambda = 0) the fluid, uniform at the start, gives the particles no force to gather by."""
    dims = (32, 32, 2)
    x, rho = _demixing_run(0.01, 1500, dims)
    c, r = _block_stats(x, rho, dims)
    assert np.corrcoef(c.ravel(), r.ravel())[0, 1] < -0.7
    assert c.var() / c.mean() > 1.5
    assert rho.min() > 0.5 * 2.0
    x0, rho0 = _demixing_run(0.0, 1500, dims)
    assert np.abs(rho0 - 2.0).max() < 0.05 * (2.0 - rho.min())  # only friction stirs it
    c0, _ = _block_stats(x0, rho0, dims)
    assert c0.var() / c0.mean() < c.var() / c.mean()
