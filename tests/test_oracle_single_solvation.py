"""The per-node momentum-conserving variant with a single solvation force (Sec. 2, the scheme
the paper describes after Eq. solvation_lambda and leaves for later), reading R16: with
kappa_A = kappa_B = 0 the only solvation force is that of Eq. (solvation_lambda), and the
particle receives, node by node, minus what it exerts on the fluid -- one force type acting
both ways, momentum conserved per particle-node pair."""
import numpy as np
import pytest

import oracle
from paper_1306_0788_gb300 import inputs


def _system(dims, lamA, gamma=0.0, mass=10.0, g=0.0):
    return oracle.System(dims=dims, tau_r=1.0, g_AB=g, g_BA=g, type=np.zeros(1, dtype=np.int32), q=np.zeros(1),
                         kappa=np.zeros((1, 2)), lam=np.array([[lamA, 0.0]]), gamma=np.array([gamma]),
                         mass=np.array([mass]), wca_eps=np.zeros((1, 1)), wca_sig=np.ones((1, 1)))


def test_particle_force_is_minus_the_sum_of_its_node_forces():
    """No Shan-Chen force and no friction: the force density on the fluid is the fluid-side
    solvation force alone, and its total over the nodes is exactly minus the force on the
    particle, in a non-uniform fluid where neither vanishes."""
    dims = (8, 8, 8)
    rA, rB = inputs.uniform_noise(dims, 1.0, 0.2, seed=3)
    f = oracle.init_equilibrium(rA, rB)
    s = _system(dims, lamA=0.05)
    x = np.array([[3.3, 4.6, 2.8]])
    v = np.zeros((1, 3))
    st, tr = oracle.step(s, f, x, v, 0, trace=True)
    assert st == 0
    node_total = tr["g"].sum(axis=(0, 1, 2, 3))
    assert np.abs(tr["f_fs"][0]).max() > 1e-4
    assert np.allclose(node_total, -tr["f_fs"][0], rtol=1e-13, atol=1e-16)
    assert np.abs(tr["f_ps"]).max() == 0.0


@pytest.mark.parametrize("lamA", [0.02, -0.02])
def test_single_solvation_force_moves_the_particle_by_the_sign_of_lambda(lamA):
    """A particle placed in the lower interface of an A-rich slab (z = 8; the slab fills the
    middle half of z): with lambda_A > 0 it is pushed from the A-rich nodes out to the B side
    (below z = 7.5 after 120 steps), with lambda_A < 0 pulled into the slab (beyond z = 10);
    fluid and particle momentum stay conserved."""
    dims = (6, 6, 32)
    rA, rB, _ = inputs.slab_and_droplets(dims, 1.9, 0.1, n_drops=0, width=3.0, seed=1)
    f = oracle.init_equilibrium(rA, rB)
    s = _system(dims, lamA=lamA, gamma=0.2, mass=5.0, g=1.68)
    z0 = 8.0
    x = np.array([[2.5, 2.5, z0]])
    v = np.zeros((1, 3))
    P0 = oracle.fluid_moments(f)[2:]
    for t in range(120):
        assert oracle.step(s, f, x, v, t)[0] == 0
    m1 = oracle.fluid_moments(f)
    P1 = m1[2:] + 5.0 * v[0]
    assert np.abs(P1 - P0).max() < 1e-14 * (m1[0] + m1[1])  # rounding of 120 steps
    if lamA > 0:
        assert x[0, 2] < 7.5
    else:
        assert x[0, 2] > 10.0
