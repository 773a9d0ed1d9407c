"""The seeded input generators that feed both the CUDA path and the oracle: determinism by
seed, the [nz, ny, nx] layout, and the promise each one makes (value ranges, where the
interfaces sit, minimum distances, bond lengths, the serving stream's distributions)."""
import numpy as np

from paper_1306_0788_gb300 import inputs


def _min_image(x, dims):
    L = np.array(dims, dtype=np.float64)
    d = x[:, None, :] - x[None, :, :]
    d -= L * np.round(d / L)
    r = np.sqrt((d ** 2).sum(-1))
    r[np.diag_indices(len(x))] = np.inf
    return r


def test_uniform_noise_layout_range_and_seed():
    a, b = inputs.uniform_noise((7, 5, 3), 2.0, 0.1, seed=3)
    assert a.shape == b.shape == (3, 5, 7)
    assert (np.abs(a - 2.0) <= 0.1).all() and (np.abs(b - 2.0) <= 0.1).all()
    a2, b2 = inputs.uniform_noise((7, 5, 3), 2.0, 0.1, seed=3)
    assert np.array_equal(a, a2) and np.array_equal(b, b2)
    assert not np.array_equal(a, inputs.uniform_noise((7, 5, 3), 2.0, 0.1, seed=4)[0])
    assert not np.array_equal(a, b)  # the two components draw independently


def test_phase_profiles_exchange_the_components():
    """rho_A + rho_B = rho_hi + rho_lo at every node and both stay within [rho_lo, rho_hi]."""
    dims = (48, 40, 64)
    fields = [inputs.slab_and_droplets(dims, 2.0, 0.1, n_drops=3, r_min=3.0, r_max=6.0, width=1.5, seed=1)[:2],
              inputs.flat_slab(dims, 2.0, 0.1), inputs.disk(dims, 9.0, 2.0, 0.1),
              inputs.sphere(dims, 9.0, 2.0, 0.1), inputs.slab_between(dims, 10.3, 50.8, 2.0, 0.1)]
    for a, b in fields:
        assert a.shape == b.shape == (64, 40, 48)
        assert np.allclose(a + b, 2.1, atol=1e-12)
        assert a.min() >= 0.1 - 1e-12 and a.max() <= 2.0 + 1e-12


def test_flat_slab_interfaces_where_stated():
    """Interfaces at z = nz/4 - 1/2 and 3 nz/4 - 1/2: the profile is half-way between the two
    nodes that straddle each, deep in the bulk phases elsewhere."""
    a, _ = inputs.flat_slab((4, 4, 32), 1.0, 0.0, width=2.0)
    prof = a[:, 0, 0]
    assert np.isclose(0.5 * (prof[7] + prof[8]), 0.5, atol=1e-12)
    assert np.isclose(0.5 * (prof[23] + prof[24]), 0.5, atol=1e-12)
    assert prof[16] > 0.99 and prof[0] < 0.01 and prof[31] < 0.01
    assert np.allclose(a, a[:, :1, :1])  # flat in x and y


def test_droplets_are_separate_and_outside_the_slab():
    dims = (64, 64, 128)
    width = 2.0
    _, _, drops = inputs.slab_and_droplets(dims, 2.0, 0.1, n_drops=6, r_min=3.0, r_max=8.0, width=width, seed=5)
    assert len(drops) >= 2
    L = np.array(dims, dtype=np.float64)
    z0, z1 = dims[2] / 4.0, 3 * dims[2] / 4.0
    for i, (c, r) in enumerate(drops):
        assert 3.0 <= r <= 8.0
        assert not (z0 - width <= c[2] <= z1 + width)
        for c2, r2 in drops[i + 1:]:
            d = c - c2
            d -= L * np.round(d / L)
            assert np.linalg.norm(d) >= r + r2 + 2 * width


def test_random_particles_keep_their_distance():
    dims = (12, 10, 8)
    x = inputs.random_particles(150, dims, 1.3, seed=2)
    assert x.shape == (150, 3)
    assert (x >= 0).all() and (x < np.array(dims)).all()
    assert _min_image(x, dims).min() > 1.3
    assert np.array_equal(x, inputs.random_particles(150, dims, 1.3, seed=2))


def test_spaced_particles_keep_half_the_spacing():
    dims = (20, 20, 20)
    x = inputs.spaced_particles(300, dims, spacing=2.5, seed=4)
    assert x.shape == (300, 3)
    assert (x >= 0).all() and (x < np.array(dims)).all()
    assert _min_image(x, dims).min() >= 2.5 / 2


def test_bead_spring_chains_bonds_and_charges():
    dims = (24, 24, 24)
    pos, bonds, q = inputs.bead_spring_chains(6, 10, dims, bond=0.97, seed=3, min_dist=0.9)
    assert pos.shape == (60, 3) and bonds.shape == (54, 2) and q.shape == (60,)
    assert all(b == a + 1 and a // 10 == b // 10 for a, b in bonds)  # consecutive, within a chain
    L = np.array(dims, dtype=np.float64)
    d = pos[bonds[:, 0]] - pos[bonds[:, 1]]
    d -= L * np.round(d / L)
    assert np.allclose(np.linalg.norm(d, axis=1), 0.97, atol=1e-9)
    r = _min_image(pos, dims)
    r[bonds[:, 0], bonds[:, 1]] = r[bonds[:, 1], bonds[:, 0]] = np.inf
    assert r.min() >= 0.9  # dilute enough that every bead found a free place
    assert (q[:30] == 1.0).all() and (q[30:] == -1.0).all()


def test_serving_stream_distributions():
    reqs = inputs.serving_requests(4000, rate=50.0, seed=7)
    t = np.array([r["arrival"] for r in reqs])
    assert (np.diff(t) > 0).all()
    assert abs(np.diff(t).mean() * 50.0 - 1.0) < 0.06  # exponential gaps of mean 1 / rate
    edges = np.array([r["edge"] for r in reqs])
    assert edges.min() >= 16 and edges.max() <= 128 and len(set(edges)) > 100
    for r in reqs:
        assert 0 <= r["np"] <= min(5000, int(0.5 * int(r["edge"] // 2.5) ** 3))
        assert 1.2 <= r["g"] <= 2.1 and 0.1 <= r["gamma"] <= 2.0 and r["steps"] == 1000
    assert reqs == inputs.serving_requests(4000, rate=50.0, seed=7)  # the same stream for the same seed


def test_sphere_and_slab_between_put_their_interfaces_where_stated():
    """The sphere is A-rich inside its radius and B-rich outside, with rho_A = rho_B at the stated
    radius (along the grid line y = z = 0.5 from the centre the zero sits at x = sqrt(R^2 - 1/2));
    slab_between has rho_A = rho_B at z0 and z1 (node k at z = k), also across the periodic wrap."""
    dims = (40, 40, 40)
    a, b = inputs.sphere(dims, 9.0, 2.0, 0.1, width=2.0)
    c = np.arange(40) - 19.5
    r = np.sqrt(c[:, None, None] ** 2 + c[None, :, None] ** 2 + c[None, None, :] ** 2)
    assert ((a - b)[r < 6.0] > 0).all() and ((a - b)[r > 12.0] < 0).all()
    d = (a - b)[20, 20, 20:]  # x = 0.5, 1.5, ... outwards
    zero = np.interp(0.0, d[::-1], c[20:][::-1])
    assert abs(zero - np.sqrt(81.0 - 0.5)) < 0.01
    for z0, z1 in ((10.3, 30.8), (30.0, 45.0)):
        a, b = inputs.slab_between((4, 4, 48), z0, z1, 2.0, 0.1, width=2.0)
        d = (a - b)[:, 0, 0]
        assert d[int(round((z0 + z1) / 2))] > 0 and d[int(round((z0 + z1) / 2 + 24)) % 48] < 0
        for zc in (z0, z1):
            k = int(np.floor(zc))
            lin = d[k % 48] + (d[(k + 1) % 48] - d[k % 48]) * (zc - k)
            assert abs(lin) < 0.01
