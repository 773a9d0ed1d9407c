"""Seeded synthetic inputs shaped like the paper's systems.

This module draws random numbers and lays out initial fields and particle
configurations; it contains none of the method's arithmetic (no equilibrium,
no forces, no streaming).  Both the CUDA path and the FP64 oracle are fed from
here, so the two always start from identical inputs.

Shapes follow the examples of the paper: binary mixtures with equal mean
densities (Sec. 4.4-4.5), flat interfaces and droplets (Secs. 4.1-4.3, Laplace
law), point particles with WCA excluded volume and bead-spring polyelectrolyte
chains (Sec. 4.4).
"""
from __future__ import annotations

import numpy as np


def rng(seed: int) -> np.random.Generator:
    return np.random.default_rng(np.random.PCG64(seed))


def uniform_noise(dims, rho0: float = 1.0, amp: float = 0.01, seed: int = 0):
    """rho_A, rho_B = rho0 + U(-amp, amp), independently per site (layout [nz, ny, nx])."""
    nx, ny, nz = dims
    g = rng(seed)
    rA = rho0 + g.uniform(-amp, amp, size=(nz, ny, nx))
    rB = rho0 + g.uniform(-amp, amp, size=(nz, ny, nx))
    return rA, rB


def _tanh_profile(dist, width):
    """0.5 (1 + tanh(dist / width)): 1 deep inside (dist > 0), 0 outside."""
    return 0.5 * (1.0 + np.tanh(dist / width))


def slab_and_droplets(dims, rho_hi: float, rho_lo: float, n_drops: int = 8,
                      r_min: float = 8.0, r_max: float = 32.0, width: float = 4.0,
                      seed: int = 0):
    """A-rich slab in the middle half of z, B-rich elsewhere, plus up to n_drops
    non-overlapping spheres of the opposite phase with radii U[r_min, r_max] placed in
    the B-rich region (interface-adsorption regime).  Returns rho_A, rho_B [nz, ny, nx]
    and the list of droplets (centre, radius)."""
    nx, ny, nz = dims
    g = rng(seed)
    z = np.arange(nz)[:, None, None] + 0.0
    y = np.arange(ny)[None, :, None] + 0.0
    x = np.arange(nx)[None, None, :] + 0.0
    z0, z1 = nz / 4.0, 3.0 * nz / 4.0
    # signed distance to the slab (positive inside), periodic-safe for the middle half
    dslab = np.minimum(z - z0, z1 - z)
    phiA = _tanh_profile(dslab, width) * np.ones((nz, ny, nx))
    drops = []
    tries = 0
    while len(drops) < n_drops and tries < 2000:
        tries += 1
        r = g.uniform(r_min, r_max)
        c = np.array([g.uniform(0, nx), g.uniform(0, ny), g.uniform(0, nz)])
        # keep droplets inside the B-rich region, away from the slab
        zc = c[2]
        dz_slab = min(abs(zc - z0), abs(zc - z1))
        if z0 - width <= zc <= z1 + width or dz_slab < r + 2 * width:
            continue
        if 2 * (r + 2 * width) > min(nx, ny, nz / 2):
            continue
        ok = True
        for (c2, r2) in drops:
            d = c - c2
            d -= np.array([nx, ny, nz]) * np.round(d / np.array([nx, ny, nz]))
            if np.linalg.norm(d) < r + r2 + 2 * width:
                ok = False
                break
        if ok:
            drops.append((c, r))
    for (c, r) in drops:
        dx = x - c[0]
        dx -= nx * np.round(dx / nx)
        dy = y - c[1]
        dy -= ny * np.round(dy / ny)
        dz = z - c[2]
        dz -= nz * np.round(dz / nz)
        dist = r - np.sqrt(dx * dx + dy * dy + dz * dz)
        phiA = np.maximum(phiA, _tanh_profile(dist, width))
    rA = rho_lo + (rho_hi - rho_lo) * phiA
    rB = rho_hi - (rho_hi - rho_lo) * phiA
    return rA, rB, drops


def flat_slab(dims, rho_hi: float, rho_lo: float, width: float = 2.0):
    """A-rich slab occupying nz/4 <= z < 3 nz/4 (two flat interfaces normal to z, at z =
    nz/4 - 1/2 and 3 nz/4 - 1/2), B-rich elsewhere, tanh profiles of the given width."""
    nx, ny, nz = dims
    z = np.arange(nz, dtype=np.float64) + 0.5
    dist = np.minimum(z - nz / 4.0, 3 * nz / 4.0 - z)
    phiA = _tanh_profile(dist, width)[:, None, None] * np.ones((nz, ny, nx))
    return rho_lo + (rho_hi - rho_lo) * phiA, rho_hi - (rho_hi - rho_lo) * phiA


def disk(dims, radius: float, rho_hi: float, rho_lo: float, width: float = 2.0):
    """A-rich cylinder (axis along z) of the given radius at the centre of the x-y plane."""
    nx, ny, nz = dims
    y = np.arange(ny)[None, :, None] - ny / 2.0 + 0.5
    x = np.arange(nx)[None, None, :] - nx / 2.0 + 0.5
    dist = radius - np.sqrt(x * x + y * y)
    phiA = _tanh_profile(dist, width) * np.ones((nz, ny, nx))
    return rho_lo + (rho_hi - rho_lo) * phiA, rho_hi - (rho_hi - rho_lo) * phiA


def sphere(dims, radius: float, rho_hi: float, rho_lo: float, width: float = 2.0):
    """A-rich sphere of the given radius centred in the box (at the middle of its central
    cell), B-rich outside, tanh profile of the given width."""
    nx, ny, nz = dims
    z = np.arange(nz)[:, None, None] - nz / 2.0 + 0.5
    y = np.arange(ny)[None, :, None] - ny / 2.0 + 0.5
    x = np.arange(nx)[None, None, :] - nx / 2.0 + 0.5
    phiA = _tanh_profile(radius - np.sqrt(x * x + y * y + z * z), width)
    return rho_lo + (rho_hi - rho_lo) * phiA, rho_hi - (rho_hi - rho_lo) * phiA


def slab_between(dims, z0: float, z1: float, rho_hi: float, rho_lo: float, width: float = 2.0):
    """A-rich slab between the planes z = z0 and z = z1 (0 <= z0 < z1 <= nz, node k at z = k),
    B-rich elsewhere, tanh profiles of the given width (periodic in z)."""
    nx, ny, nz = dims
    z = np.arange(nz, dtype=np.float64)
    mid, half = 0.5 * (z0 + z1), 0.5 * (z1 - z0)
    d = np.abs(((z - mid + nz / 2.0) % nz) - nz / 2.0)  # periodic distance from the slab's middle
    phiA = _tanh_profile(half - d, width)[:, None, None] * np.ones((nz, ny, nx))
    return rho_lo + (rho_hi - rho_lo) * phiA, rho_hi - (rho_hi - rho_lo) * phiA


def random_particles(n: int, dims, min_dist: float = 1.0, seed: int = 0, max_tries: int = 200):
    """n points uniform in the periodic box with pairwise minimum-image distance > min_dist
    (sequential rejection on a cell grid)."""
    nx, ny, nz = dims
    L = np.array([nx, ny, nz], dtype=np.float64)
    g = rng(seed)
    cs = max(min_dist, 1e-9)
    ncell = np.maximum((L // cs).astype(int), 1)
    grid = {}
    pts = np.zeros((n, 3))
    k = 0
    tries = 0
    while k < n:
        tries += 1
        if tries > max_tries * n + 1000:
            raise ValueError("could not place %d particles with min_dist %g" % (n, min_dist))
        p = g.uniform(0.0, 1.0, size=3) * L
        p = np.minimum(p, np.nextafter(L, 0))
        ci = (p / L * ncell).astype(int) % ncell
        ok = True
        if min_dist > 0:
            for dz in (-1, 0, 1):
                for dy in (-1, 0, 1):
                    for dx in (-1, 0, 1):
                        key = tuple((ci + (dx, dy, dz)) % ncell)
                        for j in grid.get(key, ()):
                            d = p - pts[j]
                            d -= L * np.round(d / L)
                            if d @ d <= min_dist * min_dist:
                                ok = False
                                break
                        if not ok:
                            break
                    if not ok:
                        break
                if not ok:
                    break
        if ok:
            pts[k] = p
            grid.setdefault(tuple(ci), []).append(k)
            k += 1
    return pts


def bead_spring_chains(n_chains: int, length: int, dims, bond: float = 0.97, seed: int = 0,
                       min_dist: float = 0.9):
    """Self-avoiding random-walk chains (step length `bond`) in a periodic box.
    Returns positions [n_chains*length, 3], bonds [n_chains*(length-1), 2] (consecutive
    beads), and charges: +1 for the first half of the chains, -1 for the second half."""
    nx, ny, nz = dims
    L = np.array([nx, ny, nz], dtype=np.float64)
    g = rng(seed)
    n = n_chains * length
    pos = np.zeros((n, 3))
    cs = 1.0
    ncell = np.maximum((L // cs).astype(int), 1)
    grid = {}

    def free(p, skip):
        ci = (p / L * ncell).astype(int) % ncell
        for dz in (-1, 0, 1):
            for dy in (-1, 0, 1):
                for dx in (-1, 0, 1):
                    for j in grid.get(tuple((ci + (dx, dy, dz)) % ncell), ()):
                        if j == skip:
                            continue
                        d = p - pos[j]
                        d -= L * np.round(d / L)
                        if d @ d < min_dist * min_dist:
                            return False
        return True

    def add(k, p):
        pos[k] = p
        ci = (p / L * ncell).astype(int) % ncell
        grid.setdefault(tuple(ci), []).append(k)

    k = 0
    for c in range(n_chains):
        while True:
            p = g.uniform(0, 1, size=3) * L
            if free(p, -1):
                break
        add(k, p % L)
        k += 1
        for b in range(1, length):
            for _ in range(1000):
                d = g.normal(size=3)
                d *= bond / np.linalg.norm(d)
                p = (pos[k - 1] + d) % L
                if free(p, k - 1):
                    break
            add(k, p)
            k += 1
    bonds = np.array([(c * length + b, c * length + b + 1) for c in range(n_chains)
                      for b in range(length - 1)], dtype=np.int32).reshape(-1, 2)
    q = np.where(np.arange(n) // length < n_chains // 2, 1.0, -1.0)
    return pos, bonds, q


def spaced_particles(n: int, dims, spacing: float = 2.0, seed: int = 0):
    """n points, at most one per cubic cell of edge `spacing` (cells chosen at random without
    replacement), each uniform in the central half of its cell: any two points are at least
    spacing / 2 apart, across the periodic boundary too.  Vectorised, for many replicas."""
    L = np.array(dims, dtype=np.float64)
    nc = np.maximum((L // spacing).astype(int), 1)
    ncell = int(nc.prod())
    if n > ncell:
        raise ValueError("at most %d particles fit with spacing %g" % (ncell, spacing))
    g = rng(seed)
    cells = g.choice(ncell, size=n, replace=False)
    ci = np.stack([cells % nc[0], (cells // nc[0]) % nc[1], cells // (nc[0] * nc[1])], axis=1)
    return (ci + 0.25 + 0.5 * g.uniform(0.0, 1.0, size=(n, 3))) * spacing


def serving_requests(n: int, rate: float, seed: int = 0, edge=(16, 128), np_max: int = 5000,
                     g_rho=(1.2, 2.1), gamma=(0.1, 2.0), steps: int = 1000, fill: float = 0.5,
                     spacing: float = 2.5):
    """A Poisson stream of n independent replica requests at `rate` per second: arrival time,
    cubic edge L ~ U{edge}, particle count ~ U{0..np_max} capped at `fill` of the cells of edge
    `spacing` in the box (spaced_particles then keeps every pair at least spacing / 2 apart),
    coupling g (times the mean density 1) ~ U[g_rho], friction gamma ~ U[gamma], and a seed
    for the replica's inputs."""
    g = rng(seed)
    t = np.cumsum(g.exponential(1.0 / rate, size=n))
    out = []
    for k in range(n):
        L = int(g.integers(edge[0], edge[1] + 1))
        cap = int(fill * int(L // spacing) ** 3)
        out.append(dict(rid=k, arrival=float(t[k]), edge=L, np=min(int(g.integers(0, np_max + 1)), cap),
                        g=float(g.uniform(*g_rho)), gamma=float(g.uniform(*gamma)), steps=steps,
                        seed=int(g.integers(0, 2**31 - 1))))
    return out
