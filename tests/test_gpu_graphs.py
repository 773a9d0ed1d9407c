"""Replayed step graphs (lbmd_set_graphs) against kernels launched one by one.

With graphs on, lbmd_step takes its steps two at a time by replaying a recorded graph of two
coupled steps: the same kernels with the same arguments in the same order, the noise counters
taken from a device-resident step base.  The two modes must therefore agree bit for bit --
populations, positions, velocities and forces -- over call sequences that mix replays with odd
direct steps (both buffer parities get a graph of their own), re-record after a setter, and run
on the legacy stream as well as on a stream of the caller's.
"""
import numpy as np
import pytest
import torch

from gpu_common import Case, make_gpu, noisy_fluid
from paper_1306_0788_gb300 import inputs
from test_gpu_parity import coupled_case

pytestmark = pytest.mark.gpu

EIGS = dict(collision=1, lam_bulk=-1.5, lam_mom=-0.7, lam_ghost=-1.2)
SCHEDULE = (3, 4, "particles", 5, 1, 2, 1)  # lbmd_step counts; "particles" re-sets them (a setter)


def _run(c, graphs, schedule=SCHEDULE, stream=None):
    from paper_1306_0788_gb300 import lbmd as L
    ctx = make_gpu(c, stream)
    try:
        L.lbmd_set_graphs(ctx, graphs)
        l0 = L.lbmd_launch_count(ctx)
        for item in schedule:
            if item == "particles":
                x, v, _ = L.lbmd_get_particles(ctx, c.n)
                L.lbmd_set_particles(ctx, x, v, c.ptype, c.q)
            else:
                L.lbmd_step(ctx, item)
        L.lbmd_sync(ctx)
        f = np.stack([L.lbmd_get_populations(ctx, 0, c.shape), L.lbmd_get_populations(ctx, 1, c.shape)])
        x, v, F = L.lbmd_get_particles(ctx, c.n)
        return dict(f=f, x=x, v=v, F=F, steps=L.lbmd_step_count(ctx), launches=L.lbmd_launch_count(ctx) - l0)
    finally:
        L.lbmd_destroy(ctx)


def _mrt(c, kT):
    for k, v in EIGS.items():
        setattr(c, k, v)
    c.kT = kT
    return c


def _cases():
    bgk = coupled_case((12, 10, 14), 24, seed=5, g=1.3, kT=0.01)
    mrt = _mrt(coupled_case((12, 10, 14), 24, seed=6, g=1.3), 0.002)
    sub = _mrt(coupled_case((12, 10, 14), 24, seed=7, g=1.1), 0.002)
    sub.md_substeps = 3
    # FENE chains of heavy beads with the interactions in units of kT = 0.01 (WCA eps = kT,
    # k = 30 kT, R0 = 1.5, screened Coulomb lB = kT)
    dims, kT = (16, 12, 10), 0.01
    pos, bonds, q = inputs.bead_spring_chains(4, 5, dims, bond=0.97, seed=8, min_dist=1.0)
    rA, rB = noisy_fluid(dims, amp=0.02, seed=8)
    n = len(pos)
    chains = Case(dims=dims, g=1.0, kT=kT, seed=8, rhoA=rA, rhoB=rB, x=pos, v=np.zeros((n, 3)),
                  ptype=np.zeros(n, dtype=np.int32), q=q, types=[(-5e-4 * kT, 5e-4 * kT, 0.01 * kT, 0.0, 1.0, 100.0)],
                  wca={(0, 0): (kT, 1.0)}, dh=(kT, 0.25, 3.0), bonds=bonds, bond_kind=2, bond_k=30 * kT, bond_r=1.5)
    rA, rB = noisy_fluid((10, 9, 8), amp=0.03, seed=9)
    fluid = _mrt(Case(dims=(10, 9, 8), tau_r=0.9, g=1.2, seed=9, rhoA=rA, rhoB=rB), 1e-4)
    half = _mrt(coupled_case((12, 10, 14), 24, seed=10, g=1.3), 0.002)
    half.storage, half.rho0 = 2, (1.0, 1.0)  # BF16, shifted
    return dict(bgk=bgk, mrt=mrt, substeps=sub, bonds=chains, fluid_only=fluid, bf16=half)


CASES = _cases()


@pytest.mark.parametrize("own_stream", [False, True])
@pytest.mark.parametrize("name", sorted(CASES))
def test_graph_replay_is_bit_identical(name, own_stream):
    c = CASES[name]
    stream = torch.cuda.Stream() if own_stream else None
    g = _run(c, True, stream=stream)
    d = _run(c, False, stream=stream)
    assert g["steps"] == d["steps"] == 16
    for k in ("f", "x", "v", "F"):
        assert g[k].shape == d[k].shape
        assert np.array_equal(g[k], d[k]), (name, k, np.abs(g[k] - d[k]).max())
    assert np.isfinite(g["f"]).all()


def test_replays_are_counted_and_profiled():
    """Four steps from a fresh context: two replays of a graph that holds two steps' kernels and
    the advance of the step base, after one launch that sets the base (so no case fell back to
    launches one by one); the lattice update's timing events are retargeted on every replay, so
    profiling sees every update."""
    from paper_1306_0788_gb300 import lbmd as L
    for name in ("bgk", "mrt", "substeps", "fluid_only"):  # the MRT ones patch the update's counter
        c = CASES[name]
        d = _run(c, False, schedule=(4,))
        g = _run(c, True, schedule=(4,))
        assert g["launches"] == d["launches"] + 1 + 2, name
    c = CASES["bgk"]
    ctx = make_gpu(c)
    try:
        L.lbmd_profile_enable(ctx, True)
        L.lbmd_step(ctx, 5)
        ms, n = L.lbmd_profile_read(ctx, reset=True)
        assert n == 5 and ms > 0.0
        L.lbmd_step(ctx, 2)
        ms, n = L.lbmd_profile_read(ctx, reset=True)
        assert n == 2 and ms > 0.0
    finally:
        L.lbmd_destroy(ctx)
