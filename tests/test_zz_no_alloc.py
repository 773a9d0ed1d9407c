"""The moment reduction for callers that cannot allocate device memory.

lbmd_fluid_moments_static serves code that runs under a fixed device-memory budget, inside a
framework that owns the CUDA allocator, or from a stream where a synchronising allocation
would stall other work: it computes the same FP64 sums as lbmd_diagnostics from populations
already on the device, with its scratch in a static device array instead of cudaMalloc.
This file is collected last so that a run stopping at the first failure has run every
other test before it.
"""
import numpy as np
import pytest

from gpu_common import make_gpu

pytestmark = pytest.mark.gpu


def _case():
    from test_gpu_parity import coupled_case
    return coupled_case((20, 18, 16), 30, seed=21, kT=0.002, min_dist=2.5)


def test_static_moments_match_diagnostics_on_two_calls():
    torch = pytest.importorskip("torch")
    from paper_1306_0788_gb300 import lbmd as L

    c = _case()
    ctx = make_gpu(c)
    out = torch.full((5,), float("nan"), dtype=torch.float64, device="cuda")
    stream = torch.cuda.current_stream()
    try:
        for nsteps in (5, 7):  # two calls in a row, on two different states
            L.lbmd_step(ctx, nsteps)
            ref = L.lbmd_diagnostics(ctx)[:5]
            f = np.stack([L.lbmd_get_populations(ctx, 0, c.shape), L.lbmd_get_populations(ctx, 1, c.shape)])
            f_dev = torch.from_numpy(np.ascontiguousarray(f)).cuda()
            out.fill_(float("nan"))
            L.lbmd_fluid_moments_static(f_dev.data_ptr(), c.dims, out.data_ptr(), stream)
            torch.cuda.synchronize()
            got = out.cpu().numpy()
            scale = abs(ref[0]) + abs(ref[1])
            assert np.isfinite(got).all()
            assert np.allclose(got[:2], ref[:2], rtol=1e-12, atol=0)
            assert np.abs(got[2:] - ref[2:]).max() <= 1e-12 * scale
    finally:
        L.lbmd_destroy(ctx)


def test_static_moments_reject_lattices_above_the_scratch_size():
    pytest.importorskip("torch")
    from paper_1306_0788_gb300 import lbmd as L

    with pytest.raises(L.LbmdError) as e:
        L.lbmd_fluid_moments_static(16, (1024, 1024, 1024), 16)  # rejected before any device access
    assert e.value.code == L.LBMD_E_INVALID_ARG
    assert "exceeds the maximum" in L.lbmd_last_error(None)
