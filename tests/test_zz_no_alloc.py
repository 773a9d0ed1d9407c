"""The moment reduction for callers that cannot allocate device memory.

lbmd_fluid_moments_static serves code that runs under a fixed device-memory budget or inside a
framework that owns the CUDA allocator, and so cannot call cudaMalloc: it computes the same
FP64 sums as lbmd_diagnostics from populations already on the device, with its scratch in a
static device array instead of a cudaMalloc'd buffer.
This file is collected last so that a run stopping at the first failure has run every
other test before it.
"""
import numpy as np
import pytest

import oracle

from gpu_common import make_gpu

pytestmark = pytest.mark.gpu


def _case():
    from test_gpu_parity import coupled_case
    return coupled_case((20, 18, 16), 30, seed=21, kT=0.002, min_dist=2.5)


def test_static_moments_match_diagnostics_and_the_oracle_on_two_calls():
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
            # and the oracle's definition of the same sums over the same FP32 values
            want = oracle.fluid_moments(f.astype(np.float64))
            assert np.allclose(got[:2], want[:2], rtol=1e-12, atol=0)
            assert np.abs(got[2:] - want[2:]).max() <= 1e-12 * scale
    finally:
        L.lbmd_destroy(ctx)


def test_static_moments_reject_lattices_above_the_scratch_size():
    pytest.importorskip("torch")
    from paper_1306_0788_gb300 import lbmd as L

    with pytest.raises(L.LbmdError) as e:
        L.lbmd_fluid_moments_static(16, (1024, 1024, 1024), 16)  # rejected before any device access
    assert e.value.code == L.LBMD_E_INVALID_ARG
    assert "exceeds the maximum" in L.lbmd_last_error(None)


def test_static_moments_reject_host_memory_before_any_launch():
    """A host pointer where device memory is required is refused with LBMD_E_INVALID_ARG (checked
    with the driver's pointer attributes before any kernel runs), for the input and the output."""
    torch = pytest.importorskip("torch")
    from paper_1306_0788_gb300 import lbmd as L

    dims = (8, 8, 8)
    host_f = np.zeros((2, 19) + dims, dtype=np.float32)
    dev_f = torch.zeros(host_f.size, dtype=torch.float32, device="cuda")
    dev_out = torch.zeros(5, dtype=torch.float64, device="cuda")
    host_out = np.zeros(5)
    for f_ptr, out_ptr in ((host_f.ctypes.data, dev_out.data_ptr()), (dev_f.data_ptr(), host_out.ctypes.data)):
        with pytest.raises(L.LbmdError) as e:
            L.lbmd_fluid_moments_static(f_ptr, dims, out_ptr, torch.cuda.current_stream())
        assert e.value.code == L.LBMD_E_INVALID_ARG
        assert "device memory" in L.lbmd_last_error(None)
    L.lbmd_fluid_moments_static(dev_f.data_ptr(), dims, dev_out.data_ptr(), torch.cuda.current_stream())
    torch.cuda.synchronize()
    assert (dev_out.cpu().numpy() == 0).all()
