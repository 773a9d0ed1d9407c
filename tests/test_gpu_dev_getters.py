"""The device-memory getters (lbmd_get_fields_dev, lbmd_get_populations_dev,
lbmd_get_particles_dev): the values of the host getters, written into caller device buffers in
the order of the caller's stream, and refused (nothing written) for host or short buffers."""
import numpy as np
import pytest

from gpu_common import make_gpu, pop_error, run_oracle
from test_gpu_parity import coupled_case

pytestmark = pytest.mark.gpu

FORMS = {"fp32, two passes": (0, 2), "fp32, one pass": (0, 1), "fp16 shifted": (1, 2)}


@pytest.mark.parametrize("form", sorted(FORMS))
def test_device_getters_equal_the_host_getters(form):
    """After 7 coupled steps, every device getter gives the host getter's values bit for bit, on a
    stream of the caller's other than the context's, with outputs left out in any combination;
    the populations also match the oracle."""
    torch = pytest.importorskip("torch")
    from paper_1306_0788_gb300 import lbmd as L

    storage, passes = FORMS[form]
    c = coupled_case((20, 18, 16), 30, seed=21, kT=0.002, min_dist=2.5)
    if storage:
        c.storage, c.rho0 = storage, (float(c.rhoA.mean()), float(c.rhoB.mean()))
    ctx = make_gpu(c, passes=passes)
    try:
        L.lbmd_step(ctx, 7)
        a, b, u = L.lbmd_get_fields(ctx, c.shape)
        f_host = [L.lbmd_get_populations(ctx, k, c.shape) for k in (0, 1)]
        x, v, F = L.lbmd_get_particles(ctx, c.n)

        s = torch.cuda.Stream()
        with torch.cuda.stream(s):
            nan = float("nan")
            da = torch.full(c.shape, nan, dtype=torch.float32, device="cuda")
            db = torch.full(c.shape, nan, dtype=torch.float32, device="cuda")
            du = torch.full(c.shape + (3,), nan, dtype=torch.float32, device="cuda")
            L.lbmd_get_fields_dev(ctx, da.data_ptr(), db.data_ptr(), du.data_ptr(), s)
            got = (da.cpu().numpy(), db.cpu().numpy(), du.cpu().numpy())
            # only some outputs: the others stay as they were
            da.fill_(nan), du.fill_(nan)
            db.fill_(-1.0)
            L.lbmd_get_fields_dev(ctx, None, db.data_ptr(), None, s)
            only_b = (da.cpu().numpy(), db.cpu().numpy(), du.cpu().numpy())
            fd = torch.full((2, 19) + c.shape, nan, dtype=torch.float32, device="cuda")
            for k in (0, 1):
                L.lbmd_get_populations_dev(ctx, k, fd[k].data_ptr(), s)
            f_dev = fd.cpu().numpy()
            px = torch.full((c.n, 3), nan, dtype=torch.float64, device="cuda")
            pv, pf = torch.full_like(px, nan), torch.full_like(px, nan)
            L.lbmd_get_particles_dev(ctx, px.data_ptr(), pv.data_ptr(), pf.data_ptr(), s)
            parts = (px.cpu().numpy(), pv.cpu().numpy(), pf.cpu().numpy())
            px.fill_(nan), pf.fill_(nan)
            L.lbmd_get_particles_dev(ctx, None, pv.data_ptr(), None, s)
            only_v = (px.cpu().numpy(), pv.cpu().numpy(), pf.cpu().numpy())
        L.lbmd_sync(ctx)
    finally:
        L.lbmd_destroy(ctx)

    for g, h in zip(got, (a, b, u)):
        assert np.array_equal(g, h)
    assert np.isnan(only_b[0]).all() and np.isnan(only_b[2]).all() and np.array_equal(only_b[1], b)
    assert np.array_equal(f_dev, np.stack(f_host))
    for g, h in zip(parts, (x, v, F)):
        assert np.array_equal(g, h)
    assert np.isnan(only_v[0]).all() and np.isnan(only_v[2]).all() and np.array_equal(only_v[1], v)
    fo, *_ = run_oracle(c, 7)
    assert pop_error(f_dev, fo) <= (1e-5 if storage == 0 else 2e-5)  # the stated 10-step bounds


def test_device_getters_refuse_host_memory():
    """A host pointer where device memory is required is refused with LBMD_E_INVALID_ARG before
    any launch (each getter, each output), as are a NULL population buffer and a component other
    than 0 or 1; the context stays usable.  (A buffer carved from a larger device allocation, as
    a caching allocator hands out, is checked against that allocation's extent only, so a short
    tensor is not caught -- the header states it.)"""
    pytest.importorskip("torch")
    from paper_1306_0788_gb300 import lbmd as L

    c = coupled_case((12, 10, 8), 6, seed=5)
    ctx = make_gpu(c)
    try:
        L.lbmd_step(ctx, 2)
        N = int(np.prod(c.dims))
        hf = np.full(19 * N, 7.0, dtype=np.float32)
        hd = np.full(3 * c.n, 7.0)
        calls = [lambda: L.lbmd_get_fields_dev(ctx, hf.ctypes.data, None, None),
                 lambda: L.lbmd_get_fields_dev(ctx, None, hf.ctypes.data, None),
                 lambda: L.lbmd_get_fields_dev(ctx, None, None, hf.ctypes.data),
                 lambda: L.lbmd_get_populations_dev(ctx, 1, hf.ctypes.data),
                 lambda: L.lbmd_get_particles_dev(ctx, hd.ctypes.data, None, None),
                 lambda: L.lbmd_get_particles_dev(ctx, None, hd.ctypes.data, None),
                 lambda: L.lbmd_get_particles_dev(ctx, None, None, hd.ctypes.data)]
        for call in calls:
            with pytest.raises(L.LbmdError) as e:
                call()
            assert e.value.code == L.LBMD_E_INVALID_ARG
            assert "device memory" in L.lbmd_last_error(ctx)
        for comp, ptr in ((2, None), (0, None)):
            with pytest.raises(L.LbmdError) as e:
                L.lbmd_get_populations_dev(ctx, comp, ptr)
            assert e.value.code == L.LBMD_E_INVALID_ARG
        assert (hf == 7.0).all() and (hd == 7.0).all()
        L.lbmd_step(ctx, 1)
        L.lbmd_sync(ctx)
    finally:
        L.lbmd_destroy(ctx)


def test_device_getters_edge_cases():
    """Before the fluid is set the field and population getters return LBMD_E_STATE; with no
    particles the particle getter writes nothing and succeeds; with every output NULL nothing is
    launched."""
    torch = pytest.importorskip("torch")
    from paper_1306_0788_gb300 import lbmd as L

    dims = (8, 6, 4)
    ctx, _ = L.lbmd_create(L.params(dims))
    try:
        buf = torch.full((19,) + dims[::-1], 7.0, dtype=torch.float32, device="cuda")
        for call in (lambda: L.lbmd_get_fields_dev(ctx, buf.data_ptr(), None, None),
                     lambda: L.lbmd_get_populations_dev(ctx, 0, buf.data_ptr())):
            with pytest.raises(L.LbmdError) as e:
                call()
            assert e.value.code == L.LBMD_E_STATE
        ones = np.ones(dims[::-1], dtype=np.float32)
        L.lbmd_init_fluid(ctx, ones, ones)
        x = torch.full((4, 3), 7.0, dtype=torch.float64, device="cuda")
        L.lbmd_get_particles_dev(ctx, x.data_ptr(), x.data_ptr(), x.data_ptr())  # no particles
        launches = L.lbmd_launch_count(ctx)
        L.lbmd_get_fields_dev(ctx, None, None, None)
        assert L.lbmd_launch_count(ctx) == launches
        L.lbmd_get_fields_dev(ctx, buf.data_ptr(), None, None)
        torch.cuda.synchronize()
        assert (x.cpu() == 7.0).all()
        assert np.allclose(buf.cpu().numpy()[0], 1.0)  # rho_A of the uniform fluid in the first N floats
    finally:
        L.lbmd_destroy(ctx)
