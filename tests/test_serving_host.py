"""Host-side pieces of the serving loop that need no GPU: the request stream and the
latency summary."""
import numpy as np

from paper_1306_0788_gb300 import inputs


def test_summary_percentiles():
    from paper_1306_0788_gb300 import serving
    recs = [dict(rid=k, arrival=0.1 * k, admitted=0.1 * k + 0.01, done=0.1 * k + 1.0, status="done", edge=16,
                 steps_taken=100) for k in range(10)]
    s = serving.summarize(recs)
    assert abs(s["p50_s"] - 1.0) < 1e-9 and abs(s["p99_service_s"] - 0.99) < 1e-9
    assert s["failed"] == 0 and s["replicas"] == 10
    assert abs(s["site_updates_per_s"] - 10 * 16 ** 3 * 100 / 1.9) < 1e-6


def test_request_stream_shape():
    reqs = inputs.serving_requests(4000, rate=50.0, seed=2)
    gaps = np.diff([0.0] + [r["arrival"] for r in reqs])
    assert abs(gaps.mean() - 1 / 50.0) < 0.1 / 50.0  # Poisson arrivals at the stated rate
    e = np.array([r["edge"] for r in reqs])
    assert e.min() == 16 and e.max() == 128
    n = np.array([r["np"] for r in reqs])
    assert n.min() >= 0 and n.max() <= 5000 and (n <= 0.5 * (e // 2.5) ** 3).all()
    g = np.array([r["g"] for r in reqs])
    assert 1.2 <= g.min() and g.max() <= 2.1


def test_spaced_particles_keep_their_distance():
    L = np.array([23.0, 17.0, 30.0])
    x = inputs.spaced_particles(600, tuple(int(v) for v in L), 2.0, seed=4)
    d = x[:, None] - x[None]
    d -= L * np.round(d / L)
    r = np.sqrt((d ** 2).sum(-1))
    np.fill_diagonal(r, np.inf)
    assert r.min() >= 1.0 and (x >= 0).all() and (x < L).all()


def test_coexistence_densities():
    """Equal chemical potential of the bulk free energy at the returned pair, mass split
    symmetric, and the tabulated pair at g rho = 1.68 (1.9103 / 0.0897)."""
    from paper_1306_0788_gb300 import serving
    for g in (1.2, 1.68, 2.1):
        hi, lo = serving.coexistence(g)
        assert abs(hi + lo - 2.0) < 1e-12
        assert abs(np.log(hi / lo) - g * (hi - lo)) < 1e-9
    hi, lo = serving.coexistence(1.68)
    assert abs(hi - 1.9103) < 1e-4 and abs(lo - 0.0897) < 1e-4
    assert serving.coexistence(0.9) == (1.0, 1.0)
