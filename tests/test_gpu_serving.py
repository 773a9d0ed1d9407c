"""The serving loop: replicas arriving over time are admitted by device memory into one batch,
run in shared launches while others join and leave, and each comes out exactly as it would
alone (bit-identical FP64 diagnostics and particle positions: the stated tolerance of the
mix is zero)."""
import numpy as np
import pytest

from paper_1306_0788_gb300 import inputs

pytestmark = pytest.mark.gpu


def test_served_replicas_equal_alone_runs_and_admission_waits_for_memory():
    from paper_1306_0788_gb300 import lbmd as L
    from paper_1306_0788_gb300 import serving

    # all ten arrive at once (whatever the service speed) and together need more than the budget
    reqs = inputs.serving_requests(10, rate=1e6, seed=5, edge=(16, 28), np_max=300, steps=60)
    biggest = max(r["edge"] for r in reqs)
    # a budget of about three of the largest replicas: admission has to wait for memory
    with serving.Server(max_slots=16, chunk=7) as probe:
        s = serving.admit(probe.batch, dict(reqs[0], edge=biggest, np=300))
        one = L.lbmd_batch_info(probe.batch)["used"]
        L.lbmd_batch_remove(probe.batch, s)
    with serving.Server(mem_budget=3 * one, max_slots=16, chunk=7) as srv:
        records, peak = srv.run(reqs, keep_particles=True)
    assert len(records) == len(reqs) and all(r["status"] == "done" for r in records)
    assert all(r["steps_taken"] == 60 for r in records)
    assert peak["peak_bytes"] <= 3 * one and peak["peak_replicas"] >= 2
    assert peak["refusals"] > 0  # admission waited for memory
    # requests joined while others were running
    overlap = any(a["admitted"] > b["admitted"] and a["admitted"] < b["done"] for a in records for b in records)
    assert overlap
    with serving.Server(max_slots=2, chunk=60) as alone:
        for r in records:
            req = reqs[r["rid"]]
            s = serving.admit(alone.batch, req)
            L.lbmd_batch_step(alone.batch, 60)
            L.lbmd_batch_poll(alone.batch, 2)
            d = L.lbmd_batch_diagnostics(alone.batch, s)
            x = L.lbmd_batch_get_particles(alone.batch, s, req["np"])[0]
            L.lbmd_batch_remove(alone.batch, s)
            assert np.array_equal(np.asarray(r["diagnostics"]), d)
            assert np.array_equal(r["x"], x)
            rA, rB = serving.replica_fluid(req)
            m0 = np.array([rA.astype(np.float32).astype(np.float64).sum(), rB.astype(np.float32).astype(np.float64).sum()])
            assert np.abs(d[:2] / m0 - 1).max() < 1e-5  # mass of each component conserved
