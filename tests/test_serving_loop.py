"""The serving loop's host logic (serving.Server.run) against a fake batch, without a GPU:
admission in arrival order while replicas fit the memory budget, continuous batching (a
replica admitted when another retires, while the rest keep running), failed replicas reported
without stopping the others, and a request that cannot fit an empty batch refused loudly."""
import time

import numpy as np
import pytest

from paper_1306_0788_gb300 import lbmd as L
from paper_1306_0788_gb300 import serving

ACTIVE, DONE, FAILED = L.LBMD_SLOT_ACTIVE, L.LBMD_SLOT_DONE, L.LBMD_SLOT_FAILED


class FakeBatch:
    """The lbmd_batch_* calls of the loop on the host: a replica costs one unit per site of a
    budget in sites; a step call advances every active replica by n steps and the clock by
    n * tick.  fail maps the k-th admitted replica to the step at which it fails."""

    def __init__(self, budget, max_slots=16, tick=1e-4, fail=None):
        self.budget, self.max_slots, self.tick = budget, max_slots, tick
        self.fail = fail or {}
        self.slots = {}
        self.added = 0
        self.offset = 0.0
        self.step_calls = []  # active replicas at each step call

    def clock(self):
        return time.perf_counter() + self.offset

    def used(self):
        return sum(s["sites"] for s in self.slots.values())

    def add(self, b, params, np_max, steps):
        sites = params.nx * params.ny * params.nz
        if self.used() + sites > self.budget or len(self.slots) >= self.max_slots:
            raise L.LbmdError(L.LBMD_E_NOMEM, "does not fit")
        slot = min(set(range(self.max_slots)) - set(self.slots))
        self.slots[slot] = dict(sites=sites, total=steps, taken=0, status=ACTIVE, order=self.added)
        self.added += 1
        return slot, 0

    def step(self, b, n):
        self.offset += n * self.tick
        self.step_calls.append(sum(s["status"] == ACTIVE for s in self.slots.values()))
        for s in self.slots.values():
            if s["status"] != ACTIVE:
                continue
            s["taken"] = min(s["total"], s["taken"] + n)
            at = self.fail.get(s["order"])
            if at is not None and s["taken"] >= at:
                s["status"], s["taken"] = FAILED, at
            elif s["taken"] >= s["total"]:
                s["status"] = DONE

    def poll(self, b, max_slots):
        st = np.zeros(max_slots, dtype=np.int32)
        for k, s in self.slots.items():
            st[k] = s["status"]
        return st

    def install(self, mp):
        noop = lambda *a, **k: None  # noqa: E731
        for name, fn in dict(lbmd_batch_create=lambda *a: object(), lbmd_batch_destroy=noop,
                             lbmd_batch_add=self.add, lbmd_batch_remove=lambda b, s: self.slots.pop(s),
                             lbmd_batch_set_types=noop, lbmd_batch_init_fluid=noop, lbmd_batch_set_particles=noop,
                             lbmd_batch_step=self.step, lbmd_batch_poll=self.poll,
                             lbmd_batch_info=lambda b: dict(budget=self.budget, used=self.used(),
                                                            occupied=len(self.slots), max_slots=self.max_slots),
                             lbmd_batch_slot_error=lambda b, s: L.LBMD_E_NONFINITE
                             if self.slots[s]["status"] == FAILED else 0,
                             lbmd_batch_step_count=lambda b, s: self.slots[s]["taken"],
                             lbmd_batch_diagnostics=lambda b, s: np.arange(8.0),
                             lbmd_batch_get_particles=lambda b, s, n: (np.zeros((n, 3)),) * 3).items():
            mp.setattr(serving.L, name, fn)


def _req(rid, steps, edge=16, arrival=0.0, npart=0):
    return dict(rid=rid, arrival=arrival, edge=edge, np=npart, g=1.5, gamma=1.0, steps=steps, seed=100 + rid)


def _run(fake, mp, reqs, chunk=25):
    fake.install(mp)
    with serving.Server(mem_budget=0, max_slots=fake.max_slots, chunk=chunk) as s:
        return s.run(reqs, clock=fake.clock)


def test_admission_in_arrival_order_and_continuous_batching(monkeypatch):
    """Budget for two 16^3 replicas, five requests at once: never more than two run, they are
    admitted in arrival order, and each later one is admitted as soon as a slot frees up --
    while its neighbour, which needs more steps, is still running."""
    fake = FakeBatch(budget=2 * 16 ** 3 + 10)
    steps = [50, 200, 50, 50, 75]
    done, info = _run(fake, monkeypatch, [_req(k, n) for k, n in enumerate(steps)])
    assert sorted(r["rid"] for r in done) == list(range(5))
    assert all(r["status"] == "done" and r["steps_taken"] == r["steps"] for r in done)
    assert all(r["diagnostics"] == list(np.arange(8.0)) for r in done)
    by = {r["rid"]: r for r in done}
    assert [r["rid"] for r in sorted(done, key=lambda r: r["admitted"])] == list(range(5))
    assert info["peak_replicas"] == 2 and max(fake.step_calls) == 2 and info["refusals"] > 0
    assert by[2]["admitted"] < by[1]["done"]  # admitted beside replica 1, not after the batch drained
    assert by[2]["admitted"] >= by[0]["done"]
    assert info["peak_bytes"] <= fake.budget


def test_failed_replica_is_reported_and_the_others_finish(monkeypatch):
    fake = FakeBatch(budget=10 * 16 ** 3, fail={1: 30})
    done, _ = _run(fake, monkeypatch, [_req(k, 100) for k in range(3)])
    by = {r["rid"]: r for r in done}
    assert by[1]["status"] == "failed" and by[1]["error"] == L.LBMD_E_NONFINITE and by[1]["steps_taken"] == 30
    assert "diagnostics" not in by[1]
    assert by[0]["status"] == by[2]["status"] == "done"
    summary = serving.summarize(done)
    assert summary["replicas"] == 3 and summary["failed"] == 1


def test_later_arrivals_wait_for_their_time(monkeypatch):
    fake = FakeBatch(budget=10 * 16 ** 3)
    done, _ = _run(fake, monkeypatch, [_req(0, 25, arrival=0.0), _req(1, 25, arrival=0.03)])
    by = {r["rid"]: r for r in done}
    assert by[1]["admitted"] >= 0.03 - 1e-9
    assert all(r["status"] == "done" for r in done)


def test_a_request_larger_than_the_empty_batch_is_refused(monkeypatch):
    fake = FakeBatch(budget=16 ** 3 - 1)
    with pytest.raises(RuntimeError, match="does not fit an empty batch"):
        _run(fake, monkeypatch, [_req(0, 25)])
