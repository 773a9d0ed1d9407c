"""Replica serving: a request loop over one batch (continuous batching).

Requests -- independent coupled LB/MD systems with their own lattice size, particle count,
Shan-Chen coupling and friction -- arrive over time.  The loop admits them in arrival order
while they fit the batch's device-memory budget (lbmd_batch_add refuses a replica that does
not fit), advances every admitted replica in the same graph-captured launches
(lbmd_batch_step), and every `chunk` steps collects the replicas that have taken all their
steps (lbmd_batch_poll), reads their results and frees their memory for the next requests.
Requests that arrive while others run join at the next chunk boundary, so their work
overlaps on the device with the replicas already there.

This module is orchestration only: every step of every replica runs in the library's
kernels, through the C ABI.
"""
from __future__ import annotations

import collections
import time

import numpy as np

from . import inputs
from . import lbmd as L

# The replica model of a request: a binary mixture at mean density 1 per component with an
# A-rich slab (the middle half of z) and a B-rich rest at the bulk coexistence densities of
# the request's g (tanh profiles of width 2), BGK tau_r = 1, point particles of one type with
# WCA (eps = sigma = 1) and friction coupling, placed at least 1.25 apart (outside the WCA
# range); g and gamma come with the request.  Started from a flat interface rather than from
# noise: with psi = rho the spinodal decomposition of a +-1 % noise drives the minority density
# negative within 200 steps from g rho = 1.68 up, and a flat interface stays positive for 1000
# steps up to g rho = 2.1.  Mass 200: the WCA core is far stiffer than an explicit update at
# dt = 1 tolerates for light particles (a close approach at m = 10 throws particles out of the
# fluid), and gamma dt / m <= 0.01 keeps the friction update in the gamma dt / m << 1 regime of
# Sec. 3.
RHO0 = 1.0
TAU_R = 1.0
KT = 1e-4
MASS = 200.0
WIDTH = 2.0
SPACING = 2.5
# Every replica checks its mass per component and total momentum against its state at admission
# every DIAG_EVERY steps and fails alone (LBMD_E_DRIFT) past DRIFT_TOL: FP32 rounding moves them by
# about 1e-8 per step, so 1e-4 over a request's steps flags only a broken state.
DIAG_EVERY = 250
DRIFT_TOL = 1e-4


def coexistence(g_rho: float):
    """Bulk coexistence densities (rho_hi, rho_lo) / rho0 of the symmetric mixture at g rho0 > 1:
    equal pressure and chemical potential of the bulk free energy (Sec. 2, ideal mixing plus
    g rho_A rho_B) give ln(x / (2 - x)) = g rho0 (2 x - 2) for x = rho_hi / rho0; bisection."""
    if not g_rho > 1.0:
        return 1.0, 1.0
    lo, hi = 1.0 + 1e-12, 2.0 - 1e-15
    for _ in range(200):
        x = 0.5 * (lo + hi)
        if np.log(x / (2.0 - x)) - g_rho * (2.0 * x - 2.0) > 0.0:
            hi = x
        else:
            lo = x
    return x, 2.0 - x


def replica_fluid(req):
    e = req["edge"]
    hi, lo = coexistence(req["g"] * RHO0)
    rA, rB, _ = inputs.slab_and_droplets((e, e, e), hi * RHO0, lo * RHO0, n_drops=0, width=WIDTH, seed=req["seed"])
    return rA, rB


def replica_params(req) -> L.lbmd_params:
    e = req["edge"]
    return L.params((e, e, e), tau_r=TAU_R, g_AB=req["g"], kT=KT, seed=req["seed"],
                    diag_every=DIAG_EVERY, drift_tol=DRIFT_TOL)


def admit(batch, req) -> int:
    """Add the request's replica to the batch and upload its initial state; raises
    LbmdError(LBMD_E_NOMEM) (nothing added) when it does not fit."""
    e = req["edge"]
    slot, _ = L.lbmd_batch_add(batch, replica_params(req), req["np"], req["steps"])
    try:
        L.lbmd_batch_set_types(batch, slot, [L.lbmd_ptype(0.0, 0.0, 0.0, 0.0, req["gamma"], MASS)],
                               [L.lbmd_pair(0, 0, 1.0, 1.0)])
        rA, rB = replica_fluid(req)
        L.lbmd_batch_init_fluid(batch, slot, rA, rB)
        n = req["np"]
        if n:
            x = inputs.spaced_particles(n, (e, e, e), SPACING, seed=req["seed"] + 1)
            L.lbmd_batch_set_particles(batch, slot, x, np.zeros((n, 3)), np.zeros(n, dtype=np.int32))
    except Exception:
        L.lbmd_batch_remove(batch, slot)
        raise
    return slot


def mean_sites(edge=(16, 128)) -> float:
    """E[L^3] for L uniform on {edge[0], ..., edge[1]}."""
    e = np.arange(edge[0], edge[1] + 1, dtype=np.float64)
    return float((e ** 3).mean())


class Server:
    def __init__(self, mem_budget: int = 0, max_slots: int = 4096, chunk: int = 25,
                 storage: int = L.LBMD_STORAGE_FP32):
        self.batch = L.lbmd_batch_create(mem_budget, storage, max_slots)
        self.max_slots = max_slots
        self.chunk = chunk

    def close(self):
        if self.batch is not None:
            L.lbmd_batch_destroy(self.batch)
            self.batch = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def calibrate(self, sample, warm: int = 10, timed: int = 40):
        """Admit `sample` together, tune the launch shape on it, and measure the saturated
        throughput in site updates per second; the sample is removed afterwards."""
        b = self.batch
        slots = [admit(b, dict(r, steps=warm + timed + 10)) for r in sample]
        try:
            L.lbmd_batch_step(b, warm)
            L.lbmd_batch_poll(b, self.max_slots)
            cfg, ms = L.lbmd_batch_tune(b)
            L.lbmd_batch_step(b, 2)
            L.lbmd_batch_poll(b, self.max_slots)
            t0 = time.perf_counter()
            L.lbmd_batch_step(b, timed)
            st = L.lbmd_batch_poll(b, self.max_slots)
            dt = time.perf_counter() - t0
            failed = int((st[slots] == L.LBMD_SLOT_FAILED).sum())
        finally:
            for s in slots:
                L.lbmd_batch_remove(b, s)
        sites = sum(r["edge"] ** 3 for r in sample)
        return dict(config=cfg, kernel_ms=ms, site_updates_per_s=sites * timed / dt, failed=failed,
                    replicas=len(sample))

    def run(self, requests, clock=time.perf_counter, keep_particles: bool = False):
        """Serve `requests` (arrival times in seconds from the start); returns one record per
        request -- arrival, admission and completion times, status, FP64 diagnostics (and the
        final particle positions with keep_particles) -- and the peak memory and concurrency."""
        b = self.batch
        pending = collections.deque(sorted(requests, key=lambda r: r["arrival"]))
        queue = collections.deque()
        running = {}  # slot -> record
        done = []
        peak_used = 0
        peak_running = 0
        refusals = 0  # admissions refused for lack of memory or slots
        t0 = clock()
        while pending or queue or running:
            now = clock() - t0
            while pending and pending[0]["arrival"] <= now:
                queue.append(pending.popleft())
            while queue:  # admission in arrival order while the replica fits
                r = queue[0]
                try:
                    slot = admit(b, r)
                except L.LbmdError as e:
                    if e.code != L.LBMD_E_NOMEM:
                        raise
                    if not running:
                        raise RuntimeError("request %d does not fit an empty batch" % r["rid"])
                    refusals += 1
                    break
                queue.popleft()
                running[slot] = dict(rid=r["rid"], arrival=r["arrival"], admitted=clock() - t0, edge=r["edge"],
                                     np=r["np"], steps=r["steps"])
            if not running:
                if pending:
                    time.sleep(max(0.0, pending[0]["arrival"] - (clock() - t0)))
                continue
            info = L.lbmd_batch_info(b)
            peak_used = max(peak_used, info["used"])
            peak_running = max(peak_running, len(running))
            L.lbmd_batch_step(b, self.chunk)
            st = L.lbmd_batch_poll(b, self.max_slots)
            now = clock() - t0
            for slot in [s for s in running if st[s] in (L.LBMD_SLOT_DONE, L.LBMD_SLOT_FAILED)]:
                rec = running.pop(slot)
                rec["done"] = now
                rec["status"] = "done" if st[slot] == L.LBMD_SLOT_DONE else "failed"
                rec["error"] = L.lbmd_batch_slot_error(b, slot)
                rec["steps_taken"] = L.lbmd_batch_step_count(b, slot)
                if rec["status"] == "done":
                    rec["diagnostics"] = L.lbmd_batch_diagnostics(b, slot).tolist()
                    if keep_particles:
                        rec["x"] = L.lbmd_batch_get_particles(b, slot, rec["np"])[0]
                L.lbmd_batch_remove(b, slot)
                done.append(rec)
        return done, dict(peak_bytes=peak_used, peak_replicas=peak_running, refusals=refusals)


def summarize(records, extra=None, t_end=None):
    """p50 / p99 of time-to-all-steps (arrival -> completion, and admission -> completion),
    queueing delay, and throughput over the run."""
    ok = [r for r in records if r["status"] == "done"]
    lat = np.array([r["done"] - r["arrival"] for r in ok])
    svc = np.array([r["done"] - r["admitted"] for r in ok])
    wait = np.array([r["admitted"] - r["arrival"] for r in ok])
    span = (t_end if t_end is not None else max(r["done"] for r in records)) - min(r["arrival"] for r in records)
    sites = sum(r["edge"] ** 3 * r["steps_taken"] for r in records)
    out = dict(replicas=len(records), failed=len(records) - len(ok),
               p50_s=float(np.percentile(lat, 50)), p99_s=float(np.percentile(lat, 99)),
               p50_service_s=float(np.percentile(svc, 50)), p99_service_s=float(np.percentile(svc, 99)),
               p99_queue_s=float(np.percentile(wait, 99)), span_s=float(span),
               replicas_per_s=len(ok) / span, site_updates_per_s=sites / span)
    if extra:
        out.update(extra)
    return out
