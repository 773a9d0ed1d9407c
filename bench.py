"""Throughput benchmark of the coupled two-component D3Q19 Shan-Chen LB / MD step.

One bench "step" is one full coupled time step (Shan-Chen force, fluid-side solvation,
coupling velocity, particle forces, momentum return, stream + collide for both components,
cell-list pair forces, particle update) over the whole lattice.  Default workload: a 256^3
lattice with a flat slab interface plus spherical droplets of radii 8-32 and 2e4 point
particles with solvation coupling preferring component B and WCA pairs (synthetic, seeded).

Prints ONE JSON line (rank 0).  `--impl reference` times the FP64 CPU oracle on a bounded
sample of the same workload instead.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "coupled 2-comp D3Q19 MLUPS & HBM-roofline %; replica p50/p99 latency"
UNIT = "MLUPS"
HBM_FALLBACK_GBS = 6800.0
HBM_NOMINAL_GBS = 7900.0
# DRAM bytes per node moved by the lattice update (dram__bytes_read + dram__bytes_write of one ncu
# capture of the bench's own 256^3 launch, per node), per (storage, lattice passes): one-pass FP32
# 2706.7 + 2717.8 MB, two-pass FP32 2690.3 + 2515.6 MB, FP16 1479.4 + 1299.3 MB, BF16 1479.5 +
# 1299.2 MB (a metric set that takes one ncu pass, so the full-size launch is captured).
COLLIDE_TRAFFIC_BYTES_PER_NODE = {("fp32", 1): 323.3, ("fp32", 2): 310.3, ("bf16", 2): 165.6, ("fp16", 2): 165.6}
# The fluctuating MRT update is bound by instruction issue, not by HBM: warp instructions per
# node of k_collide<float, true, true> (smsp__inst_executed.sum / nodes of one ncu capture of the
# 128^3 case), and the issue peak of the GPU: one warp instruction per cycle per scheduler, 4
# schedulers per SM, 152 SMs, at the SM clock.
MRT_WARP_INSTR_PER_NODE = 49.55
MRT_TRAFFIC_BYTES_PER_NODE = 289.7  # DRAM bytes per node of the same capture (160.3 read + 129.4 written)
SMS, SCHEDULERS_PER_SM = 152, 4

# The slab/droplet workload uses the density scale of the paper's ferrofluid example (Sec. 4.5):
# mean density 78.4 per component with g = 0.0214 (g rho = 1.68).  Bulk coexistence of F_bulk
# (Eq. fbulk) at g rho = 1.68 with rho_A + rho_B = 2 rho: log(rho_hi / rho_lo) = g (rho_hi - rho_lo)
# -> rho_hi / rho = 1.9103, rho_lo / rho = 0.0897.
RHO_SCALE = 78.4
G_COUPLING = 0.0214
RHO_HI, RHO_LO = 1.9103 * RHO_SCALE, 0.0897 * RHO_SCALE
# The 32^3 noise workload keeps the densities 1 +- 0.01 with g = 1.4: from noise at g rho = 1.68
# the spinodal decomposition drives the minority density negative near step 175 (FP64 oracle and
# this library alike); at 1.4 it stays positive through 1000 steps.
G_NOISE = 1.4
PARTICLE_MASS = 200.0

WORKLOADS = {
    # name: (edge, particles, description)
    "slab_droplets_256": (256, 20000, "256^3 two-component LB FP32, flat slab + 8 droplets (R 8-32), "
                                      "2e4 solvation-coupled point particles (kappa_A=-0.001, kappa_B=-0.002, gamma=1, "
                                      "m=200, kT=0.01), WCA, mean density 78.4 per component, g=0.0214"),
    "noise_32": (32, 64, "32^3 two-component LB FP32, rho=1+-0.01, g=1.4, 64 friction-coupled particles, WCA"),
    "chains_512": (512, 50000, "512^3 two-component LB FP32 demixing from 50/50 noise (mean density 78.4 per "
                                "component, g rho 1.4), 1000 bead-spring chains of 50 beads (FENE k=30 kT R0=1.5 plus WCA "
                                "eps=kT, charges +1 / -1 by chain, screened Coulomb lB=1 kappa_D=1/4 rc=3), friction + "
                                "solvation "
                                "(kappa_A = -kappa_B = -5e-4 kT, lambda_A = 0.01 kT), m=100, kT=0.01"),
    "replicas_24": (0, 0, "24 independent replicas of the serving distribution (edge 16..128, 0..5000 particles, "
                          "g rho 1.2..2.1 from a coexistence slab, gamma 0.1..2) advanced together in shared "
                          "graph-captured launches, autotuned"),
}


STORAGES = {"fp32": (0, 4), "fp16": (1, 2), "bf16": (2, 2)}  # name: (LBMD_STORAGE_*, bytes per value)

# Errors of the 16-bit storages against the FP64 oracle, as measured (one GB300 run) by the GPU
# tests of tests/test_gpu_precision.py, which assert bounds above these values: the 10-step
# population error, the Laplace pressure jump of 3-D droplets (64^3, R = 8, 12, 16, 1000 steps;
# largest relative error) and the fitted 2 gamma, the position of flat interfaces relaxing from
# off-coexistence densities (lattice units, after 500 / 2000 steps) and the particle MSD over
# 1000 steps (relative).
PRECISION_ERRORS = {
    "fp16": {"population_10_steps": 1.9e-6, "laplace_dp_3d": 0.0229, "laplace_2gamma_3d": 0.0368,
             "interface_position_500_steps": 0.0013, "interface_position_2000_steps": 0.1849,
             "msd_1000_steps": 1.8e-8, "measured_by": "tests/test_gpu_precision.py"},
    "bf16": {"population_10_steps": 1.2e-5, "laplace_dp_3d": 0.1309, "laplace_2gamma_3d": 0.0710,
             "interface_position_500_steps": 0.2666, "interface_position_2000_steps": 1.5863,
             "msd_1000_steps": 1.18e-6, "measured_by": "tests/test_gpu_precision.py"},
}


def onepass_min_bytes_per_site(storage: str = "fp32") -> int:
    """The one-pass minimum of a site update: both components' populations read and written
    once, 2 * 19 * 4 * 2 = 304 B in FP32 and 2 * 19 * 2 * 2 = 152 B with 16-bit storage."""
    return 2 * 19 * STORAGES[storage][1] * 2


def algorithmic_bytes_per_site(storage: str = "fp32", passes: int = 2) -> int:
    """Algorithmic bytes per node of the lattice update kernel: both components' populations read
    (pull) and written once, plus the node's two FP32 densities of the Shan-Chen stencil (8; the
    neighbours' come from cache), and for the one-pass update the next step's densities it writes
    (8).  FP32: 2*19*4*2 + 8 = 312 (+ 8 = 320 in one pass).  16-bit storage: the 18 moving
    populations in 2 bytes and the rest population in FP32, 2*(18*2 + 4)*2 + 8 = 168 (+ 8)."""
    b = STORAGES[storage][1]
    extra = 8 if passes == 1 else 0
    if b == 4:
        return 2 * 19 * 4 * 2 + 8 + extra
    return 2 * (18 * b + 4) * 2 + 8 + extra


def measured_hbm_peak():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        d = json.load(open(p))
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return HBM_FALLBACK_GBS, "fallback"


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 500 ms during the timed region (a
    query stalls host-side launches briefly, so the timed region is kept long)."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines = []
        self.thread = None

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.FIELDS,
                                          "--format=csv,noheader,nounits", "-lms", "500"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None
            return

        def rd():
            for line in self.proc.stdout:
                self.lines.append(line.strip())

        self.thread = threading.Thread(target=rd, daemon=True)
        self.thread.start()

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        if self.thread:
            self.thread.join(timeout=2)
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 7:
                continue
            try:
                sm.append(float(parts[0]))
                smax.append(float(parts[1]))
            except ValueError:
                continue
            for n, v in zip(names, parts[3:7]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(smax), "reasons": sorted(reasons),
                "samples": len(sm)}


def max_over_ranks(seconds: float, dist=None, device="cpu") -> float:
    """The slowest rank's time (every rank passes its own); the job finishes when it does."""
    if dist is None:
        return float(seconds)
    import torch
    t = torch.tensor([seconds], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(units_per_rank: float, world: int, seconds_max: float) -> float:
    """Units processed by all ranks (independent replicas: the same work on each) per second of
    the slowest rank."""
    return world * units_per_rank / seconds_max


# Chains of the 512^3 workload, with the interactions of the paper's polyelectrolyte example
# (Sec. 4.4) stated in units of kT: WCA with sigma = 1 and eps = kT between every pair, screened
# Coulomb with Bjerrum length 1 (prefactor lB kT), screening length 4 and a 3-cell cut-off,
# Kremer-Grest FENE bonds (k = 30 kT, R0 = 1.5) for the chain connectivity, solvation couplings
# kappa_A = -kappa_B = -5e-4 kT and lambda_A = 0.01 kT.  Beads of mass 100 (gamma dt / m = 0.01,
# Sec. 3); their contacts at a few kT stay far inside the explicit integrator's stability range
# at dt = 1, so one particle update per lattice step (--md-substeps raises it).
CHAIN_LEN, CHAIN_MASS, CHAIN_KT = 50, 100.0, 0.01
G_CHAINS = 1.4 / RHO_SCALE


def chain_model(kT: float = CHAIN_KT):
    """Particle type (kappa_A, kappa_B, lambda_A, lambda_B, gamma, mass), WCA (eps, sigma),
    screened Coulomb (lB kT, kappa_D, rc) and FENE (k, R0) of the chains workload."""
    return dict(type=(-5e-4 * kT, 5e-4 * kT, 0.01 * kT, 0.0, 1.0, CHAIN_MASS), wca=(kT, 1.0),
                dh=(1.0 * kT, 0.25, 3.0), fene=(30.0 * kT, 1.5))


def build_workload(name: str, seed: int, edge_override: int = 0):
    """dims, rho_A, rho_B, positions, types, kT, g and a dict of extras (bonds, charges,
    screened Coulomb, substeps) of a bench workload."""
    from paper_1306_0788_gb300 import inputs
    edge, npart, _ = WORKLOADS[name]
    if edge_override:
        npart = max(1, int(round(npart * (edge_override / edge) ** 3)))
        edge = edge_override
    dims = (edge, edge, edge)
    extra = {}
    if name == "chains_512":
        rA, rB = inputs.uniform_noise(dims, RHO_SCALE, 0.01 * RHO_SCALE, seed=seed)
        nch = max(2, npart // CHAIN_LEN)
        x, bonds, q = inputs.bead_spring_chains(nch, CHAIN_LEN, dims, bond=0.97, seed=seed + 1, min_dist=1.0)
        cm = chain_model()
        extra = dict(bonds=bonds, q=q, dh=cm["dh"], fene=cm["fene"], wca=cm["wca"])
        return dims, rA.astype(np.float32), rB.astype(np.float32), x, [cm["type"]], CHAIN_KT, G_CHAINS, extra
    if name == "slab_droplets_256":
        rA, rB, drops = inputs.slab_and_droplets(dims, RHO_HI, RHO_LO, n_drops=8, r_min=edge / 32,
                                                 r_max=edge / 8, width=4.0, seed=seed)
        # mass 200: gamma dt / m = 0.005 << 1 (Sec. 3) and WCA contacts stay inside the
        # stability range of the explicit integrator at dt = 1
        types = [(-0.001, -0.002, 0.0, 0.0, 1.0, PARTICLE_MASS)]
        kT, g = 0.01, G_COUPLING
    else:
        rA, rB = inputs.uniform_noise(dims, 1.0, 0.01, seed=seed)
        types = [(0.0, 0.0, 0.0, 0.0, 1.0, 1.0)]
        kT, g = 1e-4, G_NOISE
    x = inputs.random_particles(npart, dims, 2 ** (1 / 6), seed=seed + 1)
    return dims, rA.astype(np.float32), rB.astype(np.float32), x, types, kT, g, extra


def run_batch(args):
    """The batched step: one batch of 24 replicas of the serving distribution, K steps in
    graph-captured shared launches after autotuning; value = site updates per second."""
    import torch
    from paper_1306_0788_gb300 import inputs, serving
    from paper_1306_0788_gb300 import lbmd as L
    torch.cuda.set_device(0)
    reqs = inputs.serving_requests(args.replicas, rate=1.0, seed=2025, steps=args.steps + args.warmup + 10)
    sites = sum(r["edge"] ** 3 for r in reqs)
    with serving.Server(max_slots=64, chunk=25) as srv:
        b = srv.batch
        slots = [serving.admit(b, r) for r in reqs]
        L.lbmd_batch_step(b, args.warmup)
        L.lbmd_batch_poll(b, 64)
        if args.batch_config:  # a fixed launch shape instead of the autotuner's (profiling)
            L.lbmd_batch_set_config(b, *args.batch_config)
            cfg, ms = L.lbmd_batch_get_config(b), None
        else:
            cfg, ms = L.lbmd_batch_tune(b)
        L.lbmd_batch_step(b, 3)
        L.lbmd_batch_poll(b, 64)
        n0 = L.lbmd_batch_launch_count(b)
        sampler = ClockSampler(0)
        sampler.start()
        time.sleep(0.3)
        t0 = time.perf_counter()
        L.lbmd_batch_step(b, args.steps)
        st = L.lbmd_batch_poll(b, 64)
        dt = time.perf_counter() - t0
        clocks = sampler.stop()
        launches = L.lbmd_batch_launch_count(b) - n0
        failed = int((st[slots] == L.LBMD_SLOT_FAILED).sum())
    out = {"metric": METRIC, "value": round(sites * args.steps / dt / 1e6, 3), "unit": UNIT, "n_gpus": 1,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(dt / args.steps * 1e3, 5),
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
           "config": {"workload": "replicas_%d" % len(reqs), "description": WORKLOADS["replicas_24"][2].replace("24", str(len(reqs)), 1), "replicas": len(reqs),
                      "sites": sites, "particles": sum(r["np"] for r in reqs), "tuned": cfg,
                      "tuned_kernel_ms": ms, "timing": "host wall clock around lbmd_batch_step + lbmd_batch_poll"},
           "gpu_launches": int(launches), "clocks": clocks, "state_ok": failed == 0}
    print(json.dumps(out), flush=True)


def measure_single(workload: str, storage: str = "fp32", collision: str = "bgk", md_substeps: int = 1,
                   launch: str = "graph", steps: int = 20, warmup: int = 5, edge: int = 0, e2e: bool = True,
                   rank: int = 0, world: int = 1, dist=None, passes: int = 0):
    """One single-lattice measurement: warm-up, K timed steps between CUDA events on the context's
    stream (clocks sampled meanwhile), the update kernel's own event times, and optionally the
    end-to-end run through the C ABI with pinned host buffers.  Returns a dict of raw numbers."""
    import torch
    from paper_1306_0788_gb300 import lbmd as L

    dev = torch.cuda.current_device()
    stream = torch.cuda.Stream()
    dims, rA, rB, x, types, kT, g_ab, extra = build_workload(workload, seed=1234 + rank, edge_override=edge)
    npart = len(x)
    N = dims[0] * dims[1] * dims[2]
    rho0 = (float(rA.mean()), float(rB.mean()))  # shift reference of the 16-bit storages
    mrt = collision == "mrt"
    prm = L.params(dims, tau_r=1.0, g_AB=g_ab, kT=kT, seed=42 + rank, storage=STORAGES[storage][0], rho0=rho0,
                   collision=L.LBMD_COLLISION_MRT if mrt else L.LBMD_COLLISION_BGK, md_substeps=md_substeps)
    ctx, _ = L.lbmd_create(prm, stream)
    L.lbmd_set_graphs(ctx, launch == "graph")
    if passes:
        L.lbmd_set_lattice_passes(ctx, passes)
    lattice_passes = L.lbmd_get_lattice_passes(ctx)
    L.lbmd_set_types(ctx, [L.lbmd_ptype(*t) for t in types], [L.lbmd_pair(0, 0, *extra.get("wca", (1.0, 1.0)))])
    if "dh" in extra:
        L.lbmd_set_debye_hueckel(ctx, *extra["dh"])
    L.lbmd_init_fluid(ctx, rA, rB)
    L.lbmd_set_particles(ctx, x, np.zeros_like(x), np.zeros(npart, dtype=np.int32), extra.get("q"))
    if "bonds" in extra:
        L.lbmd_set_bonds(ctx, extra["bonds"], L.LBMD_BOND_FENE, *extra["fene"])

    def barrier():
        torch.cuda.synchronize()
        if dist is not None:
            dist.barrier()

    # warm-up (the graphs replayed in the timed region are recorded here)
    L.lbmd_step(ctx, warmup)
    barrier()
    launches0 = L.lbmd_launch_count(ctx)
    sampler = ClockSampler(dev)
    sampler.start()
    time.sleep(0.3)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    barrier()
    with torch.cuda.stream(stream):
        e0.record(stream)
        L.lbmd_step(ctx, steps)
        e1.record(stream)
    barrier()
    ms = e0.elapsed_time(e1)
    launches = L.lbmd_launch_count(ctx) - launches0
    # the update kernel's own duration: a second run with timing events around every update (on
    # the context's stream, inside the graphs; kept out of the step timing above, whose graphs
    # carry no events), warmed up the same way
    L.lbmd_profile_enable(ctx, True)
    L.lbmd_step(ctx, max(warmup, 3))
    barrier()
    L.lbmd_profile_read(ctx, reset=True)
    L.lbmd_step(ctx, min(steps, 300))
    barrier()
    clocks = sampler.stop()
    k_ms, k_n = L.lbmd_profile_read(ctx, reset=True)
    L.lbmd_profile_enable(ctx, False)
    state_ok = True
    try:
        L.lbmd_sync(ctx)
    except L.LbmdError:
        state_ok = False
    ms_max = max_over_ranks(ms, dist, "cuda")

    # end-to-end through the public API with host buffers (pinned), copies inside the timed region
    e2e_out = None
    if e2e:
        pin = lambda a: torch.from_numpy(np.ascontiguousarray(a)).pin_memory().numpy()  # noqa: E731
        hA, hB = pin(rA), pin(rB)
        hx, hv = pin(x.astype(np.float64)), pin(np.zeros_like(x, dtype=np.float64))
        ht = pin(np.zeros(npart, dtype=np.int32))
        outA, outB = pin(np.empty_like(rA)), pin(np.empty_like(rB))
        outU = pin(np.empty(rA.shape + (3,), dtype=np.float32))
        ox, ov, of = (pin(np.empty((npart, 3))) for _ in range(3))
        import ctypes
        p = lambda a: a.ctypes.data_as(ctypes.c_void_p)  # noqa: E731
        lib = L._lib
        barrier()
        t0 = time.perf_counter()
        rc = lib.lbmd_init_fluid(ctx, p(hA), p(hB), None)
        hq = pin(np.asarray(extra["q"], dtype=np.float64)) if "q" in extra else None
        rc |= lib.lbmd_set_particles(ctx, npart, p(hx), p(hv), p(ht), None if hq is None else p(hq))
        rc |= lib.lbmd_step(ctx, steps)
        rc |= lib.lbmd_get_fields(ctx, p(outA), p(outB), p(outU))
        rc |= lib.lbmd_get_particles(ctx, p(ox), p(ov), p(of))
        barrier()
        t_e2e = time.perf_counter() - t0
        h2d = (2 * N * 4 + npart * (6 * 8 + 4 + (8 if "q" in extra else 0))) / steps
        d2h = (5 * N * 4 + npart * 9 * 8) / steps
        e2e_out = {"value": round(whole_job_rate(N * steps, world, max_over_ranks(t_e2e, dist, "cuda")) / 1e6, 3),
                   "unit": UNIT,
                   "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(d2h), "status": int(rc),
                   "what": "lbmd_init_fluid + lbmd_set_particles (pinned host) + lbmd_step(K) + "
                           "lbmd_get_fields + lbmd_get_particles (pinned host), wall clock"}
    L.lbmd_destroy(ctx)
    return dict(dims=dims, N=N, npart=npart, kT=kT, g=g_ab, extra=extra, ms=ms_max, steps=steps,
                kernel_ms=k_ms / max(k_n, 1), kernel_launches=k_n, launches=launches, clocks=clocks,
                state_ok=state_ok, e2e=e2e_out, storage=storage, mrt=mrt, workload=workload,
                lattice_passes=lattice_passes)


def collide_roofline(m, peak, peak_kind):
    """Roofline of the lattice update kernel alone (HBM; the issue rate for the MRT update)."""
    N = m["N"]
    bps = algorithmic_bytes_per_site(m["storage"], m["lattice_passes"])
    achieved = bps * N / (m["kernel_ms"] * 1e-3) / 1e9
    if m["mrt"]:
        clk = m["clocks"].get("sm_mhz") or 2070.0
        issue_peak = SMS * SCHEDULERS_PER_SM * clk * 1e6
        issued = MRT_WARP_INSTR_PER_NODE * N / (m["kernel_ms"] * 1e-3)
        return {"bound": "alu", "scope": "kernel only (the lattice update)",
                "kernel": "k_collide (pull streaming + Shan-Chen + coupling gather + fluctuating MRT with Philox "
                          "noise, both components)",
                "achieved": round(issued / 1e12, 4), "peak": round(issue_peak / 1e12, 4),
                "peak_kind": "derived: 152 SMs x 4 schedulers x 1 warp instruction per cycle x the median SM "
                             "clock under load", "unit": "T warp-instructions/s",
                "frac": round(issued / issue_peak, 4), "instructions_per_node": MRT_WARP_INSTR_PER_NODE,
                "kernel_ms": round(m["kernel_ms"], 5), "kernel_launches": m["kernel_launches"],
                "hbm_frac": round(achieved / peak, 4),
                "traffic": int(MRT_TRAFFIC_BYTES_PER_NODE * N) if m["storage"] == "fp32" else None}
    onep = m["lattice_passes"] == 1
    return {"bound": "hbm", "scope": "kernel only (the lattice update)",
            "kernel": ("k_collide_onepass (pull streaming + Shan-Chen + coupling gather + BGK/forcing, both components, "
                       "and the next step's densities)" if onep else
                       "k_collide (pull streaming + Shan-Chen + coupling gather + BGK/forcing, both components)"),
            "achieved": round(achieved, 1), "peak": peak, "peak_kind": peak_kind, "unit": "GB/s",
            "frac": round(achieved / peak, 4), "bytes_per_site": bps,
            "frac_on_onepass_min_bytes": round(onepass_min_bytes_per_site(m["storage"]) * N / (m["kernel_ms"] * 1e-3) / 1e9 / peak, 4),
            "kernel_ms": round(m["kernel_ms"], 5), "kernel_launches": m["kernel_launches"],
            "traffic": (None if (m["storage"], m["lattice_passes"]) not in COLLIDE_TRAFFIC_BYTES_PER_NODE
                        else int(COLLIDE_TRAFFIC_BYTES_PER_NODE[(m["storage"], m["lattice_passes"])] * N))}


def step_roofline(m, peak):
    """The whole coupled step against the one-pass minimum of the lattice update (populations read
    and written once: 304 B per site in FP32, 152 B with 16-bit storage), against the measured
    copy bandwidth and the nominal 7.9 TB/s."""
    bps = onepass_min_bytes_per_site(m["storage"])
    achieved = bps * m["N"] / (m["ms"] / m["steps"] * 1e-3) / 1e9
    return {"bound": "hbm", "scope": "whole coupled step (every kernel, particles included)",
            "bytes_per_site": bps, "achieved": round(achieved, 1), "unit": "GB/s",
            "frac": round(achieved / peak, 4), "frac_of_nominal_7900": round(achieved / HBM_NOMINAL_GBS, 4)}


def sub_record(m, peak, peak_kind, label):
    """A further configuration measured in the same run, timed like the headline."""
    ms_step = m["ms"] / m["steps"]
    return {"config": {"workload": label, "lattice": list(m["dims"]), "particles": m["npart"],
                       "storage": m["storage"], "bonds": int(len(m["extra"].get("bonds", []))),
                       "lattice_passes": m["lattice_passes"]},
            "value": round(m["N"] / (ms_step * 1e-3) / 1e6, 3), "unit": UNIT, "steps": m["steps"],
            "ms_per_step": round(ms_step, 5), "roofline": collide_roofline(m, peak, peak_kind),
            "step_roofline": step_roofline(m, peak), "gpu_launches": int(m["launches"]),
            "clocks": m["clocks"], "state_ok": m["state_ok"]}


def run_cuda(args):
    if args.workload == "replicas_24":
        return run_batch(args)
    import torch

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    dist = None
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    else:
        torch.cuda.set_device(0)

    m = measure_single(args.workload, args.storage, args.collision, args.md_substeps, args.launch, args.steps,
                       args.warmup, args.edge, not args.no_e2e, rank, world, dist, args.passes)
    peak, peak_kind = measured_hbm_peak()
    N, ms_max = m["N"], m["ms"]
    value = whole_job_rate(N * args.steps, world, ms_max * 1e-3) / 1e6
    if rank == 0:
        out = {
            "metric": METRIC, "value": round(value, 3), "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": round(ms_max / args.steps, 5), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None,
            "dtype": "f32" if args.storage == "fp32" else "f32 arithmetic, %s shifted population storage" % args.storage,
            "data": "synthetic",
            "config": {"workload": args.workload + ("" if not args.edge else "@%d" % args.edge),
                       "md_substeps": args.md_substeps, "bonds": int(len(m["extra"].get("bonds", []))),
                       "description": WORKLOADS[args.workload][2],
                       "lattice": list(m["dims"]), "particles": m["npart"], "tau_r": 1.0, "g_AB": m["g"],
                       "kT": m["kT"], "storage": args.storage, "launch": args.launch,
                       "lattice_passes": m["lattice_passes"],
                       "collision": ("fluctuating MRT (Eq. MODES), eigenvalues -1, fluid noise at kT"
                                     if m["mrt"] else "BGK"),
                       "parallelism": "replicas" if world > 1 else "single",
                       "l2": "inputs larger than L2 (populations %.2f GB per buffer)" % (N * 152 / 1e9)
                       if N * 152 > 129e6 else "L2-resident lattice (latency regime)"},
            "roofline": collide_roofline(m, peak, peak_kind),
            "step_roofline": step_roofline(m, peak),
            "gpu_launches": int(m["launches"]), "e2e": m["e2e"], "clocks": m["clocks"], "state_ok": m["state_ok"],
        }
        if world == 1 and not args.no_extras:
            ext_steps = max(args.steps, 100)
            if args.workload == "slab_droplets_256" and args.storage == "fp32" and not m["mrt"] and not args.edge:
                for st in ("fp16", "bf16"):
                    ms16 = measure_single("slab_droplets_256", st, steps=ext_steps, warmup=args.warmup, e2e=False)
                    rec = sub_record(ms16, peak, peak_kind, "slab_droplets_256 (%s shifted storage)" % st)
                    rec["speedup_vs_fp32"] = round((ms_max / args.steps) / rec["ms_per_step"], 4)
                    rec["update_speedup_vs_fp32"] = round(m["kernel_ms"] / ms16["kernel_ms"], 4)
                    rec["errors_vs_fp64_oracle"] = PRECISION_ERRORS[st]
                    out["storage_" + st] = rec
            if args.workload != "chains_512" and not args.edge:
                mc = measure_single("chains_512", "fp32", steps=max(args.steps, 30), warmup=args.warmup, e2e=False)
                out["chains_512"] = sub_record(mc, peak, peak_kind, "chains_512")
        if world == 1 and args.serving > 0:
            out["serving"] = run_serving(args.serving)
        if world == 1 and not args.no_cpu_baseline:
            out["cpu_baseline"] = cpu_baseline(args.workload, budget_s=args.cpu_seconds, md_substeps=args.md_substeps)
        print(json.dumps(out), flush=True)
    if dist is not None:
        dist.barrier()
        dist.destroy_process_group()


def run_serving(n_requests: int, load: float = 0.8, chunk: int = 25, seed: int = 2024):
    """Replica serving (continuous batching): a Poisson stream of independent replicas --
    cubic lattices with edge uniform in 16..128, 0..5000 particles (capped by the packing of the
    box), g rho uniform in [1.2, 2.1] from a flat interface at coexistence, gamma uniform in
    [0.1, 2], 1000 steps each -- admitted by device memory into one batch and advanced in shared
    graph-captured launches.  The arrival rate is `load` times the batch's saturated capacity,
    measured first on a sample of the same distribution (which also runs the autotuner)."""
    from paper_1306_0788_gb300 import inputs, serving
    steps = 1000
    with serving.Server(max_slots=4096, chunk=chunk) as srv:
        sample = inputs.serving_requests(24, rate=1.0, seed=seed + 1)
        cal = srv.calibrate(sample)
        per_replica = serving.mean_sites() * steps
        capacity = cal["site_updates_per_s"] / per_replica  # replicas per second
        rate = load * capacity
        reqs = inputs.serving_requests(n_requests, rate=rate, seed=seed)
        sampler = ClockSampler(0)
        sampler.start()
        t0 = time.perf_counter()
        records, peak = srv.run(reqs)
        wall = time.perf_counter() - t0
        clocks = sampler.stop()
        info = serving.summarize(records)
    info.update({
        "stream": "%d Poisson arrivals at %.2f/s (%.0f %% of the measured capacity %.2f replicas/s); edge U{16..128}, "
                  "particles U{0..5000} capped at half the 2.5-cells, g rho U[1.2, 2.1] (flat interface at coexistence), "
                  "gamma U[0.1, 2], %d steps each"
                  % (n_requests, rate, 100 * load, capacity, steps),
        "metric": "time-to-%d-steps, arrival to completion" % steps,
        "capacity_site_updates_per_s": cal["site_updates_per_s"], "tuned": cal["config"],
        "tuned_kernel_ms": cal["kernel_ms"], "chunk_steps": chunk, "wall_s": wall,
        "peak_device_bytes": peak["peak_bytes"], "peak_replicas": peak["peak_replicas"],
        "admissions_refused": peak["refusals"], "clocks": clocks,
        "config": {"workload": "serving_stream_%d" % n_requests}})
    return {k: (round(v, 4) if isinstance(v, float) else v) for k, v in info.items()}


def oracle_sample(workload: str, edge: int, seed: int, md_substeps: int = 1):
    """A bounded sample of the workload for the CPU oracle: an edge^3 box with the same
    particle density (at least one whole chain for the chains workload) and the same fluid
    recipe and interactions."""
    import oracle
    from paper_1306_0788_gb300 import inputs
    full_edge, npart_full, _ = WORKLOADS[workload]
    dims = (edge, edge, edge)
    n = max(1, int(round(npart_full * (edge / full_edge) ** 3)))
    extra = {}
    if workload == "chains_512":
        rA, rB = inputs.uniform_noise(dims, RHO_SCALE, 0.01 * RHO_SCALE, seed=seed)
        cm = chain_model()
        nch = max(1, int(round(n / CHAIN_LEN)))
        x, bonds, q = inputs.bead_spring_chains(nch, CHAIN_LEN, dims, bond=0.97, seed=seed + 1, min_dist=1.0)
        n = len(x)
        ka, kb, la, lb, _, m = cm["type"]
        kap, lam, kT, g, eps = np.array([[ka, kb]]), np.array([[la, lb]]), CHAIN_KT, G_CHAINS, cm["wca"][0]
        extra = dict(q=np.asarray(q, dtype=np.float64), bonds=np.asarray(bonds, dtype=np.int32), bond_k=cm["fene"][0],
                     bond_r=cm["fene"][1], dh_lB=cm["dh"][0], dh_kappa=cm["dh"][1], dh_rc=cm["dh"][2])
    elif workload == "slab_droplets_256":
        rA, rB, _ = inputs.slab_and_droplets(dims, RHO_HI, RHO_LO, n_drops=1, r_min=edge / 8, r_max=edge / 8,
                                             width=4.0, seed=seed)
        kap, lam, kT, g, m, eps = np.array([[-0.001, -0.002]]), np.zeros((1, 2)), 0.01, G_COUPLING, PARTICLE_MASS, 1.0
    else:
        rA, rB = inputs.uniform_noise(dims, 1.0, 0.01, seed=seed)
        kap, lam, kT, g, m, eps = np.zeros((1, 2)), np.zeros((1, 2)), 1e-4, G_NOISE, 1.0, 1.0
    if workload != "chains_512":
        x = inputs.random_particles(n, dims, 2 ** (1 / 6), seed=seed + 1)
        extra = dict(q=np.zeros(n))
    s = oracle.System(dims=dims, tau_r=1.0, g_AB=g, g_BA=g, kT=kT, seed=42,
                      kappa=kap, lam=lam, gamma=np.ones(1), mass=np.array([m]),
                      wca_eps=np.full((1, 1), eps), wca_sig=np.ones((1, 1)), type=np.zeros(n, dtype=np.int32),
                      md_substeps=md_substeps, **extra)
    f = oracle.init_equilibrium(rA.astype(np.float32).astype(np.float64), rB.astype(np.float32).astype(np.float64))
    return s, f, x.copy(), np.zeros((n, 3)), n


def cpu_baseline(workload: str, budget_s: float = 15.0, edge: int = 32, md_substeps: int = 1):
    """The FP64 oracle as it stands, single-threaded, on a bounded sample (edge^3 with the
    workload's particle density), timed for about budget_s seconds."""
    import oracle
    s, f, x, v, n = oracle_sample(workload, edge, seed=7, md_substeps=md_substeps)
    oracle.step(s, f, x, v, 0)  # load and warm
    steps = 0
    t0 = time.perf_counter()
    while time.perf_counter() - t0 < budget_s:
        oracle.step(s, f, x, v, 1 + steps)
        steps += 1
    dt = time.perf_counter() - t0
    return {"value": round(edge ** 3 * steps / dt / 1e6, 4), "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": "%d^3 lattice, %d particles (same density and recipe), %d steps, %.1f s" % (edge, n, steps, dt)}


def run_reference(args):
    """The oracle arm: rank 0 times the FP64 CPU oracle, K steps of a bounded sample."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    import oracle
    # size the sample so that warm-up + K steps take about two minutes at ~0.3 MLUPS
    sites = max(8 ** 3, min(32 ** 3, int(0.3e6 * 120.0 / max(args.steps + args.warmup, 1))))
    edge = max(8, int(round(sites ** (1 / 3))))
    s, f, x, v, n = oracle_sample(args.workload, edge, seed=7, md_substeps=args.md_substeps)
    for k in range(args.warmup):
        oracle.step(s, f, x, v, k)
    t0 = time.perf_counter()
    for k in range(args.steps):
        oracle.step(s, f, x, v, args.warmup + k)
    dt = time.perf_counter() - t0
    value = edge ** 3 * args.steps / dt / 1e6
    out = {"impl": "reference", "metric": METRIC, "value": round(value, 4), "unit": UNIT, "n_gpus": 0,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(dt / args.steps * 1e3, 3),
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
           "config": {"workload": args.workload, "description": WORKLOADS[args.workload][2],
                      "sample": "%d^3 lattice, %d particles" % (edge, n)},
           "cpu_baseline": {"value": round(value, 4), "unit": UNIT, "cores": 1, "kind": "oracle",
                            "sample": "%d^3 lattice, %d particles, %d steps" % (edge, n, args.steps)},
           "e2e": {"value": round(value, 4), "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=1000)
    ap.add_argument("--warmup", type=int, default=20)
    ap.add_argument("--impl", choices=["cuda", "reference"], default="cuda")
    ap.add_argument("--workload", choices=sorted(WORKLOADS), default="slab_droplets_256")
    ap.add_argument("--edge", type=int, default=0, help="override the lattice edge (profiling of smaller cases)")
    ap.add_argument("--storage", choices=sorted(STORAGES), default="fp32",
                    help="population storage: FP32, or FP16 / BF16 shifted by w_i rho0 (FP32 arithmetic)")
    ap.add_argument("--collision", choices=["bgk", "mrt"], default="bgk",
                    help="BGK, or the fluctuating MRT collision with fluid noise at the workload's kT")
    ap.add_argument("--md-substeps", type=int, default=1, help="particle substeps per lattice step")
    ap.add_argument("--launch", choices=["graph", "stream"], default="graph",
                    help="lbmd_step launch mode: replayed two-step graphs, or every kernel one by one")
    ap.add_argument("--passes", type=int, choices=[0, 1, 2], default=0,
                    help="lattice update: 0 = chosen by the lattice size, 1 = one pass, 2 = density pass + update")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-seconds", type=float, default=15.0)
    ap.add_argument("--replicas", type=int, default=24, help="replicas of the replicas_24 workload")
    ap.add_argument("--batch-config", type=lambda v: [int(t) for t in v.split(",")], default=None,
                    help="tile_sites,grid_moments,grid_collide,collide_blocks: fixed batch launch shape, no autotuning")
    ap.add_argument("--serving", type=int, default=2000,
                    help="replicas in the serving stream measured after the main run (0 = skip)")
    ap.add_argument("--no-extras", action="store_true",
                    help="skip the further configurations (16-bit storages, 512^3 chains) after the main run")
    args = ap.parse_args()
    if args.warmup < 3:
        ap.error("--warmup must be >= 3")
    if args.impl == "reference":
        if args.workload == "replicas_24":
            ap.error("the oracle arm times the single-lattice workloads")
        run_reference(args)
    else:
        run_cuda(args)


if __name__ == "__main__":
    main()
