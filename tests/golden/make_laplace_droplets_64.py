"""Writes laplace_droplets_64.json: the FP64 oracle's Laplace pressure jump of 3-D droplets.

A-rich spheres of radius R = 8, 12, 16 in B, on a 64^3 periodic lattice at the density scale of
the paper's examples (mean density 78.4 per component; bulk coexistence densities 1.9103 and
0.0897 times that, for g rho = 1.68 with F_bulk of Eq. fbulk), tanh interfaces of width 2,
BGK tau_r = 1, relaxed 1000 steps.  The pressure jump follows reading 13 of the scope: the bulk
pressure p = c_s^2 (rho_A + rho_B) + c_s^2 g rho_A rho_B at the centre node minus the corner
node (0, 0, 0).  The Laplace law (Sec. 4.3) says dp = 2 gamma / R; the fit of dp against 1/R is
stored too.  Calls only the oracle (several host threads; results do not depend on them).

    python tests/golden/make_laplace_droplets_64.py [threads]
"""
import json
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import oracle  # noqa: E402
from paper_1306_0788_gb300 import inputs  # noqa: E402

N, SCALE, STEPS, WIDTH = 64, 78.4, 1000, 2.0
G = 1.68 / SCALE
RADII = (8.0, 12.0, 16.0)
HI, LO = 1.9103 * SCALE, 0.0897 * SCALE


def pressure_jump(f):
    A, B = f[0].sum(0), f[1].sum(0)
    p = (A + B) / 3.0 + G * A * B / 3.0
    return float(p[N // 2, N // 2, N // 2] - p[0, 0, 0])


def main():
    oracle.set_threads(int(sys.argv[1]) if len(sys.argv) > 1 else os.cpu_count())
    dims = (N, N, N)
    out = {"source": __doc__.strip().splitlines()[0], "recipe": __doc__.strip(), "lattice": N, "scale": SCALE,
           "g": G, "steps": STEPS, "width": WIDTH, "radii": list(RADII), "dp": []}
    for R in RADII:
        rA, rB = inputs.sphere(dims, R, HI, LO, WIDTH)
        s = oracle.System(dims=dims, tau_r=1.0, g_AB=G, g_BA=G)
        f = oracle.init_equilibrium(rA.astype(np.float32).astype(np.float64), rB.astype(np.float32).astype(np.float64))
        x = np.zeros((0, 3))
        for k in range(STEPS):
            st, _ = oracle.step(s, f, x, x.copy(), k)
            assert st == 0
        out["dp"].append(pressure_jump(f))
        print(R, out["dp"][-1], flush=True)
    inv = 1.0 / np.array(RADII)
    slope, icept = np.polyfit(inv, np.array(out["dp"]), 1)
    out["fit"] = {"two_gamma": float(slope), "intercept": float(icept)}
    with open(os.path.join(os.path.dirname(os.path.abspath(__file__)), "laplace_droplets_64.json"), "w") as fh:
        json.dump(out, fh, indent=1)


if __name__ == "__main__":
    main()
