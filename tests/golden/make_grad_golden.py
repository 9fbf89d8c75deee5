"""Writes tests/golden/grad_two_sided.json: dT/d eps at chosen sites of the
N = 101, L = 500 ribbon (Anderson +-0.15 eV, seed 4; the gradient workload)
at three energies near the charge-neutrality point, from the oracle only
(oracle.gradient.two_sided, the closed form with Dyson-assembled blocks of G).
The sites are the largest entries, sites where a reverse sweep over column
slices loses its accuracy at these energies, and seeded random sites.  Rerun
after any change to the oracle's gradient or to the workload's inputs.
"""
import json
import sys
from pathlib import Path

import numpy as np

HERE = Path(__file__).resolve().parent
sys.path.insert(0, str(HERE.parents[1]))

from oracle import gradient  # noqa: E402
import workloads  # noqa: E402

N, L, W, SEED = 101, 500, 0.15, 4
# (index into linspace(-0.8, 0.8, 128), sites (cell, orbital) to keep)
CASES = [(61, [(107, 39)]), (64, [(290, 178)]), (69, [(429, 191)])]


def main():
    eps = workloads.anderson_onsite(N, L, W, SEED)
    Es = np.linspace(-0.8, 0.8, 128)
    rng = np.random.default_rng(2024)
    out = dict(N=N, L=L, W=W, seed=SEED, eta_device=1e-8, eta_lead=1e-8, t=-2.7, cases=[])
    for ie, extra in CASES:
        E = float(Es[ie])
        T, g = gradient.two_sided(N, L, E, 1e-8, 1e-8, -2.7, eps)
        top = np.argsort(-np.abs(g).ravel())[:3]
        sites = [tuple(map(int, np.unravel_index(f, g.shape))) for f in top] + list(extra)
        sites += [(int(rng.integers(L)), int(rng.integers(2 * N))) for _ in range(4)]
        out["cases"].append(dict(E=E, T=T, scale=float(np.abs(g).max()),
                                 sites=[[n, i, float(g[n, i])] for n, i in sites]))
        print(f"E={E:+.6f} T={T:.12f} scale={np.abs(g).max():.4e}", flush=True)
    (HERE / "grad_two_sided.json").write_text(json.dumps(out, indent=1) + "\n")


if __name__ == "__main__":
    main()
