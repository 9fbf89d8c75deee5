"""Writes tests/golden/agnr245_golden.json: conductances of the W = 30 nm bench
ribbon (N = 245, M = 490 orbitals per cell, Anderson disorder +-0.25 eV from
seed 1) computed by the oracle alone (complex128, unit-cell slices):

* "L4000": the full 4000-cell ribbon at five energies of its 69-energy grid:
  -0.5 eV and the 51st grid point (about 0.294 eV), +-1 meV and +5 meV;
* "L4": the first 4 cells of the same ribbon at every grid energy except
  E = 0 (69 chains in one call is the launch configuration of the full-size
  workload);
* "L4000_E0", "L4_E0": E = 0 exactly, from oracle.rgf.transmission_modes
  (the end slices in the leads' mode basis; the full-cell decimation of
  oracle.rgf.transmission is condition-limited there).

Every other energy uses oracle.rgf.transmission with the full-cell
Sancho-Rubio decimation of oracle.leads.  About 20 minutes on 8 cores (the
4000-cell sweeps dominate); entries already in the file are kept unless
--all is given.  Rerun with --all after any change to the oracle's recursion
or decimation.
"""
import json
import sys
import time
from pathlib import Path

HERE = Path(__file__).resolve().parent
sys.path.insert(0, str(HERE.parents[1]))

import workloads  # noqa: E402
from oracle import leads, rgf  # noqa: E402

OUT = HERE / "agnr245_golden.json"
FULL_IDX = [0, 50, 65, 66, 67]     # -0.5, ~0.294, +1 meV, -1 meV, +5 meV


def main():
    w = workloads.WORKLOADS["agnr245_L4000_anderson"]
    N, W, seed = w["N"], w["W"], w["seed"]
    Es = w["energies"]()
    out = None
    if OUT.exists() and "--all" not in sys.argv:
        out = json.loads(OUT.read_text())
    if out is None:
        out = {"N": N, "W": W, "seed": seed, "eta_device": 1e-8, "eta_lead": 1e-8, "t": -2.7,
               "L4": {"L": 4, "energy_index": [], "E": [], "T": []},
               "L4000": {"L": 4000, "energy_index": [], "E": [], "T": []}}
    eps4 = workloads.anderson_onsite(N, 4, W, seed)
    t0 = time.time()
    if not out["L4"]["T"]:
        for i, e in enumerate(Es):
            if e == 0.0:
                continue
            T = rgf.transmission(N, 4, float(e), 1e-8, 1e-8, -2.7, eps4, None)
            out["L4"]["energy_index"].append(i)
            out["L4"]["E"].append(float(e))
            out["L4"]["T"].append(T)
        print(f"L4: {len(out['L4']['T'])} energies in {time.time() - t0:.0f} s", flush=True)
    i0 = int(list(Es).index(0.0))
    if "L4_E0" not in out:
        out["L4_E0"] = {"L": 4, "energy_index": i0, "E": 0.0,
                        "T": rgf.transmission_modes(N, 4, 0.0, 1e-8, 1e-8, -2.7, eps4, None)}
    eps = workloads.anderson_onsite(N, 4000, W, seed)
    for i in FULL_IDX:
        if i in out["L4000"]["energy_index"]:
            continue
        t1 = time.time()
        e = float(Es[i])
        T = rgf.transmission(N, 4000, e, 1e-8, 1e-8, -2.7, eps, None,
                             sig=leads.self_energies(N, e, 1e-8, -2.7))
        out["L4000"]["energy_index"].append(i)
        out["L4000"]["E"].append(e)
        out["L4000"]["T"].append(T)
        print(f"L4000 E={e:+.6f} T={T!r} ({time.time() - t1:.0f} s)", flush=True)
        OUT.write_text(json.dumps(out, indent=1) + "\n")
    if "L4000_E0" not in out:
        t1 = time.time()
        out["L4000_E0"] = {"L": 4000, "energy_index": i0, "E": 0.0,
                           "T": rgf.transmission_modes(N, 4000, 0.0, 1e-8, 1e-8, -2.7, eps, None)}
        print(f"L4000 E=0 T={out['L4000_E0']['T']!r} ({time.time() - t1:.0f} s)", flush=True)
    OUT.write_text(json.dumps(out, indent=1) + "\n")


if __name__ == "__main__":
    main()
