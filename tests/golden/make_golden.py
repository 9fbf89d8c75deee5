"""Writes tests/golden/mp_transmission.json: arbitrary-precision (mpmath, 40
digits) conductances of small armchair ribbons near the charge-neutrality
point, from the oracle only (oracle.mp).  Rerun after any change to the oracle's
recursion or decimation; the tests compare the complex128 oracle against it.
"""
import json
import sys
from pathlib import Path

HERE = Path(__file__).resolve().parent
sys.path.insert(0, str(HERE.parents[1]))

from oracle import mp  # noqa: E402
import workloads  # noqa: E402

CASES = [
    # (name, N, L, W, seed, E, eta_device, eta_lead)
    ("agnr11_L10_pristine_E0", 11, 10, 0.0, 0, 0.0, 1e-8, 1e-8),
    ("agnr11_L10_pristine_E1e-4", 11, 10, 0.0, 0, 1e-4, 1e-8, 1e-8),
    ("agnr5_L8_anderson_E0", 5, 8, 0.25, 7, 0.0, 1e-8, 1e-8),
    ("agnr5_L8_anderson_E1e-3", 5, 8, 0.25, 7, 1e-3, 1e-8, 1e-8),
]


def main():
    out = {}
    for name, N, L, W, seed, E, etad, etal in CASES:
        eps = workloads.anderson_onsite(N, L, W, seed) if W > 0 else None
        T = mp.transmission(N, L, E, etad, etal, eps=eps, dps=40)
        out[name] = dict(N=N, L=L, W=W, seed=seed, E=E, eta_device=etad, eta_lead=etal, T=T)
        print(name, repr(T))
    (HERE / "mp_transmission.json").write_text(json.dumps(out, indent=1) + "\n")


if __name__ == "__main__":
    main()
