"""Writes the stored expected values under tests/golden/ from the FP64 oracle.

Calls only oracle/ (and the seeded input generator). Run from the repo root:
    python tests/golden/make_golden.py
"""
import json
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

from oracle import fdas_oracle as O  # noqa: E402
from synthetic import workload  # noqa: E402


def main():
    T = O.thresholds(16, 6.0)
    with open(os.path.join(HERE, "thresholds_sigma6.json"), "w") as f:
        json.dump({"what": "T_h with P(Gamma(h,1) >= T_h) = Gaussian tail at 6 sigma",
                   "p": O.gaussian_tail(6.0),
                   "T": {str(h): v for h, v in T.items()}}, f, indent=1)
    x, p = workload("cfg1_n2e17_z50")
    _, _, _, cands, _ = O.search(x, p["zmax"], p["dz"], p["m"], p["nharm"], p["sigma"])
    with open(os.path.join(HERE, "cfg1_candidates.json"), "w") as f:
        json.dump({"what": "oracle candidates (r, j, h, H) of the 2^17-sample, zmax=50 workload",
                   "params": {k: v for k, v in p.items() if k != "chirps"},
                   "candidates": cands}, f, indent=1)


if __name__ == "__main__":
    main()
