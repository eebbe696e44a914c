"""Write the stored expected values under tests/golden/ (calls only the oracle).

Run from the repository root:  python tests/golden/make_golden.py
Only integer workloads are stored: their inputs are bit-identical on every
machine (exact integer generators), so the stored center sequences are too.
"""
import json
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

from oracle import oracle as O                          # noqa: E402
from paper_1604_03228_gb300 import inputs as I         # noqa: E402

HERE = os.path.dirname(os.path.abspath(__file__))


def write(name, w, cite):
    r = O.gonzalez(w.points, w.k, first=w.first)
    rec = {"workload": name, "cite": cite, "n": int(w.points.shape[0]), "d": int(w.points.shape[1]),
           "k": w.k, "first": w.first, "centers": [int(c) for c in r.centers],
           "sel2": [int(v) for v in r.sel2], "radius2": int(r.radius2)}
    with open(os.path.join(HERE, name + ".json"), "w") as f:
        json.dump(rec, f, indent=1)
        f.write("\n")


if __name__ == "__main__":
    write("gon_int_n10000_d2_k10", I.gon_int_10k(),
          "GON, Section 3.1; int32 coordinates uniform in [0,1023], seed 0; exact int64 oracle")
    write("gon_int13_n1000000_d10_k100", I.gon_int13_1m(),
          "GON, Section 3.1; coordinates uniform on {1..13}, seed 2; exact int64 oracle")
