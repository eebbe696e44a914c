"""Write the stored expected values under tests/golden/ (calls only the oracle).

Run from the repository root:  python tests/golden/make_golden.py
Stored workloads have inputs that are bit-identical on every machine: exact
integer generators, and the uniform float generator (53-bit integer times a
power of two, one rounding to FP32), so the stored center sequences are too.
Float records hold the canonical FP32 selection and its FP64 radius, with a
SHA-256 of the points (whole, and of the first 100,000 rows) so that a change
of the generator shows before a comparison.
"""
import hashlib
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


def write_float(name, pts, k, cite, prefix_rows=100_000):
    r = O.gonzalez(pts, k, mode="f32")
    rec = {"workload": name, "cite": cite, "n": int(pts.shape[0]), "d": int(pts.shape[1]), "k": k, "first": 0,
           "mode": "canonical FP32 selection, FP64 radius",
           "points_sha256": hashlib.sha256(pts.tobytes()).hexdigest(),
           "prefix_rows": prefix_rows,
           "prefix_sha256": hashlib.sha256(pts[:prefix_rows].tobytes()).hexdigest(),
           "centers": [int(c) for c in r.centers], "sel2_f32": [float(v) for v in r.sel2],
           "radius": float(r.radius)}
    with open(os.path.join(HERE, name + ".json"), "w") as f:
        json.dump(rec, f, indent=1)
        f.write("\n")


if __name__ == "__main__":
    write("gon_int_n10000_d2_k10", I.gon_int_10k(),
          "GON, Section 3.1; int32 coordinates uniform in [0,1023], seed 0; exact int64 oracle")
    write("gon_int13_n1000000_d10_k100", I.gon_int13_1m(),
          "GON, Section 3.1; coordinates uniform on {1..13}, seed 2; exact int64 oracle")
    pts, _, _ = I.mrg_unif_10m()
    write_float("gon_unif_n10000000_d16_k32", pts, 32,
                "GON, Section 3.1; n = 10M points uniform in [0,1)^16, seed 3 (the MRG workload's points); "
                "oracle in canonical FP32 (selection) and FP64 (radius)")
