"""Write the oracle's focal-plane intensity of four 256-row stripes of each
plate of the D sweep to tests/golden/.

Workloads: binary amplitude FZP, negative-centred, D = 1, 2, 3, 4, 5 m at
f/# = 5 (f = 5 D), lambda = 632.8 nm, dx = lambda f / (4 D) (Eq. 5), N forced
odd (Fig. 2 Stage 1; N = 1,264,223 ... 6,321,113), ROI 512 x 512 at pitch
lambda f/# / 8, centred on the focus.

Each plate's four stripes start at v = -128 rows from the axis (through the
centre: the longest chords), +R/2, -3R/4 and +0.9 R (short chords near the
rim); the central stripe's rows run every column through the dense form's
row pass, so its FP32 promotion sum over all N columns is exercised at every
D.  The
stored value is I = |sum over the four stripes of U|^2 from the oracle's O3
evaluation (Bluestein CZT rows then columns, FP64; Eq. 9-10, Sec. 2.6),
rounded to float32 (relative rounding 6e-8).

This script calls only ``oracle`` (no GPU code).  On 8 x86 cores it takes
about ten minutes.  Run from the repository root:

    python tests/golden/make_dsweep_oracle.py
"""
import json
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

import oracle as O  # noqa: E402

LAM = 632.8e-9
DIAMETERS = (1.0, 2.0, 3.0, 4.0, 5.0)
ROWS = 256


def geometry(D):
    return O.Geometry(D=D, f=5 * D, lam=LAM, M=512, p=LAM * 5 / 8)


def stripes(g):
    """First rows of the four stripes (see the module docstring)."""
    rR = int(g.R / g.dx)
    return [g.c - 128, g.c + rR // 2, g.c - (3 * rR) // 4, g.c + (9 * rR) // 10 - ROWS]


def path(D):
    return os.path.join(HERE, f"dsweep_d{D:g}m_stripes_I.npy")


def main():
    meta = {"what": "oracle O3 (FP64) intensity of the summed field of four 256-row stripes per plate",
            "layout": "I[n, m] at (x_m, y_n), x_m = (m - M/2) p; float32", "rows_per_stripe": ROWS,
            "script": "tests/golden/make_dsweep_oracle.py", "plates": {}}
    threads = O.max_threads()
    for D in DIAMETERS:
        g = geometry(D)
        t0 = time.time()
        U = np.zeros((g.M, g.M), complex)
        for j0 in stripes(g):
            U += O.field_czt(g, j0, j0 + ROWS, threads)
        I = np.abs(U) ** 2
        np.save(path(D), I.astype(np.float32), allow_pickle=False)
        meta["plates"][f"{D:g}"] = {"N": g.N, "c": g.c, "stripes": stripes(g), "file": os.path.basename(path(D)),
                                    "intensity_l2": float(np.linalg.norm(I)), "seconds": round(time.time() - t0, 1)}
        print(D, g.N, stripes(g), round(time.time() - t0, 1), flush=True)
    meta["oracle_threads"] = threads
    with open(os.path.join(HERE, "dsweep_stripes.json"), "w") as fh:
        json.dump(meta, fh, indent=1)
        fh.write("\n")


if __name__ == "__main__":
    main()
