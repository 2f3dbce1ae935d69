"""Write the oracle's SA-CZT field of the 8 mm exact-radii plate (the
SA-CZT bench workload) to tests/golden/.

Workload: binary amplitude FZP with the exact zone radii of Eq. 3,
negative-centred, D = 8 mm, f/# = 5 (f = 40 mm), lambda = 632.8 nm,
dx = lambda f / (4 D) (N = 10,115, forced odd), padded grid P = 16,384 (the
smallest power of two >= 1.5 N), ROI 512 x 512 at lambda f/# / 8, centred.

The field is oracle/saczt.py's FP64 evaluation of Fig. 5 (FFT2 of the padded
mask, the residual phase exp(i h f), IFFT2, the Fresnel chirp and the zoom
onto the ROI as two dense products, the prefactor), stored as complex64
(relative rounding 6e-8); its FP64 metrics go beside it.

This script calls only ``oracle`` (no GPU code); it holds a few 16,384^2
complex128 arrays (about 30 GB of host memory).  Run from the repository
root:

    python tests/golden/make_saczt_oracle.py
"""
import json
import os
import platform
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

import oracle as O  # noqa: E402
from oracle import saczt as SA  # noqa: E402

FIELD = os.path.join(HERE, "saczt_d8mm_field.npy")
META = os.path.join(HERE, "saczt_d8mm.json")


def geometry():
    lam = 632.8e-9
    return O.Geometry(D=8e-3, f=40e-3, lam=lam, M=512, p=lam * 5 / 8, kind=O.FZP_EXACT)


def main():
    g = geometry()
    assert g.N == 10115
    P = SA.pad_size(g.N)
    assert P == 16384
    t0 = time.time()
    U = SA.field_saczt(g, P)
    dt = time.time() - t0
    np.save(FIELD, U.astype(np.complex64), allow_pickle=False)
    m = O.metrics(g, U)
    meta = {
        "what": "oracle SA-CZT (Fig. 5, FP64 numpy) of the whole exact-radii plate",
        "workload": "binary FZP, exact radii, D=8 mm, f=40 mm, lambda=632.8 nm, N=10115, P=16384, ROI 512^2 "
                    "at lambda f/#/8",
        "geometry": {"D": g.D, "f": g.f, "lambda": g.lam, "dx": g.dx, "N": g.N, "M": g.M, "pitch": g.p,
                     "R": g.R, "P": P},
        "field_file": os.path.basename(FIELD),
        "field_layout": "U[n, m] at (x_m, y_n), x_m = (m - M/2) p; stored complex64",
        "metrics_fp64": {k: (v.tolist() if isinstance(v, np.ndarray) else float(v)) for k, v in m.items()},
        "oracle_seconds": round(dt, 1),
        "host": platform.machine(),
        "script": "tests/golden/make_saczt_oracle.py",
    }
    with open(META, "w") as fh:
        json.dump(meta, fh, indent=1)
        fh.write("\n")
    print(json.dumps({"oracle_seconds": meta["oracle_seconds"]}), "fwhm_x %.9e de_lobe %.9f" % (m["fwhm_x"], m["de_lobe"]))


if __name__ == "__main__":
    main()
