"""Write the oracle's full-aperture field of the 0.25 m plate (the Gsamples/s
workload of the plain FP32 form) to tests/golden/.

Workload: binary amplitude FZP, negative-centred, D = 0.25 m, f/# = 5
(f = 1.25 m), lambda = 632.8 nm, dx = lambda f / (4 D) (four samples per
outermost zone width, Eq. 5), N = 316,057 (forced odd, Fig. 2 Stage 1), ROI
512 x 512 at pitch lambda f/# / 8, centred on the focus.

The field is the oracle's O3 evaluation (Bluestein CZT over rows, then over
columns; Eq. 9-10, Sec. 2.6) over all N rows, in FP64.  It is stored as
complex64 (relative rounding 6e-8, far below the 1e-4 tolerance the GPU forms
are held to); the oracle's own FP64 metrics of the FP64 field go beside it.

This script calls only ``oracle`` (no GPU code).  On 8 x86 cores it took
about two hours (the stored JSON records the time and thread count).  Run from the repository root:

    python tests/golden/make_config2_oracle.py
"""
import json
import math
import os
import platform
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

import oracle as O  # noqa: E402

FIELD = os.path.join(HERE, "config2_d0.25m_field.npy")
META = os.path.join(HERE, "config2_d0.25m.json")


def geometry():
    lam = 632.8e-9
    return O.Geometry(D=0.25, f=1.25, lam=lam, M=512, p=lam * 5 / 8)


def main():
    g = geometry()
    assert g.N == 316057
    threads = O.max_threads()
    t0 = time.time()
    U = O.field_czt(g, 0, g.N, threads)
    dt = time.time() - t0
    np.save(FIELD, U.astype(np.complex64), allow_pickle=False)
    m = O.metrics(g, U)
    meta = {
        "what": "oracle O3 (Bluestein CZT rows then columns, FP64) over the whole aperture",
        "workload": "binary FZP D=0.25 m, f=1.25 m, lambda=632.8 nm, N=316057, ROI 512^2 at lambda f/#/8",
        "geometry": {"D": g.D, "f": g.f, "lambda": g.lam, "dx": g.dx, "N": g.N, "M": g.M, "pitch": g.p,
                     "R": g.R},
        "field_file": os.path.basename(FIELD),
        "field_layout": "U[n, m] at (x_m, y_n), x_m = (m - M/2) p; stored complex64",
        "metrics_fp64": {k: (v.tolist() if isinstance(v, np.ndarray) else float(v)) for k, v in m.items()},
        "intensity_l2": float(np.linalg.norm(np.abs(U) ** 2)),
        "aperture_count": O.count_aperture(g),
        "oracle_seconds": round(dt, 1),
        "oracle_threads": threads,
        "host": platform.machine(),
        "script": "tests/golden/make_config2_oracle.py",
    }
    with open(META, "w") as fh:
        json.dump(meta, fh, indent=1)
        fh.write("\n")
    print(json.dumps({k: meta[k] for k in ("oracle_seconds", "oracle_threads")}),
          "fwhm_x %.9e de_lobe %.9f" % (m["fwhm_x"], m["de_lobe"]), "airy %.9e" %
          (O.airy_fwhm_factor() * g.lam * g.f / (2 * g.R)), "ee/pi2 %.9f" %
          (O.airy_encircled(O.AIRY_NULL) / math.pi ** 2))


if __name__ == "__main__":
    main()
