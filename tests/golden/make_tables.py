"""Write the tabulated HB ingredients used as shared input by every path.

Calls only ``oracle/`` (plus the seeded input module for the media).  Each
file ``tables/<medium>_nI<n>.npz`` holds float64 arrays ``nodes`` (n_I,) and
``tau2``, ``v0``, ``v1`` (N_I, N_I), row = observation Chebyshev node,
column = source Chebyshev node, node index i = i2*n_I + i1 (Sec. 4.1,
Eq. chebinterp; media of Sec. 5.1.1).  The homogeneous and gradient media
have exact ingredients (``oracle.tables``); the Gaussian lens is built by
the oracle's Lax-Friedrichs WENO sweeping (``oracle.sweep``, Sec. 2.3) on a
mesh of h0 = 1/256, and its file also holds ``sweep_info`` (per source:
iterations and last largest update of the eikonal, v0 and v1 solves).

    python tests/golden/make_tables.py [homog|grad|lens ...]
"""
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import numpy as np  # noqa: E402

from oracle import sweep, tables  # noqa: E402
from paper_2210_02698_gb300 import workloads as W  # noqa: E402

MEDIA = {"homog": (W.HOMOGENEOUS, 16), "grad": (W.GRADIENT, 16), "lens": (W.LENS, 16)}
LENS_H0 = 1.0 / 256


def path_for(medium, n_I):
    return os.path.join(HERE, "tables", f"{medium.key}_nI{n_I}.npz")


def main(which):
    os.makedirs(os.path.join(HERE, "tables"), exist_ok=True)
    for name in which:
        medium, n_I = MEDIA[name]
        if medium.kind == "lens":
            t = sweep.build_tables(medium, n_I, h0=LENS_H0)
            extra = {"sweep_info": t["info"]}
        else:
            t = tables.build_tables(medium, n_I)
            extra = {}
        np.savez(path_for(medium, n_I), nodes=t["nodes"], tau2=t["tau2"], v0=t["v0"], v1=t["v1"], **extra)
        print("wrote", path_for(medium, n_I))


if __name__ == "__main__":
    main(sys.argv[1:] or list(MEDIA))
