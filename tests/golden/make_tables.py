"""Write the tabulated HB ingredients used as shared input by every path.

Calls only ``oracle/`` (plus the seeded input module for the media).  Each
file ``tables/<medium>_nI<n>.npz`` holds float64 arrays ``nodes`` (n_I,) and
``tau2``, ``v0``, ``v1`` (N_I, N_I), row = observation Chebyshev node,
column = source Chebyshev node, node index i = i2*n_I + i1 (Sec. 4.1,
Eq. chebinterp; media of Sec. 5.1.1).

    python tests/golden/make_tables.py
"""
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import numpy as np  # noqa: E402

from oracle import tables  # noqa: E402
from paper_2210_02698_gb300 import workloads as W  # noqa: E402

MEDIA = [(W.HOMOGENEOUS, 16), (W.GRADIENT, 16)]


def path_for(medium, n_I):
    return os.path.join(HERE, "tables", f"{medium.key}_nI{n_I}.npz")


def main():
    os.makedirs(os.path.join(HERE, "tables"), exist_ok=True)
    for medium, n_I in MEDIA:
        t = tables.build_tables(medium, n_I)
        np.savez(path_for(medium, n_I), nodes=t["nodes"], tau2=t["tau2"], v0=t["v0"], v1=t["v1"])
        print("wrote", path_for(medium, n_I))


if __name__ == "__main__":
    main()
