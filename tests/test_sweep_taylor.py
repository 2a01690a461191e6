"""hb_sweep_taylor (host code of the library, no device): the near-source
Taylor numbers of Sec. 2.2 (d = 2; Eq. recursiveT, recursiveB, C0, C1,
recursiveC) from the series of n^2 about the source.  Pins: the
homogeneous medium's exact expansion (T_2 = n0^2 r^2, every higher piece
zero, B_0 = 1 / (2 sqrt(pi)), C = 0); the constant-gradient medium's
expansion evaluated near the source against its closed-form tau^2 and v0
(oracle.tables); and the oracle's recursions (oracle.taylor) on the
gradient and lens media at several source points, to rounding."""
import math

import numpy as np
import pytest

from oracle import sweep, tables, taylor
from paper_2210_02698_gb300 import binding
from paper_2210_02698_gb300 import workloads as W


def _s2(medium, x0, z0):
    S = sweep.n2_series(medium, x0, z0, 4)
    return np.concatenate([np.asarray(p, dtype=np.float64) for p in S])


def _pieces(row, k0, k1, X, Z, start):
    s, o = 0.0, start
    for k in range(k0, k1 + 1):
        s = s + sum(row[o + m] * X ** (k - m) * Z ** m for m in range(k + 1))
        o += k + 1
    return s


def test_homogeneous_expansion_is_exact():
    n0 = 1.7
    s2 = np.zeros((1, 15))
    s2[0, 0] = n0 * n0
    out = binding.sweep_taylor(s2)[0]
    want = np.zeros(46)
    want[0], want[2] = n0 * n0, n0 * n0          # T_2 = n0^2 (X^2 + Z^2)
    want[25] = 1.0 / (2.0 * math.sqrt(math.pi))  # B_0
    assert np.array_equal(out, want)


def test_gradient_expansion_matches_closed_forms():
    med = W.GRADIENT
    x0, z0 = 0.31, 0.57
    row = binding.sweep_taylor(_s2(med, x0, z0)[None, :])[0]
    fn = tables.ingredient_functions(med)
    for r in (0.02, 0.04):
        for ang in np.linspace(0, 2 * math.pi, 7, endpoint=False):
            X, Z = r * math.cos(ang), r * math.sin(ang)
            et2, ev0, _ = fn(np.array([x0 + X]), np.array([z0 + Z]), x0, z0)
            t2 = _pieces(row, 2, 6, X, Z, 0)
            b = _pieces(row, 0, 4, X, Z, 25)
            # remainders O(r^7) and O(r^5) of the truncated series
            assert abs(t2 - et2[0]) < 50 * r ** 7 * abs(et2[0]) / r ** 2
            assert abs(b - ev0[0]) < 50 * r ** 5


@pytest.mark.parametrize("medium", [W.GRADIENT, W.LENS])
def test_matches_the_oracle_recursions(medium):
    pts = [(0.5, 0.5), (0.02, 0.97), (0.8, 0.13)]
    s2 = np.stack([_s2(medium, x, z) for x, z in pts])
    got = binding.sweep_taylor(s2)
    for k, (x, z) in enumerate(pts):
        want = sweep.taylor_input(medium, x, z)
        scale = np.maximum(np.abs(want), 1e-300)
        assert np.max(np.abs(got[k] - want) / np.maximum(scale, 1e-3 * np.abs(want).max())) < 1e-13


def test_arguments():
    with pytest.raises(binding.HBError) as e:
        binding.sweep_taylor(np.zeros((1, 15)))        # S_0 = 0
    assert e.value.status == binding.HB_ERR_ARG
    assert binding.sweep_taylor(np.zeros((0, 15))).shape == (0, 46)
