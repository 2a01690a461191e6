"""Near-source Taylor recursions for tau^2, v0, v1 (Sec. 2.2), d = 2.

Test infrastructure (see ``oracle/__init__``).  These recursions are how the
paper initialises its sweeping solvers; the oracle uses them as an
independent pin of ``tables`` near the source.

A homogeneous polynomial of degree k in the offset (x, z) = r - r0 is stored
as the coefficient vector c[0..k] of x^(k-j) z^j.

Eq. expansionT / Eq. recursiveT:
  T0 = T1 = 0,  T2 = S0 |r|^2,
  (P-1) S0 T_P = sum_{k=1}^{P-2} S_k T_{P-k}
                 - 1/4 sum_{k=2}^{P-2} grad T_{k+1} . grad T_{P-k+1},   P >= 3.
Eq. expansionV0 / Eq. recursiveB:
  B0 = n0^(d-2) / (2 pi^((d-1)/2)),
  2 P S0 B_P = - sum_{k=1}^{P-1} grad B_k . grad T_{P+2-k}
               - 1/2 sum_{k=0}^{P-1} B_k Lap T_{P+2-k}
               + d sum_{k=0}^{P-1} B_k S_{P-k},                      P >= 1
  (P = 1 is the paper's separate B1 formula).
Eq. C0, Eq. C1, Eq. recursiveC:
  2 S0 C0 = 1/2 Lap B2,
  4 S0 C1 = 1/2 Lap B3 - 1/2 Lap T3 C0 - (2-d) S1 C0,
  2 (P+1) S0 C_P = 1/2 Lap B_{P+2} - sum_{k=1}^{P-1} grad C_k . grad T_{P+2-k}
                   - 1/2 sum_{k=0}^{P-1} C_k Lap T_{P+2-k}
                   - (2-d) sum_{k=0}^{P-1} C_k S_{P-k},              P >= 2.
Orders: P_B = P_S = P_T - 2 = P_C + 2 with P_T = 6 (Sec. 2.2-2.3).
"""
import math

import numpy as np

D = 2


def _zero(k):
    return np.zeros(k + 1)


def mul(p, q):
    return np.convolve(p, q)


def grad(p):
    k = len(p) - 1
    if k == 0:
        return np.zeros(0), np.zeros(0)
    j = np.arange(k + 1)
    px = ((k - j) * p)[:k]
    pz = (j * p)[1:]
    return px, pz


def lap(p):
    k = len(p) - 1
    if k < 2:
        return np.zeros(max(k - 1, 1))
    px, pz = grad(p)
    pxx, _ = grad(px)
    _, pzz = grad(pz)
    return pxx + pzz


def dot_grad(p, q):
    px, pz = grad(p)
    qx, qz = grad(q)
    if len(px) == 0 or len(qx) == 0:
        return _zero(max(len(p) + len(q) - 4, 0))
    return mul(px, qx) + mul(pz, qz)


def evaluate(p, x, z):
    k = len(p) - 1
    x = np.asarray(x, dtype=np.float64)
    z = np.asarray(z, dtype=np.float64)
    out = np.zeros(np.broadcast(x, z).shape)
    for j, c in enumerate(p):
        out = out + c * x ** (k - j) * z**j
    return out


def n2_series_gradient(c_src, g, P):
    """S_k of n^2 = (c_src + g z)^-2 about the source: (k+1)(-g/c)^k z^k / c^2."""
    S = []
    for k in range(P + 1):
        p = _zero(k)
        p[k] = (k + 1) * (-g / c_src) ** k / c_src**2
        S.append(p)
    return S


def recursions(S, P_T=6):
    """Return (T, B, C) lists of homogeneous polynomials for the given S_k."""
    P_B = P_T - 2
    P_C = P_T - 4
    S0 = S[0][0]

    def Sk(k):
        return S[k] if k < len(S) else _zero(k)

    T = [_zero(0), _zero(1)]
    T2 = _zero(2)
    T2[0] = S0
    T2[2] = S0
    T.append(T2)
    for P in range(3, P_T + 1):
        acc = _zero(P)
        for k in range(1, P - 1):
            acc = acc + mul(Sk(k), T[P - k])
        for k in range(2, P - 1):
            acc = acc - 0.25 * dot_grad(T[k + 1], T[P - k + 1])
        T.append(acc / ((P - 1) * S0))

    def Tk(k):
        return T[k] if k < len(T) else _zero(k)

    B = [np.array([1.0 / (2.0 * math.pi ** ((D - 1) / 2.0))])]
    for P in range(1, P_B + 1):
        acc = _zero(P)
        for k in range(1, P):
            acc = acc - dot_grad(B[k], Tk(P + 2 - k))
        for k in range(0, P):
            acc = acc - 0.5 * mul(B[k], lap(Tk(P + 2 - k)))
            acc = acc + D * mul(B[k], Sk(P - k))
        B.append(acc / (2 * P * S0))

    def Bk(k):
        return B[k] if k < len(B) else _zero(k)

    C = [0.5 * lap(Bk(2)) / (2 * S0)]
    c1 = 0.5 * lap(Bk(3)) - 0.5 * mul(lap(Tk(3)), C[0]) - (2 - D) * mul(Sk(1), C[0])
    C.append(c1 / (4 * S0))
    for P in range(2, P_C + 1):
        acc = 0.5 * lap(Bk(P + 2))
        for k in range(1, P):
            acc = acc - dot_grad(C[k], Tk(P + 2 - k))
        for k in range(0, P):
            acc = acc - 0.5 * mul(C[k], lap(Tk(P + 2 - k)))
            acc = acc - (2 - D) * mul(C[k], Sk(P - k))
        C.append(acc / (2 * (P + 1) * S0))
    return T, B, C


def series_value(polys, x, z):
    return sum(evaluate(p, x, z) for p in polys)
