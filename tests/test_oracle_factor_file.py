"""Pins of the oracle's factor-file butterfly apply (oracle/factor_file.py)
against brute force: a small synthetic operator written in the documented
hb_save format is applied by the oracle and, independently, assembled as
explicit dense matrices (block-diagonal V^0 and K^L, block-sparse W^k, dense
leaves; Sec. 4.2.1 Eq. butterfly_mat, Sec. 4.2 HODBF) and multiplied out."""
import numpy as np
import pytest

from oracle.factor_file import FactorFile


def _write(path, rng, nx=4, ny=4, leaf_pts=4, Lv=2, n_I=2):
    """A random operator in the hb_save format; returns what a brute-force
    assembly needs."""
    Nv = nx * ny
    NI = n_I * n_I
    perm = rng.permutation(Nv)
    bounds = [np.arange(0, Nv + 1, Nv >> l) for l in range(Lv + 1)]
    arena = []
    n = [0]

    def put(rows, cols):
        a = rng.standard_normal((rows, cols)) + 1j * rng.standard_normal((rows, cols))
        off = n[0]
        arena.append(a.T.reshape(-1))      # column-major
        n[0] += rows * cols
        return off, a

    leaves = [put(leaf_pts, leaf_pts) for _ in range(1 << Lv)]
    bfs = []
    for l in range(1, Lv + 1):
        for p in range(1 << (l - 1)):
            for d in range(2):
                oi, si, L = 2 * p + d, 2 * p + 1 - d, Lv - l
                rank = [rng.integers(1, 4, size=1 << L) for _ in range(L + 1)]
                blocks = [[None] * (1 << L) for _ in range(L + 1)]
                for j in range(1 << L):
                    blocks[0][j] = put(int(rank[0][j]), leaf_pts)
                for k in range(1, L + 1):
                    w = 1 << (L - k)
                    for i in range(1 << k):
                        for j in range(w):
                            q1 = (i // 2) * (2 * w) + 2 * j
                            blocks[k][i * w + j] = put(int(rank[k][i * w + j]),
                                                       int(rank[k - 1][q1] + rank[k - 1][q1 + 1]))
                kl = [put(leaf_pts, int(rank[L][i])) for i in range(1 << L)]
                bfs.append((l, oi, si, L, rank, blocks, kl))
    h = 1.0 / nx
    with open(path, "wb") as f:
        wi = lambda *v: f.write(np.asarray(v, dtype="<i8").tobytes())          # noqa: E731
        wd = lambda *v: f.write(np.asarray(v, dtype="<f8").tobytes())          # noqa: E731
        f.write(b"HBFACT01")
        wi(nx, ny)
        wd(0.0, 0.0, h, 10.0)
        wd(1e-6, 20.0, 10.0)
        wi(leaf_pts, 0, 0, 0)
        wi(n_I)
        f.write(np.linspace(0, 1, n_I).astype("<f8").tobytes() * 2)
        f.write(np.zeros(3 * NI * NI, dtype="<f8").tobytes())
        f.write(np.ones(Nv, dtype="<f8").tobytes())
        wi(Lv)
        f.write(perm.astype("<i8").tobytes())
        for b in bounds:
            f.write(b.astype("<i8").tobytes())
        wi(n[0])
        f.write(np.concatenate(arena).astype("<c16").tobytes())
        f.write(np.asarray([off for off, _ in leaves], dtype="<i8").tobytes())
        wi(len(bfs))
        for (l, oi, si, L, rank, blocks, kl) in bfs:
            wi(l, oi, si, L)
            for k in range(L + 1):
                for q in range(1 << L):
                    wi(int(rank[k][q]), blocks[k][q][0])
            f.write(np.asarray([off for off, _ in kl], dtype="<i8").tobytes())
    return dict(Nv=Nv, h=h, perm=perm, bounds=bounds, leaves=leaves, bfs=bfs, Lv=Lv, leaf_pts=leaf_pts)


def _dense(op):
    """K~ in tree order, assembled from explicit matrices."""
    Nv, Lv, lp = op["Nv"], op["Lv"], op["leaf_pts"]
    K = np.zeros((Nv, Nv), complex)
    for t, (_, D) in enumerate(op["leaves"]):
        K[t * lp:(t + 1) * lp, t * lp:(t + 1) * lp] += D
    for (l, oi, si, L, rank, blocks, kl) in op["bfs"]:
        def blockdiag(mats):
            r = sum(m.shape[0] for m in mats)
            c = sum(m.shape[1] for m in mats)
            out = np.zeros((r, c), complex)
            i = j = 0
            for m in mats:
                out[i:i + m.shape[0], j:j + m.shape[1]] = m
                i += m.shape[0]
                j += m.shape[1]
            return out
        M = blockdiag([blocks[0][j][1] for j in range(1 << L)])            # V^0
        for k in range(1, L + 1):
            w = 1 << (L - k)
            prev = np.concatenate([[0], np.cumsum(rank[k - 1])])
            cur = np.concatenate([[0], np.cumsum(rank[k])])
            Wk = np.zeros((cur[-1], prev[-1]), complex)
            for i in range(1 << k):
                for j in range(w):
                    q, q1 = i * w + j, (i // 2) * (2 * w) + 2 * j
                    Wk[cur[q]:cur[q + 1], prev[q1]:prev[q1 + 2]] = blocks[k][q][1]
            M = Wk @ M
        M = blockdiag([kl[i][1] for i in range(1 << L)]) @ M                  # K^L
        r0, r1 = op["bounds"][l][oi], op["bounds"][l][oi + 1]
        c0, c1 = op["bounds"][l][si], op["bounds"][l][si + 1]
        K[r0:r1, c0:c1] += M
    return K


@pytest.mark.parametrize("seed,Lv", [(0, 2), (1, 3)])
def test_factor_file_apply_matches_brute_force(tmp_path, seed, Lv):
    rng = np.random.default_rng(seed)
    nx = 4 if Lv == 2 else 8
    op = _write(tmp_path / "op.hbf", rng, nx=nx, ny=4, leaf_pts=nx * 4 >> Lv, Lv=Lv)
    F = FactorFile(tmp_path / "op.hbf")
    K = _dense(op)
    s = rng.standard_normal((op["Nv"], 3)) + 1j * rng.standard_normal((op["Nv"], 3))
    want = np.empty_like(s)
    want[op["perm"]] = K @ (op["h"] ** 2 * s[op["perm"]])
    got = F.apply(s)
    assert np.linalg.norm(got - want) <= 1e-13 * np.linalg.norm(want)
    # the adjoint is the exact adjoint: s = h^2 K~^H u
    u = rng.standard_normal((op["Nv"], 2)) + 1j * rng.standard_normal((op["Nv"], 2))
    wantA = np.empty_like(u)
    wantA[op["perm"]] = op["h"] ** 2 * (K.conj().T @ u[op["perm"]])
    gotA = F.apply_adjoint(u)
    assert np.linalg.norm(gotA - wantA) <= 1e-13 * np.linalg.norm(wantA)
    lhs = np.vdot(F.apply(s[:, :1]), u[:, :1])
    rhs = np.vdot(s[:, :1], F.apply_adjoint(u[:, :1]))
    assert abs(lhs - rhs) <= 1e-13 * abs(lhs)


def test_factor_file_rejects_garbage(tmp_path):
    p = tmp_path / "bad.hbf"
    p.write_bytes(b"NOTHBF01" + bytes(64))
    with pytest.raises(ValueError):
        FactorFile(p)
