"""GPU batched interpolative decomposition (Eq. ID) against the oracle CPQR
on seeded matrices: skeleton indices bit-exact, V within 1e-10."""
import numpy as np
import pytest

from paper_2210_02698_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2210_02698_gb300 import build
    build.build()


def _run(mats, eps):
    import torch
    from paper_2210_02698_gb300 import binding
    m = np.array([a.shape[0] for a in mats], dtype=np.int32)
    n = np.array([a.shape[1] for a in mats], dtype=np.int32)
    off = np.concatenate([[0], np.cumsum(m.astype(np.int64) * n)[:-1]]).astype(np.int64)
    flat = np.concatenate([a.T.reshape(-1) for a in mats])         # column-major each
    A = torch.from_numpy(flat).to("cuda")
    rank = torch.zeros(len(mats), dtype=torch.int32, device="cuda")
    skel = torch.zeros(int(n.sum()), dtype=torch.int32, device="cuda")
    V = torch.zeros(int((n.astype(np.int64) ** 2).sum()), dtype=torch.complex128, device="cuda")
    binding.id_batch(A, m, n, off, eps, rank, skel, V)
    rank, skel, V = rank.cpu().numpy(), skel.cpu().numpy(), V.cpu().numpy()
    out, so, vo = [], 0, 0
    for b in range(len(mats)):
        r = int(rank[b])
        Vb = V[vo:vo + n[b] * n[b]].reshape(n[b], n[b]).T[:r]      # column-major, ld = n
        out.append((skel[so:so + r].copy(), Vb))
        so += n[b]
        vo += n[b] * n[b]
    return out


@pytest.mark.parametrize("m,n,rank,decay,eps", [(120, 40, 30, 0.6, 1e-6), (300, 64, 64, 0.8, 1e-8),
                                                (33, 90, 20, 0.5, 1e-6), (1500, 64, 50, 0.7, 1e-6)])
def test_id_matches_oracle(m, n, rank, decay, eps):
    from oracle import cpqr
    A = W.random_id_matrices(6, m, n, rank, decay, seed=m + n)
    mats = [A[b].T.copy() for b in range(6)]
    got = _run(mats, eps)
    for M, (sk, V) in zip(mats, got):
        sk0, V0, rd = cpqr.cpqr_id(M, eps)
        assert list(sk) == list(sk0)
        # V = R11^-1 R12: rounding differences grow with the conditioning of
        # R11, estimated by |R_00| / |R_(r-1)(r-1)| of the oracle's pivots
        cond = rd[0] / rd[len(sk0) - 1]
        assert np.max(np.abs(V - V0)) < 1e-14 * cond * max(1.0, np.max(np.abs(V0))) * len(sk0)


def test_id_degenerate_cases():
    from oracle import cpqr
    rng = np.random.default_rng(3)
    a = rng.standard_normal(10) + 1j * rng.standard_normal(10)
    mats = [np.stack([a, a, 0.5 * a], axis=1), np.zeros((5, 4), dtype=complex),
            (rng.standard_normal((1, 6)) + 0j), (rng.standard_normal((7, 1)) + 0j)]
    got = _run(mats, 1e-12)
    for M, (sk, V) in zip(mats, got):
        sk0, V0, _ = cpqr.cpqr_id(M, 1e-12)
        assert list(sk) == list(sk0)
        assert np.allclose(V, V0, atol=1e-12)


def test_id_tie_window_matches_oracle():
    """The constructed near-ties of the oracle's tie-window pin: the GPU
    picks the same pivots (lowest position within TIE |R_00| of the largest
    norm)."""
    from oracle import cpqr
    T = cpqr.TIE
    rng = np.random.default_rng(17)
    a = rng.standard_normal(6) + 1j * rng.standard_normal(6)
    a /= np.linalg.norm(a)
    e0 = np.zeros(5, dtype=complex)
    e0[0] = 10.0
    x = np.zeros(5, dtype=complex)
    x[1:] = rng.standard_normal(4) + 1j * rng.standard_normal(4)
    x /= np.linalg.norm(x)
    y = np.zeros(5, dtype=complex)
    y[1:] = np.roll(x[1:], 1) * np.exp(0.3j)
    mats = [np.stack([a * (1 - 0.5 * T), a, 0.1 * a[::-1]], axis=1),
            np.stack([a * (1 - 3 * T), a, 0.1 * a[::-1]], axis=1),
            np.stack([e0, y * (1 - 0.5 * T * 10.0), x], axis=1),
            np.stack([e0, y * (1 - 2.0 * T * 10.0), x], axis=1)]
    got = _run(mats, 1e-14)
    for M, (sk, V) in zip(mats, got):
        sk0, _, _ = cpqr.cpqr_id(M, 1e-14)
        assert list(sk) == list(sk0)
