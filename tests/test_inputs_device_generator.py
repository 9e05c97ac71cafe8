"""The seeded random generator of large shapes (built with torch, run here on
the CPU at a tiny size): its packed layout is the one hss_create reads, the
nested bases are orthonormal, and the assembled matrix is SPD with the
condition number its shift promises."""
import numpy as np
import pytest

from oracle import ulv as O
from paper_2311_00921_gb300 import inputs as I

torch = pytest.importorskip("torch")


def unpack(shape, D, U, E, S):
    n, b, r, L = shape
    D = D.numpy().reshape(2 ** L, b, b).transpose(0, 2, 1)      # column-major blocks
    U = U.numpy().reshape(2 ** L, r, b).transpose(0, 2, 1)
    Es, Ss, e0, s0 = {}, {}, 0, 0
    E, S = E.numpy(), S.numpy()
    for l in range(1, L):
        k = 2 ** l * 2 * r * r
        Es[l] = list(E[e0:e0 + k].reshape(2 ** l, r, 2 * r).transpose(0, 2, 1))
        e0 += k
    for l in range(1, L + 1):
        k = 2 ** (l - 1) * r * r
        Ss[l] = list(S[s0:s0 + k].reshape(2 ** (l - 1), r, r).transpose(0, 2, 1))
        s0 += k
    assert e0 == (E.size if L >= 2 else 0) and s0 == S.size
    ranks = {l: np.full(2 ** l, r, dtype=np.int64) for l in range(1, L + 1)}
    return I.HSSMatrix(levels=L, sizes=np.full(2 ** L, b, dtype=np.int64), ranks=ranks,
                       D=list(D), U=list(U), E=Es, S=Ss)


@pytest.mark.parametrize("levels,leaf,rank", [(3, 16, 4), (2, 24, 8)])
def test_random_device_generator_layout_and_spd(levels, leaf, rank):
    shape, D, U, E, S, shift = I.random_hss_device(levels, leaf, rank, seed=7, device="cpu")
    assert shape == (leaf << levels, leaf, rank, levels)
    h = unpack(shape, D, U, E, S)
    for u in h.U:                                  # orthonormal leaf bases
        np.testing.assert_allclose(u.T @ u, np.eye(rank), atol=1e-12)
    for l in h.E:                                  # orthonormal transfers
        for e in h.E[l]:
            np.testing.assert_allclose(e.T @ e, np.eye(rank), atol=1e-12)
    A = O.assemble_dense(h)
    np.testing.assert_allclose(A, A.T, atol=1e-12)
    w = np.linalg.eigvalsh(A)
    assert w[0] > 0 and w[-1] / w[0] < 4.0, (w[0], w[-1])
    # same seed, same matrix
    _, D2, _, _, S2, _ = I.random_hss_device(levels, leaf, rank, seed=7, device="cpu")
    assert torch.equal(D, D2) and torch.equal(S, S2)
