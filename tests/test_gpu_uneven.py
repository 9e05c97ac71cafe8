"""Uneven trees (leaf orders from median bisection of N points, N a multiple of
nothing; ranks min(rank, order)) through the C ABI against the oracle, which
factors the uneven tree as it is.  The library embeds the tree in the uniform
format (identity on the padded diagonal and basis directions, zero padded
couplings), so x and log det must be those of the oracle's uneven factorization.
"""
import numpy as np
import pytest

from oracle import ulv as O
from paper_2311_00921_gb300 import inputs as I

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_2311_00921_gb300 import hss  # noqa: E402


def logdet_scale(F):
    return 2.0 * sum(np.abs(np.log(np.diag(L))).sum() for l in F.LRR for L in F.LRR[l]
                     if L.size) + 2.0 * np.abs(np.log(np.diag(F.L0))).sum()


@pytest.mark.parametrize("name,n,kw", [
    ("cube_inv_4k", 3000, {}),                          # leaf 256: orders 187 / 188
    ("grid_exp_64k", 4992, {"leaf": 128, "rank": 128}),  # 128 x 39 grid; orders 78 < rank
    ("sphere_yukawa_256k", 7777, {"leaf": 512, "rank": 64}),
])
def test_uneven_tree_against_oracle(name, n, kw):
    w = I.scaled(I.WORKLOADS[name], n, **kw)
    h = I.build_hss(w)
    assert not h.uniform and h.n == n
    dev = hss.HSS(h)
    dev.factorize("fp64")
    F = O.factor(h)
    b = I.rhs(n, 3, 5)
    x = dev.solve(hss.colmajor(b)).cpu().numpy()
    x_ref = O.solve(F, b)
    err = np.linalg.norm(x - x_ref, axis=0) / np.linalg.norm(x_ref, axis=0)
    assert err.max() <= 1e-10, err
    assert abs(dev.logdet() - O.logdet(F)) <= 1e-12 * logdet_scale(F)
    # the matvec of the uneven matrix, and the mixed path with FP64 refinement
    xr = I.rhs(n, 2, 9)
    y = dev.matvec(hss.colmajor(xr)).cpu().numpy()
    y_ref = O.matvec(h, xr)
    assert np.abs(y - y_ref).max() <= 1e-13 * np.abs(y_ref).max()
    dev.factorize("fp32")
    xm = dev.solve(hss.colmajor(b)).cpu().numpy()
    res = b - O.matvec(h, xm)
    assert (np.linalg.norm(res, axis=0) / np.linalg.norm(b, axis=0)).max() <= 1e-12
    errm = np.linalg.norm(xm - x_ref, axis=0) / np.linalg.norm(x_ref, axis=0)
    assert errm.max() <= 1e-10, errm


def test_uneven_rejects_bad_sizes():
    h = I.build_hss(I.scaled(I.WORKLOADS["cube_inv_4k"], 1000, leaf=128, rank=16))
    shape, D, U, E, S, keep = hss.uneven_shape(h)
    lib = hss.load()
    out = hss._p()
    shape.n = h.n + 1                     # sizes no longer sum to n
    assert lib.hss_create(shape, D.ctypes.data, U.ctypes.data, E.ctypes.data, S.ctypes.data, 0,
                          out) == -1
    shape.n = h.n
    keep[0] = shape.leaf + 1              # an order above the leaf order
    assert lib.hss_create(shape, D.ctypes.data, U.ctypes.data, E.ctypes.data, S.ctypes.data, 0,
                          out) == -1


def test_batch_of_uneven_trees_against_oracle():
    """A batch mixing uneven trees of both kernel families (N a multiple of
    nothing, leaf orders and ranks from the bisection) with a uniform one: every
    member's x and log det against the oracle."""
    ws = [I.Workload("u0", 3000, 256, 32, "cube", "inv", 0.0, 14.4, 1, 11),
          I.Workload("u1", 4992, 128, 128, "grid2d", "exp", 0.1, 1e-4, 1, 12),
          I.Workload("u2", 2048, 128, 32, "cube", "inv", 0.0, 12.7, 1, 13),
          I.Workload("u3", 1900, 128, 64, "grid2d", "exp", 0.1, 1e-4, 1, 14)]
    mats = [I.build_hss(w) for w in ws]
    assert [m.uniform for m in mats] == [False, False, True, False]
    bt = hss.HSSBatch(mats)
    bt.factorize()
    bs = [hss.colmajor(I.rhs(m.n, 1, k)) for k, m in enumerate(mats)]
    xs = bt.solve(bs)
    lds = bt.logdet()
    for k, m in enumerate(mats):
        F = O.factor(m)
        x_ref = O.solve(F, bs[k].cpu().numpy())
        x = xs[k].cpu().numpy()
        assert np.linalg.norm(x - x_ref) <= 1e-10 * np.linalg.norm(x_ref), k
        assert abs(lds[k] - O.logdet(F)) <= 1e-12 * logdet_scale(F), k
