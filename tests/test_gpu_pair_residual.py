"""GPU: the pair-of-FP32 matvec (hss_matvec_pair) and the refinement that uses
it for its residual (residual="pair32"), against the FP64 oracle.

The pair arithmetic carries 48 significand bits: a product of inner dimension K
has an error of about sqrt(K) 2^-48 relative to |A| |x|; the tests allow
2e-13 of max(|A| |x|), which a dropped low part (~2^-24) or a lost two-sum
error term (~sqrt(K) 2^-24) would exceed by five orders of magnitude.
"""
import ctypes

import numpy as np
import pytest

from oracle import ulv as O
from paper_2311_00921_gb300 import inputs as I

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_2311_00921_gb300 import hss  # noqa: E402

PAIR_TOL = 2e-13


def abs_bound(h, x):
    """max_i (|A| |x|)_i with A assembled densely from the generators."""
    A = O.assemble_dense(h)
    return (np.abs(A) @ np.abs(x)).max()


CASES = [
    ("random_l3_leaf100_r13", lambda: I.random_hss(3, 100, 13, seed=21, orthonormal=False)),
    ("random_l2_leaf256_r32", lambda: I.random_hss(2, 256, 32, seed=22)),
    ("cube_inv_2k", lambda: I.build_hss(I.scaled(I.WORKLOADS["cube_inv_4k"], 2048, leaf=256,
                                                   rank=32))),
    ("grid_exp_4k", lambda: I.build_hss(I.scaled(I.WORKLOADS["grid_exp_64k"], 4096, leaf=256,
                                                   rank=64))),
]


@pytest.mark.parametrize("name,make", CASES, ids=[c[0] for c in CASES])
@pytest.mark.parametrize("nrhs", [1, 16, 21])
def test_pair_matvec_accuracy(name, make, nrhs):
    h = make()
    x = I.rhs(h.n, nrhs, 5)
    dev = hss.HSS(h)
    y = dev.matvec_pair(hss.colmajor(x)).cpu().numpy().reshape(x.shape)
    y_ref = O.matvec(h, x).reshape(x.shape)
    err = np.abs(y - y_ref).max() / abs_bound(h, x)
    assert err <= PAIR_TOL, f"{name}: {err:.3e}"
    # the FP64 device matvec agrees with both to the same bound
    y64 = dev.matvec(hss.colmajor(x)).cpu().numpy().reshape(x.shape)
    assert np.abs(y - y64).max() / abs_bound(h, x) <= PAIR_TOL


def test_pair_matvec_column_scaling():
    """Columns enter scaled by a power of two near 1/|x_j|: a power-of-two
    multiple of a column gives exactly that multiple of the result, columns far
    outside the FP32 range keep their relative accuracy, a zero column stays 0."""
    h = I.random_hss(3, 64, 16, seed=23)
    dev = hss.HSS(h)
    x = I.rhs(h.n, 4, 6)
    y = dev.matvec_pair(hss.colmajor(x)).cpu().numpy()
    xs = x * np.array([2.0 ** 100, 2.0 ** -90, 1.0, 0.0])
    ys = dev.matvec_pair(hss.colmajor(xs)).cpu().numpy()
    assert np.array_equal(ys[:, 0], y[:, 0] * 2.0 ** 100)
    assert np.array_equal(ys[:, 1], y[:, 1] * 2.0 ** -90)
    assert np.array_equal(ys[:, 2], y[:, 2])
    assert not ys[:, 3].any()
    xw = x[:, :2] * np.array([1e-41, 1e45])        # below / above the FP32 range
    yw = dev.matvec_pair(hss.colmajor(xw)).cpu().numpy()
    yr = O.matvec(h, xw)
    for j in range(2):
        err = np.abs(yw[:, j] - yr[:, j]).max() / abs_bound(h, xw[:, j])
        assert err <= PAIR_TOL, (j, err)


@pytest.mark.parametrize("name,make", CASES[1:], ids=[c[0] for c in CASES[1:]])
def test_mixed_refinement_pair_residual(name, make):
    """FP32 factor, residual in pair arithmetic: the true (FP64 oracle) residual
    reaches 1e-12 per column and x matches the FP64 oracle solution to 1e-10."""
    h = make()
    dev = hss.HSS(h)
    dev.factorize("fp32", ir_tol=1e-12, ir_max_it=30, residual="pair32")
    b = I.rhs(h.n, 5, 8)
    x = dev.solve(hss.colmajor(b)).cpu().numpy()
    info = dev.last_info()
    assert info["code"] == 0 and info["ir_resid"] <= 1e-12 and info["ir_iters"] <= 10, info
    res = b - O.matvec(h, x)
    assert (np.linalg.norm(res, axis=0) / np.linalg.norm(b, axis=0)).max() <= 1e-12
    x_ref = O.solve(O.factor(h), b)
    err = np.linalg.norm(x - x_ref, axis=0) / np.linalg.norm(x_ref, axis=0)
    assert err.max() <= 1e-10, err


def test_pair_residual_in_place_many_columns():
    h = I.random_hss(3, 64, 16, seed=24, orthonormal=False)
    dev = hss.HSS(h)
    dev.factorize("fp32", residual="pair32")
    b = I.rhs(h.n, 19, 9)                  # two refinement passes of 16 + 3 columns
    xb = hss.colmajor(b)
    dev.solve(xb, xb)
    x = xb.cpu().numpy()
    res = b - O.matvec(h, x)
    assert (np.linalg.norm(res, axis=0) / np.linalg.norm(b, axis=0)).max() <= 1e-12


def test_invalid_residual_option():
    h = I.random_hss(2, 32, 8, seed=25)
    dev = hss.HSS(h)
    opt = hss.Options(hss.PRECISIONS["fp32"], 30, 1e-12, 7, 0)
    rc = hss.load().hss_factorize(dev._h, ctypes.byref(opt), None)
    assert rc == -1


def test_wide_levels_mixed_against_fp64():
    """128 leaves of 512 (N = 65,536): launches wide enough for the FP32 128 x 128
    GEMM tile, the 128-row pair-GEMM tiles and the batched-GEMM Q application of
    the solve.  The mixed solution (pair residual) has a true FP64 residual
    <= 1e-12 and agrees with the FP64 factor's solution to 1e-10."""
    h = I.random_hss(7, 512, 64, seed=27, orthonormal=False, fast_bound=True)
    dev = hss.HSS(h)
    b = I.rhs(h.n, 3, 10)
    dev.factorize("fp64")
    x64 = dev.solve(hss.colmajor(b)).cpu().numpy()
    dev.factorize("fp32", residual="pair32")
    x = dev.solve(hss.colmajor(b)).cpu().numpy()
    info = dev.last_info()
    assert info["code"] == 0 and info["ir_resid"] <= 1e-12, info
    res = b - O.matvec(h, x)
    assert (np.linalg.norm(res, axis=0) / np.linalg.norm(b, axis=0)).max() <= 1e-12
    err = np.linalg.norm(x - x64, axis=0) / np.linalg.norm(x64, axis=0)
    assert err.max() <= 1e-10, err
    res64 = b - O.matvec(h, x64)
    assert (np.linalg.norm(res64, axis=0) / np.linalg.norm(b, axis=0)).max() <= 1e-12
