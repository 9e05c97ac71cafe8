"""Tensor-core (tcgen05) contractions of the mixed-precision factorization.

The TF32 / BF16 modes run W = A V and the rank-2r update of the diagonal product
on the tensor cores with hi + lo operand splitting and FP32 accumulation; every
other step is the FP32 path.  Checked against the FP32 SIMT factor (same
algorithm, so the blocks agree to the splitting's accuracy: about 2^-21 of the
block scale for TF32 x3 and 2^-16 for BF16 x3, times a modest growth factor),
and end to end: FP64 refinement reaches a 1e-12 residual and the FP64 oracle's
solution within 1e-10.  Shapes cover several 128 x 128 tiles, the lower-tile
enumeration of the update, and ragged M, N and K (zero padding).
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


def rel(a, b):
    return np.abs(a - b).max() / max(np.abs(b).max(), 1e-300)


@pytest.mark.parametrize("levels,leaf,rank", [(2, 256, 128), (3, 100, 13), (2, 384, 64)])
@pytest.mark.parametrize("mode,tol", [("tf32", 2e-5), ("bf16", 2e-3)])
def test_tensor_core_factor_matches_fp32_factor(levels, leaf, rank, mode, tol):
    h = I.random_hss(levels, leaf, rank, seed=leaf + rank, orthonormal=False)
    a, b = hss.HSS(h), hss.HSS(h)
    a.factorize("fp32")
    b.factorize(mode)
    b.sync()
    for l in range(levels, 0, -1):
        Ma, Mb = a.export("M", l), b.export("M", l)
        for i in range(2 ** l):
            err = rel(np.tril(Mb[i]), np.tril(Ma[i]))
            assert err <= tol, f"{mode} level {l} node {i}: {err:.2e}"


@pytest.mark.parametrize("mode", ["tf32", "bf16"])
@pytest.mark.parametrize("name,n,kw", [
    ("sphere_yukawa_256k", 8192, {}),
    ("cube_inv_4k", 4096, {}),
])
def test_tensor_core_refinement(mode, name, n, kw):
    w = I.scaled(I.WORKLOADS[name], n, **kw)
    h = I.build_hss(w)
    dev = hss.HSS(h)
    dev.factorize(mode, ir_tol=1e-12, ir_max_it=60)
    b = I.rhs(w.n, 4, w.seed + 5)
    x = dev.solve(hss.colmajor(b)).cpu().numpy()
    info = dev.last_info()
    assert info["code"] == 0 and info["ir_resid"] <= 1e-12, info
    res = b - O.matvec(h, x)
    assert (np.linalg.norm(res, axis=0) / np.linalg.norm(b, axis=0)).max() <= 1e-12
    x_ref = O.solve(O.factor(h), b)
    err = np.linalg.norm(x - x_ref, axis=0) / np.linalg.norm(x_ref, axis=0)
    assert err.max() <= 1e-10, err
