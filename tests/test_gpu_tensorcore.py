"""Tensor-core (tcgen05) contractions of the mixed-precision factorization.

The TF32 / BF16 modes run W = A V and the rank-2r update of the diagonal product
on the tensor cores with hi + lo operand splitting and FP32 accumulation; every
other step is the FP32 path.  Checked against the FP32 SIMT factor (same
algorithm, so the blocks agree to the splitting's accuracy: about 2^-21 of the
block scale for TF32 x3 and 2^-16 for BF16 x3, times a modest growth factor),
and end to end: FP64 refinement reaches a 1e-12 residual and the FP64 oracle's
solution within 1e-10.  Shapes cover several 128 x 128 tiles, the lower-tile
enumeration of the update, and ragged M, N and K (zero padding).  The per-step
arrays are also compared with the oracle run in float32.  The bounded waits of
the tensor-core pipeline are exercised with a wait budget that gives up at once:
the call reports HSS_ERR_TIMEOUT and the next call works normally.
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


def q_from_vt(V, T):
    return np.eye(V.shape[0]) - V @ T @ V.T


@pytest.mark.parametrize("levels,leaf,rank", [(2, 256, 128), (3, 100, 13), (3, 512, 128)])
@pytest.mark.parametrize("mode,tol", [("tf32", 1e-3), ("bf16", 3e-3)])
def test_tensor_core_factor_per_step_against_float32_oracle(levels, leaf, rank, mode, tol):
    """Every level's basis completion, factored block (L^RR and Â^SS) against
    the oracle's float32 factor: the x3 contractions keep FP32-level accuracy,
    so the bound is the one of the FP32 SIMT factor's per-step test (a few
    hundred FP32 ulps of the block's scale) with room for the BF16 split."""
    h = I.random_hss(levels, leaf, rank, seed=3 * leaf + rank, orthonormal=False)
    dev = hss.HSS(h)
    dev.factorize(mode)
    dev.sync()
    F = O.factor(h, dtype=np.float32)
    for l in range(levels, 0, -1):
        V, T, LB, M = (dev.export(k, l) for k in ("V", "T", "LB", "M"))
        for i in range(2 ** l):
            b, r = V.shape[1], V.shape[2]
            c = b - r
            assert rel(q_from_vt(V[i], T[i]), F.Q[l][i].astype(np.float64)) <= 2e-4
            assert rel(LB[i], F.LB[l][i].astype(np.float64)) <= 2e-4
            if c:
                err = rel(np.tril(M[i][:c, :c]), F.LRR[l][i].astype(np.float64))
                assert err <= tol, f"{mode} L^RR level {l} node {i}: {err:.2e}"
            err = rel(np.tril(M[i][c:, c:]), np.tril(F.SS[l][i]).astype(np.float64))
            assert err <= tol, f"{mode} SS level {l} node {i}: {err:.2e}"


@pytest.mark.parametrize("mode", ["tf32", "bf16"])
def test_tensor_core_wait_budget_runs_out(mode):
    """A negative wait budget makes every pipeline wait of the tcgen05 kernel give
    up at once (K = 256 spans 8 slabs, so every tile waits): the kernel records
    HSS_ERR_TIMEOUT, drains the MMAs it issued, frees its tensor memory and
    returns; the error surfaces at the next synchronizing call, and a normal
    factorization of the same object afterwards is correct."""
    h = I.random_hss(2, 256, 64, seed=77, orthonormal=False)
    dev = hss.HSS(h)
    dev.factorize(mode, wait_budget=-1)
    info = dev.last_info()
    assert info["code"] == -6, info
    dev.factorize(mode)
    b = I.rhs(h.n, 2, 5)
    x = dev.solve(hss.colmajor(b)).cpu().numpy()
    assert dev.last_info()["code"] == 0
    x_ref = O.solve(O.factor(h), b)
    err = np.linalg.norm(x - x_ref, axis=0) / np.linalg.norm(x_ref, axis=0)
    assert err.max() <= 1e-10, err
