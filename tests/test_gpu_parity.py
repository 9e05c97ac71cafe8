"""GPU parity: the CUDA path (through the C ABI) against the CPU oracle.

Per-step parity compares what the oracle computes node by node (basis
completion Q and L_B, the factored block L^RR / L^SR / Â^SS, the merged basis of
the next level) with the exported device arrays, on seeded inputs that span
several 64-wide GEMM tiles and 32-wide Cholesky panels with ragged tails.
End-to-end parity compares x (relative 1e-10 per column) and log det (relative
1e-12 on the scale Σ|2 log l_jj|) with the oracle, plus the HSS matvec.
Tolerances of the per-step arrays: both sides are FP64 Householder / Cholesky
of the same matrices with the same sign convention, so they agree to a small
multiple of b·ε relative to the block's norm.
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

EPS = np.finfo(np.float64).eps


def q_from_vt(V, T):
    return np.eye(V.shape[0]) - V @ T @ V.T


def check_close(a, b, tol, what):
    scale = max(np.abs(b).max(), 1e-300)
    err = np.abs(a - b).max() / scale
    assert err <= tol, f"{what}: max rel err {err:.3e} > {tol:.1e}"


def run_both(h, nrhs, seed=7):
    dev = hss.HSS(h)
    dev.factorize("fp64")
    F = O.factor(h)
    b = I.rhs(h.n, nrhs, seed)
    x = dev.solve(hss.colmajor(b)).cpu().numpy()
    return dev, F, b, x


def check_end_to_end(dev, F, b, x):
    x_ref = O.solve(F, b).reshape(x.shape)
    for j in range(x.shape[1] if x.ndim == 2 else 1):
        xa = x[:, j] if x.ndim == 2 else x
        xr = x_ref[:, j] if x.ndim == 2 else x_ref
        err = np.linalg.norm(xa - xr) / np.linalg.norm(xr)
        assert err <= 1e-10, f"column {j}: x rel err {err:.3e}"
    ld, ld_ref = dev.logdet(), O.logdet(F)
    scale = 2.0 * sum(np.abs(np.log(np.diag(L))).sum() for l in F.LRR for L in F.LRR[l]
                      if L.size) + 2.0 * np.abs(np.log(np.diag(F.L0))).sum()
    assert abs(ld - ld_ref) <= 1e-12 * scale, (ld, ld_ref)


def check_steps(dev, F, h):
    L = h.levels
    for l in range(L, 0, -1):
        V, T, LB, M = (dev.export(k, l) for k in ("V", "T", "LB", "M"))
        for i in range(2 ** l):
            b = V.shape[1]
            r = V.shape[2]
            c = b - r
            tol = 50 * b * EPS
            check_close(q_from_vt(V[i], T[i]), F.Q[l][i], tol, f"Q l={l} i={i}")
            check_close(LB[i], F.LB[l][i], tol * 10, f"L_B l={l} i={i}")
            Mi = M[i]
            if c:
                check_close(np.tril(Mi[:c, :c]), F.LRR[l][i], 1e-11, f"L^RR l={l} i={i}")
                check_close(Mi[c:, :c], F.LSR[l][i], 1e-11, f"L^SR l={l} i={i}")
            ss = np.tril(Mi[c:, c:])
            check_close(ss, np.tril(F.SS[l][i]), 1e-11, f"SS l={l} i={i}")
        if l < L:
            B = dev.export("B", l)
            for i in range(2 ** l):
                check_close(B[i], F.Bnode[l][i], 1e-11, f"merged basis l={l} i={i}")


# ---------------------------------------------------------------- per step
@pytest.mark.parametrize("levels,leaf,rank,ortho", [
    (3, 100, 13, False),     # ragged tiles and panels, non-orthonormal bases
    (2, 64, 32, True),
    (4, 96, 40, False),
])
def test_per_step_random(levels, leaf, rank, ortho):
    h = I.random_hss(levels, leaf, rank, seed=levels * 31 + leaf, orthonormal=ortho)
    dev, F, b, x = run_both(h, 3)
    check_steps(dev, F, h)
    check_end_to_end(dev, F, b, x)


@pytest.mark.parametrize("name,n,kw", [
    ("cube_inv_4k", 4096, {}),                              # the full workload
    ("grid_exp_64k", 4096, {}),                             # scaled (spd construction)
    ("sphere_yukawa_256k", 4096, {}),                       # scaled
    ("sphere_yukawa_256k", 2048, {"leaf": 128, "rank": 48}),
])
def test_per_step_kernel_workloads(name, n, kw):
    w = I.scaled(I.WORKLOADS[name], n, **kw)
    h = I.build_hss(w)
    dev, F, b, x = run_both(h, 4)
    check_steps(dev, F, h)
    check_end_to_end(dev, F, b, x)


# ---------------------------------------------------------------- end to end
@pytest.mark.parametrize("nrhs", [1, 16, 17, 35])
def test_solve_rhs_chunks(nrhs):
    w = I.scaled(I.WORKLOADS["cube_inv_4k"], 2048, leaf=128, rank=32)
    h = I.build_hss(w)
    dev, F, b, x = run_both(h, nrhs)
    check_end_to_end(dev, F, b, x)


def test_solve_in_place_and_vector():
    h = I.random_hss(3, 48, 8, seed=2)
    dev = hss.HSS(h)
    dev.factorize("fp64")
    F = O.factor(h)
    b = I.rhs(h.n, 1, 3)[:, 0]
    xb = hss.colmajor(b)
    dev.solve(xb, xb)                       # x aliases b
    np.testing.assert_allclose(xb.cpu().numpy(), O.solve(F, b), rtol=1e-10, atol=1e-14)


def test_one_level_and_full_rank_leaves():
    # L = 1 (two leaves + root) and rank = leaf (nothing eliminated at the leaves)
    for levels, leaf, rank in [(1, 64, 16), (2, 32, 32)]:
        h = I.random_hss(levels, leaf, rank, seed=11)
        dev, F, b, x = run_both(h, 2)
        check_steps(dev, F, h)
        check_end_to_end(dev, F, b, x)


def test_matches_dense_cholesky_exact_rank():
    # exact-rank kernel: A_hss equals the kernel matrix, the GPU solve must too
    w = I.Workload("poly", 16 * 2 ** 3, 16, 10, "cube", "poly2", 0.0, 3.0, 1, 21)
    h = I.build_hss(w, mode="orth")
    K = I.kernel_matrix(w, h.points)
    dev = hss.HSS(h)
    dev.factorize("fp64")
    b = I.rhs(w.n, 2, 1)
    x = dev.solve(hss.colmajor(b)).cpu().numpy()
    np.testing.assert_allclose(x, np.linalg.solve(K, b), rtol=1e-8, atol=1e-10)
    assert abs(dev.logdet() - np.linalg.slogdet(K)[1]) <= 1e-10 * abs(np.linalg.slogdet(K)[1])


@pytest.mark.parametrize("levels,leaf,rank,nrhs", [
    (4, 80, 24, 1), (4, 80, 24, 5), (4, 80, 24, 33),
    # 256 leaves: the wide-level kernels with 4-, 8- and 16-column blocks
    (8, 72, 16, 3), (8, 72, 16, 8), (8, 72, 16, 13), (8, 72, 16, 16),
])
def test_matvec(levels, leaf, rank, nrhs):
    h = I.random_hss(levels, leaf, rank, seed=5, orthonormal=False)
    dev = hss.HSS(h)
    x = I.rhs(h.n, nrhs, 9)
    y = dev.matvec(hss.colmajor(x)).cpu().numpy()
    y_ref = O.matvec(h, x).reshape(y.shape)
    check_close(y, y_ref, 1e-13, "matvec")


# ---------------------------------------------------------------- errors
def test_not_spd_reports_level_and_node():
    h = I.random_hss(3, 40, 8, seed=4)
    h.D[5] = -h.D[5]
    dev = hss.HSS(h)
    dev.factorize("fp64")          # asynchronous: the error surfaces on sync
    with pytest.raises(hss.HSSError) as ei:
        dev.logdet()
    assert ei.value.code == -3
    info = dev.last_info()
    assert info["code"] == -3 and info["level"] == 3 and info["node"] == 5
    with pytest.raises(O.NotSPD) as eo:
        O.factor(h)
    assert (eo.value.level, eo.value.node, eo.value.col) == (3, 5, info["col"])


def test_six_levels_fp64_and_mixed():
    """64 leaves of 40 (six levels, blocked Cholesky over 1-2 panels per node):
    per-step arrays, x and log det against the oracle in FP64, and the FP32
    factor under pair-residual refinement to a 1e-12 residual."""
    h = I.random_hss(6, 40, 8, seed=31, orthonormal=False)
    dev, F, b, x = run_both(h, 3)
    check_steps(dev, F, h)
    check_end_to_end(dev, F, b, x)
    dev.factorize("fp32", residual="pair32")
    x32 = dev.solve(hss.colmajor(b)).cpu().numpy()
    res = b - O.matvec(h, x32)
    assert (np.linalg.norm(res, axis=0) / np.linalg.norm(b, axis=0)).max() <= 1e-12


def test_not_spd_reports_a_late_leaf():
    h = I.random_hss(6, 40, 8, seed=32)
    h.D[37] = -h.D[37]
    dev = hss.HSS(h)
    dev.factorize("fp64")
    with pytest.raises(hss.HSSError) as ei:
        dev.logdet()
    assert ei.value.code == -3
    info = dev.last_info()
    assert info["level"] == 6 and info["node"] == 37
    with pytest.raises(O.NotSPD) as eo:
        O.factor(h)
    assert (eo.value.level, eo.value.node, eo.value.col) == (6, 37, info["col"])


def test_solve_before_factorize():
    h = I.random_hss(2, 32, 4, seed=1)
    dev = hss.HSS(h)
    with pytest.raises(hss.HSSError) as ei:
        dev.solve(hss.colmajor(np.ones(h.n)))
    assert ei.value.code == -2


# ---------------------------------------------------------------- full size, sampled
@pytest.mark.slow
def test_full_size_sphere_yukawa_sampled():
    """N = 262,144 (leaf 512, rank 128, 9 levels, 16 right-hand sides): sampled
    leaves' factor blocks against the oracle's node step, the backward error
    through the oracle's matvec, and log det against the oracle's factorization."""
    w = I.WORKLOADS["sphere_yukawa_256k"]
    h = I.build_hss(w)
    dev = hss.HSS(h)
    dev.factorize("fp64")
    b = I.rhs(w.n, w.nrhs, w.seed + 1)
    x = dev.solve(hss.colmajor(b)).cpu().numpy()
    L = h.levels
    V, T, M = dev.export("V", L), dev.export("T", L), dev.export("M", L)
    rng = np.random.default_rng(0)
    for i in rng.choice(2 ** L, 6, replace=False):
        Q, LB, Ah, LRR, LSR, SS = O.node_step(h.D[i], h.U[i])
        c = LRR.shape[0]
        check_close(q_from_vt(V[i], T[i]), Q, 50 * 512 * EPS, f"Q leaf {i}")
        check_close(np.tril(M[i][:c, :c]), LRR, 1e-11, f"L^RR leaf {i}")
        check_close(M[i][c:, :c], LSR, 1e-11, f"L^SR leaf {i}")
        check_close(np.tril(M[i][c:, c:]), np.tril(SS), 1e-11, f"SS leaf {i}")
    res = b - O.matvec(h, x)
    rel = np.linalg.norm(res, axis=0) / np.linalg.norm(b, axis=0)
    assert rel.max() <= 1e-13, rel.max()
    F = O.factor(h)
    ld_ref = O.logdet(F)
    assert abs(dev.logdet() - ld_ref) <= 1e-12 * abs(ld_ref)
    x_ref = O.solve(F, b)
    err = np.linalg.norm(x - x_ref, axis=0) / np.linalg.norm(x_ref, axis=0)
    assert err.max() <= 1e-10, err.max()


# ---------------------------------------------------------------- mixed precision + refinement
@pytest.mark.parametrize("name,n,kw", [
    ("cube_inv_4k", 4096, {}),
    ("sphere_yukawa_256k", 8192, {}),
    ("grid_exp_64k", 4096, {}),
    ("sphere_yukawa_256k", 2048, {"leaf": 128, "rank": 48}),
])
def test_mixed_fp32_refinement(name, n, kw):
    """FP32 factor as preconditioner, FP64 residual: reaches 1e-12 relative residual
    per column and the FP64 oracle's solution within 1e-10."""
    w = I.scaled(I.WORKLOADS[name], n, **kw)
    h = I.build_hss(w)
    dev = hss.HSS(h)
    dev.factorize("fp32", ir_tol=1e-12, ir_max_it=30)
    b = I.rhs(w.n, 5, w.seed + 3)
    x = dev.solve(hss.colmajor(b)).cpu().numpy()
    info = dev.last_info()
    assert info["code"] == 0 and info["ir_resid"] <= 1e-12 and info["ir_iters"] <= 10, info
    res = b - O.matvec(h, x)
    assert (np.linalg.norm(res, axis=0) / np.linalg.norm(b, axis=0)).max() <= 1e-12
    F = O.factor(h)
    x_ref = O.solve(F, b)
    err = np.linalg.norm(x - x_ref, axis=0) / np.linalg.norm(x_ref, axis=0)
    assert err.max() <= 1e-10, err
    # log det of the FP32 factor (root FP64): close to the FP64 value at FP32 accuracy
    ld_ref = O.logdet(F)
    assert abs(dev.logdet() - ld_ref) <= 1e-4 * abs(ld_ref)


def test_mixed_fp32_in_place_and_many_columns():
    h = I.random_hss(3, 64, 16, seed=12, orthonormal=False)
    dev = hss.HSS(h)
    dev.factorize("fp32")
    F = O.factor(h)
    b = I.rhs(h.n, 19, 4)        # two refinement passes of 16 + 3 columns
    xb = hss.colmajor(b)
    dev.solve(xb, xb)
    x = xb.cpu().numpy()
    x_ref = O.solve(F, b)
    err = np.linalg.norm(x - x_ref, axis=0) / np.linalg.norm(x_ref, axis=0)
    assert err.max() <= 1e-10


def test_refinement_two_lanes_and_one_lane_agree():
    """The columns of a refinement pass split over two lanes (each lane stops on
    its own columns' residuals, the lanes on two streams, or one after the other
    on the caller's stream under a serialized trace) give the solution of
    one-column solves (one lane) to the tolerance."""
    h = I.random_hss(4, 64, 16, seed=21, orthonormal=False)
    dev = hss.HSS(h)
    dev.factorize("fp32", ir_tol=1e-13, ir_lanes=2)
    b = I.rhs(h.n, 16, 8)
    b[:, 9:] *= 1e6                     # the second lane's columns at another scale
    x2 = dev.solve(hss.colmajor(b)).cpu().numpy()
    it2 = dev.last_info()["ir_iters"]
    dev.trace(True, serialize=True)
    xs = dev.solve(hss.colmajor(b)).cpu().numpy()
    dev.trace(False)
    x1 = np.stack([dev.solve(hss.colmajor(b[:, j])).cpu().numpy().reshape(-1)
                   for j in range(16)], axis=1)
    for x in (x1, x2, xs):
        res = b - O.matvec(h, x)
        assert (np.linalg.norm(res, axis=0) / np.linalg.norm(b, axis=0)).max() <= 1e-13
    assert np.array_equal(x2, xs)
    err = np.linalg.norm(x2 - x1, axis=0) / np.linalg.norm(x1, axis=0)
    assert err.max() <= 1e-11 and it2 >= 1, (err, it2)


def test_mixed_refinement_reports_no_convergence():
    h = I.random_hss(2, 32, 8, seed=3)
    dev = hss.HSS(h)
    dev.factorize("fp32", ir_tol=0.0, ir_max_it=2)   # tolerance 0 cannot be met
    with pytest.raises(hss.HSSError) as ei:
        dev.solve(hss.colmajor(np.ones(h.n)))
    assert ei.value.code == -7
    info = dev.last_info()
    assert info["ir_iters"] == 2 and info["ir_resid"] < 1e-10


@pytest.mark.parametrize("levels,leaf,rank,panel", [
    (3, 100, 13, 0), (2, 256, 32, 0), (3, 128, 48, 0),
    (3, 100, 13, 16), (2, 512, 128, 16), (3, 300, 40, 16),   # 16-column register panels
])
def test_per_step_fp32_factor(levels, leaf, rank, panel):
    """The FP32 factor against the oracle run in float32 (LAPACK sgeqrf / spotrf
    order of operations differs, so the bound is a few hundred FP32 ulps of the
    block's scale), with the basis kernel's default and 16-column panels."""
    h = I.random_hss(levels, leaf, rank, seed=levels * 7 + rank, orthonormal=False)
    dev = hss.HSS(h)
    dev.factorize("fp32", ql_panel=panel)
    F = O.factor(h, dtype=np.float32)
    for l in range(levels, 0, -1):
        V, T, LB, M = (dev.export(k, l) for k in ("V", "T", "LB", "M"))
        for i in range(2 ** l):
            b, r = V.shape[1], V.shape[2]
            c = b - r
            check_close(q_from_vt(V[i], T[i]), F.Q[l][i].astype(np.float64), 2e-4, f"Q32 l={l} i={i}")
            check_close(LB[i], F.LB[l][i].astype(np.float64), 2e-4, f"L_B32 l={l} i={i}")
            if c:
                check_close(np.tril(M[i][:c, :c]), F.LRR[l][i].astype(np.float64), 1e-3,
                            f"L^RR32 l={l} i={i}")
            check_close(np.tril(M[i][c:, c:]), np.tril(F.SS[l][i]).astype(np.float64), 1e-3,
                        f"SS32 l={l} i={i}")


@pytest.mark.slow
def test_per_step_fp32_factor_wide_tiles():
    """The FP32 factor at the benchmark's node shape (leaf 512, rank 128) with 128
    leaves, so that the wide FP32 tile (128 x 128, engaged from 2 x 152 tiles per
    launch) and the 128-row tiles of the leaf products run, per step against the
    oracle's float32 factor: basis completion, L^RR and Â^SS of every node of
    every level.  Same bounds as the small FP32 per-step test."""
    w = I.scaled(I.WORKLOADS["sphere_yukawa_256k"], 65536)
    h = I.build_hss(w)
    assert h.levels == 7 and h.leaf == 512 and h.rank == 128
    dev = hss.HSS(h)
    dev.factorize("fp32")
    dev.sync()
    F = O.factor(h, dtype=np.float32)
    for l in range(h.levels, 0, -1):
        V, T, LB, M = (dev.export(k, l) for k in ("V", "T", "LB", "M"))
        for i in range(2 ** l):
            b, r = V.shape[1], V.shape[2]
            c = b - r
            check_close(q_from_vt(V[i], T[i]), F.Q[l][i].astype(np.float64), 2e-4,
                        f"Q32 l={l} i={i}")
            check_close(LB[i], F.LB[l][i].astype(np.float64), 2e-4, f"L_B32 l={l} i={i}")
            check_close(np.tril(M[i][:c, :c]), F.LRR[l][i].astype(np.float64), 1e-3,
                        f"L^RR32 l={l} i={i}")
            check_close(M[i][c:, :c], F.LSR[l][i].astype(np.float64), 1e-3,
                        f"L^SR32 l={l} i={i}")
            check_close(np.tril(M[i][c:, c:]), np.tril(F.SS[l][i]).astype(np.float64), 1e-3,
                        f"SS32 l={l} i={i}")


def _extreme_eigs(dev, n, its=60, seed=0):
    """λ_max by power iteration on the HSS matvec and λ_min by power iteration
    on the FP64 factor's solve (inverse iteration); both on the GPU."""
    rng = np.random.default_rng(seed)
    v = hss.colmajor(rng.standard_normal((n, 1)))
    lam_max = 0.0
    for _ in range(its):
        v = v / torch.linalg.vector_norm(v)
        av = dev.matvec(v)
        lam_max = float((v * av).sum())
        v = av
    v = hss.colmajor(rng.standard_normal((n, 1)))
    mu = 0.0
    for _ in range(its):
        v = v / torch.linalg.vector_norm(v)
        iv = dev.solve(v)
        mu = float((v * iv).sum())
        v = iv
    return lam_max, 1.0 / mu


@pytest.mark.slow
def test_grid_exp_full_size_against_oracle():
    """The geostatistics workload at its stated size: N = 65,536 jittered grid,
    exp(-d/0.1) + 1e-4 I, leaf 512, rank 128, 7 levels, 8 right-hand sides, FP64.
    x within 1e-10 per column and log det within 1e-12 of Σ|2 log l_jj| against
    the oracle; the backward residual within 10x that of the oracle's own
    solution (both at the round-off that κ ≈ 2.6e5 allows), and the condition
    number estimated on the GPU (printed; the 1e-10 target assumes κ ε well
    below it)."""
    w = I.WORKLOADS["grid_exp_64k"]
    h = I.build_hss(w)
    assert (h.n, h.levels, h.leaf, h.rank) == (65536, 7, 512, 128)
    dev, F, b, x = run_both(h, w.nrhs, seed=w.seed + 1)
    lam_max, lam_min = _extreme_eigs(dev, h.n)
    kappa = lam_max / lam_min
    x_ref = O.solve(F, b)
    err = np.linalg.norm(x - x_ref, axis=0) / np.linalg.norm(x_ref, axis=0)
    res = b - O.matvec(h, x)
    rel = np.linalg.norm(res, axis=0) / np.linalg.norm(b, axis=0)
    res_o = b - O.matvec(h, x_ref)
    rel_o = np.linalg.norm(res_o, axis=0) / np.linalg.norm(b, axis=0)
    print(f"grid_exp_64k: kappa ~ {kappa:.3e} (lambda_max {lam_max:.4e}, lambda_min "
          f"{lam_min:.4e}); x rel err max {err.max():.3e}; residual max {rel.max():.3e} "
          f"(oracle's {rel_o.max():.3e}); logdet {dev.logdet():.10e} vs oracle "
          f"{O.logdet(F):.10e}")
    assert rel.max() <= max(1e-13, 10 * rel_o.max()), (rel.max(), rel_o.max())
    check_end_to_end(dev, F, b, x)
    # the mixed factor at this condition number: plain refinement still
    # contracts; the tolerance is 1e-11 because the FP64 residual of the exact
    # solution itself sits near 1e-12 here
    dev.factorize("fp32", ir_tol=1e-11, ir_max_it=30)
    xm = dev.solve(hss.colmajor(b)).cpu().numpy()
    info = dev.last_info()
    resm = b - O.matvec(h, xm)
    relm = np.linalg.norm(resm, axis=0) / np.linalg.norm(b, axis=0)
    errm = np.linalg.norm(xm - x_ref, axis=0) / np.linalg.norm(x_ref, axis=0)
    print(f"grid_exp_64k mixed fp32: {info['ir_iters']} refinement iterations, residual "
          f"{relm.max():.3e}, x rel err vs oracle {errm.max():.3e}")
    assert info["code"] == 0 and relm.max() <= 1e-11 and errm.max() <= 1e-9


# ---------------------------------------------------------------- basis completion methods
@pytest.mark.parametrize("levels,leaf,rank", [(3, 100, 13), (2, 256, 64), (4, 96, 40),
                                               (2, 32, 32), (1, 64, 16)])
def test_cholqr_basis_method(levels, leaf, rank):
    """Cholesky QR + Householder reconstruction (hss_options.basis = CHOLQR) per
    step and end to end against the oracle, like the default method; square
    bases (rank = leaf) and one level included."""
    h = I.random_hss(levels, leaf, rank, seed=levels * 13 + leaf, orthonormal=False)
    dev = hss.HSS(h)
    dev.factorize("fp64", basis="cholqr")
    F = O.factor(h)
    b = I.rhs(h.n, 3, 7)
    x = dev.solve(hss.colmajor(b)).cpu().numpy()
    check_steps(dev, F, h)
    check_end_to_end(dev, F, b, x)


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_ill_conditioned_basis_falls_back_to_householder(prec):
    """A leaf basis with two columns parallel to 1e-9: its Gram matrix is not
    numerically positive definite, so that node (and only that node) is completed
    by the Householder kernel -- its V and T are bit for bit those of the
    Householder method -- and the solve still matches the oracle."""
    h = I.random_hss(3, 64, 16, seed=91, orthonormal=False)
    rng = np.random.default_rng(5)
    h.U[5][:, 1] = h.U[5][:, 0] * (1.0 + 1e-9) + 1e-9 * rng.standard_normal(64)
    auto, ref = hss.HSS(h), hss.HSS(h)
    auto.factorize(prec, basis="cholqr")
    ref.factorize(prec, basis="householder")
    auto.sync()
    ref.sync()
    L = h.levels
    Va, Ta, Vr, Tr = auto.export("V", L), auto.export("T", L), ref.export("V", L), ref.export("T", L)
    assert np.array_equal(Va[5], Vr[5]) and np.array_equal(Ta[5], Tr[5])
    assert not np.array_equal(Va[4], Vr[4])           # a well-conditioned node: reconstruction
    tol = 50 * 64 * (EPS if prec == "fp64" else 6e-8)
    check_close(q_from_vt(Va[4], Ta[4]), q_from_vt(Vr[4], Tr[4]), tol, "Q node 4")
    b = I.rhs(h.n, 2, 3)
    x = auto.solve(hss.colmajor(b)).cpu().numpy()
    x_ref = O.solve(O.factor(h), b)
    err = np.linalg.norm(x - x_ref, axis=0) / np.linalg.norm(x_ref, axis=0)
    assert err.max() <= 1e-10, err


def test_rank_above_the_per_node_limit():
    """Rank 176 (block order 352 above the leaves) with the Cholesky QR method:
    FP64 completes the bases with the Householder kernel (the reconstruction's
    r x r block exceeds shared memory), FP32 with the reconstruction; both per
    step against the oracle."""
    h = I.random_hss(2, 256, 176, seed=176, orthonormal=False)
    dev = hss.HSS(h)
    dev.factorize("fp64", basis="cholqr")
    F = O.factor(h)
    b = I.rhs(h.n, 2, 7)
    x = dev.solve(hss.colmajor(b)).cpu().numpy()
    check_steps(dev, F, h)
    check_end_to_end(dev, F, b, x)
    dev.factorize("fp32", basis="cholqr")
    dev.sync()
    F32 = O.factor(h, dtype=np.float32)
    for l in range(h.levels, 0, -1):
        V, T = dev.export("V", l), dev.export("T", l)
        for i in range(2 ** l):
            check_close(q_from_vt(V[i], T[i]), F32.Q[l][i].astype(np.float64), 2e-4,
                        f"Q32 l={l} i={i}")


# ---------------------------------------------------------------- schedule of the solve
@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_async_and_level_schedules_agree(prec):
    """Eight levels (so the tree launches cover levels 6 .. 1 and two level-by-level
    levels sit below them): the asynchronous schedule of the upper solve levels
    and the level-by-level one give the oracle's solution."""
    h = I.random_hss(8, 32, 8, seed=8, orthonormal=False)
    F = O.factor(h)
    b = I.rhs(h.n, 16, 2)
    x_ref = O.solve(F, b)
    for sched in ("async", "levels"):
        dev = hss.HSS(h)
        dev.factorize(prec, schedule=sched)
        x = dev.solve(hss.colmajor(b)).cpu().numpy()
        err = np.linalg.norm(x - x_ref, axis=0) / np.linalg.norm(x_ref, axis=0)
        assert err.max() <= 1e-10, (sched, err.max())


def test_solve_wait_budget_runs_out():
    """The backward sweep's ready-flag waits with a budget that gives up at once:
    the solve reports HSS_ERR_TIMEOUT (with the level and node where the first
    wait gave up) at the next synchronizing call, and a normal factorization and
    solve of the same object afterwards are correct."""
    h = I.random_hss(4, 32, 8, seed=44, orthonormal=False)
    dev = hss.HSS(h)
    dev.factorize("fp64", wait_budget=-1)
    b = I.rhs(h.n, 2, 3)
    dev.solve(hss.colmajor(b))
    info = dev.last_info()
    assert info["code"] == -6 and info["level"] >= 2, info
    dev.factorize("fp64")
    x = dev.solve(hss.colmajor(b)).cpu().numpy()
    assert dev.last_info()["code"] == 0
    x_ref = O.solve(O.factor(h), b)
    err = np.linalg.norm(x - x_ref, axis=0) / np.linalg.norm(x_ref, axis=0)
    assert err.max() <= 1e-10, err


# ---------------------------------------------------------------- autotuner
@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_autotuner_choices_and_cache(prec, tmp_path):
    """hss_tune measures the candidates and keeps the fastest; the object is left
    factorized with them and still matches the oracle; a second object of the
    same shape reads the choice from the cache file instead of measuring."""
    h = I.random_hss(7, 64, 16, seed=70, orthonormal=False)
    cache = str(tmp_path / "tune.txt")
    dev = hss.HSS(h)
    t = dev.tune(prec, nrhs=4, cache=cache)
    assert t["basis"] in ("householder", "cholqr") and t["schedule"] in ("async", "levels")
    assert not t["from_cache"] and 0 < t["factor_ms"] < 1e4 and 0 < t["solve_ms"] < 1e4
    panels = t["measured"]["factor_ms_householder_panel"]
    assert set(panels) == ({"16"} if prec == "fp64" else {"16", "32"}), t
    assert t["ql_panel"] in (16, 32) and min(t["measured"]["factor_ms"].values()) == t["factor_ms"]
    assert t["ir_lanes"] == 1 or prec == "fp32"
    assert set(t["measured"]["solve_ms_by_lanes"]) == ({"1"} if prec == "fp64" else {"1", "2"})
    b = I.rhs(h.n, 4, 1)
    x = dev.solve(hss.colmajor(b)).cpu().numpy()
    x_ref = O.solve(O.factor(h), b)
    assert (np.linalg.norm(x - x_ref, axis=0) / np.linalg.norm(x_ref, axis=0)).max() <= 1e-10
    dev2 = hss.HSS(h)
    t2 = dev2.tune(prec, nrhs=4, cache=cache)
    assert t2["from_cache"] and t2["basis"] == t["basis"] and t2["schedule"] == t["schedule"]
    assert t2["ql_panel"] == t["ql_panel"]
    dev2.factorize(prec, basis="auto", schedule="auto")
    x2 = dev2.solve(hss.colmajor(b)).cpu().numpy()
    assert (np.linalg.norm(x2 - x_ref, axis=0) / np.linalg.norm(x_ref, axis=0)).max() <= 1e-10


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_leaf_768_sixteen_columns(prec):
    """The largest leaf order with 16 right-hand sides per pass in FP64 (the
    backward sweep keeps only the row-major vector in shared memory, so the
    panels fit), against the oracle."""
    h = I.random_hss(2, 768, 96, seed=768, orthonormal=False)
    dev = hss.HSS(h)
    dev.factorize(prec)
    b = I.rhs(h.n, 16, 3)
    x = dev.solve(hss.colmajor(b)).cpu().numpy()
    F = O.factor(h)
    x_ref = O.solve(F, b)
    err = np.linalg.norm(x - x_ref, axis=0) / np.linalg.norm(x_ref, axis=0)
    assert err.max() <= 1e-10, err
    if prec == "fp64":
        check_end_to_end(dev, F, b, x)


def test_ql_panel_option_checked():
    h = I.random_hss(2, 32, 8, seed=25)
    dev = hss.HSS(h)
    with pytest.raises(hss.HSSError) as ei:
        dev.factorize("fp32", ql_panel=24)
    assert ei.value.code == -1
    dev.factorize("fp64", ql_panel=32)     # FP64 has 16-column panels only: ignored
    x = dev.solve(hss.colmajor(np.ones(h.n))).cpu().numpy()
    x_ref = O.solve(O.factor(h), np.ones((h.n, 1)))
    assert np.abs(x.reshape(-1) - x_ref.reshape(-1)).max() <= 1e-10 * np.abs(x_ref).max()


# ---------------------------------------------------------------- leaf 1024
def test_leaf_1024_rank_256_mixed_against_oracle():
    """The node shape of the largest workload (leaf 1024, rank 256: the exponential
    covariance on the unit cube, N scaled to 8,192, 3 levels): the FP32 factor
    per step against the oracle's float32 factor (basis completion with 16-column
    panels and four rows a thread, L^RR, Â^SS), then FP32, TF32 x3 and BF16 x3
    factors refined to 1e-12 with the FP64 residual against the FP64 oracle's
    solution.  The FP64 factor at this rank exceeds the basis kernel's shared
    memory and is refused."""
    w = I.scaled(I.WORKLOADS["cube_exp_2m"], 8192)
    h = I.build_hss(w)
    assert (h.leaf, h.rank, h.levels) == (1024, 256, 3)
    dev = hss.HSS(h)
    dev.factorize("fp32")
    F32 = O.factor(h, dtype=np.float32)
    for l in range(h.levels, 0, -1):
        V, T, LB, M = (dev.export(k, l) for k in ("V", "T", "LB", "M"))
        for i in range(2 ** l):
            b, r = V.shape[1], V.shape[2]
            c = b - r
            check_close(q_from_vt(V[i], T[i]), F32.Q[l][i].astype(np.float64), 2e-4,
                        f"Q32 l={l} i={i}")
            check_close(LB[i], F32.LB[l][i].astype(np.float64), 2e-4, f"L_B32 l={l} i={i}")
            check_close(np.tril(M[i][:c, :c]), F32.LRR[l][i].astype(np.float64), 1e-3,
                        f"L^RR32 l={l} i={i}")
            check_close(np.tril(M[i][c:, c:]), np.tril(F32.SS[l][i]).astype(np.float64), 1e-3,
                        f"SS32 l={l} i={i}")
    b = I.rhs(h.n, 4, w.seed + 1)
    x_ref = O.solve(O.factor(h), b)
    for prec in ("fp32", "tf32", "bf16"):
        dev.factorize(prec)
        x = dev.solve(hss.colmajor(b)).cpu().numpy()
        res = b - O.matvec(h, x)
        assert (np.linalg.norm(res, axis=0) / np.linalg.norm(b, axis=0)).max() <= 1e-12, prec
        err = np.linalg.norm(x - x_ref, axis=0) / np.linalg.norm(x_ref, axis=0)
        assert err.max() <= 1e-10, (prec, err)
    with pytest.raises(hss.HSSError) as ei:
        dev.factorize("fp64")
    assert ei.value.code == -1


def test_leaf_1024_fp64_per_step():
    """FP64 at leaf 1024 with rank 160 (within the basis kernel's shared memory):
    every step of every node and the solution against the oracle."""
    h = I.random_hss(2, 1024, 160, seed=1024, orthonormal=False)
    dev, F, b, x = run_both(h, 16)
    check_steps(dev, F, h)
    check_end_to_end(dev, F, b, x)
