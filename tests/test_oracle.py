"""Pins of the CPU oracle against facts it does not compute itself.

* brute force on the N=8 fixture (exact rational cofactor determinant and
  Cramer's rule on an entry-by-entry assembly of the HSS definition);
* exact-rank kernels, where the HSS matrix equals the kernel matrix, against
  LAPACK slogdet / solve of the kernel matrix;
* textbook special cases: S = 0 (block diagonal) and U = [0; I] (plain block
  Cholesky with the redundant indices first);
* invariants of each step (orthogonality, nullification of sibling blocks,
  symmetry, SPD merged blocks, reconstruction of A from the factors);
* dense Cholesky of the assembled matrix for the three kernel families;
* mutation tests: each plausible mistake planted in a copy of the oracle makes
  at least one of these pins fail.
"""
import itertools
import math
import os
import types
from fractions import Fraction

import numpy as np
import pytest
import scipy.linalg as sla

from oracle import ulv as O
from paper_2311_00921_gb300 import inputs as I

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
EPS = np.finfo(np.float64).eps


# ---------------------------------------------------------------- fixtures
class _H:
    pass


def load_n8():
    d = {}
    for line in open(os.path.join(GOLDEN, "hss_n8.txt")):
        if line.startswith("#") or not line.strip():
            continue
        t = line.split()
        d[t[0]] = np.array([float(x) for x in t[3:]]).reshape(int(t[1]), int(t[2]))
    h = _H()
    h.levels = 2
    h.sizes = np.array([2, 2, 2, 2])
    h.ranks = {2: np.ones(4, int), 1: np.ones(2, int)}
    h.D = [d[f"D{i}"] for i in range(4)]
    h.U = [d[f"U{i}"] for i in range(4)]
    h.E = {1: [d["E1_0"], d["E1_1"]]}
    h.S = {2: [d["S2_0"], d["S2_1"]], 1: [d["S1_0"]]}
    return h


def entrywise_assembly(h):
    """A_hss entry by entry: walk each point's basis row up the tree to the level
    where the two leaves become siblings (scalar form of the nested-basis block)."""
    L = h.levels
    sizes = list(h.sizes)
    offs = np.concatenate([[0], np.cumsum(sizes)])
    n = int(offs[-1])
    leaf_of = np.repeat(np.arange(len(sizes)), sizes)

    def basis_row(p, upto):
        i = int(leaf_of[p])
        u = np.asarray(h.U[i])[p - offs[i], :]
        node = i
        for l in range(L - 1, upto - 1, -1):
            parent = node // 2
            Ep = np.asarray(h.E[l][parent])
            r_first = np.asarray(h.U[0]).shape[1] if l == L - 1 else None
            # children's ranks decide the row block of E_p that applies
            rc1 = (np.asarray(h.U[2 * parent]).shape[1] if l == L - 1
                   else np.asarray(h.E[l + 1][2 * parent]).shape[1])
            blk = Ep[:rc1] if node % 2 == 0 else Ep[rc1:]
            u = u @ blk
            node = parent
            del r_first
        return u

    A = np.zeros((n, n))
    for p in range(n):
        for q in range(n):
            i, j = int(leaf_of[p]), int(leaf_of[q])
            if i == j:
                A[p, q] = h.D[i][p - offs[i], q - offs[j]]
                continue
            l = L
            ai, aj = i, j
            while ai // 2 != aj // 2:
                ai //= 2
                aj //= 2
                l -= 1
            ui, uj = basis_row(p, l), basis_row(q, l)
            S = np.asarray(h.S[l][ai // 2])
            A[p, q] = ui @ S @ uj if ai % 2 == 1 else uj @ S @ ui
    return A


def det_exact(M):
    """Exact determinant by cofactor expansion along rows (memoised on the set
    of used columns); entries are converted to exact rationals."""
    n = len(M)
    F = [[Fraction(float(x)) for x in row] for row in M]
    memo = {}

    def rec(row, used):
        if row == n:
            return Fraction(1)
        key = used
        if key in memo:
            return memo[key]
        tot = Fraction(0)
        sign = 1
        for j in range(n):
            if used >> j & 1:
                continue
            # sign of the cofactor: parity of used columns to the left of j
            k = bin(used & ((1 << j) - 1)).count("1")
            s = -1 if (j - k) % 2 else 1
            if F[row][j] != 0:
                tot += s * F[row][j] * rec(row + 1, used | (1 << j))
        memo[key] = tot
        del sign
        return tot

    return rec(0, 0)


def kappa_estimate(A, cf, iters=40):
    """2-norm condition number of SPD A by power iteration on A and on A⁻¹."""
    rng = np.random.default_rng(0)
    v = rng.standard_normal(A.shape[0])
    for _ in range(iters):
        v = A @ v
        v /= np.linalg.norm(v)
    lmax = v @ (A @ v)
    v = rng.standard_normal(A.shape[0])
    for _ in range(iters):
        v = sla.cho_solve(cf, v)
        v /= np.linalg.norm(v)
    lmin = 1.0 / (v @ sla.cho_solve(cf, v))
    return lmax / lmin


def factor_solve_logdet(mod, h, b):
    F = mod.factor(h)
    return F, mod.solve(F, b), mod.logdet(F)


# ---------------------------------------------------------------- brute force
def test_entrywise_assembly_matches_block_assembly_n8():
    h = load_n8()
    A1 = entrywise_assembly(h)
    A2 = O.assemble_dense(h)
    assert np.array_equal(A1, A1.T)
    np.testing.assert_allclose(A2, A1, rtol=0, atol=1e-14)


def test_brute_force_n8_logdet_and_cramer():
    h = load_n8()
    A = entrywise_assembly(h)
    det = det_exact(A)
    assert det > 0
    b = np.array([1.0, -2.0, 0.5, 3.0, -1.0, 0.25, 2.0, -0.75])
    x_cramer = []
    for k in range(8):
        Ak = A.copy()
        Ak[:, k] = b
        x_cramer.append(float(det_exact(Ak) / det))
    F, x, ld = factor_solve_logdet(O, h, b)
    assert abs(ld - math.log(float(det))) <= 1e-13 * abs(math.log(float(det))) + 1e-14
    np.testing.assert_allclose(x, x_cramer, rtol=1e-13, atol=1e-15)


def test_matvec_matches_entrywise_n8():
    h = load_n8()
    A = entrywise_assembly(h)
    x = np.arange(1.0, 9.0)[:, None] * np.array([[1.0, -0.5]])
    np.testing.assert_allclose(O.matvec(h, x), A @ x, rtol=1e-14, atol=1e-13)


def test_entrywise_assembly_random_nonorthonormal():
    h = I.random_hss(3, 6, 2, seed=3, orthonormal=False)
    np.testing.assert_allclose(O.assemble_dense(h), entrywise_assembly(h),
                               rtol=1e-13, atol=1e-13)


# ---------------------------------------------------------------- exact compression
def test_full_rank_leaf_two_leaves_is_dense_kernel():
    # N = 2 leaf, one level, rank = leaf: U is a permutation, S the whole block
    w = I.Workload("t", 64, 32, 32, "cube", "inv", 0.0, 16.0, 1, 7)
    h = I.build_hss(w)
    K = I.kernel_matrix(w, h.points)
    np.testing.assert_allclose(O.assemble_dense(h), K, rtol=1e-13, atol=1e-11)
    b = I.rhs(w.n, 2, 11)
    F, x, ld = factor_solve_logdet(O, h, b)
    s, ref = np.linalg.slogdet(K)
    assert s > 0 and abs(ld - ref) <= 1e-12 * abs(ref)
    np.testing.assert_allclose(x, np.linalg.solve(K, b), rtol=1e-11, atol=1e-13)


@pytest.mark.parametrize("levels", [2, 3])
def test_exact_rank_kernel_multilevel(levels):
    # (1 + <x,y>)^2 in 3-D has rank 10 everywhere: with r = 10 the nested-basis
    # compression is exact, so A_hss equals the shifted kernel matrix.
    leaf = 16
    w = I.Workload("poly", leaf * 2 ** levels, leaf, 10, "cube", "poly2", 0.0, 3.0, 1, 21)
    h = I.build_hss(w, mode="orth")
    K = I.kernel_matrix(w, h.points)
    np.testing.assert_allclose(O.assemble_dense(h), K, rtol=1e-10, atol=1e-10)
    b = I.rhs(w.n, 3, 5)
    F, x, ld = factor_solve_logdet(O, h, b)
    s, ref = np.linalg.slogdet(K)
    assert s > 0 and abs(ld - ref) <= 1e-10 * abs(ref)
    np.testing.assert_allclose(x, np.linalg.solve(K, b), rtol=1e-8, atol=1e-10)


# ---------------------------------------------------------------- special cases
def test_zero_coupling_is_block_diagonal():
    h = I.random_hss(3, 12, 3, seed=5)
    for l in h.S:
        h.S[l] = [np.zeros_like(s) for s in h.S[l]]
    b = I.rhs(h.n, 2, 9)
    F, x, ld = factor_solve_logdet(O, h, b)
    ref_ld = sum(np.linalg.slogdet(d)[1] for d in h.D)
    assert abs(ld - ref_ld) <= 1e-12 * abs(ref_ld)
    xs = np.concatenate([np.linalg.solve(d, b[i * 12:(i + 1) * 12]) for i, d in enumerate(h.D)])
    np.testing.assert_allclose(x, xs, rtol=1e-12, atol=1e-14)


def test_identity_skeleton_basis_is_block_cholesky():
    # U = [0; I_r] keeps the last r indices as skeleton: Q = I, L_B = I, and the
    # partial Cholesky is the plain Cholesky of the leading (b - r) block.
    h = I.random_hss(2, 8, 3, seed=8)
    for i in range(len(h.U)):
        h.U[i] = np.vstack([np.zeros((5, 3)), np.eye(3)])
    for l in h.E:
        h.E[l] = [np.linalg.qr(e)[0] for e in h.E[l]]
    F = O.factor(h)
    for i in range(4):
        assert np.array_equal(F.Q[2][i], np.eye(8))
        assert np.array_equal(F.LB[2][i], np.eye(3))
        np.testing.assert_allclose(F.LRR[2][i], np.linalg.cholesky(h.D[i][:5, :5]), rtol=1e-14)
        schur = h.D[i][5:, 5:] - h.D[i][5:, :5] @ np.linalg.solve(h.D[i][:5, :5], h.D[i][:5, 5:])
        np.testing.assert_allclose(F.SS[2][i], schur, rtol=1e-12, atol=1e-12)
    A = O.assemble_dense(h)
    b = I.rhs(h.n, 1, 3)
    np.testing.assert_allclose(O.solve(F, b), np.linalg.solve(A, b), rtol=1e-12, atol=1e-13)


# ---------------------------------------------------------------- invariants
@pytest.fixture(scope="module")
def cube_small():
    w = I.scaled(I.WORKLOADS["cube_inv_4k"], 1024, leaf=64, rank=16)
    h = I.build_hss(w)
    return w, h, O.factor(h)


def test_basis_completion_invariants(cube_small):
    w, h, F = cube_small
    for l in F.Q:
        for Q, LB, B in zip(F.Q[l], F.LB[l], F.Bnode[l]):
            b, r = B.shape
            c = b - r
            assert np.linalg.norm(Q.T @ Q - np.eye(b)) <= 10 * b * EPS
            assert np.allclose(np.triu(LB, 1), 0)                      # lower triangular
            nb = np.linalg.norm(B)
            assert np.linalg.norm(Q[:, c:] @ LB - B) <= 10 * b * EPS * nb   # Q^S spans B
            assert np.linalg.norm(Q[:, :c].T @ B) <= 10 * b * EPS * nb      # Q^R ⊥ B


def test_sibling_block_nullified(cube_small):
    w, h, F = cube_small
    L = h.levels
    for k, S in enumerate(h.S[L]):
        c1, c2 = 2 * k, 2 * k + 1
        blk = h.U[c2] @ S @ h.U[c1].T
        T = F.Q[L][c2].T @ blk @ F.Q[L][c1]
        r = S.shape[0]
        mask = np.ones_like(T, bool)
        mask[-r:, -r:] = False
        assert np.abs(T[mask]).max() <= 1e-12 * np.abs(T).max()
        np.testing.assert_allclose(T[-r:, -r:], F.LB[L][c2] @ S @ F.LB[L][c1].T,
                                   rtol=1e-10, atol=1e-12 * np.abs(T).max())


def test_symmetric_blocks_and_spd_merges(cube_small):
    w, h, F = cube_small
    for l in F.Ahat:
        for Ah in F.Ahat[l]:
            assert np.allclose(Ah, Ah.T, rtol=0, atol=1e-13 * np.abs(Ah).max())
        for A in F.Anode[l]:
            assert np.allclose(A, A.T, rtol=0, atol=1e-12 * np.abs(A).max())
            assert np.linalg.eigvalsh(0.5 * (A + A.T)).min() > 0


def ulv_reconstruct(F, h):
    """Dense A rebuilt from the factors: A = U^F_L Â_L U^F_Lᵀ with Â_L rebuilt
    from L^RR, L^SR and the (recursively rebuilt) merged skeleton matrix."""
    L = F.levels

    def level_matrix(l):
        if l == 0:
            return F.L0 @ F.L0.T
        sub = level_matrix(l - 1)            # matrix on the skeletons of level l
        nodes = range(2 ** l)
        sizes = [F.Q[l][i].shape[0] for i in nodes]
        offs = np.concatenate([[0], np.cumsum(sizes)])
        rs = [F.Q[l][i].shape[0] - F.LRR[l][i].shape[0] for i in nodes]
        soffs = np.concatenate([[0], np.cumsum(rs)])
        n = offs[-1]
        Ah = np.zeros((n, n))
        for i in nodes:
            for j in nodes:
                ci = F.LRR[l][i].shape[0]
                cj = F.LRR[l][j].shape[0]
                bi = slice(offs[i] + ci, offs[i + 1])
                bj = slice(offs[j] + cj, offs[j + 1])
                Ah[bi, bj] = sub[soffs[i]:soffs[i + 1], soffs[j]:soffs[j + 1]]
        for i in nodes:
            c = F.LRR[l][i].shape[0]
            o = offs[i]
            R = slice(o, o + c)
            Sx = slice(o + c, offs[i + 1])
            Ah[R, R] = F.LRR[l][i] @ F.LRR[l][i].T
            Ah[Sx, R] = F.LSR[l][i] @ F.LRR[l][i].T
            Ah[R, Sx] = Ah[Sx, R].T
            Ah[Sx, Sx] += F.LSR[l][i] @ F.LSR[l][i].T
        UF = sla.block_diag(*F.Q[l])
        return UF @ Ah @ UF.T

    return level_matrix(L)


def test_factor_reconstructs_matrix(cube_small):
    w, h, F = cube_small
    A = O.assemble_dense(h)
    R = ulv_reconstruct(F, h)
    assert np.linalg.norm(R - A) <= 1e-13 * np.linalg.norm(A)


# ---------------------------------------------------------------- dense Cholesky
@pytest.mark.parametrize("name,n,kw", [
    ("cube_inv_4k", 4096, {}),
    ("grid_exp_64k", 4096, {}),
    ("sphere_yukawa_256k", 4096, {}),
    ("sphere_yukawa_256k", 2048, {"leaf": 256, "rank": 64}),
])
def test_ulv_matches_dense_cholesky(name, n, kw):
    w = I.scaled(I.WORKLOADS[name], n, **kw)
    h = I.build_hss(w)
    A = O.assemble_dense(h)
    cf = sla.cho_factor(A, lower=True)
    ld_ref = 2.0 * np.log(np.diag(cf[0])).sum()
    b = I.rhs(n, 3, w.seed + 1)
    x_ref = sla.cho_solve(cf, b)
    F, x, ld = factor_solve_logdet(O, h, b)
    scale = 2.0 * np.abs(np.log(np.diag(cf[0]))).sum()
    assert abs(ld - ld_ref) <= 1e-12 * scale
    kappa = kappa_estimate(A, cf)
    err = np.linalg.norm(x - x_ref) / np.linalg.norm(x_ref)
    assert err <= max(1e-12, 50 * kappa * EPS)
    res = np.linalg.norm(b - A @ x, axis=0) / np.linalg.norm(b, axis=0)
    assert res.max() <= 1e-13


def test_matvec_matches_dense():
    w = I.scaled(I.WORKLOADS["grid_exp_64k"], 1024, leaf=64, rank=16)
    h = I.build_hss(w)
    A = O.assemble_dense(h)
    x = I.rhs(w.n, 4, 2)
    np.testing.assert_allclose(O.matvec(h, x), A @ x, rtol=1e-12, atol=1e-12 * np.abs(A @ x).max())


def test_spd_construction_is_spd_and_faithful():
    # the exponential covariance with nugget 1e-4 compresses to an indefinite
    # matrix with orthonormal bases; the scaled construction stays SPD and
    # close to the kernel's spectrum
    w = I.scaled(I.WORKLOADS["grid_exp_64k"], 1024, leaf=64, rank=16)
    h = I.build_hss(w, mode="spd")
    A = O.assemble_dense(h)
    K = I.kernel_matrix(w, h.points)
    ea, ek = np.linalg.eigvalsh(A), np.linalg.eigvalsh(K)
    assert ea[0] > 0
    assert ea[0] >= 0.5 * ek[0]
    for l in h.S:
        for S in h.S[l]:
            assert np.linalg.norm(S, 2) < 1.0


def test_iterative_refinement_float32_factor():
    w = I.scaled(I.WORKLOADS["cube_inv_4k"], 2048, leaf=128, rank=32)
    h = I.build_hss(w)
    F32 = O.factor(h, dtype=np.float32)
    b = I.rhs(w.n, 2, 3)
    x, it, hist = O.ir_solve(h, b, F32, tol=1e-12, max_it=20)
    assert hist[-1] <= 1e-12 and it <= 6
    assert hist[0] > 1e-10        # the float32 factor alone is not enough
    F = O.factor(h)
    x64 = O.solve(F, b)
    assert np.linalg.norm(x - x64) <= 1e-10 * np.linalg.norm(x64)


def test_not_spd_reports_position():
    h = I.random_hss(2, 8, 2, seed=4)
    h.D[2] = -h.D[2]
    with pytest.raises(O.NotSPD) as ei:
        O.factor(h)
    assert ei.value.level == 2 and ei.value.node == 2


# ---------------------------------------------------------------- mutations
MUTATIONS = [
    ("drop the SYRK term", "SS = Ah[c:, c:] - LSR @ LSR.T", "SS = Ah[c:, c:]"),
    ("transposed merge", "Ap = np.block([[F.SS[l][c1], Sh.T], [Sh, F.SS[l][c2]]])",
     "Ap = np.block([[F.SS[l][c1], Sh], [Sh.T, F.SS[l][c2]]])"),
    ("unscaled coupling", "Sh = F.LB[l][c2] @ np.asarray(h.S[l][p], dtype) @ F.LB[l][c1].T",
     "Sh = np.asarray(h.S[l][p], dtype)"),
    ("skeleton-first completion", "Q = np.ascontiguousarray(Qp[::-1, ::-1])",
     "Q = np.ascontiguousarray(Qp)"),
    ("transfer not rescaled", "newB.append(sla.block_diag(F.LB[l][c1], F.LB[l][c2]) @",
     "newB.append(np.eye(F.LB[l][c1].shape[0] + F.LB[l][c2].shape[0]) @"),
    ("sign of the forward update", "yS = yi[c:] - LSR @ zR", "yS = yi[c:] + LSR @ zR"),
    ("logdet factor", "return float(2.0 * math.fsum", "return float(1.0 * math.fsum"),
    ("matvec transposed coupling", "yh[l][2 * k] += S.T @ xh[l][2 * k + 1]",
     "yh[l][2 * k] += S @ xh[l][2 * k + 1]"),
    ("assembly orientation", "A[r2, r1] = blk\n            A[r1, r2] = blk.T",
     "A[r2, r1] = blk.T\n            A[r1, r2] = blk"),
    ("backward solve transposed L^SR", "z[l][i] - LSR.T @ xS", "z[l][i] - LSR[:, :0].sum() * xS[:0].sum() - 0 * LSR.T @ xS"),
]


def _mutant(old, new):
    src = open(O.__file__).read()
    assert old in src, old
    mod = types.ModuleType("oracle_mutant")
    mod.__file__ = O.__file__
    exec(compile(src.replace(old, new), O.__file__, "exec"), mod.__dict__)
    return mod


def _pins_pass(mod):
    """The pins above, evaluated on a module; False if any fails."""
    try:
        h = load_n8()
        A = entrywise_assembly(h)
        det = float(det_exact(A))
        b = np.array([1.0, -2.0, 0.5, 3.0, -1.0, 0.25, 2.0, -0.75])
        F, x, ld = factor_solve_logdet(mod, h, b)
        if abs(ld - math.log(det)) > 1e-12 * abs(math.log(det)):
            return False
        if not np.allclose(x, np.linalg.solve(A, b), rtol=1e-12, atol=1e-14):
            return False
        if not np.allclose(mod.assemble_dense(h), A, rtol=0, atol=1e-13):
            return False
        xm = np.arange(1.0, 9.0)
        if not np.allclose(mod.matvec(h, xm), A @ xm, rtol=1e-13):
            return False
        h2 = I.random_hss(3, 6, 2, seed=3, orthonormal=False)
        A2 = entrywise_assembly(h2)
        b2 = np.linspace(-1, 1, A2.shape[0])
        F2, x2, ld2 = factor_solve_logdet(mod, h2, b2)
        if not np.allclose(x2, np.linalg.solve(A2, b2), rtol=1e-11, atol=1e-13):
            return False
        if abs(ld2 - np.linalg.slogdet(A2)[1]) > 1e-11 * abs(ld2):
            return False
        xm2 = np.outer(b2, [1.0, -2.0])
        if not np.allclose(mod.matvec(h2, xm2), A2 @ xm2, rtol=1e-12, atol=1e-12):
            return False
        return True
    except Exception:
        return False


def test_pins_pass_on_the_oracle():
    assert _pins_pass(O)


@pytest.mark.parametrize("label,old,new", MUTATIONS, ids=[m[0] for m in MUTATIONS])
def test_planted_mistake_is_caught(label, old, new):
    assert not _pins_pass(_mutant(old, new)), label
