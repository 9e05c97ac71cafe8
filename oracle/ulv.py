"""CPU oracle of the HSS-ULV factorization and solve (FP64, NumPy/SciPy).

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import this module.  It shares no code with
the CUDA path and imports nothing from the package.

It follows the paper step by step, one node at a time, with library primitives
(LAPACK QR / Cholesky / triangular solve via NumPy and SciPy) as the steps:

* basis completion, Eq. 2-3 (Sec. 2): every node basis B (b x r) is completed to
  a square orthogonal Q = [Q^R  Q^S] with the redundant part first and Q^S
  spanning B.  Reading: the completion is the Householder QL factorization
  B = Q [0; L_B] (LAPACK's dgeqlf convention), computed here as the QR of the
  row- and column-reversed basis.  Q^S has exactly the span of B; L_B = Q^Sᵀ B
  is r x r lower triangular.
* diagonal product (the first step of Alg. 2's node loop, Eq. dense-split):
  Â = Qᵀ A_i Q.
* partial Cholesky, Eq. partial-Cholesky (Alg. 2): L^RR = chol(Â^RR),
  L^SR = Â^SR L^RR⁻ᵀ (reading of the garbled second line), Â^SS -= L^SR L^SRᵀ.
* merge (Alg. 2, after each level): the parent of siblings (c1, c2) gets
  [[Â^SS_c1, Ŝᵀ], [Ŝ, Â^SS_c2]] with Ŝ = L_B(c2) S L_B(c1)ᵀ, and the basis
  blkdiag(L_B(c1), L_B(c2)) E_p.  (The skeleton coordinates change from Ũ to
  Q^S, which rescales the coupling and the transfer by L_B.)
* root Cholesky, the last step of Alg. 2.
* factorized form and solve, Eq. hss-ulv-final-form and the solve that follows
  it (Sec. 3.2), read as ordered products; U^F is applied transposed on the way
  down and plain on the way up.
* log-determinant from the factorized form: Q is orthogonal, so
  log det A = 2 Σ log diag(L^RR) over all nodes + 2 Σ log diag(L_0).
* HSS matvec (the product A·b of the construction-error formula, Sec. 5.1) and
  iterative refinement with a low-precision factor as preconditioner.
* ``assemble_dense``: the plain definition of the HSS matrix (nested-basis
  block formula of Sec. 2), used for dense-Cholesky checks at small N.
"""
from __future__ import annotations

import math
from typing import Dict, List

import numpy as np
import scipy.linalg as sla


# --------------------------------------------------------------------------
# definition of the HSS matrix
# --------------------------------------------------------------------------
def nested_bases(h) -> Dict[int, List[np.ndarray]]:
    """Ũ per level: Ũ_leaf = U, Ũ_p = blkdiag(Ũ_c1, Ũ_c2) E_p  (Sec. 2, nested basis)."""
    L = h.levels
    Ut = {L: [np.asarray(u, dtype=np.float64) for u in h.U]}
    for l in range(L - 1, 0, -1):
        Ut[l] = []
        for i, Ep in enumerate(h.E[l]):
            Ut[l].append(sla.block_diag(Ut[l + 1][2 * i], Ut[l + 1][2 * i + 1]) @ Ep)
    return Ut


def assemble_dense(h) -> np.ndarray:
    """A_hss as a dense N x N matrix (small N).

    Leaf diagonal blocks are D_i; the block between siblings c1=2k, c2=2k+1 of
    level l is Ũ_c2 S_{l;k} Ũ_c1ᵀ below the diagonal and its transpose above.
    """
    L = h.levels
    sizes = np.asarray(h.sizes)
    offs = np.concatenate([[0], np.cumsum(sizes)])
    n = int(offs[-1])
    A = np.zeros((n, n))
    for i, Di in enumerate(h.D):
        A[offs[i]:offs[i + 1], offs[i]:offs[i + 1]] = Di
    Ut = nested_bases(h)
    for l in range(L, 0, -1):
        span = 2 ** (L - l)
        for k, S in enumerate(h.S[l]):
            c1, c2 = 2 * k, 2 * k + 1
            r1 = slice(offs[c1 * span], offs[(c1 + 1) * span])
            r2 = slice(offs[c2 * span], offs[(c2 + 1) * span])
            blk = Ut[l][c2] @ S @ Ut[l][c1].T
            A[r2, r1] = blk
            A[r1, r2] = blk.T
    return A


# --------------------------------------------------------------------------
# ULV factorization (Alg. 2)
# --------------------------------------------------------------------------
def complete_basis(B: np.ndarray, dtype=np.float64):
    """Householder QL completion of B (b x r): returns (Q, L_B).

    Q = [Q^R Q^S] is b x b orthogonal with the redundant part first (Eq. 3) and
    B = Q [0; L_B], L_B lower triangular r x r.  Computed as the Householder QR
    of the reversed matrix F_b B F_r (LAPACK dgeqrf signs: beta = -sign(alpha)|x|),
    then Q = F_b Q' F_b and L_B = F_r R' F_r.
    """
    b, r = B.shape
    Bf = np.asarray(B, dtype=dtype)[::-1, ::-1]
    Qp, Rp = np.linalg.qr(Bf, mode="complete")
    Q = np.ascontiguousarray(Qp[::-1, ::-1])
    LB = np.ascontiguousarray(Rp[:r, :r][::-1, ::-1])
    return Q, LB


class NotSPD(np.linalg.LinAlgError):
    def __init__(self, level, node, col):
        super().__init__(f"not SPD at level {level} node {node} column {col}")
        self.level, self.node, self.col = level, node, col


def _chol(A, level, node):
    try:
        return np.linalg.cholesky(A)
    except np.linalg.LinAlgError:
        # report the first failing column like LAPACK potrf's info
        for j in range(1, A.shape[0] + 1):
            try:
                np.linalg.cholesky(A[:j, :j])
            except np.linalg.LinAlgError:
                raise NotSPD(level, node, j - 1) from None
        raise NotSPD(level, node, -1) from None


class ULVFactor:
    """Per level l (L..1) and node: Q, L_B, L^RR, L^SR, Â^SS; the root L_0."""

    def __init__(self, levels):
        self.levels = levels
        self.Q: Dict[int, List[np.ndarray]] = {}
        self.LB: Dict[int, List[np.ndarray]] = {}
        self.LRR: Dict[int, List[np.ndarray]] = {}
        self.LSR: Dict[int, List[np.ndarray]] = {}
        self.SS: Dict[int, List[np.ndarray]] = {}
        self.Ahat: Dict[int, List[np.ndarray]] = {}   # Qᵀ A Q before the Cholesky
        self.Anode: Dict[int, List[np.ndarray]] = {}  # the node's diagonal block A
        self.Bnode: Dict[int, List[np.ndarray]] = {}  # the node's basis B
        self.L0 = None
        self.dtype = np.float64


def node_step(A, B, dtype=np.float64, level=-1, node=-1):
    """One node of Alg. 2: basis completion (Eq. 2-3), diagonal product
    Â = Qᵀ A Q and partial Cholesky (Eq. partial-Cholesky).
    Returns (Q, L_B, Â, L^RR, L^SR, Â^SS)."""
    A = np.asarray(A, dtype=dtype)
    B = np.asarray(B, dtype=dtype)
    b, r = B.shape
    c = b - r
    Q, LB = complete_basis(B, dtype)
    Ah = Q.T @ A @ Q
    Ah = 0.5 * (Ah + Ah.T)
    LRR = _chol(Ah[:c, :c], level, node) if c > 0 else np.zeros((0, 0), dtype)
    if c > 0:
        LSR = sla.solve_triangular(LRR, Ah[c:, :c].T, lower=True).T
    else:
        LSR = np.zeros((r, 0), dtype)
    SS = Ah[c:, c:] - LSR @ LSR.T
    return Q, LB, Ah, LRR, LSR, SS


def factor(h, dtype=np.float64) -> ULVFactor:
    """Alg. 2: for l = L..1 {diagonal product; partial Cholesky; merge}; Cholesky(A_0).

    ``dtype`` float32 runs every step in single precision (an emulated
    low-precision factor for iterative refinement); the root stays FP64 as in
    the mixed path.
    """
    L = h.levels
    F = ULVFactor(L)
    F.dtype = dtype
    A_lvl = [np.asarray(d, dtype=dtype) for d in h.D]
    B_lvl = [np.asarray(u, dtype=dtype) for u in h.U]
    for l in range(L, 0, -1):
        for key in ("Q", "LB", "LRR", "LSR", "SS", "Ahat", "Anode", "Bnode"):
            getattr(F, key)[l] = []
        for i in range(2 ** l):
            A, B = A_lvl[i], B_lvl[i]
            Q, LB, Ah, LRR, LSR, SS = node_step(A, B, dtype, l, i)
            F.Q[l].append(Q); F.LB[l].append(LB); F.LRR[l].append(LRR)
            F.LSR[l].append(LSR); F.SS[l].append(SS); F.Ahat[l].append(Ah)
            F.Anode[l].append(A); F.Bnode[l].append(B)
        # merge (Alg. 2): parents at level l-1
        newA, newB = [], []
        for p in range(2 ** (l - 1)):
            c1, c2 = 2 * p, 2 * p + 1
            Sh = F.LB[l][c2] @ np.asarray(h.S[l][p], dtype) @ F.LB[l][c1].T
            Ap = np.block([[F.SS[l][c1], Sh.T], [Sh, F.SS[l][c2]]])
            newA.append(Ap)
            if l > 1:
                newB.append(sla.block_diag(F.LB[l][c1], F.LB[l][c2]) @
                            np.asarray(h.E[l - 1][p], dtype))
        A_lvl, B_lvl = newA, newB
    A0 = np.asarray(A_lvl[0], dtype=np.float64)              # root stays FP64
    F.A0 = A0
    F.L0 = _chol(A0, 0, 0)                                   # root Cholesky of Alg. 2
    return F


def logdet(F: ULVFactor) -> float:
    """log det A = 2 Σ_nodes Σ_j log L^RR_jj + 2 Σ_j log L_0,jj  (from the factorized form)."""
    terms = [np.log(np.diag(F.L0).astype(np.float64))]
    for l in range(F.levels, 0, -1):
        for LRR in F.LRR[l]:
            if LRR.size:
                terms.append(np.log(np.diag(LRR).astype(np.float64)))
    t = np.concatenate(terms)
    return float(2.0 * math.fsum(t.tolist()))


def solve(F: ULVFactor, b: np.ndarray) -> np.ndarray:
    """x = A⁻¹ b by the ULV forward sweep (leaves -> root), the root solve and the
    backward sweep (root -> leaves), Sec. 3.2 solve formula read as ordered products."""
    L = F.levels
    dt = F.dtype
    b = np.asarray(b)
    vec1 = b.ndim == 1
    y = np.asarray(b.reshape(b.shape[0], -1), dtype=dt)
    z = {}        # z[l][i] = L^RR⁻¹ y^R of node i
    seg = {}      # segment of node i at level l in the level's vector
    cur = y
    for l in range(L, 0, -1):
        z[l] = []
        sizes = [F.Q[l][i].shape[0] for i in range(2 ** l)]
        offs = np.concatenate([[0], np.cumsum(sizes)])
        seg[l] = offs
        parent = []
        for i in range(2 ** l):
            Q, LRR, LSR = F.Q[l][i], F.LRR[l][i], F.LSR[l][i]
            c = LRR.shape[0]
            yi = Q.T @ cur[offs[i]:offs[i + 1]]              # U^Fᵀ b
            zR = sla.solve_triangular(LRR, yi[:c], lower=True) if c else yi[:0]
            yS = yi[c:] - LSR @ zR
            z[l].append(zR)
            parent.append(yS)
        cur = np.concatenate(parent, axis=0)                 # permute into level l-1
    w = sla.cho_solve((F.L0.astype(np.float64), True), cur.astype(np.float64)).astype(dt)
    for l in range(1, L + 1):
        offs_parent_r = 0
        xs = []
        for i in range(2 ** l):
            Q, LRR, LSR = F.Q[l][i], F.LRR[l][i], F.LSR[l][i]
            c = LRR.shape[0]
            r = Q.shape[0] - c
            xS = w[offs_parent_r:offs_parent_r + r]
            offs_parent_r += r
            if c:
                xR = sla.solve_triangular(LRR, z[l][i] - LSR.T @ xS, lower=True, trans="T")
            else:
                xR = xS[:0]
            xs.append(Q @ np.concatenate([xR, xS], axis=0))   # U^F x̂
        w = np.concatenate(xs, axis=0)
    x = np.asarray(w, dtype=np.float64)
    return x[:, 0] if vec1 else x


# --------------------------------------------------------------------------
# HSS matvec and iterative refinement
# --------------------------------------------------------------------------
def matvec(h, x: np.ndarray) -> np.ndarray:
    """y = A_hss x by an upward pass (x̂ = Ũᵀ x through U and E), the sibling
    couplings at every level, a downward pass and the leaf diagonal blocks."""
    L = h.levels
    x = np.asarray(x, dtype=np.float64)
    vec1 = x.ndim == 1
    X = x.reshape(x.shape[0], -1)
    sizes = np.asarray(h.sizes)
    offs = np.concatenate([[0], np.cumsum(sizes)])
    xh = {L: [h.U[i].T @ X[offs[i]:offs[i + 1]] for i in range(2 ** L)]}
    for l in range(L - 1, 0, -1):
        xh[l] = [h.E[l][i].T @ np.concatenate([xh[l + 1][2 * i], xh[l + 1][2 * i + 1]])
                 for i in range(2 ** l)]
    yh = {l: [np.zeros_like(v) for v in xh[l]] for l in xh}
    for l in range(1, L + 1):
        for k, S in enumerate(h.S[l]):
            yh[l][2 * k + 1] += S @ xh[l][2 * k]
            yh[l][2 * k] += S.T @ xh[l][2 * k + 1]
    for l in range(1, L):
        for i in range(2 ** l):
            t = h.E[l][i] @ yh[l][i]
            r1 = yh[l + 1][2 * i].shape[0]
            yh[l + 1][2 * i] += t[:r1]
            yh[l + 1][2 * i + 1] += t[r1:]
    Y = np.zeros_like(X)
    for i in range(2 ** L):
        Y[offs[i]:offs[i + 1]] = h.D[i] @ X[offs[i]:offs[i + 1]] + h.U[i] @ yh[L][i]
    return Y[:, 0] if vec1 else Y


def ir_solve(h, b: np.ndarray, F_low: ULVFactor, tol: float = 1e-12, max_it: int = 50):
    """Iterative refinement: x_0 = M⁻¹ b; r_k = b - A_hss x_k (FP64);
    x_{k+1} = x_k + M⁻¹ r_k, with M the (low-precision) ULV factor.
    Stops when every column's ‖r‖₂/‖b‖₂ <= tol.  Returns (x, iterations, residuals)."""
    b = np.asarray(b, dtype=np.float64).reshape(b.shape[0], -1)
    bn = np.linalg.norm(b, axis=0)
    x = solve(F_low, b).reshape(b.shape)
    hist = []
    for it in range(max_it + 1):
        r = b - matvec(h, x)
        rel = np.linalg.norm(r, axis=0) / bn
        hist.append(float(rel.max()))
        if rel.max() <= tol:
            return x, it, hist
        if it == max_it:
            break
        x = x + solve(F_low, r).reshape(b.shape)
    return x, max_it, hist
