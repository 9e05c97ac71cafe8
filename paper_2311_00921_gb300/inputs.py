"""Seeded synthetic HSS inputs (points, kernel matrices, nested-basis compression).

This module builds the *input* of the ULV factorization: an HSS matrix given by
its generators (leaf diagonal blocks D, leaf bases U, transfer matrices E and
sibling couplings S), in the notation of Sec. 2 of the paper (Eq. 1, Eq. 2 and
the nested-basis block of the HSS construction figure).  It holds none of the
ULV arithmetic: no basis completion, no QᵀDQ, no Cholesky, no solve.  Both the
CPU oracle (through the tests) and the GPU path consume what it returns.

Conventions
-----------
* Points are permuted into cluster (tree) order once; every vector the solver
  sees is in that order.  ``HSSMatrix.perm[k]`` is the original index of the
  point at cluster position k.
* Levels: leaves are at level L, the root at level 0.  Node i of level l has
  children 2i and 2i+1 at level l+1.
* ``D[i]``      leaf i's dense diagonal block, b_i x b_i (symmetric).
* ``U[i]``      leaf i's basis, b_i x r_i (orthonormal columns as generated;
                the solver does not rely on orthonormality).
* ``E[l][i]``   transfer matrix of node i at level l (1 <= l <= L-1),
                (r_{2i} + r_{2i+1}) x r_i, so that the nested basis of node i is
                blkdiag(Ũ_{2i}, Ũ_{2i+1}) E[l][i].
* ``S[l][k]``   coupling between siblings 2k and 2k+1 of level l (1 <= l <= L),
                r_{2k+1} x r_{2k}: A(I_{2k+1}, I_{2k}) = Ũ_{2k+1} S Ũ_{2k}ᵀ, and the
                transposed block above the diagonal.

Compression follows the interpolative (skeleton) form of the pivoted-QR
construction: a row ID of a sampled off-diagonal block picks r skeleton points
per node; interpolation matrices are orthonormalised bottom-up and their
triangular factors are pushed into the parents' transfers and into S.
"""
from __future__ import annotations

import dataclasses
import math
from typing import Dict, List, Optional

import numpy as np
import scipy.linalg as sla


# --------------------------------------------------------------------------
# workloads
# --------------------------------------------------------------------------
@dataclasses.dataclass(frozen=True)
class Workload:
    name: str
    n: int
    leaf: int
    rank: int
    geometry: str      # "cube" | "grid2d" | "sphere" | "line"
    kernel: str        # "inv" | "exp" | "yukawa" | "poly2"
    length: float      # correlation length of "exp" (ignored otherwise)
    shift: float       # diagonal shift / nugget
    nrhs: int
    seed: int

    @property
    def levels(self) -> int:
        return max(1, int(math.ceil(math.log2(self.n / self.leaf))))


# The three single-matrix workloads of the paper's electrostatics /
# geostatistics families at the sizes the benchmark uses.  Seeds: 1000 + index.
WORKLOADS: Dict[str, Workload] = {
    # N=4,096 unit cube, 1/(d+1e-3) + N^(1/3) I, leaf 256, 4 levels, rank 32
    "cube_inv_4k": Workload("cube_inv_4k", 4096, 256, 32, "cube", "inv", 0.0,
                            16.0, 1, 1000),
    # N=65,536 jittered 256x256 grid, exp(-d/0.1) + 1e-4 I, leaf 512, 7 levels, rank 128
    "grid_exp_64k": Workload("grid_exp_64k", 65536, 512, 128, "grid2d", "exp",
                             0.1, 1e-4, 8, 1001),
    # N=262,144 unit sphere, exp(-d)/(d+1e-3) + 64 I, leaf 512, 9 levels, rank 128
    "sphere_yukawa_256k": Workload("sphere_yukawa_256k", 262144, 512, 128,
                                   "sphere", "yukawa", 0.0, 64.0, 16, 1002),
    # N=2,097,152 unit cube, exp(-d/0.05) + 1e-3 I, leaf 1024, 11 levels, rank 256
    "cube_exp_2m": Workload("cube_exp_2m", 2097152, 1024, 256, "cube", "exp",
                            0.05, 1e-3, 4, 1004),
}


def scaled(w: Workload, n: int, **kw) -> Workload:
    """Same workload family at another size (leaf/rank kept unless overridden)."""
    return dataclasses.replace(w, n=n, name=f"{w.name}@{n}", **kw)


# --------------------------------------------------------------------------
# geometry and kernels
# --------------------------------------------------------------------------
def make_points(w: Workload, rng: np.random.Generator) -> np.ndarray:
    n = w.n
    if w.geometry == "cube":
        return rng.random((n, 3))
    if w.geometry == "sphere":
        g = rng.standard_normal((n, 3))
        return g / np.linalg.norm(g, axis=1, keepdims=True)
    if w.geometry == "grid2d":
        side = int(round(math.sqrt(n)))
        if side * side != n:
            raise ValueError("grid2d needs a square point count")
        i, j = np.meshgrid(np.arange(side), np.arange(side), indexing="ij")
        jit = rng.uniform(-0.25, 0.25, size=(2, side, side))
        p = np.stack([(i + 0.5 + jit[0]) / side, (j + 0.5 + jit[1]) / side], -1)
        return p.reshape(n, 2)
    if w.geometry == "line":
        return np.sort(rng.random((n, 1)), axis=0)
    raise ValueError(w.geometry)


def kernel_block(w: Workload, xa: np.ndarray, xb: np.ndarray) -> np.ndarray:
    """K(xa, xb) without the diagonal shift."""
    diff = xa[:, None, :] - xb[None, :, :]
    d = np.sqrt(np.einsum("ijk,ijk->ij", diff, diff))
    if w.kernel == "inv":
        return 1.0 / (d + 1e-3)
    if w.kernel == "exp":
        return np.exp(-d / w.length)
    if w.kernel == "yukawa":
        return np.exp(-d) / (d + 1e-3)
    if w.kernel == "poly2":
        # (1 + <x,y>)^2: exact rank 1 + dim + dim(dim+1)/2 everywhere
        g = xa @ xb.T
        return (1.0 + g) ** 2
    raise ValueError(w.kernel)


def cluster_order(points: np.ndarray, levels: int) -> List[np.ndarray]:
    """Median bisection along the longest bounding-box axis; left gets ceil(n/2).

    Returns the leaves' index arrays (original point indices) in tree order.
    """
    def split(ids: np.ndarray, depth: int) -> List[np.ndarray]:
        if depth == levels:
            return [ids]
        p = points[ids]
        ax = int(np.argmax(p.max(0) - p.min(0)))
        order = np.argsort(p[:, ax], kind="stable")
        half = (len(ids) + 1) // 2
        return split(ids[order[:half]], depth + 1) + split(ids[order[half:]], depth + 1)

    return split(np.arange(len(points)), 0)


# --------------------------------------------------------------------------
# the HSS container
# --------------------------------------------------------------------------
@dataclasses.dataclass
class HSSMatrix:
    levels: int
    sizes: np.ndarray                  # leaf sizes b_i (2^L)
    ranks: Dict[int, np.ndarray]       # ranks[l][i], l = 1..L
    D: List[np.ndarray]
    U: List[np.ndarray]
    E: Dict[int, List[np.ndarray]]     # l = 1..L-1
    S: Dict[int, List[np.ndarray]]     # l = 1..L
    perm: Optional[np.ndarray] = None
    points: Optional[np.ndarray] = None   # cluster-ordered points
    workload: Optional[Workload] = None

    @property
    def n(self) -> int:
        return int(self.sizes.sum())

    @property
    def uniform(self) -> bool:
        return (len(set(self.sizes.tolist())) == 1 and
                all(len(set(v.tolist())) == 1 for v in self.ranks.values()))

    @property
    def leaf(self) -> int:
        return int(self.sizes[0])

    @property
    def rank(self) -> int:
        return int(self.ranks[self.levels][0])

    def stacked(self):
        """(D, U, E, S) as stacked arrays [node][rows][cols] for a uniform tree.

        E and S are dicts level -> array.  Only valid when ``uniform``.
        """
        if not self.uniform:
            raise ValueError("stacked() needs a uniform tree")
        D = np.stack(self.D)
        U = np.stack(self.U)
        E = {l: np.stack(v) for l, v in self.E.items()}
        S = {l: np.stack(v) for l, v in self.S.items()}
        return D, U, E, S


def _parallel_map(fn, items):
    """Run fn over items on a thread pool (NumPy releases the GIL in its
    element-wise kernels and BLAS calls, so row blocks evaluate in parallel)."""
    items = list(items)
    if len(items) <= 1:
        for it in items:
            fn(it)
        return
    import concurrent.futures as cf
    import os
    workers = min(len(items), os.cpu_count() or 1)
    with cf.ThreadPoolExecutor(max_workers=workers) as ex:
        list(ex.map(fn, items))


def _row_id(M: np.ndarray, k: int, rng: np.random.Generator, oversample: int = 10):
    """Row interpolative decomposition M ~= X M[sk, :] (X[sk] = I), via a
    Gaussian sketch and column-pivoted QR of the sketch's transpose."""
    m = M.shape[0]
    k = min(k, m)
    if M.shape[1] > k + oversample:
        Y = M @ rng.standard_normal((M.shape[1], k + oversample))
    else:
        Y = M
    _, R, piv = sla.qr(Y.T, mode="economic", pivoting=True)
    sk = piv[:k]
    X = np.zeros((m, k))
    X[sk, np.arange(k)] = 1.0
    if k < m:
        if R.shape[0] >= k and abs(R[k - 1, k - 1]) > 1e-13 * abs(R[0, 0]):
            T = sla.solve_triangular(R[:k, :k], R[:k, k:])
        else:  # numerically rank-deficient sketch: least squares
            T = np.linalg.lstsq(Y[sk].T, Y[piv[k:]].T, rcond=None)[0]
        X[piv[k:], :] = T.T
    return sk, X


def build_hss(w: Workload, far_samples: Optional[int] = None, mode: str = None,
              clip: float = 1e-12) -> HSSMatrix:
    """Compress the shifted kernel matrix of workload ``w`` into HSS form.

    ``mode="orth"``: orthonormal U and E (thin QR of the ID interpolation
    matrices), S = R_c2 K(sk_c2, sk_c1) R_c1ᵀ.
    ``mode="spd"``: the same skeletons, but every basis is normalised in the
    metric of the Cholesky factor Λ of its diagonal block (scaling-and-
    compression): W = orth(Λ⁻¹ X), U = Λ W (non-orthonormal), E = Λ_p W_p with
    Λ_p = chol([[I, Sᵀ], [S, I]]), and the coupling S of every sibling pair is the
    exact projection Ω_c2ᵀ A(I_c2, I_c1) Ω_c1 of the kernel block on the whitened
    nested bases (O(N² r) work: meant for N up to ~65k).  Each such S has
    2-norm < 1 (a block of an SPD matrix with identity diagonal blocks; the
    singular values are clipped at 1 - clip against round-off), and the
    assembled matrix is SPD by construction for any basis quality: at every
    level it is Λ[(I - WWᵀ) + W H Wᵀ]Λᵀ with H the SPD matrix of the level above.  Leaf D blocks are the exact shifted kernel blocks in both modes.
    The default is "spd" for the exponential covariance (tiny nugget) and
    "orth" otherwise.
    """
    if mode is None:
        mode = "spd" if w.kernel == "exp" else "orth"
    rng = np.random.default_rng(w.seed)
    pts0 = make_points(w, rng)
    L = w.levels
    leaves = cluster_order(pts0, L)
    perm = np.concatenate(leaves)
    pts = pts0[perm]
    sizes = np.array([len(x) for x in leaves], dtype=np.int64)
    offs = np.concatenate([[0], np.cumsum(sizes)])
    n = w.n
    r = w.rank
    if far_samples is None:
        far_samples = max(2 * r, 64)
    crng = np.random.default_rng(w.seed + 7919)

    def node_range(l: int, i: int):
        span = 2 ** (L - l)
        return int(offs[i * span]), int(offs[(i + 1) * span])

    def clip_norm(X):
        if mode != "spd":
            return X
        u, sv, vt = np.linalg.svd(X)
        if sv.size and sv[0] > 1.0 - clip:
            X = (u * np.minimum(sv, 1.0 - clip)) @ vt
        return X

    D = []
    for i in range(2 ** L):
        a, b = offs[i], offs[i + 1]
        blk = kernel_block(w, pts[a:b], pts[a:b])
        blk[np.diag_indices_from(blk)] += w.shift
        D.append(0.5 * (blk + blk.T))

    ranks: Dict[int, np.ndarray] = {}
    U: List[np.ndarray] = []
    E: Dict[int, List[np.ndarray]] = {}
    S: Dict[int, List[np.ndarray]] = {}
    cand = [np.arange(offs[i], offs[i + 1]) for i in range(2 ** L)]
    skel: Dict[int, List[np.ndarray]] = {}
    Rfac: Dict[int, List[np.ndarray]] = {}

    for l in range(L, 0, -1):
        nn = 2 ** l
        ranks[l] = np.zeros(nn, dtype=np.int64)
        skel[l], Rfac[l] = [], []
        if l < L:
            E[l] = []
        lam_w = []
        for i in range(nn):
            sib = i ^ 1
            pa, pb = node_range(l - 1, i // 2)
            outside = n - (pb - pa)
            J = cand[sib]
            if outside > 0 and far_samples > 0:
                far = crng.integers(0, outside, size=min(far_samples, outside))
                far = np.where(far < pa, far, far + (pb - pa))
                J = np.concatenate([J, far])
            M = kernel_block(w, pts[cand[i]], pts[J])
            sk, X = _row_id(M, r, crng)
            ranks[l][i] = X.shape[1]
            skel[l].append(cand[i][sk])
            if l == L:
                Rc = None
                Y = X
            else:
                c1, c2 = 2 * i, 2 * i + 1
                Rc = sla.block_diag(Rfac[l + 1][c1], Rfac[l + 1][c2])
                Y = Rc @ X
            if mode == "spd":
                if l == L:
                    Lam = np.linalg.cholesky(D[i])
                else:
                    Sc = S[l + 1][i]
                    r1, r2 = Sc.shape[1], Sc.shape[0]
                    T = np.block([[np.eye(r1), Sc.T], [Sc, np.eye(r2)]])
                    Lam = np.linalg.cholesky(T)
                # fit the scaled rows Λ⁻¹ (Rc) M on the skeleton rows M[sk] by
                # least squares, so the interpolation error is small in the
                # scaled metric the definiteness argument uses
                Ms = M if Rc is None else Rc @ M
                Ms = sla.solve_triangular(Lam, Ms, lower=True)
                Ysc = np.linalg.lstsq(M[sk].T, Ms.T, rcond=None)[0].T
                Wq, R = np.linalg.qr(Ysc)
                Q = Lam @ Wq
                lam_w.append((Lam, Wq))
            else:
                Q, R = np.linalg.qr(Y)
            if l == L:
                U.append(Q)
            else:
                E[l].append(Q)
            Rfac[l].append(R)
        S[l] = []
        if mode == "spd":
            # whitened nested bases Ω (|I_i| x r): Ω_leaf = Λ⁻ᵀ W,
            # Ω_p = blkdiag(Ω_c1, Ω_c2) Λ_p⁻ᵀ W_p; the coupling of a sibling
            # pair is the exact projection Ω_c2ᵀ A(I_c2, I_c1) Ω_c1, a block of
            # the SPD matrix Ωᵀ A Ω with identity diagonal blocks, so |S| < 1.
            newOm = []
            for i in range(nn):
                Lam, Wq = lam_w[i]
                Om = sla.solve_triangular(Lam, Wq, lower=True, trans="T")
                if l < L:
                    Om = np.concatenate([Om_prev[2 * i] @ Om[:Om_prev[2 * i].shape[1]],
                                         Om_prev[2 * i + 1] @ Om[Om_prev[2 * i].shape[1]:]])
                newOm.append(Om)
            Om_prev = newOm
        for k2 in range(nn // 2):
            c1, c2 = 2 * k2, 2 * k2 + 1
            if mode == "spd":
                a1, b1 = node_range(l, c1)
                a2, b2 = node_range(l, c2)
                acc = np.zeros((b2 - a2, Om_prev[c1].shape[1]))
                step = max(1, (1 << 20) // max(1, b1 - a1))

                def rows(s0, a1=a1, b1=b1, a2=a2, b2=b2, acc=acc, Om=Om_prev[c1]):
                    s1 = min(b2, s0 + step)
                    acc[s0 - a2:s1 - a2] = kernel_block(w, pts[s0:s1], pts[a1:b1]) @ Om

                _parallel_map(rows, range(a2, b2, step))
                S[l].append(clip_norm(Om_prev[c2].T @ acc))
            else:
                Kss = kernel_block(w, pts[skel[l][c2]], pts[skel[l][c1]])
                S[l].append(Rfac[l][c2] @ Kss @ Rfac[l][c1].T)
        cand = [np.concatenate([skel[l][2 * p], skel[l][2 * p + 1]])
                for p in range(nn // 2)]

    return HSSMatrix(levels=L, sizes=sizes, ranks=ranks, D=D, U=U, E=E, S=S,
                     perm=perm, points=pts, workload=w)


def kernel_matrix(w: Workload, pts: np.ndarray) -> np.ndarray:
    """Dense shifted kernel matrix on cluster-ordered points (small N only)."""
    A = kernel_block(w, pts, pts)
    A[np.diag_indices_from(A)] += w.shift
    return 0.5 * (A + A.T)


def random_hss(levels: int, leaf: int, rank: int, seed: int, *,
               shift: float = None, orthonormal: bool = True) -> HSSMatrix:
    """Random-generator HSS matrix (no kernel): SPD by a diagonal shift.

    Bases are random Gaussian (orthonormalised if requested), transfers and
    couplings Gaussian.  The shift defaults to a bound that dominates the
    off-diagonal part's norm, so the assembled matrix is SPD.
    """
    rng = np.random.default_rng(seed)
    L, r, b = levels, rank, leaf

    def basis(m, k):
        X = rng.standard_normal((m, k)) / math.sqrt(m)
        return np.linalg.qr(X)[0] if orthonormal else X

    U = [basis(b, r) for _ in range(2 ** L)]
    E = {l: [basis(2 * r, r) for _ in range(2 ** l)] for l in range(1, L)}
    S = {l: [rng.standard_normal((r, r)) / math.sqrt(r) for _ in range(2 ** (l - 1))]
         for l in range(1, L + 1)}
    if shift is None:
        # ||off-diagonal part|| <= sum_l max_k ||S_lk|| * (max nested-basis norm)^2
        nb = max(np.linalg.norm(u, 2) for u in U)
        bound = 0.0
        for l in range(L, 0, -1):
            bound += max(np.linalg.norm(s, 2) for s in S[l]) * nb * nb
            if l > 1:
                nb *= max(np.linalg.norm(e, 2) for e in E[l - 1])
        shift = 2.0 * bound + 1.0
    D = []
    for _ in range(2 ** L):
        G = rng.standard_normal((b, b)) / math.sqrt(b)
        D.append(G @ G.T + shift * np.eye(b))
    ranks = {l: np.full(2 ** l, r, dtype=np.int64) for l in range(1, L + 1)}
    return HSSMatrix(levels=L, sizes=np.full(2 ** L, b, dtype=np.int64), ranks=ranks,
                     D=D, U=U, E=E, S=S)


def rhs(n: int, nrhs: int, seed: int) -> np.ndarray:
    """N(0,1) right-hand sides, column-major n x nrhs as a Fortran-ordered array."""
    rng = np.random.default_rng(seed)
    return np.asfortranarray(rng.standard_normal((n, nrhs)))
