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
        # sx x sy jittered grid of the unit square (sx = sy when n is a square;
        # else a power-of-two sx when it divides n, else the largest divisor of
        # n not above sqrt(n))
        sx = int(round(math.sqrt(n)))
        if sx * sx != n:
            sx = 1 << int(math.ceil(math.log2(n) / 2))
        if n % sx:
            sx = max(d for d in range(1, int(math.isqrt(n)) + 1) if n % d == 0)
        sy = n // sx
        i, j = np.meshgrid(np.arange(sx), np.arange(sy), indexing="ij")
        jit = rng.uniform(-0.25, 0.25, size=(2, sx, sy))
        p = np.stack([(i + 0.5 + jit[0]) / sx, (j + 0.5 + jit[1]) / sy], -1)
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
        """One leaf order and one rank at every node of every level."""
        return (len(set(self.sizes.tolist())) == 1 and
                len({int(x) for v in self.ranks.values() for x in v}) == 1)

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
    """Run fn over items on a thread pool.  NumPy / LAPACK release the GIL; the
    BLAS is limited to one thread per call inside the pool when threadpoolctl is
    available, so the pool, not the BLAS, supplies the parallelism."""
    items = list(items)
    if len(items) <= 1:
        return [fn(it) for it in items]
    import concurrent.futures as cf
    import contextlib
    import os
    try:
        from threadpoolctl import threadpool_limits
        ctx = threadpool_limits(1)
    except Exception:  # pragma: no cover - not installed everywhere
        ctx = contextlib.nullcontext()
    workers = min(len(items), os.cpu_count() or 1)
    with ctx, cf.ThreadPoolExecutor(max_workers=workers) as ex:
        return list(ex.map(fn, items))


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


def _projected_block(w: Workload, pts_rows: np.ndarray, pts_cols: np.ndarray,
                     Om_cols: np.ndarray, device: str) -> np.ndarray:
    """K(rows, cols) @ Om_cols without forming K whole (torch, FP64, row chunks)."""
    import torch
    dev = torch.device(device)
    xc = torch.as_tensor(pts_cols, dtype=torch.float64, device=dev)
    om = torch.as_tensor(Om_cols, dtype=torch.float64, device=dev)
    out = torch.empty((len(pts_rows), om.shape[1]), dtype=torch.float64, device=dev)
    budget = (1 << 28) if dev.type == "cuda" else (1 << 23)
    step = max(1, budget // max(1, len(pts_cols)))
    for s0 in range(0, len(pts_rows), step):
        xr = torch.as_tensor(pts_rows[s0:s0 + step], dtype=torch.float64, device=dev)
        d = torch.cdist(xr, xc) if xr.shape[1] > 1 else (xr - xc.T).abs()
        if w.kernel == "inv":
            K = 1.0 / (d + 1e-3)
        elif w.kernel == "exp":
            K = torch.exp(-d / w.length)
        elif w.kernel == "yukawa":
            K = torch.exp(-d) / (d + 1e-3)
        elif w.kernel == "poly2":
            K = (1.0 + xr @ xc.T) ** 2
        else:
            raise ValueError(w.kernel)
        out[s0:s0 + step] = K @ om
    return out.cpu().numpy()


def build_hss(w: Workload, far_samples: Optional[int] = None, mode: str = "spd",
              clip: float = 1e-12, device: Optional[str] = None) -> HSSMatrix:
    """Compress the shifted kernel matrix of workload ``w`` into HSS form.

    ``mode="orth"``: orthonormal U and E (thin QR of the ID interpolation
    matrices), S = R_c2 K(sk_c2, sk_c1) R_c1ᵀ.  Fast (O(N r) kernel
    evaluations) but the compressed matrix loses definiteness once the
    compression error exceeds the smallest eigenvalue.
    ``mode="spd"`` (default): the same skeletons, but every basis is normalised
    in the metric of the Cholesky factor Λ of its diagonal block (scaling-and-
    compression): W = orth(Λ⁻¹ X) fitted by least squares in that metric,
    U = Λ W (non-orthonormal), E = Λ_p W_p with Λ_p = chol([[I, Sᵀ], [S, I]]);
    the coupling of every sibling pair is the exact projection
    Ω_c2ᵀ A(I_c2, I_c1) Ω_c1 of the kernel block on the whitened nested bases
    (Ω_leaf = Λ⁻ᵀ W, Ω_p = blkdiag(Ω_c1, Ω_c2) Λ_p⁻ᵀ W_p), an O(N² r) product
    computed in row chunks with torch (on ``device``: the GPU when available).
    Each S then has 2-norm < 1 (a block of an SPD matrix with identity diagonal
    blocks; singular values are clipped at 1 - clip against round-off) and the
    assembled matrix is SPD by construction for any basis quality: at every
    level it is Λ[(I - WWᵀ) + W H Wᵀ]Λᵀ with H the SPD matrix of the level above.
    Leaf D blocks are the exact shifted kernel blocks in both modes.
    """
    if device is None:
        try:
            import torch
            device = "cuda" if torch.cuda.is_available() else "cpu"
        except Exception:  # pragma: no cover
            device = "cpu"
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

    def node_range(l: int, i: int):
        span = 2 ** (L - l)
        return int(offs[i * span]), int(offs[(i + 1) * span])

    def clip_norm(X):
        u, sv, vt = np.linalg.svd(X)
        if sv.size and sv[0] > 1.0 - clip:
            X = (u * np.minimum(sv, 1.0 - clip)) @ vt
        return X

    def leaf_block(i):
        a, b = offs[i], offs[i + 1]
        blk = kernel_block(w, pts[a:b], pts[a:b])
        blk[np.diag_indices_from(blk)] += w.shift
        return 0.5 * (blk + blk.T)

    D = _parallel_map(leaf_block, range(2 ** L))

    ranks: Dict[int, np.ndarray] = {}
    U: List[np.ndarray] = []
    E: Dict[int, List[np.ndarray]] = {}
    S: Dict[int, List[np.ndarray]] = {}
    cand = [np.arange(offs[i], offs[i + 1]) for i in range(2 ** L)]
    skel: Dict[int, List[np.ndarray]] = {}
    Rfac: Dict[int, List[np.ndarray]] = {}
    Om_prev = None

    for l in range(L, 0, -1):
        nn = 2 ** l

        def compress(i, l=l, cand=cand):
            nrng = np.random.default_rng([w.seed, 7919, l, i])
            sib = i ^ 1
            pa, pb = node_range(l - 1, i // 2)
            outside = n - (pb - pa)
            J = cand[sib]
            if outside > 0 and far_samples > 0:
                far = nrng.integers(0, outside, size=min(far_samples, outside))
                far = np.where(far < pa, far, far + (pb - pa))
                J = np.concatenate([J, far])
            M = kernel_block(w, pts[cand[i]], pts[J])
            sk, X = _row_id(M, r, nrng)
            Rc = None
            Y = X
            if l < L:
                Rc = sla.block_diag(Rfac[l + 1][2 * i], Rfac[l + 1][2 * i + 1])
                Y = Rc @ X
            lam_w = None
            if mode == "spd":
                if l == L:
                    Lam = np.linalg.cholesky(D[i])
                else:
                    Sc = S[l + 1][i]
                    r1, r2 = Sc.shape[1], Sc.shape[0]
                    Lam = np.linalg.cholesky(np.block([[np.eye(r1), Sc.T], [Sc, np.eye(r2)]]))
                # least-squares fit of the scaled rows Λ⁻¹ (Rc) M on M[sk]
                Ms = M if Rc is None else Rc @ M
                Ms = sla.solve_triangular(Lam, Ms, lower=True)
                Ysc = np.linalg.lstsq(M[sk].T, Ms.T, rcond=None)[0].T
                Wq, R = np.linalg.qr(Ysc)
                Q = Lam @ Wq
                lam_w = (Lam, Wq)
            else:
                Q, R = np.linalg.qr(Y)
            return cand[i][sk], X.shape[1], Q, R, lam_w

        res = _parallel_map(compress, range(nn))
        ranks[l] = np.array([x[1] for x in res], dtype=np.int64)
        skel[l] = [x[0] for x in res]
        Rfac[l] = [x[3] for x in res]
        if l == L:
            U = [x[2] for x in res]
        else:
            E[l] = [x[2] for x in res]
        S[l] = []
        if mode == "spd":
            newOm = []
            for i in range(nn):
                Lam, Wq = res[i][4]
                Om = sla.solve_triangular(Lam, Wq, lower=True, trans="T")
                if l < L:
                    k1 = Om_prev[2 * i].shape[1]
                    Om = np.concatenate([Om_prev[2 * i] @ Om[:k1], Om_prev[2 * i + 1] @ Om[k1:]])
                newOm.append(Om)
            Om_prev = newOm
            for k2 in range(nn // 2):
                c1, c2 = 2 * k2, 2 * k2 + 1
                a1, b1 = node_range(l, c1)
                a2, b2 = node_range(l, c2)
                acc = _projected_block(w, pts[a2:b2], pts[a1:b1], Om_prev[c1], device)
                S[l].append(clip_norm(Om_prev[c2].T @ acc))
        else:
            for k2 in range(nn // 2):
                c1, c2 = 2 * k2, 2 * k2 + 1
                Kss = kernel_block(w, pts[skel[l][c2]], pts[skel[l][c1]])
                S[l].append(Rfac[l][c2] @ Kss @ Rfac[l][c1].T)
        cand = [np.concatenate([skel[l][2 * p], skel[l][2 * p + 1]]) for p in range(nn // 2)]

    return HSSMatrix(levels=L, sizes=sizes, ranks=ranks, D=D, U=U, E=E, S=S,
                     perm=perm, points=pts, workload=w)


def kernel_matrix(w: Workload, pts: np.ndarray) -> np.ndarray:
    """Dense shifted kernel matrix on cluster-ordered points (small N only)."""
    A = kernel_block(w, pts, pts)
    A[np.diag_indices_from(A)] += w.shift
    return 0.5 * (A + A.T)


def random_hss(levels: int, leaf: int, rank: int, seed: int, *,
               shift: float = None, orthonormal: bool = True,
               fast_bound: bool = False) -> HSSMatrix:
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
        # (fast_bound: Frobenius norms, cheap upper bounds of the 2-norms)
        nrm = (lambda a: np.linalg.norm(a)) if fast_bound else (lambda a: np.linalg.norm(a, 2))
        nb = max(nrm(u) for u in U)
        bound = 0.0
        for l in range(L, 0, -1):
            bound += max(nrm(s) for s in S[l]) * nb * nb
            if l > 1:
                nb *= max(nrm(e) for e in E[l - 1])
        shift = 2.0 * bound + 1.0
    D = []
    for _ in range(2 ** L):
        G = rng.standard_normal((b, b)) / math.sqrt(b)
        D.append(G @ G.T + shift * np.eye(b))
    ranks = {l: np.full(2 ** l, r, dtype=np.int64) for l in range(1, L + 1)}
    return HSSMatrix(levels=L, sizes=np.full(2 ** L, b, dtype=np.int64), ranks=ranks,
                     D=D, U=U, E=E, S=S)


def random_hss_device(levels: int, leaf: int, rank: int, seed: int, device="cuda"):
    """Random-generator HSS matrix built on the GPU with torch, for shapes whose
    host construction is out of reach (N = 2^21, leaf 1024, rank 256: 25 GB of
    generators).  Returns (shape, D, U, E, S, shift): float64 device tensors in
    the packed column-major layout of hss_create (D 2^L blocks b x b, U 2^L
    blocks b x r, E levels 1 .. L-1 of 2^l blocks 2r x r, S levels 1 .. L of
    2^(l-1) blocks r x r).

    U and E have orthonormal columns (QR of Gaussian blocks), so every nested
    basis is orthonormal; S is Gaussian / sqrt(r) (2-norm about 2) and D_i =
    sym(G_i) / sqrt(2b) + shift I.  The off-diagonal part's norm is at most
    sum over levels of max ||S||_2 <= 2.5 L, so shift = 2 (2.5 L) + 3 keeps the
    matrix SPD with condition number about 3.  Seeded: the same (levels, leaf,
    rank, seed) gives the same matrix on any GPU of the same arithmetic."""
    import torch
    L, b, r = levels, leaf, rank
    g = torch.Generator(device=device)
    g.manual_seed(seed)
    f64 = torch.float64
    shift = 2.0 * 2.5 * L + 3.0

    def orthonormal(count, m, k):
        out = torch.empty((count, k, m), dtype=f64, device=device)   # column-major m x k
        for c0 in range(0, count, 256):
            c1 = min(count, c0 + 256)
            q, _ = torch.linalg.qr(torch.randn((c1 - c0, m, k), generator=g, dtype=f64,
                                               device=device))
            out[c0:c1] = q.transpose(1, 2)
        return out

    D = torch.empty((2 ** L, b, b), dtype=f64, device=device)
    for c0 in range(0, 2 ** L, 256):
        c1 = min(2 ** L, c0 + 256)
        G = torch.randn((c1 - c0, b, b), generator=g, dtype=f64, device=device)
        D[c0:c1] = (G + G.transpose(1, 2)) / (2.0 * math.sqrt(2.0 * b))
        D[c0:c1].diagonal(dim1=1, dim2=2).add_(shift)
        del G
    U = orthonormal(2 ** L, b, r)
    E = (torch.cat([orthonormal(2 ** l, 2 * r, r).reshape(-1) for l in range(1, L)])
         if L >= 2 else torch.zeros(1, dtype=f64, device=device))
    S = torch.cat([(torch.randn((2 ** (l - 1), r, r), generator=g, dtype=f64, device=device)
                    / math.sqrt(r)).reshape(-1) for l in range(1, L + 1)])
    return (b << L, b, r, L), D.reshape(-1), U.reshape(-1), E, S, shift


def rhs(n: int, nrhs: int, seed: int) -> np.ndarray:
    """N(0,1) right-hand sides, column-major n x nrhs as a Fortran-ordered array."""
    rng = np.random.default_rng(seed)
    return np.asfortranarray(rng.standard_normal((n, nrhs)))


def cached_build(w: Workload, cache_dir: Optional[str], **kw) -> HSSMatrix:
    """build_hss(w), memoised in ``cache_dir`` (an .npz per workload and seed)
    so that repeated runs on one machine skip the generation."""
    if not cache_dir:
        return build_hss(w, **kw)
    import os
    os.makedirs(cache_dir, exist_ok=True)
    key = f"{w.name}_n{w.n}_l{w.leaf}_r{w.rank}_s{w.seed}_{kw.get('mode', 'spd')}.npz"
    path = os.path.join(cache_dir, key.replace("@", "_"))
    L = w.levels
    if os.path.exists(path[:-4] + ".pkl"):
        import pickle
        with open(path[:-4] + ".pkl", "rb") as f:
            return pickle.load(f)
    if os.path.exists(path):
        z = np.load(path)
        D = list(z["D"])
        U = list(z["U"])
        E = {l: list(z[f"E{l}"]) for l in range(1, L)}
        S = {l: list(z[f"S{l}"]) for l in range(1, L + 1)}
        ranks = {l: z[f"R{l}"] for l in range(1, L + 1)}
        return HSSMatrix(levels=L, sizes=z["sizes"], ranks=ranks, D=D, U=U, E=E, S=S,
                         perm=z["perm"], points=z["points"], workload=w)
    h = build_hss(w, **kw)
    if not h.uniform:   # uneven trees: pickled (blocks of different shapes)
        import pickle
        tmp = path + ".tmp.pkl"
        with open(tmp, "wb") as f:
            pickle.dump(h, f)
        os.replace(tmp, path[:-4] + ".pkl")
        return h
    if h.uniform:
        arrs = {"D": np.stack(h.D), "U": np.stack(h.U), "sizes": h.sizes, "perm": h.perm,
                "points": h.points}
        arrs.update({f"E{l}": np.stack(h.E[l]) for l in range(1, L)})
        arrs.update({f"S{l}": np.stack(h.S[l]) for l in range(1, L + 1)})
        arrs.update({f"R{l}": h.ranks[l] for l in range(1, L + 1)})
        tmp = path + ".tmp.npz"
        np.savez(tmp, **arrs)
        os.replace(tmp, path)
    return h


def batch_workloads(count: int, seed: int = 1003, n_min: int = 4096, n_max: int = 65536,
                    uniform: bool = False):
    """The batched uneven workload: `count` matrices, N log-uniform in
    [n_min, n_max] rounded to a multiple of the leaf size (the bisection tree has
    L = ceil(log2(N / leaf)) levels and leaf orders in (leaf/2, leaf]; it is
    uneven where 2^L does not divide N; with uniform=True N is rounded to
    leaf * 2^L instead), leaf drawn from {128, 256,
    512}, rank from {32, 64, 128}, kernel half 1/(d + 1e-3) on the unit cube
    (+ N^(1/3) I), half exp(-d / 0.1) on a jittered 2-D grid (+ 1e-4 I); one
    right-hand side each."""
    rng = np.random.default_rng(seed)
    out = []
    for i in range(count):
        leaf = int(rng.choice([128, 256, 512]))
        rank = int(rng.choice([32, 64, 128]))
        n_target = math.exp(rng.uniform(math.log(n_min), math.log(n_max)))
        if uniform:
            L = max(1, int(round(math.log2(n_target / leaf))))
            n = leaf * 2 ** L
        else:
            n = leaf * max(2, int(round(n_target / leaf)))
        if rng.random() < 0.5:
            w = Workload(f"batch{i}_cube_inv", n, leaf, rank, "cube", "inv", 0.0,
                         round(n ** (1.0 / 3.0), 6), 1, seed * 1000 + i)
        else:
            w = Workload(f"batch{i}_grid_exp", n, leaf, rank, "grid2d", "exp", 0.1, 1e-4, 1,
                         seed * 1000 + i)
        out.append(w)
    return out
