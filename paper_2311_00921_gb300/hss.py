"""Python binding of the C ABI in include/hss.h (ctypes; argument marshalling only).

Device memory, streams and vectors are PyTorch tensors; every step of the
factorization, solve and matvec runs in the CUDA library.  There is no CPU
fallback: if the library is missing, loading it raises.
"""
from __future__ import annotations

import ctypes
import os
from typing import Optional

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "_lib", "libhss_gb300.so")

HSS_FP64, HSS_MIXED_TF32, HSS_MIXED_BF16, HSS_MIXED_FP32 = 0, 1, 2, 3
PRECISIONS = {"fp64": HSS_FP64, "tf32": HSS_MIXED_TF32, "bf16": HSS_MIXED_BF16,
              "fp32": HSS_MIXED_FP32}
ERRORS = {0: "OK", -1: "INVALID_ARG", -2: "NOT_FACTORIZED", -3: "NOT_SPD", -4: "CUDA",
          -5: "OOM", -6: "TIMEOUT", -7: "NO_CONVERGENCE", -8: "TOO_LARGE"}

# every entry point declared in include/hss.h: name -> (restype, argtypes)
_c_int, _c_double, _p = ctypes.c_int, ctypes.c_double, ctypes.c_void_p


class Shape(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int32), ("leaf", ctypes.c_int32), ("rank", ctypes.c_int32),
                ("levels", ctypes.c_int32), ("node_sizes", ctypes.POINTER(ctypes.c_int32))]


class Options(ctypes.Structure):
    _fields_ = [("precision", ctypes.c_int32), ("ir_max_it", ctypes.c_int32),
                ("ir_tol", ctypes.c_double), ("residual", ctypes.c_int32),
                ("basis", ctypes.c_int32), ("wait_budget", ctypes.c_int64),
                ("schedule", ctypes.c_int32), ("ql_panel", ctypes.c_int32),
                ("ir_lanes", ctypes.c_int32), ("reserved", ctypes.c_int32)]


RESIDUALS = {"fp64": 0, "pair32": 1}
BASIS_METHODS = {"householder": 0, "cholqr": 1, "auto": 2}
SCHEDULES = {"async": 0, "levels": 1, "auto": 2}


class Tuning(ctypes.Structure):
    _fields_ = [("basis", ctypes.c_int32), ("schedule", ctypes.c_int32),
                ("staging", ctypes.c_int32), ("from_cache", ctypes.c_int32),
                ("factor_ms", ctypes.c_double), ("solve_ms", ctypes.c_double),
                ("factor_ms_by_basis", ctypes.c_double * 2),
                ("solve_ms_by_config", (ctypes.c_double * 2) * 2),
                ("ql_panel", ctypes.c_int32), ("ir_lanes", ctypes.c_int32),
                ("factor_ms_by_panel", ctypes.c_double * 2),
                ("solve_ms_by_lanes", ctypes.c_double * 2)]


_i32p = ctypes.POINTER(ctypes.c_int32)
SIGNATURES = {
    "hss_create": (_c_int, [ctypes.POINTER(Shape), _p, _p, _p, _p, _c_int, ctypes.POINTER(_p)]),
    "hss_factorize": (_c_int, [_p, ctypes.POINTER(Options), _p]),
    "hss_solve": (_c_int, [_p, _p, _p, ctypes.c_int32, ctypes.c_int32, _p]),
    "hss_logdet": (_c_int, [_p, ctypes.POINTER(_c_double)]),
    "hss_matvec": (_c_int, [_p, _p, _p, ctypes.c_int32, ctypes.c_int32, _p]),
    "hss_matvec_pair": (_c_int, [_p, _p, _p, ctypes.c_int32, ctypes.c_int32, _p]),
    "hss_sync": (_c_int, [_p]),
    "hss_tune": (_c_int, [_p, ctypes.POINTER(Options), ctypes.c_int32, ctypes.c_char_p, _p,
                          ctypes.POINTER(Tuning)]),
    "hss_last_info": (_c_int, [_p, _i32p, _i32p, _i32p, _i32p, ctypes.POINTER(_c_double)]),
    "hss_export": (_c_int, [_p, ctypes.c_int32, ctypes.c_int32, _p, ctypes.c_size_t]),
    "hss_trace": (_c_int, [_p, ctypes.c_int32]),
    "hss_trace_read": (_c_int, [_p, ctypes.c_int32, ctypes.POINTER(_c_double),
                                ctypes.POINTER(ctypes.c_int64), ctypes.POINTER(_c_double)]),
    "hss_launch_count": (_c_int, [_p, ctypes.POINTER(ctypes.c_int64)]),
    "hss_matvec_noalloc": (_c_int, [ctypes.POINTER(Shape), _p, _p, _p, _p, _p, _p, ctypes.c_int32,
                                    ctypes.c_int32, _p]),
    "hss_destroy": (None, [_p]),
    "hss_batch_create": (_c_int, [ctypes.c_int32, ctypes.POINTER(Shape), ctypes.POINTER(_p),
                                  ctypes.POINTER(_p), ctypes.POINTER(_p), ctypes.POINTER(_p),
                                  ctypes.POINTER(_p)]),
    "hss_batch_factorize": (_c_int, [_p, ctypes.POINTER(Options), _p]),
    "hss_batch_solve": (_c_int, [_p, ctypes.POINTER(_p), ctypes.POINTER(_p), ctypes.c_int32, _p]),
    "hss_batch_logdet": (_c_int, [_p, ctypes.POINTER(_c_double)]),
    "hss_batch_destroy": (None, [_p]),
    "hss_batch_set_graph": (_c_int, [_p, ctypes.c_int32]),
    "hss_strerror": (ctypes.c_char_p, [_c_int]),
}

_lib = None


def load():
    """Load the CUDA library (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"HSS CUDA library not built ({LIB_PATH}); run "
                               "`python -c 'import __graft_entry__ as g; g.build()'`")
        lib = ctypes.CDLL(LIB_PATH)
        for name, (res, args) in SIGNATURES.items():
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        _lib = lib
    return _lib


class HSSError(RuntimeError):
    def __init__(self, code: int, where: str):
        self.code = code
        super().__init__(f"{where}: {ERRORS.get(code, code)} ({load().hss_strerror(code).decode()})")


def _check(code: int, where: str):
    if code != 0:
        raise HSSError(code, where)


def _colmajor_blocks(blocks) -> np.ndarray:
    """Stack 2-D blocks into one buffer with each block column-major."""
    arr = np.stack([np.asarray(b, dtype=np.float64) for b in blocks])
    return np.ascontiguousarray(arr.transpose(0, 2, 1))


def _stream_ptr(stream) -> int:
    import torch
    s = stream if stream is not None else torch.cuda.current_stream()
    return int(s.cuda_stream)


def _mat_args(t):
    """(pointer, nrhs, ld) of an n x nrhs column-major float64 CUDA tensor or a vector."""
    import torch
    if t.dtype != torch.float64 or not t.is_cuda:
        raise TypeError("expected a float64 CUDA tensor")
    if t.dim() == 1:
        if t.stride(0) != 1:
            raise ValueError("vector must be contiguous")
        return t.data_ptr(), 1, t.shape[0]
    if t.dim() != 2 or t.stride(0) != 1:
        raise ValueError("matrix must be column-major (stride(0) == 1); use colmajor()")
    return t.data_ptr(), t.shape[1], max(t.stride(1), t.shape[0])


def colmajor(x, device="cuda"):
    """A column-major float64 CUDA copy of a host array / tensor (n x k or n)."""
    import torch
    t = torch.as_tensor(np.asarray(x) if not isinstance(x, torch.Tensor) else x)
    t = t.to(dtype=torch.float64)
    if t.dim() == 1:
        return t.contiguous().to(device)
    return t.t().contiguous().to(device).t()


def uneven_shape(h):
    """(shape, D, U, E, S, sizes) of a non-uniform tree for hss_create: node_sizes =
    the leaf orders, leaf = the largest of them (at least the rank), rank = the
    largest rank, generators
    packed block after block (each column-major).  The ranks must follow
    r_i = min(rank, b_i) at the leaves and min(rank, r_c1 + r_c2) above."""
    L = h.levels
    sizes = np.asarray(h.sizes, dtype=np.int32)
    rank = int(max(int(np.max(v)) for v in h.ranks.values()))
    rk = {L: np.minimum(rank, sizes)}
    for l in range(L - 1, 0, -1):
        rk[l] = np.minimum(rank, rk[l + 1][0::2] + rk[l + 1][1::2])
    for l in range(1, L + 1):
        if not np.array_equal(np.asarray(h.ranks[l]), rk[l]):
            raise ValueError("ranks do not follow min(rank, order) of an uneven tree")
    flat = lambda blocks: np.concatenate([np.asarray(b, dtype=np.float64).T.ravel()
                                          for b in blocks])
    D, U = flat(h.D), flat(h.U)
    E = (np.concatenate([flat(h.E[l]) for l in range(1, L)]) if L >= 2 else np.zeros(1))
    S = np.concatenate([flat(h.S[l]) for l in range(1, L + 1)])
    keep = np.ascontiguousarray(sizes)
    # the padded leaf order holds the largest leaf and the rank's basis columns
    shape = Shape(h.n, int(max(sizes.max(), rank)), rank, L,
                  keep.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)))
    return shape, D, U, E, S, keep


class HSS:
    """A device-resident HSS matrix (generators copied at construction); uniform
    or uneven trees (the library embeds an uneven one in the uniform format)."""

    def __init__(self, h):
        lib = load()
        L = h.levels
        if h.uniform:
            r, leaf = h.rank, h.leaf
            D = _colmajor_blocks(h.D)
            U = _colmajor_blocks(h.U)
            E = (np.concatenate([_colmajor_blocks(h.E[l]).ravel() for l in range(1, L)])
                 if L >= 2 else np.zeros(1))
            S = np.concatenate([_colmajor_blocks(h.S[l]).ravel() for l in range(1, L + 1)])
            shape = Shape(h.n, leaf, r, L)
        else:
            shape, D, U, E, S, _keep = uneven_shape(h)
            r, leaf = shape.rank, shape.leaf
        self.n, self.levels, self.rank, self.leaf = h.n, L, r, leaf
        out = _p()
        _check(lib.hss_create(ctypes.byref(shape), D.ctypes.data, U.ctypes.data, E.ctypes.data,
                              S.ctypes.data, 0, ctypes.byref(out)), "hss_create")
        self._h = out
        self.precision = None

    @classmethod
    def from_device(cls, shape, D, U, E, S):
        """An HSS object from generators already in device memory: shape = (n,
        leaf, rank, levels) of a uniform tree, D, U, E, S float64 CUDA tensors in
        the packed layout of hss_create (copied device to device)."""
        self = cls.__new__(cls)
        n, leaf, r, L = shape
        sh = Shape(n, leaf, r, L)
        out = _p()
        _check(load().hss_create(ctypes.byref(sh), D.data_ptr(), U.data_ptr(), E.data_ptr(),
                                 S.data_ptr(), 1, ctypes.byref(out)), "hss_create")
        self._h = out
        self.n, self.levels, self.rank, self.leaf = n, L, r, leaf
        self.precision = None
        return self

    def close(self):
        if getattr(self, "_h", None):
            load().hss_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def factorize(self, precision="fp64", ir_tol=1e-12, ir_max_it=30, residual="fp64",
                  stream=None, wait_budget=0, basis="householder", schedule="async",
                  ql_panel=0, ir_lanes=0):
        """residual: arithmetic of the refinement residual of the mixed modes,
        "fp64" or "pair32" (pairs of FP32 numbers, 48-bit significands).
        wait_budget: polls of a device-side pipeline wait (0 = default, < 0 =
        give up at once).  basis: "householder" or "cholqr" (Cholesky QR +
        Householder reconstruction; the method of the basis completion), or
        "auto" (the tuner's).  schedule: "async" (upper solve levels as one launch
        per direction), "levels" or "auto".  ql_panel: 16 or 32 columns per
        register panel of the Householder kernel in FP32 (0 = default).
        ir_lanes: refinement lanes of a mixed solve, 1 or 2 (0 = the tuner's
        choice under schedule="auto", else 1)."""
        opt = Options(PRECISIONS[precision], ir_max_it, ir_tol, RESIDUALS[residual],
                      BASIS_METHODS[basis], wait_budget, SCHEDULES[schedule], ql_panel,
                      ir_lanes, 0)
        _check(load().hss_factorize(self._h, ctypes.byref(opt), _stream_ptr(stream)),
               "hss_factorize")
        self.precision = precision

    def solve(self, b, x=None, stream=None):
        """x = A⁻¹ b for column-major float64 CUDA tensors (x defaults to a new tensor)."""
        import torch
        if x is None:
            x = torch.empty_like(b) if b.dim() == 1 else torch.empty(
                (b.shape[1], b.shape[0]), dtype=b.dtype, device=b.device).t()
        bp, nrhs, ld = _mat_args(b)
        xp, nrhs2, ld2 = _mat_args(x)
        if nrhs != nrhs2 or ld != ld2:
            raise ValueError("b and x need the same shape and leading dimension")
        _check(load().hss_solve(self._h, bp, xp, nrhs, ld, _stream_ptr(stream)), "hss_solve")
        return x

    def matvec(self, x, y=None, stream=None):
        import torch
        if y is None:
            y = torch.empty_like(x) if x.dim() == 1 else torch.empty(
                (x.shape[1], x.shape[0]), dtype=x.dtype, device=x.device).t()
        xp, nrhs, ld = _mat_args(x)
        yp, nrhs2, ld2 = _mat_args(y)
        if nrhs != nrhs2 or ld != ld2:
            raise ValueError("x and y need the same shape and leading dimension")
        _check(load().hss_matvec(self._h, xp, yp, nrhs, ld, _stream_ptr(stream)), "hss_matvec")
        return y

    def matvec_pair(self, x, y=None, stream=None):
        """y = A x in pair-of-FP32 arithmetic (hss_matvec_pair)."""
        import torch
        if y is None:
            y = torch.empty_like(x) if x.dim() == 1 else torch.empty(
                (x.shape[1], x.shape[0]), dtype=x.dtype, device=x.device).t()
        xp, nrhs, ld = _mat_args(x)
        yp, nrhs2, ld2 = _mat_args(y)
        if nrhs != nrhs2 or ld != ld2:
            raise ValueError("x and y need the same shape and leading dimension")
        _check(load().hss_matvec_pair(self._h, xp, yp, nrhs, ld, _stream_ptr(stream)),
               "hss_matvec_pair")
        return y

    def logdet(self) -> float:
        out = ctypes.c_double()
        _check(load().hss_logdet(self._h, ctypes.byref(out)), "hss_logdet")
        return out.value

    def sync(self):
        _check(load().hss_sync(self._h), "hss_sync")

    def tune(self, precision="fp64", nrhs=16, residual="fp64", cache=None, stream=None):
        """hss_tune: measure the candidate basis methods, solve schedules and sweep
        stagings on this object and keep the fastest (used by factorize(...,
        basis="auto", schedule="auto")).  Returns the choices as a dict."""
        opt = Options(PRECISIONS[precision], 30, 1e-12, RESIDUALS[residual], 0, 0, 0, 0)
        t = Tuning()
        _check(load().hss_tune(self._h, ctypes.byref(opt), nrhs,
                               cache.encode() if cache else None, _stream_ptr(stream),
                               ctypes.byref(t)), "hss_tune")
        self.precision = precision
        names_b = {v: k for k, v in BASIS_METHODS.items()}
        names_s = {v: k for k, v in SCHEDULES.items()}
        return {"basis": names_b[t.basis], "ql_panel": t.ql_panel,
                "schedule": names_s[t.schedule], "ir_lanes": t.ir_lanes,
                "staging": "fewest_waves" if t.staging else "largest_panels",
                "from_cache": bool(t.from_cache), "factor_ms": t.factor_ms,
                "solve_ms": t.solve_ms,
                "measured": None if t.from_cache else {
                    "factor_ms": {names_b[k]: t.factor_ms_by_basis[k] for k in range(2)
                                  if t.factor_ms_by_basis[k] > 0},
                    "factor_ms_householder_panel": {
                        f"{16 << k}": t.factor_ms_by_panel[k] for k in range(2)
                        if t.factor_ms_by_panel[k] > 0},
                    "solve_ms_by_lanes": {f"{k + 1}": t.solve_ms_by_lanes[k] for k in range(2)
                                          if t.solve_ms_by_lanes[k] > 0},
                    "solve_ms": {f"{names_s[s]}/{'fewest_waves' if g else 'largest_panels'}":
                                 t.solve_ms_by_config[s][g] for s in range(2) for g in range(2)
                                 if t.solve_ms_by_config[s][g] > 0}}}

    def last_info(self):
        lvl, node, col, it = (ctypes.c_int32() for _ in range(4))
        res = ctypes.c_double()
        code = load().hss_last_info(self._h, ctypes.byref(lvl), ctypes.byref(node),
                                    ctypes.byref(col), ctypes.byref(it), ctypes.byref(res))
        return {"code": code, "level": lvl.value, "node": node.value, "col": col.value,
                "ir_iters": it.value, "ir_resid": res.value}

    KERNELS = ("ql", "gemm", "gemm_skinny", "syr2k", "pchol", "trsv_fwd", "trsv_bwd", "other",
               "tc_gemm", "tc_syr2k", "pair_gemm", "basis_gemm", "basis_node")

    def trace(self, enable: bool, serialize: bool = False):
        """Per-launch event timing on/off; serialize also runs the basis chain on
        the caller's stream so that each logged time is the kernel's own."""
        mode = (2 if serialize else 1) if enable else 0
        _check(load().hss_trace(self._h, mode), "hss_trace")

    def trace_read(self):
        """{"kernel.f64" / "kernel.f32": (ms, launches, algorithmic flops)} of the
        logged launches (classes with no launch are left out)."""
        out = {}
        for prec, off in (("f64", 0), ("f32", len(self.KERNELS))):
            for k, name in enumerate(self.KERNELS):
                ms, n, fl = ctypes.c_double(), ctypes.c_int64(), ctypes.c_double()
                _check(load().hss_trace_read(self._h, k + off, ctypes.byref(ms), ctypes.byref(n),
                                             ctypes.byref(fl)), "hss_trace_read")
                if n.value:
                    out[f"{name}.{prec}"] = (ms.value, n.value, fl.value)
        return out

    def launch_count(self) -> int:
        v = ctypes.c_int64()
        _check(load().hss_launch_count(self._h, ctypes.byref(v)), "hss_launch_count")
        return v.value

    def export(self, what: str, level: int) -> np.ndarray:
        """Per-level factor arrays as (nodes, rows, cols) host arrays."""
        kinds = {"V": 0, "T": 1, "LB": 2, "M": 3, "B": 4}
        nodes = 2 ** level
        b = self.leaf if level == self.levels else 2 * self.rank
        r = self.rank
        rows, cols = {"V": (b, r), "T": (r, r), "LB": (r, r), "M": (b, b), "B": (b, r)}[what]
        buf = np.empty(nodes * rows * cols)
        _check(load().hss_export(self._h, kinds[what], level, buf.ctypes.data, buf.size),
               "hss_export")
        return buf.reshape(nodes, cols, rows).transpose(0, 2, 1).copy()


def packed_generators(h):
    """(D, U, E, S) of an HSS matrix as flat float64 host arrays in the packed
    column-major layout of hss_create."""
    L = h.levels
    D = _colmajor_blocks(h.D).ravel()
    U = _colmajor_blocks(h.U).ravel()
    E = (np.concatenate([_colmajor_blocks(h.E[l]).ravel() for l in range(1, L)])
         if L >= 2 else np.zeros(1))
    S = np.concatenate([_colmajor_blocks(h.S[l]).ravel() for l in range(1, L + 1)])
    return D, U, E, S


def matvec_noalloc(shape, D, U, E, S, x, y, stream=None):
    """y = A x through hss_matvec_noalloc.  D, U, E, S, x, y are CUDA tensors the
    caller owns (packed layout, see packed_generators); nothing is allocated."""
    xp, nrhs, ld = _mat_args(x)
    yp, nrhs2, ld2 = _mat_args(y)
    if nrhs != nrhs2 or ld != ld2:
        raise ValueError("x and y need the same shape and leading dimension")
    sh = Shape(*shape)
    _check(load().hss_matvec_noalloc(ctypes.byref(sh), D.data_ptr(), U.data_ptr(), E.data_ptr(),
                                     S.data_ptr(), xp, yp, nrhs, ld, _stream_ptr(stream)),
           "hss_matvec_noalloc")
    return y


class HSSBatch:
    """Many device-resident HSS matrices of uneven shapes, factored and solved
    together (hss_batch_*); members may be uniform or uneven trees."""

    def __init__(self, mats):
        lib = load()
        self.count = len(mats)
        self.n = [h.n for h in mats]
        shp, self._keep = [], []
        for h in mats:
            if h.uniform:
                shp.append(Shape(h.n, h.leaf, h.rank, h.levels))
                self._keep.append(packed_generators(h))
            else:
                s, D, U, E, S, sizes = uneven_shape(h)
                shp.append(s)
                self._keep.append((D, U, E, S, sizes))
        shapes = (Shape * self.count)(*shp)
        arr = lambda k: (_p * self.count)(*[a[k].ctypes.data for a in self._keep])
        out = _p()
        _check(lib.hss_batch_create(self.count, shapes, arr(0), arr(1), arr(2), arr(3),
                                    ctypes.byref(out)), "hss_batch_create")
        self._h = out
        self._keep = None

    def close(self):
        if getattr(self, "_h", None):
            load().hss_batch_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def factorize(self, stream=None):
        opt = Options(HSS_FP64, 0, 0.0, 0, 0, 0)
        _check(load().hss_batch_factorize(self._h, ctypes.byref(opt), _stream_ptr(stream)),
               "hss_batch_factorize")

    def use_graph(self, enable=True):
        _check(load().hss_batch_set_graph(self._h, 1 if enable else 0), "hss_batch_set_graph")

    def solve(self, bs, xs=None, stream=None):
        """bs: list of column-major float64 CUDA tensors (n_i x nrhs, ld = n_i)."""
        import torch
        if xs is None:
            xs = [torch.empty((b.shape[1], b.shape[0]), dtype=b.dtype, device=b.device).t()
                  for b in bs]
        nrhs = bs[0].shape[1]
        for b, x, n in zip(bs, xs, self.n):
            if b.shape != (n, nrhs) or x.shape != (n, nrhs) or b.stride(0) != 1 or x.stride(0) != 1:
                raise ValueError("each b_i, x_i must be n_i x nrhs column-major")
        bp = (_p * self.count)(*[b.data_ptr() for b in bs])
        xp = (_p * self.count)(*[x.data_ptr() for x in xs])
        _check(load().hss_batch_solve(self._h, bp, xp, nrhs, _stream_ptr(stream)),
               "hss_batch_solve")
        return xs

    def logdet(self):
        out = (ctypes.c_double * self.count)()
        _check(load().hss_batch_logdet(self._h, out), "hss_batch_logdet")
        return np.array(out[:])
