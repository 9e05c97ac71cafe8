"""hss_matvec_noalloc, the matvec entry point for callers that cannot allocate
device memory when they call the library (their device memory is reserved up
front by a host pool, or a cudaMalloc is not allowed in their loop).  It keeps
its per-level vectors in a fixed static device array instead of a workspace.

Checked here through the C ABI against the allocating hss_matvec and against
the oracle's HSS matvec, on two calls in a row (the static array is shared and
keeps the previous call's contents), with the tolerance of the other matvec
tests; and the size limit.  This file is collected last so that a failure here
comes after every other test has run.
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


def rel_err(a, b):
    return np.abs(a - b).max() / np.abs(b).max()


def on_device(arrays):
    return [torch.as_tensor(a).cuda() for a in arrays]


@pytest.mark.parametrize("levels,leaf,rank,nrhs", [
    (4, 80, 24, 35),     # 32 columns per pass: two passes, ragged second
    (9, 128, 128, 12),   # 8 columns per pass fit the static array: two passes
    (1, 96, 20, 3),      # one level: no transfer matrices, E unused
])
def test_noalloc_matvec_matches_allocating_matvec_twice(levels, leaf, rank, nrhs):
    h = I.random_hss(levels, leaf, rank, seed=levels + rank, orthonormal=False)
    obj = hss.HSS(h)
    D, U, E, S = on_device(hss.packed_generators(h))
    shape = (h.n, leaf, rank, levels)
    for call in range(2):
        x = hss.colmajor(I.rhs(h.n, nrhs, 100 + call))
        y_ref = obj.matvec(x).cpu().numpy()
        y = torch.full((nrhs, h.n), float("nan"), dtype=torch.float64, device="cuda").t()
        hss.matvec_noalloc(shape, D, U, E, S, x, y)
        torch.cuda.synchronize()
        y = y.cpu().numpy()
        assert rel_err(y, y_ref) <= 1e-13, f"call {call}"
        assert rel_err(y, O.matvec(h, x.cpu().numpy()).reshape(y.shape)) <= 1e-13, f"call {call}"


def test_noalloc_rejects_problems_beyond_its_scratch():
    # one column needs 2 (2^(L+1) - 2) rank doubles of the 2^21-double array;
    # L = 12, rank = 256 needs about twice that, so the call must be refused
    # before any device work (the pointers below are never dereferenced)
    levels, leaf, rank = 12, 1024, 256
    assert 2 * (2 ** (levels + 1) - 2) * rank > 2 ** 21
    lib = hss.load()
    shape = hss.Shape(leaf * 2 ** levels, leaf, rank, levels)
    dummy = torch.zeros(8, dtype=torch.float64, device="cuda")
    p = dummy.data_ptr()
    rc = lib.hss_matvec_noalloc(shape, p, p, p, p, p, p + 32, 1, shape.n, None)
    assert rc == -8
    assert lib.hss_strerror(rc).startswith(b"problem exceeds the fixed scratch")
