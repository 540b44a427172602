"""The allocation-free pair-force entry point against the allocating one.

nbody_pair_accel_noalloc serves callers that cannot allocate device memory
when they need forces (a fixed up-front memory budget, or a loop that must
not touch the allocator); it keeps its scratch in one fixed device array of
the library.  This file is collected last so that a run stopping at the
first failure has already run every other test; it also passes alone in a
fresh process (it builds and loads the library itself).
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import core as orc  # noqa: E402
from paper_2511_22468_gb300 import nbody as nb  # noqa: E402
from paper_2511_22468_gb300.inputs import plummer_sphere  # noqa: E402

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2511_22468_gb300 import build
    build.build()
    nb.lib()


def _rel_err(a, ref):
    # per-particle |a - ref| / (|ref| + 1e-3 rms|ref|), the suite's
    # acceleration tolerance measure
    a, ref = a.T, ref.T
    scale = np.linalg.norm(ref, axis=1) + 1e-3 * np.sqrt(np.mean(np.sum(ref * ref, axis=1)))
    return np.max(np.linalg.norm(a - ref, axis=1) / scale)


def test_noalloc_matches_allocating_entry_point_twice():
    dev = torch.device("cuda:0")
    # two calls in a row, the second smaller than the first: the shared
    # array keeps the first call's contents, which must not leak through
    for n, seed in ((nb.NBODY_NOALLOC_MAX_N, 3), (3001, 4)):
        x, v, m = plummer_sphere(n, seed, 1.0, 1.0, 1.0)
        m = m * np.linspace(0.5, 1.5, n)
        X = torch.tensor(x.T.copy(), device=dev)
        M = torch.tensor(m, device=dev)
        ref = torch.empty((3, n), dtype=torch.float64, device=dev)
        got = torch.full((3, n), float("nan"), dtype=torch.float64, device=dev)
        nb.nbody_pair_accel(X, M, 1.0, 0.01, (0.1, -0.2, 0.05), ref)
        nb.nbody_pair_accel_noalloc(X, M, 1.0, 0.01, (0.1, -0.2, 0.05), got)
        torch.cuda.synchronize()
        assert _rel_err(got.cpu().numpy(), ref.cpu().numpy()) <= 1e-5


def test_noalloc_matches_oracle_direct_sum():
    """A small, uneven n with unequal masses and a non-zero recentring origin
    against the oracle's FP64 direct sum (not only against the allocating
    entry point, which runs the same kernels), twice in a row.  The centre is
    a host buffer that is overwritten right after each call returns, before
    the stream has run: the call reads it by value."""
    import ctypes as C
    dev = torch.device("cuda:0")
    n = 1001
    x, v, m = plummer_sphere(n, 11, 1.0, 1.0, 1.0, center=(0.3, -0.1, 0.2))
    m = m * np.random.default_rng(12).uniform(0.5, 1.5, n)
    X = torch.tensor(x.T.copy(), device=dev)
    M = torch.tensor(m, device=dev)
    ref = orc.pair_accel(x, m, 1.0, 0.01)
    stream = torch.cuda.current_stream().cuda_stream
    for _ in range(2):
        got = torch.full((3, n), float("nan"), dtype=torch.float64, device=dev)
        cen = (C.c_double * 3)(0.3, -0.1, 0.2)
        rc = nb.lib().nbody_pair_accel_noalloc(n, C.c_void_p(X.data_ptr()),
                                               C.c_void_p(M.data_ptr()), 1.0, 0.01, cen,
                                               C.c_void_p(got.data_ptr()), C.c_void_p(stream))
        cen[0], cen[1], cen[2] = 5.0, 7.0, -9.0
        assert rc == nb.NBODY_OK
        torch.cuda.synchronize()
        assert _rel_err(got.cpu().numpy(), ref.T) <= 1e-5


def test_noalloc_rejects_sizes_beyond_its_buffer():
    dev = torch.device("cuda:0")
    n = nb.NBODY_NOALLOC_MAX_N + 1
    X = torch.zeros((3, n), dtype=torch.float64, device=dev)
    M = torch.ones(n, dtype=torch.float64, device=dev)
    out = torch.empty_like(X)
    with pytest.raises(nb.NBodyError) as e:
        nb.nbody_pair_accel_noalloc(X, M, 1.0, 0.01, (0, 0, 0), out)
    assert e.value.code == nb.NBODY_ESIZE
