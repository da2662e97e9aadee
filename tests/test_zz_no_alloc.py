"""The allocation-free per-example gradient entry point.

Callers whose device memory belongs to another allocator (or who cannot
afford an allocation in their loop) get G without any cudaMalloc: the library
keeps its caches in a static device array.  These checks call that entry point
through the C ABI and compare it with the FP64 oracle and with the regular
per_example_grads, on two calls in a row, at the FP64 tolerance of the other
tests; they check that a call leaves the device's free memory unchanged, that
a request filling the static array to its last bytes is served correctly, and
that one example more is rejected.  The file name sorts last so that a run
stopping at its first failure has already run every other test.
"""

import ctypes

import numpy as np
import pytest

from oracle import mlp as O
from synth import make_problem

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

TOL = 1e-12
SCRATCH_BYTES = 32 << 20  # the static array's size, stated in the header


@pytest.fixture(scope="module")
def hm():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1905_05559_gb300 import build
    build.build()
    import paper_1905_05559_gb300 as hm
    return hm


def _desc(hm, widths, acts):
    from paper_1905_05559_gb300 import _lib
    w = (ctypes.c_int * len(widths))(*widths)
    a = (ctypes.c_int * max(1, len(acts)))(*([_lib.ACT[x] for x in acts] or [0]))
    return _lib.HessDesc(len(widths), w, a), (w, a)


def _relerr(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def _scratch_bytes(widths, N):
    """Bytes of cache the call plans for N examples: the header's per-example
    count, each array starting on a 256-byte boundary."""
    L = len(widths)
    sizes = []
    for j in range(1, L - 1):
        sizes += [N * widths[j]] * 4
    sizes += [N * widths[j] for j in range(1, L)]
    sizes += [N * widths[-1], N, N * max(widths)]
    off = 0
    for n in sizes:
        off = (off + 255) // 256 * 256 + 8 * n
    return off


def _call(hm, pb, N, X, Y, G, stream):
    lib = hm.load()
    desc, keep = _desc(hm, pb.widths, pb.acts)
    omega = torch.as_tensor(pb.omega, device="cuda")
    return lib.per_example_grads_noalloc(ctypes.byref(desc), omega.data_ptr(), X, Y, N, G, stream)


def _noalloc(hm, pb, stream):
    X = torch.as_tensor(pb.X, device="cuda")
    Y = torch.as_tensor(pb.Y, device="cuda")
    G = torch.full((pb.N, pb.P), float("nan"), dtype=torch.float64, device="cuda")
    st = _call(hm, pb, pb.N, X.data_ptr(), Y.data_ptr(), G.data_ptr(), stream)
    assert st == 0, hm.last_error()
    torch.cuda.current_stream().synchronize()
    return G.cpu().numpy()


def test_noalloc_matches_oracle_and_per_example_grads_two_calls_in_a_row(hm):
    stream = torch.cuda.current_stream().cuda_stream
    problems = [
        make_problem([37, 9, 5], ["tanh"], 77, 3, "normal", "uniform"),
        make_problem([13, 11, 7, 3], ["sigmoid", "relu"], 50, 4, "normal", "uniform"),
    ]
    for pb in problems:  # two consecutive calls share (and overwrite) the static scratch
        G = _noalloc(hm, pb, stream)
        ref = O.per_example_grads(pb.omega, pb.widths, pb.acts, pb.X, pb.Y)
        net = hm.HessMLP(pb.widths, pb.acts, pb.omega)
        Gr = net.per_example_grads(torch.as_tensor(pb.X, device="cuda"),
                                   torch.as_tensor(pb.Y, device="cuda"), "fp64").cpu().numpy()
        assert np.isfinite(G).all()
        assert _relerr(G, ref) <= TOL
        assert _relerr(G, Gr) <= TOL


def test_noalloc_call_allocates_no_device_memory(hm):
    pb = make_problem([37, 9, 5], ["tanh"], 77, 3, "normal", "uniform")
    stream = torch.cuda.current_stream().cuda_stream
    X = torch.as_tensor(pb.X, device="cuda")
    Y = torch.as_tensor(pb.Y, device="cuda")
    G = torch.empty((pb.N, pb.P), dtype=torch.float64, device="cuda")
    omega = torch.as_tensor(pb.omega, device="cuda")
    lib = hm.load()
    desc, keep = _desc(hm, pb.widths, pb.acts)
    # warm-up: the first call under this context looks up the array's address
    assert lib.per_example_grads_noalloc(ctypes.byref(desc), omega.data_ptr(), X.data_ptr(), Y.data_ptr(),
                                         pb.N, G.data_ptr(), stream) == 0, hm.last_error()
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    alloc0 = torch.cuda.memory_allocated()
    for _ in range(3):
        assert lib.per_example_grads_noalloc(ctypes.byref(desc), omega.data_ptr(), X.data_ptr(),
                                             Y.data_ptr(), pb.N, G.data_ptr(), stream) == 0, hm.last_error()
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0
    assert torch.cuda.memory_allocated() == alloc0
    ref = O.per_example_grads(pb.omega, pb.widths, pb.acts, pb.X, pb.Y)
    assert _relerr(G.cpu().numpy(), ref) <= TOL


def test_noalloc_fills_the_array_to_its_limit(hm):
    widths, acts = [37, 9, 5], ["tanh"]
    # the largest N whose caches fit the 32 MiB array, and one more
    lo, hi = 1, 1 << 20
    while lo < hi:
        mid = (lo + hi + 1) // 2
        if _scratch_bytes(widths, mid) <= SCRATCH_BYTES:
            lo = mid
        else:
            hi = mid - 1
    Nmax = lo
    assert _scratch_bytes(widths, Nmax + 1) > SCRATCH_BYTES
    assert SCRATCH_BYTES - _scratch_bytes(widths, Nmax) < 4096  # the last cache ends near the array's end
    pb = make_problem(widths, acts, Nmax, 5, "normal", "uniform")
    stream = torch.cuda.current_stream().cuda_stream
    X = torch.as_tensor(pb.X, device="cuda")
    Y = torch.as_tensor(pb.Y, device="cuda")
    G = torch.full((pb.N, pb.P), float("nan"), dtype=torch.float64, device="cuda")
    for _ in range(2):
        st = _call(hm, pb, Nmax, X.data_ptr(), Y.data_ptr(), G.data_ptr(), stream)
        assert st == 0, hm.last_error()
        torch.cuda.synchronize()
        ref = O.per_example_grads(pb.omega, pb.widths, pb.acts, pb.X, pb.Y)
        Gh = G.cpu().numpy()
        assert np.isfinite(Gh).all()
        assert _relerr(Gh, ref) <= TOL
    # one example more crosses the limit: rejected before any work (the
    # buffers are long enough, so the size of the scratch is the only reason)
    X2 = torch.zeros((Nmax + 1, widths[0]), dtype=torch.float64, device="cuda")
    Y2 = torch.zeros((Nmax + 1, widths[-1]), dtype=torch.float64, device="cuda")
    G2 = torch.zeros((Nmax + 1, pb.P), dtype=torch.float64, device="cuda")
    st = _call(hm, pb, Nmax + 1, X2.data_ptr(), Y2.data_ptr(), G2.data_ptr(), stream)
    assert st == 1 and "scratch" in hm.last_error()


def test_noalloc_rejects_oversized_requests_and_host_pointers(hm):
    lib = hm.load()
    pb = make_problem([37, 9, 5], ["tanh"], 77, 3, "normal", "uniform")
    desc, keep = _desc(hm, pb.widths, pb.acts)
    omega = torch.as_tensor(pb.omega, device="cuda")
    X = torch.as_tensor(pb.X, device="cuda")
    Y = torch.as_tensor(pb.Y, device="cuda")
    G = torch.empty((pb.N, pb.P), dtype=torch.float64, device="cuda")
    # caches for N = 10^7 examples exceed the 32 MiB array: rejected up front
    st = lib.per_example_grads_noalloc(ctypes.byref(desc), omega.data_ptr(), X.data_ptr(),
                                       Y.data_ptr(), 10_000_000, G.data_ptr(), None)
    assert st == 1 and "scratch" in hm.last_error()
    Xh = np.ascontiguousarray(pb.X)
    st = lib.per_example_grads_noalloc(ctypes.byref(desc), omega.data_ptr(), Xh.ctypes.data,
                                       Y.data_ptr(), pb.N, G.data_ptr(), None)
    assert st == 1 and "device memory" in hm.last_error()
