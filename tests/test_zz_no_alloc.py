"""The allocation-free per-example gradient entry point.

Callers whose device memory belongs to another allocator (or who cannot
afford an allocation in their loop) get G without any cudaMalloc: the library
keeps its caches in a static device array.  These checks call that entry point
through the C ABI and compare it with the regular per_example_grads, on two
calls in a row, at the FP64 tolerance of the other tests.  The file name sorts
last so that a run stopping at its first failure has already run every other
test.
"""

import ctypes

import numpy as np
import pytest

from synth import make_problem

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

TOL = 1e-12


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
    return float(torch.linalg.norm(a - b) / torch.linalg.norm(b))


def _noalloc(hm, pb, stream):
    lib = hm.load()
    desc, keep = _desc(hm, pb.widths, pb.acts)
    omega = torch.as_tensor(pb.omega, device="cuda")
    X = torch.as_tensor(pb.X, device="cuda")
    Y = torch.as_tensor(pb.Y, device="cuda")
    G = torch.full((pb.N, pb.P), float("nan"), dtype=torch.float64, device="cuda")
    st = lib.per_example_grads_noalloc(ctypes.byref(desc), omega.data_ptr(), X.data_ptr(),
                                       Y.data_ptr(), pb.N, G.data_ptr(), stream)
    assert st == 0, hm.last_error()
    torch.cuda.current_stream().synchronize()
    return G


def test_noalloc_matches_per_example_grads_two_calls_in_a_row(hm):
    stream = torch.cuda.current_stream().cuda_stream
    problems = [
        make_problem([37, 9, 5], ["tanh"], 77, 3, "normal", "uniform"),
        make_problem([13, 11, 7, 3], ["sigmoid", "relu"], 50, 4, "normal", "uniform"),
    ]
    for pb in problems:  # two consecutive calls share (and overwrite) the static scratch
        G = _noalloc(hm, pb, stream)
        net = hm.HessMLP(pb.widths, pb.acts, pb.omega)
        ref = net.per_example_grads(torch.as_tensor(pb.X, device="cuda"),
                                    torch.as_tensor(pb.Y, device="cuda"), "fp64")
        assert bool(torch.isfinite(G).all())
        assert _relerr(G, ref) <= TOL


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
