"""Top-k OPG eigenpairs in O(k P) memory (opg_topk_eig_lowmem) against the
oracle.

The route never forms G, the Gram matrix or the OPG: passes over the examples
in chunks apply OPG to blocks of vectors (Sec. 5.4, Eq. J; Sec. 6's O(K P)
memory), and a block Krylov method with thick restarts extracts the
eigenpairs.  Checked against the oracle's eigenpairs of the same data with the
bars of the other eigen tests (FP64: eigenvalues 1e-10 of the largest,
separated eigenvectors by |q . q_ref|, every residual of the OPG
eigen-equation 1e-8 of the largest; FP32 products: eigenvalues 1e-5), with
ragged chunks, one example per chunk, a P small enough for one block, host
buffers, a rank-deficient data set and argument errors.
"""

import ctypes

import numpy as np
import pytest

from eigcheck import check_eig
from oracle import mlp as O
from synth import make_problem, named_config

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def hm():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1905_05559_gb300 import build
    build.build()
    import paper_1905_05559_gb300 as hm
    return hm


def lowmem(hm, net, X, Y, N, k, prec, chunk, block=0, allow=()):
    from paper_1905_05559_gb300 import _lib
    lib = hm.load()
    dev = isinstance(X, torch.Tensor)
    if dev:
        ev = torch.empty(k, dtype=torch.float64, device="cuda")
        Q = torch.empty((k, net.P), dtype=torch.float64, device="cuda")
        ptrs = (X.data_ptr(), Y.data_ptr(), ev.data_ptr(), Q.data_ptr())
    else:
        ev = np.empty(k)
        Q = np.empty((k, net.P))
        ptrs = (X.ctypes.data, Y.ctypes.data, ev.ctypes.data, Q.ctypes.data)
    passes = ctypes.c_int()
    st = lib.opg_topk_eig_lowmem(net.h, ctypes.c_void_p(ptrs[0]), ctypes.c_void_p(ptrs[1]), N, k,
                                 _lib.PRECISION[prec], chunk, block, ctypes.c_void_p(ptrs[2]),
                                 ctypes.c_void_p(ptrs[3]), ctypes.byref(passes))
    if st not in (0,) + tuple(allow):
        raise hm.HessError(st, hm.last_error())
    if dev:
        torch.cuda.synchronize()
        ev, Q = ev.cpu().numpy(), Q.cpu().numpy()
    return ev, Q, st, passes.value


@pytest.mark.parametrize("widths,acts,N,k,chunk,seed", [
    ([37, 9, 5], ["tanh"], 77, 6, 20, 3),
    ([70, 33, 10], ["tanh"], 300, 8, 128, 7),
    ([13, 11, 7, 3], ["sigmoid", "relu"], 200, 10, 1, 4),
    ([4, 5, 3], ["sigmoid"], 100, 5, 33, 0),
])
def test_lowmem_fp64_matches_oracle(hm, widths, acts, N, k, chunk, seed):
    pb = make_problem(widths, acts, N, seed, "normal", "uniform")
    net = hm.HessMLP(pb.widths, pb.acts, pb.omega)
    X = torch.as_tensor(pb.X, device="cuda")
    Y = torch.as_tensor(pb.Y, device="cuda")
    ev, Q, st, passes = lowmem(hm, net, X, Y, N, k, "fp64", chunk)
    assert passes >= 1
    G = O.per_example_grads(pb.omega, pb.widths, pb.acts, pb.X, pb.Y)
    check_eig(ev, Q, G, k, 1e-10, 1e-8)


def test_lowmem_benchmark_network_fp64(hm):
    pb = named_config("mlp_784_16_10")
    net = hm.HessMLP(pb.widths, pb.acts, pb.omega)
    X = torch.as_tensor(pb.X, device="cuda")
    Y = torch.as_tensor(pb.Y, device="cuda")
    k = 32
    ev, Q, st, passes = lowmem(hm, net, X, Y, pb.N, k, "fp64", 300)
    G = O.per_example_grads(pb.omega, pb.widths, pb.acts, pb.X, pb.Y)
    check_eig(ev, Q, G, k, 1e-10, 1e-7)
    # and the same eigenpairs as the Gram route on the device
    ev2, Q2, _ = net.opg_topk_eig(X, Y, k, "fp64")
    assert np.max(np.abs(ev - ev2.cpu().numpy())) <= 1e-10 * ev[0]


def test_lowmem_fp32_products(hm):
    pb = make_problem([70, 33, 10], ["tanh"], 300, 7, "normal", "uniform")
    net = hm.HessMLP(pb.widths, pb.acts, pb.omega)
    X = torch.as_tensor(pb.X, dtype=torch.float32, device="cuda")
    Y = torch.as_tensor(pb.Y, dtype=torch.float32, device="cuda")
    k = 8
    ev, Q, st, passes = lowmem(hm, net, X, Y, pb.N, k, "fp32", 64)
    f = lambda a: np.asarray(a, dtype=np.float32).astype(np.float64)  # noqa: E731
    G = O.per_example_grads(f(pb.omega), pb.widths, pb.acts, f(pb.X), f(pb.Y))
    mu, Qr, _ = O.opg_topk_eig_from_grads(G, k)
    assert np.max(np.abs(ev - mu)) <= 1e-5 * mu[0]
    OPG = G.T @ G / pb.N
    for c in range(k):
        r = OPG @ Q[c] - ev[c] * Q[c]
        assert np.linalg.norm(r) <= 1e-4 * mu[0]


def test_lowmem_host_buffers_equal_device(hm):
    pb = make_problem([37, 9, 5], ["tanh"], 77, 3, "normal", "uniform")
    net = hm.HessMLP(pb.widths, pb.acts, pb.omega)
    evh, Qh, _, _ = lowmem(hm, net, np.ascontiguousarray(pb.X), np.ascontiguousarray(pb.Y), pb.N, 5, "fp64", 25)
    evd, Qd, _, _ = lowmem(hm, net, torch.as_tensor(pb.X, device="cuda"), torch.as_tensor(pb.Y, device="cuda"),
                           pb.N, 5, "fp64", 25)
    assert np.array_equal(evh, evd) and np.array_equal(Qh, Qd)


def test_lowmem_rank_deficient(hm):
    pb = make_problem([6, 5, 4], ["tanh"], 9, 12, "normal", "uniform")
    X, Y = pb.X.copy(), pb.Y.copy()
    X[5], Y[5] = X[1], Y[1]  # a duplicated example: rank(OPG) <= 8
    net = hm.HessMLP(pb.widths, pb.acts, pb.omega)
    ev, Q, st, _ = lowmem(hm, net, torch.as_tensor(X, device="cuda"), torch.as_tensor(Y, device="cuda"), 9, 9,
                          "fp64", 4, allow=(4,))
    assert st == 4
    G = O.per_example_grads(pb.omega, pb.widths, pb.acts, X, Y)
    assert check_eig(ev, Q, G, 9, 1e-10, 1e-8)


def test_lowmem_argument_errors(hm):
    from paper_1905_05559_gb300 import _lib
    pb = make_problem([6, 4], [], 10, 1, "normal", "uniform")
    net = hm.HessMLP(pb.widths, pb.acts, pb.omega)
    X = torch.as_tensor(pb.X, dtype=torch.float32, device="cuda")
    Y = torch.as_tensor(pb.Y, dtype=torch.float32, device="cuda")
    with pytest.raises(hm.HessError) as e:
        lowmem(hm, net, X, Y, 10, 3, "bf16x3", 4)
    assert e.value.status == _lib.HESS_ERR_INVALID_ARG
    with pytest.raises(hm.HessError) as e:
        lowmem(hm, net, X, Y, 10, 11, "fp32", 4)
    assert e.value.status == _lib.HESS_ERR_INVALID_ARG
