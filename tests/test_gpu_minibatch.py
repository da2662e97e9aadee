"""Mini-batch and per-example Hessians (hessian_minibatches, Sec. 5.1)
against the FP64 oracle.

* FP64 (1e-12) with a ragged last batch, host and device buffers; bs = 1
  (per-example Hessians); bs >= N (one batch equal to exact_hessian).
* Split-BF16 through the handle's batch waves (1e-5), each matrix
  bit-identical to exact_hessian on its slice.
* Argument errors.
"""

import numpy as np
import pytest

from oracle import mlp as O
from synth import make_problem

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


def relerr(a, b):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)


def f32(a):
    return np.asarray(a, dtype=np.float32).astype(np.float64)


@pytest.mark.parametrize("bs", [1, 7, 64])
def test_minibatches_fp64(hm, bs):
    pb = make_problem([10, 8, 6, 4], ["tanh", "relu"], 23, 5, "normal", "uniform")
    net = hm.HessMLP(pb.widths, pb.acts, pb.omega)
    X = torch.as_tensor(pb.X, device="cuda")
    Y = torch.as_tensor(pb.Y, device="cuda")
    Hs = net.hessian_minibatches(X, Y, bs, "fp64").cpu().numpy()
    ref = O.minibatch_hessians(pb.omega, pb.widths, pb.acts, pb.X, pb.Y, bs)
    assert Hs.shape == ref.shape
    for b in range(ref.shape[0]):
        assert relerr(Hs[b], ref[b]) <= 1e-12
    if bs >= pb.N:
        whole = net.exact_hessian(X, Y, "fp64").cpu().numpy()
        assert np.array_equal(Hs[0], whole)
    # host buffers
    Hh = net.hessian_minibatches(np.ascontiguousarray(pb.X), np.ascontiguousarray(pb.Y), bs, "fp64")
    assert np.array_equal(Hh, Hs)


@pytest.mark.parametrize("prec", ["bf16x3", "bf16"])
def test_minibatches_tensor_cores(hm, prec):
    pb = make_problem([24, 16, 10], ["tanh"], 70, 6, "normal", "uniform")
    om = f32(pb.omega)
    net = hm.HessMLP(pb.widths, pb.acts, om)
    X = torch.as_tensor(pb.X, dtype=torch.float32, device="cuda")
    Y = torch.as_tensor(pb.Y, dtype=torch.float32, device="cuda")
    bs = 16
    Hs = net.hessian_minibatches(X, Y, bs, prec)
    ref = O.minibatch_hessians(om, pb.widths, pb.acts, f32(pb.X), f32(pb.Y), bs)
    tol = 1e-5 if prec == "bf16x3" else 1e-2
    for b in range(ref.shape[0]):
        assert relerr(Hs[b].cpu().numpy(), ref[b]) <= tol
        one = net.exact_hessian(X[b * bs:(b + 1) * bs].contiguous(), Y[b * bs:(b + 1) * bs].contiguous(),
                                prec)
        assert torch.equal(Hs[b], one)


def test_minibatch_argument_errors(hm):
    pb = make_problem([6, 5, 4], ["sigmoid"], 20, 1, "normal", "uniform")
    net = hm.HessMLP(pb.widths, pb.acts, pb.omega)
    X = torch.as_tensor(pb.X, device="cuda")
    Y = torch.as_tensor(pb.Y, device="cuda")
    with pytest.raises(hm.HessError, match="mini-batch size"):
        net.hessian_minibatches(X, Y, 0, "fp64", out=torch.empty((1, pb.P, pb.P), dtype=torch.float64,
                                                                   device="cuda"))
