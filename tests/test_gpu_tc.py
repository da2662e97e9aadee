"""GPU parity of the tensor-core (tcgen05) paths against the FP64 oracle.

Split-BF16 (hi*hi + hi*lo + lo*hi, FP32 accumulation): relative Frobenius
error <= 1e-5; plain BF16: <= 1e-2.  The oracle runs at the FP32-rounded
inputs and parameters that the library computes from.
"""

import numpy as np
import pytest

from oracle import mlp as O
from synth import make_problem, named_config

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

TOL = {"bf16x3": 1e-5, "bf16": 1e-2}


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


def dev(a):
    return torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float32, device="cuda")


CASES = [
    # one tile, single softmax layer, N = 1 (one k-block), ragged tiles and K
    ([4, 5, 3], ["sigmoid"], 100, 0),
    ([6, 4], [], 33, 5),
    ([5, 3, 2], ["relu"], 1, 6),
    ([70, 33, 10], ["tanh"], 129, 7),
    ([13, 11, 7, 3], ["sigmoid", "relu"], 50, 4),
    ([200, 24, 10], ["tanh"], 300, 11),
]


@pytest.mark.parametrize("prec", ["bf16x3", "bf16"])
@pytest.mark.parametrize("case", CASES, ids=lambda c: "x".join(map(str, c[0])) + f"_N{c[2]}")
def test_tc_opg_and_hessian(hm, case, prec):
    widths, acts, N, seed = case
    pb = make_problem(widths, acts, N, seed, "normal", "uniform")
    om, X, Y = f32(pb.omega), f32(pb.X), f32(pb.Y)
    net = hm.HessMLP(widths, acts, pb.omega)
    Xd, Yd = dev(pb.X), dev(pb.Y)
    OPG = net.opg(Xd, Yd, prec).cpu().numpy()
    Gr = O.per_example_grads(om, widths, acts, X, Y)
    assert relerr(OPG, O.opg_from_grads(Gr)) <= TOL[prec]
    assert np.array_equal(OPG, OPG.T)
    H = net.exact_hessian(Xd, Yd, prec).cpu().numpy()
    Hr = O.hessian(om, widths, acts, X, Y)
    assert relerr(H, Hr) <= TOL[prec]
    assert np.array_equal(H, H.T)
    # every entry written: no NaN from uninitialised memory
    assert np.isfinite(H).all() and np.isfinite(OPG).all()


def test_tc_results_do_not_depend_on_previous_contents(hm):
    pb = make_problem([37, 9, 5], ["tanh"], 77, 3, "normal", "uniform")
    net = hm.HessMLP(pb.widths, pb.acts, pb.omega)
    Xd, Yd = dev(pb.X), dev(pb.Y)
    P = pb.P
    a = torch.full((P, P), float("nan"), device="cuda")
    b = torch.zeros((P, P), device="cuda")
    net.exact_hessian(Xd, Yd, "bf16x3", out=a)
    net.exact_hessian(Xd, Yd, "bf16x3", out=b)
    assert torch.equal(a, b)
    net.opg(Xd, Yd, "bf16x3", out=a.fill_(float("nan")))
    net.opg(Xd, Yd, "bf16x3", out=b)
    assert torch.equal(a, b)


@pytest.fixture(scope="module")
def cfg784():
    pb = named_config("mlp_784_16_10")
    om, X, Y = f32(pb.omega), f32(pb.X), f32(pb.Y)
    G = O.per_example_grads(om, pb.widths, pb.acts, X, Y)
    return pb, (om, X, Y), G


SAMPLE_COLS = [0, 1, 783, 784, 5000, 9999, 12543, 12544, 12559, 12560, 12600, 12719, 12720, 12729]


@pytest.mark.parametrize("prec", ["bf16x3", "bf16"])
def test_tc_mlp_784_16_10_sampled(hm, cfg784, prec):
    """Full-size [784,16,10] tanh, N = 1024 (the benchmark's launch shapes)."""
    pb, (om, X, Y), G = cfg784
    net = hm.HessMLP(pb.widths, pb.acts, pb.omega)
    Xd, Yd = dev(pb.X), dev(pb.Y)
    cols = torch.tensor(SAMPLE_COLS, device="cuda")
    OPG = net.opg(Xd, Yd, prec)
    ref = (G.T @ G[:, SAMPLE_COLS]) / pb.N
    assert relerr(OPG[:, cols].cpu().numpy(), ref) <= TOL[prec]
    assert relerr(OPG[cols].cpu().numpy(), ref.T) <= TOL[prec]
    del OPG
    H = net.exact_hessian(Xd, Yd, prec)
    Href = O.hessian_columns(om, pb.widths, pb.acts, X, Y, SAMPLE_COLS)
    assert relerr(H[:, cols].cpu().numpy(), Href) <= TOL[prec]
    assert relerr(H[cols].cpu().numpy(), Href.T) <= TOL[prec]
    assert bool(torch.isfinite(H).all())


@pytest.mark.parametrize("kind", ["opg", "exact_hessian"])
def test_tc_host_buffers_match_device_buffers(hm, kind):
    # host X, Y and output: the library stages them in its workspace
    pb = make_problem([70, 33, 10], ["tanh"], 129, 7, "normal", "uniform")
    net = hm.HessMLP(pb.widths, pb.acts, pb.omega)
    Xh = np.ascontiguousarray(pb.X, dtype=np.float32)
    Yh = np.ascontiguousarray(pb.Y, dtype=np.float32)
    host = getattr(net, kind)(Xh, Yh, "bf16x3")
    assert isinstance(host, np.ndarray)
    devo = getattr(net, kind)(dev(pb.X), dev(pb.Y), "bf16x3").cpu().numpy()
    assert np.array_equal(host, devo)


@pytest.mark.parametrize("kind", ["opg", "exact_hessian"])
def test_tc_pinned_host_output_written_in_place(hm, kind):
    # a pinned host output is written by the kernels over the host link
    pb = make_problem([70, 33, 10], ["tanh"], 129, 7, "normal", "uniform")
    net = hm.HessMLP(pb.widths, pb.acts, pb.omega)
    X, Y = dev(pb.X), dev(pb.Y)
    out = torch.full((pb.P, pb.P), float("nan"), dtype=torch.float32, pin_memory=True)
    getattr(net, kind)(X, Y, "bf16x3", out=out)  # returns after its work (host buffer)
    ref = getattr(net, kind)(X, Y, "bf16x3").cpu()
    assert torch.equal(out, ref)
