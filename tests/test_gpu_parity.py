"""GPU parity: the CUDA library against the FP64 oracle, element by element.

Tolerances (relative Frobenius error against the oracle on the same inputs):
  FP64 path  <= 1e-12
  FP32 path  <= 1e-5   (oracle evaluated at the FP32-rounded inputs and omega)
Eigenvalues are compared relative to the largest one; eigenvectors by
|q . q_ref| when the eigenvalue is separated from its neighbours, otherwise by
the residual of the OPG eigen-equation.
"""

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


def relerr(a, b):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)


def dev(a, dtype):
    return torch.as_tensor(np.ascontiguousarray(a), dtype=dtype, device="cuda")


def rounded(pb, prec):
    """Inputs as the library sees them in this precision (for the oracle)."""
    if prec == "fp64":
        return pb.omega, pb.X, pb.Y
    f = lambda a: np.asarray(a, dtype=np.float32).astype(np.float64)  # noqa: E731
    return f(pb.omega), f(pb.X), f(pb.Y)


SMALL = [
    # (widths, acts, N, seed): several SIMT tiles with ragged tails, all
    # activations, one and two hidden layers, the single softmax layer, N = 1
    ([4, 5, 3], ["sigmoid"], 100, 0),
    ([37, 9, 5], ["tanh"], 77, 3),
    ([13, 11, 7, 3], ["sigmoid", "relu"], 50, 4),
    ([6, 4], [], 33, 5),
    ([5, 3, 2], ["relu"], 1, 6),
    ([70, 33, 10], ["tanh"], 129, 7),
]


def _problem(widths, acts, N, seed):
    return make_problem(widths, acts, N, seed, "normal", "uniform")


@pytest.mark.parametrize("prec,tol", [("fp64", 1e-12), ("fp32", 1e-5)])
@pytest.mark.parametrize("case", SMALL, ids=lambda c: "x".join(map(str, c[0])) + f"_N{c[2]}")
def test_small_full_matrices(hm, case, prec, tol):
    widths, acts, N, seed = case
    pb = _problem(widths, acts, N, seed)
    om, X, Y = rounded(pb, prec)
    dt = torch.float64 if prec == "fp64" else torch.float32
    net = hm.HessMLP(widths, acts, pb.omega)
    Xd, Yd = dev(pb.X, dt), dev(pb.Y, dt)
    G = net.per_example_grads(Xd, Yd, prec).cpu().numpy()
    OPG = net.opg(Xd, Yd, prec).cpu().numpy()
    H = net.exact_hessian(Xd, Yd, prec).cpu().numpy()
    Gr = O.per_example_grads(om, widths, acts, X, Y)
    assert relerr(G, Gr) <= tol
    assert relerr(OPG, O.opg_from_grads(Gr)) <= tol
    assert relerr(H, O.hessian(om, widths, acts, X, Y)) <= tol
    assert np.array_equal(OPG, OPG.T)
    assert np.array_equal(H, H.T)


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
@pytest.mark.parametrize("case", SMALL[:4] + SMALL[5:], ids=lambda c: "x".join(map(str, c[0])))
def test_small_topk_eig(hm, case, prec):
    widths, acts, N, seed = case
    pb = _problem(widths, acts, N, seed)
    # the eigen path runs in FP64 with the FP64 omega on the inputs as given
    _, X, Y = rounded(pb, prec)
    om = pb.omega
    dt = torch.float64 if prec == "fp64" else torch.float32
    net = hm.HessMLP(widths, acts, pb.omega)
    P = O.num_params(widths)
    k = min(6, N, P)
    ev, Q, st = net.opg_topk_eig(dev(pb.X, dt), dev(pb.Y, dt), k, prec, allow_deficient=True)
    Gr = O.per_example_grads(om, widths, acts, X, Y)
    deficient = check_eig(ev.cpu().numpy(), Q.cpu().numpy(), Gr, k, 1e-10, 1e-8)
    assert (st == 4) == deficient


def test_eig_rank_deficient_and_k_equals_n(hm):
    pb = _problem([6, 5, 4], ["tanh"], 9, 12)
    X, Y = pb.X.copy(), pb.Y.copy()
    X[5], Y[5] = X[1], Y[1]  # a duplicated example: rank(M) <= 8
    net = hm.HessMLP(pb.widths, pb.acts, pb.omega)
    ev, Q, st = net.opg_topk_eig(dev(X, torch.float64), dev(Y, torch.float64), 9, "fp64",
                                 allow_deficient=True)
    assert st == 4
    Gr = O.per_example_grads(pb.omega, pb.widths, pb.acts, X, Y)
    assert check_eig(ev.cpu().numpy(), Q.cpu().numpy(), Gr, 9, 1e-10, 1e-8)


def test_host_pointers_match_device_pointers(hm):
    pb = _problem([9, 7, 4], ["sigmoid"], 31, 8)
    net = hm.HessMLP(pb.widths, pb.acts, pb.omega)
    Hh = net.exact_hessian(pb.X, pb.Y, "fp64")  # numpy in, numpy out
    Hd = net.exact_hessian(dev(pb.X, torch.float64), dev(pb.Y, torch.float64), "fp64").cpu().numpy()
    assert isinstance(Hh, np.ndarray)
    assert np.array_equal(Hh, Hd)
    Gh = net.opg(pb.X, pb.Y, "fp64")
    assert relerr(Gh, O.opg(pb.omega, pb.widths, pb.acts, pb.X, pb.Y)) <= 1e-12
    ev, Q, _ = net.opg_topk_eig(pb.X, pb.Y, 3, "fp64")
    ev2, Q2, _ = net.opg_topk_eig(dev(pb.X, torch.float64), dev(pb.Y, torch.float64), 3, "fp64")
    assert np.allclose(ev, ev2.cpu().numpy(), rtol=1e-12, atol=0)


def test_example_split_linearity(hm):
    """H and OPG are means over examples: N H = N1 H_1 + N2 H_2."""
    pb = _problem([11, 6, 5], ["tanh"], 40, 9)
    net = hm.HessMLP(pb.widths, pb.acts, pb.omega)
    X, Y = dev(pb.X, torch.float64), dev(pb.Y, torch.float64)
    for fn in (net.exact_hessian, net.opg):
        full = fn(X, Y).cpu().numpy()
        a = fn(X[:17].contiguous(), Y[:17].contiguous()).cpu().numpy()
        b = fn(X[17:].contiguous(), Y[17:].contiguous()).cpu().numpy()
        assert relerr(40 * full, 17 * a + 23 * b) <= 1e-13


def test_parameter_update_and_errors(hm):
    pb = _problem([5, 4, 3], ["relu"], 12, 10)
    net = hm.HessMLP(pb.widths, pb.acts, np.zeros_like(pb.omega))
    net.set_params(pb.omega)
    X, Y = dev(pb.X, torch.float64), dev(pb.Y, torch.float64)
    H = net.exact_hessian(X, Y).cpu().numpy()
    assert relerr(H, O.hessian(pb.omega, pb.widths, pb.acts, pb.X, pb.Y)) <= 1e-12
    with pytest.raises(hm.HessError) as e:
        net.opg_topk_eig(X, Y, 13, "fp64")
    assert e.value.status == 1
    lib = hm.load()
    out = torch.empty(1, dtype=torch.float64, device="cuda")
    assert lib.opg(net.h, X.data_ptr(), Y.data_ptr(), 0, 0, out.data_ptr()) == 1
    assert lib.opg(net.h, X.data_ptr(), Y.data_ptr(), 12, 9, out.data_ptr()) == 1


# ------------------------------------------------------- full-size config
@pytest.fixture(scope="module")
def cfg784():
    pb = named_config("mlp_784_16_10")
    G64 = O.per_example_grads(pb.omega, pb.widths, pb.acts, pb.X, pb.Y)
    return pb, G64


SAMPLE_COLS = [0, 1, 783, 784, 5000, 12543, 12544, 12559, 12560, 12600, 12719, 12720, 12729]


@pytest.mark.parametrize("prec,tol", [("fp64", 1e-12), ("fp32", 1e-5)])
def test_mlp_784_16_10_sampled(hm, cfg784, prec, tol):
    """Full-size [784,16,10] tanh, N = 1024, the launch shapes the benchmark
    times; outputs checked on sampled rows and columns the oracle computes
    one by one."""
    pb, G64 = cfg784
    om, X, Y = rounded(pb, prec)
    Gr = G64 if prec == "fp64" else O.per_example_grads(om, pb.widths, pb.acts, X, Y)
    dt = torch.float64 if prec == "fp64" else torch.float32
    net = hm.HessMLP(pb.widths, pb.acts, pb.omega)
    Xd, Yd = dev(pb.X, dt), dev(pb.Y, dt)
    G = net.per_example_grads(Xd, Yd, prec)
    rows = [0, 1, 511, 1023]
    assert relerr(G[rows].cpu().numpy(), Gr[rows]) <= tol
    del G
    OPG = net.opg(Xd, Yd, prec)
    cols = torch.tensor(SAMPLE_COLS, device="cuda")
    ref = (Gr.T @ Gr[:, SAMPLE_COLS]) / pb.N
    assert relerr(OPG[:, cols].cpu().numpy(), ref) <= tol
    assert relerr(OPG[cols].cpu().numpy(), ref.T) <= tol
    del OPG
    H = net.exact_hessian(Xd, Yd, prec)
    Href = O.hessian_columns(om, pb.widths, pb.acts, X, Y, SAMPLE_COLS)
    assert relerr(H[:, cols].cpu().numpy(), Href) <= tol
    assert relerr(H[cols].cpu().numpy(), Href.T) <= tol
    # exact symmetry on a block straddling layer boundaries (bias blocks included)
    blk = H[12500:12730, 12500:12730]
    assert torch.equal(blk, blk.T)


def test_mlp_784_16_10_topk(hm, cfg784):
    pb, G64 = cfg784
    net = hm.HessMLP(pb.widths, pb.acts, pb.omega)
    ev, Q, st = net.opg_topk_eig(dev(pb.X, torch.float64), dev(pb.Y, torch.float64), 32, "fp64")
    assert st == 0
    check_eig(ev.cpu().numpy(), Q.cpu().numpy(), G64, 32, 1e-10, 1e-7)
