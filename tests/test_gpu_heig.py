"""Hessian-vector products and the top-k Hessian eigenpairs (Lanczos on the
operator v -> H v, Sec. 5.3) against the FP64 oracle.

* hessian_vector_products: random directions on small networks of each
  activation, FP64 at 1e-12 and FP32 at 1e-5 (relative Frobenius); unit
  directions reproduce the exact-Hessian columns.
* hessian_topk_eig on small networks: eigenvalues against the oracle's full
  eigendecomposition (1e-10 of the largest magnitude), eigenvectors by
  |q . q_ref| where the gap is clear, else by the oracle's residual
  ||H q - lam q||; k = P (the whole space, through breakdowns and restarts),
  ReLU, FP32 products, repeated calls bit-identical, argument errors.
* The 784-16-10 network (P = 12730, N = 1024, k = 32): eigenvalues against
  the stored oracle values, residuals through the oracle's products.
"""

import os

import numpy as np
import pytest

from oracle import mlp as O
from synth import make_problem, named_config

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


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


def dev(a, dt=torch.float64):
    return torch.as_tensor(np.ascontiguousarray(a), dtype=dt, device="cuda")


NETS = [
    ([6, 5, 4], ["sigmoid"], 40, 1),
    ([12, 9, 7, 5], ["tanh", "relu"], 33, 2),
    ([20, 16, 10], ["relu"], 64, 3),
    ([8, 6], [], 25, 4),
    ([10, 7, 6, 5, 4], ["tanh", "sigmoid", "tanh"], 50, 5),
]


@pytest.mark.parametrize("w,a,n,seed", NETS)
def test_hvp_fp64_matches_oracle(hm, w, a, n, seed):
    pb = make_problem(w, a, n, seed, "normal", "uniform")
    net = hm.HessMLP(pb.widths, pb.acts, pb.omega)
    rng = np.random.default_rng(seed)
    V = rng.standard_normal((7, pb.P))
    HV = net.hvp(dev(pb.X), dev(pb.Y), dev(V), "fp64").cpu().numpy()
    for d in range(V.shape[0]):
        ref = O.hvp(pb.omega, pb.widths, pb.acts, pb.X, pb.Y, V[d])
        assert relerr(HV[d], ref) <= 1e-12


def test_hvp_fp32_matches_oracle(hm):
    pb = make_problem([12, 9, 7, 5], ["tanh", "sigmoid"], 48, 6, "normal", "uniform")
    f32 = lambda x: np.asarray(x, dtype=np.float32)  # noqa: E731
    om = f32(pb.omega).astype(np.float64)
    net = hm.HessMLP(pb.widths, pb.acts, om)
    V = f32(np.random.default_rng(1).standard_normal((3, pb.P)))
    HV = net.hvp(dev(f32(pb.X), torch.float32), dev(f32(pb.Y), torch.float32),
                 dev(V, torch.float32), "fp32").cpu().numpy()
    for d in range(3):
        ref = O.hvp(om, pb.widths, pb.acts, f32(pb.X).astype(np.float64),
                    f32(pb.Y).astype(np.float64), V[d].astype(np.float64))
        assert relerr(HV[d], ref) <= 1e-5


def test_hvp_unit_directions_are_hessian_columns(hm):
    pb = make_problem([9, 7, 6, 4], ["tanh", "sigmoid"], 30, 7, "normal", "uniform")
    net = hm.HessMLP(pb.widths, pb.acts, pb.omega)
    X, Y = dev(pb.X), dev(pb.Y)
    H = net.exact_hessian(X, Y, "fp64").cpu().numpy()
    E = np.eye(pb.P)
    HV = net.hvp(X, Y, dev(E), "fp64").cpu().numpy()
    assert relerr(HV, H) <= 1e-12  # row d of HV = H e_d = column d (H symmetric)
    # host buffers, one direction
    v = np.ascontiguousarray(E[5])
    hv = net.hvp(np.ascontiguousarray(pb.X), np.ascontiguousarray(pb.Y), v, "fp64")
    assert isinstance(hv, np.ndarray) and relerr(hv, H[5]) <= 1e-12


def check_eigs(pb, lam, Q, lam_ref, Q_ref, tol=1e-10):
    scale = np.abs(lam_ref).max()
    assert np.abs(lam - lam_ref).max() <= tol * scale
    assert np.allclose(Q @ Q.T, np.eye(len(lam)), atol=1e-9)
    full_gap = np.r_[np.inf, -np.diff(lam_ref)]
    for c in range(len(lam)):
        gap = min(full_gap[c], full_gap[c + 1] if c + 1 < len(lam) else np.inf)
        if gap > 1e-4 * scale:
            assert abs(abs(Q[c] @ Q_ref[:, c]) - 1.0) <= 1e-8
        Hq = O.hvp(pb.omega, pb.widths, pb.acts, pb.X, pb.Y, Q[c])
        assert np.linalg.norm(Hq - lam[c] * Q[c]) <= 1e-8 * scale


@pytest.mark.parametrize("w,a,n,seed,k", [
    ([6, 5, 4], ["sigmoid"], 40, 1, 5),
    ([12, 9, 7, 5], ["tanh", "relu"], 33, 2, 12),
    ([20, 16, 10], ["relu"], 64, 3, 20),
    ([16, 12, 10], ["tanh"], 50, 8, 1),
])
def test_hessian_topk_eig_matches_oracle(hm, w, a, n, seed, k):
    pb = make_problem(w, a, n, seed, "normal", "uniform")
    net = hm.HessMLP(pb.widths, pb.acts, pb.omega)
    lam, Q, steps = net.hessian_topk_eig(dev(pb.X), dev(pb.Y), k, "fp64")
    lam_ref, Q_ref = O.hessian_topk_eig(pb.omega, pb.widths, pb.acts, pb.X, pb.Y, k)
    assert k <= steps <= pb.P
    check_eigs(pb, lam.cpu().numpy(), Q.cpu().numpy(), lam_ref, Q_ref)


def test_hessian_topk_eig_whole_space(hm):
    """k = P on a 43-parameter network: the Krylov space fills R^P (through
    breakdowns and restarts) and every eigenvalue comes out."""
    pb = make_problem([4, 5, 3], ["sigmoid"], 100, 0, "normal", "uniform")
    assert pb.P == 43
    net = hm.HessMLP(pb.widths, pb.acts, pb.omega)
    lam, Q, steps = net.hessian_topk_eig(np.ascontiguousarray(pb.X), np.ascontiguousarray(pb.Y),
                                         pb.P, "fp64")
    assert steps == pb.P
    lam_ref, Q_ref = O.hessian_topk_eig(pb.omega, pb.widths, pb.acts, pb.X, pb.Y, pb.P)
    assert np.abs(lam - lam_ref).max() <= 1e-10 * np.abs(lam_ref).max()
    assert np.allclose(Q @ Q.T, np.eye(pb.P), atol=1e-9)
    H = O.hessian(pb.omega, pb.widths, pb.acts, pb.X, pb.Y)
    assert relerr((Q.T * lam) @ Q, H) <= 1e-9


def test_hessian_topk_eig_fp32_products_and_repeatability(hm):
    pb = make_problem([12, 9, 7, 5], ["tanh", "sigmoid"], 48, 6, "normal", "uniform")
    f32 = lambda x: np.asarray(x, dtype=np.float32)  # noqa: E731
    om = f32(pb.omega).astype(np.float64)
    net = hm.HessMLP(pb.widths, pb.acts, om)
    X, Y = dev(f32(pb.X), torch.float32), dev(f32(pb.Y), torch.float32)
    lam, Q, _ = net.hessian_topk_eig(X, Y, 8, "fp32")
    lam2, Q2, _ = net.hessian_topk_eig(X, Y, 8, "fp32")
    assert torch.equal(lam, lam2) and torch.equal(Q, Q2)
    lam_ref, _ = O.hessian_topk_eig(om, pb.widths, pb.acts, f32(pb.X).astype(np.float64),
                                    f32(pb.Y).astype(np.float64), 8)
    assert np.abs(lam.cpu().numpy() - lam_ref).max() <= 1e-5 * np.abs(lam_ref).max()


def test_hessian_topk_eig_mlp_784_16_10(hm):
    pb = named_config("mlp_784_16_10")
    gold = np.loadtxt(os.path.join(GOLDEN, "hessian_top_eigs_mlp_784_16_10.txt"))
    k = 32
    net = hm.HessMLP(pb.widths, pb.acts, pb.omega)
    lam, Q, steps = net.hessian_topk_eig(dev(pb.X), dev(pb.Y), k, "fp64")
    lam, Q = lam.cpu().numpy(), Q.cpu().numpy()
    assert np.abs(lam - gold[:k]).max() <= 1e-10 * abs(gold[0])
    assert np.allclose(Q @ Q.T, np.eye(k), atol=1e-9)
    f = O.forward(pb.omega, pb.widths, pb.acts, pb.X)
    for c in (0, 1, 7, 15, 31):
        Hq = O.hvp(pb.omega, pb.widths, pb.acts, pb.X, pb.Y, Q[c], f=f)
        assert np.linalg.norm(Hq - lam[c] * Q[c]) <= 1e-8 * abs(gold[0])
    assert steps <= 8 * k + 1024


def test_hessian_operator_argument_errors(hm):
    pb = make_problem([6, 5, 4], ["sigmoid"], 20, 1, "normal", "uniform")
    net = hm.HessMLP(pb.widths, pb.acts, pb.omega)
    X, Y = dev(pb.X), dev(pb.Y)
    with pytest.raises(hm.HessError, match="k"):
        net.hessian_topk_eig(X, Y, 0, "fp64")
    with pytest.raises(hm.HessError, match="k"):
        net.hessian_topk_eig(X, Y, pb.P + 1, "fp64")
    Xf, Yf = dev(pb.X, torch.float32), dev(pb.Y, torch.float32)
    with pytest.raises(hm.HessError, match="FP64 or FP32"):
        net.hessian_topk_eig(Xf, Yf, 3, "bf16x3")
    with pytest.raises(hm.HessError, match="FP64 or FP32"):
        net.hvp(Xf, Yf, dev(np.zeros(pb.P), torch.float32), "bf16")
    with pytest.raises(ValueError):
        net.hvp(X, Y, dev(np.zeros(pb.P + 1)), "fp64")
