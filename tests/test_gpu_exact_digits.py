"""The exact-digit FP64 products on the tensor cores (the Gram matrix's wide
layer and the back-projection of the OPG eigensolver) against the FP64
oracle, at shapes where both take that route (input width and N of at least
128): eigenvalues to 1e-12 of the largest, eigenvectors by abs(q . q_ref)
and by the residual with the oracle's OPG.  One data set spreads each input
row over about 18 orders of magnitude (columns scaled from 1e-8 to 1e10), so
that the per-row power-of-two scaling and the truncation after eight digits
are exercised."""

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


def dev(a):
    return torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float64, device="cuda")


@pytest.mark.parametrize("spread", [False, True])
def test_opg_eig_through_exact_digit_products(hm, spread):
    pb = make_problem([200, 30, 10], ["tanh"], 300, 21, "normal", "uniform")
    X = pb.X.copy()
    if spread:
        X *= np.logspace(-8, 10, X.shape[1])[None, :]
    net = hm.HessMLP(pb.widths, pb.acts, pb.omega)
    k = 12
    lam, Q, _ = net.opg_topk_eig(dev(X), dev(pb.Y), k, "fp64")
    lam, Q = lam.cpu().numpy(), Q.cpu().numpy()
    lam_ref, Q_ref, _ = O.opg_topk_eig(pb.omega, pb.widths, pb.acts, X, pb.Y, k)
    assert np.abs(lam - lam_ref).max() <= 1e-12 * lam_ref[0]
    M = O.opg(pb.omega, pb.widths, pb.acts, X, pb.Y)
    gaps = np.minimum(np.r_[np.inf, -np.diff(lam_ref)], np.r_[-np.diff(lam_ref), np.inf])
    for c in range(k):
        if gaps[c] > 1e-4 * lam_ref[0]:
            assert abs(abs(Q[c] @ Q_ref[:, c]) - 1.0) <= 1e-10
        assert np.linalg.norm(M @ Q[c] - lam[c] * Q[c]) <= 1e-9 * lam_ref[0]


@pytest.mark.parametrize("widths,N,seed", [([200, 30, 10], 600, 22), ([64, 40, 10], 1024, 23)],
                         ids=["groups-ragged-ones-row", "transposed-narrow"])
def test_back_projection_digit_routes(hm, widths, N, seed):
    """The back-projection's exact-digit products: [200, 30, 10] at N = 600
    takes the first layer's R = A^T B (B of 30 x 12 = 360 columns: a group of
    256 and a ragged group of 104) with a row of ones appended to A^T for the
    bias rows; [64, 40, 10] at N = 1024 takes the transposed product of a
    narrow layer (480 rows against 64 columns)."""
    from eigcheck import check_eig
    pb = make_problem(widths, ["tanh"], N, seed, "normal", "uniform")
    net = hm.HessMLP(pb.widths, pb.acts, pb.omega)
    k = 12
    lam, Q, _ = net.opg_topk_eig(dev(pb.X), dev(pb.Y), k, "fp64")
    Gr = O.per_example_grads(pb.omega, pb.widths, pb.acts, pb.X, pb.Y)
    check_eig(lam.cpu().numpy(), Q.cpu().numpy(), Gr, k, 1e-12, 1e-10)


def test_gram_with_two_wide_layers(hm):
    """Two layers wide enough for the exact-digit Gram term ([160, 130, 10]):
    the second layer's planes are combined by a second fused launch that adds
    to the first one's double-float output."""
    from eigcheck import check_eig
    pb = make_problem([160, 130, 10], ["sigmoid"], 300, 24, "normal", "uniform")
    net = hm.HessMLP(pb.widths, pb.acts, pb.omega)
    k = 10
    lam, Q, _ = net.opg_topk_eig(dev(pb.X), dev(pb.Y), k, "fp64")
    Gr = O.per_example_grads(pb.omega, pb.widths, pb.acts, pb.X, pb.Y)
    check_eig(lam.cpu().numpy(), Q.cpu().numpy(), Gr, k, 1e-12, 1e-10)
