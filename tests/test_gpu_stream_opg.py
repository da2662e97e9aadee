"""Top-k OPG eigenpairs from chunks of examples (opg_topk_eig_streaming)
against the FP64 oracle.

* FP64 with ragged chunks, one chunk, and one example per chunk: eigenvalues
  to 1e-10 of the largest, separated eigenvectors by abs(q . q_ref), all by
  the residual ||OPG q - mu q|| with the oracle's OPG; the same values as the
  Gram route (opg_topk_eig).
* N = 70000 examples, beyond the Gram route's limit, against the oracle's
  P x P route.
* Split-BF16 chunk OPGs (1e-5); host buffers; rank deficiency; errors.
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


def dev(a, dt=torch.float64):
    return torch.as_tensor(np.ascontiguousarray(a), dtype=dt, device="cuda")


def check(pb, lam, Q, lam_ref, Q_ref, tol=1e-10, vtol=1e-8, om=None, X=None, Y=None):
    om = pb.omega if om is None else om
    X = pb.X if X is None else X
    Y = pb.Y if Y is None else Y
    scale = lam_ref[0]
    assert np.abs(lam - lam_ref).max() <= tol * scale
    M = O.opg(om, pb.widths, pb.acts, X, Y)
    gaps = np.r_[np.inf, -np.diff(lam_ref), np.inf]
    for c in range(len(lam)):
        if min(gaps[c], gaps[c + 1]) > 1e-3 * scale:
            assert abs(abs(Q[c] @ Q_ref[:, c]) - 1.0) <= vtol
        assert np.linalg.norm(M @ Q[c] - lam[c] * Q[c]) <= 1e3 * tol * scale


@pytest.mark.parametrize("chunk", [37, 1000, 1])
def test_streaming_fp64(hm, chunk):
    N = 140 if chunk == 1 else 300
    pb = make_problem([14, 10, 6], ["tanh"], N, 5, "normal", "uniform")
    net = hm.HessMLP(pb.widths, pb.acts, pb.omega)
    k = 12
    lam, Q, _ = net.opg_topk_eig_streaming(dev(pb.X), dev(pb.Y), k, "fp64", chunk=chunk)
    lam, Q = lam.cpu().numpy(), Q.cpu().numpy()
    lam_ref, Q_ref, _ = O.opg_topk_eig(pb.omega, pb.widths, pb.acts, pb.X, pb.Y, k)
    check(pb, lam, Q, lam_ref, Q_ref)
    lg, _, _ = net.opg_topk_eig(dev(pb.X), dev(pb.Y), k, "fp64")
    assert np.abs(lam - lg.cpu().numpy()).max() <= 1e-11 * lam_ref[0]


def test_streaming_beyond_gram_limit(hm):
    pb = make_problem([8, 6, 4], ["sigmoid"], 70000, 6, "normal", "uniform")
    net = hm.HessMLP(pb.widths, pb.acts, pb.omega)
    k = 10
    with pytest.raises(hm.HessError):
        net.opg_topk_eig(dev(pb.X), dev(pb.Y), k, "fp64")
    lam, Q, _ = net.opg_topk_eig_streaming(dev(pb.X), dev(pb.Y), k, "fp64", chunk=8192)
    lam_ref, Q_ref, _ = O.opg_topk_eig_direct(pb.omega, pb.widths, pb.acts, pb.X, pb.Y, k)
    check(pb, lam.cpu().numpy(), Q.cpu().numpy(), lam_ref, Q_ref)


def test_streaming_bf16x3_and_host_buffers(hm):
    pb = make_problem([40, 24, 10], ["relu"], 900, 7, "normal", "uniform")
    f32 = lambda a: np.asarray(a, dtype=np.float32)  # noqa: E731
    om = f32(pb.omega).astype(np.float64)
    net = hm.HessMLP(pb.widths, pb.acts, om)
    k = 16
    lam, Q, _ = net.opg_topk_eig_streaming(f32(pb.X), f32(pb.Y), k, "bf16x3", chunk=256)
    X64, Y64 = f32(pb.X).astype(np.float64), f32(pb.Y).astype(np.float64)
    lam_ref, Q_ref, _ = O.opg_topk_eig(om, pb.widths, pb.acts, X64, Y64, k)
    assert np.abs(lam - lam_ref).max() <= 1e-5 * lam_ref[0]
    M = O.opg(om, pb.widths, pb.acts, X64, Y64)
    for c in range(k):
        assert np.linalg.norm(M @ Q[c] - lam[c] * Q[c]) <= 1e-4 * lam_ref[0]


def test_streaming_rank_deficient_and_errors(hm):
    pb = make_problem([6, 5, 4], ["tanh"], 40, 8, "normal", "uniform")
    X = np.repeat(pb.X[:3], 10, axis=0)[:24]
    Y = np.repeat(pb.Y[:3], 10, axis=0)[:24]
    net = hm.HessMLP(pb.widths, pb.acts, pb.omega)
    lam, Q, st = net.opg_topk_eig_streaming(dev(X), dev(Y), 8, "fp64", chunk=5, allow_deficient=True)
    assert st == hm._lib.HESS_ERR_RANK_DEFICIENT
    lam = lam.cpu().numpy()
    Q = Q.cpu().numpy()
    lam_ref, _, deficient = O.opg_topk_eig(pb.omega, pb.widths, pb.acts, X, Y, 8)
    assert deficient
    live = lam_ref > 1e-13 * lam_ref[0]
    assert np.abs(lam[live] - lam_ref[live]).max() <= 1e-10 * lam_ref[0]
    assert np.all(Q[~live] == 0.0)
    with pytest.raises(hm.HessError, match="chunk"):
        net.opg_topk_eig_streaming(dev(pb.X), dev(pb.Y), 3, "fp64", chunk=0)
    with pytest.raises(hm.HessError, match="k"):
        net.opg_topk_eig_streaming(dev(pb.X), dev(pb.Y), 0, "fp64")
