"""Low-rank and full-rank approximations from K eigenpairs (Sec. 4.1, 4.2),
formed and applied implicitly (Sec. 5.5, 5.6), against the FP64 oracle.

* Formed matrices from the oracle's Hessian eigenpairs, FP64 (1e-12) and FP32
  (1e-6), low- and full-rank, lam_tilde given or lam_K; exact symmetry.
* A ragged random orthonormal basis (P = 3003, K = 37) spanning many tiles.
* Implicit products and quadratic forms, device and host buffers, b = 1 and
  b = 19, quadratic forms alone.
* The chain hessian_topk_eig -> hess_approx_form on the GPU against the
  oracle's chain (K at a spectral gap, so the approximation is unique).
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


def dev(a):
    return torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float64, device="cuda")


@pytest.fixture(scope="module")
def problem():
    pb = make_problem([12, 9, 7, 5], ["tanh", "sigmoid"], 40, 3, "normal", "uniform")
    lam, Q = O.hessian_topk_eig(pb.omega, pb.widths, pb.acts, pb.X, pb.Y, 9)
    return pb, lam, Q


@pytest.mark.parametrize("full,lt", [(False, None), (True, None), (True, 0.05)])
def test_form_matches_oracle(hm, problem, full, lt):
    pb, lam, Q = problem
    net = hm.HessMLP(pb.widths, pb.acts, pb.omega)
    ev, qs = dev(lam), dev(Q.T)
    lam_tilde = lam[-1] if (full and lt is None) else lt
    ref = O.fullrank_matrix(Q, lam, lam_tilde) if full else O.lowrank_matrix(Q, lam)
    kw = {"full": full} if lt is None else {"full": full, "lam_tilde": lt}
    out = net.approx_form(ev, qs, prec="fp64", **kw)
    o = out.cpu().numpy()
    assert relerr(o, ref) <= 1e-12
    assert np.array_equal(o, o.T)
    out32 = net.approx_form(ev, qs, prec="fp32", **kw).cpu().numpy()
    assert out32.dtype == np.float32 and relerr(out32, ref) <= 1e-6


def test_form_ragged_basis_host_buffers(hm):
    rng = np.random.default_rng(7)
    # the network only fixes the handle's P (ragged: 3003)
    widths = [1000, 3]
    P = 3003
    net = hm.HessMLP(widths, [], np.zeros(P))
    assert net.P == P
    K = 37
    Q, _ = np.linalg.qr(rng.standard_normal((P, K)))
    lam = np.sort(rng.standard_normal(K))[::-1].copy()
    out = np.empty((P, P))
    net.approx_form(np.ascontiguousarray(lam), np.ascontiguousarray(Q.T), full=True, lam_tilde=0.25, out=out)
    assert relerr(out, O.fullrank_matrix(Q, lam, 0.25)) <= 1e-12


@pytest.mark.parametrize("b", [1, 19])
@pytest.mark.parametrize("full", [False, True])
def test_apply_matches_oracle(hm, problem, b, full):
    pb, lam, Q = problem
    net = hm.HessMLP(pb.widths, pb.acts, pb.omega)
    X = np.random.default_rng(b).standard_normal((b, pb.P))
    lt = lam[-1] if full else None
    HXr, qr = O.approx_apply(Q, lam, X, lam_tilde=lt)
    HX, quad = net.approx_apply(dev(lam), dev(Q.T), dev(X), full=full)
    assert relerr(HX.cpu().numpy(), HXr) <= 1e-12
    assert np.abs(quad.cpu().numpy() - qr).max() <= 1e-12 * np.abs(qr).max()
    # host buffers, quadratic forms alone
    HX2, quad2 = net.approx_apply(np.ascontiguousarray(lam), np.ascontiguousarray(Q.T),
                                  np.ascontiguousarray(X), full=full, products=False)
    assert HX2 is None and np.abs(quad2 - qr).max() <= 1e-12 * np.abs(qr).max()


def test_chain_from_gpu_eigenpairs(hm):
    pb = make_problem([16, 12, 10], ["tanh"], 50, 8, "normal", "uniform")
    lam_all, _ = O.hessian_topk_eig(pb.omega, pb.widths, pb.acts, pb.X, pb.Y, 12)
    gaps = lam_all[:-1] - lam_all[1:]
    K = int(np.argmax(gaps[4:])) + 5  # K between 5 and 11 at the widest gap
    lam_ref, Q_ref = O.hessian_topk_eig(pb.omega, pb.widths, pb.acts, pb.X, pb.Y, K)
    net = hm.HessMLP(pb.widths, pb.acts, pb.omega)
    lam, Q, _ = net.hessian_topk_eig(dev(pb.X), dev(pb.Y), K, "fp64")
    out = net.approx_form(lam, Q, full=True).cpu().numpy()
    assert relerr(out, O.fullrank_matrix(Q_ref, lam_ref, lam_ref[-1])) <= 1e-8


def test_approx_argument_errors(hm, problem):
    pb, lam, Q = problem
    net = hm.HessMLP(pb.widths, pb.acts, pb.omega)
    ev, qs = dev(lam), dev(Q.T)
    lib = hm.load()
    with pytest.raises(hm.HessError, match="K"):
        hm._lib.check(lib.hess_approx_form(net.h, 0, hm.api._ptr(ev), hm.api._ptr(qs), 0, 0.0, 0,
                                           hm.api._ptr(dev(np.zeros((pb.P, pb.P))))))
    with pytest.raises(hm.HessError, match="FP64 or FP32"):
        net.approx_form(ev, qs, prec="bf16x3")
    with pytest.raises(hm.HessError, match="no output"):
        hm._lib.check(lib.hess_approx_apply(net.h, 9, hm.api._ptr(ev), hm.api._ptr(qs), 0, 0.0,
                                            hm.api._ptr(dev(np.zeros(pb.P))), 1, None, None))
    with pytest.raises(ValueError):
        net.approx_form(ev, dev(Q), full=False)
