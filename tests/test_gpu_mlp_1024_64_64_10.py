"""Full-size precision workload: MLP [1024,64,64,10] ReLU, P = 70410,
N = 8192.  G in FP32, the OPG symmetric rank-N update in BF16 and split-BF16
(FP32 accumulation), the top-100 OPG eigenpairs through the FP64 Gram route.

Outputs are checked on stratified samples the oracle computes one by one:
blocks of the OPG whose rows and columns hit every weight and bias tensor,
full rows of G, and all 100 eigenpairs.
"""

import numpy as np
import pytest

from oracle import mlp as O
from synth import named_config

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


@pytest.fixture(scope="module")
def cfg():
    pb = named_config("mlp_1024_64_64_10")
    return pb, (f32(pb.omega), f32(pb.X), f32(pb.Y))


def stratified(widths, per_tensor, seed):
    """Parameter indices drawn from every weight matrix and bias vector."""
    rng = np.random.default_rng(seed)
    idx = []
    for j, (ow, ob) in enumerate(O.layer_offsets(widths)):
        t_out = widths[j + 1]
        idx.extend(rng.choice(np.arange(ow, ob), size=min(per_tensor, ob - ow), replace=False))
        idx.extend(rng.choice(np.arange(ob, ob + t_out), size=min(per_tensor // 4, t_out),
                              replace=False))
    return np.sort(np.asarray(idx, dtype=np.int64))


@pytest.mark.parametrize("prec,tol", [("bf16x3", 1e-5), ("bf16", 1e-2)])
def test_opg_sampled_blocks(hm, cfg, prec, tol):
    pb, (om, X, Y) = cfg
    S = stratified(pb.widths, 64, 1)
    T = stratified(pb.widths, 64, 2)
    GS = O.per_example_grads_columns(om, pb.widths, pb.acts, X, Y, S)
    GT = O.per_example_grads_columns(om, pb.widths, pb.acts, X, Y, T)
    net = hm.HessMLP(pb.widths, pb.acts, pb.omega)
    Xd = torch.as_tensor(pb.X, dtype=torch.float32, device="cuda")
    Yd = torch.as_tensor(pb.Y, dtype=torch.float32, device="cuda")
    OPG = net.opg(Xd, Yd, prec)
    s, t = torch.as_tensor(S, device="cuda"), torch.as_tensor(T, device="cuda")
    got_st = OPG[s][:, t].cpu().numpy()
    got_ss = OPG[s][:, s].cpu().numpy()
    got_ts = OPG[t][:, s].cpu().numpy()
    del OPG
    torch.cuda.empty_cache()
    assert relerr(got_st, GS.T @ GT / pb.N) <= tol
    assert relerr(got_ss, GS.T @ GS / pb.N) <= tol
    assert np.array_equal(got_ts, got_st.T)


def test_per_example_grads_fp32_rows(hm, cfg):
    pb, (om, X, Y) = cfg
    net = hm.HessMLP(pb.widths, pb.acts, pb.omega)
    Xd = torch.as_tensor(pb.X, dtype=torch.float32, device="cuda")
    Yd = torch.as_tensor(pb.Y, dtype=torch.float32, device="cuda")
    G = net.per_example_grads(Xd, Yd, "fp32")
    rows = [0, 4095, 8191]
    ref = O.per_example_grads(om, pb.widths, pb.acts, X[rows], Y[rows])
    assert relerr(G[rows].cpu().numpy(), ref) <= 1e-5


def test_top100_eigenpairs(hm, cfg):
    pb, (om, X, Y) = cfg
    k = 100
    net = hm.HessMLP(pb.widths, pb.acts, pb.omega)
    Xd = torch.as_tensor(pb.X, dtype=torch.float32, device="cuda")
    Yd = torch.as_tensor(pb.Y, dtype=torch.float32, device="cuda")
    ev, Q, st = net.opg_topk_eig(Xd, Yd, k, "fp32")
    assert st == 0
    ev, Q = ev.cpu().numpy(), Q.cpu().numpy()
    # the eigen path runs in FP64 from the FP32 inputs with the FP64 omega
    mu, Qr, deficient = O.opg_topk_eig_factored(pb.omega, pb.widths, pb.acts, X, Y, k)
    assert not deficient
    top = mu[0]
    assert np.all(np.abs(ev - mu) <= 1e-10 * top)
    f = O.forward(pb.omega, pb.widths, pb.acts, X)
    delta, _ = O.backprop(f, Y)
    GQ = O.grads_times(f, delta, pb.widths, Q.T)
    R = O.grads_transpose_times(f, delta, pb.widths, GQ) / pb.N - Q.T * ev[None, :]
    assert np.max(np.linalg.norm(R, axis=0)) <= 1e-8 * top
    assert np.allclose(Q @ Q.T, np.eye(k), atol=1e-8)
    for c in range(k):
        gaps = [abs(mu[c] - mu[j]) for j in (c - 1, c + 1) if 0 <= j < k]
        if min(gaps) > 1e-6 * top:
            assert abs(abs(Q[c] @ Qr[:, c]) - 1.0) <= 1e-7, c
