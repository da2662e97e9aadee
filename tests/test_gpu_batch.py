"""Batched OPG + exact Hessian of many networks (hess_batch_*).

* Small uneven networks against the FP64 oracle at the split-BF16 and BF16
  tolerances.
* Networks of the many-networks workload (2-4 weight layers, P from ~500 to
  20000, N from 64 to 2048): every matrix of a multi-wave batch, with one item
  too large for the workspace (run alone), is bit-identical to the
  single-network call.
* The chunked Hessian schedule (a small operand limit) gives the same bits as
  the one-launch schedule.
* CUDA-graph replay of a repeated item list gives the same bits as direct
  runs and reads the buffers' current contents.
"""

import numpy as np
import pytest

from oracle import mlp as O
from synth import make_problem
from synth.inputs import make_batch_problem

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


SMALL = [
    ([4, 5, 3], ["sigmoid"], 100, 0),
    ([20, 9, 10], ["tanh"], 77, 1),
    ([16, 8, 12, 10], ["relu", "sigmoid"], 130, 2),
    ([33, 10], [], 64, 3),
    ([24, 17, 9, 8, 10], ["tanh", "relu", "sigmoid"], 90, 4),
]


@pytest.mark.parametrize("prec", ["bf16x3", "bf16"])
def test_batch_small_networks_vs_oracle(hm, prec):
    pbs = [make_problem(w, a, n, s, "normal", "uniform") for (w, a, n, s) in SMALL]
    nets, items, outs = [], [], []
    for pb in pbs:
        net = hm.HessMLP(pb.widths, pb.acts, pb.omega)
        o = torch.full((pb.P, pb.P), float("nan"), device="cuda")
        h = torch.full((pb.P, pb.P), float("nan"), device="cuda")
        # OPG only, Hessian only and both, across the items
        k = len(items) % 3
        items.append((net, dev(pb.X), dev(pb.Y), o if k != 1 else None, h if k != 0 else None))
        nets.append(net)
        outs.append((o if k != 1 else None, h if k != 0 else None))
    b = hm.HessBatch(256 << 20)
    info = b.run(items, prec)
    assert info["waves"] == 1 and info["items_chunked"] == 0
    for pb, (o, h) in zip(pbs, outs):
        om, X, Y = f32(pb.omega), f32(pb.X), f32(pb.Y)
        if o is not None:
            ref = O.opg(om, pb.widths, pb.acts, X, Y)
            assert relerr(o.cpu().numpy(), ref) <= TOL[prec]
        if h is not None:
            ref = O.hessian(om, pb.widths, pb.acts, X, Y)
            assert relerr(h.cpu().numpy(), ref) <= TOL[prec]


def test_batch_waves_bit_identical_to_single_calls(hm):
    pbs = [make_batch_problem(3, i) for i in range(10)]
    nets = [hm.HessMLP(pb.widths, pb.acts, pb.omega) for pb in pbs]
    Xs = [dev(pb.X) for pb in pbs]
    Ys = [dev(pb.Y) for pb in pbs]
    outs = [(torch.full((pb.P, pb.P), float("nan"), device="cuda"),
             torch.full((pb.P, pb.P), float("nan"), device="cuda")) for pb in pbs]
    # a workspace that holds a few networks per wave but not the largest alone
    b = hm.HessBatch(3 << 30)
    info = b.run([(n, x, y, o, h) for n, x, y, (o, h) in zip(nets, Xs, Ys, outs)], "bf16x3")
    assert info["waves"] >= 2
    assert info["items_chunked"] >= 1
    for net, x, y, (o, h) in zip(nets, Xs, Ys, outs):
        o1 = net.opg(x, y, "bf16x3")
        assert torch.equal(o, o1)
        del o1
        h1 = net.exact_hessian(x, y, "bf16x3")
        assert torch.equal(h, h1)
        del h1
    b.close()


def test_chunked_hessian_matches_one_launch(hm):
    pb = make_problem([120, 40, 30, 10], ["tanh", "relu"], 300, 9, "normal", "uniform")
    net = hm.HessMLP(pb.widths, pb.acts, pb.omega)
    X, Y = dev(pb.X), dev(pb.Y)
    whole = net.exact_hessian(X, Y, "bf16x3")
    net.set_operand_limit(2 << 20)
    chunked = net.exact_hessian(X, Y, "bf16x3")
    assert torch.equal(whole, chunked)
    ref = O.hessian(f32(pb.omega), pb.widths, pb.acts, f32(pb.X), f32(pb.Y))
    assert relerr(chunked.cpu().numpy(), ref) <= TOL["bf16x3"]


def test_batch_rejects_bad_items(hm):
    pb = make_problem([6, 4], [], 10, 1, "normal", "uniform")
    net = hm.HessMLP(pb.widths, pb.acts, pb.omega)
    X, Y = dev(pb.X), dev(pb.Y)
    o = torch.empty((pb.P, pb.P), device="cuda")
    b = hm.HessBatch(128 << 20)
    with pytest.raises(hm.HessError, match="device memory"):
        b.run([(net, np.ascontiguousarray(pb.X, dtype=np.float32), Y, o, None)])
    with pytest.raises(hm.HessError, match="precision"):
        b.run([(net, X, Y, o, None)], "fp32")
    with pytest.raises(hm.HessError, match="no output"):
        b.run([(net, X, Y, None, None)])


def test_batch_graph_replay(hm):
    pbs = [make_problem(w, a, n, s, "normal", "uniform") for (w, a, n, s) in SMALL[:4]]
    nets = [hm.HessMLP(pb.widths, pb.acts, pb.omega) for pb in pbs]
    Xs = [dev(pb.X) for pb in pbs]
    Ys = [dev(pb.Y) for pb in pbs]
    outs = [(torch.empty((pb.P, pb.P), device="cuda"), torch.empty((pb.P, pb.P), device="cuda"))
            for pb in pbs]
    items = [(n, x, y, o, h) for n, x, y, (o, h) in zip(nets, Xs, Ys, outs)]
    direct = hm.HessBatch(256 << 20)
    direct.run(items, "bf16x3")
    ref = [(o.clone(), h.clone()) for o, h in outs]
    b = hm.HessBatch(256 << 20)
    b.set_graphs(True)
    infos = []
    for _ in range(3):  # direct, capture + launch, replay
        for o, h in outs:
            o.fill_(float("nan"))
            h.fill_(float("nan"))
        infos.append(b.run(items, "bf16x3"))
        for (o, h), (ro, rh) in zip(outs, ref):
            assert torch.equal(o, ro) and torch.equal(h, rh)
    assert [i["graph_replayed"] for i in infos] == [False, True, True]
    assert infos[2]["waves"] == infos[0]["waves"]
    # the graph reads the buffers' current contents
    Xs[0].mul_(0.5)
    b.run(items, "bf16x3")
    o2 = outs[0][0].clone()
    direct.run(items, "bf16x3")
    assert torch.equal(o2, outs[0][0]) and not torch.equal(o2, ref[0][0])
