"""The request server: requests in a concurrent mix give the same results as
the same calls made alone; admission refuses what can never fit and delays
what does not fit now."""

import numpy as np
import pytest

from synth import make_problem, make_random_mlp

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


def _nets():
    out = []
    for i in range(3):
        widths, acts, N = make_random_mlp(3, i)
        N = min(N, 512)
        out.append(make_problem(widths, acts, N, 40 + i, "normal", "uniform"))
    return out


def _alone(hm, pb, kind, prec, k):
    net = hm.HessMLP(pb.widths, pb.acts, pb.omega)
    dt = torch.float64 if prec == "fp64" else torch.float32
    X = torch.as_tensor(pb.X, dtype=dt, device="cuda")
    Y = torch.as_tensor(pb.Y, dtype=dt, device="cuda")
    if kind == "hessian":
        return net.exact_hessian(X, Y, prec)
    if kind == "opg":
        return net.opg(X, Y, prec)
    ev, Q, _ = net.opg_topk_eig(X, Y, k, prec)
    return Q


def test_mix_equals_alone(hm):
    nets = _nets()
    srv = hm.HessServer(slots=3, budget_bytes=40 << 30)
    ids = [srv.add_network(pb.widths, pb.acts, pb.omega) for pb in nets]
    jobs = []
    for rep in range(2):
        for i, pb in enumerate(nets):
            for kind, prec in (("hessian", "bf16x3"), ("opg", "bf16x3"), ("eig", "fp32"), ("opg", "fp64")):
                dt = torch.float64 if prec == "fp64" else torch.float32
                X = torch.as_tensor(pb.X, dtype=dt, device="cuda")
                Y = torch.as_tensor(pb.Y, dtype=dt, device="cuda")
                if kind == "eig":
                    out = torch.empty((8, pb.P), dtype=torch.float64, device="cuda")
                    ev = torch.empty(8, dtype=torch.float64, device="cuda")
                    t = srv.submit(kind, ids[i], X, Y, prec, out, k=8, evals=ev)
                else:
                    out = torch.empty((pb.P, pb.P), dtype=dt, device="cuda")
                    t = srv.submit(kind, ids[i], X, Y, prec, out)
                jobs.append((t, i, kind, prec, out))
    for t, i, kind, prec, out in jobs:
        assert srv.wait(t, 120.0) == 0
    for t, i, kind, prec, out in jobs:
        ref = _alone(hm, nets[i], kind, prec, 8)
        assert torch.equal(out, ref), (kind, prec, i)
    srv.close()


def test_admission(hm):
    pb = _nets()[0]
    srv = hm.HessServer(slots=2, budget_bytes=1 << 20)  # 1 MiB: nothing fits
    nid = srv.add_network(pb.widths, pb.acts, pb.omega)
    X = torch.as_tensor(pb.X, dtype=torch.float32, device="cuda")
    Y = torch.as_tensor(pb.Y, dtype=torch.float32, device="cuda")
    out = torch.empty((pb.P, pb.P), device="cuda")
    with pytest.raises(hm.HessError) as e:
        srv.submit("hessian", nid, X, Y, "bf16x3", out)
    assert e.value.status == 7
    srv.close()
    # a budget that holds one request's workspace at a time: all still finish
    lib = hm.load()
    srv = hm.HessServer(slots=3, budget_bytes=int(1.2 * _plan(hm, pb)))
    nid = srv.add_network(pb.widths, pb.acts, pb.omega)
    outs = [torch.empty((pb.P, pb.P), device="cuda") for _ in range(4)]
    ts = [srv.submit("hessian", nid, X, Y, "bf16x3", o) for o in outs]
    assert all(srv.wait(t, 120.0) == 0 for t in ts)
    for o in outs[1:]:
        assert torch.equal(o, outs[0])
    srv.close()
    del lib


def _plan(hm, pb):
    """Workspace of one bf16x3 Hessian request, found by shrinking budgets."""
    X = torch.as_tensor(pb.X, dtype=torch.float32, device="cuda")
    Y = torch.as_tensor(pb.Y, dtype=torch.float32, device="cuda")
    out = torch.empty((pb.P, pb.P), device="cuda")
    lo, hi = 1 << 20, 64 << 30
    while hi - lo > (1 << 20):
        mid = (lo + hi) // 2
        srv = hm.HessServer(slots=1, budget_bytes=mid)
        nid = srv.add_network(pb.widths, pb.acts, pb.omega)
        try:
            t = srv.submit("hessian", nid, X, Y, "bf16x3", out)
            srv.wait(t, 120.0)
            hi = mid
        except hm.HessError:
            lo = mid
        srv.close()
    return hi


def test_concurrent_eigen_requests_of_different_sizes(hm):
    # eigen requests with different N run on several slots at once; each
    # must succeed (a per-call kernel attribute would race between slots)
    pbs = []
    for i in range(6):
        widths, acts, N = make_random_mlp(5, i)
        pbs.append(make_problem(widths, acts, min(N, 700) + 37 * i, 60 + i, "normal", "uniform"))
    srv = hm.HessServer(slots=4, budget_bytes=40 << 30)
    ids = [srv.add_network(pb.widths, pb.acts, pb.omega) for pb in pbs]
    jobs = []
    for rep in range(3):
        for i, pb in enumerate(pbs):
            X = torch.as_tensor(pb.X, dtype=torch.float32, device="cuda")
            Y = torch.as_tensor(pb.Y, dtype=torch.float32, device="cuda")
            out = torch.empty((16, pb.P), dtype=torch.float64, device="cuda")
            ev = torch.empty(16, dtype=torch.float64, device="cuda")
            jobs.append((i, srv.submit("eig", ids[i], X, Y, "fp32", out, k=16, evals=ev), out, ev))
    results = {}
    for i, t, out, ev in jobs:
        assert srv.wait(t) in (0, 4), hm.last_error()
        results.setdefault(i, []).append((ev.cpu().numpy(), out.cpu().numpy()))
    srv.close()
    for i, runs in results.items():
        ref = _alone(hm, pbs[i], "eig", "fp32", 16).cpu().numpy()
        for ev, Q in runs:
            assert np.array_equal(ev, runs[0][0]) and np.array_equal(Q, ref)
