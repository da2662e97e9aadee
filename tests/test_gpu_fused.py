"""The fused call (hess_curvature): the OPG, exact Hessian and top-k OPG
eigenpairs scheduled across two streams give the same bits as the three
single calls -- at the benchmark workload in the benchmark's configuration,
with device, pinned-host and pageable-host buffers, and through the
sequential route of the other precisions."""

import numpy as np
import pytest

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


def _single(net, X, Y, prec, k):
    o = net.opg(X, Y, prec)
    h = net.exact_hessian(X, Y, prec)
    ev, Q, _ = net.opg_topk_eig(X, Y, k, prec)
    return o, h, ev, Q


@pytest.mark.parametrize("name,k", [("mlp_784_16_10", 32)])
def test_fused_equals_single_calls_at_benchmark_size(hm, name, k):
    pb = named_config(name)
    net = hm.HessMLP(pb.widths, pb.acts, pb.omega)
    X = torch.as_tensor(pb.X, dtype=torch.float32, device="cuda")
    Y = torch.as_tensor(pb.Y, dtype=torch.float32, device="cuda")
    o1, h1, ev1, Q1 = _single(net, X, Y, "bf16x3", k)
    o = torch.full_like(o1, float("nan"))
    h = torch.full_like(h1, float("nan"))
    ev = torch.empty_like(ev1)
    Q = torch.empty_like(Q1)
    net.curvature(X, Y, "bf16x3", opg=o, hessian=h, k=k, evals=ev, evecs=Q)
    torch.cuda.synchronize()
    assert torch.equal(o, o1) and torch.equal(h, h1)
    assert torch.equal(ev, ev1) and torch.equal(Q, Q1)


@pytest.mark.parametrize("blocks", [64, 100])
def test_fused_with_a_capped_lanczos_grid(hm, blocks):
    """With the eigen step's Lanczos kernel held to fewer blocks, the fused
    call queues its contractions behind the Gram matrix on the other SMs:
    still the same bits as the single calls on the same handle, and the
    eigenvalues of the default grid to rounding."""
    pb = named_config("mlp_784_16_10")
    k = 32
    X = torch.as_tensor(pb.X, dtype=torch.float32, device="cuda")
    Y = torch.as_tensor(pb.Y, dtype=torch.float32, device="cuda")
    ref = hm.HessMLP(pb.widths, pb.acts, pb.omega)
    ev0, _, _ = ref.opg_topk_eig(X, Y, k, "bf16x3")
    net = hm.HessMLP(pb.widths, pb.acts, pb.omega)
    net.set_eig_blocks(blocks)
    o1, h1, ev1, Q1 = _single(net, X, Y, "bf16x3", k)
    o = torch.full_like(o1, float("nan"))
    h = torch.full_like(h1, float("nan"))
    ev = torch.empty_like(ev1)
    Q = torch.empty_like(Q1)
    for _ in range(2):  # twice: the second call reuses the workspace and streams
        net.curvature(X, Y, "bf16x3", opg=o, hessian=h, k=k, evals=ev, evecs=Q)
        torch.cuda.synchronize()
        assert torch.equal(o, o1) and torch.equal(h, h1)
        assert torch.equal(ev, ev1) and torch.equal(Q, Q1)
    assert float((ev - ev0).abs().max()) <= 1e-12 * float(ev0[0])


def test_fused_with_host_buffers(hm):
    pb = make_problem([70, 33, 10], ["tanh"], 129, 7, "normal", "uniform")
    net = hm.HessMLP(pb.widths, pb.acts, pb.omega)
    Xd = torch.as_tensor(pb.X, dtype=torch.float32, device="cuda")
    Yd = torch.as_tensor(pb.Y, dtype=torch.float32, device="cuda")
    o1, h1, ev1, Q1 = _single(net, Xd, Yd, "bf16x3", 6)
    # pageable inputs, a pinned OPG (written in place), a pageable H
    Xh = np.ascontiguousarray(pb.X, dtype=np.float32)
    Yh = np.ascontiguousarray(pb.Y, dtype=np.float32)
    o = torch.full((pb.P, pb.P), float("nan"), pin_memory=True)
    h = np.full((pb.P, pb.P), np.nan, dtype=np.float32)
    ev = np.empty(6)
    Q = np.empty((6, pb.P))
    net.curvature(Xh, Yh, "bf16x3", opg=o, hessian=h, k=6, evals=ev, evecs=Q)
    assert torch.equal(o, o1.cpu()) and np.array_equal(h, h1.cpu().numpy())
    assert np.array_equal(ev, ev1.cpu().numpy()) and np.array_equal(Q, Q1.cpu().numpy())


@pytest.mark.parametrize("prec", ["fp32", "fp64"])
def test_fused_other_precisions_run_the_single_calls(hm, prec):
    pb = make_problem([13, 11, 7, 3], ["sigmoid", "relu"], 50, 4, "normal", "uniform")
    net = hm.HessMLP(pb.widths, pb.acts, pb.omega)
    dt = torch.float64 if prec == "fp64" else torch.float32
    X = torch.as_tensor(pb.X, dtype=dt, device="cuda")
    Y = torch.as_tensor(pb.Y, dtype=dt, device="cuda")
    o1, h1, ev1, Q1 = _single(net, X, Y, prec, 4)
    o, h = torch.empty_like(o1), torch.empty_like(h1)
    ev, Q = torch.empty_like(ev1), torch.empty_like(Q1)
    net.curvature(X, Y, prec, opg=o, hessian=h, k=4, evals=ev, evecs=Q)
    torch.cuda.synchronize()
    assert torch.equal(o, o1) and torch.equal(h, h1) and torch.equal(ev, ev1) and torch.equal(Q, Q1)


def test_fused_argument_errors(hm):
    pb = make_problem([6, 4], [], 10, 1, "normal", "uniform")
    net = hm.HessMLP(pb.widths, pb.acts, pb.omega)
    X = torch.as_tensor(pb.X, dtype=torch.float32, device="cuda")
    Y = torch.as_tensor(pb.Y, dtype=torch.float32, device="cuda")
    with pytest.raises(hm.HessError, match="no output"):
        net.curvature(X, Y, "bf16x3")
    ev = torch.empty(20, dtype=torch.float64, device="cuda")
    Q = torch.empty((20, pb.P), dtype=torch.float64, device="cuda")
    with pytest.raises(hm.HessError, match="min"):
        net.curvature(X, Y, "bf16x3", k=20, evals=ev, evecs=Q)
