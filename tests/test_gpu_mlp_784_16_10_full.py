"""Full-matrix parity at the benchmark workload.

The [784,16,10] tanh network with N = 1024 (P = 12730) is the configuration
the benchmark times.  Here every entry of the OPG (1.6e8 entries) and of the
exact Hessian is compared with the FP64 oracle -- the OPG as G^T G / N from
the oracle's per-example gradients (Eq. hesseq2/hesseq3), the Hessian from
the oracle's P unit-vector Hessian-vector products (Eq. hesseq1, Sec. 5.1),
computed over a pool of host processes -- for every precision, with the
bars of the other parity tests (relative Frobenius error: FP64 1e-12, FP32
and split-BF16x3 1e-5, BF16 1e-2; reduced precisions against the oracle at
the FP32-rounded inputs).  The fused call of the benchmark (OPG, Hessian and
the top-32 OPG eigenpairs in split-BF16x3) is checked against the oracle too:
its matrices in full and its eigenpairs (Sec. 5.4, Eq. J) with the bars of
the eigen tests.
"""

import numpy as np
import pytest

import oracle_pool
from eigcheck import check_eig
from oracle import mlp as O
from synth import named_config

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

TOL = {"fp64": 1e-12, "fp32": 1e-5, "bf16x3": 1e-5, "bf16": 1e-2}


@pytest.fixture(scope="module")
def hm():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1905_05559_gb300 import build
    build.build()
    import paper_1905_05559_gb300 as hm
    return hm


def _f32(a):
    return np.asarray(a, dtype=np.float32).astype(np.float64)


@pytest.fixture(scope="module")
def ref():
    """Oracle G, OPG and H at the FP64 inputs and at the FP32-rounded ones."""
    pb = named_config("mlp_784_16_10")
    out = {"pb": pb}
    for key, (om, X, Y) in (("64", (pb.omega, pb.X, pb.Y)), ("32", (_f32(pb.omega), _f32(pb.X), _f32(pb.Y)))):
        G = O.per_example_grads(om, pb.widths, pb.acts, X, Y)
        out["G" + key] = G
        out["OPG" + key] = O.opg_from_grads(G)
        out["H" + key] = oracle_pool.hessian(om, pb.widths, pb.acts, X, Y)
    return out


def _relerr(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def test_oracle_references_are_consistent(ref):
    """The pooled oracle H is the oracle's own columns (spot check) and both
    references are exactly symmetric to rounding."""
    pb = ref["pb"]
    cols = [0, 784, 12543, 12729]
    Hc = O.hessian_columns(pb.omega, pb.widths, pb.acts, pb.X, pb.Y, cols)
    assert np.array_equal(ref["H64"][:, cols], Hc)
    for key in ("64", "32"):
        H = ref["H" + key]
        assert np.linalg.norm(H - H.T) <= 1e-13 * np.linalg.norm(H)


@pytest.mark.parametrize("prec", ["fp64", "fp32", "bf16x3", "bf16"])
def test_full_opg_and_hessian(hm, ref, prec):
    pb = ref["pb"]
    key = "64" if prec == "fp64" else "32"
    dt = torch.float64 if prec == "fp64" else torch.float32
    net = hm.HessMLP(pb.widths, pb.acts, pb.omega)
    X = torch.as_tensor(pb.X, dtype=dt, device="cuda")
    Y = torch.as_tensor(pb.Y, dtype=dt, device="cuda")
    OPG = net.opg(X, Y, prec).cpu().numpy().astype(np.float64)
    e = _relerr(OPG, ref["OPG" + key])
    assert e <= TOL[prec], (prec, e)
    assert np.array_equal(OPG, OPG.T)
    del OPG
    H = net.exact_hessian(X, Y, prec).cpu().numpy().astype(np.float64)
    e = _relerr(H, ref["H" + key])
    assert e <= TOL[prec], (prec, e)
    assert np.array_equal(H, H.T)
    # every 128-column block (the tensor-core tile columns) on its own
    # against the block's own norm, or its share of the whole when smaller
    Href = ref["H" + key]
    share = np.linalg.norm(Href) * np.sqrt(128 / pb.P)
    for c0 in range(0, pb.P, 128):
        blk = slice(c0, min(pb.P, c0 + 128))
        eb = np.linalg.norm(H[:, blk] - Href[:, blk]) / max(np.linalg.norm(Href[:, blk]), share)
        assert eb <= 10 * TOL[prec], (prec, c0, eb)


def test_fused_bf16x3_matrices_and_eigenpairs(hm, ref):
    pb = ref["pb"]
    k = 32
    net = hm.HessMLP(pb.widths, pb.acts, pb.omega)
    X = torch.as_tensor(pb.X, dtype=torch.float32, device="cuda")
    Y = torch.as_tensor(pb.Y, dtype=torch.float32, device="cuda")
    o = torch.full((pb.P, pb.P), float("nan"), dtype=torch.float32, device="cuda")
    h = torch.full((pb.P, pb.P), float("nan"), dtype=torch.float32, device="cuda")
    ev = torch.empty(k, dtype=torch.float64, device="cuda")
    Q = torch.empty((k, pb.P), dtype=torch.float64, device="cuda")
    st = net.curvature(X, Y, "bf16x3", opg=o, hessian=h, k=k, evals=ev, evecs=Q)
    assert st == 0
    torch.cuda.synchronize()
    assert _relerr(o.cpu().numpy().astype(np.float64), ref["OPG32"]) <= TOL["bf16x3"]
    assert _relerr(h.cpu().numpy().astype(np.float64), ref["H32"]) <= TOL["bf16x3"]
    # the eigen step is FP64 on the FP32 inputs, with the FP64 parameters
    G = O.per_example_grads(pb.omega, pb.widths, pb.acts, _f32(pb.X), _f32(pb.Y))
    check_eig(ev.cpu().numpy(), Q.cpu().numpy(), G, k, 1e-10, 1e-7)
