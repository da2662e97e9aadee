"""Tile-width autotuning: tuned contractions give the results of the
cost-model widths (each output entry is the same sum over the same K blocks
whatever the tile width) and the table round-trips through a file."""

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
    return torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float32, device="cuda")


def relerr(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def test_tuned_widths_match_cost_model_widths(hm, tmp_path):
    pb = make_problem([300, 40, 24, 10], ["tanh", "relu"], 257, 21, "normal", "uniform")
    net = hm.HessMLP(pb.widths, pb.acts, pb.omega)
    X, Y = dev(pb.X), dev(pb.Y)
    ref_o = net.opg(X, Y, "bf16x3").cpu().numpy()
    ref_h = net.exact_hessian(X, Y, "bf16x3").cpu().numpy()
    n0 = hm.autotune_entries()
    hm.autotune(True)
    try:
        o = net.opg(X, Y, "bf16x3").cpu().numpy()
        h = net.exact_hessian(X, Y, "bf16x3").cpu().numpy()
    finally:
        hm.autotune(False)
    assert hm.autotune_entries() >= n0 + 3  # the SYRK and two Hessian shapes per layer
    assert relerr(o, ref_o) <= 1e-6 and relerr(h, ref_h) <= 1e-6
    assert np.array_equal(h, h.T)
    ref = O.hessian(np.float32(pb.omega).astype(np.float64), pb.widths, pb.acts,
                    np.float32(pb.X).astype(np.float64), np.float32(pb.Y).astype(np.float64))
    assert relerr(h, ref) <= 1e-5
    path = tmp_path / "tune.txt"
    hm.autotune_save(path)
    assert len([ln for ln in path.read_text().splitlines() if not ln.startswith("#")]) == hm.autotune_entries()
    hm.autotune_load(path)
