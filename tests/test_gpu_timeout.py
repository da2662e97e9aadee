"""The bounded grid-barrier wait of the OPG eigen step gives up cleanly.

Each block of the cooperative Lanczos kernel waits at a grid barrier for at
most a fixed number of clock cycles; when the wait runs out, the block sets an
error flag, the kernel stops, and the call returns HESS_ERR_TIMEOUT.  The test
shortens that limit to one cycle through the library's test hook (so a wait
runs out at once: nothing is made to fault or hang), checks the status, then
restores the default and checks that the next call on the same handle gives
the oracle's eigenpairs.
"""

import pytest

from eigcheck import check_eig
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


def test_lanczos_barrier_timeout_then_recovery(hm):
    from paper_1905_05559_gb300 import _lib
    lib = hm.load()
    pb = make_problem([64, 16, 10], ["tanh"], 600, 11, "normal", "uniform")
    k = 8
    net = hm.HessMLP(pb.widths, pb.acts, pb.omega)
    X = torch.as_tensor(pb.X, device="cuda")
    Y = torch.as_tensor(pb.Y, device="cuda")
    try:
        assert lib.hess_debug_set_barrier_limit(1) == 0
        with pytest.raises(hm.HessError) as ei:
            net.opg_topk_eig(X, Y, k, "fp64")
        assert ei.value.status == _lib.HESS_ERR_TIMEOUT
        assert "barrier" in str(ei.value)
    finally:
        lib.hess_debug_set_barrier_limit(0)
    ev, Q, _ = net.opg_topk_eig(X, Y, k, "fp64")
    Gr = O.per_example_grads(pb.omega, pb.widths, pb.acts, pb.X, pb.Y)
    check_eig(ev.cpu().numpy(), Q.cpu().numpy(), Gr, k, 1e-10, 1e-8)
