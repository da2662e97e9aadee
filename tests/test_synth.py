"""The seeded input generator: published SplitMix64 values and the recipes."""

import numpy as np

from synth import NAMED_CONFIGS, SplitMix64Stream, make_random_mlp, named_config
from synth.inputs import GOLDEN, _mix_array, _mix_scalar


def test_splitmix64_reference_values():
    # SplitMix64 seeded with 0: the first two outputs are mix(1*GOLDEN), mix(2*GOLDEN)
    assert _mix_scalar(GOLDEN) == 0xE220A8397B1DCDAF
    assert _mix_scalar(2 * GOLDEN) == 0x6E789E6AA1B965F4
    z = np.array([GOLDEN, (2 * GOLDEN) & ((1 << 64) - 1)], dtype=np.uint64)
    assert [int(v) for v in _mix_array(z)] == [0xE220A8397B1DCDAF, 0x6E789E6AA1B965F4]


def test_stream_is_counter_based_and_deterministic():
    s1 = SplitMix64Stream(3, 7)
    a = np.concatenate([s1.uniform(5), s1.uniform(6)])
    b = SplitMix64Stream(3, 7).uniform(11)
    assert np.array_equal(a, b)
    assert not np.array_equal(b, SplitMix64Stream(3, 8).uniform(11))
    x = SplitMix64Stream(1, 1).normal(200000)
    assert abs(x.mean()) < 0.01 and abs(x.std() - 1) < 0.01
    u = SplitMix64Stream(1, 2).uniform(200000)
    assert u.min() >= 0 and u.max() < 1 and abs(u.mean() - 0.5) < 0.01


def test_named_configs_shapes():
    pb = named_config("mlp_4_5_3")
    assert pb.P == 43 and pb.X.shape == (100, 4) and pb.Y.shape == (100, 3)
    assert np.all(pb.Y.sum(axis=1) == 1)
    assert np.all(pb.omega[20:25] == 0)  # b^(2) is zero
    assert set(NAMED_CONFIGS) >= {"mlp_4_5_3", "mlp_784_16_10", "mlp_1024_64_64_10"}
    pb2 = named_config("mlp_784_16_10", N=8)
    assert pb2.P == 12730 and pb2.X.min() >= 0 and pb2.X.max() < 1


def test_random_mlp_distribution():
    for i in range(20):
        widths, acts, N = make_random_mlp(3, i)
        P = sum(widths[j] * widths[j + 1] + widths[j + 1] for j in range(len(widths) - 1))
        assert 500 <= P <= 20000 and 64 <= N <= 2048
        assert 2 <= len(widths) - 1 <= 4 and widths[-1] == 10
        assert len(acts) == len(widths) - 2
