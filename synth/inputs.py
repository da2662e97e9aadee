"""Counter-based seeded generator and the synthetic workload recipes.

Random bits come from SplitMix64 (Steele, Lea and Flood, "Fast splittable
pseudorandom number generators", OOPSLA 2014) used in counter mode: draw i of
stream (seed, sid) is mix(key(seed, sid) + (i + 1) * GOLDEN).  Uniform doubles
take the top 53 bits; normals use the Box-Muller transform on a pair of
uniforms.  The bit stream is defined here, once, so parity never depends on
another library's generator or version.

Workloads follow the dense feed-forward network of the paper (Sec. 2): widths
T_1..T_L, hidden activations, softmax output, one-hot labels.  The parameter
vector omega is laid out layer by layer as W^(l-1) (T_l x T_{l-1}, row-major)
followed by b^(l), for l = 2..L (Sec. 2, Eq. flatten).
"""

from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

MASK64 = (1 << 64) - 1
GOLDEN = 0x9E3779B97F4A7C15
_M1 = 0xBF58476D1CE4E5B9
_M2 = 0x94D049BB133111EB

# stream ids: one per random quantity, so that changing one size never shifts
# the bits of another quantity
SID_X = 1
SID_LABELS = 2
SID_W = 100
SID_B = 200
SID_STRUCT = 300


def _mix_scalar(z: int) -> int:
    z &= MASK64
    z = ((z ^ (z >> 30)) * _M1) & MASK64
    z = ((z ^ (z >> 27)) * _M2) & MASK64
    return z ^ (z >> 31)


def _mix_array(z: np.ndarray) -> np.ndarray:
    z = z.astype(np.uint64, copy=True)
    with np.errstate(over="ignore"):
        z ^= z >> np.uint64(30)
        z *= np.uint64(_M1)
        z ^= z >> np.uint64(27)
        z *= np.uint64(_M2)
        z ^= z >> np.uint64(31)
    return z


class SplitMix64Stream:
    """Counter-mode SplitMix64 stream identified by (seed, sid)."""

    def __init__(self, seed: int, sid: int):
        self.key = _mix_scalar((seed * GOLDEN) ^ (sid * 0xD1B54A32D192ED03))
        self.pos = 0

    def bits(self, n: int) -> np.ndarray:
        idx = np.arange(self.pos + 1, self.pos + n + 1, dtype=np.uint64)
        self.pos += n
        with np.errstate(over="ignore"):
            z = np.uint64(self.key) + idx * np.uint64(GOLDEN)
        return _mix_array(z)

    def uniform(self, n: int) -> np.ndarray:
        """n doubles in [0, 1) from the top 53 bits."""
        return (self.bits(n) >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)

    def normal(self, n: int) -> np.ndarray:
        """n standard normals; normal i uses uniforms 2i and 2i+1 (Box-Muller)."""
        u = self.uniform(2 * n)
        u1 = 1.0 - u[0::2]  # in (0, 1]
        u2 = u[1::2]
        return np.sqrt(-2.0 * np.log(u1)) * np.cos(2.0 * math.pi * u2)

    def integers(self, n: int, lo: int, hi: int) -> np.ndarray:
        """n integers uniform in [lo, hi] (inclusive)."""
        u = self.uniform(n)
        return lo + np.minimum(np.floor(u * (hi - lo + 1)), hi - lo).astype(np.int64)


ACT_NAMES = ("sigmoid", "tanh", "relu")


@dataclass
class Problem:
    widths: list
    acts: list  # L-2 hidden activation names
    omega: np.ndarray  # (P,) float64
    X: np.ndarray  # (N, T_1) float64
    Y: np.ndarray  # (N, T_L) float64 one-hot
    labels: np.ndarray  # (N,) int64
    meta: dict = field(default_factory=dict)

    @property
    def N(self) -> int:
        return int(self.X.shape[0])

    @property
    def P(self) -> int:
        return int(self.omega.shape[0])


def make_mlp(widths, seed: int, bias: str = "zero") -> np.ndarray:
    """Glorot-uniform weights (limit sqrt(6/(fan_in+fan_out))) and biases.

    bias = "zero" (the workloads) or "uniform" (U(-0.5, 0.5), used by tests so
    that bias coordinates are exercised at a generic point).
    """
    parts = []
    for l in range(1, len(widths)):
        fan_in, fan_out = widths[l - 1], widths[l]
        lim = math.sqrt(6.0 / (fan_in + fan_out))
        w = (2.0 * SplitMix64Stream(seed, SID_W + l).uniform(fan_in * fan_out) - 1.0) * lim
        if bias == "zero":
            b = np.zeros(fan_out)
        elif bias == "uniform":
            b = SplitMix64Stream(seed, SID_B + l).uniform(fan_out) - 0.5
        else:
            raise ValueError(bias)
        parts.append(w)
        parts.append(b)
    return np.concatenate(parts).astype(np.float64)


def make_problem(widths, acts, N: int, seed: int, x_dist: str = "normal",
                 bias: str = "zero") -> Problem:
    widths = [int(t) for t in widths]
    if len(acts) != len(widths) - 2:
        raise ValueError("need one activation per hidden layer")
    omega = make_mlp(widths, seed, bias)
    T1, TL = widths[0], widths[-1]
    sx = SplitMix64Stream(seed, SID_X)
    if x_dist == "normal":
        X = sx.normal(N * T1)
    elif x_dist == "uniform":
        X = sx.uniform(N * T1)
    else:
        raise ValueError(x_dist)
    X = X.reshape(N, T1)
    labels = SplitMix64Stream(seed, SID_LABELS).integers(N, 0, TL - 1)
    Y = np.zeros((N, TL))
    Y[np.arange(N), labels] = 1.0
    return Problem(widths, list(acts), omega, X, Y, labels,
                   meta={"seed": seed, "x_dist": x_dist, "bias": bias})


# The workloads: sizes, distributions and seeds of the curvature configurations.
NAMED_CONFIGS = {
    # [4,5,3] sigmoid, P=43, N=100, x~N(0,1), seed 0
    "mlp_4_5_3": dict(widths=[4, 5, 3], acts=["sigmoid"], N=100, seed=0, x_dist="normal"),
    # [784,16,10] tanh, P=12730, N=1024, x~U[0,1], seed 1
    "mlp_784_16_10": dict(widths=[784, 16, 10], acts=["tanh"], N=1024, seed=1, x_dist="uniform"),
    # [1024,64,64,10] ReLU, P=70410, N=8192, x~N(0,1), seed 2
    "mlp_1024_64_64_10": dict(widths=[1024, 64, 64, 10], acts=["relu", "relu"], N=8192, seed=2,
                              x_dist="normal"),
}


def named_config(name: str, N: int | None = None, bias: str = "zero") -> Problem:
    c = dict(NAMED_CONFIGS[name])
    if N is not None:
        c["N"] = N
    return make_problem(c["widths"], c["acts"], c["N"], c["seed"], c["x_dist"], bias)


def make_random_mlp(seed: int, index: int, p_lo: int = 500, p_hi: int = 20000):
    """One network of the batching distribution: 2-4 weight layers, hidden
    widths uniform in [8,128], input width in [16,512], 10 classes, hidden
    activation uniform over sigmoid/tanh/ReLU, N uniform in [64,2048]; the whole
    draw is repeated until p_lo <= P <= p_hi.  Returns (widths, acts, N).
    """
    s = SplitMix64Stream(seed, SID_STRUCT + index)
    while True:
        nl = int(s.integers(1, 2, 4)[0])  # weight layers
        t1 = int(s.integers(1, 16, 512)[0])
        hidden = [int(v) for v in s.integers(nl - 1, 8, 128)] if nl > 1 else []
        widths = [t1] + hidden + [10]
        acts = [ACT_NAMES[int(v)] for v in s.integers(nl - 1, 0, 2)] if nl > 1 else []
        N = int(s.integers(1, 64, 2048)[0])
        P = sum(widths[i] * widths[i + 1] + widths[i + 1] for i in range(len(widths) - 1))
        if p_lo <= P <= p_hi:
            return widths, acts, N



def make_batch_problem(seed: int, index: int) -> Problem:
    """Network `index` of the many-networks workload drawn with `seed`: the
    structure and N from make_random_mlp(seed, index), then a problem with
    x ~ N(0,1), uniform labels over 10 classes and Glorot weights, all from the
    seed seed * 100000 + index."""
    widths, acts, N = make_random_mlp(seed, index)
    return make_problem(widths, acts, N, seed * 100000 + index, "normal", "zero")
