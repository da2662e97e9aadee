"""Writes hessian_top_eigs_mlp_784_16_10.txt: the 40 algebraically largest
eigenvalues of the exact Hessian of the 784-16-10 tanh network (P = 12730)
at its seeded parameters and N = 1024 seeded examples, from the FP64 oracle
(full H built from Hessian-vector products, Sec. 5.1; dense symmetric
eigensolver, Sec. 5.3).  Only the oracle and the seeded input generator are
called.  Takes a few minutes on a CPU.

    python tests/golden/make_hessian_top_eigs.py
"""

import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

from oracle import mlp as O  # noqa: E402
from synth import named_config  # noqa: E402

K = 40


def main():
    pb = named_config("mlp_784_16_10")
    lam, _ = O.hessian_topk_eig(pb.omega, pb.widths, pb.acts, pb.X, pb.Y, K)
    path = os.path.join(HERE, "hessian_top_eigs_mlp_784_16_10.txt")
    with open(path, "w") as fh:
        fh.write("# 40 largest (algebraic) eigenvalues of the exact Hessian, MLP [784, 16, 10] tanh,\n")
        fh.write("# P = 12730, N = 1024, seeded inputs of synth.named_config('mlp_784_16_10');\n")
        fh.write("# written by tests/golden/make_hessian_top_eigs.py from the FP64 oracle\n")
        for v in lam:
            fh.write(f"{float(v)!r}\n")
    print(path)


if __name__ == "__main__":
    main()
