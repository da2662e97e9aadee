"""Shared check of OPG eigenpairs against the oracle (used by several GPU tests).

Eigenvalues are compared to the oracle's relative to the largest one;
eigenvectors by |q . q_ref| when the eigenvalue is separated from its
neighbours by more than 1e-6 of the largest, and always by the residual of the
OPG eigen-equation, ||G^T G q / N - mu q|| <= 1e-8 mu_1, with the sign
convention (largest-magnitude entry positive).  Null eigenvalues
(mu <= 1e-13 mu_1) must come with zero eigenvector columns.
"""

import numpy as np

from oracle import mlp as O


def check_eig(evals, evecs, G_ref, k, val_tol, vec_tol):
    mu, Q, deficient = O.opg_topk_eig_from_grads(G_ref, k)
    top = mu[0]
    assert np.all(np.abs(evals - mu) <= val_tol * top), (evals, mu)
    N = G_ref.shape[0]
    for c in range(k):
        if not (mu[c] > 1e-13 * top):
            assert np.all(evecs[c] == 0)
            continue
        gaps = [abs(mu[c] - mu[j]) for j in (c - 1, c + 1) if 0 <= j < len(mu)]
        if not gaps or min(gaps) > 1e-6 * top:
            assert abs(abs(evecs[c] @ Q[:, c]) - 1.0) <= vec_tol, c
        q = evecs[c]
        r = G_ref.T @ (G_ref @ q) / N - evals[c] * q
        assert np.linalg.norm(r) <= 1e-8 * top, c
        i = int(np.argmax(np.abs(q)))
        assert q[i] > 0
    return deficient
