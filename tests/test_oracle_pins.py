"""Pins of the FP64 oracle against facts outside itself (CPU only).

Each test ties an oracle function to something it does not compute itself:
sizes printed in the paper, finite differences of the cost, the closed form of
a single softmax layer, and invariants fixed by the mathematics.  The mutation
tests at the end plant plausible mistakes in the oracle and check that a pin
catches each of them.
"""

import os

import numpy as np
import pytest

from oracle import mlp as O
from synth import make_problem

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _tiny(widths, acts, N=7, seed=11, bias="uniform"):
    return make_problem(widths, acts, N, seed, "normal", bias)


def _relerr(a, b):
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)


def _fd_grad_per_example(pb, h=1e-4):
    """Richardson-extrapolated central differences of every C_n."""
    P = pb.P
    out = np.empty((pb.N, P))

    def d(hh, j):
        w1 = pb.omega.copy()
        w2 = pb.omega.copy()
        w1[j] += hh
        w2[j] -= hh
        c1 = O.per_example_costs(w1, pb.widths, pb.acts, pb.X, pb.Y)
        c2 = O.per_example_costs(w2, pb.widths, pb.acts, pb.X, pb.Y)
        return (c1 - c2) / (2 * hh)

    for j in range(P):
        out[:, j] = (4 * d(h / 2, j) - d(h, j)) / 3
    return out


def _fd_hessian_of_gradient(pb, h=1e-5):
    P = pb.P
    H = np.empty((P, P))
    for j in range(P):
        w1 = pb.omega.copy()
        w2 = pb.omega.copy()
        w1[j] += h
        w2[j] -= h
        g1 = O.gradient(w1, pb.widths, pb.acts, pb.X, pb.Y)
        g2 = O.gradient(w2, pb.widths, pb.acts, pb.X, pb.Y)
        H[:, j] = (g1 - g2) / (2 * h)
    return H


def _min_abs_preact(pb):
    f = O.forward(pb.omega, pb.widths, pb.acts, pb.X)
    return min(np.abs(z).min() for z in f["z"][1:-1]) if len(pb.widths) > 2 else np.inf


# ---------------------------------------------------------------- sizes ----

def _golden_sizes():
    rows = []
    with open(os.path.join(GOLDEN, "paper_sizes.txt")) as fh:
        for line in fh:
            line = line.split("--")[0].strip()
            if not line or line.startswith("#"):
                continue
            key, widths, val = line.split()
            rows.append((key, [int(t) for t in widths.split(",")], int(val)))
    return rows


def test_parameter_count_matches_paper():
    rows = [r for r in _golden_sizes() if r[0] == "P"]
    assert len(rows) >= 4
    for _, widths, P in rows:
        assert O.num_params(widths) == P
        omega = np.arange(P, dtype=np.float64)
        assert np.array_equal(O.flatten(O.unflatten(omega, widths)), omega)


def test_hessian_block_shapes_match_paper():
    """Sec. 3.3: for the 64->32 softmax layer, the W-W block is 2048 x 2048 and
    the b-b block 32 x 32; the off-diagonal (W, b) blocks are what the per-tensor
    routine misses, and they are not zero."""
    sizes = {r[0]: r[2] for r in _golden_sizes() if r[1] == [64, 32]}
    pb = make_problem([64, 32], [], 3, 5, "normal", "uniform")
    cols = [0, 1, 2047, 2048, 2079]
    Hc = O.hessian_columns(pb.omega, pb.widths, pb.acts, pb.X, pb.Y, cols)
    nW, nb = sizes["HU"], sizes["HL"]
    assert nW + nb == sizes["P"] == pb.P
    # column 0 is a weight direction: it has nonzero entries in the bias rows
    assert np.abs(Hc[nW:, 0]).max() > 1e-6
    # column 2048 is a bias direction: it has nonzero entries in the weight rows
    assert np.abs(Hc[:nW, 3]).max() > 1e-6


# ------------------------------------------------------------ forward ----

def test_cost_zero_network_is_log_classes():
    widths = [5, 4, 6]
    pb = make_problem(widths, ["tanh"], 9, 3, "normal")
    omega = np.zeros(pb.P)
    assert abs(O.cost(omega, widths, pb.acts, pb.X, pb.Y) - np.log(6.0)) < 1e-15


def test_cost_matches_cross_entropy_of_softmax():
    pb = _tiny([4, 6, 5], ["sigmoid"])
    f = O.forward(pb.omega, pb.widths, pb.acts, pb.X)
    zL = f["z"][-1]
    yhat = np.exp(zL) / np.exp(zL).sum(axis=1, keepdims=True)
    naive = -(pb.Y * np.log(yhat)).sum(axis=1)
    assert _relerr(O.per_example_costs(pb.omega, pb.widths, pb.acts, pb.X, pb.Y), naive) < 1e-14
    # a hand evaluation of the network for example 0
    params = O.unflatten(pb.omega, pb.widths)
    x = pb.X[0]
    h = 1.0 / (1.0 + np.exp(-(params[0][0] @ x + params[0][1])))
    z = params[1][0] @ h + params[1][1]
    c0 = -np.log(np.exp(z[pb.labels[0]]) / np.exp(z).sum())
    assert abs(naive[0] - c0) < 1e-13


# -------------------------------------------------------- first order ----

@pytest.mark.parametrize("act", ["sigmoid", "tanh", "relu"])
def test_per_example_grads_match_finite_differences(act):
    pb = _tiny([3, 4, 3, 3], [act, act])
    assert _min_abs_preact(pb) > 1e-3
    G = O.per_example_grads(pb.omega, pb.widths, pb.acts, pb.X, pb.Y)
    Gfd = _fd_grad_per_example(pb)
    assert _relerr(G, Gfd) < 1e-9


def test_single_layer_gradient_closed_form():
    """L = 2: g_n = (p_n - y_n) (x) [x_n; 1] in augmented-row order."""
    pb = _tiny([5, 4], [])
    G = O.per_example_grads(pb.omega, pb.widths, pb.acts, pb.X, pb.Y)
    f = O.forward(pb.omega, pb.widths, pb.acts, pb.X)
    perm = O.param_permutation(pb.widths)
    xt = np.hstack([pb.X, np.ones((pb.N, 1))])
    for n in range(pb.N):
        ref = np.kron(f["p"][n] - pb.Y[n], xt[n])
        assert np.allclose(G[n, perm], ref, rtol=0, atol=1e-15)


def test_per_example_rows_versus_summed_gradient():
    """The summed gradient is the mean of the per-example rows, and each row
    equals the gradient of the single-example cost (Sec. 3.1)."""
    pb = _tiny([4, 3, 3], ["tanh"], N=5)
    G = O.per_example_grads(pb.omega, pb.widths, pb.acts, pb.X, pb.Y)
    for n in range(pb.N):
        gn = O.gradient(pb.omega, pb.widths, pb.acts, pb.X[n:n + 1], pb.Y[n:n + 1])
        assert _relerr(G[n], gn) < 1e-15
    h = 1e-5
    fd = np.empty(pb.P)
    for j in range(pb.P):
        w1, w2 = pb.omega.copy(), pb.omega.copy()
        w1[j] += h
        w2[j] -= h
        fd[j] = (O.cost(w1, pb.widths, pb.acts, pb.X, pb.Y)
                 - O.cost(w2, pb.widths, pb.acts, pb.X, pb.Y)) / (2 * h)
    assert _relerr(G.mean(axis=0), fd) < 1e-8


# ------------------------------------------------------- second order ----

@pytest.mark.parametrize("act", ["sigmoid", "tanh", "relu"])
def test_hessian_matches_finite_differences_of_gradient(act):
    pb = _tiny([3, 4, 3, 3], [act, act], N=6, seed=21)
    assert _min_abs_preact(pb) > 1e-3
    H = O.hessian(pb.omega, pb.widths, pb.acts, pb.X, pb.Y)
    Hfd = _fd_hessian_of_gradient(pb)
    assert _relerr(H, Hfd) < 1e-8


def test_hessian_matches_second_differences_of_cost():
    """Independent of the back-propagation code: second central differences of
    the scalar cost C itself."""
    pb = _tiny([3, 3, 2], ["sigmoid"], N=4, seed=5)
    H = O.hessian(pb.omega, pb.widths, pb.acts, pb.X, pb.Y)
    h = 1e-4
    P = pb.P
    Hfd = np.empty((P, P))

    def C(w):
        return O.cost(w, pb.widths, pb.acts, pb.X, pb.Y)

    for i in range(P):
        for j in range(P):
            s = 0.0
            for si, sj, sg in ((1, 1, 1), (1, -1, -1), (-1, 1, -1), (-1, -1, 1)):
                w = pb.omega.copy()
                w[i] += si * h
                w[j] += sj * h
                s += sg * C(w)
            Hfd[i, j] = s / (4 * h * h)
    assert _relerr(H, Hfd) < 1e-5


def test_single_softmax_layer_closed_form():
    """L = 2: H = (1/N) sum_n (diag p_n - p_n p_n^T) (x) xt_n xt_n^T with
    xt = [x; 1], in augmented-row order."""
    pb = _tiny([6, 5], [], N=9, seed=3)
    H = O.hessian(pb.omega, pb.widths, pb.acts, pb.X, pb.Y)
    f = O.forward(pb.omega, pb.widths, pb.acts, pb.X)
    xt = np.hstack([pb.X, np.ones((pb.N, 1))])
    ref = np.zeros((pb.P, pb.P))
    for n in range(pb.N):
        p = f["p"][n]
        ref += np.kron(np.diag(p) - np.outer(p, p), np.outer(xt[n], xt[n]))
    ref /= pb.N
    perm = O.param_permutation(pb.widths)
    assert _relerr(H[np.ix_(perm, perm)], ref) < 1e-13


def test_hessian_symmetry_and_hvp_reciprocity():
    pb = _tiny([4, 5, 4, 3], ["tanh", "sigmoid"], N=8, seed=9)
    H = O.hessian(pb.omega, pb.widths, pb.acts, pb.X, pb.Y)
    assert np.linalg.norm(H - H.T) / np.linalg.norm(H) < 1e-14
    rng = np.random.default_rng(0)
    u, v = rng.standard_normal(pb.P), rng.standard_normal(pb.P)
    Hu = O.hvp(pb.omega, pb.widths, pb.acts, pb.X, pb.Y, u)
    Hv = O.hvp(pb.omega, pb.widths, pb.acts, pb.X, pb.Y, v)
    assert abs(u @ Hv - v @ Hu) <= 1e-13 * np.linalg.norm(Hu) * np.linalg.norm(v)
    assert np.allclose(Hv, H @ v, rtol=0, atol=1e-13 * np.linalg.norm(Hv))


def test_hvp_matches_directional_difference_of_gradient():
    """H v = d/dr grad C(omega + r v) at r = 0, by Richardson-extrapolated
    central differences of the (separately pinned) gradient along v."""
    pb = _tiny([5, 6, 4, 3], ["sigmoid", "tanh"], N=7, seed=21)
    rng = np.random.default_rng(5)
    v = rng.standard_normal(pb.P)

    def d(h):
        g1 = O.gradient(pb.omega + h * v, pb.widths, pb.acts, pb.X, pb.Y)
        g2 = O.gradient(pb.omega - h * v, pb.widths, pb.acts, pb.X, pb.Y)
        return (g1 - g2) / (2 * h)

    fd = (4 * d(5e-4) - d(1e-3)) / 3
    assert _relerr(O.hvp(pb.omega, pb.widths, pb.acts, pb.X, pb.Y, v), fd) < 1e-9


def _shift_null_vectors(widths):
    """Softmax is invariant to adding a constant to all logits (Sec. 2), so the
    direction that adds 1 to every output bias and, for each input unit r of the
    last layer, the direction adding 1 to column r of every row of W^(L-1) leave
    every C_n unchanged."""
    offs = O.layer_offsets(widths)
    ow, ob = offs[-1]
    t_in, t_out = widths[-2], widths[-1]
    P = O.num_params(widths)
    vecs = []
    u = np.zeros(P)
    u[ob:ob + t_out] = 1.0
    vecs.append(u)
    for r in range(t_in):
        u = np.zeros(P)
        for i in range(t_out):
            u[ow + i * t_in + r] = 1.0
        vecs.append(u)
    return vecs


def test_softmax_shift_null_space():
    pb = _tiny([4, 5, 3], ["tanh"], N=6, seed=2)
    H = O.hessian(pb.omega, pb.widths, pb.acts, pb.X, pb.Y)
    Gm = O.opg(pb.omega, pb.widths, pb.acts, pb.X, pb.Y)
    for u in _shift_null_vectors(pb.widths):
        assert np.linalg.norm(H @ u) <= 1e-14 * np.linalg.norm(H) * np.linalg.norm(u)
        assert np.linalg.norm(Gm @ u) <= 1e-14 * np.linalg.norm(Gm) * np.linalg.norm(u)


# --------------------------------------------------------------- OPG ----

def test_opg_invariants():
    pb = _tiny([5, 6, 4], ["sigmoid"], N=9, seed=4)
    G = O.per_example_grads(pb.omega, pb.widths, pb.acts, pb.X, pb.Y)
    M = O.opg_from_grads(G)
    assert np.linalg.norm(M - M.T) == 0.0 or np.linalg.norm(M - M.T) < 1e-15 * np.linalg.norm(M)
    ev = np.linalg.eigvalsh(M)
    assert ev.min() >= -1e-12 * ev.max()
    assert abs(np.trace(M) - (G * G).sum(axis=1).mean()) < 1e-13 * np.trace(M)
    rank = int((ev > 1e-10 * ev.max()).sum())
    assert rank <= min(pb.N, pb.P - (pb.widths[-2] + 1))
    # explicit sum of per-example outer products (Eq. hesseq2)
    ref = sum(np.outer(G[n], G[n]) for n in range(pb.N)) / pb.N
    assert _relerr(M, ref) < 1e-15
    # one example: OPG = g g^T
    g1 = O.per_example_grads(pb.omega, pb.widths, pb.acts, pb.X[:1], pb.Y[:1])[0]
    assert _relerr(O.opg(pb.omega, pb.widths, pb.acts, pb.X[:1], pb.Y[:1]), np.outer(g1, g1)) < 1e-15


def test_opg_is_not_gradient_outer_product():
    """Eq. hesseq4: the OPG differs from grad C grad C^T for N > 1."""
    pb = _tiny([3, 3, 3], ["tanh"], N=6)
    G = O.per_example_grads(pb.omega, pb.widths, pb.acts, pb.X, pb.Y)
    g = G.mean(axis=0)
    assert _relerr(O.opg_from_grads(G), np.outer(g, g)) > 0.1


# --------------------------------------------------------------- eig ----

def test_gram_routes_agree():
    pb = _tiny([6, 5, 4, 3], ["relu", "tanh"], N=10, seed=8)
    G = O.per_example_grads(pb.omega, pb.widths, pb.acts, pb.X, pb.Y)
    assert _relerr(O.gram_factored(pb.omega, pb.widths, pb.acts, pb.X, pb.Y),
                   O.gram_from_grads(G)) < 1e-14


def test_opg_topk_eig_against_full_eigendecomposition():
    pb = _tiny([6, 5, 4], ["tanh"], N=12, seed=6)
    G = O.per_example_grads(pb.omega, pb.widths, pb.acts, pb.X, pb.Y)
    OPG = O.opg_from_grads(G)
    k = 5
    mu, Q, deficient = O.opg_topk_eig_from_grads(G, k)
    assert not deficient
    lam, V = np.linalg.eigh(OPG)
    lam, V = lam[::-1], V[:, ::-1]
    assert np.allclose(mu, lam[:k], rtol=0, atol=1e-13 * lam[0])
    assert np.all(np.diff(mu) <= 0)
    for c in range(k):
        assert abs(abs(Q[:, c] @ V[:, c]) - 1.0) < 1e-10
        assert np.linalg.norm(OPG @ Q[:, c] - mu[c] * Q[:, c]) < 1e-12 * lam[0]
        assert Q[np.argmax(np.abs(Q[:, c])), c] > 0
    assert np.allclose(Q.T @ Q, np.eye(k), atol=1e-12)
    mu_all, _, _ = O.opg_topk_eig_from_grads(G, pb.N)
    assert abs(mu_all.sum() - np.trace(OPG)) < 1e-12 * np.trace(OPG)


def test_opg_eig_direct_route_matches_gram_route():
    """The P x P route (eigendecomposition of the OPG itself) gives the Gram
    route's eigenpairs (Eq. J): the same values and, for separated values,
    the same vectors."""
    pb = _tiny([7, 6, 4], ["sigmoid"], N=15, seed=12)
    lg, Qg, _ = O.opg_topk_eig(pb.omega, pb.widths, pb.acts, pb.X, pb.Y, 6)
    ld, Qd, _ = O.opg_topk_eig_direct(pb.omega, pb.widths, pb.acts, pb.X, pb.Y, 6)
    assert np.allclose(ld, lg, rtol=0, atol=1e-12 * lg[0])
    assert np.allclose(np.abs(np.sum(Qd * Qg, axis=0)), 1.0, atol=1e-9)


def test_opg_topk_eig_rank_deficient():
    """Three examples of which two are identical: the Gram matrix has rank 2,
    so asking for 3 pairs flags the null space and returns a zero vector."""
    pb = _tiny([4, 3, 3], ["sigmoid"], N=3)
    X, Y = pb.X.copy(), pb.Y.copy()
    X[2], Y[2] = X[0], Y[0]
    mu, Q, deficient = O.opg_topk_eig(pb.omega, pb.widths, pb.acts, X, Y, 3)
    assert deficient
    assert np.all(Q[:, 2] == 0.0)
    assert abs(mu[2]) < 1e-13 * mu[0]
    assert np.linalg.norm(Q[:, :2].T @ Q[:, :2] - np.eye(2)) < 1e-12


# ---------------------------------------------------------- mutations ----

def test_pins_catch_dropped_second_derivative(monkeypatch):
    """Planting sigma'' = 0 for tanh (a dropped term) breaks the FD pin."""
    pb = _tiny([3, 4, 3], ["tanh"], N=5, seed=21)
    real = O.activation

    def broken(name, z):
        a, d1, d2 = real(name, z)
        return a, d1, np.zeros_like(d2)

    Hfd = _fd_hessian_of_gradient(pb)
    monkeypatch.setattr(O, "activation", broken)
    H = O.hessian(pb.omega, pb.widths, pb.acts, pb.X, pb.Y)
    assert _relerr(H, Hfd) > 1e-4


def test_pins_catch_transposed_weight_direction(monkeypatch):
    """Planting a transposed V^(l) in the R-forward breaks the FD pin."""
    pb = _tiny([3, 3, 3], ["sigmoid"], N=5, seed=22)
    Hfd = _fd_hessian_of_gradient(pb)
    real = O.unflatten
    state = {"calls": 0}

    def broken(omega, widths):
        out = real(omega, widths)
        state["calls"] += 1
        # the first call unflattens omega (forward pass); every later call
        # unflattens a direction vector inside hvp()
        if state["calls"] > 1:
            out = [(W.T.copy() if W.shape[0] == W.shape[1] else W, b) for W, b in out]
        return out

    monkeypatch.setattr(O, "unflatten", broken)
    H = O.hessian(pb.omega, pb.widths, pb.acts, pb.X, pb.Y)
    assert _relerr(H, Hfd) > 1e-4


def test_pins_catch_unnormalised_softmax(monkeypatch):
    """Planting a softmax output that no longer sums to one (a dropped
    log-sum-exp normalisation) breaks the single-layer closed form."""
    pb = _tiny([4, 3], [], N=6, seed=3)
    f = O.forward(pb.omega, pb.widths, pb.acts, pb.X)
    xt = np.hstack([pb.X, np.ones((pb.N, 1))])
    ref = sum(np.kron(np.diag(p) - np.outer(p, p), np.outer(x, x)) for p, x in zip(f["p"], xt)) / pb.N
    perm = O.param_permutation(pb.widths)
    real_forward = O.forward

    def broken_forward(*a, **k):
        out = real_forward(*a, **k)
        out["p"] = out["p"] * 1.5
        return out

    monkeypatch.setattr(O, "forward", broken_forward)
    H = O.hessian(pb.omega, pb.widths, pb.acts, pb.X, pb.Y)
    assert _relerr(H[np.ix_(perm, perm)], ref) > 1e-3


# ------------------------------------------------- Hessian eigenpairs ----

def test_hessian_topk_eig_closed_form_two_classes():
    """One example, a single softmax layer with zero weights and two classes:
    p = (1/2, 1/2), H = (diag p - p p^T) (x) xt xt^T (augmented-row order)
    with diag p - p p^T = [[1, -1], [-1, 1]] / 4, so the only nonzero
    eigenvalue is ||xt||^2 / 2 = (||x||^2 + 1) / 2, with eigenvector
    (1, -1)/sqrt(2) (x) xt / ||xt||; every other eigenvalue is 0."""
    widths = [4, 2]
    x = np.array([[0.3, -1.2, 2.0, 0.5]])
    y = np.array([[0.0, 1.0]])
    omega = np.zeros(O.num_params(widths))
    lam, Q = O.hessian_topk_eig(omega, widths, [], x, y, 3)
    xt = np.append(x[0], 1.0)
    assert abs(lam[0] - (xt @ xt) / 2) < 1e-14 * lam[0]
    assert np.all(np.abs(lam[1:]) < 1e-14 * lam[0])
    q_aug = np.kron(np.array([1.0, -1.0]) / np.sqrt(2), xt / np.linalg.norm(xt))
    q = np.empty_like(q_aug)
    q[O.param_permutation(widths)] = q_aug
    assert abs(abs(q @ Q[:, 0]) - 1.0) < 1e-14


def test_hessian_topk_eig_closed_form_three_classes_degenerate():
    """Three classes at zero weights: diag p - p p^T = I/3 - 11^T/9 has the
    double eigenvalue 1/3 on the complement of 1, so the top two Hessian
    eigenvalues are both ||xt||^2 / 3 and their eigenvectors span
    {u (x) xt : u . 1 = 0}."""
    widths = [3, 3]
    x = np.array([[1.0, -0.5, 0.25]])
    y = np.array([[1.0, 0.0, 0.0]])
    omega = np.zeros(O.num_params(widths))
    lam, Q = O.hessian_topk_eig(omega, widths, [], x, y, 3)
    xt = np.append(x[0], 1.0)
    assert np.allclose(lam[:2], (xt @ xt) / 3, rtol=1e-14, atol=0)
    assert abs(lam[2]) < 1e-14 * lam[0]
    perm = O.param_permutation(widths)
    basis = []
    for u in (np.array([1.0, -1.0, 0.0]), np.array([1.0, 1.0, -2.0])):
        b_aug = np.kron(u / np.linalg.norm(u), xt / np.linalg.norm(xt))
        b = np.empty_like(b_aug)
        b[perm] = b_aug
        basis.append(b)
    B = np.array(basis).T
    # the two computed vectors lie in span(B) and are orthonormal
    assert np.linalg.norm(Q[:, :2] - B @ (B.T @ Q[:, :2])) < 1e-13
    assert np.allclose(Q[:, :2].T @ Q[:, :2], np.eye(2), atol=1e-14)


def _check_top_eigenpairs(pb, lam, Q, H):
    """Each pair satisfies H q = lam q with the directional-difference-pinned
    products, the vectors are orthonormal, the values descend, and every
    Rayleigh quotient on the orthogonal complement of the top-k space is at
    most lam_k (the top-k invariant subspace maximises it)."""
    k = len(lam)
    assert np.all(np.diff(lam) <= 0)
    for c in range(k):
        Hq = O.hvp(pb.omega, pb.widths, pb.acts, pb.X, pb.Y, Q[:, c])
        assert np.linalg.norm(Hq - lam[c] * Q[:, c]) < 1e-12 * abs(lam[0])
    assert np.allclose(Q.T @ Q, np.eye(k), atol=1e-13)
    rng = np.random.default_rng(3)
    for _ in range(50):
        v = rng.standard_normal(pb.P)
        v -= Q @ (Q.T @ v)
        rq = (v @ (H @ v)) / (v @ v)
        assert rq <= lam[-1] + 1e-12 * abs(lam[0])


def test_hessian_topk_eig_is_the_top_of_the_spectrum():
    """An indefinite Hessian (tanh hidden layer): the pairs pass the checks
    above, and with k = P the values sum to trace(H) and their squares to
    ||H||_F^2."""
    pb = _tiny([5, 6, 3], ["tanh"], N=8, seed=10)
    H = O.hessian(pb.omega, pb.widths, pb.acts, pb.X, pb.Y)
    full = np.linalg.eigvalsh(H)
    assert full.min() < -1e-6 * full.max()  # indefinite: 'largest' must be algebraic
    lam, Q = O.hessian_topk_eig(pb.omega, pb.widths, pb.acts, pb.X, pb.Y, 6)
    _check_top_eigenpairs(pb, lam, Q, H)
    lam_all, _ = O.hessian_topk_eig(pb.omega, pb.widths, pb.acts, pb.X, pb.Y, pb.P)
    assert abs(lam_all.sum() - np.trace(H)) < 1e-12 * np.abs(lam_all).sum()
    assert abs((lam_all ** 2).sum() - (H * H).sum()) < 1e-12 * (H * H).sum()


def test_pins_catch_eigenpairs_ordered_by_magnitude():
    """Planting the largest-magnitude eigenpairs (instead of the algebraically
    largest) is caught by the spectrum checks on an indefinite Hessian whose
    most negative eigenvalue outweighs the k-th largest."""
    pb = _tiny([5, 6, 3], ["tanh"], N=8, seed=10)
    H = O.hessian(pb.omega, pb.widths, pb.acts, pb.X, pb.Y)
    lam, U = np.linalg.eigh(H)
    k = 6
    order = np.argsort(-np.abs(lam))[:k]
    assert lam[order].min() < 0  # the planted mistake picks a negative one
    with pytest.raises(AssertionError):
        _check_top_eigenpairs(pb, lam[order], O.canonical_sign(U[:, order]), H)


# ------------------------------------ low-rank / full-rank approximations ----

def test_lowrank_with_all_eigenpairs_is_the_hessian():
    """K = P: Q diag(lam) Q^T rebuilds H (the spectral theorem), and the
    full-rank term vanishes (Q Q^T = I)."""
    pb = _tiny([5, 6, 3], ["tanh"], N=8, seed=10)
    H = O.hessian(pb.omega, pb.widths, pb.acts, pb.X, pb.Y)
    lam, Q = O.hessian_topk_eig(pb.omega, pb.widths, pb.acts, pb.X, pb.Y, pb.P)
    assert _relerr(O.lowrank_matrix(Q, lam), H) < 1e-12
    assert _relerr(O.fullrank_matrix(Q, lam, 0.7), H) < 1e-12


def test_fullrank_spectrum_and_null_space():
    """With K < P: H~ has eigenvalues lam_1..lam_K and P - K zeros; H~~ has
    lam_1..lam_K and lam_tilde (P - K times), so it is positive definite when
    lam_tilde > 0 (Appendix, full-rank derivation); H~ q_k = lam_k q_k and, for
    v orthogonal to Q, H~ v = 0 and H~~ v = lam_tilde v."""
    pb = _tiny([5, 6, 3], ["tanh"], N=8, seed=10)
    K = 5
    lam, Q = O.hessian_topk_eig(pb.omega, pb.widths, pb.acts, pb.X, pb.Y, K)
    lt = lam[-1]
    assert lt > 0
    low = np.sort(np.linalg.eigvalsh(O.lowrank_matrix(Q, lam)))[::-1]
    assert np.allclose(low[:K], lam, rtol=0, atol=1e-12 * lam[0])
    assert np.all(np.abs(low[K:]) < 1e-12 * lam[0])
    full = np.sort(np.linalg.eigvalsh(O.fullrank_matrix(Q, lam, lt)))[::-1]
    assert np.allclose(full[:K], lam, rtol=0, atol=1e-12 * lam[0])
    assert np.allclose(full[K:], lt, rtol=0, atol=1e-12 * lam[0])
    v = np.random.default_rng(2).standard_normal(pb.P)
    v -= Q @ (Q.T @ v)
    HX, quad = O.approx_apply(Q, lam, np.vstack([Q[:, 1], v]))
    assert np.linalg.norm(HX[0] - lam[1] * Q[:, 1]) < 1e-13 * lam[0]
    assert np.linalg.norm(HX[1]) < 1e-13 * lam[0] * np.linalg.norm(v)
    HX, quad = O.approx_apply(Q, lam, v[None, :], lam_tilde=lt)
    assert np.linalg.norm(HX[0] - lt * v) < 1e-13 * lam[0] * np.linalg.norm(v)
    assert abs(quad[0] - lt * (v @ v)) < 1e-12 * lam[0] * (v @ v)


def test_implicit_application_matches_the_formed_matrices():
    """The implicit products and quadratic forms of Sec. 5.5 / 5.6 equal the
    explicit x^T H~ x with H~ formed (Sec. 4.1 / 4.2)."""
    rng = np.random.default_rng(4)
    P, K = 40, 6
    Q, _ = np.linalg.qr(rng.standard_normal((P, K)))
    lam = np.sort(rng.standard_normal(K))[::-1]
    X = rng.standard_normal((3, P))
    for lt, M in ((None, O.lowrank_matrix(Q, lam)), (0.3, O.fullrank_matrix(Q, lam, 0.3))):
        HX, quad = O.approx_apply(Q, lam, X, lam_tilde=lt)
        assert np.allclose(HX, X @ M, rtol=0, atol=1e-13)
        assert np.allclose(quad, np.einsum("ip,pq,iq->i", X, M, X), rtol=0, atol=1e-12)


# --------------------------------------------------- mini-batch Hessians ----

def test_minibatch_hessians_average_to_the_full_hessian():
    """The mini-batch Hessians weighted by their sizes average to the full H
    (Eq. hesseq1 is a mean over examples), with a ragged last batch."""
    pb = _tiny([5, 6, 4, 3], ["sigmoid", "tanh"], N=11, seed=14)
    Hs = O.minibatch_hessians(pb.omega, pb.widths, pb.acts, pb.X, pb.Y, 4)
    assert Hs.shape == (3, pb.P, pb.P)
    sizes = np.array([4, 4, 3])
    H = O.hessian(pb.omega, pb.widths, pb.acts, pb.X, pb.Y)
    assert _relerr((Hs * sizes[:, None, None]).sum(axis=0) / pb.N, H) < 1e-13


def test_per_example_hessians_single_layer_closed_form():
    """bs = 1 on a single softmax layer: each per-example Hessian is
    (diag p_n - p_n p_n^T) (x) xt_n xt_n^T (augmented-row order), rank at most
    T_L - 1."""
    pb = _tiny([4, 3], [], N=5, seed=6)
    Hs = O.minibatch_hessians(pb.omega, pb.widths, pb.acts, pb.X, pb.Y, 1)
    f = O.forward(pb.omega, pb.widths, pb.acts, pb.X)
    perm = O.param_permutation(pb.widths)
    for n in range(pb.N):
        p = f["p"][n]
        xt = np.append(pb.X[n], 1.0)
        ref = np.kron(np.diag(p) - np.outer(p, p), np.outer(xt, xt))
        assert _relerr(Hs[n][np.ix_(perm, perm)], ref) < 1e-13
        ev = np.linalg.eigvalsh(Hs[n])
        assert int((np.abs(ev) > 1e-12 * np.abs(ev).max()).sum()) <= pb.widths[-1] - 1


# ------------------------------------------------- memory-light routes ----

def test_memory_light_routes_match_full_matrices():
    pb = _tiny([7, 5, 4, 3], ["relu", "tanh"], N=11, seed=13)
    G = O.per_example_grads(pb.omega, pb.widths, pb.acts, pb.X, pb.Y)
    cols = [0, 5, 34, 35, 39, 40, 60, 61, 62, pb.P - 1]
    assert np.array_equal(O.per_example_grads_columns(pb.omega, pb.widths, pb.acts, pb.X, pb.Y, cols),
                          G[:, cols])
    f = O.forward(pb.omega, pb.widths, pb.acts, pb.X)
    delta, _ = O.backprop(f, pb.Y)
    rng = np.random.default_rng(1)
    V = rng.standard_normal((pb.N, 3))
    Qm = rng.standard_normal((pb.P, 2))
    assert _relerr(O.grads_transpose_times(f, delta, pb.widths, V), G.T @ V) < 1e-14
    assert _relerr(O.grads_times(f, delta, pb.widths, Qm), G @ Qm) < 1e-14
    mu, Q, d = O.opg_topk_eig_factored(pb.omega, pb.widths, pb.acts, pb.X, pb.Y, 4)
    mu2, Q2, d2 = O.opg_topk_eig_from_grads(G, 4)
    assert d == d2 and np.allclose(mu, mu2, rtol=0, atol=1e-14 * mu2[0])
    assert np.allclose(Q, Q2, rtol=0, atol=1e-10)
