"""FP64 CPU oracle for the curvature matrices of a dense MLP.

TEST INFRASTRUCTURE ONLY.  Nothing in the product path imports, links or
runs this module: only the tests, ``__graft_entry__.smoke()`` and the
benchmark's CPU-baseline leg do.  It shares no code with the CUDA library;
the only common dependency is the seeded input generator in ``synth``.

Everything here is plain numpy in float64, written from the definitions in
"Efficient Computation of Hessian Matrices in TensorFlow" (Nilsen et al.):

* model and cost:  Sec. 2, Eq. modelfunc, Eq. cost, softmax output;
* parameter order: Sec. 2, Eq. flatten (row-wise W^(l-1) then b^(l));
* exact Hessian:   Sec. 3, Eq. hesseq1, built column by column from
  Hessian-vector products with the unit vectors (Sec. 5.1); each product is
  Pearlmutter's forward-over-reverse R-operator, one direction at a time;
* OPG:             Sec. 3, Eq. hesseq2 / hesseq3 (J^T J / N with J the
  per-example gradient matrix, one row per example);
* OPG eigenpairs:  Sec. 5.4, Eq. J (eigenvectors of J^T J are the right
  singular vectors of J), reached through the N x N Gram matrix J J^T / N;
* Hessian eigenpairs: Sec. 5.3 (the algebraically largest eigenpairs of H),
  from the full H and a dense symmetric eigensolver;
* low-rank and full-rank approximations: Sec. 4.1, 4.2 and their implicit
  application, Sec. 5.5, 5.6;
* mini-batch and per-example Hessians: Sec. 5.1.

Pins that tie this code to the mathematics (finite differences, the closed
form of a single softmax layer, invariants, the paper's printed sizes) live in
``tests/test_oracle_pins.py``.  Every function below is pinned by at least one
of them; none is "parity unpinned".
"""

from __future__ import annotations

import numpy as np

ACTS = ("sigmoid", "tanh", "relu")


# ----------------------------------------------------------------------------
# Parameter vector (Sec. 2, Eq. flatten)
# ----------------------------------------------------------------------------

def num_params(widths) -> int:
    """P = T_1 T_2 + T_2 + ... + T_{L-1} T_L + T_L (Sec. 2, after Eq. flatten)."""
    return int(sum(widths[l - 1] * widths[l] + widths[l] for l in range(1, len(widths))))


def layer_offsets(widths):
    """For each weight layer j = 1..L-1 (maps layer j to layer j+1) return
    (offset of W^(j) in omega, offset of b^(j+1) in omega)."""
    offs = []
    o = 0
    for l in range(1, len(widths)):
        offs.append((o, o + widths[l - 1] * widths[l]))
        o += widths[l - 1] * widths[l] + widths[l]
    return offs


def unflatten(omega, widths):
    """Inverse of the row-wise flatten: list of (W^(l-1), b^(l)) for l = 2..L,
    W^(l-1) of shape (T_l, T_{l-1}) (Sec. 2)."""
    out = []
    for l, (ow, ob) in zip(range(1, len(widths)), layer_offsets(widths)):
        t_in, t_out = widths[l - 1], widths[l]
        out.append((np.asarray(omega[ow:ob], dtype=np.float64).reshape(t_out, t_in),
                    np.asarray(omega[ob:ob + t_out], dtype=np.float64)))
    return out


def flatten(params) -> np.ndarray:
    """Row-wise flatten of [(W, b), ...] in layer order (Sec. 2, Eq. flatten)."""
    return np.concatenate([np.concatenate([W.reshape(-1), b]) for W, b in params])


def param_permutation(widths) -> np.ndarray:
    """perm such that omega_aug = omega[perm] lists, for every layer, output
    unit i's weight row followed by its bias: [W_i0..W_i(T-1), b_i, W_(i+1)0 ...].
    This "augmented row" order is what the single-layer closed form uses."""
    perm = []
    for l, (ow, ob) in zip(range(1, len(widths)), layer_offsets(widths)):
        t_in, t_out = widths[l - 1], widths[l]
        for i in range(t_out):
            perm.extend(range(ow + i * t_in, ow + (i + 1) * t_in))
            perm.append(ob + i)
    return np.asarray(perm, dtype=np.int64)


# ----------------------------------------------------------------------------
# Activations (hidden sigma^(l), Sec. 2): value, first and second derivative
# ----------------------------------------------------------------------------

def activation(name, z):
    """Return (sigma(z), sigma'(z), sigma''(z)).  ReLU uses sigma'(0) = 0 and
    sigma'' = 0 (the convention of TensorFlow's ReLU gradient)."""
    if name == "sigmoid":
        s = 1.0 / (1.0 + np.exp(-z))
        return s, s * (1.0 - s), s * (1.0 - s) * (1.0 - 2.0 * s)
    if name == "tanh":
        t = np.tanh(z)
        return t, 1.0 - t * t, -2.0 * t * (1.0 - t * t)
    if name == "relu":
        return np.maximum(z, 0.0), (z > 0).astype(np.float64), np.zeros_like(z)
    raise ValueError(name)


# ----------------------------------------------------------------------------
# Forward pass and cost (Sec. 2, Eq. modelfunc, Eq. cost)
# ----------------------------------------------------------------------------

def forward(omega, widths, acts, X):
    """Evaluate the network on all N inputs (rows of X).

    Returns a dict with lists indexed by layer position j = 0..L-1 (layer l = j+1):
      a[j]  : activations (a[0] = X),            shape (N, T_{j+1})
      z[j]  : pre-activations (z[0] = None)
      d1[j], d2[j] : sigma'(z), sigma''(z) for hidden layers (None otherwise)
    and 'p' (softmax output), 'lse' (log-sum-exp of the logits).
    """
    params = unflatten(omega, widths)
    L = len(widths)
    a = [np.asarray(X, dtype=np.float64)]
    z = [None]
    d1 = [None]
    d2 = [None]
    for j in range(1, L):
        W, b = params[j - 1]
        zj = a[j - 1] @ W.T + b
        z.append(zj)
        if j < L - 1:
            aj, s1, s2 = activation(acts[j - 1], zj)
            a.append(aj)
            d1.append(s1)
            d2.append(s2)
    zL = z[L - 1]
    m = zL.max(axis=1, keepdims=True)
    lse = (m + np.log(np.exp(zL - m).sum(axis=1, keepdims=True)))[:, 0]
    p = np.exp(zL - lse[:, None])
    return {"a": a, "z": z, "d1": d1, "d2": d2, "p": p, "lse": lse, "params": params}


def per_example_costs(omega, widths, acts, X, Y):
    """C_n = -sum_m y_nm log yhat_nm, written as logsumexp(z^(L)) - y . z^(L)
    when sum_m y_nm = 1 (Sec. 2, Eq. cost)."""
    f = forward(omega, widths, acts, X)
    zL = f["z"][-1]
    Y = np.asarray(Y, dtype=np.float64)
    return f["lse"] * Y.sum(axis=1) - (Y * zL).sum(axis=1)


def cost(omega, widths, acts, X, Y) -> float:
    """C = (1/N) sum_n C_n (Sec. 2, Eq. cost)."""
    return float(per_example_costs(omega, widths, acts, X, Y).mean())


# ----------------------------------------------------------------------------
# First order: per-example gradients (Sec. 3.1, Sec. 5.2)
# ----------------------------------------------------------------------------

def backprop(f, Y):
    """Per-example back-propagation.  Returns delta[j] = dC_n/dz^(j+1) for the
    layers j = 1..L-1 (delta[0] = None), each of shape (N, T_{j+1}), and
    e[j] = W^(j)^T delta[j+1] for hidden j (the error before the sigma' factor).
    For the softmax output, dC_n/dz^(L) = p_n (sum_m y_nm) - y_n."""
    params, a, d1 = f["params"], f["a"], f["d1"]
    L = len(a) + 1
    Y = np.asarray(Y, dtype=np.float64)
    delta = [None] * L
    e = [None] * L
    delta[L - 1] = f["p"] * Y.sum(axis=1, keepdims=True) - Y
    for j in range(L - 2, 0, -1):
        W_next, _ = params[j]  # W^(j+1) maps layer j+1 -> j+2 (0-based j)
        e[j] = delta[j + 1] @ W_next
        delta[j] = d1[j] * e[j]
    return delta, e


def per_example_grads(omega, widths, acts, X, Y) -> np.ndarray:
    """G (N x P): row n is dC_n/domega^T in the order of Eq. flatten.
    dC_n/dW^(l-1) = delta^(l) a^(l-1)^T and dC_n/db^(l) = delta^(l)."""
    f = forward(omega, widths, acts, X)
    delta, _ = backprop(f, Y)
    N = f["a"][0].shape[0]
    cols = []
    for j in range(1, len(widths)):
        outer = delta[j][:, :, None] * f["a"][j - 1][:, None, :]  # (N, T_out, T_in)
        cols.append(outer.reshape(N, -1))
        cols.append(delta[j])
    return np.concatenate(cols, axis=1)


def gradient(omega, widths, acts, X, Y) -> np.ndarray:
    """dC/domega = (1/N) sum_n g_n (Sec. 3: the sum that TF's gradients return,
    divided by N)."""
    return per_example_grads(omega, widths, acts, X, Y).mean(axis=0)


# ----------------------------------------------------------------------------
# OPG (Sec. 3, Eq. hesseq2 / hesseq3)
# ----------------------------------------------------------------------------

def opg_from_grads(G) -> np.ndarray:
    """OPG = (1/N) sum_n g_n g_n^T = (1/N) J^T J with J = G (N x P)."""
    G = np.asarray(G, dtype=np.float64)
    return (G.T @ G) / G.shape[0]


def opg(omega, widths, acts, X, Y) -> np.ndarray:
    return opg_from_grads(per_example_grads(omega, widths, acts, X, Y))


# ----------------------------------------------------------------------------
# Second order: Hessian-vector products and the exact Hessian
# (Sec. 3 Eq. hesseq1; Sec. 5.1; Appendix A.1)
# ----------------------------------------------------------------------------

def hvp(omega, widths, acts, X, Y, v, f=None) -> np.ndarray:
    """H v for H = (1/N) sum_n d^2 C_n / domega domega^T, by the R-operator
    R{.} = d/dr (.)(omega + r v) at r = 0 applied to the forward pass and to
    the per-example back-propagation (forward-over-reverse).

    Forward:  R{z^(2)}  = V^(1) x + v_b^(2)
              R{a^(l)}  = sigma'(z^(l)) * R{z^(l)}
              R{z^(l)}  = W^(l-1) R{a^(l-1)} + V^(l-1) a^(l-1) + v_b^(l)
    Output:   R{delta^(L)} = (diag p - p p^T) R{z^(L)} * sum_m y_m
    Backward: R{delta^(l-1)} = sigma''(z) * R{z} * (W^T delta^(l))
                             + sigma'(z) * (V^T delta^(l) + W^T R{delta^(l)})
    Gradient: R{dC_n/dW^(l-1)} = R{delta^(l)} a^(l-1)^T + delta^(l) R{a^(l-1)}^T
              R{dC_n/db^(l)}   = R{delta^(l)}
    """
    if f is None:
        f = forward(omega, widths, acts, X)
    Y = np.asarray(Y, dtype=np.float64)
    delta, e = backprop(f, Y)
    params = f["params"]
    vparams = unflatten(np.asarray(v, dtype=np.float64), widths)
    a, d1, d2 = f["a"], f["d1"], f["d2"]
    L = len(widths)
    N = a[0].shape[0]

    Ra = [np.zeros_like(a[0])]  # inputs do not depend on omega
    Rz = [None]
    for j in range(1, L):
        W, _ = params[j - 1]
        V, vb = vparams[j - 1]
        Rzj = Ra[j - 1] @ W.T + a[j - 1] @ V.T + vb
        Rz.append(Rzj)
        if j < L - 1:
            Ra.append(d1[j] * Rzj)

    p = f["p"]
    RzL = Rz[L - 1]
    Rdelta = [None] * L
    Rdelta[L - 1] = (p * RzL - p * (p * RzL).sum(axis=1, keepdims=True)) * Y.sum(axis=1, keepdims=True)
    for j in range(L - 2, 0, -1):
        W_next, _ = params[j]
        V_next, _ = vparams[j]
        Rdelta[j] = (d2[j] * Rz[j] * e[j]
                     + d1[j] * (delta[j + 1] @ V_next + Rdelta[j + 1] @ W_next))

    out = []
    for j in range(1, L):
        RgW = (Rdelta[j].T @ a[j - 1] + delta[j].T @ Ra[j - 1]) / N
        Rgb = Rdelta[j].sum(axis=0) / N
        out.append(RgW.reshape(-1))
        out.append(Rgb)
    return np.concatenate(out)


def hessian_columns(omega, widths, acts, X, Y, cols) -> np.ndarray:
    """Columns H[:, j] for j in cols, each the product of H with the unit vector
    e_j (Sec. 5.1: the full H is P products with the basis of R^P).
    Returns an array of shape (P, len(cols))."""
    P = num_params(widths)
    f = forward(omega, widths, acts, X)
    out = np.empty((P, len(cols)))
    for c, j in enumerate(cols):
        ej = np.zeros(P)
        ej[j] = 1.0
        out[:, c] = hvp(omega, widths, acts, X, Y, ej, f=f)
    return out


def hessian(omega, widths, acts, X, Y) -> np.ndarray:
    """Full exact P x P Hessian (Sec. 3, Eq. hesseq1) from P Hessian-vector
    products with unit vectors."""
    P = num_params(widths)
    return hessian_columns(omega, widths, acts, X, Y, range(P))


def hessian_topk_eig(omega, widths, acts, X, Y, k):
    """Top-k eigenpairs of the exact Hessian, eigenvalues algebraically
    largest first (Sec. 5.3: the k largest-algebraic eigenpairs of the Hessian
    operator; H is indefinite, so 'largest' is algebraic, not in magnitude).
    Here H is formed in full (Sec. 3, Eq. hesseq1) and numpy.linalg.eigh
    serves as the dense symmetric eigensolver step.  Returns (lam (k,),
    Q (P, k) with unit columns of canonical sign)."""
    H = hessian(omega, widths, acts, X, Y)
    lam, U = np.linalg.eigh(H)
    order = np.argsort(lam)[::-1][:k]
    return lam[order], canonical_sign(U[:, order])


# ----------------------------------------------------------------------------
# Low-rank and full-rank approximations from K eigenpairs (Sec. 4.1, 4.2,
# Sec. 5.5, 5.6, Appendix "Derivation of the Full-rank Approximation")
# ----------------------------------------------------------------------------

def lowrank_matrix(Q, lam) -> np.ndarray:
    """H~ = Q diag(lam) Q^T (Sec. 4.1, Eq. lowrankapprox); Q is P x K with the
    eigenvectors as columns."""
    Q = np.asarray(Q, dtype=np.float64)
    return Q @ np.diag(np.asarray(lam, dtype=np.float64)) @ Q.T


def fullrank_matrix(Q, lam, lam_tilde) -> np.ndarray:
    """H~~ = H~ + lam_tilde (I - Q Q^T) (Sec. 4.2): the remaining P - K
    eigenvalues replaced by lam_tilde (the paper's choice is lam_K)."""
    Q = np.asarray(Q, dtype=np.float64)
    P = Q.shape[0]
    return lowrank_matrix(Q, lam) + lam_tilde * (np.eye(P) - Q @ Q.T)


def approx_apply(Q, lam, X, lam_tilde=None):
    """For each row x of X (b x P): H~ x and x^T H~ x without forming a P x P
    matrix (Sec. 5.5: (x^T Q) diag(lam) (Q^T x)); with lam_tilde given, the
    full-rank operator (Sec. 5.6: + lam_tilde x^T x - lam_tilde (x^T Q)(Q^T x)).
    Returns (HX (b x P), quad (b,))."""
    Q = np.asarray(Q, dtype=np.float64)
    lam = np.asarray(lam, dtype=np.float64)
    X = np.atleast_2d(np.asarray(X, dtype=np.float64))
    C = X @ Q  # b x K: the coordinates x^T Q
    HX = (C * lam) @ Q.T
    quad = (C * C) @ lam
    if lam_tilde is not None:
        HX = HX + lam_tilde * (X - C @ Q.T)
        quad = quad + lam_tilde * ((X * X).sum(axis=1) - (C * C).sum(axis=1))
    return HX, quad


def minibatch_hessians(omega, widths, acts, X, Y, bs):
    """Hessians of consecutive mini-batches of bs examples (the last may be
    shorter), each the average of its examples' Hessians (Sec. 5.1: the
    Hessian operation fed one example, or a mini-batch); bs = 1 gives the
    per-example Hessians.  Returns an array (ceil(N / bs), P, P)."""
    X = np.asarray(X, dtype=np.float64)
    Y = np.asarray(Y, dtype=np.float64)
    N = X.shape[0]
    return np.stack([hessian(omega, widths, acts, X[b:b + bs], Y[b:b + bs]) for b in range(0, N, bs)])


# ----------------------------------------------------------------------------
# OPG eigenpairs through the Gram matrix (Sec. 4.1, Sec. 5.4, Eq. J)
# ----------------------------------------------------------------------------

def gram_from_grads(G) -> np.ndarray:
    """M = (1/N) G G^T (N x N): same nonzero eigenvalues as OPG = (1/N) G^T G."""
    G = np.asarray(G, dtype=np.float64)
    return (G @ G.T) / G.shape[0]


def gram_factored(omega, widths, acts, X, Y) -> np.ndarray:
    """The same Gram matrix without forming G: since g_n restricted to layer l
    is delta_n^(l) (x) [a_n^(l-1); 1],
    g_n . g_m = sum_l (delta_n^(l) . delta_m^(l)) (a_n^(l-1) . a_m^(l-1) + 1)."""
    f = forward(omega, widths, acts, X)
    delta, _ = backprop(f, Y)
    N = f["a"][0].shape[0]
    M = np.zeros((N, N))
    for j in range(1, len(widths)):
        M += (delta[j] @ delta[j].T) * (f["a"][j - 1] @ f["a"][j - 1].T + 1.0)
    return M / N


def canonical_sign(Q) -> np.ndarray:
    """Flip each column so that its entry of largest magnitude is positive
    (eigenvectors are defined up to sign, Sec. 4.1)."""
    Q = np.array(Q, dtype=np.float64, copy=True)
    for k in range(Q.shape[1]):
        i = int(np.argmax(np.abs(Q[:, k])))
        if Q[i, k] < 0:
            Q[:, k] = -Q[:, k]
    return Q


def opg_topk_eig_from_grads(G, k, rank_tol=1e-13):
    """Top-k eigenpairs of OPG = G^T G / N, eigenvalues algebraically sorted in
    descending order (Sec. 4.1, Sec. 5.3).  With G = U S V^T (Sec. 5.4, Eq. J)
    the OPG eigenvalues are s^2 / N, i.e. the eigenvalues mu of M = G G^T / N,
    and q_k = G^T u_k / sqrt(N mu_k).  Eigenvalues below rank_tol * mu_1 belong
    to the null space; their vectors are returned as zeros and the flag
    'rank_deficient' is set.  numpy.linalg.eigh serves as the dense symmetric
    eigensolver step."""
    G = np.asarray(G, dtype=np.float64)
    N = G.shape[0]
    M = gram_from_grads(G)
    mu, U = np.linalg.eigh(M)
    order = np.argsort(mu)[::-1][:k]
    mu = mu[order]
    U = U[:, order]
    Q = np.zeros((G.shape[1], k))
    deficient = False
    top = mu[0] if k > 0 else 0.0
    for c in range(k):
        if mu[c] > rank_tol * top and mu[c] > 0:
            Q[:, c] = (G.T @ U[:, c]) / np.sqrt(N * mu[c])
        else:
            deficient = True
    return mu, canonical_sign(Q), deficient


def opg_topk_eig(omega, widths, acts, X, Y, k, rank_tol=1e-13):
    return opg_topk_eig_from_grads(per_example_grads(omega, widths, acts, X, Y), k, rank_tol)


def opg_topk_eig_direct(omega, widths, acts, X, Y, k, rank_tol=1e-13):
    """The same eigenpairs from the P x P OPG itself (Sec. 4.1: the
    eigendecomposition of the matrix; no Gram matrix, so N may be large).
    numpy.linalg.eigh serves as the dense symmetric eigensolver step; null
    directions as in opg_topk_eig_from_grads."""
    M = opg(omega, widths, acts, X, Y)
    lam, U = np.linalg.eigh(M)
    order = np.argsort(lam)[::-1][:k]
    lam = lam[order]
    Q = U[:, order].copy()
    deficient = False
    for c in range(k):
        if not (lam[c] > rank_tol * lam[0] and lam[c] > 0):
            Q[:, c] = 0.0
            deficient = True
    return lam, canonical_sign(Q), deficient


# ----------------------------------------------------------------------------
# Memory-light routes for large P (same definitions, no N x P matrix)
# ----------------------------------------------------------------------------

def _param_coords(widths):
    """For every parameter index: (weight layer j = 1..L-1, output unit i,
    input unit k or -1 for the bias) in the order of Eq. flatten."""
    coords = []
    for j, (ow, ob) in zip(range(1, len(widths)), layer_offsets(widths)):
        t_in, t_out = widths[j - 1], widths[j]
        for i in range(t_out):
            for k in range(t_in):
                coords.append((j, i, k))
        for i in range(t_out):
            coords.append((j, i, -1))
    return coords


def per_example_grads_columns(omega, widths, acts, X, Y, cols) -> np.ndarray:
    """Columns G[:, cols] of the per-example gradient matrix:
    G[n, W^(j)_{ik}] = delta_n^(j+1)_i a_n^(j)_k and G[n, b^(j+1)_i] = delta_n^(j+1)_i."""
    f = forward(omega, widths, acts, X)
    delta, _ = backprop(f, Y)
    coords = _param_coords(widths)
    N = f["a"][0].shape[0]
    out = np.empty((N, len(cols)))
    for c, col in enumerate(cols):
        j, i, k = coords[col]
        out[:, c] = delta[j][:, i] * (f["a"][j - 1][:, k] if k >= 0 else 1.0)
    return out


def grads_transpose_times(f, delta, widths, V) -> np.ndarray:
    """G^T V for V of shape (N, m) without forming G: the block of layer j is
    sum_n V[n] delta_n^(j+1) [a_n^(j); 1]^T."""
    blocks = []
    for j in range(1, len(widths)):
        d, a = delta[j], f["a"][j - 1]
        dV = V[:, :, None] * d[:, None, :]            # (N, m, T_out)
        W = np.tensordot(dV, a, axes=([0], [0]))       # (m, T_out, T_in)
        blocks.append(W.reshape(V.shape[1], -1))
        blocks.append(V.T @ d)
    return np.concatenate(blocks, axis=1).T  # (P, m)


def grads_times(f, delta, widths, Qm) -> np.ndarray:
    """G Q for Q of shape (P, m) without forming G:
    (G q)_n = sum_j delta_n^(j+1) . (W_q^(j) a_n^(j) + b_q^(j+1))."""
    N = f["a"][0].shape[0]
    out = np.zeros((N, Qm.shape[1]))
    for j, (ow, ob) in zip(range(1, len(widths)), layer_offsets(widths)):
        t_in, t_out = widths[j - 1], widths[j]
        Wq = Qm[ow:ob].reshape(t_out, t_in, -1)
        bq = Qm[ob:ob + t_out]
        za = np.tensordot(f["a"][j - 1], Wq, axes=([1], [1])) + bq[None, :, :]  # (N, T_out, m)
        out += (delta[j][:, :, None] * za).sum(axis=1)
    return out


def opg_topk_eig_factored(omega, widths, acts, X, Y, k, rank_tol=1e-13):
    """The top-k OPG eigenpairs of Sec. 5.4 (Eq. J) without forming G: Gram
    matrix in factored form, numpy.linalg.eigh, back-projection
    q = G^T u / sqrt(N mu) in factored form."""
    f = forward(omega, widths, acts, X)
    delta, _ = backprop(f, Y)
    N = f["a"][0].shape[0]
    M = np.zeros((N, N))
    for j in range(1, len(widths)):
        M += (delta[j] @ delta[j].T) * (f["a"][j - 1] @ f["a"][j - 1].T + 1.0)
    M /= N
    mu, U = np.linalg.eigh(M)
    order = np.argsort(mu)[::-1][:k]
    mu, U = mu[order], U[:, order]
    top = mu[0]
    keep = (mu > rank_tol * top) & (mu > 0)
    Q = np.zeros((num_params(widths), k))
    if keep.any():
        Q[:, keep] = grads_transpose_times(f, delta, widths, U[:, keep]) / np.sqrt(N * mu[keep])
    return mu, canonical_sign(Q), bool((~keep).any())
