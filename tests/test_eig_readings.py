"""Host checks of two numerical constructions inside the OPG eigen step.

The paper asks for the largest eigenpairs through a Lanczos process (Sec.
5.3) and leaves open how its basis is kept orthogonal and how the small
tridiagonal problem is solved.  The double-float Lanczos kernel takes the
second classical Gram-Schmidt pass of each vector one step late, inside the
next step's single reduction, and the tridiagonal stage forms the
eigenvector of an isolated eigenvalue from a twisted factorization of
T - theta I and then takes theta as the vector's Rayleigh quotient.  These
tests restate both constructions in numpy, in the order the kernels apply
them, and hold them to what the mathematics fixes: the same tridiagonal
matrix as Lanczos with two explicit passes per step, the exact eigenvalues
of a matrix with a known spectrum, and eigenvectors of T from a dense
symmetric eigensolver.  (The CUDA kernels themselves are checked against
the oracle in the GPU tests.)
"""

import numpy as np
import pytest


def _spd(n, seed, decay=1e-3):
    rng = np.random.default_rng(seed)
    Q, _ = np.linalg.qr(rng.standard_normal((n, n)))
    lam = np.logspace(0, np.log10(decay), n)
    return (Q * lam) @ Q.T, lam


def _two_pass(M, q0, m):
    """Lanczos with classical Gram-Schmidt twice in the same step."""
    N = M.shape[0]
    Q = np.zeros((m + 1, N))
    Q[0] = q0 / np.linalg.norm(q0)
    al, be = np.zeros(m), np.zeros(m)
    for j in range(m):
        u = M @ Q[j]
        al[j] = Q[j] @ u
        w = u - Q[: j + 1].T @ (Q[: j + 1] @ u)
        w -= Q[: j + 1].T @ (Q[: j + 1] @ w)
        be[j] = np.linalg.norm(w)
        Q[j + 1] = w / be[j]
    return al, be, Q[:m]


def _lagged(M, q0, m):
    """The kernel's scheme: the vector handed to step j (w of step j-1, one
    pass only, not normalised) is corrected and normalised with the
    coefficients of step j's single reduction."""
    N = M.shape[0]
    Q = np.zeros((m, N))
    MQ = np.zeros((m, N))
    al, be = np.zeros(m), np.zeros(m)
    qt = q0 / np.linalg.norm(q0)
    for j in range(m + 1):
        full = j < m
        # the single reduction of step j
        c = Q[:j] @ qt
        nu = qt @ qt
        if full:
            ut = M @ qt
            g = MQ[:j] @ qt
            at = qt @ ut
        r = np.sqrt(nu - c @ c)
        if j > 0:
            be[j - 1] = r
        if not full:
            break
        Tc = al[:j] * c
        if j > 1:
            Tc[1:] += be[: j - 1] * c[:-1]
            Tc[:-1] += be[: j - 1] * c[1:]
        a = (at - 2.0 * (c @ g) + c @ Tc) / r ** 2
        al[j] = a
        d = (g - Tc) - a * c
        Q[j] = (qt - Q[:j].T @ c) / r
        MQ[j] = (ut - MQ[:j].T @ c) / r
        qt = (ut - a * qt - MQ[:j].T @ c - Q[:j].T @ d) / r
    return al, be, Q


@pytest.mark.parametrize("seed", [0, 1])
def test_lagged_second_pass_gives_the_two_pass_lanczos_matrix(seed):
    # a spectrum over 12 decades and enough steps for the top Ritz values to
    # converge: one Gram-Schmidt pass alone loses orthogonality here (1e-12
    # and worse), the lagged second pass keeps it at rounding level
    n, m = 240, 120
    M, lam = _spd(n, seed, decay=1e-12)
    q0 = np.random.default_rng(100 + seed).standard_normal(n)
    a2, b2, Q2 = _two_pass(M, q0, m)
    a1, b1, Q1 = _lagged(M, q0, m)
    assert np.max(np.abs(a1 - a2)) <= 1e-12 * lam[0]
    assert np.max(np.abs(b1 - b2)) <= 1e-12 * lam[0]
    # the basis stays orthonormal to rounding
    assert np.max(np.abs(Q1 @ Q1.T - np.eye(m))) <= 1e-13
    # and its Ritz values converge to the known spectrum from the top
    T = np.diag(a1) + np.diag(b1[: m - 1], 1) + np.diag(b1[: m - 1], -1)
    th = np.linalg.eigvalsh(T)[::-1]
    assert np.max(np.abs(th[:10] - lam[:10])) <= 1e-12 * lam[0]


def _twisted_vector(a, b, theta):
    """Eigenvector of the symmetric tridiagonal T (diagonal a, off-diagonal
    b) for an isolated eigenvalue theta: pivots d+ from the top and d- from
    the bottom, the twist r where gamma_r = d+_r + d-_r - (a_r - theta) is
    smallest in magnitude, z_r = 1 and the products outward."""
    m = a.size
    d = a - theta
    dp = np.zeros(m)
    dm = np.zeros(m)
    dp[0] = d[0]
    for i in range(1, m):
        dp[i] = d[i] - b[i - 1] ** 2 / dp[i - 1]
    dm[m - 1] = d[m - 1]
    for i in range(m - 2, -1, -1):
        dm[i] = d[i] - b[i] ** 2 / dm[i + 1]
    gamma = dp + dm - d
    r = int(np.argmin(np.abs(gamma)))
    z = np.zeros(m)
    z[r] = 1.0
    for i in range(r - 1, -1, -1):
        z[i] = -(b[i] / dp[i]) * z[i + 1]
    for i in range(r + 1, m):
        z[i] = -(b[i - 1] / dm[i]) * z[i - 1]
    return z / np.linalg.norm(z)


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_twisted_factorization_eigenvectors_and_rayleigh_quotients(seed):
    rng = np.random.default_rng(seed)
    m = 96
    a = rng.standard_normal(m)
    b = rng.uniform(0.1, 1.0, m - 1)
    T = np.diag(a) + np.diag(b, 1) + np.diag(b, -1)
    lam, V = np.linalg.eigh(T)
    tn = np.max(np.abs(lam))
    checked = 0
    for c in range(m - 1, m - 17, -1):  # the largest 16
        gaps = np.abs(np.delete(lam, c) - lam[c])
        if gaps.min() < 1e-6 * tn:
            continue  # a cluster: the kernel keeps inverse iteration there
        # the shift carries the bisection's error (2^-40 ||T||)
        theta = lam[c] + 2.0 ** -40 * tn
        z = _twisted_vector(a, b, theta)
        assert abs(abs(z @ V[:, c]) - 1.0) <= 1e-10
        assert np.linalg.norm(T @ z - theta * z) <= 1e-11 * tn
        rq = z @ (T @ z)
        assert abs(rq - lam[c]) <= 1e-14 * tn
        checked += 1
    assert checked >= 12
