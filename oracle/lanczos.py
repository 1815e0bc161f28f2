"""O4: Lanczos ground-state solve with full re-orthogonalisation (textbook).

The paper has no eigensolver beyond TCI ``eigh``/``eigvalsh`` (App. C.2);
this follows Golub & Van Loan, Matrix Computations (4th ed.), Sec. 10.1
(Lanczos) and Sec. 8.4 (Sturm-sequence bisection for a symmetric
tridiagonal matrix), with classical Gram-Schmidt applied twice ("CGS2").

Step j (0-based), starting from v_0 = psi / ||psi||:
    w      = H v_j
    alpha_j = <v_j, w>
    w     <- w - alpha_j v_j - beta_{j-1} v_{j-1}
    twice:  h_i = <v_i, w> for i <= j;  w <- w - sum_i h_i v_i
    beta_j = ||w||;  stop if beta_j < tol |alpha_j|;  v_{j+1} = w / beta_j
The Ritz value is the smallest eigenvalue of T = tridiag(beta, alpha, beta)
found by bisection on the Sturm count; its eigenvector y comes from inverse
iteration; the Ritz vector is x = sum_j y_j v_j.
"""
from __future__ import annotations

import numpy as np


def sturm_count(alpha, beta, x: float) -> int:
    """Number of eigenvalues of tridiag(beta, alpha, beta) strictly below x.

    LDL^T pivots q_0 = alpha_0 - x, q_i = alpha_i - x - beta_{i-1}^2 / q_{i-1};
    the count of negative pivots equals the count of eigenvalues below x
    (Sylvester inertia).  A zero pivot is replaced by a tiny negative value
    as soon as it appears (so it is counted and divides the next pivot).
    """
    m = len(alpha)
    cnt = 0
    q = 1.0
    tiny = np.finfo(float).tiny
    for i in range(m):
        if i == 0:
            q = alpha[0] - x
        else:
            q = alpha[i] - x - beta[i - 1] * beta[i - 1] / q
        if q == 0.0:
            q = -tiny
        if q < 0.0:
            cnt += 1
    return cnt


def lowest_eigenvalue_bisect(alpha, beta, max_iter: int = 200) -> float:
    """Smallest eigenvalue of the symmetric tridiagonal T by Sturm bisection."""
    alpha = np.asarray(alpha, dtype=np.float64)
    beta = np.asarray(beta, dtype=np.float64)
    m = len(alpha)
    # Gershgorin interval
    r = np.zeros(m)
    if m > 1:
        r[:-1] += np.abs(beta[: m - 1])
        r[1:] += np.abs(beta[: m - 1])
    lo = float(np.min(alpha - r))
    hi = float(np.max(alpha + r))
    for _ in range(max_iter):
        mid = 0.5 * (lo + hi)
        if mid <= lo or mid >= hi:
            break
        if sturm_count(alpha, beta, mid) >= 1:
            hi = mid
        else:
            lo = mid
    return 0.5 * (lo + hi)


def tridiag_matrix(alpha, beta):
    m = len(alpha)
    T = np.diag(np.asarray(alpha, dtype=np.float64))
    for i in range(m - 1):
        T[i, i + 1] = T[i + 1, i] = beta[i]
    return T


def tridiag_eigvec(alpha, beta, theta: float, iters: int = 3):
    """Eigenvector of T for eigenvalue ``theta`` by inverse iteration (unit norm, y[argmax|y|] > 0)."""
    T = tridiag_matrix(alpha, beta)
    m = len(alpha)
    shift = theta - 1e-10 * max(1.0, abs(theta))
    A = T - shift * np.eye(m)
    y = np.ones(m) / np.sqrt(m)
    for _ in range(iters):
        y = np.linalg.solve(A, y)
        y /= np.linalg.norm(y)
    k = int(np.argmax(np.abs(y)))
    return y if y[k] > 0 else -y


def lanczos(matvec, v0, m: int, reorth: bool = True, tol: float = 1e-12):
    """Run up to ``m`` Lanczos steps; return dict(theta, x, alpha, beta, steps).

    ``beta`` has one entry per completed step (beta_j after step j).
    """
    v = np.asarray(v0, dtype=np.float64).ravel()
    v = v / np.linalg.norm(v)
    V = [v]
    alpha, beta = [], []
    for j in range(m):
        w = np.asarray(matvec(V[j]), dtype=np.float64).ravel()
        a = float(np.dot(V[j], w))
        w = w - a * V[j]
        if j > 0:
            w = w - beta[j - 1] * V[j - 1]
        if reorth:
            for _ in range(2):
                h = np.array([np.dot(vi, w) for vi in V])
                for hi, vi in zip(h, V):
                    w = w - hi * vi
        b = float(np.linalg.norm(w))
        alpha.append(a)
        beta.append(b)
        if j == m - 1 or b < tol * abs(a):
            break
        V.append(w / b)
    k = len(alpha)
    theta = lowest_eigenvalue_bisect(alpha, beta[: k - 1])
    y = tridiag_eigvec(alpha, beta[: k - 1], theta)
    x = np.zeros_like(V[0])
    for yj, vj in zip(y, V[:k]):
        x = x + yj * vj
    return {"theta": theta, "x": x, "alpha": np.array(alpha), "beta": np.array(beta), "steps": k, "y": y}


def lanczos_real_form(matvec, v0, m: int, reorth: bool = True, tol: float = 1e-12):
    """Lanczos for a Hermitian operator on complex vectors, run on its real form.

    A Hermitian H = A + iB acting on v = x + iy is the real symmetric operator
    [[A, -B], [B, A]] on (x, y); with v stored as interleaved (re, im) pairs
    that operator acts on the float64 view of v, its spectrum is H's with every
    eigenvalue twice, so its lowest Ritz value converges to H's ground energy.
    ``lanczos`` above runs on that view unchanged; the Ritz vector is returned
    as complex128.
    """
    v0 = np.ascontiguousarray(v0, dtype=np.complex128)
    shape = v0.shape

    def mv(u):
        z = np.ascontiguousarray(u).view(np.complex128).reshape(shape)
        return np.ascontiguousarray(matvec(z), dtype=np.complex128).ravel().view(np.float64)

    r = lanczos(mv, v0.ravel().view(np.float64), m, reorth, tol)
    r["x"] = np.ascontiguousarray(r["x"]).view(np.complex128)
    return r
