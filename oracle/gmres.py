"""Right-preconditioned restarted GMRES (paper Section 5: the Krylov solver
M is used in; convergence when ||A_hat x - b_hat|| / ||b_hat|| < tol).

ORACLE -- test infrastructure only (see oracle/__init__.py).

Textbook GMRES(m) with modified Gram-Schmidt Arnoldi and Givens rotations,
x_0 = 0.  Right preconditioning: the Krylov space is built for A_hat M^{-1}
and the iterate is x = x_0 + M^{-1} V y, formed as Z y with Z_j = M^{-1} v_j.
A cycle stops when the rotated residual estimate drops below tol*||b||; the
true residual is then recomputed and a new cycle starts if it is not met.
`max_iters` caps the total number of Arnoldi steps (the paper uses 300).
"""
from __future__ import annotations

import numpy as np


def gmres(A, b, Minv, tol=1e-8, restart=30, max_iters=300):
    n = b.size
    x = np.zeros(n)
    bnorm = float(np.linalg.norm(b))
    history = []
    its = 0
    if bnorm == 0.0:
        return x, {"iters": 0, "converged": True, "rel_res": 0.0, "history": history}
    while True:
        r = b - A @ x
        beta = float(np.linalg.norm(r))
        rel = beta / bnorm
        if rel <= tol or its >= max_iters:
            return x, {"iters": its, "converged": rel <= tol, "rel_res": rel, "history": history}
        V = np.zeros((restart + 1, n))
        Z = np.zeros((restart, n))
        H = np.zeros((restart + 1, restart))
        cs = np.zeros(restart)
        sn = np.zeros(restart)
        g = np.zeros(restart + 1)
        g[0] = beta
        V[0] = r / beta
        k = 0
        for j in range(restart):
            Z[j] = Minv(V[j])
            w = A @ Z[j]
            its += 1
            for i in range(j + 1):
                H[i, j] = w @ V[i]
                w = w - H[i, j] * V[i]
            H[j + 1, j] = np.linalg.norm(w)
            for i in range(j):
                t = cs[i] * H[i, j] + sn[i] * H[i + 1, j]
                H[i + 1, j] = -sn[i] * H[i, j] + cs[i] * H[i + 1, j]
                H[i, j] = t
            denom = np.hypot(H[j, j], H[j + 1, j])
            cs[j] = H[j, j] / denom
            sn[j] = H[j + 1, j] / denom
            hj1 = H[j + 1, j]
            H[j, j] = denom
            H[j + 1, j] = 0.0
            g[j + 1] = -sn[j] * g[j]
            g[j] = cs[j] * g[j]
            k = j + 1
            history.append(abs(g[j + 1]) / bnorm)
            if hj1 != 0.0:
                V[j + 1] = w / hj1
            if abs(g[j + 1]) <= tol * bnorm or hj1 == 0.0 or its >= max_iters:
                break
        y = np.zeros(k)
        for i in range(k - 1, -1, -1):
            y[i] = (g[i] - H[i, i + 1:k] @ y[i + 1:k]) / H[i, i]
        x = x + Z[:k].T @ y
