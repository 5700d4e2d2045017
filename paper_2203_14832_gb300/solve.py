"""GMRES for linear systems whose product is an NNCA H^2 matvec, e.g. the Nystrom
matrix of a second-kind integral equation (Sec. 5, Experiment 5).

The Krylov vectors stay on the device as torch tensors; the products are the
library's (any callable y = A x on tensors shaped like b).
"""
from __future__ import annotations

import math


def gmres(matvec, b, tol: float = 1e-10, restart: int = 60, maxiter: int = 300):
    """Restarted GMRES(restart) from x0 = 0, Arnoldi by modified Gram-Schmidt,
    the small least-squares problem by Givens rotations (Saad's algorithm).

    Stops when the Arnoldi residual estimate ||b - A x|| / ||b|| <= tol, and at
    every restart and at the end checks the true residual. Returns (x, iterations,
    list of relative residual estimates, one per iteration)."""
    import torch
    bnorm = float(torch.linalg.norm(b))
    x = torch.zeros_like(b)
    if bnorm == 0.0:
        return x, 0, []
    hist = []
    it = 0
    r = b.clone()
    beta = bnorm
    while it < maxiter:
        V = [r / beta]
        H = [[0.0] * restart for _ in range(restart + 1)]   # H[i][j], (m+1) x m
        cs, sn = [0.0] * restart, [0.0] * restart
        g = [0.0] * (restart + 1)
        g[0] = beta
        k_used = 0
        for j in range(restart):
            w = matvec(V[j])
            for i in range(j + 1):   # modified Gram-Schmidt
                hij = float(torch.dot(w, V[i]))
                H[i][j] = hij
                w = w - hij * V[i]
            hn = float(torch.linalg.norm(w))
            H[j + 1][j] = hn
            # previous rotations on the new column, then the rotation that zeroes H[j+1][j]
            for i in range(j):
                t = cs[i] * H[i][j] + sn[i] * H[i + 1][j]
                H[i + 1][j] = -sn[i] * H[i][j] + cs[i] * H[i + 1][j]
                H[i][j] = t
            den = math.hypot(H[j][j], H[j + 1][j])
            cs[j], sn[j] = (H[j][j] / den, H[j + 1][j] / den) if den > 0 else (1.0, 0.0)
            H[j][j] = cs[j] * H[j][j] + sn[j] * H[j + 1][j]
            H[j + 1][j] = 0.0
            g[j + 1] = -sn[j] * g[j]
            g[j] = cs[j] * g[j]
            it += 1
            k_used = j + 1
            hist.append(abs(g[j + 1]) / bnorm)
            if hist[-1] <= tol or it >= maxiter or hn == 0.0:
                break
            V.append(w / hn)
        # x += V_k y with H_k y = g_k (upper triangular)
        y = [0.0] * k_used
        for i in range(k_used - 1, -1, -1):
            s = g[i] - sum(H[i][l] * y[l] for l in range(i + 1, k_used))
            y[i] = s / H[i][i]
        for i in range(k_used):
            x = x + y[i] * V[i]
        r = b - matvec(x)
        beta = float(torch.linalg.norm(r))
        if beta / bnorm <= tol or hist[-1] <= tol:
            break
    return x, it, hist
