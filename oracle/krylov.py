"""Restarted GMRES(m), FP64, test infrastructure only (Sec. 2.3).

Textbook GMRES (Saad & Schultz 1986): Arnoldi with modified Gram-Schmidt,
Givens rotations on the Hessenberg matrix, restart after m inner iterations,
initial guess x0 = 0.  Stops when the rotated residual estimate falls to
rtol * ||b||, or after max_it matrix-vector products in total (the paper
requires the tolerance to be met within 100 iterations).
"""
import math

import torch


def gmres(matvec, b, m=30, rtol=1e-1, max_it=100):
    n = b.numel()
    x = torch.zeros(n, dtype=b.dtype)
    beta0 = float(torch.linalg.vector_norm(b))
    stats = dict(iterations=0, restarts=0, converged=False, rel_res=0.0)
    if beta0 == 0.0:
        stats["converged"] = True
        return x, stats
    it = 0
    r = b.clone()
    while True:
        beta = float(torch.linalg.vector_norm(r))
        if beta <= rtol * beta0:
            stats.update(converged=True, rel_res=beta / beta0)
            break
        if it >= max_it:
            stats["rel_res"] = beta / beta0
            break
        V = [r / beta]
        H = [[0.0] * m for _ in range(m + 1)]
        cs, sn = [0.0] * m, [0.0] * m
        g = [0.0] * (m + 1)
        g[0] = beta
        k = 0
        res = beta
        for j in range(m):
            w = matvec(V[j])
            it += 1
            for i in range(j + 1):
                h = float(torch.dot(w, V[i]))
                H[i][j] = h
                w = w - h * V[i]
            hn = float(torch.linalg.vector_norm(w))
            H[j + 1][j] = hn
            for i in range(j):
                t = cs[i] * H[i][j] + sn[i] * H[i + 1][j]
                H[i + 1][j] = -sn[i] * H[i][j] + cs[i] * H[i + 1][j]
                H[i][j] = t
            den = math.hypot(H[j][j], H[j + 1][j])
            cs[j], sn[j] = (1.0, 0.0) if den == 0.0 else (H[j][j] / den, H[j + 1][j] / den)
            H[j][j] = cs[j] * H[j][j] + sn[j] * H[j + 1][j]
            H[j + 1][j] = 0.0
            g[j + 1] = -sn[j] * g[j]
            g[j] = cs[j] * g[j]
            res = abs(g[j + 1])
            k = j + 1
            if hn != 0.0:
                V.append(w / hn)
            if res <= rtol * beta0 or it >= max_it or hn == 0.0:
                break
        # back substitution H[:k,:k] y = g[:k]
        y = [0.0] * k
        for i in range(k - 1, -1, -1):
            s = g[i] - sum(H[i][l] * y[l] for l in range(i + 1, k))
            y[i] = s / H[i][i]
        for i in range(k):
            x = x + y[i] * V[i]
        stats["restarts"] += 1
        if res <= rtol * beta0:
            stats.update(converged=True, rel_res=res / beta0)
            break
        if it >= max_it:
            stats["rel_res"] = res / beta0
            break
        r = b - matvec(x)          # true residual at restart (not counted as an iteration)
    stats["iterations"] = it
    return x, stats
