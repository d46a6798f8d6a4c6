"""Flexible GMRES and GMRES (Sec. 2; Table 1; the coarsest solve of Sec. 3).

FGMRES(m) with right preconditioning M (Saad, Iterative Methods for Sparse
Linear Systems, Alg. 9.6): Arnoldi on A M with the preconditioned vectors
z_j kept, classical Gram-Schmidt applied twice, Givens rotations for the
least-squares problem.  A cycle ends when the rotated residual estimate
|g_{j+1}| falls to tol * ||b|| or after m steps; then x += Z y.  Between
cycles the residual is recomputed as b - A x.  Convergence of a solve is
declared on that recomputed (true) residual only.

GMRES is FGMRES with M = identity.  The coarsest system is solved with
GMRES on the even-odd Schur complement (Sec. 3) to a relative residual
epsilon of the Schur system.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

from .lattice import vdot, norm


@dataclass
class KrylovInfo:
    iterations: int = 0
    cycles: int = 0
    converged: bool = False
    true_residual: float = float("nan")   # ||b - A x|| / ||b|| at the end (nan if not computed)
    history: list = field(default_factory=list)


def givens(a: complex, b: complex):
    """c (real), s with [[c, s], [-conj(s), c]] (a, b)^T = (rho, 0)^T."""
    r = np.hypot(abs(a), abs(b))
    if r == 0.0:
        return 1.0, 0.0
    if a == 0:
        return 0.0, 1.0 if b == 0 else np.conj(b) / abs(b)
    c = abs(a) / r
    s = (a / abs(a)) * np.conj(b) / r
    return c, s


def fgmres(A, b, M=None, m: int = 10, tol: float = 1e-10, max_cycles: int = 100,
           final_residual: bool = True) -> tuple:
    """Solve A x = b from x0 = 0; returns (x, KrylovInfo).

    A, M: callables on arrays shaped like b.  M = None means no preconditioner.
    The cycle loop stops when the true residual ||b - A x|| <= tol * ||b|| or
    after max_cycles cycles.  With final_residual = False the residual after
    the last allowed cycle is not recomputed (inner solves need only x).
    """
    info = KrylovInfo()
    bnorm = norm(b)
    x = np.zeros_like(b)
    if bnorm == 0.0:
        info.converged = True
        info.true_residual = 0.0
        return x, info
    target = tol * bnorm
    r = b.copy()
    beta = bnorm
    for cycle in range(max_cycles):
        info.cycles = cycle + 1
        V = [r / beta]
        Z = []
        H = np.zeros((m + 1, m), dtype=np.complex128)
        cs = np.zeros(m)
        sn = np.zeros(m, dtype=np.complex128)
        g = np.zeros(m + 1, dtype=np.complex128)
        g[0] = beta
        k = 0
        for j in range(m):
            zj = V[j] if M is None else M(V[j])
            Z.append(zj)
            w = A(zj)
            h = np.zeros(j + 2, dtype=np.complex128)
            for _ in range(2):
                c = np.array([vdot(V[i], w) for i in range(j + 1)])
                for i in range(j + 1):
                    w = w - c[i] * V[i]
                h[:j + 1] += c
            h[j + 1] = norm(w)
            for i in range(j):                      # earlier rotations
                t = cs[i] * h[i] + sn[i] * h[i + 1]
                h[i + 1] = -np.conj(sn[i]) * h[i] + cs[i] * h[i + 1]
                h[i] = t
            hn = h[j + 1]
            cs[j], sn[j] = givens(h[j], h[j + 1])
            h[j] = cs[j] * h[j] + sn[j] * h[j + 1]
            h[j + 1] = 0.0
            g[j + 1] = -np.conj(sn[j]) * g[j]
            g[j] = cs[j] * g[j]
            H[:j + 2, j] = h
            k = j + 1
            info.iterations += 1
            info.history.append(abs(g[j + 1]) / bnorm)
            if abs(g[j + 1]) <= target or hn == 0.0:
                break
            V.append(w / hn)
        y = np.zeros(k, dtype=np.complex128)
        for i in range(k - 1, -1, -1):              # back substitution R y = g
            y[i] = (g[i] - np.dot(H[i, i + 1:k], y[i + 1:k])) / H[i, i]
        for i in range(k):
            x = x + y[i] * Z[i]
        last = cycle == max_cycles - 1
        if last and not final_residual:
            break
        r = b - A(x)
        beta = norm(r)
        info.true_residual = beta / bnorm
        if beta <= target:
            info.converged = True
            break
    return x, info


def gmres(A, b, m: int = 50, tol: float = 1e-1, max_cycles: int = 20, final_residual=True):
    return fgmres(A, b, M=None, m=m, tol=tol, max_cycles=max_cycles, final_residual=final_residual)


def coarsest_solve(eo, b, tol: float, m: int, max_cycles: int):
    """Odd-even preconditioned GMRES: GMRES on Dhat to ||rhat|| <= tol ||bhat||, then z_o."""
    bh = eo.schur_rhs(b)
    xe, info = gmres(eo.schur_apply, bh, m=m, tol=tol, max_cycles=max_cycles, final_residual=True)
    return eo.back_substitute(xe, b), info


def cgls(A, AH, b, tol: float = 1e-10, max_iter: int = 100000):
    """CGNR in its least-squares form (CG on A^+ A x = A^+ b that updates s = b - A x; Saad, Iterative
    Methods for Sparse Linear Systems, Sec. 8.3): the plain Krylov solver the method is compared
    with (Sec. 3.3 of the paper).  Stops when ||s|| <= tol ||b||; returns (x, KrylovInfo) with
    the true residual recomputed at the end.

        x = 0, s = b, r = A^+ s, p = r, gamma = |r|^2
        repeat: q = A p; alpha = gamma / |q|^2; x += alpha p; s -= alpha q;
                r = A^+ s; gamma' = |r|^2; p = r + (gamma'/gamma) p
    """
    info = KrylovInfo()
    bnorm = norm(b)
    x = np.zeros_like(b)
    if bnorm == 0.0:
        info.converged, info.true_residual = True, 0.0
        return x, info
    s = b.copy()
    r = AH(s)
    p = r.copy()
    gamma = norm(r) ** 2
    for it in range(max_iter):
        q = A(p)
        alpha = gamma / norm(q) ** 2
        x = x + alpha * p
        s = s - alpha * q
        info.iterations = it + 1
        if norm(s) <= tol * bnorm:
            break
        r = AH(s)
        g2 = norm(r) ** 2
        p = r + (g2 / gamma) * p
        gamma = g2
    info.true_residual = norm(b - A(x)) / bnorm
    info.converged = info.true_residual <= tol
    return x, info


def cg_lanczos_coefficients(Aop, v, steps: int):
    """CG on a Hermitian positive definite operator from the start vector v: the step lengths alpha_j
    and the ratios beta_j = |r_{j+1}|^2 / |r_j|^2 (stopping early when the residual vanishes)."""
    r = v.copy()
    p = r.copy()
    gamma = norm(r) ** 2
    alphas, betas = [], []
    for _ in range(steps):
        q = Aop(p)
        alpha = gamma / vdot(p, q).real
        r = r - alpha * q
        g2 = norm(r) ** 2
        alphas.append(alpha)
        betas.append(g2 / gamma)
        if g2 == 0.0:
            break
        p = r + (g2 / gamma) * p
        gamma = g2
    return np.array(alphas), np.array(betas)


def lanczos_tridiagonal(alphas, betas) -> np.ndarray:
    """The Lanczos matrix T_k of CG (Saad, Sec. 6.7.3): diagonal 1/alpha_j + beta_{j-1}/alpha_{j-1},
    off-diagonal sqrt(beta_j)/alpha_j; its eigenvalues (Ritz values) approximate the operator's."""
    k = len(alphas)
    T = np.zeros((k, k))
    for j in range(k):
        T[j, j] = 1.0 / alphas[j] + (betas[j - 1] / alphas[j - 1] if j > 0 else 0.0)
        if j + 1 < k:
            T[j, j + 1] = T[j + 1, j] = np.sqrt(betas[j]) / alphas[j]
    return T
