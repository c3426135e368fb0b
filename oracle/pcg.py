"""Textbook Jacobi-preconditioned conjugate gradients (FP64).

The paper solves its symmetric positive definite systems with CG (Section
2.4.1: BoomerAMG-preconditioned for the drugs and the linearised oxygen,
Jacobi-preconditioned inside the oxygen Newton loop), relative tolerance 1e-8.
This oracle uses the Jacobi preconditioner throughout.

Stopping rule: iterate while ||r_k||_2 > rtol * ||b||_2 (recursive residual)
and k < maxit; the returned relative residual is recomputed from b - A x.
"""

from __future__ import annotations

import dataclasses

import numpy as np


@dataclasses.dataclass
class SolveInfo:
    iterations: int
    rel_residual: float      # ||b - A x|| / ||b|| recomputed at exit
    converged: bool


def pcg(apply_A, b: np.ndarray, x0: np.ndarray, diag: np.ndarray,
        rtol: float, maxit: int):
    """Solve A x = b from x0 with the preconditioner M = diag(A)."""
    b = np.asarray(b, dtype=np.float64)
    x = np.array(x0, dtype=np.float64, copy=True)
    bnorm = float(np.sqrt(np.sum(b * b)))
    if bnorm == 0.0:
        x[...] = 0.0
        return x, SolveInfo(0, 0.0, True)
    r = b - apply_A(x)
    z = r / diag
    p = z.copy()
    rho = float(np.sum(r * z))
    rnorm = float(np.sqrt(np.sum(r * r)))
    k = 0
    while rnorm > rtol * bnorm and k < maxit:
        q = apply_A(p)
        alpha = rho / float(np.sum(p * q))
        x += alpha * p
        r -= alpha * q
        z = r / diag
        rho_new = float(np.sum(r * z))
        rnorm = float(np.sqrt(np.sum(r * r)))
        beta = rho_new / rho
        p = z + beta * p
        rho = rho_new
        k += 1
    true_r = b - apply_A(x)
    rel = float(np.sqrt(np.sum(true_r * true_r))) / bnorm
    return x, SolveInfo(k, rel, rnorm <= rtol * bnorm)
