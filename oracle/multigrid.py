"""FP64 reference of the geometric-multigrid preconditioner (test infrastructure only).

The paper preconditions its CG solves with algebraic multigrid (BoomerAMG,
Section 2.4); on the uniform CA lattice the natural counterpart is a
geometric V-cycle.  This module is the plain definition of that V-cycle and
of CG preconditioned by it, used to check the GPU kernels.

Operator on every level: (A u)_i = c_l S_l(u)_i + a_l,i u_i, with S_l the
Neumann neighbour-difference sum of laplacian_sum on the level's lattice,
diagonal d_l = c_l n_l + a_l (n_l = number of in-box face neighbours).

Hierarchy: level l+1 halves every extent (ceil(n/2); an extent of 1 stays
1); site I of level l+1 owns the children 2I + {0,1}^3 that exist on level
l.  Coefficients: c_{l+1} = c_l 2^k / 4, k the number of extents of level l
above 1 (the Laplacian rediscretised at twice the spacing in those k
directions and scaled by the 2^k times larger volume: 2 c_l on a 3-D
lattice, c_l on a flat one), and a_{l+1,I} = sum of the children's a_l
(Galerkin for the reaction).  Coarsening stops at the first level with at
most MIN_SITES sites or with every extent 1.
Transfers: restriction R = sum over children; prolongation P = R^T (copy to
children).  Smoother: Jacobi sweeps x <- x + omega (rhs - A x) / d.  Above
the coarsest level every V-cycle applies NU = 2 sweeps before the coarse
correction with the weights SMOOTH_WEIGHTS = (omega_1, omega_2), the
reciprocals of the roots of the degree-2 Chebyshev polynomial on the
interval [CHEB_LO, CHEB_HI] of the spectrum of D^-1 A that the smoother is
to damp (a Chebyshev polynomial smoother: its error polynomial
(1 - omega_1 t)(1 - omega_2 t) is the least one on that interval), and the
same two sweeps in the opposite order after it.  The coarsest level applies
NU_COARSE sweeps of weight OMEGA_COARSE.

V-cycle z = M r: on each level above the coarsest, the pre-sweeps from
x = 0, rhs_{l+1} = R (rhs_l - A_l x_l); on the coarsest, the NU_COARSE sweeps
from x = 0; on the way up x_l += P x_{l+1} followed by the post-sweeps.  The
post-smoother is the adjoint of the pre-smoother (the same polynomial in
D^-1 A) and the coarsest sweeps are a polynomial in D^-1 A too, so M is
symmetric; it is positive definite while the sweeps converge (the smoother's
error polynomial stays within [-1, 1] on the spectrum of D^-1 A, which lies
in (0, 2) for these diagonally dominant operators).

Choice of preconditioner: the paper preconditions CG with algebraic
multigrid (Section 2.4) and fixes no smoother; on the drug operator (weak
reaction next to the diffusion coupling) two Chebyshev-weighted sweeps per
side take about 60 % fewer CG iterations than one sweep of weight 0.8.
"""

from __future__ import annotations

import numpy as np

from .pcg import SolveInfo
from .stencil import laplacian_sum, neighbour_count

CHEB_LO, CHEB_HI = 0.5, 2.0
NU = 2
OMEGA_COARSE = 0.8
NU_COARSE = 16
MIN_SITES = 512


def chebyshev_weights(k: int, lo: float, hi: float):
    """Reciprocals of the k roots of the Chebyshev polynomial T_k mapped
    from [-1, 1] onto [lo, hi], the largest root first."""
    mid, half = 0.5 * (hi + lo), 0.5 * (hi - lo)
    return tuple(1.0 / (mid + half * np.cos(np.pi * (2 * i + 1) / (2 * k))) for i in range(k))


SMOOTH_WEIGHTS = chebyshev_weights(NU, CHEB_LO, CHEB_HI)


def coarse_shape(shape):
    return tuple((n + 1) // 2 for n in shape)


def restrict(u):
    """Sum over the (existing) children of every coarse site."""
    out = np.zeros(coarse_shape(u.shape))
    for dz in (0, 1):
        for dy in (0, 1):
            for dx in (0, 1):
                part = u[dz::2, dy::2, dx::2]
                out[:part.shape[0], :part.shape[1], :part.shape[2]] += part
    return out


def prolong(uc, shape):
    """Copy every coarse value to its children (the transpose of restrict)."""
    return np.repeat(np.repeat(np.repeat(uc, 2, 0), 2, 1), 2, 2)[:shape[0], :shape[1], :shape[2]]


class Level:
    def __init__(self, c, a):
        self.c = float(c)
        self.a = np.asarray(a, dtype=np.float64)
        self.d = self.c * neighbour_count(self.a.shape) + self.a

    def apply(self, u):
        return self.c * laplacian_sum(u) + self.a * u

    def sweep(self, x, rhs, omega):
        return x + omega * (rhs - self.apply(x)) / self.d


def hierarchy(c, a):
    """Levels of the operator c S + diag(a) on a's lattice."""
    levels = [Level(c, a)]
    while levels[-1].a.size > MIN_SITES and max(levels[-1].a.shape) > 1:
        lv = levels[-1]
        k = sum(1 for n in lv.a.shape if n > 1)
        levels.append(Level(lv.c * 2.0 ** k / 4.0, restrict(lv.a)))
    return levels


def vcycle(levels, r):
    """z = M r."""
    def solve(l, rhs):
        lv = levels[l]
        x = np.zeros_like(rhs)
        if l == len(levels) - 1:
            for _ in range(NU_COARSE):
                x = lv.sweep(x, rhs, OMEGA_COARSE)
            return x
        for omega in SMOOTH_WEIGHTS:
            x = lv.sweep(x, rhs, omega)
        xc = solve(l + 1, restrict(rhs - lv.apply(x)))
        x = x + prolong(xc, rhs.shape)
        for omega in reversed(SMOOTH_WEIGHTS):
            x = lv.sweep(x, rhs, omega)
        return x

    return solve(0, np.asarray(r, dtype=np.float64))


def mg_pcg(c, a, b, x0, rtol, maxit):
    """CG preconditioned by one V-cycle per iteration; stops when
    ||r|| <= rtol ||b|| (recursive residual).  Returns (x, SolveInfo)."""
    levels = hierarchy(c, a)
    A = levels[0].apply
    b = np.asarray(b, dtype=np.float64)
    x = np.array(x0, dtype=np.float64)
    bn = np.linalg.norm(b)
    if bn == 0.0:
        return np.zeros_like(b), SolveInfo(0, 0.0, True)
    r = b - A(x)
    if np.linalg.norm(r) <= rtol * bn:
        return x, SolveInfo(0, float(np.linalg.norm(r) / bn), True)
    z = vcycle(levels, r)
    p = z.copy()
    rho = float(np.sum(r * z))
    for it in range(1, maxit + 1):
        q = A(p)
        alpha = rho / float(np.sum(p * q))
        x += alpha * p
        r -= alpha * q
        rn = np.linalg.norm(r)
        if rn <= rtol * bn:
            return x, SolveInfo(it, float(np.linalg.norm(b - A(x)) / bn), True)
        z = vcycle(levels, r)
        rho_new = float(np.sum(r * z))
        p = z + (rho_new / rho) * p
        rho = rho_new
    return x, SolveInfo(maxit, float(np.linalg.norm(b - A(x)) / bn), False)
