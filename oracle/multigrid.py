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
children).  Smoother: weighted Jacobi, weight OMEGA.

V-cycle z = M r: on each level above the coarsest, NU sweeps from x = 0,
rhs_{l+1} = R (rhs_l - A_l x_l); on the coarsest, NU_COARSE sweeps from
x = 0; on the way up x_l += P x_{l+1} followed by NU sweeps.  Equal pre- and
post-smoothing with the same Jacobi weight make M symmetric; it is positive
definite while the sweeps converge.
"""

from __future__ import annotations

import numpy as np

from .pcg import SolveInfo
from .stencil import laplacian_sum, neighbour_count

OMEGA = 0.8
NU = 1
NU_COARSE = 16
MIN_SITES = 512


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

    def sweep(self, x, rhs):
        return x + OMEGA * (rhs - self.apply(x)) / self.d


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
                x = lv.sweep(x, rhs)
            return x
        for _ in range(NU):
            x = lv.sweep(x, rhs)
        xc = solve(l + 1, restrict(rhs - lv.apply(x)))
        x = x + prolong(xc, rhs.shape)
        for _ in range(NU):
            x = lv.sweep(x, rhs)
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
