"""Pins of the FP64 multigrid oracle (oracle/multigrid.py): transfer
adjointness, symmetry and definiteness of the V-cycle, the coarsest-level
sweeps against their closed-form matrix polynomial, and MG-preconditioned CG
against a dense direct solve and against Jacobi-preconditioned CG, the
smoothing weights against the closed form of the Chebyshev polynomial, and a
two-level V-cycle against its error-propagation matrix."""

import numpy as np
import pytest

from oracle import multigrid as MG
from oracle import pcg as PCG
from oracle import stencil as S


def dense(op, shape):
    n = int(np.prod(shape))
    M = np.zeros((n, n))
    for i in range(n):
        e = np.zeros(n)
        e[i] = 1.0
        M[:, i] = op(e.reshape(shape)).reshape(-1)
    return M


def test_transfers_are_adjoint_on_odd_lattices(rng):
    u = rng.standard_normal((5, 6, 7))
    v = rng.standard_normal(MG.coarse_shape(u.shape))
    assert MG.coarse_shape((5, 6, 7)) == (3, 3, 4)
    assert np.isclose(np.sum(MG.restrict(u) * v), np.sum(u * MG.prolong(v, u.shape)))
    # restriction sums, so it preserves the total
    assert np.isclose(MG.restrict(u).sum(), u.sum())


def test_coarse_operator_coefficients():
    a = np.full((4, 4, 4), 0.5)
    lv = MG.hierarchy(3.0, a)
    assert len(lv) == 1                       # 64 sites <= MIN_SITES: one level
    a = np.full((16, 16, 16), 0.5)
    lv = MG.hierarchy(3.0, a)
    assert [l.a.shape for l in lv] == [(16, 16, 16), (8, 8, 8)]
    assert lv[1].c == 6.0 and np.all(lv[1].a == 4.0)


@pytest.fixture
def small_levels(monkeypatch):
    monkeypatch.setattr(MG, "MIN_SITES", 8)


def test_vcycle_is_symmetric_positive_definite(rng, small_levels):
    shape = (5, 6, 7)
    a = rng.uniform(0.0, 3.0, shape) * (rng.random(shape) < 0.5) + 0.01
    levels = MG.hierarchy(2.0, a)
    assert len(levels) >= 3
    M = dense(lambda r: MG.vcycle(levels, r), shape)
    assert np.allclose(M, M.T, atol=1e-12 * np.abs(M).max())
    assert np.linalg.eigvalsh(0.5 * (M + M.T)).min() > 0.0


def test_single_level_is_the_jacobi_polynomial(rng):
    shape = (3, 4, 5)
    a = rng.uniform(0.1, 2.0, shape)
    levels = MG.hierarchy(1.5, a)
    assert len(levels) == 1
    A = dense(levels[0].apply, shape)
    Dinv = np.diag(1.0 / levels[0].d.reshape(-1))
    G = np.eye(A.shape[0]) - MG.OMEGA_COARSE * Dinv @ A
    # M = sum_{k < nu} G^k omega D^-1
    M = np.zeros_like(A)
    Gk = np.eye(A.shape[0])
    for _ in range(MG.NU_COARSE):
        M += Gk @ (MG.OMEGA_COARSE * Dinv)
        Gk = Gk @ G
    r = rng.standard_normal(shape)
    assert np.allclose(MG.vcycle(levels, r).reshape(-1), M @ r.reshape(-1), rtol=1e-12, atol=1e-14)


def test_smoothing_weights_are_the_chebyshev_polynomial():
    """(1 - w1 t)(1 - w2 t) = T2(s(t)) / T2(s(0)) with T2(x) = 2 x^2 - 1 and
    s(t) = (hi + lo - 2 t) / (hi - lo): the two sweeps' error polynomial is
    the scaled Chebyshev polynomial of the damped interval, bounded there by
    1 / T2(s(0)) and within [-1, 1] on all of (0, 2]."""
    lo, hi = MG.CHEB_LO, MG.CHEB_HI
    w1, w2 = MG.SMOOTH_WEIGHTS
    assert MG.NU == 2 and w1 < w2
    t = np.linspace(0.0, 2.0, 2001)
    s = (hi + lo - 2.0 * t) / (hi - lo)
    s0 = (hi + lo) / (hi - lo)
    cheb = (2.0 * s ** 2 - 1.0) / (2.0 * s0 ** 2 - 1.0)
    poly = (1.0 - w1 * t) * (1.0 - w2 * t)
    assert np.allclose(poly, cheb, rtol=0, atol=1e-14)
    on = (t >= lo) & (t <= hi)
    assert np.max(np.abs(poly[on])) <= 1.0 / (2.0 * s0 ** 2 - 1.0) + 1e-15
    assert np.max(np.abs(poly[t > 0])) < 1.0
    # degree 1 is the single sweep of weight 2 / (lo + hi)
    assert np.isclose(MG.chebyshev_weights(1, lo, hi)[0], 2.0 / (lo + hi))


def test_two_level_vcycle_is_its_error_propagation(rng, monkeypatch):
    """With two levels, I - M A = S (I - P B R A) S, S = (I - w2 D^-1 A)(I - w1 D^-1 A)
    the smoother's error propagation and B the coarse sweeps' polynomial
    sum_{k < nu} G_c^k w_c D_c^-1 (G_c = I - w_c D_c^-1 A_c): the recursive
    V-cycle against the matrix form of the two-grid method."""
    monkeypatch.setattr(MG, "MIN_SITES", 40)
    shape = (4, 5, 6)
    a = rng.uniform(0.01, 2.0, shape)
    levels = MG.hierarchy(1.7, a)
    assert len(levels) == 2
    f, cl = levels
    A = dense(f.apply, shape)
    Ac = dense(cl.apply, cl.a.shape)
    n, nc = A.shape[0], Ac.shape[0]
    R = np.zeros((nc, n))
    for i in range(n):
        e = np.zeros(n)
        e[i] = 1.0
        R[:, i] = MG.restrict(e.reshape(shape)).reshape(-1)
    P = R.T
    Dinv = np.diag(1.0 / f.d.reshape(-1))
    Dcinv = np.diag(1.0 / cl.d.reshape(-1))
    w1, w2 = MG.SMOOTH_WEIGHTS
    I = np.eye(n)
    S = (I - w2 * Dinv @ A) @ (I - w1 * Dinv @ A)
    Gc = np.eye(nc) - MG.OMEGA_COARSE * Dcinv @ Ac
    B = np.zeros_like(Ac)
    Gk = np.eye(nc)
    for _ in range(MG.NU_COARSE):
        B += Gk @ (MG.OMEGA_COARSE * Dcinv)
        Gk = Gk @ Gc
    E = S @ (I - P @ B @ R @ A) @ S
    M = dense(lambda r: MG.vcycle(levels, r), shape)
    assert np.allclose(I - M @ A, E, rtol=0, atol=1e-11)


def _drug_like(shape, rng):
    """Implicit-Euler drug operator: c = D/dx^2 = 96, a = 1/dt + psi (+ vessel exchange)."""
    c = 9.6e3 / 100.0
    a = np.full(shape, 1.0 / 60.0 + 0.01)
    vessel = rng.random(shape) < 0.1
    a[vessel] += 2.0 * rng.uniform(0.5, 1.5, vessel.sum())
    b = rng.uniform(0.0, 1.0, shape) / 60.0 + np.where(vessel, 2.0, 0.0)
    return c, a, b


def test_mg_pcg_matches_direct_solve(rng, small_levels):
    shape = (6, 7, 9)
    c, a, b = _drug_like(shape, rng)
    x, info = MG.mg_pcg(c, a, b, np.zeros(shape), 1e-12, 500)
    A = dense(lambda u: c * S.laplacian_sum(u) + a * u, shape)
    xs = np.linalg.solve(A, b.reshape(-1)).reshape(shape)
    assert info.converged
    assert np.max(np.abs(x - xs)) <= 1e-8 * np.max(np.abs(xs))


def test_mg_pcg_needs_far_fewer_iterations_than_jacobi(rng):
    shape = (32, 32, 32)
    c, a, b = _drug_like(shape, rng)
    x_mg, i_mg = MG.mg_pcg(c, a, b, np.zeros(shape), 1e-8, 2000)
    d = S.jacobi_diagonal(shape, c, a)
    x_j, i_j = PCG.pcg(lambda u: c * S.laplacian_sum(u) + a * u, b, np.zeros(shape), d, 1e-8, 5000)
    assert i_mg.converged and i_j.converged
    assert i_mg.iterations * 5 < i_j.iterations
    assert np.max(np.abs(x_mg - x_j)) <= 1e-6 * np.max(np.abs(x_j))


@pytest.mark.parametrize("shape,children", [((16, 16, 16), 8), ((1, 32, 48), 4), ((1, 1, 600), 2)])
def test_coarse_coupling_is_consistent_rediscretisation(shape, children):
    """On a quadratic field u = sum over the lattice's extended directions of
    x^2 (cell centres), the coarse operator applied to u sampled at the
    aggregates' centres equals the number of children times the fine
    operator's value at interior sites (the sum restriction convention):
    the coarse Laplacian is the rediscretised one, whatever the number of
    coarsened directions."""
    c = 3.0
    levels = MG.hierarchy(c, np.zeros(shape))
    assert len(levels) >= 2
    f, cs = levels[0], levels[1]
    def quad(shp, spacing, offset):
        grids = np.meshgrid(*[spacing * np.arange(n) + offset for n in shp], indexing="ij")
        return sum(g ** 2 for g, n in zip(grids, shp) if n > 1)
    u = quad(shape, 1.0, 0.0)
    U = quad(cs.a.shape, 2.0, 0.5)                 # aggregate centres in fine cell units
    fine = f.apply(u)[tuple(slice(1, -1) if n > 2 else slice(None) for n in shape)]
    coarse = cs.apply(U)[tuple(slice(1, -1) if n > 2 else slice(None) for n in cs.a.shape)]
    assert np.allclose(fine, fine.flat[0]) and np.allclose(coarse, coarse.flat[0])
    assert np.isclose(coarse.flat[0], children * fine.flat[0])


def test_flat_lattice_mg_pcg(rng):
    """A 2-D lattice coarsens in-plane; MG-PCG stays far ahead of Jacobi."""
    shape = (1, 64, 96)
    c, a, b = _drug_like(shape, rng)
    assert len(MG.hierarchy(c, a)) >= 3
    x_mg, i_mg = MG.mg_pcg(c, a, b, np.zeros(shape), 1e-8, 2000)
    d = S.jacobi_diagonal(shape, c, a)
    x_j, i_j = PCG.pcg(lambda u: c * S.laplacian_sum(u) + a * u, b, np.zeros(shape), d, 1e-8, 5000)
    assert i_mg.converged and i_j.converged
    assert i_mg.iterations * 4 < i_j.iterations
    assert np.max(np.abs(x_mg - x_j)) <= 1e-6 * np.max(np.abs(x_j))
