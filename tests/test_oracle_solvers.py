"""Pins for the oracle's stencil operators and PCG solves (oxygen and drugs).

Each test checks the oracle against something it does not compute itself:
an explicitly assembled dense matrix, numpy.linalg.solve, closed-form
solutions of the discrete equations, conservation laws and the discrete
maximum principle.
"""

import math

import numpy as np
import pytest

from oracle import params as Pm
from oracle import stencil as S
from oracle.model import drug_solve, o2_initial, o2_solve
from oracle.pcg import pcg


def dense_matrix(shape, coupling, reaction):
    """Assemble A by enumerating each site's face neighbours with plain loops."""
    nz, ny, nx = shape
    n = nx * ny * nz
    A = np.zeros((n, n))
    r = np.asarray(reaction).reshape(-1)
    for z in range(nz):
        for y in range(ny):
            for x in range(nx):
                i = x + nx * (y + ny * z)
                A[i, i] += r[i]
                for dx, dy, dz in ((1, 0, 0), (-1, 0, 0), (0, 1, 0), (0, -1, 0), (0, 0, 1), (0, 0, -1)):
                    xx, yy, zz = x + dx, y + dy, z + dz
                    if 0 <= xx < nx and 0 <= yy < ny and 0 <= zz < nz:
                        j = xx + nx * (yy + ny * zz)
                        A[i, i] += coupling
                        A[i, j] -= coupling
    return A


def random_state(shape, rng, p_vessel=0.12, p_cell=0.4):
    u = rng.random(shape)
    st = np.full(shape, Pm.EMPTY, dtype=np.uint8)
    st[u < p_vessel + p_cell] = Pm.PROLIF
    st[u < p_vessel] = Pm.VESSEL
    q = rng.random(shape)
    st[(st == Pm.PROLIF) & (q < 0.2)] = Pm.QUIESC
    st[(st == Pm.PROLIF) & (q > 0.9)] = Pm.DEAD
    st[(st == Pm.EMPTY) & (q > 0.95)] = Pm.STROMA
    return st


@pytest.mark.parametrize("shape", [(1, 1, 5), (2, 3, 4), (3, 3, 3), (4, 2, 5)])
def test_operator_matches_dense_assembly(shape, rng):
    u = rng.standard_normal(shape)
    reaction = rng.random(shape)
    A = dense_matrix(shape, 2.5, reaction)
    assert np.allclose(S.apply_operator(u, 2.5, reaction).reshape(-1), A @ u.reshape(-1),
                       rtol=1e-14, atol=1e-12)
    assert np.allclose(S.jacobi_diagonal(shape, 2.5, reaction).reshape(-1), np.diag(A), rtol=0, atol=1e-14)
    assert np.allclose(A, A.T)


def test_laplacian_kills_constants_and_is_symmetric(rng):
    shape = (5, 6, 7)
    assert np.allclose(S.laplacian_sum(np.full(shape, 3.7)), 0.0, atol=1e-14)
    u, v = rng.standard_normal(shape), rng.standard_normal(shape)
    assert math.isclose(np.sum(u * S.laplacian_sum(v)), np.sum(v * S.laplacian_sum(u)), rel_tol=1e-12)
    assert np.sum(u * S.laplacian_sum(u)) > 0


@pytest.mark.parametrize("shape", [(3, 3, 3), (4, 5, 6), (6, 6, 6)])
def test_o2_pcg_matches_dense_solve(shape, rng):
    cfg = Pm.Config(nx=shape[2], ny=shape[1], nz=shape[0], rtol_o2=1e-13)
    st = random_state(shape, rng)
    st[0, 0, 0] = Pm.VESSEL
    K_prev = rng.uniform(0.0, 20.0, shape)
    K, info = o2_solve(st, K_prev, cfg)
    A = dense_matrix(shape, S.o2_coupling(cfg), S.o2_reaction(st, K_prev, cfg))
    exact = np.linalg.solve(A, S.o2_rhs(st, cfg).reshape(-1))
    assert info.converged and info.rel_residual < 1e-12
    assert np.allclose(K.reshape(-1), exact, rtol=1e-10, atol=1e-10 * np.abs(exact).max())


@pytest.mark.parametrize("shape", [(3, 3, 3), (4, 5, 6), (6, 6, 6)])
def test_drug_pcg_matches_dense_solve(shape, rng):
    cfg = Pm.Config(nx=shape[2], ny=shape[1], nz=shape[0], n_drugs=2, rtol_drug=1e-13,
                    uptake_G=(0.0, 0.3, 0.0))
    st = random_state(shape, rng)
    perf = rng.lognormal(0, 0.5, shape)
    G_old = rng.random(shape)
    for d in range(2):
        G, info = drug_solve(st, perf, G_old, 0.8, cfg, d)
        A = dense_matrix(shape, S.drug_coupling(cfg, d), S.drug_reaction(st, perf, cfg, d))
        exact = np.linalg.solve(A, S.drug_rhs(st, perf, G_old, 0.8, cfg, d).reshape(-1))
        assert info.converged
        assert np.allclose(G.reshape(-1), exact, rtol=1e-10, atol=1e-12)


def cosh_profile(N, cfg, K_const):
    """Closed-form discrete solution: vessel at i = 0, consuming cells at i >= 1."""
    c = S.o2_coupling(cfg)
    k = cfg.phi_K / (cfg.K1 + K_const)
    theta = math.acosh(1.0 + k / (2.0 * c))
    ci = np.array([math.cosh((N - 0.5 - i) * theta) for i in range(N)])
    C = cfg.r_K * cfg.K0 / (cfg.r_K * ci[0] + c * (ci[0] - ci[1]))
    return C * ci


@pytest.mark.parametrize("N", [8, 33, 64])
def test_o2_discrete_cosh_profile_1d(N):
    cfg = Pm.Config(nx=N, ny=1, nz=1, rtol_o2=1e-14)
    st = np.full((1, 1, N), Pm.PROLIF, dtype=np.uint8)
    st[0, 0, 0] = Pm.VESSEL
    K_const = 7.0
    K, info = o2_solve(st, np.full(st.shape, K_const), cfg)
    ref = cosh_profile(N, cfg, K_const)
    assert np.allclose(K.reshape(-1), ref, rtol=1e-11, atol=1e-12 * ref.max())


def test_o2_discrete_cosh_profile_3d_planar():
    N, M = 24, 5
    cfg = Pm.Config(nx=N, ny=M, nz=M, rtol_o2=1e-14)
    st = np.full((M, M, N), Pm.QUIESC, dtype=np.uint8)
    st[:, :, 0] = Pm.VESSEL
    K_const = 3.0
    K, _ = o2_solve(st, np.full(st.shape, K_const), cfg)
    ref = cosh_profile(N, cfg, K_const)
    assert np.allclose(K, np.broadcast_to(ref, K.shape), rtol=1e-11, atol=1e-12 * ref.max())


def test_o2_cosh_profile_continuum_limit():
    # With the consumption length lam = sqrt(D/k) fixed, the discrete profile
    # tends to cosh((L - x)/lam)/cosh(L/lam), scaled to the computed value at
    # the vessel node, with error O(dx^2).
    errs = []
    for refine in (1, 2, 4):
        dx = 10.0 / refine
        N = 40 * refine
        cfg = Pm.Config(nx=N, ny=1, nz=1, dx=dx, rtol_o2=1e-15)
        K_const = 5.0
        st = np.full((1, 1, N), Pm.PROLIF, dtype=np.uint8)
        st[0, 0, 0] = Pm.VESSEL
        K, _ = o2_solve(st, np.full(st.shape, K_const), cfg)
        K = K.reshape(-1)
        k = cfg.phi_K / (cfg.K1 + K_const)
        lam = math.sqrt(cfg.D_K / k)
        # the last node's mirror ghost puts the no-flux plane at L = (N - 1/2) dx
        L = (N - 0.5) * dx
        x = np.arange(N) * dx
        cont = K[0] * np.cosh((L - x) / lam) / np.cosh(L / lam)
        errs.append(np.max(np.abs(K - cont)))
    rates = [math.log2(errs[i] / errs[i + 1]) for i in range(2)]
    assert all(1.8 < r < 2.2 for r in rates), (errs, rates)


def test_o2_maximum_principle_and_flux_balance(rng):
    shape = (10, 11, 12)
    cfg = Pm.Config(nx=12, ny=11, nz=10, rtol_o2=1e-12)
    st = random_state(shape, rng)
    K_prev = rng.uniform(0, 20, shape)
    K, info = o2_solve(st, K_prev, cfg)
    assert K.min() >= -1e-9 and K.max() <= cfg.K0 * (1 + 1e-12)
    # summing all rows of the system: the Neumann Laplacian cancels
    supply = np.sum(np.where(st == Pm.VESSEL, cfg.r_K * (cfg.K0 - K), 0.0))
    cons = np.sum(np.where(S.is_consumer(st), cfg.phi_K / (cfg.K1 + K_prev) * K, 0.0))
    bnorm = np.linalg.norm(S.o2_rhs(st, cfg))
    assert abs(supply - cons) <= 1e-12 * bnorm * math.sqrt(K.size) + 1e-9


def test_o2_picard_fixed_point(rng):
    shape = (8, 8, 8)
    cfg = Pm.Config(nx=8, ny=8, nz=8, rtol_o2=1e-12, picard_tol=1e-10)
    st = random_state(shape, rng)
    K, iters = o2_initial(st, cfg)
    assert iters < cfg.picard_maxit
    # K solves the nonlinear steady equation to the Picard tolerance
    nonlin = (S.o2_coupling(cfg) * S.laplacian_sum(K)
              + np.where(S.is_consumer(st), cfg.phi_K * K / (cfg.K1 + K), 0.0)
              + np.where(st == Pm.VESSEL, cfg.r_K * K, 0.0) - S.o2_rhs(st, cfg))
    assert np.linalg.norm(nonlin) <= 1e-8 * np.linalg.norm(S.o2_rhs(st, cfg))


@pytest.mark.parametrize("modes", [(1, 0, 0), (2, 3, 1), (0, 4, 5)])
def test_drug_single_fourier_mode_decay(modes):
    nz, ny, nx = 8, 9, 10
    cfg = Pm.Config(nx=nx, ny=ny, nz=nz, rtol_drug=1e-14)
    st = np.full((nz, ny, nx), Pm.EMPTY, dtype=np.uint8)
    perf = np.ones(st.shape)
    mz, my, mx = modes
    z, y, x = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    G = (np.cos(np.pi * mx * (x + 0.5) / nx) * np.cos(np.pi * my * (y + 0.5) / ny)
         * np.cos(np.pi * mz * (z + 0.5) / nz))
    c = S.drug_coupling(cfg, 0)
    lam = sum(4 * math.sin(math.pi * m / (2 * n)) ** 2 for m, n in ((mx, nx), (my, ny), (mz, nz)))
    factor = 1.0 / (1.0 + cfg.dt * (cfg.psi_G[0] + c * lam))
    G0 = G.copy()
    for n in range(1, 4):
        G, _ = drug_solve(st, perf, G, 0.0, cfg, 0)
        assert np.allclose(G, G0 * factor ** n, rtol=1e-11, atol=1e-13)


def test_drug_mass_conservation_without_reaction(rng):
    shape = (7, 8, 9)
    cfg = Pm.Config(nx=9, ny=8, nz=7, rtol_drug=1e-14, psi_G=(0.0, 0.0, 0.0))
    st = np.full(shape, Pm.PROLIF, dtype=np.uint8)       # no vessels: kappa = 0
    perf = np.ones(shape)
    G = rng.random(shape)
    m0 = G.sum()
    for _ in range(100):
        G, _ = drug_solve(st, perf, G, 1.0, cfg, 0)
    assert abs(G.sum() - m0) <= 1e-12 * m0


def test_drug_maximum_principle(rng):
    shape = (9, 9, 9)
    cfg = Pm.Config(nx=9, ny=9, nz=9, rtol_drug=1e-13)
    st = random_state(shape, rng)
    perf = rng.lognormal(0, 0.5, shape)
    G = rng.random(shape) * 0.5
    for G0 in (1.0, 0.2, 0.0):
        Gn, _ = drug_solve(st, perf, G, G0, cfg, 0)
        assert Gn.min() >= -1e-12
        assert Gn.max() <= max(G.max(), G0) * (1 + 1e-12)
        G = Gn


def test_drug_all_vessel_uniform_steady_state():
    shape = (4, 4, 4)
    cfg = Pm.Config(nx=4, ny=4, nz=4, rtol_drug=1e-14)
    st = np.full(shape, Pm.VESSEL, dtype=np.uint8)
    perf = np.ones(shape)
    G0 = 0.7
    G_star = cfg.kappa_G[0] * G0 / (cfg.kappa_G[0] + cfg.psi_G[0])
    G, _ = drug_solve(st, perf, np.full(shape, G_star), G0, cfg, 0)
    assert np.allclose(G, G_star, rtol=1e-13)
    # from zero the uniform iterate contracts by (1/dt) / (1/dt + psi + kappa) per step
    G = np.zeros(shape)
    rate = (1 / cfg.dt) / (1 / cfg.dt + cfg.psi_G[0] + cfg.kappa_G[0])
    for n in range(1, 5):
        G, _ = drug_solve(st, perf, G, G0, cfg, 0)
        assert np.allclose(G, G_star * (1 - rate ** n), rtol=1e-12)


def test_pcg_zero_rhs_and_exact_start(rng):
    A = lambda u: 2.0 * u
    b = np.zeros(10)
    x, info = pcg(A, b, rng.random(10), np.full(10, 2.0), 1e-8, 100)
    assert info.iterations == 0 and np.all(x == 0)
    b = rng.random(10)
    x, info = pcg(A, b, b / 2.0, np.full(10, 2.0), 1e-8, 100)
    assert info.iterations == 0
