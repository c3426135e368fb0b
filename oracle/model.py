"""Algorithm 1 of the paper on the 3-D lattice: initialisation and time loop.

Initialisation (Algorithm 1, steps 2-5):
  * vessels and cancer cells are seeded from the input maps: a site holds a
    vessel if u_v < p_vessel, else a cancer cell if u_c < p_cell (u are 24-bit
    Philox uniforms with distinct purposes);
  * every cancer cell draws phi ~ U(0, 1) (Section 2.2.4: "all cancer cells");
  * the initial oxygen solves Eq. (oxygen) with s_K = 0 by the fixed point of
    the lagged linearisation (Picard iteration from K = K0), standing in for
    the paper's nonlinear steady solve;
  * P = Vc = 0 and G_d = 0 (reading: the initial intracellular levels are not
    given, so they start at zero and evolve from the first step on).

One step n -> n+1 (Algorithm 1, loop body, VEGF/Avastin omitted):
  1. plasma levels G_{d,0}(t^{n+1}) (closed form);
  2. oxygen: quasi-steady solve with the consumption linearised about the
     previous K (Section 2.4.1), x0 = previous K; with o2_nonlinear set, the
     linearisation is iterated to its fixed point from the previous K instead
     (the nonlinear quasi-steady equation, solved exactly);
  3. drugs: one implicit-Euler step of Eq. (chemo), x0 = G^n (or sub-steps,
     implicit Euler or Crank-Nicolson, per drug_scheme/drug_substeps); with
     o2_scheme set, step 2 is the time-dependent oxygen equation instead;
  4. ODEs for phi, P, Vc with the new K;
  (with vegf = 1 the VEGF field of Eq. (vac_v), A = 0, is solved after
  oxygen; with vessel_interval set the vascular automaton runs after the cell
  update every vessel_interval steps; the plasma levels follow pk_model)
  5. the CA update (Section 2.5) with Philox draws keyed by the step index n:
     the 27-colour sweep, or with ca_mode 1 the synchronous update with
     Algorithm 2's higher-phi rule.
"""

from __future__ import annotations

import dataclasses
from typing import List

import numpy as np

from . import params as Pm
from . import stencil as S
from .ca import ca_update
from .ca_sync import ca_update_sync
from .odes import ode_update
from .pcg import SolveInfo, pcg
from .philox import site_uniform
from .pk import plasma_level
from .vascular import VascularStats, vascular_update


@dataclasses.dataclass
class StepStats:
    step: int
    o2: SolveInfo               # None when the O2 solve is the Picard iteration
    drugs: List[SolveInfo]
    committed: int
    kills: int
    divisions: int
    blocked: int
    counts: np.ndarray          # sites per state code 0..5 after the step
    vegf: SolveInfo = None      # the VEGF solve (vegf = 1)
    vessel_births: int = 0
    vessel_deaths: int = 0


def seed_lattice(cfg: Pm.Config, p_cell, p_vessel):
    """Initial states and cycle clocks from the maps (Algorithm 1, steps 2 and 4)."""
    sites = np.arange(cfg.n_sites, dtype=np.uint64)
    u_v = site_uniform(cfg.seed, sites, 0, Pm.PURPOSE_VESSEL).reshape(cfg.shape)
    u_c = site_uniform(cfg.seed, sites, 0, Pm.PURPOSE_CANCER).reshape(cfg.shape)
    u_p = site_uniform(cfg.seed, sites, 0, Pm.PURPOSE_PHI).reshape(cfg.shape)
    pv = np.asarray(p_vessel, dtype=np.float64).reshape(cfg.shape)
    pc = np.asarray(p_cell, dtype=np.float64).reshape(cfg.shape)
    state = np.where(u_v < pv, Pm.VESSEL, np.where(u_c < pc, Pm.PROLIF, Pm.EMPTY)).astype(np.uint8)
    phi = np.where(state == Pm.PROLIF, u_p, 0.0)
    return state, phi


def o2_solve(state, K_prev, cfg: Pm.Config, rtol=None):
    """One lagged-linearised oxygen solve, x0 = K_prev."""
    coupling = S.o2_coupling(cfg)
    reaction = S.o2_reaction(state, K_prev, cfg)
    diag = S.jacobi_diagonal(state.shape, coupling, reaction)
    b = S.o2_rhs(state, cfg)
    return pcg(lambda u: S.apply_operator(u, coupling, reaction), b, K_prev, diag,
               cfg.rtol_o2 if rtol is None else rtol, cfg.maxit)


def o2_residual_nonlinear(state, K, cfg: Pm.Config):
    """F(K) of Eq. (oxygen) with s_K = 0 and the consumption kept nonlinear:
    D_K/dx^2 S(K) + phi_K K/(K1 + K) [consumer] + r_K (K - K0) [vessel]
    (its zero is the quasi-steady oxygen field)."""
    K = np.asarray(K, dtype=np.float64)
    cons = np.where(S.is_consumer(state), cfg.phi_K * K / (cfg.K1 + K), 0.0)
    ves = np.where(S.is_vessel(state), cfg.r_K * (K - cfg.K0), 0.0)
    return S.o2_coupling(cfg) * S.laplacian_sum(K) + cons + ves


def o2_picard(state, K_start, cfg: Pm.Config):
    """Fixed point of the lagged linearisation K -> A(K)^{-1} b iterated from
    K_start until ||dK|| <= picard_tol ||K|| (or picard_maxit): the solution
    of the nonlinear quasi-steady oxygen equation.  Returns (K, iterations)."""
    K = np.array(K_start, dtype=np.float64)
    iters = 0
    for iters in range(1, cfg.picard_maxit + 1):
        K_new, _ = o2_solve(state, K, cfg)
        change = float(np.sqrt(np.sum((K_new - K) ** 2)))
        norm = float(np.sqrt(np.sum(K_new ** 2)))
        K = K_new
        if norm == 0.0 or change <= cfg.picard_tol * norm:
            break
    return K, iters


def o2_initial(state, cfg: Pm.Config):
    """Picard fixed point of the lagged linearisation, starting from K = K0."""
    return o2_picard(state, np.full(state.shape, cfg.K0, dtype=np.float64), cfg)


def drug_solve(state, perf, G_old, G0_next, cfg: Pm.Config, d: int):
    """One implicit-Euler step of Eq. (chemo) for drug d, x0 = G^n."""
    coupling = S.drug_coupling(cfg, d)
    reaction = S.drug_reaction(state, perf, cfg, d)
    diag = S.jacobi_diagonal(state.shape, coupling, reaction)
    b = S.drug_rhs(state, perf, G_old, G0_next, cfg, d)
    return pcg(lambda u: S.apply_operator(u, coupling, reaction), b, G_old, diag,
               cfg.rtol_drug, cfg.maxit)


def drug_step(state, perf, G_old, step_index: int, cfg: Pm.Config, d: int):
    """Eq. (chemo) over one CA step as drug_substeps sub-steps of h = dt/m,
    each by implicit Euler (drug_scheme 0) or Crank-Nicolson (1), the plasma
    level taken at the sub-step's end (and start, for Crank-Nicolson); each
    solve starts from the previous sub-step's field.  Returns (G, infos)."""
    m = cfg.drug_substeps
    h = cfg.dt / m
    scheme = 1 if cfg.drug_scheme == 0 else 2
    coupling = S.drug_coupling(cfg, d)
    a0 = S.drug_reaction0(state, perf, cfg, d)
    kappa = S.drug_kappa(state, perf, cfg, d)
    reaction = S.drug_reaction(state, perf, cfg, d, mass=S.time_mass(scheme, h))
    diag = S.jacobi_diagonal(state.shape, coupling, reaction)
    G = np.asarray(G_old, dtype=np.float64)
    infos = []
    for j in range(m):
        t_old = (step_index + j / m) * cfg.dt
        t_new = (step_index + (j + 1) / m) * cfg.dt
        f_old = kappa * plasma_level(cfg, d, t_old)
        f_new = kappa * plasma_level(cfg, d, t_new)
        b = S.time_rhs(scheme, h, G, coupling, a0, f_old, f_new)
        G, info = pcg(lambda u: S.apply_operator(u, coupling, reaction), b, G, diag, cfg.rtol_drug, cfg.maxit)
        infos.append(info)
    return G, infos


def vegf_step(state, V_old, Vc, cfg: Pm.Config):
    """Eq. (vac_v) with A = 0 over one CA step, stepped like the drugs
    (drug_scheme, drug_substeps): reaction psi_V, source a_V Vc at cells
    (constant over the step: Vc is the previous step's).  Returns (V, infos)."""
    m = cfg.drug_substeps
    h = cfg.dt / m
    scheme = 1 if cfg.drug_scheme == 0 else 2
    coupling = cfg.D_V / cfg.dx ** 2
    a0 = np.full(state.shape, cfg.psi_V)
    reaction = S.time_mass(scheme, h) + a0
    diag = S.jacobi_diagonal(state.shape, coupling, reaction)
    f = np.where(S.is_consumer(state), cfg.a_V * np.asarray(Vc, dtype=np.float64), 0.0)
    V = np.asarray(V_old, dtype=np.float64)
    infos = []
    for _ in range(m):
        b = S.time_rhs(scheme, h, V, coupling, a0, f, f)
        V, info = pcg(lambda u: S.apply_operator(u, coupling, reaction), b, V, diag, cfg.rtol_drug, cfg.maxit)
        infos.append(info)
    return V, infos


def o2_transient_step(state, K_old, cfg: Pm.Config):
    """Time-dependent Eq. (oxygen) (s_K = 1) over one CA step as o2_substeps
    sub-steps of h = dt/m by implicit Euler (o2_scheme 1) or Crank-Nicolson
    (2), the consumption of each sub-step linearised about its starting field
    (Section 2.4.1's linear approximation).  Returns (K, infos)."""
    if cfg.o2_nonlinear:
        raise ValueError("the nonlinear oxygen solve is the quasi-steady form only")
    m = cfg.o2_substeps
    h = cfg.dt / m
    coupling = S.o2_coupling(cfg)
    f = S.o2_rhs(state, cfg)
    K = np.asarray(K_old, dtype=np.float64)
    infos = []
    for _ in range(m):
        a0 = S.o2_reaction(state, K, cfg)
        reaction = a0 + S.time_mass(cfg.o2_scheme, h)
        diag = S.jacobi_diagonal(state.shape, coupling, reaction)
        b = S.time_rhs(cfg.o2_scheme, h, K, coupling, a0, f, f)
        K, info = pcg(lambda u: S.apply_operator(u, coupling, reaction), b, K, diag, cfg.rtol_o2, cfg.maxit)
        infos.append(info)
    return K, infos


def plasma_levels(cfg: Pm.Config, t: float):
    return [plasma_level(cfg, d, t) for d in range(cfg.n_drugs)]


class OracleSim:
    """The oracle's counterpart of one library handle (one replicate)."""

    def __init__(self, cfg: Pm.Config, p_cell, perf, p_vessel, initial_o2=True):
        self.cfg = cfg
        self.perf = np.asarray(perf, dtype=np.float64).reshape(cfg.shape)
        self.state, self.phi = seed_lattice(cfg, p_cell, p_vessel)
        self.P = np.zeros(cfg.shape)
        self.Vc = np.zeros(cfg.shape)
        self.G = [np.zeros(cfg.shape) for _ in range(cfg.n_drugs)]
        self.V = np.zeros(cfg.shape)
        self.step_index = 0
        self.history: List[StepStats] = []
        if initial_o2:
            self.K, self.picard_iterations = o2_initial(self.state, cfg)
        else:
            self.K = np.full(cfg.shape, cfg.K0)
            self.picard_iterations = 0

    # stages of one step, callable one by one
    def solve_o2(self):
        if self.cfg.o2_scheme:
            self.K, infos = o2_transient_step(self.state, self.K, self.cfg)
            return infos[-1]
        if self.cfg.o2_nonlinear:
            self.K, self.picard_iterations = o2_picard(self.state, self.K, self.cfg)
            return None
        self.K, info = o2_solve(self.state, self.K, self.cfg)
        return info

    def solve_vegf(self):
        self.V, infos = vegf_step(self.state, self.V, self.Vc, self.cfg)
        return infos[-1]

    def update_vessels(self):
        """The vascular automaton after the cell update of steps n with
        (n + 1) % vessel_interval == 0."""
        if not self.cfg.vessel_interval or (self.step_index + 1) % self.cfg.vessel_interval:
            return VascularStats()
        self.state, vs = vascular_update(self.state, self.V, self.cfg, self.step_index)
        return vs

    def solve_drugs(self):
        infos = []
        for d in range(self.cfg.n_drugs):
            self.G[d], sub = drug_step(self.state, self.perf, self.G[d], self.step_index, self.cfg, d)
            infos.append(sub[-1])
        return infos

    def update_odes(self):
        self.phi, self.P, self.Vc = ode_update(self.state, self.phi, self.P, self.Vc,
                                               self.K, self.cfg)

    def update_ca(self):
        update = ca_update_sync if self.cfg.ca_mode == 1 else ca_update
        self.state, self.phi, self.P, self.Vc, st = update(
            self.state, self.phi, self.P, self.Vc, self.K, self.G, self.cfg, self.step_index)
        return st

    def step(self, n_steps: int = 1):
        for _ in range(n_steps):
            o2 = self.solve_o2()
            vegf = self.solve_vegf() if self.cfg.vegf else None
            drugs = self.solve_drugs()
            self.update_odes()
            st = self.update_ca()
            vs = self.update_vessels()
            counts = np.bincount(self.state.reshape(-1), minlength=6)[:6]
            self.history.append(StepStats(self.step_index, o2, drugs, st.committed,
                                          st.kills, st.divisions, st.blocked, counts, vegf,
                                          vs.births, vs.deaths))
            self.step_index += 1
        return self.history[-1] if self.history else None
