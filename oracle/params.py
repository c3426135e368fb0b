"""Model parameters (Table 1) and the readings used where the paper is silent.

Every default cites Table 1 of the paper or states the reading it implements.
Units: micrometres, minutes, mmHg for oxygen, normalised plasma units for the
drugs.
"""

from __future__ import annotations

import dataclasses
import math
from typing import Tuple

# Lattice states (uint8).  The paper's L(x) in {0 empty, 1 cancer, 2 stroma}
# and G(x) in {0, 1} (Section 2.2.1 and 2.2.2) are merged into one code:
EMPTY = 0      # no cell
PROLIF = 1     # cancer cell, cycling
QUIESC = 2     # cancer cell whose last division found no free neighbour
DEAD = 3       # killed in this CA update; acts as EMPTY, cleared at the next update
VESSEL = 4     # functional vessel cross-section
STROMA = 5     # stroma cell: occupies space, consumes oxygen, never divides

CANCER_STATES = (PROLIF, QUIESC)
CONSUMER_STATES = (PROLIF, QUIESC, STROMA)   # the set X_c of Eq. (oxygen)
FREE_STATES = (EMPTY, DEAD)

# Philox counter word 3 ("purpose") for each random draw.
PURPOSE_VESSEL = 0
PURPOSE_CANCER = 1
PURPOSE_PHI = 2
PURPOSE_KILL = 3
PURPOSE_VASCULAR = 4


def _three(v):
    return (v, v, v)


@dataclasses.dataclass
class Config:
    """One simulation: lattice, numerics and model parameters."""

    nx: int
    ny: int
    nz: int
    precision: str = "f64"          # "f64" or "f32": storage precision of the compared path
    n_drugs: int = 1
    seed: int = 0

    # numerics
    dx: float = 10.0                # Table 1, Delta x (micrometres)
    dt: float = 60.0                # one CA step in minutes (hourly steps)
    rtol_o2: float = 1e-8           # Section 2.4: relative tolerance 1e-8
    rtol_drug: float = 1e-8
    maxit: int = 20000
    picard_tol: float = 1e-8        # oxygen fixed point, ||dK||/||K||
    picard_maxit: int = 100
    # 0: one solve of the lagged linearisation per step (Section 2.4.1,
    # "linear approximation"); 1: the nonlinear quasi-steady equation, as the
    # fixed point of that linearisation iterated from K_prev each step
    o2_nonlinear: int = 0
    # time discretisation (Section 2.4.1).  Drugs: 0 implicit Euler, 1
    # Crank-Nicolson, over drug_substeps equal sub-steps of dt.  Oxygen: 0
    # quasi-steady (s_K = 0); 1 implicit Euler, 2 Crank-Nicolson in time
    # (s_K = 1) over o2_substeps sub-steps, consumption linearised about the
    # field at the start of each sub-step
    drug_scheme: int = 0
    drug_substeps: int = 1
    o2_scheme: int = 0
    o2_substeps: int = 1
    # CA update: 0 the 27-colour Gauss-Seidel sweep (ca.py); 1 synchronous,
    # a contested site going to the higher phi (Algorithm 2; ca_sync.py)
    ca_mode: int = 0

    # VEGF field, Eq. (vac_v) without Avastin (A = 0), Table 1: solved every
    # step after oxygen when vegf = 1, stepped like the drugs (drug_scheme,
    # drug_substeps); released by cells at rate a_V * Vc
    vegf: int = 0
    D_V: float = 3.52e3             # um^2/min
    psi_V: float = 1e-2             # 1/min
    a_V: float = 6.66e-6            # 1/min, VEGF secretion slope
    # vascular birth-death CA (Eq. vascular_module) every vessel_interval steps
    # (0 = off; 12 = Delta v of 720 min at hourly steps)
    vessel_interval: int = 0
    V_low: float = 1e-6             # Table 1
    V_high: float = 1e-3            # reading: not published
    p_death: float = 0.1            # reading: not published
    beta_birth: float = 0.05        # reading: Pr_sprout 2 pi r0 h_c Delta v lumped (not published)
    V_sprout: float = 1e-4          # reading: not published
    # plasma pharmacokinetics per drug: 0 one-compartment exponential
    # (plasma_decay), 1 Michaelis-Menten (mm_vmax, mm_km; Eq. for fluorouracil),
    # 2 three-compartment (epi_*; Eq. for epirubicin)
    pk_model: Tuple[int, int, int] = (0, 0, 0)
    mm_vmax: float = 1.75           # ug/mL/min, Table 1
    mm_km: float = 27.0             # ug/mL, Table 1
    epi_w: Tuple[float, float, float] = (18e3, 957e3, 25e3)   # mL, Table 1
    epi_q2: float = 0.918e3         # mL/min, Table 1
    epi_q3: float = 0.25e3
    epi_cl2: float = 0.983e3
    ode_substeps: int = 60          # RK4 step h = dt / ode_substeps = 1 min (Section 2.4.2)

    # oxygen, Eq. (oxygen) and Table 1
    D_K: float = 1.05e5             # diffusion, um^2/min
    phi_K: float = 900.0            # consumption, mmHg/min per consuming site (reading)
    K1: float = 2.5                 # half-maximal consumption, mmHg
    K0: float = 20.0                # blood oxygen, mmHg
    r_K: float = 1.88e4             # supply P_K 2 pi r0 / dx^2, 1/min per vessel site

    # drugs, Eq. (chemo) and Table 1; index 0 cyclophosphamide, 1 epirubicin,
    # 2 fluorouracil
    D_G: Tuple[float, float, float] = _three(9.6e3)
    psi_G: Tuple[float, float, float] = _three(1e-2)
    kappa_G: Tuple[float, float, float] = _three(2.0)       # reading: free parameter
    uptake_G: Tuple[float, float, float] = _three(0.0)      # optional live-cell uptake
    dose_interval: int = 21                                  # steps between boluses
    dose_peak: Tuple[float, float, float] = _three(1.0)      # plasma peak = max G_{i,0}
    plasma_decay: Tuple[float, float, float] = (
        3.93e3 / 2430e3,    # cl3/u, cyclophosphamide (Eq. intrachemo3)
        0.983e3 / 18e3,     # cl2/w1, epirubicin elimination only
        1.75 / 27.0,        # v_max/k_m, fluorouracil in its linear regime
    )
    kill_b: Tuple[int, int, int] = (1, 1, 1)                 # Beta(1, b) sensitivity

    # cell cycle, Eq. (cellcycle), Table 1
    T_cycle: float = 3.74 * 24 * 60   # T_min = 3.74 days, in minutes
    K_phi: float = 1.4

    # intracellular p53 and VEGF, Eqs. (odep53), (odevegf), Table 1
    k1: float = 4e-4
    k1p: float = 0.01
    K_p53: float = 0.01
    k2: float = 2e-3
    k2p: float = 0.01
    k2pp: float = -2e-4
    J5: float = 0.04
    K_V: float = 0.01

    @property
    def shape(self):
        return (self.nz, self.ny, self.nx)

    @property
    def n_sites(self):
        return self.nx * self.ny * self.nz

    def replace(self, **kw) -> "Config":
        return dataclasses.replace(self, **kw)


def lambda0_vessel(vessel_mean: float = 0.12) -> float:
    """Poisson intensity giving P(at least one vessel) = vessel_mean."""
    return -math.log(1.0 - vessel_mean)
