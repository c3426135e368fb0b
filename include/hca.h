/*
 * hca.h -- C ABI of the GB300 (sm_103a) library for the data-parallel hot path
 * of one time step of the hybrid cellular automaton (HCA) model of
 * Lai, Tasken et al., "A scalable solver for a stochastic, hybrid cellular
 * automaton model of personalized breast cancer therapy" (arXiv:2105.00448).
 *
 * One step (Algorithm 1, loop body) on a 3-D lattice of nx*ny*nz sites:
 *   1. plasma levels G_{d,0}(t^{n+1}) of the drugs (Eq. intrachemo3, closed form);
 *   2. quasi-steady oxygen K: Eq. (oxygen) with s_K = 0 and the consumption
 *      linearised about the previous K (Section 2.4.1), 7-point stencil,
 *      Jacobi-preconditioned CG;
 *   3. drugs G_d: one implicit-Euler step of Eq. (chemo), 7-point stencil, CG;
 *   4. per-cell ODEs for phi, P, Vc (Eqs. cellcycle, odep53, odevegf);
 *   5. the stochastic CA update of committed cancer cells (Sections 2.2.1 and
 *      2.5): Beta-CDF drug kill (Eq. 1), else division into the free Moore
 *      neighbour with the highest K, resolved in a fixed 27-colour sweep with
 *      counter-based Philox4x32-10 draws keyed by (seed, site, step).
 *
 * Conventions for every function below:
 *   - Return value: HCA_OK (0) or a negative HCA_ERR_* code.  No function
 *     aborts, throws or prints.  hca_status_string() names a code.
 *   - Site order: linear index x + nx*(y + ny*z) (x fastest); field arrays are
 *     dense in that order (no padding) on the caller's side.
 *   - Precision: HCA_FP64 stores every field in double; HCA_FP32 stores fields
 *     in float and keeps all inner products and residual norms in double.
 *     Field buffers passed in or out use the handle's precision.
 *   - Streams: all device work of a handle is ordered on cfg.stream (a
 *     cudaStream_t; NULL = the legacy default stream).  hca_step and
 *     hca_stage return once the work is queued; reads, writes and
 *     hca_get_stats synchronise that stream before they return.
 *   - Ownership: the library allocates and owns all device state of a handle
 *     and frees it in hca_destroy.  Caller buffers are only read or written
 *     during the call and are never retained.
 *   - "on_device" flags: 1 = the pointer is CUDA device memory of the current
 *     device, 0 = host memory (pageable or pinned).
 *   - Thread safety: one handle must not be used by two threads at once.
 */
#ifndef HCA_H
#define HCA_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define HCA_ABI_VERSION 1

/* status codes */
#define HCA_OK 0
#define HCA_ERR_ARG (-1)           /* bad argument: size, pointer, index, config value */
#define HCA_ERR_CUDA (-2)          /* a CUDA runtime call failed */
#define HCA_ERR_OOM (-3)           /* device allocation failed */
#define HCA_ERR_NONFINITE (-4)     /* an input map or a field holds NaN/Inf */
#define HCA_ERR_NOCONV (-5)        /* a CG solve hit maxit; the step completed with its last iterate */
#define HCA_ERR_TIMEOUT (-6)       /* a bounded device wait gave up */
#define HCA_ERR_UNIMPLEMENTED (-7)
#define HCA_ERR_STATE (-8)         /* call not valid in the handle's current state */
#define HCA_ERR_IO (-9)            /* a checkpoint file could not be opened, read or written */

/* precision */
#define HCA_FP64 0
#define HCA_FP32 1

/* lattice state codes (uint8).  The paper's L(x) in {empty, cancer, stroma}
 * and vessel indicator G(x) (Sections 2.2.1-2.2.2) merged into one code. */
#define HCA_EMPTY 0
#define HCA_PROLIF 1   /* cancer cell, cycling */
#define HCA_QUIESC 2   /* cancer cell whose last division found no free neighbour */
#define HCA_DEAD 3     /* killed in the last CA update; acts as EMPTY, cleared next update */
#define HCA_VESSEL 4   /* functional vessel */
#define HCA_STROMA 5   /* stroma cell: occupies space, consumes O2, never divides */

/* field selection for hca_read_fields / hca_write_fields; fields are packed
 * one after another in increasing bit order, each nx*ny*nz elements */
#define HCA_FIELD_O2 (1u << 0)     /* oxygen K (mmHg) */
#define HCA_FIELD_DRUG0 (1u << 1)  /* drug concentrations G_0..G_2 (plasma-peak units) */
#define HCA_FIELD_DRUG1 (1u << 2)
#define HCA_FIELD_DRUG2 (1u << 3)
#define HCA_FIELD_PHI (1u << 4)    /* cell-cycle clock phi */
#define HCA_FIELD_P53 (1u << 5)    /* intracellular p53, P */
#define HCA_FIELD_VEGFC (1u << 6)  /* intracellular VEGF, Vc */
#define HCA_FIELD_PERF (1u << 7)   /* perfusion map (the vessel-exchange scale) */
#define HCA_FIELD_VEGF (1u << 8)   /* extracellular VEGF, V (ug/mL; vegf = 1) */
/* read only, FP32 handles with defect correction: the low-order FP32 words of
 * the solved fields (the solution is the two-word sum hi + lo, the FP32
 * field above being hi; Section 2.4.1's rtol-1e-8 solves are met by hi + lo) */
#define HCA_FIELD_O2_LO (1u << 9)
#define HCA_FIELD_DRUG0_LO (1u << 10)
#define HCA_FIELD_DRUG1_LO (1u << 11)
#define HCA_FIELD_DRUG2_LO (1u << 12)
#define HCA_FIELD_VEGF_LO (1u << 13)

/* stages for hca_stage; HCA_STAGE_ALL runs one full step (as hca_step(h, 1)) */
#define HCA_STAGE_O2 (1u << 0)
#define HCA_STAGE_DRUGS (1u << 1)
#define HCA_STAGE_ODE (1u << 2)
#define HCA_STAGE_CA (1u << 3)
#define HCA_STAGE_ADVANCE (1u << 4) /* step counter n -> n+1 */
#define HCA_STAGE_ALL 0x1Fu

/* CG preconditioner.  HCA_PC_JACOBI: diag(A), the textbook PCG of the
 * reference solver.  HCA_PC_MG: one symmetric geometric-multigrid V-cycle
 * per iteration (the lattice counterpart of the paper's algebraic-multigrid
 * preconditioned CG, Section 2.4): 2x2x2 agglomeration, coupling doubled per
 * level, reaction summed over the children, sum restriction, copy
 * prolongation, two Jacobi sweeps before the coarse correction and two after
 * it with the Chebyshev weights 1 / (1.25 +- 0.75 cos(pi/4)) (the degree-2
 * Chebyshev polynomial on [0.5, 2] of the spectrum of D^-1 A; before: the
 * smaller weight first, after: the larger first), 16 sweeps of weight 0.8 on
 * the coarsest level (<= 512 sites). */
#define HCA_PC_JACOBI 0
#define HCA_PC_MG 1

/* warm start of the oxygen CG */
#define HCA_WS_PREV 0     /* previous step's K */
#define HCA_WS_LEARNED 1  /* network guess (hca_set_warm_start_net), residual-checked */
#define HCA_WS_LEARNED_ALWAYS 2  /* network guess without the residual check (for measurement) */

/*
 * Simulation parameters.  Defaults (hca_config_default) are Table 1 of the
 * paper plus the readings listed per field.  Units: micrometres, minutes,
 * mmHg for oxygen, plasma-peak units for drugs.  Arrays of 3 are per drug:
 * index 0 cyclophosphamide, 1 epirubicin, 2 fluorouracil.
 */
typedef struct hca_config {
  uint32_t struct_size;  /* = sizeof(hca_config); checked */
  int32_t nx, ny, nz;    /* lattice, each >= 1; nx*ny*nz <= 2^31 - 1 */
  int32_t precision;     /* HCA_FP64 or HCA_FP32 */
  int32_t n_drugs;       /* 0..3 */
  uint64_t seed;         /* Philox key */

  double dx;             /* Table 1 Delta x = 10 um */
  double dt;             /* CA step, minutes (60) */
  double rtol_o2;        /* relative residual target of the oxygen solve (1e-8, Section 2.4.1) */
  double rtol_drug;      /* same for each drug solve (1e-8) */
  int32_t maxit;         /* CG iteration cap per solve */
  int32_t ode_substeps;  /* RK4 steps per dt for Vc (60: h = 1 min, Section 2.4.2) */
  double picard_tol;     /* O2 fixed point (initial field; every step with o2_nonlinear):
                            stop at ||dK||/||K|| <= tol */
  int32_t picard_maxit;
  int32_t dose_interval; /* CA steps between boluses; boluses at steps 0, I, 2I, ... */

  /* Eq. (oxygen), Table 1 */
  double D_K;    /* 1.05e5 um^2/min */
  double phi_K;  /* 900, consumption per consuming site (mmHg/min) */
  double K1;     /* 2.5 mmHg */
  double K0;     /* 20 mmHg */
  double r_K;    /* 1.88e4 /min: supply P_K 2 pi r0 / dx^2 per vessel site */

  /* Eq. (chemo), Table 1 and readings */
  double D_G[3];          /* 9.6e3 um^2/min */
  double psi_G[3];        /* 1e-2 /min */
  double kappa_G[3];      /* vessel exchange scale, times the perfusion map (reading: 2.0 /min) */
  double uptake_G[3];     /* optional uptake at live cancer sites (default 0) */
  double dose_peak[3];    /* plasma peak per bolus = max G_{d,0} (1.0) */
  double plasma_decay[3]; /* /min: cl3/u, cl2/w1, v_max/k_m */
  int32_t kill_b[3];      /* Beta(1, b) sensitivity, positive integers (Eq. 1; default 1) */

  /* Eqs. (cellcycle), (odep53), (odevegf), Table 1 */
  double T_cycle;  /* 3.74 days in minutes */
  double K_phi;    /* 1.4 */
  double k1, k1p, K_p53;         /* 4e-4, 0.01, 0.01 */
  double k2, k2p, k2pp, J5, K_V; /* 2e-3, 0.01, -2e-4, 0.04, 0.01 */

  /* precision scheme of HCA_FP32 (ignored for HCA_FP64) */
  double rtol_inner;     /* inner FP32 CG tolerance of a defect-correction sweep,
                            relative to its defect (1e-3); a sweep aims at half
                            the outer target instead when that is looser or at
                            most 8x tighter */
  int32_t max_outer;     /* defect-correction sweeps per oxygen solve (8) */

  int32_t warm_start;    /* HCA_WS_PREV */
  int32_t preconditioner; /* HCA_PC_JACOBI (default) or HCA_PC_MG (single-replicate handles) */
  int32_t threads_per_block; /* 0 = library choice (autotuned at creation); else 64, 128, 256 or 512; results do not depend on it */
  int32_t o2_nonlinear;  /* 0: one lagged-linearised oxygen solve per step (Section 2.4.1);
                            1: iterate that linearisation from the previous K to its fixed
                            point every step (picard_tol, picard_maxit), i.e. solve the
                            nonlinear quasi-steady Eq. (oxygen); steps then run from a host
                            loop (one convergence check per Picard iterate), not a graph.
                            Must match across a batch; not with HCA_WS_LEARNED*. */
  /* Time discretisation (Section 2.4.1).  With the spatial operator A_0 and
     source f, one sub-step of h = dt / substeps solves
       implicit Euler:   (1/h + A_0) u^k = u^{k-1}/h + f^k
       Crank-Nicolson:   (2/h + A_0) u^k = (2/h - A_0) u^{k-1} + f^{k-1} + f^k,
     each from x0 = u^{k-1}; the drugs' f is kappa perf G_{d,0}(t) at the
     sub-step's ends.  All four must match across a batch. */
  int32_t drug_scheme;   /* 0 implicit Euler (default), 1 Crank-Nicolson */
  int32_t drug_substeps; /* sub-steps per CA step (1) */
  int32_t o2_scheme;     /* 0 quasi-steady, s_K = 0 (default); 1 implicit Euler, 2 Crank-Nicolson
                            in time (s_K = 1), consumption linearised about each sub-step's
                            starting field; not with o2_nonlinear or HCA_WS_LEARNED* */
  int32_t o2_substeps;   /* sub-steps per CA step for o2_scheme 1, 2 (1) */
  int32_t ca_mode;       /* 0: 27-colour Gauss-Seidel sweep (default; later colours see earlier
                            daughters and deaths); 1: synchronous update (Section 2.5), every
                            committed cell decides on the lattice before the update and a site
                            picked by several parents goes to the highest phi, then the lowest
                            site index (Algorithm 2); must match across a batch */
  /* VEGF field and vascular automaton (Sections 2.2.2, 2.3), without Avastin:
     with vegf = 1, Eq. (vac_v) with A = 0, dV/dt = D_V lap V + a_V Vc [cell]
     - psi_V V, is solved every step after oxygen, stepped like the drugs
     (drug_scheme, drug_substeps; Vc of the previous step).  With
     vessel_interval > 0 the vascular birth-death automaton (Eq.
     vascular_module) runs after the cell update of every step n with
     (n + 1) % vessel_interval == 0: a vessel with V outside [V_low, V_high]
     is removed with probability p_death; a free site with V inside becomes a
     vessel with probability min(1, E V / sum_candidates V), E = beta_birth
     sum_vessels V / (V_sprout + V) (both sums in 2^-32 fixed point, exact).
     Needs vegf = 1. */
  int32_t vegf;
  int32_t vessel_interval;
  /* plasma pharmacokinetics per drug (Section 2.2.3): 0 one-compartment
     exponential (plasma_decay); 1 Michaelis-Menten, dG/dt = -mm_vmax G /
     (mm_km + G), each dose adding dose_peak to the level before it; 2 three
     compartments (epi_w, epi_q2, epi_q3, epi_cl2), doses superposed */
  int32_t pk_model[3];
  int32_t pad3;
  double D_V, psi_V, a_V;        /* 3.52e3 um^2/min, 1e-2 /min, 6.66e-6 /min (Table 1) */
  double V_low, V_high;          /* 1e-6 (Table 1), 1e-3 ug/mL */
  double p_death, beta_birth, V_sprout; /* 0.1, 0.05, 1e-4 ug/mL */
  double mm_vmax, mm_km;         /* 1.75 ug/mL/min, 27 ug/mL (Table 1) */
  double epi_w[3];               /* 18e3, 957e3, 25e3 mL (Table 1) */
  double epi_q2, epi_q3, epi_cl2; /* 0.918e3, 0.25e3, 0.983e3 mL/min (Table 1) */
  void* stream;          /* cudaStream_t, NULL = default stream */
} hca_config;

/* Per-replicate statistics of the most recent step (or stage). */
typedef struct hca_stats {
  int64_t step;                 /* steps completed */
  int32_t picard_iterations;    /* oxygen fixed point: of the last step with o2_nonlinear, else of the initial field */
  int32_t o2_iterations;        /* CG iterations of the last step's oxygen solves (all sweeps and sub-steps) */
  int32_t o2_sweeps;            /* defect-correction sweeps (1 for HCA_FP64) */
  int32_t drug_iterations[3];
  double o2_rel_residual;       /* ||b - A K|| / ||b|| recomputed at exit */
  double drug_rel_residual[3];
  int32_t not_converged;        /* bit 0: oxygen, bit 1+d: drug d hit maxit */
  int32_t pad0;
  int64_t committed, kills, divisions, blocked; /* last CA update */
  int64_t counts[6];            /* sites per state code after the last update */
  int32_t ws_used;              /* HCA_WS_LEARNED: 1 if the last oxygen solve started from the network's guess */
  int32_t pad1;
  double ws_r0_prev;            /* HCA_WS_LEARNED: ||b - A K_prev|| / ||b|| before the last oxygen solve */
  double ws_r0_learned;         /* HCA_WS_LEARNED: the same for the network's guess */
  int32_t vegf_iterations;      /* vegf = 1: CG iterations of the last step's VEGF solves */
  int32_t pad2;
  double vegf_rel_residual;
  int64_t vessel_births, vessel_deaths; /* last vascular update (0 on other steps) */
} hca_stats;

typedef struct hca_handle hca_handle;

/* Kernel classes timed by the optional per-launch profiler. */
#define HCA_KCLASS_SETUP 0      /* solve set-up: r = b - A x0, diagonal */
#define HCA_KCLASS_PASS_A 1     /* CG pass A: p = z + beta p, p.Ap */
#define HCA_KCLASS_PASS_B 2     /* CG pass B: x, z update, r.z, |r|^2 */
#define HCA_KCLASS_RESIDUAL 3   /* true residual at solve exit */
#define HCA_KCLASS_ODE 4        /* per-cell ODEs */
#define HCA_KCLASS_CA_COMPACT 5 /* CA commit compaction */
#define HCA_KCLASS_CA_COLOUR 6  /* CA colour sweeps */
#define HCA_KCLASS_OTHER 7
#define HCA_KCLASS_MG 8         /* multigrid: coarse levels, r scaling, level diagonals */
#define HCA_KCLASS_MG_RESTRICT0 9 /* multigrid: restriction of the pre-smoothed residual on the lattice */
#define HCA_KCLASS_MG_POST0 10  /* multigrid: prolongation + first post-sweep on the lattice */
#define HCA_KCLASS_MG_PRE0 11   /* multigrid: the two pre-sweeps on the lattice */
#define HCA_KCLASS_MG_LAST0 12  /* multigrid: last post-sweep on the lattice, r.z */
#define HCA_NKCLASS 13

typedef struct hca_profile {
  int64_t launches[HCA_NKCLASS];
  double ms[HCA_NKCLASS];      /* summed device time between CUDA events around each launch */
} hca_profile;

/* Fill *cfg with the defaults above for an nx*ny*nz lattice (FP64, 1 drug,
 * seed 0).  Returns HCA_ERR_ARG for a NULL pointer. */
int hca_config_default(hca_config* cfg, int32_t nx, int32_t ny, int32_t nz);

/* Create one simulation (Algorithm 1, steps 2-5): seed vessels and cancer
 * cells from the maps (vessel if u_v < p_vessel, else cancer if u_c <
 * p_cell, 24-bit Philox uniforms), phi ~ U(0,1) on cancer cells, P = Vc = 0,
 * G = 0, and the initial oxygen as the fixed point of the linearised steady
 * equation.  p_cell, perf, p_vessel: nx*ny*nz float each, site order above;
 * copied, the caller keeps ownership.  HCA_ERR_NONFINITE if a map holds
 * NaN/Inf or a probability lies outside [0, 1] or perf < 0. */
int hca_create(const hca_config* cfg, const float* p_cell, const float* perf,
               const float* p_vessel, int32_t maps_on_device, hca_handle** out);

/* Create n independent replicates (uneven lattices allowed) that advance
 * together: every kernel of a step covers all replicates in one launch.
 * cfgs[i] gives replicate i's lattice, seed and parameters; precision,
 * n_drugs, dt, threads_per_block and stream must agree across replicates.
 * Maps are arrays of n pointers. */
int hca_create_batch(int32_t n, const hca_config* cfgs, const float* const* p_cell,
                     const float* const* perf, const float* const* p_vessel,
                     int32_t maps_on_device, hca_handle** out);

/* Advance all replicates by n_steps full steps.  One step is the loop body
 * of Algorithm 1: plasma levels (Eq. intrachemo3), the oxygen solve
 * (Eq. oxygen, Section 2.4.1), the drug solves (Eq. chemo), the cell ODEs
 * (Eqs. cellcycle, odep53, odevegf; Section 2.4.2) and the CA update
 * (Sections 2.2.1, 2.5; Eq. 1).  Work is queued on the handle's stream (one
 * captured graph launch per step).  Returns HCA_ERR_NOCONV if any solve of
 * the last step hit maxit (its last iterate is kept and the step completed),
 * HCA_ERR_NONFINITE if a residual norm became NaN/Inf, HCA_ERR_TIMEOUT if a
 * bounded device wait gave up. */
int hca_step(hca_handle* h, int32_t n_steps);

/* Run selected stages of one step (HCA_STAGE_* mask) in their fixed order
 * O2, DRUGS, ODE, CA, ADVANCE.  The drug stage uses the plasma levels of the
 * current step index n (at t^{n+1}); the CA stage draws with step index n. */
int hca_stage(hca_handle* h, uint32_t stage_mask);

/* Copy fields of replicate rep to dst: the selected fields one after another
 * in increasing mask-bit order, each nx*ny*nz elements of the handle's
 * precision, x fastest (site x + nx*(y + ny*z)); dst is caller-owned host or
 * device memory (any pointer cudaMemcpy accepts) and the call synchronises
 * the handle's stream.  dst_bytes must be at least that size, and every
 * selected field must exist in the handle (else HCA_ERR_ARG).  These are the
 * fields Algorithm 1 carries from one step to the next (Eqs. oxygen, chemo,
 * cellcycle, odep53, odevegf). */
int hca_read_fields(hca_handle* h, int32_t rep, uint32_t field_mask, void* dst,
                    size_t dst_bytes, int32_t dst_on_device);

/* Overwrite fields of replicate rep from src (same packing as reading).
 * Used to restart from a saved state or to drive stages on given inputs. */
int hca_write_fields(hca_handle* h, int32_t rep, uint32_t field_mask, const void* src,
                     size_t src_bytes, int32_t src_on_device);

/* Copy / overwrite the uint8 lattice states (HCA_EMPTY .. HCA_STROMA) of
 * rep: the CA lattice of Section 2.2 that Algorithm 1 updates, nx*ny*nz
 * bytes, x fastest; host or device memory, synchronising the handle's
 * stream; a short buffer or a bad code is HCA_ERR_ARG. */
int hca_read_states(hca_handle* h, int32_t rep, uint8_t* dst, size_t dst_bytes,
                    int32_t dst_on_device);
int hca_write_states(hca_handle* h, int32_t rep, const uint8_t* src, size_t src_bytes,
                     int32_t src_on_device);

/* Set / get the step index n (drives plasma levels and the Philox counter). */
int hca_set_step(hca_handle* h, int64_t step);

/* Statistics of replicate rep after the last step or stage: CG iterations,
 * defect-correction sweeps and true relative residuals of the Section 2.4.1
 * solves, cell counts per state, kills and divisions of the CA update
 * (Section 2.5).  Synchronises the handle's stream. */
int hca_get_stats(hca_handle* h, int32_t rep, hca_stats* out);

/* out = A u for replicate rep, where A is the operator of the next solve
 * (which = 0: oxygen, linearised about the current K; which = 1 + d: drug d's
 * implicit-Euler operator).  u, out: nx*ny*nz elements of the handle's
 * precision.  Exposes the 7-point stencil of Eqs. (oxygen)/(chemo) alone. */
int hca_apply_operator(hca_handle* h, int32_t rep, int32_t which, const void* u, void* out,
                       int32_t on_device);

/* The launch shape the handle uses: threads per block of the sweep kernels
 * and the register cap of the FP32 CG passes.  With threads_per_block = 0
 * in the config the library picks both at creation by timing the oxygen CG
 * passes on the handle's own lattices (set HCA_NO_TUNE=1 to keep 128 / 96).
 * Results do not depend on the choice. */
int hca_get_launch_config(hca_handle* h, int32_t* threads_per_block, int32_t* pass_regs);

/* z = M r for replicate rep, with M the multigrid V-cycle (HCA_PC_MG) built
 * on the operator of the next solve of `which` (as hca_apply_operator).
 * r, z: nx*ny*nz elements of the handle's precision.  HCA_ERR_STATE unless
 * the handle was created with HCA_PC_MG.  Exposes the preconditioner alone. */
int hca_apply_preconditioner(hca_handle* h, int32_t rep, int32_t which, const void* r, void* z,
                             int32_t on_device);

/* 24-bit Philox4x32-10 uniforms u = (w0 >> 8) * 2^-24 for sites
 * site_begin .. site_begin + n - 1 with counter (site lo, site hi, step,
 * purpose) and key (seed lo, seed hi): the draws of Section 2.6's
 * per-cell streams.  dst: n floats (device or host). */
int hca_philox_uniforms(uint64_t seed, uint64_t site_begin, int64_t n, uint32_t step,
                        uint32_t purpose, float* dst, int32_t dst_on_device);

/* Block until all queued work of h is done. */
int hca_sync(hca_handle* h);

/* Number of replicates, lattice of replicate rep. */
int hca_get_shape(hca_handle* h, int32_t rep, int32_t* nx, int32_t* ny, int32_t* nz);

/* Number of this library's kernel launches since creation (for accounting). */
int64_t hca_launch_count(hca_handle* h);

/* Per-launch device timing: when enabled, every kernel launch of h is
 * bracketed by CUDA events on the handle's stream and its duration is added
 * to its class.  Enabling resets the counters.  hca_get_profile synchronises
 * the stream and returns the sums since the last enable. */
int hca_profile_enable(hca_handle* h, int32_t enable);
int hca_get_profile(hca_handle* h, hca_profile* out);

/* Allocation-free oxygen residual check (the paper has no counterpart: this
 * is a service for callers that may not allocate device memory, e.g. code
 * running inside another framework's memory pool or a real-time loop that
 * forbids cudaMalloc and its implicit synchronisation).
 *
 * Computes *rel_out = ||b - A K||_2 / ||b||_2 (0 when b = 0) for the
 * quasi-steady oxygen operator of one lattice linearised about K_prev, i.e.
 * the relative residual that hca_get_stats reports for an oxygen solve with
 * o2_scheme 0: A = -D_K Lap_h (7-point, Neumann) +
 * diag(phi_K/(K1 + K_prev)[consumer] + r_K[vessel]), b = r_K K0 [vessel].
 * Only cfg's nx, ny, nz, dx, D_K, phi_K, K1, K0, r_K and o2_scheme are used;
 * they are checked as hca_create checks them, and o2_scheme != 0 (whose
 * right-hand side depends on the previous field) is HCA_ERR_ARG.
 * state (uint8 codes), K_prev and K (double) are caller-owned DEVICE arrays
 * of nx*ny*nz elements in site order x + nx*(y + ny*z); they are only read.
 *
 * Nothing is allocated: the reduction scratch is a fixed device array inside
 * the library (about 33 KB per GPU, kept until the process exits), so the
 * lattice is limited to ny*nz <= 65536 rows (HCA_ERR_ARG beyond that).  Each
 * call looks up that array's device address in the context of the current
 * device (a host-side lookup that allocates nothing), then queues a memset of
 * its ticket, one kernel and a copy of the result to host memory on `stream`
 * (a cudaStream_t, NULL = the default stream), and synchronises `stream`
 * before it returns.  Every call shares the array: calls that overlap on the
 * GPU race and must be serialised by the caller.  Returns HCA_ERR_ARG for
 * bad arguments, HCA_ERR_CUDA for a failed CUDA call, HCA_ERR_NONFINITE for a
 * non-finite result. */
int hca_o2_residual_noalloc(const hca_config* cfg, const uint8_t* state, const double* K_prev,
                            const double* K, double* rel_out, void* stream);

/* Checkpoint and resume (no counterpart in the paper, which restarts from
 * patient data).  hca_save writes, to a new file at `path`, everything a
 * later step reads: the configurations (stream pointers stored as NULL), the
 * step counter, and per replicate the lattice states and the fields K, G_d,
 * V (when vegf = 1), phi, P, Vc and perf in the handle's precision, with the
 * low words of the FP32 defect-correction fields; it synchronises the
 * handle's stream first.  hca_load creates a handle from such a file on
 * `stream` (a cudaStream_t, NULL = default) without the initial oxygen
 * solve; stepping it continues the saved run bit for bit.  A learned
 * warm-start network is not part of the file (attach it again with
 * hca_set_warm_start_net).  Format: the 8 bytes "HCACKPT1", int32 version
 * (1), int32 sizeof(hca_config), int32 replicate count, int32 precision,
 * int64 step, int32 picard_iterations, int32 0, the configs, the perfusion
 * map of every replicate, then per replicate the states (nx*ny*nz bytes) and
 * the fields K [K_lo], G_d [G_lo_d], V [V_lo], phi, P, Vc (nx*ny*nz elements
 * each, site order x + nx*(y + ny*z); the low words only for HCA_FP32), all
 * little-endian as in memory.
 * Errors: HCA_ERR_ARG (null arguments, a file that is not a checkpoint of
 * this ABI), HCA_ERR_IO (open, read or write failed), and those of
 * hca_create_batch. */
int hca_save(hca_handle* h, const char* path);
int hca_load(const char* path, void* stream, hca_handle** out);

void hca_destroy(hca_handle* h);
const char* hca_status_string(int32_t status);

/* ------------------------------------------------ learned warm start ---
 * The paper has no counterpart: it starts every solve from the previous
 * step's field.  A small 3-D convolutional encoder-decoder predicts the
 * change of the oxygen field over one step from the lattice the solve sees;
 * the oxygen CG of Eq. (oxygen) then starts from K_prev + (K0 / HCA_NET_SCALE)
 * f(x) whenever that guess has a smaller residual than K_prev (checked on the
 * device every step, so a poor network never slows a solve beyond its own
 * cost).  The consumption term stays linearised about K_prev.
 *
 * Network (levels 0..3, channels 16, 32, 64, 64; every lattice extent a
 * multiple of 8): e0 = relu(conv(x)+b), e_l = relu(conv(pool(e_{l-1}))+b),
 * d2 = relu(conv(up(e3))+b+e2), d1 = relu(conv(up(d2))+b+e1),
 * d0 = relu(conv(up(d1))+b+e0), f = d0 . w_head + b_head; conv = 3x3x3 'same'
 * with zero padding, pool = 2x2x2 mean, up = 2x nearest.  BF16 weights and
 * activations, FP32 accumulation (tensor cores), FP32 master parameters.
 * Input channels of x (dense (D, H, W, 16) BF16, channels innermost): one-hot
 * state code 0..5, perf, K_prev / K0, HCA_NET_SCALE (b - A K_prev) /
 * (diag(A) K0), zeros.  Parameters: one FP32 array, per conv layer (order
 * enc0, enc1, enc2, enc3, dec2, dec1, dec0) the weights (27, C_out, C_in),
 * tap 9(dz+1)+3(dy+1)+(dx+1), then the biases; then 16 head weights and the
 * head bias.  Training minimises the loss below with Adam.  All arrays below are caller-owned DEVICE arrays unless
 * a flag says otherwise; lattices are dense (D, H, W) = (nz, ny, nx) with x
 * fastest.  Work runs on the stream given at creation; functions that read
 * results back synchronise it.  Errors: HCA_ERR_ARG (bad argument or
 * lattice), HCA_ERR_OOM, HCA_ERR_CUDA. */
#define HCA_NET_IN_CH 16
#define HCA_NET_SCALE 64.0

typedef struct hca_net hca_net;

/* Number of FP32 parameters. */
int hca_net_param_count(int64_t* n_out);

/* A network for D x H x W lattices (multiples of 8); trainable != 0 also
 * allocates the gradient, Adam and backward buffers.  Parameters start at 0. */
int hca_net_create(int32_t D, int32_t H, int32_t W, int32_t trainable, void* stream, hca_net** out);

/* Copy the FP32 parameters in (resets Adam's moments and step count) / out. */
int hca_net_set_params(hca_net* n, const float* params, int32_t on_device);
int hca_net_get_params(hca_net* n, float* params, int32_t on_device);

/* Features of (state uint8, perf float, K_prev float) under cfg's oxygen
 * parameters (D_K, dx, phi_K, K1, r_K, K0), then f into out (D*H*W floats).
 * x_out (optional, D*H*W*16 BF16) receives the features. */
int hca_net_forward(hca_net* n, const hca_config* cfg, const uint8_t* state, const float* perf, const float* K_prev,
                    float* out, void* x_out);

/* f of a given BF16 input x (D*H*W*16) into out. */
int hca_net_forward_x(hca_net* n, const void* x, float* out);

/* Copy a stored activation of the last forward pass (BF16, dense, channels
 * innermost) into dst: which = 0 x, 1 e0, 2 pool(e0), 3 e1, 4 pool(e1),
 * 5 e2, 6 pool(e2), 7 e3, 8 d2, 9 d1, 10 d0 (d0: trainable networks only).
 * For inspection and per-layer checks. */
int hca_net_read_activation(hca_net* n, int32_t which, void* dst);

/* Copy the gradient of the last backward pass with respect to one
 * convolution's output (after its ReLU mask; for enc0..enc2 after the skip
 * path's gradient is added) into dst (BF16, dense, channels innermost, the
 * convolution's output lattice): which = 0 enc0, 1 enc1, 2 enc2, 3 enc3,
 * 4 dec2, 5 dec1, 6 dec0.  Trainable networks only (else HCA_ERR_ARG).  For
 * per-layer checks. */
int hca_net_read_gradient(hca_net* n, int32_t which, void* dst);

/* Forward and backward on input x and target t (D*H*W floats): gradients of
 * mean((f - t)^2) into grads (param_count floats, optional) and the loss
 * into *loss (optional); both device pointers.  Needs trainable. */
int hca_net_gradients_x(hca_net* n, const void* x, const float* target, float* grads, float* loss);

/* One Adam step (Kingma & Ba 2015) on the gradients of the last backward pass. */
int hca_net_adam(hca_net* n, double lr, double beta1, double beta2, double eps);

/* Training loss L = w_mse mean((f - t)^2) + w_res mean((A e)^2) / c^2 with
 * t = HCA_NET_SCALE (K_new - K_prev) / K0, e = f - t, A the oxygen operator
 * linearised about K_prev and c = D_K / dx^2 (the second term is the
 * residual of the guess up to scale).  Weights >= 0, not both 0. */

/* Features, forward and backward for one oxygen solve (state uint8, perf,
 * K_prev, K_new float): gradients into grads (param_count floats, optional)
 * and the loss into *loss (optional), device pointers.  Asynchronous. */
int hca_net_gradients(hca_net* n, const hca_config* cfg, const uint8_t* state, const float* perf,
                      const float* K_prev, const float* K_new, double w_mse, double w_res, float* grads,
                      float* loss);

/* hca_net_gradients followed by one Adam step (beta = (0.9, 0.999),
 * eps = 1e-8); *loss (device, optional) receives the loss before the
 * update.  Asynchronous. */
int hca_net_train_step(hca_net* n, const hca_config* cfg, const uint8_t* state, const float* perf,
                       const float* K_prev, const float* K_new, double w_mse, double w_res, double lr,
                       float* loss);

/* A training run of the warm-start network in one call (no counterpart in
 * the paper; the network of this section is trained on fields the solver
 * itself generates).  The dataset is n_samples oxygen solves, each given by
 * caller-owned DEVICE arrays of the network's nz*ny*nx lattice: the lattice
 * states the solve saw (uint8), the perfusion map, K before and K after the
 * solve (float).  Step t = 0 .. iters-1 draws sample
 * floor(u_t * n_samples), u_t the 24-bit Philox uniform keyed by
 * (seed; counter t, 0, 0, 5) (the generator of Section 2.6's streams), and
 * runs hca_net_train_step on it with learning rate
 * lr * (lr_final / lr)^(t / (iters - 1)) (geometric decay; lr_final = lr
 * keeps it constant) and loss w_mse * MSE + w_res * residual loss.  losses
 * (device, iters floats, optional) receives every step's loss before its
 * update.  Asynchronous on the network's stream (hca_net_sync waits).
 * HCA_ERR_ARG for a bad field, an untrainable network or null pointers. */
typedef struct {
  uint32_t struct_size;              /* sizeof(hca_train_cfg) */
  int32_t n_samples;
  const uint8_t* const* state;       /* host array of n_samples device pointers */
  const float* const* perf;
  const float* const* K_prev;
  const float* const* K_new;
  int32_t iters;
  double lr, lr_final;
  uint64_t seed;
  double w_mse, w_res;
  float* losses;
} hca_train_cfg;
int hca_train_warmstart(hca_net* n, const hca_config* cfg, const hca_train_cfg* tc);

int hca_net_sync(hca_net* n);
int hca_net_destroy(hca_net* n);

/* Attach a network (not owned; must outlive its use) to a single-replicate
 * handle created with warm_start = HCA_WS_LEARNED(_ALWAYS) and an nz x ny x nx
 * lattice equal to the network's.  NULL detaches (the solve then starts
 * from K_prev).  Rebuilds the captured step graph on the next step. */
int hca_set_warm_start_net(hca_handle* h, hca_net* n);

#ifdef __cplusplus
}
#endif
#endif /* HCA_H */
