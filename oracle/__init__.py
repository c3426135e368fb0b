"""FP64 CPU oracle for the hybrid cellular automaton (HCA) time step.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import this package.  The library path
(``paper_2105_00448_gb300``) never calls it and has no CPU fallback.

The oracle is a plain, slow, readable restatement of the model of
Lai, Taskén et al., "A scalable solver for a stochastic, hybrid cellular
automaton model of personalized breast cancer therapy" (arXiv:2105.00448),
discretised the way the GPU path is specified: a 7-point finite-difference
stencil on the 3-D CA lattice, Jacobi-preconditioned CG, implicit Euler for the
drugs, closed-form/RK4 cell ODEs and a 27-colour sweep of the cellular
automaton.  It shares no code with the CUDA path; both take the same seeded
inputs from ``synth``.

Modules
-------
params   Table 1 parameters and the readings used where the paper is silent.
philox   Philox4x32-10 counter-based generator (Salmon et al., SC'11).
stencil  The discrete operators of Eq. (oxygen) and Eq. (chemo).
pcg      Textbook Jacobi-preconditioned conjugate gradients.
plasma   Plasma concentration after bolus doses (Eq. intrachemo3, closed form).
odes     Cell-cycle clock, p53 and intracellular VEGF (Eqs. cellcycle, odep53, odevegf).
ca       The stochastic cellular automaton update (Sections 2.2.1 and 2.5).
model    Algorithm 1: initialisation and the time loop.
convnet  FP64 reference of the learned warm-start network (no paper counterpart).
ca_sync  The synchronous CA update with Algorithm 2's higher-phi rule.
vascular The VEGF field's automaton: vessel birth and death (Eq. vascular_module).
pk       Michaelis-Menten and three-compartment plasma models (Section 2.2.3).
multigrid The geometric V-cycle preconditioner and MG-PCG.
api      The library's call names (oracle_create, oracle_step, ...) over model.

Parity status: every function is pinned by tests under ``tests/test_oracle_*``
except the ones whose docstring says "parity unpinned"; the output bits of
``philox.philox4x32_10`` are pinned against cuRAND's Philox4_32_10 device
generator, an independent implementation, in ``tests/test_gpu_philox_curand.py``
(it needs a GPU).
"""
