// Host side of the library: handle set-up, device memory, the step schedule
// (Algorithm 1 loop body: oxygen, drugs, ODEs, CA) and the C ABI of hca.h.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdio>
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <new>
#include <vector>

#include "hca_internal.cuh"

namespace hca {
void launch_setup(const Ctx& c, int which, bool fp64, CondArg cnd);
void launch_pass_a(const Ctx& c, int which, bool fp64);
void launch_pass_b(const Ctx& c, int which, void* xfield, bool fp64, CondArg cnd);
void launch_true_residual(const Ctx& c, int which, void* xfield, bool fp64);
void launch_apply(const Ctx& c, int which, int rep, const void* u, void* out, bool fp64);
void launch_diff_norms(const Ctx& c, const void* a, const void* b, bool fp64);
void launch_dc_residual(const Ctx& c, int which, const void* x_hi, const void* x_lo, bool first, CondArg outer,
                        CondArg inner);
void launch_dc_update(const Ctx& c, void* x_hi, void* x_lo);
void launch_init(const Ctx& c, const float* pc, const float* pf, const float* pv, int* err, bool fp64);
void launch_ode(const Ctx& c, bool fp64);
void launch_histogram(const Ctx& c);
void launch_philox_uniforms(unsigned long long seed, unsigned long long site0, long long n, uint32_t step,
                            uint32_t purpose, float* out, cudaStream_t stream);
void launch_advance_step(const Ctx& c, long long by);
void launch_ca_compact(const Ctx& c, bool fp64);
void launch_ca_colour(const Ctx& c, int colour, int blocks_x, bool fp64);
int ca_coop_blocks(bool fp64, int sm_count);
void launch_ca_colours(const Ctx& c, int blocks, bool fp64);
void launch_ca_sync(const Ctx& c, int blocks_x, bool fp64);
void launch_vessels(const Ctx& c, bool fp64);
void launch_mg_setup(const Ctx& c, int which, bool fp64, const MGHost& H, bool w_done);
void launch_vcycle(const Ctx& c, int which, bool fp64, const MGHost& H, int part, bool scale);
int vcycle_launches(const MGHost& H, bool scale);
int vcycle_part_launches(const MGHost& H, int part, bool scale);
void mg_coop_config(MGHost& H, bool fp64, int sm_count, long long smem_bytes);
void mg_zmarch_config(MGHost& H, const RepDesc& rd, int sm_count, const float* r, const float* w,
                      const int* lv_dims);
}  // namespace hca

using hca::Ctx;
using hca::RepDesc;

#include "net_internal.cuh"

// Optional per-launch device timing (hca_profile_enable).
struct Profiler {
  bool on = false;
  std::vector<cudaEvent_t> pool;   // 2 * kPairs events, created on first enable
  struct Rec {
    int cls;
    cudaEvent_t a, b;
  };
  std::vector<Rec> pending;
  size_t next = 0;
  long long launches[HCA_NKCLASS] = {};
  double ms[HCA_NKCLASS] = {};
};

struct hca_handle {
  Profiler prof;
  int n_reps = 0;
  bool fp64 = true;
  int n_drugs = 0;
  cudaStream_t stream = nullptr;
  int device = 0;
  std::vector<hca_config> cfgs;
  std::vector<RepDesc> reps_h;
  // the descriptors with the quasi-steady oxygen form, for the initial oxygen
  // fixed point of a handle whose oxygen equation is time-dependent
  std::vector<RepDesc> reps_qs_h;
  RepDesc* reps_qs = nullptr;
  std::vector<int2> chunks_h;
  Ctx ctx{};
  long long total = 0;        // elements per field array
  long long lists_total = 0;
  long long step = 0;
  long long launches = 0;
  int picard_iterations = 0;
  bool nonlinear = false;
  bool ca_sync = false;       // ca_mode 1: synchronous CA update, higher phi wins
  bool vegf = false;          // the VEGF field (slot 3) is solved every step
  bool vessels = false;       // some replicate runs the vascular automaton     // o2_nonlinear: a Picard solve of the oxygen equation every step
  int prev_iters[1 + hca::MAX_FIELDS] = {0, 0, 0, 0, 0};
  int maxit_all = 0;
  int max_outer = 0;
  int last_iters = 0;
  int prev_inner[1 + hca::MAX_FIELDS][16] = {};
  // step graphs (one per stage mask), built on first use
  struct Graph {
    uint32_t mask;
    cudaGraphExec_t exec;
  };
  std::vector<Graph> graphs;
  cudaStream_t cap[3] = {nullptr, nullptr, nullptr};
  bool graphs_ok = true;
  bool capturing = false;     // a step graph is being captured
  int ca_coop = 0;            // blocks of the cooperative 27-colour CA kernel (0: one launch per colour)
  int* h_pinned = nullptr;    // [0] active replicates, [1] error flag
  std::vector<void*> allocs;
  // multigrid preconditioner (single replicate)
  bool mg = false;
  hca::MGHost mgh;
  // learned warm start of the oxygen solve (single replicate)
  bool learned = false;
  hca_net* net = nullptr;
  double* ws_cand = nullptr;
  double* ws_part = nullptr;
  hcanet::WsResult* ws_res = nullptr;
};

namespace {

constexpr int kFieldAlign = 64;  // elements; keeps every replicate 256-byte aligned

#define HCA_TRY(expr)                              \
  do {                                             \
    cudaError_t e_ = (expr);                       \
    if (e_ != cudaSuccess) {                       \
      (void)cudaGetLastError();                    \
      return e_ == cudaErrorMemoryAllocation ? HCA_ERR_OOM : HCA_ERR_CUDA; \
    }                                              \
  } while (0)


// Host status of a nonzero PassSync::error code.
int sync_error_status(int e) {
  return e == hca::SYNC_ERR_TIMEOUT ? HCA_ERR_TIMEOUT : e == hca::SYNC_ERR_NOCONV ? HCA_ERR_NOCONV : HCA_ERR_NONFINITE;
}

constexpr size_t kPairs = 4096;

int prof_flush(hca_handle* h) {
  Profiler& P = h->prof;
  if (P.pending.empty()) return HCA_OK;
  HCA_TRY(cudaStreamSynchronize(h->ctx.stream));
  for (auto& r : P.pending) {
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, r.a, r.b) == cudaSuccess) P.ms[r.cls] += ms;
    else (void)cudaGetLastError();
  }
  P.pending.clear();
  P.next = 0;
  return HCA_OK;
}

cudaEvent_t prof_begin(hca_handle* h) {
  Profiler& P = h->prof;
  if (!P.on) return nullptr;
  if (P.next + 2 > P.pool.size()) prof_flush(h);
  cudaEvent_t a = P.pool[P.next++];
  cudaEventRecord(a, h->ctx.stream);
  return a;
}

void prof_end(hca_handle* h, int cls, cudaEvent_t a, int n_kernels) {
  Profiler& P = h->prof;
  if (!P.on || !a) return;
  cudaEvent_t b = P.pool[P.next++];
  cudaEventRecord(b, h->ctx.stream);
  P.pending.push_back({cls, a, b});
  P.launches[cls] += n_kernels;
}

// Launch `call` (n_kernels kernels of class cls), count it, check the launch
// and, when profiling, bracket it with events.
#define HCA_LAUNCH(h, cls, n_kernels, call)  \
  do {                                       \
    cudaEvent_t a_ = prof_begin(h);          \
    call;                                    \
    (h)->launches += (n_kernels);            \
    cudaError_t e_ = cudaGetLastError();     \
    if (e_ != cudaSuccess) return HCA_ERR_CUDA; \
    prof_end(h, cls, a_, n_kernels);         \
  } while (0)

int colour_count(int n, int r) { return r < n ? (n - r + 2) / 3 : 0; }

int next_pow2(int v) {
  int p = 1;
  while (p < v) p <<= 1;
  return p;
}

size_t elem_size(const hca_handle* h) { return h->fp64 ? sizeof(double) : sizeof(float); }

int validate(const hca_config& c) {
  if (c.struct_size != sizeof(hca_config)) return HCA_ERR_ARG;
  if (c.nx < 1 || c.ny < 1 || c.nz < 1) return HCA_ERR_ARG;
  const long long n = (long long)c.nx * c.ny * c.nz;
  if (n > 2147483647LL) return HCA_ERR_ARG;
  if (c.precision != HCA_FP64 && c.precision != HCA_FP32) return HCA_ERR_ARG;
  if (c.n_drugs < 0 || c.n_drugs > 3) return HCA_ERR_ARG;
  if (!(c.dx > 0) || !(c.dt > 0) || !(c.rtol_o2 > 0) || !(c.rtol_drug > 0)) return HCA_ERR_ARG;
  if (c.maxit < 0 || c.ode_substeps < 1 || c.picard_maxit < 0 || !(c.picard_tol >= 0)) return HCA_ERR_ARG;
  if (c.o2_nonlinear != 0 && c.o2_nonlinear != 1) return HCA_ERR_ARG;
  if (c.o2_nonlinear && c.picard_maxit < 1) return HCA_ERR_ARG;
  if (c.o2_nonlinear && c.warm_start != HCA_WS_PREV) return HCA_ERR_UNIMPLEMENTED;
  if (c.drug_scheme != 0 && c.drug_scheme != 1) return HCA_ERR_ARG;
  if (c.ca_mode != 0 && c.ca_mode != 1) return HCA_ERR_ARG;
  if (c.vegf != 0 && c.vegf != 1) return HCA_ERR_ARG;
  if (c.vessel_interval < 0 || (c.vessel_interval > 0 && !c.vegf)) return HCA_ERR_ARG;
  if (!(c.D_V >= 0) || !(c.psi_V >= 0) || !(c.a_V >= 0)) return HCA_ERR_ARG;
  if (c.vessel_interval > 0 && (!(c.V_low >= 0) || !(c.V_high > c.V_low) || !(c.p_death >= 0 && c.p_death <= 1) ||
                                !(c.beta_birth >= 0) || !(c.V_sprout > 0)))
    return HCA_ERR_ARG;
  for (int d = 0; d < 3; ++d) {
    if (c.pk_model[d] < 0 || c.pk_model[d] > 2) return HCA_ERR_ARG;
    if (d < c.n_drugs && c.pk_model[d] == 1 && (!(c.mm_vmax > 0) || !(c.mm_km > 0))) return HCA_ERR_ARG;
    if (d < c.n_drugs && c.pk_model[d] == 2 &&
        (!(c.epi_w[0] > 0) || !(c.epi_w[1] > 0) || !(c.epi_w[2] > 0) || !(c.epi_q2 > 0) || !(c.epi_q3 > 0) ||
         !(c.epi_cl2 > 0)))
      return HCA_ERR_ARG;
  }
  if (c.o2_scheme < 0 || c.o2_scheme > 2) return HCA_ERR_ARG;
  if (c.drug_substeps < 1 || c.drug_substeps > 100000 || c.o2_substeps < 1 || c.o2_substeps > 100000)
    return HCA_ERR_ARG;
  if (c.o2_scheme && (c.o2_nonlinear || c.warm_start != HCA_WS_PREV)) return HCA_ERR_UNIMPLEMENTED;
  if (c.dose_interval < 1) return HCA_ERR_ARG;
  for (int d = 0; d < c.n_drugs; ++d) {
    if (c.kill_b[d] < 1 || c.kill_b[d] > 64 || !(c.dose_peak[d] > 0)) return HCA_ERR_ARG;
    if (!(c.D_G[d] >= 0) || !(c.psi_G[d] >= 0) || !(c.kappa_G[d] >= 0) || !(c.uptake_G[d] >= 0)) return HCA_ERR_ARG;
  }
  if (!(c.D_K > 0) || !(c.phi_K >= 0) || !(c.K1 > 0) || !(c.r_K >= 0) || !(c.K0 >= 0)) return HCA_ERR_ARG;
  const int t = c.threads_per_block;
  if (!(t == 0 || t == 64 || t == 128 || t == 256 || t == 512)) return HCA_ERR_ARG;
  if (c.warm_start != HCA_WS_PREV && c.warm_start != HCA_WS_LEARNED && c.warm_start != HCA_WS_LEARNED_ALWAYS)
    return HCA_ERR_ARG;
  if (c.preconditioner != HCA_PC_JACOBI && c.preconditioner != HCA_PC_MG) return HCA_ERR_ARG;
  return HCA_OK;
}

// Plasma response of the three-compartment model to a unit bolus,
// [exp(M t)]_00 = sum_i coef_i exp(lam_i t), with M the rate matrix of the
// compartment amounts.  D M D^-1 with D = diag(w)^(-1/2) is symmetric and has
// the same (0,0) entry of its exponential, so lam_i are its eigenvalues and
// coef_i the squared first components of its unit eigenvectors (cyclic
// Jacobi rotations, FP64).
void three_compartment_response(const hca_config& c, double lam[3], double coef[3]) {
  const double w1 = c.epi_w[0], w2 = c.epi_w[1], w3 = c.epi_w[2];
  double S[3][3] = {{-(c.epi_cl2 + c.epi_q2 + c.epi_q3) / w1, c.epi_q2 / std::sqrt(w1 * w2), c.epi_q3 / std::sqrt(w1 * w3)},
                    {c.epi_q2 / std::sqrt(w1 * w2), -c.epi_q2 / w2, 0.0},
                    {c.epi_q3 / std::sqrt(w1 * w3), 0.0, -c.epi_q3 / w3}};
  double V[3][3] = {{1, 0, 0}, {0, 1, 0}, {0, 0, 1}};
  for (int sweep = 0; sweep < 64; ++sweep) {
    const double off = std::fabs(S[0][1]) + std::fabs(S[0][2]) + std::fabs(S[1][2]);
    if (off == 0.0) break;
    for (int p = 0; p < 2; ++p)
      for (int q = p + 1; q < 3; ++q) {
        if (S[p][q] == 0.0) continue;
        const double theta = (S[q][q] - S[p][p]) / (2.0 * S[p][q]);
        const double t = (theta >= 0 ? 1.0 : -1.0) / (std::fabs(theta) + std::sqrt(theta * theta + 1.0));
        const double cs = 1.0 / std::sqrt(t * t + 1.0), sn = t * cs;
        for (int k = 0; k < 3; ++k) {   // S <- S J (columns p, q)
          const double a = S[k][p], b = S[k][q];
          S[k][p] = cs * a - sn * b;
          S[k][q] = sn * a + cs * b;
        }
        for (int k = 0; k < 3; ++k) {   // S <- J^T S (rows p, q)
          const double a = S[p][k], b = S[q][k];
          S[p][k] = cs * a - sn * b;
          S[q][k] = sn * a + cs * b;
        }
        for (int k = 0; k < 3; ++k) {   // V <- V J
          const double a = V[k][p], b = V[k][q];
          V[k][p] = cs * a - sn * b;
          V[k][q] = sn * a + cs * b;
        }
      }
  }
  for (int i = 0; i < 3; ++i) {
    lam[i] = S[i][i];
    coef[i] = V[0][i] * V[0][i];
  }
}

RepDesc make_desc(const hca_config& c) {
  RepDesc r;
  std::memset(&r, 0, sizeof(r));
  r.nx = c.nx;
  r.ny = c.ny;
  r.nz = c.nz;
  r.nxp = (c.nx + 3) / 4 * 4;
  r.gpr = r.nxp / 4;
  r.lpr = std::min(32, next_pow2(r.gpr));
  r.seed = c.seed;
  r.n_drugs = c.n_drugs;
  r.maxit = c.maxit;
  r.rtol_o2 = c.rtol_o2;
  r.rtol_drug = c.rtol_drug;
  r.rtol_inner = c.rtol_inner;
  r.max_outer = c.precision == HCA_FP32 ? c.max_outer : 0;
  const double dx2 = c.dx * c.dx;
  r.c_o2 = c.D_K / dx2;
  r.phi_K = c.phi_K;
  r.K1 = c.K1;
  r.K0 = c.K0;
  r.r_K = c.r_K;
  r.inv_dt = 1.0 / c.dt;
  // time discretisation: sub-step h, mass term 1/h (implicit Euler) or 2/h
  // (Crank-Nicolson), b = bx x0 [- A x0] + source
  const double ho = c.dt / c.o2_substeps, hd = c.dt / c.drug_substeps;
  r.o2_mass = c.o2_scheme == 1 ? 1.0 / ho : c.o2_scheme == 2 ? 2.0 / ho : 0.0;
  r.bx[0] = c.o2_scheme == 1 ? 1.0 / ho : c.o2_scheme == 2 ? 4.0 / ho : 0.0;
  r.bax[0] = c.o2_scheme == 2;
  r.nsub[0] = c.o2_scheme ? c.o2_substeps : 1;
  for (int d = 0; d < hca::MAX_DRUGS; ++d) {
    r.bx[1 + d] = c.drug_scheme ? 4.0 / hd : 1.0 / hd;
    r.bax[1 + d] = c.drug_scheme == 1;
    r.nsub[1 + d] = c.drug_substeps;
  }
  for (int d = 0; d < hca::MAX_DRUGS; ++d) {
    r.c_drug[d] = c.D_G[d] / dx2;
    r.base_drug[d] = (c.drug_scheme ? 2.0 / hd : 1.0 / hd) + c.psi_G[d];
    r.kappa[d] = c.kappa_G[d];
    r.uptake[d] = c.uptake_G[d];
    r.dose_peak[d] = c.dose_peak[d] > 0 ? c.dose_peak[d] : 1.0;
    r.plasma_decay[d] = c.plasma_decay[d];
    r.kill_b[d] = c.kill_b[d];
  }
  // the VEGF field (Eq. vac_v, A = 0) in slot 3: stepped like the drugs, no
  // vessel exchange, released by the cells
  r.bx[hca::WHICH_VEGF] = c.drug_scheme ? 4.0 / hd : 1.0 / hd;
  r.bax[hca::WHICH_VEGF] = c.drug_scheme == 1;
  r.nsub[hca::WHICH_VEGF] = c.drug_substeps;
  r.c_drug[hca::VEGF_SLOT] = c.D_V / dx2;
  for (int w = 0; w <= hca::MAX_FIELDS; ++w) r.cpl32[w] = (float)(w == 0 ? r.c_o2 : r.c_drug[w - 1]);
  r.base_drug[hca::VEGF_SLOT] = (c.drug_scheme ? 2.0 / hd : 1.0 / hd) + c.psi_V;
  r.kappa[hca::VEGF_SLOT] = 0.0;
  r.uptake[hca::VEGF_SLOT] = 0.0;
  r.a_vegf = c.a_V;
  for (int d = 0; d < hca::MAX_DRUGS; ++d) {
    r.pk_model[d] = c.pk_model[d];
    if (c.pk_model[d] == 2) three_compartment_response(c, r.pk_lam[d], r.pk_coef[d]);
  }
  r.mm_vmax = c.mm_vmax;
  r.mm_km = c.mm_km;
  r.vessel_interval = c.vessel_interval;
  r.V_low = c.V_low;
  r.V_high = c.V_high;
  r.p_death = c.p_death;
  r.beta_birth = c.beta_birth;
  r.V_sprout = c.V_sprout;
  r.dose_interval_min = c.dose_interval * c.dt;
  r.dt = c.dt;
  r.T_cycle = c.T_cycle;
  r.K_phi = c.K_phi;
  r.k1 = c.k1;
  r.k1p = c.k1p;
  r.K_p53 = c.K_p53;
  r.k2 = c.k2;
  r.k2p = c.k2p;
  r.k2pp = c.k2pp;
  r.J5 = c.J5;
  r.K_V = c.K_V;
  r.ode_substeps = c.ode_substeps;
  return r;
}

template <typename P>
int dev_alloc(hca_handle* h, P** out, size_t bytes) {
  void* p = nullptr;
  cudaError_t e = cudaMalloc(&p, bytes ? bytes : 16);
  if (e != cudaSuccess) {
    (void)cudaGetLastError();
    return HCA_ERR_OOM;
  }
  h->allocs.push_back(p);
  *out = (P*)p;
  return HCA_OK;
}

void free_all(hca_handle* h) {
  if (!h) return;
  for (auto& g : h->graphs) cudaGraphExecDestroy(g.exec);
  h->graphs.clear();
  for (auto& s : h->cap)
    if (s) {
      cudaStreamDestroy(s);
      s = nullptr;
    }
  for (auto e : h->prof.pool) cudaEventDestroy(e);
  h->prof.pool.clear();
  for (void* p : h->allocs) cudaFree(p);
  h->allocs.clear();
  if (h->h_pinned) cudaFreeHost(h->h_pinned);
  h->h_pinned = nullptr;
}

void* field_ptr(hca_handle* h, uint32_t bit) {
  switch (bit) {
    case HCA_FIELD_O2: return h->ctx.K;
    case HCA_FIELD_DRUG0: return h->n_drugs > 0 ? h->ctx.G[0] : nullptr;
    case HCA_FIELD_DRUG1: return h->n_drugs > 1 ? h->ctx.G[1] : nullptr;
    case HCA_FIELD_DRUG2: return h->n_drugs > 2 ? h->ctx.G[2] : nullptr;
    case HCA_FIELD_PHI: return h->ctx.phi;
    case HCA_FIELD_P53: return h->ctx.P;
    case HCA_FIELD_VEGFC: return h->ctx.Vc;
    case HCA_FIELD_PERF: return h->ctx.perf;
    case HCA_FIELD_VEGF: return h->vegf ? h->ctx.G[hca::VEGF_SLOT] : nullptr;
    // low-order words of the FP32 defect-correction fields (read only)
    case HCA_FIELD_O2_LO: return h->ctx.K_lo;
    case HCA_FIELD_DRUG0_LO: return h->n_drugs > 0 ? h->ctx.G_lo[0] : nullptr;
    case HCA_FIELD_DRUG1_LO: return h->n_drugs > 1 ? h->ctx.G_lo[1] : nullptr;
    case HCA_FIELD_DRUG2_LO: return h->n_drugs > 2 ? h->ctx.G_lo[2] : nullptr;
    case HCA_FIELD_VEGF_LO: return h->vegf ? h->ctx.G_lo[hca::VEGF_SLOT] : nullptr;
    default: return nullptr;
  }
}

constexpr hca::CondArg kNoCond{0ull, 0};

void pass_a(hca_handle* h, int which) { hca::launch_pass_a(h->ctx, which, h->fp64); }

void pass_b(hca_handle* h, int which, void* x, hca::CondArg cnd) {
  hca::launch_pass_b(h->ctx, which, x, h->fp64, cnd);
}

// z = M r (V-cycle); also sets rho and beta for the next pass A.  first: the
// residual was just formed (start of a solve or a defect-correction sweep),
// so it may still need its power-of-two scaling.
// Inside a captured step graph the coarse levels run as one launch per
// kernel (graph-launched kernels follow each other closely, and the
// per-level kernels keep more warps per SM than the cooperative kernel:
// measured faster, also against the cooperative launch of only the levels
// below 2^18 sites); from host loops, where each launch costs host time, as
// the one cooperative launch.  HCA_MG_COOP_GRAPH=1 captures the cooperative
// launch from level 1, =2 from the first level below 2^18 sites.
void vcycle(hca_handle* h, int which, bool first) {
  if (h->capturing && h->mgh.coop_blocks > 0) {
    const char* e = std::getenv("HCA_MG_COOP_GRAPH");   // 0 none, 1 all coarse levels, else from coop_lo
    const int coop_graph = e ? e[0] - '0' : 0;
    hca::MGHost H = h->mgh;
    if (coop_graph == 0) H.coop_blocks = 0;
    else H.coop_from = coop_graph == 1 ? 1 : H.coop_lo;
    hca::launch_vcycle(h->ctx, which, h->fp64, H, -1, first);
    return;
  }
  hca::launch_vcycle(h->ctx, which, h->fp64, h->mgh, -1, first);
}

// The V-cycle from the host loop: with the profiler on, its lattice-level
// kernels are timed as classes of their own.
int vcycle_host(hca_handle* h, int which, bool first) {
  if (!h->prof.on) {
    HCA_LAUNCH(h, HCA_KCLASS_MG, hca::vcycle_launches(h->mgh, first), vcycle(h, which, first));
    return HCA_OK;
  }
  const hca::MGHost& H = h->mgh;
  const int cls[hca::kVcycleParts] = {HCA_KCLASS_MG,      HCA_KCLASS_MG_PRE0,  HCA_KCLASS_MG_RESTRICT0,
                                       HCA_KCLASS_MG,      HCA_KCLASS_MG_POST0, HCA_KCLASS_MG_LAST0};
  for (int part = 0; part < hca::kVcycleParts; ++part) {
    const int n = hca::vcycle_part_launches(H, part, first);
    if (n) HCA_LAUNCH(h, cls[part], n, hca::launch_vcycle(h->ctx, which, h->fp64, H, part, first));
  }
  return HCA_OK;
}

// coarse diagonals of the current operator (after its set-up stored d)
void mg_setup(hca_handle* h, int which, bool w_done = false) {
  hca::launch_mg_setup(h->ctx, which, h->fp64, h->mgh, w_done);
}

// CG iterations (V-cycle, pass A, pass B) on operator `which` for every
// replicate whose solve is active, updating x, until none is active or maxit
// is reached.  The first convergence check comes after about as many
// iterations as the same solve needed last time (`predict`), later ones every
// 4 iterations; with the profiler on, before every iteration (so no launch
// runs empty).  scale_first: the first V-cycle may scale r (it follows a
// defect-correction residual sweep).
int pcg_iterate(hca_handle* h, int which, void* x, int predict, bool scale_first) {
  Ctx& c = h->ctx;
  int done = 0;
  int chunk = h->prof.on ? 1 : std::max(1, predict - 2);
  for (;;) {
    HCA_TRY(cudaMemcpyAsync(h->h_pinned, &c.sync->active_count, 2 * sizeof(int), cudaMemcpyDeviceToHost, c.stream));
    HCA_TRY(cudaStreamSynchronize(c.stream));
    if (h->h_pinned[1]) return sync_error_status(h->h_pinned[1]);
    if (h->h_pinned[0] == 0 || done >= h->maxit_all) break;
    const int n = std::min(chunk, h->maxit_all - done);
    for (int k = 0; k < n; ++k) {
      if (h->mg) {
        const int rc = vcycle_host(h, which, scale_first && done + k == 0);
        if (rc) return rc;
      }
      HCA_LAUNCH(h, HCA_KCLASS_PASS_A, 1, pass_a(h, which));
      HCA_LAUNCH(h, HCA_KCLASS_PASS_B, 1, pass_b(h, which, x, kNoCond));
    }
    done += n;
    chunk = h->prof.on ? 1 : 4;
  }
  h->last_iters = done;
  return HCA_OK;
}

// One Jacobi-PCG solve of operator `which` (0 oxygen, 1 + d drug d) for all
// replicates, x0 = current field, in place (storage precision arithmetic,
// FP64 reductions).
int solve_plain(hca_handle* h, int which) {
  Ctx& c = h->ctx;
  void* x = which == 0 ? c.K : c.G[which - 1];
  HCA_LAUNCH(h, HCA_KCLASS_SETUP, 1, hca::launch_setup(c, which, h->fp64, kNoCond));
  if (h->mg) HCA_LAUNCH(h, HCA_KCLASS_MG, h->mgh.nlev, mg_setup(h, which));
  int rc = pcg_iterate(h, which, x, h->prev_inner[which][0], false);
  if (rc) return rc;
  h->prev_inner[which][0] = h->last_iters;
  HCA_LAUNCH(h, HCA_KCLASS_RESIDUAL, 2, hca::launch_true_residual(c, which, x, h->fp64));
  HCA_TRY(cudaMemcpyAsync(h->h_pinned, &c.sync->active_count, 2 * sizeof(int), cudaMemcpyDeviceToHost, c.stream));
  HCA_TRY(cudaStreamSynchronize(c.stream));
  return h->h_pinned[1] ? sync_error_status(h->h_pinned[1]) : HCA_OK;
}

// FP32 storage with defect correction: float-float (~48-bit) residual of the
// two-word solution, FP32 inner CG on the correction, two-word update;
// repeated until the relative residual (FP64 norms) meets the tolerance or
// max_outer sweeps.
int solve_dc(hca_handle* h, int which) {
  Ctx& c = h->ctx;
  void* xh = which == 0 ? c.K : c.G[which - 1];
  void* xl = which == 0 ? c.K_lo : c.G_lo[which - 1];
  for (int outer = 0;; ++outer) {
    HCA_LAUNCH(h, HCA_KCLASS_RESIDUAL, 1,
               hca::launch_dc_residual(c, which, xh, xl, outer == 0, kNoCond, kNoCond));
    if (h->mg && outer == 0) HCA_LAUNCH(h, HCA_KCLASS_MG, h->mgh.nlev - 1, mg_setup(h, which, true));
    HCA_TRY(cudaMemcpyAsync(h->h_pinned, &c.sync->active_count, 2 * sizeof(int), cudaMemcpyDeviceToHost, c.stream));
    HCA_TRY(cudaStreamSynchronize(c.stream));
    if (h->h_pinned[1]) return sync_error_status(h->h_pinned[1]);
    if (h->h_pinned[0] == 0) {
      // converged everywhere (or max_outer); zero fields whose right-hand side vanished
      HCA_LAUNCH(h, HCA_KCLASS_OTHER, 1, hca::launch_dc_update(c, xh, xl));
      break;
    }
    const int slot = std::min(outer, 15);
    int rc = pcg_iterate(h, which, c.dx, h->prev_inner[which][slot], true);
    if (rc) return rc;
    h->prev_inner[which][slot] = h->last_iters;
    HCA_LAUNCH(h, HCA_KCLASS_OTHER, 1, hca::launch_dc_update(c, xh, xl));
  }
  return HCA_OK;
}

int solve(hca_handle* h, int which) {
  if (!h->fp64 && h->max_outer > 0) return solve_dc(h, which);
  return solve_plain(h, which);
}

// ------------------------------------------------------------ step graph --
// The whole step (or a subset of its stages) captured once into a CUDA graph.
// Each CG loop is a WHILE conditional node whose body is [V-cycle, pass A,
// pass B] ([pass A, pass B] with the Jacobi preconditioner, whose z comes
// from pass B); the last block of the set-up / pass B / defect-correction
// residual kernels
// sets the loop condition on the device, so a step runs without any host
// round trip.  Loop exit is guaranteed by maxit / max_outer, with a device
// guard counter as a second stop.
// Learned warm start: replace K by the network's guess when its residual is
// smaller and point the oxygen set-up at K_prev (c.aux) for the linearisation.
int ws_before_o2(hca_handle* h, cudaStream_t s) {
  Ctx& c = h->ctx;
  c.lag = nullptr;
  if (!h->learned || !h->net) return HCA_OK;
  const RepDesc& r = h->reps_h[0];
  const hca_config& g = h->cfgs[0];
  hcanet::FeatureArgs f;
  f.state = c.state;
  f.perf = c.perf;
  f.nx = r.nx;
  f.ny = r.ny;
  f.nz = r.nz;
  f.pitch = r.nxp;
  f.base = r.off;
  f.D_K = g.D_K;
  f.dx = g.dx;
  f.phi_K = g.phi_K;
  f.K1 = g.K1;
  f.r_K = g.r_K;
  f.K0 = g.K0;
  const bool dc = !h->fp64 && h->max_outer > 0;
  const bool always = g.warm_start == HCA_WS_LEARNED_ALWAYS;
  const int rc = hcanet::ws_o2(h->net, f, h->fp64, always, c.K, dc ? static_cast<float*>(c.K_lo) : nullptr, c.aux,
                               h->ws_cand, h->ws_part, h->ws_res, s);
  if (rc) return rc;
  c.lag = c.aux;
  return HCA_OK;
}

int add_while(cudaStream_t s, cudaGraphConditionalHandle hnd, cudaGraph_t* body) {
  cudaStreamCaptureStatus st;
  cudaGraph_t g = nullptr;
  const cudaGraphNode_t* deps = nullptr;
  size_t nd = 0;
  HCA_TRY(cudaStreamGetCaptureInfo(s, &st, nullptr, &g, &deps, nullptr, &nd));
  if (st != cudaStreamCaptureStatusActive) return HCA_ERR_CUDA;
  cudaGraphNodeParams p = {};
  p.type = cudaGraphNodeTypeConditional;
  p.conditional.handle = hnd;
  p.conditional.type = cudaGraphCondTypeWhile;
  p.conditional.size = 1;
  cudaGraphNode_t node;
  HCA_TRY(cudaGraphAddNode(&node, g, deps, nullptr, nd, &p));
  HCA_TRY(cudaStreamUpdateCaptureDependencies(s, &node, nullptr, 1, cudaStreamSetCaptureDependencies));
  *body = p.conditional.phGraph_out[0];
  return HCA_OK;
}

int cap_solve(hca_handle* h, int which, cudaGraph_t G) {
  Ctx& c = h->ctx;
  cudaStream_t S = h->cap[0], S2 = h->cap[1], S3 = h->cap[2];
  const bool dc = !h->fp64 && h->max_outer > 0;
  int rc;
  if (!dc) {
    void* x = which == 0 ? c.K : c.G[which - 1];
    cudaGraphConditionalHandle H;
    HCA_TRY(cudaGraphConditionalHandleCreate(&H, G, 0, cudaGraphCondAssignDefault));
    const hca::CondArg cnd{H, 1};
    c.stream = S;
    hca::launch_setup(c, which, h->fp64, cnd);
    if (h->mg) mg_setup(h, which);
    HCA_TRY(cudaGetLastError());
    // the V-cycle opens the loop's body, so none runs after the pass B that
    // ends the loop (the set-up leaves r unscaled: no r scaling either)
    cudaGraph_t body;
    if ((rc = add_while(S, H, &body))) return rc;
    HCA_TRY(cudaStreamBeginCaptureToGraph(S2, body, nullptr, nullptr, 0, cudaStreamCaptureModeRelaxed));
    c.stream = S2;
    if (h->mg) vcycle(h, which, false);
    pass_a(h, which);
    pass_b(h, which, x, cnd);
    HCA_TRY(cudaGetLastError());
    HCA_TRY(cudaStreamEndCapture(S2, &body));
    c.stream = S;
    hca::launch_true_residual(c, which, x, h->fp64);
    HCA_TRY(cudaGetLastError());
    return HCA_OK;
  }
  void* xh = which == 0 ? c.K : c.G[which - 1];
  void* xl = which == 0 ? c.K_lo : c.G_lo[which - 1];
  cudaGraphConditionalHandle Ho, Hi;
  HCA_TRY(cudaGraphConditionalHandleCreate(&Ho, G, 0, cudaGraphCondAssignDefault));
  HCA_TRY(cudaGraphConditionalHandleCreate(&Hi, G, 0, cudaGraphCondAssignDefault));
  const hca::CondArg co{Ho, 1}, ci{Hi, 1};
  c.stream = S;
  hca::launch_dc_residual(c, which, xh, xl, true, co, ci);
  if (h->mg) mg_setup(h, which, true);
  HCA_TRY(cudaGetLastError());
  // Each loop's body opens with its V-cycle, so none runs after the residual
  // sweep that ends the outer loop or the pass B that ends an inner loop: the
  // outer body is the first inner iteration (a residual sweep that continues
  // the outer loop starts an inner solve) and the inner loop the others.
  cudaGraph_t bo, bi;
  if ((rc = add_while(S, Ho, &bo))) return rc;
  HCA_TRY(cudaStreamBeginCaptureToGraph(S2, bo, nullptr, nullptr, 0, cudaStreamCaptureModeRelaxed));
  c.stream = S2;
  if (h->mg) vcycle(h, which, true);
  pass_a(h, which);
  pass_b(h, which, c.dx, ci);
  HCA_TRY(cudaGetLastError());
  if ((rc = add_while(S2, Hi, &bi))) return rc;
  HCA_TRY(cudaStreamBeginCaptureToGraph(S3, bi, nullptr, nullptr, 0, cudaStreamCaptureModeRelaxed));
  c.stream = S3;
  if (h->mg) vcycle(h, which, false);
  pass_a(h, which);
  pass_b(h, which, c.dx, ci);
  HCA_TRY(cudaGetLastError());
  HCA_TRY(cudaStreamEndCapture(S3, &bi));
  c.stream = S2;
  hca::launch_dc_update(c, xh, xl);
  hca::launch_dc_residual(c, which, xh, xl, false, co, ci);
  HCA_TRY(cudaGetLastError());
  HCA_TRY(cudaStreamEndCapture(S2, &bo));
  c.stream = S;
  hca::launch_dc_update(c, xh, xl);
  HCA_TRY(cudaGetLastError());
  return HCA_OK;
}

// Blocks per replicate of the synchronous CA launches (all committed cells of
// a replicate in one grid-stride launch).
int ca_sync_blocks(const hca_handle* h) {
  return std::max(1, std::min(4096, 8 * h->ctx.sm_count / std::max(1, h->n_reps)));
}

int cap_stages(hca_handle* h, uint32_t mask, cudaGraph_t G) {
  Ctx& c = h->ctx;
  c.stream = h->cap[0];
  HCA_TRY(cudaMemsetAsync(c.stats, 0, sizeof(hca::DevStats) * h->n_reps, c.stream));
  HCA_TRY(cudaMemsetAsync(&c.sync->error, 0, sizeof(int), c.stream));
  HCA_TRY(cudaMemsetAsync(&c.sync->bar_count, 0, sizeof(unsigned int), c.stream));
  int rc;
  if (mask & HCA_STAGE_O2) {
    rc = ws_before_o2(h, c.stream);
    for (int j = 0; j < h->cfgs[0].o2_substeps && !rc && (j == 0 || h->cfgs[0].o2_scheme); ++j) {
      c.sub = j;
      rc = cap_solve(h, 0, G);
    }
    c.lag = nullptr;
    c.sub = 0;
    if (rc) return rc;
  }
  if ((mask & HCA_STAGE_O2) && h->vegf)
    for (int j = 0; j < h->cfgs[0].drug_substeps; ++j) {
      c.sub = j;
      rc = cap_solve(h, hca::WHICH_VEGF, G);
      c.sub = 0;
      if (rc) return rc;
    }
  if (mask & HCA_STAGE_DRUGS)
    for (int d = 0; d < h->n_drugs; ++d)
      for (int j = 0; j < h->cfgs[0].drug_substeps; ++j) {
        c.sub = j;
        rc = cap_solve(h, 1 + d, G);
        c.sub = 0;
        if (rc) return rc;
      }
  c.stream = h->cap[0];
  if (mask & HCA_STAGE_ODE) hca::launch_ode(c, h->fp64);
  if (mask & HCA_STAGE_CA) {
    HCA_TRY(cudaMemsetAsync(c.list_count, 0, sizeof(int) * 27 * h->n_reps, c.stream));
    hca::launch_ca_compact(c, h->fp64);
    if (h->ca_sync) {
      hca::launch_ca_sync(c, ca_sync_blocks(h), h->fp64);
    } else {
      if (h->ca_coop > 0) {
        hca::launch_ca_colours(c, h->ca_coop, h->fp64);
      } else {
        const int bx = std::max(1, std::min(1024, 2 * c.sm_count / std::max(1, h->n_reps)));
        for (int col = 0; col < 27; ++col) hca::launch_ca_colour(c, col, bx, h->fp64);
      }
    }
    if (h->vessels) {
      HCA_TRY(cudaMemsetAsync(c.vsum, 0, sizeof(unsigned long long) * 2 * h->n_reps, c.stream));
      hca::launch_vessels(c, h->fp64);
    }
  }
  if (mask & HCA_STAGE_ADVANCE) hca::launch_advance_step(c, 1);
  HCA_TRY(cudaGetLastError());
  return HCA_OK;
}

int build_graph(hca_handle* h, uint32_t mask, cudaGraphExec_t* out) {
  for (int k = 0; k < 3; ++k)
    if (!h->cap[k]) HCA_TRY(cudaStreamCreateWithFlags(&h->cap[k], cudaStreamNonBlocking));
  cudaGraph_t G;
  HCA_TRY(cudaGraphCreate(&G, 0));
  const cudaStream_t user = h->ctx.stream;
  int rc = HCA_OK;
  if (cudaStreamBeginCaptureToGraph(h->cap[0], G, nullptr, nullptr, 0, cudaStreamCaptureModeRelaxed) != cudaSuccess) {
    (void)cudaGetLastError();
    cudaGraphDestroy(G);
    return HCA_ERR_CUDA;
  }
  h->capturing = true;
  rc = cap_stages(h, mask, G);
  h->capturing = false;
  cudaGraph_t done = nullptr;
  cudaError_t e = cudaStreamEndCapture(h->cap[0], &done);
  h->ctx.stream = user;
  if (rc || e != cudaSuccess) {
    (void)cudaGetLastError();
    // leave any nested capture
    for (int k = 1; k < 3; ++k) {
      cudaStreamCaptureStatus st;
      if (cudaStreamIsCapturing(h->cap[k], &st) == cudaSuccess && st != cudaStreamCaptureStatusNone) {
        cudaGraph_t tmp;
        cudaStreamEndCapture(h->cap[k], &tmp);
      }
    }
    (void)cudaGetLastError();
    cudaGraphDestroy(G);
    return rc ? rc : HCA_ERR_CUDA;
  }
  e = cudaGraphInstantiate(out, G, 0);
  cudaGraphDestroy(G);
  if (e != cudaSuccess) {
    (void)cudaGetLastError();
    return HCA_ERR_CUDA;
  }
  return HCA_OK;
}

// Run one step's stages `mask` through its cached graph; returns HCA_ERR_CUDA
// (and disables graphs for the handle) if a graph cannot be built.
int run_graph(hca_handle* h, uint32_t mask, int times) {
  cudaGraphExec_t exec = nullptr;
  for (auto& g : h->graphs)
    if (g.mask == mask) exec = g.exec;
  if (!exec) {
    int rc = build_graph(h, mask, &exec);
    if (rc) {
      h->graphs_ok = false;
      return rc;
    }
    h->graphs.push_back({mask, exec});
  }
  for (int i = 0; i < times; ++i) {
    HCA_TRY(cudaGraphLaunch(exec, h->ctx.stream));
    if (mask & HCA_STAGE_ADVANCE) h->step += 1;
  }
  return HCA_OK;
}

int reset_step_stats(hca_handle* h) {
  HCA_TRY(cudaMemsetAsync(h->ctx.stats, 0, sizeof(hca::DevStats) * h->n_reps, h->ctx.stream));
  HCA_TRY(cudaMemsetAsync(&h->ctx.sync->error, 0, sizeof(int), h->ctx.stream));
  HCA_TRY(cudaMemsetAsync(&h->ctx.sync->bar_count, 0, sizeof(unsigned int), h->ctx.stream));
  return HCA_OK;
}

int run_ca(hca_handle* h) {
  Ctx& c = h->ctx;
  HCA_TRY(cudaMemsetAsync(c.list_count, 0, sizeof(int) * 27 * h->n_reps, c.stream));
  HCA_LAUNCH(h, HCA_KCLASS_CA_COMPACT, 1, hca::launch_ca_compact(c, h->fp64));
  if (h->ca_sync) {
    HCA_LAUNCH(h, HCA_KCLASS_CA_COLOUR, 4, hca::launch_ca_sync(c, ca_sync_blocks(h), h->fp64));
    return HCA_OK;
  }
  if (h->ca_coop > 0) {
    HCA_LAUNCH(h, HCA_KCLASS_CA_COLOUR, 1, hca::launch_ca_colours(c, h->ca_coop, h->fp64));
    return HCA_OK;
  }
  const int bx = std::max(1, std::min(1024, 2 * c.sm_count / std::max(1, h->n_reps)));
  for (int col = 0; col < 27; ++col) {
    HCA_LAUNCH(h, HCA_KCLASS_CA_COLOUR, 1, hca::launch_ca_colour(c, col, bx, h->fp64));
  }
  return HCA_OK;
}

int picard_oxygen(hca_handle* h);

int run_stages(hca_handle* h, uint32_t mask) {
  int rc = reset_step_stats(h);
  if (rc) return rc;
  int status = HCA_OK;
  if ((mask & HCA_STAGE_O2) && h->nonlinear) {
    rc = picard_oxygen(h);
    if (rc) return rc;
  } else if (mask & HCA_STAGE_O2) {
    rc = ws_before_o2(h, h->ctx.stream);
    for (int j = 0; j < h->cfgs[0].o2_substeps && !rc && (j == 0 || h->cfgs[0].o2_scheme); ++j) {
      h->ctx.sub = j;
      rc = solve(h, 0);
    }
    h->ctx.lag = nullptr;
    h->ctx.sub = 0;
    if (rc) return rc;
  }
  if ((mask & HCA_STAGE_O2) && h->vegf) {
    for (int j = 0; j < h->cfgs[0].drug_substeps && !rc; ++j) {
      h->ctx.sub = j;
      rc = solve(h, hca::WHICH_VEGF);
    }
    h->ctx.sub = 0;
    if (rc) return rc;
  }
  if (mask & HCA_STAGE_DRUGS) {
    for (int d = 0; d < h->n_drugs; ++d)
      for (int j = 0; j < h->cfgs[0].drug_substeps; ++j) {
        h->ctx.sub = j;
        rc = solve(h, 1 + d);
        if (rc) break;
      }
    h->ctx.sub = 0;
    if (rc) return rc;
  }
  if (mask & HCA_STAGE_ODE) {
    HCA_LAUNCH(h, HCA_KCLASS_ODE, 1, hca::launch_ode(h->ctx, h->fp64));
  }
  if (mask & HCA_STAGE_CA) {
    rc = run_ca(h);
    if (rc) return rc;
    if (h->vessels) {
      HCA_TRY(cudaMemsetAsync(h->ctx.vsum, 0, sizeof(unsigned long long) * 2 * h->n_reps, h->ctx.stream));
      HCA_LAUNCH(h, HCA_KCLASS_CA_COLOUR, 2, hca::launch_vessels(h->ctx, h->fp64));
    }
  }
  if (mask & HCA_STAGE_ADVANCE) {
    HCA_LAUNCH(h, HCA_KCLASS_OTHER, 1, hca::launch_advance_step(h->ctx, 1));
    h->step += 1;
  }
  return status;
}

int check_convergence(hca_handle* h) {
  std::vector<hca::DevStats> st(h->n_reps);
  HCA_TRY(cudaMemcpyAsync(st.data(), h->ctx.stats, sizeof(hca::DevStats) * h->n_reps, cudaMemcpyDeviceToHost,
                          h->ctx.stream));
  HCA_TRY(cudaMemcpyAsync(h->h_pinned, &h->ctx.sync->active_count, 2 * sizeof(int), cudaMemcpyDeviceToHost,
                          h->ctx.stream));
  HCA_TRY(cudaStreamSynchronize(h->ctx.stream));
  if (h->h_pinned[1]) return sync_error_status(h->h_pinned[1]);
  for (auto& s : st) {
    if (s.nonfinite) return HCA_ERR_NONFINITE;
  }
  for (auto& s : st)
    if (s.not_converged) return HCA_ERR_NOCONV;
  return HCA_OK;
}

// Launch-shape autotuner: times the oxygen CG passes (the hot pair) for each
// candidate block size (and register cap of the FP32 passes) on the handle's
// own lattices, best of three timed runs each, and keeps the fastest.  It runs at creation, on the solver's
// scratch vectors (x = aux), before anything depends on them; the reductions
// sum by rows in a fixed order, so results do not depend on the choice.
int autotune(hca_handle* h, bool tune_regs) {
  Ctx& c = h->ctx;
  const int cand_t[3] = {128, 256, 512};
  const int cand_r[4] = {64, 80, 96, 128};
  const int nr = (tune_regs && !h->fp64) ? 4 : 1;
  constexpr int kIters = 8, kReps = 3;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  HCA_TRY(cudaEventCreate(&e0));
  if (cudaEventCreate(&e1) != cudaSuccess) {
    cudaEventDestroy(e0);
    return HCA_ERR_CUDA;
  }
  float best = 1e30f;
  int bt = c.threads, br = c.pass_regs;
  int rc = HCA_OK;
  // the persistent row form runs at 128 threads: larger blocks timed faster
  // here now and then but ran pass A ~20 % slower inside a step
  const int nt = c.persist ? 1 : 3;
  for (int ti = 0; ti < nt && !rc; ++ti)
    for (int ri = 0; ri < nr && !rc; ++ri) {
      c.threads = cand_t[ti];
      if (nr > 1) c.pass_regs = cand_r[ri];
      hca::launch_setup(c, 0, h->fp64, kNoCond);
      for (int k = 0; k < 2; ++k) {   // warm-up
        pass_a(h, 0);
        pass_b(h, 0, c.aux, kNoCond);
      }
      // the best of kReps timed runs (a single run is noisy enough to pick a
      // slower shape now and then)
      float ms = 1e30f;
      for (int rep = 0; rep < kReps && !rc; ++rep) {
        cudaEventRecord(e0, c.stream);
        for (int k = 0; k < kIters; ++k) {
          pass_a(h, 0);
          pass_b(h, 0, c.aux, kNoCond);
        }
        cudaEventRecord(e1, c.stream);
        float t = 0.f;
        if (cudaGetLastError() != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess ||
            cudaEventElapsedTime(&t, e0, e1) != cudaSuccess) {
          rc = HCA_ERR_CUDA;
          break;
        }
        ms = std::min(ms, t);
      }
      if (rc) break;
      h->launches += 1 + 2 * (kReps * kIters + 2);
      if (ms < best) {
        best = ms;
        bt = c.threads;
        br = c.pass_regs;
      }
    }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  c.threads = bt;
  c.pass_regs = br;
  if (rc) return rc;
  // the timed passes may have left solver flags set; the solves reset the rest
  HCA_TRY(cudaMemsetAsync(&c.sync->error, 0, sizeof(int), c.stream));
  HCA_TRY(cudaMemsetAsync(&c.sync->bar_count, 0, sizeof(unsigned int), c.stream));
  HCA_TRY(cudaStreamSynchronize(c.stream));
  return HCA_OK;
}

// Oxygen fixed point: Picard iteration of the lagged linearisation from the
// current K (K0 at creation) until ||K_new - K_old|| <= picard_tol ||K_new||
// for every replicate; its limit solves the nonlinear quasi-steady Eq. (oxygen).
int picard_oxygen_impl(hca_handle* h);

int picard_oxygen(hca_handle* h) {
  // the fixed point is that of the quasi-steady form, whatever the time scheme
  const RepDesc* reps = h->ctx.reps;
  if (h->reps_qs) h->ctx.reps = h->reps_qs;
  const int rc = picard_oxygen_impl(h);
  h->ctx.reps = reps;
  return rc;
}

int picard_oxygen_impl(hca_handle* h) {
  Ctx& c = h->ctx;
  double tol = 0;
  int maxit = 0;
  for (auto& cf : h->cfgs) {
    tol = std::max(tol, cf.picard_tol);
    maxit = std::max(maxit, cf.picard_maxit);
  }
  const size_t bytes = (size_t)h->total * elem_size(h);
  // a replicate that has converged is frozen, so a batch gives every
  // replicate exactly the iterations it would get alone
  std::vector<int> frozen(h->n_reps, 0);
  int it = 0;
  for (it = 1; it <= maxit; ++it) {
    HCA_TRY(cudaMemcpyAsync(c.aux, c.K, bytes, cudaMemcpyDeviceToDevice, c.stream));
    int rc = solve(h, 0);
    if (rc) return rc;
    HCA_LAUNCH(h, HCA_KCLASS_OTHER, 1, hca::launch_diff_norms(c, c.K, c.aux, h->fp64));
    std::vector<hca::RepSolve> sv(h->n_reps);
    HCA_TRY(cudaMemcpyAsync(sv.data(), c.solve, sizeof(hca::RepSolve) * h->n_reps, cudaMemcpyDeviceToHost, c.stream));
    HCA_TRY(cudaStreamSynchronize(c.stream));
    bool all = true;
    for (int r = 0; r < h->n_reps; ++r) {
      if (frozen[r]) continue;
      const double change = std::sqrt(sv[r].rnorm2), norm = std::sqrt(sv[r].bnorm2);
      if (!std::isfinite(change) || !std::isfinite(norm)) return HCA_ERR_NONFINITE;
      if (norm == 0.0 || change <= h->cfgs[r].picard_tol * norm || it >= h->cfgs[r].picard_maxit) frozen[r] = 1;
      else all = false;
    }
    if (all) break;
    HCA_TRY(cudaMemcpyAsync(c.frozen, frozen.data(), sizeof(int) * h->n_reps, cudaMemcpyHostToDevice, c.stream));
  }
  HCA_TRY(cudaMemsetAsync(c.frozen, 0, sizeof(int) * h->n_reps, c.stream));
  HCA_TRY(cudaStreamSynchronize(c.stream));
  h->picard_iterations = std::min(it, maxit);
  return HCA_OK;
}

int create_impl(int n, const hca_config* cfgs, const float* const* p_cell, const float* const* perf,
                const float* const* p_vessel, int maps_on_device, hca_handle** out, bool initial_o2 = true) {
  if (!out || n < 1 || !cfgs || !p_cell || !perf || !p_vessel) return HCA_ERR_ARG;
  *out = nullptr;
  for (int i = 0; i < n; ++i) {
    int rc = validate(cfgs[i]);
    if (rc) return rc;
    if (!p_cell[i] || !perf[i] || !p_vessel[i]) return HCA_ERR_ARG;
    if (cfgs[i].precision != cfgs[0].precision || cfgs[i].n_drugs != cfgs[0].n_drugs ||
        cfgs[i].dt != cfgs[0].dt || cfgs[i].threads_per_block != cfgs[0].threads_per_block ||
        cfgs[i].stream != cfgs[0].stream || cfgs[i].o2_nonlinear != cfgs[0].o2_nonlinear ||
        cfgs[i].drug_scheme != cfgs[0].drug_scheme || cfgs[i].drug_substeps != cfgs[0].drug_substeps ||
        cfgs[i].o2_scheme != cfgs[0].o2_scheme || cfgs[i].o2_substeps != cfgs[0].o2_substeps ||
        cfgs[i].ca_mode != cfgs[0].ca_mode || cfgs[i].vegf != cfgs[0].vegf)
      return HCA_ERR_ARG;
    // the learned warm start and the multigrid hierarchy serve one lattice
    if (cfgs[i].warm_start != HCA_WS_PREV && n > 1) return HCA_ERR_UNIMPLEMENTED;
    if (cfgs[i].preconditioner != cfgs[0].preconditioner) return HCA_ERR_ARG;
  }
  hca_handle* h = new (std::nothrow) hca_handle();
  if (!h) return HCA_ERR_OOM;
  h->n_reps = n;
  h->fp64 = cfgs[0].precision == HCA_FP64;
  h->n_drugs = cfgs[0].n_drugs;
  h->stream = (cudaStream_t)cfgs[0].stream;
  h->cfgs.assign(cfgs, cfgs + n);
  h->learned = cfgs[0].warm_start != HCA_WS_PREV;
  h->mg = cfgs[0].preconditioner == HCA_PC_MG;
  h->nonlinear = cfgs[0].o2_nonlinear != 0;
  h->ca_sync = cfgs[0].ca_mode == 1;
  h->vegf = cfgs[0].vegf != 0;
  for (int i = 0; i < n; ++i) h->vessels = h->vessels || cfgs[i].vessel_interval > 0;
  if (h->nonlinear) h->graphs_ok = false;   // each Picard iterate is checked on the host
  {
    // HCA_NO_GRAPH=1 runs steps from a host loop instead of the step graph
    const char* ng = std::getenv("HCA_NO_GRAPH");
    if (ng && ng[0] == '1') h->graphs_ok = false;
  }
  cudaGetDevice(&h->device);
  int sm = 0;
  cudaDeviceGetAttribute(&sm, cudaDevAttrMultiProcessorCount, h->device);
  h->ctx.sm_count = sm > 0 ? sm : 1;

  // layout
  long long off = 0, loff = 0;
  int chunk0 = 0, super0 = 0;
  for (int i = 0; i < n; ++i) {
    RepDesc r = make_desc(cfgs[i]);
    r.off = off;
    off += ((long long)r.nxp * r.ny * r.nz + kFieldAlign - 1) / kFieldAlign * kFieldAlign;
    const int rows = r.ny * r.nz;
    r.chunk_begin = chunk0;
    // rows per chunk: CHUNK_ROWS, halved while the lattice would give fewer
    // than 1024 chunks and a chunk keeps at least one row per warp of an
    // 8-warp block (lattices with few rows, e.g. flat ones, get more blocks);
    // it depends on the lattice's shape only, so results do not depend on the
    // launch configuration or on the other replicates of a batch
    {
      const int min_rows = std::min(hca::CHUNK_ROWS, 8 * (32 / r.lpr));
      int cr = hca::CHUNK_ROWS;
      while (cr > min_rows && rows / cr < 1024) cr >>= 1;
      r.chunk_rows = cr;
    }
    r.n_chunks = (rows + r.chunk_rows - 1) / r.chunk_rows;
    r.super_begin = super0;
    r.n_supers = (r.n_chunks + hca::SUPER_CHUNKS - 1) / hca::SUPER_CHUNKS;
    super0 += r.n_supers;
    for (int k = 0; k < r.n_chunks; ++k) h->chunks_h.push_back(make_int2(i, k * r.chunk_rows));
    chunk0 += r.n_chunks;
    for (int col = 0; col < 27; ++col) {
      const int cap = colour_count(r.nx, col % 3) * colour_count(r.ny, (col / 3) % 3) * colour_count(r.nz, col / 9);
      r.list_off[col] = loff;
      r.list_cap[col] = cap;
      loff += cap;
    }
    h->maxit_all = std::max(h->maxit_all, r.maxit);
    h->max_outer = std::max(h->max_outer, r.max_outer);
    h->reps_h.push_back(r);
  }
  h->total = off;
  h->lists_total = loff;

  Ctx& c = h->ctx;
  c.n_reps = n;
  c.n_chunks = chunk0;
  c.n_supers = super0;
  // 128 threads per block measured fastest for the CG passes on GB300
  c.threads = cfgs[0].threads_per_block ? cfgs[0].threads_per_block : 128;
  c.pass_regs = 96;   // measured best at 128 threads; the autotuner may change both
  {
    // HCA_PASS_REGS=64|80|96|128 fixes the CG passes' register cap
    const char* pr = std::getenv("HCA_PASS_REGS");
    if (pr) c.pass_regs = std::atoi(pr);
  }
  c.stream = h->stream;
  const size_t es = elem_size(h);
  const size_t fbytes = (size_t)h->total * es;
  int rc = HCA_OK;
#define ALLOC(ptr, bytes) \
  if ((rc = dev_alloc(h, &(ptr), (bytes))) != HCA_OK) goto fail
  {
    RepDesc* reps_d;
    int2* chunks_d;
    ALLOC(reps_d, sizeof(RepDesc) * n);
    ALLOC(chunks_d, sizeof(int2) * chunk0);
    c.reps = reps_d;
    c.chunks = chunks_d;
    if (cfgs[0].o2_scheme) {
      h->reps_qs_h = h->reps_h;
      for (auto& r : h->reps_qs_h) {
        r.o2_mass = 0.0;
        r.bx[0] = 0.0;
        r.bax[0] = 0;
        r.nsub[0] = 1;
      }
      ALLOC(h->reps_qs, sizeof(RepDesc) * n);
    }
    ALLOC(c.state, (size_t)h->total + 16);
    ALLOC(c.K, fbytes);
    if (!h->fp64) ALLOC(c.K_lo, fbytes);
    for (int d = 0; d < h->n_drugs; ++d) ALLOC(c.G[d], fbytes);
    if (h->vegf) ALLOC(c.G[hca::VEGF_SLOT], fbytes);
    if (h->vessels) ALLOC(c.vsum, sizeof(unsigned long long) * 2 * (size_t)n);
    if (!h->fp64) {
      for (int d = 0; d < h->n_drugs; ++d) ALLOC(c.G_lo[d], fbytes);
      if (h->vegf) ALLOC(c.G_lo[hca::VEGF_SLOT], fbytes);
      ALLOC(c.dx, fbytes);
      ALLOC(c.reac, fbytes);
    }
    ALLOC(c.phi, fbytes);
    ALLOC(c.P, fbytes);
    ALLOC(c.Vc, fbytes);
    ALLOC(c.perf, fbytes);
    ALLOC(c.z, fbytes);
    ALLOC(c.p, fbytes);
    ALLOC(c.p_alt, fbytes);
    ALLOC(c.q, fbytes);
    ALLOC(c.d, fbytes);
    ALLOC(c.b, fbytes);
    ALLOC(c.aux, fbytes);
    if (h->mg) {
      // one hierarchy per replicate; each coarse level's arrays hold all
      // replicates back to back
      hca::MGHost& H = h->mgh;
      std::vector<hca::MGLevel> lv((size_t)n * hca::MG_MAXLEV);
      std::vector<int2> rep(n);
      std::vector<long long> start((size_t)hca::MG_MAXLEV * (n + 1), 0);
      for (int i = 0; i < n; ++i) {
        const RepDesc& r0 = h->reps_h[i];
        int nx = r0.nx, ny = r0.ny, nz = r0.nz;
        long long nn = (long long)nx * ny * nz;
        int nl = 1;
        start[i + 1] = start[i] + nn;   // level 0 (the lattices)
        double cs = 1.0;
        // coarsen while the level is large and some extent exceeds 1; the
        // coupling grows by 2^k / 4 for the k extents above 1 (2 on a 3-D
        // lattice, 1 on a flat one)
        while (nn > hca::MG_MIN_SITES && std::max(nx, std::max(ny, nz)) > 1 && nl < hca::MG_MAXLEV) {
          const int k = (nx > 1) + (ny > 1) + (nz > 1);
          cs *= std::ldexp(1.0, k - 2);
          nx = (nx + 1) / 2;
          ny = (ny + 1) / 2;
          nz = (nz + 1) / 2;
          nn = (long long)nx * ny * nz;
          hca::MGLevel& L = lv[(size_t)i * hca::MG_MAXLEV + nl];
          L.nx = nx;
          L.ny = ny;
          L.nz = nz;
          L.n = nn;
          L.cscale = cs;
          L.cscale32 = (float)cs;
          nl += 1;
        }
        int small = nl - 1;
        for (int l = 1; l < nl; ++l)
          if (lv[(size_t)i * hca::MG_MAXLEV + l].n <= hca::MG_SMALL_SITES) {
            small = l;
            break;
          }
        rep[i] = make_int2(nl, small);
        H.nlev = std::max(H.nlev, nl);
        H.small = std::max(H.small, small);
      }
      if (n > 1 && H.nlev > 0)
        for (int i = 0; i < n; ++i)
          if (rep[i].x == 1) {   // a batch needs a coarse level in every replicate
            rc = HCA_ERR_UNIMPLEMENTED;
            goto fail;
          }
      for (int l = 1; l < H.nlev; ++l) {
        long long tot = 0;
        for (int i = 0; i < n; ++i) {
          start[(size_t)l * (n + 1) + i] = tot;
          if (l < rep[i].x) tot += lv[(size_t)i * hca::MG_MAXLEV + l].n;
        }
        start[(size_t)l * (n + 1) + n] = tot;
        H.ntot[l] = tot;
        char* arr[5];
        for (int k = 0; k < 5; ++k) ALLOC(arr[k], es * (size_t)std::max(1LL, tot));
        for (int k = 0; k < 5; ++k)
          if (cudaMemsetAsync(arr[k], 0, es * (size_t)std::max(1LL, tot), c.stream)) {
            rc = HCA_ERR_CUDA;
            goto fail;
          }
        for (int i = 0; i < n; ++i) {
          if (l >= rep[i].x) continue;
          hca::MGLevel& L = lv[(size_t)i * hca::MG_MAXLEV + l];
          const size_t o = es * (size_t)start[(size_t)l * (n + 1) + i];
          L.x = arr[0] + o;
          L.t = arr[1] + o;
          L.rhs = arr[2] + o;
          L.d = arr[3] + o;
          L.w = arr[4] + o;
        }
      }
      H.ntot[0] = start[n];
      std::vector<long long> rowstart(n + 1, 0);
      for (int i = 0; i < n; ++i) {
        const hca::MGLevel& L1 = lv[(size_t)i * hca::MG_MAXLEV + 1];
        rowstart[i + 1] = rowstart[i] + (rep[i].x > 1 ? (long long)L1.ny * L1.nz * h->reps_h[i].gpr : 0);
      }
      H.nrowitems = rowstart[n];
      H.launches = hca::vcycle_launches(H, false);
      // row-vector coarse kernels: level l qualifies when the level's rows of
      // every replicate that runs it on the grid (l below its single-block
      // levels) are whole 4-site groups; item prefix tables per level
      // (HCA_MG_GENERIC=1 keeps the per-site form)
      std::vector<long long> post_pre((size_t)hca::MG_MAXLEV * (n + 1), 0), restr_pre(post_pre.size(), 0);
      {
        const char* gen = std::getenv("HCA_MG_GENERIC");
        const bool allow = !(gen && gen[0] == '1');
        for (int l = 1; l < H.small && allow; ++l) {
          bool ok = true;
          long long pp = 0, rp = 0;
          for (int i = 0; i < n; ++i) {
            post_pre[(size_t)l * (n + 1) + i] = pp;
            restr_pre[(size_t)l * (n + 1) + i] = rp;
            if (l >= rep[i].y) continue;   // this replicate runs level l in the single-block kernel
            const hca::MGLevel& F = lv[(size_t)i * hca::MG_MAXLEV + l];
            const hca::MGLevel& C = lv[(size_t)i * hca::MG_MAXLEV + l + 1];
            if (F.nx % 4 != 0) ok = false;
            pp += (long long)F.ny * F.nz * (F.nx / 4);
            rp += (long long)C.ny * C.nz * (F.nx / 4);
          }
          post_pre[(size_t)l * (n + 1) + n] = pp;
          restr_pre[(size_t)l * (n + 1) + n] = rp;
          if (ok) {
            H.rows_ok |= 1u << l;
            H.post_items[l] = pp;
            H.restr_items[l] = rp;
          }
        }
      }
      {
        // shared-memory footprint of the single-block levels (x, t, rhs, d, w)
        long long smem = 0;
        for (int i = 0; i < n; ++i) {
          long long s = 0;
          for (int l = rep[i].y; l < rep[i].x; ++l) s += 5 * lv[(size_t)i * hca::MG_MAXLEV + l].n * (long long)es;
          smem = std::max(smem, s);
        }
        hca::mg_coop_config(H, h->fp64, c.sm_count, smem);
        H.launches = hca::vcycle_launches(H, false);
      }
      ALLOC(c.r, fbytes);
      ALLOC(c.mg_t0, fbytes);
      ALLOC(c.mg_w, fbytes);
      if (n == 1 && !h->fp64) {
        int dims[3 * hca::MG_MAXLEV] = {};
        for (int l = 0; l < hca::MG_MAXLEV; ++l) {
          dims[3 * l] = lv[l].nx;
          dims[3 * l + 1] = lv[l].ny;
          dims[3 * l + 2] = lv[l].nz;
        }
        hca::mg_zmarch_config(H, h->reps_h[0], c.sm_count, (const float*)c.r, (const float*)c.mg_w, dims);
      }
      hca::MGLevel* lv_d;
      long long* start_d;
      long long* rowstart_d;
      int2* rep_d;
      ALLOC(rowstart_d, sizeof(long long) * (n + 1));
      ALLOC(lv_d, sizeof(hca::MGLevel) * lv.size());
      ALLOC(start_d, sizeof(long long) * start.size());
      ALLOC(rep_d, sizeof(int2) * n);
      if (cudaMemcpyAsync(lv_d, lv.data(), sizeof(hca::MGLevel) * lv.size(), cudaMemcpyHostToDevice, c.stream) ||
          cudaMemcpyAsync(start_d, start.data(), sizeof(long long) * start.size(), cudaMemcpyHostToDevice,
                          c.stream) ||
          cudaMemcpyAsync(rep_d, rep.data(), sizeof(int2) * n, cudaMemcpyHostToDevice, c.stream) ||
          cudaMemcpyAsync(rowstart_d, rowstart.data(), sizeof(long long) * (n + 1), cudaMemcpyHostToDevice,
                          c.stream) ||
          cudaStreamSynchronize(c.stream)) {
        rc = HCA_ERR_CUDA;
        goto fail;
      }
      c.mg_lv = lv_d;
      c.mg_start = start_d;
      c.mg_rep = rep_d;
      c.mg_rowstart = rowstart_d;
      {
        long long* pre_d;
        ALLOC(pre_d, sizeof(long long) * 2 * post_pre.size());
        if (cudaMemcpyAsync(pre_d, post_pre.data(), sizeof(long long) * post_pre.size(), cudaMemcpyHostToDevice,
                            c.stream) ||
            cudaMemcpyAsync(pre_d + post_pre.size(), restr_pre.data(), sizeof(long long) * restr_pre.size(),
                            cudaMemcpyHostToDevice, c.stream) ||
            cudaStreamSynchronize(c.stream)) {
          rc = HCA_ERR_CUDA;
          goto fail;
        }
        c.mg_post_items = pre_d;
        c.mg_restr_items = pre_d + post_pre.size();
      }
      c.mg = 1;
    }
    if (h->learned) {
      ALLOC(h->ws_cand, sizeof(double) * (size_t)h->total);
      ALLOC(h->ws_part, sizeof(double) * 3 * hcanet::kWsNormBlocks);
      ALLOC(h->ws_res, sizeof(hcanet::WsResult));
    }
    ALLOC(c.partial, sizeof(double) * hca::NDOT * chunk0);
    ALLOC(c.sync, sizeof(hca::PassSync));
    ALLOC(c.solve, sizeof(hca::RepSolve) * n);
    ALLOC(c.stats, sizeof(hca::DevStats) * n);
    ALLOC(c.step, sizeof(long long));
    ALLOC(c.lists, sizeof(uint32_t) * (size_t)std::max(1LL, h->lists_total));
    if (h->ca_sync) {
      ALLOC(c.ca_dec, sizeof(long long) * (size_t)std::max(1LL, h->lists_total));
      ALLOC(c.claim_phi, sizeof(unsigned long long) * (size_t)h->total);
      ALLOC(c.claim_idx, sizeof(unsigned int) * (size_t)h->total);
    }
    ALLOC(c.list_count, sizeof(int) * 27 * n);
    ALLOC(c.n_kernels, sizeof(unsigned long long));
    ALLOC(c.frozen, sizeof(int) * n);
    ALLOC(c.rowp, sizeof(double) * hca::NDOT * hca::CHUNK_ROWS * (size_t)chunk0);
    ALLOC(c.chunk_cnt, sizeof(int) * (size_t)chunk0);
    ALLOC(c.superp, sizeof(double) * hca::NDOT * (size_t)super0);
    ALLOC(c.super_cnt, sizeof(int) * (size_t)super0);
    if (cudaMallocHost(&h->h_pinned, 4 * sizeof(int)) != cudaSuccess) {
      (void)cudaGetLastError();
      rc = HCA_ERR_OOM;
      goto fail;
    }
    h->h_pinned[0] = h->h_pinned[1] = 0;
    cudaStream_t s = c.stream;
    if ((h->reps_qs &&
         cudaMemcpyAsync(h->reps_qs, h->reps_qs_h.data(), sizeof(RepDesc) * n, cudaMemcpyHostToDevice, s)) ||
        cudaMemcpyAsync(reps_d, h->reps_h.data(), sizeof(RepDesc) * n, cudaMemcpyHostToDevice, s) ||
        cudaMemcpyAsync(chunks_d, h->chunks_h.data(), sizeof(int2) * chunk0, cudaMemcpyHostToDevice, s)) {
      rc = HCA_ERR_CUDA;
      goto fail;
    }
    // zero every device array (padding sites must hold 0)
    void* zero_list[] = {c.K, c.K_lo, c.G[0], c.G[1], c.G[2], c.G[3], c.G_lo[0], c.G_lo[1], c.G_lo[2], c.G_lo[3], c.dx,
                         c.phi, c.P, c.Vc, c.perf, c.z, c.p, c.p_alt, c.q, c.d, c.b, c.aux, c.reac, c.r, c.mg_t0, c.mg_w};
    for (void* p : zero_list)
      if (p && cudaMemsetAsync(p, 0, fbytes, s)) {
        rc = HCA_ERR_CUDA;
        goto fail;
      }
    if (cudaMemsetAsync(c.state, 0, (size_t)h->total + 16, s) || cudaMemsetAsync(c.sync, 0, sizeof(hca::PassSync), s) ||
        cudaMemsetAsync(c.solve, 0, sizeof(hca::RepSolve) * n, s) ||
        cudaMemsetAsync(c.stats, 0, sizeof(hca::DevStats) * n, s) || cudaMemsetAsync(c.step, 0, sizeof(long long), s) ||
        cudaMemsetAsync(c.list_count, 0, sizeof(int) * 27 * n, s) ||
        cudaMemsetAsync(c.n_kernels, 0, sizeof(unsigned long long), s) ||
        cudaMemsetAsync(c.frozen, 0, sizeof(int) * n, s) ||
        cudaMemsetAsync(c.chunk_cnt, 0, sizeof(int) * (size_t)chunk0, s) ||
        cudaMemsetAsync(c.super_cnt, 0, sizeof(int) * (size_t)super0, s) ||
        (h->ws_res && cudaMemsetAsync(h->ws_res, 0, sizeof(hcanet::WsResult), s))) {
      rc = HCA_ERR_CUDA;
      goto fail;
    }
    {
      hca::PassSync ps{};
      ps.guard_limit = h->maxit_all + 4;
      ps.guard_outer_limit = h->max_outer + 2;
      if (cudaMemcpyAsync(c.sync, &ps, sizeof(ps), cudaMemcpyHostToDevice, s) || cudaStreamSynchronize(s)) {
        rc = HCA_ERR_CUDA;
        goto fail;
      }
    }
    // maps -> padded float staging buffers
    float *pc_d = nullptr, *pf_d = nullptr, *pv_d = nullptr;
    int* err_d = nullptr;
    const size_t mbytes = (size_t)h->total * sizeof(float);
    if (cudaMalloc(&pc_d, mbytes) || cudaMalloc(&pf_d, mbytes) || cudaMalloc(&pv_d, mbytes) ||
        cudaMalloc(&err_d, sizeof(int))) {
      (void)cudaGetLastError();
      cudaFree(pc_d);
      cudaFree(pf_d);
      cudaFree(pv_d);
      cudaFree(err_d);
      rc = HCA_ERR_OOM;
      goto fail;
    }
    bool ok = cudaMemsetAsync(pc_d, 0, mbytes, s) == cudaSuccess && cudaMemsetAsync(pf_d, 0, mbytes, s) == cudaSuccess &&
              cudaMemsetAsync(pv_d, 0, mbytes, s) == cudaSuccess && cudaMemsetAsync(err_d, 0, sizeof(int), s) == cudaSuccess;
    for (int i = 0; i < n && ok; ++i) {
      const RepDesc& r = h->reps_h[i];
      const float* srcs[3] = {p_cell[i], perf[i], p_vessel[i]};
      float* dsts[3] = {pc_d, pf_d, pv_d};
      for (int k = 0; k < 3 && ok; ++k)
        ok = cudaMemcpy2DAsync(dsts[k] + r.off, (size_t)r.nxp * sizeof(float), srcs[k], (size_t)r.nx * sizeof(float),
                               (size_t)r.nx * sizeof(float), (size_t)r.ny * r.nz, cudaMemcpyDefault, s) == cudaSuccess;
    }
    if (ok) {
      hca::launch_init(c, pc_d, pf_d, pv_d, err_d, h->fp64);
      h->launches++;
      ok = cudaGetLastError() == cudaSuccess;
    }
    int err_h = 0;
    if (ok) ok = cudaMemcpyAsync(&err_h, err_d, sizeof(int), cudaMemcpyDeviceToHost, s) == cudaSuccess;
    if (ok) ok = cudaStreamSynchronize(s) == cudaSuccess;
    cudaFree(pc_d);
    cudaFree(pf_d);
    cudaFree(pv_d);
    cudaFree(err_d);
    if (!ok) {
      (void)cudaGetLastError();
      rc = HCA_ERR_CUDA;
      goto fail;
    }
    if (err_h) {
      rc = HCA_ERR_NONFINITE;
      goto fail;
    }
    {
      // a common groups-per-lane count lets the passes use a compile-time trip count
      int ni = -1;
      for (auto& r : h->reps_h) {
        const int v = (r.gpr + r.lpr - 1) / r.lpr;
        ni = (ni < 0 || ni == v) ? v : 0;
      }
      c.pass_ni = ni == 1 || ni == 2 || ni == 4 ? ni : 0;
      h->mgh.ni = c.pass_ni;
      // persistent row kernels for one FP32 lattice with one row per warp
      // (HCA_PERSIST=0 keeps one block per chunk)
      const char* pe = std::getenv("HCA_PERSIST");
      c.persist = (!(pe && pe[0] == '0') && n == 1 && !h->fp64 && h->reps_h[0].lpr == 32 && c.pass_ni > 0) ? 1 : 0;
      const char* pd = std::getenv("HCA_PDL");
      c.pdl = (pd && pd[0] == '0') ? 0 : 1;
      // a V-cycle whose z no solve reads (after the pass B, set-up or residual
      // sweep that ended every replicate's iteration) returns at once
      c.skip_idle = 1;
      // the 27 colour sweeps of the CA in one cooperative launch (HCA_CA_COOP=0: one launch per colour)
      h->ca_coop = hca::ca_coop_blocks(h->fp64, c.sm_count);
    }
    if (!cfgs[0].threads_per_block) {
      const char* nt = std::getenv("HCA_NO_TUNE");
      if (!(nt && nt[0] == '1')) {
        rc = autotune(h, std::getenv("HCA_PASS_REGS") == nullptr);
        if (rc) goto fail;
      }
    }
    if (initial_o2) {
      rc = picard_oxygen(h);
      if (rc) goto fail;
    }
    rc = reset_step_stats(h);
    if (rc) goto fail;
  }
#undef ALLOC
  *out = h;
  return HCA_OK;
fail:
  free_all(h);
  delete h;
  return rc;
}

int copy_field(hca_handle* h, int rep, void* field, size_t es, void* host_or_dev, bool to_user, size_t user_offset_elems) {
  const RepDesc& r = h->reps_h[rep];
  char* f = (char*)field + (size_t)r.off * es;
  char* u = (char*)host_or_dev + user_offset_elems * es;
  cudaError_t e;
  if (to_user)
    e = cudaMemcpy2DAsync(u, (size_t)r.nx * es, f, (size_t)r.nxp * es, (size_t)r.nx * es, (size_t)r.ny * r.nz,
                          cudaMemcpyDefault, h->ctx.stream);
  else
    e = cudaMemcpy2DAsync(f, (size_t)r.nxp * es, u, (size_t)r.nx * es, (size_t)r.nx * es, (size_t)r.ny * r.nz,
                          cudaMemcpyDefault, h->ctx.stream);
  if (e != cudaSuccess) {
    (void)cudaGetLastError();
    return HCA_ERR_CUDA;
  }
  return HCA_OK;
}

int check_rep(hca_handle* h, int rep) { return (h && rep >= 0 && rep < h->n_reps) ? HCA_OK : HCA_ERR_ARG; }

// ---------------------------------------------------------- checkpoints --
struct CkptHeader {
  char magic[8];
  int32_t version, config_size, n_reps, precision;
  int64_t step;
  int32_t picard_iterations, pad;
};
constexpr char kCkptMagic[8] = {'H', 'C', 'A', 'C', 'K', 'P', 'T', '1'};

// The device fields of replicate `rep` in checkpoint order (null entries are
// skipped consistently on save and load).
std::vector<void*> ckpt_fields(hca_handle* h) {
  Ctx& c = h->ctx;
  std::vector<void*> f{c.K, c.K_lo};
  for (int d = 0; d < h->n_drugs; ++d) {
    f.push_back(c.G[d]);
    f.push_back(c.G_lo[d]);
  }
  if (h->vegf) {
    f.push_back(c.G[hca::VEGF_SLOT]);
    f.push_back(c.G_lo[hca::VEGF_SLOT]);
  }
  f.push_back(c.phi);
  f.push_back(c.P);
  f.push_back(c.Vc);
  return f;
}

// Copy the states of replicate rep between the device and a host buffer.
int copy_states(hca_handle* h, int rep, uint8_t* host, bool to_host) {
  const RepDesc& r = h->reps_h[rep];
  const cudaError_t e =
      to_host ? cudaMemcpy2DAsync(host, (size_t)r.nx, h->ctx.state + r.off, (size_t)r.nxp, (size_t)r.nx,
                                  (size_t)r.ny * r.nz, cudaMemcpyDeviceToHost, h->ctx.stream)
              : cudaMemcpy2DAsync(h->ctx.state + r.off, (size_t)r.nxp, host, (size_t)r.nx, (size_t)r.nx,
                                  (size_t)r.ny * r.nz, cudaMemcpyHostToDevice, h->ctx.stream);
  if (e != cudaSuccess) {
    (void)cudaGetLastError();
    return HCA_ERR_CUDA;
  }
  return HCA_OK;
}

}  // namespace

// ==================================================================== ABI ==
extern "C" {

int hca_config_default(hca_config* c, int32_t nx, int32_t ny, int32_t nz) {
  if (!c) return HCA_ERR_ARG;
  std::memset(c, 0, sizeof(*c));
  c->struct_size = sizeof(hca_config);
  c->nx = nx;
  c->ny = ny;
  c->nz = nz;
  c->precision = HCA_FP64;
  c->n_drugs = 1;
  c->seed = 0;
  c->dx = 10.0;
  c->dt = 60.0;
  c->rtol_o2 = 1e-8;
  c->rtol_drug = 1e-8;
  c->maxit = 20000;
  c->ode_substeps = 60;
  c->picard_tol = 1e-8;
  c->picard_maxit = 100;
  c->drug_substeps = 1;
  c->o2_substeps = 1;
  c->D_V = 3.52e3;
  c->psi_V = 1e-2;
  c->a_V = 6.66e-6;
  c->V_low = 1e-6;
  c->V_high = 1e-3;
  c->p_death = 0.1;
  c->beta_birth = 0.05;
  c->V_sprout = 1e-4;
  c->mm_vmax = 1.75;
  c->mm_km = 27.0;
  c->epi_w[0] = 18e3;
  c->epi_w[1] = 957e3;
  c->epi_w[2] = 25e3;
  c->epi_q2 = 0.918e3;
  c->epi_q3 = 0.25e3;
  c->epi_cl2 = 0.983e3;
  c->dose_interval = 21;
  c->D_K = 1.05e5;
  c->phi_K = 900.0;
  c->K1 = 2.5;
  c->K0 = 20.0;
  c->r_K = 1.88e4;
  for (int d = 0; d < 3; ++d) {
    c->D_G[d] = 9.6e3;
    c->psi_G[d] = 1e-2;
    c->kappa_G[d] = 2.0;
    c->uptake_G[d] = 0.0;
    c->dose_peak[d] = 1.0;
    c->kill_b[d] = 1;
  }
  c->plasma_decay[0] = 3.93e3 / 2430e3;  // cl3 / u, cyclophosphamide
  c->plasma_decay[1] = 0.983e3 / 18e3;   // cl2 / w1, epirubicin elimination
  c->plasma_decay[2] = 1.75 / 27.0;      // v_max / k_m, fluorouracil, linear regime
  c->T_cycle = 3.74 * 24 * 60;
  c->K_phi = 1.4;
  c->k1 = 4e-4;
  c->k1p = 0.01;
  c->K_p53 = 0.01;
  c->k2 = 2e-3;
  c->k2p = 0.01;
  c->k2pp = -2e-4;
  c->J5 = 0.04;
  c->K_V = 0.01;
  c->rtol_inner = 1e-3;
  c->max_outer = 8;
  c->warm_start = HCA_WS_PREV;
  c->preconditioner = HCA_PC_JACOBI;
  c->threads_per_block = 0;
  c->stream = nullptr;
  return HCA_OK;
}

int hca_create(const hca_config* cfg, const float* p_cell, const float* perf, const float* p_vessel,
               int32_t maps_on_device, hca_handle** out) {
  if (!cfg) return HCA_ERR_ARG;
  return create_impl(1, cfg, &p_cell, &perf, &p_vessel, maps_on_device, out);
}

int hca_create_batch(int32_t n, const hca_config* cfgs, const float* const* p_cell, const float* const* perf,
                     const float* const* p_vessel, int32_t maps_on_device, hca_handle** out) {
  return create_impl(n, cfgs, p_cell, perf, p_vessel, maps_on_device, out);
}

int hca_step(hca_handle* h, int32_t n_steps) {
  if (!h || n_steps < 0) return HCA_ERR_ARG;
  if (n_steps == 0) return HCA_OK;
  if (h->graphs_ok && !h->prof.on && run_graph(h, HCA_STAGE_ALL, n_steps) == HCA_OK) return check_convergence(h);
  for (int s = 0; s < n_steps; ++s) {
    int rc = run_stages(h, HCA_STAGE_ALL);
    if (rc) return rc;
  }
  return check_convergence(h);
}

int hca_stage(hca_handle* h, uint32_t mask) {
  if (!h || (mask & ~HCA_STAGE_ALL)) return HCA_ERR_ARG;
  if (!mask) return HCA_OK;
  if (h->graphs_ok && !h->prof.on && run_graph(h, mask, 1) == HCA_OK) return check_convergence(h);
  int rc = run_stages(h, mask);
  if (rc) return rc;
  return check_convergence(h);
}

int hca_read_fields(hca_handle* h, int32_t rep, uint32_t mask, void* dst, size_t dst_bytes, int32_t dst_on_device) {
  if (check_rep(h, rep) || !dst || (mask & ~0x3FFFu) || !mask) return HCA_ERR_ARG;
  const RepDesc& r = h->reps_h[rep];
  const size_t es = elem_size(h);
  const size_t per = (size_t)r.nx * r.ny * r.nz;
  size_t k = 0;
  for (uint32_t bit = 1; bit <= 0x2000u; bit <<= 1)
    if (mask & bit) {
      if (!field_ptr(h, bit)) return HCA_ERR_ARG;
      ++k;
    }
  if (dst_bytes < k * per * es) return HCA_ERR_ARG;
  (void)dst_on_device;
  size_t slot = 0;
  for (uint32_t bit = 1; bit <= 0x2000u; bit <<= 1) {
    if (!(mask & bit)) continue;
    int rc = copy_field(h, rep, field_ptr(h, bit), es, dst, true, slot * per);
    if (rc) return rc;
    ++slot;
  }
  HCA_TRY(cudaStreamSynchronize(h->ctx.stream));
  return HCA_OK;
}

int hca_write_fields(hca_handle* h, int32_t rep, uint32_t mask, const void* src, size_t src_bytes,
                     int32_t src_on_device) {
  if (check_rep(h, rep) || !src || (mask & ~0x1FFu) || !mask) return HCA_ERR_ARG;
  const RepDesc& r = h->reps_h[rep];
  const size_t es = elem_size(h);
  const size_t per = (size_t)r.nx * r.ny * r.nz;
  size_t k = 0;
  for (uint32_t bit = 1; bit <= 0x100u; bit <<= 1)
    if (mask & bit) {
      if (!field_ptr(h, bit)) return HCA_ERR_ARG;
      ++k;
    }
  if (src_bytes < k * per * es) return HCA_ERR_ARG;
  (void)src_on_device;
  size_t slot = 0;
  for (uint32_t bit = 1; bit <= 0x100u; bit <<= 1) {
    if (!(mask & bit)) continue;
    int rc = copy_field(h, rep, field_ptr(h, bit), es, const_cast<void*>(src), false, slot * per);
    if (rc) return rc;
    void* lo = nullptr;
    if (bit == HCA_FIELD_O2) lo = h->ctx.K_lo;
    if (bit == HCA_FIELD_VEGF) lo = h->ctx.G_lo[hca::VEGF_SLOT];
    for (int d = 0; d < h->n_drugs; ++d)
      if (bit == (HCA_FIELD_DRUG0 << d)) lo = h->ctx.G_lo[d];
    if (lo) {
      // a written field replaces any low-order correction word
      const RepDesc& rr = h->reps_h[rep];
      HCA_TRY(cudaMemsetAsync((char*)lo + (size_t)rr.off * es, 0, (size_t)rr.nxp * rr.ny * rr.nz * es, h->ctx.stream));
    }
    ++slot;
  }
  HCA_TRY(cudaStreamSynchronize(h->ctx.stream));
  return HCA_OK;
}

int hca_read_states(hca_handle* h, int32_t rep, uint8_t* dst, size_t dst_bytes, int32_t dst_on_device) {
  if (check_rep(h, rep) || !dst) return HCA_ERR_ARG;
  const RepDesc& r = h->reps_h[rep];
  if (dst_bytes < (size_t)r.nx * r.ny * r.nz) return HCA_ERR_ARG;
  (void)dst_on_device;
  HCA_TRY(cudaMemcpy2DAsync(dst, (size_t)r.nx, h->ctx.state + r.off, (size_t)r.nxp, (size_t)r.nx, (size_t)r.ny * r.nz,
                            cudaMemcpyDefault, h->ctx.stream));
  HCA_TRY(cudaStreamSynchronize(h->ctx.stream));
  return HCA_OK;
}

int hca_write_states(hca_handle* h, int32_t rep, const uint8_t* src, size_t src_bytes, int32_t src_on_device) {
  if (check_rep(h, rep) || !src) return HCA_ERR_ARG;
  const RepDesc& r = h->reps_h[rep];
  if (src_bytes < (size_t)r.nx * r.ny * r.nz) return HCA_ERR_ARG;
  (void)src_on_device;
  HCA_TRY(cudaMemcpy2DAsync(h->ctx.state + r.off, (size_t)r.nxp, src, (size_t)r.nx, (size_t)r.nx, (size_t)r.ny * r.nz,
                            cudaMemcpyDefault, h->ctx.stream));
  HCA_TRY(cudaStreamSynchronize(h->ctx.stream));
  return HCA_OK;
}

int hca_set_step(hca_handle* h, int64_t step) {
  if (!h || step < 0) return HCA_ERR_ARG;
  long long v = step;
  HCA_TRY(cudaMemcpyAsync(h->ctx.step, &v, sizeof(v), cudaMemcpyHostToDevice, h->ctx.stream));
  HCA_TRY(cudaStreamSynchronize(h->ctx.stream));
  h->step = step;
  return HCA_OK;
}

int hca_get_stats(hca_handle* h, int32_t rep, hca_stats* out) {
  if (check_rep(h, rep) || !out) return HCA_ERR_ARG;
  Ctx& c = h->ctx;
  for (int r = 0; r < h->n_reps; ++r)
    HCA_TRY(cudaMemsetAsync(&c.stats[r].counts[0], 0, sizeof(long long) * 6, c.stream));
  HCA_LAUNCH(h, HCA_KCLASS_OTHER, 1, hca::launch_histogram(c));
  hca::DevStats st;
  HCA_TRY(cudaMemcpyAsync(&st, &c.stats[rep], sizeof(st), cudaMemcpyDeviceToHost, c.stream));
  HCA_TRY(cudaStreamSynchronize(c.stream));
  std::memset(out, 0, sizeof(*out));
  out->step = h->step;
  out->picard_iterations = h->picard_iterations;
  out->o2_iterations = st.iters[0];
  out->o2_sweeps = st.sweeps[0];
  for (int d = 0; d < 3; ++d) {
    out->drug_iterations[d] = st.iters[1 + d];
    out->drug_rel_residual[d] = st.rel[1 + d];
  }
  out->o2_rel_residual = st.rel[0];
  out->vegf_iterations = st.iters[hca::WHICH_VEGF];
  out->vegf_rel_residual = st.rel[hca::WHICH_VEGF];
  out->vessel_births = st.vessel_births;
  out->vessel_deaths = st.vessel_deaths;
  out->not_converged = st.not_converged;
  out->committed = st.committed;
  out->kills = st.kills;
  out->divisions = st.divisions;
  out->blocked = st.blocked;
  for (int k = 0; k < 6; ++k) out->counts[k] = st.counts[k];
  if (h->learned && h->net) {
    hcanet::WsResult w;
    HCA_TRY(cudaMemcpy(&w, h->ws_res, sizeof(w), cudaMemcpyDeviceToHost));
    out->ws_used = w.used;
    out->ws_r0_prev = w.r0_prev;
    out->ws_r0_learned = w.r0_learned;
  }
  return HCA_OK;
}

int hca_get_launch_config(hca_handle* h, int32_t* threads_per_block, int32_t* pass_regs) {
  if (!h || !threads_per_block || !pass_regs) return HCA_ERR_ARG;
  *threads_per_block = h->ctx.threads;
  *pass_regs = h->fp64 ? 128 : h->ctx.pass_regs;
  return HCA_OK;
}

int hca_set_warm_start_net(hca_handle* h, hca_net* n) {
  if (!h) return HCA_ERR_ARG;
  if (n && (!h->learned || !hcanet::ws_fits(n, h->reps_h[0].nx, h->reps_h[0].ny, h->reps_h[0].nz))) return HCA_ERR_ARG;
  HCA_TRY(cudaStreamSynchronize(h->ctx.stream));
  for (auto& g : h->graphs) cudaGraphExecDestroy(g.exec);
  h->graphs.clear();
  h->net = n;
  return HCA_OK;
}

int hca_apply_preconditioner(hca_handle* h, int32_t rep, int32_t which, const void* r, void* z, int32_t on_device) {
  if (check_rep(h, rep) || !r || !z || which < 0 || which > h->n_drugs) return HCA_ERR_ARG;
  if (!h->mg) return HCA_ERR_STATE;
  (void)on_device;
  const size_t es = elem_size(h);
  Ctx& c = h->ctx;
  // the set-up of a solve of `which` writes the diagonal (its other outputs
  // are rewritten by the next solve)
  HCA_LAUNCH(h, HCA_KCLASS_SETUP, 1, hca::launch_setup(c, which, h->fp64, kNoCond));
  HCA_LAUNCH(h, HCA_KCLASS_MG, h->mgh.nlev, mg_setup(h, which));
  int rc = copy_field(h, rep, c.r, es, const_cast<void*>(r), false, 0);
  if (rc) return rc;
  c.skip_idle = 0;   // z is wanted whether or not the set-up found the solve converged
  HCA_LAUNCH(h, HCA_KCLASS_MG, hca::vcycle_launches(h->mgh, true), vcycle(h, which, true));
  c.skip_idle = 1;
  rc = copy_field(h, rep, c.z, es, z, true, 0);
  if (rc) return rc;
  HCA_TRY(cudaStreamSynchronize(c.stream));
  return HCA_OK;
}

int hca_apply_operator(hca_handle* h, int32_t rep, int32_t which, const void* u, void* out, int32_t on_device) {
  if (check_rep(h, rep) || !u || !out || which < 0 || which > h->n_drugs) return HCA_ERR_ARG;
  (void)on_device;
  const size_t es = elem_size(h);
  int rc = copy_field(h, rep, h->ctx.p, es, const_cast<void*>(u), false, 0);
  if (rc) return rc;
  HCA_LAUNCH(h, HCA_KCLASS_OTHER, 1, hca::launch_apply(h->ctx, which, rep, h->ctx.p, h->ctx.z, h->fp64));
  rc = copy_field(h, rep, h->ctx.z, es, out, true, 0);
  if (rc) return rc;
  // restore the invariant that padding holds 0 in p (u had none) and clear p
  HCA_TRY(cudaMemsetAsync(h->ctx.p, 0, (size_t)h->total * es, h->ctx.stream));
  HCA_TRY(cudaStreamSynchronize(h->ctx.stream));
  return HCA_OK;
}

int hca_philox_uniforms(uint64_t seed, uint64_t site_begin, int64_t n, uint32_t step, uint32_t purpose, float* dst,
                        int32_t dst_on_device) {
  if (!dst || n < 0) return HCA_ERR_ARG;
  if (n == 0) return HCA_OK;
  float* d = dst;
  if (!dst_on_device) {
    if (cudaMalloc(&d, (size_t)n * sizeof(float)) != cudaSuccess) {
      (void)cudaGetLastError();
      return HCA_ERR_OOM;
    }
  }
  hca::launch_philox_uniforms(seed, site_begin, n, step, purpose, d, 0);
  cudaError_t e = cudaGetLastError();
  if (e == cudaSuccess && !dst_on_device) e = cudaMemcpy(dst, d, (size_t)n * sizeof(float), cudaMemcpyDeviceToHost);
  if (e == cudaSuccess) e = cudaDeviceSynchronize();
  if (!dst_on_device) cudaFree(d);
  if (e != cudaSuccess) {
    (void)cudaGetLastError();
    return HCA_ERR_CUDA;
  }
  return HCA_OK;
}

int hca_sync(hca_handle* h) {
  if (!h) return HCA_ERR_ARG;
  HCA_TRY(cudaStreamSynchronize(h->ctx.stream));
  return HCA_OK;
}

int hca_get_shape(hca_handle* h, int32_t rep, int32_t* nx, int32_t* ny, int32_t* nz) {
  if (!h) return HCA_ERR_ARG;
  if (rep < 0) return h->n_reps;
  if (check_rep(h, rep)) return HCA_ERR_ARG;
  if (nx) *nx = h->reps_h[rep].nx;
  if (ny) *ny = h->reps_h[rep].ny;
  if (nz) *nz = h->reps_h[rep].nz;
  return HCA_OK;
}

int64_t hca_launch_count(hca_handle* h) {
  if (!h) return -1;
  unsigned long long n = 0;
  if (cudaMemcpyAsync(&n, h->ctx.n_kernels, sizeof(n), cudaMemcpyDeviceToHost, h->ctx.stream) != cudaSuccess ||
      cudaStreamSynchronize(h->ctx.stream) != cudaSuccess) {
    (void)cudaGetLastError();
    return -1;
  }
  return (int64_t)n;
}

int hca_profile_enable(hca_handle* h, int32_t enable) {
  if (!h) return HCA_ERR_ARG;
  Profiler& P = h->prof;
  int rc = prof_flush(h);
  if (rc) return rc;
  if (enable && P.pool.empty()) {
    P.pool.resize(2 * kPairs);
    for (auto& e : P.pool)
      if (cudaEventCreate(&e) != cudaSuccess) {
        (void)cudaGetLastError();
        return HCA_ERR_CUDA;
      }
  }
  for (int k = 0; k < HCA_NKCLASS; ++k) {
    P.launches[k] = 0;
    P.ms[k] = 0.0;
  }
  P.on = enable != 0;
  return HCA_OK;
}

int hca_get_profile(hca_handle* h, hca_profile* out) {
  if (!h || !out) return HCA_ERR_ARG;
  int rc = prof_flush(h);
  if (rc) return rc;
  for (int k = 0; k < HCA_NKCLASS; ++k) {
    out->launches[k] = h->prof.launches[k];
    out->ms[k] = h->prof.ms[k];
  }
  return HCA_OK;
}

int hca_save(hca_handle* h, const char* path) {
  if (!h || !path) return HCA_ERR_ARG;
  HCA_TRY(cudaStreamSynchronize(h->ctx.stream));
  FILE* f = std::fopen(path, "wb");
  if (!f) return HCA_ERR_IO;
  CkptHeader hd{};
  std::memcpy(hd.magic, kCkptMagic, 8);
  hd.version = 1;
  hd.config_size = (int32_t)sizeof(hca_config);
  hd.n_reps = h->n_reps;
  hd.precision = h->fp64 ? HCA_FP64 : HCA_FP32;
  hd.step = h->step;
  hd.picard_iterations = h->picard_iterations;
  bool ok = std::fwrite(&hd, sizeof(hd), 1, f) == 1;
  for (int i = 0; i < h->n_reps && ok; ++i) {
    hca_config cf = h->cfgs[i];
    cf.stream = nullptr;
    ok = std::fwrite(&cf, sizeof(cf), 1, f) == 1;
  }
  const size_t es = elem_size(h);
  int rc = HCA_OK;
  // the perfusion maps of every replicate first (creation needs them), then
  // per replicate the states and the fields
  for (int i = 0; i < h->n_reps && ok && !rc; ++i) {
    const RepDesc& r = h->reps_h[i];
    const size_t n = (size_t)r.nx * r.ny * r.nz;
    std::vector<char> buf(n * es);
    rc = copy_field(h, i, h->ctx.perf, es, buf.data(), true, 0);
    if (!rc && cudaStreamSynchronize(h->ctx.stream) != cudaSuccess) rc = HCA_ERR_CUDA;
    if (!rc) ok = std::fwrite(buf.data(), es, n, f) == n;
  }
  for (int i = 0; i < h->n_reps && ok && !rc; ++i) {
    const RepDesc& r = h->reps_h[i];
    const size_t n = (size_t)r.nx * r.ny * r.nz;
    std::vector<char> buf(n * es);
    rc = copy_states(h, i, (uint8_t*)buf.data(), true);
    if (!rc && cudaStreamSynchronize(h->ctx.stream) != cudaSuccess) rc = HCA_ERR_CUDA;
    if (!rc) ok = std::fwrite(buf.data(), 1, n, f) == n;
    for (void* fld : ckpt_fields(h)) {
      if (!fld || rc || !ok) continue;
      rc = copy_field(h, i, fld, es, buf.data(), true, 0);
      if (!rc && cudaStreamSynchronize(h->ctx.stream) != cudaSuccess) rc = HCA_ERR_CUDA;
      if (!rc) ok = std::fwrite(buf.data(), es, n, f) == n;
    }
  }
  if (std::fclose(f) != 0) ok = false;
  if (rc) return rc;
  return ok ? HCA_OK : HCA_ERR_IO;
}

int hca_load(const char* path, void* stream, hca_handle** out) {
  if (!path || !out) return HCA_ERR_ARG;
  *out = nullptr;
  FILE* f = std::fopen(path, "rb");
  if (!f) return HCA_ERR_IO;
  CkptHeader hd{};
  int rc = HCA_OK;
  std::vector<hca_config> cfgs;
  std::vector<std::vector<float>> perf;
  hca_handle* h = nullptr;
  if (std::fread(&hd, sizeof(hd), 1, f) != 1) rc = HCA_ERR_IO;
  else if (std::memcmp(hd.magic, kCkptMagic, 8) != 0 || hd.version != 1 ||
           hd.config_size != (int32_t)sizeof(hca_config) || hd.n_reps < 1 || hd.n_reps > (1 << 20))
    rc = HCA_ERR_ARG;
  if (!rc) {
    cfgs.resize(hd.n_reps);
    if (std::fread(cfgs.data(), sizeof(hca_config), hd.n_reps, f) != (size_t)hd.n_reps) rc = HCA_ERR_IO;
  }
  // validate before any allocation sized from the file
  for (int i = 0; i < hd.n_reps && !rc; ++i) {
    cfgs[i].stream = stream;
    rc = validate(cfgs[i]);
    if (!rc && cfgs[i].precision != hd.precision) rc = HCA_ERR_ARG;
  }
  std::vector<std::vector<char>> perf_raw;
  if (!rc) {
    // creation needs maps: zero densities and the saved perfusion (written
    // back in the handle's precision below); states and fields are then
    // overwritten, so only perfusion's bounds check matters
    const size_t es = hd.precision == HCA_FP64 ? 8 : 4;
    perf.resize(hd.n_reps);
    perf_raw.resize(hd.n_reps);
    for (int i = 0; i < hd.n_reps && !rc; ++i) {
      const size_t n = (size_t)cfgs[i].nx * cfgs[i].ny * cfgs[i].nz;
      perf_raw[i].resize(n * es);
      if (std::fread(perf_raw[i].data(), es, n, f) != n) {
        rc = HCA_ERR_IO;
        break;
      }
      perf[i].resize(n);
      for (size_t k = 0; k < n; ++k)
        perf[i][k] = es == 8 ? (float)((const double*)perf_raw[i].data())[k] : ((const float*)perf_raw[i].data())[k];
    }
    if (!rc) {
      std::vector<std::vector<float>> zeros(hd.n_reps);
      std::vector<const float*> pz(hd.n_reps), pp(hd.n_reps);
      for (int i = 0; i < hd.n_reps; ++i) {
        zeros[i].assign(perf[i].size(), 0.f);
        pz[i] = zeros[i].data();
        pp[i] = perf[i].data();
      }
      rc = create_impl(hd.n_reps, cfgs.data(), pz.data(), pp.data(), pz.data(), 0, &h, false);
    }
  }
  for (int i = 0; h && i < h->n_reps && !rc; ++i) {
    const RepDesc& r = h->reps_h[i];
    const size_t n = (size_t)r.nx * r.ny * r.nz, es = elem_size(h);
    std::vector<char> buf(n * es);
    // perfusion in the handle's precision exactly as saved (creation rounded it through FP32)
    rc = copy_field(h, i, h->ctx.perf, es, perf_raw[i].data(), false, 0);
    if (!rc && std::fread(buf.data(), 1, n, f) != n) rc = HCA_ERR_IO;
    if (!rc) rc = copy_states(h, i, (uint8_t*)buf.data(), false);
    if (!rc && cudaStreamSynchronize(h->ctx.stream) != cudaSuccess) rc = HCA_ERR_CUDA;
    for (void* fld : ckpt_fields(h)) {
      if (!fld || rc) continue;
      if (std::fread(buf.data(), es, n, f) != n) rc = HCA_ERR_IO;
      if (!rc) rc = copy_field(h, i, fld, es, buf.data(), false, 0);
      if (!rc && cudaStreamSynchronize(h->ctx.stream) != cudaSuccess) rc = HCA_ERR_CUDA;
    }
  }
  std::fclose(f);
  if (!rc && h) {
    h->picard_iterations = hd.picard_iterations;
    rc = hca_set_step(h, hd.step);
  }
  if (rc) {
    if (h) hca_destroy(h);
    return rc;
  }
  *out = h;
  return HCA_OK;
}

void hca_destroy(hca_handle* h) {
  if (!h) return;
  cudaStreamSynchronize(h->ctx.stream);
  free_all(h);
  delete h;
}

const char* hca_status_string(int32_t s) {
  switch (s) {
    case HCA_OK: return "ok";
    case HCA_ERR_ARG: return "invalid argument";
    case HCA_ERR_CUDA: return "CUDA runtime error";
    case HCA_ERR_OOM: return "device memory exhausted";
    case HCA_ERR_NONFINITE: return "non-finite value in an input or a solver norm";
    case HCA_ERR_NOCONV: return "a CG solve reached maxit";
    case HCA_ERR_TIMEOUT: return "a bounded device wait gave up";
    case HCA_ERR_UNIMPLEMENTED: return "not implemented";
    case HCA_ERR_STATE: return "call not valid in the current state";
    case HCA_ERR_IO: return "checkpoint file input/output failed";
    default: return "unknown status";
  }
}

}  // extern "C"
