// Internal device/host definitions shared by the library's translation units.
//
// Data layout (HBM): every field of every replicate lives in one array per
// field.  Replicate r's site (x, y, z) is element off_r + x + nxp_r*(y + ny_r*z)
// where nxp_r = nx_r rounded up to a multiple of 4, so each row starts on a
// 16-byte (float) / 32-byte (double) boundary and a thread moves 4 sites with
// one vector access.  Sites x >= nx are padding: they hold 0 in every field
// and are masked out of every update and reduction.
//
// Work decomposition: the (y, z) rows of a replicate are cut into fixed
// chunks of CHUNK_ROWS consecutive rows (row j = y + ny*z).  One thread block
// processes one chunk.  Inner products are summed per row in a fixed lane
// order, per chunk in a fixed tree, and per replicate over its chunks in a
// fixed order, so every reduction result is a function of the lattice alone:
// it does not depend on the block size chosen by the autotuner or on the
// other replicates of a batch.
#pragma once

#include <utility>

#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/hca.h"

namespace hca {

constexpr int VEC = 4;          // sites per thread access
constexpr int CHUNK_ROWS = 32;  // rows per reduction chunk
constexpr int NDOT = 3;         // inner products carried per pass
constexpr int MAX_DRUGS = 3;
// linear fields solved besides oxygen: the drugs in slots 0..2 and the VEGF
// field (Eq. vac_v, A = 0) in slot 3, solved as operator `which` = 1 + slot
constexpr int MAX_FIELDS = 4;
constexpr int VEGF_SLOT = 3;
constexpr int WHICH_VEGF = 1 + VEGF_SLOT;
constexpr int SUPER_CHUNKS = 64;  // chunks per second-level reduction group

// ---------------------------------------------------------------- params --
// Per-replicate constants, read-only on the device.
struct RepDesc {
  int nx, ny, nz, nxp;
  long long off;          // element offset of site (0,0,0)
  int gpr;                // 4-site groups per row = nxp / 4
  int lpr;                // lanes per row (power of two, <= 32)
  int chunk_begin;        // first chunk of this replicate in the chunk table
  int n_chunks;
  int chunk_rows;         // rows per chunk (a power of two <= CHUNK_ROWS, from the lattice's shape)
  int super_begin;        // first group of SUPER_CHUNKS chunks of this replicate
  int n_supers;
  unsigned long long seed;
  int n_drugs;
  int maxit;
  double rtol_o2, rtol_drug, rtol_inner;
  int max_outer;          // defect-correction sweeps per solve (FP32 storage); 0 = plain FP32 CG
  // oxygen (Eq. oxygen)
  double c_o2;            // D_K / dx^2
  double phi_K, K1, K0, r_K;
  // drugs (Eq. chemo), implicit Euler
  double c_drug[MAX_FIELDS];   // D_G / dx^2 (slot 3: D_V / dx^2)
  float cpl32[1 + MAX_FIELDS]; // the couplings of operators 0 (c_o2), 1.. (c_drug) rounded to FP32
  double base_drug[MAX_FIELDS];// mass term + psi_G (slot 3: + psi_V)
  double inv_dt;
  // time discretisation per operator (0 oxygen, 1 + d drug d): the reaction
  // carries the mass term (o2_mass; inside base_drug), the right-hand side is
  // b = bx x0 - (bax ? A x0 : 0) + source, with the oxygen source doubled and
  // the drug source taken at both ends of the sub-step when bax (Crank-Nicolson)
  double o2_mass;
  double bx[1 + MAX_FIELDS];
  int bax[1 + MAX_FIELDS];
  int nsub[1 + MAX_FIELDS];   // sub-steps per CA step
  double kappa[MAX_FIELDS];   // slot 3: 0 (no vessel exchange)
  double uptake[MAX_FIELDS];  // slot 3: 0
  double a_vegf;              // VEGF release per unit Vc at cell sites
  // plasma pharmacokinetics per drug: 0 exponential, 1 Michaelis-Menten,
  // 2 three compartments (unit-bolus response sum_i pk_coef e^{pk_lam t})
  int pk_model[MAX_DRUGS];
  double mm_vmax, mm_km;
  double pk_lam[MAX_DRUGS][3], pk_coef[MAX_DRUGS][3];
  // vascular automaton
  int vessel_interval;        // steps between updates, 0 = off
  double V_low, V_high, p_death, beta_birth, V_sprout;
  double dose_peak[MAX_DRUGS];
  double plasma_decay[MAX_DRUGS];
  double dose_interval_min;  // minutes between boluses
  int kill_b[MAX_DRUGS];
  // cell ODEs
  double dt, T_cycle, K_phi, k1, k1p, K_p53, k2, k2p, k2pp, J5, K_V;
  int ode_substeps;
  // CA colour lists: capacity offsets per colour (in the replicate's segment)
  long long list_off[27];
  int list_cap[27];
};

// Per-replicate CG scalars, rewritten by each solve.
struct RepSolve {
  double rho;      // r.z
  double alpha, beta;
  double bnorm2, rnorm2, rtol;
  double rel_true;
  int iters;
  int active;
  int zero_b;
  int maxit;
  int outer;       // defect-correction sweeps done in this solve
  int dc_apply;    // 1: the last inner solve's correction is to be added
  double bb_outer; // |b|^2 of the defect-corrected system (from its first sweep)
  double scale;    // power of two applied to the inner problem (1 for plain solves)
};

// Per-replicate statistics written by kernels; copied out by hca_get_stats.
struct DevStats {
  long long committed, kills, divisions, blocked;
  long long counts[6];
  int iters[1 + MAX_FIELDS];
  int sweeps[1 + MAX_FIELDS];
  int not_converged;
  double rel[1 + MAX_FIELDS];
  int nonfinite;
  int pad;
  long long vessel_births, vessel_deaths;
};

// Shared state for the last-block finalisation of a pass.
struct PassSync {
  unsigned int ticket;
  int active_count;     // replicates still iterating after the last pass B
  int error;            // nonzero: a norm became NaN/Inf
  int parity;           // which direction buffer holds the current p (0: p, 1: p_alt)
  int guard;            // CG passes since the solve's set-up (loop insurance)
  int guard_outer;      // defect-correction sweeps since the solve's first sweep
  int guard_limit;      // passes after which a graph loop is forced to stop
  int guard_outer_limit;
  // grid barrier of the cooperative coarse-level V-cycle kernel: arrivals
  // since the last release, and the release generation the waiters poll
  unsigned int bar_count;
  unsigned int bar_gen;
};

// PassSync::error codes (read back by the host): 1 a norm became NaN/Inf,
// 2 a defect-correction solve stopped at its sweep limit, 3 a bounded device
// wait gave up
constexpr int SYNC_ERR_NONFINITE = 1;
constexpr int SYNC_ERR_NOCONV = 2;
constexpr int SYNC_ERR_TIMEOUT = 3;

// A conditional-node handle of the step graph that a kernel's last block sets
// (valid = 0 outside graph execution).
struct CondArg {
  unsigned long long h;
  int valid;
};

// ------------------------------------------------------------- vectors ---
template <typename T> struct V4 { T a[4]; };

__device__ __forceinline__ V4<float> ld4(const float* p) {
  float4 v = *reinterpret_cast<const float4*>(p);
  return V4<float>{{v.x, v.y, v.z, v.w}};
}
__device__ __forceinline__ V4<double> ld4(const double* p) {
  double2 u = reinterpret_cast<const double2*>(p)[0];
  double2 v = reinterpret_cast<const double2*>(p)[1];
  return V4<double>{{u.x, u.y, v.x, v.y}};
}
__device__ __forceinline__ void st4(float* p, const V4<float>& v) {
  *reinterpret_cast<float4*>(p) = make_float4(v.a[0], v.a[1], v.a[2], v.a[3]);
}
__device__ __forceinline__ void st4(double* p, const V4<double>& v) {
  reinterpret_cast<double2*>(p)[0] = make_double2(v.a[0], v.a[1]);
  reinterpret_cast<double2*>(p)[1] = make_double2(v.a[2], v.a[3]);
}
template <typename T> __device__ __forceinline__ V4<T> zero4() { return V4<T>{{T(0), T(0), T(0), T(0)}}; }

__device__ __forceinline__ uchar4 ld_state4(const uint8_t* p) {
  return *reinterpret_cast<const uchar4*>(p);
}
__device__ __forceinline__ uint8_t st_at(const uchar4& s, int k) {
  return k == 0 ? s.x : (k == 1 ? s.y : (k == 2 ? s.z : s.w));
}

// The CG direction and operator arithmetic of pass A, with its roundings
// fixed (no contraction left to the compiler) so that every kernel forming
// them gets the same bits: p = zs z + beta p_old, q = d p - c nb, and the
// accumulation s += p q.
__device__ __forceinline__ float cg_dir(float zs, float z, float beta, float p) {
  return __fmaf_rn(beta, p, __fmul_rn(zs, z));
}
__device__ __forceinline__ float cg_apply(float d, float p, float c, float nb) {
  return __fmaf_rn(d, p, -__fmul_rn(c, nb));
}
__device__ __forceinline__ float cg_madd(float a, float b, float s) { return __fmaf_rn(a, b, s); }
__device__ __forceinline__ double cg_dir(double zs, double z, double beta, double p) { return zs * z + beta * p; }
__device__ __forceinline__ double cg_apply(double d, double p, double c, double nb) { return d * p - c * nb; }
__device__ __forceinline__ double cg_madd(double a, double b, double s) { return s + a * b; }

// state classes
__device__ __forceinline__ bool is_consumer(uint8_t s) {
  return s == HCA_PROLIF || s == HCA_QUIESC || s == HCA_STROMA;
}
__device__ __forceinline__ bool is_cancer(uint8_t s) { return s == HCA_PROLIF || s == HCA_QUIESC; }
__device__ __forceinline__ bool is_vessel(uint8_t s) { return s == HCA_VESSEL; }
__device__ __forceinline__ bool is_free(uint8_t s) { return s == HCA_EMPTY || s == HCA_DEAD; }

// ------------------------------------------------------------- philox ---
// Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11): ten rounds of two
// 32x32->64 multiplies with Weyl key increments between rounds.
struct Philox4 { uint32_t w[4]; };

__host__ __device__ __forceinline__ Philox4 philox4x32_10(uint32_t c0, uint32_t c1, uint32_t c2,
                                                          uint32_t c3, uint32_t k0, uint32_t k1) {
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    const unsigned long long p0 = 0xD2511F53ull * (unsigned long long)c0;
    const unsigned long long p1 = 0xCD9E8D57ull * (unsigned long long)c2;
    const uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
    const uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
    const uint32_t n0 = hi1 ^ c1 ^ k0, n2 = hi0 ^ c3 ^ k1;
    c0 = n0; c1 = lo1; c2 = n2; c3 = lo0;
    k0 += 0x9E3779B9u;
    k1 += 0xBB67AE85u;
  }
  return Philox4{{c0, c1, c2, c3}};
}

// 24-bit uniform in [0, 1), exact in float: (w0 >> 8) * 2^-24.
__host__ __device__ __forceinline__ float site_uniform(unsigned long long seed, unsigned long long site,
                                                       uint32_t step, uint32_t purpose) {
  Philox4 o = philox4x32_10((uint32_t)site, (uint32_t)(site >> 32), step, purpose, (uint32_t)seed,
                            (uint32_t)(seed >> 32));
  return (float)(o.w[0] >> 8) * 5.9604644775390625e-08f;
}

enum Purpose : uint32_t { PURPOSE_VESSEL = 0, PURPOSE_CANCER = 1, PURPOSE_PHI = 2, PURPOSE_KILL = 3, PURPOSE_VASCULAR = 4 };

// ------------------------------------------------------ row iteration ---
// Geometry of one row (y, z) of replicate rd.
struct RowGeo {
  long long base;   // element index of (0, y, z)
  long long sy, sz; // strides to the y and z neighbour rows
  int y, z;
  bool ym, yp, zm, zp;  // neighbour rows inside the box
};

__device__ __forceinline__ RowGeo row_geo(const RepDesc& rd, int j) {
  RowGeo g;
  g.y = j % rd.ny;
  g.z = j / rd.ny;
  g.sy = rd.nxp;
  g.sz = (long long)rd.nxp * rd.ny;
  g.base = rd.off + (long long)j * rd.nxp;
  g.ym = g.y > 0;
  g.yp = g.y < rd.ny - 1;
  g.zm = g.z > 0;
  g.zp = g.z < rd.nz - 1;
  return g;
}

__device__ __forceinline__ int neighbour_count(const RepDesc& rd, const RowGeo& g, int x) {
  return (x > 0) + (x < rd.nx - 1) + g.ym + g.yp + g.zm + g.zp;
}

// Sum of a lane-partial double over the `lpr` lanes of a row segment (fixed
// xor tree; every lane of the warp must call it).
__device__ __forceinline__ double row_reduce(double v, int lpr) {
  for (int o = lpr >> 1; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o, 32);
  return v;
}

__device__ __forceinline__ void set_cond(const CondArg& c, bool v) {
  if (c.valid) cudaGraphSetConditional((cudaGraphConditionalHandle)c.h, v ? 1u : 0u);
}

}  // namespace hca

namespace hca {

// Device pointers and launch parameters of one handle, passed by value to
// every kernel.  Field pointers are typed per precision by the kernels.
// One coarse level of the multigrid hierarchy (dense, x fastest).
struct MGLevel {
  int nx, ny, nz, pad;
  long long n;
  void *x, *t, *rhs, *d, *w;   // iterate, second iterate, right-hand side, diagonal, 1 / diagonal
  double cscale;            // coupling of this level / coupling of the lattice (2^level)
  float cscale32;           // the same in FP32 (exact)
};

// multigrid constants (the FP64 reference uses the same).  Above the
// coarsest level a V-cycle smooths with two Jacobi sweeps before the coarse
// correction, of weights MG_W1 then MG_W2, and two after it, MG_W2 then
// MG_W1: the reciprocals of the roots 1.25 +- 0.75 cos(pi/4) of the
// degree-2 Chebyshev polynomial on [0.5, 2] (a Chebyshev polynomial
// smoother for the spectrum of D^-1 A).  The coarsest level takes
// MG_NU_COARSE sweeps of weight MG_OMEGA_COARSE.
constexpr double MG_W1 = 1.0 / (1.25 + 0.75 * 0.70710678118654752440);
constexpr double MG_W2 = 1.0 / (1.25 - 0.75 * 0.70710678118654752440);
constexpr double MG_OMEGA_COARSE = 0.8;
constexpr int MG_NU_COARSE = 16;
constexpr long long MG_MIN_SITES = 512;     // coarsening stops at or below this size
constexpr long long MG_SMALL_SITES = 4096;  // levels this small run inside one block

constexpr int MG_MAXLEV = 16;
constexpr int kVcycleParts = 6;   // launch groups of a V-cycle (see launch_vcycle)

// Host summary of the hierarchies of a handle's replicates (launch geometry).
struct MGHost {
  int nlev = 0;                  // most levels of any replicate
  // the coarse levels of a V-cycle in one cooperative launch (grid barriers
  // between levels): blocks of that launch (0 = one launch per level) and
  // the shared memory of its single-block levels (0 = they stay in global memory)
  int coop_blocks = 0;
  int small_smem = 0;
  int coop_cfg = 0;              // launch shape of the cooperative kernel (threads, register budget)
  // first level of the cooperative launch: 1 in host loops; in captured
  // graphs the first level small enough for it (coop_lo), the levels above
  // keep their per-level kernels
  int coop_from = 1;
  int coop_lo = 1;
  bool small_smem_ok = false;    // the standalone single-block kernel runs in shared memory
  int small = 0;                 // 1 + deepest grid-kernel level of any replicate
  long long ntot[MG_MAXLEV] = {};  // sites of level l summed over the replicates
  long long nrowitems = 0;         // (level-1 row, lattice 4-site group) items over the replicates
  int launches = 0;              // kernels per V-cycle
  int ni = 0;                    // groups per lane in a row of the lattice (1, 2, 4; 0 = other)
  unsigned rows_ok = 0;          // bit l: every replicate's level-l rows are whole 4-site groups
  long long post_items[MG_MAXLEV] = {};   // row-kernel items per level over the replicates
  long long restr_items[MG_MAXLEV] = {};
  // the lattice's pre-sweeps in plane-marching form (one FP32 lattice; 0 =
  // row form): slabs along z, planes per slab, tiles along x and y
  int zm_slabs = 0;
  int zm_zs = 0;
  int zm_tx = 0, zm_ty = 0;
  int zm_mode = 0;               // 2: TMA-staged planes (default), 1: planes prefetched into registers
  // grid levels' pre-sweeps and last post-sweep in plane-marching form
  // (0 slabs: row form): slabs, planes per slab, tiles along x and y
  int zl_slabs[MG_MAXLEV] = {};
  int zl_zs[MG_MAXLEV] = {};
  int zl_tx[MG_MAXLEV] = {}, zl_ty[MG_MAXLEV] = {};
  // TMA tensor maps of r and 1/d over the lattice (x extent nx: the copy
  // engine fills sites outside the lattice with zeros)
  CUtensorMap zm_map_r, zm_map_w;
};

struct Ctx {
  const RepDesc* reps;
  int n_reps;
  const int2* chunks;  // (replicate, first row) per chunk
  int n_chunks;
  int threads;
  int sm_count;
  cudaStream_t stream;
  uint8_t* state;
  void* K;       // oxygen
  void* K_lo;    // FP32 scheme: low-order words of the solved fields
  void* G[MAX_FIELDS];      // drugs, then the VEGF field in slot 3
  void* G_lo[MAX_FIELDS];
  unsigned long long* vsum;  // vascular automaton: [rep][2] fixed-point sums
  void* dx;      // FP32 scheme: correction of the inner solve
  void* aux;     // scratch field (previous iterate of the initial oxygen fixed point)
  int sub;          // sub-step of the current solve within the CA step (plasma times)
  const void* lag;  // oxygen linearisation point (K_prev) when the solve starts elsewhere; null: the start field
  // multigrid preconditioner (single replicate): residual r (the Jacobi form
  // carries z = r / d instead), level-0 scratch, coarse level table
  int pass_regs;    // register cap of the FP32 CG passes (64, 80, 96, 128)
  int pass_ni;      // groups per lane in a row shared by all replicates (1, 2, 4; 0 = differs)
  int mg;           // 0: Jacobi (z = r / d), 1: V-cycle (z = M r)
  int persist;         // 1: the CG passes and the lattice post-sweep run in persistent row form (one FP32 lattice)
  int pdl;             // 1: the CG and V-cycle kernels launch with programmatic dependent launch
  int skip_idle;       // 1 (solves): a V-cycle's kernels return at once when the set-up, residual
                       // sweep or pass B before it left no replicate iterating (nothing reads its z)
  void* r;
  void* mg_t0;
  void* mg_w;         // 1 / d on the lattice (0 where d = 0)
  const void* mg_lv;  // device MGLevel[n_reps][MG_MAXLEV] (level 0 unused)
  const long long* mg_start;  // [MG_MAXLEV][n_reps + 1] prefix sums of each level's sites over the replicates
  const int2* mg_rep;         // per replicate: (levels, first single-block level)
  const long long* mg_rowstart;  // [n_reps + 1] prefix of level-1 rows x lattice groups per row
  // row-vector coarse kernels: [MG_MAXLEV][n_reps + 1] prefix sums of the items
  // (4-site groups) of the post-sweep on level l and of the restriction l -> l + 1
  const long long* mg_post_items;
  const long long* mg_restr_items;
  void* reac;    // FP32 scheme: reaction part a of the diagonal d = c n + a
  void* phi;
  void* P;
  void* Vc;
  void* perf;
  void* z;       // preconditioned residual z = r / d
  void* p;       // search direction (two buffers: pass A reads one, writes the other)
  void* p_alt;
  void* q;           // A p of the current direction (written by pass A, read by pass B)
  void* d;       // operator diagonal
  void* b;       // right-hand side (drugs) / defect (oxygen correction solve)
  double* partial;
  PassSync* sync;
  RepSolve* solve;
  DevStats* stats;
  long long* step;        // device step counter n
  uint32_t* lists;
  int* list_count;        // [rep][27]
  // synchronous CA update (ca_mode 1): per list slot the decision (target
  // element, -1 blocked, -2 killed); per field element the highest claiming
  // phi (its bits) and the lowest claiming site among those
  long long* ca_dec;
  unsigned long long* claim_phi;
  unsigned int* claim_idx;
  unsigned long long* n_kernels;  // kernels that ran (counted by block 0 of each)
  int* frozen;            // [rep] 1: solves leave this replicate's field untouched
  // fixed-order reductions: row sums -> chunk sums -> group sums -> replicate
  double* rowp;           // [chunk][CHUNK_ROWS][NDOT]
  int* chunk_cnt;         // [chunk] warps done
  double* superp;         // [group][NDOT]
  int* super_cnt;         // [group] chunks done
  int n_supers;
};

// Float-float accumulator: an unevaluated sum hi + lo of two FP32 words,
// updated with Knuth's error-free TwoSum, so sums keep ~48 significant bits
// while running on the FP32 pipes (GB300's FP64 rate is a small fraction of
// its FP32 rate; the CG inner products would otherwise be FP64-ALU bound).
struct FF {
  float hi, lo;
};

__device__ __forceinline__ FF ff_add(FF a, float b) {
  const float s = __fadd_rn(a.hi, b);
  const float bb = __fsub_rn(s, a.hi);
  const float err = __fadd_rn(__fsub_rn(a.hi, __fsub_rn(s, bb)), __fsub_rn(b, bb));
  return FF{s, __fadd_rn(a.lo, err)};
}

__device__ __forceinline__ FF ff_add(FF a, FF b) {
  FF r = ff_add(a, b.hi);
  r.lo = __fadd_rn(r.lo, b.lo);
  return r;
}

// Exact product a*b = hi + lo (one FMA recovers the rounding error).
__device__ __forceinline__ FF ff_two_prod(float a, float b) {
  const float p = __fmul_rn(a, b);
  return FF{p, __fmaf_rn(a, b, -p)};
}

// (x.hi + x.lo) * b to ~48 bits
__device__ __forceinline__ FF ff_mul(FF x, float b) {
  FF p = ff_two_prod(x.hi, b);
  p.lo = __fmaf_rn(x.lo, b, p.lo);
  return p;
}

// (x.hi + x.lo) * (y.hi + y.lo) to ~48 bits
__device__ __forceinline__ FF ff_mul(FF x, FF y) {
  FF p = ff_two_prod(x.hi, y.hi);
  p.lo = __fmaf_rn(x.hi, y.lo, __fmaf_rn(x.lo, y.hi, p.lo));
  return p;
}

__device__ __forceinline__ FF ff_neg(FF x) { return FF{-x.hi, -x.lo}; }

// Row sum of float-float lane partials over the row's lane segment (fixed
// xor tree).
__device__ __forceinline__ FF row_reduce_ff(FF v, int lpr) {
  for (int o = lpr >> 1; o > 0; o >>= 1) {
    FF w;
    w.hi = __shfl_xor_sync(0xffffffffu, v.hi, o, 32);
    w.lo = __shfl_xor_sync(0xffffffffu, v.lo, o, 32);
    v = ff_add(v, w);
  }
  return v;
}

// The row slot keeps the float-float pair itself (two FP32 words in the
// slot's 8 bytes); the chunk reduction converts it to FP64 as hi + lo, one
// row per lane, instead of every lane of every row (FP64 runs at a small
// fraction of the FP32 rate on this GPU).  The same FP64 values either way.
__device__ __forceinline__ void store_row_ff(const Ctx& c, int chunk, int rl, bool row_ok, int sl, int lpr,
                                             const FF* acc, int ndot) {
  for (int k = 0; k < ndot; ++k) {
    const FF v = row_reduce_ff(acc[k], lpr);
    if (row_ok && sl == 0)
      *reinterpret_cast<float2*>(&c.rowp[((long long)chunk * CHUNK_ROWS + rl) * NDOT + k]) = make_float2(v.hi, v.lo);
  }
}

// A row slot's value: an FP64 sum, or (FFROWS) a float-float pair.
template <bool FFROWS>
__device__ __forceinline__ double row_slot(const Ctx& c, long long i) {
  if (FFROWS) {
    const float2 f = __ldcg(reinterpret_cast<const float2*>(&c.rowp[i]));
    return (double)f.x + (double)f.y;
  }
  return __ldcg(&c.rowp[i]);
}

// Row sum of a lane-partial over the row's lane segment, written to the
// row slot of the chunk (by the segment's first lane).
__device__ __forceinline__ void store_row(const Ctx& c, int chunk, int rl, bool row_ok, int sl, int lpr,
                                          const double* acc, int ndot) {
  for (int k = 0; k < ndot; ++k) {
    const double v = row_reduce(acc[k], lpr);
    if (row_ok && sl == 0) c.rowp[((long long)chunk * CHUNK_ROWS + rl) * NDOT + k] = v;
  }
}

// Every warp of a block calls this after its rows (no block barrier).  The
// last warp to finish a chunk sums the chunk's 32 row slots (fixed xor tree);
// the last chunk to finish a group of SUPER_CHUNKS chunks sums the group's
// chunk sums (fixed lane order); the last group to finish sums, per
// replicate, its groups (fixed lane order) and calls fin(rep, sums) from one
// lane; fin returns 1 if the replicate's solve stays active.  The number of
// active replicates goes to sync->active_count and to post(n_active).  The
// summation order depends on the lattice only, not on the block size, on the
// other replicates of a batch or on which warp performs it.
// The rest of warp_epilogue once a chunk's row slots are all written: the
// calling warp sums the chunk and continues to the group and replicate levels.
template <bool FFROWS, class Fin, class Post>
__device__ __forceinline__ void warp_chunk_done(const Ctx& c, int ndot, int chunk, Fin fin, Post post);

template <bool FFROWS = false, class Fin, class Post>
__device__ __forceinline__ void warp_epilogue(const Ctx& c, int ndot, int chunk, Fin fin, Post post) {
  const unsigned FULLM = 0xffffffffu;
  const int lane = threadIdx.x & 31;
  const int nw = blockDim.x >> 5;
  __syncwarp();
  int t = 0;
  if (lane == 0) {
    __threadfence();
    t = atomicAdd(&c.chunk_cnt[chunk], 1);
  }
  t = __shfl_sync(FULLM, t, 0);
  if (t != nw - 1) return;
  warp_chunk_done<FFROWS>(c, ndot, chunk, fin, post);
}

template <bool FFROWS, class Fin, class Post>
__device__ __forceinline__ void warp_chunk_done(const Ctx& c, int ndot, int chunk, Fin fin, Post post) {
  const unsigned FULLM = 0xffffffffu;
  const int lane = threadIdx.x & 31;
  int t = 0;
  __threadfence();
  const int2 ch = c.chunks[chunk];
  const RepDesc& rd = c.reps[ch.x];
  const int nrows = min(rd.chunk_rows, rd.ny * rd.nz - ch.y);
  for (int k = 0; k < ndot; ++k) {
    double v = lane < nrows ? row_slot<FFROWS>(c, ((long long)chunk * CHUNK_ROWS + lane) * NDOT + k) : 0.0;
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(FULLM, v, o);
    if (lane == 0) c.partial[(long long)chunk * NDOT + k] = v;
  }
  // group of chunks
  const int lc = chunk - rd.chunk_begin;
  const int gi = lc / SUPER_CHUNKS;
  const int sg = rd.super_begin + gi;
  const int g0 = rd.chunk_begin + gi * SUPER_CHUNKS;
  const int n_in = min(SUPER_CHUNKS, rd.n_chunks - gi * SUPER_CHUNKS);
  if (lane == 0) {
    c.chunk_cnt[chunk] = 0;
    __threadfence();
    t = atomicAdd(&c.super_cnt[sg], 1);
  }
  t = __shfl_sync(FULLM, t, 0);
  if (t != n_in - 1) return;
  __threadfence();
  for (int k = 0; k < ndot; ++k) {
    double v = 0.0;
    for (int i = lane; i < n_in; i += 32) v += __ldcg(&c.partial[(long long)(g0 + i) * NDOT + k]);
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(FULLM, v, o);
    if (lane == 0) c.superp[(long long)sg * NDOT + k] = v;
  }
  if (lane == 0) {
    c.super_cnt[sg] = 0;
    __threadfence();
    t = (int)atomicAdd(&c.sync->ticket, 1u);
  }
  t = __shfl_sync(FULLM, t, 0);
  if (t != c.n_supers - 1) return;
  __threadfence();
  int n_active = 0;
  for (int r = 0; r < c.n_reps; ++r) {
    const RepDesc& rr = c.reps[r];
    double sums[NDOT] = {0.0, 0.0, 0.0};
    for (int k = 0; k < ndot; ++k) {
      double v = 0.0;
      for (int i = lane; i < rr.n_supers; i += 32) v += __ldcg(&c.superp[(long long)(rr.super_begin + i) * NDOT + k]);
      for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(FULLM, v, o);
      sums[k] = v;
    }
    if (lane == 0) n_active += fin(r, sums);
  }
  if (lane == 0) {
    c.sync->active_count = n_active;
    post(n_active);
    __threadfence();
    c.sync->ticket = 0u;
  }
}

template <bool FFROWS = false, class Fin>
__device__ __forceinline__ void warp_epilogue(const Ctx& c, int ndot, int chunk, Fin fin) {
  warp_epilogue<FFROWS>(c, ndot, chunk, fin, [](int) {});
}

// Grid-wide barrier of a cooperative launch (every block is resident).
// PassSync::bar_count counts the arrivals of the launch: barrier k of the
// launch opens when it reaches (k + 1) * gridDim.x, and the last block to
// leave the kernel (grid_exit) sets it back to 0 for the next launch.  A
// wait gives up after kBarrierTimeoutNs of device time and records
// SYNC_ERR_TIMEOUT (the host returns HCA_ERR_TIMEOUT and the step sets the
// counter back to 0), so no kernel waits forever; later barriers and
// launches then return at once.
constexpr unsigned long long kBarrierTimeoutNs = 1000000000ull;   // 1 s

__device__ __forceinline__ unsigned long long device_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}
__device__ __forceinline__ unsigned ld_acquire_gpu(const unsigned* p) {
  unsigned v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

static __device__ __noinline__ bool grid_barrier(PassSync* sy, int k) {
  __shared__ int s_ok;
  __syncthreads();
  if (threadIdx.x == 0) {
    int ok = 1;
    if (*(volatile int*)&sy->error == SYNC_ERR_TIMEOUT) {
      ok = 0;
    } else {
      const unsigned target = (unsigned)(k + 1) * gridDim.x;
      __threadfence();   // this block's writes before its arrival
      atomicAdd(&sy->bar_count, 1u);
      if (ld_acquire_gpu(&sy->bar_count) < target) {
        const unsigned long long t0 = device_ns();
        while (ld_acquire_gpu(&sy->bar_count) < target) {
          if (device_ns() - t0 > kBarrierTimeoutNs) {
            atomicExch(&sy->error, SYNC_ERR_TIMEOUT);
            ok = 0;
            break;
          }
          __nanosleep(20);
        }
      }
      __threadfence();   // the other blocks' writes before this block reads on
    }
    s_ok = ok;
  }
  __syncthreads();
  return s_ok != 0;
}

// Leave a launch that passed nbar barriers: the last block out resets the
// arrival counter.
__device__ __forceinline__ void grid_exit(PassSync* sy, int nbar) {
  if (threadIdx.x == 0 && atomicAdd(&sy->bar_count, 1u) == (unsigned)(nbar + 1) * gridDim.x - 1u)
    atomicExch(&sy->bar_count, 0u);
}

// Count this kernel launch (call once, at kernel entry).
// At the entry of every kernel: wait until the kernel before it in the
// stream has completed and its memory is visible (programmatic dependent
// launch: a kernel launched with the programmatic-serialization attribute may
// start while its predecessor drains; without it the wait returns at once),
// then let the next kernel start launching, and count the launch.
#define HCA_COUNT_KERNEL(c)                                                  \
  do {                                                                       \
    asm volatile("griddepcontrol.wait;" ::: "memory");                       \
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");          \
    if (blockIdx.x == 0 && blockIdx.y == 0 && blockIdx.z == 0 && threadIdx.x == 0)           \
      atomicAdd((c).n_kernels, 1ull);                                        \
  } while (0)

// Entry of a V-cycle kernel: HCA_COUNT_KERNEL, then return at once when the
// set-up, residual sweep or pass B before the V-cycle left no replicate
// iterating (the solve or its inner loop ends; nothing reads this V-cycle's
// z).  Every block reads the same count: only those kernels write it, and
// none of them runs between the V-cycle's first and last kernel.
#define HCA_VC_ENTRY(c)                                                          \
  HCA_COUNT_KERNEL(c);                                                           \
  if ((c).skip_idle && *(volatile const int*)&(c).sync->active_count == 0) return

// Launch with programmatic dependent launch when enabled (pdl: the handle's
// setting; HCA_PDL=0 turns it off): the kernel's blocks may be scheduled
// while the previous kernel drains, and wait at HCA_COUNT_KERNEL.
template <typename... KArgs, typename... Args>
inline cudaError_t launch_k(bool pdl, void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem,
                            cudaStream_t s, Args&&... args) {
  if (!pdl) {
    kernel<<<grid, block, smem, s>>>(std::forward<Args>(args)...);
    return cudaSuccess;
  }
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, kernel, std::forward<Args>(args)...);
}

// Operator selector: 0 = oxygen, 1 + d = drug d.
__device__ __forceinline__ double op_coupling(const RepDesc& rd, int which) {
  return which == 0 ? rd.c_o2 : rd.c_drug[which - 1];
}
// The coupling in the field precision (FP32: the stored rounding, no
// conversion on the FP64 pipe).
template <typename T>
__device__ __forceinline__ T op_coupling_t(const RepDesc& rd, int which);
template <>
__device__ __forceinline__ float op_coupling_t<float>(const RepDesc& rd, int which) {
  return rd.cpl32[which];
}
template <>
__device__ __forceinline__ double op_coupling_t<double>(const RepDesc& rd, int which) {
  return op_coupling(rd, which);
}

// Plasma level G_{d,0}(t) after boluses at 0, I dt, 2 I dt, ... (closed form
// of the one-compartment model, doses superposed).
__device__ __forceinline__ double plasma_level(double t, double peak, double decay, double interval) {
  if (t < 0.0) return 0.0;
  double total = 0.0;
  for (long long n = 0; (double)n * interval <= t; ++n) {
    total += peak * exp(-decay * (t - (double)n * interval));
    if (interval <= 0.0) break;
  }
  return total;
}

// Plasma level seen by a drug sub-step: G_{d,0} at its end (t_k), plus at its
// start (t_{k-1}) under Crank-Nicolson; t_k = (step + (sub + 1) / m) dt.
// Principal branch of Lambert W for x = e^L > 0, given L: Newton on
// f(w) = w + ln w - L (w > 0), from w = L - ln L (L > 1) or w = e^L.  Written
// from the definition w e^w = x; a fixed number of steps (quadratic
// convergence) keeps the result independent of data-dependent stopping.
__device__ __forceinline__ double lambert_w_exp(double L) {
  double w = L > 1.0 ? L - log(L) : exp(L);
  for (int i = 0; i < 8; ++i) {
    const double f = w + log(w) - L;
    w = fmax(w - f * w / (w + 1.0), 0.5 * w);
  }
  return w;
}

// Michaelis-Menten plasma level a time s after the level G_s:
// G = k_m W((G_s / k_m) exp((G_s - v_max s) / k_m)).
__device__ __forceinline__ double mm_decay(double G_s, double s, double vmax, double km) {
  if (G_s <= 0.0) return 0.0;
  return km * lambert_w_exp(log(G_s / km) + (G_s - vmax * s) / km);
}

// Plasma level of drug dg at time t under its model (doses of dose_peak at
// 0, I dt, 2 I dt, ...).
__device__ __forceinline__ double plasma_at(const RepDesc& rd, int dg, double t) {
  const double peak = rd.dose_peak[dg], I = rd.dose_interval_min;
  if (rd.pk_model[dg] == 1) {
    if (t < 0.0) return 0.0;
    double G = 0.0, t_prev = 0.0;
    for (long long n = 0; (double)n * I <= t; ++n) {
      const double tn = (double)n * I;
      G = n > 0 ? mm_decay(G, tn - t_prev, rd.mm_vmax, rd.mm_km) + peak : peak;
      t_prev = tn;
      if (I <= 0.0) break;
    }
    return mm_decay(G, t - t_prev, rd.mm_vmax, rd.mm_km);
  }
  if (rd.pk_model[dg] == 2) {
    if (t < 0.0) return 0.0;
    double total = 0.0;
    for (long long n = 0; (double)n * I <= t; ++n) {
      const double s = t - (double)n * I;
      for (int i = 0; i < 3; ++i) total += peak * rd.pk_coef[dg][i] * exp(rd.pk_lam[dg][i] * s);
      if (I <= 0.0) break;
    }
    return total;
  }
  return plasma_level(t, peak, rd.plasma_decay[dg], I);
}

__device__ __forceinline__ double substep_plasma(const RepDesc& rd, int which, long long step, int sub) {
  if (which == WHICH_VEGF) return 0.0;
  const int dg = which - 1;
  const double m = (double)rd.nsub[which];
  const double t_new = ((double)step + (double)(sub + 1) / m) * rd.dt;
  double g = plasma_at(rd, dg, t_new);
  if (rd.bax[which]) g += plasma_at(rd, dg, ((double)step + (double)sub / m) * rd.dt);
  return g;
}

}  // namespace hca
