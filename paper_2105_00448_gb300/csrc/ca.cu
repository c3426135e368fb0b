// The stochastic cellular-automaton update (Sections 2.2.1 and 2.5).
//
// 1. compaction: DEAD sites become EMPTY; every cancer cell with phi >= 1 is
//    committed and appended to the list of its colour
//    c = (x mod 3) + 3 (y mod 3) + 9 (z mod 3);
// 2. one launch per colour c = 0..26, in order: each committed cell of the
//    colour is killed with probability 1 - prod_d (1 - x_d)^{b_d},
//    x_d = clamp(G_d / max G_{d,0}, 0, 1) (Eq. 1 with a = 1), decided by a
//    Philox draw keyed by (seed, site, step, KILL); otherwise it divides into
//    the free (EMPTY or DEAD) Moore neighbour with the highest K (first in
//    dz, dy, dx order on ties), both cells becoming PROLIF with
//    phi = P = Vc = 0; with no free neighbour it becomes QUIESC with phi = 0.
//
// (ca_mode 1 replaces step 2 by the synchronous update further below.)
//
// Same-colour sites are at least 3 apart along some axis, so their closed
// Moore neighbourhoods are disjoint: the cells of one launch never touch the
// same site and the outcome does not depend on thread order.  Later colours
// see the daughters and deaths of earlier ones.
//
// This translation unit is compiled with -fmad=false and the kill test uses
// explicit round-to-nearest intrinsics, so the decision is the same IEEE
// arithmetic as a plain CPU evaluation in the storage precision.
#include <cstdlib>

#include "hca_internal.cuh"

namespace hca {
namespace {

constexpr unsigned FULL = 0xffffffffu;

__device__ __forceinline__ float rn_div(float a, float b) { return __fdiv_rn(a, b); }
__device__ __forceinline__ double rn_div(double a, double b) { return __ddiv_rn(a, b); }
__device__ __forceinline__ float rn_mul(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ double rn_mul(double a, double b) { return __dmul_rn(a, b); }
__device__ __forceinline__ float rn_sub(float a, float b) { return __fsub_rn(a, b); }
__device__ __forceinline__ double rn_sub(double a, double b) { return __dsub_rn(a, b); }

// The drug kill test of a committed cell (Eq. 1 with a = 1), in round-to-
// nearest arithmetic of the storage precision.
template <typename T>
__device__ __forceinline__ bool killed(const Ctx& c, const RepDesc& rd, long long e, uint32_t site, uint32_t step) {
  const T u = (T)site_uniform(rd.seed, site, step, PURPOSE_KILL);
  T surv = T(1);
  for (int d = 0; d < rd.n_drugs; ++d) {
    T xd = rn_div(((const T*)c.G[d])[e], (T)rd.dose_peak[d]);
    if (xd > T(1)) xd = T(1);
    if (xd < T(0)) xd = T(0);
    const T f = rn_sub(T(1), xd);
    for (int q = 0; q < rd.kill_b[d]; ++q) surv = rn_mul(surv, f);
  }
  const T p_kill = rn_sub(T(1), surv);
  return u < p_kill;
}

// The free Moore neighbour of (x, y, z) with the highest K (first in dz, dy,
// dx order on ties), as a field element, or -1.  Every state and K of the
// in-box neighbourhood is loaded first (one memory round trip instead of one
// per neighbour: no other cell of the same colour touches this
// neighbourhood), then the neighbours are scanned in that order.
template <typename T>
__device__ __forceinline__ long long best_free(const Ctx& c, const RepDesc& rd, int x, int y, int z) {
  const T* K = (const T*)c.K;
  const long long sy = rd.nxp, sz = (long long)rd.nxp * rd.ny;
  uint8_t st[27];
  T kv[27];
#pragma unroll
  for (int t = 0; t < 27; ++t) {
    const int dz = t / 9 - 1, dy = (t / 3) % 3 - 1, dx = t % 3 - 1;
    const int xx = x + dx, yy = y + dy, zz = z + dz;
    const bool in = t != 13 && xx >= 0 && xx < rd.nx && yy >= 0 && yy < rd.ny && zz >= 0 && zz < rd.nz;
    const long long nbi = rd.off + xx + sy * yy + sz * zz;
    st[t] = in ? c.state[nbi] : (uint8_t)HCA_VESSEL;   // not free
    kv[t] = in ? K[nbi] : T(0);
  }
  long long best = -1;
  T best_K = T(0);
#pragma unroll
  for (int t = 0; t < 27; ++t) {
    if (!is_free(st[t])) continue;
    if (best < 0 || kv[t] > best_K) {
      const int dz = t / 9 - 1, dy = (t / 3) % 3 - 1, dx = t % 3 - 1;
      best = rd.off + (x + dx) + sy * (y + dy) + sz * (z + dz);
      best_K = kv[t];
    }
  }
  return best;
}

template <typename T>
__global__ void __launch_bounds__(512) k_ca_compact(Ctx c) {
  HCA_COUNT_KERNEL(c);
  __shared__ unsigned int s_committed;
  if (threadIdx.x == 0) s_committed = 0;
  __syncthreads();
  const int2 ch = c.chunks[blockIdx.x];
  const int rep = ch.x;
  const RepDesc& rd = c.reps[rep];
  const int nrows = min(rd.chunk_rows, rd.ny * rd.nz - ch.y);
  const long long base0 = rd.off + (long long)ch.y * rd.nxp;
  const int ngroups = nrows * rd.gpr;
  const int lane = threadIdx.x & 31;
  int* cnt = c.list_count + rep * 27;
  unsigned int my_committed = 0;
  for (int gb = 0; gb < ngroups; gb += blockDim.x) {
    const int gi = gb + threadIdx.x;
    const bool ok = gi < ngroups;
    int rl = 0, g = 0;
    if (ok) {
      rl = gi / rd.gpr;
      g = gi % rd.gpr;
    }
    const int j = ch.y + rl;
    const int y = j % rd.ny, z = j / rd.ny;
    const long long e = base0 + (long long)rl * rd.nxp + 4LL * g;
    uchar4 st = ok ? ld_state4(c.state + e) : make_uchar4(0, 0, 0, 0);
    bool changed = false;
    bool any_cancer = false;
    uint8_t sv[4] = {st.x, st.y, st.z, st.w};
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      if (sv[k] == HCA_DEAD) {
        sv[k] = HCA_EMPTY;
        changed = true;
      }
      any_cancer |= is_cancer(sv[k]);
    }
    V4<T> phi = zero4<T>();
    if (ok && any_cancer) phi = ld4((const T*)c.phi + e);
    if (ok && changed) *reinterpret_cast<uchar4*>(c.state + e) = make_uchar4(sv[0], sv[1], sv[2], sv[3]);
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      const int x = 4 * g + k;
      const bool commit = ok && x < rd.nx && is_cancer(sv[k]) && phi.a[k] >= T(1);
      const int col = commit ? (x % 3) + 3 * (y % 3) + 9 * (z % 3) : -1;
      const unsigned m = __match_any_sync(FULL, col);
      const int leader = __ffs(m) - 1;
      const int rank = __popc(m & ((1u << lane) - 1u));
      int basev = 0;
      if (commit && lane == leader) basev = atomicAdd(cnt + col, __popc(m));
      basev = __shfl_sync(FULL, basev, leader);
      if (commit) {
        const unsigned long long site = (unsigned long long)x + (unsigned long long)rd.nx * ((unsigned long long)y + (unsigned long long)rd.ny * z);
        c.lists[rd.list_off[col] + basev + rank] = (uint32_t)site;
        my_committed++;
      }
    }
  }
  if (my_committed) atomicAdd(&s_committed, my_committed);
  __syncthreads();
  if (threadIdx.x == 0 && s_committed)
    atomicAdd((unsigned long long*)&c.stats[rep].committed, (unsigned long long)s_committed);
}

template <typename T>
__global__ void __launch_bounds__(256) k_ca_colour(Ctx c, int colour) {
  HCA_COUNT_KERNEL(c);
  __shared__ unsigned int s_cnt[3];
  if (threadIdx.x < 3) s_cnt[threadIdx.x] = 0;
  __syncthreads();
  const int rep = blockIdx.y;
  const RepDesc& rd = c.reps[rep];
  const int n = c.list_count[rep * 27 + colour];
  const uint32_t step = (uint32_t)(*c.step);
  T* phi = (T*)c.phi;
  T* P = (T*)c.P;
  T* Vc = (T*)c.Vc;
  unsigned int kills = 0, divs = 0, blocked = 0;
  const long long sy = rd.nxp, sz = (long long)rd.nxp * rd.ny;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const uint32_t site = c.lists[rd.list_off[colour] + i];
    const int x = (int)(site % (uint32_t)rd.nx);
    const int y = (int)((site / (uint32_t)rd.nx) % (uint32_t)rd.ny);
    const int z = (int)(site / ((uint32_t)rd.nx * (uint32_t)rd.ny));
    const long long e = rd.off + x + sy * y + sz * z;
    if (killed<T>(c, rd, e, site, step)) {
      c.state[e] = HCA_DEAD;
      phi[e] = T(0);
      P[e] = T(0);
      Vc[e] = T(0);
      kills++;
      continue;
    }
    const long long best = best_free<T>(c, rd, x, y, z);
    if (best >= 0) {
      c.state[best] = HCA_PROLIF;
      c.state[e] = HCA_PROLIF;
      phi[e] = T(0);
      P[e] = T(0);
      Vc[e] = T(0);
      phi[best] = T(0);
      P[best] = T(0);
      Vc[best] = T(0);
      divs++;
    } else {
      c.state[e] = HCA_QUIESC;
      phi[e] = T(0);
      blocked++;
    }
  }
  if (kills) atomicAdd(&s_cnt[0], kills);
  if (divs) atomicAdd(&s_cnt[1], divs);
  if (blocked) atomicAdd(&s_cnt[2], blocked);
  __syncthreads();
  if (threadIdx.x == 0) {
    DevStats& st = c.stats[rep];
    if (s_cnt[0]) atomicAdd((unsigned long long*)&st.kills, (unsigned long long)s_cnt[0]);
    if (s_cnt[1]) atomicAdd((unsigned long long*)&st.divisions, (unsigned long long)s_cnt[1]);
    if (s_cnt[2]) atomicAdd((unsigned long long*)&st.blocked, (unsigned long long)s_cnt[2]);
  }
}

// All 27 colour sweeps in one cooperative launch: colour c's cells of every
// replicate (the per-cell step of k_ca_colour, unchanged), then a grid
// barrier (bounded: see grid_barrier) before colour c + 1, so later colours
// see earlier colours' daughters and deaths exactly as with one launch per
// colour; the results are bit-identical to those launches.
template <typename T>
__global__ void __launch_bounds__(256) k_ca_colours(Ctx c) {
  HCA_COUNT_KERNEL(c);
  __shared__ unsigned int s_cnt[3];
  const uint32_t step = (uint32_t)(*c.step);
  T* phi = (T*)c.phi;
  T* P = (T*)c.P;
  T* Vc = (T*)c.Vc;
  if (*(volatile int*)&c.sync->error == SYNC_ERR_TIMEOUT) return;
  for (int colour = 0; colour < 27; ++colour) {
    for (int rep = 0; rep < c.n_reps; ++rep) {
      if (threadIdx.x < 3) s_cnt[threadIdx.x] = 0;
      __syncthreads();
      const RepDesc& rd = c.reps[rep];
      const int n = c.list_count[rep * 27 + colour];
      const long long sy = rd.nxp, sz = (long long)rd.nxp * rd.ny;
      unsigned int kills = 0, divs = 0, blocked = 0;
      for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const uint32_t site = c.lists[rd.list_off[colour] + i];
        const int x = (int)(site % (uint32_t)rd.nx);
        const int y = (int)((site / (uint32_t)rd.nx) % (uint32_t)rd.ny);
        const int z = (int)(site / ((uint32_t)rd.nx * (uint32_t)rd.ny));
        const long long e = rd.off + x + sy * y + sz * z;
        if (killed<T>(c, rd, e, site, step)) {
          c.state[e] = HCA_DEAD;
          phi[e] = T(0);
          P[e] = T(0);
          Vc[e] = T(0);
          kills++;
          continue;
        }
        const long long best = best_free<T>(c, rd, x, y, z);
        if (best >= 0) {
          c.state[best] = HCA_PROLIF;
          c.state[e] = HCA_PROLIF;
          phi[e] = T(0);
          P[e] = T(0);
          Vc[e] = T(0);
          phi[best] = T(0);
          P[best] = T(0);
          Vc[best] = T(0);
          divs++;
        } else {
          c.state[e] = HCA_QUIESC;
          phi[e] = T(0);
          blocked++;
        }
      }
      if (kills) atomicAdd(&s_cnt[0], kills);
      if (divs) atomicAdd(&s_cnt[1], divs);
      if (blocked) atomicAdd(&s_cnt[2], blocked);
      __syncthreads();
      if (threadIdx.x == 0) {
        DevStats& st = c.stats[rep];
        if (s_cnt[0]) atomicAdd((unsigned long long*)&st.kills, (unsigned long long)s_cnt[0]);
        if (s_cnt[1]) atomicAdd((unsigned long long*)&st.divisions, (unsigned long long)s_cnt[1]);
        if (s_cnt[2]) atomicAdd((unsigned long long*)&st.blocked, (unsigned long long)s_cnt[2]);
      }
    }
    if (colour < 26 && !grid_barrier(c.sync, colour)) return;
  }
  grid_exit(c.sync, 26);
}

// ------------------------------------------------- synchronous update ---
// ca_mode 1 (Section 2.5 read with Algorithm 2's rule): every committed cell
// decides against the lattice as it was before the update, and a site picked
// by several parents goes to the highest phi, then the lowest site index.
// Four launches over all 27 colour lists of a replicate:
//   decide: kill test and target (best free neighbour), claim slots reset;
//   claim_phi: atomicMax of phi's bits at the target (phi >= 1 > 0, so the
//              bit patterns order like the values);
//   claim_idx: atomicMin of the site among the claims with the winning phi;
//   apply: kills, divisions of the winners, the rest blocked.
// Nothing the first three write is read by a decision, so thread order does
// not matter.

// Slot of the i-th committed cell of a replicate, taking the colour lists in
// order; -1 past the end.
__device__ __forceinline__ long long slot_of(const Ctx& c, const RepDesc& rd, int rep, int i) {
  const int* cnt = c.list_count + rep * 27;
  for (int col = 0; col < 27; ++col) {
    const int n = cnt[col];
    if (i < n) return rd.list_off[col] + i;
    i -= n;
  }
  return -1;
}

__device__ __forceinline__ int committed_total(const Ctx& c, int rep) {
  int t = 0;
  for (int col = 0; col < 27; ++col) t += c.list_count[rep * 27 + col];
  return t;
}

template <typename T>
__device__ __forceinline__ unsigned long long phi_bits(T v) {
  if constexpr (sizeof(T) == 4) return (unsigned long long)__float_as_uint((float)v);
  else return (unsigned long long)__double_as_longlong((double)v);
}

template <typename T>
__global__ void __launch_bounds__(256) k_ca_sync_decide(Ctx c) {
  HCA_COUNT_KERNEL(c);
  const int rep = blockIdx.y;
  const RepDesc& rd = c.reps[rep];
  const int n = committed_total(c, rep);
  const uint32_t step = (uint32_t)(*c.step);
  const long long sy = rd.nxp, sz = (long long)rd.nxp * rd.ny;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const long long slot = slot_of(c, rd, rep, i);
    const uint32_t site = c.lists[slot];
    const int x = (int)(site % (uint32_t)rd.nx);
    const int y = (int)((site / (uint32_t)rd.nx) % (uint32_t)rd.ny);
    const int z = (int)(site / ((uint32_t)rd.nx * (uint32_t)rd.ny));
    const long long e = rd.off + x + sy * y + sz * z;
    long long dec = -2;
    if (!killed<T>(c, rd, e, site, step)) {
      dec = best_free<T>(c, rd, x, y, z);
      if (dec >= 0) {
        c.claim_phi[dec] = 0ull;
        c.claim_idx[dec] = 0xffffffffu;
      }
    }
    c.ca_dec[slot] = dec;
  }
}

template <typename T>
__global__ void __launch_bounds__(256) k_ca_sync_claim(Ctx c, int pass) {
  HCA_COUNT_KERNEL(c);
  const int rep = blockIdx.y;
  const RepDesc& rd = c.reps[rep];
  const int n = committed_total(c, rep);
  const T* phi = (const T*)c.phi;
  const long long sy = rd.nxp, sz = (long long)rd.nxp * rd.ny;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const long long slot = slot_of(c, rd, rep, i);
    const long long t = c.ca_dec[slot];
    if (t < 0) continue;
    const uint32_t site = c.lists[slot];
    const int x = (int)(site % (uint32_t)rd.nx);
    const int y = (int)((site / (uint32_t)rd.nx) % (uint32_t)rd.ny);
    const int z = (int)(site / ((uint32_t)rd.nx * (uint32_t)rd.ny));
    const unsigned long long b = phi_bits<T>(phi[rd.off + x + sy * y + sz * z]);
    if (pass == 0) atomicMax(c.claim_phi + t, b);
    else if (c.claim_phi[t] == b) atomicMin(c.claim_idx + t, site);
  }
}

template <typename T>
__global__ void __launch_bounds__(256) k_ca_sync_apply(Ctx c) {
  HCA_COUNT_KERNEL(c);
  __shared__ unsigned int s_cnt[3];
  if (threadIdx.x < 3) s_cnt[threadIdx.x] = 0;
  __syncthreads();
  const int rep = blockIdx.y;
  const RepDesc& rd = c.reps[rep];
  const int n = committed_total(c, rep);
  T* phi = (T*)c.phi;
  T* P = (T*)c.P;
  T* Vc = (T*)c.Vc;
  unsigned int kills = 0, divs = 0, blocked = 0;
  const long long sy = rd.nxp, sz = (long long)rd.nxp * rd.ny;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const long long slot = slot_of(c, rd, rep, i);
    const long long t = c.ca_dec[slot];
    const uint32_t site = c.lists[slot];
    const int x = (int)(site % (uint32_t)rd.nx);
    const int y = (int)((site / (uint32_t)rd.nx) % (uint32_t)rd.ny);
    const int z = (int)(site / ((uint32_t)rd.nx * (uint32_t)rd.ny));
    const long long e = rd.off + x + sy * y + sz * z;
    if (t == -2) {
      c.state[e] = HCA_DEAD;
      phi[e] = T(0);
      P[e] = T(0);
      Vc[e] = T(0);
      kills++;
    } else if (t >= 0 && c.claim_idx[t] == site) {
      c.state[t] = HCA_PROLIF;
      c.state[e] = HCA_PROLIF;
      phi[e] = T(0);
      P[e] = T(0);
      Vc[e] = T(0);
      phi[t] = T(0);
      P[t] = T(0);
      Vc[t] = T(0);
      divs++;
    } else {
      c.state[e] = HCA_QUIESC;
      phi[e] = T(0);
      blocked++;
    }
  }
  if (kills) atomicAdd(&s_cnt[0], kills);
  if (divs) atomicAdd(&s_cnt[1], divs);
  if (blocked) atomicAdd(&s_cnt[2], blocked);
  __syncthreads();
  if (threadIdx.x == 0) {
    DevStats& st = c.stats[rep];
    if (s_cnt[0]) atomicAdd((unsigned long long*)&st.kills, (unsigned long long)s_cnt[0]);
    if (s_cnt[1]) atomicAdd((unsigned long long*)&st.divisions, (unsigned long long)s_cnt[1]);
    if (s_cnt[2]) atomicAdd((unsigned long long*)&st.blocked, (unsigned long long)s_cnt[2]);
  }
}

// --------------------------------------------------- vascular automaton ---
// Every vessel_interval steps, after the cell update (Eq. vascular_module,
// Section 2.2.2, A = 0): one Philox draw u per site keyed (seed, site, step,
// VASCULAR).  A vessel with V outside [V_low, V_high] is removed if
// u < p_death; a free site with V inside becomes a vessel if
// u < min(1, (beta_birth S1 (V / V_high)) / S2), where S1 = sum over vessels of
// floor(2^32 V / (V_sprout + V)) and S2 = sum over candidate sites of
// floor(2^32 V / V_high): exact integer sums, so the probability does not
// depend on summation order.  Two launches: the sums (atomic 64-bit integer
// adds), then the update.

__device__ __forceinline__ bool vessel_step(const Ctx& c, const RepDesc& rd) {
  return rd.vessel_interval > 0 && ((*c.step) + 1) % rd.vessel_interval == 0;
}

template <typename T>
__global__ void __launch_bounds__(512) k_vessel_sums(Ctx c) {
  HCA_COUNT_KERNEL(c);
  __shared__ unsigned long long s_sum[2];
  const int2 ch = c.chunks[blockIdx.x];
  const int rep = ch.x;
  const RepDesc& rd = c.reps[rep];
  if (!vessel_step(c, rd)) return;
  if (threadIdx.x < 2) s_sum[threadIdx.x] = 0ull;
  __syncthreads();
  const int nrows = min(rd.chunk_rows, rd.ny * rd.nz - ch.y);
  const long long base0 = rd.off + (long long)ch.y * rd.nxp;
  const T* V = (const T*)c.G[VEGF_SLOT];
  unsigned long long a1 = 0ull, a2 = 0ull;
  for (int i = threadIdx.x; i < nrows * rd.nxp; i += blockDim.x) {
    const int rl = i / rd.nxp, x = i - rl * rd.nxp;
    if (x >= rd.nx) continue;
    const long long e = base0 + (long long)rl * rd.nxp + x;
    const uint8_t s = c.state[e];
    const double v = (double)V[e];
    if (s == HCA_VESSEL) a1 += (unsigned long long)floor(v / (rd.V_sprout + v) * 4294967296.0);
    else if (is_free(s) && v >= rd.V_low && v <= rd.V_high)
      a2 += (unsigned long long)floor(v / rd.V_high * 4294967296.0);
  }
  for (int o = 16; o > 0; o >>= 1) {
    a1 += __shfl_xor_sync(FULL, a1, o);
    a2 += __shfl_xor_sync(FULL, a2, o);
  }
  if ((threadIdx.x & 31) == 0) {
    atomicAdd(&s_sum[0], a1);
    atomicAdd(&s_sum[1], a2);
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    atomicAdd(&c.vsum[2 * rep], s_sum[0]);
    atomicAdd(&c.vsum[2 * rep + 1], s_sum[1]);
  }
}

template <typename T>
__global__ void __launch_bounds__(512) k_vessel_update(Ctx c) {
  HCA_COUNT_KERNEL(c);
  __shared__ unsigned int s_cnt[2];
  const int2 ch = c.chunks[blockIdx.x];
  const int rep = ch.x;
  const RepDesc& rd = c.reps[rep];
  if (!vessel_step(c, rd)) return;
  if (threadIdx.x < 2) s_cnt[threadIdx.x] = 0u;
  __syncthreads();
  const int nrows = min(rd.chunk_rows, rd.ny * rd.nz - ch.y);
  const long long base0 = rd.off + (long long)ch.y * rd.nxp;
  const T* V = (const T*)c.G[VEGF_SLOT];
  const double S1 = (double)c.vsum[2 * rep], S2 = (double)c.vsum[2 * rep + 1];
  const uint32_t step = (uint32_t)(*c.step);
  unsigned int births = 0, deaths = 0;
  for (int i = threadIdx.x; i < nrows * rd.nxp; i += blockDim.x) {
    const int rl = i / rd.nxp, x = i - rl * rd.nxp;
    if (x >= rd.nx) continue;
    const long long e = base0 + (long long)rl * rd.nxp + x;
    const uint8_t s = c.state[e];
    const double v = (double)V[e];
    const bool in_range = v >= rd.V_low && v <= rd.V_high;
    const bool vessel = s == HCA_VESSEL;
    if (!(vessel && !in_range) && !(is_free(s) && in_range && S2 > 0.0)) continue;
    const int j = ch.y + rl;
    const unsigned long long site = (unsigned long long)x + (unsigned long long)rd.nx * (unsigned long long)j;
    const double u = (double)site_uniform(rd.seed, site, step, PURPOSE_VASCULAR);
    if (vessel) {
      if (u < rd.p_death) {
        c.state[e] = HCA_EMPTY;
        deaths++;
      }
    } else {
      const double p = fmin(1.0, __ddiv_rn(__dmul_rn(__dmul_rn(rd.beta_birth, S1), __ddiv_rn(v, rd.V_high)), S2));
      if (u < p) {
        c.state[e] = HCA_VESSEL;
        births++;
      }
    }
  }
  if (births) atomicAdd(&s_cnt[0], births);
  if (deaths) atomicAdd(&s_cnt[1], deaths);
  __syncthreads();
  if (threadIdx.x == 0) {
    if (s_cnt[0]) atomicAdd((unsigned long long*)&c.stats[rep].vessel_births, (unsigned long long)s_cnt[0]);
    if (s_cnt[1]) atomicAdd((unsigned long long*)&c.stats[rep].vessel_deaths, (unsigned long long)s_cnt[1]);
  }
}

}  // namespace

void launch_ca_compact(const Ctx& c, bool fp64) {
  if (fp64) k_ca_compact<double><<<c.n_chunks, c.threads, 0, c.stream>>>(c);
  else k_ca_compact<float><<<c.n_chunks, c.threads, 0, c.stream>>>(c);
}

// Blocks of the cooperative colour kernel (0 where cooperative launches are
// unavailable or HCA_CA_COOP=0): every block resident at once.
int ca_coop_blocks(bool fp64, int sm_count) {
  const char* env = std::getenv("HCA_CA_COOP");
  if (env && env[0] == '0') return 0;
  int dev = 0, coop = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev) != cudaSuccess ||
      !coop) {
    (void)cudaGetLastError();
    return 0;
  }
  const void* fn = fp64 ? (const void*)k_ca_colours<double> : (const void*)k_ca_colours<float>;
  int per_sm = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, 256, 0) != cudaSuccess || per_sm < 1) {
    (void)cudaGetLastError();
    return 0;
  }
  return per_sm * sm_count;
}

void launch_ca_colours(const Ctx& c, int blocks, bool fp64) {
  Ctx cc = c;
  void* args[] = {&cc};
  const void* fn = fp64 ? (const void*)k_ca_colours<double> : (const void*)k_ca_colours<float>;
  (void)cudaLaunchCooperativeKernel(fn, dim3(blocks), dim3(256), args, 0, c.stream);
}

void launch_ca_colour(const Ctx& c, int colour, int blocks_x, bool fp64) {
  dim3 grid(blocks_x, c.n_reps);
  if (fp64) k_ca_colour<double><<<grid, 256, 0, c.stream>>>(c, colour);
  else k_ca_colour<float><<<grid, 256, 0, c.stream>>>(c, colour);
}

void launch_ca_sync(const Ctx& c, int blocks_x, bool fp64) {
  dim3 grid(blocks_x, c.n_reps);
  if (fp64) {
    k_ca_sync_decide<double><<<grid, 256, 0, c.stream>>>(c);
    k_ca_sync_claim<double><<<grid, 256, 0, c.stream>>>(c, 0);
    k_ca_sync_claim<double><<<grid, 256, 0, c.stream>>>(c, 1);
    k_ca_sync_apply<double><<<grid, 256, 0, c.stream>>>(c);
  } else {
    k_ca_sync_decide<float><<<grid, 256, 0, c.stream>>>(c);
    k_ca_sync_claim<float><<<grid, 256, 0, c.stream>>>(c, 0);
    k_ca_sync_claim<float><<<grid, 256, 0, c.stream>>>(c, 1);
    k_ca_sync_apply<float><<<grid, 256, 0, c.stream>>>(c);
  }
}

void launch_vessels(const Ctx& c, bool fp64) {
  if (fp64) {
    k_vessel_sums<double><<<c.n_chunks, c.threads, 0, c.stream>>>(c);
    k_vessel_update<double><<<c.n_chunks, c.threads, 0, c.stream>>>(c);
  } else {
    k_vessel_sums<float><<<c.n_chunks, c.threads, 0, c.stream>>>(c);
    k_vessel_update<float><<<c.n_chunks, c.threads, 0, c.stream>>>(c);
  }
}

}  // namespace hca
