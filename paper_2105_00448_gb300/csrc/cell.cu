// Lattice initialisation, the per-cell ODEs and small utility kernels.
//
// Initialisation (Algorithm 1, steps 2-5): a site holds a vessel if
// u_v < p_vessel, else a cancer cell if u_c < p_cell; cancer cells draw
// phi = u_phi ~ U(0, 1).  u are 24-bit Philox uniforms keyed by
// (seed, site, 0, purpose).  P = Vc = 0, G = 0, K = K0 (start of the initial
// oxygen fixed point).
//
// ODEs over one step dt with K fixed at the cell's site (Section 2.4.2):
//   phi += dt K / (T (K_phi + K))                         (Eq. cellcycle, exact)
//   P(s) = P0 e^{-lam s} - k1 expm1(-lam s) / lam,  lam = k1' K/(K_p53 + K)
//                                                          (Eq. odep53, exact)
//   Vc: classical RK4 with h = dt / substeps on Eq. (odevegf), P taken from
//       its exact solution at each stage time (the exponential advanced
//       half-step by half-step through the expm1 addition formula).
// phi is advanced for cancer cells, P and Vc for every cell (cancer, stroma).
#include "hca_internal.cuh"

namespace hca {
namespace {

__device__ __forceinline__ float t_exp(float v) { return expf(v); }
__device__ __forceinline__ double t_exp(double v) { return exp(v); }
__device__ __forceinline__ float t_expm1(float v) { return expm1f(v); }
__device__ __forceinline__ double t_expm1(double v) { return expm1(v); }

template <typename T>
__global__ void __launch_bounds__(512) k_init(Ctx c, const float* __restrict__ pc, const float* __restrict__ pf,
                                              const float* __restrict__ pv, int* __restrict__ err) {
  HCA_COUNT_KERNEL(c);
  const int2 ch = c.chunks[blockIdx.x];
  const RepDesc& rd = c.reps[ch.x];
  const int nrows = min(rd.chunk_rows, rd.ny * rd.nz - ch.y);
  const long long base0 = rd.off + (long long)ch.y * rd.nxp;
  const int ngroups = nrows * rd.gpr;
  for (int gi = threadIdx.x; gi < ngroups; gi += blockDim.x) {
    const int rl = gi / rd.gpr, g = gi % rd.gpr;
    const int j = ch.y + rl;
    const int y = j % rd.ny, z = j / rd.ny;
    const long long e = base0 + (long long)rl * rd.nxp + 4LL * g;
    uchar4 st = make_uchar4(0, 0, 0, 0);
    V4<T> phi = zero4<T>(), perf = zero4<T>(), K = zero4<T>();
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      const int x = 4 * g + k;
      if (x >= rd.nx) continue;
      const float p_c = pc[e + k], p_f = pf[e + k], p_v = pv[e + k];
      if (!(p_c >= 0.f && p_c <= 1.f) || !(p_v >= 0.f && p_v <= 1.f) || !(p_f >= 0.f) || !isfinite(p_f))
        atomicOr(err, 1);
      const unsigned long long site = (unsigned long long)x + (unsigned long long)rd.nx * ((unsigned long long)y + (unsigned long long)rd.ny * z);
      const float u_v = site_uniform(rd.seed, site, 0u, PURPOSE_VESSEL);
      const float u_c = site_uniform(rd.seed, site, 0u, PURPOSE_CANCER);
      const float u_p = site_uniform(rd.seed, site, 0u, PURPOSE_PHI);
      uint8_t s = HCA_EMPTY;
      if (u_v < p_v) s = HCA_VESSEL;
      else if (u_c < p_c) s = HCA_PROLIF;
      if (k == 0) st.x = s; else if (k == 1) st.y = s; else if (k == 2) st.z = s; else st.w = s;
      phi.a[k] = s == HCA_PROLIF ? (T)u_p : T(0);
      perf.a[k] = (T)p_f;
      K.a[k] = (T)rd.K0;
    }
    *reinterpret_cast<uchar4*>(c.state + e) = st;
    st4((T*)c.phi + e, phi);
    st4((T*)c.P + e, zero4<T>());
    st4((T*)c.Vc + e, zero4<T>());
    st4((T*)c.perf + e, perf);
    st4((T*)c.K + e, K);
    if (c.K_lo) st4((T*)c.K_lo + e, zero4<T>());
    for (int d = 0; d < rd.n_drugs; ++d) {
      st4((T*)c.G[d] + e, zero4<T>());
      if (c.G_lo[d]) st4((T*)c.G_lo[d] + e, zero4<T>());
    }
  }
}

// v / (J5 + v) of the Vc rate: in FP32 the fast division (__fdividef, two
// units in the last place; the rate's error enters Vc only through the small
// increment h f, so Vc keeps FP32 accuracy), in FP64 the IEEE division.
__device__ __forceinline__ float sat(float v, float d) { return __fdividef(v, d); }
__device__ __forceinline__ double sat(double v, double d) { return v / d; }

template <typename T>
__device__ __forceinline__ T p53_at(T P0, T lam, T s, T k1) {
  return lam != T(0) ? P0 * t_exp(-lam * s) - k1 * t_expm1(-lam * s) / lam : P0 + k1 * s;
}

// Per-cell ODEs over one chunk of rows.  A warp packs the consuming sites of
// its four-site groups into a shared-memory list and its lanes take the
// list's entries 32 at a time; a partial last batch waits in the list for
// the warp's next groups, so the 60-substep RK4 keeps every lane busy
// whatever the mix of cells and empty sites (each site's arithmetic is
// unchanged).
template <typename T>
__global__ void __launch_bounds__(512) k_ode(Ctx c) {
  HCA_COUNT_KERNEL(c);
  constexpr int kMaxWarps = 16;
  __shared__ long long s_site[kMaxWarps][128 + 32];
  const int2 ch = c.chunks[blockIdx.x];
  const RepDesc& rd = c.reps[ch.x];
  const int nrows = min(rd.chunk_rows, rd.ny * rd.nz - ch.y);
  const long long base0 = rd.off + (long long)ch.y * rd.nxp;
  const int ngroups = nrows * rd.gpr;
  const T dt = (T)rd.dt, Tc = (T)rd.T_cycle, Kphi = (T)rd.K_phi;
  const T k1 = (T)rd.k1, k1p = (T)rd.k1p, Kp53 = (T)rd.K_p53;
  const T k2 = (T)rd.k2, k2p = (T)rd.k2p, k2pp = (T)rd.k2pp, J5 = (T)rd.J5, KV = (T)rd.K_V;
  const int nsub = rd.ode_substeps;
  const T h = (T)(rd.dt / nsub);
  const T half = T(0.5) * h;
  const T sixth = h / T(6);
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const T* __restrict__ KK = (const T*)c.K;
  T* __restrict__ PHI = (T*)c.phi;
  T* __restrict__ PP = (T*)c.P;
  T* __restrict__ VV = (T*)c.Vc;
  long long* list = s_site[wid];
  auto cell = [&](long long q) {
    const uint8_t s = c.state[q];
    const T Kk = KK[q];
    if (is_cancer(s)) PHI[q] = PHI[q] + dt * Kk / (Tc * (Kphi + Kk));
    const T lam = k1p * Kk / (Kp53 + Kk);
    const T decay = k2p * Kk / (KV + Kk);
    const T P0 = PP[q];
    T v = VV[q];
    // one classical RK4 substep of Vc with P at the stage times (Pa, Pb, Pc)
    auto rk4 = [&](T Pa, T Pb, T Pc) {
      const T f1 = k2 + k2pp * Pa * sat(v, J5 + v) - decay * v;
      const T v2 = v + half * f1;
      const T f2 = k2 + k2pp * Pb * sat(v2, J5 + v2) - decay * v2;
      const T v3 = v + half * f2;
      const T f3 = k2 + k2pp * Pb * sat(v3, J5 + v3) - decay * v3;
      const T v4 = v + h * f3;
      const T f4 = k2 + k2pp * Pc * sat(v4, J5 + v4) - decay * v4;
      v = v + sixth * (f1 + T(2) * f2 + T(2) * f3 + f4);
    };
    T Pa = P0;
    if (lam != T(0)) {
      // P(s) = P0 e^{-lam s} + k1 (1 - e^{-lam s}) / lam = P0 + E(s) (P0 - k1 / lam) with
      // E(s) = expm1(-lam s).  The stage times are multiples of h/2, and
      // expm1(a + b) = expm1(a) + expm1(b) + expm1(a) expm1(b), so E advances
      // by one half-step with E <- E + q + E q, q = expm1(-lam h/2): one
      // transcendental per cell instead of two per substep (the recurrence
      // adds ~1 ulp of E per half-step)
      const T A0 = P0 - k1 / lam;
      const T qh = t_expm1(-lam * half);
      T E = T(0);
      for (int m = 0; m < nsub; ++m) {
        E = E + qh + E * qh;
        const T Pb = P0 + E * A0;
        E = E + qh + E * qh;
        const T Pc = P0 + E * A0;
        rk4(Pa, Pb, Pc);
        Pa = Pc;
      }
    } else {
      // no p53 decay (K = 0): P grows linearly, P(s) = P0 + k1 s
      for (int m = 0; m < nsub; ++m) {
        const T s0 = (T)m * h;
        const T Pb = P0 + k1 * (s0 + half);
        const T Pc = P0 + k1 * (s0 + h);
        rk4(Pa, Pb, Pc);
        Pa = Pc;
      }
    }
    VV[q] = v;
    PP[q] = p53_at(P0, lam, dt, k1);
  };
  int n = 0;   // cells waiting in the warp's list (fewer than 32)
  for (int gbase = 0; gbase < ngroups; gbase += blockDim.x) {
    const int gi = gbase + threadIdx.x;
    unsigned live = 0;
    long long e = 0;
    if (gi < ngroups) {
      const int rl = gi / rd.gpr, g = gi % rd.gpr;
      e = base0 + (long long)rl * rd.nxp + 4LL * g;
      const uchar4 st = ld_state4(c.state + e);
#pragma unroll
      for (int k = 0; k < 4; ++k)
        if (is_consumer(st_at(st, k)) && 4 * g + k < rd.nx) live |= 1u << k;
    }
    // exclusive prefix of the live counts over the warp's lanes
    const int cnt = __popc(live);
    int pre = cnt;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int v = __shfl_up_sync(0xffffffffu, pre, o);
      if (lane >= o) pre += v;
    }
    const int total = n + __shfl_sync(0xffffffffu, pre, 31);
    pre += n - cnt;
#pragma unroll
    for (int k = 0; k < 4; ++k)
      if (live >> k & 1u) list[pre++] = e + k;
    __syncwarp();
    const int full = total & ~31;
    for (int j = 0; j < full; j += 32) cell(list[j + lane]);
    // the partial batch moves to the front of the list
    n = total - full;
    const long long keep = lane < n ? list[full + lane] : 0;
    __syncwarp();
    if (lane < n) list[lane] = keep;
    __syncwarp();
  }
  if (lane < n) cell(list[lane]);
}

// Sites per state code, per replicate (into stats[rep].counts).
__global__ void __launch_bounds__(512) k_histogram(Ctx c) {
  HCA_COUNT_KERNEL(c);
  __shared__ unsigned int h[6];
  if (threadIdx.x < 6) h[threadIdx.x] = 0;
  __syncthreads();
  const int2 ch = c.chunks[blockIdx.x];
  const RepDesc& rd = c.reps[ch.x];
  const int nrows = min(rd.chunk_rows, rd.ny * rd.nz - ch.y);
  const long long base0 = rd.off + (long long)ch.y * rd.nxp;
  unsigned int loc[6] = {0, 0, 0, 0, 0, 0};
  for (int i = threadIdx.x; i < nrows * rd.nx; i += blockDim.x) {
    const int rl = i / rd.nx, x = i % rd.nx;
    const uint8_t s = c.state[base0 + (long long)rl * rd.nxp + x];
    if (s < 6) loc[s]++;
  }
  for (int k = 0; k < 6; ++k)
    if (loc[k]) atomicAdd(&h[k], loc[k]);
  __syncthreads();
  if (threadIdx.x < 6 && h[threadIdx.x])
    atomicAdd((unsigned long long*)&c.stats[ch.x].counts[threadIdx.x], (unsigned long long)h[threadIdx.x]);
}

__global__ void k_philox_uniforms(unsigned long long seed, unsigned long long site0, long long n, uint32_t step,
                                  uint32_t purpose, float* out) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    out[i] = site_uniform(seed, site0 + (unsigned long long)i, step, purpose);
}

__global__ void k_advance_step(long long* step, long long by, unsigned long long* n_kernels) {
  if (threadIdx.x == 0 && blockIdx.x == 0) {
    *step += by;
    atomicAdd(n_kernels, 1ull);
  }
}

}  // namespace

void launch_init(const Ctx& c, const float* pc, const float* pf, const float* pv, int* err, bool fp64) {
  if (fp64) k_init<double><<<c.n_chunks, c.threads, 0, c.stream>>>(c, pc, pf, pv, err);
  else k_init<float><<<c.n_chunks, c.threads, 0, c.stream>>>(c, pc, pf, pv, err);
}

void launch_ode(const Ctx& c, bool fp64) {
  if (fp64) launch_k(c.pdl != 0, k_ode<double>, dim3(c.n_chunks), dim3(c.threads), 0, c.stream, c);
  else launch_k(c.pdl != 0, k_ode<float>, dim3(c.n_chunks), dim3(c.threads), 0, c.stream, c);
}

void launch_histogram(const Ctx& c) { k_histogram<<<c.n_chunks, c.threads, 0, c.stream>>>(c); }

void launch_philox_uniforms(unsigned long long seed, unsigned long long site0, long long n, uint32_t step,
                            uint32_t purpose, float* out, cudaStream_t stream) {
  long long blocks = (n + 255) / 256;
  if (blocks > 4096) blocks = 4096;
  if (blocks < 1) blocks = 1;
  k_philox_uniforms<<<(unsigned)blocks, 256, 0, stream>>>(seed, site0, n, step, purpose, out);
}

void launch_advance_step(const Ctx& c, long long by) { k_advance_step<<<1, 32, 0, c.stream>>>(c.step, by, c.n_kernels); }

}  // namespace hca
