// Geometric-multigrid V-cycle preconditioner for the CG solves of
// Eqs. (oxygen) and (chemo): z = M r with M one symmetric V-cycle.
//
// The paper preconditions CG with algebraic multigrid (BoomerAMG,
// Section 2.4); on the uniform lattice the geometric counterpart needs no
// setup beyond summing reaction coefficients.  Level l+1 halves every extent
// (ceil); its site owns the existing children 2I + {0,1}^3.  Coupling
// c_{l+1} = 2 c_l (the Laplacian at twice the spacing, scaled by the 8x
// volume); reaction a_{l+1} = sum of the children's a_l; diagonal
// d_l = c_l n_l + a_l with n_l the in-box neighbour count (Neumann).
// Restriction sums over the children, prolongation copies to them, the
// smoother is Jacobi with Chebyshev weights (two sweeps before the coarse
// correction, MG_W1 then MG_W2, and two after it, MG_W2 then MG_W1;
// MG_NU_COARSE sweeps of weight MG_OMEGA_COARSE on the coarsest level), so M
// is symmetric.
//
// Level 0 is the solver's padded field layout: rhs = r, diagonal = d, 1/d in
// mg_w; z holds the pre-smoothed iterate v between the pre-sweep kernel and
// the restriction, mg_t0 the part v' of the first post-sweep that the
// restriction leaves for the post-sweep kernels (or the iterate when the
// lattice is the coarsest level); coarser levels are dense arrays, the replicates of a batch
// concatenated per level (each replicate has its own hierarchy; a per-level
// prefix table maps a flattened site index to its replicate).  Levels of at
// most MG_SMALL_SITES sites run inside one block per replicate (block
// barriers between sweeps).  The last kernel, the last post-sweep on level 0,
// also forms rho = r.z with the fixed-order reductions of the CG passes and
// sets beta, per replicate.

#include <algorithm>
#include <cstdlib>
#include <type_traits>

#include "hca_internal.cuh"
#include "row_ops.cuh"
#include "tc.cuh"

namespace hca {

int persist_grid(const void* fn, int threads, int sm_count);

namespace {

constexpr int kMgThreads = 256;
constexpr int kSmallThreads = 1024;

template <typename T>
struct View {
  int nx, ny, nz;
  long long off, sy, sz;
  T *x, *t, *rhs, *d, *w;   // w = 1 / d (0 where d = 0): the sweeps divide nowhere
  T c;
  __device__ __forceinline__ long long n() const { return (long long)nx * ny * nz; }
  __device__ __forceinline__ long long at(int X, int Y, int Z) const { return off + X + sy * Y + sz * Z; }
  // 32-bit arithmetic: lattices hold fewer than 2^31 sites (64-bit division
  // would dominate these kernels' instruction count)
  __device__ __forceinline__ void coords(long long s, int& X, int& Y, int& Z) const {
    const unsigned u = (unsigned)s, q = u / (unsigned)nx;
    X = (int)(u - q * (unsigned)nx);
    Z = (int)(q / (unsigned)ny);
    Y = (int)(q - (unsigned)Z * (unsigned)ny);
  }
  __device__ __forceinline__ int nbcount(int X, int Y, int Z) const {
    return (X > 0) + (X < nx - 1) + (Y > 0) + (Y < ny - 1) + (Z > 0) + (Z < nz - 1);
  }
  // (A u)_e
  __device__ __forceinline__ T apply(const T* __restrict__ u, int X, int Y, int Z, long long e) const {
    T nb = T(0);
    if (X > 0) nb += u[e - 1];
    if (X < nx - 1) nb += u[e + 1];
    if (Y > 0) nb += u[e - sy];
    if (Y < ny - 1) nb += u[e + sy];
    if (Z > 0) nb += u[e - sz];
    if (Z < nz - 1) nb += u[e + sz];
    return d[e] * u[e] - c * nb;
  }
};

template <typename T>
__device__ __forceinline__ View<T> view(const Ctx& c, int which, int r, int l) {
  const RepDesc& rd = c.reps[r];
  View<T> v;
  const T c0 = op_coupling_t<T>(rd, which);
  if (l == 0) {
    v.nx = rd.nx;
    v.ny = rd.ny;
    v.nz = rd.nz;
    v.off = rd.off;
    v.sy = rd.nxp;
    v.sz = (long long)rd.nxp * rd.ny;
    v.x = (T*)c.mg_t0;
    v.t = (T*)c.mg_t0;   // level 0 prolongs in place
    v.rhs = (T*)c.r;
    v.d = (T*)c.d;
    v.w = (T*)c.mg_w;
    v.c = c0;
    return v;
  }
  const MGLevel& L = ((const MGLevel*)c.mg_lv)[r * MG_MAXLEV + l];
  v.nx = L.nx;
  v.ny = L.ny;
  v.nz = L.nz;
  v.off = 0;
  v.sy = L.nx;
  v.sz = (long long)L.nx * L.ny;
  v.x = (T*)L.x;
  v.t = (T*)L.t;
  v.rhs = (T*)L.rhs;
  v.d = (T*)L.d;
  v.w = (T*)L.w;
  v.c = c0 * (sizeof(T) == 4 ? (T)L.cscale32 : (T)L.cscale);
  return v;
}

// Replicate that owns flattened site q of level l: the last r with
// start[l][r] <= q (replicates without level l have empty ranges).
__device__ __forceinline__ int rep_of(const Ctx& c, int l, long long q) {
  const long long* st = c.mg_start + (long long)l * (c.n_reps + 1);
  int lo = 0, hi = c.n_reps;
  while (hi - lo > 1) {
    const int mid = (lo + hi) >> 1;
    if (st[mid] <= q) lo = mid;
    else hi = mid;
  }
  return lo;
}

__device__ __forceinline__ long long rep_start(const Ctx& c, int l, int r) {
  return c.mg_start[(long long)l * (c.n_reps + 1) + r];
}

// The replicate of the flattened sites a thread visits, with its views on
// levels l and l + 1, refreshed only when a site falls outside the cached
// replicate's range (a thread's consecutive sites nearly always share one).
template <typename T>
struct RepCursor {
  int r = -1;
  long long lo = 0, hi = 0;
  View<T> F, C;
  __device__ __forceinline__ bool at(const Ctx& c, int which, int l, long long q, bool coarse) {
    if (q >= lo && q < hi) return false;
    r = rep_of(c, l, q);
    lo = rep_start(c, l, r);
    hi = rep_start(c, l, r + 1);
    F = view<T>(c, which, r, l);
    if (coarse) C = view<T>(c, which, r, l + 1);
    return true;
  }
};

// ------------------------------------------------------ per-site steps --
// d_C(I) = c_C n_C(I) + sum over children of max(0, d_F - c_F n_F); w_C = 1 / d_C.
// FP64 fields: in FP64.  FP32 fields: in FP32 (FP64 runs at a small fraction
// of the FP32 rate on this GPU); d_F - c_F n_F is then exact whenever
// c_F n_F is within a factor two of d_F (Sterbenz), i.e. the recovered
// reaction carries only the rounding of the stored FP32 diagonal and of c_F n_F.
__device__ __forceinline__ float nbcount_f(int X, int Y, int Z, int nx, int ny, int nz) {
  return ((X > 0 ? 1.f : 0.f) + (X < nx - 1 ? 1.f : 0.f)) + ((Y > 0 ? 1.f : 0.f) + (Y < ny - 1 ? 1.f : 0.f)) +
         ((Z > 0 ? 1.f : 0.f) + (Z < nz - 1 ? 1.f : 0.f));
}

template <typename T>
__device__ void coarse_diag_at(const View<T>& F, const View<T>& C, long long S);

template <>
__device__ void coarse_diag_at<float>(const View<float>& F, const View<float>& C, long long S) {
  int X, Y, Z;
  C.coords(S, X, Y, Z);
  float a = 0.f;
  for (int k = 0; k < 8; ++k) {
    const int x = 2 * X + (k & 1), y = 2 * Y + ((k >> 1) & 1), z = 2 * Z + (k >> 2);
    if (x < F.nx && y < F.ny && z < F.nz)
      a += fmaxf(0.f, F.d[F.at(x, y, z)] - F.c * nbcount_f(x, y, z, F.nx, F.ny, F.nz));
  }
  const float dc = C.c * nbcount_f(X, Y, Z, C.nx, C.ny, C.nz) + a;
  C.d[C.at(X, Y, Z)] = dc;
  C.w[C.at(X, Y, Z)] = dc != 0.f ? 1.f / dc : 0.f;
}

template <>
__device__ void coarse_diag_at<double>(const View<double>& F, const View<double>& C, long long S) {
  int X, Y, Z;
  C.coords(S, X, Y, Z);
  double a = 0.0;
  for (int k = 0; k < 8; ++k) {
    const int x = 2 * X + (k & 1), y = 2 * Y + ((k >> 1) & 1), z = 2 * Z + (k >> 2);
    if (x < F.nx && y < F.ny && z < F.nz)
      a += fmax(0.0, F.d[F.at(x, y, z)] - F.c * F.nbcount(x, y, z));
  }
  const double dc = C.c * C.nbcount(X, Y, Z) + a;
  C.d[C.at(X, Y, Z)] = dc;
  C.w[C.at(X, Y, Z)] = dc != 0.0 ? 1.0 / dc : 0.0;
}

// w = 1 / d on the lattice
template <typename T>
__device__ void lattice_w_at(const View<T>& V, long long s) {
  int X, Y, Z;
  V.coords(s, X, Y, Z);
  const long long e = V.at(X, Y, Z);
  const T d = V.d[e];
  V.w[e] = d != T(0) ? T(1) / d : T(0);
}

// Every sweep of weight om at a site scales by om * w, one rounding: the
// row-vector and per-site forms below form it the same way.
template <typename T>
__device__ __forceinline__ T wt(double om, T w) {
  return (T)om * w;
}

// rhs - (A u) at a site with diagonal d and neighbour sum nb, as
// rhs - fma(d, u, -(c nb)): one explicit rounding order, so that the
// per-site and row-vector forms of a step give the same bits whatever the
// compiler would contract.
template <typename T>
__device__ __forceinline__ T resid(T rhs, T d, T u, T c, T nb) {
  return rhs - fma(d, u, -(c * nb));
}

// a * b rounded on its own (never contracted into a following sum)
__device__ __forceinline__ float mul_rn(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ double mul_rn(double a, double b) { return __dmul_rn(a, b); }

// dst = (om / d) rhs: a sweep from zero
template <typename T>
__device__ void sweep_first_at(const View<T>& V, T* __restrict__ dst, long long s, double om) {
  int X, Y, Z;
  V.coords(s, X, Y, Z);
  const long long e = V.at(X, Y, Z);
  dst[e] = wt(om, V.w[e]) * V.rhs[e];
}

// dst = src + (om / d)(rhs - A src)
template <typename T>
__device__ void sweep_at(const View<T>& V, const T* __restrict__ src, T* __restrict__ dst, long long s, double om) {
  int X, Y, Z;
  V.coords(s, X, Y, Z);
  const long long e = V.at(X, Y, Z);
  const T r = V.rhs[e] - V.apply(src, X, Y, Z, e);
  dst[e] = fma(wt(om, V.w[e]), r, src[e]);
}

// rhs_C(I) = sum over children of (rhs_F - A_F x_F)
template <typename T>
__device__ void restrict_residual_at(const View<T>& F, const View<T>& C, long long S) {
  int X, Y, Z;
  C.coords(S, X, Y, Z);
  T acc = T(0);
  for (int k = 0; k < 8; ++k) {
    const int x = 2 * X + (k & 1), y = 2 * Y + ((k >> 1) & 1), z = 2 * Z + (k >> 2);
    if (x < F.nx && y < F.ny && z < F.nz) {
      const long long e = F.at(x, y, z);
      const T* u = F.x;
      T nb = T(0);
      if (x > 0) nb += u[e - 1];
      if (x < F.nx - 1) nb += u[e + 1];
      if (y > 0) nb += u[e - F.sy];
      if (y < F.ny - 1) nb += u[e + F.sy];
      if (z > 0) nb += u[e - F.sz];
      if (z < F.nz - 1) nb += u[e + F.sz];
      acc += resid(F.rhs[e], F.d[e], u[e], F.c, nb);
    }
  }
  C.rhs[C.at(X, Y, Z)] = acc;
}

// Coordinates of the sites s0, s0 + st, s0 + 2 st, ... of a dense level
// (s = X + nx (Y + ny Z)), advanced by mixed-radix addition instead of a
// division per site.
struct Walk {
  int X, Y, Z, ax, ay, az, nx, ny;
  __device__ __forceinline__ Walk(int s0, int st, int nx_, int ny_) : nx(nx_), ny(ny_) {
    int q = s0 / nx;
    X = s0 - q * nx;
    Z = q / ny;
    Y = q - Z * ny;
    q = st / nx;
    ax = st - q * nx;
    az = q / ny;
    ay = q - az * ny;
  }
  __device__ __forceinline__ void next() {
    X += ax;
    int cy = X >= nx;
    if (cy) X -= nx;
    Y += ay + cy;
    cy = Y >= ny;
    if (cy) Y -= ny;
    Z += az + cy;
  }
};

// The per-site steps on a dense level (element index = site index s) at
// known coordinates: the same arithmetic, in the same order, as sweep_at /
// restrict_residual_at.
template <typename T>
__device__ __forceinline__ void sweep_xyz(const View<T>& V, const T* src, T* dst, int X, int Y, int Z, int s,
                                          double om) {
  const T r = V.rhs[s] - V.apply(src, X, Y, Z, s);
  dst[s] = fma(wt(om, V.w[s]), r, src[s]);
}

template <typename T>
__device__ __forceinline__ void restrict_residual_xyz(const View<T>& F, const View<T>& C, int X, int Y, int Z, int S) {
  T acc = T(0);
  for (int k = 0; k < 8; ++k) {
    const int x = 2 * X + (k & 1), y = 2 * Y + ((k >> 1) & 1), z = 2 * Z + (k >> 2);
    if (x < F.nx && y < F.ny && z < F.nz) {
      const long long e = x + (long long)F.nx * (y + (long long)F.ny * z);
      acc += F.rhs[e] - F.apply(F.x, x, y, z, e);
    }
  }
  C.rhs[S] = acc;
}

// x_F += P x_C (in place: a site reads only its own x and its coarse cell)
template <typename T>
__device__ __forceinline__ void prolong_xyz(const View<T>& F, const View<T>& C, int X, int Y, int Z, int s) {
  F.x[s] = F.x[s] + C.x[(X >> 1) + (long long)C.nx * ((Y >> 1) + (long long)C.ny * (Z >> 1))];
}

// The three sweeps of a grid level l >= 1 around its coarse correction, each
// fused with the step before it (the iterate they start from is formed at
// the site and its neighbours, not stored):
//   SM_PRE:  x = u + (W2 / d)(rhs - A u), u = (W1 / d) rhs (both pre-sweeps)
//   SM_POST: t = u + (W2 / d)(rhs - A u), u = x + P x_C (prolongation, first post-sweep)
//   SM_LAST: x = t + (W1 / d)(rhs - A t) (second post-sweep)
// Neighbour sums in the order x - 1, x + 1, y - 1, y + 1, z - 1, z + 1 (the
// row-vector form smooth_rows forms the same sums).
enum { SM_PRE = 0, SM_POST = 1, SM_LAST = 2 };

template <typename T, int MODE>
__device__ void smooth_at(const View<T>& F, const View<T>& C, long long s) {
  auto u = [&](int x, int y, int z) {
    const long long ef = F.at(x, y, z);
    if (MODE == SM_PRE) return mul_rn(wt(MG_W1, F.w[ef]), F.rhs[ef]);
    if (MODE == SM_POST) return F.x[ef] + C.x[C.at(x >> 1, y >> 1, z >> 1)];
    return F.t[ef];
  };
  int X, Y, Z;
  F.coords(s, X, Y, Z);
  const long long e = F.at(X, Y, Z);
  T nb = T(0);
  if (X > 0) nb += u(X - 1, Y, Z);
  if (X < F.nx - 1) nb += u(X + 1, Y, Z);
  if (Y > 0) nb += u(X, Y - 1, Z);
  if (Y < F.ny - 1) nb += u(X, Y + 1, Z);
  if (Z > 0) nb += u(X, Y, Z - 1);
  if (Z < F.nz - 1) nb += u(X, Y, Z + 1);
  const T uc = u(X, Y, Z);
  const T res = resid(F.rhs[e], F.d[e], uc, F.c, nb);
  const T out = fma(wt(MODE == SM_LAST ? MG_W1 : MG_W2, F.w[e]), res, uc);
  if (MODE == SM_POST) F.t[e] = out;
  else F.x[e] = out;
}

// Grid-stride loop over the flattened sites of level l of every replicate
// (a per-site lookup of the owning replicate in the level's prefix table).
#define HCA_MG_FOR_SITES_FROM(l, t0, st)                                                              \
  for (long long q = (t0); q < c.mg_start[(long long)(l) * (c.n_reps + 1) + c.n_reps]; q += (st))
#define HCA_MG_FOR_SITES(l) \
  HCA_MG_FOR_SITES_FROM(l, blockIdx.x * (long long)blockDim.x + threadIdx.x, (long long)gridDim.x * blockDim.x)

// This thread's first item and the stride of a grid-stride loop.
__device__ __forceinline__ long long grid_t0() { return blockIdx.x * (long long)blockDim.x + threadIdx.x; }
__device__ __forceinline__ long long grid_st() { return (long long)gridDim.x * blockDim.x; }

// ------------------------------------------------------- grid kernels ---
template <typename T>
__global__ void __launch_bounds__(kMgThreads) k_mg_w0(Ctx c, int which) {
  HCA_COUNT_KERNEL(c);
  RepCursor<T> k;
  HCA_MG_FOR_SITES(0) {
    k.at(c, which, 0, q, false);
    lattice_w_at<T>(k.F, q - k.lo);
  }
}

template <typename T>
__global__ void __launch_bounds__(kMgThreads) k_mg_diag(Ctx c, int which, int l) {
  HCA_COUNT_KERNEL(c);
  RepCursor<T> k;
  View<T> Fm;
  HCA_MG_FOR_SITES(l) {
    if (k.at(c, which, l, q, false)) Fm = view<T>(c, which, k.r, l - 1);
    coarse_diag_at<T>(Fm, k.F, q - k.lo);
  }
}

// The defect-correction residual is stored unscaled: on the first
// application of a rescaled inner solve, r *= scale (elementwise, in place);
// replicates past that return at once.
template <typename T>
__global__ void __launch_bounds__(kMgThreads) k_mg_scale0(Ctx c, int which) {
  HCA_VC_ENTRY(c);
  RepCursor<T> k;
  bool skip = true;
  T sc = T(1);
  HCA_MG_FOR_SITES(0) {
    if (k.at(c, which, 0, q, false)) {
      const RepSolve& sv = c.solve[k.r];
      skip = sv.iters != 0 || sv.scale == 1.0;
      sc = (T)sv.scale;
    }
    if (skip) continue;
    int X, Y, Z;
    k.F.coords(q - k.lo, X, Y, Z);
    k.F.rhs[k.F.at(X, Y, Z)] *= sc;
  }
}

// k_mg_scale0 for one lattice as a stream of four-site groups (row-major,
// vector loads and stores; padding sites are left as they are).
template <typename T>
__global__ void __launch_bounds__(256) k_mg_scale0_rows(Ctx c) {
  HCA_VC_ENTRY(c);
  const RepSolve& sv = c.solve[0];
  if (sv.iters != 0 || sv.scale == 1.0) return;
  const T sc = (T)sv.scale;
  const RepDesc& rd = c.reps[0];
  T* __restrict__ r = (T*)c.r + rd.off;
  const long long ng = (long long)rd.gpr * rd.ny * rd.nz;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < ng; i += (long long)gridDim.x * blockDim.x) {
    const long long row = i / rd.gpr;
    const int x0 = 4 * (int)(i - row * rd.gpr);
    T* p = r + row * rd.nxp + x0;
    V4<T> v = ld4(p);
#pragma unroll
    for (int e = 0; e < 4; ++e)
      if (x0 + e < rd.nx) v.a[e] *= sc;
    st4(p, v);
  }
}

// The lattice as the coarsest level (single replicate): t0 = (omega / d) r
template <typename T>
__global__ void __launch_bounds__(kMgThreads) k_mg_first0(Ctx c, int which) {
  HCA_VC_ENTRY(c);
  const View<T> V = view<T>(c, which, 0, 0);
  for (long long s = blockIdx.x * (long long)blockDim.x + threadIdx.x; s < V.n(); s += (long long)gridDim.x * blockDim.x)
    sweep_first_at<T>(V, V.x, s, MG_OMEGA_COARSE);
}

template <typename T>
__global__ void __launch_bounds__(kMgThreads) k_mg_sweep0(Ctx c, int which, const T* src, T* dst) {
  HCA_VC_ENTRY(c);
  const View<T> V = view<T>(c, which, 0, 0);
  for (long long s = blockIdx.x * (long long)blockDim.x + threadIdx.x; s < V.n(); s += (long long)gridDim.x * blockDim.x)
    sweep_at<T>(V, src, dst, s, MG_OMEGA_COARSE);
}

// Restriction of the pre-smoothed residual from level l to l + 1 for the
// replicates whose level l is swept by grid kernels (l below their first
// single-block level).  MULTI = false: one replicate, whose views are fixed
// for the whole loop (fewer registers).  t0, st: this thread's first item
// and the loop stride.
template <typename T, bool MULTI>
__device__ __forceinline__ void restrict_sites(const Ctx& c, int which, int l, long long t0, long long st) {
  if (!MULTI) {
    const View<T> F = view<T>(c, which, 0, l), C = view<T>(c, which, 0, l + 1);
    for (long long s = t0; s < C.n(); s += st) restrict_residual_at<T>(F, C, s);
    return;
  }
  RepCursor<T> k;   // cursor on level l + 1 (its F is the coarse view)
  View<T> Ff;
  bool skip = true;
  HCA_MG_FOR_SITES_FROM(l + 1, t0, st) {
    if (k.at(c, which, l + 1, q, false)) {
      skip = l >= c.mg_rep[k.r].y;
      Ff = view<T>(c, which, k.r, l);
    }
    if (skip) continue;
    restrict_residual_at<T>(Ff, k.F, q - k.lo);
  }
}

template <typename T, bool MULTI>
__global__ void __launch_bounds__(kMgThreads) k_mg_restrict(Ctx c, int which, int l) {
  HCA_VC_ENTRY(c);
  restrict_sites<T, MULTI>(c, which, l, grid_t0(), grid_st());
}

// One of the sweeps of smooth_at over the sites of grid level l.
template <typename T, bool MULTI, int MODE>
__device__ __forceinline__ void smooth_sites(const Ctx& c, int which, int l, long long t0, long long st) {
  if (!MULTI) {
    const View<T> F = view<T>(c, which, 0, l), C = view<T>(c, which, 0, l + 1);
    for (long long s = t0; s < F.n(); s += st) smooth_at<T, MODE>(F, C, s);
    return;
  }
  RepCursor<T> k;
  bool skip = true;
  HCA_MG_FOR_SITES_FROM(l, t0, st) {
    if (k.at(c, which, l, q, true)) skip = l >= c.mg_rep[k.r].y;
    if (skip) continue;
    smooth_at<T, MODE>(k.F, k.C, q - k.lo);
  }
}

template <typename T, bool MULTI, int MODE>
__global__ void __launch_bounds__(kMgThreads) k_mg_smooth(Ctx c, int which, int l) {
  HCA_VC_ENTRY(c);
  smooth_sites<T, MULTI, MODE>(c, which, l, grid_t0(), grid_st());
}

// Replicate owning item q of a prefix table (the last r with pre[r] <= q).
__device__ __forceinline__ int rep_of_items(const long long* pre, int n, long long q) {
  int lo = 0, hi = n;
  while (hi - lo > 1) {
    const int mid = (lo + hi) >> 1;
    if (pre[mid] <= q) lo = mid;
    else hi = mid;
  }
  return lo;
}

// The sweeps of smooth_at on grid level l >= 1 in row-vector form (every
// replicate's level rows a whole number of 4-site groups; items of a batch
// found through the level's prefix table): one thread per group; every load
// of the group (the arrays that form u on its row and the four neighbour
// rows, the sites left and right of it, the row's rhs, 1/d and d, for
// SM_POST the level-(l+1) correction under each row) is issued before u is
// formed.  The same arithmetic, in the same order, as smooth_at.
template <typename T, int MODE>
__device__ __forceinline__ void smooth_rows(const Ctx& c, int which, int l, long long t0, long long st) {
  const long long* pre = c.mg_post_items + (long long)l * (c.n_reps + 1);
  const long long items = pre[c.n_reps];
  int r = -1;
  long long lo = 0, hi = 0;
  View<T> F, C;
  int gpr = 1;
  for (long long qq = t0; qq < items; qq += st) {
    if (qq < lo || qq >= hi) {   // the replicate changes rarely along a thread's items
      r = rep_of_items(pre, c.n_reps, qq);
      lo = pre[r];
      hi = pre[r + 1];
      F = view<T>(c, which, r, l);
      C = view<T>(c, which, r, l + 1);
      gpr = F.nx >> 2;
    }
    const long long q = qq - lo;
    const int j = (int)(q % gpr);
    const long long R = q / gpr;
    const int Y = (int)(R % F.ny), Z = (int)(R / F.ny);
    const int X0 = 4 * j;
    const long long e = F.at(X0, Y, Z);
    const bool rok[5] = {true, Y > 0, Y < F.ny - 1, Z > 0, Z < F.nz - 1};
    const long long roff[5] = {0, -F.sy, F.sy, -F.sz, F.sz};
    const bool has_l = j > 0, has_r = j + 1 < gpr;
    V4<T> U[5], RH0, W0;
    T ul, ur;
    const V4<T> D = ld4(F.d + e);
    if (MODE == SM_PRE) {
      V4<T> RH[5], WV[5];
#pragma unroll
      for (int t = 0; t < 5; ++t) {
        RH[t] = ld4_if(F.rhs + e + roff[t], rok[t]);
        WV[t] = ld4_if(F.w + e + roff[t], rok[t]);
      }
      const T wl = has_l ? F.w[e - 1] : T(0), rl = has_l ? F.rhs[e - 1] : T(0);
      const T wr = has_r ? F.w[e + 4] : T(0), rr = has_r ? F.rhs[e + 4] : T(0);
#pragma unroll
      for (int t = 0; t < 5; ++t)
#pragma unroll
        for (int k = 0; k < 4; ++k) U[t].a[k] = rok[t] ? mul_rn(wt(MG_W1, WV[t].a[k]), RH[t].a[k]) : T(0);
      ul = has_l ? mul_rn(wt(MG_W1, wl), rl) : T(0);
      ur = has_r ? mul_rn(wt(MG_W1, wr), rr) : T(0);
      RH0 = RH[0];
      W0 = WV[0];
    } else {
      const T* src = MODE == SM_POST ? F.x : F.t;
      const int ry[5] = {Y, Y - 1, Y + 1, Y, Y};
      const int rz[5] = {Z, Z, Z, Z - 1, Z + 1};
      V4<T> XV[5];
      T C0[5], C1[5];
#pragma unroll
      for (int t = 0; t < 5; ++t) {
        XV[t] = ld4_if(src + e + roff[t], rok[t]);
        if (MODE == SM_POST) {
          const long long cb = rok[t] ? C.at(2 * j, ry[t] >> 1, rz[t] >> 1) : 0;
          C0[t] = rok[t] ? C.x[cb] : T(0);
          C1[t] = rok[t] ? C.x[cb + 1] : T(0);
        }
      }
      RH0 = ld4(F.rhs + e);
      W0 = ld4(F.w + e);
      const T xl = has_l ? src[e - 1] : T(0), xr = has_r ? src[e + 4] : T(0);
      if (MODE == SM_POST) {
        const long long cy = C.at(0, Y >> 1, Z >> 1);
        const T cl = has_l ? C.x[cy + 2 * j - 1] : T(0), cr = has_r ? C.x[cy + 2 * j + 2] : T(0);
#pragma unroll
        for (int t = 0; t < 5; ++t)
#pragma unroll
          for (int k = 0; k < 4; ++k) U[t].a[k] = rok[t] ? XV[t].a[k] + (k < 2 ? C0[t] : C1[t]) : T(0);
        ul = has_l ? xl + cl : T(0);
        ur = has_r ? xr + cr : T(0);
      } else {
#pragma unroll
        for (int t = 0; t < 5; ++t) U[t] = rok[t] ? XV[t] : zero4<T>();
        ul = xl;
        ur = xr;
      }
    }
    V4<T> Xo;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      T nb = T(0);
      if (k > 0 || has_l) nb += k > 0 ? U[0].a[k - 1] : ul;
      if (k < 3 || has_r) nb += k < 3 ? U[0].a[k + 1] : ur;
      if (rok[1]) nb += U[1].a[k];
      if (rok[2]) nb += U[2].a[k];
      if (rok[3]) nb += U[3].a[k];
      if (rok[4]) nb += U[4].a[k];
      const T uc = U[0].a[k];
      const T res = resid(RH0.a[k], D.a[k], uc, F.c, nb);
      Xo.a[k] = fma(wt(MODE == SM_LAST ? MG_W1 : MG_W2, W0.a[k]), res, uc);
    }
    *reinterpret_cast<V4<T>*>((MODE == SM_POST ? F.t : F.x) + e) = Xo;
  }
}

template <typename T, int MODE>
__global__ void __launch_bounds__(kMgThreads) k_mg_smooth_rows(Ctx c, int which, int l) {
  HCA_VC_ENTRY(c);
  smooth_rows<T, MODE>(c, which, l, grid_t0(), grid_st());
}

// Restriction of the pre-smoothed residual from grid level l >= 1 to l + 1
// in row-vector form (every replicate's level-l rows whole 4-site groups;
// batches as in k_mg_smooth_rows): one thread per group of the four fine rows
// (2Y + dy, 2Z + dz) under coarse row (Y, Z), producing coarse sites 2j,
// 2j + 1; all loads of a dz half (x on its 2 own and 6 outer rows, rhs and d
// on the own rows, the x neighbours at the group's ends) are issued before
// its residuals are formed.  The same arithmetic, children in the same order,
// as restrict_residual_at.
template <typename T>
__device__ __forceinline__ void restrict_rows(const Ctx& c, int which, int l, long long t0, long long st) {
  const long long* pre = c.mg_restr_items + (long long)l * (c.n_reps + 1);
  const long long items = pre[c.n_reps];
  int r = -1;
  long long lo = 0, hi = 0;
  View<T> F, C;
  int gpr = 1;
  for (long long qq = t0; qq < items; qq += st) {
    if (qq < lo || qq >= hi) {
      r = rep_of_items(pre, c.n_reps, qq);
      lo = pre[r];
      hi = pre[r + 1];
      F = view<T>(c, which, r, l);
      C = view<T>(c, which, r, l + 1);
      gpr = F.nx >> 2;
    }
    const long long q = qq - lo;
    const int j = (int)(q % gpr);
    const long long R = q / gpr;
    const int Y = (int)(R % C.ny), Z = (int)(R / C.ny);
    const int y0 = 2 * Y, z0 = 2 * Z, x0 = 4 * j;
    const long long eb = F.at(x0, y0, z0);
    const bool hasl = x0 > 0, hasr = x0 + 4 < F.nx;
    const bool y1 = y0 + 1 < F.ny;
    T acc[2] = {T(0), T(0)};
    // children in the order of restrict_residual_at (dz outer, dy, dx inner),
    // one dz half b at a time: slots 0, 1 the half's own rows (y0, y0 + 1),
    // 2, 3 rows y0 - 1 and y0 + 2, 4, 5 the other half's own rows, 6, 7 the
    // outer z row (z0 - 1 or z0 + 2) under y0, y0 + 1
#pragma unroll
    for (int b = 0; b < 2; ++b) {
      if (z0 + b >= F.nz) break;
      const int ob = 1 - b;
      const bool zo = b ? z0 + 2 < F.nz : z0 > 0;
      const long long zoff = b ? 2 * F.sz : -F.sz;
      const bool ok[8] = {true, y1, y0 > 0, y0 + 2 < F.ny, z0 + ob < F.nz, y1 && z0 + ob < F.nz, zo, zo && y1};
      const long long off[8] = {F.sz * b, F.sy + F.sz * b, -F.sy + F.sz * b, 2 * F.sy + F.sz * b,
                                F.sz * ob, F.sy + F.sz * ob, zoff, F.sy + zoff};
      V4<T> XV[8], RV[2], DV[2];
#pragma unroll
      for (int t = 0; t < 8; ++t) XV[t] = ld4_if(F.x + eb + off[t], ok[t]);
#pragma unroll
      for (int t = 0; t < 2; ++t) {
        RV[t] = ld4_if(F.rhs + eb + off[t], ok[t]);
        DV[t] = ld4_if(F.d + eb + off[t], ok[t]);
      }
      T xl[2], xr[2];
#pragma unroll
      for (int t = 0; t < 2; ++t) {
        xl[t] = (ok[t] && hasl) ? F.x[eb + off[t] - 1] : T(0);
        xr[t] = (ok[t] && hasr) ? F.x[eb + off[t] + 4] : T(0);
      }
#pragma unroll
      for (int a = 0; a < 2; ++a) {
        if (!ok[a]) continue;
        const int ym = a ? 0 : 2, yp = a ? 3 : 1;           // rows y - 1, y + 1
        const int zm = b ? 4 + a : 6 + a, zp = b ? 6 + a : 4 + a;  // rows z - 1, z + 1
#pragma unroll
        for (int e = 0; e < 4; ++e) {
          const int x = x0 + e;
          T nb = T(0);
          if (x > 0) nb += e == 0 ? xl[a] : XV[a].a[e - 1];
          if (x < F.nx - 1) nb += e == 3 ? xr[a] : XV[a].a[e + 1];
          if (y0 + a > 0) nb += XV[ym].a[e];
          if (y0 + a < F.ny - 1) nb += XV[yp].a[e];
          if (z0 + b > 0) nb += XV[zm].a[e];
          if (z0 + b < F.nz - 1) nb += XV[zp].a[e];
          acc[e >> 1] += resid(RV[a].a[e], DV[a].a[e], XV[a].a[e], F.c, nb);
        }
      }
    }
    const long long cb = C.at(2 * j, Y, Z);
    C.rhs[cb] = acc[0];
    C.rhs[cb + 1] = acc[1];
  }
}

template <typename T>
__global__ void __launch_bounds__(128) k_mg_restrict_rows(Ctx c, int which, int l) {
  HCA_VC_ENTRY(c);
  restrict_rows<T>(c, which, l, grid_t0(), grid_st());
}

// Item q of the lattice's row-vector kernels (one thread per 4-site group of
// the fine rows 2Y, 2Y + 1 x 2Z, 2Z + 1 under level-1 row (Y, Z), items of a
// batch through the prefix table mg_rowstart): its replicate, level 1 and
// fine geometry.
struct Item0 {
  int r, j, Y, Z, y0, z0, x0;
  long long sy, sz, eb;
};
__device__ __forceinline__ Item0 item0(const Ctx& c, long long q) {
  Item0 I;
  int lo = 0, hi = c.n_reps;
  while (hi - lo > 1) {
    const int mid = (lo + hi) >> 1;
    if (c.mg_rowstart[mid] <= q) lo = mid;
    else hi = mid;
  }
  I.r = lo;
  const RepDesc& rd = c.reps[I.r];
  const MGLevel& L1 = ((const MGLevel*)c.mg_lv)[I.r * MG_MAXLEV + 1];
  const long long it = q - c.mg_rowstart[I.r];
  I.j = (int)(it % rd.gpr);
  const long long R = it / rd.gpr;
  I.Y = (int)(R % L1.ny);
  I.Z = (int)(R / L1.ny);
  I.sy = rd.nxp;
  I.sz = (long long)rd.nxp * rd.ny;
  I.y0 = 2 * I.Y;
  I.z0 = 2 * I.Z;
  I.x0 = 4 * I.j;
  I.eb = rd.off + (long long)I.x0 + I.sy * I.y0 + I.sz * I.z0;   // fine (x0, y0, z0)
  return I;
}

// The two pre-smoothing sweeps from zero at one site, shared by the row and
// plane-marching forms (every product rounded on its own, so both give the
// same bits): u = (W1 / d) r at every site; with nb the sum of the six
// neighbours' u (order x-, x+, y-, y+, z-, z+), v = u + (W2 / d)(r - A u)
// where the diagonal term d u is taken as W1 r (equal up to the rounding of
// 1/d), so d is not read.
template <typename T>
__device__ __forceinline__ T pre0_u(T r, T w) {
  return mul_rn(wt(MG_W1, w), r);
}
template <typename T>
__device__ __forceinline__ T pre0_site(T r, T w, T u, T cpl, T nb) {
  const T du = w != T(0) ? mul_rn((T)MG_W1, r) : T(0);
  const T res = r - (du - mul_rn(cpl, nb));
  return fma(wt(MG_W2, w), res, u);
}

// Both pre-smoothing sweeps on the lattice in row-vector form (pre0_site),
// stored into dst (the z buffer, free until the last post-sweep): r and 1/d,
// 8 B per site.  Every load of an item (its four own rows, their eight outer
// neighbour rows, the x neighbours at the group's ends) is issued before u is
// formed.
template <typename T>
__global__ void __launch_bounds__(128, 5) k_mg_pre0(Ctx c, int which, T* __restrict__ dst) {
  HCA_VC_ENTRY(c);
  const T* __restrict__ rr = (const T*)c.r;
  const T* __restrict__ ww = (const T*)c.mg_w;
  const long long total = c.mg_rowstart[c.n_reps];
  for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < total;
       q += (long long)gridDim.x * blockDim.x) {
    const Item0 I = item0(c, q);
    const RepDesc& rd = c.reps[I.r];
    const long long sy = I.sy, sz = I.sz, eb = I.eb;
    const int y0 = I.y0, z0 = I.z0, x0 = I.x0;
    const T cpl = op_coupling_t<T>(rd, which);
    const bool hasl = x0 > 0, hasr = x0 + 4 < rd.nx;
    const bool y1 = y0 + 1 < rd.ny;
    // one dz half b at a time with its eight rows in registers: slots 0, 1
    // the half's own rows (y0, y0 + 1), 2, 3 rows y0 - 1 and y0 + 2, 4, 5 the
    // other half's own rows, 6, 7 the outer z row (z0 - 1 or z0 + 2) under y0, y0 + 1
#pragma unroll
    for (int b = 0; b < 2; ++b) {
      if (z0 + b >= rd.nz) break;
      const int ob = 1 - b;
      const bool zo = b ? z0 + 2 < rd.nz : z0 > 0;
      const long long zoff = b ? 2 * sz : -sz;
      const bool ok[8] = {true, y1, y0 > 0, y0 + 2 < rd.ny, z0 + ob < rd.nz, y1 && z0 + ob < rd.nz, zo, zo && y1};
      const long long off[8] = {sz * b, sy + sz * b, -sy + sz * b, 2 * sy + sz * b, sz * ob, sy + sz * ob, zoff,
                                sy + zoff};
      V4<T> RV[8], WV[8];
#pragma unroll
      for (int t = 0; t < 8; ++t) {
        RV[t] = ld4_if(rr + eb + off[t], ok[t]);
        WV[t] = ld4_if(ww + eb + off[t], ok[t]);
      }
      T lr[2], lw[2], rrr[2], rw[2];
#pragma unroll
      for (int t = 0; t < 2; ++t) {
        lr[t] = (ok[t] && hasl) ? rr[eb + off[t] - 1] : T(0);
        lw[t] = (ok[t] && hasl) ? ww[eb + off[t] - 1] : T(0);
        rrr[t] = (ok[t] && hasr) ? rr[eb + off[t] + 4] : T(0);
        rw[t] = (ok[t] && hasr) ? ww[eb + off[t] + 4] : T(0);
      }
      // u = (W1 / d) r (zero outside the lattice: w = 0 on padding and missing rows)
      V4<T> U[8];
#pragma unroll
      for (int t = 0; t < 8; ++t)
#pragma unroll
        for (int e = 0; e < 4; ++e) U[t].a[e] = (x0 + e < rd.nx) ? pre0_u(RV[t].a[e], WV[t].a[e]) : T(0);
#pragma unroll
      for (int a = 0; a < 2; ++a) {
        if (!ok[a]) continue;
        const V4<T>& ymr = a ? U[0] : U[2];                 // row y - 1
        const V4<T>& ypr = a ? U[3] : U[1];                 // row y + 1
        const V4<T>& zmr = b ? U[4 + a] : U[6 + a];         // row z - 1
        const V4<T>& zpr = b ? U[6 + a] : U[4 + a];         // row z + 1
        const T ul = pre0_u(lr[a], lw[a]), ur = pre0_u(rrr[a], rw[a]);
        V4<T> VO = zero4<T>();   // zero on padding
#pragma unroll
        for (int e = 0; e < 4; ++e) {
          const int x = x0 + e;
          if (x >= rd.nx) continue;
          const T left = e == 0 ? ul : U[a].a[e - 1];
          const T right = e == 3 ? ur : U[a].a[e + 1];
          const T nb = (x > 0 ? left : T(0)) + (x < rd.nx - 1 ? right : T(0)) + ymr.a[e] + ypr.a[e] + zmr.a[e] + zpr.a[e];
          VO.a[e] = pre0_site(RV[a].a[e], WV[a].a[e], U[a].a[e], cpl, nb);
        }
        st4(dst + eb + off[a], VO);
      }
    }
  }
}

// Plane-marching form of k_mg_pre0 for one FP32 lattice.  A block owns a
// tile of kZmG four-site groups by kZmY rows and a slab of planes, and walks
// up z: each thread keeps its group's u on planes z - 1, z and z + 1 in
// registers, and u on plane z of the tile with a one-site halo goes to
// shared memory (two buffers, one barrier per plane) for the x and y
// neighbours.  So r and 1/d are read once per site (the halo's from L2), and
// the loads of plane z + 2 are in flight during plane z's arithmetic.
// Threads 0 .. 2 kZmG - 1 also load the two halo rows (groups), the next
// 2 kZmY threads the halo sites at the tile's x ends.  Per site the
// arithmetic is k_mg_pre0's (pre0_site, same neighbour order).
constexpr int kZmG = 8, kZmY = 16, kZmThreads = kZmG * kZmY;
constexpr int kZmPitch = 4 * kZmG + 8;   // tile row in shared memory: left halo at 3, groups from 4, right halo at 4 + 4 kZmG

__global__ void __launch_bounds__(kZmThreads, 7) k_mg_pre0_z(Ctx c, int which, float* __restrict__ dst, int zs) {
  HCA_VC_ENTRY(c);
  __shared__ __align__(16) float ub[2][kZmY + 2][kZmPitch];
  const RepDesc& rd = c.reps[0];
  const float* __restrict__ rr = (const float*)c.r;
  const float* __restrict__ ww = (const float*)c.mg_w;
  const float cpl = op_coupling_t<float>(rd, which);
  const int t = threadIdx.x, g = t % kZmG, ty = t / kZmG;
  const int G = blockIdx.x * kZmG + g, y = blockIdx.y * kZmY + ty;
  const int x0 = 4 * G;
  const bool own = G < rd.gpr && y < rd.ny;
  const long long sy = rd.nxp, sz = (long long)rd.nxp * rd.ny;
  const long long eo = rd.off + x0 + sy * y;
  // halo role: 1 a group of halo row y0 - 1 or y0 + kZmY, 2 a site at x0 - 1 or x0 + 4 kZmG
  int hrole = 0, hrow = 0, hcol = 0, hx = 0;
  bool hok = false;
  long long he = 0;
  if (t < 2 * kZmG) {
    hrole = 1;
    const int hy = blockIdx.y * kZmY + (t < kZmG ? -1 : kZmY), hg = blockIdx.x * kZmG + t % kZmG;
    hok = hy >= 0 && hy < rd.ny && hg < rd.gpr;
    he = rd.off + 4LL * hg + sy * hy;
    hx = 4 * hg;
    hrow = t < kZmG ? 0 : kZmY + 1;
    hcol = 4 + 4 * (t % kZmG);
  } else if (t < 2 * kZmG + 2 * kZmY) {
    hrole = 2;
    const int k = t - 2 * kZmG, side = k / kZmY, row = k % kZmY;
    hx = side ? 4 * kZmG * (blockIdx.x + 1) : 4 * kZmG * blockIdx.x - 1;
    const int hy = blockIdx.y * kZmY + row;
    hok = hx >= 0 && hx < rd.nx && hy < rd.ny;
    he = rd.off + hx + sy * hy;
    hrow = row + 1;
    hcol = side ? 4 + 4 * kZmG : 3;
  }
  const int zb = blockIdx.z * zs, ze = min(rd.nz, zb + zs);
  auto ld_own = [&](int z, V4<float>& R, V4<float>& W) {
    const bool ok = own && z >= 0 && z < rd.nz;
    R = ld4_if(rr + eo + sz * z, ok);
    W = ld4_if(ww + eo + sz * z, ok);
  };
  auto ld_halo = [&](int z, V4<float>& R, V4<float>& W) {
    const bool ok = hok && z >= 0 && z < rd.nz;
    if (hrole == 1) {
      R = ld4_if(rr + he + sz * z, ok);
      W = ld4_if(ww + he + sz * z, ok);
    } else {
      R.a[0] = (hrole == 2 && ok) ? rr[he + sz * z] : 0.f;
      W.a[0] = (hrole == 2 && ok) ? ww[he + sz * z] : 0.f;
    }
  };
  auto u_of = [&](const V4<float>& R, const V4<float>& W, int xb) {
    V4<float> U;
#pragma unroll
    for (int e = 0; e < 4; ++e) U.a[e] = (xb + e < rd.nx) ? pre0_u(R.a[e], W.a[e]) : 0.f;
    return U;
  };
  // u of plane z (own group and halo role) into buffer z & 1
  auto put = [&](int z, const V4<float>& U, const V4<float>& HR, const V4<float>& HW) {
    float* row = &ub[z & 1][ty + 1][4 + 4 * g];
    *reinterpret_cast<float4*>(row) = make_float4(U.a[0], U.a[1], U.a[2], U.a[3]);
    if (hrole == 1) {
      const V4<float> H = u_of(HR, HW, hx);
      *reinterpret_cast<float4*>(&ub[z & 1][hrow][hcol]) = make_float4(H.a[0], H.a[1], H.a[2], H.a[3]);
    } else if (hrole == 2) {
      ub[z & 1][hrow][hcol] = pre0_u(HR.a[0], HW.a[0]);
    }
  };
  V4<float> Rc, Wc, Rn, Wn, HRn, HWn, up, uc;
  {
    V4<float> Rp, Wp, HRc, HWc;
    ld_own(zb - 1, Rp, Wp);
    ld_own(zb, Rc, Wc);
    ld_halo(zb, HRc, HWc);
    ld_own(zb + 1, Rn, Wn);
    ld_halo(zb + 1 < ze ? zb + 1 : -1, HRn, HWn);
    up = u_of(Rp, Wp, x0);
    uc = u_of(Rc, Wc, x0);
    put(zb, uc, HRc, HWc);
  }
  __syncthreads();
  for (int z = zb; z < ze; ++z) {
    V4<float> Rnn, Wnn, HRnn, HWnn;
    ld_own(z + 2 <= ze ? z + 2 : -1, Rnn, Wnn);
    ld_halo(z + 2 < ze ? z + 2 : -1, HRnn, HWnn);
    const V4<float> un = u_of(Rn, Wn, x0);   // plane z + 1 (zero above the lattice)
    if (z + 1 < ze) put(z + 1, un, HRn, HWn);
    const float* mid = &ub[z & 1][ty + 1][4 + 4 * g];
    const float4 ym = *reinterpret_cast<const float4*>(mid - kZmPitch);
    const float4 yp = *reinterpret_cast<const float4*>(mid + kZmPitch);
    const float lft = mid[-1], rgt = mid[4];
    if (own) {
      const float ymv[4] = {ym.x, ym.y, ym.z, ym.w}, ypv[4] = {yp.x, yp.y, yp.z, yp.w};
      V4<float> VO = zero4<float>();   // zero on padding
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        const int x = x0 + e;
        if (x >= rd.nx) continue;
        const float left = e == 0 ? lft : uc.a[e - 1];
        const float right = e == 3 ? rgt : uc.a[e + 1];
        const float nb = (x > 0 ? left : 0.f) + (x < rd.nx - 1 ? right : 0.f) + ymv[e] + ypv[e] + up.a[e] + un.a[e];
        VO.a[e] = pre0_site(Rc.a[e], Wc.a[e], uc.a[e], cpl, nb);
      }
      st4(dst + eo + sz * z, VO);
    }
    up = uc;
    uc = un;
    Rc = Rn;
    Wc = Wn;
    Rn = Rnn;
    Wn = Wnn;
    HRn = HRnn;
    HWn = HWnn;
    __syncthreads();
  }
}

// Plane-marching form of k_mg_smooth_rows<float, MODE> on grid level l >= 1
// of one FP32 lattice: the fused pre-sweeps (SM_PRE: u = (W1 / d) rhs formed
// at every site, x = u + (W2 / d)(rhs - A u)), the prolongation fused with
// the first post-sweep (SM_POST: u = x + P x_C formed at every site, t = u +
// (W2 / d)(rhs - A u)) and the last post-sweep (SM_LAST: u = t, x = t +
// (W1 / d)(rhs - A t)).  The tiles, slabs, halo
// roles and register prefetch of k_mg_pre0_z; the level's rows are whole
// four-site groups.  Per site the row form's arithmetic: the neighbours'
// u summed in the order x - 1, x + 1, y - 1, y + 1, z - 1, z + 1 (only those
// inside the level), resid and one fused multiply-add.
template <int MODE>
__global__ void __launch_bounds__(kZmThreads, 7) k_mg_smooth_z(Ctx c, int which, int l, int zs) {
  HCA_VC_ENTRY(c);
  __shared__ __align__(16) float ub[2][kZmY + 2][kZmPitch];
  const View<float> F = view<float>(c, which, 0, l);
  const int gpr = F.nx >> 2;
  const int t = threadIdx.x, g = t % kZmG, ty = t / kZmG;
  const int G = blockIdx.x * kZmG + g, y = blockIdx.y * kZmY + ty;
  const int x0 = 4 * G;
  const bool own = G < gpr && y < F.ny;
  const long long sy = F.sy, sz = F.sz;
  const long long eo = x0 + sy * y;
  // u's source: rhs (with 1/d), x (plus the coarse correction) or t
  const float* __restrict__ ua = MODE == SM_PRE ? F.rhs : MODE == SM_POST ? F.x : F.t;
  const View<float> C = view<float>(c, which, 0, MODE == SM_POST ? l + 1 : l);
  // the coarse correction P x_C at fine (x, y, z): level l + 1's value of its cell
  auto pxc = [&](int x, int yy, int z) {
    return C.x[(x >> 1) + (long long)C.nx * ((yy >> 1) + (long long)C.ny * (z >> 1))];
  };
  int hrole = 0, hrow = 0, hcol = 0, hx = 0, hy = 0;
  bool hok = false;
  long long he = 0;
  if (t < 2 * kZmG) {
    hrole = 1;
    hy = blockIdx.y * kZmY + (t < kZmG ? -1 : kZmY);
    const int hg = blockIdx.x * kZmG + t % kZmG;
    hok = hy >= 0 && hy < F.ny && hg < gpr;
    hx = 4 * hg;
    he = 4LL * hg + sy * hy;
    hrow = t < kZmG ? 0 : kZmY + 1;
    hcol = 4 + 4 * (t % kZmG);
  } else if (t < 2 * kZmG + 2 * kZmY) {
    hrole = 2;
    const int k = t - 2 * kZmG, side = k / kZmY, row = k % kZmY;
    hx = side ? 4 * kZmG * (blockIdx.x + 1) : 4 * kZmG * blockIdx.x - 1;
    hy = blockIdx.y * kZmY + row;
    hok = hx >= 0 && hx < F.nx && hy < F.ny;
    he = hx + sy * hy;
    hrow = row + 1;
    hcol = side ? 4 + 4 * kZmG : 3;
  }
  const int zb = blockIdx.z * zs, ze = min(F.nz, zb + zs);
  auto u_of = [&](const V4<float>& A, const V4<float>& W) {
    if (MODE != SM_PRE) return A;
    V4<float> U;
#pragma unroll
    for (int e = 0; e < 4; ++e) U.a[e] = mul_rn(wt(MG_W1, W.a[e]), A.a[e]);
    return U;
  };
  // u of a group (x0 = 4 G, row yy) with both of its coarse cells
  auto u_post = [&](const V4<float>& A, int xg, int yy, int z, bool ok) {
    V4<float> U = zero4<float>();
    if (ok) {
      const float c0 = pxc(xg, yy, z), c1 = pxc(xg + 2, yy, z);
#pragma unroll
      for (int e = 0; e < 4; ++e) U.a[e] = A.a[e] + (e < 2 ? c0 : c1);
    }
    return U;
  };
  // u of the own group on plane z (0 outside the level)
  auto u_own = [&](int z) {
    const bool ok = own && z >= 0 && z < F.nz;
    const V4<float> A = ld4_if(ua + eo + sz * z, ok);
    if (MODE == SM_POST) return u_post(A, x0, y, z, ok);
    const V4<float> W = MODE == SM_PRE ? ld4_if(F.w + eo + sz * z, ok) : A;
    return u_of(A, W);
  };
  auto u_halo = [&](int z) {
    const bool ok = hok && z >= 0 && z < ze;
    V4<float> A = zero4<float>(), W = zero4<float>();
    if (hrole == 1) {
      A = ld4_if(ua + he + sz * z, ok);
      if (MODE == SM_POST) return u_post(A, hx, hy, z, ok);
      if (MODE == SM_PRE) W = ld4_if(F.w + he + sz * z, ok);
    } else if (hrole == 2 && ok) {
      A.a[0] = ua[he + sz * z];
      if (MODE == SM_POST) A.a[0] = A.a[0] + pxc(hx, hy, z);
      if (MODE == SM_PRE) W.a[0] = F.w[he + sz * z];
    }
    if (MODE == SM_POST) return A;
    return u_of(A, W);
  };
  auto put = [&](int z, const V4<float>& U, const V4<float>& H) {
    *reinterpret_cast<float4*>(&ub[z & 1][ty + 1][4 + 4 * g]) = make_float4(U.a[0], U.a[1], U.a[2], U.a[3]);
    if (hrole == 1) *reinterpret_cast<float4*>(&ub[z & 1][hrow][hcol]) = make_float4(H.a[0], H.a[1], H.a[2], H.a[3]);
    else if (hrole == 2) ub[z & 1][hrow][hcol] = H.a[0];
  };
  auto ld_site = [&](const float* a, int z) { return ld4_if(a + eo + sz * z, own && z < ze); };
  V4<float> up = u_own(zb - 1), uc = u_own(zb), un = u_own(zb + 1);
  V4<float> Rc = ld_site(F.rhs, zb), Dc = ld_site(F.d, zb), Wc = ld_site(F.w, zb);
  V4<float> Hn = u_halo(zb + 1);
  put(zb, uc, u_halo(zb));
  __syncthreads();
  for (int z = zb; z < ze; ++z) {
    const V4<float> unn = u_own(z + 2 <= ze ? z + 2 : -1);
    const V4<float> Hnn = u_halo(z + 2);
    const V4<float> Rn = ld_site(F.rhs, z + 1), Dn = ld_site(F.d, z + 1), Wn = ld_site(F.w, z + 1);
    if (z + 1 < ze) put(z + 1, un, Hn);
    if (own) {
      const float* mid = &ub[z & 1][ty + 1][4 + 4 * g];
      const float4 a = *reinterpret_cast<const float4*>(mid - kZmPitch);
      const float4 b = *reinterpret_cast<const float4*>(mid + kZmPitch);
      const float ym[4] = {a.x, a.y, a.z, a.w}, yp[4] = {b.x, b.y, b.z, b.w};
      const float lft = mid[-1], rgt = mid[4];
      V4<float> Xo;
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        const int x = x0 + k;
        float nb = 0.f;
        if (x > 0) nb += k > 0 ? uc.a[k - 1] : lft;
        if (x < F.nx - 1) nb += k < 3 ? uc.a[k + 1] : rgt;
        if (y > 0) nb += ym[k];
        if (y < F.ny - 1) nb += yp[k];
        if (z > 0) nb += up.a[k];
        if (z < F.nz - 1) nb += un.a[k];
        const float u0 = uc.a[k];
        const float res = resid(Rc.a[k], Dc.a[k], u0, F.c, nb);
        Xo.a[k] = fmaf(wt(MODE == SM_LAST ? MG_W1 : MG_W2, Wc.a[k]), res, u0);
      }
      *reinterpret_cast<V4<float>*>((MODE == SM_POST ? F.t : F.x) + eo + sz * z) = Xo;
    }
    up = uc;
    uc = un;
    un = unn;
    Rc = Rn;
    Dc = Dn;
    Wc = Wn;
    Hn = Hnn;
    __syncthreads();
  }
}

// TMA form of the plane-marching pre-sweeps (same tiles, slabs and
// per-site arithmetic as k_mg_pre0_z).  One thread issues, per plane, two
// tensor copies (r and 1/d) of the box x0 - 4 .. x0 + 4 kZmG + 3 by
// y0 - 1 .. y0 + kZmY into one of kTmStages shared-memory stages, completing
// on the stage's mbarrier; the copy engine fills sites outside the lattice
// with zeros, so the halo needs no bounds checks.  A plane is consumed
// kTmStages - 2 planes after its copy was issued; a stage is refilled after
// the block barrier that follows its last use.  Waits are bounded: on a
// timeout the block records SYNC_ERR_TIMEOUT, waits (bounded) for its copies
// in flight and returns.
constexpr int kTmW = 4 * kZmG + 8, kTmH = kZmY + 2;
constexpr int kTmPlane = kTmW * kTmH;                      // floats per array and plane
constexpr int kTmPlaneF = ((kTmPlane * 4 + 127) / 128) * 32;  // stage slot in floats (128-byte multiple)
constexpr int kTmStages = 4;
constexpr int kTmSmem = kTmStages * 2 * kTmPlaneF * 4 + 128;
constexpr int kTmWaitLimit = 1 << 20;

__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(tc::smem_u32(bar)), "r"(bytes)
               : "memory");
}
__device__ __forceinline__ void tma_load_3d(float* sdst, const CUtensorMap* map, int x, int y, int z, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], [%5];" ::
          "r"(tc::smem_u32(sdst)),
      "l"((unsigned long long)map), "r"(x), "r"(y), "r"(z), "r"(tc::smem_u32(bar))
      : "memory");
}

__global__ void __launch_bounds__(kZmThreads, 7)
    k_mg_pre0_t(Ctx c, int which, float* __restrict__ dst, int zs, const __grid_constant__ CUtensorMap tm_r,
                const __grid_constant__ CUtensorMap tm_w) {
  HCA_VC_ENTRY(c);
  extern __shared__ __align__(128) float tsm_raw[];
  __shared__ __align__(8) uint64_t bar[kTmStages];
  // stage slots start on a 128-byte boundary (the launch adds 128 bytes)
  float* tsm = reinterpret_cast<float*>((reinterpret_cast<uintptr_t>(tsm_raw) + 127) & ~uintptr_t(127));
  const RepDesc& rd = c.reps[0];
  const float cpl = op_coupling_t<float>(rd, which);
  const int t = threadIdx.x, g = t % kZmG, ty = t / kZmG;
  const int G = blockIdx.x * kZmG + g, y = blockIdx.y * kZmY + ty;
  const int x0 = 4 * G;
  const bool own = G < rd.gpr && y < rd.ny;
  const long long sy = rd.nxp, sz = (long long)rd.nxp * rd.ny;
  const long long eo = rd.off + x0 + sy * y;
  const int zb = blockIdx.z * zs, ze = min(rd.nz, zb + zs);
  const int bx = 4 * kZmG * blockIdx.x - 4, by = kZmY * blockIdx.y - 1;
  const int nk = ze - zb + 2;   // planes zb - 1 .. ze, plane p at k = p - zb + 1
  if (t == 0) {
    for (int s = 0; s < kTmStages; ++s) tc::mbar_init(&bar[s], 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  }
  __syncthreads();
  auto slot = [&](int k, int a) { return tsm + (2 * (k % kTmStages) + a) * kTmPlaneF; };
  auto issue = [&](int k) {
    uint64_t* b = &bar[k % kTmStages];
    mbar_expect_tx(b, 2 * kTmPlane * 4);
    tma_load_3d(slot(k, 0), &tm_r, bx, by, zb - 1 + k, b);
    tma_load_3d(slot(k, 1), &tm_w, bx, by, zb - 1 + k, b);
  };
  auto ready = [&](int k) { return tc::mbar_wait(&bar[k % kTmStages], (uint32_t)((k / kTmStages) & 1), kTmWaitLimit); };
  int issued = min(kTmStages, nk);
  if (t == 0)
    for (int k = 0; k < issued; ++k) issue(k);
  // own group in a box: row ty + 1, columns 4 + 4 g ..
  const int oc = (ty + 1) * kTmW + 4 + 4 * g;
  auto own4 = [&](int k, int a) {
    const float4 v = *reinterpret_cast<const float4*>(slot(k, a) + oc);
    V4<float> r;
    r.a[0] = v.x;
    r.a[1] = v.y;
    r.a[2] = v.z;
    r.a[3] = v.w;
    return r;
  };
  auto u_of = [&](const V4<float>& R, const V4<float>& W) {
    V4<float> U;
#pragma unroll
    for (int e = 0; e < 4; ++e) U.a[e] = (x0 + e < rd.nx) ? pre0_u(R.a[e], W.a[e]) : 0.f;
    return U;
  };
  bool ok = ready(0);
  ok = ready(1) && ok;
  V4<float> up, uc, Rc, Wc;
  if (ok) {
    up = u_of(own4(0, 0), own4(0, 1));
    Rc = own4(1, 0);
    Wc = own4(1, 1);
    uc = u_of(Rc, Wc);
  }
  bool failed = false;   // the same in every thread of the block
  for (int z = zb;; ++z) {
    const bool more = z < ze;
    if (more && ok) ok = ready(z - zb + 2);
    // one decision per block: every thread stops together on a timeout
    if (__syncthreads_or(!ok)) {
      failed = true;
      break;
    }
    if (!more) break;
    const int k = z - zb + 1;
    // every thread is past plane z - 1: its stage takes plane k - 1 + kTmStages
    if (t == 0 && k - 1 + kTmStages < nk) {
      issue(k - 1 + kTmStages);
      issued = k + kTmStages;
    }
    const V4<float> Rn = own4(k + 1, 0), Wn = own4(k + 1, 1);
    const V4<float> un = u_of(Rn, Wn);   // plane z + 1 (zero above the lattice)
    if (own) {
      const float* br = slot(k, 0) + oc;
      const float* bw = slot(k, 1) + oc;
      const float4 ymr = *reinterpret_cast<const float4*>(br - kTmW), ymw = *reinterpret_cast<const float4*>(bw - kTmW);
      const float4 ypr = *reinterpret_cast<const float4*>(br + kTmW), ypw = *reinterpret_cast<const float4*>(bw + kTmW);
      const float ymv[4] = {pre0_u(ymr.x, ymw.x), pre0_u(ymr.y, ymw.y), pre0_u(ymr.z, ymw.z), pre0_u(ymr.w, ymw.w)};
      const float ypv[4] = {pre0_u(ypr.x, ypw.x), pre0_u(ypr.y, ypw.y), pre0_u(ypr.z, ypw.z), pre0_u(ypr.w, ypw.w)};
      const float lft = pre0_u(br[-1], bw[-1]), rgt = pre0_u(br[4], bw[4]);
      V4<float> VO = zero4<float>();   // zero on padding
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        const int x = x0 + e;
        if (x >= rd.nx) continue;
        const float left = e == 0 ? lft : uc.a[e - 1];
        const float right = e == 3 ? rgt : uc.a[e + 1];
        const float nb = (x > 0 ? left : 0.f) + (x < rd.nx - 1 ? right : 0.f) + ymv[e] + ypv[e] + up.a[e] + un.a[e];
        VO.a[e] = pre0_site(Rc.a[e], Wc.a[e], uc.a[e], cpl, nb);
      }
      st4(dst + eo + sz * z, VO);
    }
    up = uc;
    uc = un;
    Rc = Rn;
    Wc = Wn;
  }
  if (failed) {
    // a copy did not complete in time: record it, and let this block's
    // copies in flight land before its shared memory is released
    if (t == 0) {
      c.sync->error = SYNC_ERR_TIMEOUT;
      for (int k = max(0, issued - kTmStages); k < issued; ++k) (void)ready(k);
    }
    __syncthreads();
  }
}

// One site of the lattice's restriction sweep, shared by the row and
// plane-marching forms: with rn = r + c sum_nb v, the residual r - A v =
// rn - d v (one fused multiply-add) and the first post-sweep's part
// v + (W2 / d)(r - A v) = (1 - W2) v + W2 rn / d (0 where d = 0).
template <typename T>
__device__ __forceinline__ T restrict0_res(T rn, T d, T v) {
  return fma(-d, v, rn);
}
template <typename T>
__device__ __forceinline__ T restrict0_vp(T rn, T d, T v) {
  return d != T(0) ? fma((T)MG_W2, rn / d, mul_rn((T)(1.0 - MG_W2), v)) : T(0);
}

// Restriction from the lattice to level 1 in row-vector form, from the
// pre-smoothed iterate v (src, stored by k_mg_pre0): rhs_1 = R (r - A v).  It
// also stores v' = v + (W2 / d)(r - A v) = (1 - W2) v + W2 (r + c sum_nb v) / d
// into mg_t0, the part of the first post-sweep that does not depend on the
// coarse correction (the post-sweep kernel adds the rest).  Per item and dz
// half: v on the 2 own and 6 outer rows, r and d on the own rows, the x
// neighbours of v at the group's ends, all loaded before the residuals are
// formed: 16.5 B per site.  Children in the order of restrict_residual_at.
template <typename T>
__global__ void __launch_bounds__(128, 4) k_mg_restrict0_rows(Ctx c, int which, const T* __restrict__ src) {
  HCA_VC_ENTRY(c);
  T* __restrict__ vo = (T*)c.mg_t0;
  const T* __restrict__ rr = (const T*)c.r;
  const T* __restrict__ dd = (const T*)c.d;
  const MGLevel* LV = (const MGLevel*)c.mg_lv;
  const long long total = c.mg_rowstart[c.n_reps];
  for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < total;
       q += (long long)gridDim.x * blockDim.x) {
    const Item0 I = item0(c, q);
    const RepDesc& rd = c.reps[I.r];
    const MGLevel& L1 = LV[I.r * MG_MAXLEV + 1];
    const long long sy = I.sy, sz = I.sz, eb = I.eb;
    const int y0 = I.y0, z0 = I.z0, x0 = I.x0;
    const T cpl = op_coupling_t<T>(rd, which);
    const bool hasl = x0 > 0, hasr = x0 + 4 < rd.nx;
    const bool y1 = y0 + 1 < rd.ny;
    T acc0 = T(0), acc1 = T(0);
#pragma unroll
    for (int b = 0; b < 2; ++b) {
      if (z0 + b >= rd.nz) break;
      const int ob = 1 - b;
      const bool zo = b ? z0 + 2 < rd.nz : z0 > 0;
      const long long zoff = b ? 2 * sz : -sz;
      const bool ok[8] = {true, y1, y0 > 0, y0 + 2 < rd.ny, z0 + ob < rd.nz, y1 && z0 + ob < rd.nz, zo, zo && y1};
      const long long off[8] = {sz * b, sy + sz * b, -sy + sz * b, 2 * sy + sz * b, sz * ob, sy + sz * ob, zoff,
                                sy + zoff};
      V4<T> XV[8], RV[2], DV[2];
#pragma unroll
      for (int t = 0; t < 8; ++t) XV[t] = ld4_if(src + eb + off[t], ok[t]);
#pragma unroll
      for (int t = 0; t < 2; ++t) {
        RV[t] = ld4_if(rr + eb + off[t], ok[t]);
        DV[t] = ld4_if(dd + eb + off[t], ok[t]);
      }
      T xl[2], xr[2];
#pragma unroll
      for (int t = 0; t < 2; ++t) {
        xl[t] = (ok[t] && hasl) ? src[eb + off[t] - 1] : T(0);
        xr[t] = (ok[t] && hasr) ? src[eb + off[t] + 4] : T(0);
      }
#pragma unroll
      for (int a = 0; a < 2; ++a) {
        if (!ok[a]) continue;
        const V4<T>& ymr = a ? XV[0] : XV[2];                 // row y - 1
        const V4<T>& ypr = a ? XV[3] : XV[1];                 // row y + 1
        const V4<T>& zmr = b ? XV[4 + a] : XV[6 + a];         // row z - 1
        const V4<T>& zpr = b ? XV[6 + a] : XV[4 + a];         // row z + 1
        V4<T> VO = zero4<T>();   // zero on padding
#pragma unroll
        for (int e = 0; e < 4; ++e) {
          const int x = x0 + e;
          if (x >= rd.nx) continue;
          const T left = e == 0 ? xl[a] : XV[a].a[e - 1];
          const T right = e == 3 ? xr[a] : XV[a].a[e + 1];
          const T nb = (x > 0 ? left : T(0)) + (x < rd.nx - 1 ? right : T(0)) + ymr.a[e] + ypr.a[e] + zmr.a[e] + zpr.a[e];
          const T rn = fma(cpl, nb, RV[a].a[e]);   // r + c sum_nb v
          const T res = restrict0_res(rn, DV[a].a[e], XV[a].a[e]);
          if (e < 2) acc0 += res;
          else acc1 += res;
          VO.a[e] = restrict0_vp(rn, DV[a].a[e], XV[a].a[e]);
        }
        st4(vo + eb + off[a], VO);
      }
    }
    T* rhs1 = (T*)L1.rhs;
    const long long cb = ((long long)I.Z * L1.ny + I.Y) * L1.nx + 2 * I.j;
    if (2 * I.j < L1.nx) rhs1[cb] = acc0;
    if (2 * I.j + 1 < L1.nx) rhs1[cb + 1] = acc1;
  }
}

// The view of single-block level l of replicate r with its arrays in the
// block's shared memory `sm` (levels l0 .. l packed one after another, five
// arrays x, t, rhs, d, w of n_l elements each), or in global memory when sm
// is null.
template <typename T, bool SMEM>
__device__ __forceinline__ View<T> small_view(const Ctx& c, int which, int r, int l0, int l, T* sm) {
  View<T> v = view<T>(c, which, r, l);
  if (!SMEM) return v;
  long long o = 0;
  for (int k = l0; k < l; ++k) o += 5 * ((const MGLevel*)c.mg_lv)[r * MG_MAXLEV + k].n;
  const long long n = v.n();
  v.x = sm + o;
  v.t = sm + o + n;
  v.rhs = sm + o + 2 * n;
  v.d = sm + o + 3 * n;
  v.w = sm + o + 4 * n;
  return v;
}

// Asynchronous copies (cp.async) from global to shared memory.
template <int B>
__device__ __forceinline__ void cp_async(void* sdst, const void* gsrc) {
  const unsigned sa = (unsigned)__cvta_generic_to_shared(sdst);
  asm volatile("cp.async.ca.shared.global [%0], [%1], %2;" ::"r"(sa), "l"(gsrc), "n"(B) : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;" ::: "memory"); }

// Start copying the diagonals and 1/d of replicate r's single-block
// levels into shared memory (they do not change during a V-cycle); the copies
// complete in the background until cp_async_wait_all.
template <typename T>
__device__ void small_prefetch(const Ctx& c, int which, int r, int tid, int nthr, T* sm) {
  const int l0 = c.mg_rep[r].y, last = c.mg_rep[r].x - 1;
  for (int l = l0; l <= last; ++l) {
    const View<T> G = view<T>(c, which, r, l), V = small_view<T, true>(c, which, r, l0, l, sm);
    const int n = (int)V.n();
    for (int s = tid; s < n; s += nthr) {
      cp_async<sizeof(T)>(V.d + s, G.d + s);
      cp_async<sizeof(T)>(V.w + s, G.w + s);
    }
  }
}

// The whole sub-cycle of replicate r's levels small .. nlev-1 by one block
// (tid, nthr: this thread and the block's threads; block barriers between
// sweeps).  With sm, the cycle runs in shared memory (the same arithmetic in
// the same order as in global memory): the diagonals and 1/d of those
// levels are copied in (already under way when `prefetched`), then the
// right-hand side of the first level; afterwards the first level's iterate,
// the only array later kernels read, is written back.
template <typename T, bool SMEM>
__device__ void small_cycle(const Ctx& c, int which, int r, int tid, int nthr, T* sm, bool prefetched) {
  const int l0 = c.mg_rep[r].y, last = c.mg_rep[r].x - 1;
  if (SMEM) {
    if (!prefetched) small_prefetch<T>(c, which, r, tid, nthr, sm);
    const View<T> G = view<T>(c, which, r, l0), V = small_view<T, true>(c, which, r, l0, l0, sm);
    const int n = (int)V.n();
    // all loads of a batch before its stores (the copies may not be reordered
    // across the stores to shared memory otherwise)
    for (int base = tid; base < n; base += 8 * nthr) {
      T v[8];
#pragma unroll
      for (int k = 0; k < 8; ++k) {
        const int s = base + k * nthr;
        v[k] = s < n ? G.rhs[s] : T(0);
      }
#pragma unroll
      for (int k = 0; k < 8; ++k) {
        const int s = base + k * nthr;
        if (s < n) V.rhs[s] = v[k];
      }
    }
    cp_async_wait_all();
    __syncthreads();
  }
  for (int l = l0; l < last; ++l) {
    // pre-smoothing: t = (W1 / d) rhs, x = t + (W2 / d)(rhs - A t); rhs_C = R (rhs - A x)
    const View<T> V = small_view<T, SMEM>(c, which, r, l0, l, sm);
    const int n = (int)V.n();
    for (int s = tid; s < n; s += nthr) sweep_first_at<T>(V, V.t, s, MG_W1);
    __syncthreads();
    {
      Walk w(tid, nthr, V.nx, V.ny);
      for (int s = tid; s < n; s += nthr, w.next()) sweep_xyz<T>(V, V.t, V.x, w.X, w.Y, w.Z, s, MG_W2);
    }
    __syncthreads();
    const View<T> C = small_view<T, SMEM>(c, which, r, l0, l + 1, sm);
    const int nc = (int)C.n();
    Walk w(tid, nthr, C.nx, C.ny);
    for (int s = tid; s < nc; s += nthr, w.next()) restrict_residual_xyz<T>(V, C, w.X, w.Y, w.Z, s);
    __syncthreads();
  }
  {
    const View<T> V = small_view<T, SMEM>(c, which, r, l0, last, sm);
    const int n = (int)V.n();
    for (int s = tid; s < n; s += nthr) sweep_first_at<T>(V, V.x, s, MG_OMEGA_COARSE);
    __syncthreads();
    for (int k = 1; k < MG_NU_COARSE; ++k) {
      const bool odd = k & 1;
      Walk w(tid, nthr, V.nx, V.ny);
      for (int s = tid; s < n; s += nthr, w.next())
        sweep_xyz<T>(V, odd ? V.x : V.t, odd ? V.t : V.x, w.X, w.Y, w.Z, s, MG_OMEGA_COARSE);
      __syncthreads();
    }
    if ((MG_NU_COARSE & 1) == 0) {   // the last sweep wrote t
      for (int s = tid; s < n; s += nthr) V.x[s] = V.t[s];
      __syncthreads();
    }
  }
  for (int l = last - 1; l >= l0; --l) {
    // x += P x_C, then t = x + (W2 / d)(rhs - A x), x = t + (W1 / d)(rhs - A t)
    const View<T> V = small_view<T, SMEM>(c, which, r, l0, l, sm);
    const View<T> C = small_view<T, SMEM>(c, which, r, l0, l + 1, sm);
    const int n = (int)V.n();
    {
      Walk w(tid, nthr, V.nx, V.ny);
      for (int s = tid; s < n; s += nthr, w.next()) prolong_xyz<T>(V, C, w.X, w.Y, w.Z, s);
    }
    __syncthreads();
    {
      Walk w(tid, nthr, V.nx, V.ny);
      for (int s = tid; s < n; s += nthr, w.next()) sweep_xyz<T>(V, V.x, V.t, w.X, w.Y, w.Z, s, MG_W2);
    }
    __syncthreads();
    {
      Walk w(tid, nthr, V.nx, V.ny);
      for (int s = tid; s < n; s += nthr, w.next()) sweep_xyz<T>(V, V.t, V.x, w.X, w.Y, w.Z, s, MG_W1);
    }
    __syncthreads();
  }
  if (SMEM) {
    const View<T> G = view<T>(c, which, r, l0), V = small_view<T, true>(c, which, r, l0, l0, sm);
    const int n = (int)V.n();
    for (int s = tid; s < n; s += nthr) G.x[s] = V.x[s];
  }
}

// The sub-cycle of the single-block levels, one block per replicate, in
// global memory.
template <typename T>
__global__ void __launch_bounds__(kSmallThreads) k_mg_small(Ctx c, int which) {
  HCA_VC_ENTRY(c);
  small_cycle<T, false>(c, which, blockIdx.x, threadIdx.x, blockDim.x, nullptr, false);
}

// The same sub-cycle with the single-block levels in the block's dynamic
// shared memory (the same arithmetic in the same order).
template <typename T>
__global__ void __launch_bounds__(kSmallThreads) k_mg_small_smem(Ctx c, int which) {
  HCA_VC_ENTRY(c);
  extern __shared__ __align__(16) unsigned char small_smem[];
  small_cycle<T, true>(c, which, blockIdx.x, threadIdx.x, blockDim.x, (T*)small_smem, false);
}

// ------------------------------------- coarse levels in one cooperative launch --
// Levels lo .. nlev-1 of one V-cycle in one cooperative launch: the
// pre-sweeps and restrictions l -> l + 1 for l = lo .. small-1, the
// single-block sub-cycle (block b takes replicates b, b + grid, ...; its
// levels in dynamic shared memory when small_smem > 0), then the two
// post-sweeps of l = small-1 .. lo, with a grid barrier between consecutive
// phases.  Each phase is the loop body of
// the corresponding per-level kernel over this launch's threads, so the
// result is bit-identical to the per-level launches.  rows_ok: bit l selects
// the row-vector form of level l (as for the per-level kernels).
template <typename T, int NT, int MINB>
__global__ void __launch_bounds__(NT, MINB) k_mg_coarse(Ctx c, int which, int lo, int small, unsigned rows_ok,
                                                         int use_smem) {
  HCA_VC_ENTRY(c);
  extern __shared__ __align__(16) unsigned char mg_smem[];
  T* sm = (T*)mg_smem;
  const long long t0 = grid_t0(), st = grid_st();
  const bool multi = c.n_reps > 1;
  if (*(volatile int*)&c.sync->error == SYNC_ERR_TIMEOUT) return;
  // the single-block levels' constant arrays start moving into shared memory
  // while the restrictions run
  const bool pre = use_smem && blockIdx.x < c.n_reps;
  if (pre) small_prefetch<T>(c, which, blockIdx.x, threadIdx.x, blockDim.x, sm);
  int k = 0;
  for (int l = lo; l < small; ++l) {
    const bool rows = rows_ok >> l & 1u;
    if (rows) smooth_rows<T, SM_PRE>(c, which, l, t0, st);
    else if (multi) smooth_sites<T, true, SM_PRE>(c, which, l, t0, st);
    else smooth_sites<T, false, SM_PRE>(c, which, l, t0, st);
    if (!grid_barrier(c.sync, k++)) return;
    if (rows) restrict_rows<T>(c, which, l, t0, st);
    else if (multi) restrict_sites<T, true>(c, which, l, t0, st);
    else restrict_sites<T, false>(c, which, l, t0, st);
    if (!grid_barrier(c.sync, k++)) return;
  }
  for (int r = blockIdx.x; r < c.n_reps; r += gridDim.x) {
    if (use_smem) small_cycle<T, true>(c, which, r, threadIdx.x, blockDim.x, sm, pre && r == (int)blockIdx.x);
    else small_cycle<T, false>(c, which, r, threadIdx.x, blockDim.x, nullptr, false);
    __syncthreads();
  }
  if (!grid_barrier(c.sync, k++)) return;
  for (int l = small - 1; l >= lo; --l) {
    const bool rows = rows_ok >> l & 1u;
    if (rows) smooth_rows<T, SM_POST>(c, which, l, t0, st);
    else if (multi) smooth_sites<T, true, SM_POST>(c, which, l, t0, st);
    else smooth_sites<T, false, SM_POST>(c, which, l, t0, st);
    if (!grid_barrier(c.sync, k++)) return;
    if (rows) smooth_rows<T, SM_LAST>(c, which, l, t0, st);
    else if (multi) smooth_sites<T, true, SM_LAST>(c, which, l, t0, st);
    else smooth_sites<T, false, SM_LAST>(c, which, l, t0, st);
    if (l > lo && !grid_barrier(c.sync, k++)) return;
  }
  grid_exit(c.sync, k);
}

// ------------------------------------------ level-0 post-smoothing + rho --
// PROLONG: the first post-sweep of u = v + p, p = P x_1 the coarse correction
// and v the pre-smoothed iterate.  With v' = v + (W2 / d)(r - A v), stored
// by the restriction kernel in mg_t0, and (1 / d) d = 1,
//   y = u + (W2 / d)(r - A u) = v' + (1 - W2) p + (W2 / d) c sum_nb p,
// so the kernel streams v' and 1/d, reads p from the coarse level (piecewise
// constant: three of a site's neighbours share its coarse cell) and writes y
// over v' in place (each site reads and writes only its own element).
// Otherwise: z = u + (om / d)(r - A u) = (1 - om) u + (om / d)(r + c sum_nb u)
// with u = src, into z (the second post-sweep, om = W1, or the last sweep of
// the coarsest level, om = MG_OMEGA_COARSE, when the lattice is the coarsest
// level): reads u, r and 1/d, 16 B per site with the write; then rho = r.z with the fixed-order reductions
// of the CG passes and beta = rho / rho_old (0 on the first application of a
// solve).
template <typename T, bool PROLONG, int NI, bool PERSIST = false>
__global__ void __maxnreg__(64) k_mg_post0(Ctx c, int which, const T* __restrict__ src, T om) {
  HCA_VC_ENTRY(c);
  const int2 ch = PERSIST ? make_int2(0, 0) : c.chunks[blockIdx.x];
  const RepDesc& rd = c.reps[ch.x];
  const int nrows = min(rd.chunk_rows, rd.ny * rd.nz - ch.y);
  const T* __restrict__ rr = (const T*)c.r;
  const T* __restrict__ ww = (const T*)c.mg_w;
  T* yy = (T*)c.mg_t0;   // read and written in place by PROLONG
  T* __restrict__ zz = (T*)c.z;
  const T cpl = op_coupling_t<T>(rd, which);
  const T* __restrict__ x1 = nullptr;
  int nx1 = 0, ny1 = 0;
  if (PROLONG) {
    const MGLevel& L1 = ((const MGLevel*)c.mg_lv)[ch.x * MG_MAXLEV + 1];
    x1 = (const T*)L1.x;
    nx1 = L1.nx;
    ny1 = L1.ny;
  }
  const RowIter it = row_iter(rd);
  // one row j (chunk slot rl of `chunk`; row_ok false: a padding slot of the last chunk)
  auto row = [&](int chunk, int rl, bool row_ok, int j) {
    const RowGeo geo = row_geo(rd, j);
    const int y = j % rd.ny, z = j / rd.ny;
    LaneAcc<T> acc[1];
    // groups per lane in a row: a compile-time count (NI > 0) lets the
    // compiler issue the loads of all of them before the first is used
    const int niter = NI > 0 ? NI : it.niter;
    if (PROLONG) {
      // coarse rows of the site row and of its y and z neighbours outside
      // its coarse cell; in-cell neighbours (one along y, one along z, where
      // inside the lattice) carry the site's own p
      const int yo = (y & 1) ? y + 1 : y - 1, zo = (z & 1) ? z + 1 : z - 1;
      const bool yout = yo >= 0 && yo < rd.ny, zout = zo >= 0 && zo < rd.nz;
      const T nin = (T)(int)(((y & 1) || y + 1 < rd.ny) + ((z & 1) || z + 1 < rd.nz));
      const long long cown = ((long long)(z >> 1) * ny1 + (y >> 1)) * nx1;
      const long long cy = yout ? ((long long)(z >> 1) * ny1 + (yo >> 1)) * nx1 : cown;
      const long long cz = zout ? ((long long)(zo >> 1) * ny1 + (y >> 1)) * nx1 : cown;
#pragma unroll
      for (int itn = 0; itn < niter; ++itn) {
        const int g = itn * it.lpr + it.sl;
        const bool gok = row_ok && g < rd.gpr;
        const long long e = geo.base + 4LL * g;
        const bool two = 4 * g + 2 < rd.nx;   // the group reaches coarse cell 2g + 1
        const V4<T> V = ld4_if(yy + e, gok);
        const V4<T> W = ld4_if(ww + e, gok);
        const T C0 = gok ? x1[cown + 2 * g] : T(0);
        const T C1 = gok && two ? x1[cown + 2 * g + 1] : T(0);
        const T Cl = gok && g > 0 ? x1[cown + 2 * g - 1] : T(0);
        const T Cr = gok && 4 * g + 4 < rd.nx ? x1[cown + 2 * g + 2] : T(0);
        const T Y0 = gok && yout ? x1[cy + 2 * g] : T(0);
        const T Y1 = gok && yout && two ? x1[cy + 2 * g + 1] : T(0);
        const T Z0 = gok && zout ? x1[cz + 2 * g] : T(0);
        const T Z1 = gok && zout && two ? x1[cz + 2 * g + 1] : T(0);
        if (gok) {
          V4<T> Yo;
#pragma unroll
          for (int k = 0; k < 4; ++k) {
            Yo.a[k] = T(0);
            const int x = 4 * g + k;
            if (x < rd.nx && W.a[k] != T(0)) {
              const T p = k < 2 ? C0 : C1;
              const T pl = x > 0 ? (k == 0 ? Cl : k < 3 ? C0 : C1) : T(0);
              const T pr = x < rd.nx - 1 ? (k == 3 ? Cr : k == 0 ? C0 : C1) : T(0);
              const T nb = ((pl + pr) + mul_rn(nin, p)) + ((k < 2 ? Y0 : Y1) + (k < 2 ? Z0 : Z1));
              Yo.a[k] = fma(wt(MG_W2, W.a[k]), cpl * nb, fma((T)(1.0 - MG_W2), p, V.a[k]));
            }
          }
          st4(yy + e, Yo);
        }
      }
    } else {
      T carry = T(0);
      const T om1 = T(1) - om;
#pragma unroll
      for (int itn = 0; itn < niter; ++itn) {
        const int g = itn * it.lpr + it.sl;
        const bool gok = row_ok && g < rd.gpr;
        const long long e = geo.base + 4LL * g;
        const bool rok[5] = {gok, gok && geo.ym, gok && geo.yp, gok && geo.zm, gok && geo.zp};
        const long long roff[5] = {0, -geo.sy, geo.sy, -geo.sz, geo.sz};
        V4<T> UU[5];
#pragma unroll
        for (int q = 0; q < 5; ++q) UU[q] = ld4_if(src + e + roff[q], rok[q]);
        const V4<T> R = ld4_if(rr + e, gok);
        const V4<T> W = ld4_if(ww + e, gok);
        const bool last_lane = it.sl == it.lpr - 1 && gok && g + 1 < rd.gpr;
        const T un = last_lane ? src[e + 4] : T(0);
        const V4<T>& U = UU[0];
        T left, right;
        x_neighbours(U, g, rd.gpr, it.sl, it.lpr, gok, carry, left, right, [&] { return un; });
        if (gok) {
          V4<T> Zo;
          T rz = T(0);
#pragma unroll
          for (int k = 0; k < 4; ++k) {
            Zo.a[k] = T(0);
            if (4 * g + k < rd.nx && W.a[k] != T(0)) {
              // u + (om / d)(r - A u) = (1 - om) u + (om / d)(r + c sum_nb u)
              const T rn = fma(cpl, nb_sum(U, k, left, right, UU[1], UU[2], UU[3], UU[4]), R.a[k]);
              Zo.a[k] = fma(om * W.a[k], rn, om1 * U.a[k]);
              rz += R.a[k] * Zo.a[k];
            }
          }
          st4(zz + e, Zo);
          acc[0].add(rz);   // float-float lane sums for FP32 (r is scaled to O(1))
        }
      }
    }
    if (!PROLONG) store_rows_acc(c, chunk, rl, row_ok, it.sl, it.lpr, acc, 1);
  };
  if (PERSIST) {
    const int R = rd.ny * rd.nz, cr = rd.chunk_rows;
    for (int j = persist_row_begin(R) + it.warp; j < persist_row_end(R); j += it.nw) row(j / cr, j % cr, true, j);
  } else {
    for (int rbase = it.warp * it.rpw; rbase < rd.chunk_rows; rbase += it.nw * it.rpw) {
      const int rl = rbase + it.sub;
      const bool row_ok = rl < nrows;
      row(blockIdx.x, rl, row_ok, ch.y + (row_ok ? rl : 0));
    }
  }
  if (PROLONG) return;
  auto fin = [&](int r, const double* s1) -> int {
    RepSolve& s = c.solve[r];
    if (!s.active) return 0;
    if (!(s1[0] > 0.0) || !isfinite(s1[0])) {
      if (!isfinite(s1[0])) c.sync->error = 1;
      s.active = 0;
      return 0;
    }
    s.beta = s.iters == 0 ? 0.0 : s1[0] / s.rho;
    s.rho = s1[0];
    return 1;
  };
  // float-float row slots for FP32 fields (LaneAcc<float>)
  if (PERSIST) block_arrivals<sizeof(T) == 4>(c, 1, fin, [](int) {});
  else warp_epilogue<sizeof(T) == 4>(c, 1, blockIdx.x, fin);
}

// Launch shapes of the cooperative coarse-level kernel: 0 = 256 threads with
// up to 255 registers (one block per SM), 1 = 256 threads, 128 registers (two
// blocks per SM), 2 = 512 threads, 128 registers (one block per SM).
template <typename T>
const void* coarse_fn(int cfg) {
  return cfg == 1 ? (const void*)k_mg_coarse<T, 256, 2>
                  : cfg == 2 ? (const void*)k_mg_coarse<T, 512, 1> : (const void*)k_mg_coarse<T, 256, 1>;
}
inline int coarse_threads(int cfg) { return cfg == 2 ? 512 : 256; }

int grid_for(long long n) {
  const long long b = (n + kMgThreads - 1) / kMgThreads;
  return (int)std::max(1LL, std::min(b, 152LL * 16));
}

// One of the lattice's post-sweep kernels (k_mg_post0), in the persistent
// row form when the handle uses it.
template <typename T, bool PROLONG>
void launch_post0(const Ctx& c, int which, const MGHost& H, const T* src, T om) {
  cudaStream_t s = c.stream;
  const bool pdl = c.pdl != 0;
  if (c.persist && (H.ni == 1 || H.ni == 2 || H.ni == 4)) {
    const void* fn = H.ni == 1   ? (const void*)k_mg_post0<T, PROLONG, 1, true>
                     : H.ni == 2 ? (const void*)k_mg_post0<T, PROLONG, 2, true>
                                 : (const void*)k_mg_post0<T, PROLONG, 4, true>;
    const dim3 g(persist_grid(fn, c.threads, c.sm_count));
    switch (H.ni) {
      case 1: launch_k(pdl, k_mg_post0<T, PROLONG, 1, true>, g, dim3(c.threads), 0, s, c, which, src, om); break;
      case 2: launch_k(pdl, k_mg_post0<T, PROLONG, 2, true>, g, dim3(c.threads), 0, s, c, which, src, om); break;
      default: launch_k(pdl, k_mg_post0<T, PROLONG, 4, true>, g, dim3(c.threads), 0, s, c, which, src, om); break;
    }
    return;
  }
  const dim3 g(c.n_chunks);
  switch (H.ni) {
    case 1: launch_k(pdl, k_mg_post0<T, PROLONG, 1>, g, dim3(c.threads), 0, s, c, which, src, om); break;
    case 2: launch_k(pdl, k_mg_post0<T, PROLONG, 2>, g, dim3(c.threads), 0, s, c, which, src, om); break;
    case 4: launch_k(pdl, k_mg_post0<T, PROLONG, 4>, g, dim3(c.threads), 0, s, c, which, src, om); break;
    default: launch_k(pdl, k_mg_post0<T, PROLONG, 0>, g, dim3(c.threads), 0, s, c, which, src, om); break;
  }
}

// Level l >= 1 sweeps in plane-marching form (one FP32 lattice; configured
// by mg_zmarch_config).
template <typename T>
bool zlevel(const MGHost& H, int l) {
  return std::is_same<T, float>::value && l < MG_MAXLEV && H.zl_slabs[l] > 0 && (H.rows_ok >> l & 1u);
}

// part: -1 = whole cycle; 0 = r scaling (only with `scale`: right after a
// residual was formed, i.e. at the start of a solve or a defect-correction
// sweep); 1 = the lattice's pre-sweeps; 2 = its restriction; 3 = the coarse
// levels; 4 = the lattice's prolongation and first post-sweep; 5 = its last
// post-sweep with r.z.  A lattice that is the coarsest level runs its sweeps
// as part 3.
template <typename T>
void vcycle_t(const Ctx& c, int which, const MGHost& H, int part, bool scale) {
  cudaStream_t s = c.stream;
  T* t0 = (T*)c.mg_t0;
  T* z = (T*)c.z;
  const bool all = part < 0;
  const bool multi = c.n_reps > 1;
  if (scale && (all || part == 0)) {
    if (c.n_reps == 1)
      launch_k(c.pdl != 0, k_mg_scale0_rows<T>, dim3(grid_for(H.ntot[0] / 4 + 1)), dim3(kMgThreads), 0, s, c);
    else
      launch_k(c.pdl != 0, k_mg_scale0<T>, dim3(grid_for(H.ntot[0])), dim3(kMgThreads), 0, s, c, which);
  }
  if (H.nlev == 1) {
    if (!all && part != 3) return;
    // the lattice is the coarsest level (single replicate): MG_NU_COARSE
    // sweeps, the last one in post0
    k_mg_first0<T><<<grid_for(H.ntot[0]), kMgThreads, 0, s>>>(c, which);
    for (int k = 1; k < MG_NU_COARSE - 1; ++k) {
      const bool odd = k & 1;
      k_mg_sweep0<T><<<grid_for(H.ntot[0]), kMgThreads, 0, s>>>(c, which, odd ? t0 : z, odd ? z : t0);
    }
    const T* src = ((MG_NU_COARSE - 2) & 1) ? z : t0;
    k_mg_post0<T, false, 0><<<c.n_chunks, c.threads, 0, s>>>(c, which, src, (T)MG_OMEGA_COARSE);
    return;
  }
  // 128 threads: the lattice kernels keep ~20-28 vector loads per thread in flight
  const int nb = (int)std::max(1LL, std::min((H.nrowitems + 127) / 128, 152LL * 16));
  // register budgets (blocks per SM): 5 for the pre-sweeps (a few spilled
  // registers; measured 71.4 -> 67.6 us at 256^3), 4 for the restriction
  // (61.4 us; 65.5 us with 5)
  const bool pdl = c.pdl != 0;
  if (all || part == 1) {
    if constexpr (std::is_same<T, float>::value) {
      if (H.zm_slabs > 0 && H.zm_mode == 2) {
        launch_k(pdl, k_mg_pre0_t, dim3(H.zm_tx, H.zm_ty, H.zm_slabs), dim3(kZmThreads), (size_t)kTmSmem, s, c, which,
                 z, H.zm_zs, H.zm_map_r, H.zm_map_w);
      } else if (H.zm_slabs > 0) {
        launch_k(pdl, k_mg_pre0_z, dim3(H.zm_tx, H.zm_ty, H.zm_slabs), dim3(kZmThreads), 0, s, c, which, z, H.zm_zs);
      } else {
        launch_k(pdl, k_mg_pre0<T>, dim3(nb), dim3(128), 0, s, c, which, z);
      }
    } else {
      launch_k(pdl, k_mg_pre0<T>, dim3(nb), dim3(128), 0, s, c, which, z);
    }
  }
  if (all || part == 2) launch_k(pdl, k_mg_restrict0_rows<T>, dim3(nb), dim3(128), 0, s, c, which, (const T*)z);
  if (all || part == 3) {
    // levels 1 .. lo-1 by per-level kernels, lo .. nlev-1 in the cooperative
    // launch when there is one (lo = small: no level in it but the
    // single-block ones, which then run in their own kernel)
    const bool coop = H.coop_blocks > 0 && H.coop_from < H.small;
    const int lo = coop ? H.coop_from : H.small;
    for (int l = 1; l < lo; ++l) {
      if (zlevel<T>(H, l)) {
        launch_k(pdl, k_mg_smooth_z<SM_PRE>, dim3(H.zl_tx[l], H.zl_ty[l], H.zl_slabs[l]), dim3(kZmThreads), 0, s, c,
                 which, l, H.zl_zs[l]);
        launch_k(pdl, k_mg_restrict_rows<T>, dim3((int)std::min((H.restr_items[l] + 127) / 128, 152LL * 16)), dim3(128),
                 0, s, c, which, l);
      } else if (H.rows_ok >> l & 1u) {
        launch_k(pdl, k_mg_smooth_rows<T, SM_PRE>, dim3(grid_for(H.post_items[l])), dim3(kMgThreads), 0, s, c, which, l);
        // 128 threads: ~12 vector loads per thread in flight
        launch_k(pdl, k_mg_restrict_rows<T>, dim3((int)std::min((H.restr_items[l] + 127) / 128, 152LL * 16)), dim3(128),
                 0, s, c, which, l);
      } else if (multi) {
        launch_k(pdl, k_mg_smooth<T, true, SM_PRE>, dim3(grid_for(H.ntot[l])), dim3(kMgThreads), 0, s, c, which, l);
        launch_k(pdl, k_mg_restrict<T, true>, dim3(grid_for(H.ntot[l + 1])), dim3(kMgThreads), 0, s, c, which, l);
      } else {
        launch_k(pdl, k_mg_smooth<T, false, SM_PRE>, dim3(grid_for(H.ntot[l])), dim3(kMgThreads), 0, s, c, which, l);
        launch_k(pdl, k_mg_restrict<T, false>, dim3(grid_for(H.ntot[l + 1])), dim3(kMgThreads), 0, s, c, which, l);
      }
    }
    if (coop) {
      Ctx cc = c;
      int wh = which, l0 = lo, sm = H.small, use = H.small_smem > 0;
      unsigned rows = H.rows_ok;
      void* args[] = {&cc, &wh, &l0, &sm, &rows, &use};
      (void)cudaLaunchCooperativeKernel(coarse_fn<T>(H.coop_cfg), dim3(H.coop_blocks),
                                        dim3(coarse_threads(H.coop_cfg)), args, (size_t)H.small_smem, s);
    } else if (H.small_smem > 0 && H.small_smem_ok) {
      launch_k(pdl, k_mg_small_smem<T>, dim3(c.n_reps), dim3(kSmallThreads), (size_t)H.small_smem, s, c, which);
    } else {
      launch_k(pdl, k_mg_small<T>, dim3(c.n_reps), dim3(kSmallThreads), 0, s, c, which);
    }
    for (int l = lo - 1; l >= 1; --l) {
      if (zlevel<T>(H, l)) {
        launch_k(pdl, k_mg_smooth_z<SM_POST>, dim3(H.zl_tx[l], H.zl_ty[l], H.zl_slabs[l]), dim3(kZmThreads), 0, s, c,
                 which, l, H.zl_zs[l]);
        launch_k(pdl, k_mg_smooth_z<SM_LAST>, dim3(H.zl_tx[l], H.zl_ty[l], H.zl_slabs[l]), dim3(kZmThreads), 0, s, c,
                 which, l, H.zl_zs[l]);
      } else if (H.rows_ok >> l & 1u) {
        launch_k(pdl, k_mg_smooth_rows<T, SM_POST>, dim3(grid_for(H.post_items[l])), dim3(kMgThreads), 0, s, c, which, l);
        launch_k(pdl, k_mg_smooth_rows<T, SM_LAST>, dim3(grid_for(H.post_items[l])), dim3(kMgThreads), 0, s, c, which, l);
      } else if (multi) {
        launch_k(pdl, k_mg_smooth<T, true, SM_POST>, dim3(grid_for(H.ntot[l])), dim3(kMgThreads), 0, s, c, which, l);
        launch_k(pdl, k_mg_smooth<T, true, SM_LAST>, dim3(grid_for(H.ntot[l])), dim3(kMgThreads), 0, s, c, which, l);
      } else {
        launch_k(pdl, k_mg_smooth<T, false, SM_POST>, dim3(grid_for(H.ntot[l])), dim3(kMgThreads), 0, s, c, which, l);
        launch_k(pdl, k_mg_smooth<T, false, SM_LAST>, dim3(grid_for(H.ntot[l])), dim3(kMgThreads), 0, s, c, which, l);
      }
    }
  }
  if (all || part == 4) launch_post0<T, true>(c, which, H, nullptr, T(0));
  if (all || part == 5) launch_post0<T, false>(c, which, H, t0, (T)MG_W1);
}

template <typename T>
void mg_setup_t(const Ctx& c, int which, const MGHost& H, bool w_done) {
  const bool pdl = c.pdl != 0;
  if (!w_done) launch_k(pdl, k_mg_w0<T>, dim3(grid_for(H.ntot[0])), dim3(kMgThreads), 0, c.stream, c, which);
  for (int l = 1; l < H.nlev; ++l)
    launch_k(pdl, k_mg_diag<T>, dim3(grid_for(H.ntot[l])), dim3(kMgThreads), 0, c.stream, c, which, l);
}

// The launch forms of the coarse levels: the single-block levels in shared
// memory when they fit one block's opt-in maximum (else global memory), and
// the geometry of the cooperative coarse-level kernel.
template <typename T>
int coop_config_t(MGHost& H, int sm_count, long long smem_bytes) {
  H.coop_blocks = 0;
  H.small_smem = 0;
  H.small_smem_ok = false;
  int dev = 0, coop = 0, optin = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess) {
    (void)cudaGetLastError();
    return 0;
  }
  const int smem = smem_bytes <= optin ? (int)smem_bytes : 0;
  const char* ss = std::getenv("HCA_MG_SMALL_SMEM");
  if (smem > 0 && !(ss && ss[0] == '0')) {
    if (cudaFuncSetAttribute((const void*)k_mg_small_smem<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem) ==
        cudaSuccess) {
      H.small_smem = smem;
      H.small_smem_ok = true;
    } else {
      (void)cudaGetLastError();
    }
  }
  const char* env = std::getenv("HCA_MG_COOP");
  if ((env && env[0] == '0') || !coop) return 0;
  // launch shape (HCA_MG_COOP_CFG=0, 1, 2 selects another one)
  const char* cs = std::getenv("HCA_MG_COOP_CFG");
  const int cfg = (cs && cs[0] >= '0' && cs[0] <= '2') ? cs[0] - '0' : 0;
  const void* fn = coarse_fn<T>(cfg);
  if (cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, H.small_smem) != cudaSuccess) {
    (void)cudaGetLastError();
    return 0;
  }
  int per_sm = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, coarse_threads(cfg), H.small_smem) != cudaSuccess ||
      per_sm < 1) {
    (void)cudaGetLastError();
    return 0;
  }
  H.coop_blocks = per_sm * sm_count;
  H.coop_cfg = cfg;
  // the first level small enough for the cooperative launch's threads
  // inside graphs (about one 4-site group per thread and level): 2^18 sites
  H.coop_lo = 1;
  while (H.coop_lo < H.small && H.ntot[H.coop_lo] > (1LL << 18)) ++H.coop_lo;
  return 0;
}

}  // namespace

int vcycle_part_launches(const MGHost& H, int part, bool scale);

int vcycle_launches(const MGHost& H, bool scale) {
  int n = 0;
  for (int part = 0; part < kVcycleParts; ++part) n += vcycle_part_launches(H, part, scale);
  return n;
}

// Choose the coarse-level launch form of a hierarchy (after H.small and
// H.rows_ok are known): one cooperative launch when the device supports it
// (HCA_MG_COOP=0 keeps one launch per level).  smem_bytes: the largest
// shared-memory footprint of any replicate's single-block levels.
void mg_coop_config(MGHost& H, bool fp64, int sm_count, long long smem_bytes) {
  if (H.nlev <= 1) {
    H.coop_blocks = 0;
    H.small_smem = 0;
    return;
  }
  if (fp64) coop_config_t<double>(H, sm_count, smem_bytes);
  else coop_config_t<float>(H, sm_count, smem_bytes);
}
// (H.small: the deepest grid-kernel level + 1 over the batch)

// A 3-D tensor map over one lattice array (x extent nx, rows nxp apart),
// box kTmW x kTmH x 1, zero fill outside.  False if the driver entry point is
// missing or the encoding is refused.
bool lattice_map(CUtensorMap* m, const float* base, const RepDesc& rd) {
  using Encode = CUresult (*)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                              const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                              CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);
  static Encode enc = nullptr;
  if (!enc) {
    void* fn = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q) != cudaSuccess ||
        q != cudaDriverEntryPointSuccess || !fn) {
      (void)cudaGetLastError();
      return false;
    }
    enc = (Encode)fn;
  }
  const float* p = base + rd.off;
  if ((reinterpret_cast<uintptr_t>(p) & 15u) || (rd.nxp * 4) % 16) return false;
  const cuuint64_t dims[3] = {(cuuint64_t)rd.nx, (cuuint64_t)rd.ny, (cuuint64_t)rd.nz};
  const cuuint64_t strides[2] = {(cuuint64_t)rd.nxp * 4, (cuuint64_t)rd.nxp * rd.ny * 4};
  const cuuint32_t box[3] = {(cuuint32_t)kTmW, (cuuint32_t)kTmH, 1};
  const cuuint32_t es[3] = {1, 1, 1};
  return enc(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, const_cast<float*>(p), dims, strides, box, es,
             CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
             CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

// Form and geometry of the lattice's pre-sweeps on one FP32 lattice rd
// (arrays r and w): the plane-marching kernel with its planes staged by TMA
// tensor copies (default; the register-prefetch form when the tensor maps
// cannot be made or HCA_MG_ZMARCH=1), or the row form (HCA_MG_ZMARCH=0).
// Tiles of kZmG groups by kZmY rows; the planes split into slabs so that
// the grid is a whole number of waves of resident blocks, at most
// HCA_MG_ZM_WAVES (default 1 for the TMA form, 2 for the register form:
// measured best at 256^3).
void mg_zmarch_config(MGHost& H, const RepDesc& rd, int sm_count, const float* r, const float* w,
                      const int* lv_dims) {
  H.zm_slabs = 0;
  const char* e = std::getenv("HCA_MG_ZMARCH");
  if ((e && e[0] == '0') || H.nlev <= 1) return;
  H.zm_mode = (e && e[0] == '1') ? 1 : 2;
  if (H.zm_mode == 2 && !(lattice_map(&H.zm_map_r, r, rd) && lattice_map(&H.zm_map_w, w, rd))) H.zm_mode = 1;
  const void* fn = H.zm_mode == 2 ? (const void*)k_mg_pre0_t : (const void*)k_mg_pre0_z;
  int per_sm = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, kZmThreads, H.zm_mode == 2 ? kTmSmem : 0) !=
          cudaSuccess ||
      per_sm < 1) {
    (void)cudaGetLastError();
    return;
  }
  const char* wv = std::getenv("HCA_MG_ZM_WAVES");
  const double waves = wv ? std::max(0.05, std::atof(wv)) : (H.zm_mode == 2 ? 1.0 : 2.0);
  H.zm_tx = (rd.gpr + kZmG - 1) / kZmG;
  H.zm_ty = (rd.ny + kZmY - 1) / kZmY;
  const double tiles = (double)H.zm_tx * H.zm_ty;
  const long long want = (long long)(waves * sm_count * per_sm / tiles);   // whole waves at most
  const int slabs = (int)std::max(1LL, std::min((long long)rd.nz, want));
  H.zm_zs = (rd.nz + slabs - 1) / slabs;
  H.zm_slabs = (rd.nz + H.zm_zs - 1) / H.zm_zs;
  // grid levels with whole-group rows: the same tiles, slabs for at most
  // HCA_MG_ZL_WAVES waves (default 1); HCA_MG_ZLEVELS=0 keeps their row form
  const char* zl = std::getenv("HCA_MG_ZLEVELS");
  if (zl && zl[0] == '0') return;
  int per_sm_l = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm_l, (const void*)k_mg_smooth_z<SM_PRE>, kZmThreads, 0) !=
          cudaSuccess ||
      per_sm_l < 1) {
    (void)cudaGetLastError();
    return;
  }
  const char* lw = std::getenv("HCA_MG_ZL_WAVES");
  const double lwaves = lw ? std::max(0.05, std::atof(lw)) : 1.0;
  for (int l = 1; l < std::min(H.small, MG_MAXLEV); ++l) {
    if (!(H.rows_ok >> l & 1u)) continue;
    const int nx = lv_dims[3 * l], ny = lv_dims[3 * l + 1], nz = lv_dims[3 * l + 2];
    if (nx % 4) continue;
    H.zl_tx[l] = (nx / 4 + kZmG - 1) / kZmG;
    H.zl_ty[l] = (ny + kZmY - 1) / kZmY;
    const double tl = (double)H.zl_tx[l] * H.zl_ty[l];
    const long long wl = (long long)(lwaves * sm_count * per_sm_l / tl);
    const int sl = (int)std::max(1LL, std::min((long long)nz, wl));
    H.zl_zs[l] = (nz + sl - 1) / sl;
    H.zl_slabs[l] = (nz + H.zl_zs[l] - 1) / H.zl_zs[l];
  }
}

// w_done: the lattice's 1/d is already in place (the first defect-correction
// residual sweep of an FP32 solve forms it).
void launch_mg_setup(const Ctx& c, int which, bool fp64, const MGHost& H, bool w_done) {
  if (fp64) mg_setup_t<double>(c, which, H, w_done);
  else mg_setup_t<float>(c, which, H, w_done);
}

void launch_vcycle(const Ctx& c, int which, bool fp64, const MGHost& H, int part, bool scale) {
  if (fp64) vcycle_t<double>(c, which, H, part, scale);
  else vcycle_t<float>(c, which, H, part, scale);
}

int vcycle_part_launches(const MGHost& H, int part, bool scale) {
  if (part == 0) return scale ? 1 : 0;
  if (H.nlev == 1) return part == 3 ? MG_NU_COARSE : 0;
  if (part == 3) {
    const int lo = H.coop_blocks > 0 && H.coop_from < H.small ? H.coop_from : H.small;
    return 4 * (lo - 1) + 1;
  }
  return 1;
}

}  // namespace hca
