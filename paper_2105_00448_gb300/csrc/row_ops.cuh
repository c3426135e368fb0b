// Row-segment helpers shared by the kernels that sweep the padded field
// layout: a warp's lanes hold consecutive 4-site groups of one x-row; the x
// neighbours of a group come from lane shuffles.
#pragma once

#include "hca_internal.cuh"

namespace hca {

constexpr unsigned FULL = 0xffffffffu;

template <typename T>
__device__ __forceinline__ V4<T> ld4_if(const T* p, bool ok) {
  return ok ? ld4(p) : zero4<T>();
}

template <typename T>
__device__ __forceinline__ T sel(const V4<T>& v, int k) {
  return v.a[k];
}

// Neighbours of a 4-site group along x.  `v` is this lane's group; lanes of a
// row segment hold consecutive groups.  carry holds the last site of the
// previous iteration's last lane.  right_at() loads the site after the group
// for the segment's last lane.
template <typename T, class RightAt>
__device__ __forceinline__ void x_neighbours(const V4<T>& v, int g, int gpr, int sl, int lpr, bool gok,
                                             T& carry, T& left, T& right, RightAt right_at) {
  const T up = __shfl_up_sync(FULL, v.a[3], 1, lpr);
  const T dn = __shfl_down_sync(FULL, v.a[0], 1, lpr);
  left = sl > 0 ? up : (g > 0 ? carry : T(0));
  if (sl < lpr - 1) right = dn;
  else right = (gok && g + 1 < gpr) ? right_at() : T(0);
  carry = __shfl_sync(FULL, v.a[3], lpr - 1, lpr);
}

template <typename T>
__device__ __forceinline__ T nb_sum(const V4<T>& v, int k, T left, T right, const V4<T>& ym, const V4<T>& yp,
                                    const V4<T>& zm, const V4<T>& zp) {
  const T l = k == 0 ? left : v.a[k - 1];
  const T r = k == 3 ? right : v.a[k + 1];
  return ((l + r) + (ym.a[k] + yp.a[k])) + (zm.a[k] + zp.a[k]);
}

struct RowIter {
  int warp, lane, lpr, rpw, sub, sl, nw, niter;
};
__device__ __forceinline__ RowIter row_iter(const RepDesc& rd) {
  RowIter it;
  it.warp = threadIdx.x >> 5;
  it.lane = threadIdx.x & 31;
  it.lpr = rd.lpr;
  it.rpw = 32 / rd.lpr;
  it.sub = it.lane / rd.lpr;
  it.sl = it.lane % rd.lpr;
  it.nw = blockDim.x >> 5;
  it.niter = (rd.gpr + rd.lpr - 1) / rd.lpr;
  return it;
}

// Per-lane accumulator of a pass: float-float for FP32 fields, double for FP64.
template <typename T> struct LaneAcc;
template <> struct LaneAcc<float> {
  FF v{0.f, 0.f};
  __device__ __forceinline__ void add(float x) { v = ff_add(v, x); }
};
template <> struct LaneAcc<double> {
  double v = 0.0;
  __device__ __forceinline__ void add(double x) { v += x; }
};

__device__ __forceinline__ void store_rows_acc(const Ctx& c, int chunk, int rl, bool row_ok, int sl, int lpr,
                                               const LaneAcc<float>* acc, int ndot) {
  FF a[NDOT];
  for (int k = 0; k < ndot; ++k) a[k] = acc[k].v;
  store_row_ff(c, chunk, rl, row_ok, sl, lpr, a, ndot);
}
__device__ __forceinline__ void store_rows_acc(const Ctx& c, int chunk, int rl, bool row_ok, int sl, int lpr,
                                               const LaneAcc<double>* acc, int ndot) {
  double a[NDOT];
  for (int k = 0; k < ndot; ++k) a[k] = acc[k].v;
  store_row(c, chunk, rl, row_ok, sl, lpr, a, ndot);
}

// Persistent row kernels (one lattice, one row per warp): block b of the
// grid updates the rows [R b / G, R (b + 1) / G) of the lattice's R rows, its
// warps taking them in turn; row sums go to the same chunk slots as in the
// one-block-per-chunk form.
__device__ __forceinline__ int persist_row_begin(int R) { return (int)((long long)R * blockIdx.x / gridDim.x); }
__device__ __forceinline__ int persist_row_end(int R) { return (int)((long long)R * (blockIdx.x + 1) / gridDim.x); }

// Chunk arrivals of a persistent row kernel, once per block after all its
// rows: each chunk the block touched receives the number of its rows the
// block wrote (an atomic add); the arrival that completes a chunk hands it to
// one warp of this block, which sums it in the fixed tree of warp_epilogue and
// continues to the group and replicate levels.  The same sums, in the same
// order, as the one-block-per-chunk form; only who finishes differs.
template <bool FFROWS = false, class Fin, class Post>
__device__ void block_arrivals(const Ctx& c, int ndot, Fin fin, Post post) {
  const RepDesc& rd = c.reps[0];
  const int R = rd.ny * rd.nz, cr = rd.chunk_rows;
  const int jb = persist_row_begin(R), je = persist_row_end(R);
  __shared__ int s_done[64];
  __shared__ int s_n;
  __threadfence();   // this thread's row sums are visible before the arrivals
  __syncthreads();
  if (je <= jb) return;
  const int c0 = jb / cr, c1 = (je - 1) / cr;
  for (int base = c0; base <= c1; base += 64) {
    if (threadIdx.x == 0) s_n = 0;
    __syncthreads();
    const int ci = base + (int)threadIdx.x;
    if (threadIdx.x < 64 && ci <= c1) {
      const int lo = max(jb, ci * cr), hi = min(je, min(R, (ci + 1) * cr));
      const int n = hi - lo, full = min(cr, R - ci * cr);
      if (atomicAdd(&c.chunk_cnt[ci], n) + n == full) s_done[atomicAdd(&s_n, 1)] = ci;
    }
    __syncthreads();
    const int nd = s_n;
    for (int i = (int)(threadIdx.x >> 5); i < nd; i += (int)(blockDim.x >> 5)) warp_chunk_done<FFROWS>(c, ndot, s_done[i], fin, post);
    __syncthreads();
  }
}

}  // namespace hca
