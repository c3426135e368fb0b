// Matrix-free 7-point operators and the Jacobi-preconditioned CG passes for
// the oxygen (Eq. oxygen, s_K = 0, consumption linearised about the previous
// K as in Section 2.4.1) and drug (Eq. chemo, one implicit-Euler step) solves.
//
// Operator at site i (Neumann boundaries: out-of-box neighbours are omitted):
//     (A u)_i = d_i u_i - c * sum_{j in box, |i-j| = 1} u_j,
//     d_i = c * n_i + a_i,      c = D / dx^2,  n_i = in-box neighbour count,
//     oxygen: a_i = phi_K / (K1 + K_prev,i) [consumer] + r_K [vessel],  b_i = r_K K0 [vessel]
//     drug:   a_i = 1/dt + psi + kappa perf_i [vessel] + uptake [cancer],
//             b_i = G^n_i / dt + kappa perf_i G_0(t^{n+1}) [vessel].
//
// CG is carried in the preconditioned residual z = r / d instead of r, so
// the direction update p = z + beta p needs no division at neighbour sites:
//   pass A: p = z + beta p;  q = A p, stored;  sigma = p.q
//   pass B: x += alpha p;  z -= alpha q / d;  rho = r.z = sum d z^2,
//           |r|^2 = sum (d z)^2  (multigrid form: r -= alpha q, |r|^2; the
//           V-cycle then forms z = M r and rho)
// HBM traffic per site and iteration: pass A reads z, p, d and writes p and
// q (20 B, FP32); pass B reads p, q, x, z (+ d, Jacobi form) and writes x, z
// (24-28 B): 44 B, against the two-pass minimum of 40 B in which pass B
// re-forms A p from p's neighbour rows instead of streaming q.
// Neighbour rows are re-read through L1/L2.  Pass A rebuilds the new
// direction at neighbour sites from the old one, so the old and new
// directions live in two buffers that swap roles every iteration (an in-place
// update would let one block read a neighbour row another block has already
// overwritten); a parity bit in device memory, flipped by pass B, names the
// current buffer, so the same two kernels form the body of a graph loop.
#include <mutex>
#include <vector>

#include <cstdlib>

#include "hca_internal.cuh"
#include "row_ops.cuh"

namespace hca {
namespace {

// a + k p for the drug reaction: in FP32 rounded after the product and after
// the sum (no fused multiply-add), so the stored FP32 coefficients of the
// system are the plain IEEE result of these operations.
__device__ __forceinline__ float add_prod(float a, float k, float p) { return __fadd_rn(a, __fmul_rn(k, p)); }
__device__ __forceinline__ double add_prod(double a, double k, double p) { return a + k * p; }

// The coefficients of operator `which` in the field precision, converted
// from the handle's FP64 parameters once per thread: the conversions run on
// the FP64 pipe (a small fraction of the FP32 rate on this GPU), and the
// parameters sit in global memory, where the compiler cannot keep them in
// registers across the kernel's own stores.
template <typename T>
struct Coef {
  T cpl, phi_K, K1, r_K, o2_mass, base, kappa, uptake;
};
template <typename T, int KIND>
__device__ __forceinline__ Coef<T> coef(const RepDesc& rd, int which) {
  Coef<T> q;
  q.cpl = op_coupling_t<T>(rd, which);
  q.phi_K = q.K1 = q.r_K = q.o2_mass = q.base = q.kappa = q.uptake = T(0);
  if (KIND == 0) {
    q.phi_K = (T)rd.phi_K;
    q.K1 = (T)rd.K1;
    q.r_K = (T)rd.r_K;
    q.o2_mass = (T)rd.o2_mass;
  } else {
    const int dd = which - 1;
    q.base = (T)rd.base_drug[dd];
    q.kappa = (T)rd.kappa[dd];
    q.uptake = (T)rd.uptake[dd];
  }
  return q;
}

// Reaction coefficient a of the operator at one site (d = c n + a).
template <typename T, int KIND>
__device__ __forceinline__ T reaction_site(const Coef<T>& q, uint8_t s, T K_prev, T pf) {
  T a;
  if (KIND == 0) {
    a = is_consumer(s) ? q.phi_K / (q.K1 + K_prev) : T(0);
    if (is_vessel(s)) a += q.r_K;
    a += q.o2_mass;   // 0 for the quasi-steady form
  } else {
    a = q.base;
    if (is_vessel(s)) a = add_prod(a, q.kappa, pf);
    if (is_cancer(s)) a += q.uptake;
  }
  return a;
}

// Diagonal of the operator at one site.
template <typename T, int KIND>
__device__ __forceinline__ T diag_site(const Coef<T>& q, int n_nb, uint8_t s, T K_prev, T pf) {
  return q.cpl * (T)n_nb + reaction_site<T, KIND>(q, s, K_prev, pf);
}

// ------------------------------------------------------------------ setup --
// r = b - A x0 with x0 the current field; writes d, z = r/d (and b for drugs
// and the time-dependent oxygen form); reduces rho = r.z, |r|^2, |b|^2.
template <typename T, int KIND>
__global__ void __launch_bounds__(512) k_setup(Ctx c, int which, CondArg cnd) {
  HCA_COUNT_KERNEL(c);
  __shared__ double s_G0;
  const int2 ch = c.chunks[blockIdx.x];
  const RepDesc& rd = c.reps[ch.x];
  const int nrows = min(rd.chunk_rows, rd.ny * rd.nz - ch.y);
  const T* __restrict__ x = KIND == 0 ? (const T*)c.K : (const T*)c.G[which - 1];
  const T* __restrict__ perf = (const T*)c.perf;
  T* __restrict__ dd = (T*)c.d;
  T* __restrict__ zz = (T*)c.z;
  T* __restrict__ bb = (T*)c.b;
  if (KIND == 1) {
    if (threadIdx.x == 0) s_G0 = substep_plasma(rd, which, *c.step, c.sub);
    __syncthreads();
  }
  const T G0 = KIND == 1 ? (T)s_G0 : T(0);
  const Coef<T> q = coef<T, KIND>(rd, which);
  const T cpl = q.cpl;
  const T bx = (T)rd.bx[which];
  const bool bax = rd.bax[which] != 0;
  const bool o2t = KIND == 0 && rd.bx[0] != 0.0;   // time-dependent oxygen: b depends on x0
  const T bvessel = (T)(bax ? 2.0 * rd.r_K * rd.K0 : rd.r_K * rd.K0);
  const T av = (T)(bax ? 2.0 * rd.a_vegf : rd.a_vegf);
  const RowIter it = row_iter(rd);
  for (int rbase = it.warp * it.rpw; rbase < rd.chunk_rows; rbase += it.nw * it.rpw) {
    const int rl = rbase + it.sub;
    const bool row_ok = rl < nrows;
    const RowGeo geo = row_geo(rd, ch.y + (row_ok ? rl : 0));
    double acc[NDOT] = {0.0, 0.0, 0.0};
    T carry = T(0);
    for (int itn = 0; itn < it.niter; ++itn) {
      const int g = itn * it.lpr + it.sl;
      const bool gok = row_ok && g < rd.gpr;
      const long long e = geo.base + 4LL * g;
      const V4<T> X = ld4_if(x + e, gok);
      const V4<T> ym = ld4_if(x + e - geo.sy, gok && geo.ym);
      const V4<T> yp = ld4_if(x + e + geo.sy, gok && geo.yp);
      const V4<T> zm = ld4_if(x + e - geo.sz, gok && geo.zm);
      const V4<T> zp = ld4_if(x + e + geo.sz, gok && geo.zp);
      T left, right;
      x_neighbours(X, g, rd.gpr, it.sl, it.lpr, gok, carry, left, right, [&] { return x[e + 4]; });
      if (gok) {
        const uchar4 st = ld_state4(c.state + e);
        V4<T> PF = zero4<T>();
        if (KIND == 1) PF = ld4(perf + e);
        // the VEGF field's source is the cells' release a_V Vc (doubled under Crank-Nicolson)
        const bool vegf = KIND == 1 && which == WHICH_VEGF;
        const V4<T> VC = vegf ? ld4((const T*)c.Vc + e) : zero4<T>();
        const V4<T> LG = (KIND == 0 && c.lag) ? ld4((const T*)c.lag + e) : X;
        V4<T> D, Z, B, RR = zero4<T>();
        T g_rho = 0, g_rr = 0, g_bb = 0;
#pragma unroll
        for (int k = 0; k < 4; ++k) {
          const int xk = 4 * g + k;
          const uint8_t s = st_at(st, k);
          T dk = T(0), zk = T(0), bk = T(0);
          if (xk < rd.nx) {
            dk = diag_site<T, KIND>(q, neighbour_count(rd, geo, xk), s, LG.a[k], PF.a[k]);
            if (KIND == 0) bk = (is_vessel(s) ? bvessel : T(0)) + (o2t ? X.a[k] * bx : T(0));
            else if (vegf) bk = X.a[k] * bx + (is_consumer(s) ? av * VC.a[k] : T(0));
            else bk = X.a[k] * bx + (is_vessel(s) ? q.kappa * PF.a[k] * G0 : T(0));
            const T ax = dk * X.a[k] - cpl * nb_sum(X, k, left, right, ym, yp, zm, zp);
            if (bax) bk -= ax;   // Crank-Nicolson: b = (4/h) x0 - A x0 + f^{k-1} + f^k
            const T r = bk - ax;
            RR.a[k] = r;
            zk = dk != T(0) ? r / dk : T(0);   // d = 0 only for an isolated, empty 1-site box
            g_rho += r * zk;
            g_rr += r * r;
            g_bb += bk * bk;
          }
          D.a[k] = dk;
          Z.a[k] = zk;
          B.a[k] = bk;
        }
        st4(dd + e, D);
        st4(zz + e, Z);
        if (c.mg) st4((T*)c.r + e, RR);
        if (KIND == 1 || o2t) st4(bb + e, B);
        acc[0] += (double)g_rho;
        acc[1] += (double)g_rr;
        acc[2] += (double)g_bb;
      }
    }
    store_row(c, blockIdx.x, rl, row_ok, it.sl, it.lpr, acc, 3);
  }
  const double rtol = KIND == 0 ? rd.rtol_o2 : rd.rtol_drug;
  (void)rtol;
  warp_epilogue(c, 3, blockIdx.x,
                 [&](int r, const double* s3) -> int {
                   const RepDesc& rr = c.reps[r];
                   RepSolve& sv = c.solve[r];
                   const double tol = which == 0 ? rr.rtol_o2 : rr.rtol_drug;
                   if (c.frozen[r]) {
                     sv.active = 0;
                     sv.zero_b = 0;
                     sv.iters = 0;
                     sv.rnorm2 = 0.0;
                     sv.bnorm2 = 1.0;
                     sv.scale = 1.0;
                     return 0;
                   }
                   sv.rho = s3[0];
                   sv.rnorm2 = s3[1];
                   sv.bnorm2 = s3[2];
                   sv.alpha = 0.0;
                   sv.beta = 0.0;
                   sv.scale = 1.0;
                   sv.iters = 0;
                   sv.rtol = tol;
                   sv.maxit = rr.maxit;
                   sv.zero_b = s3[2] == 0.0;
                   const bool fin = isfinite(s3[0]) && isfinite(s3[1]) && isfinite(s3[2]);
                   if (!fin) c.sync->error = 1;
                   sv.active = fin && !sv.zero_b && sqrt(s3[1]) > tol * sqrt(s3[2]) && rr.maxit > 0;
                   return sv.active;
                 },
                 [&](int n_active) {
                   c.sync->parity = 0;
                   c.sync->guard = 0;
                   set_cond(cnd, n_active > 0);
                 });
}

// ----------------------------------------------------------------- pass A --
// All loads of a group (own site and the four neighbour rows) are issued
// before any value is used, so a group costs one memory round trip.
// PERSIST: the persistent row form (one lattice, one row per warp; see
// block_arrivals), else one block per chunk.
template <typename T, int REGS, int NI, bool PERSIST>
__global__ void __maxnreg__(REGS) k_pass_a(Ctx c, int which) {
  HCA_COUNT_KERNEL(c);
  const int2 ch = PERSIST ? make_int2(0, 0) : c.chunks[blockIdx.x];
  const RepDesc& rd = c.reps[ch.x];
  const RepSolve sv = c.solve[ch.x];
  if (sv.active) {
    const int nrows = min(rd.chunk_rows, rd.ny * rd.nz - ch.y);
    const int gpr = rd.gpr;
    const int par = c.sync->parity;
    const T* __restrict__ pp = (const T*)(par ? c.p_alt : c.p);
    T* __restrict__ p_new = (T*)(par ? c.p : c.p_alt);
    const T* __restrict__ zz = (const T*)c.z;
    const T* __restrict__ dd = (const T*)c.d;
    T* __restrict__ qq = (T*)c.q;
    const T beta = (T)sv.beta;
    const bool use_p = sv.beta != 0.0;
    // the first iteration of a rescaled inner solve starts from scale * z
    // (the V-cycle scales r itself before it forms z)
    const T zs = (sv.iters == 0 && !c.mg) ? (T)sv.scale : T(1);
    const T cpl = op_coupling_t<T>(rd, which);
    const RowIter it = row_iter(rd);
    // one row j (chunk slot rl of `chunk`; row_ok false: a padding slot of the last chunk)
    auto row = [&](int chunk, int rl, bool row_ok, int j) {
      const RowGeo geo = row_geo(rd, j);
      LaneAcc<T> acc[1];
      T carry = T(0);
      // groups per lane in a row: a compile-time count (NI > 0) lets the
      // compiler issue the loads of all of them before the first is used
      const int niter = NI > 0 ? NI : it.niter;
#pragma unroll
      for (int itn = 0; itn < niter; ++itn) {
        const int g = itn * it.lpr + it.sl;
        const bool gok = row_ok && g < gpr;
        const long long e = geo.base + 4LL * g;
        const bool last_lane = it.sl == it.lpr - 1 && gok && g + 1 < gpr;
        // issue every load of this group
        const V4<T> z0 = ld4_if(zz + e, gok);
        const V4<T> zym = ld4_if(zz + e - geo.sy, gok && geo.ym);
        const V4<T> zyp = ld4_if(zz + e + geo.sy, gok && geo.yp);
        const V4<T> zzm = ld4_if(zz + e - geo.sz, gok && geo.zm);
        const V4<T> zzp = ld4_if(zz + e + geo.sz, gok && geo.zp);
        const V4<T> D = ld4_if(dd + e, gok);
        const T zr = last_lane ? zz[e + 4] : T(0);
        V4<T> p0 = zero4<T>(), pym = zero4<T>(), pyp = zero4<T>(), pzm = zero4<T>(), pzp = zero4<T>();
        T pr = T(0);
        if (use_p) {
          p0 = ld4_if(pp + e, gok);
          pym = ld4_if(pp + e - geo.sy, gok && geo.ym);
          pyp = ld4_if(pp + e + geo.sy, gok && geo.yp);
          pzm = ld4_if(pp + e - geo.sz, gok && geo.zm);
          pzp = ld4_if(pp + e + geo.sz, gok && geo.zp);
          pr = last_lane ? pp[e + 4] : T(0);
        }
        // new direction at the site and at its neighbours: p = z + beta p_old
        V4<T> PN, ym, yp, zm, zp;
#pragma unroll
        for (int k = 0; k < 4; ++k) {
          PN.a[k] = cg_dir(zs, z0.a[k], beta, p0.a[k]);
          ym.a[k] = cg_dir(zs, zym.a[k], beta, pym.a[k]);
          yp.a[k] = cg_dir(zs, zyp.a[k], beta, pyp.a[k]);
          zm.a[k] = cg_dir(zs, zzm.a[k], beta, pzm.a[k]);
          zp.a[k] = cg_dir(zs, zzp.a[k], beta, pzp.a[k]);
        }
        const T right_next = cg_dir(zs, zr, beta, pr);
        T left, right;
        x_neighbours(PN, g, gpr, it.sl, it.lpr, gok, carry, left, right, [&] { return right_next; });
        if (gok) {
          T g_s = 0;
          V4<T> Q;
#pragma unroll
          for (int k = 0; k < 4; ++k) {
            Q.a[k] = cg_apply(D.a[k], PN.a[k], cpl, nb_sum(PN, k, left, right, ym, yp, zm, zp));
            g_s = cg_madd(PN.a[k], Q.a[k], g_s);
          }
          st4(p_new + e, PN);
          st4(qq + e, Q);   // pass B reads A p instead of re-forming it from p's neighbours
          acc[0].add(g_s);
        }
      }
      store_rows_acc(c, chunk, rl, row_ok, it.sl, it.lpr, acc, 1);
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
  }
  auto fin = [&](int r, const double* s1) -> int {
    RepSolve& s = c.solve[r];
    if (!s.active) return 0;
    if (!(s1[0] > 0.0) || !isfinite(s1[0])) {
      if (!isfinite(s1[0])) c.sync->error = 1;
      s.active = 0;
      return 0;
    }
    s.alpha = s.rho / s1[0];
    return 1;
  };
  // float-float row slots for FP32 fields (LaneAcc<float>)
  if (PERSIST) block_arrivals<sizeof(T) == 4>(c, 1, fin, [](int) {});
  else warp_epilogue<sizeof(T) == 4>(c, 1, blockIdx.x, fin);
}

// ----------------------------------------------------------------- pass B --
template <typename T, int REGS, int NI, bool PERSIST>
__global__ void __maxnreg__(REGS) k_pass_b(Ctx c, int which, void* xfield, CondArg cnd) {
  HCA_COUNT_KERNEL(c);
  const int2 ch = PERSIST ? make_int2(0, 0) : c.chunks[blockIdx.x];
  const RepDesc& rd = c.reps[ch.x];
  const RepSolve sv = c.solve[ch.x];
  if (sv.active) {
    const int nrows = min(rd.chunk_rows, rd.ny * rd.nz - ch.y);
    const int gpr = rd.gpr, nx = rd.nx;
    // Jacobi form: z = r / d is carried; V-cycle form: r itself (already scaled)
    const bool mg = c.mg != 0;
    T* __restrict__ zz = (T*)(mg ? c.r : c.z);
    const T* __restrict__ pp = (const T*)(c.sync->parity ? c.p : c.p_alt);
    const T* __restrict__ dd = (const T*)c.d;
    const T* __restrict__ qq = (const T*)c.q;
    T* __restrict__ xx = (T*)xfield;
    const T alpha = (T)sv.alpha;
    const T zs = (sv.iters == 0 && !mg) ? (T)sv.scale : T(1);
    const RowIter it = row_iter(rd);
    auto row = [&](int chunk, int rl, bool row_ok, int j) {
      const RowGeo geo = row_geo(rd, j);
      LaneAcc<T> acc[2];
      // groups per lane in a row: a compile-time count (NI > 0) lets the
      // compiler issue the loads of all of them before the first is used
      const int niter = NI > 0 ? NI : it.niter;
#pragma unroll
      for (int itn = 0; itn < niter; ++itn) {
        const int g = itn * it.lpr + it.sl;
        const bool gok = row_ok && g < gpr;
        const long long e = geo.base + 4LL * g;
        // issue every load of this group (A p comes from pass A)
        const V4<T> P = ld4_if(pp + e, gok);
        const V4<T> Q = ld4_if(qq + e, gok);
        const V4<T> D = mg ? zero4<T>() : ld4_if(dd + e, gok);
        V4<T> X = ld4_if(xx + e, gok);
        V4<T> Z = ld4_if(zz + e, gok);
        if (gok) {
          T g_rho = 0, g_rr = 0;
#pragma unroll
          for (int k = 0; k < 4; ++k) {
            if (4 * g + k < nx) {
              const T q = Q.a[k];
              X.a[k] += alpha * P.a[k];
              if (mg) {
                Z.a[k] -= alpha * q;
                g_rr += Z.a[k] * Z.a[k];
              } else {
                Z.a[k] = zs * Z.a[k] - alpha * (q / D.a[k]);
                const T r = D.a[k] * Z.a[k];
                g_rho += r * Z.a[k];
                g_rr += r * r;
              }
            }
          }
          st4(xx + e, X);
          st4(zz + e, Z);
          acc[0].add(g_rho);
          acc[1].add(g_rr);
        }
      }
      store_rows_acc(c, chunk, rl, row_ok, it.sl, it.lpr, acc, 2);
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
  }
  auto fin = [&](int r, const double* s2) -> int {
    RepSolve& s = c.solve[r];
    if (!s.active) return 0;
    s.iters += 1;
    if (!isfinite(s2[0]) || !isfinite(s2[1])) {
      c.sync->error = 1;
      s.active = 0;
      return 0;
    }
    if (!c.mg) {   // the V-cycle form sets beta and rho after z = M r
      s.beta = s2[0] / s.rho;
      s.rho = s2[0];
    }
    s.rnorm2 = s2[1];
    const bool conv = sqrt(s2[1]) <= s.rtol * sqrt(s.bnorm2);
    if (conv || s.iters >= s.maxit) s.active = 0;
    return s.active;
  };
  auto post = [&](int n_active) {
    c.sync->parity ^= 1;
    const int g = ++c.sync->guard;
    bool go = n_active > 0;
    if (go && g >= c.sync->guard_limit) {
      // every replicate stops at maxit; this only guards the graph loop
      c.sync->error = 2;
      go = false;
    }
    set_cond(cnd, go);
  };
  if (PERSIST) block_arrivals<sizeof(T) == 4>(c, 2, fin, post);
  else warp_epilogue<sizeof(T) == 4>(c, 2, blockIdx.x, fin, post);
}

// ----------------------------------------------------------- true residual --
// rr = |b - A x|^2 with b rebuilt from the state (oxygen) or read back (drug);
// zeroes x where b = 0.  Records iterations and the relative residual in the
// statistics slot `which`.
template <typename T, int KIND>
__global__ void __launch_bounds__(512) k_true_residual(Ctx c, int which, void* xfield) {
  HCA_COUNT_KERNEL(c);
  const int2 ch = c.chunks[blockIdx.x];
  const RepDesc& rd = c.reps[ch.x];
  const RepSolve sv = c.solve[ch.x];
  const int nrows = min(rd.chunk_rows, rd.ny * rd.nz - ch.y);
  T* __restrict__ xx = (T*)xfield;
  const T* __restrict__ dd = (const T*)c.d;
  const T* __restrict__ bb = (const T*)c.b;
  const T cpl = op_coupling_t<T>(rd, which);
  const T bvessel = (T)(rd.r_K * rd.K0);
  const RowIter it = row_iter(rd);
  for (int rbase = it.warp * it.rpw; rbase < rd.chunk_rows; rbase += it.nw * it.rpw) {
    const int rl = rbase + it.sub;
    const bool row_ok = rl < nrows;
    const RowGeo geo = row_geo(rd, ch.y + (row_ok ? rl : 0));
    double acc[NDOT] = {0.0, 0.0, 0.0};
    T carry = T(0);
    for (int itn = 0; itn < it.niter; ++itn) {
      const int g = itn * it.lpr + it.sl;
      const bool gok = row_ok && g < rd.gpr;
      const long long e = geo.base + 4LL * g;
      const V4<T> X = ld4_if(xx + e, gok);
      const V4<T> ym = ld4_if(xx + e - geo.sy, gok && geo.ym);
      const V4<T> yp = ld4_if(xx + e + geo.sy, gok && geo.yp);
      const V4<T> zm = ld4_if(xx + e - geo.sz, gok && geo.zm);
      const V4<T> zp = ld4_if(xx + e + geo.sz, gok && geo.zp);
      T left, right;
      x_neighbours(X, g, rd.gpr, it.sl, it.lpr, gok, carry, left, right, [&] { return xx[e + 4]; });
      if (gok) {
        const V4<T> D = ld4(dd + e);
        V4<T> B;
        if (KIND == 0 && rd.bx[0] != 0.0) {
          B = ld4(bb + e);
        } else if (KIND == 0) {
          const uchar4 st = ld_state4(c.state + e);
#pragma unroll
          for (int k = 0; k < 4; ++k) B.a[k] = is_vessel(st_at(st, k)) ? bvessel : T(0);
        } else {
          B = ld4(bb + e);
        }
        T g_rr = 0;
#pragma unroll
        for (int k = 0; k < 4; ++k) {
          if (4 * g + k < rd.nx) {
            const T r = B.a[k] - (D.a[k] * X.a[k] - cpl * nb_sum(X, k, left, right, ym, yp, zm, zp));
            g_rr += r * r;
          }
        }
        acc[0] += (double)g_rr;
      }
    }
    store_row(c, blockIdx.x, rl, row_ok, it.sl, it.lpr, acc, 1);
  }
  warp_epilogue(c, 1, blockIdx.x,
                 [&](int r, const double* s1) -> int {
                   RepSolve& s = c.solve[r];
                   DevStats& st = c.stats[r];
                   s.rel_true = s.zero_b ? 0.0 : sqrt(s1[0] / s.bnorm2);
                   st.iters[which] += s.iters;
                   st.rel[which] = s.rel_true;
                   if (!s.zero_b && !(sqrt(s.rnorm2) <= s.rtol * sqrt(s.bnorm2))) st.not_converged |= 1 << which;
                   if (!isfinite(s1[0])) {
                     c.sync->error = 1;
                     st.nonfinite = 1;
                   }
                   return 0;
                 });
  (void)sv;
}

// x = 0 for replicates whose right-hand side vanished.
template <typename T>
__global__ void k_zero_if_b_zero(Ctx c, void* xfield) {
  HCA_COUNT_KERNEL(c);
  const int2 ch = c.chunks[blockIdx.x];
  if (!c.solve[ch.x].zero_b) return;
  const RepDesc& rd = c.reps[ch.x];
  const int nrows = min(rd.chunk_rows, rd.ny * rd.nz - ch.y);
  T* xx = (T*)xfield;
  const long long base = rd.off + (long long)ch.y * rd.nxp;
  const long long n = (long long)nrows * rd.nxp;
  for (long long i = threadIdx.x; i < n; i += blockDim.x) xx[base + i] = T(0);
}

// ---------------------------------------------------------- apply operator --
// out = A u for one replicate (operator `which`, diagonal rebuilt from the
// state, the current K and the perfusion map).  Used to expose the stencil.
template <typename T, int KIND>
__global__ void __launch_bounds__(512) k_apply(Ctx c, int which, int rep, const T* __restrict__ u,
                                               T* __restrict__ out) {
  HCA_COUNT_KERNEL(c);
  const int2 ch = c.chunks[blockIdx.x];
  if (ch.x != rep) return;
  const RepDesc& rd = c.reps[ch.x];
  const int nrows = min(rd.chunk_rows, rd.ny * rd.nz - ch.y);
  const T* __restrict__ K = (const T*)c.K;
  const T* __restrict__ perf = (const T*)c.perf;
  const Coef<T> q = coef<T, KIND>(rd, which);
  const T cpl = q.cpl;
  const RowIter it = row_iter(rd);
  for (int rbase = it.warp * it.rpw; rbase < rd.chunk_rows; rbase += it.nw * it.rpw) {
    const int rl = rbase + it.sub;
    const bool row_ok = rl < nrows;
    const RowGeo geo = row_geo(rd, ch.y + (row_ok ? rl : 0));
    T carry = T(0);
    for (int itn = 0; itn < it.niter; ++itn) {
      const int g = itn * it.lpr + it.sl;
      const bool gok = row_ok && g < rd.gpr;
      const long long e = geo.base + 4LL * g;
      const V4<T> U = ld4_if(u + e, gok);
      const V4<T> ym = ld4_if(u + e - geo.sy, gok && geo.ym);
      const V4<T> yp = ld4_if(u + e + geo.sy, gok && geo.yp);
      const V4<T> zm = ld4_if(u + e - geo.sz, gok && geo.zm);
      const V4<T> zp = ld4_if(u + e + geo.sz, gok && geo.zp);
      T left, right;
      x_neighbours(U, g, rd.gpr, it.sl, it.lpr, gok, carry, left, right, [&] { return u[e + 4]; });
      if (gok) {
        const uchar4 st = ld_state4(c.state + e);
        const V4<T> KK = ld4(K + e);
        const V4<T> PF = ld4(perf + e);
        V4<T> O;
#pragma unroll
        for (int k = 0; k < 4; ++k) {
          const int xk = 4 * g + k;
          O.a[k] = T(0);
          if (xk < rd.nx) {
            const T dk = diag_site<T, KIND>(q, neighbour_count(rd, geo, xk), st_at(st, k), KK.a[k], PF.a[k]);
            O.a[k] = dk * U.a[k] - cpl * nb_sum(U, k, left, right, ym, yp, zm, zp);
          }
        }
        st4(out + e, O);
      }
    }
  }
}

// |a - b|^2 and |a|^2 per replicate (into solve[rep].rnorm2 / bnorm2); used
// by the fixed-point iteration of the initial oxygen field.
template <typename T>
__global__ void __launch_bounds__(512) k_diff_norms(Ctx c, const T* __restrict__ a, const T* __restrict__ b) {
  HCA_COUNT_KERNEL(c);
  const int2 ch = c.chunks[blockIdx.x];
  const RepDesc& rd = c.reps[ch.x];
  const int nrows = min(rd.chunk_rows, rd.ny * rd.nz - ch.y);
  const RowIter it = row_iter(rd);
  for (int rbase = it.warp * it.rpw; rbase < rd.chunk_rows; rbase += it.nw * it.rpw) {
    const int rl = rbase + it.sub;
    const bool row_ok = rl < nrows;
    const RowGeo geo = row_geo(rd, ch.y + (row_ok ? rl : 0));
    double acc[NDOT] = {0.0, 0.0, 0.0};
    for (int itn = 0; itn < it.niter; ++itn) {
      const int g = itn * it.lpr + it.sl;
      if (row_ok && g < rd.gpr) {
        const long long e = geo.base + 4LL * g;
        const V4<T> A = ld4(a + e), B = ld4(b + e);
        T s0 = 0, s1 = 0;
#pragma unroll
        for (int k = 0; k < 4; ++k) {
          const T df = A.a[k] - B.a[k];
          s0 += df * df;
          s1 += A.a[k] * A.a[k];
        }
        acc[0] += (double)s0;
        acc[1] += (double)s1;
      }
    }
    store_row(c, blockIdx.x, rl, row_ok, it.sl, it.lpr, acc, 2);
  }
  warp_epilogue(c, 2, blockIdx.x,
                 [&](int r, const double* s2) -> int {
                   c.solve[r].rnorm2 = s2[0];
                   c.solve[r].bnorm2 = s2[1];
                   return 0;
                 });
}

// A sum of FP32 terms s * 2^ex kept as m * 2^e in FP32 arithmetic (the
// terms are scaled sums of a few squares, so m stays of order one; terms more
// than 2^126 below the running sum underflow to zero), converted to FP64 once.
struct ScaledAcc {
  float m = 0.f;
  int e = 0;
  __device__ __forceinline__ void add(float s, int ex) {
    if (s == 0.f) return;
    if (m == 0.f) {
      m = s;
      e = ex;
    } else if (ex > e) {
      m = scalbnf(m, e - ex) + s;
      e = ex;
    } else {
      m += scalbnf(s, ex - e);
    }
  }
  // m 2^e in FP64, exactly: 2^e is built from its bits when it is a normal
  // double (two FP64-pipe instructions instead of a library ldexp)
  __device__ __forceinline__ double value() const {
    if (m == 0.f) return 0.0;
    if (e < -1022 || e > 1023) return ldexp((double)m, e);
    return (double)m * __longlong_as_double((long long)(e + 1023) << 52);
  }
};

// The sum of a row's lane accumulators (lane segments of lpr lanes, fixed
// xor tree: partners form the same sum, so every lane of the segment ends
// with it) in FP32 arithmetic, converted to FP64 once per row.
__device__ __forceinline__ double row_reduce_scaled(ScaledAcc a, int lpr) {
  for (int o = lpr >> 1; o > 0; o >>= 1) {
    const float bm = __shfl_xor_sync(0xffffffffu, a.m, o, 32);
    const int be = __shfl_xor_sync(0xffffffffu, a.e, o, 32);
    if (bm != 0.f) {
      if (a.m == 0.f) {
        a.m = bm;
        a.e = be;
      } else {
        const int e = max(a.e, be);
        a.m = scalbnf(a.m, a.e - e) + scalbnf(bm, be - e);
        a.e = e;
      }
    }
  }
  return a.value();
}

// --------------------------------------------------- defect correction ---
// FP32 storage scheme.  The solution is kept as two FP32 words, x = x_hi +
// x_lo.  Each sweep evaluates the residual r = b - A x to about 48 bits
// (float-float arithmetic) from the two-word solution, with the diagonal
// rebuilt exactly as c n + a from the stored FP32 reaction coefficient a (storing d = c n + a itself in FP32 would
// round away most digits of the small reaction part: 1/dt + psi ~ 0.03 next to
// c n ~ 600 for a drug).  It stops the solve when |r| <= rtol |b| (FP64 norms)
// and otherwise starts an FP32 inner CG on the correction, A32 dx = fl32(r),
// dx0 = 0, to the inner tolerance, where A32 uses the FP32 diagonal.  The first
// sweep of a solve (FIRST) also builds and stores a, d (and b for a drug).
// With the multigrid preconditioner (MG) the kernel stores r for the V-cycle,
// which forms z itself; otherwise it stores the Jacobi z = r / d and sums r.z.
// Per site the arithmetic is FP32 and float-float (FP64 runs at a small
// fraction of the FP32 rate on this GPU).
// The epilogue of a row kernel in either form (block per chunk, or
// persistent rows with block-level chunk arrivals).
template <bool PERSIST, class Fin, class Post>
__device__ __forceinline__ void dc_epilogue(const Ctx& c, int ndot, int chunk, Fin fin, Post post) {
  if (PERSIST) block_arrivals(c, ndot, fin, post);
  else warp_epilogue(c, ndot, chunk, fin, post);
}

template <int KIND, bool FIRST, bool MG, bool PERSIST = false, int REGS = 128>
__global__ void __launch_bounds__(512) __maxnreg__(REGS) k_dc_residual(Ctx c, int which, const float* __restrict__ x_hi,
                                                     const float* __restrict__ x_lo, CondArg outer,
                                                     CondArg inner) {
  HCA_COUNT_KERNEL(c);
  __shared__ double s_G0;
  const int2 ch = PERSIST ? make_int2(0, 0) : c.chunks[blockIdx.x];
  const RepDesc& rd = c.reps[ch.x];
  const RepSolve sv = c.solve[ch.x];
  const bool live = FIRST || sv.active || sv.dc_apply;
  if (KIND == 1 && FIRST) {
    if (threadIdx.x == 0) s_G0 = substep_plasma(rd, which, *c.step, c.sub);
    __syncthreads();
  }
  if (live) {
    const int nrows = min(rd.chunk_rows, rd.ny * rd.nz - ch.y);
    float* __restrict__ dd = (float*)c.d;
    float* __restrict__ aa = (float*)c.reac;
    float* __restrict__ zz = (float*)c.z;
    float* __restrict__ bb = (float*)c.b;
    float* __restrict__ dxv = (float*)c.dx;
    const float* __restrict__ perf = (const float*)c.perf;
    const Coef<float> q = coef<float, KIND>(rd, which);
    const double cpl = (double)q.cpl;
    const float G0 = KIND == 1 && FIRST ? (float)s_G0 : 0.f;
    const bool bax = rd.bax[which] != 0;
    const bool o2t = KIND == 0 && rd.bx[0] != 0.0;
    const double bx = rd.bx[which];
    // bx as an unevaluated float pair (b = bx x0 + ... is formed to ~48 bits)
    const float bx_hi = (float)bx, bx_lo = (float)(bx - (double)bx_hi);
    const float bvessel = (float)(bax ? 2.0 * rd.r_K * rd.K0 : rd.r_K * rd.K0);
    const float av = (float)(bax ? 2.0 * rd.a_vegf : rd.a_vegf);
    const RowIter it = row_iter(rd);
    const float cpl32 = (float)cpl;
    // one row j (chunk slot rl of `chunk`; row_ok false: a padding slot of the last chunk)
    auto row = [&](int chunk, int rl, bool row_ok, int j) {
      const RowGeo geo = row_geo(rd, j);
      ScaledAcc la[NDOT];
      float carry_h = 0.f, carry_l = 0.f;
      for (int itn = 0; itn < it.niter; ++itn) {
        const int g = itn * it.lpr + it.sl;
        const bool gok = row_ok && g < rd.gpr;
        const long long e = geo.base + 4LL * g;
        // the two-word solution x_hi + x_lo at the group and its neighbour rows
        const V4<float> Xh = ld4_if(x_hi + e, gok), Xl = ld4_if(x_lo + e, gok);
        const V4<float> ymh = ld4_if(x_hi + e - geo.sy, gok && geo.ym), yml = ld4_if(x_lo + e - geo.sy, gok && geo.ym);
        const V4<float> yph = ld4_if(x_hi + e + geo.sy, gok && geo.yp), ypl = ld4_if(x_lo + e + geo.sy, gok && geo.yp);
        const V4<float> zmh = ld4_if(x_hi + e - geo.sz, gok && geo.zm), zml = ld4_if(x_lo + e - geo.sz, gok && geo.zm);
        const V4<float> zph = ld4_if(x_hi + e + geo.sz, gok && geo.zp), zpl = ld4_if(x_lo + e + geo.sz, gok && geo.zp);
        // every other load of the group is issued here too, before any value
        // is used, so a group costs one memory round trip: the site after the
        // group (the segment's last lane), and d, a, b (later sweeps) or the
        // state, perfusion and Vc (the first sweep)
        const bool last_lane = it.sl == it.lpr - 1 && gok && g + 1 < rd.gpr;
        const float rnh = last_lane ? x_hi[e + 4] : 0.f, rnl = last_lane ? x_lo[e + 4] : 0.f;
        const bool vegf = KIND == 1 && which == WHICH_VEGF;
        V4<float> D = zero4<float>(), B = zero4<float>(), AR = zero4<float>(), SRC = zero4<float>();
        V4<float> PF = zero4<float>(), VC = zero4<float>();
        uchar4 st = make_uchar4(0, 0, 0, 0);
        if (gok && FIRST) {
          st = ld_state4(c.state + e);
          if (KIND == 1) PF = ld4(perf + e);
          if (vegf) VC = ld4((const float*)c.Vc + e);
        } else if (gok) {
          if (!MG) D = ld4(dd + e);
          AR = ld4(aa + e);
          B = ld4(bb + e);
        }
        float lh, rh, ll, rlo;
        x_neighbours(Xh, g, rd.gpr, it.sl, it.lpr, gok, carry_h, lh, rh, [&] { return rnh; });
        x_neighbours(Xl, g, rd.gpr, it.sl, it.lpr, gok, carry_l, ll, rlo, [&] { return rnl; });
        if (gok) {
          if (FIRST) {
#pragma unroll
            for (int k = 0; k < 4; ++k) {
              const int xk = 4 * g + k;
              const uint8_t s = st_at(st, k);
              D.a[k] = 0.f;
              B.a[k] = 0.f;
              AR.a[k] = 0.f;
              SRC.a[k] = 0.f;
              if (xk < rd.nx) {
                // x0 bx to ~48 bits, rounded once; x0 rounded to FP32
                const FF xbx = ff_mul(FF{Xh.a[k], Xl.a[k]}, FF{bx_hi, bx_lo});
                const float xb32 = __fadd_rn(xbx.hi, xbx.lo);
                const float xk32 = __fadd_rn(Xh.a[k], Xl.a[k]);
                // the operator is linearised about K_prev: the start field, or c.lag when the solve starts from another guess
                const float lag = (KIND == 0 && c.lag) ? ((const float*)c.lag)[e + k] : xk32;
                AR.a[k] = reaction_site<float, KIND>(q, s, lag, PF.a[k]);
                D.a[k] = cpl32 * (float)neighbour_count(rd, geo, xk) + AR.a[k];
                if (KIND == 0) {
                  SRC.a[k] = is_vessel(s) ? bvessel : 0.f;
                  B.a[k] = SRC.a[k] + (o2t ? xb32 : 0.f);
                } else {
                  if (vegf) SRC.a[k] = is_consumer(s) ? av * VC.a[k] : 0.f;
                  else SRC.a[k] = is_vessel(s) ? __fmul_rn(__fmul_rn(q.kappa, PF.a[k]), G0) : 0.f;
                  B.a[k] = __fadd_rn(xb32, SRC.a[k]);
                }
              }
            }
            st4(dd + e, D);
            st4(aa + e, AR);
            if (MG) {   // 1/d for the V-cycle's sweeps (0 where d = 0), as k_mg_w0 forms it
              V4<float> Wv;
#pragma unroll
              for (int k = 0; k < 4; ++k) Wv.a[k] = D.a[k] != 0.f ? 1.f / D.a[k] : 0.f;
              st4((float*)c.mg_w + e, Wv);
            }
          }
          V4<float> Z, R32 = zero4<float>();
#pragma unroll
          for (int k = 0; k < 4; ++k) {
            Z.a[k] = 0.f;
            if (4 * g + k < rd.nx) {
              // r = b - (d x - c sum_nb x) in float-float (~48 bits): the
              // operator's terms cancel to the small defect; d = c n + a is
              // formed exactly from the stored reaction a
              const FF xv{Xh.a[k], Xl.a[k]};
              const FF L{k == 0 ? lh : Xh.a[k - 1], k == 0 ? ll : Xl.a[k - 1]};
              const FF Rr{k == 3 ? rh : Xh.a[k + 1], k == 3 ? rlo : Xl.a[k + 1]};
              const FF nb = ff_add(ff_add(ff_add(L, Rr), ff_add(FF{ymh.a[k], yml.a[k]}, FF{yph.a[k], ypl.a[k]})),
                                   ff_add(FF{zmh.a[k], zml.a[k]}, FF{zph.a[k], zpl.a[k]}));
              const FF d = ff_add(ff_two_prod(cpl32, (float)neighbour_count(rd, geo, 4 * g + k)), AR.a[k]);
              const FF t = ff_add(ff_mul(d, xv), ff_neg(ff_mul(nb, cpl32)));
              // Crank-Nicolson: b = (4/h) x0 - A x0 + source, formed once from the start field
              if (FIRST && bax) {
                const FF bf = ff_add(ff_add(ff_mul(xv, FF{bx_hi, bx_lo}), SRC.a[k]), ff_neg(t));
                B.a[k] = __fadd_rn(bf.hi, bf.lo);
              }
              const FF rf = ff_add(ff_neg(t), B.a[k]);
              const float r32 = __fadd_rn(rf.hi, rf.lo);
              if (!MG) Z.a[k] = D.a[k] != 0.f ? r32 / D.a[k] : 0.f;
              R32.a[k] = r32;
            }
          }
          if (FIRST) st4(bb + e, B);
          // the group's |r|^2, r.z and |b|^2: each 4-term sum is taken in
          // FP32 after an exact power-of-two scaling by the group's largest
          // magnitude (a decayed field's residual, ~1e-22, would underflow
          // when squared unscaled); the lane keeps its groups' sums as a
          // scaled FP32 pair and enters the FP64 row sums once per row (FP64
          // arithmetic is a small fraction of FP32's on this GPU)
          auto scaled_sum = [](const V4<float>& v, ScaledAcc& acc) {
            float m = 0.f;
#pragma unroll
            for (int k = 0; k < 4; ++k) m = fmaxf(m, fabsf(v.a[k]));
            if (m == 0.f) return;
            const int ex = ilogbf(m);
            float s2 = 0.f;
#pragma unroll
            for (int k = 0; k < 4; ++k) {
              const float u = scalbnf(v.a[k], -ex);
              s2 += u * u;
            }
            acc.add(s2, 2 * ex);
          };
          scaled_sum(R32, la[0]);
          if (FIRST) scaled_sum(B, la[1]);
          if (!MG) {
            // r.z with z = r / d: scale r and z by the same power (|z| may be
            // far from |r|, so each is scaled by its own group maximum)
            float mr = 0.f, mz = 0.f;
#pragma unroll
            for (int k = 0; k < 4; ++k) {
              mr = fmaxf(mr, fabsf(R32.a[k]));
              mz = fmaxf(mz, fabsf(Z.a[k]));
            }
            if (mr > 0.f && mz > 0.f) {
              const int er = ilogbf(mr), ez = ilogbf(mz);
              float s = 0.f;
#pragma unroll
              for (int k = 0; k < 4; ++k) s += scalbnf(R32.a[k], -er) * scalbnf(Z.a[k], -ez);
              la[2].add(s, er + ez);
            }
          }
          if (MG) st4((float*)c.r + e, R32);
          else st4(zz + e, Z);
          st4(dxv + e, zero4<float>());
        }
      }
#pragma unroll
      for (int k = 0; k < NDOT; ++k) {
        const double v = row_reduce_scaled(la[k], it.lpr);
        if (row_ok && it.sl == 0) c.rowp[((long long)chunk * CHUNK_ROWS + rl) * NDOT + k] = v;
      }
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
  }
  dc_epilogue<PERSIST>(c, 3, blockIdx.x,
                 [&](int r, const double* s3) -> int {
                   const RepDesc& rr = c.reps[r];
                   RepSolve& s = c.solve[r];
                   DevStats& st = c.stats[r];
                   if (FIRST) {
                     s.outer = 0;
                     s.zero_b = 0;
                     s.dc_apply = 0;
                     s.active = 0;
                     s.iters = 0;
                     if (c.frozen[r]) return 0;
                   } else if (!s.dc_apply) {
                     return 0;        // this replicate finished in an earlier sweep
                   }
                   st.iters[which] += s.iters;
                   st.sweeps[which] += 1;
                   // |b|^2 is summed on the first sweep only (b does not change)
                   if (FIRST) s.bb_outer = s3[1];
                   const double bb = s.bb_outer;
                   if (!isfinite(s3[0]) || !isfinite(bb) || !isfinite(s3[2])) {
                     c.sync->error = 1;
                     st.nonfinite = 1;
                     s.active = 0;
                     s.dc_apply = 0;
                     return 0;
                   }
                   const double tol = which == 0 ? rr.rtol_o2 : rr.rtol_drug;
                   if (bb == 0.0) {
                     s.zero_b = 1;
                     s.rel_true = 0.0;
                     st.rel[which] = 0.0;
                     s.active = 0;
                     s.dc_apply = 0;
                     return 0;
                   }
                   const double rel = sqrt(s3[0] / bb);
                   s.rel_true = rel;
                   st.rel[which] = rel;
                   if (rel <= tol || s.outer >= rr.max_outer) {
                     if (rel > tol) st.not_converged |= 1 << which;
                     s.active = 0;
                     s.dc_apply = 0;
                     return 0;
                   }
                   // start the inner FP32 solve A dx = fl32(r), rescaled by a
                   // power of two so that its values are O(1) per site (the
                   // residual of a decayed field can be ~1e-22, whose FP32
                   // squares underflow); the update divides the scale out
                   s.outer += 1;
                   const double n_sites = (double)rr.nx * rr.ny * rr.nz;
                   const double rms = sqrt(s3[0] / n_sites);
                   int e = rms > 0.0 ? -ilogb(rms) : 0;
                   e = e < -120 ? -120 : (e > 120 ? 120 : e);
                   const double sc = ldexp(1.0, e);
                   s.scale = sc;
                   s.rho = s3[2] * sc * sc;
                   s.rnorm2 = s3[0] * sc * sc;
                   s.bnorm2 = s3[0] * sc * sc;
                   // inner tolerance: rtol_inner relative to this sweep's
                   // defect, or, when the outer target is within a factor 8
                   // of that (or looser), the reduction that reaches half the
                   // outer target, so the last sweep neither over-solves nor
                   // falls just short and costs another sweep
                   const double q = 0.5 * tol / rel;
                   s.rtol = q >= 0.125 * rr.rtol_inner ? q : rr.rtol_inner;
                   s.maxit = rr.maxit;
                   s.iters = 0;
                   s.alpha = 0.0;
                   s.beta = 0.0;
                   s.dc_apply = 1;
                   // the multigrid form leaves rho to the V-cycle (s3[2] = 0)
                   s.active = (MG ? s3[0] > 0.0 : s3[2] > 0.0) ? 1 : 0;
                   return s.active;
                 },
                 [&](int n_active) {
                   c.sync->parity = 0;
                   c.sync->guard = 0;
                   const int g = FIRST ? (c.sync->guard_outer = 0) : ++c.sync->guard_outer;
                   bool go = n_active > 0;
                   if (go && g >= c.sync->guard_outer_limit) {
                     c.sync->error = 2;
                     go = false;
                   }
                   set_cond(outer, go);
                   set_cond(inner, go);
                 });
}

// x_hi + x_lo += dx (two-word sum), or x = 0 for a vanishing right-hand side.
__global__ void __launch_bounds__(512) k_dc_update(Ctx c, float* __restrict__ x_hi, float* __restrict__ x_lo) {
  HCA_COUNT_KERNEL(c);
  const int2 ch = c.chunks[blockIdx.x];
  const RepSolve sv = c.solve[ch.x];
  if (!sv.dc_apply && !sv.zero_b) return;
  const RepDesc& rd = c.reps[ch.x];
  const int nrows = min(rd.chunk_rows, rd.ny * rd.nz - ch.y);
  const long long base0 = rd.off + (long long)ch.y * rd.nxp;
  const int ngroups = nrows * rd.gpr;
  const float* __restrict__ dxv = (const float*)c.dx;
  const float inv_s = (float)(1.0 / sv.scale);   // a power of two: exact
  for (int gi = threadIdx.x; gi < ngroups; gi += blockDim.x) {
    const int rl = gi / rd.gpr, g = gi % rd.gpr;
    const long long e = base0 + (long long)rl * rd.nxp + 4LL * g;
    if (sv.zero_b) {
      st4(x_hi + e, zero4<float>());
      st4(x_lo + e, zero4<float>());
      continue;
    }
    V4<float> H = ld4(x_hi + e), L = ld4(x_lo + e);
    V4<float> D = ld4(dxv + e);
#pragma unroll
    for (int k = 0; k < 4; ++k) D.a[k] = __fmul_rn(D.a[k], inv_s);
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      // two-sum of hi and dx, then renormalise with the low word
      const float s = __fadd_rn(H.a[k], D.a[k]);
      const float bv = __fsub_rn(s, H.a[k]);
      const float err = __fadd_rn(__fsub_rn(H.a[k], __fsub_rn(s, bv)), __fsub_rn(D.a[k], bv));
      const float lo = __fadd_rn(L.a[k], err);
      const float hi = __fadd_rn(s, lo);
      L.a[k] = __fsub_rn(lo, __fsub_rn(hi, s));
      H.a[k] = hi;
    }
    st4(x_hi + e, H);
    st4(x_lo + e, L);
  }
}

}  // namespace

// ------------------------------------------------------------- launchers --
int persist_grid(const void* fn, int threads, int sm_count);

template <int KIND, bool FIRST, bool MG>
static void launch_dc_residual_v(const Ctx& c, int which, const float* x_hi, const float* x_lo, CondArg outer,
                                 CondArg inner) {
  if (c.persist) {
    // a 96-register cap: 16 -> 20 warps per SM (measured 176 -> 170 us per launch at 256^3)
    const int g = persist_grid((const void*)k_dc_residual<KIND, FIRST, MG, true, 96>, c.threads, c.sm_count);
    launch_k(c.pdl != 0, k_dc_residual<KIND, FIRST, MG, true, 96>, dim3(g), dim3(c.threads), 0, c.stream, c, which, x_hi,
             x_lo, outer, inner);
  } else {
    launch_k(c.pdl != 0, k_dc_residual<KIND, FIRST, MG, false>, dim3(c.n_chunks), dim3(c.threads), 0, c.stream, c, which,
             x_hi, x_lo, outer, inner);
  }
}

template <int KIND>
static void launch_dc_residual_t(const Ctx& c, int which, const float* x_hi, const float* x_lo, bool first,
                                 CondArg outer, CondArg inner) {
  if (first && c.mg) launch_dc_residual_v<KIND, true, true>(c, which, x_hi, x_lo, outer, inner);
  else if (first) launch_dc_residual_v<KIND, true, false>(c, which, x_hi, x_lo, outer, inner);
  else if (c.mg) launch_dc_residual_v<KIND, false, true>(c, which, x_hi, x_lo, outer, inner);
  else launch_dc_residual_v<KIND, false, false>(c, which, x_hi, x_lo, outer, inner);
}

void launch_dc_residual(const Ctx& c, int which, const void* x_hi, const void* x_lo, bool first, CondArg outer,
                        CondArg inner) {
  if (which == 0) launch_dc_residual_t<0>(c, which, (const float*)x_hi, (const float*)x_lo, first, outer, inner);
  else launch_dc_residual_t<1>(c, which, (const float*)x_hi, (const float*)x_lo, first, outer, inner);
}

void launch_dc_update(const Ctx& c, void* x_hi, void* x_lo) {
  launch_k(c.pdl != 0, k_dc_update, dim3(c.n_chunks), dim3(c.threads), 0, c.stream, c, (float*)x_hi, (float*)x_lo);
}

void launch_diff_norms(const Ctx& c, const void* a, const void* b, bool fp64) {
  if (fp64) k_diff_norms<double><<<c.n_chunks, c.threads, 0, c.stream>>>(c, (const double*)a, (const double*)b);
  else k_diff_norms<float><<<c.n_chunks, c.threads, 0, c.stream>>>(c, (const float*)a, (const float*)b);
}

template <typename T>
static void launch_setup_t(const Ctx& c, int which, CondArg cnd) {
  if (which == 0) k_setup<T, 0><<<c.n_chunks, c.threads, 0, c.stream>>>(c, which, cnd);
  else k_setup<T, 1><<<c.n_chunks, c.threads, 0, c.stream>>>(c, which, cnd);
}

void launch_setup(const Ctx& c, int which, bool fp64, CondArg cnd) {
  if (fp64) launch_setup_t<double>(c, which, cnd);
  else launch_setup_t<float>(c, which, cnd);
}

// Blocks of a persistent row kernel: every block resident at once (its
// occupancy at `threads` per block times the SM count), cached per kernel.
int persist_grid(const void* fn, int threads, int sm_count) {
  struct Entry {
    const void* fn;
    int threads, sm, grid;
  };
  static std::mutex mu;
  static std::vector<Entry> cache;
  std::lock_guard<std::mutex> lock(mu);
  for (const Entry& e : cache)
    if (e.fn == fn && e.threads == threads && e.sm == sm_count) return e.grid;
  int per = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, fn, threads, 0) != cudaSuccess || per < 1) {
    (void)cudaGetLastError();
    per = 1;
  }
  cache.push_back({fn, threads, sm_count, per * sm_count});
  return per * sm_count;
}

template <int REGS, int NI>
static void launch_ab_f32(const Ctx& c, int which, bool a, void* xfield, CondArg cnd) {
  const bool pdl = c.pdl != 0;
  if (NI > 0 && c.persist) {
    if (a) {
      const void* fn = (const void*)k_pass_a<float, REGS, NI, true>;
      launch_k(pdl, k_pass_a<float, REGS, NI, true>, dim3(persist_grid(fn, c.threads, c.sm_count)), dim3(c.threads), 0,
               c.stream, c, which);
    } else {
      const void* fn = (const void*)k_pass_b<float, REGS, NI, true>;
      launch_k(pdl, k_pass_b<float, REGS, NI, true>, dim3(persist_grid(fn, c.threads, c.sm_count)), dim3(c.threads), 0,
               c.stream, c, which, xfield, cnd);
    }
    return;
  }
  if (a) launch_k(pdl, k_pass_a<float, REGS, NI, false>, dim3(c.n_chunks), dim3(c.threads), 0, c.stream, c, which);
  else launch_k(pdl, k_pass_b<float, REGS, NI, false>, dim3(c.n_chunks), dim3(c.threads), 0, c.stream, c, which, xfield, cnd);
}

template <int REGS>
static void launch_ab_f32_ni(const Ctx& c, int which, bool a, void* xfield, CondArg cnd) {
  switch (c.pass_ni) {
    case 1: launch_ab_f32<REGS, 1>(c, which, a, xfield, cnd); break;
    case 2: launch_ab_f32<REGS, 2>(c, which, a, xfield, cnd); break;
    case 4: launch_ab_f32<REGS, 4>(c, which, a, xfield, cnd); break;
    default: launch_ab_f32<REGS, 0>(c, which, a, xfield, cnd); break;
  }
}

static void launch_ab(const Ctx& c, int which, bool fp64, bool a, void* xfield, CondArg cnd) {
  if (fp64) {
    if (a) k_pass_a<double, 128, 0, false><<<c.n_chunks, c.threads, 0, c.stream>>>(c, which);
    else k_pass_b<double, 128, 0, false><<<c.n_chunks, c.threads, 0, c.stream>>>(c, which, xfield, cnd);
    return;
  }
  switch (c.pass_regs) {
    case 64: launch_ab_f32_ni<64>(c, which, a, xfield, cnd); break;
    case 96: launch_ab_f32_ni<96>(c, which, a, xfield, cnd); break;
    case 128: launch_ab_f32_ni<128>(c, which, a, xfield, cnd); break;
    default: launch_ab_f32_ni<80>(c, which, a, xfield, cnd); break;
  }
}

void launch_pass_a(const Ctx& c, int which, bool fp64) { launch_ab(c, which, fp64, true, nullptr, CondArg{0ull, 0}); }

void launch_pass_b(const Ctx& c, int which, void* xfield, bool fp64, CondArg cnd) {
  launch_ab(c, which, fp64, false, xfield, cnd);
}

void launch_true_residual(const Ctx& c, int which, void* xfield, bool fp64) {
  if (fp64) {
    if (which == 0) k_true_residual<double, 0><<<c.n_chunks, c.threads, 0, c.stream>>>(c, which, xfield);
    else k_true_residual<double, 1><<<c.n_chunks, c.threads, 0, c.stream>>>(c, which, xfield);
    k_zero_if_b_zero<double><<<c.n_chunks, c.threads, 0, c.stream>>>(c, xfield);
  } else {
    if (which == 0) k_true_residual<float, 0><<<c.n_chunks, c.threads, 0, c.stream>>>(c, which, xfield);
    else k_true_residual<float, 1><<<c.n_chunks, c.threads, 0, c.stream>>>(c, which, xfield);
    k_zero_if_b_zero<float><<<c.n_chunks, c.threads, 0, c.stream>>>(c, xfield);
  }
}

void launch_apply(const Ctx& c, int which, int rep, const void* u, void* out, bool fp64) {
  if (fp64) {
    if (which == 0) k_apply<double, 0><<<c.n_chunks, c.threads, 0, c.stream>>>(c, which, rep, (const double*)u, (double*)out);
    else k_apply<double, 1><<<c.n_chunks, c.threads, 0, c.stream>>>(c, which, rep, (const double*)u, (double*)out);
  } else {
    if (which == 0) k_apply<float, 0><<<c.n_chunks, c.threads, 0, c.stream>>>(c, which, rep, (const float*)u, (float*)out);
    else k_apply<float, 1><<<c.n_chunks, c.threads, 0, c.stream>>>(c, which, rep, (const float*)u, (float*)out);
  }
}

}  // namespace hca
