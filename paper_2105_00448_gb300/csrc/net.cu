// Learned initial guess for the oxygen solve: a 3-D convolutional
// encoder-decoder on BF16 tensor cores, its backward pass and Adam, all as
// hand-written kernels.  The paper has no counterpart (it warm-starts every
// solve from the previous step); the network, its input features and its
// training loss are defined in the FP64 reference of the test suite.
//
// Layout: activations are dense (D, H, W, C) BF16 tensors with C innermost;
// a 3x3x3 weight tensor is (27, C_out, C_in) with tap t = 9(dz+1)+3(dy+1)+(dx+1).
// Parameters live in one FP32 array (conv weights, then biases, per layer;
// then the 16 head weights and the head bias); BF16 copies of the conv
// weights, and of their tap-flipped transposes for the input gradient, are
// refreshed after every update.
//
// Convolutions are implicit GEMMs: M = output sites (tiles of 16 consecutive
// x by TZ x TY rows), N = C_out, K = 27 C_in.  A block stages its input halo
// once in shared memory (XOR-swizzled 16-byte chunks, conflict-free for
// ldmatrix row gathers), stages the weights one z-plane of taps at a time,
// and every warp runs mma.m16n8k16 BF16 -> FP32 over its rows.  The nearest
// 2x upsampling of the decoder is folded into the halo gather; the sum over
// the 2x2x2 children that its gradient needs is folded into the epilogue.

#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstdlib>
#include <cstring>
#include <new>
#include <vector>

#include "hca.h"
#include "net_internal.cuh"
#include "tc.cuh"

namespace hcanet {

using bf16 = __nv_bfloat16;
namespace tc = hca::tc;

constexpr int kThreads = 128;
constexpr int kRowX = 16;   // sites per tile row (one m16 MMA tile)
constexpr int kTY = 4;      // tile rows along y

// conv layers: name order enc0, enc1, enc2, enc3, dec2, dec1, dec0
constexpr int kCI[7] = {16, 16, 32, 64, 64, 64, 32};
constexpr int kCO[7] = {16, 32, 64, 64, 64, 32, 16};

struct ParamLayout {
  long long w_off[7], b_off[7], hw_off, hb_off, total, wq_off[7], wq_total;
};

inline ParamLayout param_layout() {
  ParamLayout L{};
  long long o = 0, q = 0;
  for (int i = 0; i < 7; ++i) {
    L.w_off[i] = o;
    o += 27LL * kCO[i] * kCI[i];
    L.b_off[i] = o;
    o += kCO[i];
    L.wq_off[i] = q;
    q += 27LL * kCO[i] * kCI[i];
  }
  L.hw_off = o;
  o += 16;
  L.hb_off = o;
  o += 1;
  L.total = o;
  L.wq_total = q;
  return L;
}

// ------------------------------------------------------------ helpers ---
__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void ldsm_x4(uint32_t addr, uint32_t (&r)[4]) {
  asm volatile("ldmatrix.sync.aligned.m8n8.x4.shared.b16 {%0,%1,%2,%3}, [%4];\n"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
               : "r"(addr));
}

__device__ __forceinline__ void ldsm_x4_t(uint32_t addr, uint32_t (&r)[4]) {
  asm volatile("ldmatrix.sync.aligned.m8n8.x4.trans.shared.b16 {%0,%1,%2,%3}, [%4];\n"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
               : "r"(addr));
}

__device__ __forceinline__ void mma16816(float (&c)[4], const uint32_t (&a)[4], uint32_t b0, uint32_t b1) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
      "{%0,%1,%2,%3};\n"
      : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

// 16-byte chunk j of row h of a shared-memory matrix with C bf16 per row,
// XOR-swizzled so that 8 consecutive rows hit 8 distinct bank groups.
template <int C>
__device__ __forceinline__ int chunk_pos(int h, int j) {
  constexpr int NCH = C / 8;
  constexpr int S = NCH == 8 ? 0 : NCH == 4 ? 1 : 2;
  return h * NCH + (j ^ ((h >> S) & (NCH - 1)));
}

__device__ __forceinline__ float bfr(float v) { return __bfloat162float(__float2bfloat16_rn(v)); }

__device__ __forceinline__ uint32_t pack_bf2(float lo, float hi) {
  __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);
  return *reinterpret_cast<uint32_t*>(&v);
}

// halo geometry of a conv tile (input coordinates)
template <int TZ, bool UP>
struct Halo {
  static constexpr int HZ = UP ? TZ / 2 + 2 : TZ + 2;
  static constexpr int HY = UP ? kTY / 2 + 2 : kTY + 2;
  static constexpr int HX = UP ? kRowX / 2 + 2 : kRowX + 2;
  static constexpr int N = HZ * HY * HX;
  // halo row of tile-local output site (tz, ty, x) shifted by (dz, dy, dx)
  __device__ __forceinline__ static int row(int tz, int ty, int x, int dz, int dy, int dx) {
    if (UP) return ((((tz + dz) >> 1) + 1) * HY + (((ty + dy) >> 1) + 1)) * HX + (((x + dx) >> 1) + 1);
    return ((tz + dz + 1) * HY + (ty + dy + 1)) * HX + (x + dx + 1);
  }
};

// Stage the halo of a tile whose output origin is (z0, y0, x0) (all even).
template <int CI, int TZ, bool UP>
__device__ __forceinline__ void stage_halo(char* sm, const bf16* __restrict__ in, int Di, int Hi, int Wi, int z0,
                                           int y0, int x0) {
  using HL = Halo<TZ, UP>;
  constexpr int NCH = CI / 8;
  const int oz = UP ? (z0 >> 1) - 1 : z0 - 1;
  const int oy = UP ? (y0 >> 1) - 1 : y0 - 1;
  const int ox = UP ? (x0 >> 1) - 1 : x0 - 1;
  for (int i = threadIdx.x; i < HL::N * NCH; i += blockDim.x) {
    const int h = i / NCH, j = i - h * NCH;
    const int hx = h % HL::HX, hy = (h / HL::HX) % HL::HY, hz = h / (HL::HX * HL::HY);
    const int gz = oz + hz, gy = oy + hy, gx = ox + hx;
    uint4 v = make_uint4(0u, 0u, 0u, 0u);
    if (gz >= 0 && gz < Di && gy >= 0 && gy < Hi && gx >= 0 && gx < Wi)
      v = __ldg(reinterpret_cast<const uint4*>(in + (((long long)gz * Hi + gy) * Wi + gx) * CI) + j);
    *reinterpret_cast<uint4*>(sm + 16 * chunk_pos<CI>(h, j)) = v;
  }
}

// ----------------------------------------------------- forward / dgrad ---
enum { EPI_FWD = 0, EPI_HEAD = 1, EPI_RAW = 2, EPI_DOWN = 3 };

struct ConvArgs {
  const bf16* in;      // input (Di, Hi, Wi, CI)
  const bf16* w;       // weights (27, CO, CI)
  const float* bias;   // CO (EPI_FWD / EPI_HEAD)
  const bf16* skip;    // (D, H, W, CO) or null
  bf16* out;           // (D, H, W, CO) (EPI_FWD; EPI_HEAD: optional)
  float* out_f;        // EPI_HEAD: (D, H, W); EPI_RAW: (D, H, W, CO); EPI_DOWN: (D/2, H/2, W/2, CO)
  const float* head_w; // 16 (EPI_HEAD)
  const float* head_b; // 1 (EPI_HEAD)
  int D, H, W;         // output lattice
  int Di, Hi, Wi;      // input lattice (D/2.. when UP)
};

template <int CI, int CO, int MT, bool UP, int EPI>
constexpr int conv_smem_bytes() {
  constexpr int TZ = MT;  // 4 warps x MT rows = TZ x kTY rows
  constexpr int halo = Halo<TZ, UP>::N * CI * 2;
  constexpr int red = EPI == EPI_DOWN ? 4 * MT * 8 * CO * 4 : 0;
  return (halo > red ? halo : red) + 9 * CO * CI * 2;
}

template <int CI, int CO, int MT, bool UP, int EPI>
__global__ void __launch_bounds__(kThreads) k_conv(const ConvArgs a) {
  constexpr int TZ = MT;
  constexpr int NT = CO / 8;        // n8 tiles
  constexpr int KC = CI / 16;       // k16 steps per tap
  using HL = Halo<TZ, UP>;
  extern __shared__ __align__(128) char smem[];
  constexpr int kHaloBytes = conv_smem_bytes<CI, CO, MT, UP, EPI>() - 9 * CO * CI * 2;
  char* sh = smem;
  char* sw = smem + kHaloBytes;

  const int z0 = blockIdx.z * TZ, y0 = blockIdx.y * kTY, x0 = blockIdx.x * kRowX;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  stage_halo<CI, TZ, UP>(sh, a.in, a.Di, a.Hi, a.Wi, z0, y0, x0);

  float acc[MT][NT][4];
#pragma unroll
  for (int m = 0; m < MT; ++m)
#pragma unroll
    for (int n = 0; n < NT; ++n)
#pragma unroll
      for (int e = 0; e < 4; ++e) acc[m][n][e] = 0.f;

  const uint32_t shb = smem_u32(sh), swb = smem_u32(sw);
  const int q = lane >> 3;
  const int a_x = (lane & 7) + ((q & 1) << 3), a_j = q >> 1;        // A rows / k half
  const int b_co = (lane & 7) + ((q >> 1) << 3), b_j = q & 1;       // B rows / k half

  for (int dz = -1; dz <= 1; ++dz) {
    __syncthreads();   // previous plane's weights fully consumed (and halo staged)
    {
      constexpr int NCH = CI / 8;
      const bf16* wp = a.w + (long long)(dz + 1) * 9 * CO * CI;
      for (int i = threadIdx.x; i < 9 * CO * NCH; i += blockDim.x) {
        const int r = i / NCH, j = i - r * NCH;
        *reinterpret_cast<uint4*>(sw + 16 * chunk_pos<CI>(r, j)) =
            __ldg(reinterpret_cast<const uint4*>(wp + (long long)r * CI) + j);
      }
    }
    __syncthreads();
#pragma unroll 1
    for (int t9 = 0; t9 < 9; ++t9) {
      const int dy = t9 / 3 - 1, dx = t9 % 3 - 1;
#pragma unroll
      for (int kc = 0; kc < KC; ++kc) {
        uint32_t b[NT][2];
#pragma unroll
        for (int np = 0; np < NT / 2; ++np) {
          uint32_t r[4];
          const int row = t9 * CO + np * 16 + b_co;
          ldsm_x4(swb + 16 * chunk_pos<CI>(row, 2 * kc + b_j), r);
          b[2 * np][0] = r[0];
          b[2 * np][1] = r[1];
          b[2 * np + 1][0] = r[2];
          b[2 * np + 1][1] = r[3];
        }
#pragma unroll
        for (int m = 0; m < MT; ++m) {
          const int rr = warp * MT + m;
          const int tz = rr / kTY, ty = rr - tz * kTY;
          const int h = HL::row(tz, ty, a_x, dz, dy, dx);
          uint32_t af[4];
          ldsm_x4(shb + 16 * chunk_pos<CI>(h, 2 * kc + a_j), af);
#pragma unroll
          for (int n = 0; n < NT; ++n) mma16816(acc[m][n], af, b[n][0], b[n][1]);
        }
      }
    }
  }

  // ------------------------------------------------------------ epilogue
  const int cq = (lane & 3) * 2;
  if (EPI == EPI_DOWN) {
    __syncthreads();   // halo no longer read: reuse it for the 2x2x2 sums
    float* red = reinterpret_cast<float*>(smem);
#pragma unroll
    for (int m = 0; m < MT; ++m) {
      const int rr = warp * MT + m;
#pragma unroll
      for (int n = 0; n < NT; ++n)
#pragma unroll
        for (int hf = 0; hf < 2; ++hf) {
          // sum the x pair (lanes l and l ^ 4 hold x and x ^ 1)
          float v0 = acc[m][n][2 * hf], v1 = acc[m][n][2 * hf + 1];
          v0 += __shfl_xor_sync(0xffffffffu, v0, 4);
          v1 += __shfl_xor_sync(0xffffffffu, v1, 4);
          const int x = (lane >> 2) + 8 * hf;
          if ((x & 1) == 0) {
            float* p = red + ((rr * 8 + (x >> 1)) * CO) + n * 8 + cq;
            p[0] = v0;
            p[1] = v1;
          }
        }
    }
    __syncthreads();
    const int Dc = a.D >> 1, Hc = a.H >> 1, Wc = a.W >> 1;
    constexpr int NOUT = (TZ / 2) * (kTY / 2) * 8 * CO;
    for (int i = threadIdx.x; i < NOUT; i += blockDim.x) {
      const int co = i % CO, xp = (i / CO) % 8, cy = (i / (CO * 8)) % (kTY / 2), cz = i / (CO * 8 * (kTY / 2));
      const int r00 = (2 * cz) * kTY + 2 * cy;
      auto R = [&](int r) { return red[(r * 8 + xp) * CO + co]; };
      const float v = (R(r00) + R(r00 + 1)) + (R(r00 + kTY) + R(r00 + kTY + 1));
      const int Z = (z0 >> 1) + cz, Y = (y0 >> 1) + cy, X = (x0 >> 1) + xp;
      if (Z < Dc && Y < Hc && X < Wc) a.out_f[(((long long)Z * Hc + Y) * Wc + X) * CO + co] = v;
    }
    return;
  }

#pragma unroll
  for (int m = 0; m < MT; ++m) {
    const int rr = warp * MT + m;
    const int tz = rr / kTY, ty = rr - tz * kTY;
    const int z = z0 + tz, y = y0 + ty;
#pragma unroll
    for (int hf = 0; hf < 2; ++hf) {
      const int x = x0 + (lane >> 2) + 8 * hf;
      const bool ok = z < a.D && y < a.H && x < a.W;
      const long long site = ((long long)z * a.H + y) * a.W + x;
      float head = 0.f;
#pragma unroll
      for (int n = 0; n < NT; ++n) {
        const int co = n * 8 + cq;
        float v0 = acc[m][n][2 * hf], v1 = acc[m][n][2 * hf + 1];
        if (EPI == EPI_RAW) {
          if (ok) *reinterpret_cast<float2*>(a.out_f + site * CO + co) = make_float2(v0, v1);
          continue;
        }
        v0 += a.bias[co];
        v1 += a.bias[co + 1];
        if (a.skip && ok) {
          const __nv_bfloat162 s = *reinterpret_cast<const __nv_bfloat162*>(a.skip + site * CO + co);
          v0 += __low2float(s);
          v1 += __high2float(s);
        }
        v0 = fmaxf(v0, 0.f);
        v1 = fmaxf(v1, 0.f);
        if (ok && a.out) *reinterpret_cast<uint32_t*>(a.out + site * CO + co) = pack_bf2(v0, v1);
        if (EPI == EPI_HEAD) head += bfr(v0) * a.head_w[co] + bfr(v1) * a.head_w[co + 1];
      }
      if (EPI == EPI_HEAD) {
        head += __shfl_xor_sync(0xffffffffu, head, 1);
        head += __shfl_xor_sync(0xffffffffu, head, 2);
        if (ok && (lane & 3) == 0) a.out_f[site] = head + a.head_b[0];
      }
    }
  }
}

// ------------------------------------- forward on the fifth-gen tensor cores --
// The same convolution (EPI_FWD or EPI_HEAD) as k_conv, on tcgen05.  A tile
// is TZ planes of 8 (x) by 16 (y) output sites, each plane one M = 128 MMA
// tile (row r = x + 8 y) with its own FP32 accumulator of CO columns in
// tensor memory.  The input halo of a tile is staged in shared memory at the
// output resolution (the decoder's nearest upsampling folded into the
// staging), 16-byte channel chunks stored chunk-major: the 8 sites of a core
// matrix (8 consecutive x) are contiguous, the chunk stride is the halo
// size, the 8-site groups (rows y) are one halo row apart, and a tap's shift
// moves only the start address.  Persistent blocks: all 27 taps' weights are
// staged once as (tap, CI chunk, CO) core matrices; the next tile's halo is
// copied asynchronously (cp.async, zero-filled outside the lattice) into the
// second of two buffers while one thread per warp issues the current tile's
// 27 CI/16 MMAs of its planes (K = 16 each; each issuing thread commits to
// the mbarrier) and the warps read the accumulators back
// (bias, skip, ReLU, head) once an mbarrier signals their completion
// (bounded wait: a timeout sets *status and ends the block).  Requires
// W % 8 == 0 and H % 16 == 0.
constexpr int kTcX = 8, kTcY = 16;

template <int CI, int TZ>
constexpr uint32_t tc_halo_bytes() {
  return (uint32_t)(CI / 8) * (kTcX + 2) * (kTcY + 2) * (TZ + 2) * 16u;
}
template <int CI, int CO, int TZ>
constexpr uint32_t tc_conv_smem_bytes() {
  return 2u * tc_halo_bytes<CI, TZ>() + 27u * CI * CO * 2u + 16u;
}
template <int CO, int TZ>
constexpr uint32_t tc_cols() {
  return TZ * CO <= 32 ? 32u : TZ * CO <= 64 ? 64u : TZ * CO <= 128 ? 128u : TZ * CO <= 256 ? 256u : 512u;
}

// 16-byte copy from global to shared memory; src_bytes = 0 writes zeros
// (the source is not read).
__device__ __forceinline__ void cp_async16_zfill(void* sdst, const void* gsrc, int src_bytes) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(smem_u32(sdst)), "l"(gsrc), "r"(src_bytes)
               : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory"); }

// Start the copies of tile `tile`'s halo into sh (the tile's output origin
// from its index over (W/8, H/16, ceil(D/TZ))).
template <int CI, int TZ, bool UP>
__device__ __forceinline__ void tc_stage_halo(char* sh, const ConvArgs& a, int tile, int tx, int ty) {
  constexpr int HX = kTcX + 2, HY = kTcY + 2, HZ = TZ + 2, NH = HX * HY * HZ, NCH = CI / 8;
  const int x0 = (tile % tx) * kTcX, y0 = ((tile / tx) % ty) * kTcY, z0 = (tile / (tx * ty)) * TZ;
  for (int i = threadIdx.x; i < NH * NCH; i += blockDim.x) {
    const int h = i % NH, j = i / NH;
    const int hx = h % HX, hy = (h / HX) % HY, hz = h / (HX * HY);
    const int gz = z0 - 1 + hz, gy = y0 - 1 + hy, gx = x0 - 1 + hx;
    const bool in = gz >= 0 && gz < a.D && gy >= 0 && gy < a.H && gx >= 0 && gx < a.W;
    const int iz = UP ? gz >> 1 : gz, iy = UP ? gy >> 1 : gy, ix = UP ? gx >> 1 : gx;
    const bf16* src = in ? a.in + (((long long)iz * a.Hi + iy) * a.Wi + ix) * CI + 8 * j : a.in;
    cp_async16_zfill(sh + (uint32_t)j * (NH * 16u) + (uint32_t)h * 16u, src, in ? 16 : 0);
  }
}

template <int CI, int CO, int TZ, bool UP, int EPI>
__global__ void __launch_bounds__(128) k_conv_tc(const ConvArgs a, int* status) {
  static_assert(CI % 16 == 0 && CO % 16 == 0 && CO <= 256, "tcgen05 conv shapes");
  static_assert(EPI == EPI_FWD || EPI == EPI_HEAD, "forward epilogues only");
  constexpr int HX = kTcX + 2, HY = kTcY + 2, NH = HX * HY * (TZ + 2);
  constexpr int NCH = CI / 8;
  constexpr uint32_t HALO_B = tc_halo_bytes<CI, TZ>(), TAP_B = CI * CO * 2;
  constexpr uint32_t NCOL = tc_cols<CO, TZ>();
  extern __shared__ __align__(128) char smem[];
  char* shb0 = smem;
  char* sw = smem + 2 * HALO_B;
  uint64_t* mbar = reinterpret_cast<uint64_t*>(sw + 27 * TAP_B);
  __shared__ uint32_t tmem_holder;
  const int t = threadIdx.x, warp = t >> 5;
  const int tx = a.W / kTcX, ty = a.H / kTcY, tz = (a.D + TZ - 1) / TZ;
  const int ntiles = tx * ty * tz;
  // weights (27, CO, CI) as core matrices: (tap, CI chunk j, CO group g), once
  for (int i = t; i < 27 * CO * NCH; i += blockDim.x) {
    const int j = i % NCH, co = (i / NCH) % CO, tap = i / (NCH * CO);
    cp_async16_zfill(sw + tap * TAP_B + (uint32_t)j * (CO * 16u) + (uint32_t)(co >> 3) * 128u + (uint32_t)(co & 7) * 16u,
                     a.w + ((long long)tap * CO + co) * CI + 8 * j, 16);
  }
  if ((int)blockIdx.x < ntiles) tc_stage_halo<CI, TZ, UP>(shb0, a, blockIdx.x, tx, ty);
  cp_async_commit();
  if (t == 0) tc::mbar_init(mbar, 4);   // one arrival per issuing warp
  if (warp == 0) tc::alloc(&tmem_holder, NCOL);
  tc::fence_before();
  __syncthreads();
  tc::fence_after();
  const uint32_t tmem = tmem_holder;
  const uint32_t swb = tc::smem_u32(sw);
  int it = 0;
  bool alive = true;
  for (int tile = blockIdx.x; tile < ntiles && alive; tile += gridDim.x, ++it) {
    char* sh = shb0 + (it & 1) * HALO_B;
    const int next = tile + gridDim.x;
    if (next < ntiles) tc_stage_halo<CI, TZ, UP>(shb0 + ((it + 1) & 1) * HALO_B, a, next, tx, ty);
    cp_async_commit();
    cp_async_wait<1>();   // everything but the group just committed: this tile's halo (and the weights)
    tc::fence_async_smem();
    __syncthreads();
    const int x0 = (tile % tx) * kTcX, y0 = ((tile / tx) % ty) * kTcY, z0 = (tile / (tx * ty)) * TZ;
    if ((t & 31) == 0) {
      // lane 0 of each warp issues the MMAs of planes warp, warp + 4, ...
      constexpr uint32_t idesc = tc::idesc_bf16(128, CO);
      const uint32_t shb = tc::smem_u32(sh);
      for (int p = warp; p < TZ; p += 4)
        for (int tap = 0; tap < 27; ++tap) {
          const int dz = tap / 9 - 1, dy = (tap / 3) % 3 - 1, dx = tap % 3 - 1;
          const uint32_t shift = (uint32_t)(((p + dz + 1) * HY + (dy + 1)) * HX + (dx + 1)) * 16u;
#pragma unroll
          for (int kc = 0; kc < CI / 16; ++kc) {
            const uint64_t ad = tc::smem_desc(shb + shift + 2u * kc * (NH * 16u), NH * 16u, HX * 16u);
            const uint64_t bd = tc::smem_desc(swb + tap * TAP_B + 2u * kc * (CO * 16u), CO * 16u, 128u);
            tc::mma_bf16(tmem + (uint32_t)(p * CO), ad, bd, idesc, tap > 0 || kc > 0);
          }
        }
      tc::commit(mbar);
    }
    const bool done = tc::mbar_wait(mbar, (uint32_t)(it & 1), 1 << 22);
    if (!done && (t & 31) == 0) atomicExch(status, 1);
    alive = __syncthreads_and(done) != 0;   // one decision for the whole block
    tc::fence_after();
    if (alive) {
      const int r = t;   // tile row: x = r % 8, y = r / 8 (TMEM lane r)
      const int x = x0 + (r & 7), y = y0 + (r >> 3);
      for (int p = 0; p < TZ; ++p) {
        const int z = z0 + p;
        const bool ok = z < a.D;
        const long long site = ((long long)z * a.H + y) * a.W + x;
        float head = 0.f;
#pragma unroll
        for (int c0 = 0; c0 < CO; c0 += 16) {
          float v[16];
          tc::ld16(tmem + ((uint32_t)(32 * warp) << 16) + (uint32_t)(p * CO + c0), v);
          if (!ok) continue;
          uint32_t packed[8];
#pragma unroll
          for (int k = 0; k < 16; k += 2) {
            float v0 = v[k] + a.bias[c0 + k], v1 = v[k + 1] + a.bias[c0 + k + 1];
            if (a.skip) {
              const __nv_bfloat162 sk = *reinterpret_cast<const __nv_bfloat162*>(a.skip + site * CO + c0 + k);
              v0 += __low2float(sk);
              v1 += __high2float(sk);
            }
            v0 = fmaxf(v0, 0.f);
            v1 = fmaxf(v1, 0.f);
            packed[k / 2] = pack_bf2(v0, v1);
            if (EPI == EPI_HEAD) head += bfr(v0) * a.head_w[c0 + k] + bfr(v1) * a.head_w[c0 + k + 1];
          }
          if (a.out) {
            uint4* o = reinterpret_cast<uint4*>(a.out + site * CO + c0);
            o[0] = make_uint4(packed[0], packed[1], packed[2], packed[3]);
            o[1] = make_uint4(packed[4], packed[5], packed[6], packed[7]);
          }
        }
        if (EPI == EPI_HEAD && ok) a.out_f[site] = head + a.head_b[0];
      }
    }
    tc::fence_before();
    __syncthreads();   // accumulators read and this halo buffer free before the next tile reuses them
  }
  cp_async_wait<0>();
  __syncthreads();
  if (warp == 0) tc::dealloc(tmem, NCOL);
}

// ------------------------------------------------------------- wgrad ---
// dW[t, co, ci] = sum over sites m of gy[m, co] x[m + off_t, ci] (x = the
// layer input, upsampled on the fly when UP).  M = co (m16 tiles), N = ci,
// K = sites.  A warp owns P (tap, co-tile) units with all ci; blockIdx.y picks
// the unit group; blocks along x split the sites and write FP32 partials that
// a second kernel sums in a fixed order.
struct WgArgs {
  const bf16* in;
  const bf16* gy;
  float* part;         // [gridDim.x][27][CO][CI]
  int D, H, W, Di, Hi, Wi;
  int tiles_x, tiles_y, tiles_z;
};

constexpr int kWgMT = 2;   // 8 tile rows (TZ = 2)

template <int CI, int CO, bool UP>
constexpr int wgrad_smem_bytes() {
  return Halo<kWgMT, UP>::N * CI * 2 + 4 * kWgMT * kRowX * CO * 2;
}

template <int CI, int CO, bool UP>
__global__ void __launch_bounds__(kThreads) k_wgrad(const WgArgs a) {
  constexpr int TZ = kWgMT;
  constexpr int ROWS = 4 * kWgMT;
  constexpr int NT = CI / 8;
  constexpr int P = 128 / CI;           // units per warp
  constexpr int MTILES = CO / 16;
  constexpr int U = 27 * MTILES;
  using HL = Halo<TZ, UP>;
  extern __shared__ __align__(128) char smem[];
  char* sh = smem;
  char* sg = smem + HL::N * CI * 2;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int q = lane >> 3;

  float acc[P][NT][4];
#pragma unroll
  for (int i = 0; i < P; ++i)
#pragma unroll
    for (int n = 0; n < NT; ++n)
#pragma unroll
      for (int e = 0; e < 4; ++e) acc[i][n][e] = 0.f;

  const int ubase = (blockIdx.y * 4 + warp) * P;
  const uint32_t shb = smem_u32(sh), sgb = smem_u32(sg);
  const int n_tiles = a.tiles_x * a.tiles_y * a.tiles_z;
  for (int tile = blockIdx.x; tile < n_tiles; tile += gridDim.x) {
    const int bx = tile % a.tiles_x, by = (tile / a.tiles_x) % a.tiles_y, bz = tile / (a.tiles_x * a.tiles_y);
    const int z0 = bz * TZ, y0 = by * kTY, x0 = bx * kRowX;
    __syncthreads();
    stage_halo<CI, TZ, UP>(sh, a.in, a.Di, a.Hi, a.Wi, z0, y0, x0);
    {
      constexpr int NCH = CO / 8;
      for (int i = threadIdx.x; i < ROWS * kRowX * NCH; i += blockDim.x) {
        const int s = i / NCH, j = i - s * NCH;
        const int x = s % kRowX, rr = s / kRowX;
        const int z = z0 + rr / kTY, y = y0 + rr % kTY, xx = x0 + x;
        uint4 v = make_uint4(0u, 0u, 0u, 0u);
        if (z < a.D && y < a.H && xx < a.W)
          v = __ldg(reinterpret_cast<const uint4*>(a.gy + (((long long)z * a.H + y) * a.W + xx) * CO) + j);
        *reinterpret_cast<uint4*>(sg + 16 * chunk_pos<CO>(s, j)) = v;
      }
    }
    __syncthreads();
#pragma unroll 1
    for (int rr = 0; rr < ROWS; ++rr) {
      const int tz = rr / kTY, ty = rr - tz * kTY;
#pragma unroll
      for (int i = 0; i < P; ++i) {
        const int u = ubase + i;
        if (u >= U) break;
        const int tap = u / MTILES, mt = u - tap * MTILES;
        const int dz = tap / 9 - 1, dy = (tap / 3) % 3 - 1, dx = tap % 3 - 1;
        uint32_t af[4];
        {
          const int s = rr * kRowX + (lane & 7) + ((q >> 1) << 3);
          ldsm_x4_t(sgb + 16 * chunk_pos<CO>(s, 2 * mt + (q & 1)), af);
        }
        const int h = HL::row(tz, ty, (lane & 7) + ((q & 1) << 3), dz, dy, dx);
#pragma unroll
        for (int np = 0; np < NT / 2; ++np) {
          uint32_t r[4];
          ldsm_x4_t(shb + 16 * chunk_pos<CI>(h, 2 * np + (q >> 1)), r);
          mma16816(acc[i][2 * np], af, r[0], r[1]);
          mma16816(acc[i][2 * np + 1], af, r[2], r[3]);
        }
      }
    }
  }
  float* part = a.part + (long long)blockIdx.x * 27 * CO * CI;
  const int cq = (lane & 3) * 2;
#pragma unroll
  for (int i = 0; i < P; ++i) {
    const int u = ubase + i;
    if (u >= U) break;
    const int tap = u / MTILES, mt = u - tap * MTILES;
#pragma unroll
    for (int n = 0; n < NT; ++n)
#pragma unroll
      for (int hf = 0; hf < 2; ++hf) {
        const int co = mt * 16 + (lane >> 2) + 8 * hf, ci = n * 8 + cq;
        *reinterpret_cast<float2*>(part + ((long long)tap * CO + co) * CI + ci) =
            make_float2(acc[i][n][2 * hf], acc[i][n][2 * hf + 1]);
      }
  }
}

// dst[i] = sum_g part[g][i], g = 0 .. G-1 in order (deterministic split-K reduce)
__global__ void k_sum_parts(const float* __restrict__ part, int G, long long n, float* __restrict__ dst) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    float s = 0.f;
    for (int g = 0; g < G; ++g) s += part[(long long)g * n + i];
    dst[i] = s;
  }
}

// ------------------------------------------------------- elementwise ---
// 2x2x2 average pooling, children summed in a fixed order.
template <int C>
__global__ void k_pool(const bf16* __restrict__ in, bf16* __restrict__ out, int D, int H, int W) {
  constexpr int NCH = C / 8;
  const int Dc = D / 2, Hc = H / 2, Wc = W / 2;
  const long long n = (long long)Dc * Hc * Wc * NCH;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const int j = (int)(i % NCH);
    const long long s = i / NCH;
    const int X = (int)(s % Wc), Y = (int)((s / Wc) % Hc), Z = (int)(s / ((long long)Wc * Hc));
    float acc[8];
#pragma unroll
    for (int e = 0; e < 8; ++e) acc[e] = 0.f;
#pragma unroll
    for (int c = 0; c < 8; ++c) {
      const int z = 2 * Z + (c >> 2), y = 2 * Y + ((c >> 1) & 1), x = 2 * X + (c & 1);
      const uint4 v = __ldg(reinterpret_cast<const uint4*>(in + (((long long)z * H + y) * W + x) * C) + j);
      const __nv_bfloat162* p = reinterpret_cast<const __nv_bfloat162*>(&v);
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        acc[2 * e] += __low2float(p[e]);
        acc[2 * e + 1] += __high2float(p[e]);
      }
    }
    uint4 o;
    uint32_t* po = reinterpret_cast<uint32_t*>(&o);
#pragma unroll
    for (int e = 0; e < 4; ++e) po[e] = pack_bf2(acc[2 * e] * 0.125f, acc[2 * e + 1] * 0.125f);
    *reinterpret_cast<uint4*>(out + s * C + j * 8) = o;
  }
}

constexpr int kEwThreads = 256;

// Per-block channel sums written to part[blockIdx.x][C] in a fixed order:
// vals[t][c] (one row of 8 channels per thread for the channel chunk j(t)).
template <int C>
__device__ __forceinline__ void block_channel_sums(float (&v)[8], int j, float* __restrict__ part, float* sbuf) {
  // sbuf: kEwThreads * 8 floats
#pragma unroll
  for (int e = 0; e < 8; ++e) sbuf[threadIdx.x * 8 + e] = v[e];
  __syncthreads();
  constexpr int NCH = C / 8;
  for (int c = threadIdx.x; c < C; c += blockDim.x) {
    const int jj = c / 8, e = c % 8;
    float s = 0.f;
    for (int t = jj; t < (int)blockDim.x; t += NCH) s += sbuf[t * 8 + e];
    part[(long long)blockIdx.x * C + c] = s;
  }
  (void)j;
}

// Gradient of a layer's pre-activation from the raw gradient of its output:
//   POOL = 0: g[i] = [y_i > 0] graw[i]                       (same lattice)
//   POOL = 1: g[i] = [y_i > 0] (skip[i] + graw[parent(i)] / 8) (graw one level down)
// y is the layer's stored BF16 output; skip may alias g.  Per-block channel
// sums of g go to part (the bias gradient).
template <int C, int POOL>
__global__ void __launch_bounds__(kEwThreads) k_combine(const float* __restrict__ graw, const bf16* __restrict__ y,
                                                        const bf16* skip, bf16* g, int D, int H, int W,
                                                        float* __restrict__ part) {
  __shared__ float sbuf[kEwThreads * 8];
  constexpr int NCH = C / 8;
  const long long n = (long long)D * H * W * NCH;
  const long long stride = (long long)gridDim.x * blockDim.x;
  const long long i0 = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  const int j = (int)(i0 % NCH);   // fixed per thread: stride is a multiple of NCH
  float bs[8];
#pragma unroll
  for (int e = 0; e < 8; ++e) bs[e] = 0.f;
  for (long long i = i0; i < n; i += stride) {
    const long long s = i / NCH;
    const uint4 yv = *reinterpret_cast<const uint4*>(y + s * C + j * 8);
    const __nv_bfloat162* py = reinterpret_cast<const __nv_bfloat162*>(&yv);
    float gv[8];
    if (POOL) {
      const int x = (int)(s % W), yy = (int)((s / W) % H), z = (int)(s / ((long long)W * H));
      const long long ps = (((long long)(z >> 1) * (H >> 1) + (yy >> 1)) * (W >> 1) + (x >> 1));
      const float4 g0 = *reinterpret_cast<const float4*>(graw + ps * C + j * 8);
      const float4 g1 = *reinterpret_cast<const float4*>(graw + ps * C + j * 8 + 4);
      const uint4 sv = *reinterpret_cast<const uint4*>(skip + s * C + j * 8);
      const __nv_bfloat162* pk = reinterpret_cast<const __nv_bfloat162*>(&sv);
      const float gr[8] = {g0.x, g0.y, g0.z, g0.w, g1.x, g1.y, g1.z, g1.w};
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        gv[2 * e] = __low2float(pk[e]) + gr[2 * e] * 0.125f;
        gv[2 * e + 1] = __high2float(pk[e]) + gr[2 * e + 1] * 0.125f;
      }
    } else {
      const float4 g0 = *reinterpret_cast<const float4*>(graw + s * C + j * 8);
      const float4 g1 = *reinterpret_cast<const float4*>(graw + s * C + j * 8 + 4);
      const float gr[8] = {g0.x, g0.y, g0.z, g0.w, g1.x, g1.y, g1.z, g1.w};
#pragma unroll
      for (int e = 0; e < 8; ++e) gv[e] = gr[e];
    }
    uint4 o;
    uint32_t* po = reinterpret_cast<uint32_t*>(&o);
#pragma unroll
    for (int e = 0; e < 4; ++e) {
      const float a0 = __low2float(py[e]) > 0.f ? gv[2 * e] : 0.f;
      const float a1 = __high2float(py[e]) > 0.f ? gv[2 * e + 1] : 0.f;
      bs[2 * e] += a0;
      bs[2 * e + 1] += a1;
      po[e] = pack_bf2(a0, a1);
    }
    *reinterpret_cast<uint4*>(g + s * C + j * 8) = o;
  }
  block_channel_sums<C>(bs, j, part, sbuf);
}

// Head and loss: out = d0 . hw + hb was written by the last convolution.
// gout = 2 (out - target) / N (or gbuf, the residual loss's gradient);
// gd0 = [d0 > 0] gout hw.  Per-block partials:
// [0,16) head-weight gradient, 16 head-bias gradient, [17,33) dec0 bias
// gradient, 33 sum of squared errors.
constexpr int kHeadParts = 34;

__global__ void __launch_bounds__(kEwThreads) k_head_bwd(const bf16* __restrict__ d0, const float* __restrict__ out,
                                                         const float* __restrict__ target, const float* __restrict__ gbuf,
                                                         const float* __restrict__ hw, long long N,
                                                         bf16* __restrict__ gd0, float* __restrict__ part) {
  __shared__ float sbuf[kEwThreads];
  float acc[kHeadParts];
#pragma unroll
  for (int k = 0; k < kHeadParts; ++k) acc[k] = 0.f;
  const float scale = 2.0f / (float)N;
  for (long long s = blockIdx.x * (long long)blockDim.x + threadIdx.x; s < N; s += (long long)gridDim.x * blockDim.x) {
    float go;
    if (gbuf) {
      go = gbuf[s];
    } else {
      const float diff = out[s] - target[s];
      go = scale * diff;
      acc[33] += diff * diff;
    }
    acc[16] += go;
    const uint4* pd = reinterpret_cast<const uint4*>(d0 + s * 16);
    uint4 o[2];
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const uint4 v = pd[h];
      const __nv_bfloat162* p = reinterpret_cast<const __nv_bfloat162*>(&v);
      uint32_t* po = reinterpret_cast<uint32_t*>(&o[h]);
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        const int c = h * 8 + 2 * e;
        const float y0 = __low2float(p[e]), y1 = __high2float(p[e]);
        acc[c] += y0 * go;
        acc[c + 1] += y1 * go;
        const float g0 = y0 > 0.f ? go * hw[c] : 0.f;
        const float g1 = y1 > 0.f ? go * hw[c + 1] : 0.f;
        acc[17 + c] += g0;
        acc[17 + c + 1] += g1;
        po[e] = pack_bf2(g0, g1);
      }
    }
    reinterpret_cast<uint4*>(gd0 + s * 16)[0] = o[0];
    reinterpret_cast<uint4*>(gd0 + s * 16)[1] = o[1];
  }
  for (int k = 0; k < kHeadParts; ++k) {
    sbuf[threadIdx.x] = acc[k];
    __syncthreads();
    for (int w = blockDim.x / 2; w > 0; w >>= 1) {
      if ((int)threadIdx.x < w) sbuf[threadIdx.x] += sbuf[threadIdx.x + w];
      __syncthreads();
    }
    if (threadIdx.x == 0) part[(long long)blockIdx.x * kHeadParts + k] = sbuf[0];
    __syncthreads();
  }
}

// Sum per-block partials part[b][k] (b = 0 .. nb-1 in order) into dst[map(k)].
__global__ void k_scatter_parts(const float* __restrict__ part, int nb, int width, float* __restrict__ grads,
                                const long long* __restrict__ dst_index, float* __restrict__ loss, float loss_scale) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= width) return;
  float s = 0.f;
  for (int b = 0; b < nb; ++b) s += part[(long long)b * width + k];
  const long long d = dst_index[k];
  if (d >= 0) grads[d] = s;
  else if (loss) *loss = s * loss_scale;
}

// Training target NET_SCALE (K_new - K_prev) / K0.
__global__ void k_target(const float* __restrict__ Kp, const float* __restrict__ Kn, long long n, float scale,
                         float* __restrict__ t) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    t[i] = scale * (Kn[i] - Kp[i]);
}

// Residual loss L = mean(u^2), u = A e / c, e = out - target, A the oxygen
// operator lagged at K_prev (dense lattice), c = D_K / dx^2.
__device__ __forceinline__ float o2_diag(const FeatureArgs& f, const float* __restrict__ Kp, long long e, int cnt,
                                         float cpl) {
  const uint8_t st = f.state[e];
  const bool consumer = st == HCA_PROLIF || st == HCA_QUIESC || st == HCA_STROMA;
  const float reac = (consumer ? (float)f.phi_K / ((float)f.K1 + Kp[e]) : 0.f) + (st == HCA_VESSEL ? (float)f.r_K : 0.f);
  return cpl * (float)cnt + reac;
}

// v = (A w) / c on the dense lattice, w = a - b (b may be null).
__device__ __forceinline__ float apply_scaled(const FeatureArgs& f, const float* __restrict__ Kp,
                                              const float* __restrict__ a, const float* __restrict__ b, long long s,
                                              float cpl) {
  const int xx = (int)(s % f.nx), yy = (int)((s / f.nx) % f.ny), zz = (int)(s / ((long long)f.nx * f.ny));
  const long long sy = f.nx, sz = (long long)f.nx * f.ny;
  auto w = [&](long long i) { return b ? a[i] - b[i] : a[i]; };
  float nb = 0.f;
  int cnt = 0;
  if (xx > 0) { nb += w(s - 1); ++cnt; }
  if (xx < f.nx - 1) { nb += w(s + 1); ++cnt; }
  if (yy > 0) { nb += w(s - sy); ++cnt; }
  if (yy < f.ny - 1) { nb += w(s + sy); ++cnt; }
  if (zz > 0) { nb += w(s - sz); ++cnt; }
  if (zz < f.nz - 1) { nb += w(s + sz); ++cnt; }
  const float d = o2_diag(f, Kp, s, cnt, cpl);
  return (d * w(s) - cpl * nb) / cpl;
}

__global__ void __launch_bounds__(kEwThreads) k_res_u(FeatureArgs f, const float* __restrict__ Kp,
                                                      const float* __restrict__ out, const float* __restrict__ tgt,
                                                      float* __restrict__ u, float* __restrict__ part) {
  __shared__ float sb[kEwThreads];
  const long long n = (long long)f.nx * f.ny * f.nz;
  const float cpl = (float)(f.D_K / (f.dx * f.dx));
  float acc = 0.f;
  for (long long s = blockIdx.x * (long long)blockDim.x + threadIdx.x; s < n; s += (long long)gridDim.x * blockDim.x) {
    const float v = apply_scaled(f, Kp, out, tgt, s, cpl);
    u[s] = v;
    acc += v * v;
  }
  sb[threadIdx.x] = acc;
  __syncthreads();
  for (int w = blockDim.x / 2; w > 0; w >>= 1) {
    if ((int)threadIdx.x < w) sb[threadIdx.x] += sb[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) part[blockIdx.x] = sb[0];
}

// dL/dout of L = w_mse mean(e^2) + w_res mean(u^2):
//   2 w_mse e / N + 2 w_res (A u) / (c N); per-block sums of e^2 into part.
__global__ void __launch_bounds__(kEwThreads) k_loss_grad(FeatureArgs f, const float* __restrict__ Kp,
                                                          const float* __restrict__ out, const float* __restrict__ tgt,
                                                          const float* __restrict__ u, float w_mse, float w_res,
                                                          float* __restrict__ g, float* __restrict__ part) {
  __shared__ float sb[kEwThreads];
  const long long n = (long long)f.nx * f.ny * f.nz;
  const float cpl = (float)(f.D_K / (f.dx * f.dx));
  const float sc = 2.0f / (float)n;
  float acc = 0.f;
  for (long long s = blockIdx.x * (long long)blockDim.x + threadIdx.x; s < n; s += (long long)gridDim.x * blockDim.x) {
    const float e = out[s] - tgt[s];
    acc += e * e;
    float v = w_mse * sc * e;
    if (w_res != 0.f) v += w_res * sc * apply_scaled(f, Kp, u, nullptr, s, cpl);
    g[s] = v;
  }
  sb[threadIdx.x] = acc;
  __syncthreads();
  for (int w = blockDim.x / 2; w > 0; w >>= 1) {
    if ((int)threadIdx.x < w) sb[threadIdx.x] += sb[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) part[blockIdx.x] = sb[0];
}

// loss = sa * sum(pa[0..nb)) + sb * sum(pb[0..nb)), blocks in order
__global__ void k_sum_loss(const float* __restrict__ pa, int nb, float sa, const float* __restrict__ pb, float sb,
                           float* __restrict__ loss) {
  if (threadIdx.x || blockIdx.x) return;
  float a = 0.f, b = 0.f;
  for (int i = 0; i < nb; ++i) {
    a += pa[i];
    b += pb[i];
  }
  *loss = sa * a + sb * b;
}

// Adam (Kingma & Ba 2015, Algorithm 1) with FP32 master weights.
__global__ void k_adam(float* __restrict__ w, const float* __restrict__ g, float* __restrict__ m,
                       float* __restrict__ v, long long n, float lr, float b1, float b2, float eps, float c1,
                       float c2) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const float gi = g[i];
    const float mi = b1 * m[i] + (1.f - b1) * gi;
    const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    const float mh = mi / c1, vh = vi / c2;
    w[i] -= lr * mh / (sqrtf(vh) + eps);
  }
}

// BF16 copies of the conv weights: wq (27, CO, CI) and wt (27, CI, CO) with
// wt[t][ci][co] = w[26 - t][co][ci] (the input-gradient convolution).
struct QuantTable {
  long long w_off[7], q_off[7];
  int ci[7], co[7];
};

__global__ void k_quantize(const float* __restrict__ params, QuantTable T, bf16* __restrict__ wq,
                           bf16* __restrict__ wt, long long total) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total; i += (long long)gridDim.x * blockDim.x) {
    int l = 0;
    while (l < 6 && i >= T.q_off[l + 1]) ++l;
    const long long k = i - T.q_off[l];
    const int CI = T.ci[l], CO = T.co[l];
    const int ci = (int)(k % CI), co = (int)((k / CI) % CO), t = (int)(k / ((long long)CI * CO));
    const float v = params[T.w_off[l] + k];
    wq[i] = __float2bfloat16_rn(v);
    wt[T.q_off[l] + ((long long)(26 - t) * CI + ci) * CO + co] = __float2bfloat16_rn(v);
  }
}

// ------------------------------------------------------------ features ---
// Network input for one oxygen solve: one-hot state (6), perf, K_prev / K0,
// NET_SCALE (b - A K_prev) / (diag(A) K0) for the operator of Eq. (oxygen)
// lagged at K_prev (7-point stencil, homogeneous Neumann), zeros.  Fields are
// read with a row pitch (the solver's padded layout or dense); x is dense.
template <typename T>
__global__ void k_features(FeatureArgs f, const T* __restrict__ K, bf16* __restrict__ x) {
  const long long n = (long long)f.nx * f.ny * f.nz;
  const long long sy = f.pitch, sz = (long long)f.pitch * f.ny;
  const float cpl = (float)(f.D_K / (f.dx * f.dx));
  for (long long s = blockIdx.x * (long long)blockDim.x + threadIdx.x; s < n; s += (long long)gridDim.x * blockDim.x) {
    const int xx = (int)(s % f.nx), yy = (int)((s / f.nx) % f.ny), zz = (int)(s / ((long long)f.nx * f.ny));
    const long long e = f.base + xx + sy * yy + sz * zz;
    const uint8_t st = f.state[e];
    const float k = (float)K[e];
    float nb = 0.f;
    int cnt = 0;
    if (xx > 0) { nb += (float)K[e - 1]; ++cnt; }
    if (xx < f.nx - 1) { nb += (float)K[e + 1]; ++cnt; }
    if (yy > 0) { nb += (float)K[e - sy]; ++cnt; }
    if (yy < f.ny - 1) { nb += (float)K[e + sy]; ++cnt; }
    if (zz > 0) { nb += (float)K[e - sz]; ++cnt; }
    if (zz < f.nz - 1) { nb += (float)K[e + sz]; ++cnt; }
    const bool consumer = st == HCA_PROLIF || st == HCA_QUIESC || st == HCA_STROMA;
    const bool vessel = st == HCA_VESSEL;
    const float reac = (consumer ? (float)f.phi_K / ((float)f.K1 + k) : 0.f) + (vessel ? (float)f.r_K : 0.f);
    const float d = cpl * (float)cnt + reac;
    const float b = vessel ? (float)(f.r_K * f.K0) : 0.f;
    const float r = b - (d * k - cpl * nb);
    const float ch8 = d != 0.f ? (float)kNetScale * r / (d * (float)f.K0) : 0.f;
    uint4 o[2];
    uint32_t* po = reinterpret_cast<uint32_t*>(o);
    po[0] = pack_bf2(st == 0 ? 1.f : 0.f, st == 1 ? 1.f : 0.f);
    po[1] = pack_bf2(st == 2 ? 1.f : 0.f, st == 3 ? 1.f : 0.f);
    po[2] = pack_bf2(st == 4 ? 1.f : 0.f, st == 5 ? 1.f : 0.f);
    po[3] = pack_bf2((float)static_cast<const T*>(f.perf)[e], k / (float)f.K0);
    po[4] = pack_bf2(ch8, 0.f);
    po[5] = po[6] = po[7] = 0u;
    reinterpret_cast<uint4*>(x + s * 16)[0] = o[0];
    reinterpret_cast<uint4*>(x + s * 16)[1] = o[1];
  }
}

// ----------------------------------------------- warm-start selection ---
// cand = K_prev + (K0 / NET_SCALE) out (FP64); lag = K_prev in the solver's
// storage type (the point the consumption term is linearised about).
template <typename T>
__global__ void k_ws_candidate(FeatureArgs f, const T* __restrict__ K, const float* __restrict__ K_lo,
                               const float* __restrict__ out, double* __restrict__ cand, T* __restrict__ lag) {
  const long long n = (long long)f.nx * f.ny * f.nz;
  const long long sy = f.pitch, sz = (long long)f.pitch * f.ny;
  for (long long s = blockIdx.x * (long long)blockDim.x + threadIdx.x; s < n; s += (long long)gridDim.x * blockDim.x) {
    const int xx = (int)(s % f.nx), yy = (int)((s / f.nx) % f.ny), zz = (int)(s / ((long long)f.nx * f.ny));
    const long long e = f.base + xx + sy * yy + sz * zz;
    const double kp = (double)K[e] + (K_lo ? (double)K_lo[e] : 0.0);
    cand[e] = kp + f.K0 / kNetScale * (double)out[s];
    lag[e] = (T)kp;
  }
}

// Per-block partial sums of |b - A u|^2 for u = K_prev and u = cand, and |b|^2,
// FP64, A lagged at K_prev.
template <typename T>
__global__ void __launch_bounds__(kEwThreads) k_ws_norms(FeatureArgs f, const T* __restrict__ K,
                                                         const float* __restrict__ K_lo, const double* __restrict__ cand,
                                                         double* __restrict__ part) {
  __shared__ double sb[3][kEwThreads];
  const long long n = (long long)f.nx * f.ny * f.nz;
  const long long sy = f.pitch, sz = (long long)f.pitch * f.ny;
  const double cpl = f.D_K / (f.dx * f.dx);
  double a0 = 0.0, a1 = 0.0, a2 = 0.0;
  auto kp = [&](long long e) { return (double)K[e] + (K_lo ? (double)K_lo[e] : 0.0); };
  for (long long s = blockIdx.x * (long long)blockDim.x + threadIdx.x; s < n; s += (long long)gridDim.x * blockDim.x) {
    const int xx = (int)(s % f.nx), yy = (int)((s / f.nx) % f.ny), zz = (int)(s / ((long long)f.nx * f.ny));
    const long long e = f.base + xx + sy * yy + sz * zz;
    const uint8_t st = f.state[e];
    const double k = kp(e);
    double nbp = 0.0, nbc = 0.0;
    int cnt = 0;
    const long long off[6] = {-1, 1, -sy, sy, -sz, sz};
    const bool in[6] = {xx > 0, xx < f.nx - 1, yy > 0, yy < f.ny - 1, zz > 0, zz < f.nz - 1};
#pragma unroll
    for (int q = 0; q < 6; ++q)
      if (in[q]) {
        nbp += kp(e + off[q]);
        nbc += cand[e + off[q]];
        ++cnt;
      }
    const bool consumer = st == HCA_PROLIF || st == HCA_QUIESC || st == HCA_STROMA;
    const bool vessel = st == HCA_VESSEL;
    const double reac = (consumer ? f.phi_K / (f.K1 + k) : 0.0) + (vessel ? f.r_K : 0.0);
    const double d = cpl * cnt + reac;
    const double b = vessel ? f.r_K * f.K0 : 0.0;
    const double rp = b - (d * k - cpl * nbp);
    const double rc = b - (d * cand[e] - cpl * nbc);
    a0 += rp * rp;
    a1 += rc * rc;
    a2 += b * b;
  }
  sb[0][threadIdx.x] = a0;
  sb[1][threadIdx.x] = a1;
  sb[2][threadIdx.x] = a2;
  __syncthreads();
  for (int w = blockDim.x / 2; w > 0; w >>= 1) {
    if ((int)threadIdx.x < w)
      for (int k = 0; k < 3; ++k) sb[k][threadIdx.x] += sb[k][threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x < 3) part[blockIdx.x * 3 + threadIdx.x] = sb[threadIdx.x][0];
}

__global__ void k_ws_decide(const double* __restrict__ part, int nb, int always, WsResult* __restrict__ res) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  double s[3] = {0.0, 0.0, 0.0};
  for (int b = 0; b < nb; ++b)
    for (int k = 0; k < 3; ++k) s[k] += part[b * 3 + k];
  const double bn = s[2] > 0.0 ? sqrt(s[2]) : 1.0;
  res->r0_prev = sqrt(s[0]) / bn;
  res->r0_learned = sqrt(s[1]) / bn;
  res->used = always || ((s[1] == s[1]) && s[1] < s[0]) ? 1 : 0;
}

template <typename T>
__global__ void k_ws_apply(FeatureArgs f, const WsResult* __restrict__ res, const double* __restrict__ cand,
                           T* __restrict__ K, float* __restrict__ K_lo) {
  if (!res->used) return;
  const long long n = (long long)f.nx * f.ny * f.nz;
  const long long sy = f.pitch, sz = (long long)f.pitch * f.ny;
  for (long long s = blockIdx.x * (long long)blockDim.x + threadIdx.x; s < n; s += (long long)gridDim.x * blockDim.x) {
    const int xx = (int)(s % f.nx), yy = (int)((s / f.nx) % f.ny), zz = (int)(s / ((long long)f.nx * f.ny));
    const long long e = f.base + xx + sy * yy + sz * zz;
    const double c = cand[e];
    const T hi = (T)c;
    K[e] = hi;
    if (K_lo) K_lo[e] = (float)(c - (double)hi);
  }
}

}  // namespace hcanet

// ====================================================================== host
using namespace hcanet;

struct hca_net {
  int D = 0, H = 0, W = 0;
  int device = 0;
  int sm_count = 148;
  cudaStream_t stream = nullptr;
  ParamLayout L{};
  int Ld[4], Lh[4], Lw[4];
  long long Ln[4];
  std::vector<void*> allocs;
  float *params = nullptr, *grads = nullptr, *m = nullptr, *v = nullptr;
  long long adam_t = 0;
  bf16 *wq = nullptr, *wt = nullptr;
  bf16 *x = nullptr, *e0 = nullptr, *p0 = nullptr, *e1 = nullptr, *p1 = nullptr, *e2 = nullptr, *p2 = nullptr,
       *e3 = nullptr, *d2 = nullptr, *d1 = nullptr, *d0 = nullptr;
  // gradients with respect to each convolution's output (BF16): g0..g2 the
  // decoder's (dec0, dec1, dec2), g3 enc3's, ge0..ge2 the encoder's after
  // the skip path's gradient is added (enc0, enc1, enc2)
  bf16 *g0 = nullptr, *g1 = nullptr, *g2 = nullptr, *g3 = nullptr;
  bf16 *ge0 = nullptr, *ge1 = nullptr, *ge2 = nullptr;
  float *out = nullptr, *tgt = nullptr, *ru = nullptr, *rg = nullptr, *graw = nullptr, *wpart = nullptr, *bpart = nullptr, *loss = nullptr;
  long long wpart_n = 0;
  int bpart_blocks = 0;
  long long* head_index = nullptr;   // device: destination of the 34 head partials
  long long* bias_index = nullptr;   // device: 7 x 64 destinations of the bias partials
  bool trainable = false;
  // the full-resolution layers (enc0, dec0 + head) of the forward pass on the
  // fifth-generation tensor cores (k_conv_tc); tc_status: set by a kernel whose
  // completion wait timed out
  bool use_tc = false;
  int* tc_status = nullptr;
};

namespace {

int net_alloc(hca_net* n, void** p, size_t bytes) {
  if (cudaMalloc(p, bytes ? bytes : 16) != cudaSuccess) {
    cudaGetLastError();
    return HCA_ERR_OOM;
  }
  n->allocs.push_back(*p);
  return HCA_OK;
}

#define NET_ALLOC(ptr, bytes)                                             \
  do {                                                                    \
    void* _p = nullptr;                                                   \
    int _rc = net_alloc(n, &_p, (bytes));                                 \
    if (_rc) return _rc;                                                  \
    ptr = static_cast<decltype(ptr)>(_p);                                 \
  } while (0)

#define NET_CUDA(x)                         \
  do {                                      \
    cudaError_t _e = (x);                   \
    if (_e != cudaSuccess) {                \
      cudaGetLastError();                   \
      return HCA_ERR_CUDA;                  \
    }                                       \
  } while (0)

int ew_blocks(long long n, int sm) {
  const long long b = (n + kEwThreads - 1) / kEwThreads;
  return (int)std::max(1LL, std::min(b, (long long)sm * 8));
}

template <int CI, int CO, int MT, bool UP, int EPI>
int conv_attr() {
  constexpr int sm = conv_smem_bytes<CI, CO, MT, UP, EPI>();
  NET_CUDA(cudaFuncSetAttribute(k_conv<CI, CO, MT, UP, EPI>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm));
  return HCA_OK;
}

template <int CI, int CO, bool UP>
int wgrad_attr() {
  constexpr int sm = wgrad_smem_bytes<CI, CO, UP>();
  NET_CUDA(cudaFuncSetAttribute(k_wgrad<CI, CO, UP>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm));
  return HCA_OK;
}

int set_attributes() {
  int rc = 0;
  if ((rc = conv_attr<16, 16, 4, false, EPI_FWD>())) return rc;
  if ((rc = conv_attr<16, 32, 4, false, EPI_FWD>())) return rc;
  if ((rc = conv_attr<32, 64, 2, false, EPI_FWD>())) return rc;
  if ((rc = conv_attr<64, 64, 2, false, EPI_FWD>())) return rc;
  if ((rc = conv_attr<64, 64, 2, true, EPI_FWD>())) return rc;
  if ((rc = conv_attr<64, 32, 4, true, EPI_FWD>())) return rc;
  if ((rc = conv_attr<32, 16, 4, true, EPI_HEAD>())) return rc;
  if ((rc = conv_attr<16, 32, 4, false, EPI_DOWN>())) return rc;
  if ((rc = conv_attr<32, 64, 2, false, EPI_DOWN>())) return rc;
  if ((rc = conv_attr<64, 64, 2, false, EPI_DOWN>())) return rc;
  if ((rc = conv_attr<64, 64, 2, false, EPI_RAW>())) return rc;
  if ((rc = conv_attr<64, 32, 4, false, EPI_RAW>())) return rc;
  if ((rc = conv_attr<32, 16, 4, false, EPI_RAW>())) return rc;
  if ((rc = wgrad_attr<16, 16, false>())) return rc;
  if ((rc = wgrad_attr<16, 32, false>())) return rc;
  if ((rc = wgrad_attr<32, 64, false>())) return rc;
  if ((rc = wgrad_attr<64, 64, false>())) return rc;
  if ((rc = wgrad_attr<64, 64, true>())) return rc;
  if ((rc = wgrad_attr<64, 32, true>())) return rc;
  if ((rc = wgrad_attr<32, 16, true>())) return rc;
  return HCA_OK;
}

template <int CI, int CO, int TZ, bool UP, int EPI>
bool conv_tc_attr() {
  if (cudaFuncSetAttribute(k_conv_tc<CI, CO, TZ, UP, EPI>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)tc_conv_smem_bytes<CI, CO, TZ>()) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return true;
}

// One tcgen05 convolution launch; (D, H, W) is the output lattice.
template <int CI, int CO, int TZ, bool UP, int EPI>
void conv_tc(cudaStream_t s, int* status, const bf16* in, const bf16* w, const float* bias, const bf16* skip,
             bf16* out, float* out_f, const float* hw, const float* hb, int D, int H, int W) {
  ConvArgs a;
  a.in = in;
  a.w = w;
  a.bias = bias;
  a.skip = skip;
  a.out = out;
  a.out_f = out_f;
  a.head_w = hw;
  a.head_b = hb;
  a.D = D;
  a.H = H;
  a.W = W;
  a.Di = UP ? D / 2 : D;
  a.Hi = UP ? H / 2 : H;
  a.Wi = UP ? W / 2 : W;
  const int ntiles = (W / kTcX) * (H / kTcY) * ((D + TZ - 1) / TZ);
  int per = 1;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_conv_tc<CI, CO, TZ, UP, EPI>, 128,
                                                    tc_conv_smem_bytes<CI, CO, TZ>()) != cudaSuccess || per < 1) {
    cudaGetLastError();
    per = 1;
  }
  int dev = 0, sms = 148;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const int grid = std::min(ntiles, per * sms);
  k_conv_tc<CI, CO, TZ, UP, EPI><<<grid, 128, tc_conv_smem_bytes<CI, CO, TZ>(), s>>>(a, status);
}

// One convolution launch; (D, H, W) is the output lattice.
template <int CI, int CO, int MT, bool UP, int EPI>
void conv(cudaStream_t s, const bf16* in, const bf16* w, const float* bias, const bf16* skip, bf16* out,
          float* out_f, const float* hw, const float* hb, int D, int H, int W) {
  ConvArgs a;
  a.in = in;
  a.w = w;
  a.bias = bias;
  a.skip = skip;
  a.out = out;
  a.out_f = out_f;
  a.head_w = hw;
  a.head_b = hb;
  a.D = D;
  a.H = H;
  a.W = W;
  a.Di = UP ? D / 2 : D;
  a.Hi = UP ? H / 2 : H;
  a.Wi = UP ? W / 2 : W;
  const dim3 grid((W + kRowX - 1) / kRowX, (H + kTY - 1) / kTY, (D + MT - 1) / MT);
  k_conv<CI, CO, MT, UP, EPI><<<grid, kThreads, conv_smem_bytes<CI, CO, MT, UP, EPI>(), s>>>(a);
}

// Weight gradient of one layer into grads[w_off ...]; (D, H, W) = output lattice.
template <int CI, int CO, bool UP>
void wgrad(hca_net* n, cudaStream_t s, const bf16* in, const bf16* gy, int D, int H, int W, float* dst) {
  WgArgs a;
  a.in = in;
  a.gy = gy;
  a.part = n->wpart;
  a.D = D;
  a.H = H;
  a.W = W;
  a.Di = UP ? D / 2 : D;
  a.Hi = UP ? H / 2 : H;
  a.Wi = UP ? W / 2 : W;
  a.tiles_x = (W + kRowX - 1) / kRowX;
  a.tiles_y = (H + kTY - 1) / kTY;
  a.tiles_z = (D + kWgMT - 1) / kWgMT;
  constexpr int P = 128 / CI;
  constexpr int U = 27 * (CO / 16);
  const int gy_blocks = (U + 4 * P - 1) / (4 * P);
  const int n_tiles = a.tiles_x * a.tiles_y * a.tiles_z;
  const long long per = 27LL * CO * CI;
  int G = std::max(1, std::min(n_tiles, 2 * n->sm_count / gy_blocks));
  G = (int)std::min<long long>(G, n->wpart_n / per);
  k_wgrad<CI, CO, UP><<<dim3(G, gy_blocks), kThreads, wgrad_smem_bytes<CI, CO, UP>(), s>>>(a);
  k_sum_parts<<<ew_blocks(per, n->sm_count), kEwThreads, 0, s>>>(n->wpart, G, per, dst);
}

template <int C, int POOL>
void combine(hca_net* n, cudaStream_t s, const float* graw, const bf16* y, const bf16* skip, bf16* g, int lvl,
             int layer) {
  const long long cnt = n->Ln[lvl] * (C / 8);
  const int nb = std::min(ew_blocks(cnt, n->sm_count), n->bpart_blocks);
  k_combine<C, POOL><<<nb, kEwThreads, 0, s>>>(graw, y, skip, g, n->Ld[lvl], n->Lh[lvl], n->Lw[lvl], n->bpart);
  k_scatter_parts<<<1, 64, 0, s>>>(n->bpart, nb, C, n->grads, n->bias_index + 64 * layer, nullptr, 0.f);
}

template <int C>
void pool(hca_net* n, cudaStream_t s, const bf16* in, bf16* out, int lvl) {
  const long long cnt = n->Ln[lvl + 1] * (C / 8);
  k_pool<C><<<ew_blocks(cnt, n->sm_count), kEwThreads, 0, s>>>(in, out, n->Ld[lvl], n->Lh[lvl], n->Lw[lvl]);
}

const bf16* Wq(hca_net* n, int l) { return n->wq + n->L.wq_off[l]; }
const bf16* Wt(hca_net* n, int l) { return n->wt + n->L.wq_off[l]; }
const float* Bias(hca_net* n, int l) { return n->params + n->L.b_off[l]; }

// Forward pass from n->x; with keep_d0 the last activation is stored (training).
void forward(hca_net* n, cudaStream_t s, bool keep_d0) {
  const int* D = n->Ld;
  const int* H = n->Lh;
  const int* W = n->Lw;
  if (n->use_tc)
    conv_tc<16, 16, 4, false, EPI_FWD>(s, n->tc_status, n->x, Wq(n, 0), Bias(n, 0), nullptr, n->e0, nullptr, nullptr,
                                       nullptr, D[0], H[0], W[0]);
  else
    conv<16, 16, 4, false, EPI_FWD>(s, n->x, Wq(n, 0), Bias(n, 0), nullptr, n->e0, nullptr, nullptr, nullptr, D[0],
                                    H[0], W[0]);
  pool<16>(n, s, n->e0, n->p0, 0);
  conv<16, 32, 4, false, EPI_FWD>(s, n->p0, Wq(n, 1), Bias(n, 1), nullptr, n->e1, nullptr, nullptr, nullptr, D[1], H[1], W[1]);
  pool<32>(n, s, n->e1, n->p1, 1);
  conv<32, 64, 2, false, EPI_FWD>(s, n->p1, Wq(n, 2), Bias(n, 2), nullptr, n->e2, nullptr, nullptr, nullptr, D[2], H[2], W[2]);
  pool<64>(n, s, n->e2, n->p2, 2);
  conv<64, 64, 2, false, EPI_FWD>(s, n->p2, Wq(n, 3), Bias(n, 3), nullptr, n->e3, nullptr, nullptr, nullptr, D[3], H[3], W[3]);
  conv<64, 64, 2, true, EPI_FWD>(s, n->e3, Wq(n, 4), Bias(n, 4), n->e2, n->d2, nullptr, nullptr, nullptr, D[2], H[2], W[2]);
  conv<64, 32, 4, true, EPI_FWD>(s, n->d2, Wq(n, 5), Bias(n, 5), n->e1, n->d1, nullptr, nullptr, nullptr, D[1], H[1], W[1]);
  if (n->use_tc)
    conv_tc<32, 16, 4, true, EPI_HEAD>(s, n->tc_status, n->d1, Wq(n, 6), Bias(n, 6), n->e0, keep_d0 ? n->d0 : nullptr,
                                       n->out, n->params + n->L.hw_off, n->params + n->L.hb_off, D[0], H[0], W[0]);
  else
    conv<32, 16, 4, true, EPI_HEAD>(s, n->d1, Wq(n, 6), Bias(n, 6), n->e0, keep_d0 ? n->d0 : nullptr, n->out,
                                    n->params + n->L.hw_off, n->params + n->L.hb_off, D[0], H[0], W[0]);
}

// Backward pass after forward(keep_d0 = true): the MSE loss against target,
// or (gbuf != null) the output gradient in gbuf; fills n->grads (and n->loss
// for the MSE loss).
void backward(hca_net* n, cudaStream_t s, const float* target, const float* gbuf) {
  const int* D = n->Ld;
  const int* H = n->Lh;
  const int* W = n->Lw;
  const ParamLayout& L = n->L;
  {
    const int nb = std::min(ew_blocks(n->Ln[0], n->sm_count), n->bpart_blocks);
    k_head_bwd<<<nb, kEwThreads, 0, s>>>(n->d0, n->out, target, gbuf, n->params + L.hw_off, n->Ln[0], n->g0,
                                         n->bpart);
    k_scatter_parts<<<1, 64, 0, s>>>(n->bpart, nb, kHeadParts, n->grads, n->head_index, gbuf ? nullptr : n->loss,
                                     1.0f / (float)n->Ln[0]);
  }
  // dec0: input up(d1), output gradient g0
  wgrad<32, 16, true>(n, s, n->d1, n->g0, D[0], H[0], W[0], n->grads + L.w_off[6]);
  conv<16, 32, 4, false, EPI_DOWN>(s, n->g0, Wt(n, 6), nullptr, nullptr, nullptr, n->graw, nullptr, nullptr, D[0], H[0], W[0]);
  combine<32, 0>(n, s, n->graw, n->d1, nullptr, n->g1, 1, 5);
  // dec1: input up(d2)
  wgrad<64, 32, true>(n, s, n->d2, n->g1, D[1], H[1], W[1], n->grads + L.w_off[5]);
  conv<32, 64, 2, false, EPI_DOWN>(s, n->g1, Wt(n, 5), nullptr, nullptr, nullptr, n->graw, nullptr, nullptr, D[1], H[1], W[1]);
  combine<64, 0>(n, s, n->graw, n->d2, nullptr, n->g2, 2, 4);
  // dec2: input up(e3)
  wgrad<64, 64, true>(n, s, n->e3, n->g2, D[2], H[2], W[2], n->grads + L.w_off[4]);
  conv<64, 64, 2, false, EPI_DOWN>(s, n->g2, Wt(n, 4), nullptr, nullptr, nullptr, n->graw, nullptr, nullptr, D[2], H[2], W[2]);
  combine<64, 0>(n, s, n->graw, n->e3, nullptr, n->g3, 3, 3);
  // enc3: input p2
  wgrad<64, 64, false>(n, s, n->p2, n->g3, D[3], H[3], W[3], n->grads + L.w_off[3]);
  conv<64, 64, 2, false, EPI_RAW>(s, n->g3, Wt(n, 3), nullptr, nullptr, nullptr, n->graw, nullptr, nullptr, D[3], H[3], W[3]);
  combine<64, 1>(n, s, n->graw, n->e2, n->g2, n->ge2, 2, 2);
  // enc2: input p1
  wgrad<32, 64, false>(n, s, n->p1, n->ge2, D[2], H[2], W[2], n->grads + L.w_off[2]);
  conv<64, 32, 4, false, EPI_RAW>(s, n->ge2, Wt(n, 2), nullptr, nullptr, nullptr, n->graw, nullptr, nullptr, D[2], H[2], W[2]);
  combine<32, 1>(n, s, n->graw, n->e1, n->g1, n->ge1, 1, 1);
  // enc1: input p0
  wgrad<16, 32, false>(n, s, n->p0, n->ge1, D[1], H[1], W[1], n->grads + L.w_off[1]);
  conv<32, 16, 4, false, EPI_RAW>(s, n->ge1, Wt(n, 1), nullptr, nullptr, nullptr, n->graw, nullptr, nullptr, D[1], H[1], W[1]);
  combine<16, 1>(n, s, n->graw, n->e0, n->g0, n->ge0, 0, 0);
  // enc0: input x
  wgrad<16, 16, false>(n, s, n->x, n->ge0, D[0], H[0], W[0], n->grads + L.w_off[0]);
}

void quantize(hca_net* n, cudaStream_t s) {
  QuantTable T;
  for (int l = 0; l < 7; ++l) {
    T.w_off[l] = n->L.w_off[l];
    T.q_off[l] = n->L.wq_off[l];
    T.ci[l] = kCI[l];
    T.co[l] = kCO[l];
  }
  k_quantize<<<ew_blocks(n->L.wq_total, n->sm_count), kEwThreads, 0, s>>>(n->params, T, n->wq, n->wt, n->L.wq_total);
}

template <typename T>
void features(hca_net* n, cudaStream_t s, const FeatureArgs& f, const T* K) {
  k_features<T><<<ew_blocks(n->Ln[0], n->sm_count), kEwThreads, 0, s>>>(f, K, n->x);
}

int adam_update(hca_net* n, double lr, double beta1, double beta2, double eps) {
  n->adam_t += 1;
  const double c1 = 1.0 - std::pow(beta1, (double)n->adam_t), c2 = 1.0 - std::pow(beta2, (double)n->adam_t);
  k_adam<<<ew_blocks(n->L.total, n->sm_count), kEwThreads, 0, n->stream>>>(
      n->params, n->grads, n->m, n->v, n->L.total, (float)lr, (float)beta1, (float)beta2, (float)eps, (float)c1,
      (float)c2);
  quantize(n, n->stream);
  NET_CUDA(cudaGetLastError());
  return HCA_OK;
}

int check_dims(int D, int H, int W) {
  if (D < 8 || H < 8 || W < 8 || D % 8 || H % 8 || W % 8) return HCA_ERR_ARG;
  if ((long long)D * H * W > (1LL << 31) / 16) return HCA_ERR_ARG;
  return HCA_OK;
}

int create_impl(int D, int H, int W, int trainable, void* stream, hca_net** out) {
  int rc = check_dims(D, H, W);
  if (rc) return rc;
  hca_net* n = new (std::nothrow) hca_net();
  if (!n) return HCA_ERR_OOM;
  *out = n;
  n->D = D;
  n->H = H;
  n->W = W;
  n->trainable = trainable != 0;
  n->stream = static_cast<cudaStream_t>(stream);
  NET_CUDA(cudaGetDevice(&n->device));
  NET_CUDA(cudaDeviceGetAttribute(&n->sm_count, cudaDevAttrMultiProcessorCount, n->device));
  if ((rc = set_attributes())) return rc;
  n->L = param_layout();
  for (int l = 0; l < 4; ++l) {
    n->Ld[l] = D >> l;
    n->Lh[l] = H >> l;
    n->Lw[l] = W >> l;
    n->Ln[l] = (long long)n->Ld[l] * n->Lh[l] * n->Lw[l];
  }
  const long long* Ln = n->Ln;
  const size_t b2 = sizeof(bf16);
  NET_ALLOC(n->params, n->L.total * sizeof(float));
  NET_ALLOC(n->wq, n->L.wq_total * b2);
  NET_ALLOC(n->wt, n->L.wq_total * b2);
  NET_ALLOC(n->tc_status, sizeof(int));
  NET_CUDA(cudaMemset(n->tc_status, 0, sizeof(int)));
  {
    // tcgen05 forward for the full-resolution layers with HCA_NET_TC=1
    // (compute capability 10.x; tiles of 8 x 16 sites).  Off by default: with
    // 16 output channels every MMA is M128 N16 K16 and the 27 taps' small
    // instructions, with the upsampled layer's output-resolution halo, cost
    // more than the mma.sync kernel (256^3 forward 4.99 against 3.81 ms)
    int major = 0;
    NET_CUDA(cudaDeviceGetAttribute(&major, cudaDevAttrComputeCapabilityMajor, n->device));
    const char* e = std::getenv("HCA_NET_TC");
    n->use_tc = major == 10 && W % kTcX == 0 && H % kTcY == 0 && (e && e[0] == '1') &&
                conv_tc_attr<16, 16, 4, false, EPI_FWD>() && conv_tc_attr<32, 16, 4, true, EPI_HEAD>();
  }
  NET_ALLOC(n->x, Ln[0] * 16 * b2);
  NET_ALLOC(n->e0, Ln[0] * 16 * b2);
  NET_ALLOC(n->p0, Ln[1] * 16 * b2);
  NET_ALLOC(n->e1, Ln[1] * 32 * b2);
  NET_ALLOC(n->p1, Ln[2] * 32 * b2);
  NET_ALLOC(n->e2, Ln[2] * 64 * b2);
  NET_ALLOC(n->p2, Ln[3] * 64 * b2);
  NET_ALLOC(n->e3, Ln[3] * 64 * b2);
  NET_ALLOC(n->d2, Ln[2] * 64 * b2);
  NET_ALLOC(n->d1, Ln[1] * 32 * b2);
  NET_ALLOC(n->out, Ln[0] * sizeof(float));
  NET_CUDA(cudaMemsetAsync(n->params, 0, n->L.total * sizeof(float), n->stream));
  if (n->trainable) {
    NET_ALLOC(n->d0, Ln[0] * 16 * b2);
    NET_ALLOC(n->tgt, Ln[0] * sizeof(float));
    NET_ALLOC(n->ru, Ln[0] * sizeof(float));
    NET_ALLOC(n->rg, Ln[0] * sizeof(float));
    NET_ALLOC(n->grads, n->L.total * sizeof(float));
    NET_ALLOC(n->m, n->L.total * sizeof(float));
    NET_ALLOC(n->v, n->L.total * sizeof(float));
    NET_ALLOC(n->g0, Ln[0] * 16 * b2);
    NET_ALLOC(n->g1, Ln[1] * 32 * b2);
    NET_ALLOC(n->g2, Ln[2] * 64 * b2);
    NET_ALLOC(n->g3, Ln[3] * 64 * b2);
    NET_ALLOC(n->ge0, Ln[0] * 16 * b2);
    NET_ALLOC(n->ge1, Ln[1] * 32 * b2);
    NET_ALLOC(n->ge2, Ln[2] * 64 * b2);
    NET_ALLOC(n->graw, std::max({Ln[1] * 32, Ln[2] * 64, Ln[3] * 64}) * sizeof(float));
    n->wpart_n = (long long)2 * n->sm_count * 27 * 16 * 16 + 27LL * 64 * 64 * 32;
    NET_ALLOC(n->wpart, n->wpart_n * sizeof(float));
    n->bpart_blocks = n->sm_count * 8;
    NET_ALLOC(n->bpart, (size_t)n->bpart_blocks * 64 * sizeof(float));   // >= 2 * bpart_blocks for the loss
    NET_ALLOC(n->loss, sizeof(float));
    NET_ALLOC(n->head_index, kHeadParts * sizeof(long long));
    NET_ALLOC(n->bias_index, 7 * 64 * sizeof(long long));
    std::vector<long long> hi(kHeadParts, -1), bi(7 * 64, -1);
    for (int c = 0; c < 16; ++c) {
      hi[c] = n->L.hw_off + c;
      hi[17 + c] = n->L.b_off[6] + c;
    }
    hi[16] = n->L.hb_off;
    for (int l = 0; l < 7; ++l)
      for (int c = 0; c < kCO[l]; ++c) bi[64 * l + c] = n->L.b_off[l] + c;
    NET_CUDA(cudaMemcpyAsync(n->head_index, hi.data(), hi.size() * sizeof(long long), cudaMemcpyHostToDevice, n->stream));
    NET_CUDA(cudaMemcpyAsync(n->bias_index, bi.data(), bi.size() * sizeof(long long), cudaMemcpyHostToDevice, n->stream));
    NET_CUDA(cudaMemsetAsync(n->m, 0, n->L.total * sizeof(float), n->stream));
    NET_CUDA(cudaMemsetAsync(n->v, 0, n->L.total * sizeof(float), n->stream));
    NET_CUDA(cudaMemsetAsync(n->grads, 0, n->L.total * sizeof(float), n->stream));
  }
  quantize(n, n->stream);
  NET_CUDA(cudaGetLastError());
  NET_CUDA(cudaStreamSynchronize(n->stream));
  return HCA_OK;
}

FeatureArgs dense_args(const hca_net* n, const hca_config* cfg, const uint8_t* state, const float* perf) {
  FeatureArgs f;
  f.state = state;
  f.perf = perf;
  f.nx = n->W;
  f.ny = n->H;
  f.nz = n->D;
  f.pitch = n->W;
  f.base = 0;
  f.D_K = cfg->D_K;
  f.dx = cfg->dx;
  f.phi_K = cfg->phi_K;
  f.K1 = cfg->K1;
  f.r_K = cfg->r_K;
  f.K0 = cfg->K0;
  return f;
}

}  // namespace

namespace hcanet {

bool ws_fits(const hca_net* n, int nx, int ny, int nz) { return n && n->W == nx && n->H == ny && n->D == nz; }

int ws_o2(hca_net* n, const FeatureArgs& f, bool fp64, bool always, void* K, float* K_lo, void* lag, double* cand,
          double* part, WsResult* res, cudaStream_t s) {
  if (!ws_fits(n, f.nx, f.ny, f.nz)) return HCA_ERR_ARG;
  const int nb = ew_blocks(n->Ln[0], n->sm_count);
  const int nbn = std::min(nb, kWsNormBlocks);
  if (fp64) {
    const double* Kd = static_cast<const double*>(K);
    features<double>(n, s, f, Kd);
    forward(n, s, false);
    k_ws_candidate<double><<<nb, kEwThreads, 0, s>>>(f, Kd, nullptr, n->out, cand, static_cast<double*>(lag));
    k_ws_norms<double><<<nbn, kEwThreads, 0, s>>>(f, Kd, nullptr, cand, part);
    k_ws_decide<<<1, 32, 0, s>>>(part, nbn, always ? 1 : 0, res);
    k_ws_apply<double><<<nb, kEwThreads, 0, s>>>(f, res, cand, static_cast<double*>(K), nullptr);
  } else {
    const float* Kf = static_cast<const float*>(K);
    features<float>(n, s, f, Kf);
    forward(n, s, false);
    k_ws_candidate<float><<<nb, kEwThreads, 0, s>>>(f, Kf, K_lo, n->out, cand, static_cast<float*>(lag));
    k_ws_norms<float><<<nbn, kEwThreads, 0, s>>>(f, Kf, K_lo, cand, part);
    k_ws_decide<<<1, 32, 0, s>>>(part, nbn, always ? 1 : 0, res);
    k_ws_apply<float><<<nb, kEwThreads, 0, s>>>(f, res, cand, static_cast<float*>(K), K_lo);
  }
  NET_CUDA(cudaGetLastError());
  return HCA_OK;
}

}  // namespace hcanet

// ================================================================ C ABI
extern "C" {

int hca_net_param_count(int64_t* n_out) {
  if (!n_out) return HCA_ERR_ARG;
  *n_out = param_layout().total;
  return HCA_OK;
}

int hca_net_create(int32_t D, int32_t H, int32_t W, int32_t trainable, void* stream, hca_net** out) {
  if (!out) return HCA_ERR_ARG;
  *out = nullptr;
  hca_net* n = nullptr;
  const int rc = create_impl(D, H, W, trainable, stream, &n);
  if (rc) {
    if (n) hca_net_destroy(n);
    return rc;
  }
  *out = n;
  return HCA_OK;
}

int hca_net_set_params(hca_net* n, const float* params, int32_t on_device) {
  if (!n || !params) return HCA_ERR_ARG;
  NET_CUDA(cudaMemcpyAsync(n->params, params, n->L.total * sizeof(float),
                           on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, n->stream));
  if (n->trainable) {
    NET_CUDA(cudaMemsetAsync(n->m, 0, n->L.total * sizeof(float), n->stream));
    NET_CUDA(cudaMemsetAsync(n->v, 0, n->L.total * sizeof(float), n->stream));
    n->adam_t = 0;
  }
  quantize(n, n->stream);
  NET_CUDA(cudaGetLastError());
  NET_CUDA(cudaStreamSynchronize(n->stream));
  return HCA_OK;
}

int hca_net_get_params(hca_net* n, float* params, int32_t on_device) {
  if (!n || !params) return HCA_ERR_ARG;
  NET_CUDA(cudaMemcpyAsync(params, n->params, n->L.total * sizeof(float),
                           on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, n->stream));
  NET_CUDA(cudaStreamSynchronize(n->stream));
  return HCA_OK;
}

int hca_net_forward(hca_net* n, const hca_config* cfg, const uint8_t* state, const float* perf, const float* K_prev,
                    float* out, void* x_out) {
  if (!n || !cfg || !state || !perf || !K_prev || !out) return HCA_ERR_ARG;
  const FeatureArgs f = dense_args(n, cfg, state, perf);
  features<float>(n, n->stream, f, K_prev);
  if (x_out)
    NET_CUDA(cudaMemcpyAsync(x_out, n->x, n->Ln[0] * 16 * sizeof(bf16), cudaMemcpyDeviceToDevice, n->stream));
  forward(n, n->stream, false);
  NET_CUDA(cudaMemcpyAsync(out, n->out, n->Ln[0] * sizeof(float), cudaMemcpyDeviceToDevice, n->stream));
  NET_CUDA(cudaGetLastError());
  NET_CUDA(cudaStreamSynchronize(n->stream));
  return HCA_OK;
}

int hca_net_forward_x(hca_net* n, const void* x, float* out) {
  if (!n || !x || !out) return HCA_ERR_ARG;
  NET_CUDA(cudaMemcpyAsync(n->x, x, n->Ln[0] * 16 * sizeof(bf16), cudaMemcpyDeviceToDevice, n->stream));
  forward(n, n->stream, n->trainable);
  NET_CUDA(cudaMemcpyAsync(out, n->out, n->Ln[0] * sizeof(float), cudaMemcpyDeviceToDevice, n->stream));
  NET_CUDA(cudaGetLastError());
  NET_CUDA(cudaStreamSynchronize(n->stream));
  return HCA_OK;
}

int hca_net_read_activation(hca_net* n, int32_t which, void* dst) {
  if (!n || !dst || which < 0 || which > 10) return HCA_ERR_ARG;
  bf16* src[11] = {n->x, n->e0, n->p0, n->e1, n->p1, n->e2, n->p2, n->e3, n->d2, n->d1, n->d0};
  const int lvl[11] = {0, 0, 1, 1, 2, 2, 3, 3, 2, 1, 0};
  const int ch[11] = {16, 16, 16, 32, 32, 64, 64, 64, 64, 32, 16};
  if (!src[which]) return HCA_ERR_ARG;
  NET_CUDA(cudaMemcpyAsync(dst, src[which], n->Ln[lvl[which]] * ch[which] * sizeof(bf16), cudaMemcpyDeviceToDevice,
                           n->stream));
  NET_CUDA(cudaStreamSynchronize(n->stream));
  return HCA_OK;
}

int hca_net_read_gradient(hca_net* n, int32_t which, void* dst) {
  if (!n || !dst || which < 0 || which > 6 || !n->trainable) return HCA_ERR_ARG;
  // convolution order enc0, enc1, enc2, enc3, dec2, dec1, dec0
  bf16* src[7] = {n->ge0, n->ge1, n->ge2, n->g3, n->g2, n->g1, n->g0};
  const int lvl[7] = {0, 1, 2, 3, 2, 1, 0};
  const int ch[7] = {16, 32, 64, 64, 64, 32, 16};
  NET_CUDA(cudaMemcpyAsync(dst, src[which], n->Ln[lvl[which]] * ch[which] * sizeof(bf16), cudaMemcpyDeviceToDevice,
                           n->stream));
  NET_CUDA(cudaStreamSynchronize(n->stream));
  return HCA_OK;
}

int hca_net_gradients_x(hca_net* n, const void* x, const float* target, float* grads, float* loss) {
  if (!n || !x || !target || !n->trainable) return HCA_ERR_ARG;
  NET_CUDA(cudaMemcpyAsync(n->x, x, n->Ln[0] * 16 * sizeof(bf16), cudaMemcpyDeviceToDevice, n->stream));
  forward(n, n->stream, true);
  backward(n, n->stream, target, nullptr);
  if (grads)
    NET_CUDA(cudaMemcpyAsync(grads, n->grads, n->L.total * sizeof(float), cudaMemcpyDeviceToDevice, n->stream));
  if (loss) NET_CUDA(cudaMemcpyAsync(loss, n->loss, sizeof(float), cudaMemcpyDeviceToDevice, n->stream));
  NET_CUDA(cudaGetLastError());
  NET_CUDA(cudaStreamSynchronize(n->stream));
  return HCA_OK;
}

int hca_net_gradients(hca_net* n, const hca_config* cfg, const uint8_t* state, const float* perf,
                      const float* K_prev, const float* K_new, double w_mse, double w_res, float* grads,
                      float* loss) {
  if (!n || !cfg || !state || !perf || !K_prev || !K_new || !n->trainable) return HCA_ERR_ARG;
  if (!(w_mse >= 0) || !(w_res >= 0) || !(w_mse + w_res > 0)) return HCA_ERR_ARG;
  const FeatureArgs f = dense_args(n, cfg, state, perf);
  cudaStream_t s = n->stream;
  const int nb = ew_blocks(n->Ln[0], n->sm_count);
  const int nr = std::min(nb, n->bpart_blocks);
  features<float>(n, s, f, K_prev);
  k_target<<<nb, kEwThreads, 0, s>>>(K_prev, K_new, n->Ln[0], (float)(kNetScale / cfg->K0), n->tgt);
  forward(n, s, true);
  k_res_u<<<nr, kEwThreads, 0, s>>>(f, K_prev, n->out, n->tgt, n->ru, n->bpart);
  k_loss_grad<<<nr, kEwThreads, 0, s>>>(f, K_prev, n->out, n->tgt, n->ru, (float)w_mse, (float)w_res, n->rg,
                                        n->bpart + n->bpart_blocks);
  k_sum_loss<<<1, 32, 0, s>>>(n->bpart, nr, (float)w_res / (float)n->Ln[0], n->bpart + n->bpart_blocks,
                              (float)w_mse / (float)n->Ln[0], n->loss);
  backward(n, s, n->tgt, n->rg);
  if (grads) NET_CUDA(cudaMemcpyAsync(grads, n->grads, n->L.total * sizeof(float), cudaMemcpyDeviceToDevice, s));
  if (loss) NET_CUDA(cudaMemcpyAsync(loss, n->loss, sizeof(float), cudaMemcpyDeviceToDevice, s));
  NET_CUDA(cudaGetLastError());
  return HCA_OK;
}

int hca_net_train_step(hca_net* n, const hca_config* cfg, const uint8_t* state, const float* perf,
                       const float* K_prev, const float* K_new, double w_mse, double w_res, double lr,
                       float* loss) {
  if (!(lr > 0)) return HCA_ERR_ARG;
  const int rc = hca_net_gradients(n, cfg, state, perf, K_prev, K_new, w_mse, w_res, nullptr, loss);
  if (rc) return rc;
  return adam_update(n, lr, 0.9, 0.999, 1e-8);
}

// The training sample of step t: floor(u * n) for the 24-bit uniform of the
// Philox4x32-10 output word 0 at counter (t, 0, 0, 5), key (seed lo, seed hi).
static int train_sample(uint64_t seed, int t, int n) {
  uint32_t c[4] = {(uint32_t)t, 0u, 0u, 5u};
  uint32_t k0 = (uint32_t)seed, k1 = (uint32_t)(seed >> 32);
  for (int r = 0; r < 10; ++r) {
    const unsigned long long p0 = 0xD2511F53ull * (unsigned long long)c[0];
    const unsigned long long p1 = 0xCD9E8D57ull * (unsigned long long)c[2];
    const uint32_t n0 = (uint32_t)(p1 >> 32) ^ c[1] ^ k0, n2 = (uint32_t)(p0 >> 32) ^ c[3] ^ k1;
    c[1] = (uint32_t)p1;
    c[3] = (uint32_t)p0;
    c[0] = n0;
    c[2] = n2;
    k0 += 0x9E3779B9u;
    k1 += 0xBB67AE85u;
  }
  const double u = (double)(c[0] >> 8) * 5.9604644775390625e-08;
  return std::min(n - 1, (int)(u * n));
}

int hca_train_warmstart(hca_net* n, const hca_config* cfg, const hca_train_cfg* tc) {
  if (!n || !cfg || !tc || tc->struct_size != sizeof(hca_train_cfg) || !n->trainable) return HCA_ERR_ARG;
  if (tc->n_samples < 1 || tc->iters < 0 || !tc->state || !tc->perf || !tc->K_prev || !tc->K_new) return HCA_ERR_ARG;
  if (!(tc->lr > 0) || !(tc->lr_final > 0)) return HCA_ERR_ARG;
  for (int i = 0; i < tc->n_samples; ++i)
    if (!tc->state[i] || !tc->perf[i] || !tc->K_prev[i] || !tc->K_new[i]) return HCA_ERR_ARG;
  for (int t = 0; t < tc->iters; ++t) {
    const int i = train_sample(tc->seed, t, tc->n_samples);
    const double a = tc->iters > 1 ? tc->lr * std::pow(tc->lr_final / tc->lr, (double)t / (tc->iters - 1)) : tc->lr;
    const int rc = hca_net_train_step(n, cfg, tc->state[i], tc->perf[i], tc->K_prev[i], tc->K_new[i], tc->w_mse,
                                      tc->w_res, a, tc->losses ? tc->losses + t : nullptr);
    if (rc) return rc;
  }
  return HCA_OK;
}

int hca_net_adam(hca_net* n, double lr, double beta1, double beta2, double eps) {
  if (!n || !n->trainable || !(lr > 0) || !(beta1 >= 0 && beta1 < 1) || !(beta2 >= 0 && beta2 < 1) || !(eps >= 0))
    return HCA_ERR_ARG;
  const int rc = adam_update(n, lr, beta1, beta2, eps);
  if (rc) return rc;
  NET_CUDA(cudaStreamSynchronize(n->stream));
  return HCA_OK;
}

int hca_net_sync(hca_net* n) {
  if (!n) return HCA_ERR_ARG;
  NET_CUDA(cudaStreamSynchronize(n->stream));
  return HCA_OK;
}

int hca_net_destroy(hca_net* n) {
  if (!n) return HCA_OK;
  if (n->stream) cudaStreamSynchronize(n->stream);
  for (void* p : n->allocs) cudaFree(p);
  delete n;
  return HCA_OK;
}

}  // extern "C"
