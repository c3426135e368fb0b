// hca_o2_residual_noalloc: the oxygen solve's true-residual check on
// caller-owned device arrays, without any device allocation.
//
// Who needs this: code that may not call cudaMalloc on the path where it
// checks a field -- for example a caller running inside another framework's
// memory pool that must not be bypassed, a real-time loop where an
// allocation's latency or its implicit device synchronisation is not
// allowed, or an embedding that only hands the library raw pointers.  Such a
// caller cannot create a handle (which owns its device buffers) just to ask
// "how well does this K solve the oxygen system linearised about K_prev?".
//
// This entry point answers that with the same arithmetic as the handle's
// true-residual kernel: per site r = b - A(K_prev) K with the 7-point
// Neumann operator, summed per 32-row chunk and then over chunks in a fixed
// order.  The per-chunk partial sums, the finishing ticket and the result
// live in the file-scope device array `g_noalloc` below instead of memory
// the caller or the library would allocate.  Its size is fixed at compile
// time (kNoAllocMaxChunks chunks: ny * nz <= 65536 rows, e.g. 256 x 256 in
// y, z with any nx), it occupies about 33 KB on every GPU that loads the library
// until the process exits, and every call shares it.  Calls that overlap on
// the GPU (two streams, or two host threads) race on it and must be
// serialised by the caller.
//
// The array's device address is looked up on every call, with the caller's
// device current (cudaGetSymbolAddress is a host-side lookup and allocates
// nothing).  A cached address could outlive the context it belongs to: after
// a device reset the module is loaded again and the array may move.
#include <cuda_runtime.h>

#include "hca_internal.cuh"

namespace {

constexpr int kNoAllocMaxChunks = 2048;
constexpr int kNoAllocRows = 32;       // rows per chunk
constexpr int kNoAllocThreads = 256;   // fixed: the reduction order depends on it

struct NoAllocScratch {
  double partial[kNoAllocMaxChunks][2];  // per chunk: |r|^2, |b|^2
  double result[2];                      // |r| / |b|, |b|^2
  unsigned int ticket;
  unsigned int pad[3];
};

static __device__ __align__(256) NoAllocScratch g_noalloc;

__global__ void __launch_bounds__(kNoAllocThreads) k_o2_residual_noalloc(
    NoAllocScratch* __restrict__ sc, int nx, int ny, int nz, double c, double phi_K, double K1, double K0,
    double r_K, const uint8_t* __restrict__ state, const double* __restrict__ K_prev,
    const double* __restrict__ K) {
  const int rows = ny * nz;
  const int row0 = blockIdx.x * kNoAllocRows;
  const int nrow = min(kNoAllocRows, rows - row0);
  const long long nsite = (long long)nrow * nx;
  const long long plane = (long long)nx * ny;
  double rr = 0.0, bb = 0.0;
  for (long long t = threadIdx.x; t < nsite; t += kNoAllocThreads) {
    const int j = row0 + (int)(t / nx);
    const int x = (int)(t % nx);
    const int y = j % ny, z = j / ny;
    const long long i = (long long)j * nx + x;
    const uint8_t s = state[i];
    double a = 0.0;
    if (s == HCA_PROLIF || s == HCA_QUIESC || s == HCA_STROMA) a = phi_K / (K1 + K_prev[i]);
    if (s == HCA_VESSEL) a += r_K;
    int n = 0;
    double nb = 0.0;
    if (x > 0) { nb += K[i - 1]; ++n; }
    if (x < nx - 1) { nb += K[i + 1]; ++n; }
    if (y > 0) { nb += K[i - nx]; ++n; }
    if (y < ny - 1) { nb += K[i + nx]; ++n; }
    if (z > 0) { nb += K[i - plane]; ++n; }
    if (z < nz - 1) { nb += K[i + plane]; ++n; }
    const double b = s == HCA_VESSEL ? r_K * K0 : 0.0;
    const double r = b - ((c * n + a) * K[i] - c * nb);
    rr += r * r;
    bb += b * b;
  }
  // fixed-order block reduction: warp xor trees, then warp sums in order
  __shared__ double s_w[kNoAllocThreads / 32][2];
  for (int o = 16; o > 0; o >>= 1) {
    rr += __shfl_xor_sync(0xffffffffu, rr, o);
    bb += __shfl_xor_sync(0xffffffffu, bb, o);
  }
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (lane == 0) {
    s_w[warp][0] = rr;
    s_w[warp][1] = bb;
  }
  __syncthreads();
  __shared__ unsigned int s_ticket;
  if (threadIdx.x == 0) {
    double a0 = 0.0, a1 = 0.0;
    for (int w = 0; w < kNoAllocThreads / 32; ++w) {
      a0 += s_w[w][0];
      a1 += s_w[w][1];
    }
    sc->partial[blockIdx.x][0] = a0;
    sc->partial[blockIdx.x][1] = a1;
    __threadfence();
    s_ticket = atomicAdd(&sc->ticket, 1u);
  }
  __syncthreads();
  if (s_ticket != gridDim.x - 1) return;
  // last block: chunk partials in a fixed order (thread t takes t, t + 256, ...)
  __threadfence();
  double p0 = 0.0, p1 = 0.0;
  for (int k = threadIdx.x; k < (int)gridDim.x; k += kNoAllocThreads) {
    p0 += __ldcg(&sc->partial[k][0]);
    p1 += __ldcg(&sc->partial[k][1]);
  }
  for (int o = 16; o > 0; o >>= 1) {
    p0 += __shfl_xor_sync(0xffffffffu, p0, o);
    p1 += __shfl_xor_sync(0xffffffffu, p1, o);
  }
  __syncthreads();
  if (lane == 0) {
    s_w[warp][0] = p0;
    s_w[warp][1] = p1;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double a0 = 0.0, a1 = 0.0;
    for (int w = 0; w < kNoAllocThreads / 32; ++w) {
      a0 += s_w[w][0];
      a1 += s_w[w][1];
    }
    sc->result[0] = a1 > 0.0 ? sqrt(a0 / a1) : 0.0;
    sc->result[1] = a1;
    sc->ticket = 0u;
  }
}

}  // namespace

extern "C" int hca_o2_residual_noalloc(const hca_config* cfg, const uint8_t* state, const double* K_prev,
                                       const double* K, double* rel_out, void* stream) {
  if (!cfg || !state || !K_prev || !K || !rel_out) return HCA_ERR_ARG;
  if (cfg->struct_size != sizeof(hca_config)) return HCA_ERR_ARG;
  if (cfg->nx < 1 || cfg->ny < 1 || cfg->nz < 1 || !(cfg->dx > 0)) return HCA_ERR_ARG;
  // the same parameter checks as handle creation, for the fields read here
  if (!(cfg->D_K > 0) || !(cfg->phi_K >= 0) || !(cfg->K1 > 0) || !(cfg->r_K >= 0) || !(cfg->K0 >= 0))
    return HCA_ERR_ARG;
  // only the quasi-steady operator: with a time-dependent oxygen scheme the
  // handle's right-hand side also depends on the previous field
  if (cfg->o2_scheme != 0) return HCA_ERR_ARG;
  const long long rows = (long long)cfg->ny * cfg->nz;
  const long long chunks = (rows + kNoAllocRows - 1) / kNoAllocRows;
  if (chunks > kNoAllocMaxChunks) return HCA_ERR_ARG;   // beyond the fixed scratch size
  if ((long long)cfg->nx * rows > 2147483647LL) return HCA_ERR_ARG;
  // device address of the scratch array in the current device's context (the
  // host-side symbol is only a stand-in, not a device address)
  void* addr = nullptr;
  if (cudaGetSymbolAddress(&addr, g_noalloc) != cudaSuccess || !addr) {
    (void)cudaGetLastError();
    return HCA_ERR_CUDA;
  }
  NoAllocScratch* sc = (NoAllocScratch*)addr;
  cudaStream_t s = (cudaStream_t)stream;
  // the ticket must start at zero (a previous call that failed mid-way may
  // have left it otherwise); the partials are fully overwritten
  if (cudaMemsetAsync(&sc->ticket, 0, sizeof(unsigned int), s) != cudaSuccess) {
    (void)cudaGetLastError();
    return HCA_ERR_CUDA;
  }
  const double c = cfg->D_K / (cfg->dx * cfg->dx);
  k_o2_residual_noalloc<<<(unsigned)chunks, kNoAllocThreads, 0, s>>>(sc, cfg->nx, cfg->ny, cfg->nz, c, cfg->phi_K,
                                                                       cfg->K1, cfg->K0, cfg->r_K, state, K_prev, K);
  double res[2] = {0.0, 0.0};
  if (cudaGetLastError() != cudaSuccess ||
      cudaMemcpyAsync(res, sc->result, sizeof(res), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
      cudaStreamSynchronize(s) != cudaSuccess) {
    (void)cudaGetLastError();
    return HCA_ERR_CUDA;
  }
  if (!isfinite(res[0])) return HCA_ERR_NONFINITE;
  *rel_out = res[0];
  return HCA_OK;
}
