// Interface between the solver engine and the warm-start network (net.cu).
#pragma once

#include <cuda_runtime.h>

#include <cstdint>

struct hca_net;

namespace hcanet {

// Scale of the network's residual input channel and of its output: the
// guess is K_prev + (K0 / kNetScale) f(x).
constexpr double kNetScale = 64.0;

// Fields of one oxygen solve: site (x, y, z) is element base + x + pitch*(y + ny*z).
struct FeatureArgs {
  const uint8_t* state;
  const void* perf;      // same element type as the oxygen field
  int nx, ny, nz;
  long long pitch;
  long long base;
  double D_K, dx, phi_K, K1, r_K, K0;
};

// Relative residuals ||b - A u|| / ||b|| of the two candidate initial guesses
// (A lagged at K_prev) and which one the solve starts from.
struct WsResult {
  double r0_prev;
  double r0_learned;
  int used;
  int pad;
};

constexpr int kWsNormBlocks = 1024;

// Replace the oxygen field K (FP64, or FP32 with optional low word K_lo) by
// the network's guess when that guess has the smaller residual (always: in
// any case); lag receives
// K_prev in the field's type.  cand: FP64 scratch of the field's padded size;
// part: 3 * kWsNormBlocks doubles.  Asynchronous on s; capturable.
int ws_o2(hca_net* n, const FeatureArgs& f, bool fp64, bool always, void* K, float* K_lo, void* lag, double* cand,
          double* part, WsResult* res, cudaStream_t s);

// Whether a network was made for this lattice (nz, ny, nx) = (D, H, W).
bool ws_fits(const hca_net* n, int nx, int ny, int nz);

}  // namespace hcanet
