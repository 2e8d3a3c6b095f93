// Diagonal energy tables of the Rydberg Hamiltonian (arXiv 2510.09813, Eq. (3)).
//
// The diagonal E(b) = sum_{q<r} V_qr b_q b_r - sum_q delta_q b_q is never stored
// as a 2^N vector (the paper's emulator stores it, Sec. III.A). For a contiguous
// tile with its high bits fixed to tau it splits into
//   E(b) = E_hi(tau) + sum_{q<L} w_q(tau) b_q + Q[b mod 2^L],
// with Q a per-register table and (w, E_hi) per tile. This kernel writes, once
// per time step (delta changes per step, the Krylov iterations of the step
// reuse them), each tile's two 64-entry half tables: the w sums over the low
// six tile bits, and E_hi plus the w sums over the rest. They are formed in
// FP64 and rounded once to the working precision, so a tile pass forms E(b)
// from three rounded terms.
#include "kernels.h"
#include "rsv_common.cuh"

namespace rsv {

template <typename Real>
__global__ void diag_table_kernel(const StepParams* __restrict__ sp, const double* __restrict__ vmat, int n, int L,
                                  int64_t num_tiles, Real* __restrict__ out) {
  const int64_t tile = (int64_t)blockIdx.x * (blockDim.x / 32) + (threadIdx.x >> 5);
  const int lane = threadIdx.x & 31;
  if (tile >= num_tiles) return;
  // w_q for the tile bits: lane q < L
  double w = 0.0;
  if (lane < L) {
    w = -sp->delta[lane];
    for (int r = L; r < n; ++r)
      if ((tile >> (r - L)) & 1) w += vmat[lane * kMaxAtoms + r];
  }
  // E_hi: lane l owns high bit q = L + l and sums its row of the pair energies
  double e = 0.0;
  const int q = L + lane;
  if (q < n && ((tile >> (q - L)) & 1)) {
    e = -sp->delta[q];
    for (int r = q + 1; r < n; ++r)
      if ((tile >> (r - L)) & 1) e += vmat[q * kMaxAtoms + r];
  }
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) e += __shfl_xor_sync(0xffffffffu, e, off);
  // half tables: lane l writes entries l and l + 32 of each half, in FP64
  // before the one rounding to the working precision
  Real* row = out + tile * kDiagStride;
#pragma unroll
  for (int h = 0; h < 2; ++h) {
    const int i = lane + 32 * h;
    double lo = 0.0, hi = e;
#pragma unroll
    for (int b = 0; b < 6; ++b) {
      const double wl = __shfl_sync(0xffffffffu, w, b);
      const double wh = __shfl_sync(0xffffffffu, w, 6 + b);
      if ((i >> b) & 1) {
        if (b < L) lo += wl;
        if (6 + b < L) hi += wh;
      }
    }
    row[i] = (Real)lo;
    row[kDiagHalf + i] = (Real)hi;
  }
}

cudaError_t launch_diag_table(const StepParams* sp, const double* vmat, int n, int L, int64_t num_tiles, void* out,
                              bool c64, cudaStream_t stream) {
  if (L > 12 || n - L > 32) return cudaErrorInvalidValue;
  const int warps = 8;
  const int64_t blocks = (num_tiles + warps - 1) / warps;
  if (c64)
    diag_table_kernel<float><<<(unsigned)blocks, warps * 32, 0, stream>>>(sp, vmat, n, L, num_tiles,
                                                                         static_cast<float*>(out));
  else
    diag_table_kernel<double><<<(unsigned)blocks, warps * 32, 0, stream>>>(sp, vmat, n, L, num_tiles,
                                                                          static_cast<double*>(out));
  return cudaGetLastError();
}

}  // namespace rsv
