// Diagonal energy tables of the Rydberg Hamiltonian (arXiv 2510.09813, Eq. (3)).
//
// The diagonal E(b) = sum_{q<r} V_qr b_q b_r - sum_q delta_q b_q is never stored
// as a 2^N vector (the paper's emulator stores it, Sec. III.A). For a contiguous
// tile with its high bits fixed to tau it splits into
//   E(b) = E_hi(tau) + sum_{q<L} w_q(tau) b_q + Q[b mod 2^L],
// with Q a per-register table and (w, E_hi) one short row per tile. This kernel
// writes those rows once per time step in FP64 (delta changes per step, the
// Krylov iterations of the step reuse them).
#include "kernels.h"
#include "rsv_common.cuh"

namespace rsv {

__global__ void diag_table_kernel(const StepParams* __restrict__ sp, const double* __restrict__ vmat, int n, int L,
                                  int64_t num_tiles, double* __restrict__ out) {
  const int64_t tile = (int64_t)blockIdx.x * (blockDim.x / 32) + (threadIdx.x >> 5);
  const int lane = threadIdx.x & 31;
  if (tile >= num_tiles) return;
  double* row = out + tile * kDiagStride;
  if (lane < L) {
    double w = -sp->delta[lane];
    for (int r = L; r < n; ++r)
      if ((tile >> (r - L)) & 1) w += vmat[lane * kMaxAtoms + r];
    row[lane] = w;
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
  if (lane == 0) row[kDiagStride - 1] = e;
}

cudaError_t launch_diag_table(const StepParams* sp, const double* vmat, int n, int L, int64_t num_tiles, double* out,
                              cudaStream_t stream) {
  if (L > kDiagStride - 1 || n - L > 32) return cudaErrorInvalidValue;
  const int warps = 8;
  const int64_t blocks = (num_tiles + warps - 1) / warps;
  diag_table_kernel<<<(unsigned)blocks, warps * 32, 0, stream>>>(sp, vmat, n, L, num_tiles, out);
  return cudaGetLastError();
}

}  // namespace rsv
