// Inner products for expectation values of the Hamiltonian (arXiv 2510.09813,
// Eq. (3)): <psi|H|psi> = <psi, y> and <psi|H^2|psi> = |y|^2 with y = H psi.
// Products are exact (TwoProduct) and sums compensated for complex64; FP64 for
// complex128. One grid-stride pass over 16-byte vectors.
#include "kernels.h"
#include "rsv_common.cuh"

namespace rsv {

namespace {

template <typename Real>
__global__ void __launch_bounds__(kThreads) dot3_kernel(const void* xv, const void* yv, int64_t nvec,
                                                         double* partials) {
  using vec = typename CplxT<Real>::vec;
  using Acc = typename AccFor<Real>::type;
  constexpr int NV = 1 << CplxT<Real>::kLogVec;
  __shared__ double s_red[3 * (kThreads / 32)];
  const vec* x = reinterpret_cast<const vec*>(xv);
  const vec* y = reinterpret_cast<const vec*>(yv);
  Acc re, im, yy;
  for (int64_t i = (int64_t)blockIdx.x * kThreads + threadIdx.x; i < nvec; i += (int64_t)gridDim.x * kThreads) {
    Real a[2 * NV], b[2 * NV];
    *reinterpret_cast<vec*>(a) = x[i];
    *reinterpret_cast<vec*>(b) = y[i];
#pragma unroll
    for (int e = 0; e < NV; ++e) {
      const Real ar = a[2 * e], ai = a[2 * e + 1], br = b[2 * e], bi = b[2 * e + 1];
      // conj(a) b = (ar br + ai bi) + i (ar bi - ai br)
      re.dot(ar, br);
      re.dot(ai, bi);
      im.dot(ar, bi);
      im.dot(-ai, br);
      yy.dot(br, br);
      yy.dot(bi, bi);
    }
  }
  Acc acc[3] = {re, im, yy};
  block_reduce_write<3>(acc, s_red, partials + (int64_t)blockIdx.x * 3, 3);
}

}  // namespace

cudaError_t launch_dot3(const void* x, const void* y, int64_t dim, bool c64, double* partials, int grid,
                        cudaStream_t stream) {
  if (c64)
    dot3_kernel<float><<<grid, kThreads, 0, stream>>>(x, y, dim / 2, partials);
  else
    dot3_kernel<double><<<grid, kThreads, 0, stream>>>(x, y, dim, partials);
  return cudaGetLastError();
}

}  // namespace rsv
