// Laser phase by a gauge transform (arXiv 2510.09813, Eq. (3) with phi_i != 0).
//
// With the phases phi_q constant over a time step and U = exp(-i sum_q phi_q n_q),
// conjugating one atom's drive gives U sigma_x U^dagger = cos(phi) sigma_x -
// sin(phi) sigma_y, while the diagonal commutes with U, so H(phi) = U H(0) U^dagger
// and exp(-i tau H(phi)) = U exp(-i tau H(0)) U^dagger. The step then runs the
// streaming passes with real flip coefficients, between two diagonal phase
// passes: psi_b *= exp(+i theta(b)) before (U^dagger) and exp(-i theta(b)) after
// (U), with theta(b) = sum_q phi_q b_q.
//
// theta is split at bit L (about n/2): exp(i theta(b)) = lo[b mod 2^L] *
// hi[b >> L], two tables formed in FP64 (one sincos of an FP64 sum per entry) and rounded once
// to the working precision, so a phase pass multiplies each amplitude by the
// product of two rounded unit numbers.
#include <algorithm>

#include "kernels.h"
#include "rsv_common.cuh"

namespace rsv {

namespace {

template <typename Real>
struct Cplx2;
template <>
struct Cplx2<float> {
  using T = float2;
};
template <>
struct Cplx2<double> {
  using T = double2;
};

template <typename Real>
__global__ void phase_table_kernel(const StepParams* __restrict__ sp, int n, int L, typename Cplx2<Real>::T* lo,
                                   typename Cplx2<Real>::T* hi) {
  const int64_t nlo = int64_t(1) << L, nhi = int64_t(1) << (n - L);
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < nlo + nhi; i += (int64_t)gridDim.x * blockDim.x) {
    const bool low = i < nlo;
    const int64_t bits = low ? i : i - nlo;
    const int q0 = low ? 0 : L, q1 = low ? L : n;
    double th = 0.0;
    for (int q = q0; q < q1; ++q)
      if ((bits >> (q - q0)) & 1) th += sp->phi[q];
    double s, c;
    sincos(th, &s, &c);
    typename Cplx2<Real>::T v;
    v.x = (Real)c;
    v.y = (Real)s;
    if (low) lo[bits] = v;
    else hi[bits] = v;
  }
}

// psi_b *= lo[b mod 2^L] * hi[b >> L], conjugated when conj != 0. One complex
// amplitude per thread step; a warp's amplitudes share their hi entry.
template <typename Real>
__global__ void __launch_bounds__(kThreads) phase_apply_kernel(typename Cplx2<Real>::T* __restrict__ psi,
                                                               int64_t dim, int L,
                                                               const typename Cplx2<Real>::T* __restrict__ lo,
                                                               const typename Cplx2<Real>::T* __restrict__ hi,
                                                               int conj) {
  const int64_t lmask = (int64_t(1) << L) - 1;
  const Real sg = conj ? (Real)-1 : (Real)1;
  for (int64_t b = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; b < dim; b += (int64_t)gridDim.x * blockDim.x) {
    const typename Cplx2<Real>::T a = __ldg(lo + (b & lmask)), h = __ldg(hi + (b >> L));
    const Real pr = a.x * h.x - a.y * h.y;
    const Real pi = sg * (a.x * h.y + a.y * h.x);
    const typename Cplx2<Real>::T x = __ldcs(psi + b);
    typename Cplx2<Real>::T y;
    y.x = x.x * pr - x.y * pi;
    y.y = x.x * pi + x.y * pr;
    __stcs(psi + b, y);
  }
}

}  // namespace

size_t phase_table_bytes(int n, int L, bool c64) {
  const size_t entry = c64 ? sizeof(float2) : sizeof(double2);
  return entry * ((size_t(1) << L) + (size_t(1) << (n - L)));
}

cudaError_t launch_phase_table(const StepParams* sp, int n, int L, void* table, bool c64, cudaStream_t stream) {
  if (L < 0 || L > n || n > kMaxAtoms) return cudaErrorInvalidValue;
  const int64_t total = (int64_t(1) << L) + (int64_t(1) << (n - L));
  const int grid = (int)std::min<int64_t>((total + kThreads - 1) / kThreads, 4096);
  if (c64) {
    auto* lo = static_cast<float2*>(table);
    phase_table_kernel<float><<<grid, kThreads, 0, stream>>>(sp, n, L, lo, lo + (int64_t(1) << L));
  } else {
    auto* lo = static_cast<double2*>(table);
    phase_table_kernel<double><<<grid, kThreads, 0, stream>>>(sp, n, L, lo, lo + (int64_t(1) << L));
  }
  return cudaGetLastError();
}

cudaError_t launch_phase_apply(void* psi, int n, int L, const void* table, bool conj, bool c64, int grid,
                               cudaStream_t stream) {
  if (L < 0 || L > n || grid <= 0) return cudaErrorInvalidValue;
  const int64_t dim = int64_t(1) << n;
  if (c64) {
    const auto* lo = static_cast<const float2*>(table);
    phase_apply_kernel<float><<<grid, kThreads, 0, stream>>>(static_cast<float2*>(psi), dim, L, lo,
                                                             lo + (int64_t(1) << L), conj ? 1 : 0);
  } else {
    const auto* lo = static_cast<const double2*>(table);
    phase_apply_kernel<double><<<grid, kThreads, 0, stream>>>(static_cast<double2*>(psi), dim, L, lo,
                                                              lo + (int64_t(1) << L), conj ? 1 : 0);
  }
  return cudaGetLastError();
}

}  // namespace rsv
