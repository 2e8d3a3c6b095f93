// Kernels of the pulse gradient (arXiv 2510.09813, Sec. V: expectation values
// are differentiable with respect to the pulse tensors) and of the overlap
// with a target state (Sec. III results).
//
// The adjoint method runs backwards in time with conjugated vectors, so that
// every evolution is a forward Lanczos step: for mu = conj(lambda) and
// nu = conj(psi), lambda(s) = exp(-i H (s - tau)) lambda_{k+1} becomes
// mu(s) = exp(-i conj(H) (tau - s)) mu_{k+1}, and the same for nu. conj(H) is
// H with every phase negated. Along that evolution the step's derivative
// integrand <lambda(s)| G |psi(s)> is a bilinear sum over mu and conj(nu):
//     S0_q = sum_{b_q = 0} mu_b conj(nu_{b ^ 2^q}),
//     S1_q = sum_{b_q = 1} mu_b conj(nu_{b ^ 2^q}),
//     D_q  = sum_{b_q = 1} mu_b conj(nu_b),
// from which the host forms the Omega, delta and phi derivatives of atom q.
#include "kernels.h"
#include "rsv_common.cuh"

namespace rsv {

namespace {

// out_b = w(b) conj(in_b) with w(b) = sum_q w_bits[q] b_q (w_bits NULL: w = 1).
template <typename Real>
__global__ void __launch_bounds__(kThreads) conj_weight_kernel(const void* inv, void* outv, int64_t nvec, int n,
                                                               const double* w_bits) {
  using vec = typename CplxT<Real>::vec;
  constexpr int LV = CplxT<Real>::kLogVec, NV = 1 << LV;
  __shared__ double s_w[kMaxAtoms];
  if (threadIdx.x < kMaxAtoms) s_w[threadIdx.x] = (w_bits && (int)threadIdx.x < n) ? w_bits[threadIdx.x] : 0.0;
  __syncthreads();
  const vec* in = reinterpret_cast<const vec*>(inv);
  vec* out = reinterpret_cast<vec*>(outv);
  for (int64_t i = (int64_t)blockIdx.x * kThreads + threadIdx.x; i < nvec; i += (int64_t)gridDim.x * kThreads) {
    Real a[2 * NV];
    *reinterpret_cast<vec*>(a) = in[i];
#pragma unroll
    for (int e = 0; e < NV; ++e) {
      double w = 1.0;
      if (w_bits) {
        const int64_t b = (i << LV) | e;
        w = 0.0;
        for (int q = 0; q < n; ++q)
          if ((b >> q) & 1) w += s_w[q];
      }
      a[2 * e] = (Real)(w * (double)a[2 * e]);
      a[2 * e + 1] = (Real)(-w * (double)a[2 * e + 1]);
    }
    out[i] = *reinterpret_cast<vec*>(a);
  }
}

// Block (chunk c, bit q): S0_q, S1_q, D_q over the chunk's vectors, as
// re/im pairs, into partials[(q * gridDim.x + c) * 6 + 0..5].
template <typename Real>
__global__ void __launch_bounds__(kThreads) generator_kernel(const void* muv, const void* nuv, int64_t nvec,
                                                             double* partials) {
  using vec = typename CplxT<Real>::vec;
  using Acc = typename AccFor<Real>::type;
  constexpr int LV = CplxT<Real>::kLogVec, NV = 1 << LV;
  __shared__ double s_red[6 * (kThreads / 32)];
  const int q = blockIdx.y;
  const vec* mu = reinterpret_cast<const vec*>(muv);
  const vec* nu = reinterpret_cast<const vec*>(nuv);
  // the partner of amplitude b is b ^ 2^q: another vector for q >= LV, the
  // other lane of the same vector for q < LV (complex64, q = 0)
  const bool in_vec = q < LV;
  const int64_t pmask = in_vec ? 0 : (int64_t(1) << (q - LV));
  Acc s0r, s0i, s1r, s1i, dr, di;
  for (int64_t i = (int64_t)blockIdx.x * kThreads + threadIdx.x; i < nvec; i += (int64_t)gridDim.x * kThreads) {
    Real m[2 * NV], x[2 * NV], p[2 * NV];
    *reinterpret_cast<vec*>(m) = mu[i];
    *reinterpret_cast<vec*>(x) = nu[i];
    *reinterpret_cast<vec*>(p) = in_vec ? nu[i] : nu[i ^ pmask];
#pragma unroll
    for (int e = 0; e < NV; ++e) {
      const int64_t b = (i << LV) | e;
      const int pe = in_vec ? (e ^ 1) : e;
      const Real mr = m[2 * e], mi = m[2 * e + 1];
      const Real pr = p[2 * pe], pi = p[2 * pe + 1];
      // mu_b conj(nu_partner) = (mr pr + mi pi) + i (mi pr - mr pi)
      if ((b >> q) & 1) {
        s1r.dot(mr, pr);
        s1r.dot(mi, pi);
        s1i.dot(mi, pr);
        s1i.dot(-mr, pi);
        const Real xr = x[2 * e], xi = x[2 * e + 1];
        dr.dot(mr, xr);
        dr.dot(mi, xi);
        di.dot(mi, xr);
        di.dot(-mr, xi);
      } else {
        s0r.dot(mr, pr);
        s0r.dot(mi, pi);
        s0i.dot(mi, pr);
        s0i.dot(-mr, pi);
      }
    }
  }
  Acc acc[6] = {s0r, s0i, s1r, s1i, dr, di};
  block_reduce_write<6>(acc, s_red, partials + ((int64_t)q * gridDim.x + blockIdx.x) * 6, 6);
}

// acc[q * 6 + v] += weight * sum_c partials[(q * nchunks + c) * 6 + v], in a
// fixed order (deterministic).
__global__ void __launch_bounds__(kThreads) generator_accumulate_kernel(const double* partials, int nchunks, int n,
                                                                        double weight, double* acc) {
  for (int t = threadIdx.x; t < 6 * n; t += kThreads) {
    const int q = t / 6, v = t % 6;
    double s = 0.0;
    for (int c = 0; c < nchunks; ++c) s += partials[((int64_t)q * nchunks + c) * 6 + v];
    acc[t] += weight * s;
  }
}

// <a|b> = sum conj(a) b (re, im), |a|^2, |b|^2 per block.
template <typename Real>
__global__ void __launch_bounds__(kThreads) overlap_kernel(const void* av, const void* bv, int64_t nvec,
                                                           double* partials) {
  using vec = typename CplxT<Real>::vec;
  using Acc = typename AccFor<Real>::type;
  constexpr int NV = 1 << CplxT<Real>::kLogVec;
  __shared__ double s_red[4 * (kThreads / 32)];
  const vec* a = reinterpret_cast<const vec*>(av);
  const vec* b = reinterpret_cast<const vec*>(bv);
  Acc re, im, aa, bb;
  for (int64_t i = (int64_t)blockIdx.x * kThreads + threadIdx.x; i < nvec; i += (int64_t)gridDim.x * kThreads) {
    Real x[2 * NV], y[2 * NV];
    *reinterpret_cast<vec*>(x) = a[i];
    *reinterpret_cast<vec*>(y) = b[i];
#pragma unroll
    for (int e = 0; e < NV; ++e) {
      const Real xr = x[2 * e], xi = x[2 * e + 1], yr = y[2 * e], yi = y[2 * e + 1];
      re.dot(xr, yr);
      re.dot(xi, yi);
      im.dot(xr, yi);
      im.dot(-xi, yr);
      aa.dot(xr, xr);
      aa.dot(xi, xi);
      bb.dot(yr, yr);
      bb.dot(yi, yi);
    }
  }
  Acc acc[4] = {re, im, aa, bb};
  block_reduce_write<4>(acc, s_red, partials + (int64_t)blockIdx.x * 4, 4);
}

}  // namespace

cudaError_t launch_conj_weight(const void* in, void* out, int64_t dim, bool c64, int n, const double* w_bits,
                               int grid, cudaStream_t stream) {
  if (c64)
    conj_weight_kernel<float><<<grid, kThreads, 0, stream>>>(in, out, dim / 2, n, w_bits);
  else
    conj_weight_kernel<double><<<grid, kThreads, 0, stream>>>(in, out, dim, n, w_bits);
  return cudaGetLastError();
}

cudaError_t launch_generator(const void* mu, const void* nu, int64_t dim, bool c64, int n, int nchunks,
                             double* partials, double weight, double* acc, cudaStream_t stream) {
  const dim3 grid(nchunks, n);
  if (c64)
    generator_kernel<float><<<grid, kThreads, 0, stream>>>(mu, nu, dim / 2, partials);
  else
    generator_kernel<double><<<grid, kThreads, 0, stream>>>(mu, nu, dim, partials);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  generator_accumulate_kernel<<<1, kThreads, 0, stream>>>(partials, nchunks, n, weight, acc);
  return cudaGetLastError();
}

cudaError_t launch_overlap(const void* a, const void* b, int64_t dim, bool c64, double* partials, int grid,
                           cudaStream_t stream) {
  if (c64)
    overlap_kernel<float><<<grid, kThreads, 0, stream>>>(a, b, dim / 2, partials);
  else
    overlap_kernel<double><<<grid, kThreads, 0, stream>>>(a, b, dim, partials);
  return cudaGetLastError();
}

}  // namespace rsv
