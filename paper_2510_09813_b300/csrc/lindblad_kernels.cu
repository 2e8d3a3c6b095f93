// Open-system dynamics (arXiv 2510.09813, Sec. III.A): the Lindblad master
// equation d rho/dt = L(rho) on the vectorised density matrix, evolved by a
// Krylov (Arnoldi) exponential, since L is not Hermitian.
//
// Layout: rho is a 2^n x 2^n complex matrix stored row-major, so vec(rho)
// has 2n index bits, the row r in bits [n, 2n) and the column c in bits
// [0, n). Noise channels per atom (bit q): Rydberg dephasing
// L = sqrt(gd_q) n_q and spontaneous decay L = sqrt(gr_q) |0><1|_q. Then
//   L(rho)[r,c] = d(r,c) rho[r,c]
//               - i sum_q <r|h_q|r^q> rho[r^q, c] + i sum_q <c^q|h_q|c> rho[r, c^q]
//               + sum_q gr_q [r_q = c_q = 0] rho[r^q, c^q],
//   d(r,c) = -i (E(r) - E(c)) - sum_q (gd_q / 2 [r_q != c_q] + gr_q / 2 (r_q + c_q)),
// with E the diagonal of Eq. (3) and <0|h_q|1> = Omega_q/2 e^{+i phi_q},
// <1|h_q|0> its conjugate.
//
// Precision: complex128 works in FP64 throughout. complex64 keeps rho and the
// Krylov basis in FP32 and does the products in FP32 (B300's FP64 rate is a
// small fraction of its FP32 rate, and FP64 arithmetic bounds these kernels),
// while inner products and norms are accumulated exactly-rounded-product,
// compensated-sum (FP64-class), as in the pure-state complex64 path.
#include "kernels.h"
#include "rsv_common.cuh"

namespace rsv {

namespace {

template <typename Real>
struct Cx;
template <>
struct Cx<float> {
  using T = float2;
};
template <>
struct Cx<double> {
  using T = double2;
};

template <typename T>
__device__ __forceinline__ T cmul(T a, T b) {
  return T{a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x};
}

template <typename Real>
__global__ void __launch_bounds__(kThreads) lindblad_apply_kernel(const typename Cx<Real>::T* __restrict__ x,
                                                                  typename Cx<Real>::T* __restrict__ y,
                                                                  const Real* __restrict__ E, int64_t total,
                                                                  const LindbladParams p) {
  using T = typename Cx<Real>::T;
  __shared__ Real s_hre[kLindbladMaxAtoms], s_him[kLindbladMaxAtoms], s_gd[kLindbladMaxAtoms],
      s_gr[kLindbladMaxAtoms];
  const int n = p.n;
  if (threadIdx.x < n) {
    s_hre[threadIdx.x] = (Real)p.hre[threadIdx.x];
    s_him[threadIdx.x] = (Real)p.him[threadIdx.x];
    s_gd[threadIdx.x] = (Real)(0.5 * p.gd[threadIdx.x]);
    s_gr[threadIdx.x] = (Real)p.gr[threadIdx.x];
  }
  __syncthreads();
  const int64_t cmask = (int64_t(1) << n) - 1;
  for (int64_t idx = (int64_t)blockIdx.x * kThreads + threadIdx.x; idx < total;
       idx += (int64_t)gridDim.x * kThreads) {
    const int r = (int)(idx >> n), c = (int)(idx & cmask);
    Real decay = 0;
    T acc{0, 0};
    for (int q = 0; q < n; ++q) {
      const int br = (r >> q) & 1, bc = (c >> q) & 1;
      decay += s_gd[q] * (Real)(br ^ bc) + (Real)0.5 * s_gr[q] * (Real)(br + bc);
      const T h01{s_hre[q], s_him[q]};   // <0|h|1>
      const T h10{s_hre[q], -s_him[q]};  // <1|h|0>
      // -i <r|h|r^q> rho[r^q, c]
      const T tr = cmul(br ? h10 : h01, x[idx ^ (int64_t(1) << (n + q))]);
      acc.x += tr.y;
      acc.y -= tr.x;
      // +i <c^q|h|c> rho[r, c^q]
      const T tc = cmul(bc ? h01 : h10, x[idx ^ (int64_t(1) << q)]);
      acc.x -= tc.y;
      acc.y += tc.x;
      // decay jump: rho[r^q, c^q] (both bits 1) feeds [r, c] (both bits 0)
      if (!br && !bc && s_gr[q] > (Real)0) {
        const T v = x[idx ^ (int64_t(1) << (n + q)) ^ (int64_t(1) << q)];
        acc.x += s_gr[q] * v.x;
        acc.y += s_gr[q] * v.y;
      }
    }
    const T v = x[idx];
    const T d{-decay, -(E[r] - E[c])};
    const T dv = cmul(d, v);
    y[idx] = T{acc.x + dv.x, acc.y + dv.y};
  }
}

// Block (chunk c, vector k): sum conj(V_k) w over the chunk ->
// partials[(k * gridDim.x + c) * 2 + {re, im}].
template <typename Real>
__global__ void __launch_bounds__(kThreads) multi_dot_kernel(const typename Cx<Real>::T* const* __restrict__ V,
                                                             const typename Cx<Real>::T* __restrict__ w,
                                                             int64_t total, double* __restrict__ partials) {
  using T = typename Cx<Real>::T;
  using Acc = typename AccFor<Real>::type;
  __shared__ double s_red[2 * (kThreads / 32)];
  const T* v = V[blockIdx.y];
  Acc re, im;
  for (int64_t i = (int64_t)blockIdx.x * kThreads + threadIdx.x; i < total; i += (int64_t)gridDim.x * kThreads) {
    const T a = v[i], b = w[i];
    re.dot(a.x, b.x);
    re.dot(a.y, b.y);
    im.dot(a.x, b.y);
    im.dot(-a.y, b.x);
  }
  Acc acc[2] = {re, im};
  block_reduce_write<2>(acc, s_red, partials + ((int64_t)blockIdx.y * gridDim.x + blockIdx.x) * 2, 2);
}

// out[2k + part] = sum_c partials[(k * nchunks + c) * 2 + part], fixed order.
__global__ void __launch_bounds__(kThreads) reduce_dots_kernel(const double* __restrict__ partials, int nchunks,
                                                               int nvec, double* __restrict__ out) {
  for (int t = threadIdx.x; t < 2 * nvec; t += kThreads) {
    const int k = t >> 1, part = t & 1;
    double s = 0.0;
    for (int c = 0; c < nchunks; ++c) s += partials[((int64_t)k * nchunks + c) * 2 + part];
    out[t] = s;
  }
}

// w = (overwrite ? 0 : w) - sum_k coef_k V_k, and per block |w|^2 into
// partials[blockIdx.x].
template <typename Real>
__global__ void __launch_bounds__(kThreads) multi_axpy_kernel(const typename Cx<Real>::T* const* __restrict__ V,
                                                              const double* __restrict__ coef, int nvec,
                                                              typename Cx<Real>::T* __restrict__ w, int64_t total,
                                                              int overwrite, double* __restrict__ partials) {
  using T = typename Cx<Real>::T;
  using Acc = typename AccFor<Real>::type;
  __shared__ Real s_c[2 * kLindbladMaxKrylov];
  __shared__ double s_red[kThreads / 32];
  for (int t = threadIdx.x; t < 2 * nvec; t += kThreads) s_c[t] = (Real)coef[t];
  __syncthreads();
  Acc nrm;
  for (int64_t i = (int64_t)blockIdx.x * kThreads + threadIdx.x; i < total; i += (int64_t)gridDim.x * kThreads) {
    T a = overwrite ? T{0, 0} : w[i];
    for (int k = 0; k < nvec; ++k) {
      const T v = V[k][i];
      const Real cr = s_c[2 * k], ci = s_c[2 * k + 1];
      a.x -= cr * v.x - ci * v.y;
      a.y -= cr * v.y + ci * v.x;
    }
    w[i] = a;
    nrm.dot(a.x, a.x);
    nrm.dot(a.y, a.y);
  }
  Acc acc[1] = {nrm};
  block_reduce_write<1>(acc, s_red, partials + blockIdx.x, 1);
}

__global__ void __launch_bounds__(kThreads) reduce_sum_kernel(const double* __restrict__ partials, int count,
                                                              double* __restrict__ out) {
  __shared__ double s[kThreads];
  double v = 0.0;
  for (int i = threadIdx.x; i < count; i += kThreads) v += partials[i];
  s[threadIdx.x] = v;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int i = 0; i < kThreads; ++i) t += s[i];
    out[0] = t;
  }
}

}  // namespace

cudaError_t launch_lindblad_apply(const void* x, void* y, const void* E, const LindbladParams& p, bool c64, int grid,
                                  cudaStream_t stream) {
  const int64_t total = int64_t(1) << (2 * p.n);
  if (c64)
    lindblad_apply_kernel<float><<<grid, kThreads, 0, stream>>>(static_cast<const float2*>(x),
                                                                static_cast<float2*>(y),
                                                                static_cast<const float*>(E), total, p);
  else
    lindblad_apply_kernel<double><<<grid, kThreads, 0, stream>>>(static_cast<const double2*>(x),
                                                                 static_cast<double2*>(y),
                                                                 static_cast<const double*>(E), total, p);
  return cudaGetLastError();
}

cudaError_t launch_multi_dot(const void* const* V, int nvec, const void* w, int64_t total, bool c64, int nchunks,
                             double* partials, double* out, cudaStream_t stream) {
  const dim3 grid(nchunks, nvec);
  if (c64)
    multi_dot_kernel<float><<<grid, kThreads, 0, stream>>>(reinterpret_cast<const float2* const*>(V),
                                                           static_cast<const float2*>(w), total, partials);
  else
    multi_dot_kernel<double><<<grid, kThreads, 0, stream>>>(reinterpret_cast<const double2* const*>(V),
                                                            static_cast<const double2*>(w), total, partials);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  reduce_dots_kernel<<<1, kThreads, 0, stream>>>(partials, nchunks, nvec, out);
  return cudaGetLastError();
}

cudaError_t launch_multi_axpy(const void* const* V, const double* coef, int nvec, void* w, int64_t total, bool c64,
                              bool overwrite, int grid, double* partials, double* norm2_out, cudaStream_t stream) {
  if (nvec > kLindbladMaxKrylov) return cudaErrorInvalidValue;
  if (c64)
    multi_axpy_kernel<float><<<grid, kThreads, 0, stream>>>(reinterpret_cast<const float2* const*>(V), coef, nvec,
                                                            static_cast<float2*>(w), total, overwrite ? 1 : 0,
                                                            partials);
  else
    multi_axpy_kernel<double><<<grid, kThreads, 0, stream>>>(reinterpret_cast<const double2* const*>(V), coef,
                                                             nvec, static_cast<double2*>(w), total,
                                                             overwrite ? 1 : 0, partials);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  reduce_sum_kernel<<<1, kThreads, 0, stream>>>(partials, grid, norm2_out);
  return cudaGetLastError();
}

}  // namespace rsv
