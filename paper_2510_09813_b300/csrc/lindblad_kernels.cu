// Open-system dynamics (arXiv 2510.09813, Sec. III.A): the Lindblad master
// equation d rho/dt = L(rho) on the vectorised density matrix, evolved by a
// Krylov (Arnoldi) exponential, since L is not Hermitian.
//
// Layout: rho is a 2^n x 2^n complex128 matrix stored row-major, so
// vec(rho) has 2n index bits, the row r in bits [n, 2n) and the column c in
// bits [0, n). Noise channels per atom (bit q): Rydberg dephasing
// L = sqrt(gd_q) n_q and spontaneous decay L = sqrt(gr_q) |0><1|_q. Then
//   L(rho)[r,c] = d(r,c) rho[r,c]
//               - i sum_q <r|h_q|r^q> rho[r^q, c] + i sum_q <c^q|h_q|c> rho[r, c^q]
//               + sum_q gr_q [r_q = c_q = 0] rho[r^q, c^q],
//   d(r,c) = -i (E(r) - E(c)) - sum_q (gd_q / 2 [r_q != c_q] + gr_q / 2 (r_q + c_q)),
// with E the diagonal of Eq. (3) and <0|h_q|1> = Omega_q/2 e^{+i phi_q},
// <1|h_q|0> its conjugate.
#include "kernels.h"
#include "rsv_common.cuh"

namespace rsv {

namespace {

__device__ __forceinline__ double2 cmul(double2 a, double2 b) {
  return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__device__ __forceinline__ double2 cadd(double2 a, double2 b) { return make_double2(a.x + b.x, a.y + b.y); }

__global__ void __launch_bounds__(kThreads) lindblad_apply_kernel(const double2* __restrict__ x,
                                                                  double2* __restrict__ y,
                                                                  const double* __restrict__ E, int64_t total,
                                                                  const LindbladParams p) {
  const int n = p.n;
  const int64_t cmask = (int64_t(1) << n) - 1;
  for (int64_t idx = (int64_t)blockIdx.x * kThreads + threadIdx.x; idx < total;
       idx += (int64_t)gridDim.x * kThreads) {
    const int64_t r = idx >> n, c = idx & cmask;
    double decay = 0.0;
    double2 acc = make_double2(0.0, 0.0);
    for (int q = 0; q < n; ++q) {
      const int br = (int)((r >> q) & 1), bc = (int)((c >> q) & 1);
      decay += 0.5 * p.gd[q] * (double)(br ^ bc) + 0.5 * p.gr[q] * (double)(br + bc);
      const double2 h01 = make_double2(p.hre[q], p.him[q]);  // <0|h|1>
      const double2 h10 = make_double2(p.hre[q], -p.him[q]); // <1|h|0>
      // -i <r|h|r^q> rho[r^q, c]
      const double2 hr = br ? h10 : h01;
      const double2 tr = cmul(hr, x[idx ^ (int64_t(1) << (n + q))]);
      acc = cadd(acc, make_double2(tr.y, -tr.x));
      // +i <c^q|h|c> rho[r, c^q]
      const double2 hc = bc ? h01 : h10;
      const double2 tc = cmul(hc, x[idx ^ (int64_t(1) << q)]);
      acc = cadd(acc, make_double2(-tc.y, tc.x));
      // decay jump: rho[r^q, c^q] (both bits 1) feeds [r, c] (both bits 0)
      if (!br && !bc && p.gr[q] > 0.0) {
        const double2 v = x[idx ^ (int64_t(1) << (n + q)) ^ (int64_t(1) << q)];
        acc.x += p.gr[q] * v.x;
        acc.y += p.gr[q] * v.y;
      }
    }
    const double2 v = x[idx];
    const double2 d = make_double2(-decay, -(E[r] - E[c]));
    y[idx] = cadd(acc, cmul(d, v));
  }
}

// Block (chunk c, vector k): sum conj(V_k) w over the chunk ->
// partials[(k * gridDim.x + c) * 2 + {re, im}].
__global__ void __launch_bounds__(kThreads) multi_dot_kernel(const double2* const* __restrict__ V,
                                                             const double2* __restrict__ w, int64_t total,
                                                             double* __restrict__ partials) {
  __shared__ double s_red[2 * (kThreads / 32)];
  const double2* v = V[blockIdx.y];
  AccD re, im;
  for (int64_t i = (int64_t)blockIdx.x * kThreads + threadIdx.x; i < total; i += (int64_t)gridDim.x * kThreads) {
    const double2 a = v[i], b = w[i];
    re.dot(a.x, b.x);
    re.dot(a.y, b.y);
    im.dot(a.x, b.y);
    im.dot(-a.y, b.x);
  }
  AccD acc[2] = {re, im};
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
__global__ void __launch_bounds__(kThreads) multi_axpy_kernel(const double2* const* __restrict__ V,
                                                              const double* __restrict__ coef, int nvec,
                                                              double2* __restrict__ w, int64_t total, int overwrite,
                                                              double* __restrict__ partials) {
  __shared__ double s_c[2 * kLindbladMaxKrylov];
  __shared__ double s_red[kThreads / 32];
  for (int t = threadIdx.x; t < 2 * nvec; t += kThreads) s_c[t] = coef[t];
  __syncthreads();
  AccD nrm;
  for (int64_t i = (int64_t)blockIdx.x * kThreads + threadIdx.x; i < total; i += (int64_t)gridDim.x * kThreads) {
    double2 a = overwrite ? make_double2(0.0, 0.0) : w[i];
    for (int k = 0; k < nvec; ++k) {
      const double2 v = V[k][i];
      const double cr = s_c[2 * k], ci = s_c[2 * k + 1];
      a.x -= cr * v.x - ci * v.y;
      a.y -= cr * v.y + ci * v.x;
    }
    w[i] = a;
    nrm.dot(a.x, a.x);
    nrm.dot(a.y, a.y);
  }
  AccD acc[1] = {nrm};
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

cudaError_t launch_lindblad_apply(const void* x, void* y, const double* E, const LindbladParams& p, int grid,
                                  cudaStream_t stream) {
  const int64_t total = int64_t(1) << (2 * p.n);
  lindblad_apply_kernel<<<grid, kThreads, 0, stream>>>(static_cast<const double2*>(x), static_cast<double2*>(y), E,
                                                       total, p);
  return cudaGetLastError();
}

cudaError_t launch_multi_dot(const void* const* V, int nvec, const void* w, int64_t total, int nchunks,
                             double* partials, double* out, cudaStream_t stream) {
  const dim3 grid(nchunks, nvec);
  multi_dot_kernel<<<grid, kThreads, 0, stream>>>(reinterpret_cast<const double2* const*>(V),
                                                  static_cast<const double2*>(w), total, partials);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  reduce_dots_kernel<<<1, kThreads, 0, stream>>>(partials, nchunks, nvec, out);
  return cudaGetLastError();
}

cudaError_t launch_multi_axpy(const void* const* V, const double* coef, int nvec, void* w, int64_t total,
                              bool overwrite, int grid, double* partials, double* norm2_out, cudaStream_t stream) {
  if (nvec > kLindbladMaxKrylov) return cudaErrorInvalidValue;
  multi_axpy_kernel<<<grid, kThreads, 0, stream>>>(reinterpret_cast<const double2* const*>(V), coef, nvec,
                                                   static_cast<double2*>(w), total, overwrite ? 1 : 0, partials);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  reduce_sum_kernel<<<1, kThreads, 0, stream>>>(partials, grid, norm2_out);
  return cudaGetLastError();
}

}  // namespace rsv
