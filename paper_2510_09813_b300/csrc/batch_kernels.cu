// Batched time evolution of many small registers in one persistent launch
// (arXiv 2510.09813, Eq. (3), Eq. (6), Sec. III.A for each register).
//
// Each CTA takes registers from a shared work counter (largest first) and
// runs a register's whole pulse sequence before taking the next: per time
// step the midpoint Hamiltonian, the Lanczos recurrence, the FP64
// tridiagonal exponential with its acceptance test and substeps, the combine
// psi = |psi| sum_k u_k v_k and the occupations <n_i>. Nothing returns to the
// host between steps.
//
// Matvec of one Krylov vector v (2^n amplitudes, in global memory, L2-resident
// for the sizes this kernel serves): chunks of 2^T amplitudes (T = min(n, TB))
// are staged in shared memory; flips of bits < T read the staged chunk, flips
// of bits >= T read the partner chunk from global memory (coalesced). The
// diagonal E(b) = E_hi(chunk) + sum_{q<T} w_q b_q + Q[b mod 2^T] is never
// stored: Q is a per-register shared table, (w_q, E_hi) a per-chunk row.
// Registers with n <= TB are one chunk: forming v_j from (u, v_{j-1}) fuses
// into the staging, so an iteration is a single sweep.
#include "kernels.h"
#include "krylov_math.cuh"
#include "rsv_common.cuh"

namespace rsv {

template <typename Real>
struct BatchCfg;
template <>
struct BatchCfg<float> {
  static constexpr int TB = 12;  // 2^12 complex64 = 32 KiB chunk
};
template <>
struct BatchCfg<double> {
  static constexpr int TB = 11;  // 2^11 complex128 = 32 KiB chunk
};

template <typename Real>
size_t batch_dynamic_smem() {
  using C2 = typename CplxT<Real>::type;
  return (sizeof(C2) + sizeof(Real)) << BatchCfg<Real>::TB;
}

namespace {

template <typename Real>
struct Shared {
  using C2 = typename CplxT<Real>::type;
  double V[kBatchMaxAtoms][kBatchMaxAtoms];  // pair energies by bit position
  double delta[kBatchMaxAtoms];
  Real h[kBatchMaxAtoms];                    // Omega/2
  Real hc[kBatchMaxAtoms], hs[kBatchMaxAtoms];  // Omega/2 cos phi, Omega/2 sin phi
  Real w[BatchCfg<Real>::TB];
  Real ehi;
  double al[kMaxKrylov], be[kMaxKrylov + 1], ur[kMaxKrylov], ui[kMaxKrylov];
  Real cr[kMaxKrylov], ci[kMaxKrylov];
  ChebWork cw;
  double red[(kBatchMaxAtoms + 1) * (kThreads / 32)];
  double tot[kBatchMaxAtoms + 1];
  double tau;
  double tau_take, err, alpha, beta;
  int status;
  int m;
  int item;
};

__device__ __forceinline__ float2 cmul_re(float2 x, float r) { return make_float2(x.x * r, x.y * r); }
__device__ __forceinline__ double2 cmul_re(double2 x, double r) { return make_double2(x.x * r, x.y * r); }

template <typename C2, typename Real>
__device__ __forceinline__ C2 make_c(Real re, Real im) {
  C2 z;
  z.x = re;
  z.y = im;
  return z;
}

// Per-chunk diagonal row: s.w[q] = sum_{r >= T} V_qr b_r - delta_q (q < T) and
// s.ehi = sum_{T <= q < r} V_qr b_q b_r - sum_{q >= T} delta_q b_q for the high
// bits b_r of chunk c. One warp.
template <typename Real>
__device__ void chunk_row(Shared<Real>& s, int n, int T, int64_t c, int lane) {
  if (lane < T) {
    double w = -s.delta[lane];
    for (int r = T; r < n; ++r)
      if ((c >> (r - T)) & 1) w += s.V[lane][r];
    s.w[lane] = (Real)w;
  }
  if (lane == 0) {
    double e = 0.0;
    for (int q = T; q < n; ++q) {
      if (!((c >> (q - T)) & 1)) continue;
      e -= s.delta[q];
      for (int r = q + 1; r < n; ++r)
        if ((c >> (r - T)) & 1) e += s.V[q][r];
    }
    s.ehi = (Real)e;
  }
}

// Flip term c_q(b) p of Eq. (3) with the phase: Omega/2 e^{+i phi} when bit q
// of b is 0, Omega/2 e^{-i phi} when it is 1.
template <typename Real, bool PHI>
__device__ __forceinline__ void add_flip(const Shared<Real>& s, int q, bool bit, typename CplxT<Real>::type p, Real& yr,
                                         Real& yi) {
  if (PHI) {
    const Real hc = s.hc[q];
    const Real hs = bit ? -s.hs[q] : s.hs[q];
    yr = fma(hc, p.x, fma(-hs, p.y, yr));
    yi = fma(hc, p.y, fma(hs, p.x, yi));
  } else {
    const Real h = s.h[q];
    yr = fma(h, p.x, yr);
    yi = fma(h, p.y, yi);
  }
}

// Diagonal and flips of bits q < T of the amplitude at chunk-local index blo
// of a contiguous chunk staged in s_x; lin = sum_{q<T} w_q b_q.
template <typename Real, bool PHI>
__device__ __forceinline__ typename CplxT<Real>::type apply_low(const Shared<Real>& s,
                                                                 const typename CplxT<Real>::type* s_x,
                                                                 const Real* s_q, int T, int blo, Real lin) {
  using C2 = typename CplxT<Real>::type;
  const C2 x = s_x[blo];
  const Real e = s.ehi + lin + s_q[blo];
  Real yr = e * x.x, yi = e * x.y;
  for (int q = 0; q < T; ++q) add_flip<Real, PHI>(s, q, (blo >> q) & 1, s_x[blo ^ (1 << q)], yr, yi);
  return make_c<C2>(yr, yi);
}

template <typename Acc, typename Real>
__device__ __forceinline__ void acc_dot3(Acc& r0, Acc& r1, Acc& r2, Real xr, Real xi, Real yr, Real yi) {
  if constexpr (sizeof(Real) == 4) {
    r0.add(fmaf(xi, yi, xr * yr));
    r1.add(fmaf(yi, yi, yr * yr));
    r2.add(fmaf(xi, xi, xr * xr));
  } else {
    r0.dot(xr, yr);
    r0.dot(xi, yi);
    r1.dot(yr, yr);
    r1.dot(yi, yi);
    r2.dot(xr, xr);
    r2.dot(xi, xi);
  }
}

// One Lanczos iteration j of a register (all threads of the CTA):
//   v_j = (u - a v_{j-1}) * sc (j > 0) or psi * sc (j = 0), written to basis[j];
//   u   = H v_j - bprev v_{j-1};
//   Re<v_j, u>, |u|^2, |v_j|^2 -> s.tot[0..2].
// Pass A walks contiguous chunks of 2^T amplitudes: it forms v_j while staging
// it, then applies the diagonal and the flips of bits < T. For n > T, pass B
// walks strided chunks (2^cb contiguous amplitudes times every value of the
// h = n - T high bits, cb = T - h) staged from v_j and adds the flips of the
// high bits to u. Every global access is a coalesced run of the chunk layout.
template <typename Real, bool PHI>
__device__ void lanczos_iteration(Shared<Real>& s, typename CplxT<Real>::type* s_x, const Real* s_q, int n, int T,
                                  const typename CplxT<Real>::type* src, typename CplxT<Real>::type* basis_j,
                                  const typename CplxT<Real>::type* basis_prev, typename CplxT<Real>::type* u,
                                  int j, Real a, Real sc, Real bprev) {
  using C2 = typename CplxT<Real>::type;
  using Acc = typename AccFor<Real>::type;
  constexpr int KMAX = 1 << (BatchCfg<Real>::TB - 8);
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int64_t D = int64_t(1) << n;
  const int chunk = 1 << T;
  const int per = chunk >= kThreads ? chunk / kThreads : 1;
  const bool active = tid < chunk;
  const int64_t nch = D >> T;
  Acc r0, r1, r2;
  for (int64_t c = 0; c < nch; ++c) {
    const int64_t base = c << T;
    if (warp == 0) chunk_row(s, n, T, c, lane);
    if (active) {
#pragma unroll
      for (int k = 0; k < KMAX; ++k) {
        if (k >= per) break;
        const int blo = tid + k * kThreads;
        const C2 x = src[base + blo];
        C2 v;
        if (j == 0) {
          v = cmul_re(x, sc);
        } else {
          const C2 p = basis_prev[base + blo];
          v = make_c<C2>((x.x - a * p.x) * sc, (x.y - a * p.y) * sc);
        }
        s_x[blo] = v;
        basis_j[base + blo] = v;
      }
    }
    __syncthreads();
    if (active) {
      Real lin_t = 0;
      for (int q = 0; q < T && q < 8; ++q)
        if ((tid >> q) & 1) lin_t += s.w[q];
#pragma unroll
      for (int k = 0; k < KMAX; ++k) {
        if (k >= per) break;
        const int blo = tid + k * kThreads;
        Real lin = lin_t;
        for (int q = 8; q < T; ++q)
          if ((k >> (q - 8)) & 1) lin += s.w[q];
        C2 y = apply_low<Real, PHI>(s, s_x, s_q, T, blo, lin);
        if (j > 0) {
          // v_{j-1} again (this thread read the same words while staging)
          const C2 p = basis_prev[base + blo];
          y.x = fma(-bprev, p.x, y.x);
          y.y = fma(-bprev, p.y, y.y);
        }
        u[base + blo] = y;
        if (nch == 1) {
          const C2 x = s_x[blo];
          acc_dot3(r0, r1, r2, x.x, x.y, y.x, y.y);
        }
      }
    }
    __syncthreads();
  }
  if (nch > 1) {
    const int h = n - T, cb = T - h;
    const int64_t nsc = int64_t(1) << (T - cb);
    const int lowmask = (1 << cb) - 1;
    for (int64_t g = 0; g < nsc; ++g) {
#pragma unroll
      for (int k = 0; k < KMAX; ++k) {
        if (k >= per) break;
        const int idx = tid + k * kThreads;
        const int64_t b = ((int64_t)(idx >> cb) << T) | (g << cb) | (idx & lowmask);
        s_x[idx] = basis_j[b];
      }
      __syncthreads();
#pragma unroll
      for (int k = 0; k < KMAX; ++k) {
        if (k >= per) break;
        const int idx = tid + k * kThreads;
        const int64_t b = ((int64_t)(idx >> cb) << T) | (g << cb) | (idx & lowmask);
        C2 y = u[b];
        for (int q = T; q < n; ++q) {
          const int bit = cb + (q - T);
          add_flip<Real, PHI>(s, q, (idx >> bit) & 1, s_x[idx ^ (1 << bit)], y.x, y.y);
        }
        u[b] = y;
        const C2 x = s_x[idx];
        acc_dot3(r0, r1, r2, x.x, x.y, y.x, y.y);
      }
      __syncthreads();
    }
  }
  Acc acc[3] = {r0, r1, r2};
  block_reduce_write<3>(acc, s.red, s.tot, 3);
}

// psi = sum_{k<m} (cr_k + i ci_k) basis_k (combine) or psi as is (observe),
// with |psi|^2 -> s.tot[0] and sum_b |psi_b|^2 b_q -> s.tot[1 + q].
template <typename Real>
__device__ void combine_observe(Shared<Real>& s, int n, int T, typename CplxT<Real>::type* psi,
                                const typename CplxT<Real>::type* basis, int64_t stride, int m, bool combine) {
  using C2 = typename CplxT<Real>::type;
  using Acc = typename AccFor<Real>::type;
  constexpr int KB = BatchCfg<Real>::TB - 8;
  constexpr int HB = kBatchMaxAtoms - 8;
  const int tid = threadIdx.x;
  const int64_t D = int64_t(1) << n;
  const int chunk = 1 << T;
  const int per = chunk >= kThreads ? chunk / kThreads : 1;
  const bool active = tid < chunk;
  const int64_t nch = D >> T;
  Acc tot, reg[KB > 0 ? KB : 1], hi[HB];
  if (active) {
    for (int64_t c = 0; c < nch; ++c) {
      Acc ct;
      for (int k = 0; k < per; ++k) {
        const int64_t b = (c << T) + tid + k * kThreads;
        C2 x;
        if (combine) {
          Real xr = 0, xi = 0;
          for (int i = 0; i < m; ++i) {
            const C2 v = basis[i * stride + b];
            const Real cr = s.cr[i], ci = s.ci[i];
            xr = fma(cr, v.x, fma(-ci, v.y, xr));
            xi = fma(cr, v.y, fma(ci, v.x, xi));
          }
          x = make_c<C2>(xr, xi);
          psi[b] = x;
        } else {
          x = psi[b];
        }
        Acc pv;
        pv.dot(x.x, x.x);
        pv.dot(x.y, x.y);
        ct.merge_acc(pv);
#pragma unroll
        for (int r = 0; r < KB; ++r)
          if ((k >> r) & 1) reg[r].merge_acc(pv);
      }
      tot.merge_acc(ct);
#pragma unroll
      for (int h = 0; h < HB; ++h)
        if (T + h < n && ((c >> h) & 1)) hi[h].merge_acc(ct);
    }
  }
  Acc out[kBatchMaxAtoms + 1];
  out[0] = tot;
#pragma unroll
  for (int q = 0; q < kBatchMaxAtoms; ++q) {
    if (q >= n) continue;
    if (q < 8) {
      if ((tid >> q) & 1) out[1 + q] = tot;
    } else if (q < T) {
#pragma unroll
      for (int r = 0; r < KB; ++r)
        if (r == q - 8) out[1 + q] = reg[r];
    } else {
#pragma unroll
      for (int h = 0; h < HB; ++h)
        if (h == q - T) out[1 + q] = hi[h];
    }
  }
  block_reduce_write<kBatchMaxAtoms + 1>(out, s.red, s.tot, n + 1);
}

}  // namespace

template <typename Real>
__global__ void __launch_bounds__(kThreads, 2) batch_kernel(const BatchArgs A) {
  using C2 = typename CplxT<Real>::type;
  constexpr int TB = BatchCfg<Real>::TB;
  extern __shared__ __align__(16) unsigned char dyn[];
  C2* s_x = reinterpret_cast<C2*>(dyn);
  Real* s_q = reinterpret_cast<Real*>(dyn + (sizeof(C2) << TB));
  __shared__ Shared<Real> s;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  C2* states = reinterpret_cast<C2*>(A.states);
  C2* work = reinterpret_cast<C2*>(A.work) + (int64_t)blockIdx.x * A.work_stride;

  for (;;) {
    if (tid == 0) s.item = atomicAdd(A.next, 1);
    __syncthreads();
    const int qi = s.item;
    if (qi >= A.count) break;
    const BatchItem it = A.items[A.order[qi]];
    const int n = it.n;
    const int T = n < TB ? n : TB;
    const int64_t D = int64_t(1) << n;
    C2* psi = states + it.state_off;
    C2* u = work + (int64_t)A.m_max * D;
    const double* V = A.vmat + it.vmat_off;
    for (int i = tid; i < n * n; i += kThreads) s.V[i / n][i % n] = V[i];
    __syncthreads();
    // Q[t] = sum_{q<r<T} V_qr t_q t_r over the low bits of b (FP64, rounded once)
    for (int t = tid; t < (1 << T); t += kThreads) {
      double e = 0.0;
      for (int r = 1; r < T; ++r) {
        if (!((t >> r) & 1)) continue;
        for (int q = 0; q < r; ++q)
          if ((t >> q) & 1) e += s.V[q][r];
      }
      s_q[t] = (Real)e;
    }
    // initial |psi|^2 and occupation row 0
    combine_observe<Real>(s, n, T, psi, nullptr, 0, 0, false);
    double norm2 = s.tot[0];
    int row = 0;
    auto record = [&](int r) {
      if (r < it.occ_rows && tid < n) A.occ[it.occ_off + (int64_t)r * n + tid] = s.tot[1 + (n - 1 - tid)];
    };
    record(row++);
    int last_m = 0;
    int64_t iters = 0, subs = 0;
    double max_err = 0.0;
    int status = 0;
    for (int step = 0; step < it.steps && status == 0; ++step) {
      const double* P = A.params + it.param_off + (int64_t)step * (1 + 3 * n);
      __syncthreads();
      if (tid < n) {
        const double h = 0.5 * P[1 + tid];
        const double ph = it.has_phi ? P[1 + 2 * n + tid] : 0.0;
        s.h[tid] = (Real)h;
        s.hc[tid] = (Real)(h * cos(ph));
        s.hs[tid] = (Real)(h * sin(ph));
        s.delta[tid] = P[1 + n + tid];
      }
      if (tid == 0) s.tau = P[0];
      __syncthreads();
      double tau_rem = s.tau;
      int sub = 0;
      while (tau_rem > 0.0 && norm2 > 0.0) {
        const double b0 = sqrt(norm2);
        const int check_from = last_m > 2 ? last_m - 2 : 1;
        double a = 0.0, sc = 1.0 / b0, bprev = 0.0;
        int m = 0;
        for (int j = 0; j < A.m_max; ++j) {
          C2* bj = work + (int64_t)j * D;
          const C2* bp = j > 0 ? work + (int64_t)(j - 1) * D : nullptr;
          const C2* src = j == 0 ? psi : u;
          if (it.has_phi)
            lanczos_iteration<Real, true>(s, s_x, s_q, n, T, src, bj, bp, u, j, (Real)a, (Real)sc, (Real)bprev);
          else
            lanczos_iteration<Real, false>(s, s_x, s_q, n, T, src, bj, bp, u, j, (Real)a, (Real)sc, (Real)bprev);
          ++iters;
          m = j + 1;
          if (warp == 0) {
            const LanczosScalars ls = lanczos_scalars(s.tot[0], s.tot[1], s.tot[2]);
            const double alpha = ls.alpha, beta = ls.beta;
            const int mk = ls.vanished ? m - 1 : m;  // accepted dimension if the space ends here
            if (lane == 0) {
              s.al[j] = alpha;
              s.be[m] = beta;
            }
            __syncwarp();
            double tn = 0.0;
            for (int i = lane; i < mk; i += 32)
              tn = fmax(tn, fabs(s.al[i]) + fabs(s.be[i + 1]) + (i > 0 ? fabs(s.be[i]) : 0.0));
#pragma unroll
            for (int off = 16; off > 0; off >>= 1) tn = fmax(tn, __shfl_xor_sync(0xffffffffu, tn, off));
            const bool breakdown = ls.vanished || beta <= A.breakdown * fmax(tn, 1e-300);
            const bool check = breakdown || m >= check_from || m >= A.m_max;
            const KrylovDecision d = krylov_decide(s.al, s.be, mk, ls.vanished ? 0.0 : beta, tau_rem, breakdown,
                                                   check, A.m_max, A.tol, s.ur, s.ui, s.cw);
            if (d.status != kContinue) {
              for (int i = lane; i < mk; i += 32) {
                s.cr[i] = (Real)(b0 * s.ur[i]);
                s.ci[i] = (Real)(b0 * s.ui[i]);
              }
            }
            if (lane == 0) {
              s.m = mk;
              s.status = d.status;
              s.tau_take = d.tau_take;
              s.err = d.err;
              s.alpha = alpha;
              s.beta = beta;
            }
          }
          __syncthreads();
          if (s.status != kContinue) {
            m = s.m;
            break;
          }
          a = s.alpha;
          sc = 1.0 / s.beta;
          bprev = s.beta;
        }
        const int st = s.status;
        const double take = s.tau_take;
        max_err = fmax(max_err, s.err);
        last_m = m;
        double rem = tau_rem - take;
        if (st == kDone || rem <= 1e-14 * tau_rem) rem = 0.0;
        combine_observe<Real>(s, n, T, psi, work, D, m, true);
        norm2 = s.tot[0];
        tau_rem = rem;
        if (tau_rem > 0.0) {
          ++sub;
          ++subs;
          if (sub > A.max_substeps) {
            status = -3;
            break;
          }
        }
      }
      const int done = step + 1;
      if ((it.obs_stride > 0 && done % it.obs_stride == 0) || done == it.steps) record(row++);
    }
    if (tid == 0) {
      BatchOut o;
      o.iterations = iters;
      o.substeps = subs;
      o.max_err = max_err;
      o.norm2 = norm2;
      o.status = status;
      o.rows = row < it.occ_rows ? row : it.occ_rows;
      A.out[A.order[qi]] = o;
    }
    __syncthreads();
  }
}

cudaError_t launch_batch(const BatchArgs& a, bool c64, int grid, cudaStream_t stream) {
  if (c64)
    batch_kernel<float><<<grid, kThreads, batch_dynamic_smem<float>(), stream>>>(a);
  else
    batch_kernel<double><<<grid, kThreads, batch_dynamic_smem<double>(), stream>>>(a);
  return cudaGetLastError();
}

int batch_prepare(bool c64) {
  int nb = 0;
  // several CTAs per SM need the shared-memory side of the L1/shared split
  if (c64) {
    cudaFuncSetAttribute(batch_kernel<float>, cudaFuncAttributePreferredSharedMemoryCarveout, 100);
    cudaFuncSetAttribute(batch_kernel<float>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)batch_dynamic_smem<float>());
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, batch_kernel<float>, kThreads, batch_dynamic_smem<float>());
  } else {
    cudaFuncSetAttribute(batch_kernel<double>, cudaFuncAttributePreferredSharedMemoryCarveout, 100);
    cudaFuncSetAttribute(batch_kernel<double>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)batch_dynamic_smem<double>());
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, batch_kernel<double>, kThreads, batch_dynamic_smem<double>());
  }
  return nb;
}

}  // namespace rsv
