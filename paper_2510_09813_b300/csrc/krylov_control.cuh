// The Krylov control step of one Lanczos iteration (arXiv 2510.09813,
// Sec. III.A), shared by the stand-alone scalar kernel and the streaming
// passes, whose last CTA runs it at the end of an iteration's last pass.
#pragma once

#include "kernels.h"
#include "krylov_math.cuh"
#include "rsv_common.cuh"
#include "tma.cuh"

namespace rsv {

// ---------------------------------------------------------------------------
// The Krylov control step after the last streaming pass of iteration j:
// reduce the passes' partial sums into alpha_j and beta_{j+1}, test the
// Krylov space (a-posteriori estimate, breakdown, m_max) with the small
// exponential exp(-i tau T_m) e_1, and write what the next pass or the combine
// needs.
//
// Four warps, one per SM sub-partition: FP64 instructions occupy a
// sub-partition's FP64 unit for about 70 cycles each and do not pipeline
// within a warp, so the launch keeps their count on the critical path small.
// Every load the launch needs is issued first; the norm bound of T_m is kept
// in the state (one row added per iteration); the tridiagonal and the kept
// Chebyshev expansion are read only when the convergence test runs.
// ---------------------------------------------------------------------------
constexpr int kControlThreads = 128;

__device__ __forceinline__ uint64_t global_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

struct ControlSmem {
  double part[3][kControlThreads / 32];
  double al[kMaxKrylov], be[kMaxKrylov + 1];
  double ur[kMaxKrylov], ui[kMaxKrylov];
  ChebWork cw;
};

// Threads 0 .. kControlThreads-1 of the calling CTA run it (the others must
// not); they meet at named barrier 1. `w` is shared memory of the CTA.
static __device__ __noinline__ void krylov_control(const ScalarArgs& A, ControlSmem& w) {
  double (&s_part)[3][kControlThreads / 32] = w.part;
  double* s_al = w.al;
  double* s_be = w.be;
  double* s_ur = w.ur;
  double* s_ui = w.ui;
  ChebWork& s_w = w.cw;
  KState* ks = A.ks;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const uint64_t t_start = global_ns();
  // ---- loads, all issued before any of them is used ----
  const int status0 = ks->status;
  const int j = ks->j;
  double v[3] = {0.0, 0.0, 0.0};
  for (int p = tid; p < A.nparts; p += kControlThreads) {
#pragma unroll
    for (int i = 0; i < 3; ++i) v[i] += __ldcg(A.partials + (int64_t)p * 3 + i);  // other CTAs' stores
  }
  const int m = j + 1;
  const bool maybe_check = m >= A.check_from || m >= A.m_max;
  double tn_prev = 0.0, beta_j = 0.0, tau_rem = 0.0, b0 = 0.0;
  double al_i = 0.0, al_i2 = 0.0, be_i = 0.0;  // rows of T_m by lane (and lane + 32)
  if (warp == 0) {
    tn_prev = ks->tnorm;
    beta_j = j > 0 ? ks->beta[j] : 0.0;  // beta[0] is |psi|, not an entry of T
    tau_rem = ks->tau_rem;
    b0 = ks->beta[0];
    if (maybe_check) {
      if (lane < j) al_i = ks->alpha[lane];
      if (lane <= j) be_i = ks->beta[lane];
      if (lane + 32 < j) al_i2 = ks->alpha[lane + 32];
    }
  }
  if (status0 != kContinue) return;  // uniform: the Krylov space is already accepted
  // ---- partial sums: per warp, then four rows ----
#pragma unroll
  for (int i = 0; i < 3; ++i) {
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) v[i] += __shfl_xor_sync(0xffffffffu, v[i], off);
  }
  if (lane == 0) {
#pragma unroll
    for (int i = 0; i < 3; ++i) s_part[i][warp] = v[i];
  }
  named_bar_sync(1, kControlThreads);
  if (warp != 0) return;
  double rs = 0.0;  // lane i < 3: sum i
  if (lane < 3)
    for (int q = 0; q < kControlThreads / 32; ++q) rs += s_part[lane][q];
  const double r0 = __shfl_sync(0xffffffffu, rs, 0), r1 = __shfl_sync(0xffffffffu, rs, 1),
               r2 = __shfl_sync(0xffffffffu, rs, 2);
  // alpha_j = Re<v_j, u_j> / |v_j|^2 and beta_{j+1} = |u_j - alpha_j v_j| expanded
  // as |u|^2 - 2 alpha Re<v,u> + alpha^2 |v|^2 = |u|^2 - alpha Re<v,u>.
  const LanczosScalars ls = lanczos_scalars(r0, r1, r2);
  const double alpha = ls.alpha, beta = ls.beta;
  const int mk = ls.vanished ? m - 1 : m;  // accepted dimension if this space ends here
  // Gershgorin bound of T_mk: the previous rows' maximum and row j
  const double tn = ls.vanished ? tn_prev : fmax(tn_prev, fabs(alpha) + fabs(beta_j) + fabs(beta));
  const bool breakdown = ls.vanished || beta <= A.breakdown * fmax(tn, 1e-300);
  const bool check = breakdown || maybe_check;
  KrylovDecision d{kContinue, 0.0, 0.0};
  if (check) {
    if (!maybe_check) {  // a breakdown before the expected dimension: load now
      if (lane < j) al_i = ks->alpha[lane];
      if (lane <= j) be_i = ks->beta[lane];
      if (lane + 32 < j) al_i2 = ks->alpha[lane + 32];
    }
    if (lane < m) s_al[lane] = (lane == j) ? alpha : al_i;
    if (lane + 32 < m) s_al[lane + 32] = (lane + 32 == j) ? alpha : al_i2;
    for (int i = lane; i <= m; i += 32) s_be[i] = (i == m) ? beta : (i <= j && i < 32 ? be_i : ks->beta[i]);
    // the kept expansion comes from the previous launch (global) and goes back
    // after use; only its header and the Bessel factors matter
    if (lane == 0) {
      s_w.c_valid = A.cache->c_valid;
      s_w.c_pieces = A.cache->c_pieces;
      s_w.kmax = A.cache->kmax;
      s_w.c_lo = A.cache->c_lo;
      s_w.c_hi = A.cache->c_hi;
      s_w.c_tau = A.cache->c_tau;
      s_w.c_pc = A.cache->c_pc;
      s_w.c_ps = A.cache->c_ps;
    }
    __syncwarp();
    if (s_w.c_valid) {
      for (int k = lane; k <= s_w.kmax; k += 32) {
        s_w.J[k] = A.cache->J[k];
        s_w.jh[k] = A.cache->jh[k];
        s_w.jl[k] = A.cache->jl[k];
      }
    }
    __syncwarp();
    d = krylov_decide(s_al, s_be, mk, ls.vanished ? 0.0 : beta, tau_rem, breakdown, true, A.m_max, A.tol, s_ur,
                      s_ui, s_w);
    if (s_w.c_valid) {
      for (int k = lane; k <= s_w.kmax; k += 32) {
        A.cache->J[k] = s_w.J[k];
        A.cache->jh[k] = s_w.jh[k];
        A.cache->jl[k] = s_w.jl[k];
      }
      if (lane == 0) {
        A.cache->c_pieces = s_w.c_pieces;
        A.cache->kmax = s_w.kmax;
        A.cache->c_lo = s_w.c_lo;
        A.cache->c_hi = s_w.c_hi;
        A.cache->c_tau = s_w.c_tau;
        A.cache->c_pc = s_w.c_pc;
        A.cache->c_ps = s_w.c_ps;
        A.cache->c_valid = 1;
      }
    }
  }
  const int status = d.status;
  const double tau_take = d.tau_take, err = d.err;
  if (lane == 0) {
    ks->alpha[j] = alpha;
    ks->beta[m] = beta;
    ks->tnorm = tn;
    ks->total_iterations += 1;
  }
  if (status != kContinue) {
    for (int i = lane; i < mk; i += 32) {
      ks->coef_re[i] = b0 * s_ur[i];
      ks->coef_im[i] = b0 * s_ui[i];
    }
    if (lane == 0) {
      double rem = tau_rem - tau_take;
      if (status == kDone || rem <= 1e-14 * tau_rem) rem = 0.0;
      ks->m = mk;
      ks->tau_taken = tau_take;
      ks->tau_rem = rem;
      ks->err_est = err;
      ks->max_err_est = fmax(ks->max_err_est, err);
      ks->status = status;
    }
  } else if (lane == 0) {
    ks->form_a = alpha;
    ks->form_s = 1.0 / beta;
    ks->beta_prev = beta;
    ks->j = j + 1;
  }
  if (lane == 0) {
    const uint64_t dt = global_ns() - t_start;
    ks->ctl_ns += dt;
    ks->ctl_steps += 1;
    if (check) {
      ks->chk_ns += dt;
      ks->chk_steps += 1;
    }
  }
}

// Tail of the last streaming pass of a Lanczos iteration, reached by every
// thread of a CTA after its last block barrier (red: the warps' three partial
// sums). Thread 0 stores the CTA's sums; with A.ks set (the control step
// fused into the pass), it then counts the CTA in ks->arrivals, and the CTA
// that arrives last runs krylov_control in `ring`, the pass's shared-memory
// ring, whose copies have all landed. The usual last-block pattern: each CTA
// fences its stores before its arrival, the last one fences after it. After a
// timed-out wait (error word set) the step is skipped; the host reports it.
template <int kWarps>
__device__ __forceinline__ void pass_tail(const ScalarArgs& A, double* partials, const double (&red)[3][kWarps],
                                          const int* err, unsigned char* ring) {
  __shared__ int s_run;
  if (threadIdx.x == 0) {
#pragma unroll
    for (int v = 0; v < 3; ++v) {
      double sum = 0.0;
      for (int w = 0; w < kWarps; ++w) sum += red[v][w];
      partials[(int64_t)blockIdx.x * 3 + v] = sum;
    }
    int run = 0;
    if (A.ks) {
      __threadfence();
      if (atomicAdd(&A.ks->arrivals, 1u) == gridDim.x - 1) {
        __threadfence();
        A.ks->arrivals = 0;  // every CTA of this launch has counted itself
        run = *reinterpret_cast<const volatile int*>(err) == 0;
      }
    }
    s_run = run;
  }
  if (!A.ks) return;  // uniform over the launch
  __syncthreads();
  if (s_run && threadIdx.x < kControlThreads) krylov_control(A, *reinterpret_cast<ControlSmem*>(ring));
}

}  // namespace rsv
