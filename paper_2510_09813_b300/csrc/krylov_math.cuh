// FP64 small-matrix part of the Lanczos step (arXiv 2510.09813, Sec. III.A):
// exp(-i tau T_m) e_1 for the real symmetric tridiagonal T_m, and the
// acceptance test of a Krylov space with its substep choice. Used by the
// streaming path's scalar kernel and by the batched kernel.
#pragma once

#include "rsv_common.cuh"

namespace rsv {

constexpr int kMaxBessel = 640;
constexpr double kXMax = 400.0;  // largest Chebyshev argument per piece
constexpr int kMaxPieces = 4096;

// ---------------------------------------------------------------------------
// exp(-i tau T) w for a real symmetric tridiagonal T (m <= kMaxKrylov).
//
// Chebyshev expansion (Tal-Ezer & Kosloff, J. Chem. Phys. 81, 3967 (1984)):
// with T = cen + rad * S, spec(S) in [-1, 1] by Gershgorin,
//   exp(-i x S) = J_0(x) + 2 sum_{k>=1} (-i)^k J_k(x) T_k(S),   x = tau * rad,
// (the Jacobi-Anger expansion) and T_k(S) w by the three-term recurrence.
// J_k(x) comes from Miller's backward recurrence normalised by
// J_0 + 2 sum_k J_{2k} = 1. Long times are split into pieces with x <= kXMax.
// Called by one full warp; w lives in shared memory (re, im arrays).
// ---------------------------------------------------------------------------
// Warp-collective: J[0..K] = J_k(x). The backward recurrence itself is serial
// (lane 0) and multiplies by a hoisted 2/x instead of dividing (FP64 division
// is a long dependent sequence on this part, and it sat inside the loop); the
// normalisation sum and the scaling are spread over the warp.
__device__ inline void bessel_miller(double x, int K, double* J) {
  const int lane = threadIdx.x & 31;
  int M = K + 20 + (int)(5.0f * cbrtf((float)x));
  if (M > kMaxBessel - 2) M = kMaxBessel - 2;
  if (lane == 0) {
    const double two_over_x = 2.0 / x;
    double jp1 = 0.0, jk = 1e-280;
    J[M] = jk;
    for (int k = M; k >= 1; --k) {
      const double jm1 = fma((double)k * two_over_x, jk, -jp1);
      J[k - 1] = jm1;
      jp1 = jk;
      jk = jm1;
      if (fabs(jm1) > 1e250) {
        for (int i = k - 1; i <= M; ++i) J[i] *= 1e-250;
        jp1 *= 1e-250;
        jk *= 1e-250;
      }
    }
  }
  __syncwarp();
  // normalisation J_0 + 2 sum_k J_{2k} = 1, summed in a fixed order per lane
  double s = 0.0;
  for (int k = 2 + 2 * lane; k <= M; k += 64) s += J[k];
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) s += __shfl_xor_sync(0xffffffffu, s, off);
  const double inv = 1.0 / (J[0] + 2.0 * s);
  __syncwarp();
  for (int k = lane; k <= K; k += 32) J[k] *= inv;
  __syncwarp();
}

struct ChebWork {
  double pr[kMaxKrylov], pi[kMaxKrylov];  // phi_{k-1}
  double cr[kMaxKrylov], ci[kMaxKrylov];  // phi_k
  double ar[kMaxKrylov], ai[kMaxKrylov];  // accumulated sum
  double J[kMaxBessel];
  int kmax;
};

// Apply S = (T - cen)/rad to (vr, vi) component i.
__device__ __forceinline__ void apply_s(const double* al, const double* be, int m, double cen, double irad, int i,
                                        const double* vr, const double* vi, double& outr, double& outi) {
  double r = (al[i] - cen) * vr[i], im = (al[i] - cen) * vi[i];
  if (i > 0) {
    r = fma(be[i], vr[i - 1], r);
    im = fma(be[i], vi[i - 1], im);
  }
  if (i + 1 < m) {
    r = fma(be[i + 1], vr[i + 1], r);
    im = fma(be[i + 1], vi[i + 1], im);
  }
  outr = r * irad;
  outi = im * irad;
}

__device__ __forceinline__ void acc_term(int k, double jk, double pr, double pi, double& ar, double& ai) {
  // a_k = (2 - delta_k0) (-i)^k J_k
  const double c = (k == 0) ? jk : 2.0 * jk;
  switch (k & 3) {
    case 0: ar = fma(c, pr, ar); ai = fma(c, pi, ai); break;
    case 1: ar = fma(c, pi, ar); ai = fma(-c, pr, ai); break;
    case 2: ar = fma(-c, pr, ar); ai = fma(-c, pi, ai); break;
    default: ar = fma(-c, pi, ar); ai = fma(c, pr, ai); break;
  }
}

// (ur, ui) <- exp(-i tau T_m) e_1.  al[0..m-1], be[1..m-1]; warp-collective.
__device__ inline void cheb_expm_e1(const double* al, const double* be, int m, double tau, double* ur, double* ui,
                             ChebWork& w) {
  const int lane = threadIdx.x & 31;
  double lo = 1e308, hi = -1e308;
  for (int i = lane; i < m; i += 32) {
    const double bl = i > 0 ? fabs(be[i]) : 0.0;
    const double br = i + 1 < m ? fabs(be[i + 1]) : 0.0;
    lo = fmin(lo, al[i] - bl - br);
    hi = fmax(hi, al[i] + bl + br);
  }
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) {
    lo = fmin(lo, __shfl_xor_sync(0xffffffffu, lo, off));
    hi = fmax(hi, __shfl_xor_sync(0xffffffffu, hi, off));
  }
  const double cen = 0.5 * (lo + hi), rad = 0.5 * (hi - lo);
  for (int i = lane; i < m; i += 32) {
    ur[i] = (i == 0) ? 1.0 : 0.0;
    ui[i] = 0.0;
  }
  __syncwarp();
  if (!(rad > 1e-300) || m == 1) {
    if (lane == 0) {
      double s, c;
      sincos(tau * cen, &s, &c);
      ur[0] = c;
      ui[0] = -s;
    }
    __syncwarp();
    return;
  }
  // |tau| * spectral radius beyond kMaxPieces pieces (or not finite) means the
  // tridiagonal is not a physical one (corrupted recurrence): report NaN, which
  // no acceptance test passes, instead of looping over an unbounded piece count
  const double xt = tau * rad;
  if (!(xt <= kXMax * kMaxPieces)) {
    for (int i = lane; i < m; i += 32) {
      ur[i] = __longlong_as_double(0x7ff8000000000000ll);
      ui[i] = ur[i];
    }
    __syncwarp();
    return;
  }
  int pieces = (int)ceil(xt / kXMax);
  if (pieces < 1) pieces = 1;
  const double tp = tau / pieces, x = tp * rad, irad = 1.0 / rad;
  int K = (int)(x + 12.0f * cbrtf((float)x) + 30.0f);
  if (K > kMaxBessel - 40) K = kMaxBessel - 40;
  if (x < 1e-6) {
    if (lane == 0) {
      // power series J_k(x) = (x/2)^k / k! (1 - (x/2)^2 / (k+1) + ...), k <= 3
      const double h = 0.5 * x;
      w.J[0] = 1.0 - h * h;
      w.J[1] = h * (1.0 - 0.5 * h * h);
      w.J[2] = 0.5 * h * h;
      w.J[3] = h * h * h / 6.0;
      w.kmax = 3;
    }
  } else {
    bessel_miller(x, K, w.J);
    if (lane == 0) {
      int kmax = K;
      while (kmax > 1 && kmax > x && fabs(w.J[kmax]) < 1e-18) --kmax;
      w.kmax = kmax;
    }
  }
  __syncwarp();
  const int kmax = w.kmax;
  double ps, pc;
  sincos(tp * cen, &ps, &pc);
  if (m <= 32) {
    // Register path, one component per lane: the three-term recurrence
    // phi_{k+1} = 2 S phi_k - phi_{k-1} with 2 S's entries folded into three
    // per-lane coefficients and the neighbours phi_k[i -+ 1] by shuffles, so a
    // term costs 8 FP64 instructions (FP64 issues slowly on this part).
    const int i = lane;
    const bool act = i < m;
    const double a2 = act ? 2.0 * (al[i] - cen) * irad : 0.0;
    const double bl = (act && i > 0) ? 2.0 * be[i] * irad : 0.0;
    const double br = (act && i + 1 < m) ? 2.0 * be[i + 1] * irad : 0.0;
    double uR = act ? ur[i] : 0.0, uI = act ? ui[i] : 0.0;
    for (int piece = 0; piece < pieces; ++piece) {
      double pR = uR, pI = uI;  // phi_0
      double aR = w.J[0] * pR, aI = w.J[0] * pI;
      // phi_1 = S phi_0
      double cR = 0.5 * fma(a2, pR, fma(bl, __shfl_up_sync(0xffffffffu, pR, 1), br * __shfl_down_sync(0xffffffffu, pR, 1)));
      double cI = 0.5 * fma(a2, pI, fma(bl, __shfl_up_sync(0xffffffffu, pI, 1), br * __shfl_down_sync(0xffffffffu, pI, 1)));
      {
        const double c = 2.0 * w.J[1];  // (-i)^1
        aR = fma(c, cI, aR);
        aI = fma(-c, cR, aI);
      }
      for (int k = 2; k <= kmax; ++k) {
        const double nR = fma(a2, cR, fma(bl, __shfl_up_sync(0xffffffffu, cR, 1),
                                          fma(br, __shfl_down_sync(0xffffffffu, cR, 1), -pR)));
        const double nI = fma(a2, cI, fma(bl, __shfl_up_sync(0xffffffffu, cI, 1),
                                          fma(br, __shfl_down_sync(0xffffffffu, cI, 1), -pI)));
        pR = cR;
        pI = cI;
        cR = nR;
        cI = nI;
        const double c = 2.0 * w.J[k];
        switch (k & 3) {  // (-i)^k
          case 0: aR = fma(c, nR, aR); aI = fma(c, nI, aI); break;
          case 1: aR = fma(c, nI, aR); aI = fma(-c, nR, aI); break;
          case 2: aR = fma(-c, nR, aR); aI = fma(-c, nI, aI); break;
          default: aR = fma(-c, nI, aR); aI = fma(c, nR, aI); break;
        }
      }
      // u = exp(-i tp cen) * acc
      uR = pc * aR + ps * aI;
      uI = pc * aI - ps * aR;
    }
    if (act) {
      ur[i] = uR;
      ui[i] = uI;
    }
    __syncwarp();
    return;
  }
  for (int piece = 0; piece < pieces; ++piece) {
    // phi_0 = u, phi_1 = S u
    for (int i = lane; i < m; i += 32) {
      w.pr[i] = ur[i];
      w.pi[i] = ui[i];
      w.ar[i] = 0.0;
      w.ai[i] = 0.0;
      acc_term(0, w.J[0], ur[i], ui[i], w.ar[i], w.ai[i]);
    }
    __syncwarp();
    for (int i = lane; i < m; i += 32) {
      double r, im;
      apply_s(al, be, m, cen, irad, i, w.pr, w.pi, r, im);
      w.cr[i] = r;
      w.ci[i] = im;
      acc_term(1, w.J[1], r, im, w.ar[i], w.ai[i]);
    }
    __syncwarp();
    for (int k = 2; k <= kmax; ++k) {
      double nr[2], ni[2];
      int cnt = 0;
      for (int i = lane; i < m; i += 32, ++cnt) {
        double r, im;
        apply_s(al, be, m, cen, irad, i, w.cr, w.ci, r, im);
        nr[cnt] = 2.0 * r - w.pr[i];
        ni[cnt] = 2.0 * im - w.pi[i];
      }
      __syncwarp();
      cnt = 0;
      for (int i = lane; i < m; i += 32, ++cnt) {
        w.pr[i] = w.cr[i];
        w.pi[i] = w.ci[i];
        w.cr[i] = nr[cnt];
        w.ci[i] = ni[cnt];
        acc_term(k, w.J[k], nr[cnt], ni[cnt], w.ar[i], w.ai[i]);
      }
      __syncwarp();
    }
    // u = exp(-i tp cen) * acc
    for (int i = lane; i < m; i += 32) {
      const double r = w.ar[i], im = w.ai[i];
      ur[i] = pc * r + ps * im;
      ui[i] = pc * im - ps * r;
    }
    __syncwarp();
  }
}

// ---------------------------------------------------------------------------
// Lanczos scalars from the sums of one iteration, r0 = Re<v_j, u>,
// r1 = |u|^2, r2 = |v_j|^2 (u = H v_j - beta_j v_{j-1}):
//   alpha_j = r0 / r2,  beta_{j+1}^2 = |u - alpha_j v_j|^2 = r1 - alpha_j r0.
// v_j vanishes (r2 = 0) only when the previous beta was rounding noise of an
// exhausted Krylov space; the caller then drops v_j and accepts dimension j.
// ---------------------------------------------------------------------------
struct LanczosScalars {
  double alpha, beta;
  bool vanished;
};

__device__ inline LanczosScalars lanczos_scalars(double r0, double r1, double r2) {
  LanczosScalars l;
  l.vanished = !(r2 > 0.0) || !isfinite(r0) || !isfinite(r1) || !isfinite(r2);
  l.alpha = l.vanished ? 0.0 : r0 / r2;
  const double b2 = l.vanished ? 0.0 : r1 - l.alpha * r0;
  l.beta = b2 > 0.0 ? sqrt(b2) : 0.0;
  return l;
}

// ---------------------------------------------------------------------------
// Acceptance of the Krylov space of dimension m (warp-collective; one warp).
//
// The a-posteriori estimate err(t) = beta_m |[exp(-i t T_m) e_1]_{m-1}| is
// taken relative to |psi| (T_m comes from the normalised start vector).
//   - breakdown or err(tau_rem) <= tol: accept the whole remaining time;
//   - m == m_max otherwise: the largest t <= tau_rem meeting tol, found by
//     halving and then 4 bisection steps in log t, is accepted as a substep;
//   - else: continue the recurrence.
// On acceptance (ur, ui) holds exp(-i t T_m) e_1 for the accepted t.
// ---------------------------------------------------------------------------
struct KrylovDecision {
  int32_t status;   // kContinue, kDone or kDonePartial
  double tau_take;
  double err;
};

__device__ inline KrylovDecision krylov_decide(const double* al, const double* be, int m, double beta, double tau_rem,
                                        bool breakdown, bool check, int m_max, double tol, double* ur, double* ui,
                                        ChebWork& w) {
  KrylovDecision d{kContinue, 0.0, 0.0};
  if (!check) return d;
  cheb_expm_e1(al, be, m, tau_rem, ur, ui, w);
  d.err = beta * hypot(ur[m - 1], ui[m - 1]);
  if (breakdown || d.err <= tol) {
    d.status = kDone;
    d.tau_take = tau_rem;
  } else if (m >= m_max) {
    double t = tau_rem, t_bad = tau_rem;
    for (int it = 0; it < 64; ++it) {
      t_bad = t;
      t *= 0.5;
      cheb_expm_e1(al, be, m, t, ur, ui, w);
      if (beta * hypot(ur[m - 1], ui[m - 1]) <= tol) break;
    }
    for (int it = 0; it < 4; ++it) {
      const double tm = sqrt(t * t_bad);
      cheb_expm_e1(al, be, m, tm, ur, ui, w);
      const double em = beta * hypot(ur[m - 1], ui[m - 1]);
      if (em <= tol) t = tm;
      else t_bad = tm;
    }
    cheb_expm_e1(al, be, m, t, ur, ui, w);
    d.err = beta * hypot(ur[m - 1], ui[m - 1]);
    d.status = kDonePartial;
    d.tau_take = t;
  }
  return d;
}

}  // namespace rsv
