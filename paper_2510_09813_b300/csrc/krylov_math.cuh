// FP64 small-matrix part of the Lanczos step (arXiv 2510.09813, Sec. III.A):
// exp(-i tau T_m) e_1 for the real symmetric tridiagonal T_m, and the
// acceptance test of a Krylov space with its substep choice. Used by the
// streaming path's scalar kernel and by the batched kernel.
#pragma once

#include "dword.cuh"
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
  double J[kMaxBessel];                   // J_k(x), FP64
  float jh[kMaxBessel], jl[kMaxBessel];   // (2 - delta_k0) J_k(x) as double words
  int kmax;
  // The expansion (interval, pieces, Bessel factors, phase) is kept for reuse:
  // it holds for every T_m whose Gershgorin interval lies in [c_lo, c_hi], at
  // time c_tau. Successive Krylov dimensions of one step usually fit in the
  // interval of the first, widened by a tenth, so Miller's recurrence (FP64,
  // serial) runs about once per step rather than once per check.
  int c_valid, c_pieces;
  double c_lo, c_hi, c_tau, c_pc, c_ps;
};

// Forget the kept expansion (lane 0, before the first use of w).
__device__ __forceinline__ void cheb_reset(ChebWork& w) { w.c_valid = 0; }

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
  for (int i = lane; i < m; i += 32) {
    ur[i] = (i == 0) ? 1.0 : 0.0;
    ui[i] = 0.0;
  }
  __syncwarp();
  if (!(hi - lo > 2e-300) || m == 1) {
    if (lane == 0) {
      double s, c;
      sincos(tau * 0.5 * (lo + hi), &s, &c);
      ur[0] = c;
      ui[0] = -s;
    }
    __syncwarp();
    return;
  }
  const bool hit = w.c_valid && w.c_tau == tau && w.c_lo <= lo && hi <= w.c_hi;
  if (!hit) {
    const double span = hi - lo;
    const double lo2 = lo - 0.05 * span, hi2 = hi + 0.05 * span;
    const double cen = 0.5 * (lo2 + hi2), rad = 0.5 * (hi2 - lo2);
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
    const double tp = tau / pieces, x = tp * rad;
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
    for (int k = lane; k <= w.kmax; k += 32) {
      const DW c = dw_from(k == 0 ? w.J[0] : 2.0 * w.J[k]);
      w.jh[k] = c.hi;
      w.jl[k] = c.lo;
    }
    if (lane == 0) {
      double ps, pc;
      sincos(tp * cen, &ps, &pc);
      w.c_pc = pc;
      w.c_ps = ps;
      w.c_lo = lo2;
      w.c_hi = hi2;
      w.c_tau = tau;
      w.c_pieces = pieces;
      w.c_valid = 1;
    }
    __syncwarp();
  }
  const double cen = 0.5 * (w.c_lo + w.c_hi), irad = 1.0 / (0.5 * (w.c_hi - w.c_lo));
  const int kmax = w.kmax, pieces = w.c_pieces;
  const double pc = w.c_pc, ps = w.c_ps;
  if (m <= 32) {
    // Register path in double words, one component per lane: the three-term
    // recurrence phi_{k+1} = 2 S phi_k - phi_{k-1} with 2 S's entries folded
    // into three per-lane coefficients and the neighbours phi_k[i -+ 1] by
    // shuffles. A term costs about 130 FP32 instructions, against 8 FP64 ones
    // at some 70 cycles each.
    const int i = lane;
    const bool act = i < m;
    const DW a2 = dw_from(act ? 2.0 * (al[i] - cen) * irad : 0.0);
    const DW bl = dw_from((act && i > 0) ? 2.0 * be[i] * irad : 0.0);
    const DW br = dw_from((act && i + 1 < m) ? 2.0 * be[i + 1] * irad : 0.0);
    const DW pcw = dw_from(pc), psw = dw_from(ps), zero{0.f, 0.f};
    DW uR{i == 0 ? 1.f : 0.f, 0.f}, uI = zero;
    for (int piece = 0; piece < pieces; ++piece) {
      DW pR = uR, pI = uI;  // phi_0
      const DW j0{w.jh[0], w.jl[0]};
      DW aR = dw_axpy(zero, j0, pR), aI = dw_axpy(zero, j0, pI);
      // phi_1 = S phi_0 = (2 S phi_0) / 2
      DW cR = dw_stencil(a2, pR, bl, dw_shfl_up(pR, 1), br, dw_shfl_down(pR, 1), zero);
      DW cI = dw_stencil(a2, pI, bl, dw_shfl_up(pI, 1), br, dw_shfl_down(pI, 1), zero);
      cR = DW{0.5f * cR.hi, 0.5f * cR.lo};
      cI = DW{0.5f * cI.hi, 0.5f * cI.lo};
      {
        const DW c1{w.jh[1], w.jl[1]};  // (-i)^1
        aR = dw_axpy(aR, c1, cI);
        aI = dw_axpy(aI, dw_neg(c1), cR);
      }
      for (int k = 2; k <= kmax; ++k) {
        const DW nR = dw_stencil(a2, cR, bl, dw_shfl_up(cR, 1), br, dw_shfl_down(cR, 1), pR);
        const DW nI = dw_stencil(a2, cI, bl, dw_shfl_up(cI, 1), br, dw_shfl_down(cI, 1), pI);
        pR = cR;
        pI = cI;
        cR = nR;
        cI = nI;
        const DW ck{w.jh[k], w.jl[k]};
        switch (k & 3) {  // (-i)^k
          case 0: aR = dw_axpy(aR, ck, nR); aI = dw_axpy(aI, ck, nI); break;
          case 1: aR = dw_axpy(aR, ck, nI); aI = dw_axpy(aI, dw_neg(ck), nR); break;
          case 2: aR = dw_axpy(aR, dw_neg(ck), nR); aI = dw_axpy(aI, dw_neg(ck), nI); break;
          default: aR = dw_axpy(aR, dw_neg(ck), nI); aI = dw_axpy(aI, ck, nR); break;
        }
      }
      // u = exp(-i tp cen) * acc
      uR = dw_stencil(pcw, aR, psw, aI, zero, zero, zero);
      uI = dw_stencil(pcw, aI, dw_neg(psw), aR, zero, zero, zero);
    }
    if (act) {
      ur[i] = dw_value(uR);
      ui[i] = dw_value(uI);
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
    // The largest t < tau_rem whose estimate meets tol. The estimate falls
    // like a power of t (t^m for small t), so each guess is a secant step on
    // log err against log t towards 0.85 tol, from the failing end of the
    // bracket [t_lo meets tol, t_hi does not] with the bracket's slope; a
    // guess outside the bracket is replaced by its geometric middle. The search
    // stops once an accepted t has an estimate of at least 0.6 tol or the
    // bracket is within 3%: two or three evaluations where halving and four
    // bisections took six or seven. Guesses are FP32 (only t_lo's FP64
    // evaluation decides).
    double t_hi = tau_rem, e_hi = d.err, t_lo = 0.0, e_lo = 0.0;
    float slope = (float)m;
    bool ur_at_lo = false;
    for (int it = 0; it < 24; ++it) {
      double t = t_hi * (double)exp2f(log2f(0.85f * (float)(tol / e_hi)) / slope);
      if (!(t > t_lo && t < t_hi)) t = t_lo > 0.0 ? sqrt(t_lo * t_hi) : 0.25 * t_hi;
      cheb_expm_e1(al, be, m, t, ur, ui, w);
      const double e = beta * hypot(ur[m - 1], ui[m - 1]);
      ur_at_lo = e <= tol;
      if (ur_at_lo) {
        t_lo = t;
        e_lo = e;
        if (e >= 0.6 * tol || t_hi <= 1.03 * t_lo) break;
      } else {
        t_hi = t;
        e_hi = e;
      }
      if (t_lo > 0.0 && e_lo > 0.0 && e_hi > e_lo) slope = log2f((float)(e_hi / e_lo)) / log2f((float)(t_hi / t_lo));
      if (!(slope >= 0.5f)) slope = 0.5f;
    }
    if (!(t_lo > 0.0)) {
      // not found in the budget (an estimate that does not fall with t):
      // halve until it meets tol, as a last resort
      t_lo = t_hi;
      for (int it = 0; it < 64; ++it) {
        t_lo *= 0.5;
        cheb_expm_e1(al, be, m, t_lo, ur, ui, w);
        if (beta * hypot(ur[m - 1], ui[m - 1]) <= tol) break;
      }
      ur_at_lo = true;
    }
    if (!ur_at_lo) cheb_expm_e1(al, be, m, t_lo, ur, ui, w);
    d.err = beta * hypot(ur[m - 1], ui[m - 1]);
    d.status = kDonePartial;
    d.tau_take = t_lo;
  }
  return d;
}

}  // namespace rsv
