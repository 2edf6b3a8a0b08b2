// Adaptive Lanczos approximation of exp(-i tau Hbar) psibar (Sec. VI.B, Eqs. 36-38).
//
// All orbitals of the block run the recurrence together, each with its own
// tridiagonal T, stopping index and sub-steps:
//   q_0 = psi / ||psi||;  w = Hbar q_j;  alpha_j = Re(q_j^H w)
//   w -= alpha_j q_j + beta_{j-1} q_{j-1};  beta_j = ||w||;  q_{j+1} = w / beta_j
//   y = exp(-i tau T_{j+1}) e_1,  eps = tau beta_j ||psi|| |y_j|,  stop at eps <= tol
//   psi_out = ||psi|| sum_j y_j q_j
// Basis vectors are stored unnormalized (V_j) with q_j = s_j V_j, and s_j is
// folded into the next apply's gather.  alpha_j comes out of the element kernel
// as sum_e u_e^H H_e u_e (element partial sums); the three-term update and the
// partial sums of beta_j^2 are fused into the assembly of Hbar q_j.
//
// The small exponential exp(-i tau T) e_1 of the real symmetric tridiagonal T
// is evaluated on the device by the Chebyshev (Jacobi-Anger) expansion
//   exp(-i tau x) = e^{-i tau c} sum_n (2 - delta_n0) (-i)^n J_n(tau R) T_n((x - c)/R)
// on the Gershgorin interval [c - R, c + R] of T, with the Bessel values J_n
// from Miller's backward recurrence normalized by J_0 + 2 sum J_2k = 1.  It
// replaces the eigendecomposition of T (either is allowed by the paper, Eq. 37);
// its truncation error is below 1e-16.
//
// With a cap k_max the unconverged basis serves the largest sub-step
// tau_rem / 2^m whose estimate meets the tolerance, and the recurrence restarts.
#include <cmath>
#include <cstddef>

#include "elements.cuh"
#include "tdks_internal.h"

namespace {

using tdks::d2df_bits;
using tdks::Df;
using tdks::DfAcc;
using tdks::df_norm;
using tdks::dfa_madd;
using tdks::f2d_bits;
using tdks::from_d;

constexpr int kThreads = 256;
constexpr int kBlocks = 608;
constexpr int kBessMax = 3072;

__device__ __forceinline__ double block_reduce_sum(double v, double* red) {
  for (int off = 16; off > 0; off >>= 1) v += __shfl_down_sync(0xffffffffu, v, off);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
  __syncthreads();
  double s = 0.0;
  if (threadIdx.x == 0)
    for (int k = 0; k < (int)(blockDim.x >> 5); ++k) s += red[k];
  __syncthreads();
  return s;
}

__device__ __forceinline__ double sum_fixed(const double* part, int n, double* red) {
  double v = 0.0;
  for (int k = threadIdx.x; k < n; k += blockDim.x) v += part[k];
  for (int off = 16; off > 0; off >>= 1) v += __shfl_down_sync(0xffffffffu, v, off);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
  __syncthreads();
  double s = 0.0;
  for (int k = 0; k < (int)(blockDim.x >> 5); ++k) s += red[k];
  __syncthreads();
  return s;
}

__global__ void k_kry_init(KryOrb* kry, int n_orb, double tau) {
  const int o = blockIdx.x * blockDim.x + threadIdx.x;
  if (o >= n_orb) return;
  KryOrb& K = kry[o];
  K.t_rem = tau;
  K.tau_sub = 0.0;
  K.status = KRY_ACTIVE;
  K.k = 0;
  K.k_total = 0;
  K.nsub = 0;
  K.applies = 0;
  K.pad = 0;
  K.err = INFINITY;
  K.cv = 0;      // the small-exponential cache lives for one exponential
}

__global__ void k_norm_part(const double2* v, int64_t stride, long long n, const KryOrb* kry,
                            double* part, int64_t pstride) {
  __shared__ double red[kThreads / 32];
  const int o = blockIdx.y;
  double acc = 0.0;
  if (kry[o].status == KRY_ACTIVE) {
    const double2* p = v + (long long)o * stride;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x) {
      const double2 a = p[i];
      acc = fma(a.x, a.x, fma(a.y, a.y, acc));
    }
  }
  const double s = block_reduce_sum(acc, red);
  if (threadIdx.x == 0) part[(long long)o * pstride + blockIdx.x] = s;
}

__global__ void k_kry_start(KryOrb* kry, const double* part, int64_t pstride, int nb) {
  __shared__ double red[kThreads / 32];
  const int o = blockIdx.x;
  KryOrb& K = kry[o];
  if (K.status != KRY_ACTIVE) return;
  const double s = sum_fixed(part + (long long)o * pstride, nb, red);
  if (threadIdx.x == 0) {
    const double nrm = sqrt(s);
    K.nrm = nrm;
    K.k = 0;
    K.err = INFINITY;
    if (!isfinite(nrm)) {
      K.status = KRY_FAILED;
    } else if (nrm == 0.0) {
      K.status = KRY_CONVERGED;   // exp of the zero vector: recombination writes zeros
      K.tau_sub = K.t_rem;
    } else {
      K.s[0] = 1.0 / nrm;
    }
  }
}

// ---- small exponential on one warp -----------------------------------------
struct ChebWork {
  double J[kBessMax + 1];
  double a[TDKS_KMAX], b[TDKS_KMAX];
  double at[TDKS_KMAX], bt[TDKS_KMAX];   // 2 (a - c)/R and 2 b/R
  double v0[TDKS_KMAX], v1[TDKS_KMAX], v2[TDKS_KMAX];
  double yr[TDKS_KMAX], yi[TDKS_KMAX];
  double scal[4];
};

__device__ __forceinline__ double warp_min(double v) {
  for (int off = 16; off > 0; off >>= 1) v = fmin(v, __shfl_xor_sync(0xffffffffu, v, off));
  return v;
}
__device__ __forceinline__ double warp_max(double v) {
  for (int off = 16; off > 0; off >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, off));
  return v;
}

// y = exp(-i tau T) e_1 into W.yr/W.yi[0..m-1] (T from W.a, W.b); false if the
// expansion would need more than kBessMax terms.  Called by a full warp.  With a cache
// (the orbital's Lanczos state): an expansion on any interval holding the Gershgorin set
// of T is valid, so the cached interval and Bessel coefficients are reused while T's
// set lies inside it (same time); otherwise the set widened by 1/32 of its width on each
// side becomes the new cached interval.  The cache is emptied when an exponential starts,
// so results depend only on the exponential's own inputs.
__device__ bool cheb_exp(int m, double tau, ChebWork& W, KryOrb* C = nullptr) {
  const int lane = threadIdx.x & 31;
  if (m == 1) {
    if (lane == 0) {
      double sn, cs;
      sincos(tau * W.a[0], &sn, &cs);
      W.yr[0] = cs;
      W.yi[0] = -sn;
    }
    __syncwarp();
    return true;
  }
  double lo = INFINITY, hi = -INFINITY;
  for (int i = lane; i < m; i += 32) {
    const double r = (i > 0 ? fabs(W.b[i - 1]) : 0.0) + (i < m - 1 ? fabs(W.b[i]) : 0.0);
    lo = fmin(lo, W.a[i] - r);
    hi = fmax(hi, W.a[i] + r);
  }
  lo = warp_min(lo);
  hi = warp_max(hi);
  const bool reuse = C && C->cv && C->ctau == tau && lo >= C->clo && hi <= C->chi;
  if (reuse) {
    lo = C->clo;
    hi = C->chi;
  } else if (C) {
    const double wd = (hi - lo) * (1.0 / 32.0);
    lo -= wd;
    hi += wd;
  }
  const double c = 0.5 * (hi + lo);
  const double R = 0.5 * (hi - lo);
  double sn, cs;
  sincos(tau * c, &sn, &cs);
  const double z = tau * R;
  if (!(R > 1e-300) || !(z > 1e-280)) {
    for (int i = lane; i < m; i += 32) {
      W.yr[i] = (i == 0) ? cs : 0.0;
      W.yi[i] = (i == 0) ? -sn : 0.0;
    }
    __syncwarp();
    return true;
  }
  const int N = reuse ? C->cN : (int)ceil(z + 14.0 * cbrt(z) + 25.0);
  if (N > kBessMax) return false;
  if (reuse) {
    for (int k = lane; k <= N; k += 32) W.J[k] = C->cJ[k];
    __syncwarp();
  } else {
    if (lane == 0) {
      // Miller: b_{n-1} = (2n/z) b_n - b_{n+1} from n = M down to 1.  The factor is
      // n (2/z) with n carried as a double (exact), and the overflow test reads the
      // exponent bits, so the FP64 pipe sees two instructions per step.
      const int M = N + 20;
      const double two_inv_z = 2.0 * (1.0 / z);
      double bn1 = 0.0, bn = 1e-280, nd = (double)M, Stail = 0.0;
      for (int n = M; n >= 1; --n, nd -= 1.0) {
        const double bm = (nd * two_inv_z) * bn - bn1;
        const int idx = n - 1;
        if (idx <= N) W.J[idx] = bm;
        else if ((idx & 1) == 0) Stail += 2.0 * bm;   // even terms past N enter the sum only
        bn1 = bn;
        bn = bm;
        if ((((unsigned long long)__double_as_longlong(bn) >> 52) & 0x7ffull) > 1853ull) {   // |bn| > 2^830
          bn *= 1e-250;
          bn1 *= 1e-250;
          Stail *= 1e-250;
          for (int k = idx; k <= N && k <= M; ++k) W.J[k] *= 1e-250;
        }
      }
      W.scal[0] = Stail;
    }
    __syncwarp();
    // normalization J_0 + 2 sum_{k >= 1} J_2k = 1 (the sum in a fixed order), then J_n
    // for n >= 1 stored doubled: the expansion uses 2 J_n
    {
      double sp = 0.0;
      for (int k = 2 + 2 * lane; k <= N; k += 64) sp += W.J[k];
      for (int off = 16; off > 0; off >>= 1) sp += __shfl_down_sync(0xffffffffu, sp, off);
      const double S = W.J[0] + 2.0 * __shfl_sync(0xffffffffu, sp, 0) + W.scal[0];
      const double inv = 1.0 / S;
      __syncwarp();
      for (int k = lane; k <= N; k += 32) W.J[k] *= (k == 0 ? inv : 2.0 * inv);
    }
    if (C && N <= kChebCache) {
      __syncwarp();
      for (int k = lane; k <= N; k += 32) C->cJ[k] = W.J[k];
      if (lane == 0) {
        C->clo = lo;
        C->chi = hi;
        C->ctau = tau;
        C->cN = N;
        C->cv = 1;
      }
    }
  }
  const double invR = 1.0 / R;
  const double two_invR = 2.0 * invR;
  // scaled tridiagonal of X = (T - c)/R, doubled: the recurrence v_n = 2 X v_{n-1} - v_{n-2}
  for (int i = lane; i < m; i += 32) {
    W.at[i] = two_invR * (W.a[i] - c);
    W.bt[i] = (i < m - 1) ? two_invR * W.b[i] : 0.0;
  }
  // v0 = e_1, v1 = X e_1
  for (int i = lane; i < m; i += 32) {
    W.v0[i] = (i == 0) ? 1.0 : 0.0;
    double t = (i == 0) ? (W.a[0] - c) : 0.0;
    if (i == 1) t = W.b[0];
    W.v1[i] = t * invR;
  }
  __syncwarp();
  double accr[TDKS_KMAX / 32], acci[TDKS_KMAX / 32];
  for (int r = 0; r < TDKS_KMAX / 32; ++r) {
    const int i = lane + 32 * r;
    accr[r] = (i < m) ? W.J[0] * W.v0[i] : 0.0;
    acci[r] = (i < m) ? -W.J[1] * W.v1[i] : 0.0;
  }
  double* vp = W.v0;
  double* vc = W.v1;
  double* vn = W.v2;
  for (int n = 2; n <= N; ++n) {
    for (int r = 0; r < TDKS_KMAX / 32; ++r) {
      const int i = lane + 32 * r;
      if (i < m) {
        double t = fma(W.at[i], vc[i], -vp[i]);
        if (i > 0) t = fma(W.bt[i - 1], vc[i - 1], t);
        if (i < m - 1) t = fma(W.bt[i], vc[i + 1], t);
        vn[i] = t;
      }
    }
    __syncwarp();
    // (-i)^n 2 J_n T_n: real part for even n, imaginary for odd, signs by n mod 4
    const double cf = W.J[n];
    const int ph = n & 3;
    const double sg = (ph == 0 || ph == 3) ? cf : -cf;
    for (int r = 0; r < TDKS_KMAX / 32; ++r) {
      const int i = lane + 32 * r;
      if (i < m) {
        if (ph & 1) acci[r] = fma(sg, vn[i], acci[r]);
        else accr[r] = fma(sg, vn[i], accr[r]);
      }
    }
    double* t = vp;
    vp = vc;
    vc = vn;
    vn = t;
    __syncwarp();
  }
  for (int r = 0; r < TDKS_KMAX / 32; ++r) {
    const int i = lane + 32 * r;
    if (i < m) {
      // multiply by e^{-i tau c} = cs - i sn
      W.yr[i] = accr[r] * cs + acci[r] * sn;
      W.yi[i] = acci[r] * cs - accr[r] * sn;
    }
  }
  __syncwarp();
  return true;
}

// exp(-i tau T) e_1 for either sign of tau: for tau < 0 it is the complex
// conjugate of exp(-i |tau| T) e_1 (T and e_1 are real).
__device__ bool cheb_exp_signed(int m, double tau, ChebWork& W, KryOrb* C = nullptr) {
  const bool ok = cheb_exp(m, fabs(tau), W, C);
  if (ok && tau < 0.0) {
    for (int i = (threadIdx.x & 31); i < m; i += 32) W.yi[i] = -W.yi[i];
    __syncwarp();
  }
  return ok;
}

// One warp per orbital: beta_j, small exponential, a-posteriori estimate, decision.
// Decision after the apply of basis vector j (beta = ||w||): small exponential,
// a-posteriori estimate, and continue / converged / sub-step / failed.  Called
// by one full warp.
__device__ void kry_decide(KryOrb& K, int j, int kmax, double tol, double beta, ChebWork& W,
                           double theta = -1.0) {
  const int lane = threadIdx.x & 31;
  const int m = j + 1;
  for (int i = lane; i < m; i += 32) {
    W.a[i] = K.alpha[i];
    W.b[i] = (i < m - 1) ? K.beta[i] : 0.0;
  }
  __syncwarp();
  int decision = 0;   // 0 continue, 1 converged, 2 sub-step, -1 failed
  double tau_used = K.t_rem;
  double est = INFINITY;
  if (!isfinite(beta)) {
    decision = -1;
  } else {
    const bool ok = cheb_exp_signed(m, K.t_rem, W, &K);
    const double err = ok ? fabs(K.t_rem) * beta * K.nrm * hypot(W.yr[m - 1], W.yi[m - 1]) : INFINITY;
    est = err;
    if (ok && (err <= tol || beta == 0.0)) {
      decision = 1;
    } else if (m >= kmax) {
      decision = -1;
      for (int s = 1; s < 60; ++s) {
        const double ts = ldexp(K.t_rem, -s);
        const bool ok2 = cheb_exp_signed(m, ts, W);
        const double e2 = ok2 ? fabs(ts) * beta * K.nrm * hypot(W.yr[m - 1], W.yi[m - 1]) : INFINITY;
        if (ok2 && e2 <= tol) {
          decision = 2;
          tau_used = ts;
          break;
        }
      }
    }
  }
  for (int i = lane; i < m; i += 32) {
    K.yre[i] = W.yr[i];
    K.yim[i] = W.yi[i];
  }
  if (lane == 0) {
    K.applies += 1;
    K.beta[j] = beta;
    K.k = m;
    K.err = est;
    K.f32 = (decision == 0 && est <= theta) ? 1 : 0;   // batched relaxed schedule
    if (decision == 0) {
      K.s[j + 1] = 1.0 / beta;
    } else if (decision == 1) {
      K.status = KRY_CONVERGED;
      K.tau_sub = K.t_rem;
    } else if (decision == 2) {
      K.status = KRY_SUBSTEP;
      K.tau_sub = tau_used;
    } else {
      K.status = KRY_FAILED;
    }
  }
}

__global__ void k_kry_exp(int j, int kmax, double tol, KryOrb* kry, const double* npart,
                          int64_t npstride, int nb, const double* xpart, int nx) {
  __shared__ ChebWork W;
  const int o = blockIdx.x;
  const int lane = threadIdx.x;
  KryOrb& K = kry[o];
  if (K.status != KRY_ACTIVE) return;
  double v = 0.0;
  for (int k = lane; k < nb; k += 32) v += npart[(long long)o * npstride + k];
  for (int k = lane; k < nx; k += 32) v += xpart[(long long)o * nx + k];   // nonlocal correction
  for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
  kry_decide(K, j, kmax, tol, sqrt(v), W);
}

// out = ||psi|| sum_j y_j s_j V_j
__global__ void k_kry_recomb(long long n, double2* out, int64_t so, const double2* V0, int64_t s0,
                             const double2* Vw, int64_t sw, int kmax, const KryOrb* kry) {
  __shared__ double cr[TDKS_KMAX], ci[TDKS_KMAX];
  const int o = blockIdx.y;
  const KryOrb& K = kry[o];
  const int st = K.status;
  if (st != KRY_CONVERGED && st != KRY_SUBSTEP) return;
  const int m = K.k;
  for (int j = threadIdx.x; j < m; j += blockDim.x) {
    const double f = K.nrm * K.s[j];
    cr[j] = f * K.yre[j];
    ci[j] = f * K.yim[j];
  }
  __syncthreads();
  const double2* v0 = V0 + (long long)o * s0;
  const double2* vw = Vw + (long long)o * sw;
  double2* dst = out + (long long)o * so;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x) {
    double re = 0.0, im = 0.0;
#pragma unroll 4
    for (int j = 0; j < m; ++j) {
      const double2 v = (j == 0) ? v0[i] : vw[(long long)(j - 1) * n + i];
      re = fma(cr[j], v.x, fma(-ci[j], v.y, re));
      im = fma(cr[j], v.y, fma(ci[j], v.x, im));
    }
    dst[i] = make_double2(re, im);
  }
}

// Double-float recombination (double-float contraction runs): out_i = sum_j c_j V_j[i]
// with c_j = ||psi|| s_j y_j as double-float pairs and each FP64 vector entry split
// exactly into a pair on the integer pipe; the sums are carried as unnormalized
// (hi, err) pairs and rounded once to FP64.  ~2^-48 relative per term, like the
// double-float contractions, at a fraction of the FP64 pipe's work (4 FP64 FMAs
// per complex term otherwise).
struct RecombCoef {
  Df r, i, ni;   // c_j: real, imaginary, negated imaginary part
};
__device__ __forceinline__ RecombCoef recomb_coef(double f, double yr, double yi) {
  RecombCoef c;
  c.r = from_d<Df>(f * yr);
  c.i = from_d<Df>(f * yi);
  c.ni = Df{-c.i.hi, -c.i.lo};
  return c;
}
__device__ __forceinline__ double2 recomb_df_node(const RecombCoef* __restrict__ cf, int m,
                                                 const double2* __restrict__ v0,
                                                 const double2* __restrict__ vw, long long n,
                                                 long long i) {
  DfAcc ar{0.f, 0.f}, ai{0.f, 0.f};
#pragma unroll 2
  for (int j = 0; j < m; ++j) {
    const double2 v = (j == 0) ? v0[i] : vw[(long long)(j - 1) * n + i];
    const Df vx = d2df_bits(v.x), vy = d2df_bits(v.y);
    const RecombCoef c = cf[j];
    dfa_madd(ar, c.r, vx);
    dfa_madd(ar, c.ni, vy);
    dfa_madd(ai, c.r, vy);
    dfa_madd(ai, c.i, vx);
  }
  const Df r = df_norm(ar.hi, ar.err), s = df_norm(ai.hi, ai.err);
  return make_double2(f2d_bits(r.hi) + f2d_bits(r.lo), f2d_bits(s.hi) + f2d_bits(s.lo));
}

__global__ void k_kry_recomb_df(long long n, double2* out, int64_t so, const double2* V0, int64_t s0,
                                const double2* Vw, int64_t sw, const KryOrb* kry) {
  __shared__ RecombCoef cf[TDKS_KMAX];
  const int o = blockIdx.y;
  const KryOrb& K = kry[o];
  const int st = K.status;
  if (st != KRY_CONVERGED && st != KRY_SUBSTEP) return;
  const int m = K.k;
  for (int j = threadIdx.x; j < m; j += blockDim.x) cf[j] = recomb_coef(K.nrm * K.s[j], K.yre[j], K.yim[j]);
  __syncthreads();
  const double2* v0 = V0 + (long long)o * s0;
  const double2* vw = Vw + (long long)o * sw;
  double2* dst = out + (long long)o * so;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x)
    dst[i] = recomb_df_node(cf, m, v0, vw, n, i);
}

__global__ void k_kry_after(KryOrb* kry, int n_orb) {
  const int o = blockIdx.x * blockDim.x + threadIdx.x;
  if (o >= n_orb) return;
  KryOrb& K = kry[o];
  if (K.status == KRY_CONVERGED || K.status == KRY_SUBSTEP) {
    K.k_total += K.k;
    K.nsub += 1;
    if (K.k > K.pad) K.pad = K.k;       // largest dimension seen
    if (K.status == KRY_CONVERGED) {
      K.t_rem = 0.0;
      K.status = KRY_DONE;
    } else {
      K.t_rem -= K.tau_sub;
      K.status = (K.nsub >= TDKS_MAX_SUBSTEPS) ? KRY_FAILED : KRY_ACTIVE;
    }
  }
}

// ---- optional re-orthogonalization (classical Gram-Schmidt, two passes) --------
// After the three-term update has written w = V_{j+1}, w -= sum_i q_i (q_i^H w) over
// i = 0..j, twice; q_i = s_i V_i.  Partial dots per (chunk, i, orbital), summed in a
// fixed order; then ||w||^2 is recomputed for beta_j.
constexpr int kRoChunks = 128;

__global__ void k_ro_dot(long long n, const double2* V0, int64_t s0, const double2* VW, int64_t wsorb,
                         int j, const KryOrb* kry, double2* part) {
  __shared__ double red[2][kThreads / 32];
  const int o = blockIdx.z, i = blockIdx.y;
  const KryOrb& K = kry[o];
  if (K.status != KRY_ACTIVE) return;
  const double2* q = (i == 0) ? V0 + (long long)o * s0 : VW + (long long)o * wsorb + (long long)(i - 1) * n;
  const double2* w = VW + (long long)o * wsorb + (long long)j * n;
  const long long chunk = (n + gridDim.x - 1) / gridDim.x;
  const long long e1 = min(n, (blockIdx.x + 1) * chunk);
  double re = 0.0, im = 0.0;
  for (long long e = blockIdx.x * chunk + threadIdx.x; e < e1; e += blockDim.x) {
    const double2 a = q[e], x = w[e];
    re = fma(a.x, x.x, fma(a.y, x.y, re));
    im = fma(a.x, x.y, fma(-a.y, x.x, im));
  }
  for (int off = 16; off > 0; off >>= 1) {
    re += __shfl_down_sync(0xffffffffu, re, off);
    im += __shfl_down_sync(0xffffffffu, im, off);
  }
  if ((threadIdx.x & 31) == 0) {
    red[0][threadIdx.x >> 5] = re;
    red[1][threadIdx.x >> 5] = im;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double sr = 0.0, si = 0.0;
    for (int k = 0; k < kThreads / 32; ++k) {
      sr += red[0][k];
      si += red[1][k];
    }
    const double sc = K.s[i];
    part[((long long)o * TDKS_KMAX + i) * gridDim.x + blockIdx.x] = make_double2(sc * sr, sc * si);
  }
}

// h[o][i] = sum of the chunk partials (ascending), one warp per (i, orbital)
__global__ void k_ro_fin(const KryOrb* kry, const double2* part, int nch, double2* h) {
  const int o = blockIdx.y, i = blockIdx.x;
  if (kry[o].status != KRY_ACTIVE) return;
  if (threadIdx.x == 0) {
    double sr = 0.0, si = 0.0;
    const double2* p = part + ((long long)o * TDKS_KMAX + i) * nch;
    for (int k = 0; k < nch; ++k) {
      sr += p[k].x;
      si += p[k].y;
    }
    h[(long long)o * TDKS_KMAX + i] = make_double2(sr, si);
  }
}

// w -= sum_i h_i s_i V_i
__global__ void k_ro_update(long long n, const double2* V0, int64_t s0, double2* VW, int64_t wsorb, int j,
                            const KryOrb* kry, const double2* h) {
  __shared__ double hr[TDKS_KMAX], hi[TDKS_KMAX];
  const int o = blockIdx.y;
  const KryOrb& K = kry[o];
  if (K.status != KRY_ACTIVE) return;
  for (int i = threadIdx.x; i <= j; i += blockDim.x) {
    const double2 v = h[(long long)o * TDKS_KMAX + i];
    hr[i] = v.x * K.s[i];
    hi[i] = v.y * K.s[i];
  }
  __syncthreads();
  const double2* v0 = V0 + (long long)o * s0;
  const double2* vw = VW + (long long)o * wsorb;
  double2* w = VW + (long long)o * wsorb + (long long)j * n;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n;
       e += (long long)gridDim.x * blockDim.x) {
    double2 x = w[e];
    for (int i = 0; i <= j; ++i) {
      const double2 q = (i == 0) ? v0[e] : vw[(long long)(i - 1) * n + e];
      x.x -= hr[i] * q.x - hi[i] * q.y;
      x.y -= hr[i] * q.y + hi[i] * q.x;
    }
    w[e] = x;
  }
}

// ---- batched exponential: per-orbital state machine over many systems --------
// RESTART -> (norm) ACTIVE -> (apply, decide) ACTIVE | CONVERGED | SUBSTEP | FAILED;
// CONVERGED/SUBSTEP -> (recombine) DONE | RESTART.  One pass of the loop body
// advances every orbital by one step of this machine.
__device__ __forceinline__ const double2* bcur(const BSys& S, const KryOrb& K, int o) {
  return (K.nsub == 0 ? S.in : S.out) + (long long)o * S.n_int;
}

__global__ void k_bkry_init(const BSys* __restrict__ sys, const BOrb* __restrict__ orbs, int n,
                            double factor) {
  const int g = blockIdx.x * blockDim.x + threadIdx.x;
  if (g >= n) return;
  const BOrb b = orbs[g];
  const BSys& S = sys[b.sys];
  KryOrb& K = S.kry[b.o];
  K.t_rem = factor * S.dt;
  K.tau_sub = 0.0;
  K.status = KRY_RESTART;
  K.k = 0;
  K.k_total = 0;
  K.nsub = 0;
  K.applies = 0;
  K.pad = 0;
  K.err = INFINITY;
  K.f32 = 0;
  K.cv = 0;      // the small-exponential cache lives for one exponential
}

// partial ||v||^2 of the (re)starting orbitals, one block per chunk of n_int / n_rblk entries
__global__ void k_bnorm_part(const BSys* __restrict__ sys, const BRow* __restrict__ rows) {
  __shared__ double red[kThreads / 32];
  const BRow w = rows[blockIdx.x];
  const BSys& S = sys[w.sys];
  const KryOrb& K = S.kry[w.o];
  if (K.status != KRY_RESTART) return;
  const double2* v = bcur(S, K, w.o);
  const long long chunk = (S.n_int + S.n_rblk - 1) / S.n_rblk;
  const long long i1 = min(S.n_int, (w.rblk + 1) * chunk);
  double acc = 0.0;
  for (long long i = w.rblk * chunk + threadIdx.x; i < i1; i += blockDim.x) {
    const double2 a = v[i];
    acc = fma(a.x, a.x, fma(a.y, a.y, acc));
  }
  const double t = block_reduce_sum(acc, red);
  if (threadIdx.x == 0) S.npart[(long long)w.o * S.n_rblk + w.rblk] = t;
}

__global__ void k_bkry_start(const BSys* __restrict__ sys, const BOrb* __restrict__ orbs) {
  __shared__ double red[kThreads / 32];
  const BOrb b = orbs[blockIdx.x];
  const BSys& S = sys[b.sys];
  KryOrb& K = S.kry[b.o];
  if (K.status != KRY_RESTART) return;
  const double t = sum_fixed(S.npart + (long long)b.o * S.n_rblk, S.n_rblk, red);
  if (threadIdx.x == 0) {
    const double nrm = sqrt(t);
    K.nrm = nrm;
    K.k = 0;
    K.f32 = 0;                    // the first product of a (sub-)step: double-float
    if (!isfinite(nrm)) {
      K.status = KRY_FAILED;
    } else if (nrm == 0.0) {
      K.status = KRY_CONVERGED;   // exp of the zero vector: recombination writes zeros
      K.tau_sub = K.t_rem;
    } else {
      K.s[0] = 1.0 / nrm;
      K.status = KRY_ACTIVE;
    }
  }
}

// beta_j, small exponential and decision: one warp per orbital, j = K.k
__global__ void k_bkry_exp(const BSys* __restrict__ sys, const BOrb* __restrict__ orbs, double tol,
                           double theta) {
  __shared__ ChebWork W;
  const BOrb b = orbs[blockIdx.x];
  const BSys& S = sys[b.sys];
  KryOrb& K = S.kry[b.o];
  if (K.status != KRY_ACTIVE) return;
  const int lane = threadIdx.x;
  const double* np = S.npart + (long long)b.o * S.n_rblk;
  double v = 0.0;
  for (int k = lane; k < S.n_rblk; k += 32) v += np[k];
  for (int k = lane; k < S.kb_nblk; k += 32) v += S.kb_part[(long long)b.o * S.kb_nblk + k];   // nonlocal
  for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
  const int j = K.k;
  kry_decide(K, j, S.kmax, tol, sqrt(v), W, theta);
}

// out = ||psi|| sum_j y_j s_j V_j of converged / sub-stepped orbitals, one block per chunk
__global__ void k_brecomb(const BSys* __restrict__ sys, const BRow* __restrict__ rows) {
  __shared__ double cr[TDKS_KMAX], ci[TDKS_KMAX];
  const BRow w = rows[blockIdx.x];
  const BSys& S = sys[w.sys];
  const KryOrb& K = S.kry[w.o];
  const int st = K.status;
  if (st != KRY_CONVERGED && st != KRY_SUBSTEP) return;
  const int m = K.k;
  for (int j = threadIdx.x; j < m; j += blockDim.x) {
    const double f = K.nrm * K.s[j];
    cr[j] = f * K.yre[j];
    ci[j] = f * K.yim[j];
  }
  __syncthreads();
  const long long n = S.n_int;
  const double2* v0 = bcur(S, K, w.o);
  const double2* vw = S.Vw + (long long)w.o * S.kmax * n;
  double2* dst = S.out + (long long)w.o * n;
  const long long chunk = (n + S.n_rblk - 1) / S.n_rblk;
  const long long i1 = min(n, (w.rblk + 1) * chunk);
  for (long long i = w.rblk * chunk + threadIdx.x; i < i1; i += blockDim.x) {
    double re = 0.0, im = 0.0;
#pragma unroll 4
    for (int j = 0; j < m; ++j) {
      const double2 v = (j == 0) ? v0[i] : vw[(long long)(j - 1) * n + i];
      re = fma(cr[j], v.x, fma(-ci[j], v.y, re));
      im = fma(cr[j], v.y, fma(ci[j], v.x, im));
    }
    dst[i] = make_double2(re, im);
  }
}

__global__ void k_brecomb_df(const BSys* __restrict__ sys, const BRow* __restrict__ rows) {
  __shared__ RecombCoef cf[TDKS_KMAX];
  const BRow w = rows[blockIdx.x];
  const BSys& S = sys[w.sys];
  const KryOrb& K = S.kry[w.o];
  const int st = K.status;
  if (st != KRY_CONVERGED && st != KRY_SUBSTEP) return;
  const int m = K.k;
  for (int j = threadIdx.x; j < m; j += blockDim.x) cf[j] = recomb_coef(K.nrm * K.s[j], K.yre[j], K.yim[j]);
  __syncthreads();
  const long long n = S.n_int;
  const double2* v0 = bcur(S, K, w.o);
  const double2* vw = S.Vw + (long long)w.o * S.kmax * n;
  double2* dst = S.out + (long long)w.o * n;
  const long long chunk = (n + S.n_rblk - 1) / S.n_rblk;
  const long long i1 = min(n, (w.rblk + 1) * chunk);
  for (long long i = w.rblk * chunk + threadIdx.x; i < i1; i += blockDim.x)
    dst[i] = recomb_df_node(cf, m, v0, vw, n, i);
}

__global__ void k_bkry_after(const BSys* __restrict__ sys, const BOrb* __restrict__ orbs, int n) {
  const int g = blockIdx.x * blockDim.x + threadIdx.x;
  if (g >= n) return;
  const BOrb b = orbs[g];
  KryOrb& K = sys[b.sys].kry[b.o];
  if (K.status == KRY_CONVERGED || K.status == KRY_SUBSTEP) {
    K.k_total += K.k;
    K.nsub += 1;
    if (K.k > K.pad) K.pad = K.k;
    if (K.status == KRY_CONVERGED) {
      K.t_rem = 0.0;
      K.status = KRY_DONE;
    } else {
      K.t_rem -= K.tau_sub;
      K.status = (K.nsub >= TDKS_MAX_SUBSTEPS) ? KRY_FAILED : KRY_RESTART;
    }
  }
}

__global__ void k_bloop_begin(cudaGraphConditionalHandle h, int* iter, int* qctr, int n_q) {
  if (threadIdx.x < n_q) qctr[threadIdx.x] = 0;
  if (threadIdx.x == 0) {
    *iter = 0;
    cudaGraphSetConditional(h, 1u);
  }
}

// Loop condition: continue while some orbital is still in the recurrence, none
// failed and the pass count is below the cap (bit 1 of *err: failure, bit 2: cap).
__global__ void k_bloop_control(cudaGraphConditionalHandle h, const BSys* __restrict__ sys,
                                const BOrb* __restrict__ orbs, int n, int* iter, int cap, int* err,
                                int* qctr, int n_q) {
  __shared__ int s_act, s_fail;
  if (threadIdx.x < n_q) qctr[threadIdx.x] = 0;
  if (threadIdx.x == 0) {
    s_act = 0;
    s_fail = 0;
  }
  __syncthreads();
  int act = 0, fail = 0;
  for (int g = threadIdx.x; g < n; g += blockDim.x) {
    const BOrb b = orbs[g];
    const int st = sys[b.sys].kry[b.o].status;
    act |= (st == KRY_RESTART || st == KRY_ACTIVE);
    fail |= (st == KRY_FAILED);
  }
  if (act) atomicOr(&s_act, 1);
  if (fail) atomicOr(&s_fail, 1);
  __syncthreads();
  if (threadIdx.x == 0) {
    const int it = *iter + 1;
    *iter = it;
    if (s_fail) atomicOr(err, 1);
    if (s_act && !s_fail && it >= cap) atomicOr(err, 2);
    cudaGraphSetConditional(h, (s_act && !s_fail && it < cap) ? 1u : 0u);
  }
}

// orbital-vector applies x interior DoFs and the largest Krylov dimension of the
// exponential; per system its largest sub-step count and its applies
__global__ void k_bkry_stats(const BSys* __restrict__ sys, const BOrb* __restrict__ orbs, int n,
                             unsigned long long* dof_applies, int* kseen, unsigned long long* sys_sub) {
  const int g = blockIdx.x * blockDim.x + threadIdx.x;
  if (g >= n) return;
  const BOrb b = orbs[g];
  const BSys& S = sys[b.sys];
  const KryOrb& K = S.kry[b.o];
  atomicAdd(dof_applies, (unsigned long long)K.applies * (unsigned long long)S.n_int);
  atomicMax(kseen, K.pad);
  atomicMax(&sys_sub[2 * b.sys], (unsigned long long)K.nsub);
  atomicAdd(&sys_sub[2 * b.sys + 1], (unsigned long long)K.applies);
}

int grid_for(long long n) {
  long long b = (n + kThreads - 1) / kThreads;
  return (int)(b < kBlocks ? (b < 1 ? 1 : b) : kBlocks);
}

}  // namespace

tdks_status ensure_part(tdks_ctx* c, int n_orb, int64_t per_orb) {
  // the buffer is sized at context creation for the system's orbital count
  if (!c->d_part || per_orb > c->part_stride || n_orb > c->n_orb)
    return tdks_fail(c, TDKS_ERR_ARG, "partial-sum buffer too small for this call");
  return TDKS_OK;
}

static tdks_status ensure_krylov(tdks_ctx* c, int w, int n_orb, int kmax) {
  if (!c->d_kryw[w]) {
    if (cudaMalloc(&c->d_kryw[w], (size_t)c->n_orb * sizeof(KryOrb)) != cudaSuccess) {
      cudaGetLastError();
      return tdks_fail(c, TDKS_ERR_NOMEM, "Lanczos state");
    }
  }
  if (c->d_Vw[w] && c->Vw_orb[w] >= n_orb && c->Vw_kmax[w] == kmax) return TDKS_OK;
  if (c->d_Vw[w]) cudaFree(c->d_Vw[w]);
  c->d_Vw[w] = nullptr;
  const size_t bytes = (size_t)n_orb * kmax * c->n_int * sizeof(double2);
  if (cudaMalloc(&c->d_Vw[w], bytes) != cudaSuccess) {
    cudaGetLastError();
    return tdks_fail(c, TDKS_ERR_NOMEM, "Krylov basis (" + std::to_string(bytes >> 20) + " MiB)");
  }
  c->Vw_orb[w] = n_orb;
  c->Vw_kmax[w] = kmax;
  return TDKS_OK;
}

static tdks_status ensure_reorth(tdks_ctx* c) {
  if (c->d_ro_part) return TDKS_OK;
  if (cudaMalloc(&c->d_ro_part, (size_t)c->n_orb * TDKS_KMAX * kRoChunks * sizeof(double2)) != cudaSuccess ||
      cudaMalloc(&c->d_ro_h, (size_t)c->n_orb * TDKS_KMAX * sizeof(double2)) != cudaSuccess) {
    cudaGetLastError();
    return tdks_fail(c, TDKS_ERR_NOMEM, "re-orthogonalization buffers");
  }
  return TDKS_OK;
}

struct KrySummary {
  int k, status, k_total, nsub, applies, kseen;
  double err;
};
static_assert(offsetof(KryOrb, err) - offsetof(KryOrb, k) == offsetof(KrySummary, err),
              "KrySummary mirrors KryOrb from k to err");

static tdks_status read_summary(tdks_ctx* c, const KryOrb* kry, int n_orb, KrySummary* h) {
  TDKS_CU(c, cudaMemcpy2DAsync(h, sizeof(KrySummary), &kry[0].k, sizeof(KryOrb),
                               sizeof(KrySummary), n_orb, cudaMemcpyDeviceToHost, c->stream));
  TDKS_CU(c, cudaStreamSynchronize(c->stream));
  c->n_state_reads += 1;
  return TDKS_OK;
}

tdks_status run_expm(tdks_ctx* c, const double2* in, double2* out, int n_orb, double tau,
                     double tol, int kmax, int prec, int* k_used, int* kmax_seen,
                     int64_t* applies, int* nsub) {
  return run_expm_ws(c, 0, in, out, n_orb, tau, tol, kmax, prec, k_used, kmax_seen, applies, nsub);
}

// Lanczos exponential with workspace w (0 for propagation; 1 is a second basis
// kept alive alongside the first by the adjoint).  The basis V_0 = in (when no
// sub-step is needed), V_1.. in the workspace, and the per-orbital state stay
// valid until the next call on the same workspace.
__global__ void k_kry_ctl(const KryOrb* __restrict__ kry, int n_orb, double theta, int mixed,
                          cudaGraphConditionalHandle h64, cudaGraphConditionalHandle h32,
                          int* __restrict__ n32) {
  __shared__ double red[kThreads / 32];
  int any = 0;
  double emax = 0.0;
  for (int o = threadIdx.x; o < n_orb; o += blockDim.x) {
    if (kry[o].status == KRY_ACTIVE) {
      any = 1;
      const double e = kry[o].err;
      emax = (e > emax || e != e) ? e : emax;     // NaN propagates (no FP32 products then)
    }
  }
  any = __syncthreads_or(any);
  for (int off = 16; off > 0; off >>= 1) {
    const double t = __shfl_xor_sync(0xffffffffu, emax, off);
    emax = (t > emax || t != t) ? t : emax;
  }
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = emax;
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int k = 1; k < (int)(blockDim.x >> 5); ++k) emax = (red[k] > emax || red[k] != red[k]) ? red[k] : emax;
    emax = (red[0] > emax || red[0] != red[0]) ? red[0] : emax;
    if (!mixed) {
      cudaGraphSetConditional(h64, any ? 1u : 0u);
    } else {
      const bool f32 = any && emax <= theta;
      cudaGraphSetConditional(h32, f32 ? 1u : 0u);
      cudaGraphSetConditional(h64, (any && !f32) ? 1u : 0u);
      if (f32) *n32 += 1;
    }
  }
}

__global__ void k_stamp(unsigned long long* t) {
  unsigned long long v;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(v));
  *t = v;
}

// Kernels of Lanczos iteration j on workspace VW: the Hbar application of q_j with the
// fused three-term update (contraction arithmetic pj), the optional CGS2 passes, and the
// small exponential with the stopping decision.  Timing of the application: stamp
// (device loop) receives %globaltimer before and after it, ev (host loop) two events.
static tdks_status iteration_kernels(tdks_ctx* c, KryOrb* kry, const double2* cur, double2* VW,
                                     int64_t wsorb, long long n, int n_orb, int j, int kmax, int pj,
                                     double tol, int nb, int nasm, unsigned long long* stamp,
                                     cudaEvent_t* ev) {
  const int64_t ps = c->part_stride;
  double* apart = c->d_part;
  double* npart = c->d_part + (int64_t)c->n_orb * ps;
  const double2* Vj = (j == 0) ? cur : VW + (int64_t)(j - 1) * n;
  const int64_t sj = (j == 0) ? n : wsorb;
  const double2* Vm = (j == 1) ? cur : (j >= 2 ? VW + (int64_t)(j - 2) * n : nullptr);
  const int64_t sm = (j == 1) ? n : wsorb;
  double2* Vn = VW + (int64_t)j * n;
  // Hbar q_j and the three-term update fused: V_{j+1} = Hbar q_j - alpha_j q_j - beta q_{j-1}
  ApplyArgs a{Vj, sj, Vn, wsorb, n_orb, kry, j, apart, ps, 1, Vm, sm, npart, ps, 0};
  if (stamp) k_stamp<<<1, 1, 0, c->stream>>>(stamp + 2 * j);
  if (ev) TDKS_CU(c, cudaEventRecord(ev[0], c->stream));
  TDKS_TRY(launch_hbar_apply(c, a, pj));
  if (stamp) k_stamp<<<1, 1, 0, c->stream>>>(stamp + 2 * j + 1);
  if (ev) TDKS_CU(c, cudaEventRecord(ev[1], c->stream));
  if (c->lanczos_reorth) {
    TDKS_TRY(ensure_reorth(c));
    for (int pass = 0; pass < 2; ++pass) {
      k_ro_dot<<<dim3(kRoChunks, j + 1, n_orb), kThreads, 0, c->stream>>>(n, cur, n, VW, wsorb, j, kry,
                                                                          c->d_ro_part);
      k_ro_fin<<<dim3(j + 1, n_orb), 32, 0, c->stream>>>(kry, c->d_ro_part, kRoChunks, c->d_ro_h);
      k_ro_update<<<dim3(nb, n_orb), kThreads, 0, c->stream>>>(n, cur, n, VW, wsorb, j, kry, c->d_ro_h);
    }
    // ||w||^2 after the passes (the assembly's and the nonlocal partials are stale)
    k_norm_part<<<dim3(nb, n_orb), kThreads, 0, c->stream>>>(VW + (int64_t)j * n, wsorb, n, kry, npart, ps);
    k_kry_exp<<<n_orb, 32, 0, c->stream>>>(j, kmax, tol, kry, npart, ps, nb, nullptr, 0);
  } else {
    k_kry_exp<<<n_orb, 32, 0, c->stream>>>(j, kmax, tol, kry, npart, ps, nasm, kb_norm_parts(c),
                                           kb_norm_blocks(c));
  }
  TDKS_CU(c, cudaGetLastError());
  return TDKS_OK;
}

// ---- the Lanczos loop of one sub-step on the device -------------------------------
// The iterations j = 0 .. k_max-1 of a sub-step are captured once into a CUDA graph:
// iteration 0 unconditionally, every later iteration as a conditional IF node (two
// sibling nodes under TDKS_MIXED, one per contraction arithmetic).  After iteration j
// a one-block kernel sets the conditions of iteration j+1: some orbital still active
// and, under TDKS_MIXED, whether every active orbital's estimate is <= relax * tol.  An
// iteration whose condition stays 0 is skipped by the graph, so one launch runs the
// whole loop and the host reads the Lanczos state once per sub-step instead of once per
// iteration.  Each iteration keeps its own launch parameters (the kernels are those of
// the host-driven loop), so the results are identical.  Graphs are cached per
// starting vector and settings.
struct KGraph {
  const double2* cur = nullptr;
  const void* VW = nullptr;
  const void* evec = nullptr;
  const void* kb = nullptr;
  int n_orb = 0, kmax = 0, prec = 0, reorth = 0, opc = 0, timing = 0;
  unsigned f32_stages = 0;
  int len = 0;                             // iterations captured (<= kmax)
  double tol = 0.0, relax = 0.0;
  cudaGraph_t g = nullptr;
  cudaGraphExec_t exec = nullptr;
};

struct KGraphCache {
  std::vector<KGraph> graphs;
  cudaStream_t cap = nullptr, body = nullptr;
  unsigned long long* d_stamp = nullptr;   // [2 * TDKS_KMAX]
  int* d_n32 = nullptr;                    // FP32 iterations of the last launch
  unsigned long long* h_stamp = nullptr;   // pinned copies
  int* h_n32 = nullptr;
  bool broken = false;                     // a capture failed: host-driven loop from now on
  int len_hint = 16;                       // iterations to capture: the most needed so far + 8
};

static void kgraph_clear(KGraphCache* K) {
  for (auto& G : K->graphs) {
    if (G.exec) cudaGraphExecDestroy(G.exec);
    if (G.g) cudaGraphDestroy(G.g);
  }
  K->graphs.clear();
}

void kgraph_free(tdks_ctx* c) {
  KGraphCache* K = static_cast<KGraphCache*>(c->kgraph);
  if (!K) return;
  kgraph_clear(K);
  if (K->cap) cudaStreamDestroy(K->cap);
  if (K->body) cudaStreamDestroy(K->body);
  cudaFree(K->d_stamp);
  cudaFree(K->d_n32);
  cudaFreeHost(K->h_stamp);
  cudaFreeHost(K->h_n32);
  delete K;
  c->kgraph = nullptr;
}

static tdks_status kgraph_cache(tdks_ctx* c, KGraphCache** out) {
  if (!c->kgraph) {
    KGraphCache* K = new KGraphCache();
    c->kgraph = K;
    if (cudaStreamCreateWithFlags(&K->cap, cudaStreamNonBlocking) != cudaSuccess ||
        cudaStreamCreateWithFlags(&K->body, cudaStreamNonBlocking) != cudaSuccess ||
        cudaMalloc(&K->d_stamp, 2 * TDKS_KMAX * sizeof(unsigned long long)) != cudaSuccess ||
        cudaMalloc(&K->d_n32, sizeof(int)) != cudaSuccess ||
        cudaMallocHost(&K->h_stamp, 2 * TDKS_KMAX * sizeof(unsigned long long)) != cudaSuccess ||
        cudaMallocHost(&K->h_n32, sizeof(int)) != cudaSuccess) {
      cudaGetLastError();
      kgraph_free(c);
      return tdks_fail(c, TDKS_ERR_NOMEM, "device Lanczos loop buffers");
    }
  }
  *out = static_cast<KGraphCache*>(c->kgraph);
  return TDKS_OK;
}

// Inside an active capture of stream `cap`: append IF nodes (one per handle) that all
// depend on the current capture dependencies; returns their body graphs.  The capture
// then continues after all of them.
static tdks_status add_if_nodes(tdks_ctx* c, cudaStream_t cap, const cudaGraphConditionalHandle* h,
                                int nh, cudaGraph_t* bodies) {
  cudaStreamCaptureStatus cs;
  cudaGraph_t g = nullptr;
  const cudaGraphNode_t* deps = nullptr;
  size_t nd = 0;
  TDKS_CU(c, cudaStreamGetCaptureInfo(cap, &cs, nullptr, &g, &deps, nullptr, &nd));
  if (cs != cudaStreamCaptureStatusActive) return tdks_fail(c, TDKS_ERR_CUDA, "stream is not capturing");
  std::vector<cudaGraphNode_t> dv(deps, deps + nd);
  cudaGraphNode_t nodes[2];
  for (int i = 0; i < nh; ++i) {
    cudaGraphNodeParams p = {cudaGraphNodeTypeConditional};
    p.conditional.handle = h[i];
    p.conditional.type = cudaGraphCondTypeIf;
    p.conditional.size = 1;
    TDKS_CU(c, cudaGraphAddNode(&nodes[i], g, dv.data(), nullptr, dv.size(), &p));
    bodies[i] = p.conditional.phGraph_out[0];
  }
  TDKS_CU(c, cudaStreamUpdateCaptureDependencies(cap, nodes, nullptr, nh, cudaStreamSetCaptureDependencies));
  return TDKS_OK;
}

// Capture of iterations 0 .. kmax-1 of a sub-step starting from `cur`.
static tdks_status capture_loop(tdks_ctx* c, KGraphCache* K, KGraph& G, KryOrb* kry, double2* VW,
                                int64_t wsorb, long long n, int nb, int nasm) {
  const int kmax = G.kmax, n_orb = G.n_orb, L = G.len;
  const bool mixed = G.prec == TDKS_MIXED;
  const int p64 = mixed ? TDKS_DF64 : G.prec;
  const double theta = G.relax * G.tol;
  unsigned long long* stamp = G.timing ? K->d_stamp : nullptr;
  std::vector<cudaGraphConditionalHandle> h64(kmax + 1), h32(kmax + 1);
  TDKS_CU(c, cudaGraphCreate(&G.g, 0));
  for (int j = 1; j < L; ++j) {
    TDKS_CU(c, cudaGraphConditionalHandleCreate(&h64[j], G.g, 0, cudaGraphCondAssignDefault));
    if (mixed) TDKS_CU(c, cudaGraphConditionalHandleCreate(&h32[j], G.g, 0, cudaGraphCondAssignDefault));
  }
  cudaStream_t saved = c->stream;
  const int64_t save_launch = c->n_launch, save_apply = c->n_apply_launch;
  TDKS_CU(c, cudaStreamBeginCaptureToGraph(K->cap, G.g, nullptr, nullptr, 0, cudaStreamCaptureModeRelaxed));
  c->stream = K->cap;
  tdks_status st = TDKS_OK;
  auto ctl = [&](int jn) {
    k_kry_ctl<<<1, kThreads, 0, c->stream>>>(kry, n_orb, theta, mixed ? 1 : 0, h64[jn], h32[jn], K->d_n32);
  };
  st = iteration_kernels(c, kry, G.cur, VW, wsorb, n, n_orb, 0, kmax, p64, G.tol, nb, nasm, stamp, nullptr);
  if (st == TDKS_OK && L > 1) ctl(1);
  for (int j = 1; j < L && st == TDKS_OK; ++j) {
    const int nv = mixed ? 2 : 1;
    const cudaGraphConditionalHandle hh[2] = {h64[j], h32[j]};
    cudaGraph_t bodies[2] = {nullptr, nullptr};
    st = add_if_nodes(c, K->cap, hh, nv, bodies);
    for (int v = 0; v < nv && st == TDKS_OK; ++v) {
      if (cudaStreamBeginCaptureToGraph(K->body, bodies[v], nullptr, nullptr, 0,
                                        cudaStreamCaptureModeRelaxed) != cudaSuccess) {
        st = tdks_fail(c, TDKS_ERR_CUDA, "loop body capture");
        break;
      }
      c->stream = K->body;
      st = iteration_kernels(c, kry, G.cur, VW, wsorb, n, n_orb, j, kmax, v == 1 ? TDKS_FP32 : p64, G.tol,
                             nb, nasm, stamp, nullptr);
      if (st == TDKS_OK && j + 1 < L) ctl(j + 1);
      cudaGraph_t outb = nullptr;
      const cudaError_t e = cudaStreamEndCapture(K->body, &outb);
      c->stream = K->cap;
      if (st == TDKS_OK && e != cudaSuccess) st = tdks_fail(c, TDKS_ERR_CUDA, std::string("loop body capture: ") + cudaGetErrorString(e));
    }
  }
  cudaGraph_t outg = nullptr;
  const cudaError_t e = cudaStreamEndCapture(K->cap, &outg);
  c->stream = saved;
  c->n_launch = save_launch;
  c->n_apply_launch = save_apply;
  if (st != TDKS_OK) return st;
  if (e != cudaSuccess) return tdks_fail(c, TDKS_ERR_CUDA, std::string("loop capture: ") + cudaGetErrorString(e));
  TDKS_CU(c, cudaGraphInstantiate(&G.exec, G.g, 0));
  return TDKS_OK;
}

static tdks_status get_loop_graph(tdks_ctx* c, KGraphCache* K, const double2* cur, KryOrb* kry, double2* VW,
                                  int64_t wsorb, long long n, int n_orb, int kmax, int len, int prec,
                                  double tol, int nb, int nasm, KGraph** out) {
  for (auto& G : K->graphs) {
    if (G.cur == cur && G.VW == VW && G.evec == c->d_evec && G.kb == c->kb && G.n_orb == n_orb &&
        G.kmax == kmax && G.len == len && G.prec == prec && G.reorth == c->lanczos_reorth && G.opc == c->opc_force &&
        G.timing == (c->timing ? 1 : 0) && G.tol == tol && G.relax == c->mixed_relax &&
        G.f32_stages == c->f32_stages) {
      *out = &G;
      return TDKS_OK;
    }
  }
  if (K->graphs.size() >= 8) kgraph_clear(K);
  TDKS_TRY(ensure_evec(c, n_orb));     // the capture must not reallocate the element results
  K->graphs.emplace_back();
  KGraph& G = K->graphs.back();
  G.cur = cur;
  G.VW = VW;
  G.evec = c->d_evec;
  G.kb = c->kb;
  G.n_orb = n_orb;
  G.kmax = kmax;
  G.len = len;
  G.prec = prec;
  G.reorth = c->lanczos_reorth;
  G.opc = c->opc_force;
  G.timing = c->timing ? 1 : 0;
  G.tol = tol;
  G.relax = c->mixed_relax;
  G.f32_stages = c->f32_stages;
  const tdks_status st = capture_loop(c, K, G, kry, VW, wsorb, n, nb, nasm);
  if (st != TDKS_OK) {
    if (G.exec) cudaGraphExecDestroy(G.exec);
    if (G.g) cudaGraphDestroy(G.g);
    K->graphs.pop_back();
    return st;
  }
  *out = &K->graphs.back();
  return TDKS_OK;
}

tdks_status run_expm_ws(tdks_ctx* c, int w, const double2* in, double2* out, int n_orb, double tau,
                        double tol, int kmax, int prec, int* k_used, int* kmax_seen,
                        int64_t* applies, int* nsub) {
  if (kmax < 1 || kmax > TDKS_KMAX) return tdks_fail(c, TDKS_ERR_ARG, "k_max must be in [1, 128]");
  if (n_orb < 1 || n_orb > c->n_orb) return tdks_fail(c, TDKS_ERR_ARG, "n_orb out of range");
  const long long n = c->n_int;
  const int bpc = hbar_blocks_per_color(c);
  TDKS_TRY(ensure_part(c, n_orb, 8 * (int64_t)bpc));
  TDKS_TRY(ensure_krylov(c, w, n_orb, kmax));
  if (c->lanczos_reorth) TDKS_TRY(ensure_reorth(c));
  KryOrb* kry = c->d_kryw[w];
  double2* VW = c->d_Vw[w];
  const int64_t ps = c->part_stride;
  double* npart = c->d_part + (int64_t)c->n_orb * ps;
  const int nb = grid_for(n);
  const int nasm = assemble_blocks(c, n_orb);   // partials of ||w||^2 per orbital
  const int64_t wsorb = (int64_t)kmax * n;   // stride between orbitals in the workspace
  std::vector<KrySummary> h(n_orb);
  // the device-driven loop, unless disabled or the stream is being captured by the caller
  bool device_loop = c->device_loop != 0;
  KGraphCache* K = nullptr;
  if (device_loop) {
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(c->stream, &cs) != cudaSuccess || cs != cudaStreamCaptureStatusNone) device_loop = false;
  }
  if (device_loop) {
    TDKS_TRY(kgraph_cache(c, &K));
    if (K->broken) device_loop = false;
  }
  k_kry_init<<<(n_orb + 63) / 64, 64, 0, c->stream>>>(kry, n_orb, tau);
  c->n_launch += 1;
  TDKS_CU(c, cudaGetLastError());
  if (c->timing && !c->ev[0]) {
    TDKS_CU(c, cudaEventCreate(&c->ev[0]));
    TDKS_CU(c, cudaEventCreate(&c->ev[1]));
  }
  int n_active = n_orb;
  const double2* cur = in;
  for (int sub = 0; sub <= TDKS_MAX_SUBSTEPS; ++sub) {
    k_norm_part<<<dim3(nb, n_orb), kThreads, 0, c->stream>>>(cur, n, n, kry, npart, ps);
    k_kry_start<<<n_orb, kThreads, 0, c->stream>>>(kry, npart, ps, nb);
    c->n_launch += 2;
    TDKS_CU(c, cudaGetLastError());
    int j0 = 0;                // first iteration left to the host
    KGraph* G = nullptr;
    const int len = device_loop ? (K->len_hint < kmax ? K->len_hint : kmax) : 0;
    if (device_loop) {
      if (get_loop_graph(c, K, cur, kry, VW, wsorb, n, n_orb, kmax, len, prec, tol, nb, nasm, &G) != TDKS_OK) {
        // capture is not available here: the host-driven loop from now on
        cudaGetLastError();
        K->broken = true;
        device_loop = false;
        c->err.clear();
      }
    }
    if (G) {
      std::vector<int> app0(n_orb);
      for (int o = 0; o < n_orb; ++o) app0[o] = h[o].applies;
      TDKS_CU(c, cudaMemsetAsync(K->d_n32, 0, sizeof(int), c->stream));
      TDKS_CU(c, cudaGraphLaunch(G->exec, c->stream));
      TDKS_CU(c, cudaMemcpyAsync(K->h_n32, K->d_n32, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
      if (c->timing)
        TDKS_CU(c, cudaMemcpyAsync(K->h_stamp, K->d_stamp, 2 * kmax * sizeof(unsigned long long),
                                   cudaMemcpyDeviceToHost, c->stream));
      TDKS_TRY(read_summary(c, kry, n_orb, h.data()));
      // work of the loop: applications per orbital, iterations run, FP32 iterations
      int iters = 0;
      for (int o = 0; o < n_orb; ++o) {
        const int d = h[o].applies - app0[o];
        c->n_apply_units += (int64_t)d * c->n_elem;
        iters = d > iters ? d : iters;
      }
      c->n_apply_launch += iters;
      if (iters + 8 > K->len_hint) K->len_hint = ((iters + 8 + 7) / 8) * 8;
      c->n_apply_fp32 += *K->h_n32;
      c->n_launch += (int64_t)iters * (c->lanczos_reorth ? 11 : 4) + (iters > 0 ? iters - 1 : 0);
      if (c->timing)
        for (int j = 0; j < iters; ++j) c->apply_ms += 1e-6 * (double)(K->h_stamp[2 * j + 1] - K->h_stamp[2 * j]);
      n_active = 0;
      for (int o = 0; o < n_orb; ++o) n_active += (h[o].status == KRY_ACTIVE);
      j0 = n_active ? len : kmax;
    }
    {
      // the host-driven loop: every iteration when the device loop is off, or the
      // iterations beyond the captured length (the next capture is longer)
      if (j0 > 0 && j0 < kmax) {
        const int need = j0 + 16;
        K->len_hint = ((need + 7) / 8) * 8;
      }
      for (int j = j0; j < kmax; ++j) {
        // TDKS_MIXED: the error a matrix-vector product of iteration j contributes to
        // the exponential scales with the weight |y_j| of q_j, which the a-posteriori
        // estimate of the previous iteration bounds (eps = tau beta ||psi|| |y|); once
        // every active orbital's estimate is below relax * tol, the FP32 rounding of
        // the remaining products is far below the tolerance (relaxed inexact Krylov
        // products), so they run with FP32 contractions.  Double-float before that.
        int pj = prec == TDKS_MIXED ? TDKS_DF64 : prec;
        if (prec == TDKS_MIXED && j > 0) {
          double emax = 0.0;
          for (int o = 0; o < n_orb; ++o)
            if (h[o].status == KRY_ACTIVE) emax = (h[o].err > emax || h[o].err != h[o].err) ? h[o].err : emax;
          if (emax <= c->mixed_relax * tol) pj = TDKS_FP32;
        }
        if (pj == TDKS_FP32 && prec == TDKS_MIXED) c->n_apply_fp32 += 1;
        TDKS_TRY(iteration_kernels(c, kry, cur, VW, wsorb, n, n_orb, j, kmax, pj, tol, nb, nasm, nullptr,
                                   c->timing ? c->ev : nullptr));
        c->n_apply_units += (int64_t)n_active * c->n_elem;
        c->n_launch += c->lanczos_reorth ? 8 : 1;
        TDKS_TRY(read_summary(c, kry, n_orb, h.data()));
        if (c->timing) {
          float ms = 0.f;
          TDKS_CU(c, cudaEventElapsedTime(&ms, c->ev[0], c->ev[1]));
          c->apply_ms += ms;
        }
        n_active = 0;
        for (int o = 0; o < n_orb; ++o) n_active += (h[o].status == KRY_ACTIVE);
        if (!n_active) break;
      }
    }
    if (prec == TDKS_DF64 || prec == TDKS_MIXED)
      k_kry_recomb_df<<<dim3(nb, n_orb), kThreads, 0, c->stream>>>(n, out, n, cur, n, VW, wsorb, kry);
    else
      k_kry_recomb<<<dim3(nb, n_orb), kThreads, 0, c->stream>>>(n, out, n, cur, n, VW, wsorb,
                                                               kmax, kry);
    k_kry_after<<<(n_orb + 63) / 64, 64, 0, c->stream>>>(kry, n_orb);
    c->n_launch += 2;
    TDKS_CU(c, cudaGetLastError());
    TDKS_TRY(read_summary(c, kry, n_orb, h.data()));
    bool any = false, failed = false;
    for (int o = 0; o < n_orb; ++o) {
      any |= (h[o].status == KRY_ACTIVE);
      failed |= (h[o].status == KRY_FAILED);
    }
    if (failed)
      return tdks_fail(c, TDKS_ERR_NOT_CONVERGED,
                       "Lanczos: no admissible sub-step, sub-step cap or non-finite norm");
    if (!any) break;
    n_active = 0;
    for (int o = 0; o < n_orb; ++o) n_active += (h[o].status == KRY_ACTIVE);
    cur = out;
  }
  int64_t napp = 0;
  int kseen = 0, ns = 0;
  for (int o = 0; o < n_orb; ++o) {
    if (k_used) k_used[o] = h[o].k_total;
    napp += h[o].applies;
    kseen = h[o].kseen > kseen ? h[o].kseen : kseen;
    ns += h[o].nsub - 1;
  }
  if (kmax_seen) *kmax_seen = kseen;
  if (applies) *applies = napp;
  if (nsub) *nsub = ns;
  return TDKS_OK;
}

// ---- batched exponential launchers ------------------------------------------
cudaError_t launch_bkry_init(const BSys* sys, const BOrb* orbs, int n, double factor, cudaStream_t st) {
  k_bkry_init<<<(n + 63) / 64, 64, 0, st>>>(sys, orbs, n, factor);
  return cudaGetLastError();
}

cudaError_t launch_bkry_prepare(const BSys* sys, const BOrb* orbs, int n, const BRow* rows, int n_rows,
                                cudaStream_t st) {
  k_bnorm_part<<<n_rows, kThreads, 0, st>>>(sys, rows);
  k_bkry_start<<<n, kThreads, 0, st>>>(sys, orbs);
  return cudaGetLastError();
}

cudaError_t launch_bkry_exp(const BSys* sys, const BOrb* orbs, int n, double tol, double theta,
                            cudaStream_t st) {
  k_bkry_exp<<<n, 32, 0, st>>>(sys, orbs, tol, theta);
  return cudaGetLastError();
}

cudaError_t launch_bkry_finish(const BSys* sys, const BOrb* orbs, int n, const BRow* rows, int n_rows,
                               int prec, cudaStream_t st) {
  if (prec == TDKS_DF64 || prec == TDKS_MIXED) k_brecomb_df<<<n_rows, kThreads, 0, st>>>(sys, rows);
  else k_brecomb<<<n_rows, kThreads, 0, st>>>(sys, rows);
  k_bkry_after<<<(n + 63) / 64, 64, 0, st>>>(sys, orbs, n);
  return cudaGetLastError();
}

cudaError_t launch_bloop_begin(cudaGraphConditionalHandle h, int* iter, int* qctr, int n_q,
                               cudaStream_t st) {
  if (n_q > 32) return cudaErrorInvalidValue;
  k_bloop_begin<<<1, 32, 0, st>>>(h, iter, qctr, n_q);
  return cudaGetLastError();
}

cudaError_t launch_bloop_control(cudaGraphConditionalHandle h, const BSys* sys, const BOrb* orbs, int n,
                                 int* iter, int cap, int* err, int* qctr, int n_q, cudaStream_t st) {
  if (n_q > kThreads) return cudaErrorInvalidValue;
  k_bloop_control<<<1, kThreads, 0, st>>>(h, sys, orbs, n, iter, cap, err, qctr, n_q);
  return cudaGetLastError();
}

cudaError_t launch_bkry_stats(const BSys* sys, const BOrb* orbs, int n, unsigned long long* dof_applies,
                              int* kseen, unsigned long long* sys_sub, cudaStream_t st) {
  k_bkry_stats<<<(n + 63) / 64, 64, 0, st>>>(sys, orbs, n, dof_applies, kseen, sys_sub);
  return cudaGetLastError();
}
