// Potentials of the three models of Sec. 3 (plus a free massive field), on the
// device.  Written independently of the CPU oracle.
//
//   FREE     V = m2/2 phi^2                                    p = {m2}
//   CHAOTIC2 V = m2/2 phi^2 + g2/2 phi^2 chi^2      (Sec. 3.1)  p = {m2, g2}
//   OSCILLON V = m2/2 phi^2 - lam/4 phi^4 + g/6 phi^6 (Sec. 3.2) p = {m2, lam, g}
//   QBALL    V = m2 u (1 + K ln(u/M^2)), u = |Phi|^2 = (phi1^2 + phi2^2)/2
//                                                    (Sec. 3.3)  p = {m2, K, M}
//
// Pot<M>::eval gives V and dV/dphi_i in float64.  Pot<M>::split_prep gives,
// at the float64 background phi0, V(phi0), V'(phi0) and the float32 constants
// of the difference forms.  It runs in one thread per stage, where every
// float64 instruction is ~70 cycles of latency on GB300, so constants that are
// only used in float32 are formed in float32 (fp: the parameters in float32;
// slots 4 and 5 hold m2/2 and params[1]/2) wherever that costs at most an ulp.
// Pot<M>::SplitK / diff give,
// in float32, the differences dV'_i = V'_i(phi0 + d) - V'_i(phi0) and
// dV = V(phi0 + d) - V(phi0) around a float64 background phi0, written so that
// every term carries at least one factor of d (no cancellation for small d):
// this is the bulk arithmetic of the split-FP32 form, where phi = phi0 + d
// (the homogeneous/perturbation split of Sec. 2.2, Eq. phi-lin).
#pragma once

#include <cuda_runtime.h>

namespace pycool {

enum ModelId { M_FREE = 0, M_CHAOTIC2 = 1, M_OSCILLON = 2, M_QBALL = 3,
               // potentials compiled at run time (pycool_model_define), 1 or 2 fields:
               // their V and V' come from arrays the compiled kernel fills
               M_RUNTIME1 = 4, M_RUNTIME2 = 5 };

template <int M> struct Pot;

// ---------------------------------------------------------------- FREE
template <> struct Pot<M_FREE> {
  static constexpr int NF = 1;
  struct K { double m2, hm2; };
  __device__ static K prep(const double* p, const double*) { return K{p[0], 0.5 * p[0]}; }
  __device__ static void eval(const K& k, const double* f, double* dV, double& V) {
    dV[0] = k.m2 * f[0];
    V = k.hm2 * f[0] * f[0];
  }
  struct SplitK { float m2, hm2, p0, two_p0; };
  __device__ static SplitK split_prep(const K& pk, const double*, const double*, const float* fp,
                                      const double* phi0, double* dV0, double& V0) {
    eval(pk, phi0, dV0, V0);
    const float p0 = (float)phi0[0];
    return SplitK{fp[0], fp[4], p0, 2.f * p0};
  }
  __device__ static void diff(const SplitK& k, const float* d, float* dVd, float& dVv) {
    dVd[0] = k.m2 * d[0];
    dVv = k.hm2 * (d[0] * (k.two_p0 + d[0]));
  }
};

// ---------------------------------------------------------------- CHAOTIC2
template <> struct Pot<M_CHAOTIC2> {
  static constexpr int NF = 2;
  struct K { double m2, g2; };
  __device__ static K prep(const double* p, const double*) { return K{p[0], p[1]}; }
  __device__ static void eval(const K& k, const double* f, double* dV, double& V) {
    const double ph2 = f[0] * f[0];
    const double t = fma(k.g2, f[1] * f[1], k.m2);       // m2 + g2 chi^2
    dV[0] = f[0] * t;                                   // m2 phi + g2 phi chi^2
    dV[1] = (k.g2 * ph2) * f[1];                        // g2 phi^2 chi
    V = ph2 * (0.5 * t);                                // phi^2 (m2 + g2 chi^2) / 2
  }
  struct SplitK { float m2, g2, hm2, hg2, p0, c0, two_p0, two_c0, p0sq, c0sq; };
  __device__ static SplitK split_prep(const K& pk, const double*, const double*, const float* fp,
                                      const double* b, double* dV0, double& V0) {
    eval(pk, b, dV0, V0);
    SplitK k;
    k.m2 = fp[0]; k.g2 = fp[1];
    k.hm2 = fp[4]; k.hg2 = fp[5];
    k.p0 = (float)b[0]; k.c0 = (float)b[1];
    k.two_p0 = 2.f * k.p0; k.two_c0 = 2.f * k.c0;   // exact
    k.p0sq = k.p0 * k.p0; k.c0sq = k.c0 * k.c0;     // within an ulp of the float64 square
    return k;
  }
  // P = phi^2, Q = chi^2:  dP = d_phi (2 phi0 + d_phi),  dQ = d_chi (2 chi0 + d_chi)
  //   dV'_phi = m2 d_phi + g2 (d_phi Q + phi0 dQ)
  //   dV'_chi = g2 (dP chi + P0 d_chi)
  //   dV      = m2/2 dP + g2/2 (dP Q + P0 dQ)
  __device__ static void diff(const SplitK& k, const float* d, float* dVd, float& dVv) {
    const float dp = d[0], dc = d[1];
    const float dP = dp * (k.two_p0 + dp);
    const float dQ = dc * (k.two_c0 + dc);
    const float Q = k.c0sq + dQ;
    const float ch = k.c0 + dc;
    dVd[0] = fmaf(k.m2, dp, k.g2 * fmaf(dp, Q, k.p0 * dQ));
    dVd[1] = k.g2 * fmaf(dP, ch, k.p0sq * dc);
    dVv = fmaf(k.hm2, dP, k.hg2 * fmaf(dP, Q, k.p0sq * dQ));
  }
};

// ---------------------------------------------------------------- OSCILLON
template <> struct Pot<M_OSCILLON> {
  static constexpr int NF = 1;
  struct K { double m2, lam, g, hm2, qlam, sg; };
  __device__ static K prep(const double* p, const double*) {
    return K{p[0], p[1], p[2], 0.5 * p[0], 0.25 * p[1], p[2] * (1.0 / 6.0)};
  }
  __device__ static void eval(const K& k, const double* f, double* dV, double& V) {
    const double x2 = f[0] * f[0];
    dV[0] = f[0] * fma(x2, fma(k.g, x2, -k.lam), k.m2);   // m2 x - lam x^3 + g x^5
    V = x2 * fma(x2, fma(k.sg, x2, -k.qlam), k.hm2);      // m2/2 x^2 - lam/4 x^4 + g/6 x^6
  }
  // V' and V are polynomials, so their differences are exact Taylor polynomials
  // in d around x0 whose coefficients are
  //   dV'(d) = d (c1 + d (c2 + d (c3 + d (c4 + d c5))))
  //     c1 = m2 - 3 lam x0^2 + 5 g x0^4,  c2 = -3 lam x0 + 10 g x0^3,
  //     c3 = -lam + 10 g x0^2,  c4 = 5 g x0,  c5 = g
  //   dV(d)  = d (e1 + d (e2 + d (e3 + d (e4 + d (e5 + d e6)))))
  //     e1 = m2 x0 - lam x0^3 + g x0^5,  e2 = m2/2 - 3 lam/2 x0^2 + 5 g/2 x0^4,
  //     e3 = -lam x0 + 10 g/3 x0^3,  e4 = -lam/4 + 5 g/2 x0^2,  e5 = g x0,  e6 = g/6
  struct SplitK { float c[5], e[6]; };
  // The leading coefficients c1 = V''(x0) and e1 = V'(x0) are formed in float64
  // (they may be small differences of larger terms); the higher-order ones
  // multiply at least d^2 and are formed in float32.
  __device__ static SplitK split_prep(const K& pk, const double* p, const double*, const float* fp,
                                      const double* b, double* dV0, double& V0) {
    eval(pk, b, dV0, V0);
    const double m2 = p[0], lam = p[1], g = p[2];
    const double x = b[0], x2 = x * x, x4 = x2 * x2;
    SplitK k;
    k.c[0] = (float)fma(x4, 5.0 * g, fma(x2, -3.0 * lam, m2));   // V''(x0)
    k.e[0] = (float)dV0[0];                                      // V'(x0)
    const float mf = fp[0], lf = fp[1], gf = fp[2];
    const float xf = (float)x, xf2 = xf * xf, xf3 = xf2 * xf, xf4 = xf2 * xf2;
    k.c[1] = fmaf(10.f * gf, xf3, -3.f * lf * xf);
    k.c[2] = fmaf(10.f * gf, xf2, -lf);
    k.c[3] = 5.f * gf * xf;
    k.c[4] = gf;
    k.e[1] = fmaf(2.5f * gf, xf4, fmaf(-1.5f * lf, xf2, 0.5f * mf));
    k.e[2] = fmaf((10.f / 3.f) * gf, xf3, -lf * xf);
    k.e[3] = fmaf(2.5f * gf, xf2, -0.25f * lf);
    k.e[4] = gf * xf;
    k.e[5] = gf * (1.f / 6.f);
    return k;
  }
  __device__ static void diff(const SplitK& k, const float* dd, float* dVd, float& dVv) {
    const float d = dd[0];
    dVd[0] = d * fmaf(d, fmaf(d, fmaf(d, fmaf(d, k.c[4], k.c[3]), k.c[2]), k.c[1]), k.c[0]);
    dVv = d * fmaf(d, fmaf(d, fmaf(d, fmaf(d, fmaf(d, k.e[5], k.e[4]), k.e[3]), k.e[2]), k.e[1]),
                   k.e[0]);
  }
};

// ---------------------------------------------------------------- QBALL
template <> struct Pot<M_QBALL> {
  static constexpr int NF = 2;
  struct K { double m2, K1, mK, lnM2, m2K1; };
  // dv[0] = ln(M^2), computed once on the host
  __device__ static K prep(const double* p, const double* dv) {
    return K{p[0], 1.0 + p[1], p[0] * p[1], dv[0], p[0] * (1.0 + p[1])};
  }
  // u = (f1^2 + f2^2)/2 ; V' = m2 (1 + K + K ln(u/M^2)) f_i ; V = m2 u (1 + K ln(u/M^2))
  __device__ static void eval(const K& k, const double* f, double* dV, double& V) {
    const double u = 0.5 * fma(f[0], f[0], f[1] * f[1]);
    if (u > 0.0) {
      const double l = log(u) - k.lnM2;
      const double kl = k.mK * l;                          // m2 K ln(u/M^2)
      const double fac = fma(k.m2, k.K1, kl);              // m2 (1 + K) + m2 K ln
      dV[0] = fac * f[0];
      dV[1] = fac * f[1];
      V = u * (k.m2 + kl);
    } else {
      dV[0] = 0.0; dV[1] = 0.0; V = 0.0;
    }
  }
  // For the FP64 sweep: from u2 = |Phi|^2 = 2u, the factor fac of V'_i =
  // fac f_i and twice the potential,
  //   fac = m2 (1 + K) + m2 K l,   V2 = 2V = u2 (m2 + m2 K l),   l = ln(u/M^2),
  // with the logarithm taken near a reference u_ref (the sweep's per-stage
  // value at one site, the same in every block): hinv = 1/(2 u_ref), lref =
  // ln(u_ref/M^2), x = u/u_ref - 1 = u2 hinv - 1 and l = lref + log1p(x) by its
  // Taylor series sum_k (-1)^(k+1) x^k / k -- 5 terms for |x| < 2^-12 (the
  // first omitted term is below 2^-60 |x|), 11 terms for |x| < 2^-5 (below
  // 2^-60 |x|) -- and the full logarithm farther away or without a reference
  // (hinv = 0 gives x = -1).  The tiers are chosen on the high word of x as an
  // integer, and Phi = 0 on the bits of u2 (never negative), so that no
  // float64 instruction is spent on the tests.
  __device__ static void fac_near(const K& k, double u2, double hinv, double lref, double& fac,
                                  double& V2) {
    if (__double_as_longlong(u2) == 0) {   // Phi = 0: V = V' = 0
      fac = 0.0;
      V2 = 0.0;
      return;
    }
    const double x = fma(u2, hinv, -1.0);
    const int hx = __double2hiint(x) & 0x7fffffff;
    double l;
    if (hx < 0x3F300000) {            // |x| < 2^-12
      double q = fma(x, 0.2, -0.25);
      q = fma(q, x, 1.0 / 3.0);
      q = fma(q, x, -0.5);
      q = fma(q, x, 1.0);
      l = fma(q, x, lref);
    } else if (hx < 0x3FA00000) {     // |x| < 2^-5
      double q = fma(x, -1.0 / 12.0, 1.0 / 11.0);
      q = fma(q, x, -0.1);
      q = fma(q, x, 1.0 / 9.0);
      q = fma(q, x, -0.125);
      q = fma(q, x, 1.0 / 7.0);
      q = fma(q, x, -1.0 / 6.0);
      q = fma(q, x, 0.2);
      q = fma(q, x, -0.25);
      q = fma(q, x, 1.0 / 3.0);
      q = fma(q, x, -0.5);
      q = fma(q, x, 1.0);
      l = fma(q, x, lref);
    } else {
      l = log(0.5 * u2) - k.lnM2;
    }
    fac = fma(k.mK, l, k.m2K1);
    V2 = u2 * fma(k.mK, l, k.m2);
  }
  // du = d1 (p1 + d1/2) + d2 (p2 + d2/2),  l = log1p(du/u0)
  //   dV'_i = m2 [ A d_i + K l (p_i + d_i) ],  A = 1 + K + K L0
  //   dV    = m2 [ B du + K l (u0 + du) ],      B = 1 + K L0,  L0 = ln(u0/M^2)
  struct SplitK { float m2, K, A, B, p1, p2, u0, inv_u0; int direct; float lnM2; };
  // one logarithm for V(phi0), V'(phi0) and the constants (dv[0] = ln M^2)
  __device__ static SplitK split_prep(const K& pk, const double* p, const double* dv, const float*,
                                      const double* b, double* dV0, double& V0) {
    SplitK k;
    const double u0 = 0.5 * fma(b[0], b[0], b[1] * b[1]);
    k.m2 = (float)p[0]; k.K = (float)p[1];
    k.p1 = (float)b[0]; k.p2 = (float)b[1];
    k.lnM2 = (float)dv[0];
    k.direct = !(u0 > 1e-30);
    const double L = u0 > 0.0 ? log(u0) - dv[0] : 0.0;   // ln(u0 / M^2)
    const double L0 = k.direct ? 0.0 : L;
    k.A = (float)(1.0 + p[1] + p[1] * L0);
    k.B = (float)(1.0 + p[1] * L0);
    k.u0 = (float)u0;
    k.inv_u0 = k.direct ? 0.f : (float)__drcp_rn(u0);
    if (u0 > 0.0) {  // as eval(), with the logarithm above
      const double kl = pk.mK * L;
      const double fac = fma(pk.m2, pk.K1, kl);
      dV0[0] = fac * b[0];
      dV0[1] = fac * b[1];
      V0 = u0 * (pk.m2 + kl);
    } else {
      dV0[0] = 0.0; dV0[1] = 0.0; V0 = 0.0;
    }
    return k;
  }
  // GENERAL: the caller knows k.direct == 0 (a background away from the
  // origin, every stage of a practical run), so the test per site is dropped.
  template <bool GENERAL = false>
  __device__ static void diff(const SplitK& k, const float* d, float* dVd, float& dVv) {
    if (!GENERAL && k.direct) {  // background at the origin: V(phi0) = V'(phi0) = 0
      const float u = 0.5f * fmaf(d[0], d[0], d[1] * d[1]);
      if (u > 0.f) {
        const float l = logf(u) - k.lnM2;
        const float fac = k.m2 * fmaf(k.K, l, 1.f + k.K);
        dVd[0] = fac * d[0]; dVd[1] = fac * d[1];
        dVv = k.m2 * u * fmaf(k.K, l, 1.f);
      } else {
        dVd[0] = 0.f; dVd[1] = 0.f; dVv = 0.f;
      }
      return;
    }
    const float du = fmaf(d[0], fmaf(0.5f, d[0], k.p1), d[1] * fmaf(0.5f, d[1], k.p2));
    const float u = k.u0 + du;
    if (u > 0.f) {
      // log1p(y), y = du / u0: for |y| < 2^-7 the Taylor series y - y^2/2 +
      // y^3/3 - y^4/4 (the first omitted term is below 2^-30 |y|, under the
      // rounding of float32), else log1pf
      const float y = du * k.inv_u0;
      float l;
      if (fabsf(y) < 0.0078125f) {
        float q = fmaf(y, -0.25f, 0.333333343f);
        q = fmaf(q, y, -0.5f);
        l = fmaf(q * y, y, y);
      } else {
        l = log1pf(y);
      }
      const float Kl = k.K * l;
      dVd[0] = k.m2 * fmaf(k.A, d[0], Kl * (k.p1 + d[0]));
      dVd[1] = k.m2 * fmaf(k.A, d[1], Kl * (k.p2 + d[1]));
      dVv = k.m2 * fmaf(k.B, du, Kl * u);
    } else {  // |Phi| = 0 here: V = V' = 0
      dVd[0] = -k.m2 * k.A * k.p1;
      dVd[1] = -k.m2 * k.A * k.p2;
      dVv = -k.m2 * k.B * k.u0;
    }
  }
};

// ---------------------------------------------------------------- RUNTIME
// A potential given at run time: its values reach the sweep through arrays
// (rt_kick), so these records carry nothing.
template <int NFIELDS> struct PotRuntime {
  static constexpr int NF = NFIELDS;
  struct K {};
  struct SplitK {};
  __device__ static K prep(const double*, const double*) { return K{}; }
};
template <> struct Pot<M_RUNTIME1> : PotRuntime<1> {};
template <> struct Pot<M_RUNTIME2> : PotRuntime<2> {};

}  // namespace pycool
