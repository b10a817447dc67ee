// The potentials of models.cuh as difference forms in double-float arithmetic,
// for the split-DD form: phi = phi0 + d with the lattice mean phi0 in float64
// and the fluctuation d a double-float (dd.cuh).  For each model,
//   PotDD<M>::prep  : at the float64 background phi0 (one thread per stage):
//                     V(phi0), V'(phi0) in float64 and the double-float
//                     constants of the difference forms;
//   PotDD<M>::diff  : per site, dV'_i = V'_i(phi0 + d) - V'_i(phi0) and
//                     dV = V(phi0 + d) - V(phi0), written so that every term
//                     carries a factor of d (no cancellation for small d).
// The forms are those of models.cuh (Sec. 3: the potentials; Sec. 2.2, Eq.
// phi-lin: the homogeneous/perturbation split), evaluated with ~48-bit
// significands instead of 24, so that the fluctuations keep float64-class
// accuracy relative to the whole field.
#pragma once

#include <math.h>

#include "dd.cuh"
#include "models.cuh"

namespace pycool {

template <int M> struct PotDD;

// ---------------------------------------------------------------- FREE
template <> struct PotDD<M_FREE> {
  struct SplitK { dd m2, hm2, two_p0; };
  __device__ static SplitK prep(const Pot<M_FREE>::K& pk, const double*, const double*,
                                const double* phi0, double* dV0, double& V0) {
    Pot<M_FREE>::eval(pk, phi0, dV0, V0);
    return SplitK{dd(pk.m2), dd(pk.hm2), dd(2.0 * phi0[0])};
  }
  __device__ static void diff(const SplitK& k, const dd* d, dd* dVd, dd& dVv) {
    dVd[0] = k.m2 * d[0];
    dVv = k.hm2 * (d[0] * (k.two_p0 + d[0]));   // (free field: a few operations)
  }
};

// ---------------------------------------------------------------- CHAOTIC2
template <> struct PotDD<M_CHAOTIC2> {
  struct SplitK { dd m2, g2, hm2, hg2, p0, c0, two_p0, two_c0, p0sq, c0sq; };
  __device__ static SplitK prep(const Pot<M_CHAOTIC2>::K& pk, const double* p, const double*,
                                const double* b, double* dV0, double& V0) {
    Pot<M_CHAOTIC2>::eval(pk, b, dV0, V0);
    SplitK k;
    k.m2 = dd(p[0]); k.g2 = dd(p[1]);
    k.hm2 = dd(0.5 * p[0]); k.hg2 = dd(0.5 * p[1]);
    k.p0 = dd(b[0]); k.c0 = dd(b[1]);
    k.two_p0 = dd(2.0 * b[0]); k.two_c0 = dd(2.0 * b[1]);
    k.p0sq = dd(b[0] * b[0]); k.c0sq = dd(b[1] * b[1]);
    return k;
  }
  // P = phi^2, Q = chi^2: dP = d_phi (2 phi0 + d_phi), dQ = d_chi (2 chi0 + d_chi)
  //   dV'_phi = m2 d_phi + g2 (d_phi Q + phi0 dQ),  dV'_chi = g2 (dP chi + P0 d_chi)
  //   dV      = m2/2 dP + g2/2 (dP Q + P0 dQ)
  __device__ static void diff(const SplitK& k, const dd* d, dd* dVd, dd& dVv) {
    const dd dp = d[0], dc = d[1];
    const dd dP = dp * (k.two_p0 + dp);
    const dd dQ = dc * (k.two_c0 + dc);
    const dd Q = k.c0sq + dQ;
    const dd ch = k.c0 + dc;
    const dd mix = dd_fma(dp, Q, k.p0 * dQ);
    dVd[0] = dd_fma(k.m2, dp, k.g2 * mix);
    dVd[1] = k.g2 * dd_fma(dP, ch, k.p0sq * dc);
    dVv = dd_fma(k.hm2, dP, k.hg2 * dd_fma(dP, Q, k.p0sq * dQ));
  }
};

// ---------------------------------------------------------------- OSCILLON
template <> struct PotDD<M_OSCILLON> {
  // dV'(d) = d (c1 + d (c2 + d (c3 + d (c4 + d c5))))
  // dV(d)  = d (e1 + d (e2 + d (e3 + d (e4 + d (e5 + d e6)))))
  // with the Taylor coefficients of models.cuh, formed in float64 here.
  struct SplitK { dd c[5], e[6]; };
  __device__ static SplitK prep(const Pot<M_OSCILLON>::K& pk, const double* p, const double*,
                                const double* b, double* dV0, double& V0) {
    Pot<M_OSCILLON>::eval(pk, b, dV0, V0);
    const double m2 = p[0], lam = p[1], g = p[2];
    const double x = b[0], x2 = x * x, x3 = x2 * x, x4 = x2 * x2;
    SplitK k;
    k.c[0] = dd(fma(x4, 5.0 * g, fma(x2, -3.0 * lam, m2)));
    k.c[1] = dd(fma(10.0 * g, x3, -3.0 * lam * x));
    k.c[2] = dd(fma(10.0 * g, x2, -lam));
    k.c[3] = dd(5.0 * g * x);
    k.c[4] = dd(g);
    k.e[0] = dd(dV0[0]);
    k.e[1] = dd(fma(2.5 * g, x4, fma(-1.5 * lam, x2, 0.5 * m2)));
    k.e[2] = dd(fma((10.0 / 3.0) * g, x3, -lam * x));
    k.e[3] = dd(fma(2.5 * g, x2, -0.25 * lam));
    k.e[4] = dd(g * x);
    k.e[5] = dd(g * (1.0 / 6.0));
    return k;
  }
  __device__ static void diff(const SplitK& k, const dd* dd_, dd* dVd, dd& dVv) {
    const dd d = dd_[0];
    dd t = dd_fma(d, k.c[4], k.c[3]);
    t = dd_fma(d, t, k.c[2]);
    t = dd_fma(d, t, k.c[1]);
    t = dd_fma(d, t, k.c[0]);
    dVd[0] = d * t;
    dd u = dd_fma(d, k.e[5], k.e[4]);
    u = dd_fma(d, u, k.e[3]);
    u = dd_fma(d, u, k.e[2]);
    u = dd_fma(d, u, k.e[1]);
    u = dd_fma(d, u, k.e[0]);
    dVv = d * u;
  }
};

// ---------------------------------------------------------------- QBALL
// log(1 + x) for a double-float x: for |x| < 2^-12 its Taylor series
// x - x^2/2 + x^3/3 - x^4/4 + x^5/5 with the first two terms in double-float
// and the rest in float (x^3/3 is below 2^-24 of the sum, so float leaves
// 2^-48; the first omitted term is below 2^-60 of it); for |x| < 2^-5 the
// series of 2 atanh(s), s = x / (2 + x):  2 s (1 + s^2/3 + s^4/5 + s^6/7 + ...),
// the first two terms in double-float and the rest in float (|s| < 2^-6, so
// s^4/5 is 2^-26 of the sum and s^8/9 under 2^-51); otherwise the float64 log1p.
__device__ __forceinline__ dd dd_log1p(dd x) {
  if (fabsf(x.hi) < 0.000244140625f) {
    const dd h = dd_sqr(x);
    const float xh = x.hi;
    const float tail = fmul(xh, fmul(xh, fmul(xh, ffma(xh, ffma(xh, 0.2f, -0.25f),
                                                      0.333333333f))));
    return (x - dd(fmul(0.5f, h.hi), fmul(0.5f, h.lo))) + tail;
  }
  if (fabsf(x.hi) < 0.03125f) {
    const dd s = dd_div(x, x + 2.0f);
    const dd s2 = dd_sqr(s);
    const float w = fmul(s2.hi, ffma(s2.hi, 1.0f / 7.0f, 1.0f / 5.0f));
    const dd t = s2 * (dd(0.3333333432674408f, -9.934107758624577e-09f) + w);   // 1/3 + w
    const dd r = s * (t + 1.0f);
    return dd(fadd(r.hi, r.hi), fadd(r.lo, r.lo));
  }
  return dd(log1p((double)x));
}

template <> struct PotDD<M_QBALL> {
  // du = d1 (p1 + d1/2) + d2 (p2 + d2/2),  l = log1p(du/u0)
  //   dV'_i = m2 [ A d_i + K l (p_i + d_i) ],  A = 1 + K + K L0
  //   dV    = m2 [ B du + K l (u0 + du) ],      B = 1 + K L0,  L0 = ln(u0/M^2)
  // with m2 folded into the constants: mA = m2 A, mB = m2 B, mK = m2 K.
  // direct (background at the origin, V(phi0) = V'(phi0) = 0): the potential
  // of the fluctuation itself, u = |d|^2/2, with a float64 logarithm.
  struct SplitK { dd m2, K, A, B, p1, p2, u0, inv_u0, hp1, hp2; int direct; double lnM2, Kd, m2d; };
  __device__ static SplitK prep(const Pot<M_QBALL>::K& pk, const double* p, const double* dv,
                                const double* b, double* dV0, double& V0) {
    SplitK k;
    const double u0 = 0.5 * fma(b[0], b[0], b[1] * b[1]);
    k.direct = !(u0 > 1e-30);
    const double L = u0 > 0.0 ? log(u0) - dv[0] : 0.0;
    const double L0 = k.direct ? 0.0 : L;
    k.m2 = dd(p[0]); k.K = dd(p[0] * p[1]);
    k.A = dd(p[0] * (1.0 + p[1] + p[1] * L0));
    k.B = dd(p[0] * (1.0 + p[1] * L0));
    k.p1 = dd(b[0]); k.p2 = dd(b[1]);
    k.u0 = dd(u0);
    k.inv_u0 = k.direct ? dd() : dd(1.0 / u0);
    k.hp1 = dd(0.5 * b[0]); k.hp2 = dd(0.5 * b[1]);
    k.lnM2 = dv[0]; k.Kd = p[1]; k.m2d = p[0];
    if (u0 > 0.0) {
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
  __device__ static void diff(const SplitK& k, const dd* d, dd* dVd, dd& dVv) {
    if (k.direct) {
      const double d1 = (double)d[0], d2 = (double)d[1];
      const double u = 0.5 * fma(d1, d1, d2 * d2);
      if (u > 0.0) {
        const double l = log(u) - k.lnM2;
        const double fac = k.m2d * fma(k.Kd, l, 1.0 + k.Kd);
        dVd[0] = dd(fac * d1); dVd[1] = dd(fac * d2);
        dVv = dd(k.m2d * u * fma(k.Kd, l, 1.0));
      } else {
        dVd[0] = dd(); dVd[1] = dd(); dVv = dd();
      }
      return;
    }
    const dd du = dd_fma(d[0], dd_fma(0.5f, d[0], k.p1), d[1] * dd_fma(0.5f, d[1], k.p2));
    const dd u = k.u0 + du;
    if (u.hi > 0.f) {
      const dd Kl = k.K * dd_log1p(du * k.inv_u0);   // m2 K l
      dVd[0] = dd_fma(k.A, d[0], Kl * (k.p1 + d[0]));
      dVd[1] = dd_fma(k.A, d[1], Kl * (k.p2 + d[1]));
      dVv = dd_fma(k.B, du, Kl * u);
    } else {   // |Phi| = 0 here: V = V' = 0
      dVd[0] = -(k.A * k.p1);
      dVd[1] = -(k.A * k.p2);
      dVv = -(k.B * k.u0);
    }
  }
};

}  // namespace pycool
