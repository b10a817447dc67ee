// The fused stage sweep: one launch advances every lattice site through one
// second-order stage of Sec. 2.3,
//     Phi_H1(h/2) Phi_H2(h/2) Phi_H3(h) Phi_H2(h/2) Phi_H1(h/2),
// with the exact flows of Eq. split-Phi.  Consecutive stages share their
// boundary: the trailing Phi_H2(h_prev/2) Phi_H1(h_prev/2) of one stage and the
// leading Phi_H1(h/2) Phi_H2(h/2) of the next act on (a, p_a) as scalar updates
// (pi is unchanged by H1 and H2, so sum pi^2 from the previous sweep is exact
// for both Phi_H2's) and on phi as ONE drift with coefficient
//     c = h_prev / (2 a_old^2) + h / (2 a_new^2).
// A sweep therefore does, per site:
//     phi* = phi + c pi                              (drift, Phi_H2)
//     pi*  = pi + [a^2 D[phi*]/dx^2 - a^4 V'(phi*)] h (kick, Phi_H3)
// and reduces sum pi*^2, sum phi* D[phi*], sum V(phi*) for the p_a kicks.
// A "flush" sweep applies only the pending trailing half-stage (drift with
// c = h_prev/(2 a^2), then Phi_H1(h_prev/2)) and leaves a synchronised state,
// reducing the sums the energies of Eq. rho-pres need.
//
// Tiling: a block owns a TX x TY column tile and a z-chunk of ZC planes and
// streams z upward (the paper's GPU code marches z the same way).  The drifted
// plane phi*(z) lives in shared memory; the Laplacian of Eq. D is split by
// z-offset into
//     S_mid(p) = c0 ctr + c1 sum(4 faces) + c2 sum(4 corners)   (in-plane)
//     S_off(p) = c1 ctr + c2 sum(4 faces) + c3 sum(4 corners)   (for planes z+-1)
// so D(z) = S_off(z-1) + S_mid(z) + S_off(z+1) needs one resident plane and
// two registers per site.
//
// Two kernels share this arithmetic:
//   sweep_tma   (n a multiple of 32): each plane's tile and its two halo rows
//               arrive by TMA (cp.async.bulk.tensor, mbarrier completion) in a
//               3-slot shared-memory ring, two planes ahead of the compute;
//               x-neighbours come from warp shuffles (one warp = one tile row)
//               and the two halo columns from plain loads.  No periodic wrap
//               is ever asked of the TMA: halo rows are fetched at wrapped y.
//   sweep_plain (any n): plain loads with modular indices, ragged tiles masked.
//
// Reductions: per-thread column sums (Kahan in float) -> warp butterfly ->
// fixed-order sum of the 8 warps -> one partial per block and quantity.  The
// last block to arrive (atomic ticket; nobody waits) sums the partials in
// block order (Neumaier), applies the p_a kick of Phi_H3 and advances the
// Background.  Results are bitwise reproducible and depend only on the
// lattice, not on what it is batched with.
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>
#include <math.h>

#include <type_traits>

#include "internal.cuh"
#include "models.cuh"
#include "models_dd.cuh"

namespace pycool {

// ---------------------------------------------------------------------------
// Scalar part of the merged half-stages (every block computes it identically).
// ---------------------------------------------------------------------------
struct Coef {
  double c;      // drift coefficient
  double kD;     // a^2 h / dx^2
  double kV;     // a^4 h
  double a;      // a after the leading Phi_H1's
  double pa;     // p_a after the leading Phi_H2 (before this stage's Phi_H3)
  double h;      // this stage's step (0 for a flush)
  double deta;   // the conformal step of this stage's time step (h = w_i deta)
};

// The boundary between two stages splits into the part that needs only a,
// h_prev and h (PreCoef: formed ahead of the lattice sums where the caller
// can) and the part that needs p_a and sum pi^2 (prestage_p).
struct PreCoef {
  double a;      // a before the leading Phi_H1's
  double ia3;    // 1/a^3
  double hh;     // h_prev/2
  double c0;     // h_prev/(2 a^2): the trailing drift of the previous stage
  double g1;     // -(h_prev [+ h])/2 / (12 V_L m^2): the Phi_H1 flows' da/dp_a
  double nVLrm;  // -V_L rho_m
  double hn;     // h/2
  double hdx;    // h / dx^2
  double h;      // this stage's step (0 for a flush)
  double deta;   // the time step's conformal step (physical steps: found in prestage_p)
  // physical-time steps (Sec. 3.1), a stage that starts a time step: h is
  // w0 dt / a_n with a_n the scale factor of the synchronised state, known
  // only after the trailing Phi_H2 has moved p_a
  int adapt;
  double w0;     // the stage weight
  double g0;     // -(h_prev/2) / (6 V_L m^2): the trailing Phi_H1's da/dp_a
  double gm;     // -(1/2) / (6 V_L m^2): the leading Phi_H1's da/dp_a per unit h
  double dt, dx2inv;
};

// ia: 1/a (the caller's reciprocal, so that it can be formed early).
// h: this stage's step; deta: its time step's conformal step; adapt != 0: a
// physical-time step starts here and h is derived in prestage_p (h ignored).
__device__ __forceinline__ PreCoef prestage_a(double a, double ia, double hp, double h,
                                              const SimDesc& d, int mode, double deta = 0.0,
                                              int adapt = 0, double w0 = 0.0) {
  PreCoef q;
  const double ia2 = ia * ia;
  q.a = a;
  q.ia3 = ia2 * ia;
  q.hh = 0.5 * hp;
  q.c0 = q.hh * ia2;
  q.nVLrm = -(d.VL * d.rho_m0);
  q.deta = deta;
  q.adapt = (mode == MODE_SWEEP) ? adapt : 0;
  q.w0 = w0;
  q.g0 = -(d.inv6VLm2 * q.hh);
  q.gm = -(d.inv6VLm2 * 0.5);
  q.dt = d.dt;
  q.dx2inv = d.dx2inv;
  if (mode == MODE_SWEEP) {
    q.g1 = -(d.inv6VLm2 * (0.5 * (hp + h)));
    q.hn = 0.5 * h;
    q.hdx = h * d.dx2inv;
    q.h = h;
  } else {
    q.g1 = -(d.inv6VLm2 * q.hh);
    q.hn = 0.0; q.hdx = 0.0; q.h = 0.0;
  }
  return q;
}

// The scalar half-steps of a stage boundary, given p_a and sum pi^2 (pi is
// unchanged by H1 and H2, so the previous sweep's sum serves both Phi_H2's).
__device__ __forceinline__ Coef prestage_p(const PreCoef& q, double pa, double s2, int mode) {
  Coef k;
  // trailing Phi_H2(h_prev/2) of the previous stage: p_a += [sum pi^2/a^3 - V_L rho_m] h_prev/2
  pa = fma(fma(s2, q.ia3, q.nVLrm), q.hh, pa);
  double a, hn = q.hn, hdx = q.hdx, h = q.h;
  k.deta = q.deta;
  if (q.adapt) {
    // a physical-time step starts: the trailing Phi_H1(h_prev/2) gives the
    // synchronised a_n, the step is d-eta = dt / a_n (Sec. 3.1), then the
    // leading Phi_H1(h/2) of its first stage, h = w_0 d-eta
    const double an = fma(pa, q.g0, q.a);
    k.deta = q.dt / an;
    h = q.w0 * k.deta;
    hn = 0.5 * h;
    hdx = h * q.dx2inv;
    a = fma(pa, q.gm * h, an);
  } else {
    // Phi_H1(h_prev/2) [Phi_H1(h/2)] merged (p_a is constant under H1): a -= p_a dt' / (12 V_L m^2)
    a = fma(pa, q.g1, q.a);
  }
  k.a = a;
  if (mode != MODE_SWEEP) {
    k.c = q.c0; k.kD = 0.0; k.kV = 0.0; k.pa = pa; k.h = 0.0;
    return k;
  }
  // one reciprocal per value of a instead of divisions: an FP64 division costs
  // ~450 cycles of a single thread on GB300
  const double ia = __drcp_rn(a), ia2 = ia * ia;
  // leading Phi_H2(h/2)
  k.pa = fma(fma(s2, ia2 * ia, q.nVLrm), hn, pa);
  k.c = fma(hn, ia2, q.c0);
  const double a2 = a * a;
  k.kD = a2 * hdx;
  k.kV = (a2 * a2) * h;
  k.h = h;
  return k;
}

// ia_a: 1/b.a if the caller already has it (a negative value means "compute it").
// The step of the stage a Background is about to run: w_i dt (conformal), or
// w_i d-eta of the running time step (physical; d-eta found at its first stage).
__device__ __forceinline__ double stage_step(const SimDesc& d, int stage, double deta, int mode) {
  if (mode != MODE_SWEEP) return 0.0;
  return d.w[stage] * (d.physical ? deta : d.dt);
}

__device__ __forceinline__ Coef prestage(const Background& b, const SimDesc& d, int mode,
                                         double ia_a = -1.0) {
  const double h = stage_step(d, (int)b.stage, b.deta, mode);
  const int adapt = d.physical && b.stage == 0;
  const double ia = ia_a > 0.0 ? ia_a : __drcp_rn(b.a);
  return prestage_p(prestage_a(b.a, ia, b.h_prev, h, d, mode, d.physical ? b.deta : d.dt, adapt,
                               d.w[b.stage]),
                    b.pa, b.sum_pi2, mode);
}

// Explicitly typed fused multiply-add: float arithmetic must stay on the FP32
// pipe (GB300's FP64 rate is ~1/60 of FP32).
__device__ __forceinline__ float madd(float a, float b, float c) { return __fmaf_rn(a, b, c); }
__device__ __forceinline__ double madd(double a, double b, double c) { return __fma_rn(a, b, c); }

__device__ __forceinline__ bool is_fin(double x) { return isfinite(x); }

// ---------------------------------------------------------------------------
// Deterministic block reduction of NQ doubles; result in out[0..NQ) (shared).
// ---------------------------------------------------------------------------
template <int NQ>
__device__ __forceinline__ void block_sum(double (&v)[NQ], double* sred, double* out) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int q = 0; q < NQ; ++q) {
    double x = v[q];
#pragma unroll
    for (int m = 16; m >= 1; m >>= 1) x += __shfl_xor_sync(0xffffffffu, x, m);
    v[q] = x;
  }
  if (lane == 0) {
#pragma unroll
    for (int q = 0; q < NQ; ++q) sred[warp * NQ + q] = v[q];
  }
  __syncthreads();
  if (threadIdx.x < NQ) {
    double s = 0.0;
#pragma unroll
    for (int w = 0; w < kThreads / 32; ++w) s += sred[w * NQ + threadIdx.x];
    out[threadIdx.x] = s;
  }
  __syncthreads();
}

// Reduction slot layout.
template <int NF, int PREC> struct Slots;
template <int NF> struct Slots<NF, PREC_FP64> {
  // pi^2[f], phi D[f], V, (phi-K)[f], (phi-K)^2[f]
  static constexpr int PI2 = 0, PHID = NF, V = 2 * NF, DPHI = 2 * NF + 1, DPHI2 = 3 * NF + 1;
  static constexpr int NQ = 4 * NF + 1;
};
template <int NF> struct Slots<NF, PREC_SPLIT> {
  // dpi[f], dpi^2[f], dphi D[f], dV, dphi[f], dphi^2[f]
  static constexpr int DPI = 0, DPI2 = NF, PHID = 2 * NF, V = 3 * NF, DPHI = 3 * NF + 1,
                       DPHI2 = 4 * NF + 1;
  static constexpr int NQ = 5 * NF + 1;
};
template <int NF> struct Slots<NF, PREC_DD> : Slots<NF, PREC_SPLIT> {};

// The working type of a form: float64, float, or a double-float pair.
template <int PREC> struct WorkT { using type = float; };
template <> struct WorkT<PREC_FP64> { using type = double; };
template <> struct WorkT<PREC_DD> { using type = dd; };
// The constants of a split form's difference forms.
template <int MODEL, int PREC> struct SplitKOf { using type = typename Pot<MODEL>::SplitK; };
template <int MODEL> struct SplitKOf<MODEL, PREC_DD> { using type = typename PotDD<MODEL>::SplitK; };

template <typename T, int V> struct Vec;
template <> struct Vec<float, 1> { using type = float; };
template <> struct Vec<float, 2> { using type = float2; };
template <> struct Vec<float, 4> { using type = float4; };
template <> struct Vec<double, 1> { using type = double; };
template <> struct Vec<double, 2> { using type = double2; };
template <> struct Vec<dd, 1> { using type = float2; };
template <> struct Vec<dd, 2> { using type = float4; };

// Load / store VX consecutive elements (aligned to VX * sizeof(T)).
template <typename T, int VX>
__device__ __forceinline__ void vload(const T* p, T (&v)[VX]) {
  using VT = typename Vec<T, VX>::type;
  const VT x = *reinterpret_cast<const VT*>(p);
  const T* e = reinterpret_cast<const T*>(&x);
#pragma unroll
  for (int j = 0; j < VX; ++j) v[j] = e[j];
}
template <typename T, int VX>
__device__ __forceinline__ void vstore(T* p, const T (&v)[VX]) {
  using VT = typename Vec<T, VX>::type;
  VT x;
  T* e = reinterpret_cast<T*>(&x);
#pragma unroll
  for (int j = 0; j < VX; ++j) e[j] = v[j];
  *reinterpret_cast<VT*>(p) = x;
}

// Kahan-compensated accumulation for the float path; plain for double.
template <typename T> struct Acc {
  T s, c;
  __device__ __forceinline__ void zero() { s = 0; c = 0; }
  __device__ __forceinline__ void add(T x) {
    if constexpr (sizeof(T) == 4) {
      const T y = x - c;
      const T t = s + y;
      c = (t - s) - y;
      s = t;
    } else {
      s += x;
    }
  }
  __device__ __forceinline__ double value() const { return (double)s - (double)c; }
};

// ---------------------------------------------------------------------------
// Per-launch context: the coefficients every block derives from the
// Background (identically), and the per-site update.
// ---------------------------------------------------------------------------
// Shift K of a flush's variance sums, sum (phi - K) and sum (phi - K)^2
// (FP64 form): the drifted value of field f at site 0, read from the flush's
// input arrays (buffers `cur`; c: the flush's drift coefficient).  A value of
// the field itself lies within a few standard deviations of its lattice mean,
// so the two sums do not cancel; a stale shift (the previous flush's mean)
// would, since the mean moves by O(1) over an oscillation while the variance
// can be 1e-10.  Every block computes the same K from the same two values.
__device__ __forceinline__ double flush_shift(const SimDesc& d, int cur, int f, double c) {
  const double* ph = static_cast<const double*>(d.phi[cur & 1]);
  const double* pv = static_cast<const double*>(d.pi[(cur >> 1) & 1]);
  return fma(c, __ldcg(pv + (size_t)f * d.S), __ldcg(ph + (size_t)f * d.S));
}

template <int MODEL, int PREC>
struct Ctx {
  using P = Pot<MODEL>;
  static constexpr int NF = P::NF;
  using T = typename WorkT<PREC>::type;
  using SL = Slots<NF, PREC>;
  Coef k;
  typename P::K pk;
  T cdrift, kD, kV;
  T nkVg;                          // FP64 chaotic model: -kV g2 (folded into the chi kick)
  T mu_phi[NF], mu_pi[NF];
  T shiftK[NF];
  double phi0s[NF], pi0s[NF], V0;  // split forms: background after drift / kick
  typename SplitKOf<MODEL, PREC>::type sk;
  double q_inv, q_lref;            // FP64 Q-ball: 1/(2 u_ref), ln(u_ref/M^2) (0, 0: no reference)

  __device__ __forceinline__ void init(const Background& bg, const SimDesc& d, int mode,
                                       double ia_a = -1.0) {
    set_coef(prestage(bg, d, mode, ia_a), d, mode, P::prep(d.params, d.derived));
    if constexpr (PREC != PREC_FP64) {
      double p0[2 * NF];
      recenter(bg.mu_phi, bg.mu_pi, bg.phi0, bg.pi0, p0);
      split_tail(d, mode, p0);
    } else {
#pragma unroll
      for (int f = 0; f < NF; ++f)
        shiftK[f] = (mode == MODE_FLUSH) ? (T)flush_shift(d, bg.cur, f, k.c) : (T)0;
      set_qref(d, bg.cur);
    }
  }

  //   set_qref (FP64 Q-ball): the reference of the logarithm, |Phi|^2/2 of the
  //   drifted field at site 0 of the stage's input buffers (every block reads
  //   the same two values, so every block uses the same reference)
  __device__ __forceinline__ void set_qref(const SimDesc& d, int cur) {
    if constexpr (PREC == PREC_FP64 && MODEL == M_QBALL) {
      const double f0 = flush_shift(d, cur, 0, k.c), f1 = flush_shift(d, cur, 1, k.c);
      const double u = 0.5 * fma(f0, f0, f1 * f1);
      q_inv = u > 0.0 ? 0.5 / u : 0.0;
      q_lref = u > 0.0 ? log(u) - pk.lnM2 : 0.0;
    }
  }

  // The pieces of init, in the order a stage boundary can form them.
  //   set_coef: the working-precision coefficients of the scalar half-steps
  __device__ __forceinline__ void set_coef(const Coef& kk, const SimDesc& d, int mode,
                                           const typename P::K& pkk) {
    k = kk;
    pk = pkk;
    cdrift = (T)k.c; kD = (T)k.kD; kV = (T)k.kV;
    if constexpr (PREC == PREC_FP64) {
      if constexpr (MODEL == M_CHAOTIC2) nkVg = -k.kV * d.params[1];
      V0 = 0.0;
#pragma unroll
      for (int f = 0; f < NF; ++f) { mu_phi[f] = 0; mu_pi[f] = 0; phi0s[f] = 0; pi0s[f] = 0; }
    }
  }
  //   recenter (split form): the float means mu of the fluctuations move into
  //   the float64 background; p0 = re-centred (phi0[0..NF), pi0[0..NF))
  __device__ __forceinline__ void recenter(const double* mphi, const double* mpi,
                                           const double* phi0, const double* pi0, double* p0) {
#pragma unroll
    for (int f = 0; f < NF; ++f) {
      mu_phi[f] = (T)mphi[f];
      mu_pi[f] = (T)mpi[f];
      p0[f] = phi0[f] + (double)mu_phi[f];
      p0[NF + f] = pi0[f] + (double)mu_pi[f];
      shiftK[f] = T(0.0);
    }
  }
  //   split_tail (split form): the background's own drift and kick, and the
  //   float constants of the difference forms at the drifted background
  __device__ __forceinline__ void split_tail(const SimDesc& d, int mode, const double* p0) {
    double dV0[NF];
#pragma unroll
    for (int f = 0; f < NF; ++f) phi0s[f] = fma(k.c, p0[NF + f], p0[f]);   // background drift
    if constexpr (PREC == PREC_DD)
      sk = PotDD<MODEL>::prep(pk, d.params, d.derived, phi0s, dV0, V0);
    else
      sk = P::split_prep(pk, d.params, d.derived, d.fparams, phi0s, dV0, V0);
#pragma unroll
    for (int f = 0; f < NF; ++f)  // background kick (D[phi0] = 0)
      pi0s[f] = (mode == MODE_SWEEP) ? fma(-k.kV, dV0[f], p0[NF + f]) : p0[NF + f];
  }

  // The kick of Phi_H3 and the per-site sums for one site.
  //   phj: drifted fields, D: Laplacian, pim: momenta -> pin: new momenta
  // GENERAL (split Q-ball): the background is away from the origin (see Pot::diff).
  template <bool GENERAL = false>
  __device__ __forceinline__ void site(int mode, const T (&phj)[NF], const T (&D)[NF],
                                       const T (&pim)[NF], T (&pin)[NF], T* ps) const {
    if constexpr (PREC == PREC_FP64 && MODEL == M_CHAOTIC2) {
      // V = phi^2 (m2 + g2 chi^2)/2; the kicks with kV folded into the products,
      // and 2V accumulated (halved once, in post_stage): 4 DMUL + 6 DFMA
      const double ph2 = phj[0] * phj[0];
      const double t = fma(pk.g2, phj[1] * phj[1], pk.m2);      // m2 + g2 chi^2
      if (mode == MODE_SWEEP) {
        pin[0] = madd(kD, D[0], madd(-kV * phj[0], t, pim[0]));   // - kV phi (m2 + g2 chi^2)
        pin[1] = madd(kD, D[1], madd(nkVg * ph2, phj[1], pim[1]));   // - kV g2 phi^2 chi
      }
#pragma unroll
      for (int f = 0; f < NF; ++f) {
        if (mode == MODE_SWEEP) {
          ps[SL::PI2 + f] = madd(pin[f], pin[f], ps[SL::PI2 + f]);
        } else {
          pin[f] = pim[f];
          ps[SL::PI2 + f] = madd(pim[f], pim[f], ps[SL::PI2 + f]);
          const T dd = phj[f] - shiftK[f];
          ps[SL::DPHI + f] += dd;
          ps[SL::DPHI2 + f] = madd(dd, dd, ps[SL::DPHI2 + f]);
        }
        ps[SL::PHID + f] = madd(phj[f], D[f], ps[SL::PHID + f]);
      }
      ps[SL::V] = madd(ph2, t, ps[SL::V]);
    } else if constexpr (PREC == PREC_FP64 && MODEL == M_QBALL) {
      // V'_i = fac phi_i and 2V from |Phi|^2 (Pot::fac_near: the logarithm
      // near the stage's reference value); the kicks as pi - (kV fac) phi_i,
      // and 2V accumulated (halved once, in post_stage)
      const double u2 = fma(phj[0], phj[0], phj[1] * phj[1]);
      double fac, V2;
      P::fac_near(pk, u2, q_inv, q_lref, fac, V2);
      if (mode == MODE_SWEEP) {
        const double kf = -kV * fac;
#pragma unroll
        for (int f = 0; f < NF; ++f) pin[f] = madd(kD, D[f], madd(kf, phj[f], pim[f]));
      }
#pragma unroll
      for (int f = 0; f < NF; ++f) {
        if (mode == MODE_SWEEP) {
          ps[SL::PI2 + f] = madd(pin[f], pin[f], ps[SL::PI2 + f]);
        } else {
          pin[f] = pim[f];
          ps[SL::PI2 + f] = madd(pim[f], pim[f], ps[SL::PI2 + f]);
          const T dd = phj[f] - shiftK[f];
          ps[SL::DPHI + f] += dd;
          ps[SL::DPHI2 + f] = madd(dd, dd, ps[SL::DPHI2 + f]);
        }
        ps[SL::PHID + f] = madd(phj[f], D[f], ps[SL::PHID + f]);
      }
      ps[SL::V] += V2;
    } else if constexpr (PREC == PREC_FP64) {
      double dV[NF], V;
      P::eval(pk, phj, dV, V);
#pragma unroll
      for (int f = 0; f < NF; ++f) {
        if (mode == MODE_SWEEP) {
          pin[f] = madd(kD, D[f], madd(-kV, (T)dV[f], pim[f]));
          ps[SL::PI2 + f] = madd(pin[f], pin[f], ps[SL::PI2 + f]);
        } else {
          pin[f] = pim[f];
          ps[SL::PI2 + f] = madd(pim[f], pim[f], ps[SL::PI2 + f]);
          const T dd = phj[f] - shiftK[f];
          ps[SL::DPHI + f] += dd;
          ps[SL::DPHI2 + f] = madd(dd, dd, ps[SL::DPHI2 + f]);
        }
        ps[SL::PHID + f] = madd(phj[f], D[f], ps[SL::PHID + f]);
      }
      ps[SL::V] += V;
    } else {
      float dVd[NF], dVv;
      if constexpr (MODEL == M_QBALL) P::template diff<GENERAL>(sk, phj, dVd, dVv);
      else P::diff(sk, phj, dVd, dVv);
#pragma unroll
      for (int f = 0; f < NF; ++f) {
        pin[f] = (mode == MODE_SWEEP) ? madd(kD, D[f], madd(-kV, dVd[f], pim[f])) : pim[f];
        ps[SL::DPI + f] += pin[f];
        ps[SL::DPI2 + f] = madd(pin[f], pin[f], ps[SL::DPI2 + f]);
        ps[SL::PHID + f] = madd(phj[f], D[f], ps[SL::PHID + f]);
        ps[SL::DPHI + f] += phj[f];
        if (mode != MODE_SWEEP)   // the variance is only reported at synchronised states
          ps[SL::DPHI2 + f] = madd(phj[f], phj[f], ps[SL::DPHI2 + f]);
      }
      ps[SL::V] += dVv;
    }
  }
};

// The kick and the per-site sums of the split-DD form (double-float
// fluctuations; the sums gather in running double-float accumulators).
template <int MODEL>
__device__ __forceinline__ void site_dd(const Ctx<MODEL, PREC_DD>& cx, int mode,
                                        const dd (&phj)[Pot<MODEL>::NF],
                                        const dd (&D)[Pot<MODEL>::NF],
                                        const dd (&pim)[Pot<MODEL>::NF],
                                        dd (&pin)[Pot<MODEL>::NF], DDAcc* acc) {
  constexpr int NF = Pot<MODEL>::NF;
  using SL = Slots<NF, PREC_DD>;
  dd dVd[NF], dVv;
  PotDD<MODEL>::diff(cx.sk, phj, dVd, dVv);
#pragma unroll
  for (int f = 0; f < NF; ++f) {
    pin[f] = (mode == MODE_SWEEP) ? dd_fma(cx.kD, D[f], dd_fma(-cx.kV, dVd[f], pim[f])) : pim[f];
    // a sweep's sum of the momentum fluctuations sets the re-centring shift
    // (exact bookkeeping for any value) and enters sum pi^2 only as
    // 2 pi0 sum dpi, a term first order in the fluctuations: high parts in
    // plain float (its rounding is below 1e-12 of sum pi^2); a flush's sum in
    // double-float
    if (mode == MODE_SWEEP) acc[SL::DPI + f].add_fast(pin[f].hi);
    else acc[SL::DPI + f].add(pin[f]);
    acc[SL::DPI2 + f].add_sqr(pin[f]);
    acc[SL::PHID + f].add_prod(phj[f], D[f]);
    if (mode == MODE_SWEEP) {
      // a sweep's sum of the fluctuations only sets the re-centring shift,
      // which moves into the background exactly as it leaves the
      // fluctuations: any value of it is exact bookkeeping
      acc[SL::DPHI + f].add_fast(phj[f].hi);
    } else {  // a flush's sums give the field's mean and variance: double-float
      acc[SL::DPHI + f].add(phj[f]);
      acc[SL::DPHI2 + f].add_sqr(phj[f]);
    }
  }
  acc[SL::V].add(dVv);
}

// Error-free addition of float pairs (hi, lo): TwoSum on the high parts.
__device__ __forceinline__ void pair_add(float& hi, float& lo, float bh, float bl) {
  const float s = hi + bh;
  const float bp = s - hi;
  const float err = (hi - (s - bp)) + (bh - bp);
  lo = (lo + bl) + err;
  hi = s;
}

// Block sums of the float path without the FP64 pipe in the hot part: each
// thread's Kahan pair (s, -c) goes through a warp butterfly of float pairs;
// lane 0 of each warp widens its pair to one double; NQ threads add the 8
// warps in order.  Result in out[0..NQ) (shared).
template <int NQ>
__device__ __forceinline__ void block_sum_pairs(const Acc<float>* acc, double* sred,
                                                double* out) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int q = 0; q < NQ; ++q) {
    float hi = acc[q].s, lo = -acc[q].c;
#pragma unroll
    for (int m = 16; m >= 1; m >>= 1) {
      const float bh = __shfl_xor_sync(0xffffffffu, hi, m);
      const float bl = __shfl_xor_sync(0xffffffffu, lo, m);
      pair_add(hi, lo, bh, bl);
    }
    if (lane == 0) sred[warp * NQ + q] = (double)hi + (double)lo;
  }
  __syncthreads();
  if (threadIdx.x < NQ) {
    double s = 0.0;
#pragma unroll
    for (int w = 0; w < kThreads / 32; ++w) s += sred[w * NQ + threadIdx.x];
    out[threadIdx.x] = s;
  }
  __syncthreads();
}

// Block sums of a kernel: float64 butterfly for the FP64 form (per-thread
// double sums), float pairs for the split form.
template <int PREC, int NQ, typename T>
__device__ __forceinline__ void block_partials(const Acc<T>* acc, const T* accd_s, double* sred,
                                               double* sout) {
  __syncthreads();
  if constexpr (PREC == PREC_FP64) {
    double v[NQ];
#pragma unroll
    for (int q = 0; q < NQ; ++q) v[q] = (double)accd_s[q];
    block_sum<NQ>(v, sred, sout);
  } else {
    block_sum_pairs<NQ>(reinterpret_cast<const Acc<float>*>(acc), sred, sout);
  }
}

// ---------------------------------------------------------------------------
// Fixed-order fold of P rows of NQ doubles (row r at src[r * kNQ + q]) into
// out[0..NQ) (shared), by the whole block.  Warp w folds quantities w and
// w + 8: lane k sums rows k, k + 32, k + 64, ... in that order, then a
// shuffle tree adds lane k + h into k for h = 16, 8, 4, 2, 1.  The order
// depends on P alone.  No shared-memory levels or block barriers: on GB300 a
// dependent FP64 add costs ~60 cycles, so the fold is latency-bound.
// ---------------------------------------------------------------------------
template <int NQ>
__device__ __forceinline__ void fold_rows(const double* src, int P, double* out) {
  static_assert(NQ <= 2 * (kThreads / 32), "two quantities per warp at most");
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int q0 = warp, q1 = warp + kThreads / 32;
  double s0 = 0.0, s1 = 0.0;
  for (int r = lane; r < P; r += 32) {
    if (q0 < NQ) s0 += __ldcg(&src[(size_t)r * kNQ + q0]);
    if (q1 < NQ) s1 += __ldcg(&src[(size_t)r * kNQ + q1]);
  }
#pragma unroll
  for (int h = 16; h >= 1; h >>= 1) {
    s0 += __shfl_down_sync(0xffffffffu, s0, h);
    s1 += __shfl_down_sync(0xffffffffu, s1, h);
  }
  if (lane == 0) {
    if (q0 < NQ) out[q0] = s0;
    if (q1 < NQ) out[q1] = s1;
  }
  __syncthreads();
}

// ---------------------------------------------------------------------------
// Scalars between stages.
// ---------------------------------------------------------------------------
// The coefficients that turn a stage's reduced slots into lattice sums and
// the p_a kick; they depend only on the stage's Ctx, so a caller can form
// them before the sums arrive.
template <int NF> struct SumCoef {
  double ka, kb, pa;         // Phi_H3: p_a += ka sum phi D + kb sum V
  double spi[NF], tpi[NF];   // split form: S pi0s and 2 pi0s
};

template <int MODEL, int PREC, typename C>
__device__ __forceinline__ SumCoef<C::NF> sum_coef(const C& cx, const SimDesc& d) {
  SumCoef<C::NF> q;
  // Phi_H3(h): p_a += h a^3 [sum phi D/(a^2 dx^2) - 4 sum V]   (Eq. split-Phi)
  const double a = cx.k.a, h = cx.k.h;
  q.ka = (h * a) * d.dx2inv;
  q.kb = -4.0 * (h * ((a * a) * a));
  q.pa = cx.k.pa;
#pragma unroll
  for (int f = 0; f < C::NF; ++f) {
    q.spi[f] = (PREC != PREC_FP64) ? (double)d.S * cx.pi0s[f] : 0.0;
    q.tpi[f] = (PREC != PREC_FP64) ? 2.0 * cx.pi0s[f] : 0.0;
  }
  return q;
}

template <int NF>
__device__ __forceinline__ double pa_kick(const SumCoef<NF>& q, double sum_phiD, double sum_V) {
  return fma(q.ka, sum_phiD, fma(q.kb, sum_V, q.pa));
}

// Lattice sums of a stage from its reduced slots (NQ doubles, Slots<NF, PREC>):
// per field sum pi^2, sum phi D, sum (phi - K), sum (phi - K)^2, and sum V.
template <int MODEL, int PREC, typename C>
__device__ __forceinline__ void stage_sums(const C& cx, const SumCoef<C::NF>& q,
                                           const SimDesc& d, int mode, const double* sout,
                                           double* fpi2, double* fphiD, double* fdphi,
                                           double* fdphi2, double& sum_pi2, double& sum_phiD,
                                           double& sum_V) {
  using SL = typename C::SL;
  constexpr int NF = C::NF;
  if constexpr (PREC == PREC_FP64) {
#pragma unroll
    for (int f = 0; f < NF; ++f) {
      fpi2[f] = sout[SL::PI2 + f];
      fphiD[f] = sout[SL::PHID + f];
      fdphi[f] = (mode == MODE_FLUSH) ? sout[SL::DPHI + f] : 0.0;
      fdphi2[f] = (mode == MODE_FLUSH) ? sout[SL::DPHI2 + f] : 0.0;
    }
    // the chaotic and Q-ball models' FP64 sites accumulate 2V (see Ctx::site)
    sum_V = (MODEL == M_CHAOTIC2 || MODEL == M_QBALL) ? 0.5 * sout[SL::V] : sout[SL::V];
  } else {
#pragma unroll
    for (int f = 0; f < NF; ++f) {
      // sum (pi0 + dpi)^2 = S pi0^2 + 2 pi0 sum dpi + sum dpi^2
      fpi2[f] = fma(q.spi[f], cx.pi0s[f], fma(q.tpi[f], sout[SL::DPI + f], sout[SL::DPI2 + f]));
      fphiD[f] = sout[SL::PHID + f];  // sum (phi0 + d) D[d] = sum d D[d]  (sum D = 0)
      fdphi[f] = sout[SL::DPHI + f];
      fdphi2[f] = sout[SL::DPHI2 + f];
    }
    sum_V = fma((double)d.S, cx.V0, sout[SL::V]);  // sum V = S V(phi0) + sum dV
  }
  sum_pi2 = fpi2[0];
  sum_phiD = fphiD[0];
#pragma unroll
  for (int f = 1; f < NF; ++f) { sum_pi2 += fpi2[f]; sum_phiD += fphiD[f]; }
}

// ---------------------------------------------------------------------------
// Background update after a stage, from the stage's lattice sums `sout`
// (NQ doubles, slot layout Slots<NF, PREC>): the p_a kick of Phi_H3 (Eq.
// split-Phi) and the stage/step counters for a sweep; the H = 0 root (Eq. H2),
// the synchronised sums and the field statistics for a flush.  Shared by the
// per-launch kernels (last block) and the persistent kernel.
// ---------------------------------------------------------------------------
template <int MODEL, int PREC, typename C>
__device__ __forceinline__ void post_stage(const C& cx, const SumCoef<C::NF>& q,
                                           const SimDesc& d, int mode, const double* sout,
                                           const Background& bg, Background& nb) {
  using SL = typename C::SL;
  constexpr int NF = C::NF;
  nb = bg;
  double sum_pi2, sum_phiD, sum_V;
  double fpi2[NF], fphiD[NF], fdphi[NF], fdphi2[NF];
  stage_sums<MODEL, PREC>(cx, q, d, mode, sout, fpi2, fphiD, fdphi, fdphi2, sum_pi2, sum_phiD,
                          sum_V);

  const Coef& k = cx.k;
  double a = k.a, pa = k.pa;
  bool ok = is_fin(sum_pi2) && is_fin(sum_phiD) && is_fin(sum_V);
  if (mode == MODE_SWEEP) {
    pa = pa_kick(q, sum_phiD, sum_V);
    nb.eta = bg.eta + k.h;
    nb.h_prev = k.h;
    nb.deta = k.deta;
    nb.stage = bg.stage + 1;
    if (nb.stage >= d.nstages) { nb.stage = 0; nb.steps_done = bg.steps_done + 1; }
    nb.sweeps_done = bg.sweeps_done + 1;
    nb.sweeps_left = bg.sweeps_left - 1;
    nb.mode = nb.sweeps_left > 0 ? MODE_SWEEP : MODE_FLUSH;
    nb.cur = bg.cur ^ 3;
  } else {
    if (bg.init_pa) {
      // H = 0 (Eq. H2): p_a^2/(12 V_L m^2) = sum pi^2/(2a^2) - a^2 sum phiD/(2dx^2) + a^4 sum V
      //                                      + V_L rho_r + a V_L rho_m
      const double E = sum_pi2 / (2.0 * a * a) - 0.5 * a * a * sum_phiD * d.dx2inv +
                       (a * a) * (a * a) * sum_V + d.VL * d.rho_r0 + a * d.VL * d.rho_m0;
      pa = (d.inv6VLm2 == 0.0) ? 0.0 : -sqrt(12.0 * d.VL * d.mpl2 * E);
      nb.init_pa = 0;
    }
    nb.h_prev = 0.0;
    nb.mode = MODE_IDLE;
    nb.cur = bg.cur ^ 1;
#pragma unroll
    for (int f = 0; f < NF; ++f) {
      nb.s_pi2[f] = fpi2[f];
      nb.s_phiD[f] = fphiD[f];
      // shifted-data mean and variance: K = the flush's shift (FP64) or phi0 (split)
      const double K = (PREC == PREC_FP64) ? (double)cx.shiftK[f] : cx.phi0s[f];
      const double m1 = fdphi[f] * d.invS;
      nb.mean[f] = K + m1;
      nb.var[f] = fma(fdphi2[f], d.invS, -m1 * m1);
      ok = ok && is_fin(fdphi[f]) && is_fin(fdphi2[f]);
    }
    nb.s_V = sum_V;
  }
  nb.a = a;
  nb.pa = pa;
  nb.sum_pi2 = sum_pi2;
  if constexpr (PREC != PREC_FP64) {
#pragma unroll
    for (int f = 0; f < NF; ++f) {
      nb.phi0[f] = cx.phi0s[f];
      nb.mu_phi[f] = fdphi[f] * d.invS;
      if (mode == MODE_SWEEP) {
        nb.pi0[f] = cx.pi0s[f];
        nb.mu_pi[f] = sout[SL::DPI + f] * d.invS;
      }
      ok = ok && is_fin(cx.phi0s[f]) && is_fin(cx.pi0s[f]);
    }
  }
  ok = ok && is_fin(a) && is_fin(pa);
  if (!ok) {
    nb.error = 1;
    nb.mode = MODE_IDLE;
  }
}

template <int MODEL, int PREC, typename C>
__device__ __forceinline__ void post_stage(const C& cx, const SimDesc& d, int mode,
                                           const double* sout, const Background& bg,
                                           Background& nb) {
  post_stage<MODEL, PREC>(cx, sum_coef<MODEL, PREC>(cx, d), d, mode, sout, bg, nb);
}

// The next stage's Ctx from this SWEEP stage's reduced slots, in the pieces
// that a stage boundary can run on different threads; together they give
// exactly what post_stage followed by Ctx::init gives.
//   chain_coef: sum pi^2, sum phi D, sum V -> p_a kick -> the next stage's
//     scalar half-steps (qn: prestage_a of the next stage, formed early)
template <int MODEL, int PREC, typename C>
__device__ __forceinline__ Coef chain_coef(const C& cx, const SumCoef<C::NF>& q,
                                           const PreCoef& qn, const SimDesc& d,
                                           const double* sout, int mode_next) {
  constexpr int NF = C::NF;
  double sum_pi2, sum_phiD, sum_V;
  double fpi2[NF], fphiD[NF], fdphi[NF], fdphi2[NF];
  stage_sums<MODEL, PREC>(cx, q, d, MODE_SWEEP, sout, fpi2, fphiD, fdphi, fdphi2, sum_pi2,
                          sum_phiD, sum_V);
  return prestage_p(qn, pa_kick(q, sum_phiD, sum_V), sum_pi2, mode_next);
}
//   chain_means (split form): the re-centring shifts of the next stage
//     (post_stage's mu_phi, mu_pi) and the background they move into
template <int PREC, typename C>
__device__ __forceinline__ void chain_means(const C& cx, const SimDesc& d, const double* sout,
                                            double* mphi, double* mpi) {
  using SL = typename C::SL;
#pragma unroll
  for (int f = 0; f < C::NF; ++f) {
    mphi[f] = sout[SL::DPHI + f] * d.invS;
    mpi[f] = sout[SL::DPI + f] * d.invS;
  }
}

// Ticket increment with acquire-release semantics at GPU scope: it publishes
// the caller's earlier stores (the row it wrote) and, for the block that takes
// the last ticket, makes every other block's row visible.
__device__ __forceinline__ unsigned int ticket_add(unsigned int* p) {
  unsigned int old;
  asm volatile("atom.acq_rel.gpu.global.add.u32 %0, [%1], 1;" : "=r"(old) : "l"(p) : "memory");
  return old;
}

// ---------------------------------------------------------------------------
// Block finish: partials, tickets, and (last block) the background update.
// sout holds this block's NQ sums on entry.  Two levels, so that almost all
// of the fold overlaps the sweep: the last block of each group of kGroup
// consecutive blocks folds the group's rows into one group row; the last group
// to finish folds the group rows and advances the background.  Thread 0 writes
// each row and takes the ticket; the block barrier after it orders the other
// threads' reads of the rows.
// ---------------------------------------------------------------------------
template <int MODEL, int PREC, typename C>
__device__ __forceinline__ void finish_block(const C& cx, const SimDesc& d, int mode, int cta,
                                             double* sout, int* s_last) {
  using SL = typename C::SL;
  constexpr int NF = C::NF;
  constexpr int NQ = SL::NQ;
  const int tid = threadIdx.x;
  const int g = cta / kGroup;
  const int g0 = g * kGroup;
  const int gn = min(kGroup, d.ncta - g0);
  if (tid == 0) {
#pragma unroll
    for (int q = 0; q < NQ; ++q) d.partials[(size_t)cta * kNQ + q] = sout[q];
    *s_last = (ticket_add(&d.gticket[g]) == (unsigned int)(gn - 1));
  }
  __syncthreads();
  if (!*s_last) return;

  // ---- last block of group g: fold the group's rows ------------------------
  fold_rows<NQ>(d.partials + (size_t)g0 * kNQ, gn, sout);
  if (tid == 0) {
    d.gticket[g] = 0u;  // every block of the group has counted
#pragma unroll
    for (int q = 0; q < NQ; ++q) d.gpartials[(size_t)g * kNQ + q] = sout[q];
    *s_last = (ticket_add(d.ticket) == (unsigned int)(d.ngroups - 1));
  }
  __syncthreads();
  if (!*s_last) return;

  // ---- last group: fold the group rows, then the background update ---------
  fold_rows<NQ>(d.gpartials, d.ngroups, sout);
  if (tid != 0) return;

  Background* bgp = d.bg;
  Background nb;
  post_stage<MODEL, PREC>(cx, d, mode, sout, *bgp, nb);
  *bgp = nb;  // published to the next launch by the kernel boundary
  *d.ticket = 0u;
}

__device__ __forceinline__ int member_of(const LaunchTable& tab, int b) {
  int lo = 0, hi = tab.count - 1;
  while (lo < hi) {  // largest m with cta_offset[m] <= b
    const int mid = (lo + hi + 1) >> 1;
    if (tab.cta_offset[mid] <= b) lo = mid; else hi = mid - 1;
  }
  return lo;
}

__device__ __forceinline__ int wrapi(int v, int n) { return v < 0 ? v + n : (v >= n ? v - n : v); }

// ---------------------------------------------------------------------------
// TMA / mbarrier primitives (inline PTX, sm_90+).
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count)
               : "memory");
}
__device__ __forceinline__ void fence_mbar_init() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)),
               "r"(bytes)
               : "memory");
}
__device__ __forceinline__ bool mbar_try(uint64_t* bar, uint32_t parity) {
  uint32_t done;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
      " selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(done)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return done != 0;
}
// Bounded wait: gives up after `limit` clocks and reports it.
// (try_wait itself suspends the thread for a while; the clock is read only
// every 32 polls so that a waiting warp issues few instructions.)
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity,
                                          long long limit = kWaitLimit) {
  if (mbar_try(bar, parity)) return true;
  const long long t0 = clock64();
  for (uint32_t i = 1;; ++i) {
    if (mbar_try(bar, parity)) return true;
    if ((i & 31u) == 0u && clock64() - t0 > limit) return false;
  }
}
__device__ __forceinline__ void fence_proxy_async() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}
__device__ __forceinline__ void tensormap_acquire(const void* map) {
  asm volatile("fence.proxy.tensormap::generic.acquire.gpu [%0], 128;" ::"l"(map) : "memory");
}
__device__ __forceinline__ void tma_load_3d(void* dst, const CUtensorMap* map, int x, int y, int z,
                                            uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%2, %3, %4}], [%5];" ::"r"(smem_u32(dst)),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(z), "r"(smem_u32(bar))
      : "memory");
}

template <int STENCIL> struct StencilW {
  static constexpr bool kCorners = (STENCIL == 27);
};

// ---------------------------------------------------------------------------
// TMA-staged sweep (n % 32 == 0).  256 threads = 8 warps; warp w owns tile row
// y0 + w, lane l owns sites x0 + l*VX .. +VX-1.
// ---------------------------------------------------------------------------
template <int MODEL, int STENCIL, int PREC, int VX>
__global__ void __launch_bounds__(kThreads, 2) sweep_tma(const LaunchTable tab) {
  using C = Ctx<MODEL, PREC>;
  using T = typename C::T;
  using SL = typename C::SL;
  constexpr int NF = C::NF;
  constexpr int NQ = SL::NQ;
  constexpr bool CORNERS = StencilW<STENCIL>::kCorners;
  constexpr int TY = kMaxTY;          // 8 rows, one per warp
  constexpr int TX = 32 * VX;         // tile width
  constexpr int ROWS = TY + 2;        // with the two halo rows
  constexpr int NSLOT = 3;
  constexpr uint32_t kPlaneBytes = 2u * NF * ROWS * TX * sizeof(T);

  __shared__ __align__(128) T stage[NSLOT][2][NF][ROWS][TX];   // [slot][phi/pi][f][row][x]
  __shared__ T colb[NSLOT][NF][2][ROWS];                        // halo columns x0-1, x0+TX
  __shared__ __align__(8) uint64_t mbar[NSLOT];
  __shared__ double sred[(kThreads / 32) * NQ];
  __shared__ double sout[NQ];
  __shared__ int s_last, s_fault;

  const int mem = member_of(tab, blockIdx.x);
  const SimDesc& d = *tab.desc[mem];
  const int cta = blockIdx.x - tab.cta_offset[mem];
  const Background& bgr = *d.bg;
  const int mode = bgr.mode;
  if (mode == MODE_IDLE) return;

  const int n = d.n;
  const int tile = cta % (d.tiles_x * d.tiles_y);
  const int zch = cta / (d.tiles_x * d.tiles_y);
  const int x0 = (tile % d.tiles_x) * TX;
  const int y0 = (tile / d.tiles_x) * TY;
  const int z0 = zch * d.zc;
  const int zend = min(n, z0 + d.zc);
  const int Q = zend - z0 + 2;                 // planes z0-1 .. zend
  const int tid = threadIdx.x;
  const int lane = tid & 31, ly = tid >> 5;
  const int gx = x0 + lane * VX, gy = y0 + ly;
  const size_t S = (size_t)d.S;
  const size_t nn = (size_t)n * n;

  __shared__ C s_ctx;   // scalar context: computed once, by one thread (FP64 pipe is scarce)
  const int ib = bgr.cur;  // bit0: phi buffer, bit1: pi buffer
  const T* __restrict__ phi_in = (const T*)d.phi[ib & 1];
  T* __restrict__ phi_out = (T*)d.phi[(ib & 1) ^ 1];
  const T* __restrict__ pi_in = (const T*)d.pi[(ib >> 1) & 1];
  T* __restrict__ pi_out = (T*)d.pi[((ib >> 1) & 1) ^ 1];
  const CUtensorMap* tphi_main = &d.tmap[ib & 1][0];
  const CUtensorMap* tphi_row = &d.tmap[ib & 1][1];
  const CUtensorMap* tpi_main = &d.tmap[2 + ((ib >> 1) & 1)][0];
  const CUtensorMap* tpi_row = &d.tmap[2 + ((ib >> 1) & 1)][1];
  const int yl = wrapi(y0 - 1, n), yh = wrapi(y0 + TY, n);

  // stencil weights (Eq. D): 7pt (-6, 1, 0, 0); iso27 (-128, 14, 3, 1)/30
  const T c0 = CORNERS ? (T)(-128.0 / 30.0) : (T)(-6.0);
  const T c1 = CORNERS ? (T)(14.0 / 30.0) : (T)1.0;
  const T c2 = CORNERS ? (T)(3.0 / 30.0) : (T)0.0;
  const T c3 = CORNERS ? (T)(1.0 / 30.0) : (T)0.0;

  // halo columns: threads [64, 64 + 2 ROWS): side = left/right, row = y0-1 .. y0+TY
  const bool hcol = tid >= 64 && tid < 64 + 2 * ROWS;
  int hc_side = 0, hc_row = 0;
  size_t hc_off = 0;
  if (hcol) {
    const int t = tid - 64;
    hc_side = t / ROWS;
    hc_row = t % ROWS;
    const int xx = hc_side == 0 ? wrapi(x0 - 1, n) : wrapi(x0 + TX, n);
    const int yy = wrapi(y0 - 1 + hc_row, n);
    hc_off = (size_t)yy * n + xx;
  }
  T sp[NF], sq[NF];
#pragma unroll
  for (int f = 0; f < NF; ++f) { sp[f] = 0; sq[f] = 0; }
  auto load_col = [&](int p) {
    if (hcol) {
      const size_t o = (size_t)wrapi(p, n) * nn + hc_off;
#pragma unroll
      for (int f = 0; f < NF; ++f) { sp[f] = phi_in[f * S + o]; sq[f] = pi_in[f * S + o]; }
    }
  };
  auto issue = [&](int q) {  // one thread: all TMA copies of plane z0 - 1 + q
    const int s = q % NSLOT;
    const int zw = wrapi(z0 - 1 + q, n);
    mbar_expect_tx(&mbar[s], kPlaneBytes);
#pragma unroll
    for (int f = 0; f < NF; ++f) {
      const int zz = f * n + zw;
      tma_load_3d(&stage[s][0][f][1][0], tphi_main, x0, y0, zz, &mbar[s]);
      tma_load_3d(&stage[s][0][f][0][0], tphi_row, x0, yl, zz, &mbar[s]);
      tma_load_3d(&stage[s][0][f][ROWS - 1][0], tphi_row, x0, yh, zz, &mbar[s]);
      tma_load_3d(&stage[s][1][f][1][0], tpi_main, x0, y0, zz, &mbar[s]);
      tma_load_3d(&stage[s][1][f][0][0], tpi_row, x0, yl, zz, &mbar[s]);
      tma_load_3d(&stage[s][1][f][ROWS - 1][0], tpi_row, x0, yh, zz, &mbar[s]);
    }
  };

  if (tid == 0) {
    for (int s = 0; s < NSLOT; ++s) mbar_init(&mbar[s], 1);
    fence_mbar_init();
    tensormap_acquire(tphi_main);
    tensormap_acquire(tphi_row);
    tensormap_acquire(tpi_main);
    tensormap_acquire(tpi_row);
    s_fault = 0;
  }
  __syncthreads();
  if (tid == 0) {
    issue(0);
    if (Q > 1) issue(1);
  } else if (tid == 32) {
    s_ctx.init(bgr, d, mode);  // while the first planes are in flight
  }
  load_col(z0 - 1);
  __syncthreads();
  const C cx = s_ctx;

  Acc<T> acc[NQ];
  T accd_s[NQ];   // float64 path: plain per-thread sums
#pragma unroll
  for (int q = 0; q < NQ; ++q) { acc[q].zero(); accd_s[q] = (T)0; }
  // rotating registers: part_m = S_off(z-1) + S_mid(z) of the plane z = p - 1
  // awaiting output; so_m = S_off(p - 1) (iso27 only; it is phi* for 7pt);
  // ph_m / pi_m = drifted phi and (re-centred) momentum of plane p - 1.
  T part_m[NF][VX], so_m[NF][VX], ph_m[NF][VX], pi_m[NF][VX];
#pragma unroll
  for (int f = 0; f < NF; ++f)
#pragma unroll
    for (int j = 0; j < VX; ++j) part_m[f][j] = so_m[f][j] = ph_m[f][j] = pi_m[f][j] = (T)0;

  int q = 0;
  for (; q < Q; ++q) {
    const int s = q % NSLOT;
    const int p = z0 - 1 + q;
    if (!mbar_wait(&mbar[s], (uint32_t)((q / NSLOT) & 1))) atomicOr(&s_fault, 1);

    // drift this plane in place: phi* = phi + c pi (re-centred in the split form)
    T cur_ph[NF][VX], cur_pi[NF][VX];
#pragma unroll
    for (int f = 0; f < NF; ++f) {
      T ph[VX], pv[VX];
      vload<T, VX>(&stage[s][0][f][ly + 1][lane * VX], ph);
      vload<T, VX>(&stage[s][1][f][ly + 1][lane * VX], pv);
#pragma unroll
      for (int j = 0; j < VX; ++j) {
        if constexpr (PREC == PREC_SPLIT) { ph[j] -= cx.mu_phi[f]; pv[j] -= cx.mu_pi[f]; }
        cur_pi[f][j] = pv[j];
        cur_ph[f][j] = madd(cx.cdrift, pv[j], ph[j]);
      }
      vstore<T, VX>(&stage[s][0][f][ly + 1][lane * VX], cur_ph[f]);
    }
    if (tid < 64) {  // the two halo rows
      const int r = tid < 32 ? 0 : ROWS - 1;
#pragma unroll
      for (int f = 0; f < NF; ++f) {
        T ph[VX], pv[VX];
        vload<T, VX>(&stage[s][0][f][r][lane * VX], ph);
        vload<T, VX>(&stage[s][1][f][r][lane * VX], pv);
#pragma unroll
        for (int j = 0; j < VX; ++j) {
          if constexpr (PREC == PREC_SPLIT) { ph[j] -= cx.mu_phi[f]; pv[j] -= cx.mu_pi[f]; }
          ph[j] = madd(cx.cdrift, pv[j], ph[j]);
        }
        vstore<T, VX>(&stage[s][0][f][r][lane * VX], ph);
      }
    } else if (hcol) {  // the two halo columns
#pragma unroll
      for (int f = 0; f < NF; ++f) {
        T ph = sp[f], pv = sq[f];
        if constexpr (PREC == PREC_SPLIT) { ph -= cx.mu_phi[f]; pv -= cx.mu_pi[f]; }
        colb[s][f][hc_side][hc_row] = madd(cx.cdrift, pv, ph);
      }
      if (q + 1 < Q) load_col(p + 1);
    }
    // every thread's generic reads and writes of the slot recycled below come
    // before the TMA copy (async proxy) that refills it: a proxy fence by each
    // thread, then the block barrier
    fence_proxy_async();
    __syncthreads();
    if (s_fault) break;
    if (tid == 0 && q + 2 < Q) issue(q + 2);

    T so_new[NF][VX], smid_new[NF][VX];   // S_off(p), S_mid(p)
#pragma unroll
    for (int f = 0; f < NF; ++f) {
      T dn[VX], up[VX];
      vload<T, VX>(&stage[s][0][f][ly][lane * VX], dn);
      vload<T, VX>(&stage[s][0][f][ly + 2][lane * VX], up);
      T left = __shfl_up_sync(0xffffffffu, cur_ph[f][VX - 1], 1);
      T right = __shfl_down_sync(0xffffffffu, cur_ph[f][0], 1);
      if (lane == 0) left = colb[s][f][0][ly + 1];
      if (lane == 31) right = colb[s][f][1][ly + 1];
      T dl = 0, dr = 0, ul = 0, ur = 0;
      if constexpr (CORNERS) {
        dl = __shfl_up_sync(0xffffffffu, dn[VX - 1], 1);
        dr = __shfl_down_sync(0xffffffffu, dn[0], 1);
        ul = __shfl_up_sync(0xffffffffu, up[VX - 1], 1);
        ur = __shfl_down_sync(0xffffffffu, up[0], 1);
        if (lane == 0) { dl = colb[s][f][0][ly]; ul = colb[s][f][0][ly + 2]; }
        if (lane == 31) { dr = colb[s][f][1][ly]; ur = colb[s][f][1][ly + 2]; }
      }
#pragma unroll
      for (int j = 0; j < VX; ++j) {
        const T ctr = cur_ph[f][j];
        const T L = j > 0 ? cur_ph[f][j - 1] : left;
        const T R = j < VX - 1 ? cur_ph[f][j + 1] : right;
        const T faces = (dn[j] + up[j]) + (L + R);
        if constexpr (CORNERS) {
          const T DL = j > 0 ? dn[j - 1] : dl;
          const T DR = j < VX - 1 ? dn[j + 1] : dr;
          const T UL = j > 0 ? up[j - 1] : ul;
          const T UR = j < VX - 1 ? up[j + 1] : ur;
          const T corners = (DL + DR) + (UL + UR);
          smid_new[f][j] = madd(c2, corners, madd(c1, faces, c0 * ctr));
          so_new[f][j] = madd(c3, corners, madd(c2, faces, c1 * ctr));
        } else {
          smid_new[f][j] = madd(c0, ctr, faces);
          so_new[f][j] = ctr;
        }
      }
    }
    if (q >= 2) {  // output plane z = p - 1
      const size_t o = (size_t)(p - 1) * nn + (size_t)gy * n + gx;
      // float: per-plane partials then Kahan; double: straight into the accumulators
      T ps_local[NQ];
      T* ps = ps_local;
      if constexpr (PREC == PREC_FP64) {
        ps = accd_s;
      } else {
#pragma unroll
        for (int i = 0; i < NQ; ++i) ps_local[i] = (T)0;
      }
      T pin[NF][VX];
#pragma unroll
      for (int j = 0; j < VX; ++j) {
        T phj[NF], Dj[NF], pmj[NF], pnj[NF];
#pragma unroll
        for (int f = 0; f < NF; ++f) {
          phj[f] = ph_m[f][j];
          Dj[f] = part_m[f][j] + so_new[f][j];
          pmj[f] = pi_m[f][j];
        }
        cx.site(mode, phj, Dj, pmj, pnj, ps);
#pragma unroll
        for (int f = 0; f < NF; ++f) pin[f][j] = pnj[f];
      }
#pragma unroll
      for (int f = 0; f < NF; ++f) {
        vstore<T, VX>(phi_out + f * S + o, ph_m[f]);
        if (mode == MODE_SWEEP) vstore<T, VX>(pi_out + f * S + o, pin[f]);
      }
      if constexpr (PREC == PREC_SPLIT) {
#pragma unroll
        for (int i = 0; i < NQ; ++i) acc[i].add(ps_local[i]);
      }
    }
#pragma unroll
    for (int f = 0; f < NF; ++f)
#pragma unroll
      for (int j = 0; j < VX; ++j) {
        part_m[f][j] = (CORNERS ? so_m[f][j] : ph_m[f][j]) + smid_new[f][j];
        if constexpr (CORNERS) so_m[f][j] = so_new[f][j];
        ph_m[f][j] = cur_ph[f][j];
        pi_m[f][j] = cur_pi[f][j];
      }
  }

  if (s_fault) {
    // a TMA copy never completed: record it, drain what is in flight (bounded), stop
    if (tid == 0) {
      atomicOr(d.fault, 1);
      for (int r = q; r < Q && r < q + 2; ++r)
        mbar_wait(&mbar[r % NSLOT], (uint32_t)((r / NSLOT) & 1));
    }
    return;
  }
  block_partials<PREC, NQ, T>(acc, accd_s, sred, sout);
  finish_block<MODEL, PREC>(s_ctx, d, mode, cta, sout, &s_last);
}

__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}
// 4-byte asynchronous global -> shared copy.
__device__ __forceinline__ void cp_async4(void* dst, const void* src) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(smem_u32(dst)), "l"(src)
               : "memory");
}
// Arrive on `bar` once this thread's earlier cp.async copies have landed; the
// arrival counts toward the barrier's expected count (.noinc).
__device__ __forceinline__ void cp_async_arrive_noinc(uint64_t* bar) {
  asm volatile("cp.async.mbarrier.arrive.noinc.shared::cta.b64 [%0];" ::"r"(smem_u32(bar))
               : "memory");
}
// halo-column rows a lane needs: its own row (7-point) or three rows (iso-27)
#define CR_OF(corners) ((corners) ? 3 : 1)

// Depth of the split sweep's TMA ring: kPipeSlots slots, kPipeLead planes in
// flight ahead of the plane being computed (the slot being recycled was
// released kPipeSlots - kPipeLead planes earlier).  On GB300 the serving mix
// ran 1.8 % faster closed-loop with 8 slots / 5 in flight than with 6 / 4
// (two 85 KB blocks per SM).
constexpr int kPipeSlots = 8;
constexpr int kPipeLead = 5;

template <int NF, int VX>
constexpr size_t pipe_smem_bytes() {
  return sizeof(float) * (size_t)kPipeSlots * 2 * NF * (kMaxTY + 2) * 32 * VX;
}

// ---------------------------------------------------------------------------
// Split-FP32 sweep (n % 32 == 0): barrier-free warp pipeline.
//
// The float32 form is bound by HBM, so its sweep keeps every SM streaming:
//   - block b owns tile b mod T and z-chunk b / T, so blocks that run together
//     are neighbouring tiles at the same z and the halo rows they read hit L2
//     (a plane-balanced persistent grid with unaligned z-ranges was measured
//     to re-read ~60% more from DRAM);
//   - thread 0 keeps LEAD planes of TMA copies in flight in an NSLOT-deep ring
//     ("full" mbarriers, transaction-counted); each warp owns one tile row,
//     drifts the three rows it needs in registers (never written back),
//     releases the slot (one arrival per warp on the slot's "empty" mbarrier,
//     which thread 0 waits on before recycling it), and does the stencil, kick
//     and sums from registers; no block barrier in the z loop;
//   - lanes 0 and 31 fetch the two halo columns themselves, two planes ahead.
// ---------------------------------------------------------------------------
template <int MODEL, int STENCIL, int VX>
__global__ void __launch_bounds__(kThreads, 2) sweep_split_pipe(const LaunchTable tab) {
  constexpr int PREC = PREC_SPLIT;
  using C = Ctx<MODEL, PREC>;
  using SL = typename C::SL;
  constexpr int NF = C::NF;
  constexpr int NQ = SL::NQ;
  constexpr bool CORNERS = StencilW<STENCIL>::kCorners;
  constexpr int TY = kMaxTY;
  constexpr int TX = 32 * VX;
  constexpr int ROWS = TY + 2;
  constexpr int NWARP = kThreads / 32;
  constexpr int NSLOT = kPipeSlots, LEAD = kPipeLead;
  constexpr int NCOL = 2 * NF * 2 * ROWS;       // halo-column values per plane
  constexpr uint32_t kPlaneBytes = 2u * NF * ROWS * TX * sizeof(float);

  // the ring lives in dynamic shared memory (pipe_smem_bytes(), above the 48 KB static limit)
  extern __shared__ __align__(128) unsigned char pipe_smem[];
  auto& stage = *reinterpret_cast<float (*)[NSLOT][2][NF][ROWS][TX]>(pipe_smem);
  __shared__ float colb[NSLOT][2][NF][2][ROWS];   // [slot][phi/pi][f][left/right][row]
  __shared__ __align__(8) uint64_t full[NSLOT], empty[NSLOT];
  __shared__ double sred[(kThreads / 32) * NQ];
  __shared__ double sout[NQ];
  __shared__ int s_last, s_fault;
  __shared__ C s_ctx;

  const int mem = member_of(tab, blockIdx.x);
  const SimDesc& d = *tab.desc[mem];
  const int cta = blockIdx.x - tab.cta_offset[mem];
  const Background& bgr = *d.bg;
  const int mode = bgr.mode;
  if (mode == MODE_IDLE) return;

  const int n = d.n;
  const int tiles_x = d.tiles_x;
  const int tid = threadIdx.x;
  const int lane = tid & 31, ly = tid >> 5;
  const size_t S = (size_t)d.S;
  const size_t nn = (size_t)n * n;
  const int ib = bgr.cur;
  const float* __restrict__ phi_in = (const float*)d.phi[ib & 1];
  float* __restrict__ phi_out = (float*)d.phi[(ib & 1) ^ 1];
  const float* __restrict__ pi_in = (const float*)d.pi[(ib >> 1) & 1];
  float* __restrict__ pi_out = (float*)d.pi[((ib >> 1) & 1) ^ 1];
  const CUtensorMap* tphi_main = &d.tmap[ib & 1][0];
  const CUtensorMap* tphi_row = &d.tmap[ib & 1][1];
  const CUtensorMap* tpi_main = &d.tmap[2 + ((ib >> 1) & 1)][0];
  const CUtensorMap* tpi_row = &d.tmap[2 + ((ib >> 1) & 1)][1];

  // this block's tile and z-chunk: consecutive blocks are neighbouring tiles at
  // the same z, so the halo rows one block reads were just read by another (L2)
  const int tile = cta % (tiles_x * d.tiles_y);
  const int zch = cta / (tiles_x * d.tiles_y);
  const int x0 = (tile % tiles_x) * TX;
  const int y0 = (tile / tiles_x) * TY;
  const int z0 = zch * d.zc;
  const int Q = min(n, z0 + d.zc) - z0 + 2;   // planes z0 - 1 .. z1
  const int yl = wrapi(y0 - 1, n), yh = wrapi(y0 + TY, n);
  const int xl = wrapi(x0 - 1, n), xr = wrapi(x0 + TX, n);

  if (tid == 0) {
    for (int s = 0; s < NSLOT; ++s) {
      mbar_init(&full[s], 1 + 32);        // the TMA transaction + one warp of cp.async
      mbar_init(&empty[s], NWARP);
    }
    fence_mbar_init();
    s_fault = 0;
  }
  if (lane == 0) {
    tensormap_acquire(tphi_main);
    tensormap_acquire(tphi_row);
    tensormap_acquire(tpi_main);
    tensormap_acquire(tpi_row);
  }
  __syncthreads();
  const float c0 = CORNERS ? (float)(-128.0 / 30.0) : -6.0f;
  const float c1 = CORNERS ? (float)(14.0 / 30.0) : 1.0f;
  const float c2 = CORNERS ? (float)(3.0 / 30.0) : 0.0f;
  const float c3 = CORNERS ? (float)(1.0 / 30.0) : 0.0f;

  // Producer of plane q, run by every lane of warp q mod NWARP: lane 0 issues
  // the TMA copies of the tile and its two halo rows, all lanes copy the two
  // halo columns with cp.async; both complete on full[q mod NSLOT].
  auto produce = [&](int q) {
    const int s = q % NSLOT;
    const int zw = wrapi(z0 - 1 + q, n);
    const size_t zoff = (size_t)zw * nn;
    if (lane == 0) {
      mbar_expect_tx(&full[s], kPlaneBytes);
#pragma unroll
      for (int f = 0; f < NF; ++f) {
        const int zz = f * n + zw;
        tma_load_3d(&stage[s][0][f][1][0], tphi_main, x0, y0, zz, &full[s]);
        tma_load_3d(&stage[s][0][f][0][0], tphi_row, x0, yl, zz, &full[s]);
        tma_load_3d(&stage[s][0][f][ROWS - 1][0], tphi_row, x0, yh, zz, &full[s]);
        tma_load_3d(&stage[s][1][f][1][0], tpi_main, x0, y0, zz, &full[s]);
        tma_load_3d(&stage[s][1][f][0][0], tpi_row, x0, yl, zz, &full[s]);
        tma_load_3d(&stage[s][1][f][ROWS - 1][0], tpi_row, x0, yh, zz, &full[s]);
      }
    }
    for (int i = lane; i < NCOL; i += 32) {
      const int row = i % ROWS;
      const int side = (i / ROWS) & 1;
      const int f = (i / (2 * ROWS)) % NF;
      const int arr = i / (2 * ROWS * NF);
      const size_t off = zoff + (size_t)wrapi(y0 - 1 + row, n) * n + (side ? xr : xl);
      cp_async4(&colb[s][arr][f][side][row], (arr ? pi_in : phi_in) + f * S + off);
    }
    cp_async_arrive_noinc(&full[s]);
  };
  static_assert(LEAD < NWARP, "the last warp must not produce the first planes");
  for (int q = ly; q < LEAD && q < Q; q += NWARP) produce(q);
  if (tid == kThreads - 32) s_ctx.init(bgr, d, mode);  // while the first planes are in flight
  __syncthreads();
  const C cx = s_ctx;
  // re-centring of the output: phi* = phi + c pi - (mu_phi + c mu_pi); the
  // stencil works on phi + c pi (D of a constant is zero)
  float Mf[NF];
#pragma unroll
  for (int f = 0; f < NF; ++f) Mf[f] = madd(cx.cdrift, cx.mu_pi[f], cx.mu_phi[f]);

  Acc<float> acc[NQ];
#pragma unroll
  for (int i = 0; i < NQ; ++i) acc[i].zero();
  // rotating registers: part_m = S_off(z-1) + S_mid(z) of the plane z = p - 1
  // awaiting output; so_m = S_off(p - 1) (iso27); ph_m / pi_m = drifted field
  // (not re-centred) and re-centred momentum of plane p - 1
  float part_m[NF][VX], so_m[NF][VX], ph_m[NF][VX], pi_m[NF][VX];
#pragma unroll
  for (int f = 0; f < NF; ++f)
#pragma unroll
    for (int j = 0; j < VX; ++j) part_m[f][j] = so_m[f][j] = ph_m[f][j] = pi_m[f][j] = 0.f;

  int q = 0;
  for (; q < Q; ++q) {
    const int s = q % NSLOT;
    const int p = z0 - 1 + q;
    // the producer role rotates over the warps: plane q + LEAD, once every warp
    // has released the slot's previous plane (q + LEAD - NSLOT)
    const int qn = q + LEAD;
    bool ok = true;
    if (qn < Q && qn % NWARP == ly) {
      const int rr = qn - NSLOT;
      if (rr >= 0) ok = mbar_wait(&empty[rr % NSLOT], (uint32_t)((rr / NSLOT) & 1));
      if (__all_sync(0xffffffffu, ok)) produce(qn);
    }
    ok = ok && mbar_wait(&full[s], (uint32_t)((q / NSLOT) & 1));
    // every exit decision is taken by the whole warp (shuffles and __syncwarp follow)
    if (!__all_sync(0xffffffffu, ok)) {
      if (lane == 0) atomicOr(&s_fault, 1);
      break;
    }
    // the three rows this warp needs, drifted in registers (not written back)
    float cur_ph[NF][VX], cur_pi[NF][VX], dn[NF][VX], up[NF][VX];
#pragma unroll
    for (int f = 0; f < NF; ++f) {
      float a[VX], b[VX];
      vload<float, VX>(&stage[s][0][f][ly + 1][lane * VX], a);
      vload<float, VX>(&stage[s][1][f][ly + 1][lane * VX], b);
#pragma unroll
      for (int j = 0; j < VX; ++j) {
        cur_pi[f][j] = b[j] - cx.mu_pi[f];
        cur_ph[f][j] = madd(cx.cdrift, b[j], a[j]);
      }
      vload<float, VX>(&stage[s][0][f][ly][lane * VX], a);
      vload<float, VX>(&stage[s][1][f][ly][lane * VX], b);
#pragma unroll
      for (int j = 0; j < VX; ++j) dn[f][j] = madd(cx.cdrift, b[j], a[j]);
      vload<float, VX>(&stage[s][0][f][ly + 2][lane * VX], a);
      vload<float, VX>(&stage[s][1][f][ly + 2][lane * VX], b);
#pragma unroll
      for (int j = 0; j < VX; ++j) up[f][j] = madd(cx.cdrift, b[j], a[j]);
    }
    // halo columns (lane 0: left, lane 31: right), rows ly .. ly + 2 of the slot
    float el[NF][CR_OF(CORNERS)];
    {
      const int side = lane == 31 ? 1 : 0;
#pragma unroll
      for (int f = 0; f < NF; ++f)
#pragma unroll
        for (int rr = 0; rr < CR_OF(CORNERS); ++rr) {
          const int row = ly + 1 + rr - (CR_OF(CORNERS) - 1) / 2;
          el[f][rr] = madd(cx.cdrift, colb[s][1][f][side][row], colb[s][0][f][side][row]);
        }
    }
    // The slot is refilled by a TMA copy (async proxy): this thread's generic
    // reads of it are ordered before that write by a proxy fence, ahead of the
    // release (without it, a refill could land under a read still in flight).
    fence_proxy_async();
    __syncwarp();
    if (lane == 0) mbar_arrive(&empty[s]);   // this warp is done with the slot

    float so_new[NF][VX], smid_new[NF][VX];
#pragma unroll
    for (int f = 0; f < NF; ++f) {
      constexpr int CR = CR_OF(CORNERS);
      float left = __shfl_up_sync(0xffffffffu, cur_ph[f][VX - 1], 1);
      float right = __shfl_down_sync(0xffffffffu, cur_ph[f][0], 1);
      if (lane == 0) left = el[f][(CR - 1) / 2];
      if (lane == 31) right = el[f][(CR - 1) / 2];
      float dl = 0.f, dr = 0.f, ul = 0.f, ur = 0.f;
      if constexpr (CORNERS) {
        dl = __shfl_up_sync(0xffffffffu, dn[f][VX - 1], 1);
        dr = __shfl_down_sync(0xffffffffu, dn[f][0], 1);
        ul = __shfl_up_sync(0xffffffffu, up[f][VX - 1], 1);
        ur = __shfl_down_sync(0xffffffffu, up[f][0], 1);
        if (lane == 0) { dl = el[f][0]; ul = el[f][CR - 1]; }
        if (lane == 31) { dr = el[f][0]; ur = el[f][CR - 1]; }
      }
#pragma unroll
      for (int j = 0; j < VX; ++j) {
        const float ctr = cur_ph[f][j];
        const float L = j > 0 ? cur_ph[f][j - 1] : left;
        const float R = j < VX - 1 ? cur_ph[f][j + 1] : right;
        const float faces = (dn[f][j] + up[f][j]) + (L + R);
        if constexpr (CORNERS) {
          const float DL = j > 0 ? dn[f][j - 1] : dl;
          const float DR = j < VX - 1 ? dn[f][j + 1] : dr;
          const float UL = j > 0 ? up[f][j - 1] : ul;
          const float UR = j < VX - 1 ? up[f][j + 1] : ur;
          const float corners = (DL + DR) + (UL + UR);
          smid_new[f][j] = madd(c2, corners, madd(c1, faces, c0 * ctr));
          so_new[f][j] = madd(c3, corners, madd(c2, faces, c1 * ctr));
        } else {
          smid_new[f][j] = madd(c0, ctr, faces);
          so_new[f][j] = ctr;
        }
      }
    }
    if (q >= 2) {  // output plane z = p - 1
      const size_t o = (size_t)(p - 1) * nn + (size_t)(y0 + ly) * n + x0 + lane * VX;
      float ps[NQ];
#pragma unroll
      for (int i = 0; i < NQ; ++i) ps[i] = 0.f;
      float pin[NF][VX], phs[NF][VX];
#pragma unroll
      for (int j = 0; j < VX; ++j) {
        float phj[NF], Dj[NF], pmj[NF], pnj[NF];
#pragma unroll
        for (int f = 0; f < NF; ++f) {
          phs[f][j] = ph_m[f][j] - Mf[f];   // the re-centred drifted field
          phj[f] = phs[f][j];
          Dj[f] = part_m[f][j] + so_new[f][j];
          pmj[f] = pi_m[f][j];
        }
        cx.site(mode, phj, Dj, pmj, pnj, ps);
#pragma unroll
        for (int f = 0; f < NF; ++f) pin[f][j] = pnj[f];
      }
#pragma unroll
      for (int f = 0; f < NF; ++f) {
        vstore<float, VX>(phi_out + f * S + o, phs[f]);
        if (mode == MODE_SWEEP) vstore<float, VX>(pi_out + f * S + o, pin[f]);
      }
#pragma unroll
      for (int i = 0; i < NQ; ++i)
        if (mode != MODE_SWEEP || i < SL::DPHI2 || i >= SL::DPHI2 + NF) acc[i].add(ps[i]);
    }
#pragma unroll
    for (int f = 0; f < NF; ++f)
#pragma unroll
      for (int j = 0; j < VX; ++j) {
        part_m[f][j] = (CORNERS ? so_m[f][j] : ph_m[f][j]) + smid_new[f][j];
        if constexpr (CORNERS) so_m[f][j] = so_new[f][j];
        ph_m[f][j] = cur_ph[f][j];
        pi_m[f][j] = cur_pi[f][j];
      }
  }

  block_partials<PREC, NQ, float>(acc, nullptr, sred, sout);
  if (s_fault) {
    // a copy or a release never completed: record it, drain what may be in flight (bounded)
    if (tid == 0) {
      atomicOr(d.fault, 1);
      for (int rr = q; rr < Q && rr < q + LEAD; ++rr)
        mbar_wait(&full[rr % NSLOT], (uint32_t)((rr / NSLOT) & 1));
    }
    return;
  }
  finish_block<MODEL, PREC>(s_ctx, d, mode, cta, sout, &s_last);
}

// ---------------------------------------------------------------------------
// Plain-load sweep (any n): one site per thread, modular indices, ragged tiles.
// ---------------------------------------------------------------------------
template <int MODEL, int STENCIL, int PREC>
__global__ void __launch_bounds__(kThreads, 2) sweep_plain(const LaunchTable tab) {
  using C = Ctx<MODEL, PREC>;
  using T = typename C::T;
  using SL = typename C::SL;
  constexpr int NF = C::NF;
  constexpr int NQ = SL::NQ;
  constexpr bool CORNERS = StencilW<STENCIL>::kCorners;

  __shared__ T sm[2][NF][kMaxTY + 2][kMaxTXT + 2];
  __shared__ double sred[(kThreads / 32) * NQ];
  __shared__ double sout[NQ];
  __shared__ int s_last;

  const int mem = member_of(tab, blockIdx.x);
  const SimDesc& d = *tab.desc[mem];
  const int cta = blockIdx.x - tab.cta_offset[mem];
  const Background& bgr = *d.bg;
  const int mode = bgr.mode;
  if (mode == MODE_IDLE) return;

  const int n = d.n;
  const int TX = d.txt, TY = d.ty;
  const int tile = cta % (d.tiles_x * d.tiles_y);
  const int zch = cta / (d.tiles_x * d.tiles_y);
  const int x0 = (tile % d.tiles_x) * TX;
  const int y0 = (tile / d.tiles_x) * TY;
  const int z0 = zch * d.zc;
  const int zend = min(n, z0 + d.zc);
  const int tid = threadIdx.x;
  const bool active = tid < TX * TY;
  const int lx = active ? tid % TX : 0;
  const int ly = active ? tid / TX : 0;
  const int gx = x0 + lx, gy = y0 + ly;
  const bool valid = active && gx < n && gy < n;
  const size_t own_off = (size_t)wrapi(gy, n) * n + wrapi(gx, n);
  const size_t S = (size_t)d.S;
  const size_t nn = (size_t)n * n;

  __shared__ C s_ctx;   // scalar context: computed once, by one thread (FP64 pipe is scarce)
  if (threadIdx.x == 0) s_ctx.init(bgr, d, mode);
  __syncthreads();
  const C cx = s_ctx;
  const int ib = bgr.cur;
  const T* __restrict__ phi_in = (const T*)d.phi[ib & 1];
  T* __restrict__ phi_out = (T*)d.phi[(ib & 1) ^ 1];
  const T* __restrict__ pi_in = (const T*)d.pi[(ib >> 1) & 1];
  T* __restrict__ pi_out = (T*)d.pi[((ib >> 1) & 1) ^ 1];

  const T c0 = CORNERS ? (T)(-128.0 / 30.0) : (T)(-6.0);
  const T c1 = CORNERS ? (T)(14.0 / 30.0) : (T)1.0;
  const T c2 = CORNERS ? (T)(3.0 / 30.0) : (T)0.0;
  const T c3 = CORNERS ? (T)(1.0 / 30.0) : (T)0.0;

  // halo ring: (TX+2) cells below, (TX+2) above, TY left, TY right
  const int nhalo = 2 * (TX + 2) + 2 * TY;
  int hx = 0, hy = 0;
  if (tid < nhalo) {
    int t = tid;
    if (t < TX + 2) { hx = t - 1; hy = -1; }
    else if ((t -= TX + 2) < TX + 2) { hx = t - 1; hy = TY; }
    else if ((t -= TX + 2) < TY) { hx = -1; hy = t; }
    else { t -= TY; hx = TX; hy = t; }
  }
  const size_t halo_off = (size_t)wrapi(y0 + hy, n) * n + wrapi(x0 + hx, n);

  T rp[NF], rq[NF], hp[NF], hq[NF];
#pragma unroll
  for (int f = 0; f < NF; ++f) { rp[f] = rq[f] = hp[f] = hq[f] = 0; }
  auto load_raw = [&](int p) {
    const size_t zoff = (size_t)wrapi(p, n) * nn;
#pragma unroll
    for (int f = 0; f < NF; ++f) {
      if (active) { rp[f] = phi_in[f * S + zoff + own_off]; rq[f] = pi_in[f * S + zoff + own_off]; }
      if (tid < nhalo) { hp[f] = phi_in[f * S + zoff + halo_off]; hq[f] = pi_in[f * S + zoff + halo_off]; }
    }
  };

  Acc<T> acc[NQ];
  T accd_s[NQ];   // float64 path: plain per-thread sums
#pragma unroll
  for (int q = 0; q < NQ; ++q) { acc[q].zero(); accd_s[q] = (T)0; }
  T part_m[NF], so_m[NF], ph_m[NF], pi_m[NF];
#pragma unroll
  for (int f = 0; f < NF; ++f) part_m[f] = so_m[f] = ph_m[f] = pi_m[f] = (T)0;

  load_raw(z0 - 1);
  for (int p = z0 - 1; p <= zend; ++p) {
    const int buf = (p - z0 + 1) & 1;
    T cur_ph[NF], cur_pi[NF];
#pragma unroll
    for (int f = 0; f < NF; ++f) {
      T ph = rp[f], pv = rq[f];
      if constexpr (PREC == PREC_SPLIT) { ph -= cx.mu_phi[f]; pv -= cx.mu_pi[f]; }
      cur_pi[f] = pv;
      cur_ph[f] = madd(cx.cdrift, pv, ph);
      if (active) sm[buf][f][ly + 1][lx + 1] = cur_ph[f];
      if (tid < nhalo) {
        T h1 = hp[f], h2 = hq[f];
        if constexpr (PREC == PREC_SPLIT) { h1 -= cx.mu_phi[f]; h2 -= cx.mu_pi[f]; }
        sm[buf][f][hy + 1][hx + 1] = madd(cx.cdrift, h2, h1);
      }
    }
    if (p < zend) load_raw(p + 1);
    __syncthreads();
    T so_new[NF], smid_new[NF];
#pragma unroll
    for (int f = 0; f < NF; ++f) {
      const T ctr = sm[buf][f][ly + 1][lx + 1];
      const T faces = (sm[buf][f][ly][lx + 1] + sm[buf][f][ly + 2][lx + 1]) +
                      (sm[buf][f][ly + 1][lx] + sm[buf][f][ly + 1][lx + 2]);
      if constexpr (CORNERS) {
        const T corners = (sm[buf][f][ly][lx] + sm[buf][f][ly][lx + 2]) +
                          (sm[buf][f][ly + 2][lx] + sm[buf][f][ly + 2][lx + 2]);
        smid_new[f] = madd(c2, corners, madd(c1, faces, c0 * ctr));
        so_new[f] = madd(c3, corners, madd(c2, faces, c1 * ctr));
      } else {
        smid_new[f] = madd(c0, ctr, faces);
        so_new[f] = ctr;
      }
    }
    if (p >= z0 + 1 && valid) {
      const size_t o = (size_t)(p - 1) * nn + (size_t)gy * n + gx;
      T ps_local[NQ];
      T* ps = ps_local;
      if constexpr (PREC == PREC_FP64) {
        ps = accd_s;
      } else {
#pragma unroll
        for (int i = 0; i < NQ; ++i) ps_local[i] = (T)0;
      }
      T Dj[NF], pnj[NF];
#pragma unroll
      for (int f = 0; f < NF; ++f) Dj[f] = part_m[f] + so_new[f];
      cx.site(mode, ph_m, Dj, pi_m, pnj, ps);
#pragma unroll
      for (int f = 0; f < NF; ++f) {
        phi_out[f * S + o] = ph_m[f];
        if (mode == MODE_SWEEP) pi_out[f * S + o] = pnj[f];
      }
      if constexpr (PREC == PREC_SPLIT) {
#pragma unroll
        for (int i = 0; i < NQ; ++i) acc[i].add(ps_local[i]);
      }
    }
#pragma unroll
    for (int f = 0; f < NF; ++f) {
      part_m[f] = (CORNERS ? so_m[f] : ph_m[f]) + smid_new[f];
      if constexpr (CORNERS) so_m[f] = so_new[f];
      ph_m[f] = cur_ph[f];
      pi_m[f] = cur_pi[f];
    }
  }
  block_partials<PREC, NQ, T>(acc, accd_s, sred, sout);
  finish_block<MODEL, PREC>(s_ctx, d, mode, cta, sout, &s_last);
}

// ---------------------------------------------------------------------------
// Fourth-order stencil (13 points: the centre and two sites each way along
// every axis), per-axis weights (-1, 16, -30, 16, -1)/12: a plain-load sweep.
// Each thread owns one (x, y) column of a tile and marches z with a register
// queue of its column's drifted values at z-2 .. z+2; the eight in-plane
// neighbours are read (and drifted) from global memory (L1/L2), the column's
// own momenta from its queue.  The kick, sums and block finish are those of
// the other kernels (Ctx::site, block_partials, finish_block).
// ---------------------------------------------------------------------------
template <int MODEL, int PREC>
__global__ void __launch_bounds__(kThreads, 2) sweep_wide(const LaunchTable tab) {
  using C = Ctx<MODEL, PREC>;
  using T = typename C::T;
  using SL = typename C::SL;
  constexpr int NF = C::NF;
  constexpr int NQ = SL::NQ;
  __shared__ double sred[(kThreads / 32) * NQ];
  __shared__ double sout[NQ];
  __shared__ int s_last;
  __shared__ C s_ctx;

  const int mem = member_of(tab, blockIdx.x);
  const SimDesc& d = *tab.desc[mem];
  const int cta = blockIdx.x - tab.cta_offset[mem];
  const Background& bgr = *d.bg;
  const int mode = bgr.mode;
  if (mode == MODE_IDLE) return;

  const int n = d.n;
  const int TX = d.txt, TY = d.ty;
  const int tile = cta % (d.tiles_x * d.tiles_y);
  const int zch = cta / (d.tiles_x * d.tiles_y);
  const int x0 = (tile % d.tiles_x) * TX;
  const int y0 = (tile / d.tiles_x) * TY;
  const int z0 = zch * d.zc;
  const int zend = min(n, z0 + d.zc);
  const int tid = threadIdx.x;
  const bool active = tid < TX * TY;
  const int gx = x0 + (active ? tid % TX : 0), gy = y0 + (active ? tid / TX : 0);
  const bool valid = active && gx < n && gy < n;
  const size_t S = (size_t)d.S, nn = (size_t)n * n;

  if (tid == 0) s_ctx.init(bgr, d, mode);
  __syncthreads();
  const C cx = s_ctx;
  const int ib = bgr.cur;
  const T* __restrict__ phi_in = (const T*)d.phi[ib & 1];
  T* __restrict__ phi_out = (T*)d.phi[(ib & 1) ^ 1];
  const T* __restrict__ pi_in = (const T*)d.pi[(ib >> 1) & 1];
  T* __restrict__ pi_out = (T*)d.pi[((ib >> 1) & 1) ^ 1];
  const T w1 = (T)(16.0 / 12.0), w2 = (T)(-1.0 / 12.0), w0 = (T)(-90.0 / 12.0);
  T Mf[NF];   // split form: re-centring of the drifted field
#pragma unroll
  for (int f = 0; f < NF; ++f) Mf[f] = madd(cx.cdrift, cx.mu_pi[f], cx.mu_phi[f]);

  // drifted field value (re-centred momenta in the split form: the stencil
  // works on phi + c pi, D of a constant being zero)
  auto drifted = [&](int f, int z, int y, int x) -> T {
    const size_t o = (size_t)f * S + (size_t)wrapi(z, n) * nn + (size_t)wrapi(y, n) * n + wrapi(x, n);
    return madd(cx.cdrift, pi_in[o], phi_in[o]);
  };
  Acc<T> acc[NQ];
  T accd_s[NQ];
#pragma unroll
  for (int q = 0; q < NQ; ++q) { acc[q].zero(); accd_s[q] = (T)0; }

  if (valid) {
    T qz[NF][5], qp[NF];   // column queue z-2 .. z+2; momentum at z
#pragma unroll
    for (int f = 0; f < NF; ++f)
#pragma unroll
      for (int k = 0; k < 4; ++k) qz[f][k] = drifted(f, z0 - 2 + k, gy, gx);
    for (int z = z0; z < zend; ++z) {
      T phj[NF], Dj[NF], pmj[NF], pnj[NF];
#pragma unroll
      for (int f = 0; f < NF; ++f) {
        qz[f][4] = drifted(f, z + 2, gy, gx);
        const size_t own = (size_t)f * S + (size_t)z * nn + (size_t)gy * n + gx;
        qp[f] = pi_in[own];
        if constexpr (PREC == PREC_SPLIT) qp[f] -= cx.mu_pi[f];
        const T near = (qz[f][1] + qz[f][3]) +
                       ((drifted(f, z, gy - 1, gx) + drifted(f, z, gy + 1, gx)) +
                        (drifted(f, z, gy, gx - 1) + drifted(f, z, gy, gx + 1)));
        const T far = (qz[f][0] + qz[f][4]) +
                      ((drifted(f, z, gy - 2, gx) + drifted(f, z, gy + 2, gx)) +
                       (drifted(f, z, gy, gx - 2) + drifted(f, z, gy, gx + 2)));
        Dj[f] = madd(w0, qz[f][2], madd(w2, far, w1 * near));
        phj[f] = qz[f][2];
        if constexpr (PREC == PREC_SPLIT) phj[f] -= Mf[f];
        pmj[f] = qp[f];
      }
      T ps_local[NQ];
      T* ps = ps_local;
      if constexpr (PREC == PREC_FP64) {
        ps = accd_s;
      } else {
#pragma unroll
        for (int i = 0; i < NQ; ++i) ps_local[i] = (T)0;
      }
      cx.site(mode, phj, Dj, pmj, pnj, ps);
      const size_t o = (size_t)z * nn + (size_t)gy * n + gx;
#pragma unroll
      for (int f = 0; f < NF; ++f) {
        phi_out[f * S + o] = phj[f];
        if (mode == MODE_SWEEP) pi_out[f * S + o] = pnj[f];
      }
      if constexpr (PREC == PREC_SPLIT) {
#pragma unroll
        for (int i = 0; i < NQ; ++i) acc[i].add(ps_local[i]);
      }
#pragma unroll
      for (int f = 0; f < NF; ++f)
#pragma unroll
        for (int k = 0; k < 4; ++k) qz[f][k] = qz[f][k + 1];
    }
  }
  block_partials<PREC, NQ, T>(acc, accd_s, sred, sout);
  finish_block<MODEL, PREC>(s_ctx, d, mode, cta, sout, &s_last);
}

// ---------------------------------------------------------------------------
// Potentials compiled at run time (FP64 form, per-stage, plain loads).  A
// stage is three launches: rt_drift (phi* = phi + c pi into d.rt_phis), the
// compiled kernel (V'(phi*) and V(phi*) into d.rt_dV, d.rt_V), and rt_kick
// (the Laplacian of phi*, the kick, the sums and the block finish, which
// advances the Background).  Both library kernels derive the stage's
// coefficients from the same Background record, which only the last block of
// rt_kick changes.
// ---------------------------------------------------------------------------
template <int MODEL>
__global__ void __launch_bounds__(kThreads) rt_drift(const LaunchTable tab) {
  using C = Ctx<MODEL, PREC_FP64>;
  constexpr int NF = C::NF;
  __shared__ C s_ctx;
  const SimDesc& d = *tab.desc[0];
  const Background& bgr = *d.bg;
  const int mode = bgr.mode;
  if (mode == MODE_IDLE) return;
  if (threadIdx.x == 0) s_ctx.init(bgr, d, mode);
  __syncthreads();
  const double c = s_ctx.cdrift;
  const int ib = bgr.cur;
  const double* __restrict__ phi = (const double*)d.phi[ib & 1];
  const double* __restrict__ pi = (const double*)d.pi[(ib >> 1) & 1];
  const size_t total = (size_t)NF * (size_t)d.S;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < total;
       i += (size_t)gridDim.x * blockDim.x)
    d.rt_phis[i] = fma(c, pi[i], phi[i]);
}

template <int MODEL, int STENCIL>
__global__ void __launch_bounds__(kThreads, 2) rt_kick(const LaunchTable tab) {
  using C = Ctx<MODEL, PREC_FP64>;
  using SL = typename C::SL;
  constexpr int NF = C::NF;
  constexpr int NQ = SL::NQ;
  constexpr bool CORNERS = StencilW<STENCIL>::kCorners;
  __shared__ double sred[(kThreads / 32) * NQ];
  __shared__ double sout[NQ];
  __shared__ int s_last;
  __shared__ C s_ctx;
  const SimDesc& d = *tab.desc[0];
  const int cta = blockIdx.x;
  const Background& bgr = *d.bg;
  const int mode = bgr.mode;
  if (mode == MODE_IDLE) return;
  const int n = d.n;
  const int TX = d.txt, TY = d.ty;
  const int tile = cta % (d.tiles_x * d.tiles_y);
  const int zch = cta / (d.tiles_x * d.tiles_y);
  const int x0 = (tile % d.tiles_x) * TX, y0 = (tile / d.tiles_x) * TY;
  const int z0 = zch * d.zc, zend = min(n, z0 + d.zc);
  const int tid = threadIdx.x;
  const bool active = tid < TX * TY;
  const int gx = x0 + (active ? tid % TX : 0), gy = y0 + (active ? tid / TX : 0);
  const bool valid = active && gx < n && gy < n;
  const size_t S = (size_t)d.S, nn = (size_t)n * n;
  if (tid == 0) s_ctx.init(bgr, d, mode);
  __syncthreads();
  const C cx = s_ctx;
  const int ib = bgr.cur;
  double* __restrict__ phi_out = (double*)d.phi[(ib & 1) ^ 1];
  const double* __restrict__ pi_in = (const double*)d.pi[(ib >> 1) & 1];
  double* __restrict__ pi_out = (double*)d.pi[((ib >> 1) & 1) ^ 1];
  const double c0 = CORNERS ? -128.0 / 30.0 : -6.0, c1 = CORNERS ? 14.0 / 30.0 : 1.0;
  const double c2 = CORNERS ? 3.0 / 30.0 : 0.0, c3 = CORNERS ? 1.0 / 30.0 : 0.0;
  double ps[NQ];
  Acc<double> acc[NQ];
#pragma unroll
  for (int q = 0; q < NQ; ++q) ps[q] = 0.0;
  if (valid) {
    for (int z = z0; z < zend; ++z) {
      const size_t o = (size_t)z * nn + (size_t)gy * n + gx;
#pragma unroll
      for (int f = 0; f < NF; ++f) {
        const double* ph = d.rt_phis + (size_t)f * S;
        const double ctr = ph[o];
        double D;
        if constexpr (STENCIL == 13) {
          // the fourth-order stencil: +-1 and +-2 along each axis
          auto at = [&](int dz, int dy, int dx) {
            return ph[(size_t)((z + dz + 2 * n) % n) * nn + (size_t)((gy + dy + 2 * n) % n) * n +
                      (gx + dx + 2 * n) % n];
          };
          const double near = (at(-1, 0, 0) + at(1, 0, 0)) + (at(0, -1, 0) + at(0, 1, 0)) +
                              (at(0, 0, -1) + at(0, 0, 1));
          const double far = (at(-2, 0, 0) + at(2, 0, 0)) + (at(0, -2, 0) + at(0, 2, 0)) +
                             (at(0, 0, -2) + at(0, 0, 2));
          D = fma(-90.0 / 12.0, ctr, fma(-1.0 / 12.0, far, (16.0 / 12.0) * near));
        } else {
          double faces = 0.0, edges = 0.0, corners = 0.0;
          for (int dz = -1; dz <= 1; ++dz)
            for (int dy = -1; dy <= 1; ++dy)
              for (int dx = -1; dx <= 1; ++dx) {
                const int cls = (dz != 0) + (dy != 0) + (dx != 0);
                if (cls == 0 || (!CORNERS && cls > 1)) continue;
                const double v = ph[(size_t)wrapi(z + dz, n) * nn +
                                    (size_t)wrapi(gy + dy, n) * n + wrapi(gx + dx, n)];
                if (cls == 1) faces += v; else if (cls == 2) edges += v; else corners += v;
              }
          D = fma(c3, corners, fma(c2, edges, fma(c1, faces, c0 * ctr)));
        }
        const double pim = pi_in[(size_t)f * S + o];
        double pin = pim;
        if (mode == MODE_SWEEP) {
          pin = fma(cx.kD, D, fma(-cx.kV, d.rt_dV[(size_t)f * S + o], pim));
          pi_out[(size_t)f * S + o] = pin;
        }
        phi_out[(size_t)f * S + o] = ctr;
        ps[SL::PI2 + f] = fma(pin, pin, ps[SL::PI2 + f]);
        ps[SL::PHID + f] = fma(ctr, D, ps[SL::PHID + f]);
        if (mode != MODE_SWEEP) {
          const double dd = ctr - cx.shiftK[f];
          ps[SL::DPHI + f] += dd;
          ps[SL::DPHI2 + f] = fma(dd, dd, ps[SL::DPHI2 + f]);
        }
      }
      ps[SL::V] += d.rt_V[o];
    }
  }
  block_partials<PREC_FP64, NQ, double>(acc, ps, sred, sout);
  finish_block<MODEL, PREC_FP64>(s_ctx, d, mode, cta, sout, &s_last);
}

// Launch helper: dispatch (model, stencil, path/vx) at runtime to an instance.
// grid == 0 only prepares the instance (its shared-memory attribute), so that
// callers can do it before a stream capture.
template <int PREC>
cudaError_t launch_sweep_impl(int model, int stencil, int vx, int tma, const LaunchTable& t,
                              int grid, cudaStream_t s) {
  const dim3 g(grid), b(kThreads);
#define PYCOOL_PLAIN(M, ST)                                              \
  if (!tma && model == M && stencil == ST) {                             \
    if (grid == 0) return cudaSuccess;                                   \
    sweep_plain<M, ST, PREC><<<g, b, 0, s>>>(t);                         \
    return cudaGetLastError();                                           \
  }
#define PYCOOL_WIDE(M)                                                   \
  if (model == M && stencil == 13) {                                     \
    if (grid == 0) return cudaSuccess;                                   \
    sweep_wide<M, PREC><<<g, b, 0, s>>>(t);                              \
    return cudaGetLastError();                                           \
  }
  PYCOOL_WIDE(M_FREE) PYCOOL_WIDE(M_CHAOTIC2) PYCOOL_WIDE(M_OSCILLON) PYCOOL_WIDE(M_QBALL)
#undef PYCOOL_WIDE
#define PYCOOL_TMA(M, ST, V)                                             \
  if constexpr (V * Pot<M>::NF * (PREC == PREC_FP64 ? 8 : 4) <= 16) {    \
    if (tma && model == M && stencil == ST && vx == V) {                 \
      if constexpr (PREC == PREC_SPLIT) {                                \
        constexpr size_t smem = pipe_smem_bytes<Pot<M>::NF, V>();        \
        static const cudaError_t attr = cudaFuncSetAttribute(            \
            sweep_split_pipe<M, ST, V>,                                  \
            cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);     \
        if (attr != cudaSuccess || grid == 0) return attr;               \
        sweep_split_pipe<M, ST, V><<<g, b, smem, s>>>(t);                \
      } else {                                                           \
        if (grid == 0) return cudaSuccess;                               \
        sweep_tma<M, ST, PREC, V><<<g, b, 0, s>>>(t);                    \
      }                                                                  \
      return cudaGetLastError();                                         \
    }                                                                    \
  }
#define PYCOOL_FOR_MODELS(X, V)                                          \
  X(M_FREE, 7 V) X(M_FREE, 27 V) X(M_CHAOTIC2, 7 V) X(M_CHAOTIC2, 27 V)  \
  X(M_OSCILLON, 7 V) X(M_OSCILLON, 27 V) X(M_QBALL, 7 V) X(M_QBALL, 27 V)
#define PYCOOL_NOV
#define PYCOOL_V1 , 1
#define PYCOOL_V2 , 2
#define PYCOOL_V4 , 4
  PYCOOL_FOR_MODELS(PYCOOL_PLAIN, PYCOOL_NOV)
  PYCOOL_FOR_MODELS(PYCOOL_TMA, PYCOOL_V1)
  PYCOOL_FOR_MODELS(PYCOOL_TMA, PYCOOL_V2)
  if constexpr (PREC == PREC_SPLIT) { PYCOOL_FOR_MODELS(PYCOOL_TMA, PYCOOL_V4) }
#undef PYCOOL_V4
#undef PYCOOL_V2
#undef PYCOOL_V1
#undef PYCOOL_NOV
#undef PYCOOL_FOR_MODELS
#undef PYCOOL_TMA
#undef PYCOOL_PLAIN
  return cudaErrorInvalidValue;
}

}  // namespace pycool
