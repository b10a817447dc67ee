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
// streams z upward (Sec. 2.4 marches z the same way).  The drifted plane
// phi*(z) with a one-site halo lives in shared memory (double-buffered, one
// barrier per plane); the Laplacian of Eq. D is split by z-offset into
//     S_mid(p) = c0 ctr + c1 sum(4 faces) + c2 sum(4 corners)   (in-plane)
//     S_off(p) = c1 ctr + c2 sum(4 faces) + c3 sum(4 corners)   (for planes z+-1)
// so D(z) = S_off(z-1) + S_mid(z) + S_off(z+1) needs only one resident plane.
// Periodic wrap is done with modular indices; ragged tiles (n not a multiple
// of the tile) load wrapped values and mask their outputs.
//
// Reductions: per-thread column sums -> warp butterfly -> fixed-order sum of
// the 8 warps -> one partial per block and quantity.  The last block to arrive
// (atomic ticket; nobody waits) sums the partials in block order (Neumaier),
// applies the p_a kick of Phi_H3 and advances the Background.  Results are
// bitwise reproducible and depend only on the lattice, not on the batch.
#pragma once

#include <cuda_runtime.h>
#include <math.h>

#include <type_traits>

#include "internal.cuh"
#include "models.cuh"

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
};

__device__ __forceinline__ Coef prestage(const Background& b, const SimDesc& d, int mode) {
  Coef k;
  const double hp = b.h_prev;
  const double h = (mode == MODE_SWEEP) ? d.w[b.stage] * d.dt : 0.0;
  double a = b.a;
  double pa = b.pa;
  // trailing Phi_H2(h_prev/2) of the previous stage: p_a += [sum pi^2/a^3 - V_L rho_m] h_prev/2
  pa = pa + (b.sum_pi2 / (a * a * a) - d.VL * d.rho_m0) * (0.5 * hp);
  double c = 0.5 * hp / (a * a);
  if (mode != MODE_SWEEP) {
    // trailing Phi_H1(h_prev/2): a -= p_a h_prev / (12 V_L m^2)
    a = a - pa * d.inv6VLm2 * (0.5 * hp);
    k.c = c; k.kD = 0.0; k.kV = 0.0; k.a = a; k.pa = pa; k.h = 0.0;
    return k;
  }
  // Phi_H1(h_prev/2) Phi_H1(h/2) merged (p_a is constant under H1)
  a = a - pa * d.inv6VLm2 * (0.5 * (hp + h));
  // leading Phi_H2(h/2)
  pa = pa + (b.sum_pi2 / (a * a * a) - d.VL * d.rho_m0) * (0.5 * h);
  c = c + 0.5 * h / (a * a);
  k.c = c;
  k.kD = a * a * h * d.dx2inv;
  k.kV = (a * a) * (a * a) * h;
  k.a = a; k.pa = pa; k.h = h;
  return k;
}

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

__device__ __forceinline__ bool is_fin(double x) { return isfinite(x); }

template <int STENCIL, typename T> struct StencilC;
template <typename T> struct StencilC<7, T> {
  static constexpr bool kCorners = false;
};
template <typename T> struct StencilC<27, T> {
  static constexpr bool kCorners = true;
};

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

// ---------------------------------------------------------------------------
// The sweep kernel.
// ---------------------------------------------------------------------------
template <int MODEL, int STENCIL, int PREC>
__global__ void __launch_bounds__(kThreads)
sweep_kernel(const LaunchTable tab) {
  using P = Pot<MODEL>;
  constexpr int NF = P::NF;
  using T = typename std::conditional<PREC == PREC_FP64, double, float>::type;
  using SL = Slots<NF, PREC>;
  constexpr int NQ = SL::NQ;
  constexpr bool CORNERS = StencilC<STENCIL, T>::kCorners;

  __shared__ T sm[2][NF][kMaxTY + 2][kMaxTX + 2];
  __shared__ double sred[(kThreads / 32) * NQ];
  __shared__ double sout[NQ];
  __shared__ int s_last;

  // ---- which simulation and tile ------------------------------------------
  int mem = 0;
  {
    const int b = blockIdx.x;
    int lo = 0, hi = tab.count - 1;
    while (lo < hi) {  // largest m with cta_offset[m] <= b
      const int mid = (lo + hi + 1) >> 1;
      if (tab.cta_offset[mid] <= b) lo = mid; else hi = mid - 1;
    }
    mem = lo;
  }
  const SimDesc& d = *tab.desc[mem];
  const int cta = blockIdx.x - tab.cta_offset[mem];
  Background* bgp = d.bg;
  const Background bg = *bgp;
  const int mode = bg.mode;
  if (mode == MODE_IDLE) return;

  const int n = d.n;
  const int TX = d.tx, TY = d.ty;
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
  const int wx = gx >= n ? gx - n : gx;
  const int wy = gy >= n ? gy - n : gy;
  const size_t S = (size_t)d.S;
  const size_t nn = (size_t)n * n;

  const int ib = bg.cur;  // bit0: phi buffer, bit1: pi buffer
  const T* __restrict__ phi_in = (const T*)d.phi[ib & 1];
  T* __restrict__ phi_out = (T*)d.phi[(ib & 1) ^ 1];
  const T* __restrict__ pi_in = (const T*)d.pi[(ib >> 1) & 1];
  T* __restrict__ pi_out = (T*)d.pi[((ib >> 1) & 1) ^ 1];

  // ---- scalar coefficients -------------------------------------------------
  const Coef k = prestage(bg, d, mode);
  const typename P::K pk = P::prep(d.params);
  T cdrift, kD, kV;
  T mu_phi[NF], mu_pi[NF];
  double phi0s[NF], pi0s[NF], V0 = 0.0;  // split background after drift / kick
  typename P::SplitK sk;
  if constexpr (PREC == PREC_SPLIT) {
    cdrift = (T)k.c; kD = (T)k.kD; kV = (T)k.kV;
    double phi0p[NF], pi0p[NF], dV0[NF];
#pragma unroll
    for (int f = 0; f < NF; ++f) {
      mu_phi[f] = (float)bg.mu_phi[f];
      mu_pi[f] = (float)bg.mu_pi[f];
      phi0p[f] = bg.phi0[f] + (double)mu_phi[f];
      pi0p[f] = bg.pi0[f] + (double)mu_pi[f];
      phi0s[f] = fma(k.c, pi0p[f], phi0p[f]);
    }
    P::eval(pk, phi0s, dV0, V0);
#pragma unroll
    for (int f = 0; f < NF; ++f)
      pi0s[f] = (mode == MODE_SWEEP) ? fma(-k.kV, dV0[f], pi0p[f]) : pi0p[f];
    sk = P::split_prep(d.params, phi0s);
  } else {
    cdrift = k.c; kD = k.kD; kV = k.kV;
#pragma unroll
    for (int f = 0; f < NF; ++f) { mu_phi[f] = 0; mu_pi[f] = 0; }
  }
  T shiftK[NF];
#pragma unroll
  for (int f = 0; f < NF; ++f) shiftK[f] = (PREC == PREC_FP64) ? (T)bg.shift[f] : (T)0;

  // stencil weights (Eq. D): 7pt (-6, 1, 0, 0); iso27 (-128, 14, 3, 1)/30
  const T c0 = CORNERS ? (T)(-128.0 / 30.0) : (T)(-6.0);
  const T c1 = CORNERS ? (T)(14.0 / 30.0) : (T)1.0;
  const T c2 = CORNERS ? (T)(3.0 / 30.0) : (T)0.0;
  const T c3 = CORNERS ? (T)(1.0 / 30.0) : (T)0.0;

  // halo ring of the tile: (TX+2) cells below, (TX+2) above, TY left, TY right
  const int nhalo = 2 * (TX + 2) + 2 * TY;
  int hx = 0, hy = 0;
  if (tid < nhalo) {
    int t = tid;
    if (t < TX + 2) { hx = t - 1; hy = -1; }
    else if ((t -= TX + 2) < TX + 2) { hx = t - 1; hy = TY; }
    else if ((t -= TX + 2) < TY) { hx = -1; hy = t; }
    else { t -= TY; hx = TX; hy = t; }
  }
  int hgx = x0 + hx, hgy = y0 + hy;
  hgx = hgx < 0 ? hgx + n : (hgx >= n ? hgx - n : hgx);
  hgy = hgy < 0 ? hgy + n : (hgy >= n ? hgy - n : hgy);

  // per-thread accumulators
  T acc[NQ];
#pragma unroll
  for (int q = 0; q < NQ; ++q) acc[q] = (T)0;

  // rotating registers (per field)
  T so_mm[NF], so_m[NF], smid_m[NF], ph_m[NF], pi_m[NF];
#pragma unroll
  for (int f = 0; f < NF; ++f) { so_mm[f] = so_m[f] = smid_m[f] = ph_m[f] = pi_m[f] = (T)0; }

  for (int p = z0 - 1; p <= zend; ++p) {
    const int buf = (p - z0 + 1) & 1;
    const int zw = p < 0 ? p + n : (p >= n ? p - n : p);
    const size_t zoff = (size_t)zw * nn;
    T cur_ph[NF], cur_pi[NF];
    // own cell
    if (active) {
      const size_t o = zoff + (size_t)wy * n + wx;
#pragma unroll
      for (int f = 0; f < NF; ++f) {
        T ph = phi_in[f * S + o], pv = pi_in[f * S + o];
        if constexpr (PREC == PREC_SPLIT) { ph -= mu_phi[f]; pv -= mu_pi[f]; }
        cur_pi[f] = pv;
        cur_ph[f] = fma(cdrift, pv, ph);
        sm[buf][f][ly + 1][lx + 1] = cur_ph[f];
      }
    }
    // halo cells
    if (tid < nhalo) {
      const size_t o = zoff + (size_t)hgy * n + hgx;
#pragma unroll
      for (int f = 0; f < NF; ++f) {
        T ph = phi_in[f * S + o], pv = pi_in[f * S + o];
        if constexpr (PREC == PREC_SPLIT) { ph -= mu_phi[f]; pv -= mu_pi[f]; }
        sm[buf][f][hy + 1][hx + 1] = fma(cdrift, pv, ph);
      }
    }
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
        smid_new[f] = fma(c2, corners, fma(c1, faces, c0 * ctr));
        so_new[f] = fma(c3, corners, fma(c2, faces, c1 * ctr));
      } else {
        smid_new[f] = fma(c0, ctr, faces);
        so_new[f] = ctr;
      }
    }
    if (p >= z0 + 1 && valid) {
      // output plane z = p - 1
      const int z = p - 1;
      const size_t o = (size_t)z * nn + (size_t)gy * n + gx;
      T D[NF];
#pragma unroll
      for (int f = 0; f < NF; ++f) D[f] = (so_mm[f] + so_new[f]) + smid_m[f];
      if (mode == MODE_SWEEP) {
        T pin[NF];
        if constexpr (PREC == PREC_FP64) {
          double dV[NF], V;
          P::eval(pk, ph_m, dV, V);
#pragma unroll
          for (int f = 0; f < NF; ++f) {
            pin[f] = fma(kD, D[f], fma(-kV, dV[f], pi_m[f]));
            acc[SL::PI2 + f] = fma(pin[f], pin[f], acc[SL::PI2 + f]);
            acc[SL::PHID + f] = fma(ph_m[f], D[f], acc[SL::PHID + f]);
          }
          acc[SL::V] += V;
        } else {
          float dVd[NF], dVv;
          P::diff(sk, ph_m, dVd, dVv);
#pragma unroll
          for (int f = 0; f < NF; ++f) {
            pin[f] = fmaf(kD, D[f], fmaf(-kV, dVd[f], pi_m[f]));
            acc[SL::DPI + f] += pin[f];
            acc[SL::DPI2 + f] = fmaf(pin[f], pin[f], acc[SL::DPI2 + f]);
            acc[SL::PHID + f] = fmaf(ph_m[f], D[f], acc[SL::PHID + f]);
            acc[SL::DPHI + f] += ph_m[f];
            acc[SL::DPHI2 + f] = fmaf(ph_m[f], ph_m[f], acc[SL::DPHI2 + f]);
          }
          acc[SL::V] += dVv;
        }
#pragma unroll
        for (int f = 0; f < NF; ++f) {
          phi_out[f * S + o] = ph_m[f];
          pi_out[f * S + o] = pin[f];
        }
      } else {  // flush: drift only, pi unchanged
        if constexpr (PREC == PREC_FP64) {
          double dV[NF], V;
          P::eval(pk, ph_m, dV, V);
#pragma unroll
          for (int f = 0; f < NF; ++f) {
            acc[SL::PI2 + f] = fma(pi_m[f], pi_m[f], acc[SL::PI2 + f]);
            acc[SL::PHID + f] = fma(ph_m[f], D[f], acc[SL::PHID + f]);
            const T dd = ph_m[f] - shiftK[f];
            acc[SL::DPHI + f] += dd;
            acc[SL::DPHI2 + f] = fma(dd, dd, acc[SL::DPHI2 + f]);
          }
          acc[SL::V] += V;
        } else {
          float dVd[NF], dVv;
          P::diff(sk, ph_m, dVd, dVv);
#pragma unroll
          for (int f = 0; f < NF; ++f) {
            acc[SL::DPI + f] += pi_m[f];
            acc[SL::DPI2 + f] = fmaf(pi_m[f], pi_m[f], acc[SL::DPI2 + f]);
            acc[SL::PHID + f] = fmaf(ph_m[f], D[f], acc[SL::PHID + f]);
            acc[SL::DPHI + f] += ph_m[f];
            acc[SL::DPHI2 + f] = fmaf(ph_m[f], ph_m[f], acc[SL::DPHI2 + f]);
          }
          acc[SL::V] += dVv;
        }
#pragma unroll
        for (int f = 0; f < NF; ++f) phi_out[f * S + o] = ph_m[f];
      }
    }
#pragma unroll
    for (int f = 0; f < NF; ++f) {
      so_mm[f] = so_m[f];
      so_m[f] = so_new[f];
      smid_m[f] = smid_new[f];
      ph_m[f] = cur_ph[f];
      pi_m[f] = cur_pi[f];
    }
  }

  // ---- block partials -------------------------------------------------------
  double accd[NQ];
#pragma unroll
  for (int q = 0; q < NQ; ++q) accd[q] = (double)acc[q];
  __syncthreads();
  block_sum<NQ>(accd, sred, sout);
  if (tid < NQ) d.partials[(size_t)cta * kNQ + tid] = sout[tid];
  __threadfence();
  __syncthreads();
  if (tid == 0) {
    const unsigned int t = atomicAdd(d.ticket, 1u);
    s_last = (t == (unsigned int)(d.ncta - 1));
  }
  __syncthreads();
  if (!s_last) return;
  __threadfence();

  // ---- last block: fixed-order fold of the partials -----------------------
  double tot[NQ];
#pragma unroll
  for (int q = 0; q < NQ; ++q) {
    double s = 0.0, comp = 0.0;  // Neumaier
    for (int c = tid; c < d.ncta; c += kThreads) {
      const double x = __ldcg(&d.partials[(size_t)c * kNQ + q]);
      const double t = s + x;
      comp += (fabs(s) >= fabs(x)) ? (s - t) + x : (x - t) + s;
      s = t;
    }
    tot[q] = s + comp;
  }
  block_sum<NQ>(tot, sred, sout);
  if (tid != 0) return;

  Background nb = *bgp;  // (identical to bg: nobody else writes it during the launch)
  const double Sd = (double)d.S;
  double sum_pi2 = 0.0, sum_phiD = 0.0, sum_V = 0.0;
  double fpi2[NF], fphiD[NF], fdphi[NF], fdphi2[NF];
  if constexpr (PREC == PREC_FP64) {
#pragma unroll
    for (int f = 0; f < NF; ++f) {
      fpi2[f] = sout[SL::PI2 + f];
      fphiD[f] = sout[SL::PHID + f];
      fdphi[f] = (mode == MODE_FLUSH) ? sout[SL::DPHI + f] : 0.0;
      fdphi2[f] = (mode == MODE_FLUSH) ? sout[SL::DPHI2 + f] : 0.0;
    }
    sum_V = sout[SL::V];
  } else {
#pragma unroll
    for (int f = 0; f < NF; ++f) {
      // sum (pi0 + dpi)^2 = S pi0^2 + 2 pi0 sum dpi + sum dpi^2
      fpi2[f] = fma(Sd * pi0s[f], pi0s[f], fma(2.0 * pi0s[f], sout[SL::DPI + f], sout[SL::DPI2 + f]));
      fphiD[f] = sout[SL::PHID + f];  // sum (phi0 + d) D[d] = sum d D[d]  (sum D = 0)
      fdphi[f] = sout[SL::DPHI + f];
      fdphi2[f] = sout[SL::DPHI2 + f];
    }
    sum_V = fma(Sd, V0, sout[SL::V]);  // sum V = S V(phi0) + sum dV
  }
#pragma unroll
  for (int f = 0; f < NF; ++f) { sum_pi2 += fpi2[f]; sum_phiD += fphiD[f]; }

  double a = k.a, pa = k.pa;
  bool ok = is_fin(sum_pi2) && is_fin(sum_phiD) && is_fin(sum_V);
  if (mode == MODE_SWEEP) {
    // Phi_H3(h): p_a += h a^3 [sum phi D/(a^2 dx^2) - 4 sum V]
    pa = pa + k.h * (a * sum_phiD * d.dx2inv - 4.0 * (a * a * a) * sum_V);
    nb.eta = bg.eta + k.h;
    nb.h_prev = k.h;
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
      // shifted-data mean and variance: K = shift (FP64) or phi0 (split)
      const double K = (PREC == PREC_FP64) ? bg.shift[f] : phi0s[f];
      const double m1 = fdphi[f] / Sd;
      nb.mean[f] = K + m1;
      nb.var[f] = fdphi2[f] / Sd - m1 * m1;
      ok = ok && is_fin(fdphi[f]) && is_fin(fdphi2[f]);
      // the next flush shifts by the mean just measured (keeps the variance well-conditioned)
      if (PREC == PREC_FP64) nb.shift[f] = nb.mean[f];
    }
    nb.s_V = sum_V;
  }
  nb.a = a;
  nb.pa = pa;
  nb.sum_pi2 = sum_pi2;
  if constexpr (PREC == PREC_SPLIT) {
#pragma unroll
    for (int f = 0; f < NF; ++f) {
      nb.phi0[f] = phi0s[f];
      nb.mu_phi[f] = fdphi[f] / Sd;
      if (mode == MODE_SWEEP) {
        nb.pi0[f] = pi0s[f];
        nb.mu_pi[f] = sout[SL::DPI + f] / Sd;
      }
      ok = ok && is_fin(phi0s[f]) && is_fin(pi0s[f]);
    }
  }
  ok = ok && is_fin(a) && is_fin(pa);
  if (!ok) {
    nb.error = 1;
    nb.mode = MODE_IDLE;
  }
  *bgp = nb;
  *d.ticket = 0u;
  __threadfence();
}

// Launch helper: dispatch (model, stencil) at runtime to a template instance.
template <int PREC>
cudaError_t launch_sweep_impl(int model, int stencil, const LaunchTable& t, int grid,
                              cudaStream_t s) {
  const dim3 g(grid), b(kThreads);
#define PYCOOL_CASE(M, ST)                                               \
  if (model == M && stencil == ST) {                                     \
    sweep_kernel<M, ST, PREC><<<g, b, 0, s>>>(t);                        \
    return cudaGetLastError();                                           \
  }
  PYCOOL_CASE(M_FREE, 7) PYCOOL_CASE(M_FREE, 27)
  PYCOOL_CASE(M_CHAOTIC2, 7) PYCOOL_CASE(M_CHAOTIC2, 27)
  PYCOOL_CASE(M_OSCILLON, 7) PYCOOL_CASE(M_OSCILLON, 27)
  PYCOOL_CASE(M_QBALL, 7) PYCOOL_CASE(M_QBALL, 27)
#undef PYCOOL_CASE
  return cudaErrorInvalidValue;
}

}  // namespace pycool
