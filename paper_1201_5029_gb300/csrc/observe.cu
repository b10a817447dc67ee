// Output-interval observables (Sec. 2.1 Eq. rho-pres with the gradient stencil
// of Eq. G; the spectra of the post-processing, Sec. 2.4), computed at a
// synchronised state on the device:
//   energy_fields : rho(x) and P(x) at every site (7-, 27- or 13-point G),
//       rho = sum_i [pi_i^2/(2 a^6) + G[phi_i]/(2 a^2 dx^2)] + V(phi),
//       P   = sum_i [pi_i^2/(2 a^6) - G[phi_i]/(6 a^2 dx^2)] - V(phi),
//       (a potential given at run time: V from its compiled kernel, run on
//       the same state just before),
//       G[phi](x) = 1/2 sum_alpha c_d(alpha) (phi(alpha) - phi(x))^2;
//     the split forms take the differences phi(alpha) - phi(x) from the
//     fluctuations alone (the background cancels) and V in float64 at
//     phi0 + fluctuation;
//   field_values : one field or momentum of the current state in float64
//     (the input of the spectrum's transform);
//   spectrum_bins : the shell sums of |F_k|^2 / S^2 over the half spectrum of
//     a real transform (modes with a conjugate outside it count twice), one
//     block per shell summing its modes in a fixed host-made order, so the
//     result is reproducible bit for bit.
// These run at output times only; each is one pass over the lattice
// (memory-bound, plain loads).
#include <cufft.h>

#include <cstring>

#include "internal.cuh"
#include "models.cuh"
#include "runtime.h"

namespace pycool {

namespace {

// A value of field f at site i of a buffer, in float64: FP64 stores it,
// the split forms store the fluctuation (float or a double-float pair).
template <int PREC>
__device__ __forceinline__ double fluct_at(const void* buf, size_t i) {
  if constexpr (PREC == PREC_FP64) {
    return __ldg(static_cast<const double*>(buf) + i);
  } else if constexpr (PREC == PREC_SPLIT) {
    return (double)__ldg(static_cast<const float*>(buf) + i);
  } else {
    const float2 v = __ldg(static_cast<const float2*>(buf) + i);
    return (double)v.x + (double)v.y;
  }
}

struct ObsArgs {
  const void* phi;
  const void* pi;
  double* rho;
  double* P;
  int n, nf;
  const double* Vext;   // potentials given at run time: V at every site (the compiled kernel's)
  double a, dx2inv;
  double phi0[kMaxFields], pi0[kMaxFields];   // split forms: background (0 for FP64)
  double params[8], derived[4];
};

template <int MODEL, int STENCIL, int PREC>
__global__ void __launch_bounds__(256) energy_fields_kernel(const ObsArgs o) {
  using P = Pot<MODEL>;
  constexpr int NF = P::NF;
  const double c[4] = {0.0, STENCIL == 27 ? 14.0 / 30.0 : 1.0, STENCIL == 27 ? 3.0 / 30.0 : 0.0,
                       STENCIL == 27 ? 1.0 / 30.0 : 0.0};
  const int n = o.n;
  const size_t nn = (size_t)n * n, S = nn * n;
  const typename P::K pk = P::prep(o.params, o.derived);
  const double a2 = o.a * o.a, a6 = a2 * a2 * a2;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < S;
       i += (size_t)gridDim.x * blockDim.x) {
    const int x = (int)(i % n), y = (int)((i / n) % n), z = (int)(i / nn);
    double kin = 0.0, grad = 0.0, f[NF];
#pragma unroll
    for (int fi = 0; fi < NF; ++fi) {
      const void* pb = static_cast<const char*>(o.phi) + (size_t)fi * S * prec_word(PREC);
      const void* qb = static_cast<const char*>(o.pi) + (size_t)fi * S * prec_word(PREC);
      const double ctr = fluct_at<PREC>(pb, i);
      double G = 0.0;
      if constexpr (STENCIL == 13) {
        // the 13-point stencil: the sites at +-1 (weight 16/12) and +-2
        // (weight -1/12) along each axis
        const double ck[2] = {16.0 / 12.0, -1.0 / 12.0};
#pragma unroll
        for (int axis = 0; axis < 3; ++axis)
#pragma unroll
          for (int k = 1; k <= 2; ++k)
#pragma unroll
            for (int sgn = -1; sgn <= 1; sgn += 2) {
              const int o = sgn * k;
              const int zz = axis == 0 ? (z + o + 2 * n) % n : z;
              const int yy = axis == 1 ? (y + o + 2 * n) % n : y;
              const int xx = axis == 2 ? (x + o + 2 * n) % n : x;
              const double diff = fluct_at<PREC>(pb, ((size_t)zz * n + yy) * n + xx) - ctr;
              G = fma(0.5 * ck[k - 1], diff * diff, G);
            }
      } else {
        for (int dz = -1; dz <= 1; ++dz)
          for (int dy = -1; dy <= 1; ++dy)
            for (int dx = -1; dx <= 1; ++dx) {
              const int cls = (dz != 0) + (dy != 0) + (dx != 0);
              if (cls == 0 || c[cls] == 0.0) continue;
              const int zz = (z + dz + n) % n, yy = (y + dy + n) % n, xx = (x + dx + n) % n;
              const double diff = fluct_at<PREC>(pb, ((size_t)zz * n + yy) * n + xx) - ctr;
              G = fma(0.5 * c[cls], diff * diff, G);
            }
      }
      const double q = o.pi0[fi] + fluct_at<PREC>(qb, i);
      kin = fma(q, q, kin);
      grad += G;
      f[fi] = o.phi0[fi] + ctr;
    }
    double V;
    if constexpr (MODEL == M_RUNTIME1 || MODEL == M_RUNTIME2) {
      V = o.Vext[i];
    } else {
      double dV[NF];
      P::eval(pk, f, dV, V);
    }
    const double k = kin / (2.0 * a6), g = grad * o.dx2inv / a2;
    o.rho[i] = k + 0.5 * g + V;
    o.P[i] = k - g / 6.0 - V;
  }
}

template <int PREC>
__global__ void field_values_kernel(const void* buf, double base, double* out, size_t S) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < S;
       i += (size_t)gridDim.x * blockDim.x)
    out[i] = base + fluct_at<PREC>(buf, i);
}

// One block per shell: the shell's modes (indices into the half spectrum, in
// the host's order), |F|^2 times 2 for modes whose conjugate lies outside the
// half spectrum, summed per thread in order, then a fixed tree over the block.
__global__ void __launch_bounds__(256) spectrum_bins_kernel(const cufftDoubleComplex* spec, int n,
                                                            const int32_t* order,
                                                            const int32_t* start, double invS2,
                                                            double* power) {
  __shared__ double red[256];
  const int b = blockIdx.x;
  const int nh = n / 2 + 1;
  double acc = 0.0;
  for (int j = start[b] + threadIdx.x; j < start[b + 1]; j += blockDim.x) {
    const int m = __ldg(&order[j]);
    const int kx = m % nh;
    const bool twice = kx > 0 && 2 * kx != n;
    const cufftDoubleComplex v = spec[m];
    const double p = fma(v.x, v.x, v.y * v.y);
    acc += twice ? 2.0 * p : p;
  }
  red[threadIdx.x] = acc;
  __syncthreads();
  for (int h = 128; h > 0; h >>= 1) {
    if ((int)threadIdx.x < h) red[threadIdx.x] += red[threadIdx.x + h];
    __syncthreads();
  }
  if (threadIdx.x == 0) power[b] = red[0] * invS2;
}

ObsArgs obs_args(const SimDesc& d, const Background& b) {
  ObsArgs o;
  memset(&o, 0, sizeof(o));
  o.phi = d.phi[b.cur & 1];
  o.pi = d.pi[(b.cur >> 1) & 1];
  o.n = d.n;
  o.nf = d.nf;
  o.a = b.a;
  o.dx2inv = d.dx2inv;
  for (int f = 0; f < d.nf; ++f) {
    o.phi0[f] = d.prec == PREC_FP64 ? 0.0 : b.phi0[f];
    o.pi0[f] = d.prec == PREC_FP64 ? 0.0 : b.pi0[f];
  }
  for (int i = 0; i < 8; ++i) o.params[i] = d.params[i];
  for (int i = 0; i < 4; ++i) o.derived[i] = d.derived[i];
  return o;
}

unsigned grid_for(size_t work) {
  const size_t g = (work + 255) / 256;
  return (unsigned)(g < 152 * 32 ? g : 152 * 32);
}

}  // namespace

cudaError_t launch_energy_fields(const SimDesc& d, const Background& b, double* rho, double* P,
                                 cudaStream_t s) {
  ObsArgs o = obs_args(d, b);
  o.rho = rho;
  o.P = P;
  o.Vext = d.rt_V;
  const unsigned g = grid_for((size_t)d.S);
#define PYCOOL_OBS(M, ST, PR)                                                            \
  if (d.model == M && d.stencil == ST && d.prec == PR) {                                 \
    energy_fields_kernel<M, ST, PR><<<g, 256, 0, s>>>(o);                               \
    return cudaGetLastError();                                                           \
  }
#define PYCOOL_OBS_M(M, PR) PYCOOL_OBS(M, 7, PR) PYCOOL_OBS(M, 27, PR) PYCOOL_OBS(M, 13, PR)
#define PYCOOL_OBS_P(PR)                                                                 \
  PYCOOL_OBS_M(M_FREE, PR) PYCOOL_OBS_M(M_CHAOTIC2, PR) PYCOOL_OBS_M(M_OSCILLON, PR)      \
  PYCOOL_OBS_M(M_QBALL, PR)
  PYCOOL_OBS_P(PREC_FP64)
  PYCOOL_OBS_P(PREC_SPLIT)
  PYCOOL_OBS_P(PREC_DD)
  PYCOOL_OBS_M(M_RUNTIME1, PREC_FP64)
  PYCOOL_OBS_M(M_RUNTIME2, PREC_FP64)
#undef PYCOOL_OBS_P
#undef PYCOOL_OBS_M
#undef PYCOOL_OBS
  return cudaErrorInvalidValue;
}

cudaError_t launch_field_values(const SimDesc& d, const Background& b, int which, int f,
                                double* out, cudaStream_t s) {
  const size_t S = (size_t)d.S;
  const void* buf = which == 0 ? d.phi[b.cur & 1] : d.pi[(b.cur >> 1) & 1];
  buf = static_cast<const char*>(buf) + (size_t)f * S * prec_word(d.prec);
  const double base = d.prec == PREC_FP64 ? 0.0 : (which == 0 ? b.phi0[f] : b.pi0[f]);
  const unsigned g = grid_for(S);
  if (d.prec == PREC_FP64) field_values_kernel<PREC_FP64><<<g, 256, 0, s>>>(buf, base, out, S);
  else if (d.prec == PREC_SPLIT) field_values_kernel<PREC_SPLIT><<<g, 256, 0, s>>>(buf, base, out, S);
  else field_values_kernel<PREC_DD><<<g, 256, 0, s>>>(buf, base, out, S);
  return cudaGetLastError();
}

cudaError_t launch_spectrum_bins(const void* spec, int n, const int32_t* order,
                                 const int32_t* start, int nbins, double* power, cudaStream_t s) {
  const double S = (double)n * n * n;
  spectrum_bins_kernel<<<nbins, 256, 0, s>>>(static_cast<const cufftDoubleComplex*>(spec), n,
                                             order, start, 1.0 / (S * S), power);
  return cudaGetLastError();
}

}  // namespace pycool
