// Growth functions of the linearised evolution (Sec. 2.2): the background
// fields, a and p_a evolve without the perturbations (H^(2) neglected, Eqs.
// a-lin, phi-0) and every Fourier mode of the perturbations obeys the linear
// equations of Eq. Phik-1, in which a mode enters only through k_eff^2.  One
// thread takes one distinct k_eff^2 and advances the 2N_f x 2N_f transfer
// matrix T of its modes, (dPhi, dPi)(eta) = T (dPhi, dPi)(0), through the same
// split-Hamiltonian stages as the lattice (Sec. 2.3):
//   Phi_H1(h): a   -= p_a h / (6 V_L m_pl^2)
//   Phi_H2(h): p_a += V_L [sum_i pi0_i^2 / a^3 - rho_m0] h,
//              phi0 += pi0 h / a^2,   T_dPhi += T_dPi h / a^2
//   Phi_H3(h): p_a -= 4 V_L a^3 V(phi0) h,   pi0 -= a^4 V'(phi0) h,
//              T_dPi -= [k_eff^2 a^2 / dx^2 + a^4 M(phi0)] T_dPhi h
// with M the matrix of second derivatives of V at the background.  Every
// thread evolves the (identical) background itself, so threads never wait on
// one another; the work is FP64 scalar arithmetic, a few hundred operations
// per stage and k_eff^2 value.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include "internal.cuh"
#include "models.cuh"
#include "runtime.h"

namespace pycool {

struct LinArgs {
  const double* k2;       // distinct k_eff^2 values (dimensionless symbols)
  long long nk;
  double* T;              // out: nk x (2N_f)^2, row-major (rows dPhi_0.., dPi_0..)
  double* bg;             // out: a, p_a, phi0[N_f], pi0[N_f] (written by thread 0)
  double a0, pa0, phi0[2], pi0[2];
  double w[kMaxStages];
  int nstages;
  long long steps;
  double dt, dx2inv, VL, inv6VLm2, rho_m0;
  double params[8], derived[4];
};

// Second derivatives of the potentials of Sec. 3 at the background.
template <int MODEL> struct Hess;
template <> struct Hess<M_FREE> {
  __device__ static void get(const double* p, const double*, const double*, double (&M)[1][1]) {
    M[0][0] = p[0];
  }
};
template <> struct Hess<M_CHAOTIC2> {   // V = m2 phi^2/2 + g2 phi^2 chi^2/2
  __device__ static void get(const double* p, const double*, const double* f, double (&M)[2][2]) {
    M[0][0] = p[0] + p[1] * f[1] * f[1];
    M[0][1] = M[1][0] = 2.0 * p[1] * f[0] * f[1];
    M[1][1] = p[1] * f[0] * f[0];
  }
};
template <> struct Hess<M_OSCILLON> {   // V = m2 x^2/2 - lam x^4/4 + g x^6/6
  __device__ static void get(const double* p, const double*, const double* f, double (&M)[1][1]) {
    const double x2 = f[0] * f[0];
    M[0][0] = p[0] - 3.0 * p[1] * x2 + 5.0 * p[2] * x2 * x2;
  }
};
template <> struct Hess<M_QBALL> {      // V = m2 u (1 + K ln(u/M^2)), u = |phi|^2/2
  __device__ static void get(const double* p, const double* dv, const double* f,
                             double (&M)[2][2]) {
    const double u = 0.5 * (f[0] * f[0] + f[1] * f[1]);
    const double fac = p[0] * (1.0 + p[1] + p[1] * (log(u) - dv[0]));
    const double c = p[0] * p[1] / u;
    M[0][0] = fac + c * f[0] * f[0];
    M[0][1] = M[1][0] = c * f[0] * f[1];
    M[1][1] = fac + c * f[1] * f[1];
  }
};

template <int MODEL>
__global__ void __launch_bounds__(128) linear_growth(const LinArgs a) {
  using P = Pot<MODEL>;
  constexpr int NF = P::NF, N2 = 2 * NF;
  const long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= a.nk) return;
  const typename P::K pk = P::prep(a.params, a.derived);
  const double q = a.k2[k] * a.dx2inv;   // k_eff^2 / dx^2
  double A = a.a0, PA = a.pa0, f0[NF], p0[NF], T[N2][N2];
#pragma unroll
  for (int i = 0; i < NF; ++i) { f0[i] = a.phi0[i]; p0[i] = a.pi0[i]; }
#pragma unroll
  for (int r = 0; r < N2; ++r)
#pragma unroll
    for (int c = 0; c < N2; ++c) T[r][c] = (r == c) ? 1.0 : 0.0;

  auto h1 = [&](double h) { A = A - PA * a.inv6VLm2 * h; };
  auto h2 = [&](double h) {
    double s2 = 0.0;
#pragma unroll
    for (int i = 0; i < NF; ++i) s2 += p0[i] * p0[i];
    const double a2 = A * A;
    PA = PA + a.VL * (s2 / (a2 * A) - a.rho_m0) * h;
#pragma unroll
    for (int i = 0; i < NF; ++i) f0[i] = f0[i] + p0[i] / a2 * h;
#pragma unroll
    for (int i = 0; i < NF; ++i)
#pragma unroll
      for (int c = 0; c < N2; ++c) T[i][c] = T[i][c] + T[NF + i][c] / a2 * h;
  };
  auto h3 = [&](double h) {
    double dV[NF], V, M[NF][NF];
    P::eval(pk, f0, dV, V);
    Hess<MODEL>::get(a.params, a.derived, f0, M);
    const double a2 = A * A, a4 = a2 * a2;
#pragma unroll
    for (int i = 0; i < NF; ++i)
#pragma unroll
      for (int c = 0; c < N2; ++c) {
        double m = 0.0;
#pragma unroll
        for (int j = 0; j < NF; ++j) m += M[i][j] * T[j][c];
        T[NF + i][c] = T[NF + i][c] - (q * a2 * T[i][c] + a4 * m) * h;
      }
    PA = PA - 4.0 * a.VL * (a2 * A) * V * h;
#pragma unroll
    for (int i = 0; i < NF; ++i) p0[i] = p0[i] - a4 * dV[i] * h;
  };

  for (long long s = 0; s < a.steps; ++s)
    for (int i = 0; i < a.nstages; ++i) {
      const double h = a.w[i] * a.dt;
      h1(0.5 * h);
      h2(0.5 * h);
      h3(h);
      h2(0.5 * h);
      h1(0.5 * h);
    }
  double* out = a.T + (size_t)k * N2 * N2;
#pragma unroll
  for (int r = 0; r < N2; ++r)
#pragma unroll
    for (int c = 0; c < N2; ++c) out[r * N2 + c] = T[r][c];
  if (k == 0) {
    a.bg[0] = A;
    a.bg[1] = PA;
#pragma unroll
    for (int i = 0; i < NF; ++i) { a.bg[2 + i] = f0[i]; a.bg[2 + NF + i] = p0[i]; }
  }
}

cudaError_t launch_linear_growth(int model, const LinArgs& a, cudaStream_t s) {
  const unsigned grid = (unsigned)((a.nk + 127) / 128);
  switch (model) {
    case M_FREE: linear_growth<M_FREE><<<grid, 128, 0, s>>>(a); break;
    case M_CHAOTIC2: linear_growth<M_CHAOTIC2><<<grid, 128, 0, s>>>(a); break;
    case M_OSCILLON: linear_growth<M_OSCILLON><<<grid, 128, 0, s>>>(a); break;
    case M_QBALL: linear_growth<M_QBALL><<<grid, 128, 0, s>>>(a); break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

}  // namespace pycool

using namespace pycool;

// The distinct values of k_eff^2 (the symbol of -D on plane waves, Eq. D)
// over the n^3 lattice modes, and each mode's index into them.  Values that
// differ by less than 1e-12 (equal symbols reached through different cosines)
// count as one.
extern "C" __attribute__((visibility("default"))) pycool_status pycool_linear_modes(
    int32_t n, int32_t stencil, double* values, int64_t cap, int64_t* count, int32_t* index) {
  if (n < 1 || n > 1024 || !count || cap < 0 ||
      (stencil != PYCOOL_STENCIL_7PT && stencil != PYCOOL_STENCIL_ISO27))
    return PYCOOL_E_INVALID;
  // coefficients by neighbour class (number of non-zero offsets), Eq. D
  const double c7[4] = {-6.0, 1.0, 0.0, 0.0};
  const double c27[4] = {-128.0 / 30.0, 14.0 / 30.0, 3.0 / 30.0, 1.0 / 30.0};
  const double* c = stencil == PYCOOL_STENCIL_7PT ? c7 : c27;
  // one axis: wave number m (numpy FFT order) -> cos(2 pi m / n)
  std::vector<double> cs(n);
  for (int m = 0; m < n; ++m) {
    const int mm = m <= (n - 1) / 2 ? m : m - n;
    cs[m] = std::cos(2.0 * M_PI * mm / n);
  }
  const size_t S = (size_t)n * n * n;
  std::vector<double> k2(S);
  for (int z = 0; z < n; ++z)
    for (int y = 0; y < n; ++y)
      for (int x = 0; x < n; ++x) {
        const double cz = cs[z], cy = cs[y], cx = cs[x];
        // sum over the offsets of each class of c_d cos(k.o): products of cosines
        const double sym = c[0] + 2.0 * c[1] * (cz + cy + cx) +
                           4.0 * c[2] * (cz * cy + cz * cx + cy * cx) + 8.0 * c[3] * cz * cy * cx;
        k2[((size_t)z * n + y) * n + x] = -sym;
      }
  std::vector<double> sorted(k2);
  std::sort(sorted.begin(), sorted.end());
  std::vector<double> vals;
  for (double v : sorted)
    if (vals.empty() || v - vals.back() > 1e-12 * std::fmax(1.0, std::fabs(v))) vals.push_back(v);
  *count = (int64_t)vals.size();
  if (values) {
    if (cap < (int64_t)vals.size()) return PYCOOL_E_INVALID;
    for (size_t i = 0; i < vals.size(); ++i) values[i] = vals[i];
  }
  if (index) {
    for (size_t i = 0; i < S; ++i) {
      // the last value not above k2[i] + tolerance
      const double v = k2[i];
      auto it = std::upper_bound(vals.begin(), vals.end(), v + 1e-12 * std::fmax(1.0, std::fabs(v)));
      index[i] = (int32_t)((it - vals.begin()) - 1);
    }
  }
  return PYCOOL_OK;
}

extern "C" __attribute__((visibility("default"))) pycool_status pycool_linear_growth(
    const pycool_config* cfg, double a0, double pa0, const double* phi0, const double* pi0,
    const double* k2, int64_t nk, int64_t steps, double* T, double* background,
    void* cuda_stream) {
  const pycool_status v = validate(cfg);
  if (v != PYCOOL_OK) return v;
  if (!phi0 || !pi0 || !k2 || !T || !background || nk < 1 || steps < 0 || !(a0 > 0.0) ||
      !std::isfinite(pa0))
    return PYCOOL_E_INVALID;
  const int nf = model_nfields(cfg->model);
  LinArgs a;
  std::memset(&a, 0, sizeof(a));
  a.nk = nk;
  a.a0 = a0;
  a.pa0 = pa0;
  for (int i = 0; i < nf; ++i) { a.phi0[i] = phi0[i]; a.pi0[i] = pi0[i]; }
  a.nstages = stage_table(cfg->order, a.w);
  a.steps = steps;
  a.dt = cfg->dt;
  const double dx = cfg->L / cfg->n;
  a.dx2inv = 1.0 / (dx * dx);
  a.VL = (double)cfg->n * cfg->n * cfg->n;
  a.inv6VLm2 = std::isinf(cfg->mpl) ? 0.0 : 1.0 / (6.0 * a.VL * cfg->mpl * cfg->mpl);
  a.rho_m0 = cfg->rho_mat0;
  for (int i = 0; i < 8; ++i) a.params[i] = cfg->params[i];
  if (cfg->model == PYCOOL_MODEL_QBALL) a.derived[0] = std::log(cfg->params[2] * cfg->params[2]);
  const size_t n2 = (size_t)(2 * nf) * (2 * nf);
  cudaStream_t s = (cudaStream_t)cuda_stream;
  double *dk = nullptr, *dT = nullptr, *dbg = nullptr;
  pycool_status st = PYCOOL_OK;
  if (cudaMalloc((void**)&dk, (size_t)nk * sizeof(double)) != cudaSuccess ||
      cudaMalloc((void**)&dT, (size_t)nk * n2 * sizeof(double)) != cudaSuccess ||
      cudaMalloc((void**)&dbg, 8 * sizeof(double)) != cudaSuccess) {
    st = PYCOOL_E_NOMEM;
  } else {
    a.k2 = dk;
    a.T = dT;
    a.bg = dbg;
    if (cudaMemcpyAsync(dk, k2, (size_t)nk * sizeof(double), cudaMemcpyHostToDevice, s) !=
            cudaSuccess ||
        launch_linear_growth(cfg->model, a, s) != cudaSuccess ||
        cudaMemcpyAsync(T, dT, (size_t)nk * n2 * sizeof(double), cudaMemcpyDeviceToHost, s) !=
            cudaSuccess ||
        cudaMemcpyAsync(background, dbg, (size_t)(2 + 2 * nf) * sizeof(double),
                        cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess)
      st = PYCOOL_E_CUDA;
  }
  cudaFree(dk);
  cudaFree(dT);
  cudaFree(dbg);
  return st;
}
