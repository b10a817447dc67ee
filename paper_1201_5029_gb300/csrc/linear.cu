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
#include <cufft.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <map>
#include <memory>
#include <mutex>
#include <tuple>
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
  const double* bg_in;    // device: initial phi0[N_f], pi0[N_f] (NULL: the fields below)
  double a0, pa0, phi0[2], pi0[2];
  double w[kMaxStages];
  int nstages;
  long long steps;
  int physical;           // d-eta = dt / a at each step's start (Sec. 3.1), else dt
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
  for (int i = 0; i < NF; ++i) {
    f0[i] = a.bg_in ? a.bg_in[i] : a.phi0[i];
    p0[i] = a.bg_in ? a.bg_in[NF + i] : a.pi0[i];
  }
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

  for (long long s = 0; s < a.steps; ++s) {
    const double deta = a.physical ? a.dt / A : a.dt;   // the background's a at the step's start
    for (int i = 0; i < a.nstages; ++i) {
      const double h = a.w[i] * deta;
      h1(0.5 * h);
      h2(0.5 * h);
      h3(h);
      h2(0.5 * h);
      h1(0.5 * h);
    }
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

// The background of lattice fields (Eq. phi-lin): the lattice means of the
// 2 N_f arrays phi_0..phi_{N-1}, pi_0.. (src[j] = array j, S values each),
// summed in a fixed order -- per block a strided range and a fixed tree, then
// the block sums in order by one block -- so the means are reproducible.
constexpr int kMeanBlocks = 128;
__global__ void __launch_bounds__(256) linear_means_partial(const double* const* src, long long S,
                                                            double* part) {
  __shared__ double red[256];
  const int j = blockIdx.y;
  double acc = 0.0;
  for (long long i = blockIdx.x * 256LL + threadIdx.x; i < S; i += (long long)kMeanBlocks * 256)
    acc += src[j][i];
  red[threadIdx.x] = acc;
  __syncthreads();
  for (int h = 128; h > 0; h >>= 1) {
    if ((int)threadIdx.x < h) red[threadIdx.x] += red[threadIdx.x + h];
    __syncthreads();
  }
  if (threadIdx.x == 0) part[(size_t)j * kMeanBlocks + blockIdx.x] = red[0];
}
__global__ void linear_means_fold(const double* part, int narr, double invS, double* bg_in) {
  const int j = threadIdx.x;   // one thread per array
  if (j >= narr) return;
  double s = 0.0;
  for (int b = 0; b < kMeanBlocks; ++b) s += part[(size_t)j * kMeanBlocks + b];
  bg_in[j] = s * invS;         // [phi0_0 .. phi0_{N_f-1}, pi0_0 ..]
}
// dst_f = src_f - mean_f (the perturbations, Eq. phi-lin), into the output
// arrays that later receive the evolved fields
__global__ void linear_subtract(const double* const* src, double* const* dst, long long S,
                                int narr, const double* bg_in) {
  const long long total = S * narr;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
       i += (long long)gridDim.x * blockDim.x) {
    const int j = (int)(i / S);
    const long long e = i - (long long)j * S;
    dst[j][e] = src[j][e] - bg_in[j];
  }
}
// the k = 0 coefficients of the perturbations (zero up to rounding) cleared
__global__ void linear_clear_mean(cufftDoubleComplex* spec, long long half, int nf) {
  const int i = threadIdx.x;
  if (i >= 2 * nf) return;
  spec[(size_t)i * half].x = 0.0;
  spec[(size_t)i * half].y = 0.0;
}

// Each Fourier mode of the perturbations at the later time from its initial
// value (Sec. 2.2, after Eq. Phik-1): y(eta) = T[k_eff^2 of the mode] y(0),
// y = (dPhi_1..dPhi_N, dPi_1..dPi_N), T real, scaled by 1/S for the
// unnormalised inverse transform; the k = 0 coefficient becomes the evolved
// background, so the inverse transform gives background + perturbations.
template <int NF>
__global__ void __launch_bounds__(256) linear_apply(cufftDoubleComplex* __restrict__ spec,
                                                    long long half,
                                                    const int32_t* __restrict__ index,
                                                    const double* __restrict__ T,
                                                    const double* __restrict__ bg_end, double invS) {
  constexpr int N2 = 2 * NF;
  for (long long m = blockIdx.x * (long long)blockDim.x + threadIdx.x; m < half;
       m += (long long)gridDim.x * blockDim.x) {
    cufftDoubleComplex y[N2], r[N2];
#pragma unroll
    for (int j = 0; j < N2; ++j) y[j] = spec[(size_t)j * half + m];
    if (m == 0) {
#pragma unroll
      for (int j = 0; j < N2; ++j) { r[j].x = bg_end[2 + j]; r[j].y = 0.0; }
    } else {
      const double* t = T + (size_t)__ldg(&index[m]) * N2 * N2;
#pragma unroll
      for (int i = 0; i < N2; ++i) {
        double re = 0.0, im = 0.0;
#pragma unroll
        for (int j = 0; j < N2; ++j) {
          const double tij = __ldg(&t[i * N2 + j]);
          re = fma(tij, y[j].x, re);
          im = fma(tij, y[j].y, im);
        }
        r[i].x = re * invS;
        r[i].y = im * invS;
      }
    }
#pragma unroll
    for (int j = 0; j < N2; ++j) spec[(size_t)j * half + m] = r[j];
  }
}

cudaError_t launch_linear_apply(int nf, cufftDoubleComplex* spec, long long half,
                                const int32_t* index, const double* T, const double* bg_end,
                                double invS, cudaStream_t s) {
  const long long want = (half + 255) / 256;
  const unsigned grid = (unsigned)std::min<long long>(want, 152LL * 16);
  if (nf == 1)
    linear_apply<1><<<grid, 256, 0, s>>>(spec, half, index, T, bg_end, invS);
  else
    linear_apply<2><<<grid, 256, 0, s>>>(spec, half, index, T, bg_end, invS);
  return cudaGetLastError();
}

// The distinct k_eff^2 values (ascending) of an n^3 lattice and each mode's
// index into them (modes in numpy FFT order, [z][y][x]).
bool linear_modes_host(int n, int stencil, std::vector<double>& vals, std::vector<int32_t>* index) {
  // coefficients by neighbour class (number of non-zero offsets), Eq. D
  const double c7[4] = {-6.0, 1.0, 0.0, 0.0};
  const double c27[4] = {-128.0 / 30.0, 14.0 / 30.0, 3.0 / 30.0, 1.0 / 30.0};
  const double* c = stencil == PYCOOL_STENCIL_7PT ? c7 : c27;
  const bool fourth = stencil == PYCOOL_STENCIL_4TH;
  // one axis: wave number m (numpy FFT order) -> cos(2 pi m / n); the
  // fourth-order stencil's part of one axis, -(2 (16/12) cos t - 2 (1/12) cos 2t)
  std::vector<double> cs(n), ax4(n);
  for (int m = 0; m < n; ++m) {
    const int mm = m <= (n - 1) / 2 ? m : m - n;
    cs[m] = std::cos(2.0 * M_PI * mm / n);
    ax4[m] = -(2.0 * (16.0 / 12.0) * cs[m] + 2.0 * (-1.0 / 12.0) * std::cos(4.0 * M_PI * mm / n));
  }
  const size_t S = (size_t)n * n * n;
  std::vector<double> k2(S);
  for (int z = 0; z < n; ++z)
    for (int y = 0; y < n; ++y)
      for (int x = 0; x < n; ++x) {
        const double cz = cs[z], cy = cs[y], cx = cs[x];
        double v;
        if (fourth) {   // the centre (-90/12) and the two sites each way along every axis
          v = 90.0 / 12.0 + ax4[z] + ax4[y] + ax4[x];
        } else {
          // sum over the offsets of each class of c_d cos(k.o): products of cosines
          const double sym = c[0] + 2.0 * c[1] * (cz + cy + cx) +
                             4.0 * c[2] * (cz * cy + cz * cx + cy * cx) +
                             8.0 * c[3] * cz * cy * cx;
          v = -sym;
        }
        k2[((size_t)z * n + y) * n + x] = v;
      }
  std::vector<double> sorted(k2);
  std::sort(sorted.begin(), sorted.end());
  vals.clear();
  for (double v : sorted)
    if (vals.empty() || v - vals.back() > 1e-12 * std::fmax(1.0, std::fabs(v))) vals.push_back(v);
  if (index) {
    index->resize(S);
    for (size_t i = 0; i < S; ++i) {
      // the last value not above k2[i] + tolerance
      const double v = k2[i];
      auto it = std::upper_bound(vals.begin(), vals.end(), v + 1e-12 * std::fmax(1.0, std::fabs(v)));
      (*index)[i] = (int32_t)((it - vals.begin()) - 1);
    }
  }
  return true;
}

// Per-process caches of pycool_linear_evolve: the host tables of a lattice
// (distinct k_eff^2 values, each half-spectrum mode's index) per (n, stencil),
// and the forward/inverse FFT plans per (n, N_f, device).  A plan is used
// under its own lock (its stream is set per call).
struct LinTables {
  std::vector<double> vals;
  std::vector<int32_t> hidx;
};
struct LinPlans {
  cufftHandle fwd = 0, inv = 0;
  std::mutex mu;
};
std::mutex g_lin_mu;
std::map<std::pair<int, int>, std::shared_ptr<const LinTables>> g_lin_tables;
std::map<std::tuple<int, int, int>, std::shared_ptr<LinPlans>> g_lin_plans;

std::shared_ptr<const LinTables> linear_tables(int n, int stencil) {
  {
    std::lock_guard<std::mutex> lk(g_lin_mu);
    auto it = g_lin_tables.find({n, stencil});
    if (it != g_lin_tables.end()) return it->second;
  }
  auto t = std::make_shared<LinTables>();
  std::vector<int32_t> full;
  linear_modes_host(n, stencil, t->vals, &full);
  const int nh = n / 2 + 1;
  t->hidx.resize((size_t)n * n * nh);
  for (int z = 0; z < n; ++z)
    for (int y = 0; y < n; ++y)
      for (int x = 0; x < nh; ++x)
        t->hidx[((size_t)z * n + y) * nh + x] = full[((size_t)z * n + y) * n + x];
  std::lock_guard<std::mutex> lk(g_lin_mu);
  return g_lin_tables.emplace(std::make_pair(n, stencil), t).first->second;
}

std::shared_ptr<LinPlans> linear_plans(int n, int nf, int device) {
  std::lock_guard<std::mutex> lk(g_lin_mu);
  auto key = std::make_tuple(n, nf, device);
  auto it = g_lin_plans.find(key);
  if (it != g_lin_plans.end()) return it->second;
  auto p = std::make_shared<LinPlans>();
  int dims[3] = {n, n, n};
  const int S = n * n * n, half = n * n * (n / 2 + 1);
  if (cufftPlanMany(&p->fwd, 3, dims, nullptr, 1, S, nullptr, 1, half, CUFFT_D2Z, nf) !=
      CUFFT_SUCCESS)
    return nullptr;
  if (cufftPlanMany(&p->inv, 3, dims, nullptr, 1, half, nullptr, 1, S, CUFFT_Z2D, nf) !=
      CUFFT_SUCCESS) {
    cufftDestroy(p->fwd);
    return nullptr;
  }
  g_lin_plans.emplace(key, p);
  return p;
}

}  // namespace pycool

using namespace pycool;

// The distinct values of k_eff^2 (the symbol of -D on plane waves, Eq. D)
// over the n^3 lattice modes, and each mode's index into them.  Values that
// differ by less than 1e-12 (equal symbols reached through different cosines)
// count as one.
extern "C" __attribute__((visibility("default"))) pycool_status pycool_linear_modes(
    int32_t n, int32_t stencil, double* values, int64_t cap, int64_t* count, int32_t* index) {
  if (n < 1 || n > 512 || !count || cap < 0 ||
      (stencil != PYCOOL_STENCIL_7PT && stencil != PYCOOL_STENCIL_ISO27 &&
       stencil != PYCOOL_STENCIL_4TH))
    return PYCOOL_E_INVALID;
  std::vector<double> vals;
  std::vector<int32_t> idx;
  linear_modes_host(n, stencil, vals, index ? &idx : nullptr);
  *count = (int64_t)vals.size();
  if (values) {
    if (cap < (int64_t)vals.size()) return PYCOOL_E_INVALID;
    for (size_t i = 0; i < vals.size(); ++i) values[i] = vals[i];
  }
  if (index) std::memcpy(index, idx.data(), idx.size() * sizeof(int32_t));
  return PYCOOL_OK;
}

extern "C" __attribute__((visibility("default"))) pycool_status pycool_linear_growth(
    const pycool_config* cfg, double a0, double pa0, const double* phi0, const double* pi0,
    const double* k2, int64_t nk, int64_t steps, double* T, double* background,
    void* cuda_stream) {
  const pycool_status v = validate(cfg);
  if (v != PYCOOL_OK) return v;
  if (cfg->model >= kRuntimeModelBase) return PYCOOL_E_INVALID;   // no second derivatives
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
  a.physical = cfg->time_step == PYCOOL_TIME_PHYSICAL ? 1 : 0;
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

// The whole linearised evolution of lattice fields on the device.
extern "C" __attribute__((visibility("default"))) pycool_status pycool_linear_evolve(
    const pycool_config* cfg, double a0, double pa0, const double* phi, const double* pi,
    int64_t steps, double* phi_out, double* pi_out, double* background, void* cuda_stream) {
  const pycool_status v = validate(cfg);
  if (v != PYCOOL_OK) return v;
  if (cfg->model >= kRuntimeModelBase) return PYCOOL_E_INVALID;   // no second derivatives
  if (!phi || !pi || !phi_out || !pi_out || !background || steps < 0 || !(a0 > 0.0) ||
      !std::isfinite(pa0) || cfg->n < 2 || cfg->n > 512)
    return PYCOOL_E_INVALID;
  {  // the outputs serve as scratch while the inputs are read: no overlap
    const size_t bytes = (size_t)model_nfields(cfg->model) * cfg->n * cfg->n * cfg->n * 8;
    const uintptr_t in[2] = {(uintptr_t)phi, (uintptr_t)pi};
    const uintptr_t out[2] = {(uintptr_t)phi_out, (uintptr_t)pi_out};
    for (int i = 0; i < 2; ++i)
      for (int j = 0; j < 2; ++j)
        if (out[i] < in[j] + bytes && in[j] < out[i] + bytes) return PYCOOL_E_INVALID;
    if (out[0] < out[1] + bytes && out[1] < out[0] + bytes) return PYCOOL_E_INVALID;
  }
  const int nf = model_nfields(cfg->model);
  const int n = cfg->n;
  const long long S = (long long)n * n * n;
  const long long half = (long long)n * n * (n / 2 + 1);   // coefficients of a real transform
  const std::shared_ptr<const LinTables> tab = linear_tables(n, cfg->stencil);
  const std::vector<double>& vals = tab->vals;
  const std::vector<int32_t>& hidx = tab->hidx;
  int device = 0;
  if (cudaGetDevice(&device) != cudaSuccess) return PYCOOL_E_CUDA;
  const std::shared_ptr<LinPlans> plans = linear_plans(n, nf, device);
  if (!plans) return PYCOOL_E_CUDA;
  std::lock_guard<std::mutex> plan_lock(plans->mu);
  const long long nk = (long long)vals.size();
  const size_t N2 = (size_t)(2 * nf) * (2 * nf);

  LinArgs a;
  std::memset(&a, 0, sizeof(a));
  a.nk = nk;
  a.a0 = a0;
  a.pa0 = pa0;
  a.nstages = stage_table(cfg->order, a.w);
  a.steps = steps;
  a.dt = cfg->dt;
  a.physical = cfg->time_step == PYCOOL_TIME_PHYSICAL ? 1 : 0;
  const double dx = cfg->L / n;
  a.dx2inv = 1.0 / (dx * dx);
  a.VL = (double)S;
  a.inv6VLm2 = std::isinf(cfg->mpl) ? 0.0 : 1.0 / (6.0 * a.VL * cfg->mpl * cfg->mpl);
  a.rho_m0 = cfg->rho_mat0;
  for (int i = 0; i < 8; ++i) a.params[i] = cfg->params[i];
  if (cfg->model == PYCOOL_MODEL_QBALL) a.derived[0] = std::log(cfg->params[2] * cfg->params[2]);

  cudaStream_t s = (cudaStream_t)cuda_stream;
  cufftDoubleComplex* spec = nullptr;   // [phi, pi][N_f][half]
  double *dk = nullptr, *dT = nullptr, *dbg = nullptr, *dpart = nullptr;
  double** dptrs = nullptr;             // [2][2 N_f]: source and destination arrays
  int32_t* didx = nullptr;
  const cufftHandle fwd = plans->fwd, inv = plans->inv;
  pycool_status st = PYCOOL_OK;
  do {
    if (injected_alloc_failure() ||
        cudaMalloc((void**)&spec, (size_t)2 * nf * half * sizeof(cufftDoubleComplex)) !=
            cudaSuccess ||
        cudaMalloc((void**)&dk, (size_t)nk * sizeof(double)) != cudaSuccess ||
        cudaMalloc((void**)&dT, (size_t)nk * N2 * sizeof(double)) != cudaSuccess ||
        cudaMalloc((void**)&dbg, 16 * sizeof(double)) != cudaSuccess ||
        cudaMalloc((void**)&didx, (size_t)half * sizeof(int32_t)) != cudaSuccess ||
        cudaMalloc((void**)&dpart, (size_t)2 * nf * kMeanBlocks * sizeof(double)) != cudaSuccess ||
        cudaMalloc((void**)&dptrs, 8 * sizeof(double*)) != cudaSuccess) {
      cudaGetLastError();
      st = PYCOOL_E_NOMEM;
      break;
    }
    if (cufftSetStream(fwd, s) != CUFFT_SUCCESS || cufftSetStream(inv, s) != CUFFT_SUCCESS) {
      st = PYCOOL_E_CUDA;
      break;
    }
    a.k2 = dk;
    a.T = dT;
    a.bg = dbg;
    a.bg_in = dbg + 8;
    cufftDoubleComplex* sphi = spec;
    cufftDoubleComplex* spi = spec + (size_t)nf * half;
    if (cudaMemcpyAsync(dk, vals.data(), (size_t)nk * sizeof(double), cudaMemcpyHostToDevice, s) !=
            cudaSuccess ||
        cudaMemcpyAsync(didx, hidx.data(), (size_t)half * sizeof(int32_t), cudaMemcpyHostToDevice,
                        s) != cudaSuccess) { st = PYCOOL_E_CUDA; break; }
    // 1. background: the lattice means (fixed-order sums); the perturbations
    //    (fields minus means) go to the output arrays, which serve as the
    //    transforms' real input (the background never enters a transform)
    double* hptrs[8];
    for (int f = 0; f < nf; ++f) {
      hptrs[f] = const_cast<double*>(phi) + (size_t)f * S;
      hptrs[nf + f] = const_cast<double*>(pi) + (size_t)f * S;
      hptrs[4 + f] = phi_out + (size_t)f * S;
      hptrs[4 + nf + f] = pi_out + (size_t)f * S;
    }
    if (cudaMemcpyAsync(dptrs, hptrs, sizeof(hptrs), cudaMemcpyHostToDevice, s) != cudaSuccess) {
      st = PYCOOL_E_CUDA;
      break;
    }
    linear_means_partial<<<dim3(kMeanBlocks, 2 * nf), 256, 0, s>>>(dptrs, S, dpart);
    linear_means_fold<<<1, 32, 0, s>>>(dpart, 2 * nf, 1.0 / (double)S, dbg + 8);
    linear_subtract<<<152 * 8, 256, 0, s>>>(dptrs, dptrs + 4, S, 2 * nf, dbg + 8);
    // 2. forward transforms of the perturbations (every field), k = 0 cleared
    if (cudaGetLastError() != cudaSuccess ||
        cufftExecD2Z(fwd, phi_out, sphi) != CUFFT_SUCCESS ||
        cufftExecD2Z(fwd, pi_out, spi) != CUFFT_SUCCESS) {
      st = PYCOOL_E_CUDA;
      break;
    }
    linear_clear_mean<<<1, 32, 0, s>>>(spec, half, nf);
    // 3. growth functions of the distinct k_eff^2 (background evolved per thread)
    // 4. every mode: T y(0) / S, k = 0 -> the evolved background
    if (cudaGetLastError() != cudaSuccess || launch_linear_growth(cfg->model, a, s) != cudaSuccess ||
        launch_linear_apply(nf, spec, half, didx, dT, dbg, 1.0 / (double)S, s) != cudaSuccess) {
      st = PYCOOL_E_CUDA;
      break;
    }
    // 5. inverse transforms into the caller's arrays
    if (cufftExecZ2D(inv, sphi, phi_out) != CUFFT_SUCCESS ||
        cufftExecZ2D(inv, spi, pi_out) != CUFFT_SUCCESS) {
      st = PYCOOL_E_CUDA;
      break;
    }
    if (cudaMemcpyAsync(background, dbg, (size_t)(2 + 2 * nf) * sizeof(double),
                        cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess)
      st = PYCOOL_E_CUDA;
  } while (0);
  cudaFree(spec);
  cudaFree(dk);
  cudaFree(dT);
  cudaFree(dbg);
  cudaFree(didx);
  cudaFree(dpart);
  cudaFree(dptrs);
  return st;
}
