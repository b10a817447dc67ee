// An allocation-free entry point: one fused stage sweep (or one synchronising
// flush sweep) of the FP64 form whose scratch memory -- the background record,
// the launch descriptor, the per-block partial sums and the ticket -- lives in
// a file-scope device array instead of memory the caller or the library
// allocates.  It is for callers that cannot call cudaMalloc: code whose device
// memory is owned by another allocator (a framework's caching allocator or a
// pre-reserved arena that leaves nothing to cudaMalloc), and latency-sensitive
// host loops that cannot afford cudaMalloc/cudaFree, which may synchronise the
// whole device.  The caller passes the field arrays; nothing else is needed.
#include <cuda_runtime.h>

#include <cmath>
#include <cstring>
#include <mutex>

#include "../../include/pycool.h"
#include "internal.cuh"
#include "runtime.h"

#define PYCOOL_API extern "C" __attribute__((visibility("default")))

using namespace pycool;

namespace {

// The shared scratch.  Every GPU that loads this library holds it until the
// process exits.  Layout: [Background][SimDesc][workspace: tickets, fault word,
// partial sums (the simulation workspace layout)].
constexpr size_t kOffBg = 0;
constexpr size_t kOffDesc = 1024;
constexpr size_t kOffWs = 4096;
constexpr size_t kWsAvail = PYCOOL_NOALLOC_SCRATCH_BYTES - kOffWs;
static_assert(sizeof(Background) <= kOffDesc - kOffBg, "background record does not fit");
static_assert(sizeof(SimDesc) <= kOffWs - kOffDesc, "descriptor does not fit");

static __device__ __align__(256) unsigned char g_noalloc_scratch[PYCOOL_NOALLOC_SCRATCH_BYTES];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
char* g_base[kMaxDevices] = {nullptr};

// Device address of the scratch array on the current device (looked up once
// per device, with that device current).
cudaError_t scratch_base(char** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lk(g_mu);
  if (!g_base[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return e;
    g_base[dev] = (char*)p;
  }
  *out = g_base[dev];
  return cudaSuccess;
}

bool aligned16(const void* p) { return ((uintptr_t)p & 15) == 0; }

// Do the byte ranges [a, a + bytes) and [b, b + bytes) share a byte?
bool overlap(const void* a, const void* b, size_t bytes) {
  const uintptr_t x = (uintptr_t)a, y = (uintptr_t)b;
  return x < y + bytes && y < x + bytes;
}

}  // namespace

PYCOOL_API size_t pycool_noalloc_max_blocks(void) {
  // the workspace grows with the block count: largest count that fits
  int lo = 0, hi = (int)(kWsAvail / (kNQ * sizeof(double)));
  while (lo < hi) {
    const int mid = (lo + hi + 1) / 2;
    Layout L;
    workspace_layout(mid, L);
    if (L.ws_bytes <= kWsAvail) lo = mid; else hi = mid - 1;
  }
  return (size_t)lo;
}

PYCOOL_API pycool_status pycool_sweep_noalloc(const pycool_config* cfg, const double* phi_in,
                                              const double* pi_in, double* phi_out,
                                              double* pi_out, int32_t flush,
                                              pycool_stage_state* state, void* cuda_stream) {
  pycool_status st = validate(cfg);
  if (st != PYCOOL_OK) return st;
  // FP64 form, conformal steps (the state record carries no physical-time step)
  if (cfg->precision != PYCOOL_FP64 || cfg->time_step != PYCOOL_TIME_CONFORMAL ||
      cfg->model >= kRuntimeModelBase)
    return PYCOOL_E_INVALID;
  if (!state || !phi_in || !pi_in || !phi_out || (!flush && !pi_out)) return PYCOOL_E_INVALID;
  if (!aligned16(phi_in) || !aligned16(pi_in) || !aligned16(phi_out) ||
      (pi_out && !aligned16(pi_out)))
    return PYCOOL_E_INVALID;
  if (!(state->a > 0.0) || !std::isfinite(state->a)) return PYCOOL_E_INVALID;
  // p_a from H = 0 is taken by a flush only (a run starts with one)
  if (!flush && state->init_pa) return PYCOOL_E_INVALID;
  // the sweep reads neighbours of phi_in while it writes phi_out (and pi_out):
  // an output that shares memory with an input, or with the other output,
  // would be read after it was overwritten
  const size_t bytes = (size_t)model_nfields(cfg->model) * (size_t)cfg->n * (size_t)cfg->n *
                       (size_t)cfg->n * sizeof(double);
  if (overlap(phi_out, phi_in, bytes) || overlap(phi_out, pi_in, bytes)) return PYCOOL_E_INVALID;
  if (!flush && (overlap(pi_out, pi_in, bytes) || overlap(pi_out, phi_in, bytes) ||
                 overlap(pi_out, phi_out, bytes)))
    return PYCOOL_E_INVALID;
  const Layout L = layout_for(*cfg);
  if (L.ws_bytes > kWsAvail) return PYCOOL_E_INVALID;  // too large for the scratch
  cudaStream_t stream = (cudaStream_t)cuda_stream;
  char* base = nullptr;
  cudaError_t e = scratch_base(&base);
  if (e != cudaSuccess) return PYCOOL_E_CUDA;

  // descriptor: the caller's arrays are buffer 0 (read) and buffer 1 (written)
  SimDesc d;
  fill_desc(d, *cfg, L, base + kOffBg, base + kOffWs);
  d.phi[0] = const_cast<double*>(phi_in);
  d.phi[1] = phi_out;
  d.pi[0] = const_cast<double*>(pi_in);
  d.pi[1] = flush ? const_cast<double*>(pi_in) : pi_out;  // a flush leaves pi unchanged
  if (encode_tensor_maps(d) != cudaSuccess) return PYCOOL_E_CUDA;

  Background b;
  std::memset(&b, 0, sizeof(b));
  b.a = state->a;
  b.pa = (flush && state->init_pa) ? 0.0 : state->pa;
  b.eta = state->eta;
  b.h_prev = state->h_prev;
  b.sum_pi2 = state->sum_pi2;
  b.stage = state->stage;
  b.steps_done = state->steps_done;
  b.sweeps_left = 1;
  b.mode = flush ? MODE_FLUSH : MODE_SWEEP;
  b.cur = 0;
  b.init_pa = (flush && state->init_pa) ? 1 : 0;

  // the shared scratch keeps the last call's contents: tickets and fault must start at 0
  if (cudaMemcpyAsync(base + kOffDesc, &d, sizeof(d), cudaMemcpyHostToDevice, stream) !=
          cudaSuccess ||
      cudaMemcpyAsync(base + kOffBg, &b, sizeof(b), cudaMemcpyHostToDevice, stream) !=
          cudaSuccess ||
      cudaMemsetAsync(base + kOffWs, 0, L.off_partials, stream) != cudaSuccess)
    return PYCOOL_E_CUDA;
  LaunchTable t;
  std::memset(&t, 0, sizeof(t));
  t.count = 1;
  t.cta_offset[0] = 0;
  t.cta_offset[1] = L.geo.ncta;
  t.desc[0] = (const SimDesc*)(base + kOffDesc);
  if (launch_sweep(d, t, L.geo.ncta, stream) != cudaSuccess) return PYCOOL_E_CUDA;
  Background r;
  int32_t fault = 0;
  if (cudaMemcpyAsync(&r, base + kOffBg, sizeof(r), cudaMemcpyDeviceToHost, stream) !=
          cudaSuccess ||
      cudaMemcpyAsync(&fault, d.fault, sizeof(fault), cudaMemcpyDeviceToHost, stream) !=
          cudaSuccess ||
      cudaStreamSynchronize(stream) != cudaSuccess)
    return PYCOOL_E_CUDA;
  if (fault) return PYCOOL_E_TIMEOUT;

  state->a = r.a;
  state->pa = r.pa;
  state->eta = r.eta;
  state->h_prev = r.h_prev;
  state->sum_pi2 = r.sum_pi2;
  state->stage = r.stage;
  state->steps_done = r.steps_done;
  state->init_pa = 0;
  state->error = r.error;
  if (flush) observables(r, d, cfg->mpl, cfg->rho_rad0, cfg->rho_mat0, &state->obs);
  return r.error ? PYCOOL_E_NONFINITE : PYCOOL_OK;
}
