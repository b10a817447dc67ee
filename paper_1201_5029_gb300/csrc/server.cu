// Serving: many simulations resident on one GPU, advanced together.
//
// A persistent host thread owns the device work.  Requests (config, initial-
// condition recipe, seed, steps) queue up; the thread admits them while the
// HBM budget and the slot count allow, sub-allocating their state from one
// arena reserved at start-up.  Admitted simulations get device-generated
// initial conditions (Philox4x32-10 counter-based normals, Box-Muller), an
// initial reduction sweep (p_a from the constraint) and their step count, then
// join the group of resident simulations that share a kernel instance (model,
// precision, stencil, staging path, vector width).  One launch per group
// advances every member by one stage: each member's stage index, weights,
// coefficients and sums live in its own device records, so members of any
// order and lattice size share a launch and finish independently (their blocks
// return at once when their record says idle).  A group replays K launches as
// a CUDA graph on its own stream, rebuilt only when its membership changes.
// Finished members (record idle after their flush) are retired at graph
// boundaries: their observables are read, the latency from submission is
// recorded and their memory returns to the arena.
//
// Large FP64 members (side a multiple of 32, at least persist_min_n, 256 by
// default) run on the persistent kernel instead: between the groups' graph
// replays, each gets one cooperative launch of as many stage sweeps as a graph
// holds, alone on the GPU (a cooperative grid holds every SM, so it never
// shares the device with another launch).  The launch leaves the merged stage
// boundary pending, as a per-stage launch does; the member's last launch ends
// with the flush.  Which path a member takes depends on its own config only.
//
// Per-member arithmetic and reduction order depend only on that member's
// lattice, so a result is bit-identical whether the simulation ran alone or in
// a mix.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <cmath>
#include <condition_variable>
#include <cstdio>
#include <cstring>
#include <deque>
#include <iterator>
#include <limits>
#include <map>
#include <memory>
#include <mutex>
#include <new>
#include <thread>
#include <vector>

#include "../../include/pycool.h"
#include "internal.cuh"
#include "runtime.h"

#define PYCOOL_API extern "C" __attribute__((visibility("default")))

using namespace pycool;

namespace {

// default side from which FP64 members run on the persistent kernel
constexpr int kPersistMinN = 256;

// ---------------------------------------------------------------------------
// Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11): ten rounds of
//   (c0, c1, c2, c3) -> (hi(M1 c2) ^ c1 ^ k0, lo(M1 c2), hi(M0 c0) ^ c3 ^ k1, lo(M0 c0)),
// the key advanced by (W0, W1) before every round but the first.
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint4 philox4x32_10(uint4 c, uint2 k) {
  const uint32_t M0 = 0xD2511F53u, M1 = 0xCD9E8D57u, W0 = 0x9E3779B9u, W1 = 0xBB67AE85u;
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    if (r > 0) { k.x += W0; k.y += W1; }
    const uint32_t hi0 = __umulhi(M0, c.x), lo0 = M0 * c.x;
    const uint32_t hi1 = __umulhi(M1, c.z), lo1 = M1 * c.z;
    c = make_uint4(hi1 ^ c.y ^ k.x, lo1, hi0 ^ c.w ^ k.y, lo0);
  }
  return c;
}

// Standard normal `comp` (0..3) of counter block `blk` of array `arr`:
// u = (x + 1/2) 2^-32 in (0, 1); Box-Muller on (u0, u1) -> comps 0, 1 and on
// (u2, u3) -> comps 2, 3 (cos for even, sin for odd).
__device__ __forceinline__ double normal_at(uint64_t seed, uint32_t arr, uint32_t blk, int comp) {
  const uint4 r = philox4x32_10(make_uint4(blk, arr, 0u, 0u),
                                make_uint2((uint32_t)seed, (uint32_t)(seed >> 32)));
  const double s = 2.3283064365386963e-10;  // 2^-32
  const uint32_t a = comp < 2 ? r.x : r.z, b = comp < 2 ? r.y : r.w;
  const double u1 = ((double)a + 0.5) * s, u2 = ((double)b + 0.5) * s;
  const double rad = sqrt(-2.0 * log(u1));
  const double th = 6.283185307179586 * u2;
  return (comp & 1) ? rad * sin(th) : rad * cos(th);
}

// White-noise initial conditions into buffer 0.  Element e of field f uses
// normal (e mod 4) of counter block e/4 of array f (phi) or N_f + f (pi):
//   FP64 : phi_f = bg_f + noise z,  pi_f = mom_f + noise z
//   split: the fluctuations noise z in float32 (bg, mom are the background)
__global__ void ic_white_kernel(void* phi, void* pi, long long S, int nf, int split, double bg0,
                                double bg1, double mom0, double mom1, double noise,
                                unsigned long long seed) {
  const long long total = S * nf;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
       i += (long long)gridDim.x * blockDim.x) {
    const int f = (int)(i / S);
    const long long e = i - (long long)f * S;
    const double zp = normal_at(seed, (uint32_t)f, (uint32_t)(e >> 2), (int)(e & 3));
    const double zq = normal_at(seed, (uint32_t)(nf + f), (uint32_t)(e >> 2), (int)(e & 3));
    if (split) {
      ((float*)phi)[i] = (float)(noise * zp);
      ((float*)pi)[i] = (float)(noise * zq);
    } else {
      ((double*)phi)[i] = (f == 0 ? bg0 : bg1) + noise * zp;
      ((double*)pi)[i] = (f == 0 ? mom0 : mom1) + noise * zq;
    }
  }
}

double now_s() {
  return std::chrono::duration<double>(std::chrono::steady_clock::now().time_since_epoch())
      .count();
}

size_t round256(size_t x) { return (x + 255) & ~(size_t)255; }

// First-fit sub-allocator over one device arena (256-byte granules).
class Arena {
 public:
  bool init(size_t bytes) {
    bytes &= ~(size_t)255;
    if (bytes == 0 || injected_alloc_failure() ||
        cudaMalloc((void**)&base_, bytes) != cudaSuccess) {
      cudaGetLastError();
      base_ = nullptr;
      return false;
    }
    size_ = bytes;
    free_[0] = bytes;
    return true;
  }
  void release() {
    if (base_) cudaFree(base_);
    base_ = nullptr;
  }
  char* alloc(size_t bytes) {
    bytes = round256(bytes);
    for (auto it = free_.begin(); it != free_.end(); ++it) {
      if (it->second >= bytes) {
        const size_t off = it->first, sz = it->second;
        free_.erase(it);
        if (sz > bytes) free_[off + bytes] = sz - bytes;
        return base_ + off;
      }
    }
    return nullptr;
  }
  void free(char* p, size_t bytes) {
    bytes = round256(bytes);
    const size_t off = (size_t)(p - base_);
    auto next = free_.lower_bound(off);
    if (next != free_.end() && off + bytes == next->first) {
      bytes += next->second;
      next = free_.erase(next);
    }
    if (next != free_.begin()) {
      auto prev = std::prev(next);
      if (prev->first + prev->second == off) {
        prev->second += bytes;
        return;
      }
    }
    free_[off] = bytes;
  }
  size_t capacity() const { return size_; }

 private:
  char* base_ = nullptr;
  size_t size_ = 0;
  std::map<size_t, size_t> free_;
};

struct Request {
  uint64_t ticket;
  pycool_config cfg;
  pycool_ic ic;
  uint64_t seed;
  int64_t steps;
  double t_submit;
};

struct Result {
  bool done = false;
  pycool_status status = PYCOOL_OK;
  pycool_observables obs{};
};

struct Member {
  Request req;
  Layout L;
  SimDesc hdesc;
  char* state = nullptr;
  char* ws = nullptr;
  int group = -1;              // per-stage members: their group; persistent members: -1
  bool persist = false;        // advanced by the persistent kernel, alone on the GPU
  PParams pp;                  // its launch parameters (plan, tensor maps, barrier count)
  long long sweeps_left = 0;   // stage sweeps still to run (persistent members)
};

struct Group {
  int model = 0, prec = 0, stencil = 0, tma = 0, vx = 0;
  std::vector<int> members;   // slot indices
  cudaGraphExec_t graph = nullptr;
  bool dirty = true;
  cudaStream_t stream = nullptr;
};

}  // namespace

struct pycool_server {
  int max_slots = 0;
  int stages_per_graph = 8;
  // FP64 requests whose side is a multiple of 32 and at least this run on the
  // persistent kernel (0: none); read at admission
  std::atomic<int> persist_min_n{kPersistMinN};
  Arena arena;
  int device = 0;
  cudaStream_t setup = nullptr, capture = nullptr;
  std::vector<std::unique_ptr<Member>> slots;   // resident simulations (nullptr = free)
  std::vector<Group> groups;
  Background* h_bg = nullptr;                   // pinned mirror, one record per slot
  int32_t* h_fault = nullptr;                   // pinned, one fault word per slot
  std::mutex mu;
  std::condition_variable cv_work, cv_done;
  std::deque<Request> queue;
  std::map<uint64_t, Result> results;
  std::vector<uint64_t> cancel;                 // resident tickets to retire at the next boundary
  uint64_t next_ticket = 1;
  bool stop = false;
  pycool_status fatal = PYCOOL_OK;
  std::vector<double> latencies;
  double site_updates = 0.0, t_first = -1.0, t_last = -1.0;
  std::thread thr;
};

namespace {

// A request's layout: the persistent kernel's (sim_layout) for FP64 members on
// a lattice it takes (side a multiple of 32, at least persist_min_n), else the
// per-stage kernels'.
Layout member_layout(const pycool_server* s, const pycool_config& c, bool* persist) {
  const int mn = s->persist_min_n.load();
  if (mn > 0 && c.precision == PYCOOL_FP64 && c.n >= mn && c.n % 32 == 0) {
    const Layout L = sim_layout(c);
    if (L.off_prows) {
      *persist = true;
      return L;
    }
  }
  *persist = false;
  return layout_for(c);
}

size_t footprint(const pycool_server* s, const pycool_config& c) {
  bool persist = false;
  const Layout L = member_layout(s, c, &persist);
  return round256(L.state_bytes) + round256(L.ws_bytes);
}

int group_for(pycool_server* s, const SimDesc& d) {
  for (size_t g = 0; g < s->groups.size(); ++g) {
    const Group& G = s->groups[g];
    if (G.model == d.model && G.prec == d.prec && G.stencil == d.stencil && G.tma == d.tma &&
        G.vx == d.vx)
      return (int)g;
  }
  Group G;
  G.model = d.model; G.prec = d.prec; G.stencil = d.stencil; G.tma = d.tma; G.vx = d.vx;
  if (cudaStreamCreateWithFlags(&G.stream, cudaStreamNonBlocking) != cudaSuccess) return -1;
  s->groups.push_back(G);
  return (int)s->groups.size() - 1;
}

#define SCK(call)                                        \
  do {                                                   \
    cudaError_t e__ = (call);                            \
    if (e__ != cudaSuccess) {                            \
      std::fprintf(stderr, "pycool server: %s: %s\n", #call, cudaGetErrorString(e__)); \
      return PYCOOL_E_CUDA;                              \
    }                                                    \
  } while (0)

// Admission: memory, descriptor, initial conditions, initial reduction, step count.
pycool_status admit(pycool_server* s, const Request& r, int slot) {
  auto m = std::make_unique<Member>();
  m->req = r;
  bool persist = false;
  m->L = member_layout(s, r.cfg, &persist);
  m->state = s->arena.alloc(m->L.state_bytes);
  if (!m->state) return PYCOOL_E_NOMEM;
  m->ws = s->arena.alloc(m->L.ws_bytes);
  if (!m->ws) {
    s->arena.free(m->state, m->L.state_bytes);
    return PYCOOL_E_NOMEM;
  }
  fill_desc(m->hdesc, r.cfg, m->L, m->state, m->ws);
  SCK(encode_tensor_maps(m->hdesc));
  const SimDesc& d = m->hdesc;
  const bool split = d.prec == PREC_SPLIT;
  Background b;
  std::memset(&b, 0, sizeof(b));
  b.a = r.ic.a0 > 0.0 ? r.ic.a0 : 1.0;
  b.init_pa = 1;
  b.mode = MODE_FLUSH;  // the first launch only reduces (h_prev = 0)
  for (int f = 0; f < d.nf; ++f) {
    if (split) {
      b.phi0[f] = r.ic.background[f];
      b.pi0[f] = r.ic.momentum[f];
    }
  }
  cudaStream_t st = s->setup;
  SCK(cudaMemcpyAsync(m->state + m->L.off_desc, &m->hdesc, sizeof(SimDesc), cudaMemcpyHostToDevice, st));
  SCK(cudaMemcpyAsync(m->state + m->L.off_bg, &b, sizeof(b), cudaMemcpyHostToDevice, st));
  SCK(cudaMemsetAsync(m->ws, 0, m->L.off_partials, st));
  ic_white_kernel<<<2048, 256, 0, st>>>(d.phi[0], d.pi[0], (long long)d.S, d.nf, split ? 1 : 0,
                                        r.ic.background[0], r.ic.background[1], r.ic.momentum[0],
                                        r.ic.momentum[1], r.ic.noise, (unsigned long long)r.seed);
  SCK(cudaGetLastError());
  LaunchTable t;
  std::memset(&t, 0, sizeof(t));
  t.count = 1;
  t.cta_offset[1] = m->L.geo.ncta;
  t.desc[0] = (const SimDesc*)(m->state + m->L.off_desc);
  SCK(launch_sweep(d, t, m->L.geo.ncta, st));
  if (persist) {   // the plan for this device, the tensor maps, the occupancy check
    bool fits = false;
    const pycool_status ps =
        persist_setup(r.cfg, m->hdesc, m->L, m->state, m->ws, st, m->pp, &fits);
    if (ps == PYCOOL_E_CUDA) return ps;
    // a plan the host check refuses, or one block per SM that does not fit:
    // the per-stage kernels (the layout holds theirs too)
    persist = ps == PYCOOL_OK && fits;
  }
  if (persist) {
    SCK(cudaStreamSynchronize(st));
    m->persist = true;
    m->sweeps_left = (long long)r.steps * d.nstages;
    s->slots[slot] = std::move(m);
    return PYCOOL_OK;
  }
  SCK(launch_arm((Background*)(m->state + m->L.off_bg), (long long)r.steps * d.nstages, st));
  SCK(cudaStreamSynchronize(st));
  const int g = group_for(s, d);
  if (g < 0) return PYCOOL_E_CUDA;
  m->group = g;
  s->groups[g].members.push_back(slot);
  s->groups[g].dirty = true;
  s->slots[slot] = std::move(m);
  return PYCOOL_OK;
}

// Capture K stage launches of every member of a group into one graph.
pycool_status rebuild(pycool_server* s, Group& G) {
  if (G.graph) {
    cudaGraphExecDestroy(G.graph);
    G.graph = nullptr;
  }
  G.dirty = false;
  if (G.members.empty()) return PYCOOL_OK;
  std::vector<LaunchTable> tables;
  std::vector<int> grids;
  for (size_t i = 0; i < G.members.size(); i += kMaxMembers) {
    LaunchTable t;
    std::memset(&t, 0, sizeof(t));
    int off = 0;
    for (size_t j = i; j < G.members.size() && j < i + kMaxMembers; ++j) {
      const Member& m = *s->slots[G.members[j]];
      t.cta_offset[t.count] = off;
      t.desc[t.count] = (const SimDesc*)(m.state + m.L.off_desc);
      off += m.L.geo.ncta;
      t.count++;
    }
    t.cta_offset[t.count] = off;
    tables.push_back(t);
    grids.push_back(off);
  }
  const SimDesc& d0 = s->slots[G.members[0]]->hdesc;
  cudaGraph_t graph = nullptr;
  SCK(cudaStreamBeginCapture(s->capture, cudaStreamCaptureModeThreadLocal));
  cudaError_t le = cudaSuccess;
  for (int k = 0; k < s->stages_per_graph && le == cudaSuccess; ++k)
    for (size_t i = 0; i < tables.size() && le == cudaSuccess; ++i)
      le = launch_sweep(d0, tables[i], grids[i], s->capture);
  const cudaError_t ee = cudaStreamEndCapture(s->capture, &graph);
  SCK(le);
  SCK(ee);
  const cudaError_t ie = cudaGraphInstantiate(&G.graph, graph, 0);
  cudaGraphDestroy(graph);
  SCK(ie);
  return PYCOOL_OK;
}

void retire(pycool_server* s, int slot, const Background& b, int32_t fault, bool cancelled) {
  Member& m = *s->slots[slot];
  Result res;
  res.done = true;
  res.status = fault ? PYCOOL_E_TIMEOUT
                     : (b.error ? PYCOOL_E_NONFINITE : (cancelled ? PYCOOL_E_CANCELLED : PYCOOL_OK));
  observables(b, m.hdesc, m.req.cfg.mpl, m.req.cfg.rho_rad0, m.req.cfg.rho_mat0, &res.obs);
  const double t = now_s();
  {
    std::lock_guard<std::mutex> lk(s->mu);
    s->results[m.req.ticket] = res;
    if (!cancelled) {   // the latency and rate figures describe completed requests only
      s->latencies.push_back(t - m.req.t_submit);
      s->site_updates += (double)m.hdesc.S * (double)b.sweeps_done;
      s->t_last = t;
    }
  }
  s->cv_done.notify_all();
  if (m.group >= 0) {
    Group& G = s->groups[m.group];
    G.members.erase(std::find(G.members.begin(), G.members.end(), slot));
    G.dirty = true;
  }
  s->arena.free(m.ws, m.L.ws_bytes);
  s->arena.free(m.state, m.L.state_bytes);
  s->slots[slot].reset();
}

void fail_all(pycool_server* s, pycool_status st) {
  std::lock_guard<std::mutex> lk(s->mu);
  s->fatal = st;
  for (auto& kv : s->results)
    if (!kv.second.done) {
      kv.second.done = true;
      kv.second.status = st;
    }
  s->cv_done.notify_all();
}

void server_loop(pycool_server* s) {
  cudaSetDevice(s->device);
  for (;;) {
    // 1. admission
    std::vector<Request> take;
    int resident = 0;
    for (auto& p : s->slots) resident += p ? 1 : 0;
    {
      std::unique_lock<std::mutex> lk(s->mu);
      if (resident == 0)
        s->cv_work.wait(lk, [&] { return s->stop || !s->queue.empty(); });
      if (s->stop) break;
      int free_slots = s->max_slots - resident;
      for (auto it = s->queue.begin(); it != s->queue.end() && free_slots > 0;) {
        take.push_back(*it);
        it = s->queue.erase(it);
        --free_slots;
      }
    }
    std::vector<Request> back;
    for (const Request& r : take) {
      int slot = -1;
      for (int i = 0; i < s->max_slots; ++i)
        if (!s->slots[i]) { slot = i; break; }
      const pycool_status st = slot < 0 ? PYCOOL_E_NOMEM : admit(s, r, slot);
      if (st == PYCOOL_E_NOMEM) {
        back.push_back(r);            // not enough free arena now: wait for a retirement
      } else if (st != PYCOOL_OK) {
        fail_all(s, st);
        return;
      } else {
        std::lock_guard<std::mutex> lk(s->mu);
        if (s->t_first < 0) s->t_first = now_s();
      }
    }
    if (!back.empty()) {
      std::lock_guard<std::mutex> lk(s->mu);
      for (auto it = back.rbegin(); it != back.rend(); ++it) {
        auto c = std::find(s->cancel.begin(), s->cancel.end(), it->ticket);
        if (c != s->cancel.end()) {   // cancelled while it waited for memory
          s->cancel.erase(c);
          s->results[it->ticket].done = true;
          s->results[it->ticket].status = PYCOOL_E_CANCELLED;
          s->cv_done.notify_all();
          continue;
        }
        s->queue.push_front(*it);
      }
    }
    // 2. one graph replay per group, then a copy of every member's record
    bool any = false;
    for (Group& G : s->groups) {
      if (G.members.empty()) continue;
      if (G.dirty && rebuild(s, G) != PYCOOL_OK) { fail_all(s, PYCOOL_E_CUDA); return; }
      if (cudaGraphLaunch(G.graph, G.stream) != cudaSuccess) { fail_all(s, PYCOOL_E_CUDA); return; }
      for (int slot : G.members) {
        const Member& m = *s->slots[slot];
        cudaMemcpyAsync(&s->h_bg[slot], m.state + m.L.off_bg, sizeof(Background),
                        cudaMemcpyDeviceToHost, G.stream);
        cudaMemcpyAsync(&s->h_fault[slot], m.ws + m.L.off_ticket + 128, sizeof(int32_t),
                        cudaMemcpyDeviceToHost, G.stream);
      }
      any = true;
    }
    bool persistent = false;
    for (const auto& p : s->slots) persistent = persistent || (p && p->persist);
    if (!any && !persistent) continue;
    for (Group& G : s->groups) {
      if (G.members.empty()) continue;
      if (cudaStreamSynchronize(G.stream) != cudaSuccess) { fail_all(s, PYCOOL_E_CUDA); return; }
    }
    // 2b. persistent members, one after another, each alone on the GPU (every
    //     group's launches have completed): one cooperative launch of up to a
    //     graph's worth of stage sweeps; the last launch of a member ends with
    //     the flush, the others leave the stage boundary pending
    if (persistent) {
      for (int slot = 0; slot < s->max_slots; ++slot) {
        Member* m = s->slots[slot].get();
        if (!m || !m->persist) continue;
        if (m->sweeps_left > 0) {
          const long long k = std::min<long long>(m->sweeps_left, s->stages_per_graph);
          m->pp.nsweeps = k;
          m->pp.flush = k == m->sweeps_left ? 1 : 0;
          if (launch_persist(m->hdesc, m->pp, m->pp.g.G, s->setup, nullptr) != cudaSuccess) {
            fail_all(s, PYCOOL_E_CUDA);
            return;
          }
          // one grid barrier per pass (the sweeps and the flush, if any)
          m->pp.bar_base += (unsigned long long)(k + m->pp.flush) * (unsigned long long)m->pp.g.G;
          m->sweeps_left -= k;
        }
        cudaMemcpyAsync(&s->h_bg[slot], m->state + m->L.off_bg, sizeof(Background),
                        cudaMemcpyDeviceToHost, s->setup);
        cudaMemcpyAsync(&s->h_fault[slot], m->ws + m->L.off_ticket + 128, sizeof(int32_t),
                        cudaMemcpyDeviceToHost, s->setup);
      }
      if (cudaStreamSynchronize(s->setup) != cudaSuccess) { fail_all(s, PYCOOL_E_CUDA); return; }
    }
    // 3. retire finished members (per-stage: record idle after their flush;
    //    persistent: every sweep and the flush launched), stopped ones (a
    //    non-finite sum) and cancelled ones (every launch has completed here)
    std::vector<uint64_t> cancel;
    {
      std::lock_guard<std::mutex> lk(s->mu);
      cancel.swap(s->cancel);
    }
    for (int slot = 0; slot < s->max_slots; ++slot) {
      if (!s->slots[slot]) continue;
      const Member& m = *s->slots[slot];
      const Background& b = s->h_bg[slot];
      const bool cut = std::find(cancel.begin(), cancel.end(), m.req.ticket) != cancel.end();
      const bool done = m.persist ? m.sweeps_left == 0 : b.mode == MODE_IDLE;
      if (done || b.error || s->h_fault[slot] || cut)
        retire(s, slot, b, s->h_fault[slot], cut && !done);
    }
  }
}

}  // namespace

PYCOOL_API pycool_status pycool_server_create(size_t hbm_budget, int32_t max_slots,
                                              pycool_server** out) {
  if (!out || max_slots <= 0 || hbm_budget < (1u << 20)) return PYCOOL_E_INVALID;
  *out = nullptr;
  pycool_server* s = new (std::nothrow) pycool_server();
  if (!s) return PYCOOL_E_NOMEM;
  s->max_slots = max_slots;
  if (cudaGetDevice(&s->device) != cudaSuccess) { delete s; return PYCOOL_E_CUDA; }
  if (!s->arena.init(hbm_budget)) { delete s; return PYCOOL_E_NOMEM; }
  if (cudaStreamCreateWithFlags(&s->setup, cudaStreamNonBlocking) != cudaSuccess ||
      cudaStreamCreateWithFlags(&s->capture, cudaStreamNonBlocking) != cudaSuccess ||
      cudaMallocHost((void**)&s->h_bg, sizeof(Background) * (size_t)max_slots) != cudaSuccess ||
      cudaMallocHost((void**)&s->h_fault, sizeof(int32_t) * (size_t)max_slots) != cudaSuccess) {
    s->arena.release();
    delete s;
    return PYCOOL_E_CUDA;
  }
  s->slots.resize(max_slots);
  s->thr = std::thread(server_loop, s);
  *out = s;
  return PYCOOL_OK;
}

PYCOOL_API pycool_status pycool_server_submit(pycool_server* s, const pycool_config* cfg,
                                              const pycool_ic* ic, uint64_t seed, int64_t steps,
                                              uint64_t* ticket) {
  if (!s || !cfg || !ic || !ticket || steps < 0) return PYCOOL_E_INVALID;
  const pycool_status st = validate(cfg);
  if (st != PYCOOL_OK) return st;
  if (cfg->precision == PYCOOL_SPLIT_DD) return PYCOOL_E_INVALID;   // no per-stage DD kernel
  if (cfg->model >= kRuntimeModelBase) return PYCOOL_E_INVALID;     // one launch per group only
  if (!std::isfinite(ic->noise) || ic->noise < 0.0) return PYCOOL_E_INVALID;
  if (footprint(s, *cfg) > s->arena.capacity()) return PYCOOL_E_NOMEM;  // could never fit
  Request r;
  r.cfg = *cfg;
  r.ic = *ic;
  r.seed = seed;
  r.steps = steps;
  r.t_submit = now_s();
  {
    std::lock_guard<std::mutex> lk(s->mu);
    if (s->fatal != PYCOOL_OK) return PYCOOL_E_STATE;
    r.ticket = s->next_ticket++;
    s->results[r.ticket] = Result();
    s->queue.push_back(r);
  }
  *ticket = r.ticket;
  s->cv_work.notify_all();
  return PYCOOL_OK;
}

PYCOOL_API pycool_status pycool_server_wait(pycool_server* s, uint64_t ticket, double timeout_s,
                                            pycool_observables* out) {
  if (!s) return PYCOOL_E_INVALID;
  std::unique_lock<std::mutex> lk(s->mu);
  auto it = s->results.find(ticket);
  if (it == s->results.end()) return PYCOOL_E_NOT_FOUND;
  auto ready = [&] { return s->results[ticket].done; };
  if (timeout_s < 0.0) {
    s->cv_done.wait(lk, ready);
  } else if (!s->cv_done.wait_for(lk, std::chrono::duration<double>(timeout_s), ready)) {
    return PYCOOL_E_TIMEOUT;
  }
  const Result r = s->results[ticket];
  s->results.erase(ticket);
  if (out) *out = r.obs;
  return r.status;
}

PYCOOL_API pycool_status pycool_server_cancel(pycool_server* s, uint64_t ticket) {
  if (!s) return PYCOOL_E_INVALID;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    auto it = s->results.find(ticket);
    if (it == s->results.end()) return PYCOOL_E_NOT_FOUND;
    if (it->second.done) return PYCOOL_E_STATE;   // finished already: collect it with wait
    for (auto q = s->queue.begin(); q != s->queue.end(); ++q) {
      if (q->ticket == ticket) {                  // not admitted yet: drop it from the queue
        s->queue.erase(q);
        it->second.done = true;
        it->second.status = PYCOOL_E_CANCELLED;
        s->cv_done.notify_all();
        return PYCOOL_OK;
      }
    }
    s->cancel.push_back(ticket);                  // resident (or being admitted)
  }
  s->cv_work.notify_all();
  return PYCOOL_OK;
}

PYCOOL_API pycool_status pycool_server_set_persistent_min_n(pycool_server* s, int32_t n) {
  if (!s || n < 0 || (n > 0 && (n < 32 || n % 32))) return PYCOOL_E_INVALID;
  s->persist_min_n.store(n);
  return PYCOOL_OK;
}

PYCOOL_API pycool_status pycool_server_stats(pycool_server* s, double* p50_s, double* p99_s,
                                             double* site_updates_per_s, int64_t* completed) {
  if (!s) return PYCOOL_E_INVALID;
  std::lock_guard<std::mutex> lk(s->mu);
  std::vector<double> l = s->latencies;
  std::sort(l.begin(), l.end());
  auto pct = [&](double p) {
    if (l.empty()) return std::numeric_limits<double>::quiet_NaN();
    const size_t i = std::min(l.size() - 1, (size_t)std::ceil(p * (double)l.size()) - 1);
    return l[i];
  };
  if (p50_s) *p50_s = pct(0.50);
  if (p99_s) *p99_s = pct(0.99);
  if (site_updates_per_s)
    *site_updates_per_s = (s->t_last > s->t_first && s->t_first >= 0)
                              ? s->site_updates / (s->t_last - s->t_first)
                              : 0.0;
  if (completed) *completed = (int64_t)l.size();
  return PYCOOL_OK;
}

PYCOOL_API void pycool_server_destroy(pycool_server* s) {
  if (!s) return;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    s->stop = true;
  }
  s->cv_work.notify_all();
  if (s->thr.joinable()) s->thr.join();
  cudaDeviceSynchronize();
  for (Group& G : s->groups) {
    if (G.graph) cudaGraphExecDestroy(G.graph);
    if (G.stream) cudaStreamDestroy(G.stream);
  }
  if (s->setup) cudaStreamDestroy(s->setup);
  if (s->capture) cudaStreamDestroy(s->capture);
  if (s->h_bg) cudaFreeHost(s->h_bg);
  if (s->h_fault) cudaFreeHost(s->h_fault);
  s->arena.release();
  cudaGetLastError();
  delete s;
}
