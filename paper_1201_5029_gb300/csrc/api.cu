// Host runtime behind include/pycool.h: simulation objects, device memory
// layout, CUDA-graph replay of the sweep chain, observables, checkpoints.
#include <cuda_runtime.h>
#include <cufft.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <new>
#include <thread>
#include <vector>

#include "../../include/pycool.h"
#include "models.cuh"
#include "internal.cuh"
#include "runtime.h"

#define PYCOOL_API extern "C" __attribute__((visibility("default")))

using namespace pycool;

namespace pycool {

// ---------------------------------------------------------------------------
// Stage weights (Sec. 2.3): leapfrog; the triple jump of Eq. Phi-rec with
// n = 1 for order 4; the symmetric compositions of Table 1 for orders 6 and 8
// (w_1 outermost, centre = 1 - 2 sum of the listed weights).
// ---------------------------------------------------------------------------
int stage_table(int order, double* w) {
  switch (order) {
    case 2:
      w[0] = 1.0;
      return 1;
    case 4: {
      const double c = std::cbrt(2.0);
      w[0] = w[2] = 1.0 / (2.0 - c);
      w[1] = -c / (2.0 - c);
      return 3;
    }
    case 6: {
      static const double half[3] = {0.78451361047755726382, 0.23557321335935813368,
                                     -1.17767998417887100695};
      double s = 0.0;
      for (int i = 0; i < 3; ++i) { w[i] = w[6 - i] = half[i]; s += half[i]; }
      w[3] = 1.0 - 2.0 * s;
      return 7;
    }
    case 8: {
      static const double half[7] = {0.74167036435061295345,  -0.40910082580003159400,
                                     0.19075471029623837995,  -0.57386247111608226666,
                                     0.29906418130365592384,  0.33462491824529818378,
                                     0.31529309239676659663};
      double s = 0.0;
      for (int i = 0; i < 7; ++i) { w[i] = w[14 - i] = half[i]; s += half[i]; }
      w[7] = 1.0 - 2.0 * s;
      return 15;
    }
    default:
      return -1;
  }
}

int model_nfields(int model) {
  if (model >= kRuntimeModelBase) return runtime_model_nfields(model);
  switch (model) {
    case PYCOOL_MODEL_FREE: return 1;
    case PYCOOL_MODEL_CHAOTIC2: return 2;
    case PYCOOL_MODEL_OSCILLON: return 1;
    case PYCOOL_MODEL_QBALL: return 2;
    default: return -1;
  }
}

static size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

// Blocks of the split forms' initial-mean reduction (a fixed grid, so the
// summation order and the result depend on the lattice alone).
constexpr int kMeanBlocks = 304;

Layout layout_for(const pycool_config& c) {
  Layout L;
  const int nf = model_nfields(c.model);
  const size_t S = (size_t)c.n * c.n * c.n;
  const size_t word = c.precision == PYCOOL_SPLIT_FP32 ? 4 : 8;
  const bool runtime = c.model >= kRuntimeModelBase;
  L.geo = choose_geometry(c.n, (int)word, nf, c.stencil == PYCOOL_STENCIL_4TH || runtime);
  L.field_bytes = align256((size_t)nf * S * word);
  L.off_bg = 0;
  L.off_desc = align256(sizeof(Background));
  L.off_fields = L.off_desc + align256(sizeof(SimDesc));
  L.state_bytes = L.off_fields + 4 * L.field_bytes;
  workspace_layout(L.geo.ncta, L);
  L.off_prows = 0;
  L.off_punits = 0;
  L.off_rt = 0;
  L.off_mean = 0;
  if (runtime) {   // drifted fields, V' (N_f n^3 each) and V (n^3)
    L.off_rt = align256(L.ws_bytes);
    L.ws_bytes = L.off_rt + 2 * align256((size_t)nf * S * 8) + align256(S * 8);
  }
  return L;
}

Layout sim_layout(const pycool_config& c) {
  Layout L = layout_for(c);
  L.off_mean = align256(L.ws_bytes);
  L.ws_bytes = L.off_mean + align256((size_t)2 * kMeanBlocks * sizeof(double));
  // the persistent kernel: n a multiple of 32, compiled models; the 13-point
  // stencil in the FP64 and split-DD forms only (its per-stage fallback,
  // like the split-FP32 form's, keeps the plain geometry)
  const bool persist_ok =
      L.geo.tma || (c.stencil == PYCOOL_STENCIL_4TH && c.n % 32 == 0 &&
                    c.model < kRuntimeModelBase && c.precision != PYCOOL_SPLIT_FP32);
  if (persist_ok) {
    L.off_prows = align256(L.ws_bytes);
    L.off_punits = L.off_prows + align256((size_t)2 * kMaxPBlocks * kNQ * sizeof(double));
    L.ws_bytes = L.off_punits + align256((size_t)kMaxPBlocks * kMaxPUnits * sizeof(int4)) +
                 align256((size_t)(kMaxPBlocks + 1) * sizeof(int));
  }
  return L;
}

// Persistent geometry and work assignment.  Tiles are 32 vx x 16 sites (vx
// sites per lane along x, vx * N_f * word <= 16 bytes).  Each tile's z-axis is
// cut into equal ranges: rc of them for tiles clear of the periodic y boundary,
// rw for the tiles whose halo rows cross it (their TMA copies take one box per
// field instead of one for all fields).  A unit (tile, z-range) costs its
// planes, each of its two z-halo planes counted as a fraction h of a plane
// (FP64: only their drift is recomputed; split: their loads cost about as
// much as the compute), times a penalty for the wrap tiles (split: 1.2,
// measured; FP64, bound by float64 arithmetic: 1).  The units are dealt in
// z-major order (blocks that run together work on neighbouring tiles at the
// same z, so halo rows and columns hit L2), each to the least loaded block; a
// block processes its units in the order dealt.  (rc, rw) minimises the
// busiest block's cost, then the total.
PGeo plan_units(int n, int word, int nf, int prec, int sms, long long l2_bytes,
                std::vector<int4>* units, std::vector<int>* off, int halo) {
  PGeo g;
  std::memset(&g, 0, sizeof(g));
  g.n = n;
  g.halo = halo;
  g.vx = 1;
  for (int v = 4; v >= 1; v /= 2)
    if (v * nf * word <= 16 && n % (32 * v) == 0) { g.vx = v; break; }
  g.tx = 32 * g.vx;
  g.tiles_x = n / g.tx;
  const int tiles_y = n / 16;
  g.ntiles = g.tiles_x * tiles_y;
  // Cost of a block's work, fitted to per-block timings of the persistent
  // kernel on GB300: a plane costs 1 (pen for the tiles at the y wrap, whose
  // halo rows arrive by per-field boxes) and a unit adds 2h (its two z-halo
  // planes and the switch).  In the split form a unit costs ~2 us more
  // than its planes whether or not the stage's traffic stays in L2; in plane
  // units that is h ~1.5 for an L2-resident lattice (fast planes) and ~0.3
  // for a larger one.  The float64 form is bound by its arithmetic: h ~0.25.
  const double stage_bytes = 4.0 * nf * (double)n * n * n * word;   // phi, pi read and written
  const bool l2_resident = l2_bytes > 0 && stage_bytes <= 0.75 * (double)l2_bytes;
  const double h = prec != PREC_SPLIT ? 0.25 : (l2_resident ? 1.5 : 0.3);
  const double pen = prec != PREC_SPLIT ? 1.0 : 1.24;
  constexpr int kMinPiece = 4;   // planes: no unit shorter than this is cut off a chunk
  const int cap = std::min(sms, kMaxPBlocks);
  auto is_wrap = [&](int t) {
    const int ty = t / g.tiles_x;
    return ty == 0 || ty == tiles_y - 1;
  };
  struct U { int z0, z1, t, b; };
  // Deal at target T: the tiles' z-chunks (rc per clear tile, rw per wrap
  // tile) in z-major order, each to the least loaded block (ties to the lower
  // index); a chunk that would take that block past T is cut there and its
  // rest stays at the head of the list.  false: T is too small for cap blocks.
  std::vector<U> base, out;
  std::vector<std::pair<double, int>> heap;
  auto cmp = [](const std::pair<double, int>& x, const std::pair<double, int>& y) {
    return x.first != y.first ? x.first > y.first : x.second > y.second;
  };
  auto chunks = [&](int rc, int rw) {
    base.clear();
    for (int t = 0; t < g.ntiles; ++t) {
      const int R = is_wrap(t) ? rw : rc;
      for (int r = 0; r < R; ++r)
        base.push_back(U{(int)((long long)r * n / R), (int)((long long)(r + 1) * n / R), t, -1});
    }
    std::stable_sort(base.begin(), base.end(), [](const U& x, const U& y) {
      return x.z0 != y.z0 ? x.z0 < y.z0 : x.t < y.t;
    });
  };
  auto deal = [&](double T) -> bool {
    out.clear();
    heap.clear();
    for (int b = 0; b < cap; ++b) heap.push_back({0.0, b});
    std::make_heap(heap.begin(), heap.end(), cmp);
    for (size_t i = 0; i < base.size(); ++i) {
      U u = base[i];
      while (u.z0 < u.z1) {
        std::pop_heap(heap.begin(), heap.end(), cmp);
        auto& top = heap.back();
        const double p = is_wrap(u.t) ? pen : 1.0;
        const int len = u.z1 - u.z0;
        int k = len;
        if (top.first + (len + 2.0 * halo * h) * p > T + 1e-9) {
          k = (int)std::floor((T - top.first) / p - 2.0 * halo * h);
          if (len - k < kMinPiece) k = len - kMinPiece;
          if (k < kMinPiece) return false;   // the least loaded block is full: so are all
        }
        out.push_back(U{u.z0, u.z0 + k, u.t, top.second});
        top.first += (k + 2.0 * halo * h) * p;
        std::push_heap(heap.begin(), heap.end(), cmp);
        u.z0 += k;
      }
    }
    return true;
  };
  auto measure = [&](double& mx, double& tot, int& maxcount, int& used) {
    std::vector<double> load(cap, 0.0);
    std::vector<int> count(cap, 0);
    for (const U& u : out) {
      load[u.b] += (u.z1 - u.z0 + 2.0 * halo * h) * (is_wrap(u.t) ? pen : 1.0);
      count[u.b] += 1;
    }
    mx = *std::max_element(load.begin(), load.end());
    tot = 0.0;
    for (double v : load) tot += v;
    maxcount = *std::max_element(count.begin(), count.end());
    used = 0;
    for (int b = 0; b < cap; ++b) used += count[b] > 0;
  };
  // the smallest feasible T for each chunking (bisection), then the chunking
  // with the least loaded slowest block (ties: less total work, fewer chunks)
  const double work = (double)n * g.tiles_x * ((tiles_y - 2) + 2 * pen);
  double best = 1e300, best_tot = 1e300, best_T = 0.0;
  for (int rc = 1; rc <= std::min(16, std::max(1, n / kMinPiece)); ++rc) {
    const int rws[3] = {rc, (rc * 12 + 9) / 10, (rc * 13 + 9) / 10};
    for (int j = 0; j < 3; ++j) {
      const int rw = std::min(rws[j], std::max(1, n / kMinPiece));
      if (j > 0 && rw == std::min(rws[j - 1], std::max(1, n / kMinPiece))) continue;
      if (pen == 1.0 && rw != rc) continue;
      chunks(rc, rw);
      double lo = work / cap, hi = (double)n * pen + 2.0 * halo * h * pen + lo;
      while (!deal(hi)) hi *= 2.0;
      for (int it = 0; it < 40 && hi - lo > 1e-3; ++it) {
        const double mid = 0.5 * (lo + hi);
        if (deal(mid)) hi = mid; else lo = mid;
      }
      deal(hi);
      double mx, tot;
      int maxcount, used;
      measure(mx, tot, maxcount, used);
      if (maxcount > kMaxPUnits) continue;
      if (mx < best - 1e-9 || (mx < best + 1e-9 && tot < best_tot - 1e-9)) {
        best = mx;
        best_tot = tot;
        best_T = hi;
        g.rc = rc;
        g.rw = rw;
      }
    }
  }
  chunks(g.rc, g.rw);
  deal(best_T);
  // blocks without a unit (small lattices) are dropped: ties go to the lower
  // index, so the used blocks are 0 .. G-1
  int G = 0;
  for (const U& u : out) G = std::max(G, u.b + 1);
  g.G = G;
  g.nunits = (int)out.size();
  if (units && off) {
    off->assign(G + 1, 0);
    for (const U& u : out) (*off)[u.b + 1] += 1;
    for (int b = 0; b < G; ++b) (*off)[b + 1] += (*off)[b];
    units->assign(out.size(), int4{0, 0, 0, 0});
    std::vector<int> fill(off->begin(), off->end() - 1);
    for (const U& u : out)   // per block, in the order dealt
      (*units)[fill[u.b]++] =
          int4{(u.t % g.tiles_x) * g.tx, (u.t / g.tiles_x) * 16, u.z0, u.z1 - u.z0 + 2 * halo};
  }
  return g;
}

// A plan the kernel may trust: every unit inside the lattice, every (tile, z)
// pair in exactly one unit, at most kMaxPUnits units per block.
static bool check_plan(const PGeo& g, const std::vector<int4>& units, const std::vector<int>& off) {
  if (g.G < 1 || g.G > kMaxPBlocks || (int)off.size() != g.G + 1 || off[0] != 0 ||
      off[g.G] != (int)units.size() || (int)units.size() != g.nunits)
    return false;
  std::vector<unsigned char> seen((size_t)g.ntiles * g.n, 0);
  for (int b = 0; b < g.G; ++b) {
    if (off[b + 1] < off[b] || off[b + 1] - off[b] > kMaxPUnits) return false;
    for (int i = off[b]; i < off[b + 1]; ++i) {
      const int4 u = units[i];
      const int planes = u.w - 2 * g.halo;
      if (u.x < 0 || u.x % g.tx || u.x + g.tx > g.n || u.y < 0 || u.y % 16 || u.y + 16 > g.n ||
          u.z < 0 || planes < 1 || u.z + planes > g.n)
        return false;
      const size_t t = (size_t)(u.y / 16) * g.tiles_x + u.x / g.tx;
      for (int z = u.z; z < u.z + planes; ++z)
        if (seen[t * g.n + z]++) return false;
    }
  }
  for (unsigned char c : seen)
    if (c != 1) return false;
  return true;
}

PYCOOL_API pycool_status pycool_persist_plan(int32_t n, int32_t nf, int32_t precision,
                                             int32_t stencil, int32_t sms, int64_t l2_bytes,
                                             int32_t* geo, int32_t* units, int32_t cap_units,
                                             int32_t* uoff, int32_t cap_blocks) {
  if (n < 32 || n % 32 || (nf != 1 && nf != 2) || sms < 1 || l2_bytes < 0 || !geo ||
      (precision != PYCOOL_FP64 && precision != PYCOOL_SPLIT_FP32 &&
       precision != PYCOOL_SPLIT_DD) ||
      (stencil != PYCOOL_STENCIL_7PT && stencil != PYCOOL_STENCIL_ISO27 &&
       stencil != PYCOOL_STENCIL_4TH) ||
      (stencil == PYCOOL_STENCIL_4TH && precision == PYCOOL_SPLIT_FP32))
    return PYCOOL_E_INVALID;
  const int prec = precision == PYCOOL_FP64 ? PREC_FP64
                   : (precision == PYCOOL_SPLIT_DD ? PREC_DD : PREC_SPLIT);
  std::vector<int4> u;
  std::vector<int> off;
  const PGeo g = plan_units(n, prec_word(prec), nf, prec, sms, l2_bytes, &u, &off,
                            stencil == PYCOOL_STENCIL_4TH ? 2 : 1);
  if (!check_plan(g, u, off)) return PYCOOL_E_INVALID;
  const int32_t vals[10] = {g.n, g.vx, g.tx, g.tiles_x, g.ntiles, g.rc, g.rw, g.nunits, g.G,
                            g.halo};
  for (int i = 0; i < 10; ++i) geo[i] = vals[i];
  if (units) {
    if (cap_units < g.nunits) return PYCOOL_E_INVALID;
    for (int i = 0; i < g.nunits; ++i) {
      units[4 * i + 0] = u[i].x; units[4 * i + 1] = u[i].y;
      units[4 * i + 2] = u[i].z; units[4 * i + 3] = u[i].w;
    }
  }
  if (uoff) {
    if (cap_blocks < g.G) return PYCOOL_E_INVALID;
    for (int b = 0; b <= g.G; ++b) uoff[b] = off[b];
  }
  return PYCOOL_OK;
}

void workspace_layout(int ncta, Layout& L) {
  const size_t ngroups = ((size_t)ncta + kGroup - 1) / kGroup;
  L.off_ticket = 0;
  L.off_gticket = 256;
  L.off_partials = L.off_gticket + align256(ngroups * sizeof(unsigned int));
  L.off_gpartials = L.off_partials + align256((size_t)ncta * kNQ * sizeof(double));
  L.ws_bytes = L.off_gpartials + align256(ngroups * kNQ * sizeof(double));
}

pycool_status validate(const pycool_config* c) {
  if (!c) return PYCOOL_E_INVALID;
  if (c->n < 1 || c->n > 1024) return PYCOOL_E_INVALID;
  if (model_nfields(c->model) < 0) return PYCOOL_E_INVALID;
  if (c->order != 2 && c->order != 4 && c->order != 6 && c->order != 8) return PYCOOL_E_INVALID;
  if (c->precision != PYCOOL_FP64 && c->precision != PYCOOL_SPLIT_FP32 &&
      c->precision != PYCOOL_SPLIT_DD)
    return PYCOOL_E_INVALID;
  if (c->stencil != PYCOOL_STENCIL_7PT && c->stencil != PYCOOL_STENCIL_ISO27 &&
      c->stencil != PYCOOL_STENCIL_4TH)
    return PYCOOL_E_INVALID;
  // the fourth-order stencil: a per-stage kernel in the FP64 and split-FP32
  // forms, the persistent kernel in the FP64 and split-DD forms (n % 32 == 0)
  if (c->stencil == PYCOOL_STENCIL_4TH && c->precision == PYCOOL_SPLIT_DD && c->n % 32 != 0)
    return PYCOOL_E_INVALID;
  // a potential given at run time: the FP64 form (any stencil)
  if (c->model >= kRuntimeModelBase && c->precision != PYCOOL_FP64) return PYCOOL_E_INVALID;
  // its +-2 neighbours wrap once around the lattice at most: n >= 4
  if (c->stencil == PYCOOL_STENCIL_4TH && c->n < 4) return PYCOOL_E_INVALID;
  if (c->time_step != PYCOOL_TIME_CONFORMAL && c->time_step != PYCOOL_TIME_PHYSICAL)
    return PYCOOL_E_INVALID;
  if (!(c->L > 0.0) || !std::isfinite(c->L)) return PYCOOL_E_INVALID;
  if (!std::isfinite(c->dt) || c->dt == 0.0) return PYCOOL_E_INVALID;
  if (!(c->mpl > 0.0)) return PYCOOL_E_INVALID;
  if (!std::isfinite(c->rho_rad0) || !std::isfinite(c->rho_mat0)) return PYCOOL_E_INVALID;
  for (int i = 0; i < PYCOOL_MAX_PARAMS; ++i)
    if (!std::isfinite(c->params[i])) return PYCOOL_E_INVALID;
  if (c->model == PYCOOL_MODEL_QBALL && !(c->params[2] > 0.0)) return PYCOOL_E_INVALID;
  // linear stability of every stage at a = 1: |h| omega_max < 2,
  // omega_max^2 = max|symbol of D| / dx^2 + |m2|  (7pt: 12, iso27: 92/15, 4th: 16)
  double w[kMaxStages];
  const int s = stage_table(c->order, w);
  double wmax = 0.0;
  for (int i = 0; i < s; ++i) wmax = std::fmax(wmax, std::fabs(w[i]));
  const double dx = c->L / c->n;
  const double sym = c->stencil == PYCOOL_STENCIL_7PT ? 12.0
                    : (c->stencil == PYCOOL_STENCIL_4TH ? 16.0 : 92.0 / 15.0);
  const double om = std::sqrt(sym / (dx * dx) + std::fabs(c->params[0]));
  if (std::fabs(c->dt) * wmax * om >= 2.0) return PYCOOL_E_UNSTABLE_DT;
  return PYCOOL_OK;
}

void fill_desc(SimDesc& d, const pycool_config& c, const Layout& L, char* state, char* ws) {
  std::memset(&d, 0, sizeof(d));
  d.n = c.n;
  d.nf = model_nfields(c.model);
  d.model = c.model >= kRuntimeModelBase ? (d.nf == 1 ? M_RUNTIME1 : M_RUNTIME2) : c.model;
  d.rt_index = c.model >= kRuntimeModelBase ? c.model - kRuntimeModelBase : -1;
  d.stencil = c.stencil;
  d.prec = c.precision == PYCOOL_SPLIT_FP32 ? PREC_SPLIT
           : (c.precision == PYCOOL_SPLIT_DD ? PREC_DD : PREC_FP64);
  d.nstages = stage_table(c.order, d.w);
  d.physical = c.time_step == PYCOOL_TIME_PHYSICAL ? 1 : 0;
  d.tma = L.geo.tma; d.vx = L.geo.vx; d.txt = L.geo.txt;
  d.tx = L.geo.tx; d.ty = L.geo.ty; d.zc = L.geo.zc;
  d.tiles_x = L.geo.tiles_x; d.tiles_y = L.geo.tiles_y;
  d.zchunks = L.geo.zchunks; d.ncta = L.geo.ncta;  d.S = (int64_t)c.n * c.n * c.n;
  d.dt = c.dt;
  const double dx = c.L / c.n;
  d.dx2inv = 1.0 / (dx * dx);
  d.VL = (double)d.S;
  const bool stat = std::isinf(c.mpl);
  d.mpl2 = stat ? INFINITY : c.mpl * c.mpl;
  d.inv6VLm2 = stat ? 0.0 : 1.0 / (6.0 * d.VL * d.mpl2);
  d.rho_r0 = c.rho_rad0;
  d.rho_m0 = c.rho_mat0;
  for (int i = 0; i < 8; ++i) d.params[i] = c.params[i];
  d.invS = 1.0 / (double)d.S;
  if (c.model == PYCOOL_MODEL_QBALL) d.derived[0] = std::log(c.params[2] * c.params[2]);
  for (int i = 0; i < 4; ++i) d.fparams[i] = (float)c.params[i];
  d.fparams[4] = (float)(0.5 * c.params[0]);
  d.fparams[5] = (float)(0.5 * c.params[1]);
  char* f = state + L.off_fields;
  d.phi[0] = f;
  d.phi[1] = f + L.field_bytes;
  d.pi[0] = f + 2 * L.field_bytes;
  d.pi[1] = f + 3 * L.field_bytes;
  d.bg = (Background*)(state + L.off_bg);
  d.ticket = (unsigned int*)(ws + L.off_ticket);
  d.fault = (int32_t*)(ws + L.off_ticket + 128);
  d.partials = (double*)(ws + L.off_partials);
  d.gticket = (unsigned int*)(ws + L.off_gticket);
  d.gpartials = (double*)(ws + L.off_gpartials);
  d.ngroups = (L.geo.ncta + kGroup - 1) / kGroup;
  if (L.off_rt) {
    const size_t fb = align256((size_t)d.nf * (size_t)d.S * 8);
    d.rt_phis = (double*)(ws + L.off_rt);
    d.rt_dV = (double*)(ws + L.off_rt + fb);
    d.rt_V = (double*)(ws + L.off_rt + 2 * fb);
  }
}

// TMA descriptors for the four field buffers (see SimDesc::tmap).  The driver
// entry point is looked up at run time, so the library needs no libcuda at link.
typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*,
                                  const cuuint64_t*, const cuuint64_t*, const cuuint32_t*,
                                  const cuuint32_t*, CUtensorMapInterleave, CUtensorMapSwizzle,
                                  CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

static cudaError_t encode_fn(EncodeTiledFn* out) {
  static EncodeTiledFn fn = nullptr;
  if (!fn) {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    cudaError_t e = cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000,
                                                     cudaEnableDefault, &q);
    if (e != cudaSuccess) return e;
    if (q != cudaDriverEntryPointSuccess || !p) return cudaErrorNotSupported;
    fn = (EncodeTiledFn)p;
  }
  *out = fn;
  return cudaSuccess;
}

// One 3-D map of a field buffer viewed as x: n, y: n, z: N_f n (fields stacked in z).
static cudaError_t encode_box(EncodeTiledFn fn, CUtensorMap* m, const SimDesc& d, void* buf,
                              int bx, int by) {
  const size_t word = d.prec == PREC_SPLIT ? 4 : 8;
  const CUtensorMapDataType dt =
      d.prec == PREC_SPLIT ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32 : CU_TENSOR_MAP_DATA_TYPE_FLOAT64;
  const cuuint64_t dims[3] = {(cuuint64_t)d.n, (cuuint64_t)d.n, (cuuint64_t)d.n * d.nf};
  const cuuint64_t strides[2] = {(cuuint64_t)d.n * word, (cuuint64_t)d.n * d.n * word};
  const cuuint32_t box[3] = {(cuuint32_t)bx, (cuuint32_t)by, 1};
  const cuuint32_t estr[3] = {1, 1, 1};
  const CUresult r = fn(m, dt, 3, buf, dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                        CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                        CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorInvalidValue;
}

cudaError_t encode_tensor_maps(SimDesc& d) {
  if (!d.tma) return cudaSuccess;
  EncodeTiledFn fn = nullptr;
  cudaError_t e = encode_fn(&fn);
  if (e != cudaSuccess) return e;
  void* bufs[4] = {d.phi[0], d.phi[1], d.pi[0], d.pi[1]};
  for (int b = 0; b < 4; ++b) {
    if ((e = encode_box(fn, &d.tmap[b][0], d, bufs[b], d.tx, d.ty)) != cudaSuccess) return e;
    if ((e = encode_box(fn, &d.tmap[b][1], d, bufs[b], d.tx, 1)) != cudaSuccess) return e;
  }
  return cudaSuccess;
}

// The persistent kernel's boxes over the four field buffers viewed as one 5-D
// tensor (x: n, y: n, z: n, field: N_f, buffer: 4); see PParams::tm.
cudaError_t encode_persist_maps(const SimDesc& d, const PGeo& g, PParams& p) {
  EncodeTiledFn fn = nullptr;
  cudaError_t e = encode_fn(&fn);
  if (e != cudaSuccess) return e;
  const size_t word = d.prec == PREC_SPLIT ? 4 : 8;
  const cuuint64_t n = (cuuint64_t)d.n;
  const cuuint64_t bstride = (cuuint64_t)((const char*)d.phi[1] - (const char*)d.phi[0]);
  if ((const char*)d.pi[0] - (const char*)d.phi[0] != (ptrdiff_t)(2 * bstride) ||
      (const char*)d.pi[1] - (const char*)d.phi[0] != (ptrdiff_t)(3 * bstride) || bstride % 16)
    return cudaErrorInvalidValue;
  const CUtensorMapDataType dt =
      d.prec == PREC_SPLIT ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32 : CU_TENSOR_MAP_DATA_TYPE_FLOAT64;
  const cuuint64_t dims[5] = {n, n, n, (cuuint64_t)d.nf, 4};
  const cuuint64_t strides[4] = {n * word, n * n * word, n * n * n * word, bstride};
  const cuuint32_t estr[5] = {1, 1, 1, 1, 1};
  const int cw = (int)(16 / word);
  const int H = g.halo;   // halo rows per side of the tile box and of the wrap tiles' row box
  const int shapes[6][3] = {{g.tx, 16 + 2 * H, d.nf}, {cw, 18, d.nf}, {g.tx, 16, 1},
                            {g.tx, H, 1},             {cw, 16, 1},    {cw, 1, 1}};
  for (int k = 0; k < 6; ++k) {
    const cuuint32_t box[5] = {(cuuint32_t)shapes[k][0], (cuuint32_t)shapes[k][1], 1,
                               (cuuint32_t)shapes[k][2], 1};
    const CUresult r = fn(&p.tm[k], dt, 5, d.phi[0], dims, strides, box, estr,
                          CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                          CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) return cudaErrorInvalidValue;
  }
  return cudaSuccess;
}

cudaError_t launch_persist(const SimDesc& d, const PParams& p, int grid, cudaStream_t s, int* bps) {
  if (d.prec == PREC_SPLIT) return launch_persist_split(d.model, d.stencil, p.g.vx, p, grid, s, bps);
  if (d.stencil == 13)
    return d.prec == PREC_DD ? launch_persist_dd_wide(d.model, d.stencil, p.g.vx, p, grid, s, bps)
                             : launch_persist_fp64_wide(d.model, d.stencil, p.g.vx, p, grid, s, bps);
  if (d.prec == PREC_DD) return launch_persist_dd(d.model, d.stencil, p.g.vx, p, grid, s, bps);
  return launch_persist_fp64(d.model, d.stencil, p.g.vx, p, grid, s, bps);
}

cudaError_t launch_sweep(const SimDesc& d, const LaunchTable& t, int grid, cudaStream_t s) {
  if (d.model == M_RUNTIME1 || d.model == M_RUNTIME2) return launch_runtime_stage(d, t, grid, s);
  if (d.prec == PREC_SPLIT) return launch_sweep_split(d.model, d.stencil, d.vx, d.tma, t, grid, s);
  // the split-DD form runs on the persistent kernel only (no per-stage instance)
  if (d.prec == PREC_DD) return grid == 0 ? cudaSuccess : cudaErrorInvalidValue;
  return launch_sweep_fp64(d.model, d.stencil, d.vx, d.tma, t, grid, s);
}

__global__ void arm_kernel(Background* bg, long long nsweeps) {
  if (bg->error || bg->mode != MODE_IDLE || nsweeps <= 0) return;
  bg->sweeps_left = nsweeps;
  bg->mode = MODE_SWEEP;
}


// ---------------------------------------------------------------------------
// Split forms' initial state on the device: the lattice mean of one field is
// the float64 background phi0, and the rest, x - phi0, is stored as float32
// (SPLIT_FP32) or as a double-float pair hi + lo (SPLIT_DD).
// The mean is a compensated sum (Knuth's TwoSum on a running float64 sum, the
// rounding errors gathered separately) over a fixed grid-stride order, a fixed
// tree in each block, and one block that folds the block sums in block order:
// reproducible bit for bit for a given lattice.
// ---------------------------------------------------------------------------
__device__ __forceinline__ void mean_two_sum(double a, double b, double& s, double& e) {
  s = a + b;
  const double bb = s - a;
  e = (a - (s - bb)) + (b - bb);
}

__device__ __forceinline__ void mean_block_tree(double s, double c, double* ss, double* cc) {
  const int t = threadIdx.x;
  ss[t] = s;
  cc[t] = c;
  __syncthreads();
  for (int h = blockDim.x / 2; h > 0; h >>= 1) {
    if (t < h) {
      double u, e;
      mean_two_sum(ss[t], ss[t + h], u, e);
      ss[t] = u;
      cc[t] += cc[t + h] + e;
    }
    __syncthreads();
  }
}

__global__ void __launch_bounds__(256) mean_partial_kernel(const double* __restrict__ x,
                                                           long long S, double* part) {
  __shared__ double ss[256], cc[256];
  double s = 0.0, c = 0.0;
  for (long long i = blockIdx.x * 256LL + threadIdx.x; i < S; i += (long long)gridDim.x * 256) {
    double u, e;
    mean_two_sum(s, x[i], u, e);
    s = u;
    c += e;
  }
  mean_block_tree(s, c, ss, cc);
  if (threadIdx.x == 0) {
    part[2 * blockIdx.x] = ss[0];
    part[2 * blockIdx.x + 1] = cc[0];
  }
}

__global__ void __launch_bounds__(256) mean_fold_kernel(const double* __restrict__ part, int nb,
                                                        long long S, double* mean) {
  __shared__ double ss[256], cc[256];
  double s = 0.0, c = 0.0;
  for (int b = threadIdx.x; b < nb; b += 256) {
    double u, e;
    mean_two_sum(s, part[2 * b], u, e);
    s = u;
    c += part[2 * b + 1] + e;
  }
  mean_block_tree(s, c, ss, cc);
  if (threadIdx.x == 0) *mean = (ss[0] + cc[0]) / (double)S;
}

// out[i] = x[i] - mean as float32, or as the pair (hi, lo) with
// hi = fl32(x - mean), lo = fl32((x - mean) - hi).
__global__ void split_store_kernel(const double* __restrict__ x, const double* mean, void* out,
                                   long long S, int pair) {
  const double m = *mean;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < S;
       i += (long long)gridDim.x * blockDim.x) {
    const double v = x[i] - m;
    const float hi = __double2float_rn(v);
    if (pair)
      static_cast<float2*>(out)[i] = make_float2(hi, __double2float_rn(v - (double)hi));
    else
      static_cast<float*>(out)[i] = hi;
  }
}

// The inverse for a read-out: out[i] = base + fluctuation, in float64, for
// elements [i0, i0 + count) of one field.
__global__ void split_load_kernel(const void* __restrict__ d, const double* base, double* out,
                                  long long i0, long long count, int pair) {
  const double b = *base;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < count;
       i += (long long)gridDim.x * blockDim.x) {
    double v;
    if (pair) {
      const float2 p = static_cast<const float2*>(d)[i0 + i];
      v = (double)p.x + (double)p.y;
    } else {
      v = (double)static_cast<const float*>(d)[i0 + i];
    }
    out[i] = b + v;
  }
}


cudaError_t launch_arm(Background* bg, long long nsweeps, cudaStream_t s) {
  arm_kernel<<<1, 1, 0, s>>>(bg, nsweeps);
  return cudaGetLastError();
}

void observables(const Background& b, const SimDesc& d, double mpl, double rho_r0,
                 double rho_m0, pycool_observables* out) {
  std::memset(out, 0, sizeof(*out));
  const double S = (double)d.S, a = b.a;
  const double dx2 = 1.0 / d.dx2inv;
  out->eta = b.eta;
  out->a = a;
  out->pa = b.pa;
  double kin = 0.0, grad = 0.0;
  for (int f = 0; f < d.nf; ++f) {
    out->rho_kin[f] = b.s_pi2[f] / (2.0 * std::pow(a, 6) * S);
    out->rho_grad[f] = -b.s_phiD[f] / (2.0 * a * a * dx2 * S);
    out->mean[f] = b.mean[f];
    out->variance[f] = b.var[f];
    kin += out->rho_kin[f];
    grad += out->rho_grad[f];
  }
  out->rho_pot = b.s_V / S;
  out->rho = kin + grad + out->rho_pot;
  out->P = kin - grad / 3.0 - out->rho_pot;
  if (std::isinf(mpl)) {
    out->H = 0.0;
    out->residual = NAN;
  } else {
    out->H = -b.pa / (6.0 * S * mpl * mpl * a * a);
    const double rt = out->rho + rho_r0 / std::pow(a, 4) + rho_m0 / (a * a * a);
    out->residual = std::fabs(rt / (3.0 * mpl * mpl * out->H * out->H) - 1.0);
  }
  out->steps_done = b.steps_done;
  out->sweeps_done = b.sweeps_done;
}

}  // namespace pycool

// ---------------------------------------------------------------------------
// Simulation object
// ---------------------------------------------------------------------------
struct pycool_sim {
  pycool_config cfg{};
  Layout L{};
  SimDesc hdesc{};
  int nf = 0, nstages = 0;
  int device = 0;
  cudaStream_t stream = nullptr;
  cudaStream_t cap_stream = nullptr;
  char* state = nullptr;
  char* ws = nullptr;
  bool own_state = false, own_ws = false;
  SimDesc* d_desc = nullptr;
  Background* d_bg = nullptr;
  LaunchTable table{};
  cudaGraphExec_t graph = nullptr;
  int graph_len = 0;
  cudaEvent_t done = nullptr;
  bool initialised = false;
  bool poisoned = false;
  int64_t launches = 0;
  // persistent evolve kernel (n a multiple of 32): one cooperative launch per
  // evolve(); otherwise a chain of per-stage launches replayed as a graph
  bool persist = false;
  PParams pp{};
  long long stall_limit = 0;   // > 0: the next persistent launch is a fault test
  // spectrum (made at the first pycool_spectrum call): FFT plan, buffers and
  // the half-spectrum modes ordered by shell
  bool spec_ready = false;
  cufftHandle spec_plan = 0;
  double* spec_tmp = nullptr;       // n^3 float64 field
  void* spec_out = nullptr;         // n n (n/2 + 1) complex coefficients
  int32_t* spec_order = nullptr;    // half-spectrum modes grouped by shell
  int32_t* spec_start = nullptr;    // shell b: spec_order[spec_start[b] .. spec_start[b + 1])
  double* spec_power = nullptr;     // per shell
  std::vector<int64_t> spec_count;  // modes per shell over the full spectrum
};

static constexpr int kGraphLen = 16;

// Host-side fault injection: the next `count` device allocations the library
// makes report failure, as a cudaMalloc that ran out of memory would.
static std::atomic<int> g_fail_allocs{0};

namespace pycool {
bool injected_alloc_failure() {
  int c = g_fail_allocs.load();
  while (c > 0)
    if (g_fail_allocs.compare_exchange_weak(c, c - 1)) return true;
  return false;
}
}  // namespace pycool

PYCOOL_API pycool_status pycool_debug_fail_alloc(int32_t count) {
  if (count < 0) return PYCOOL_E_INVALID;
  g_fail_allocs.store(count);
  return PYCOOL_OK;
}

PYCOOL_API pycool_status pycool_debug_barrier_stall(pycool_sim* sim, int64_t wait_limit_clocks) {
  if (!sim || wait_limit_clocks <= 0) return PYCOOL_E_INVALID;
  if (!sim->persist) return PYCOOL_E_STATE;   // only the persistent kernel has a grid barrier
  sim->stall_limit = (long long)wait_limit_clocks;
  return PYCOOL_OK;
}

static pycool_status cuda_fail(pycool_sim* s, cudaError_t e, const char* what) {
  if (s) s->poisoned = true;
  std::fprintf(stderr, "pycool: CUDA error in %s: %s\n", what, cudaGetErrorString(e));
  return PYCOOL_E_CUDA;
}

#define CK(call)                                                     \
  do {                                                               \
    cudaError_t e__ = (call);                                        \
    if (e__ != cudaSuccess) return cuda_fail(sim, e__, #call);       \
  } while (0)

PYCOOL_API int pycool_stages_per_step(int32_t order) {
  double w[kMaxStages];
  return stage_table(order, w);
}

PYCOOL_API pycool_status pycool_stage_weights(int32_t order, double* w, int32_t* count) {
  if (!w || !count) return PYCOOL_E_INVALID;
  const int s = stage_table(order, w);
  if (s < 0) return PYCOOL_E_INVALID;
  *count = s;
  return PYCOOL_OK;
}

PYCOOL_API pycool_status pycool_query_bytes(const pycool_config* cfg, size_t* state_bytes,
                                            size_t* workspace_bytes) {
  const pycool_status st = validate(cfg);
  if (st != PYCOOL_OK) return st;
  const Layout L = sim_layout(*cfg);
  if (state_bytes) *state_bytes = L.state_bytes;
  if (workspace_bytes) *workspace_bytes = L.ws_bytes;
  return PYCOOL_OK;
}

static pycool_status build_graph(pycool_sim* sim) {
  cudaGraph_t g = nullptr;
  CK(cudaStreamBeginCapture(sim->cap_stream, cudaStreamCaptureModeThreadLocal));
  cudaError_t le = cudaSuccess;
  for (int i = 0; i < kGraphLen && le == cudaSuccess; ++i)
    le = launch_sweep(sim->hdesc, sim->table, sim->L.geo.ncta, sim->cap_stream);
  cudaError_t ee = cudaStreamEndCapture(sim->cap_stream, &g);
  if (le != cudaSuccess) return cuda_fail(sim, le, "capture launch");
  if (ee != cudaSuccess) return cuda_fail(sim, ee, "cudaStreamEndCapture");
  cudaError_t ie = cudaGraphInstantiate(&sim->graph, g, 0);
  cudaGraphDestroy(g);
  if (ie != cudaSuccess) return cuda_fail(sim, ie, "cudaGraphInstantiate");
  sim->graph_len = kGraphLen;
  return PYCOOL_OK;
}

// Persistent path for a state and workspace laid out by sim_layout(): the
// geometry and work plan for this device (uploaded into the workspace on
// stream st), the tensor maps and the occupancy check.  *fits is false if one
// block per SM does not fit (the caller then runs the per-stage kernels).
pycool_status pycool::persist_setup(const pycool_config& cfg, const SimDesc& hd, const Layout& L,
                                    char* state, char* ws, cudaStream_t st, PParams& p,
                                    bool* fits) {
#define PCK(call)                                                    \
  do {                                                               \
    cudaError_t e__ = (call);                                        \
    if (e__ != cudaSuccess) return cuda_fail(nullptr, e__, #call);   \
  } while (0)
  *fits = false;
  int dev = 0, sms = 0, l2 = 0;
  PCK(cudaGetDevice(&dev));
  PCK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  PCK(cudaDeviceGetAttribute(&l2, cudaDevAttrL2CacheSize, dev));
  if (!L.off_prows || !L.off_punits) return PYCOOL_E_INVALID;   // not a persistent layout
  std::vector<int4> units;
  std::vector<int> uoff;
  const PGeo g = plan_units(cfg.n, prec_word(hd.prec), model_nfields(cfg.model), hd.prec, sms,
                            l2, &units, &uoff, hd.stencil == 13 ? 2 : 1);
  std::memset(&p, 0, sizeof(p));
  p.g = g;
  int4* d_units = (int4*)(ws + L.off_punits);
  int* d_uoff = (int*)(ws + L.off_punits +
                       align256((size_t)kMaxPBlocks * kMaxPUnits * sizeof(int4)));
  if (units.size() > (size_t)kMaxPBlocks * kMaxPUnits || uoff.size() > (size_t)kMaxPBlocks + 1 ||
      !check_plan(g, units, uoff))
    return PYCOOL_E_INVALID;
  PCK(cudaMemcpyAsync(d_units, units.data(), units.size() * sizeof(int4), cudaMemcpyHostToDevice,
                      st));
  PCK(cudaMemcpyAsync(d_uoff, uoff.data(), uoff.size() * sizeof(int), cudaMemcpyHostToDevice, st));
  PCK(cudaStreamSynchronize(st));   // the host vectors go out of scope below
  p.units = d_units;
  p.uoff = d_uoff;
  PCK(encode_persist_maps(hd, g, p));
  p.d = (const SimDesc*)(state + L.off_desc);
  p.bg = (Background*)(state + L.off_bg);
  p.bar = (unsigned long long*)(ws + L.off_ticket + 64);
  p.bar_base = 0;
  p.rows = ws + L.off_prows;
  p.fault = hd.fault;
  p.wait_limit = kWaitLimit;
  p.bar_extra = 0;
  p.flush = 1;
  int bps = 0;
  PCK(launch_persist(hd, p, 0, st, &bps));
  *fits = bps >= 1 && g.G <= bps * sms;
  return PYCOOL_OK;
#undef PCK
}

static pycool_status setup_persist(pycool_sim* sim) {
  bool fits = false;
  const pycool_status st = persist_setup(sim->cfg, sim->hdesc, sim->L, sim->state, sim->ws,
                                         sim->stream, sim->pp, &fits);
  if (st == PYCOOL_E_CUDA) sim->poisoned = true;
  if (st != PYCOOL_OK) return st;
  sim->persist = fits;
  return PYCOOL_OK;
}

// One cooperative launch: nsweeps stage sweeps and the flush.  The grid
// barrier counter is monotonic (zeroed with the workspace counters); the host
// tracks how many arrivals earlier launches made.
static pycool_status launch_persist_sweeps(pycool_sim* sim, long long nsweeps) {
  sim->pp.nsweeps = nsweeps;
  if (sim->stall_limit > 0) {
    // fault test (pycool_debug_barrier_stall): this launch's first grid
    // barrier waits for one arrival more than there are blocks, with a short
    // limit; every block gives up, records the fault and returns
    PParams q = sim->pp;
    q.wait_limit = sim->stall_limit;
    q.bar_extra = 1;
    sim->stall_limit = 0;
    CK(launch_persist(sim->hdesc, q, q.g.G, sim->stream, nullptr));
  } else {
    CK(launch_persist(sim->hdesc, sim->pp, sim->pp.g.G, sim->stream, nullptr));
  }
  sim->pp.bar_base += (unsigned long long)(nsweeps + 1) * (unsigned long long)sim->pp.g.G;
  sim->launches += 1;
  return PYCOOL_OK;
}

PYCOOL_API pycool_status pycool_create(const pycool_config* cfg, void* dev_state,
                                       void* dev_workspace, void* cuda_stream,
                                       pycool_sim** out) {
  if (!out) return PYCOOL_E_INVALID;
  *out = nullptr;
  pycool_status st = validate(cfg);
  if (st != PYCOOL_OK) return st;
  if (((uintptr_t)dev_state & 255) || ((uintptr_t)dev_workspace & 255)) return PYCOOL_E_INVALID;
  pycool_sim* sim = new (std::nothrow) pycool_sim();
  if (!sim) return PYCOOL_E_NOMEM;
  sim->cfg = *cfg;
  sim->L = sim_layout(*cfg);
  sim->nf = model_nfields(cfg->model);
  sim->stream = (cudaStream_t)cuda_stream;
  cudaError_t e = cudaGetDevice(&sim->device);
  if (e != cudaSuccess) { delete sim; return cuda_fail(nullptr, e, "cudaGetDevice"); }
  sim->state = (char*)dev_state;
  sim->ws = (char*)dev_workspace;
  if (!sim->state) {
    if (injected_alloc_failure() ||
        cudaMalloc((void**)&sim->state, sim->L.state_bytes) != cudaSuccess) {
      cudaGetLastError();
      delete sim;
      return PYCOOL_E_NOMEM;
    }
    sim->own_state = true;
  }
  if (!sim->ws) {
    if (injected_alloc_failure() || cudaMalloc((void**)&sim->ws, sim->L.ws_bytes) != cudaSuccess) {
      cudaGetLastError();
      if (sim->own_state) cudaFree(sim->state);
      delete sim;
      return PYCOOL_E_NOMEM;
    }
    sim->own_ws = true;
  }
  fill_desc(sim->hdesc, *cfg, sim->L, sim->state, sim->ws);
  e = encode_tensor_maps(sim->hdesc);
  if (e != cudaSuccess) {
    cuda_fail(nullptr, e, "cuTensorMapEncodeTiled");
    if (sim->own_state) cudaFree(sim->state);
    if (sim->own_ws) cudaFree(sim->ws);
    delete sim;
    return PYCOOL_E_CUDA;
  }
  sim->nstages = sim->hdesc.nstages;
  sim->d_desc = (SimDesc*)(sim->state + sim->L.off_desc);
  sim->d_bg = (Background*)(sim->state + sim->L.off_bg);
  Background b;
  std::memset(&b, 0, sizeof(b));
  b.a = 1.0;
  b.mode = MODE_IDLE;
  st = PYCOOL_OK;
  do {
    if ((e = cudaMemcpyAsync(sim->d_desc, &sim->hdesc, sizeof(SimDesc), cudaMemcpyHostToDevice,
                             sim->stream)) != cudaSuccess) break;
    if ((e = cudaMemcpyAsync(sim->d_bg, &b, sizeof(b), cudaMemcpyHostToDevice, sim->stream)) !=
        cudaSuccess) break;
    if ((e = cudaMemsetAsync(sim->ws, 0, sim->L.ws_bytes, sim->stream)) != cudaSuccess) break;
    if ((e = cudaStreamSynchronize(sim->stream)) != cudaSuccess) break;
    if ((e = cudaStreamCreateWithFlags(&sim->cap_stream, cudaStreamNonBlocking)) != cudaSuccess)
      break;
    if ((e = cudaEventCreateWithFlags(&sim->done, cudaEventDisableTiming)) != cudaSuccess) break;
  } while (0);
  if (e != cudaSuccess) {
    cuda_fail(sim, e, "pycool_create");
    pycool_destroy(sim);
    return PYCOOL_E_CUDA;
  }
  sim->table.count = 1;
  sim->table.cta_offset[0] = 0;
  sim->table.cta_offset[1] = sim->L.geo.ncta;
  sim->table.desc[0] = sim->d_desc;
  // set the kernel's shared-memory attribute now, not inside the graph capture
  e = launch_sweep(sim->hdesc, sim->table, 0, sim->stream);
  if (e != cudaSuccess) {
    cuda_fail(sim, e, "kernel attributes");
    pycool_destroy(sim);
    return PYCOOL_E_CUDA;
  }
  if (sim->L.off_prows) {
    st = setup_persist(sim);
    if (st != PYCOOL_OK) {
      pycool_destroy(sim);
      return st;
    }
  }
  if (!sim->persist && sim->hdesc.prec == PREC_DD) {
    // the split-DD form has only the persistent kernel (n a multiple of 32)
    pycool_destroy(sim);
    return PYCOOL_E_INVALID;
  }
  if (!sim->persist) {
    st = build_graph(sim);
    if (st != PYCOOL_OK) {
      pycool_destroy(sim);
      return st;
    }
  }
  *out = sim;
  return PYCOOL_OK;
}

static pycool_status read_bg(pycool_sim* sim, Background* b) {
  CK(cudaMemcpyAsync(b, sim->d_bg, sizeof(Background), cudaMemcpyDeviceToHost, sim->stream));
  CK(cudaStreamSynchronize(sim->stream));
  return PYCOOL_OK;
}

static pycool_status launch_one(pycool_sim* sim) {
  CK(launch_sweep(sim->hdesc, sim->table, sim->L.geo.ncta, sim->stream));
  sim->launches += 1;
  return PYCOOL_OK;
}

// The split forms' initial state (Background already on the device, phi0 and
// pi0 still 0): per field, the device mean goes into Background.phi0[f] /
// pi0[f], then the fluctuation into buffer 0.  Host inputs are staged, one
// field at a time, in the simulation's own buffers that the initial state does
// not use yet: phi buffer 1 (and, for SPLIT_FP32 with its 4-byte words, pi
// buffer 0 after it) for phi; pi buffer 0 and 1 for pi, whose fluctuation is
// then written to phi buffer 1 and moved to pi buffer 0.  Nothing is allocated.
static pycool_status split_initial(pycool_sim* sim, const double* phi, const double* pi,
                                   bool on_device) {
  const size_t S = (size_t)sim->hdesc.S;
  const int pair = sim->hdesc.prec == PREC_DD ? 1 : 0;
  const size_t word = pair ? 8 : 4;
  char* f0 = (char*)sim->hdesc.phi[0];
  char* f1 = (char*)sim->hdesc.phi[1];
  char* p0 = (char*)sim->hdesc.pi[0];
  double* part = (double*)(sim->ws + sim->L.off_mean);
  const int nb = (int)std::min<size_t>(kMeanBlocks, (S + 4095) / 4096);
  const unsigned sg = (unsigned)std::min<size_t>(152 * 8, (S + 255) / 256);
  for (int which = 0; which < 2; ++which) {
    const double* src_all = which == 0 ? phi : pi;
    for (int f = 0; f < sim->nf; ++f) {
      const double* x = src_all + (size_t)f * S;
      // float64 staging of one field (8 S bytes), disjoint from the output
      double* stage = (double*)(which == 0 ? f1 : p0);
      char* out = which == 0 ? f0 + (size_t)f * S * word : f1 + (size_t)f * S * word;
      if (!on_device) {
        CK(cudaMemcpyAsync(stage, x, S * sizeof(double), cudaMemcpyHostToDevice, sim->stream));
        x = stage;
      }
      double* mean = which == 0 ? &sim->d_bg->phi0[f] : &sim->d_bg->pi0[f];
      mean_partial_kernel<<<nb, 256, 0, sim->stream>>>(x, (long long)S, part);
      mean_fold_kernel<<<1, 256, 0, sim->stream>>>(part, nb, (long long)S, mean);
      split_store_kernel<<<sg, 256, 0, sim->stream>>>(x, mean, out, (long long)S, pair);
      CK(cudaGetLastError());
      sim->launches += 3;
    }
  }
  // the momenta's fluctuations, written to phi buffer 1, into pi buffer 0
  CK(cudaMemcpyAsync(p0, f1, (size_t)sim->nf * S * word, cudaMemcpyDeviceToDevice, sim->stream));
  return PYCOOL_OK;
}

PYCOOL_API pycool_status pycool_set_initial(pycool_sim* sim, const double* phi, const double* pi,
                                            int on_device, double a0, double pa0) {
  if (!sim || !phi || !pi) return PYCOOL_E_INVALID;
  if (sim->poisoned) return PYCOOL_E_STATE;
  if (!(a0 > 0.0) || !std::isfinite(a0)) return PYCOOL_E_INVALID;
  const size_t S = (size_t)sim->hdesc.S;
  const int nf = sim->nf;
  const size_t count = (size_t)nf * S;
  Background b;
  std::memset(&b, 0, sizeof(b));
  b.a = a0;
  b.init_pa = std::isnan(pa0) ? 1 : 0;
  b.pa = std::isnan(pa0) ? 0.0 : pa0;
  b.mode = MODE_FLUSH;  // the first launch only reduces (h_prev = 0 -> no drift)
  b.cur = 0;
  CK(cudaStreamSynchronize(sim->stream));
  if (sim->hdesc.prec == PREC_FP64) {
    const cudaMemcpyKind kind = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
    CK(cudaMemcpyAsync(sim->hdesc.phi[0], phi, count * sizeof(double), kind, sim->stream));
    CK(cudaMemcpyAsync(sim->hdesc.pi[0], pi, count * sizeof(double), kind, sim->stream));
    CK(cudaMemcpyAsync(sim->d_bg, &b, sizeof(b), cudaMemcpyHostToDevice, sim->stream));
  } else {
    // split forms: phi0 = the lattice mean (float64), the rest as float32 or
    // as a double-float pair, all on the device (split_initial)
    CK(cudaMemcpyAsync(sim->d_bg, &b, sizeof(b), cudaMemcpyHostToDevice, sim->stream));
    pycool_status st = split_initial(sim, phi, pi, on_device != 0);
    if (st != PYCOOL_OK) return st;
  }
  CK(cudaMemsetAsync(sim->ws, 0, sim->L.off_partials, sim->stream));
  sim->pp.bar_base = 0;
  // the reducing flush: sums of the initial state (and p_a from H = 0)
  pycool_status st = sim->persist ? launch_persist_sweeps(sim, 0) : launch_one(sim);
  if (st != PYCOOL_OK) return st;
  CK(cudaEventRecord(sim->done, sim->stream));
  CK(cudaStreamSynchronize(sim->stream));
  sim->initialised = true;
  return PYCOOL_OK;
}

PYCOOL_API pycool_status pycool_evolve(pycool_sim* sim, int64_t steps) {
  if (!sim || steps < 0) return PYCOOL_E_INVALID;
  if (sim->poisoned) return PYCOOL_E_STATE;
  if (!sim->initialised) return PYCOOL_E_STATE;
  if (steps == 0) return PYCOOL_OK;
  const long long nsweeps = (long long)steps * sim->nstages;
  if (sim->persist) {
    pycool_status st = launch_persist_sweeps(sim, nsweeps);
    if (st != PYCOOL_OK) return st;
    CK(cudaEventRecord(sim->done, sim->stream));
    return PYCOOL_OK;
  }
  CK(launch_arm(sim->d_bg, nsweeps, sim->stream));
  sim->launches += 1;
  long long left = nsweeps + 1;  // + the synchronising flush
  while (left >= sim->graph_len) {
    CK(cudaGraphLaunch(sim->graph, sim->stream));
    sim->launches += sim->graph_len;
    left -= sim->graph_len;
  }
  for (; left > 0; --left) {
    pycool_status st = launch_one(sim);
    if (st != PYCOOL_OK) return st;
  }
  CK(cudaEventRecord(sim->done, sim->stream));
  return PYCOOL_OK;
}

PYCOOL_API pycool_status pycool_sync(pycool_sim* sim, double timeout_s) {
  if (!sim) return PYCOOL_E_INVALID;
  if (sim->poisoned) return PYCOOL_E_STATE;
  const auto t0 = std::chrono::steady_clock::now();
  for (;;) {
    const cudaError_t q = cudaEventQuery(sim->done);
    if (q == cudaSuccess) break;
    if (q != cudaErrorNotReady) return cuda_fail(sim, q, "cudaEventQuery");
    if (timeout_s >= 0.0) {
      const double el =
          std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
      if (el > timeout_s) return PYCOOL_E_TIMEOUT;
    }
    std::this_thread::sleep_for(std::chrono::microseconds(50));
  }
  int32_t fault = 0;
  CK(cudaMemcpy(&fault, sim->hdesc.fault, sizeof(fault), cudaMemcpyDeviceToHost));
  if (fault) {  // a device-side wait gave up: the state can no longer be trusted
    sim->poisoned = true;
    return PYCOOL_E_TIMEOUT;
  }
  Background b;
  pycool_status st = read_bg(sim, &b);
  if (st != PYCOOL_OK) return st;
  if (b.error) return PYCOOL_E_NONFINITE;
  return PYCOOL_OK;
}

PYCOOL_API pycool_status pycool_energies(pycool_sim* sim, pycool_observables* out) {
  if (!sim || !out) return PYCOOL_E_INVALID;
  if (!sim->initialised) return PYCOOL_E_STATE;
  pycool_status st = pycool_sync(sim, -1.0);
  if (st != PYCOOL_OK) return st;
  Background b;
  st = read_bg(sim, &b);
  if (st != PYCOOL_OK) return st;
  observables(b, sim->hdesc, sim->cfg.mpl, sim->cfg.rho_rad0, sim->cfg.rho_mat0, out);
  return PYCOOL_OK;
}

PYCOOL_API pycool_status pycool_field_stats(pycool_sim* sim, int32_t field, double* mean,
                                            double* variance) {
  if (!sim || field < 0 || field >= sim->nf) return PYCOOL_E_INVALID;
  pycool_observables e;
  pycool_status st = pycool_energies(sim, &e);
  if (st != PYCOOL_OK) return st;
  if (mean) *mean = e.mean[field];
  if (variance) *variance = e.variance[field];
  return PYCOOL_OK;
}

PYCOOL_API pycool_status pycool_get_fields(pycool_sim* sim, double* phi, double* pi,
                                           int on_device) {
  if (!sim) return PYCOOL_E_INVALID;
  if (!sim->initialised) return PYCOOL_E_STATE;
  pycool_status st = pycool_sync(sim, -1.0);
  if (st != PYCOOL_OK && st != PYCOOL_E_NONFINITE) return st;
  Background b;
  st = read_bg(sim, &b);
  if (st != PYCOOL_OK) return st;
  const size_t S = (size_t)sim->hdesc.S;
  const size_t count = (size_t)sim->nf * S;
  const void* src_phi = sim->hdesc.phi[b.cur & 1];
  const void* src_pi = sim->hdesc.pi[(b.cur >> 1) & 1];
  if (sim->hdesc.prec == PREC_FP64) {
    const cudaMemcpyKind kind = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
    if (phi) CK(cudaMemcpyAsync(phi, src_phi, count * sizeof(double), kind, sim->stream));
    if (pi) CK(cudaMemcpyAsync(pi, src_pi, count * sizeof(double), kind, sim->stream));
    CK(cudaStreamSynchronize(sim->stream));
    return b.error ? PYCOOL_E_NONFINITE : PYCOOL_OK;
  }
  // split forms: phi0 + dphi evaluated in float64 (split-DD: dphi = hi + lo) on
  // the device; for host outputs through the phi buffer the current state does
  // not use, in chunks of its size
  const int pair = sim->hdesc.prec == PREC_DD ? 1 : 0;
  double* stage = (double*)sim->hdesc.phi[(b.cur & 1) ^ 1];
  const size_t chunk = sim->L.field_bytes / sizeof(double);
  for (int which = 0; which < 2; ++which) {
    double* dst = which == 0 ? phi : pi;
    if (!dst) continue;
    const void* src = which == 0 ? src_phi : src_pi;
    for (int f = 0; f < sim->nf; ++f) {
      const double* base = which == 0 ? &sim->d_bg->phi0[f] : &sim->d_bg->pi0[f];
      for (size_t i0 = 0; i0 < S; i0 += chunk) {
        const size_t m = std::min(chunk, S - i0);
        double* out = on_device ? dst + (size_t)f * S + i0 : stage;
        const unsigned g = (unsigned)std::min<size_t>(152 * 8, (m + 255) / 256);
        split_load_kernel<<<g, 256, 0, sim->stream>>>(src, base, out, (long long)((size_t)f * S + i0),
                                                     (long long)m, pair);
        CK(cudaGetLastError());
        sim->launches += 1;
        if (!on_device)
          CK(cudaMemcpyAsync(dst + (size_t)f * S + i0, stage, m * sizeof(double),
                             cudaMemcpyDeviceToHost, sim->stream));
      }
    }
  }
  CK(cudaStreamSynchronize(sim->stream));
  return b.error ? PYCOOL_E_NONFINITE : PYCOOL_OK;
}

PYCOOL_API pycool_status pycool_checkpoint_size(pycool_sim* sim, size_t* size) {
  if (!sim || !size) return PYCOOL_E_INVALID;
  const size_t word = prec_word(sim->hdesc.prec);
  *size = sizeof(Background) + 2 * (size_t)sim->nf * (size_t)sim->hdesc.S * word;
  return PYCOOL_OK;
}

PYCOOL_API pycool_status pycool_checkpoint_save(pycool_sim* sim, void* buf, size_t cap) {
  if (!sim || !buf) return PYCOOL_E_INVALID;
  if (!sim->initialised) return PYCOOL_E_STATE;
  size_t need = 0;
  pycool_checkpoint_size(sim, &need);
  if (cap < need) return PYCOOL_E_INVALID;
  pycool_status st = pycool_sync(sim, -1.0);
  if (st != PYCOOL_OK) return st;
  Background b;
  st = read_bg(sim, &b);
  if (st != PYCOOL_OK) return st;
  if (b.mode != MODE_IDLE) return PYCOOL_E_STATE;
  const size_t word = prec_word(sim->hdesc.prec);
  const size_t fb = (size_t)sim->nf * (size_t)sim->hdesc.S * word;
  char* p = (char*)buf;
  std::memcpy(p, &b, sizeof(b));
  CK(cudaMemcpy(p + sizeof(b), sim->hdesc.phi[b.cur & 1], fb, cudaMemcpyDeviceToHost));
  CK(cudaMemcpy(p + sizeof(b) + fb, sim->hdesc.pi[(b.cur >> 1) & 1], fb, cudaMemcpyDeviceToHost));
  return PYCOOL_OK;
}

PYCOOL_API pycool_status pycool_checkpoint_load(pycool_sim* sim, const void* buf, size_t size) {
  if (!sim || !buf) return PYCOOL_E_INVALID;
  if (sim->poisoned) return PYCOOL_E_STATE;
  size_t need = 0;
  pycool_checkpoint_size(sim, &need);
  if (size != need) return PYCOOL_E_INVALID;
  Background b;
  std::memcpy(&b, buf, sizeof(b));
  if (b.mode != MODE_IDLE || b.error) return PYCOOL_E_INVALID;
  const size_t word = prec_word(sim->hdesc.prec);
  const size_t fb = (size_t)sim->nf * (size_t)sim->hdesc.S * word;
  const char* p = (const char*)buf;
  CK(cudaStreamSynchronize(sim->stream));
  CK(cudaMemcpy(sim->hdesc.phi[b.cur & 1], p + sizeof(b), fb, cudaMemcpyHostToDevice));
  CK(cudaMemcpy(sim->hdesc.pi[(b.cur >> 1) & 1], p + sizeof(b) + fb, fb, cudaMemcpyHostToDevice));
  CK(cudaMemcpy(sim->d_bg, &b, sizeof(b), cudaMemcpyHostToDevice));
  CK(cudaMemset(sim->ws, 0, sim->L.off_partials));
  sim->pp.bar_base = 0;
  CK(cudaEventRecord(sim->done, sim->stream));
  sim->initialised = true;
  return PYCOOL_OK;
}

PYCOOL_API int32_t pycool_spectrum_bins(int32_t n) {
  if (n < 1 || n > 1024) return -1;
  return (int32_t)std::floor(std::sqrt(3.0) * n / 2.0) + 2;
}

// The synchronised state that the observables read.
static pycool_status observed_state(pycool_sim* sim, Background* b) {
  if (!sim->initialised) return PYCOOL_E_STATE;
  pycool_status st = pycool_sync(sim, -1.0);
  if (st != PYCOOL_OK) return st;
  st = read_bg(sim, b);
  if (st != PYCOOL_OK) return st;
  return b->mode == MODE_IDLE ? PYCOOL_OK : PYCOOL_E_STATE;
}

PYCOOL_API pycool_status pycool_energy_fields(pycool_sim* sim, double* rho, double* P,
                                              int on_device) {
  if (!sim || !rho || !P) return PYCOOL_E_INVALID;
  if (sim->poisoned) return PYCOOL_E_STATE;
  Background b;
  pycool_status st = observed_state(sim, &b);
  if (st != PYCOOL_OK) return st;
  if (sim->cfg.model >= kRuntimeModelBase) {
    // V at every site of the current fields: the compiled potential kernel
    // into the simulation's runtime scratch (the FP64 form: plain fields)
    CK(launch_runtime_potential(sim->hdesc, (const double*)sim->hdesc.phi[b.cur & 1],
                                sim->stream));
    sim->launches += 1;
  }
  const size_t bytes = (size_t)sim->hdesc.S * sizeof(double);
  if (on_device) {
    CK(launch_energy_fields(sim->hdesc, b, rho, P, sim->stream));
    sim->launches += 1;
    CK(cudaStreamSynchronize(sim->stream));
    return PYCOOL_OK;
  }
  double *dr = nullptr, *dp = nullptr;
  if (injected_alloc_failure() || cudaMalloc((void**)&dr, bytes) != cudaSuccess ||
      cudaMalloc((void**)&dp, bytes) != cudaSuccess) {
    cudaGetLastError();
    cudaFree(dr);
    return PYCOOL_E_NOMEM;
  }
  cudaError_t e = launch_energy_fields(sim->hdesc, b, dr, dp, sim->stream);
  if (e == cudaSuccess) e = cudaMemcpyAsync(rho, dr, bytes, cudaMemcpyDeviceToHost, sim->stream);
  if (e == cudaSuccess) e = cudaMemcpyAsync(P, dp, bytes, cudaMemcpyDeviceToHost, sim->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(sim->stream);
  cudaFree(dr);
  cudaFree(dp);
  if (e != cudaSuccess) return cuda_fail(sim, e, "pycool_energy_fields");
  sim->launches += 1;
  return PYCOOL_OK;
}

// Shell of each half-spectrum mode, the modes grouped by shell (counting
// sort: ascending index within a shell), the FFT plan and the buffers.
static pycool_status spectrum_setup(pycool_sim* sim) {
  const int n = sim->cfg.n, nh = n / 2 + 1, nb = pycool_spectrum_bins(n);
  const size_t half = (size_t)n * n * nh;
  std::vector<int32_t> shell(half), start(nb + 1, 0), order(half);
  sim->spec_count.assign(nb, 0);
  for (int z = 0; z < n; ++z)
    for (int y = 0; y < n; ++y)
      for (int x = 0; x < nh; ++x) {
        const long long mz = z <= n / 2 ? z : z - n, my = y <= n / 2 ? y : y - n;
        const long long r2 = mz * mz + my * my + (long long)x * x;
        const int b = (int)std::lround(std::sqrt((double)r2));
        const size_t m = ((size_t)z * n + y) * nh + x;
        shell[m] = b;
        start[b + 1] += 1;
        sim->spec_count[b] += (x > 0 && 2 * x != n) ? 2 : 1;
      }
  for (int b = 0; b < nb; ++b) start[b + 1] += start[b];
  std::vector<int32_t> fill(start.begin(), start.end() - 1);
  for (size_t m = 0; m < half; ++m) order[fill[shell[m]]++] = (int32_t)m;
  if (injected_alloc_failure() ||
      cudaMalloc((void**)&sim->spec_tmp, (size_t)sim->hdesc.S * sizeof(double)) != cudaSuccess ||
      cudaMalloc(&sim->spec_out, half * sizeof(cufftDoubleComplex)) != cudaSuccess ||
      cudaMalloc((void**)&sim->spec_order, half * sizeof(int32_t)) != cudaSuccess ||
      cudaMalloc((void**)&sim->spec_start, (nb + 1) * sizeof(int32_t)) != cudaSuccess ||
      cudaMalloc((void**)&sim->spec_power, nb * sizeof(double)) != cudaSuccess) {
    cudaGetLastError();
    return PYCOOL_E_NOMEM;
  }
  CK(cudaMemcpy(sim->spec_order, order.data(), half * sizeof(int32_t), cudaMemcpyHostToDevice));
  CK(cudaMemcpy(sim->spec_start, start.data(), (nb + 1) * sizeof(int32_t), cudaMemcpyHostToDevice));
  if (cufftPlan3d(&sim->spec_plan, n, n, n, CUFFT_D2Z) != CUFFT_SUCCESS) return PYCOOL_E_CUDA;
  sim->spec_ready = true;
  return PYCOOL_OK;
}

PYCOOL_API pycool_status pycool_spectrum(pycool_sim* sim, int32_t which, int32_t field,
                                         double* power, int64_t* count, int32_t nbins) {
  if (!sim || !power || (which != 0 && which != 1) || field < 0 || field >= sim->nf ||
      nbins != pycool_spectrum_bins(sim->cfg.n))
    return PYCOOL_E_INVALID;
  if (sim->poisoned) return PYCOOL_E_STATE;
  Background b;
  pycool_status st = observed_state(sim, &b);
  if (st != PYCOOL_OK) return st;
  if (!sim->spec_ready) {
    st = spectrum_setup(sim);
    if (st != PYCOOL_OK) return st;
  }
  if (cufftSetStream(sim->spec_plan, sim->stream) != CUFFT_SUCCESS) return PYCOOL_E_CUDA;
  CK(launch_field_values(sim->hdesc, b, which, field, sim->spec_tmp, sim->stream));
  if (cufftExecD2Z(sim->spec_plan, sim->spec_tmp, (cufftDoubleComplex*)sim->spec_out) !=
      CUFFT_SUCCESS)
    return PYCOOL_E_CUDA;
  CK(launch_spectrum_bins(sim->spec_out, sim->cfg.n, sim->spec_order, sim->spec_start, nbins,
                          sim->spec_power, sim->stream));
  CK(cudaMemcpyAsync(power, sim->spec_power, nbins * sizeof(double), cudaMemcpyDeviceToHost,
                     sim->stream));
  CK(cudaStreamSynchronize(sim->stream));
  sim->launches += 2;
  if (count)
    for (int i = 0; i < nbins; ++i) count[i] = sim->spec_count[i];
  return PYCOOL_OK;
}

PYCOOL_API int64_t pycool_kernel_launches(const pycool_sim* sim) {
  return sim ? sim->launches : -1;
}

PYCOOL_API pycool_status pycool_set_stream(pycool_sim* sim, void* cuda_stream) {
  if (!sim) return PYCOOL_E_INVALID;
  pycool_status st = pycool_sync(sim, -1.0);
  if (st != PYCOOL_OK && st != PYCOOL_E_NONFINITE && st != PYCOOL_E_STATE) return st;
  sim->stream = (cudaStream_t)cuda_stream;
  return PYCOOL_OK;
}

PYCOOL_API void pycool_destroy(pycool_sim* sim) {
  if (!sim) return;
  cudaStreamSynchronize(sim->stream);
  if (sim->spec_ready) cufftDestroy(sim->spec_plan);
  cudaFree(sim->spec_tmp);
  cudaFree(sim->spec_out);
  cudaFree(sim->spec_order);
  cudaFree(sim->spec_start);
  cudaFree(sim->spec_power);
  if (sim->graph) cudaGraphExecDestroy(sim->graph);
  if (sim->done) cudaEventDestroy(sim->done);
  if (sim->cap_stream) cudaStreamDestroy(sim->cap_stream);
  if (sim->own_state && sim->state) cudaFree(sim->state);
  if (sim->own_ws && sim->ws) cudaFree(sim->ws);
  cudaGetLastError();
  delete sim;
}

PYCOOL_API const char* pycool_strerror(pycool_status s) {
  switch (s) {
    case PYCOOL_OK: return "ok";
    case PYCOOL_E_INVALID: return "invalid argument or configuration";
    case PYCOOL_E_UNSTABLE_DT: return "time step breaks the linear stability bound";
    case PYCOOL_E_NOMEM: return "out of memory";
    case PYCOOL_E_CUDA: return "CUDA error (simulation poisoned)";
    case PYCOOL_E_NONFINITE: return "non-finite lattice sum (evolution stopped)";
    case PYCOOL_E_TIMEOUT: return "timed out";
    case PYCOOL_E_STATE: return "call not valid in the current state";
    case PYCOOL_E_BUSY: return "busy";
    case PYCOOL_E_NOT_FOUND: return "unknown ticket";
    case PYCOOL_E_CANCELLED: return "request cancelled";
  }
  return "unknown status";
}
