// Device-side records shared by the sweep kernels and the host runtime.
//
// One simulation = one SimDesc (immutable, device memory) + one Background
// (mutable, device memory) + double-buffered field arrays + a partial-sum
// workspace.  Every sweep kernel reads its simulation's Background at start,
// streams its tile, writes one partial per reduced quantity, and the last
// block to finish (atomic ticket, no spin-wait) folds the partials in a fixed
// order and advances the Background.  So a whole evolve() is a chain of
// identical launches with no host round trip, and replays as a CUDA graph.
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>

#include <cstdint>
#include <vector>

namespace pycool {

constexpr int kMaxFields = 2;
constexpr int kMaxStages = 15;
constexpr int kThreads = 256;      // threads per block, every kernel
constexpr int kMaxTXT = 32;        // threads per tile row (x, contiguous)
constexpr int kMaxTY = 8;          // tile height (y)
constexpr int kNQ = 12;            // reduction slots per block
constexpr int kMaxMembers = 64;    // simulations per batched launch
constexpr int kGroup = 32;         // blocks per first-level fold group
constexpr int kRuntimeModelBase = 16;         // first id of a potential given at run time
constexpr int kRuntimeModelMax = 64;          // such potentials per process
constexpr long long kWaitLimit = 1ll << 31;   // default limit of a device-side wait
                                              // (SM clocks, about a second)

enum Mode : int32_t { MODE_IDLE = 0, MODE_SWEEP = 1, MODE_FLUSH = 2 };
// PREC_DD: the split form with double-float fluctuations (float pairs, 8 bytes
// per value) -- float64-class accuracy, arithmetic on the FP32 pipe.
enum Prec : int32_t { PREC_FP64 = 0, PREC_SPLIT = 1, PREC_DD = 2 };
// bytes per stored field value
constexpr int prec_word(int prec) { return prec == PREC_SPLIT ? 4 : 8; }

// Mutable background record.  a, p_a, eta and the pending half-stage are the
// scalar part of the state (Sec. 2.3, Eq. split-Phi: Phi_H1 moves a, Phi_H2 and
// Phi_H3 kick p_a).  Between two sweeps the state is "staggered": the trailing
// Phi_H2(h/2) Phi_H1(h/2) of the last stage (step h_prev) is still pending and
// is applied, merged with the next stage's leading Phi_H1 Phi_H2, at the start
// of the next sweep.
struct alignas(16) Background {
  double a, pa, eta;
  double sum_pi2;            // sum over fields and sites of pi^2 (current pi)
  double h_prev;             // pending half-stage step; 0 = synchronised
  int64_t stage;             // stage-table index of the next sweep
  int64_t sweeps_left;       // sweeps before the synchronising flush
  int64_t sweeps_done, steps_done;
  int32_t mode;              // Mode
  int32_t cur;               // bit 0: buffer holding phi, bit 1: buffer holding pi
  int32_t error;             // 1: a lattice sum was not finite (evolution stopped)
  int32_t init_pa;           // 1: the next flush sets p_a from H = 0
  // Sums of the last flush (synchronised state), per field.
  double s_pi2[kMaxFields], s_phiD[kMaxFields], s_V;
  double mean[kMaxFields], var[kMaxFields];         // field mean and variance
  double shift[kMaxFields];                         // unused (kept: checkpoint layout)
  // Split form: lattice-mean background and pending re-centring shifts.
  double phi0[kMaxFields], pi0[kMaxFields];
  double mu_phi[kMaxFields], mu_pi[kMaxFields];
  double deta;               // conformal step of the running time step (physical-time steps)
  double pad[3];
};

struct alignas(64) SimDesc {
  // TMA descriptors of the four field buffers (phi 0, phi 1, pi 0, pi 1), each as
  // [0] a TX x TY x 1 box (the tile) and [1] a TX x 1 x 1 box (one halo row).
  // The tensor is the buffer viewed as x: n, y: n, z: N_f n (fields stacked in z).
  CUtensorMap tmap[4][2];
  int32_t n, nf, model, stencil, prec, nstages;
  int32_t physical;           // 1: physical-time steps, d-eta = dt / a per step (Sec. 3.1)
  int32_t tma;                // 1: TMA-staged kernel (n % 32 == 0), 0: plain loads
  int32_t vx;                 // sites per thread along x (TMA kernel)
  int32_t txt;                // threads per tile row
  int32_t tx, ty, zc, tiles_x, tiles_y, zchunks, ncta;
  int64_t S;                  // n^3
  double dt, dx2inv, VL, inv6VLm2, mpl2, rho_r0, rho_m0;
  double invS;                // 1 / n^3
  double params[8];
  double derived[4];          // host-computed model constants (Q-ball: ln M^2)
  float fparams[8];           // params[] and, from slot 4 on, half of params 0 and 1, in float32
  double w[kMaxStages];
  void* phi[2];
  void* pi[2];
  double* partials;           // ncta * kNQ: one row per block
  double* gpartials;          // ngroups * kNQ: one row per group of kGroup blocks
  unsigned int* ticket;       // groups folded so far
  unsigned int* gticket;      // per group: blocks finished so far
  int32_t ngroups;
  int32_t* fault;             // set when a device-side wait gave up
  Background* bg;
  // potentials compiled at run time: the drifted fields, V' and V of a stage
  double* rt_phis;            // N_f n^3
  double* rt_dV;              // N_f n^3
  double* rt_V;               // n^3
  int32_t rt_index;           // the registry entry of the potential (-1: none)
};

struct LaunchTable {
  int32_t count;
  int32_t cta_offset[kMaxMembers + 1];
  const SimDesc* desc[kMaxMembers];
};

// Geometry of the z-streamed tiling, a function of (n, word size, N_f) alone,
// so the reduction order of a lattice does not depend on what it is batched
// with.  A block is 256 threads.
//   TMA kernel (n % 32 == 0): 32 lanes x 8 rows, each lane owns vx sites along
//     x (vx * N_f * word <= 16 bytes), tile = 32 vx x 8, n % (32 vx) == 0.
//   plain kernel (other n): one site per thread, txt x ty threads (ragged tiles).
struct Geometry {
  int tma, vx, txt, tx, ty, zc, tiles_x, tiles_y, zchunks, ncta;
};

// plain: the plain-load geometry whatever n (the fourth-order stencil's kernel).
inline Geometry choose_geometry(int n, int word, int nf, bool plain = false) {
  Geometry g;
  g.tma = (n % 32 == 0 && !plain) ? 1 : 0;
  g.vx = 1;
  if (g.tma) {
    for (int v = 16 / (word * nf); v >= 2; v /= 2)
      if (n % (32 * v) == 0) { g.vx = v; break; }
    g.txt = 32;
    g.ty = kMaxTY;
  } else {
    g.txt = n >= 32 ? 32 : n;
    g.ty = n >= kMaxTY ? kMaxTY : n;
  }
  g.tx = g.txt * g.vx;
  g.tiles_x = (n + g.tx - 1) / g.tx;
  g.tiles_y = (n + g.ty - 1) / g.ty;
  const int tiles = g.tiles_x * g.tiles_y;
  const int target = 2 * 152;           // two blocks per SM on 152 SMs
  const int min_zc = n >= 128 ? 16 : 4;  // bound the z-halo re-read overhead
  int zc = 64;
  while (zc > min_zc && (long long)tiles * ((n + zc - 1) / zc) < target) zc /= 2;
  if (zc > n) zc = n;
  g.zc = zc;
  g.zchunks = (n + zc - 1) / zc;
  g.ncta = tiles * g.zchunks;
  return g;
}

// ---------------------------------------------------------------------------
// Persistent evolve kernel (persist.cuh): one cooperative launch per evolve()
// call, one 512-thread block per SM, tiles of 32 vx x 16 sites.
// ---------------------------------------------------------------------------
constexpr int kMaxPBlocks = 208;           // blocks (SMs) of the persistent kernel at most
constexpr int kMaxPUnits = 64;             // work units per block

// Geometry, chosen on the host (a function of n, word, N_f, the SM count and
// the L2 size): tiles of tx x 16 sites, each tile's z-axis cut into chunks (rc
// for tiles clear of the periodic y boundary, rw for the tiles whose halo rows
// cross it), the chunks dealt to the G blocks and cut where a block reaches
// the common target (plan_units); each block reads its units from a table.
struct PGeo {
  int n, vx, tx, tiles_x, ntiles, rc, rw, nunits, G;
  int halo;   // z-halo planes (and halo rows) per side: 1, or 2 for the 13-point stencil
};

// Kernel parameters, passed as one __grid_constant__ struct (the tensor maps
// live in parameter space, as TMA wants them).
struct PParams {
  // [box]: the four field buffers (phi0, phi1, pi0, pi1: equally spaced in the
  // state block) viewed as ONE 5-D tensor (x: n, y: n, z: n, field: N_f,
  // buffer: 4), so that a stage switch uses the same six descriptors;
  // cw = 16 bytes / word; every box spans one buffer and one z-plane:
  // (with H = 2 halo rows, the 13-point stencil: box 0 is tx x 20 x N_f, box 3 tx x 2 x 1)
  //   0: tx x 18 x N_f  tile with both halo rows, every field (y0 > 0, y0 + 16 < n)
  //   1: cw x 18 x N_f  halo column with its corner cells, every field (same tiles)
  //   2: tx x 16 x 1    tile rows of one field        (tiles at the y wrap)
  //   3: tx x 1 x 1     one halo row of one field
  //   4: cw x 16 x 1    halo column of one field
  //   5: cw x 1 x 1     one corner cell of one field
  CUtensorMap tm[6];
  const SimDesc* d;
  Background* bg;
  unsigned long long* bar;       // grid barrier: arrivals so far (monotonic)
  unsigned long long bar_base;   // arrivals before this launch
  void* rows;              // [2][G][kNQ] doubles (FP64) or float pairs (split)
  const int4* units;       // every block's units in processing order: (x0, y0, z0, planes)
  const int* uoff;         // block b's units are units[uoff[b] .. uoff[b + 1])
  int32_t* fault;
  PGeo g;
  long long nsweeps;       // stage sweeps of this launch (then one flush if flush != 0)
  int flush;               // 1: end with the flush; 0 (nsweeps >= 1, FP64 form only): end
                           //    after the last sweep, the stage boundary pending
  long long wait_limit;    // clocks after which a device-side wait gives up
  unsigned long long bar_extra;  // added to every grid-barrier target: 0, or 1 to
                                 // make the first barrier unreachable (fault test)
};

// The persistent geometry and its unit table (units grouped by block; off has
// G + 1 entries).
PGeo plan_units(int n, int word, int nf, int prec, int sms, long long l2_bytes,
                std::vector<int4>* units, std::vector<int>* off, int halo = 1);

// Launchers (one translation unit per precision).
cudaError_t launch_sweep_fp64(int model, int stencil, int vx, int tma, const LaunchTable& t, int grid,
                              cudaStream_t s);
cudaError_t launch_sweep_split(int model, int stencil, int vx, int tma, const LaunchTable& t, int grid,
                               cudaStream_t s);
// grid == 0: set the kernel attributes and report blocks per SM in *bps.
cudaError_t launch_persist_fp64(int model, int stencil, int vx, const PParams& p, int grid,
                                cudaStream_t s, int* bps);
cudaError_t launch_persist_split(int model, int stencil, int vx, const PParams& p, int grid,
                                 cudaStream_t s, int* bps);
cudaError_t launch_persist_dd(int model, int stencil, int vx, const PParams& p, int grid,
                              cudaStream_t s, int* bps);
// the 13-point stencil's instances (FP64 and split-DD)
cudaError_t launch_persist_fp64_wide(int model, int stencil, int vx, const PParams& p, int grid,
                                     cudaStream_t s, int* bps);
cudaError_t launch_persist_dd_wide(int model, int stencil, int vx, const PParams& p, int grid,
                                   cudaStream_t s, int* bps);

}  // namespace pycool
