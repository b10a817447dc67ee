// The persistent evolve kernel: one cooperative launch advances a lattice
// through every stage of an evolve() call -- `nsweeps` fused stage sweeps
// (Sec. 2.3, one per second-order stage Phi1(h/2) Phi2(h/2) Phi3(h) Phi2(h/2)
// Phi1(h/2), drift merged across stage boundaries exactly as in sweep.cuh)
// and the synchronising flush -- with one resident block per SM.
//
// Why: a stage is a global dependency (the drift coefficient of stage i+1
// needs a and p_a after Phi_H3 of stage i, i.e. lattice-wide sums of stage i),
// so a per-stage launch pays the launch ramp, the tail of its last block and a
// re-derivation of the scalar coefficients in every block, every stage.  Here:
//   - each block walks a fixed list of work units (tile x z-range) that the
//     host planned (plan_units: chunks of the tiles' z-columns dealt in z order
//     to the least-loaded block, cut to a common target), and the TMA ring
//     runs on across unit ends;
//   - all loads are TMA (tile, two halo rows, two 16-byte halo-column boxes,
//     and for the 27-point stencil four corner cells) into an mbarrier ring;
//   - at the end of a stage every block writes one row of partial sums; a
//     grid barrier (monotonic arrival counter, bounded spin) separates
//     stages; every block then copies all rows into shared memory (one bulk
//     copy) and folds them in the same fixed order, so every block derives
//     bit-identical sums, background and coefficients without another
//     launch, and block 0 alone writes the final Background back.
// The per-site arithmetic (drift, Eq. D, kick, sums) is that of sweep.cuh
// (Ctx<>::site, the same potentials and difference forms), so the FP64 and
// split-FP32 forms compute what the per-launch kernels compute, in a different
// (fixed) summation order.
//
// FP64 form: a plane is drifted once into a shared-memory buffer (one block
// barrier per plane), since FP64 arithmetic is the binding resource on GB300.
// Split-FP32 form: barrier-free warp pipeline (each warp drifts the three rows
// it needs in registers; "empty" mbarriers release slots; the producer role
// rotates over the warps), since that form is bound by memory traffic.
#pragma once

#include "sweep.cuh"

namespace pycool {

constexpr int kPThreads = 512;               // one block per SM
constexpr int kPWarps = kPThreads / 32;
constexpr int kPTY = kPWarps;                // tile rows: one per warp
constexpr int kColFieldBytes = 512;          // halo column of one field (y-wrap layout)
constexpr int kPSmemBudget = 220 * 1024;     // dynamic shared memory per block (227 KB less static)
constexpr int kKahanGroups = kPThreads / 4;  // split form: one compensated sum per 4 lanes
constexpr int kSplitLead = 6;                // split ring: planes in flight at most ...
constexpr int kSplitSlack = 3;               // ... and at least this many slots beyond them
static_assert(kPTY * 16 == 256, "column box layout assumes 16 rows of 16 bytes");
static_assert((kPTY + 2) * 16 <= kColFieldBytes, "a dense 18-row column fits a field's slot");

// Slot layout (elements of WORD bytes), every TMA destination 128-byte aligned:
//   main[arr][f][TY+2][TX]      rows 0 and TY+1 are the halo rows
//   col[arr][side][...]         the x-1 / x+TX halo columns of all fields, in one
//                               of two layouts: tiles clear of the y wrap get one
//                               dense box [f][TY+2][CW]; tiles at the wrap get per
//                               field [f][512 B: low cell | TY rows | high cell]
// H: halo rows (and z-halo planes) per side, 1 for the 7- and 27-point
// stencils, 2 for the 13-point one (main rows 0 .. H-1 and TY+H .. TY+2H-1 are
// halo rows; the column layouts are the same for both, a column box being 16
// bytes wide: two columns of 8-byte values).
template <int NF, int VX, int WORD, int H = 1>
struct PLayout {
  static constexpr int TX = 32 * VX;
  static constexpr int CW = 16 / WORD;                                // column box width
  static constexpr int MAIN = (kPTY + 2 * H) * TX;                    // elements per (array, field)
  static constexpr int COLF = kColFieldBytes / WORD;                  // elements per field column
  static constexpr int SLOT = 2 * NF * (MAIN + 2 * COLF);             // elements per slot
  static constexpr int SLOT_BYTES = SLOT * WORD;
  __device__ static constexpr int main_off(int arr, int f) { return (arr * NF + f) * MAIN; }
  __device__ static constexpr int col_base(int arr, int side) {
    return 2 * NF * MAIN + (arr * 2 + side) * NF * COLF;
  }
  // element offset of field f, column row r (0 = y0-1, 1..TY = tile rows, TY+1 = y0+TY)
  __device__ static constexpr int col_dense(int f, int r) { return (f * (kPTY + 2) + r) * CW; }
  __device__ static constexpr int col_wrap(int f, int r) {
    return f * COLF + (r == 0 ? 0 : (128 + (r - 1) * 16) / WORD);
  }
};

// TMA ring of a form: NSLOT slots, LEAD planes in flight ahead of the plane
// being computed.  FP64 (ALU-bound): three slots.  Split (memory-bound): as
// many slots as fit beside the compensated sums, at most ten, and LEAD =
// min(kSplitLead, NSLOT - kSplitSlack).  The slack lets the producer (whose
// role rotates over the warps) refill a slot while the slowest warp is still
// a few planes behind; on GB300, 6 planes in flight with 3-4 slots of slack
// beat both more planes with less slack and fewer planes with more (256^3:
// 7/3 0.446, 6/4 0.428, 5/5 0.434 ms per step).
//   FP64 extra: two drifted-plane buffers [NF][TY+2][TX] (one per plane parity)
//               and the block-reduction scratch [NQ][threads].
//   split extra: the compensated sums [NQ][threads / 4] float pairs, or every
//               block's row of the stage sums (the fold reads them there),
//               whichever is larger.
// The FP64 and split-DD forms (bound by arithmetic: ALU) share the FP64 ring.
template <int PREC, int NF, int VX, int NQ, int H = 1>
struct PRing {
  static constexpr bool ALU = PREC != PREC_SPLIT;
  using LY = PLayout<NF, VX, prec_word(PREC), H>;
  static constexpr int DRIFT_ELEMS = NF * (kPTY + 2 * H) * LY::TX;
  // FP64 and split-DD: NDRIFT planes in flight, each the drifted phi rows
  // (with the halo rows), the pi of the own rows (re-centred for split-DD) and
  // the halo-column values (up to 3 rows per edge lane)
  static constexpr int NDRIFT = ALU ? 4 : 2;
  static constexpr int PI_ELEMS = NF * kPTY * LY::TX;
  static constexpr int COL_ELEMS = NF * kPTY * 2 * 3;
  static constexpr int DRIFT_WORDS =
      ALU ? NDRIFT * (DRIFT_ELEMS + PI_ELEMS + COL_ELEMS) : 2 * DRIFT_ELEMS;
  static constexpr int KAHAN_BYTES = NQ * kKahanGroups * 8;
  static constexpr int ROWS_BYTES = kMaxPBlocks * kNQ * 8;
  static constexpr int EXTRA_BYTES =
      ALU ? DRIFT_WORDS * 8 + NQ * kPThreads * 8
          : (KAHAN_BYTES > ROWS_BYTES ? KAHAN_BYTES : ROWS_BYTES);
  static constexpr int FIT = (kPSmemBudget - EXTRA_BYTES) / LY::SLOT_BYTES;
  static constexpr int NSLOT = ALU ? 3 : (FIT < 10 ? FIT : 10);
  static constexpr int LEAD = ALU ? 2
                              : (NSLOT - kSplitSlack < kSplitLead ? NSLOT - kSplitSlack : kSplitLead);
  // warps that issue a stage's first LEAD planes at a stage boundary (the
  // others fold the block sums), each every PRE-th plane
  static constexpr int PRE = LEAD < kPWarps - NQ ? LEAD : kPWarps - NQ;
  static constexpr int RING_BYTES = NSLOT * LY::SLOT_BYTES;
  static constexpr int SMEM_BYTES = RING_BYTES + EXTRA_BYTES;
  static_assert(NSLOT >= 5 || ALU, "split ring too shallow");
  static_assert(SMEM_BYTES <= kPSmemBudget, "shared memory of the persistent kernel");
  static_assert(PRE >= 1, "a warp to issue the first planes beside the folds");
};

template <int STENCIL> constexpr int halo_of() { return STENCIL == 13 ? 2 : 1; }

template <int MODEL, int PREC, int VX, int STENCIL>
constexpr size_t persist_smem_bytes() {
  return (size_t)PRing<PREC, Pot<MODEL>::NF, VX, Slots<Pot<MODEL>::NF, PREC>::NQ,
                       halo_of<STENCIL>()>::SMEM_BYTES;
}

// Shared-memory state of a block, passed to the stage functions.
struct PShared {
  const SimDesc* d;       // shared-memory copy of the simulation descriptor
  unsigned char* ring;
  float2* kahan;          // split: [NQ][kKahanGroups] compensated sums (s, c)
  double* drift;          // FP64: two drifted planes [parity][NF][TY+2][TX]
  double* red;            // FP64: block-reduction scratch [NQ][kPThreads]
  uint64_t* full;
  uint64_t* empty;
  uint64_t* dbar;         // split-DD: per drift buffer, every warp has drifted its plane
  const int4* units;      // (x0, y0, z0, Q): tile origin, first output plane, planes incl. halos
  int nunits;
  uint32_t* issued;       // per slot: 1 + ring index of the last plane issued
  long long limit;        // clocks after which a wait gives up
};

// Vector store to global memory (st.global: the output arrays are global, and
// a generic store would make the address space a run-time question).
template <typename T, int VX>
__device__ __forceinline__ void gstore(T* p, const T (&v)[VX]) {
  using VT = typename Vec<T, VX>::type;
  VT x;
  T* e = reinterpret_cast<T*>(&x);
#pragma unroll
  for (int j = 0; j < VX; ++j) e[j] = v[j];
  __stwb(reinterpret_cast<VT*>(p), x);
}

// Advance a (unit, plane) position by one plane.
__device__ __forceinline__ void padvance(const PShared& sm, int& ui, int& uq) {
  if (ui < sm.nunits && ++uq == sm.units[ui].w) { ++ui; uq = 0; }
}

__device__ __forceinline__ void fence_proxy_async_global() {
  asm volatile("fence.proxy.async.global;" ::: "memory");
}
__device__ __forceinline__ unsigned long long ld_acquire_u64(const unsigned long long* p) {
  unsigned long long v;
  asm volatile("ld.acquire.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void red_release_add_u64(unsigned long long* p, unsigned long long v) {
  asm volatile("red.release.gpu.global.add.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}

// Grid barrier of the cooperative launch: a monotonic arrival counter.
// Thread 0 adds its arrival with release semantics (publishing the block's
// global writes, ordered before it by the block barrier) and polls the
// counter with acquire loads until every block of this barrier has arrived
// (target = arrivals before it + G).  The poll is bounded by `limit` clocks
// (~2^31, about a second, unless a test asks for less); on timeout it reports
// false instead of waiting on.
__device__ __forceinline__ bool grid_barrier(unsigned long long* count, unsigned long long target,
                                             long long limit) {
  bool ok = true;
  __syncthreads();
  if (threadIdx.x == 0) {
    red_release_add_u64(count, 1ull);
    if (ld_acquire_u64(count) < target) {
      const long long t0 = clock64();
      for (uint32_t i = 1; ld_acquire_u64(count) < target; ++i)
        if ((i & 63u) == 0u && clock64() - t0 > limit) { ok = false; break; }
    }
  }
  return ok;
}

__device__ __forceinline__ void tma_load_5d(void* dst, const CUtensorMap* map, int x, int y, int z,
                                            int f, int buf, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.tensor.5d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%2, %3, %4, %5, %6}], [%7];" ::"r"(smem_u32(dst)),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(z), "r"(f), "r"(buf),
      "r"(smem_u32(bar))
      : "memory");
}

// Does unit u's tile (rows y0-1 .. y0+TY) stay clear of the periodic y wrap?
__device__ __forceinline__ bool yclear(int4 u, int n) { return u.y > 0 && u.y + kPTY < n; }

// Issue the TMA copies of plane q of unit u into `slot` (one thread): tile,
// halo rows, halo columns (and, 27-point stencil, corner cells) of phi and pi
// of every field.  A tile clear of the y wrap takes 3 boxes per array (tile
// with both halo rows, two columns, all fields at once); a tile at the wrap
// takes its rows and cells one field at a time.  Every box is in bounds: x0
// and the column x are multiples of 16 bytes, wrapped rows are separate boxes.
//
// H = 2 (13-point stencil): the tile box and the wrap tiles' halo-row boxes are
// H rows deeper (their tensor maps are made so for such a simulation), the
// column boxes unchanged (two columns each, rows y0-1 .. y0+TY, of which the
// stencil uses the tile rows), and a unit starts H planes below its first
// output plane.
template <int NF, int VX, int WORD, bool CORNERS, int H = 1>
__device__ __forceinline__ void pproduce(const PParams& p, int ib, int4 u, int q,
                                         unsigned char* slot, uint64_t* bar) {
  static_assert(H == 1 || !CORNERS, "corner cells belong to the 27-point stencil");
  using LY = PLayout<NF, VX, WORD, H>;
  constexpr int TX = LY::TX, CW = LY::CW;
  constexpr uint32_t kClear = 2u * NF * ((kPTY + 2 * H) * TX * WORD + 2 * (kPTY + 2) * 16);
  constexpr uint32_t kWrap =
      2u * NF * ((kPTY + 2 * H) * TX * WORD + 2 * kPTY * 16 + (CORNERS ? 4 * 16 : 0));
  const int n = p.g.n;
  const int zw = wrapi(u.z - H + q, n);
  const int xl = (u.x == 0 ? n : u.x) - CW;
  const int xr = (u.x + TX == n) ? 0 : u.x + TX;
  const CUtensorMap* m = p.tm;
  if (yclear(u, n)) {
    mbar_expect_tx(bar, kClear);
#pragma unroll
    for (int arr = 0; arr < 2; ++arr) {
      const int bi = arr == 0 ? (ib & 1) : 2 + ((ib >> 1) & 1);   // buffer of phi / pi
      tma_load_5d(slot + (size_t)LY::main_off(arr, 0) * WORD, &m[0], u.x, u.y - H, zw, 0, bi, bar);
      tma_load_5d(slot + (size_t)LY::col_base(arr, 0) * WORD, &m[1], xl, u.y - 1, zw, 0, bi, bar);
      tma_load_5d(slot + (size_t)LY::col_base(arr, 1) * WORD, &m[1], xr, u.y - 1, zw, 0, bi, bar);
    }
    return;
  }
  // the H halo rows each side (rows never split across the wrap: n and the
  // tile origins are multiples of 16)
  const int yl = wrapi(u.y - H, n), yh = wrapi(u.y + kPTY, n);
  mbar_expect_tx(bar, kWrap);
#pragma unroll
  for (int arr = 0; arr < 2; ++arr) {
    const int bi = arr == 0 ? (ib & 1) : 2 + ((ib >> 1) & 1);
#pragma unroll
    for (int f = 0; f < NF; ++f) {
      unsigned char* mb = slot + (size_t)LY::main_off(arr, f) * WORD;
      tma_load_5d(mb + (size_t)H * TX * WORD, &m[2], u.x, u.y, zw, f, bi, bar);
      tma_load_5d(mb, &m[3], u.x, yl, zw, f, bi, bar);
      tma_load_5d(mb + (size_t)(kPTY + H) * TX * WORD, &m[3], u.x, yh, zw, f, bi, bar);
#pragma unroll
      for (int side = 0; side < 2; ++side) {
        unsigned char* cb = slot + (size_t)(LY::col_base(arr, side) + f * LY::COLF) * WORD;
        const int xc = side ? xr : xl;
        tma_load_5d(cb + 128, &m[4], xc, u.y, zw, f, bi, bar);
        if constexpr (CORNERS) {
          tma_load_5d(cb, &m[5], xc, yl, zw, f, bi, bar);
          tma_load_5d(cb + 128 + kPTY * 16, &m[5], xc, yh, zw, f, bi, bar);
        }
      }
    }
  }
}

// Stencil parts of one plane (Eq. D split by z-offset, as in sweep.cuh):
//   S_mid = c0 ctr + c1 faces + c2 corners,  S_off = c1 ctr + c2 faces + c3 corners.
// MID = false computes S_off only (the two z-halo planes of a unit).
template <typename T, int VX, bool CORNERS, bool MID>
__device__ __forceinline__ void plane_parts(const T (&ctr)[VX], const T (&dn)[VX], const T (&up)[VX],
                                            T left, T right, T dl, T dr, T ul, T ur,
                                            T (&smid)[VX], T (&so)[VX]) {
  const T c0 = CORNERS ? (T)(-128.0 / 30.0) : (T)(-6.0);
  const T c1 = CORNERS ? (T)(14.0 / 30.0) : (T)1.0;
  const T c2 = CORNERS ? (T)(3.0 / 30.0) : (T)0.0;
  const T c3 = CORNERS ? (T)(1.0 / 30.0) : (T)0.0;
#pragma unroll
  for (int j = 0; j < VX; ++j) {
    if constexpr (!CORNERS) {
      so[j] = ctr[j];
      if constexpr (MID) {
        const T L = j > 0 ? ctr[j - 1] : left;
        const T R = j < VX - 1 ? ctr[j + 1] : right;
        if constexpr (std::is_same<T, dd>::value)
          smid[j] = dd_sum4_axpy(dn[j], up[j], L, R, -6.0f, ctr[j]);
        else
          smid[j] = madd(c0, ctr[j], (dn[j] + up[j]) + (L + R));
      }
    } else {
      const T L = j > 0 ? ctr[j - 1] : left;
      const T R = j < VX - 1 ? ctr[j + 1] : right;
      const T faces = (dn[j] + up[j]) + (L + R);
      const T DL = j > 0 ? dn[j - 1] : dl;
      const T DR = j < VX - 1 ? dn[j + 1] : dr;
      const T UL = j > 0 ? up[j - 1] : ul;
      const T UR = j < VX - 1 ? up[j + 1] : ur;
      const T corners = (DL + DR) + (UL + UR);
      if constexpr (MID) smid[j] = madd(c2, corners, madd(c1, faces, c0 * ctr[j]));
      so[j] = madd(c3, corners, madd(c2, faces, c1 * ctr[j]));
    }
  }
}

__device__ __forceinline__ float shfl_up1(float v) { return __shfl_up_sync(0xffffffffu, v, 1); }
__device__ __forceinline__ double shfl_up1(double v) { return __shfl_up_sync(0xffffffffu, v, 1); }
__device__ __forceinline__ dd shfl_up1(dd v) { return dd_shfl_up(v, 1); }
__device__ __forceinline__ float shfl_down1(float v) { return __shfl_down_sync(0xffffffffu, v, 1); }
__device__ __forceinline__ double shfl_down1(double v) {
  return __shfl_down_sync(0xffffffffu, v, 1);
}
__device__ __forceinline__ dd shfl_down1(dd v) { return dd_shfl_down(v, 1); }

// x-neighbours of a lane's VX sites (shuffles; lanes 0 and 31 take the halo
// column) and the four diagonal neighbours (27-point stencil), then the parts.
template <typename T, int VX, bool CORNERS, bool MID, int CR>
__device__ __forceinline__ void lane_parts(const T (&ctr)[VX], const T (&dn)[VX], const T (&up)[VX],
                                           const T (&el)[CR], T (&smid)[VX], T (&so)[VX]) {
  const int lane = threadIdx.x & 31;
  T left = T(0.0), right = T(0.0), dl = T(0.0), dr = T(0.0), ul = T(0.0), ur = T(0.0);
  if (MID || CORNERS) {
    left = shfl_up1(ctr[VX - 1]);
    right = shfl_down1(ctr[0]);
    if (lane == 0) left = el[(CR - 1) / 2];
    if (lane == 31) right = el[(CR - 1) / 2];
  }
  if constexpr (CORNERS) {
    dl = shfl_up1(dn[VX - 1]);
    dr = shfl_down1(dn[0]);
    ul = shfl_up1(up[VX - 1]);
    ur = shfl_down1(up[0]);
    if (lane == 0) { dl = el[0]; ul = el[CR - 1]; }
    if (lane == 31) { dr = el[0]; ur = el[CR - 1]; }
  }
  plane_parts<T, VX, CORNERS, MID>(ctr, dn, up, left, right, dl, dr, ul, ur, smid, so);
}

// FP64 and split-DD forms: drift of ring plane gg (of unit uu) into drift
// buffer gg % NDRIFT, then this warp's arrival on the buffer's mbarrier.  Returns false if the plane's
// copies did not land within the limit (the buffer then holds garbage, which
// the caller never uses: the stage fails).
template <int MODEL, int STENCIL, int VX, int PREC>
__device__ __forceinline__ bool drift_alu(const Ctx<MODEL, PREC>& cx, const PShared& sm,
                                          uint32_t gg, int4 uu, int n) {
  static_assert(PREC == PREC_FP64 || PREC == PREC_DD, "the FP64 and split-DD forms");
  using T = typename std::conditional<PREC == PREC_DD, dd, double>::type;
  constexpr int NF = Ctx<MODEL, PREC>::NF;
  constexpr int NQ = Ctx<MODEL, PREC>::SL::NQ;
  constexpr bool CORNERS = StencilW<STENCIL>::kCorners;
  constexpr int CR = CORNERS ? 3 : 1;
  constexpr int H = halo_of<STENCIL>();
  using LY = PLayout<NF, VX, 8, H>;
  using RG = PRing<PREC, NF, VX, NQ, H>;
  constexpr int TX = LY::TX, CW = LY::CW, NSLOT = RG::NSLOT, NB = RG::NDRIFT;
  static_assert(H == 1 || CW >= 2, "two halo columns per column box");
  const int tid = threadIdx.x, lane = tid & 31, ly = tid >> 5;
  const int side = lane == 31 ? 1 : 0;
  const bool edge = lane == 0 || lane == 31;
  const int own = (ly + H) * TX + lane * VX;
  const int s = gg % NSLOT, b = gg % NB;
  // the 2H halo rows of this plane go to warps 2H j .. 2H j + 2H - 1, j = gg mod (16 / 2H)
  const int hw = (ly - 2 * H * (int)(gg % (kPWarps / (2 * H))) + kPWarps) % kPWarps;
  const bool ok = mbar_wait(&sm.full[s], (gg / NSLOT) & 1, sm.limit);
  const T* sl = (const T*)(sm.ring + (size_t)s * LY::SLOT_BYTES);
  T* dp = reinterpret_cast<T*>(sm.drift) + (size_t)b * RG::DRIFT_ELEMS;
  T* pp = reinterpret_cast<T*>(sm.drift) + (size_t)NB * RG::DRIFT_ELEMS + (size_t)b * RG::PI_ELEMS;
  T* cp = reinterpret_cast<T*>(sm.drift) + (size_t)NB * (RG::DRIFT_ELEMS + RG::PI_ELEMS) +
          (size_t)b * RG::COL_ELEMS;
  const T cd = cx.cdrift;
  const bool clear = yclear(uu, n);
#pragma unroll
  for (int f = 0; f < NF; ++f) {
    const T* mph = sl + LY::main_off(0, f);
    const T* mpi = sl + LY::main_off(1, f);
    T* dph = dp + f * (kPTY + 2 * H) * TX;
    T a[VX], c[VX];
    vload<T, VX>(&mph[own], a);
    vload<T, VX>(&mpi[own], c);
    T q[VX];
#pragma unroll
    for (int jj = 0; jj < VX; ++jj) {
      if constexpr (PREC == PREC_DD) q[jj] = c[jj] - cx.mu_pi[f];   // re-centred
      else q[jj] = c[jj];
      a[jj] = madd(cd, c[jj], a[jj]);
    }
    vstore<T, VX>(&dph[own], a);
    vstore<T, VX>(&pp[(f * kPTY + ly) * TX + lane * VX], q);
    if (hw < 2 * H) {   // the halo rows rotate over the warps, plane by plane
      const int r = (hw < H ? hw : kPTY + hw) * TX + lane * VX;
      vload<T, VX>(&mph[r], a);
      vload<T, VX>(&mpi[r], c);
#pragma unroll
      for (int jj = 0; jj < VX; ++jj) a[jj] = madd(cd, c[jj], a[jj]);
      vstore<T, VX>(&dph[r], a);
    }
    if (edge) {
      if constexpr (H == 1) {   // the adjacent column, rows ly - 1 .. ly + 1 (CR of them)
        const T* cph = sl + LY::col_base(0, side) + (side ? 0 : CW - 1);
        const T* cpi = sl + LY::col_base(1, side) + (side ? 0 : CW - 1);
#pragma unroll
        for (int rr = 0; rr < CR; ++rr) {
          const int r = ly + 1 + rr - (CR - 1) / 2;
          const int row = clear ? LY::col_dense(f, r) : LY::col_wrap(f, r);
          cp[((f * kPTY + ly) * 2 + side) * 3 + rr] = madd(cd, cpi[row], cph[row]);
        }
      } else {   // both columns of this side (k = 0 adjacent, 1 far), row ly
        const int row = clear ? LY::col_dense(f, ly + 1) : LY::col_wrap(f, ly + 1);
#pragma unroll
        for (int k = 0; k < 2; ++k) {
          const int cc = side ? k : CW - 1 - k;
          const T* cph = sl + LY::col_base(0, side) + cc;
          const T* cpi = sl + LY::col_base(1, side) + cc;
          cp[((f * kPTY + ly) * 2 + side) * 3 + k] = madd(cd, cpi[row], cph[row]);
        }
      }
    }
  }
  // The ring slot read above is refilled by a TMA copy (async proxy) once
  // every warp has arrived: a proxy fence orders this thread's generic reads
  // of it before that write.
  fence_proxy_async();
  // one arrival for the warp: __syncwarp orders the lanes' shared-memory
  // writes before lane 0's arrival, whose release makes them visible to the
  // threads whose wait (acquire) observes the completed phase
  __syncwarp();
  if (lane == 0) mbar_arrive(&sm.dbar[b]);
  return ok;
}

// ---------------------------------------------------------------------------
// FP64 form.
// ---------------------------------------------------------------------------
// One stage of the FP64 form over this block's units.  The planes flow
// through the drift buffers as in the split-DD form (below): each warp drifts
// plane g + 1 (drift_alu), then waits until every warp has drifted plane g and
// computes it, with no block barrier in the z loop; the halo rows and the copy
// issue rotate over the warps.  Returns false if a wait gave up (the caller
// combines the threads' results).  gq: ring planes consumed before this stage.
template <int MODEL, int STENCIL, int VX, int MODE>
__device__ __forceinline__ bool stage_fp64(const PParams& p, const Ctx<MODEL, PREC_FP64>& cx,
                                           const PShared& sm, uint32_t gq, int ib, double* accd) {
  using C = Ctx<MODEL, PREC_FP64>;
  using T = double;
  using SL = typename C::SL;
  constexpr int NF = C::NF;
  constexpr bool CORNERS = StencilW<STENCIL>::kCorners;
  constexpr int CR = CORNERS ? 3 : 1;
  using LY = PLayout<NF, VX, 8>;
  using RG = PRing<PREC_FP64, NF, VX, SL::NQ>;
  constexpr int TX = LY::TX;
  constexpr int NSLOT = RG::NSLOT, LEAD = RG::LEAD, NB = RG::NDRIFT;
  static_assert(LEAD + 1 == NSLOT, "the stage issues plane gq + LEAD, then g + NSLOT at plane g");
  const SimDesc& d = *sm.d;
  const int tid = threadIdx.x, lane = tid & 31, ly = tid >> 5;
  const int n = p.g.n;
  const size_t S = (size_t)d.S, nn = (size_t)n * n;
  T* __restrict__ phi_out = (T*)d.phi[(ib & 1) ^ 1];
  T* __restrict__ pi_out = (T*)d.pi[((ib >> 1) & 1) ^ 1];
  const int side = lane == 31 ? 1 : 0;
  const bool edge = lane == 0 || lane == 31;
  const int own = (ly + 1) * TX + lane * VX;          // this lane's sites in a slot row
  bool ok = true;

  // producer position (see stage_dd): plane gq + LEAD now, plane g + NSLOT at plane g
  int pui = 0, puq = 0;
  for (int l = 0; l < LEAD; ++l) padvance(sm, pui, puq);
  if (tid == kPThreads - 32 && pui < sm.nunits) {
    const uint32_t gp = gq + LEAD;
    pproduce<NF, VX, 8, CORNERS>(p, ib, sm.units[pui], puq,
                                 sm.ring + (size_t)(gp % NSLOT) * LY::SLOT_BYTES,
                                 &sm.full[gp % NSLOT]);
    sm.issued[gp % NSLOT] = gp + 1;
  }
  padvance(sm, pui, puq);

  uint32_t g = gq;
  if (sm.nunits > 0) ok = drift_alu<MODEL, STENCIL, VX, PREC_FP64>(cx, sm, g, sm.units[0], n);
  for (int i = 0; i < sm.nunits && ok; ++i) {
    const int4 u = sm.units[i];
    const int Q = u.w;
    const size_t o0 = (size_t)u.z * nn + (size_t)(u.y + ly) * n + u.x + lane * VX;
    T part_m[NF][VX], so_m[NF][VX], ph_m[NF][VX], pi_m[NF][VX];
#pragma unroll
    for (int f = 0; f < NF; ++f)
#pragma unroll
      for (int jj = 0; jj < VX; ++jj) part_m[f][jj] = so_m[f][jj] = ph_m[f][jj] = pi_m[f][jj] = 0.0;
    for (int q = 0; q < Q; ++q, ++g) {
      // look ahead: drift the stage's next plane
      if (q + 1 < Q)
        ok = drift_alu<MODEL, STENCIL, VX, PREC_FP64>(cx, sm, g + 1, u, n) && ok;
      else if (i + 1 < sm.nunits)
        ok = drift_alu<MODEL, STENCIL, VX, PREC_FP64>(cx, sm, g + 1, sm.units[i + 1], n) && ok;
      // every warp has drifted plane g
      ok = mbar_wait(&sm.dbar[g % NB], (g / NB) & 1, sm.limit) && ok;
      if (!ok) break;
      if (tid == 32 * (int)((2 * ((g + 1) % (kPWarps / 2)) + 2) % kPWarps) && pui < sm.nunits) {
        const uint32_t gp = g + NSLOT;   // into slot g % NSLOT, free now
        pproduce<NF, VX, 8, CORNERS>(p, ib, sm.units[pui], puq,
                                     sm.ring + (size_t)(gp % NSLOT) * LY::SLOT_BYTES,
                                     &sm.full[gp % NSLOT]);
        sm.issued[gp % NSLOT] = gp + 1;
      }
      padvance(sm, pui, puq);

      const int b = g % NB;
      const T* dp = sm.drift + (size_t)b * RG::DRIFT_ELEMS;
      const T* pp = sm.drift + (size_t)NB * RG::DRIFT_ELEMS + (size_t)b * RG::PI_ELEMS;
      const T* cp = sm.drift + (size_t)NB * (RG::DRIFT_ELEMS + RG::PI_ELEMS) +
                    (size_t)b * RG::COL_ELEMS;
      T cur_ph[NF][VX], cur_pi[NF][VX], el[NF][CR];
      const bool mid = q > 0 && q < Q - 1;   // the z-halo planes need S_off only
      T so_new[NF][VX], smid_new[NF][VX];
#pragma unroll
      for (int f = 0; f < NF; ++f) {
        const T* dph = dp + f * (kPTY + 2) * TX;
        vload<T, VX>(&dph[own], cur_ph[f]);
        vload<T, VX>(&pp[(f * kPTY + ly) * TX + lane * VX], cur_pi[f]);
#pragma unroll
        for (int rr = 0; rr < CR; ++rr)
          el[f][rr] = edge ? cp[((f * kPTY + ly) * 2 + side) * 3 + rr] : 0.0;
        T dn[VX], up[VX];
#pragma unroll
        for (int jj = 0; jj < VX; ++jj) dn[jj] = up[jj] = 0.0;
        if (mid || CORNERS) {
          vload<T, VX>(&dph[own - TX], dn);
          vload<T, VX>(&dph[own + TX], up);
        }
        if (mid)
          lane_parts<T, VX, CORNERS, true, CR>(cur_ph[f], dn, up, el[f], smid_new[f], so_new[f]);
        else
          lane_parts<T, VX, CORNERS, false, CR>(cur_ph[f], dn, up, el[f], smid_new[f], so_new[f]);
      }
      if (q >= 2) {  // output plane z0 + q - 2
        const size_t o = o0 + (size_t)(q - 2) * nn;
        T pin[NF][VX];
#pragma unroll
        for (int jj = 0; jj < VX; ++jj) {
          T phj[NF], Dj[NF], pmj[NF], pnj[NF];
#pragma unroll
          for (int f = 0; f < NF; ++f) {
            phj[f] = ph_m[f][jj];
            Dj[f] = part_m[f][jj] + so_new[f][jj];
            pmj[f] = pi_m[f][jj];
          }
          cx.site(MODE, phj, Dj, pmj, pnj, accd);
#pragma unroll
          for (int f = 0; f < NF; ++f) pin[f][jj] = pnj[f];
        }
#pragma unroll
        for (int f = 0; f < NF; ++f) {
          gstore<T, VX>(phi_out + f * S + o, ph_m[f]);
          if (MODE == MODE_SWEEP) gstore<T, VX>(pi_out + f * S + o, pin[f]);
        }
      }
      if (mid) {
#pragma unroll
        for (int f = 0; f < NF; ++f)
#pragma unroll
          for (int jj = 0; jj < VX; ++jj)
            part_m[f][jj] = (CORNERS ? so_m[f][jj] : ph_m[f][jj]) + smid_new[f][jj];
      }
#pragma unroll
      for (int f = 0; f < NF; ++f)
#pragma unroll
        for (int jj = 0; jj < VX; ++jj) {
          if constexpr (CORNERS) so_m[f][jj] = so_new[f][jj];
          ph_m[f][jj] = cur_ph[f][jj];
          pi_m[f][jj] = cur_pi[f][jj];
        }
    }
  }
  return ok;
}

// ---------------------------------------------------------------------------
// Split-DD form: phi = phi0 + d with the background phi0 in float64 (advanced
// by the scalar chain) and the fluctuation d stored and updated as a
// double-float (two float32 per value, 8 bytes: the traffic of the FP64
// form).  The arithmetic is that of the split-FP32 form (stencil on
// phi + c pi, re-centred output, difference forms of V') in double-float on
// the FP32 pipe.
//
// Planes flow through NDRIFT shared-memory drift buffers without a block
// barrier in the z loop: at plane g a warp first drifts plane g + 1 (its own
// row, the halo rows for warps 2j and 2j + 1, j = (g + 1) mod 8, the halo
// columns for lanes 0 and 31)
// into buffer (g + 1) % NDRIFT and arrives on that buffer's mbarrier, then
// waits until every warp has drifted plane g and computes plane g from buffer
// g % NDRIFT.  A warp can so run up to one plane ahead of the slowest one.
// Buffer (g + 1) % NDRIFT was last read for plane g + 1 - NDRIFT; a warp
// writing it has passed the wait for plane g - 1, which every warp arrived at
// after finishing plane g - 3, so NDRIFT = 4 buffers suffice.  Ring slot
// g % NSLOT is free once every warp has drifted plane g: the last warp then
// issues plane g + NSLOT into it.
// ---------------------------------------------------------------------------
// One stage over this block's units.  This thread's stage sums (NQ
// double-floats, the running accumulators folded in every KGROUP planes) live
// in its own slots of the block-reduction scratch, sm.red[q * threads + tid]
// (free during the sweep), to keep registers for the sweep.
// Returns false if a wait gave up (the caller combines the threads' results).
template <int MODEL, int STENCIL, int VX, int MODE>
__device__ __forceinline__ bool stage_dd(const PParams& p, const Ctx<MODEL, PREC_DD>& cx,
                                         const PShared& sm, uint32_t gq, int ib) {
  using C = Ctx<MODEL, PREC_DD>;
  using T = dd;
  using SL = typename C::SL;
  constexpr int NF = C::NF;
  constexpr int NQ = SL::NQ;
  constexpr bool CORNERS = StencilW<STENCIL>::kCorners;
  constexpr int CR = CORNERS ? 3 : 1;
  using LY = PLayout<NF, VX, 8>;
  using RG = PRing<PREC_DD, NF, VX, NQ>;
  constexpr int TX = LY::TX;
  constexpr int NSLOT = RG::NSLOT, LEAD = RG::LEAD, NB = RG::NDRIFT;
  constexpr int KGROUP = 8;   // output planes per running accumulator before it is folded
  static_assert(LEAD + 1 == NSLOT, "the stage issues plane gq + LEAD, then g + NSLOT at plane g");
  const SimDesc& d = *sm.d;
  const int tid = threadIdx.x, lane = tid & 31, ly = tid >> 5;
  const int n = p.g.n;
  const size_t S = (size_t)d.S, nn = (size_t)n * n;
  T* __restrict__ phi_out = (T*)d.phi[(ib & 1) ^ 1];
  T* __restrict__ pi_out = (T*)d.pi[((ib >> 1) & 1) ^ 1];
  const T cd = cx.cdrift;
  // re-centring: phi* = phi + c pi - (mu_phi + c mu_pi); the stencil works on
  // phi + c pi (D of a constant is zero)
  T Mf[NF];
#pragma unroll
  for (int f = 0; f < NF; ++f) Mf[f] = dd_fma(cd, cx.mu_pi[f], cx.mu_phi[f]);
  const int own = (ly + 1) * TX + lane * VX;          // this lane's sites in a slot row
  const int side = lane == 31 ? 1 : 0;
  const bool edge = lane == 0 || lane == 31;
  DDAcc acc[NQ];
  dd* tot = reinterpret_cast<dd*>(sm.red) + tid;        // tot[q * kPThreads]
#pragma unroll
  for (int i = 0; i < NQ; ++i) {
    acc[i].zero();
    tot[i * kPThreads] = dd(0.f, 0.f);
  }
  int kg = 0;
  bool ok = true;

  // producer position: the kernel issued planes gq .. gq + LEAD - 1; this
  // stage issues plane gq + LEAD now (its slot held the previous stage's last
  // plane, drifted by every warp) and plane g + NSLOT at plane g
  int pui = 0, puq = 0;
  for (int l = 0; l < LEAD; ++l) padvance(sm, pui, puq);
  const bool producer = tid == kPThreads - 32;
  if (producer && pui < sm.nunits) {
    const uint32_t gp = gq + LEAD;
    pproduce<NF, VX, 8, CORNERS>(p, ib, sm.units[pui], puq,
                                 sm.ring + (size_t)(gp % NSLOT) * LY::SLOT_BYTES,
                                 &sm.full[gp % NSLOT]);
    sm.issued[gp % NSLOT] = gp + 1;
  }
  padvance(sm, pui, puq);

  uint32_t g = gq;
  if (sm.nunits > 0) ok = drift_alu<MODEL, STENCIL, VX, PREC_DD>(cx, sm, g, sm.units[0], n);
  for (int i = 0; i < sm.nunits && ok; ++i) {
    const int4 u = sm.units[i];
    const int Q = u.w;
    const size_t o0 = (size_t)u.z * nn + (size_t)(u.y + ly) * n + u.x + lane * VX;
    T part_m[NF][VX], so_m[NF][VX], ph_m[NF][VX], pi_m[NF][VX];
#pragma unroll
    for (int f = 0; f < NF; ++f)
#pragma unroll
      for (int jj = 0; jj < VX; ++jj)
        part_m[f][jj] = so_m[f][jj] = ph_m[f][jj] = pi_m[f][jj] = T(0.0);
    for (int q = 0; q < Q; ++q, ++g) {
      // look ahead: drift the stage's next plane
      if (q + 1 < Q)
        ok = drift_alu<MODEL, STENCIL, VX, PREC_DD>(cx, sm, g + 1, u, n) && ok;
      else if (i + 1 < sm.nunits)
        ok = drift_alu<MODEL, STENCIL, VX, PREC_DD>(cx, sm, g + 1, sm.units[i + 1], n) && ok;
      // every warp has drifted plane g
      ok = mbar_wait(&sm.dbar[g % NB], (g / NB) & 1, sm.limit) && ok;
      if (!ok) break;
      // the copies of plane g + NSLOT: lane 0 of the warp two after the ones
      // that drift plane g + 1's halo rows
      if (tid == 32 * (int)((2 * ((g + 1) % (kPWarps / 2)) + 2) % kPWarps) && pui < sm.nunits) {
        const uint32_t gp = g + NSLOT;   // into slot g % NSLOT, free now
        pproduce<NF, VX, 8, CORNERS>(p, ib, sm.units[pui], puq,
                                     sm.ring + (size_t)(gp % NSLOT) * LY::SLOT_BYTES,
                                     &sm.full[gp % NSLOT]);
        sm.issued[gp % NSLOT] = gp + 1;
      }
      padvance(sm, pui, puq);

      const int b = g % NB;
      const T* dp = reinterpret_cast<const T*>(sm.drift) + (size_t)b * RG::DRIFT_ELEMS;
      const T* pp = reinterpret_cast<const T*>(sm.drift) + (size_t)NB * RG::DRIFT_ELEMS +
                    (size_t)b * RG::PI_ELEMS;
      const T* cp = reinterpret_cast<const T*>(sm.drift) +
                    (size_t)NB * (RG::DRIFT_ELEMS + RG::PI_ELEMS) + (size_t)b * RG::COL_ELEMS;
      T cur_ph[NF][VX], cur_pi[NF][VX], el[NF][CR];
      const bool mid = q > 0 && q < Q - 1;   // the z-halo planes need S_off only
      T so_new[NF][VX], smid_new[NF][VX];
#pragma unroll
      for (int f = 0; f < NF; ++f) {
        const T* dph = dp + f * (kPTY + 2) * TX;
        vload<T, VX>(&dph[own], cur_ph[f]);
        vload<T, VX>(&pp[(f * kPTY + ly) * TX + lane * VX], cur_pi[f]);
#pragma unroll
        for (int rr = 0; rr < CR; ++rr)
          el[f][rr] = edge ? cp[((f * kPTY + ly) * 2 + side) * 3 + rr] : T(0.0);
        T dn[VX], up[VX];
#pragma unroll
        for (int jj = 0; jj < VX; ++jj) dn[jj] = up[jj] = T(0.0);
        if (mid || CORNERS) {
          vload<T, VX>(&dph[own - TX], dn);
          vload<T, VX>(&dph[own + TX], up);
        }
        if (mid)
          lane_parts<T, VX, CORNERS, true, CR>(cur_ph[f], dn, up, el[f], smid_new[f], so_new[f]);
        else
          lane_parts<T, VX, CORNERS, false, CR>(cur_ph[f], dn, up, el[f], smid_new[f], so_new[f]);
      }
      if (q >= 2) {  // output plane z0 + q - 2
        const size_t o = o0 + (size_t)(q - 2) * nn;
        T pin[NF][VX], phs[NF][VX];
#pragma unroll
        for (int jj = 0; jj < VX; ++jj) {
          T phj[NF], Dj[NF], pmj[NF], pnj[NF];
#pragma unroll
          for (int f = 0; f < NF; ++f) {
            phs[f][jj] = ph_m[f][jj] - Mf[f];   // the re-centred drifted field
            phj[f] = phs[f][jj];
            Dj[f] = part_m[f][jj] + so_new[f][jj];
            pmj[f] = pi_m[f][jj];
          }
          site_dd<MODEL>(cx, MODE, phj, Dj, pmj, pnj, acc);
#pragma unroll
          for (int f = 0; f < NF; ++f) pin[f][jj] = pnj[f];
        }
#pragma unroll
        for (int f = 0; f < NF; ++f) {
          gstore<T, VX>(phi_out + f * S + o, phs[f]);
          if (MODE == MODE_SWEEP) gstore<T, VX>(pi_out + f * S + o, pin[f]);
        }
        if (++kg == KGROUP) {
          kg = 0;
#pragma unroll
          for (int i2 = 0; i2 < NQ; ++i2) {
            dd t = tot[i2 * kPThreads];
            acc[i2].fold(t);
            tot[i2 * kPThreads] = t;
          }
        }
      }
      if (mid) {
#pragma unroll
        for (int f = 0; f < NF; ++f)
#pragma unroll
          for (int jj = 0; jj < VX; ++jj)
            part_m[f][jj] = (CORNERS ? so_m[f][jj] : ph_m[f][jj]) + smid_new[f][jj];
      }
#pragma unroll
      for (int f = 0; f < NF; ++f)
#pragma unroll
        for (int jj = 0; jj < VX; ++jj) {
          if constexpr (CORNERS) so_m[f][jj] = so_new[f][jj];
          ph_m[f][jj] = cur_ph[f][jj];
          pi_m[f][jj] = cur_pi[f][jj];
        }
    }
  }
#pragma unroll
  for (int i2 = 0; i2 < NQ; ++i2) {
    dd t = tot[i2 * kPThreads];
    acc[i2].fold(t);
    tot[i2 * kPThreads] = t;
  }
  return ok;
}

// ---------------------------------------------------------------------------
// 13-point (fourth-order) stencil, FP64 and split-DD forms: per axis
// D_axis = (-f(-2) + 16 f(-1) - 30 f(0) + 16 f(+1) - f(+2)) / 12 (Sec. 2.1,
// after Eq. G).  The planes flow through the drift pipeline of the other
// stencils with two halo rows, columns and planes each side.  A plane's
// in-plane part m = w1 (x and y neighbours at 1) + w2 (at 2) + w0 centre (w0
// for all three axes) is completed along z by a queue of two partial sums: when
// plane p arrives, plane p - 2 gets its last term w2 f(p) and is output, plane
// p - 1 gets w1 f(p), and plane p starts as m(p) + w1 f(p - 1) + w2 f(p - 2).
// The split-DD form sums 12 D with the integer weights (16, -1, -90: exact in
// float) and multiplies by 1/12 once per site.
// ---------------------------------------------------------------------------
template <typename T, int VX>
__device__ __forceinline__ void wide_shuffles(const T (&ctr)[VX], T (&e)[VX + 4]) {
  // e[j + 2] = the drifted value at x0 + lane VX + j, j = -2 .. VX + 1
#pragma unroll
  for (int j = 0; j < VX; ++j) e[j + 2] = ctr[j];
  if constexpr (VX == 1) {
    e[1] = shfl_up1(ctr[0]);
    e[3] = shfl_down1(ctr[0]);
    e[0] = shfl_up1(e[1]);     // lane - 2
    e[4] = shfl_down1(e[3]);   // lane + 2
  } else {
    static_assert(VX == 2, "one or two sites per lane");
    e[0] = shfl_up1(ctr[0]);
    e[1] = shfl_up1(ctr[1]);
    e[4] = shfl_down1(ctr[0]);
    e[5] = shfl_down1(ctr[1]);
  }
}

template <int MODEL, int VX, int MODE, int PREC>
__device__ __forceinline__ bool stage_wide(const PParams& p, const Ctx<MODEL, PREC>& cx,
                                           const PShared& sm, uint32_t gq, int ib, double* accd) {
  using C = Ctx<MODEL, PREC>;
  using T = typename std::conditional<PREC == PREC_DD, dd, double>::type;
  using SL = typename C::SL;
  constexpr int NF = C::NF;
  constexpr int NQ = SL::NQ;
  constexpr int H = 2;
  using LY = PLayout<NF, VX, 8, H>;
  using RG = PRing<PREC, NF, VX, NQ, H>;
  constexpr int TX = LY::TX;
  constexpr int NSLOT = RG::NSLOT, LEAD = RG::LEAD, NB = RG::NDRIFT;
  constexpr int KGROUP = 8;   // split-DD: output planes per running accumulator
  static_assert(LEAD + 1 == NSLOT, "the stage issues plane gq + LEAD, then g + NSLOT at plane g");
  const SimDesc& d = *sm.d;
  const int tid = threadIdx.x, lane = tid & 31, ly = tid >> 5;
  const int n = p.g.n;
  const size_t S = (size_t)d.S, nn = (size_t)n * n;
  T* __restrict__ phi_out = (T*)d.phi[(ib & 1) ^ 1];
  T* __restrict__ pi_out = (T*)d.pi[((ib >> 1) & 1) ^ 1];
  const int own = (ly + H) * TX + lane * VX;
  // weights: FP64 the stencil's own; split-DD 12 x them, then 1/12 at the end
  const T w1 = PREC == PREC_DD ? T(16.0) : T(16.0 / 12.0);
  const T w2 = PREC == PREC_DD ? T(-1.0) : T(-1.0 / 12.0);
  const T w0 = PREC == PREC_DD ? T(-90.0) : T(-90.0 / 12.0);
  const T inv12 = T(1.0 / 12.0);
  T Mf[NF];   // split-DD: the re-centring of the drifted field
#pragma unroll
  for (int f = 0; f < NF; ++f) {
    if constexpr (PREC == PREC_DD) Mf[f] = dd_fma(cx.cdrift, cx.mu_pi[f], cx.mu_phi[f]);
    else Mf[f] = 0.0;
  }
  DDAcc acc[PREC == PREC_DD ? NQ : 1];
  dd* tot = reinterpret_cast<dd*>(sm.red) + tid;   // split-DD stage sums, tot[q * kPThreads]
  if constexpr (PREC == PREC_DD) {
#pragma unroll
    for (int i = 0; i < NQ; ++i) {
      acc[i].zero();
      tot[i * kPThreads] = dd(0.f, 0.f);
    }
  }
  int kg = 0;
  bool ok = true;

  int pui = 0, puq = 0;
  for (int l = 0; l < LEAD; ++l) padvance(sm, pui, puq);
  if (tid == kPThreads - 32 && pui < sm.nunits) {
    const uint32_t gp = gq + LEAD;
    pproduce<NF, VX, 8, false, H>(p, ib, sm.units[pui], puq,
                                  sm.ring + (size_t)(gp % NSLOT) * LY::SLOT_BYTES,
                                  &sm.full[gp % NSLOT]);
    sm.issued[gp % NSLOT] = gp + 1;
  }
  padvance(sm, pui, puq);

  uint32_t g = gq;
  if (sm.nunits > 0) ok = drift_alu<MODEL, 13, VX, PREC>(cx, sm, g, sm.units[0], n);
  for (int i = 0; i < sm.nunits && ok; ++i) {
    const int4 u = sm.units[i];
    const int Q = u.w;
    const size_t o0 = (size_t)u.z * nn + (size_t)(u.y + ly) * n + u.x + lane * VX;
    // z queue: partial sums of planes p-1, p-2; drifted field and momentum at p-1, p-2
    T P1[NF][VX], P2[NF][VX], c1[NF][VX], c2[NF][VX], q1[NF][VX], q2[NF][VX];
#pragma unroll
    for (int f = 0; f < NF; ++f)
#pragma unroll
      for (int jj = 0; jj < VX; ++jj)
        P1[f][jj] = P2[f][jj] = c1[f][jj] = c2[f][jj] = q1[f][jj] = q2[f][jj] = T(0.0);
    for (int q = 0; q < Q; ++q, ++g) {
      if (q + 1 < Q)
        ok = drift_alu<MODEL, 13, VX, PREC>(cx, sm, g + 1, u, n) && ok;
      else if (i + 1 < sm.nunits)
        ok = drift_alu<MODEL, 13, VX, PREC>(cx, sm, g + 1, sm.units[i + 1], n) && ok;
      ok = mbar_wait(&sm.dbar[g % NB], (g / NB) & 1, sm.limit) && ok;
      if (!ok) break;
      if (tid == 32 * (int)((4 * ((g + 1) % (kPWarps / 4)) + 4) % kPWarps) && pui < sm.nunits) {
        const uint32_t gp = g + NSLOT;   // into slot g % NSLOT, free now
        pproduce<NF, VX, 8, false, H>(p, ib, sm.units[pui], puq,
                                      sm.ring + (size_t)(gp % NSLOT) * LY::SLOT_BYTES,
                                      &sm.full[gp % NSLOT]);
        sm.issued[gp % NSLOT] = gp + 1;
      }
      padvance(sm, pui, puq);
      const int b = g % NB;
      const T* dp = reinterpret_cast<const T*>(sm.drift) + (size_t)b * RG::DRIFT_ELEMS;
      const T* pp = reinterpret_cast<const T*>(sm.drift) + (size_t)NB * RG::DRIFT_ELEMS +
                    (size_t)b * RG::PI_ELEMS;
      const T* cp = reinterpret_cast<const T*>(sm.drift) +
                    (size_t)NB * (RG::DRIFT_ELEMS + RG::PI_ELEMS) + (size_t)b * RG::COL_ELEMS;
      const bool mid = q >= 2 && q < Q - 2;   // a plane whose sites are output
      T cur[NF][VX], qn[NF][VX], D[NF][VX];
#pragma unroll
      for (int f = 0; f < NF; ++f) {
        const T* dph = dp + f * (kPTY + 2 * H) * TX;
        vload<T, VX>(&dph[own], cur[f]);
        vload<T, VX>(&pp[(f * kPTY + ly) * TX + lane * VX], qn[f]);
        T m[VX];
#pragma unroll
        for (int jj = 0; jj < VX; ++jj) m[jj] = T(0.0);
        if (mid) {   // q is the same in the whole block: every lane shuffles
          T e[VX + 4];
          wide_shuffles<T, VX>(cur[f], e);
          // the lanes at the tile's x edges take the halo columns ([0] adjacent, [1] far)
          const T* cl = cp + ((f * kPTY + ly) * 2 + 0) * 3;
          const T* cr = cp + ((f * kPTY + ly) * 2 + 1) * 3;
          if (lane == 0) { e[1] = cl[0]; e[0] = cl[1]; }
          if (lane == 31) { e[VX + 2] = cr[0]; e[VX + 3] = cr[1]; }
          if constexpr (VX == 1) {
            if (lane == 1) e[0] = cl[0];
            if (lane == 30) e[4] = cr[0];
          }
          T dn1[VX], up1[VX], dn2[VX], up2[VX];
          vload<T, VX>(&dph[own - TX], dn1);
          vload<T, VX>(&dph[own + TX], up1);
          vload<T, VX>(&dph[own - 2 * TX], dn2);
          vload<T, VX>(&dph[own + 2 * TX], up2);
#pragma unroll
          for (int jj = 0; jj < VX; ++jj) {
            const T nr = (dn1[jj] + up1[jj]) + (e[jj + 1] + e[jj + 3]);
            const T fr = (dn2[jj] + up2[jj]) + (e[jj] + e[jj + 4]);
            m[jj] = madd(w0, cur[f][jj], madd(w2, fr, w1 * nr));
          }
        }
#pragma unroll
        for (int jj = 0; jj < VX; ++jj) {
          D[f][jj] = madd(w2, cur[f][jj], P2[f][jj]);   // plane p - 2: its last term
          const T np1 = madd(w1, cur[f][jj], P1[f][jj]);
          P1[f][jj] = madd(w2, c2[f][jj], madd(w1, c1[f][jj], m[jj]));
          P2[f][jj] = np1;
        }
      }
      if (q >= 4) {  // output plane z0 + q - 4
        const size_t o = o0 + (size_t)(q - 4) * nn;
        T pin[NF][VX], phs[NF][VX];
#pragma unroll
        for (int jj = 0; jj < VX; ++jj) {
          T phj[NF], Dj[NF], pmj[NF], pnj[NF];
#pragma unroll
          for (int f = 0; f < NF; ++f) {
            if constexpr (PREC == PREC_DD) {
              phs[f][jj] = c2[f][jj] - Mf[f];   // the re-centred drifted field
              Dj[f] = D[f][jj] * inv12;
            } else {
              phs[f][jj] = c2[f][jj];
              Dj[f] = D[f][jj];
            }
            phj[f] = phs[f][jj];
            pmj[f] = q2[f][jj];
          }
          if constexpr (PREC == PREC_DD) site_dd<MODEL>(cx, MODE, phj, Dj, pmj, pnj, acc);
          else cx.site(MODE, phj, Dj, pmj, pnj, accd);
#pragma unroll
          for (int f = 0; f < NF; ++f) pin[f][jj] = pnj[f];
        }
#pragma unroll
        for (int f = 0; f < NF; ++f) {
          gstore<T, VX>(phi_out + f * S + o, phs[f]);
          if (MODE == MODE_SWEEP) gstore<T, VX>(pi_out + f * S + o, pin[f]);
        }
        if constexpr (PREC == PREC_DD) {
          if (++kg == KGROUP) {
            kg = 0;
#pragma unroll
            for (int i2 = 0; i2 < NQ; ++i2) {
              dd t = tot[i2 * kPThreads];
              acc[i2].fold(t);
              tot[i2 * kPThreads] = t;
            }
          }
        }
      }
#pragma unroll
      for (int f = 0; f < NF; ++f)
#pragma unroll
        for (int jj = 0; jj < VX; ++jj) {
          c2[f][jj] = c1[f][jj];
          c1[f][jj] = cur[f][jj];
          q2[f][jj] = q1[f][jj];
          q1[f][jj] = qn[f][jj];
        }
    }
  }
  if constexpr (PREC == PREC_DD) {
#pragma unroll
    for (int i2 = 0; i2 < NQ; ++i2) {
      dd t = tot[i2 * kPThreads];
      acc[i2].fold(t);
      tot[i2 * kPThreads] = t;
    }
  }
  return ok;
}

// ---------------------------------------------------------------------------
// Split-FP32 form.
// ---------------------------------------------------------------------------
// Producer of ring plane gp (one warp): waits until every warp has released
// the slot's previous plane, then lane 0 issues the copies.  Kept out of line
// (it runs once per plane in one warp); its shared-memory pointers come by
// value, so the caller's PShared stays in registers, not on the stack.
template <int NF, int VX, bool CORNERS, int NSLOT>
__device__ __noinline__ bool produce_split(const PParams& p, unsigned char* ring, uint64_t* full,
                                           uint64_t* empty, uint32_t* issued, long long limit,
                                           int ib, uint32_t gp, int4 u, int q) {
  using LY = PLayout<NF, VX, 4>;
  bool ok = true;
  if (gp >= (uint32_t)NSLOT) {
    const uint32_t rr = gp - NSLOT;
    ok = mbar_wait(&empty[rr % NSLOT], (rr / NSLOT) & 1, limit);
  }
  if (!__all_sync(0xffffffffu, ok)) return false;
  if ((threadIdx.x & 31) == 0) {
    pproduce<NF, VX, 4, CORNERS>(p, ib, u, q, ring + (size_t)(gp % NSLOT) * LY::SLOT_BYTES,
                                 &full[gp % NSLOT]);
    issued[gp % NSLOT] = gp + 1;
  }
  return true;
}

// Add the float partials of each group of four lanes into the group's
// compensated sums (shared memory, one (s, c) pair per group and quantity):
// the four lanes' partials are summed first by a butterfly (the same sum in
// every lane of the group, whatever the order of the adds).  Every lane of
// the warp calls it.
template <int NQ>
__device__ __forceinline__ void kahan_flush(float2* kahan, float (&ps)[NQ]) {
  const int grp = threadIdx.x >> 2;
  const bool lead = (threadIdx.x & 3) == 0;
#pragma unroll
  for (int i = 0; i < NQ; ++i) {
    float x = ps[i];
    x += __shfl_xor_sync(0xffffffffu, x, 1);
    x += __shfl_xor_sync(0xffffffffu, x, 2);
    if (lead) {
      float2 v = kahan[i * kKahanGroups + grp];
      const float y = x - v.y;
      const float t = v.x + y;
      v.y = (t - v.x) - y;
      v.x = t;
      kahan[i * kKahanGroups + grp] = v;
    }
    ps[i] = 0.f;
  }
}

// One stage of the split-FP32 form: barrier-free warp pipeline.  Ring plane
// gq + j is produced by warp (gq + j) mod 16; every warp drifts the three rows
// it needs in registers and releases the slot.  Returns false
// (warp-uniformly) if a wait gave up.
template <int MODEL, int STENCIL, int VX, int MODE, bool GENERAL = false>
__device__ __forceinline__ bool stage_split(const PParams& p, const Ctx<MODEL, PREC_SPLIT>& cx,
                                            const PShared& sm, uint32_t gq, int ib) {
  using C = Ctx<MODEL, PREC_SPLIT>;
  using SL = typename C::SL;
  constexpr int NF = C::NF;
  constexpr int NQ = SL::NQ;
  constexpr bool CORNERS = StencilW<STENCIL>::kCorners;
  constexpr int CR = CORNERS ? 3 : 1;
  using LY = PLayout<NF, VX, 4>;
  using RG = PRing<PREC_SPLIT, NF, VX, NQ>;
  constexpr int TX = LY::TX, CW = LY::CW;
  constexpr int NSLOT = RG::NSLOT, LEAD = RG::LEAD;
  constexpr int KGROUP = 8;   // output planes per float partial before a compensated add
  const SimDesc& d = *sm.d;
  const int tid = threadIdx.x, lane = tid & 31, ly = tid >> 5;
  const int n = p.g.n;
  const size_t S = (size_t)d.S, nn = (size_t)n * n;
  float* __restrict__ phi_out = (float*)d.phi[(ib & 1) ^ 1];
  float* __restrict__ pi_out = (float*)d.pi[((ib >> 1) & 1) ^ 1];
  const float cd = cx.cdrift;
  // re-centring: phi* = phi + c pi - (mu_phi + c mu_pi); the stencil works on
  // phi + c pi (D of a constant is zero)
  float Mf[NF];
#pragma unroll
  for (int f = 0; f < NF; ++f) Mf[f] = madd(cd, cx.mu_pi[f], cx.mu_phi[f]);
  const int side = lane == 31 ? 1 : 0;
  const int own = (ly + 1) * TX + lane * VX;

#pragma unroll
  for (int i = 0; i < NQ; ++i)   // each group's lead lane owns its sums
    if ((tid & 3) == 0) sm.kahan[i * kKahanGroups + (tid >> 2)] = make_float2(0.f, 0.f);
  float ps[NQ];
#pragma unroll
  for (int i = 0; i < NQ; ++i) ps[i] = 0.f;
  int kg = 0;

  // producer position, LEAD planes ahead (pQ: planes of its unit, 0 past the last)
  int pui = 0, puq = 0;
  for (int l = 0; l < LEAD; ++l) padvance(sm, pui, puq);
  int pQ = pui < sm.nunits ? sm.units[pui].w : 0;
  bool ok = true;
  uint32_t g = gq;
  // ring slot of plane g and the parity of its pass over the ring, kept
  // incrementally (NSLOT need not be a power of two)
  int s = (int)(gq % NSLOT);
  uint32_t par = (gq / NSLOT) & 1u;
  for (int i = 0; i < sm.nunits; ++i) {
    const int4 u = sm.units[i];
    const int Q = u.w;
    const bool clear = yclear(u, n);
    const size_t o0 = (size_t)u.z * nn + (size_t)(u.y + ly) * n + u.x + lane * VX;
    // this lane's halo-column rows in a slot (the layout differs at the y wrap)
    int crow[NF][CR];
#pragma unroll
    for (int f = 0; f < NF; ++f)
#pragma unroll
      for (int rr = 0; rr < CR; ++rr) {
        const int r = ly + 1 + rr - (CR - 1) / 2;
        crow[f][rr] = clear ? LY::col_dense(f, r) : LY::col_wrap(f, r);
      }
    float part_m[NF][VX], so_m[NF][VX], ph_m[NF][VX], pi_m[NF][VX];
#pragma unroll
    for (int f = 0; f < NF; ++f)
#pragma unroll
      for (int jj = 0; jj < VX; ++jj) part_m[f][jj] = so_m[f][jj] = ph_m[f][jj] = pi_m[f][jj] = 0.f;
    // two planes per trip lets the compiler rename the rotated registers
    // (the 27-point stencil keeps one: it would spill)
    constexpr int kUnroll = CORNERS ? 1 : 2;
#pragma unroll kUnroll
    for (int q = 0; q < Q; ++q, ++g) {
      if (pQ > 0) {
        const uint32_t gp = g + LEAD;
        if ((int)(gp % kPWarps) == ly)
          ok = produce_split<NF, VX, CORNERS, NSLOT>(p, sm.ring, sm.full, sm.empty, sm.issued,
                                                     sm.limit, ib, gp, sm.units[pui], puq) &&
               ok;
        if (++puq == pQ) {
          ++pui;
          puq = 0;
          pQ = pui < sm.nunits ? sm.units[pui].w : 0;
        }
      }
      ok = ok && mbar_wait(&sm.full[s], par, sm.limit);
      if (!__all_sync(0xffffffffu, ok)) return false;
      const float* sl = (const float*)(sm.ring + (size_t)s * LY::SLOT_BYTES);
      // the three rows this warp needs and the halo-column values, drifted in registers
      float cur_ph[NF][VX], cur_pi[NF][VX], dn[NF][VX], up[NF][VX], el[NF][CR];
#pragma unroll
      for (int f = 0; f < NF; ++f) {
        const float* mph = sl + LY::main_off(0, f);
        const float* mpi = sl + LY::main_off(1, f);
        float a[VX], b[VX];
        vload<float, VX>(&mph[own], a);
        vload<float, VX>(&mpi[own], b);
#pragma unroll
        for (int jj = 0; jj < VX; ++jj) {
          cur_pi[f][jj] = b[jj] - cx.mu_pi[f];
          cur_ph[f][jj] = madd(cd, b[jj], a[jj]);
        }
        vload<float, VX>(&mph[own - TX], a);
        vload<float, VX>(&mpi[own - TX], b);
#pragma unroll
        for (int jj = 0; jj < VX; ++jj) dn[f][jj] = madd(cd, b[jj], a[jj]);
        vload<float, VX>(&mph[own + TX], a);
        vload<float, VX>(&mpi[own + TX], b);
#pragma unroll
        for (int jj = 0; jj < VX; ++jj) up[f][jj] = madd(cd, b[jj], a[jj]);
        const float* cph = sl + LY::col_base(0, side) + (side ? 0 : CW - 1);
        const float* cpi = sl + LY::col_base(1, side) + (side ? 0 : CW - 1);
#pragma unroll
        for (int rr = 0; rr < CR; ++rr) el[f][rr] = madd(cd, cpi[crow[f][rr]], cph[crow[f][rr]]);
      }
      fence_proxy_async();   // generic reads of the slot before the TMA copy that refills it
      __syncwarp();
      if (lane == 0) mbar_arrive(&sm.empty[s]);   // this warp is done with the slot
      if (++s == NSLOT) { s = 0; par ^= 1u; }

      const bool mid = q > 0 && q < Q - 1;   // the z-halo planes need S_off only
      float so_new[NF][VX], smid_new[NF][VX];
#pragma unroll
      for (int f = 0; f < NF; ++f) {
        if (mid)
          lane_parts<float, VX, CORNERS, true, CR>(cur_ph[f], dn[f], up[f], el[f], smid_new[f],
                                                   so_new[f]);
        else
          lane_parts<float, VX, CORNERS, false, CR>(cur_ph[f], dn[f], up[f], el[f], smid_new[f],
                                                    so_new[f]);
      }
      if (q >= 2) {  // output plane z0 + q - 2
        const size_t o = o0 + (size_t)(q - 2) * nn;
        float pin[NF][VX], phs[NF][VX];
#pragma unroll
        for (int jj = 0; jj < VX; ++jj) {
          float phj[NF], Dj[NF], pmj[NF], pnj[NF];
#pragma unroll
          for (int f = 0; f < NF; ++f) {
            phs[f][jj] = ph_m[f][jj] - Mf[f];   // the re-centred drifted field
            phj[f] = phs[f][jj];
            Dj[f] = part_m[f][jj] + so_new[f][jj];
            pmj[f] = pi_m[f][jj];
          }
          cx.template site<GENERAL>(MODE, phj, Dj, pmj, pnj, ps);
#pragma unroll
          for (int f = 0; f < NF; ++f) pin[f][jj] = pnj[f];
        }
#pragma unroll
        for (int f = 0; f < NF; ++f) {
          gstore<float, VX>(phi_out + f * S + o, phs[f]);
          if (MODE == MODE_SWEEP) gstore<float, VX>(pi_out + f * S + o, pin[f]);
        }
        if (++kg == KGROUP) {
          kg = 0;
          kahan_flush<NQ>(sm.kahan, ps);
        }
      }
      if (mid) {
#pragma unroll
        for (int f = 0; f < NF; ++f)
#pragma unroll
          for (int jj = 0; jj < VX; ++jj)
            part_m[f][jj] = (CORNERS ? so_m[f][jj] : ph_m[f][jj]) + smid_new[f][jj];
      }
#pragma unroll
      for (int f = 0; f < NF; ++f)
#pragma unroll
        for (int jj = 0; jj < VX; ++jj) {
          if constexpr (CORNERS) so_m[f][jj] = so_new[f][jj];
          ph_m[f][jj] = cur_ph[f][jj];
          pi_m[f][jj] = cur_pi[f][jj];
        }
    }
  }
  kahan_flush<NQ>(sm.kahan, ps);
  return true;
}

// Plane l (< LEAD) of a stage, issued by lane 0 of the calling warp.  Used at
// stage starts, the first LEAD planes spread over a few warps.  Every plane of the previous stage has
// been consumed and released before the block barrier that precedes this
// call, so the slot needs no wait (the "empty" phases still complete as usual).
template <int PREC, int NF, int VX, bool CORNERS, int NSLOT, int H = 1>
__device__ __forceinline__ void prefetch_plane(const PParams& p, const PShared& sm, int ib,
                                               uint32_t gq, int l) {
  constexpr int WORD = prec_word(PREC);
  using LY = PLayout<NF, VX, WORD, H>;
  int ui = 0, uq = 0;
  for (int j = 0; j < l; ++j) padvance(sm, ui, uq);
  if (ui >= sm.nunits || (threadIdx.x & 31) != 0) return;
  const uint32_t gp = gq + l;
  pproduce<NF, VX, WORD, CORNERS, H>(p, ib, sm.units[ui], uq,
                                     sm.ring + (size_t)(gp % NSLOT) * LY::SLOT_BYTES,
                                     &sm.full[gp % NSLOT]);
  sm.issued[gp % NSLOT] = gp + 1;
}

// Untiled bulk copy global -> shared (16-byte aligned, size a multiple of 16),
// completing on `bar` (transaction count).
__device__ __forceinline__ void bulk_load(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
      ::"r"(smem_u32(dst)), "l"(reinterpret_cast<uint64_t>(src)), "r"(bytes), "r"(smem_u32(bar))
      : "memory");
}

__device__ __forceinline__ void named_sync(int id, int count) {
  asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(count) : "memory");
}
__device__ __forceinline__ void named_arrive(int id, int count) {
  asm volatile("bar.arrive %0, %1;" ::"r"(id), "r"(count) : "memory");
}

// ---------------------------------------------------------------------------
// The kernel.
// ---------------------------------------------------------------------------
template <int MODEL, int STENCIL, int PREC, int VX>
__global__ void __launch_bounds__(kPThreads, 1) evolve_persist(const __grid_constant__ PParams p) {
  using C = Ctx<MODEL, PREC>;
  using SL = typename C::SL;
  constexpr int NQ = SL::NQ;
  constexpr int NF = C::NF;
  constexpr bool CORNERS = StencilW<STENCIL>::kCorners;
  constexpr int H = halo_of<STENCIL>();
  static_assert(STENCIL != 13 || PREC != PREC_SPLIT, "the 13-point stencil: FP64 and split-DD");
  using RG = PRing<PREC, NF, VX, NQ, H>;
  constexpr int NSLOT = RG::NSLOT, LEAD = RG::LEAD, PRE = RG::PRE;
  static_assert(NQ <= kPWarps, "one warp per reduced quantity");
  static_assert(PREC == PREC_SPLIT || (size_t)kMaxPBlocks * kNQ * 8 <= (size_t)NQ * kPThreads * 8,
                "the rows of every block fit the reduction scratch");

  extern __shared__ __align__(128) unsigned char dsm[];
  __shared__ __align__(8) uint64_t full[NSLOT], empty[NSLOT], foldbar, dbar[RG::NDRIFT];
  // background and stage coefficients, double-buffered: at a stage boundary
  // one thread derives the next coefficients while another does the rest of
  // the background bookkeeping
  __shared__ __align__(16) Background sbv[2];
  __shared__ C sctxv[2];
  // formed during the fold: the sums-to-kick coefficients of this stage and
  // the sums-independent half of the next stage's scalar half-steps
  __shared__ SumCoef<NF> s_sc;
  __shared__ PreCoef s_qn;
  __shared__ double s_p0[2 * NF];   // split form: the next stage's re-centred background
  // the scalar chain between stages reads the descriptor many times; the
  // ring leaves little L1, so it is kept in shared memory
  __shared__ __align__(64) SimDesc s_desc;
  __shared__ double sums[kNQ];
  __shared__ int4 s_units[kMaxPUnits];
  __shared__ uint32_t s_issued[NSLOT];
  __shared__ int s_bad;
  __shared__ int s_fold;   // parity of a rows copy issued and not yet folded; -1: none

  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const SimDesc& d = s_desc;
  const int G = p.g.G;
  static_assert(sizeof(SimDesc) % 8 == 0, "descriptor copied as 8-byte words");
  for (int i = tid; i < (int)(sizeof(SimDesc) / 8); i += kPThreads)
    reinterpret_cast<unsigned long long*>(&s_desc)[i] =
        __ldg(reinterpret_cast<const unsigned long long*>(p.d) + i);
  PShared sm;
  sm.d = &s_desc;
  sm.ring = dsm;
  sm.kahan = reinterpret_cast<float2*>(dsm + RG::RING_BYTES);
  sm.drift = reinterpret_cast<double*>(dsm + RG::RING_BYTES);
  sm.red = reinterpret_cast<double*>(dsm + RG::RING_BYTES) + RG::DRIFT_WORDS;
  sm.full = full;
  sm.empty = empty;
  sm.dbar = dbar;
  sm.units = s_units;
  sm.issued = s_issued;
  sm.limit = p.wait_limit;
  const int ubeg = __ldg(&p.uoff[blockIdx.x]);
  sm.nunits = min(__ldg(&p.uoff[blockIdx.x + 1]) - ubeg, kMaxPUnits);   // host: <= kMaxPUnits

  if (tid == 0) {
    for (int s = 0; s < NSLOT; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], kPWarps);
    }
    mbar_init(&foldbar, 1);
    for (int b = 0; b < RG::NDRIFT; ++b) mbar_init(&dbar[b], kPWarps);
    fence_mbar_init();
    s_bad = 0;
    s_fold = -1;
  }
  if (tid < NSLOT) s_issued[tid] = 0;
  if (tid < 6) {   // bring the tensor maps into the descriptor cache
    const CUtensorMap* m = &p.tm[tid];
    asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(m)) : "memory");
  }
  if (tid < sm.nunits) s_units[tid] = p.units[ubeg + tid];   // this block's units, in order
  static_assert(sizeof(Background) % 8 == 0, "background copied as 8-byte words");
  if (tid < (int)(sizeof(Background) / 8))
    reinterpret_cast<unsigned long long*>(&sbv[0])[tid] =
        __ldcg(reinterpret_cast<const unsigned long long*>(p.bg) + tid);
  __syncthreads();
  if (sbv[0].error) return;   // a stopped simulation stays stopped (same in every block)
  if (tid == 0) {
    sbv[0].sweeps_left = p.nsweeps;
    sbv[0].mode = p.nsweeps > 0 ? MODE_SWEEP : MODE_FLUSH;
  }
  int cb = 0;   // current buffer of sbv / sctxv
  uint32_t np = 0;
  for (int i = 0; i < sm.nunits; ++i) np += (uint32_t)s_units[i].w;
  uint32_t gq = 0;
  const long long K = p.nsweeps;
  // the launch's last pass: the flush (k == K), or, for a launch that leaves
  // the merged stage boundary pending for the next launch (p.flush == 0), the
  // last stage sweep; the Background written back is then a sweep's, as after
  // a per-stage launch
  const long long KL = p.flush ? K : K - 1;
  bool fault = false;
  int ib = sbv[0].cur;
  // stage 0: its first planes are in flight while one thread derives the
  // scalar coefficients (the FP64 chain of the merged half-stages)
  {
    for (int l = kPWarps - 1 - warp; l < LEAD; l += kPWarps)   // warp 15 - l issues plane l
      prefetch_plane<PREC, NF, VX, CORNERS, NSLOT, H>(p, sm, ib, gq, l);
    if (tid == 0) sctxv[0].init(sbv[0], d, K > 0 ? MODE_SWEEP : MODE_FLUSH);
    __syncthreads();
    fault = s_bad != 0;
  }
  for (long long k = 0; k <= KL && !fault; ++k) {
    const int mode = (k < K) ? MODE_SWEEP : MODE_FLUSH;
    const C cx = sctxv[cb];
    // @stage-start

    // ---- the sweep (per-thread sums) ----
    bool ok = true;
    double accd[NQ];
#pragma unroll
    for (int q = 0; q < NQ; ++q) accd[q] = 0.0;
    if constexpr (STENCIL == 13) {
      ok = (mode == MODE_SWEEP) ? stage_wide<MODEL, VX, MODE_SWEEP, PREC>(p, cx, sm, gq, ib, accd)
                                : stage_wide<MODEL, VX, MODE_FLUSH, PREC>(p, cx, sm, gq, ib, accd);
      if constexpr (PREC == PREC_DD) {
        const dd* tot = reinterpret_cast<const dd*>(sm.red) + tid;
#pragma unroll
        for (int q = 0; q < NQ; ++q) accd[q] = (double)tot[q * kPThreads];
      }
    } else if constexpr (PREC == PREC_FP64) {
      ok = (mode == MODE_SWEEP)
               ? stage_fp64<MODEL, STENCIL, VX, MODE_SWEEP>(p, cx, sm, gq, ib, accd)
               : stage_fp64<MODEL, STENCIL, VX, MODE_FLUSH>(p, cx, sm, gq, ib, accd);
    } else if constexpr (PREC == PREC_DD) {
      ok = (mode == MODE_SWEEP) ? stage_dd<MODEL, STENCIL, VX, MODE_SWEEP>(p, cx, sm, gq, ib)
                                : stage_dd<MODEL, STENCIL, VX, MODE_FLUSH>(p, cx, sm, gq, ib);
      // this thread's stage sums, from its own scratch slots (overwritten below)
      const dd* tot = reinterpret_cast<const dd*>(sm.red) + tid;
#pragma unroll
      for (int q = 0; q < NQ; ++q) accd[q] = (double)tot[q * kPThreads];
    } else {
      // the Q-ball's difference forms have a branch for a background at the
      // origin; a stage whose background is away from it runs without the test
      // (7-point stencil: the 27-point one would spill with both instances)
      if constexpr (MODEL == M_QBALL && !CORNERS) {
        if (!cx.sk.direct)
          ok = (mode == MODE_SWEEP)
                   ? stage_split<MODEL, STENCIL, VX, MODE_SWEEP, true>(p, cx, sm, gq, ib)
                   : stage_split<MODEL, STENCIL, VX, MODE_FLUSH, true>(p, cx, sm, gq, ib);
        else
          ok = (mode == MODE_SWEEP) ? stage_split<MODEL, STENCIL, VX, MODE_SWEEP>(p, cx, sm, gq, ib)
                                    : stage_split<MODEL, STENCIL, VX, MODE_FLUSH>(p, cx, sm, gq, ib);
      } else {
        ok = (mode == MODE_SWEEP) ? stage_split<MODEL, STENCIL, VX, MODE_SWEEP>(p, cx, sm, gq, ib)
                                  : stage_split<MODEL, STENCIL, VX, MODE_FLUSH>(p, cx, sm, gq, ib);
      }
    }
    if (!ok) atomicOr(&s_bad, 1);
    gq += np;
    // global stores of this stage will be read by TMA (async proxy) next stage
    fence_proxy_async_global();
    __syncthreads();
    // @units-done
    if (s_bad) { fault = true; break; }

    // ---- block sums: one warp per quantity over the 512 threads' values, fixed order ----
    if constexpr (PREC != PREC_SPLIT) {
      double* red = sm.red;
#pragma unroll
      for (int q = 0; q < NQ; ++q) red[q * kPThreads + tid] = accd[q];
      __syncthreads();
      if (warp < NQ) {
        // 16 values per lane summed as a pairwise tree (depth 4: FP64 latency is long)
        double x[kPThreads / 32];
#pragma unroll
        for (int r = 0; r < kPThreads / 32; ++r) x[r] = red[warp * kPThreads + lane + 32 * r];
#pragma unroll
        for (int w = kPThreads / 64; w >= 1; w >>= 1)
#pragma unroll
          for (int r = 0; r < w; ++r) x[r] = x[2 * r] + x[2 * r + 1];
        double v = x[0];
#pragma unroll
        for (int h = 16; h >= 1; h >>= 1) v += __shfl_down_sync(0xffffffffu, v, h);
        if (lane == 0) {
          reinterpret_cast<double*>(p.rows)[((size_t)(k & 1) * G + blockIdx.x) * kNQ + warp] = v;
          fence_proxy_async_global();   // the rows are read back by bulk copies
        }
      }
    } else {
      if (warp < NQ) {
        float hi = 0.f, lo = 0.f;
#pragma unroll
        for (int r = 0; r < kKahanGroups / 32; ++r) {
          const float2 v = sm.kahan[warp * kKahanGroups + lane + 32 * r];
          pair_add(hi, lo, v.x, -v.y);
        }
#pragma unroll
        for (int h = 16; h >= 1; h >>= 1) {
          const float bh = __shfl_down_sync(0xffffffffu, hi, h);
          const float bl = __shfl_down_sync(0xffffffffu, lo, h);
          pair_add(hi, lo, bh, bl);
        }
        if (lane == 0) {
          reinterpret_cast<float2*>(p.rows)[((size_t)(k & 1) * G + blockIdx.x) * kNQ + warp] =
              make_float2(hi, lo);
          fence_proxy_async_global();   // the rows are read back by bulk copies
        }
      }
    }
    // the reduction scratch is overwritten by the rows' bulk copy below
    fence_proxy_async();
    if (!grid_barrier(p.bar, p.bar_base + (unsigned long long)(k + 1) * G + p.bar_extra,
                      p.wait_limit))
      s_bad = 1;
    // while thread 0 waits for the other blocks, warp 14 forms what the scalar
    // chain needs that does not depend on the sums: this stage's SumCoef and
    // the next stage's PreCoef (it starts from a = k.a, h_prev = k.h)
    if (warp == kPWarps - 2 && lane == 0) {
      s_sc = sum_coef<MODEL, PREC>(sctxv[cb], d);
      if (k < KL) {
        const int mn = k + 1 < K ? MODE_SWEEP : MODE_FLUSH;
        const int sn = sbv[cb].stage + 1 < d.nstages ? sbv[cb].stage + 1 : 0;
        const Coef& kc = sctxv[cb].k;
        const double hn = stage_step(d, sn, kc.deta, mn);
        s_qn = prestage_a(kc.a, __drcp_rn(kc.a), kc.h, hn, d, mn, d.physical ? kc.deta : d.dt,
                          d.physical && sn == 0, d.w[sn]);
      }
    }
    __syncthreads();
    // @released
    if (s_bad) { fault = true; break; }

    // ---- after the barrier, on disjoint warps:
    //   warps 0..NQ-1 fold every block's row (in block order, identically in
    //     every block); the next stage's copies wait until these latency-
    //     critical loads have landed (named barrier 1), so that they are not
    //     queued behind the copies;
    //   warps 15, 14, ... (PRE of them) issue the next stage's first LEAD
    //     planes, every PRE-th plane each (its buffers are known: a sweep
    //     swaps phi and pi, a flush swaps phi) ----
    const int ib_next = ib ^ (mode == MODE_SWEEP ? 3 : 1);
    const bool pre = k < KL;
    constexpr int kPreThreads = (1 + PRE) * 32;
    using FT = typename std::conditional<PREC != PREC_SPLIT, double, float2>::type;
    // every block's row arrives by one bulk copy into the (now free) reduction
    // scratch: one request stream per block instead of 8-byte loads of the
    // same lines by every block
    FT* srows = reinterpret_cast<FT*>(PREC != PREC_SPLIT ? (void*)sm.red : (void*)sm.kahan);
    if (warp == 0) {
      if (lane == 0) {
        const uint32_t bytes = (uint32_t)(G * kNQ * sizeof(FT));
        mbar_expect_tx(&foldbar, bytes);
        bulk_load(srows, reinterpret_cast<const FT*>(p.rows) + (size_t)(k & 1) * G * kNQ, bytes,
                  &foldbar);
        s_fold = (int)(k & 1);
      }
      __syncwarp();
      if (pre) named_arrive(1, kPreThreads);   // the next stage's copies queue behind it
    }
    if (warp < NQ) {
      if (!mbar_wait(&foldbar, (uint32_t)(k & 1), p.wait_limit)) atomicOr(&s_bad, 1);
      if constexpr (PREC != PREC_SPLIT) {
        double v = 0.0;
        for (int r = lane; r < G; r += 32) v += srows[(size_t)r * kNQ + warp];   // row order
#pragma unroll
        for (int h = 16; h >= 1; h >>= 1) v += __shfl_down_sync(0xffffffffu, v, h);
        if (lane == 0) sums[warp] = v;
      } else {
        float hi = 0.f, lo = 0.f;
        for (int r = lane; r < G; r += 32) {
          const float2 x = srows[(size_t)r * kNQ + warp];
          pair_add(hi, lo, x.x, x.y);
        }
#pragma unroll
        for (int h = 16; h >= 1; h >>= 1) {
          const float bh = __shfl_down_sync(0xffffffffu, hi, h);
          const float bl = __shfl_down_sync(0xffffffffu, lo, h);
          pair_add(hi, lo, bh, bl);
        }
        if (lane == 0) sums[warp] = (double)hi + (double)lo;
      }
      // @sums-written
    } else {
      const int l0 = kPWarps - 1 - warp;
      if (pre && l0 < PRE) {
        named_sync(1, kPreThreads);
        for (int l = l0; l < LEAD; l += PRE)
          prefetch_plane<PREC, NF, VX, CORNERS, NSLOT, H>(p, sm, ib_next, gq, l);
      }
      // @prefetch-issued
    }
    __syncthreads();
    // @folded
    if (tid == 0 && !s_bad) s_fold = -1;   // every folding warp saw the copy land
    // ---- in parallel, on warps of different schedulers, identically in
    //      every block: the next stage's coefficients (warp 14: sums -> p_a
    //      kick -> scalar half-steps -> split background), the split form's
    //      re-centring (warp 12, joined to warp 14 by named barrier 2) and the
    //      bookkeeping of this stage (warp 13) ----
    // (the current Ctx is read from shared memory here, not from the sweep's
    // register copy, so that the copy's live range ends with the sweep)
    const C& cc = sctxv[cb];
    if (warp == kPWarps - 2) {
      if (pre) {
        const int mn = k + 1 < K ? MODE_SWEEP : MODE_FLUSH;
        C& nx = sctxv[cb ^ 1];
        if (lane == 0) {
          nx.set_coef(chain_coef<MODEL, PREC>(cc, s_sc, s_qn, d, sums, mn), d, mn, cc.pk);
          if constexpr (PREC == PREC_FP64) {   // the next stage's input is this stage's output
#pragma unroll
            for (int f = 0; f < NF; ++f)
              nx.shiftK[f] = (mn == MODE_FLUSH) ? flush_shift(d, ib_next, f, nx.k.c) : 0.0;
            nx.set_qref(d, ib_next);
          }
        }
        if constexpr (PREC != PREC_FP64) {
          __syncwarp();
          named_sync(2, 64);
          if (lane == 0) nx.split_tail(d, mn, s_p0);
        }
      }
      // @chain-done
    } else if (warp == kPWarps - 4) {
      if constexpr (PREC != PREC_FP64) {
        if (pre) {
          if (lane == 0) {
            double mphi[NF], mpi[NF];
            chain_means<PREC>(cc, d, sums, mphi, mpi);
            sctxv[cb ^ 1].recenter(mphi, mpi, cc.phi0s, cc.pi0s, s_p0);
          }
          __syncwarp();
          named_arrive(2, 64);
        }
      }
    } else if (tid == kPThreads - 96) {
      post_stage<MODEL, PREC>(cc, s_sc, d, mode, sums, sbv[cb], sbv[cb ^ 1]);
      // @book-done
    }
    __syncthreads();
    // @coefficients
    cb ^= 1;
    if (s_bad) { fault = true; break; }
    if (sbv[cb].error) break;   // identical sums in every block: every block stops here
    ib = ib_next;
  }

  // copies issued for a stage that will not run (a stop after a non-finite
  // sum, or a fault) must land before the block exits (bounded waits)
  __syncthreads();
  if (tid == 0) {
    if (fault) atomicOr(p.fault, 1);
    for (int s = 0; s < NSLOT; ++s)
      if (s_issued[s]) mbar_wait(&full[s], ((s_issued[s] - 1u) / NSLOT) & 1u);
    if (s_fold >= 0) mbar_wait(&foldbar, (uint32_t)s_fold);   // a rows copy still in flight
  }
  if (fault) return;   // the state is not trusted any more (the host poisons the simulation)
  if (blockIdx.x == 0 && tid < (int)(sizeof(Background) / 8))
    reinterpret_cast<unsigned long long*>(p.bg)[tid] =
        reinterpret_cast<const unsigned long long*>(&sbv[cb])[tid];
}

// Launch helper (one translation unit per precision and stencil set: WIDE =
// the 13-point stencil).  grid == 0: only set
// the kernel's shared-memory attribute and report its occupancy in *bps.
template <int PREC, bool WIDE = false>
cudaError_t launch_persist_impl(int model, int stencil, int vx, const PParams& p, int grid,
                                cudaStream_t s, int* bps) {
#define PYCOOL_P(M, ST, V)                                                                  \
  if constexpr (V * Pot<M>::NF * prec_word(PREC) <= 16) {                                  \
    if (model == M && stencil == ST && vx == V) {                                           \
      constexpr size_t smem = persist_smem_bytes<M, PREC, V, ST>();                         \
      auto kern = evolve_persist<M, ST, PREC, V>;                                           \
      if (grid == 0) {                                                                      \
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, \
                                             (int)smem);                                    \
        if (e != cudaSuccess) return e;                                                     \
        return cudaOccupancyMaxActiveBlocksPerMultiprocessor(bps, kern, kPThreads, smem);   \
      }                                                                                     \
      cudaLaunchConfig_t cfg = {};                                                          \
      cfg.gridDim = dim3(grid);                                                             \
      cfg.blockDim = dim3(kPThreads);                                                       \
      cfg.dynamicSmemBytes = smem;                                                          \
      cfg.stream = s;                                                                       \
      cudaLaunchAttribute attr[1];                                                          \
      attr[0].id = cudaLaunchAttributeCooperative;                                          \
      attr[0].val.cooperative = 1;                                                          \
      cfg.attrs = attr;                                                                     \
      cfg.numAttrs = 1;                                                                     \
      return cudaLaunchKernelEx(&cfg, kern, p);                                             \
    }                                                                                       \
  }
#define PYCOOL_PM(X, V)                                                                     \
  X(M_FREE, 7, V) X(M_FREE, 27, V) X(M_CHAOTIC2, 7, V) X(M_CHAOTIC2, 27, V)                 \
  X(M_OSCILLON, 7, V) X(M_OSCILLON, 27, V) X(M_QBALL, 7, V) X(M_QBALL, 27, V)
#define PYCOOL_PW(X, V) X(M_FREE, 13, V) X(M_CHAOTIC2, 13, V) X(M_OSCILLON, 13, V) X(M_QBALL, 13, V)
  if constexpr (WIDE) {
    static_assert(PREC != PREC_SPLIT, "the 13-point stencil: FP64 and split-DD");
    PYCOOL_PW(PYCOOL_P, 1)
    PYCOOL_PW(PYCOOL_P, 2)
  } else {
    PYCOOL_PM(PYCOOL_P, 1)
    PYCOOL_PM(PYCOOL_P, 2)
    if constexpr (PREC == PREC_SPLIT) { PYCOOL_PM(PYCOOL_P, 4) }
  }
#undef PYCOOL_PW
#undef PYCOOL_PM
#undef PYCOOL_P
  return cudaErrorInvalidValue;
}

}  // namespace pycool
