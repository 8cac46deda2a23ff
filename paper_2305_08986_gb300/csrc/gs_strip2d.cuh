// 2D velocity-block kernel (y = A x, y = b - A x, and the fused Chebyshev step) on Cartesian Q2
// quadrilaterals: the operator of Eq. "form_a_j" (symmetric part, 2 eta eps, alpha mass) that the
// multigrid smoother of Sec. 4 applies on every level.
//
// Work decomposition.  A CTA (8 warps) owns a column strip of 31 cells and a segment of R = 8 nb - 1
// cell rows.  Lane l of every warp evaluates cell column cs0 - 1 + l (lane 0: the column left of the
// strip, whose right-hand node column belongs to the strip); the CTA marches up the segment in nb
// batches of 8 cell rows, warp w taking row r0 - 1 + 8 k + w of batch k (batch 0, warp 0: the row
// below the segment).  Every cell of the mesh is evaluated by exactly one CTA apart from one halo
// column and one halo row per CTA (32 x 8 nb evaluated for 31 x (8 nb - 1) owned), and every node is
// written by exactly one thread.
//
// Memory pipeline.  For batch k the CTA needs a 65 x 17 node window of x (both components) and the
// epilogue operands (b; d, D^-1) of its owned nodes, a 64 x 17 window.  Every window row is one bulk
// copy (cp.async.bulk, the TMA engine) issued by one thread and completing on an mbarrier: a row
// starts at an arbitrary element (the node rows have an odd length), so the copy covers the 16-byte
// chunks around it and the row's alignment phase is recorded; the few rows at the two ends of a
// vector are copied element by element instead.  The x window of batch k + 1 is in flight while batch
// k's cells are evaluated (two buffers).  The operand rows are read only by the warp that owns their
// nodes, so each warp refetches its own rows for batch k + 1 right after its epilogue of batch k,
// completing on a per-warp mbarrier (one buffer, a full batch of lead).  The per-cell data (eta,
// alpha, constraint mask) of batch k + 1 is loaded into registers during batch k.
// Every mbarrier wait is bounded: a wait that gives up sets TileArgs::err and the launch completes.
//
// Sums.  A cell's 18 results (9 nodes x 2 components) are reduced without a shared-memory round
// trip per cell: the left node column of a cell receives the right column of the cell to its left
// by a warp shuffle, and the bottom node row receives the top row of the cells below and below-left
// through a 6-value exchange slot per lane (warp w -> w + 1 behind a named barrier of the two warps;
// warp 7 -> warp 0 of the next batch behind the batch's CTA barrier).  Every node sums its <= 4 cell contributions in the order
// (own + left) + below + below-left, the order of the cell-tile kernel (gs_tile2d.cuh), so the two
// kernels give the same bits and the choice between them never changes a result.
//
// Constraints.  Constrained columns enter as zero: a per-cell 9-bit mask of the cell's constrained
// local nodes (precomputed on meshes with obstacle cells, bit 15 marking an obstacle cell; from the
// Dirichlet faces otherwise) selects the staged values; constrained rows are identity rows.
#pragma once
#include <stdint.h>

#include "gs_cell.cuh"
#include "gs_kernels.h"

namespace gs {
namespace strip2d {

constexpr int NT = 256;            // threads per CTA
constexpr int NW = NT / 32;        // warps = cell rows per batch
constexpr int EC = 32;             // evaluated cell columns per strip
constexpr int OC = EC - 1;         // owned cell columns per strip
constexpr int XR = 2 * NW + 1;     // node rows of a batch window (17)
constexpr int XW = 2 * EC + 1;     // node columns of the x window (65)
constexpr int BW = 2 * OC + 2;     // node columns of the operand window (64)
constexpr int NX = 6;              // exchanged values per lane: top node row (3 nodes) x 2 components

template <typename T>
struct Dims {
  static constexpr int V = 16 / (int)sizeof(T);               // elements per 16-byte chunk
  static constexpr int XCH = (XW + 2 * (V - 1)) / V;           // chunks per x row (any phase)
  static constexpr int BCH = (BW + 2 * (V - 1)) / V;           // chunks per operand row
  static constexpr int XS = XCH * V;                           // shared row pitch, x window
  static constexpr int BS = BCH * V;                           // shared row pitch, operand window
};

template <int MODE>
struct ModeVecs {  // operand vectors staged for the epilogue
  static constexpr int N = MODE == TILE_CHEB ? 3 : (MODE == TILE_RESID ? 1 : 0);
};

__device__ __forceinline__ void cp_async16(void* smem, const void* gmem) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(s), "l"(gmem));
}
template <typename T>
__device__ __forceinline__ void cp_async_elem(T* smem, const T* gmem, bool load) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
  if (sizeof(T) == 4)
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;\n" ::"r"(s), "l"(gmem), "r"(load ? 4 : 0));
  else
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8, %2;\n" ::"r"(s), "l"(gmem), "r"(load ? 8 : 0));
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory"); }

// Alignment phase (in elements) of element e of vector v within its 16-byte chunk.
template <typename T>
__device__ __forceinline__ int phase_of(const T* v, long long e) {
  return (int)((reinterpret_cast<uintptr_t>(v + e) / sizeof(T)) & (Dims<T>::V - 1));
}

// Constrained local nodes of cell (c0, c1) from the Dirichlet faces (bit la + 3 lb).
__device__ __forceinline__ unsigned face_cell_mask(const Geom& g, int c0, int c1) {
  const unsigned f = g.faces;
  unsigned m = 0;
  if ((f & 1u) && c0 == 0) m |= 0x049u;
  if ((f & 2u) && c0 == g.n[0] - 1) m |= 0x124u;
  if ((f & 4u) && c1 == 0) m |= 0x007u;
  if ((f & 8u) && c1 == g.n[1] - 1) m |= 0x1C0u;
  return m;
}

template <typename T, int MODE>
struct Smem {
  using D = Dims<T>;
  static constexpr int NV = ModeVecs<MODE>::N;
  static constexpr int XROWS = 2 * XR;                   // x rows per batch (two components)
  static constexpr int BROWS = NV * 2 * XR;              // operand rows per batch
  static constexpr int WROWS = NV * 6;                   // operand rows a warp copies (and arrives for)
  static constexpr int X_ELEMS = 2 * XROWS * D::XS;      // two buffers
  static constexpr int B_ELEMS = BROWS * D::BS;          // one buffer, rows owned by warps
  static constexpr int E_ELEMS = 2 * NW * NX * 32;       // exchange slots: [batch parity][warp]
  static constexpr int PH_OFF = 8 * (2 + NW);            // phase tables after the mbarriers
  static constexpr int HEAD_BYTES = ((PH_OFF + 2 * XROWS + BROWS + 15) / 16) * 16;
  static constexpr size_t BYTES = HEAD_BYTES + sizeof(T) * (size_t)(X_ELEMS + B_ELEMS + E_ELEMS);
};

__device__ __forceinline__ unsigned smem_u32(const void* p) { return (unsigned)__cvta_generic_to_shared(p); }
__device__ __forceinline__ void mbar_init(uint64_t* bar, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_arrive_tx(uint64_t* bar, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(smem_u32(bar)), "r"(bytes)
               : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, unsigned parity) {
  unsigned ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
// Wait for the phase of `bar` with the given parity.  Gives up after about a second (the copies it
// waits for are in bounds and complete in microseconds), records the failure in *err and returns,
// so that a lost completion ends the launch with an error status instead of a hang.
__device__ __forceinline__ void mbar_wait(uint64_t* bar, unsigned parity, int* err) {
  if (mbar_try_wait(bar, parity)) return;
  const long long t0 = clock64();
  while (!mbar_try_wait(bar, parity)) {
    if (clock64() - t0 > (1LL << 31)) {
      if (err) atomicOr(err, 1);
      return;
    }
  }
}
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, unsigned bytes, uint64_t* bar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];\n" ::"r"(
                   smem_u32(dst)),
               "l"(src), "r"(bytes), "r"(smem_u32(bar))
               : "memory");
}
__device__ __forceinline__ void fence_proxy_async() { asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory"); }
// Named barrier id (1..15) shared by two warps: the producer warp arrives, the consumer warp waits.
__device__ __forceinline__ void named_arrive(int id) { asm volatile("bar.arrive %0, 64;\n" ::"r"(id) : "memory"); }
__device__ __forceinline__ void named_sync(int id) { asm volatile("bar.sync %0, 64;\n" ::"r"(id) : "memory"); }

// Copy one window row: the 16-byte chunks covering the row that starts at element e_lo of vector v
// land in the shared row srow (16-byte aligned), element e_lo at srow[phase].  One bulk copy
// completing on `bar` when the chunks lie inside the vector (valid elements [0, vlen)); at the two
// ends of the vector element-wise cp.async with zero fill instead, committed as one group (waited
// for with cp.async.wait_group by the copying thread before the next barrier).
// Arrives on `bar` once, with the bytes it expects.  Returns the phase.
template <typename T, int CH>
__device__ __forceinline__ int stage_row(T* srow, const T* v, long long vlen, long long e_lo, uint64_t* bar) {
  constexpr int V = Dims<T>::V;
  const int phase = phase_of(v, e_lo);
  const long long e = e_lo - phase;
  if (e >= 0 && e + CH * V <= vlen) {
    mbar_arrive_tx(bar, CH * 16);
    bulk_g2s(srow, v + e, CH * 16, bar);
  } else {
    mbar_arrive_tx(bar, 0);
    for (int i = 0; i < CH * V; ++i) {
      const bool ok = e + i >= 0 && e + i < vlen;
      cp_async_elem(srow + i, ok ? v + e + i : v, ok);
    }
    cp_async_commit();  // cp.async.wait_group covers committed groups only
  }
  return phase;
}

template <typename T, int MODE>
__device__ __forceinline__ void strip2d_body(const TileArgs<T>& A, int bid) {
  using D = Dims<T>;
  using SM = Smem<T, MODE>;
  constexpr int NV = SM::NV;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  uint64_t* xbar = reinterpret_cast<uint64_t*>(smem_raw);      // [2]: x window buffers
  uint64_t* obar = xbar + 2;                                    // [NW]: each warp's operand rows
  uint8_t* xph = smem_raw + SM::PH_OFF;                         // [buf][comp][row]
  uint8_t* bph = xph + 2 * SM::XROWS;                           // [vec][comp][row]
  T* sx = reinterpret_cast<T*>(smem_raw + SM::HEAD_BYTES);      // [buf][comp][row][XS]
  T* sb = sx + SM::X_ELEMS;                                     // [vec][comp][row][BS]
  T* sxch = sb + SM::B_ELEMS;                                   // [slot][value][lane]

  const Geom& g = A.g;
  const OpCoef<T>& c = A.c;
  const bool raw = A.raw != 0;
  const int nstrips = A.tiles[0];
  const int nb = A.tiles[2];
  const int R = NW * nb - 1;
  const int strip = bid % nstrips, seg = bid / nstrips;
  const int cs0 = strip * OC, r0 = seg * R;
  const int n0 = g.n[0], n1 = g.n[1];
  const int nv0 = g.nv[0], nv1 = g.nv[1];
  const int Nv = (int)g.Nv;        // the launcher checks 2 N_v < 2^31
  const long long vlen = 2LL * Nv;
  const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
  const int I0 = 2 * (cs0 - 1);   // first node column of the x window
  const int Ib = 2 * cs0;         // first node column of the operand window
  const int own_lo = 2 * r0, own_hi = 2 * (r0 + R);  // owned node rows [own_lo, own_hi) (+ 2 n1 at the top)
  // row-copy roles: threads [0, XROWS) copy x rows; lanes [0, WROWS) of warp w copy the operand
  // rows that only warp w reads (node rows 2 w and 2 w + 1 of the batch; warp NW - 1 also row 2 NW)
  const bool xrole = tid < SM::XROWS;
  const bool brole = NV > 0 && lane < SM::WROWS;

  if (tid == 0) {
    mbar_init(&xbar[0], SM::XROWS);
    mbar_init(&xbar[1], SM::XROWS);
    if (NV > 0)
      for (int i = 0; i < NW; ++i) mbar_init(&obar[i], SM::WROWS);
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
  }
  __syncthreads();

  auto stage_x = [&](int k) {  // x row of batch k for thread tid < XROWS: comp = tid / XR, row tid % XR
    const int comp = tid / XR, jr = tid - comp * XR;
    const int J = 2 * (r0 - 1) + 2 * NW * k + jr;
    uint64_t* bar = &xbar[k & 1];
    if (J < 0 || J >= nv1) {
      mbar_arrive_tx(bar, 0);
      return;
    }
    T* dst = sx + ((k & 1) * SM::XROWS + tid) * D::XS;
    const long long e_lo = (long long)comp * Nv + (long long)J * nv0 + I0;
    xph[(k & 1) * SM::XROWS + tid] = (uint8_t)stage_row<T, D::XCH>(dst, A.xu, vlen, e_lo, bar);
  };
  auto stage_b = [&](int k) {  // operand row of batch k for lane < WROWS of warp w (vc = vec * 2 + comp)
    int vc, jr;
    if (lane < 4 * NV) {
      vc = lane >> 1;
      jr = 2 * w + (lane & 1);
    } else {
      vc = lane - 4 * NV;
      jr = 2 * NW;  // the mesh's top node row, read by warp NW - 1 only
    }
    const int vec = vc >> 1, comp = vc & 1;
    const int J = 2 * (r0 - 1) + 2 * NW * k + jr;
    const bool need = (lane < 4 * NV || w == NW - 1) && J < nv1 &&
                      ((J >= own_lo && J < own_hi) || J == 2 * n1) &&
                      !(MODE == TILE_CHEB && vec == 1 && !A.use_d);
    uint64_t* bar = &obar[w];
    if (!need) {
      mbar_arrive_tx(bar, 0);
      return;
    }
    const T* v = vec == 0 ? A.bu : (vec == 1 ? (const T*)A.d : A.dinv);
    const long long e_lo = (long long)comp * Nv + (long long)J * nv0 + Ib;
    const int row = vc * XR + jr;
    bph[row] = (uint8_t)stage_row<T, D::BCH>(sb + row * D::BS, v, vlen, e_lo, bar);
  };
  // per-cell data of the cell a thread evaluates in batch k (loaded one batch ahead)
  struct CellData {
    T eta, alpha;
    unsigned cmv;  // constrained local nodes (bits 0..8), obstacle cell (bit 15)
    int cell;
    bool inmesh;
  };
  auto load_cell = [&](int k) {
    CellData d;
    const int c0 = cs0 - 1 + lane, c1 = r0 - 1 + NW * k + w;
    d.inmesh = c0 >= 0 && c0 < n0 && c1 >= 0 && c1 < n1;
    d.cell = d.inmesh ? c0 + n0 * c1 : 0;
    d.cmv = 0;
    d.eta = T(0);
    d.alpha = T(1);
    if (d.inmesh) {
      d.cmv = g.ccmask ? (unsigned)g.ccmask[d.cell] : face_cell_mask(g, c0, c1);
      d.eta = A.eta[d.cell];
      if (A.alpha) d.alpha = A.alpha[d.cell];
    }
    return d;
  };

  if (xrole) stage_x(0);
  if (brole) stage_b(0);
  CellData cd = load_cell(0);

#pragma unroll 1
  for (int k = 0; k < nb; ++k) {
    mbar_wait(&xbar[k & 1], (unsigned)((k >> 1) & 1), A.err);
    cp_async_wait<0>();
    __syncthreads();  // (A) x window of batch k visible; batch k - 1 finished with every buffer
    if (k + 1 < nb && xrole) {  // batch k + 1's x window fills the buffer batch k - 1 used
      fence_proxy_async();
      stage_x(k + 1);
    }
    const CellData cur = cd;
    if (k + 1 < nb) cd = load_cell(k + 1);

    const int t = NW * k + w;          // processed row index within the segment (0: halo row)
    const int c0 = cs0 - 1 + lane, c1 = r0 - 1 + t;
    const bool inmesh = cur.inmesh;
    const int cell = cur.cell;
    const unsigned cmv = cur.cmv;
    const unsigned cm = raw ? 0u : (cmv & 0x1FFu);
    const bool active = inmesh && !(cmv & 0x8000u) && cm != 0x1FFu;
    const T* xb = sx + (k & 1) * (SM::XROWS * D::XS);
    const uint8_t* xp = xph + (k & 1) * SM::XROWS;
    const T* xrow[2][3];  // the cell's three node rows of each component
#pragma unroll
    for (int comp = 0; comp < 2; ++comp)
#pragma unroll
      for (int lb = 0; lb < 3; ++lb) {
        const int r = comp * XR + 2 * w + lb;
        xrow[comp][lb] = xb + r * D::XS + xp[r] + 2 * lane;
      }

    T y[2][9];
#pragma unroll
    for (int i = 0; i < 9; ++i) y[0][i] = y[1][i] = T(0);
    if (active) {
      const T eta = cur.eta * c.eta_scale;
      OpCoef<T> cK = c;
      if (A.alpha) cK.mm = c.mm * cur.alpha;
      T xl[2][9];
#pragma unroll
      for (int comp = 0; comp < 2; ++comp)
#pragma unroll
        for (int lb = 0; lb < 3; ++lb)
#pragma unroll
          for (int la = 0; la < 3; ++la) xl[comp][la + 3 * lb] = xrow[comp][lb][la];
      if (cm) {  // constrained columns enter as zero
#pragma unroll
        for (int i = 0; i < 9; ++i)
          if ((cm >> i) & 1u) xl[0][i] = xl[1][i] = T(0);
      }
      cell_A2(xl, y, eta, cK);
    }
    // top node row, unreduced, to the warp above (warp NW - 1: to warp 0 of the next batch, which
    // reads it after the next barrier (A)); slots alternate with the batch parity, and a warp can
    // be at most one batch ahead of another (barrier (A)), so a slot is never overwritten unread
    {
      T* slot = sxch + ((k & 1) * NW + w) * (NX * 32);
#pragma unroll
      for (int comp = 0; comp < 2; ++comp)
#pragma unroll
        for (int la = 0; la < 3; ++la) slot[(comp * 3 + la) * 32 + lane] = y[comp][6 + la];
      if (w < NW - 1) named_arrive(1 + w);  // slot of warp w is ready for warp w + 1
    }
    // x-reduction: the left node column receives the right column of the cell to the left
#pragma unroll
    for (int comp = 0; comp < 2; ++comp)
#pragma unroll
      for (int lb = 0; lb < 3; ++lb) {
        const T v = __shfl_up_sync(0xffffffffu, y[comp][2 + 3 * lb], 1);
        if (lane > 0) y[comp][3 * lb] += v;
      }
    if (w > 0) named_sync(w);  // the slot of warp w - 1 is ready
    // y-reduction of the bottom node row: + the cell below (C), then + the cell below-left (D), so
    // an interior vertex sums ((own + left) + below) + below-left, a fixed order
    if (t >= 1) {
      const T* slot = w > 0 ? sxch + ((k & 1) * NW + w - 1) * (NX * 32) : sxch + (((k - 1) & 1) * NW + NW - 1) * (NX * 32);
#pragma unroll
      for (int comp = 0; comp < 2; ++comp) {
        y[comp][0] += slot[(comp * 3 + 0) * 32 + lane];
        if (lane > 0) y[comp][0] += slot[(comp * 3 + 2) * 32 + lane - 1];
        y[comp][1] += slot[(comp * 3 + 1) * 32 + lane];
        y[comp][2] += slot[(comp * 3 + 2) * 32 + lane];
      }
    }

    // ---- epilogue: owned nodes (2 c0 + la, 2 c1 + lb), la, lb in {0, 1}; the right / top mesh
    // boundary nodes (la = 2 / lb = 2) belong to the last cell column / row ----
    if (NV > 0) {  // this warp's operand rows of batch k
      mbar_wait(&obar[w], (unsigned)(k & 1), A.err);
      cp_async_wait<0>();
      __syncwarp();
    }
    if (inmesh && lane >= 1 && t >= 1) {
      const int node0 = 2 * c0 + nv0 * (2 * c1);
      const int bcol0 = 2 * (lane - 1);
      const unsigned con_bits = raw ? 0u : cmv;
      // node row lb, columns la in [0, la_n): result, operands and stores through per-row pointers
      auto node_row = [&](int lb, int la_n) {
        const int jr = 2 * w + lb;
#pragma unroll
        for (int comp = 0; comp < 2; ++comp) {
          const int off = comp * Nv + node0 + nv0 * lb;
          const T* xr = xrow[comp][lb];
          const T* br = nullptr;
          const T* dr = nullptr;
          const T* ir = nullptr;
          if (MODE != TILE_APPLY) {
            const int rb = comp * XR + jr;
            br = sb + rb * D::BS + bph[rb] + bcol0;
            if (MODE == TILE_CHEB) {
              const int rd = rb + 2 * XR, ri = rb + 4 * XR;
              dr = sb + rd * D::BS + bph[rd] + bcol0;
              ir = sb + ri * D::BS + bph[ri] + bcol0;
            }
          }
#pragma unroll
          for (int la = 0; la < 3; ++la) {
            if (la >= la_n) break;
            const bool con = (con_bits >> (la + 3 * lb)) & 1u;
            const T xin = xr[la];
            const T ax = con ? xin : y[comp][la + 3 * lb];
            if (MODE == TILE_APPLY) {
              A.yu[off + la] = ax;
            } else if (MODE == TILE_RESID) {
              A.yu[off + la] = br[la] - ax;
            } else {
              T dn = A.c2 * ir[la] * (br[la] - ax);
              if (A.use_d) dn += A.c1 * dr[la];
              A.d[off + la] = dn;
              A.xout[off + la] = xin + dn;
            }
          }
        }
      };
      if (c0 < n0 - 1) {  // the common case: two node rows of two nodes
        node_row(0, 2);
        node_row(1, 2);
      } else {            // last cell column: also the mesh's right boundary node column
        node_row(0, 3);
        node_row(1, 3);
      }
      if (c1 == n1 - 1) node_row(2, c0 < n0 - 1 ? 2 : 3);  // last cell row: the top boundary row
    }
    if (NV > 0 && k + 1 < nb) {  // the warp is done with its operand rows: fetch batch k + 1's
      __syncwarp();
      if (brole) {
        fence_proxy_async();
        stage_b(k + 1);
      }
    }
  }
}

template <typename T, int MODE>
struct Strip2dK {
  using Args = TileArgs<T>;
  static constexpr int THREADS = NT, MINB = sizeof(T) == 4 ? 3 : 1;
  static __device__ __forceinline__ void body(const Args& a, int blk, int) { strip2d_body<T, MODE>(a, blk); }
};

}  // namespace strip2d

// y = A x (TILE_APPLY), y = b - A x (TILE_RESID) or the fused Chebyshev step (TILE_CHEB) on a 2D
// level with the strip kernel (gs_strip2d.cu).
template <typename T>
cudaError_t launch_strip2d(int mode, TileArgs<T> a, cudaStream_t st);

}  // namespace gs
