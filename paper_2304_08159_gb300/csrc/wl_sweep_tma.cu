// TMA-staged multigrid kernels of project! (Section 2): the red-black Gauss-Seidel
// sweep (red-black ordering is this library's reading of the smoother) and the fine
// residual / divergence pass.  Same arithmetic and results as k_sweep and
// k_residual; the difference is how the data reaches shared memory.
//
// A tile of 64 x 8 cells (64 x 16 on large split levels) marches up through `tz`
// planes.  For every plane the five fields it needs (iterate, right-hand side, the three
// face-coefficient fields) are fetched by the tensor-memory accelerator as 72 x 12 boxes
// (72 x 20; tile + halo, x start 16-byte aligned) into two rings of plane slots (iterate: planes k-1..k+3;
// coefficients: planes k..k+3), one plane ahead of the plane being relaxed, each
// staged plane completing on its own mbarrier.  Red (and black) cells are two floats
// apart, so a warp takes 16 cells from each of two adjacent rows: their red columns
// have opposite parity and the row pitch is 8 banks, so the two half-warps touch
// disjoint banks and no shared access conflicts.  Out-of-range elements are
// zero-filled by the copy engine, which is exactly the value a non-periodic wall
// needs (face coefficient 0 across it), so the relaxation itself carries no
// boundary logic (tiles that form their coefficients count a cell's faces for its
// diagonal and sum its zero-filled neighbours like any other).  A tile whose footprint crosses a periodic x or y side takes the
// wrapping variant (uniform tiles only), which overwrites the zero-filled halo elements
// past the side with the wrapped cells' values, read from global memory one plane ahead.
#include <cuda.h>

#include <algorithm>

#include "wl_dev.cuh"
#include "wl_kernels.h"

namespace wl {

namespace {

constexpr int TX = SWEEP_TX, TY = SWEEP_TY;  // tile
constexpr int BX = TX + 8, BY = TY + 4;  // box: x from i0-4 (aligned), y from j0-2
constexpr int BOX = BX * BY;          // floats per field per plane
constexpr int LEAD = 1;         // bundles staged ahead of the iteration that waits for them
constexpr int XR = LEAD + 4;    // iterate slots (planes k-1 .. k+2, and LEAD more in flight)
constexpr int L2R = LEAD + 3;   // L2 slots (planes k .. k+2, and LEAD more in flight)
constexpr int CR = LEAD + 2;    // z, L0, L1 slots (planes k, k+1, and LEAD more in flight)
constexpr int NBB = 2;          // bundle mbarriers (a power of two, > LEAD)
constexpr int SW_NT = 128;      // sweep threads: 4 warps
static_assert(NBB > LEAD && (NBB & (NBB - 1)) == 0, "bundle barriers");
static_assert(BOX * 4 % 128 == 0, "iterate slots keep 128-byte alignment");
// Sweep boxes for a tile height TYV: 8 rows, or 16 on the large split levels (twice the
// cells per warp and plane for the same per-plane bookkeeping, a 1-row halo on 16 rows
// instead of 8).  Iterate box TYV + 4 rows from j0-2; coefficient boxes CROWS rows from
// j0-1 (L1: one more, the upper face of the last row).
template <int TYV>
struct SwGeom {
  static constexpr int BY = TYV + 4, BOX = BX * BY;
  static constexpr int CROWS = TYV + 2, L1ROWS = TYV + 3;
  static constexpr int CSLOT = (BX * CROWS + 31) / 32 * 32, L1SLOT = (BX * L1ROWS + 31) / 32 * 32;
  static_assert(BOX * 4 % 128 == 0, "iterate slots keep 128-byte alignment");
};
constexpr unsigned kWaitLimit = 1u << 21;      // wait attempts
constexpr unsigned kSuspendNs = 10000;         // longest sleep of one attempt
constexpr uint64_t kWaitNs = 2000000000ull;    // longest wait (2 s)

__device__ __forceinline__ uint32_t smem_addr(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}
// One wait attempt: the thread may sleep until the phase completes, for at most
// kSuspendNs, so waiting warps leave the issue slots to the warps with work.
__device__ __forceinline__ bool mbar_try_wait(uint32_t bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(bar), "r"(parity), "n"(kSuspendNs)
      : "memory");
  return ok != 0;
}
__device__ __forceinline__ uint64_t global_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}
// bounded wait: false if the phase did not complete within limit_ns of wall time
// (or kWaitLimit attempts)
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity, uint64_t limit_ns = kWaitNs) {
  if (mbar_try_wait(bar, parity)) return true;
  const uint64_t t0 = global_ns();
  for (unsigned it = 0; it < kWaitLimit; ++it) {
    if (mbar_try_wait(bar, parity)) return true;
    if (global_ns() - t0 > limit_ns) return false;
  }
  return false;
}
__device__ __forceinline__ void tma_load(uint32_t dst, const CUtensorMap* map, int x, int y, int z, uint32_t bar,
                                         int rank) {
  wl_in(x & 3, 1, WL_DBG_TMA);  // the inner coordinate's byte offset must be a multiple of 16
  if (rank == 3)
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], [%5];" ::"r"(
            dst),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(z), "r"(bar)
        : "memory");
  else
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::"r"(
            dst),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(bar)
        : "memory");
}

// shared loads / stores at a 32-bit shared-window byte address (+ immediate offset)
__device__ __forceinline__ float lds(uint32_t a) {
  float v;
  asm volatile("ld.shared.f32 %0, [%1];" : "=f"(v) : "r"(a));
  return v;
}
template <int OFF>
__device__ __forceinline__ float lds(uint32_t a) {
  float v;
  asm volatile("ld.shared.f32 %0, [%1+%2];" : "=f"(v) : "r"(a), "n"(OFF));
  return v;
}
__device__ __forceinline__ void sts(uint32_t a, float v) { asm volatile("st.shared.f32 [%0], %1;" ::"r"(a), "f"(v)); }

}  // namespace

// UNI: the variant for tiles outside the level's band box, whose face coefficients are
// the level's free-stream value uval (0 on the walls): only the iterate and the
// right-hand side are staged, the coefficients are formed from the cell's position
// (same values, same operation order, same bits), and the smaller rings fit more
// blocks per SM.  WRAP (uniform only): the tiles whose footprint crosses a periodic x
// or y side, the others' the tiles that cross none.  TYV: the tile height (8, or 16 on
// large levels split into band and uniform tiles and periodic in neither x nor y).
template <int D, bool UNI, bool WRAP, int TYV>
__global__ void __launch_bounds__(SW_NT, WRAP           ? SWEEP_WRAP_BLOCKS_PER_SM
                                         : TYV == 16    ? (UNI ? SWEEP16_UNI_BLOCKS_PER_SM : SWEEP16_BLOCKS_PER_SM)
                                         : UNI          ? SWEEP_UNI_BLOCKS_PER_SM
                                                        : SWEEP_BLOCKS_PER_SM)
    k_sweep_tma(const __grid_constant__ SweepMaps m, SweepTmaArgs a) {
  static_assert(UNI || !WRAP, "wrapping tiles are uniform");
  static_assert(TYV == 8 || (TYV == 16 && !WRAP), "tile heights: 8, or 16 without wrapping");
  constexpr int TY = TYV, BY = SwGeom<TYV>::BY, BOX = SwGeom<TYV>::BOX;
  constexpr int CROWS = SwGeom<TYV>::CROWS, L1ROWS = SwGeom<TYV>::L1ROWS;
  constexpr int CSLOT = SwGeom<TYV>::CSLOT, L1SLOT = SwGeom<TYV>::L1SLOT;
  extern __shared__ float smf[];
  // 128-byte aligned slot rings (iterate, L2, z, L0, L1), then the mbarriers, all
  // addressed by 32-bit float offsets into smf
  const int ox = (int)(((128u - (smem_addr(smf) & 127u)) & 127u) >> 2);
  constexpr int O_L2 = XR * BOX, O_Z = O_L2 + (UNI ? 0 : L2R * CSLOT), O_L0 = O_Z + CR * CSLOT,
                O_L1 = O_L0 + (UNI ? 0 : CR * CSLOT), O_BAR = O_L1 + (UNI ? 0 : CR * L1SLOT);
  uint64_t* bars = reinterpret_cast<uint64_t*>(smf + ox + O_BAR);
  const Grid& g = a.g;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int i0 = (blockIdx.x + a.t0[0]) * TX, j0 = (blockIdx.y + a.t0[1]) * TY;
  const int k0 = (D == 3) ? (blockIdx.z + a.t0[2]) * a.tz : 0;
  if (i0 >= g.n[0] || j0 >= g.n[1] || k0 >= g.n[2]) return;
  const int k1 = (D == 3) ? min(k0 + a.tz, g.n[2]) : 1;
  if (sweep_tile_wraps_xy(g, i0, j0) != WRAP) return;  // the other launch's tile
  if (tile_in_band(a.band, D, i0, j0, k0, k1, TY) == UNI) return;  // the other variant's tile
  // a plane past a periodic z side is staged from its wrapped plane
  const bool pz = D == 3 && is_per(g, 2);
  auto wz = [&](int p) { return pz ? wrap_per(p, g.n[2]) : p; };
  // Ring slots: iterate plane p lives in slot (p - k0 + 2) mod XR, coefficient plane
  // p in slot (p - k0 + 1) mod L2R (L2) or mod CR (z, L0, L1).
  auto Xs = [&](int s) { return ox + s * BOX; };
  auto L2s = [&](int s) { return ox + O_L2 + s * CSLOT; };
  auto Zs = [&](int s) { return ox + O_Z + s * CSLOT; };
  auto L0s = [&](int s) { return ox + O_L0 + s * CSLOT; };
  auto L1s = [&](int s) { return ox + O_L1 + s * L1SLOT; };
  auto sa = [&](int o) { return smem_addr(smf + o); };
  auto xslot = [&](int p) { return (p - k0 + 2) % XR; };
  auto l2slot = [&](int p) { return (p - k0 + 1) % L2R; };
  auto cslot = [&](int p) { return (p - k0 + 1) % CR; };
  // barrier 0: the prologue's planes; barriers 1..NBB: bundle b, round robin
  auto bbar = [&](int b) { return smem_addr(&bars[1 + ((b - k0) & (NBB - 1))]); };
  auto bphase = [&](int b) { return (uint32_t)(((b - k0) / NBB) & 1); };

  if (tid == 0) {
    for (int s = 0; s <= NBB; ++s) mbar_init(smem_addr(&bars[s]), 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();

  // thread 0 staging.  Coefficient boxes start one row above the tile (j0-1), the
  // iterate's two rows above (j0-2); all start 4 columns left of the tile.
  auto ld_x = [&](int p, uint32_t bar) { tma_load(sa(Xs(xslot(p))), &m.x, i0 - 4, j0 - 2, wz(p), bar, D); };
  auto ld_l2 = [&](int p, uint32_t bar) { tma_load(sa(L2s(l2slot(p))), &m.L2, i0 - 4, j0 - 1, wz(p), bar, D); };
  auto ld_z = [&](int p, uint32_t bar) { tma_load(sa(Zs(cslot(p))), &m.z, i0 - 4, j0 - 1, wz(p), bar, D); };
  auto ld_c = [&](int p, uint32_t bar) {
    const int c = cslot(p);
    ld_z(p, bar);
    tma_load(sa(L0s(c)), &m.L0, i0 - 4, j0 - 1, wz(p), bar, D);
    tma_load(sa(L1s(c)), &m.L1, i0 - 4, j0 - 1, wz(p), bar, D);
  };
  constexpr uint32_t kXB = BOX * 4, kCB = BX * CROWS * 4, kL1B = BX * L1ROWS * 4;
  int b_issued = k0 - 1;  // (thread 0) last bundle staged
  // bundle b (waited at the start of iteration b): iterate and L2 of plane b+2,
  // z, L0, L1 of plane b+1 (UNI: iterate and z)
  auto issue_bundle = [&](int b) {
    b_issued = b;
    if (UNI) {
      mbar_expect_tx(bbar(b), (a.has_x ? kXB : 0u) + kCB);
      if (a.has_x) ld_x(b + 2, bbar(b));
      ld_z(b + 1, bbar(b));
      return;
    }
    mbar_expect_tx(bbar(b), (a.has_x ? kXB : 0u) + 3 * kCB + kL1B);
    if (a.has_x) ld_x(b + 2, bbar(b));
    ld_l2(b + 2, bbar(b));
    ld_c(b + 1, bbar(b));
  };
  // iterate := (staged iterate or 0) + prolonged coarse correction, on plane p.  The
  // box starts at an even cell, so it covers 36 x (TY/2 + 2) coarse cells; each thread owns
  // up to NCR of them and adds each one's value to its 2 x 2 fine cells.  Two fine planes share
  // a coarse plane: a thread keeps the values of the last coarse plane it loaded, and
  // the loop loads the next plane's one iteration ahead of their use.
  const float xcm = a.xc_cs ? ldexpf(1.f, -a.st->cs_used) : 1.f;  // removes the coarse levels' scale
  const bool fix = !a.has_x || a.xc;
  constexpr int CBX = BX / 2, CBOX = CBX * (BY / 2), NCR = (CBOX + SW_NT - 1) / SW_NT;
  static_assert(BX % 2 == 0 && BY % 2 == 0, "coarse box");
  int cxy[NCR], ceo[NCR];  // coarse in-plane index (-1: outside the grid), fine box offset (-1: none)
#pragma unroll
  for (int r = 0; r < NCR; ++r) {
    const int t = tid + SW_NT * r, cr = t / CBX, cc = t - cr * CBX;
    int ci = (i0 >> 1) - 2 + cc, cj = (j0 >> 1) - 1 + cr;
    if (is_per(g, 0)) ci = wrap_per(ci, a.cn[0]);  // a wrapping tile
    if (is_per(g, 1)) cj = wrap_per(cj, a.cn[1]);
    ceo[r] = t < CBOX ? 2 * cr * BX + 2 * cc : -1;
    cxy[r] = (t < CBOX && a.xc && ci >= 0 && ci < a.cn[0] && cj >= 0 && cj < a.cn[1]) ? ci + a.cn[0] * cj : -1;
  }
  float cv[NCR];
#pragma unroll
  for (int r = 0; r < NCR; ++r) cv[r] = 0.f;
  int ckey = -2;  // coarse plane whose values cv holds (-1: outside the grid)
  const long long cplane = (long long)a.cn[0] * a.cn[1];
  auto load_c = [&](int p) {
    const int wp = D == 3 ? wz(p) : p;  // the coarse correction of a wrapped plane
    const int kz = (wp >= 0 && wp < g.n[2]) ? (wp >> 1) : -1;
    if (kz == ckey) return;
    ckey = kz;
    const long long cb = cplane * kz;
#pragma unroll
    for (int r = 0; r < NCR; ++r) {
      const long long ci = cb + cxy[r];
      cv[r] = (kz >= 0 && cxy[r] >= 0 && wl_in(ci, cplane * a.cn[2], WL_DBG_COARSE))
                  ? xcm * ld_st(a.xc, a.xctype, ci)
                  : 0.f;
    }
  };
  auto apply_c = [&](int p) {
    float* X = smf + Xs(xslot(p));
#pragma unroll
    for (int r = 0; r < NCR; ++r) {
      if (ceo[r] < 0) continue;
      float2* q0 = reinterpret_cast<float2*>(X + ceo[r]);
      float2* q1 = reinterpret_cast<float2*>(X + ceo[r] + BX);
      if (!a.has_x) {  // from zero: each of the 2 x 2 cells is 0 + the coarse value
        const float c = 0.f + cv[r];
        *q0 = make_float2(c, c);
        *q1 = make_float2(c, c);
      } else {
        const float2 v0 = *q0, v1 = *q1;
        *q0 = make_float2(v0.x + cv[r], v0.y + cv[r]);
        *q1 = make_float2(v1.x + cv[r], v1.y + cv[r]);
      }
    }
  };
  auto fix_x = [&](int p) {
    load_c(p);
    apply_c(p);
  };
  // WRAP: the halo elements past a periodic x / y side, which the copy engine zero-fills,
  // hold the wrapped cells' values: in the iterate box rows 0-1 / 10-11 (y j0-2, j0-1 /
  // j0+8, j0+9) and columns 0-3 / 68-71, in the right-hand side box row 0 / 9 (y j0-1 /
  // j0+8) and the same columns.  The entries form one list per box, full-width row
  // strips first, then the column strips over the remaining rows; thread t takes
  // entries t, t + 128, ...  Each entry keeps its box offset (-1: none, or a cell past
  // a wall) and the wrapped cell's index in its plane.
  constexpr int NWX = 3, NWZ = 2;  // list lengths <= 352 and <= 208
  int wxo[NWX], wzo[NWZ];
  unsigned wxq[NWX], wzq[NWZ];
  float wxv[NWX], wzv[NWZ];  // values of the next planes to patch
  if constexpr (WRAP) {
    const bool px = is_per(g, 0), py = is_per(g, 1);
    const bool wl = px && i0 == 0, wr = px && i0 + TX == g.n[0];
    const bool wt = py && j0 == 0, wb = py && j0 + TY == g.n[1];
    // rows: box height, ry: rows of one wrapped strip, y0: the box's first y
    auto entry = [&](int t, int rows, int ry, int y0, int& off, unsigned& q) {
      const int rt = wt ? ry : 0, rb = wb ? ry : 0, hr = rows - rt - rb;
      const int nrow = (rt + rb) * BX, ncol = ((wl ? 1 : 0) + (wr ? 1 : 0)) * 4 * hr;
      int row, col;
      if (t < nrow) {
        const int r = t / BX;
        row = r < rt ? r : rows - rb + (r - rt);
        col = t - r * BX;
      } else if (t < nrow + ncol) {
        const int u = t - nrow, sd = u / (4 * hr), v = u - sd * 4 * hr;
        row = rt + (v >> 2);
        col = (wl && sd == 0) ? (v & 3) : BX - 4 + (v & 3);
      } else {
        off = -1;
        q = 0u;
        return;
      }
      int gi = i0 - 4 + col, gj = y0 + row;
      if (px) gi = wrap_per(gi, g.n[0]);
      if (py) gj = wrap_per(gj, g.n[1]);
      const bool in = gi >= 0 && gi < g.n[0] && gj >= 0 && gj < g.n[1];
      off = in ? row * BX + col : -1;
      q = in ? (unsigned)gi + (unsigned)g.n[0] * (unsigned)gj : 0u;
    };
#pragma unroll
    for (int r = 0; r < NWX; ++r) entry(tid + SW_NT * r, BY, 2, j0 - 2, wxo[r], wxq[r]);
#pragma unroll
    for (int r = 0; r < NWZ; ++r) entry(tid + SW_NT * r, CROWS, 1, j0 - 1, wzo[r], wzq[r]);
  }
  // in-plane offset of plane p's wrapped plane, or -1 past a wall in z
  auto wplane = [&](int p) -> long long {
    if (D == 2) return 0;
    const int w = wz(p);
    return (w >= 0 && w < g.n[2]) ? (long long)g.n[0] * g.n[1] * w : -1;
  };
  auto wload_x = [&](int p, float* v) {
    const long long o = wplane(p);
#pragma unroll
    for (int r = 0; r < NWX; ++r)
      v[r] = (o >= 0 && wxo[r] >= 0 && wl_in(o + wxq[r], g.nc, WL_DBG_SWEEP)) ? a.xsrc[o + wxq[r]] : 0.f;
  };
  auto wload_z = [&](int p, float* v) {
    const long long o = wplane(p);
#pragma unroll
    for (int r = 0; r < NWZ; ++r)
      v[r] = (o >= 0 && wzo[r] >= 0 && wl_in(o + wzq[r], g.nc, WL_DBG_SWEEP)) ? a.zsrc[o + wzq[r]] : 0.f;
  };
  auto wstore_x = [&](int p, const float* v) {
    float* X = smf + Xs(xslot(p));
#pragma unroll
    for (int r = 0; r < NWX; ++r)
      if (wxo[r] >= 0) X[wxo[r]] = v[r];
  };
  auto wstore_z = [&](int p, const float* v) {
    float* Z = smf + Zs(cslot(p));
#pragma unroll
    for (int r = 0; r < NWZ; ++r)
      if (wzo[r] >= 0) Z[wzo[r]] = v[r];
  };
  // Operand planes of a relaxation (shared byte addresses): iterate planes below /
  // at / above, and the coefficient planes (shifted one row so that one shared
  // offset e addresses the iterate box and the coefficient boxes).
  struct Planes {
    uint32_t xm, x0, xp, z, l0, l1, l2, l2u;
  };
  const uint32_t sb = smem_addr(smf);
  // sxm: slot of the iterate plane below; sl: L2 slot of the plane; sc: z/L0/L1 slot
  auto planes = [&](int sxm, int sl, int sc) -> Planes {
    Planes P;
    P.xm = sb + 4u * Xs(sxm);
    P.x0 = sb + 4u * Xs(sxm + 1 < XR ? sxm + 1 : sxm + 1 - XR);
    P.xp = sb + 4u * Xs(sxm + 2 < XR ? sxm + 2 : sxm + 2 - XR);
    P.z = sb + 4u * (Zs(sc) - BX);
    P.l0 = sb + 4u * (L0s(sc) - BX);
    P.l1 = sb + 4u * (L1s(sc) - BX);
    P.l2 = sb + 4u * (L2s(sl) - BX);
    P.l2u = sb + 4u * (L2s(sl + 1 < L2R ? sl + 1 : 0) - BX);
    return P;
  };
  auto planes_of = [&](int p) { return planes(xslot(p - 1), l2slot(p), cslot(p)); };
  // Gauss-Seidel value of the cell at shared byte offset e (all operands staged;
  // out-of-range faces carry 0, so cells outside the grid come out as 0).
  // Same operation order as k_sweep (upper then lower face; x, y, z), same bits.
  // UNI: coefficients from the cell's position.  mxy: bit 0/1 lower/upper x face
  // present, 2/3 lower/upper y face, 4 cell inside the grid in x and y; zlo/zhi: lower /
  // upper z face present, kin: plane inside the grid.
  const float uv = a.uval;
  // UNI tile whose x/y footprint touches no wall: on a plane with both z faces
  // (zfull) every cell it relaxes, halo included, has all its faces, each coefficient is
  // uv, so the relaxation is the same FMA chain with uv and the diagonal the constant
  // 2D uv (the same bits as relax_cnt and as the loading kernel's relax)
  const bool interior = UNI && i0 >= 4 && i0 + TX + 4 <= g.n[0] && j0 >= 2 && j0 + TY + 2 <= g.n[1];
  const float dg_int = D == 3 ? (uv + uv) + (uv + uv) + (uv + uv) : (uv + uv) + (uv + uv);
  auto relax_fast = [&](const Planes& P, uint32_t e) -> float {
    const uint32_t x0 = P.x0 + e;
    float sum = fmaf(uv, lds<4>(x0), 0.f);
    sum = fmaf(uv, lds<-4>(x0), sum);
    sum = fmaf(uv, lds<4 * BX>(x0), sum);
    sum = fmaf(uv, lds<-4 * BX>(x0), sum);
    if (D == 3) {
      sum = fmaf(uv, lds(P.xp + e), sum);
      sum = fmaf(uv, lds(P.xm + e), sum);
    }
    return __fdividef(sum - lds(P.z + e), dg_int);
  };
  // two cells at once in packed FP32 pairs (each lane rounds as relax_fast does)
  auto relax_fast2 = [&](const Planes& P, uint32_t e0, uint32_t e1) -> float2 {
    const uint32_t a0 = P.x0 + e0, a1 = P.x0 + e1;
    const float2 u2 = make_float2(uv, uv);
    float2 sum = fma2(u2, make_float2(lds<4>(a0), lds<4>(a1)), make_float2(0.f, 0.f));
    sum = fma2(u2, make_float2(lds<-4>(a0), lds<-4>(a1)), sum);
    sum = fma2(u2, make_float2(lds<4 * BX>(a0), lds<4 * BX>(a1)), sum);
    sum = fma2(u2, make_float2(lds<-4 * BX>(a0), lds<-4 * BX>(a1)), sum);
    if (D == 3) {
      sum = fma2(u2, make_float2(lds(P.xp + e0), lds(P.xp + e1)), sum);
      sum = fma2(u2, make_float2(lds(P.xm + e0), lds(P.xm + e1)), sum);
    }
    const float2 d = sub2(sum, make_float2(lds(P.z + e0), lds(P.z + e1)));
    return make_float2(__fdividef(d.x, dg_int), __fdividef(d.y, dg_int));
  };
  // UNI cell of a tile touching a wall: the masked relaxation (coefficient uv on
  // present faces, 0 on missing ones, as the loading kernel's relax with the level's
  // coefficients) from the constant-coefficient FMA chain.  A face is missing only where
  // the neighbour lies outside the grid (non-periodic side), and every such neighbour
  // holds +0 in the box (zero fill of the copy, or a 0 written by this relaxation for a
  // cell outside), so each term uv * 0 adds the same +0 as 0 * x would; the running sum
  // is never -0 (it starts from +0 and an exact cancellation rounds to +0), so the sums
  // agree bit for bit.  The diagonal is nf uv with nf the cell's present faces: exact,
  // as the masked sum of 0s and uv is (uv a power of two).  Cells outside the grid give 0.
  auto dg_of = [&](uint32_t mxy, int nz) { return uv * (float)(__popc(mxy & 15u) + nz); };
  auto relax_cnt = [&](const Planes& P, uint32_t e, uint32_t mxy, int nz, bool kin) -> float {
    const uint32_t x0 = P.x0 + e;
    float sum = fmaf(uv, lds<4>(x0), 0.f);
    sum = fmaf(uv, lds<-4>(x0), sum);
    sum = fmaf(uv, lds<4 * BX>(x0), sum);
    sum = fmaf(uv, lds<-4 * BX>(x0), sum);
    if (D == 3) {
      sum = fmaf(uv, lds(P.xp + e), sum);
      sum = fmaf(uv, lds(P.xm + e), sum);
    }
    const float dg = dg_of(mxy, nz);
    return ((mxy & 16u) && kin && dg > 0.f) ? __fdividef(sum - lds(P.z + e), dg) : 0.f;
  };
  auto relax_cnt2 = [&](const Planes& P, uint32_t e0, uint32_t e1, uint32_t m0, uint32_t m1, int nz,
                        bool kin) -> float2 {
    const uint32_t a0 = P.x0 + e0, a1 = P.x0 + e1;
    const float2 u2 = make_float2(uv, uv);
    float2 sum = fma2(u2, make_float2(lds<4>(a0), lds<4>(a1)), make_float2(0.f, 0.f));
    sum = fma2(u2, make_float2(lds<-4>(a0), lds<-4>(a1)), sum);
    sum = fma2(u2, make_float2(lds<4 * BX>(a0), lds<4 * BX>(a1)), sum);
    sum = fma2(u2, make_float2(lds<-4 * BX>(a0), lds<-4 * BX>(a1)), sum);
    if (D == 3) {
      sum = fma2(u2, make_float2(lds(P.xp + e0), lds(P.xp + e1)), sum);
      sum = fma2(u2, make_float2(lds(P.xm + e0), lds(P.xm + e1)), sum);
    }
    const float2 d = sub2(sum, make_float2(lds(P.z + e0), lds(P.z + e1)));
    const float dg0 = dg_of(m0, nz), dg1 = dg_of(m1, nz);
    return make_float2(((m0 & 16u) && kin && dg0 > 0.f) ? __fdividef(d.x, dg0) : 0.f,
                       ((m1 & 16u) && kin && dg1 > 0.f) ? __fdividef(d.y, dg1) : 0.f);
  };
  auto relax = [&](const Planes& P, uint32_t e) -> float {
    const uint32_t x0 = P.x0 + e, l0 = P.l0 + e, l1 = P.l1 + e;
    const float l0u = lds<4>(l0), l0d = lds(l0), l1u = lds<4 * BX>(l1), l1d = lds(l1);
    float sum = fmaf(l0u, lds<4>(x0), 0.f);
    sum = fmaf(l0d, lds<-4>(x0), sum);
    float dg = l0u + l0d;
    sum = fmaf(l1u, lds<4 * BX>(x0), sum);
    sum = fmaf(l1d, lds<-4 * BX>(x0), sum);
    dg += l1u + l1d;
    if (D == 3) {
      const float lu = lds(P.l2u + e), ll = lds(P.l2 + e);
      sum = fmaf(lu, lds(P.xp + e), sum);
      sum = fmaf(ll, lds(P.xm + e), sum);
      dg += lu + ll;
    }
    return (dg > 0.f) ? __fdividef(sum - lds(P.z + e), dg) : 0.f;
  };
  // Red cells of plane p cover the tile plus a 1-cell halo (rows -1..TY, columns
  // -1..64): TY+2 tasks of 32 (two adjacent rows x half the tile's columns) and TY+2
  // edge-column cells.  Warp w takes red tasks w, w+4, .., w+TY-4 (NRH = TY/4 of them,
  // in pairs), and a last red task: w+TY for warps 0-1, or TY/2+1 edge cells (the upper
  // half of the rows on warp 2, the lower half on warp 3).  Black cells of plane k (rows
  // 0..TY-1): TY tasks, w, w+4, .. in pairs.  So every warp relaxes NRH/2 red pairs, one
  // red single and NRH/2 black pairs per plane (TY 8: one of each; TY 16: two pairs of
  // each).  Shared byte offsets into the iterate box, for even and odd planes.
  constexpr int NRH = TY / 4, NEDGE = TY / 2 + 1;
  static_assert(NRH % 2 == 0, "tasks in pairs");
  uint32_t er[NRH + 1][2], eb[NRH][2];
  uint32_t mr[NRH + 1][2], mb[NRH][2];  // UNI: face masks of each task's cell (relax_cnt)
  auto xymask = [&](int col, int row) -> uint32_t {
    const int gi = i0 + col, gj = j0 + row;
    const bool px = is_per(g, 0), py = is_per(g, 1);
    // past a periodic side (a wrapping tile's halo) the cell is the wrapped one
    const bool in = ((gi >= 0 && gi < g.n[0]) || px) && ((gj >= 0 && gj < g.n[1]) || py);
    return (gi > 0 || px ? 1u : 0u) | (gi + 1 < g.n[0] || px ? 2u : 0u) | (gj > 0 || py ? 4u : 0u) |
           (gj + 1 < g.n[1] || py ? 8u : 0u) | (in ? 16u : 0u);
  };
  const bool third = warp < 2 || lane < NEDGE;  // this lane has a last red cell
  {
    const int ib0 = 2 * (lane & 15);
#pragma unroll
    for (int h = 0; h <= NRH; ++h) {
      const int t = warp + 4 * h;
      const int jr = 2 * (t >> 1) + (lane >> 4) - 1, jb = jr + 1;
      const int ib = 32 * (t & 1) + ib0;
      const int je = (warp == 2) ? lane - 1 : lane + NEDGE - 1;  // edge rows (last cell of warps 2, 3)
#pragma unroll
      for (int par = 0; par < 2; ++par) {
        int cr = ib + ((i0 + j0 + jr + par) & 1), rr = jr;
        if (h == NRH && warp >= 2) {
          cr = ((i0 + j0 + je + par) & 1) ? -1 : 64;
          rr = je;
        }
        er[h][par] = 4u * ((rr + 2) * BX + cr + 4);
        if (UNI) mr[h][par] = xymask(cr, rr);
        if (h < NRH) {
          const int cb = ib + ((i0 + j0 + jb + par + 1) & 1);
          eb[h][par] = 4u * ((jb + 2) * BX + cb + 4);
          if (UNI) mb[h][par] = xymask(cb, jb);
        }
      }
    }
  }
  // UNI, tiles that touch a wall: bit t of fast_m is set when every lane's cell of task t
  // (red 2h+par, the last red 2 NRH+par, black BLK+2h+par) is inside the grid with all
  // four x/y faces, so that on a plane with both z faces the task takes relax_fast (same
  // bits)
  constexpr int BLK = 2 * NRH + 2;
  uint32_t fast_m = 0u;
  if (UNI) {
#pragma unroll
    for (int par = 0; par < 2; ++par) {
#pragma unroll
      for (int h = 0; h < NRH; ++h) {
        if (__all_sync(0xffffffffu, mr[h][par] == 31u)) fast_m |= 1u << (2 * h + par);
        if (__all_sync(0xffffffffu, mb[h][par] == 31u)) fast_m |= 1u << (BLK + 2 * h + par);
      }
      if (__all_sync(0xffffffffu, !third || mr[NRH][par] == 31u)) fast_m |= 1u << (2 * NRH + par);
    }
  }
  // UNI: z faces and range of plane kk
  auto zmask = [&](int kk, bool& zlo, bool& zhi, bool& kin) {
    zlo = kk > 0 || pz;
    zhi = kk + 1 < g.n[2] || pz;
    kin = pz || (kk >= 0 && kk < g.n[2]);
  };
  // plane kk is in the grid with both z faces
  auto zfull = [&](int kk) { return D == 2 || pz || (kk > 0 && kk + 1 < g.n[2]); };
  // red cells of plane kk (parity par) whose operands are P
  auto red_plane = [&](const Planes& P, int par, int kk) {
    auto pk = [&](const uint32_t(&v)[2]) { return par ? v[1] : v[0]; };
    const uint32_t e2 = pk(er[NRH]);
    if (UNI && interior && zfull(kk)) {
#pragma unroll
      for (int hp = 0; hp < NRH / 2; ++hp) {
        const uint32_t e0 = pk(er[2 * hp]), e1 = pk(er[2 * hp + 1]);
        const float2 v = relax_fast2(P, e0, e1);
        sts(P.x0 + e0, v.x);
        sts(P.x0 + e1, v.y);
      }
      if (third) sts(P.x0 + e2, relax_fast(P, e2));
      return;
    }
    if constexpr (UNI) {
      bool zlo, zhi, kin;
      zmask(kk, zlo, zhi, kin);
      const uint32_t fm = (zlo && zhi && kin) ? fast_m >> par : 0u;
      const int nz = D == 3 ? (zlo ? 1 : 0) + (zhi ? 1 : 0) : 0;
#pragma unroll
      for (int hp = 0; hp < NRH / 2; ++hp) {
        const uint32_t e0 = pk(er[2 * hp]), e1 = pk(er[2 * hp + 1]);
        const uint32_t b0 = 1u << (4 * hp), b1 = 4u << (4 * hp);
        const float2 v = ((fm & (b0 | b1)) == (b0 | b1)) ? relax_fast2(P, e0, e1)
                                                          : relax_cnt2(P, e0, e1, pk(mr[2 * hp]), pk(mr[2 * hp + 1]), nz, kin);
        sts(P.x0 + e0, v.x);
        sts(P.x0 + e1, v.y);
      }
      if (third) sts(P.x0 + e2, ((fm >> (2 * NRH)) & 1u) ? relax_fast(P, e2) : relax_cnt(P, e2, pk(mr[NRH]), nz, kin));
    } else {
#pragma unroll
      for (int hp = 0; hp < NRH / 2; ++hp) {
        const uint32_t e0 = pk(er[2 * hp]), e1 = pk(er[2 * hp + 1]);
        const float v0 = relax(P, e0), v1 = relax(P, e1);
        sts(P.x0 + e0, v0);
        sts(P.x0 + e1, v1);
      }
      if (third) sts(P.x0 + e2, relax(P, e2));
    }
  };
  // black cells of plane kk (parity par) whose operands are P
  auto black_plane = [&](const Planes& P, int par, int kk) {
    auto pk = [&](const uint32_t(&v)[2]) { return par ? v[1] : v[0]; };
    if (UNI && interior && zfull(kk)) {
#pragma unroll
      for (int hp = 0; hp < NRH / 2; ++hp) {
        const uint32_t e0 = pk(eb[2 * hp]), e1 = pk(eb[2 * hp + 1]);
        const float2 v = relax_fast2(P, e0, e1);
        sts(P.x0 + e0, v.x);
        sts(P.x0 + e1, v.y);
      }
      return;
    }
    if constexpr (UNI) {
      bool zlo, zhi, kin;
      zmask(kk, zlo, zhi, kin);
      const uint32_t fm = (zlo && zhi && kin) ? fast_m >> (BLK + par) : 0u;
      const int nz = D == 3 ? (zlo ? 1 : 0) + (zhi ? 1 : 0) : 0;
#pragma unroll
      for (int hp = 0; hp < NRH / 2; ++hp) {
        const uint32_t e0 = pk(eb[2 * hp]), e1 = pk(eb[2 * hp + 1]);
        const uint32_t b0 = 1u << (4 * hp), b1 = 4u << (4 * hp);
        const float2 v = ((fm & (b0 | b1)) == (b0 | b1)) ? relax_fast2(P, e0, e1)
                                                          : relax_cnt2(P, e0, e1, pk(mb[2 * hp]), pk(mb[2 * hp + 1]), nz, kin);
        sts(P.x0 + e0, v.x);
        sts(P.x0 + e1, v.y);
      }
    } else {
#pragma unroll
      for (int hp = 0; hp < NRH / 2; ++hp) {
        const uint32_t e0 = pk(eb[2 * hp]), e1 = pk(eb[2 * hp + 1]);
        const float v0 = relax(P, e0), v1 = relax(P, e1);
        sts(P.x0 + e0, v0);
        sts(P.x0 + e1, v1);
      }
    }
  };
  // Write the tile's plane k: 32 TY column pairs, pairs t, t + 128, .. for thread t;
  // pair (tx, ty) is columns 2tx, 2tx+1 of row ty (n0 % 4 == 0, so both columns
  // exist when the first does).
  constexpr int NST = 32 * TY / SW_NT;
  bool st_own[NST];
  long long q0[NST];
  int est[NST];
#pragma unroll
  for (int r = 0; r < NST; ++r) {
    const int pos = tid + SW_NT * r, stx = pos & 31, sty = pos >> 5;
    const int gi = i0 + 2 * stx, gj = j0 + sty;
    st_own[r] = gi < g.n[0] && gj < g.n[1];
    q0[r] = (long long)gi + (long long)g.n[0] * gj;
    est[r] = (sty + 2) * BX + 2 * stx + 4;
  }
  const long long qk = (long long)g.n[0] * g.n[1];
  float2 hph[NST], hpl[NST];  // ph, pl of the next plane to store
#pragma unroll
  for (int r = 0; r < NST; ++r) hph[r] = hpl[r] = make_float2(0.f, 0.f);
  auto prefetch = [&](int k) {
    if (!a.ph || k >= k1) return;
#pragma unroll
    for (int r = 0; r < NST; ++r)
      if (st_own[r] && wl_in(q0[r] + (D == 3 ? qk * k : 0) + 1, g.nc, WL_DBG_SWEEP)) {
        const long long q = q0[r] + (D == 3 ? qk * k : 0);
        hph[r] = *reinterpret_cast<const float2*>(a.ph + q);
        hpl[r] = *reinterpret_cast<const float2*>(a.pl + q);
      }
  };
  auto store = [&](int Xk, int k) {
#pragma unroll
    for (int r = 0; r < NST; ++r) {
      if (!st_own[r]) continue;
      if (!wl_in(q0[r] + (D == 3 ? qk * k : 0) + 1, g.nc, WL_DBG_SWEEP)) continue;
      const float2 v = *reinterpret_cast<const float2*>(smf + Xk + est[r]);
      const long long q = q0[r] + (D == 3 ? qk * k : 0);
      if (a.ph) {
        // (ph, pl) += v for both columns at once in packed pairs (the scalar bits)
        float2 sh, sl;
        two_sum2(hph[r], v, sh, sl);
        sl = add2(sl, hpl[r]);
        const float2 nh = add2(sh, sl);
        *reinterpret_cast<float2*>(a.ph + q) = nh;
        *reinterpret_cast<float2*>(a.pl + q) = sub2(sl, sub2(nh, sh));
      } else {
        *reinterpret_cast<float2*>(a.x_out + q) = v;
      }
    }
  };
  // a copy timed out: flag it, wait (bounded) for the copies still in flight so none
  // lands after the block has left, then leave
  auto bail = [&](bool prologue_pending, int b_fail) {
    if (tid == 0) {
      atomicOr(&a.st->status, 4);
      if (prologue_pending) mbar_wait(smem_addr(&bars[0]), 0);
      for (int b = b_fail; b <= b_issued; ++b) mbar_wait(bbar(b), bphase(b));
    }
    __syncthreads();
  };

  // ---- prologue: iterate planes k0-2..k0+1, coefficients k0-1..k0 (L2 to k0+1),
  // and the first LEAD bundles
  const int plo = (D == 3) ? k0 - 2 : 0, phi = (D == 3) ? k0 + 1 : 0;
  if (tid == 0) {
    const int ncp = (D == 3) ? 2 : 1, nl2 = (D == 3) ? 3 : 0;
    const uint32_t b0 = smem_addr(&bars[0]);
    if (UNI)
      mbar_expect_tx(b0, (a.has_x ? (uint32_t)(phi - plo + 1) * kXB : 0u) + (uint32_t)ncp * kCB);
    else
      mbar_expect_tx(b0, (a.has_x ? (uint32_t)(phi - plo + 1) * kXB : 0u) + (uint32_t)ncp * (2 * kCB + kL1B) +
                             (uint32_t)nl2 * kCB);
    if (a.has_x)
      for (int p = plo; p <= phi; ++p) ld_x(p, b0);
    for (int p = (D == 3 ? k0 - 1 : 0); p <= (D == 3 ? k0 : 0); ++p) {
      if (UNI)
        ld_z(p, b0);
      else
        ld_c(p, b0);
    }
    if (D == 3 && !UNI)
      for (int p = k0 - 1; p <= k0 + 1; ++p) ld_l2(p, b0);
    if (D == 3)
      for (int b = k0; b < k0 + LEAD && b <= k1 - 1; ++b) issue_bundle(b);
  }
  // WRAP: the prologue's patch values, read while the copies are in flight
  float wpx[4][NWX], wpz[2][NWZ];
  if constexpr (WRAP) {
    if (a.has_x)
      for (int p = plo; p <= phi; ++p) wload_x(p, wpx[p - plo]);
    for (int p = (D == 3 ? k0 - 1 : 0); p <= (D == 3 ? k0 : 0); ++p) wload_z(p, wpz[p - (D == 3 ? k0 - 1 : 0)]);
  }
  {
    const bool ok = mbar_wait(smem_addr(&bars[0]), 0);
    if (__syncthreads_or(!ok)) return bail(true, k0);
  }
  if constexpr (WRAP) {
    if (a.has_x)
      for (int p = plo; p <= phi; ++p) wstore_x(p, wpx[p - plo]);
    for (int p = (D == 3 ? k0 - 1 : 0); p <= (D == 3 ? k0 : 0); ++p) wstore_z(p, wpz[p - (D == 3 ? k0 - 1 : 0)]);
    __syncthreads();
    if (D == 3) {  // bundle k0's planes
      if (a.has_x) wload_x(k0 + 2, wxv);
      wload_z(k0 + 1, wzv);
    }
  }
  if (fix) {
    for (int p = plo; p <= phi; ++p) fix_x(p);
    __syncthreads();
    if (D == 3 && k0 + 2 <= k1 + 1) load_c(k0 + 2);
  }
  if constexpr (D == 2) {
    prefetch(0);
    const Planes P = planes_of(0);
    red_plane(P, 0, 0);
    __syncthreads();
    black_plane(P, 0, 0);
    __syncthreads();
    store(Xs(xslot(0)), 0);
    return;
  } else {
  // red cells of planes k0-1 and k0 (independent of each other)
  for (int p = k0 - 1; p <= k0; ++p) red_plane(planes_of(p), p & 1, p);
  prefetch(k0);

  // ---- iteration k: red cells of plane k+1, then black cells of plane k, and the
  // store of plane k-1
  int sx = xslot(k0 - 1), sl = l2slot(k0), sc = cslot(k0);  // rolling slots of planes k-1 / k / k
  for (int k = k0; k < k1; ++k) {
    {
      const bool ok = mbar_wait(bbar(k), bphase(k));
      if (__syncthreads_or(!ok)) return bail(false, k);
      if constexpr (WRAP) {  // bundle k: iterate plane k+2, right-hand side plane k+1
        if (a.has_x) wstore_x(k + 2, wxv);
        wstore_z(k + 1, wzv);
        __syncthreads();
        if (k + 1 <= k1 - 1) {  // bundle k+1's, used by the next iteration
          if (a.has_x) wload_x(k + 3, wxv);
          wload_z(k + 2, wzv);
        }
      }
      if (fix) {
        apply_c(k + 2);
        __syncthreads();
        if (k + 3 <= k1 + 1) load_c(k + 3);  // used by the next iteration
      }
    }
    // every thread is past iteration k-1, the last use of iterate plane k-2 and of
    // coefficient plane k-1, the slots bundle k+LEAD fills
    if (tid == 0 && k + LEAD <= k1 - 1) {
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      issue_bundle(k + LEAD);
    }
    if (k > k0) {
      store(Xs(sx), k - 1);
      prefetch(k);
    }
    const int par = k & 1;
    const int sx1 = sx + 1 < XR ? sx + 1 : 0;
    const int sl1 = sl + 1 < L2R ? sl + 1 : 0;
    const int sc1 = sc + 1 < CR ? sc + 1 : 0;
    red_plane(planes(sx1, sl1, sc1), par ^ 1, k + 1);
    __syncthreads();
    black_plane(planes(sx, sl, sc), par, k);
    sx = sx1;
    sl = sl1;
    sc = sc1;
  }
  __syncthreads();
  store(Xs(sx), k1 - 1);
  }
}

// ---------------------------------------------------------------------------
// Fine residual / divergence pass (3-D, no periodic side), TMA-staged.  Per plane the
// fields go to two rings: "column" fields needed at planes k-1..k+1 (pressure hi/lo,
// z-face coefficients, and in divergence mode the z-velocity) in 4 slots, "plane"
// fields needed only at plane k (right-hand side or x/y velocities, x/y face
// coefficients) in 3 slots; plane k+2 is staged while plane k is computed.  Boxes are
// as tall as each field needs: the pressure with a 1-row halo (rows -1..8), the upper
// faces of y (rows 0..8), everything else the tile's rows 0..7; all 72 wide from
// i0-4.  Each thread computes cells (lane, row) and (lane + 32, row) of the 64 x 8
// tile, so the restriction pairs x neighbours by a shuffle, y neighbours through
// shared memory and z neighbours in registers.  Zero fill supplies L = 0 across the
// walls; the velocity on an upper wall face is the boundary value, patched explicitly.
constexpr int RS_P = 736, RS_8 = 576, RS_9 = 672;  // slot floats: 72 x 10, 72 x 8, 72 x 9 (128-byte multiples)
constexpr int RS_PROWS = TY + 2, RS_8ROWS = TY, RS_9ROWS = TY + 1;
// UNI: tiles outside the band box, whose coefficients are 1 (0 on the walls): the
// coefficient fields are neither staged nor kept.
template <bool DIV, bool DF, bool UNI>
struct ResidLayout {
  // column slot: ph, [pl], L2, [u2]; plane slot: DIV: u0, u1, L0, L1; else z, L0, L1
  static constexpr int oPL = RS_P, oL2 = RS_P * (DF ? 2 : 1), oU2 = oL2 + (UNI ? 0 : RS_8);
  static constexpr int ASZ = oU2 + (DIV ? RS_8 : 0);
  static constexpr int oU0 = 0, oU1 = RS_8, oL0 = DIV ? RS_8 + RS_9 : RS_8, oL1 = oL0 + RS_8, oZ = 0;
  static constexpr int BSZ = UNI ? oL0 : oL1 + RS_9;
  static constexpr int SA = 4, SB = 3, NBAR = 4;
  static constexpr size_t bytes = ((size_t)SA * ASZ + (size_t)SB * BSZ) * sizeof(float);
};

// WRAP (uniform tiles only): the tiles on a periodic x or y side, whose halo cells past
// the side are patched from the wrapped cells (the others' tiles: none).  Planes past a
// periodic z side are staged from their wrapped planes in every variant.
template <bool DIV, bool DF, bool UNI, bool WRAP>
__global__ void __launch_bounds__(256, WRAP ? 4 : UNI ? 5 : 1) k_resid_tma(const __grid_constant__ ResidMaps m,
                                                                             ResidTmaArgs a) {
  static_assert(UNI || !WRAP, "wrapping tiles are uniform");
  using LY = ResidLayout<DIV, DF, UNI>;
  constexpr int SA = LY::SA, SB = LY::SB, NBAR = LY::NBAR;
  extern __shared__ unsigned char smem_raw[];
  float* abase = reinterpret_cast<float*>((reinterpret_cast<uintptr_t>(smem_raw) + 127) & ~uintptr_t(127));
  float* bbase = abase + (size_t)SA * LY::ASZ;
  uint64_t* bars = reinterpret_cast<uint64_t*>(bbase + (size_t)SB * LY::BSZ);
  __shared__ float s_r[8][64];
  __shared__ unsigned s_m[8];
  const Grid& g = a.g;
  const int tid = threadIdx.x, lane = tid & 31, ty = tid >> 5;
  const int i0 = (blockIdx.x + a.t0[0]) * TX, j0 = (blockIdx.y + a.t0[1]) * TY;
  const int kb = (blockIdx.z + a.t0[2]) * a.tz;
  if (i0 >= g.n[0] || j0 >= g.n[1] || kb >= g.n[2]) return;
  const int ke = min(kb + a.tz, g.n[2]);
  if (tile_in_band(a.band, 3, i0, j0, kb, ke) == UNI) return;  // the other variant's tile
  if (UNI && resid_tile_wraps_xy(g, i0, j0) != WRAP) return;    // the other launch's tile
  const bool px = g.per & 1u, py = g.per & 2u, pz = g.per & 4u;
  const int pa_first = kb - 1, pb_first = kb, p_last = ke;
  // column slot / plane slot of plane p (fields at the LY offsets)
  auto A = [&](int p) -> float* { return abase + (size_t)((p - pa_first) % SA) * LY::ASZ; };
  auto B = [&](int p) -> float* { return bbase + (size_t)((p - pb_first) % SB) * LY::BSZ; };
  auto bar = [&](int p) { return smem_addr(&bars[(p - pa_first) % NBAR]); };
  auto phase = [&](int p) { return (uint32_t)(((p - pa_first) / NBAR) & 1); };
  constexpr uint32_t kPB = BX * RS_PROWS * 4, k8B = BX * RS_8ROWS * 4, k9B = BX * RS_9ROWS * 4;

  if (tid == 0) {
    for (int b = 0; b < NBAR; ++b) mbar_init(smem_addr(&bars[b]), 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
  int p_issued = pa_first - 1;
  auto issue = [&](int p) {  // thread 0: stage plane p
    if (p > p_last) return;
    p_issued = p;
    const bool plane = p >= pb_first && p < ke;
    const uint32_t col = (DF ? 2 : 1) * kPB + (UNI ? 0u : k8B) + (DIV ? k8B : 0);
    const uint32_t pln = (DIV ? k8B + k9B : k8B) + (UNI ? 0u : k8B + k9B);
    const uint32_t br = bar(p);
    mbar_expect_tx(br, col + (plane ? pln : 0u));
    const int x = i0 - 4;
    const int pp = pz ? wrap_per(p, g.n[2]) : p;  // a plane past a periodic z side: its wrapped plane
    float* Ap = A(p);
    tma_load(smem_addr(Ap), &m.ph, x, j0 - 1, pp, br, 3);
    if (DF) tma_load(smem_addr(Ap + LY::oPL), &m.pl, x, j0 - 1, pp, br, 3);
    if (!UNI) tma_load(smem_addr(Ap + LY::oL2), &m.L2, x, j0, pp, br, 3);
    if (DIV) tma_load(smem_addr(Ap + LY::oU2), &m.u2, x, j0, pp, br, 3);
    if (plane) {
      float* Bp = B(p);
      if (DIV) {
        tma_load(smem_addr(Bp + LY::oU0), &m.u0, x, j0, p, br, 3);
        tma_load(smem_addr(Bp + LY::oU1), &m.u1, x, j0, p, br, 3);
      } else {
        tma_load(smem_addr(Bp + LY::oZ), &m.z, x, j0, p, br, 3);
      }
      if (!UNI) {
        tma_load(smem_addr(Bp + LY::oL0), &m.L0, x, j0, p, br, 3);
        tma_load(smem_addr(Bp + LY::oL1), &m.L1, x, j0, p, br, 3);
      }
    }
  };
  // WRAP: the halo cells past a periodic x / y side that the stencil reads, which the copy
  // engine zero-fills, hold the wrapped cells' values: the pressure boxes' column 3 / 68
  // (x = -1 / n0; rows 1..8, the tile's rows) and row 0 / 9 (y = -1 / n1; columns 4..67),
  // in divergence mode also the x-velocity box's column 68 and the y-velocity box's row 8
  // (the upper faces at x = n0, y = n1).  Only planes the block computes need them.  The
  // entries form one list (left, right, top, bottom strips); thread t takes entries t
  // and t + 256, each with its shared offset (column slot, or for a velocity the plane
  // slot), its field (0 pressure hi, 1 lo, 2 u_x, 3 u_y) and the wrapped cell's index
  // in its plane.  A plane's values are read from global memory one plane ahead.
  constexpr int NE = 2;
  int we_off[NE], we_f[NE];
  unsigned we_q[NE];
  float we_v[NE];
  if constexpr (WRAP) {
    const int n0 = g.n[0], n1 = g.n[1], nfp = DF ? 2 : 1;
    const bool wl = px && i0 == 0, wr = px && i0 + TX >= n0;
    const bool wt = py && j0 == 0, wb = py && j0 + TY >= n1;
    const int nl = wl ? nfp * TY : 0, nr = wr ? nfp * TY + (DIV ? TY : 0) : 0;
    const int nt = wt ? nfp * TX : 0, nb = wb ? nfp * TX + (DIV ? TX : 0) : 0;
#pragma unroll
    for (int r = 0; r < NE; ++r) {
      int t = tid + 256 * r, off = -1, f = 0;
      unsigned q = 0u;
      if (t < nl) {  // x = -1: cell n0 - 1 of the row
        f = t / TY;
        const int row = t - f * TY;
        off = (f == 1 ? LY::oPL : 0) + (row + 1) * BX + 3;
        q = (unsigned)(n0 - 1) + (unsigned)n0 * (unsigned)(j0 + row);
      } else if ((t -= nl) < nr) {  // x = n0: cell 0 of the row
        f = t / TY;
        const int row = t - f * TY;
        if (f < nfp) {
          off = (f == 1 ? LY::oPL : 0) + (row + 1) * BX + 4 + TX;
        } else {
          f = 2;
          off = LY::oU0 + row * BX + 4 + TX;
        }
        q = (unsigned)n0 * (unsigned)(j0 + row);
      } else if ((t -= nr) < nt) {  // y = -1: row n1 - 1
        f = t / TX;
        const int col = t - f * TX;
        off = (f == 1 ? LY::oPL : 0) + col + 4;
        q = (unsigned)(i0 + col) + (unsigned)n0 * (unsigned)(n1 - 1);
      } else if ((t -= nt) < nb) {  // y = n1: row 0
        f = t / TX;
        const int col = t - f * TX;
        if (f < nfp) {
          off = (f == 1 ? LY::oPL : 0) + (TY + 1) * BX + col + 4;
        } else {
          f = 3;
          off = LY::oU1 + TY * BX + col + 4;
        }
        q = (unsigned)(i0 + col);
      }
      we_off[r] = off;
      we_f[r] = f;
      we_q[r] = q;
      we_v[r] = 0.f;
    }
  }
  auto wload = [&](int p) {  // the patch values of plane p (kb <= p < ke)
    const long long o = (long long)g.n[0] * g.n[1] * p;
#pragma unroll
    for (int r = 0; r < NE; ++r)
      if (we_off[r] >= 0 && wl_in(o + we_q[r], g.nc, WL_DBG_RESID)) we_v[r] = __ldg(a.wsrc[we_f[r]] + o + we_q[r]);
  };
  auto wstore = [&](int p) {
#pragma unroll
    for (int r = 0; r < NE; ++r)
      if (we_off[r] >= 0) (we_f[r] >= 2 ? B(p) : A(p))[we_off[r]] = we_v[r];
  };
  auto bail = [&](int p_fail) {
    if (tid == 0) {
      atomicOr(&a.st->status, 4);
      for (int p = p_fail; p <= p_issued; ++p) mbar_wait(bar(p), phase(p));
    }
    __syncthreads();
  };
  if (tid == 0)
    for (int p = pa_first; p <= min(pa_first + 2, p_last); ++p) issue(p);
  if constexpr (WRAP) wload(kb);  // plane kb's patches, read while its copies are in flight
  for (int p = pa_first; p <= kb; ++p) {
    const bool ok = mbar_wait(bar(p), phase(p));
    if (__syncthreads_or(!ok)) return bail(p);
  }
  if constexpr (WRAP) {
    wstore(kb);  // read from the next iteration on, after its barrier
    if (kb + 1 < ke) wload(kb + 1);
  }
  const float inv = DIV ? a.inv_w * a.st->inv_dtf : 0.f;
  unsigned mbits = 0u;
  float vpair[2] = {0.f, 0.f};
  for (int k = kb; k < ke; ++k) {
    {
      const bool ok = mbar_wait(bar(k + 1), phase(k + 1));
      if (__syncthreads_or(!ok)) return bail(k + 1);
    }
    if constexpr (WRAP) {
      // plane k+1's halo (computed next iteration, after its barrier); plane k's compute
      // below reads only plane k+1's own cells
      if (k + 1 < ke) wstore(k + 1);
      if (k + 2 < ke) wload(k + 2);
    }
    // every thread is past plane k-2's column fields and plane k-1's plane fields
    if (tid == 0) {
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      issue(k + 2);
    }
    const float* A0 = A(k);
    const float* Am = A(k - 1);
    const float* Ap = A(k + 1);
    const float* B0 = B(k);
    const float* ph0 = A0;
    const float* pl0 = A0 + LY::oPL;
    const float* phm = Am;
    const float* plm = Am + LY::oPL;
    const float* php = Ap;
    const float* plp = Ap + LY::oPL;
    const float* L0 = B0 + LY::oL0;
    const float* L1 = B0 + LY::oL1;
    const float* L2 = A0 + LY::oL2;
    const float* L2u = Ap + LY::oL2;
    const int gj = j0 + ty;
    // this thread's cells (lane, ty) and (lane + 32, ty): right-hand side, face
    // coefficients (x up/down, y up/down, z up/down) and whether the cell exists
    float zv[2], cf[2][6];
    bool inb[2];
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int ii = lane + 32 * h;
      const int gi = i0 + ii;
      const int c = ty * BX + ii + 4;  // the boxes other than the pressure (from row 0)
      const bool in = gi < g.n[0] && gj < g.n[1];
      inb[h] = in;
      if (DIV) {
        const float* U0 = B0 + LY::oU0;
        const float* U1 = B0 + LY::oU1;
        const float uxp = (gi + 1 < g.n[0] || px)
                              ? U0[c + 1]
                              : ((a.uxe && in) ? __ldg(a.uxe + gj + (long long)g.n[1] * k) : g.U[0]);
        const float uyp = (gj + 1 < g.n[1] || py) ? U1[c + BX] : g.U[1];
        const float uzp = (k + 1 < g.n[2] || pz) ? (Ap + LY::oU2)[c] : g.U[2];
        float div = 0.f;
        div += uxp - U0[c];
        div += uyp - U1[c];
        div += uzp - (A0 + LY::oU2)[c];
        zv[h] = div * inv;
        const long long qz = (long long)gi + (long long)g.n[0] * ((long long)gj + (long long)g.n[1] * k);
        if (in && wl_in(qz, g.nc, WL_DBG_RESID)) a.z[qz] = zv[h];
      } else {
        zv[h] = (B0 + LY::oZ)[c];
      }
      // face coefficients: staged, or (UNI) 1 inside the grid and 0 across a wall
      if (UNI) {
        cf[h][0] = (gi + 1 < g.n[0] || px) ? 1.f : 0.f;
        cf[h][1] = (gi > 0 || px) ? 1.f : 0.f;
        cf[h][2] = (gj + 1 < g.n[1] || py) ? 1.f : 0.f;
        cf[h][3] = (gj > 0 || py) ? 1.f : 0.f;
        cf[h][4] = (k + 1 < g.n[2] || pz) ? 1.f : 0.f;
        cf[h][5] = (k > 0 || pz) ? 1.f : 0.f;
      } else {
        cf[h][0] = L0[c + 1];
        cf[h][1] = L0[c];
        cf[h][2] = L1[c + BX];
        cf[h][3] = L1[c];
        cf[h][4] = L2u[c];
        cf[h][5] = L2[c];
      }
    }
    const int e0 = (ty + 1) * BX + lane + 4;  // pressure boxes (from row -1); the second cell is 32 further
    float rr[2];
    if (DF) {
      // both cells at once in packed FP32 pairs (each lane rounds as the scalar
      // operation would: the same error-free transformations, the same bits)
      auto P2 = [&](const float* f, int o) { return make_float2(f[e0 + o], f[e0 + 32 + o]); };
      auto C2 = [&](int t) { return make_float2(cf[0][t], cf[1][t]); };
      const float2 h0 = P2(ph0, 0), l0 = P2(pl0, 0);
      const float2 Lc[6] = {C2(0), C2(1), C2(2), C2(3), C2(4), C2(5)};
      const float2 hn[6] = {P2(ph0, 1), P2(ph0, -1), P2(ph0, BX), P2(ph0, -BX), P2(php, 0), P2(phm, 0)};
      const float2 ln[6] = {P2(pl0, 1), P2(pl0, -1), P2(pl0, BX), P2(pl0, -BX), P2(plp, 0), P2(plm, 0)};
      // a cell whose face coefficients are all 1 or 0 (every uniform-tile cell, and most of
      // a band tile's) takes the short form; the choice is the cell's own, so every kernel
      // gives a cell the same bits (a missing neighbour across a wall reads 0 with a 0
      // coefficient: adds exactly 0)
      auto unit = [&](int h) {
        bool ok = true;
#pragma unroll
        for (int t = 0; t < 6; ++t) ok = ok && (cf[h][t] == 0.f || cf[h][t] == 1.f);
        return ok;
      };
      const bool q0 = UNI || unit(0), q1 = UNI || unit(1);
      float2 rf = make_float2(0.f, 0.f), rg = make_float2(0.f, 0.f);
      if (q0 || q1) {
        // short form: the present neighbours' pressures summed in double-float, minus
        // nf p0 (nf faces, a small integer: nf h0 exact by TwoProd)
        float2 S = mul2(Lc[0], hn[0]), Se = make_float2(0.f, 0.f), Sl = mul2(Lc[0], ln[0]);
        float2 nf = Lc[0];
#pragma unroll
        for (int f = 1; f < 6; ++f) {
          float2 e;
          two_sum2(S, mul2(Lc[f], hn[f]), S, e);
          Se = add2(Se, e);
          Sl = fma2(Lc[f], ln[f], Sl);
          nf = add2(nf, Lc[f]);
        }
        float2 T, Te, Dh, Dl, rh, rl;
        two_prod2(nf, h0, T, Te);
        Te = fma2(nf, l0, Te);
        two_sum2(S, neg2(T), Dh, Dl);
        Dl = add2(Dl, sub2(add2(Se, Sl), Te));
        two_sum2(make_float2(zv[0], zv[1]), neg2(Dh), rh, rl);
        rf = add2(rh, sub2(rl, Dl));
      }
      if (!UNI && !(q0 && q1)) {
        // general form, face by face: the exact difference to the neighbour times its
        // coefficient (TwoSum, TwoProd), accumulated in double-float
        float2 ah = make_float2(0.f, 0.f), al = make_float2(0.f, 0.f);
#pragma unroll
        for (int f = 0; f < 6; ++f) {
          float2 dh, dl, th, tl, sh, sl;
          two_sum2(hn[f], neg2(h0), dh, dl);
          dl = add2(dl, sub2(ln[f], l0));
          two_prod2(Lc[f], dh, th, tl);
          tl = fma2(Lc[f], dl, tl);
          two_sum2(ah, th, sh, sl);
          ah = sh;
          al = add2(al, add2(sl, tl));
        }
        float2 rh, rl;
        two_sum2(make_float2(zv[0], zv[1]), neg2(ah), rh, rl);
        rg = add2(rh, sub2(rl, al));
      }
      rr[0] = q0 ? rf.x : rg.x;
      rr[1] = q1 ? rf.y : rg.y;
    } else {
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const int e = e0 + 32 * h;
        const float x0 = ph0[e];
        float acc = 0.f;
        acc += cf[h][0] * (ph0[e + 1] - x0) + cf[h][1] * (ph0[e - 1] - x0);
        acc += cf[h][2] * (ph0[e + BX] - x0) + cf[h][3] * (ph0[e - BX] - x0);
        acc += cf[h][4] * (php[e] - x0) + cf[h][5] * (phm[e] - x0);
        rr[h] = zv[h] - acc;
      }
    }
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int gi = i0 + lane + 32 * h;
      float r = rr[h];
      if (inb[h]) {
        const long long qr = (long long)gi + (long long)g.n[0] * ((long long)gj + (long long)g.n[1] * k);
        if (a.rout && wl_in(qr, g.nc, WL_DBG_RESID)) a.rout[qr] = r;
        mbits = max(mbits, __float_as_uint(fabsf(r)));
      } else {
        r = 0.f;
      }
      vpair[h] = ((k - kb) & 1) ? vpair[h] + r : r;
    }
    // restriction of each plane pair: x pairs by shuffle, y pairs in shared memory
    if (a.zc && ((k - kb) & 1)) {
#pragma unroll
      for (int h = 0; h < 2; ++h) s_r[ty][lane + 32 * h] = vpair[h] + __shfl_xor_sync(0xffffffffu, vpair[h], 1);
      __syncthreads();
      if (tid < 128) {
        const int cx = tid & 31, cy = tid >> 5;
        const float sum = s_r[2 * cy][2 * cx] + s_r[2 * cy + 1][2 * cx];
        const int I = (i0 >> 1) + cx, J = (j0 >> 1) + cy, K = k >> 1;
        const long long qc = (long long)I + (long long)a.cn[0] * ((long long)J + (long long)a.cn[1] * K);
        if (I < a.cn[0] && J < a.cn[1] && K < a.cn[2] &&
            wl_in(qc, (long long)a.cn[0] * a.cn[1] * a.cn[2], WL_DBG_RESID))
          st_st(a.zc, a.zctype, qc, sum * a.zcmul);
      }
    }
    __syncthreads();
  }
  const unsigned mb = block_max_bits<256>(mbits, s_m);
  if (tid == 0 && mb) atomicMax(&a.st->norm_bits, mb);
}

// Self-test of the bounded wait: one thread waits on an mbarrier that nothing
// arrives at, so the wait has to give up after limit_ns; *gave_up records it.
__global__ void k_wait_probe(uint64_t limit_ns, int* gave_up) {
  __shared__ uint64_t bar;
  if (threadIdx.x == 0) {
    mbar_init(smem_addr(&bar), 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    *gave_up = mbar_wait(smem_addr(&bar), 0, limit_ns) ? 0 : 1;
  }
}

int launch_wait_probe(uint64_t limit_ns, int* gave_up, cudaStream_t s) {
  k_wait_probe<<<1, 32, 0, s>>>(limit_ns, gave_up);
  return 0;
}

// tiles [lo, hi) along one direction whose footprint [t*w - pad_lo, t*w + w + pad_hi)
// (clamped by n for the z march) meets the band box [blo, bhi)
static void band_tiles(int n, int w, int pad, int blo, int bhi, int& lo, int& hi) {
  const int nt = (n + w - 1) / w;
  lo = nt;
  hi = 0;
  for (int t = 0; t < nt; ++t) {
    const int a0 = t * w, a1 = std::min(a0 + w, n);
    if (a0 - pad < bhi && a1 + pad > blo) {
      lo = std::min(lo, t);
      hi = t + 1;
    }
  }
}

double band_tile_fraction(int D, const Grid& g, int tz, const BandBox& b, int ty) {
  int lo[3], hi[3];
  band_tiles(g.n[0], TX, 4, b.lo[0], b.hi[0], lo[0], hi[0]);
  band_tiles(g.n[1], ty, 2, b.lo[1], b.hi[1], lo[1], hi[1]);
  if (D == 3)
    band_tiles(g.n[2], tz, 2, b.lo[2], b.hi[2], lo[2], hi[2]);
  else {
    lo[2] = 0;
    hi[2] = 1;
  }
  const double all = (double)((g.n[0] + TX - 1) / TX) * ((g.n[1] + ty - 1) / ty) *
                     (D == 3 ? (g.n[2] + tz - 1) / tz : 1);
  double band = 1.0;
  for (int d = 0; d < 3; ++d) band *= std::max(0, hi[d] - lo[d]);
  return band / all;
}

template <bool DIV, bool DF, bool UNI, bool WRAP>
void launch_resid_tma_v(const ResidMaps& m, const ResidTmaArgs& a, dim3 grd, cudaStream_t s) {
  const size_t smem = ResidLayout<DIV, DF, UNI>::bytes + ResidLayout<DIV, DF, UNI>::NBAR * sizeof(uint64_t) + 128;
  static bool attr = false;
  if (!attr) {
    cudaFuncSetAttribute(k_resid_tma<DIV, DF, UNI, WRAP>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    cudaFuncSetAttribute(k_resid_tma<DIV, DF, UNI, WRAP>, cudaFuncAttributePreferredSharedMemoryCarveout,
                         (int)cudaSharedmemCarveoutMaxShared);
    attr = true;
  }
  k_resid_tma<DIV, DF, UNI, WRAP><<<grd, 256, smem, s>>>(m, a);
}
template <bool UNI, bool WRAP>
void launch_resid_tma_w(const ResidMaps& m, const ResidTmaArgs& a, dim3 grd, cudaStream_t s) {
  if (a.div && a.df)
    launch_resid_tma_v<true, true, UNI, WRAP>(m, a, grd, s);
  else if (a.div)
    launch_resid_tma_v<true, false, UNI, WRAP>(m, a, grd, s);
  else if (a.df)
    launch_resid_tma_v<false, true, UNI, WRAP>(m, a, grd, s);
  else
    launch_resid_tma_v<false, false, UNI, WRAP>(m, a, grd, s);
}
// the loading tiles, or the uniform ones (with a second launch for the tiles on a
// periodic x / y side)
template <bool UNI>
void launch_resid_tma_u(const ResidMaps& m, const ResidTmaArgs& a, dim3 grd, cudaStream_t s) {
  launch_resid_tma_w<UNI, false>(m, a, grd, s);
  if (UNI && (a.g.per & 3u)) launch_resid_tma_w<true, true>(m, a, grd, s);
}

bool resid_band_wraps(const Grid& g, int tz, const BandBox& b) {
  if (!(g.per & 3u)) return false;
  if (!b.on) return true;  // every tile loads its coefficients
  int lo[3], hi[3];
  band_tiles(g.n[0], TX, 4, b.lo[0], b.hi[0], lo[0], hi[0]);
  band_tiles(g.n[1], TY, 2, b.lo[1], b.hi[1], lo[1], hi[1]);
  band_tiles(g.n[2], tz, 2, b.lo[2], b.hi[2], lo[2], hi[2]);
  if (hi[0] <= lo[0] || hi[1] <= lo[1] || hi[2] <= lo[2]) return false;
  for (int tj = lo[1]; tj < hi[1]; ++tj)
    for (int ti = lo[0]; ti < hi[0]; ++ti)
      if (resid_tile_wraps_xy(g, ti * TX, tj * TY)) return true;
  return false;
}

int launch_resid_tma(const ResidMaps& m, const ResidTmaArgs& a0, cudaStream_t s, const SideStream* side) {
  const Grid& g = a0.g;
  ResidTmaArgs a = a0;
  a.t0[0] = a.t0[1] = a.t0[2] = 0;
  const dim3 full((g.n[0] + TX - 1) / TX, (g.n[1] + TY - 1) / TY, (g.n[2] + a.tz - 1) / a.tz);
  if (!a.band.on) {
    launch_resid_tma_u<false>(m, a, full, s);
    return 0;
  }
  int lo[3], hi[3];
  band_tiles(g.n[0], TX, 4, a.band.lo[0], a.band.hi[0], lo[0], hi[0]);
  band_tiles(g.n[1], TY, 2, a.band.lo[1], a.band.hi[1], lo[1], hi[1]);
  band_tiles(g.n[2], a.tz, 2, a.band.lo[2], a.band.hi[2], lo[2], hi[2]);
  if (hi[0] <= lo[0] || hi[1] <= lo[1] || hi[2] <= lo[2]) {
    launch_resid_tma_u<true>(m, a, full, s);
    return 0;
  }
  ResidTmaArgs b = a;
  for (int d = 0; d < 3; ++d) b.t0[d] = lo[d];
  const dim3 grd(hi[0] - lo[0], hi[1] - lo[1], hi[2] - lo[2]);
  if (side) {  // the band tiles beside the uniform ones
    cudaEventRecord(side->fork, s);
    cudaStreamWaitEvent(side->aux, side->fork, 0);
    if (side->hook) side->hook(side->ctx, 1, 1, side->aux);
    launch_resid_tma_u<false>(m, b, grd, side->aux);
    if (side->hook) side->hook(side->ctx, 1, 0, side->aux);
    if (side->hook) side->hook(side->ctx, 0, 1, s);
    launch_resid_tma_u<true>(m, a, full, s);
    if (side->hook) side->hook(side->ctx, 0, 0, s);
    cudaEventRecord(side->join, side->aux);
    cudaStreamWaitEvent(s, side->join, 0);
  } else {
    launch_resid_tma_u<false>(m, b, grd, s);
    launch_resid_tma_u<true>(m, a, full, s);
  }
  return 0;
}

template <int TYV>
size_t sweep_tma_smem(bool uni) {
  using G = SwGeom<TYV>;
  const size_t rings = uni ? (size_t)XR * G::BOX + (size_t)CR * G::CSLOT
                           : (size_t)XR * G::BOX + (size_t)L2R * G::CSLOT + (size_t)CR * (2 * G::CSLOT + G::L1SLOT);
  return rings * sizeof(float) + (1 + NBB) * sizeof(uint64_t) + 128;
}

template <int D, bool UNI, bool WRAP, int TYV>
void launch_sweep_tma_t(const SweepMaps& m, const SweepTmaArgs& a, dim3 grd, cudaStream_t s) {
  const size_t smem = sweep_tma_smem<TYV>(UNI);
  static bool attr = false;
  if (!attr) {  // all of the unified L1/shared storage as shared memory: the blocks per SM are smem-bound
    cudaFuncSetAttribute(k_sweep_tma<D, UNI, WRAP, TYV>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    cudaFuncSetAttribute(k_sweep_tma<D, UNI, WRAP, TYV>, cudaFuncAttributePreferredSharedMemoryCarveout,
                         (int)cudaSharedmemCarveoutMaxShared);
    attr = true;
  }
  k_sweep_tma<D, UNI, WRAP, TYV><<<grd, SW_NT, smem, s>>>(m, a);
}
// tile height 16 (3-D, plain tiles only) or 8
template <int D, bool UNI, bool WRAP = false>
void launch_sweep_tma_v(const SweepMaps& m, const SweepTmaArgs& a, dim3 grd, cudaStream_t s) {
  if constexpr (D == 3 && !WRAP) {
    if (a.ty == SWEEP_TY16) return launch_sweep_tma_t<D, UNI, WRAP, SWEEP_TY16>(m, a, grd, s);
  }
  launch_sweep_tma_t<D, UNI, WRAP, 8>(m, a, grd, s);
}

namespace {

// The tiles that cross no periodic side: those meeting the level's band box run the
// loading kernel, the others the uniform one; without a split every tile loads its
// coefficients.
void launch_plain(int D, const SweepMaps& m, const SweepTmaArgs& a0, cudaStream_t s, const SideStream* side) {
  const Grid& g = a0.g;
  const int tz = D == 3 ? a0.tz : 1;
  const int ty = (D == 3 && a0.ty == SWEEP_TY16) ? SWEEP_TY16 : TY;
  const dim3 full((g.n[0] + TX - 1) / TX, (g.n[1] + ty - 1) / ty, D == 3 ? (g.n[2] + tz - 1) / tz : 1);
  SweepTmaArgs a = a0;
  a.ty = ty;
  a.t0[0] = a.t0[1] = a.t0[2] = 0;
  if (!a.band.on) {
    if (D == 3)
      launch_sweep_tma_v<3, false>(m, a, full, s);
    else
      launch_sweep_tma_v<2, false>(m, a, full, s);
    return;
  }
  auto uni = [&](cudaStream_t st) {
    if (D == 3)
      launch_sweep_tma_v<3, true>(m, a, full, st);
    else
      launch_sweep_tma_v<2, true>(m, a, full, st);
  };
  int lo[3], hi[3];
  band_tiles(g.n[0], TX, 4, a.band.lo[0], a.band.hi[0], lo[0], hi[0]);
  band_tiles(g.n[1], ty, 2, a.band.lo[1], a.band.hi[1], lo[1], hi[1]);
  if (D == 3)
    band_tiles(g.n[2], tz, 2, a.band.lo[2], a.band.hi[2], lo[2], hi[2]);
  else {
    lo[2] = 0;
    hi[2] = 1;
  }
  if (hi[0] <= lo[0] || hi[1] <= lo[1] || hi[2] <= lo[2]) {
    uni(s);
    return;
  }
  SweepTmaArgs b = a;
  for (int d = 0; d < 3; ++d) b.t0[d] = lo[d];
  const dim3 grd(hi[0] - lo[0], hi[1] - lo[1], hi[2] - lo[2]);
  auto band = [&](cudaStream_t st) {
    if (D == 3)
      launch_sweep_tma_v<3, false>(m, b, grd, st);
    else
      launch_sweep_tma_v<2, false>(m, b, grd, st);
  };
  if (side) {  // the band tiles beside the uniform ones
    cudaEventRecord(side->fork, s);
    cudaStreamWaitEvent(side->aux, side->fork, 0);
    if (side->hook) side->hook(side->ctx, 1, 1, side->aux);
    band(side->aux);
    if (side->hook) side->hook(side->ctx, 1, 0, side->aux);
    if (side->hook) side->hook(side->ctx, 0, 1, s);
    uni(s);
    if (side->hook) side->hook(side->ctx, 0, 0, s);
    cudaEventRecord(side->join, side->aux);
    cudaStreamWaitEvent(s, side->join, 0);
  } else {
    band(s);
    uni(s);
  }
}

}  // namespace

int launch_sweep_tma(int D, const SweepMaps& m, const SweepTmaArgs& a0, cudaStream_t s, const SideStream* side) {
  if (a0.plain) launch_plain(D, m, a0, s, side);
  if (a0.wrap) {  // the tiles across a periodic x / y side (all uniform), after the others
    const Grid& g = a0.g;
    const int tz = D == 3 ? a0.tzw : 1;
    const dim3 full((g.n[0] + TX - 1) / TX, (g.n[1] + TY - 1) / TY, D == 3 ? (g.n[2] + tz - 1) / tz : 1);
    SweepTmaArgs a = a0;
    a.tz = tz;
    a.t0[0] = a.t0[1] = a.t0[2] = 0;
    if (D == 3)
      launch_sweep_tma_v<3, true, true>(m, a, full, s);
    else
      launch_sweep_tma_v<2, true, true>(m, a, full, s);
  }
  return 0;
}

}  // namespace wl

namespace wl {
unsigned dbg_take_sweep() {
#ifdef WL_DEBUG_BOUNDS
  unsigned v = 0, z = 0;
  cudaMemcpyFromSymbol(&v, wl_dbg_bits, sizeof(v));
  cudaMemcpyToSymbol(wl_dbg_bits, &z, sizeof(z));
  return v;
#else
  return 0u;
#endif
}
}  // namespace wl
