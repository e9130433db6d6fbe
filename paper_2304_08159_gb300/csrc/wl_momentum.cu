// Momentum stage kernels: convdiff! fused with BDIM! and BC! (Table 2).
//
// One Heun stage (Section 2: explicit adaptive time stepping; the Heun form is this
// library's reading):
//   stage 1: f = u0 + dt r(u0),  u' = mu0 f + mu1 . grad f
//   stage 2: f = u0 + dt r(u'),  u  = (u' + mu0 f + mu1 . grad f) / 2
// with r(u)_c[I] = sum_j F_cj[I] - F_cj[I+e_j] the finite-volume convection-diffusion
// residual and (mu0, mu1) the BDIM moments (Section 2, Weymouth & Yue 2011).  The
// body velocity is zero.  k_stage computes everything but the mu1 term, which is
// non-zero only in the thin band |d| < eps around the body and is added by
// k_bdim_band over the body's bounding box.
#include <algorithm>
#include <cstdlib>
#include <type_traits>

#include "wl_dev.cuh"
#include "wl_kernels.h"
#include "wl_stage_dev.cuh"

namespace wl {

constexpr int ST_TX = 32, ST_TY = 8, ST_TZ = 32;
constexpr int ST_HX = ST_TX + 4, ST_HY = ST_TY + 4;
template <int N>
using IC = std::integral_constant<int, N>;

// Tile of ST_TX x ST_TY columns marching upward through ST_TZ planes.  The velocity
// of planes k-1..k+2 (with a 2-cell in-plane halo) sits in a 4-plane shared ring;
// plane k+3 is loaded into registers while plane k is computed.
// Each thread computes the lower x-, y- and z-face fluxes of its cell; the upper x/y
// fluxes come from the neighbour through shared memory, the upper z flux is carried
// in registers to the next plane, so every face flux is evaluated once.  The plane loop
// is unrolled by the ring's length, so every ring slot, and with it every shared
// operand offset, is a compile-time constant.
template <int D>
__device__ __forceinline__ void stage_body(const StageArgs& a, const uint3 bid) {
  constexpr int NP = (D == 3) ? 4 : 1;
  constexpr int HX = ST_HX, PL = ST_HY * ST_HX, NE = PL;
  __shared__ float s_u[D * NP * PL];
  __shared__ float s_fx[D][ST_TY][ST_TX + 1];
  __shared__ float s_fy[D][ST_TY + 1][ST_TX];
  const Grid& g = a.g;
  const int tid = threadIdx.x, tx = tid % ST_TX, ty = tid / ST_TX, warp = tid >> 5, lane = tid & 31;
  const int i0 = bid.x * ST_TX, j0 = bid.y * ST_TY;
  const int k0 = (D == 3) ? bid.z * ST_TZ : 0;
  const int k1 = (D == 3) ? min(k0 + ST_TZ, g.n[2]) : 1;
  const int i = i0 + tx, j = j0 + ty;
  const bool own_cell = (i < g.n[0]) && (j < g.n[1]);
  const float dt = *a.dt;
  const bool adv = a.advect != 0;
  const float nu = a.nu;
  // this tile overlaps the body's band box: its faces there keep f for the mu1 term
  const bool box_tile = a.fbox && i0 < a.blo[0] + a.bn[0] && i0 + ST_TX > a.blo[0] && j0 < a.blo[1] + a.bn[1] &&
                        j0 + ST_TY > a.blo[1] && k0 < a.blo[2] + a.bn[2] && k1 > a.blo[2];
  // component c of ring slot sl starts at soff(c, sl); a tile position (ii, jj) adds
  // (jj + 2) * HX + ii + 2.  Plane kk lives in slot (kk - k0 + 2) mod NP.
  auto soff = [](int c, int sl) { return (c * NP + sl) * PL; };

  // A plane of the velocity (2-cell in-plane halo) moves in two steps: fetch() loads
  // this thread's elements e = tid, tid + 256 (at most two per component) into
  // registers, commit() stores them into the plane's ring slot, so the loads of plane
  // k+3 are in flight while the fluxes of plane k are formed.
  const bool xy_inner = (i0 >= 2) && (i0 + ST_TX + 2 <= g.n[0]) && (j0 >= 2) && (j0 + ST_TY + 2 <= g.n[1]);
  const long long nxy = (long long)g.n[0] * g.n[1];
  const long long fbase = (long long)(i0 - 2) + (long long)g.n[0] * (j0 - 2);  // halo origin (inner tiles)
  int foff[2];  // element offsets from it
#pragma unroll
  for (int h = 0; h < 2; ++h) {
    const int e = tid + 256 * h, row = e / HX;
    foff[h] = (e - row * HX) + g.n[0] * row;
  }
  float rv[2][D];
  auto fetch = [&](int kk) {
    const bool inner = xy_inner && (D == 2 || (kk >= 0 && kk < g.n[2]));
    const long long qk = fbase + ((D == 3) ? nxy * kk : 0);
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int e = tid + 256 * h;
      if (e >= NE) break;
      if (inner) {
#pragma unroll
        for (int c = 0; c < D; ++c)
          rv[h][c] = wl_in(qk + foff[h], g.nc, WL_DBG_STAGE) ? __ldg(a.u[c] + qk + foff[h]) : 0.f;
      } else {
        const int row = e / HX, col = e - row * HX;
#pragma unroll
        for (int c = 0; c < D; ++c) rv[h][c] = load_u_bc<D>(a.u[c], c, g, i0 - 2 + col, j0 - 2 + row, kk);
      }
    }
  };
  auto commit = [&](int sl) {
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int e = tid + 256 * h;
      if (e >= NE) break;
#pragma unroll
      for (int c = 0; c < D; ++c) s_u[soff(c, sl) + e] = rv[h][c];
    }
  };

  // Lower-face fluxes of the u_c control volume at tile position pos, with plane k in
  // slot S (and k-1 in SM, whose u_x / u_y advect u_z across the x / y faces).
  auto flux_x = [&](auto C, auto S, auto SM, int pos) -> float {
    constexpr int c = decltype(C)::value, s = decltype(S)::value, sm = decltype(SM)::value;
    const float* U = s_u + soff(c, s) + pos;
    const float* A = s_u + soff(0, s) + pos;
    const float a2 = A[0] + (c == 0 ? A[-1] : (c == 1 ? A[-HX] : s_u[soff(0, sm) + pos]));
    return mom_flux(U[-2], U[-1], U[0], U[1], a2, nu, adv);
  };
  auto flux_y = [&](auto C, auto S, auto SM, int pos) -> float {
    constexpr int c = decltype(C)::value, s = decltype(S)::value, sm = decltype(SM)::value;
    const float* U = s_u + soff(c, s) + pos;
    const float* A = s_u + soff(1, s) + pos;
    const float a2 = A[0] + (c == 0 ? A[-1] : (c == 1 ? A[-HX] : s_u[soff(1, sm) + pos]));
    return mom_flux(U[-2 * HX], U[-HX], U[0], U[HX], a2, nu, adv);
  };
  // lower z-face flux at plane kf, planes kf-2 .. kf+1 in slots Q0 .. Q3
  auto flux_z = [&](auto C, auto Q0, auto Q1, auto Q2, auto Q3, int pos) -> float {
    constexpr int c = decltype(C)::value, q0 = decltype(Q0)::value, q1 = decltype(Q1)::value,
                  q2 = decltype(Q2)::value, q3 = decltype(Q3)::value;
    const float* A = s_u + soff(2, q2) + pos;  // u_z at plane kf
    const float a2 = A[0] + (c == 0 ? A[-1] : (c == 1 ? A[-HX] : s_u[soff(2, q1) + pos]));
    return mom_flux(s_u[soff(c, q0) + pos], s_u[soff(c, q1) + pos], s_u[soff(c, q2) + pos], s_u[soff(c, q3) + pos],
                    a2, nu, adv);
  };
  const int own = (ty + 2) * HX + (tx + 2);
  const long long qij = own_cell ? (long long)i + (long long)g.n[0] * j : 0;

  float fzl[3] = {0.f, 0.f, 0.f};
  if constexpr (D == 3) {
    // planes k0-2 .. k0+1 in slots 0 .. 3
    for (int t = 0; t < 4; ++t) {
      fetch(k0 - 2 + t);
      commit(t);
    }
    fetch(k0 + 2);
    __syncthreads();
    fzl[0] = flux_z(IC<0>{}, IC<0>{}, IC<1>{}, IC<2>{}, IC<3>{}, own);
    fzl[1] = flux_z(IC<1>{}, IC<0>{}, IC<1>{}, IC<2>{}, IC<3>{}, own);
    fzl[2] = flux_z(IC<2>{}, IC<0>{}, IC<1>{}, IC<2>{}, IC<3>{}, own);
    __syncthreads();
  }

  // plane k, with k - k0 = PH (mod NP): plane k+t sits in slot (PH + t + 2) mod NP
  auto step = [&](auto PHc, int k) {
    constexpr int PH = decltype(PHc)::value;
    constexpr int S0 = (PH + 2) % NP, SM1 = (PH + 1) % NP;
    [[maybe_unused]] constexpr int SP1 = (PH + 3) % NP, SP2 = PH % NP;
    using I0 = IC<S0>;
    using Im = IC<SM1>;
    // plane k+2 into the slot of plane k-2 (last read by the z fluxes of face k)
    if constexpr (D == 3) {
      commit(SP2);
    } else {
      fetch(0);
      commit(0);
    }
    __syncthreads();
    // in flight while the fluxes are formed: plane k+3 (the last plane used is k1+1),
    // and this cell's mu0 and stage-1 velocity
    if (D == 3 && k + 3 <= k1 + 1) fetch(k + 3);
    const long long qg = qij + (D == 3 ? nxy * k : 0);
    float m0[D], u0v[D];
#pragma unroll
    for (int c = 0; c < D; ++c) {
      m0[c] = own_cell ? __ldg(a.mu0[c] + qg) : 0.f;
      u0v[c] = (own_cell && a.stage != 1) ? __ldg(a.u0[c] + qg) : 0.f;
    }
    float fzu[3] = {0.f, 0.f, 0.f};
    s_fx[0][ty][tx] = flux_x(IC<0>{}, I0{}, Im{}, own);
    s_fy[0][ty][tx] = flux_y(IC<0>{}, I0{}, Im{}, own);
    s_fx[1][ty][tx] = flux_x(IC<1>{}, I0{}, Im{}, own);
    s_fy[1][ty][tx] = flux_y(IC<1>{}, I0{}, Im{}, own);
    if constexpr (D == 3) {
      s_fx[2][ty][tx] = flux_x(IC<2>{}, I0{}, Im{}, own);
      s_fy[2][ty][tx] = flux_y(IC<2>{}, I0{}, Im{}, own);
      // face k+1: planes k-1 .. k+2
      fzu[0] = flux_z(IC<0>{}, Im{}, I0{}, IC<SP1>{}, IC<SP2>{}, own);
      fzu[1] = flux_z(IC<1>{}, Im{}, I0{}, IC<SP1>{}, IC<SP2>{}, own);
      fzu[2] = flux_z(IC<2>{}, Im{}, I0{}, IC<SP1>{}, IC<SP2>{}, own);
    }
    // fluxes through the upper edge faces of the tile: the x edge (D x ST_TY faces) on
    // warp 0, the y edge of component c (ST_TX faces) on warp c + 1
    if (warp == 0) {
      if (lane < D * ST_TY) {
        const int c = lane / ST_TY, row = lane - c * ST_TY, pos = (row + 2) * HX + ST_TX + 2;
        const float f = c == 0 ? flux_x(IC<0>{}, I0{}, Im{}, pos)
                               : (c == 1 ? flux_x(IC<1>{}, I0{}, Im{}, pos) : flux_x(IC<D - 1>{}, I0{}, Im{}, pos));
        s_fx[c][row][ST_TX] = f;
      }
    } else if (warp <= D) {
      const int pos = (ST_TY + 2) * HX + lane + 2;
      if (warp == 1)
        s_fy[0][ST_TY][lane] = flux_y(IC<0>{}, I0{}, Im{}, pos);
      else if (warp == 2)
        s_fy[1][ST_TY][lane] = flux_y(IC<1>{}, I0{}, Im{}, pos);
      else
        s_fy[D - 1][ST_TY][lane] = flux_y(IC<D - 1>{}, I0{}, Im{}, pos);
    }
    __syncthreads();
    if (own_cell) {
      const int I[3] = {i, j, k};
#pragma unroll
      for (int c = 0; c < D; ++c) {
        float r = (s_fx[c][ty][tx] - s_fx[c][ty][tx + 1]) + (s_fy[c][ty][tx] - s_fy[c][ty + 1][tx]);
        if (D == 3) r += fzl[c] - fzu[c];
        const bool upd = is_per(g, c) || I[c] >= 1;
        float ov, f = g.U[c];
        if (!upd) {
          ov = g.U[c];
        } else {
          const float uc = s_u[soff(c, S0) + own];
          const float u0 = (a.stage == 1) ? uc : u0v[c];
          f = fmaf(dt, r, u0);
          const float m = m0[c];
          ov = (a.stage == 1) ? m * f : 0.5f * fmaf(m, f, uc);
        }
        if (wl_in(qg, g.nc, WL_DBG_STAGE)) a.out[c][qg] = ov;
        if (box_tile) {  // keep f inside the body's band box for the mu1 term
          const unsigned bi = (unsigned)(i - a.blo[0]), bj = (unsigned)(j - a.blo[1]), bk = (unsigned)(k - a.blo[2]);
          if (bi < (unsigned)a.bn[0] && bj < (unsigned)a.bn[1] && bk < (unsigned)a.bn[2])
          {
            const long long fi = (long long)c * a.bn[0] * a.bn[1] * a.bn[2] + bi + (long long)a.bn[0] * (bj + (long long)a.bn[1] * bk);
            if (wl_in(fi, g.nc, WL_DBG_BAND)) a.fbox[fi] = f;
          }
        }
      }
    }
#pragma unroll
    for (int c = 0; c < D; ++c) fzl[c] = fzu[c];
  };
  if constexpr (D == 3) {
    for (int kb = k0; kb < k1; kb += NP) {
      step(IC<0>{}, kb);
      if (kb + 1 < k1) step(IC<1>{}, kb + 1);
      if (kb + 2 < k1) step(IC<2>{}, kb + 2);
      if (kb + 3 < k1) step(IC<3>{}, kb + 3);
    }
  } else {
    step(IC<0>{}, 0);
  }
}
template <int D>
__global__ void __launch_bounds__(256, 4) k_stage(StageArgs a) { stage_body<D>(a, blockIdx); }

// ---------------------------------------------------------------------------
// 3-D stage kernel with two x-adjacent cells per thread.  The same fluxes and blend as
// k_stage, in the same operation order: mom_flux2 is mom_flux lane by lane (the packed
// FP32 operations round each lane as the scalar operation does), so both kernels give
// the same bits.  A tile of 64 x 8 cells marches up 32 planes; thread (l, w) owns cells
// (2l, w) and (2l+1, w).  The velocity of planes k-1..k+2 (box x i0-2..i0+65, y
// j0-2..j0+9) sits in a 4-plane shared ring, read as aligned pairs; plane k+3 is loaded
// into registers while plane k is computed.  A thread forms the lower x-, y- and z-face
// fluxes of its two cells: the upper x flux of cell 2l is its own lower flux of 2l+1,
// that of 2l+1 comes from lane l+1 by a shuffle; upper y fluxes come from the next row
// through shared memory; the upper z flux is carried to the next plane in registers.
// The fluxes through the tile's upper x edge (column 64; 3 components x 8 rows) are
// formed by lanes 0..23 of warp 0, those through its upper y edge (row 8) by warps
// 1..3, one component each.  ADV: convection on (the viscous flux alone otherwise).
constexpr int S3_TX = 64, S3_TY = 8, S3_TZ = 32;
constexpr int S3_HX = S3_TX + 4, S3_HY = S3_TY + 4, S3_PL = S3_HX * S3_HY;
constexpr int S3_NP = 4;
constexpr int S3_NPAIR = S3_PL / 2;  // float pairs per component per plane

// mom_flux on two lanes at once (each lane: the same operations as mom_flux)
template <bool ADV>
__device__ __forceinline__ float2 mom_flux2(float2 m2, float2 m1, float2 p0, float2 p1, float2 a2, float nu) {
  const float2 diff = mul2(make_float2(nu, nu), sub2(p0, m1));
  if (!ADV) return neg2(diff);
  const bool px = a2.x > 0.f, py = a2.y > 0.f;
  const float2 uu = make_float2(px ? m2.x : p1.x, py ? m2.y : p1.y);
  const float2 cc = make_float2(px ? m1.x : p0.x, py ? m1.y : p0.y);
  const float2 dd = make_float2(px ? p0.x : m1.x, py ? p0.y : m1.y);
  const float2 dD = sub2(dd, cc), dU = sub2(cc, uu);
  const float2 ad = make_float2(fabsf(dD.x), fabsf(dD.y)), au = make_float2(fabsf(dU.x), fabsf(dU.y));
  const float2 two = make_float2(2.f, 2.f);
  const float2 t2u = mul2(two, au), t2d = mul2(two, ad);
  const float2 mid = mul2(fma2(two, ad, au), make_float2(1.f / 3.f, 1.f / 3.f));
  const float tx = fminf(fminf(t2u.x, mid.x), t2d.x), ty = fminf(fminf(t2u.y, mid.y), t2d.y);
  const float2 pr = mul2(dU, dD);
  const float2 lim = make_float2(pr.x > 0.f ? copysignf(tx, dD.x) : 0.f, pr.y > 0.f ? copysignf(ty, dD.y) : 0.f);
  const float2 half = make_float2(0.5f, 0.5f);
  const float2 phi = fma2(half, lim, cc);
  return fma2(mul2(half, a2), phi, neg2(diff));
}

template <bool ADV>
__device__ __forceinline__ void stage3_body(const StageArgs& a, const uint3 bid) {
  constexpr int HX = S3_HX, PL = S3_PL, NP = S3_NP;
  __shared__ __align__(16) float s_u[3 * NP * PL];
  __shared__ __align__(16) float s_fy[3][S3_TY + 1][S3_TX];
  __shared__ float s_fxe[3][S3_TY];
  const Grid& g = a.g;
  const int tid = threadIdx.x, lane = tid & 31, ty = tid >> 5;
  const int i0 = bid.x * S3_TX, j0 = bid.y * S3_TY;
  const int tzb = a.tz > 0 ? a.tz : S3_TZ;
  const int k0 = bid.z * tzb;
  const int k1 = min(k0 + tzb, g.n[2]);
  const int i = i0 + 2 * lane, j = j0 + ty;
  const bool own_cell = (i < g.n[0]) && (j < g.n[1]);  // n_0 even: both cells or neither
  const float dt = *a.dt;
  const float nu = a.nu;
  const bool box_tile = a.fbox && i0 < a.blo[0] + a.bn[0] && i0 + S3_TX > a.blo[0] && j0 < a.blo[1] + a.bn[1] &&
                        j0 + S3_TY > a.blo[1] && k0 < a.blo[2] + a.bn[2] && k1 > a.blo[2];
  // ring slot sl holds one plane of the three components: component c at (3 sl + c) PL
  auto soff = [](int c, int sl) { return (3 * sl + c) * PL; };
  auto ld2 = [&](int o) { return *reinterpret_cast<const float2*>(s_u + o); };

  // plane fetch: pair e = tid, tid + 256 of each component's 34 x 12 pairs
  const bool xy_inner = (i0 >= 2) && (i0 + S3_TX + 2 <= g.n[0]) && (j0 >= 2) && (j0 + S3_TY + 2 <= g.n[1]);
  const long long nxy = (long long)g.n[0] * g.n[1];
  const long long fbase = (long long)(i0 - 2) + (long long)g.n[0] * (j0 - 2);
  int foff[2], fsh[2];
#pragma unroll
  for (int h = 0; h < 2; ++h) {
    const int e = tid + 256 * h, row = e / (HX / 2), cp = e - row * (HX / 2);
    foff[h] = 2 * cp + g.n[0] * row;
    fsh[h] = row * HX + 2 * cp;
  }
  // A tile on a side (not xy_inner) maps every fetched element to the array as load_u_bc
  // does.  The x and y part of that mapping is the same on every plane, so it is taken
  // once: each element's mapped in-plane index, and whether it lies on or past a
  // boundary in x (component 0 reads U_0 there) or y (component 1 reads U_1); per plane
  // only z is mapped (component 2 reads U_2 on or past a z boundary).  Same indices and
  // values as load_u_bc (which the convective exit keeps using).
  const bool side_map = !xy_inner && !g.exit;
  int bofs[2] = {0, 0};  // mapped in-plane index of the pair's first element
  // bits 8h + 2el: x boundary, 8h + 2el + 1: y boundary; bits 8h + 4..5: the second
  // element's index minus the first's (0: 0, 1: 1, 2: 1 - n_0, a periodic wrap)
  unsigned bflag = 0u;
  if (side_map) {
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int e = tid + 256 * h, row = e / (HX / 2), col = 2 * (e - row * (HX / 2));
      int first = 0;
#pragma unroll
      for (int el = 0; el < 2; ++el) {
        int I = i0 - 2 + col + el, J = j0 - 2 + row;
        bool bx = false, by = false;
        if (is_per(g, 0)) {
          I = wrap_per(I, g.n[0]);
        } else {
          bx = I <= 0 || I >= g.n[0];
          I = I < 0 ? 0 : (I >= g.n[0] ? g.n[0] - 1 : I);
        }
        if (is_per(g, 1)) {
          J = wrap_per(J, g.n[1]);
        } else {
          by = J <= 0 || J >= g.n[1];
          J = J < 0 ? 0 : (J >= g.n[1] ? g.n[1] - 1 : J);
        }
        const int q = I + g.n[0] * J;
        if (el == 0) {
          bofs[h] = q;
          first = q;
        } else {
          const int d = q - first;
          bflag |= (d == 0 ? 0u : (d == 1 ? 1u : 2u)) << (8 * h + 4);
        }
        bflag |= (bx ? 1u : 0u) << (8 * h + 2 * el);
        bflag |= (by ? 2u : 0u) << (8 * h + 2 * el);
      }
    }
  }
  float2 rv[2][3];
  auto fetch = [&](int kk) {
    const bool inner = xy_inner && kk >= 0 && kk < g.n[2];
    const long long qk = fbase + nxy * kk;
    int K = kk;
    bool bz = false;
    if (is_per(g, 2)) {
      K = wrap_per(K, g.n[2]);
    } else {
      bz = K <= 0 || K >= g.n[2];
      K = K < 0 ? 0 : (K >= g.n[2] ? g.n[2] - 1 : K);
    }
    const long long kb = nxy * K;
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int e = tid + 256 * h;
      if (e >= S3_NPAIR) break;
      if (inner) {
#pragma unroll
        for (int c = 0; c < 3; ++c)
          rv[h][c] = wl_in(qk + foff[h] + 1, g.nc, WL_DBG_STAGE)
                         ? __ldg(reinterpret_cast<const float2*>(a.u[c] + qk + foff[h]))
                         : make_float2(0.f, 0.f);
      } else if (side_map) {
#pragma unroll
        for (int c = 0; c < 3; ++c) {
          float v[2];
          const unsigned dc = (bflag >> (8 * h + 4)) & 3u;
          const int d1 = dc == 0u ? 0 : (dc == 1u ? 1 : 1 - g.n[0]);
#pragma unroll
          for (int el = 0; el < 2; ++el) {
            const unsigned f = bflag >> (8 * h + 2 * el);
            const bool bnd = c == 0 ? (f & 1u) != 0 : (c == 1 ? (f & 2u) != 0 : bz);
            const long long q = kb + bofs[h] + (el ? d1 : 0);
            v[el] = bnd ? g.U[c] : (wl_in(q, g.nc, WL_DBG_STAGE) ? __ldg(a.u[c] + q) : 0.f);
          }
          rv[h][c] = make_float2(v[0], v[1]);
        }
      } else {
        const int row = e / (HX / 2), col = 2 * (e - row * (HX / 2));
#pragma unroll
        for (int c = 0; c < 3; ++c)
          rv[h][c] = make_float2(load_u_bc<3>(a.u[c], c, g, i0 - 2 + col, j0 - 2 + row, kk),
                                 load_u_bc<3>(a.u[c], c, g, i0 - 1 + col, j0 - 2 + row, kk));
      }
    }
  };
  auto commit = [&](int sl) {
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int e = tid + 256 * h;
      if (e >= S3_NPAIR) break;
#pragma unroll
      for (int c = 0; c < 3; ++c) *reinterpret_cast<float2*>(s_u + soff(c, sl) + fsh[h]) = rv[h][c];
    }
  };
  const int own = (ty + 2) * HX + 2 * lane + 2;  // box position of cell 2l
  // the pair (U[p-1], U[p]) from the aligned pairs A = (U[p-2], U[p-1]), B = (U[p], U[p+1])
  auto mid2 = [](float2 A, float2 B) { return make_float2(A.y, B.x); };

  // lower x-face fluxes of the two cells, component C, plane slot S (plane k), SM (k-1)
  auto flux_x = [&](auto C, int sl, int sm) -> float2 {
    constexpr int c = decltype(C)::value;
    const int o = soff(c, sl) + own;
    const float2 A = ld2(o - 2), B = ld2(o), Cn = ld2(o + 2);
    float2 a2;
    if (c == 0) {
      a2 = add2(B, mid2(A, B));
    } else {
      const int ox = soff(0, sl) + own;
      a2 = add2(ld2(ox), c == 1 ? ld2(ox - HX) : ld2(soff(0, sm) + own));
    }
    return mom_flux2<ADV>(A, mid2(A, B), B, mid2(B, Cn), a2, nu);
  };
  auto flux_y = [&](auto C, int sl, int sm) -> float2 {
    constexpr int c = decltype(C)::value;
    const int o = soff(c, sl) + own;
    const int oy = soff(1, sl) + own;
    const float2 Y0 = ld2(oy);
    float2 a2;
    if (c == 0)
      a2 = add2(Y0, mid2(ld2(oy - 2), Y0));
    else if (c == 1)
      a2 = add2(Y0, ld2(oy - HX));
    else
      a2 = add2(Y0, ld2(soff(1, sm) + own));
    return mom_flux2<ADV>(ld2(o - 2 * HX), ld2(o - HX), ld2(o), ld2(o + HX), a2, nu);
  };
  // lower z-face flux at plane kf, planes kf-2 .. kf+1 in slots Q0 .. Q3
  auto flux_z = [&](auto C, int q0, int q1, int q2, int q3) -> float2 {
    constexpr int c = decltype(C)::value;
    const int oz = soff(2, q2) + own;
    const float2 Z0 = ld2(oz);
    float2 a2;
    if (c == 0)
      a2 = add2(Z0, mid2(ld2(oz - 2), Z0));
    else if (c == 1)
      a2 = add2(Z0, ld2(oz - HX));
    else
      a2 = add2(Z0, ld2(soff(2, q1) + own));
    return mom_flux2<ADV>(ld2(soff(c, q0) + own), ld2(soff(c, q1) + own), ld2(soff(c, q2) + own),
                          ld2(soff(c, q3) + own), a2, nu);
  };
  // warp 0, lanes 0..23: the flux through the upper x edge (face i0+64) of row lane%8,
  // component lane/8 (scalar mom_flux, operand addresses chosen per lane)
  auto edge_x = [&](int sl, int sm) {
    const int c = lane >> 3, row = lane & 7;
    const int pe = (row + 2) * HX + S3_TX + 2;  // box position of cell 64
    const float* U = s_u + soff(c, sl) + pe;
    const float* A = s_u + soff(0, sl) + pe;
    const float other = c == 0 ? A[-1] : (c == 1 ? A[-HX] : s_u[soff(0, sm) + pe]);
    s_fxe[c][row] = mom_flux(U[-2], U[-1], U[0], U[1], A[0] + other, nu, ADV);
  };
  // warps 1..3: the fluxes through the upper y edge (row 8) of component warp-1
  auto edge_y = [&](auto C, int sl, int sm) {
    constexpr int c = decltype(C)::value;
    const int p8 = (S3_TY + 2) * HX + 2 * lane + 2;
    const int o = soff(c, sl) + p8, oy = soff(1, sl) + p8;
    const float2 Y0 = ld2(oy);
    float2 a2;
    if (c == 0)
      a2 = add2(Y0, mid2(ld2(oy - 2), Y0));
    else if (c == 1)
      a2 = add2(Y0, ld2(oy - HX));
    else
      a2 = add2(Y0, ld2(soff(1, sm) + p8));
    const float2 f = mom_flux2<ADV>(ld2(o - 2 * HX), ld2(o - HX), ld2(o), ld2(o + HX), a2, nu);
    *reinterpret_cast<float2*>(&s_fy[c][S3_TY][2 * lane]) = f;
  };
  const long long qij = own_cell ? (long long)i + (long long)g.n[0] * j : 0;

  float2 fzl[3];
  // planes k0-2 .. k0+1 in slots 0 .. 3
  for (int t = 0; t < 4; ++t) {
    fetch(k0 - 2 + t);
    commit(t);
  }
  fetch(k0 + 2);
  __syncthreads();
  fzl[0] = flux_z(IC<0>{}, 0, 1, 2, 3);
  fzl[1] = flux_z(IC<1>{}, 0, 1, 2, 3);
  fzl[2] = flux_z(IC<2>{}, 0, 1, 2, 3);
  __syncthreads();

  // plane k: plane k+t sits in slot (k - k0 + t + 2) mod NP (run-time slots keep the
  // loop body a single copy: unrolled by the ring length it overflowed the instruction
  // cache)
  auto step = [&](int k) {
    const int PH = (k - k0) & (NP - 1);
    const int S0 = (PH + 2) & (NP - 1), SM1 = (PH + 1) & (NP - 1), SP1 = (PH + 3) & (NP - 1), SP2 = PH;
    commit(SP2);  // plane k+2 into the slot of plane k-2
    __syncthreads();
    if (k + 3 <= k1 + 1) fetch(k + 3);
    const long long qg = qij + nxy * k;
    float2 m0[3], u0v[3];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      m0[c] = own_cell ? __ldg(reinterpret_cast<const float2*>(a.mu0[c] + qg)) : make_float2(0.f, 0.f);
      u0v[c] = (own_cell && a.stage != 1) ? __ldg(reinterpret_cast<const float2*>(a.u0[c] + qg))
                                          : make_float2(0.f, 0.f);
    }
    float2 fx[3], fzu[3];
    fx[0] = flux_x(IC<0>{}, S0, SM1);
    fx[1] = flux_x(IC<1>{}, S0, SM1);
    fx[2] = flux_x(IC<2>{}, S0, SM1);
    *reinterpret_cast<float2*>(&s_fy[0][ty][2 * lane]) = flux_y(IC<0>{}, S0, SM1);
    *reinterpret_cast<float2*>(&s_fy[1][ty][2 * lane]) = flux_y(IC<1>{}, S0, SM1);
    *reinterpret_cast<float2*>(&s_fy[2][ty][2 * lane]) = flux_y(IC<2>{}, S0, SM1);
    // face k+1: planes k-1 .. k+2
    fzu[0] = flux_z(IC<0>{}, SM1, S0, SP1, SP2);
    fzu[1] = flux_z(IC<1>{}, SM1, S0, SP1, SP2);
    fzu[2] = flux_z(IC<2>{}, SM1, S0, SP1, SP2);
    if (ty == 0) {
      if (lane < 24) edge_x(S0, SM1);
    } else if (ty == 1) {
      edge_y(IC<0>{}, S0, SM1);
    } else if (ty == 2) {
      edge_y(IC<1>{}, S0, SM1);
    } else if (ty == 3) {
      edge_y(IC<2>{}, S0, SM1);
    }
    __syncthreads();
    float nxt[3];  // lower x flux of lane l+1's first cell (every lane takes part)
#pragma unroll
    for (int c = 0; c < 3; ++c) nxt[c] = __shfl_down_sync(0xffffffffu, fx[c].x, 1);
    if (own_cell) {
      const int I[3] = {i, j, k};
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        // upper x faces: (lower flux of 2l+1, lower flux of 2l+2 from lane l+1 or the edge)
        const float2 fxu = make_float2(fx[c].y, lane == 31 ? s_fxe[c][ty] : nxt[c]);
        const float2 fyu = *reinterpret_cast<const float2*>(&s_fy[c][ty + 1][2 * lane]);
        const float2 fyl = *reinterpret_cast<const float2*>(&s_fy[c][ty][2 * lane]);
        const float2 r = add2(add2(sub2(fx[c], fxu), sub2(fyl, fyu)), sub2(fzl[c], fzu[c]));
        const float2 uc = ld2(soff(c, S0) + own);
        const float2 u0 = (a.stage == 1) ? uc : u0v[c];
        const float2 f = fma2(make_float2(dt, dt), r, u0);
        const float2 mf = mul2(m0[c], f);
        float2 ov = (a.stage == 1) ? mf : mul2(make_float2(0.5f, 0.5f), fma2(m0[c], f, uc));
        float2 fo = f;
        // boundary faces of a non-periodic direction keep U_c (only i = 0 can be the pair's first cell)
        const bool upd0 = is_per(g, c) || I[c] >= 1;
        const bool upd1 = is_per(g, c) || (c == 0 ? i + 1 : I[c]) >= 1;
        if (!upd0) ov.x = fo.x = g.U[c];
        if (!upd1) ov.y = fo.y = g.U[c];
        if (wl_in(qg + 1, g.nc, WL_DBG_STAGE)) *reinterpret_cast<float2*>(a.out[c] + qg) = ov;
        if (box_tile) {  // keep f inside the body's band box for the mu1 term
          const unsigned bj = (unsigned)(j - a.blo[1]), bk = (unsigned)(k - a.blo[2]);
          if (bj < (unsigned)a.bn[1] && bk < (unsigned)a.bn[2]) {
            const long long base =
                (long long)c * a.bn[0] * a.bn[1] * a.bn[2] + (long long)a.bn[0] * (bj + (long long)a.bn[1] * bk);
            const unsigned b0 = (unsigned)(i - a.blo[0]), b1 = (unsigned)(i + 1 - a.blo[0]);
            if (b0 < (unsigned)a.bn[0] && wl_in(base + b0, g.nc, WL_DBG_BAND)) a.fbox[base + b0] = fo.x;
            if (b1 < (unsigned)a.bn[0] && wl_in(base + b1, g.nc, WL_DBG_BAND)) a.fbox[base + b1] = fo.y;
          }
        }
      }
    }
#pragma unroll
    for (int c = 0; c < 3; ++c) fzl[c] = fzu[c];
  };
  for (int k = k0; k < k1; ++k) step(k);
}
template <bool ADV>
__global__ void __launch_bounds__(256, 3) k_stage3(StageArgs a) { stage3_body<ADV>(a, blockIdx); }

// mu1 term of BDIM over the body's bounding box: out_c[I] += s * sum_j mu1_j (f[I+e_j]
// - f[I-e_j]) / 2 with mu1 = eps K1(d/eps) n at the face (s = 1 in stage 1, 1/2 in
// stage 2).  mu1 vanishes for |d| >= eps, so only band faces do work.
template <int D>
__device__ __forceinline__ void bdim_band_body(const StageArgs& a, const Body& b, int lo0, int lo1, int lo2, int bx,
                                               int by, int bz, const uint3 bid) {
  const long long nbox = (long long)bx * by * bz;
  const long long t = (long long)bid.x * blockDim.x + threadIdx.x;
  if (t >= nbox * D) return;
  const int c = (int)(t / nbox);
  long long rem = t - (long long)c * nbox;
  const int i = lo0 + (int)(rem % bx);
  rem /= bx;
  const int j = lo1 + (int)(rem % by);
  const int k = lo2 + (int)(rem / by);
  const Grid& g = a.g;
  const int I[3] = {i, j, k};
  if (!(is_per(g, c) || I[c] >= 1)) return;
  double x[3] = {i + 0.5, j + 0.5, k + 0.5};
  x[c] -= 0.5;
  // most faces of the box lie well outside the band: an FP32 distance half a cell past
  // eps skips them before the FP64 evaluation (which alone decides for the others)
  if (fabsf(body_dist_f<D>(b, x)) > (float)b.eps + 0.5f) return;
  double nrm[3];
  const double d = body_sdf<D>(b, x, nrm);
  if (!(fabs(d) < b.eps)) return;
  const double k1 = b.eps * kernel_K1(d / b.eps);
  const float dt = *a.dt;
  // f at a face: from the stage kernel's box when the face is inside it (in range),
  // else evaluated here with the BC mapping
  auto fget = [&](const int* F) -> float {
    if (a.fbox) {
      const unsigned bi = (unsigned)(F[0] - a.blo[0]), bj = (unsigned)(F[1] - a.blo[1]),
                     bk = (unsigned)(F[2] - a.blo[2]);
      if (bi < (unsigned)a.bn[0] && bj < (unsigned)a.bn[1] && bk < (unsigned)a.bn[2])
        return a.fbox[(long long)c * a.bn[0] * a.bn[1] * a.bn[2] + bi + (long long)a.bn[0] * (bj + (long long)a.bn[1] * bk)];
    }
    return f_at<D>(a, c, F[0], F[1], F[2], dt);
  };
  float acc = 0.f;
#pragma unroll
  for (int jd = 0; jd < D; ++jd) {
    int P[3] = {i, j, k}, M[3] = {i, j, k};
    P[jd] += 1;
    M[jd] -= 1;
    const float fp = fget(P);
    const float fm = fget(M);
    acc += (float)(k1 * nrm[jd]) * 0.5f * (fp - fm);
  }
  const long long q = cell_index(g, i, j, k);
  if (wl_in(q, g.nc, WL_DBG_BAND)) a.out[c][q] += (a.stage == 1 ? 1.f : 0.5f) * acc;
}
template <int D>
__global__ void __launch_bounds__(256) k_bdim_band(StageArgs a, Body b, int lo0, int lo1, int lo2, int bx,
                                                    int by, int bz) {
  bdim_band_body<D>(a, b, lo0, lo1, lo2, bx, by, bz, blockIdx);
}

// Planes per block of k_stage3: the fewest waves of blocks (3 resident per SM) times the
// planes a block stages (its own and the 3 of its z halo), from 4 to 48 planes
// (512x256x256: 37 planes, 4 waves of 1792 blocks; 32 planes in 4.5 waves measured the
// same; the 128^3 vortex: 10 planes, 416 blocks).  WL_STAGE_TZ overrides.
int stage3_planes(const Grid& g) {
  static int nsm = 0;
  if (nsm <= 0) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
        nsm <= 0) {
      cudaGetLastError();
      nsm = 152;
    }
  }
  if (const char* e = std::getenv("WL_STAGE_TZ")) return std::max(1, std::atoi(e));
  const long long cols = (long long)((g.n[0] + S3_TX - 1) / S3_TX) * ((g.n[1] + S3_TY - 1) / S3_TY);
  const long long wave = 3LL * nsm;
  int best = S3_TZ;
  double best_cost = 1e300;
  for (int tz = 48; tz >= 4; --tz) {
    const long long nb = cols * ((g.n[2] + tz - 1) / tz);
    const double cost = (double)((nb + wave - 1) / wave) * (std::min(tz, g.n[2]) + 3);
    if (cost < best_cost) {
      best_cost = cost;
      best = tz;
    }
  }
  return best;
}

// ---------------------------------------------------------------------------
int launch_stage(int D, const StageArgs& a, cudaStream_t s) {
  const Grid& g = a.g;
  dim3 blk(256);
  const bool v1 = std::getenv("WL_STAGE_V1") != nullptr;  // the one-cell-per-thread kernel
  if (D == 3 && g.n[0] % 2 == 0 && !v1) {
    const int tz = a.tz > 0 ? a.tz : S3_TZ;
    dim3 grd((g.n[0] + S3_TX - 1) / S3_TX, (g.n[1] + S3_TY - 1) / S3_TY, (g.n[2] + tz - 1) / tz);
    if (a.advect)
      k_stage3<true><<<grd, blk, 0, s>>>(a);
    else
      k_stage3<false><<<grd, blk, 0, s>>>(a);
  } else if (D == 3) {
    dim3 grd((g.n[0] + ST_TX - 1) / ST_TX, (g.n[1] + ST_TY - 1) / ST_TY, (g.n[2] + ST_TZ - 1) / ST_TZ);
    k_stage<3><<<grd, blk, 0, s>>>(a);
  } else {
    dim3 grd((g.n[0] + ST_TX - 1) / ST_TX, (g.n[1] + ST_TY - 1) / ST_TY, 1);
    k_stage<2><<<grd, blk, 0, s>>>(a);
  }
  return 0;
}

// Convective exit (reading: BC! of the paper names the boundary conditions only): the
// normal velocity e on the upper x face is carried out at the free-stream speed U,
// de/dt = -U (e - u[n_0 - 1]), by the same Heun stages as the interior:
// f_e = e0 - dt U (e_in - u_in[n_0 - 1]), out_e = f_e (stage 1) or (e_in + f_e)/2
// (stage 2); then the plane is shifted so that its mean is U: the flux out equals the
// flux in (the other boundaries' net flux is zero), as the projection's Neumann problem
// needs.  One block, the sum in FP64 in a fixed order.
template <int D>
__global__ void __launch_bounds__(1024) k_exit_stage(Grid g, const float* u0x, const float* uinx, float* outx,
                                                     const float* dtp, int stage) {
  __shared__ double sh[32];
  const int n0 = g.n[0], n1 = g.n[1], n2 = D == 3 ? g.n[2] : 1;
  const long long ne = (long long)n1 * n2;
  const float dt = *dtp, U = g.U[0];
  double sum = 0.0;
  for (long long q = threadIdx.x; q < ne; q += 1024) {
    const int j = (int)(q % n1), k = (int)(q / n1);
    const float e0 = u0x[g.nc + q], ei = uinx[g.nc + q];
    const float ul = uinx[(long long)(n0 - 1) + (long long)n0 * ((long long)j + (long long)n1 * k)];
    const float f = fmaf(-dt * U, ei - ul, e0);
    const float v = stage == 1 ? f : 0.5f * (ei + f);
    outx[g.nc + q] = v;
    sum += v;
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) sum += __shfl_xor_sync(0xffffffffu, sum, o);
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = sum;
  __syncthreads();
  double tot = 0.0;
  for (int w = 0; w < 32; ++w) tot += sh[w];
  const float shift = (float)((double)U - tot / (double)ne);
  for (long long q = threadIdx.x; q < ne; q += 1024) outx[g.nc + q] += shift;
}

int launch_exit_stage(int D, const Grid& g, const float* u0x, const float* uinx, float* outx, const float* dt, int stage,
                      cudaStream_t s) {
  if (D == 3)
    k_exit_stage<3><<<1, 1024, 0, s>>>(g, u0x, uinx, outx, dt, stage);
  else
    k_exit_stage<2><<<1, 1024, 0, s>>>(g, u0x, uinx, outx, dt, stage);
  return 0;
}

__global__ void k_fill(float* p, long long n, float v) {
  const long long q = (long long)blockIdx.x * 256 + threadIdx.x;
  if (q < n) p[q] = v;
}
int launch_fill(float* p, long long n, float v, cudaStream_t s) {
  if (n > 0) k_fill<<<(int)((n + 255) / 256), 256, 0, s>>>(p, n, v);
  return 0;
}

bool stage_band_box(int D, const Grid& g, const Body& b, int* lo, int* hi) {
  if (b.kind == 0) return false;
  if (b.kind == 3) {  // the cells bracketing the band, two cells wider
    for (int d = 0; d < 3; ++d) {
      if (d >= D) {
        lo[d] = 0;
        hi[d] = 1;
        continue;
      }
      if (b.bhi[d] <= b.blo[d]) return false;  // no band cell
      lo[d] = std::max(0, b.blo[d] - 2);
      hi[d] = std::min(g.n[d], b.bhi[d] + 2);
    }
    return true;
  }
  double ext = b.r1 + b.eps + 2.0;
  if (b.kind == 2) ext = b.r1 + b.r2 + b.eps + 2.0;
  for (int d = 0; d < 3; ++d) {
    if (d >= D) {
      lo[d] = 0;
      hi[d] = 1;
      continue;
    }
    // the torus's axis is along x: its surface spans c_x +- r there
    const double e = (b.kind == 2 && d == 0) ? b.r2 + b.eps + 2.0 : ext;
    lo[d] = (int)fmax(0.0, floor(b.c[d] - e));
    hi[d] = (int)fmin((double)g.n[d], ceil(b.c[d] + e) + 1.0);
    if (hi[d] <= lo[d]) return false;  // body outside the grid: no band
  }
  return true;
}

int launch_band(int D, const StageArgs& a, const Body& b, cudaStream_t s) {
  const Grid& g = a.g;
  if (b.kind != 0) {
    // bounding box of the faces within eps of the surface
    int lo[3], hi[3];
    if (!stage_band_box(D, g, b, lo, hi)) return 0;
    const int bx = hi[0] - lo[0], by = hi[1] - lo[1], bz = hi[2] - lo[2];
    const long long n = (long long)bx * by * bz * D;
    const int nb = (int)((n + 255) / 256);
    if (D == 3)
      k_bdim_band<3><<<nb, 256, 0, s>>>(a, b, lo[0], lo[1], lo[2], bx, by, bz);
    else
      k_bdim_band<2><<<nb, 256, 0, s>>>(a, b, lo[0], lo[1], lo[2], bx, by, bz);
  }
  return 0;
}


// ---------------------------------------------------------------------------
// Batched launches (many small simulations, one launch; see BatchSlot).
__device__ __forceinline__ int batch_block(const BatchGrid& bg, uint3& bid) {
  const int b = (int)blockIdx.x;
  int lo = 0, hi = bg.n;  // bg.start[lo] <= b < bg.start[hi]
  while (hi - lo > 1) {
    const int m = (lo + hi) >> 1;
    if (bg.start[m] <= b) lo = m; else hi = m;
  }
  const unsigned local = (unsigned)(b - bg.start[lo]), gx = bg.gx[lo], gy = bg.gy[lo];
  bid = make_uint3(local % gx, (local / gx) % gy, local / (gx * gy));
  wl_in(bid.z, (unsigned)(bg.start[lo + 1] - bg.start[lo]) / (gx * gy), WL_DBG_BATCH);
  return bg.slot[lo];
}

dim3 stage_grid(int D, const Grid& g) {
  if (D == 3 && g.n[0] % 2 == 0)
    return dim3((g.n[0] + S3_TX - 1) / S3_TX, (g.n[1] + S3_TY - 1) / S3_TY, (g.n[2] + S3_TZ - 1) / S3_TZ);
  if (D == 3) return dim3((g.n[0] + ST_TX - 1) / ST_TX, (g.n[1] + ST_TY - 1) / ST_TY, (g.n[2] + ST_TZ - 1) / ST_TZ);
  return dim3((g.n[0] + ST_TX - 1) / ST_TX, (g.n[1] + ST_TY - 1) / ST_TY, 1);
}
dim3 band_grid(int D, const int* bn) {
  const long long n = (long long)bn[0] * bn[1] * bn[2] * D;
  return dim3((unsigned)((n + 255) / 256), 1, 1);
}

// a batch holds 3-D slots of even n_0 (the pair kernel) with convection on, or 2-D slots
template <int D>
__global__ void __launch_bounds__(256, 3) kb_stage(const BatchSlot* __restrict__ t, const __grid_constant__ BatchGrid bg,
                                                   int stage) {
  uint3 bid;
  const int s = batch_block(bg, bid);
  if constexpr (D == 3)
    stage3_body<true>(t[s].stage[stage - 1], bid);
  else
    stage_body<2>(t[s].stage[stage - 1], bid);
}
template <int D>
__global__ void __launch_bounds__(256) kb_band(const BatchSlot* __restrict__ t, const __grid_constant__ BatchGrid bg,
                                               int stage) {
  uint3 bid;
  const BatchSlot& sl = t[batch_block(bg, bid)];
  bdim_band_body<D>(sl.stage[stage - 1], sl.body, sl.blo[0], sl.blo[1], sl.blo[2], sl.bn[0], sl.bn[1], sl.bn[2], bid);
}

int launch_batch_stage(int D, const BatchSlot* t, const BatchGrid& bg, int stage, cudaStream_t s) {
  if (bg.n == 0) return 0;
  if (D == 3)
    kb_stage<3><<<bg.start[bg.n], 256, 0, s>>>(t, bg, stage);
  else
    kb_stage<2><<<bg.start[bg.n], 256, 0, s>>>(t, bg, stage);
  return 0;
}
int launch_batch_band(int D, const BatchSlot* t, const BatchGrid& bg, int stage, cudaStream_t s) {
  if (bg.n == 0) return 0;
  if (D == 3)
    kb_band<3><<<bg.start[bg.n], 256, 0, s>>>(t, bg, stage);
  else
    kb_band<2><<<bg.start[bg.n], 256, 0, s>>>(t, bg, stage);
  return 0;
}

}  // namespace wl

namespace wl {
unsigned dbg_take_momentum() {
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
