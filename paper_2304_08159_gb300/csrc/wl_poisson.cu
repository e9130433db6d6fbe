// Pressure projection (project!, Table 2) and the geometric-multigrid Poisson solve
// on the BDIM-modified matrix (Section 2; Lauber 2022; Weymouth 2022), the CFL time
// step (CFL!, Table 2), the body measure and the pressure force.
//
// Poisson operator with face coefficients L (Section 2):
//   (A x)[I] = sum_c L_c[I+e_c] (x[I+e_c] - x[I]) + L_c[I] (x[I-e_c] - x[I]),
// L = mu0 at faces and 0 on non-periodic boundary faces.  The solver works on the
// pressure itself: A p = div(u)/(w dt), which is the system A x = div(u) with
// x = p w dt scaled by 1/(w dt); the tolerance test converts back to x units.
//
// Multigrid cycle V(0, post): residual + restriction (sum of the 2^D children) in one
// pass, recursive coarse levels with zero initial guess, coarse face coefficient =
// half the sum of the 2^(D-1) fine faces it covers, the coarsest level solved by
// FP64 conjugate gradients, piecewise-constant prolongation fused into the first
// smoothing sweep, red-black Gauss-Seidel sweeps (red: i+j+k even, first).  Cells
// whose row is zero (all faces blocked by the body) carry x = 0.
#include <cooperative_groups.h>
#include <type_traits>

#include "wl_dev.cuh"
#include "wl_kernels.h"

namespace wl {

__device__ __forceinline__ void cell_coords(int D, int blk_y, int tid, int& tx, int& ty, int& tz) {
  tx = tid & 31;
  if (D == 3) {
    ty = (tid >> 5) & 3;
    tz = tid >> 7;
  } else {
    ty = tid >> 5;
    tz = 0;
  }
  (void)blk_y;
}

// Upper/lower neighbour of linear cell q along c (wrapping periodic sides); `has` is
// false on a non-periodic side, where the face coefficient is zero.
__device__ __forceinline__ long long nb_up(const Grid& g, int c, int Ic, long long q, long long stc, bool& has) {
  if (Ic + 1 < g.n[c]) {
    has = true;
    return q + stc;
  }
  has = is_per(g, c);
  return has ? q - (long long)(g.n[c] - 1) * stc : q;
}
__device__ __forceinline__ long long nb_dn(const Grid& g, int c, int Ic, long long q, long long stc) {
  if (Ic > 0) return q - stc;
  return is_per(g, c) ? q + (long long)(g.n[c] - 1) * stc : q;
}

// ---------------------------------------------------------------------------
// k_residual: one pass over a level computing (per mode)
//   RES_DIVERGENCE: z = div(u)/(w dt) (stored), r = z - A x, max|r|, restrict r
//   RES_RESIDUAL:   r = z - A x, max|r|, restrict r
//   RES_RESTRICT:   restrict z (coarse levels whose iterate is still zero)
//   RES_DIV_ONLY:   z = div(u) (raw, for inspection)
// A block is 32 x 8 cell columns walking RS_ZP pairs of planes (3-D), so each
// block holds whole 2^D families of children for the restriction (the z pair is
// summed in registers, x pairs by a shuffle, y pairs through shared memory) and
// issues a single atomic for the norm.
constexpr int RS_ZP = 2;

template <int D>
__device__ __forceinline__ float residual_cell(const ResArgs& a, int i, int j, int k, unsigned& mbits, float zvm) {
  const Grid& g = a.g;
  const long long q = cell_index(g, i, j, k);
  const long long st[3] = {1, (long long)g.n[0], (long long)g.n[0] * g.n[1]};
  const int I[3] = {i, j, k};
  float z;
  if (a.mode == RES_DIVERGENCE || a.mode == RES_DIV_ONLY) {
    float div = 0.f;
#pragma unroll
    for (int c = 0; c < D; ++c) {
      bool has;
      const long long qu = nb_up(g, c, I[c], q, st[c], has);
      const float up =
          has ? __ldg(a.u[c] + qu) : ((c == 0 && g.exit) ? __ldg(a.u[0] + exit_index(g, I[1], I[2])) : g.U[c]);
      div += up - __ldg(a.u[c] + q);
    }
    z = (a.mode == RES_DIV_ONLY) ? div : div * a.inv_w * a.st->inv_dtf;
    if (wl_in(q, g.nc, WL_DBG_RESID)) a.z[q] = z;
    if (a.mode == RES_DIV_ONLY) return 0.f;
  } else {
    z = ld_st(a.z, a.ztype, q);
  }
  if (a.mode == RES_RESTRICT) {
    if (a.zconv) st_st(a.zconv, a.zconvtype, q, z * zvm);
    return z;
  }
  float r;
  if (a.ph) {
    // r = z - sum_f L_f (p_nb - p_0) with p = ph + pl in double-float arithmetic; faces
    // in the order x up, x down, y up, y down (, z up, z down)
    const float h0 = __ldg(a.ph + q), l0 = __ldg(a.pl + q);
    float Lf[2 * D], hn[2 * D], ln[2 * D];
    bool unit = true;
#pragma unroll
    for (int c = 0; c < D; ++c) {
      bool has;
      long long qu = nb_up(g, c, I[c], q, st[c], has);
      long long qm = nb_dn(g, c, I[c], q, st[c]);
      if (!wl_in(qu, g.nc, WL_DBG_RESID)) qu = q;
      if (!wl_in(qm, g.nc, WL_DBG_RESID)) qm = q;
      Lf[2 * c] = has ? (a.uni ? a.uval : __ldg(a.L[c] + qu)) : 0.f;
      Lf[2 * c + 1] = a.uni ? ((I[c] > 0 || is_per(g, c)) ? a.uval : 0.f) : __ldg(a.L[c] + q);
      hn[2 * c] = __ldg(a.ph + qu);
      ln[2 * c] = __ldg(a.pl + qu);
      hn[2 * c + 1] = __ldg(a.ph + qm);
      ln[2 * c + 1] = __ldg(a.pl + qm);
    }
#pragma unroll
    for (int f = 0; f < 2 * D; ++f) unit = unit && (Lf[f] == 0.f || Lf[f] == 1.f);
    float rh, rl;
    if (unit) {
      // every coefficient 1 or 0: the present neighbours' pressures summed in
      // double-float, minus nf p0 (nf faces, a small integer: nf h0 exact by TwoProd)
      float S = __fmul_rn(Lf[0], hn[0]), Se = 0.f, Sl = __fmul_rn(Lf[0], ln[0]), nf = Lf[0];
#pragma unroll
      for (int f = 1; f < 2 * D; ++f) {
        float e;
        two_sum(S, __fmul_rn(Lf[f], hn[f]), S, e);
        Se = __fadd_rn(Se, e);
        Sl = fmaf(Lf[f], ln[f], Sl);
        nf = __fadd_rn(nf, Lf[f]);
      }
      float T, Te, Dh, Dl;
      two_prod(nf, h0, T, Te);
      Te = fmaf(nf, l0, Te);
      two_sum(S, -T, Dh, Dl);
      Dl = __fadd_rn(Dl, __fsub_rn(__fadd_rn(Se, Sl), Te));
      two_sum(z, -Dh, rh, rl);
      r = __fadd_rn(rh, __fsub_rn(rl, Dl));
    } else {
      // face by face: the exact difference to the neighbour times its coefficient
      // (TwoSum, TwoProd), accumulated in double-float
      float ah = 0.f, al = 0.f;
#pragma unroll
      for (int f = 0; f < 2 * D; ++f) {
        float dh, dl, th, tl, sh, sl;
        two_sum(hn[f], -h0, dh, dl);
        dl += ln[f] - l0;
        two_prod(Lf[f], dh, th, tl);
        tl = fmaf(Lf[f], dl, tl);
        two_sum(ah, th, sh, sl);
        ah = sh;
        al += sl + tl;
      }
      two_sum(z, -ah, rh, rl);
      r = rh + (rl - al);
    }
  } else {
    const float x0 = __ldg(a.x + q);
    float acc = 0.f;
#pragma unroll
    for (int c = 0; c < D; ++c) {
      bool has;
      long long qu = nb_up(g, c, I[c], q, st[c], has);
      long long qm = nb_dn(g, c, I[c], q, st[c]);
      if (!wl_in(qu, g.nc, WL_DBG_RESID)) qu = q;
      if (!wl_in(qm, g.nc, WL_DBG_RESID)) qm = q;
      const float Lu = has ? (a.uni ? a.uval : __ldg(a.L[c] + qu)) : 0.f;
      const float Ll = a.uni ? ((I[c] > 0 || is_per(g, c)) ? a.uval : 0.f) : __ldg(a.L[c] + q);
      acc += Lu * (__ldg(a.x + qu) - x0) + Ll * (__ldg(a.x + qm) - x0);
    }
    r = z - acc;
  }
  if (a.rout && wl_in(q, g.nc, WL_DBG_RESID)) a.rout[q] = r;
  mbits = max(mbits, __float_as_uint(fabsf(r)));
  return r;
}

template <int D>
__device__ __forceinline__ void residual_body(const ResArgs& a, const uint3 bid) {
  __shared__ float s_r[8][32];
  __shared__ unsigned s_m[8];
  // the coarse levels' scale folded into the restriction's multipliers
  const float S = a.apply_cs ? ldexpf(1.f, a.st->cs_used) : 1.f;
  const float zcm = a.zcmul * S, zvm = a.zconvmul * S;
  const Grid& g = a.g;
  const int tid = threadIdx.x, tx = tid & 31, ty = tid >> 5;
  const int i = bid.x * 32 + tx, j = bid.y * 8 + ty;
  const bool inxy = i < g.n[0] && j < g.n[1];
  const int kb = (D == 3) ? bid.z * 2 * RS_ZP : 0;
  const int ke = (D == 3) ? min(kb + 2 * RS_ZP, g.n[2]) : 1;
  unsigned mbits = 0u;
  for (int k = kb; k < ke; k += (D == 3 ? 2 : 1)) {
    float v = 0.f;
    if (inxy) {
      v = residual_cell<D>(a, i, j, k, mbits, zvm);
      if (D == 3 && k + 1 < ke) v += residual_cell<D>(a, i, j, k + 1, mbits, zvm);
    }
    if (a.zc) {
      v += __shfl_xor_sync(0xffffffffu, v, 1);
      s_r[ty][tx] = v;
      __syncthreads();
      if (tid < 64) {
        const int cx = tid & 15, cy = tid >> 4;
        const float sum = s_r[2 * cy][2 * cx] + s_r[2 * cy + 1][2 * cx];
        const int I = bid.x * 16 + cx, J = bid.y * 4 + cy, K = (D == 3) ? (k >> 1) : 0;
        if (I < a.cn[0] && J < a.cn[1] && K < a.cn[2]) {
          const long long qc = (long long)I + (long long)a.cn[0] * ((long long)J + (long long)a.cn[1] * K);
          if (wl_in(qc, (long long)a.cn[0] * a.cn[1] * a.cn[2], WL_DBG_RESID)) st_st(a.zc, a.zctype, qc, sum * zcm);
        }
      }
      __syncthreads();
    }
  }
  if (a.mode == RES_RESIDUAL || a.mode == RES_DIVERGENCE) {
    const unsigned m = block_max_bits<256>(mbits, s_m);
    if (tid == 0 && m) atomicMax(&a.st->norm_bits, m);
  }
}
template <int D>
__global__ void __launch_bounds__(256) k_residual(ResArgs a) { residual_body<D>(a, blockIdx); }

// RES_RESTRICT alone (coarse levels): one thread per coarse cell loads its 2^D children
// at once (x pairs as float2 when the field is FP32) and sums them in the fused pass's
// order (z pairs, then x pairs, then y pairs: the same bits), storing the 16-bit copy
// of z on the way when the level keeps one.  Every restricting level has even sides.
template <int D>
__device__ __forceinline__ void restrict_body(const ResArgs& a, const uint3 bid, const unsigned nbx) {
  const float S = a.apply_cs ? ldexpf(1.f, a.st->cs_used) : 1.f;
  const float zcm = a.zcmul * S, zvm = a.zconvmul * S;
  const Grid& g = a.g;
  const int c0 = a.cn[0], c1 = a.cn[1];
  const long long ncc = (long long)c0 * c1 * (D == 3 ? a.cn[2] : 1);
  const long long n0 = g.n[0], nn = (long long)g.n[0] * g.n[1];
  const bool plain = a.ztype == ST_F32 && !a.zconv;
  for (long long t = (long long)bid.x * 256 + threadIdx.x; t < ncc; t += (long long)nbx * 256) {
    const int I = (int)(t % c0);
    const long long r = t / c0;
    const int J = (int)(r % c1), K = (int)(r / c1);
    const long long b = 2LL * I + n0 * (2LL * J) + (D == 3 ? nn * (2LL * K) : 0);
    if (!wl_in(b + 1 + n0 + (D == 3 ? nn : 0), g.nc, WL_DBG_RESTRICT)) continue;  // the last child
    // children (dx, dy, dz) at b + dx + n0 dy + nn dz
    float v[2][2][2];
    if (plain) {
      const float* z = a.z;
#pragma unroll
      for (int dz = 0; dz < (D == 3 ? 2 : 1); ++dz)
#pragma unroll
        for (int dy = 0; dy < 2; ++dy) {
          const float2 p = __ldg(reinterpret_cast<const float2*>(z + b + n0 * dy + nn * dz));
          v[dz][dy][0] = p.x;
          v[dz][dy][1] = p.y;
        }
    } else {
#pragma unroll
      for (int dz = 0; dz < (D == 3 ? 2 : 1); ++dz)
#pragma unroll
        for (int dy = 0; dy < 2; ++dy)
#pragma unroll
          for (int dx = 0; dx < 2; ++dx) {
            const long long q = b + dx + n0 * dy + nn * dz;
            const float zq = ld_st(a.z, a.ztype, q);
            if (a.zconv) st_st(a.zconv, a.zconvtype, q, zq * zvm);
            v[dz][dy][dx] = zq;
          }
    }
    float sum;
    if (D == 3) {
      const float a00 = v[0][0][0] + v[1][0][0], a10 = v[0][0][1] + v[1][0][1];
      const float a01 = v[0][1][0] + v[1][1][0], a11 = v[0][1][1] + v[1][1][1];
      sum = (a00 + a10) + (a01 + a11);
    } else {
      sum = (v[0][0][0] + v[0][0][1]) + (v[0][1][0] + v[0][1][1]);
    }
    st_st(a.zc, a.zctype, t, sum * zcm);
  }
}
template <int D>
__global__ void __launch_bounds__(256) k_restrict(ResArgs a) { restrict_body<D>(a, blockIdx, gridDim.x); }

int launch_residual(int D, const ResArgs& a, cudaStream_t s) {
  const Grid& g = a.g;
  if (a.mode == RES_RESTRICT && a.zc) {
    const long long ncc = (long long)a.cn[0] * a.cn[1] * (D == 3 ? a.cn[2] : 1);
    const int blocks = (int)std::min<long long>((ncc + 255) / 256, 152LL * 8 * 4);
    if (D == 3)
      k_restrict<3><<<blocks, 256, 0, s>>>(a);
    else
      k_restrict<2><<<blocks, 256, 0, s>>>(a);
    return 0;
  }
  if (D == 3) {
    dim3 grd((g.n[0] + 31) / 32, (g.n[1] + 7) / 8, (g.n[2] + 2 * RS_ZP - 1) / (2 * RS_ZP));
    k_residual<3><<<grd, 256, 0, s>>>(a);
  } else {
    dim3 grd((g.n[0] + 31) / 32, (g.n[1] + 7) / 8, 1);
    k_residual<2><<<grd, 256, 0, s>>>(a);
  }
  return 0;
}

// ---------------------------------------------------------------------------
// k_sweep: one red-black Gauss-Seidel sweep (all red cells, then all black cells),
// out of place (x_in -> x_out), with the prolongation of a coarse correction fused
// into the read of x_in.  A tile of 64 x 8 cells marches up through `tz` planes;
// planes k-1..k+2 of the iterate (2-cell in-plane halo) sit in a 4-plane shared ring.
// At plane k: red cells of plane k+1 are relaxed on the tile plus a 1-cell halo
// (using old black values), then black cells of plane k on the tile (using the new
// red values), and plane k is written.  Halo red cells are recomputed by every tile
// that needs them, from the same inputs, so tiles never exchange data.  All global
// loads of an iteration (the new plane of the iterate and the coefficients and
// right-hand side of the cells relaxed in it) are issued together, before the
// first barrier, so each plane pays one memory latency.
constexpr int SW_TX = 64, SW_TY = 8;
constexpr int SW_HX = SW_TX + 4, SW_HY = SW_TY + 4;
constexpr int SW_RED = (SW_TY + 2) * (SW_TX + 2) / 2;  // red cells of the tile plus halo, per plane
constexpr int SW_LOADS = (SW_HY * SW_HX + 255) / 256;

struct RelaxIn {
  float z, Lu[3], Ll[3];
  bool ok;
};

// Offsets of the tile footprint's columns / rows / planes after the boundary mapping
// (periodic wrap; -1 outside a non-periodic side), so that every load of the march
// is a table read and two adds whether or not the tile touches the boundary.
template <int D, typename T>
__device__ __forceinline__ void sweep_body(const SweepArgs& a, const uint3 bid) {
  const T* __restrict__ xin = reinterpret_cast<const T*>(a.x_in);
  const T* __restrict__ zf = reinterpret_cast<const T*>(a.z);
  const T* __restrict__ Lf[3] = {reinterpret_cast<const T*>(a.L[0]), reinterpret_cast<const T*>(a.L[1]),
                                 reinterpret_cast<const T*>(a.L[2])};
  T* xout = reinterpret_cast<T*>(a.x_out);
  const float xcm = a.cs ? ldexpf(1.f, -a.cs->cs_used) : 1.f;  // removes the coarse levels' scale
  constexpr int NP = (D == 3) ? 4 : 1;
  __shared__ float s_x[NP][SW_HY][SW_HX];
  __shared__ int s_xo[SW_HX], s_yo[SW_HY], s_cxo[SW_HX], s_cyo[SW_HY];
  const Grid& g = a.g;
  const int tid = threadIdx.x, tx = tid & 31, ty = tid >> 5;
  const int i0 = bid.x * SW_TX, j0 = bid.y * SW_TY;
  const int k0 = (D == 3) ? bid.z * a.tz : 0;
  const int k1 = (D == 3) ? min(k0 + a.tz, g.n[2]) : 1;
  if (a.only_wrapping && !sweep_tile_wraps_xy(g, i0, j0)) return;
  const int n0 = g.n[0], nn = g.n[0] * g.n[1];
  const int cn0 = a.cn[0], cnn = a.cn[0] * a.cn[1];
  auto wrap = [&](int q, int d) -> int {  // mapped index along d, or -1
    const int n = g.n[d];
    if (q >= 0 && q < n) return q;
    if (!is_per(g, d)) return -1;
    return wrap_per(q, n);  // (a footprint wider than the level can reach past one period)
  };
  for (int t = tid; t < SW_HX + SW_HY; t += 256) {
    if (t < SW_HX) {
      const int m = wrap(i0 - 2 + t, 0);
      s_xo[t] = m;
      s_cxo[t] = m >= 0 ? (m >> 1) : -1;
    } else {
      const int r = t - SW_HX;
      const int m = wrap(j0 - 2 + r, 1);
      s_yo[r] = m >= 0 ? m * n0 : -1;
      s_cyo[r] = m >= 0 ? (m >> 1) * cn0 : -1;
    }
  }
  __syncthreads();
  auto zoff = [&](int kk) -> int {
    if (D == 2) return 0;
    const int m = wrap(kk, 2);
    return m >= 0 ? m * nn : -1;
  };
  auto czoff = [&](int kk) -> int {
    if (D == 2) return 0;
    const int m = wrap(kk, 2);
    return m >= 0 ? (m >> 1) * cnn : -1;
  };
  auto slot = [&](int kk) { return (D == 3) ? ((kk - k0 + 2) & 3) : 0; };
  // iterate value at footprint position (col, row) of a plane (with the prolonged correction)
  auto xeff = [&](int col, int row, int zo, int czo) -> float {
    const int xo = s_xo[col], yo = s_yo[row];
    float v = 0.f;
    if (xo >= 0 && yo >= 0 && zo >= 0) {
      if (xin && wl_in(xo + yo + zo, g.nc, WL_DBG_SWEEP)) v = ldf(xin, xo + yo + zo);
      if (a.xc && wl_in(s_cxo[col] + s_cyo[row] + czo, (long long)cn0 * a.cn[1] * a.cn[2], WL_DBG_COARSE))
        v += xcm * ld_st(a.xc, a.xctype, s_cxo[col] + s_cyo[row] + czo);
    }
    return v;
  };
  // right-hand side and face coefficients of the cell at tile position (ii, jj); on a
  // level without a body (uni) the coefficients are formed: uval on every face, 0 on a
  // non-periodic wall face (the values stored there, so the same bits)
  const bool uni = a.uni != 0;
  const float uv = a.uval;
  const bool px = is_per(g, 0), py = is_per(g, 1), pz = is_per(g, 2);
  auto fetch = [&](int ii, int jj, int zo, int zou, RelaxIn& c) {
    const int col = ii + 2, row = jj + 2;
    const int xo = s_xo[col], yo = s_yo[row];
    c.ok = xo >= 0 && yo >= 0 && zo >= 0;
    if (!c.ok) return;
    const int q = xo + yo + zo;
    if (!wl_in(q, g.nc, WL_DBG_SWEEP) || !wl_in(xo + yo + (zou >= 0 ? zou : zo), g.nc, WL_DBG_SWEEP)) {
      c.ok = false;
      return;
    }
    c.z = ldf(zf, q);
    if constexpr (!std::is_same<T, float>::value) c.z *= a.zmul;
    const int xu = s_xo[col + 1], yu = s_yo[row + 1];
    if (uni) {
      c.Ll[0] = (xo > 0 || px) ? uv : 0.f;
      c.Lu[0] = xu >= 0 ? uv : 0.f;
      c.Ll[1] = (yo > 0 || py) ? uv : 0.f;
      c.Lu[1] = yu >= 0 ? uv : 0.f;
      if (D == 3) {
        c.Ll[2] = (zo > 0 || pz) ? uv : 0.f;
        c.Lu[2] = zou >= 0 ? uv : 0.f;
      }
      return;
    }
    c.Ll[0] = ldf(Lf[0], q);
    c.Lu[0] = xu >= 0 ? ldf(Lf[0], xu + yo + zo) : 0.f;
    c.Ll[1] = ldf(Lf[1], q);
    c.Lu[1] = yu >= 0 ? ldf(Lf[1], xo + yu + zo) : 0.f;
    if (D == 3) {
      c.Ll[2] = ldf(Lf[2], q);
      c.Lu[2] = zou >= 0 ? ldf(Lf[2], xo + yo + zou) : 0.f;
    }
  };
  // Gauss-Seidel value from the shared neighbours (0 for a cell with no equation)
  auto relax = [&](const RelaxIn& c, int ii, int jj, int kk) -> float {
    const int sl = slot(kk);
    float sum = 0.f, dg = 0.f;
#pragma unroll
    for (int d = 0; d < D; ++d) {
      float xu, xd;
      if (d == 0) {
        xu = s_x[sl][jj + 2][ii + 3];
        xd = s_x[sl][jj + 2][ii + 1];
      } else if (d == 1) {
        xu = s_x[sl][jj + 3][ii + 2];
        xd = s_x[sl][jj + 1][ii + 2];
      } else {
        xu = s_x[slot(kk + 1)][jj + 2][ii + 2];
        xd = s_x[slot(kk - 1)][jj + 2][ii + 2];
      }
      sum = fmaf(c.Lu[d], xu, sum);
      sum = fmaf(c.Ll[d], xd, sum);
      dg += c.Lu[d] + c.Ll[d];
    }
    return (dg > 0.f) ? __fdividef(sum - c.z, dg) : 0.f;
  };
  auto red_pos = [&](int e, int kr, int& ii, int& jj) {
    constexpr int RW = (SW_TX + 2) / 2;
    const int row = e / RW, m = e - row * RW;
    jj = row - 1;
    ii = -1 + 2 * m + ((i0 - 1 + j0 + jj + kr) & 1);
  };
  auto load_plane = [&](int kk) {
    const int zo = zoff(kk), czo = czoff(kk);
    for (int e = tid; e < SW_HY * SW_HX; e += 256) {
      const int row = e / SW_HX, col = e - row * SW_HX;
      s_x[slot(kk)][row][col] = xeff(col, row, zo, czo);
    }
  };
  auto red_plane = [&](int kr) {
    const int zo = zoff(kr), zou = zoff(kr + 1);
    for (int e = tid; e < SW_RED; e += 256) {
      int ii, jj;
      red_pos(e, kr, ii, jj);
      RelaxIn c;
      fetch(ii, jj, zo, zou, c);
      if (c.ok) s_x[slot(kr)][jj + 2][ii + 2] = relax(c, ii, jj, kr);
    }
  };

  if (D == 3) {
    load_plane(k0 - 2);
    load_plane(k0 - 1);
    load_plane(k0);
    load_plane(k0 + 1);
    __syncthreads();
    red_plane(k0 - 1);
    red_plane(k0);
    __syncthreads();
  }
  const int P0 = (i0 + j0 + ty) & 1;  // parity of column 2*tx in plane 0
  // The global loads of iteration k are issued one phase of iteration k-1 ahead of
  // their use, each into registers that phase has just freed: the new iterate plane
  // (k+2) after the previous one is committed, the red cells' operands (plane k+1)
  // after the red phase, the black cell's (plane k) after the black phase.
  float xv[SW_LOADS];
  auto load_x = [&](int k) {
    const int kn = (D == 3) ? k + 2 : 0;
    const int zn = zoff(kn), czn = czoff(kn);
#pragma unroll
    for (int m = 0; m < SW_LOADS; ++m) {
      const int e = tid + 256 * m;
      xv[m] = 0.f;
      if (e < SW_HY * SW_HX) {
        const int row = e / SW_HX, col = e - row * SW_HX;
        xv[m] = xeff(col, row, zn, czn);
      }
    }
  };
  RelaxIn rc[2];
  int rii[2], rjj[2];
  auto load_red = [&](int k) {
    const int kr = (D == 3) ? k + 1 : 0;
    const int zr = zoff(kr), zru = zoff(kr + 1);
#pragma unroll
    for (int m = 0; m < 2; ++m) {
      const int e = tid + 256 * m;
      rc[m].ok = false;
      if (e < SW_RED) {
        red_pos(e, kr, rii[m], rjj[m]);
        fetch(rii[m], rjj[m], zr, zru, rc[m]);
      }
    }
  };
  RelaxIn bc;
  int P = 0, ib = 0, ir = 0;
  auto load_black = [&](int k) {
    P = (P0 + k) & 1;
    ib = 2 * tx + (P ^ 1);
    ir = 2 * tx + P;
    bc.ok = false;
    if (i0 + ib < g.n[0] && j0 + ty < g.n[1]) fetch(ib, ty, zoff(k), zoff(k + 1), bc);
  };
  load_x(k0);
  load_red(k0);
  load_black(k0);
  for (int k = k0; k < k1; ++k) {
    const bool more = k + 1 < k1;
    // ---- new plane into the ring (2-D: the only plane)
    const int kn = (D == 3) ? k + 2 : 0;
#pragma unroll
    for (int m = 0; m < SW_LOADS; ++m) {
      const int e = tid + 256 * m;
      if (e < SW_HY * SW_HX) {
        const int row = e / SW_HX, col = e - row * SW_HX;
        s_x[slot(kn)][row][col] = xv[m];
      }
    }
    if (more) load_x(k + 1);
    __syncthreads();
    // ---- red cells of plane kr on the tile plus halo
    const int kr = (D == 3) ? k + 1 : 0;
#pragma unroll
    for (int m = 0; m < 2; ++m)
      if (rc[m].ok) s_x[slot(kr)][rjj[m] + 2][rii[m] + 2] = relax(rc[m], rii[m], rjj[m], kr);
    if (more) load_red(k + 1);
    __syncthreads();
    // ---- black cells of plane k on the tile, one per thread; write plane k
    const float vb = bc.ok ? relax(bc, ib, ty, k) : 0.f;
    const float vr = s_x[slot(k)][ty + 2][ir + 2];
    const int gi = i0 + 2 * tx, gj = j0 + ty;
    if (gj < g.n[1] && gi < g.n[0]) {
      const int q = gi + n0 * gj + zoff(k);
      const float v0 = P ? vb : vr, v1 = P ? vr : vb;
      const bool two = gi + 1 < g.n[0];
      if (std::is_same<T, float>::value && a.ph) {
        // last sweep of a correction cycle: fold the correction into ph + pl
        const float vv[2] = {v0, v1};
#pragma unroll
        for (int t = 0; t < 2; ++t) {
          if (t == 1 && !two) continue;
          float sh, sl, nh, nl;
          two_sum(a.ph[q + t], vv[t], sh, sl);
          sl += a.pl[q + t];
          fast_two_sum(sh, sl, nh, nl);
          if (wl_in(q + t, g.nc, WL_DBG_SWEEP)) {
            a.ph[q + t] = nh;
            a.pl[q + t] = nl;
          }
        }
      } else if (two && (n0 & 1) == 0) {
        st_pair(xout, q, v0, v1);
      } else {
        if (wl_in(q + (two ? 1 : 0), g.nc, WL_DBG_SWEEP)) {
          xout[q] = from_f<T>(v0);
          if (two) xout[q + 1] = from_f<T>(v1);
        }
      }
    }
    if (more) load_black(k + 1);
    __syncthreads();
  }
}
template <int D, typename T>
__global__ void __launch_bounds__(256) k_sweep(SweepArgs a) { sweep_body<D, T>(a, blockIdx); }

// Planes per block of the sweep kernels (at most 32 per march): the z-blocking that
// minimises the modelled time, whole waves of blocks (blocks_per_sm resident per SM, the
// kernel's own residency) times the planes a block marches through plus about 1.5 planes
// of prologue and epilogue work.
int sweep_planes_per_block(const Grid& g, int blocks_per_sm) {
  const long long tiles = (long long)((g.n[0] + SW_TX - 1) / SW_TX) * ((g.n[1] + SW_TY - 1) / SW_TY);
  return sweep_planes_for_columns(g.n[2], tiles, blocks_per_sm);
}

// The same for a launch over `tiles` tile columns of n2 planes.
int sweep_planes_for_columns(int n2, long long tiles, int blocks_per_sm) {
  static int nsm = 0;
  if (nsm <= 0) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
        nsm <= 0) {
      cudaGetLastError();
      nsm = 152;
    }
  }
  const long long wave = (long long)blocks_per_sm * nsm;
  int best = 2;
  double best_cost = 1e300;
  for (int tz = 2; tz <= 32; ++tz) {
    const long long nb = tiles * ((n2 + tz - 1) / tz);
    const double cost = (double)((nb + wave - 1) / wave) * (tz + 1.5);
    if (cost < best_cost) {
      best_cost = cost;
      best = tz;
    }
  }
  return best;
}

// resident blocks per SM of the table kernel for a level's storage type (from the
// occupancy calculator once per variant; its register count decides it)
int sweep_table_blocks_per_sm(int D, int stype) {
  static int cache[2][3] = {};
  if (D < 2 || D > 3 || stype < 0 || stype > 2) return SWEEP_BLOCKS_PER_SM;
  int& c = cache[D - 2][stype];
  if (c > 0) return c;
  int n = 0;
  cudaError_t e;
  if (D == 3)
    e = stype == ST_BF16 ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_sweep<3, __nv_bfloat16>, 256, 0)
        : stype == ST_F16 ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_sweep<3, __half>, 256, 0)
                          : cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_sweep<3, float>, 256, 0);
  else
    e = stype == ST_BF16 ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_sweep<2, __nv_bfloat16>, 256, 0)
        : stype == ST_F16 ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_sweep<2, __half>, 256, 0)
                          : cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_sweep<2, float>, 256, 0);
  if (e != cudaSuccess || n <= 0) {
    cudaGetLastError();
    n = SWEEP_BLOCKS_PER_SM;
  }
  return c = n;
}

template <int D>
void launch_sweep_d(const SweepArgs& a, dim3 grd, cudaStream_t s) {
  if (a.stype == ST_BF16)
    k_sweep<D, __nv_bfloat16><<<grd, 256, 0, s>>>(a);
  else if (a.stype == ST_F16)
    k_sweep<D, __half><<<grd, 256, 0, s>>>(a);
  else
    k_sweep<D, float><<<grd, 256, 0, s>>>(a);
}

int launch_sweep(int D, const SweepArgs& a, cudaStream_t s) {
  const Grid& g = a.g;
  if (D == 3) {
    dim3 grd((g.n[0] + SW_TX - 1) / SW_TX, (g.n[1] + SW_TY - 1) / SW_TY, (g.n[2] + a.tz - 1) / a.tz);
    launch_sweep_d<3>(a, grd, s);
  } else {
    dim3 grd((g.n[0] + SW_TX - 1) / SW_TX, (g.n[1] + SW_TY - 1) / SW_TY, 1);
    launch_sweep_d<2>(a, grd, s);
  }
  return 0;
}

// ---------------------------------------------------------------------------
// Coarsest level: Jacobi-preconditioned conjugate gradients in FP64 by one block,
// on B = -A (positive semi-definite) with the right-hand side projected onto the
// range (mean over active cells removed) and the solution returned with zero mean.
__device__ double block_sum_d(double v, double* sh) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  __syncthreads();
  if (l == 0) sh[w] = v;
  __syncthreads();
  double t = 0.0;
  if (threadIdx.x == 0) {
    for (int k = 0; k < (int)(blockDim.x >> 5); ++k) t += sh[k];
    sh[8] = t;
  }
  __syncthreads();
  return sh[8];
}

template <int D>
__global__ void __launch_bounds__(256) k_coarse_cg(CoarseArgs a) {
  __shared__ double sh[9];
  const Grid& g = a.g;
  const long long nc = g.nc;
  double* xr = a.work;
  double* rr = a.work + nc;
  double* pr = a.work + 2 * nc;
  double* ap = a.work + 3 * nc;
  double* dgv = a.work + 4 * nc;
  const long long st[3] = {1, (long long)g.n[0], (long long)g.n[0] * g.n[1]};
  auto coords = [&](long long q, int* I) {
    I[0] = (int)(q % g.n[0]);
    long long t = q / g.n[0];
    I[1] = (int)(t % g.n[1]);
    I[2] = (int)(t / g.n[1]);
  };
  // B v at cell q (B = -A)
  auto applyB = [&](const double* v, long long q) -> double {
    int I[3];
    coords(q, I);
    double s = 0.0;
#pragma unroll
    for (int c = 0; c < D; ++c) {
      bool has;
      long long qu = nb_up(g, c, I[c], q, st[c], has);
      long long qm = nb_dn(g, c, I[c], q, st[c]);
      if (!wl_in(qu, g.nc, WL_DBG_RESID)) qu = q;
      if (!wl_in(qm, g.nc, WL_DBG_RESID)) qm = q;
      const double Lu = has ? (double)a.L[c][qu] : 0.0;
      const double Ll = (double)a.L[c][q];
      s += Lu * (v[q] - v[qu]) + Ll * (v[q] - v[qm]);
    }
    return s;
  };
  double bs = 0.0, cnt = 0.0;
  for (long long q = threadIdx.x; q < nc; q += blockDim.x) {
    int I[3];
    coords(q, I);
    double dg = 0.0;
#pragma unroll
    for (int c = 0; c < D; ++c) {
      bool has;
      const long long qu = nb_up(g, c, I[c], q, st[c], has);
      dg += (has ? (double)a.L[c][qu] : 0.0) + (double)a.L[c][q];
    }
    dgv[q] = dg;
    xr[q] = 0.0;
    if (dg > 0.0) {
      bs += (double)a.z[q];
      cnt += 1.0;
    }
  }
  bs = block_sum_d(bs, sh);
  cnt = block_sum_d(cnt, sh);
  const double mean = cnt > 0.0 ? bs / cnt : 0.0;
  double rz = 0.0, bb = 0.0;
  for (long long q = threadIdx.x; q < nc; q += blockDim.x) {
    if (dgv[q] > 0.0) {
      const double r = -((double)a.z[q] - mean);  // b - B*0 with b = -(z - mean)
      rr[q] = r;
      const double zz = r / dgv[q];
      pr[q] = zz;
      rz += r * zz;
      bb += r * r;
    } else {
      rr[q] = 0.0;
      pr[q] = 0.0;
    }
  }
  rz = block_sum_d(rz, sh);
  bb = block_sum_d(bb, sh);
  if (bb > 0.0) {
    for (int it = 0; it < a.maxit; ++it) {
      __syncthreads();
      double pap = 0.0;
      for (long long q = threadIdx.x; q < nc; q += blockDim.x) {
        const double s = (dgv[q] > 0.0) ? applyB(pr, q) : 0.0;
        ap[q] = s;
        pap += pr[q] * s;
      }
      pap = block_sum_d(pap, sh);
      if (!(pap > 0.0)) break;
      const double alpha = rz / pap;
      double r2 = 0.0;
      for (long long q = threadIdx.x; q < nc; q += blockDim.x) {
        xr[q] += alpha * pr[q];
        rr[q] -= alpha * ap[q];
        r2 += rr[q] * rr[q];
      }
      r2 = block_sum_d(r2, sh);
      if (r2 <= a.rtol * a.rtol * bb) break;
      double rz2 = 0.0;
      for (long long q = threadIdx.x; q < nc; q += blockDim.x) {
        const double zz = (dgv[q] > 0.0) ? rr[q] / dgv[q] : 0.0;
        ap[q] = zz;
        rz2 += rr[q] * zz;
      }
      rz2 = block_sum_d(rz2, sh);
      const double beta = rz2 / rz;
      rz = rz2;
      for (long long q = threadIdx.x; q < nc; q += blockDim.x) pr[q] = ap[q] + beta * pr[q];
    }
  }
  __syncthreads();
  double xs = 0.0;
  for (long long q = threadIdx.x; q < nc; q += blockDim.x)
    if (dgv[q] > 0.0) xs += xr[q];
  xs = block_sum_d(xs, sh);
  const double xm = cnt > 0.0 ? xs / cnt : 0.0;
  for (long long q = threadIdx.x; q < nc; q += blockDim.x) a.x[q] = (dgv[q] > 0.0) ? (float)(xr[q] - xm) : 0.f;
}

int launch_coarse(int D, const CoarseArgs& a, cudaStream_t s) {
  if (D == 3)
    k_coarse_cg<3><<<1, 256, 0, s>>>(a);
  else
    k_coarse_cg<2><<<1, 256, 0, s>>>(a);
  return 0;
}

// ---------------------------------------------------------------------------
// k_correct: u_c[I] -= w dt L_c[I] (p[I] - p[I-e_c]) (the pressure-gradient loop of
// Section 2, all components in one pass) and, after the last projection of a step,
// the CFL out-flux max_I sum_c max(0, u_c[I+e_c]) + max(0, -u_c[I]) of the corrected
// field (upper faces corrected on the fly, so no second pass).  32 x 8 columns per
// block walking CR_Z planes; one atomic per block.
constexpr int CR_Z = 4;

template <int D>
__device__ __forceinline__ void correct_body(const CorrArgs& a, const uint3 bid) {
  __shared__ unsigned s_m[8];
  const Grid& g = a.g;
  const int tid = threadIdx.x, tx = tid & 31, ty = tid >> 5;
  const int i = bid.x * 32 + tx, j = bid.y * 8 + ty;
  const bool inxy = i < g.n[0] && j < g.n[1];
  const int kb = (D == 3) ? bid.z * CR_Z : 0;
  const int ke = (D == 3) ? min(kb + CR_Z, g.n[2]) : 1;
  const float s = a.w * a.st->dtf;
  const long long st[3] = {1, (long long)g.n[0], (long long)g.n[0] * g.n[1]};
  // pressure difference p[qa] - p[qb]; for the double-float pressure the hi parts
  // are subtracted first (exact when they are within a factor 2 of each other)
  auto dp = [&](long long qa, long long qb) -> float {
    if (a.ph) return (__ldg(a.ph + qa) - __ldg(a.ph + qb)) + (__ldg(a.pl + qa) - __ldg(a.pl + qb));
    return __ldg(a.x + qa) - __ldg(a.x + qb);
  };
  float m = 0.f;
  for (int k = kb; k < ke && inxy; ++k) {
    const long long q = cell_index(g, i, j, k);
    const int I[3] = {i, j, k};
    float mc = 0.f;
#pragma unroll
    for (int c = 0; c < D; ++c) {
      const long long qm = nb_dn(g, c, I[c], q, st[c]);
      const float Ll = __ldg(a.L[c] + q);
      const float ulo = __ldg(a.u_in[c] + q) - s * Ll * dp(q, qm);
      if (wl_in(q, g.nc, WL_DBG_CORRECT)) a.u_out[c][q] = ulo;
      if (a.cfl) {
        bool has;
        const long long qu = nb_up(g, c, I[c], q, st[c], has);
        const float uup = has ? __ldg(a.u_in[c] + qu) - s * __ldg(a.L[c] + qu) * dp(qu, q)
                              : ((c == 0 && g.exit) ? __ldg(a.u_in[0] + exit_index(g, I[1], I[2])) : g.U[c]);
        mc += fmaxf(0.f, uup) + fmaxf(0.f, -ulo);
      }
    }
    m = fmaxf(m, mc);
  }
  if (a.cfl) {
    const unsigned mb = block_max_bits<256>(__float_as_uint(fabsf(m)), s_m);
    if (tid == 0) atomicMax(&a.st->cfl_bits, mb);
  }
}
template <int D>
__global__ void __launch_bounds__(256) k_correct(CorrArgs a) { correct_body<D>(a, blockIdx); }

// 3-D correction (+ CFL) with one thread per cell column marching up C3_Z planes:
// the column's pressure (hi, lo), z-velocity and z-face coefficients sit in a window
// over planes k-1..k+1, x neighbours come from the adjacent lanes by shuffles, and
// the in-plane neighbour offsets are fixed per thread.  Same arithmetic as k_correct.
constexpr int C3_Z = 16;

template <bool DF, bool CFL>
__device__ __forceinline__ void correct3_body(const CorrArgs& a, const uint3 bid) {
  __shared__ unsigned s_m[8];
  const Grid& g = a.g;
  const int tid = threadIdx.x, lane = tid & 31, ty = tid >> 5;
  const int i = bid.x * 32 + lane, j = bid.y * 8 + ty;
  const int n0 = g.n[0], n1 = g.n[1], n2 = g.n[2];
  const bool inxy = i < n0 && j < n1;
  const bool per0 = is_per(g, 0), per1 = is_per(g, 1), per2 = is_per(g, 2);
  const long long nn = (long long)n0 * n1;
  const int kb = bid.z * C3_Z, ke = min(kb + C3_Z, n2);
  const int ic = min(i, n0 - 1), jc = min(j, n1 - 1);
  const long long c0 = ic + (long long)n0 * jc;
  const long long cxm = ((ic > 0) ? ic - 1 : (per0 ? n0 - 1 : ic)) + (long long)n0 * jc;
  const long long cxp = ((ic + 1 < n0) ? ic + 1 : (per0 ? 0 : ic)) + (long long)n0 * jc;
  const long long cym = ic + (long long)n0 * ((jc > 0) ? jc - 1 : (per1 ? n1 - 1 : jc));
  const long long cyp = ic + (long long)n0 * ((jc + 1 < n1) ? jc + 1 : (per1 ? 0 : jc));
  const bool hxp = (ic + 1 < n0) || per0, hyp = (jc + 1 < n1) || per1;
  const bool edge_xm = (lane == 0) || (i == 0), edge_xp = (lane == 31) || (i + 1 >= n0);
  auto zoff = [&](int k) -> long long {
    if (k < 0) return (per2 ? k + n2 : 0) * nn;
    if (k >= n2) return (per2 ? k - n2 : n2 - 1) * nn;
    return (long long)k * nn;
  };
  const float s = a.w * a.st->dtf;
  const float* P = DF ? a.ph : a.x;
  // p[qa] - p[qb] from (hi, lo) pairs, hi parts first
  auto dp = [&](float ha, float la, float hb, float lb) -> float { return DF ? (ha - hb) + (la - lb) : ha - hb; };
  float wh[3], wl[3];
  {
    const long long o[3] = {zoff(kb - 1), zoff(kb), zoff(kb + 1)};
#pragma unroll
    for (int t = 0; t < 3; ++t) {
      wh[t] = __ldg(P + o[t] + c0);
      wl[t] = DF ? __ldg(a.pl + o[t] + c0) : 0.f;
    }
  }
  // per-plane operands, loaded two planes ahead of their use: y neighbour's pressure,
  // face coefficients and velocity of the cell, and (CFL) the upper y face's operands
  struct PlaneVals {
    float ymh, yml, L0, L1, L2, u0, u1, u2, yph, ypl, uyp, Lyp;
  };
  auto load_plane = [&](int k, PlaneVals& v) {
    const long long ok = zoff(k), q = ok + c0;
    v.ymh = __ldg(P + ok + cym);
    v.yml = DF ? __ldg(a.pl + ok + cym) : 0.f;
    v.L0 = __ldg(a.L[0] + q);
    v.L1 = __ldg(a.L[1] + q);
    v.L2 = __ldg(a.L[2] + q);
    v.u0 = __ldg(a.u_in[0] + q);
    v.u1 = __ldg(a.u_in[1] + q);
    v.u2 = __ldg(a.u_in[2] + q);
    if (CFL && hyp) {
      v.yph = __ldg(P + ok + cyp);
      v.ypl = DF ? __ldg(a.pl + ok + cyp) : 0.f;
      v.uyp = __ldg(a.u_in[1] + ok + cyp);
      v.Lyp = __ldg(a.L[1] + ok + cyp);
    }
  };
  PlaneVals cur, nxt;
  load_plane(kb, cur);
  load_plane(kb + 1, nxt);
  float m = 0.f;
  for (int k = kb; k < ke; ++k) {
    const long long ok = zoff(k);
    const long long q = ok + c0;
    // plane k+2 in flight (past the column's end an in-range plane whose values go
    // unused; the upper z face of plane k reads the next plane's own velocity and
    // coefficient)
    PlaneVals nx2;
    load_plane(k + 2, nx2);
    float xmh = __shfl_up_sync(0xffffffffu, wh[1], 1), xml = __shfl_up_sync(0xffffffffu, wl[1], 1);
    if (edge_xm) {
      xmh = __ldg(P + ok + cxm);
      xml = DF ? __ldg(a.pl + ok + cxm) : 0.f;
    }
    const float lo0 = cur.u0 - s * cur.L0 * dp(wh[1], wl[1], xmh, xml);
    const float lo1 = cur.u1 - s * cur.L1 * dp(wh[1], wl[1], cur.ymh, cur.yml);
    const float lo2 = cur.u2 - s * cur.L2 * dp(wh[1], wl[1], wh[0], wl[0]);
    if (inxy) {
      if (wl_in(q, g.nc, WL_DBG_CORRECT)) {
        a.u_out[0][q] = lo0;
        a.u_out[1][q] = lo1;
        a.u_out[2][q] = lo2;
      }
    }
    if (CFL) {
      // corrected upper faces: x from the next lane, y loaded, z from the window
      float uxp = __shfl_down_sync(0xffffffffu, cur.u0, 1), Lxp = __shfl_down_sync(0xffffffffu, cur.L0, 1);
      float xph = __shfl_down_sync(0xffffffffu, wh[1], 1), xpl = __shfl_down_sync(0xffffffffu, wl[1], 1);
      if (edge_xp) {
        uxp = __ldg(a.u_in[0] + ok + cxp);
        Lxp = __ldg(a.L[0] + ok + cxp);
        xph = __ldg(P + ok + cxp);
        xpl = DF ? __ldg(a.pl + ok + cxp) : 0.f;
      }
      const float up0 = hxp ? uxp - s * Lxp * dp(xph, xpl, wh[1], wl[1])
                            : (g.exit ? __ldg(a.u_in[0] + exit_index(g, jc, k)) : g.U[0]);
      const float up1 = hyp ? cur.uyp - s * cur.Lyp * dp(cur.yph, cur.ypl, wh[1], wl[1]) : g.U[1];
      const float up2 = (k + 1 < n2 || per2) ? nxt.u2 - s * nxt.L2 * dp(wh[2], wl[2], wh[1], wl[1]) : g.U[2];
      float mc = 0.f;
      mc += fmaxf(0.f, up0) + fmaxf(0.f, -lo0);
      mc += fmaxf(0.f, up1) + fmaxf(0.f, -lo1);
      mc += fmaxf(0.f, up2) + fmaxf(0.f, -lo2);
      if (inxy) m = fmaxf(m, mc);
    }
    if (k + 1 < ke) {
      const long long o2 = zoff(k + 2);
      wh[0] = wh[1];
      wl[0] = wl[1];
      wh[1] = wh[2];
      wl[1] = wl[2];
      wh[2] = __ldg(P + o2 + c0);
      wl[2] = DF ? __ldg(a.pl + o2 + c0) : 0.f;
    }
    cur = nxt;
    nxt = nx2;
  }
  if (CFL) {
    const unsigned mb = block_max_bits<256>(__float_as_uint(fabsf(m)), s_m);
    if (tid == 0) atomicMax(&a.st->cfl_bits, mb);
  }
}
template <bool DF, bool CFL>
__global__ void __launch_bounds__(256) k_correct3(CorrArgs a) { correct3_body<DF, CFL>(a, blockIdx); }

int launch_correct(int D, const CorrArgs& a, cudaStream_t s) {
  const Grid& g = a.g;
  if (D == 3 && a.u_in[0] != a.u_out[0]) {  // out of place (in place keeps the plain kernel)
    dim3 grd((g.n[0] + 31) / 32, (g.n[1] + 7) / 8, (g.n[2] + C3_Z - 1) / C3_Z);
    const bool df = a.ph != nullptr;
    if (df && a.cfl)
      k_correct3<true, true><<<grd, 256, 0, s>>>(a);
    else if (df)
      k_correct3<true, false><<<grd, 256, 0, s>>>(a);
    else if (a.cfl)
      k_correct3<false, true><<<grd, 256, 0, s>>>(a);
    else
      k_correct3<false, false><<<grd, 256, 0, s>>>(a);
    return 0;
  }
  if (D == 3) {
    dim3 grd((g.n[0] + 31) / 32, (g.n[1] + 7) / 8, (g.n[2] + CR_Z - 1) / CR_Z);
    k_correct<3><<<grd, 256, 0, s>>>(a);
  } else {
    dim3 grd((g.n[0] + 31) / 32, (g.n[1] + 7) / 8, 1);
    k_correct<2><<<grd, 256, 0, s>>>(a);
  }
  return 0;
}

// CFL out-flux maximum of a velocity field without a correction (initial dt).
template <int D>
__global__ void __launch_bounds__(256) k_cfl_only(Grid g, const float* u0, const float* u1, const float* u2,
                                                   DevState* st) {
  __shared__ unsigned s_m[8];
  const float* u[3] = {u0, u1, u2};
  const long long q = (long long)blockIdx.x * 256 + threadIdx.x;
  float m = 0.f;
  if (q < g.nc) {
    const long long stv[3] = {1, (long long)g.n[0], (long long)g.n[0] * g.n[1]};
    int I[3];
    I[0] = (int)(q % g.n[0]);
    long long t = q / g.n[0];
    I[1] = (int)(t % g.n[1]);
    I[2] = (int)(t / g.n[1]);
#pragma unroll
    for (int c = 0; c < D; ++c) {
      bool has;
      const long long qu = nb_up(g, c, I[c], q, stv[c], has);
      const float uup = has ? u[c][qu] : ((c == 0 && g.exit) ? u[0][exit_index(g, I[1], I[2])] : g.U[c]);
      m += fmaxf(0.f, uup) + fmaxf(0.f, -u[c][q]);
    }
  }
  const unsigned mb = block_max_bits<256>(__float_as_uint(fabsf(m)), s_m);
  if (threadIdx.x == 0) atomicMax(&st->cfl_bits, mb);
}

int launch_cfl_only(int D, const Grid& g, const float* const* u, DevState* st, cudaStream_t s) {
  const int nb = (int)((g.nc + 255) / 256);
  if (D == 3)
    k_cfl_only<3><<<nb, 256, 0, s>>>(g, u[0], u[1], u[2], st);
  else
    k_cfl_only<2><<<nb, 256, 0, s>>>(g, u[0], u[1], u[1], st);
  return 0;
}

// ---------------------------------------------------------------------------
// Device-side control of the V-cycle loop: reads the residual maximum of the pass
// just finished, converts it to x units (times w dt), counts V-cycles, records the
// outcome and sets the graph's while-condition.  No host round trip.
__device__ __forceinline__ bool decide_state(DevState* st, int first, int proj, float w, double tol, int maxit) {
  const float nrm = __uint_as_float(st->norm_bits);
  st->norm_bits = 0u;
  // scale of the 16-bit coarse levels for the cycle that corrects this residual: its
  // max-norm maps to [2^-6, 2^-5), which leaves FP16 room for the corrections (a smooth
  // error is at most ~(n/pi)^2 times its residual) and keeps the residual normal
  if (nrm > 0.f && isfinite(nrm)) st->cs_used = min(max(-ilogbf(nrm) - 6, -100), 100);
  const float res = (float)((double)nrm * (double)w * st->dt);
  if (first) {
    st->iter = 0;
  } else {
    st->iter += 1;
    st->total_vcycles += 1;
  }
  const bool finite = isfinite(res);
  const bool cont = finite && (double)res > tol && st->iter < maxit;
  if (!finite) st->status |= 1;
  if (!cont) {
    st->last_iters[proj] = st->iter;
    st->last_res[proj] = res;
    if (finite && (double)res > tol) st->status |= 2;
    if (!(res <= st->worst_res)) st->worst_res = res;
  }
  st->res_x = res;
  st->cond = cont ? 1 : 0;
  return cont;
}
__global__ void k_decide(DevState* st, cudaGraphConditionalHandle h, int use_handle, int first, int proj, float w,
                         double tol, int maxit) {
  const bool cont = decide_state(st, first, proj, w, tol, maxit);
  if (use_handle) cudaGraphSetConditional(h, cont ? 1u : 0u);
}

int launch_decide(DevState* st, cudaGraphConditionalHandle h, int use_handle, int first, int proj, float w,
                  double tol, int maxit, cudaStream_t s) {
  k_decide<<<1, 1, 0, s>>>(st, h, use_handle, first, proj, w, tol, maxit);
  return 0;
}

// End of a step: advance the clock and take the next dt from the CFL maximum
// (dt = min(dt_cap, 1/(max out-flux + 2 D nu)), CFL! of Table 2), or keep dt fixed.
// advance = 0: only set dt (initial condition).
__device__ __forceinline__ void step_end_state(DevState* st, int D, double nu, double dt_cap, double dt_fixed,
                                               int advance, double* ring, int cap, const double* F) {
  const double used = st->dt;
  if (advance) {
    st->time += used;
    st->steps += 1;
    if (ring && cap > 0) {
      // the step's record: step, time, dt, V-cycles and final residuals of both
      // projections, CFL out-flux maximum, then (metrics on) KE, max |div u|, force
      double* r = ring + (size_t)(st->mcount % cap) * NMETRIC;
      const double nan = __longlong_as_double(0x7ff8000000000000ll);
      r[0] = (double)st->steps;
      r[1] = st->time;
      r[2] = used;
      r[3] = st->last_iters[0];
      r[4] = st->last_iters[1];
      r[5] = st->last_res[0];
      r[6] = st->last_res[1];
      r[7] = (double)__uint_as_float(st->cfl_bits);
      r[8] = F ? st->ke : nan;
      r[9] = F ? (double)__uint_as_float(st->maxdiv_bits) : nan;
      for (int d = 0; d < 3; ++d) r[10 + d] = (F && d < D) ? F[d] : nan;
      st->mcount += 1;
    }
  }
  double dn;
  if (dt_fixed > 0.0) {
    dn = dt_fixed;
  } else {
    const double m = (double)__uint_as_float(st->cfl_bits);
    dn = fmin(dt_cap, 1.0 / (m + 2.0 * D * nu));
  }
  if (!isfinite(dn) || !(dn > 0.0)) {
    st->status |= 1;
    dn = used;
  }
  st->dt = dn;
  st->dtf = (float)dn;
  st->inv_dtf = (float)(1.0 / dn);
  st->cfl_bits = 0u;
}
__global__ void k_step_end(DevState* st, int D, double nu, double dt_cap, double dt_fixed, int advance,
                           double* ring, int cap, const double* F) {
  step_end_state(st, D, nu, dt_cap, dt_fixed, advance, ring, cap, F);
}

// refresh the FP32 copies after the host wrote dt
__global__ void k_sync_dt(DevState* st) {
  st->dtf = (float)st->dt;
  st->inv_dtf = (float)(1.0 / st->dt);
}

int launch_sync_dt(DevState* st, cudaStream_t s) {
  k_sync_dt<<<1, 1, 0, s>>>(st);
  return 0;
}

int launch_step_end(DevState* st, int D, double nu, double dt_cap, double dt_fixed, double* ring, int cap,
                    const double* F, cudaStream_t s) {
  k_step_end<<<1, 1, 0, s>>>(st, D, nu, dt_cap, dt_fixed, 1, ring, cap, F);
  return 0;
}

int launch_set_dt_from_cfl(DevState* st, int D, double nu, double dt_cap, double dt_fixed, cudaStream_t s) {
  k_step_end<<<1, 1, 0, s>>>(st, D, nu, dt_cap, dt_fixed, 0, nullptr, 0, nullptr);
  return 0;
}

// Metrics of a velocity: per block the FP64 sum of u_c^2 over its cells (grid-stride, a
// fixed pattern, then a fixed-order block sum) and the running max |div u| (atomic max of
// float bits: order-free).  div u = sum_c u_c[I+e_c] - u_c[I], the upper face of a
// non-periodic side being U_c (the stored exit plane for x with a convective exit).
template <int D>
__global__ void __launch_bounds__(256) k_metrics_u(Grid g, const float* u0, const float* u1, const float* u2,
                                                    DevState* st, double* partials) {
  __shared__ double sh[8];
  __shared__ unsigned sm[8];
  const float* u[3] = {u0, u1, u2};
  const long long st2[3] = {1, (long long)g.n[0], (long long)g.n[0] * g.n[1]};
  double e = 0.0;
  unsigned mx = 0u;
  for (long long q = (long long)blockIdx.x * 256 + threadIdx.x; q < g.nc; q += (long long)gridDim.x * 256) {
    int I[3];
    I[0] = (int)(q % g.n[0]);
    const long long t = q / g.n[0];
    I[1] = (int)(t % g.n[1]);
    I[2] = (int)(t / g.n[1]);
    float div = 0.f;
#pragma unroll
    for (int c = 0; c < D; ++c) {
      const float v = u[c][q];
      e += (double)v * (double)v;
      float up;
      if (I[c] + 1 < g.n[c])
        up = u[c][q + st2[c]];
      else if (is_per(g, c))
        up = u[c][q - (long long)(g.n[c] - 1) * st2[c]];
      else if (c == 0 && g.exit)
        up = u[0][exit_index(g, I[1], I[2])];
      else
        up = g.U[c];
      div += up - v;
    }
    mx = max(mx, __float_as_uint(fabsf(div)));
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    e += __shfl_xor_sync(0xffffffffu, e, o);
    mx = max(mx, __shfl_xor_sync(0xffffffffu, mx, o));
  }
  if ((threadIdx.x & 31) == 0) {
    sh[threadIdx.x >> 5] = e;
    sm[threadIdx.x >> 5] = mx;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double a = 0.0;
    unsigned m = 0u;
    for (int w = 0; w < 8; ++w) {
      a += sh[w];
      m = max(m, sm[w]);
    }
    partials[blockIdx.x] = a;
    atomicMax(&st->maxdiv_bits, m);
  }
}

// sum of the npart partials in a fixed order (strided per thread, then a fixed tree)
__global__ void __launch_bounds__(256) k_metrics_final(DevState* st, const double* partials, int npart, double inv_n) {
  __shared__ double sh[256];
  double a = 0.0;
  for (int b = threadIdx.x; b < npart; b += 256) a += partials[b];
  sh[threadIdx.x] = a;
  __syncthreads();
  for (int w = 128; w > 0; w >>= 1) {
    if (threadIdx.x < w) sh[threadIdx.x] += sh[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) st->ke = 0.5 * sh[0] * inv_n;
}

__global__ void k_clear_maxdiv(DevState* st) { st->maxdiv_bits = 0u; }

int launch_metrics_u(int D, const Grid& g, const float* const* u, DevState* st, double* partials, int npart,
                     cudaStream_t s) {
  k_clear_maxdiv<<<1, 1, 0, s>>>(st);
  if (D == 3)
    k_metrics_u<3><<<npart, 256, 0, s>>>(g, u[0], u[1], u[2], st, partials);
  else
    k_metrics_u<2><<<npart, 256, 0, s>>>(g, u[0], u[1], u[1], st, partials);
  k_metrics_final<<<1, 256, 0, s>>>(st, partials, npart, 1.0 / (double)g.nc);
  return 0;
}

// ---------------------------------------------------------------------------
// Body measure (once per sim): L_c = mu0 = K0(d/eps) at each lower c-face, with d
// the signed distance of the face centre (Section 2), zero on non-periodic boundary
// faces.  FP64 evaluation, stored as float.
template <int D>
__global__ void k_measure(Grid g, Body b, float* L0, float* L1, float* L2) {
  float* L[3] = {L0, L1, L2};
  const long long q = (long long)blockIdx.x * 256 + threadIdx.x;
  if (q >= g.nc) return;
  int I[3];
  I[0] = (int)(q % g.n[0]);
  long long t = q / g.n[0];
  I[1] = (int)(t % g.n[1]);
  I[2] = (int)(t / g.n[1]);
#pragma unroll
  for (int c = 0; c < D; ++c) {
    double v = 1.0;
    if (b.kind != 0) {
      double x[3] = {I[0] + 0.5, I[1] + 0.5, I[2] + 0.5}, n[3];
      x[c] -= 0.5;
      const double d = body_sdf<D>(b, x, n);
      v = kernel_K0(d / b.eps);
    }
    if (!is_per(g, c) && I[c] == 0) v = 0.0;
    L[c][q] = (float)v;
  }
}

int launch_measure(int D, const Grid& g, const Body& b, float* const* L, cudaStream_t s) {
  const int nb = (int)((g.nc + 255) / 256);
  if (D == 3)
    k_measure<3><<<nb, 256, 0, s>>>(g, b, L[0], L[1], L[2]);
  else
    k_measure<2><<<nb, 256, 0, s>>>(g, b, L[0], L[1], L[1]);
  return 0;
}

// Coarse face coefficient = half the sum of the 2^(D-1) fine faces it covers.
template <int D>
__global__ void k_coarsen(Grid f, const float* F0, const float* F1, const float* F2, Grid c, float* C0, float* C1,
                          float* C2) {
  const float* Fl[3] = {F0, F1, F2};
  float* Cl[3] = {C0, C1, C2};
  const long long q = (long long)blockIdx.x * 256 + threadIdx.x;
  if (q >= c.nc) return;
  int J[3];
  J[0] = (int)(q % c.n[0]);
  long long t = q / c.n[0];
  J[1] = (int)(t % c.n[1]);
  J[2] = (int)(t / c.n[1]);
#pragma unroll
  for (int cc = 0; cc < D; ++cc) {
    double sum = 0.0;
    const int a0 = (cc == 0) ? 1 : 2, a1 = (cc == 1) ? 1 : 2, a2 = (D == 3 && cc != 2) ? 2 : 1;
    for (int dk = 0; dk < a2; ++dk)
      for (int dj = 0; dj < a1; ++dj)
        for (int di = 0; di < a0; ++di) {
          const int I0 = 2 * J[0] + di, I1 = 2 * J[1] + dj, I2 = (D == 3) ? 2 * J[2] + dk : 0;
          sum += (double)Fl[cc][(long long)I0 + (long long)f.n[0] * ((long long)I1 + (long long)f.n[1] * I2)];
        }
    Cl[cc][q] = (float)(0.5 * sum);
  }
}

int launch_coarsen(int D, const Grid& fine, const float* const* Lf, const Grid& coarse, float* const* Lc,
                   cudaStream_t s) {
  const int nb = (int)((coarse.nc + 255) / 256);
  if (D == 3)
    k_coarsen<3><<<nb, 256, 0, s>>>(fine, Lf[0], Lf[1], Lf[2], coarse, Lc[0], Lc[1], Lc[2]);
  else
    k_coarsen<2><<<nb, 256, 0, s>>>(fine, Lf[0], Lf[1], Lf[1], coarse, Lc[0], Lc[1], Lc[1]);
  return 0;
}

// Initial velocity: kind 0 uniform U; kind 1 Taylor-Green vortex (k = 2 pi / n_0),
// each component sampled at its own face centres.
template <int D>
__global__ void k_set_ic(Grid g, int kind, double amp, float* u0, float* u1, float* u2) {
  float* u[3] = {u0, u1, u2};
  const long long q = (long long)blockIdx.x * 256 + threadIdx.x;
  if (q >= g.nc) return;
  int I[3];
  I[0] = (int)(q % g.n[0]);
  long long t = q / g.n[0];
  I[1] = (int)(t % g.n[1]);
  I[2] = (int)(t / g.n[1]);
  const double kw = 2.0 * 3.141592653589793 / g.n[0];
#pragma unroll
  for (int c = 0; c < D; ++c) {
    double v = g.U[c];
    if (kind == 1) {
      double x[3] = {I[0] + 0.5, I[1] + 0.5, I[2] + 0.5};
      x[c] -= 0.5;
      const double cz = (D == 3) ? cos(kw * x[2]) : 1.0;
      if (c == 0)
        v = amp * sin(kw * x[0]) * cos(kw * x[1]) * cz;
      else if (c == 1)
        v = -amp * cos(kw * x[0]) * sin(kw * x[1]) * cz;
      else
        v = 0.0;
    }
    if (!is_per(g, c) && I[c] == 0) v = g.U[c];  // boundary faces always carry U
    u[c][q] = (float)v;
  }
}

int launch_set_ic(int D, const Grid& g, int kind, double amp, float* const* u, cudaStream_t s) {
  const int nb = (int)((g.nc + 255) / 256);
  if (D == 3)
    k_set_ic<3><<<nb, 256, 0, s>>>(g, kind, amp, u[0], u[1], u[2]);
  else
    k_set_ic<2><<<nb, 256, 0, s>>>(g, kind, amp, u[0], u[1], u[1]);
  return 0;
}

// ---------------------------------------------------------------------------
// Pressure force F_d = -sum_cells (p - pbar) n_d K_eps(d) (FP64).  Pass 1: per-block
// partial sums of p and of the active-cell count over a fixed grid (deterministic).
// Pass 2 (one block): pbar from the partials in a fixed order, then the band sum over
// the body's bounding box.
template <int D>
__global__ void __launch_bounds__(256) k_force_partials(Grid g, const float* p, const float* pl, const float* L0,
                                                         const float* L1, const float* L2, double* part) {
  __shared__ double sh[9];
  const float* L[3] = {L0, L1, L2};
  const long long st[3] = {1, (long long)g.n[0], (long long)g.n[0] * g.n[1]};
  double sp = 0.0, sc = 0.0;
  for (long long q = (long long)blockIdx.x * 256 + threadIdx.x; q < g.nc; q += (long long)gridDim.x * 256) {
    int I[3];
    I[0] = (int)(q % g.n[0]);
    long long t = q / g.n[0];
    I[1] = (int)(t % g.n[1]);
    I[2] = (int)(t / g.n[1]);
    float dg = 0.f;
#pragma unroll
    for (int c = 0; c < D; ++c) {
      bool has;
      const long long qu = nb_up(g, c, I[c], q, st[c], has);
      dg += (has ? L[c][qu] : 0.f) + L[c][q];
    }
    if (dg > 0.f) {
      sp += (double)p[q] + (pl ? (double)pl[q] : 0.0);
      sc += 1.0;
    }
  }
  sp = block_sum_d(sp, sh);
  sc = block_sum_d(sc, sh);
  if (threadIdx.x == 0) {
    part[2 * blockIdx.x] = sp;
    part[2 * blockIdx.x + 1] = sc;
  }
}

template <int D>
__global__ void __launch_bounds__(256) k_force_final(Grid g, Body b, const float* p, const float* pl,
                                                      const double* part, int npart,
                                                      int lo0, int lo1, int lo2, int bx, int by, int bz,
                                                      double* out) {
  __shared__ double sh[9];
  double sp = 0.0, sc = 0.0;
  for (int k = threadIdx.x; k < npart; k += 256) {
    sp += part[2 * k];
    sc += part[2 * k + 1];
  }
  sp = block_sum_d(sp, sh);
  sc = block_sum_d(sc, sh);
  const double pbar = sc > 0.0 ? sp / sc : 0.0;
  double F[3] = {0.0, 0.0, 0.0};
  const long long nbox = (long long)bx * by * bz;
  for (long long t = threadIdx.x; t < nbox; t += 256) {
    const int i = lo0 + (int)(t % bx);
    const long long r = t / bx;
    const int j = lo1 + (int)(r % by);
    const int k = lo2 + (int)(r / by);
    double x[3] = {i + 0.5, j + 0.5, k + 0.5}, n[3];
    const double d = body_sdf<D>(b, x, n);
    if (!(fabs(d) < b.eps)) continue;
    const double K = (1.0 + cospi(d / b.eps)) / (2.0 * b.eps);
    const long long q = cell_index(g, i, j, k);
    const double pp = ((double)p[q] + (pl ? (double)pl[q] : 0.0)) - pbar;
#pragma unroll
    for (int dd = 0; dd < D; ++dd) F[dd] -= pp * n[dd] * K;
  }
  for (int dd = 0; dd < D; ++dd) {
    const double v = block_sum_d(F[dd], sh);
    if (threadIdx.x == 0) out[dd] = v;
  }
  if (threadIdx.x == 0) out[3] = pbar;
}

// viscous force: F_i = sum over cells with |d| < eps of 2 nu S_ij n_j K_eps(d), with the
// strain rate S = (grad u + grad u^T)/2 at the cell centre: du_c/dx_c from the cell's two
// c-faces, du_c/dx_e (e != c) by the central difference of the cell-centred u_c (the mean
// of its two faces); neighbours outside the grid through the BC mapping.  One block, FP64
// accumulation in a fixed order (deterministic).
template <int D>
__global__ void __launch_bounds__(256) k_viscous_force(Grid g, Body b, const float* u0, const float* u1,
                                                        const float* u2, double nu, int lo0, int lo1, int lo2,
                                                        int bx, int by, int bz, double* out) {
  __shared__ double sh[9];
  const float* u[3] = {u0, u1, u2};
  auto U = [&](int c, const int* J) { return (double)load_u_bc<D>(u[c], c, g, J[0], J[1], J[2]); };
  double F[3] = {0.0, 0.0, 0.0};
  const long long nbox = (long long)bx * by * bz;
  for (long long t = threadIdx.x; t < nbox; t += 256) {
    const int i = lo0 + (int)(t % bx);
    const long long r = t / bx;
    const int j = lo1 + (int)(r % by);
    const int k = lo2 + (int)(r / by);
    double x[3] = {i + 0.5, j + 0.5, k + 0.5}, n[3];
    const double d = body_sdf<D>(b, x, n);
    if (!(fabs(d) < b.eps)) continue;
    const double K = (1.0 + cospi(d / b.eps)) / (2.0 * b.eps);
    const int I[3] = {i, j, k};
    double G[3][3] = {{0.0}};  // G[c][e] = du_c/dx_e
#pragma unroll
    for (int c = 0; c < D; ++c)
#pragma unroll
      for (int e = 0; e < D; ++e) {
        if (c == e) {
          int J[3] = {i, j, k};
          J[c] += 1;
          G[c][e] = U(c, J) - U(c, I);
        } else {
          int P0[3] = {i, j, k}, M0[3] = {i, j, k};
          P0[e] += 1;
          M0[e] -= 1;
          int P1[3] = {P0[0], P0[1], P0[2]}, M1[3] = {M0[0], M0[1], M0[2]};
          P1[c] += 1;
          M1[c] += 1;
          G[c][e] = 0.5 * (0.5 * (U(c, P0) + U(c, P1)) - 0.5 * (U(c, M0) + U(c, M1)));
        }
      }
#pragma unroll
    for (int a = 0; a < D; ++a)
#pragma unroll
      for (int e = 0; e < D; ++e) F[a] += 2.0 * nu * 0.5 * (G[a][e] + G[e][a]) * n[e] * K;
  }
  for (int dd = 0; dd < D; ++dd) {
    const double v = block_sum_d(F[dd], sh);
    if (threadIdx.x == 0) out[dd] = v;
  }
}

// cells around the body that can hold band cells: the body's bounding box grown by eps + 1
void force_box(int D, const Grid& g, const Body& b, int* lo, int* hi) {
  double ext = b.r1 + b.eps + 1.0;
  if (b.kind == 2) ext = b.r1 + b.r2 + b.eps + 1.0;
  for (int d = 0; d < 3; ++d) {
    lo[d] = 0;
    hi[d] = 1;
  }
  if (b.kind == 3) {  // the cells bracketing the band, one cell wider
    for (int d = 0; d < D; ++d) {
      lo[d] = std::max(0, b.blo[d] - 1);
      hi[d] = std::min(g.n[d], std::max(b.bhi[d] + 1, lo[d]));
      if (b.bhi[d] <= b.blo[d]) hi[d] = lo[d];
    }
  } else if (b.kind != 0) {
    for (int d = 0; d < D; ++d) {
      lo[d] = (int)fmax(0.0, floor(b.c[d] - ext));
      hi[d] = (int)fmin((double)g.n[d], ceil(b.c[d] + ext) + 1.0);
      if (hi[d] < lo[d]) hi[d] = lo[d];
    }
  } else {
    hi[0] = lo[0];
  }
}

int launch_viscous_force(int D, const Grid& g, const Body& b, const float* const* u, double nu, double* out,
                         cudaStream_t s) {
  int lo[3], hi[3];
  force_box(D, g, b, lo, hi);
  const int bx = hi[0] - lo[0], by = hi[1] - lo[1], bz = hi[2] - lo[2];
  if (D == 3)
    k_viscous_force<3><<<1, 256, 0, s>>>(g, b, u[0], u[1], u[2], nu, lo[0], lo[1], lo[2], bx, by, bz, out);
  else
    k_viscous_force<2><<<1, 256, 0, s>>>(g, b, u[0], u[1], u[1], nu, lo[0], lo[1], lo[2], bx, by, bz, out);
  return 0;
}

int launch_forces(int D, const Grid& g, const Body& b, const float* p, const float* pl, const float* const* L,
                  double* partials, int npart, double* out, cudaStream_t s) {
  if (D == 3)
    k_force_partials<3><<<npart, 256, 0, s>>>(g, p, pl, L[0], L[1], L[2], partials);
  else
    k_force_partials<2><<<npart, 256, 0, s>>>(g, p, pl, L[0], L[1], L[1], partials);
  int lo[3], hi[3];
  force_box(D, g, b, lo, hi);
  const int bx = hi[0] - lo[0], by = hi[1] - lo[1], bz = hi[2] - lo[2];
  if (D == 3)
    k_force_final<3><<<1, 256, 0, s>>>(g, b, p, pl, partials, npart, lo[0], lo[1], lo[2], bx, by, bz, out);
  else
    k_force_final<2><<<1, 256, 0, s>>>(g, b, p, pl, partials, npart, lo[0], lo[1], lo[2], bx, by, bz, out);
  return 0;
}

}  // namespace wl

namespace wl {

// Boundary faces of non-periodic directions always carry U_c (used after a caller
// overwrites the velocity): only the lower boundary plane of each component c is
// touched (blockIdx.y = c), one thread per face of that plane.
template <int D>
__global__ void k_fix_bfaces(Grid g, float* u0, float* u1, float* u2) {
  const int c = blockIdx.y;
  if (c >= D || is_per(g, c)) return;
  float* u = c == 0 ? u0 : (c == 1 ? u1 : u2);
  const int da = c == 0 ? 1 : 0, db = c == 2 ? 1 : 2;  // the plane's two directions
  const long long na = g.n[da], np = na * g.n[db];  // n[2] = 1 in 2-D
  for (long long t = (long long)blockIdx.x * 256 + threadIdx.x; t < np; t += (long long)gridDim.x * 256) {
    int I[3] = {0, 0, 0};
    I[da] = (int)(t % na);
    I[db] = (int)(t / na);
    u[cell_index(g, I[0], I[1], I[2])] = g.U[c];
  }
}

int launch_fix_bfaces(int D, const Grid& g, float* const* u, cudaStream_t s) {
  long long np = 0;  // largest boundary plane
  for (int c = 0; c < D; ++c) np = std::max(np, g.nc / g.n[c]);
  const dim3 grd((unsigned)std::min<long long>((np + 255) / 256, 152LL * 16), (unsigned)D);
  if (D == 3)
    k_fix_bfaces<3><<<grd, 256, 0, s>>>(g, u[0], u[1], u[2]);
  else
    k_fix_bfaces<2><<<grd, 256, 0, s>>>(g, u[0], u[1], u[1]);
  return 0;
}

}  // namespace wl

namespace wl {

// Column j of the pseudo-inverse of the coarsest operator: G e_j = the zero-mean
// solution of A x = e_j - (1/n_active) 1 over the active cells (0 for an inactive
// column), by FP64 Jacobi-preconditioned CG in shared memory, one block per column.
// Built once per sim; applying it is then a small FP64 matrix-vector product.
template <int D>
__global__ void __launch_bounds__(256) k_build_pinv(DenseArgs a) {
  extern __shared__ double sm[];
  __shared__ double sh[9];
  const Grid& g = a.g;
  const int nc = (int)g.nc;
  double* xr = sm;
  double* rr = sm + nc;
  double* pr = sm + 2 * nc;
  double* ap = sm + 3 * nc;
  double* dgv = sm + 4 * nc;
  const int j = blockIdx.x;
  const long long st[3] = {1, (long long)g.n[0], (long long)g.n[0] * g.n[1]};
  auto coords = [&](long long q, int* I) {
    I[0] = (int)(q % g.n[0]);
    long long t = q / g.n[0];
    I[1] = (int)(t % g.n[1]);
    I[2] = (int)(t / g.n[1]);
  };
  double cnt = 0.0;
  for (int q = threadIdx.x; q < nc; q += blockDim.x) {
    int I[3];
    coords(q, I);
    double dg = 0.0;
#pragma unroll
    for (int c = 0; c < D; ++c) {
      bool has;
      const long long qu = nb_up(g, c, I[c], q, st[c], has);
      dg += (has ? (double)a.L[c][qu] : 0.0) + (double)a.L[c][q];
    }
    dgv[q] = dg;
    xr[q] = 0.0;
    cnt += dg > 0.0 ? 1.0 : 0.0;
  }
  cnt = block_sum_d(cnt, sh);
  if (!(dgv[j] > 0.0) || cnt <= 1.0) {
    for (int q = threadIdx.x; q < nc; q += blockDim.x) a.G[(long long)j * nc + q] = 0.0;
    return;
  }
  // B = -A, c = -(e_j - 1/n) on active cells
  double rz = 0.0, bb = 0.0;
  for (int q = threadIdx.x; q < nc; q += blockDim.x) {
    if (dgv[q] > 0.0) {
      const double r = -((q == j ? 1.0 : 0.0) - 1.0 / cnt);
      rr[q] = r;
      pr[q] = r / dgv[q];
      rz += r * pr[q];
      bb += r * r;
    } else {
      rr[q] = 0.0;
      pr[q] = 0.0;
    }
  }
  rz = block_sum_d(rz, sh);
  bb = block_sum_d(bb, sh);
  const int maxit = 4 * nc + 100;
  for (int it = 0; it < maxit; ++it) {
    __syncthreads();
    double pap = 0.0;
    for (int q = threadIdx.x; q < nc; q += blockDim.x) {
      double sv = 0.0;
      if (dgv[q] > 0.0) {
        int I[3];
        coords(q, I);
#pragma unroll
        for (int c = 0; c < D; ++c) {
          bool has;
          const long long qu = nb_up(g, c, I[c], q, st[c], has);
          const long long qm = nb_dn(g, c, I[c], q, st[c]);
          const double Lu = has ? (double)a.L[c][qu] : 0.0;
          const double Ll = (double)a.L[c][q];
          sv += Lu * (pr[q] - pr[qu]) + Ll * (pr[q] - pr[qm]);
        }
      }
      ap[q] = sv;
      pap += pr[q] * sv;
    }
    pap = block_sum_d(pap, sh);
    if (!(pap > 0.0)) break;
    const double alpha = rz / pap;
    double r2 = 0.0;
    for (int q = threadIdx.x; q < nc; q += blockDim.x) {
      xr[q] += alpha * pr[q];
      rr[q] -= alpha * ap[q];
      r2 += rr[q] * rr[q];
    }
    r2 = block_sum_d(r2, sh);
    if (r2 <= 1e-28 * bb) break;
    double rz2 = 0.0;
    for (int q = threadIdx.x; q < nc; q += blockDim.x) {
      const double zz = dgv[q] > 0.0 ? rr[q] / dgv[q] : 0.0;
      ap[q] = zz;
      rz2 += rr[q] * zz;
    }
    rz2 = block_sum_d(rz2, sh);
    const double beta = rz2 / rz;
    rz = rz2;
    for (int q = threadIdx.x; q < nc; q += blockDim.x) pr[q] = ap[q] + beta * pr[q];
  }
  __syncthreads();
  double xs = 0.0;
  for (int q = threadIdx.x; q < nc; q += blockDim.x)
    if (dgv[q] > 0.0) xs += xr[q];
  xs = block_sum_d(xs, sh);
  const double xm = xs / cnt;
  for (int q = threadIdx.x; q < nc; q += blockDim.x)
    a.G[(long long)j * nc + q] = dgv[q] > 0.0 ? xr[q] - xm : 0.0;
}

int launch_build_pinv(int D, const DenseArgs& a, cudaStream_t s) {
  const int nc = (int)a.g.nc;
  const size_t smem = sizeof(double) * 5 * nc;
  if (D == 3)
    k_build_pinv<3><<<nc, 256, smem, s>>>(a);
  else
    k_build_pinv<2><<<nc, 256, smem, s>>>(a);
  return 0;
}

// Coarsest solve x = G z in FP64 (G column-major: coalesced row reads).
__global__ void __launch_bounds__(1024) k_apply_pinv(DenseArgs a) {
  extern __shared__ double zs[];
  const int nc = (int)a.g.nc;
  for (int q = threadIdx.x; q < nc; q += blockDim.x) zs[q] = (double)a.z[q];
  __syncthreads();
  for (int i = threadIdx.x; i < nc; i += blockDim.x) {
    double acc = 0.0;
    // unrolled so that many rows of G are in flight; the sum keeps its order
#pragma unroll 16
    for (int jj = 0; jj < nc; ++jj) acc += __ldg(a.G + (long long)jj * nc + i) * zs[jj];
    a.x[i] = (float)acc;
  }
}

int launch_apply_pinv(const DenseArgs& a, cudaStream_t s) {
  const int nc = (int)a.g.nc;
  int nt = ((nc + 31) / 32) * 32;
  if (nt > 1024) nt = 1024;
  k_apply_pinv<<<1, nt, sizeof(double) * nc, s>>>(a);
  return 0;
}

// ---------------------------------------------------------------------------
// k_vcycle_tail: the small levels of a V-cycle in one block of shared memory.  The same
// arithmetic, in the same order, as the per-level kernels it replaces (restriction of
// RES_RESTRICT: z pairs, then x pairs, then y pairs; k_apply_pinv; k_sweep's
// prolongation and relaxation), without a launch per level and sweep.  Values in shared
// memory carry no per-level storage scale.
size_t vcycle_tail_smem(int D, const int (*n)[3], int nl) {
  size_t b = 0;
  for (int l = 0; l < nl; ++l) b += sizeof(float) * (size_t)(D + 2) * n[l][0] * n[l][1] * n[l][2];
  b = (b + 7) & ~size_t(7);  // the coarsest right-hand side in FP64 follows
  return b + sizeof(double) * (size_t)n[nl - 1][0] * n[nl - 1][1] * n[nl - 1][2];
}

template <int D>
__device__ __forceinline__ void vcycle_tail_body(const TailArgs& a, const uint3 bid) {
  extern __shared__ float tsm[];
  // shared-memory layout: per level, D coefficient fields, z, x (all levels < 2^31 cells)
  auto level_base = [&](int l) {
    int off = 0;
    for (int m = 0; m < l; ++m) off += (D + 2) * a.n[m][0] * a.n[m][1] * a.n[m][2];
    return tsm + off;
  };
  auto ncells = [&](int l) { return a.n[l][0] * a.n[l][1] * a.n[l][2]; };
  const int tid = threadIdx.x;
  for (int l = 0; l < a.nl; ++l) {
    float* b = level_base(l);
    const int nc = ncells(l);
    for (int c = 0; c < D; ++c)
      for (int q = tid; q < nc; q += kTailThreads) b[c * nc + q] = ld_st(a.L[l][c], a.st[l], q);
  }
  {
    const int nc = ncells(0);
    float* z0 = level_base(0) + D * nc;
    for (int q = tid; q < nc; q += kTailThreads) z0[q] = a.zmul * ld_st(a.z, a.st[0], q);
  }
  __syncthreads();
  // restriction down to the coarsest level (the iterate of every tail level starts at 0)
  for (int l = 0; l + 1 < a.nl; ++l) {
    const int f0 = a.n[l][0], f1 = a.n[l][1];
    const int c0 = a.n[l + 1][0], c1 = a.n[l + 1][1];
    const float* zf = level_base(l) + D * ncells(l);
    float* zc = level_base(l + 1) + D * ncells(l + 1);
    const int ncc = ncells(l + 1);
    for (int q = tid; q < ncc; q += kTailThreads) {
      const int I = q % c0, t = q / c0;
      const int J = t % c1, K = t / c1;
      const int b0 = 2 * I + f0 * (2 * J + f1 * 2 * K);  // child (2I, 2J, 2K)
      float sum;
      if (D == 3) {
        const int sz = f0 * f1;
        const float a00 = zf[b0] + zf[b0 + sz];
        const float a10 = zf[b0 + 1] + zf[b0 + 1 + sz];
        const float a01 = zf[b0 + f0] + zf[b0 + f0 + sz];
        const float a11 = zf[b0 + f0 + 1] + zf[b0 + f0 + 1 + sz];
        sum = (a00 + a10) + (a01 + a11);
      } else {
        sum = (zf[b0] + zf[b0 + 1]) + (zf[b0 + f0] + zf[b0 + f0 + 1]);
      }
      zc[q] = sum;
    }
    __syncthreads();
  }
  // coarsest level: x = G z in FP64
  {
    const int lc = a.nl - 1;
    const int nc = ncells(lc);
    float* zc = level_base(lc) + D * nc;
    float* xc = zc + nc;
    // z in FP64 once (the FP64 pipe is the bound here), after the levels' data
    const int nf = (int)(level_base(a.nl) - tsm);
    double* zd = reinterpret_cast<double*>(tsm + ((nf + 1) & ~1));
    for (int i = tid; i < nc; i += kTailThreads) zd[i] = (double)zc[i];
    __syncthreads();
    for (int i = tid; i < nc; i += kTailThreads) {
      double acc = 0.0;
      // unrolled so that many rows of G are in flight; the sum keeps its order
#pragma unroll 16
      for (int jj = 0; jj < nc; ++jj) acc += __ldg(a.G + (long long)jj * nc + i) * zd[jj];
      xc[i] = (float)acc;
    }
    __syncthreads();
  }
  // up: prolong (piecewise constant) and smooth each level
  for (int l = a.nl - 2; l >= 0; --l) {
    const int n0 = a.n[l][0], n1 = a.n[l][1], n2 = a.n[l][2];
    const int nc = n0 * n1 * n2;
    const int c0 = a.n[l + 1][0], c1 = a.n[l + 1][1];
    float* b = level_base(l);
    const float* Lc[3] = {b, b + (D > 1 ? nc : 0), b + (D > 2 ? 2 * nc : nc)};
    const float* zl = b + D * nc;
    float* xl = b + (D + 1) * nc;
    const float* xcoarse = level_base(l + 1) + (D + 1) * ncells(l + 1);
    for (int q = tid; q < nc; q += kTailThreads) {
      const int i = q % n0, t = q / n0;
      const int j = t % n1, k = t / n1;
      xl[q] = 0.f + xcoarse[(i >> 1) + c0 * ((j >> 1) + c1 * (k >> 1))];
    }
    __syncthreads();
    const int st[3] = {1, n0, n0 * n1};
    const int nd[3] = {n0, n1, n2};
    const int h0 = n0 >> 1;  // cells of one colour per row (n0 is even on every level above the coarsest)
    const int nhalf = nc >> 1;
    for (int sw = 0; sw < a.post; ++sw) {
      for (int color = 0; color < 2; ++color) {
        for (int m = tid; m < nhalf; m += kTailThreads) {
          const int row = m / h0;
          const int j = row % n1, k = row / n1;
          const int i = 2 * (m - row * h0) + ((j + k + color) & 1);
          const int q = i + n0 * row;
          const int I[3] = {i, j, k};
          float sum = 0.f, dg = 0.f;
#pragma unroll
          for (int d = 0; d < D; ++d) {
            float Lu = 0.f, xu = 0.f, xd = 0.f;
            if (I[d] + 1 < nd[d]) {
              Lu = Lc[d][q + st[d]];
              xu = xl[q + st[d]];
            } else if ((a.per >> d) & 1u) {
              Lu = Lc[d][q - (nd[d] - 1) * st[d]];
              xu = xl[q - (nd[d] - 1) * st[d]];
            }
            const float Ll = Lc[d][q];
            if (I[d] > 0)
              xd = xl[q - st[d]];
            else if ((a.per >> d) & 1u)
              xd = xl[q + (nd[d] - 1) * st[d]];
            sum = fmaf(Lu, xu, sum);
            sum = fmaf(Ll, xd, sum);
            dg += Lu + Ll;
          }
          xl[q] = (dg > 0.f) ? __fdividef(sum - zl[q], dg) : 0.f;
        }
        __syncthreads();
      }
    }
  }
  {
    const int nc = ncells(0);
    const float* x0 = level_base(0) + (D + 1) * nc;
    for (int q = tid; q < nc; q += kTailThreads) st_st(a.x, a.st[0], q, x0[q]);
  }
}
template <int D>
__global__ void __launch_bounds__(kTailThreads) k_vcycle_tail(TailArgs a) { vcycle_tail_body<D>(a, blockIdx); }

int launch_vcycle_tail(int D, const TailArgs& a, cudaStream_t s) {
  const size_t smem = vcycle_tail_smem(D, a.n, a.nl);
  static bool attr[2] = {false, false};
  if (!attr[D - 2]) {
    if (D == 3)
      cudaFuncSetAttribute(k_vcycle_tail<3>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kTailSmemMax);
    else
      cudaFuncSetAttribute(k_vcycle_tail<2>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kTailSmemMax);
    attr[D - 2] = true;
  }
  if (D == 3)
    k_vcycle_tail<3><<<1, kTailThreads, smem, s>>>(a);
  else
    k_vcycle_tail<2><<<1, kTailThreads, smem, s>>>(a);
  return 0;
}

// ---------------------------------------------------------------------------
// k_vcycle_ctail: the coarse end of a V-cycle in one thread-block cluster.  The levels
// are cut into slices along their slowest direction (z in 3-D, y in 2-D); block r of
// the C blocks keeps slices [ceil(r n/C), ceil((r+1) n/C)) of every level (the D face
// coefficients, the right-hand side and the iterate) in its shared memory, and reads
// a neighbouring slice another block keeps through distributed shared memory.  A
// cluster barrier separates the phases (load, each restriction, the coarsest solve,
// each prolongation and each colour of each sweep).  The arithmetic, and its order, is
// k_vcycle_tail's, so the bits are too; the cluster lets the tail take levels too large
// for one block (tens of thousands of cells), which otherwise cost a launch per sweep.
namespace {
constexpr int kCtailMaxC = 16;

struct CtailLayout {  // per level l and block r: first slice and float offset of its data
  int lo[kTailMaxLevels][kCtailMaxC + 1];
  int base[kTailMaxLevels][kCtailMaxC];
  int zd;             // float offset of the coarsest right-hand side in FP64 (even)
  int total;          // floats of the largest block's share, zd included
};

template <int D>
__host__ __device__ inline void ctail_layout(const int (*n)[3], int nl, int C, CtailLayout& Ly) {
  int tot_max = 0;
  for (int r = 0; r < C; ++r) {
    int off = 0;
    for (int l = 0; l < nl; ++l) {
      const int S = D == 3 ? n[l][2] : n[l][1], Z = D == 3 ? n[l][0] * n[l][1] : n[l][0];
      const int lo = (r * S + C - 1) / C, hi = ((r + 1) * S + C - 1) / C;
      Ly.lo[l][r] = lo;
      Ly.lo[l][r + 1] = hi;
      Ly.base[l][r] = off;
      off += (D + 2) * (hi - lo) * Z;
    }
    off = (off + 1) & ~1;
    if (off > tot_max) tot_max = off;
  }
  // the FP64 coarsest right-hand side sits after the largest share, the same offset in every block
  const int ncc = n[nl - 1][0] * n[nl - 1][1] * n[nl - 1][2];
  Ly.zd = tot_max;
  Ly.total = tot_max + 2 * ncc;
}
}  // namespace

size_t vcycle_ctail_smem(int D, const int (*n)[3], int nl, int C) {
  CtailLayout Ly;
  if (D == 3)
    ctail_layout<3>(n, nl, C, Ly);
  else
    ctail_layout<2>(n, nl, C, Ly);
  return sizeof(float) * (size_t)Ly.total;
}

template <int D>
__global__ void __launch_bounds__(kTailThreads) k_vcycle_ctail(TailArgs a) {
  namespace cg = cooperative_groups;
  cg::cluster_group cl = cg::this_cluster();
  extern __shared__ __align__(16) float tsm[];
  __shared__ CtailLayout Ly;
  const int C = (int)cl.num_blocks(), r = (int)cl.block_rank(), tid = threadIdx.x;
  if (tid == 0) ctail_layout<D>(a.n, a.nl, C, Ly);
  __syncthreads();
  auto S_of = [&](int l) { return D == 3 ? a.n[l][2] : a.n[l][1]; };
  auto Z_of = [&](int l) { return D == 3 ? a.n[l][0] * a.n[l][1] : a.n[l][0]; };
  // field f (0..D-1 coefficients, D right-hand side, D+1 iterate) of slice s of level l,
  // in the shared memory of the block that keeps it
  auto slice = [&](int l, int f, int s) -> float* {
    const int S = S_of(l), ow = (s * C) / S;
    const int lo = Ly.lo[l][ow], cnt = Ly.lo[l][ow + 1] - lo, Z = Z_of(l);
    float* p = tsm + Ly.base[l][ow] + (size_t)f * cnt * Z + (size_t)(s - lo) * Z;
    return ow == r ? p : cl.map_shared_rank(p, ow);
  };
  auto mine = [&](int l, int f) { return tsm + Ly.base[l][r] + (size_t)f * (Ly.lo[l][r + 1] - Ly.lo[l][r]) * Z_of(l); };
  // load this block's slices: coefficients of every level, the first level's right-hand side
  for (int l = 0; l < a.nl; ++l) {
    const int Z = Z_of(l), q0 = Ly.lo[l][r] * Z, nq = (Ly.lo[l][r + 1] - Ly.lo[l][r]) * Z;
    for (int c = 0; c < D; ++c) {
      float* b = mine(l, c);
      for (int q = tid; q < nq; q += kTailThreads) b[q] = ld_st(a.L[l][c], a.st[l], q0 + q);
    }
    if (l == 0) {
      float* z0 = mine(0, D);
      for (int q = tid; q < nq; q += kTailThreads) z0[q] = a.zmul * ld_st(a.z, a.st[0], q0 + q);
    }
  }
  cl.sync();
  // restriction down to the coarsest level (child (2I, 2J, 2K) first; z pairs, then x,
  // then y, as k_vcycle_tail)
  for (int l = 0; l + 1 < a.nl; ++l) {
    const int f0 = a.n[l][0], c0 = a.n[l + 1][0], c1 = a.n[l + 1][1];
    const int Zc = Z_of(l + 1), lo = Ly.lo[l + 1][r], nq = (Ly.lo[l + 1][r + 1] - lo) * Zc;
    float* zc = mine(l + 1, D);
    for (int m = tid; m < nq; m += kTailThreads) {
      const int q = lo * Zc + m;  // the coarse cell's index in its level
      const int I = q % c0, t = q / c0;
      float sum;
      if (D == 3) {
        const int J = t % c1, K = t / c1;
        const float* s0 = slice(l, D, 2 * K);
        const float* s1 = slice(l, D, 2 * K + 1);
        const int b0 = 2 * I + f0 * 2 * J;
        const float a00 = s0[b0] + s1[b0];
        const float a10 = s0[b0 + 1] + s1[b0 + 1];
        const float a01 = s0[b0 + f0] + s1[b0 + f0];
        const float a11 = s0[b0 + f0 + 1] + s1[b0 + f0 + 1];
        sum = (a00 + a10) + (a01 + a11);
      } else {
        const int J = t;
        const float* s0 = slice(l, D, 2 * J);
        const float* s1 = slice(l, D, 2 * J + 1);
        sum = (s0[2 * I] + s0[2 * I + 1]) + (s1[2 * I] + s1[2 * I + 1]);
      }
      zc[m] = sum;
    }
    cl.sync();
  }
  // coarsest level: x = G z in FP64, each block its own slices' rows
  {
    const int lc = a.nl - 1;
    const int nc = a.n[lc][0] * a.n[lc][1] * a.n[lc][2], Z = Z_of(lc);
    double* zd = reinterpret_cast<double*>(tsm + Ly.zd);
    for (int i = tid; i < nc; i += kTailThreads) zd[i] = (double)slice(lc, D, i / Z)[i % Z];
    __syncthreads();
    const int lo = Ly.lo[lc][r], nq = (Ly.lo[lc][r + 1] - lo) * Z;
    float* xc = mine(lc, D + 1);
    for (int m = tid; m < nq; m += kTailThreads) {
      const int i = lo * Z + m;
      double acc = 0.0;
#pragma unroll 16
      for (int jj = 0; jj < nc; ++jj) acc += __ldg(a.G + (long long)jj * nc + i) * zd[jj];
      xc[m] = (float)acc;
    }
    cl.sync();
  }
  // up: prolong (piecewise constant) and smooth each level
  for (int l = a.nl - 2; l >= 0; --l) {
    const int n0 = a.n[l][0], n1 = a.n[l][1], n2 = a.n[l][2];
    const int c0 = a.n[l + 1][0], c1 = a.n[l + 1][1];
    const int S = S_of(l), Z = Z_of(l), lo = Ly.lo[l][r], cnt = Ly.lo[l][r + 1] - lo, nq = cnt * Z;
    float* xl = mine(l, D + 1);
    const float* zl = mine(l, D);
    for (int m = tid; m < nq; m += kTailThreads) {
      const int q = lo * Z + m;
      const int i = q % n0, t = q / n0;
      const int j = t % n1, k = t / n1;
      const int sc = D == 3 ? (k >> 1) : (j >> 1);
      const int w = D == 3 ? (i >> 1) + c0 * (j >> 1) : (i >> 1);
      xl[m] = 0.f + slice(l + 1, D + 1, sc)[w];
    }
    (void)c1;
    cl.sync();
    const int nd[3] = {n0, n1, n2};
    const int h0 = n0 >> 1;            // cells of one colour per row (n0 even above the coarsest)
    const int rows = cnt * (Z / n0);   // this block's rows
    const int nhalf = rows * h0;
    for (int sw = 0; sw < a.post; ++sw) {
      for (int color = 0; color < 2; ++color) {
        for (int m = tid; m < nhalf; m += kTailThreads) {
          const int rw = m / h0;
          const int grow = lo * (Z / n0) + rw;  // the row's index in the level
          const int j = D == 3 ? grow % n1 : grow, k = D == 3 ? grow / n1 : 0;
          const int i = 2 * (m - rw * h0) + ((j + k + color) & 1);
          const int I[3] = {i, j, k};
          const int sl = D == 3 ? k : j;   // the cell's slice and its place in it
          const int w = D == 3 ? i + n0 * j : i;
          const int ml = (sl - lo) * Z + w;
          float sum = 0.f, dg = 0.f;
#pragma unroll
          for (int d = 0; d < D; ++d) {
            float Lu = 0.f, xu = 0.f, xd = 0.f;
            const bool per = (a.per >> d) & 1u;
            const float* Ld = mine(l, d);
            if (d < D - 1) {  // a direction within the slice
              const int st = d == 0 ? 1 : n0;
              if (I[d] + 1 < nd[d]) {
                Lu = Ld[ml + st];
                xu = xl[ml + st];
              } else if (per) {
                Lu = Ld[ml - (nd[d] - 1) * st];
                xu = xl[ml - (nd[d] - 1) * st];
              }
              if (I[d] > 0)
                xd = xl[ml - st];
              else if (per)
                xd = xl[ml + (nd[d] - 1) * st];
            } else {  // across slices
              if (I[d] + 1 < nd[d]) {
                Lu = slice(l, d, sl + 1)[w];
                xu = slice(l, D + 1, sl + 1)[w];
              } else if (per) {
                Lu = slice(l, d, 0)[w];
                xu = slice(l, D + 1, 0)[w];
              }
              if (I[d] > 0)
                xd = slice(l, D + 1, sl - 1)[w];
              else if (per)
                xd = slice(l, D + 1, S - 1)[w];
            }
            const float Ll = Ld[ml];
            sum = fmaf(Lu, xu, sum);
            sum = fmaf(Ll, xd, sum);
            dg += Lu + Ll;
          }
          xl[ml] = (dg > 0.f) ? __fdividef(sum - zl[ml], dg) : 0.f;
        }
        cl.sync();
      }
    }
  }
  {
    const int Z = Z_of(0), q0 = Ly.lo[0][r] * Z, nq = (Ly.lo[0][r + 1] - Ly.lo[0][r]) * Z;
    const float* x0 = mine(0, D + 1);
    for (int q = tid; q < nq; q += kTailThreads) st_st(a.x, a.st[0], q0 + q, x0[q]);
  }
}

// cluster size C (8 or 16) whose blocks fit with `smem` bytes each, or 0
int vcycle_ctail_cluster(int D, size_t smem, int C) {
  auto fn = D == 3 ? (void*)k_vcycle_ctail<3> : (void*)k_vcycle_ctail<2>;
  if (cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess ||
      (C > 8 && cudaFuncSetAttribute(fn, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) != cudaSuccess)) {
    cudaGetLastError();
    return 0;
  }
  cudaLaunchConfig_t cfg{};
  cfg.gridDim = dim3(C, 1, 1);
  cfg.blockDim = dim3(kTailThreads, 1, 1);
  cfg.dynamicSmemBytes = smem;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeClusterDimension;
  at[0].val.clusterDim.x = C;
  at[0].val.clusterDim.y = 1;
  at[0].val.clusterDim.z = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  int nclus = 0;
  if (cudaOccupancyMaxActiveClusters(&nclus, fn, &cfg) != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  return nclus >= 1 ? C : 0;
}

int launch_vcycle_ctail(int D, const TailArgs& a, int C, cudaStream_t s) {
  const size_t smem = vcycle_ctail_smem(D, a.n, a.nl, C);
  cudaLaunchConfig_t cfg{};
  cfg.gridDim = dim3(C, 1, 1);
  cfg.blockDim = dim3(kTailThreads, 1, 1);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeClusterDimension;
  at[0].val.clusterDim.x = C;
  at[0].val.clusterDim.y = 1;
  at[0].val.clusterDim.z = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  if (D == 3) return cudaLaunchKernelEx(&cfg, k_vcycle_ctail<3>, a) == cudaSuccess ? 0 : -1;
  return cudaLaunchKernelEx(&cfg, k_vcycle_ctail<2>, a) == cudaSuccess ? 0 : -1;
}

// ph + pl rounded to FP32
__global__ void k_df_round(const float* ph, const float* pl, float* out, long long n) {
  const long long q = (long long)blockIdx.x * 256 + threadIdx.x;
  if (q < n) out[q] = ph[q] + pl[q];
}

int launch_df_round(const float* ph, const float* pl, float* out, long long n, cudaStream_t s) {
  k_df_round<<<(int)((n + 255) / 256), 256, 0, s>>>(ph, pl, out, n);
  return 0;
}

// (ph, pl) += e
__global__ void k_df_add(float* ph, float* pl, const float* e, long long n) {
  const long long q = (long long)blockIdx.x * 256 + threadIdx.x;
  if (q >= n) return;
  float sh, sl, nh, nl;
  two_sum(ph[q], e[q], sh, sl);
  sl += pl[q];
  fast_two_sum(sh, sl, nh, nl);
  ph[q] = nh;
  pl[q] = nl;
}

int launch_df_add(float* ph, float* pl, const float* e, long long n, cudaStream_t s) {
  k_df_add<<<(int)((n + 255) / 256), 256, 0, s>>>(ph, pl, e, n);
  return 0;
}

__global__ void k_to_storage(const float* in, void* out, int type, long long n) {
  const long long q = (long long)blockIdx.x * 256 + threadIdx.x;
  if (q < n) st_st(out, type, q, in[q]);
}

int launch_to_storage(const float* in, void* out, int type, long long n, cudaStream_t s) {
  k_to_storage<<<(int)((n + 255) / 256), 256, 0, s>>>(in, out, type, n);
  return 0;
}


// ---------------------------------------------------------------------------
// Batched launches (many small simulations, one launch; see BatchSlot).
__device__ __forceinline__ int batch_block_p(const BatchGrid& bg, uint3& bid, unsigned& nb) {
  const int b = (int)blockIdx.x;
  int lo = 0, hi = bg.n;  // bg.start[lo] <= b < bg.start[hi]
  while (hi - lo > 1) {
    const int m = (lo + hi) >> 1;
    if (bg.start[m] <= b) lo = m; else hi = m;
  }
  const unsigned local = (unsigned)(b - bg.start[lo]), gx = bg.gx[lo], gy = bg.gy[lo];
  bid = make_uint3(local % gx, (local / gx) % gy, local / (gx * gy));
  wl_in(bid.z, (unsigned)(bg.start[lo + 1] - bg.start[lo]) / (gx * gy), WL_DBG_BATCH);
  nb = (unsigned)(bg.start[lo + 1] - bg.start[lo]);
  return bg.slot[lo];
}

dim3 residual_grid(int D, const Grid& g) {
  if (D == 3) return dim3((g.n[0] + 31) / 32, (g.n[1] + 7) / 8, (g.n[2] + 2 * RS_ZP - 1) / (2 * RS_ZP));
  return dim3((g.n[0] + 31) / 32, (g.n[1] + 7) / 8, 1);
}
dim3 restrict_grid(int D, const ResArgs& a) {
  const long long ncc = (long long)a.cn[0] * a.cn[1] * (D == 3 ? a.cn[2] : 1);
  return dim3((unsigned)std::min<long long>((ncc + 255) / 256, 152LL * 8 * 4), 1, 1);
}
dim3 sweep_grid(int D, const SweepArgs& a) {
  const Grid& g = a.g;
  return dim3((g.n[0] + SW_TX - 1) / SW_TX, (g.n[1] + SW_TY - 1) / SW_TY, D == 3 ? (g.n[2] + a.tz - 1) / a.tz : 1);
}
dim3 correct_grid(int D, const CorrArgs& a) {
  const Grid& g = a.g;
  if (D == 3 && a.u_in[0] != a.u_out[0]) return dim3((g.n[0] + 31) / 32, (g.n[1] + 7) / 8, (g.n[2] + C3_Z - 1) / C3_Z);
  if (D == 3) return dim3((g.n[0] + 31) / 32, (g.n[1] + 7) / 8, (g.n[2] + CR_Z - 1) / CR_Z);
  return dim3((g.n[0] + 31) / 32, (g.n[1] + 7) / 8, 1);
}

// the V-cycle launches skip slots whose projection has converged (cond 0)
template <int D>
__global__ void __launch_bounds__(256) kb_residual(const BatchSlot* __restrict__ t, const __grid_constant__ BatchGrid bg,
                                                   int which, int vcycle) {
  uint3 bid;
  unsigned nb;
  const BatchSlot& sl = t[batch_block_p(bg, bid, nb)];
  if (vcycle && sl.ds->cond == 0) return;
  residual_body<D>(which < 2 ? sl.div[which] : sl.res, bid);
}
template <int D>
__global__ void __launch_bounds__(256) kb_restrict(const BatchSlot* __restrict__ t, const __grid_constant__ BatchGrid bg,
                                                   int level) {
  uint3 bid;
  unsigned nb;
  const BatchSlot& sl = t[batch_block_p(bg, bid, nb)];
  if (sl.ds->cond == 0) return;
  restrict_body<D>(sl.restr[level], bid, nb);
}
template <int D>
__global__ void __launch_bounds__(kTailThreads) kb_tail(const BatchSlot* __restrict__ t,
                                                        const __grid_constant__ BatchGrid bg) {
  uint3 bid;
  unsigned nb;
  const BatchSlot& sl = t[batch_block_p(bg, bid, nb)];
  if (sl.ds->cond == 0) return;
  vcycle_tail_body<D>(sl.tail, bid);
}
template <int D>
__global__ void __launch_bounds__(256) kb_sweep(const BatchSlot* __restrict__ t, const __grid_constant__ BatchGrid bg,
                                                int level, int it) {
  uint3 bid;
  unsigned nb;
  const BatchSlot& sl = t[batch_block_p(bg, bid, nb)];
  if (sl.ds->cond == 0 || it >= sl.post) return;
  sweep_body<D, float>(sl.sweep[level][it], bid);
}
// 3-D slots: the out-of-place corrector with the double-float pressure; 2-D: k_correct
template <int D, bool CFL>
__global__ void __launch_bounds__(256) kb_correct(const BatchSlot* __restrict__ t, const __grid_constant__ BatchGrid bg,
                                                  int which) {
  uint3 bid;
  unsigned nb;
  const BatchSlot& sl = t[batch_block_p(bg, bid, nb)];
  if constexpr (D == 3)
    correct3_body<true, CFL>(sl.corr[which], bid);
  else
    correct_body<2>(sl.corr[which], bid);
}
// one thread per slot: its V-cycle decision (as k_decide); the loop continues while any
// slot's does
__global__ void __launch_bounds__(kBatchMax) kb_decide(const BatchSlot* __restrict__ t,
                                                       const __grid_constant__ BatchGrid bg,
                                                       cudaGraphConditionalHandle h, int first, int proj) {
  bool cont = false;
  if ((int)threadIdx.x < bg.n) {
    const BatchSlot& sl = t[bg.slot[threadIdx.x]];
    if (first || sl.ds->cond) cont = decide_state(sl.ds, first, proj, sl.w[proj], sl.tol, sl.maxit);
  }
  const bool any = __syncthreads_or(cont);
  if (threadIdx.x == 0) cudaGraphSetConditional(h, any ? 1u : 0u);
}
__global__ void __launch_bounds__(kBatchMax) kb_step_end(const BatchSlot* __restrict__ t,
                                                         const __grid_constant__ BatchGrid bg) {
  if ((int)threadIdx.x >= bg.n) return;
  const BatchSlot& sl = t[bg.slot[threadIdx.x]];
  step_end_state(sl.ds, sl.D, sl.nu, sl.dt_cap, sl.dt_fixed, 1, sl.ring, sl.ring_cap, nullptr);
}

int launch_batch_residual(int D, const BatchSlot* t, const BatchGrid& bg, int which, int vcycle, cudaStream_t s) {
  if (bg.n == 0) return 0;
  if (D == 3)
    kb_residual<3><<<bg.start[bg.n], 256, 0, s>>>(t, bg, which, vcycle);
  else
    kb_residual<2><<<bg.start[bg.n], 256, 0, s>>>(t, bg, which, vcycle);
  return 0;
}
int launch_batch_restrict(int D, const BatchSlot* t, const BatchGrid& bg, int level, cudaStream_t s) {
  if (bg.n == 0) return 0;
  if (D == 3)
    kb_restrict<3><<<bg.start[bg.n], 256, 0, s>>>(t, bg, level);
  else
    kb_restrict<2><<<bg.start[bg.n], 256, 0, s>>>(t, bg, level);
  return 0;
}
int launch_batch_tail(int D, const BatchSlot* t, const BatchGrid& bg, size_t smem, cudaStream_t s) {
  if (bg.n == 0) return 0;
  static bool attr[2] = {false, false};
  if (!attr[D - 2]) {
    if (D == 3)
      cudaFuncSetAttribute(kb_tail<3>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kTailSmemMax);
    else
      cudaFuncSetAttribute(kb_tail<2>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kTailSmemMax);
    attr[D - 2] = true;
  }
  if (D == 3)
    kb_tail<3><<<bg.start[bg.n], kTailThreads, smem, s>>>(t, bg);
  else
    kb_tail<2><<<bg.start[bg.n], kTailThreads, smem, s>>>(t, bg);
  return 0;
}
int launch_batch_sweep(int D, const BatchSlot* t, const BatchGrid& bg, int level, int it, cudaStream_t s) {
  if (bg.n == 0) return 0;
  if (D == 3)
    kb_sweep<3><<<bg.start[bg.n], 256, 0, s>>>(t, bg, level, it);
  else
    kb_sweep<2><<<bg.start[bg.n], 256, 0, s>>>(t, bg, level, it);
  return 0;
}
int launch_batch_correct(int D, const BatchSlot* t, const BatchGrid& bg, int which, cudaStream_t s) {
  if (bg.n == 0) return 0;
  if (D == 3 && which == 1)
    kb_correct<3, true><<<bg.start[bg.n], 256, 0, s>>>(t, bg, which);
  else if (D == 3)
    kb_correct<3, false><<<bg.start[bg.n], 256, 0, s>>>(t, bg, which);
  else
    kb_correct<2, false><<<bg.start[bg.n], 256, 0, s>>>(t, bg, which);
  return 0;
}
int launch_batch_decide(const BatchSlot* t, const BatchGrid& bg, cudaGraphConditionalHandle h, int first, int proj,
                        cudaStream_t s) {
  kb_decide<<<1, kBatchMax, 0, s>>>(t, bg, h, first, proj);
  return 0;
}
int launch_batch_step_end(const BatchSlot* t, const BatchGrid& bg, cudaStream_t s) {
  if (bg.n == 0) return 0;
  kb_step_end<<<1, kBatchMax, 0, s>>>(t, bg);
  return 0;
}

}  // namespace wl

namespace wl {
unsigned dbg_take_poisson() {
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
