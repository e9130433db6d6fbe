// Reverse-mode derivative (adjoint) of the time step at a fixed dt with respect to the
// circle/sphere parameters theta = (R, c_0, .., c_{D-1}): the differentiable use of the
// solver (Section 1; the body enters through its signed-distance function, Section 2).
//
// Each kernel is the transpose of a forward kernel's arithmetic (same FP32 values, the
// same branch of the limiter and of the upwind switch as the forward takes):
//   k_adj_convdiff    convdiff! (k_stage's fluxes): per face flux, F' = r'[I] - r'[I-e_j],
//                     scattered to the velocities the flux reads (atomics; BC mapping:
//                     periodic wrap, tangential clamp, prescribed normal faces dropped)
//   k_adj_stage_local the mu0 blend of BDIM!: f' = s mu0 v'
//   k_adj_band        the mu1 term of BDIM! on the body band, its mu0 / mu1 cotangents
//   k_adj_proj_rhs /  project!: with y = A^+ (D(L u') + x'), v' = u' - G y and
//   k_adj_proj_out    L' = -(G x) v' (the Poisson solve itself runs the forward multigrid:
//                     the operator is symmetric)
//   k_adj_force_theta the pressure force's weights n K_eps(d)
//   k_adj_moments     mu0 = K0(d/eps) (and L = mu0) at every band face
// The projection is differentiated as the exact projection; the forward and adjoint
// solves stop at their tolerances.  dt is held fixed (the CFL maximum is not
// differentiated).
#include "wl_dev.cuh"
#include "wl_kernels.h"
#include "wl_stage_dev.cuh"

namespace wl {

namespace {

__device__ __forceinline__ bool face_updated(const Grid& g, int c, const int* I) { return is_per(g, c) || I[c] >= 1; }

// Storage index of velocity component c at face index I (possibly outside the
// interior), or -1 where the BC prescribes the value (the mapping of load_u_bc).
template <int D>
__device__ __forceinline__ long long map_face(const Grid& g, int c, const int* Iin) {
  int I[3] = {Iin[0], Iin[1], Iin[2]};
#pragma unroll
  for (int d = 0; d < D; ++d) {
    int q = I[d];
    const int n = g.n[d];
    if (is_per(g, d)) {
      q = (q < 0) ? q + n : ((q >= n) ? q - n : q);
    } else {
      if (d == c && (q <= 0 || q >= n)) return -1;
      q = q < 0 ? 0 : (q >= n ? n - 1 : q);
    }
    I[d] = q;
  }
  return cell_index(g, I[0], I[1], D == 3 ? I[2] : 0);
}

// circle / sphere: d = |x - c| - R, n = (x - c)/|x - c|, and their derivatives with
// respect to theta = (R, c_0, .., c_{D-1}): dd[t], dn[j][t].
template <int D>
__device__ double sdf_theta(const Body& b, const double* x, double* n, double* dd, double (*dn)[4]) {
  double r2 = 0.0;
#pragma unroll
  for (int d = 0; d < D; ++d) r2 += (x[d] - b.c[d]) * (x[d] - b.c[d]);
  const double r = sqrt(r2);
  n[0] = n[1] = n[2] = 0.0;
#pragma unroll
  for (int d = 0; d < D; ++d) n[d] = r > 0.0 ? (x[d] - b.c[d]) / r : 0.0;
  dd[0] = -1.0;
#pragma unroll
  for (int j = 0; j < 3; ++j) dn[j][0] = 0.0;
#pragma unroll
  for (int k = 0; k < D; ++k) {
    dd[1 + k] = -n[k];
#pragma unroll
    for (int j = 0; j < D; ++j) dn[j][1 + k] = r > 0.0 ? -((j == k ? 1.0 : 0.0) - n[j] * n[k]) / r : 0.0;
  }
  return r - b.r1;
}

// the body's bounding box of cells/faces within `pad` of the band
void band_box(int D, const Grid& g, const Body& b, double pad, int* lo, int* hi) {
  for (int d = 0; d < 3; ++d) {
    lo[d] = 0;
    hi[d] = 1;
    if (d >= D) continue;
    lo[d] = (int)fmax(0.0, floor(b.c[d] - b.r1 - b.eps - pad));
    hi[d] = (int)fmin((double)g.n[d], ceil(b.c[d] + b.r1 + b.eps + pad) + 1.0);
    if (hi[d] < lo[d]) hi[d] = lo[d];
  }
}

__device__ double block_sum(double v, double* sh) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  __syncthreads();
  if (l == 0) sh[w] = v;
  __syncthreads();
  if (w == 0) {
    v = (l < (int)(blockDim.x >> 5)) ? sh[l] : 0.0;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if (l == 0) sh[8] = v;
  }
  __syncthreads();
  return sh[8];
}

template <int D>
__device__ __forceinline__ bool cell_active(const Grid& g, const float* const* L, long long q, const int* I) {
  const long long st[3] = {1, (long long)g.n[0], (long long)g.n[0] * g.n[1]};
  float dg = 0.f;
#pragma unroll
  for (int c = 0; c < D; ++c) {
    long long qu;
    bool has;
    if (I[c] + 1 < g.n[c]) {
      qu = q + st[c];
      has = true;
    } else {
      has = is_per(g, c);
      qu = q - (long long)(g.n[c] - 1) * st[c];
    }
    dg += (has ? L[c][qu] : 0.f) + L[c][q];
  }
  return dg > 0.f;
}

__device__ __forceinline__ void coords(const Grid& g, long long q, int* I) {
  I[0] = (int)(q % g.n[0]);
  const long long t = q / g.n[0];
  I[1] = (int)(t % g.n[1]);
  I[2] = (int)(t / g.n[1]);
}

}  // namespace

// ---------------------------------------------------------------------------
// Geometry constants of the force adjoint: Na (active cells) and W = sum over band
// cells of n K_eps(d); zeroes theta.  Partials per block, then one block in a fixed order.
template <int D>
__global__ void __launch_bounds__(256) k_adj_setup_partials(Grid g, Body b, const float* L0, const float* L1,
                                                            const float* L2, double* part) {
  __shared__ double sh[9];
  const float* L[3] = {L0, L1, L2};
  double v[4] = {0.0, 0.0, 0.0, 0.0};
  for (long long q = (long long)blockIdx.x * 256 + threadIdx.x; q < g.nc; q += (long long)gridDim.x * 256) {
    int I[3];
    coords(g, q, I);
    if (cell_active<D>(g, L, q, I)) v[0] += 1.0;
    double x[3] = {I[0] + 0.5, I[1] + 0.5, I[2] + 0.5}, n[3];
    const double d = body_sdf<D>(b, x, n);
    if (fabs(d) < b.eps) {
      const double K = (1.0 + cospi(d / b.eps)) / (2.0 * b.eps);
#pragma unroll
      for (int k = 0; k < D; ++k) v[1 + k] += n[k] * K;
    }
  }
  for (int t = 0; t < 4; ++t) {
    const double s = block_sum(v[t], sh);
    if (threadIdx.x == 0) part[4 * blockIdx.x + t] = s;
  }
}

__global__ void __launch_bounds__(256) k_adj_setup_final(const double* part, int npart, AdjState* as) {
  __shared__ double sh[9];
  for (int t = 0; t < 4; ++t) {
    double v = 0.0;
    for (int k = threadIdx.x; k < npart; k += 256) v += part[4 * k + t];
    v = block_sum(v, sh);
    if (threadIdx.x == 0) {
      if (t == 0)
        as->Na = v;
      else
        as->W[t - 1] = v;
    }
  }
  if (threadIdx.x < 4) as->theta[threadIdx.x] = 0.0;
  if (threadIdx.x == 0) as->mean = 0.0;
}

int launch_adj_setup(int D, const Grid& g, const Body& b, const float* const* L, AdjState* as, double* part,
                     int npart, cudaStream_t s) {
  if (D == 3)
    k_adj_setup_partials<3><<<npart, 256, 0, s>>>(g, b, L[0], L[1], L[2], part);
  else
    k_adj_setup_partials<2><<<npart, 256, 0, s>>>(g, b, L[0], L[1], L[1], part);
  k_adj_setup_final<<<1, 256, 0, s>>>(part, npart, as);
  return 0;
}

// ---------------------------------------------------------------------------
// Force weights: F = -sum_band (p - pbar) w, w = n K_eps(d).  For the cotangent g of F:
// theta' += -sum_band (p - pbar) g . dw/dtheta (one block over the band box; pbar is
// the active-cell mean the forward force kernel leaves in pmean).
template <int D>
__global__ void __launch_bounds__(256) k_adj_force_theta(Grid g, Body b, const float* p, const double* pmean,
                                                         const double* gF, int lo0, int lo1, int lo2, int bx, int by,
                                                         int bz, AdjState* as) {
  __shared__ double sh[9];
  const double pbar = *pmean;
  double gv[3] = {0.0, 0.0, 0.0};
  for (int d = 0; d < D; ++d) gv[d] = gF[d];
  double acc[4] = {0.0, 0.0, 0.0, 0.0};
  const long long nbox = (long long)bx * by * bz;
  for (long long t = threadIdx.x; t < nbox; t += 256) {
    const int i = lo0 + (int)(t % bx);
    const long long r = t / bx;
    const int j = lo1 + (int)(r % by);
    const int k = lo2 + (int)(r / by);
    double x[3] = {i + 0.5, j + 0.5, k + 0.5}, n[3], dd[4], dn[3][4];
    const double d = sdf_theta<D>(b, x, n, dd, dn);
    if (!(fabs(d) < b.eps)) continue;
    const double K = (1.0 + cospi(d / b.eps)) / (2.0 * b.eps);
    const double Kp = -3.141592653589793 * sinpi(d / b.eps) / (2.0 * b.eps * b.eps);
    const double pp = (double)p[cell_index(g, i, j, k)] - pbar;
#pragma unroll
    for (int tt = 0; tt <= D; ++tt) {
      double gw = 0.0;
#pragma unroll
      for (int e = 0; e < D; ++e) gw += gv[e] * (dn[e][tt] * K + n[e] * Kp * dd[tt]);
      acc[tt] -= pp * gw;
    }
  }
  for (int tt = 0; tt <= D; ++tt) {
    const double v = block_sum(acc[tt], sh);
    if (threadIdx.x == 0) as->theta[tt] += v;
  }
}

int launch_adj_force_theta(int D, const Grid& g, const Body& b, const float* p, const double* pmean,
                           const double* gF, AdjState* as, cudaStream_t s) {
  int lo[3], hi[3];
  band_box(D, g, b, 1.0, lo, hi);
  const int bx = hi[0] - lo[0], by = hi[1] - lo[1], bz = hi[2] - lo[2];
  if (D == 3)
    k_adj_force_theta<3><<<1, 256, 0, s>>>(g, b, p, pmean, gF, lo[0], lo[1], lo[2], bx, by, bz, as);
  else
    k_adj_force_theta<2><<<1, 256, 0, s>>>(g, b, p, pmean, gF, lo[0], lo[1], lo[2], bx, by, bz, as);
  return 0;
}

// ---------------------------------------------------------------------------
// Right-hand side of the adjoint Poisson solve of a projection:
//   b[I] = sum_c L_c[I+e_c] u'_c[I+e_c] - L_c[I] u'_c[I]     (the transpose of the
//          correction u_c[I] -= L_c[I] (x[I] - x[I-e_c]) applied to u')
//        + fmul * (-(g . w_I) + [I active] (g . W)/Na)        (the force through p = x/(w dt))
// with u' zero on faces the BC prescribes; then its mean over the active cells is
// removed (partials per block, one block in a fixed order, then the subtraction).
template <int D>
__global__ void __launch_bounds__(256) k_adj_proj_rhs(Grid g, Body b, const float* ub0, const float* ub1,
                                                      const float* ub2, const float* L0, const float* L1,
                                                      const float* L2, const double* gF, double fmul,
                                                      const AdjState* as, int lo0, int lo1, int lo2, int hi0,
                                                      int hi1, int hi2, float* rhs, double* part) {
  __shared__ double sh[9];
  const float* L[3] = {L0, L1, L2};
  const float* ub[3] = {ub0, ub1, ub2};
  const long long st[3] = {1, (long long)g.n[0], (long long)g.n[0] * g.n[1]};
  double gW = 0.0, gv[3] = {0.0, 0.0, 0.0};
  if (gF) {
    for (int d = 0; d < D; ++d) {
      gv[d] = gF[d];
      gW += gv[d] * as->W[d];
    }
  }
  const double Na = as->Na;
  double sum = 0.0;
  for (long long q = (long long)blockIdx.x * 256 + threadIdx.x; q < g.nc; q += (long long)gridDim.x * 256) {
    int I[3];
    coords(g, q, I);
    float v = 0.f;
#pragma unroll
    for (int c = 0; c < D; ++c) {
      if (face_updated(g, c, I)) v -= L[c][q] * ub[c][q];
      bool has;
      long long qu;
      if (I[c] + 1 < g.n[c]) {
        qu = q + st[c];
        has = true;
      } else {
        has = is_per(g, c);
        qu = q - (long long)(g.n[c] - 1) * st[c];
      }
      if (has) v += L[c][qu] * ub[c][qu];  // the upper face is updated (interior or periodic)
    }
    const bool act = cell_active<D>(g, L, q, I);
    if (gF) {
      double f = act && Na > 0.0 ? gW / Na : 0.0;
      if (I[0] >= lo0 && I[0] < hi0 && I[1] >= lo1 && I[1] < hi1 && I[2] >= lo2 && I[2] < hi2) {
        double x[3] = {I[0] + 0.5, I[1] + 0.5, I[2] + 0.5}, n[3];
        const double d = body_sdf<D>(b, x, n);
        if (fabs(d) < b.eps) {
          const double K = (1.0 + cospi(d / b.eps)) / (2.0 * b.eps);
          for (int e = 0; e < D; ++e) f -= gv[e] * n[e] * K;
        }
      }
      v += (float)(fmul * f);
    }
    if (!act) v = 0.f;
    rhs[q] = v;
    sum += v;
  }
  sum = block_sum(sum, sh);
  if (threadIdx.x == 0) part[blockIdx.x] = sum;
}

__global__ void __launch_bounds__(256) k_adj_mean_final(const double* part, int npart, AdjState* as) {
  __shared__ double sh[9];
  double v = 0.0;
  for (int k = threadIdx.x; k < npart; k += 256) v += part[k];
  v = block_sum(v, sh);
  if (threadIdx.x == 0) as->mean = as->Na > 0.0 ? v / as->Na : 0.0;
}

template <int D>
__global__ void __launch_bounds__(256) k_adj_sub_mean(Grid g, const float* L0, const float* L1, const float* L2,
                                                      const AdjState* as, float* rhs) {
  const float* L[3] = {L0, L1, L2};
  const long long q = (long long)blockIdx.x * 256 + threadIdx.x;
  if (q >= g.nc) return;
  int I[3];
  coords(g, q, I);
  if (cell_active<D>(g, L, q, I)) rhs[q] = (float)((double)rhs[q] - as->mean);
}

int launch_adj_proj_rhs(int D, const Grid& g, const Body& b, const float* const* ub, const float* const* L,
                        const double* gF, double fmul, AdjState* as, float* rhs, double* part, int npart,
                        cudaStream_t s) {
  int lo[3], hi[3];
  band_box(D, g, b, 1.0, lo, hi);
  if (D == 3)
    k_adj_proj_rhs<3><<<npart, 256, 0, s>>>(g, b, ub[0], ub[1], ub[2], L[0], L[1], L[2], gF, fmul, as, lo[0], lo[1],
                                            lo[2], hi[0], hi[1], hi[2], rhs, part);
  else
    k_adj_proj_rhs<2><<<npart, 256, 0, s>>>(g, b, ub[0], ub[1], ub[1], L[0], L[1], L[1], gF, fmul, as, lo[0], lo[1],
                                            lo[2], hi[0], hi[1], hi[2], rhs, part);
  k_adj_mean_final<<<1, 256, 0, s>>>(part, npart, as);
  const int nb = (int)((g.nc + 255) / 256);
  if (D == 3)
    k_adj_sub_mean<3><<<nb, 256, 0, s>>>(g, L[0], L[1], L[2], as, rhs);
  else
    k_adj_sub_mean<2><<<nb, 256, 0, s>>>(g, L[0], L[1], L[1], as, rhs);
  return 0;
}

// v'_c[I] = u'_c[I] - (y[I] - y[I-e_c]) on faces the step updates (0 elsewhere) and the
// coefficient cotangent mbar_c[I] += -(x[I] - x[I-e_c]) v'_c[I], x = xmul * p.
template <int D>
__global__ void __launch_bounds__(256) k_adj_proj_out(Grid g, const float* ub0, const float* ub1, const float* ub2,
                                                      const float* y, const float* p, float xmul, float* vb0,
                                                      float* vb1, float* vb2, float* mb0, float* mb1, float* mb2) {
  const long long t = (long long)blockIdx.x * 256 + threadIdx.x;
  if (t >= g.nc * D) return;
  const int c = (int)(t / g.nc);
  const long long q = t - (long long)c * g.nc;
  const float* ub[3] = {ub0, ub1, ub2};
  float* vb[3] = {vb0, vb1, vb2};
  float* mb[3] = {mb0, mb1, mb2};
  int I[3];
  coords(g, q, I);
  if (!face_updated(g, c, I)) {
    vb[c][q] = 0.f;
    return;
  }
  const long long stc = c == 0 ? 1 : (c == 1 ? (long long)g.n[0] : (long long)g.n[0] * g.n[1]);
  const long long qm = I[c] > 0 ? q - stc : q + (long long)(g.n[c] - 1) * stc;  // periodic wrap at I_c = 0
  const float v = ub[c][q] - (y[q] - y[qm]);
  vb[c][q] = v;
  mb[c][q] -= xmul * (p[q] - p[qm]) * v;
}

int launch_adj_proj_out(int D, const Grid& g, const float* const* ub, const float* y, const float* p, float xmul,
                        float* const* vb, float* const* mbar, cudaStream_t s) {
  const int nb = (int)((g.nc * D + 255) / 256);
  if (D == 3)
    k_adj_proj_out<3><<<nb, 256, 0, s>>>(g, ub[0], ub[1], ub[2], y, p, xmul, vb[0], vb[1], vb[2], mbar[0], mbar[1],
                                         mbar[2]);
  else
    k_adj_proj_out<2><<<nb, 256, 0, s>>>(g, ub[0], ub[1], ub[1], y, p, xmul, vb[0], vb[1], vb[1], mbar[0], mbar[1],
                                         mbar[1]);
  return 0;
}

// ---------------------------------------------------------------------------
// mu0 blend of a stage (out = s (mu0 f [+ u'])): f' = s mu0 v' on updated faces, and in
// stage 2 the direct part u'' = v'/2.
template <int D>
__global__ void __launch_bounds__(256) k_adj_stage_local(Grid g, const float* vb0, const float* vb1,
                                                         const float* vb2, const float* m0, const float* m1,
                                                         const float* m2, float sfac, float* fb0, float* fb1,
                                                         float* fb2, float* up0, float* up1, float* up2) {
  const long long t = (long long)blockIdx.x * 256 + threadIdx.x;
  if (t >= g.nc * D) return;
  const int c = (int)(t / g.nc);
  const long long q = t - (long long)c * g.nc;
  const float* vb[3] = {vb0, vb1, vb2};
  const float* mu[3] = {m0, m1, m2};
  float* fb[3] = {fb0, fb1, fb2};
  float* up[3] = {up0, up1, up2};
  int I[3];
  coords(g, q, I);
  const bool upd = face_updated(g, c, I);
  const float v = upd ? vb[c][q] : 0.f;
  fb[c][q] = mu[c][q] * (sfac * v);
  if (up0) up[c][q] = 0.5f * v;
}

int launch_adj_stage_local(int D, const Grid& g, const float* const* vb, const float* const* mu0, float sfac,
                           float* const* fb, float* const* up, cudaStream_t s) {
  const int nb = (int)((g.nc * D + 255) / 256);
  float* u0 = up ? up[0] : nullptr;
  float* u1 = up ? up[1] : nullptr;
  float* u2 = up ? up[2] : nullptr;
  if (D == 3)
    k_adj_stage_local<3><<<nb, 256, 0, s>>>(g, vb[0], vb[1], vb[2], mu0[0], mu0[1], mu0[2], sfac, fb[0], fb[1], fb[2],
                                            u0, u1, u2);
  else
    k_adj_stage_local<2><<<nb, 256, 0, s>>>(g, vb[0], vb[1], vb[1], mu0[0], mu0[1], mu0[1], sfac, fb[0], fb[1], fb[1],
                                            u0, u1, u1);
  return 0;
}

// mu1 term on the band: out_c[I] += s sum_j mu1_j (f[I+e_j] - f[I-e_j])/2 with
// mu1 = eps K1(d/eps) n.  Transpose: f'[I +- e_j] +-= s mu1_j v'/2 (BC-mapped), the mu0
// cotangent s v' f[I] into mbar, and theta' += s v' (f[I+e_j] - f[I-e_j])/2 dmu1_j/dtheta
// with d(eps K1(d/eps))/dd = -s K(s), s = d/eps.
template <int D>
__global__ void __launch_bounds__(256) k_adj_band(StageArgs a, Body b, const float* vb0, const float* vb1,
                                                  const float* vb2, float sfac, float* fb0, float* fb1, float* fb2,
                                                  float* mb0, float* mb1, float* mb2, int lo0, int lo1, int lo2,
                                                  int bx, int by, int bz, AdjState* as) {
  const long long nbox = (long long)bx * by * bz;
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= nbox * D) return;
  const int c = (int)(t / nbox);
  long long rem = t - (long long)c * nbox;
  const int i = lo0 + (int)(rem % bx);
  rem /= bx;
  const int j = lo1 + (int)(rem % by);
  const int k = lo2 + (int)(rem / by);
  const Grid& g = a.g;
  const int I[3] = {i, j, k};
  if (!face_updated(g, c, I)) return;
  double x[3] = {i + 0.5, j + 0.5, k + 0.5};
  x[c] -= 0.5;
  double n[3], dd[4], dn[3][4];
  const double d = sdf_theta<D>(b, x, n, dd, dn);
  if (!(fabs(d) < b.eps)) return;
  const float* vb[3] = {vb0, vb1, vb2};
  float* fb[3] = {fb0, fb1, fb2};
  float* mb[3] = {mb0, mb1, mb2};
  const long long q = cell_index(g, i, j, k);
  const float vs = sfac * vb[c][q];
  const float dtf = *a.dt;
  mb[c][q] += vs * f_at<D>(a, c, i, j, k, dtf);
  const double sc = d / b.eps, K = 0.5 * (1.0 + cospi(sc));
  const double k1 = b.eps * kernel_K1(sc), k1p = -sc * K;
  double th[4] = {0.0, 0.0, 0.0, 0.0};
#pragma unroll
  for (int jd = 0; jd < D; ++jd) {
    int P[3] = {i, j, k}, M[3] = {i, j, k};
    P[jd] += 1;
    M[jd] -= 1;
    const float fp = f_at<D>(a, c, P[0], P[1], P[2], dtf);
    const float fm = f_at<D>(a, c, M[0], M[1], M[2], dtf);
    const float m1 = (float)(k1 * n[jd]) * 0.5f * vs;
    const long long ip = map_face<D>(g, c, P), im = map_face<D>(g, c, M);
    if (ip >= 0) atomicAdd(fb[c] + ip, m1);
    if (im >= 0) atomicAdd(fb[c] + im, -m1);
    const double gfd = (double)vs * 0.5 * ((double)fp - (double)fm);
#pragma unroll
    for (int tt = 0; tt <= D; ++tt) th[tt] += gfd * (k1p * n[jd] * dd[tt] + k1 * dn[jd][tt]);
  }
#pragma unroll
  for (int tt = 0; tt <= D; ++tt) atomicAdd(&as->theta[tt], th[tt]);
}

int launch_adj_band(int D, const StageArgs& a, const Body& b, const float* const* vb, float sfac, float* const* fb,
                    float* const* mbar, AdjState* as, cudaStream_t s) {
  int lo[3], hi[3];
  band_box(D, a.g, b, 2.0, lo, hi);
  const int bx = hi[0] - lo[0], by = hi[1] - lo[1], bz = hi[2] - lo[2];
  const long long n = (long long)bx * by * bz * D;
  if (n <= 0) return 0;
  const int nb = (int)((n + 255) / 256);
  if (D == 3)
    k_adj_band<3><<<nb, 256, 0, s>>>(a, b, vb[0], vb[1], vb[2], sfac, fb[0], fb[1], fb[2], mbar[0], mbar[1], mbar[2],
                                     lo[0], lo[1], lo[2], bx, by, bz, as);
  else
    k_adj_band<2><<<nb, 256, 0, s>>>(a, b, vb[0], vb[1], vb[1], sfac, fb[0], fb[1], fb[1], mbar[0], mbar[1], mbar[1],
                                     lo[0], lo[1], lo[2], bx, by, bz, as);
  return 0;
}

// ---------------------------------------------------------------------------
// f = u0 + dt r(u) on updated faces: u0' += f', and with r' = dt f' the transpose of
// convdiff!, r_c[I] = sum_j F_cj[I] - F_cj[I+e_j]: every face flux gets
// F' = r'_c[I] - r'_c[I-e_j] and scatters F' dF/du to the velocities it reads.  One
// thread per face (c, I) handles the lower j-fluxes of its control volume (and, on the
// last cell of a non-periodic direction, the flux through the upper boundary face).
template <int D>
__device__ __forceinline__ void flux_adjoint(const Grid& g, const float* const* u, int c, int j, const int* J,
                                             float Fb, float nu, bool adv, float* const* ubin) {
  int m2[3] = {J[0], J[1], J[2]}, m1[3] = {J[0], J[1], J[2]}, p1[3] = {J[0], J[1], J[2]};
  int jc[3] = {J[0], J[1], J[2]};
  m2[j] -= 2;
  m1[j] -= 1;
  p1[j] += 1;
  jc[c] -= 1;
  const long long im1 = map_face<D>(g, c, m1), ip0 = map_face<D>(g, c, J);
  // viscous part: F = ... - nu (u[J] - u[J-e_j])
  if (ip0 >= 0) atomicAdd(ubin[c] + ip0, -nu * Fb);
  if (im1 >= 0) atomicAdd(ubin[c] + im1, nu * Fb);
  if (!adv) return;
  auto U = [&](int comp, const int* P) { return load_u_bc<D>(u[comp], comp, g, P[0], P[1], P[2]); };
  const float vm2 = U(c, m2), vm1 = U(c, m1), vp0 = U(c, J), vp1 = U(c, p1);
  const float a2 = U(j, J) + U(j, jc);
  // the forward's branch (mom_flux): upwind side, limiter case
  const bool pos = a2 > 0.f;
  const float uu = pos ? vm2 : vp1, cc = pos ? vm1 : vp0, dd = pos ? vp0 : vm1;
  const float dD = dd - cc, dU = cc - uu;
  const float ad = fabsf(dD), au = fabsf(dU);
  const float xa = 2.f * au, xb = (2.f * ad + au) * (1.f / 3.f), xc = 2.f * ad;
  float gu = 0.f, gc = 1.f, gd = 0.f;
  float lim = 0.f;
  if (dU * dD > 0.f) {
    if (xa <= xb && xa <= xc) {  // phi = cc + (cc - uu)
      gu = -1.f;
      gc = 2.f;
    } else if (xb <= xc) {       // phi = (5 cc + 2 dd - uu)/6
      gu = -1.f / 6.f;
      gc = 5.f / 6.f;
      gd = 1.f / 3.f;
    } else {                     // phi = dd
      gc = 0.f;
      gd = 1.f;
    }
    lim = copysignf(fminf(fminf(xa, xb), xc), dD);
  }
  const float phi = fmaf(0.5f, lim, cc);
  // F = (a2/2) phi: d/d a2 = phi/2 for both advecting velocities
  const long long ia = map_face<D>(g, j, J), ib = map_face<D>(g, j, jc);
  if (ia >= 0) atomicAdd(ubin[j] + ia, 0.5f * phi * Fb);
  if (ib >= 0) atomicAdd(ubin[j] + ib, 0.5f * phi * Fb);
  const float ha = 0.5f * a2 * Fb;
  const long long iu = map_face<D>(g, c, pos ? m2 : p1), ic = pos ? im1 : ip0, id = pos ? ip0 : im1;
  if (iu >= 0 && gu != 0.f) atomicAdd(ubin[c] + iu, ha * gu);
  if (ic >= 0 && gc != 0.f) atomicAdd(ubin[c] + ic, ha * gc);
  if (id >= 0 && gd != 0.f) atomicAdd(ubin[c] + id, ha * gd);
}

template <int D>
__global__ void __launch_bounds__(256) k_adj_convdiff(Grid g, const float* u0p, const float* u1p, const float* u2p,
                                                      const float* fb0, const float* fb1, const float* fb2,
                                                      const float* dtp, float nu, int advect, float* o0, float* o1,
                                                      float* o2, float* i0, float* i1, float* i2) {
  const long long t = (long long)blockIdx.x * 256 + threadIdx.x;
  if (t >= g.nc * D) return;
  const int c = (int)(t / g.nc);
  const long long q = t - (long long)c * g.nc;
  const float* u[3] = {u0p, u1p, u2p};
  const float* fb[3] = {fb0, fb1, fb2};
  float* ub0[3] = {o0, o1, o2};
  float* ubin[3] = {i0, i1, i2};
  const float dt = *dtp;
  const bool adv = advect != 0;
  int I[3];
  coords(g, q, I);
  const float f = fb[c][q];
  if (f != 0.f) atomicAdd(ub0[c] + q, f);  // f = u0 + dt r
  // r' of face (c, J): dt f' on updated faces, 0 elsewhere (J may wrap periodically)
  auto rbar = [&](const int* J) -> float {
    int K[3] = {J[0], J[1], J[2]};
#pragma unroll
    for (int d = 0; d < D; ++d) {
      if (K[d] < 0 || K[d] >= g.n[d]) {
        if (!is_per(g, d)) return 0.f;
        K[d] = K[d] < 0 ? K[d] + g.n[d] : K[d] - g.n[d];
      }
    }
    if (!face_updated(g, c, K)) return 0.f;
    return dt * fb[c][cell_index(g, K[0], K[1], D == 3 ? K[2] : 0)];
  };
  const float r0 = face_updated(g, c, I) ? dt * f : 0.f;
#pragma unroll
  for (int j = 0; j < D; ++j) {
    int M[3] = {I[0], I[1], I[2]};
    M[j] -= 1;
    const float Fb = r0 - rbar(M);
    if (Fb != 0.f) flux_adjoint<D>(g, u, c, j, I, Fb, nu, adv, ubin);
    if (!is_per(g, j) && I[j] == g.n[j] - 1 && r0 != 0.f) {
      int P[3] = {I[0], I[1], I[2]};
      P[j] += 1;
      flux_adjoint<D>(g, u, c, j, P, -r0, nu, adv, ubin);
    }
  }
}

int launch_adj_convdiff(int D, const Grid& g, const float* const* u, const float* const* fb, const float* dt, float nu,
                        int advect, float* const* ub0, float* const* ubin, cudaStream_t s) {
  const int nb = (int)((g.nc * D + 255) / 256);
  if (D == 3)
    k_adj_convdiff<3><<<nb, 256, 0, s>>>(g, u[0], u[1], u[2], fb[0], fb[1], fb[2], dt, nu, advect, ub0[0], ub0[1],
                                         ub0[2], ubin[0], ubin[1], ubin[2]);
  else
    k_adj_convdiff<2><<<nb, 256, 0, s>>>(g, u[0], u[1], u[1], fb[0], fb[1], fb[1], dt, nu, advect, ub0[0], ub0[1],
                                         ub0[1], ubin[0], ubin[1], ubin[1]);
  return 0;
}

// ---------------------------------------------------------------------------
// theta' += sum over band faces of mbar_c[I] dmu0/dtheta, mu0 = K0(d/eps), K0' = K:
// mbar holds the cotangents of mu0 (BDIM blend) and of L = mu0 (projections); the
// non-periodic boundary faces have L = 0 fixed and are not updated, so they carry none.
template <int D>
__global__ void __launch_bounds__(256) k_adj_moments(Grid g, Body b, const float* mb0, const float* mb1,
                                                     const float* mb2, int lo0, int lo1, int lo2, int bx, int by,
                                                     int bz, AdjState* as) {
  __shared__ double sh[9];
  const float* mb[3] = {mb0, mb1, mb2};
  const long long nbox = (long long)bx * by * bz;
  double acc[4] = {0.0, 0.0, 0.0, 0.0};
  for (long long t = (long long)blockIdx.x * 256 + threadIdx.x; t < nbox * D; t += (long long)gridDim.x * 256) {
    const int c = (int)(t / nbox);
    long long rem = t - (long long)c * nbox;
    const int i = lo0 + (int)(rem % bx);
    rem /= bx;
    const int j = lo1 + (int)(rem % by);
    const int k = lo2 + (int)(rem / by);
    const int I[3] = {i, j, k};
    if (!face_updated(g, c, I)) continue;
    double x[3] = {i + 0.5, j + 0.5, k + 0.5};
    x[c] -= 0.5;
    double n[3], dd[4], dn[3][4];
    const double d = sdf_theta<D>(b, x, n, dd, dn);
    const double sc = d / b.eps;
    if (!(fabs(sc) < 1.0)) continue;
    const double w = (double)mb[c][cell_index(g, i, j, k)] * 0.5 * (1.0 + cospi(sc)) / b.eps;
#pragma unroll
    for (int tt = 0; tt <= D; ++tt) acc[tt] += w * dd[tt];
  }
  for (int tt = 0; tt <= D; ++tt) {
    const double v = block_sum(acc[tt], sh);
    if (threadIdx.x == 0) atomicAdd(&as->theta[tt], v);
  }
}

int launch_adj_moments(int D, const Grid& g, const Body& b, const float* const* mbar, AdjState* as, cudaStream_t s) {
  int lo[3], hi[3];
  band_box(D, g, b, 2.0, lo, hi);
  const int bx = hi[0] - lo[0], by = hi[1] - lo[1], bz = hi[2] - lo[2];
  const long long n = (long long)bx * by * bz * D;
  if (n <= 0) return 0;
  const int nb = (int)std::min<long long>((n + 255) / 256, 1024);
  if (D == 3)
    k_adj_moments<3><<<nb, 256, 0, s>>>(g, b, mbar[0], mbar[1], mbar[2], lo[0], lo[1], lo[2], bx, by, bz, as);
  else
    k_adj_moments<2><<<nb, 256, 0, s>>>(g, b, mbar[0], mbar[1], mbar[1], lo[0], lo[1], lo[2], bx, by, bz, as);
  return 0;
}

}  // namespace wl
