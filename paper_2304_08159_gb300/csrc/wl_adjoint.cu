// Reverse-mode derivative (adjoint) of the time step at a fixed dt with respect to the
// body parameters theta, circle/sphere (R, c_0, .., c_{D-1}) or torus (R, r, c_x, c_y,
// c_z): the differentiable use of the solver (Section 1; the body enters through its
// signed-distance function, Section 2).
//
// Each kernel is the transpose of a forward kernel's arithmetic (same FP32 values, the
// same branch of the limiter and of the upwind switch as the forward takes):
//   k_adj_convdiff    convdiff! (k_stage's fluxes): per face flux, F' = r'[I] - r'[I-e_j],
//                     gathered by every face from the fluxes that read it (BC mapping:
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
      q = wrap_per(q, n);
    } else {
      if (d == c && (q <= 0 || q >= n)) return -1;
      q = q < 0 ? 0 : (q >= n ? n - 1 : q);
    }
    I[d] = q;
  }
  return cell_index(g, I[0], I[1], D == 3 ? I[2] : 0);
}

// Logical positions along direction d that component c's face index K_d stands for:
// the periodic images within [-2, n+1], the clamped positions past a wall for a
// tangential direction, none for a prescribed normal face.  At most 5 (n = 1).
__device__ __forceinline__ int face_preimages(const Grid& g, int c, int d, int k, int* out) {
  const int n = g.n[d];
  int m = 0;
  if (is_per(g, d)) {
    for (int p = k - ((k + 2) / n) * n; p <= n + 1 && m < 5; p += n) out[m++] = p;
  } else if (d == c) {
    if (k >= 1) out[m++] = k;
  } else {
    const int lo = k == 0 ? -2 : k, hi = k == n - 1 ? n + 1 : k;
    for (int p = lo; p <= hi && m < 5; ++p) out[m++] = p;
  }
  return m;
}

// Number of body parameters theta: circle/sphere (R, c_0, .., c_{D-1}); torus
// (R, r, c_x, c_y, c_z), R the ring radius in the y-z plane, r the tube radius.
__host__ __device__ __forceinline__ int n_theta(int kind, int D) { return kind == 2 ? 5 : D + 1; }

// The body's signed distance d and normal n at x, and their derivatives with respect to
// theta: dd[t], dn[j][t].  A centre shift moves the field: dd/dc_k = -n_k, dn_j/dc_k =
// -H_jk with H the Hessian of d.
//   circle/sphere: d = |x - c| - R, n = (x - c)/rho; dd/dR = -1, H = (I - n n^T)/rho.
//   torus: (a, b, c) = x - c, rho = |(b, c)|, e = (b, c)/rho, q = rho - R, s = |(a, q)|:
//     d = s - r, n = (a, q e)/s; dd/dR = -q/s, dd/dr = -1; dn_0/dR = a q/s^3,
//     dn_e/dR = -a^2 e/s^3; H_00 = q^2/s^3, H_0e = -a q e/s^3,
//     H_ee' = a^2 e e'/s^3 + (q/s)(delta_ee' - e e')/rho.
template <int D>
__device__ double sdf_theta(const Body& b, const double* x, double* n, double* dd, double (*dn)[5]) {
#pragma unroll
  for (int t = 0; t < 5; ++t) {
    dd[t] = 0.0;
#pragma unroll
    for (int j = 0; j < 3; ++j) dn[j][t] = 0.0;
  }
  double H[3][3] = {{0.0, 0.0, 0.0}, {0.0, 0.0, 0.0}, {0.0, 0.0, 0.0}};
  n[0] = n[1] = n[2] = 0.0;
  double dist;
  int c0 = 1;
  if (D == 3 && b.kind == 2) {
    const double a = x[0] - b.c[0], bb = x[1] - b.c[1], cc = x[2] - b.c[2];
    const double rho = sqrt(bb * bb + cc * cc), q = rho - b.r1, sd = sqrt(a * a + q * q);
    const double e[3] = {0.0, rho > 0.0 ? bb / rho : 0.0, rho > 0.0 ? cc / rho : 0.0};
    if (sd > 0.0) {
      const double s3 = sd * sd * sd;
      n[0] = a / sd;
      n[1] = q / sd * e[1];
      n[2] = q / sd * e[2];
      dd[0] = -q / sd;
      dn[0][0] = a * q / s3;
      dn[1][0] = -(a * a / s3) * e[1];
      dn[2][0] = -(a * a / s3) * e[2];
      H[0][0] = q * q / s3;
#pragma unroll
      for (int j = 1; j < 3; ++j) H[0][j] = H[j][0] = -a * q * e[j] / s3;
#pragma unroll
      for (int j = 1; j < 3; ++j)
#pragma unroll
        for (int k = 1; k < 3; ++k)
          H[j][k] = e[j] * e[k] * a * a / s3 + (rho > 0.0 ? (q / sd) * ((j == k ? 1.0 : 0.0) - e[j] * e[k]) / rho : 0.0);
    }
    dd[1] = -1.0;
    c0 = 2;
    dist = sd - b.r2;
  } else {
    double r2 = 0.0;
#pragma unroll
    for (int d = 0; d < D; ++d) r2 += (x[d] - b.c[d]) * (x[d] - b.c[d]);
    const double r = sqrt(r2);
#pragma unroll
    for (int d = 0; d < D; ++d) n[d] = r > 0.0 ? (x[d] - b.c[d]) / r : 0.0;
    dd[0] = -1.0;
#pragma unroll
    for (int j = 0; j < D; ++j)
#pragma unroll
      for (int k = 0; k < D; ++k) H[j][k] = r > 0.0 ? ((j == k ? 1.0 : 0.0) - n[j] * n[k]) / r : 0.0;
    dist = r - b.r1;
  }
#pragma unroll
  for (int k = 0; k < D; ++k) {
    dd[c0 + k] = -n[k];
#pragma unroll
    for (int j = 0; j < D; ++j) dn[j][c0 + k] = -H[j][k];
  }
  return dist;
}

// the body's bounding box of cells/faces within `pad` of the band
void band_box(int D, const Grid& g, const Body& b, double pad, int* lo, int* hi) {
  for (int d = 0; d < 3; ++d) {
    lo[d] = 0;
    hi[d] = 1;
    if (d >= D) continue;
    const double ext = b.kind == 2 ? (d == 0 ? b.r2 : b.r1 + b.r2) : b.r1;  // torus: tube across x, ring in y-z
    lo[d] = (int)fmax(0.0, floor(b.c[d] - ext - b.eps - pad));
    hi[d] = (int)fmin((double)g.n[d], ceil(b.c[d] + ext + b.eps + pad) + 1.0);
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
  if (threadIdx.x < 5) as->theta[threadIdx.x] = 0.0;
  if (threadIdx.x == 0) {
    as->mean = 0.0;
    as->bnorm_bits = 0u;
    as->iter = 0;
    as->total_iter = 0;
    as->flags = 0;
    as->rec_slot = 0;
  }
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
  double acc[5] = {0.0, 0.0, 0.0, 0.0, 0.0};
  const int NT = n_theta(b.kind, D);
  const long long nbox = (long long)bx * by * bz;
  for (long long t = threadIdx.x; t < nbox; t += 256) {
    const int i = lo0 + (int)(t % bx);
    const long long r = t / bx;
    const int j = lo1 + (int)(r % by);
    const int k = lo2 + (int)(r / by);
    double x[3] = {i + 0.5, j + 0.5, k + 0.5}, n[3], dd[5], dn[3][5];
    const double d = sdf_theta<D>(b, x, n, dd, dn);
    if (!(fabs(d) < b.eps)) continue;
    const double K = (1.0 + cospi(d / b.eps)) / (2.0 * b.eps);
    const double Kp = -3.141592653589793 * sinpi(d / b.eps) / (2.0 * b.eps * b.eps);
    const double pp = (double)p[cell_index(g, i, j, k)] - pbar;
#pragma unroll
    for (int tt = 0; tt < 5; ++tt) {
      if (tt >= NT) break;
      double gw = 0.0;
#pragma unroll
      for (int e = 0; e < D; ++e) gw += gv[e] * (dn[e][tt] * K + n[e] * Kp * dd[tt]);
      acc[tt] -= pp * gw;
    }
  }
  for (int tt = 0; tt < NT; ++tt) {
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
  if (threadIdx.x == 0) {
    as->mean = as->Na > 0.0 ? v / as->Na : 0.0;
    as->bnorm_bits = 0u;
  }
}

template <int D>
__global__ void __launch_bounds__(256) k_adj_sub_mean(Grid g, const float* L0, const float* L1, const float* L2,
                                                      AdjState* as, float* rhs) {
  const float* L[3] = {L0, L1, L2};
  const long long q = (long long)blockIdx.x * 256 + threadIdx.x;
  float m = 0.f;  // |b| (the max-norm: order-free, so atomics keep it deterministic)
  if (q < g.nc) {
    int I[3];
    coords(g, q, I);
    if (cell_active<D>(g, L, q, I)) {
      const float v = (float)((double)rhs[q] - as->mean);
      rhs[q] = v;
      m = fabsf(v);
    }
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
  if ((threadIdx.x & 31) == 0 && m > 0.f) atomicMax(&as->bnorm_bits, __float_as_uint(m));
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
// with d(eps K1(d/eps))/dd = -s K(s), s = d/eps.  k_adj_band takes the band faces' own
// terms (mbar, theta as per-block partials); k_adj_band_fb gathers the f' terms, each
// face summing the band faces beside it in a fixed order.

// a band face of component c at I: updated, inside the source box and |d| < eps at the
// face centre; its normal n and the weight eps K1(d/eps)
template <int D>
__device__ __forceinline__ bool band_face(const Grid& g, const Body& b, int c, const int* I, const int* lo,
                                          const int* hi, double* n, double& k1) {
#pragma unroll
  for (int d = 0; d < D; ++d)
    if (I[d] < lo[d] || I[d] >= hi[d]) return false;
  if (!face_updated(g, c, I)) return false;
  double x[3] = {I[0] + 0.5, I[1] + 0.5, I[2] + 0.5};
  x[c] -= 0.5;
  double dd[5], dn[3][5];
  const double d = sdf_theta<D>(b, x, n, dd, dn);
  if (!(fabs(d) < b.eps)) return false;
  k1 = b.eps * kernel_K1(d / b.eps);
  return true;
}

template <int D>
__global__ void __launch_bounds__(256) k_adj_band(StageArgs a, Body b, const float* vb0, const float* vb1,
                                                  const float* vb2, float sfac, float* mb0, float* mb1, float* mb2,
                                                  int lo0, int lo1, int lo2, int bx, int by, int bz, double* part) {
  __shared__ double sh[9];
  const long long nbox = (long long)bx * by * bz;
  const Grid& g = a.g;
  const float* vb[3] = {vb0, vb1, vb2};
  float* mb[3] = {mb0, mb1, mb2};
  const float dtf = *a.dt;
  double th[5] = {0.0, 0.0, 0.0, 0.0, 0.0};
  const int NT = n_theta(b.kind, D);
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
    double n[3], dd[5], dn[3][5];
    const double d = sdf_theta<D>(b, x, n, dd, dn);
    if (!(fabs(d) < b.eps)) continue;
    const long long q = cell_index(g, i, j, k);
    const float vs = sfac * vb[c][q];
    mb[c][q] += vs * f_at<D>(a, c, i, j, k, dtf);
    const double sc = d / b.eps, K = 0.5 * (1.0 + cospi(sc));
    const double k1 = b.eps * kernel_K1(sc), k1p = -sc * K;
#pragma unroll
    for (int jd = 0; jd < D; ++jd) {
      int P[3] = {i, j, k}, M[3] = {i, j, k};
      P[jd] += 1;
      M[jd] -= 1;
      const float fp = f_at<D>(a, c, P[0], P[1], P[2], dtf);
      const float fm = f_at<D>(a, c, M[0], M[1], M[2], dtf);
      const double gfd = (double)vs * 0.5 * ((double)fp - (double)fm);
#pragma unroll
      for (int tt = 0; tt < 5; ++tt) th[tt] += gfd * (k1p * n[jd] * dd[tt] + k1 * dn[jd][tt]);
    }
  }
  for (int tt = 0; tt < NT; ++tt) {
    const double v = block_sum(th[tt], sh);
    if (threadIdx.x == 0) part[(size_t)tt * gridDim.x + blockIdx.x] = v;
  }
}

// f'_c[K] += sum over the positions P that map to K and the band faces I = P -+ e_j of
// +- s mu1_j v'_c[I]/2; the target box covers the source box grown by one face (all of a
// periodic direction the grown box wraps in)
template <int D>
__global__ void __launch_bounds__(256) k_adj_band_fb(Grid g, Body b, const float* vb0, const float* vb1,
                                                     const float* vb2, float sfac, float* fb0, float* fb1, float* fb2,
                                                     int lo0, int lo1, int lo2, int hi0, int hi1, int hi2, int t0,
                                                     int t1, int t2, int tx, int ty, int tzn) {
  const long long nt = (long long)tx * ty * tzn;
  const long long t = (long long)blockIdx.x * 256 + threadIdx.x;
  if (t >= nt * D) return;
  const int c = (int)(t / nt);
  long long rem = t - (long long)c * nt;
  int K[3];
  K[0] = t0 + (int)(rem % tx);
  rem /= tx;
  K[1] = t1 + (int)(rem % ty);
  K[2] = t2 + (int)(rem / ty);
  const int lo[3] = {lo0, lo1, lo2}, hi[3] = {hi0, hi1, hi2};
  const float* vb[3] = {vb0, vb1, vb2};
  float* fb[3] = {fb0, fb1, fb2};
  int pre[3][5], np[3] = {1, 1, 1};
  pre[1][0] = pre[2][0] = 0;
#pragma unroll
  for (int d = 0; d < D; ++d) np[d] = face_preimages(g, c, d, K[d], pre[d]);
  float acc = 0.f;
  bool any = false;
  for (int a0 = 0; a0 < np[0]; ++a0)
    for (int a1 = 0; a1 < np[1]; ++a1)
      for (int a2 = 0; a2 < np[2]; ++a2) {
        const int P[3] = {pre[0][a0], pre[1][a1], D == 3 ? pre[2][a2] : 0};
#pragma unroll
        for (int jd = 0; jd < D; ++jd) {
#pragma unroll
          for (int sgn = 0; sgn < 2; ++sgn) {  // the band face below P (+), then above (-)
            int I[3] = {P[0], P[1], P[2]};
            I[jd] += sgn ? 1 : -1;
            double n[3], k1;
            if (!band_face<D>(g, b, c, I, lo, hi, n, k1)) continue;
            const float vs = sfac * vb[c][cell_index(g, I[0], I[1], D == 3 ? I[2] : 0)];
            const float m1 = (float)(k1 * n[jd]) * 0.5f * vs;
            acc += sgn ? -m1 : m1;
            any = true;
          }
        }
      }
  if (any) fb[c][cell_index(g, K[0], K[1], D == 3 ? K[2] : 0)] += acc;
}

// theta' += the partials of nb blocks, each component summed in one fixed order
__global__ void __launch_bounds__(256) k_adj_theta_accum(const double* part, int nb, int nt, AdjState* as) {
  __shared__ double sh[9];
  for (int tt = 0; tt < nt; ++tt) {
    double v = 0.0;
    for (int k = threadIdx.x; k < nb; k += 256) v += part[(size_t)tt * nb + k];
    v = block_sum(v, sh);
    if (threadIdx.x == 0) as->theta[tt] += v;
  }
}

int launch_adj_band(int D, const StageArgs& a, const Body& b, const float* const* vb, float sfac, float* const* fb,
                    float* const* mbar, AdjState* as, double* part, int npart, cudaStream_t s) {
  int lo[3], hi[3];
  band_box(D, a.g, b, 2.0, lo, hi);
  const int bx = hi[0] - lo[0], by = hi[1] - lo[1], bz = hi[2] - lo[2];
  const long long n = (long long)bx * by * bz * D;
  if (n <= 0) return 0;
  const int nb = (int)std::min<long long>((n + 255) / 256, npart / n_theta(b.kind, D));
  const float* v2 = D == 3 ? vb[2] : vb[1];
  if (D == 3)
    k_adj_band<3><<<nb, 256, 0, s>>>(a, b, vb[0], vb[1], vb[2], sfac, mbar[0], mbar[1], mbar[2], lo[0], lo[1], lo[2],
                                     bx, by, bz, part);
  else
    k_adj_band<2><<<nb, 256, 0, s>>>(a, b, vb[0], vb[1], vb[1], sfac, mbar[0], mbar[1], mbar[1], lo[0], lo[1], lo[2],
                                     bx, by, bz, part);
  k_adj_theta_accum<<<1, 256, 0, s>>>(part, nb, n_theta(b.kind, D), as);
  int t0[3] = {0, 0, 0}, tn[3] = {1, 1, 1};
  for (int d = 0; d < D; ++d) {
    const int nd = a.g.n[d];
    int tl = lo[d] - 1, th = hi[d] + 1;
    if (((a.g.per >> d) & 1u) && (tl < 0 || th > nd)) {
      tl = 0;
      th = nd;
    }
    tl = std::max(tl, 0);
    th = std::min(th, nd);
    t0[d] = tl;
    tn[d] = th - tl;
  }
  const long long nt = (long long)tn[0] * tn[1] * tn[2] * D;
  const int nbt = (int)((nt + 255) / 256);
  if (D == 3)
    k_adj_band_fb<3><<<nbt, 256, 0, s>>>(a.g, b, vb[0], vb[1], v2, sfac, fb[0], fb[1], fb[2], lo[0], lo[1], lo[2],
                                         hi[0], hi[1], hi[2], t0[0], t0[1], t0[2], tn[0], tn[1], tn[2]);
  else
    k_adj_band_fb<2><<<nbt, 256, 0, s>>>(a.g, b, vb[0], vb[1], v2, sfac, fb[0], fb[1], fb[1], lo[0], lo[1], lo[2],
                                         hi[0], hi[1], hi[2], t0[0], t0[1], t0[2], tn[0], tn[1], tn[2]);
  return 0;
}

// ---------------------------------------------------------------------------
// f = u0 + dt r(u) on updated faces: u0' += f', and with r' = dt f' the transpose of
// convdiff!, r_c[I] = sum_j F_cj[I] - F_cj[I+e_j].  Flux F_cj[J] (component c, through
// the lower j-face of the control volume at J) exists for J_j in [0, n_j) (and J_j = n_j,
// the upper boundary face, on a wall) and J_d in [0, n_d) otherwise; its cotangent is
// F' = R_c[J] - R_c[J-e_j], R_c = dt f'_c on updated faces (periodic wrap) and 0
// elsewhere.  The flux reads
//   u_c at J-2e_j, J-e_j, J, J+e_j (viscous: J and J-e_j; advective: the upwind three)
//   u_j at J and J-e_c             (the advecting velocity a2 = u_j[J] + u_j[J-e_c])
// and F' times each partial derivative belongs to the face those positions map to.
// The transpose is a gather: the thread of face (c', K) visits every logical position P
// that maps to K (periodic images, the clamped tangential positions past a wall) and
// every flux that reads P, and sums their terms in one fixed order, so the result does
// not depend on the order threads run in.

// Cotangent weights of one flux, as the forward (mom_flux) branches: the upwind side,
// the limiter case and its derivative weights on the upwind three.
struct FluxBar {
  float Fb;              // F'
  float ha, gu, gc, gd;  // advective part: F' a2/2 and dphi/d(uu, cc, dd)
  float hp;              // F' phi/2: the derivative through each advecting velocity
  bool pos;              // a2 > 0 (upwind from below)
};

template <int D>
__device__ __forceinline__ float rbar_at(const Grid& g, const float* fb, int c, const int* J, float dt) {
  int K[3] = {J[0], J[1], J[2]};
#pragma unroll
  for (int d = 0; d < D; ++d) {
    if (K[d] < 0 || K[d] >= g.n[d]) {
      if (!is_per(g, d)) return 0.f;
      K[d] = wrap_per(K[d], g.n[d]);
    }
  }
  if (!face_updated(g, c, K)) return 0.f;
  return dt * fb[cell_index(g, K[0], K[1], D == 3 ? K[2] : 0)];
}

// F' and the weights of flux (c, j) at J; false where J is not a flux position or F' = 0
template <int D>
__device__ __forceinline__ bool flux_bar(const Grid& g, const float* const* u, const float* fb, float dt, bool adv,
                                         int c, int j, const int* J, FluxBar& o) {
#pragma unroll
  for (int d = 0; d < D; ++d) {
    const int hi = g.n[d] + ((d == j && !is_per(g, d)) ? 1 : 0);
    if (J[d] < 0 || J[d] >= hi) return false;
  }
  int M[3] = {J[0], J[1], J[2]};
  M[j] -= 1;
  o.Fb = rbar_at<D>(g, fb, c, J, dt) - rbar_at<D>(g, fb, c, M, dt);
  if (o.Fb == 0.f) return false;
  if (!adv) return true;
  int m2[3] = {J[0], J[1], J[2]}, p1[3] = {J[0], J[1], J[2]}, jc[3] = {J[0], J[1], J[2]};
  m2[j] -= 2;
  p1[j] += 1;
  jc[c] -= 1;
  auto U = [&](int comp, const int* P) { return load_u_bc<D>(u[comp], comp, g, P[0], P[1], P[2]); };
  const float vm2 = U(c, m2), vm1 = U(c, M), vp0 = U(c, J), vp1 = U(c, p1);
  const float a2 = U(j, J) + U(j, jc);
  o.pos = a2 > 0.f;
  const float uu = o.pos ? vm2 : vp1, cc = o.pos ? vm1 : vp0, dd = o.pos ? vp0 : vm1;
  const float dD = dd - cc, dU = cc - uu;
  const float ad = fabsf(dD), au = fabsf(dU);
  const float xa = 2.f * au, xb = (2.f * ad + au) * (1.f / 3.f), xc = 2.f * ad;
  o.gu = 0.f;
  o.gc = 1.f;
  o.gd = 0.f;
  float lim = 0.f;
  if (dU * dD > 0.f) {
    if (xa <= xb && xa <= xc) {  // phi = cc + (cc - uu)
      o.gu = -1.f;
      o.gc = 2.f;
    } else if (xb <= xc) {       // phi = (5 cc + 2 dd - uu)/6
      o.gu = -1.f / 6.f;
      o.gc = 5.f / 6.f;
      o.gd = 1.f / 3.f;
    } else {                     // phi = dd
      o.gc = 0.f;
      o.gd = 1.f;
    }
    lim = copysignf(fminf(fminf(xa, xb), xc), dD);
  }
  const float phi = fmaf(0.5f, lim, cc);
  o.hp = 0.5f * phi * o.Fb;
  o.ha = 0.5f * a2 * o.Fb;
  return true;
}

// sum over the fluxes that read position P of component c of F' dF/du(P), in a fixed order
template <int D>
__device__ float flux_gather_at(const Grid& g, const float* const* u, const float* const* fb, float dt, float nu,
                                bool adv, int c, const int* P) {
  float acc = 0.f;
  FluxBar f;
#pragma unroll 1
  for (int j = 0; j < D; ++j) {
    int J[3] = {P[0], P[1], P[2]};
    // P = J (viscous -nu F'; the advective cc or dd)
    if (flux_bar<D>(g, u, fb[c], dt, adv, c, j, J, f)) {
      acc += -nu * f.Fb;
      if (adv) acc += f.ha * (f.pos ? f.gd : f.gc);
    }
    // P = J - e_j (viscous +nu F'; cc or dd)
    J[j] = P[j] + 1;
    if (flux_bar<D>(g, u, fb[c], dt, adv, c, j, J, f)) {
      acc += nu * f.Fb;
      if (adv) acc += f.ha * (f.pos ? f.gc : f.gd);
    }
    if (!adv) continue;
    // P = J - 2e_j: the upwind uu from below
    J[j] = P[j] + 2;
    if (flux_bar<D>(g, u, fb[c], dt, adv, c, j, J, f) && f.pos) acc += f.ha * f.gu;
    // P = J + e_j: the upwind uu from above
    J[j] = P[j] - 1;
    if (flux_bar<D>(g, u, fb[c], dt, adv, c, j, J, f) && !f.pos) acc += f.ha * f.gu;
  }
  if (!adv) return acc;
  // P as an advecting velocity: fluxes (m, j = c) at J = P and J = P + e_m
#pragma unroll 1
  for (int m = 0; m < D; ++m) {
    int J[3] = {P[0], P[1], P[2]};
    if (flux_bar<D>(g, u, fb[m], dt, adv, m, c, J, f)) acc += f.hp;
    J[m] = P[m] + 1;
    if (flux_bar<D>(g, u, fb[m], dt, adv, m, c, J, f)) acc += f.hp;
  }
  return acc;
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
  int K[3];
  coords(g, q, K);
  int pre[3][5], np[3] = {1, 1, 1};
  pre[1][0] = pre[2][0] = 0;
#pragma unroll
  for (int d = 0; d < D; ++d) np[d] = face_preimages(g, c, d, K[d], pre[d]);
  float acc = 0.f;
  for (int a = 0; a < np[0]; ++a)
    for (int b = 0; b < np[1]; ++b)
      for (int e = 0; e < np[2]; ++e) {
        const int P[3] = {pre[0][a], pre[1][b], D == 3 ? pre[2][e] : 0};
        acc += flux_gather_at<D>(g, u, fb, dt, nu, adv, c, P);
      }
  const float f = fb[c][q];  // f = u0 + dt r: u0' += f'
  if (ub0[c] == ubin[c]) {
    ubin[c][q] = (ubin[c][q] + f) + acc;
  } else {
    ub0[c][q] += f;
    ubin[c][q] += acc;
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
                                                     int bz, double* part) {
  __shared__ double sh[9];
  const float* mb[3] = {mb0, mb1, mb2};
  const long long nbox = (long long)bx * by * bz;
  double acc[5] = {0.0, 0.0, 0.0, 0.0, 0.0};
  const int NT = n_theta(b.kind, D);
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
    double n[3], dd[5], dn[3][5];
    const double d = sdf_theta<D>(b, x, n, dd, dn);
    const double sc = d / b.eps;
    if (!(fabs(sc) < 1.0)) continue;
    const double w = (double)mb[c][cell_index(g, i, j, k)] * 0.5 * (1.0 + cospi(sc)) / b.eps;
#pragma unroll
    for (int tt = 0; tt < 5; ++tt) acc[tt] += w * dd[tt];
  }
  for (int tt = 0; tt < NT; ++tt) {
    const double v = block_sum(acc[tt], sh);
    if (threadIdx.x == 0) part[(size_t)tt * gridDim.x + blockIdx.x] = v;
  }
}

int launch_adj_moments(int D, const Grid& g, const Body& b, const float* const* mbar, AdjState* as, double* part,
                       int npart, cudaStream_t s) {
  int lo[3], hi[3];
  band_box(D, g, b, 2.0, lo, hi);
  const int bx = hi[0] - lo[0], by = hi[1] - lo[1], bz = hi[2] - lo[2];
  const long long n = (long long)bx * by * bz * D;
  if (n <= 0) return 0;
  const int nb = (int)std::min<long long>((n + 255) / 256, npart / n_theta(b.kind, D));
  if (D == 3)
    k_adj_moments<3><<<nb, 256, 0, s>>>(g, b, mbar[0], mbar[1], mbar[2], lo[0], lo[1], lo[2], bx, by, bz, part);
  else
    k_adj_moments<2><<<nb, 256, 0, s>>>(g, b, mbar[0], mbar[1], mbar[1], lo[0], lo[1], lo[2], bx, by, bz, part);
  k_adj_theta_accum<<<1, 256, 0, s>>>(part, nb, n_theta(b.kind, D), as);
  return 0;
}

// V-cycle decision of an adjoint solve (the forward's decision with a relative stop):
// stop once ||r||_inf <= rtol ||b||_inf (or r = 0; ||b||_inf from the right-hand side),
// or, flagged, at maxit cycles or a non-finite residual.  Resets the max-norm and sets
// the 16-bit coarse levels' scale as the forward's decision does.
__global__ void k_adj_decide(DevState* st, AdjState* as, cudaGraphConditionalHandle h, int use_handle, int first,
                             double rtol, int maxit) {
  const float nrm = __uint_as_float(st->norm_bits);
  st->norm_bits = 0u;
  if (nrm > 0.f && isfinite(nrm)) st->cs_used = min(max(-ilogbf(nrm) - 6, -100), 100);
  const double r = (double)nrm, bnorm = (double)__uint_as_float(as->bnorm_bits);
  if (first) {
    as->iter = 0;
  } else {
    as->iter += 1;
    as->total_iter += 1;
  }
  bool cont = false;
  if (!isfinite(r))
    as->flags |= 1;
  else if (r <= rtol * bnorm || r == 0.0)
    cont = false;
  else if (as->iter >= maxit)
    as->flags |= 2;
  else
    cont = true;
  st->cond = cont ? 1 : 0;
  if (use_handle) cudaGraphSetConditional(h, cont ? 1u : 0u);
}

int launch_adj_decide(DevState* st, AdjState* as, cudaGraphConditionalHandle h, int use_handle, int first,
                      double rtol, int maxit, cudaStream_t s) {
  k_adj_decide<<<1, 1, 0, s>>>(st, as, h, use_handle, first, rtol, maxit);
  return 0;
}

__global__ void __launch_bounds__(256) k_adj_record(const float* s0, const float* s1, const float* s2, int nf,
                                                    const float* pl, float* seg, const AdjState* as, size_t stride,
                                                    int off, long long n) {
  const long long t = (long long)blockIdx.x * 256 + threadIdx.x;
  if (t >= n * nf) return;
  const int f = (int)(t / n);
  const long long q = t - (long long)f * n;
  const float* src = f == 0 ? s0 : (f == 1 ? s1 : s2);
  float* dst = seg + (size_t)as->rec_slot * stride + (size_t)(off + f) * n;
  dst[q] = pl ? src[q] + pl[q] : src[q];
}

int launch_adj_record(const float* const* src, int nf, const float* pl, float* seg, const AdjState* as,
                      size_t stride, int off, long long n, cudaStream_t s) {
  if (n <= 0 || nf <= 0) return 0;
  k_adj_record<<<(int)((n * nf + 255) / 256), 256, 0, s>>>(src[0], nf > 1 ? src[1] : src[0], nf > 2 ? src[2] : src[0],
                                                           nf, pl, seg, as, stride, off, n);
  return 0;
}

__global__ void k_adj_set_slot(AdjState* as, int slot) { as->rec_slot = slot; }

__global__ void __launch_bounds__(256) k_adj_warm(float* x, float* xl, const float* yprev, const AdjState* as,
                                                  long long n) {
  const long long q = (long long)blockIdx.x * 256 + threadIdx.x;
  if (q >= n) return;
  x[q] = as->bnorm_bits ? yprev[q] : 0.f;
  if (xl) xl[q] = 0.f;
}

int launch_adj_warm(float* x, float* xl, const float* yprev, const AdjState* as, long long n, cudaStream_t s) {
  k_adj_warm<<<(int)((n + 255) / 256), 256, 0, s>>>(x, xl, yprev, as, n);
  return 0;
}

int launch_adj_set_slot(AdjState* as, int slot, cudaStream_t s) {
  k_adj_set_slot<<<1, 1, 0, s>>>(as, slot);
  return 0;
}

}  // namespace wl
