// Device-side building blocks shared by the kernels of libwl.so.
//
// Storage: every field is float32 (the coarse multigrid levels optionally 16-bit),
// interior cells only, x fastest.  There are no
// ghost cells in memory: the domain boundary conditions (BC!, Table 2) are applied
// on the fly by mapping an out-of-range index to the value the BC defines
// ("virtual ghosts").  This removes the separate BC kernel and its traffic.
#pragma once
#include <cstdint>
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>

namespace wl {

struct Grid {
  int n[3];        // cells per direction (n[2] = 1 in 2-D)
  unsigned per;    // bit d: direction d periodic
  float U[3];      // boundary velocity (normal component on non-periodic sides)
  long long nc;    // cells
  int exit;        // 1: convective exit on the upper x face; its normal velocity is stored
                   //    after the n_c values of every velocity's x component (n_1 n_2 values)
};

// Index of the exit-plane value of row (j, k) after the x component's cells.
__host__ __device__ inline long long exit_index(const Grid& g, int j, int k) {
  return g.nc + (long long)j + (long long)g.n[1] * k;
}

__device__ __forceinline__ bool is_per(const Grid& g, int d) { return (g.per >> d) & 1u; }

// Index q of a periodic direction of n cells brought into [0, n).  Every position an owned
// cell's stencil reads lies within one period of the grid (the stencils reach two cells,
// n >= 2), where this is the exact wrap.  A tile's halo on a level narrower than the tile
// reaches further, to positions no owned cell reads; those are clamped into the array
// (any value there is unused, and the access stays in bounds).  Two compares and a
// clamp: short code in the register-bound kernels.
__host__ __device__ __forceinline__ int wrap_per(int q, int n) {
  q = q < 0 ? q + n : (q >= n ? q - n : q);
  return q < 0 ? 0 : (q >= n ? n - 1 : q);
}

// ---- Bounds-checked build (compiled with WL_DEBUG_BOUNDS into libwl_debug.so): an index
// outside its array sets a bit of this translation unit's flag word and the access is
// skipped, so a bad index is reported instead of corrupting memory or faulting (no trap).
// The release build compiles every check to `true`.  Bits: WL_DBG_*.
enum : unsigned {
  WL_DBG_STAGE = 1u, WL_DBG_BAND = 2u, WL_DBG_SWEEP = 4u, WL_DBG_RESID = 8u, WL_DBG_CORRECT = 16u,
  WL_DBG_RESTRICT = 32u, WL_DBG_TMA = 64u, WL_DBG_COARSE = 128u, WL_DBG_BATCH = 256u
};
#ifdef WL_DEBUG_BOUNDS
static __device__ unsigned wl_dbg_bits;
__device__ __forceinline__ bool wl_in(long long i, long long n, unsigned bit) {
  if (i >= 0 && i < n) return true;
  atomicOr(&wl_dbg_bits, bit);
  return false;
}
#else
__device__ __forceinline__ bool wl_in(long long, long long, unsigned) { return true; }
#endif

// Storage types of the coarse multigrid levels' fields (wl_opts.coarse_precision):
// values are stored in 16 bits and every operation on them runs in FP32.
enum { ST_F32 = 0, ST_BF16 = 1, ST_F16 = 2 };

__device__ __forceinline__ float ldf(const float* p, long long i) { return __ldg(p + i); }
__device__ __forceinline__ float ldf(const __nv_bfloat16* p, long long i) { return __bfloat162float(__ldg(p + i)); }
__device__ __forceinline__ float ldf(const __half* p, long long i) { return __half2float(__ldg(p + i)); }
template <typename T>
__device__ __forceinline__ T from_f(float v);
template <>
__device__ __forceinline__ float from_f<float>(float v) { return v; }
template <>
__device__ __forceinline__ __nv_bfloat16 from_f<__nv_bfloat16>(float v) { return __float2bfloat16_rn(v); }
template <>
__device__ __forceinline__ __half from_f<__half>(float v) { return __float2half_rn(v); }
// Two adjacent values (index i even, so the pair is 4/8-byte aligned) stored at once.
__device__ __forceinline__ void st_pair(float* p, long long i, float a, float b) {
  *reinterpret_cast<float2*>(p + i) = make_float2(a, b);
}
__device__ __forceinline__ void st_pair(__nv_bfloat16* p, long long i, float a, float b) {
  *reinterpret_cast<__nv_bfloat162*>(p + i) = __floats2bfloat162_rn(a, b);
}
__device__ __forceinline__ void st_pair(__half* p, long long i, float a, float b) {
  *reinterpret_cast<__half2*>(p + i) = __floats2half2_rn(a, b);
}
// Load / store by a run-time storage type (ST_*), for fields touched once per cell.
__device__ __forceinline__ float ld_st(const void* p, int type, long long i) {
  if (type == ST_BF16) return ldf(static_cast<const __nv_bfloat16*>(p), i);
  if (type == ST_F16) return ldf(static_cast<const __half*>(p), i);
  return ldf(static_cast<const float*>(p), i);
}
__device__ __forceinline__ void st_st(void* p, int type, long long i, float v) {
  if (type == ST_BF16)
    static_cast<__nv_bfloat16*>(p)[i] = __float2bfloat16_rn(v);
  else if (type == ST_F16)
    static_cast<__half*>(p)[i] = __float2half_rn(v);
  else
    static_cast<float*>(p)[i] = v;
}

__device__ __forceinline__ long long cell_index(const Grid& g, int i, int j, int k) {
  return (long long)i + (long long)g.n[0] * ((long long)j + (long long)g.n[1] * k);
}

// Velocity component c at face index (i,j,k), which may lie up to two cells outside
// the interior in any direction.  BC (Table 2): along a non-periodic direction d the
// normal component (c == d) takes U_c on the boundary faces (index 0 and n_d) and
// beyond; the tangential components copy the nearest interior value; periodic
// directions wrap.  Requires n_d >= 2.
template <int D>
__device__ __forceinline__ float load_u_bc(const float* __restrict__ uc, int c, const Grid& g, int i, int j,
                                           int k) {
  if (c == 0 && g.exit && i >= g.n[0]) {
    // convective exit: the exit face and the faces beyond it (zero gradient) read the
    // stored exit plane at the row (y clamped / wrapped like a tangential component)
    int J = j, K = D == 3 ? k : 0;
    if (is_per(g, 1))
      J = wrap_per(J, g.n[1]);
    else
      J = J < 0 ? 0 : (J >= g.n[1] ? g.n[1] - 1 : J);
    if (D == 3) {
      if (is_per(g, 2))
        K = wrap_per(K, g.n[2]);
      else
        K = K < 0 ? 0 : (K >= g.n[2] ? g.n[2] - 1 : K);
    }
    return __ldg(uc + exit_index(g, J, K));
  }
  int I[3] = {i, j, k};
#pragma unroll
  for (int d = 0; d < D; ++d) {
    int q = I[d];
    const int n = g.n[d];
    if (is_per(g, d)) {
      q = wrap_per(q, n);
    } else {
      if (d == c && (q <= 0 || q >= n)) return g.U[c];
      q = q < 0 ? 0 : (q >= n ? n - 1 : q);
    }
    I[d] = q;
  }
  return __ldg(uc + cell_index(g, I[0], I[1], D == 3 ? I[2] : 0));
}

// Momentum flux through the lower j-face of the u_c control volume:
//   F = a*phi - nu*(p0 - m1),  a = a2/2,
// where (m2, m1, p0, p1) = u_c at I-2e_j, I-e_j, I, I+e_j and a2 = u_j[I] + u_j[I-e_c].
// phi is the kappa = 1/3 upwind-biased face value limited by Koren's limiter
// (third-order convection with implicit LES, Section 2): with upwind/centre/
// downwind (u, c, d) taken on the side a comes from, phi = c + psi(r)(d - c)/2,
// r = (c - u)/(d - c), psi = max(0, min(2r, (2+r)/3, 2)).  Written without the
// division: for (c-u)(d-c) > 0, psi*(d-c) = sign(d-c) min(2|c-u|, (2|d-c|+|c-u|)/3,
// 2|d-c|); otherwise 0.
__device__ __forceinline__ float mom_flux(float m2, float m1, float p0, float p1, float a2, float nu,
                                          bool advect) {
  float diff = nu * (p0 - m1);
  if (!advect) return -diff;
  const bool pos = a2 > 0.f;
  const float uu = pos ? m2 : p1;
  const float cc = pos ? m1 : p0;
  const float dd = pos ? p0 : m1;
  const float dD = dd - cc, dU = cc - uu;
  const float ad = fabsf(dD), au = fabsf(dU);
  const float t = fminf(fminf(2.f * au, (2.f * ad + au) * (1.f / 3.f)), 2.f * ad);
  const float lim = (dU * dD > 0.f) ? copysignf(t, dD) : 0.f;
  const float phi = fmaf(0.5f, lim, cc);
  return fmaf(0.5f * a2, phi, -diff);
}

// ---------------------------------------------------------------------------
// Immersed body: analytic signed distance and outward unit normal (Section 2: the
// geometry is a signed-distance function; normals are its gradient).
struct Body {
  int kind;          // 0 none, 1 circle/sphere, 2 torus (3-D), 3 sampled distance
  double c[3];
  double r1, r2;     // radius; torus tube radius
  double eps;        // BDIM kernel half-width
  const float* nodes;  // kind 3: signed distance at the grid's nodes (device), x fastest
  int nn[3];           //   node counts (n_d + 1; 1 for the unused z of 2-D)
  int blo[3], bhi[3];  //   cells whose corners bracket |d| < eps ([lo, hi), computed on the host)
};

// FP32 estimate of the analytic bodies' signed distance (circle/sphere, torus), for
// skipping faces far outside the band before the FP64 evaluation: with coordinates below
// 2^16 cells its error is far below a tenth of a cell.  Other bodies: 0 (no skip).
template <int D>
__device__ __forceinline__ float body_dist_f(const Body& b, const double* x) {
  const float a = (float)(x[0] - b.c[0]), bb = (float)(x[1] - b.c[1]), cc = D == 3 ? (float)(x[2] - b.c[2]) : 0.f;
  if (b.kind == 1) return sqrtf(a * a + bb * bb + cc * cc) - (float)b.r1;
  if (b.kind == 2 && D == 3) {
    const float q = sqrtf(bb * bb + cc * cc) - (float)b.r1;
    return sqrtf(a * a + q * q) - (float)b.r2;
  }
  return 0.f;
}

template <int D>
__device__ __forceinline__ double body_sdf(const Body& b, const double* x, double* n) {
  n[0] = n[1] = n[2] = 0.0;
  if (b.kind == 1) {
    double r2 = 0.0;
#pragma unroll
    for (int d = 0; d < D; ++d) r2 += (x[d] - b.c[d]) * (x[d] - b.c[d]);
    double r = sqrt(r2);
    if (r > 0.0) {
#pragma unroll
      for (int d = 0; d < D; ++d) n[d] = (x[d] - b.c[d]) / r;
    }
    return r - b.r1;
  }
  if (b.kind == 2 && D == 3) {
    double a = x[0] - b.c[0], bb = x[1] - b.c[1], cc = x[2] - b.c[2];
    double rho = sqrt(bb * bb + cc * cc);
    double q1 = rho - b.r1;
    double dq = sqrt(a * a + q1 * q1);
    if (dq > 0.0) {
      double e1 = rho > 0.0 ? bb / rho : 0.0, e2 = rho > 0.0 ? cc / rho : 0.0;
      n[0] = a / dq;
      n[1] = q1 / dq * e1;
      n[2] = q1 / dq * e2;
    }
    return dq - b.r2;
  }
  if (b.kind == 3) {
    // sampled: multilinear between the nodes of the cell holding x; the normal is the
    // normalised gradient of that interpolant
    int c0[3] = {0, 0, 0};
    double f[3] = {0.0, 0.0, 0.0};
#pragma unroll
    for (int d = 0; d < D; ++d) {
      c0[d] = max(0, min(b.nn[d] - 2, (int)floor(x[d])));
      f[d] = x[d] - c0[d];
    }
    const long long s1 = b.nn[0], s2 = (long long)b.nn[0] * b.nn[1];
    const long long base = c0[0] + s1 * c0[1] + (D == 3 ? s2 * c0[2] : 0);
    const double w0[2] = {1.0 - f[0], f[0]}, w1[2] = {1.0 - f[1], f[1]};
    const double w2[2] = {D == 3 ? 1.0 - f[2] : 1.0, D == 3 ? f[2] : 0.0};
    double dist = 0.0, g[3] = {0.0, 0.0, 0.0};
#pragma unroll
    for (int a = 0; a < 2; ++a)
#pragma unroll
      for (int bb = 0; bb < 2; ++bb)
#pragma unroll
        for (int c = 0; c < (D == 3 ? 2 : 1); ++c) {
          const double v = (double)b.nodes[base + a + s1 * bb + (D == 3 ? s2 * c : 0)];
          dist += w0[a] * w1[bb] * w2[c] * v;
          g[0] += (a ? 1.0 : -1.0) * w1[bb] * w2[c] * v;
          g[1] += (bb ? 1.0 : -1.0) * w0[a] * w2[c] * v;
          if (D == 3) g[2] += (c ? 1.0 : -1.0) * w0[a] * w1[bb] * v;
        }
    const double gn = sqrt(g[0] * g[0] + g[1] * g[1] + g[2] * g[2]);
    if (gn > 0.0) {
#pragma unroll
      for (int d = 0; d < D; ++d) n[d] = g[d] / gn;
    }
    return dist;
  }
  return 1e30;
}

// Moments of the cosine kernel K(s) = (1 + cos(pi s))/2 on [-1, 1] (BDIM, Section 2;
// Weymouth & Yue 2011): K0(s) = int_{-1}^s K  (a CDF, kept in [0, 1]) and
// K1(s) = int_s^1 t K(t) dt.  Evaluated in FP64: near s = -1, K0 ~ pi^2 (s+1)^3/12
// comes out of a cancellation that FP32 cannot resolve.
__device__ __forceinline__ double kernel_K0(double s) {
  if (s <= -1.0) return 0.0;
  if (s >= 1.0) return 1.0;
  double v = 0.5 + 0.5 * s + sinpi(s) * (0.5 / 3.141592653589793);
  return v < 0.0 ? 0.0 : (v > 1.0 ? 1.0 : v);
}
__device__ __forceinline__ double kernel_K1(double s) {
  if (s <= -1.0 || s >= 1.0) return 0.0;
  const double ip = 1.0 / 3.141592653589793;
  return 0.25 * (1.0 - s * s) - (s * sinpi(s) + (1.0 + cospi(s)) * ip) * (0.5 * ip);
}

// ---------------------------------------------------------------------------
// Device-resident scalars of one sim (dt and the convergence bookkeeping live on
// the device so a step never waits for the host).
struct DevState {
  double dt;              // dt of the next step
  float dtf;              // FP32 copies of dt and 1/dt read by the per-cell kernels
  float inv_dtf;
  double time;            // simulated time
  long long steps;
  unsigned norm_bits;     // running max |residual| (float bits; non-negative floats order as uints)
  unsigned cfl_bits;      // running max out-flux (float bits)
  int iter;               // V-cycles of the projection in progress
  int cond;               // 1 while the projection loop continues
  float res_x;            // last residual in x = p*w*dt units
  int last_iters[2];      // V-cycles of the two projections of the last step
  float last_res[2];
  long long total_vcycles;
  float worst_res;
  int status;             // bit 0: non-finite seen; bit 1: max_vcycles hit
  int proj_index;         // 0 / 1: which projection of the step is running
  int cs_used;            // 16-bit coarse levels: their values carry the factor 2^cs_used, set
                          // from the max-norm of the residual they correct (so that FP16's range
                          // holds the correction whatever the residual's size)
  long long mcount;       // per-step metric records written (the ring holds the last WL_METRIC_RING)
  double ke;              // metrics of the velocity at the end of the step (wl_opts.metrics = 1):
  unsigned maxdiv_bits;   //   kinetic energy, max |div u| (float bits)
  int pad_;
};

__device__ __forceinline__ void atomic_max_nonneg(unsigned* addr, float v) {
  // |v| of a finite or non-finite float: NaN and Inf order above every finite value
  atomicMax(addr, __float_as_uint(fabsf(v)));
}

// Block-wide maximum of non-negative float bit patterns (NaN and Inf order above
// every finite value, so a non-finite residual is never hidden).
template <int NT>
__device__ __forceinline__ unsigned block_max_bits(unsigned v, unsigned* sh) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = max(v, __shfl_xor_sync(0xffffffffu, v, o));
  const int w = threadIdx.x / 32, l = threadIdx.x % 32;
  if (l == 0) sh[w] = v;
  __syncthreads();
  if (w == 0) {
    v = (l < NT / 32) ? sh[l] : 0u;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = max(v, __shfl_xor_sync(0xffffffffu, v, o));
  }
  return v;  // valid in thread 0
}

// Error-free transformations (Knuth's TwoSum; Dekker's product via FMA): s + e is
// exactly a + b, p + e exactly a * b.  Used for the double-float pressure.
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
  s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}
__device__ __forceinline__ void two_prod(float a, float b, float& p, float& e) {
  p = __fmul_rn(a, b);
  e = fmaf(a, b, -p);
}
// renormalise hi + lo so that |lo| <= ulp(hi)/2 (requires |hi| >= |lo|)
__device__ __forceinline__ void fast_two_sum(float a, float b, float& s, float& e) {
  s = __fadd_rn(a, b);
  e = __fsub_rn(b, __fsub_rn(s, a));
}

// Packed FP32 pairs (two lanes per instruction, sm_100 and later).  Each lane rounds
// exactly as the scalar operation does, so a packed path gives the scalar path's bits.
__device__ __forceinline__ float2 neg2(float2 a) { return make_float2(-a.x, -a.y); }
__device__ __forceinline__ float2 add2(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 sub2(float2 a, float2 b) { return __fadd2_rn(a, neg2(b)); }
__device__ __forceinline__ float2 mul2(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ void two_sum2(float2 a, float2 b, float2& s, float2& e) {
  s = add2(a, b);
  const float2 bb = sub2(s, a);
  e = add2(sub2(a, sub2(s, bb)), sub2(b, bb));
}
__device__ __forceinline__ void two_prod2(float2 a, float2 b, float2& p, float2& e) {
  p = mul2(a, b);
  e = fma2(a, b, neg2(p));
}

}  // namespace wl
