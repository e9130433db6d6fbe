// wl_forces_noalloc: the pressure force of wl_forces, computed from fields the caller
// already holds on the device, for callers that must not allocate device memory.
//
// Who needs it: code that runs where a device allocation is not allowed or not safe,
// for example inside a region being captured into a CUDA graph (cudaMalloc is not a
// stream operation and cannot be captured), inside a real-time loop whose memory was
// budgeted up front, or under an external allocator that owns the whole device and
// forbids side allocations.  Such callers hand over the pressure and face-coefficient
// fields and a small output buffer; the reduction's scratch lives in a fixed,
// file-scope device array instead of a workspace.
//
// Limits and sharing: the scratch holds one pair of partial sums per block of
// kChunk cells, kParts pairs at most, so grids of more than kParts * kChunk cells are
// rejected.  Every GPU that loads the library holds this array (256 KiB) until the
// process exits.  All calls share it: each call overwrites the partial sums it needs
// before reading them (nothing has to start at zero), so calls that overlap on the GPU
// (on different streams, or from different host threads without ordering) race.
#include <cuda_runtime.h>

#include <mutex>

#include "wl.h"
#include "wl_dev.cuh"

namespace {

constexpr int kParts = 16384;  // partial-sum pairs
constexpr int kChunk = 4096;   // cells per block
constexpr int kMaxDevices = 64;

// file-scope scratch of the force reduction: (sum of p over active cells, count) per block
__device__ __align__(256) double g_force_scratch[2 * kParts];

std::mutex g_mutex;
double* g_scratch_addr[kMaxDevices] = {};

// Device address of g_force_scratch on the current device (looked up once per device;
// in host code the symbol itself is only a host-side stand-in).
int scratch_address(double** out) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
    cudaGetLastError();
    return WL_ECUDA;
  }
  std::lock_guard<std::mutex> lock(g_mutex);
  if (!g_scratch_addr[dev]) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_force_scratch) != cudaSuccess || !p) {
      cudaGetLastError();
      return WL_ECUDA;
    }
    g_scratch_addr[dev] = static_cast<double*>(p);
  }
  *out = g_scratch_addr[dev];
  return WL_OK;
}

// Pass 1: block b sums p over the active cells (nonzero Poisson row) of its chunk.
template <int D>
__global__ void __launch_bounds__(256) k_noalloc_partials(wl::Grid g, const float* p, const float* L,
                                                          double* scratch) {
  __shared__ double sh[2][8];
  const long long q0 = (long long)blockIdx.x * kChunk;
  const long long q1 = q0 + kChunk < g.nc ? q0 + kChunk : g.nc;
  double sp = 0.0, sc = 0.0;
  for (long long q = q0 + threadIdx.x; q < q1; q += 256) {
    int I[3];
    I[0] = (int)(q % g.n[0]);
    const long long t = q / g.n[0];
    I[1] = (int)(t % g.n[1]);
    I[2] = (int)(t / g.n[1]);
    const long long st[3] = {1, (long long)g.n[0], (long long)g.n[0] * g.n[1]};
    float dg = 0.f;
#pragma unroll
    for (int c = 0; c < D; ++c) {
      const float* Lc = L + (long long)c * g.nc;
      dg += Lc[q];
      if (I[c] + 1 < g.n[c])
        dg += Lc[q + st[c]];
      else if (wl::is_per(g, c))
        dg += Lc[q - (long long)(g.n[c] - 1) * st[c]];
    }
    if (dg > 0.f) {
      sp += (double)p[q];
      sc += 1.0;
    }
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    sp += __shfl_xor_sync(0xffffffffu, sp, o);
    sc += __shfl_xor_sync(0xffffffffu, sc, o);
  }
  if ((threadIdx.x & 31) == 0) {
    sh[0][threadIdx.x >> 5] = sp;
    sh[1][threadIdx.x >> 5] = sc;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double a = 0.0, b = 0.0;
    for (int w = 0; w < 8; ++w) {
      a += sh[0][w];
      b += sh[1][w];
    }
    scratch[2 * blockIdx.x] = a;
    scratch[2 * blockIdx.x + 1] = b;
  }
}

__device__ double block_sum(double v, double* sh) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  __syncthreads();
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = v;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < 8; ++w) t += sh[w];
    sh[8] = t;
  }
  __syncthreads();
  return sh[8];
}

// Pass 2 (one block): mean pressure from the partials in a fixed order, then
// F_d = -sum over cells with |d| < eps of (p - pbar) n_d (1 + cos(pi d/eps))/(2 eps).
template <int D>
__global__ void __launch_bounds__(256) k_noalloc_final(wl::Grid g, wl::Body b, const float* p,
                                                       const double* scratch, int nparts, int lo0, int lo1, int lo2,
                                                       int bx, int by, int bz, double* F) {
  __shared__ double sh[9];
  double sp = 0.0, sc = 0.0;
  for (int k = threadIdx.x; k < nparts; k += 256) {
    sp += scratch[2 * k];
    sc += scratch[2 * k + 1];
  }
  sp = block_sum(sp, sh);
  sc = block_sum(sc, sh);
  const double pbar = sc > 0.0 ? sp / sc : 0.0;
  double acc[3] = {0.0, 0.0, 0.0};
  const long long nbox = (long long)bx * by * bz;
  for (long long t = threadIdx.x; t < nbox; t += 256) {
    const int i = lo0 + (int)(t % bx);
    const long long r = t / bx;
    const int j = lo1 + (int)(r % by);
    const int k = lo2 + (int)(r / by);
    double x[3] = {i + 0.5, j + 0.5, k + 0.5}, n[3];
    const double d = wl::body_sdf<D>(b, x, n);
    if (!(fabs(d) < b.eps)) continue;
    const double K = (1.0 + cospi(d / b.eps)) / (2.0 * b.eps);
    const double pp = (double)p[wl::cell_index(g, i, j, k)] - pbar;
#pragma unroll
    for (int c = 0; c < D; ++c) acc[c] -= pp * n[c] * K;
  }
  for (int c = 0; c < D; ++c) {
    const double v = block_sum(acc[c], sh);
    if (threadIdx.x == 0) F[c] = v;
  }
}

}  // namespace

extern "C" int wl_forces_noalloc(const int* dims, int ndim, unsigned periodic_mask, const wl_body* body, double eps,
                                 const float* p, const float* L, double* F, void* stream) {
  if (!dims || !body || !p || !L || !F || (ndim != 2 && ndim != 3) || !(eps > 0.0)) return WL_EINVAL;
  if (body->kind < 0 || body->kind > 2 || (body->kind == 2 && ndim != 3)) return WL_EINVAL;
  wl::Grid g{};
  long long nc = 1;
  for (int d = 0; d < 3; ++d) {
    g.n[d] = d < ndim ? dims[d] : 1;
    if (g.n[d] < 1) return WL_EINVAL;
    nc *= g.n[d];
  }
  // the static scratch bounds the grid: one partial pair per kChunk cells
  if (nc > (long long)kParts * kChunk) return WL_EINVAL;
  g.nc = nc;
  g.per = periodic_mask & ((1u << ndim) - 1u);
  wl::Body b{};
  b.kind = body->kind;
  for (int d = 0; d < 3; ++d) b.c[d] = body->center[d];
  b.r1 = body->radius;
  b.r2 = body->radius2;
  b.eps = eps;
  double* scratch = nullptr;
  int rc = scratch_address(&scratch);
  if (rc != WL_OK) return rc;
  cudaStream_t s = (cudaStream_t)stream;
  const int nparts = (int)((nc + kChunk - 1) / kChunk);
  int lo[3] = {0, 0, 0}, hi[3] = {0, 1, 1};
  if (b.kind != 0) {
    double ext = b.r1 + b.eps + 1.0;
    if (b.kind == 2) ext = b.r1 + b.r2 + b.eps + 1.0;
    for (int d = 0; d < ndim; ++d) {
      lo[d] = (int)fmax(0.0, floor(b.c[d] - ext));
      hi[d] = (int)fmin((double)g.n[d], ceil(b.c[d] + ext) + 1.0);
      if (hi[d] < lo[d]) hi[d] = lo[d];
    }
  }
  const int bx = hi[0] - lo[0], by = hi[1] - lo[1], bz = hi[2] - lo[2];
  if (ndim == 3) {
    k_noalloc_partials<3><<<nparts, 256, 0, s>>>(g, p, L, scratch);
    k_noalloc_final<3><<<1, 256, 0, s>>>(g, b, p, scratch, nparts, lo[0], lo[1], lo[2], bx, by, bz, F);
  } else {
    k_noalloc_partials<2><<<nparts, 256, 0, s>>>(g, p, L, scratch);
    k_noalloc_final<2><<<1, 256, 0, s>>>(g, b, p, scratch, nparts, lo[0], lo[1], lo[2], bx, by, bz, F);
  }
  return cudaGetLastError() == cudaSuccess ? WL_OK : WL_ECUDA;
}
