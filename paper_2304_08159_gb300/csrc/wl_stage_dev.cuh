// Point-wise evaluation of one Heun stage's pieces (convdiff! residual and the
// BDIM field f = u0 + dt r(u), Section 2) straight from global memory with the BC
// mapping, for the few faces of the body band (BDIM's mu1 term and its adjoint).
#pragma once
#include "wl_dev.cuh"
#include "wl_kernels.h"

namespace wl {

// convdiff residual r_c at face (i,j,k) (which must be an updated face), read
// straight from global memory with the BC mapping; used for the few band faces.
template <int D>
__device__ float conv_residual(const float* const* u, int c, const Grid& g, int i, int j, int k, float nu,
                               bool adv) {
  auto U = [&](int comp, int ii, int jj, int kk) { return load_u_bc<D>(u[comp], comp, g, ii, jj, kk); };
  float r = 0.f;
#pragma unroll
  for (int d = 0; d < D; ++d) {
#pragma unroll
    for (int side = 0; side < 2; ++side) {
      int J[3] = {i, j, k};
      J[d] += side;
      int e[3] = {0, 0, 0};
      e[d] = 1;
      int ec[3] = {0, 0, 0};
      ec[c] = 1;
      const float a2 = U(d, J[0], J[1], J[2]) + U(d, J[0] - ec[0], J[1] - ec[1], J[2] - ec[2]);
      const float F = mom_flux(U(c, J[0] - 2 * e[0], J[1] - 2 * e[1], J[2] - 2 * e[2]),
                               U(c, J[0] - e[0], J[1] - e[1], J[2] - e[2]), U(c, J[0], J[1], J[2]),
                               U(c, J[0] + e[0], J[1] + e[1], J[2] + e[2]), a2, nu, adv);
      r += side ? -F : F;
    }
  }
  return r;
}

// f_c = u0 + dt r(u) at a face that may lie outside the interior: the same BC as the
// velocity gives its value there (Dirichlet faces carry U_c; others map inward).
template <int D>
__device__ float f_at(const StageArgs& a, int c, int i, int j, int k, float dt) {
  const Grid& g = a.g;
  if (c == 0 && g.exit && i >= g.n[0]) {
    // convective exit: f_e = e0 - dt U (e_in - u_in[n_0 - 1]) at the row (the exit update
    // before its flux correction)
    const float e0 = load_u_bc<D>(a.u0[0], 0, g, g.n[0], j, k);
    const float ei = load_u_bc<D>(a.u[0], 0, g, g.n[0], j, k);
    const float ul = load_u_bc<D>(a.u[0], 0, g, g.n[0] - 1, j, k);
    return fmaf(-dt * g.U[0], ei - ul, e0);
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
  const float r = conv_residual<D>(a.u, c, g, I[0], I[1], I[2], a.nu, a.advect != 0);
  return fmaf(dt, r, __ldg(a.u0[c] + cell_index(g, I[0], I[1], I[2])));
}

}  // namespace wl
