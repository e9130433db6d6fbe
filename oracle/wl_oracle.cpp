// FP64 CPU oracle of the WaterLily time step (convection-diffusion, BDIM blend,
// pressure projection, CFL, pressure force).
//
// TEST INFRASTRUCTURE ONLY.  Only tests/, __graft_entry__.smoke() and the
// cpu_baseline / reference legs of bench.py may load this library.  The GPU
// library shares no code, header or constant with it.
//
// Everything here is plain loops in double precision, written to be checked by
// eye against the method, not to be fast.  Grid units throughout: cell width 1,
// cell I (0-based, I_d in [0,n_d)) has its centre at I + 1/2, and u_c[I] is the
// velocity component c on the lower c-face of cell I (the staggered indexing of
// the pressure-gradient loop in Section 2: u[I,i] -= coeff[I,i]*(p[I]-p[I-del(i)])).
//
// Sources (the paper states the method only by name, Section 2):
//   * incompressible Navier-Stokes on a uniform staggered Cartesian grid, a
//     third-order finite-volume convection scheme with implicit LES (Section 2);
//     reading: kappa=1/3 upwind-biased face value limited by Koren's (1993) TVD
//     limiter; viscous flux by central difference;
//   * explicit adaptive time stepping (Section 2); reading: Heun predictor-corrector
//     with a projection after each stage, dt from the convective out-flux CFL rule;
//   * Boundary Data Immersion Method (Section 2, Weymouth & Yue 2011): u = mu0*f +
//     mu1 . grad f with the zeroth/first moments of the cosine kernel of half-width eps;
//   * BDIM-modified Poisson matrix (Section 2, Lauber 2022): face coefficients = mu0;
//   * geometric multigrid Poisson solver (Section 2, Weymouth 2022) - the oracle's
//     reference projection uses Jacobi-preconditioned CG to a tight tolerance; the
//     V-cycle below exists to check the GPU V-cycle one cycle at a time;
//   * the step's routines convdiff!, BDIM!, BC!, project!, CFL! (Table 2).
//
// Parity pins for every function are in tests/test_oracle_*.py.

#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <vector>
#include <algorithm>

namespace {

typedef std::vector<double> vec;

struct Level {
  int n[3];
  long ncell;
  vec L[3];  // L[c][cell]: coefficient of the lower c-face of each cell
};

struct OSim {
  int D;
  int n[3];           // interior cells per direction (n[2] = 1 in 2-D)
  int g[3];           // ghost width per direction (2, or 0 for the unused z of 2-D)
  int np[3];          // padded extents
  long ncell, npad;
  unsigned periodic;  // bit d set: direction d is periodic
  double nu;
  double U[3];
  int body_kind;      // 0 none, 1 circle/sphere, 2 torus, 3 sampled distance (nodes)
  vec nodes;          // body_kind 3: signed distance at the grid's nodes (positions (i, j, k),
                      // (n0+1)(n1+1)(n2+1) values in 3-D, (n0+1)(n1+1) in 2-D, x fastest)
  double center[3], radius, radius2, eps;
  int advect;         // 1: full convection-diffusion; 0: diffusion only (Stokes checks)
  int exit_bc = 0;    // 1: convective exit on the upper x face (see exit_stage)
  double dt, dt_cap, t;
  long nsteps;
  vec u[3];           // padded velocity, BC applied
  vec p;              // pressure, cells
  vec mu0[3];         // cells (lower faces)
  vec mu1[3][3];      // mu1[c][j][cell]: component j of mu1*n at the lower c-face
  std::vector<Level> lev;  // lev[0].L = Poisson face coefficients of the fine grid
  int last_iters;
  double last_resid;
};

inline bool is_per(const OSim& s, int d) { return (s.periodic >> d) & 1u; }

inline long cidx(const OSim& s, int i, int j, int k) {
  return i + (long)s.n[0] * (j + (long)s.n[1] * k);
}
inline long pidx(const OSim& s, int i, int j, int k) {
  return (i + s.g[0]) + (long)s.np[0] * ((j + s.g[1]) + (long)s.np[1] * (k + s.g[2]));
}
inline long pidx(const OSim& s, const int* I) { return pidx(s, I[0], I[1], I[2]); }

// ---------------------------------------------------------------------------
// Kernel moments of the cosine kernel K(s) = (1 + cos(pi s))/2 on [-1, 1]
// (BDIM, Section 2): K0(s) = int_{-1}^{s} K, K1(s) = int_{s}^{1} t K(t) dt.
// Outside the kernel's support the integrals are exactly 0 or 1; K0 is the integral
// of a non-negative kernel of unit mass, so it is kept in [0, 1] where rounding of the
// closed form near s = -1 (a cancellation) could step outside.
double K0(double s) {
  if (s <= -1.0) return 0.0;
  if (s >= 1.0) return 1.0;
  double v = 0.5 + 0.5 * s + std::sin(M_PI * s) / (2.0 * M_PI);
  return std::max(0.0, std::min(1.0, v));
}
double K1(double s) {
  if (s <= -1.0 || s >= 1.0) return 0.0;
  return 0.25 * (1.0 - s * s) - (s * std::sin(M_PI * s) + (1.0 + std::cos(M_PI * s)) / M_PI) / (2.0 * M_PI);
}

// Signed distance and outward unit normal of the body at point x (D coordinates).
double sdf(const OSim& s, const double* x, double* nrm) {
  for (int d = 0; d < 3; ++d) nrm[d] = 0.0;
  if (s.body_kind == 1) {  // circle (2-D) / sphere (3-D)
    double r2 = 0.0;
    for (int d = 0; d < s.D; ++d) r2 += (x[d] - s.center[d]) * (x[d] - s.center[d]);
    double r = std::sqrt(r2);
    if (r > 0.0)
      for (int d = 0; d < s.D; ++d) nrm[d] = (x[d] - s.center[d]) / r;
    return r - s.radius;
  }
  if (s.body_kind == 2 && s.D == 3) {  // torus: ring radius `radius` in the y-z plane, tube radius `radius2`
    double a = x[0] - s.center[0], b = x[1] - s.center[1], c = x[2] - s.center[2];
    double rho = std::sqrt(b * b + c * c);
    double q0 = a, q1 = rho - s.radius;
    double dq = std::sqrt(q0 * q0 + q1 * q1);
    if (dq > 0.0) {
      double e1 = (rho > 0.0) ? b / rho : 0.0, e2 = (rho > 0.0) ? c / rho : 0.0;
      nrm[0] = q0 / dq;
      nrm[1] = q1 / dq * e1;
      nrm[2] = q1 / dq * e2;
    }
    return dq - s.radius2;
  }
  if (s.body_kind == 3) {  // sampled: multilinear between the nodes of the cell holding x
    const int D = s.D;
    int c0[3] = {0, 0, 0};
    double f[3] = {0.0, 0.0, 0.0};
    for (int d = 0; d < D; ++d) {
      c0[d] = std::max(0, std::min(s.n[d] - 1, (int)std::floor(x[d])));
      f[d] = x[d] - c0[d];
    }
    const long s0 = 1, s1 = s.n[0] + 1, s2 = (long)(s.n[0] + 1) * (s.n[1] + 1);
    const long base = c0[0] * s0 + c0[1] * s1 + (D == 3 ? c0[2] * s2 : 0);
    // corner values v[a][b][c] at node offsets (a, b, c)
    double v[2][2][2];
    for (int a = 0; a < 2; ++a)
      for (int b = 0; b < 2; ++b)
        for (int c = 0; c < 2; ++c) v[a][b][c] = s.nodes[base + a * s0 + b * s1 + (D == 3 ? c * s2 : 0)];
    const double w0[2] = {1.0 - f[0], f[0]}, w1[2] = {1.0 - f[1], f[1]};
    const double w2[2] = {D == 3 ? 1.0 - f[2] : 1.0, D == 3 ? f[2] : 0.0};
    double d = 0.0, g[3] = {0.0, 0.0, 0.0};
    for (int a = 0; a < 2; ++a)
      for (int b = 0; b < 2; ++b)
        for (int c = 0; c < (D == 3 ? 2 : 1); ++c) {
          d += w0[a] * w1[b] * w2[c] * v[a][b][c];
          g[0] += (a ? 1.0 : -1.0) * w1[b] * w2[c] * v[a][b][c];
          g[1] += (b ? 1.0 : -1.0) * w0[a] * w2[c] * v[a][b][c];
          if (D == 3) g[2] += (c ? 1.0 : -1.0) * w0[a] * w1[b] * v[a][b][c];
        }
    const double gn = std::sqrt(g[0] * g[0] + g[1] * g[1] + g[2] * g[2]);
    if (gn > 0.0)
      for (int dd = 0; dd < D; ++dd) nrm[dd] = g[dd] / gn;
    return d;
  }
  return 1e30;  // no body: everything is fluid
}

// ---------------------------------------------------------------------------
// BC! (Table 2).  Applied direction by direction, each over the full padded range
// of the other directions.  Non-periodic direction d: the normal component u_d
// takes the boundary value U_d on both boundary faces (index 0 and n_d) and on the
// ghost faces outside them; the other components copy the nearest interior value
// (zero gradient).  Periodic direction d: every component wraps.
void apply_bc(const OSim& s, vec* f) {
  for (int d = 0; d < s.D; ++d) {
    const int lo[3] = {-s.g[0], -s.g[1], -s.g[2]};
    const int hi[3] = {s.n[0] + s.g[0], s.n[1] + s.g[1], s.n[2] + s.g[2]};
    for (int c = 0; c < s.D; ++c) {
      vec& a = f[c];
#pragma omp parallel for collapse(2)
      for (int k = lo[2]; k < hi[2]; ++k)
        for (int j = lo[1]; j < hi[1]; ++j)
          for (int i = lo[0]; i < hi[0]; ++i) {
            int I[3] = {i, j, k};
            int q = I[d];
            bool ghost = (q < 0 || q >= s.n[d]);
            bool bface = (!is_per(s, d) && c == d && q == 0);
            if (!ghost && !bface) continue;
            int J[3] = {I[0], I[1], I[2]};
            if (is_per(s, d)) {
              J[d] = ((q % s.n[d]) + s.n[d]) % s.n[d];
              a[pidx(s, I)] = a[pidx(s, J)];
            } else if (c == d && d == 0 && s.exit_bc && q >= s.n[0]) {
              // convective exit: the exit face (q = n_0) keeps the value exit_stage gave it,
              // the faces beyond copy it (zero gradient)
              if (q > s.n[0]) {
                J[0] = s.n[0];
                a[pidx(s, I)] = a[pidx(s, J)];
              }
            } else if (c == d) {
              a[pidx(s, I)] = s.U[c];
            } else {
              J[d] = std::max(0, std::min(s.n[d] - 1, q));
              a[pidx(s, I)] = a[pidx(s, J)];
            }
          }
    }
  }
}

// A face (c, I) is updated by the momentum step unless it is a boundary face of a
// non-periodic direction (I_c = 0 there; the face n_c is outside the stored range).
inline bool updated(const OSim& s, int c, const int* I) {
  return is_per(s, c) || I[c] >= 1;
}

// kappa = 1/3 upwind-biased face value with Koren's limiter: phi = c + psi(r)(d - c)/2,
// r = (c - u)/(d - c), psi(r) = max(0, min(2r, (2 + r)/3, 2)); phi = c when d == c.
double face_value(double uu, double cc, double dd) {
  if (dd == cc) return cc;
  double r = (cc - uu) / (dd - cc);
  double psi = std::max(0.0, std::min(std::min(2.0 * r, (2.0 + r) / 3.0), 2.0));
  return cc + 0.5 * psi * (dd - cc);
}

// Momentum flux of component c through the lower j-face of the u_c control volume
// at face index I (I may be one past the interior in direction j).
double flux(const OSim& s, const vec* u, int c, int j, const int* I) {
  auto at = [&](int comp, int dj, int dc) {
    int J[3] = {I[0], I[1], I[2]};
    J[j] += dj;
    J[c] += dc;
    return u[comp][pidx(s, J)];
  };
  double diff = -s.nu * (at(c, 0, 0) - at(c, -1, 0));
  if (!s.advect) return diff;
  // advecting velocity at the face: mean of u_j at I and at I - e_c
  double a = 0.5 * (at(j, 0, 0) + at(j, 0, -1));
  double phi;
  if (a > 0.0)
    phi = face_value(at(c, -2, 0), at(c, -1, 0), at(c, 0, 0));
  else
    phi = face_value(at(c, 1, 0), at(c, 0, 0), at(c, -1, 0));
  return a * phi + diff;
}

// convdiff! (Table 2): r_c[I] = sum_j F_cj[I] - F_cj[I + e_j] on updated faces, 0 elsewhere.
void convdiff(const OSim& s, const vec* u, vec* r) {
  for (int c = 0; c < s.D; ++c) {
    r[c].assign(s.ncell, 0.0);
#pragma omp parallel for collapse(2)
    for (int k = 0; k < s.n[2]; ++k)
      for (int j = 0; j < s.n[1]; ++j)
        for (int i = 0; i < s.n[0]; ++i) {
          int I[3] = {i, j, k};
          if (!updated(s, c, I)) continue;
          double sum = 0.0;
          for (int d = 0; d < s.D; ++d) {
            int Ip[3] = {i, j, k};
            Ip[d] += 1;
            sum += flux(s, u, c, d, I) - flux(s, u, c, d, Ip);
          }
          r[c][cidx(s, i, j, k)] = sum;
        }
  }
}

// Convective exit (reading: the paper's BC! names the boundary conditions only).  On the
// upper x face the normal velocity e is carried out of the domain at the free-stream
// speed U = U_x: de/dt = -U (e - u_x[n_0 - 1]) (first-order upwind difference across
// the last cell), integrated by the same Heun stages as the interior: f_e = e0 - dt U
// (e_in - u_in[n_0 - 1]) from the stage's input velocity, out_e = f_e (stage 1) or
// (e' + f_e)/2 (stage 2).  Then the exit plane is shifted uniformly so that it carries
// out exactly the flux that enters (the mean of out_e equals U: the net flux through the
// other boundaries is zero), which the projection's Neumann problem needs.  The
// tangential components keep zero gradient.
void exit_f(const OSim& s, double dt, const vec* u0, const vec* uin, vec* f) {
  const int n0 = s.n[0];
  for (int k = 0; k < s.n[2]; ++k)
    for (int j = 0; j < s.n[1]; ++j) {
      const long qe = pidx(s, n0, j, k), ql = pidx(s, n0 - 1, j, k);
      f[0][qe] = u0[0][qe] - dt * s.U[0] * (uin[0][qe] - uin[0][ql]);
    }
}
// The state's exit plane into the x component of a padded velocity (interior arrays given
// through the C interface carry no exit face).
void copy_exit(const OSim& s, vec* u) {
  if (!s.exit_bc) return;
  for (int k = 0; k < s.n[2]; ++k)
    for (int j = 0; j < s.n[1]; ++j) u[0][pidx(s, s.n[0], j, k)] = s.u[0][pidx(s, s.n[0], j, k)];
}
void exit_out(const OSim& s, int stage, const vec* u1, const vec* f, vec* out) {
  const int n0 = s.n[0];
  double sum = 0.0;
  for (int k = 0; k < s.n[2]; ++k)
    for (int j = 0; j < s.n[1]; ++j) {
      const long qe = pidx(s, n0, j, k);
      const double v = (stage == 1) ? f[0][qe] : 0.5 * (u1[0][qe] + f[0][qe]);
      out[0][qe] = v;
      sum += v;
    }
  const double shift = s.U[0] - sum / ((double)s.n[1] * s.n[2]);
  for (int k = 0; k < s.n[2]; ++k)
    for (int j = 0; j < s.n[1]; ++j) out[0][pidx(s, n0, j, k)] += shift;
}

// BDIM! (Table 2, Weymouth & Yue 2011) for one Heun stage.
//   stage 1: f = u0 + dt r(u0);  out = mu0 f + sum_j mu1_j (f[I+e_j] - f[I-e_j])/2
//   stage 2: f = u0 + dt r(u1);  out = (u1 + mu0 f + mu1 . grad f) / 2
// f's boundary and ghost faces are filled with the same BC as u.  The body velocity
// is zero.  `uin` is u0 in stage 1 and u1 in stage 2; `out` is padded, BC applied.
void bdim_stage(const OSim& s, int stage, double dt, const vec* u0, const vec* u1, vec* out) {
  const vec* uin = (stage == 1) ? u0 : u1;
  vec r[3];
  convdiff(s, uin, r);
  vec f[3];
  for (int c = 0; c < s.D; ++c) {
    f[c] = u0[c];
#pragma omp parallel for collapse(2)
    for (int k = 0; k < s.n[2]; ++k)
      for (int j = 0; j < s.n[1]; ++j)
        for (int i = 0; i < s.n[0]; ++i) {
          int I[3] = {i, j, k};
          if (!updated(s, c, I)) continue;
          f[c][pidx(s, I)] = u0[c][pidx(s, I)] + dt * r[c][cidx(s, i, j, k)];
        }
  }
  if (s.exit_bc) exit_f(s, dt, u0, uin, f);
  apply_bc(s, f);
  for (int c = 0; c < s.D; ++c) {
    out[c] = uin[c];
#pragma omp parallel for collapse(2)
    for (int k = 0; k < s.n[2]; ++k)
      for (int j = 0; j < s.n[1]; ++j)
        for (int i = 0; i < s.n[0]; ++i) {
          int I[3] = {i, j, k};
          if (!updated(s, c, I)) continue;
          long ci = cidx(s, i, j, k);
          double v = s.mu0[c][ci] * f[c][pidx(s, I)];
          for (int d = 0; d < s.D; ++d) {
            int Ip[3] = {i, j, k}, Im[3] = {i, j, k};
            Ip[d] += 1;
            Im[d] -= 1;
            v += s.mu1[c][d][ci] * 0.5 * (f[c][pidx(s, Ip)] - f[c][pidx(s, Im)]);
          }
          out[c][pidx(s, I)] = (stage == 1) ? v : 0.5 * (u1[c][pidx(s, I)] + v);
        }
  }
  if (s.exit_bc) exit_out(s, stage, u1, f, out);
  apply_bc(s, out);
}

// ---------------------------------------------------------------------------
// Poisson operator with BDIM face coefficients (Section 2, Lauber 2022):
//   (A x)[I] = sum_c L_c[I+e_c] (x[I+e_c] - x[I]) + L_c[I] (x[I-e_c] - x[I]).
// Face n_c of a periodic direction is face 0; of a non-periodic direction it has L = 0.
struct Op {
  int D;
  int n[3];
  unsigned periodic;
  const vec* L;
  long ncell;
  long idx(int i, int j, int k) const { return i + (long)n[0] * (j + (long)n[1] * k); }
  // neighbour of cell I in direction c (dir = +1/-1), -1 when outside a non-periodic side
  long nb(const int* I, int c, int dir) const {
    int J[3] = {I[0], I[1], I[2]};
    J[c] += dir;
    if (J[c] < 0 || J[c] >= n[c]) {
      if (!((periodic >> c) & 1u)) return -1;
      J[c] = (J[c] + n[c]) % n[c];
    }
    return idx(J[0], J[1], J[2]);
  }
  double Lupper(const int* I, int c) const {  // coefficient of the upper c-face of cell I
    long q = nb(I, c, +1);
    return q < 0 ? 0.0 : L[c][q];
  }
  double Llower(const int* I, int c) const { return L[c][idx(I[0], I[1], I[2])]; }
  double diag(const int* I) const {
    double s = 0.0;
    for (int c = 0; c < D; ++c) s += Lupper(I, c) + Llower(I, c);
    return s;
  }
  void apply(const vec& x, vec& y) const {
    y.assign(ncell, 0.0);
#pragma omp parallel for collapse(2)
    for (int k = 0; k < n[2]; ++k)
      for (int j = 0; j < n[1]; ++j)
        for (int i = 0; i < n[0]; ++i) {
          int I[3] = {i, j, k};
          long q = idx(i, j, k);
          double s = 0.0;
          for (int c = 0; c < D; ++c) {
            long qp = nb(I, c, +1), qm = nb(I, c, -1);
            if (qp >= 0) s += Lupper(I, c) * (x[qp] - x[q]);
            if (qm >= 0) s += Llower(I, c) * (x[qm] - x[q]);
          }
          y[q] = s;
        }
  }
  void diagonal(vec& dg) const {
    dg.assign(ncell, 0.0);
#pragma omp parallel for collapse(2)
    for (int k = 0; k < n[2]; ++k)
      for (int j = 0; j < n[1]; ++j)
        for (int i = 0; i < n[0]; ++i) {
          int I[3] = {i, j, k};
          dg[idx(i, j, k)] = diag(I);
        }
  }
};

Op make_op(const OSim& s, const Level& l) {
  Op o;
  o.D = s.D;
  for (int d = 0; d < 3; ++d) o.n[d] = l.n[d];
  o.periodic = s.periodic;
  o.L = l.L;
  o.ncell = l.ncell;
  return o;
}

double norm_inf(const vec& a) {
  double m = 0.0;
  const long n = (long)a.size();
#pragma omp parallel for reduction(max : m)
  for (long q = 0; q < n; ++q) m = std::max(m, std::fabs(a[q]));
  return m;
}

// Remove the mean over active cells (diagonal > 0); inactive cells are set to 0.
void remove_mean_active(vec& a, const vec& dg) {
  double sum = 0.0;
  long cnt = 0;
  const long n = (long)a.size();
#pragma omp parallel for reduction(+ : sum, cnt)
  for (long q = 0; q < n; ++q)
    if (dg[q] > 0.0) {
      sum += a[q];
      ++cnt;
    }
  double m = cnt ? sum / cnt : 0.0;
#pragma omp parallel for
  for (long q = 0; q < n; ++q) a[q] = (dg[q] > 0.0) ? a[q] - m : 0.0;
}

// Jacobi-preconditioned conjugate gradients on -A x = -z over the active cells,
// started from x, stopped when ||z - A x||_inf <= tol.  z is first projected onto
// the range of A (its mean over active cells removed).  Returns iterations used.
int pcg(const Op& A, vec& x, const vec& zin, double tol, int maxit, double* resid) {
  vec dg;
  A.diagonal(dg);
  vec z = zin;
  remove_mean_active(z, dg);
  const long n = A.ncell;
  for (long q = 0; q < n; ++q)
    if (dg[q] <= 0.0) x[q] = 0.0;
  vec Ax, r(n), zz(n), pp(n), Ap;
  A.apply(x, Ax);
#pragma omp parallel for
  for (long q = 0; q < n; ++q) r[q] = (dg[q] > 0.0) ? (z[q] - Ax[q]) : 0.0;  // r = z - Ax
  double rn = norm_inf(r);
  int it = 0;
  if (rn <= tol) {
    if (resid) *resid = rn;
    return 0;
  }
  // work with B = -A (positive semi-definite), b = -z, residual rho = b - Bx = -(z - Ax) = -r
  double rz = 0.0;
#pragma omp parallel for reduction(+ : rz)
  for (long q = 0; q < n; ++q) {
    zz[q] = (dg[q] > 0.0) ? -r[q] / dg[q] : 0.0;
    pp[q] = zz[q];
    rz += -r[q] * zz[q];
  }
  for (it = 1; it <= maxit; ++it) {
    A.apply(pp, Ap);  // A p ; B p = -A p
    double pBp = 0.0;
#pragma omp parallel for reduction(+ : pBp)
    for (long q = 0; q < n; ++q) pBp += pp[q] * (-Ap[q]);
    if (pBp <= 0.0) break;
    double alpha = rz / pBp;
#pragma omp parallel for
    for (long q = 0; q < n; ++q) {
      x[q] += alpha * pp[q];
      r[q] -= alpha * Ap[q];  // r = z - A x
    }
    rn = norm_inf(r);
    if (rn <= tol) {
      A.apply(x, Ax);  // confirm with the true residual
#pragma omp parallel for
      for (long q = 0; q < n; ++q) r[q] = (dg[q] > 0.0) ? (z[q] - Ax[q]) : 0.0;
      rn = norm_inf(r);
      if (rn <= tol) break;
    }
    double rz2 = 0.0;
#pragma omp parallel for reduction(+ : rz2)
    for (long q = 0; q < n; ++q) {
      zz[q] = (dg[q] > 0.0) ? -r[q] / dg[q] : 0.0;
      rz2 += -r[q] * zz[q];
    }
    double beta = rz2 / rz;
    rz = rz2;
#pragma omp parallel for
    for (long q = 0; q < n; ++q) pp[q] = zz[q] + beta * pp[q];
  }
  if (resid) *resid = rn;
  return it;
}

// Dense solve of A x = z on the active cells with the constraint sum(x) = 0, by
// Gaussian elimination with partial pivoting on the bordered matrix [A 1; 1^T 0].
// z is first projected onto the range (mean removed).  For small grids only.
int dense_solve(const Op& A, vec& x, const vec& zin) {
  vec dg;
  A.diagonal(dg);
  vec z = zin;
  remove_mean_active(z, dg);
  std::vector<long> act;
  std::vector<long> pos(A.ncell, -1);
  for (long q = 0; q < A.ncell; ++q)
    if (dg[q] > 0.0) {
      pos[q] = (long)act.size();
      act.push_back(q);
    }
  long m = (long)act.size();
  long N = m + 1;
  vec M((size_t)N * N, 0.0), b(N, 0.0);
  vec e(A.ncell, 0.0), col;
  for (long a = 0; a < m; ++a) {  // column a of A restricted to active cells
    e[act[a]] = 1.0;
    A.apply(e, col);
    e[act[a]] = 0.0;
    for (long r = 0; r < m; ++r) M[r * N + a] = col[act[r]];
    M[a * N + m] = 1.0;
    M[m * N + a] = 1.0;
    b[a] = z[act[a]];
  }
  for (long k = 0; k < N; ++k) {  // elimination
    long piv = k;
    for (long r = k + 1; r < N; ++r)
      if (std::fabs(M[r * N + k]) > std::fabs(M[piv * N + k])) piv = r;
    if (M[piv * N + k] == 0.0) return -1;
    if (piv != k) {
      for (long c = 0; c < N; ++c) std::swap(M[k * N + c], M[piv * N + c]);
      std::swap(b[k], b[piv]);
    }
    for (long r = k + 1; r < N; ++r) {
      double f = M[r * N + k] / M[k * N + k];
      if (f == 0.0) continue;
      for (long c = k; c < N; ++c) M[r * N + c] -= f * M[k * N + c];
      b[r] -= f * b[k];
    }
  }
  vec y(N, 0.0);
  for (long k = N - 1; k >= 0; --k) {
    double sum = b[k];
    for (long c = k + 1; c < N; ++c) sum -= M[k * N + c] * y[c];
    y[k] = sum / M[k * N + k];
  }
  x.assign(A.ncell, 0.0);
  for (long a = 0; a < m; ++a) x[act[a]] = y[a];
  return 0;
}

// ---------------------------------------------------------------------------
// Multigrid hierarchy (Section 2, Weymouth 2022).  Reading: halve while every
// direction is even and larger than 4; coarse face coefficient = half the sum of
// the 2^(D-1) fine faces it covers; restriction sums the 2^D children; prolongation
// is piecewise constant; the coarse initial guess is zero; the coarsest level is
// solved exactly (mean zero over active cells); smoothing is red-black Gauss-Seidel
// (red: i+j+k even, updated first).
void build_levels(OSim& s) {
  while (true) {
    Level& f = s.lev.back();
    bool ok = true;
    for (int d = 0; d < s.D; ++d)
      if (f.n[d] % 2 != 0 || f.n[d] <= 4) ok = false;
    if (!ok) break;
    Level c;
    for (int d = 0; d < 3; ++d) c.n[d] = (d < s.D) ? f.n[d] / 2 : 1;
    c.ncell = (long)c.n[0] * c.n[1] * c.n[2];
    for (int cc = 0; cc < s.D; ++cc) {
      c.L[cc].assign(c.ncell, 0.0);
#pragma omp parallel for collapse(2)
      for (int k = 0; k < c.n[2]; ++k)
        for (int j = 0; j < c.n[1]; ++j)
          for (int i = 0; i < c.n[0]; ++i) {
            int J[3] = {i, j, k};
            double sum = 0.0;
            // fine faces: index 2J_cc in direction cc, children 2J_d..2J_d+1 in the others
            int a0 = (cc == 0) ? 1 : 2, a1 = (cc == 1 || s.D < 2) ? 1 : 2, a2 = (cc == 2 || s.D < 3) ? 1 : 2;
            for (int dk = 0; dk < a2; ++dk)
              for (int dj = 0; dj < a1; ++dj)
                for (int di = 0; di < a0; ++di) {
                  int I[3] = {2 * J[0] + di, (s.D > 1 ? 2 * J[1] : 0) + dj, (s.D > 2 ? 2 * J[2] : 0) + dk};
                  sum += f.L[cc][I[0] + (long)f.n[0] * (I[1] + (long)f.n[1] * I[2])];
                }
            c.L[cc][i + (long)c.n[0] * (j + (long)c.n[1] * k)] = 0.5 * sum;
          }
    }
    s.lev.push_back(c);
  }
}

void rb_sweep(const Op& A, vec& x, const vec& z) {
  for (int color = 0; color < 2; ++color)
#pragma omp parallel for collapse(2)
    for (int k = 0; k < A.n[2]; ++k)
      for (int j = 0; j < A.n[1]; ++j)
        for (int i = 0; i < A.n[0]; ++i) {
          if (((i + j + k) & 1) != color) continue;
          int I[3] = {i, j, k};
          double dgn = A.diag(I);
          if (dgn <= 0.0) continue;
          double sum = 0.0;
          for (int c = 0; c < A.D; ++c) {
            long qp = A.nb(I, c, +1), qm = A.nb(I, c, -1);
            if (qp >= 0) sum += A.Lupper(I, c) * x[qp];
            if (qm >= 0) sum += A.Llower(I, c) * x[qm];
          }
          x[A.idx(i, j, k)] = (sum - z[A.idx(i, j, k)]) / dgn;
        }
}

void vcycle(const OSim& s, int l, vec& x, const vec& z, int pre, int post) {
  Op A = make_op(s, s.lev[l]);
  if (l == (int)s.lev.size() - 1) {
    vec dg;
    A.diagonal(dg);
    long nact = 0;
    for (double v : dg) nact += (v > 0.0);
    if (nact <= 2048) {
      dense_solve(A, x, z);
    } else {
      x.assign(A.ncell, 0.0);
      double zn = norm_inf(z);
      pcg(A, x, z, 1e-14 * std::max(zn, 1e-300), 100000, nullptr);
      remove_mean_active(x, dg);
    }
    return;
  }
  for (int it = 0; it < pre; ++it) rb_sweep(A, x, z);
  vec Ax;
  A.apply(x, Ax);
  const Level& c = s.lev[l + 1];
  vec zc(c.ncell, 0.0), xc(c.ncell, 0.0);
  // restriction: each coarse cell sums the residual of its 2^D children
#pragma omp parallel for collapse(2)
  for (int ck = 0; ck < c.n[2]; ++ck)
    for (int cj = 0; cj < c.n[1]; ++cj)
      for (int ci = 0; ci < c.n[0]; ++ci) {
        double sum = 0.0;
        for (int dk = 0; dk < (s.D > 2 ? 2 : 1); ++dk)
          for (int dj = 0; dj < 2; ++dj)
            for (int di = 0; di < 2; ++di) {
              long q = A.idx(2 * ci + di, 2 * cj + dj, (s.D > 2 ? 2 * ck : 0) + dk);
              sum += z[q] - Ax[q];
            }
        zc[ci + (long)c.n[0] * (cj + (long)c.n[1] * ck)] = sum;
      }
  vcycle(s, l + 1, xc, zc, pre, post);
  // piecewise-constant prolongation of the correction onto the active cells
  // (cells with a zero row have no equation and keep x = 0)
#pragma omp parallel for collapse(2)
  for (int k = 0; k < A.n[2]; ++k)
    for (int j = 0; j < A.n[1]; ++j)
      for (int i = 0; i < A.n[0]; ++i) {
        int I[3] = {i, j, k};
        if (A.diag(I) <= 0.0) continue;
        int ci = i / 2, cj = (s.D > 1) ? j / 2 : 0, ck = (s.D > 2) ? k / 2 : 0;
        x[A.idx(i, j, k)] += xc[ci + (long)c.n[0] * (cj + (long)c.n[1] * ck)];
      }
  for (int it = 0; it < post; ++it) rb_sweep(A, x, z);
}

// ---------------------------------------------------------------------------
// Geometry (measure, Section 2): mu0 = K0(d/eps), mu1 = eps K1(d/eps) n at every
// face; Poisson coefficient L = mu0 except L = 0 on non-periodic boundary faces.
void measure(OSim& s) {
  for (int c = 0; c < s.D; ++c) {
    s.mu0[c].assign(s.ncell, 1.0);
    for (int d = 0; d < 3; ++d) s.mu1[c][d].assign(s.ncell, 0.0);
  }
  if (s.body_kind != 0) {
    for (int c = 0; c < s.D; ++c)
#pragma omp parallel for collapse(2)
      for (int k = 0; k < s.n[2]; ++k)
        for (int j = 0; j < s.n[1]; ++j)
          for (int i = 0; i < s.n[0]; ++i) {
            double x[3] = {i + 0.5, j + 0.5, k + 0.5};
            x[c] -= 0.5;  // lower c-face
            double nrm[3];
            double d = sdf(s, x, nrm);
            long q = cidx(s, i, j, k);
            s.mu0[c][q] = K0(d / s.eps);
            for (int jj = 0; jj < s.D; ++jj) s.mu1[c][jj][q] = s.eps * K1(d / s.eps) * nrm[jj];
          }
  }
  Level l0;
  for (int d = 0; d < 3; ++d) l0.n[d] = s.n[d];
  l0.ncell = s.ncell;
  for (int c = 0; c < s.D; ++c) l0.L[c] = s.mu0[c];
  // zero the non-periodic boundary faces
  for (int c = 0; c < s.D; ++c) {
    if (is_per(s, c)) continue;
    for (int k = 0; k < s.n[2]; ++k)
      for (int j = 0; j < s.n[1]; ++j)
        for (int i = 0; i < s.n[0]; ++i) {
          int I[3] = {i, j, k};
          if (I[c] == 0) l0.L[c][cidx(s, i, j, k)] = 0.0;
        }
  }
  s.lev.clear();
  s.lev.push_back(l0);
  build_levels(s);
}

// Divergence z[I] = sum_c u_c[I+e_c] - u_c[I] (u padded with BC applied).
void divergence(const OSim& s, const vec* u, vec& z) {
  z.assign(s.ncell, 0.0);
#pragma omp parallel for collapse(2)
  for (int k = 0; k < s.n[2]; ++k)
    for (int j = 0; j < s.n[1]; ++j)
      for (int i = 0; i < s.n[0]; ++i) {
        double sum = 0.0;
        for (int c = 0; c < s.D; ++c) {
          int I[3] = {i, j, k}, Ip[3] = {i, j, k};
          Ip[c] += 1;
          sum += u[c][pidx(s, Ip)] - u[c][pidx(s, I)];
        }
        z[cidx(s, i, j, k)] = sum;
      }
}

// project! (Table 2) with weight w: x0 = p w dt; solve A x = div u; subtract the
// mean of x over active cells; u_c[I] -= L_c[I] (x[I] - x[I-e_c]) (Section 2 listing);
// BC; p = x / (w dt).
// solver 0: Jacobi-PCG (the reference projection); solver 1: V(0,post) cycles of the
// multigrid hierarchy until ||z - A x||_inf <= tol or maxit cycles.
void project(OSim& s, vec* u, double w, double dt, double tol, int maxit, int solver = 0, int post = 4) {
  Op A = make_op(s, s.lev[0]);
  vec z, dg;
  divergence(s, u, z);
  A.diagonal(dg);
  vec x(s.ncell);
  for (long q = 0; q < s.ncell; ++q) x[q] = s.p[q] * w * dt;
  double res = 0.0;
  if (solver == 0) {
    s.last_iters = pcg(A, x, z, tol, maxit, &res);
  } else {
    int it = 0;
    vec Ax;
    while (true) {
      A.apply(x, Ax);
      res = 0.0;
#pragma omp parallel for reduction(max : res)
      for (long q = 0; q < s.ncell; ++q) res = std::max(res, std::fabs(z[q] - Ax[q]));
      if (res <= tol || it >= maxit) break;
      vcycle(s, 0, x, z, 0, post);
      ++it;
    }
    s.last_iters = it;
  }
  s.last_resid = res;
  remove_mean_active(x, dg);
  for (int c = 0; c < s.D; ++c)
#pragma omp parallel for collapse(2)
    for (int k = 0; k < s.n[2]; ++k)
      for (int j = 0; j < s.n[1]; ++j)
        for (int i = 0; i < s.n[0]; ++i) {
          int I[3] = {i, j, k};
          long qm = A.nb(I, c, -1);
          long q = cidx(s, i, j, k);
          double L = A.Llower(I, c);
          if (qm >= 0 && L != 0.0) u[c][pidx(s, I)] -= L * (x[q] - x[qm]);
        }
  apply_bc(s, u);
  for (long q = 0; q < s.ncell; ++q) s.p[q] = x[q] / (w * dt);
}

// CFL! (Table 2): dt = min(dt_cap, 1/(max_I sum_c [max(0,u_c[I+e_c]) + max(0,-u_c[I])] + 2 D nu)).
double cfl(const OSim& s) {
  double m = 0.0;
#pragma omp parallel for collapse(2) reduction(max : m)
  for (int k = 0; k < s.n[2]; ++k)
    for (int j = 0; j < s.n[1]; ++j)
      for (int i = 0; i < s.n[0]; ++i) {
        double sum = 0.0;
        for (int c = 0; c < s.D; ++c) {
          int I[3] = {i, j, k}, Ip[3] = {i, j, k};
          Ip[c] += 1;
          sum += std::max(0.0, s.u[c][pidx(s, Ip)]) + std::max(0.0, -s.u[c][pidx(s, I)]);
        }
        m = std::max(m, sum);
      }
  return std::min(s.dt_cap, 1.0 / (m + 2.0 * s.D * s.nu));
}

// ===========================================================================
// Reverse-mode derivative (adjoint) of the time step at a fixed dt with respect to the
// body parameters theta (circle/sphere (R, c_0, .., c_{D-1}); torus (R, r, c_0, c_1, c_2):
// the body enters through its signed distance, Section 2) (the differentiable-solver
// use of the method, Section 1).  Every routine is the transpose of the forward routine
// it names, written out from that routine's arithmetic.  Where the forward is not
// differentiable (the limiter's switch points, the upwind switch at a = 0) the
// derivative of the branch the forward takes is used.  A projection is differentiated as
// the exact projection (A x = div u solved exactly); the forward solves it to a tight
// tolerance.  dt is held fixed: the CFL rule is a maximum over the field and is not
// differentiated.

// Derivative of face_value(uu, cc, dd) with respect to (uu, cc, dd).
void face_value_grad(double uu, double cc, double dd, double* g) {
  g[0] = 0.0;  // phi = cc unless the limiter is active
  g[1] = 1.0;
  g[2] = 0.0;
  if (dd == cc) return;
  const double r = (cc - uu) / (dd - cc);
  const double a = 2.0 * r, b = (2.0 + r) / 3.0;
  const double m = std::min(std::min(a, b), 2.0);
  if (m <= 0.0) return;  // psi = 0
  if (m == a) {          // psi = 2r: phi = 2 cc - uu
    g[0] = -1.0;
    g[1] = 2.0;
  } else if (m == b) {   // psi = (2 + r)/3: phi = (5 cc + 2 dd - uu)/6
    g[0] = -1.0 / 6.0;
    g[1] = 5.0 / 6.0;
    g[2] = 2.0 / 6.0;
  } else {               // psi = 2: phi = dd
    g[1] = 0.0;
    g[2] = 1.0;
  }
}

// Transpose of flux(): ubar (padded) += Fbar * dF/du at the faces flux() reads.
void flux_adjoint(const OSim& s, const vec* u, int c, int j, const int* I, double Fbar, vec* ubar) {
  auto pos = [&](int dj, int dc) {
    int J[3] = {I[0], I[1], I[2]};
    J[j] += dj;
    J[c] += dc;
    return pidx(s, J);
  };
  ubar[c][pos(0, 0)] -= s.nu * Fbar;
  ubar[c][pos(-1, 0)] += s.nu * Fbar;
  if (!s.advect) return;
  const double a = 0.5 * (u[j][pos(0, 0)] + u[j][pos(0, -1)]);
  long q[3];
  if (a > 0.0) {
    q[0] = pos(-2, 0);
    q[1] = pos(-1, 0);
    q[2] = pos(0, 0);
  } else {
    q[0] = pos(1, 0);
    q[1] = pos(0, 0);
    q[2] = pos(-1, 0);
  }
  const double phi = face_value(u[c][q[0]], u[c][q[1]], u[c][q[2]]);
  double gr[3];
  face_value_grad(u[c][q[0]], u[c][q[1]], u[c][q[2]], gr);
  ubar[j][pos(0, 0)] += 0.5 * phi * Fbar;
  ubar[j][pos(0, -1)] += 0.5 * phi * Fbar;
  for (int t = 0; t < 3; ++t) ubar[c][q[t]] += a * gr[t] * Fbar;
}

// Transpose of apply_bc(): the cotangent of every ghost or boundary face moves to the
// face it was copied from (periodic wrap, tangential zero gradient) or is dropped (a
// prescribed normal velocity), direction by direction in the reverse order.
void apply_bc_adjoint(const OSim& s, vec* f) {
  for (int d = s.D - 1; d >= 0; --d) {
    const int lo[3] = {-s.g[0], -s.g[1], -s.g[2]};
    const int hi[3] = {s.n[0] + s.g[0], s.n[1] + s.g[1], s.n[2] + s.g[2]};
    for (int c = 0; c < s.D; ++c) {
      vec& a = f[c];
      for (int k = lo[2]; k < hi[2]; ++k)
        for (int j = lo[1]; j < hi[1]; ++j)
          for (int i = lo[0]; i < hi[0]; ++i) {
            int I[3] = {i, j, k};
            int q = I[d];
            bool ghost = (q < 0 || q >= s.n[d]);
            bool bface = (!is_per(s, d) && c == d && q == 0);
            if (!ghost && !bface) continue;
            const long qi = pidx(s, I);
            const double v = a[qi];
            a[qi] = 0.0;
            int J[3] = {I[0], I[1], I[2]};
            if (is_per(s, d)) {
              J[d] = ((q % s.n[d]) + s.n[d]) % s.n[d];
              a[pidx(s, J)] += v;
            } else if (c != d) {
              J[d] = std::max(0, std::min(s.n[d] - 1, q));
              a[pidx(s, J)] += v;
            }
          }
    }
  }
}

// Transpose of convdiff() at u (padded, BC applied): ubar (padded) += (dr/du)^T rbar
// with rbar on interior cells; only interior entries of ubar change.
void convdiff_adjoint(const OSim& s, const vec* u, const vec* rbar, vec* ubar) {
  vec ub[3];
  for (int c = 0; c < s.D; ++c) ub[c].assign(s.npad, 0.0);
  for (int c = 0; c < s.D; ++c)
    for (int k = 0; k < s.n[2]; ++k)
      for (int j = 0; j < s.n[1]; ++j)
        for (int i = 0; i < s.n[0]; ++i) {
          int I[3] = {i, j, k};
          if (!updated(s, c, I)) continue;
          const double rb = rbar[c][cidx(s, i, j, k)];
          if (rb == 0.0) continue;
          for (int d = 0; d < s.D; ++d) {  // r_c[I] = sum_d F_cd[I] - F_cd[I + e_d]
            int Ip[3] = {i, j, k};
            Ip[d] += 1;
            flux_adjoint(s, u, c, d, I, rb, ub);
            flux_adjoint(s, u, c, d, Ip, -rb, ub);
          }
        }
  apply_bc_adjoint(s, ub);
  for (int c = 0; c < s.D; ++c)
    for (long q = 0; q < s.npad; ++q) ubar[c][q] += ub[c][q];
}

// Transpose of bdim_stage() at (u0, u1) (padded, BC applied): given outbar (interior
// cells), accumulate the cotangents of u0 and u1 (padded arrays, interior entries) and
// of the BDIM moments mu0bar[c][cell], mu1bar[c][j][cell].
void bdim_stage_adjoint(const OSim& s, int stage, double dt, const vec* u0, const vec* u1, const vec* outbar,
                        vec* u0bar, vec* u1bar, vec* mu0bar, vec (*mu1bar)[3]) {
  const vec* uin = (stage == 1) ? u0 : u1;
  vec r[3], f[3], fb[3], rb[3];
  convdiff(s, uin, r);  // recompute f as the forward does
  for (int c = 0; c < s.D; ++c) {
    f[c] = u0[c];
    for (int k = 0; k < s.n[2]; ++k)
      for (int j = 0; j < s.n[1]; ++j)
        for (int i = 0; i < s.n[0]; ++i) {
          int I[3] = {i, j, k};
          if (updated(s, c, I)) f[c][pidx(s, I)] = u0[c][pidx(s, I)] + dt * r[c][cidx(s, i, j, k)];
        }
  }
  apply_bc(s, f);
  for (int c = 0; c < s.D; ++c) fb[c].assign(s.npad, 0.0);
  for (int c = 0; c < s.D; ++c)
    for (int k = 0; k < s.n[2]; ++k)
      for (int j = 0; j < s.n[1]; ++j)
        for (int i = 0; i < s.n[0]; ++i) {
          int I[3] = {i, j, k};
          if (!updated(s, c, I)) continue;  // boundary faces carry the BC value
          const long ci = cidx(s, i, j, k), pi = pidx(s, I);
          const double ob = outbar[c][ci];
          const double vb = (stage == 1) ? ob : 0.5 * ob;
          if (stage == 2) u1bar[c][pi] += 0.5 * ob;
          fb[c][pi] += s.mu0[c][ci] * vb;
          mu0bar[c][ci] += vb * f[c][pi];
          for (int d = 0; d < s.D; ++d) {
            int Ip[3] = {i, j, k}, Im[3] = {i, j, k};
            Ip[d] += 1;
            Im[d] -= 1;
            fb[c][pidx(s, Ip)] += 0.5 * s.mu1[c][d][ci] * vb;
            fb[c][pidx(s, Im)] -= 0.5 * s.mu1[c][d][ci] * vb;
            mu1bar[c][d][ci] += vb * 0.5 * (f[c][pidx(s, Ip)] - f[c][pidx(s, Im)]);
          }
        }
  apply_bc_adjoint(s, fb);
  for (int c = 0; c < s.D; ++c) {
    rb[c].assign(s.ncell, 0.0);
    for (int k = 0; k < s.n[2]; ++k)
      for (int j = 0; j < s.n[1]; ++j)
        for (int i = 0; i < s.n[0]; ++i) {
          int I[3] = {i, j, k};
          const long pi = pidx(s, I);
          u0bar[c][pi] += fb[c][pi];  // f = u0 + dt r
          if (updated(s, c, I)) rb[c][cidx(s, i, j, k)] = dt * fb[c][pi];
        }
  }
  convdiff_adjoint(s, uin, rb, (stage == 1) ? u0bar : u1bar);
}

// Transpose of project() at its converged solution x (x units, mean removed over the
// active cells): given the interior cotangent ubar_out of the corrected velocity and a
// cotangent xbar_in of x, set vbar (padded; interior entries) to the cotangent of the
// velocity before the projection and accumulate the cotangent of the Poisson face
// coefficients into Lbar.  With y = A^+ (xbar_in + D(L ubar)):
//   vbar = ubar - G y,   Lbar_c[I] -= (x[I] - x[I-e_c]) (vbar_c[I]).
void project_adjoint(const OSim& s, const vec& x, const vec* ubar_out, const vec& xbar_in, double rtol, vec* vbar,
                     vec* Lbar) {
  Op A = make_op(s, s.lev[0]);
  vec dg;
  A.diagonal(dg);
  vec ub[3];
  for (int c = 0; c < s.D; ++c) {
    ub[c] = ubar_out[c];
    for (int k = 0; k < s.n[2]; ++k)
      for (int j = 0; j < s.n[1]; ++j)
        for (int i = 0; i < s.n[0]; ++i) {
          int I[3] = {i, j, k};
          if (!updated(s, c, I)) ub[c][cidx(s, i, j, k)] = 0.0;  // boundary faces: BC values
        }
  }
  vec xb = xbar_in;
  for (int c = 0; c < s.D; ++c)
    for (int k = 0; k < s.n[2]; ++k)
      for (int j = 0; j < s.n[1]; ++j)
        for (int i = 0; i < s.n[0]; ++i) {
          int I[3] = {i, j, k};
          const long qm = A.nb(I, c, -1), q = cidx(s, i, j, k);
          if (qm < 0) continue;
          const double v = A.Llower(I, c) * ub[c][q];  // u_c[I] -= L (x[I] - x[I-e_c])
          xb[q] -= v;
          xb[qm] += v;
        }
  vec y(s.ncell, 0.0);
  double res = 0.0;
  pcg(A, y, xb, rtol * std::max(norm_inf(xb), 1e-300), 1000000, &res);
  remove_mean_active(y, dg);
  for (int c = 0; c < s.D; ++c) {
    vbar[c].assign(s.npad, 0.0);
    for (int k = 0; k < s.n[2]; ++k)
      for (int j = 0; j < s.n[1]; ++j)
        for (int i = 0; i < s.n[0]; ++i) vbar[c][pidx(s, i, j, k)] = ub[c][cidx(s, i, j, k)];
  }
  for (int k = 0; k < s.n[2]; ++k)  // D^T y: z[I] = sum_c u_c[I + e_c] - u_c[I]
    for (int j = 0; j < s.n[1]; ++j)
      for (int i = 0; i < s.n[0]; ++i) {
        const double yv = y[cidx(s, i, j, k)];
        for (int c = 0; c < s.D; ++c) {
          int I[3] = {i, j, k}, Ip[3] = {i, j, k};
          Ip[c] += 1;
          vbar[c][pidx(s, Ip)] += yv;
          vbar[c][pidx(s, I)] -= yv;
        }
      }
  apply_bc_adjoint(s, vbar);
  for (int c = 0; c < s.D; ++c)
    for (int k = 0; k < s.n[2]; ++k)
      for (int j = 0; j < s.n[1]; ++j)
        for (int i = 0; i < s.n[0]; ++i) {
          int I[3] = {i, j, k};
          const long qm = A.nb(I, c, -1), q = cidx(s, i, j, k);
          if (qm < 0) continue;
          Lbar[c][q] -= (x[q] - x[qm]) * vbar[c][pidx(s, I)];
        }
}

// Number of body parameters theta: circle/sphere (R, c_0, .., c_{D-1}); torus
// (R, r, c_0, c_1, c_2) with R the ring radius in the y-z plane and r the tube radius.
int n_theta(const OSim& s) { return s.body_kind == 2 ? 5 : s.D + 1; }

// Derivatives of the body's signed distance d and its outward normal n = grad d at x with
// respect to theta: dd[t], dn[j][t].  Moving the centre by dc moves the field by dc, so
// dd/dc_k = -n_k and dn_j/dc_k = -H_jk (H the Hessian of d).
//   circle/sphere: d = |x - c| - R, n = (x - c)/rho, rho = |x - c|;
//     dd/dR = -1, dn/dR = 0, H_jk = (delta_jk - n_j n_k)/rho.
//   torus: with (a, b, c) = x - c, rho = sqrt(b^2 + c^2), e = (b, c)/rho, q = rho - R,
//     s = sqrt(a^2 + q^2): d = s - r, n = (a/s, (q/s) e);
//     dd/dR = -q/s, dd/dr = -1, dn_0/dR = a q/s^3, dn_e/dR = -(a^2/s^3) e, dn/dr = 0;
//     H_00 = q^2/s^3, H_0e = -a q e/s^3, H_ee' = e e' a^2/s^3 + (q/s)(delta_ee' - e e')/rho.
void sdf_theta_grad(const OSim& s, const double* x, double* dd, double dn[3][5]) {
  for (int t = 0; t < 5; ++t) {
    dd[t] = 0.0;
    for (int j = 0; j < 3; ++j) dn[j][t] = 0.0;
  }
  double H[3][3] = {{0, 0, 0}, {0, 0, 0}, {0, 0, 0}}, n[3] = {0.0, 0.0, 0.0};
  int c0 = 1;  // index of c_0 in theta
  if (s.body_kind == 2) {
    const double a = x[0] - s.center[0], b = x[1] - s.center[1], c = x[2] - s.center[2];
    const double rho = std::sqrt(b * b + c * c), q = rho - s.radius, sd = std::sqrt(a * a + q * q);
    const double e[3] = {0.0, rho > 0.0 ? b / rho : 0.0, rho > 0.0 ? c / rho : 0.0};
    if (sd > 0.0) {
      const double s3 = sd * sd * sd;
      n[0] = a / sd;
      n[1] = q / sd * e[1];
      n[2] = q / sd * e[2];
      dd[0] = -q / sd;
      dn[0][0] = a * q / s3;
      for (int j = 1; j < 3; ++j) dn[j][0] = -(a * a / s3) * e[j];
      H[0][0] = q * q / s3;
      for (int j = 1; j < 3; ++j) H[0][j] = H[j][0] = -a * q * e[j] / s3;
      for (int j = 1; j < 3; ++j)
        for (int k = 1; k < 3; ++k)
          H[j][k] = e[j] * e[k] * a * a / s3 + (rho > 0.0 ? (q / sd) * ((j == k ? 1.0 : 0.0) - e[j] * e[k]) / rho : 0.0);
    }
    dd[1] = -1.0;
    c0 = 2;
  } else {
    double rho2 = 0.0;
    for (int d = 0; d < s.D; ++d) rho2 += (x[d] - s.center[d]) * (x[d] - s.center[d]);
    const double rho = std::sqrt(rho2);
    for (int d = 0; d < s.D; ++d) n[d] = rho > 0.0 ? (x[d] - s.center[d]) / rho : 0.0;
    dd[0] = -1.0;
    for (int j = 0; j < s.D; ++j)
      for (int k = 0; k < s.D; ++k) H[j][k] = rho > 0.0 ? ((j == k ? 1.0 : 0.0) - n[j] * n[k]) / rho : 0.0;
  }
  for (int k = 0; k < s.D; ++k) {
    dd[c0 + k] = -n[k];
    for (int j = 0; j < s.D; ++j) dn[j][c0 + k] = -H[j][k];
  }
}

// Pressure force of p (forces() of the C interface) and its adjoint: for a cotangent
// Fbar, pbar (cells) and the theta-cotangent of the force weights n K_eps(d), added to tb.
void force_adjoint(const OSim& s, const vec& p, const double* Fbar, double* F, vec& pbar, double* tb) {
  Op A = make_op(s, s.lev[0]);
  vec dg;
  A.diagonal(dg);
  double sum = 0.0;
  long cnt = 0;
  for (long q = 0; q < s.ncell; ++q)
    if (dg[q] > 0.0) {
      sum += p[q];
      ++cnt;
    }
  const double pm = cnt ? sum / cnt : 0.0;
  for (int d = 0; d < 3; ++d) F[d] = 0.0;
  pbar.assign(s.ncell, 0.0);
  double wg = 0.0;  // sum over band cells of Fbar . n K
  for (int k = 0; k < s.n[2]; ++k)
    for (int j = 0; j < s.n[1]; ++j)
      for (int i = 0; i < s.n[0]; ++i) {
        double x[3] = {i + 0.5, j + 0.5, k + 0.5}, nrm[3];
        const double d = sdf(s, x, nrm);
        if (std::fabs(d) >= s.eps) continue;
        const long q = cidx(s, i, j, k);
        const double K = (1.0 + std::cos(M_PI * d / s.eps)) / (2.0 * s.eps);
        const double Kp = -M_PI * std::sin(M_PI * d / s.eps) / (2.0 * s.eps * s.eps);
        const double pp = p[q] - pm;
        double gw = 0.0;
        for (int dd = 0; dd < s.D; ++dd) {
          F[dd] -= pp * nrm[dd] * K;
          gw += Fbar[dd] * nrm[dd] * K;
        }
        pbar[q] -= gw;
        wg += gw;
        double ddt[5], dn[3][5];
        sdf_theta_grad(s, x, ddt, dn);
        for (int t = 0; t < n_theta(s); ++t)
          for (int dd = 0; dd < s.D; ++dd)
            tb[t] -= Fbar[dd] * pp * (dn[dd][t] * K + nrm[dd] * Kp * ddt[t]);
      }
  for (long q = 0; q < s.ncell; ++q)  // the mean pm over active cells
    if (dg[q] > 0.0) pbar[q] += wg / cnt;
}

// theta-cotangent of the BDIM moments and the Poisson coefficients (measure()):
// mu0 = K0(d/eps), L = mu0 except on non-periodic boundary faces (fixed 0),
// mu1_j = eps K1(d/eps) n_j; K0' = K, K1'(s) = -s K(s).
void moments_adjoint(const OSim& s, const vec* mu0bar, const vec* Lbar, const vec (*mu1bar)[3], double* tb) {
  for (int c = 0; c < s.D; ++c)
    for (int k = 0; k < s.n[2]; ++k)
      for (int j = 0; j < s.n[1]; ++j)
        for (int i = 0; i < s.n[0]; ++i) {
          double x[3] = {i + 0.5, j + 0.5, k + 0.5}, nrm[3];
          x[c] -= 0.5;
          const double d = sdf(s, x, nrm), sc = d / s.eps;
          if (std::fabs(sc) >= 1.0) continue;
          int I[3] = {i, j, k};
          const long q = cidx(s, i, j, k);
          const double K = 0.5 * (1.0 + std::cos(M_PI * sc));
          const bool bnd = !is_per(s, c) && I[c] == 0;
          const double g0 = mu0bar[c][q] + (bnd ? 0.0 : Lbar[c][q]);
          double ddt[5], dn[3][5];
          sdf_theta_grad(s, x, ddt, dn);
          const double k1 = s.eps * K1(sc), k1p = -sc * K;
          for (int t = 0; t < n_theta(s); ++t) {
            tb[t] += g0 * K / s.eps * ddt[t];
            for (int jj = 0; jj < s.D; ++jj) tb[t] += mu1bar[c][jj][q] * (k1p * nrm[jj] * ddt[t] + k1 * dn[jj][t]);
          }
        }
}

// nsteps full steps at fixed dt from the current state, then the gradient of
// J = sum_n gF[n] . F_n (F_n the pressure force after step n) with respect to theta.
// F receives nsteps * D forces, tb n_theta values.  The state advances.
void rollout_grad(OSim& s, int nsteps, double dt, double tol, const double* gF, double* F, double* tb) {
  const int D = s.D;
  std::vector<std::vector<vec>> U0(nsteps), UP(nsteps);
  std::vector<vec> X1(nsteps), X2(nsteps), P2(nsteps);
  for (int n = 0; n < nsteps; ++n) {
    vec u0[3], u1[3];
    for (int c = 0; c < D; ++c) u0[c] = s.u[c];
    bdim_stage(s, 1, dt, u0, u0, u1);
    project(s, u1, 1.0, dt, tol, 1000000, 0);
    X1[n] = s.p;
    for (auto& v : X1[n]) v *= dt;
    UP[n].assign(u1, u1 + D);
    bdim_stage(s, 2, dt, u0, u1, s.u);
    project(s, s.u, 0.5, dt, tol, 1000000, 0);
    X2[n] = s.p;
    for (auto& v : X2[n]) v *= 0.5 * dt;
    P2[n] = s.p;
    U0[n].assign(u0, u0 + D);
    s.t += dt;
    s.nsteps += 1;
  }
  s.dt = dt;
  for (int t = 0; t < n_theta(s); ++t) tb[t] = 0.0;
  vec mu0bar[3], Lbar[3], mu1bar[3][3], ub[3];
  for (int c = 0; c < D; ++c) {
    mu0bar[c].assign(s.ncell, 0.0);
    Lbar[c].assign(s.ncell, 0.0);
    for (int j = 0; j < 3; ++j) mu1bar[c][j].assign(s.ncell, 0.0);
    ub[c].assign(s.ncell, 0.0);
  }
  const double rtol = 1e-13;
  for (int n = nsteps - 1; n >= 0; --n) {
    double Fn[3];
    vec pb;
    force_adjoint(s, P2[n], gF + (long)n * D, Fn, pb, tb);
    for (int d = 0; d < D; ++d) F[(long)n * D + d] = Fn[d];
    for (auto& v : pb) v /= 0.5 * dt;  // p = x / (w dt)
    vec v2b[3], v1b[3], u0b[3], upb[3], ubi[3];
    project_adjoint(s, X2[n], ub, pb, rtol, v2b, Lbar);
    for (int c = 0; c < D; ++c) {
      u0b[c].assign(s.npad, 0.0);
      upb[c].assign(s.npad, 0.0);
      ubi[c].assign(s.ncell, 0.0);
      for (int k = 0; k < s.n[2]; ++k)
        for (int j = 0; j < s.n[1]; ++j)
          for (int i = 0; i < s.n[0]; ++i) ubi[c][cidx(s, i, j, k)] = v2b[c][pidx(s, i, j, k)];
    }
    bdim_stage_adjoint(s, 2, dt, U0[n].data(), UP[n].data(), ubi, u0b, upb, mu0bar, mu1bar);
    for (int c = 0; c < D; ++c)
      for (int k = 0; k < s.n[2]; ++k)
        for (int j = 0; j < s.n[1]; ++j)
          for (int i = 0; i < s.n[0]; ++i) ubi[c][cidx(s, i, j, k)] = upb[c][pidx(s, i, j, k)];
    project_adjoint(s, X1[n], ubi, vec(s.ncell, 0.0), rtol, v1b, Lbar);
    for (int c = 0; c < D; ++c)
      for (int k = 0; k < s.n[2]; ++k)
        for (int j = 0; j < s.n[1]; ++j)
          for (int i = 0; i < s.n[0]; ++i) ubi[c][cidx(s, i, j, k)] = v1b[c][pidx(s, i, j, k)];
    bdim_stage_adjoint(s, 1, dt, U0[n].data(), U0[n].data(), ubi, u0b, u0b, mu0bar, mu1bar);
    for (int c = 0; c < D; ++c)
      for (int k = 0; k < s.n[2]; ++k)
        for (int j = 0; j < s.n[1]; ++j)
          for (int i = 0; i < s.n[0]; ++i) ub[c][cidx(s, i, j, k)] = u0b[c][pidx(s, i, j, k)];
  }
  moments_adjoint(s, mu0bar, Lbar, mu1bar, tb);
}

}  // namespace

// ===========================================================================
// C interface (ctypes).  Fields cross the interface as interior arrays, x fastest:
// velocity as D consecutive blocks of ncell doubles (the lower faces of each cell),
// scalars as ncell doubles.
extern "C" {

void* or_create(int D, const int* dims, double nu, const double* U, unsigned periodic, int body_kind,
                const double* center, double radius, double radius2, double eps, int advect, double dt_cap) {
  if (D < 2 || D > 3) return nullptr;
  OSim* s = new OSim();
  s->D = D;
  for (int d = 0; d < 3; ++d) {
    s->n[d] = (d < D) ? dims[d] : 1;
    s->g[d] = (d < D) ? 2 : 0;
    s->np[d] = s->n[d] + 2 * s->g[d];
    s->U[d] = (d < D) ? U[d] : 0.0;
    s->center[d] = (center && d < D) ? center[d] : 0.0;
  }
  s->ncell = (long)s->n[0] * s->n[1] * s->n[2];
  s->npad = (long)s->np[0] * s->np[1] * s->np[2];
  s->periodic = periodic;
  s->nu = nu;
  s->body_kind = body_kind;
  s->radius = radius;
  s->radius2 = radius2;
  s->eps = eps;
  s->advect = advect;
  s->dt_cap = dt_cap;
  s->t = 0.0;
  s->nsteps = 0;
  s->last_iters = 0;
  s->last_resid = 0.0;
  for (int c = 0; c < D; ++c) s->u[c].assign(s->npad, 0.0);
  s->p.assign(s->ncell, 0.0);
  measure(*s);
  s->dt = 0.0;
  return s;
}

// A body given by its signed distance sampled at the grid's nodes (body_kind 3): the
// field replaces the closed-form distance, and the moments and levels are rebuilt.
void or_set_body_nodes(void* h, const double* nodes) {
  OSim* s = (OSim*)h;
  const long nn = (long)(s->n[0] + 1) * (s->n[1] + 1) * (s->D == 3 ? s->n[2] + 1 : 1);
  s->nodes.assign(nodes, nodes + nn);
  s->body_kind = 3;
  measure(*s);
}

void or_destroy(void* h) { delete (OSim*)h; }

// Convective exit on the upper x face (exit_f / exit_out); x must not be periodic.  The
// exit face starts at U_x.  Returns 0, or -1 if x is periodic.
int or_set_exit(void* h, int on) {
  OSim* s = (OSim*)h;
  if (on && is_per(*s, 0)) return -1;
  s->exit_bc = on ? 1 : 0;
  if (on)
    for (int k = 0; k < s->n[2]; ++k)
      for (int j = 0; j < s->n[1]; ++j) s->u[0][pidx(*s, s->n[0], j, k)] = s->U[0];
  apply_bc(*s, s->u);
  return 0;
}
// Set the exit plane's normal velocity (n_1 * n_2 values, y fastest).
void or_set_exit_plane(void* h, const double* in) {
  OSim* s = (OSim*)h;
  for (int k = 0; k < s->n[2]; ++k)
    for (int j = 0; j < s->n[1]; ++j) s->u[0][pidx(*s, s->n[0], j, k)] = in[j + (long)s->n[1] * k];
  apply_bc(*s, s->u);
}
// The exit plane's normal velocity (n_1 * n_2 values, y fastest).
void or_get_exit(void* h, double* out) {
  OSim* s = (OSim*)h;
  for (int k = 0; k < s->n[2]; ++k)
    for (int j = 0; j < s->n[1]; ++j) out[j + (long)s->n[1] * k] = s->u[0][pidx(*s, s->n[0], j, k)];
}

int or_nlevels(void* h) { return (int)((OSim*)h)->lev.size(); }
void or_level_dims(void* h, int l, int* dims) {
  OSim* s = (OSim*)h;
  for (int d = 0; d < 3; ++d) dims[d] = s->lev[l].n[d];
}
// Face coefficients of level l: D blocks of that level's ncell.
void or_get_level_L(void* h, int l, double* out) {
  OSim* s = (OSim*)h;
  const Level& lv = s->lev[l];
  for (int c = 0; c < s->D; ++c) std::memcpy(out + c * lv.ncell, lv.L[c].data(), lv.ncell * sizeof(double));
}
void or_get_mu0(void* h, double* out) {
  OSim* s = (OSim*)h;
  for (int c = 0; c < s->D; ++c) std::memcpy(out + c * s->ncell, s->mu0[c].data(), s->ncell * sizeof(double));
}
// mu1: D*D blocks, block (c*D + j) = component j of mu1 n at the lower c-faces.
void or_get_mu1(void* h, double* out) {
  OSim* s = (OSim*)h;
  for (int c = 0; c < s->D; ++c)
    for (int j = 0; j < s->D; ++j)
      std::memcpy(out + (c * s->D + j) * s->ncell, s->mu1[c][j].data(), s->ncell * sizeof(double));
}

void or_set_u(void* h, const double* in) {
  OSim* s = (OSim*)h;
  for (int c = 0; c < s->D; ++c)
    for (int k = 0; k < s->n[2]; ++k)
      for (int j = 0; j < s->n[1]; ++j)
        for (int i = 0; i < s->n[0]; ++i) s->u[c][pidx(*s, i, j, k)] = in[c * s->ncell + cidx(*s, i, j, k)];
  apply_bc(*s, s->u);
}
void or_get_u(void* h, double* out) {
  OSim* s = (OSim*)h;
  for (int c = 0; c < s->D; ++c)
    for (int k = 0; k < s->n[2]; ++k)
      for (int j = 0; j < s->n[1]; ++j)
        for (int i = 0; i < s->n[0]; ++i) out[c * s->ncell + cidx(*s, i, j, k)] = s->u[c][pidx(*s, i, j, k)];
}
// Padded velocity with every ghost and boundary face (for BC checks): D blocks of npad.
long or_npad(void* h) { return ((OSim*)h)->npad; }
void or_get_u_padded(void* h, double* out) {
  OSim* s = (OSim*)h;
  for (int c = 0; c < s->D; ++c) std::memcpy(out + c * s->npad, s->u[c].data(), s->npad * sizeof(double));
}
void or_set_p(void* h, const double* in) {
  OSim* s = (OSim*)h;
  std::memcpy(s->p.data(), in, s->ncell * sizeof(double));
}
void or_get_p(void* h, double* out) {
  OSim* s = (OSim*)h;
  std::memcpy(out, s->p.data(), s->ncell * sizeof(double));
}
double or_get_dt(void* h) { return ((OSim*)h)->dt; }
void or_set_dt(void* h, double dt) { ((OSim*)h)->dt = dt; }
double or_get_time(void* h) { return ((OSim*)h)->t; }
int or_last_iters(void* h) { return ((OSim*)h)->last_iters; }
double or_last_resid(void* h) { return ((OSim*)h)->last_resid; }

// Initial condition: kind 0 uniform U; kind 1 Taylor-Green vortex sampled at each
// component's own face positions with wavenumber k = 2 pi / n_0 and amplitude `amp`.
// Then BC and the initial dt from the CFL rule.
void or_set_ic(void* h, int kind, double amp) {
  OSim* s = (OSim*)h;
  double kw = 2.0 * M_PI / s->n[0];
  for (int c = 0; c < s->D; ++c)
    for (int k = 0; k < s->n[2]; ++k)
      for (int j = 0; j < s->n[1]; ++j)
        for (int i = 0; i < s->n[0]; ++i) {
          double v = s->U[c];
          if (kind == 1) {
            double x[3] = {i + 0.5, j + 0.5, k + 0.5};
            x[c] -= 0.5;
            double cz = (s->D == 3) ? std::cos(kw * x[2]) : 1.0;
            if (c == 0) v = amp * std::sin(kw * x[0]) * std::cos(kw * x[1]) * cz;
            else if (c == 1) v = -amp * std::cos(kw * x[0]) * std::sin(kw * x[1]) * cz;
            else v = 0.0;
          }
          s->u[c][pidx(*s, i, j, k)] = v;
        }
  if (s->exit_bc)  // the exit face starts at the free stream
    for (int k = 0; k < s->n[2]; ++k)
      for (int j = 0; j < s->n[1]; ++j) s->u[0][pidx(*s, s->n[0], j, k)] = s->U[0];
  apply_bc(*s, s->u);
  std::fill(s->p.begin(), s->p.end(), 0.0);
  s->dt = cfl(*s);
  s->t = 0.0;
  s->nsteps = 0;
}

// r = convdiff(u) for an interior velocity u (BC applied internally).
void or_convdiff(void* h, const double* uin, double* rout) {
  OSim* s = (OSim*)h;
  vec u[3], r[3];
  for (int c = 0; c < s->D; ++c) {
    u[c].assign(s->npad, 0.0);
    for (int k = 0; k < s->n[2]; ++k)
      for (int j = 0; j < s->n[1]; ++j)
        for (int i = 0; i < s->n[0]; ++i) u[c][pidx(*s, i, j, k)] = uin[c * s->ncell + cidx(*s, i, j, k)];
  }
  copy_exit(*s, u);
  apply_bc(*s, u);
  convdiff(*s, u, r);
  for (int c = 0; c < s->D; ++c) std::memcpy(rout + c * s->ncell, r[c].data(), s->ncell * sizeof(double));
}

// One BDIM stage on interior arrays: stage 1 uses u0 only; stage 2 uses u0 and u1.
void or_bdim_stage(void* h, int stage, double dt, const double* u0in, const double* u1in, double* out) {
  OSim* s = (OSim*)h;
  vec u0[3], u1[3], o[3];
  for (int c = 0; c < s->D; ++c) {
    u0[c].assign(s->npad, 0.0);
    u1[c].assign(s->npad, 0.0);
    for (int k = 0; k < s->n[2]; ++k)
      for (int j = 0; j < s->n[1]; ++j)
        for (int i = 0; i < s->n[0]; ++i) {
          long q = c * s->ncell + cidx(*s, i, j, k);
          u0[c][pidx(*s, i, j, k)] = u0in[q];
          if (u1in) u1[c][pidx(*s, i, j, k)] = u1in[q];
        }
  }
  copy_exit(*s, u0);
  copy_exit(*s, u1);
  apply_bc(*s, u0);
  apply_bc(*s, u1);
  bdim_stage(*s, stage, dt, u0, u1, o);
  for (int c = 0; c < s->D; ++c)
    for (int k = 0; k < s->n[2]; ++k)
      for (int j = 0; j < s->n[1]; ++j)
        for (int i = 0; i < s->n[0]; ++i) out[c * s->ncell + cidx(*s, i, j, k)] = o[c][pidx(*s, i, j, k)];
}

void or_divergence(void* h, double* z) {
  OSim* s = (OSim*)h;
  vec zz;
  divergence(*s, s->u, zz);
  std::memcpy(z, zz.data(), s->ncell * sizeof(double));
}

// y = A_l x on level l.
void or_poisson_apply(void* h, int l, const double* x, double* y) {
  OSim* s = (OSim*)h;
  Op A = make_op(*s, s->lev[l]);
  vec xx(x, x + A.ncell), yy;
  A.apply(xx, yy);
  std::memcpy(y, yy.data(), A.ncell * sizeof(double));
}
void or_poisson_diag(void* h, int l, double* dg) {
  OSim* s = (OSim*)h;
  Op A = make_op(*s, s->lev[l]);
  vec d;
  A.diagonal(d);
  std::memcpy(dg, d.data(), A.ncell * sizeof(double));
}
int or_pcg(void* h, int l, double* x, const double* z, double tol, int maxit, double* resid) {
  OSim* s = (OSim*)h;
  Op A = make_op(*s, s->lev[l]);
  vec xx(x, x + A.ncell), zz(z, z + A.ncell);
  int it = pcg(A, xx, zz, tol, maxit, resid);
  std::memcpy(x, xx.data(), A.ncell * sizeof(double));
  return it;
}
int or_dense_solve(void* h, int l, double* x, const double* z) {
  OSim* s = (OSim*)h;
  Op A = make_op(*s, s->lev[l]);
  vec xx, zz(z, z + A.ncell);
  int rc = dense_solve(A, xx, zz);
  std::memcpy(x, xx.data(), A.ncell * sizeof(double));
  return rc;
}
// One V-cycle on the fine level: x updated in place; returns ||z - A x||_inf after it.
double or_vcycle(void* h, double* x, const double* z, int pre, int post) {
  OSim* s = (OSim*)h;
  vec xx(x, x + s->ncell), zz(z, z + s->ncell);
  vcycle(*s, 0, xx, zz, pre, post);
  std::memcpy(x, xx.data(), s->ncell * sizeof(double));
  Op A = make_op(*s, s->lev[0]);
  vec Ax;
  A.apply(xx, Ax);
  double m = 0.0;
  for (long q = 0; q < s->ncell; ++q) m = std::max(m, std::fabs(zz[q] - Ax[q]));
  return m;
}
void or_rb_sweep(void* h, int l, double* x, const double* z) {
  OSim* s = (OSim*)h;
  Op A = make_op(*s, s->lev[l]);
  vec xx(x, x + A.ncell), zz(z, z + A.ncell);
  rb_sweep(A, xx, zz);
  std::memcpy(x, xx.data(), A.ncell * sizeof(double));
}

// project! on the state velocity with weight w and the given dt.
void or_project(void* h, double w, double dt, double tol, int maxit, int solver) {
  OSim* s = (OSim*)h;
  project(*s, s->u, w, dt, tol, maxit, solver);
}

// One full time step (Heun; see the header).  dt_fixed > 0 keeps dt fixed.
void or_step(void* h, int nsteps, double tol, int maxit, double dt_fixed, int solver) {
  OSim* s = (OSim*)h;
  for (int it = 0; it < nsteps; ++it) {
    double dt = (dt_fixed > 0.0) ? dt_fixed : s->dt;
    vec u0[3], u1[3];
    for (int c = 0; c < s->D; ++c) u0[c] = s->u[c];
    bdim_stage(*s, 1, dt, u0, u0, u1);
    project(*s, u1, 1.0, dt, tol, maxit, solver);
    bdim_stage(*s, 2, dt, u0, u1, s->u);
    project(*s, s->u, 0.5, dt, tol, maxit, solver);
    s->t += dt;
    s->nsteps += 1;
    s->dt = (dt_fixed > 0.0) ? dt_fixed : cfl(*s);
  }
}

double or_cfl(void* h) { return cfl(*(OSim*)h); }

// Pressure force F_d = -sum_cells (p - mean_active p) n_d K_eps(d), K_eps = (1 + cos(pi d/eps))/(2 eps)
// for |d| < eps (cell centres, volume 1).
void or_forces(void* h, double* F) {
  OSim* s = (OSim*)h;
  Op A = make_op(*s, s->lev[0]);
  vec dg;
  A.diagonal(dg);
  double sum = 0.0;
  long cnt = 0;
  for (long q = 0; q < s->ncell; ++q)
    if (dg[q] > 0.0) {
      sum += s->p[q];
      ++cnt;
    }
  double pm = cnt ? sum / cnt : 0.0;
  for (int d = 0; d < 3; ++d) F[d] = 0.0;
  if (s->body_kind == 0) return;
  for (int k = 0; k < s->n[2]; ++k)
    for (int j = 0; j < s->n[1]; ++j)
      for (int i = 0; i < s->n[0]; ++i) {
        double x[3] = {i + 0.5, j + 0.5, k + 0.5}, nrm[3];
        double d = sdf(*s, x, nrm);
        if (std::fabs(d) >= s->eps) continue;
        double K = (1.0 + std::cos(M_PI * d / s->eps)) / (2.0 * s->eps);
        double pp = s->p[cidx(*s, i, j, k)] - pm;
        for (int dd = 0; dd < s->D; ++dd) F[dd] -= pp * nrm[dd] * K;
      }
}

// Viscous force on the body (reading: the paper states no force; this is the viscous
// part of the surface integral, kernel-weighted like the pressure force):
// F_i = sum_cells 2 nu S_ij n_j K_eps(d) over cells with |d| < eps, with the strain rate
// S = (grad u + grad u^T)/2 at the cell centre: du_c/dx_c from the cell's two c-faces,
// du_c/dx_e (e != c) by the central difference of the cell-centred u_c (the mean of its
// two faces) over the neighbours at -e and +e.  Ghosts carry the BC.
void or_viscous_force(void* h, double* F) {
  OSim* s = (OSim*)h;
  for (int d = 0; d < 3; ++d) F[d] = 0.0;
  if (s->body_kind == 0) return;
  auto uc = [&](int c, const int* I) {  // u_c at the centre of cell I
    int J[3] = {I[0], I[1], I[2]};
    J[c] += 1;
    return 0.5 * (s->u[c][pidx(*s, I)] + s->u[c][pidx(*s, J)]);
  };
  for (int k = 0; k < s->n[2]; ++k)
    for (int j = 0; j < s->n[1]; ++j)
      for (int i = 0; i < s->n[0]; ++i) {
        double x[3] = {i + 0.5, j + 0.5, k + 0.5}, nrm[3];
        double d = sdf(*s, x, nrm);
        if (std::fabs(d) >= s->eps) continue;
        double K = (1.0 + std::cos(M_PI * d / s->eps)) / (2.0 * s->eps);
        const int I[3] = {i, j, k};
        double G[3][3] = {{0.0}};  // G[c][e] = du_c/dx_e
        for (int c = 0; c < s->D; ++c)
          for (int e = 0; e < s->D; ++e) {
            if (c == e) {
              int J[3] = {i, j, k};
              J[c] += 1;
              G[c][e] = s->u[c][pidx(*s, J)] - s->u[c][pidx(*s, I)];
            } else {
              int Jp[3] = {i, j, k}, Jm[3] = {i, j, k};
              Jp[e] += 1;
              Jm[e] -= 1;
              G[c][e] = 0.5 * (uc(c, Jp) - uc(c, Jm));
            }
          }
        for (int a = 0; a < s->D; ++a)
          for (int b = 0; b < s->D; ++b) F[a] += 2.0 * s->nu * 0.5 * (G[a][b] + G[b][a]) * nrm[b] * K;
      }
}

// Kinetic energy E = 1/2 sum_faces sum_c u_c^2 / ncell (stored lower faces).
double or_kinetic_energy(void* h) {
  OSim* s = (OSim*)h;
  double e = 0.0;
  for (int c = 0; c < s->D; ++c)
    for (int k = 0; k < s->n[2]; ++k)
      for (int j = 0; j < s->n[1]; ++j)
        for (int i = 0; i < s->n[0]; ++i) {
          double v = s->u[c][pidx(*s, i, j, k)];
          e += v * v;
        }
  return 0.5 * e / s->ncell;
}

double or_K0(double x) { return K0(x); }
double or_K1(double x) { return K1(x); }
double or_face_value(double uu, double cc, double dd) { return face_value(uu, cc, dd); }
double or_psi(double r) { return std::max(0.0, std::min(std::min(2.0 * r, (2.0 + r) / 3.0), 2.0)); }
double or_sdf(void* h, const double* x, double* nrm) { return sdf(*(OSim*)h, x, nrm); }

// ---- adjoint (reverse-mode derivative) entry points; see rollout_grad and the
// transposes above.  Interior arrays as for the forward routines.
namespace {
void to_padded(const OSim& s, const double* in, vec* u) {
  for (int c = 0; c < s.D; ++c) {
    u[c].assign(s.npad, 0.0);
    for (int k = 0; k < s.n[2]; ++k)
      for (int j = 0; j < s.n[1]; ++j)
        for (int i = 0; i < s.n[0]; ++i) u[c][pidx(s, i, j, k)] = in[c * s.ncell + cidx(s, i, j, k)];
  }
  copy_exit(s, u);
  apply_bc(s, u);
}
void from_padded(const OSim& s, const vec* u, double* out) {
  for (int c = 0; c < s.D; ++c)
    for (int k = 0; k < s.n[2]; ++k)
      for (int j = 0; j < s.n[1]; ++j)
        for (int i = 0; i < s.n[0]; ++i) out[c * s.ncell + cidx(s, i, j, k)] = u[c][pidx(s, i, j, k)];
}
}  // namespace

// ubar = (d convdiff / du)^T rbar at u.
void or_convdiff_adjoint(void* h, const double* uin, const double* rbar, double* ubar) {
  OSim* s = (OSim*)h;
  vec u[3], rb[3], ub[3];
  to_padded(*s, uin, u);
  for (int c = 0; c < s->D; ++c) {
    rb[c].assign(rbar + c * s->ncell, rbar + (c + 1) * s->ncell);
    ub[c].assign(s->npad, 0.0);
  }
  convdiff_adjoint(*s, u, rb, ub);
  from_padded(*s, ub, ubar);
}

// Transpose of one BDIM stage at (u0, u1): outbar -> u0bar, u1bar (D blocks each),
// mu0bar (D blocks), mu1bar (D*D blocks, block c*D + j).
void or_stage_adjoint(void* h, int stage, double dt, const double* u0in, const double* u1in, const double* outbar,
                      double* u0bar, double* u1bar, double* mu0bar, double* mu1bar) {
  OSim* s = (OSim*)h;
  vec u0[3], u1[3], ob[3], u0b[3], u1b[3], m0b[3], m1b[3][3];
  to_padded(*s, u0in, u0);
  to_padded(*s, u1in ? u1in : u0in, u1);
  for (int c = 0; c < s->D; ++c) {
    ob[c].assign(outbar + c * s->ncell, outbar + (c + 1) * s->ncell);
    u0b[c].assign(s->npad, 0.0);
    u1b[c].assign(s->npad, 0.0);
    m0b[c].assign(s->ncell, 0.0);
    for (int j = 0; j < 3; ++j) m1b[c][j].assign(s->ncell, 0.0);
  }
  bdim_stage_adjoint(*s, stage, dt, u0, u1, ob, u0b, u1b, m0b, m1b);
  from_padded(*s, u0b, u0bar);
  from_padded(*s, u1b, u1bar);
  for (int c = 0; c < s->D; ++c) {
    std::memcpy(mu0bar + c * s->ncell, m0b[c].data(), s->ncell * sizeof(double));
    for (int j = 0; j < s->D; ++j) std::memcpy(mu1bar + (c * s->D + j) * s->ncell, m1b[c][j].data(), s->ncell * sizeof(double));
  }
}

// Transpose of project! of the velocity v (interior) with weight w: the forward solve
// (PCG to tol) gives x; then ubar (D blocks) and pbar (cells, cotangent of p) give
// vbar (D blocks) and Lbar (D blocks).  The state is not changed.
void or_project_adjoint(void* h, const double* vin, double w, double dt, double tol, const double* ubar,
                        const double* pbar, double* vbar, double* Lbar) {
  OSim* s = (OSim*)h;
  OSim t = *s;  // work on a copy of the state
  vec v[3], ub[3], vb[3], Lb[3];
  to_padded(t, vin, v);
  std::fill(t.p.begin(), t.p.end(), 0.0);
  project(t, v, w, dt, tol, 1000000, 0);
  vec x = t.p;
  for (auto& q : x) q *= w * dt;
  vec xb(pbar, pbar + s->ncell);
  for (auto& q : xb) q /= w * dt;
  for (int c = 0; c < s->D; ++c) {
    ub[c].assign(ubar + c * s->ncell, ubar + (c + 1) * s->ncell);
    Lb[c].assign(s->ncell, 0.0);
  }
  project_adjoint(t, x, ub, xb, 1e-13, vb, Lb);
  from_padded(t, vb, vbar);
  for (int c = 0; c < s->D; ++c) std::memcpy(Lbar + c * s->ncell, Lb[c].data(), s->ncell * sizeof(double));
}

// Force of the pressure p (cells) and its adjoint for Fbar: pbar (cells) and the
// theta-cotangent of the force weights (n_theta values: circle/sphere D + 1, torus 5).
void or_force_adjoint(void* h, const double* p, const double* Fbar, double* F, double* pbar, double* tb) {
  OSim* s = (OSim*)h;
  vec pp(p, p + s->ncell), pb;
  for (int t = 0; t < n_theta(*s); ++t) tb[t] = 0.0;
  force_adjoint(*s, pp, Fbar, F, pb, tb);
  std::memcpy(pbar, pb.data(), s->ncell * sizeof(double));
}

// theta-cotangent of field cotangents of the moments and coefficients (moments_adjoint).
void or_moments_adjoint(void* h, const double* mu0bar, const double* Lbar, const double* mu1bar, double* tb) {
  OSim* s = (OSim*)h;
  vec m0[3], Lb[3], m1[3][3];
  for (int c = 0; c < s->D; ++c) {
    m0[c].assign(mu0bar + c * s->ncell, mu0bar + (c + 1) * s->ncell);
    Lb[c].assign(Lbar + c * s->ncell, Lbar + (c + 1) * s->ncell);
    for (int j = 0; j < 3; ++j)
      m1[c][j] = (j < s->D) ? vec(mu1bar + (c * s->D + j) * s->ncell, mu1bar + (c * s->D + j + 1) * s->ncell)
                            : vec(s->ncell, 0.0);
  }
  for (int t = 0; t < n_theta(*s); ++t) tb[t] = 0.0;
  moments_adjoint(*s, m0, Lb, m1, tb);
}

// Differentiated rollout (rollout_grad): returns 0, or -1 unless the body is a circle/sphere.
int or_rollout_grad(void* h, int nsteps, double dt, double tol, const double* gF, double* F, double* tb) {
  OSim* s = (OSim*)h;
  if (!(s->body_kind == 1 || (s->body_kind == 2 && s->D == 3)) || nsteps < 1 || !(dt > 0.0) || s->exit_bc)
    return -1;
  rollout_grad(*s, nsteps, dt, tol, gF, F, tb);
  return 0;
}


}  // extern "C"
