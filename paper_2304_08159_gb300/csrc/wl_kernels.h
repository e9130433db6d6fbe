// Internal launch interface between the host runtime (wl_api.cu) and the kernels.
#pragma once
#include <cuda.h>
#include <cuda_runtime.h>
#include "wl_dev.cuh"

namespace wl {

struct StageArgs {
  const float* u[3];    // velocity whose convection-diffusion residual is taken
  const float* u0[3];   // start-of-step velocity
  const float* mu0[3];  // BDIM zeroth moment on updated faces (= Poisson coefficient there)
  float* out[3];
  Grid g;
  const float* dt;      // device scalar (FP32 copy of the step's dt)
  float nu;
  int stage;            // 1 or 2
  int advect;
  float* fbox;          // if set: f = u0 + dt r(u) of every face in the body's band box (D blocks of
  int blo[3], bn[3];    //   bn[0]*bn[1]*bn[2] values, box origin blo), kept for the mu1 term
  int tz;               // 3-D two-cell kernel: planes per block (0: the default 32)
};
// planes per block of the 3-D stage kernel for grid g: as many blocks as fill the GPU
// (small grids), at most 32 planes (the z halo is re-read once per block)
int stage3_planes(const Grid& g);
// Faces whose f the mu1 term of BDIM reads: the body's band (|d| < eps) and one face
// beyond, boxed ([lo, hi) per direction, clamped to the grid); false if the box is empty.
bool stage_band_box(int D, const Grid& g, const Body& b, int* lo, int* hi);

// residual / divergence / restriction modes of k_residual
enum { RES_RESIDUAL = 0, RES_DIVERGENCE = 1, RES_RESTRICT = 2, RES_DIV_ONLY = 3 };

// The fine-level pressure of precision mode 1 is an unevaluated sum ph + pl of two
// FP32 fields (a "double-float"); arithmetic on it uses error-free transformations,
// so no FP64 instruction runs per cell (FP64 throughput is a small fraction of FP32
// on this GPU).
struct ResArgs {
  const float* u[3];   // RES_DIVERGENCE / RES_DIV_ONLY: velocity
  const float* x;      // current unknown (RES_RESIDUAL / RES_DIVERGENCE), unless ph is set
  const float* ph;     // if set: unknown = ph + pl, residual formed in double-float
  const float* pl;
  float* rout;         // if set: the residual is stored here (right-hand side of the correction cycle)
  const float* L[3];   // face coefficients of this level
  float* z;            // right-hand side of this level (written by the divergence modes)
  float* zc;           // restricted residual for the next level (may be null)
  Grid g;
  int cn[3];           // next level's dims
  int ztype;           // storage type (ST_*) of z in RES_RESTRICT mode (else ST_F32)
  int zctype;          // storage type of zc
  float zcmul;         // zc = zcmul * (sum of the 2^D children): the levels' scale ratio
  float* zconv;        // RES_RESTRICT: if set, also store zconvmul * z here (type zconvtype)
  int zconvtype;
  float zconvmul;
  int apply_cs;        // multiply zc and zconv by 2^(st->cs_used) as well
  float inv_w;         // divergence modes: z = div u * inv_w / dt
  DevState* st;        // dt and the running max |residual|
  int mode;
  int uni;             // 1: no body on the level, so every face coefficient is uval (0 across
  float uval;          //   a non-periodic wall) and is formed instead of loaded
};

// A 16-bit level (stype != ST_F32) keeps x_in, z, L and x_out in that type (the
// pointers are then reinterpreted) and stores its right-hand side scaled: the value
// used is zmul * z.
struct SweepArgs {
  const float* x_in;   // current iterate, or null for zero
  const float* xc;     // coarse correction added by piecewise-constant prolongation, or null
  const float* z;
  const float* L[3];
  float* x_out;
  int stype;           // storage type (ST_*) of x_in, z, L, x_out
  int xctype;          // storage type of xc
  float zmul;
  const DevState* cs;  // if set, xc carries the factor 2^(cs->cs_used), removed on reading
  float* ph;           // if set: add the swept values into the double-float field ph + pl
  float* pl;           //   instead of writing x_out
  Grid g;
  int cn[3];
  int tz;              // planes per block (3-D)
  int only_wrapping;   // 1: sweep only the tiles whose footprint crosses a periodic side
  int uni;             // 1: no body on the level, so every face coefficient is uval (0 across
  float uval;          //   a non-periodic wall) and is formed instead of loaded
};

// Region of a level (level cell coordinates, [lo, hi) per direction) whose face
// coefficients may differ from the level's free-stream value: the body's band box
// scaled to the level.  Tiles whose footprint misses it take the staged kernels'
// uniform variants, which compute the coefficients (free-stream value, 0 on walls)
// instead of loading them.  on = 0: no split, every tile loads its coefficients.
struct BandBox {
  int on;
  int lo[3], hi[3];
};

// TMA-staged sweep (wl_sweep_tma.cu): tensor maps of the fields of one level
// (box 72 x 12 [x 1], x start 16-byte aligned, zero fill out of range).
struct SweepMaps {
  CUtensorMap x, z, L0, L1, L2;
};
struct SweepTmaArgs {
  int has_x;           // stage the iterate (else it starts from zero)
  const float* xc;     // coarse correction to prolong into it, or null
  int xctype;          // storage type (ST_*) of xc
  int xc_cs;           // xc carries the factor 2^(st->cs_used), removed on reading
  float* x_out;
  float* ph;           // if set: fold the result into ph + pl instead of writing x_out
  float* pl;
  Grid g;
  int cn[3];
  int tz;
  DevState* st;        // status bit 2 set if a staged copy never arrived
  BandBox band;        // tiles outside it: coefficients = uval (0 on walls), not loaded
  float uval;
  int t0[3];           // first tile of the launch (the band tiles' launch starts inside the grid)
  int plain;           // sweep the tiles that cross no periodic x / y side
  int wrap;            // also sweep (uniform variant, tzw planes per block) the tiles that
                       // cross one; their halo
                       // elements past the side are read from the wrapped cells of:
  const float* xsrc;   //   the staged iterate (has_x)
  const float* zsrc;   //   the staged right-hand side
  int tzw;             // planes per block of the wrapping tiles' launch (its own residency)
  int ty;              // tile height of the plain tiles: 8, or 16 (SWEEP_TY16; maps with its boxes)
};

// Dense pseudo-inverse of the coarsest operator (column-major, FP64), used when the
// coarsest level has at most kDenseCoarse cells.
constexpr int kDenseCoarse = 1024;
struct DenseArgs {
  const float* L[3];
  Grid g;
  double* G;           // nc x nc, column j = A^+ e_j
  const float* z;
  float* x;
};

// The coarse end of a V-cycle in one block (k_vcycle_tail): levels lf .. lf + nl - 1
// (the last one the coarsest, solved by its dense pseudo-inverse), all held in shared
// memory.  Reads level lf's right-hand side, writes level lf's smoothed correction.
constexpr int kTailMaxLevels = 8;
constexpr int kTailThreads = 1024;
constexpr size_t kTailSmemMax = 200 * 1024;  // bytes of shared memory the tail may use
struct TailArgs {
  int nl;
  int n[kTailMaxLevels][3];
  const float* L[kTailMaxLevels][3];  // each level's coefficients (storage type st[l])
  int st[kTailMaxLevels];
  const float* z;                      // level lf's right-hand side (type st[0]), value = zmul * stored
  float zmul;
  float* x;                            // level lf's correction out (type st[0])
  const double* G;                     // coarsest pseudo-inverse, column-major
  int post;
  unsigned per;
};
int launch_vcycle_tail(int D, const TailArgs& a, cudaStream_t s);
size_t vcycle_tail_smem(int D, const int (*n)[3], int nl);
// the same coarse end in one cluster of C blocks (each keeping slices of every level):
// shared bytes of the largest block, whether a cluster of C such blocks can run (C or
// 0; sets the kernel's attributes), and the launch
size_t vcycle_ctail_smem(int D, const int (*n)[3], int nl, int C);
int vcycle_ctail_cluster(int D, size_t smem, int C);
int launch_vcycle_ctail(int D, const TailArgs& a, int C, cudaStream_t s);

struct CoarseArgs {
  const float* z;
  const float* L[3];
  float* x;
  Grid g;
  double* work;        // 5 * g.nc doubles
  int maxit;
  double rtol;
};

struct CorrArgs {
  const float* u_in[3];
  float* u_out[3];
  const float* x;      // pressure p (plain FP32), unless ph is set
  const float* ph;     // double-float pressure ph + pl
  const float* pl;
  const float* L[3];
  Grid g;
  float w;
  int cfl;             // also accumulate the CFL out-flux maximum
  DevState* st;        // dt and the CFL maximum
};

int launch_stage(int D, const StageArgs& a, cudaStream_t s);
int launch_band(int D, const StageArgs& a, const Body& b, cudaStream_t s);
// Convective exit of one stage: the exit plane of outx from those of u0x and uinx (and
// u_in's last x faces), shifted so that its mean is U_x.  One block.
int launch_exit_stage(int D, const Grid& g, const float* u0x, const float* uinx, float* outx, const float* dt, int stage,
                      cudaStream_t s);
// fill n floats with v
int launch_fill(float* p, long long n, float v, cudaStream_t s);
int launch_residual(int D, const ResArgs& a, cudaStream_t s);
int launch_sweep(int D, const SweepArgs& a, cudaStream_t s);
// A second stream on which the loading (band) tiles' launch runs beside the uniform
// tiles' launch (fork / join by events; captured as parallel graph branches).
struct SideStream {
  cudaStream_t aux;
  cudaEvent_t fork, join;
  // profiling only: called before (begin 1) and after (begin 0) the uniform (band 0) and
  // the band-tile (band 1) launch, on the stream that launch goes to
  void (*hook)(void* ctx, int band, int begin, cudaStream_t st);
  void* ctx;
};
int launch_sweep_tma(int D, const SweepMaps& m, const SweepTmaArgs& a, cudaStream_t s, const SideStream* side);
// fraction of a level's sweep tiles (tz planes per block) that meet the band box
double band_tile_fraction(int D, const Grid& g, int tz, const BandBox& b, int ty);  // ty: tile height

// TMA-staged fine residual / divergence (3-D, levels with no periodic side)
struct ResidMaps {
  CUtensorMap ph, pl, z, u0, u1, u2, L0, L1, L2;  // ph: the pressure (hi part, or the FP32 pressure)
};
struct ResidTmaArgs {
  int div;             // divergence mode: z = div u * inv_w / dt is formed and stored
  int df;              // pressure is the double-float ph + pl
  float* z;            // divergence mode: right-hand side out
  float* rout;         // residual out (or null)
  float* zc;           // restricted residual (or null)
  int zctype;          // storage type (ST_*) of zc
  float zcmul;         // zc = zcmul * (sum of the 2^D children)
  Grid g;
  int cn[3];
  int tz;              // planes per block (even)
  float inv_w;
  DevState* st;        // dt, residual maximum, timeout flag
  BandBox band;        // tiles outside it: coefficients 1 (0 on walls), not loaded
  int t0[3];           // first tile of the launch
  const float* uxe;    // divergence mode with a convective exit: the velocity's exit plane
  // periodic x / y sides: the fields whose halo cells past such a side a tile patches
  // (pressure hi or the FP32 pressure, pressure lo, and in divergence mode u_x, u_y)
  const float* wsrc[4];
};
int launch_resid_tma(const ResidMaps& m, const ResidTmaArgs& a, cudaStream_t s, const SideStream* side);
// A residual tile (64 x 8 cells at i0, j0) on a periodic x or y side of the grid: its
// stencil reads halo cells past the side
__host__ __device__ inline bool resid_tile_wraps_xy(const Grid& g, int i0, int j0) {
  return ((g.per & 1u) && (i0 == 0 || i0 + 64 >= g.n[0])) || ((g.per & 2u) && (j0 == 0 || j0 + 8 >= g.n[1]));
}
// whether a tile of the band box (which loads its coefficients) lies on a periodic x / y side
bool resid_band_wraps(const Grid& g, int tz, const BandBox& b);
int launch_wait_probe(uint64_t limit_ns, int* gave_up, cudaStream_t s);
// planes per block of the sweep kernels for blocks_per_sm resident blocks
int sweep_planes_per_block(const Grid& g, int blocks_per_sm);
int sweep_planes_for_columns(int n2, long long tiles, int blocks_per_sm);
int sweep_table_blocks_per_sm(int D, int stype);

// Both sweep kernels cut a level into the same tiles of 64 x 8 cells and `tz` planes.
// k_sweep_tma stages planes past a periodic z side from their wrapped planes.  A tile
// whose TMA footprint (x i0-4..i0+67, y j0-2..j0+9) crosses a periodic x or y side is
// swept by k_sweep_tma's wrapping variant when the level's periodic sides are whole
// tiles (sweep_wrap_shape_ok) and every such tile is uniform, else by k_sweep.
constexpr int SWEEP_TX = 64, SWEEP_TY = 8;
// rows of the sweep's coefficient boxes (z, L0, L2; L1 takes one more), from j0-1
constexpr int SWEEP_CROWS = SWEEP_TY + 2;
// resident blocks per SM of the staged sweep (shared memory bound) and of its uniform
// variant (register bound)
constexpr int SWEEP_BLOCKS_PER_SM = 4;
constexpr int SWEEP_UNI_BLOCKS_PER_SM = 8;
constexpr int SWEEP_WRAP_BLOCKS_PER_SM = 5;  // the wrapping variant (register bound)
// tiles of 64 x 16 cells (large split levels with no periodic x / y side): shared memory
// bound, the uniform variant 44 KB per block, the loading one 97 KB
constexpr int SWEEP_TY16 = 16;
constexpr int SWEEP16_UNI_BLOCKS_PER_SM = 5;
constexpr int SWEEP16_BLOCKS_PER_SM = 2;
// blocks per SM the fine residual's z-blocking assumes for its split launches
constexpr int RESID_UNI_WAVE_BLOCKS = 6;
// The tile's staged footprint (x i0-4..i0+67, y j0-2..j0+ty+1, planes k0-2..k1+1)
// meets the band box (always true without a split).  ty: the tile height.
__host__ __device__ inline bool tile_in_band(const BandBox& b, int D, int i0, int j0, int k0, int k1,
                                             int ty = SWEEP_TY) {
  if (!b.on) return true;
  if (i0 - 4 >= b.hi[0] || i0 + SWEEP_TX + 4 <= b.lo[0]) return false;
  if (j0 - 2 >= b.hi[1] || j0 + ty + 2 <= b.lo[1]) return false;
  if (D == 3 && (k0 - 2 >= b.hi[2] || k1 + 2 <= b.lo[2])) return false;
  return true;
}
// The tile's footprint crosses a periodic x or y side (the staged sweep stages planes
// past a periodic z side from their wrapped planes; x and y wraps go to k_sweep).
__host__ __device__ inline bool sweep_tile_wraps_xy(const Grid& g, int i0, int j0) {
  if ((g.per & 1u) && (i0 - 4 < 0 || i0 + SWEEP_TX + 4 > g.n[0])) return true;
  if ((g.per & 2u) && (j0 - 2 < 0 || j0 + SWEEP_TY + 2 > g.n[1])) return true;
  return false;
}
// The level's periodic x / y sides are whole tiles (n_0 % 64 == 0, n_1 % 8 == 0), so every
// halo element of a tile past such a side is a cell of the wrapped tile column / row,
// and a plane's cells have a 32-bit index.
__host__ __device__ inline bool sweep_wrap_shape_ok(const Grid& g) {
  return (!(g.per & 1u) || g.n[0] % SWEEP_TX == 0) && (!(g.per & 2u) || g.n[1] % SWEEP_TY == 0) &&
         (long long)g.n[0] * g.n[1] < (1ll << 31);
}
__host__ __device__ inline bool sweep_tile_wraps(const Grid& g, int D, int i0, int j0, int k0, int k1) {
  if ((g.per & 1u) && (i0 - 4 < 0 || i0 + SWEEP_TX + 4 > g.n[0])) return true;
  if ((g.per & 2u) && (j0 - 2 < 0 || j0 + SWEEP_TY + 2 > g.n[1])) return true;
  if (D == 3 && (g.per & 4u) && (k0 - 2 < 0 || k1 + 2 > g.n[2])) return true;
  return false;
}
int launch_coarse(int D, const CoarseArgs& a, cudaStream_t s);
int launch_correct(int D, const CorrArgs& a, cudaStream_t s);
int launch_decide(DevState* st, cudaGraphConditionalHandle h, int use_handle, int first, int proj, float w,
                  double tol, int maxit, cudaStream_t s);
// End of a step: advance the clock, record the step's metrics in the ring (NMETRIC doubles
// per record, `cap` records; F: the metric force, or null when metrics are off), set the
// next dt from the CFL maximum.
constexpr int NMETRIC = 13;
int launch_step_end(DevState* st, int D, double nu, double dt_cap, double dt_fixed, double* ring, int cap,
                    const double* F, cudaStream_t s);
// Kinetic energy 0.5 sum_c sum_I u_c[I]^2 / n and max |div u| of velocity u into st->ke and
// st->maxdiv_bits: per-block FP64 partials (npart blocks) summed in a fixed order.
int launch_metrics_u(int D, const Grid& g, const float* const* u, DevState* st, double* partials, int npart,
                     cudaStream_t s);
int launch_measure(int D, const Grid& g, const Body& b, float* const* L, cudaStream_t s);
int launch_coarsen(int D, const Grid& fine, const float* const* Lf, const Grid& coarse, float* const* Lc,
                   cudaStream_t s);
int launch_set_ic(int D, const Grid& g, int kind, double amp, float* const* u, cudaStream_t s);
int launch_cfl_only(int D, const Grid& g, const float* const* u, DevState* st, cudaStream_t s);
int launch_viscous_force(int D, const Grid& g, const Body& b, const float* const* u, double nu, double* out,
                         cudaStream_t s);
int launch_forces(int D, const Grid& g, const Body& b, const float* p, const float* pl, const float* const* L,
                  double* partials, int npart, double* out, cudaStream_t s);
int launch_build_pinv(int D, const DenseArgs& a, cudaStream_t s);
int launch_apply_pinv(const DenseArgs& a, cudaStream_t s);
// ph + pl -> out (FP32 rounding of the double-float pressure)
int launch_df_round(const float* ph, const float* pl, float* out, long long n, cudaStream_t s);
// (ph, pl) += e (double-float accumulate)
int launch_df_add(float* ph, float* pl, const float* e, long long n, cudaStream_t s);
// FP32 -> storage type (ST_*) copy of n values (coarse-level face coefficients)
int launch_to_storage(const float* in, void* out, int type, long long n, cudaStream_t s);
int launch_sync_dt(DevState* st, cudaStream_t s);

}  // namespace wl

namespace wl {

// ---- reverse-mode derivative of the time step (wl_adjoint.cu)
struct AdjState {
  double theta[5];  // dJ/dtheta, accumulated: (R, c_0, .., c_{D-1}) or, torus, (R, r, c_x, c_y, c_z)
  double W[3];      // sum over band cells of the force weights n K_eps(d)
  double Na;        // active cells (nonzero Poisson row)
  double mean;      // mean over active cells of the last adjoint right-hand side
  unsigned bnorm_bits;  // ||b||_inf of the adjoint right-hand side (float bits)
  int iter;         // V-cycles of the running adjoint solve
  int total_iter;   // V-cycles of all adjoint solves of the backward pass
  int flags;        // 1: a non-finite adjoint residual, 2: an adjoint solve hit max_vcycles
  int rec_slot;     // the segment slot the recomputed step records into
};
int launch_adj_setup(int D, const Grid& g, const Body& b, const float* const* L, AdjState* as, double* part,
                     int npart, cudaStream_t s);
int launch_adj_force_theta(int D, const Grid& g, const Body& b, const float* p, const double* pmean,
                           const double* gF, AdjState* as, cudaStream_t s);
int launch_adj_proj_rhs(int D, const Grid& g, const Body& b, const float* const* ub, const float* const* L,
                        const double* gF, double fmul, AdjState* as, float* rhs, double* part, int npart,
                        cudaStream_t s);
int launch_adj_proj_out(int D, const Grid& g, const float* const* ub, const float* y, const float* p, float xmul,
                        float* const* vb, float* const* mbar, cudaStream_t s);
int launch_adj_stage_local(int D, const Grid& g, const float* const* vb, const float* const* mu0, float sfac,
                           float* const* fb, float* const* up, cudaStream_t s);
int launch_adj_band(int D, const StageArgs& a, const Body& b, const float* const* vb, float sfac, float* const* fb,
                    float* const* mbar, AdjState* as, double* part, int npart, cudaStream_t s);
int launch_adj_convdiff(int D, const Grid& g, const float* const* u, const float* const* fb, const float* dt, float nu,
                        int advect, float* const* ub0, float* const* ubin, cudaStream_t s);
int launch_adj_moments(int D, const Grid& g, const Body& b, const float* const* mbar, AdjState* as, double* part,
                       int npart, cudaStream_t s);
// the adjoint solve's V-cycle decision: continue while ||r||_inf > rtol ||b||_inf (b: the
// first residual) and fewer than maxit cycles ran; sets the WHILE node's condition
int launch_adj_decide(DevState* st, AdjState* as, cudaGraphConditionalHandle h, int use_handle, int first,
                      double rtol, int maxit, cudaStream_t s);
// recording of a recomputed step: fields src[0..nf) (nf = 1 with pl: the FP32 rounding
// ph + pl of a double-float pressure) into seg + rec_slot * stride + (off + f) * n, the
// slot read on the device, so one graph serves every slot
int launch_adj_record(const float* const* src, int nf, const float* pl, float* seg, const AdjState* as,
                      size_t stride, int off, long long n, cudaStream_t s);
int launch_adj_set_slot(AdjState* as, int slot, cudaStream_t s);
// start of an adjoint solve: the iterate (x, or the double-float pair x + xl) from the
// same projection's solution one step later (yprev), or 0 if the right-hand side is 0
int launch_adj_warm(float* x, float* xl, const float* yprev, const AdjState* as, long long n, cudaStream_t s);

}  // namespace wl

namespace wl {
int launch_set_dt_from_cfl(DevState* st, int D, double nu, double dt_cap, double dt_fixed, cudaStream_t s);
int launch_fix_bfaces(int D, const Grid& g, float* const* u, cudaStream_t s);
}  // namespace wl

namespace wl {
// ---- batched steps of many small simulations (serving): one launch of each kernel of
// the step covers every simulation of a batch.  Each simulation ("slot") keeps its own
// fields and device state; its arguments for every launch of its step sit in a device
// table of BatchSlot, built on the host with the same argument builders as its own
// step.  Block b of a batched launch belongs to slot bg.slot[s] for bg.start[s] <= b <
// bg.start[s+1] and takes the block index it would have in that slot's own launch, so
// every slot runs the same kernel bodies on the same inputs as alone (the same bits).
constexpr int kBatchMax = 64;      // simulations in one batched launch
constexpr int kBatchLevels = 8;    // multigrid levels above a slot's small-level tail
constexpr int kBatchPost = 8;      // sweeps per level
struct BatchSlot {
  DevState* ds;
  int D;
  StageArgs stage[2];              // stage 1, stage 2
  Body body;
  int band;                        // the mu1 band term runs (a body with a band box)
  int blo[3], bn[3];               // its box
  ResArgs div[2];                  // divergence of the stage output (w = 1, 1/2)
  ResArgs res;                     // fine residual of a V-cycle
  int nrestr;                      // restrictions of levels 1 .. nrestr
  ResArgs restr[kBatchLevels];
  int nsmooth;                     // levels 0 .. nsmooth-1 smoothed above the tail
  int post;                        // sweeps per level
  SweepArgs sweep[kBatchLevels][kBatchPost];
  TailArgs tail;
  CorrArgs corr[2];
  float w[2];
  double tol;
  int maxit;
  double nu, dt_cap, dt_fixed;
  double* ring;                    // metric ring (step end) of ring_cap records
  int ring_cap;
};
struct BatchGrid {
  int n;                           // slots in this launch
  int slot[kBatchMax];             // their indices in the table
  int start[kBatchMax + 1];        // first block of each (start[n] = total)
  unsigned gx[kBatchMax], gy[kBatchMax];  // each slot's own grid in x and y
};
int launch_batch_stage(int D, const BatchSlot* t, const BatchGrid& bg, int stage, cudaStream_t s);
int launch_batch_band(int D, const BatchSlot* t, const BatchGrid& bg, int stage, cudaStream_t s);
// which: 0 / 1 divergence after stage 1 / 2, 2 the fine residual (vcycle: slots whose
// projection has converged skip the launch)
int launch_batch_residual(int D, const BatchSlot* t, const BatchGrid& bg, int which, int vcycle, cudaStream_t s);
int launch_batch_restrict(int D, const BatchSlot* t, const BatchGrid& bg, int level, cudaStream_t s);
int launch_batch_tail(int D, const BatchSlot* t, const BatchGrid& bg, size_t smem, cudaStream_t s);
int launch_batch_sweep(int D, const BatchSlot* t, const BatchGrid& bg, int level, int it, cudaStream_t s);
int launch_batch_correct(int D, const BatchSlot* t, const BatchGrid& bg, int which, cudaStream_t s);
// V-cycle control of every slot (first: right after the divergence); sets h to whether
// any slot's projection continues
int launch_batch_decide(const BatchSlot* t, const BatchGrid& bg, cudaGraphConditionalHandle h, int first, int proj,
                        cudaStream_t s);
int launch_batch_step_end(const BatchSlot* t, const BatchGrid& bg, cudaStream_t s);
// grids of the single-simulation launches, for the batched ones
dim3 stage_grid(int D, const Grid& g);
dim3 band_grid(int D, const int* bn);
dim3 residual_grid(int D, const Grid& g);
dim3 restrict_grid(int D, const ResArgs& a);
dim3 sweep_grid(int D, const SweepArgs& a);
dim3 correct_grid(int D, const CorrArgs& a);
}  // namespace wl

namespace wl {
// Bounds-checked build: take (read and clear) the index-check flag word of each
// translation unit (0 in a release build).
unsigned dbg_take_momentum();
unsigned dbg_take_poisson();
unsigned dbg_take_sweep();
}  // namespace wl
