// Host runtime and C ABI of libwl.so (declared in include/wl.h).
//
// A sim owns one device workspace carved into: three velocity buffers (A: the state
// and start-of-step u0, B: stage output, C: projected predictor), the multigrid
// levels (face coefficients, right-hand side, iterate and a ping-pong iterate), the
// device-resident scalars (DevState), the coarsest-level CG vectors and the force
// partial sums.  One time step (simstep!, Section 3) is enqueued as
//   stage 1 (A -> B), project w=1 (B, corrected into C),
//   stage 2 (C, A -> B), project w=1/2 (B, corrected into A, with the CFL maximum),
//   step end (clock, next dt).
// Each projection's V-cycle loop is a CUDA-graph conditional WHILE node whose
// condition a one-thread kernel sets from the residual after every cycle, so a
// whole step runs without a host round trip.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_runtime.h>

#include <cmath>
#include <cstdio>
#include <atomic>
#include <cstdlib>
#include <cstring>
#include <string>
#include <tuple>
#include <vector>

#include "wl.h"
#include "wl_kernels.h"

using namespace wl;

namespace {

struct LevelBuf {
  Grid g;
  float* L[3];                    // face coefficients in FP32 (hierarchy construction, coarsest solve)
  float* Lk[3];                   // the coefficients the level's kernels read (storage type st)
  float* z;                       // right-hand side, iterate, ping-pong iterate (storage type st;
  float* x;                       //   a 16-bit level's pointers are reinterpreted by the kernels)
  float* x2;
  int st;                         // storage type ST_* of Lk, z, x, x2
  float zs;                       // z is stored scaled: stored = zs * value (a power of two)
  int tma_tiles, wrap_tiles;      // sweep tiles for the staged kernel / across a periodic side (table kernel)
  int wrap_tma_tiles;             // tiles across a periodic side for the staged kernel's wrapping variant
  int tzw;                        // planes per block of its launch
  BandBox band;                   // region whose coefficients may differ from uval (staged kernels)
  float uval;                     // the level's coefficient away from the body: 2^(l (D-2))
  int ty = SWEEP_TY;              // tile height of the staged sweep's plain tiles (8, or SWEEP_TY16)
  float* z32;                     // a 16-bit level 1: the restricted fine residual in FP32, converted
                                  // (with the scale DevState::cs_used) by level 1's restriction pass
  bool tma;                       // tensor maps below are valid (n_0 % 4 == 0)
  CUtensorMap mx, mx2, mz, mL[3];  // TMA descriptors of this level's fields
  CUtensorMap sz, sL[3];           // the sweep's shorter coefficient boxes
};

constexpr int kMaxLevels = 16;
constexpr long long kTailCells = 4096;  // largest hierarchy tail (cells) run by k_vcycle_tail
constexpr long long kCtailCells = 1 << 17;  // largest hierarchy tail run by one cluster (k_vcycle_ctail)
constexpr int kForceParts = 1024;
constexpr int kMetricRing = WL_METRIC_RING;

}  // namespace

struct wl_sim {
  unsigned long long uid = 0;  // unique per sim of the process (a batch keys its graphs on it)
  std::vector<size_t> canaries;  // bounds-checked build: workspace offsets of the canary gaps
  int D = 0;
  Grid g{};
  double nu = 0.0;
  Body body{};
  wl_opts o{};
  cudaStream_t st = nullptr;  // caller's stream
  cudaStream_t cs = nullptr;  // private stream used only for graph capture
  SideStream side{};          // second stream for the band tiles' launches (beside the uniform tiles)
  int nlev = 0;
  LevelBuf lev[kMaxLevels]{};
  float* ua[3]{};
  float* ub[3]{};
  float* uc[3]{};
  DevState* ds = nullptr;
  DevState* hs = nullptr;     // pinned host mirror
  double* cg_work = nullptr;
  double* fpart = nullptr;
  double* fout = nullptr;
  double* mring = nullptr;    // per-step metric records (kMetricRing x NMETRIC doubles)
  double* mforce = nullptr;   // the pressure force of the step's metrics
  float* ph = nullptr;        // precision 1: fine-level pressure as the double-float ph + pl
  float* pl = nullptr;
  CUtensorMap srf{};          // TMA descriptor of rf (sweep box)
  CUtensorMap mph{}, mpl{};   // TMA descriptors of the fine pressure (ph: hi part or FP32 pressure)
  CUtensorMap mu[3][3]{};     // TMA descriptors of the velocity buffers A, B, C (components)
  bool resid_tma = false;     // the fine residual uses the TMA-staged kernel
  float* body_nodes = nullptr;  // WL_BODY_FIELD: device copy of the sampled distance
  int tail_lf = 0;            // > 0: levels tail_lf .. nlev-1 run as one block (k_vcycle_tail)
  int ctail_lf = 0;           // > 0: levels ctail_lf .. nlev-1 run as one cluster (k_vcycle_ctail) ...
  int ctail_c = 0;            //   of ctail_c blocks
  float* rf = nullptr;        // precision 1: FP32 residual, right-hand side of each correction cycle
  double* G = nullptr;        // dense pseudo-inverse of the coarsest operator (small coarsest levels)
  char* ws = nullptr;
  size_t ws_bytes = 0;
  bool own_ws = false;
  cudaGraph_t graph = nullptr;
  cudaGraph_t vbody = nullptr;   // the first projection's V-cycle body (owned by graph)
  cudaGraphExec_t exec = nullptr;
  cudaEvent_t join = nullptr;  // wl_step_batch: end of this sim's part of a batch round
  cudaGraphConditionalHandle hc[2]{};
  bool poisoned = false;
  std::string err;
  // per-launch event pairs while wl_profile_step runs (class, start, stop)
  std::vector<std::tuple<int, cudaEvent_t, cudaEvent_t>>* prof = nullptr;
  // differentiated rollout (wl_grad_forward / wl_grad_backward)
  struct Grad {
    int nsteps = 0, every = 0, nseg = 0;
    char* mem = nullptr;
    bool own = false;
    float* ck = nullptr;       // checkpoints 0..nseg: D velocity fields + 2 pressure fields each
    DevState* ckst = nullptr;  // the device state of each checkpoint
    float* seg = nullptr;      // per step of a segment: u^n (D), u' (D), p after each projection (2)
    float* adj = nullptr;      // u' of the state (D), of u^n (D), of the predictor (D), v', f', mbar (D each), y1, y2
    double* rec = nullptr;     // force after each step (nsteps x D)
    double* gF = nullptr;      // cotangents of those forces (nsteps x D)
    AdjState* as = nullptr;
    double* part = nullptr;    // reduction partials (4 x kForceParts)
    bool ready = false;        // a forward rollout is recorded
    // the recording step (a step graph with the recording kernels) and the adjoint
    // Poisson solve of each projection (its V-cycles in a WHILE node), built for this
    // workspace
    cudaGraph_t rgraph = nullptr, sgraph[2]{};
    cudaGraphExec_t rexec = nullptr, sexec[2]{};
    cudaGraphConditionalHandle rhc[2]{}, shc[2]{};
  } gr;
};

namespace {

void free_grad_graphs(wl_sim::Grad& G);

int fail(wl_sim* s, int code, const std::string& msg) {
  if (s) s->err = msg;
  return code;
}

int cuda_check(wl_sim* s, cudaError_t e, const char* what) {
  if (e == cudaSuccess) return WL_OK;
  return fail(s, WL_ECUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

#define WL_CUDA(s, call)                                 \
  do {                                                   \
    int _rc = cuda_check((s), (call), #call);            \
    if (_rc != WL_OK) return _rc;                        \
  } while (0)

// Time one launch with a pair of events when profiling (host-driven steps only).
size_t prof_begin(wl_sim* s, cudaStream_t st, int cls) {
  cudaEvent_t a, b;
  cudaEventCreate(&a);
  cudaEventCreate(&b);
  cudaEventRecord(a, st);
  s->prof->emplace_back(cls, a, b);
  return s->prof->size() - 1;
}
void prof_end(wl_sim* s, cudaStream_t st, size_t i) { cudaEventRecord(std::get<2>((*s->prof)[i]), st); }

#define PROF(s, st, cls, call)                                 \
  do {                                                         \
    const size_t prof_i_ = (s)->prof ? prof_begin((s), (st), (cls)) : 0; \
    call;                                                      \
    if ((s)->prof) prof_end((s), (st), prof_i_);               \
  } while (0)

// The fine level's split launches (uniform tiles on the sim's stream, band tiles beside
// them on the side stream), each timed on its own stream while wl_profile_step runs.
struct ProfSplit {
  wl_sim* s;
  int cls[2];  // uniform, band
  size_t idx[2];
};
void prof_split_hook(void* ctx, int band, int begin, cudaStream_t st) {
  ProfSplit* h = static_cast<ProfSplit*>(ctx);
  if (begin)
    h->idx[band] = prof_begin(h->s, st, h->cls[band]);
  else
    prof_end(h->s, st, h->idx[band]);
}

// Multigrid levels: halve while every direction is even and larger than 4.
int plan_levels(const int* n, int D, int out[][3]) {
  int l = 0;
  int cur[3] = {n[0], n[1], D == 3 ? n[2] : 1};
  while (true) {
    for (int d = 0; d < 3; ++d) out[l][d] = cur[d];
    ++l;
    bool ok = l < kMaxLevels;
    for (int d = 0; d < D; ++d)
      if (cur[d] % 2 != 0 || cur[d] <= 4) ok = false;
    if (!ok) break;
    for (int d = 0; d < D; ++d) cur[d] /= 2;
  }
  return l;
}

// Tensor-map encoder from the driver (no link-time dependency on libcuda).
PFN_cuTensorMapEncodeTiled_v12000 tensor_map_encoder() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  static bool tried = false;
  if (!tried) {
    tried = true;
    void* f = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &f, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = (PFN_cuTensorMapEncodeTiled_v12000)f;
    else
      cudaGetLastError();
  }
  return fn;
}

// Smallest level (cells) that takes 16-row sweep tiles (WL_TY16_MIN_CELLS overrides).
long long ty16_min_cells() {
  const char* e = std::getenv("WL_TY16_MIN_CELLS");
  return e ? std::atoll(e) : (1ll << 18);
}

// Planes per block of the staged sweep on level l: whole waves of its resident blocks
// per SM (the fine level's 8-row tiles: waves of 4 of the 8, measured: 256x128x128 as
// the fine level, 1.85 -> 1.79 ms per step with twice the planes; the same grid as level
// 1 of the 512x256x256 sphere lost 0.13 ms per step with them).
int staged_sweep_tz(const LevelBuf& L, int l) {
  if (L.ty == SWEEP_TY16) {
    const char* e = std::getenv(l == 0 ? "WL_TY16_BPS0" : "WL_TY16_BPS");
    const int bps = e ? std::atoi(e) : SWEEP16_UNI_BLOCKS_PER_SM;
    const long long tiles = (long long)((L.g.n[0] + SWEEP_TX - 1) / SWEEP_TX) * (L.g.n[1] / SWEEP_TY16);
    return sweep_planes_for_columns(L.g.n[2], tiles, bps > 0 ? bps : SWEEP16_UNI_BLOCKS_PER_SM);
  }
  const int bps = L.band.on ? (l == 0 ? SWEEP_UNI_BLOCKS_PER_SM / 2 : SWEEP_UNI_BLOCKS_PER_SM) : SWEEP_BLOCKS_PER_SM;
  return sweep_planes_per_block(L.g, bps);
}

// Box of 72 x rows [x 1] floats over a level field (x fastest), zero fill out of
// range.  Needs n_0 % 4 == 0 (16-byte row pitch) and a 16-byte aligned base.
bool make_field_map(CUtensorMap* m, const float* ptr, const Grid& g, int D, int rows = SWEEP_TY + 4) {
  auto enc = tensor_map_encoder();
  if (!enc || g.n[0] % 4 != 0 || ((uintptr_t)ptr & 15u)) return false;
  cuuint64_t dims[3] = {(cuuint64_t)g.n[0], (cuuint64_t)g.n[1], (cuuint64_t)g.n[2]};
  cuuint64_t strides[2] = {(cuuint64_t)g.n[0] * 4, (cuuint64_t)g.n[0] * g.n[1] * 4};
  cuuint32_t box[3] = {(cuuint32_t)(SWEEP_TX + 8), (cuuint32_t)rows, 1};
  cuuint32_t es[3] = {1, 1, 1};
  CUresult r = enc(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, (cuuint32_t)D, (void*)ptr, dims, strides, box, es,
                   CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                   CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS;
}

// Carves the workspace into 256-byte aligned arrays.  The bounds-checked build leaves a
// 256-byte canary after every array (filled with 0xA5 at creation and checked by
// wl_debug_bounds), so a write past an array's end shows up there.
#ifdef WL_DEBUG_BOUNDS
constexpr size_t kCanary = 256;
#else
constexpr size_t kCanary = 0;
#endif
struct Carver {
  char* base;
  size_t off = 0;
  std::vector<size_t>* canaries = nullptr;
  void* take(size_t bytes) {
    off = (off + 255) & ~size_t(255);
    void* p = base ? base + off : nullptr;
    off += bytes;
    if (kCanary) {
      off = (off + 255) & ~size_t(255);
      if (canaries) canaries->push_back(off);
      off += kCanary;
    }
    return p;
  }
};

// Walks the workspace layout; with base == nullptr only measures it.
// Storage type of level l: the coarse levels between the fine and the coarsest one
// take wl_opts.coarse_precision (FP32 arithmetic on 16-bit values); the fine and the
// coarsest level stay FP32.
int level_storage(int l, int nlev, int cprec) { return (l >= 1 && l + 1 < nlev) ? cprec : ST_F32; }
size_t esize(int st) { return st == ST_F32 ? sizeof(float) : 2; }

size_t layout(wl_sim* s, int D, const int* dims, int precision, int cprec, int exit_bc, char* base) {
  int ld[kMaxLevels][3];
  const int nlev = plan_levels(dims, D, ld);
  Carver cv{base};
  if (s && base) {
    s->canaries.clear();
    cv.canaries = &s->canaries;
  }
  const long long nc = (long long)ld[0][0] * ld[0][1] * ld[0][2];
  const long long ne = exit_bc ? (long long)ld[0][1] * ld[0][2] : 0;  // exit plane after u_x
  float** bufs[3] = {s ? s->ua : nullptr, s ? s->ub : nullptr, s ? s->uc : nullptr};
  for (int b = 0; b < 3; ++b)
    for (int c = 0; c < D; ++c) {
      void* p = cv.take(sizeof(float) * (nc + (c == 0 ? ne : 0)));
      if (s) bufs[b][c] = (float*)p;
    }
  for (int l = 0; l < nlev; ++l) {
    const long long n = (long long)ld[l][0] * ld[l][1] * ld[l][2];
    const int st = level_storage(l, nlev, cprec);
    for (int c = 0; c < D; ++c) {
      void* p = cv.take(sizeof(float) * n);
      void* pk = st == ST_F32 ? p : cv.take(esize(st) * n);
      if (s) {
        s->lev[l].L[c] = (float*)p;
        s->lev[l].Lk[c] = (float*)pk;
      }
    }
    void* z = cv.take(esize(st) * n);
    void* x = cv.take(esize(st) * n);
    void* x2 = cv.take(esize(st) * n);
    void* z32 = (l == 1 && st != ST_F32) ? cv.take(sizeof(float) * n) : nullptr;
    if (s) {
      s->lev[l].z32 = (float*)z32;
      s->lev[l].z = (float*)z;
      s->lev[l].x = (float*)x;
      s->lev[l].x2 = (float*)x2;
      s->lev[l].st = st;
      // a 16-bit level holds the mean rather than the sum of its 2^(D l) fine cells
      s->lev[l].zs = st == ST_F32 ? 1.f : ldexpf(1.f, -D * l);
    }
  }
  void* ds = cv.take(sizeof(DevState));
  const long long ncoarse = (long long)ld[nlev - 1][0] * ld[nlev - 1][1] * ld[nlev - 1][2];
  void* cg = cv.take(sizeof(double) * 5 * ncoarse);
  void* fp = cv.take(sizeof(double) * 2 * kForceParts);
  void* fo = cv.take(sizeof(double) * 4);
  void* mr = cv.take(sizeof(double) * NMETRIC * kMetricRing);
  void* mf = cv.take(sizeof(double) * 4);
  void* ph = precision == 1 ? cv.take(sizeof(float) * nc) : nullptr;
  void* pl = precision == 1 ? cv.take(sizeof(float) * nc) : nullptr;
  void* rf = precision == 1 ? cv.take(sizeof(float) * nc) : nullptr;
  void* G = ncoarse <= kDenseCoarse ? cv.take(sizeof(double) * ncoarse * ncoarse) : nullptr;
  if (s) {
    s->ds = (DevState*)ds;
    s->cg_work = (double*)cg;
    s->fpart = (double*)fp;
    s->fout = (double*)fo;
    s->mring = (double*)mr;
    s->mforce = (double*)mf;
    s->ph = (float*)ph;
    s->pl = (float*)pl;
    s->rf = (float*)rf;
    s->G = (double*)G;
    s->nlev = nlev;
    for (int l = 0; l < nlev; ++l) {
      Grid& g = s->lev[l].g;
      g = s->g;
      for (int d = 0; d < 3; ++d) g.n[d] = ld[l][d];
      g.nc = (long long)ld[l][0] * ld[l][1] * ld[l][2];
    }
    for (int b = 0; b < 3; ++b)
      for (int c = D; c < 3; ++c) bufs[b][c] = bufs[b][D - 1];  // 2-D: unused slot aliases a valid pointer
    for (int l = 0; l < nlev; ++l)
      for (int c = D; c < 3; ++c) {
        s->lev[l].L[c] = s->lev[l].L[D - 1];
        s->lev[l].Lk[c] = s->lev[l].Lk[D - 1];
      }
  }
  return cv.off;
}

// ------------------------------------------------------------------- enqueue helpers
const SideStream* side_of(wl_sim* s) { return s->side.aux ? &s->side : nullptr; }

StageArgs stage_args(wl_sim* s, int stage) {
  StageArgs a{};
  for (int c = 0; c < 3; ++c) {
    a.u[c] = stage == 1 ? s->ua[c] : s->uc[c];
    a.u0[c] = s->ua[c];
    a.mu0[c] = s->lev[0].L[c];
    a.out[c] = s->ub[c];
  }
  a.g = s->g;
  a.dt = &s->ds->dtf;
  a.nu = (float)s->nu;
  a.stage = stage;
  a.advect = s->o.advect;
  if (s->D == 3) a.tz = stage3_planes(s->g);
  // f of the body's band box goes to the fine level's ping-pong iterate, which is free
  // until the projection's sweeps
  int lo[3], hi[3];
  if (stage_band_box(s->D, s->g, s->body, lo, hi)) {
    const long long vol = (long long)(hi[0] - lo[0]) * (hi[1] - lo[1]) * (hi[2] - lo[2]);
    if (vol * s->D <= s->g.nc) {
      a.fbox = s->lev[0].x2;
      for (int d = 0; d < 3; ++d) {
        a.blo[d] = lo[d];
        a.bn[d] = hi[d] - lo[d];
      }
    }
  }
  return a;
}

void enq_stage(wl_sim* s, int stage, cudaStream_t st) {
  const StageArgs a = stage_args(s, stage);
  PROF(s, st, WL_KCLASS_STAGE, launch_stage(s->D, a, st));
  if (s->g.exit) PROF(s, st, WL_KCLASS_STAGE, launch_exit_stage(s->D, s->g, s->ua[0], a.u[0], s->ub[0], a.dt, stage, st));
  if (s->body.kind != 0) PROF(s, st, WL_KCLASS_BAND, launch_band(s->D, a, s->body, st));
}

ResArgs res_args(wl_sim* s, int l, int mode) {
  ResArgs a{};
  const LevelBuf& L = s->lev[l];
  for (int c = 0; c < 3; ++c) a.L[c] = L.Lk[c];
  // no body: the band box is empty and every coefficient is the level's free-stream value
  a.uni = (L.band.on && L.band.lo[0] >= L.band.hi[0]) ? 1 : 0;
  a.uval = L.uval;
  a.x = L.x;
  a.z = L.z;
  a.zc = (l + 1 < s->nlev) ? s->lev[l + 1].z : nullptr;
  a.g = L.g;
  a.ztype = L.st;
  a.zctype = ST_F32;
  a.zcmul = 1.f;
  if (l + 1 < s->nlev) {
    for (int d = 0; d < 3; ++d) a.cn[d] = s->lev[l + 1].g.n[d];
    if (l == 0 && s->lev[1].z32) {
      a.zc = s->lev[1].z32;  // the fine level restricts into level 1's FP32 staging field
    } else {
      a.zctype = s->lev[l + 1].st;
      a.zcmul = s->lev[l + 1].zs / L.zs;
    }
  }
  if (L.z32) {
    // level 1's pass reads the FP32 restricted residual, stores its 16-bit copy and
    // restricts further, both with the scale 2^cs_used chosen from the fine residual
    a.z = L.z32;
    a.ztype = ST_F32;
    a.zconv = L.z;
    a.zconvtype = L.st;
    a.zconvmul = L.zs;
    a.zcmul = (l + 1 < s->nlev) ? s->lev[l + 1].zs : 1.f;
    a.apply_cs = 1;
  }
  a.inv_w = 1.f;
  a.st = s->ds;
  a.mode = mode;
  return a;
}

// arguments of the index-table kernel k_residual for the fine level (mode RES_RESIDUAL,
// or RES_DIVERGENCE of velocity buffer `ubuf` 0/1/2 = A/B/C with weight w)
ResArgs fine_res_args(wl_sim* s, int mode, int ubuf, float w) {
  ResArgs a = res_args(s, 0, mode);
  float* const* ub[3] = {s->ua, s->ub, s->uc};
  if (mode == RES_DIVERGENCE)
    for (int c = 0; c < 3; ++c) a.u[c] = ub[ubuf][c];
  a.inv_w = 1.f / w;
  a.ph = s->ph;
  a.pl = s->pl;
  a.rout = s->rf;
  return a;
}

// fine-level residual (mode RES_RESIDUAL) or divergence + residual (RES_DIVERGENCE,
// of velocity buffer `ubuf` 0/1/2 = A/B/C), with the restriction and the max-norm
void enq_fine_residual(wl_sim* s, int mode, int ubuf, float w, cudaStream_t st) {
  const LevelBuf& L = s->lev[0];
  if (s->resid_tma) {
    ResidMaps m{};
    m.ph = s->mph;
    m.pl = s->mpl;
    m.z = L.mz;
    m.L0 = L.mL[0];
    m.L1 = L.mL[1];
    m.L2 = L.mL[2];
    if (mode == RES_DIVERGENCE) {
      m.u0 = s->mu[ubuf][0];
      m.u1 = s->mu[ubuf][1];
      m.u2 = s->mu[ubuf][2];
    }
    ResidTmaArgs t{};
    t.div = mode == RES_DIVERGENCE;
    t.df = s->ph != nullptr;
    t.z = L.z;
    t.rout = s->rf;
    t.zc = (s->nlev > 1) ? s->lev[1].z : nullptr;
    t.g = L.g;
    t.zctype = ST_F32;
    t.zcmul = 1.f;
    if (s->nlev > 1) {
      for (int d = 0; d < 3; ++d) t.cn[d] = s->lev[1].g.n[d];
      if (s->lev[1].z32) t.zc = s->lev[1].z32;  // FP32 staging of a 16-bit level 1
    }
    const int tz = sweep_planes_per_block(L.g, L.band.on ? RESID_UNI_WAVE_BLOCKS : SWEEP_BLOCKS_PER_SM);
    t.tz = tz + (tz & 1);
    t.inv_w = 1.f / w;
    t.st = s->ds;
    t.band = L.band;
    float* const* ub[3] = {s->ua, s->ub, s->uc};
    if (s->g.exit && mode == RES_DIVERGENCE) t.uxe = ub[ubuf][0] + s->g.nc;
    t.wsrc[0] = s->ph ? s->ph : L.x;
    t.wsrc[1] = s->pl;
    if (mode == RES_DIVERGENCE) {
      t.wsrc[2] = ub[ubuf][0];
      t.wsrc[3] = ub[ubuf][1];
    }
    ProfSplit ps{s, {WL_KCLASS_RESID_FINE_UNI, WL_KCLASS_RESID_FINE_BANDT}, {0, 0}};
    SideStream sp = s->side;
    sp.hook = prof_split_hook;
    sp.ctx = &ps;
    PROF(s, st, WL_KCLASS_RESID_FINE, launch_resid_tma(m, t, st, (s->prof && side_of(s)) ? &sp : side_of(s)));
    return;
  }
  PROF(s, st, WL_KCLASS_RESID_FINE, launch_residual(s->D, fine_res_args(s, mode, ubuf, w), st));
}

// divergence of u (scaled by 1/(w dt)), first residual, restriction, first decision
void enq_proj_head(wl_sim* s, int ubuf, float w, int proj, cudaStream_t st, int use_h) {
  enq_fine_residual(s, RES_DIVERGENCE, ubuf, w, st);
  PROF(s, st, WL_KCLASS_CONTROL, launch_decide(s->ds, s->hc[proj], use_h, 1, proj, w, s->o.tol, s->o.max_vcycles, st));
}

// the index-table kernel's arguments of sweep `it` of level l, as enq_smooth forms them
// (the same buffers, coarse correction and double-float store)
SweepArgs smooth_args(wl_sim* s, int l, int it) {
  LevelBuf& L = s->lev[l];
  const int P = s->o.post;
  const bool refine = (l == 0 && s->ph);
  SweepArgs a{};
  for (int c = 0; c < 3; ++c) a.L[c] = L.Lk[c];
  a.z = refine ? s->rf : L.z;
  a.g = L.g;
  for (int d = 0; d < 3; ++d) a.cn[d] = s->lev[l + 1].g.n[d];
  a.stype = L.st;
  a.xctype = s->lev[l + 1].st;
  a.zmul = 1.f / L.zs;
  if (l == 0 && s->lev[1].z32) a.cs = s->ds;
  a.tz = sweep_planes_per_block(L.g, sweep_table_blocks_per_sm(s->D, L.st));
  a.uni = (L.band.on && L.band.lo[0] >= L.band.hi[0]) ? 1 : 0;
  a.uval = L.uval;
  float* bufs[2] = {L.x, L.x2};
  const bool from_x = (l == 0 && !refine);
  int out = from_x ? 1 : ((P % 2 == 1) ? 0 : 1);
  int in = from_x ? 0 : -1;
  for (int k = 0; k < it; ++k) {
    in = out;
    out ^= 1;
  }
  a.x_in = in >= 0 ? bufs[in] : nullptr;
  a.xc = (it == 0) ? s->lev[l + 1].x : nullptr;
  a.x_out = bufs[out];
  a.ph = (refine && it == P - 1) ? s->ph : nullptr;
  a.pl = (refine && it == P - 1) ? s->pl : nullptr;
  a.only_wrapping = 0;
  return a;
}

// post sweeps on level l with the coarse correction of level l+1 prolonged into the
// first one.  Coarse levels start from zero and end in lev[l].x.  The fine level
// either smooths the FP32 pressure in place of the iterate (precision 0), or smooths
// a correction from zero against the residual rf and adds the result of the last
// sweep into the FP64 pressure (precision 1, iterative refinement).
void enq_smooth(wl_sim* s, int l, cudaStream_t st) {
  LevelBuf& L = s->lev[l];
  const int P = s->o.post;
  const bool refine = (l == 0 && s->ph);
  SweepArgs a{};
  for (int c = 0; c < 3; ++c) a.L[c] = L.Lk[c];
  a.z = refine ? s->rf : L.z;
  a.g = L.g;
  for (int d = 0; d < 3; ++d) a.cn[d] = s->lev[l + 1].g.n[d];
  a.stype = L.st;
  a.xctype = s->lev[l + 1].st;
  a.zmul = 1.f / L.zs;
  // the coarse levels' values carry the factor 2^cs_used; the fine level removes it
  if (l == 0 && s->lev[1].z32) a.cs = s->ds;
  // z-blocking for each kernel's own residency: the table kernel (tiles across a periodic
  // side, 16-bit levels) and the staged one (uniform or loading variant)
  a.tz = sweep_planes_per_block(L.g, sweep_table_blocks_per_sm(s->D, L.st));
  // planes per block of the staged sweep (whole waves of its resident blocks)
  const int tz_staged = staged_sweep_tz(L, l);
  // no body: the band box is empty and every coefficient is the level's free-stream value
  a.uni = (L.band.on && L.band.lo[0] >= L.band.hi[0]) ? 1 : 0;
  a.uval = L.uval;
  float* bufs[2] = {L.x, L.x2};
  const CUtensorMap* bmaps[2] = {&L.mx, &L.mx2};
  const bool from_x = (l == 0 && !refine);  // precision 0: the fine iterate is the pressure itself
  // choose the first output so that the last one lands in bufs[0]
  int out = from_x ? 1 : ((P % 2 == 1) ? 0 : 1);
  int in = from_x ? 0 : -1;
  for (int it = 0; it < P; ++it) {
    a.x_in = in >= 0 ? bufs[in] : nullptr;
    a.xc = (it == 0) ? s->lev[l + 1].x : nullptr;
    a.x_out = bufs[out];
    a.ph = (refine && it == P - 1) ? s->ph : nullptr;
    a.pl = (refine && it == P - 1) ? s->pl : nullptr;
    if (L.tma && (L.tma_tiles > 0 || L.wrap_tma_tiles > 0)) {
      SweepMaps m;
      m.x = in >= 0 ? *bmaps[in] : L.mx;
      m.z = refine ? s->srf : L.sz;
      m.L0 = L.sL[0];
      m.L1 = L.sL[1];
      m.L2 = L.sL[s->D == 3 ? 2 : 0];
      SweepTmaArgs t{};
      t.has_x = in >= 0;
      t.xc = a.xc;
      t.xctype = a.xctype;
      t.xc_cs = a.cs != nullptr;
      t.band = L.band;
      t.uval = L.uval;
      t.x_out = a.x_out;
      t.ph = a.ph;
      t.pl = a.pl;
      t.g = a.g;
      for (int d = 0; d < 3; ++d) t.cn[d] = a.cn[d];
      t.tz = tz_staged;
      t.st = s->ds;
      t.plain = L.tma_tiles > 0;
      t.wrap = L.wrap_tma_tiles > 0;
      t.xsrc = a.x_in;
      t.zsrc = refine ? s->rf : L.z;
      t.tzw = L.tzw;
      t.ty = L.ty;
      ProfSplit ps{s, {WL_KCLASS_SWEEP_FINE_UNI, WL_KCLASS_SWEEP_FINE_BANDT}, {0, 0}};
      SideStream sp = s->side;
      sp.hook = prof_split_hook;
      sp.ctx = &ps;
      const SideStream* sd = (s->prof && l == 0 && side_of(s)) ? &sp : side_of(s);
      PROF(s, st, l == 0 ? WL_KCLASS_SWEEP_FINE : WL_KCLASS_SWEEP_COARSE, launch_sweep_tma(s->D, m, t, st, sd));
      a.only_wrapping = 1;  // tiles crossing a periodic side
      if (L.wrap_tiles > 0) PROF(s, st, l == 0 ? WL_KCLASS_SWEEP_FINE : WL_KCLASS_SWEEP_COARSE, launch_sweep(s->D, a, st));
    } else {
      a.only_wrapping = 0;
      PROF(s, st, l == 0 ? WL_KCLASS_SWEEP_FINE : WL_KCLASS_SWEEP_COARSE, launch_sweep(s->D, a, st));
    }
    in = out;
    out ^= 1;
  }
  if (!refine && in != 0) cudaMemcpyAsync(L.x, bufs[in], esize(L.st) * L.g.nc, cudaMemcpyDeviceToDevice, st);
}

// coarsest solve of level l: x = A^+ z (dense FP64 pseudo-inverse when small, FP64 CG otherwise)
void enq_coarsest(wl_sim* s, int l, const float* z, float* x, cudaStream_t st) {
  LevelBuf& L = s->lev[l];
  if (s->G && l == s->nlev - 1) {
    DenseArgs d{};
    for (int c = 0; c < 3; ++c) d.L[c] = L.L[c];
    d.g = L.g;
    d.G = s->G;
    d.z = z;
    d.x = x;
    PROF(s, st, WL_KCLASS_COARSEST, launch_apply_pinv(d, st));
    return;
  }
  CoarseArgs a{};
  a.z = z;
  for (int c = 0; c < 3; ++c) a.L[c] = L.L[c];
  a.x = x;
  a.g = L.g;
  a.work = s->cg_work;
  a.maxit = (int)std::min<long long>(4 * L.g.nc + 100, 100000);
  a.rtol = 1e-12;
  PROF(s, st, WL_KCLASS_COARSEST, launch_coarse(s->D, a, st));
}

// the coarse end of a V-cycle (levels lf .. nlev-1) in one block or one cluster
TailArgs tail_args(wl_sim* s, int lf) {
  TailArgs t{};
  t.nl = s->nlev - lf;
  for (int l = 0; l < t.nl; ++l) {
    const LevelBuf& L = s->lev[lf + l];
    for (int d = 0; d < 3; ++d) t.n[l][d] = L.g.n[d];
    for (int c = 0; c < 3; ++c) t.L[l][c] = L.Lk[c];
    t.st[l] = L.st;
  }
  t.z = s->lev[lf].z;
  t.zmul = 1.f / s->lev[lf].zs;
  t.x = s->lev[lf].x;
  t.G = s->G;
  t.post = s->o.post;
  t.per = s->g.per;
  return t;
}

// restriction down the coarse levels, coarsest solve, prolongation + smoothing up to
// the fine level (whose right-hand side and restricted residual are already set)
void enq_vcycle_core(wl_sim* s, cudaStream_t st) {
  const int Lv = s->nlev;
  if (Lv == 1) {  // no coarse level: solve the fine level directly
    if (s->ph) {
      enq_coarsest(s, 0, s->rf, s->lev[0].x2, st);
      launch_df_add(s->ph, s->pl, s->lev[0].x2, s->g.nc, st);
    } else {
      enq_coarsest(s, 0, s->lev[0].z, s->lev[0].x, st);
    }
    return;
  }
  if (s->ctail_lf > 0) {  // the coarse levels in one cluster
    const int lf = s->ctail_lf;
    for (int l = 1; l < lf; ++l) PROF(s, st, WL_KCLASS_RESTRICT, launch_residual(s->D, res_args(s, l, RES_RESTRICT), st));
    PROF(s, st, WL_KCLASS_SWEEP_COARSE, launch_vcycle_ctail(s->D, tail_args(s, lf), s->ctail_c, st));
    for (int l = lf - 1; l >= 0; --l) enq_smooth(s, l, st);
    return;
  }
  if (s->tail_lf > 0) {  // the small levels in one block
    const int lf = s->tail_lf;
    for (int l = 1; l < lf; ++l) PROF(s, st, WL_KCLASS_RESTRICT, launch_residual(s->D, res_args(s, l, RES_RESTRICT), st));
    PROF(s, st, WL_KCLASS_SWEEP_COARSE, launch_vcycle_tail(s->D, tail_args(s, lf), st));
    for (int l = lf - 1; l >= 0; --l) enq_smooth(s, l, st);
    return;
  }
  for (int l = 1; l + 1 < Lv; ++l) PROF(s, st, WL_KCLASS_RESTRICT, launch_residual(s->D, res_args(s, l, RES_RESTRICT), st));
  enq_coarsest(s, Lv - 1, s->lev[Lv - 1].z, s->lev[Lv - 1].x, st);
  for (int l = Lv - 2; l >= 0; --l) enq_smooth(s, l, st);
}

void enq_vcycle(wl_sim* s, float w, int proj, cudaStream_t st, int use_h) {
  enq_vcycle_core(s, st);
  enq_fine_residual(s, RES_RESIDUAL, 0, 1.f, st);
  PROF(s, st, WL_KCLASS_CONTROL, launch_decide(s->ds, s->hc[proj], use_h, 0, proj, w, s->o.tol, s->o.max_vcycles, st));
}

CorrArgs corr_args(wl_sim* s, float* const* uin, float* const* uout, float w, int cfl) {
  CorrArgs a{};
  for (int c = 0; c < 3; ++c) {
    a.u_in[c] = uin[c];
    a.u_out[c] = uout[c];
    a.L[c] = s->lev[0].L[c];
  }
  a.x = s->lev[0].x;
  a.ph = s->ph;
  a.pl = s->pl;
  a.g = s->g;
  a.w = w;
  a.cfl = cfl;
  a.st = s->ds;
  return a;
}

void enq_correct(wl_sim* s, float* const* uin, float* const* uout, float w, int cfl, cudaStream_t st) {
  PROF(s, st, WL_KCLASS_CORRECT, launch_correct(s->D, corr_args(s, uin, uout, w, cfl), st));
  if (s->g.exit && uout[0] != uin[0])  // the exit plane is not corrected: carry it over
    cudaMemcpyAsync(uout[0] + s->g.nc, uin[0] + s->g.nc, sizeof(float) * (size_t)s->g.n[1] * s->g.n[2],
                    cudaMemcpyDeviceToDevice, st);
}

// End of a step: with wl_opts.metrics the end-of-step velocity's kinetic energy and
// max |div u| and the pressure force go into the step's metric record; then the clock,
// the record and the next dt.
void enq_step_end(wl_sim* s, cudaStream_t st) {
  if (s->o.metrics) {
    const float* u[3] = {s->ua[0], s->ua[1], s->ua[2]};
    PROF(s, st, WL_KCLASS_CONTROL, launch_metrics_u(s->D, s->g, u, s->ds, s->fpart, kForceParts, st));
    if (s->body.kind != 0) {
      const float* L[3] = {s->lev[0].L[0], s->lev[0].L[1], s->lev[0].L[2]};
      PROF(s, st, WL_KCLASS_CONTROL,
           launch_forces(s->D, s->g, s->body, s->ph ? s->ph : s->lev[0].x, s->pl, L, s->fpart, kForceParts,
                         s->mforce, st));
    }
  }
  PROF(s, st, WL_KCLASS_CONTROL,
       launch_step_end(s->ds, s->D, s->nu, s->o.dt_cap, s->o.dt_fixed, s->mring, kMetricRing,
                       s->o.metrics ? s->mforce : nullptr, st));
}

int sync_state(wl_sim* s) {
  WL_CUDA(s, cudaMemcpyAsync(s->hs, s->ds, sizeof(DevState), cudaMemcpyDeviceToHost, s->st));
  WL_CUDA(s, cudaStreamSynchronize(s->st));
  return WL_OK;
}

// projection loop driven from the host (used outside graphs)
int host_projection(wl_sim* s, int ubuf, float w, int proj) {
  enq_proj_head(s, ubuf, w, proj, s->st, 0);
  int rc = sync_state(s);
  if (rc) return rc;
  while (s->hs->cond) {
    enq_vcycle(s, w, proj, s->st, 0);
    rc = sync_state(s);
    if (rc) return rc;
  }
  return WL_OK;
}

// FP32 copy of the fine-level pressure into dst
void copy_pressure(wl_sim* s, float* dst, cudaStream_t st) {
  if (s->ph)
    launch_df_round(s->ph, s->pl, dst, s->g.nc, st);
  else
    cudaMemcpyAsync(dst, s->lev[0].x, sizeof(float) * s->g.nc, cudaMemcpyDeviceToDevice, st);
}

// What the adjoint of a step keeps, in the segment slot the gradient state names:
// u^n (D fields, offset 0), u' (D fields, offset D) and the FP32 pressure after each
// projection (offsets 2D and 2D+1).
enum { REC_UN = 0, REC_UP = 1, REC_P1 = 2, REC_P2 = 3 };
void enq_record(wl_sim* s, int what, cudaStream_t st) {
  const int D = s->D;
  const long long n = s->g.nc;
  const size_t stride = (size_t)(2 * D + 2) * (size_t)n;
  if (what == REC_UN || what == REC_UP) {
    launch_adj_record(what == REC_UN ? s->ua : s->uc, D, nullptr, s->gr.seg, s->gr.as, stride,
                      what == REC_UN ? 0 : D, n, st);
    return;
  }
  const float* src[1] = {s->ph ? s->ph : s->lev[0].x};
  launch_adj_record(src, 1, s->ph ? s->pl : nullptr, s->gr.seg, s->gr.as, stride, 2 * D + (what == REC_P2 ? 1 : 0),
                    n, st);
}

// One step through the host-driven sequence; record: keep what the adjoint of the step
// needs (enq_record).
int host_step(wl_sim* s, bool record = false) {
  if (record) enq_record(s, REC_UN, s->st);
  enq_stage(s, 1, s->st);
  int rc = host_projection(s, 1, 1.f, 0);
  if (rc) return rc;
  if (record) enq_record(s, REC_P1, s->st);
  enq_correct(s, s->ub, s->uc, 1.f, 0, s->st);
  if (record) enq_record(s, REC_UP, s->st);
  enq_stage(s, 2, s->st);
  rc = host_projection(s, 1, 0.5f, 1);
  if (rc) return rc;
  if (record) enq_record(s, REC_P2, s->st);
  enq_correct(s, s->ub, s->ua, 0.5f, 1, s->st);
  enq_step_end(s, s->st);
  return cuda_check(s, cudaGetLastError(), "step launch");
}

int capture_leaf(wl_sim* s, std::vector<cudaGraphNode_t>& leaf) {
  cudaStreamCaptureStatus cst;
  const cudaGraphNode_t* deps = nullptr;
  size_t nd = 0;
  WL_CUDA(s, cudaStreamGetCaptureInfo(s->cs, &cst, nullptr, nullptr, &deps, nullptr, &nd));
  leaf.assign(deps, deps + nd);
  return WL_OK;
}

// A WHILE node after deps whose body is one V-cycle and its decision (the captured
// enq_vcycle, which sets the condition through s->hc[proj]); returns the body graph.
int add_while(wl_sim* s, cudaGraph_t g, const std::vector<cudaGraphNode_t>& deps, int proj, float w,
              cudaGraphNode_t* node, cudaGraph_t* body_out = nullptr) {
  cudaGraphNodeParams cp{};
  cp.type = cudaGraphNodeTypeConditional;
  cp.conditional.handle = s->hc[proj];
  cp.conditional.type = cudaGraphCondTypeWhile;
  cp.conditional.size = 1;
  WL_CUDA(s, cudaGraphAddNode(node, g, deps.data(), nullptr, deps.size(), &cp));
  cudaGraph_t body = cp.conditional.phGraph_out[0];
  if (body_out) *body_out = body;
  WL_CUDA(s, cudaStreamBeginCaptureToGraph(s->cs, body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal));
  enq_vcycle(s, w, proj, s->cs, 1);
  cudaGraph_t out = nullptr;
  WL_CUDA(s, cudaStreamEndCapture(s->cs, &out));
  return WL_OK;
}

// One step as a graph: three captured segments joined by two WHILE nodes.  record: the
// step that also keeps what its adjoint needs (enq_record), with its own condition handles
// (the captured decisions address s->hc, which holds them while this graph is built).
int build_step_graph_into(wl_sim* s, bool record, cudaGraph_t* gout, cudaGraphExec_t* eout,
                          cudaGraphConditionalHandle* hcs) {
  cudaGraph_t g = nullptr;
  WL_CUDA(s, cudaGraphCreate(&g, 0));
  *gout = g;
  for (int p = 0; p < 2; ++p) WL_CUDA(s, cudaGraphConditionalHandleCreate(&hcs[p], g, 0, 0));
  const cudaGraphConditionalHandle keep[2] = {s->hc[0], s->hc[1]};
  s->hc[0] = hcs[0];
  s->hc[1] = hcs[1];
  std::vector<cudaGraphNode_t> leaf;
  cudaGraph_t out = nullptr;
  cudaGraphNode_t w1, w2;
  int rc = WL_OK;
  do {
    // segment 1: stage 1, divergence + first residual
    rc = cuda_check(s, cudaStreamBeginCaptureToGraph(s->cs, g, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal),
                    "capture");
    if (rc) break;
    if (record) enq_record(s, REC_UN, s->cs);
    enq_stage(s, 1, s->cs);
    enq_proj_head(s, 1, 1.f, 0, s->cs, 1);
    rc = capture_leaf(s, leaf);
    const int rc2 = cuda_check(s, cudaStreamEndCapture(s->cs, &out), "capture");
    if (rc || (rc = rc2)) break;
    cudaGraph_t body = nullptr;
    if ((rc = add_while(s, g, leaf, 0, 1.f, &w1, &body))) break;
    if (!record) s->vbody = body;
    // segment 2: correction, stage 2, divergence + first residual
    rc = cuda_check(s, cudaStreamBeginCaptureToGraph(s->cs, g, &w1, nullptr, 1, cudaStreamCaptureModeThreadLocal),
                    "capture");
    if (rc) break;
    if (record) enq_record(s, REC_P1, s->cs);
    enq_correct(s, s->ub, s->uc, 1.f, 0, s->cs);
    if (record) enq_record(s, REC_UP, s->cs);
    enq_stage(s, 2, s->cs);
    enq_proj_head(s, 1, 0.5f, 1, s->cs, 1);
    rc = capture_leaf(s, leaf);
    const int rc3 = cuda_check(s, cudaStreamEndCapture(s->cs, &out), "capture");
    if (rc || (rc = rc3)) break;
    if ((rc = add_while(s, g, leaf, 1, 0.5f, &w2))) break;
    // segment 3: correction with the CFL maximum, step end
    rc = cuda_check(s, cudaStreamBeginCaptureToGraph(s->cs, g, &w2, nullptr, 1, cudaStreamCaptureModeThreadLocal),
                    "capture");
    if (rc) break;
    if (record) enq_record(s, REC_P2, s->cs);
    enq_correct(s, s->ub, s->ua, 0.5f, 1, s->cs);
    enq_step_end(s, s->cs);
    if ((rc = cuda_check(s, cudaStreamEndCapture(s->cs, &out), "capture"))) break;
    rc = cuda_check(s, cudaGraphInstantiate(eout, g, 0), "graph instantiate");
  } while (false);
  if (!record) {
    s->hc[0] = hcs[0];
    s->hc[1] = hcs[1];
  } else {
    s->hc[0] = keep[0];
    s->hc[1] = keep[1];
  }
  return rc;
}

int build_step_graph(wl_sim* s) {
  cudaGraphConditionalHandle h[2]{};
  return build_step_graph_into(s, false, &s->graph, &s->exec, h);
}

int set_dt_from_ic(wl_sim* s) {
  const float* u[3] = {s->ua[0], s->ua[1], s->ua[2]};
  launch_cfl_only(s->D, s->g, u, s->ds, s->st);
  launch_set_dt_from_cfl(s->ds, s->D, s->nu, s->o.dt_cap, s->o.dt_fixed, s->st);
  return cuda_check(s, cudaGetLastError(), "initial dt");
}

int reset_state(wl_sim* s) {
  WL_CUDA(s, cudaMemsetAsync(s->ds, 0, sizeof(DevState), s->st));
  WL_CUDA(s, cudaMemsetAsync(s->lev[0].x, 0, sizeof(float) * s->g.nc, s->st));
  if (s->ph) WL_CUDA(s, cudaMemsetAsync(s->ph, 0, sizeof(float) * s->g.nc, s->st));
  if (s->pl) WL_CUDA(s, cudaMemsetAsync(s->pl, 0, sizeof(float) * s->g.nc, s->st));
  return WL_OK;
}

bool valid_field(int which) { return which >= WL_FIELD_U && which <= WL_FIELD_EXIT; }

// the three velocity buffers' exit planes start at the free stream
void init_exit(wl_sim* s) {
  if (!s->g.exit) return;
  const long long ne = (long long)s->g.n[1] * s->g.n[2];
  launch_fill(s->ua[0] + s->g.nc, ne, s->g.U[0], s->st);
  launch_fill(s->ub[0] + s->g.nc, ne, s->g.U[0], s->st);
  launch_fill(s->uc[0] + s->g.nc, ne, s->g.U[0], s->st);
}

}  // namespace

// =========================================================================== C ABI
extern "C" {

void wl_default_opts(wl_opts* o) {
  if (!o) return;
  std::memset(o, 0, sizeof(*o));
  o->tol = 1e-6;
  o->max_vcycles = 32;
  o->post = 4;
  o->eps = 1.0;
  o->dt_cap = 10.0;
  o->dt_fixed = 0.0;
  o->periodic_mask = 0u;
  o->advect = 1;
  o->precision = 1;
  o->use_graph = 1;
  o->stream = nullptr;
  o->workspace = nullptr;
  o->workspace_bytes = 0;
  o->coarse_precision = 0;
}

size_t wl_workspace_bytes(const int* dims, int ndim, const wl_opts* opts) {
  if (!dims || (ndim != 2 && ndim != 3)) return 0;
  for (int d = 0; d < ndim; ++d)
    if (dims[d] < 2) return 0;
  wl_opts o;
  wl_default_opts(&o);
  if (opts) o = *opts;
  if (o.coarse_precision < 0 || o.coarse_precision > 2) return 0;
  return layout(nullptr, ndim, dims, o.precision, o.coarse_precision, o.exit_bc ? 1 : 0, nullptr);
}

int wl_create(const int* dims, int ndim, double nu, const double* U, const wl_body* body, const wl_opts* opts,
              wl_handle* out) {
  if (!out) return WL_EINVAL;
  *out = nullptr;
  if (!dims || !U || (ndim != 2 && ndim != 3)) return WL_EINVAL;
  for (int d = 0; d < ndim; ++d)
    if (dims[d] < 2 || dims[d] > (1 << 20)) return WL_EINVAL;
  const long long nc = (long long)dims[0] * dims[1] * (ndim == 3 ? dims[2] : 1);
  if (nc > (1LL << 31)) return WL_EINVAL;
  if (!(nu >= 0.0) || !std::isfinite(nu)) return WL_EINVAL;
  wl_opts o;
  wl_default_opts(&o);
  if (opts) o = *opts;
  if (!(o.tol > 0.0) || o.max_vcycles < 0 || o.post < 1 || !(o.eps > 0.0) || !(o.dt_cap > 0.0) ||
      o.precision < 0 || o.precision > 1 || o.coarse_precision < 0 || o.coarse_precision > 2 || o.exit_bc < 0 ||
      o.exit_bc > 1 || o.metrics < 0 || o.metrics > 1)
    return WL_EINVAL;
  if (o.exit_bc && ((o.periodic_mask & 1u) || !(U[0] > 0.0))) return WL_EINVAL;  // exit: x walls, outflow
  if (body && (body->kind < 0 || body->kind > 3 || (body->kind == 2 && ndim != 3) ||
               (body->kind == 3 && !body->sdf_nodes)))
    return WL_EINVAL;
  wl_sim* s = new wl_sim();
  static std::atomic<unsigned long long> next_uid{1};
  s->uid = next_uid.fetch_add(1);
  s->D = ndim;
  s->o = o;
  s->nu = nu;
  s->st = (cudaStream_t)o.stream;
  for (int d = 0; d < 3; ++d) {
    s->g.n[d] = d < ndim ? dims[d] : 1;
    s->g.U[d] = d < ndim ? (float)U[d] : 0.f;
    if (d < ndim && !std::isfinite(U[d])) {
      delete s;
      return WL_EINVAL;
    }
  }
  s->g.per = o.periodic_mask & ((1u << ndim) - 1u);
  s->g.nc = nc;
  s->g.exit = o.exit_bc ? 1 : 0;
  s->body.kind = body ? body->kind : 0;
  for (int d = 0; d < 3; ++d) s->body.c[d] = body ? body->center[d] : 0.0;
  s->body.r1 = body ? body->radius : 0.0;
  s->body.r2 = body ? body->radius2 : 0.0;
  s->body.eps = o.eps;
  s->body.nodes = nullptr;
  if (s->body.kind == 3) {
    // the sampled distance: a device copy, and the cells whose corner values bracket
    // |d| < eps (a multilinear value lies between its corners' values)
    long long nn = 1;
    for (int d = 0; d < 3; ++d) {
      s->body.nn[d] = d < ndim ? dims[d] + 1 : 1;
      nn *= s->body.nn[d];
    }
    const float* v = body->sdf_nodes;
    for (long long q = 0; q < nn; ++q)
      if (!std::isfinite(v[q])) {
        delete s;
        return WL_EINVAL;
      }
    for (int d = 0; d < 3; ++d) {
      s->body.blo[d] = d < ndim ? dims[d] : 0;
      s->body.bhi[d] = d < ndim ? 0 : 1;
    }
    const int n0 = s->g.n[0], n1 = s->g.n[1], n2 = ndim == 3 ? s->g.n[2] : 1;
    const long long s1 = s->body.nn[0], s2 = s1 * s->body.nn[1];
    for (int k = 0; k < n2; ++k)
      for (int j = 0; j < n1; ++j)
        for (int i = 0; i < n0; ++i) {
          float lo = 1e30f, hi = -1e30f;
          for (int c = 0; c < (ndim == 3 ? 8 : 4); ++c) {
            const float w = v[(i + (c & 1)) + s1 * (j + ((c >> 1) & 1)) + s2 * (k + ((c >> 2) & 1))];
            lo = std::min(lo, w);
            hi = std::max(hi, w);
          }
          if (lo < o.eps && hi > -o.eps) {
            const int I[3] = {i, j, k};
            for (int d = 0; d < ndim; ++d) {
              s->body.blo[d] = std::min(s->body.blo[d], I[d]);
              s->body.bhi[d] = std::max(s->body.bhi[d], I[d] + 1);
            }
          }
        }
    if (cudaMalloc(&s->body_nodes, sizeof(float) * nn) != cudaSuccess) {
      cudaGetLastError();
      delete s;
      return WL_ENOMEM;
    }
    if (cudaMemcpy(s->body_nodes, v, sizeof(float) * nn, cudaMemcpyHostToDevice) != cudaSuccess) {
      cudaGetLastError();
      cudaFree(s->body_nodes);
      delete s;
      return WL_ECUDA;
    }
    s->body.nodes = s->body_nodes;
  }
  const size_t need = layout(nullptr, ndim, dims, o.precision, o.coarse_precision, o.exit_bc ? 1 : 0, nullptr);
  if (o.workspace) {
    if (o.workspace_bytes < need || ((uintptr_t)o.workspace & 255u)) {
      delete s;
      return WL_ENOMEM;
    }
    s->ws = (char*)o.workspace;
    s->own_ws = false;
  } else {
    void* p = nullptr;
    if (cudaMalloc(&p, need) != cudaSuccess) {
      cudaGetLastError();
      delete s;
      return WL_ENOMEM;
    }
    s->ws = (char*)p;
    s->own_ws = true;
  }
  s->ws_bytes = need;
  layout(s, ndim, dims, o.precision, o.coarse_precision, o.exit_bc ? 1 : 0, s->ws);
  for (size_t off : s->canaries) cudaMemsetAsync(s->ws + off, 0xA5, kCanary, s->st);
  // Staged kernels: tiles away from the body take the variant that forms the face
  // coefficients (the level's free-stream value 2^(l (D-2)), 0 on walls) instead of
  // loading them.  The band box (faces with mu0 < 1 lie inside it) scaled to each level,
  // one cell wider; without a body every tile is uniform.  The band tiles then run as a
  // second launch beside the uniform one; measured, that pays only where they are a small
  // part of the level (<= 5 % of its tiles: the fine level of large grids), so other
  // levels load every coefficient.
  {
    int lo[3], hi[3];
    const bool body = stage_band_box(ndim, s->g, s->body, lo, hi);
    const bool split = !std::getenv("WL_NO_UNIFORM");
    // The largest band-tile fraction a level splits at: 5 %, 8 % on levels of at least 2^24
    // cells (measured: the 512x256x256 donut's fine level, 5.2 %: 9.73 -> 7.61 ms per
    // step split; the 256x128x128 sphere's, 6.9 %: 1.714 -> 1.728 ms).  WL_UNIFORM_ALL:
    // split every level; WL_SPLIT_MAX: one fraction for every level.
    const char* sm = std::getenv("WL_SPLIT_MAX");
    for (int l = 0; l < s->nlev; ++l) {
      LevelBuf& L = s->lev[l];
      L.uval = ldexpf(1.f, l * (ndim - 2));
      for (int d = 0; d < 3; ++d) {
        if (body) {
          L.band.lo[d] = (lo[d] >> l) - 1;
          L.band.hi[d] = ((hi[d] + (1 << l) - 1) >> l) + 1;
        } else {  // empty box
          L.band.lo[d] = 1 << 30;
          L.band.hi[d] = -(1 << 30);
        }
      }
      const int tz = sweep_planes_per_block(L.g, SWEEP_UNI_BLOCKS_PER_SM);
      const double frac_max = std::getenv("WL_UNIFORM_ALL") ? 2.0
                              : sm                           ? std::atof(sm)
                              : (L.g.nc >= (1ll << 24) ? 0.08 : 0.05);
      L.band.on = (split && band_tile_fraction(ndim, L.g, tz, L.band, SWEEP_TY) <= frac_max) ? 1 : 0;
      // 16-row tiles on the large split levels that are periodic in neither x nor y: a
      // warp relaxes twice the cells per plane for the same per-plane bookkeeping
      L.ty = (ndim == 3 && L.band.on && !(L.g.per & 3u) && L.g.n[1] % SWEEP_TY16 == 0 &&
              L.g.nc >= ty16_min_cells())
                 ? SWEEP_TY16
                 : SWEEP_TY;
      // tiles the staged sweep takes and tiles across a periodic side (launches with
      // no tile of their kind are skipped).  The staged kernel takes the latter too when
      // the periodic sides are whole tiles and all of those tiles are uniform.
      // Tile columns (x, y) of each kind; the wrapping launch blocks z for its own tile
      // columns and residency, and the band test uses its tiles.
      L.tma_tiles = L.wrap_tiles = L.wrap_tma_tiles = 0;
      const int ntx = (L.g.n[0] + SWEEP_TX - 1) / SWEEP_TX, nty = (L.g.n[1] + SWEEP_TY - 1) / SWEEP_TY;
      for (int tj = 0; tj < nty; ++tj)
        for (int ti = 0; ti < ntx; ++ti) {
          if (sweep_tile_wraps_xy(L.g, ti * SWEEP_TX, tj * SWEEP_TY))
            ++L.wrap_tiles;
          else
            ++L.tma_tiles;
        }
      L.tzw = sweep_planes_for_columns(L.g.n[2], std::max(L.wrap_tiles, 1), SWEEP_WRAP_BLOCKS_PER_SM);
      bool wrap_uni = L.band.on && sweep_wrap_shape_ok(L.g);
      const int nz = ndim == 3 ? (L.g.n[2] + L.tzw - 1) / L.tzw : 1;
      for (int tj = 0; tj < nty && wrap_uni; ++tj)
        for (int ti = 0; ti < ntx; ++ti) {
          if (!sweep_tile_wraps_xy(L.g, ti * SWEEP_TX, tj * SWEEP_TY)) continue;
          for (int tk = 0; tk < nz; ++tk) {
            const int k0 = ndim == 3 ? tk * L.tzw : 0, k1 = ndim == 3 ? std::min(k0 + L.tzw, L.g.n[2]) : 1;
            if (tile_in_band(L.band, ndim, ti * SWEEP_TX, tj * SWEEP_TY, k0, k1)) wrap_uni = false;
          }
        }
      if (wrap_uni) {
        L.wrap_tma_tiles = L.wrap_tiles;
        L.wrap_tiles = 0;
      }
    }
  }
  // The coarse end of the V-cycle runs in one block from the largest level whose
  // hierarchy below holds at most kTailCells cells (the coarsest solved densely; a
  // 16-bit level 1 keeps its staged conversion, so the tail starts at level 2 or below).
  // Measured in a CUDA graph: a per-level launch costs ~2.5 us, the block ~4 us plus its
  // sweeps on one SM, so the tail pays for small levels only (with 9K cells it lost).
  if (s->G && s->nlev >= 3 && !std::getenv("WL_NO_TAIL")) {
    int n[kMaxLevels][3];
    long long cells = 0;
    for (int l = 0; l < s->nlev; ++l)
      for (int d = 0; d < 3; ++d) n[l][d] = s->lev[l].g.n[d];
    const int lmin = s->lev[1].z32 ? 2 : 1;
    for (int lf = s->nlev - 1; lf >= lmin; --lf) {  // grow the tail upwards while it stays small
      cells += s->lev[lf].g.nc;
      if (cells > kTailCells || s->nlev - lf > kTailMaxLevels ||
          vcycle_tail_smem(ndim, n + lf, s->nlev - lf) > kTailSmemMax)
        break;
      if (lf + 2 <= s->nlev) s->tail_lf = lf;
    }
  }
  int rc = WL_OK;
  if (cudaMallocHost(&s->hs, sizeof(DevState)) != cudaSuccess) rc = fail(s, WL_ENOMEM, "pinned host state");
  if (!rc) rc = cuda_check(s, cudaStreamCreateWithFlags(&s->cs, cudaStreamNonBlocking), "capture stream");
  if (!rc) rc = cuda_check(s, cudaStreamCreateWithFlags(&s->side.aux, cudaStreamNonBlocking), "side stream");
  if (!rc) rc = cuda_check(s, cudaEventCreateWithFlags(&s->side.fork, cudaEventDisableTiming), "side event");
  if (!rc) rc = cuda_check(s, cudaEventCreateWithFlags(&s->side.join, cudaEventDisableTiming), "side event");
  if (!rc && !std::getenv("WL_NO_TMA")) {  // tensor maps for the staged sweep
    for (int l = 0; l < s->nlev; ++l) {
      LevelBuf& L = s->lev[l];
      if (L.st != ST_F32) {  // 16-bit levels use the table sweep
        L.tma = false;
        continue;
      }
      // sweep boxes: iterate 12 rows, coefficients 10 (L1: 11); residual boxes: 8 rows
      // (faces of y: 9)
      // (the sweep's boxes follow the level's tile height: iterate ty + 4 rows, coefficients
      // ty + 2, L1 ty + 3)
      const int crows = L.ty + 2;
      bool ok = make_field_map(&L.mx, L.x, L.g, ndim, L.ty + 4) && make_field_map(&L.mx2, L.x2, L.g, ndim, L.ty + 4) &&
                make_field_map(&L.mz, L.z, L.g, ndim, SWEEP_TY) && make_field_map(&L.sz, L.z, L.g, ndim, crows);
      for (int c = 0; c < ndim; ++c)
        ok = ok && make_field_map(&L.mL[c], L.L[c], L.g, ndim, SWEEP_TY + (c == 1 ? 1 : 0)) &&
             make_field_map(&L.sL[c], L.L[c], L.g, ndim, crows + (c == 1 ? 1 : 0));
      if (l == 0 && s->rf) ok = ok && make_field_map(&s->srf, s->rf, L.g, ndim, crows);
      L.tma = ok;
    }
    // fine residual: 3-D; with a periodic x / y side when those sides are whole tiles
    // and the tiles on them are uniform (they patch their halo; see k_resid_tma)
    LevelBuf& L0 = s->lev[0];
    const int rtz0 = sweep_planes_per_block(L0.g, L0.band.on ? RESID_UNI_WAVE_BLOCKS : SWEEP_BLOCKS_PER_SM);
    bool ok = L0.tma && ndim == 3 && !std::getenv("WL_NO_RESID_TMA") &&
              (!(s->g.per & 3u) || (sweep_wrap_shape_ok(s->g) && !resid_band_wraps(s->g, rtz0 + (rtz0 & 1), L0.band)));
    // pressure boxes with a 1-row halo: 10 rows from j0-1
    if (ok) ok = make_field_map(&s->mph, s->ph ? s->ph : L0.x, L0.g, ndim, SWEEP_TY + 2);
    if (ok && s->pl) ok = make_field_map(&s->mpl, s->pl, L0.g, ndim, SWEEP_TY + 2);
    float** bufs[3] = {s->ua, s->ub, s->uc};
    for (int b = 0; b < 3 && ok; ++b)
      for (int c = 0; c < ndim && ok; ++c)
        ok = make_field_map(&s->mu[b][c], bufs[b][c], L0.g, ndim, SWEEP_TY + (c == 1 ? 1 : 0));
    s->resid_tma = ok;
  }
  // The coarse end from a larger level in one thread-block cluster (16 blocks, else 8):
  // its levels are split between the blocks' shared memories, so tens of thousands of
  // cells fit, and the sweeps of a level that would take a launch each run between
  // cluster barriers.  Measured: a cluster phase costs about a microsecond, so the
  // cluster pays where it replaces levels swept by the index-table kernel (periodic
  // levels narrower than a tile: 12 us a launch) and loses where the staged sweeps run
  // (a few us a launch inside a graph); taken only where it covers more levels than the
  // one-block tail and one of them uses the table kernel.  FP32 coarse levels only (a
  // tail keeps its levels in FP32, which would take levels the 16-bit modes store in
  // 16 bits out of them).  WL_CTAIL_ALWAYS drops the table-level condition (tests).
  if (!rc && s->G && s->nlev >= 3 && !std::getenv("WL_NO_TAIL") && !std::getenv("WL_NO_CTAIL") &&
      s->o.coarse_precision == WL_COARSE_FP32) {
    int n[kMaxLevels][3];
    for (int l = 0; l < s->nlev; ++l)
      for (int d = 0; d < 3; ++d) n[l][d] = s->lev[l].g.n[d];
    auto table_level = [&](int l) {
      const LevelBuf& L = s->lev[l];
      return !(L.tma && (L.tma_tiles > 0 || L.wrap_tma_tiles > 0)) || L.wrap_tiles > 0;
    };
    for (int C = 16; C >= 8 && !s->ctail_lf; C -= 8) {
      int best = 0;
      long long cl_cells = 0;
      for (int lf = s->nlev - 1; lf >= 1; --lf) {
        cl_cells += s->lev[lf].g.nc;
        if (cl_cells > kCtailCells || s->nlev - lf > kTailMaxLevels ||
            vcycle_ctail_smem(ndim, n + lf, s->nlev - lf, C) > kTailSmemMax)
          break;
        if (lf + 2 <= s->nlev) best = lf;
      }
      const int top = s->tail_lf > 0 ? s->tail_lf : s->nlev;
      bool table = false;
      for (int l = best; best > 0 && l < top; ++l) table = table || table_level(l);
      if (best > 0 && best < top && (table || std::getenv("WL_CTAIL_ALWAYS")) &&
          vcycle_ctail_cluster(ndim, vcycle_ctail_smem(ndim, n + best, s->nlev - best, C), C) == C) {
        s->ctail_lf = best;
        s->ctail_c = C;
      }
    }
  }
  if (!rc) {
    launch_measure(ndim, s->g, s->body, s->lev[0].L, s->st);
    for (int l = 1; l < s->nlev; ++l) {
      const float* Lf[3] = {s->lev[l - 1].L[0], s->lev[l - 1].L[1], s->lev[l - 1].L[2]};
      launch_coarsen(ndim, s->lev[l - 1].g, Lf, s->lev[l].g, s->lev[l].L, s->st);
    }
    for (int l = 0; l < s->nlev; ++l) {
      const LevelBuf& L = s->lev[l];
      if (L.st != ST_F32)
        for (int c = 0; c < ndim; ++c) launch_to_storage(L.L[c], L.Lk[c], L.st, L.g.nc, s->st);
      cudaMemsetAsync(L.x, 0, esize(L.st) * L.g.nc, s->st);
      cudaMemsetAsync(L.z, 0, esize(L.st) * L.g.nc, s->st);
      if (L.z32) cudaMemsetAsync(L.z32, 0, sizeof(float) * L.g.nc, s->st);
    }
    if (s->rf) cudaMemsetAsync(s->rf, 0, sizeof(float) * s->g.nc, s->st);
    if (s->G) {
      DenseArgs d{};
      LevelBuf& Lc = s->lev[s->nlev - 1];
      for (int c = 0; c < 3; ++c) d.L[c] = Lc.L[c];
      d.g = Lc.g;
      d.G = s->G;
      launch_build_pinv(ndim, d, s->st);
    }
    rc = reset_state(s);
  }
  if (!rc) {
    launch_set_ic(ndim, s->g, 0, 0.0, s->ua, s->st);
    init_exit(s);
    rc = set_dt_from_ic(s);
  }
  if (!rc) rc = cuda_check(s, cudaStreamSynchronize(s->st), "create");
  if (rc) {
    wl_destroy(s);
    return rc;
  }
  *out = s;
  return WL_OK;
}

void wl_destroy(wl_handle s) {
  if (!s) return;
  if (s->st) cudaStreamSynchronize(s->st);
  else cudaDeviceSynchronize();
  if (s->exec) cudaGraphExecDestroy(s->exec);
  if (s->graph) cudaGraphDestroy(s->graph);
  if (s->join) cudaEventDestroy(s->join);
  if (s->cs) cudaStreamDestroy(s->cs);
  if (s->side.aux) cudaStreamDestroy(s->side.aux);
  if (s->side.fork) cudaEventDestroy(s->side.fork);
  if (s->side.join) cudaEventDestroy(s->side.join);
  if (s->hs) cudaFreeHost(s->hs);
  if (s->own_ws && s->ws) cudaFree(s->ws);
  free_grad_graphs(s->gr);
  if (s->gr.own && s->gr.mem) cudaFree(s->gr.mem);
  if (s->body_nodes) cudaFree(s->body_nodes);
  delete s;
}

const char* wl_last_error(wl_handle s) { return s ? s->err.c_str() : "null handle"; }

int wl_set_ic(wl_handle s, int kind, double amp, const float* src, int src_is_device) {
  if (!s) return WL_EINVAL;
  if (kind < 0 || kind > 2 || (kind == 2 && !src)) return fail(s, WL_EINVAL, "wl_set_ic: bad kind/source");
  if (kind == 2) {
    for (int c = 0; c < s->D; ++c)
      WL_CUDA(s, cudaMemcpyAsync(s->ua[c], src + (size_t)c * s->g.nc, sizeof(float) * s->g.nc,
                                 src_is_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, s->st));
    launch_fix_bfaces(s->D, s->g, s->ua, s->st);
  } else {
    launch_set_ic(s->D, s->g, kind, amp, s->ua, s->st);
  }
  init_exit(s);
  int rc = reset_state(s);
  if (rc) return rc;
  rc = set_dt_from_ic(s);
  if (rc) return rc;
  s->poisoned = false;
  return cuda_check(s, cudaStreamSynchronize(s->st), "wl_set_ic");
}

int wl_step(wl_handle s, int nsteps) {
  if (!s || nsteps < 0) return WL_EINVAL;
  if (s->poisoned) return fail(s, WL_ENONFINITE, "sim is poisoned by a non-finite value");
  if (!s->o.use_graph) {
    for (int n = 0; n < nsteps; ++n) {
      int rc = host_step(s);
      if (rc) return rc;
    }
    return WL_OK;
  }
  if (!s->exec) {
    int rc = build_step_graph(s);
    if (rc) return rc;
  }
  for (int n = 0; n < nsteps; ++n) WL_CUDA(s, cudaGraphLaunch(s->exec, s->st));
  return WL_OK;
}

int wl_step_batch(const wl_handle* hs, int n, int nsteps, void* stream) {
  if ((!hs && n > 0) || n < 0 || nsteps < 0) return WL_EINVAL;
  cudaStream_t cs = (cudaStream_t)stream;
  cudaEvent_t fork = nullptr;
  if (cudaEventCreateWithFlags(&fork, cudaEventDisableTiming) != cudaSuccess ||
      cudaEventRecord(fork, cs) != cudaSuccess) {
    cudaGetLastError();
    if (fork) cudaEventDestroy(fork);
    return WL_ECUDA;
  }
  int first = WL_OK;
  for (int i = 0; i < n; ++i) {
    wl_handle s = hs[i];
    int rc = WL_OK;
    if (!s) {
      rc = WL_EINVAL;
    } else if (s->poisoned) {
      rc = fail(s, WL_ENONFINITE, "sim is poisoned by a non-finite value");
    } else {
      const bool own = s->st != cs;
      if (own && !s->join) rc = cuda_check(s, cudaEventCreateWithFlags(&s->join, cudaEventDisableTiming), "join event");
      if (!rc && own) rc = cuda_check(s, cudaStreamWaitEvent(s->st, fork, 0), "fork");
      if (!rc) rc = wl_step(s, nsteps);
      if (!rc && own) rc = cuda_check(s, cudaEventRecord(s->join, s->st), "join record");
      if (!rc && own) rc = cuda_check(s, cudaStreamWaitEvent(cs, s->join, 0), "join");
    }
    if (rc && !first) first = rc;
  }
  cudaEventDestroy(fork);
  return first;
}

int wl_stage(wl_handle s, int stage) {
  if (!s || (stage != 1 && stage != 2)) return WL_EINVAL;
  enq_stage(s, stage, s->st);
  return cuda_check(s, cudaGetLastError(), "wl_stage");
}

int wl_project(wl_handle s, double w, int* vcycles_out, double* resid_out) {
  if (!s || !(w > 0.0)) return WL_EINVAL;
  int rc = host_projection(s, 0, (float)w, 0);
  if (rc) return rc;
  enq_correct(s, s->ua, s->ua, (float)w, 0, s->st);  // no neighbour reads: in place is safe
  rc = sync_state(s);
  if (rc) return rc;
  if (vcycles_out) *vcycles_out = s->hs->last_iters[0];
  if (resid_out) *resid_out = s->hs->last_res[0];
  if (!std::isfinite(s->hs->last_res[0])) {
    s->poisoned = true;
    return fail(s, WL_ENONFINITE, "non-finite residual");
  }
  return (s->hs->last_res[0] > s->o.tol) ? WL_WNOTCONV : WL_OK;
}

int wl_gmg_vcycle(wl_handle s, double* resid_inf_out) {
  if (!s) return WL_EINVAL;
  // restrict the residual of the held system, run one cycle, measure the residual
  enq_fine_residual(s, RES_RESIDUAL, 0, 1.f, s->st);
  enq_vcycle_core(s, s->st);
  WL_CUDA(s, cudaMemsetAsync(&s->ds->norm_bits, 0, sizeof(unsigned), s->st));
  enq_fine_residual(s, RES_RESIDUAL, 0, 1.f, s->st);
  int rc = sync_state(s);
  if (rc) return rc;
  const float r = reinterpret_cast<const float&>(s->hs->norm_bits);
  WL_CUDA(s, cudaMemsetAsync(&s->ds->norm_bits, 0, sizeof(unsigned), s->st));
  if (resid_inf_out) *resid_inf_out = r;
  return cuda_check(s, cudaStreamSynchronize(s->st), "wl_gmg_vcycle");
}

int wl_forces(wl_handle s, double* F) {
  if (!s || !F) return WL_EINVAL;
  const float* L[3] = {s->lev[0].L[0], s->lev[0].L[1], s->lev[0].L[2]};
  launch_forces(s->D, s->g, s->body, s->ph ? s->ph : s->lev[0].x, s->pl, L, s->fpart, kForceParts, s->fout,
                s->st);
  double h[4];
  WL_CUDA(s, cudaMemcpyAsync(h, s->fout, sizeof(h), cudaMemcpyDeviceToHost, s->st));
  WL_CUDA(s, cudaStreamSynchronize(s->st));
  for (int d = 0; d < s->D; ++d) F[d] = h[d];
  return WL_OK;
}

int wl_viscous_force(wl_handle s, double* F) {
  if (!s || !F) return WL_EINVAL;
  const float* u[3] = {s->ua[0], s->ua[1], s->ua[2]};
  launch_viscous_force(s->D, s->g, s->body, u, s->nu, s->fout, s->st);
  double h[3];
  WL_CUDA(s, cudaMemcpyAsync(h, s->fout, sizeof(h), cudaMemcpyDeviceToHost, s->st));
  WL_CUDA(s, cudaStreamSynchronize(s->st));
  for (int d = 0; d < s->D; ++d) F[d] = h[d];
  return WL_OK;
}

int wl_get_field(wl_handle s, int which, void* dst, int dst_is_device) {
  if (!s || !dst || !valid_field(which)) return WL_EINVAL;
  const cudaMemcpyKind kind = dst_is_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
  const size_t nb = sizeof(float) * s->g.nc;
  char* d = (char*)dst;
  switch (which) {
    case WL_FIELD_U:
      for (int c = 0; c < s->D; ++c) WL_CUDA(s, cudaMemcpyAsync(d + c * nb, s->ua[c], nb, kind, s->st));
      break;
    case WL_FIELD_P:
      if (s->ph) launch_df_round(s->ph, s->pl, s->lev[0].x2, s->g.nc, s->st);
      WL_CUDA(s, cudaMemcpyAsync(d, s->ph ? s->lev[0].x2 : s->lev[0].x, nb, kind, s->st));
      break;
    case WL_FIELD_DIV: {
      ResArgs a = res_args(s, 0, RES_DIV_ONLY);
      for (int c = 0; c < 3; ++c) a.u[c] = s->ua[c];
      a.z = s->lev[0].x2;
      a.zc = nullptr;
      launch_residual(s->D, a, s->st);
      WL_CUDA(s, cudaMemcpyAsync(d, s->lev[0].x2, nb, kind, s->st));
      break;
    }
    case WL_FIELD_MU0:
      for (int c = 0; c < s->D; ++c) WL_CUDA(s, cudaMemcpyAsync(d + c * nb, s->lev[0].L[c], nb, kind, s->st));
      break;
    case WL_FIELD_Z:
      WL_CUDA(s, cudaMemcpyAsync(d, s->lev[0].z, nb, kind, s->st));
      break;
    case WL_FIELD_UPRED:
      for (int c = 0; c < s->D; ++c) WL_CUDA(s, cudaMemcpyAsync(d + c * nb, s->uc[c], nb, kind, s->st));
      break;
    case WL_FIELD_USTAGE:
      for (int c = 0; c < s->D; ++c) WL_CUDA(s, cudaMemcpyAsync(d + c * nb, s->ub[c], nb, kind, s->st));
      break;
    case WL_FIELD_EXIT:
      if (!s->g.exit) return fail(s, WL_EINVAL, "no convective exit");
      WL_CUDA(s, cudaMemcpyAsync(d, s->ua[0] + s->g.nc, sizeof(float) * (size_t)s->g.n[1] * s->g.n[2], kind, s->st));
      break;
    default:
      return WL_EINVAL;
  }
  if (!dst_is_device) WL_CUDA(s, cudaStreamSynchronize(s->st));
  return cuda_check(s, cudaGetLastError(), "wl_get_field");
}

int wl_set_field(wl_handle s, int which, const void* src, int src_is_device) {
  if (!s || !src) return WL_EINVAL;
  const cudaMemcpyKind kind = src_is_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
  const size_t nb = sizeof(float) * s->g.nc;
  const char* p = (const char*)src;
  switch (which) {
    case WL_FIELD_U:
      for (int c = 0; c < s->D; ++c) WL_CUDA(s, cudaMemcpyAsync(s->ua[c], p + c * nb, nb, kind, s->st));
      launch_fix_bfaces(s->D, s->g, s->ua, s->st);
      break;
    case WL_FIELD_P:
      WL_CUDA(s, cudaMemcpyAsync(s->ph ? s->ph : s->lev[0].x, p, nb, kind, s->st));
      if (s->pl) WL_CUDA(s, cudaMemsetAsync(s->pl, 0, nb, s->st));
      break;
    case WL_FIELD_Z:
      WL_CUDA(s, cudaMemcpyAsync(s->lev[0].z, p, nb, kind, s->st));
      break;
    case WL_FIELD_UPRED:
      for (int c = 0; c < s->D; ++c) WL_CUDA(s, cudaMemcpyAsync(s->uc[c], p + c * nb, nb, kind, s->st));
      launch_fix_bfaces(s->D, s->g, s->uc, s->st);
      break;
    case WL_FIELD_EXIT:
      if (!s->g.exit) return fail(s, WL_EINVAL, "no convective exit");
      WL_CUDA(s, cudaMemcpyAsync(s->ua[0] + s->g.nc, p, sizeof(float) * (size_t)s->g.n[1] * s->g.n[2], kind, s->st));
      break;
    default:
      return fail(s, WL_EINVAL, "field is read-only");
  }
  WL_CUDA(s, cudaStreamSynchronize(s->st));
  return cuda_check(s, cudaGetLastError(), "wl_set_field");
}

int wl_get_dt(wl_handle s, double* dt) {
  if (!s || !dt) return WL_EINVAL;
  int rc = sync_state(s);
  if (rc) return rc;
  *dt = s->hs->dt;
  return WL_OK;
}

int wl_set_dt(wl_handle s, double dt) {
  if (!s || !(dt > 0.0) || !std::isfinite(dt)) return WL_EINVAL;
  WL_CUDA(s, cudaMemcpyAsync(&s->ds->dt, &dt, sizeof(double), cudaMemcpyHostToDevice, s->st));
  launch_sync_dt(s->ds, s->st);
  WL_CUDA(s, cudaStreamSynchronize(s->st));
  return WL_OK;
}

int wl_get_time(wl_handle s, double* t, long long* steps) {
  if (!s) return WL_EINVAL;
  int rc = sync_state(s);
  if (rc) return rc;
  if (t) *t = s->hs->time;
  if (steps) *steps = s->hs->steps;
  return WL_OK;
}

int wl_status(wl_handle s, int* last_vcycles, long long* total_vcycles, double* worst_resid) {
  if (!s) return WL_EINVAL;
  int rc = sync_state(s);
  if (rc) return rc;
  const DevState h = *s->hs;
  if (last_vcycles) {
    last_vcycles[0] = h.last_iters[0];
    last_vcycles[1] = h.last_iters[1];
  }
  if (total_vcycles) *total_vcycles = h.total_vcycles;
  if (worst_resid) *worst_resid = h.worst_res;
  // clear the sticky flags for the next interval
  int zero = 0;
  float fz = 0.f;
  WL_CUDA(s, cudaMemcpyAsync(&s->ds->status, &zero, sizeof(int), cudaMemcpyHostToDevice, s->st));
  WL_CUDA(s, cudaMemcpyAsync(&s->ds->worst_res, &fz, sizeof(float), cudaMemcpyHostToDevice, s->st));
  WL_CUDA(s, cudaStreamSynchronize(s->st));
  if (h.status & 1) {
    s->poisoned = true;
    return fail(s, WL_ENONFINITE, "non-finite dt or residual");
  }
  if (h.status & 4) return fail(s, WL_ETIMEOUT, "a staged copy of the sweep did not arrive in time");
  if (h.status & 2) return WL_WNOTCONV;
  return WL_OK;
}

// kernel nodes of a graph (not descending into conditional nodes' bodies)
static int graph_kernels(cudaGraph_t g) {
  size_t n = 0;
  if (!g || cudaGraphGetNodes(g, nullptr, &n) != cudaSuccess) return -1;
  std::vector<cudaGraphNode_t> v(n);
  if (n && cudaGraphGetNodes(g, v.data(), &n) != cudaSuccess) return -1;
  int k = 0;
  for (size_t i = 0; i < n; ++i) {
    cudaGraphNodeType t;
    if (cudaGraphNodeGetType(v[i], &t) == cudaSuccess && t == cudaGraphNodeTypeKernel) ++k;
  }
  return k;
}

int wl_graph_kernels(wl_handle s, int* per_step, int* per_vcycle) {
  if (!s || !per_step || !per_vcycle) return WL_EINVAL;
  if (!s->graph || !s->vbody) return fail(s, WL_EINVAL, "no step graph (use_graph = 0 or no step yet)");
  *per_step = graph_kernels(s->graph);
  *per_vcycle = graph_kernels(s->vbody);
  if (*per_step < 0 || *per_vcycle < 0) return cuda_check(s, cudaGetLastError(), "graph nodes");
  return WL_OK;
}

int wl_profile_step(wl_handle s, int nsteps, double* ms, long long* launches) {
  if (!s || nsteps < 1 || !ms || !launches) return WL_EINVAL;
  if (s->poisoned) return fail(s, WL_ENONFINITE, "sim is poisoned by a non-finite value");
  std::vector<std::tuple<int, cudaEvent_t, cudaEvent_t>> rec;
  rec.reserve(4096);
  s->prof = &rec;
  int rc = WL_OK;
  for (int n = 0; n < nsteps && rc == WL_OK; ++n) rc = host_step(s);
  s->prof = nullptr;
  if (rc == WL_OK) rc = cuda_check(s, cudaStreamSynchronize(s->st), "wl_profile_step");
  for (int k = 0; k < WL_KCLASS_COUNT; ++k) {
    ms[k] = 0.0;
    launches[k] = 0;
  }
  for (auto& t : rec) {
    float e = 0.f;
    if (rc == WL_OK && cudaEventElapsedTime(&e, std::get<1>(t), std::get<2>(t)) == cudaSuccess) {
      ms[std::get<0>(t)] += e;
      launches[std::get<0>(t)] += 1;
    }
    cudaEventDestroy(std::get<1>(t));
    cudaEventDestroy(std::get<2>(t));
  }
  return rc;
}

int wl_wait_probe(double seconds, double* elapsed_ms) {
  if (!(seconds > 0.0) || seconds > 10.0) return WL_EINVAL;
  int* flag = nullptr;
  if (cudaMalloc(&flag, sizeof(int)) != cudaSuccess) {
    cudaGetLastError();
    return WL_ENOMEM;
  }
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  int rc = WL_OK, gave_up = 0;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) rc = WL_ECUDA;
  if (!rc) {
    cudaMemset(flag, 0, sizeof(int));
    cudaEventRecord(e0, 0);
    launch_wait_probe((uint64_t)(seconds * 1e9), flag, 0);
    cudaEventRecord(e1, 0);
    if (cudaMemcpy(&gave_up, flag, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess) rc = WL_ECUDA;
  }
  if (!rc && elapsed_ms) {
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    *elapsed_ms = ms;
  }
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  cudaFree(flag);
  if (cudaGetLastError() != cudaSuccess && !rc) rc = WL_ECUDA;
  if (rc) return rc;
  return gave_up ? WL_ETIMEOUT : WL_OK;
}

int wl_levels(wl_handle s, int* nlevels) {
  if (!s || !nlevels) return WL_EINVAL;
  *nlevels = s->nlev;
  return WL_OK;
}

int wl_level_dims(wl_handle s, int l, int* dims) {
  if (!s || !dims || l < 0 || l >= s->nlev) return WL_EINVAL;
  for (int d = 0; d < 3; ++d) dims[d] = s->lev[l].g.n[d];
  return WL_OK;
}

}  // extern "C"

// --------------------------------------------------------------- differentiated rollout
namespace {

size_t grad_layout(wl_sim* s, int nsteps, int every, char* base) {
  const int D = s->D;
  const size_t n = (size_t)s->g.nc;
  const int nseg = (nsteps + every - 1) / every;
  Carver cv{base};  // (the gradient workspace's canary gaps are not recorded: not checked)
  void* ck = cv.take(sizeof(float) * n * (D + 2) * (size_t)(nseg + 1));
  void* ckst = cv.take(sizeof(DevState) * (size_t)(nseg + 1));
  void* seg = cv.take(sizeof(float) * n * (2 * D + 2) * (size_t)every);
  void* adj = cv.take(sizeof(float) * n * (6 * D + 2));
  void* rec = cv.take(sizeof(double) * (size_t)nsteps * D);
  void* gF = cv.take(sizeof(double) * (size_t)nsteps * D);
  void* as = cv.take(sizeof(AdjState));
  void* part = cv.take(sizeof(double) * 4 * kForceParts);
  if (base) {
    wl_sim::Grad& G = s->gr;
    G.nsteps = nsteps;
    G.every = every;
    G.nseg = nseg;
    G.ck = (float*)ck;
    G.ckst = (DevState*)ckst;
    G.seg = (float*)seg;
    G.adj = (float*)adj;
    G.rec = (double*)rec;
    G.gF = (double*)gF;
    G.as = (AdjState*)as;
    G.part = (double*)part;
  }
  return cv.off;
}

float* ck_field(wl_sim* s, int k, int f) { return s->gr.ck + ((size_t)k * (s->D + 2) + f) * (size_t)s->g.nc; }

// checkpoint k: the velocity, the fine-level pressure and the device state
void save_ck(wl_sim* s, int k) {
  const size_t nb = sizeof(float) * (size_t)s->g.nc;
  for (int c = 0; c < s->D; ++c) cudaMemcpyAsync(ck_field(s, k, c), s->ua[c], nb, cudaMemcpyDeviceToDevice, s->st);
  cudaMemcpyAsync(ck_field(s, k, s->D), s->ph ? s->ph : s->lev[0].x, nb, cudaMemcpyDeviceToDevice, s->st);
  if (s->pl) cudaMemcpyAsync(ck_field(s, k, s->D + 1), s->pl, nb, cudaMemcpyDeviceToDevice, s->st);
  cudaMemcpyAsync(s->gr.ckst + k, s->ds, sizeof(DevState), cudaMemcpyDeviceToDevice, s->st);
}
void restore_ck(wl_sim* s, int k) {
  const size_t nb = sizeof(float) * (size_t)s->g.nc;
  for (int c = 0; c < s->D; ++c) cudaMemcpyAsync(s->ua[c], ck_field(s, k, c), nb, cudaMemcpyDeviceToDevice, s->st);
  cudaMemcpyAsync(s->ph ? s->ph : s->lev[0].x, ck_field(s, k, s->D), nb, cudaMemcpyDeviceToDevice, s->st);
  if (s->pl) cudaMemcpyAsync(s->pl, ck_field(s, k, s->D + 1), nb, cudaMemcpyDeviceToDevice, s->st);
  cudaMemcpyAsync(s->ds, s->gr.ckst + k, sizeof(DevState), cudaMemcpyDeviceToDevice, s->st);
}

// adjoint fields: [0,D) cotangent of the state, [D,2D) of u^n, [2D,3D) of the
// predictor u', [3D,4D) v', [4D,5D) f', [5D,6D) the coefficient cotangent, 6D and 6D+1:
// the adjoint pressures y of projections 1 and 2 (kept from step to step: each solve
// starts from its projection's solution one step later)
struct AdjFields {
  float* f[8][3];
};
AdjFields adj_fields(wl_sim* s) {
  AdjFields a{};
  const int D = s->D;
  for (int b = 0; b < 6; ++b)
    for (int c = 0; c < 3; ++c) a.f[b][c] = s->gr.adj + (size_t)(b * D + (c < D ? c : D - 1)) * s->g.nc;
  for (int c = 0; c < 3; ++c) {
    a.f[6][c] = s->gr.adj + (size_t)(6 * D) * s->g.nc;
    a.f[7][c] = s->gr.adj + (size_t)(6 * D + 1) * s->g.nc;
  }
  return a;
}

constexpr double kAdjRtol = 1e-7;

// The adjoint Poisson solve of projection k (0, 1) as a graph: solve A y = b (b in the
// fine right-hand side, mean-free over the active cells) with the forward multigrid to
// ||b - A y||_inf <= kAdjRtol ||b||_inf, starting from the projection's y of one step
// later (kept in y), the V-cycles in a WHILE node that the device's decision ends (at
// max_vcycles, flagged, or a non-finite residual, flagged); the solution (FP32) into y.
int build_adj_solve_graph(wl_sim* s, int k, float* y) {
  wl_sim::Grad& G = s->gr;
  WL_CUDA(s, cudaGraphCreate(&G.sgraph[k], 0));
  WL_CUDA(s, cudaGraphConditionalHandleCreate(&G.shc[k], G.sgraph[k], 0, 0));
  std::vector<cudaGraphNode_t> leaf;
  cudaGraph_t out = nullptr;
  WL_CUDA(s, cudaStreamBeginCaptureToGraph(s->cs, G.sgraph[k], nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal));
  launch_adj_warm(s->ph ? s->ph : s->lev[0].x, s->pl, y, G.as, s->g.nc, s->cs);
  cudaMemsetAsync(&s->ds->norm_bits, 0, sizeof(unsigned), s->cs);
  enq_fine_residual(s, RES_RESIDUAL, 0, 1.f, s->cs);
  launch_adj_decide(s->ds, G.as, G.shc[k], 1, 1, kAdjRtol, s->o.max_vcycles, s->cs);
  int rc = capture_leaf(s, leaf);
  WL_CUDA(s, cudaStreamEndCapture(s->cs, &out));
  if (rc) return rc;
  cudaGraphNodeParams cp{};
  cp.type = cudaGraphNodeTypeConditional;
  cp.conditional.handle = G.shc[k];
  cp.conditional.type = cudaGraphCondTypeWhile;
  cp.conditional.size = 1;
  cudaGraphNode_t wn;
  WL_CUDA(s, cudaGraphAddNode(&wn, G.sgraph[k], leaf.data(), nullptr, leaf.size(), &cp));
  WL_CUDA(s, cudaStreamBeginCaptureToGraph(s->cs, cp.conditional.phGraph_out[0], nullptr, nullptr, 0,
                                           cudaStreamCaptureModeThreadLocal));
  enq_vcycle_core(s, s->cs);
  enq_fine_residual(s, RES_RESIDUAL, 0, 1.f, s->cs);
  launch_adj_decide(s->ds, G.as, G.shc[k], 1, 0, kAdjRtol, s->o.max_vcycles, s->cs);
  WL_CUDA(s, cudaStreamEndCapture(s->cs, &out));
  WL_CUDA(s, cudaStreamBeginCaptureToGraph(s->cs, G.sgraph[k], &wn, nullptr, 1, cudaStreamCaptureModeThreadLocal));
  copy_pressure(s, y, s->cs);
  WL_CUDA(s, cudaStreamEndCapture(s->cs, &out));
  WL_CUDA(s, cudaGraphInstantiate(&G.sexec[k], G.sgraph[k], 0));
  return WL_OK;
}

void free_grad_graphs(wl_sim::Grad& G) {
  if (G.rexec) cudaGraphExecDestroy(G.rexec);
  if (G.rgraph) cudaGraphDestroy(G.rgraph);
  G.rexec = nullptr;
  G.rgraph = nullptr;
  for (int k = 0; k < 2; ++k) {
    if (G.sexec[k]) cudaGraphExecDestroy(G.sexec[k]);
    if (G.sgraph[k]) cudaGraphDestroy(G.sgraph[k]);
    G.sexec[k] = nullptr;
    G.sgraph[k] = nullptr;
  }
}

int adj_solve(wl_sim* s, int k, float* y) {
  wl_sim::Grad& G = s->gr;
  if (!G.sexec[k]) {
    int rc = build_adj_solve_graph(s, k, y);
    if (rc) return rc;
  }
  WL_CUDA(s, cudaGraphLaunch(G.sexec[k], s->st));
  return WL_OK;
}

// Adjoint of step n (its recorded slot m): the cotangent of u^{n+1} in field block 0 and
// of the force after the step in gF[n] give the cotangent of u^n in block 0 and add to
// theta and to the coefficient cotangent.
int adj_step(wl_sim* s, int m, int n) {
  const int D = s->D;
  const size_t nc = (size_t)s->g.nc;
  float* rec = s->gr.seg + (size_t)m * (2 * D + 2) * nc;
  float* un[3];
  float* up[3];
  for (int c = 0; c < 3; ++c) {
    un[c] = rec + (size_t)(c < D ? c : D - 1) * nc;
    up[c] = rec + (size_t)(D + (c < D ? c : D - 1)) * nc;
  }
  float* p1 = rec + (size_t)(2 * D) * nc;
  float* p2 = rec + (size_t)(2 * D + 1) * nc;
  AdjFields A = adj_fields(s);
  float* const* ub = A.f[0];
  float* const* ub0 = A.f[1];
  float* const* ubp = A.f[2];
  float* const* vb = A.f[3];
  float* const* fb = A.f[4];
  float* const* mb = A.f[5];
  float* y1 = A.f[6][0];
  float* y2 = A.f[7][0];
  const float* L[3] = {s->lev[0].L[0], s->lev[0].L[1], s->lev[0].L[2]};
  const double dt = s->o.dt_fixed;
  const double* g = s->gr.gF + (size_t)n * D;
  cudaStream_t st = s->st;
  // force after the step: F = -sum (p - pbar) n K_eps(d), p = x2 / (dt/2)
  launch_forces(D, s->g, s->body, p2, nullptr, L, s->fpart, kForceParts, s->fout, st);
  launch_adj_force_theta(D, s->g, s->body, p2, s->fout + 3, g, s->gr.as, st);
  // projection 2 (w = 1/2)
  launch_adj_proj_rhs(D, s->g, s->body, ub, L, g, 1.0 / (0.5 * dt), s->gr.as, s->lev[0].z, s->gr.part, kForceParts, st);
  int rc = adj_solve(s, 1, y2);
  if (rc) return rc;
  launch_adj_proj_out(D, s->g, ub, y2, p2, (float)(0.5 * dt), vb, mb, st);
  // stage 2: out = (u' + mu0 f + mu1 . grad f)/2, f = u^n + dt r(u')
  launch_adj_stage_local(D, s->g, vb, L, 0.5f, fb, ubp, st);
  StageArgs a = stage_args(s, 2);
  for (int c = 0; c < 3; ++c) {
    a.u[c] = up[c];
    a.u0[c] = un[c];
  }
  launch_adj_band(D, a, s->body, vb, 0.5f, fb, mb, s->gr.as, s->gr.part, kForceParts, st);
  for (int c = 0; c < D; ++c) cudaMemsetAsync(ub0[c], 0, sizeof(float) * nc, st);
  launch_adj_convdiff(D, s->g, up, fb, &s->ds->dtf, (float)s->nu, s->o.advect, ub0, ubp, st);
  // projection 1 (w = 1)
  launch_adj_proj_rhs(D, s->g, s->body, ubp, L, nullptr, 0.0, s->gr.as, s->lev[0].z, s->gr.part, kForceParts, st);
  rc = adj_solve(s, 0, y1);
  if (rc) return rc;
  launch_adj_proj_out(D, s->g, ubp, y1, p1, (float)dt, vb, mb, st);
  // stage 1: out = mu0 f + mu1 . grad f, f = u^n + dt r(u^n)
  launch_adj_stage_local(D, s->g, vb, L, 1.f, fb, nullptr, st);
  a = stage_args(s, 1);
  for (int c = 0; c < 3; ++c) a.u[c] = a.u0[c] = un[c];
  launch_adj_band(D, a, s->body, vb, 1.f, fb, mb, s->gr.as, s->gr.part, kForceParts, st);
  launch_adj_convdiff(D, s->g, un, fb, &s->ds->dtf, (float)s->nu, s->o.advect, ub0, ub0, st);
  for (int c = 0; c < D; ++c) cudaMemcpyAsync(ub[c], ub0[c], sizeof(float) * nc, cudaMemcpyDeviceToDevice, st);
  return cuda_check(s, cudaGetLastError(), "adjoint step");
}

int grad_check(wl_sim* s) {
  if (!(s->body.kind == 1 || (s->body.kind == 2 && s->D == 3)))
    return fail(s, WL_EINVAL, "gradients need a circle/sphere or torus body");
  if (s->g.exit) return fail(s, WL_EINVAL, "the convective exit is not differentiated");
  if (!(s->o.dt_fixed > 0.0)) return fail(s, WL_EINVAL, "gradients need a fixed dt (wl_opts.dt_fixed > 0)");
  if (s->poisoned) return fail(s, WL_ENONFINITE, "sim is poisoned");
  return WL_OK;
}

}  // namespace

size_t wl_grad_workspace_bytes(wl_handle s, int nsteps, int every) {
  if (!s || nsteps < 1 || every < 1) return 0;
  return grad_layout(s, nsteps, std::min(every, nsteps), nullptr);
}

int wl_grad_forward(wl_handle s, int nsteps, int every, void* workspace, size_t workspace_bytes, double* F) {
  if (!s || nsteps < 1 || every < 1 || !F) return WL_EINVAL;
  int rc = grad_check(s);
  if (rc) return rc;
  every = std::min(every, nsteps);
  const size_t need = grad_layout(s, nsteps, every, nullptr);
  wl_sim::Grad& G = s->gr;
  cudaStreamSynchronize(s->st);
  free_grad_graphs(G);
  if (G.own && G.mem) cudaFree(G.mem);
  G = wl_sim::Grad{};
  if (workspace) {
    if (workspace_bytes < need || ((uintptr_t)workspace & 255u)) return fail(s, WL_ENOMEM, "gradient workspace too small");
    G.mem = (char*)workspace;
  } else {
    void* p = nullptr;
    if (cudaMalloc(&p, need) != cudaSuccess) {
      cudaGetLastError();
      return fail(s, WL_ENOMEM, "gradient workspace");
    }
    G.mem = (char*)p;
    G.own = true;
  }
  grad_layout(s, nsteps, every, G.mem);
  WL_CUDA(s, cudaMemsetAsync(&s->ds->status, 0, sizeof(int), s->st));
  if (s->o.use_graph && !s->exec && (rc = build_step_graph(s))) return rc;
  for (int n = 0; n < nsteps; ++n) {
    if (n % every == 0) save_ck(s, n / every);
    if (s->o.use_graph)
      WL_CUDA(s, cudaGraphLaunch(s->exec, s->st));
    else if ((rc = host_step(s)))
      return rc;
    const float* L[3] = {s->lev[0].L[0], s->lev[0].L[1], s->lev[0].L[2]};
    launch_forces(s->D, s->g, s->body, s->ph ? s->ph : s->lev[0].x, s->pl, L, s->fpart, kForceParts, s->fout, s->st);
    WL_CUDA(s, cudaMemcpyAsync(G.rec + (size_t)n * s->D, s->fout, sizeof(double) * s->D, cudaMemcpyDeviceToDevice,
                               s->st));
  }
  save_ck(s, G.nseg);
  WL_CUDA(s, cudaMemcpyAsync(F, G.rec, sizeof(double) * nsteps * s->D, cudaMemcpyDeviceToHost, s->st));
  rc = sync_state(s);
  if (rc) return rc;
  if (s->hs->status & 1) {
    s->poisoned = true;
    return fail(s, WL_ENONFINITE, "non-finite value in the rollout");
  }
  G.ready = true;
  return (s->hs->status & 2) ? WL_WNOTCONV : WL_OK;
}

int wl_grad_backward(wl_handle s, const double* gF, double* theta_bar) {
  if (!s || !gF || !theta_bar) return WL_EINVAL;
  int rc = grad_check(s);
  if (rc) return rc;
  wl_sim::Grad& G = s->gr;
  if (!G.ready) return fail(s, WL_EINVAL, "wl_grad_backward needs a wl_grad_forward first");
  const int D = s->D;
  const size_t nc = (size_t)s->g.nc;
  WL_CUDA(s, cudaMemcpyAsync(G.gF, gF, sizeof(double) * G.nsteps * D, cudaMemcpyHostToDevice, s->st));
  const float* L[3] = {s->lev[0].L[0], s->lev[0].L[1], s->lev[0].L[2]};
  launch_adj_setup(D, s->g, s->body, L, G.as, G.part, kForceParts, s->st);
  AdjFields A = adj_fields(s);
  for (int c = 0; c < D; ++c) {
    cudaMemsetAsync(A.f[0][c], 0, sizeof(float) * nc, s->st);  // J has no term in the final state
    cudaMemsetAsync(A.f[5][c], 0, sizeof(float) * nc, s->st);
  }
  cudaMemsetAsync(A.f[6][0], 0, sizeof(float) * nc * 2, s->st);  // the adjoint solves' first starts
  if (s->o.use_graph && !G.rexec && (rc = build_step_graph_into(s, true, &G.rgraph, &G.rexec, G.rhc))) return rc;
  for (int k = G.nseg - 1; k >= 0; --k) {
    const int n0 = k * G.every, n1 = std::min(n0 + G.every, G.nsteps);
    restore_ck(s, k);
    for (int n = n0; n < n1; ++n) {  // recompute the segment, keeping what the adjoint needs
      launch_adj_set_slot(G.as, n - n0, s->st);
      if (s->o.use_graph)
        WL_CUDA(s, cudaGraphLaunch(G.rexec, s->st));
      else if ((rc = host_step(s, true)))
        return rc;
    }
    for (int n = n1 - 1; n >= n0; --n) {
      rc = adj_step(s, n - n0, n);
      if (rc) return rc;
    }
  }
  launch_adj_moments(D, s->g, s->body, A.f[5], G.as, G.part, kForceParts, s->st);
  restore_ck(s, G.nseg);
  AdjState as{};
  WL_CUDA(s, cudaMemcpyAsync(&as, G.as, sizeof(as), cudaMemcpyDeviceToHost, s->st));
  WL_CUDA(s, cudaStreamSynchronize(s->st));
  const int nt = s->body.kind == 2 ? 5 : D + 1;
  for (int t = 0; t < nt; ++t) theta_bar[t] = as.theta[t];
  rc = cuda_check(s, cudaGetLastError(), "wl_grad_backward");
  if (rc) return rc;
  if (as.flags & 1) {
    s->poisoned = true;
    return fail(s, WL_ENONFINITE, "non-finite adjoint residual");
  }
  if (as.flags & 2) return fail(s, WL_WNOTCONV, "an adjoint solve hit max_vcycles");
  return WL_OK;
}

int wl_kernel_paths(wl_handle s, unsigned* paths) {
  if (!s || !paths) return WL_EINVAL;
  *paths = (s->resid_tma ? WL_PATH_RESID_STAGED : 0u) | (s->ctail_lf > 0 ? WL_PATH_CLUSTER_TAIL : 0u) |
           (s->ctail_lf == 0 && s->tail_lf > 0 ? WL_PATH_BLOCK_TAIL : 0u);
  for (int l = 0; l < s->nlev; ++l)
    if (s->lev[l].tma && s->lev[l].ty == SWEEP_TY16) *paths |= WL_PATH_TALL_TILES;
  return WL_OK;
}

int wl_level_split(wl_handle s, int l, int* split, double* band_fraction) {
  if (!s || l < 0 || l >= s->nlev) return WL_EINVAL;
  const LevelBuf& L = s->lev[l];
  const bool on = L.tma && L.band.on;
  if (split) *split = on ? 1 : 0;
  if (band_fraction)
    *band_fraction = on ? band_tile_fraction(s->D, L.g, staged_sweep_tz(L, l), L.band, L.ty) : 1.0;
  return WL_OK;
}

// --------------------------------------------------------------- checkpoint / resume
namespace {

// Header of a saved state; the payload follows it: the velocity (D fields of nc values,
// then the exit plane when the sim has one), the fine pressure (ph and pl at precision 1,
// the FP32 pressure otherwise) and the device state.
struct SaveHeader {
  char magic[8];
  int version;
  int D;
  int n[3];
  unsigned per;
  int precision;
  int exit;
  int state_bytes;  // sizeof(DevState)
  int pad;
  long long nc;
  long long bytes;  // header + payload
  double nu;
  double U[3];
};
constexpr char kSaveMagic[8] = {'W', 'L', 'S', 'T', 'A', 'T', 'E', '1'};

long long exit_values(const wl_sim* s) { return s->g.exit ? (long long)s->g.n[1] * s->g.n[2] : 0; }
int npressure(const wl_sim* s) { return s->ph ? 2 : 1; }

size_t state_bytes(const wl_sim* s) {
  return sizeof(SaveHeader) + sizeof(float) * ((size_t)s->D * s->g.nc + exit_values(s) + npressure(s) * s->g.nc) +
         sizeof(DevState);
}

SaveHeader make_header(const wl_sim* s) {
  SaveHeader h{};
  std::memcpy(h.magic, kSaveMagic, sizeof(kSaveMagic));
  h.version = 1;
  h.D = s->D;
  for (int d = 0; d < 3; ++d) h.n[d] = s->g.n[d];
  h.per = s->g.per;
  h.precision = s->ph ? 1 : 0;
  h.exit = s->g.exit;
  h.state_bytes = (int)sizeof(DevState);
  h.nc = s->g.nc;
  h.bytes = (long long)state_bytes(s);
  h.nu = s->nu;
  for (int d = 0; d < 3; ++d) h.U[d] = s->g.U[d];
  return h;
}

}  // namespace

extern "C" size_t wl_state_bytes(wl_handle s) { return s ? state_bytes(s) : 0; }

extern "C" int wl_save(wl_handle s, void* dst, size_t dst_bytes, int dst_is_device) {
  if (!s || !dst) return WL_EINVAL;
  if (dst_bytes < state_bytes(s)) return fail(s, WL_EINVAL, "wl_save: destination smaller than wl_state_bytes");
  const SaveHeader h = make_header(s);
  const cudaMemcpyKind d2x = dst_is_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
  char* p = static_cast<char*>(dst);
  if (dst_is_device)
    WL_CUDA(s, cudaMemcpyAsync(p, &h, sizeof(h), cudaMemcpyHostToDevice, s->st));
  else
    std::memcpy(p, &h, sizeof(h));
  p += sizeof(h);
  const size_t nb = sizeof(float) * (size_t)s->g.nc;
  for (int c = 0; c < s->D; ++c, p += nb) WL_CUDA(s, cudaMemcpyAsync(p, s->ua[c], nb, d2x, s->st));
  if (s->g.exit) {
    const size_t eb = sizeof(float) * (size_t)exit_values(s);
    WL_CUDA(s, cudaMemcpyAsync(p, s->ua[0] + s->g.nc, eb, d2x, s->st));
    p += eb;
  }
  if (s->ph) {
    WL_CUDA(s, cudaMemcpyAsync(p, s->ph, nb, d2x, s->st));
    WL_CUDA(s, cudaMemcpyAsync(p + nb, s->pl, nb, d2x, s->st));
    p += 2 * nb;
  } else {
    WL_CUDA(s, cudaMemcpyAsync(p, s->lev[0].x, nb, d2x, s->st));
    p += nb;
  }
  WL_CUDA(s, cudaMemcpyAsync(p, s->ds, sizeof(DevState), d2x, s->st));
  // a host destination (and the header's staging copy) must be complete on return
  WL_CUDA(s, cudaStreamSynchronize(s->st));
  return WL_OK;
}

extern "C" int wl_load(wl_handle s, const void* src, size_t src_bytes, int src_is_device) {
  if (!s || !src) return WL_EINVAL;
  if (src_bytes < sizeof(SaveHeader)) return fail(s, WL_EINVAL, "wl_load: source smaller than a state header");
  SaveHeader h{};
  if (src_is_device) {
    WL_CUDA(s, cudaMemcpyAsync(&h, src, sizeof(h), cudaMemcpyDeviceToHost, s->st));
    WL_CUDA(s, cudaStreamSynchronize(s->st));
  } else {
    std::memcpy(&h, src, sizeof(h));
  }
  const SaveHeader want = make_header(s);
  bool same = std::memcmp(h.magic, kSaveMagic, sizeof(kSaveMagic)) == 0 && h.version == want.version &&
              h.D == want.D && h.per == want.per && h.precision == want.precision && h.exit == want.exit &&
              h.state_bytes == want.state_bytes && h.nc == want.nc && h.bytes == want.bytes && h.nu == want.nu;
  for (int d = 0; d < 3; ++d) same = same && h.n[d] == want.n[d] && h.U[d] == want.U[d];
  if (!same) return fail(s, WL_EINVAL, "wl_load: the saved state belongs to a different simulation setup");
  if (src_bytes < (size_t)h.bytes) return fail(s, WL_EINVAL, "wl_load: source shorter than the saved state");
  const cudaMemcpyKind x2d = src_is_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
  const char* p = static_cast<const char*>(src) + sizeof(h);
  const size_t nb = sizeof(float) * (size_t)s->g.nc;
  for (int c = 0; c < s->D; ++c, p += nb) WL_CUDA(s, cudaMemcpyAsync(s->ua[c], p, nb, x2d, s->st));
  if (s->g.exit) {
    const size_t eb = sizeof(float) * (size_t)exit_values(s);
    WL_CUDA(s, cudaMemcpyAsync(s->ua[0] + s->g.nc, p, eb, x2d, s->st));
    p += eb;
  }
  if (s->ph) {
    WL_CUDA(s, cudaMemcpyAsync(s->ph, p, nb, x2d, s->st));
    WL_CUDA(s, cudaMemcpyAsync(s->pl, p + nb, nb, x2d, s->st));
    p += 2 * nb;
  } else {
    WL_CUDA(s, cudaMemcpyAsync(s->lev[0].x, p, nb, x2d, s->st));
    p += nb;
  }
  WL_CUDA(s, cudaMemcpyAsync(s->ds, p, sizeof(DevState), x2d, s->st));
  WL_CUDA(s, cudaStreamSynchronize(s->st));
  s->poisoned = false;
  return WL_OK;
}

// --------------------------------------------------------------- per-step metrics
extern "C" int wl_get_metrics(wl_handle s, double* out, int max_records, int* n_out) {
  if (!s || (!out && max_records > 0) || max_records < 0) return WL_EINVAL;
  int rc = sync_state(s);
  if (rc) return rc;
  const long long total = s->hs->mcount;
  const long long have = total < kMetricRing ? total : kMetricRing;
  const long long n = have < max_records ? have : max_records;
  std::vector<double> ring((size_t)NMETRIC * kMetricRing);
  WL_CUDA(s, cudaMemcpyAsync(ring.data(), s->mring, sizeof(double) * ring.size(), cudaMemcpyDeviceToHost, s->st));
  WL_CUDA(s, cudaStreamSynchronize(s->st));
  // the last n records, oldest first: ring slots (total - n) .. (total - 1) mod kMetricRing
  for (long long r = 0; r < n; ++r) {
    const long long slot = (total - n + r) % kMetricRing;
    std::memcpy(out + r * NMETRIC, ring.data() + slot * NMETRIC, sizeof(double) * NMETRIC);
  }
  if (n_out) *n_out = (int)n;
  return WL_OK;
}

// --------------------------------------------------------------- batched small simulations
namespace {

// A simulation goes into a batched launch when it is small and uses the options the
// batched kernels cover: the double-float pressure, FP32 levels, convection on, no
// convective exit, no per-step metric reductions, a small-level tail, at most
// kBatchLevels levels above it and kBatchPost sweeps; 3-D needs an even n_0.
bool batchable(const wl_sim* s, long long max_cells) {
  return s && !s->poisoned && s->g.nc <= max_cells && (s->D == 2 || s->D == 3) && s->ph && !s->g.exit &&
         s->o.coarse_precision == WL_COARSE_FP32 && s->o.advect && !s->o.metrics && s->tail_lf > 0 &&
         s->tail_lf <= kBatchLevels && s->o.post >= 1 && s->o.post <= kBatchPost &&
         (s->D == 2 || s->g.n[0] % 2 == 0);
}

BatchSlot batch_slot(wl_sim* s) {
  BatchSlot b{};
  b.ds = s->ds;
  b.D = s->D;
  b.stage[0] = stage_args(s, 1);
  b.stage[1] = stage_args(s, 2);
  b.stage[0].tz = b.stage[1].tz = 0;  // the batched launch's block map takes the default planes
  b.body = s->body;
  int lo[3], hi[3];
  b.band = (s->body.kind != 0 && stage_band_box(s->D, s->g, s->body, lo, hi)) ? 1 : 0;
  for (int d = 0; d < 3; ++d) {
    b.blo[d] = b.band ? lo[d] : 0;
    b.bn[d] = b.band ? hi[d] - lo[d] : 0;
  }
  b.div[0] = fine_res_args(s, RES_DIVERGENCE, 1, 1.f);
  b.div[1] = fine_res_args(s, RES_DIVERGENCE, 1, 0.5f);
  b.res = fine_res_args(s, RES_RESIDUAL, 0, 1.f);
  const int lf = s->tail_lf;
  b.nrestr = lf - 1;
  for (int l = 1; l < lf; ++l) b.restr[l] = res_args(s, l, RES_RESTRICT);
  b.nsmooth = lf;
  b.post = s->o.post;
  for (int l = 0; l < lf; ++l)
    for (int it = 0; it < s->o.post; ++it) b.sweep[l][it] = smooth_args(s, l, it);
  b.tail = tail_args(s, s->tail_lf);
  b.corr[0] = corr_args(s, s->ub, s->uc, 1.f, 0);
  b.corr[1] = corr_args(s, s->ub, s->ua, 0.5f, 1);
  b.w[0] = 1.f;
  b.w[1] = 0.5f;
  b.tol = s->o.tol;
  b.maxit = s->o.max_vcycles;
  b.nu = s->nu;
  b.dt_cap = s->o.dt_cap;
  b.dt_fixed = s->o.dt_fixed;
  b.ring = s->mring;
  b.ring_cap = kMetricRing;
  return b;
}

// a batched launch over the slots listed in `grid` (slot index, that slot's own grid)
BatchGrid batch_grid(const std::vector<std::pair<int, dim3>>& grid) {
  BatchGrid bg{};
  bg.n = (int)grid.size();
  int b = 0;
  for (int i = 0; i < bg.n; ++i) {
    bg.slot[i] = grid[i].first;
    bg.start[i] = b;
    bg.gx[i] = grid[i].second.x;
    bg.gy[i] = grid[i].second.y;
    b += (int)(grid[i].second.x * grid[i].second.y * grid[i].second.z);
  }
  bg.start[bg.n] = b;
  return bg;
}

}  // namespace

struct wl_batch_s {
  long long max_cells = 0;
  cudaStream_t cs = nullptr;  // capture stream
  struct Group {
    std::vector<unsigned long long> key;  // the slots (sim uids) of the current graph, in order
    BatchSlot* dtab = nullptr;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    cudaGraphConditionalHandle hc[2]{};
  } grp[2];  // 2-D and 3-D slots
  // the batched graphs run on the caller's stream, in order with everything else queued
  // there; events hand the slots' own streams over to it and back
  std::vector<cudaEvent_t> ev_in;  // one per slot: its own stream's work before the round
  cudaEvent_t ev_out = nullptr;    // the caller's stream after the batched graphs
  std::string err;
};

namespace {

int batch_fail(wl_batch_s* b, int code, const std::string& msg) {
  b->err = msg;
  return code;
}
#define WL_BCUDA(b, call)                                                         \
  do {                                                                            \
    cudaError_t _e = (call);                                                      \
    if (_e != cudaSuccess) return batch_fail((b), WL_ECUDA, std::string(#call) + ": " + cudaGetErrorString(_e)); \
  } while (0)

// One step of every slot of group G as a graph: the single-simulation step's launch
// sequence with each launch covering all slots, the two projections' V-cycle loops in
// conditional WHILE nodes that run while any slot's projection continues (a slot whose
// projection has converged skips the loop's launches).
int build_group_graph(wl_batch_s* b, wl_batch_s::Group& G, int D, const std::vector<BatchSlot>& slots) {
  const int n = (int)slots.size();
  std::vector<std::pair<int, dim3>> gs, gband[2], gres, gtail, gcorr[2], gall;
  int maxr = 0, maxs = 0, maxp = 0;
  size_t tail_smem = 0;
  for (int i = 0; i < n; ++i) {
    const BatchSlot& sl = slots[i];
    gs.push_back({i, stage_grid(D, sl.stage[0].g)});
    if (sl.band)
      for (int st = 0; st < 2; ++st) gband[st].push_back({i, band_grid(D, sl.bn)});
    gres.push_back({i, residual_grid(D, sl.res.g)});
    gtail.push_back({i, dim3(1, 1, 1)});
    for (int w = 0; w < 2; ++w) gcorr[w].push_back({i, correct_grid(D, sl.corr[w])});
    gall.push_back({i, dim3(1, 1, 1)});
    maxr = std::max(maxr, sl.nrestr);
    maxs = std::max(maxs, sl.nsmooth);
    maxp = std::max(maxp, sl.post);
    tail_smem = std::max(tail_smem, vcycle_tail_smem(D, sl.tail.n, sl.tail.nl));
  }
  std::vector<BatchGrid> grestr(maxr + 1), gsweep(maxs);
  for (int l = 1; l <= maxr; ++l) {
    std::vector<std::pair<int, dim3>> v;
    for (int i = 0; i < n; ++i)
      if (slots[i].nrestr >= l) v.push_back({i, restrict_grid(D, slots[i].restr[l])});
    grestr[l] = batch_grid(v);
  }
  for (int l = 0; l < maxs; ++l) {
    std::vector<std::pair<int, dim3>> v;
    for (int i = 0; i < n; ++i)
      if (slots[i].nsmooth > l) v.push_back({i, sweep_grid(D, slots[i].sweep[l][0])});
    gsweep[l] = batch_grid(v);
  }
  const BatchGrid bs = batch_grid(gs), bres = batch_grid(gres), btail = batch_grid(gtail), ball = batch_grid(gall);
  const BatchGrid bband[2] = {batch_grid(gband[0]), batch_grid(gband[1])};
  const BatchGrid bcorr[2] = {batch_grid(gcorr[0]), batch_grid(gcorr[1])};
  const BatchSlot* t = G.dtab;

  cudaGraph_t g = nullptr;
  WL_BCUDA(b, cudaGraphCreate(&g, 0));
  for (int p = 0; p < 2; ++p) WL_BCUDA(b, cudaGraphConditionalHandleCreate(&G.hc[p], g, 0, 0));
  auto vcycle = [&](int proj) {
    for (int l = 1; l <= maxr; ++l) launch_batch_restrict(D, t, grestr[l], l, b->cs);
    launch_batch_tail(D, t, btail, tail_smem, b->cs);
    for (int l = maxs - 1; l >= 0; --l)
      for (int it = 0; it < maxp; ++it) launch_batch_sweep(D, t, gsweep[l], l, it, b->cs);
    launch_batch_residual(D, t, bres, 2, 1, b->cs);
    launch_batch_decide(t, ball, G.hc[proj], 0, proj, b->cs);
  };
  std::vector<cudaGraphNode_t> leaf;
  cudaGraph_t out = nullptr;
  cudaGraphNode_t prev = nullptr;
  for (int proj = 0; proj < 2; ++proj) {
    WL_BCUDA(b, cudaStreamBeginCaptureToGraph(b->cs, g, prev ? &prev : nullptr, nullptr, prev ? 1 : 0,
                                              cudaStreamCaptureModeThreadLocal));
    if (proj == 1) launch_batch_correct(D, t, bcorr[0], 0, b->cs);
    launch_batch_stage(D, t, bs, proj + 1, b->cs);
    launch_batch_band(D, t, bband[proj], proj + 1, b->cs);
    launch_batch_residual(D, t, bres, proj, 0, b->cs);
    launch_batch_decide(t, ball, G.hc[proj], 1, proj, b->cs);
    {
      cudaStreamCaptureStatus cst;
      const cudaGraphNode_t* deps = nullptr;
      size_t nd = 0;
      WL_BCUDA(b, cudaStreamGetCaptureInfo(b->cs, &cst, nullptr, nullptr, &deps, nullptr, &nd));
      leaf.assign(deps, deps + nd);
    }
    WL_BCUDA(b, cudaStreamEndCapture(b->cs, &out));
    cudaGraphNodeParams cp{};
    cp.type = cudaGraphNodeTypeConditional;
    cp.conditional.handle = G.hc[proj];
    cp.conditional.type = cudaGraphCondTypeWhile;
    cp.conditional.size = 1;
    cudaGraphNode_t wnode;
    WL_BCUDA(b, cudaGraphAddNode(&wnode, g, leaf.data(), nullptr, leaf.size(), &cp));
    WL_BCUDA(b, cudaStreamBeginCaptureToGraph(b->cs, cp.conditional.phGraph_out[0], nullptr, nullptr, 0,
                                              cudaStreamCaptureModeThreadLocal));
    vcycle(proj);
    WL_BCUDA(b, cudaStreamEndCapture(b->cs, &out));
    prev = wnode;
  }
  WL_BCUDA(b, cudaStreamBeginCaptureToGraph(b->cs, g, &prev, nullptr, 1, cudaStreamCaptureModeThreadLocal));
  launch_batch_correct(D, t, bcorr[1], 1, b->cs);
  launch_batch_step_end(t, ball, b->cs);
  WL_BCUDA(b, cudaStreamEndCapture(b->cs, &out));
  if (G.exec) cudaGraphExecDestroy(G.exec);
  if (G.graph) cudaGraphDestroy(G.graph);
  G.exec = nullptr;
  G.graph = g;
  WL_BCUDA(b, cudaGraphInstantiate(&G.exec, g, 0));
  return WL_OK;
}

}  // namespace

extern "C" int wl_batch_create(long long max_cells, wl_batch* out) {
  if (!out || max_cells < 0) return WL_EINVAL;
  *out = nullptr;
  auto* b = new wl_batch_s();
  b->max_cells = max_cells;
  bool ok = cudaStreamCreateWithFlags(&b->cs, cudaStreamNonBlocking) == cudaSuccess;
  ok = ok && cudaEventCreateWithFlags(&b->ev_out, cudaEventDisableTiming) == cudaSuccess;
  b->ev_in.assign(2 * kBatchMax, nullptr);
  for (auto& e : b->ev_in) ok = ok && cudaEventCreateWithFlags(&e, cudaEventDisableTiming) == cudaSuccess;
  for (auto& G : b->grp) ok = ok && cudaMalloc(&G.dtab, sizeof(BatchSlot) * kBatchMax) == cudaSuccess;
  if (!ok) {
    cudaGetLastError();
    wl_batch_destroy(b);
    return WL_ECUDA;
  }
  *out = b;
  return WL_OK;
}

extern "C" void wl_batch_destroy(wl_batch b) {
  if (!b) return;
  cudaDeviceSynchronize();  // no batched graph is still running
  for (auto& G : b->grp) {
    if (G.exec) cudaGraphExecDestroy(G.exec);
    if (G.graph) cudaGraphDestroy(G.graph);
    if (G.dtab) cudaFree(G.dtab);
  }
  for (auto& e : b->ev_in)
    if (e) cudaEventDestroy(e);
  if (b->ev_out) cudaEventDestroy(b->ev_out);
  if (b->cs) cudaStreamDestroy(b->cs);
  delete b;
}

extern "C" const char* wl_batch_last_error(wl_batch b) { return b ? b->err.c_str() : "null batch"; }

extern "C" int wl_batch_step(wl_batch b, const wl_handle* hs, int n, void* stream, void* small_done) {
  if (!b || (!hs && n > 0) || n < 0) return WL_EINVAL;
  cudaStream_t cs = (cudaStream_t)stream;
  cudaEvent_t fork = nullptr;
  WL_BCUDA(b, cudaEventCreateWithFlags(&fork, cudaEventDisableTiming));
  WL_BCUDA(b, cudaEventRecord(fork, cs));
  int first = WL_OK;
  std::vector<wl_sim*> small[2], large;
  for (int i = 0; i < n; ++i) {
    wl_sim* s = hs[i];
    if (!s) {
      if (first == WL_OK) first = WL_EINVAL;
      continue;
    }
    if (s->poisoned) {
      if (first == WL_OK) first = WL_ENONFINITE;
      continue;
    }
    const int gi = s->D - 2;
    if (batchable(s, b->max_cells) && (int)small[gi].size() < kBatchMax)
      small[gi].push_back(s);
    else
      large.push_back(s);
  }
  // the large simulations: each its own step graph on its own stream
  for (wl_sim* s : large) {
    int rc = WL_OK;
    if (cudaStreamWaitEvent(s->st, fork, 0) != cudaSuccess) rc = WL_ECUDA;
    if (rc == WL_OK && !s->exec) rc = build_step_graph(s);
    if (rc == WL_OK && cudaGraphLaunch(s->exec, s->st) != cudaSuccess) rc = WL_ECUDA;
    if (rc == WL_OK && !s->join && cudaEventCreateWithFlags(&s->join, cudaEventDisableTiming) != cudaSuccess)
      rc = WL_ECUDA;
    if (rc == WL_OK && cudaEventRecord(s->join, s->st) != cudaSuccess) rc = WL_ECUDA;
    if (rc != WL_OK) {
      cudaGetLastError();
      if (first == WL_OK) first = rc;
    }
  }
  // the small ones: one batched graph per dimension, on the caller's stream after the work
  // already queued on each slot's own stream (every batched kernel, table upload and graph
  // rebuild is then in order with the caller's stream)
  int ne = 0;
  for (int gi = 0; gi < 2; ++gi)
    for (wl_sim* s : small[gi]) {
      WL_BCUDA(b, cudaEventRecord(b->ev_in[ne], s->st));
      WL_BCUDA(b, cudaStreamWaitEvent(cs, b->ev_in[ne], 0));
      ++ne;
    }
  for (int gi = 0; gi < 2; ++gi) {
    auto& G = b->grp[gi];
    auto& v = small[gi];
    if (v.empty()) continue;
    std::vector<unsigned long long> key;
    for (wl_sim* s : v) key.push_back(s->uid);
    if (key != G.key) {
      std::vector<BatchSlot> slots;
      for (wl_sim* s : v) slots.push_back(batch_slot(s));
      // in stream order after the previous graph that read the table (a pageable source is
      // staged before the call returns, so `slots` may go)
      WL_BCUDA(b, cudaMemcpyAsync(G.dtab, slots.data(), sizeof(BatchSlot) * slots.size(), cudaMemcpyHostToDevice,
                                  cs));
      G.key.clear();
      int rc = build_group_graph(b, G, gi + 2, slots);
      if (rc) return rc;
      G.key = key;
    }
    WL_BCUDA(b, cudaGraphLaunch(G.exec, cs));
  }
  if (ne > 0) {
    WL_BCUDA(b, cudaEventRecord(b->ev_out, cs));
    for (int gi = 0; gi < 2; ++gi)
      for (wl_sim* s : small[gi]) WL_BCUDA(b, cudaStreamWaitEvent(s->st, b->ev_out, 0));  // later work on the slot
  }
  if (small_done) WL_BCUDA(b, cudaEventRecord((cudaEvent_t)small_done, cs));
  for (wl_sim* s : large)
    if (s->join) cudaStreamWaitEvent(cs, s->join, 0);
  cudaEventDestroy(fork);
  if (cudaGetLastError() != cudaSuccess && first == WL_OK) first = WL_ECUDA;
  return first;
}

extern "C" int wl_event_elapsed(void* start, void* end, float* ms) {
  if (!start || !end || !ms) return WL_EINVAL;
  return cudaEventElapsedTime(ms, (cudaEvent_t)start, (cudaEvent_t)end) == cudaSuccess ? WL_OK : WL_ECUDA;
}

extern "C" int wl_debug_bounds(wl_handle s, unsigned* flags) {
  if (!s || !flags) return WL_EINVAL;
  *flags = 0u;
#ifdef WL_DEBUG_BOUNDS
  WL_CUDA(s, cudaStreamSynchronize(s->st));
  unsigned f = dbg_take_momentum() | dbg_take_poisson() | dbg_take_sweep();
  std::vector<unsigned char> buf(kCanary);
  for (size_t off : s->canaries) {
    WL_CUDA(s, cudaMemcpy(buf.data(), s->ws + off, kCanary, cudaMemcpyDeviceToHost));
    for (unsigned char c : buf)
      if (c != 0xA5) f |= 0x80000000u;
  }
  *flags = f;
  return WL_OK;
#else
  return WL_NODEBUG;
#endif
}
