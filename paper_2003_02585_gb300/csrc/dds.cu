// libdds C ABI (include/dds.h): set-up, sweeps, FGMRES and helpers.
//
// Host code only; every arithmetic step of set-up and solve runs in the kernels of
// k_factor.cu, k_sweep.cu and k_krylov.cu.  The host builds the small tables (PML stretching,
// line-block coefficients, routing, step schedules) and drives the launches.
#include <algorithm>
#include <array>
#include <atomic>
#include <chrono>
#include <cmath>
#include <complex>
#include <cstdio>
#include <cstring>
#include <new>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <string>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "../../include/dds.h"
#include "dds_internal.cuh"

using namespace dds;
using cd = std::complex<double>;

namespace {

// Device bytes held on behalf of one context and its cap (0 = none).  Allocations made while a
// context's call runs (inside its Busy guard, or its set-up) count against that context.
struct MemAcct {
  std::atomic<size_t> used{0};   // (a server may release its slots from another thread)
  size_t budget = 0;
};
thread_local MemAcct *tl_acct = nullptr;

struct DBuf {
  void *p = nullptr;
  size_t n = 0;
  MemAcct *acct = nullptr;   // the context charged for these bytes
  DBuf() = default;
  DBuf(const DBuf &) = delete;
  DBuf &operator=(const DBuf &) = delete;
  ~DBuf() { release(); }
  void release() {
    if (p) {
      cudaFree(p);
      if (acct) acct->used -= n;
    }
    p = nullptr;
    n = 0;
    acct = nullptr;
  }
  cudaError_t ensure(size_t bytes) {
    if (bytes <= n && p) return cudaSuccess;
    release();
    if (bytes == 0) bytes = 16;
    MemAcct *a = tl_acct;
    if (a && a->budget && a->used + bytes > a->budget) return cudaErrorMemoryAllocation;
    cudaError_t e = cudaMalloc(&p, bytes);
    if (e == cudaSuccess) {
      n = bytes;
      acct = a;
      if (a) a->used += bytes;
    } else {
      p = nullptr;
      cudaGetLastError();   // a failed allocation must not surface at a later launch check
    }
    return e;
  }
  template <class T> T *as() const { return reinterpret_cast<T *>(p); }
};

// NVTX range over a scope (host side): the API calls, each DDM application, each FGMRES
// iteration and, outside graph capture, each sweep step, so that a timeline tool shows the
// method's structure.  Without a tool attached the calls do nothing.
struct NvtxRange {
  explicit NvtxRange(const char *name) { nvtxRangePushA(name); }
  ~NvtxRange() { nvtxRangePop(); }
  NvtxRange(const NvtxRange &) = delete;
  NvtxRange &operator=(const NvtxRange &) = delete;
};

struct StepPlan {            // launch lists of one (direction, step) or one phase
  int col_off = 0, ncols = 0;
  int pan_off = 0, npanels = 0, pc = 1;
  int grp_off = 0, ngrp = 0;   // factor groups of the panels (zero-work skipping)
};

// right-hand sides per call: the batched FP64 kernels put the RHS on gridDim.y
constexpr int kMaxRhs = 65535;
// sweeps of one strip-DDM call (dds_sweep_strip)
constexpr int kMaxStripSweeps = 64;

struct CallPlan {            // all launch lists for one nrhs
  int nrhs = 0;
  std::vector<StepPlan> steps;   // [dir][step] for the direct plan (substitution panels)
  std::vector<StepPlan> tsteps;  // [dir][step] for the trace plan (trace-step panels)
  StepPlan all;                  // every (sub, rhs) column (trace plan phases, local solves)
  DBuf cols, panels, tpanels;
  // zero-work skipping: factor groups of every substitution launch, and the packed column and
  // panel lists that k_compact_panels writes (same index space as cols / panels)
  DBuf groups, dcols, dpans;
  struct TraceTable {
    int n = -1, nlev = 0;
    DBuf buf, cols, levs;            // k_trace_sweeps: items, their columns, level offsets
    int tn = -1, tnlev = 0, tslots = 0;
    DBuf tunits, tcols;              // k_trace_tc: units, their columns
    DBuf tuoff, tcunits, tcoff, tchunks;   // k_trace_tc: per-CTA unit and chunk streams
    int tG = 0;                      // k_trace_tc: CTAs the streams were dealt to
    DBuf tneed, tready;              // k_trace_tc: publications expected / made per slot
  };
  std::map<int, TraceTable> trace_steps;   // rounds -> item lists of the cooperative launch
};

}  // namespace

// releases a server's device memory and detaches it from its context (defined with the server)
void server_orphan(dds_server *srv);

struct dds_ctx {
  MemAcct acct;   // first member: destroyed after every buffer that reports to it
  std::mutex mu;
  std::string err;
  Geom g{};
  int precision = 0, plan = 0;
  bool single = false;   // sweeps in complex single precision (every precision but DDS_FP64)
  int split = -1;        // tensor-core substitution pieces: 0 = TF32, 1 = BF16, -1 = none
  int tc_m = 0;          // middle block of the two-sided tensor-core chain (0: one-sided)
  int tune_pc = 0;       // tensor-core panel width chosen by dds_autotune (0: automatic)
  int tune_np = 1;       // tensor-core panels per CTA (or CTA pair) chosen by dds_autotune
  int trace_per_sm = 2;  // CTAs per SM of the cooperative trace launch
  double h = 0, omega = 0, S = 0;
  int P = 0, power = 2, H = 0;
  cudaStream_t stream = nullptr;
  long long launches = 0;
  double setup_seconds = 0;
  int nfac = 0;
  std::vector<int> fac_of_sub;
  std::vector<std::vector<std::vector<int>>> step_subs;  // [dir][step] -> subs (by factor)
  int nsteps = 0, ndirs = 0;
  // device tables
  DBuf sinv64, sinv32, cpl64, cpl32, coef64, coef32, k2glob, gmap64, gmap32, status;
  DBuf tctiles;  // block inverses split into tensor-core pieces (layout of k_subst_tc.cu)
  DBuf bigtiles, bigB, bigacc;   // blocks wider than 128 nodes: tiles, B pieces, accumulator
  DBuf tttiles;          // the trace map split into tensor-core pieces (k_trace_tc.cu)
  bool trace_tc_avail = false;  // tttiles exist
  bool trace_tc = false; // trace solves on the tensor cores (k_trace_tc) or CUDA cores
  bool big_tc = false;
  DBuf errflag;  // set by kernels whose bounded waits gave up
  DBuf gbar;     // step counters of the cooperative trace-sweep launch
  DBuf nzflag;   // per work slot: the assembled right-hand side has a nonzero entry
  DBuf badrhs;   // per RHS of a DDM application: its source has a NaN or infinite entry
  bool zero_skip = true;   // drop the substitutions of zero right-hand sides (Algorithm 2.1)
  unsigned wait_limit = 1u << 20;   // polls of a level-completion wait before it gives up
  DBuf solve_stats;        // [0] local solves run, [1] local solves assembled (u64)
  DBuf an_glob[3], iah_glob[3];
  DBuf stc0, stcp[3];  // global stencil (centre, coupling to +e_a)
  Tables tb{};
  // per-call workspaces
  std::map<int, std::unique_ptr<CallPlan>> plans;
  std::map<int, std::vector<int>> routes;  // rounds -> route[L][6]
  DBuf route_dev;
  int route_rounds = -1;
  std::vector<int> in_mask, out_mask;  // per sweep: sides that can receive / must send a trace
  DBuf work, gtr, acc, rawf, bbuf, stage_in, stage_out, dots_part, dots_out, coefbuf, scalebuf;
  DBuf Vbig, Zbig;   // Krylov bases
  // CUDA graphs of whole DDM applications, keyed by (b, u, nrhs, rounds); captured on gstream
  // servers made on this context: destroying the context first releases their device memory
  // (while its accounting still exists) and leaves them orphaned
  std::vector<dds_server *> servers;
  struct GraphEntry { cudaGraphExec_t exec = nullptr; long long nodes = 0; };
  std::map<std::array<long long, 4>, GraphEntry> graphs;
  cudaStream_t gstream = nullptr;
  cudaEvent_t gev[2] = {nullptr, nullptr};
  // host results: the solution's device-to-host copy runs on its own stream, overlapping the
  // final true-residual computation
  cudaStream_t out_stream = nullptr;
  cudaEvent_t out_ev = nullptr;
  bool use_graphs = true;
  void clear_graphs() {
    for (auto &kv : graphs)
      if (kv.second.exec) cudaGraphExecDestroy(kv.second.exec);
    graphs.clear();
  }
  // profiler: event pairs around launches, folded into per-kind totals on read
  bool profiling = false;
  std::vector<std::array<cudaEvent_t, 2>> ev_pool;
  std::vector<int> ev_kind;
  size_t ev_used = 0;
  long long prof_count[DDS_K_COUNT] = {0};
  double prof_ms[DDS_K_COUNT] = {0};
  ~dds_ctx() {
    clear_graphs();
    if (gstream) cudaStreamDestroy(gstream);
    if (out_stream) cudaStreamDestroy(out_stream);
    if (out_ev) cudaEventDestroy(out_ev);
    for (auto &e : gev)
      if (e) cudaEventDestroy(e);
    for (auto &e : ev_pool) {
      cudaEventDestroy(e[0]);
      cudaEventDestroy(e[1]);
    }
  }
};

namespace {

#define CK(call)                                                                 \
  do {                                                                           \
    cudaError_t e_ = (call);                                                     \
    if (e_ != cudaSuccess) {                                                     \
      ctx->err = std::string(#call) + ": " + cudaGetErrorString(e_);             \
      return e_ == cudaErrorMemoryAllocation ? DDS_ENOMEM : DDS_ECUDA;           \
    }                                                                            \
  } while (0)

// launch of kernel family `kind`, timed with an event pair when profiling is on
#define LAUNCHK(kind, call)                                                      \
  do {                                                                           \
    ++ctx->launches;                                                             \
    cudaEvent_t *ev_ = prof_begin(ctx, kind);                                    \
    CK(call);                                                                    \
    if (ev_) CK(cudaEventRecord(ev_[1], ctx->stream));                           \
  } while (0)
#define LAUNCH(call) LAUNCHK(DDS_K_OTHER, call)

cudaEvent_t *prof_begin(dds_ctx *ctx, int kind) {
  if (!ctx->profiling) return nullptr;
  if (ctx->ev_used == ctx->ev_pool.size()) {
    std::array<cudaEvent_t, 2> e;
    if (cudaEventCreate(&e[0]) != cudaSuccess) return nullptr;
    if (cudaEventCreate(&e[1]) != cudaSuccess) { cudaEventDestroy(e[0]); return nullptr; }
    ctx->ev_pool.push_back(e);
    ctx->ev_kind.push_back(kind);
  }
  ctx->ev_kind[ctx->ev_used] = kind;
  cudaEvent_t *e = ctx->ev_pool[ctx->ev_used].data();
  if (cudaEventRecord(e[0], ctx->stream) != cudaSuccess) return nullptr;
  ++ctx->ev_used;
  return e;
}

// fold recorded event pairs into the per-kind totals (synchronises the stream)
cudaError_t prof_fold(dds_ctx *ctx) {
  if (ctx->ev_used == 0) return cudaSuccess;
  cudaError_t e = cudaStreamSynchronize(ctx->stream);
  if (e != cudaSuccess) return e;
  for (size_t i = 0; i < ctx->ev_used; ++i) {
    float ms = 0.f;
    e = cudaEventElapsedTime(&ms, ctx->ev_pool[i][0], ctx->ev_pool[i][1]);
    if (e != cudaSuccess) return e;
    ctx->prof_count[ctx->ev_kind[i]] += 1;
    ctx->prof_ms[ctx->ev_kind[i]] += ms;
  }
  ctx->ev_used = 0;
  return cudaSuccess;
}

// ---------------------------------------------------------------------------- PML tables ----
// sigma(t) = S ((t/h - H) / P)^power beyond the halo, alpha = 1 + i sigma  (Eq. 2.1-2.2)
cd alpha_at(double t_over_h, int H, int P, double S, int power) {
  double s = 0.0;
  if (t_over_h > H) s = S * std::pow((t_over_h - H) / P, power);
  return cd(1.0, s);
}

// alphas on an axis of `count` nodes whose node p sits at (p + first) h, box [0, len] (in h)
void axis_alphas(int count, double first, double len, int H, int P, double S, int power,
                 std::vector<cd> &an, std::vector<cd> &ah) {
  an.resize(count);
  ah.resize(count + 1);
  auto dist = [&](double x) { return std::max(std::max(-x, x - len), 0.0); };
  for (int p = 0; p < count; ++p) an[p] = alpha_at(dist(p + first), H, P, S, power);
  for (int q = 0; q <= count; ++q) ah[q] = alpha_at(dist(q - 0.5 + first), H, P, S, power);
}

std::vector<std::array<int, 3>> sweep_dirs(int dim) {
  // Eq. 2.9 / Eq. 4.2: x1 flips fastest, then x2, then x3
  std::vector<std::array<int, 3>> d;
  for (int i = 0; i < (1 << dim); ++i) {
    std::array<int, 3> v{0, 0, 0};
    for (int a = 0; a < dim; ++a) v[a] = ((i >> a) & 1) ? -1 : 1;
    d.push_back(v);
  }
  return d;
}

bool similar(const int *v1, const int *v2, int dim) {
  // Section 2.3 (2D): v1 . v2 > 0; Section 4 (3D): also v1(k) v2(k) >= 0 for every k
  int dot = 0;
  bool comp = true;
  for (int a = 0; a < dim; ++a) {
    dot += v1[a] * v2[a];
    if (v1[a] * v2[a] < 0) comp = false;
  }
  return dim == 2 ? dot > 0 : (dot > 0 && comp);
}

bool barred(const int *D, const int *dgen, const int *duse, int dim) {
  if (dim == 2) {  // Rule 2.5: opposite sweep directions
    return dgen[0] == -duse[0] && dgen[1] == -duse[1];
  }
  // Rule 4.2: a plane projection where D has exactly one zero and the sweeps are opposite
  const int pl[3][2] = {{0, 1}, {0, 2}, {1, 2}};
  for (auto &pq : pl) {
    const int zeros = (D[pq[0]] == 0) + (D[pq[1]] == 0);
    if (zeros != 1) continue;
    if (dgen[pq[0]] == -duse[pq[0]] && dgen[pq[1]] == -duse[pq[1]]) return true;
  }
  return false;
}

// Sweep program of one DDM application, as indices into sweep_dirs(dim).  prog >= 1: `prog`
// rounds of the 2^n diagonal sweeps in the order of Eq. 2.9 / 4.2.  prog <= -1: the
// one-dimensional sweeping DDM of Section 3.2 on a strip partition (one axis a with N_a > 1):
// -prog sweeps along a, forward (+) first, then alternating; every other component is +1 (no
// neighbour lies along it).  Two strip sweeps are Algorithm 2.1 / 4.1 on the strip with its
// empty sweeps left out; the third is the extra forward sweep of Theorem 3.6.
std::vector<int> sweep_program(const Geom &g, int prog) {
  std::vector<int> seq;
  const int nd = 1 << g.dim;
  if (prog >= 1) {
    for (int l = 0; l < nd * prog; ++l) seq.push_back(l % nd);
    return seq;
  }
  int a = g.dim - 1;
  for (int b = 0; b < g.dim; ++b)
    if (g.parts[b] > 1) a = b;
  for (int k = 0; k < -prog; ++k) seq.push_back((k & 1) ? (1 << a) : 0);
  return seq;
}

// a strip partition: at most one axis cut into more than one part
bool is_strip(const Geom &g) {
  int cut = 0;
  for (int b = 0; b < g.dim; ++b) cut += g.parts[b] > 1;
  return cut <= 1;
}

std::vector<int> build_route(const Geom &g, int prog) {
  const int dim = g.dim;
  const auto dirs = sweep_dirs(dim);
  const std::vector<int> seq = sweep_program(g, prog);
  const int L = (int)seq.size();
  std::vector<int> route(L * 6, -1);
  for (int l = 0; l < L; ++l) {
    for (int d = 0; d < 2 * dim; ++d) {
      int D[3] = {0, 0, 0};
      D[d >> 1] = (d & 1) ? -1 : 1;
      for (int lp = l; lp < L; ++lp) {
        // Rule 2.4 / 4.1 and Rule 2.5 / 4.2: smallest usable sweep
        if (!similar(D, dirs[seq[lp]].data(), dim)) continue;
        if (lp > l && barred(D, dirs[seq[l]].data(), dirs[seq[lp]].data(), dim)) continue;
        route[l * 6 + d] = lp;
        break;
      }
    }
  }
  return route;
}

bool is_device_ptr(const void *p) {
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

template <class T> cudaError_t upload(DBuf &b, const std::vector<T> &v, cudaStream_t st) {
  cudaError_t e = b.ensure(v.size() * sizeof(T));
  if (e != cudaSuccess) return e;
  if (v.empty()) return cudaSuccess;
  e = cudaMemcpyAsync(b.p, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice, st);
  if (e != cudaSuccess) return e;
  return cudaStreamSynchronize(st);
}

int pick_pc(int ncols, int max_pc) {
  // widest panel that still leaves about two CTAs per SM of independent panels
  int pc = 1;
  while (pc * 2 <= max_pc && ncols / (pc * 2) >= 2 * 152) pc *= 2;
  return pc;
}

int pick_pc_stream(const Geom &g, int ncols);

int pick_pc_tc(const Geom &g, int split, bool twisted, int ncols) {
  // the tensor-core kernel holds one CTA per SM (two per panel for the two-sided chain) and its
  // MMA time does not depend on the panel width: the narrowest panel (8, 16 or 32 columns)
  // that fits the columns into one wave
  const int per = twisted ? 2 : 1;
  int pc = 8;
  while (pc < 32 && per * ((ncols + pc - 1) / pc) > 152 && subst_tc_ok(g, split, pc * 2, twisted))
    pc *= 2;
  return subst_tc_ok(g, split, pc, twisted) ? pc : 0;
}

int pick_pc_stream(const Geom &g, int ncols) {
  // the streamed kernel holds one CTA per SM: the narrowest panel that fits the columns into
  // one wave of 152 CTAs, widened further only while the shared memory allows
  int pc = 1;
  while (pc < 16 && (ncols + pc - 1) / pc > 152 && subst_stream_ok(g, pc * 2)) pc *= 2;
  return subst_stream_ok(g, pc) ? pc : 0;
}

void add_panels(const std::vector<Col> &cols, int c0, int c1, const std::vector<int> &fac, int pc,
                std::vector<Panel> &panels) {
  int i = c0;
  while (i < c1) {
    const int f = fac[cols[i].sub];
    int j = i;
    while (j < c1 && j - i < pc && fac[cols[j].sub] == f) ++j;
    panels.push_back(Panel{i, j - i, f, 0});
    i = j;
  }
}

int max_pc_for(const dds_ctx *ctx, size_t elem) {
  // shared memory of the substitution panel: Mb * pc * elem bytes (<= 96 KB)
  int pc = 8;
  while (pc > 1 && (size_t)ctx->g.Mb * pc * elem > 96 * 1024) pc /= 2;
  return pc;
}

CallPlan *get_plan(dds_ctx *ctx, int nrhs) {
  auto it = ctx->plans.find(nrhs);
  if (it != ctx->plans.end()) return it->second.get();
  auto cp = std::make_unique<CallPlan>();
  cp->nrhs = nrhs;
  const Geom &g = ctx->g;
  const size_t elem = ctx->single ? sizeof(float2) : sizeof(double2);
  const int maxpc = max_pc_for(ctx, elem);
  std::vector<Col> cols;
  std::vector<Panel> panels;
  std::vector<int4> groups;
  // every (sub, rhs), subs grouped by factor
  std::vector<int> order(g.nsub);
  for (int s = 0; s < g.nsub; ++s) order[s] = s;
  std::stable_sort(order.begin(), order.end(),
                   [&](int a, int b) { return ctx->fac_of_sub[a] < ctx->fac_of_sub[b]; });
  auto emit = [&](const std::vector<int> &subs, int pc_cap, bool trace) {
    StepPlan sp;
    sp.col_off = (int)cols.size();
    for (size_t i = 0; i < subs.size(); ++i)
      for (int r = 0; r < nrhs; ++r)
        cols.push_back(Col{subs[i], r, (int)(cols.size() - sp.col_off), 0});
    sp.ncols = (int)cols.size() - sp.col_off;
    if (trace) {  // trace-step panels of 8 columns (4 or 2 where the inputs would not fit)
      sp.pc = pc_cap;
    } else {
      int spc = 0;
      if (ctx->single && ctx->big_tc) {
        spc = sp.ncols <= 8 ? 8 : (sp.ncols <= 16 ? 16 : 32);
      } else if (ctx->single && ctx->split >= 0) {
        spc = pick_pc_tc(ctx->g, ctx->split, ctx->tc_m > 0, sp.ncols);
        if (ctx->tune_pc > 0 && subst_tc_ok(ctx->g, ctx->split, ctx->tune_pc, ctx->tc_m > 0))
          spc = ctx->tune_pc;
      }
      if (ctx->single && spc == 0) spc = pick_pc_stream(ctx->g, sp.ncols);
      sp.pc = spc > 0 ? spc : pick_pc(sp.ncols, pc_cap);
    }
    sp.pan_off = (int)panels.size();
    add_panels(cols, sp.col_off, sp.col_off + sp.ncols, ctx->fac_of_sub, sp.pc, panels);
    sp.npanels = (int)panels.size() - sp.pan_off;
    if (!trace) {
      // runs of panels sharing a factor: the units of zero-work compaction
      sp.grp_off = (int)groups.size();
      for (int q = sp.pan_off; q < sp.pan_off + sp.npanels;) {
        int e = q;
        while (e < sp.pan_off + sp.npanels && panels[e].factor == panels[q].factor) ++e;
        groups.push_back(make_int4(panels[q].col0, panels[e - 1].col0 + panels[e - 1].ncol, q, e));
        q = e;
      }
      sp.ngrp = (int)groups.size() - sp.grp_off;
    }
    return sp;
  };
  cp->all = emit(order, maxpc, false);
  for (int dir = 0; dir < ctx->ndirs; ++dir)
    for (int s = 0; s < ctx->nsteps; ++s) cp->steps.push_back(emit(ctx->step_subs[dir][s], maxpc, false));
  const int tmax = 8;   // trace-step panels: 8 columns
  for (int dir = 0; dir < ctx->ndirs; ++dir)
    for (int s = 0; s < ctx->nsteps; ++s) cp->tsteps.push_back(emit(ctx->step_subs[dir][s], tmax, true));
  if (upload(cp->cols, cols, ctx->stream) != cudaSuccess) return nullptr;
  if (upload(cp->panels, panels, ctx->stream) != cudaSuccess) return nullptr;
  if (upload(cp->groups, groups, ctx->stream) != cudaSuccess) return nullptr;
  if (cp->dcols.ensure(cols.size() * sizeof(Col)) != cudaSuccess) return nullptr;
  if (cp->dpans.ensure(panels.size() * sizeof(Panel)) != cudaSuccess) return nullptr;
  // trace-step panels with their columns inline (panels wider than 8 columns keep the first 8,
  // and only trace-step panels, which have at most 8, are read through this table)
  std::vector<TracePanel> tp(panels.size());
  for (size_t i = 0; i < panels.size(); ++i) {
    TracePanel t{};
    t.factor = panels[i].factor;
    t.ncol = std::min(panels[i].ncol, 8);
    for (int c = 0; c < t.ncol; ++c) {
      t.sub[c] = cols[panels[i].col0 + c].sub;
      t.rhs[c] = cols[panels[i].col0 + c].rhs;
    }
    tp[i] = t;
  }
  if (upload(cp->tpanels, tp, ctx->stream) != cudaSuccess) return nullptr;
  CallPlan *raw = cp.get();
  ctx->plans[nrhs] = std::move(cp);
  return raw;
}

dds_status set_route(dds_ctx *ctx, int rounds) {
  if (ctx->route_rounds == rounds) return DDS_OK;
  const std::vector<int> r = build_route(ctx->g, rounds);
  CK(upload(ctx->route_dev, r, ctx->stream));
  const int L = (int)r.size() / 6, ns = 2 * ctx->g.dim;
  ctx->in_mask.assign(L, 0);
  ctx->out_mask.assign(L, 0);
  for (int l = 0; l < L; ++l)
    for (int d = 0; d < ns; ++d) {
      const int lp = r[l * 6 + d];
      if (lp < 0) continue;
      ctx->out_mask[l] |= 1 << d;          // side d of a sweep-l solve sends a trace
      ctx->in_mask[lp] |= 1 << (d ^ 1);    // ... which the neighbour receives on side d^1
    }
  ctx->route_rounds = rounds;
  return DDS_OK;
}

// substitutions of a panel list: the shared-memory-streamed FP32 kernel where it fits (pc up to
// 16), else the direct-load kernel (pc up to 8)
template <typename R>
cudaError_t subst_any(dds_ctx *ctx, int npan, const Panel *pans, const Col *cols,
                      const typename Cx<R>::T *sinv, const typename Cx<R>::T *cpl,
                      typename Cx<R>::T *work, int pc, const int *nz = nullptr) {
  if constexpr (sizeof(R) == 4) {
    if (ctx->big_tc) {
      // all columns of the launch, stage by stage over the whole GPU: K-split so that the units
      // of one stage fill about two waves of SMs
      const Geom &g = ctx->g;
      const int rt = (g.Mb + 127) / 128;
      const int ksplit = std::max(1, (2 * 152 + rt * npan - 1) / (rt * npan));
      size_t acc_bytes = 0;
      const size_t bbytes = big_scratch_bytes(g, ctx->split, pc, npan, &acc_bytes);
      if (ctx->bigB.n < bbytes || ctx->bigacc.n < acc_bytes) return cudaErrorInvalidValue;
      cudaError_t e = cudaMemsetAsync(ctx->bigB.p, 0, bbytes, ctx->stream);
      if (e == cudaSuccess) e = cudaMemsetAsync(ctx->bigacc.p, 0, acc_bytes, ctx->stream);
      if (e != cudaSuccess) return e;
      return launch_subst_big(ctx->stream, g, ctx->split, npan, pans, cols,
                              ctx->bigtiles.as<unsigned char>(), cpl, work, pc, ksplit,
                              ctx->bigacc.as<float2>(), ctx->bigB.as<unsigned char>(),
                              ctx->errflag.as<int>(), &ctx->launches);
    }
    if (ctx->split >= 0 && subst_tc_ok(ctx->g, ctx->split, pc, ctx->tc_m > 0)) {
      const int np = subst_tc_ok(ctx->g, ctx->split, pc, ctx->tc_m > 0, ctx->tune_np) ? ctx->tune_np : 1;
      return launch_subst_tc(ctx->stream, ctx->g, ctx->split, npan, pans, cols,
                             ctx->tctiles.as<unsigned char>(), cpl, work, pc,
                             ctx->errflag.as<int>(), ctx->tc_m, nz, np);
    }
    if (subst_stream_ok(ctx->g, pc))
      return launch_subst_stream(ctx->stream, ctx->g, npan, pans, cols, sinv, cpl, work, pc,
                                 ctx->errflag.as<int>());
  }
  return launch_subst<R>(ctx->stream, ctx->g, npan, pans, cols, sinv, cpl, work, pc);
}

dds_status check_errflag(dds_ctx *ctx) {
  int flag = 0;
  CK(cudaMemcpyAsync(&flag, ctx->errflag.p, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream));
  CK(cudaStreamSynchronize(ctx->stream));
  if (flag != 0) {
    CK(cudaMemsetAsync(ctx->errflag.p, 0, sizeof(int), ctx->stream));
    ctx->err = "a bounded device-side wait gave up (code " + std::to_string(flag) + ")";
    return DDS_ETIMEOUT;
  }
  return DDS_OK;
}

// ------------------------------------------------------------------------------------------
// one DDM application (Algorithm 2.1 / 4.1): b (J-scaled, device, nrhs fields) -> u (device)
// ------------------------------------------------------------------------------------------
// Dataflow schedule of the trace solves of one DDM application (trace plan).  The trace solve
// (sweep l, subdomain X) reads only slot l of X, which receives the traces of every (l', Y) with
// route[l'][d] = l and X the neighbour of Y across d.  Its level is one more than the deepest of
// those producers (0 without any), computed in sweep and step order.  Per level and sweep one
// entry holds that sweep's subdomains of the level, as panels of 8 (subdomain, RHS) columns of
// one factor.  Returns the number of levels.
std::vector<int> trace_depths(const dds_ctx *ctx, int rounds, int *nlev_out) {
  const Geom &g = ctx->g;
  const std::vector<int> seq = sweep_program(g, rounds);
  const int L = (int)seq.size(), ns = g.nsub;
  const std::vector<int> route = build_route(g, rounds);
  std::vector<std::vector<int>> prod((size_t)L * ns);
  for (int lq = 0; lq < L; ++lq)
    for (int y = 0; y < ns; ++y)
      for (int d = 0; d < g.nsides; ++d) {
        const int lp = route[lq * 6 + d], x = sub_neighbour(g, y, d);
        if (lp >= 0 && x >= 0) prod[(size_t)lp * ns + x].push_back(lq * ns + y);
      }
  std::vector<int> depth((size_t)L * ns, -1);
  int nlev = 0;
  for (int l = 0; l < L; ++l) {
    const int dir = seq[l];
    for (int s = 0; s < ctx->nsteps; ++s)
      for (int x : ctx->step_subs[dir][s]) {
        int dmax = -1;
        for (int q : prod[(size_t)l * ns + x]) dmax = std::max(dmax, depth[q]);
        depth[(size_t)l * ns + x] = dmax + 1;
        nlev = std::max(nlev, dmax + 2);
      }
  }
  *nlev_out = nlev;
  return depth;
}

int build_trace_schedule(dds_ctx *ctx, int nrhs, int rounds, std::vector<TraceItem> &items,
                         std::vector<int> &lev_off) {
  std::vector<TracePanel> tp;
  const Geom &g = ctx->g;
  const int L = (int)sweep_program(g, rounds).size(), ns = g.nsub;
  const std::vector<int> route = build_route(g, rounds);
  int nlev = 0;
  const std::vector<int> depth = trace_depths(ctx, rounds, &nlev);
  for (int v = 0; v < nlev; ++v) {
    const size_t first = items.size();
    lev_off.push_back((int)first);
    for (int l = 0; l < L; ++l) {
      std::vector<int> subs;
      for (int x = 0; x < ns; ++x)
        if (depth[(size_t)l * ns + x] == v) subs.push_back(x);
      if (subs.empty()) continue;
      std::stable_sort(subs.begin(), subs.end(),
                       [&](int a, int b) { return ctx->fac_of_sub[a] < ctx->fac_of_sub[b]; });
      const int pan_off = (int)tp.size();
      TracePanel cur{};
      cur.factor = -1;
      for (int x : subs)
        for (int r = 0; r < nrhs; ++r) {
          if (cur.ncol == 8 || (cur.ncol > 0 && cur.factor != ctx->fac_of_sub[x])) {
            tp.push_back(cur);
            cur = TracePanel{};
          }
          cur.factor = ctx->fac_of_sub[x];
          cur.sub[cur.ncol] = x;
          cur.rhs[cur.ncol] = r;
          ++cur.ncol;
        }
      if (cur.ncol > 0) tp.push_back(cur);
      trace_items_for(g, tp.data(), pan_off, (int)tp.size(), l, route.data(), ctx->in_mask[l],
                      items);
    }
    // heaviest items first, so that the snake deal over the CTAs balances: cost ~ a fixed part
    // (staging, reduction, barriers; about 0.7 of a full tile's FMAs at 80 inputs) plus the
    // FMAs, which a tile with at most 32 live rows runs in half the time
    auto cost = [&](const TraceItem &t) {
      const int n = (t.h.z >> 16) & 0xFFFF, dout = t.h.w & 0xFF, tile = (t.h.w >> 8) & 0xFF;
      const bool half = 2 * g.Lt[dout] - tile * 64 <= 32;
      return 56 + (half ? n / 2 : n);
    };
    std::stable_sort(items.begin() + first, items.end(),
                     [&](const TraceItem &a, const TraceItem &b) { return cost(a) > cost(b); });
  }
  lev_off.push_back((int)items.size());
  return nlev;
}

// Work units of the tensor-core trace launch (k_trace_tc.cu), on the same dataflow levels.  Per
// level and sweep, the level's subdomains (by factor) times every RHS are cut into column tiles
// of at most 32 columns of one factor; a tile yields one unit per 128-row tile of the stacked
// output rows that holds a routed side with a neighbour of some column.  The unit multiplies the
// inputs of the sides that receive in this sweep and have a neighbour of some column (kmask);
// in the first sweep it also adds the raw own-source lines (a unit without inputs then only does
// that).  need[] receives, per slot, the publications its trace solve waits for.  Returns the
// number of levels.
int build_tc_trace_schedule(dds_ctx *ctx, int nrhs, int rounds, std::vector<int4> &units,
                            std::vector<int> &ucols, std::vector<int> &lev_off,
                            std::vector<unsigned> &need) {
  const Geom &g = ctx->g;
  const int L = (int)sweep_program(g, rounds).size(), ns = g.nsub;
  const std::vector<int> route = build_route(g, rounds);
  int nlev = 0;
  const std::vector<int> depth = trace_depths(ctx, rounds, &nlev);
  constexpr int kCols = 32;
  const int RT = (g.T + 127) / 128;
  need.assign((size_t)L * ns, 0u);
  // the publications a unit makes (k_trace_tc's epilogue counts the same): per subdomain of its
  // tile and per side whose rows lie in its row tile, routed and with a neighbour
  auto publish = [&](int l, int rt, const std::vector<int> &tile) {
    int prevX = -1;
    for (int col : tile) {
      const int X = col % ns;
      if (X == prevX) continue;
      prevX = X;
      for (int d = 0; d < g.nsides; ++d) {
        if (g.toff[d] >= 128 * (rt + 1) || g.toff[d] + 2 * g.Lt[d] <= 128 * rt) continue;
        const int lq = route[l * 6 + d], Y = sub_neighbour(g, X, d);
        if (lq >= 0 && Y >= 0) ++need[(size_t)lq * ns + Y];
      }
    }
  };
  for (int v = 0; v < nlev; ++v) {
    lev_off.push_back((int)units.size());
    for (int l = 0; l < L; ++l) {
      std::vector<int> subs;
      for (int x = 0; x < ns; ++x)
        if (depth[(size_t)l * ns + x] == v) subs.push_back(x);
      if (subs.empty()) continue;
      std::stable_sort(subs.begin(), subs.end(),
                       [&](int a, int b) { return ctx->fac_of_sub[a] < ctx->fac_of_sub[b]; });
      std::vector<int> tile;   // (rhs * nsub + sub) of the current column tile
      int fac = -1;
      auto flush = [&]() {
        if (tile.empty()) return;
        int nb = 0;   // sides with a neighbour for some column
        for (int c : tile)
          for (int d = 0; d < g.nsides; ++d)
            if (sub_neighbour(g, c % ns, d) >= 0) nb |= 1 << d;
        int outs = 0;
        for (int d = 0; d < g.nsides; ++d)
          if (((nb >> d) & 1) && route[l * 6 + d] >= 0) outs |= 1 << d;
        const int kmask = ctx->in_mask[l] & nb;
        const int raw = l == 0 ? 1 : 0;
        if (outs != 0 && (kmask != 0 || raw)) {
          const int col0 = (int)ucols.size();
          ucols.insert(ucols.end(), tile.begin(), tile.end());
          for (int rt = 0; rt < RT; ++rt) {
            bool need = false;
            for (int d = 0; d < g.nsides; ++d)
              if (((outs >> d) & 1) && g.toff[d] < 128 * (rt + 1) &&
                  g.toff[d] + 2 * g.Lt[d] > 128 * rt)
                need = true;
            if (!need) continue;
            // one unit multiplies the inputs of every received side into one accumulator, so
            // each output is added into its receiver once
            units.push_back(make_int4(fac | ((int)tile.size() << 24), l | (rt << 16), col0,
                                      kmask | (raw << 8)));
            publish(l, rt, tile);
          }
        }
        tile.clear();
      };
      for (int x : subs) {
        if (ctx->fac_of_sub[x] != fac) {
          flush();
          fac = ctx->fac_of_sub[x];
        }
        for (int r = 0; r < nrhs; ++r) {
          if ((int)tile.size() == kCols) flush();
          tile.push_back(r * ns + x);
        }
      }
      flush();
    }
    // heaviest units first (K-steps of the received sides), so that the snake deal balances
    auto cost = [&](const int4 &u) {
      int k = 0;
      for (int d = 0; d < g.nsides; ++d)
        if ((u.w >> d) & 1) k += 2 * g.Lt[d];
      return k;
    };
    std::stable_sort(units.begin() + lev_off.back(), units.end(),
                     [&](const int4 &a, const int4 &b) { return cost(a) > cost(b); });
  }
  lev_off.push_back((int)units.size());
  return nlev;
}

// workspaces of one DDM application; *grown is set if any buffer moved (cached graphs go stale)
template <typename R>
dds_status prepare_ddm(dds_ctx *ctx, int nrhs, int rounds, bool *grown) {
  using C = typename Cx<R>::T;
  const Geom &g = ctx->g;
  dds_status rs = set_route(ctx, rounds);
  if (rs != DDS_OK) return rs;
  CallPlan *cp = get_plan(ctx, nrhs);
  if (!cp) { ctx->err = "failed to upload launch lists"; return DDS_ENOMEM; }
  const int L = (int)sweep_program(g, rounds).size();
  const long long slot = (long long)nrhs * g.nsub * g.T;
  const bool trace_plan = ctx->plan == DDS_PLAN_TRACE;
  long long work_cols = (long long)g.nsub * nrhs;
  if (!trace_plan) {
    work_cols = 0;
    for (auto &sp : cp->steps) work_cols = std::max<long long>(work_cols, sp.ncols);
  }
  if (trace_plan) {
    // schedule of the cooperative trace launch (uploaded outside any stream capture)
    auto &tt = cp->trace_steps[rounds];
    if (tt.n < 0 && (long long)nrhs * g.nsub > INT32_MAX) {   // item column words are 32-bit
      ctx->err = "trace-operator plan: right-hand sides x subdomains exceed 2^31";
      return DDS_EINVAL;
    }
    if (tt.n < 0) {
      std::vector<TraceItem> items;
      std::vector<int> lev;
      tt.nlev = build_trace_schedule(ctx, nrhs, rounds, items, lev);
      std::vector<int4> hdr(items.size());
      std::vector<int2> cw(items.size() * 8);
      for (size_t i = 0; i < items.size(); ++i) {
        hdr[i] = items[i].h;
        for (int c = 0; c < 8; ++c) cw[i * 8 + c] = items[i].col[c];
      }
      CK(upload(tt.buf, hdr, ctx->stream));
      CK(upload(tt.cols, cw, ctx->stream));
      CK(upload(tt.levs, lev, ctx->stream));
      tt.n = (int)items.size();
      void *gb0 = ctx->gbar.p;
      CK(ctx->gbar.ensure(trace_counter_bytes(std::max(tt.nlev, 1))));
      if (gb0 != ctx->gbar.p) *grown = true;
    }
    if (ctx->trace_tc && tt.tn < 0) {
      std::vector<int4> units;
      std::vector<int> ucols, lev;
      std::vector<unsigned> need;
      tt.tnlev = build_tc_trace_schedule(ctx, nrhs, rounds, units, ucols, lev, need);
      int dev = 0, nsm = 0;
      CK(cudaGetDevice(&dev));
      CK(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
      std::vector<int> uoff, coff;
      std::vector<int2> cunits;
      std::vector<int4> chunks;
      if (!build_tt_streams(g, ctx->split, nsm, units, lev, uoff, cunits, coff, chunks)) {
        ctx->err = "tensor-core trace streams cannot be built for this geometry";
        return DDS_EINVAL;
      }
      CK(upload(tt.tunits, units, ctx->stream));
      CK(upload(tt.tcols, ucols, ctx->stream));
      CK(upload(tt.tuoff, uoff, ctx->stream));
      CK(upload(tt.tcunits, cunits, ctx->stream));
      CK(upload(tt.tcoff, coff, ctx->stream));
      CK(upload(tt.tchunks, chunks, ctx->stream));
      tt.tG = nsm;
      CK(upload(tt.tneed, need, ctx->stream));
      CK(tt.tready.ensure(need.size() * sizeof(unsigned)));
      tt.tslots = (int)need.size();
      tt.tn = (int)units.size();
    }
  }
  if (ctx->big_tc && ctx->single) {
    // scratch of the stage-parallel substitutions, sized for the widest launch (allocated here,
    // outside any stream capture)
    size_t bmax = 0, amax = 0;
    auto need = [&](const StepPlan &sp) {
      if (sp.npanels <= 0) return;
      size_t ab = 0;
      bmax = std::max(bmax, big_scratch_bytes(g, ctx->split, sp.pc, sp.npanels, &ab));
      amax = std::max(amax, ab);
    };
    need(cp->all);
    for (auto &sp : cp->steps) need(sp);
    void *b0 = ctx->bigB.p, *a0 = ctx->bigacc.p;
    CK(ctx->bigB.ensure(bmax));
    CK(ctx->bigacc.ensure(amax));
    *grown = *grown || b0 != ctx->bigB.p || a0 != ctx->bigacc.p;
  }
  void *w0 = ctx->work.p, *g0 = ctx->gtr.p, *r0 = ctx->rawf.p, *z0 = ctx->nzflag.p;
  CK(ctx->nzflag.ensure(work_cols * sizeof(int)));
  void *bad0 = ctx->badrhs.p;
  CK(ctx->badrhs.ensure((size_t)nrhs * sizeof(int)));
  *grown = *grown || bad0 != ctx->badrhs.p;
  *grown = *grown || z0 != ctx->nzflag.p;
  CK(ctx->work.ensure(work_cols * g.Nloc * sizeof(C)));
  CK(ctx->gtr.ensure(L * slot * sizeof(C)));
  if (trace_plan) CK(ctx->rawf.ensure(slot * sizeof(C)));
  *grown = *grown || w0 != ctx->work.p || g0 != ctx->gtr.p || r0 != ctx->rawf.p;
  return DDS_OK;
}

template <typename R>
dds_status run_ddm(dds_ctx *ctx, const double2 *b, int nrhs, double2 *u, int rounds) {
  using C = typename Cx<R>::T;
  const Geom &g = ctx->g;
  cudaStream_t st = ctx->stream;
  CallPlan *cp = get_plan(ctx, nrhs);
  if (!cp) { ctx->err = "failed to upload launch lists"; return DDS_ENOMEM; }
  const C *sinv = ctx->single ? (const C *)ctx->sinv32.p : (const C *)ctx->sinv64.p;
  const C *cpl = ctx->single ? (const C *)ctx->cpl32.p : (const C *)ctx->cpl64.p;
  const C *gmap = ctx->single ? (const C *)ctx->gmap32.p : (const C *)ctx->gmap64.p;
  const std::vector<int> seq = sweep_program(g, rounds);
  const int L = (int)seq.size();
  const long long slot = (long long)nrhs * g.nsub * g.T;
  const bool trace_plan = ctx->plan == DDS_PLAN_TRACE;
  CK(cudaMemsetAsync(ctx->gtr.p, 0, L * slot * sizeof(C), st));
  C *work = ctx->work.as<C>();
  C *gtr = ctx->gtr.as<C>();
  const Col *cols = cp->cols.as<Col>();
  int *nzf = ctx->nzflag.as<int>();   // per work slot: nonzero right-hand side
  int *badf = ctx->badrhs.as<int>();  // per RHS: non-finite source entry
  CK(cudaMemsetAsync(badf, 0, (size_t)nrhs * sizeof(int), st));
  const Panel *pans = cp->panels.as<Panel>();
  const int *route = ctx->route_dev.as<int>();
  // the panels of one substitution launch: with zero-work skipping, the columns whose assembled
  // right-hand side is nonzero, packed by k_compact_panels after the assembly
  const Panel *dpans = cp->dpans.as<Panel>();
  const Col *dcols = cp->dcols.as<Col>();
  auto skip = [&](const StepPlan &sp) -> cudaError_t {
    return launch_compact_panels(st, sp.ngrp, cp->groups.as<int4>() + sp.grp_off, pans, cols,
                                 nzf, cp->dcols.as<Col>(), cp->dpans.as<Panel>(), sp.pc,
                                 ctx->solve_stats.as<unsigned long long>());
  };
  const bool zs = ctx->zero_skip;
  const Panel *spans = zs ? dpans : pans;
  const Col *scols = zs ? dcols : cols;
  if (!trace_plan) {
    CK(cudaMemsetAsync(u, 0, (size_t)nrhs * g.Nglob * sizeof(double2), st));
    // not while a graph is captured (capture runs on gstream)
    const bool annotate = !(ctx->gstream && ctx->stream == ctx->gstream);
    for (int l = 0; l < L; ++l) {
      const int dir = seq[l];
      for (int s = 0; s < ctx->nsteps; ++s) {
        const StepPlan &sp = cp->steps[dir * ctx->nsteps + s];
        if (sp.ncols == 0) continue;
        char label[48];
        if (annotate) std::snprintf(label, sizeof label, "sweep %d step %d", l + 1, s + 1);
        if (annotate) nvtxRangePushA(label);
        LAUNCHK(DDS_K_ASSEMBLE, launch_assemble<R>(st, g, ctx->tb, sp.ncols, cols + sp.col_off, work, b, nullptr,
                                  l == 0, gtr + l * slot, (long long)g.nsub * g.T, g.T, 1, 0, nzf,
                                  l == 0 ? badf : nullptr));
        if (zs) LAUNCH(skip(sp));
        LAUNCHK(DDS_K_SUBST, subst_any<R>(ctx, sp.npanels, spans + sp.pan_off, scols, sinv, cpl, work, sp.pc, nzf));
        LAUNCHK(DDS_K_EXTRACT, launch_extract<R>(st, g, sp.ncols, cols + sp.col_off, work, u, 1, nullptr, gtr,
                                 route, l, nrhs));
        if (annotate) nvtxRangePop();
      }
    }
  } else {
    C *rawf = ctx->rawf.as<C>();
    const StepPlan &all = cp->all;
    // own sources: x_f = A_R^{-1} b_own; keep its raw trace lines
    LAUNCHK(DDS_K_ASSEMBLE, launch_assemble<R>(st, g, ctx->tb, all.ncols, cols + all.col_off, work, b, nullptr, 1,
                              (const C *)nullptr, 0, 0, 1, 0, nzf, badf));
    if (zs) LAUNCH(skip(all));
    LAUNCHK(DDS_K_SUBST, subst_any<R>(ctx, all.npanels, spans + all.pan_off, scols, sinv, cpl, work, all.pc, nzf));
    LAUNCHK(DDS_K_EXTRACT, launch_extract<R>(st, g, all.ncols, cols + all.col_off, work, u, 0, rawf,
                             (C *)nullptr, route, 0, nrhs));
    // sweeps: every trace solve of every sweep through the trace map, in one cooperative launch
    // over the dataflow levels (host-built item lists, a counter wait between levels)
    auto tti = cp->trace_steps.find(rounds);   // built by prepare_ddm
    if (tti == cp->trace_steps.end() || tti->second.n < 0) {
      ctx->err = "trace item table missing";
      return DDS_EINVAL;
    }
    const CallPlan::TraceTable &tt = tti->second;
    if constexpr (sizeof(R) == 4) {
      if (ctx->trace_tc) {
        if (tt.tn < 0) {
          ctx->err = "tensor-core trace schedule missing";
          return DDS_EINVAL;
        }
        LAUNCHK(DDS_K_TRACE_STEP,
                launch_trace_tc(st, g, ctx->split, tt.tunits.as<int4>(), tt.tcols.as<int>(),
                                tt.tuoff.as<int>(), tt.tcunits.as<int2>(), tt.tcoff.as<int>(),
                                tt.tchunks.as<int4>(), tt.tn, tt.tG,
                                ctx->tttiles.as<unsigned char>(),
                                route, (float2 *)gtr, (const float2 *)rawf, nrhs,
                                tt.tready.as<unsigned>(), tt.tneed.as<unsigned>(), tt.tslots,
                                ctx->errflag.as<int>(), ctx->wait_limit));
      }
    }
    if (!(sizeof(R) == 4 && ctx->trace_tc))
      LAUNCHK(DDS_K_TRACE_STEP, launch_trace_sweeps<R>(st, g, tt.buf.as<int4>(), tt.cols.as<int2>(),
                                                       tt.n, tt.levs.as<int>(), tt.nlev, gmap, gtr,
                                                       rawf, nrhs, ctx->gbar.as<unsigned>(),
                                                       ctx->errflag.as<int>(), ctx->trace_per_sm,
                                                       ctx->wait_limit));
    // own nodes: u = A_R^{-1}(b_own + potentials of all traces received in every sweep)
    LAUNCHK(DDS_K_ASSEMBLE, launch_assemble<R>(st, g, ctx->tb, all.ncols, cols + all.col_off, work, b, nullptr, 1,
                              gtr, (long long)g.nsub * g.T, g.T, L, slot, nzf));
    if (zs) LAUNCH(skip(all));
    LAUNCHK(DDS_K_SUBST, subst_any<R>(ctx, all.npanels, spans + all.pan_off, scols, sinv, cpl, work, all.pc, nzf));
    LAUNCHK(DDS_K_EXTRACT, launch_extract<R>(st, g, all.ncols, cols + all.col_off, work, u, 2, (C *)nullptr,
                             (C *)nullptr, route, 0, nrhs));
  }
  return DDS_OK;
}

dds_status enqueue_ddm(dds_ctx *ctx, const double2 *b, int nrhs, double2 *u, int rounds) {
  return ctx->single ? run_ddm<float>(ctx, b, nrhs, u, rounds)
                                     : run_ddm<double>(ctx, b, nrhs, u, rounds);
}

// One DDM application.  Without profiling, the ~2 + (sweeps x steps) dependent launches are
// captured once into a CUDA graph per (b, u, nrhs, rounds) and replayed on an internal stream
// ordered after and before the caller's stream by events.
dds_status ddm(dds_ctx *ctx, const double2 *b, int nrhs, double2 *u, int rounds) {
  NvtxRange range("DDM application");
  bool grown = false;
  dds_status r = ctx->single ? prepare_ddm<float>(ctx, nrhs, rounds, &grown)
                                             : prepare_ddm<double>(ctx, nrhs, rounds, &grown);
  if (r != DDS_OK) {
    // a failed allocation may have released a buffer that cached graphs still name
    ctx->clear_graphs();
    return r;
  }
  if (grown) ctx->clear_graphs();
  if (!ctx->use_graphs || ctx->profiling) {
    r = enqueue_ddm(ctx, b, nrhs, u, rounds);
    if (r == DDS_OK && ctx->ev_used > 4096) CK(prof_fold(ctx));
    return r;
  }
  if (!ctx->gstream) {
    CK(cudaStreamCreateWithFlags(&ctx->gstream, cudaStreamNonBlocking));
    CK(cudaEventCreateWithFlags(&ctx->gev[0], cudaEventDisableTiming));
    CK(cudaEventCreateWithFlags(&ctx->gev[1], cudaEventDisableTiming));
  }
  const std::array<long long, 4> key = {(long long)(uintptr_t)b, (long long)(uintptr_t)u, nrhs,
                                         rounds};
  auto it = ctx->graphs.find(key);
  if (it == ctx->graphs.end()) {
    if (ctx->graphs.size() >= 64) ctx->clear_graphs();
    cudaStream_t caller = ctx->stream;
    const long long l0 = ctx->launches;
    ctx->stream = ctx->gstream;
    cudaGraph_t graph = nullptr;
    cudaError_t e = cudaStreamBeginCapture(ctx->gstream, cudaStreamCaptureModeThreadLocal);
    if (e == cudaSuccess) {
      r = enqueue_ddm(ctx, b, nrhs, u, rounds);
      e = cudaStreamEndCapture(ctx->gstream, &graph);
    }
    ctx->stream = caller;
    if (e != cudaSuccess || r != DDS_OK) {
      if (graph) cudaGraphDestroy(graph);
      if (r != DDS_OK) return r;
      CK(e);
    }
    dds_ctx::GraphEntry ge;
    ge.nodes = ctx->launches - l0;
    ctx->launches = l0;
    e = cudaGraphInstantiate(&ge.exec, graph, 0);
    cudaGraphDestroy(graph);
    CK(e);
    it = ctx->graphs.emplace(key, ge).first;
  }
  CK(cudaEventRecord(ctx->gev[0], ctx->stream));
  CK(cudaStreamWaitEvent(ctx->gstream, ctx->gev[0], 0));
  CK(cudaGraphLaunch(it->second.exec, ctx->gstream));
  CK(cudaEventRecord(ctx->gev[1], ctx->gstream));
  CK(cudaStreamWaitEvent(ctx->stream, ctx->gev[1], 0));
  ctx->launches += it->second.nodes;
  return DDS_OK;
}

// ------------------------------------------------------------------------------------------
// set-up
// ------------------------------------------------------------------------------------------
dds_status validate(const dds_problem *p, std::string &err) {
  if (!p) { err = "null problem"; return DDS_EINVAL; }
  if (p->dim != 2 && p->dim != 3) { err = "dim must be 2 or 3"; return DDS_EINVAL; }
  for (int a = 0; a < p->dim; ++a) {
    if (p->n[a] <= 0 || p->parts[a] <= 0 || p->n[a] % p->parts[a]) {
      err = "n[a] must be a positive multiple of parts[a]";
      return DDS_EINVAL;
    }
  }
  if (!p->c) { err = "null wave speed"; return DDS_EINVAL; }
  if (p->pml_cells < 1 || p->halo < 0 || p->h <= 0 || p->omega <= 0 || p->pml_power < 1) {
    err = "invalid PML / grid parameters";
    return DDS_EINVAL;
  }
  if (p->precision < DDS_FP64 || p->precision > DDS_MIXED_FP32) { err = "bad precision"; return DDS_EINVAL; }
  if (p->plan < 0 || p->plan > 2) { err = "bad plan"; return DDS_EINVAL; }
  return DDS_OK;
}

template <typename R>
dds_status build_trace_map(dds_ctx *ctx) {
  // column k of the map = raw trace lines of A_R^{-1} (commutator source of unit trace k),
  // computed in FP64 for every distinct factor; then the back-trace correction is folded in.
  const Geom &g = ctx->g;
  cudaStream_t st = ctx->stream;
  const long long TT = gmap_elems(g, ctx->nfac);
  CK(ctx->gmap64.ensure(TT * sizeof(double2)));
  const int chunk = std::min(g.T, 1024);
  CK(ctx->work.ensure((long long)chunk * g.Nloc * sizeof(double2)));
  std::vector<Col> cols(chunk);
  for (int q = 0; q < chunk; ++q) cols[q] = Col{0, 0, q, 0};
  DBuf dcols, dpans;
  for (int f = 0; f < ctx->nfac; ++f) {
    int sub0 = 0;
    while (ctx->fac_of_sub[sub0] != f) ++sub0;
    for (int q = 0; q < chunk; ++q) cols[q].sub = sub0;
    CK(upload(dcols, cols, st));
    for (int k0 = 0; k0 < g.T; k0 += chunk) {
      const int nk = std::min(chunk, g.T - k0);
      std::vector<Panel> pans;
      const int pc = 4;
      for (int i = 0; i < nk; i += pc) pans.push_back(Panel{i, std::min(pc, nk - i), f, 0});
      CK(upload(dpans, pans, st));
      double2 *work = ctx->work.as<double2>();
      LAUNCH(launch_unit_traces<double>(st, g, ctx->tb, k0, nk, work));
      LAUNCHK(DDS_K_SUBST, launch_subst<double>(st, g, (int)pans.size(), dpans.as<Panel>(), dcols.as<Col>(),
                                  ctx->sinv64.as<double2>(), ctx->cpl64.as<double2>(), work, pc));
      LAUNCH(launch_raw_lines<double>(st, g, nk, work, ctx->gmap64.as<double2>(), f, k0));
      CK(cudaStreamSynchronize(st));
    }
    LAUNCH(launch_gmap_backtrace(st, g, ctx->gmap64.as<double2>(), f));
  }
  if (ctx->single) {
    CK(ctx->gmap32.ensure(TT * sizeof(float2)));
    LAUNCH(launch_convert_c64_c32(st, ctx->gmap64.as<double2>(), ctx->gmap32.as<float2>(), TT));
  }
  CK(cudaStreamSynchronize(st));
  return DDS_OK;
}

dds_status setup_impl(dds_ctx *ctx, const dds_problem *p) {
  const auto t0 = std::chrono::steady_clock::now();
  Geom &g = ctx->g;
  g.dim = p->dim;
  ctx->precision = p->precision;
  ctx->single = p->precision != DDS_FP64;
  ctx->split = p->precision == DDS_MIXED ? 0 : (p->precision == DDS_MIXED_BF16 ? 1 : -1);
  ctx->plan = p->plan;   // DDS_PLAN_AUTO is resolved once the block size is known
  ctx->h = p->h;
  ctx->omega = p->omega;
  ctx->S = p->pml_strength;
  ctx->P = p->pml_cells;
  ctx->power = p->pml_power;
  ctx->H = p->halo;
  g.E = p->halo + p->pml_cells;
  for (int a = 0; a < 3; ++a) {
    const bool on = a < p->dim;
    g.n[a] = on ? p->n[a] : 1;
    g.parts[a] = on ? p->parts[a] : 1;
    g.m[a] = g.n[a] / g.parts[a];
    g.M[a] = on ? g.m[a] + 2 * g.E : 1;
    g.G[a] = on ? g.n[a] + 2 * g.E : 1;
  }
  g.nsub = g.parts[0] * g.parts[1] * g.parts[2];
  g.Nloc = (long long)g.M[0] * g.M[1] * g.M[2];
  g.Nglob = (long long)g.G[0] * g.G[1] * g.G[2];
  if (g.Nglob >= (1LL << 31)) {   // the global-grid kernels index nodes with 32-bit integers
    ctx->err = "global extended grid of " + std::to_string(g.Nglob) + " nodes exceeds 2^31 - 1";
    return DDS_EINVAL;
  }
  g.Ml = g.M[p->dim - 1];
  g.Mb = (int)(g.Nloc / g.Ml);
  // automatic plan: the trace-operator plan in 2D while lines have at most 128 nodes (its T x T
  // map takes T unit-trace solves to build); the direct plan otherwise
  if (ctx->plan == DDS_PLAN_AUTO) ctx->plan = (p->dim == 2 && g.Mb <= 128) ? DDS_PLAN_TRACE : DDS_PLAN_DIRECT;
  g.St = ((long long)g.Mb * g.Mb + 1) / 2 * 2;
  g.nsides = 2 * p->dim;
  g.T = 0;
  for (int d = 0; d < 6; ++d) {
    g.Lt[d] = 0;
    g.toff[d] = g.T;
    if (d >= g.nsides) continue;
    int lt = 1;
    for (int b = 0; b < p->dim; ++b)
      if (b != (d >> 1)) lt *= g.M[b];
    g.Lt[d] = lt;
    g.T += 2 * lt;
  }
  if (ctx->plan == DDS_PLAN_TRACE && g.T >= 65536) {   // trace items pack input indices in 16 bits
    ctx->err = "trace vectors too long for the trace-operator plan (T = " + std::to_string(g.T) + ")";
    return DDS_EINVAL;
  }
  // line blocks that fit in shared memory are factored by one CTA per operator; larger ones
  // in global memory, one pivot step per launch
  const bool big_blocks = (size_t)g.Mb * g.Mb * 16 + g.Mb * 20 > 227 * 1024;
  const int dim = p->dim;
  const double h = p->h;
  const double ih2 = 1.0 / (h * h);
  // ---- PML stretching: local (translation invariant) and global alphas
  std::vector<cd> lan[3], lah[3], gan[3], gah[3];
  for (int a = 0; a < 3; ++a) {
    if (a < dim) {
      axis_alphas(g.M[a], -g.E + 0.5, g.m[a], p->halo, p->pml_cells, p->pml_strength,
                  p->pml_power, lan[a], lah[a]);
      axis_alphas(g.G[a], -g.E + 0.5, g.n[a], p->halo, p->pml_cells, p->pml_strength,
                  p->pml_power, gan[a], gah[a]);
    } else {
      lan[a].assign(1, cd(1, 0));
      lah[a].assign(2, cd(1, 0));
      gan[a].assign(1, cd(1, 0));
      gah[a].assign(2, cd(1, 0));
    }
  }
  // ---- wave numbers: global (nearest interior node) and per subdomain (Eq. 2.8)
  const long long nint = (long long)g.n[0] * g.n[1] * g.n[2];
  std::vector<double> cint(p->c, p->c + nint);
  for (double v : cint)
    if (!(v > 0)) { ctx->err = "wave speed must be positive"; return DDS_EINVAL; }
  auto clampi = [](int v, int lo, int hi) { return v < lo ? lo : (v > hi ? hi : v); };
  std::vector<double> k2g(g.Nglob);
  for (int p2 = 0; p2 < g.G[2]; ++p2)
    for (int p1 = 0; p1 < g.G[1]; ++p1)
      for (int p0 = 0; p0 < g.G[0]; ++p0) {
        const int i0 = clampi(p0 - g.E, 0, g.n[0] - 1);
        const int i1 = clampi(p1 - g.E, 0, g.n[1] - 1);
        const int i2 = dim == 3 ? clampi(p2 - g.E, 0, g.n[2] - 1) : 0;
        const double kk = p->omega / cint[i0 + (long long)g.n[0] * (i1 + (long long)g.n[1] * i2)];
        k2g[p0 + (long long)g.G[0] * (p1 + (long long)g.G[1] * p2)] = kk * kk;
      }
  // per-subdomain kappa^2 on the extended grid; deduplicate identical fields
  std::vector<std::vector<double>> fac_k2;
  ctx->fac_of_sub.assign(g.nsub, -1);
  for (int s = 0; s < g.nsub; ++s) {
    int k[3];
    sub_index(g, s, k);
    std::vector<double> k2(g.Nloc);
    for (int l2 = 0; l2 < g.M[2]; ++l2)
      for (int l1 = 0; l1 < g.M[1]; ++l1)
        for (int l0 = 0; l0 < g.M[0]; ++l0) {
          const int i0 = clampi(k[0] * g.m[0] + l0 - g.E, k[0] * g.m[0], (k[0] + 1) * g.m[0] - 1);
          const int i1 = clampi(k[1] * g.m[1] + l1 - g.E, k[1] * g.m[1], (k[1] + 1) * g.m[1] - 1);
          const int i2 = dim == 3 ? clampi(k[2] * g.m[2] + l2 - g.E, k[2] * g.m[2], (k[2] + 1) * g.m[2] - 1) : 0;
          const double kk = p->omega / cint[i0 + (long long)g.n[0] * (i1 + (long long)g.n[1] * i2)];
          k2[l0 + (long long)g.M[0] * (l1 + (long long)g.M[1] * l2)] = kk * kk;
        }
    int found = -1;
    for (size_t f = 0; f < fac_k2.size(); ++f)
      if (fac_k2[f] == k2) { found = (int)f; break; }
    if (found < 0) {
      found = (int)fac_k2.size();
      fac_k2.push_back(std::move(k2));
    }
    ctx->fac_of_sub[s] = found;
  }
  ctx->nfac = (int)fac_k2.size();
  // ---- line-block coefficients of every distinct operator
  const int Mb = g.Mb, Ml = g.Ml, la = dim - 1;
  const long long per = (long long)Ml * Mb;
  std::vector<double2> dg(ctx->nfac * per), offx(ctx->nfac * per), offy, cpl(ctx->nfac * per);
  if (dim == 3) offy.resize(ctx->nfac * per);
  auto tprod = [&](int a, const int i[3]) {  // prod_{b != a} alpha_b / h^2
    cd t(ih2, 0.0);
    for (int b = 0; b < dim; ++b)
      if (b != a) t *= lan[b][i[b]];
    return t;
  };
  for (int f = 0; f < ctx->nfac; ++f) {
    for (long long q = 0; q < g.Nloc; ++q) {
      int i[3] = {(int)(q % g.M[0]), (int)((q / g.M[0]) % g.M[1]), (int)(q / ((long long)g.M[0] * g.M[1]))};
      cd J(1.0, 0.0);
      for (int a = 0; a < dim; ++a) J *= lan[a][i[a]];
      cd diag = fac_k2[f][q] * J;
      for (int a = 0; a < dim; ++a) diag -= tprod(a, i) * (1.0 / lah[a][i[a]] + 1.0 / lah[a][i[a] + 1]);
      const int j = i[la];
      const int r = (int)(q - (long long)j * Mb);
      const long long o = f * per + (long long)j * Mb + r;
      dg[o] = make_double2(diag.real(), diag.imag());
      cd ox = (i[0] + 1 < g.M[0]) ? tprod(0, i) / lah[0][i[0] + 1] : cd(0, 0);
      offx[o] = make_double2(ox.real(), ox.imag());
      if (dim == 3) {
        cd oy = (i[1] + 1 < g.M[1]) ? tprod(1, i) / lah[1][i[1] + 1] : cd(0, 0);
        offy[o] = make_double2(oy.real(), oy.imag());
      }
      cd cp = (i[la] + 1 < g.M[la]) ? tprod(la, i) / lah[la][i[la] + 1] : cd(0, 0);
      cpl[o] = make_double2(cp.real(), cp.imag());
    }
  }
  // ---- commutator couplings per side: prod_{tangential b} alpha_b / h^2
  std::vector<double2> coef(g.T / 2);
  std::vector<float2> coef32(g.T / 2);
  for (int d = 0; d < g.nsides; ++d) {
    const int a = d >> 1;
    for (int t = 0; t < g.Lt[d]; ++t) {
      int tt = t;
      cd c(ih2, 0.0);
      for (int b = 0; b < dim; ++b) {
        if (b == a) continue;
        c *= lan[b][tt % g.M[b]];
        tt /= g.M[b];
      }
      coef[g.toff[d] / 2 + t] = make_double2(c.real(), c.imag());
      coef32[g.toff[d] / 2 + t] = make_float2((float)c.real(), (float)c.imag());
    }
  }
  // ---- step schedules (Eq. 2.10-2.11 / 4.3-4.4), subdomains grouped by factor
  const auto dirs = sweep_dirs(dim);
  ctx->ndirs = (int)dirs.size();
  ctx->nsteps = 1;  // N1 + N2 - 1 (2D), N1 + N2 + N3 - 2 (3D)
  for (int a = 0; a < dim; ++a) ctx->nsteps += g.parts[a] - 1;
  ctx->step_subs.assign(ctx->ndirs, std::vector<std::vector<int>>(ctx->nsteps));
  for (int di = 0; di < ctx->ndirs; ++di) {
    for (int s = 0; s < g.nsub; ++s) {
      int k[3];
      sub_index(g, s, k);
      int step = 0;
      for (int a = 0; a < dim; ++a) step += dirs[di][a] == 1 ? k[a] : g.parts[a] - 1 - k[a];
      ctx->step_subs[di][step].push_back(s);
    }
    for (auto &v : ctx->step_subs[di])
      std::stable_sort(v.begin(), v.end(), [&](int a, int b) { return ctx->fac_of_sub[a] < ctx->fac_of_sub[b]; });
  }
  // ---- global stencil of the J-scaled operator (centre and coupling to p + e_a per node)
  std::vector<double2> st0(g.Nglob), stp[3];
  for (int a = 0; a < dim; ++a) stp[a].resize(g.Nglob);
  for (long long q = 0; q < g.Nglob; ++q) {
    const int pp[3] = {(int)(q % g.G[0]), (int)((q / g.G[0]) % g.G[1]),
                       (int)(q / ((long long)g.G[0] * g.G[1]))};
    cd J(1.0, 0.0);
    for (int a = 0; a < dim; ++a) J *= gan[a][pp[a]];
    cd diag = k2g[q] * J;
    for (int a = 0; a < dim; ++a) {
      cd T(ih2, 0.0);
      for (int b = 0; b < dim; ++b)
        if (b != a) T *= gan[b][pp[b]];
      diag -= T * (1.0 / gah[a][pp[a]] + 1.0 / gah[a][pp[a] + 1]);
      const cd c = pp[a] + 1 < g.G[a] ? T / gah[a][pp[a] + 1] : cd(0.0, 0.0);
      stp[a][q] = make_double2(c.real(), c.imag());
    }
    st0[q] = make_double2(diag.real(), diag.imag());
  }
  // ---- upload tables
  cudaStream_t st = ctx->stream;
  CK(upload(ctx->stc0, st0, st));
  ctx->tb.c0 = ctx->stc0.as<double2>();
  for (int a = 0; a < 3; ++a) {
    if (a < dim) CK(upload(ctx->stcp[a], stp[a], st));
    else CK(ctx->stcp[a].ensure(16));
    ctx->tb.cp[a] = ctx->stcp[a].as<double2>();
  }
  CK(upload(ctx->coef64, coef, st));
  CK(upload(ctx->coef32, coef32, st));
  CK(upload(ctx->k2glob, k2g, st));
  for (int a = 0; a < 3; ++a) {
    std::vector<double2> an(gan[a].size()), iah(gah[a].size());
    for (size_t q = 0; q < an.size(); ++q) an[q] = make_double2(gan[a][q].real(), gan[a][q].imag());
    for (size_t q = 0; q < iah.size(); ++q) {
      const cd v = 1.0 / gah[a][q];
      iah[q] = make_double2(v.real(), v.imag());
    }
    CK(upload(ctx->an_glob[a], an, st));
    CK(upload(ctx->iah_glob[a], iah, st));
    ctx->tb.an_glob64[a] = ctx->an_glob[a].as<double2>();
    ctx->tb.iah_glob64[a] = ctx->iah_glob[a].as<double2>();
  }
  ctx->tb.coef64 = ctx->coef64.as<double2>();
  ctx->tb.coef32 = ctx->coef32.as<float2>();
  ctx->tb.k2_glob = ctx->k2glob.as<double>();
  ctx->tb.inv_h2 = ih2;
  // ---- factor (FP64 Schur chain on the GPU)
  DBuf ddg, doffx, doffy, dcpl;
  CK(upload(ddg, dg, st));
  CK(upload(doffx, offx, st));
  if (dim == 3) CK(upload(doffy, offy, st));
  CK(upload(dcpl, cpl, st));
  const long long sinv_elems = (long long)ctx->nfac * Ml * g.St;
  CK(ctx->sinv64.ensure(sinv_elems * sizeof(double2)));
  CK(ctx->sinv32.ensure(sinv_elems * sizeof(float2)));
  CK(ctx->status.ensure(sizeof(int)));
  CK(cudaMemsetAsync(ctx->status.p, 0, sizeof(int), st));
  CK(ctx->errflag.ensure(sizeof(int)));
  CK(cudaMemsetAsync(ctx->errflag.p, 0, sizeof(int), st));
  CK(ctx->solve_stats.ensure(2 * sizeof(unsigned long long)));
  CK(cudaMemsetAsync(ctx->solve_stats.p, 0, 2 * sizeof(unsigned long long), st));

  CK(cudaMemsetAsync(ctx->sinv64.p, 0, sinv_elems * sizeof(double2), st));
  CK(cudaMemsetAsync(ctx->sinv32.p, 0, sinv_elems * sizeof(float2), st));
  if (!big_blocks) {
    LAUNCH(launch_factor(st, ctx->nfac, Mb, Ml, g.St, g.M[0], ddg.as<double2>(), doffx.as<double2>(),
                         dim == 3 ? doffy.as<double2>() : nullptr, dcpl.as<double2>(),
                         ctx->sinv64.as<double2>(), ctx->sinv32.as<float2>(), ctx->status.as<int>()));
  } else {
    DBuf Sbuf, colk, piv;
    CK(Sbuf.ensure((size_t)Mb * Mb * sizeof(double2)));
    CK(colk.ensure((size_t)Mb * sizeof(double2)));
    CK(piv.ensure((size_t)Mb * sizeof(int)));
    for (int f = 0; f < ctx->nfac; ++f)
      CK(launch_factor_big(st, f, Mb, Ml, g.St, g.M[0], ddg.as<double2>(), doffx.as<double2>(),
                           dim == 3 ? doffy.as<double2>() : nullptr, dcpl.as<double2>(),
                           Sbuf.as<double2>(), colk.as<double2>(), piv.as<int>(),
                           ctx->sinv64.as<double2>(), ctx->sinv32.as<float2>(),
                           ctx->status.as<int>(), &ctx->launches));
    CK(cudaStreamSynchronize(st));
  }
  int status = 0;
  CK(cudaMemcpyAsync(&status, ctx->status.p, sizeof(int), cudaMemcpyDeviceToHost, st));
  CK(cudaStreamSynchronize(st));
  if (status != 0) { ctx->err = "singular pivot in the Schur-complement factorisation"; return DDS_EINVAL; }
  CK(ctx->cpl64.ensure(ctx->nfac * per * sizeof(double2)));
  CK(cudaMemcpyAsync(ctx->cpl64.p, dcpl.p, ctx->nfac * per * sizeof(double2), cudaMemcpyDeviceToDevice, st));
  CK(ctx->cpl32.ensure(ctx->nfac * per * sizeof(float2)));
  LAUNCH(launch_convert_c64_c32(st, ctx->cpl64.as<double2>(), ctx->cpl32.as<float2>(), ctx->nfac * per));
  CK(cudaStreamSynchronize(st));
  if (ctx->plan == DDS_PLAN_TRACE) {
    dds_status r = build_trace_map<double>(ctx);
    if (r != DDS_OK) return r;
  }
  if (ctx->split >= 0 && subst_tc_ok(g, ctx->split, 8, false)) {
    // Two-sided (twisted) factorisation where the chain is long enough and the blocks fit the
    // in-shared-memory factor kernel: T_j^{-1} (j > m) and Z_m^{-1} in FP64, then every inverse
    // split into tensor-core pieces.
    const int m = (!big_blocks && subst_tc_ok(g, ctx->split, 8, true)) ? tc_middle_block(g) : 0;
    DBuf tw;
    if (m > 0) {
      CK(tw.ensure(sinv_elems * sizeof(double2)));
      LAUNCH(launch_factor_twisted(st, ctx->nfac, Mb, Ml, g.St, g.M[0], m, ddg.as<double2>(),
                                   doffx.as<double2>(), dim == 3 ? doffy.as<double2>() : nullptr,
                                   dcpl.as<double2>(), ctx->sinv64.as<double2>(),
                                   tw.as<double2>(), ctx->status.as<int>()));
      int status2 = 0;
      CK(cudaMemcpyAsync(&status2, ctx->status.p, sizeof(int), cudaMemcpyDeviceToHost, st));
      CK(cudaStreamSynchronize(st));
      if (status2 != 0) { ctx->err = "singular pivot in the two-sided factorisation"; return DDS_EINVAL; }
    }
    CK(ctx->tctiles.ensure((size_t)tc_tiles_bytes(g, ctx->split, ctx->nfac)));
    LAUNCH(launch_split_tc(st, g, ctx->split, ctx->nfac, ctx->sinv64.as<double2>(),
                           m > 0 ? tw.as<double2>() : nullptr, m, ctx->tctiles.as<unsigned char>()));
    CK(cudaStreamSynchronize(st));
    ctx->tc_m = m;
  } else if (ctx->split >= 0 && g.Mb > 128) {
    // blocks wider than 128 nodes: stage-parallel tensor-core substitutions (k_subst_big.cu)
    CK(ctx->bigtiles.ensure((size_t)big_tiles_bytes(g, ctx->split, ctx->nfac)));
    LAUNCH(launch_split_big(st, g, ctx->split, ctx->nfac, ctx->sinv64.as<double2>(),
                            ctx->bigtiles.as<unsigned char>()));
    CK(cudaStreamSynchronize(st));
    ctx->big_tc = true;
  } else {
    ctx->split = -1;   // FP32 CUDA-core substitutions
  }
  if (ctx->plan == DDS_PLAN_TRACE && ctx->single && ctx->split >= 0 &&
      tt_shape(g, ctx->split, nullptr)) {
    // trace solves on the tensor cores with the substitutions' piece type
    CK(ctx->tttiles.ensure((size_t)tt_tiles_bytes(g, ctx->split, ctx->nfac)));
    LAUNCH(launch_split_trace(st, g, ctx->split, ctx->nfac, ctx->gmap64.as<double2>(),
                              ctx->tttiles.as<unsigned char>()));
    CK(cudaStreamSynchronize(st));
    ctx->trace_tc_avail = ctx->trace_tc = true;
  }
  if (ctx->single) ctx->sinv64.release(), ctx->gmap64.release();
  ctx->setup_seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
  return DDS_OK;
}

// ------------------------------------------------------------------------------------------
// host-pointer staging
// ------------------------------------------------------------------------------------------
struct Staged {
  const double2 *in = nullptr;
  double2 *out = nullptr;
  bool in_host = false, out_host = false;
};

dds_status stage_in(dds_ctx *ctx, const void *ptr, size_t bytes, const double2 **dev) {
  if (is_device_ptr(ptr)) { *dev = (const double2 *)ptr; return DDS_OK; }
  CK(ctx->stage_in.ensure(bytes));
  CK(cudaMemcpyAsync(ctx->stage_in.p, ptr, bytes, cudaMemcpyHostToDevice, ctx->stream));
  *dev = ctx->stage_in.as<double2>();
  return DDS_OK;
}

dds_status stage_out_ptr(dds_ctx *ctx, void *ptr, size_t bytes, double2 **dev, bool *host) {
  if (is_device_ptr(ptr)) { *dev = (double2 *)ptr; *host = false; return DDS_OK; }
  CK(ctx->stage_out.ensure(bytes));
  *dev = ctx->stage_out.as<double2>();
  *host = true;
  return DDS_OK;
}

dds_status finish_out(dds_ctx *ctx, void *ptr, size_t bytes, bool host) {
  if (host) CK(cudaMemcpyAsync(ptr, ctx->stage_out.p, bytes, cudaMemcpyDeviceToHost, ctx->stream));
  CK(cudaStreamSynchronize(ctx->stream));
  return DDS_OK;
}

struct Busy {
  dds_ctx *c;
  bool ok;
  MemAcct *prev;
  explicit Busy(dds_ctx *cc) : c(cc), ok(cc->mu.try_lock()), prev(tl_acct) {
    if (ok) tl_acct = &cc->acct;   // this call's allocations count against its context
  }
  ~Busy() {
    if (ok) {
      tl_acct = prev;
      c->mu.unlock();
    }
  }
};

// ------------------------------------------------------------------------------------------
// FGMRES (right preconditioned, x0 = 0, classical Gram-Schmidt with reorthogonalisation where the
// tolerance needs it, Givens rotations, unnormalised basis with host scales)
// The basis lives in two contiguous device buffers V[maxit+1][nrhs][N], Z[maxit][nrhs][N];
// Gram-Schmidt coefficients stay on the device between the dot and update kernels, and the
// host reads them once per iteration for the Hessenberg / Givens bookkeeping.
// ------------------------------------------------------------------------------------------
dds_status fgmres(dds_ctx *ctx, const double2 *f, int nrhs, double2 *x, double tol, int maxit,
                  int rounds, int *iters, std::vector<double> &relres, void *x_host = nullptr) {
  const Geom &g = ctx->g;
  cudaStream_t st = ctx->stream;
  const long long N = g.Nglob;
  const long long vs = (long long)nrhs * N;  // elements per basis vector (all RHS)
  const size_t vbytes = (size_t)vs * sizeof(double2);
  if (ctx->Vbig.ensure((size_t)(maxit + 1) * vbytes) != cudaSuccess ||
      ctx->Zbig.ensure((size_t)maxit * vbytes) != cudaSuccess) {
    cudaGetLastError();
    ctx->err = "out of device memory for the Krylov basis";
    return DDS_ENOMEM;
  }
  double2 *V = ctx->Vbig.as<double2>();
  double2 *Z = ctx->Zbig.as<double2>();
  const int nblk = dots_blocks(N, nrhs);
  CK(ctx->dots_part.ensure((size_t)nrhs * (maxit + 2) * nblk * sizeof(double2)));
  // hdev: [h1: nrhs*(j+1)] [h2: nrhs*(j+1)] [norm^2: nrhs]
  CK(ctx->dots_out.ensure((size_t)nrhs * (2 * maxit + 4) * sizeof(double2)));
  CK(ctx->coefbuf.ensure((size_t)nrhs * (maxit + 1) * sizeof(double2)));
  double2 *hdev = ctx->dots_out.as<double2>();
  double2 *part = ctx->dots_part.as<double2>();
  CK(ctx->scalebuf.ensure((size_t)nrhs * (2 * maxit + 2) * sizeof(double)));   // both passes
  std::vector<double2> hh((size_t)nrhs * (2 * maxit + 4));
  // The basis is kept unnormalised: slot i holds V'_i = s_i V_i with host scales s_i per RHS
  // (no normalisation pass over the data).  Inner products d_i = V'_i^H w' give
  // h_ij = d_i / (s_i s_j), the update w' -= sum_i (d_i / s_i^2) V'_i removes the same
  // projections, the DDM is linear so Z'_j = s_j Z_j, and x = sum_j (y_j / s_j) Z'_j.
  // V'_0 = b = J f, s_0 = beta = ||b||.
  const double2 *b = V;
  LAUNCHK(DDS_K_KRYLOV, launch_scale_J(st, g, ctx->tb, nrhs, f, V));
  LAUNCHK(DDS_K_KRYLOV, launch_dots(st, N, nrhs, 1, b, 0, N, b, N, part, hdev, nblk));
  CK(cudaMemcpyAsync(hh.data(), hdev, nrhs * sizeof(double2), cudaMemcpyDeviceToHost, st));
  CK(cudaStreamSynchronize(st));
  std::vector<double> beta(nrhs);
  for (int r = 0; r < nrhs; ++r) beta[r] = std::sqrt(std::max(hh[r].x, 0.0));
  // a right-hand side with a NaN or infinite entry has a non-finite norm: it is not iterated,
  // its field is set to NaN and its relative residual reported as NaN (the others go on)
  std::vector<char> bad(nrhs, 0);
  for (int r = 0; r < nrhs; ++r) bad[r] = !std::isfinite(hh[r].x);
  std::vector<double> sc((size_t)nrhs * (maxit + 1), 0.0);   // s_i per RHS
  for (int r = 0; r < nrhs; ++r) sc[(size_t)r * (maxit + 1)] = beta[r];
  auto inv2 = [](double v) {   // 1 / v^2, 0 for a vanished vector
    const double q = v > 0.0 ? 1.0 / (v * v) : 0.0;
    return std::isfinite(q) ? q : 0.0;
  };
  std::vector<double> cscale((size_t)nrhs * (maxit + 1));
  const int m = maxit;
  std::vector<cd> H((size_t)nrhs * (m + 1) * m, cd(0, 0)), cs((size_t)nrhs * m), sn((size_t)nrhs * m),
      gg((size_t)nrhs * (m + 1), cd(0, 0));
  std::vector<int> kused(nrhs, 0);
  std::vector<char> done(nrhs, 0);
  for (int r = 0; r < nrhs; ++r) {
    gg[(size_t)r * (m + 1)] = beta[r];
    if (beta[r] == 0 || bad[r]) done[r] = 1;
  }
  auto Hat = [&](int r, int i, int j) -> cd & { return H[((size_t)r * (m + 1) + i) * m + j]; };
  int k = 0;
  for (int j = 0; j < m; ++j) {
    char label[32];
    std::snprintf(label, sizeof label, "FGMRES iteration %d", j + 1);
    NvtxRange it_range(label);
    double2 *Vj = V + j * vs, *Zj = Z + j * vs, *W = V + (j + 1) * vs;
    dds_status rs = ddm(ctx, Vj, nrhs, Zj, rounds);
    if (rs != DDS_OK) return rs;
    LAUNCHK(DDS_K_KRYLOV, launch_apply_A(st, g, ctx->tb, nrhs, Zj, W, 0));
    const int nv = j + 1;
    // classical Gram-Schmidt with the second pass only where it is needed (DGKS criterion):
    // pass 1 also returns ||W||^2 (W is basis slot j+1, the last of the nv+1 vectors)
    double2 *h1 = hdev;                                        // [nrhs][nv + 1]
    double2 *h2 = hdev + (size_t)nrhs * (nv + 1);              // [nrhs][nv]
    double2 *hn = h2 + (size_t)nrhs * nv;                      // [nrhs]
    // update scales 1 / s_i^2, laid out like h1 ([nrhs][nv + 1]) and like h2 ([nrhs][nv])
    for (int r = 0; r < nrhs; ++r)
      for (int i = 0; i <= nv; ++i)
        cscale[(size_t)r * (nv + 1) + i] = i < nv ? inv2(sc[(size_t)r * (m + 1) + i]) : 0.0;
    double *cs1 = ctx->scalebuf.as<double>();
    CK(cudaMemcpyAsync(cs1, cscale.data(), (size_t)nrhs * (nv + 1) * sizeof(double),
                       cudaMemcpyHostToDevice, st));
    LAUNCHK(DDS_K_KRYLOV, launch_dots(st, N, nrhs, nv + 1, V, vs, N, W, N, part, h1, nblk));
    LAUNCHK(DDS_K_KRYLOV, launch_combination(st, N, nrhs, nv, V, vs, N, h1, nv + 1, -1.0, W, N,
                                             false, part, hn, nblk, cs1));
    CK(cudaMemcpyAsync(hh.data(), hdev, (size_t)nrhs * (2 * nv + 2) * sizeof(double2),
                       cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    // Reorthogonalise where the first pass cancelled enough to matter.  After one classical pass
    // the new vector's loss of orthogonality is about sqrt(N) eps ||w0|| / ||w1|| (inner products
    // of length N rounded in FP64); FGMRES to tol needs it well below tol, so the second pass runs
    // where ||w1|| < eta ||w0||, eta = sqrt(N) eps / (0.01 tol), capped at the DGKS 1/sqrt(2).
    const double eta = std::min(std::sqrt(0.5), std::sqrt((double)N) * 2.2e-16 / (0.01 * tol));
    bool second = false;
    for (int r = 0; r < nrhs; ++r) {
      const double w0 = hh[(size_t)r * (nv + 1) + nv].x, w1 = hh[(size_t)nrhs * (2 * nv + 1) + r].x;
      if (!(w1 > eta * eta * w0)) second = true;   // squared norms
    }
    // The second pass only keeps V_{j+1} orthogonal.  If the first-pass column already meets the
    // tolerance for every active RHS (or this is the last iteration), V_{j+1} is never used and
    // the pass is skipped: the first-pass coefficients are accurate to rounding in ||w0||, and
    // the true residual below decides convergence.
    if (second) {
      bool last = j + 1 == m;
      if (!last) {
        last = true;
        for (int r = 0; r < nrhs && last; ++r) {
          if (done[r]) continue;
          std::vector<cd> col(j + 2);
          const double sj = sc[(size_t)r * (m + 1) + j];
          if (!(sj > 0.0)) continue;
          for (int i = 0; i <= j; ++i) {
            const double2 a = hh[(size_t)r * (nv + 1) + i];
            const double si = sc[(size_t)r * (m + 1) + i];
            col[i] = si > 0.0 ? cd(a.x, a.y) / (si * sj) : cd(0, 0);
          }
          col[j + 1] = std::sqrt(std::max(hh[(size_t)nrhs * (2 * nv + 1) + r].x, 0.0)) / sj;
          for (int i = 0; i < j; ++i) {
            const cd a = col[i], bb = col[i + 1];
            const cd c = cs[(size_t)r * m + i], sv = sn[(size_t)r * m + i];
            col[i] = c * a + sv * bb;
            col[i + 1] = -std::conj(sv) * a + std::conj(c) * bb;
          }
          const double rr = std::hypot(std::abs(col[j]), std::abs(col[j + 1]));
          const cd gj = gg[(size_t)r * (m + 1) + j];
          const double est = rr > 0 ? std::abs(col[j + 1]) / rr * std::abs(gj) : 0.0;
          if (!(est / beta[r] < tol)) last = false;
        }
      }
      if (last) second = false;
    }
    std::vector<double2> h2h((size_t)nrhs * nv, make_double2(0.0, 0.0));
    if (second) {
      for (int r = 0; r < nrhs; ++r)
        for (int i = 0; i < nv; ++i)
          cscale[(size_t)r * nv + i] = inv2(sc[(size_t)r * (m + 1) + i]);
      double *cs2 = ctx->scalebuf.as<double>() + (size_t)nrhs * (nv + 1);
      CK(cudaMemcpyAsync(cs2, cscale.data(), (size_t)nrhs * nv * sizeof(double),
                         cudaMemcpyHostToDevice, st));
      LAUNCHK(DDS_K_KRYLOV, launch_dots(st, N, nrhs, nv, V, vs, N, W, N, part, h2, nblk));
      LAUNCHK(DDS_K_KRYLOV, launch_combination(st, N, nrhs, nv, V, vs, N, h2, nv, -1.0, W, N,
                                               false, part, hn, nblk, cs2));
      CK(cudaMemcpyAsync(h2h.data(), h2, (size_t)nrhs * nv * sizeof(double2), cudaMemcpyDeviceToHost, st));
      CK(cudaMemcpyAsync(hh.data() + (size_t)nrhs * (2 * nv + 1), hn, nrhs * sizeof(double2),
                         cudaMemcpyDeviceToHost, st));
      CK(cudaStreamSynchronize(st));
    }
    for (int r = 0; r < nrhs; ++r) {
      // s_{j+1} = ||W'||, and the Hessenberg column in normalised terms
      const double wn = std::sqrt(std::max(hh[(size_t)nrhs * (2 * nv + 1) + r].x, 0.0));
      const double sj = sc[(size_t)r * (m + 1) + j];
      sc[(size_t)r * (m + 1) + j + 1] = wn;
      for (int i = 0; i <= j; ++i) {
        const double2 a = hh[(size_t)r * (nv + 1) + i], bq = h2h[(size_t)r * nv + i];
        const double si = sc[(size_t)r * (m + 1) + i];
        Hat(r, i, j) = si > 0.0 && sj > 0.0 ? cd(a.x + bq.x, a.y + bq.y) / (si * sj) : cd(0, 0);
      }
      Hat(r, j + 1, j) = sj > 0.0 ? wn / sj : 0.0;
    }
    k = j + 1;
    bool all = true;
    for (int r = 0; r < nrhs; ++r) {
      const double hnorm = std::abs(Hat(r, j + 1, j));
      if (done[r]) continue;
      for (int i = 0; i < j; ++i) {  // previous rotations
        const cd a = Hat(r, i, j), bb = Hat(r, i + 1, j);
        const cd c = cs[(size_t)r * m + i], s = sn[(size_t)r * m + i];
        Hat(r, i, j) = c * a + s * bb;
        Hat(r, i + 1, j) = -std::conj(s) * a + std::conj(c) * bb;
      }
      const cd a = Hat(r, j, j), bb = Hat(r, j + 1, j);
      const double rr = std::hypot(std::abs(a), std::abs(bb));
      cd c(1, 0), s(0, 0);
      if (rr > 0) { c = std::conj(a / rr); s = std::conj(bb / rr); }
      cs[(size_t)r * m + j] = c;
      sn[(size_t)r * m + j] = s;
      Hat(r, j, j) = c * a + s * bb;
      Hat(r, j + 1, j) = 0.0;
      const cd gj = gg[(size_t)r * (m + 1) + j];
      gg[(size_t)r * (m + 1) + j + 1] = -std::conj(s) * gj;
      gg[(size_t)r * (m + 1) + j] = c * gj;
      kused[r] = j + 1;
      const double res = std::abs(gg[(size_t)r * (m + 1) + j + 1]) / beta[r];
      if (res < tol || hnorm == 0.0) done[r] = 1;
      else all = false;
    }
    if (all) break;
  }
  *iters = k;
  // x = sum_i Z_i y_i per RHS (one update kernel over all k basis vectors)
  std::vector<double2> ycoef((size_t)nrhs * std::max(k, 1), make_double2(0.0, 0.0));
  for (int r = 0; r < nrhs; ++r) {
    const int kr = kused[r];
    std::vector<cd> y(kr, cd(0, 0));
    for (int i = kr - 1; i >= 0; --i) {
      cd s = gg[(size_t)r * (m + 1) + i];
      for (int q = i + 1; q < kr; ++q) s -= Hat(r, i, q) * y[q];
      y[i] = s / Hat(r, i, i);
    }
    for (int i = 0; i < kr; ++i) {   // x = sum_i (y_i / s_i) Z'_i
      const double si = sc[(size_t)r * (m + 1) + i];
      const cd yi = si > 0.0 ? y[i] / si : cd(0, 0);
      ycoef[(size_t)r * k + i] = make_double2(yi.real(), yi.imag());
    }
  }
  if (k > 0) {
    CK(cudaMemcpyAsync(ctx->coefbuf.p, ycoef.data(), (size_t)nrhs * k * sizeof(double2),
                       cudaMemcpyHostToDevice, st));
    LAUNCHK(DDS_K_KRYLOV, launch_combination(st, N, nrhs, k, Z, vs, N, ctx->coefbuf.as<double2>(),
                                             k, 1.0, x, N, true, nullptr, nullptr, 0));
  } else {
    CK(cudaMemsetAsync(x, 0, vbytes, st));
  }
  for (int r = 0; r < nrhs; ++r)
    if (bad[r]) CK(cudaMemsetAsync(x + (size_t)r * N, 0xFF, (size_t)N * sizeof(double2), st));
  if (x_host != nullptr) {
    // x is final: its copy to the host overlaps the true-residual computation below
    if (!ctx->out_stream) CK(cudaStreamCreateWithFlags(&ctx->out_stream, cudaStreamNonBlocking));
    if (!ctx->out_ev) CK(cudaEventCreateWithFlags(&ctx->out_ev, cudaEventDisableTiming));
    CK(cudaEventRecord(ctx->out_ev, st));
    CK(cudaStreamWaitEvent(ctx->out_stream, ctx->out_ev, 0));
    CK(cudaMemcpyAsync(x_host, x, vbytes, cudaMemcpyDeviceToHost, ctx->out_stream));
  }
  // true residual: R = A x - b (b = V'_0 stays in slot 0; slot 1 is free now)
  double2 *Rv = V + vs;
  LAUNCHK(DDS_K_KRYLOV, launch_apply_A(st, g, ctx->tb, nrhs, x, Rv, 0, b));
  LAUNCHK(DDS_K_KRYLOV, launch_dots(st, N, nrhs, 1, Rv, 0, N, Rv, N, part, hdev, nblk));
  CK(cudaMemcpyAsync(hh.data(), hdev, nrhs * sizeof(double2), cudaMemcpyDeviceToHost, st));
  CK(cudaStreamSynchronize(st));
  relres.assign(nrhs, 0.0);
  bool ok = true;
  for (int r = 0; r < nrhs; ++r) {
    relres[r] = bad[r] ? std::nan("") : (beta[r] > 0 ? std::sqrt(std::max(hh[r].x, 0.0)) / beta[r] : 0.0);
    if (!(relres[r] < tol)) ok = false;
  }
  return ok ? DDS_OK : DDS_ENOCONV;
}

}  // namespace

// ============================================================================================
// C ABI
// ============================================================================================
extern "C" {

dds_status dds_setup(const dds_problem *prob, dds_ctx **out) {
  if (!out) return DDS_EINVAL;
  std::unique_ptr<dds_ctx> ctx(new (std::nothrow) dds_ctx());
  if (!ctx) return DDS_ENOMEM;
  dds_status v = validate(prob, ctx->err);
  if (v != DDS_OK) {
    std::fprintf(stderr, "dds_setup: %s\n", ctx->err.c_str());
    return v;
  }
  ctx->stream = nullptr;
  NvtxRange range("dds_setup");
  MemAcct *prev = tl_acct;
  tl_acct = &ctx->acct;   // set-up allocations count against the new context
  dds_status r = setup_impl(ctx.get(), prob);
  tl_acct = prev;
  if (r != DDS_OK) {
    std::fprintf(stderr, "dds_setup: %s\n", ctx->err.c_str());
    return r;
  }
  *out = ctx.release();
  return DDS_OK;
}

// the DDM as a direct solver with sweep program `prog` (sweep_program): J-scaling of f, one
// DDM application, the error flag and the copy back to a host u
static dds_status sweep_impl(dds_ctx *ctx, const void *f, int nrhs, void *u, int prog) {
  NvtxRange range(prog > 0 ? "dds_sweep" : "dds_sweep_strip");
  const size_t bytes = (size_t)nrhs * ctx->g.Nglob * sizeof(double2);
  const double2 *fd;
  double2 *ud;
  bool uh;
  dds_status r = stage_in(ctx, f, bytes, &fd);
  if (r != DDS_OK) return r;
  r = stage_out_ptr(ctx, u, bytes, &ud, &uh);
  if (r != DDS_OK) return r;
  CK(ctx->bbuf.ensure(bytes));
  LAUNCHK(DDS_K_KRYLOV, launch_scale_J(ctx->stream, ctx->g, ctx->tb, nrhs, fd, ctx->bbuf.as<double2>()));
  r = ddm(ctx, ctx->bbuf.as<double2>(), nrhs, ud, prog);
  if (r != DDS_OK) return r;
  r = check_errflag(ctx);   // (synchronises the stream)
  if (r != DDS_OK) return r;
  // a right-hand side whose source has a NaN or infinite entry gets a NaN field: the local
  // solves of the single-precision modes need not carry a NaN through (the tensor-core split
  // products do not), and a finite field would hide the bad input
  std::vector<int> badh(nrhs, 0);
  CK(cudaMemcpyAsync(badh.data(), ctx->badrhs.p, nrhs * sizeof(int), cudaMemcpyDeviceToHost,
                     ctx->stream));
  CK(cudaStreamSynchronize(ctx->stream));
  for (int q = 0; q < nrhs; ++q)
    if (badh[q]) CK(cudaMemsetAsync(ud + (size_t)q * ctx->g.Nglob, 0xFF, ctx->g.Nglob * sizeof(double2), ctx->stream));
  return finish_out(ctx, u, bytes, uh);
}

dds_status dds_sweep(dds_ctx *ctx, const void *f, int nrhs, void *u, int rounds) {
  if (!ctx) return DDS_EINVAL;
  Busy busy(ctx);
  if (!busy.ok) return DDS_EBUSY;
  ctx->err.clear();
  if (!f || !u || nrhs <= 0 || nrhs > kMaxRhs || rounds < 1) { ctx->err = "invalid argument"; return DDS_EINVAL; }
  return sweep_impl(ctx, f, nrhs, u, rounds);
}

dds_status dds_sweep_strip(dds_ctx *ctx, const void *f, int nrhs, void *u, int nsweeps) {
  if (!ctx) return DDS_EINVAL;
  Busy busy(ctx);
  if (!busy.ok) return DDS_EBUSY;
  ctx->err.clear();
  if (!f || !u || nrhs <= 0 || nrhs > kMaxRhs || nsweeps < 1 || nsweeps > kMaxStripSweeps) {
    ctx->err = "invalid argument";
    return DDS_EINVAL;
  }
  if (!is_strip(ctx->g)) {
    ctx->err = "dds_sweep_strip needs a strip partition (one axis with more than one part)";
    return DDS_EINVAL;
  }
  return sweep_impl(ctx, f, nrhs, u, -nsweeps);
}

dds_status dds_solve(dds_ctx *ctx, const void *f, int nrhs, void *u, double tol, int maxit,
                     int rounds, int *iters, double *relres) {
  if (!ctx) return DDS_EINVAL;
  Busy busy(ctx);
  if (!busy.ok) return DDS_EBUSY;
  ctx->err.clear();
  if (!f || !u || nrhs <= 0 || nrhs > kMaxRhs || rounds < 1 || maxit < 1 || !(tol > 0)) {
    ctx->err = "invalid argument";
    return DDS_EINVAL;
  }
  NvtxRange range("dds_solve");
  const size_t bytes = (size_t)nrhs * ctx->g.Nglob * sizeof(double2);
  const double2 *fd;
  double2 *ud;
  bool uh;
  dds_status r = stage_in(ctx, f, bytes, &fd);
  if (r != DDS_OK) return r;
  r = stage_out_ptr(ctx, u, bytes, &ud, &uh);
  if (r != DDS_OK) return r;
  int it = 0;
  std::vector<double> rel;
  dds_status rs = fgmres(ctx, fd, nrhs, ud, tol, maxit, rounds, &it, rel, uh ? u : nullptr);
  if (uh && ctx->out_stream) {
    // the host copy started inside fgmres (once x was final); wait for it on every path
    const cudaError_t e = cudaStreamSynchronize(ctx->out_stream);
    if (e != cudaSuccess && rs == DDS_OK) CK(e);
  }
  if (rs != DDS_OK && rs != DDS_ENOCONV) return rs;
  r = check_errflag(ctx);
  if (r != DDS_OK) return r;
  if (iters) *iters = it;
  if (relres) for (int q = 0; q < nrhs; ++q) relres[q] = rel[q];
  r = finish_out(ctx, u, bytes, false);   // host results were copied by fgmres
  if (r != DDS_OK) return r;
  if (rs == DDS_ENOCONV) ctx->err = "FGMRES did not reach the tolerance within maxit";
  return rs;
}

dds_status dds_apply(dds_ctx *ctx, const void *u, int nrhs, void *Au) {
  if (!ctx) return DDS_EINVAL;
  Busy busy(ctx);
  if (!busy.ok) return DDS_EBUSY;
  ctx->err.clear();
  if (!u || !Au || nrhs <= 0 || nrhs > kMaxRhs) { ctx->err = "invalid argument"; return DDS_EINVAL; }
  const size_t bytes = (size_t)nrhs * ctx->g.Nglob * sizeof(double2);
  const double2 *ud;
  double2 *od;
  bool oh;
  dds_status r = stage_in(ctx, u, bytes, &ud);
  if (r != DDS_OK) return r;
  r = stage_out_ptr(ctx, Au, bytes, &od, &oh);
  if (r != DDS_OK) return r;
  LAUNCHK(DDS_K_KRYLOV, launch_apply_A(ctx->stream, ctx->g, ctx->tb, nrhs, ud, od, 1));
  return finish_out(ctx, Au, bytes, oh);
}

dds_status dds_local_solve(dds_ctx *ctx, int sub, const void *b, int nrhs, void *x) {
  if (!ctx) return DDS_EINVAL;
  Busy busy(ctx);
  if (!busy.ok) return DDS_EBUSY;
  ctx->err.clear();
  const Geom &g = ctx->g;
  if (!b || !x || nrhs <= 0 || sub < 0 || sub >= g.nsub) { ctx->err = "invalid argument"; return DDS_EINVAL; }
  const size_t bytes = (size_t)nrhs * g.Nloc * sizeof(double2);
  const double2 *bd;
  double2 *xd;
  bool xh;
  dds_status r = stage_in(ctx, b, bytes, &bd);
  if (r != DDS_OK) return r;
  r = stage_out_ptr(ctx, x, bytes, &xd, &xh);
  if (r != DDS_OK) return r;
  cudaStream_t st = ctx->stream;
  std::vector<Col> cols(nrhs);
  for (int q = 0; q < nrhs; ++q) cols[q] = Col{sub, q, q, 0};
  const bool mixed = ctx->single;
  const bool tc = mixed && ctx->split >= 0 && subst_tc_ok(g, ctx->split, 8, ctx->tc_m > 0);
  const int pc = tc ? 8 : std::min(4, max_pc_for(ctx, mixed ? sizeof(float2) : sizeof(double2)));
  std::vector<Panel> pans;
  for (int i = 0; i < nrhs; i += pc) pans.push_back(Panel{i, std::min(pc, nrhs - i), ctx->fac_of_sub[sub], 0});
  DBuf dcols, dpans;
  CK(upload(dcols, cols, st));
  CK(upload(dpans, pans, st));
  const long long n = (long long)nrhs * g.Nloc;
  if (mixed) {
    CK(ctx->work.ensure(n * sizeof(float2)));
    LAUNCH(launch_copy_local<float>(st, n, bd, ctx->work.as<float2>(), 1));
    if (tc)
      LAUNCHK(DDS_K_SUBST, subst_any<float>(ctx, (int)pans.size(), dpans.as<Panel>(), dcols.as<Col>(),
                                            ctx->sinv32.as<float2>(), ctx->cpl32.as<float2>(),
                                            ctx->work.as<float2>(), pc));
    else
      LAUNCHK(DDS_K_SUBST, launch_subst<float>(st, g, (int)pans.size(), dpans.as<Panel>(), dcols.as<Col>(),
                               ctx->sinv32.as<float2>(), ctx->cpl32.as<float2>(), ctx->work.as<float2>(), pc));
    LAUNCH(launch_copy_local_back<float>(st, n, ctx->work.as<float2>(), xd));
  } else {
    CK(ctx->work.ensure(n * sizeof(double2)));
    LAUNCH(launch_copy_local<double>(st, n, bd, ctx->work.as<double2>(), 1));
    LAUNCHK(DDS_K_SUBST, launch_subst<double>(st, g, (int)pans.size(), dpans.as<Panel>(), dcols.as<Col>(),
                                ctx->sinv64.as<double2>(), ctx->cpl64.as<double2>(), ctx->work.as<double2>(), pc));
    LAUNCH(launch_copy_local_back<double>(st, n, ctx->work.as<double2>(), xd));
  }
  // a bounded wait that gave up inside the substitutions leaves x wrong: report it here (and
  // clear the flag) instead of passing it on to the next call
  r = check_errflag(ctx);
  if (r != DDS_OK) return r;
  return finish_out(ctx, x, bytes, xh);
}

dds_status dds_set_stream(dds_ctx *ctx, void *cuda_stream) {
  if (!ctx) return DDS_EINVAL;
  Busy busy(ctx);
  if (!busy.ok) return DDS_EBUSY;
  ctx->stream = (cudaStream_t)cuda_stream;
  return DDS_OK;
}

dds_status dds_get_info(const dds_ctx *ctx, dds_info_t *info) {
  if (!ctx || !info) return DDS_EINVAL;
  for (int a = 0; a < 3; ++a) {
    info->G[a] = ctx->g.G[a];
    info->M[a] = ctx->g.M[a];
  }
  info->n_sub = ctx->g.nsub;
  info->n_factors = ctx->nfac;
  info->trace_len = ctx->g.T;
  info->plan = ctx->plan;
  info->factor_bytes = (long long)(ctx->sinv64.n + ctx->sinv32.n + ctx->gmap64.n + ctx->gmap32.n +
                                   ctx->tctiles.n + ctx->bigtiles.n + ctx->tttiles.n);
  info->setup_seconds = ctx->setup_seconds;
  info->device_bytes = (long long)ctx->acct.used;
  info->trace_kernel = ctx->plan != DDS_PLAN_TRACE ? -1 : (ctx->single && ctx->trace_tc ? 0 : ctx->trace_per_sm);
  info->subst_kernel = !ctx->single ? 0 : (ctx->split < 0 ? 1 : (ctx->big_tc ? 3 : 2));
  return DDS_OK;
}

long long dds_kernel_launches(const dds_ctx *ctx) { return ctx ? ctx->launches : 0; }

dds_status dds_autotune(dds_ctx *ctx, int nrhs, int rounds, int max_entries, int *n_entries,
                        double *table, int *best) {
  if (!ctx || nrhs <= 0 || rounds < 1 || !n_entries || !best || (max_entries > 0 && !table))
    return DDS_EINVAL;
  Busy busy(ctx);
  if (!busy.ok) return DDS_EBUSY;
  ctx->err.clear();
  const Geom &g = ctx->g;
  // substitution shapes (panel width, panels per CTA); 0 = automatic (non-tensor-core paths)
  std::vector<std::array<int, 2>> pcs = {{0, 1}};
  if (ctx->single && ctx->split >= 0) {
    pcs.clear();
    for (int np : {1, 2})
      for (int pc : {8, 16, 32})
        if (subst_tc_ok(g, ctx->split, pc, ctx->tc_m > 0, np)) pcs.push_back({pc, np});
  }
  // trace kernel: 1 or 2 = CUDA-core kernel with that many CTAs per SM, 0 = tensor-core kernel
  std::vector<int> pers = {ctx->trace_tc ? 0 : ctx->trace_per_sm};
  if (ctx->plan == DDS_PLAN_TRACE) {
    pers = {1, 2};
    if (ctx->trace_tc_avail) pers.push_back(0);
  }
  // synthetic right-hand sides, nonzero everywhere so that no local solve is skipped as zero
  // work (every byte 0x3F: each double is a finite ~5e-4)
  DBuf bb, uu;
  const size_t bytes = (size_t)nrhs * g.Nglob * sizeof(double2);
  CK(bb.ensure(bytes));
  CK(uu.ensure(bytes));
  CK(cudaMemsetAsync(bb.p, 0x3F, bytes, ctx->stream));
  cudaEvent_t e0, e1;
  CK(cudaEventCreate(&e0));
  CK(cudaEventCreate(&e1));
  const bool prof = ctx->profiling;
  ctx->profiling = false;
  double best_ms = 1e300;
  int best_pc = ctx->tune_pc, best_np = ctx->tune_np, best_per = ctx->trace_tc ? 0 : ctx->trace_per_sm;
  int n = 0;
  dds_status r = DDS_OK;
  for (const auto &shape : pcs)
    for (int per : pers) {
      const int pc = shape[0];
      ctx->tune_pc = pc;
      ctx->tune_np = shape[1];
      ctx->trace_tc = per == 0;
      if (per > 0) ctx->trace_per_sm = per;
      ctx->clear_graphs();
      ctx->plans.clear();
      r = ddm(ctx, bb.as<double2>(), nrhs, uu.as<double2>(), rounds);   // build + capture
      if (r != DDS_OK) break;
      const int reps = 3;
      cudaEventRecord(e0, ctx->stream);
      for (int k = 0; k < reps && r == DDS_OK; ++k)
        r = ddm(ctx, bb.as<double2>(), nrhs, uu.as<double2>(), rounds);
      cudaEventRecord(e1, ctx->stream);
      if (r != DDS_OK) break;
      cudaEventSynchronize(e1);
      float ms = 0.f;
      cudaEventElapsedTime(&ms, e0, e1);
      const double per_app = ms / reps;
      if (n < max_entries) {
        table[4 * n + 0] = pc;
        table[4 * n + 1] = shape[1];
        table[4 * n + 2] = per;
        table[4 * n + 3] = per_app;
      }
      ++n;
      if (per_app < best_ms) {
        best_ms = per_app;
        best_pc = pc;
        best_np = shape[1];
        best_per = per;
      }
    }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  ctx->profiling = prof;
  ctx->tune_pc = best_pc;
  ctx->tune_np = best_np;
  ctx->trace_tc = best_per == 0;
  if (best_per > 0) ctx->trace_per_sm = best_per;
  ctx->clear_graphs();
  ctx->plans.clear();
  if (r != DDS_OK) return r;
  CK(cudaStreamSynchronize(ctx->stream));
  *n_entries = n;
  best[0] = best_pc;
  best[1] = best_per;
  best[2] = best_np;
  return check_errflag(ctx);
}

dds_status dds_tensor_rate(int kind, double *tflops) {
  if (!tflops || (kind != 0 && kind != 1)) return DDS_EINVAL;
  *tflops = 0.0;
  int *err = nullptr;
  if (cudaMalloc(&err, sizeof(int)) != cudaSuccess) {
    cudaGetLastError();
    return DDS_ENOMEM;
  }
  int herr = 0;
  double flops = 0.0;
  float ms = 0.f;
  cudaError_t e = cudaMemset(err, 0, sizeof(int));
  if (e == cudaSuccess) e = measure_mma_rate(kind, 16384, err, &flops, &ms);
  if (e == cudaSuccess) e = cudaMemcpy(&herr, err, sizeof(int), cudaMemcpyDeviceToHost);
  cudaFree(err);
  if (e != cudaSuccess) return DDS_ECUDA;
  if (herr != 0) return DDS_ETIMEOUT;
  if (ms > 0.f) *tflops = flops / (ms * 1e-3) / 1e12;
  return DDS_OK;
}

dds_status dds_work_per_ddm(dds_ctx *ctx, int nrhs, int rounds, double *subst_flops,
                            double *trace_flops) {
  if (!ctx || nrhs <= 0 || rounds < 1 || !subst_flops || !trace_flops) return DDS_EINVAL;
  Busy busy(ctx);
  if (!busy.ok) return DDS_EBUSY;
  const Geom &g = ctx->g;
  dds_status r = set_route(ctx, rounds);
  if (r != DDS_OK) return r;
  const std::vector<int> route = build_route(g, rounds);
  const int L = (int)route.size() / 6;
  const double per_solve = 16.0 * g.Ml * (double)g.Mb * g.Mb;
  // substitutions: trace plan = own-source solves + final solves of every (sub, RHS);
  // direct plan = one solve per (sub, RHS) per sweep
  const double nsolves = ctx->plan == DDS_PLAN_TRACE ? 2.0 * g.nsub * nrhs : (double)L * g.nsub * nrhs;
  *subst_flops = per_solve * nsolves;
  // trace map applications (trace plan): per (sweep, sub, RHS), complex map rows of the routed
  // sides that have a neighbour times the inputs of the receiving sides that have one
  double tf = 0.0;
  if (ctx->plan == DDS_PLAN_TRACE) {
    for (int l = 0; l < L; ++l)
      for (int sub = 0; sub < g.nsub; ++sub) {
        double rows = 0.0, inputs = 0.0;
        for (int d = 0; d < g.nsides; ++d) {
          if (sub_neighbour(g, sub, d) < 0) continue;
          if (((ctx->out_mask[l] >> d) & 1) && route[l * 6 + d] >= 0) rows += 2.0 * g.Lt[d];
          if ((ctx->in_mask[l] >> d) & 1) inputs += 2.0 * g.Lt[d];
        }
        tf += 8.0 * rows * inputs * nrhs;
      }
  }
  *trace_flops = tf;
  return DDS_OK;
}

dds_status dds_profile(dds_ctx *ctx, int enable) {
  if (!ctx) return DDS_EINVAL;
  Busy busy(ctx);
  if (!busy.ok) return DDS_EBUSY;
  CK(prof_fold(ctx));
  ctx->profiling = enable != 0;
  if (enable)
    for (int k = 0; k < DDS_K_COUNT; ++k) ctx->prof_count[k] = 0, ctx->prof_ms[k] = 0.0;
  return DDS_OK;
}

dds_status dds_profile_read(dds_ctx *ctx, int kind, long long *launches, double *ms) {
  if (!ctx || kind < 0 || kind >= DDS_K_COUNT) return DDS_EINVAL;
  Busy busy(ctx);
  if (!busy.ok) return DDS_EBUSY;
  CK(prof_fold(ctx));
  if (launches) *launches = ctx->prof_count[kind];
  if (ms) *ms = ctx->prof_ms[kind];
  return DDS_OK;
}

dds_status dds_set_launch_shape(dds_ctx *ctx, int panel_width, int panels_per_cta,
                                int trace_kernel) {
  if (!ctx) return DDS_EINVAL;
  Busy busy(ctx);
  if (!busy.ok) return DDS_EBUSY;
  ctx->err.clear();
  const Geom &g = ctx->g;
  const bool tc = ctx->single && ctx->split >= 0;
  if (panel_width != 0 && !(tc && subst_tc_ok(g, ctx->split, panel_width, ctx->tc_m > 0,
                                               panels_per_cta))) {
    ctx->err = "dds_set_launch_shape: panel width / panels per CTA not available here";
    return DDS_EINVAL;
  }
  if (panel_width == 0 && panels_per_cta != 1) {
    ctx->err = "dds_set_launch_shape: panels per CTA needs an explicit panel width";
    return DDS_EINVAL;
  }
  if (trace_kernel < 0 || trace_kernel > 2 || (trace_kernel == 0 && !ctx->trace_tc_avail)) {
    ctx->err = "dds_set_launch_shape: trace kernel not available here";
    return DDS_EINVAL;
  }
  ctx->tune_pc = panel_width;
  ctx->tune_np = panels_per_cta;
  ctx->trace_tc = trace_kernel == 0;
  if (trace_kernel > 0) ctx->trace_per_sm = trace_kernel;
  ctx->clear_graphs();
  ctx->plans.clear();
  return DDS_OK;
}

dds_status dds_set_memory_budget(dds_ctx *ctx, long long bytes, long long *in_use) {
  if (!ctx || bytes < 0) return DDS_EINVAL;
  Busy busy(ctx);
  if (!busy.ok) return DDS_EBUSY;
  ctx->err.clear();
  ctx->acct.budget = (size_t)bytes;
  if (in_use) *in_use = (long long)ctx->acct.used;
  return DDS_OK;
}

dds_status dds_set_wait_limit(dds_ctx *ctx, long long polls) {
  if (!ctx || polls < 0 || polls > 0xFFFFFFFFLL) return DDS_EINVAL;
  Busy busy(ctx);
  if (!busy.ok) return DDS_EBUSY;
  ctx->err.clear();
  ctx->wait_limit = polls == 0 ? (1u << 20) : (unsigned)polls;
  ctx->clear_graphs();   // the limit is a launch argument of the captured launches
  return DDS_OK;
}

dds_status dds_set_zero_skip(dds_ctx *ctx, int enable) {
  if (!ctx) return DDS_EINVAL;
  Busy busy(ctx);
  if (!busy.ok) return DDS_EBUSY;
  ctx->err.clear();
  if ((enable != 0) != ctx->zero_skip) {
    ctx->zero_skip = enable != 0;
    ctx->clear_graphs();   // the captured launch sequences differ
  }
  return DDS_OK;
}

dds_status dds_local_solve_counts(dds_ctx *ctx, long long *solved, long long *assembled,
                                  int reset) {
  if (!ctx) return DDS_EINVAL;
  Busy busy(ctx);
  if (!busy.ok) return DDS_EBUSY;
  ctx->err.clear();
  unsigned long long h[2] = {0, 0};
  CK(cudaMemcpyAsync(h, ctx->solve_stats.p, sizeof(h), cudaMemcpyDeviceToHost, ctx->stream));
  CK(cudaStreamSynchronize(ctx->stream));
  if (solved) *solved = (long long)h[0];
  if (assembled) *assembled = (long long)h[1];
  if (reset) {
    CK(cudaMemsetAsync(ctx->solve_stats.p, 0, sizeof(h), ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
  }
  return DDS_OK;
}

const char *dds_last_error(const dds_ctx *ctx) { return ctx ? ctx->err.c_str() : "null context"; }

void dds_destroy(dds_ctx *ctx) {
  if (!ctx) return;
  if (ctx->stream) cudaStreamSynchronize(ctx->stream);
  else cudaDeviceSynchronize();
  for (dds_server *srv : ctx->servers) server_orphan(srv);
  delete ctx;
}

}  // extern "C"

// ============================================================================================
// Continuous-batching server: one FGMRES per slot, one batched DDM per step for all slots
// ============================================================================================
struct dds_server {
  dds_ctx *ctx = nullptr;
  int S = 0, maxit = 0, rounds = 1;
  size_t reserve = 0;   // budget bytes kept free for what a step allocates besides the slots
  double tol = 1e-6;
  long long N = 0;
  DBuf V, Z, B, U, bin, bout, hdev, part, coef;
  DBuf offs, hb;   // batched Arnoldi: per-entry base offsets, and h / norms in batch order
  struct Slot {
    int state = 0;              // 0 free, 1 active, 2 finished (waiting for poll)
    long long tag = 0;
    int j = 0, kused = 0;
    double beta = 0, relres = 0;
    std::vector<cd> H, cs, sn, g;
  };
  std::vector<Slot> slots;
  // a submitted source waiting for a slot: in a device buffer, or, when the context's budget has
  // no room for one more, in host memory (copied to the device at admission)
  struct Queued {
    long long tag;
    std::unique_ptr<DBuf> buf;
    std::vector<double2> host;
  };
  std::deque<Queued> queue;
  // spent queue buffers, reused by later submissions (no cudaMalloc / cudaFree per request,
  // both of which synchronise the whole device); reuse is ordered by the context's stream
  std::vector<std::unique_ptr<DBuf>> pool;
  std::deque<int> finished;
  double2 *Vs(int s, int j) { return V.as<double2>() + ((long long)s * (maxit + 1) + j) * N; }
  double2 *Zs(int s, int j) { return Z.as<double2>() + ((long long)s * maxit + j) * N; }
  double2 *Bs(int s) { return B.as<double2>() + (long long)s * N; }
  double2 *Us(int s) { return U.as<double2>() + (long long)s * N; }
  double2 *Hd(int s) { return hdev.as<double2>() + (long long)s * (2 * maxit + 3); }
};

namespace {

#define SCK(call)                                                                \
  do {                                                                           \
    cudaError_t e_ = (call);                                                     \
    if (e_ != cudaSuccess) {                                                     \
      srv->ctx->err = std::string(#call) + ": " + cudaGetErrorString(e_);        \
      return DDS_ECUDA;                                                          \
    }                                                                            \
  } while (0)

int server_nblk(const dds_server *srv) {
  return (int)((srv->N + dots_chunk() - 1) / dots_chunk());
}

// x = sum_i Z_i y_i from the slot's Hessenberg system, then the true residual
// Finish slots `fin`: x = sum_i y_i Z_i from the slot's Hessenberg system, then the true
// residual ||A x - b|| / ||b||; batched over the slots with the same basis length (offset tables
// address their vectors), one readback for all.
dds_status server_finalize(dds_server *srv, const std::vector<int> &fin) {
  if (fin.empty()) return DDS_OK;
  dds_ctx *ctx = srv->ctx;
  cudaStream_t st = ctx->stream;
  const long long N = srv->N;
  const int m = srv->maxit;
  const long long vslot = (long long)(m + 1) * N, zslot = (long long)m * N;
  std::map<int, std::vector<int>> groups;   // basis length -> slots
  for (int s : fin) groups[srv->slots[s].kused].push_back(s);
  double2 *hb = srv->hb.as<double2>();
  long long *doff = srv->offs.as<long long>();
  double2 *coef = srv->coef.as<double2>();
  std::vector<std::pair<int, long long>> where;   // (slot, norm index in hb)
  long long used = 0;
  for (auto &grp : groups) {
    const int kr = grp.first, kg = (int)grp.second.size();
    std::vector<double2> yc((size_t)kg * std::max(kr, 1), make_double2(0.0, 0.0));
    std::vector<long long> off(3 * (size_t)srv->S);
    for (int i = 0; i < kg; ++i) {
      const int s = grp.second[i];
      auto &sl = srv->slots[s];
      auto Hat = [&](int a, int b) -> cd & { return sl.H[(size_t)a * m + b]; };
      std::vector<cd> y(kr, cd(0, 0));
      for (int a = kr - 1; a >= 0; --a) {
        cd t = sl.g[a];
        for (int q = a + 1; q < kr; ++q) t -= Hat(a, q) * y[q];
        y[a] = t / Hat(a, a);
      }
      for (int a = 0; a < kr; ++a) yc[(size_t)i * kr + a] = make_double2(y[a].real(), y[a].imag());
      off[i] = (long long)s * zslot;                // Z_0
      off[srv->S + i] = (long long)s * N;           // U (solution) and B (source): slot s
      off[2 * srv->S + i] = (long long)s * vslot;   // residual in V_0 (no longer needed)
      where.emplace_back(s, used + i);
    }
    const long long *zo = doff, *uo = doff + srv->S, *wo = doff + 2 * srv->S;
    SCK(cudaMemcpyAsync(doff, off.data(), 3 * srv->S * sizeof(long long), cudaMemcpyHostToDevice, st));
    double2 *U = srv->U.as<double2>(), *Vb = srv->V.as<double2>();
    if (kr > 0) {
      // coefficients after the unit entries of the residual update: [kg ones][kg * kr y]
      std::vector<double2> cbuf((size_t)kg + yc.size());
      for (int i = 0; i < kg; ++i) cbuf[i] = make_double2(1.0, 0.0);
      std::copy(yc.begin(), yc.end(), cbuf.begin() + kg);
      SCK(cudaMemcpyAsync(coef, cbuf.data(), cbuf.size() * sizeof(double2), cudaMemcpyHostToDevice, st));
      ctx->launches += 1;
      SCK(launch_combination(st, N, kg, kr, srv->Z.as<double2>(), N, 0, coef + kg, kr, 1.0, U, 0,
                             true, nullptr, nullptr, 0, nullptr, zo, uo));
    } else {
      const std::vector<double2> ones((size_t)kg, make_double2(1.0, 0.0));
      SCK(cudaMemcpyAsync(coef, ones.data(), kg * sizeof(double2), cudaMemcpyHostToDevice, st));
      for (int i = 0; i < kg; ++i)
        SCK(cudaMemsetAsync(srv->Us(grp.second[i]), 0, N * sizeof(double2), st));
    }
    // residual W = A x - b and its squared norm in the same update pass
    ctx->launches += 3;
    SCK(launch_apply_A(st, ctx->g, ctx->tb, kg, U, Vb, 0, nullptr, uo, wo));
    SCK(launch_combination(st, N, kg, 1, srv->B.as<double2>(), 0, 0, coef, 1, -1.0, Vb, 0, false,
                           srv->part.as<double2>(), hb + used, server_nblk(srv), nullptr, uo, wo));
    used += kg;
    // the next group's tables and coefficients are copied in stream order, after these kernels
  }
  std::vector<double2> r2((size_t)used);
  SCK(cudaMemcpyAsync(r2.data(), hb, (size_t)used * sizeof(double2), cudaMemcpyDeviceToHost, st));
  SCK(cudaStreamSynchronize(st));
  for (auto &w : where) {
    auto &sl = srv->slots[w.first];
    sl.relres = sl.beta > 0 ? std::sqrt(std::max(r2[w.second].x, 0.0)) / sl.beta : 0.0;
    sl.state = 2;
    srv->finished.push_back(w.first);
  }
  return DDS_OK;
}

}  // namespace

void server_orphan(dds_server *srv) {
  if (!srv) return;
  srv->queue.clear();
  srv->pool.clear();
  srv->finished.clear();
  srv->slots.clear();
  for (DBuf *b : {&srv->V, &srv->Z, &srv->B, &srv->U, &srv->bin, &srv->bout, &srv->hdev,
                  &srv->part, &srv->coef, &srv->offs, &srv->hb})
    b->release();
  srv->S = 0;
  srv->ctx = nullptr;
}

namespace {

dds_status server_admit(dds_server *srv) {
  dds_ctx *ctx = srv->ctx;
  cudaStream_t st = ctx->stream;
  const long long N = srv->N;
  // every admission of this step is launched first; their norms come back in one read
  std::vector<int> admitted;
  std::vector<double2> b2(srv->S);
  std::vector<std::vector<double2>> kept;
  for (int s = 0; s < srv->S && !srv->queue.empty(); ++s) {
    auto &sl = srv->slots[s];
    if (sl.state != 0) continue;
    auto req = std::move(srv->queue.front());
    srv->queue.pop_front();
    sl = dds_server::Slot();
    sl.state = 1;
    sl.tag = req.tag;
    const int m = srv->maxit;
    sl.H.assign((size_t)(m + 1) * m, cd(0, 0));
    sl.cs.assign(m, cd(0, 0));
    sl.sn.assign(m, cd(0, 0));
    sl.g.assign(m + 1, cd(0, 0));
    ctx->launches += 3;
    const double2 *src = nullptr;
    if (req.buf) {
      src = req.buf->as<double2>();
    } else {
      // a source queued in host memory goes through this slot's part of the DDM input buffer
      // (rewritten later in the step, on the same stream)
      double2 *stage = srv->bin.as<double2>() + (long long)s * N;
      SCK(cudaMemcpyAsync(stage, req.host.data(), (size_t)N * sizeof(double2),
                          cudaMemcpyHostToDevice, st));
      src = stage;
      kept.push_back(std::move(req.host));   // alive until the synchronisation below
    }
    SCK(launch_scale_J(st, ctx->g, ctx->tb, 1, src, srv->Bs(s)));
    if (req.buf) srv->pool.push_back(std::move(req.buf));   // later copies into it follow on the stream
    SCK(launch_dots(st, N, 1, 1, srv->Bs(s), 0, 0, srv->Bs(s), 0, srv->part.as<double2>(),
                    srv->Hd(s), server_nblk(srv)));
    SCK(launch_scale_by_norm(st, N, 1, srv->Bs(s), srv->Hd(s), srv->Vs(s, 0)));
    SCK(cudaMemcpyAsync(&b2[s], srv->Hd(s), sizeof(double2), cudaMemcpyDeviceToHost, st));
    admitted.push_back(s);
  }
  if (admitted.empty()) return DDS_OK;
  SCK(cudaStreamSynchronize(st));
  std::vector<int> zero;
  for (int s : admitted) {
    auto &sl = srv->slots[s];
    sl.beta = std::sqrt(std::max(b2[s].x, 0.0));
    sl.g[0] = sl.beta;
    if (sl.beta == 0.0) {   // zero source: the solution is zero
      sl.kused = 0;
      zero.push_back(s);
    }
  }
  dds_status rz = server_finalize(srv, zero);
  if (rz != DDS_OK) return rz;
  return DDS_OK;
}

dds_status server_step(dds_server *srv, int *active_out, int *queued_out) {
  dds_ctx *ctx = srv->ctx;
  cudaStream_t st = ctx->stream;
  const long long N = srv->N;
  dds_status r = server_admit(srv);
  if (r != DDS_OK) return r;
  std::vector<int> act;
  for (int s = 0; s < srv->S; ++s)
    if (srv->slots[s].state == 1) act.push_back(s);
  const int k = (int)act.size();
  if (k > 0) {
    // one batched DDM application over every active slot's current Krylov vector
    for (int i = 0; i < k; ++i)
      SCK(cudaMemcpyAsync(srv->bin.as<double2>() + (long long)i * N,
                          srv->Vs(act[i], srv->slots[act[i]].j), N * sizeof(double2),
                          cudaMemcpyDeviceToDevice, st));
    r = ddm(ctx, srv->bin.as<double2>(), k, srv->bout.as<double2>(), srv->rounds);
    if (r == DDS_ENOMEM && !srv->pool.empty()) {
      // idle queue buffers give their memory back to the step, which is tried once more
      SCK(cudaStreamSynchronize(st));
      srv->pool.clear();
      ctx->err.clear();
      r = ddm(ctx, srv->bin.as<double2>(), k, srv->bout.as<double2>(), srv->rounds);
    }
    if (r != DDS_OK) return r;
    const int nblk = server_nblk(srv);
    const long long vslot = (long long)(srv->maxit + 1) * N, zslot = (long long)srv->maxit * N;
    for (int i = 0; i < k; ++i) {
      const int s = act[i];
      SCK(cudaMemcpyAsync(srv->Zs(s, srv->slots[s].j), srv->bout.as<double2>() + (long long)i * N,
                          N * sizeof(double2), cudaMemcpyDeviceToDevice, st));
    }
    // FP64 Arnoldi step, batched over the active slots at the same iteration j (their vectors
    // are addressed through offset tables): classical Gram-Schmidt twice, the norm with the
    // second update, then normalisation.  hb holds, per group, h1 [k][j+1], h2 [k][j+1] and
    // the squared norms [k].
    std::map<int, std::vector<int>> groups;   // j -> slots
    for (int s : act) groups[srv->slots[s].j].push_back(s);
    std::vector<long long> off(3 * (size_t)srv->S);
    std::vector<std::array<long long, 3>> where(srv->S);   // slot -> (h1, h2, norm) offsets in hb
    long long used = 0;
    double2 *hb = srv->hb.as<double2>();
    long long *doff = srv->offs.as<long long>();
    for (auto &grp : groups) {
      const int j = grp.first, kg = (int)grp.second.size(), nv = j + 1;
      for (int i = 0; i < kg; ++i) {
        const int s = grp.second[i];
        off[i] = (long long)s * zslot + (long long)j * N;                   // Z_j
        off[srv->S + i] = (long long)s * vslot;                             // V_0
        off[2 * srv->S + i] = (long long)s * vslot + (long long)(j + 1) * N;   // W = V_{j+1}
        where[s] = {used + (long long)i * nv, used + (long long)kg * nv + (long long)i * nv,
                    used + 2LL * kg * nv + i};
      }
      SCK(cudaMemcpyAsync(doff, off.data(), 3 * srv->S * sizeof(long long),
                          cudaMemcpyHostToDevice, st));
      const long long *zo = doff, *vo = doff + srv->S, *wo = doff + 2 * srv->S;
      double2 *h1 = hb + used, *h2 = h1 + (long long)kg * nv, *hn = h2 + (long long)kg * nv;
      double2 *Vb = srv->V.as<double2>();
      ctx->launches += 6;
      SCK(launch_apply_A(st, ctx->g, ctx->tb, kg, srv->Z.as<double2>(), Vb, 0, nullptr, zo, wo));
      SCK(launch_dots(st, N, kg, nv, Vb, N, 0, Vb, 0, srv->part.as<double2>(), h1, nblk, vo, wo));
      SCK(launch_combination(st, N, kg, nv, Vb, N, 0, h1, nv, -1.0, Vb, 0, false, nullptr,
                             nullptr, 0, nullptr, vo, wo));
      SCK(launch_dots(st, N, kg, nv, Vb, N, 0, Vb, 0, srv->part.as<double2>(), h2, nblk, vo, wo));
      SCK(launch_combination(st, N, kg, nv, Vb, N, 0, h2, nv, -1.0, Vb, 0, false,
                             srv->part.as<double2>(), hn, nblk, nullptr, vo, wo));
      SCK(launch_scale_by_norm(st, N, kg, Vb, hn, Vb, wo));
      used += 2LL * kg * nv + kg;
      // (the next group's offset table is copied in stream order, after these kernels)
    }
    std::vector<double2> hh((size_t)used);
    SCK(cudaMemcpyAsync(hh.data(), hb, (size_t)used * sizeof(double2), cudaMemcpyDeviceToHost, st));
    SCK(cudaStreamSynchronize(st));
    const int m = srv->maxit;
    std::vector<int> fin;   // slots that finish this step
    for (int i = 0; i < k; ++i) {
      const int s = act[i];
      auto &sl = srv->slots[s];
      const int j = sl.j;
      const double2 *h1 = hh.data() + where[s][0], *h2 = hh.data() + where[s][1];
      auto Hat = [&](int a, int b) -> cd & { return sl.H[(size_t)a * m + b]; };
      for (int q = 0; q <= j; ++q) Hat(q, j) = cd(h1[q].x + h2[q].x, h1[q].y + h2[q].y);
      const double hn = std::sqrt(std::max(hh[where[s][2]].x, 0.0));
      Hat(j + 1, j) = hn;
      for (int q = 0; q < j; ++q) {
        const cd a = Hat(q, j), bb = Hat(q + 1, j), c = sl.cs[q], sn = sl.sn[q];
        Hat(q, j) = c * a + sn * bb;
        Hat(q + 1, j) = -std::conj(sn) * a + std::conj(c) * bb;
      }
      const cd a = Hat(j, j), bb = Hat(j + 1, j);
      const double rr = std::hypot(std::abs(a), std::abs(bb));
      cd c(1, 0), sn(0, 0);
      if (rr > 0) { c = std::conj(a / rr); sn = std::conj(bb / rr); }
      sl.cs[j] = c;
      sl.sn[j] = sn;
      Hat(j, j) = c * a + sn * bb;
      Hat(j + 1, j) = 0.0;
      const cd gj = sl.g[j];
      sl.g[j + 1] = -std::conj(sn) * gj;
      sl.g[j] = c * gj;
      sl.j = j + 1;
      sl.kused = j + 1;
      const double res = std::abs(sl.g[j + 1]) / sl.beta;
      if (res < srv->tol || hn == 0.0 || sl.j >= m) fin.push_back(s);
    }
    r = server_finalize(srv, fin);
    if (r != DDS_OK) return r;
  }
  r = check_errflag(ctx);
  if (r != DDS_OK) return r;
  int a = 0;
  for (auto &sl : srv->slots) a += sl.state == 1;
  if (active_out) *active_out = a;
  if (queued_out) *queued_out = (int)srv->queue.size();
  return DDS_OK;
}

}  // namespace

extern "C" {

// device bytes one server slot needs: its Krylov basis and batch fields, its share of the
// Arnoldi scratch, and its columns in the DDM work buffers of a batched application
static size_t server_slot_bytes(const dds_ctx *ctx, int maxit, int rounds) {
  const Geom &g = ctx->g;
  const size_t fb = (size_t)g.Nglob * sizeof(double2);
  const size_t elem = ctx->single ? sizeof(float2) : sizeof(double2);
  const size_t L = sweep_program(g, rounds).size();
  size_t b = fb * ((size_t)(maxit + 1) + (size_t)maxit + 4);
  b += (size_t)(2 * (2 * maxit + 3) + (maxit + 2)) * sizeof(double2) + 3 * sizeof(long long);
  b += (size_t)(maxit + 2) * ((size_t)g.Nglob / dots_chunk() + 2) * sizeof(double2);
  b += (size_t)g.nsub * ((size_t)g.Nloc * elem + (L + 1) * (size_t)g.T * elem + 2 * sizeof(int));
  return b;
}

dds_status dds_server_create(dds_ctx *ctx, int max_slots, double tol, int maxit, int rounds,
                             dds_server **out) {
  if (!ctx || !out || max_slots < 1 || maxit < 1 || rounds < 1 || !(tol > 0)) return DDS_EINVAL;
  Busy busy(ctx);   // the slots' memory counts against the context (dds_set_memory_budget)
  if (!busy.ok) return DDS_EBUSY;
  ctx->err.clear();
  // admission by device memory: as many slots as seven eighths of what the context's budget (or,
  // without one, 90% of the device's free memory) leaves room for, up to max_slots
  const size_t per_slot = server_slot_bytes(ctx, maxit, rounds);
  size_t room = 0;
  if (ctx->acct.budget) {
    room = ctx->acct.budget > ctx->acct.used ? ctx->acct.budget - ctx->acct.used : 0;
  } else {
    size_t fr = 0, tot = 0;
    CK(cudaMemGetInfo(&fr, &tot));
    room = fr / 10 * 9;
  }
  // an eighth of the room stays free for what a step allocates besides the slots: the DDM plan
  // of each batch size (trace schedules, tables) and the growth of shared work buffers
  const size_t reserve = room / 8;
  room -= reserve;
  const long long fit = (long long)(room / per_slot);
  if (fit < 1) {
    ctx->err = "dds_server_create: one slot needs " + std::to_string(per_slot) +
               " device bytes, " + std::to_string(room) + " are available";
    return DDS_ENOMEM;
  }
  std::unique_ptr<dds_server> srv(new (std::nothrow) dds_server());
  if (!srv) return DDS_ENOMEM;
  srv->ctx = ctx;
  srv->S = (int)std::min<long long>(max_slots, fit);
  srv->reserve = ctx->acct.budget ? reserve : 0;
  srv->maxit = maxit;
  srv->rounds = rounds;
  srv->tol = tol;
  srv->N = ctx->g.Nglob;
  const size_t fb = (size_t)srv->N * sizeof(double2);
  const size_t S = (size_t)srv->S;
  bool ok = srv->V.ensure(S * (maxit + 1) * fb) == cudaSuccess &&
            srv->Z.ensure(S * maxit * fb) == cudaSuccess &&
            srv->B.ensure(S * fb) == cudaSuccess && srv->U.ensure(S * fb) == cudaSuccess &&
            srv->bin.ensure(S * fb) == cudaSuccess && srv->bout.ensure(S * fb) == cudaSuccess &&
            srv->hdev.ensure(S * (2 * maxit + 3) * sizeof(double2)) == cudaSuccess &&
            srv->part.ensure(S * (maxit + 2) * (srv->N / dots_chunk() + 2) * sizeof(double2)) ==
                cudaSuccess &&
            srv->coef.ensure(S * (maxit + 2) * sizeof(double2)) == cudaSuccess &&
            srv->offs.ensure(3 * S * sizeof(long long)) == cudaSuccess &&
            srv->hb.ensure(S * (2 * maxit + 3) * sizeof(double2)) == cudaSuccess;
  if (!ok) {
    cudaGetLastError();
    ctx->err = "dds_server_create: device memory for " + std::to_string(srv->S) +
               " slots is not available";
    return DDS_ENOMEM;
  }
  srv->slots.resize(srv->S);
  ctx->servers.push_back(srv.get());
  *out = srv.release();
  return DDS_OK;
}

int dds_server_slots(const dds_server *srv) { return srv ? srv->S : 0; }

dds_status dds_server_submit(dds_server *srv, const void *f, long long tag) {
  if (!srv || !f || !srv->ctx) return DDS_EINVAL;
  dds_ctx *ctx = srv->ctx;
  Busy busy(ctx);
  if (!busy.ok) return DDS_EBUSY;
  // waiting sources take device copies while the budget has room beyond the reserve a step
  // needs; the rest wait in host memory
  std::unique_ptr<DBuf> buf;
  if (!srv->pool.empty()) {
    buf = std::move(srv->pool.back());
    srv->pool.pop_back();
  } else {
    buf = std::make_unique<DBuf>();
  }
  const size_t fb = (size_t)srv->N * sizeof(double2);
  dds_server::Queued q{tag, nullptr, {}};
  const bool room = buf->p || !ctx->acct.budget ||
                    ctx->acct.used + fb + srv->reserve <= ctx->acct.budget;
  const cudaError_t e = room ? buf->ensure(fb) : cudaErrorMemoryAllocation;
  if (e != cudaSuccess && buf->p) srv->pool.push_back(std::move(buf));   // kept for later
  if (e == cudaSuccess) {
    CK(cudaMemcpyAsync(buf->p, f, fb, is_device_ptr(f) ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice,
                       ctx->stream));
    q.buf = std::move(buf);
  } else if (e == cudaErrorMemoryAllocation) {
    // no device room for one more waiting source (the budget, or the device itself): it waits
    // in host memory instead
    cudaGetLastError();
    try {
      q.host.resize((size_t)srv->N);
    } catch (const std::bad_alloc &) {
      ctx->err = "dds_server_submit: no device or host memory for the source";
      return DDS_ENOMEM;
    }
    if (is_device_ptr(f))
      CK(cudaMemcpyAsync(q.host.data(), f, fb, cudaMemcpyDeviceToHost, ctx->stream));
    else
      std::memcpy(q.host.data(), f, fb);
  } else {
    CK(e);
  }
  CK(cudaStreamSynchronize(ctx->stream));
  srv->queue.push_back(std::move(q));
  return DDS_OK;
}

dds_status dds_server_step(dds_server *srv, int *active, int *queued) {
  if (!srv || !srv->ctx) return DDS_EINVAL;
  Busy busy(srv->ctx);
  if (!busy.ok) return DDS_EBUSY;
  srv->ctx->err.clear();
  return server_step(srv, active, queued);
}

dds_status dds_server_poll(dds_server *srv, long long *tag, void *u, int *iters, double *relres) {
  if (!srv || !u || !srv->ctx) return DDS_EINVAL;
  dds_ctx *ctx = srv->ctx;
  Busy busy(ctx);
  if (!busy.ok) return DDS_EBUSY;
  if (srv->finished.empty()) return DDS_EBUSY;
  const int s = srv->finished.front();
  auto &sl = srv->slots[s];
  const size_t fb = (size_t)srv->N * sizeof(double2);
  CK(cudaMemcpyAsync(u, srv->Us(s), fb, is_device_ptr(u) ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost,
                     ctx->stream));
  CK(cudaStreamSynchronize(ctx->stream));
  if (tag) *tag = sl.tag;
  if (iters) *iters = sl.kused;
  if (relres) *relres = sl.relres;
  srv->finished.pop_front();
  sl.state = 0;
  return DDS_OK;
}

void dds_server_destroy(dds_server *srv) {
  if (!srv) return;
  if (dds_ctx *ctx = srv->ctx) {   // (an orphaned server's context is gone already)
    if (ctx->stream) cudaStreamSynchronize(ctx->stream);
    auto &v = ctx->servers;
    v.erase(std::remove(v.begin(), v.end(), srv), v.end());
  }
  delete srv;
}

}  // extern "C"

// ============================================================================================
// Allocation-free local solve
//
// Some callers cannot let this library call cudaMalloc: a host program whose device memory is
// fully reserved by another allocator (a framework's caching allocator, a fixed serving budget)
// gets an out-of-memory error or evicts its own cache, and every cudaMalloc / cudaFree may
// synchronise the whole device, stalling that caller's other streams.  dds_local_solve_noalloc
// gives them the block-tridiagonal local solve with all of its scratch (the working copy of the
// right-hand sides and the launch descriptors) in the fixed device array below, which is part
// of the loaded module: every GPU that loads libdds holds these bytes until the process exits.
// ============================================================================================
namespace {

constexpr size_t kStaticScratchBytes = size_t(8) << 20;   // 8 MiB per device
constexpr size_t kStaticDescBytes = size_t(16) << 10;     // first 16 KiB: column/panel lists
constexpr int kStaticMaxRhs = 256;
constexpr int kMaxDevices = 64;

static __device__ __align__(256) unsigned char dds_static_scratch[kStaticScratchBytes];
static_assert(kStaticMaxRhs * (sizeof(Col) + sizeof(Panel)) <= kStaticDescBytes,
              "descriptor area too small");

std::mutex g_static_mu;
void *g_static_addr[kMaxDevices] = {nullptr};

// device address of dds_static_scratch on the current device (looked up once per device)
cudaError_t static_scratch_address(void **out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lk(g_static_mu);
  if (!g_static_addr[dev]) {
    void *p = nullptr;
    e = cudaGetSymbolAddress(&p, dds_static_scratch);
    if (e != cudaSuccess) return e;
    g_static_addr[dev] = p;
  }
  *out = g_static_addr[dev];
  return cudaSuccess;
}

}  // namespace

extern "C" dds_status dds_local_solve_noalloc(dds_ctx *ctx, int sub, const void *b, int nrhs,
                                              void *x) {
  if (!ctx) return DDS_EINVAL;
  Busy busy(ctx);
  if (!busy.ok) return DDS_EBUSY;
  ctx->err.clear();
  const Geom &g = ctx->g;
  if (!b || !x || nrhs <= 0 || sub < 0 || sub >= g.nsub) { ctx->err = "invalid argument"; return DDS_EINVAL; }
  if (!is_device_ptr(b) || !is_device_ptr(x)) {
    ctx->err = "dds_local_solve_noalloc needs device pointers for b and x";
    return DDS_EINVAL;
  }
  const bool mixed = ctx->single;
  const size_t elem = mixed ? sizeof(float2) : sizeof(double2);
  const long long n = (long long)nrhs * g.Nloc;
  if (nrhs > kStaticMaxRhs || (size_t)n * elem > kStaticScratchBytes - kStaticDescBytes) {
    ctx->err = "dds_local_solve_noalloc: " + std::to_string(nrhs) + " right-hand sides of " +
               std::to_string(g.Nloc) + " nodes need " + std::to_string((size_t)n * elem) +
               " scratch bytes; the static scratch holds " +
               std::to_string(kStaticScratchBytes - kStaticDescBytes) + " (and at most " +
               std::to_string(kStaticMaxRhs) + " right-hand sides)";
    return DDS_EINVAL;
  }
  void *base = nullptr;
  CK(static_scratch_address(&base));
  unsigned char *scratch = static_cast<unsigned char *>(base);
  Col *dcols = reinterpret_cast<Col *>(scratch);
  Panel *dpans = reinterpret_cast<Panel *>(scratch + kStaticMaxRhs * sizeof(Col));
  void *work = scratch + kStaticDescBytes;
  // launch descriptors, built on the stack and copied into the static scratch
  Col cols[kStaticMaxRhs];
  Panel pans[kStaticMaxRhs];
  const bool tc = mixed && ctx->split >= 0 && subst_tc_ok(g, ctx->split, 8, ctx->tc_m > 0);
  const int pc = tc ? 8 : std::min(4, max_pc_for(ctx, elem));
  int npan = 0;
  for (int q = 0; q < nrhs; ++q) cols[q] = Col{sub, q, q, 0};
  for (int i = 0; i < nrhs; i += pc) pans[npan++] = Panel{i, std::min(pc, nrhs - i), ctx->fac_of_sub[sub], 0};
  cudaStream_t st = ctx->stream;
  CK(cudaMemcpyAsync(dcols, cols, nrhs * sizeof(Col), cudaMemcpyHostToDevice, st));
  CK(cudaMemcpyAsync(dpans, pans, npan * sizeof(Panel), cudaMemcpyHostToDevice, st));
  const double2 *bd = static_cast<const double2 *>(b);
  double2 *xd = static_cast<double2 *>(x);
  if (mixed) {
    float2 *w = static_cast<float2 *>(work);
    LAUNCH(launch_copy_local<float>(st, n, bd, w, 1));
    if (tc)
      LAUNCHK(DDS_K_SUBST, subst_any<float>(ctx, npan, dpans, dcols, ctx->sinv32.as<float2>(),
                                            ctx->cpl32.as<float2>(), w, pc));
    else
      LAUNCHK(DDS_K_SUBST, launch_subst<float>(st, g, npan, dpans, dcols, ctx->sinv32.as<float2>(),
                                               ctx->cpl32.as<float2>(), w, pc));
    LAUNCH(launch_copy_local_back<float>(st, n, w, xd));
  } else {
    double2 *w = static_cast<double2 *>(work);
    LAUNCH(launch_copy_local<double>(st, n, bd, w, 1));
    LAUNCHK(DDS_K_SUBST, launch_subst<double>(st, g, npan, dpans, dcols, ctx->sinv64.as<double2>(),
                                              ctx->cpl64.as<double2>(), w, pc));
    LAUNCH(launch_copy_local_back<double>(st, n, w, xd));
  }
  // synchronises the stream; DDS_ETIMEOUT (flag cleared) if a bounded wait gave up
  return check_errflag(ctx);
}
