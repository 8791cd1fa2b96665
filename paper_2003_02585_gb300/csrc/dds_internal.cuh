// Internal declarations shared by the libdds translation units.
//
// Layouts (all device arrays, x1 fastest):
//   global fields      [rhs][G2][G1][G0]             complex double (interleaved)
//   local work         [slot][Ml][Mb]                complex R  (Ml blocks of Mb nodes; the
//                                                    block axis is the last axis, x2 in 2D,
//                                                    x3 in 3D)
//   block inverses     [factor][j][s][r]             S_j^{-1}, complex R
//   block couplings    [factor][j][r]                A(line j, line j+1) at in-block index r
//   trace vectors      [..][T]                       per side d (d = 2a + (sign < 0)):
//                                                    [a-line Lt_d][b-line Lt_d] at toff_d;
//                                                    a on the holder's outer line, b on its
//                                                    inner line; tangential index t runs over
//                                                    the other axes, lowest axis fastest
#pragma once

#include <cuda_runtime.h>
#include <cstdint>
#include <vector>

namespace dds {

// ------------------------------------------------------------------------------------------
// complex helpers (interleaved float2 / double2)
// ------------------------------------------------------------------------------------------
template <typename R> struct Cx;
template <> struct Cx<float> { using T = float2; };
template <> struct Cx<double> { using T = double2; };

template <typename C> __host__ __device__ inline C cmk(double re, double im) {
  C z; z.x = (decltype(z.x))re; z.y = (decltype(z.y))im; return z;
}
__host__ __device__ inline float2 cadd(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
__host__ __device__ inline double2 cadd(double2 a, double2 b) { return make_double2(a.x + b.x, a.y + b.y); }
__host__ __device__ inline float2 csub(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }
__host__ __device__ inline double2 csub(double2 a, double2 b) { return make_double2(a.x - b.x, a.y - b.y); }
__host__ __device__ inline float2 cmul(float2 a, float2 b) {
  return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__host__ __device__ inline double2 cmul(double2 a, double2 b) {
  return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
// acc += a * b
__host__ __device__ inline void cfma(float2 &acc, float2 a, float2 b) {
  acc.x = fmaf(a.x, b.x, acc.x); acc.x = fmaf(-a.y, b.y, acc.x);
  acc.y = fmaf(a.x, b.y, acc.y); acc.y = fmaf(a.y, b.x, acc.y);
}
__host__ __device__ inline void cfma(double2 &acc, double2 a, double2 b) {
  acc.x = fma(a.x, b.x, acc.x); acc.x = fma(-a.y, b.y, acc.x);
  acc.y = fma(a.x, b.y, acc.y); acc.y = fma(a.y, b.x, acc.y);
}
template <typename C> __host__ __device__ inline C czero() { C z; z.x = 0; z.y = 0; return z; }
__host__ __device__ inline float2 to_c(double2 a, float2) { return make_float2((float)a.x, (float)a.y); }
__host__ __device__ inline double2 to_c(double2 a, double2) { return a; }
__host__ __device__ inline double2 to_c64(float2 a) { return make_double2(a.x, a.y); }
__host__ __device__ inline double2 to_c64(double2 a) { return a; }

// ------------------------------------------------------------------------------------------
// geometry of one problem
// ------------------------------------------------------------------------------------------
struct Geom {
  int dim;
  int n[3], parts[3], m[3], M[3], G[3];
  int E;
  int nsub;
  long long Nloc, Nglob;   // nodes of one extended subdomain / of the global extended grid
  int Mb, Ml;              // block size (nodes of a line/plane) and number of blocks
  long long St;            // element stride between block inverses (Mb^2 rounded up to even,
                           // so that every tile starts on a 16-byte boundary)
  int nsides;              // 2 * dim
  int Lt[6];               // line length of side d
  int toff[6];             // offset of side d in a trace vector
  int T;                   // trace vector length (sum of 2 * Lt)
};

// subdomain multi-index from its linear index (x1 fastest)
__host__ __device__ inline void sub_index(const Geom &g, int s, int k[3]) {
  k[0] = s % g.parts[0];
  k[1] = (s / g.parts[0]) % g.parts[1];
  k[2] = g.dim == 3 ? s / (g.parts[0] * g.parts[1]) : 0;
}
__host__ __device__ inline int sub_linear(const Geom &g, const int k[3]) {
  return k[0] + g.parts[0] * (k[1] + g.parts[1] * k[2]);
}
// neighbour across side d or -1
__host__ __device__ inline int sub_neighbour(const Geom &g, int s, int d) {
  int k[3];
  sub_index(g, s, k);
  int a = d >> 1, sg = (d & 1) ? -1 : 1;
  k[a] += sg;
  if (k[a] < 0 || k[a] >= g.parts[a]) return -1;
  return sub_linear(g, k);
}
// local index, along axis a of side d, of the inner (first own) / outer line
__host__ __device__ inline int inner_line(const Geom &g, int d) {
  int a = d >> 1;
  return (d & 1) ? g.E : g.E + g.m[a] - 1;
}
__host__ __device__ inline int outer_line(const Geom &g, int d) {
  int a = d >> 1;
  return (d & 1) ? g.E - 1 : g.E + g.m[a];
}
// local linear index of the node at position l along axis a and tangential index t
__host__ __device__ inline long long line_node(const Geom &g, int a, int l, int t) {
  int i[3] = {0, 0, 0};
  for (int b = 0; b < g.dim; ++b) {
    if (b == a) { i[b] = l; continue; }
    i[b] = t % g.M[b];
    t /= g.M[b];
  }
  return i[0] + (long long)g.M[0] * (i[1] + (long long)g.M[1] * i[2]);
}
// own range [lo, hi) of subdomain k on axis a, in local indices (exterior sides not cut)
__host__ __device__ inline void own_range(const Geom &g, const int k[3], int a, int &lo, int &hi) {
  lo = (k[a] == 0) ? 0 : g.E;
  hi = (k[a] == g.parts[a] - 1) ? g.M[a] : g.E + g.m[a];
}

// ------------------------------------------------------------------------------------------
// the FP64 / FP32 trace map (trace plan): per factor [output side d][row tile of 64][input
// k = 0..T)[64 rows], rows past 2 Lt_d zero, so the rows of one tile for a run of consecutive
// inputs are one contiguous slice
// ------------------------------------------------------------------------------------------
constexpr int kTraceRows = 64;

__host__ __device__ inline int trace_tiles(const Geom &g, int d) {
  return (2 * g.Lt[d] + kTraceRows - 1) / kTraceRows;
}
__host__ __device__ inline int trace_max_tiles(const Geom &g) {
  int m = 0;
  for (int d = 0; d < g.nsides; ++d) m = trace_tiles(g, d) > m ? trace_tiles(g, d) : m;
  return m;
}
// element offset of (factor f, side d, tile tl, input k, row r) in the tiled trace map
__host__ __device__ inline long long gmap_index(const Geom &g, int f, int d, int tl, long long k,
                                                int r) {
  const long long per_tile = (long long)g.T * kTraceRows;
  const long long per_side = per_tile * trace_max_tiles(g);
  const long long per_fac = per_side * g.nsides;
  return f * per_fac + d * per_side + tl * per_tile + k * kTraceRows + r;
}

// Level completion counters of the cooperative trace launches: eight words per dataflow level
// (arrivals spread over them by CTA index), zeroed before every launch
constexpr int kStepCounters = 8;

__device__ inline unsigned ld_acquire_gpu(const unsigned *p) {
  unsigned v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

// ------------------------------------------------------------------------------------------
// work descriptors
// ------------------------------------------------------------------------------------------
struct Col { int sub; int rhs; int slot; int pad; };     // one (subdomain, RHS) local problem
struct Panel { int col0; int ncol; int factor; int pad; }; // columns sharing one factor

// device-side tables built at setup
struct Tables {
  const double2 *coef64;   // [T/2]: per side d, Lt_d commutator couplings c_d(t) at toff_d / 2
  const float2 *coef32;
  const double2 *an_glob64[3];  // alpha at global nodes per axis
  const double2 *iah_glob64[3]; // 1 / alpha at global half points per axis (G+1 entries;
                                // entry q lies between nodes q-1 and q)
  const double *k2_glob;        // kappa^2 on the global extended grid
  double inv_h2;                // 1 / h^2
  const double2 *c0;            // global stencil: centre coefficient per node
  const double2 *cp[3];         // global stencil: coupling of node p to p + e_a (0 on the edge)
};

// Raise a kernel's dynamic shared-memory limit to the largest value a launch may ask for (227 KB
// minus its static shared memory), once per device (the attribute persists on that device).
template <typename F>
inline cudaError_t smem_limit_once(F *kernel, bool (&done)[64]) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev >= 0 && dev < 64 && done[dev]) return cudaSuccess;
  cudaFuncAttributes fa;
  e = cudaFuncGetAttributes(&fa, kernel);
  if (e != cudaSuccess) return e;
  e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           227 * 1024 - (int)fa.sharedSizeBytes);
  if (e == cudaSuccess && dev >= 0 && dev < 64) done[dev] = true;
  return e;
}

// ------------------------------------------------------------------------------------------
// launch wrappers (each returns the CUDA error of the launch)
// ------------------------------------------------------------------------------------------
cudaError_t launch_factor(cudaStream_t st, int nfac, int Mb, int Ml, long long St, int M0,
                          const double2 *dg,
                          const double2 *offx, const double2 *offy, const double2 *cpl,
                          double2 *sinv64, float2 *sinv32, int *status);

cudaError_t launch_factor_twisted(cudaStream_t st, int nfac, int Mb, int Ml, long long St, int M0,
                                  int m, const double2 *dg, const double2 *offx,
                                  const double2 *offy, const double2 *cpl,
                                  const double2 *sinv64, double2 *tw64, int *status);
cudaError_t launch_factor_big(cudaStream_t st, int f, int Mb, int Ml, long long St, int M0,
                              const double2 *dg, const double2 *offx, const double2 *offy,
                              const double2 *cpl, double2 *S, double2 *colk, int *piv,
                              double2 *sinv64, float2 *sinv32, int *status,
                              long long *launches);

template <typename R>
cudaError_t launch_assemble(cudaStream_t st, const Geom &g, const Tables &tb, int ncols,
                            const Col *cols, typename Cx<R>::T *work, const double2 *b,
                            const double2 *unused, int with_source,
                            const typename Cx<R>::T *traces, long long trace_rhs_stride,
                            long long trace_sub_stride, int nslots, long long slot_stride,
                            int *nzflag = nullptr, int *badrhs = nullptr);

// zero-work skipping: pack the columns with a nonzero right-hand side (nz[slot]) of each
// group (int4: column range [x, y), panel range [z, w), one factor) into dcols / dpans (same
// index space as cols / panels; surplus panels get ncol = 0); stats[0] += live columns,
// stats[1] += columns
cudaError_t launch_compact_panels(cudaStream_t st, int ngroups, const int4 *groups,
                                  const Panel *pans, const Col *cols, const int *nz, Col *dcols,
                                  Panel *dpans, int pc, unsigned long long *stats);

template <typename R>
cudaError_t launch_subst(cudaStream_t st, const Geom &g, int npanels, const Panel *panels,
                         const Col *cols, const typename Cx<R>::T *sinv,
                         const typename Cx<R>::T *cpl, typename Cx<R>::T *work, int pc);

cudaError_t launch_subst_stream(cudaStream_t st, const Geom &g, int npanels, const Panel *panels,
                                const Col *cols, const float2 *sinv, const float2 *cpl,
                                float2 *work, int pc, int *err);
bool subst_stream_ok(const Geom &g, int pc);

// tensor-core substitutions (k_subst_tc.cu); kind 0 = TF32 pieces, 1 = BF16 pieces
// stage-parallel tensor-core substitutions for blocks wider than 128 nodes (k_subst_big.cu)
long long big_tiles_bytes(const Geom &g, int kind, int nfac);
cudaError_t launch_split_big(cudaStream_t st, const Geom &g, int kind, int nfac,
                             const double2 *sinv64, unsigned char *tiles);
size_t big_scratch_bytes(const Geom &g, int kind, int pc, int npanels, size_t *acc_bytes);
cudaError_t launch_subst_big(cudaStream_t st, const Geom &g, int kind, int npanels,
                             const Panel *panels, const Col *cols, const unsigned char *tiles,
                             const float2 *cpl, float2 *work, int pc, int ksplit, float2 *acc,
                             unsigned char *B, int *err, long long *launches);

// m > 0: two-sided chain split at block m, one 2-CTA cluster per np panels; m = 0: one-sided
// nz (optional): per work slot, nonzero if the column's right-hand side has a nonzero entry;
// panels whose columns are all zero are dropped (their solution is the zero already in work)
// np: panels per CTA (or CTA pair), 1, or 2 for pc <= 16 (one panel's epilogue under the
// other's MMAs)
cudaError_t launch_subst_tc(cudaStream_t st, const Geom &g, int kind, int npanels,
                            const Panel *panels, const Col *cols, const unsigned char *tiles,
                            const float2 *cpl, float2 *work, int pc, int *err, int m,
                            const int *nz = nullptr, int np = 1);
bool subst_tc_ok(const Geom &g, int kind, int pc, bool twisted, int np = 1);
int tc_middle_block(const Geom &g);   // m of the two-sided chain (0: too few blocks)
long long tc_tiles_bytes(const Geom &g, int kind, int nfac);
// tiles j < m from sinv64, j >= m from tw64 (m = 0 or tw64 null: all from sinv64)
cudaError_t launch_split_tc(cudaStream_t st, const Geom &g, int kind, int nfac,
                            const double2 *sinv64, const double2 *tw64, int m,
                            unsigned char *tiles);

// tensor-core trace solves (k_trace_tc.cu): split-map shape, its set-up and the cooperative
// launch over the dataflow levels (units: int4 headers, ucols: RHS * nsub + subdomain words)
struct TtShape {
  int kind, EK, KE;      // piece type, elements per 16 bytes, elements per K-step
  int RT;                // 128-row tiles of the stacked output rows
  int KP;                // stacked inputs, each side padded to a multiple of 16
  int kpo[6], kpn[6];    // offset / padded count of side d's inputs
  long long rt_bytes, fac_bytes;
  size_t smem;
};
// dense MMA rate (M = 128, N = 256) of piece type `kind` on every SM: flops and time of `iters`
// MMAs per SM (k_rate.cu)
cudaError_t measure_mma_rate(int kind, int iters, int *err, double *flops, float *ms);
bool tt_shape(const Geom &g, int kind, TtShape *s);
long long tt_tiles_bytes(const Geom &g, int kind, int nfac);
cudaError_t launch_split_trace(cudaStream_t st, const Geom &g, int kind, int nfac,
                               const double2 *gmap64, unsigned char *tiles);
bool build_tt_streams(const Geom &g, int kind, int G, const std::vector<int4> &units,
                      const std::vector<int> &lev_off, std::vector<int> &uoff,
                      std::vector<int2> &cunits, std::vector<int> &coff,
                      std::vector<int4> &chunks);
// G must be the CTA count the streams were built for (the device's SM count); nunits = units in
// all streams
cudaError_t launch_trace_tc(cudaStream_t st, const Geom &g, int kind, const int4 *units,
                            const int *ucols, const int *uoff, const int2 *cunits,
                            const int *coff, const int4 *chunks, int nunits, int G,
                            const unsigned char *tiles, const int *route, float2 *gtr,
                            const float2 *rawf, int nrhs, unsigned *ready, const unsigned *need,
                            int nslots, int *err, unsigned wait_limit);

template <typename R>
cudaError_t launch_extract(cudaStream_t st, const Geom &g, int ncols, const Col *cols,
                           const typename Cx<R>::T *work, double2 *u, int own_mode,
                           typename Cx<R>::T *raw_out, typename Cx<R>::T *g_traces,
                           const int *route, int l, int nrhs);

// a trace-step panel with its columns' (subdomain, RHS) inline (one load level in the kernel)
struct TracePanel {
  int factor, ncol;
  int sub[8], rhs[8];
};

size_t trace_counter_bytes(int nlevels);  // level counters of one launch (gbar)
size_t trace_smem_bytes(size_t elem, int nlevels);

// Work items of the cooperative trace launch (80 bytes each):
//   h.x = factor | (columns << 24), h.y = sweep l | (target slot << 16),
//   h.z = first input | (inputs << 16), h.w = output side | (row tile << 8) | (raw << 16)
//   col[c] = (RHS * nsub + subdomain of column c, RHS * nsub + its neighbour across the output
//            side or -1), (-1, -1) past the last column
// (raw: add the raw own-source lines).  trace_items_for appends the items of the sweep-l trace
// solves of panels [p0, p1).
struct TraceItem {
  int4 h;
  int2 col[8];
};
void trace_items_for(const Geom &g, const TracePanel *tp, int p0, int p1, int l, const int *route,
                     int in_mask, std::vector<TraceItem> &out);

// every trace solve of one DDM application in one cooperative launch: level v's items are
// records lev_off[v] .. lev_off[v + 1] - 1 of hdr (headers) and cols (8 column pairs each);
// gbar: the level counters, zeroed by the launch
template <typename R>
cudaError_t launch_trace_sweeps(cudaStream_t st, const Geom &g, const int4 *hdr, const int2 *cols,
                                int nitems, const int *lev_off, int nlevels,
                                const typename Cx<R>::T *gmap, typename Cx<R>::T *g_traces,
                                const typename Cx<R>::T *rawf, int nrhs, unsigned *gbar, int *err,
                                int ctas_per_sm, unsigned wait_limit);

template <typename R>
cudaError_t launch_unit_traces(cudaStream_t st, const Geom &g, const Tables &tb, int k0, int nk,
                               typename Cx<R>::T *work);

template <typename R>
cudaError_t launch_raw_lines(cudaStream_t st, const Geom &g, int nk, const typename Cx<R>::T *work,
                             typename Cx<R>::T *gmap, int f, int k0);

cudaError_t launch_gmap_backtrace(cudaStream_t st, const Geom &g, double2 *gmap, int f);
long long gmap_elems(const Geom &g, int nfac);
cudaError_t launch_convert_c64_c32(cudaStream_t st, const double2 *in, float2 *out, long long n);
template <typename R>
cudaError_t launch_copy_local(cudaStream_t st, long long n, const double2 *in,
                              typename Cx<R>::T *out, int to_work);
template <typename R>
cudaError_t launch_copy_local_back(cudaStream_t st, long long n, const typename Cx<R>::T *in,
                                   double2 *out);

// Krylov / operator kernels (FP64)
// Au = A u (divided by J if divide_by_J), minus sub when sub is not null
// Batched FP64 kernels: entry r of a vector family starts at base + r * stride, or at
// base + off[r] when an offset table (device memory) is given (non-contiguous server slots).
cudaError_t launch_apply_A(cudaStream_t st, const Geom &g, const Tables &tb, int nrhs,
                           const double2 *u, double2 *Au, int divide_by_J,
                           const double2 *sub = nullptr, const long long *uoff = nullptr,
                           const long long *aoff = nullptr);
cudaError_t launch_scale_J(cudaStream_t st, const Geom &g, const Tables &tb, int nrhs,
                           const double2 *f, double2 *b);
cudaError_t launch_dots(cudaStream_t st, long long N, int nrhs, int nv, const double2 *V,
                        long long v_stride_vec, long long v_stride_rhs, const double2 *w,
                        long long w_stride_rhs, double2 *partial, double2 *out, int nblk,
                        const long long *voff = nullptr, const long long *woff = nullptr);
// w = (overwrite ? 0 : w) + sign * sum_i V_i coef_i (x cscale_i if given) per RHS; with nrm2, also
// nrm2[rhs] = ||w[rhs]||^2 of the result in the same pass (nblk blocks per RHS, partial sized
// nrhs * nblk)
cudaError_t launch_combination(cudaStream_t st, long long N, int nrhs, int nv, const double2 *V,
                               long long vsv, long long vsr, const double2 *coef, int cstride,
                               double sign, double2 *w, long long wsr, bool overwrite,
                               double2 *partial, double2 *nrm2, int nblk,
                               const double *cscale = nullptr, const long long *voff = nullptr,
                               const long long *woff = nullptr);
cudaError_t launch_scale_by_norm(cudaStream_t st, long long N, int nrhs, const double2 *in,
                                const double2 *nrm2, double2 *out, const long long *off = nullptr);
int dots_chunk();
int dots_blocks(long long N, int nrhs);   // blocks per RHS of the dot / norm kernels

}  // namespace dds
