// Sweep kernels: right-hand-side assembly (own source + trace potentials), block-tridiagonal
// forward/back substitution, trace extraction with the back-trace correction and routing,
// own-node accumulation, and the trace-operator step.
//
// Trace potential (Section 2.3, discretised as a subdomain solve with a particular source):
// for a trace (a, b) on side d, a on the outer line and b on the inner line of the receiver,
//   rhs[outer_d] += c_d * b,   rhs[inner_d] -= c_d * a,
// c_d = prod_{tangential axes} alpha / h^2 (the coupling of the two lines; alpha = 1 on the
// interface), which is the commutator [A_R, chi_H] applied to the trace.
#include "async_copy.cuh"
#include "dds_internal.cuh"

namespace dds {

// ------------------------------------------------------------------------------------------
// K1: assemble local right-hand sides
// ------------------------------------------------------------------------------------------
template <typename R>
__global__ void k_assemble(Geom g, Tables tb, const Col *__restrict__ cols,
                           typename Cx<R>::T *__restrict__ work, const double2 *__restrict__ b,
                           int with_source, const typename Cx<R>::T *__restrict__ traces,
                           long long trs_rhs, long long trs_sub, int nslots,
                           long long slot_stride, int *__restrict__ nzflag) {
  using C = typename Cx<R>::T;
  const Col c = cols[blockIdx.x];
  bool nz = false;   // any nonzero entry written (the local solve of a zero source is zero)
  C *x = work + (long long)c.slot * g.Nloc;
  for (long long i = threadIdx.x; i < g.Nloc; i += blockDim.x) x[i] = czero<C>();
  __syncthreads();
  int k[3];
  sub_index(g, c.sub, k);
  if (with_source) {
    int lo[3] = {0, 0, 0}, hi[3] = {1, 1, 1};
    for (int a = 0; a < g.dim; ++a) own_range(g, k, a, lo[a], hi[a]);
    const int w0 = hi[0] - lo[0], w1 = hi[1] - lo[1], w2 = hi[2] - lo[2];
    const long long cnt = (long long)w0 * w1 * w2;
    const double2 *bb = b + (long long)c.rhs * g.Nglob;
    for (long long idx = threadIdx.x; idx < cnt; idx += blockDim.x) {
      int i0 = lo[0] + (int)(idx % w0);
      int i1 = lo[1] + (int)((idx / w0) % w1);
      int i2 = lo[2] + (int)(idx / ((long long)w0 * w1));
      long long loc = i0 + (long long)g.M[0] * (i1 + (long long)g.M[1] * i2);
      long long p0 = (long long)k[0] * g.m[0] + i0;
      long long p1 = (long long)k[1] * g.m[1] + i1;
      long long p2 = g.dim == 3 ? (long long)k[2] * g.m[2] + i2 : 0;
      long long glob = p0 + (long long)g.G[0] * (p1 + (long long)g.G[1] * p2);
      const C v = to_c(bb[glob], C());
      nz = nz || v.x != 0 || v.y != 0;
      x[loc] = v;
    }
  }
  const C *tr = traces ? traces + (long long)c.rhs * trs_rhs + (long long)c.sub * trs_sub : nullptr;
  for (int d = 0; tr != nullptr && d < g.nsides; ++d) {
    __syncthreads();  // lines of different sides may share nodes
    if (sub_neighbour(g, c.sub, d) < 0) continue;
    const int a = d >> 1, Lt = g.Lt[d], off = g.toff[d];
    const int li = inner_line(g, d), lo = outer_line(g, d);
    for (int t = threadIdx.x; t < Lt; t += blockDim.x) {
      C cd;
      if constexpr (sizeof(R) == 4) cd = tb.coef32[off / 2 + t];
      else cd = tb.coef64[off / 2 + t];
      C av = tr[off + t], bv = tr[off + Lt + t];
      for (int q = 1; q < nslots; ++q) {   // sum of the traces of several sweeps
        av = cadd(av, tr[q * slot_stride + off + t]);
        bv = cadd(bv, tr[q * slot_stride + off + Lt + t]);
      }
      const long long no = line_node(g, a, lo, t), ni = line_node(g, a, li, t);
      x[no] = cadd(x[no], cmul(cd, bv));
      x[ni] = csub(x[ni], cmul(cd, av));
      nz = nz || av.x != 0 || av.y != 0 || bv.x != 0 || bv.y != 0;
    }
  }
  if (nzflag != nullptr) {
    const int any = __syncthreads_or(nz);
    if (threadIdx.x == 0) nzflag[c.slot] = any;
  }
}

// ------------------------------------------------------------------------------------------
// K2 + K3: block-tridiagonal substitutions for a panel of columns sharing one factor
//   forward  y_0 = S_0^{-1} b_0,  y_j = S_j^{-1} (b_j - C_{j-1} y_{j-1})
//   backward x_{Ml-1} = y_{Ml-1}, x_j = y_j - S_j^{-1} (C_j x_{j+1})
// C_j = diag(cpl_j) couples block j and j+1 (A is complex symmetric).
// ------------------------------------------------------------------------------------------
template <typename R, int PC>
__global__ void __launch_bounds__(128) k_subst(Geom g, const Panel *__restrict__ panels,
                                               const Col *__restrict__ cols,
                                               const typename Cx<R>::T *__restrict__ sinv,
                                               const typename Cx<R>::T *__restrict__ cpl,
                                               typename Cx<R>::T *__restrict__ work) {
  using C = typename Cx<R>::T;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C *v = reinterpret_cast<C *>(smem_raw);  // [Mb][PC]
  const Panel p = panels[blockIdx.x];
  const int Mb = g.Mb, Ml = g.Ml;
  const C *Sf = sinv + (long long)p.factor * Ml * g.St;
  const C *cf = cpl + (long long)p.factor * Ml * (long long)Mb;
  C *xs[PC];
#pragma unroll
  for (int c = 0; c < PC; ++c)
    xs[c] = c < p.ncol ? work + (long long)cols[p.col0 + c].slot * g.Nloc : nullptr;

  for (int pass = 0; pass < 2; ++pass) {
    const int jbeg = pass == 0 ? 0 : Ml - 2;
    const int jend = pass == 0 ? Ml : -1;
    const int jstep = pass == 0 ? 1 : -1;
    for (int j = jbeg; j != jend; j += jstep) {
      for (int idx = threadIdx.x; idx < Mb * PC; idx += blockDim.x) {
        const int r = idx / PC, c = idx % PC;
        C val = czero<C>();
        if (c < p.ncol) {
          C *x = work + (long long)cols[p.col0 + c].slot * g.Nloc;
          if (pass == 0) {
            val = x[(long long)j * Mb + r];
            if (j > 0) val = csub(val, cmul(cf[(long long)(j - 1) * Mb + r], x[(long long)(j - 1) * Mb + r]));
          } else {
            val = cmul(cf[(long long)j * Mb + r], x[(long long)(j + 1) * Mb + r]);
          }
        }
        v[r * PC + c] = val;
      }
      __syncthreads();
      const C *Sj = Sf + (long long)j * g.St;
      for (int r = threadIdx.x; r < Mb; r += blockDim.x) {
        C acc[PC];
#pragma unroll
        for (int c = 0; c < PC; ++c) acc[c] = czero<C>();
#pragma unroll 4
        for (int s = 0; s < Mb; ++s) {
          const C a = Sj[(long long)s * Mb + r];
#pragma unroll
          for (int c = 0; c < PC; ++c) cfma(acc[c], a, v[s * PC + c]);
        }
#pragma unroll
        for (int c = 0; c < PC; ++c) {
          if (c < p.ncol) {
            C *dst = xs[c] + (long long)j * Mb + r;
            *dst = pass == 0 ? acc[c] : csub(*dst, acc[c]);
          }
        }
      }
      __syncthreads();
    }
  }
}

// ------------------------------------------------------------------------------------------
// K4 + K5: own accumulation, raw trace lines, routed outgoing traces
//   outgoing trace on side d: a = x[inner_d] - b_in_d, b = x[outer_d], added to the slot
//   g[route[l][d]][rhs][neighbour][opposite side]
// ------------------------------------------------------------------------------------------
template <typename R>
__global__ void k_extract(Geom g, const Col *__restrict__ cols,
                          const typename Cx<R>::T *__restrict__ work, double2 *__restrict__ u,
                          int own_mode, typename Cx<R>::T *__restrict__ raw_out,
                          typename Cx<R>::T *__restrict__ gtr, const int *__restrict__ route,
                          int l, int nrhs) {
  using C = typename Cx<R>::T;
  const Col c = cols[blockIdx.x];
  const C *x = work + (long long)c.slot * g.Nloc;
  int k[3];
  sub_index(g, c.sub, k);
  if (own_mode) {
    int lo[3] = {0, 0, 0}, hi[3] = {1, 1, 1};
    for (int a = 0; a < g.dim; ++a) own_range(g, k, a, lo[a], hi[a]);
    const int w0 = hi[0] - lo[0], w1 = hi[1] - lo[1], w2 = hi[2] - lo[2];
    const long long cnt = (long long)w0 * w1 * w2;
    double2 *uu = u + (long long)c.rhs * g.Nglob;
    for (long long idx = threadIdx.x; idx < cnt; idx += blockDim.x) {
      int i0 = lo[0] + (int)(idx % w0);
      int i1 = lo[1] + (int)((idx / w0) % w1);
      int i2 = lo[2] + (int)(idx / ((long long)w0 * w1));
      long long loc = i0 + (long long)g.M[0] * (i1 + (long long)g.M[1] * i2);
      long long p0 = (long long)k[0] * g.m[0] + i0;
      long long p1 = (long long)k[1] * g.m[1] + i1;
      long long p2 = g.dim == 3 ? (long long)k[2] * g.m[2] + i2 : 0;
      long long glob = p0 + (long long)g.G[0] * (p1 + (long long)g.G[1] * p2);
      const double2 xv = to_c64(x[loc]);
      uu[glob] = own_mode == 1 ? cadd(uu[glob], xv) : xv;
    }
  }
  if (raw_out != nullptr) {
    C *raw = raw_out + ((long long)c.rhs * g.nsub + c.sub) * g.T;
    for (int d = 0; d < g.nsides; ++d) {
      const int a = d >> 1, Lt = g.Lt[d], off = g.toff[d];
      const int li = inner_line(g, d), lo = outer_line(g, d);
      for (int t = threadIdx.x; t < Lt; t += blockDim.x) {
        raw[off + t] = x[line_node(g, a, li, t)];
        raw[off + Lt + t] = x[line_node(g, a, lo, t)];
      }
    }
  }
  if (gtr != nullptr) {
    const long long slot_stride = (long long)nrhs * g.nsub * g.T;
    for (int d = 0; d < g.nsides; ++d) {
      const int nb = sub_neighbour(g, c.sub, d);
      const int lp = route[l * 6 + d];
      if (nb < 0 || lp < 0) continue;
      const int a = d >> 1, Lt = g.Lt[d];
      const int li = inner_line(g, d), lo = outer_line(g, d);
      const C *bin = gtr + l * slot_stride + ((long long)c.rhs * g.nsub + c.sub) * g.T +
                     g.toff[d] + Lt;
      C *dst = gtr + lp * slot_stride + ((long long)c.rhs * g.nsub + nb) * g.T + g.toff[d ^ 1];
      for (int t = threadIdx.x; t < Lt; t += blockDim.x) {
        const C av = csub(x[line_node(g, a, li, t)], bin[t]);
        const C bv = x[line_node(g, a, lo, t)];
        dst[t] = cadd(dst[t], av);
        dst[Lt + t] = cadd(dst[Lt + t], bv);
      }
    }
  }
}

// ------------------------------------------------------------------------------------------
// Trace-operator step: for every (sub, rhs) column of the step,
//   out = Gmap_F * in (+ raw own-source lines in sweep 1),   in = incoming traces of the sweep,
// routed like k_extract.  Gmap already contains the back-trace correction; acc += in for the
// final own-node solve.  Only input sides that can receive a trace in this sweep (in_mask) and
// output sides with a route (out_mask) are touched -- the other terms are exactly zero or
// unused.
// Gmap layout per factor: [output side d][row tile of 64][input k = 0..T)[64 rows], rows past
// 2 Lt_d zero.  A CTA (256 threads) owns one row tile and one panel of PC columns; the tile's
// rows for the active inputs stream through a two-slot shared-memory ring in chunks of KC
// inputs (bulk copies on mbarriers).  Thread (r = t & 63, h = t >> 6) owns row r and columns
// h*PC/4 .. h*PC/4 + PC/4.
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
long long gmap_elems(const Geom &g, int nfac) { return gmap_index(g, nfac, 0, 0, 0, 0); }

// The active inputs of a sweep (the sides in in_mask) are cut into segments of at most
// kTraceSeg consecutive inputs of one side.  A CTA (128 threads) owns one 64-row tile of one
// output side, one panel of PC = 8 columns and one input segment: its map slice
// (segment x 64 rows, contiguous in the tiled layout) arrives by one bulk copy while the threads
// gather the panel's inputs, then thread (rp = t & 31, cq = t >> 5) accumulates rows 2 rp,
// 2 rp + 1 x columns 2 cq, 2 cq + 1 from shared memory.  Segments of one output add into the
// destination slot with atomics (the slot accumulates with += in any case).  The CTA has 256
// threads: two halves share the segment and meet in shared memory.
constexpr int kTraceSeg = 104;

__host__ __device__ inline int trace_nseg(const Geom &g, int in_mask) {
  int n = 0;
  for (int d = 0; d < g.nsides; ++d)
    if ((in_mask >> d) & 1) n += (2 * g.Lt[d] + kTraceSeg - 1) / kTraceSeg;
  return n;
}

template <typename C> __device__ inline void atomic_cadd(C *dst, C v);
template <> __device__ inline void atomic_cadd<float2>(float2 *dst, float2 v) {
  atomicAdd(&dst->x, v.x);
  atomicAdd(&dst->y, v.y);
}
template <> __device__ inline void atomic_cadd<double2>(double2 *dst, double2 v) {
  atomicAdd(&dst->x, v.x);
  atomicAdd(&dst->y, v.y);
}

// Step completion counters of the cooperative launch: after its items of step s a CTA adds 1
// to cnt[8 s + (blockIdx % 8)] (eight words, so arrivals do not all hit one address); a CTA
// with items in step s + 1 first waits until the eight words of step s sum to gridDim.x.  CTAs
// without items never wait.  The counters are zeroed before every launch.  The wait is bounded:
// on a timeout the CTA records code 4 and goes on (results wrong, launch ends, the host reports
// DDS_ETIMEOUT).
constexpr int kStepCounters = 8;

__device__ inline unsigned ld_acquire_gpu(const unsigned *p) {
  unsigned v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ inline void step_arrive(unsigned *cnt, int s) {
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    atomicAdd(cnt + s * kStepCounters + (blockIdx.x % kStepCounters), 1u);
  }
}
__device__ inline void step_wait(const unsigned *cnt, int s, int *err) {
  if (threadIdx.x < 32) {
    // warp 0 polls the eight counters; the full-warp sum keeps every lane's exit decision
    // identical.  Once any wait has given up (err set) no later wait spins.
    const int lane = threadIdx.x;
    uint32_t spins = 0;
    for (;;) {
      unsigned v = lane < kStepCounters ? ld_acquire_gpu(cnt + s * kStepCounters + lane) : 0u;
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
      if (v >= gridDim.x) break;
      int stop = 0;
      if (lane == 0) stop = (++spins > (1u << 20)) || *reinterpret_cast<volatile int *>(err) != 0;
      stop = __shfl_sync(0xffffffffu, stop, 0);
      if (stop) {
        if (lane == 0) atomicExch(err, 4);
        break;
      }
      __nanosleep(64);
    }
  }
  __syncthreads();
}

// per-item descriptors staged in shared memory before the item's inputs are ready
struct TraceItemSmem {
  long long cbase[8];   // input trace base of each column (-1: no column)
  int sub[8], rhs[8];
  int ncol;
};

// Work item of a trace step: output side dout, 64-row tile `tile`, panel p, input segment
// [k0, k0 + n).  The map slice is in Gs (bulk copy on `bar`, issued with the descriptors by
// trace_prep); inputs come from L2 (ld.global.cg: other CTAs of this launch wrote them).
template <typename R>
__device__ void trace_item(const Geom &g, typename Cx<R>::T *__restrict__ gtr,
                           const typename Cx<R>::T *__restrict__ rawf, const int *__restrict__ route,
                           int l, int nrhs, int dout, int tile, int k0, int n, bool first_seg,
                           typename Cx<R>::T *Gs, typename Cx<R>::T *vin, uint64_t *bar,
                           uint32_t phase, const TraceItemSmem &it, int *err) {
  using C = typename Cx<R>::T;
  constexpr int PC = 8;
  constexpr int kPer = (PC * kTraceSeg + 255) / 256;
  const int T = g.T;
  const long long slot_stride = (long long)nrhs * g.nsub * T;
  {
    C v[kPer];
#pragma unroll
    for (int u = 0; u < kPer; ++u) {
      const int idx = threadIdx.x + u * 256;
      v[u] = czero<C>();
      if (idx < PC * kTraceSeg) {
        const int c = idx / kTraceSeg, kk = idx - c * kTraceSeg;
        const long long b = it.cbase[c];
        if (b >= 0 && kk < n) {
          const C *src = gtr + b + k0 + kk;
          if constexpr (sizeof(R) == 4) {
            const float2 t = __ldcg(reinterpret_cast<const float2 *>(src));
            v[u].x = t.x; v[u].y = t.y;
          } else {
            const double2 t = __ldcg(reinterpret_cast<const double2 *>(src));
            v[u].x = t.x; v[u].y = t.y;
          }
        }
      }
    }
#pragma unroll
    for (int u = 0; u < kPer; ++u) {
      const int idx = threadIdx.x + u * 256;
      if (idx < PC * kTraceSeg) vin[idx] = v[u];
    }
  }
  const bool ok = mbar_wait(bar, phase);
  if (__syncthreads_or(!ok)) {
    if (threadIdx.x == 0) {
      atomicExch(err, 3);
      mbar_wait(bar, phase);
    }
    __syncthreads();
    return;
  }
  // two halves of the segment, 128 threads each; thread (rp, cq) of a half: rows 2rp, 2rp+1,
  // columns 2cq, 2cq+1.  Inputs are consumed four at a time with the next four prefetched.
  const int half = threadIdx.x >> 7, lt = threadIdx.x & 127;
  const int rp = lt & 31, cq = lt >> 5;
  const int nh = ((n + 7) / 8) * 4;                 // inputs of half 0 (a multiple of 4)
  const int i0 = half == 0 ? 0 : nh, i1 = half == 0 ? min(n, nh) : n;
  const C *A = Gs + 2 * rp;
  const C *v0 = vin + (2 * cq) * kTraceSeg;
  const C *v1 = v0 + kTraceSeg;
  C o00 = czero<C>(), o01 = czero<C>(), o10 = czero<C>(), o11 = czero<C>();
  auto step4 = [&](const C (&a)[4][2], const C (&b0)[4], const C (&b1)[4]) {
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      cfma(o00, a[u][0], b0[u]);
      cfma(o01, a[u][0], b1[u]);
      cfma(o10, a[u][1], b0[u]);
      cfma(o11, a[u][1], b1[u]);
    }
  };
  auto load4 = [&](int i, C (&a)[4][2], C (&b0)[4], C (&b1)[4]) {
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      a[u][0] = A[(i + u) * kTraceRows];
      a[u][1] = A[(i + u) * kTraceRows + 1];
      b0[u] = v0[i + u];
      b1[u] = v1[i + u];
    }
  };
  int i = i0;
  if (i + 4 <= i1) {
    C a[4][2], b0[4], b1[4];
    load4(i, a, b0, b1);
    for (; i + 8 <= i1; i += 4) {
      C an[4][2], bn0[4], bn1[4];
      load4(i + 4, an, bn0, bn1);
      step4(a, b0, b1);
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        a[u][0] = an[u][0];
        a[u][1] = an[u][1];
        b0[u] = bn0[u];
        b1[u] = bn1[u];
      }
    }
    step4(a, b0, b1);
    i += 4;
  }
  for (; i < i1; ++i) {
    const C a0 = A[i * kTraceRows], a1 = A[i * kTraceRows + 1];
    cfma(o00, a0, v0[i]);
    cfma(o01, a0, v1[i]);
    cfma(o10, a1, v0[i]);
    cfma(o11, a1, v1[i]);
  }
  // half 1 hands its partial sums to half 0 through the input buffer
  __syncthreads();
  C *red = vin + (long long)lt * 4;
  if (half == 1) {
    red[0] = o00;
    red[1] = o01;
    red[2] = o10;
    red[3] = o11;
  }
  __syncthreads();
  if (half == 0) {
    o00 = cadd(o00, red[0]);
    o01 = cadd(o01, red[1]);
    o10 = cadd(o10, red[2]);
    o11 = cadd(o11, red[3]);
    const int rows = 2 * g.Lt[dout];
    const int lp = route[l * 6 + dout];
    const int rr = tile * kTraceRows + 2 * rp;     // rows rr, rr + 1 (rows is even)
    if (rr < rows && lp >= 0) {
      const int grow = g.toff[dout] + rr;          // row in the full trace vector
      const C res[2][2] = {{o00, o10}, {o01, o11}}; // [column][row]
#pragma unroll
      for (int jj = 0; jj < 2; ++jj) {
        const int cg = 2 * cq + jj;
        if (cg >= it.ncol) continue;
        const int csub_ = it.sub[cg], crhs = it.rhs[cg];
        C v0r = res[jj][0], v1r = res[jj][1];
        if (rawf != nullptr && first_seg) {
          const C *rw = rawf + ((long long)crhs * g.nsub + csub_) * T + grow;
          v0r = cadd(v0r, rw[0]);
          v1r = cadd(v1r, rw[1]);
        }
        const int nb = sub_neighbour(g, csub_, dout);
        if (nb < 0) continue;
        C *dst = gtr + lp * slot_stride + ((long long)crhs * g.nsub + nb) * T + g.toff[dout ^ 1] + rr;
        if constexpr (sizeof(R) == 4) {
          // both rows in one 16-byte vector atomic (T, the side offsets and rr are even)
          red_add_f4(reinterpret_cast<float4 *>(dst), make_float4(v0r.x, v0r.y, v1r.x, v1r.y));
        } else {
          atomic_cadd(dst, v0r);
          atomic_cadd(dst + 1, v1r);
        }
      }
    }
  }
  __syncthreads();   // Gs, vin and the descriptors are reused by the next item
}

// item -> (output side, tile, panel, input segment) of step sd; false if the item is empty
__device__ inline bool trace_decode(const Geom &g, const TraceStep &sd, int tiles_per_side,
                                    int item, int &dout, int &tile, int &panel, int &k0, int &n,
                                    int &seg) {
  seg = item % sd.nseg;
  int rest = item / sd.nseg;
  const int xt = rest % (sd.nout * tiles_per_side);
  panel = rest / (sd.nout * tiles_per_side);
  int which = xt / tiles_per_side;
  tile = xt % tiles_per_side;
  dout = -1;
  for (int d = 0; d < g.nsides; ++d)
    if ((sd.out_mask >> d) & 1) {
      if (which == 0) { dout = d; break; }
      --which;
    }
  if (dout < 0 || tile >= trace_tiles(g, dout)) return false;
  int sgi = seg;
  n = 0;
  for (int d = 0; d < g.nsides; ++d) {
    if (!((sd.in_mask >> d) & 1)) continue;
    const int ns = (2 * g.Lt[d] + kTraceSeg - 1) / kTraceSeg;
    if (sgi < ns) {
      k0 = g.toff[d] + sgi * kTraceSeg;
      n = min(kTraceSeg, 2 * g.Lt[d] - sgi * kTraceSeg);
      break;
    }
    sgi -= ns;
  }
  return n > 0;
}

// Every trace solve of one DDM application in one cooperative launch.  The schedule is a list of
// dataflow levels: a trace solve (sweep l, subdomain X) sits one level below the deepest solve
// whose traces are routed into its slot l, so every level only reads slots that earlier levels
// completed.  The items of a level are dealt round-robin over the CTAs; a CTA with items in
// level v first waits until every CTA is done with level v - 1 (counters above).  The step
// table sits in shared memory; the descriptors and map slice of a CTA's first item of the next
// level depend on no trace and are staged before that wait.
constexpr int kMaxSmemSteps = 384;

template <typename R>
__global__ void __launch_bounds__(256) k_trace_sweeps(Geom g, const TraceStep *__restrict__ steps,
                                                      int nsteps,
                                                      const TracePanel *__restrict__ panels,
                                                      const typename Cx<R>::T *__restrict__ gmap,
                                                      typename Cx<R>::T *__restrict__ gtr,
                                                      const typename Cx<R>::T *__restrict__ rawf,
                                                      const int *__restrict__ route, int nrhs,
                                                      int tiles_per_side, unsigned *cnt,
                                                      int *__restrict__ err) {
  using C = typename Cx<R>::T;
  constexpr int PC = 8;
  extern __shared__ __align__(128) unsigned char smem_raw[];
  C *Gs = reinterpret_cast<C *>(smem_raw);                   // map slice [k][64]
  C *vin = Gs + kTraceSeg * kTraceRows;                      // inputs [col][k]
  uint64_t *bar = reinterpret_cast<uint64_t *>(vin + PC * kTraceSeg);
  TraceStep *st_s = reinterpret_cast<TraceStep *>(bar + 2);  // schedule (nsteps <= kMaxSmemSteps)
  __shared__ TraceItemSmem it;
  const bool smem_steps = nsteps <= kMaxSmemSteps;
  for (int i = threadIdx.x; smem_steps && i < nsteps; i += blockDim.x) st_s[i] = steps[i];
  if (threadIdx.x == 0) {
    mbar_init(bar, 1);
    mbar_init_fence();
  }
  __syncthreads();
  auto step_at = [&](int e) { return smem_steps ? st_s[e] : steps[e]; };
  const long long slot_stride = (long long)nrhs * g.nsub * g.T;
  const int G = (int)gridDim.x, b = (int)blockIdx.x;
  uint32_t phase = 0;
  // stage the descriptors and issue the map-slice copy (all threads call; ends with a barrier)
  auto prep = [&](const TraceStep &sd, int panel, int dout, int tile, int k0, int n) {
    const TracePanel *tp = panels + sd.pan_off + panel;
    if (threadIdx.x == 0) {
      const uint32_t bytes = (uint32_t)(n * kTraceRows * sizeof(C));
      fence_proxy_async();   // earlier generic reads of Gs before the async write
      mbar_arrive_expect_tx(bar, bytes);
      bulk_g2s(Gs, gmap + gmap_index(g, tp->factor, dout, tile, k0, 0), bytes, bar);
      it.ncol = tp->ncol;
    }
    if (threadIdx.x < PC) {
      const int c = threadIdx.x;
      const int sub = tp->sub[c], rhs = tp->rhs[c];
      it.sub[c] = sub;
      it.rhs[c] = rhs;
      it.cbase[c] = c < tp->ncol ? sd.l * slot_stride + ((long long)rhs * g.nsub + sub) * g.T : -1;
    }
    __syncthreads();
  };
  // the entry and item of this CTA's first work in the level starting at entry e0 (or -1)
  auto first_in_level = [&](int e0, int &item) {
    const TraceStep s0 = step_at(e0);
    if (b >= s0.level_items) return -1;
    for (int e = e0; e < nsteps; ++e) {
      const TraceStep se = step_at(e);
      if (se.level != s0.level) break;
      if (b >= se.off && b < se.off + se.nitems) { item = b - se.off; return e; }
    }
    return -1;
  };
  int pre_e = -1, pre_item = -1;   // staged item (descriptors + map slice in flight)
  int level = -1;
  for (int e = 0; e < nsteps; ++e) {
    const TraceStep sd = step_at(e);
    if (sd.level != level) {
      if (level >= 0) {
        step_arrive(cnt, level);
        // stage this CTA's first item of the new level, then wait for the previous level
        int item = -1;
        const int ef = first_in_level(e, item);
        if (ef >= 0) {
          const TraceStep sf = step_at(ef);
          int dout, tile, panel, k0, n, seg;
          if (trace_decode(g, sf, tiles_per_side, item, dout, tile, panel, k0, n, seg)) {
            prep(sf, panel, dout, tile, k0, n);
            pre_e = ef;
            pre_item = item;
          }
        }
        if (b < sd.level_items) step_wait(cnt, level, err);
      }
      level = sd.level;
    }
    // this CTA's items of entry e: global level index off + item = b (mod G)
    int item = ((b - sd.off) % G + G) % G;
    for (; item < sd.nitems; item += G) {
      int dout, tile, panel, k0, n, seg;
      if (!trace_decode(g, sd, tiles_per_side, item, dout, tile, panel, k0, n, seg)) continue;
      if (!(e == pre_e && item == pre_item)) prep(sd, panel, dout, tile, k0, n);
      trace_item<R>(g, gtr, sd.l == 0 ? rawf : nullptr, route, sd.l, nrhs, dout, tile, k0, n,
                    seg == 0, Gs, vin, bar, phase, it, err);
      phase ^= 1u;
    }
  }
  // a staged item is always consumed by its level, so no copy is in flight here
}

// ------------------------------------------------------------------------------------------
// Trace-map construction helpers
// ------------------------------------------------------------------------------------------
// slot q holds the commutator source of the unit trace entry k0 + q
template <typename R>
__global__ void k_unit_traces(Geom g, Tables tb, int k0, int nk,
                              typename Cx<R>::T *__restrict__ work) {
  using C = typename Cx<R>::T;
  const int q = blockIdx.x;
  if (q >= nk) return;
  C *x = work + (long long)q * g.Nloc;
  for (long long i = threadIdx.x; i < g.Nloc; i += blockDim.x) x[i] = czero<C>();
  __syncthreads();
  if (threadIdx.x != 0) return;
  const int kk = k0 + q;
  int d = 0;
  while (d + 1 < g.nsides && kk >= g.toff[d + 1]) ++d;
  const int Lt = g.Lt[d], within = kk - g.toff[d];
  const int is_b = within >= Lt, t = is_b ? within - Lt : within;
  C cd;
  if constexpr (sizeof(R) == 4) cd = tb.coef32[g.toff[d] / 2 + t];
  else cd = tb.coef64[g.toff[d] / 2 + t];
  const int a = d >> 1;
  if (is_b) {
    x[line_node(g, a, outer_line(g, d), t)] = cd;
  } else {
    C z = czero<C>();
    x[line_node(g, a, inner_line(g, d), t)] = csub(z, cd);
  }
}

// column k0 + q of the trace map = raw trace lines of the solution in slot q (tiled layout)
template <typename R>
__global__ void k_raw_lines(Geom g, const typename Cx<R>::T *__restrict__ work,
                            typename Cx<R>::T *__restrict__ gmap, int f, int k0) {
  using C = typename Cx<R>::T;
  const int q = blockIdx.x;
  const long long kk = k0 + q;
  const C *x = work + (long long)q * g.Nloc;
  for (int d = 0; d < g.nsides; ++d) {
    const int a = d >> 1, Lt = g.Lt[d];
    const int li = inner_line(g, d), lo = outer_line(g, d);
    for (int ro = threadIdx.x; ro < trace_tiles(g, d) * kTraceRows; ro += blockDim.x) {
      C v = czero<C>();
      if (ro < Lt) v = x[line_node(g, a, li, ro)];
      else if (ro < 2 * Lt) v = x[line_node(g, a, lo, ro - Lt)];
      gmap[gmap_index(g, f, d, ro / kTraceRows, kk, ro % kTraceRows)] = v;
    }
  }
}

// back-trace correction folded into the map: a_out_d(t) -= b_in_d(t)
__global__ void k_gmap_backtrace(Geom g, double2 *gmap, int f) {
  for (int d = 0; d < g.nsides; ++d) {
    const int Lt = g.Lt[d], off = g.toff[d];
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < Lt; t += gridDim.x * blockDim.x) {
      const long long kk = off + Lt + t;   // b-line input of side d
      double2 *e = gmap + gmap_index(g, f, d, t / kTraceRows, kk, t % kTraceRows);
      e->x -= 1.0;
    }
  }
}

template <typename R>
__global__ void k_copy_local(long long n, const double2 *__restrict__ in,
                             typename Cx<R>::T *__restrict__ out) {
  using C = typename Cx<R>::T;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x)
    out[i] = to_c(in[i], C());
}
template <typename R>
__global__ void k_copy_local_back(long long n, const typename Cx<R>::T *__restrict__ in,
                                  double2 *__restrict__ out) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x)
    out[i] = to_c64(in[i]);
}

// ------------------------------------------------------------------------------------------
// launch wrappers
// ------------------------------------------------------------------------------------------
template <typename R>
cudaError_t launch_assemble(cudaStream_t st, const Geom &g, const Tables &tb, int ncols,
                            const Col *cols, typename Cx<R>::T *work, const double2 *b,
                            const double2 *, int with_source, const typename Cx<R>::T *traces,
                            long long trs_rhs, long long trs_sub, int nslots,
                            long long slot_stride, int *nzflag) {
  if (ncols <= 0) return cudaSuccess;
  k_assemble<R><<<ncols, 256, 0, st>>>(g, tb, cols, work, b, with_source, traces, trs_rhs,
                                       trs_sub, nslots, slot_stride, nzflag);
  return cudaGetLastError();
}

template <typename R, int PC>
static cudaError_t subst_pc(cudaStream_t st, const Geom &g, int npanels, const Panel *panels,
                            const Col *cols, const typename Cx<R>::T *sinv,
                            const typename Cx<R>::T *cpl, typename Cx<R>::T *work) {
  using C = typename Cx<R>::T;
  const size_t smem = (size_t)g.Mb * PC * sizeof(C);
  static bool done[64] = {false};
  cudaError_t e = smem_limit_once(k_subst<R, PC>, done);
  if (e != cudaSuccess) return e;
  k_subst<R, PC><<<npanels, 128, smem, st>>>(g, panels, cols, sinv, cpl, work);
  return cudaGetLastError();
}

template <typename R>
cudaError_t launch_subst(cudaStream_t st, const Geom &g, int npanels, const Panel *panels,
                         const Col *cols, const typename Cx<R>::T *sinv,
                         const typename Cx<R>::T *cpl, typename Cx<R>::T *work, int pc) {
  if (npanels <= 0) return cudaSuccess;
  switch (pc) {
    case 1: return subst_pc<R, 1>(st, g, npanels, panels, cols, sinv, cpl, work);
    case 2: return subst_pc<R, 2>(st, g, npanels, panels, cols, sinv, cpl, work);
    case 4: return subst_pc<R, 4>(st, g, npanels, panels, cols, sinv, cpl, work);
    case 8: return subst_pc<R, 8>(st, g, npanels, panels, cols, sinv, cpl, work);
    default: return cudaErrorInvalidValue;
  }
}

template <typename R>
cudaError_t launch_extract(cudaStream_t st, const Geom &g, int ncols, const Col *cols,
                           const typename Cx<R>::T *work, double2 *u, int own_mode,
                           typename Cx<R>::T *raw_out, typename Cx<R>::T *g_traces,
                           const int *route, int l, int nrhs) {
  if (ncols <= 0) return cudaSuccess;
  k_extract<R><<<ncols, 256, 0, st>>>(g, cols, work, u, own_mode, raw_out, g_traces, route, l,
                                      nrhs);
  return cudaGetLastError();
}

template <typename R>
cudaError_t launch_trace_sweeps(cudaStream_t st, const Geom &g, const TraceStep *steps, int nsteps,
                                int nlevels, const TracePanel *panels,
                                const typename Cx<R>::T *gmap, typename Cx<R>::T *gtr,
                                const typename Cx<R>::T *rawf, const int *route, int nrhs,
                                unsigned *gbar, int *err, int ctas_per_sm) {
  if (nsteps <= 0) return cudaSuccess;
  using C = typename Cx<R>::T;
  const size_t smem = trace_step_smem(g, 8, sizeof(C));
  static bool done[64] = {false};
  cudaError_t e = smem_limit_once(k_trace_sweeps<R>, done);
  if (e != cudaSuccess) return e;
  int dev = 0, nsm = 0, per_sm = 0;
  if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
  if ((e = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
  if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_trace_sweeps<R>, 256, smem)) !=
      cudaSuccess)
    return e;
  if (per_sm < 1) return cudaErrorInvalidConfiguration;
  cudaLaunchConfig_t cfg = {};
  e = cudaMemsetAsync(gbar, 0, trace_counter_bytes(nlevels), st);
  if (e != cudaSuccess) return e;
  cfg.gridDim = dim3((unsigned)(nsm * std::max(1, std::min(per_sm, ctas_per_sm))));
  cfg.blockDim = dim3(256);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeCooperative;
  attr[0].val.cooperative = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, k_trace_sweeps<R>, g, steps, nsteps, panels, gmap, gtr,
                            rawf, route, nrhs, trace_max_tiles(g), gbar, err);
}

size_t trace_counter_bytes(int nlevels) { return (size_t)nlevels * kStepCounters * sizeof(unsigned); }

int trace_step_items(const Geom &g, int npanels, int in_mask, int out_mask, int *nout, int *nseg) {
  int no = 0;
  for (int d = 0; d < g.nsides; ++d) no += (out_mask >> d) & 1;
  const int ns = trace_nseg(g, in_mask);
  if (nout) *nout = no;
  if (nseg) *nseg = ns;
  return no * trace_max_tiles(g) * npanels * ns;
}

size_t trace_step_smem(const Geom &, int pc, size_t elem) {
  return ((size_t)kTraceSeg * kTraceRows + (size_t)pc * kTraceSeg) * elem + 16 +
         (size_t)kMaxSmemSteps * sizeof(TraceStep);
}

template <typename R>
cudaError_t launch_unit_traces(cudaStream_t st, const Geom &g, const Tables &tb, int k0, int nk,
                               typename Cx<R>::T *work) {
  if (nk <= 0) return cudaSuccess;
  k_unit_traces<R><<<nk, 256, 0, st>>>(g, tb, k0, nk, work);
  return cudaGetLastError();
}

template <typename R>
cudaError_t launch_raw_lines(cudaStream_t st, const Geom &g, int nk,
                             const typename Cx<R>::T *work, typename Cx<R>::T *gmap, int f,
                             int k0) {
  if (nk <= 0) return cudaSuccess;
  k_raw_lines<R><<<nk, 128, 0, st>>>(g, work, gmap, f, k0);
  return cudaGetLastError();
}

cudaError_t launch_gmap_backtrace(cudaStream_t st, const Geom &g, double2 *gmap, int f) {
  k_gmap_backtrace<<<8, 128, 0, st>>>(g, gmap, f);
  return cudaGetLastError();
}

template <typename R>
cudaError_t launch_copy_local(cudaStream_t st, long long n, const double2 *in,
                              typename Cx<R>::T *out, int) {
  if (n <= 0) return cudaSuccess;
  k_copy_local<R><<<(unsigned)((n + 255) / 256 < 4096 ? (n + 255) / 256 : 4096), 256, 0, st>>>(n, in, out);
  return cudaGetLastError();
}
template <typename R>
cudaError_t launch_copy_local_back(cudaStream_t st, long long n, const typename Cx<R>::T *in,
                                   double2 *out) {
  if (n <= 0) return cudaSuccess;
  k_copy_local_back<R><<<(unsigned)((n + 255) / 256 < 4096 ? (n + 255) / 256 : 4096), 256, 0, st>>>(n, in, out);
  return cudaGetLastError();
}

#define DDS_INST(R)                                                                             \
  template cudaError_t launch_assemble<R>(cudaStream_t, const Geom &, const Tables &, int,     \
                                          const Col *, Cx<R>::T *, const double2 *,           \
                                          const double2 *, int, const Cx<R>::T *, long long,   \
                                          long long, int, long long, int *);                    \
  template cudaError_t launch_subst<R>(cudaStream_t, const Geom &, int, const Panel *,         \
                                       const Col *, const Cx<R>::T *, const Cx<R>::T *,        \
                                       Cx<R>::T *, int);                                        \
  template cudaError_t launch_extract<R>(cudaStream_t, const Geom &, int, const Col *,         \
                                         const Cx<R>::T *, double2 *, int, Cx<R>::T *,         \
                                         Cx<R>::T *, const int *, int, int);                    \
  template cudaError_t launch_trace_sweeps<R>(cudaStream_t, const Geom &, const TraceStep *,   \
                                              int, int, const TracePanel *,                     \
                                              const Cx<R>::T *, Cx<R>::T *, const Cx<R>::T *,  \
                                              const int *, int, unsigned *, int *, int);        \
  template cudaError_t launch_unit_traces<R>(cudaStream_t, const Geom &, const Tables &, int,  \
                                             int, Cx<R>::T *);                                  \
  template cudaError_t launch_raw_lines<R>(cudaStream_t, const Geom &, int, const Cx<R>::T *,  \
                                           Cx<R>::T *, int, int);                               \
  template cudaError_t launch_copy_local<R>(cudaStream_t, long long, const double2 *,          \
                                            Cx<R>::T *, int);                                   \
  template cudaError_t launch_copy_local_back<R>(cudaStream_t, long long, const Cx<R>::T *,    \
                                                 double2 *);

DDS_INST(float)
DDS_INST(double)

}  // namespace dds
