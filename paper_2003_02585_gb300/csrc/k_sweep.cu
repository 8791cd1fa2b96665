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
                           long long slot_stride, int *__restrict__ nzflag,
                           int *__restrict__ badrhs) {
  using C = typename Cx<R>::T;
  const Col c = cols[blockIdx.x];
  bool nz = false;   // any nonzero entry written (the local solve of a zero source is zero)
  bool bad = false;  // a NaN or infinite source entry (its RHS is reported as NaN)
  C *x = work + (long long)c.slot * g.Nloc;
  int k[3];
  sub_index(g, c.sub, k);
  // every local node written once: the source on the own range, zero elsewhere; consecutive
  // threads take consecutive nodes (32-bit index arithmetic), four loads in flight per thread
  {
    int lo[3] = {0, 0, 0}, hi[3] = {0, 0, 0};
    if (with_source)
      for (int a = 0; a < g.dim; ++a) own_range(g, k, a, lo[a], hi[a]);
    const double2 *bb = b + (long long)c.rhs * g.Nglob + (long long)k[0] * g.m[0] +
                        (long long)g.G[0] * ((long long)k[1] * g.m[1] +
                                             (long long)g.G[1] * (g.dim == 3 ? (long long)k[2] * g.m[2] : 0));
    const int M0 = g.M[0], M1 = g.M[1], nloc = (int)g.Nloc;
    const long long G0 = g.G[0], G01 = (long long)g.G[0] * g.G[1];
    constexpr int U = 4;
    for (int e0 = threadIdx.x; e0 < nloc; e0 += U * blockDim.x) {
      C v[U];
#pragma unroll
      for (int u = 0; u < U; ++u) {
        const int e = e0 + u * blockDim.x;
        v[u] = czero<C>();
        const int i0 = e % M0, r = e / M0, i1 = r % M1, i2 = r / M1;
        if (e < nloc && i0 >= lo[0] && i0 < hi[0] && i1 >= lo[1] && i1 < hi[1] &&
            (g.dim < 3 || (i2 >= lo[2] && i2 < hi[2]))) {
          const double2 s = bb[i0 + G0 * i1 + G01 * i2];
          v[u] = to_c(s, C());
          nz = nz || v[u].x != 0 || v[u].y != 0;
          bad = bad || !isfinite(s.x) || !isfinite(s.y);
        }
      }
#pragma unroll
      for (int u = 0; u < U; ++u) {
        const int e = e0 + u * blockDim.x;
        if (e < nloc) x[e] = v[u];
      }
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
  if (badrhs != nullptr) {
    const int anybad = __syncthreads_or(bad);
    if (threadIdx.x == 0 && anybad) atomicOr(badrhs + c.rhs, 1);
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
  if (p.ncol == 0) return;   // an empty panel of a compacted list (zero-work skipping)
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
    // the own range, one warp per grid row (x1 fastest, coalesced on both sides)
    int lo[3] = {0, 0, 0}, hi[3] = {1, 1, 1};
    for (int a = 0; a < g.dim; ++a) own_range(g, k, a, lo[a], hi[a]);
    const int w1 = hi[1] - lo[1], rows = w1 * (hi[2] - lo[2]);
    double2 *uu = u + (long long)c.rhs * g.Nglob;
    const int lane = threadIdx.x & 31, nw = blockDim.x >> 5;
    for (int row = threadIdx.x >> 5; row < rows; row += nw) {
      const int i1 = lo[1] + row % w1, i2 = lo[2] + row / w1;
      const long long p1 = (long long)k[1] * g.m[1] + i1;
      const long long p2 = g.dim == 3 ? (long long)k[2] * g.m[2] + i2 : 0;
      double2 *urow = uu + (long long)k[0] * g.m[0] + (long long)g.G[0] * (p1 + (long long)g.G[1] * p2);
      const C *xr = x + (long long)g.M[0] * (i1 + (long long)g.M[1] * i2);
      for (int i0 = lo[0] + lane; i0 < hi[0]; i0 += 32) {
        const double2 xv = to_c64(xr[i0]);
        urow[i0] = own_mode == 1 ? cadd(urow[i0], xv) : xv;
      }
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
// Trace operator of every sweep (the trace-transfer form of the sweeps): for every (sub, rhs)
// column of a sweep-l subdomain solve,
//   out_d = Gmap_F,d * in (+ the raw own-source lines in the first sweep),
// where in = the traces received in slot l and out_d goes to the neighbour across side d, into
// the slot the route names.  Gmap already holds the back-trace correction.  Only output sides
// with a route and a neighbour, and receiving sides with a neighbour (in_mask), are touched:
// every other term is exactly zero or unused.
// Gmap layout per factor: [output side d][row tile of 64][input k = 0..T)[64 rows], rows past
// 2 Lt_d zero, so the rows of one tile for a run of consecutive inputs are one contiguous slice.
// ------------------------------------------------------------------------------------------
long long gmap_elems(const Geom &g, int nfac) { return gmap_index(g, nfac, 0, 0, 0, 0); }

// Work items of the cooperative trace launch (built on the host, TraceItem): one output side,
// one 64-row tile, one panel of up to 8 columns and one segment of at most kTraceSeg consecutive
// inputs of one receiving side.  A CTA (256 threads) runs an item as
//   map slice (n inputs x 64 rows) -> shared memory by one bulk copy on an mbarrier,
//   inputs (n x 8 columns) -> one of two shared-memory buffers by cp.async (slots written by
//   earlier levels; the next item's inputs land in the other buffer during this item's FMAs),
//   four K-groups of 64 threads; thread (row pair rp, column group cg) of a group accumulates
//   rows 2 rp, 2 rp + 1 x columns 4 cg .. 4 cg + 3 over its quarter of the inputs (a tile with
//   at most 32 live rows: eight K-groups over 16 row pairs), on packed two-lane FMAs,
//   the partial tiles meet in shared memory; every thread then owns one (column, row pair)
//   and adds it into the receiver's slot with one vector reduction (segments of one output meet
//   there; the slot accumulates with += in any case).
// Item records carry their columns' slot offsets precomputed; warp 0 fetches a record one item
// ahead of writing its descriptors, and the next item's map-slice copy is issued as soon as the
// slice buffer is free.
constexpr int kTraceSeg = 104;

template <typename C> __device__ inline void atomic_cadd(C *dst, C v);
template <> __device__ inline void atomic_cadd<float2>(float2 *dst, float2 v) {
  atomicAdd(&dst->x, v.x);
  atomicAdd(&dst->y, v.y);
}
template <> __device__ inline void atomic_cadd<double2>(double2 *dst, double2 v) {
  atomicAdd(&dst->x, v.x);
  atomicAdd(&dst->y, v.y);
}

// Level completion counters of the cooperative launch: after its items of level v a CTA adds 1
// to cnt[8 v + (blockIdx % 8)] (eight words, so arrivals do not all hit one address); a CTA with
// items in level v + 1 first waits until the eight words of level v sum to gridDim.x.  CTAs
// without items never wait.  The counters are zeroed before every launch.  The wait is bounded:
// on a timeout the CTA records code 4 and goes on (results wrong, launch ends, the host reports
// DDS_ETIMEOUT).
__device__ inline void step_arrive(unsigned *cnt, int s) {
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    atomicAdd(cnt + s * kStepCounters + (blockIdx.x % kStepCounters), 1u);
  }
}
__device__ inline void step_wait(const unsigned *cnt, int s, int *err, unsigned limit) {
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
      if (lane == 0) stop = (++spins > limit) || *reinterpret_cast<volatile int *>(err) != 0;
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

// descriptors of a staged item in shared memory (three buffers: the item in flight, the next
// one, whose inputs are loaded during the current FMAs, and the one after, written meanwhile)
struct TraceItemSmem {
  long long cbase[8];   // input trace base of each column in the trace slots (-1: no column)
  long long dbase[8];   // output base in the receiver's slot (-1: no receiver)
  long long rbase[8];   // raw own-source line base of the output side
  int factor, ncol, n, k0, tile, dout, raw, pad;
};

// an item record, fetched by warp 0 one item ahead of its staging: the header (every lane) and
// the column pair of lane c < 8 (independent loads, no chain)
struct TracePre {
  int4 h;
  int2 col;
};

__device__ inline TracePre trace_fetch(const int4 *__restrict__ hdr, const int2 *__restrict__ cols,
                                       long long idx) {
  TracePre p;
  const int lane = threadIdx.x & 31;
  p.h = __ldg(hdr + idx);
  p.col = lane < 8 ? __ldg(cols + idx * 8 + lane) : make_int2(-1, -1);
  return p;
}

// warp 0: write an item's descriptors (no copy yet)
__device__ inline void trace_describe(const Geom &g, const TracePre &p, TraceItemSmem &it,
                                      long long slot_stride) {
  const int lane = threadIdx.x & 31;
  const int l = p.h.y & 0xFFFF, lp = (p.h.y >> 16) & 0xFFFF;
  const int dout = p.h.w & 0xFF;
  if (lane == 0) {
    it.factor = p.h.x & 0xFFFFFF;
    it.ncol = (p.h.x >> 24) & 0xFF;
    it.k0 = p.h.z & 0xFFFF;
    it.n = (p.h.z >> 16) & 0xFFFF;
    it.dout = dout;
    it.tile = (p.h.w >> 8) & 0xFF;
    it.raw = (p.h.w >> 16) & 1;
  }
  if (lane < 8) {
    const int own = p.col.x, nbo = p.col.y;   // (RHS, subdomain) column / its receiver
    it.cbase[lane] = own >= 0 ? l * slot_stride + (long long)own * g.T : -1;
    it.dbase[lane] = nbo >= 0 ? lp * slot_stride + (long long)nbo * g.T + g.toff[dout ^ 1] : -1;
    it.rbase[lane] = (long long)own * g.T + g.toff[dout];
  }
}

// thread 0: issue the map-slice copy of a described item (a plain arrival for a raw-only item),
// so that every item completes exactly one phase of `bar`
template <typename C>
__device__ inline void trace_copy(const Geom &g, const TraceItemSmem &it, C *Gs, uint64_t *bar,
                                  const C *__restrict__ gmap) {
  if (it.n > 0) {
    const uint32_t bytes = (uint32_t)(it.n * kTraceRows * sizeof(C));
    fence_proxy_async();   // earlier generic reads of Gs before the async write
    mbar_arrive_expect_tx(bar, bytes);
    bulk_g2s(Gs, gmap + gmap_index(g, it.factor, it.dout, it.tile, it.k0, 0), bytes, bar);
  } else {
    mbar_arrive(bar);
  }
}

// the item's inputs, copied asynchronously (cp.async, zero fill for missing columns and past n):
// element (column c, input kk) of thread idx = c * kTraceSeg + kk (runs of one column are
// contiguous in the slot) goes to vin[kk][c]; the caller commits and waits
template <typename C>
__device__ inline void trace_gather(const TraceItemSmem &it, const C *gtr, C *vin) {
  for (int idx = threadIdx.x; idx < 8 * kTraceSeg; idx += 256) {
    const int c = idx / kTraceSeg, kk = idx - c * kTraceSeg;
    const long long b = it.cbase[c];
    const bool live = b >= 0 && kk < it.n;
    const C *src = live ? gtr + b + it.k0 + kk : gtr;
    if constexpr (sizeof(C) == 8)
      cp_async8(vin + kk * 8 + c, src, live ? 8u : 0u);
    else
      cp_async16(vin + kk * 8 + c, src, live ? 16u : 0u);
  }
  cp_async_commit();
}

// two consecutive complex values from shared memory (one 16-byte load in single precision)
__device__ inline void lds2(const float2 *p, float2 &x, float2 &y) {
  const float4 t = *reinterpret_cast<const float4 *>(p);
  x = make_float2(t.x, t.y);
  y = make_float2(t.z, t.w);
}
__device__ inline void lds2(const double2 *p, double2 &x, double2 &y) {
  x = p[0];
  y = p[1];
}

// Partial tile of K-group kg of KG: rows 2 rp, 2 rp + 1 (A = map slice + 2 rp, row stride 64)
// times columns 4 cg .. 4 cg + 3 (B = inputs + 4 cg, input stride 8) over the group's share of
// the n inputs.  Single precision runs on packed two-lane FMAs: per (row, column)
//   P += (a.re, a.re) * (b.re, b.im),   Q += (a.im, a.im) * (b.im, b.re),
//   a b = (P.re - Q.re, P.im + Q.im),
// which halves the FMA instructions issued against four scalar FMAs per complex product.
__device__ inline void trace_tile_fma(const float2 *A, const float2 *B, int n, int kg, int KG,
                                      float2 (&acc)[2][4]) {
  const int nq = (n + KG - 1) / KG;
  const int i0 = min(n, kg * nq), i1 = min(n, i0 + nq);
  float2 P[2][4], Q[2][4];
#pragma unroll
  for (int j = 0; j < 4; ++j) P[0][j] = P[1][j] = Q[0][j] = Q[1][j] = make_float2(0.f, 0.f);
#pragma unroll 4
  for (int i = i0; i < i1; ++i) {
    float2 a0, a1, b[4];
    lds2(A + i * kTraceRows, a0, a1);
    lds2(B + i * 8, b[0], b[1]);
    lds2(B + i * 8 + 2, b[2], b[3]);
    const float2 a0r = make_float2(a0.x, a0.x), a0i = make_float2(a0.y, a0.y);
    const float2 a1r = make_float2(a1.x, a1.x), a1i = make_float2(a1.y, a1.y);
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const float2 bs = make_float2(b[j].y, b[j].x);
      P[0][j] = __ffma2_rn(a0r, b[j], P[0][j]);
      Q[0][j] = __ffma2_rn(a0i, bs, Q[0][j]);
      P[1][j] = __ffma2_rn(a1r, b[j], P[1][j]);
      Q[1][j] = __ffma2_rn(a1i, bs, Q[1][j]);
    }
  }
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    acc[0][j] = make_float2(P[0][j].x - Q[0][j].x, P[0][j].y + Q[0][j].y);
    acc[1][j] = make_float2(P[1][j].x - Q[1][j].x, P[1][j].y + Q[1][j].y);
  }
}
__device__ inline void trace_tile_fma(const double2 *A, const double2 *B, int n, int kg, int KG,
                                      double2 (&acc)[2][4]) {
  const int nq = (n + KG - 1) / KG;
  const int i0 = min(n, kg * nq), i1 = min(n, i0 + nq);
#pragma unroll
  for (int j = 0; j < 4; ++j) acc[0][j] = acc[1][j] = make_double2(0.0, 0.0);
#pragma unroll 4
  for (int i = i0; i < i1; ++i) {
    double2 a0, a1, b0, b1, b2, b3;
    lds2(A + i * kTraceRows, a0, a1);
    lds2(B + i * 8, b0, b1);
    lds2(B + i * 8 + 2, b2, b3);
    cfma(acc[0][0], a0, b0); cfma(acc[0][1], a0, b1);
    cfma(acc[0][2], a0, b2); cfma(acc[0][3], a0, b3);
    cfma(acc[1][0], a1, b0); cfma(acc[1][1], a1, b1);
    cfma(acc[1][2], a1, b2); cfma(acc[1][3], a1, b3);
  }
}

// Every trace solve of one DDM application in one cooperative launch.  The schedule is a list of
// dataflow levels: a trace solve (sweep l, subdomain X) sits one level below the deepest solve
// whose traces are routed into its slot l, so every level only reads slots that earlier levels
// completed.  The items of level v are records lev_off[v] .. lev_off[v + 1] - 1, heaviest first;
// CTA b takes positions b, 2G - 1 - b, 2G + b, ... (a snake over the G CTAs).  A CTA with items
// in level v first waits until every CTA is done with level v - 1 (counters above); the
// descriptors and map slice of its first item depend on no trace and are staged before that
// wait.  Per item (two CTA barriers):
//   wait for the map slice; the next item's inputs are loaded into registers; FMAs;
//   barrier; the next item's map-slice copy is issued and its inputs stored, the partial tiles
//   written, the item after it described;  barrier;  reduction and vector reductions into the
//   receivers' slots.
constexpr int kMaxSmemLevels = 1024;

template <typename R>
__global__ void __launch_bounds__(256, sizeof(R) == 4 ? 2 : 1)
    k_trace_sweeps(Geom g, const int4 *__restrict__ hdr, const int2 *__restrict__ cols,
                   const int *__restrict__ lev_off, int nlev,
                   const typename Cx<R>::T *__restrict__ gmap, typename Cx<R>::T *__restrict__ gtr,
                   const typename Cx<R>::T *__restrict__ rawf, int nrhs, unsigned *cnt,
                   int *__restrict__ err, unsigned wait_limit) {
  using C = typename Cx<R>::T;
  extern __shared__ __align__(128) unsigned char smem_raw[];
  C *Gs = reinterpret_cast<C *>(smem_raw);            // map slice [k][64 rows]
  C *vin2 = Gs + kTraceSeg * kTraceRows;              // inputs [2 buffers][k][8 columns]
  C *red = vin2 + 2 * 8 * kTraceSeg;                  // partial tiles [K-group][col][row pair][2]
                                                      // (4 K-groups x 32 row pairs, or 8 x 16)
  uint64_t *bar = reinterpret_cast<uint64_t *>(red + 4 * 8 * 64);
  int *lo_s = reinterpret_cast<int *>(bar + 2);       // level offsets (nlev < kMaxSmemLevels)
  __shared__ TraceItemSmem its[3];
  const bool lv_smem = nlev < kMaxSmemLevels;
  for (int i = threadIdx.x; lv_smem && i <= nlev; i += blockDim.x) lo_s[i] = lev_off[i];
  if (threadIdx.x == 0) {
    mbar_init(bar, 1);
    mbar_init_fence();
  }
  __syncthreads();
  auto lev = [&](int v) { return lv_smem ? lo_s[v] : __ldg(lev_off + v); };
  const int G = (int)gridDim.x, b = (int)blockIdx.x, tid = threadIdx.x, warp = tid >> 5;
  auto pos = [&](int r) { return r * G + ((r & 1) ? G - 1 - b : b); };
  const long long slot_stride = (long long)nrhs * g.nsub * g.T;
  // epilogue roles: column ec, row pair rp (compute roles per item below)
  const int rp = tid & 31, ec = tid >> 5;
  int s = 0;   // descriptor buffer of the current item (the next ones: s + 1, s + 2 mod 3)
  int vb = 0;  // input buffer of the current item
  uint32_t phase = 0;
  TracePre pre;   // warp 0: the record of the item after the next
  for (int v = 0; v < nlev; ++v) {
    const int base = lev(v), Nv = lev(v + 1) - base;
    if (v > 0) step_arrive(cnt, v - 1);
    if (pos(0) >= Nv) continue;
    if (warp == 0) {
      // the first three records of the level in one round of loads
      const bool h1 = pos(1) < Nv, h2 = pos(2) < Nv;
      const TracePre p0 = trace_fetch(hdr, cols, base + pos(0));
      const TracePre p1 = h1 ? trace_fetch(hdr, cols, base + pos(1)) : p0;
      if (h2) pre = trace_fetch(hdr, cols, base + pos(2));
      trace_describe(g, p0, its[s], slot_stride);
      __syncwarp();
      if (tid == 0) trace_copy<C>(g, its[s], Gs, bar, gmap);
      if (h1) trace_describe(g, p1, its[(s + 1) % 3], slot_stride);
    }
    __syncthreads();
    if (v > 0) step_wait(cnt, v - 1, err, wait_limit);
    trace_gather<C>(its[s], gtr, vin2 + vb * 8 * kTraceSeg);
    cp_async_wait_all();
    for (int r = 0; pos(r) < Nv; ++r) {
      const TraceItemSmem &it = its[s];
      TraceItemSmem &nx = its[(s + 1) % 3];
      const bool next = pos(r + 1) < Nv, next2 = pos(r + 2) < Nv;
      const C *vin = vin2 + vb * 8 * kTraceSeg;
      const bool ok = mbar_wait(bar, phase);
      if (__syncthreads_or(!ok) && tid == 0) {
        atomicExch(err, 3);
        mbar_wait(bar, phase);   // bounded second wait for the copy in flight
      }
      // the next item's inputs (slots of earlier levels) land in the other buffer meanwhile
      if (next) trace_gather<C>(nx, gtr, vin2 + (vb ^ 1) * 8 * kTraceSeg);
      // Compute roles: a full tile has four K-groups of 64 threads (32 row pairs x 2 column
      // groups); a tile with at most 32 live rows (the last tile of a side) has eight K-groups of
      // 32 threads over its 16 live row pairs, so its FMAs take half the time.
      const bool half = 2 * g.Lt[it.dout] - it.tile * kTraceRows <= kTraceRows / 2;
      const int KG = half ? 8 : 4;
      const int kg = half ? tid >> 5 : tid >> 6, crp = half ? tid & 15 : tid & 31;
      const int cg = half ? (tid >> 4) & 1 : (tid >> 5) & 1;
      const int RPS = half ? 16 : 32;   // row pairs per (K-group, column) in the partial tiles
      C acc[2][4];
      trace_tile_fma(Gs + 2 * crp, vin + 4 * cg, it.n, kg, KG, acc);
      __syncthreads();   // Gs and this item's inputs are free
      if (next && tid == 32) trace_copy<C>(g, nx, Gs, bar, gmap);
      if (next2 && warp == 0) {
        trace_describe(g, pre, its[(s + 2) % 3], slot_stride);
        if (pos(r + 3) < Nv) pre = trace_fetch(hdr, cols, base + pos(r + 3));
      }
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        C *p = red + (((kg * 8 + 4 * cg + j) * RPS + crp) << 1);
        p[0] = acc[0][j];
        p[1] = acc[1][j];
      }
      cp_async_wait_all();
      __syncthreads();   // partial tiles, next inputs and descriptors are in place
      {
        C o0 = czero<C>(), o1 = czero<C>();
        // (a half tile has no row pairs past 16: their rows are past 2 Lt)
        for (int q = 0; q < KG && rp < RPS; ++q) {
          C u0, u1;
          lds2(red + (((q * 8 + ec) * RPS + rp) << 1), u0, u1);
          o0 = cadd(o0, u0);
          o1 = cadd(o1, u1);
        }
        const int rr = it.tile * kTraceRows + 2 * rp;   // rows rr, rr + 1 (2 Lt is even)
        const long long db = it.dbase[ec];
        if (ec < it.ncol && db >= 0 && rr < 2 * g.Lt[it.dout]) {
          if (it.raw) {
            const C *rw = rawf + it.rbase[ec] + rr;
            o0 = cadd(o0, rw[0]);
            o1 = cadd(o1, rw[1]);
          }
          C *dst = gtr + db + rr;
          if constexpr (sizeof(R) == 4) {
            // both rows in one 16-byte vector reduction (T, the side offsets and rr are even)
            red_add_f4(reinterpret_cast<float4 *>(dst), make_float4(o0.x, o0.y, o1.x, o1.y));
          } else {
            atomic_cadd(dst, o0);
            atomic_cadd(dst + 1, o1);
          }
        }
      }
      s = (s + 1) % 3;
      phase ^= 1u;
      vb ^= 1;
    }
  }
  // every staged item is consumed in its level, so no copy is in flight here
}

// ------------------------------------------------------------------------------------------
// Zero-work skipping (Algorithm 2.1: "if f_ij != 0 solve, else u_ij = 0").  A local problem
// whose assembled right-hand side is exactly zero has the zero solution, which its work slot
// already holds, so its substitutions are dropped.  One CTA per group of consecutive panels
// that share a factor (gr = column range [x, y), panel range [z, w)): the group's columns with
// a nonzero right-hand side (nz[slot], written by k_assemble) are packed, in their order, into
// dcols[x ...]; the group's panels become ceil(live / pc) panels of up to pc packed columns
// followed by empty ones (ncol = 0, which every substitution kernel leaves at once).
// stats[0] += live columns, stats[1] += columns.
// ------------------------------------------------------------------------------------------
__global__ void __launch_bounds__(1024)
    k_compact_panels(const int4 *__restrict__ groups, const Panel *__restrict__ pans,
                     const Col *__restrict__ cols, const int *__restrict__ nz,
                     Col *__restrict__ dcols, Panel *__restrict__ dpans, int pc,
                     unsigned long long *__restrict__ stats) {
  __shared__ int wsum[32];
  const int4 gr = groups[blockIdx.x];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nw = blockDim.x >> 5;
  int carry = 0;   // live columns packed so far (the same in every thread)
  for (int base = gr.x; base < gr.y; base += blockDim.x) {
    const int i = base + tid;
    const bool live = i < gr.y && nz[cols[i].slot] != 0;
    const unsigned m = __ballot_sync(0xffffffffu, live);
    if (lane == 0) wsum[warp] = __popc(m);
    __syncthreads();
    if (warp == 0) {
      int v = lane < nw ? wsum[lane] : 0;
      for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(0xffffffffu, v, o);
        if (lane >= o) v += y;
      }
      wsum[lane] = v;   // inclusive over warps
    }
    __syncthreads();
    const int before = warp > 0 ? wsum[warp - 1] : 0;
    if (live) dcols[gr.x + carry + before + __popc(m & ((1u << lane) - 1u))] = cols[i];
    carry += wsum[nw - 1];
    __syncthreads();   // wsum is rewritten in the next chunk
  }
  const int n = carry, factor = pans[gr.z].factor;
  const int need = (n + pc - 1) / pc;
  for (int q = tid; q < gr.w - gr.z; q += blockDim.x) {
    Panel p;
    p.factor = factor;
    p.pad = 0;
    p.col0 = q < need ? gr.x + q * pc : gr.x;
    p.ncol = q < need ? min(pc, n - q * pc) : 0;
    dpans[gr.z + q] = p;
  }
  if (tid == 0) {
    atomicAdd(stats, (unsigned long long)n);
    atomicAdd(stats + 1, (unsigned long long)(gr.y - gr.x));
  }
}

cudaError_t launch_compact_panels(cudaStream_t st, int ngroups, const int4 *groups,
                                  const Panel *pans, const Col *cols, const int *nz, Col *dcols,
                                  Panel *dpans, int pc, unsigned long long *stats) {
  if (ngroups <= 0) return cudaSuccess;
  k_compact_panels<<<ngroups, 1024, 0, st>>>(groups, pans, cols, nz, dcols, dpans, pc, stats);
  return cudaGetLastError();
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
                            long long slot_stride, int *nzflag, int *badrhs) {
  if (ncols <= 0) return cudaSuccess;
  k_assemble<R><<<ncols, 256, 0, st>>>(g, tb, cols, work, b, with_source, traces, trs_rhs,
                                       trs_sub, nslots, slot_stride, nzflag, badrhs);
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
cudaError_t launch_trace_sweeps(cudaStream_t st, const Geom &g, const int4 *hdr, const int2 *cols,
                                int nitems, const int *lev_off, int nlevels,
                                const typename Cx<R>::T *gmap, typename Cx<R>::T *gtr,
                                const typename Cx<R>::T *rawf, int nrhs, unsigned *gbar, int *err,
                                int ctas_per_sm, unsigned wait_limit) {
  if (nitems <= 0 || nlevels <= 0) return cudaSuccess;
  const size_t smem = trace_smem_bytes(sizeof(typename Cx<R>::T), nlevels);
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
  return cudaLaunchKernelEx(&cfg, k_trace_sweeps<R>, g, hdr, cols, lev_off, nlevels, gmap, gtr,
                            rawf, nrhs, gbar, err, wait_limit);
}

size_t trace_counter_bytes(int nlevels) { return (size_t)nlevels * kStepCounters * sizeof(unsigned); }

size_t trace_smem_bytes(size_t elem, int nlevels) {
  size_t b = ((size_t)kTraceSeg * kTraceRows + 2 * 8 * kTraceSeg + 4 * 8 * 64) * elem + 16;
  if (nlevels < kMaxSmemLevels) b += (size_t)(nlevels + 1) * sizeof(int);
  return b;
}

// Items of the sweep-l trace solves of the panels tp[p0, p1): per panel, every output side with a
// route and a neighbour of some column, every 64-row tile of it and every input segment of the
// receiving sides (in_mask) that have a neighbour of some column; a side's 2 Lt inputs are cut
// into the fewest segments of at most kTraceSeg, of equal length.  In the first sweep one item
// per output tile also adds the raw own-source lines (an input-free item if nothing is received).
void trace_items_for(const Geom &g, const TracePanel *tp, int p0, int p1, int l, const int *route,
                     int in_mask, std::vector<TraceItem> &out) {
  for (int p = p0; p < p1; ++p) {
    const TracePanel &pn = tp[p];
    auto any_nb = [&](int d) {
      for (int c = 0; c < pn.ncol; ++c)
        if (sub_neighbour(g, pn.sub[c], d) >= 0) return true;
      return false;
    };
    TraceItem it{};
    for (int dout = 0; dout < g.nsides; ++dout) {
      const int lp = route[l * 6 + dout];
      if (lp < 0 || !any_nb(dout)) continue;
      for (int c = 0; c < 8; ++c) {
        if (c >= pn.ncol) { it.col[c] = make_int2(-1, -1); continue; }
        const int nb = sub_neighbour(g, pn.sub[c], dout);
        it.col[c] = make_int2(pn.rhs[c] * g.nsub + pn.sub[c], nb >= 0 ? pn.rhs[c] * g.nsub + nb : -1);
      }
      for (int tile = 0; tile < trace_tiles(g, dout); ++tile) {
        int raw = l == 0 ? 1 : 0;
        auto emit = [&](int k0, int n) {
          it.h = make_int4(pn.factor | (pn.ncol << 24), l | (lp << 16), k0 | (n << 16),
                           dout | (tile << 8) | (raw << 16));
          out.push_back(it);
          raw = 0;
        };
        for (int sd = 0; sd < g.nsides; ++sd) {
          if (!((in_mask >> sd) & 1) || !any_nb(sd)) continue;
          const int len = 2 * g.Lt[sd], ns = (len + kTraceSeg - 1) / kTraceSeg;
          for (int j = 0; j < ns; ++j) {
            const int a = j * len / ns, e = (j + 1) * len / ns;
            emit(g.toff[sd] + a, e - a);
          }
        }
        if (raw) emit(0, 0);
      }
    }
  }
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
                                          long long, int, long long, int *, int *);             \
  template cudaError_t launch_subst<R>(cudaStream_t, const Geom &, int, const Panel *,         \
                                       const Col *, const Cx<R>::T *, const Cx<R>::T *,        \
                                       Cx<R>::T *, int);                                        \
  template cudaError_t launch_extract<R>(cudaStream_t, const Geom &, int, const Col *,         \
                                         const Cx<R>::T *, double2 *, int, Cx<R>::T *,         \
                                         Cx<R>::T *, const int *, int, int);                    \
  template cudaError_t launch_trace_sweeps<R>(cudaStream_t, const Geom &, const int4 *,         \
                                              const int2 *, int, const int *, int,              \
                                              const Cx<R>::T *, Cx<R>::T *, const Cx<R>::T *,  \
                                              int, unsigned *, int *, int, unsigned);           \
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
