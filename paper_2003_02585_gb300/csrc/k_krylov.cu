// FP64 kernels for the global problem: the J-scaled PML operator (Eq. 2.3 / 4.1 times J,
// 5/7-point stencil), J-scaling of sources, and the batched reductions and vector updates of
// flexible GMRES (Section 5.2: GMRES with the DDM as preconditioner).
#include "dds_internal.cuh"

namespace dds {

__device__ inline double2 crecip64(double2 z) {
  const double m = z.x * z.x + z.y * z.y;
  return make_double2(z.x / m, -z.y / m);
}

// (A u)_p = sum_a (prod_{b != a} alpha_b) / h^2 [ (u_{p+e_a} - u_p) / alpha_a(p+1/2)
//                                               - (u_p - u_{p-e_a}) / alpha_a(p-1/2) ]
//           + kappa^2 J u_p,          Dirichlet outside the extended grid.
// The stencil is precomputed per node at set-up (tb.c0: centre, tb.cp[a]: coupling to p + e_a,
// so the coupling to p - e_a is tb.cp[a][p - e_a]); each thread applies it to every RHS.
// One thread per (node, RHS): the stencil coefficients of a node are re-read per RHS (from L1/L2)
// so that every FP64 pipe has independent work.  Outside the PML every coefficient is real: two
// FMAs per stencil term.
template <int DIM>
__global__ void __launch_bounds__(256) k_apply_A(Geom g, Tables tb, int nrhs, const double2 *__restrict__ u,
                          double2 *__restrict__ Au, int divide_by_J,
                          const double2 *__restrict__ sub, const long long *__restrict__ uoff,
                          const long long *__restrict__ aoff) {
  const int N = (int)g.Nglob;
  const int G0 = g.G[0], G1 = g.G[1];
  const long long total = (long long)nrhs * N;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
       i += (long long)gridDim.x * blockDim.x) {
    const int r = (int)(i / N), q = (int)(i - (long long)r * N);
    int p[3];
    p[0] = q % G0;
    p[1] = (q / G0) % G1;
    p[2] = DIM == 3 ? q / (G0 * G1) : 0;
    const double2 *ur = u + (uoff != nullptr ? uoff[r] : (long long)r * N) + q;
    const double2 c0 = tb.c0[q];
    double2 cpv[DIM], cmv[DIM], up[DIM], um[DIM];
    int st = 1;
    // "every imaginary part is zero" on the integer pipe (the FP64 pipe is the scarce one):
    // OR of the bit patterns with the sign bit dropped
    unsigned long long imag = (unsigned long long)__double_as_longlong(c0.y) << 1;
#pragma unroll
    for (int a = 0; a < DIM; ++a) {
      const bool hp = p[a] + 1 < g.G[a], hm = p[a] > 0;
      cpv[a] = hp ? tb.cp[a][q] : make_double2(0.0, 0.0);
      cmv[a] = hm ? tb.cp[a][q - st] : make_double2(0.0, 0.0);
      up[a] = hp ? ur[st] : make_double2(0.0, 0.0);
      um[a] = hm ? ur[-st] : make_double2(0.0, 0.0);
      imag |= ((unsigned long long)__double_as_longlong(cpv[a].y) << 1) |
              ((unsigned long long)__double_as_longlong(cmv[a].y) << 1);
      st *= g.G[a];
    }
    const bool real = imag == 0ull;
    const double2 uc = ur[0];
    // a subtracted vector (the residual) starts the chain when no J division follows
    const bool fold = sub != nullptr && !divide_by_J;
    double2 sum;
    if (real) {
      // one FMA chain per component: 2 + 4 DIM FP64 operations per node and RHS (the FP64
      // pipe, not latency, bounds this kernel: every node and RHS is an independent thread)
      double sx, sy;
      if (fold) {
        const double2 s0 = sub[i];
        sx = fma(c0.x, uc.x, -s0.x);
        sy = fma(c0.x, uc.y, -s0.y);
      } else {
        sx = c0.x * uc.x;
        sy = c0.x * uc.y;
      }
#pragma unroll
      for (int a = 0; a < DIM; ++a) {
        sx = fma(cpv[a].x, up[a].x, sx);
        sy = fma(cpv[a].x, up[a].y, sy);
        sx = fma(cmv[a].x, um[a].x, sx);
        sy = fma(cmv[a].x, um[a].y, sy);
      }
      sum = make_double2(sx, sy);
    } else {
      sum = cmul(c0, uc);
#pragma unroll
      for (int a = 0; a < DIM; ++a) {
        cfma(sum, cpv[a], up[a]);
        cfma(sum, cmv[a], um[a]);
      }
    }
    if (divide_by_J) {
      double2 J = make_double2(1.0, 0.0);
      for (int a = 0; a < DIM; ++a) J = cmul(J, tb.an_glob64[a][p[a]]);
      sum = cmul(sum, crecip64(J));
    }
    if (sub != nullptr && !(fold && real)) sum = csub(sum, sub[i]);
    Au[aoff != nullptr ? aoff[r] + q : i] = sum;
  }
}

// b[rhs] = J f[rhs], J = prod_a alpha_a(x_a) at the node; one thread per node, all RHS
__global__ void k_scale_J(Geom g, Tables tb, int nrhs, const double2 *__restrict__ f,
                          double2 *__restrict__ b) {
  const int N = (int)g.Nglob;
  const int G0 = g.G[0], G1 = g.G[1];
  for (int q = blockIdx.x * blockDim.x + threadIdx.x; q < N; q += gridDim.x * blockDim.x) {
    int p[3];
    p[0] = q % G0;
    p[1] = (q / G0) % G1;
    p[2] = g.dim == 3 ? q / (G0 * G1) : 0;
    double2 J = make_double2(1.0, 0.0);
    for (int a = 0; a < g.dim; ++a) J = cmul(J, tb.an_glob64[a][p[a]]);
    if (J.y == 0.0) {
      for (int r = 0; r < nrhs; ++r) {
        const double2 v = f[(long long)r * N + q];
        b[(long long)r * N + q] = make_double2(J.x * v.x, J.x * v.y);
      }
    } else {
      for (int r = 0; r < nrhs; ++r) b[(long long)r * N + q] = cmul(J, f[(long long)r * N + q]);
    }
  }
}

// partial[(rhs * nv + i) * nblk + blk] = sum over the block's elements of conj(V_i) * w.
// Grid-stride over elements, up to four vectors per pass over w, four elements per iteration in
// flight; each thread keeps its running sums in registers and the block reduces them once.  A
// vector that is w itself (a norm) costs two FMAs per element instead of four.
constexpr int kDotThreads = 256;
constexpr int kDotChunk = kDotThreads * 24;   // elements per block (sets nblk)

template <int NV>
__global__ void __launch_bounds__(kDotThreads) k_dots(long long N, int nv, int i0,
                                                     const double2 *__restrict__ V, long long vsv,
                                                     long long vsr, const double2 *__restrict__ w,
                                                     long long wsr, double2 *__restrict__ partial,
                                                     const long long *__restrict__ voff,
                                                     const long long *__restrict__ woff) {
  __shared__ double red[2 * NV][kDotThreads / 32];
  const int blk = blockIdx.x, nblk = gridDim.x;
  const int rhs = blockIdx.y;
  const double2 *ww = w + (woff != nullptr ? woff[rhs] : rhs * wsr);
  const double2 *vb = V + (voff != nullptr ? voff[rhs] : rhs * vsr);
  const double2 *v[NV];
  bool self[NV];
  double sr[NV], si[NV];
#pragma unroll
  for (int i = 0; i < NV; ++i) {
    v[i] = vb + (i0 + i) * vsv;
    self[i] = v[i] == ww;
    sr[i] = 0.0;
    si[i] = 0.0;
  }
  const long long stride = (long long)nblk * kDotThreads;
  long long n = (long long)blk * kDotThreads + threadIdx.x;
  for (; n + 3 * stride < N; n += 4 * stride) {
    double2 b[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) b[u] = ww[n + u * stride];
#pragma unroll
    for (int i = 0; i < NV; ++i) {
      if (self[i]) {
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          sr[i] = fma(b[u].x, b[u].x, sr[i]);
          sr[i] = fma(b[u].y, b[u].y, sr[i]);
        }
      } else {
        double2 a[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) a[u] = v[i][n + u * stride];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          sr[i] = fma(a[u].x, b[u].x, sr[i]);
          sr[i] = fma(a[u].y, b[u].y, sr[i]);
          si[i] = fma(a[u].x, b[u].y, si[i]);
          si[i] = fma(-a[u].y, b[u].x, si[i]);
        }
      }
    }
  }
  for (; n < N; n += stride) {
    const double2 b = ww[n];
#pragma unroll
    for (int i = 0; i < NV; ++i) {
      if (self[i]) {
        sr[i] = fma(b.x, b.x, sr[i]);
        sr[i] = fma(b.y, b.y, sr[i]);
      } else {
        const double2 a = v[i][n];
        sr[i] = fma(a.x, b.x, sr[i]);
        sr[i] = fma(a.y, b.y, sr[i]);
        si[i] = fma(a.x, b.y, si[i]);
        si[i] = fma(-a.y, b.x, si[i]);
      }
    }
  }
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int i = 0; i < NV; ++i) {
    for (int o = 16; o > 0; o >>= 1) {
      sr[i] += __shfl_down_sync(0xffffffffu, sr[i], o);
      si[i] += __shfl_down_sync(0xffffffffu, si[i], o);
    }
    if (lane == 0) {
      red[2 * i][warp] = sr[i];
      red[2 * i + 1][warp] = si[i];
    }
  }
  __syncthreads();
  if (threadIdx.x < NV) {
    const int i = threadIdx.x;
    double tr = 0.0, ti = 0.0;
    for (int q = 0; q < kDotThreads / 32; ++q) {
      tr += red[2 * i][q];
      ti += red[2 * i + 1][q];
    }
    partial[((long long)rhs * nv + i0 + i) * nblk + blk] = make_double2(tr, ti);
  }
}

int dots_chunk() { return kDotChunk; }

// Blocks per RHS for the dot and norm kernels: one resident wave over the whole GPU (at the
// occupancy of the widest dot kernel), never more than one block per 256 elements.  A grid of
// ceil(N / kDotChunk) blocks per RHS left a half-empty second wave at 640^2 x 16 RHS.
int dots_blocks(long long N, int nrhs) {
  int dev = 0, nsm = 0, per_sm = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_dots<4>, kDotThreads, 0) !=
          cudaSuccess) {
    cudaGetLastError();
    return (int)std::max<long long>(1, (N + kDotChunk - 1) / kDotChunk);
  }
  const long long want = ((long long)nsm * std::max(per_sm, 1) + nrhs - 1) / std::max(nrhs, 1);
  return (int)std::max<long long>(1, std::min(want, (N + kDotThreads - 1) / kDotThreads));
}

__global__ void k_dots_reduce(int count, int nblk, const double2 *__restrict__ partial,
                              double2 *__restrict__ out) {
  const int q = blockIdx.x;
  if (q >= count) return;
  double sr = 0.0, si = 0.0;
  for (int b = threadIdx.x; b < nblk; b += 32) {
    sr += partial[(long long)q * nblk + b].x;
    si += partial[(long long)q * nblk + b].y;
  }
  for (int o = 16; o > 0; o >>= 1) {
    sr += __shfl_down_sync(0xffffffffu, sr, o);
    si += __shfl_down_sync(0xffffffffu, si, o);
  }
  if (threadIdx.x == 0) out[q] = make_double2(sr, si);
}

// w[rhs] = (overwrite ? 0 : w[rhs]) + sign * sum_{i < nv} V_i[rhs] * coef[rhs * cstride + i]
//          (* cscale[rhs * cstride + i] when cscale is given)
// (grid.y = rhs).  The signed coefficients sit in shared memory; two elements per thread and
// iteration are in flight.  With `partial`, the block also sums |w|^2 of the result into
// partial[rhs * gridDim.x + blockIdx.x] (the norm of a Gram-Schmidt update in the same pass).
constexpr int kCombMaxNv = 64;

__global__ void __launch_bounds__(256) k_combination(long long N, int nv,
                                                     const double2 *__restrict__ V, long long vsv,
                                                     long long vsr, const double2 *__restrict__ coef,
                                                     int cstride, double sign,
                                                     const double *__restrict__ cscale,
                                                     double2 *__restrict__ w, long long wsr,
                                                     int overwrite, double2 *__restrict__ partial,
                                                     const long long *__restrict__ voff,
                                                     const long long *__restrict__ woff) {
  __shared__ double2 cs[kCombMaxNv];
  __shared__ double red[8];
  const int rhs = blockIdx.y;
  for (int i = threadIdx.x; i < nv; i += blockDim.x) {
    const double2 c = coef[(long long)rhs * cstride + i];
    const double f = cscale != nullptr ? sign * cscale[(long long)rhs * cstride + i] : sign;
    cs[i] = make_double2(f * c.x, f * c.y);
  }
  __syncthreads();
  double2 *ww = w + (woff != nullptr ? woff[rhs] : rhs * wsr);
  const double2 *vr = V + (voff != nullptr ? voff[rhs] : rhs * vsr);
  const long long stride = (long long)gridDim.x * blockDim.x;
  long long n = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  double nrm = 0.0;
  for (; n + stride < N; n += 2 * stride) {
    double2 a0 = make_double2(0.0, 0.0), a1 = a0;
    if (!overwrite) {
      a0 = ww[n];
      a1 = ww[n + stride];
    }
    for (int i = 0; i < nv; ++i) {
      const double2 c = cs[i];
      const double2 v0 = vr[i * vsv + n], v1 = vr[i * vsv + n + stride];
      cfma(a0, v0, c);
      cfma(a1, v1, c);
    }
    ww[n] = a0;
    ww[n + stride] = a1;
    nrm = fma(a0.x, a0.x, nrm);
    nrm = fma(a0.y, a0.y, nrm);
    nrm = fma(a1.x, a1.x, nrm);
    nrm = fma(a1.y, a1.y, nrm);
  }
  for (; n < N; n += stride) {
    double2 a0 = overwrite ? make_double2(0.0, 0.0) : ww[n];
    for (int i = 0; i < nv; ++i) cfma(a0, vr[i * vsv + n], cs[i]);
    ww[n] = a0;
    nrm = fma(a0.x, a0.x, nrm);
    nrm = fma(a0.y, a0.y, nrm);
  }
  if (partial == nullptr) return;
  for (int o = 16; o > 0; o >>= 1) nrm += __shfl_down_sync(0xffffffffu, nrm, o);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (lane == 0) red[warp] = nrm;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int q = 0; q < (int)(blockDim.x >> 5); ++q) t += red[q];
    partial[(long long)rhs * gridDim.x + blockIdx.x] = make_double2(t, 0.0);
  }
}

// out[rhs] = in[rhs] / sqrt(Re nrm2[rhs]) (0 where the norm vanishes)   (grid.y = rhs)
__global__ void k_scale_by_norm(long long N, const double2 *__restrict__ in,
                                const double2 *__restrict__ nrm2, double2 *__restrict__ out,
                                const long long *__restrict__ off) {
  const int rhs = blockIdx.y;
  const double q = nrm2[rhs].x;
  const double s = q > 0.0 ? 1.0 / sqrt(q) : 0.0;
  const long long base = off != nullptr ? off[rhs] : (long long)rhs * N;
  for (long long n = blockIdx.x * (long long)blockDim.x + threadIdx.x; n < N;
       n += (long long)gridDim.x * blockDim.x)
    out[base + n] = make_double2(in[base + n].x * s, in[base + n].y * s);
}

static inline unsigned grid_for(long long n) {
  long long b = (n + 255) / 256;
  return (unsigned)(b < 152 * 16 ? (b < 1 ? 1 : b) : 152 * 16);
}

// blocks per RHS for an N-element sweep repeated over nrhs (grid.y = nrhs)
static inline dim3 grid_rhs(long long N, int nrhs) {
  long long want = (152 * 8 + nrhs - 1) / nrhs;
  long long b = (N + 255) / 256;
  return dim3((unsigned)(b < want ? (b < 1 ? 1 : b) : want), (unsigned)nrhs);
}

cudaError_t launch_apply_A(cudaStream_t st, const Geom &g, const Tables &tb, int nrhs,
                           const double2 *u, double2 *Au, int divide_by_J, const double2 *sub,
                           const long long *uoff, const long long *aoff) {
  const unsigned grid = grid_for(g.Nglob * (long long)nrhs);
  if (g.dim == 2)
    k_apply_A<2><<<grid, 256, 0, st>>>(g, tb, nrhs, u, Au, divide_by_J, sub, uoff, aoff);
  else
    k_apply_A<3><<<grid, 256, 0, st>>>(g, tb, nrhs, u, Au, divide_by_J, sub, uoff, aoff);
  return cudaGetLastError();
}

cudaError_t launch_scale_J(cudaStream_t st, const Geom &g, const Tables &tb, int nrhs,
                           const double2 *f, double2 *b) {
  k_scale_J<<<grid_for(g.Nglob), 256, 0, st>>>(g, tb, nrhs, f, b);
  return cudaGetLastError();
}

cudaError_t launch_dots(cudaStream_t st, long long N, int nrhs, int nv, const double2 *V,
                        long long vsv, long long vsr, const double2 *w, long long wsr,
                        double2 *partial, double2 *out, int nblk, const long long *voff,
                        const long long *woff) {
  dim3 grid(nblk, nrhs);
  for (int i0 = 0; i0 < nv; i0 += 4) {
    switch (std::min(4, nv - i0)) {
      case 1: k_dots<1><<<grid, kDotThreads, 0, st>>>(N, nv, i0, V, vsv, vsr, w, wsr, partial, voff, woff); break;
      case 2: k_dots<2><<<grid, kDotThreads, 0, st>>>(N, nv, i0, V, vsv, vsr, w, wsr, partial, voff, woff); break;
      case 3: k_dots<3><<<grid, kDotThreads, 0, st>>>(N, nv, i0, V, vsv, vsr, w, wsr, partial, voff, woff); break;
      default: k_dots<4><<<grid, kDotThreads, 0, st>>>(N, nv, i0, V, vsv, vsr, w, wsr, partial, voff, woff); break;
    }
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  k_dots_reduce<<<nrhs * nv, 32, 0, st>>>(nrhs * nv, nblk, partial, out);
  return cudaGetLastError();
}

cudaError_t launch_combination(cudaStream_t st, long long N, int nrhs, int nv, const double2 *V,
                               long long vsv, long long vsr, const double2 *coef, int cstride,
                               double sign, double2 *w, long long wsr, bool overwrite,
                               double2 *partial, double2 *nrm2, int nblk, const double *cscale,
                               const long long *voff, const long long *woff) {
  const dim3 grid = nrm2 != nullptr ? dim3((unsigned)nblk, (unsigned)nrhs) : grid_rhs(N, nrhs);
  // groups of at most kCombMaxNv vectors; the norm comes with the last group
  for (int i0 = 0; i0 < nv || i0 == 0; i0 += kCombMaxNv) {
    const int cnt = std::min(kCombMaxNv, nv - i0);
    const bool last = i0 + kCombMaxNv >= nv;
    k_combination<<<grid, 256, 0, st>>>(N, std::max(cnt, 0), V + i0 * vsv, vsv, vsr, coef + i0,
                                        cstride, sign, cscale != nullptr ? cscale + i0 : nullptr,
                                        w, wsr, overwrite && i0 == 0 ? 1 : 0,
                                        nrm2 != nullptr && last ? partial : nullptr, voff, woff);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess || last) break;
  }
  if (nrm2 == nullptr) return cudaGetLastError();
  k_dots_reduce<<<nrhs, 32, 0, st>>>(nrhs, nblk, partial, nrm2);
  return cudaGetLastError();
}

cudaError_t launch_scale_by_norm(cudaStream_t st, long long N, int nrhs, const double2 *in,
                                const double2 *nrm2, double2 *out, const long long *off) {
  k_scale_by_norm<<<grid_rhs(N, nrhs), 256, 0, st>>>(N, in, nrm2, out, off);
  return cudaGetLastError();
}

}  // namespace dds
