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
__global__ void k_apply_A(Geom g, Tables tb, int nrhs, const double2 *__restrict__ u,
                          double2 *__restrict__ Au, int divide_by_J) {
  const long long total = g.Nglob * nrhs;
  for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < total;
       idx += (long long)gridDim.x * blockDim.x) {
    const long long q = idx % g.Nglob;
    const long long base = idx - q;
    int p[3];
    p[0] = (int)(q % g.G[0]);
    p[1] = (int)((q / g.G[0]) % g.G[1]);
    p[2] = g.dim == 3 ? (int)(q / ((long long)g.G[0] * g.G[1])) : 0;
    double2 an[3];
    double2 J = make_double2(1.0, 0.0);
    for (int a = 0; a < g.dim; ++a) {
      an[a] = tb.an_glob64[a][p[a]];
      J = cmul(J, an[a]);
    }
    const double2 uc = u[idx];
    double2 sum = cmul(make_double2(tb.k2_glob[q] * J.x, tb.k2_glob[q] * J.y), uc);
    long long stride = 1;
    for (int a = 0; a < g.dim; ++a) {
      double2 T = make_double2(tb.inv_h2, 0.0);
      for (int b = 0; b < g.dim; ++b)
        if (b != a) T = cmul(T, an[b]);
      const double2 up = (p[a] + 1 < g.G[a]) ? u[idx + stride] : make_double2(0.0, 0.0);
      const double2 um = (p[a] > 0) ? u[idx - stride] : make_double2(0.0, 0.0);
      const double2 fl = cmul(csub(up, uc), tb.iah_glob64[a][p[a] + 1]);
      const double2 bl = cmul(csub(uc, um), tb.iah_glob64[a][p[a]]);
      sum = cadd(sum, cmul(T, csub(fl, bl)));
      stride *= g.G[a];
    }
    if (divide_by_J) sum = cmul(sum, crecip64(J));
    Au[base + q] = sum;
  }
}

__global__ void k_scale_J(Geom g, Tables tb, int nrhs, const double2 *__restrict__ f,
                          double2 *__restrict__ b) {
  const long long total = g.Nglob * nrhs;
  for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < total;
       idx += (long long)gridDim.x * blockDim.x) {
    const long long q = idx % g.Nglob;
    int p[3];
    p[0] = (int)(q % g.G[0]);
    p[1] = (int)((q / g.G[0]) % g.G[1]);
    p[2] = g.dim == 3 ? (int)(q / ((long long)g.G[0] * g.G[1])) : 0;
    double2 J = make_double2(1.0, 0.0);
    for (int a = 0; a < g.dim; ++a) J = cmul(J, tb.an_glob64[a][p[a]]);
    b[idx] = cmul(J, f[idx]);
  }
}

// partial[(rhs * nv + i) * nblk + blk] = sum over the block's chunk of conj(V_i) * w
__global__ void k_dots(long long N, int nv, const double2 *__restrict__ V, long long vsv,
                       long long vsr, const double2 *__restrict__ w, long long wsr,
                       double2 *__restrict__ partial) {
  const int blk = blockIdx.x, nblk = gridDim.x;
  const int rhs = blockIdx.y, i = blockIdx.z;
  const double2 *v = V + i * vsv + rhs * vsr;
  const double2 *ww = w + rhs * wsr;
  double sr = 0.0, si = 0.0;
  for (long long n = blk * (long long)blockDim.x + threadIdx.x; n < N;
       n += (long long)nblk * blockDim.x) {
    const double2 a = v[n], b = ww[n];
    sr = fma(a.x, b.x, sr);
    sr = fma(a.y, b.y, sr);
    si = fma(a.x, b.y, si);
    si = fma(-a.y, b.x, si);
  }
  __shared__ double red[2][32];
  for (int o = 16; o > 0; o >>= 1) {
    sr += __shfl_down_sync(0xffffffffu, sr, o);
    si += __shfl_down_sync(0xffffffffu, si, o);
  }
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (lane == 0) { red[0][warp] = sr; red[1][warp] = si; }
  __syncthreads();
  if (warp == 0) {
    const int nw = blockDim.x >> 5;
    sr = lane < nw ? red[0][lane] : 0.0;
    si = lane < nw ? red[1][lane] : 0.0;
    for (int o = 16; o > 0; o >>= 1) {
      sr += __shfl_down_sync(0xffffffffu, sr, o);
      si += __shfl_down_sync(0xffffffffu, si, o);
    }
    if (lane == 0) partial[((long long)rhs * nv + i) * nblk + blk] = make_double2(sr, si);
  }
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

// w[rhs] += sign * sum_i V_i[rhs] * coef[rhs * nv + i]
__global__ void k_sub_combination(long long N, int nrhs, int nv, const double2 *__restrict__ V,
                                  long long vsv, long long vsr, const double2 *__restrict__ coef,
                                  double2 *__restrict__ w, long long wsr, double sign) {
  const long long total = N * nrhs;
  for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < total;
       idx += (long long)gridDim.x * blockDim.x) {
    const int rhs = (int)(idx / N);
    const long long n = idx % N;
    double2 acc = make_double2(0.0, 0.0);
    for (int i = 0; i < nv; ++i) cfma(acc, V[i * vsv + rhs * vsr + n], coef[(long long)rhs * nv + i]);
    double2 *dst = w + rhs * wsr + n;
    dst->x += sign * acc.x;
    dst->y += sign * acc.y;
  }
}

__global__ void k_scale_vec(long long N, int nrhs, const double2 *__restrict__ in,
                            const double *__restrict__ inv_scale, double2 *__restrict__ out) {
  const long long total = N * nrhs;
  for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < total;
       idx += (long long)gridDim.x * blockDim.x) {
    const double s = inv_scale[idx / N];
    out[idx] = make_double2(in[idx].x * s, in[idx].y * s);
  }
}

static inline unsigned grid_for(long long n) {
  long long b = (n + 255) / 256;
  return (unsigned)(b < 152 * 16 ? (b < 1 ? 1 : b) : 152 * 16);
}

cudaError_t launch_apply_A(cudaStream_t st, const Geom &g, const Tables &tb, int nrhs,
                           const double2 *u, double2 *Au, int divide_by_J) {
  k_apply_A<<<grid_for(g.Nglob * nrhs), 256, 0, st>>>(g, tb, nrhs, u, Au, divide_by_J);
  return cudaGetLastError();
}

cudaError_t launch_scale_J(cudaStream_t st, const Geom &g, const Tables &tb, int nrhs,
                           const double2 *f, double2 *b) {
  k_scale_J<<<grid_for(g.Nglob * nrhs), 256, 0, st>>>(g, tb, nrhs, f, b);
  return cudaGetLastError();
}

cudaError_t launch_dots(cudaStream_t st, long long N, int nrhs, int nv, const double2 *V,
                        long long vsv, long long vsr, const double2 *w, long long wsr,
                        double2 *partial, double2 *out, int nblk) {
  dim3 grid(nblk, nrhs, nv);
  k_dots<<<grid, 256, 0, st>>>(N, nv, V, vsv, vsr, w, wsr, partial);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  k_dots_reduce<<<nrhs * nv, 32, 0, st>>>(nrhs * nv, nblk, partial, out);
  return cudaGetLastError();
}

cudaError_t launch_sub_combination(cudaStream_t st, long long N, int nrhs, int nv,
                                   const double2 *V, long long vsv, long long vsr,
                                   const double2 *coef, double2 *w, long long wsr, double sign) {
  k_sub_combination<<<grid_for(N * nrhs), 256, 0, st>>>(N, nrhs, nv, V, vsv, vsr, coef, w, wsr,
                                                        sign);
  return cudaGetLastError();
}

cudaError_t launch_scale_vec(cudaStream_t st, long long N, int nrhs, const double2 *in,
                             const double *inv_scale, double2 *out) {
  k_scale_vec<<<grid_for(N * nrhs), 256, 0, st>>>(N, nrhs, in, inv_scale, out);
  return cudaGetLastError();
}

}  // namespace dds
