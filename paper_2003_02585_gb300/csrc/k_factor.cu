// Block-tridiagonal LU of an extended subdomain operator, FP64 (set-up, once per distinct
// operator).  With the unknowns ordered in blocks along the last axis,
//   A = tridiag(C_{j-1}, D_j, C_j),   C_j = diag(cpl_j),
//   S_0 = D_0,   S_j = D_j - C_{j-1} S_{j-1}^{-1} C_{j-1},
// and the substitutions only need S_j^{-1}, which is formed explicitly.  One CTA walks the
// whole Schur chain of one operator with S_j held in shared memory: the Schur update reads
// S_{j-1}^{-1} in place, then S_j is inverted in place by Gauss-Jordan elimination with partial
// (row) pivoting and a final column unscramble.
#include "dds_internal.cuh"

namespace dds {

__device__ inline double2 crecip(double2 z) {
  const double m = z.x * z.x + z.y * z.y;
  return make_double2(z.x / m, -z.y / m);
}

// One chain of the factorisation per CTA (factor f = blockIdx.x), over `count` blocks starting
// at j0 in direction dir:
//   dir = +1 (from the top):    S_j = D_j - C_{j-1} S_{j-1}^{-1} C_{j-1}
//   dir = -1 (from the bottom): T_j = D_j - C_j T_{j+1}^{-1} C_j
// The previous block's inverse is either the chain's own last result (in shared memory) or, for
// the first block when prev_inv is given, tile j0 - dir of prev_inv.  When extra_inv is given,
// the last block of the chain also subtracts C_j X C_j with X = tile j + 1 of extra_inv (the
// middle block of the two-sided factorisation: Z_m = D_m - C_{m-1} S_{m-1}^{-1} C_{m-1}
// - C_m T_{m+1}^{-1} C_m).  Each inverse is stored as [s][r] at tile j of out64 (and out32).
__global__ void __launch_bounds__(1024) k_factor(int Mb, int Ml, long long St, int M0,
                                                 const double2 *__restrict__ dg,
                                                 const double2 *__restrict__ offx,
                                                 const double2 *__restrict__ offy,
                                                 const double2 *__restrict__ cpl,
                                                 double2 *__restrict__ sinv64,
                                                 float2 *__restrict__ sinv32,
                                                 int *__restrict__ status, int j0, int count,
                                                 int dir, const double2 *__restrict__ prev_inv,
                                                 const double2 *__restrict__ extra_inv) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  double2 *S = reinterpret_cast<double2 *>(smem_raw);      // [Mb][Mb] row-major
  double2 *colk = S + (size_t)Mb * Mb;                       // [Mb]
  int *piv = reinterpret_cast<int *>(colk + Mb);             // [Mb]
  const int f = blockIdx.x;
  const int tid = threadIdx.x, nt = blockDim.x;
  const int lane = tid & 31, warp = tid >> 5;
  const long long fb = (long long)f * Ml * Mb;
  const long long MbMb = (long long)Mb * Mb;
  if (prev_inv != nullptr) {
    const long long pb = ((long long)f * Ml + (j0 - dir)) * St;
    for (long long idx = tid; idx < MbMb; idx += nt) {
      const int r = (int)(idx / Mb), s = (int)(idx % Mb);
      S[idx] = prev_inv[pb + (long long)s * Mb + r];
    }
    __syncthreads();
  }

  for (int jj = 0; jj < count; ++jj) {
    const int j = j0 + dir * jj;
    const bool has_prev = jj > 0 || prev_inv != nullptr;
    // coupling between block j and the previous block of the chain
    const int jc = dir > 0 ? j - 1 : j;
    const bool extra = extra_inv != nullptr && jj == count - 1;
    const long long xb = ((long long)f * Ml + (j + 1)) * St;
    // ---- S_j = D_j - C S_prev^{-1} C  (- C_j X C_j for the middle block)
    for (long long idx = tid; idx < MbMb; idx += nt) {
      const int r = (int)(idx / Mb), s = (int)(idx % Mb);
      double2 val = make_double2(0.0, 0.0);
      if (has_prev) {
        const double2 cr = cpl[fb + (long long)jc * Mb + r];
        const double2 cs = cpl[fb + (long long)jc * Mb + s];
        val = cmul(cmul(cr, S[idx]), cs);
        val.x = -val.x;
        val.y = -val.y;
      }
      if (extra) {
        const double2 cr = cpl[fb + (long long)j * Mb + r];
        const double2 cs = cpl[fb + (long long)j * Mb + s];
        const double2 t = cmul(cmul(cr, extra_inv[xb + (long long)s * Mb + r]), cs);
        val.x -= t.x;
        val.y -= t.y;
      }
      const long long lb = fb + (long long)j * Mb;
      if (r == s) val = cadd(val, dg[lb + r]);
      else if (s == r + 1) val = cadd(val, offx[lb + r]);
      else if (r == s + 1) val = cadd(val, offx[lb + s]);
      if (offy != nullptr) {
        if (s == r + M0) val = cadd(val, offy[lb + r]);
        else if (r == s + M0) val = cadd(val, offy[lb + s]);
      }
      S[idx] = val;
    }
    __syncthreads();
    // ---- in-place Gauss-Jordan inversion with partial pivoting
    for (int k = 0; k < Mb; ++k) {
      if (warp == 0) {
        double best = -1.0;
        int bi = k;
        for (int r = k + lane; r < Mb; r += 32) {
          const double2 z = S[(long long)r * Mb + k];
          const double m = z.x * z.x + z.y * z.y;
          if (m > best) { best = m; bi = r; }
        }
        for (int o = 16; o > 0; o >>= 1) {
          const double ob = __shfl_down_sync(0xffffffffu, best, o);
          const int oi = __shfl_down_sync(0xffffffffu, bi, o);
          if (ob > best || (ob == best && oi < bi)) { best = ob; bi = oi; }
        }
        if (lane == 0) {
          piv[k] = bi;
          if (!(best > 0.0)) atomicExch(status, 1);
        }
      }
      __syncthreads();
      const int p = piv[k];
      if (p != k) {
        for (int s = tid; s < Mb; s += nt) {
          const double2 t = S[(long long)k * Mb + s];
          S[(long long)k * Mb + s] = S[(long long)p * Mb + s];
          S[(long long)p * Mb + s] = t;
        }
        __syncthreads();
      }
      const double2 pinv = crecip(S[(long long)k * Mb + k]);
      __syncthreads();
      for (int s = tid; s < Mb; s += nt) {
        const double2 v = S[(long long)k * Mb + s];
        S[(long long)k * Mb + s] = (s == k) ? pinv : cmul(v, pinv);
      }
      for (int r = tid; r < Mb; r += nt) colk[r] = (r == k) ? make_double2(0.0, 0.0) : S[(long long)r * Mb + k];
      __syncthreads();
      for (long long idx = tid; idx < MbMb; idx += nt) {
        const int r = (int)(idx / Mb), s = (int)(idx % Mb);
        if (r == k) continue;
        double2 v = (s == k) ? make_double2(0.0, 0.0) : S[idx];
        const double2 prod = cmul(colk[r], S[(long long)k * Mb + s]);
        v.x -= prod.x;
        v.y -= prod.y;
        S[idx] = v;
      }
      __syncthreads();
    }
    for (int k = Mb - 1; k >= 0; --k) {
      const int p = piv[k];
      if (p != k) {
        for (int r = tid; r < Mb; r += nt) {
          const double2 t = S[(long long)r * Mb + k];
          S[(long long)r * Mb + k] = S[(long long)r * Mb + p];
          S[(long long)r * Mb + p] = t;
        }
      }
      __syncthreads();
    }
    // ---- store S_j^{-1} as [s][r] (thread r of a substitution reads along r)
    const long long ob = ((long long)f * Ml + j) * St;
    for (long long idx = tid; idx < MbMb; idx += nt) {
      const int s = (int)(idx / Mb), r = (int)(idx % Mb);
      const double2 v = S[(long long)r * Mb + s];
      sinv64[ob + idx] = v;
      if (sinv32 != nullptr) sinv32[ob + idx] = make_float2((float)v.x, (float)v.y);
    }
    __syncthreads();
  }
}

static size_t factor_smem(int Mb) {
  return (size_t)Mb * Mb * sizeof(double2) + Mb * sizeof(double2) + Mb * sizeof(int);
}

cudaError_t launch_factor(cudaStream_t st, int nfac, int Mb, int Ml, long long St, int M0,
                          const double2 *dg,
                          const double2 *offx, const double2 *offy, const double2 *cpl,
                          double2 *sinv64, float2 *sinv32, int *status) {
  const size_t smem = factor_smem(Mb);
  cudaError_t e = cudaFuncSetAttribute(k_factor, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)smem);
  if (e != cudaSuccess) return e;
  k_factor<<<nfac, 1024, smem, st>>>(Mb, Ml, St, M0, dg, offx, offy, cpl, sinv64, sinv32, status,
                                     0, Ml, 1, nullptr, nullptr);
  return cudaGetLastError();
}

// The blocks m..Ml-1 of the two-sided factorisation, given the top chain S_j^{-1} (sinv64):
// T_j^{-1} for j = Ml-1 down to m+1, then Z_m^{-1}; written as tiles m..Ml-1 of tw64.
cudaError_t launch_factor_twisted(cudaStream_t st, int nfac, int Mb, int Ml, long long St, int M0,
                                  int m, const double2 *dg, const double2 *offx,
                                  const double2 *offy, const double2 *cpl,
                                  const double2 *sinv64, double2 *tw64, int *status) {
  if (m < 1 || m > Ml - 2) return cudaErrorInvalidValue;
  const size_t smem = factor_smem(Mb);
  cudaError_t e = cudaFuncSetAttribute(k_factor, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)smem);
  if (e != cudaSuccess) return e;
  k_factor<<<nfac, 1024, smem, st>>>(Mb, Ml, St, M0, dg, offx, offy, cpl, tw64, nullptr, status,
                                     Ml - 1, Ml - 1 - m, -1, nullptr, nullptr);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  k_factor<<<nfac, 1024, smem, st>>>(Mb, Ml, St, M0, dg, offx, offy, cpl, tw64, nullptr, status,
                                     m, 1, 1, sinv64, tw64);
  return cudaGetLastError();
}

__global__ void k_convert(const double2 *__restrict__ in, float2 *__restrict__ out, long long n) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x)
    out[i] = make_float2((float)in[i].x, (float)in[i].y);
}

cudaError_t launch_convert_c64_c32(cudaStream_t st, const double2 *in, float2 *out, long long n) {
  if (n <= 0) return cudaSuccess;
  k_convert<<<1024, 256, 0, st>>>(in, out, n);
  return cudaGetLastError();
}

}  // namespace dds

// ------------------------------------------------------------------------------------------
// Large blocks (Mb too big for shared memory): the same Schur chain and Gauss-Jordan inversion
// with partial pivoting, in global memory.  S holds S_j (row-major, [r][s]); per pivot k one
// single-CTA kernel finds the pivot, swaps rows, scales the pivot row and saves column k, and
// a grid-wide kernel applies the rank-1 update to every other row.
// ------------------------------------------------------------------------------------------
namespace dds {

// S (holding S_{j-1}^{-1}, or anything if j == 0)  ->  S_j = D_j - C_{j-1} S_{j-1}^{-1} C_{j-1}
__global__ void k_big_schur(int Mb, int M0, int j, const double2 *__restrict__ dg,
                            const double2 *__restrict__ offx, const double2 *__restrict__ offy,
                            const double2 *__restrict__ cpl, double2 *__restrict__ S) {
  const long long n2 = (long long)Mb * Mb;
  for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < n2;
       idx += (long long)gridDim.x * blockDim.x) {
    const int r = (int)(idx / Mb), s = (int)(idx % Mb);
    double2 val = make_double2(0.0, 0.0);
    if (j > 0) {
      const double2 cr = cpl[(long long)(j - 1) * Mb + r];
      const double2 cs = cpl[(long long)(j - 1) * Mb + s];
      val = cmul(cmul(cr, S[idx]), cs);
      val.x = -val.x;
      val.y = -val.y;
    }
    const long long lb = (long long)j * Mb;
    if (r == s) val = cadd(val, dg[lb + r]);
    else if (s == r + 1) val = cadd(val, offx[lb + r]);
    else if (r == s + 1) val = cadd(val, offx[lb + s]);
    if (offy != nullptr) {
      if (s == r + M0) val = cadd(val, offy[lb + r]);
      else if (r == s + M0) val = cadd(val, offy[lb + s]);
    }
    S[idx] = val;
  }
}

__global__ void __launch_bounds__(1024) k_big_pivot(int Mb, int k, double2 *__restrict__ S,
                                                    double2 *__restrict__ colk,
                                                    int *__restrict__ piv,
                                                    int *__restrict__ status) {
  __shared__ double bestv[32];
  __shared__ int besti[32];
  __shared__ int p_sh;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  double best = -1.0;
  int bi = k;
  for (int r = k + tid; r < Mb; r += blockDim.x) {
    const double2 z = S[(long long)r * Mb + k];
    const double m = z.x * z.x + z.y * z.y;
    if (m > best) { best = m; bi = r; }
  }
  for (int o = 16; o > 0; o >>= 1) {
    const double ob = __shfl_down_sync(0xffffffffu, best, o);
    const int oi = __shfl_down_sync(0xffffffffu, bi, o);
    if (ob > best || (ob == best && oi < bi)) { best = ob; bi = oi; }
  }
  if (lane == 0) { bestv[warp] = best; besti[warp] = bi; }
  __syncthreads();
  if (tid == 0) {
    double b = -1.0;
    int i = k;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w)
      if (bestv[w] > b || (bestv[w] == b && besti[w] < i)) { b = bestv[w]; i = besti[w]; }
    p_sh = i;
    piv[k] = i;
    if (!(b > 0.0)) atomicExch(status, 1);
  }
  __syncthreads();
  const int p = p_sh;
  if (p != k)
    for (int s = tid; s < Mb; s += blockDim.x) {
      const double2 t = S[(long long)k * Mb + s];
      S[(long long)k * Mb + s] = S[(long long)p * Mb + s];
      S[(long long)p * Mb + s] = t;
    }
  __syncthreads();
  const double2 pinv = crecip(S[(long long)k * Mb + k]);
  __syncthreads();
  for (int s = tid; s < Mb; s += blockDim.x) {
    const double2 v = S[(long long)k * Mb + s];
    S[(long long)k * Mb + s] = (s == k) ? pinv : cmul(v, pinv);
  }
  for (int r = tid; r < Mb; r += blockDim.x)
    colk[r] = (r == k) ? make_double2(0.0, 0.0) : S[(long long)r * Mb + k];
}

__global__ void k_big_update(int Mb, int k, double2 *__restrict__ S,
                             const double2 *__restrict__ colk) {
  const long long n2 = (long long)Mb * Mb;
  for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < n2;
       idx += (long long)gridDim.x * blockDim.x) {
    const int r = (int)(idx / Mb), s = (int)(idx % Mb);
    if (r == k) continue;
    double2 v = (s == k) ? make_double2(0.0, 0.0) : S[idx];
    const double2 prod = cmul(colk[r], S[(long long)k * Mb + s]);
    v.x -= prod.x;
    v.y -= prod.y;
    S[idx] = v;
  }
}

// undo the row pivoting on the inverse: swap columns k and piv[k] for k = Mb-1 .. 0
__global__ void k_big_unscramble(int Mb, double2 *__restrict__ S, const int *__restrict__ piv) {
  for (int r = blockIdx.x * blockDim.x + threadIdx.x; r < Mb; r += gridDim.x * blockDim.x) {
    double2 *row = S + (long long)r * Mb;
    for (int k = Mb - 1; k >= 0; --k) {
      const int p = piv[k];
      if (p != k) {
        const double2 t = row[k];
        row[k] = row[p];
        row[p] = t;
      }
    }
  }
}

// store S_j^{-1} as [s][r] in both precisions
__global__ void k_big_store(int Mb, const double2 *__restrict__ S, double2 *__restrict__ out64,
                            float2 *__restrict__ out32) {
  const long long n2 = (long long)Mb * Mb;
  for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < n2;
       idx += (long long)gridDim.x * blockDim.x) {
    const int s = (int)(idx / Mb), r = (int)(idx % Mb);
    const double2 v = S[(long long)r * Mb + s];
    out64[idx] = v;
    out32[idx] = make_float2((float)v.x, (float)v.y);
  }
}

static unsigned big_grid(long long n2) {
  const long long b = (n2 + 255) / 256;
  return (unsigned)(b < 152 * 32 ? b : 152 * 32);
}

cudaError_t launch_factor_big(cudaStream_t st, int f, int Mb, int Ml, long long St, int M0,
                              const double2 *dg, const double2 *offx, const double2 *offy,
                              const double2 *cpl, double2 *S, double2 *colk, int *piv,
                              double2 *sinv64, float2 *sinv32, int *status,
                              long long *launches) {
  const long long n2 = (long long)Mb * Mb;
  const long long fb = (long long)f * Ml * Mb;
  for (int j = 0; j < Ml; ++j) {
    k_big_schur<<<big_grid(n2), 256, 0, st>>>(Mb, M0, j, dg + fb, offx + fb,
                                               offy ? offy + fb : nullptr, cpl + fb, S);
    ++*launches;
    for (int k = 0; k < Mb; ++k) {
      k_big_pivot<<<1, 1024, 0, st>>>(Mb, k, S, colk, piv, status);
      k_big_update<<<big_grid(n2), 256, 0, st>>>(Mb, k, S, colk);
      *launches += 2;
    }
    k_big_unscramble<<<(Mb + 127) / 128, 128, 0, st>>>(Mb, S, piv);
    const long long ob = ((long long)f * Ml + j) * St;
    k_big_store<<<big_grid(n2), 256, 0, st>>>(Mb, S, sinv64 + ob, sinv32 + ob);
    *launches += 2;
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

}  // namespace dds
