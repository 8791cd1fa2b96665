// Block-tridiagonal substitutions, complex FP32, with the block inverses streamed through shared
// memory.  Same arithmetic as k_subst in k_sweep.cu:
//   forward  y_0 = S_0^{-1} b_0,  y_j = S_j^{-1} (b_j - C_{j-1} y_{j-1})
//   backward x_{Ml-1} = y_{Ml-1}, x_j = y_j - S_j^{-1} (C_j x_{j+1})
// One CTA (256 threads) runs the whole 2 Ml - 1 stage chain of one panel of right-hand sides.
// Stage q needs the Mb x Mb tile S_{j(q)}^{-1}; tiles are fetched by one-shot bulk copies into a
// two-slot shared-memory ring completed on mbarriers, so the tile of stage q + 2 is in flight
// while stage q computes.  Thread (r, half) accumulates row r over half of the K range; the two
// halves are summed through shared memory.  The operands of the stage epilogue (b_{j+1} or y_j
// and the coupling) are loaded before the K loop so their latency hides behind it.
#include "async_copy.cuh"
#include "dds_internal.cuh"

namespace dds {

template <int PC>
__global__ void __launch_bounds__(256, 1) k_subst_stream(Geom g, const Panel *__restrict__ panels,
                                                         const Col *__restrict__ cols,
                                                         const float2 *__restrict__ sinv,
                                                         const float2 *__restrict__ cpl,
                                                         float2 *__restrict__ work,
                                                         int *__restrict__ err) {
  extern __shared__ __align__(128) unsigned char smem_raw[];
  const int Mb = g.Mb, Ml = g.Ml;
  const long long St = g.St;
  float2 *tiles = reinterpret_cast<float2 *>(smem_raw);   // [2][St]
  float2 *vbuf = tiles + 2 * St;                          // [2][Mb][PC]
  float2 *red = vbuf + 2 * Mb * PC;                       // [Mb][PC]
  uint64_t *bars = reinterpret_cast<uint64_t *>(red + Mb * PC);
  const Panel p = panels[blockIdx.x];
  if (p.ncol == 0) return;   // an empty panel of a compacted list (zero-work skipping)
  const float2 *Sf = sinv + (long long)p.factor * Ml * St;
  const float2 *cf = cpl + (long long)p.factor * Ml * (long long)Mb;
  const int tid = threadIdx.x;
  const int r = tid & 127, half = tid >> 7;
  const int nst = 2 * Ml - 1;
  const uint32_t tile_bytes = (uint32_t)(St * sizeof(float2));
  float2 *xs[PC];
#pragma unroll
  for (int c = 0; c < PC; ++c)
    xs[c] = c < p.ncol ? work + (long long)cols[p.col0 + c].slot * g.Nloc : nullptr;
  auto block_of = [&](int q) { return q < Ml ? q : 2 * Ml - 2 - q; };

  if (tid == 0) {
    mbar_init(&bars[0], 1);
    mbar_init(&bars[1], 1);
    mbar_init_fence();
  }
  __syncthreads();
  if (tid == 0) {
    for (int q = 0; q < 2 && q < nst; ++q) {
      mbar_arrive_expect_tx(&bars[q], tile_bytes);
      bulk_g2s(tiles + q * St, Sf + (long long)block_of(q) * St, tile_bytes, &bars[q]);
    }
  }
  for (int idx = tid; idx < Mb * PC; idx += blockDim.x) {
    const int rr = idx / PC, c = idx % PC;
    vbuf[idx] = c < p.ncol ? work[(long long)cols[p.col0 + c].slot * g.Nloc + rr]
                           : make_float2(0.f, 0.f);
  }
  __syncthreads();

  const int kh = (Mb + 1) / 2;
  const int k0 = half * kh, k1 = min(Mb, k0 + kh);
  const bool row = r < Mb;
  for (int q = 0; q < nst; ++q) {
    const int j = block_of(q);
    const bool fwd = q < Ml;
    const int buf = q & 1;
    const float2 *T = tiles + buf * St;
    const float2 *vin = vbuf + buf * Mb * PC;
    float2 *vout = vbuf + (buf ^ 1) * Mb * PC;
    // epilogue operands, loaded early
    float2 pre[PC];
    float2 cn = make_float2(0.f, 0.f);
#pragma unroll
    for (int c = 0; c < PC; ++c) pre[c] = make_float2(0.f, 0.f);
    if (half == 0 && row) {
      if (fwd) {
        if (j + 1 < Ml) {
#pragma unroll
          for (int c = 0; c < PC; ++c)
            if (c < p.ncol) pre[c] = xs[c][(long long)(j + 1) * Mb + r];
          cn = cf[(long long)j * Mb + r];
        } else if (Ml >= 2) {
          cn = cf[(long long)(Ml - 2) * Mb + r];
        }
      } else {
#pragma unroll
        for (int c = 0; c < PC; ++c)
          if (c < p.ncol) pre[c] = xs[c][(long long)j * Mb + r];
        if (j > 0) cn = cf[(long long)(j - 1) * Mb + r];
      }
    }
    const bool ok = mbar_wait(&bars[buf], (q >> 1) & 1);
    float2 acc[PC];
#pragma unroll
    for (int c = 0; c < PC; ++c) acc[c] = make_float2(0.f, 0.f);
    if (row) {
#pragma unroll 4
      for (int s = k0; s < k1; ++s) {
        const float2 a = T[s * Mb + r];
        const float2 *vv = vin + s * PC;
#pragma unroll
        for (int c = 0; c < PC; ++c) cfma(acc[c], a, vv[c]);
      }
      if (half == 1) {
#pragma unroll
        for (int c = 0; c < PC; ++c) red[r * PC + c] = acc[c];
      }
    }
    if (__syncthreads_or(!ok)) {
      // a tile never arrived: report, let the copies still in flight land, and leave
      if (tid == 0) {
        atomicExch(err, 2);
        mbar_wait(&bars[buf], (q >> 1) & 1);
        if (q + 1 < nst) mbar_wait(&bars[buf ^ 1], ((q + 1) >> 1) & 1);
      }
      __syncthreads();
      return;
    }
    if (tid == 0 && q + 2 < nst) {
      fence_proxy_async();
      mbar_arrive_expect_tx(&bars[buf], tile_bytes);
      bulk_g2s(tiles + buf * St, Sf + (long long)block_of(q + 2) * St, tile_bytes, &bars[buf]);
    }
    if (half == 0 && row) {
#pragma unroll
      for (int c = 0; c < PC; ++c) acc[c] = cadd(acc[c], red[r * PC + c]);
      if (fwd) {
#pragma unroll
        for (int c = 0; c < PC; ++c) {
          if (c < p.ncol) xs[c][(long long)j * Mb + r] = acc[c];
          vout[r * PC + c] = (j + 1 < Ml) ? csub(pre[c], cmul(cn, acc[c])) : cmul(cn, acc[c]);
        }
      } else {
#pragma unroll
        for (int c = 0; c < PC; ++c) {
          const float2 xv = csub(pre[c], acc[c]);
          if (c < p.ncol) xs[c][(long long)j * Mb + r] = xv;
          vout[r * PC + c] = cmul(cn, xv);
        }
      }
    }
    __syncthreads();
  }
}

size_t subst_stream_smem(const Geom &g, int pc) {
  return (size_t)(2 * g.St + 3 * (long long)g.Mb * pc) * sizeof(float2) + 2 * sizeof(uint64_t);
}

bool subst_stream_ok(const Geom &g, int pc) {
  return g.Mb <= 128 && subst_stream_smem(g, pc) <= 227 * 1024;
}

template <int PC>
static cudaError_t stream_pc(cudaStream_t st, const Geom &g, int npanels, const Panel *panels,
                             const Col *cols, const float2 *sinv, const float2 *cpl,
                             float2 *work, int *err) {
  const size_t smem = subst_stream_smem(g, PC);
  static bool done[64] = {false};
  cudaError_t e = smem_limit_once(k_subst_stream<PC>, done);
  if (e != cudaSuccess) return e;
  k_subst_stream<PC><<<npanels, 256, smem, st>>>(g, panels, cols, sinv, cpl, work, err);
  return cudaGetLastError();
}

cudaError_t launch_subst_stream(cudaStream_t st, const Geom &g, int npanels, const Panel *panels,
                                const Col *cols, const float2 *sinv, const float2 *cpl,
                                float2 *work, int pc, int *err) {
  if (npanels <= 0) return cudaSuccess;
  switch (pc) {
    case 1: return stream_pc<1>(st, g, npanels, panels, cols, sinv, cpl, work, err);
    case 2: return stream_pc<2>(st, g, npanels, panels, cols, sinv, cpl, work, err);
    case 4: return stream_pc<4>(st, g, npanels, panels, cols, sinv, cpl, work, err);
    case 8: return stream_pc<8>(st, g, npanels, panels, cols, sinv, cpl, work, err);
    case 16: return stream_pc<16>(st, g, npanels, panels, cols, sinv, cpl, work, err);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace dds
