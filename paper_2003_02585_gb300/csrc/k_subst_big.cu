// Block substitutions for line/plane blocks too wide for one CTA (Mb > 128, the 3D plane blocks),
// stage-parallel on the tensor cores.  Same recurrences as the other substitution kernels:
//   forward  y_0 = S_0^{-1} b_0,  y_j = S_j^{-1} (b_j - C_{j-1} y_{j-1})
//   backward x_{Ml-1} = y_{Ml-1}, x_j = y_j - S_j^{-1} (C_j x_{j+1})
// Each of the 2 Ml - 1 stages is one GEMM over all columns of the launch, S_j^{-1} V (Mb x Mb
// times Mb x columns), spread over the whole GPU:
//   k_big_mma  one CTA per unit (128-row tile of S_j^{-1}, panel of PC columns, K segment; the
//              panels of one tile segment adjacent in the grid, so they share its reads in L2):
//              the unit's pre-split A tiles and the matching B pieces stream through a two-slot
//              shared-memory ring (bulk copies on mbarriers); four tcgen05.mma per K-step into
//              two TMEM accumulators (split products, as in k_subst_tc.cu); the unit's partial
//              product is added into an FP32 accumulator with 8-byte vector atomics;
//   k_big_epi  per (panel, row, column): y_j or x_j from the accumulator, stored; the next
//              stage's right-hand side formed and written as B pieces; the accumulator cleared.
// Both launches of every stage are captured in the DDM application's CUDA graph.
#include "async_copy.cuh"
#include "dds_internal.cuh"
#include "umma.cuh"

namespace dds {

// ---- layouts --------------------------------------------------------------------------------
// A (per factor f, block j): [row tile rt][K-step t][comp][g][128 rows][16 bytes]; components
// 0/1 = pieces 0/1 of Re S_j^{-1}, 2/3 of Im; K-step t covers columns 2 EK t .. 2 EK t + 2 EK - 1.
// B (per panel, one stage): [K-step t][g][4 PC rows][16 bytes]; rows [piece0 re | piece0 im |
// piece1 re | piece1 im], PC each.
struct BigShape {
  int kind, EK, RT, KT, PC, KSPLIT, KTU;   // KTU = K-steps per unit
  long long a_tile;                         // bytes of one (f, j) tile
  size_t smem;
  int KS;                                   // K-steps per ring chunk
};

static inline int big_ek(int kind) { return kind == 0 ? 4 : 8; }

bool big_shape(const Geom &g, int kind, int pc, int ksplit, BigShape *s) {
  BigShape t;
  t.kind = kind;
  t.EK = big_ek(kind);
  t.PC = pc;
  if (pc != 8 && pc != 16 && pc != 32) return false;
  t.RT = (g.Mb + 127) / 128;
  const int kstep = 2 * t.EK;
  t.KT = (g.Mb + kstep - 1) / kstep;
  t.KSPLIT = std::max(1, std::min(ksplit, t.KT));
  t.KTU = (t.KT + t.KSPLIT - 1) / t.KSPLIT;
  t.KSPLIT = (t.KT + t.KTU - 1) / t.KTU;
  t.a_tile = (long long)t.RT * t.KT * 128 * 128;   // 128 rows x 16 B x 8 (comp, g) per K-step
  const size_t per_step = 16384 + (size_t)128 * pc;   // A + B bytes of one K-step
  const size_t budget = 227 * 1024 - 2048;
  t.KS = 8;
  while (t.KS > 1 && 2 * per_step * t.KS + 2048 > budget) --t.KS;
  t.smem = 2 * per_step * t.KS + 2048;
  if (s) *s = t;
  return g.Mb > 128;
}

long long big_tiles_bytes(const Geom &g, int kind, int nfac) {
  BigShape t;
  big_shape(g, kind, 8, 1, &t);
  return (long long)nfac * g.Ml * t.a_tile;
}

template <int KIND>
__global__ void k_split_big(const double2 *__restrict__ sinv, unsigned char *__restrict__ out,
                            int nfac, int Mb, int Ml, long long St, int RT, int KT) {
  constexpr int EK = KIND == 0 ? 4 : 8, ES = 16 / EK;
  const long long rows = (long long)RT * 128, kcols = (long long)KT * 2 * EK;
  const long long total = (long long)nfac * Ml * rows * kcols;
  const long long tile = (long long)RT * KT * 128 * 128;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
       i += (long long)gridDim.x * blockDim.x) {
    const int m = (int)(i % rows);
    const int k = (int)((i / rows) % kcols);
    const long long fj = i / (rows * kcols);
    double2 a = make_double2(0.0, 0.0);
    if (m < Mb && k < Mb) a = sinv[fj * St + (long long)k * Mb + m];
    const int rt = m >> 7, mr = m & 127;
    const int t = k / (2 * EK), gg = (k / EK) & 1;
    unsigned char *base = out + fj * tile + ((long long)rt * KT + t) * 16384 + mr * 16 + (k % EK) * ES;
    const double parts[2] = {a.x, a.y};
#pragma unroll
    for (int e = 0; e < 2; ++e) {
      const double x = parts[e];
      unsigned char *p0 = base + ((2 * e + 0) * 2 + gg) * 2048;
      unsigned char *p1 = base + ((2 * e + 1) * 2 + gg) * 2048;
      if (KIND == 0) {
        const float x0 = umma::tf32_rna((float)x);
        const float x1 = umma::tf32_rna((float)(x - (double)x0));
        *reinterpret_cast<float *>(p0) = x0;
        *reinterpret_cast<float *>(p1) = x1;
      } else {
        const unsigned short b0 = umma::bf16_rn_bits((float)x);
        const unsigned short b1 = umma::bf16_rn_bits((float)(x - (double)umma::bf16_to_float(b0)));
        *reinterpret_cast<unsigned short *>(p0) = b0;
        *reinterpret_cast<unsigned short *>(p1) = b1;
      }
    }
  }
}

cudaError_t launch_split_big(cudaStream_t st, const Geom &g, int kind, int nfac,
                             const double2 *sinv64, unsigned char *tiles) {
  BigShape t;
  if (!big_shape(g, kind, 8, 1, &t)) return cudaErrorInvalidValue;
  const long long total = (long long)nfac * g.Ml * t.RT * 128 * (long long)t.KT * 2 * t.EK;
  const int blocks = (int)std::min<long long>((total + 255) / 256, 152LL * 32);
  if (kind == 0)
    k_split_big<0><<<blocks, 256, 0, st>>>(sinv64, tiles, nfac, g.Mb, g.Ml, g.St, t.RT, t.KT);
  else
    k_split_big<1><<<blocks, 256, 0, st>>>(sinv64, tiles, nfac, g.Mb, g.Ml, g.St, t.RT, t.KT);
  return cudaGetLastError();
}

// ---- split pieces of one value (round to nearest, ties away, on the bit pattern) -------------
__device__ __forceinline__ float big_round_tf32(float x) {
  return __uint_as_float((__float_as_uint(x) + 0x1000u) & 0xFFFFE000u);
}
__device__ __forceinline__ unsigned short big_round_bf16(float x) {
  return (unsigned short)((__float_as_uint(x) + 0x8000u) >> 16);
}

// write the pieces of v for (row k, column c) of a panel's B operand of one stage
template <int KIND>
__device__ __forceinline__ void big_put_b(unsigned char *Bp, int PC, int k, int c, float2 v) {
  constexpr int EK = KIND == 0 ? 4 : 8, ES = 16 / EK;
  const int t = k / (2 * EK), gg = (k / EK) & 1;
  unsigned char *base = Bp + (long long)t * 128 * PC + (long long)gg * 64 * PC + (k % EK) * ES;
  const int n[4] = {c, PC + c, 2 * PC + c, 3 * PC + c};
  if (KIND == 0) {
    float w[4];
    w[0] = big_round_tf32(v.x);
    w[1] = big_round_tf32(v.y);
    w[2] = big_round_tf32(v.x - w[0]);
    w[3] = big_round_tf32(v.y - w[1]);
#pragma unroll
    for (int i = 0; i < 4; ++i) *reinterpret_cast<float *>(base + n[i] * 16) = w[i];
  } else {
    unsigned short b[4];
    b[0] = big_round_bf16(v.x);
    b[1] = big_round_bf16(v.y);
    b[2] = big_round_bf16(v.x - umma::bf16_to_float(b[0]));
    b[3] = big_round_bf16(v.y - umma::bf16_to_float(b[1]));
#pragma unroll
    for (int i = 0; i < 4; ++i) *reinterpret_cast<unsigned short *>(base + n[i] * 16) = b[i];
  }
}

struct BigArgs {
  int RT, KT, KTU, KS, PC;
  long long a_tile, b_panel;   // bytes of an A tile (f, j) and of a panel's B operand
};

// ---- one stage's GEMM: unit = (row tile, panel, K segment) ------------------------------------
template <int PC, int KIND>
__global__ void __launch_bounds__(192, 1)
    k_big_mma(BigArgs a, int Mb, int Ml, const Panel *__restrict__ panels,
              const unsigned char *__restrict__ tiles, int j, const unsigned char *__restrict__ B,
              float2 *__restrict__ acc, int *__restrict__ err) {
  constexpr int NCOL = 8 * PC;
  constexpr int NALLOC = NCOL <= 64 ? 64 : (NCOL <= 128 ? 128 : 256);
  constexpr uint32_t kIdN4 = KIND == 0 ? umma::idesc_tf32(128, 4 * PC) : umma::idesc_bf16(128, 4 * PC);
  constexpr uint32_t kIdN2 = KIND == 0 ? umma::idesc_tf32(128, 2 * PC) : umma::idesc_bf16(128, 2 * PC);
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  __shared__ uint64_t bars[6];   // full[2], empty[2], dready, drain
  __shared__ uint32_t tmem_base;
  __shared__ int abort_flag;
  uint64_t *full = bars, *empty = bars + 2, *dready = bars + 4, *drain = bars + 5;
  // the panel index varies fastest: the CTAs that read the same (row tile, K segment) of S_j^{-1}
  // run side by side, so that the tile comes from HBM once and from L2 for the other panels
  const int unit = blockIdx.x;
  const int npan = (int)(gridDim.x / (a.RT * ((a.KT + a.KTU - 1) / a.KTU)));
  const int pn = unit % npan;
  const int rt = (unit / npan) % a.RT;
  const int ks = unit / (npan * a.RT);
  const Panel p = panels[pn];
  if (p.ncol == 0) return;   // an empty panel of a compacted list: its B and acc stay zero
  const int t0 = ks * a.KTU, nt = min(a.KTU, a.KT - t0);
  const uint32_t a_step = 16384u, b_step = 128u * PC;
  const uint32_t slot_bytes = (a_step + b_step) * a.KS;
  const int nch = (nt + a.KS - 1) / a.KS;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  auto aborted = [&]() { return *reinterpret_cast<volatile int *>(&abort_flag) != 0; };
  auto fail = [&](int code) {
    atomicExch(err, code);
    *reinterpret_cast<volatile int *>(&abort_flag) = 1;
  };
  if (tid == 0) {
    mbar_init(&full[0], 1);
    mbar_init(&full[1], 1);
    mbar_init(&empty[0], 1);
    mbar_init(&empty[1], 1);
    mbar_init(dready, 1);
    mbar_init(drain, 1);
    abort_flag = 0;
    mbar_init_fence();
  }
  if (warp == 5) {
    umma::tmem_alloc(&tmem_base, NALLOC);
    umma::tmem_relinquish();
  }
  umma::fence_before_sync();
  __syncthreads();
  umma::fence_after_sync();
  const uint32_t tmem = tmem_base;
  const unsigned char *At = tiles + ((long long)p.factor * Ml + j) * a.a_tile +
                            ((long long)rt * a.KT + t0) * a_step;
  const unsigned char *Bt = B + (long long)pn * a.b_panel + (long long)t0 * b_step;

  if (warp == 4) {
    // producer: chunk c = K-steps [c KS, c KS + KS) of the unit, A then B in one slot
    if (lane == 0) {
      int last0 = -1, last1 = -1;
      for (int c = 0; c < nch; ++c) {
        const int s = c & 1;
        if (c >= 2 && !mbar_wait(&empty[s], ((c >> 1) - 1) & 1)) { fail(21); break; }
        if (aborted()) break;
        const int n = min(a.KS, nt - c * a.KS);
        unsigned char *slot = smem_raw + (size_t)s * slot_bytes;
        mbar_arrive_expect_tx(&full[s], (uint32_t)n * (a_step + b_step));
        bulk_g2s(slot, At + (long long)c * a.KS * a_step, (uint32_t)n * a_step, &full[s]);
        bulk_g2s(slot + (size_t)a.KS * a_step, Bt + (long long)c * a.KS * b_step,
                 (uint32_t)n * b_step, &full[s]);
        if (s == 0) last0 = c; else last1 = c;
      }
      if (last0 >= 0 && !mbar_wait(&full[0], (last0 >> 1) & 1)) atomicExch(err, 22);
      if (last1 >= 0 && !mbar_wait(&full[1], (last1 >> 1) & 1)) atomicExch(err, 22);
    }
  } else if (warp == 5) {
    // MMA issuer
    if (lane == 0) {
      const uint64_t dA = (uint64_t)a_step >> 4, dC = 4096u >> 4, dB = (uint64_t)b_step >> 4;
      const uint32_t d1 = tmem, d2 = tmem + 4 * PC;
      bool ok = true;
      for (int c = 0; c < nch && ok; ++c) {
        const int s = c & 1;
        if (!mbar_wait(&full[s], (c >> 1) & 1)) { fail(23); ok = false; break; }
        umma::fence_after_sync();
        const int n = min(a.KS, nt - c * a.KS);
        unsigned char *slot = smem_raw + (size_t)s * slot_bytes;
        uint64_t ad = umma::smem_desc(umma::saddr(slot), 2048, 128);
        uint64_t bd = umma::smem_desc(umma::saddr(slot + (size_t)a.KS * a_step), 64u * PC, 128);
        for (int t = 0; t < n; ++t) {
          const uint32_t first = (c > 0 || t > 0) ? 1u : 0u;
          if (KIND == 0) {
            umma::mma_tf32(d1, ad, bd, kIdN4, first);
            umma::mma_tf32(d1, ad + dC, bd, kIdN2, 1);
            umma::mma_tf32(d2, ad + 2 * dC, bd, kIdN4, first);
            umma::mma_tf32(d2, ad + 3 * dC, bd, kIdN2, 1);
          } else {
            umma::mma_bf16(d1, ad, bd, kIdN4, first);
            umma::mma_bf16(d1, ad + dC, bd, kIdN2, 1);
            umma::mma_bf16(d2, ad + 2 * dC, bd, kIdN4, first);
            umma::mma_bf16(d2, ad + 3 * dC, bd, kIdN2, 1);
          }
          ad += dA;
          bd += dB;
        }
        umma::mma_commit(&empty[s]);
      }
      if (ok) umma::mma_commit(dready);
      umma::mma_commit(drain);
      if (!mbar_wait(drain, 0)) atomicExch(err, 24);
    }
  } else {
    // epilogue: row r of the tile; the unit's partial products go to the accumulator
    const int r = tid;
    const int row = rt * 128 + r;
    int ok = 1;
    if (lane == 0) ok = mbar_wait(dready, 0) ? 1 : 0;
    ok = __shfl_sync(0xffffffffu, ok, 0);
    if (ok && !aborted()) {
      umma::fence_after_sync();
      const uint32_t lane_base = (uint32_t)((warp & 3) * 32) << 16;
      float2 *dst = acc + ((long long)pn * Mb + row) * PC;
#pragma unroll 1
      for (int c0 = 0; c0 < PC; c0 += 8) {
        float d[4][16];
        // columns c0..c0+7 of: D1 piece 0 [re | im], D1 piece 1, D2 piece 0, D2 piece 1
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          const uint32_t base = (uint32_t)((u >> 1) * 4 * PC + (u & 1) * 2 * PC);
          umma::tmem_ld8(tmem + lane_base + base + c0, &d[u][0]);
          umma::tmem_ld8(tmem + lane_base + base + PC + c0, &d[u][8]);
        }
        umma::tmem_wait_ld();
        if (row < Mb) {
#pragma unroll
          for (int h = 0; h < 8; ++h) {
            const int c = c0 + h;
            if (c >= p.ncol) break;
            const float p_re = d[0][h] + d[1][h], p_im = d[0][8 + h] + d[1][8 + h];
            const float q_re = d[2][h] + d[3][h], q_im = d[2][8 + h] + d[3][8 + h];
            red_add_f2(dst + c, make_float2(p_re - q_im, p_im + q_re));
          }
        }
      }
    } else if (lane == 0) {
      fail(25);
    }
  }
  umma::fence_before_sync();
  __syncthreads();
  if (warp == 5) {
    umma::fence_after_sync();
    umma::tmem_dealloc(tmem, NALLOC);
  }
}

// ---- one stage's element-wise part -------------------------------------------------------------
// kind 0: prologue (B of the first stage = b_0); 1: forward stage j; 2: backward stage j.
template <int KIND>
__global__ void k_big_epi(int Mb, int Ml, long long Nloc, int npan, int PC,
                          const Panel *__restrict__ panels, const Col *__restrict__ cols,
                          const float2 *__restrict__ cpl, float2 *__restrict__ work,
                          float2 *__restrict__ acc, unsigned char *__restrict__ B,
                          long long b_panel, int kind, int j) {
  const long long total = (long long)npan * Mb * PC;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
       i += (long long)gridDim.x * blockDim.x) {
    const int c = (int)(i % PC);
    const int r = (int)((i / PC) % Mb);
    const int pn = (int)(i / ((long long)PC * Mb));
    const Panel p = panels[pn];
    unsigned char *Bp = B + (long long)pn * b_panel;
    if (c >= p.ncol) {
      if (kind == 0) big_put_b<KIND>(Bp, PC, r, c, make_float2(0.f, 0.f));
      continue;
    }
    float2 *x = work + (long long)cols[p.col0 + c].slot * Nloc;
    const float2 *cf = cpl + (long long)p.factor * Ml * Mb;
    float2 v = make_float2(0.f, 0.f);
    bool more = true;
    if (kind == 0) {
      v = x[r];
    } else {
      float2 *ap = acc + ((long long)pn * Mb + r) * PC + c;
      const float2 d = *ap;
      *ap = make_float2(0.f, 0.f);
      if (kind == 1) {
        x[(long long)j * Mb + r] = d;                                       // y_j
        if (j + 1 < Ml) v = csub(x[(long long)(j + 1) * Mb + r], cmul(cf[(long long)j * Mb + r], d));
        else if (Ml >= 2) v = cmul(cf[(long long)(Ml - 2) * Mb + r], d);  // last forward block
        else more = false;
      } else {
        const float2 xv = csub(x[(long long)j * Mb + r], d);              // x_j
        x[(long long)j * Mb + r] = xv;
        if (j > 0) v = cmul(cf[(long long)(j - 1) * Mb + r], xv);
        else more = false;
      }
    }
    if (more) big_put_b<KIND>(Bp, PC, r, c, v);
  }
}

// ---- the whole substitution of one panel list ---------------------------------------------------
template <int PC, int KIND>
static cudaError_t big_run(cudaStream_t st, const Geom &g, const BigShape &t, int npanels,
                           const Panel *panels, const Col *cols, const unsigned char *tiles,
                           const float2 *cpl, float2 *work, float2 *acc, unsigned char *B,
                           int *err, long long *launches) {
  static bool done[64] = {false};
  cudaError_t e = smem_limit_once(k_big_mma<PC, KIND>, done);
  if (e != cudaSuccess) return e;
  const long long b_panel = (long long)t.KT * 128 * PC;
  BigArgs a{t.RT, t.KT, t.KTU, t.KS, PC, t.a_tile, b_panel};
  const int units = t.RT * t.KSPLIT * npanels;
  const long long elems = (long long)npanels * g.Mb * PC;
  const int eblocks = (int)std::min<long long>((elems + 255) / 256, 152LL * 8);
  k_big_epi<KIND><<<eblocks, 256, 0, st>>>(g.Mb, g.Ml, g.Nloc, npanels, PC, panels, cols, cpl,
                                           work, acc, B, b_panel, 0, 0);
  ++*launches;
  for (int q = 0; q < 2 * g.Ml - 1; ++q) {
    const bool fwd = q < g.Ml;
    const int j = fwd ? q : 2 * g.Ml - 2 - q;
    k_big_mma<PC, KIND><<<units, 192, t.smem, st>>>(a, g.Mb, g.Ml, panels, tiles, j, B, acc, err);
    k_big_epi<KIND><<<eblocks, 256, 0, st>>>(g.Mb, g.Ml, g.Nloc, npanels, PC, panels, cols, cpl,
                                             work, acc, B, b_panel, fwd ? 1 : 2, j);
    *launches += 2;
  }
  return cudaGetLastError();
}

size_t big_scratch_bytes(const Geom &g, int kind, int pc, int npanels, size_t *acc_bytes) {
  BigShape t;
  big_shape(g, kind, pc, 1, &t);
  if (acc_bytes) *acc_bytes = (size_t)npanels * g.Mb * pc * sizeof(float2);
  return (size_t)npanels * t.KT * 128 * pc;
}

cudaError_t launch_subst_big(cudaStream_t st, const Geom &g, int kind, int npanels,
                             const Panel *panels, const Col *cols, const unsigned char *tiles,
                             const float2 *cpl, float2 *work, int pc, int ksplit, float2 *acc,
                             unsigned char *B, int *err, long long *launches) {
  if (npanels <= 0) return cudaSuccess;
  BigShape t;
  if (!big_shape(g, kind, pc, ksplit, &t)) return cudaErrorInvalidValue;
  if (kind == 0) {
    switch (pc) {
      case 8: return big_run<8, 0>(st, g, t, npanels, panels, cols, tiles, cpl, work, acc, B, err, launches);
      case 16: return big_run<16, 0>(st, g, t, npanels, panels, cols, tiles, cpl, work, acc, B, err, launches);
      case 32: return big_run<32, 0>(st, g, t, npanels, panels, cols, tiles, cpl, work, acc, B, err, launches);
    }
  } else {
    switch (pc) {
      case 8: return big_run<8, 1>(st, g, t, npanels, panels, cols, tiles, cpl, work, acc, B, err, launches);
      case 16: return big_run<16, 1>(st, g, t, npanels, panels, cols, tiles, cpl, work, acc, B, err, launches);
      case 32: return big_run<32, 1>(st, g, t, npanels, panels, cols, tiles, cpl, work, acc, B, err, launches);
    }
  }
  return cudaErrorInvalidValue;
}

}  // namespace dds
