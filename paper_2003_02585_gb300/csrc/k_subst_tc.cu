// Block-tridiagonal substitutions on the 5th-generation tensor cores (tcgen05), complex single
// precision through split products with FP32 accumulation in tensor memory.
//
// Same recurrences as k_subst / k_subst_stream:
//   forward  y_0 = S_0^{-1} b_0,  y_j = S_j^{-1} (b_j - C_{j-1} y_{j-1})
//   backward x_{Ml-1} = y_{Ml-1}, x_j = y_j - S_j^{-1} (C_j x_{j+1})
// Stage q of the 2 Ml - 1 stage chain is one complex product S_j^{-1} V (Mb x Mb times Mb x PC).
//
// Split products.  Every real operand is a sum of two pieces, x = x0 + x1 with x0 = rn(x) and
// x1 = rn(x - x0) in TF32 (10 explicit mantissa bits, 8 K columns per instruction) or BF16
// (7 bits, 16 K columns per instruction), and a b ~ a0 b0 + a0 b1 + a1 b0.  The complex product
// is real-ified with the right-hand sides' real and imaginary parts side by side in N:
//   B = [V0_re V0_im | V1_re V1_im]   (4 PC rows of the K-major B operand; pieces 0 then 1)
//   D1 = A0_re B + A1_re B[:2PC]      = Re(S^{-1}) V   (pieces summed in the epilogue)
//   D2 = A0_im B + A1_im B[:2PC]      = Im(S^{-1}) V
//   S^{-1} V = (D1_re - D2_im) + i (D1_im + D2_re)
// so one K-step is four MMAs (M = 128, N = 4 PC or 2 PC) into two TMEM accumulators of 4 PC
// FP32 columns each.
//
// Pipeline per CTA (one panel of PC right-hand sides sharing one factor):
//   producer warp   streams the pre-split S_j^{-1} tiles in stage order through a two-slot
//                   shared-memory ring with bulk copies completed on mbarriers;
//   MMA warp        one elected thread issues the stage's MMAs once the ring slot is full and
//                   the epilogue has written the stage's B operand, and commits to mbarriers
//                   that free the slot and signal the accumulator;
//   epilogue warps  4 NG warps (TMEM lane quarter = warp % 4 = row block, warp / 4 = column
//                   group) read the accumulator, form x_j, store it, and write the next
//                   stage's B operand (split into pieces) into shared memory.
// Every wait is bounded; on a timeout the CTA records an error code, lets its copies and MMAs
// drain, frees its tensor memory and exits.
#include "async_copy.cuh"
#include "dds_internal.cuh"
#include "umma.cuh"

namespace dds {

// ---------------------------------------------------------------------------------------------
// Layout of the split block inverses.  Tile (f, j) = S_j^{-1} of factor f, ks K-steps of
// 128 * Mp bytes each: [K-step t][comp][g][row m < Mp][16 bytes], comp 0/1 = pieces 0/1 of the
// real part, 2/3 = pieces 0/1 of the imaginary part, g = which 16-byte core-matrix column of
// the K-step.  Element (m, k) sits at t = k / (2 EK), g = (k / EK) % 2, byte (k % EK) * es
// (EK elements of es bytes per 16 bytes).  Zero outside m < Mb, k < Mb.

struct TcShape {
  int kind;      // 0 = TF32 pieces, 1 = BF16 pieces
  int EK;        // elements per 16 bytes
  int Mp, Kp;    // rows (Mb rounded up to 8) and K columns (rounded up to one K-step)
  int ks;        // K-steps per tile
  int KS;        // K-steps per ring chunk
  int nch;       // chunks per stage
  int LB;        // bytes per 16-byte K group of the B operand (4 PC rows + 16 bytes of pad)
  long long tile_bytes;
  size_t smem;
};

static size_t tc_static_smem() { return 1024; }

bool tc_shape(const Geom &g, int kind, int pc, TcShape *s, bool twisted = false, int np = 1) {
  TcShape t;
  t.kind = kind;
  t.EK = kind == 0 ? 4 : 8;
  t.Mp = (g.Mb + 7) / 8 * 8;
  t.Kp = (g.Mb + 2 * t.EK - 1) / (2 * t.EK) * (2 * t.EK);
  if (t.Mp > 128 || t.Kp > 128) return false;
  if (pc != 8 && pc != 16 && pc != 32) return false;
  if (np != 1 && !(np == 2 && pc <= 16)) return false;
  t.ks = t.Kp / (2 * t.EK);
  t.LB = 4 * pc * 16 + 16;
  t.tile_bytes = (long long)t.ks * 128 * t.Mp;
  // B operand, plus the exchange buffer [128 rows][pc] of the two-sided chain, per panel
  const size_t bbytes = (size_t)np * ((size_t)(t.Kp / t.EK) * t.LB + (twisted ? (size_t)128 * pc * 8 : 0));
  const size_t budget = 227 * 1024 - tc_static_smem();
  for (int nch = 1; nch <= t.ks; ++nch) {
    const int KS = (t.ks + nch - 1) / nch;
    const size_t smem = 2 * (size_t)KS * 128 * t.Mp + bbytes + 2048;
    if (smem <= budget) {
      t.KS = KS;
      t.nch = (t.ks + KS - 1) / KS;
      t.smem = smem;
      if (s) *s = t;
      return true;
    }
  }
  return false;
}

long long tc_tiles_bytes(const Geom &g, int kind, int nfac) {
  TcShape t;
  if (!tc_shape(g, kind, 8, &t)) return 0;
  return (long long)nfac * g.Ml * t.tile_bytes;
}

template <int KIND>
__global__ void k_split_tc(const double2 *__restrict__ sinv, const double2 *__restrict__ tw,
                           int m, unsigned char *__restrict__ out, int nfac, int Mb, int Ml,
                           long long St, int Mp, int Kp) {
  constexpr int EK = KIND == 0 ? 4 : 8, ES = 16 / EK;
  const long long total = (long long)nfac * Ml * Kp * Mp;
  const long long tile = (long long)(Kp / (2 * EK)) * 128 * Mp;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
       i += (long long)gridDim.x * blockDim.x) {
    const int mm = (int)(i % Mp);
    const int k = (int)((i / Mp) % Kp);
    const long long fj = i / ((long long)Mp * Kp);
    double2 a = make_double2(0.0, 0.0);
    if (mm < Mb && k < Mb) {
      // two-sided factorisation: tiles from the middle block down come from tw
      const double2 *src = (tw != nullptr && (int)(fj % Ml) >= m) ? tw : sinv;
      a = src[fj * St + (long long)k * Mb + mm];
    }
    const int t = k / (2 * EK), gg = (k / EK) & 1;
    unsigned char *base = out + fj * tile + (long long)t * 128 * Mp + (long long)mm * 16 + (k % EK) * ES;
    const double parts[2] = {a.x, a.y};
#pragma unroll
    for (int e = 0; e < 2; ++e) {
      const double x = parts[e];
      unsigned char *p0 = base + (long long)((2 * e + 0) * 2 + gg) * Mp * 16;
      unsigned char *p1 = base + (long long)((2 * e + 1) * 2 + gg) * Mp * 16;
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

cudaError_t launch_split_tc(cudaStream_t st, const Geom &g, int kind, int nfac,
                            const double2 *sinv64, const double2 *tw64, int m,
                            unsigned char *tiles) {
  TcShape t;
  if (!tc_shape(g, kind, 8, &t)) return cudaErrorInvalidValue;
  const long long total = (long long)nfac * g.Ml * t.Kp * t.Mp;
  const int threads = 256;
  const int blocks = (int)std::min<long long>((total + threads - 1) / threads, 152LL * 16);
  if (kind == 0)
    k_split_tc<0><<<blocks, threads, 0, st>>>(sinv64, tw64, m, tiles, nfac, g.Mb, g.Ml, g.St, t.Mp,
                                              t.Kp);
  else
    k_split_tc<1><<<blocks, threads, 0, st>>>(sinv64, tw64, m, tiles, nfac, g.Mb, g.Ml, g.St, t.Mp,
                                              t.Kp);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------------------------

struct TcArgs {
  int Mp, Kp, ks, KS, nch, LB;
  long long tile_bytes;
};

// Pieces of an FP32 value by rounding its bit pattern to nearest (ties away from zero): the
// 10 (TF32) or 7 (BF16) explicit mantissa bits of x0, then the same for x1 = x - x0, which is
// exact in FP32.  Integer adds and masks, no conversion instructions.
__device__ __forceinline__ float round_tf32(float x) {
  return __uint_as_float((__float_as_uint(x) + 0x1000u) & 0xFFFFE000u);
}
__device__ __forceinline__ unsigned short round_bf16(float x) {
  return (unsigned short)((__float_as_uint(x) + 0x8000u) >> 16);
}

// write the two pieces of v (row k of the B operand) for rows n_re (real part) and n_im
// (imaginary part) of piece 0, and the same rows + 2 PC of piece 1
template <int KIND, int PC>
__device__ __forceinline__ void put_b(unsigned char *sB, int LB, int k, int n_re, int n_im,
                                      float2 v) {
  constexpr int EK = KIND == 0 ? 4 : 8, ES = 16 / EK;
  const int off = (k / EK) * LB + (k % EK) * ES;
  const int n[4] = {n_re, n_im, n_re + 2 * PC, n_im + 2 * PC};
  if (KIND == 0) {
    float w[4];
    w[0] = round_tf32(v.x);
    w[1] = round_tf32(v.y);
    w[2] = round_tf32(v.x - w[0]);
    w[3] = round_tf32(v.y - w[1]);
#pragma unroll
    for (int i = 0; i < 4; ++i)
      *reinterpret_cast<float *>(sB + off + (n[i] >> 3) * 128 + (n[i] & 7) * 16) = w[i];
  } else {
    unsigned short b[4];
    b[0] = round_bf16(v.x);
    b[1] = round_bf16(v.y);
    b[2] = round_bf16(v.x - umma::bf16_to_float(b[0]));
    b[3] = round_bf16(v.y - umma::bf16_to_float(b[1]));
#pragma unroll
    for (int i = 0; i < 4; ++i)
      *reinterpret_cast<unsigned short *>(sB + off + (n[i] >> 3) * 128 + (n[i] & 7) * 16) = b[i];
  }
}

// Stage map of one CTA.  The chain is split at block m: role 0 runs blocks 0..m-1 forward, the
// middle block m, then m-1..0 backward; role 1 (two-sided factorisation only) runs Ml-1..m+1
// forward, the middle block, then m+1..Ml-1 backward.  The one-sided chain is role 0 with
// m = Ml - 1 (its "middle" is the last block).  Tiles: S_j^{-1} for j < m, the middle inverse
// (Z_m^{-1}, or S_{Ml-1}^{-1} one-sided) at m, T_j^{-1} for j > m.
struct TcStage {
  int j;      // block
  int kind;   // 0 forward, 1 middle, 2 backward
  int jn;     // block of the next stage of this CTA (-1: none)
};
__device__ inline TcStage tc_stage(int role, int q, int m, int Ml) {
  TcStage t;
  if (role == 0) {
    if (q < m) { t.j = q; t.kind = 0; t.jn = q + 1; }
    else if (q == m) { t.j = m; t.kind = 1; t.jn = m - 1; }
    else { t.j = 2 * m - q; t.kind = 2; t.jn = t.j - 1; }
  } else {
    const int nf = Ml - 1 - m;
    if (q < nf) { t.j = Ml - 1 - q; t.kind = 0; t.jn = t.j - 1; }
    else if (q == nf) { t.j = m; t.kind = 1; t.jn = m + 1 < Ml ? m + 1 : -1; }
    else { t.j = m + (q - nf); t.kind = 2; t.jn = t.j + 1 < Ml ? t.j + 1 : -1; }
  }
  if (t.jn < 0) t.jn = -1;
  return t;
}
__device__ inline int tc_nstages(int role, int m, int Ml) {
  return role == 0 ? 2 * m + 1 : 2 * (Ml - 1 - m) + 1;
}

// NP panels per CTA (1 or 2): each panel has its own tensor-memory accumulator pair, B operand,
// exchange buffer and barriers; the MMA issuer and the epilogue take the panels in turn at every
// stage, so the epilogue of one panel runs while the other panel's MMAs do.
template <int PC, int KIND, int NG, bool TW, int NP>
__global__ void __launch_bounds__(32 * (4 * NG + 2), 1)
    k_subst_tc(Geom g, TcArgs a, const Panel *__restrict__ panels, int npanels,
               const Col *__restrict__ cols, const unsigned char *__restrict__ tiles,
               const float2 *__restrict__ cpl, float2 *__restrict__ work, int *__restrict__ err,
               int m, const int *__restrict__ nz) {
  constexpr int H = PC / NG;            // columns per epilogue thread
  constexpr int NEPI = 128 * NG;        // epilogue threads
  constexpr int NCOL = 8 * PC;          // TMEM columns per panel: D1 [0, 4PC), D2 [4PC, 8PC)
  constexpr int NALL = NP * NCOL;
  constexpr int NALLOC = NALL <= 32 ? 32 : (NALL <= 64 ? 64 : (NALL <= 128 ? 128 : (NALL <= 256 ? 256 : 512)));
  constexpr uint32_t kIdN4 = KIND == 0 ? umma::idesc_tf32(128, 4 * PC) : umma::idesc_bf16(128, 4 * PC);
  constexpr uint32_t kIdN2 = KIND == 0 ? umma::idesc_tf32(128, 2 * PC) : umma::idesc_bf16(128, 2 * PC);
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  // full[2], empty[2], drain, then per panel: dready, bready, xbar
  __shared__ uint64_t bars[5 + 3 * NP];
  __shared__ uint32_t tmem_base;
  __shared__ int abort_flag;
  uint64_t *full = bars, *empty = bars + 2, *drain = bars + 4;
  uint64_t *dready = bars + 5, *bready = bars + 5 + NP, *xbar = bars + 5 + 2 * NP;

  const int Mb = g.Mb, Ml = g.Ml;
  const int role = TW ? (int)cluster_ctarank() : 0;
  const int nst = tc_nstages(role, m, Ml);
  const int nfwd = role == 0 ? m : Ml - 1 - m;   // forward stages before the middle block
  const long long chunk_bytes = (long long)a.KS * 128 * a.Mp;
  const size_t bbytes = (size_t)(a.Kp / (KIND == 0 ? 4 : 8)) * a.LB;
  unsigned char *ring = smem_raw;
  auto sBp = [&](int h) { return smem_raw + 2 * chunk_bytes + (size_t)h * bbytes; };
  // exchange buffers of the two-sided chain: the peer's coupling terms, [panel][row][PC]
  float2 *xch0 = reinterpret_cast<float2 *>(smem_raw + 2 * chunk_bytes + (size_t)NP * bbytes);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  // this CTA's panels: NP consecutive entries of the list, of which the empty ones (a compacted
  // list's spares, or, with nz, panels whose columns all have zero right-hand sides: their solution
  // is the zero already in work) are dropped; both CTAs of a cluster see the same and agree
  Panel P[NP];
  int np_act = 0;
  {
    const int pair = TW ? blockIdx.x / 2 : blockIdx.x;
#pragma unroll
    for (int h = 0; h < NP; ++h) {
      const int idx = pair * NP + h;
      if (idx >= npanels) continue;
      const Panel p = panels[idx];
      if (p.ncol == 0) continue;
      if (nz != nullptr) {
        int any = 0;
        for (int c = 0; c < p.ncol; ++c) any |= nz[cols[p.col0 + c].slot];
        if (!any) continue;
      }
#pragma unroll
      for (int k = 0; k < NP; ++k)
        if (k == np_act) P[k] = p;
      ++np_act;
    }
  }
  if (np_act == 0) return;
  // two panels of one factor read the same tile at every stage: it is streamed once and both
  // panels' MMAs read it (half the L2 traffic of the tiles, which paces the chain)
  const bool shared = NP == 2 && np_act == 2 && P[0].factor == P[NP - 1].factor;
  const int streams = shared ? 1 : np_act;   // tile streams per stage
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
    mbar_init(drain, 1);
#pragma unroll
    for (int h = 0; h < NP; ++h) {
      mbar_init(&dready[h], 1);
      mbar_init(&bready[h], NEPI / 32);   // one arrival per epilogue warp
      mbar_init(&xbar[h], NEPI);          // one remote arrival per epilogue thread of the peer
    }
    abort_flag = 0;
    mbar_init_fence();
  }
  if (warp == 4 * NG + 1) {
    umma::tmem_alloc(&tmem_base, NALLOC);
    umma::tmem_relinquish();
  }
  umma::fence_before_sync();
  if (TW) cluster_sync_all();   // both CTAs' barriers exist before any remote arrival
  else __syncthreads();
  umma::fence_after_sync();
  const uint32_t tmem = tmem_base;

  if (warp == 4 * NG) {
    // ---------------- producer: the tiles of every (stage, stream) through the two-slot ring
    if (lane == 0) {
      int last0 = -1, last1 = -1;
      const int nchunks = nst * streams * a.nch;
      for (int i = 0; i < nchunks; ++i) {
        const int s = i & 1;
        if (i >= 2 && !mbar_wait(&empty[s], ((i >> 1) - 1) & 1)) { fail(11); break; }
        if (aborted()) break;
        const int q = i / (streams * a.nch), h = (i / a.nch) % streams, c = i % a.nch;
        const int nks = min(a.KS, a.ks - c * a.KS);
        const uint32_t bytes = (uint32_t)nks * 128u * (uint32_t)a.Mp;
        const int j = tc_stage(role, q, m, Ml).j;
        int fac = P[0].factor;
#pragma unroll
        for (int k = 1; k < NP; ++k)
          if (h == k) fac = P[k].factor;
        const unsigned char *src = tiles + ((long long)fac * Ml + j) * a.tile_bytes +
                                   (long long)c * a.KS * 128 * a.Mp;
        mbar_arrive_expect_tx(&full[s], bytes);
        bulk_g2s(ring + s * chunk_bytes, src, bytes, &full[s]);
        if (s == 0) last0 = i; else last1 = i;
      }
      // no copy may still be landing when the CTA leaves
      if (last0 >= 0 && !mbar_wait(&full[0], (last0 >> 1) & 1)) atomicExch(err, 12);
      if (last1 >= 0 && !mbar_wait(&full[1], (last1 >> 1) & 1)) atomicExch(err, 12);
    }
  } else if (warp == 4 * NG + 1) {
    // ---------------- MMA issuer: at every stage, each panel in turn once its B operand is in
    if (lane == 0) {
      const uint32_t lbo_a = (uint32_t)a.Mp * 16u;
      const uint64_t dA = (uint64_t)8 * a.Mp;              // one K-step of A, in 16-byte units
      const uint64_t dC = (uint64_t)2 * a.Mp;              // one component of A
      const uint64_t dB = (uint64_t)(2 * a.LB) >> 4;       // one K-step of B
      int i = 0;                                           // ring chunks consumed
      bool ok = true;
      // the MMAs of panel h on ring slot s, chunk c of the stage
      auto issue = [&](int h, int s, int c) {
        const uint64_t b0 = umma::smem_desc(umma::saddr(sBp(h)), (uint32_t)a.LB, 128);
        const uint32_t d1 = tmem + (uint32_t)h * NCOL, d2 = d1 + 4 * PC;
        const int nks = min(a.KS, a.ks - c * a.KS);
        uint64_t ad = umma::smem_desc(umma::saddr(ring + s * chunk_bytes), lbo_a, 128);
        uint64_t bd = b0 + (uint64_t)(c * a.KS) * dB;
        for (int t = 0; t < nks; ++t) {
          const uint32_t acc = (c > 0 || t > 0) ? 1u : 0u;
          if (KIND == 0) {
            umma::mma_tf32(d1, ad, bd, kIdN4, acc);
            umma::mma_tf32(d1, ad + dC, bd, kIdN2, 1);
            umma::mma_tf32(d2, ad + 2 * dC, bd, kIdN4, acc);
            umma::mma_tf32(d2, ad + 3 * dC, bd, kIdN2, 1);
          } else {
            umma::mma_bf16(d1, ad, bd, kIdN4, acc);
            umma::mma_bf16(d1, ad + dC, bd, kIdN2, 1);
            umma::mma_bf16(d2, ad + 2 * dC, bd, kIdN4, acc);
            umma::mma_bf16(d2, ad + 3 * dC, bd, kIdN2, 1);
          }
          ad += dA;
          bd += dB;
        }
      };
      for (int q = 0; q < nst && ok; ++q) {
        if (shared) {
          // one tile stream for both panels: panel 0's MMAs, then panel 1's, on every chunk.
          // Panel 1's operand is waited for only before its first MMA, and panel 0's accumulator
          // is released right after its last, so each panel's epilogue overlaps the other's MMAs.
          if (!mbar_wait(&bready[0], q & 1)) { fail(13); ok = false; break; }
          if (aborted()) { ok = false; break; }
          for (int c = 0; c < a.nch; ++c, ++i) {
            const int s = i & 1;
            if (!mbar_wait(&full[s], (i >> 1) & 1)) { fail(14); ok = false; break; }
            umma::fence_after_sync();
            issue(0, s, c);
            if (c == a.nch - 1) umma::mma_commit(&dready[0]);
            if (c == 0) {
              if (!mbar_wait(&bready[1], q & 1)) { fail(13); ok = false; break; }
              umma::fence_after_sync();
            }
            issue(1, s, c);
            umma::mma_commit(&empty[s]);   // the slot is free once these MMAs have read it
          }
          if (!ok) break;
          umma::mma_commit(&dready[1]);
          continue;
        }
        for (int h = 0; h < np_act && ok; ++h) {
          if (!mbar_wait(&bready[h], q & 1)) { fail(13); ok = false; break; }
          if (aborted()) { ok = false; break; }
          umma::fence_after_sync();
          for (int c = 0; c < a.nch; ++c, ++i) {
            const int s = i & 1;
            if (!mbar_wait(&full[s], (i >> 1) & 1)) { fail(14); ok = false; break; }
            umma::fence_after_sync();
            issue(h, s, c);
            umma::mma_commit(&empty[s]);   // the slot is free once these MMAs have read it
          }
          if (!ok) break;
          umma::mma_commit(&dready[h]);
        }
      }
      umma::mma_commit(drain);
      if (!mbar_wait(drain, 0)) atomicExch(err, 15);
    }
  } else {
    // ---------------- epilogue: row r of the block, columns grp*H .. grp*H + H - 1, each panel
    const int r = tid & 127, grp = tid >> 7;
    const bool row = r < Mb, krow = r < a.Kp;
    float2 *xs[NP][H];
    const float2 *cf[NP];
#pragma unroll
    for (int h = 0; h < NP; ++h) {
      const Panel &p = P[h];
      const bool act = h < np_act;
      cf[h] = cpl + (long long)(act ? p.factor : 0) * Ml * (long long)Mb;
#pragma unroll
      for (int k = 0; k < H; ++k) {
        const int c = grp * H + k;
        xs[h][k] = (act && c < p.ncol) ? work + (long long)cols[p.col0 + c].slot * g.Nloc : nullptr;
      }
    }
    // B operand of the first stage of every panel: the right-hand side of its block
    {
      const int j = tc_stage(role, 0, m, Ml).j;
#pragma unroll
      for (int h = 0; h < NP; ++h) {
        if (h >= np_act) break;
        if (krow) {
#pragma unroll
          for (int k = 0; k < H; ++k) {
            const float2 v = (row && xs[h][k]) ? xs[h][k][(long long)j * Mb + r] : make_float2(0.f, 0.f);
            put_b<KIND, PC>(sBp(h), a.LB, r, grp * 2 * H + k, grp * 2 * H + H + k, v);
          }
        }
        fence_proxy_async();
        umma::fence_before_sync();
        __syncwarp();
        if (lane == 0) mbar_arrive(&bready[h]);
      }
    }
    const uint32_t lane_base = (uint32_t)((warp & 3) * 32) << 16;
    bool stop = false;
    for (int q = 0; q < nst && !stop; ++q) {
      const TcStage st = tc_stage(role, q, m, Ml);
      const bool exch = TW && st.kind == 0 && q == nfwd - 1;   // last forward stage
      const bool more = q + 1 < nst;
#pragma unroll
      for (int h = 0; h < NP; ++h) {
        if (h >= np_act || stop) break;
        // epilogue operands, loaded before the accumulator is ready: the right-hand side of the
        // next block (forward), this block's forward result (backward), the coupling to the next
        float2 pre[H];
        float2 cn = make_float2(0.f, 0.f);
#pragma unroll
        for (int k = 0; k < H; ++k) pre[k] = make_float2(0.f, 0.f);
        if (row) {
          const int jp = st.kind == 0 ? st.jn : (st.kind == 2 ? st.j : -1);
          if (jp >= 0) {
#pragma unroll
            for (int k = 0; k < H; ++k)
              if (xs[h][k]) pre[k] = xs[h][k][(long long)jp * Mb + r];
          }
          if (st.jn >= 0) cn = cf[h][(long long)min(st.j, st.jn) * Mb + r];
        }
        // one lane per warp polls the accumulator barrier; the warp follows it
        int ok = 1;
        if (lane == 0) ok = mbar_wait(&dready[h], q & 1) ? 1 : 0;
        ok = __shfl_sync(0xffffffffu, ok, 0);
        if (!ok) { if (lane == 0) fail(16); stop = true; break; }
        if (aborted()) { stop = true; break; }
        umma::fence_after_sync();
        // accumulator runs of this column group: D1 piece 0, D1 piece 1, D2 piece 0, D2 piece 1
        float d[4][2 * H];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          const uint32_t col = (uint32_t)(h * NCOL + (u >> 1) * 4 * PC + (u & 1) * 2 * PC + grp * 2 * H);
#pragma unroll
          for (int c8 = 0; c8 < 2 * H; c8 += 8) umma::tmem_ld8(tmem + lane_base + col + c8, &d[u][c8]);
        }
        umma::tmem_wait_ld();
        float2 xo[H], vv[H];
#pragma unroll
        for (int k = 0; k < H; ++k) {
          const float p_re = d[0][k] + d[1][k], p_im = d[0][H + k] + d[1][H + k];
          const float q_re = d[2][k] + d[3][k], q_im = d[2][H + k] + d[3][H + k];
          const float2 acc = make_float2(p_re - q_im, p_im + q_re);
          if (st.kind == 2) {
            xo[k] = csub(pre[k], acc);            // x_j = y_j - S_j^{-1} C x_next
            vv[k] = cmul(cn, xo[k]);
          } else if (st.kind == 1) {
            xo[k] = acc;                          // middle block: x_m
            vv[k] = cmul(cn, acc);
          } else {
            xo[k] = acc;                          // forward: y_j (or z_j)
            vv[k] = exch ? cmul(cn, acc) : csub(pre[k], cmul(cn, acc));
          }
          if (!row) vv[k] = make_float2(0.f, 0.f);
        }
        if (exch) {
          // the coupling term C y of this half goes to the peer; the peer's comes back
          float2 *xch = xch0 + (size_t)h * 128 * PC;
          const uint32_t peer = (uint32_t)(role ^ 1);
          if (row) {
#pragma unroll
            for (int k = 0; k < H; ++k)
              st_cluster_f2(cluster_map(xch + r * PC + grp * H + k, peer), vv[k]);
          }
          // every thread releases its own remote writes and acquires the peer's
          mbar_arrive_remote(cluster_map(&xbar[h], peer));
          const int okx = __all_sync(0xffffffffu, mbar_wait_cluster(&xbar[h], 0) ? 1 : 0);
          if (!okx) { if (lane == 0) fail(17); stop = true; break; }
#pragma unroll
          for (int k = 0; k < H; ++k) {
            const float2 other = row ? xch[r * PC + grp * H + k] : make_float2(0.f, 0.f);
            vv[k] = row ? csub(csub(pre[k], vv[k]), other) : make_float2(0.f, 0.f);
          }
        }
        if (more && krow) {
#pragma unroll
          for (int k = 0; k < H; ++k)
            put_b<KIND, PC>(sBp(h), a.LB, r, grp * 2 * H + k, grp * 2 * H + H + k, vv[k]);
        }
        if (more) {
          fence_proxy_async();
          umma::fence_before_sync();
          __syncwarp();
          if (lane == 0) mbar_arrive(&bready[h]);
        }
        // x_j leaves for global memory while the next MMAs run (the middle block once)
        const bool store = !(TW && st.kind == 1 && role == 1);
#pragma unroll
        for (int k = 0; k < H; ++k)
          if (store && row && xs[h][k]) xs[h][k][(long long)st.j * Mb + r] = xo[k];
      }
    }
  }
  umma::fence_before_sync();
  __syncthreads();
  if (warp == 4 * NG + 1) {
    umma::fence_after_sync();
    umma::tmem_dealloc(tmem, NALLOC);
  }
  if (TW) cluster_sync_all();   // no CTA leaves while its peer may still touch its memory
}

template <int PC, int KIND, bool TW, int NP>
static cudaError_t tc_launch(cudaStream_t st, const Geom &g, const TcShape &t, int npanels,
                             const Panel *panels, const Col *cols, const unsigned char *tiles,
                             const float2 *cpl, float2 *work, int *err, int m, const int *nz) {
  constexpr int NG = 2;   // two epilogue column groups (measured faster than four at 16 columns)
  static bool done[64] = {false};
  cudaError_t e = smem_limit_once(k_subst_tc<PC, KIND, NG, TW, NP>, done);
  if (e != cudaSuccess) return e;
  TcArgs a{t.Mp, t.Kp, t.ks, t.KS, t.nch, t.LB, t.tile_bytes};
  const int groups = (npanels + NP - 1) / NP;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)(TW ? 2 * groups : groups));
  cfg.blockDim = dim3(32 * (4 * NG + 2));
  cfg.dynamicSmemBytes = t.smem;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = 2;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = TW ? 1 : 0;
  return cudaLaunchKernelEx(&cfg, k_subst_tc<PC, KIND, NG, TW, NP>, g, a, panels, npanels, cols,
                            tiles, cpl, work, err, TW ? m : g.Ml - 1, nz);
}

template <int KIND, bool TW>
static cudaError_t tc_dispatch(cudaStream_t st, const Geom &g, const TcShape &t, int npanels,
                               const Panel *panels, const Col *cols, const unsigned char *tiles,
                               const float2 *cpl, float2 *work, int pc, int *err, int m,
                               const int *nz, int np) {
  if (np == 2) {
    switch (pc) {
      case 8: return tc_launch<8, KIND, TW, 2>(st, g, t, npanels, panels, cols, tiles, cpl, work, err, m, nz);
      case 16: return tc_launch<16, KIND, TW, 2>(st, g, t, npanels, panels, cols, tiles, cpl, work, err, m, nz);
    }
    return cudaErrorInvalidValue;
  }
  switch (pc) {
    case 8: return tc_launch<8, KIND, TW, 1>(st, g, t, npanels, panels, cols, tiles, cpl, work, err, m, nz);
    case 16: return tc_launch<16, KIND, TW, 1>(st, g, t, npanels, panels, cols, tiles, cpl, work, err, m, nz);
    case 32: return tc_launch<32, KIND, TW, 1>(st, g, t, npanels, panels, cols, tiles, cpl, work, err, m, nz);
  }
  return cudaErrorInvalidValue;
}

cudaError_t launch_subst_tc(cudaStream_t st, const Geom &g, int kind, int npanels,
                            const Panel *panels, const Col *cols, const unsigned char *tiles,
                            const float2 *cpl, float2 *work, int pc, int *err, int m,
                            const int *nz, int np) {
  if (npanels <= 0) return cudaSuccess;
  const bool tw = m > 0;
  TcShape t;
  if (!tc_shape(g, kind, pc, &t, tw, np)) return cudaErrorInvalidValue;
  if (kind == 0)
    return tw ? tc_dispatch<0, true>(st, g, t, npanels, panels, cols, tiles, cpl, work, pc, err, m, nz, np)
              : tc_dispatch<0, false>(st, g, t, npanels, panels, cols, tiles, cpl, work, pc, err, m, nz, np);
  return tw ? tc_dispatch<1, true>(st, g, t, npanels, panels, cols, tiles, cpl, work, pc, err, m, nz, np)
            : tc_dispatch<1, false>(st, g, t, npanels, panels, cols, tiles, cpl, work, pc, err, m, nz, np);
}

bool subst_tc_ok(const Geom &g, int kind, int pc, bool twisted, int np) {
  return tc_shape(g, kind, pc, nullptr, twisted, np);
}

int tc_middle_block(const Geom &g) { return g.Ml >= 4 ? (g.Ml - 1) / 2 : 0; }

}  // namespace dds
