// Trace transfer on the 5th-generation tensor cores (tcgen05): every trace solve of one DDM
// application of the trace-operator plan as complex split-product GEMMs.
//
// The trace solve of (sweep l, subdomain X) maps the traces X received in slot l to the traces it
// sends (Lemma 2.2 in discrete form, the back-trace correction folded into the map):
//   out[R] = sum_k Map_f[R][k] in_l,X[k]   (+ the raw own-source lines in the first sweep),
// R over the stacked output rows of every side (side d at toff_d .. toff_d + 2 Lt_d), k over the
// inputs of the sides that receive in sweep l.  Row R of side d is added to the slot
// route[l][d] of the neighbour across d, at its side d ^ 1.  All (l, X, RHS) columns of one
// dataflow level that share a factor and a sweep share the map, so a level is a GEMM
//   (128-row tile of Map_f) x (K = received inputs) x (32 columns)
// per work unit, run with the split products of k_subst_tc.cu (pieces a = a0 + a1, b = b0 + b1,
// a b ~ a0 b0 + a0 b1 + a1 b0, TF32 or BF16 pieces, FP32 accumulation in tensor memory) and the
// real-ified complex form: B = [b0_re | b0_im | b1_re | b1_im] (4 x 32 rows of the K-major B
// operand), D1 = A0_re B + A1_re B[:64], D2 = A0_im B + A1_im B[:64].
//
// One CTA per SM, cooperative launch.  The host deals the units of every dataflow level (the
// schedule of k_trace_sweeps) over the CTAs and gives each CTA its units and their chunks
// (runs of at most four K-steps of one input side) as flat streams in run order, so that no
// role walks a schedule on the device.  There is no barrier between levels: a unit waits only
// until the trace solves routed into its own slots have published (per-slot counters against
// host-computed totals), so the levels overlap.  Warp roles:
//   warps 0-3   epilogue: TMEM lane quarter = warp; row R of the tile per thread; forms the
//               complex outputs of the 32 columns and adds them into the receivers' slots with
//               vector reductions; then publishes the unit on the receivers' counters;
//   warps 4-11  B producers: once the unit's slots are complete, copy its inputs from the trace
//               slots (cp.async, L1 bypassed: other CTAs wrote them) a few chunks ahead, split
//               them into pieces and store them in the canonical K-major layout of the ring slot;
//   warp 12     A producer: streams the pre-split map tiles through the two-slot ring with bulk
//               copies completed on the slot's mbarrier (it depends on no trace, so it runs
//               ahead);
//   warp 13     MMA issuer (one thread) and owner of the tensor memory: two accumulator pairs,
//               so that the epilogue of one unit runs under the MMAs of the next.
// Every wait is bounded; on a timeout the CTA records an error code, stops issuing work, lets its
// copies and MMAs drain, frees its tensor memory and leaves (the host reports DDS_ETIMEOUT).
#include <algorithm>

#include "async_copy.cuh"
#include "dds_internal.cuh"
#include "umma.cuh"

namespace dds {

namespace {

constexpr int kTtCols = 32;        // complex columns per unit
constexpr int kTtKS = 4;           // K-steps per ring chunk
constexpr int kTtSlots = 2;        // B ring slots (one chunk each)
constexpr int kTtASlots = 3;       // A ring slots (one chunk each)
constexpr int kTtStep = 16384;     // bytes of one K-step of an A tile (4 comps x 2 x 128 x 16)
constexpr int kTtLB = 4 * kTtCols * 16 + 16;   // bytes per 16-byte K group of B (+16: banks)
constexpr int kTtBStep = 2 * kTtLB;            // bytes of one K-step of B
constexpr int kTtASlotBytes = kTtKS * kTtStep;
constexpr int kTtBSlotBytes = kTtKS * kTtBStep;
constexpr int kTtBWarps = 8;       // B-producer warps
constexpr int kTtBThreads = 32 * kTtBWarps;
constexpr int kTtAWarp = 4 + kTtBWarps, kTtMmaWarp = kTtAWarp + 1;
constexpr int kTtThreads = 32 * (kTtMmaWarp + 1);
constexpr int kTtTmemCols = 512;   // two accumulator pairs of 8 x 32 FP32 columns

}  // namespace

// Split-map layout, per factor: [row tile rt][K-step t][comp][g][row m < 128][16 bytes]; comp
// 0/1 = pieces 0/1 of the real part, 2/3 of the imaginary part; g = which 16-byte core-matrix
// column of the K-step (the canonical K-major no-swizzle layout, as k_subst_tc.cu).  Inputs are
// stacked by side with side d at kpo[d], its 2 Lt_d values padded to a multiple of 16.
bool tt_shape(const Geom &g, int kind, TtShape *s) {
  TtShape t{};
  t.kind = kind;
  t.EK = kind == 0 ? 4 : 8;
  t.KE = 2 * t.EK;
  t.RT = (g.T + 127) / 128;
  int off = 0;
  for (int d = 0; d < 6; ++d) {
    t.kpo[d] = off;
    t.kpn[d] = d < g.nsides ? (2 * g.Lt[d] + 15) / 16 * 16 : 0;
    off += t.kpn[d];
  }
  t.KP = off;
  t.rt_bytes = (long long)(t.KP / t.KE) * kTtStep;
  t.fac_bytes = (long long)t.RT * t.rt_bytes;
  t.smem = (size_t)kTtASlots * kTtASlotBytes + (size_t)kTtSlots * kTtBSlotBytes + 1024;
  if (t.smem > 227 * 1024) return false;
  if (s) *s = t;
  return true;
}

long long tt_tiles_bytes(const Geom &g, int kind, int nfac) {
  TtShape t;
  if (!tt_shape(g, kind, &t)) return 0;
  return (long long)nfac * t.fac_bytes;
}

// The work of each CTA of a G-CTA launch, in the order it runs it: the units of every dataflow
// level dealt in a snake (unit j of a level goes to CTA j % G on even rounds j / G and to
// CTA G - 1 - j % G on odd ones), heaviest first as the host sorted them; and the chunks of those
// units, one descriptor each:
//   x = unit index | (1 << 30 on the unit's first chunk)
//   y = global K-step of the chunk's map tile (factor, row tile and input side folded in)
//   z = offset of the chunk's first input within a trace slot column (toff[d] + k0)
//   w = K-steps of the chunk | (inputs that exist, the rest being padding) << 8
// Units (x = unit index, y = its chunks) and chunks are stored CTA by CTA with offsets.
bool build_tt_streams(const Geom &g, int kind, int G, const std::vector<int4> &units,
                      const std::vector<int> &lev_off, std::vector<int> &uoff,
                      std::vector<int2> &cunits, std::vector<int> &coff,
                      std::vector<int4> &chunks) {
  TtShape t;
  if (!tt_shape(g, kind, &t) || G <= 0 || units.size() >= (1u << 30)) return false;
  const int nlev = (int)lev_off.size() - 1;
  std::vector<std::vector<int>> per(G);
  for (int v = 0; v < nlev; ++v)
    for (int j = lev_off[v]; j < lev_off[v + 1]; ++j) {
      const int r = (j - lev_off[v]) / G, w = (j - lev_off[v]) % G;
      per[(r & 1) ? G - 1 - w : w].push_back(j);
    }
  const long long steps = t.KP / t.KE;   // K-steps of one row tile of one factor
  uoff.assign(1, 0);
  coff.assign(1, 0);
  cunits.clear();
  chunks.clear();
  for (int b = 0; b < G; ++b) {
    for (int j : per[b]) {
      const int4 h = units[j];
      const int fac = h.x & 0xFFFFFF, rt = (h.y >> 16) & 0xFFFF, kmask = h.w & 0xFF;
      int nch = 0;
      for (int d = 0; d < g.nsides; ++d) {
        if (!((kmask >> d) & 1)) continue;
        const int ns = t.kpn[d] / t.KE;
        for (int t0 = 0; t0 < ns; t0 += kTtKS) {
          const int nks = std::min(kTtKS, ns - t0), k0 = t0 * t.KE;
          const int live = std::min(nks * t.KE, 2 * g.Lt[d] - k0);
          const long long a = ((long long)fac * t.RT + rt) * steps + t.kpo[d] / t.KE + t0;
          if (a > INT32_MAX || live <= 0) return false;
          chunks.push_back(make_int4(j | (nch == 0 ? 1 << 30 : 0), (int)a, g.toff[d] + k0,
                                     nks | (live << 8)));
          ++nch;
        }
      }
      cunits.push_back(make_int2(j, nch));
    }
    uoff.push_back((int)cunits.size());
    coff.push_back((int)chunks.size());
  }
  return true;
}

template <int KIND>
__global__ void k_split_trace(const double2 *__restrict__ gmap, unsigned char *__restrict__ out,
                              Geom g, TtShape t, int nfac) {
  constexpr int EK = KIND == 0 ? 4 : 8, ES = 16 / EK;
  const long long rows = (long long)t.RT * 128;
  const long long total = (long long)nfac * rows * t.KP;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
       i += (long long)gridDim.x * blockDim.x) {
    const int R = (int)(i % rows);
    const int kp = (int)((i / rows) % t.KP);
    const int f = (int)(i / (rows * t.KP));
    // output side / row of R, input side / index of kp
    double2 a = make_double2(0.0, 0.0);
    int dout = -1, din = -1;
    for (int d = 0; d < g.nsides; ++d) {
      if (R >= g.toff[d] && R < g.toff[d] + 2 * g.Lt[d]) dout = d;
      if (kp >= t.kpo[d] && kp < t.kpo[d] + t.kpn[d]) din = d;
    }
    if (dout >= 0 && din >= 0 && kp - t.kpo[din] < 2 * g.Lt[din]) {
      const int ro = R - g.toff[dout];
      const long long k = g.toff[din] + (kp - t.kpo[din]);
      a = gmap[gmap_index(g, f, dout, ro / kTraceRows, k, ro % kTraceRows)];
    }
    const int rt = R / 128, m = R % 128;
    const int ts = kp / t.KE, gg = (kp / EK) & 1;
    unsigned char *base = out + (long long)f * t.fac_bytes + (long long)rt * t.rt_bytes +
                          (long long)ts * kTtStep + (long long)gg * 128 * 16 + m * 16 + (kp % EK) * ES;
    const double parts[2] = {a.x, a.y};
#pragma unroll
    for (int e = 0; e < 2; ++e) {
      const double x = parts[e];
      unsigned char *p0 = base + (long long)(2 * e + 0) * 2 * 128 * 16;
      unsigned char *p1 = base + (long long)(2 * e + 1) * 2 * 128 * 16;
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

cudaError_t launch_split_trace(cudaStream_t st, const Geom &g, int kind, int nfac,
                               const double2 *gmap64, unsigned char *tiles) {
  TtShape t;
  if (!tt_shape(g, kind, &t)) return cudaErrorInvalidValue;
  const long long total = (long long)nfac * t.RT * 128 * t.KP;
  const int blocks = (int)std::min<long long>((total + 255) / 256, 152LL * 16);
  if (kind == 0)
    k_split_trace<0><<<blocks, 256, 0, st>>>(gmap64, tiles, g, t, nfac);
  else
    k_split_trace<1><<<blocks, 256, 0, st>>>(gmap64, tiles, g, t, nfac);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------------------------
// Work units (host-built): hdr = (factor | columns << 24, sweep | row tile << 16, first column
// word, input sides mask | raw << 8); column words = RHS * nsub + subdomain.

struct TtUnit {
  int factor, ncol, l, rt, col0, kmask, raw;
};
__device__ inline TtUnit tt_unit(const int4 *units, int idx) {
  const int4 h = __ldg(units + idx);
  TtUnit u;
  u.factor = h.x & 0xFFFFFF;
  u.ncol = (h.x >> 24) & 0xFF;
  u.l = h.y & 0xFFFF;
  u.rt = (h.y >> 16) & 0xFFFF;
  u.col0 = h.z;
  u.kmask = h.w & 0xFF;
  u.raw = (h.w >> 8) & 1;
  return u;
}

// the pieces of v written as B rows c (real) and 32 + c (imaginary) of piece 0, and the same
// rows + 64 of piece 1, at K position k of the chunk
template <int KIND>
__device__ __forceinline__ void tt_put_b(unsigned char *sB, int k, int c, float2 v) {
  constexpr int EK = KIND == 0 ? 4 : 8, ES = 16 / EK;
  const int off = (k / EK) * kTtLB + (k % EK) * ES;
  const int n[4] = {c, kTtCols + c, 2 * kTtCols + c, 3 * kTtCols + c};
  if (KIND == 0) {
    float w[4];
    w[0] = __uint_as_float((__float_as_uint(v.x) + 0x1000u) & 0xFFFFE000u);
    w[1] = __uint_as_float((__float_as_uint(v.y) + 0x1000u) & 0xFFFFE000u);
    const float rx = v.x - w[0], ry = v.y - w[1];
    w[2] = __uint_as_float((__float_as_uint(rx) + 0x1000u) & 0xFFFFE000u);
    w[3] = __uint_as_float((__float_as_uint(ry) + 0x1000u) & 0xFFFFE000u);
#pragma unroll
    for (int i = 0; i < 4; ++i)
      *reinterpret_cast<float *>(sB + off + (n[i] >> 3) * 128 + (n[i] & 7) * 16) = w[i];
  } else {
    unsigned short b[4];
    b[0] = (unsigned short)((__float_as_uint(v.x) + 0x8000u) >> 16);
    b[1] = (unsigned short)((__float_as_uint(v.y) + 0x8000u) >> 16);
    b[2] = (unsigned short)((__float_as_uint(v.x - umma::bf16_to_float(b[0])) + 0x8000u) >> 16);
    b[3] = (unsigned short)((__float_as_uint(v.y - umma::bf16_to_float(b[1])) + 0x8000u) >> 16);
#pragma unroll
    for (int i = 0; i < 4; ++i)
      *reinterpret_cast<unsigned short *>(sB + off + (n[i] >> 3) * 128 + (n[i] & 7) * 16) = b[i];
  }
}

__device__ inline void named_sync(int id, int threads) {
  asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(threads) : "memory");
}

template <int KIND>
__global__ void __launch_bounds__(kTtThreads, 1)
    k_trace_tc(Geom g, const int4 *__restrict__ units, const int *__restrict__ ucols,
               const int *__restrict__ uoff, const int2 *__restrict__ cunits,
               const int *__restrict__ coff, const int4 *__restrict__ chunks,
               const unsigned char *__restrict__ tiles, const int *__restrict__ route,
               float2 *__restrict__ gtr, const float2 *__restrict__ rawf, int nrhs,
               unsigned *ready, const unsigned *__restrict__ need, int *__restrict__ err,
               unsigned wait_limit) {
  constexpr uint32_t kIdN4 = KIND == 0 ? umma::idesc_tf32(128, 4 * kTtCols)
                                       : umma::idesc_bf16(128, 4 * kTtCols);
  constexpr uint32_t kIdN2 = KIND == 0 ? umma::idesc_tf32(128, 2 * kTtCols)
                                       : umma::idesc_bf16(128, 2 * kTtCols);
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  // fullA[a]: A bytes; emptyA[a]: MMA commit; full[s]: one arrival per B-producer warp;
  // empty[s]: MMA commit; accf[b]: MMA
  // commit; acce[b]: one arrival per epilogue warp; drain: final MMA commit
  __shared__ uint64_t fullA[kTtASlots], emptyA[kTtASlots], full[kTtSlots], empty[kTtSlots];
  __shared__ uint64_t accf[2], acce[2], drain;
  __shared__ uint32_t tmem_base;
  __shared__ int abort_flag;
  __shared__ int ready_flag[2];   // B producers: the last input check (alternating)
  __shared__ int pcol[2][kTtCols];   // B producers: column words of the unit being staged
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int b = (int)blockIdx.x;
  // this CTA's units and chunks (host-built streams)
  const int u_beg = __ldg(uoff + b), u_end = __ldg(uoff + b + 1);
  const int c_beg = __ldg(coff + b), c_end = __ldg(coff + b + 1);
  auto aborted = [&]() { return *reinterpret_cast<volatile int *>(&abort_flag) != 0; };
  auto fail = [&](int code) {
    atomicExch(err, code);
    *reinterpret_cast<volatile int *>(&abort_flag) = 1;
  };
  auto slotA = [&](int a) { return smem_raw + (size_t)a * kTtASlotBytes; };
  auto slotB = [&](int s) {
    return smem_raw + (size_t)kTtASlots * kTtASlotBytes + (size_t)s * kTtBSlotBytes;
  };
  const long long slot_stride = (long long)nrhs * g.nsub * g.T;

  if (tid == 0) {
    for (int a = 0; a < kTtASlots; ++a) {
      mbar_init(&fullA[a], 1);
      mbar_init(&emptyA[a], 1);
    }
    for (int s = 0; s < kTtSlots; ++s) {
      mbar_init(&full[s], kTtBWarps);
      mbar_init(&empty[s], 1);
    }
    for (int q = 0; q < 2; ++q) {
      mbar_init(&accf[q], 1);
      mbar_init(&acce[q], 4);
    }
    mbar_init(&drain, 1);
    abort_flag = 0;
    mbar_init_fence();
  }
  if (warp == kTtMmaWarp) {
    umma::tmem_alloc(&tmem_base, kTtTmemCols);
    umma::tmem_relinquish();
  }
  umma::fence_before_sync();
  __syncthreads();
  umma::fence_after_sync();
  const uint32_t tmem = tmem_base;

  if (warp == kTtAWarp) {
    // ---------------- A producer: the map tiles of this CTA's chunks, in order
    if (lane == 0) {
      int ci = 0;   // chunks issued
      for (int j = c_beg; j < c_end && !aborted(); ++j, ++ci) {
        const int4 dsc = __ldg(chunks + j);
        const int a = ci % kTtASlots;
        if (ci >= kTtASlots && !mbar_wait(&emptyA[a], ((ci / kTtASlots) - 1) & 1)) {
          fail(21);
          break;
        }
        if (aborted()) break;
        const uint32_t bytes = (uint32_t)(dsc.w & 0xFF) * kTtStep;
        mbar_arrive_expect_tx(&fullA[a], bytes);
        bulk_g2s(slotA(a), tiles + (long long)dsc.y * kTtStep, bytes, &fullA[a]);
      }
      // no copy may still be landing when the CTA leaves: wait for the last chunk of each slot
      for (int a = 0; a < kTtASlots && a < ci; ++a) {
        const int last = a + (ci - 1 - a) / kTtASlots * kTtASlots;
        if (!mbar_wait(&fullA[a], (last / kTtASlots) & 1)) atomicExch(err, 22);
      }
    }
  } else if (warp == kTtMmaWarp) {
    // ---------------- MMA issuer
    if (lane == 0) {
      const uint32_t lbo_a = 128u * 16u;
      const uint64_t dA = (uint64_t)kTtStep >> 4;        // one K-step of A (16-byte units)
      const uint64_t dC = (uint64_t)(2 * 128 * 16) >> 4; // one component of A
      const uint64_t dB = (uint64_t)kTtBStep >> 4;       // one K-step of B
      int ci = 0, mi = 0;   // chunks consumed, MMA units issued
      for (int ui = u_beg; ui < u_end && !aborted(); ++ui) {
        {
          const int nch = __ldg(cunits + ui).y;
          if (nch == 0) continue;
          const int q = mi & 1;
          if (mi >= 2 && !mbar_wait(&acce[q], ((mi >> 1) - 1) & 1)) { fail(23); break; }
          umma::fence_after_sync();
          const uint32_t d1 = tmem + (uint32_t)q * (8 * kTtCols), d2 = d1 + 4 * kTtCols;
          bool ok = true;
          for (int c = 0; c < nch; ++c, ++ci) {
            const int s = ci % kTtSlots, a = ci % kTtASlots;
            const int nks = __ldg(&chunks[c_beg + ci].w) & 0xFF;
            if (!mbar_wait(&full[s], (ci / kTtSlots) & 1) ||
                !mbar_wait(&fullA[a], (ci / kTtASlots) & 1)) {
              fail(24);
              ok = false;
              break;
            }
            if (aborted()) { ok = false; break; }
            umma::fence_after_sync();
            uint64_t ad = umma::smem_desc(umma::saddr(slotA(a)), lbo_a, 128);
            uint64_t bd = umma::smem_desc(umma::saddr(slotB(s)), (uint32_t)kTtLB, 128);
            for (int k = 0; k < nks; ++k) {
              const uint32_t acc = (c > 0 || k > 0) ? 1u : 0u;
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
            umma::mma_commit(&empty[s]);   // the slots are free once these MMAs have read them
            umma::mma_commit(&emptyA[a]);
          }
          if (!ok) break;
          umma::mma_commit(&accf[q]);
          ++mi;
        }
      }
      umma::mma_commit(&drain);
      if (!mbar_wait(&drain, 0)) atomicExch(err, 25);
    }
  } else if (warp >= 4) {
    // ---------------- B producers: inputs of this CTA's chunks, split into pieces
    // Dataflow instead of level barriers: before the first load of a unit's inputs, warp 4
    // waits until every trace solve routed into the unit's slots (l, X) has published
    // (ready[l nsub + X] == need[l nsub + X]).  Thread pt owns the pairs of consecutive inputs
    // p = pt + 256 i of every chunk (column p / kPairs, inputs 2 (p % kPairs) and the next): it
    // loads them from the trace slots into registers (L2 only: other CTAs wrote them) two chunks
    // ahead of their split, across unit and level boundaries, and splits them itself into the
    // ring slot, so the inputs never pass through shared memory.  The unit's column words sit in a
    // shared table (two, by unit parity), written by the readiness check.
    constexpr int kPairs = kTtKS * (KIND == 0 ? 8 : 16) / 2;   // input pairs per column
    constexpr int kPer = kTtCols * kPairs / kTtBThreads;        // pairs per thread and chunk
    const int pt = tid - 128;   // 0 .. kTtBThreads - 1
    // are the unit's inputs complete (every producer routed into its slots has published)?  Lane
    // c of warp 4 polls the slot of column c (all columns at once), `block` = until it is complete
    // (bounded) or once, and puts the column word into table `tab`; the answer goes to all
    // producer threads through a shared flag (two, alternating, so that a reader of one check
    // never races the next write).  The table of unit n is written only after every producer
    // thread has passed the check of unit n - 1, so after its loads of unit n - 2.
    int check_no = 0;
    auto inputs_ready = [&](const TtUnit &u, int tab, bool block) {
      const int fl = check_no++ & 1;
      if (warp == 4) {
        int ok = 1, col = -1;
        if (lane < u.ncol) {
          col = __ldg(ucols + u.col0 + lane);
          const long long sl = (long long)u.l * g.nsub + col % g.nsub;
          const unsigned want = __ldg(need + sl);
          uint32_t spins = 0;
          while (ld_acquire_gpu(ready + sl) < want) {
            if (!block) { ok = 0; break; }
            if (++spins > wait_limit || *reinterpret_cast<volatile int *>(err) != 0) {
              atomicExch(err, 4);
              *reinterpret_cast<volatile int *>(&abort_flag) = 1;
              break;   // go on (results are wrong, the host reports DDS_ETIMEOUT)
            }
            __nanosleep(32);
          }
        }
        pcol[tab][lane] = col;
        ok = __all_sync(0xffffffffu, ok);
        if (lane == 0) ready_flag[fl] = ok;
      }
      named_sync(2, kTtBThreads);
      return ready_flag[fl] != 0;
    };
    // load this thread's pairs of chunk `dsc` of unit `u` (column table `tab`); zeros where the
    // column or the input does not exist
    auto load = [&](float4 (&rb)[kPer], const int4 &dsc, const TtUnit &u, int tab) {
      const int live = dsc.w >> 8;
      const float2 *src0 = gtr + (long long)u.l * slot_stride + dsc.z;
      const int *cols = pcol[tab];
#pragma unroll
      for (int i = 0; i < kPer; ++i) {
        const int q = pt + i * kTtBThreads;
        const int c2 = q / kPairs, kk = 2 * (q % kPairs);
        rb[i] = make_float4(0.f, 0.f, 0.f, 0.f);
        if (c2 < u.ncol && kk < live)
          rb[i] = __ldcg(reinterpret_cast<const float4 *>(src0 + (long long)cols[c2] * g.T + kk));
      }
    };
    // Chunk `staged` is the next to load (into register buffer staged % 3), chunk ci the next to
    // split.  Loads run up to two chunks ahead.  A unit is entered only once its inputs are
    // complete, without waiting, except when its chunk is the one to split now (then nothing
    // earlier is pending in these threads, so the wait cannot hold up the trace solves it waits
    // for).
    const int nchunks = c_end - c_beg;
    int staged = 0, un = -1, hdr_at = -1;   // chunks loaded, ordinal of the loading unit
    int4 dP = nchunks > 0 ? __ldg(chunks + c_beg) : make_int4(0, 0, 0, 0);
    TtUnit uP{};
    float4 rb0[kPer], rb1[kPer], rb2[kPer];
    auto fill = [&](int ci) {
      while (staged < nchunks && staged <= ci + 2) {
        if ((dP.x >> 30) & 1) {   // first chunk of a unit
          if (hdr_at != staged) {
            uP = tt_unit(units, dP.x & 0x3FFFFFFF);
            hdr_at = staged;
          }
          if (!inputs_ready(uP, (un + 1) & 1, staged == ci)) break;
          ++un;
        }
        switch (staged % 3) {
          case 0: load(rb0, dP, uP, un & 1); break;
          case 1: load(rb1, dP, uP, un & 1); break;
          default: load(rb2, dP, uP, un & 1); break;
        }
        ++staged;
        if (staged < nchunks) dP = __ldg(chunks + c_beg + staged);
      }
    };
    // split chunk ci (held in rb) into B ring slot ci % 2; every K-step of the slot is written,
    // the MMAs read only the chunk's own
    auto split = [&](const float4 (&rb)[kPer], int ci) {
      const int s = ci % kTtSlots;
      if (ci >= kTtSlots && !aborted()) {
        // (after an abort no wait is made: the MMAs may have stopped consuming)
        int okw = 1;
        if (lane == 0) okw = mbar_wait(&empty[s], ((ci / kTtSlots) - 1) & 1) ? 1 : 0;
        okw = __shfl_sync(0xffffffffu, okw, 0);
        if (!okw && lane == 0) fail(26);
      }
      if (!aborted()) {
        unsigned char *sB = slotB(s);
#pragma unroll
        for (int i = 0; i < kPer; ++i) {
          const int q = pt + i * kTtBThreads;
          const int c2 = q / kPairs, kk = 2 * (q % kPairs);
          tt_put_b<KIND>(sB, kk, c2, make_float2(rb[i].x, rb[i].y));
          tt_put_b<KIND>(sB, kk + 1, c2, make_float2(rb[i].z, rb[i].w));
        }
      }
      fence_proxy_async();   // the generic writes of B before the MMAs' async reads
      __syncwarp();
      if (lane == 0) mbar_arrive(&full[s]);
    };
    for (int ci = 0; ci < nchunks; ci += 3) {
      fill(ci);
      split(rb0, ci);
      if (ci + 1 < nchunks) {
        fill(ci + 1);
        split(rb1, ci + 1);
      }
      if (ci + 2 < nchunks) {
        fill(ci + 2);
        split(rb2, ci + 2);
      }
    }
  } else {
    // ---------------- epilogue: row R of the unit's tile, every column
    const uint32_t lane_base = (uint32_t)(warp * 32) << 16;
    int mi = 0;
    for (int ui = u_beg; ui < u_end; ++ui) {
      {
        const int2 cu = __ldg(cunits + ui);
        const TtUnit u = tt_unit(units, cu.x);
        const int nch = cu.y;
        const int R = u.rt * 128 + warp * 32 + lane;
        int dout = -1, ro = 0, dst_off = 0;
#pragma unroll
        for (int d = 0; d < 6; ++d)
          if (d < g.nsides && R >= g.toff[d] && R < g.toff[d] + 2 * g.Lt[d]) {
            dout = d;
            ro = R - g.toff[d];
            dst_off = g.toff[d ^ 1] + ro;   // the same row of the receiver's side d ^ 1
          }
        const int lp = dout >= 0 ? __ldg(route + u.l * 6 + dout) : -1;
        // lane c holds the column word of column c (loaded before the accumulator wait)
        const int mycol = lane < u.ncol ? __ldg(ucols + u.col0 + lane) : -1;
        float2 out[kTtCols];
#pragma unroll
        for (int c = 0; c < kTtCols; ++c) out[c] = make_float2(0.f, 0.f);
        if (nch > 0) {
          const int q = mi & 1;
          int ok = 1;
          if (lane == 0) ok = (!aborted() && mbar_wait(&accf[q], (mi >> 1) & 1)) ? 1 : 0;
          ok = __shfl_sync(0xffffffffu, ok, 0);
          if (!ok && lane == 0 && !aborted()) fail(27);
          if (ok) {
            umma::fence_after_sync();
            const uint32_t d1 = tmem + lane_base + (uint32_t)q * (8 * kTtCols);
            const uint32_t d2 = d1 + 4 * kTtCols;
#pragma unroll
            for (int cg = 0; cg < kTtCols; cg += 8) {
              float x[8][8];
              umma::tmem_ld8(d1 + cg, x[0]);                   // A_re b0_re (+ A_re1 b0_re)
              umma::tmem_ld8(d1 + kTtCols + cg, x[1]);         // A_re b0_im
              umma::tmem_ld8(d1 + 2 * kTtCols + cg, x[2]);     // A_re0 b1_re
              umma::tmem_ld8(d1 + 3 * kTtCols + cg, x[3]);     // A_re0 b1_im
              umma::tmem_ld8(d2 + cg, x[4]);                   // A_im b0_re
              umma::tmem_ld8(d2 + kTtCols + cg, x[5]);
              umma::tmem_ld8(d2 + 2 * kTtCols + cg, x[6]);
              umma::tmem_ld8(d2 + 3 * kTtCols + cg, x[7]);
              umma::tmem_wait_ld();
#pragma unroll
              for (int i = 0; i < 8; ++i) {
                const float p_re = x[0][i] + x[2][i], p_im = x[1][i] + x[3][i];
                const float q_re = x[4][i] + x[6][i], q_im = x[5][i] + x[7][i];
                out[cg + i] = make_float2(p_re - q_im, p_im + q_re);
              }
            }
          }
          umma::fence_before_sync();
          __syncwarp();
          if (lane == 0) mbar_arrive(&acce[q]);
          ++mi;
        }
        // the raw own-source lines of this row (first sweep), then rows in pairs: lanes 2j and
        // 2j + 1 hold rows R and R + 1 of one side (sides have an even number of rows from an
        // even offset), so each exchanges one value per column pair with its partner and adds
        // two rows of one column with one 16-byte vector reduction
        const bool live = dout >= 0 && lp >= 0 && !aborted();
        if (u.raw) {
#pragma unroll
          for (int c = 0; c < kTtCols; ++c) {
            const int col = __shfl_sync(0xffffffffu, mycol, c);
            if (c < u.ncol && dout >= 0) {
              const float2 w = __ldg(rawf + (long long)col * g.T + R);
              out[c] = make_float2(out[c].x + w.x, out[c].y + w.y);
            }
          }
        }
        const bool odd = lane & 1;
        float2 *slot = gtr + (long long)(lp >= 0 ? lp : 0) * slot_stride + dst_off - (odd ? 1 : 0);
#pragma unroll
        for (int c = 0; c < kTtCols; c += 2) {
          const float2 mine = odd ? out[c + 1] : out[c];
          const float2 send = odd ? out[c] : out[c + 1];
          const float2 got = make_float2(__shfl_xor_sync(0xffffffffu, send.x, 1),
                                         __shfl_xor_sync(0xffffffffu, send.y, 1));
          const int cc = c + (odd ? 1 : 0);
          const int col = __shfl_sync(0xffffffffu, mycol, cc);
          if (live && cc < u.ncol) {
            const int X = col % g.nsub, rhs = col - X;   // rhs * nsub
            const int Y = sub_neighbour(g, X, dout);
            if (Y >= 0) {
              const float4 v = odd ? make_float4(got.x, got.y, mine.x, mine.y)
                                   : make_float4(mine.x, mine.y, got.x, got.y);
              red_add_f4(reinterpret_cast<float4 *>(slot + (long long)(rhs + Y) * g.T), v);
            }
          }
        }
        // each thread's reductions are performed before the unit is published
        __threadfence();
        // publish the unit: one count per (receiving slot, subdomain of the tile, side whose
        // rows lie in this row tile), as the host counted them into need[]; lane c of warp 0
        // takes column c when its subdomain differs from column c - 1's
        named_sync(1, 128);
        if (warp == 0) {
          const int X = mycol >= 0 ? mycol % g.nsub : -1;
          const int Xp = __shfl_up_sync(0xffffffffu, X, 1);
          if (X >= 0 && (lane == 0 || X != Xp)) {
            for (int d = 0; d < g.nsides; ++d) {
              if (g.toff[d] >= 128 * (u.rt + 1) || g.toff[d] + 2 * g.Lt[d] <= 128 * u.rt) continue;
              const int lq = __ldg(route + u.l * 6 + d), Y = sub_neighbour(g, X, d);
              if (lq >= 0 && Y >= 0) atomicAdd(ready + (long long)lq * g.nsub + Y, 1u);
            }
          }
        }
      }
    }
  }
  umma::fence_before_sync();
  __syncthreads();
  if (warp == kTtMmaWarp) {
    umma::fence_after_sync();
    umma::tmem_dealloc(tmem, kTtTmemCols);
  }
}

cudaError_t launch_trace_tc(cudaStream_t st, const Geom &g, int kind, const int4 *units,
                            const int *ucols, const int *uoff, const int2 *cunits,
                            const int *coff, const int4 *chunks, int nunits, int G,
                            const unsigned char *tiles, const int *route, float2 *gtr,
                            const float2 *rawf, int nrhs, unsigned *ready, const unsigned *need,
                            int nslots, int *err, unsigned wait_limit) {
  if (nunits <= 0) return cudaSuccess;
  TtShape t;
  if (!tt_shape(g, kind, &t)) return cudaErrorInvalidValue;
  static bool done0[64] = {false}, done1[64] = {false};
  cudaError_t e = kind == 0 ? smem_limit_once(k_trace_tc<0>, done0)
                            : smem_limit_once(k_trace_tc<1>, done1);
  if (e != cudaSuccess) return e;
  int dev = 0, nsm = 0, per_sm = 0;
  if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
  if ((e = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
  // one CTA per SM (it owns the whole tensor memory), all resident: the streams were dealt for G
  if (G != nsm) return cudaErrorInvalidConfiguration;
  e = kind == 0 ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_trace_tc<0>, kTtThreads, t.smem)
                : cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_trace_tc<1>, kTtThreads, t.smem);
  if (e != cudaSuccess) return e;
  if (per_sm < 1) return cudaErrorInvalidConfiguration;
  e = cudaMemsetAsync(ready, 0, (size_t)nslots * sizeof(unsigned), st);
  if (e != cudaSuccess) return e;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)G);
  cfg.blockDim = dim3(kTtThreads);
  cfg.dynamicSmemBytes = t.smem;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeCooperative;
  attr[0].val.cooperative = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  if (kind == 0)
    return cudaLaunchKernelEx(&cfg, k_trace_tc<0>, g, units, ucols, uoff, cunits, coff, chunks,
                              tiles, route, gtr, rawf, nrhs, ready, need, err, wait_limit);
  return cudaLaunchKernelEx(&cfg, k_trace_tc<1>, g, units, ucols, uoff, cunits, coff, chunks,
                            tiles, route, gtr, rawf, nrhs, ready, need, err, wait_limit);
}

}  // namespace dds
