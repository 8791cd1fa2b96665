// Dense tensor-core rate of this GPU for the split-product piece types, measured the way the
// substitution and trace kernels use the tensor cores: tcgen05.mma.cta_group::1 with M = 128,
// N = 256, K-major operands in shared memory (no swizzle), FP32 accumulation in tensor memory.
// One CTA per SM; one thread issues `iters` back-to-back MMAs on fixed operands into one
// accumulator and commits them to an mbarrier.  The operands are finite non-zero values (every
// 32-bit word 0x3F803F80: two BF16 ones, or an FP32 value near 1), so that the data-dependent
// power draw resembles a real product.  The result is the ceiling the roofline fractions of the
// tensor-core kernels can be read against, next to the nominal one.
#include "async_copy.cuh"
#include "dds_internal.cuh"
#include "umma.cuh"

namespace dds {

namespace {

constexpr int kRateN = 256;
constexpr int kRateA = 128 * 32;      // one K-step of A: 128 rows x 32 bytes (8 TF32 / 16 BF16)
constexpr int kRateB = kRateN * 32;   // one K-step of B

template <int KIND>
__global__ void __launch_bounds__(128, 1) k_mma_rate(int iters, int *__restrict__ err) {
  __shared__ __align__(1024) unsigned char sm[kRateA + kRateB];
  __shared__ uint64_t bar;
  __shared__ uint32_t tbase;
  const int tid = threadIdx.x;
  for (int i = tid; i < (kRateA + kRateB) / 16; i += blockDim.x)
    reinterpret_cast<uint4 *>(sm)[i] = make_uint4(0x3F803F80u, 0x3F803F80u, 0x3F803F80u, 0x3F803F80u);
  if (tid == 0) {
    mbar_init(&bar, 1);
    mbar_init_fence();
  }
  if (tid < 32) {
    umma::tmem_alloc(&tbase, kRateN);
    umma::tmem_relinquish();
  }
  fence_proxy_async();   // the operand writes before the MMAs' async reads
  umma::fence_before_sync();
  __syncthreads();
  umma::fence_after_sync();
  const uint32_t tmem = tbase;
  if (tid == 0) {
    // core matrices of 8 rows x 16 bytes: the two K-adjacent ones 16 * rows bytes apart, 8-row
    // groups 128 bytes apart
    const uint64_t ad = umma::smem_desc(umma::saddr(sm), 128u * 16u, 128u);
    const uint64_t bd = umma::smem_desc(umma::saddr(sm + kRateA), (uint32_t)kRateN * 16u, 128u);
    constexpr uint32_t id = KIND == 0 ? umma::idesc_tf32(128, kRateN) : umma::idesc_bf16(128, kRateN);
    for (int i = 0; i < iters; ++i) {
      if (KIND == 0)
        umma::mma_tf32(tmem, ad, bd, id, i > 0 ? 1u : 0u);
      else
        umma::mma_bf16(tmem, ad, bd, id, i > 0 ? 1u : 0u);
    }
    umma::mma_commit(&bar);
    if (!mbar_wait(&bar, 0)) atomicExch(err, 30);
  }
  umma::fence_before_sync();
  __syncthreads();
  if (tid < 32) {
    umma::fence_after_sync();
    umma::tmem_dealloc(tmem, kRateN);
  }
}

}  // namespace

cudaError_t measure_mma_rate(int kind, int iters, int *err, double *flops, float *ms) {
  int dev = 0, nsm = 0;
  cudaError_t e;
  if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
  if ((e = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
  cudaStream_t st;
  if ((e = cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking)) != cudaSuccess) return e;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if ((e = cudaEventCreate(&e0)) == cudaSuccess && (e = cudaEventCreate(&e1)) == cudaSuccess) {
    auto launch = [&](int n) {
      if (kind == 0)
        k_mma_rate<0><<<nsm, 128, 0, st>>>(n, err);
      else
        k_mma_rate<1><<<nsm, 128, 0, st>>>(n, err);
      return cudaGetLastError();
    };
    // a warm-up launch, then the timed one
    if ((e = launch(iters / 8 + 1)) == cudaSuccess && (e = cudaEventRecord(e0, st)) == cudaSuccess &&
        (e = launch(iters)) == cudaSuccess && (e = cudaEventRecord(e1, st)) == cudaSuccess &&
        (e = cudaEventSynchronize(e1)) == cudaSuccess)
      e = cudaEventElapsedTime(ms, e0, e1);
    const int K = kind == 0 ? 8 : 16;
    *flops = 2.0 * 128 * kRateN * K * (double)iters * nsm;
  }
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  cudaStreamDestroy(st);
  return e;
}

}  // namespace dds
