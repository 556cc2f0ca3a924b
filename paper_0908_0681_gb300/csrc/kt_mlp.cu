// BF16 tensor-core GEMM (tcgen05, TMEM accumulator) and the small MLP built on it.
//
// kt_gemm_bf16: C[M][N] (FP32) = A[M][K] . B[N][K]^T with A, B in BF16, row-major,
// both K-contiguous. One CTA of 128 threads computes a 128 x BN tile (BN <= 256, a
// multiple of 16): the K dimension is staged through shared memory 64 columns at a
// time in the canonical no-swizzle K-major layout of the tensor core (8 x 16-byte
// core matrices; LBO = 128 B between core matrices along K, SBO = 1024 B between
// 8-row groups), one thread issues tcgen05.mma (kind::f16, M = 128, N = BN, K = 16
// per instruction) into a TMEM accumulator, tcgen05.commit arrives on an mbarrier,
// and every wait on that mbarrier is bounded (on timeout the kernel records an
// error flag and stops issuing). The epilogue reads TMEM with tcgen05.ld (each
// warp its 32 lanes = 32 rows) and writes FP32 to global memory.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <stdint.h>

#include "kt_internal.h"

namespace kt {
namespace mlp {

constexpr int BM = 128;       // rows per CTA (TMEM lanes)
constexpr int BK = 64;        // K columns per shared-memory stage
constexpr int MAX_BN = 256;   // accumulator columns
constexpr int WAIT_LIMIT = 1 << 21;  // polls of 32+ ns each: the wait gives up after ~0.1-1 s

__device__ __forceinline__ uint32_t smem_u32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

// Shared-memory matrix descriptor (no swizzle, K-major).
__device__ __forceinline__ uint64_t smem_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr & 0x3FFFF) >> 4);        // start address
  d |= (uint64_t)((lbo & 0x3FFFF) >> 4) << 16;    // leading-dimension byte offset (along K)
  d |= (uint64_t)((sbo & 0x3FFFF) >> 4) << 32;    // stride-dimension byte offset (8-row groups)
  d |= (uint64_t)1 << 46;                         // descriptor version of tcgen05
  // base offset 0, absolute LBO mode 0, layout type 0 = no swizzle
  return d;
}

// Instruction descriptor of kind::f16: FP32 accumulator, BF16 A and B, both K-major.
__device__ __forceinline__ uint32_t instr_desc(int M, int N) {
  return (1u << 4)                     // D format FP32
         | (1u << 7)                   // A format BF16
         | (1u << 10)                  // B format BF16
         | ((uint32_t)(N >> 3) << 17)  // N / 8
         | ((uint32_t)(M >> 4) << 24); // M / 16
}

__device__ __forceinline__ void mbar_init(uint32_t addr, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(addr), "r"(count));
}

// Bounded wait on an mbarrier phase (non-blocking polls with a short sleep);
// false on timeout.
__device__ __forceinline__ bool mbar_wait(uint32_t addr, uint32_t phase) {
  for (int it = 0; it < WAIT_LIMIT; ++it) {
    uint32_t done;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.test_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(done)
        : "r"(addr), "r"(phase)
        : "memory");
    if (done) return true;
    __nanosleep(32);
  }
  return false;
}

// Copy a [rows x 64] BF16 chunk (row stride ld elements, columns k0 .. k0+63, zero
// beyond kmax or beyond the valid rows) into the core-matrix layout at dst.
__device__ __forceinline__ void stage_tile(uint8_t *dst, const __nv_bfloat16 *src, int ld, int row0, int rows_valid,
                                           int rows, int k0, int kmax) {
  // one 16-byte piece (8 BF16 of one row) per iteration
  const int pieces = rows * (BK / 8);
  for (int p = threadIdx.x; p < pieces; p += blockDim.x) {
    const int r = p / (BK / 8), kg = p - r * (BK / 8);
    const int k = k0 + kg * 8;
    uint4 v = make_uint4(0, 0, 0, 0);
    if (r < rows_valid && k < kmax) v = *reinterpret_cast<const uint4 *>(src + (size_t)(row0 + r) * ld + k);
    // core matrix (r / 8, kg): 8 rows x 16 bytes, row r % 8
    uint8_t *c = dst + (size_t)(r >> 3) * 1024 + kg * 128 + (r & 7) * 16;
    *reinterpret_cast<uint4 *>(c) = v;
  }
}

__global__ void __launch_bounds__(128) gemm_bf16_kernel(const __nv_bfloat16 *__restrict__ A, int lda,
                                                        const __nv_bfloat16 *__restrict__ B, int ldb, float *C, int ldc,
                                                        int M, int N, int K, int BN, int *err) {
  extern __shared__ __align__(1024) uint8_t smem[];
  uint8_t *sA = smem;                      // 128 x 64 BF16 = 16 KB
  uint8_t *sB = smem + BM * BK * 2;        // BN x 64 BF16 <= 32 KB
  __shared__ __align__(8) uint64_t mbar;
  __shared__ uint32_t tmem_base_sh;
  __shared__ int abort_sh;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int m0 = blockIdx.x * BM, n0 = blockIdx.y * BN;
  const int bn = (N - n0) < BN ? (N - n0) : BN;  // multiple of 16 (N is)
  const uint32_t ncols = 256;                    // power of two >= bn
  const uint32_t mb = smem_u32(&mbar);
  if (threadIdx.x == 0) {
    mbar_init(mb, 1);
    abort_sh = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_base_sh)),
                 "r"(ncols));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = tmem_base_sh;
  const uint32_t idesc = instr_desc(BM, bn);
  uint32_t phase = 0;
  for (int k0 = 0; k0 < K; k0 += BK) {
    stage_tile(sA, A, lda, m0, M - m0, BM, k0, K);
    stage_tile(sB, B, ldb, n0, bn, bn, k0, K);
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    __syncthreads();
    if (threadIdx.x == 0 && !abort_sh) {
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      const int ksteps = (K - k0) < BK ? (K - k0) / 16 : BK / 16;
      for (int s = 0; s < ksteps; ++s) {
        const uint64_t ad = smem_desc(smem_u32(sA) + s * 256, 128, 1024);
        const uint64_t bd = smem_desc(smem_u32(sB) + s * 256, 128, 1024);
        const uint32_t acc = (k0 > 0 || s > 0) ? 1u : 0u;
        asm volatile(
            "{\n\t.reg .pred p;\n\t"
            "setp.ne.b32 p, %4, 0;\n\t"
            "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(tmem),
            "l"(ad), "l"(bd), "r"(idesc), "r"(acc));
      }
      asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(mb)
                   : "memory");
    }
    // every thread waits for the MMAs that read this stage before it is overwritten
    if (!abort_sh) {
      const bool ok = mbar_wait(mb, phase);
      if (!ok) {
        abort_sh = 1;
        if (lane == 0) atomicExch(err, 1);
      }
    }
    phase ^= 1u;
    __syncthreads();
    if (abort_sh) {
      // give the MMAs of this stage one more bounded wait before the accumulator is freed
      mbar_wait(mb, phase ^ 1u);
      break;
    }
  }
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  if (!abort_sh) {
    // epilogue: warp w reads TMEM lanes 32w .. 32w+31 (rows), 32 columns at a time
    const int row = m0 + warp * 32 + lane;
    for (int c0 = 0; c0 < bn; c0 += 32) {
      uint32_t r[32];
      const uint32_t taddr = tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)c0;
      asm volatile(
          "tcgen05.ld.sync.aligned.32x32b.x32.b32 "
          "{%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15, "
          "%16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];"
          : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
            "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
            "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
            "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
          : "r"(taddr));
      asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
      if (row < M) {
#pragma unroll
        for (int j = 0; j < 32; ++j)
          if (c0 + j < bn) C[(size_t)row * ldc + n0 + c0 + j] = __uint_as_float(r[j]);
      }
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(ncols));
}

}  // namespace mlp

// C = A . B^T; requirements checked by the caller-facing entry point.
int gemm_bf16(const void *A, int lda, const void *B, int ldb, float *C, int ldc, int M, int N, int K, int *err,
              cudaStream_t st) {
  const int BN = N <= mlp::MAX_BN ? N : 128;
  const size_t smem = (size_t)mlp::BM * mlp::BK * 2 + (size_t)BN * mlp::BK * 2;
  static bool attr = false;
  if (!attr) {
    cudaFuncSetAttribute(mlp::gemm_bf16_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, 64 * 1024);
    attr = true;
  }
  dim3 grid((unsigned)((M + mlp::BM - 1) / mlp::BM), (unsigned)((N + BN - 1) / BN));
  mlp::gemm_bf16_kernel<<<grid, 128, smem, st>>>((const __nv_bfloat16 *)A, lda, (const __nv_bfloat16 *)B, ldb, C, ldc,
                                                 M, N, K, BN, err);
  return (int)cudaGetLastError();
}

}  // namespace kt

extern "C" kt_status kt_gemm_bf16(const void *A, int32_t lda, const void *B, int32_t ldb, float *C, int32_t ldc,
                                  int32_t M, int32_t N, int32_t K, int32_t *err, void *stream) {
  if (!A || !B || !C || !err || M < 1 || N < 16 || K < 16 || (N % 16) || (K % 16) || lda < K || ldb < K || ldc < N ||
      (lda % 8) || (ldb % 8) || ((uintptr_t)A % 16) || ((uintptr_t)B % 16))
    return KT_EINVAL;
  return kt::gemm_bf16(A, lda, B, ldb, C, ldc, M, N, K, err, (cudaStream_t)stream) == 0 ? KT_OK : KT_ECUDA;
}
