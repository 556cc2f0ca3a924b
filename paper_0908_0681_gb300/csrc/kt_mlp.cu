// BF16 tensor-core GEMM (tcgen05, TMEM accumulator) and the small MLP built on it.
//
// kt_gemm_bf16: C[M][N] (FP32) = A[M][K] . B[N][K]^T with A, B in BF16, row-major,
// both K-contiguous. One CTA of 128 threads computes a 128 x BN tile (BN <= 256, a
// multiple of 16): the K dimension is staged through shared memory 64 columns at a
// time in the no-swizzle K-major layout of the tensor core (8 x 16-byte core
// matrices), one thread issues tcgen05.mma (kind::f16, M = 128, N = BN, K = 16 per
// instruction) into a TMEM accumulator, tcgen05.commit arrives on mbarriers, and every
// wait on an mbarrier is bounded (on timeout the kernel records an error flag and
// stops issuing). The epilogue reads TMEM with tcgen05.ld (each warp its 32 lanes =
// 32 rows) and writes FP32 to global memory. Two kernels: gemm_bf16_tma_kernel feeds
// three stages by TMA (the default), gemm_bf16_kernel stages one chunk at a time with
// ordinary loads (LBO = 128 B along K, SBO = 1024 B between 8-row groups) when the
// driver offers no tensor-map encoder.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <math.h>
#include <stdint.h>

#include <new>

#include "kt_internal.h"

namespace kt {
namespace mlp {

constexpr int BM = 128;       // rows per CTA (TMEM lanes)
constexpr int BK = 64;        // K columns per shared-memory stage
constexpr int MAX_BN = 256;   // accumulator columns
constexpr int MAX_SPLITS = 16;  // K slices of the weight-gradient products (K = batch)
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
                                                        int M, int N, int K, int BN, int kslice, int *err) {
  extern __shared__ __align__(1024) uint8_t smem[];
  uint8_t *sA = smem;                      // 128 x 64 BF16 = 16 KB
  uint8_t *sB = smem + BM * BK * 2;        // BN x 64 BF16 <= 32 KB
  __shared__ __align__(8) uint64_t mbar;
  __shared__ uint32_t tmem_base_sh;
  __shared__ int abort_sh;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int m0 = blockIdx.x * BM, n0 = blockIdx.y * BN;
  // split K: this CTA reduces over [kb, K) of its slice and writes partial sums to slab z of C
  const int kb = blockIdx.z * kslice;
  A += kb;
  B += kb;
  C += (size_t)blockIdx.z * M * ldc;
  K = min(K - kb, kslice);
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

// TMA-fed variant. Each 64-column chunk of K arrives as eight 2-D tensor-map boxes of
// 8 columns x rows (16-byte rows), one per group of 8 K columns, so that a box is a
// column of 8 x 16-byte core matrices: the same no-swizzle K-major layout as above with
// LBO = rows * 16 B between core matrices along K and SBO = 128 B between 8-row groups.
// STAGES chunks are in flight: thread 0 issues the copies (cp.async.bulk.tensor; an
// mbarrier per stage counts their bytes), thread 32 issues the MMAs of a stage once its
// bytes have landed and commits them to the stage's "empty" mbarrier, which the copy of
// the chunk STAGES later waits for. Every wait is bounded.
constexpr int STAGES = 3;

__device__ __forceinline__ void mbar_expect_tx(uint32_t addr, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(addr), "r"(bytes) : "memory");
}

__device__ __forceinline__ void tma_load_2d(uint32_t dst, const CUtensorMap *map, int x, int y, uint32_t mbar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];"
      ::"r"(dst), "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(mbar)
      : "memory");
}

__global__ void __launch_bounds__(128) gemm_bf16_tma_kernel(const __grid_constant__ CUtensorMap ta,
                                                            const __grid_constant__ CUtensorMap tb, float *C, int ldc,
                                                            int M, int N, int K, int BN, int kslice, int *err) {
  extern __shared__ __align__(1024) uint8_t smem[];
  __shared__ __align__(8) uint64_t full[STAGES], empty[STAGES], done;
  __shared__ uint32_t tmem_base_sh;
  __shared__ int abort_sh;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int stage_a = BM * BK * 2, stage_b = BN * BK * 2;
  const uint32_t sa0 = smem_u32(smem), sb0 = sa0 + STAGES * stage_a;
  const int m0 = blockIdx.x * BM, n0 = blockIdx.y * BN;
  const int bn = (N - n0) < BN ? (N - n0) : BN;
  const int kb = blockIdx.z * kslice, ke = min(K, kb + kslice);
  const int nchunks = (ke - kb + BK - 1) / BK;
  C += (size_t)blockIdx.z * M * ldc;
  const uint32_t ncols = 256;
  if (threadIdx.x == 0) {
    for (int s = 0; s < STAGES; ++s) {
      mbar_init(smem_u32(&full[s]), 1);
      mbar_init(smem_u32(&empty[s]), 1);
    }
    mbar_init(smem_u32(&done), 1);
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
  if (threadIdx.x == 0) {
    // copies: chunk c into stage c % STAGES once the MMAs of chunk c - STAGES are done
    for (int c = 0; c < nchunks; ++c) {
      const int s = c % STAGES, u = c / STAGES;
      if (c >= STAGES && !mbar_wait(smem_u32(&empty[s]), (uint32_t)((u - 1) & 1))) {
        abort_sh = 1;
        atomicExch(err, 1);
        break;
      }
      const uint32_t fb = smem_u32(&full[s]);
      mbar_expect_tx(fb, (uint32_t)(stage_a + stage_b));
      const int k = kb + c * BK;
      for (int g = 0; g < BK / 8; ++g) {
        tma_load_2d(sa0 + s * stage_a + g * (BM * 16), &ta, k + 8 * g, m0, fb);
        tma_load_2d(sb0 + s * stage_b + g * (BN * 16), &tb, k + 8 * g, n0, fb);
      }
    }
  } else if (threadIdx.x == 32) {
    const uint32_t idesc = instr_desc(BM, bn);
    for (int c = 0; c < nchunks; ++c) {
      const int s = c % STAGES, u = c / STAGES;
      if (*(volatile int *)&abort_sh || !mbar_wait(smem_u32(&full[s]), (uint32_t)(u & 1))) {
        abort_sh = 1;
        atomicExch(err, 1);
        break;
      }
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      const int k = kb + c * BK;
      const int ksteps = (ke - k) < BK ? (ke - k) / 16 : BK / 16;
      for (int t = 0; t < ksteps; ++t) {
        // K step t: core-matrix columns 2t and 2t+1 of the stage (boxes 2t and 2t+1)
        const uint64_t ad = smem_desc(sa0 + s * stage_a + 2 * t * (BM * 16), BM * 16, 128);
        const uint64_t bd = smem_desc(sb0 + s * stage_b + 2 * t * (BN * 16), BN * 16, 128);
        const uint32_t acc = (c > 0 || t > 0) ? 1u : 0u;
        asm volatile(
            "{\n\t.reg .pred p;\n\t"
            "setp.ne.b32 p, %4, 0;\n\t"
            "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(tmem),
            "l"(ad), "l"(bd), "r"(idesc), "r"(acc));
      }
      asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                       smem_u32(&empty[s]))
                   : "memory");
    }
    // completion of every MMA issued (also after an abort, before the accumulator is freed)
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(&done))
                 : "memory");
  }
  if (!mbar_wait(smem_u32(&done), 0u)) {
    abort_sh = 1;
    if (lane == 0) atomicExch(err, 1);
  }
  __syncwarp();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  __syncthreads();
  if (!abort_sh) {
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

// cuTensorMapEncodeTiled from the driver (through the runtime), or null if unavailable.
PFN_cuTensorMapEncodeTiled_v12000 tensor_map_encoder() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  static bool tried = false;
  if (!tried) {
    tried = true;
    void *p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
    cudaGetLastError();
  }
  return fn;
}

int gemm_splits(int K, int splits) {
  const int kslice = ((K + splits - 1) / splits + mlp::BK - 1) / mlp::BK * mlp::BK;
  return (K + kslice - 1) / kslice;
}

// C = A . B^T; requirements checked by the caller-facing entry point. The TMA-fed kernel
// when the driver provides tensor maps, else the kernel that stages with ordinary loads.
int gemm_bf16(const void *A, int lda, const void *B, int ldb, float *C, int ldc, int M, int N, int K, int *err,
              void *st_, int splits) {
  cudaStream_t st = (cudaStream_t)st_;
  // column tile: the whole N when it fits the accumulator, narrower (128, then 64 columns)
  // while the grid would have fewer than 64 CTAs, so that small batches still spread out
  const int gm = (M + mlp::BM - 1) / mlp::BM, gz = gemm_splits(K, splits);
  int BN = N <= mlp::MAX_BN ? N : 128;
  for (const int w : {128, 64})
    if (BN > w && gm * ((N + BN - 1) / BN) * gz < 64) BN = w;
  const int kslice_t = ((K + splits - 1) / splits + mlp::BK - 1) / mlp::BK * mlp::BK;
  if (PFN_cuTensorMapEncodeTiled_v12000 enc = tensor_map_encoder()) {
    CUtensorMap ta, tb;
    const cuuint64_t da[2] = {(cuuint64_t)K, (cuuint64_t)M}, db[2] = {(cuuint64_t)K, (cuuint64_t)N};
    const cuuint64_t sa[1] = {(cuuint64_t)lda * 2}, sb[1] = {(cuuint64_t)ldb * 2};
    const cuuint32_t ba[2] = {8, (cuuint32_t)mlp::BM}, bb[2] = {8, (cuuint32_t)BN}, es[2] = {1, 1};
    if (enc(&ta, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void *>(A), da, sa, ba, es, CU_TENSOR_MAP_INTERLEAVE_NONE,
            CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) ==
            CUDA_SUCCESS &&
        enc(&tb, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void *>(B), db, sb, bb, es, CU_TENSOR_MAP_INTERLEAVE_NONE,
            CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) ==
            CUDA_SUCCESS) {
      const size_t smem_t = (size_t)mlp::STAGES * ((size_t)mlp::BM * mlp::BK * 2 + (size_t)BN * mlp::BK * 2);
      static bool attr_t = false;
      if (!attr_t) {
        cudaFuncSetAttribute(mlp::gemm_bf16_tma_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)(mlp::STAGES * (mlp::BM + mlp::MAX_BN) * mlp::BK * 2));
        attr_t = true;
      }
      dim3 grid((unsigned)gm, (unsigned)((N + BN - 1) / BN), (unsigned)((K + kslice_t - 1) / kslice_t));
      mlp::gemm_bf16_tma_kernel<<<grid, 128, smem_t, st>>>(ta, tb, C, ldc, M, N, K, BN, kslice_t, err);
      return (int)cudaGetLastError();
    }
  }
  const size_t smem = (size_t)mlp::BM * mlp::BK * 2 + (size_t)BN * mlp::BK * 2;
  static bool attr = false;
  if (!attr) {
    cudaFuncSetAttribute(mlp::gemm_bf16_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, 64 * 1024);
    attr = true;
  }
  // every slice holds at least one 64-column chunk of K (its offset keeps rows 16-byte aligned)
  const int kslice = ((K + splits - 1) / splits + mlp::BK - 1) / mlp::BK * mlp::BK;
  dim3 grid((unsigned)((M + mlp::BM - 1) / mlp::BM), (unsigned)((N + BN - 1) / BN), (unsigned)((K + kslice - 1) / kslice));
  mlp::gemm_bf16_kernel<<<grid, 128, smem, st>>>((const __nv_bfloat16 *)A, lda, (const __nv_bfloat16 *)B, ldb, C, ldc,
                                                 M, N, K, BN, kslice, err);
  return (int)cudaGetLastError();
}

}  // namespace kt

// ---------------------------------------------------------------------------
// The surrogate network y = w3 . relu(W2 relu(W1 x + b1) + b2) + b3 (hidden 256):
// BF16 operands on the tensor cores (kt_gemm_bf16), FP32 accumulation, FP32
// master weights, biases, output layer and Adam state.
// ---------------------------------------------------------------------------
namespace kt {
namespace mlp {

constexpr int H = 256;

__global__ void to_bf16_kernel(const float *__restrict__ src, __nv_bfloat16 *dst, long long n) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) dst[i] = __float2bfloat16_rn(src[i]);
}

// dst[c][r] = src[r][c] (FP32 -> BF16), src [R][C] row-major
__global__ void transpose_bf16_kernel(const float *__restrict__ src, __nv_bfloat16 *dst, int R, int C) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= (long long)R * C) return;
  const int r = (int)(i / C), c = (int)(i - (long long)r * C);
  dst[(size_t)c * R + r] = __float2bfloat16_rn(src[i]);
}

// dst[c][r] = src[r][c] for BF16 matrices
__global__ void transpose_b16_kernel(const __nv_bfloat16 *__restrict__ src, __nv_bfloat16 *dst, int R, int C) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= (long long)R * C) return;
  const int r = (int)(i / C), c = (int)(i - (long long)r * C);
  dst[(size_t)c * R + r] = src[i];
}

// H1 = relu(Z1 + b1) in BF16 (row-major; with HT also transposed)
__global__ void act1_kernel(const float *__restrict__ Z1, const float *__restrict__ b1, __nv_bfloat16 *H1,
                            __nv_bfloat16 *H1T, int B) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= (long long)B * H) return;
  const int b = (int)(i / H), j = (int)(i - (long long)b * H);
  const __nv_bfloat16 h = __float2bfloat16_rn(fmaxf(Z1[i] + b1[j], 0.f));
  H1[i] = h;
  if (H1T) H1T[(size_t)j * B + b] = h;
}

// y_b = w3 . relu(Z2_b + b2) + b3 (warp per row); H2 keeps relu(...) when given
__global__ void out_kernel(const float *__restrict__ Z2, const float *__restrict__ b2, const float *__restrict__ w3,
                           const float *__restrict__ b3, float *H2, float *y, int B) {
  const int row = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
  if (row >= B) return;
  float acc = 0.f;
  for (int j = lane; j < H; j += 32) {
    const float h = fmaxf(Z2[(size_t)row * H + j] + b2[j], 0.f);
    if (H2) H2[(size_t)row * H + j] = h;
    acc = fmaf(h, w3[j], acc);
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  if (lane == 0) y[row] = acc + b3[0];
}

// dy = 2 (y - t) / B; loss += (y - t)^2 / B
__global__ void loss_kernel(const float *__restrict__ y, const float *__restrict__ t, float *dy, float *loss, int B) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  float c = 0.f;
  if (b < B) {
    const float r = y[b] - t[b];
    dy[b] = 2.f * r / (float)B;
    c = r * r / (float)B;
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) c += __shfl_xor_sync(0xffffffffu, c, o);
  if ((threadIdx.x & 31) == 0 && c != 0.f) atomicAdd(loss, c);
}

// dZ2 = dy w3^T masked by relu'(Z2 + b2), BF16 in both layouts
__global__ void dz2_kernel(const float *__restrict__ Z2, const float *__restrict__ b2, const float *__restrict__ w3,
                           const float *__restrict__ dy, __nv_bfloat16 *dZ2, __nv_bfloat16 *dZ2T, int B) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= (long long)B * H) return;
  const int b = (int)(i / H), j = (int)(i - (long long)b * H);
  const float d = (Z2[i] + b2[j] > 0.f) ? dy[b] * w3[j] : 0.f;
  const __nv_bfloat16 v = __float2bfloat16_rn(d);
  dZ2[i] = v;
  dZ2T[(size_t)j * B + b] = v;
}

// Column sums over the batch, gw3_j = sum_b dy_b H2_bj, gb2_j = sum_b dZ2_bj and
// gb3 = sum_b dy_b (FP32), in two deterministic passes: one block of H threads per chunk
// of ROWS rows writes the chunk's sums, then one block adds the chunks in order.
constexpr int ROWS = 128;
__global__ void out_grads_part_kernel(const float *__restrict__ Z2, const float *__restrict__ b2,
                                      const float *__restrict__ w3, const float *__restrict__ H2,
                                      const float *__restrict__ dy, float *pw3, float *pb2, float *pb3, int B) {
  __shared__ float sh[H];
  const int c = blockIdx.x, j = threadIdx.x;
  const int r0 = c * ROWS, r1 = min(B, r0 + ROWS);
  float a = 0.f, s = 0.f;
  for (int b = r0; b < r1; ++b) {
    const float d = dy[b];
    a = fmaf(d, H2[(size_t)b * H + j], a);
    if (Z2[(size_t)b * H + j] + b2[j] > 0.f) s = fmaf(d, w3[j], s);
  }
  pw3[(size_t)c * H + j] = a;
  pb2[(size_t)c * H + j] = s;
  sh[j] = (j < ROWS && r0 + j < r1) ? dy[r0 + j] : 0.f;
  __syncthreads();
  for (int o = H / 2; o > 0; o >>= 1) {
    if (j < o) sh[j] += sh[j + o];
    __syncthreads();
  }
  if (j == 0) pb3[c] = sh[0];
}
__global__ void out_grads_sum_kernel(const float *__restrict__ pw3, const float *__restrict__ pb2,
                                     const float *__restrict__ pb3, float *gw3, float *gb2, float *gb3, int nc) {
  const int j = threadIdx.x;
  float a = 0.f, s = 0.f, t = 0.f;
  for (int c = 0; c < nc; ++c) {
    a += pw3[(size_t)c * H + j];
    s += pb2[(size_t)c * H + j];
    if (j == 0) t += pb3[c];
  }
  gw3[j] = a;
  gb2[j] = s;
  if (j == 0) gb3[0] = t;
}

// Sum of split-K partial products: out[i] = sum over slabs s of part[s n + i], in order.
__global__ void splitk_sum_kernel(const float *__restrict__ part, float *out, int S, long long n) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  float a = 0.f;
  for (int s = 0; s < S; ++s) a += part[(size_t)s * n + i];
  out[i] = a;
}

// dZ1 = dH1 masked by relu'(Z1 + b1): BF16 transposed [H][B]; gb1 column sums (FP32)
__global__ void dz1_kernel(const float *__restrict__ dH1, const float *__restrict__ Z1, const float *__restrict__ b1,
                           __nv_bfloat16 *dZ1T, int B) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= (long long)B * H) return;
  const int b = (int)(i / H), j = (int)(i - (long long)b * H);
  const float d = (Z1[i] + b1[j] > 0.f) ? dH1[i] : 0.f;
  dZ1T[(size_t)j * B + b] = __float2bfloat16_rn(d);
}
__global__ void gb1_part_kernel(const float *__restrict__ dH1, const float *__restrict__ Z1,
                                const float *__restrict__ b1, float *pb1, int B) {
  const int c = blockIdx.x, j = threadIdx.x;
  const int r0 = c * ROWS, r1 = min(B, r0 + ROWS);
  float s = 0.f;
  for (int b = r0; b < r1; ++b)
    if (Z1[(size_t)b * H + j] + b1[j] > 0.f) s += dH1[(size_t)b * H + j];
  pb1[(size_t)c * H + j] = s;
}

// Adam (Kingma & Ba 2015, Algorithm 1) on the packed FP32 parameters
__global__ void adam_kernel(float *p, const float *__restrict__ g, float *m, float *v, long long n, float lr, float bc1,
                            float bc2) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const float gi = g[i];
  const float mi = 0.9f * m[i] + 0.1f * gi;
  const float vi = 0.999f * v[i] + 0.001f * gi * gi;
  m[i] = mi;
  v[i] = vi;
  p[i] -= lr * (mi / bc1) / (sqrtf(vi / bc2) + 1e-8f);
}

inline unsigned blocks(long long n, int t = 256) { return (unsigned)((n + t - 1) / t); }

}  // namespace mlp
}  // namespace kt

struct kt_mlp {
  int n_in = 0, maxB = 0, step = 0, lastB = 0;
  long long P = 0;
  void *mem = nullptr;
  float *p = nullptr, *g = nullptr, *m = nullptr, *v = nullptr;
  float *W1, *b1, *W2, *b2, *w3, *b3;
  float *gW1, *gb1, *gW2, *gb2, *gw3, *gb3;
  __nv_bfloat16 *W1b, *W2b, *W2Tb;
  float *Z1, *Z2, *H2, *dH1, *y, *dy, *loss;
  __nv_bfloat16 *H1b, *H1Tb, *dZ2b, *dZ2Tb, *dZ1Tb, *XTb;
  float *part;               // split-K slabs of the weight gradients
  float *pw3, *pb2, *pb3, *pb1;  // per-chunk column sums
  int *err;
};

namespace kt {

int mlp_inputs(const kt_mlp *n) { return n->n_in; }
int mlp_max_batch(const kt_mlp *n) { return n->maxB; }

int mlp_refresh_bf16(kt_mlp *n, cudaStream_t st) {
  using namespace mlp;
  to_bf16_kernel<<<blocks((long long)H * n->n_in), 256, 0, st>>>(n->W1, n->W1b, (long long)H * n->n_in);
  to_bf16_kernel<<<blocks((long long)H * H), 256, 0, st>>>(n->W2, n->W2b, (long long)H * H);
  transpose_bf16_kernel<<<blocks((long long)H * H), 256, 0, st>>>(n->W2, n->W2Tb, H, H);
  return (int)cudaGetLastError();
}

// y[B] = network(X [B][n_in] BF16); with train, keeps what the backward pass needs
int mlp_forward(kt_mlp *n, const void *X, int B, float *y, bool train, void *st_) {
  using namespace mlp;
  cudaStream_t st = (cudaStream_t)st_;
  int rc = gemm_bf16(X, n->n_in, n->W1b, n->n_in, n->Z1, H, B, H, n->n_in, n->err, st);
  if (rc) return rc;
  act1_kernel<<<blocks((long long)B * H), 256, 0, st>>>(n->Z1, n->b1, n->H1b, train ? n->H1Tb : nullptr, B);
  rc = gemm_bf16(n->H1b, H, n->W2b, H, n->Z2, H, B, H, H, n->err, st);
  if (rc) return rc;
  out_kernel<<<blocks((long long)B * 32), 256, 0, st>>>(n->Z2, n->b2, n->w3, n->b3, train ? n->H2 : nullptr, y, B);
  return (int)cudaGetLastError();
}

}  // namespace kt

extern "C" {

kt_status kt_mlp_create(int32_t n_in, int32_t max_batch, kt_mlp **out) {
  using namespace kt::mlp;
  if (!out || n_in < 16 || (n_in % 16) || max_batch < 16 || (max_batch % 16)) return KT_EINVAL;
  *out = nullptr;
  kt_mlp *n = new (std::nothrow) kt_mlp();
  if (!n) return KT_ENOMEM;
  n->n_in = n_in;
  n->maxB = max_batch;
  n->P = (long long)H * n_in + H + (long long)H * H + H + H + 1;
  const size_t B = max_batch, P = n->P;
  size_t off = 0;
  auto take = [&](size_t bytes) {
    const size_t at = off;
    off += (bytes + 255) / 256 * 256;
    return at;
  };
  const size_t o_p = take(P * 4), o_g = take(P * 4), o_m = take(P * 4), o_v = take(P * 4),
               o_w1b = take((size_t)H * n_in * 2), o_w2b = take((size_t)H * H * 2), o_w2t = take((size_t)H * H * 2),
               o_z1 = take(B * H * 4), o_z2 = take(B * H * 4), o_h2 = take(B * H * 4), o_dh1 = take(B * H * 4),
               o_y = take(B * 4), o_dy = take(B * 4), o_loss = take(4), o_h1 = take(B * H * 2), o_h1t = take(B * H * 2),
               o_dz2 = take(B * H * 2), o_dz2t = take(B * H * 2), o_dz1t = take(B * H * 2),
               o_xt = take(B * (size_t)n_in * 2), o_err = take(4),
               o_part = take((size_t)kt::mlp::MAX_SPLITS * H * (n_in > H ? n_in : H) * 4),
               o_pw3 = take((B / ROWS + 1) * H * 4), o_pb2 = take((B / ROWS + 1) * H * 4), o_pb3 = take((B / ROWS + 1) * 4),
               o_pb1 = take((B / ROWS + 1) * H * 4);
  if (cudaMalloc(&n->mem, off) != cudaSuccess) {
    cudaGetLastError();
    delete n;
    return KT_ENOMEM;
  }
  cudaMemset(n->mem, 0, off);
  char *b = (char *)n->mem;
  n->p = (float *)(b + o_p);
  n->g = (float *)(b + o_g);
  n->m = (float *)(b + o_m);
  n->v = (float *)(b + o_v);
  float *q = n->p, *r = n->g;
  n->W1 = q; n->gW1 = r; q += (size_t)H * n_in; r += (size_t)H * n_in;
  n->b1 = q; n->gb1 = r; q += H; r += H;
  n->W2 = q; n->gW2 = r; q += (size_t)H * H; r += (size_t)H * H;
  n->b2 = q; n->gb2 = r; q += H; r += H;
  n->w3 = q; n->gw3 = r; q += H; r += H;
  n->b3 = q; n->gb3 = r;
  n->part = (float *)(b + o_part);
  n->pw3 = (float *)(b + o_pw3);
  n->pb2 = (float *)(b + o_pb2);
  n->pb3 = (float *)(b + o_pb3);
  n->pb1 = (float *)(b + o_pb1);
  n->W1b = (__nv_bfloat16 *)(b + o_w1b);
  n->W2b = (__nv_bfloat16 *)(b + o_w2b);
  n->W2Tb = (__nv_bfloat16 *)(b + o_w2t);
  n->Z1 = (float *)(b + o_z1);
  n->Z2 = (float *)(b + o_z2);
  n->H2 = (float *)(b + o_h2);
  n->dH1 = (float *)(b + o_dh1);
  n->y = (float *)(b + o_y);
  n->dy = (float *)(b + o_dy);
  n->loss = (float *)(b + o_loss);
  n->H1b = (__nv_bfloat16 *)(b + o_h1);
  n->H1Tb = (__nv_bfloat16 *)(b + o_h1t);
  n->dZ2b = (__nv_bfloat16 *)(b + o_dz2);
  n->dZ2Tb = (__nv_bfloat16 *)(b + o_dz2t);
  n->dZ1Tb = (__nv_bfloat16 *)(b + o_dz1t);
  n->XTb = (__nv_bfloat16 *)(b + o_xt);
  n->err = (int *)(b + o_err);
  if (cudaDeviceSynchronize() != cudaSuccess) {
    cudaGetLastError();
    kt_mlp_destroy(n);
    return KT_ECUDA;
  }
  *out = n;
  return KT_OK;
}

kt_status kt_mlp_num_params(const kt_mlp *n, int64_t *count) {
  if (!n || !count) return KT_EINVAL;
  *count = n->P;
  return KT_OK;
}

kt_status kt_mlp_set_params(kt_mlp *n, const float *host) {
  if (!n || !host) return KT_EINVAL;
  if (cudaMemcpy(n->p, host, (size_t)n->P * 4, cudaMemcpyHostToDevice) != cudaSuccess) return KT_ECUDA;
  cudaMemset(n->m, 0, (size_t)n->P * 4);
  cudaMemset(n->v, 0, (size_t)n->P * 4);
  n->step = 0;
  if (kt::mlp_refresh_bf16(n, 0) != 0) return KT_ECUDA;
  return cudaDeviceSynchronize() == cudaSuccess ? KT_OK : KT_ECUDA;
}

kt_status kt_mlp_get_params(kt_mlp *n, float *host) {
  if (!n || !host) return KT_EINVAL;
  return cudaMemcpy(host, n->p, (size_t)n->P * 4, cudaMemcpyDeviceToHost) == cudaSuccess ? KT_OK : KT_ECUDA;
}

kt_status kt_mlp_get_grads(kt_mlp *n, float *host) {
  if (!n || !host) return KT_EINVAL;
  return cudaMemcpy(host, n->g, (size_t)n->P * 4, cudaMemcpyDeviceToHost) == cudaSuccess ? KT_OK : KT_ECUDA;
}

kt_status kt_mlp_forward(kt_mlp *n, const void *X, int32_t B, float *y, void *stream) {
  if (!n || !X || !y || B < 1 || B > n->maxB || ((uintptr_t)X % 16)) return KT_EINVAL;
  return kt::mlp_forward(n, X, B, y, false, stream) == 0 ? KT_OK : KT_ECUDA;
}

kt_status kt_mlp_backward(kt_mlp *n, const void *X, const float *t, int32_t B, float *loss, void *stream) {
  using namespace kt::mlp;
  if (!n || !X || !t || B < 16 || (B % 16) || B > n->maxB || ((uintptr_t)X % 16)) return KT_EINVAL;
  cudaStream_t st = (cudaStream_t)stream;
  const int nin = n->n_in;
  if (kt::mlp_forward(n, X, B, n->y, true, st) != 0) return KT_ECUDA;
  cudaMemsetAsync(n->loss, 0, 4, st);
  loss_kernel<<<blocks(B), 256, 0, st>>>(n->y, t, n->dy, n->loss, B);
  dz2_kernel<<<blocks((long long)B * H), 256, 0, st>>>(n->Z2, n->b2, n->w3, n->dy, n->dZ2b, n->dZ2Tb, B);
  const int nc = (B + ROWS - 1) / ROWS;
  out_grads_part_kernel<<<nc, H, 0, st>>>(n->Z2, n->b2, n->w3, n->H2, n->dy, n->pw3, n->pb2, n->pb3, B);
  out_grads_sum_kernel<<<1, H, 0, st>>>(n->pw3, n->pb2, n->pb3, n->gw3, n->gb2, n->gb3, nc);
  // weight gradients reduce over the batch: split K = B over several CTAs, then sum the slabs
  const int S = kt::gemm_splits(B, MAX_SPLITS);
  // dW2 = dZ2^T H1: A = dZ2T [H][B], B-operand = H1T [H][B]
  if (kt::gemm_bf16(n->dZ2Tb, B, n->H1Tb, B, n->part, H, H, H, B, n->err, st, MAX_SPLITS)) return KT_ECUDA;
  splitk_sum_kernel<<<blocks((long long)H * H), 256, 0, st>>>(n->part, n->gW2, S, (long long)H * H);
  // dH1 = dZ2 W2: A = dZ2 [B][H], B-operand = W2T [H(in)][H(out)]
  if (kt::gemm_bf16(n->dZ2b, H, n->W2Tb, H, n->dH1, H, B, H, H, n->err, st)) return KT_ECUDA;
  dz1_kernel<<<blocks((long long)B * H), 256, 0, st>>>(n->dH1, n->Z1, n->b1, n->dZ1Tb, B);
  gb1_part_kernel<<<nc, H, 0, st>>>(n->dH1, n->Z1, n->b1, n->pb1, B);
  splitk_sum_kernel<<<1, H, 0, st>>>(n->pb1, n->gb1, nc, H);
  // dW1 = dZ1^T X: A = dZ1T [H][B], B-operand = XT [n_in][B]
  transpose_b16_kernel<<<blocks((long long)B * nin), 256, 0, st>>>((const __nv_bfloat16 *)X, n->XTb, B, nin);
  if (kt::gemm_bf16(n->dZ1Tb, B, n->XTb, B, n->part, nin, H, nin, B, n->err, st, MAX_SPLITS)) return KT_ECUDA;
  splitk_sum_kernel<<<blocks((long long)H * nin), 256, 0, st>>>(n->part, n->gW1, S, (long long)H * nin);
  if (loss) cudaMemcpyAsync(loss, n->loss, 4, cudaMemcpyDeviceToDevice, st);
  n->lastB = B;
  return cudaGetLastError() == cudaSuccess ? KT_OK : KT_ECUDA;
}

kt_status kt_mlp_get_tape(kt_mlp *n, int32_t B, float *z1, uint16_t *h1, float *z2, float *dy, uint16_t *dz2,
                          float *dh1, uint16_t *dz1) {
  using namespace kt::mlp;
  if (!n || B < 1 || B != n->lastB) return KT_EINVAL;
  if (cudaDeviceSynchronize() != cudaSuccess) return KT_ECUDA;
  const size_t bh = (size_t)B * H;
  const struct {
    void *dst;
    const void *src;
    size_t bytes;
  } cp[] = {{z1, n->Z1, bh * 4}, {h1, n->H1b, bh * 2}, {z2, n->Z2, bh * 4}, {dy, n->dy, (size_t)B * 4},
            {dz2, n->dZ2b, bh * 2}, {dh1, n->dH1, bh * 4}, {dz1, n->dZ1Tb, bh * 2}};
  for (const auto &c : cp)
    if (c.dst && cudaMemcpy(c.dst, c.src, c.bytes, cudaMemcpyDeviceToHost) != cudaSuccess) return KT_ECUDA;
  return KT_OK;
}

kt_status kt_mlp_adam(kt_mlp *n, float lr, void *stream) {
  using namespace kt::mlp;
  if (!n || !(lr > 0.f)) return KT_EINVAL;
  cudaStream_t st = (cudaStream_t)stream;
  n->step += 1;
  const float bc1 = 1.f - powf(0.9f, (float)n->step), bc2 = 1.f - powf(0.999f, (float)n->step);
  adam_kernel<<<blocks(n->P), 256, 0, st>>>(n->p, n->g, n->m, n->v, n->P, lr, bc1, bc2);
  if (kt::mlp_refresh_bf16(n, st) != 0) return KT_ECUDA;
  return cudaGetLastError() == cudaSuccess ? KT_OK : KT_ECUDA;
}

kt_status kt_mlp_error(kt_mlp *n, int32_t *out) {
  if (!n || !out) return KT_EINVAL;
  if (cudaDeviceSynchronize() != cudaSuccess) return KT_ECUDA;
  return cudaMemcpy(out, n->err, 4, cudaMemcpyDeviceToHost) == cudaSuccess ? KT_OK : KT_ECUDA;
}

void kt_mlp_destroy(kt_mlp *n) {
  if (!n) return;
  if (n->mem) cudaFree(n->mem);
  delete n;
}

}  // extern "C"

extern "C" kt_status kt_gemm_bf16(const void *A, int32_t lda, const void *B, int32_t ldb, float *C, int32_t ldc,
                                  int32_t M, int32_t N, int32_t K, int32_t *err, void *stream) {
  if (!A || !B || !C || !err || M < 1 || N < 16 || K < 16 || (N % 16) || (K % 16) || lda < K || ldb < K || ldc < N ||
      (lda % 8) || (ldb % 8) || ((uintptr_t)A % 16) || ((uintptr_t)B % 16))
    return KT_EINVAL;
  return kt::gemm_bf16(A, lda, B, ldb, C, ldc, M, N, K, err, stream) == 0 ? KT_OK : KT_ECUDA;
}
