// Building blocks of the tcgen05 kernels (apply_tc.cu, gemm_tc.cu): operand
// formats, the 128-byte-swizzled K-major shared-memory layout and its matrix
// descriptor, the instruction descriptor, bounded mbarrier waits, MMA issue
// and TMEM loads, all as inline PTX for sm_103a.
#pragma once
#include <cuda_bf16.h>
#include <cstdint>

#include "common.cuh"

namespace t2s2 {
namespace tc {

// Iterations of a bounded mbarrier wait (each a try_wait with its own
// hardware time slice) before the kernel gives up and reports an error.
constexpr unsigned kSpinLimit = 1u << 24;

// Operand traits: element bytes, K per MMA, format code of the descriptor.
template <int P>
struct Op;
template <>
struct Op<T2S2_BF16_REFINE> {
  static constexpr int kBytes = 2, kMmaK = 16, kFmt = 1;  // BF16
  __device__ static void store(unsigned char* p, double v) {
    *reinterpret_cast<__nv_bfloat16*>(p) = __double2bfloat16(v);
  }
  // eight values rounded and packed into one 16-byte chunk, in K order
  __device__ static uint4 pack16(const double (&v)[8]) {
    uint32_t w[4];
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const uint32_t lo = __bfloat16_as_ushort(__double2bfloat16(v[2 * i]));
      const uint32_t hi = __bfloat16_as_ushort(__double2bfloat16(v[2 * i + 1]));
      w[i] = lo | (hi << 16);
    }
    return make_uint4(w[0], w[1], w[2], w[3]);
  }
};
template <>
struct Op<T2S2_TF32_REFINE> {
  static constexpr int kBytes = 4, kMmaK = 8, kFmt = 2;  // TF32
  __device__ static void store(unsigned char* p, double v) {
    uint32_t r;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"((float)v));
    *reinterpret_cast<uint32_t*>(p) = r;
  }
  // four values rounded into one 16-byte chunk, in K order
  __device__ static uint4 pack16(const double (&v)[4]) {
    uint32_t w[4];
#pragma unroll
    for (int i = 0; i < 4; ++i) asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(w[i]) : "f"((float)v[i]));
    return make_uint4(w[0], w[1], w[2], w[3]);
  }
};

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

// Byte offset of element (row, k) of a K-major operand tile of `rows` rows,
// split along K into 128-byte swizzle rows: K-block kb = k / (128 / E) holds
// rows / 8 groups of 8 rows x 128 bytes (1024 bytes each); inside a group the
// 16-byte chunk c of row r sits at chunk position c ^ (r mod 8).
template <int E>
__device__ __forceinline__ uint32_t sw128_off(int row, int k, int rows) {
  constexpr int W = 128 / E;  // elements per swizzle row
  const int kb = k / W, bo = (k % W) * E;
  const int r8 = row & 7;
  return (uint32_t)(kb * (rows * 128) + (row >> 3) * 1024 + r8 * 128 + (((bo >> 4) ^ r8) << 4) + (bo & 15));
}

// Shared-memory matrix descriptor for a 128-byte-swizzled K-major tile:
// start address >> 4, leading offset 16 B (unused for this layout), stride
// between 8-row groups 1024 B, descriptor version 1, swizzle mode 128 B.
__device__ __forceinline__ uint64_t sdesc_sw128(uint32_t addr) {
  uint64_t d = 0;
  d |= (uint64_t)((addr >> 4) & 0x3FFFu);
  d |= (uint64_t)1u << 16;
  d |= (uint64_t)(1024u >> 4) << 32;
  d |= (uint64_t)1u << 46;
  d |= (uint64_t)2u << 61;
  return d;
}

// Instruction descriptor: FP32 accumulator (bits 4-5), A and B formats (bits
// 7-9, 10-12), both K-major (bits 15, 16 clear), N >> 3 (bits 17-22), M >> 4
// (bits 24-28).
__host__ __device__ constexpr uint32_t make_idesc(int fmt, int M, int N) {
  return (1u << 4) | ((uint32_t)fmt << 7) | ((uint32_t)fmt << 10) | ((uint32_t)(N >> 3) << 17) |
         ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity) {
  for (unsigned it = 0; it < kSpinLimit; ++it) {
    uint32_t done;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.b32 %0, 1, 0, p;\n\t}\n"
        : "=r"(done)
        : "r"(bar), "r"(parity)
        : "memory");
    if (done) return true;
  }
  return false;
}

template <int P>
__device__ __forceinline__ void issue_mma(uint32_t tmem, uint64_t da, uint64_t db, uint32_t idesc, uint32_t acc);

template <>
__device__ __forceinline__ void issue_mma<T2S2_BF16_REFINE>(uint32_t tmem, uint64_t da, uint64_t db,
                                                            uint32_t idesc, uint32_t acc) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(tmem),
      "l"(da), "l"(db), "r"(idesc), "r"(acc)
      : "memory");
}

template <>
__device__ __forceinline__ void issue_mma<T2S2_TF32_REFINE>(uint32_t tmem, uint64_t da, uint64_t db,
                                                            uint32_t idesc, uint32_t acc) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(tmem),
      "l"(da), "l"(db), "r"(idesc), "r"(acc)
      : "memory");
}

__device__ __forceinline__ void tmem_ld32(uint32_t taddr, uint32_t (&v)[32]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 "
      "{%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
      "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
      : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),
        "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]),
        "=r"(v[15]), "=r"(v[16]), "=r"(v[17]), "=r"(v[18]), "=r"(v[19]), "=r"(v[20]), "=r"(v[21]),
        "=r"(v[22]), "=r"(v[23]), "=r"(v[24]), "=r"(v[25]), "=r"(v[26]), "=r"(v[27]), "=r"(v[28]),
        "=r"(v[29]), "=r"(v[30]), "=r"(v[31])
      : "r"(taddr)
      : "memory");
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}


__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void tmem_alloc(uint32_t slot_smem, uint32_t ncols) {
  asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(slot_smem), "r"(ncols)
               : "memory");
  asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}

__device__ __forceinline__ void tmem_dealloc(uint32_t tmem, uint32_t ncols) {
  asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(ncols) : "memory");
}

__device__ __forceinline__ void mma_commit(uint32_t bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar)
               : "memory");
}

// One-dimensional bulk copy (TMA, no tensor map) of `bytes` (a multiple of 16)
// from global memory at `src` (16-byte aligned) into shared memory at `dst`
// (16-byte aligned), completing `bytes` transactions on the mbarrier `bar`.
__device__ __forceinline__ void bulk_g2s(uint32_t dst, const void* src, uint32_t bytes, uint32_t bar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
               ::"r"(dst), "l"(src), "r"(bytes), "r"(bar)
               : "memory");
}

// Arrive once on `bar` and announce `bytes` of transactions to wait for.
__device__ __forceinline__ void mbar_arrive_expect_tx(uint32_t bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}

__device__ __forceinline__ void fence_smem_to_async() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}
__device__ __forceinline__ void fence_before_sync() {
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void fence_after_sync() {
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}

}  // namespace tc
}  // namespace t2s2
