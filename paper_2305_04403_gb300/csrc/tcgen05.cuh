// tcgen05.cuh -- inline-PTX building blocks for the 5th-generation tensor
// cores of sm_100-family GPUs (tcgen05.mma with the accumulator in tensor
// memory), used by the network kernels:
//   * tensor-memory allocation (one warp), loads of accumulator rows into
//     registers, and the fences that order them against thread barriers;
//   * shared-memory matrix descriptors for the canonical K-major layout
//     without swizzle;
//   * the instruction descriptor of a BF16 x BF16 -> FP32 product;
//   * an mbarrier that tcgen05.commit arrives on, waited on with a bound.
//
// Canonical K-major layout without swizzle (used for every operand here):
// the matrix (R rows x K columns, BF16) is cut into core matrices of 8 rows
// x 8 columns; a core matrix is 128 contiguous bytes (its 8 rows of 16
// bytes); core matrices adjacent along K are `lbo` bytes apart and groups
// of 8 rows `sbo` bytes apart.  Here lbo = 128 and sbo = (K / 8) * 128:
//     byte offset of (r, k) = (r / 8) * sbo + (k / 8) * 128 + (r % 8) * 16 + (k % 8) * 2.
// One tcgen05.mma of kind::f16 consumes K = 16, i.e. two core matrices
// along K: the descriptor of k-block kb starts at base + 256 * kb.
//
// The same bytes read as an MN-major operand (the transposed matrix: M or N
// along the 16-byte rows, K along the 8-row groups) need no copy: its core
// matrices are the same 8 x 16-byte blocks.  Without swizzle the MN-major
// descriptor takes the distance between core matrices adjacent along K (the
// stored matrix's row-group stride, `sbo` above) as its leading offset and
// the distance between core matrices adjacent along MN (128 bytes) as its
// stride offset (measured: the other assignment gives wrong products); k-block
// kb (16 rows of the stored matrix) starts at base + 2 * sbo * kb.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace wob {
namespace tc {

__device__ __forceinline__ uint32_t smem_addr(const void* p)
{
    return (uint32_t)__cvta_generic_to_shared(p);
}

// Byte offset of element (r, k) of a K-major canonical matrix with K columns.
__device__ __forceinline__ uint32_t kmajor_offset(int r, int k, int K)
{
    return (uint32_t)((r >> 3) * (K / 8) * 128 + (k >> 3) * 128 + (r & 7) * 16 + (k & 7) * 2);
}

// Shared-memory matrix descriptor: start address, leading- and
// stride-dimension byte offsets (all >> 4), descriptor version 1 (bits
// 46-47), no base offset, relative leading offset, no swizzle (bits 61-63).
__device__ __forceinline__ uint64_t smem_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo)
{
    uint64_t d = (uint64_t)((saddr & 0x3FFFFu) >> 4);
    d |= (uint64_t)((lbo >> 4) & 0x3FFFu) << 16;
    d |= (uint64_t)((sbo >> 4) & 0x3FFFu) << 32;
    d |= (uint64_t)1 << 46;
    return d;
}

// Instruction descriptor of kind::f16: FP32 accumulator (bits 4-5 = 1), A
// and B BF16 (bits 7-9 and 10-12 = 1), A and B K-major (bits 15, 16 = 0) or
// MN-major (1), N >> 3 in bits 17-22, M >> 4 in bits 24-28.
__host__ __device__ constexpr uint32_t idesc_bf16_f32(int M, int N, bool a_mn = false,
                                                      bool b_mn = false)
{
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)a_mn << 15) | ((uint32_t)b_mn << 16) |
           ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

// D[tmem] (+)= A[smem] * B[smem]^T for one K = 16 block; issued by one thread.
__device__ __forceinline__ void mma_bf16(uint32_t d_tmem, uint64_t a_desc, uint64_t b_desc,
                                         uint32_t idesc, bool accumulate)
{
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n"
        :
        : "r"(d_tmem), "l"(a_desc), "l"(b_desc), "r"(idesc), "r"((uint32_t)accumulate)
        : "memory");
}

// The mbarrier at `mbar` receives one arrival when every tcgen05.mma this
// thread issued before has completed.
__device__ __forceinline__ void commit(uint32_t mbar)
{
    asm volatile(
        "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(
            mbar)
        : "memory");
}

__device__ __forceinline__ void fence_before_sync()
{
    asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
}
__device__ __forceinline__ void fence_after_sync()
{
    asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
}
// Generic-proxy writes to shared memory become visible to the tensor cores.
__device__ __forceinline__ void fence_proxy_async()
{
    asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
}

// Tensor-memory allocation of `ncols` columns (a power of two >= 32) by one
// whole warp; the address is written to shared memory at `dst`.
__device__ __forceinline__ void tmem_alloc(uint32_t dst, uint32_t ncols)
{
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(dst),
                 "r"(ncols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n" ::: "memory");
}
__device__ __forceinline__ void tmem_free(uint32_t taddr, uint32_t ncols)
{
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(taddr),
                 "r"(ncols)
                 : "memory");
}

// 16 consecutive FP32 columns of the calling thread's tensor-memory lane
// (warp w of the CTA reads lanes 32 (w % 4) .. + 31; `taddr` carries the
// warp's lane base in bits 16-31 and the first column in bits 0-15).
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float (&v)[16])
{
    uint32_t r[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 "
        "{%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];\n"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
          "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]),
          "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr)
        : "memory");
#pragma unroll
    for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}
__device__ __forceinline__ void tmem_wait_ld()
{
    asm volatile("tcgen05.wait::ld.sync.aligned;\n" ::: "memory");
}

// Barrier of the `count` threads that use named barrier `id` (1..15).
__device__ __forceinline__ void bar_sync(int id, int count)
{
    asm volatile("bar.sync %0, %1;\n" ::"r"(id), "r"(count) : "memory");
}
// As bar_sync, returning whether any of the threads passed true.
__device__ __forceinline__ bool bar_sync_or(int id, int count, bool v)
{
    uint32_t r;
    asm volatile(
        "{\n\t.reg .pred p, q;\n\t"
        "setp.ne.u32 q, %1, 0;\n\t"
        "bar.red.or.pred p, %2, %3, q;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}\n"
        : "=r"(r)
        : "r"((uint32_t)v), "r"(id), "r"(count)
        : "memory");
    return r != 0;
}

__device__ __forceinline__ void mbar_init(uint32_t mbar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(mbar), "r"(count) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
}

// Wait for the phase with parity `parity` of the mbarrier to complete; gives
// up after `limit` polls and returns false (the caller records an error and
// winds down without waiting again).
__device__ __forceinline__ bool mbar_wait(uint32_t mbar, uint32_t parity, uint32_t limit)
{
    for (uint32_t i = 0; i < limit; ++i) {
        uint32_t done;
        asm volatile(
            "{\n\t.reg .pred p;\n\t"
            "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
            "selp.u32 %0, 1, 0, p;\n\t}\n"
            : "=r"(done)
            : "r"(mbar), "r"(parity)
            : "memory");
        if (done) return true;
    }
    return false;
}

}  // namespace tc
}  // namespace wob
