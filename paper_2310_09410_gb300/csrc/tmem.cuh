// Tensor memory (tcgen05) used as per-lane storage: a CTA allocates columns
// of the SM's 128-lane x 512-column array of 32-bit cells; warp w reaches the
// 32 lanes of quadrant w % 4, and lane l of the warp reads and writes tensor
// lane 32 (w % 4) + l.  Address = (lane << 16) | column.
#pragma once

namespace opf {

// One warp: allocate `cols` columns (a power of 2, >= 32), base address to
// *dst_smem; the permit is given up so that other CTAs on the SM can allocate.
__device__ __forceinline__ void tm_alloc(unsigned *dst_smem, int cols) {
    const unsigned a = (unsigned)__cvta_generic_to_shared(dst_smem);
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(a), "r"(cols) : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}
// The allocating warp frees the columns.
__device__ __forceinline__ void tm_dealloc(unsigned taddr, int cols) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(cols) : "memory");
}
// Order tensor-memory accesses of different warps around a thread barrier.
__device__ __forceinline__ void tm_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tm_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tm_wait_ld() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }
__device__ __forceinline__ void tm_wait_st() { asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory"); }

// 4 consecutive columns of the thread's lane (the values are usable after tm_wait_ld).
__device__ __forceinline__ void tm_ld4(unsigned taddr, float (&v)[4]) {
    unsigned r[4];
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x4.b32 {%0, %1, %2, %3}, [%4];"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
                 : "r"(taddr)
                 : "memory");
#pragma unroll
    for (int e = 0; e < 4; ++e) v[e] = __uint_as_float(r[e]);
}
__device__ __forceinline__ void tm_st4(unsigned taddr, const float (&v)[4]) {
    asm volatile("tcgen05.st.sync.aligned.32x32b.x4.b32 [%0], {%1, %2, %3, %4};" ::"r"(taddr),
                 "r"(__float_as_uint(v[0])), "r"(__float_as_uint(v[1])), "r"(__float_as_uint(v[2])),
                 "r"(__float_as_uint(v[3]))
                 : "memory");
}

}  // namespace opf
