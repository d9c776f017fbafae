// Tensor memory (TMEM) used as a per-thread store: single-instruction PTX wrappers for the
// tcgen05 allocation, 32x32b loads and stores, waits and fences.
//
// A warp reaches the 32 TMEM lanes of its quadrant (warp index within its warpgroup, i.e.
// warp index mod 4); with the 32x32b shape thread t of the warp reads and writes lane
// (quadrant base + t), and .x4 moves four consecutive 32-bit columns (one Q4: four cells of a
// row).  An address is (lane << 16) + column, relative to the allocation's base.  tcgen05.ld
// and tcgen05.st complete asynchronously: a load's registers are valid after tcgen05.wait::ld,
// and data stored is read back only after tcgen05.wait::st.  All of these are executed by
// whole warps (.sync.aligned), from warp-uniform control flow.
#pragma once

#include "fdtd_seg.cuh"

namespace fdtd {
namespace seg {

// allocate `cols` columns (a power of two >= 32) for this CTA; one whole warp executes it and
// the TMEM address lands in shared memory at dst
template <uint32_t cols>
__device__ __forceinline__ void tm_alloc(uint32_t* dst) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_u32(dst)),
                 "r"(cols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}
// release them (one whole warp, after every access of the CTA has completed)
template <uint32_t cols>
__device__ __forceinline__ void tm_dealloc(uint32_t taddr) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(cols)
                 : "memory");
}
__device__ __forceinline__ void tm_fence_before() {
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void tm_fence_after() {
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void tm_st(uint32_t taddr, const Q4& q) {
    asm volatile("tcgen05.st.sync.aligned.32x32b.x4.b32 [%0], {%1, %2, %3, %4};" ::"r"(taddr),
                 "f"(q.v[0]), "f"(q.v[1]), "f"(q.v[2]), "f"(q.v[3])
                 : "memory");
}
__device__ __forceinline__ void tm_st(uint32_t taddr, const float* v) {
    asm volatile("tcgen05.st.sync.aligned.32x32b.x4.b32 [%0], {%1, %2, %3, %4};" ::"r"(taddr),
                 "f"(v[0]), "f"(v[1]), "f"(v[2]), "f"(v[3])
                 : "memory");
}
__device__ __forceinline__ void tm_ld(uint32_t taddr, Q4& q) {
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x4.b32 {%0, %1, %2, %3}, [%4];"
                 : "=f"(q.v[0]), "=f"(q.v[1]), "=f"(q.v[2]), "=f"(q.v[3])
                 : "r"(taddr)
                 : "memory");
}
__device__ __forceinline__ void tm_wait_st() {
    asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
}
// wait for this thread's outstanding TMEM loads; the loaded registers pass through the asm so
// that no use of them is scheduled before the wait
__device__ __forceinline__ void tm_wait_ld(Q4& a) {
    asm volatile("tcgen05.wait::ld.sync.aligned;"
                 : "+f"(a.v[0]), "+f"(a.v[1]), "+f"(a.v[2]), "+f"(a.v[3])::"memory");
}
__device__ __forceinline__ void tm_wait_ld(Q4& a, Q4& b) {
    asm volatile("tcgen05.wait::ld.sync.aligned;"
                 : "+f"(a.v[0]), "+f"(a.v[1]), "+f"(a.v[2]), "+f"(a.v[3]), "+f"(b.v[0]),
                   "+f"(b.v[1]), "+f"(b.v[2]), "+f"(b.v[3])::"memory");
}
__device__ __forceinline__ void tm_wait_ld(Q4& a, Q4& b, Q4& c) {
    asm volatile("tcgen05.wait::ld.sync.aligned;"
                 : "+f"(a.v[0]), "+f"(a.v[1]), "+f"(a.v[2]), "+f"(a.v[3]), "+f"(b.v[0]),
                   "+f"(b.v[1]), "+f"(b.v[2]), "+f"(b.v[3]), "+f"(c.v[0]), "+f"(c.v[1]),
                   "+f"(c.v[2]), "+f"(c.v[3])::"memory");
}
__device__ __forceinline__ void tm_wait_ld(Q4& a, Q4& b, Q4& c, Q4& d) {
    asm volatile("tcgen05.wait::ld.sync.aligned;"
                 : "+f"(a.v[0]), "+f"(a.v[1]), "+f"(a.v[2]), "+f"(a.v[3]), "+f"(b.v[0]),
                   "+f"(b.v[1]), "+f"(b.v[2]), "+f"(b.v[3]), "+f"(c.v[0]), "+f"(c.v[1]),
                   "+f"(c.v[2]), "+f"(c.v[3]), "+f"(d.v[0]), "+f"(d.v[1]), "+f"(d.v[2]),
                   "+f"(d.v[3])::"memory");
}
__device__ __forceinline__ void tm_wait_ld(Q4& a, Q4& b, Q4& c, Q4& d, Q4& e) {
    asm volatile("tcgen05.wait::ld.sync.aligned;"
                 : "+f"(a.v[0]), "+f"(a.v[1]), "+f"(a.v[2]), "+f"(a.v[3]), "+f"(b.v[0]),
                   "+f"(b.v[1]), "+f"(b.v[2]), "+f"(b.v[3]), "+f"(c.v[0]), "+f"(c.v[1]),
                   "+f"(c.v[2]), "+f"(c.v[3]), "+f"(d.v[0]), "+f"(d.v[1]), "+f"(d.v[2]),
                   "+f"(d.v[3]), "+f"(e.v[0]), "+f"(e.v[1]), "+f"(e.v[2]), "+f"(e.v[3])::"memory");
}

}  // namespace seg
}  // namespace fdtd
