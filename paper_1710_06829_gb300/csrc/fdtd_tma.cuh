// TMA descriptors, mbarrier / bulk-tensor PTX helpers and image-writing stores
// shared by the fused step kernels.
#pragma once

#include <cuda.h>

#include "fdtd_internal.cuh"

namespace fdtd {

struct FusedMaps {
    CUtensorMap e[3];   // E boxes of the input set
    CUtensorMap b[3];   // B boxes of the input set
};

struct FusedPlan {
    int dtype;
    FusedMaps maps[2];   // indexed by input set
};

// ---------------------------------------------------------------- PTX helpers

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count)
                 : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)),
                 "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

// bounded wait: at most `tries` polls (each poll may suspend the thread for a short,
// hardware-defined time); false when the phase did not complete
__device__ __forceinline__ bool mbar_wait_n(uint64_t* bar, uint32_t parity, uint32_t tries) {
    for (uint32_t it = 0; it < tries; ++it)
        if (mbar_try_wait(bar, parity)) return true;
    return false;
}

// the kernels' wait: about a second at most
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity) {
    return mbar_wait_n(bar, parity, 1u << 20);
}

__device__ __forceinline__ void tma_load_3d(void* dst, const CUtensorMap* map, int x, int y, int z,
                                            uint64_t* bar) {
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes"
        " [%0], [%1, {%2, %3, %4}], [%5];" ::"r"(smem_u32(dst)),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(z), "r"(smem_u32(bar))
        : "memory");
}

// L2 prefetch of one tensor-map box (no shared memory is written and there is no completion
// to wait for; a box reaching past the array is clipped like a load)
__device__ __forceinline__ void tma_prefetch_3d(const CUtensorMap* map, int x, int y, int z) {
    asm volatile("cp.async.bulk.prefetch.tensor.3d.L2.global.tile [%0, {%1, %2, %3}];" ::"l"(
                     reinterpret_cast<uint64_t>(map)),
                 "r"(x), "r"(y), "r"(z)
                 : "memory");
}

template <typename T>
__device__ __forceinline__ void store_img(const Geom& g, T* F, int i, int j, int k, T v) {
    const long long base = (long long)k * g.nyp;
    F[(base + j + PY) * g.nxp + i + PX] = v;
    const bool xedge = (i < PX) || (i >= g.nx - PX);
    const bool yedge = (j < PY) || (j >= g.ny - PY);
    if (!xedge && !yedge) return;
    for (int my = -2; my <= 2; ++my) {
        const int jj = j + my * g.ny;
        if (jj < -PY || jj >= g.ny + PY) continue;
        for (int mx = -1; mx <= 1; ++mx) {
            const int ii = i + mx * g.nx;
            if (ii < -PX || ii >= g.nx + PX) continue;
            if (mx == 0 && my == 0) continue;
            F[(base + jj + PY) * g.nxp + ii + PX] = v;
        }
    }
}

}  // namespace fdtd
