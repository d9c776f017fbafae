// Helpers of the FP32 segment kernels (forward step, adjoint E update): a thread owns W = 4
// consecutive cells of one row, read and written as 16-byte vectors; values one cell beyond
// the segment come from the neighbouring lanes by warp shuffle; owned results are stored with
// their periodic images (the ghosts of the padded layout).
#pragma once

#include "fdtd_tma.cuh"

namespace fdtd {
namespace seg {

constexpr unsigned FULL = 0xffffffffu;

struct Q4 {
    float v[4];
};

__device__ __forceinline__ Q4 ldq(const float* s, int idx) {
    const float4 a = *reinterpret_cast<const float4*>(s + idx);
    Q4 q;
    q.v[0] = a.x; q.v[1] = a.y; q.v[2] = a.z; q.v[3] = a.w;
    return q;
}

__device__ __forceinline__ void unpackv(const float4& a, float* o) {
    o[0] = a.x; o[1] = a.y; o[2] = a.z; o[3] = a.w;
}

// value held by lane-1 / lane+1 (the caller overrides it in the lanes at the end of a row)
__device__ __forceinline__ float from_left(float v) { return __shfl_up_sync(FULL, v, 1); }
__device__ __forceinline__ float from_right(float v) { return __shfl_down_sync(FULL, v, 1); }

__device__ __forceinline__ void stv(float* F, unsigned idx, const float* v) {
    *reinterpret_cast<float4*>(F + idx) = make_float4(v[0], v[1], v[2], v[3]);
}

// Destination of one W-cell segment (i0 .. i0+W-1, j) in every plane, fixed for the whole
// launch: the in-plane offset of the owned cells and, for a segment within PX of the x ends or
// PY of the y ends, the offsets of its periodic images (the ghosts of the padded layout).
// All offsets are 32-bit element offsets (the padded array has fewer than 2^31 elements).
struct SegOut {
    unsigned ro;   // in-plane offset of cell i0
    int xi, yi;    // x image offset (+-nx or 0), y image offset (+-ny nxp or 0)
    bool img;
};

__device__ __forceinline__ SegOut seg_out(const Geom& g, int i0, int j, bool edge_tile) {
    SegOut d;
    d.ro = (unsigned)((j + PY) * g.nxp + PX + i0);
    d.xi = 0;
    d.yi = 0;
    if (edge_tile) {
        if (i0 < PX) d.xi = g.nx;
        else if (i0 >= g.nx - PX) d.xi = -g.nx;
        if (j < PY) d.yi = g.ny * g.nxp;
        else if (j >= g.ny - PY) d.yi = -g.ny * g.nxp;
    }
    d.img = (d.xi | d.yi) != 0;
    return d;
}

// store a segment at plane offset `po` (plane index x padded plane size) and its images
__device__ __forceinline__ void put_seg(float* F, unsigned po, const SegOut& d, const float* v) {
    const unsigned o = po + d.ro;
    stv(F, o, v);
    if (d.img) {
        if (d.xi) stv(F, o + d.xi, v);
        if (d.yi) {
            stv(F, o + d.yi, v);
            if (d.xi) stv(F, o + d.yi + d.xi, v);
        }
    }
}

}  // namespace seg
}  // namespace fdtd
