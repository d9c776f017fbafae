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

// Taps of the extended stencil D*_a (Eq. D*) on the four cells at in-plane index e of a field
// whose plane slots are Fm (p-1), F0 (p), F1 (p+1), F2 (p+2), in shared memory with rows of EW
// floats.  For each cell u the consumer receives, in the argument order of dstar_diff,
//   d_a = F[+a] - F[0], F[+2a], F[-a], d_bp, d_bm, d_cp, d_cm   (b, c: the transverse axes)
// with d_bp = F[+a+b] - F[+b] etc., the differences taken as dstar_taps takes them.  Each
// stencil row is one 16-byte load of the lane's own cells; values beyond the segment come from
// lane -1 / lane +1 by shuffle, and lanes with no neighbour lane in their row (lb / rb) read
// them from shared memory.  All 32 lanes of the warp must call together.

// D*_z: transverse x, then y
template <int EW, class Fn>
__device__ __forceinline__ void taps_z(const float* Fm, const float* F0, const float* F1,
                                       const float* F2, int e, bool lb, bool rb, Fn&& fn) {
    const Q4 c1 = ldq(F1, e), c0 = ldq(F0, e), c2 = ldq(F2, e), cm = ldq(Fm, e);
    const Q4 p1 = ldq(F1, e + EW), p0 = ldq(F0, e + EW), m1 = ldq(F1, e - EW),
             m0 = ldq(F0, e - EW);
    float d[6];   // d[k] = F1 - F0 at x-1+k
#pragma unroll
    for (int u = 0; u < 4; ++u) d[1 + u] = c1.v[u] - c0.v[u];
    d[0] = from_left(d[4]);
    d[5] = from_right(d[1]);
    if (lb) d[0] = F1[e - 1] - F0[e - 1];
    if (rb) d[5] = F1[e + 4] - F0[e + 4];
#pragma unroll
    for (int u = 0; u < 4; ++u)
        fn(u, d[1 + u], c2.v[u], cm.v[u], d[2 + u], d[u], p1.v[u] - p0.v[u], m1.v[u] - m0.v[u]);
}

// D*_y: transverse x, then z
template <int EW, class Fn>
__device__ __forceinline__ void taps_y(const float* Fm, const float* F0, const float* F1, int e,
                                       bool lb, bool rb, Fn&& fn) {
    const Q4 a0 = ldq(F0, e), a1 = ldq(F0, e + EW), a2 = ldq(F0, e + 2 * EW),
             am = ldq(F0, e - EW);
    const Q4 b1 = ldq(F1, e), b1p = ldq(F1, e + EW), bm = ldq(Fm, e), bmp = ldq(Fm, e + EW);
    float d[6];   // d[k] = F0(y+1) - F0(y) at x-1+k
#pragma unroll
    for (int u = 0; u < 4; ++u) d[1 + u] = a1.v[u] - a0.v[u];
    d[0] = from_left(d[4]);
    d[5] = from_right(d[1]);
    if (lb) d[0] = F0[e + EW - 1] - F0[e - 1];
    if (rb) d[5] = F0[e + EW + 4] - F0[e + 4];
#pragma unroll
    for (int u = 0; u < 4; ++u)
        fn(u, d[1 + u], a2.v[u], am.v[u], d[2 + u], d[u], b1p.v[u] - b1.v[u], bmp.v[u] - bm.v[u]);
}

// D*_x: transverse y, then z
template <int EW, class Fn>
__device__ __forceinline__ void taps_x(const float* Fm, const float* F0, const float* F1, int e,
                                       bool lb, bool rb, Fn&& fn) {
    const Q4 R = ldq(F0, e), Yp = ldq(F0, e + EW), Ym = ldq(F0, e - EW), Z1 = ldq(F1, e),
             Zm = ldq(Fm, e);
    float r[7];                           // F0 at x-1 .. x+5
    float yp[5], ym[5], z1[5], zm[5];     // x .. x+4
#pragma unroll
    for (int u = 0; u < 4; ++u) {
        r[1 + u] = R.v[u];
        yp[u] = Yp.v[u];
        ym[u] = Ym.v[u];
        z1[u] = Z1.v[u];
        zm[u] = Zm.v[u];
    }
    r[0] = from_left(R.v[3]);
    r[5] = from_right(R.v[0]);
    r[6] = from_right(R.v[1]);
    yp[4] = from_right(Yp.v[0]);
    ym[4] = from_right(Ym.v[0]);
    z1[4] = from_right(Z1.v[0]);
    zm[4] = from_right(Zm.v[0]);
    if (lb) r[0] = F0[e - 1];
    if (rb) {
        r[5] = F0[e + 4];
        r[6] = F0[e + 5];
        yp[4] = F0[e + EW + 4];
        ym[4] = F0[e - EW + 4];
        z1[4] = F1[e + 4];
        zm[4] = Fm[e + 4];
    }
#pragma unroll
    for (int u = 0; u < 4; ++u)
        fn(u, r[u + 2] - r[u + 1], r[u + 3], r[u], yp[u + 1] - yp[u], ym[u + 1] - ym[u],
           z1[u + 1] - z1[u], zm[u + 1] - zm[u]);
}

}  // namespace seg
}  // namespace fdtd

namespace fdtd {
namespace seg {

// ---- paired FP32 arithmetic (f32x2: two lanes of data per instruction, IEEE round to nearest,
// so every result equals the scalar operation's).  A pair holds two neighbouring cells.
using u64 = unsigned long long;

__device__ __forceinline__ u64 pk(float a, float b) {
    u64 r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(a), "f"(b));
    return r;
}
__device__ __forceinline__ void upk(u64 r, float& a, float& b) {
    asm("mov.b64 {%0, %1}, %2;" : "=f"(a), "=f"(b) : "l"(r));
}
__device__ __forceinline__ u64 add2(u64 a, u64 b) {
    u64 r;
    asm("add.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
    return r;
}
__device__ __forceinline__ u64 sub2(u64 a, u64 b) {
    u64 r;
    asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
    return r;
}
__device__ __forceinline__ u64 mul2(u64 a, u64 b) {
    u64 r;
    asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
    return r;
}
__device__ __forceinline__ u64 fma2(u64 a, u64 b, u64 c) {
    u64 r;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(r) : "l"(a), "l"(b), "l"(c));
    return r;
}
__device__ __forceinline__ u64 lo2(const Q4& q) { return pk(q.v[0], q.v[1]); }
__device__ __forceinline__ u64 hi2(const Q4& q) { return pk(q.v[2], q.v[3]); }

// dstar_diff on a pair of cells, with the transverse sums already formed:
//   cA d_a + cD (f_a2 - f_am1) + cBb sb + cBc sc, in the order of dstar_diff
__device__ __forceinline__ u64 dstar_pair(u64 da, u64 a2, u64 am1, u64 sb, u64 sc, u64 cA, u64 cD,
                                          u64 cBb, u64 cBc) {
    u64 v = mul2(cA, da);
    v = fma2(cD, sub2(a2, am1), v);
    v = fma2(cBb, sb, v);
    v = fma2(cBc, sc, v);
    return v;
}

// The D* operators (times dt) on the four cells at in-plane index e, with the thread's own row
// of each plane passed in (the kernel keeps those in tensor memory) and the other rows and the
// row-end scalars read from the shared-memory planes Fm (p-1), F0 (p), F1 (p+1):
//   dstar_z2: D*_z (transverse x, then y) on two cell pairs; c0, c1, c2, cm = own rows of
//             planes p, p+1, p+2, p-1;
//   dstar_y2: D*_y (transverse x, then z) on two cell pairs; a0, b1, bm = own rows of p, p+1, p-1;
//   dstar_x4: D*_x (transverse y, then z) per cell;  R, Z1, Zm = own rows of p, p+1, p-1.
// The differences and their rounding order are those of taps_z / taps_y / taps_x followed by
// dstar_diff (dstar_pair on cell pairs), so every kernel's B is bitwise the same.
template <int EW>
__device__ __forceinline__ void dstar_z2(const float* F0, const float* F1, const Q4& c0,
                                         const Q4& c1, const Q4& c2, const Q4& cm, int e, bool lb,
                                         bool rb, u64 cA, u64 cD, u64 cBx, u64 cBy, u64 out[2]) {
    const Q4 p1 = ldq(F1, e + EW), p0 = ldq(F0, e + EW), m1 = ldq(F1, e - EW),
             m0 = ldq(F0, e - EW);
    const u64 dlo = sub2(lo2(c1), lo2(c0)), dhi = sub2(hi2(c1), hi2(c0));
    float d[6];
    upk(dlo, d[1], d[2]);
    upk(dhi, d[3], d[4]);
    d[0] = from_left(d[4]);
    d[5] = from_right(d[1]);
    if (lb) d[0] = F1[e - 1] - F0[e - 1];
    if (rb) d[5] = F1[e + 4] - F0[e + 4];
    const u64 sylo = add2(sub2(lo2(p1), lo2(p0)), sub2(lo2(m1), lo2(m0)));
    const u64 syhi = add2(sub2(hi2(p1), hi2(p0)), sub2(hi2(m1), hi2(m0)));
    out[0] = dstar_pair(dlo, lo2(c2), lo2(cm), pk(d[2] + d[0], d[3] + d[1]), sylo, cA, cD, cBx, cBy);
    out[1] = dstar_pair(dhi, hi2(c2), hi2(cm), pk(d[4] + d[2], d[5] + d[3]), syhi, cA, cD, cBx, cBy);
}

template <int EW>
__device__ __forceinline__ void dstar_y2(const float* Fm, const float* F0, const float* F1,
                                         const Q4& a0, const Q4& b1, const Q4& bm, int e, bool lb,
                                         bool rb, u64 cA, u64 cD, u64 cBx, u64 cBz, u64 out[2]) {
    const Q4 a1 = ldq(F0, e + EW), a2 = ldq(F0, e + 2 * EW), am = ldq(F0, e - EW);
    const Q4 b1p = ldq(F1, e + EW), bmp = ldq(Fm, e + EW);
    const u64 dlo = sub2(lo2(a1), lo2(a0)), dhi = sub2(hi2(a1), hi2(a0));
    float d[6];
    upk(dlo, d[1], d[2]);
    upk(dhi, d[3], d[4]);
    d[0] = from_left(d[4]);
    d[5] = from_right(d[1]);
    if (lb) d[0] = F0[e + EW - 1] - F0[e - 1];
    if (rb) d[5] = F0[e + EW + 4] - F0[e + 4];
    const u64 szlo = add2(sub2(lo2(b1p), lo2(b1)), sub2(lo2(bmp), lo2(bm)));
    const u64 szhi = add2(sub2(hi2(b1p), hi2(b1)), sub2(hi2(bmp), hi2(bm)));
    out[0] = dstar_pair(dlo, lo2(a2), lo2(am), pk(d[2] + d[0], d[3] + d[1]), szlo, cA, cD, cBx, cBz);
    out[1] = dstar_pair(dhi, hi2(a2), hi2(am), pk(d[4] + d[2], d[5] + d[3]), szhi, cA, cD, cBx, cBz);
}

template <int EW>
__device__ __forceinline__ void dstar_x4(const float* Fm, const float* F0, const float* F1,
                                         const Q4& R, const Q4& Z1, const Q4& Zm, int e, bool lb,
                                         bool rb, float cA, float cD, float cBy, float cBz,
                                         float out[4]) {
    const Q4 Yp = ldq(F0, e + EW), Ym = ldq(F0, e - EW);
    float r[7];
    float yp[5], ym[5], z1[5], zm[5];
#pragma unroll
    for (int u = 0; u < 4; ++u) {
        r[1 + u] = R.v[u];
        yp[u] = Yp.v[u];
        ym[u] = Ym.v[u];
        z1[u] = Z1.v[u];
        zm[u] = Zm.v[u];
    }
    r[0] = from_left(R.v[3]);
    r[5] = from_right(R.v[0]);
    r[6] = from_right(R.v[1]);
    yp[4] = from_right(Yp.v[0]);
    ym[4] = from_right(Ym.v[0]);
    z1[4] = from_right(Z1.v[0]);
    zm[4] = from_right(Zm.v[0]);
    if (lb) r[0] = F0[e - 1];
    if (rb) {
        r[5] = F0[e + 4];
        r[6] = F0[e + 5];
        yp[4] = F0[e + EW + 4];
        ym[4] = F0[e - EW + 4];
        z1[4] = F1[e + 4];
        zm[4] = Fm[e + 4];
    }
#pragma unroll
    for (int u = 0; u < 4; ++u)
        out[u] = dstar_diff(r[u + 2] - r[u + 1], r[u + 3], r[u], yp[u + 1] - yp[u],
                            ym[u + 1] - ym[u], z1[u + 1] - z1[u], zm[u + 1] - zm[u], cA, cD, cBy,
                            cBz);
}

}  // namespace seg
}  // namespace fdtd
