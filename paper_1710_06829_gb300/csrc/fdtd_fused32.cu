// FP32 fused leapfrog step (one launch per leapfrog step).
//
// A CTA owns a 64 x 8 (x, y) tile and a chunk of 32 planes and marches through it.  E^n planes
// arrive by TMA (cp.async.bulk.tensor.3d) as 72 x 12 boxes (x0-4 .., y0-2 ..) into a ring of five
// shared-memory slots, one plane ahead of use, completion signalled on mbarriers.  Iteration `it`
// forms B^{n+1/2} on plane p = z0-1+it (tile, halo row y0-1, halo column x0-1) and E^{n+1} on
// plane p-1, so one block barrier per plane suffices; B^{n+1/2} lives in a small shared ring
// (B_x, B_y: 3 planes, B_z: 2 planes).  B^{n-1/2} is not staged: each thread prefetches its
// own segment of the next plane from HBM into registers while the current plane is computed.
//
// Work per thread: W consecutive cells of one row.  Every stencil row a thread needs is read as
// W-wide shared-memory vectors (a window of 3W values covers the x reach -1 .. W+1), so one
// load serves several taps; a warp covers whole rows, so a vector load of a warp never
// conflicts.  Owned results leave as W-wide stores; a segment at the edge of the domain also
// writes its periodic images (the ghosts of the padded layout).  Plane bookkeeping uses
// counters (no integer division in the loop).
//
// Per-cell arithmetic is dstar_taps / ampere_comp with the same operands in the same order as
// the reference-form kernels: the fields are bitwise equal.  Every mbarrier wait is bounded
// (fdtd_tma.cuh); on expiry the CTA raises *err, drains its copies in flight (bounded) and
// returns.
#include "fdtd_tma.cuh"

namespace fdtd {
namespace f32seg {

constexpr int W = 4;                                            // cells per thread (along x)
constexpr int TX = 64, TY = 8, D = 1;   // z-chunk length: launch parameter (zchunk_len)
constexpr int NSEG = TX / W;                                    // segments per row
constexpr int NT = ((NSEG * (TY + 1) + TY + 1 + 31) / 32) * 32;  // B tasks + halo column
constexpr int EW = TX + 8, EH = TY + 4, EPL = EW * EH;        // E box 72 x 12 (x0-4.., y0-2..)
constexpr int ESLOT = ((EPL * 4 + 127) / 128) * 128 / 4;        // floats per E slot
constexpr int BW = TX + 4, BH = TY + 1, BPL = BW * BH;         // B^{n+1/2} plane: x0-4.., y0-1..
constexpr int BSLOT = ((BPL * 4 + 127) / 128) * 128 / 4;
constexpr int NE = D + 4, NS = D + 1;
constexpr size_t OFF_E = 0;
constexpr size_t OFF_BN = OFF_E + (size_t)NE * 3 * ESLOT * 4;   // Bx[3], By[3], Bz[2]
constexpr size_t OFF_BAR = OFF_BN + (size_t)8 * BSLOT * 4;
constexpr size_t SMEM = OFF_BAR + (size_t)(NS + 1) * 8;
constexpr uint32_t UNIT_BYTES = 3u * EPL * 4;
constexpr uint32_t PRO_BYTES = 9u * EPL * 4;

// W-wide vector of floats (8 bytes for W = 2, 16 bytes for W = 4)
template <int N>
struct VecT;
template <>
struct VecT<2> {
    using type = float2;
};
template <>
struct VecT<4> {
    using type = float4;
};
using Vec = typename VecT<W>::type;

__device__ __forceinline__ void unpackv(const float2& a, float* o) { o[0] = a.x; o[1] = a.y; }
__device__ __forceinline__ void unpackv(const float4& a, float* o) {
    o[0] = a.x; o[1] = a.y; o[2] = a.z; o[3] = a.w;
}
__device__ __forceinline__ void packv(const float* o, float2& a) { a.x = o[0]; a.y = o[1]; }
__device__ __forceinline__ void packv(const float* o, float4& a) {
    a.x = o[0]; a.y = o[1]; a.z = o[2]; a.w = o[3];
}

__device__ __forceinline__ void ldv(const float* s, int idx, float* o) {
    unpackv(*reinterpret_cast<const Vec*>(s + idx), o);
}

struct Win {
    float v[3 * W];   // v[k] = F[idx - W + k]
};

__device__ __forceinline__ Win win(const float* s, int idx) {
    Win w;
    ldv(s, idx - W, w.v);
    ldv(s, idx, w.v + W);
    ldv(s, idx + W, w.v + 2 * W);
    return w;
}

// D*_a (times dt) on the W cells starting at in-plane index e, for the field whose
// plane slots are Fm (p-1), F0 (p), F1 (p+1), F2 (p+2).  Tap order as dstar_taps expects.
template <int A>
__device__ __forceinline__ void dstarw(const float* Fm, const float* F0, const float* F1,
                                       const float* F2, int e, float cA, float cD, float cBb,
                                       float cBc, float out[W]) {
    if constexpr (A == 0) {   // axis x; transverse y, then z
        const Win w0 = win(F0, e), wyp = win(F0, e + EW), wym = win(F0, e - EW);
        const Win w1 = win(F1, e), wm = win(Fm, e);
#pragma unroll
        for (int u = 0; u < W; ++u)
            out[u] = dstar_taps(w0.v[W + 1 + u], w0.v[W + u], w0.v[W + 2 + u], w0.v[W - 1 + u],
                                wyp.v[W + 1 + u], wyp.v[W + u], wym.v[W + 1 + u], wym.v[W + u],
                                w1.v[W + 1 + u], w1.v[W + u], wm.v[W + 1 + u], wm.v[W + u], cA, cD,
                                cBb, cBc);
    } else if constexpr (A == 1) {   // axis y; transverse x, then z
        const Win w0 = win(F0, e), wyp = win(F0, e + EW);
        float a2[W], am[W], c1[W], c1p[W], cm[W], cmp[W];
        ldv(F0, e + 2 * EW, a2);
        ldv(F0, e - EW, am);
        ldv(F1, e, c1);
        ldv(F1, e + EW, c1p);
        ldv(Fm, e, cm);
        ldv(Fm, e + EW, cmp);
#pragma unroll
        for (int u = 0; u < W; ++u)
            out[u] = dstar_taps(wyp.v[W + u], w0.v[W + u], a2[u], am[u], wyp.v[W + 1 + u],
                                w0.v[W + 1 + u], wyp.v[W - 1 + u], w0.v[W - 1 + u], c1p[u], c1[u],
                                cmp[u], cm[u], cA, cD, cBb, cBc);
    } else {   // axis z; transverse x, then y
        const Win w1 = win(F1, e), w0 = win(F0, e);
        float a2[W], am[W], p1[W], p0[W], m1[W], m0[W];
        ldv(F2, e, a2);
        ldv(Fm, e, am);
        ldv(F1, e + EW, p1);
        ldv(F0, e + EW, p0);
        ldv(F1, e - EW, m1);
        ldv(F0, e - EW, m0);
#pragma unroll
        for (int u = 0; u < W; ++u)
            out[u] = dstar_taps(w1.v[W + u], w0.v[W + u], a2[u], am[u], w1.v[W + 1 + u],
                                w0.v[W + 1 + u], w1.v[W - 1 + u], w0.v[W - 1 + u], p1[u], p0[u],
                                m1[u], m0[u], cA, cD, cBb, cBc);
    }
}

__device__ __forceinline__ void stv(float* F, unsigned idx, const float* v) {
    Vec a;
    packv(v, a);
    *reinterpret_cast<Vec*>(F + idx) = a;
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

__global__ void __launch_bounds__(NT, 3)
step_kernel(const __grid_constant__ FusedMaps maps, Geom g, Mult<float> m, FieldSet<float> in,
            FieldSet<float> out, const float* __restrict__ spy, const float* __restrict__ spz,
            const float* __restrict__ jyz, const float* __restrict__ jx_row,
            float* __restrict__ h0, float* __restrict__ h1, float* __restrict__ h2, int tz,
            int* __restrict__ err) {
    extern __shared__ __align__(128) unsigned char smem[];
    float* sE = reinterpret_cast<float*>(smem + OFF_E);
    float* sB = reinterpret_cast<float*>(smem + OFF_BN);
    uint64_t* bar = reinterpret_cast<uint64_t*>(smem + OFF_BAR);

    const int ntx = g.nx / TX, nty = g.ny / TY;
    int w = blockIdx.x;
    const int tx = w % ntx;
    w /= ntx;
    const int ty = w % nty;
    const int zc = w / nty;
    const int x0 = tx * TX, y0 = ty * TY, z0 = zc * tz;
    const int zend = min(z0 + tz, g.nz);
    const int niter = zend - z0 + 1;   // B planes z0-1 .. zend-1
    const int tid = threadIdx.x;
    // tiles that own cells with periodic images (the ghosts of the padded layout)
    const bool edge = (x0 < PX) || (x0 + TX > g.nx - PX) || (y0 < PY) || (y0 + TY > g.ny - PY);

    auto wrapz = [&](int q) {
        int r = q % g.nz;
        return r < 0 ? r + g.nz : r;
    };
    auto eslot = [&](int q) { return (q - (z0 - 2)) % NE; };
    auto Ep = [&](int q, int c) { return sE + (eslot(q) * 3 + c) * ESLOT; };
    auto issue_unit = [&](int u) {
        const int qe = z0 + 1 + u;   // leading E plane of iteration u
        uint64_t* b = &bar[u % NS];
        mbar_expect_tx(b, UNIT_BYTES);
        for (int c = 0; c < 3; ++c) tma_load_3d(Ep(qe, c), &maps.e[c], x0, y0, wrapz(qe), b);
    };

    // ---- task of this thread in the B phase
    //   tid <  144: segment (bx = 4 (tid % 16), by = tid / 16 - 1), by in [-1, TY)
    //   tid in [144, 153): halo column cell (bx = -1, by = tid - 145)
    const bool bseg = tid < NSEG * (TY + 1);
    const bool bcol = !bseg && tid < NSEG * (TY + 1) + TY + 1;
    const int b_bx = bseg ? W * (tid % NSEG) : -1;
    const int b_by = bseg ? tid / NSEG - 1 : tid - NSEG * (TY + 1) - 1;
    const unsigned b_off = (unsigned)((y0 + b_by + PY) * g.nxp + (x0 + b_bx + PX));
    const unsigned plane = (unsigned)g.plane;
    int b_y = y0 + b_by;
    if (b_y < 0) b_y += g.ny;
    // owned-cell destinations of this thread's B segment and E segment
    const SegOut b_dst = seg_out(g, x0 + b_bx, y0 + (b_by < 0 ? 0 : b_by), edge);
    const int e_by = tid / NSEG, e_bx = W * (tid % NSEG);
    const SegOut e_dst = seg_out(g, x0 + e_bx, y0 + (e_by < TY ? e_by : 0), edge);

    if (tid == 0) {
        for (int s = 0; s <= NS; ++s) mbar_init(&bar[s], 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    }
    __syncthreads();
    int issued = 0;
    if (tid == 0) {
        mbar_expect_tx(&bar[NS], PRO_BYTES);
        for (int q = z0 - 2; q <= z0; ++q)
            for (int c = 0; c < 3; ++c) tma_load_3d(Ep(q, c), &maps.e[c], x0, y0, wrapz(q), &bar[NS]);
        for (int u = 0; u <= D && u < niter; ++u) {
            issue_unit(u);
            issued = u + 1;
        }
    }

    // B^{n-1/2} of this thread's task, prefetched one plane ahead
    float bo[3][W];
#pragma unroll
    for (int c = 0; c < 3; ++c)
#pragma unroll
        for (int u = 0; u < W; ++u) bo[c][u] = 0.0f;
    float bn[3][W];   // next plane's B^{n-1/2}, loaded at the start of the current B phase
    auto load_bold = [&](int qw, float (&dst)[3][W]) {   // qw: wrapped plane index
        const unsigned o = (unsigned)qw * plane + b_off;
        if (bseg) {
#pragma unroll
            for (int c = 0; c < 3; ++c) unpackv(__ldg(reinterpret_cast<const Vec*>(in.c[3 + c] + o)), dst[c]);
        } else if (bcol) {
#pragma unroll
            for (int c = 0; c < 3; ++c) dst[c][0] = __ldg(in.c[3 + c] + o);
        }
    };
    load_bold(wrapz(z0 - 1), bo);

    const float mdt = -m.dt;
    // B^{n+1/2} ring: B_x, B_y keep planes p, p-1, p-2 (slot (p+6) mod 3); B_z keeps p, p-1.
    // Iteration it forms B^{n+1/2} on plane p = z0 - 1 + it (it < niter) and E^{n+1} on
    // plane p - 1 (when z0 <= p - 1 < zend).  One block barrier per iteration.
    // Thread 0 waits for each plane's copies before the block barrier that precedes the
    // plane's iteration; the other threads' own waits then return at once (no spinning).
    bool failed = false;
    int it = 0;
    {
        bool ok0 = true;
        if (tid == 0) ok0 = mbar_wait(&bar[NS], 0) && mbar_wait(&bar[0], 0);
        failed = __syncthreads_or(!ok0);
    }
    // plane bookkeeping by counters (no integer division in the loop):
    //   pw = p mod nz, qw = (p-1) mod nz, s_m = ring slot of plane p-1 = it mod NE,
    //   r3 = (p+6) mod 3 (B_x / B_y ring), r2 = (p+6) mod 2 (B_z ring)
    int pw = wrapz(z0 - 1), qw = wrapz(z0 - 2);
    int s_m = 0;
    int r3 = (z0 + 5) % 3, r2 = (z0 + 5) % 2;
    for (; !failed && it <= niter; ++it, qw = pw, pw = (pw + 1 == g.nz ? 0 : pw + 1),
                                   s_m = (s_m + 1 == NE ? 0 : s_m + 1), r3 = (r3 == 2 ? 0 : r3 + 1),
                                   r2 ^= 1) {
        const int p = z0 - 1 + it;
        // E^n ring slots of planes p-1 .. p+2
        const int s_0 = s_m + 1 == NE ? 0 : s_m + 1;
        const int s_1 = s_0 + 1 == NE ? 0 : s_0 + 1;
        const int s_2 = s_1 + 1 == NE ? 0 : s_1 + 1;
        const float* Pm = sE + s_m * 3 * ESLOT;
        const float* P0 = sE + s_0 * 3 * ESLOT;
        const float* P1 = sE + s_1 * 3 * ESLOT;
        const float* P2 = sE + s_2 * 3 * ESLOT;
        bool ok = true;
        if (it < niter) {
            if (it == 0) ok = mbar_wait(&bar[NS], 0);
            ok = ok && mbar_wait(&bar[it % NS], (uint32_t)((it / NS) & 1));
        }
        // ---- B^{n+1/2}(p)
        // B^{n+1/2} ring slots: plane p (current), p-1, p-2
        const int r3m = r3 == 0 ? 2 : r3 - 1, r3mm = r3m == 0 ? 2 : r3m - 1;
        if (ok && it < niter) {
            // issue the next plane's B^{n-1/2} loads first: they complete during this plane's work
            if (it + 1 < niter) load_bold(pw + 1 == g.nz ? 0 : pw + 1, bn);
            float* Bxc = sB + r3 * BSLOT;
            float* Byc = sB + (3 + r3) * BSLOT;
            float* Bzc = sB + (6 + r2) * BSLOT;
            if (bseg) {
                const int e = (b_by + 2) * EW + (b_bx + 4);
                float dz[W], dy[W], bxv[W], byv[W], bzv[W];
                // B_x = B_x + (D*_z E_y - D*_y E_z)
                dstarw<2>((Pm + 1 * ESLOT), (P0 + 1 * ESLOT), (P1 + 1 * ESLOT), (P2 + 1 * ESLOT), e,
                          m.cA[2], m.cD[2], m.cB[2][0], m.cB[2][1], dz);
                dstarw<1>((Pm + 2 * ESLOT), (P0 + 2 * ESLOT), (P1 + 2 * ESLOT), nullptr, e, m.cA[1],
                          m.cD[1], m.cB[1][0], m.cB[1][2], dy);
#pragma unroll
                for (int u = 0; u < W; ++u) bxv[u] = bo[0][u] + (dz[u] - dy[u]);
                // B_y = B_y + (D*_x E_z - D*_z E_x)
                dstarw<0>((Pm + 2 * ESLOT), (P0 + 2 * ESLOT), (P1 + 2 * ESLOT), nullptr, e, m.cA[0],
                          m.cD[0], m.cB[0][1], m.cB[0][2], dy);
                dstarw<2>((Pm + 0 * ESLOT), (P0 + 0 * ESLOT), (P1 + 0 * ESLOT), (P2 + 0 * ESLOT), e,
                          m.cA[2], m.cD[2], m.cB[2][0], m.cB[2][1], dz);
#pragma unroll
                for (int u = 0; u < W; ++u) byv[u] = bo[1][u] + (dy[u] - dz[u]);
                // B_z = B_z + (D*_y E_x - D*_x E_y)
                dstarw<1>((Pm + 0 * ESLOT), (P0 + 0 * ESLOT), (P1 + 0 * ESLOT), nullptr, e, m.cA[1],
                          m.cD[1], m.cB[1][0], m.cB[1][2], dy);
                dstarw<0>((Pm + 1 * ESLOT), (P0 + 1 * ESLOT), (P1 + 1 * ESLOT), nullptr, e, m.cA[0],
                          m.cD[0], m.cB[0][1], m.cB[0][2], dz);
#pragma unroll
                for (int u = 0; u < W; ++u) bzv[u] = bo[2][u] + (dy[u] - dz[u]);
                if (spy != nullptr) {
                    const float f = spy[b_y] * spz[pw];
#pragma unroll
                    for (int u = 0; u < W; ++u) { bxv[u] *= f; byv[u] *= f; bzv[u] *= f; }
                }
                const int bi = (b_by + 1) * BW + (b_bx + 4);
                stv(Bxc, bi, bxv);
                stv(Byc, bi, byv);
                stv(Bzc, bi, bzv);
                if (p >= z0 && b_by >= 0) {
                    const unsigned po = (unsigned)pw * plane;
                    put_seg(out.c[3], po, b_dst, bxv);
                    put_seg(out.c[4], po, b_dst, byv);
                    put_seg(out.c[5], po, b_dst, bzv);
                }
            } else if (bcol) {
                // halo column x0-1: one cell, scalar taps (not stored to HBM)
                const int e = (b_by + 2) * EW + 3;
                const float* Em[3] = {(Pm + 0 * ESLOT), (Pm + 1 * ESLOT), (Pm + 2 * ESLOT)};
                const float* E0[3] = {(P0 + 0 * ESLOT), (P0 + 1 * ESLOT), (P0 + 2 * ESLOT)};
                const float* E1[3] = {(P1 + 0 * ESLOT), (P1 + 1 * ESLOT), (P1 + 2 * ESLOT)};
                const float* E2[3] = {(P2 + 0 * ESLOT), (P2 + 1 * ESLOT), (P2 + 2 * ESLOT)};
#define DX(c)                                                                                   \
    dstar_taps(E0[c][e + 1], E0[c][e], E0[c][e + 2], E0[c][e - 1], E0[c][e + 1 + EW],          \
               E0[c][e + EW], E0[c][e + 1 - EW], E0[c][e - EW], E1[c][e + 1], E1[c][e],         \
               Em[c][e + 1], Em[c][e], m.cA[0], m.cD[0], m.cB[0][1], m.cB[0][2])
#define DY(c)                                                                                   \
    dstar_taps(E0[c][e + EW], E0[c][e], E0[c][e + 2 * EW], E0[c][e - EW], E0[c][e + EW + 1],   \
               E0[c][e + 1], E0[c][e + EW - 1], E0[c][e - 1], E1[c][e + EW], E1[c][e],         \
               Em[c][e + EW], Em[c][e], m.cA[1], m.cD[1], m.cB[1][0], m.cB[1][2])
#define DZ(c)                                                                                   \
    dstar_taps(E1[c][e], E0[c][e], E2[c][e], Em[c][e], E1[c][e + 1], E0[c][e + 1],             \
               E1[c][e - 1], E0[c][e - 1], E1[c][e + EW], E0[c][e + EW], E1[c][e - EW],        \
               E0[c][e - EW], m.cA[2], m.cD[2], m.cB[2][0], m.cB[2][1])
                float bxs = bo[0][0] + (DZ(1) - DY(2));
                float bys = bo[1][0] + (DX(2) - DZ(0));
                float bzs = bo[2][0] + (DY(0) - DX(1));
#undef DX
#undef DY
#undef DZ
                if (spy != nullptr) {
                    const float f = spy[b_y] * spz[pw];
                    bxs *= f;
                    bys *= f;
                    bzs *= f;
                }
                const int bi = (b_by + 1) * BW + 3;
                Bxc[bi] = bxs;
                Byc[bi] = bys;
                Bzc[bi] = bzs;
            }
            // prefetch next plane's B^{n-1/2} while E is formed
#pragma unroll
            for (int c = 0; c < 3; ++c)
#pragma unroll
                for (int u = 0; u < W; ++u) bo[c][u] = bn[c][u];
        }
        // ---- E^{n+1}(p - 1)
        const int q = p - 1;
        if (ok && q >= z0 && q < zend && tid < NSEG * TY) {
            const int by = e_by, bx = e_bx;
            const int e = (by + 2) * EW + (bx + 4);
            const int bi = (by + 1) * BW + (bx + 4);
            const float* Bxc = sB + r3m * BSLOT;
            const float* Byc = sB + (3 + r3m) * BSLOT;
            const float* Bzc = sB + (6 + (r2 ^ 1)) * BSLOT;
            const float* Bxp = sB + r3mm * BSLOT;
            const float* Byp = sB + (3 + r3mm) * BSLOT;
            float E0x[W], E0y[W], E0z[W];
            ldv(Pm + 0 * ESLOT, e, E0x);
            ldv(Pm + 1 * ESLOT, e, E0y);
            ldv(Pm + 2 * ESLOT, e, E0z);
            float Bz[W + 1], By[W + 1], tmp[W];   // [0] = value at x-1, [1 + u] = cell u
            float Bzy[W], Byz[W], Bx[W], Bxz[W], Bxy[W];
            ldv(Bzc, bi, Bz + 1);
            ldv(Bzc, bi - W, tmp);
            Bz[0] = tmp[W - 1];
            ldv(Bzc, bi - BW, Bzy);
            ldv(Byc, bi, By + 1);
            ldv(Byc, bi - W, tmp);
            By[0] = tmp[W - 1];
            ldv(Byp, bi, Byz);
            ldv(Bxc, bi, Bx);
            ldv(Bxp, bi, Bxz);
            ldv(Bxc, bi - BW, Bxy);
            float ex[W], ey[W], ez[W];
#pragma unroll
            for (int u = 0; u < W; ++u) {
                ex[u] = ampere_comp(E0x[u], Bz[1 + u], Bzy[u], By[1 + u], Byz[u], m.cE[1], m.cE[2]);
                ey[u] = ampere_comp(E0y[u], Bx[u], Bxz[u], Bz[1 + u], Bz[u], m.cE[2], m.cE[0]);
                ez[u] = ampere_comp(E0z[u], By[1 + u], By[u], Bx[u], Bxy[u], m.cE[0], m.cE[1]);
            }
            const int i0 = x0 + bx, j = y0 + by;
            if (jx_row != nullptr) {
                float jv[W];
                unpackv(__ldg(reinterpret_cast<const Vec*>(jx_row + i0)), jv);
                const float sy = jyz[j], sz = jyz[g.ny + qw];
#pragma unroll
                for (int u = 0; u < W; ++u) ex[u] = fma(mdt, (jv[u] * sy) * sz, ex[u]);
            }
            if (spy != nullptr) {
                const float f = spy[j] * spz[qw];
#pragma unroll
                for (int u = 0; u < W; ++u) { ex[u] *= f; ey[u] *= f; ez[u] *= f; }
            }
            const unsigned po = (unsigned)qw * plane;
            put_seg(out.c[0], po, e_dst, ex);
            put_seg(out.c[1], po, e_dst, ey);
            put_seg(out.c[2], po, e_dst, ez);
            if (h0 != nullptr) {
                put_seg(h0, po, e_dst, ex);
                put_seg(h1, po, e_dst, ey);
                put_seg(h2, po, e_dst, ez);
            }
        }
        bool ok_next = true;
        if (tid == 0 && it + 1 < niter)
            ok_next = mbar_wait(&bar[(it + 1) % NS], (uint32_t)(((it + 1) / NS) & 1));
        if (__syncthreads_or(!ok || !ok_next)) {
            failed = true;
            break;
        }
        if (tid == 0 && it + D + 1 < niter) {
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            issue_unit(it + D + 1);
            issued = it + D + 2;
        }
    }
    if (failed) {
        // the state written by this launch is not valid; drain this CTA's copies in flight
        if (tid == 0) {
            atomicExch(err, 1);
            if (it == 0) mbar_wait(&bar[NS], 0);
            for (int u = it; u < issued; ++u) mbar_wait(&bar[u % NS], (uint32_t)((u / NS) & 1));
        }
        __syncthreads();
    }
}

}  // namespace f32seg

bool fused32_supported(const Geom& g) {
    // 32-bit element offsets inside the kernel
    return g.nx % f32seg::TX == 0 && g.ny % f32seg::TY == 0 && g.nx >= f32seg::TX &&
           g.ny >= f32seg::TY && g.total < (1LL << 31);
}

bool fused32_prepare() {
    return cudaFuncSetAttribute(f32seg::step_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)f32seg::SMEM) == cudaSuccess;
}

int resident_slots(const void* kernel, int threads, size_t smem) {
    int dev = 0, sms = 0, per_sm = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, threads, smem) != cudaSuccess ||
        sms <= 0 || per_sm <= 0)
        return 0;
    return sms * per_sm;
}

int zchunk_len(int tiles_xy, int nz, int slots, int tz_min, int tz_max) {
    // A CTA marches tz planes plus about two planes of fixed cost (the z-halo B plane and the
    // prologue copies); CTAs run in waves of `slots`.  Minimise waves x (tz + 2) over chunk
    // lengths tz_min..tz_max; ties go to the longer chunk.
    const int hi = nz < tz_max ? nz : tz_max;
    if (slots <= 0) return hi;
    int best = hi;
    long long best_cost = -1;
    for (int tz = hi; tz >= tz_min || tz == nz; --tz) {
        const long long ctas = (long long)tiles_xy * ((nz + tz - 1) / tz);
        const long long waves = (ctas + slots - 1) / slots;
        const long long cost = waves * (tz + 2);
        if (best_cost < 0 || cost < best_cost) {
            best_cost = cost;
            best = tz;
        }
        if (tz <= 1) break;
    }
    return best;
}

static int fused32_tz(const Geom& g) {
    using namespace f32seg;
    static int slots = -1;
    if (slots < 0) slots = resident_slots((const void*)step_kernel, NT, SMEM);
    // measured at 256^3 (456 resident CTAs): 37-plane chunks (2 full waves) 0.218 ms per step,
    // 32-plane chunks (2.25 waves) 0.269 ms
    return zchunk_len((g.nx / TX) * (g.ny / TY), g.nz, slots, 16, 64);
}

void launch_fused32(const FusedMaps& maps, FieldSet<float> in, const Geom& g, const Mult<float>& m,
                    FieldSet<float> out, const float* spy, const float* spz, const float* jyz,
                    const float* jx_row, float* hist_E[3], int* err, cudaStream_t st) {
    using namespace f32seg;
    const int tz = fused32_tz(g);
    const int nblk = (g.nx / TX) * (g.ny / TY) * ((g.nz + tz - 1) / tz);
    step_kernel<<<nblk, NT, SMEM, st>>>(maps, g, m, in, out, spy, spz, jyz, jx_row, hist_E[0],
                                        hist_E[1], hist_E[2], tz, err);
}

}  // namespace fdtd
