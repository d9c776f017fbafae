// FP32 fused leapfrog step with 4-cell x-segments per thread.
//
// Same schedule as the generic fused kernel (fdtd_fused.cu): a CTA owns a
// 64 x 8 (x, y) tile and marches a chunk of 32 planes; E^n planes arrive by TMA
// as 72 x 12 boxes into a ring of shared-memory slots (one plane ahead of use,
// mbarrier completion); for each plane p the CTA forms B^{n+1/2}(p) on the
// tile plus the halo row y0-1 and halo column x0-1, then E^{n+1}(p).
//
// What differs is the work per thread.  Each thread owns four consecutive
// cells in x and reads every stencil row it needs as 16-byte shared-memory
// vectors (a row window of 12 values covers the x reach -1 .. +5 of four
// cells), so one load serves up to four taps.  B^{n-1/2} is not staged: each
// thread prefetches its own 16-byte segment of the next plane from HBM into
// registers while the current plane is computed.  Owned results leave as
// 16-byte stores; a segment at the edge of the domain also writes its periodic
// images (the padded layout's ghosts).
//
// The per-cell arithmetic is dstar_taps / ampere_comp with the same operands in
// the same order as the reference-form kernels: the fields are bitwise equal.
// Every mbarrier wait is bounded (see fdtd_tma.cuh); on expiry the CTA raises
// *err, drains its copies in flight (bounded) and returns.
#include "fdtd_tma.cuh"

namespace fdtd {
namespace f32seg {

constexpr int TX = 64, TY = 8, TZ = 32, D = 1, NT = 160;
constexpr int EW = TX + 8, EH = TY + 4, EPL = EW * EH;       // E box 72 x 12 (x0-4.., y0-2..)
constexpr int ESLOT = ((EPL * 4 + 127) / 128) * 128 / 4;       // floats per E slot
constexpr int BW = TX + 4, BH = TY + 1, BPL = BW * BH;        // B^{n+1/2} plane: x0-4.., y0-1..
constexpr int BSLOT = ((BPL * 4 + 127) / 128) * 128 / 4;
constexpr int NE = D + 4, NS = D + 1;
constexpr int NSEG = TX / 4;                                   // segments per row (16)
constexpr size_t OFF_E = 0;
constexpr size_t OFF_BN = OFF_E + (size_t)NE * 3 * ESLOT * 4;  // Bx[3], By[3], Bz[2]
constexpr size_t OFF_BAR = OFF_BN + (size_t)8 * BSLOT * 4;
constexpr size_t SMEM = OFF_BAR + (size_t)(NS + 1) * 8;
constexpr uint32_t UNIT_BYTES = 3u * EPL * 4;
constexpr uint32_t PRO_BYTES = 9u * EPL * 4;

struct Win {
    float v[12];   // v[k] = F[idx - 4 + k]
};

__device__ __forceinline__ float4 ld4(const float* s, int idx) {
    return *reinterpret_cast<const float4*>(s + idx);
}

__device__ __forceinline__ Win win(const float* s, int idx) {
    Win w;
    const float4 a = ld4(s, idx - 4), b = ld4(s, idx), c = ld4(s, idx + 4);
    w.v[0] = a.x; w.v[1] = a.y; w.v[2] = a.z; w.v[3] = a.w;
    w.v[4] = b.x; w.v[5] = b.y; w.v[6] = b.z; w.v[7] = b.w;
    w.v[8] = c.x; w.v[9] = c.y; w.v[10] = c.z; w.v[11] = c.w;
    return w;
}

// D*_a (times dt) on the four cells starting at in-plane index e, for the field whose
// plane slots are Fm (p-1), F0 (p), F1 (p+1), F2 (p+2).  Tap order as dstar_taps expects.
template <int A>
__device__ __forceinline__ void dstar4(const float* Fm, const float* F0, const float* F1,
                                       const float* F2, int e, float cA, float cD, float cBb,
                                       float cBc, float out[4]) {
    if constexpr (A == 0) {   // axis x; transverse y, then z
        const Win w0 = win(F0, e), wyp = win(F0, e + EW), wym = win(F0, e - EW);
        const Win w1 = win(F1, e), wm = win(Fm, e);
#pragma unroll
        for (int u = 0; u < 4; ++u)
            out[u] = dstar_taps(w0.v[5 + u], w0.v[4 + u], w0.v[6 + u], w0.v[3 + u], wyp.v[5 + u],
                                wyp.v[4 + u], wym.v[5 + u], wym.v[4 + u], w1.v[5 + u], w1.v[4 + u],
                                wm.v[5 + u], wm.v[4 + u], cA, cD, cBb, cBc);
    } else if constexpr (A == 1) {   // axis y; transverse x, then z
        const Win w0 = win(F0, e), wyp = win(F0, e + EW);
        const float4 yp2 = ld4(F0, e + 2 * EW), ym = ld4(F0, e - EW);
        const float4 z1 = ld4(F1, e), z1p = ld4(F1, e + EW), zm = ld4(Fm, e), zmp = ld4(Fm, e + EW);
        const float a2[4] = {yp2.x, yp2.y, yp2.z, yp2.w};
        const float am[4] = {ym.x, ym.y, ym.z, ym.w};
        const float c1[4] = {z1.x, z1.y, z1.z, z1.w};
        const float c1p[4] = {z1p.x, z1p.y, z1p.z, z1p.w};
        const float cm[4] = {zm.x, zm.y, zm.z, zm.w};
        const float cmp[4] = {zmp.x, zmp.y, zmp.z, zmp.w};
#pragma unroll
        for (int u = 0; u < 4; ++u)
            out[u] = dstar_taps(wyp.v[4 + u], w0.v[4 + u], a2[u], am[u], wyp.v[5 + u], w0.v[5 + u],
                                wyp.v[3 + u], w0.v[3 + u], c1p[u], c1[u], cmp[u], cm[u], cA, cD,
                                cBb, cBc);
    } else {   // axis z; transverse x, then y
        const Win w1 = win(F1, e), w0 = win(F0, e);
        const float4 z2 = ld4(F2, e), zm = ld4(Fm, e);
        const float4 w1p = ld4(F1, e + EW), w0p = ld4(F0, e + EW);
        const float4 w1m = ld4(F1, e - EW), w0m = ld4(F0, e - EW);
        const float a2[4] = {z2.x, z2.y, z2.z, z2.w};
        const float am[4] = {zm.x, zm.y, zm.z, zm.w};
        const float p1[4] = {w1p.x, w1p.y, w1p.z, w1p.w};
        const float p0[4] = {w0p.x, w0p.y, w0p.z, w0p.w};
        const float m1[4] = {w1m.x, w1m.y, w1m.z, w1m.w};
        const float m0[4] = {w0m.x, w0m.y, w0m.z, w0m.w};
#pragma unroll
        for (int u = 0; u < 4; ++u)
            out[u] = dstar_taps(w1.v[4 + u], w0.v[4 + u], a2[u], am[u], w1.v[5 + u], w0.v[5 + u],
                                w1.v[3 + u], w0.v[3 + u], p1[u], p0[u], m1[u], m0[u], cA, cD, cBb,
                                cBc);
    }
}

__device__ __forceinline__ void st4(float* F, long long idx, float4 v) {
    *reinterpret_cast<float4*>(F + idx) = v;
}

// Destination of one 4-cell segment (i0 .. i0+3, j, k) and of its periodic images
// (the images exist only for segments at the domain edge; needs nx >= 8, ny >= 4).
struct SegDst {
    long long o1, o2;   // owned row offset; image row offset (valid if yimg)
    bool xl, xr, yimg;
};

__device__ __forceinline__ SegDst seg_dst(const Geom& g, int i0, int j, int k, bool edge_tile) {
    SegDst d;
    const long long rowk = (long long)k * g.nyp;
    d.o1 = (rowk + j + PY) * g.nxp + PX + i0;
    d.xl = edge_tile && i0 == 0;
    d.xr = edge_tile && i0 == g.nx - 4;
    d.yimg = false;
    d.o2 = 0;
    if (edge_tile) {
        int jj = 0;
        if (j < PY) { jj = j + g.ny; d.yimg = true; }
        else if (j >= g.ny - PY) { jj = j - g.ny; d.yimg = true; }
        d.o2 = (rowk + jj + PY) * g.nxp + PX + i0;
    }
    return d;
}

__device__ __forceinline__ void put_seg(float* F, const SegDst& d, int nx, bool edge_tile,
                                        float4 v) {
    st4(F, d.o1, v);
    if (edge_tile) {
        if (d.xl) st4(F, d.o1 + nx, v);
        if (d.xr) st4(F, d.o1 - nx, v);
        if (d.yimg) {
            st4(F, d.o2, v);
            if (d.xl) st4(F, d.o2 + nx, v);
            if (d.xr) st4(F, d.o2 - nx, v);
        }
    }
}

__global__ void __launch_bounds__(NT, 3)
step_kernel(const __grid_constant__ FusedMaps maps, Geom g, Mult<float> m, FieldSet<float> in,
            FieldSet<float> out, const float* __restrict__ spy, const float* __restrict__ spz,
            const float* __restrict__ jyz, const float* __restrict__ jx_row,
            float* __restrict__ h0, float* __restrict__ h1, float* __restrict__ h2,
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
    const int x0 = tx * TX, y0 = ty * TY, z0 = zc * TZ;
    const int zend = min(z0 + TZ, g.nz);
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
    const int b_bx = bseg ? 4 * (tid % NSEG) : -1;
    const int b_by = bseg ? tid / NSEG - 1 : tid - NSEG * (TY + 1) - 1;
    const long long b_off = (long long)(y0 + b_by + PY) * g.nxp + (x0 + b_bx + PX);
    int b_y = y0 + b_by;
    if (b_y < 0) b_y += g.ny;

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
    float4 bo[3] = {make_float4(0, 0, 0, 0), make_float4(0, 0, 0, 0), make_float4(0, 0, 0, 0)};
    auto load_bold = [&](int q) {
        const long long o = (long long)wrapz(q) * g.plane + b_off;
        if (bseg) {
#pragma unroll
            for (int c = 0; c < 3; ++c) bo[c] = __ldg(reinterpret_cast<const float4*>(in.c[3 + c] + o));
        } else if (bcol) {
#pragma unroll
            for (int c = 0; c < 3; ++c) bo[c].x = __ldg(in.c[3 + c] + o);
        }
    };
    load_bold(z0 - 1);

    const float mdt = -m.dt;
    // B^{n+1/2} ring: B_x, B_y keep planes p, p-1, p-2; B_z keeps p, p-1.
    auto sBx = [&](int q) { return sB + ((q + 6) % 3) * BSLOT; };
    auto sBy = [&](int q) { return sB + (3 + (q + 6) % 3) * BSLOT; };
    auto sBz = [&](int q) { return sB + (6 + (q + 6) % 2) * BSLOT; };
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
    for (; !failed && it <= niter; ++it) {
        const int p = z0 - 1 + it;
        // E^n ring slots of planes p-1 .. p+2
        const int s_m = eslot(p - 1);
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
        if (ok && it < niter) {
            const int pw = wrapz(p);
            float* Bxc = sBx(p);
            float* Byc = sBy(p);
            float* Bzc = sBz(p);
            if (bseg) {
                const int e = (b_by + 2) * EW + (b_bx + 4);
                float dz[4], dy[4], bxv[4], byv[4], bzv[4];
                // B_x = B_x + (D*_z E_y - D*_y E_z)
                dstar4<2>((Pm + 1 * ESLOT), (P0 + 1 * ESLOT), (P1 + 1 * ESLOT), (P2 + 1 * ESLOT), e, m.cA[2], m.cD[2],
                          m.cB[2][0], m.cB[2][1], dz);
                dstar4<1>((Pm + 2 * ESLOT), (P0 + 2 * ESLOT), (P1 + 2 * ESLOT), nullptr, e, m.cA[1], m.cD[1],
                          m.cB[1][0], m.cB[1][2], dy);
                bxv[0] = bo[0].x + (dz[0] - dy[0]);
                bxv[1] = bo[0].y + (dz[1] - dy[1]);
                bxv[2] = bo[0].z + (dz[2] - dy[2]);
                bxv[3] = bo[0].w + (dz[3] - dy[3]);
                // B_y = B_y + (D*_x E_z - D*_z E_x)
                dstar4<0>((Pm + 2 * ESLOT), (P0 + 2 * ESLOT), (P1 + 2 * ESLOT), nullptr, e, m.cA[0], m.cD[0],
                          m.cB[0][1], m.cB[0][2], dy);
                dstar4<2>((Pm + 0 * ESLOT), (P0 + 0 * ESLOT), (P1 + 0 * ESLOT), (P2 + 0 * ESLOT), e, m.cA[2], m.cD[2],
                          m.cB[2][0], m.cB[2][1], dz);
                byv[0] = bo[1].x + (dy[0] - dz[0]);
                byv[1] = bo[1].y + (dy[1] - dz[1]);
                byv[2] = bo[1].z + (dy[2] - dz[2]);
                byv[3] = bo[1].w + (dy[3] - dz[3]);
                // B_z = B_z + (D*_y E_x - D*_x E_y)
                dstar4<1>((Pm + 0 * ESLOT), (P0 + 0 * ESLOT), (P1 + 0 * ESLOT), nullptr, e, m.cA[1], m.cD[1],
                          m.cB[1][0], m.cB[1][2], dy);
                dstar4<0>((Pm + 1 * ESLOT), (P0 + 1 * ESLOT), (P1 + 1 * ESLOT), nullptr, e, m.cA[0], m.cD[0],
                          m.cB[0][1], m.cB[0][2], dz);
                bzv[0] = bo[2].x + (dy[0] - dz[0]);
                bzv[1] = bo[2].y + (dy[1] - dz[1]);
                bzv[2] = bo[2].z + (dy[2] - dz[2]);
                bzv[3] = bo[2].w + (dy[3] - dz[3]);
                if (spy != nullptr) {
                    const float f = spy[b_y] * spz[pw];
#pragma unroll
                    for (int u = 0; u < 4; ++u) { bxv[u] *= f; byv[u] *= f; bzv[u] *= f; }
                }
                const int bi = (b_by + 1) * BW + (b_bx + 4);
                const float4 vx = make_float4(bxv[0], bxv[1], bxv[2], bxv[3]);
                const float4 vy = make_float4(byv[0], byv[1], byv[2], byv[3]);
                const float4 vz = make_float4(bzv[0], bzv[1], bzv[2], bzv[3]);
                *reinterpret_cast<float4*>(Bxc + bi) = vx;
                *reinterpret_cast<float4*>(Byc + bi) = vy;
                *reinterpret_cast<float4*>(Bzc + bi) = vz;
                if (p >= z0 && b_by >= 0) {
                    const SegDst d = seg_dst(g, x0 + b_bx, y0 + b_by, pw, edge);
                    put_seg(out.c[3], d, g.nx, edge, vx);
                    put_seg(out.c[4], d, g.nx, edge, vy);
                    put_seg(out.c[5], d, g.nx, edge, vz);
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
                float bxs = bo[0].x + (DZ(1) - DY(2));
                float bys = bo[1].x + (DX(2) - DZ(0));
                float bzs = bo[2].x + (DY(0) - DX(1));
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
            if (it + 1 < niter) load_bold(p + 1);
        }
        // ---- E^{n+1}(p - 1)
        const int q = p - 1;
        if (ok && q >= z0 && q < zend && tid < NSEG * TY) {
            const int qw = wrapz(q);
            const int by = tid / NSEG, bx = 4 * (tid % NSEG);
            const int e = (by + 2) * EW + (bx + 4);
            const int bi = (by + 1) * BW + (bx + 4);
            const float* Bxc = sBx(q);
            const float* Byc = sBy(q);
            const float* Bzc = sBz(q);
            const float* Bxp = sBx(q - 1);
            const float* Byp = sBy(q - 1);
            const float4 ex4 = ld4((Pm + 0 * ESLOT), e), ey4 = ld4((Pm + 1 * ESLOT), e), ez4 = ld4((Pm + 2 * ESLOT), e);
            const float4 bz0 = ld4(Bzc, bi), bzym = ld4(Bzc, bi - BW), bzxm = ld4(Bzc, bi - 4);
            const float4 by0 = ld4(Byc, bi), byzm = ld4(Byp, bi), byxm = ld4(Byc, bi - 4);
            const float4 bx0 = ld4(Bxc, bi), bxzm = ld4(Bxp, bi), bxym = ld4(Bxc, bi - BW);
            const float E0x[4] = {ex4.x, ex4.y, ex4.z, ex4.w};
            const float E0y[4] = {ey4.x, ey4.y, ey4.z, ey4.w};
            const float E0z[4] = {ez4.x, ez4.y, ez4.z, ez4.w};
            const float Bz[5] = {bzxm.w, bz0.x, bz0.y, bz0.z, bz0.w};   // Bz[1 + u + dx]
            const float Bzy[4] = {bzym.x, bzym.y, bzym.z, bzym.w};
            const float By[5] = {byxm.w, by0.x, by0.y, by0.z, by0.w};
            const float Byz[4] = {byzm.x, byzm.y, byzm.z, byzm.w};
            const float Bx[4] = {bx0.x, bx0.y, bx0.z, bx0.w};
            const float Bxz[4] = {bxzm.x, bxzm.y, bxzm.z, bxzm.w};
            const float Bxy[4] = {bxym.x, bxym.y, bxym.z, bxym.w};
            float ex[4], ey[4], ez[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                ex[u] = ampere_comp(E0x[u], Bz[1 + u], Bzy[u], By[1 + u], Byz[u], m.cE[1], m.cE[2]);
                ey[u] = ampere_comp(E0y[u], Bx[u], Bxz[u], Bz[1 + u], Bz[u], m.cE[2], m.cE[0]);
                ez[u] = ampere_comp(E0z[u], By[1 + u], By[u], Bx[u], Bxy[u], m.cE[0], m.cE[1]);
            }
            const int i0 = x0 + bx, j = y0 + by;
            if (jx_row != nullptr) {
                const float4 j4 = __ldg(reinterpret_cast<const float4*>(jx_row + i0));
                const float jv[4] = {j4.x, j4.y, j4.z, j4.w};
                const float sy = jyz[j], sz = jyz[g.ny + qw];
#pragma unroll
                for (int u = 0; u < 4; ++u) ex[u] = fma(mdt, (jv[u] * sy) * sz, ex[u]);
            }
            if (spy != nullptr) {
                const float f = spy[j] * spz[qw];
#pragma unroll
                for (int u = 0; u < 4; ++u) { ex[u] *= f; ey[u] *= f; ez[u] *= f; }
            }
            const float4 vx = make_float4(ex[0], ex[1], ex[2], ex[3]);
            const float4 vy = make_float4(ey[0], ey[1], ey[2], ey[3]);
            const float4 vz = make_float4(ez[0], ez[1], ez[2], ez[3]);
            const SegDst d = seg_dst(g, i0, j, qw, edge);
            put_seg(out.c[0], d, g.nx, edge, vx);
            put_seg(out.c[1], d, g.nx, edge, vy);
            put_seg(out.c[2], d, g.nx, edge, vz);
            if (h0 != nullptr) {
                put_seg(h0, d, g.nx, edge, vx);
                put_seg(h1, d, g.nx, edge, vy);
                put_seg(h2, d, g.nx, edge, vz);
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
    return g.nx % f32seg::TX == 0 && g.ny % f32seg::TY == 0 && g.nx >= f32seg::TX &&
           g.ny >= f32seg::TY;
}

bool fused32_prepare() {
    return cudaFuncSetAttribute(f32seg::step_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)f32seg::SMEM) == cudaSuccess;
}

void launch_fused32(const FusedMaps& maps, FieldSet<float> in, const Geom& g, const Mult<float>& m,
                    FieldSet<float> out, const float* spy, const float* spz, const float* jyz,
                    const float* jx_row, float* hist_E[3], int* err, cudaStream_t st) {
    using namespace f32seg;
    const int nblk = (g.nx / TX) * (g.ny / TY) * ((g.nz + TZ - 1) / TZ);
    step_kernel<<<nblk, NT, SMEM, st>>>(maps, g, m, in, out, spy, spz, jyz, jx_row, hist_E[0],
                                        hist_E[1], hist_E[2], err);
}

}  // namespace fdtd
