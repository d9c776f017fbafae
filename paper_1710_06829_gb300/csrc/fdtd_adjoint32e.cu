// FP32 adjoint E update, mu staged by TMA (the second half of a reverse leapfrog step).
//
// After the adjoint B half has written mu = S (lambda_B + dt G^T l_E) into lambda_B, every
// owned cell gets
//   lambda_E <- S lambda_E + dt F^T mu,   F E = -D* x E,
// i.e. per component  E_x: S lE_x + (DT_y mu_z - DT_z mu_y),  E_y: S lE_y + (DT_z mu_x - DT_x mu_z),
// E_z: S lE_z + (DT_x mu_y - DT_y mu_x), where DT_a is the transpose of the extended stencil D*_a
// (Eq. D*): along a it reaches -2 .. +1, transversally +-1 (the mirror image of D*_a).  The
// transposed taps, for a field G on B positions and backward differences d(k) = G[k-a] - G[k]:
//   DT_a G = cA d(0) + cD (G[-2a] - G[+a]) + cBb (d(-b) + d(+b)) + cBc (d(-c) + d(+c)).
//
// A CTA owns a 64 x 8 (x, y) tile and a chunk of tz planes; mu planes arrive by TMA as 72 x 12
// boxes (x0-4 .., y0-2 ..) into a five-slot shared ring (planes q-2 .. q+1 in use, q+2 in
// flight), completion on mbarriers with bounded waits.  A thread owns four consecutive cells
// of one row (a warp two rows, four warps the tile): each stencil row is one 16-byte shared
// load, values beyond the segment come from neighbouring lanes by shuffle (row-end lanes read
// them).  lambda_E of the own cells is read from HBM one plane ahead and written in place
// (each cell is read and written by its owner only; mu is read-only here).
//
// Every mbarrier wait is bounded; on expiry the CTA raises *err, drains its copies in flight
// (bounded) and returns.
#include "fdtd_seg.cuh"

namespace fdtd {
namespace adj32e {

using namespace seg;

constexpr int W = 4, TX = 64, TY = 8, D = 1;
constexpr int NSEG = TX / W;
constexpr int NT = NSEG * TY;                                  // 128 threads, one segment each
constexpr int EW = TX + 8, EH = TY + 4, EPL = EW * EH;         // mu box 72 x 12
constexpr int ESLOT = ((EPL * 4 + 127) / 128) * 128 / 4;
constexpr int NE = D + 4, NS = D + 1;
constexpr size_t OFF_BAR = (size_t)NE * 3 * ESLOT * 4;
constexpr size_t SMEM = OFF_BAR + (size_t)(NS + 1) * 8;
constexpr uint32_t UNIT_BYTES = 3u * EPL * 4;
constexpr uint32_t PRO_BYTES = 9u * EPL * 4;

// DT_z on the four cells at e of a field with plane slots Gmm (q-2), Gm (q-1), G0 (q), Gp (q+1);
// transverse x, then y
__device__ __forceinline__ void dtz(const float* Gmm, const float* Gm, const float* G0,
                                    const float* Gp, int e, bool lb, bool rb, float cA, float cD,
                                    float cBx, float cBy, float out[4]) {
    const Q4 cm = ldq(Gm, e), c0 = ldq(G0, e), cmm = ldq(Gmm, e), cp = ldq(Gp, e);
    const Q4 ym = ldq(Gm, e - EW), y0m = ldq(G0, e - EW), yp = ldq(Gm, e + EW),
             y0p = ldq(G0, e + EW);
    float d[6];   // d[k] = G(q-1) - G(q) at x-1+k
#pragma unroll
    for (int u = 0; u < 4; ++u) d[1 + u] = cm.v[u] - c0.v[u];
    d[0] = from_left(d[4]);
    d[5] = from_right(d[1]);
    if (lb) d[0] = Gm[e - 1] - G0[e - 1];
    if (rb) d[5] = Gm[e + 4] - G0[e + 4];
#pragma unroll
    for (int u = 0; u < 4; ++u)
        out[u] = dstar_diff(d[1 + u], cmm.v[u], cp.v[u], d[u], d[2 + u], ym.v[u] - y0m.v[u],
                            yp.v[u] - y0p.v[u], cA, cD, cBx, cBy);
}

// DT_y: transverse x, then z
__device__ __forceinline__ void dty(const float* Gm, const float* G0, const float* Gp, int e,
                                    bool lb, bool rb, float cA, float cD, float cBx, float cBz,
                                    float out[4]) {
    const Q4 a0 = ldq(G0, e), am = ldq(G0, e - EW), amm = ldq(G0, e - 2 * EW),
             ap = ldq(G0, e + EW);
    const Q4 zm = ldq(Gm, e), zmy = ldq(Gm, e - EW), zp = ldq(Gp, e), zpy = ldq(Gp, e - EW);
    float d[6];   // d[k] = G(y-1) - G(y) at x-1+k, plane q
#pragma unroll
    for (int u = 0; u < 4; ++u) d[1 + u] = am.v[u] - a0.v[u];
    d[0] = from_left(d[4]);
    d[5] = from_right(d[1]);
    if (lb) d[0] = G0[e - EW - 1] - G0[e - 1];
    if (rb) d[5] = G0[e - EW + 4] - G0[e + 4];
#pragma unroll
    for (int u = 0; u < 4; ++u)
        out[u] = dstar_diff(d[1 + u], amm.v[u], ap.v[u], d[u], d[2 + u], zmy.v[u] - zm.v[u],
                            zpy.v[u] - zp.v[u], cA, cD, cBx, cBz);
}

// DT_x: transverse y, then z
__device__ __forceinline__ void dtx(const float* Gm, const float* G0, const float* Gp, int e,
                                    bool lb, bool rb, float cA, float cD, float cBy, float cBz,
                                    float out[4]) {
    const Q4 R = ldq(G0, e), Ym = ldq(G0, e - EW), Yp = ldq(G0, e + EW), Zm = ldq(Gm, e),
             Zp = ldq(Gp, e);
    float r[7];                           // G(q) at x-2 .. x+4
    float ym[5], yp[5], zm[5], zp[5];     // x-1 .. x+3
#pragma unroll
    for (int u = 0; u < 4; ++u) {
        r[2 + u] = R.v[u];
        ym[1 + u] = Ym.v[u];
        yp[1 + u] = Yp.v[u];
        zm[1 + u] = Zm.v[u];
        zp[1 + u] = Zp.v[u];
    }
    r[0] = from_left(R.v[2]);
    r[1] = from_left(R.v[3]);
    r[6] = from_right(R.v[0]);
    ym[0] = from_left(Ym.v[3]);
    yp[0] = from_left(Yp.v[3]);
    zm[0] = from_left(Zm.v[3]);
    zp[0] = from_left(Zp.v[3]);
    if (lb) {
        r[0] = G0[e - 2];
        r[1] = G0[e - 1];
        ym[0] = G0[e - EW - 1];
        yp[0] = G0[e + EW - 1];
        zm[0] = Gm[e - 1];
        zp[0] = Gp[e - 1];
    }
    if (rb) r[6] = G0[e + 4];
#pragma unroll
    for (int u = 0; u < 4; ++u)
        out[u] = dstar_diff(r[u + 1] - r[u + 2], r[u], r[u + 3], ym[u] - ym[u + 1],
                            yp[u] - yp[u + 1], zm[u] - zm[u + 1], zp[u] - zp[u + 1], cA, cD, cBy,
                            cBz);
}

__global__ void __launch_bounds__(NT, 4)
adjE_kernel(const __grid_constant__ FusedMaps maps, Geom g, Mult<float> m, FieldSet<float> lam,
            const float* __restrict__ spy, const float* __restrict__ spz, int tz,
            int* __restrict__ err) {
    extern __shared__ __align__(128) unsigned char smem[];
    float* sG = reinterpret_cast<float*>(smem);
    uint64_t* bar = reinterpret_cast<uint64_t*>(smem + OFF_BAR);

    const int ntx = g.nx / TX, nty = g.ny / TY;
    int w = blockIdx.x;
    const int tx = w % ntx;
    w /= ntx;
    const int ty = w % nty;
    const int zc = w / nty;
    const int x0 = tx * TX, y0 = ty * TY, z0 = zc * tz;
    const int zend = min(z0 + tz, g.nz);
    const int niter = zend - z0;
    const int tid = threadIdx.x;
    const bool edge = (x0 < PX) || (x0 + TX > g.nx - PX) || (y0 < PY) || (y0 + TY > g.ny - PY);

    auto wrapz = [&](int q) {
        int r = q % g.nz;
        return r < 0 ? r + g.nz : r;
    };
    auto gslot = [&](int q) { return (q - (z0 - 2)) % NE; };
    auto Gp_ = [&](int q, int c) { return sG + (gslot(q) * 3 + c) * ESLOT; };
    auto issue_unit = [&](int u) {
        const int qe = z0 + 1 + u;   // leading mu plane of iteration u
        uint64_t* b = &bar[u % NS];
        mbar_expect_tx(b, UNIT_BYTES);
        for (int c = 0; c < 3; ++c) tma_load_3d(Gp_(qe, c), &maps.e[c], x0, y0, wrapz(qe), b);
    };

    const int by = tid / NSEG, bx = W * (tid % NSEG);
    const bool lb = bx == 0, rb = bx == TX - W;
    const int e = (by + 2) * EW + (bx + 4);
    const int j = y0 + by;
    const unsigned plane = (unsigned)g.plane;
    const SegOut dst = seg_out(g, x0 + bx, j, edge);

    if (tid == 0) {
        for (int s = 0; s <= NS; ++s) mbar_init(&bar[s], 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    }
    __syncthreads();
    int issued = 0;
    if (tid == 0 && niter > 0) {
        mbar_expect_tx(&bar[NS], PRO_BYTES);
        for (int q = z0 - 2; q <= z0; ++q)
            for (int c = 0; c < 3; ++c) tma_load_3d(Gp_(q, c), &maps.e[c], x0, y0, wrapz(q), &bar[NS]);
        for (int u = 0; u <= D && u < niter; ++u) {
            issue_unit(u);
            issued = u + 1;
        }
    }

    // lambda_E of the own cells, prefetched one plane ahead (moved at the start of an iteration)
    float lo[3][W], ln[3][W];
    auto load_lam = [&](int qw, float (&to)[3][W]) {
        const unsigned o = (unsigned)qw * plane + dst.ro;
#pragma unroll
        for (int c = 0; c < 3; ++c) unpackv(*reinterpret_cast<const float4*>(lam.c[c] + o), to[c]);
    };
    if (niter > 0) load_lam(wrapz(z0), ln);

    bool failed = false;
    int it = 0;
    {
        bool ok0 = true;
        if (tid == 0 && niter > 0) ok0 = mbar_wait(&bar[NS], 0) && mbar_wait(&bar[0], 0);
        failed = __syncthreads_or(!ok0);
    }
    // qw = q mod nz; s_mm = ring slot of plane q-2 = it mod NE
    int qw = wrapz(z0);
    int s_mm = 0;
    for (; !failed && it < niter;
         ++it, qw = (qw + 1 == g.nz ? 0 : qw + 1), s_mm = (s_mm + 1 == NE ? 0 : s_mm + 1)) {
        const int s_m = s_mm + 1 == NE ? 0 : s_mm + 1;
        const int s_0 = s_m + 1 == NE ? 0 : s_m + 1;
        const int s_p = s_0 + 1 == NE ? 0 : s_0 + 1;
        const float* Qmm = sG + s_mm * 3 * ESLOT;
        const float* Qm = sG + s_m * 3 * ESLOT;
        const float* Q0 = sG + s_0 * 3 * ESLOT;
        const float* Qp = sG + s_p * 3 * ESLOT;
        bool ok = true;
        if (it == 0) ok = mbar_wait(&bar[NS], 0);
        ok = ok && mbar_wait(&bar[it % NS], (uint32_t)((it / NS) & 1));
        ok = __all_sync(FULL, ok);
        if (ok) {
#pragma unroll
            for (int c = 0; c < 3; ++c)
#pragma unroll
                for (int u = 0; u < W; ++u) lo[c][u] = ln[c][u];
            if (it + 1 < niter) load_lam(qw + 1 == g.nz ? 0 : qw + 1, ln);
            float s0 = 1.0f;
            if (spy != nullptr) s0 = spy[j] * spz[qw];
            float t1[W], t2[W], ex[W], ey[W], ez[W];
            // E_x: S lE_x + (DT_y mu_z - DT_z mu_y)
            dty(Qm + 2 * ESLOT, Q0 + 2 * ESLOT, Qp + 2 * ESLOT, e, lb, rb, m.cA[1], m.cD[1],
                m.cB[1][0], m.cB[1][2], t1);
            dtz(Qmm + ESLOT, Qm + ESLOT, Q0 + ESLOT, Qp + ESLOT, e, lb, rb, m.cA[2], m.cD[2],
                m.cB[2][0], m.cB[2][1], t2);
#pragma unroll
            for (int u = 0; u < W; ++u) ex[u] = __fmaf_rn(s0, lo[0][u], __fsub_rn(t1[u], t2[u]));
            // E_y: S lE_y + (DT_z mu_x - DT_x mu_z)
            dtz(Qmm, Qm, Q0, Qp, e, lb, rb, m.cA[2], m.cD[2], m.cB[2][0], m.cB[2][1], t1);
            dtx(Qm + 2 * ESLOT, Q0 + 2 * ESLOT, Qp + 2 * ESLOT, e, lb, rb, m.cA[0], m.cD[0],
                m.cB[0][1], m.cB[0][2], t2);
#pragma unroll
            for (int u = 0; u < W; ++u) ey[u] = __fmaf_rn(s0, lo[1][u], __fsub_rn(t1[u], t2[u]));
            // E_z: S lE_z + (DT_x mu_y - DT_y mu_x)
            dtx(Qm + ESLOT, Q0 + ESLOT, Qp + ESLOT, e, lb, rb, m.cA[0], m.cD[0], m.cB[0][1],
                m.cB[0][2], t1);
            dty(Qm, Q0, Qp, e, lb, rb, m.cA[1], m.cD[1], m.cB[1][0], m.cB[1][2], t2);
#pragma unroll
            for (int u = 0; u < W; ++u) ez[u] = __fmaf_rn(s0, lo[2][u], __fsub_rn(t1[u], t2[u]));
            const unsigned po = (unsigned)qw * plane;
            put_seg(lam.c[0], po, dst, ex);
            put_seg(lam.c[1], po, dst, ey);
            put_seg(lam.c[2], po, dst, ez);
        }
        bool ok_next = true;
        if (tid == 0 && it + 1 < niter)
            ok_next = mbar_wait(&bar[(it + 1) % NS], (uint32_t)(((it + 1) / NS) & 1));
        if (__syncthreads_or(!ok || !ok_next)) {
            failed = true;
            break;
        }
        // the next unit's three copies are issued by lane 0 of warps 1, 2, 3 (one component
        // each; warp 1 also posts the expected bytes), so that no warp carries the whole issue
        // on top of its share of the stencil; thread 0 keeps the waits
        if (it + D + 1 < niter) {
            const int c = tid / 32 - 1;
            if ((tid & 31) == 0 && c >= 0 && c < 3) {
                const int u = it + D + 1, qe = z0 + 1 + u;
                uint64_t* b = &bar[u % NS];
                asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                if (c == 0) mbar_expect_tx(b, UNIT_BYTES);
                tma_load_3d(Gp_(qe, c), &maps.e[c], x0, y0, wrapz(qe), b);
            }
            issued = it + D + 2;
        }
    }
    if (failed) {
        if (tid == 0) {
            atomicOr(err, ERR_WAIT);
            if (it == 0) mbar_wait(&bar[NS], 0);
            for (int u = it; u < issued; ++u) mbar_wait(&bar[u % NS], (uint32_t)((u / NS) & 1));
        }
        __syncthreads();
    }
}

}  // namespace adj32e

bool adjoint32e_supported(const Geom& g) {
    return g.nx % adj32e::TX == 0 && g.ny % adj32e::TY == 0 && g.nx >= adj32e::TX &&
           g.ny >= adj32e::TY && g.total < (1LL << 31);
}

bool adjoint32e_prepare() {
    return cudaFuncSetAttribute(adj32e::adjE_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)adj32e::SMEM) == cudaSuccess;
}

static int adjoint32e_tz(const Geom& g) {
    static int slots = -1;
    if (slots < 0) slots = resident_slots((const void*)adj32e::adjE_kernel, adj32e::NT, adj32e::SMEM);
    return zchunk_len((g.nx / adj32e::TX) * (g.ny / adj32e::TY), g.nz, slots, 16, 64);
}

// maps.e[c]: 72 x 12 boxes of mu_c (= lambda_B component c after the adjoint B half)
void launch_adjoint32_E(const FusedMaps& maps, const Geom& g, const Mult<float>& m,
                        FieldSet<float> lam, const float* spy, const float* spz, int* err,
                        cudaStream_t st) {
    const int tz = adjoint32e_tz(g);
    const int nblk = (g.nx / adj32e::TX) * (g.ny / adj32e::TY) * ((g.nz + tz - 1) / tz);
    adj32e::adjE_kernel<<<nblk, adj32e::NT, adj32e::SMEM, st>>>(maps, g, m, lam, spy, spz, tz, err);
}

}  // namespace fdtd
