// FP32 adjoint B half-step with the fused coefficient gradient, E^n staged by TMA.
//
// Computes, for every owned cell (see fdtd_adjoint.cu for the derivation),
//   mu = S (lambda_B + dt G^T (S lambda_E))            -> written to lambda_B (in place)
//   g_theta += mu . (dF/dtheta) E^n                     -> FP32 per thread, FP64 per block
// where (dF/dtheta) E^n are the derivative brackets of the extended stencil (Eq. D* with alpha
// eliminated by Eq. alpha).  The brackets need E^n at x-1..x+2, y-1..y+2, z-1..z+2 around the
// cell: E^n planes arrive by TMA as 72 x 12 boxes into a five-slot shared ring (same schedule
// as the fused forward step), and each thread evaluates the brackets of four consecutive
// cells from one 16-byte shared-memory vector per stencil row, the values beyond its segment
// coming from neighbouring lanes by shuffle (seg::taps_*).  lambda_E (own cell and its +x, +y, +z
// neighbours) and lambda_B (own cell) are read from HBM directly; only mu is written.
//
// Every mbarrier wait is bounded; on expiry the CTA raises *err, drains its copies in flight
// (bounded) and returns.
#include "fdtd_seg.cuh"

namespace fdtd {
namespace adj32 {

using namespace seg;

constexpr int TX = 64, TY = 8, D = 1, NT = 128;   // z-chunk length: launch parameter
constexpr int EW = TX + 8, EH = TY + 4, EPL = EW * EH;
constexpr int ESLOT = ((EPL * 4 + 127) / 128) * 128 / 4;
constexpr int NE = D + 4, NS = D + 1;
constexpr size_t OFF_BAR = (size_t)NE * 3 * ESLOT * 4;
constexpr size_t SMEM = OFF_BAR + (size_t)(NS + 1) * 8;
constexpr uint32_t UNIT_BYTES = 3u * EPL * 4;
constexpr uint32_t PRO_BYTES = 9u * EPL * 4;

__device__ __forceinline__ void unpack(float4 a, float o[4]) {
    o[0] = a.x; o[1] = a.y; o[2] = a.z; o[3] = a.w;
}

// Gradient brackets (Sec. 2 with alpha eliminated by Eq. alpha; without 1/dx_a) of D*_a at a
// cell, from the taps of seg::taps_* (d_a = F[+a] - F[0], ...):
//   d/d delta_a: (F[+2a] - F[-a]) - 3 d_a,   d/d beta_ab: (d_bp + d_bm) - 2 d_a,   likewise c.
// acc[0..2] += w * (delta, beta_ab, beta_ac brackets)
template <int EW>
struct Brackets {
    float* acc;
    const float* w;
    __device__ __forceinline__ void operator()(int u, float da, float a2, float am1, float bp,
                                               float bm, float cp, float cm) const {
        acc[0] = fmaf(w[u], (a2 - am1) - 3.0f * da, acc[0]);
        acc[1] = fmaf(w[u], (bp + bm) - 2.0f * da, acc[1]);
        acc[2] = fmaf(w[u], (cp + cm) - 2.0f * da, acc[2]);
    }
};


__global__ void __launch_bounds__(NT, 3)
adjB_kernel(const __grid_constant__ FusedMaps maps, Geom g, Mult<float> m, FieldSet<float> lam,
            const float* __restrict__ spy, const float* __restrict__ spz,
            double* __restrict__ partials, int tz, int* __restrict__ err) {
    extern __shared__ __align__(128) unsigned char smem[];
    float* sE = reinterpret_cast<float*>(smem);
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
    auto eslot = [&](int q) { return (q - (z0 - 1)) % NE; };
    auto Ep = [&](int q, int c) { return sE + (eslot(q) * 3 + c) * ESLOT; };
    auto issue_unit = [&](int u) {
        const int qe = z0 + 2 + u;   // leading E^n plane of iteration u
        uint64_t* b = &bar[u % NS];
        mbar_expect_tx(b, UNIT_BYTES);
        for (int c = 0; c < 3; ++c) tma_load_3d(Ep(qe, c), &maps.e[c], x0, y0, wrapz(qe), b);
    };

    const int by = tid / 16, bx = 4 * (tid % 16);
    const int i0 = x0 + bx, j = y0 + by;
    const int e = (by + 2) * EW + (bx + 4);
    const bool lb = bx == 0, rb = bx == TX - 4;   // row-end lanes (no shuffle neighbour)
    const unsigned plane = (unsigned)g.plane;
    const SegOut dst = seg_out(g, i0, j, edge);

    if (tid == 0) {
        for (int s = 0; s <= NS; ++s) mbar_init(&bar[s], 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    }
    __syncthreads();
    int issued = 0;
    if (tid == 0) {
        mbar_expect_tx(&bar[NS], PRO_BYTES);
        for (int q = z0 - 1; q <= z0 + 1; ++q)
            for (int c = 0; c < 3; ++c) tma_load_3d(Ep(q, c), &maps.e[c], x0, y0, wrapz(q), &bar[NS]);
        for (int u = 0; u <= D && u < niter; ++u) {
            issue_unit(u);
            issued = u + 1;
        }
    }

    float racc[9];
    double acc[9];
#pragma unroll
    for (int q = 0; q < 9; ++q) {
        racc[q] = 0.0f;
        acc[q] = 0.0;
    }
    const float* lEx = lam.c[0];
    const float* lEy = lam.c[1];
    const float* lEz = lam.c[2];
    const int Y = g.nxp;
    // lambda of this thread's cells (own, +x, +y, +z; lambda_B own), prefetched one plane ahead
    struct Lam {
        float ex[5], ey[5], ez[5], exy[4], ezy[4], exz[4], eyz[4], bx[4], by[4], bz[4];
    } L;
    auto load_lam = [&](int q) {
        const int qw = wrapz(q);
        const unsigned c = (unsigned)qw * plane + dst.ro;
        const int zp = (wrapz(q + 1) - qw) * (int)plane;
        unpack(__ldg(reinterpret_cast<const float4*>(lEx + c)), L.ex);
        unpack(__ldg(reinterpret_cast<const float4*>(lEy + c)), L.ey);
        unpack(__ldg(reinterpret_cast<const float4*>(lEz + c)), L.ez);
        L.ey[4] = __ldg(lEy + c + 4);
        L.ez[4] = __ldg(lEz + c + 4);
        unpack(__ldg(reinterpret_cast<const float4*>(lEx + c + Y)), L.exy);
        unpack(__ldg(reinterpret_cast<const float4*>(lEz + c + Y)), L.ezy);
        unpack(__ldg(reinterpret_cast<const float4*>(lEx + c + zp)), L.exz);
        unpack(__ldg(reinterpret_cast<const float4*>(lEy + c + zp)), L.eyz);
        unpack(*reinterpret_cast<const float4*>(lam.c[3] + c), L.bx);
        unpack(*reinterpret_cast<const float4*>(lam.c[4] + c), L.by);
        unpack(*reinterpret_cast<const float4*>(lam.c[5] + c), L.bz);
    };
    if (niter > 0) load_lam(z0);
    bool failed = false;
    int it = 0;
    // counters: pw = p mod nz, s_m = ring slot of plane p-1 = it mod NE
    int pw = wrapz(z0), s_m = 0;
    for (; it < niter; ++it, pw = (pw + 1 == g.nz ? 0 : pw + 1), s_m = (s_m + 1 == NE ? 0 : s_m + 1)) {
        const int p = z0 + it;
        const int s_0 = s_m + 1 == NE ? 0 : s_m + 1;
        const int s_1 = s_0 + 1 == NE ? 0 : s_0 + 1;
        const int s_2 = s_1 + 1 == NE ? 0 : s_1 + 1;
        bool ok = true;
        if (it == 0) ok = mbar_wait(&bar[NS], 0);
        ok = ok && mbar_wait(&bar[it % NS], (uint32_t)((it / NS) & 1));
        ok = __all_sync(FULL, ok);   // keeps the shuffles below warp-uniform
        if (ok) {
            // l_E = S lambda_E at the cells and their +x, +y, +z neighbours
            float s0 = 1.0f, syp = 1.0f, szp = 1.0f;
            if (spy != nullptr) {
                const int jp = j + 1 < g.ny ? j + 1 : 0;
                s0 = spy[j] * spz[pw];
                syp = spy[jp] * spz[pw];
                szp = spy[j] * spz[pw + 1 == g.nz ? 0 : pw + 1];
            }
            float mux[4], muy[4], muz[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                // a fixed rounding order (intrinsics are never contracted), the one the
                // one-kernel reverse step uses on cell pairs
                const float ex0 = __fmul_rn(s0, L.ex[u]), ey0 = __fmul_rn(s0, L.ey[u]),
                            ez0 = __fmul_rn(s0, L.ez[u]);
                const float gx = __fmaf_rn(m.cE[2], __fmaf_rn(-szp, L.eyz[u], ey0),
                                           __fmul_rn(-m.cE[1], __fmaf_rn(-syp, L.ezy[u], ez0)));
                const float gy = __fmaf_rn(m.cE[0], __fmaf_rn(-s0, L.ez[u + 1], ez0),
                                           __fmul_rn(-m.cE[2], __fmaf_rn(-szp, L.exz[u], ex0)));
                const float gz = __fmaf_rn(m.cE[1], __fmaf_rn(-syp, L.exy[u], ex0),
                                           __fmul_rn(-m.cE[0], __fmaf_rn(-s0, L.ey[u + 1], ey0)));
                mux[u] = __fmul_rn(s0, __fadd_rn(L.bx[u], gx));
                muy[u] = __fmul_rn(s0, __fadd_rn(L.by[u], gy));
                muz[u] = __fmul_rn(s0, __fadd_rn(L.bz[u], gz));
            }
            if (it + 1 < niter) load_lam(p + 1);
            // gradient brackets from the E^n ring (planes p-1 .. p+2 in slots s_m .. s_2)
            const float* Pm = sE + s_m * 3 * ESLOT;
            const float* P0 = sE + s_0 * 3 * ESLOT;
            const float* P1 = sE + s_1 * 3 * ESLOT;
            const float* P2 = sE + s_2 * 3 * ESLOT;
            float nmux[4], nmuy[4], nmuz[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                nmux[u] = -mux[u];
                nmuy[u] = -muy[u];
                nmuz[u] = -muz[u];
            }
            // B_y gets D*_x E_z, B_z gets -D*_x E_y  (x brackets: racc 0..2)
            taps_x<EW>(Pm + 2 * ESLOT, P0 + 2 * ESLOT, P1 + 2 * ESLOT, e, lb, rb, Brackets<EW>{racc + 0, muy});
            taps_x<EW>(Pm + ESLOT, P0 + ESLOT, P1 + ESLOT, e, lb, rb, Brackets<EW>{racc + 0, nmuz});
            // B_z gets D*_y E_x, B_x gets -D*_y E_z  (y brackets: racc 3..5)
            taps_y<EW>(Pm, P0, P1, e, lb, rb, Brackets<EW>{racc + 3, muz});
            taps_y<EW>(Pm + 2 * ESLOT, P0 + 2 * ESLOT, P1 + 2 * ESLOT, e, lb, rb, Brackets<EW>{racc + 3, nmux});
            // B_x gets D*_z E_y, B_y gets -D*_z E_x  (z brackets: racc 6..8)
            taps_z<EW>(Pm + ESLOT, P0 + ESLOT, P1 + ESLOT, P2 + ESLOT, e, lb, rb, Brackets<EW>{racc + 6, mux});
            taps_z<EW>(Pm, P0, P1, P2, e, lb, rb, Brackets<EW>{racc + 6, nmuy});
#pragma unroll
            for (int q = 0; q < 9; ++q) {   // one FP64 add per 4 cells and coefficient
                acc[q] += (double)racc[q];
                racc[q] = 0.0f;
            }
            // mu -> lambda_B (own cells and, at the domain edge, their images)
            const unsigned po = (unsigned)pw * plane;
            put_seg(lam.c[3], po, dst, mux);
            put_seg(lam.c[4], po, dst, muy);
            put_seg(lam.c[5], po, dst, muz);
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
                const int u = it + D + 1, qe = z0 + 2 + u;
                uint64_t* b = &bar[u % NS];
                asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                if (c == 0) mbar_expect_tx(b, UNIT_BYTES);
                tma_load_3d(Ep(qe, c), &maps.e[c], x0, y0, wrapz(qe), b);
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
        return;
    }
    // block reduction of the FP64 accumulators
    __shared__ double red[NT / 32][9];
    const int wp = tid >> 5, l = tid & 31;
#pragma unroll
    for (int q = 0; q < 9; ++q) {
        double v = acc[q];
        for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
        if (l == 0) red[wp][q] = v;
    }
    __syncthreads();
    if (tid < 9) {
        double v = 0.0;
        for (int ww = 0; ww < NT / 32; ++ww) v += red[ww][tid];
        partials[(long long)blockIdx.x * 9 + tid] += v;
    }
}

}  // namespace adj32

bool adjoint32_supported(const Geom& g) {
    return g.nx % adj32::TX == 0 && g.ny % adj32::TY == 0 && g.nx >= adj32::TX &&
           g.ny >= adj32::TY;
}

static int adjoint32_tz(const Geom& g) {
    static int slots = -1;
    if (slots < 0) slots = resident_slots((const void*)adj32::adjB_kernel, adj32::NT, adj32::SMEM);
    // shorter chunks suit this kernel: at 256^3, 19 planes 0.37 ms, 26: 0.38, 37: 0.42
    return zchunk_len((g.nx / adj32::TX) * (g.ny / adj32::TY), g.nz, slots, 16, 24);
}

int adjoint32_blocks(const Geom& g) {
    const int tz = adjoint32_tz(g);
    return (g.nx / adj32::TX) * (g.ny / adj32::TY) * ((g.nz + tz - 1) / tz);
}

bool adjoint32_prepare() {
    return cudaFuncSetAttribute(adj32::adjB_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)adj32::SMEM) == cudaSuccess;
}

void launch_adjoint32_B(const FusedMaps& maps, const Geom& g, const Mult<float>& m,
                        FieldSet<float> lam, const float* spy, const float* spz, double* partials,
                        int* err, cudaStream_t st) {
    adj32::adjB_kernel<<<adjoint32_blocks(g), adj32::NT, adj32::SMEM, st>>>(
        maps, g, m, lam, spy, spz, partials, adjoint32_tz(g), err);
}

}  // namespace fdtd
