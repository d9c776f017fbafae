// FP32 adjoint B half-step with the fused coefficient gradient, E^n staged by TMA.
//
// Computes, for every owned cell (see fdtd_adjoint.cu for the derivation),
//   mu = S (lambda_B + dt G^T (S lambda_E))            -> written to lambda_B (in place)
//   g_theta += mu . (dF/dtheta) E^n                     -> FP32 per thread, FP64 per block
// where (dF/dtheta) E^n are the derivative brackets of the extended stencil (Eq. D* with alpha
// eliminated by Eq. alpha).  The brackets need E^n at x-1..x+2, y-1..y+2, z-1..z+2 around the
// cell: E^n planes arrive by TMA as 72 x 12 boxes into a five-slot shared ring (same schedule
// as the fused forward step), and each thread evaluates the brackets of four consecutive
// cells from 16-byte shared-memory row windows.  lambda_E (own cell and its +x, +y, +z
// neighbours) and lambda_B (own cell) are read from HBM directly; only mu is written.
//
// Every mbarrier wait is bounded; on expiry the CTA raises *err, drains its copies in flight
// (bounded) and returns.
#include "fdtd_tma.cuh"

namespace fdtd {
namespace adj32 {

constexpr int TX = 64, TY = 8, D = 1, NT = 128;   // z-chunk length: launch parameter
constexpr int EW = TX + 8, EH = TY + 4, EPL = EW * EH;
constexpr int ESLOT = ((EPL * 4 + 127) / 128) * 128 / 4;
constexpr int NE = D + 4, NS = D + 1;
constexpr size_t OFF_BAR = (size_t)NE * 3 * ESLOT * 4;
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

__device__ __forceinline__ void unpack(float4 a, float o[4]) {
    o[0] = a.x; o[1] = a.y; o[2] = a.z; o[3] = a.w;
}

// derivative brackets of D*_A (without 1/dx_A) for four cells at in-plane index e:
//   dd = (F[+2a] - F[-a]) - 3 ax,  db = (F[+a+b] - F[+b]) + (F[+a-b] - F[-b]) - 2 ax,
//   dc likewise for the second transverse axis, ax = F[+a] - F[0]
template <int A>
__device__ __forceinline__ void brackets4(const float* Fm, const float* F0, const float* F1,
                                          const float* F2, int e, float dd[4], float db[4],
                                          float dc[4]) {
    if constexpr (A == 0) {   // axis x; b = y, c = z
        const Win w0 = win(F0, e), wyp = win(F0, e + EW), wym = win(F0, e - EW);
        const Win w1 = win(F1, e), wm = win(Fm, e);
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const float ax = w0.v[5 + u] - w0.v[4 + u];
            dd[u] = (w0.v[6 + u] - w0.v[3 + u]) - 3.0f * ax;
            db[u] = (wyp.v[5 + u] - wyp.v[4 + u]) + (wym.v[5 + u] - wym.v[4 + u]) - 2.0f * ax;
            dc[u] = (w1.v[5 + u] - w1.v[4 + u]) + (wm.v[5 + u] - wm.v[4 + u]) - 2.0f * ax;
        }
    } else if constexpr (A == 1) {   // axis y; b = x, c = z
        const Win w0 = win(F0, e), wyp = win(F0, e + EW);
        float a2[4], am[4], c1[4], c1p[4], cm[4], cmp[4];
        unpack(ld4(F0, e + 2 * EW), a2);
        unpack(ld4(F0, e - EW), am);
        unpack(ld4(F1, e), c1);
        unpack(ld4(F1, e + EW), c1p);
        unpack(ld4(Fm, e), cm);
        unpack(ld4(Fm, e + EW), cmp);
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const float ax = wyp.v[4 + u] - w0.v[4 + u];
            dd[u] = (a2[u] - am[u]) - 3.0f * ax;
            db[u] = (wyp.v[5 + u] - w0.v[5 + u]) + (wyp.v[3 + u] - w0.v[3 + u]) - 2.0f * ax;
            dc[u] = (c1p[u] - c1[u]) + (cmp[u] - cm[u]) - 2.0f * ax;
        }
    } else {   // axis z; b = x, c = y
        const Win w1 = win(F1, e), w0 = win(F0, e);
        float a2[4], am[4], p1[4], p0[4], m1[4], m0[4];
        unpack(ld4(F2, e), a2);
        unpack(ld4(Fm, e), am);
        unpack(ld4(F1, e + EW), p1);
        unpack(ld4(F0, e + EW), p0);
        unpack(ld4(F1, e - EW), m1);
        unpack(ld4(F0, e - EW), m0);
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const float ax = w1.v[4 + u] - w0.v[4 + u];
            dd[u] = (a2[u] - am[u]) - 3.0f * ax;
            db[u] = (w1.v[5 + u] - w0.v[5 + u]) + (w1.v[3 + u] - w0.v[3 + u]) - 2.0f * ax;
            dc[u] = (p1[u] - p0[u]) + (m1[u] - m0[u]) - 2.0f * ax;
        }
    }
}

__device__ __forceinline__ void st4(float* F, long long idx, float4 v) {
    *reinterpret_cast<float4*>(F + idx) = v;
}

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
    const long long Y = g.nxp;
    // lambda of this thread's cells (own, +x, +y, +z; lambda_B own), prefetched one plane ahead
    struct Lam {
        float ex[5], ey[5], ez[5], exy[4], ezy[4], exz[4], eyz[4], bx[4], by[4], bz[4];
    } L;
    auto load_lam = [&](int q) {
        const int qw = wrapz(q);
        const long long c = ((long long)qw * g.nyp + j + PY) * g.nxp + PX + i0;
        const long long zp = (long long)(wrapz(q + 1) - qw) * g.plane;
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
    for (; it < niter; ++it) {
        const int p = z0 + it;
        bool ok = true;
        if (it == 0) ok = mbar_wait(&bar[NS], 0);
        ok = ok && mbar_wait(&bar[it % NS], (uint32_t)((it / NS) & 1));
        if (ok) {
            const int pw = wrapz(p);
            const long long c = ((long long)pw * g.nyp + j + PY) * g.nxp + PX + i0;
            // l_E = S lambda_E at the cells and their +x, +y, +z neighbours
            float s0 = 1.0f, syp = 1.0f, szp = 1.0f;
            if (spy != nullptr) {
                const int jp = j + 1 < g.ny ? j + 1 : 0;
                s0 = spy[j] * spz[pw];
                syp = spy[jp] * spz[pw];
                szp = spy[j] * spz[wrapz(p + 1)];
            }
            float mux[4], muy[4], muz[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const float ex0 = s0 * L.ex[u], ey0 = s0 * L.ey[u], ez0 = s0 * L.ez[u];
                const float ezx = s0 * L.ez[u + 1];
                const float eyx = s0 * L.ey[u + 1];
                const float nx_ = L.bx[u] + (m.cE[2] * (ey0 - szp * L.eyz[u]) - m.cE[1] * (ez0 - syp * L.ezy[u]));
                const float ny_ = L.by[u] + (m.cE[0] * (ez0 - ezx) - m.cE[2] * (ex0 - szp * L.exz[u]));
                const float nz_ = L.bz[u] + (m.cE[1] * (ex0 - syp * L.exy[u]) - m.cE[0] * (ey0 - eyx));
                mux[u] = s0 * nx_;
                muy[u] = s0 * ny_;
                muz[u] = s0 * nz_;
            }
            if (it + 1 < niter) load_lam(p + 1);
            // gradient brackets from the E^n ring
            float dd[4], db[4], dc[4], fd[4], fb[4], fc[4];
            brackets4<0>(Ep(p - 1, 2), Ep(p, 2), Ep(p + 1, 2), nullptr, e, dd, db, dc);   // D*_x E_z
            brackets4<0>(Ep(p - 1, 1), Ep(p, 1), Ep(p + 1, 1), nullptr, e, fd, fb, fc);   // D*_x E_y
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                racc[0] += muy[u] * dd[u] - muz[u] * fd[u];
                racc[1] += muy[u] * db[u] - muz[u] * fb[u];
                racc[2] += muy[u] * dc[u] - muz[u] * fc[u];
            }
            brackets4<1>(Ep(p - 1, 0), Ep(p, 0), Ep(p + 1, 0), nullptr, e, dd, db, dc);   // D*_y E_x
            brackets4<1>(Ep(p - 1, 2), Ep(p, 2), Ep(p + 1, 2), nullptr, e, fd, fb, fc);   // D*_y E_z
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                racc[3] += muz[u] * dd[u] - mux[u] * fd[u];
                racc[4] += muz[u] * db[u] - mux[u] * fb[u];
                racc[5] += muz[u] * dc[u] - mux[u] * fc[u];
            }
            brackets4<2>(Ep(p - 1, 1), Ep(p, 1), Ep(p + 1, 1), Ep(p + 2, 1), e, dd, db, dc);   // D*_z E_y
            brackets4<2>(Ep(p - 1, 0), Ep(p, 0), Ep(p + 1, 0), Ep(p + 2, 0), e, fd, fb, fc);   // D*_z E_x
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                racc[6] += mux[u] * dd[u] - muy[u] * fd[u];
                racc[7] += mux[u] * db[u] - muy[u] * fb[u];
                racc[8] += mux[u] * dc[u] - muy[u] * fc[u];
            }
#pragma unroll
            for (int q = 0; q < 9; ++q) {   // one FP64 add per 4 cells and coefficient
                acc[q] += (double)racc[q];
                racc[q] = 0.0f;
            }
            // mu -> lambda_B (own cells and, at the domain edge, their images)
            const float4 vx = make_float4(mux[0], mux[1], mux[2], mux[3]);
            const float4 vy = make_float4(muy[0], muy[1], muy[2], muy[3]);
            const float4 vz = make_float4(muz[0], muz[1], muz[2], muz[3]);
            if (!edge) {
                st4(lam.c[3], c, vx);
                st4(lam.c[4], c, vy);
                st4(lam.c[5], c, vz);
            } else {
                for (int u = 0; u < 4; ++u) {
                    store_img(g, lam.c[3], i0 + u, j, pw, mux[u]);
                    store_img(g, lam.c[4], i0 + u, j, pw, muy[u]);
                    store_img(g, lam.c[5], i0 + u, j, pw, muz[u]);
                }
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
        if (tid == 0) {
            atomicExch(err, 1);
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
