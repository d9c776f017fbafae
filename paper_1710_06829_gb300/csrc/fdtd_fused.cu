// Fused leapfrog step: one launch advances (E^n, B^{n-1/2}) -> (E^{n+1}, B^{n+1/2}).
//
// Each CTA owns a TX x TY tile in (x, y) and a chunk of TZ planes in z and
// marches through it plane by plane.  For plane p it
//   1. computes B^{n+1/2} on the tile plus one halo column (x0-1) and one halo
//      row (y0-1) from E^n planes p-1 .. p+2 (extended stencil, Eq. D*) and
//      B^{n-1/2} plane p;  the tile part is written to HBM;
//   2. computes E^{n+1} on plane p from E^n(p), B^{n+1/2}(p) and B^{n+1/2}(p-1)
//      (Yee stencil) and writes it to HBM.
// E^n planes arrive as (TX+8) x (TY+4) boxes and B^{n-1/2} planes as
// (TX+4) x (TY+1) boxes through TMA (cp.async.bulk.tensor) into a ring of
// shared-memory slots, D planes ahead of use, completion signalled on
// mbarriers.  Every HBM byte of the state is read once and written once per
// step apart from the tile halos (served mostly by L2).  Inputs and outputs are
// different buffers (ping-pong), so neighbouring CTAs never see a half-updated
// state.  The padded layout (see fdtd_internal.cuh) keeps every box inside
// the array: no wrap in x or y inside a tile; z wraps by plane index.
//
// Arithmetic goes through dstar_taps / ampere_comp, the same helpers as the
// reference-form kernels, so both produce bitwise-identical fields.
//
// Every mbarrier wait is bounded; on expiry the CTA raises *err, waits (again
// bounded) for its copies in flight and returns without writing.
#include <type_traits>

#include "fdtd_tma.cuh"

namespace fdtd {

template <typename T>
struct FusedCfg;

template <>
struct FusedCfg<float> {
    static constexpr int TX = 64, TY = 8, TZ = 32, D = 2, NT = 256;
};
template <>
struct FusedCfg<double> {
    static constexpr int TX = 64, TY = 8, TZ = 32, D = 1, NT = 256;
};

template <typename T>
struct Layout {
    using C = FusedCfg<T>;
    static constexpr int TX = C::TX, TY = C::TY;
    static constexpr int EW = TX + 8, EH = TY + 4, EPL = EW * EH;   // E box: x0-4 .. x0+TX+3, y0-2 .. y0+TY+1
    static constexpr int BW = TX + 4, BH = TY + 1, BPL = BW * BH;   // B box: x0-4 .. x0+TX-1, y0-1 .. y0+TY-1
    static constexpr int NE = C::D + 4, NB = C::D + 1, NS = C::D + 1;
    static constexpr int ESLOT = ((EPL * (int)sizeof(T) + 127) / 128) * 128 / (int)sizeof(T);
    static constexpr int BSLOT = ((BPL * (int)sizeof(T) + 127) / 128) * 128 / (int)sizeof(T);
    static constexpr size_t OFF_E = 0;
    static constexpr size_t OFF_BOLD = OFF_E + (size_t)NE * 3 * ESLOT * sizeof(T);
    static constexpr size_t OFF_BNEW = OFF_BOLD + (size_t)NB * 3 * BSLOT * sizeof(T);
    static constexpr size_t OFF_BAR = OFF_BNEW + (size_t)2 * 3 * BSLOT * sizeof(T);
    static constexpr size_t SMEM = OFF_BAR + (size_t)(NS + 1) * 8;
    static constexpr uint32_t UNIT_BYTES = 3u * EPL * sizeof(T) + 3u * BPL * sizeof(T);
    static constexpr uint32_t PRO_BYTES = 9u * EPL * sizeof(T);
};

// ---------------------------------------------------------------- kernel

template <typename T>
__global__ void __launch_bounds__(FusedCfg<T>::NT)
step_fused_kernel(const __grid_constant__ FusedMaps maps, Geom g, Mult<T> m, FieldSet<T> out,
                  const T* __restrict__ spy, const T* __restrict__ spz,
                  const T* __restrict__ jyz, const T* __restrict__ jx_row, T* __restrict__ h0,
                  T* __restrict__ h1, T* __restrict__ h2, int* __restrict__ err) {
    using Lc = Layout<T>;
    constexpr int TX = Lc::TX, TY = Lc::TY, TZ = FusedCfg<T>::TZ, D = FusedCfg<T>::D;
    constexpr int NT = FusedCfg<T>::NT;
    constexpr int EW = Lc::EW, BW = Lc::BW;
    constexpr int NE = Lc::NE, NB = Lc::NB, NS = Lc::NS;
    extern __shared__ __align__(128) unsigned char smem[];
    T* sE = reinterpret_cast<T*>(smem + Lc::OFF_E);
    T* sBo = reinterpret_cast<T*>(smem + Lc::OFF_BOLD);
    T* sBn = reinterpret_cast<T*>(smem + Lc::OFF_BNEW);
    uint64_t* bar = reinterpret_cast<uint64_t*>(smem + Lc::OFF_BAR);

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

    auto wrapz = [&](int q) {
        int r = q % g.nz;
        return r < 0 ? r + g.nz : r;
    };
    auto eslot = [&](int q) { return (q - (z0 - 2)) % NE; };
    auto Eplane = [&](int q, int c) { return sE + ((size_t)eslot(q) * 3 + c) * Lc::ESLOT; };
    auto issue_unit = [&](int u) {
        const int p = z0 - 1 + u;
        const int qe = p + 2;
        uint64_t* b = &bar[u % NS];
        mbar_expect_tx(b, Lc::UNIT_BYTES);
        for (int c = 0; c < 3; ++c) tma_load_3d(Eplane(qe, c), &maps.e[c], x0, y0, wrapz(qe), b);
        for (int c = 0; c < 3; ++c)
            tma_load_3d(sBo + ((size_t)(u % NB) * 3 + c) * Lc::BSLOT, &maps.b[c], x0, y0 + 1,
                        wrapz(p), b);
    };

    if (tid == 0) {
        for (int s = 0; s <= NS; ++s) mbar_init(&bar[s], 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    }
    __syncthreads();
    int issued = 0;   // units issued (thread 0 only)
    if (tid == 0) {
        mbar_expect_tx(&bar[NS], Lc::PRO_BYTES);
        for (int q = z0 - 2; q <= z0; ++q)
            for (int c = 0; c < 3; ++c) tma_load_3d(Eplane(q, c), &maps.e[c], x0, y0, wrapz(q), &bar[NS]);
        for (int u = 0; u <= D && u < niter; ++u) {
            issue_unit(u);
            issued = u + 1;
        }
    }

    const T mdt = -m.dt;
    bool failed = false;
    T fin = T(0);   // non-finite detection (nonfinite_acc): stays 0 while every E value is finite
    int it = 0;
    for (; it < niter; ++it) {
        const int p = z0 - 1 + it;
        bool ok = true;
        if (it == 0) ok = mbar_wait(&bar[NS], 0);
        ok = ok && mbar_wait(&bar[it % NS], (uint32_t)((it / NS) & 1));
        if (__syncthreads_or(!ok)) {
            failed = true;
            break;
        }
        const int pw = wrapz(p);
        // ---- 1. B^{n+1/2} on plane p: tile plus halo column x0-1 and halo row y0-1
        {
            const T* Bo = sBo + (size_t)(it % NB) * 3 * Lc::BSLOT;
            T* Bn = sBn + (size_t)(p & 1) * 3 * Lc::BSLOT;
            const T* Em[3] = {Eplane(p - 1, 0), Eplane(p - 1, 1), Eplane(p - 1, 2)};
            const T* E0[3] = {Eplane(p, 0), Eplane(p, 1), Eplane(p, 2)};
            const T* E1[3] = {Eplane(p + 1, 0), Eplane(p + 1, 1), Eplane(p + 1, 2)};
            const T* E2[3] = {Eplane(p + 2, 0), Eplane(p + 2, 1), Eplane(p + 2, 2)};
            for (int cc = tid; cc < (TX + 1) * (TY + 1); cc += NT) {
                const int bx = cc % (TX + 1) - 1, by = cc / (TX + 1) - 1;
                const int e = (by + 2) * EW + (bx + 4);
                const int bi = (by + 1) * BW + (bx + 4);
                // D*_x F: axial x, transverse y (+-EW), then z (planes p+1 / p-1)
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
                T bxv = Bo[0 * Lc::BSLOT + bi] + (DZ(1) - DY(2));
                T byv = Bo[1 * Lc::BSLOT + bi] + (DX(2) - DZ(0));
                T bzv = Bo[2 * Lc::BSLOT + bi] + (DY(0) - DX(1));
#undef DX
#undef DY
#undef DZ
                if (spy != nullptr) {
                    int yy = y0 + by;
                    if (yy < 0) yy += g.ny;
                    const T f = spy[yy] * spz[pw];
                    bxv *= f;
                    byv *= f;
                    bzv *= f;
                }
                Bn[0 * Lc::BSLOT + bi] = bxv;
                Bn[1 * Lc::BSLOT + bi] = byv;
                Bn[2 * Lc::BSLOT + bi] = bzv;
                if (p >= z0 && bx >= 0 && by >= 0) {
                    store_img(g, out.c[3], x0 + bx, y0 + by, pw, bxv);
                    store_img(g, out.c[4], x0 + bx, y0 + by, pw, byv);
                    store_img(g, out.c[5], x0 + bx, y0 + by, pw, bzv);
                }
            }
        }
        __syncthreads();
        // ---- 2. E^{n+1} on plane p
        if (p >= z0) {
            const T* Bc = sBn + (size_t)(p & 1) * 3 * Lc::BSLOT;
            const T* Bp = sBn + (size_t)((p - 1) & 1) * 3 * Lc::BSLOT;
            const T* E0x = Eplane(p, 0);
            const T* E0y = Eplane(p, 1);
            const T* E0z = Eplane(p, 2);
            const T* Bx = Bc;
            const T* By = Bc + Lc::BSLOT;
            const T* Bz = Bc + 2 * Lc::BSLOT;
            const T* Bxm = Bp;
            const T* Bym = Bp + Lc::BSLOT;
            for (int cc = tid; cc < TX * TY; cc += NT) {
                const int bx = cc % TX, by = cc / TX;
                const int e = (by + 2) * EW + (bx + 4);
                const int bi = (by + 1) * BW + (bx + 4);
                T ex = ampere_comp(E0x[e], Bz[bi], Bz[bi - BW], By[bi], Bym[bi], m.cE[1], m.cE[2]);
                T ey = ampere_comp(E0y[e], Bx[bi], Bxm[bi], Bz[bi], Bz[bi - 1], m.cE[2], m.cE[0]);
                T ez = ampere_comp(E0z[e], By[bi], By[bi - 1], Bx[bi], Bx[bi - BW], m.cE[0], m.cE[1]);
                const int i = x0 + bx, j = y0 + by;
                if (jx_row != nullptr) {
                    const T jx = (jx_row[i] * jyz[j]) * jyz[g.ny + pw];
                    ex = fma(mdt, jx, ex);
                }
                if (spy != nullptr) {
                    const T f = spy[j] * spz[pw];
                    ex *= f;
                    ey *= f;
                    ez *= f;
                }
                fin = nonfinite_acc(nonfinite_acc(nonfinite_acc(fin, ex), ey), ez);
                store_img(g, out.c[0], i, j, pw, ex);
                store_img(g, out.c[1], i, j, pw, ey);
                store_img(g, out.c[2], i, j, pw, ez);
                if (h0 != nullptr) {
                    store_img(g, h0, i, j, pw, ex);
                    store_img(g, h1, i, j, pw, ey);
                    store_img(g, h2, i, j, pw, ez);
                }
            }
        }
        __syncthreads();
        if (tid == 0 && it + D + 1 < niter) {
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            issue_unit(it + D + 1);
            issued = it + D + 2;
        }
    }
    if (!(fin == T(0))) atomicOr(err, ERR_FIELD);
    if (failed) {
        // drain the copies this CTA still has in flight (bounded), then report
        if (tid == 0) {
            atomicOr(err, ERR_WAIT);
            if (it == 0) mbar_wait(&bar[NS], 0);
            for (int u = it; u < issued; ++u) mbar_wait(&bar[u % NS], (uint32_t)((u / NS) & 1));
        }
        __syncthreads();
    }
}

// ---------------------------------------------------------------- host side

typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*,
                                  const cuuint64_t*, const cuuint64_t*, const cuuint32_t*,
                                  const cuuint32_t*, CUtensorMapInterleave, CUtensorMapSwizzle,
                                  CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

static EncodeTiledFn encode_fn() {
    static EncodeTiledFn fn = nullptr;
    if (!fn) {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault,
                                             &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = (EncodeTiledFn)p;
    }
    return fn;
}

void launch_fused32_range(const FusedMaps& maps, FieldSet<float> in, const Geom& g,
                          const Mult<float>& m, FieldSet<float> out, const float* spy,
                          const float* spz, int zs, int ze, int* err, cudaStream_t st);
bool fused32_supported(const Geom& g);
int fused32_ebox_w();
bool fused32_prepare();
void launch_fused32(const FusedMaps& maps, FieldSet<float> in, const Geom& g, const Mult<float>& m,
                    FieldSet<float> out, const float* spy, const float* spz, const float* jyz,
                    const float* jx_row, float* hist_E[3], int* err, cudaStream_t st);

template <typename T>
bool fused_supported(const Geom& g) {
    if constexpr (std::is_same<T, float>::value) return fused32_supported(g);
    using C = FusedCfg<T>;
    return g.nx % C::TX == 0 && g.ny % C::TY == 0 && g.nx >= C::TX && g.ny >= C::TY;
}

template <typename T>
static bool encode(CUtensorMap* map, const Geom& g, T* base, int bw, int bh) {
    EncodeTiledFn fn = encode_fn();
    if (!fn) return false;
    const cuuint64_t dims[3] = {(cuuint64_t)g.nxp, (cuuint64_t)g.nyp, (cuuint64_t)g.nz};
    const cuuint64_t strides[2] = {(cuuint64_t)g.nxp * sizeof(T), (cuuint64_t)g.plane * sizeof(T)};
    const cuuint32_t box[3] = {(cuuint32_t)bw, (cuuint32_t)bh, 1};
    const cuuint32_t estr[3] = {1, 1, 1};
    const CUtensorMapDataType dt =
        sizeof(T) == 4 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32 : CU_TENSOR_MAP_DATA_TYPE_FLOAT64;
    return fn(map, dt, 3, (void*)base, dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
              CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
              CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

// E^n box (72 x 12, FP32) of one padded array, as the adjoint kernel reads it
bool encode_ebox_f32(CUtensorMap* map, const Geom& g, float* base) {
    return encode<float>(map, g, base, Layout<float>::EW, Layout<float>::EH);
}

// a bw x bh box (FP32) of one padded array
bool encode_box_f32(CUtensorMap* map, const Geom& g, float* base, int bw, int bh) {
    return encode<float>(map, g, base, bw, bh);
}

template <typename T>
FusedPlan* fused_plan_create(const Geom& g, T* const set0[6], T* const set1[6]) {
    if (!fused_supported<T>(g)) return nullptr;
    FusedPlan* p = new FusedPlan();
    p->dtype = sizeof(T) == 4 ? FDTD_F32 : FDTD_F64;
    using Lc = Layout<T>;
    for (int s = 0; s < 2; ++s) {
        T* const* set = s == 0 ? set0 : set1;
        for (int c = 0; c < 3; ++c) {
            const int ew = std::is_same<T, float>::value ? fused32_ebox_w() : Lc::EW;
            if (!encode<T>(&p->maps[s].e[c], g, set[c], ew, Lc::EH) ||
                !encode<T>(&p->maps[s].b[c], g, set[3 + c], Lc::BW, Lc::BH)) {
                delete p;
                return nullptr;
            }
        }
    }
    bool ok;
    if constexpr (std::is_same<T, float>::value)
        ok = fused32_prepare();
    else
        ok = cudaFuncSetAttribute(step_fused_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)Lc::SMEM) == cudaSuccess;
    if (!ok) {
        delete p;
        return nullptr;
    }
    return p;
}

void fused_plan_destroy(FusedPlan* p) { delete p; }

void launch_step_fused32_range(const FusedPlan* plan, int in_set, const Geom& g,
                               const Mult<float>& m, FieldSet<float> in, FieldSet<float> out,
                               const float* sponge_y, const float* sponge_z, int zs, int ze,
                               int* err, cudaStream_t st) {
    launch_fused32_range(plan->maps[in_set], in, g, m, out, sponge_y, sponge_z, zs, ze, err, st);
}

// ---------------------------------------------------------------- L2 discard

// Drops the 128-byte lines [lo[c], hi[c]) (line indices of absolute addresses) of six arrays
// from L2 without writing them back (discard.global.L2); their contents become undefined.
__global__ void discard_l2_kernel(unsigned long long lo0, unsigned long long lo1,
                                  unsigned long long lo2, unsigned long long lo3,
                                  unsigned long long lo4, unsigned long long lo5,
                                  unsigned long long n) {
    const unsigned long long lo[6] = {lo0, lo1, lo2, lo3, lo4, lo5};
    const unsigned long long stride = (unsigned long long)gridDim.x * blockDim.x;
    for (unsigned long long t = (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x; t < 6 * n;
         t += stride) {
        const unsigned long long a = (lo[t / n] + t % n) * 128ull;
        asm volatile("discard.global.L2 [%0], 128;" ::"l"(a) : "memory");
    }
}

void launch_discard_planes(const Geom& g, size_t esz, void* const arr[6], int p0, int p1,
                           cudaStream_t st) {
    if (p1 <= p0) return;
    const unsigned long long pb = (unsigned long long)g.plane * esz;
    unsigned long long lo[6];
    unsigned long long n = ~0ull;
    for (int c = 0; c < 6; ++c) {
        const unsigned long long b = reinterpret_cast<unsigned long long>(arr[c]);
        const unsigned long long first = (b + p0 * pb + 127) / 128, last = (b + p1 * pb) / 128;
        lo[c] = first;
        const unsigned long long nc = last > first ? last - first : 0;
        n = nc < n ? nc : n;   // the arrays have equal sizes and alignments in practice
    }
    if (n == 0) return;
    const unsigned long long total = 6 * n;
    const int blk = 256;
    const int grd = (int)((total + blk - 1) / blk < 4096 ? (total + blk - 1) / blk : 4096);
    discard_l2_kernel<<<grd, blk, 0, st>>>(lo[0], lo[1], lo[2], lo[3], lo[4], lo[5], n);
}

template <typename T>
void launch_step_fused(const FusedPlan* plan, int in_set, const Geom& g, const Mult<T>& m,
                       FieldSet<T> in, FieldSet<T> out, const T* sponge_y, const T* sponge_z,
                       const T* jyz, const T* jx_row, T* hist_E[3], int* err, cudaStream_t st) {
    if constexpr (std::is_same<T, float>::value) {
        launch_fused32(plan->maps[in_set], in, g, m, out, sponge_y, sponge_z, jyz, jx_row, hist_E,
                       err, st);
        return;
    }
    using C = FusedCfg<T>;
    const int nblk = (g.nx / C::TX) * (g.ny / C::TY) * ((g.nz + C::TZ - 1) / C::TZ);
    step_fused_kernel<T><<<nblk, C::NT, Layout<T>::SMEM, st>>>(
        plan->maps[in_set], g, m, out, sponge_y, sponge_z, jyz, jx_row, hist_E[0], hist_E[1],
        hist_E[2], err);
}

template bool fused_supported<float>(const Geom&);
template bool fused_supported<double>(const Geom&);
template FusedPlan* fused_plan_create<float>(const Geom&, float* const[6], float* const[6]);
template FusedPlan* fused_plan_create<double>(const Geom&, double* const[6], double* const[6]);
template void launch_step_fused<float>(const FusedPlan*, int, const Geom&, const Mult<float>&,
                                       FieldSet<float>, FieldSet<float>, const float*, const float*, const float*,
                                       const float*, float* [3], int*, cudaStream_t);
template void launch_step_fused<double>(const FusedPlan*, int, const Geom&, const Mult<double>&,
                                        FieldSet<double>, FieldSet<double>, const double*, const double*,
                                        const double*, const double*, double* [3], int*,
                                        cudaStream_t);

}  // namespace fdtd
