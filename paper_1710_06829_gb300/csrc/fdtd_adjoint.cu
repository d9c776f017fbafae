// Adjoint (transposed) leapfrog step with the fused stencil-coefficient gradient.
//
// The forward step is u^{n+1} = M u^n + s^n with
//   B1 = S (B0 + dt F E0),   E1 = S (E0 + dt (G B1 - J)),
// F E = -D* x E (extended stencil, Eq. D*), G B = D x B (Yee), S the diagonal
// sponge (identity without absorbing layers).  For the adjoint state
// lambda = (lambda_E, lambda_B) attached to u^{n+1}:
//   l_E = S lambda_E,   mu = S (lambda_B + dt G^T l_E),
//   lambda_E <- l_E + dt F^T mu,   lambda_B <- mu,
//   dL/dtheta += dt <mu, (dF/dtheta) E0>.
// With alpha eliminated by Eq. (alpha), for D*_a applied to a field F:
//   d/d delta_a:  [(F[+2a] - F[-a]) - 3 (F[+a] - F[0])] / dx_a
//   d/d beta_ab:  [(F[+a+b] - F[+b]) + (F[+a-b] - F[-b]) - 2 (F[+a] - F[0])] / dx_a
// Kernel adjB computes mu (written to lambda_B) and the gradient partials;
// kernel adjE then updates lambda_E from the new lambda_B.
#include "fdtd_internal.cuh"

namespace fdtd {

__device__ __forceinline__ long long zoff_a(const Geom& g, int k, int dz) {
    int kk = (k + dz) % g.nz;
    if (kk < 0) kk += g.nz;
    return (long long)(kk - k) * g.plane;
}

template <typename T>
__device__ __forceinline__ void store_images_a(const Geom& g, T* F, int i, int j, int k, T v) {
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

// sponge factor of the cell whose owned index is (j, k) possibly shifted by one
template <typename T>
__device__ __forceinline__ T sp_at(const Geom& g, const T* spy, const T* spz, int j, int k) {
    if (spy == nullptr) return T(1);
    int jj = j % g.ny;
    if (jj < 0) jj += g.ny;
    int kk = k % g.nz;
    if (kk < 0) kk += g.nz;
    return spy[jj] * spz[kk];
}

// Gradient brackets of D*_a at c for field F: returns (d/d delta_a, d/d beta_ab, d/d beta_ac)
// without the 1/dx_a factor.
template <typename T>
__device__ __forceinline__ void dcoef(const T* __restrict__ F, long long c, long long a1,
                                      long long a2, long long am1, long long bp, long long bm,
                                      long long cp, long long cm, T& dd, T& db, T& dc) {
    const T ax = F[c + a1] - F[c];
    dd = (F[c + a2] - F[c + am1]) - T(3) * ax;
    db = (F[c + a1 + bp] - F[c + bp]) + (F[c + a1 + bm] - F[c + bm]) - T(2) * ax;
    dc = (F[c + a1 + cp] - F[c + cp]) + (F[c + a1 + cm] - F[c + cm]) - T(2) * ax;
}

constexpr int ADJ_THREADS = 256;

int adjoint_B_blocks(const Geom& g) {
    long long b = (long long)g.ny * g.nz;   // one x-row per block and sweep
    if (b > 152 * 8) b = 152 * 8;
    return (int)b;
}

// partials layout: [block][9] = per axis a (x, y, z): d/d delta_a, d/d beta_a,b1, d/d beta_a,b2
// with b1 < b2 the two other axes.  Accumulated across steps (+=) by the owning block.
// A block walks whole x-rows (j, k); each thread sums at most ADJ_FLUSH cell terms in the
// field precision before adding them to its FP64 accumulators, so the FP64 pipe (slow on
// this part) sees one add per ADJ_FLUSH cells; block and grid totals are FP64.
constexpr int ADJ_FLUSH = 16;

template <typename T>
__global__ void __launch_bounds__(ADJ_THREADS)
adjoint_B_kernel(Geom g, Mult<T> m, FieldSet<T> lam, const T* __restrict__ Ex,
                 const T* __restrict__ Ey, const T* __restrict__ Ez, const T* __restrict__ spy,
                 const T* __restrict__ spz, double* __restrict__ partials) {
    double acc[9];
    T racc[9];
#pragma unroll
    for (int q = 0; q < 9; ++q) {
        acc[q] = 0.0;
        racc[q] = T(0);
    }
    int cnt = 0;
    const int rows = g.ny * g.nz;
    const long long Y = g.nxp;
    const T* lEx = lam.c[0];
    const T* lEy = lam.c[1];
    const T* lEz = lam.c[2];
    for (int r = blockIdx.x; r < rows; r += gridDim.x) {
        const int j = r % g.ny, k = r / g.ny;
        const long long rowbase = pidx(g, 0, j, k);
        const long long zp1 = zoff_a(g, k, 1), zm1 = zoff_a(g, k, -1), zp2 = zoff_a(g, k, 2);
        // l_E = S lambda_E at the cell and its +x, +y, +z neighbours
        const T s0 = sp_at(g, spy, spz, j, k);
        const T sxp = s0;
        const T syp = sp_at(g, spy, spz, j + 1, k);
        const T szp = sp_at(g, spy, spz, j, k + 1);
        for (int i = threadIdx.x; i < g.nx; i += blockDim.x) {
            const long long c = rowbase + i;
            const T ex0 = s0 * lEx[c], ey0 = s0 * lEy[c], ez0 = s0 * lEz[c];
            // G^T l_E (transposed backward differences = forward differences with a minus sign)
            T nx_ = lam.c[3][c] + (m.cE[2] * (ey0 - szp * lEy[c + zp1]) - m.cE[1] * (ez0 - syp * lEz[c + Y]));
            T ny_ = lam.c[4][c] + (m.cE[0] * (ez0 - sxp * lEz[c + 1]) - m.cE[2] * (ex0 - szp * lEx[c + zp1]));
            T nz_ = lam.c[5][c] + (m.cE[1] * (ex0 - syp * lEx[c + Y]) - m.cE[0] * (ey0 - sxp * lEy[c + 1]));
            const T mux = s0 * nx_, muy = s0 * ny_, muz = s0 * nz_;
            // gradient: axis x appears as +mu_y D*_x E_z - mu_z D*_x E_y
            T d0, d1, d2, e0, e1, e2;
            dcoef(Ez, c, 1, 2, -1, Y, -Y, zp1, zm1, d0, d1, d2);
            dcoef(Ey, c, 1, 2, -1, Y, -Y, zp1, zm1, e0, e1, e2);
            racc[0] += muy * d0 - muz * e0;
            racc[1] += muy * d1 - muz * e1;
            racc[2] += muy * d2 - muz * e2;
            // axis y: +mu_z D*_y E_x - mu_x D*_y E_z   (transverse order x, z)
            dcoef(Ex, c, Y, 2 * Y, -Y, 1, -1, zp1, zm1, d0, d1, d2);
            dcoef(Ez, c, Y, 2 * Y, -Y, 1, -1, zp1, zm1, e0, e1, e2);
            racc[3] += muz * d0 - mux * e0;
            racc[4] += muz * d1 - mux * e1;
            racc[5] += muz * d2 - mux * e2;
            // axis z: +mu_x D*_z E_y - mu_y D*_z E_x   (transverse order x, y)
            dcoef(Ey, c, zp1, zp2, zm1, 1, -1, Y, -Y, d0, d1, d2);
            dcoef(Ex, c, zp1, zp2, zm1, 1, -1, Y, -Y, e0, e1, e2);
            racc[6] += mux * d0 - muy * e0;
            racc[7] += mux * d1 - muy * e1;
            racc[8] += mux * d2 - muy * e2;
            if (++cnt == ADJ_FLUSH) {
#pragma unroll
                for (int q = 0; q < 9; ++q) {
                    acc[q] += (double)racc[q];
                    racc[q] = T(0);
                }
                cnt = 0;
            }
            store_images_a(g, lam.c[3], i, j, k, mux);
            store_images_a(g, lam.c[4], i, j, k, muy);
            store_images_a(g, lam.c[5], i, j, k, muz);
        }
    }
#pragma unroll
    for (int q = 0; q < 9; ++q) acc[q] += (double)racc[q];
    __shared__ double red[ADJ_THREADS / 32][9];
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
#pragma unroll
    for (int q = 0; q < 9; ++q) {
        double v = acc[q];
        for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
        if (l == 0) red[w][q] = v;
    }
    __syncthreads();
    if (threadIdx.x < 9) {
        double v = 0.0;
        for (int ww = 0; ww < ADJ_THREADS / 32; ++ww) v += red[ww][threadIdx.x];
        partials[(long long)blockIdx.x * 9 + threadIdx.x] += v;
    }
}

// lambda_E <- S lambda_E + dt F^T mu,  F^T from the transposed taps of D*:
//   (D*_a)^T G = alpha_a (G[-a] - G[0]) + delta_a (G[-2a] - G[+a])
//              + sum_b beta_ab ((G[-a-b] - G[-b]) + (G[-a+b] - G[+b])).
template <typename T>
__device__ __forceinline__ T dstarT_at(const T* __restrict__ G, long long c, long long am1,
                                       long long am2, long long ap1, long long bp, long long bm,
                                       long long cp, long long cm, T cA, T cD, T cBb, T cBc) {
    T v = cA * (G[c + am1] - G[c]);
    v = fma(cD, G[c + am2] - G[c + ap1], v);
    v = fma(cBb, (G[c + am1 + bm] - G[c + bm]) + (G[c + am1 + bp] - G[c + bp]), v);
    v = fma(cBc, (G[c + am1 + cm] - G[c + cm]) + (G[c + am1 + cp] - G[c + cp]), v);
    return v;
}

template <typename T>
__global__ void adjoint_E_kernel(Geom g, Mult<T> m, FieldSet<T> lam, const T* __restrict__ spy,
                                 const T* __restrict__ spz) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= g.nx) return;
    for (int k = blockIdx.z; k < g.nz; k += gridDim.z)
        for (int j = blockIdx.y; j < g.ny; j += gridDim.y) {
            const long long c = pidx(g, i, j, k);
            const long long Y = g.nxp;
            const long long zp1 = zoff_a(g, k, 1), zm1 = zoff_a(g, k, -1), zm2 = zoff_a(g, k, -2);
            const T* mux = lam.c[3];
            const T* muy = lam.c[4];
            const T* muz = lam.c[5];
#define DTX(G) dstarT_at(G, c, -1, -2, 1, Y, -Y, zp1, zm1, m.cA[0], m.cD[0], m.cB[0][1], m.cB[0][2])
#define DTY(G) dstarT_at(G, c, -Y, -2 * Y, Y, 1, -1, zp1, zm1, m.cA[1], m.cD[1], m.cB[1][0], m.cB[1][2])
#define DTZ(G) dstarT_at(G, c, zm1, zm2, zp1, 1, -1, Y, -Y, m.cA[2], m.cD[2], m.cB[2][0], m.cB[2][1])
            const T s0 = sp_at(g, spy, spz, j, k);
            const T ex = s0 * lam.c[0][c] + (DTY(muz) - DTZ(muy));
            const T ey = s0 * lam.c[1][c] + (DTZ(mux) - DTX(muz));
            const T ez = s0 * lam.c[2][c] + (DTX(muy) - DTY(mux));
#undef DTX
#undef DTY
#undef DTZ
            store_images_a(g, lam.c[0], i, j, k, ex);
            store_images_a(g, lam.c[1], i, j, k, ey);
            store_images_a(g, lam.c[2], i, j, k, ez);
        }
}

template <typename T>
void launch_adjoint_B_v0(const Geom& g, const Mult<T>& m, FieldSet<T> lam, const T* E_hist[3],
                         const T* sponge_y, const T* sponge_z, double* partials, int nblk,
                         cudaStream_t st) {
    adjoint_B_kernel<T><<<nblk, ADJ_THREADS, 0, st>>>(g, m, lam, E_hist[0], E_hist[1], E_hist[2],
                                                        sponge_y, sponge_z, partials);
}

template <typename T>
void launch_adjoint_E_v0(const Geom& g, const Mult<T>& m, FieldSet<T> lam, const T* sponge_y,
                         const T* sponge_z, cudaStream_t st) {
    dim3 blk(128), grd((g.nx + 127) / 128, (unsigned)(g.ny < 65535 ? g.ny : 65535),
                        (unsigned)(g.nz < 65535 ? g.nz : 65535));   // j, k loop in the kernel
    adjoint_E_kernel<T><<<grd, blk, 0, st>>>(g, m, lam, sponge_y, sponge_z);
}

template void launch_adjoint_B_v0<float>(const Geom&, const Mult<float>&, FieldSet<float>,
                                         const float* [3], const float*, const float*, double*,
                                         int, cudaStream_t);
template void launch_adjoint_B_v0<double>(const Geom&, const Mult<double>&, FieldSet<double>,
                                          const double* [3], const double*, const double*,
                                          double*, int, cudaStream_t);
template void launch_adjoint_E_v0<float>(const Geom&, const Mult<float>&, FieldSet<float>,
                                         const float*, const float*, cudaStream_t);
template void launch_adjoint_E_v0<double>(const Geom&, const Mult<double>&, FieldSet<double>,
                                          const double*, const double*, cudaStream_t);

// grad12[beta row-major 3x3, delta 3] += scale_a * sum_b partials[b][.]  (one block, fixed order)
__global__ void reduce_grad_kernel(const double* __restrict__ part, int nblocks, GradScale sc,
                                   double* __restrict__ grad) {
    __shared__ double red[9][32];
    const int q = threadIdx.y;       // 0..8
    const int l = threadIdx.x;       // 0..31
    double v = 0.0;
    for (int b = l; b < nblocks; b += 32) v += part[(long long)b * 9 + q];
    red[q][l] = v;
    __syncthreads();
    if (l == 0) {
        double s = 0.0;
        for (int t = 0; t < 32; ++t) s += red[q][t];
        const int a = q / 3, which = q % 3;
        if (which == 0) {
            grad[9 + a] += sc.s[q] * s;
        } else {
            // transverse axes of a in increasing order
            const int b = (which == 1) ? (a == 0 ? 1 : 0) : (a == 2 ? 1 : 2);
            grad[a * 3 + b] += sc.s[q] * s;
        }
    }
}

void launch_reduce_grad(const double* part, int nblocks, GradScale sc, double* grad12,
                        cudaStream_t st) {
    reduce_grad_kernel<<<1, dim3(32, 9), 0, st>>>(part, nblocks, sc, grad12);
}

}  // namespace fdtd
