// Diagnostics on the library-owned state (all accumulation in FP64, deterministic).
//
//   energy in a window:   (1/2) sum (E^2 + B^2) dV over cells with i in the periodic x-window
//                          [x_lo, x_lo + x_len) and j, k inside [margin, n - margin);
//   plane-wave amplitude:  sum_cells F_c exp(-i k . r_c), r_c the component's staggered
//                          position (App. A) -- the measured phase advance per step gives the
//                          scheme's omega(k) (Sec. 3), its envelope the group velocity (Sec. 5);
//   energy moments:        sum e (1, cos th, sin th) dV with e = (1/2) F^2 per component at its
//                          staggered position and th = 2 pi x_a / L_a along one axis: the
//                          circular mean atan2(S, C) L_a / 2 pi is the centroid of a wave
//                          packet on the periodic grid, its speed the group velocity (Sec. 5);
//   divergences:           D* . B (Eq. divstarb, extended stencil), Yee D . B and D . E
//                          (Eq. divE) written per cell to a dense caller buffer.
// Partials: one FP64 value (or pair) per block, summed in a fixed order by one block.
#include <cmath>

#include "fdtd_internal.cuh"

namespace fdtd {

constexpr int DG_THREADS = 256;

int diag_blocks(const Geom& g) {
    const long long cells = (long long)g.nx * g.ny * g.nz;
    long long b = (cells + DG_THREADS - 1) / DG_THREADS;
    if (b > 152 * 8) b = 152 * 8;
    if (b < 1) b = 1;
    return (int)b;
}

template <int NV>
__device__ __forceinline__ void block_reduce_store(double (&v)[NV], double* __restrict__ part) {
    __shared__ double red[DG_THREADS / 32][NV];
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
#pragma unroll
    for (int q = 0; q < NV; ++q) {
        double x = v[q];
        for (int o = 16; o > 0; o >>= 1) x += __shfl_down_sync(0xffffffffu, x, o);
        if (l == 0) red[w][q] = x;
    }
    __syncthreads();
    if (threadIdx.x < NV) {
        double x = 0.0;
        for (int ww = 0; ww < DG_THREADS / 32; ++ww) x += red[ww][threadIdx.x];
        part[(long long)blockIdx.x * NV + threadIdx.x] = x;
    }
}

template <typename T>
__global__ void __launch_bounds__(DG_THREADS)
energy_kernel(Geom g, FieldSet<T> s, int x_lo, int x_len, int my, int mz, double* part) {
    double acc[1] = {0.0};
    const long long n = (long long)x_len * (g.ny - 2 * my) * (g.nz - 2 * mz);
    const int ny_in = g.ny - 2 * my;
    for (long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x; t < n;
         t += (long long)gridDim.x * blockDim.x) {
        const int ii = (int)(t % x_len);
        const long long r = t / x_len;
        const int j = my + (int)(r % ny_in);
        const int k = mz + (int)(r / ny_in);
        int i = (x_lo + ii) % g.nx;
        if (i < 0) i += g.nx;
        const long long c = pidx(g, i, j, k);
#pragma unroll
        for (int q = 0; q < 6; ++q) {
            const double v = (double)s.c[q][c];
            acc[0] += v * v;
        }
    }
    block_reduce_store<1>(acc, part);
}

// sum F exp(-i k.r) with r = ((i + ox) dx, (j + oy) dy, (k + oz) dz); phases in FP64
template <typename T>
__global__ void __launch_bounds__(DG_THREADS)
planewave_kernel(Geom g, const T* __restrict__ F, double kx, double ky, double kz, double ox,
                 double oy, double oz, double* part) {
    double acc[2] = {0.0, 0.0};
    const long long n = (long long)g.nx * g.ny * g.nz;
    for (long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x; t < n;
         t += (long long)gridDim.x * blockDim.x) {
        const int i = (int)(t % g.nx);
        const long long r = t / g.nx;
        const int j = (int)(r % g.ny);
        const int k = (int)(r / g.ny);
        const double ph = kx * (i + ox) + ky * (j + oy) + kz * (k + oz);
        double sn, cs;
        sincos(ph, &sn, &cs);
        const double v = (double)F[pidx(g, i, j, k)];
        acc[0] += v * cs;
        acc[1] -= v * sn;
    }
    block_reduce_store<2>(acc, part);
}

// sum over components and cells of (1/2) F^2 (1, cos th, sin th), th = 2 pi (idx_a + off) / n_a
// with off = 1/2 for the components staggered along a (App. A positions)
template <typename T>
__global__ void __launch_bounds__(DG_THREADS)
moments_kernel(Geom g, FieldSet<T> s, int axis, double* part) {
    double acc[3] = {0.0, 0.0, 0.0};
    const long long n = (long long)g.nx * g.ny * g.nz;
    const int na = axis == 0 ? g.nx : axis == 1 ? g.ny : g.nz;
    const double w = 2.0 * M_PI / na;
    // staggered along `axis`: E_a, and the two B components other than B_a
    bool half[6];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        half[c] = c == axis;
        half[3 + c] = c != axis;
    }
    for (long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x; t < n;
         t += (long long)gridDim.x * blockDim.x) {
        const int i = (int)(t % g.nx);
        const long long r = t / g.nx;
        const int j = (int)(r % g.ny);
        const int k = (int)(r / g.ny);
        const int ia = axis == 0 ? i : axis == 1 ? j : k;
        double s0, c0, sh, ch;
        sincos(w * ia, &s0, &c0);
        sincos(w * (ia + 0.5), &sh, &ch);
        const long long c = pidx(g, i, j, k);
        double e0 = 0.0, eh = 0.0;
#pragma unroll
        for (int q = 0; q < 6; ++q) {
            const double v = (double)s.c[q][c];
            if (half[q]) eh += v * v;
            else e0 += v * v;
        }
        acc[0] += e0 + eh;
        acc[1] += e0 * c0 + eh * ch;
        acc[2] += e0 * s0 + eh * sh;
    }
    block_reduce_store<3>(acc, part);
}

__global__ void final_sum_kernel(const double* __restrict__ part, int nblocks, int nv, double scale,
                                 double* __restrict__ out) {
    __shared__ double red[4][32];
    const int q = threadIdx.y, l = threadIdx.x;
    double v = 0.0;
    for (int b = l; b < nblocks; b += 32) v += part[(long long)b * nv + q];
    red[q][l] = v;
    __syncthreads();
    if (l == 0) {
        double s = 0.0;
        for (int t = 0; t < 32; ++t) s += red[q][t];
        out[q] = scale * s;
    }
}

// ---- divergences (dense output, FP64) -----------------------------------------------------

__device__ __forceinline__ long long zo(const Geom& g, int k, int dz) {
    int kk = (k + dz) % g.nz;
    if (kk < 0) kk += g.nz;
    return (long long)(kk - k) * g.plane;
}

// which: 0 = D*.B (extended, forward type, at cell corners), 1 = Yee D.B (forward type),
//        2 = D.E (Yee, backward type, at nodes).  Multipliers carry 1/dx (not dt).
template <typename T>
__global__ void divergence_kernel(Geom g, Mult<double> w, FieldSet<T> s, int which,
                                  double* __restrict__ out) {
    const long long n = (long long)g.nx * g.ny * g.nz;
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= n) return;
    const int i = (int)(t % g.nx);
    const long long r = t / g.nx;
    const int j = (int)(r % g.ny);
    const int k = (int)(r / g.ny);
    const long long c = pidx(g, i, j, k);
    const long long Y = g.nxp;
    const long long zp1 = zo(g, k, 1), zm1 = zo(g, k, -1), zp2 = zo(g, k, 2);
    double v = 0.0;
    if (which == 2) {
        const T* Ex = s.c[0];
        const T* Ey = s.c[1];
        const T* Ez = s.c[2];
        v = w.cE[0] * ((double)Ex[c] - (double)Ex[c - 1]) + w.cE[1] * ((double)Ey[c] - (double)Ey[c - Y]) +
            w.cE[2] * ((double)Ez[c] - (double)Ez[c + zm1]);
    } else {
        const T* B[3] = {s.c[3], s.c[4], s.c[5]};
        const long long a1[3] = {1, Y, zp1}, a2[3] = {2, 2 * Y, zp2}, am1[3] = {-1, -Y, zm1};
        const long long tp[3][2] = {{Y, zp1}, {1, zp1}, {1, Y}};
        const long long tm[3][2] = {{-Y, zm1}, {-1, zm1}, {-1, -Y}};
        for (int a = 0; a < 3; ++a) {
            const T* F = B[a];
            const double ax = (double)F[c + a1[a]] - (double)F[c];
            if (which == 1) {
                v += w.cE[a] * ax;
                continue;
            }
            double d = w.cA[a] * ax + w.cD[a] * ((double)F[c + a2[a]] - (double)F[c + am1[a]]);
            const int b[2] = {a == 0 ? 1 : 0, a == 2 ? 1 : 2};
            for (int q = 0; q < 2; ++q) {
                d += w.cB[a][b[q]] * (((double)F[c + a1[a] + tp[a][q]] - (double)F[c + tp[a][q]]) +
                                      ((double)F[c + a1[a] + tm[a][q]] - (double)F[c + tm[a][q]]));
            }
            v += d;
        }
    }
    out[t] = v;
}

template <typename T>
void launch_energy(const Geom& g, FieldSet<T> s, int x_lo, int x_len, int my, int mz, double dV,
                   double* part, double* out, cudaStream_t st) {
    const int nb = diag_blocks(g);
    energy_kernel<T><<<nb, DG_THREADS, 0, st>>>(g, s, x_lo, x_len, my, mz, part);
    final_sum_kernel<<<1, dim3(32, 1), 0, st>>>(part, nb, 1, 0.5 * dV, out);
}

template <typename T>
void launch_planewave(const Geom& g, const T* F, const double k[3], const double off[3],
                      double* part, double* out, cudaStream_t st) {
    const int nb = diag_blocks(g);
    planewave_kernel<T><<<nb, DG_THREADS, 0, st>>>(g, F, k[0], k[1], k[2], off[0], off[1], off[2],
                                                   part);
    final_sum_kernel<<<1, dim3(32, 2), 0, st>>>(part, nb, 2, 1.0, out);
}

template <typename T>
void launch_moments(const Geom& g, FieldSet<T> s, int axis, double dV, double* part, double* out,
                    cudaStream_t st) {
    const int nb = diag_blocks(g);
    moments_kernel<T><<<nb, DG_THREADS, 0, st>>>(g, s, axis, part);
    final_sum_kernel<<<1, dim3(32, 3), 0, st>>>(part, nb, 3, 0.5 * dV, out);
}

template <typename T>
void launch_divergence(const Geom& g, const Mult<double>& w, FieldSet<T> s, int which, double* out,
                       cudaStream_t st) {
    const long long n = (long long)g.nx * g.ny * g.nz;
    divergence_kernel<T><<<(unsigned)((n + 255) / 256), 256, 0, st>>>(g, w, s, which, out);
}

template void launch_energy<float>(const Geom&, FieldSet<float>, int, int, int, int, double,
                                   double*, double*, cudaStream_t);
template void launch_energy<double>(const Geom&, FieldSet<double>, int, int, int, int, double,
                                    double*, double*, cudaStream_t);
template void launch_planewave<float>(const Geom&, const float*, const double[3], const double[3],
                                      double*, double*, cudaStream_t);
template void launch_planewave<double>(const Geom&, const double*, const double[3],
                                       const double[3], double*, double*, cudaStream_t);
template void launch_moments<float>(const Geom&, FieldSet<float>, int, double, double*, double*,
                                    cudaStream_t);
template void launch_moments<double>(const Geom&, FieldSet<double>, int, double, double*, double*,
                                     cudaStream_t);
template void launch_divergence<float>(const Geom&, const Mult<double>&, FieldSet<float>, int,
                                       double*, cudaStream_t);
template void launch_divergence<double>(const Geom&, const Mult<double>&, FieldSet<double>, int,
                                        double*, cudaStream_t);

}  // namespace fdtd
