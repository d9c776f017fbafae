// Macro-particle kernels of the PIC cycle: gather + Boris push + Esirkepov current, and the
// charge density.
//
// Particle shape: first order (cloud in cell); node i of axis a carries max(0, 1 - |x/dx_a - i|).
// Gather: each field component is interpolated from its own staggered positions (App. A):
//   E_x (i+1/2, j, k), E_y (i, j+1/2, k), E_z (i, j, k+1/2),
//   B_x (i, j+1/2, k+1/2), B_y (i+1/2, j, k+1/2), B_z (i+1/2, j+1/2, k),
// with B at the integer time level the mean of B^{n-1/2} and B^{n+1/2}.
// Push: Boris's relativistic scheme in u = gamma v (c = 1): half electric kick, rotation
// about t = (q/m)(dt/2) B / gamma^-, half electric kick; then x += dt u / gamma.
// Current: Esirkepov's decomposition of the shape change S1 - S0 into W_x + W_y + W_z,
//   W_x = dSx (S0y S0z + dSy S0z / 2 + S0y dSz / 2 + dSy dSz / 3)   (and cyclically),
//   J_x(i+1/2) - J_x(i-1/2) = -q W_x(i) / (dt dy dz),
// so that (rho^{n+1} - rho^n)/dt + D.J^{n+1/2} = 0 holds to rounding (App. A numerical
// continuity equation) and Gauss's law D.E = rho (Eq. divE) is kept.  A particle moves less
// than a cell per step (|v| < c, c dt < dx on any stable grid), so per axis its old and new
// supports fit a 3-node window starting at floor(g0) + min(0, floor(g1) - floor(g0)); each
// particle adds at most 2 x 3 x 3 face values per component with global reductions.
//
// One thread per particle, grid-stride; the J arrays use the padded field layout (owned cells
// only, no images: the Ampere kernel reads owned cells).
#include <cmath>

#include "pic.cuh"

namespace fdtd {
namespace picd {

constexpr int THREADS = 256;

__device__ __forceinline__ int wrapi(int i, int n) {
    int r = i % n;
    return r < 0 ? r + n : r;
}

// first-order weights of grid coordinate gc on nodes i0 = floor(gc) and i1 = i0 + 1 (wrapped)
template <typename T>
struct Lin {
    int i0, i1;
    T w0, w1;
};

template <typename T>
__device__ __forceinline__ Lin<T> lin(T gc, int n) {
    const T f = floor(gc);
    Lin<T> l;
    l.w1 = gc - f;
    l.w0 = T(1) - l.w1;
    l.i0 = wrapi((int)f, n);
    l.i1 = l.i0 + 1 == n ? 0 : l.i0 + 1;
    return l;
}

template <typename T>
__device__ __forceinline__ T gather(const T* __restrict__ F, const Geom& g, const Lin<T>& a,
                                    const Lin<T>& b, const Lin<T>& c) {
    T out = T(0);
#pragma unroll
    for (int ia = 0; ia < 2; ++ia)
#pragma unroll
        for (int ib = 0; ib < 2; ++ib)
#pragma unroll
            for (int ic = 0; ic < 2; ++ic) {
                const T w = (ia ? a.w1 : a.w0) * (ib ? b.w1 : b.w0) * (ic ? c.w1 : c.w0);
                out += w * F[pidx(g, ia ? a.i1 : a.i0, ib ? b.i1 : b.i0, ic ? c.i1 : c.i0)];
            }
    return out;
}

// the same for the time mean (F0 + F1) / 2
template <typename T>
__device__ __forceinline__ T gather_mean(const T* __restrict__ F0, const T* __restrict__ F1,
                                         const Geom& g, const Lin<T>& a, const Lin<T>& b,
                                         const Lin<T>& c) {
    T out = T(0);
#pragma unroll
    for (int ia = 0; ia < 2; ++ia)
#pragma unroll
        for (int ib = 0; ib < 2; ++ib)
#pragma unroll
            for (int ic = 0; ic < 2; ++ic) {
                const long long o = pidx(g, ia ? a.i1 : a.i0, ib ? b.i1 : b.i0, ic ? c.i1 : c.i0);
                const T w = (ia ? a.w1 : a.w0) * (ib ? b.w1 : b.w0) * (ic ? c.w1 : c.w0);
                out += w * (T(0.5) * (F0[o] + F1[o]));
            }
    return out;
}

// old-shape weights, shape change and absolute first node of the 3-node window of one axis
template <typename T>
struct Win {
    int start;
    T S0[3], dS[3];
};

template <typename T>
__device__ __forceinline__ Win<T> window(T g0, T g1) {
    const T f0 = floor(g0), f1 = floor(g1);
    const int s = (int)(f1 - f0);   // -1, 0 or 1 for a move of less than one cell
    Win<T> w;
    w.start = (int)f0 + (s < 0 ? s : 0);
#pragma unroll
    for (int m = 0; m < 3; ++m) {
        const T node = (T)(w.start + m);
        const T s0 = fmax(T(0), T(1) - fabs(g0 - node));
        const T s1 = fmax(T(0), T(1) - fabs(g1 - node));
        w.S0[m] = s0;
        w.dS[m] = s1 - s0;
    }
    return w;
}

template <typename T>
__device__ __forceinline__ bool finite3(T a, T b, T c) {
    return isfinite(a) && isfinite(b) && isfinite(c);
}

// J_a face values of one particle: axis a carries the cumulative sum, b and c the weights
template <typename T>
__device__ __forceinline__ void deposit_axis(T* __restrict__ J, const Geom& g, const Win<T>& wa,
                                             const Win<T>& wb, const Win<T>& wc, int na, int nb,
                                             int nc, int axis, T scale) {
    const T third = T(1) / T(3);
#pragma unroll
    for (int mb = 0; mb < 3; ++mb)
#pragma unroll
        for (int mc = 0; mc < 3; ++mc) {
            const T f = wb.S0[mb] * wc.S0[mc] + T(0.5) * wb.dS[mb] * wc.S0[mc] +
                        T(0.5) * wb.S0[mb] * wc.dS[mc] + third * wb.dS[mb] * wc.dS[mc];
            if (f == T(0)) continue;
            const T c0 = wa.dS[0] * f;
            const T c1 = c0 + wa.dS[1] * f;
            const int ib = wrapi(wb.start + mb, nb), ic = wrapi(wc.start + mc, nc);
#pragma unroll
            for (int ma = 0; ma < 2; ++ma) {
                const T v = ma == 0 ? c0 : c1;
                if (v == T(0)) continue;
                const int ia = wrapi(wa.start + ma, na);
                int i, j, k;
                if (axis == 0) { i = ia; j = ib; k = ic; }
                else if (axis == 1) { i = ib; j = ia; k = ic; }
                else { i = ib; j = ic; k = ia; }
                atomicAdd(J + pidx(g, i, j, k), scale * v);
            }
        }
}

template <typename T>
__global__ void __launch_bounds__(THREADS) push_kernel(PushArgs<T> a) {
    const Geom& g = a.g;
    const T lim = T(1073741824);   // 2^30 cells
    for (long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x; p < a.n;
         p += (long long)gridDim.x * blockDim.x) {
        const T x = a.x[0][p], y = a.x[1][p], z = a.x[2][p];
        const T ux = a.u[0][p], uy = a.u[1][p], uz = a.u[2][p];
        if (!finite3(x, y, z) || !finite3(ux, uy, uz)) {
            atomicOr(a.err, 2);
            continue;
        }
        const T gx = x * a.inv_dx[0], gy = y * a.inv_dx[1], gz = z * a.inv_dx[2];
        if (fabs(gx) > lim || fabs(gy) > lim || fabs(gz) > lim) {
            atomicOr(a.err, 2);
            continue;
        }
        // ---- gather at x^n
        const Lin<T> nx_ = lin(gx, g.nx), ny_ = lin(gy, g.ny), nz_ = lin(gz, g.nz);
        const Lin<T> sx = lin(gx - T(0.5), g.nx), sy = lin(gy - T(0.5), g.ny),
                     sz = lin(gz - T(0.5), g.nz);
        const T Ex = gather(a.E[0], g, sx, ny_, nz_);
        const T Ey = gather(a.E[1], g, nx_, sy, nz_);
        const T Ez = gather(a.E[2], g, nx_, ny_, sz);
        const T Bx = gather_mean(a.B0[0], a.B1[0], g, nx_, sy, sz);
        const T By = gather_mean(a.B0[1], a.B1[1], g, sx, ny_, sz);
        const T Bz = gather_mean(a.B0[2], a.B1[2], g, sx, sy, nz_);
        // ---- Boris push u^{n-1/2} -> u^{n+1/2}
        const T h = a.h;
        const T umx = ux + h * Ex, umy = uy + h * Ey, umz = uz + h * Ez;
        const T gm = sqrt(T(1) + umx * umx + umy * umy + umz * umz);
        const T tx = h * Bx / gm, ty = h * By / gm, tz = h * Bz / gm;
        const T t2 = tx * tx + ty * ty + tz * tz;
        const T den = T(1) + t2;
        const T sxv = T(2) * tx / den, syv = T(2) * ty / den, szv = T(2) * tz / den;
        const T upx = umx + (umy * tz - umz * ty);
        const T upy = umy + (umz * tx - umx * tz);
        const T upz = umz + (umx * ty - umy * tx);
        const T u1x = umx + (upy * szv - upz * syv) + h * Ex;
        const T u1y = umy + (upz * sxv - upx * szv) + h * Ey;
        const T u1z = umz + (upx * syv - upy * sxv) + h * Ez;
        const T g1 = sqrt(T(1) + u1x * u1x + u1y * u1y + u1z * u1z);
        const T x1 = x + a.dt * u1x / g1, y1 = y + a.dt * u1y / g1, z1 = z + a.dt * u1z / g1;
        // ---- Esirkepov current J^{n+1/2} from x^n -> x^{n+1}
        const Win<T> wx = window(gx, x1 * a.inv_dx[0]);
        const Win<T> wy = window(gy, y1 * a.inv_dx[1]);
        const Win<T> wz = window(gz, z1 * a.inv_dx[2]);
        deposit_axis(a.J[0], g, wx, wy, wz, g.nx, g.ny, g.nz, 0, a.jscale[0]);
        deposit_axis(a.J[1], g, wy, wx, wz, g.ny, g.nx, g.nz, 1, a.jscale[1]);
        deposit_axis(a.J[2], g, wz, wx, wy, g.nz, g.nx, g.ny, 2, a.jscale[2]);
        // ---- new state, positions wrapped into [0, L)
        T xw = x1, yw = y1, zw = z1;
        if (xw < T(0)) xw += a.L[0]; else if (xw >= a.L[0]) xw -= a.L[0];
        if (yw < T(0)) yw += a.L[1]; else if (yw >= a.L[1]) yw -= a.L[1];
        if (zw < T(0)) zw += a.L[2]; else if (zw >= a.L[2]) zw -= a.L[2];
        a.x[0][p] = xw; a.x[1][p] = yw; a.x[2][p] = zw;
        a.u[0][p] = u1x; a.u[1][p] = u1y; a.u[2][p] = u1z;
    }
}

template <typename T>
__global__ void __launch_bounds__(THREADS)
rho_kernel(Geom g, const T* __restrict__ x0, const T* __restrict__ x1, const T* __restrict__ x2,
           long long n, T ix, T iy, T iz, T scale, T* __restrict__ rho, int* err) {
    const T lim = T(1073741824);
    for (long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x; p < n;
         p += (long long)gridDim.x * blockDim.x) {
        const T gx = x0[p] * ix, gy = x1[p] * iy, gz = x2[p] * iz;
        if (!finite3(gx, gy, gz) || fabs(gx) > lim || fabs(gy) > lim || fabs(gz) > lim) {
            atomicOr(err, 2);
            continue;
        }
        const Lin<T> a = lin(gx, g.nx), b = lin(gy, g.ny), c = lin(gz, g.nz);
#pragma unroll
        for (int ia = 0; ia < 2; ++ia)
#pragma unroll
            for (int ib = 0; ib < 2; ++ib)
#pragma unroll
                for (int ic = 0; ic < 2; ++ic) {
                    const T w = (ia ? a.w1 : a.w0) * (ib ? b.w1 : b.w0) * (ic ? c.w1 : c.w0);
                    const long long o = ((long long)(ic ? c.i1 : c.i0) * g.ny + (ib ? b.i1 : b.i0)) * g.nx +
                                        (ia ? a.i1 : a.i0);
                    if (w != T(0)) atomicAdd(rho + o, scale * w);
                }
    }
}

inline unsigned blocks_for(long long n) {
    long long b = (n + THREADS - 1) / THREADS;
    if (b > 152LL * 16) b = 152LL * 16;
    if (b < 1) b = 1;
    return (unsigned)b;
}

}  // namespace picd

template <typename T>
void launch_pic_push(const PushArgs<T>& a, cudaStream_t st) {
    if (a.n <= 0) return;
    picd::push_kernel<T><<<picd::blocks_for(a.n), picd::THREADS, 0, st>>>(a);
}

template <typename T>
void launch_deposit_rho(const Geom& g, const T* const x[3], long long n, const T inv_dx[3],
                        T scale, T* rho, int* err, cudaStream_t st) {
    if (n <= 0) return;
    picd::rho_kernel<T><<<picd::blocks_for(n), picd::THREADS, 0, st>>>(
        g, x[0], x[1], x[2], n, inv_dx[0], inv_dx[1], inv_dx[2], scale, rho, err);
}

template void launch_pic_push<float>(const PushArgs<float>&, cudaStream_t);
template void launch_pic_push<double>(const PushArgs<double>&, cudaStream_t);
template void launch_deposit_rho<float>(const Geom&, const float* const[3], long long,
                                        const float[3], float, float*, int*, cudaStream_t);
template void launch_deposit_rho<double>(const Geom&, const double* const[3], long long,
                                         const double[3], double, double*, int*, cudaStream_t);

}  // namespace fdtd
