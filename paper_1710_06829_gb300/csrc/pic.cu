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
// supports fit the 4-node window floor(g0) - 1 .. floor(g0) + 2.
//
// Ampere's law is linear in J, so the cycle first forms E^{n+1} without the current (the
// vacuum step kernel) and the push adds -dt J^{n+1/2} into its owned cells: no current
// array, no extra pass over the grid; a small kernel then copies the owned cells near the x
// and y ends to their periodic images (the ghosts the next step reads).
//
// Warps move through the particle array together.  When all 32 particles of a warp sit in one
// cell (a dense bunch, particles kept in cell order), the warp loads the 3 x 3 x 3 node block
// of each field once (27 lanes) and every particle interpolates from it by shuffles, and each
// face value of the current is summed over the warp by shuffles before one global addition;
// otherwise every lane gathers and adds on its own.
#include <climits>
#include <cmath>

#include "pic.cuh"

namespace fdtd {
namespace picd {

constexpr int THREADS = 256;
constexpr unsigned FULL = 0xffffffffu;

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

// old-shape weights and shape change on the 4-node window f0 - 1 .. f0 + 2 of one axis
// (f0 = floor(g0)): it holds the old support (f0, f0 + 1) and, for a move of less than one
// cell, the new one; it depends on the old position only, so particles of one cell share it
template <typename T>
struct Win {
    int idx[4];   // the four nodes, wrapped into [0, n)
    T s1, s2;     // old-shape weights of nodes f0, f0 + 1 (those of f0 - 1 and f0 + 2 are 0)
    T dS[4];      // shape change S1 - S0 on the four nodes
    __device__ __forceinline__ T S0(int m) const { return m == 1 ? s1 : (m == 2 ? s2 : T(0)); }
};

template <typename T>
__device__ __forceinline__ Win<T> window(T g0, T g1, int n) {
    const T f0 = floor(g0);
    Win<T> w;
    w.idx[0] = wrapi((int)f0 - 1, n);
#pragma unroll
    for (int m = 1; m < 4; ++m) w.idx[m] = w.idx[m - 1] + 1 == n ? 0 : w.idx[m - 1] + 1;
#pragma unroll
    for (int m = 0; m < 4; ++m) {
        const T node = f0 + (T)(m - 1);
        const T s0 = fmax(T(0), T(1) - fabs(g0 - node));
        const T s1 = fmax(T(0), T(1) - fabs(g1 - node));
        if (m == 1) w.s1 = s0;
        if (m == 2) w.s2 = s0;
        w.dS[m] = s1 - s0;
    }
    return w;
}

// a finite coordinate moved into [0, L] (unchanged when already inside)
template <typename T>
__device__ __forceinline__ T into_box(T x, T L) {
    if (x >= T(0) && x < L) return x;
    const T r = x - L * floor(x / L);
    return r < T(0) ? T(0) : (r > L ? L : r);
}

template <typename T>
__device__ __forceinline__ bool finite3(T a, T b, T c) {
    return isfinite(a) && isfinite(b) && isfinite(c);
}

// where -dt J goes: the owned cells of E^{n+1}, times the absorbing-layer factor if any
template <typename T>
struct Sink {
    T* E[3];
    const T* spy;
    const T* spz;
    Geom g;

    // owned cell (wrapped node indices); the ghosts are refreshed after the push
    __device__ __forceinline__ void add(int axis, int i, int j, int k, T v) const {
        if (spy != nullptr) v *= spy[j] * spz[k];
        T* Ea = axis == 0 ? E[0] : (axis == 1 ? E[1] : E[2]);   // no local-memory indexing
        atomicAdd(Ea + pidx(g, i, j, k), v);
    }
};

template <typename T>
__device__ __forceinline__ T warp_sum(T v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(FULL, v, o);
    return v;
}

template <typename T>
__device__ __forceinline__ T pick4(int m, T a, T b, T c, T d) {
    return m == 0 ? a : (m == 1 ? b : (m == 2 ? c : d));
}

template <typename T>
__device__ __forceinline__ Win<T> pick_win(int m, const Win<T>& a, const Win<T>& b,
                                           const Win<T>& c) {
    Win<T> w;
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        w.idx[q] = m == 0 ? a.idx[q] : (m == 1 ? b.idx[q] : c.idx[q]);
        w.dS[q] = m == 0 ? a.dS[q] : (m == 1 ? b.dS[q] : c.dS[q]);
    }
    w.s1 = m == 0 ? a.s1 : (m == 1 ? b.s1 : c.s1);
    w.s2 = m == 0 ? a.s2 : (m == 1 ? b.s2 : c.s2);
    return w;
}

// -dt J^{n+1/2} of one particle into E^{n+1}.  For component a the axis a carries the
// cumulative sum of W_a over its window (faces f0 - 1/2 .. f0 + 3/2; the sum over the whole
// window vanishes) and the other two axes b < c the weights; escale[a] = q / (dx_b dx_c)
// turns the cumulative sum into -dt J_a.  `uni` (warp-uniform): every lane of the warp is
// live with the same windows, so each face value is summed over the warp by shuffles and
// lane 0 adds it once; otherwise every lane adds its own values.  The axis, b and c loops stay
// rolled (operands picked by selects) to keep the kernel's code small: unrolled, the
// reduction sites made the kernel instruction-cache bound.
template <typename T>
__device__ __forceinline__ void deposit(const Sink<T>& sink, const Win<T>& wx, const Win<T>& wy,
                                        const Win<T>& wz, const T escale[3], bool uni) {
    const T third = T(1) / T(3);
    const bool lane0 = (threadIdx.x & 31) == 0;
#pragma unroll 1
    for (int axis = 0; axis < 3; ++axis) {
        const Win<T> wa = pick_win(axis, wx, wy, wz);
        const Win<T> wb = axis == 0 ? wy : wx;
        const Win<T> wc = axis == 2 ? wy : wz;
        const T scale = axis == 0 ? escale[0] : (axis == 1 ? escale[1] : escale[2]);
        const bool moved = wa.dS[0] != T(0) || wa.dS[1] != T(0) || wa.dS[2] != T(0);
        if (uni ? !__any_sync(FULL, moved) : !moved) continue;
#pragma unroll 1
        for (int mb = 0; mb < 4; ++mb) {
            const T s0b = wb.S0(mb);
            const T dsb = pick4(mb, wb.dS[0], wb.dS[1], wb.dS[2], wb.dS[3]);
            const int ib = pick4(mb, wb.idx[0], wb.idx[1], wb.idx[2], wb.idx[3]);
#pragma unroll 1
            for (int mc = 0; mc < 4; ++mc) {
                const T s0c = wc.S0(mc);
                const T dsc = pick4(mc, wc.dS[0], wc.dS[1], wc.dS[2], wc.dS[3]);
                const T f = s0b * s0c + T(0.5) * dsb * s0c + T(0.5) * s0b * dsc +
                            third * dsb * dsc;
                if (uni ? !__any_sync(FULL, f != T(0)) : f == T(0)) continue;
                const int ic = pick4(mc, wc.idx[0], wc.idx[1], wc.idx[2], wc.idx[3]);
                T cum = T(0);
#pragma unroll
                for (int ma = 0; ma < 3; ++ma) {
                    cum += wa.dS[ma] * f;
                    T v = scale * cum;
                    if (uni) {
                        v = warp_sum(v);
                        if (!lane0) continue;
                    }
                    if (v == T(0)) continue;
                    const int ia = wa.idx[ma];
                    // (i, j, k) of the face: axis a gets ia, the others ib (lower) and ic
                    const int i = axis == 0 ? ia : ib;
                    const int j = axis == 0 ? ib : (axis == 1 ? ia : ic);
                    const int k = axis == 2 ? ia : ic;
                    sink.add(axis, i, j, k, v);
                }
            }
        }
    }
}

// first-order weights of one axis relative to the node f0 - 1 of a warp whose particles all
// have old node f0: l0 (0 or 1) is the local index of the lower of the two nodes used
template <typename T>
struct Loc {
    int l0;
    T w0, w1;
};

template <typename T>
__device__ __forceinline__ Loc<T> loc(T gc, int f0) {
    const T f = floor(gc);
    Loc<T> l;
    l.w1 = gc - f;
    l.w0 = T(1) - l.w1;
    l.l0 = (int)f - (f0 - 1);
    return l;
}

// interpolation from the 3 x 3 x 3 node block of the warp (lane a + 3 b + 9 c holds node
// (f0x - 1 + a, f0y - 1 + b, f0z - 1 + c) of the component in `val`); the same weights and
// summation order as gather()
template <typename T>
__device__ __forceinline__ T interp27(T val, const Loc<T>& a, const Loc<T>& b, const Loc<T>& c) {
    T out = T(0);
#pragma unroll
    for (int ia = 0; ia < 2; ++ia)
#pragma unroll
        for (int ib = 0; ib < 2; ++ib)
#pragma unroll
            for (int ic = 0; ic < 2; ++ic) {
                const T w = (ia ? a.w1 : a.w0) * (ib ? b.w1 : b.w0) * (ic ? c.w1 : c.w0);
                const int lane = (a.l0 + ia) + 3 * (b.l0 + ib) + 9 * (c.l0 + ic);
                out += w * __shfl_sync(FULL, val, lane);
            }
    return out;
}

template <typename T>
__global__ void __launch_bounds__(THREADS, 4) push_kernel(PushArgs<T> a) {
    const Geom& g = a.g;
    Sink<T> sink;
    sink.g = g;
    for (int c = 0; c < 3; ++c) sink.E[c] = a.Eout[c];
    sink.spy = a.spy;
    sink.spz = a.spz;
    // the loop bound is warp-uniform, so every lane of a warp runs every iteration
    for (long long base = (long long)blockIdx.x * blockDim.x; base < a.n;
         base += (long long)gridDim.x * blockDim.x) {
        const long long p = base + threadIdx.x;
        bool live = p < a.n;
        T x = 0, y = 0, z = 0, ux = 0, uy = 0, uz = 0;
        if (live) {
            x = a.x[0][p]; y = a.x[1][p]; z = a.x[2][p];
            ux = a.u[0][p]; uy = a.u[1][p]; uz = a.u[2][p];
            if (!finite3(x, y, z) || !finite3(ux, uy, uz)) {
                atomicOr(a.err, ERR_PARTICLE);
                live = false;
            } else {
                x = into_box(x, a.L[0]); y = into_box(y, a.L[1]); z = into_box(z, a.L[2]);
            }
        }
        const T gx = x * a.inv_dx[0], gy = y * a.inv_dx[1], gz = z * a.inv_dx[2];
        const int fx = live ? (int)floor(gx) : 0, fy = live ? (int)floor(gy) : 0,
                  fz = live ? (int)floor(gz) : 0;
        // warp-uniform: all 32 particles live in one cell (same old node on every axis).  Every
        // lane reaches these shuffles (no short-circuit evaluation around them).
        const int f0x = __shfl_sync(FULL, fx, 0);
        const int f0y = __shfl_sync(FULL, fy, 0);
        const int f0z = __shfl_sync(FULL, fz, 0);
        const bool same = live && fx == f0x && fy == f0y && fz == f0z;
        const bool uni = __all_sync(FULL, same);
        // ---- gather at x^n
        T Ex = 0, Ey = 0, Ez = 0, Bx = 0, By = 0, Bz = 0;
        if (uni) {
            // the warp loads the 3 x 3 x 3 node block once (27 lanes, one value per array) and
            // every particle interpolates from it by shuffles
            const int l = threadIdx.x & 31;
            T v0 = 0, v1 = 0, v2 = 0, v3 = 0, v4 = 0, v5 = 0;
            if (l < 27) {
                const long long o = pidx(g, wrapi(f0x - 1 + l % 3, g.nx),
                                         wrapi(f0y - 1 + (l / 3) % 3, g.ny),
                                         wrapi(f0z - 1 + l / 9, g.nz));
                v0 = a.E[0][o]; v1 = a.E[1][o]; v2 = a.E[2][o];
                v3 = T(0.5) * (a.B0[0][o] + a.B1[0][o]);
                v4 = T(0.5) * (a.B0[1][o] + a.B1[1][o]);
                v5 = T(0.5) * (a.B0[2][o] + a.B1[2][o]);
            }
            const Loc<T> nxl = loc(gx, f0x), nyl = loc(gy, f0y), nzl = loc(gz, f0z);
            const Loc<T> sxl = loc(gx - T(0.5), f0x), syl = loc(gy - T(0.5), f0y),
                         szl = loc(gz - T(0.5), f0z);
            Ex = interp27(v0, sxl, nyl, nzl);
            Ey = interp27(v1, nxl, syl, nzl);
            Ez = interp27(v2, nxl, nyl, szl);
            Bx = interp27(v3, nxl, syl, szl);
            By = interp27(v4, sxl, nyl, szl);
            Bz = interp27(v5, sxl, syl, nzl);
        } else if (live) {
            const Lin<T> nx_ = lin(gx, g.nx), ny_ = lin(gy, g.ny), nz_ = lin(gz, g.nz);
            const Lin<T> sx = lin(gx - T(0.5), g.nx), sy = lin(gy - T(0.5), g.ny),
                         sz = lin(gz - T(0.5), g.nz);
            Ex = gather(a.E[0], g, sx, ny_, nz_);
            Ey = gather(a.E[1], g, nx_, sy, nz_);
            Ez = gather(a.E[2], g, nx_, ny_, sz);
            Bx = gather_mean(a.B0[0], a.B1[0], g, nx_, sy, sz);
            By = gather_mean(a.B0[1], a.B1[1], g, sx, ny_, sz);
            Bz = gather_mean(a.B0[2], a.B1[2], g, sx, sy, nz_);
        }
        Win<T> wx, wy, wz;
        if (live) {
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
            wx = window(gx, x1 * a.inv_dx[0], g.nx);
            wy = window(gy, y1 * a.inv_dx[1], g.ny);
            wz = window(gz, z1 * a.inv_dx[2], g.nz);
            // ---- new state, positions wrapped into [0, L)
            T xw = x1, yw = y1, zw = z1;
            if (xw < T(0)) xw += a.L[0]; else if (xw >= a.L[0]) xw -= a.L[0];
            if (yw < T(0)) yw += a.L[1]; else if (yw >= a.L[1]) yw -= a.L[1];
            if (zw < T(0)) zw += a.L[2]; else if (zw >= a.L[2]) zw -= a.L[2];
            a.x[0][p] = xw; a.x[1][p] = yw; a.x[2][p] = zw;
            a.u[0][p] = u1x; a.u[1][p] = u1y; a.u[2][p] = u1z;
        } else {
#pragma unroll
            for (int m = 0; m < 4; ++m) {
                wx.idx[m] = wy.idx[m] = wz.idx[m] = 0;
                wx.dS[m] = wy.dS[m] = wz.dS[m] = T(0);
            }
            wx.s1 = wx.s2 = wy.s1 = wy.s2 = wz.s1 = wz.s2 = T(0);
        }
        // ---- Esirkepov current: -dt J^{n+1/2} into E^{n+1} (the windows start at the old
        // node - 1, so a uniform warp shares them)
        if (uni || live) deposit(sink, wx, wy, wz, a.escale, uni);   // uni: the whole warp
    }
}

// ghost cells of the padded layout (periodic images of owned cells), per plane: the PY rows
// below and above the owned rows (whole padded rows) and the PX columns left and right of
// every owned row.  Each thread copies one ghost cell of each of the three arrays from its
// owned image.
template <typename T>
__global__ void __launch_bounds__(THREADS)
refresh_kernel(Geom g, T* __restrict__ F0, T* __restrict__ F1, T* __restrict__ F2) {
    const long long rows_cells = 2LL * PY * g.nxp;        // ghost rows of one plane
    const long long per_plane = rows_cells + 2LL * PX * g.ny;
    const long long total = per_plane * g.nz;
    for (long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x; t < total;
         t += (long long)gridDim.x * blockDim.x) {
        const int k = (int)(t / per_plane);
        const long long r = t - (long long)k * per_plane;
        int ip, jp;
        if (r < rows_cells) {
            const int row = (int)(r / g.nxp);
            ip = (int)(r - (long long)row * g.nxp);
            jp = row < PY ? row : g.ny + row;   // rows 0 .. PY-1 and ny+PY .. ny+2PY-1
        } else {
            const int q = (int)(r - rows_cells);
            const int row = q / (2 * PX), col = q - row * (2 * PX);
            jp = PY + row;
            ip = col < PX ? col : g.nx + col;   // columns 0 .. PX-1 and nx+PX .. nx+2PX-1
        }
        const int i = wrapi(ip - PX, g.nx), j = wrapi(jp - PY, g.ny);
        const long long dst = ((long long)k * g.nyp + jp) * g.nxp + ip;
        const long long src = pidx(g, i, j, k);
        F0[dst] = F0[src];
        F1[dst] = F1[src];
        F2[dst] = F2[src];
    }
}

template <typename T>
__global__ void __launch_bounds__(THREADS)
rho_kernel(Geom g, const T* __restrict__ x0, const T* __restrict__ x1, const T* __restrict__ x2,
           long long n, T ix, T iy, T iz, T Lx, T Ly, T Lz, T scale, T* __restrict__ rho, int* err) {
    for (long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x; p < n;
         p += (long long)gridDim.x * blockDim.x) {
        T x = x0[p], y = x1[p], z = x2[p];
        if (!finite3(x, y, z)) {
            atomicOr(err, ERR_PARTICLE);
            continue;
        }
        x = into_box(x, Lx); y = into_box(y, Ly); z = into_box(z, Lz);
        const Lin<T> a = lin(x * ix, g.nx), b = lin(y * iy, g.ny), c = lin(z * iz, g.nz);
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
void launch_refresh_images(const Geom& g, T* F0, T* F1, T* F2, cudaStream_t st) {
    const long long total = (2LL * PY * g.nxp + 2LL * PX * g.ny) * g.nz;
    picd::refresh_kernel<T><<<picd::blocks_for(total), picd::THREADS, 0, st>>>(g, F0, F1, F2);
}

template <typename T>
void launch_deposit_rho(const Geom& g, const T* const x[3], long long n, const T inv_dx[3],
                        const T L[3], T scale, T* rho, int* err, cudaStream_t st) {
    if (n <= 0) return;
    picd::rho_kernel<T><<<picd::blocks_for(n), picd::THREADS, 0, st>>>(
        g, x[0], x[1], x[2], n, inv_dx[0], inv_dx[1], inv_dx[2], L[0], L[1], L[2], scale, rho, err);
}

template void launch_pic_push<float>(const PushArgs<float>&, cudaStream_t);
template void launch_pic_push<double>(const PushArgs<double>&, cudaStream_t);
template void launch_refresh_images<float>(const Geom&, float*, float*, float*, cudaStream_t);
template void launch_refresh_images<double>(const Geom&, double*, double*, double*, cudaStream_t);
template void launch_deposit_rho<float>(const Geom&, const float* const[3], long long,
                                        const float[3], const float[3], float, float*, int*,
                                        cudaStream_t);
template void launch_deposit_rho<double>(const Geom&, const double* const[3], long long,
                                         const double[3], const double[3], double, double*, int*,
                                         cudaStream_t);

}  // namespace fdtd
