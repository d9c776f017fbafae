// Reference-form leapfrog kernels (one thread per cell, in place) and the
// small state-management kernels: pack/unpack between dense caller layout
// and the padded library layout, the rigid-bunch current table and the probe
// kernels.
//
// Faraday half step (App. A, update eqs. for B; Eq. D* for the stencil):
//   B_x += dt (D*_z E_y - D*_y E_z),  B_y += dt (D*_x E_z - D*_z E_x),
//   B_z += dt (D*_y E_x - D*_x E_y),
// with D*_a a forward-type 12-tap difference (E positions -> B positions):
//   D*_a F = [alpha_a (F[+a] - F[0]) + delta_a (F[+2a] - F[-a])
//             + sum_{b != a} beta_ab ((F[+a+b] - F[+b]) + (F[+a-b] - F[-b]))] / dx_a.
// Ampere step (Yee stencil, backward differences B positions -> E positions):
//   E_x += dt (D_y B_z - D_z B_y - J_x), and cyclically.
#include <cmath>

#include "fdtd_internal.cuh"
#include "pic.cuh"

namespace fdtd {

__device__ __forceinline__ long long zoff(const Geom& g, int k, int dz) {
    int kk = (k + dz) % g.nz;
    if (kk < 0) kk += g.nz;
    return (long long)(kk - k) * g.plane;
}

// D*_a F (already multiplied by dt) at padded index c.
//   a1/a2/am1: offsets of +a, +2a, -a;  bp/bm, cp/cm: offsets of +-b and +-c.
template <typename T>
__device__ __forceinline__ T dstar_at(const T* __restrict__ F, long long c, long long a1,
                                      long long a2, long long am1, long long bp, long long bm,
                                      long long cp, long long cm, T cA, T cD, T cBb, T cBc) {
    return dstar_taps(F[c + a1], F[c], F[c + a2], F[c + am1], F[c + a1 + bp], F[c + bp],
                      F[c + a1 + bm], F[c + bm], F[c + a1 + cp], F[c + cp], F[c + a1 + cm],
                      F[c + cm], cA, cD, cBb, cBc);
}

template <typename T>
__device__ __forceinline__ void store_images(const Geom& g, T* F, int i, int j, int k, T v) {
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

template <typename T>
__global__ void faraday_v0_kernel(Geom g, Mult<T> m, FieldSet<T> s, const T* __restrict__ spy,
                                  const T* __restrict__ spz) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= g.nx) return;
    for (int k = blockIdx.z; k < g.nz; k += gridDim.z)
        for (int j = blockIdx.y; j < g.ny; j += gridDim.y) {
            const long long c = pidx(g, i, j, k);
            const long long Y = g.nxp;
            const long long zp1 = zoff(g, k, 1), zm1 = zoff(g, k, -1), zp2 = zoff(g, k, 2);
            const T* Ex = s.c[0];
            const T* Ey = s.c[1];
            const T* Ez = s.c[2];
            // D*_x: axis x, transverse y then z;  D*_y: axis y, transverse x then z;  D*_z: axis z.
#define DSX(F) dstar_at(F, c, 1, 2, -1, Y, -Y, zp1, zm1, m.cA[0], m.cD[0], m.cB[0][1], m.cB[0][2])
#define DSY(F) dstar_at(F, c, Y, 2 * Y, -Y, 1, -1, zp1, zm1, m.cA[1], m.cD[1], m.cB[1][0], m.cB[1][2])
#define DSZ(F) dstar_at(F, c, zp1, zp2, zm1, 1, -1, Y, -Y, m.cA[2], m.cD[2], m.cB[2][0], m.cB[2][1])
            T bx = s.c[3][c] + (DSZ(Ey) - DSY(Ez));
            T by = s.c[4][c] + (DSX(Ez) - DSZ(Ex));
            T bz = s.c[5][c] + (DSY(Ex) - DSX(Ey));
#undef DSX
#undef DSY
#undef DSZ
            if (spy != nullptr) {
                const T f = spy[j] * spz[k];
                bx *= f; by *= f; bz *= f;
            }
            store_images(g, s.c[3], i, j, k, bx);
            store_images(g, s.c[4], i, j, k, by);
            store_images(g, s.c[5], i, j, k, bz);
        }
}

template <typename T>
__global__ void ampere_v0_kernel(Geom g, Mult<T> m, FieldSet<T> s, const T* __restrict__ spy,
                                 const T* __restrict__ spz, const T* __restrict__ jyz,
                                 const T* __restrict__ jx_row, int* __restrict__ err) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= g.nx) return;
    T fin = T(0);   // non-finite detection (nonfinite_acc)
    for (int k = blockIdx.z; k < g.nz; k += gridDim.z)
        for (int j = blockIdx.y; j < g.ny; j += gridDim.y) {
            const long long c = pidx(g, i, j, k);
            const long long Y = g.nxp;
            const long long zm1 = zoff(g, k, -1);
            const T* Bx = s.c[3];
            const T* By = s.c[4];
            const T* Bz = s.c[5];
            T ex = ampere_comp(s.c[0][c], Bz[c], Bz[c - Y], By[c], By[c + zm1], m.cE[1], m.cE[2]);
            T ey = ampere_comp(s.c[1][c], Bx[c], Bx[c + zm1], Bz[c], Bz[c - 1], m.cE[2], m.cE[0]);
            T ez = ampere_comp(s.c[2][c], By[c], By[c - 1], Bx[c], Bx[c - Y], m.cE[0], m.cE[1]);
            if (jx_row != nullptr) {
                // J_x^{n+1/2} at (i+1/2, j, k): x-profile x transverse profile, both tabulated.
                const T jx = (jx_row[i] * jyz[j]) * jyz[g.ny + k];
                ex = fma(-m.dt, jx, ex);
            }
            if (spy != nullptr) {
                const T f = spy[j] * spz[k];
                ex *= f; ey *= f; ez *= f;
            }
            fin = nonfinite_acc(nonfinite_acc(nonfinite_acc(fin, ex), ey), ez);
            store_images(g, s.c[0], i, j, k, ex);
            store_images(g, s.c[1], i, j, k, ey);
            store_images(g, s.c[2], i, j, k, ez);
        }
    if (!(fin == T(0))) atomicOr(err, ERR_FIELD);
}

template <typename T>
void launch_faraday_v0(const Geom& g, const Mult<T>& m, FieldSet<T> s, const T* sponge_y,
                       const T* sponge_z, cudaStream_t st) {
    dim3 blk(128), grd((g.nx + 127) / 128, (unsigned)(g.ny < 65535 ? g.ny : 65535),
                        (unsigned)(g.nz < 65535 ? g.nz : 65535));   // j, k loop in the kernel
    faraday_v0_kernel<T><<<grd, blk, 0, st>>>(g, m, s, sponge_y, sponge_z);
}

template <typename T>
void launch_ampere_v0(const Geom& g, const Mult<T>& m, FieldSet<T> s, const T* sponge_y,
                      const T* sponge_z, const T* jyz, const T* jx_row, int* err, cudaStream_t st) {
    dim3 blk(128), grd((g.nx + 127) / 128, (unsigned)(g.ny < 65535 ? g.ny : 65535),
                        (unsigned)(g.nz < 65535 ? g.nz : 65535));   // j, k loop in the kernel
    ampere_v0_kernel<T><<<grd, blk, 0, st>>>(g, m, s, sponge_y, sponge_z, jyz, jx_row, err);
}

// ---------------------------------------------------------------------------
// PIC cycle field halves (one thread per cell, out of place so that the particle push sees
// both B^{n-1/2} and B^{n+1/2}; the current J^{n+1/2} is three padded arrays at the E
// positions, App. A numerical continuity equation)
// ---------------------------------------------------------------------------

template <typename T>
__global__ void faraday_oop_kernel(Geom g, Mult<T> m, FieldSet<T> in, FieldSet<T> out,
                                   const T* __restrict__ spy, const T* __restrict__ spz) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= g.nx) return;
    for (int k = blockIdx.z; k < g.nz; k += gridDim.z)
        for (int j = blockIdx.y; j < g.ny; j += gridDim.y) {
            const long long c = pidx(g, i, j, k);
            const long long Y = g.nxp;
            const long long zp1 = zoff(g, k, 1), zm1 = zoff(g, k, -1), zp2 = zoff(g, k, 2);
            const T* Ex = in.c[0];
            const T* Ey = in.c[1];
            const T* Ez = in.c[2];
#define DSX(F) dstar_at(F, c, 1, 2, -1, Y, -Y, zp1, zm1, m.cA[0], m.cD[0], m.cB[0][1], m.cB[0][2])
#define DSY(F) dstar_at(F, c, Y, 2 * Y, -Y, 1, -1, zp1, zm1, m.cA[1], m.cD[1], m.cB[1][0], m.cB[1][2])
#define DSZ(F) dstar_at(F, c, zp1, zp2, zm1, 1, -1, Y, -Y, m.cA[2], m.cD[2], m.cB[2][0], m.cB[2][1])
            T bx = in.c[3][c] + (DSZ(Ey) - DSY(Ez));
            T by = in.c[4][c] + (DSX(Ez) - DSZ(Ex));
            T bz = in.c[5][c] + (DSY(Ex) - DSX(Ey));
#undef DSX
#undef DSY
#undef DSZ
            if (spy != nullptr) {
                const T f = spy[j] * spz[k];
                bx *= f; by *= f; bz *= f;
            }
            store_images(g, out.c[3], i, j, k, bx);
            store_images(g, out.c[4], i, j, k, by);
            store_images(g, out.c[5], i, j, k, bz);
        }
}

template <typename T>
__global__ void ampere_current_kernel(Geom g, Mult<T> m, FieldSet<T> in, FieldSet<T> bset,
                                      const T* __restrict__ Jx, const T* __restrict__ Jy,
                                      const T* __restrict__ Jz, FieldSet<T> out,
                                      const T* __restrict__ spy, const T* __restrict__ spz,
                                      int* __restrict__ err) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= g.nx) return;
    T fin = T(0);   // non-finite detection (nonfinite_acc)
    for (int k = blockIdx.z; k < g.nz; k += gridDim.z)
        for (int j = blockIdx.y; j < g.ny; j += gridDim.y) {
            const long long c = pidx(g, i, j, k);
            const long long Y = g.nxp;
            const long long zm1 = zoff(g, k, -1);
            const T* Bx = bset.c[3];
            const T* By = bset.c[4];
            const T* Bz = bset.c[5];
            T ex = ampere_comp(in.c[0][c], Bz[c], Bz[c - Y], By[c], By[c + zm1], m.cE[1], m.cE[2]);
            T ey = ampere_comp(in.c[1][c], Bx[c], Bx[c + zm1], Bz[c], Bz[c - 1], m.cE[2], m.cE[0]);
            T ez = ampere_comp(in.c[2][c], By[c], By[c - 1], Bx[c], Bx[c - Y], m.cE[0], m.cE[1]);
            if (Jx != nullptr) {
                ex = fma(-m.dt, Jx[c], ex);
                ey = fma(-m.dt, Jy[c], ey);
                ez = fma(-m.dt, Jz[c], ez);
            }
            if (spy != nullptr) {
                const T f = spy[j] * spz[k];
                ex *= f; ey *= f; ez *= f;
            }
            fin = nonfinite_acc(nonfinite_acc(nonfinite_acc(fin, ex), ey), ez);
            store_images(g, out.c[0], i, j, k, ex);
            store_images(g, out.c[1], i, j, k, ey);
            store_images(g, out.c[2], i, j, k, ez);
        }
    if (!(fin == T(0))) atomicOr(err, ERR_FIELD);
}

template <typename T>
void launch_faraday_oop(const Geom& g, const Mult<T>& m, FieldSet<T> in, FieldSet<T> out,
                        const T* sponge_y, const T* sponge_z, cudaStream_t st) {
    dim3 blk(128), grd((g.nx + 127) / 128, (unsigned)(g.ny < 65535 ? g.ny : 65535),
                        (unsigned)(g.nz < 65535 ? g.nz : 65535));   // j, k loop in the kernel
    faraday_oop_kernel<T><<<grd, blk, 0, st>>>(g, m, in, out, sponge_y, sponge_z);
}

template <typename T>
void launch_ampere_current(const Geom& g, const Mult<T>& m, FieldSet<T> in, FieldSet<T> bset,
                           const T* const J[3], FieldSet<T> out, const T* sponge_y,
                           const T* sponge_z, int* err, cudaStream_t st) {
    dim3 blk(128), grd((g.nx + 127) / 128, (unsigned)(g.ny < 65535 ? g.ny : 65535),
                        (unsigned)(g.nz < 65535 ? g.nz : 65535));   // j, k loop in the kernel
    const T* Jx = J ? J[0] : nullptr;
    const T* Jy = J ? J[1] : nullptr;
    const T* Jz = J ? J[2] : nullptr;
    ampere_current_kernel<T><<<grd, blk, 0, st>>>(g, m, in, bset, Jx, Jy, Jz, out, sponge_y,
                                                  sponge_z, err);
}

template void launch_faraday_oop<float>(const Geom&, const Mult<float>&, FieldSet<float>,
                                        FieldSet<float>, const float*, const float*,
                                        cudaStream_t);
template void launch_faraday_oop<double>(const Geom&, const Mult<double>&, FieldSet<double>,
                                         FieldSet<double>, const double*, const double*,
                                         cudaStream_t);
template void launch_ampere_current<float>(const Geom&, const Mult<float>&, FieldSet<float>,
                                           FieldSet<float>, const float* const[3],
                                           FieldSet<float>, const float*, const float*,
                                           int*, cudaStream_t);
template void launch_ampere_current<double>(const Geom&, const Mult<double>&, FieldSet<double>,
                                            FieldSet<double>, const double* const[3],
                                            FieldSet<double>, const double*, const double*,
                                            int*, cudaStream_t);

// E += -dt J (times the absorbing-layer factor) at the owned cells, J dense [nz][ny][nx] at the E
// positions (NULL components skipped); the caller refreshes the images afterwards.
template <typename T>
__global__ void current_kernel(Geom g, T* __restrict__ E0, T* __restrict__ E1, T* __restrict__ E2,
                               const T* __restrict__ J0, const T* __restrict__ J1,
                               const T* __restrict__ J2, T mdt, const T* __restrict__ spy,
                               const T* __restrict__ spz) {
    const long long n = (long long)g.nx * g.ny * g.nz;
    for (long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x; t < n;
         t += (long long)gridDim.x * blockDim.x) {
        const int i = (int)(t % g.nx);
        const long long r = t / g.nx;
        const int j = (int)(r % g.ny);
        const int k = (int)(r / g.ny);
        const T f = spy != nullptr ? spy[j] * spz[k] : T(1);
        const long long c = pidx(g, i, j, k);
        if (J0 != nullptr) E0[c] += (mdt * J0[t]) * f;
        if (J1 != nullptr) E1[c] += (mdt * J1[t]) * f;
        if (J2 != nullptr) E2[c] += (mdt * J2[t]) * f;
    }
}

template <typename T>
void launch_current(const Geom& g, T* const E[3], const T* const J[3], T dt, const T* sponge_y,
                    const T* sponge_z, cudaStream_t st) {
    const long long n = (long long)g.nx * g.ny * g.nz;
    long long b = (n + 255) / 256;
    if (b > 152LL * 32) b = 152LL * 32;
    current_kernel<T><<<(unsigned)b, 256, 0, st>>>(g, E[0], E[1], E[2], J[0], J[1], J[2], -dt,
                                                  sponge_y, sponge_z);
}
template void launch_current<float>(const Geom&, float* const[3], const float* const[3], float,
                                    const float*, const float*, cudaStream_t);
template void launch_current<double>(const Geom&, double* const[3], const double* const[3], double,
                                     const double*, const double*, cudaStream_t);

template void launch_faraday_v0<float>(const Geom&, const Mult<float>&, FieldSet<float>,
                                       const float*, const float*, cudaStream_t);
template void launch_faraday_v0<double>(const Geom&, const Mult<double>&, FieldSet<double>,
                                        const double*, const double*, cudaStream_t);
template void launch_ampere_v0<float>(const Geom&, const Mult<float>&, FieldSet<float>,
                                      const float*, const float*, const float*, const float*,
                                      int*, cudaStream_t);
template void launch_ampere_v0<double>(const Geom&, const Mult<double>&, FieldSet<double>,
                                       const double*, const double*, const double*,
                                       const double*, int*, cudaStream_t);

// ---------------------------------------------------------------------------
// rigid bunch: x-profile table for n consecutive steps
//   X_m(i) = [Phi(d/s) - Phi((d - v dt)/s)] * q / (dy dz dt),  d = wrap(x_{i+1/2} - x_c^{n0+m}),
// so that J_x = X_m(i) g_y(j) g_z(k) with g the cell-integrated transverse Gaussians.
// ---------------------------------------------------------------------------

__device__ double phi_diff(double a, double b) {
    // Phi(a) - Phi(b) without cancellation in either tail.
    const double r = 0.70710678118654752440;
    if (a > 0.0 && b > 0.0) return 0.5 * (erfc(b * r) - erfc(a * r));
    if (a < 0.0 && b < 0.0) return 0.5 * (erfc(-a * r) - erfc(-b * r));
    return 0.5 * (erf(a * r) - erf(b * r));
}

template <typename T>
__global__ void bunch_table_kernel(int nx, int n, double x0, double vdt, double inv_sig,
                                   double scale, double dx, double Lx, long long step0, T* out) {
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= (long long)n * nx) return;
    const int m = (int)(t / nx), i = (int)(t % nx);
    const double xc = x0 + vdt * (double)(step0 + m);
    const double xf = (i + 0.5) * dx;
    double d = xf - xc;
    d = d - Lx * floor(d / Lx + 0.5);   // minimum image in [-Lx/2, Lx/2)
    out[t] = (T)(scale * phi_diff(d * inv_sig, (d - vdt) * inv_sig));
}

template <typename T>
void launch_bunch_table(int nx, int n, double x0, double vdt, double inv_sig, double scale,
                        double dx, double Lx, long long step0, T* out, cudaStream_t st) {
    const long long tot = (long long)n * nx;
    bunch_table_kernel<T><<<(unsigned)((tot + 255) / 256), 256, 0, st>>>(
        nx, n, x0, vdt, inv_sig, scale, dx, Lx, step0, out);
}
template void launch_bunch_table<float>(int, int, double, double, double, double, double, double,
                                        long long, float*, cudaStream_t);
template void launch_bunch_table<double>(int, int, double, double, double, double, double,
                                         double, long long, double*, cudaStream_t);

// ---------------------------------------------------------------------------
// layout conversion
// ---------------------------------------------------------------------------

template <typename T>
__global__ void unpack_kernel(Geom g, const T* __restrict__ dense, T* __restrict__ padded) {
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= g.total) return;
    const int ip = (int)(t % g.nxp);
    const long long r = t / g.nxp;
    const int jp = (int)(r % g.nyp);
    const int k = (int)(r / g.nyp);
    int i = (ip - PX) % g.nx;
    if (i < 0) i += g.nx;
    int j = (jp - PY) % g.ny;
    if (j < 0) j += g.ny;
    padded[t] = dense == nullptr ? T(0) : dense[((long long)k * g.ny + j) * g.nx + i];
}

template <typename T>
__global__ void pack_kernel(Geom g, const T* __restrict__ padded, T* __restrict__ dense) {
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const long long n = (long long)g.nx * g.ny * g.nz;
    if (t >= n) return;
    const int i = (int)(t % g.nx);
    const long long r = t / g.nx;
    const int j = (int)(r % g.ny);
    const int k = (int)(r / g.ny);
    dense[t] = padded[pidx(g, i, j, k)];
}

template <typename T>
void launch_unpack(const Geom& g, const T* dense, T* padded, cudaStream_t st) {
    unpack_kernel<T><<<(unsigned)((g.total + 255) / 256), 256, 0, st>>>(g, dense, padded);
}
template <typename T>
void launch_pack(const Geom& g, const T* padded, T* dense, cudaStream_t st) {
    const long long n = (long long)g.nx * g.ny * g.nz;
    pack_kernel<T><<<(unsigned)((n + 255) / 256), 256, 0, st>>>(g, padded, dense);
}
// Periodic images only: every ghost cell of the padded array (rows 0 .. PY-1 and
// ny+PY .. nyp-1, columns 0 .. PX-1 and nx+PX .. nxp-1 of the owned rows) takes the value of the
// owned cell it is the image of.  After a host transfer has written the owned cells directly.
template <typename T>
__global__ void ghosts_kernel(Geom g, T* __restrict__ F) {
    const long long per = 2LL * PY * g.nxp + 2LL * PX * g.ny;   // ghost cells per plane
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= per * g.nz) return;
    const int k = (int)(t / per);
    int r = (int)(t - (long long)k * per);
    int ip, jp;
    const int rows = 2 * PY * g.nxp;
    if (r < rows) {   // ghost rows
        const int row = r / g.nxp;
        ip = r - row * g.nxp;
        jp = row < PY ? row : g.ny + row;
    } else {          // ghost columns of the owned rows
        r -= rows;
        const int jo = r / (2 * PX);
        const int c = r - jo * 2 * PX;
        jp = jo + PY;
        ip = c < PX ? c : g.nx + c;
    }
    int i = (ip - PX) % g.nx;
    if (i < 0) i += g.nx;
    int j = (jp - PY) % g.ny;
    if (j < 0) j += g.ny;
    const long long base = (long long)k * g.plane;
    F[base + (long long)jp * g.nxp + ip] = F[base + (long long)(j + PY) * g.nxp + (i + PX)];
}

template <typename T>
void launch_fill_ghosts(const Geom& g, T* padded, cudaStream_t st) {
    const long long n = (2LL * PY * g.nxp + 2LL * PX * g.ny) * g.nz;
    ghosts_kernel<T><<<(unsigned)((n + 255) / 256), 256, 0, st>>>(g, padded);
}
template void launch_fill_ghosts<float>(const Geom&, float*, cudaStream_t);
template void launch_fill_ghosts<double>(const Geom&, double*, cudaStream_t);
template void launch_unpack<float>(const Geom&, const float*, float*, cudaStream_t);
template void launch_unpack<double>(const Geom&, const double*, double*, cudaStream_t);
template void launch_pack<float>(const Geom&, const float*, float*, cudaStream_t);
template void launch_pack<double>(const Geom&, const double*, double*, cudaStream_t);

// ---------------------------------------------------------------------------
// probe: loss += sum_{j,k} (F[x_p, j, k] - T[k][j])^2   (one block: fixed summation order)
// ---------------------------------------------------------------------------

template <typename T>
__global__ void probe_loss_kernel(Geom g, const T* __restrict__ F, int xp,
                                  const T* __restrict__ target, double* loss) {
    double acc = 0.0;
    const int n = g.ny * g.nz;
    for (int t = threadIdx.x; t < n; t += blockDim.x) {
        const int j = t % g.ny, k = t / g.ny;
        const double d = (double)F[pidx(g, xp, j, k)] - (double)target[(long long)k * g.ny + j];
        acc += d * d;
    }
    __shared__ double red[32];
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x < 32) {
        acc = threadIdx.x < (blockDim.x >> 5) ? red[threadIdx.x] : 0.0;
        for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
        if (threadIdx.x == 0) *loss += acc;
    }
}

// lambda_E[x_p, j, k] += 2 (F[x_p, j, k] - T[k][j]), written with its periodic images.
template <typename T>
__global__ void probe_adjoint_kernel(Geom g, T* __restrict__ lam, const T* __restrict__ F, int xp,
                                     const T* __restrict__ target) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= g.ny * g.nz) return;
    const int j = t % g.ny, k = t / g.ny;
    const long long c = pidx(g, xp, j, k);
    const T v = lam[c] + T(2) * (F[c] - target[(long long)k * g.ny + j]);
    store_images(g, lam, xp, j, k, v);
}

template <typename T>
void launch_probe_loss(const Geom& g, const T* E, int x_index, const T* target, double* loss,
                       cudaStream_t st) {
    probe_loss_kernel<T><<<1, 1024, 0, st>>>(g, E, x_index, target, loss);
}
template <typename T>
void launch_probe_adjoint(const Geom& g, T* lamE, const T* E, int x_index, const T* target,
                          cudaStream_t st) {
    const int n = g.ny * g.nz;
    probe_adjoint_kernel<T><<<(n + 255) / 256, 256, 0, st>>>(g, lamE, E, x_index, target);
}
template void launch_probe_loss<float>(const Geom&, const float*, int, const float*, double*,
                                       cudaStream_t);
template void launch_probe_loss<double>(const Geom&, const double*, int, const double*, double*,
                                        cudaStream_t);
template void launch_probe_adjoint<float>(const Geom&, float*, const float*, int, const float*,
                                          cudaStream_t);
template void launch_probe_adjoint<double>(const Geom&, double*, const double*, int,
                                           const double*, cudaStream_t);

}  // namespace fdtd
