// Internal declarations shared by the libfdtd translation units.
//
// State layout in HBM.  Every field array is stored padded in x and y and
// unpadded in z:
//     element (i, j, k), 0 <= i < nx, 0 <= j < ny, 0 <= k < nz, lives at
//     base[(k * nyp + (j + PY)) * nxp + (i + PX)],  nxp = nx + 2 PX, nyp = ny + 2 PY.
// The PX x-columns and PY y-rows on each side hold periodic images of the
// owned cells (ghosts).  Every kernel that writes an owned cell also writes
// its images, so a tile load never wraps in x or y; z neighbours wrap by
// plane index.  PX = 4 keeps every x-row 16-byte aligned (TMA boxes start on
// a 16-byte boundary) and covers the widest x reach of the step
// (E at i-2 .. i+2 and B at i-1); PY = 2 covers y reaches -2 .. +2.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/fdtd.h"

namespace fdtd {

constexpr int PX = 4;
constexpr int PY = 2;

struct Geom {
    int nx, ny, nz;
    int nxp, nyp;
    long long plane;   // nxp * nyp elements
    long long total;   // plane * nz elements (one padded array)
};

inline Geom make_geom(int nx, int ny, int nz) {
    Geom g;
    g.nx = nx; g.ny = ny; g.nz = nz;
    g.nxp = nx + 2 * PX;
    g.nyp = ny + 2 * PY;
    g.plane = (long long)g.nxp * g.nyp;
    g.total = g.plane * nz;
    return g;
}

__host__ __device__ inline long long pidx(const Geom& g, int i, int j, int k) {
    return ((long long)k * g.nyp + (j + PY)) * g.nxp + (i + PX);
}

// Update multipliers, computed in FP64 on the host and rounded once to T:
//   cA[a] = dt alpha_a / dx_a, cD[a] = dt delta_a / dx_a, cB[a][b] = dt beta_ab / dx_a,
//   cE[a] = dt / dx_a (c^2 dt / dx_a with c = 1).
template <typename T>
struct Mult {
    T cA[3], cD[3], cB[3][3], cE[3];
    T dt;
};

// D*_a F times dt (Eq. D*), from its 12 tap values, in one fixed rounding order shared by
// every kernel (so all step kernels give bitwise-identical B):
//   cA (F[+a] - F[0]) + cD (F[+2a] - F[-a]) + cBb ((F[+a+b] - F[+b]) + (F[+a-b] - F[-b]))
//                                          + cBc ((F[+a+c] - F[+c]) + (F[+a-c] - F[-c]))
// dstar_diff takes the five differences along a already formed (d_a = F[+a] - F[0],
// d_bp = F[+a+b] - F[+b], ...), so a kernel can form each difference once and share it between
// neighbouring cells; dstar_taps forms them from the 12 tap values.  Both round identically.
template <typename T>
__device__ __forceinline__ T dstar_diff(T d_a, T f_a2, T f_am1, T d_bp, T d_bm, T d_cp, T d_cm,
                                        T cA, T cD, T cBb, T cBc) {
    T v = cA * d_a;
    v = fma(cD, f_a2 - f_am1, v);
    v = fma(cBb, d_bp + d_bm, v);
    v = fma(cBc, d_cp + d_cm, v);
    return v;
}

template <typename T>
__device__ __forceinline__ T dstar_taps(T f_a1, T f_0, T f_a2, T f_am1, T f_a1bp, T f_bp, T f_a1bm,
                                        T f_bm, T f_a1cp, T f_cp, T f_a1cm, T f_cm, T cA, T cD,
                                        T cBb, T cBc) {
    return dstar_diff(f_a1 - f_0, f_a2, f_am1, f_a1bp - f_bp, f_a1bm - f_bm, f_a1cp - f_cp,
                      f_a1cm - f_cm, cA, cD, cBb, cBc);
}

// One Ampere component: E + (c1 (P - P[-a1]) - c2 (Q - Q[-a2])), in a fixed rounding order.
template <typename T>
__device__ __forceinline__ T ampere_comp(T e, T p0, T pm, T q0, T qm, T c1, T c2) {
    const T t = c2 * (q0 - qm);
    return e + fma(c1, p0 - pm, -t);
}

// Non-finite detection folded into the E update: acc accumulates v * 0, which is 0 for every
// finite v and NaN once an infinite or NaN v passes, so one comparison after the march tells
// whether any E value a thread wrote was not finite.  A non-finite B^{n+1/2} always reaches
// E^{n+1} of the same step (every D x B term has a non-zero multiplier), so checking E covers
// both fields.  Error-flag bits of the handle: 1 = a bounded wait expired, 2 = a particle was
// not finite, 4 = a field value was not finite.
constexpr int ERR_WAIT = 1, ERR_PARTICLE = 2, ERR_FIELD = 4;

template <typename T>
__device__ __forceinline__ T nonfinite_acc(T acc, T v) {
    return fma(v, T(0), acc);
}

template <typename T>
struct FieldSet {
    T* c[6];   // Ex, Ey, Ez, Bx, By, Bz (padded)
};

// ---- kernels launched from the host translation unit ----------------------

template <typename T>
void launch_faraday_v0(const Geom& g, const Mult<T>& m, FieldSet<T> s, const T* sponge_y,
                       const T* sponge_z, cudaStream_t st);
template <typename T>
void launch_ampere_v0(const Geom& g, const Mult<T>& m, FieldSet<T> s, const T* sponge_y,
                      const T* sponge_z, const T* jyz, const T* jx_row, int* err, cudaStream_t st);

// Fused leapfrog step: reads (E^n, B^{n-1/2}) from state set `in_set`, writes
// (E^{n+1}, B^{n+1/2}) to `out` (padded, images included).  hist_E (entries
// nullable) receives E^{n+1}.  The plan holds the TMA descriptors of both sets.
struct FusedPlan;
template <typename T>
bool fused_supported(const Geom& g);
template <typename T>
FusedPlan* fused_plan_create(const Geom& g, T* const set0[6], T* const set1[6]);
void fused_plan_destroy(FusedPlan* p);
template <typename T>
void launch_step_fused(const FusedPlan* plan, int in_set, const Geom& g, const Mult<T>& m,
                       FieldSet<T> in, FieldSet<T> out, const T* sponge_y, const T* sponge_z,
                       const T* jyz, const T* jx_row, T* hist_E[3], int* err, cudaStream_t st);

// FP32 fused step on the planes zs .. ze-1 only (no current, no history)
void launch_step_fused32_range(const FusedPlan* plan, int in_set, const Geom& g,
                               const Mult<float>& m, FieldSet<float> in, FieldSet<float> out,
                               const float* sponge_y, const float* sponge_z, int zs, int ze,
                               int* err, cudaStream_t st);
// Drop the planes p0 .. p1-1 of six padded arrays from L2 without writing them back (whole
// 128-byte lines inside the range only); their contents become undefined.
void launch_discard_planes(const Geom& g, size_t esz, void* const arr[6], int p0, int p1,
                           cudaStream_t st);

template <typename T>
void launch_adjoint_B_v0(const Geom& g, const Mult<T>& m, FieldSet<T> lam, const T* E_hist[3],
                         const T* sponge_y, const T* sponge_z, double* partials, int nblk,
                         cudaStream_t st);
template <typename T>
void launch_adjoint_E_v0(const Geom& g, const Mult<T>& m, FieldSet<T> lam, const T* sponge_y,
                         const T* sponge_z, cudaStream_t st);
int adjoint_B_blocks(const Geom& g);

template <typename T>
void launch_probe_loss(const Geom& g, const T* E, int x_index, const T* target, double* loss,
                       cudaStream_t st);
template <typename T>
void launch_probe_adjoint(const Geom& g, T* lamE, const T* E, int x_index, const T* target,
                          cudaStream_t st);
template <typename T>
void launch_pack(const Geom& g, const T* padded, T* dense, cudaStream_t st);
template <typename T>
void launch_unpack(const Geom& g, const T* dense, T* padded, cudaStream_t st);
// the periodic images (ghost cells) of a padded array from its owned cells
template <typename T>
void launch_fill_ghosts(const Geom& g, T* padded, cudaStream_t st);

// grad12[beta 3x3 row-major, delta 3] += s[q] * sum over blocks of partial q, where partial
// q = 3a + w is (axis a; w = 0: delta_a, 1 / 2: beta of the first / second other axis).
struct GradScale {
    double s[9];
};
void launch_reduce_grad(const double* part, int nblocks, GradScale sc, double* grad12,
                        cudaStream_t st);

// Resident CTAs of `kernel` on the whole device (SMs x CTAs per SM; 0 if unknown), and the
// z-chunk length in [tz_min, tz_max] of a tiled plane-marching kernel with `tiles_xy` CTAs per
// z-chunk that fills whole waves of `slots` CTAs best.
int resident_slots(const void* kernel, int threads, size_t smem);
// the same for a kernel that allocates tmem_cols TMEM columns per CTA (the occupancy API
// under-reports those)
int resident_slots_tmem(const void* kernel, int threads, size_t smem, int tmem_cols);
int zchunk_len(int tiles_xy, int nz, int slots, int tz_min, int tz_max);

// thread-local error message
void set_error(const char* fmt, ...);

}  // namespace fdtd
