// Declarations of the macro-particle coupling (one PIC cycle per leapfrog step).
#pragma once

#include "fdtd_internal.cuh"

namespace fdtd {

// Faraday half step out of place: out.B = in.B + dt (-D* x in.E) (Eq. D*), images included,
// times the absorbing-layer factor sponge_y[j] sponge_z[k] when the sponge is non-NULL.
// Only the B arrays of `out` are written.
template <typename T>
void launch_faraday_oop(const Geom& g, const Mult<T>& m, FieldSet<T> in, FieldSet<T> out,
                        const T* sponge_y, const T* sponge_z, cudaStream_t st);

// Ampere step with a current on the grid: out.E = in.E + dt (D x Bh - J) (Yee stencil), with
// Bh = the B arrays of `bset` and J three padded arrays at the E positions (J NULL: no
// current); images included; sponge as for the Faraday half.
template <typename T>
void launch_ampere_current(const Geom& g, const Mult<T>& m, FieldSet<T> in, FieldSet<T> bset,
                           const T* const J[3], FieldSet<T> out, const T* sponge_y,
                           const T* sponge_z, int* err, cudaStream_t st);

// Per-particle gather (E^n, B^n = (B0 + B1) / 2), Boris push, move, and Esirkepov's current as
// -dt J^{n+1/2} added into the owned cells of Eout (E^{n+1} without the current, padded; times
// the absorbing-layer factor when spy is non-NULL); launch_refresh_images then brings its
// ghosts up to date.  Positions outside the box are wrapped first.
// Particles whose position or momentum is not finite are left unchanged and raise bit 2 of
// *err.
template <typename T>
struct PushArgs {
    Geom g;
    const T* E[3];
    const T* B0[3];
    const T* B1[3];
    T* Eout[3];
    const T* spy;
    const T* spz;
    T* x[3];
    T* u[3];
    long long n;
    T inv_dx[3];
    T L[3];
    T h;           // (q/m) dt / 2
    T dt;
    T escale[3];   // q / (dx_b dx_c): the cumulative shape change of axis a times this is -dt J_a
    int* err;
};
template <typename T>
void launch_pic_push(const PushArgs<T>& a, cudaStream_t st);

// Copy every owned cell that has periodic images (the ghosts of the padded layout) to them,
// for three padded arrays.
template <typename T>
void launch_refresh_images(const Geom& g, T* F0, T* F1, T* F2, cudaStream_t st);

// rho at the nodes (first-order shape) added into a dense [nz][ny][nx] array; positions outside
// the box [0, L) are wrapped first, non-finite ones raise bit 2 of *err and add nothing.
template <typename T>
void launch_deposit_rho(const Geom& g, const T* const x[3], long long n, const T inv_dx[3],
                        const T L[3], T scale, T* rho, int* err, cudaStream_t st);

}  // namespace fdtd
