// Dispersion norm (Sec. 4, Eq. norm) and its exact gradient over a midpoint k-grid.
//
// Per point k (k_i = (m_i + 1/2) pi / (N_i dx_i)):
//   s_i^2 = sin^2(k_i dx_i / 2) / dx_i^2,  c_i = cos(k_i dx_i)
//   S = sum_i s_i^2 A_i,  A_i = alpha_i + delta_i (1 + 2 c_i) + 2 sum_{j != i} beta_ij c_j
//                                                           (Eq. dispersion_relation)
//   omega = (2/dt) asin(dt sqrt S),  r = omega - |k|
//   f  += w r^2
//   df += w 2 r (d omega/d theta),  with d omega/dS = 1/(sqrt S sqrt(1 - dt^2 S)),
//         dS/d beta_ij = 2 s_i^2 (c_j - 1),  dS/d delta_i = 2 s_i^2 (c_i - 1),
//         d omega/d dt = -omega/dt + 2 sqrt S / (dt sqrt(1 - dt^2 S)).
// Everything per point and every accumulation is FP64.  Per-axis values
// (k_i, s_i^2, c_i) come from a small table built by the first kernel;
// the main kernel is a grid-stride loop with warp-shuffle block reduction
// into per-block partials; a one-block kernel sums the partials in a fixed
// order (deterministic result).
#include <cmath>

#include "fdtd_internal.cuh"

namespace fdtd {

constexpr int NQ = 11;   // f, dbeta x 6 (xy, xz, yx, yz, zx, zy), ddelta x 3, ddt
constexpr int NORM_THREADS = 256;

struct NormParams {
    double alpha[3], delta[3], beta[3][3];
    double dt;
    int N[3];
    int dims;
    int weight;
    double wparam;   // cone: cos(half-angle); gauss: dy / width
    long long npts;
    double pref;     // prod(dx) * prod(pi / (N_i dx_i))
};

__global__ void norm_table_kernel(NormParams p, double dx0, double dx1, double dx2,
                                  double* __restrict__ tab) {
    // tab layout: for axis a: [k (N_a)], [s2 (N_a)], [c (N_a)] consecutively
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    int off = 0;
    const double dxa[3] = {dx0, dx1, dx2};
    for (int a = 0; a < 3; ++a) {
        const int n = p.N[a];
        if (t < n) {
            double k = 0.0;
            if (a < p.dims) k = (t + 0.5) * M_PI / (n * dxa[a]);
            const double sn = sin(0.5 * k * dxa[a]) / dxa[a];
            tab[off + t] = k;
            tab[off + n + t] = sn * sn;
            tab[off + 2 * n + t] = cos(k * dxa[a]);
        }
        off += 3 * n;
    }
}

__global__ void __launch_bounds__(NORM_THREADS)
norm_kernel(NormParams p, const double* __restrict__ tab, double* __restrict__ partials) {
    double acc[NQ];
#pragma unroll
    for (int q = 0; q < NQ; ++q) acc[q] = 0.0;
    const double* kx = tab;
    const double* s2x = tab + p.N[0];
    const double* cx = tab + 2 * p.N[0];
    const double* ky = tab + 3 * p.N[0];
    const double* s2y = ky + p.N[1];
    const double* cy = ky + 2 * p.N[1];
    const double* kz = tab + 3 * p.N[0] + 3 * p.N[1];
    const double* s2z = kz + p.N[2];
    const double* cz = kz + 2 * p.N[2];
    const double dt = p.dt;
    const double inv_dt = 1.0 / dt, two_over_dt = 2.0 * inv_dt;
    for (long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x; t < p.npts;
         t += (long long)gridDim.x * blockDim.x) {
        const int mx = (int)(t % p.N[0]);
        const long long r = t / p.N[0];
        const int my = (int)(r % p.N[1]);
        const int mz = (int)(r / p.N[1]);
        const double k[3] = {kx[mx], ky[my], kz[mz]};
        const double s2[3] = {s2x[mx], s2y[my], s2z[mz]};
        const double c[3] = {cx[mx], cy[my], cz[mz]};
        double S = 0.0;
#pragma unroll
        for (int i = 0; i < 3; ++i) {
            double A = p.alpha[i] + p.delta[i] * (1.0 + 2.0 * c[i]);
#pragma unroll
            for (int j = 0; j < 3; ++j)
                if (j != i) A += 2.0 * p.beta[i][j] * c[j];
            S += s2[i] * A;
        }
        const double kn = sqrt(k[0] * k[0] + k[1] * k[1] + k[2] * k[2]);
        double w = 1.0;
        if (p.weight == FDTD_W_CONE_X) {
            w = (k[0] >= kn * p.wparam) ? 1.0 : 0.0;
        } else if (p.weight == FDTD_W_GAUSS_Y) {
            const double u = k[1] * p.wparam;
            w = exp(-u * u);
        }
        if (w == 0.0) continue;
        // one division per point: sqrt(S) / (dt sqrt(1 - dt^2 S)) = S dwdS / dt
        const double sq = sqrt(S);
        const double om = two_over_dt * asin(dt * sq);
        const double res = om - kn;
        const double root = sqrt(1.0 - dt * dt * S);
        const double dwdS = 1.0 / (sq * root);
        const double g = 2.0 * w * res;
        acc[0] += w * res * res;
        const double gs2 = 2.0 * g * dwdS;
        const double tx = gs2 * s2[0], ty = gs2 * s2[1], tz = gs2 * s2[2];
        const double cx1 = c[0] - 1.0, cy1 = c[1] - 1.0, cz1 = c[2] - 1.0;
        // beta: (x,y), (x,z), (y,x), (y,z), (z,x), (z,y)
        acc[1] += tx * cy1;
        acc[2] += tx * cz1;
        acc[3] += ty * cx1;
        acc[4] += ty * cz1;
        acc[5] += tz * cx1;
        acc[6] += tz * cy1;
        acc[7] += tx * cx1;
        acc[8] += ty * cy1;
        acc[9] += tz * cz1;
        acc[10] += g * inv_dt * (2.0 * S * dwdS - om);
    }
    __shared__ double red[NORM_THREADS / 32][NQ];
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
#pragma unroll
    for (int q = 0; q < NQ; ++q) {
        double v = acc[q];
        for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
        if (l == 0) red[w][q] = v;
    }
    __syncthreads();
    if (threadIdx.x < NQ) {
        double v = 0.0;
        for (int ww = 0; ww < NORM_THREADS / 32; ++ww) v += red[ww][threadIdx.x];
        partials[(long long)blockIdx.x * NQ + threadIdx.x] = v;
    }
}

// out[14] = {f, dbeta 3x3 row-major, ddelta 3, ddt}
__global__ void norm_final_kernel(const double* __restrict__ part, int nblocks, double pref,
                                  double* __restrict__ out) {
    __shared__ double red[NQ][32];
    const int q = threadIdx.y, l = threadIdx.x;
    double v = 0.0;
    for (int b = l; b < nblocks; b += 32) v += part[(long long)b * NQ + q];
    red[q][l] = v;
    __syncthreads();
    if (l == 0) {
        double s = 0.0;
        for (int t = 0; t < 32; ++t) s += red[q][t];
        s *= pref;
        // map q -> out slot
        const int slot[NQ] = {0, 1 + 1, 1 + 2, 1 + 3, 1 + 5, 1 + 6, 1 + 7, 10, 11, 12, 13};
        out[slot[q]] = s;
    }
    if (q == 0 && l < 3) out[1 + 4 * l] = 0.0;   // diagonal of d/d beta
}

int norm_blocks(long long npts) {
    long long b = (npts + NORM_THREADS - 1) / NORM_THREADS;
    if (b > 152 * 16) b = 152 * 16;
    if (b < 1) b = 1;
    return (int)b;
}

size_t norm_scratch_doubles(const int N[3], long long npts) {
    return (size_t)3 * (N[0] + N[1] + N[2]) + (size_t)norm_blocks(npts) * NQ + 14;
}

// Runs the three kernels on `st` using `scratch` (norm_scratch_doubles() doubles);
// the 14 results land in scratch's last 14 entries and are returned via *out_dev.
void launch_disp_norm(const double alpha[3], const double beta[3][3], const double delta[3],
                      double dt, const double dx[3], int dims, const int N[3], int weight,
                      double wparam, double* scratch, double** out_dev, cudaStream_t st) {
    NormParams p;
    for (int i = 0; i < 3; ++i) {
        p.alpha[i] = alpha[i];
        p.delta[i] = delta[i];
        for (int j = 0; j < 3; ++j) p.beta[i][j] = beta[i][j];
        p.N[i] = i < dims ? N[i] : 1;
    }
    p.dt = dt;
    p.dims = dims;
    p.weight = weight;
    if (weight == FDTD_W_CONE_X) p.wparam = cos(wparam);
    else if (weight == FDTD_W_GAUSS_Y) p.wparam = dx[1] / wparam;
    else p.wparam = 0.0;
    p.npts = (long long)p.N[0] * p.N[1] * p.N[2];
    double pref = 1.0;
    for (int i = 0; i < dims; ++i) pref *= dx[i] * (M_PI / (p.N[i] * dx[i]));
    p.pref = pref;
    double* tab = scratch;
    const size_t ntab = (size_t)3 * (p.N[0] + p.N[1] + p.N[2]);
    double* part = scratch + ntab;
    const int nb = norm_blocks(p.npts);
    double* out = part + (size_t)nb * NQ;
    int nmax = p.N[0] > p.N[1] ? p.N[0] : p.N[1];
    if (p.N[2] > nmax) nmax = p.N[2];
    norm_table_kernel<<<(nmax + 255) / 256, 256, 0, st>>>(p, dx[0], dx[1], dx[2], tab);
    norm_kernel<<<nb, NORM_THREADS, 0, st>>>(p, tab, part);
    norm_final_kernel<<<1, dim3(32, NQ), 0, st>>>(part, nb, pref, out);
    *out_dev = out;
}

}  // namespace fdtd

namespace fdtd {

// omega(k) of Eq. (dispersion_relation) at n arbitrary wave vectors (FP64 per point).
__global__ void omega_kernel(NormParams p, double dx0, double dx1, double dx2,
                             const double* __restrict__ k, int n, double* __restrict__ out) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= n) return;
    const double dxa[3] = {dx0, dx1, dx2};
    double s2[3], c[3];
    for (int i = 0; i < 3; ++i) {
        const double ki = i < p.dims ? k[3 * t + i] : 0.0;
        const double sn = sin(0.5 * ki * dxa[i]) / dxa[i];
        s2[i] = sn * sn;
        c[i] = cos(ki * dxa[i]);
    }
    double S = 0.0;
    for (int i = 0; i < 3; ++i) {
        double A = p.alpha[i] + p.delta[i] * (1.0 + 2.0 * c[i]);
        for (int j = 0; j < 3; ++j)
            if (j != i) A += 2.0 * p.beta[i][j] * c[j];
        S += s2[i] * A;
    }
    out[t] = 2.0 / p.dt * asin(p.dt * sqrt(S));
}

void launch_omega(const double alpha[3], const double beta[3][3], const double delta[3], double dt,
                  const double dx[3], int dims, const double* k_dev, int n, double* out_dev,
                  cudaStream_t st) {
    NormParams p;
    for (int i = 0; i < 3; ++i) {
        p.alpha[i] = alpha[i];
        p.delta[i] = delta[i];
        for (int j = 0; j < 3; ++j) p.beta[i][j] = beta[i][j];
    }
    p.dt = dt;
    p.dims = dims;
    omega_kernel<<<(n + 127) / 128, 128, 0, st>>>(p, dx[0], dx[1], dx[2], k_dev, n, out_dev);
}

}  // namespace fdtd

namespace fdtd {

// ---- group-velocity norm (the conclusions' proposal; this library's reading) ----------------
// f_g = prefactor * sum w (|d omega/dk| - 1)^2 on the same midpoint grid, with
//   A_i = alpha_i + delta_i (1 + 2 c_i) + 2 sum_{j != i} beta_ij c_j       (as in norm_kernel)
//   G_m = dS/dk_m = sin(k_m dx_m)/(2 dx_m) A_m - 2 dx_m sin(k_m dx_m) (delta_m s_m^2
//                                                    + sum_{i != m} beta_im s_i^2)
//   |v_g| = w_S |G|,  w_S = 1 / (sqrt(S) sqrt(1 - dt^2 S)),
// and the gradient by the chain rule (w_SS = -w_S^3 (1 - 2 dt^2 S) / 2, d w_S/d dt = w_S^3 dt S^2):
//   d|v_g| = w_SS dS |G| + w_S (G . dG) / |G|, with dS/d beta_ij = 2 s_i^2 (c_j - 1),
//   dS/d delta_i = 2 s_i^2 (c_i - 1), dG_m/d beta_ij = [m=i] sin_i (c_j - 1)/dx_i
//   - [m=j] 2 dx_j sin_j s_i^2, dG_m/d delta_i = [m=i] (sin_i (c_i - 1)/dx_i - 2 dx_i sin_i s_i^2).
// FP64 throughout; per-block partials and the fixed-order final sum of norm_kernel.

struct GroupParams {
    NormParams n;
    double dx[3];
};

__global__ void group_table_kernel(GroupParams p, double* __restrict__ tab) {
    // tab layout: for axis a: [k], [s2], [c], [sin(k dx)] of N_a entries each
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    int off = 0;
    for (int a = 0; a < 3; ++a) {
        const int n = p.n.N[a];
        if (t < n) {
            double k = 0.0;
            if (a < p.n.dims) k = (t + 0.5) * M_PI / (n * p.dx[a]);
            const double sn = sin(0.5 * k * p.dx[a]) / p.dx[a];
            tab[off + t] = k;
            tab[off + n + t] = sn * sn;
            tab[off + 2 * n + t] = cos(k * p.dx[a]);
            tab[off + 3 * n + t] = sin(k * p.dx[a]);
        }
        off += 4 * n;
    }
}

__global__ void __launch_bounds__(NORM_THREADS)
group_norm_kernel(GroupParams gp, const double* __restrict__ tab, double* __restrict__ partials) {
    const NormParams& p = gp.n;
    double acc[NQ];
#pragma unroll
    for (int q = 0; q < NQ; ++q) acc[q] = 0.0;
    const double* T[3];
    {
        int off = 0;
        for (int a = 0; a < 3; ++a) {
            T[a] = tab + off;
            off += 4 * p.N[a];
        }
    }
    const double dt = p.dt;
    for (long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x; t < p.npts;
         t += (long long)gridDim.x * blockDim.x) {
        const int mi[3] = {(int)(t % p.N[0]), (int)((t / p.N[0]) % p.N[1]),
                           (int)(t / ((long long)p.N[0] * p.N[1]))};
        double k[3], s2[3], c[3], sn[3];
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            const int n = p.N[a];
            k[a] = T[a][mi[a]];
            s2[a] = T[a][n + mi[a]];
            c[a] = T[a][2 * n + mi[a]];
            sn[a] = T[a][3 * n + mi[a]];
        }
        double A[3], S = 0.0;
#pragma unroll
        for (int i = 0; i < 3; ++i) {
            double a = p.alpha[i] + p.delta[i] * (1.0 + 2.0 * c[i]);
#pragma unroll
            for (int j = 0; j < 3; ++j)
                if (j != i) a += 2.0 * p.beta[i][j] * c[j];
            A[i] = a;
            S += s2[i] * a;
        }
        const double kn = sqrt(k[0] * k[0] + k[1] * k[1] + k[2] * k[2]);
        double w = 1.0;
        if (p.weight == FDTD_W_CONE_X) {
            w = (k[0] >= kn * p.wparam) ? 1.0 : 0.0;
        } else if (p.weight == FDTD_W_GAUSS_Y) {
            const double u = k[1] * p.wparam;
            w = exp(-u * u);
        }
        if (w == 0.0) continue;
        double G[3];
#pragma unroll
        for (int m = 0; m < 3; ++m) {
            double tm = p.delta[m] * s2[m];
#pragma unroll
            for (int i = 0; i < 3; ++i)
                if (i != m) tm += p.beta[i][m] * s2[i];
            G[m] = sn[m] / (2.0 * gp.dx[m]) * A[m] - 2.0 * gp.dx[m] * sn[m] * tm;
        }
        const double Gn = sqrt(G[0] * G[0] + G[1] * G[1] + G[2] * G[2]);
        const double wS = 1.0 / (sqrt(S) * sqrt(1.0 - dt * dt * S));
        const double vg = wS * Gn;
        const double r = vg - 1.0;
        acc[0] += w * r * r;
        const double cm = 2.0 * w * r;
        const double wS3 = wS * wS * wS;
        const double wSS = -0.5 * wS3 * (1.0 - 2.0 * dt * dt * S);
        const double a1 = cm * wSS * Gn;   // times dS/dtheta
        const double a2 = cm * wS / Gn;    // times G . dG/dtheta
        // beta: (x,y), (x,z), (y,x), (y,z), (z,x), (z,y)  (same slots as norm_kernel)
        const int bi[6] = {0, 0, 1, 1, 2, 2}, bj[6] = {1, 2, 0, 2, 0, 1};
#pragma unroll
        for (int q = 0; q < 6; ++q) {
            const int i = bi[q], j = bj[q];
            const double dS = 2.0 * s2[i] * (c[j] - 1.0);
            const double GdG = G[i] * sn[i] * (c[j] - 1.0) / gp.dx[i] -
                               G[j] * 2.0 * gp.dx[j] * sn[j] * s2[i];
            acc[1 + q] += a1 * dS + a2 * GdG;
        }
#pragma unroll
        for (int i = 0; i < 3; ++i) {
            const double dS = 2.0 * s2[i] * (c[i] - 1.0);
            const double GdG = G[i] * (sn[i] * (c[i] - 1.0) / gp.dx[i] - 2.0 * gp.dx[i] * sn[i] * s2[i]);
            acc[7 + i] += a1 * dS + a2 * GdG;
        }
        acc[10] += cm * wS3 * dt * S * S * Gn;
    }
    __shared__ double red[NORM_THREADS / 32][NQ];
    const int wq = threadIdx.x >> 5, l = threadIdx.x & 31;
#pragma unroll
    for (int q = 0; q < NQ; ++q) {
        double v = acc[q];
        for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
        if (l == 0) red[wq][q] = v;
    }
    __syncthreads();
    if (threadIdx.x < NQ) {
        double v = 0.0;
        for (int ww = 0; ww < NORM_THREADS / 32; ++ww) v += red[ww][threadIdx.x];
        partials[(long long)blockIdx.x * NQ + threadIdx.x] = v;
    }
}

size_t group_scratch_doubles(const int N[3], long long npts) {
    return (size_t)4 * (N[0] + N[1] + N[2]) + (size_t)norm_blocks(npts) * NQ + 14;
}

void launch_disp_group_norm(const double alpha[3], const double beta[3][3], const double delta[3],
                            double dt, const double dx[3], int dims, const int N[3], int weight,
                            double wparam, double* scratch, double** out_dev, cudaStream_t st) {
    GroupParams gp;
    NormParams& p = gp.n;
    for (int i = 0; i < 3; ++i) {
        p.alpha[i] = alpha[i];
        p.delta[i] = delta[i];
        for (int j = 0; j < 3; ++j) p.beta[i][j] = beta[i][j];
        p.N[i] = i < dims ? N[i] : 1;
        gp.dx[i] = dx[i];
    }
    p.dt = dt;
    p.dims = dims;
    p.weight = weight;
    if (weight == FDTD_W_CONE_X) p.wparam = cos(wparam);
    else if (weight == FDTD_W_GAUSS_Y) p.wparam = dx[1] / wparam;
    else p.wparam = 0.0;
    p.npts = (long long)p.N[0] * p.N[1] * p.N[2];
    double pref = 1.0;
    for (int i = 0; i < dims; ++i) pref *= dx[i] * (M_PI / (p.N[i] * dx[i]));
    p.pref = pref;
    double* tab = scratch;
    const size_t ntab = (size_t)4 * (p.N[0] + p.N[1] + p.N[2]);
    double* part = scratch + ntab;
    const int nb = norm_blocks(p.npts);
    double* out = part + (size_t)nb * NQ;
    int nmax = p.N[0] > p.N[1] ? p.N[0] : p.N[1];
    if (p.N[2] > nmax) nmax = p.N[2];
    group_table_kernel<<<(nmax + 255) / 256, 256, 0, st>>>(gp, tab);
    group_norm_kernel<<<nb, NORM_THREADS, 0, st>>>(gp, tab, part);
    norm_final_kernel<<<1, dim3(32, NQ), 0, st>>>(part, nb, pref, out);
    *out_dev = out;
}

}  // namespace fdtd
