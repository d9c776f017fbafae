// Constrained coefficient update (the minimisation of Sec. 4, done as projected gradient
// descent in FP64 on the GPU).
//
// Free parameters theta (n <= 16) map linearly onto the 13 scheme parameters
// c = (beta 3x3 row-major, delta 3, dt):  c = c0 + T^T theta  (T is n x 13, the parameter
// tying of Sec. 4, e.g. beta_xy = beta_yx, delta_x = delta_y).  Given the gradient g of the
// objective with respect to c (the layout of disp_norm_eval's out[1..13]), one update is
//   theta' = clip(theta - eta T g, lo, hi),   c' = c0 + T^T theta'.
#include "fdtd_internal.cuh"

namespace fdtd {

constexpr int CU_MAXN = 16;

struct CoeffUpdateArgs {
    int n;
    double eta;
    double theta[CU_MAXN], lo[CU_MAXN], hi[CU_MAXN];
    double g[13], c0[13];
    double T[CU_MAXN][13];
};

// one warp: lane i < n owns theta_i, lane j < 13 forms c'_j
__global__ void coeff_update_kernel(CoeffUpdateArgs a, double* __restrict__ out) {
    __shared__ double th[CU_MAXN];
    const int l = threadIdx.x;
    if (l < a.n) {
        double gi = 0.0;
        for (int j = 0; j < 13; ++j) gi = fma(a.T[l][j], a.g[j], gi);
        double v = a.theta[l] - a.eta * gi;
        v = fmin(fmax(v, a.lo[l]), a.hi[l]);
        th[l] = v;
        out[l] = v;
    }
    __syncwarp();
    if (l < 13) {
        double c = a.c0[l];
        for (int i = 0; i < a.n; ++i) c = fma(a.T[i][l], th[i], c);
        out[a.n + l] = c;
    }
}

}  // namespace fdtd

using namespace fdtd;

int fdtd_coeff_update(int32_t n, const double* theta, const double* grad13, const double* T,
                      const double* c0, double eta, const double* lo, const double* hi,
                      double* out_dev, void* stream) {
    if (n < 1 || n > CU_MAXN || !theta || !grad13 || !T || !c0 || !lo || !hi || !out_dev) {
        set_error("fdtd_coeff_update: bad argument (1 <= n <= %d, no NULL pointers)", CU_MAXN);
        return FDTD_EINVAL;
    }
    CoeffUpdateArgs a;
    a.n = n;
    a.eta = eta;
    for (int i = 0; i < n; ++i) {
        a.theta[i] = theta[i];
        a.lo[i] = lo[i];
        a.hi[i] = hi[i];
        if (!(lo[i] <= hi[i])) {
            set_error("fdtd_coeff_update: lo[%d] > hi[%d]", i, i);
            return FDTD_EINVAL;
        }
        for (int j = 0; j < 13; ++j) a.T[i][j] = T[i * 13 + j];
    }
    for (int j = 0; j < 13; ++j) {
        a.g[j] = grad13[j];
        a.c0[j] = c0[j];
    }
    cudaStream_t st = (cudaStream_t)stream;
    coeff_update_kernel<<<1, 32, 0, st>>>(a, out_dev);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) {
        set_error("fdtd_coeff_update: %s", cudaGetErrorString(e));
        return FDTD_ECUDA;
    }
    return FDTD_OK;
}
