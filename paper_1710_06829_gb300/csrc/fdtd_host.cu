// Host side of libfdtd: the C ABI declared in include/fdtd.h.
//
// Coefficient preprocessing (FP64): alpha from Eq. (alpha), exact extremes of
// S(k) over the Brillouin box for Eq. (constraints), update multipliers
// rounded once to the working precision.  State management (padded library
// layout, ping-pong sets, adjoint state, recorded E history, checkpoint
// slots) and the launch sequences of the forward and adjoint steps.
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <mutex>
#include <new>
#include <type_traits>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "fdtd_tma.cuh"
#include "pic.cuh"

namespace fdtd {

static thread_local char g_err[512] = "no error";

void set_error(const char* fmt, ...) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_err, sizeof(g_err), fmt, ap);
    va_end(ap);
}

template <typename T>
void launch_current(const Geom& g, T* const E[3], const T* const J[3], T dt, const T* sponge_y,
                    const T* sponge_z, cudaStream_t st);
template <typename T>
void launch_bunch_table(int nx, int n, double x0, double vdt, double inv_sig, double scale,
                        double dx, double Lx, long long step0, T* out, cudaStream_t st);
void launch_disp_norm(const double alpha[3], const double beta[3][3], const double delta[3],
                      double dt, const double dx[3], int dims, const int N[3], int weight,
                      double wparam, double* scratch, double** out_dev, cudaStream_t st);
size_t group_scratch_doubles(const int N[3], long long npts);
void launch_disp_group_norm(const double alpha[3], const double beta[3][3], const double delta[3],
                            double dt, const double dx[3], int dims, const int N[3], int weight,
                            double wparam, double* scratch, double** out_dev, cudaStream_t st);
size_t norm_scratch_doubles(const int N[3], long long npts);
int diag_blocks(const Geom& g);
void launch_omega(const double alpha[3], const double beta[3][3], const double delta[3], double dt,
                  const double dx[3], int dims, const double* k_dev, int n, double* out_dev,
                  cudaStream_t st);
bool encode_ebox_f32(CUtensorMap* map, const Geom& g, float* base);
bool encode_box_f32(CUtensorMap* map, const Geom& g, float* base, int bw, int bh);
bool adjoint32_supported(const Geom& g);
int adjoint32_blocks(const Geom& g);
bool adjoint32_prepare();
void launch_adjoint32_B(const FusedMaps& maps, const Geom& g, const Mult<float>& m,
                        FieldSet<float> lam, const float* spy, const float* spz, double* partials,
                        int* err, cudaStream_t st);
bool adjoint32e_supported(const Geom& g);
bool adjoint32e_prepare();
bool adjoint32f_supported(const Geom& g);
bool adjoint32f_prepare();
int adjoint32f_blocks(const Geom& g);
void launch_adjoint32_fused(const FusedMaps& maps, const Geom& g, const Mult<float>& m,
                            FieldSet<float> lam, FieldSet<float> out, const float* const E[3],
                            const float* spy, const float* spz, double* partials, int* err,
                            cudaStream_t st);
void launch_adjoint32_E(const FusedMaps& maps, const Geom& g, const Mult<float>& m,
                        FieldSet<float> lam, const float* spy, const float* spz, int* err,
                        cudaStream_t st);
template <typename T>
void launch_energy(const Geom& g, FieldSet<T> s, int x_lo, int x_len, int my, int mz, double dV,
                   double* part, double* out, cudaStream_t st);
template <typename T>
void launch_planewave(const Geom& g, const T* F, const double k[3], const double off[3],
                      double* part, double* out, cudaStream_t st);
template <typename T>
void launch_moments(const Geom& g, FieldSet<T> s, int axis, double dV, double* part, double* out,
                    cudaStream_t st);
template <typename T>
void launch_divergence(const Geom& g, const Mult<double>& w, FieldSet<T> s, int which, double* out,
                       cudaStream_t st);

// ---------------------------------------------------------------------------
// coefficient preprocessing
// ---------------------------------------------------------------------------

struct Clean {
    double beta[3][3];
    double delta[3];
    double alpha[3];
};

static Clean clean_coeffs(const fdtd_coeffs* c, int dims) {
    Clean r;
    for (int i = 0; i < 3; ++i) {
        r.delta[i] = (i < dims) ? c->delta[i] : 0.0;
        for (int j = 0; j < 3; ++j)
            r.beta[i][j] = (i != j && i < dims && j < dims) ? c->beta[i][j] : 0.0;
    }
    for (int i = 0; i < 3; ++i)
        r.alpha[i] = 1.0 - 2.0 * (r.beta[i][0] + r.beta[i][1] + r.beta[i][2]) - 3.0 * r.delta[i];
    return r;
}

// S as a quadratic in u_i = s_i^2 in [0, 1/dx_i^2] (Sec. 3 with alpha eliminated):
//   S(u) = sum_i u_i - sum_i 4 dx_i^2 delta_i u_i^2 - sum_{i != j} 4 dx_j^2 beta_ij u_i u_j.
// Its extremes over the box are attained where every coordinate is at a bound or
// free with vanishing partial derivative; all 3^dims patterns are solved.
static void S_extremes(const Clean& cc, const double dx[3], int dims, double* smin,
                       double* smax) {
    double Q[3][3] = {{0}};
    for (int i = 0; i < dims; ++i) {
        Q[i][i] = 4.0 * dx[i] * dx[i] * cc.delta[i];
        for (int j = 0; j < dims; ++j)
            if (i != j) Q[i][j] = 2.0 * (dx[j] * dx[j] * cc.beta[i][j] + dx[i] * dx[i] * cc.beta[j][i]);
    }
    double ub[3];
    for (int i = 0; i < 3; ++i) ub[i] = 1.0 / (dx[i] * dx[i]);
    double lo = 1e300, hi = -1e300;
    int npat = 1;
    for (int i = 0; i < dims; ++i) npat *= 3;
    for (int p = 0; p < npat; ++p) {
        int pat[3] = {0, 0, 0};
        int t = p;
        for (int i = 0; i < dims; ++i) { pat[i] = t % 3; t /= 3; }
        double u[3] = {0, 0, 0};
        int fr[3], nf = 0;
        for (int i = 0; i < dims; ++i) {
            if (pat[i] == 1) u[i] = ub[i];
            if (pat[i] == 2) fr[nf++] = i;
        }
        bool ok = true;
        if (nf > 0) {
            // solve 2 Q_FF u_F = 1 - 2 Q_F,fixed u_fixed by Gaussian elimination with pivoting
            double A[3][4];
            for (int r = 0; r < nf; ++r) {
                double rhs = 1.0;
                for (int j = 0; j < dims; ++j)
                    if (pat[j] != 2) rhs -= 2.0 * Q[fr[r]][j] * u[j];
                for (int s = 0; s < nf; ++s) A[r][s] = 2.0 * Q[fr[r]][fr[s]];
                A[r][nf] = rhs;
            }
            double scale = 0.0;
            for (int r = 0; r < nf; ++r)
                for (int s = 0; s < nf; ++s) scale = fmax(scale, fabs(A[r][s]));
            for (int col = 0; col < nf && ok; ++col) {
                int piv = col;
                for (int r = col + 1; r < nf; ++r)
                    if (fabs(A[r][col]) > fabs(A[piv][col])) piv = r;
                if (fabs(A[piv][col]) <= 1e-13 * fmax(scale, 1.0)) { ok = false; break; }
                for (int s = 0; s <= nf; ++s) { double tmp = A[col][s]; A[col][s] = A[piv][s]; A[piv][s] = tmp; }
                for (int r = 0; r < nf; ++r) {
                    if (r == col) continue;
                    const double f = A[r][col] / A[col][col];
                    for (int s = col; s <= nf; ++s) A[r][s] -= f * A[col][s];
                }
            }
            if (!ok) continue;
            for (int r = 0; r < nf; ++r) {
                const double v = A[r][nf] / A[r][r];
                const int i = fr[r];
                if (v < -1e-15 || v > ub[i] * (1.0 + 1e-15)) { ok = false; break; }
                u[i] = fmin(fmax(v, 0.0), ub[i]);
            }
            if (!ok) continue;
        }
        double S = 0.0;
        for (int i = 0; i < dims; ++i) S += u[i];
        for (int i = 0; i < dims; ++i)
            for (int j = 0; j < dims; ++j) S -= Q[i][j] * u[i] * u[j];
        lo = fmin(lo, S);
        hi = fmax(hi, S);
    }
    *smin = lo;
    *smax = hi;
}

static int validate(const Clean& cc, const double dx[3], int dims, double dt) {
    for (int i = 0; i < 3; ++i) {
        if (!std::isfinite(cc.delta[i]) || !std::isfinite(cc.alpha[i])) {
            set_error("non-finite coefficient");
            return FDTD_EINVAL;
        }
        for (int j = 0; j < 3; ++j)
            if (!std::isfinite(cc.beta[i][j])) {
                set_error("non-finite coefficient");
                return FDTD_EINVAL;
            }
    }
    if (!(dt > 0.0) || !std::isfinite(dt)) {
        set_error("dt must be positive and finite (got %g)", dt);
        return FDTD_EINVAL;
    }
    double smin, smax;
    S_extremes(cc, dx, dims, &smin, &smax);
    if (smin < -1e-12) {
        set_error("Eq. (constraints) violated: min_k S = %.6g < 0", smin);
        return FDTD_EUNSTABLE;
    }
    if (dt * dt * smax > 1.0 + 1e-12) {
        set_error("Eq. (constraints) violated: dt^2 max_k S = %.12g > 1 (dt_max = %.12g)",
                  dt * dt * smax, 1.0 / sqrt(smax));
        return FDTD_EUNSTABLE;
    }
    return FDTD_OK;
}

// zcouple = false (batched 2D problems): every multiplier of a z difference is zero, so
// the planes never exchange values.
template <typename T>
static Mult<T> make_mult(const Clean& cc, const double dx[3], double dt, bool zcouple = true) {
    Mult<T> m;
    for (int a = 0; a < 3; ++a) {
        m.cA[a] = (T)(dt * cc.alpha[a] / dx[a]);
        m.cD[a] = (T)(dt * cc.delta[a] / dx[a]);
        for (int b = 0; b < 3; ++b) m.cB[a][b] = (T)(dt * cc.beta[a][b] / dx[a]);
        m.cE[a] = (T)(dt / dx[a]);
    }
    if (!zcouple) {
        m.cA[2] = m.cD[2] = m.cE[2] = (T)0;
        for (int b = 0; b < 3; ++b) m.cB[2][b] = m.cB[b][2] = (T)0;
    }
    m.dt = (T)dt;
    return m;
}

}  // namespace fdtd

using namespace fdtd;

#define CK(call)                                                                        \
    do {                                                                                \
        cudaError_t e_ = (call);                                                        \
        if (e_ != cudaSuccess) {                                                        \
            set_error("%s failed: %s (%s:%d)", #call, cudaGetErrorString(e_), __FILE__, \
                      __LINE__);                                                        \
            return e_ == cudaErrorMemoryAllocation ? FDTD_ENOMEM : FDTD_ECUDA;          \
        }                                                                               \
    } while (0)

struct fdtd_handle {
    fdtd_grid grid;
    double dx[3];
    double dt;
    fdtd_coeffs coeffs;
    Clean cc;
    cudaStream_t stream;
    Geom g;
    size_t esz;
    char* state;        // 2 sets x 6 padded arrays
    int cur;
    char* lam;          // 6 padded arrays
    char* hist;         // history: snapshots x 3 padded arrays
    int hist_cap;
    int hist_len;       // snapshots stored
    long long hist_step0;
    std::vector<char*> ckpt;
    std::vector<long long> ckpt_step;
    char* aux;          // sponge_y[ny], sponge_z[nz], bunch_y[ny], bunch_z[nz] (T)
    char* jx;           // bunch x-profile table [cap][nx]
    int jx_cap;
    double* partials;   // adjoint gradient partials
    int npart;
    cudaStream_t xfer;  // copy stream of the host transfers (created on first use)
    cudaEvent_t filled[2];   // ordering events between the handle's stream and the copy stream
    long long step;
    int use_fused;
    double* dpart;      // diagnostics partials (3 per block)
    std::vector<FusedMaps> hist_maps;   // TMA descriptors of each history snapshot (FP32 adjoint)
    FusedMaps lam_maps;                 // .e[c]: TMA descriptors of lambda_B component c (FP32)
    bool lam_staged = false;            // lam_maps valid: the staged FP32 adjoint E kernel runs
    // FP32 one-kernel reverse step: two adjoint state sets (the kernel writes the other one),
    // lam_emaps[s].e[c] / .b[c] the TMA descriptors of lambda_E / lambda_B component c of set s
    bool lam_fused = false;
    int lam_sets = 1, lam_cur = 0;
    FusedMaps lam_emaps[2];
    int adj_split = 0;                  // FDTD_ADJOINT_SPLIT=1: the two-kernel reverse step
    FusedPlan* plan;    // TMA descriptors of both state sets (nullptr: reference-form kernels)
    int* err_dev;       // ERR_WAIT: a bounded wait inside a kernel expired; ERR_PARTICLE: a
                        // particle with a non-finite (or out-of-range) position or momentum;
                        // ERR_FIELD: a step wrote a non-finite field value
    int tblock = 1;     // temporal blocking: 1 (one launch per step) or 2 (pairs by slabs)
    int tslab = 32;     // slab length in planes of the blocked schedule

    void* arr(int set, int c) { return state + ((size_t)set * 6 + c) * g.total * esz; }
    void* lam_arr(int c) { return lam_arr_set(lam_cur, c); }
    void* lam_arr_set(int set, int c) { return lam + ((size_t)set * 6 + c) * g.total * esz; }
    void* hist_arr(int snap, int c) { return hist + ((size_t)snap * 3 + c) * g.total * esz; }
};

template <typename T>
static FieldSet<T> fieldset(fdtd_handle* h, int set) {
    FieldSet<T> s;
    for (int c = 0; c < 6; ++c) s.c[c] = (T*)h->arr(set, c);
    return s;
}

template <typename T>
static FieldSet<T> lamset(fdtd_handle* h) {
    FieldSet<T> s;
    for (int c = 0; c < 6; ++c) s.c[c] = (T*)h->lam_arr(c);
    return s;
}

template <typename T>
static int upload_aux(fdtd_handle* h) {
    const int ny = h->g.ny, nz = h->g.nz;
    std::vector<T> a(2 * (size_t)(ny + nz), (T)1);
    const int L = h->grid.absorb_cells;
    const double sg = h->grid.absorb_sigma;
    auto prof = [&](int n, int idx) -> double {
        if (L <= 0) return 1.0;
        int d = 0;
        if (idx < L) d = L - idx;
        else if (idx >= n - L) d = idx - (n - L - 1);
        if (d <= 0) return 1.0;
        const double x = (double)d / L;
        return 1.0 - sg * x * x * x;
    };
    for (int j = 0; j < ny; ++j) a[j] = (T)prof(ny, j);
    for (int k = 0; k < nz; ++k) a[ny + k] = h->grid.batched ? (T)1 : (T)prof(nz, k);
    CK(cudaMemcpyAsync(h->aux, a.data(), a.size() / 2 * sizeof(T), cudaMemcpyHostToDevice,
                       h->stream));
    CK(cudaStreamSynchronize(h->stream));
    return FDTD_OK;
}

static double Phi(double x) { return 0.5 * erfc(-x / sqrt(2.0)); }

template <typename T>
static int upload_bunch_yz(fdtd_handle* h, const fdtd_source* src) {
    const int ny = h->g.ny, nz = h->g.nz;
    std::vector<T> a((size_t)(ny + nz));
    const double Ly = ny * h->dx[1], Lz = nz * h->dx[2];
    for (int j = 0; j < ny; ++j) {
        double d = j * h->dx[1] - src->y0;
        d = d - Ly * floor(d / Ly + 0.5);
        a[j] = (T)(Phi((d + 0.5 * h->dx[1]) / src->sigma_perp) -
                   Phi((d - 0.5 * h->dx[1]) / src->sigma_perp));
    }
    for (int k = 0; k < nz; ++k) {
        double d = k * h->dx[2] - src->z0;
        d = d - Lz * floor(d / Lz + 0.5);
        a[ny + k] = (T)(Phi((d + 0.5 * h->dx[2]) / src->sigma_perp) -
                        Phi((d - 0.5 * h->dx[2]) / src->sigma_perp));
    }
    T* dst = (T*)h->aux + (ny + nz);
    CK(cudaMemcpyAsync(dst, a.data(), a.size() * sizeof(T), cudaMemcpyHostToDevice, h->stream));
    CK(cudaStreamSynchronize(h->stream));
    return FDTD_OK;
}

// Exported functions: C linkage comes from their declarations in fdtd.h.

const char* fdtd_last_error(void) { return g_err; }

// NVTX range around an entry point that launches GPU work: the range names the call in a
// profiler's timeline (ncu --nvtx, nsys); without a tool attached NVTX does nothing.
namespace {
struct NvtxRange {
    explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
    NvtxRange(const NvtxRange&) = delete;
    NvtxRange& operator=(const NvtxRange&) = delete;
};
}  // namespace

int fdtd_dt_max(const fdtd_coeffs* coeffs, const double dx[3], int32_t dims, double* dt_max,
                double* s_min, double* s_max) {
    if (!coeffs || !dx || dims < 1 || dims > 3) {
        set_error("fdtd_dt_max: bad argument");
        return FDTD_EINVAL;
    }
    for (int i = 0; i < 3; ++i)
        if (!(dx[i] > 0)) {
            set_error("dx must be positive");
            return FDTD_EINVAL;
        }
    Clean cc = clean_coeffs(coeffs, dims);
    double lo, hi;
    S_extremes(cc, dx, dims, &lo, &hi);
    if (s_min) *s_min = lo;
    if (s_max) *s_max = hi;
    if (dt_max) *dt_max = hi > 0 ? 1.0 / sqrt(hi) : INFINITY;
    return FDTD_OK;
}

int fdtd_create(const fdtd_grid* grid, const double dx[3], double dt, const fdtd_coeffs* coeffs,
                void* stream, fdtd_handle** out) {
    if (!grid || !dx || !coeffs || !out) {
        set_error("fdtd_create: NULL argument");
        return FDTD_EINVAL;
    }
    *out = nullptr;
    const fdtd_grid& G = *grid;
    if (G.dims < 1 || G.dims > 3) { set_error("dims must be 1, 2 or 3"); return FDTD_EINVAL; }
    if (G.nx < 4 || G.nx % 4 != 0) { set_error("nx must be a positive multiple of 4"); return FDTD_EINVAL; }
    if (G.ny < 1 || G.nz < 1) { set_error("ny, nz must be >= 1"); return FDTD_EINVAL; }
    if (G.batched != 0 && G.batched != 1) { set_error("batched must be 0 or 1"); return FDTD_EINVAL; }
    if (G.batched && G.dims != 2) { set_error("batched needs dims == 2"); return FDTD_EINVAL; }
    if (G.dims <= 2 && G.nz != 1 && !G.batched) {
        set_error("dims < 3 needs nz == 1 (or batched = 1)");
        return FDTD_EINVAL;
    }
    if (G.dims == 1 && G.ny != 1) { set_error("dims == 1 needs ny == 1"); return FDTD_EINVAL; }
    if (G.dtype != FDTD_F32 && G.dtype != FDTD_F64) { set_error("bad dtype"); return FDTD_EINVAL; }
    if (G.absorb_cells < 0 || 2 * G.absorb_cells > G.ny ||
        (G.absorb_cells > 0 && !G.batched && 2 * G.absorb_cells > G.nz)) {
        set_error("absorbing layers do not fit the grid");
        return FDTD_EINVAL;
    }
    if (G.absorb_cells > 0 && !(G.absorb_sigma >= 0.0 && G.absorb_sigma < 1.0)) {
        set_error("absorb_sigma must be in [0, 1)");
        return FDTD_EINVAL;
    }
    for (int i = 0; i < 3; ++i)
        if (!(dx[i] > 0) || !std::isfinite(dx[i])) { set_error("dx must be positive"); return FDTD_EINVAL; }
    Clean cc = clean_coeffs(coeffs, G.dims);
    int rc = validate(cc, dx, G.dims, dt);
    if (rc) return rc;

    fdtd_handle* h = new (std::nothrow) fdtd_handle();
    if (!h) { set_error("host allocation failed"); return FDTD_ENOMEM; }
    h->grid = G;
    for (int i = 0; i < 3; ++i) h->dx[i] = dx[i];
    h->dt = dt;
    h->coeffs = *coeffs;
    h->cc = cc;
    h->stream = (cudaStream_t)stream;
    h->g = make_geom(G.nx, G.ny, G.nz);
    h->esz = G.dtype == FDTD_F32 ? 4 : 8;
    h->cur = 0;
    h->step = 0;
    h->use_fused = 1;
    const size_t arr = (size_t)h->g.total * h->esz;
    cudaError_t e = cudaMalloc(&h->state, 12 * arr);
    if (e == cudaSuccess) e = cudaMalloc(&h->aux, 2 * (size_t)(G.ny + G.nz) * h->esz);
    if (e != cudaSuccess) {
        set_error("cudaMalloc of %zu bytes failed: %s", 12 * arr, cudaGetErrorString(e));
        fdtd_destroy(h);
        return e == cudaErrorMemoryAllocation ? FDTD_ENOMEM : FDTD_ECUDA;
    }
    e = cudaMemsetAsync(h->state, 0, 12 * arr, h->stream);
    if (e != cudaSuccess) {
        set_error("cudaMemsetAsync failed: %s", cudaGetErrorString(e));
        fdtd_destroy(h);
        return FDTD_ECUDA;
    }
    rc = G.dtype == FDTD_F32 ? upload_aux<float>(h) : upload_aux<double>(h);
    if (rc) { fdtd_destroy(h); return rc; }
    e = cudaMalloc(&h->err_dev, sizeof(int));
    if (e == cudaSuccess) e = cudaMemsetAsync(h->err_dev, 0, sizeof(int), h->stream);
    if (e != cudaSuccess) {
        set_error("cudaMalloc failed: %s", cudaGetErrorString(e));
        fdtd_destroy(h);
        return FDTD_ECUDA;
    }
    // FDTD_FUSED=0 in the environment selects the reference-form kernels (same arithmetic).
    const char* env = getenv("FDTD_FUSED");
    h->use_fused = !(env && env[0] == '0');
    // FDTD_ADJOINT_SPLIT=1 selects the two-kernel FP32 reverse step (mu, then lambda_E, in place)
    const char* env_split = getenv("FDTD_ADJOINT_SPLIT");
    h->adj_split = env_split && env_split[0] == '1';
    if (h->use_fused) {
        if (G.dtype == FDTD_F32) {
            float* s0[6];
            float* s1[6];
            for (int c = 0; c < 6; ++c) { s0[c] = (float*)h->arr(0, c); s1[c] = (float*)h->arr(1, c); }
            h->plan = fused_plan_create<float>(h->g, s0, s1);
        } else {
            double* s0[6];
            double* s1[6];
            for (int c = 0; c < 6; ++c) { s0[c] = (double*)h->arr(0, c); s1[c] = (double*)h->arr(1, c); }
            h->plan = fused_plan_create<double>(h->g, s0, s1);
        }
    }
    *out = h;
    return FDTD_OK;
}

int fdtd_set_coeffs(fdtd_handle* h, double dt, const fdtd_coeffs* coeffs) {
    if (!h || !coeffs) { set_error("NULL argument"); return FDTD_EINVAL; }
    Clean cc = clean_coeffs(coeffs, h->grid.dims);
    int rc = validate(cc, h->dx, h->grid.dims, dt);
    if (rc) return rc;
    h->cc = cc;
    h->coeffs = *coeffs;
    h->dt = dt;
    return FDTD_OK;
}

static int ensure_xfer(fdtd_handle* h) {
    if (h->xfer) return FDTD_OK;
    CK(cudaStreamCreateWithFlags(&h->xfer, cudaStreamNonBlocking));
    for (int b = 0; b < 2; ++b) CK(cudaEventCreateWithFlags(&h->filled[b], cudaEventDisableTiming));
    return FDTD_OK;
}

// One 3D copy between a dense host array (nx, ny, nz) and the owned cells of a padded device
// array (x offset PX, y offset PY, row pitch nxp, nyp rows per plane)
template <typename T>
static cudaMemcpy3DParms owned_copy(const Geom& g, void* host, T* dev, bool to_device) {
    cudaMemcpy3DParms p = {};
    const cudaPitchedPtr hp = make_cudaPitchedPtr(host, (size_t)g.nx * sizeof(T), g.nx, g.ny);
    const cudaPitchedPtr dp = make_cudaPitchedPtr(dev, (size_t)g.nxp * sizeof(T), g.nxp, g.nyp);
    const cudaPos owned = make_cudaPos((size_t)PX * sizeof(T), PY, 0);
    if (to_device) {
        p.srcPtr = hp;
        p.dstPtr = dp;
        p.dstPos = owned;
        p.kind = cudaMemcpyHostToDevice;
    } else {
        p.srcPtr = dp;
        p.srcPos = owned;
        p.dstPtr = hp;
        p.kind = cudaMemcpyDeviceToHost;
    }
    p.extent = make_cudaExtent((size_t)g.nx * sizeof(T), g.ny, g.nz);
    return p;
}

// the copy stream starts after everything already queued on the handle's stream
static int xfer_after_stream(fdtd_handle* h) {
    CK(cudaEventRecord(h->filled[0], h->stream));
    CK(cudaStreamWaitEvent(h->xfer, h->filled[0], 0));
    return FDTD_OK;
}

// Host -> device: each component's owned cells are copied straight into the padded array on the
// copy stream (one 3D copy), then the periodic images are refreshed on the handle's stream.  A
// device source goes through the unpacking kernel (padded layout and images in one pass).
template <typename T>
static int copy_in(fdtd_handle* h, void* const fields[6], int32_t mem, T* const dst[6]) {
    if (mem == FDTD_MEM_HOST) {
        int rc = ensure_xfer(h);
        if (rc) return rc;
        rc = xfer_after_stream(h);   // the arrays may still be in use on the handle's stream
        if (rc) return rc;
        for (int c = 0; c < 6; ++c)
            if (fields && fields[c]) {
                const cudaMemcpy3DParms p = owned_copy<T>(h->g, fields[c], dst[c], true);
                CK(cudaMemcpy3DAsync(&p, h->xfer));
            }
        CK(cudaEventRecord(h->filled[1], h->xfer));
        CK(cudaStreamWaitEvent(h->stream, h->filled[1], 0));
    }
    for (int c = 0; c < 6; ++c) {
        const T* src = (const T*)(fields ? fields[c] : nullptr);
        if (src && mem == FDTD_MEM_HOST)
            launch_fill_ghosts<T>(h->g, dst[c], h->stream);
        else
            launch_unpack<T>(h->g, src, dst[c], h->stream);   // NULL source: zeros
        CK(cudaGetLastError());
    }
    if (mem == FDTD_MEM_HOST) CK(cudaStreamSynchronize(h->stream));
    return FDTD_OK;
}

// Device -> host: one 3D copy of each component's owned cells on the copy stream, after the
// work queued on the handle's stream; to device memory, the packing kernel.
template <typename T>
static int copy_out(fdtd_handle* h, void* const fields[6], int32_t mem, T* const srcs[6]) {
    if (mem == FDTD_MEM_HOST) {
        int rc = ensure_xfer(h);
        if (rc) return rc;
        rc = xfer_after_stream(h);
        if (rc) return rc;
        for (int c = 0; c < 6; ++c)
            if (fields[c]) {
                const cudaMemcpy3DParms p = owned_copy<T>(h->g, fields[c], srcs[c], false);
                CK(cudaMemcpy3DAsync(&p, h->xfer));
            }
        CK(cudaStreamSynchronize(h->xfer));
        return FDTD_OK;
    }
    for (int c = 0; c < 6; ++c) {
        if (!fields[c]) continue;
        launch_pack<T>(h->g, srcs[c], (T*)fields[c], h->stream);
        CK(cudaGetLastError());
    }
    return FDTD_OK;
}

int fdtd_set_state(fdtd_handle* h, void* const fields[6], int32_t mem, int64_t step0) {
    NvtxRange nvtx_range("fdtd_set_state");
    if (!h || (mem != FDTD_MEM_DEVICE && mem != FDTD_MEM_HOST)) {
        set_error("fdtd_set_state: bad argument");
        return FDTD_EINVAL;
    }
    h->cur = 0;
    h->step = step0;
    h->hist_len = 0;
    if (h->grid.dtype == FDTD_F32) {
        float* d[6];
        for (int c = 0; c < 6; ++c) d[c] = (float*)h->arr(0, c);
        return copy_in<float>(h, fields, mem, d);
    }
    double* d[6];
    for (int c = 0; c < 6; ++c) d[c] = (double*)h->arr(0, c);
    return copy_in<double>(h, fields, mem, d);
}

int fdtd_get_state(fdtd_handle* h, void* const fields[6], int32_t mem) {
    NvtxRange nvtx_range("fdtd_get_state");
    if (!h || !fields || (mem != FDTD_MEM_DEVICE && mem != FDTD_MEM_HOST)) {
        set_error("fdtd_get_state: bad argument");
        return FDTD_EINVAL;
    }
    if (h->grid.dtype == FDTD_F32) {
        float* s[6];
        for (int c = 0; c < 6; ++c) s[c] = (float*)h->arr(h->cur, c);
        return copy_out<float>(h, fields, mem, s);
    }
    double* s[6];
    for (int c = 0; c < 6; ++c) s[c] = (double*)h->arr(h->cur, c);
    return copy_out<double>(h, fields, mem, s);
}

int fdtd_get_step(fdtd_handle* h, int64_t* step) {
    if (!h || !step) { set_error("NULL argument"); return FDTD_EINVAL; }
    *step = h->step;
    return FDTD_OK;
}

static int ensure_lam(fdtd_handle* h) {
    if (h->lam) return FDTD_OK;
    const size_t arr = (size_t)h->g.total * h->esz;
    const bool fused = h->grid.dtype == FDTD_F32 && h->plan && !h->adj_split &&
                       adjoint32f_supported(h->g) && adjoint32f_prepare();
    h->lam_sets = fused ? 2 : 1;
    h->lam_cur = 0;
    CK(cudaMalloc(&h->lam, (size_t)h->lam_sets * 6 * arr));
    CK(cudaMemsetAsync(h->lam, 0, (size_t)h->lam_sets * 6 * arr, h->stream));
    h->lam_staged = false;
    h->lam_fused = false;
    if (fused) {
        bool ok = true;
        for (int s = 0; s < 2; ++s)
            for (int c = 0; c < 3; ++c)
                ok = ok && encode_ebox_f32(&h->lam_emaps[s].e[c], h->g, (float*)h->lam_arr_set(s, c)) &&
                     encode_box_f32(&h->lam_emaps[s].b[c], h->g, (float*)h->lam_arr_set(s, 3 + c), 72, 11);
        h->lam_fused = ok;   // otherwise the two-kernel reverse step runs on set 0
    }
    if (!h->lam_fused && h->grid.dtype == FDTD_F32 && h->plan && adjoint32e_supported(h->g) &&
        adjoint32e_prepare()) {
        bool ok = true;
        for (int c = 0; c < 3; ++c)
            ok = ok && encode_ebox_f32(&h->lam_maps.e[c], h->g, (float*)h->lam_arr(3 + c));
        h->lam_staged = ok;   // otherwise the reference-form adjoint E kernel runs
    }
    return FDTD_OK;
}

int fdtd_set_adjoint(fdtd_handle* h, void* const fields[6], int32_t mem) {
    NvtxRange nvtx_range("fdtd_set_adjoint");
    if (!h || (mem != FDTD_MEM_DEVICE && mem != FDTD_MEM_HOST)) {
        set_error("fdtd_set_adjoint: bad argument");
        return FDTD_EINVAL;
    }
    int rc = ensure_lam(h);
    if (rc) return rc;
    if (h->grid.dtype == FDTD_F32) {
        float* d[6];
        for (int c = 0; c < 6; ++c) d[c] = (float*)h->lam_arr(c);
        return copy_in<float>(h, fields, mem, d);
    }
    double* d[6];
    for (int c = 0; c < 6; ++c) d[c] = (double*)h->lam_arr(c);
    return copy_in<double>(h, fields, mem, d);
}

int fdtd_get_adjoint(fdtd_handle* h, void* const fields[6], int32_t mem) {
    NvtxRange nvtx_range("fdtd_get_adjoint");
    if (!h || !fields || (mem != FDTD_MEM_DEVICE && mem != FDTD_MEM_HOST)) {
        set_error("fdtd_get_adjoint: bad argument");
        return FDTD_EINVAL;
    }
    int rc = ensure_lam(h);
    if (rc) return rc;
    if (h->grid.dtype == FDTD_F32) {
        float* s[6];
        for (int c = 0; c < 6; ++c) s[c] = (float*)h->lam_arr(c);
        return copy_out<float>(h, fields, mem, s);
    }
    double* s[6];
    for (int c = 0; c < 6; ++c) s[c] = (double*)h->lam_arr(c);
    return copy_out<double>(h, fields, mem, s);
}

static int ensure_hist(fdtd_handle* h, int snaps) {
    if (h->hist_cap >= snaps) return FDTD_OK;
    if (h->hist) { cudaFree(h->hist); h->hist = nullptr; h->hist_cap = 0; }
    h->hist_maps.clear();
    const size_t arr = (size_t)h->g.total * h->esz;
    CK(cudaMalloc(&h->hist, (size_t)snaps * 3 * arr));
    h->hist_cap = snaps;
    if (h->grid.dtype == FDTD_F32 && h->plan && adjoint32_supported(h->g) && adjoint32_prepare()) {
        h->hist_maps.resize(snaps);
        for (int s = 0; s < snaps; ++s)
            for (int c = 0; c < 3; ++c)
                if (!encode_ebox_f32(&h->hist_maps[s].e[c], h->g, (float*)h->hist_arr(s, c))) {
                    h->hist_maps.clear();
                    return FDTD_OK;   // the reference-form adjoint kernels will be used
                }
    }
    return FDTD_OK;
}

static int ensure_jx(fdtd_handle* h, int n) {
    if (h->jx_cap >= n) return FDTD_OK;
    if (h->jx) { cudaFree(h->jx); h->jx = nullptr; h->jx_cap = 0; }
    CK(cudaMalloc(&h->jx, (size_t)n * h->g.nx * h->esz));
    h->jx_cap = n;
    return FDTD_OK;
}

template <typename T>
static int snapshot(fdtd_handle* h, int snap) {
    const size_t arr = (size_t)h->g.total * sizeof(T);
    for (int c = 0; c < 3; ++c)
        CK(cudaMemcpyAsync(h->hist_arr(snap, c), h->arr(h->cur, c), arr, cudaMemcpyDeviceToDevice,
                           h->stream));
    return FDTD_OK;
}

// Two leapfrog steps, temporally blocked through L2 (FP32 fused path, no current, probe or
// history).  The z axis is cut into S slabs [b_s, b_{s+1}) of at least 3 planes.  With A the
// current state set and B the other one, step 1 (A -> B) and step 2 (B -> A) run slab by slab,
// step 2 trailing one slab behind step 1:
//     1(0) 1(1)  | 1(2) 2(1) | 1(3) 2(2) | ... | 1(S-1) 2(S-2) |  2(S-1) 2(0)
// so that step 2 of slab s reads the intermediate state (E^{n+1}, B^{n+1/2}) of slabs s-1 .. s+1
// shortly after step 1 wrote it, from L2 rather than DRAM.  Ordering (every slab >= 3 planes):
// step 2 of slab s needs B planes b_s - 2 .. b_{s+1} + 1, written by step 1 of slabs s-1 .. s+1;
// step 2 of slab s overwrites the A planes of slab s, which step 1 of slab s+1 (launched just
// before) still reads (down to b_{s+1} - 2) and step 1 of slabs >= s+2 never reads; step 1 of
// slab 0 reads the A planes nz-2, nz-1 and step 1 of slab S-1 the A planes 0, 1 before step 2
// of those slabs runs (2(0) comes last).  Intermediate planes that no later step-2 launch reads
// are dropped from L2 without being written back (launch_discard_planes), so the pair moves
// the state through DRAM about once in each direction instead of twice; set B holds undefined
// values afterwards (nothing reads it before the next step overwrites it).
static int step_pair_blocked(fdtd_handle* h, const Mult<float>& m, const float* spy,
                             const float* spz) {
    const Geom& g = h->g;
    const int S = g.nz / h->tslab;
    const int A = h->cur, B = 1 - h->cur;
    FieldSet<float> fa = fieldset<float>(h, A), fb = fieldset<float>(h, B);
    void* bset[6];
    for (int c = 0; c < 6; ++c) bset[c] = fb.c[c];
    auto b = [&](int s) { return (int)((long long)s * g.nz / S); };
    auto step1 = [&](int s) {
        launch_step_fused32_range(h->plan, A, g, m, fa, fb, spy, spz, b(s), b(s + 1), h->err_dev,
                                  h->stream);
    };
    auto step2 = [&](int s) {
        launch_step_fused32_range(h->plan, B, g, m, fb, fa, spy, spz, b(s), b(s + 1), h->err_dev,
                                  h->stream);
    };
    // B planes still needed by step 2 of slab 0: nz-2, nz-1, 0 .. b_1 + 1; the rest of the
    // intermediate state is dropped as soon as step 2 has passed it
    int dropped = b(1) + 2;
    auto drop_to = [&](int hi) {
        if (hi > dropped) {
            launch_discard_planes(g, sizeof(float), bset, dropped, hi, h->stream);
            dropped = hi;
        }
    };
    step1(0);
    step1(1);
    for (int s = 1; s + 1 < S; ++s) {
        step1(s + 1);
        step2(s);
        drop_to(b(s + 1) - 2);   // step 2 of slab s+1 reads from b_{s+1} - 2 on
    }
    step2(S - 1);
    step2(0);
    drop_to(g.nz);
    launch_discard_planes(g, sizeof(float), bset, 0, b(1) + 2 < g.nz ? b(1) + 2 : g.nz, h->stream);
    CK(cudaGetLastError());
    h->step += 2;
    return FDTD_OK;
}

template <typename T>
static int step_impl(fdtd_handle* h, int n, const fdtd_source* src, const fdtd_probe* probe,
                     double* loss, int record) {
    const Geom& g = h->g;
    const Mult<T> m = make_mult<T>(h->cc, h->dx, h->dt, !h->grid.batched);
    const T* spy = nullptr;
    const T* spz = nullptr;
    if (h->grid.absorb_cells > 0) {
        spy = (const T*)h->aux;
        spz = spy + g.ny;
    }
    const bool bunch = src && src->kind == FDTD_SRC_BUNCH && n > 0;
    const bool dense = src && src->kind == FDTD_SRC_DENSE && n > 0;
    const T* jyz = nullptr;
    if (bunch) {
        int rc = upload_bunch_yz<T>(h, src);
        if (rc) return rc;
        rc = ensure_jx(h, n);
        if (rc) return rc;
        jyz = (const T*)h->aux + (g.ny + g.nz);
        launch_bunch_table<T>(g.nx, n, src->x0, src->v * h->dt, 1.0 / src->sigma_par,
                              src->q / (h->dx[1] * h->dx[2] * h->dt), h->dx[0], g.nx * h->dx[0],
                              h->step, (T*)h->jx, h->stream);
        CK(cudaGetLastError());
    }
    if (record) {
        int rc = ensure_hist(h, n + 1);
        if (rc) return rc;
        h->hist_len = n + 1;
        h->hist_step0 = h->step;
    }
    const bool fused = h->plan != nullptr;
    if constexpr (std::is_same<T, float>::value) {
        // temporally blocked pairs: FP32 fused path, no current, probe or history, >= 2 slabs
        if (h->tblock == 2 && fused && !bunch && !dense && !probe && !record &&
            g.nz / h->tslab >= 2) {
            for (; n >= 2; n -= 2) {
                int rc = step_pair_blocked(h, m, spy, spz);
                if (rc) return rc;
            }
        }
    }
    for (int s = 0; s < n; ++s) {
        if (record && !fused) {
            int rc = snapshot<T>(h, s);
            if (rc) return rc;
        }
        const T* jrow = bunch ? (const T*)h->jx + (size_t)s * g.nx : nullptr;
        if (fused) {
            T* hE[3] = {nullptr, nullptr, nullptr};
            if (record) {
                if (s == 0) {
                    int rc = snapshot<T>(h, 0);
                    if (rc) return rc;
                }
                for (int c = 0; c < 3; ++c) hE[c] = (T*)h->hist_arr(s + 1, c);
            }
            launch_step_fused<T>(h->plan, h->cur, g, m, fieldset<T>(h, h->cur),
                                 fieldset<T>(h, 1 - h->cur), spy, spz, jyz, jrow, hE, h->err_dev,
                                 h->stream);
            h->cur = 1 - h->cur;
        } else {
            FieldSet<T> fs = fieldset<T>(h, h->cur);
            launch_faraday_v0<T>(g, m, fs, spy, spz, h->stream);
            launch_ampere_v0<T>(g, m, fs, spy, spz, jyz, jrow, h->err_dev, h->stream);
        }
        CK(cudaGetLastError());
        if (dense) {
            // Ampere's law is linear in J: E^{n+1} = (E^{n+1} without J) - dt J
            FieldSet<T> now = fieldset<T>(h, h->cur);
            T* E[3] = {now.c[0], now.c[1], now.c[2]};
            const T* J[3] = {(const T*)src->J[0], (const T*)src->J[1], (const T*)src->J[2]};
            launch_current<T>(g, E, J, (T)h->dt, spy, spz, h->stream);
            CK(cudaGetLastError());
            launch_refresh_images<T>(g, E[0], E[1], E[2], h->stream);
            CK(cudaGetLastError());
            // the fused kernel wrote this step's history snapshot before the current was added
            if (record && fused) {
                int rc = snapshot<T>(h, s + 1);
                if (rc) return rc;
            }
        }
        h->step += 1;
        if (probe) {
            const T* tgt = (const T*)probe->target + (size_t)(h->step - 1) * g.ny * g.nz;
            launch_probe_loss<T>(g, (const T*)h->arr(h->cur, probe->component), probe->x_index,
                                 tgt, loss, h->stream);
            CK(cudaGetLastError());
        }
    }
    if (record && !fused) {
        int rc = snapshot<T>(h, n);
        if (rc) return rc;
    }
    if (record && fused && n == 0) {
        int rc = snapshot<T>(h, 0);
        if (rc) return rc;
    }
    return FDTD_OK;
}

int fdtd_step(fdtd_handle* h, int32_t n, const fdtd_source* src, const fdtd_probe* probe,
              double* loss_dev, int32_t record) {
    NvtxRange nvtx_range("fdtd_step");
    if (!h || n < 0) { set_error("fdtd_step: bad argument"); return FDTD_EINVAL; }
    if (src && src->kind != FDTD_SRC_NONE && src->kind != FDTD_SRC_BUNCH &&
        src->kind != FDTD_SRC_DENSE) {
        set_error("unknown source kind %d", src->kind);
        return FDTD_EINVAL;
    }
    if (src && src->kind == FDTD_SRC_BUNCH && h->grid.batched) {
        set_error("the bunch source is not defined for batched 2D problems");
        return FDTD_EINVAL;
    }
    if (src && src->kind == FDTD_SRC_BUNCH && !(src->sigma_par > 0 && src->sigma_perp > 0)) {
        set_error("bunch widths must be positive");
        return FDTD_EINVAL;
    }
    if (probe) {
        if (probe->component < 0 || probe->component > 2 || probe->x_index < 0 ||
            probe->x_index >= h->g.nx || !probe->target || !loss_dev) {
            set_error("bad probe");
            return FDTD_EINVAL;
        }
        if (h->step + n > probe->target_steps) {
            set_error("probe target holds %lld steps, run needs %lld",
                      (long long)probe->target_steps, (long long)(h->step + n));
            return FDTD_EINVAL;
        }
    }
    if (h->grid.dtype == FDTD_F32) return step_impl<float>(h, n, src, probe, loss_dev, record);
    return step_impl<double>(h, n, src, probe, loss_dev, record);
}

int fdtd_checkpoint(fdtd_handle* h, int32_t slot, int32_t op) {
    NvtxRange nvtx_range("fdtd_checkpoint");
    if (!h || slot < 0 || (op != 0 && op != 1)) { set_error("fdtd_checkpoint: bad argument"); return FDTD_EINVAL; }
    const size_t arr = (size_t)h->g.total * h->esz;
    if ((size_t)slot >= h->ckpt.size()) {
        if (op == 1) { set_error("checkpoint slot %d is empty", slot); return FDTD_ESTATE; }
        h->ckpt.resize(slot + 1, nullptr);
        h->ckpt_step.resize(slot + 1, -1);
    }
    if (op == 0) {
        if (!h->ckpt[slot]) CK(cudaMalloc(&h->ckpt[slot], 6 * arr));
        for (int c = 0; c < 6; ++c)
            CK(cudaMemcpyAsync(h->ckpt[slot] + c * arr, h->arr(h->cur, c), arr,
                               cudaMemcpyDeviceToDevice, h->stream));
        h->ckpt_step[slot] = h->step;
    } else {
        if (!h->ckpt[slot]) { set_error("checkpoint slot %d is empty", slot); return FDTD_ESTATE; }
        for (int c = 0; c < 6; ++c)
            CK(cudaMemcpyAsync(h->arr(h->cur, c), h->ckpt[slot] + c * arr, arr,
                               cudaMemcpyDeviceToDevice, h->stream));
        h->step = h->ckpt_step[slot];
        h->hist_len = 0;
    }
    return FDTD_OK;
}

template <typename T>
static int adjoint_impl(fdtd_handle* h, int n, const fdtd_probe* probe, double* grad) {
    const Geom& g = h->g;
    const Mult<T> m = make_mult<T>(h->cc, h->dx, h->dt, !h->grid.batched);
    const T* spy = nullptr;
    const T* spz = nullptr;
    if (h->grid.absorb_cells > 0) {
        spy = (const T*)h->aux;
        spz = spy + g.ny;
    }
    int rc = ensure_lam(h);
    if (rc) return rc;
    const bool staged = std::is_same<T, float>::value && !h->hist_maps.empty();
    const bool one_kernel = staged && h->lam_fused;
    const int nblk = one_kernel ? adjoint32f_blocks(g) : staged ? adjoint32_blocks(g) : adjoint_B_blocks(g);
    if (h->npart < nblk) {
        if (h->partials) cudaFree(h->partials);
        h->partials = nullptr;
        CK(cudaMalloc(&h->partials, (size_t)nblk * 9 * sizeof(double)));
        h->npart = nblk;
    }
    CK(cudaMemsetAsync(h->partials, 0, (size_t)nblk * 9 * sizeof(double), h->stream));
    const int top = h->hist_len - 1;   // newest snapshot index
    for (int r = 0; r < n; ++r) {
        FieldSet<T> lam = lamset<T>(h);
        const int snap_after = top - r;        // E^{s+1}
        const int snap_before = top - r - 1;   // E^{s}
        const long long s_after = h->hist_step0 + snap_after;
        if (probe) {
            const T* tgt = (const T*)probe->target + (size_t)(s_after - 1) * g.ny * g.nz;
            launch_probe_adjoint<T>(g, lam.c[probe->component],
                                    (const T*)h->hist_arr(snap_after, probe->component),
                                    probe->x_index, tgt, h->stream);
        }
        const T* E[3] = {(const T*)h->hist_arr(snap_before, 0), (const T*)h->hist_arr(snap_before, 1),
                         (const T*)h->hist_arr(snap_before, 2)};
        if constexpr (std::is_same<T, float>::value) {
            if (one_kernel) {   // lambda^{s+1} (set lam_cur) -> lambda^s (the other set)
                FieldSet<float> nxt;
                for (int c = 0; c < 6; ++c) nxt.c[c] = (float*)h->lam_arr_set(h->lam_cur ^ 1, c);
                launch_adjoint32_fused(h->lam_emaps[h->lam_cur], g, m, lam, nxt, E, spy, spz,
                                       h->partials, h->err_dev, h->stream);
                CK(cudaGetLastError());
                h->lam_cur ^= 1;
                continue;
            }
        }
        if constexpr (std::is_same<T, float>::value) {
            if (staged)
                launch_adjoint32_B(h->hist_maps[snap_before], g, m, lam, spy, spz, h->partials,
                                   h->err_dev, h->stream);
            else
                launch_adjoint_B_v0<T>(g, m, lam, E, spy, spz, h->partials, nblk, h->stream);
        } else {
            launch_adjoint_B_v0<T>(g, m, lam, E, spy, spz, h->partials, nblk, h->stream);
        }
        if constexpr (std::is_same<T, float>::value) {
            if (staged && h->lam_staged)
                launch_adjoint32_E(h->lam_maps, g, m, lam, spy, spz, h->err_dev, h->stream);
            else
                launch_adjoint_E_v0<T>(g, m, lam, spy, spz, h->stream);
        } else {
            launch_adjoint_E_v0<T>(g, m, lam, spy, spz, h->stream);
        }
        CK(cudaGetLastError());
    }
    // scale of each partial: dt/dx_a, zero for entries that refer to an absent axis
    // (their brackets may mix independent batched problems)
    GradScale sc;
    const int dims = h->grid.dims;
    for (int a = 0; a < 3; ++a) {
        const int b1 = a == 0 ? 1 : 0, b2 = a == 2 ? 1 : 2;
        const double s_a = a < dims ? h->dt / h->dx[a] : 0.0;
        sc.s[3 * a + 0] = s_a;
        sc.s[3 * a + 1] = b1 < dims ? s_a : 0.0;
        sc.s[3 * a + 2] = b2 < dims ? s_a : 0.0;
    }
    launch_reduce_grad(h->partials, nblk, sc, grad, h->stream);
    CK(cudaGetLastError());
    h->hist_len -= n;
    return FDTD_OK;
}

int fdtd_step_adjoint(fdtd_handle* h, int32_t n, const fdtd_probe* probe, double* grad_dev) {
    NvtxRange nvtx_range("fdtd_step_adjoint");
    if (!h || n < 0 || !grad_dev) { set_error("fdtd_step_adjoint: bad argument"); return FDTD_EINVAL; }
    if (h->hist_len < n + 1) {
        set_error("history holds %d snapshots, %d reverse steps need %d", h->hist_len, n, n + 1);
        return FDTD_ESTATE;
    }
    if (probe) {
        if (probe->component < 0 || probe->component > 2 || probe->x_index < 0 ||
            probe->x_index >= h->g.nx || !probe->target) {
            set_error("bad probe");
            return FDTD_EINVAL;
        }
        if (h->hist_step0 + h->hist_len - 1 > probe->target_steps) {
            set_error("probe target too short");
            return FDTD_EINVAL;
        }
    }
    if (h->grid.dtype == FDTD_F32) return adjoint_impl<float>(h, n, probe, grad_dev);
    return adjoint_impl<double>(h, n, probe, grad_dev);
}

static int ensure_dpart(fdtd_handle* h) {
    if (h->dpart) return FDTD_OK;
    CK(cudaMalloc(&h->dpart, (size_t)diag_blocks(h->g) * 3 * sizeof(double)));
    return FDTD_OK;
}

int fdtd_diagnostic(fdtd_handle* h, int32_t kind, const double* params, double* out_dev) {
    NvtxRange nvtx_range("fdtd_diagnostic");
    if (!h || !params || !out_dev) { set_error("fdtd_diagnostic: NULL argument"); return FDTD_EINVAL; }
    int rc = ensure_dpart(h);
    if (rc) return rc;
    const Geom& g = h->g;
    const bool f32 = h->grid.dtype == FDTD_F32;
    if (kind == FDTD_DIAG_ENERGY) {
        const int x_lo = (int)params[0], x_len = (int)params[1], margin = (int)params[2];
        // the margin trims y always and z when z is a spatial axis (nz > 1, not batched)
        const int my = margin, mz = (g.nz > 1 && !h->grid.batched) ? margin : 0;
        if (x_len < 1 || x_len > g.nx || margin < 0 || 2 * my >= g.ny || 2 * mz >= g.nz) {
            set_error("fdtd_diagnostic: bad energy window");
            return FDTD_EINVAL;
        }
        const double dV = h->dx[0] * h->dx[1] * h->dx[2];
        if (f32) launch_energy<float>(g, fieldset<float>(h, h->cur), x_lo, x_len, my, mz, dV, h->dpart, out_dev, h->stream);
        else launch_energy<double>(g, fieldset<double>(h, h->cur), x_lo, x_len, my, mz, dV, h->dpart, out_dev, h->stream);
    } else if (kind == FDTD_DIAG_PLANEWAVE) {
        const int comp = (int)params[0];
        if (comp < 0 || comp > 5) { set_error("fdtd_diagnostic: component must be 0..5"); return FDTD_EINVAL; }
        static const double offs[6][3] = {{0.5, 0, 0}, {0, 0.5, 0}, {0, 0, 0.5},
                                          {0, 0.5, 0.5}, {0.5, 0, 0.5}, {0.5, 0.5, 0}};
        const double kd[3] = {params[1] * h->dx[0], params[2] * h->dx[1], params[3] * h->dx[2]};
        if (f32) launch_planewave<float>(g, (const float*)h->arr(h->cur, comp), kd, offs[comp], h->dpart, out_dev, h->stream);
        else launch_planewave<double>(g, (const double*)h->arr(h->cur, comp), kd, offs[comp], h->dpart, out_dev, h->stream);
    } else if (kind == FDTD_DIAG_MOMENTS) {
        const int axis = (int)params[0];
        if (axis < 0 || axis > 2) { set_error("fdtd_diagnostic: axis must be 0..2"); return FDTD_EINVAL; }
        const double dV = h->dx[0] * h->dx[1] * h->dx[2];
        if (f32) launch_moments<float>(g, fieldset<float>(h, h->cur), axis, dV, h->dpart, out_dev, h->stream);
        else launch_moments<double>(g, fieldset<double>(h, h->cur), axis, dV, h->dpart, out_dev, h->stream);
    } else {
        set_error("fdtd_diagnostic: unknown kind %d", kind);
        return FDTD_EINVAL;
    }
    CK(cudaGetLastError());
    return FDTD_OK;
}

int fdtd_divergence(fdtd_handle* h, int32_t which, double* out_dev) {
    NvtxRange nvtx_range("fdtd_divergence");
    if (!h || !out_dev || which < 0 || which > 2) {
        set_error("fdtd_divergence: bad argument");
        return FDTD_EINVAL;
    }
    // multipliers of the difference operators themselves (1/dx_a, not dt/dx_a)
    const Mult<double> w = make_mult<double>(h->cc, h->dx, 1.0, !h->grid.batched);
    if (h->grid.dtype == FDTD_F32) launch_divergence<float>(h->g, w, fieldset<float>(h, h->cur), which, out_dev, h->stream);
    else launch_divergence<double>(h->g, w, fieldset<double>(h, h->cur), which, out_dev, h->stream);
    CK(cudaGetLastError());
    return FDTD_OK;
}

// One thread waits, with the kernels' bounded-wait helper, on an mbarrier phase that no
// copy and no thread will ever complete; when its polls run out it raises the handle's error
// flag exactly as an expired wait in a step kernel does, and returns.
__global__ void wait_expiry_kernel(uint32_t tries, int* err) {
    __shared__ uint64_t bar;
    if (threadIdx.x == 0) {
        mbar_init(&bar, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        if (!mbar_wait_n(&bar, 0, tries)) atomicOr(err, ERR_WAIT);
        asm volatile("mbarrier.inval.shared::cta.b64 [%0];" ::"r"(smem_u32(&bar)) : "memory");
    }
}

int fdtd_set_temporal_blocking(fdtd_handle* h, int32_t T, int32_t slab_planes) {
    if (!h || (T != 1 && T != 2) || slab_planes < 0 || (slab_planes > 0 && slab_planes < 3)) {
        set_error("fdtd_set_temporal_blocking: T must be 1 or 2 and slab_planes 0 or >= 3");
        return FDTD_EINVAL;
    }
    h->tblock = T;
    h->tslab = slab_planes > 0 ? slab_planes : 32;
    return FDTD_OK;
}

int fdtd_selftest_wait_expiry(fdtd_handle* h, int32_t tries) {
    if (!h || tries < 1 || tries > (1 << 20)) {
        set_error("fdtd_selftest_wait_expiry: bad argument");
        return FDTD_EINVAL;
    }
    wait_expiry_kernel<<<1, 32, 0, h->stream>>>((uint32_t)tries, h->err_dev);
    CK(cudaGetLastError());
    return FDTD_OK;
}

int fdtd_sync(fdtd_handle* h) {
    if (!h) { set_error("NULL handle"); return FDTD_EINVAL; }
    CK(cudaStreamSynchronize(h->stream));
    CK(cudaGetLastError());
    int flag = 0;
    CK(cudaMemcpy(&flag, h->err_dev, sizeof(int), cudaMemcpyDeviceToHost));
    if (flag) {
        cudaMemset(h->err_dev, 0, sizeof(int));
        if (flag & ERR_WAIT) {
            set_error("a bounded wait inside a step kernel expired; the state is not valid");
            return FDTD_ETIMEOUT;
        }
        if (flag & ERR_FIELD) {
            set_error("a step wrote a non-finite field value (the fields blew up, or the state or "
                      "the current held an infinity or NaN)");
            return FDTD_ENONFINITE;
        }
        set_error("a particle position or momentum was not finite; such particles were left "
                  "unchanged and deposited nothing");
        return FDTD_ENONFINITE;
    }
    return FDTD_OK;
}

// ---- macro-particles (PIC cycle) --------------------------------------------------------

static int check_species(const fdtd_handle* h, const fdtd_species* sp, int32_t nsp,
                         const char* who) {
    if (nsp < 0 || (nsp > 0 && !sp)) {
        set_error("%s: bad species list", who);
        return FDTD_EINVAL;
    }
    if (h->grid.dims != 3 || h->grid.batched) {
        set_error("%s: particles need a 3D grid (dims = 3, not batched)", who);
        return FDTD_EINVAL;
    }
    for (int s = 0; s < nsp; ++s) {
        if (sp[s].n < 0) { set_error("%s: species %d has a negative count", who, s); return FDTD_EINVAL; }
        if (sp[s].n == 0) continue;
        for (int a = 0; a < 3; ++a)
            if (!sp[s].x[a] || !sp[s].u[a]) {
                set_error("%s: species %d has a NULL array", who, s);
                return FDTD_EINVAL;
            }
        if (!std::isfinite(sp[s].q) || !std::isfinite(sp[s].q_over_m)) {
            set_error("%s: species %d has a non-finite charge or charge-to-mass ratio", who, s);
            return FDTD_EINVAL;
        }
    }
    return FDTD_OK;
}

template <typename T>
static int pic_impl(fdtd_handle* h, int n, const fdtd_species* sp, int nsp) {
    const Geom& g = h->g;
    const Mult<T> m = make_mult<T>(h->cc, h->dx, h->dt, true);
    const T* spy = nullptr;
    const T* spz = nullptr;
    if (h->grid.absorb_cells > 0) {
        spy = (const T*)h->aux;
        spz = spy + g.ny;
    }
    h->hist_len = 0;   // a PIC cycle has no recorded adjoint
    for (int s = 0; s < n; ++s) {
        FieldSet<T> cur = fieldset<T>(h, h->cur), nxt = fieldset<T>(h, 1 - h->cur);
        // (E^{n+1} without the current, B^{n+1/2}) into the other set: Ampere's law is linear
        // in J, so the particles add -dt J^{n+1/2} to E^{n+1} afterwards
        if (h->plan) {
            T* hE[3] = {nullptr, nullptr, nullptr};
            launch_step_fused<T>(h->plan, h->cur, g, m, cur, nxt, spy, spz, nullptr, nullptr, hE,
                                 h->err_dev, h->stream);
        } else {
            launch_faraday_oop<T>(g, m, cur, nxt, spy, spz, h->stream);
            CK(cudaGetLastError());
            launch_ampere_current<T>(g, m, cur, nxt, nullptr, nxt, spy, spz, h->err_dev, h->stream);
        }
        CK(cudaGetLastError());
        for (int q = 0; q < nsp; ++q) {
            if (sp[q].n == 0) continue;
            PushArgs<T> a;
            a.g = g;
            for (int c = 0; c < 3; ++c) {
                const int b = c == 0 ? 1 : 0, d = c == 2 ? 1 : 2;
                a.E[c] = cur.c[c];
                a.B0[c] = cur.c[3 + c];
                a.B1[c] = nxt.c[3 + c];
                a.Eout[c] = nxt.c[c];
                a.x[c] = (T*)sp[q].x[c];
                a.u[c] = (T*)sp[q].u[c];
                a.inv_dx[c] = (T)(1.0 / h->dx[c]);
                a.escale[c] = (T)(sp[q].q / (h->dx[b] * h->dx[d]));
            }
            a.spy = spy;
            a.spz = spz;
            a.L[0] = (T)(g.nx * h->dx[0]);
            a.L[1] = (T)(g.ny * h->dx[1]);
            a.L[2] = (T)(g.nz * h->dx[2]);
            a.n = sp[q].n;
            a.h = (T)(0.5 * sp[q].q_over_m * h->dt);
            a.dt = (T)h->dt;
            a.err = h->err_dev;
            launch_pic_push<T>(a, h->stream);
            CK(cudaGetLastError());
        }
        launch_refresh_images<T>(g, nxt.c[0], nxt.c[1], nxt.c[2], h->stream);
        CK(cudaGetLastError());
        h->cur = 1 - h->cur;
        h->step += 1;
    }
    return FDTD_OK;
}

int fdtd_pic_step(fdtd_handle* h, int32_t n, const fdtd_species* species, int32_t nspecies) {
    NvtxRange nvtx_range("fdtd_pic_step");
    if (!h || n < 0) { set_error("fdtd_pic_step: bad argument"); return FDTD_EINVAL; }
    int rc = check_species(h, species, nspecies, "fdtd_pic_step");
    if (rc) return rc;
    if (h->grid.dtype == FDTD_F32) return pic_impl<float>(h, n, species, nspecies);
    return pic_impl<double>(h, n, species, nspecies);
}

template <typename T>
static int rho_impl(fdtd_handle* h, const fdtd_species* sp, int nsp, T* rho) {
    const T inv_dx[3] = {(T)(1.0 / h->dx[0]), (T)(1.0 / h->dx[1]), (T)(1.0 / h->dx[2])};
    const T L[3] = {(T)(h->g.nx * h->dx[0]), (T)(h->g.ny * h->dx[1]), (T)(h->g.nz * h->dx[2])};
    const double vol = h->dx[0] * h->dx[1] * h->dx[2];
    for (int q = 0; q < nsp; ++q) {
        if (sp[q].n == 0) continue;
        const T* x[3] = {(const T*)sp[q].x[0], (const T*)sp[q].x[1], (const T*)sp[q].x[2]};
        launch_deposit_rho<T>(h->g, x, sp[q].n, inv_dx, L, (T)(sp[q].q / vol), rho, h->err_dev,
                              h->stream);
        CK(cudaGetLastError());
    }
    return FDTD_OK;
}

int fdtd_deposit_rho(fdtd_handle* h, const fdtd_species* species, int32_t nspecies,
                     void* rho_dev) {
    NvtxRange nvtx_range("fdtd_deposit_rho");
    if (!h || !rho_dev) { set_error("fdtd_deposit_rho: bad argument"); return FDTD_EINVAL; }
    int rc = check_species(h, species, nspecies, "fdtd_deposit_rho");
    if (rc) return rc;
    if (h->grid.dtype == FDTD_F32) return rho_impl<float>(h, species, nspecies, (float*)rho_dev);
    return rho_impl<double>(h, species, nspecies, (double*)rho_dev);
}

void fdtd_destroy(fdtd_handle* h) {
    if (!h) return;
    cudaStreamSynchronize(h->stream);
    if (h->state) cudaFree(h->state);
    if (h->lam) cudaFree(h->lam);
    if (h->hist) cudaFree(h->hist);
    if (h->aux) cudaFree(h->aux);
    if (h->jx) cudaFree(h->jx);
    if (h->partials) cudaFree(h->partials);
    if (h->xfer) {
        cudaStreamSynchronize(h->xfer);
        for (int b = 0; b < 2; ++b) cudaEventDestroy(h->filled[b]);
        cudaStreamDestroy(h->xfer);
    }
    if (h->err_dev) cudaFree(h->err_dev);
    if (h->dpart) cudaFree(h->dpart);
    if (h->plan) fused_plan_destroy(h->plan);
    for (char* p : h->ckpt)
        if (p) cudaFree(p);
    delete h;
}

int disp_norm_eval(const fdtd_coeffs* coeffs, double dt, const double dx[3], int32_t dims,
                   const int32_t N[3], int32_t weight, double weight_param, double* out,
                   void* stream) {
    NvtxRange nvtx_range("disp_norm_eval");
    if (!coeffs || !dx || !N || !out || dims < 1 || dims > 3) {
        set_error("disp_norm_eval: bad argument");
        return FDTD_EINVAL;
    }
    for (int i = 0; i < dims; ++i)
        if (N[i] < 1 || !(dx[i] > 0)) { set_error("disp_norm_eval: bad grid"); return FDTD_EINVAL; }
    if (weight != FDTD_W_UNIFORM && weight != FDTD_W_CONE_X && weight != FDTD_W_GAUSS_Y) {
        set_error("unknown weight %d", weight);
        return FDTD_EINVAL;
    }
    if (weight == FDTD_W_GAUSS_Y && !(weight_param > 0)) { set_error("gauss width must be > 0"); return FDTD_EINVAL; }
    Clean cc = clean_coeffs(coeffs, dims);
    int rc = validate(cc, dx, dims, dt);
    if (rc) return rc;
    cudaStream_t st = (cudaStream_t)stream;
    int Nd[3];
    long long npts = 1;
    for (int i = 0; i < 3; ++i) {
        Nd[i] = i < dims ? N[i] : 1;
        npts *= Nd[i];
    }
    const size_t nscr = norm_scratch_doubles(Nd, npts);
    double* scratch = nullptr;
    CK(cudaMallocAsync((void**)&scratch, nscr * sizeof(double), st));
    double* res = nullptr;
    launch_disp_norm(cc.alpha, cc.beta, cc.delta, dt, dx, dims, Nd, weight, weight_param, scratch,
                     &res, st);
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaMemcpyAsync(out, res, 14 * sizeof(double), cudaMemcpyDeviceToHost, st);
    cudaFreeAsync(scratch, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) {
        set_error("disp_norm_eval: %s", cudaGetErrorString(e));
        return FDTD_ECUDA;
    }
    return FDTD_OK;
}


int disp_group_norm_eval(const fdtd_coeffs* coeffs, double dt, const double dx[3], int32_t dims,
                         const int32_t N[3], int32_t weight, double weight_param, double* out,
                         void* stream) {
    NvtxRange nvtx_range("disp_group_norm_eval");
    if (!coeffs || !dx || !N || !out || dims < 1 || dims > 3) {
        set_error("disp_group_norm_eval: bad argument");
        return FDTD_EINVAL;
    }
    for (int i = 0; i < dims; ++i)
        if (N[i] < 1 || !(dx[i] > 0)) { set_error("disp_group_norm_eval: bad grid"); return FDTD_EINVAL; }
    if (weight != FDTD_W_UNIFORM && weight != FDTD_W_CONE_X && weight != FDTD_W_GAUSS_Y) {
        set_error("unknown weight %d", weight);
        return FDTD_EINVAL;
    }
    if (weight == FDTD_W_GAUSS_Y && !(weight_param > 0)) { set_error("gauss width must be > 0"); return FDTD_EINVAL; }
    Clean cc = clean_coeffs(coeffs, dims);
    int rc = validate(cc, dx, dims, dt);
    if (rc) return rc;
    cudaStream_t st = (cudaStream_t)stream;
    int Nd[3];
    long long npts = 1;
    for (int i = 0; i < 3; ++i) {
        Nd[i] = i < dims ? N[i] : 1;
        npts *= Nd[i];
    }
    const size_t nscr = group_scratch_doubles(Nd, npts);
    double* scratch = nullptr;
    CK(cudaMallocAsync((void**)&scratch, nscr * sizeof(double), st));
    double* res = nullptr;
    launch_disp_group_norm(cc.alpha, cc.beta, cc.delta, dt, dx, dims, Nd, weight, weight_param,
                           scratch, &res, st);
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaMemcpyAsync(out, res, 14 * sizeof(double), cudaMemcpyDeviceToHost, st);
    cudaFreeAsync(scratch, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) {
        set_error("disp_group_norm_eval: %s", cudaGetErrorString(e));
        return FDTD_ECUDA;
    }
    return FDTD_OK;
}

int disp_omega_eval(const fdtd_coeffs* coeffs, double dt, const double dx[3], int32_t dims,
                    const double* k_dev, int32_t n, double* omega_dev, void* stream) {
    NvtxRange nvtx_range("disp_omega_eval");
    if (!coeffs || !dx || !k_dev || !omega_dev || n < 0 || dims < 1 || dims > 3) {
        set_error("disp_omega_eval: bad argument");
        return FDTD_EINVAL;
    }
    for (int i = 0; i < 3; ++i)
        if (!(dx[i] > 0)) { set_error("dx must be positive"); return FDTD_EINVAL; }
    Clean cc = clean_coeffs(coeffs, dims);
    int rc = validate(cc, dx, dims, dt);
    if (rc) return rc;
    if (n == 0) return FDTD_OK;
    launch_omega(cc.alpha, cc.beta, cc.delta, dt, dx, dims, k_dev, n, omega_dev, (cudaStream_t)stream);
    CK(cudaGetLastError());
    return FDTD_OK;
}

// ---------------------------------------------------------------------------
// disp_norm_eval_noalloc: the dispersion norm without any device allocation.
//
// Some callers cannot allocate device memory at the moment they need the norm:
// code running while a CUDA graph is being built on another stream of the same
// device, a host that pre-reserves every byte of the GPU for its own pool, or a
// plug-in that is not allowed to touch the allocator at all.  For them this entry
// point runs the same three kernels as disp_norm_eval on a fixed scratch area
// that the library declares statically on every device it is loaded on (512 KiB,
// held until the process exits) instead of asking cudaMallocAsync for one.
//
// The host never uses the array's name as a device address: on the first call on
// a device (with that device current) cudaGetSymbolAddress yields its address,
// which is cached per device (with the context it belongs to) and passed to the
// kernels.  That first call is the set-up; make it before capturing any stream into
// a graph.
// ---------------------------------------------------------------------------

namespace {

constexpr int kNoallocMaxN = 4096;              // per k-axis
constexpr size_t kNoallocDoubles = 64 * 1024;   // 3*(3*4096) table + partials + results fit
constexpr int kNoallocMaxDevices = 64;

static __device__ __align__(256) double g_norm_scratch[kNoallocDoubles];

// The array's address on a device is fixed for the life of the device's context; resetting the
// device (cudaDeviceReset) and creating a new primary context loads the module again, and the
// array may then sit elsewhere.  So the cached address is kept together with the context it
// was looked up in, and is looked up again whenever the current context differs.
struct NoallocSlot {
    void* ctx;
    double* addr;
};
static NoallocSlot g_norm_scratch_slot[kNoallocMaxDevices];

// the calling thread's current context (driver API through the runtime's entry-point lookup, so
// the library needs no link against the driver library); nullptr when it cannot be queried
void* current_context() {
    using Fn = CUresult (*)(CUcontext*);
    static Fn fn = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess && q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<Fn>(p);
    });
    CUcontext c = nullptr;
    if (fn == nullptr || fn(&c) != CUDA_SUCCESS) return nullptr;
    return c;
}

int noalloc_scratch_address(double** out) {
    int dev = -1;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) {
        set_error("disp_norm_eval_noalloc: cudaGetDevice failed: %s", cudaGetErrorString(e));
        return FDTD_ECUDA;
    }
    if (dev < 0 || dev >= kNoallocMaxDevices) {
        set_error("disp_norm_eval_noalloc: device ordinal %d out of range", dev);
        return FDTD_EINVAL;
    }
    void* ctx = current_context();
    static std::mutex mu;
    std::lock_guard<std::mutex> lock(mu);
    NoallocSlot& slot = g_norm_scratch_slot[dev];
    if (slot.addr == nullptr || slot.ctx != ctx) {
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_norm_scratch);
        if (e != cudaSuccess || p == nullptr) {
            set_error("disp_norm_eval_noalloc: cudaGetSymbolAddress failed: %s",
                      cudaGetErrorString(e));
            return FDTD_ECUDA;
        }
        // the context may only exist once the runtime has set it up for the lookup above
        slot.ctx = ctx != nullptr ? ctx : current_context();
        slot.addr = static_cast<double*>(p);
    }
    *out = slot.addr;
    return FDTD_OK;
}

}  // namespace

int disp_norm_eval_noalloc(const fdtd_coeffs* coeffs, double dt, const double dx[3], int32_t dims,
                           const int32_t N[3], int32_t weight, double weight_param, double* out,
                           void* stream) {
    NvtxRange nvtx_range("disp_norm_eval_noalloc");
    if (!coeffs || !dx || !N || !out || dims < 1 || dims > 3) {
        set_error("disp_norm_eval_noalloc: bad argument");
        return FDTD_EINVAL;
    }
    for (int i = 0; i < dims; ++i) {
        if (N[i] < 1 || !(dx[i] > 0)) {
            set_error("disp_norm_eval_noalloc: bad grid");
            return FDTD_EINVAL;
        }
        if (N[i] > kNoallocMaxN) {
            set_error("disp_norm_eval_noalloc: N[%d] = %d exceeds the static scratch limit of %d "
                      "points per axis (use disp_norm_eval)", i, N[i], kNoallocMaxN);
            return FDTD_EINVAL;
        }
    }
    if (weight != FDTD_W_UNIFORM && weight != FDTD_W_CONE_X && weight != FDTD_W_GAUSS_Y) {
        set_error("unknown weight %d", weight);
        return FDTD_EINVAL;
    }
    if (weight == FDTD_W_GAUSS_Y && !(weight_param > 0)) {
        set_error("gauss width must be > 0");
        return FDTD_EINVAL;
    }
    Clean cc = clean_coeffs(coeffs, dims);
    int rc = validate(cc, dx, dims, dt);
    if (rc) return rc;
    int Nd[3];
    long long npts = 1;
    for (int i = 0; i < 3; ++i) {
        Nd[i] = i < dims ? N[i] : 1;
        npts *= Nd[i];
    }
    if (norm_scratch_doubles(Nd, npts) > kNoallocDoubles) {
        set_error("disp_norm_eval_noalloc: grid needs more than the %zu-double static scratch",
                  kNoallocDoubles);
        return FDTD_EINVAL;
    }
    double* scratch = nullptr;
    rc = noalloc_scratch_address(&scratch);
    if (rc) return rc;
    // Nothing in the scratch needs clearing: the kernels write every table entry, every
    // per-block partial and every result slot before reading it in this same call.
    cudaStream_t st = (cudaStream_t)stream;
    double* res = nullptr;
    launch_disp_norm(cc.alpha, cc.beta, cc.delta, dt, dx, dims, Nd, weight, weight_param, scratch,
                     &res, st);
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaMemcpyAsync(out, res, 14 * sizeof(double), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) {
        set_error("disp_norm_eval_noalloc: %s", cudaGetErrorString(e));
        return FDTD_ECUDA;
    }
    return FDTD_OK;
}
