// FP32 reverse leapfrog step in one kernel: mu, lambda_E and the coefficient gradient.
//
// One reverse step (derivation in fdtd_adjoint.cu) maps the adjoint state (lambda_E, lambda_B)
// attached to u^{n+1} to the one attached to u^n:
//   l_E = S lambda_E,   mu = S (lambda_B + dt G^T l_E),
//   lambda_E' = l_E + dt F^T mu,   lambda_B' = mu,   g_theta += dt <mu, (dF/dtheta) E^n>.
// F^T mu is formed with the transposed extended stencils DT_a (reach -2 .. +1 along a, +-1
// across; see fdtd_adjoint32e.cu), and the gradient in its transposed form.  With alpha
// eliminated by Eq. (alpha), D*_a is affine in (delta_a, beta_ab, beta_ac), and over the
// periodic grid
//   sum_c mu(c) (dD*_a/dtheta F)(c) = sum_c F(c) (T_theta mu)(c),
//   T_delta_a mu = (mu[-2a] - mu[+a]) - 3 d(0),   T_beta_ab mu = (d(-b) + d(+b)) - 2 d(0),
// with d(k) = mu[k-a] - mu[k]: the very differences DT_a combines,
//   DT_a mu = cA d(0) + cD (mu[-2a] - mu[+a]) + cBb (d(-b) + d(+b)) + cBc (d(-c) + d(+c)).
// So one set of mu taps gives both lambda_E' and the gradient terms, and E^n is read at the
// own cells only.  (The sum equals that of the forward form; only the rounding order differs.)
// Each DT_a mu_m that enters lambda_E'_k with sign s adds s E^n_k (T_theta mu_m) to the
// gradient of D*_a's coefficients.
//
// A CTA owns a 64 x 8 (x, y) tile and a chunk of z planes z0 .. zend-1 and marches z:
//   phase A, plane p: mu(p) on the tile and on the halo the transposed stencils reach
//     (x0-2 .. x0+64, y0-2 .. y0+8), from lambda_E planes p and p+1 (TMA boxes 72 x 12 at
//     x0-4, y0-2, three-slot ring) and lambda_B(p) (TMA boxes 72 x 11, two-slot ring), both
//     copied two planes ahead; mu goes to a five-plane shared ring and, for the own cells of
//     planes z0 .. zend-1, to lambda_B';
//   phase B, plane q = p-2: lambda_E'(q) and the gradient terms of the own cells, from mu
//     planes q-2 .. q+1 (formed in the four previous iterations), lambda_E(q) and E^n(q) (HBM,
//     one plane ahead).
// Within an iteration phase B runs first: it reads none of the plane's new copies, so the
// copies get its duration to land before phase A waits for them.  One block barrier per plane.
// mu of the halo planes z0-2, z0-1 and zend is recomputed by each chunk.  Each thread's own rows of mu (five planes) and of lambda_E (three planes) are
// also kept in tensor memory (TMEM, 128 columns per CTA), written once in phase A and read in
// phase B, which then takes only the neighbouring rows from the shared ring.  The result goes
// to the other adjoint state set: CTAs of neighbouring tiles read halos of lambda_E and
// lambda_B, so an in-place update would race.
//
// Threads: two groups of four warps; in phase B both take the 128 own segments (row o / 16,
// x offset 4 (o % 16) for o = thread mod 128) and split the six transposed stencils three and
// three.  Phase A (mu on 195 four-cell segments: the 128 own ones, rows -2, -1 and 8, and the
// columns x0-4 (rows -1 .. 8) and x0+64 (rows -1 .. 7)) runs own rows 0-5 in warps 0-2, own
// rows 6-7 in warp 7 (each in a warp of the TMEM quadrant that holds them), the halo in warps
// 4-6; lanes without a segment compute a copy whose result is dropped (the warp's shuffles need
// every lane).  Thread PRODUCER (an idle lane of warp 6) waits for and issues the TMA copies.
// Every mbarrier wait is bounded; on expiry the CTA raises *err, drains its copies in flight
// (bounded) and returns.
#include "fdtd_tmem.cuh"

namespace fdtd {
namespace adj32f {

using namespace seg;

constexpr int W = 4, TX = 64, TY = 8;
constexpr int NSEG = TX / W;
constexpr int NOWN = NSEG * TY;                                 // 128 own segments
constexpr int NT = 2 * NOWN;                                    // 256 threads: two groups
constexpr int PRODUCER = NT - 48;                               // lane 16 of warp 6
constexpr int LW = TX + 8, LH = TY + 4, LPL = LW * LH;          // lambda_E box 72 x 12
constexpr int LSLOT = ((LPL * 4 + 127) / 128) * 128 / 4;
constexpr int MH = TY + 3, MPL = LW * MH;                       // mu plane 72 x 11
constexpr int MSLOT = ((MPL * 4 + 127) / 128) * 128 / 4;
constexpr int NL = 3, NB = 2, NM = 5, NS = 2;   // lambda_E, lambda_B, mu ring slots
constexpr size_t OFF_B = (size_t)NL * 3 * LSLOT * 4;             // lambda_B boxes 72 x 11
constexpr size_t OFF_M = OFF_B + (size_t)NB * 3 * MSLOT * 4;
constexpr size_t OFF_Y = OFF_M + (size_t)NM * 3 * MSLOT * 4;      // DT_x mu_z, 2 x 128 x 4
constexpr size_t OFF_BAR = OFF_Y + (size_t)2 * NOWN * W * 4;
constexpr size_t OFF_TM = OFF_BAR + (size_t)(NS + 1) * 8;      // TMEM address
constexpr size_t SMEM = OFF_TM + 16;
// TMEM columns of a thread's own segment (lane = own segment o): mu component c of ring slot s
// at 4 (c NM + s); lambda_E component c of plane p at COL_LE + 4 (3 c + (p's iteration mod 3))
constexpr uint32_t TM_COLS = 128;   // per CTA (two CTAs per SM: 256 of the 512 columns)
constexpr int COL_LE = 4 * 3 * NM;
static_assert(COL_LE + 4 * 9 <= (int)TM_COLS, "TMEM columns");
constexpr uint32_t UNIT_BYTES = 3u * (LPL + MPL) * 4;   // lambda_E and lambda_B boxes
constexpr uint32_t PRO_BYTES = 3u * LPL * 4;
static_assert(LW == 72 && LH == 12, "the lambda_E boxes are the 72 x 12 boxes of encode_ebox_f32");
static_assert(MH == 11, "the lambda_B boxes are 72 x 11 (encode_box_f32)");

// Gradient terms of one cell: s w (T_delta, T_beta_b, T_beta_c) with T_delta = t2 - 3 d0,
// T_beta = sb - 2 d0, T_beta_c = sc - 2 d0, accumulated as the four sums acc[0..3] of s w times
// (t2, sb, sc, d0) (four FMAs a cell instead of six); grad_terms() forms the three terms from
// them once per plane
template <bool NEG>
__device__ __forceinline__ void bracket_acc(float* acc, float w, float d0, float t2, float sb,
                                            float sc) {
    const float ww = NEG ? -w : w;
    acc[0] = fmaf(ww, t2, acc[0]);
    acc[1] = fmaf(ww, sb, acc[1]);
    acc[2] = fmaf(ww, sc, acc[2]);
    acc[3] = fmaf(ww, d0, acc[3]);
}

// DT_z of a mu component on the four cells at e (transverse x, then y): the own row of planes
// q-2 .. q+1 in cmm, cm, c0, cp (from TMEM), the neighbouring rows from the shared planes Gm
// (q-1) and G0 (q); gradient terms of D*_z (delta_z, beta_zx, beta_zy)
template <bool NEG>
__device__ __forceinline__ void dtz_g(const float* Gm, const float* G0, const Q4& cmm,
                                      const Q4& cm, const Q4& c0, const Q4& cp, int e, bool lb,
                                      bool rb, float cA, float cD, float cBx, float cBy,
                                      const float* w, float* acc, float out[4]) {
    const Q4 ym = ldq(Gm, e - LW), y0m = ldq(G0, e - LW), yp = ldq(Gm, e + LW),
             y0p = ldq(G0, e + LW);
    float d[6];   // d[k] = G(q-1) - G(q) at x-1+k
#pragma unroll
    for (int u = 0; u < 4; ++u) d[1 + u] = cm.v[u] - c0.v[u];
    d[0] = from_left(d[4]);
    d[5] = from_right(d[1]);
    if (lb) d[0] = Gm[e - 1] - G0[e - 1];
    if (rb) d[5] = Gm[e + 4] - G0[e + 4];
#pragma unroll
    for (int u = 0; u < 4; ++u) {
        const float dym = ym.v[u] - y0m.v[u], dyp = yp.v[u] - y0p.v[u];
        out[u] = dstar_diff(d[1 + u], cmm.v[u], cp.v[u], d[u], d[2 + u], dym, dyp, cA, cD, cBx, cBy);
        bracket_acc<NEG>(acc, w[u], d[1 + u], cmm.v[u] - cp.v[u], d[u] + d[2 + u], dym + dyp);
    }
}

// DT_y (transverse x, then z); own rows of planes q-1, q, q+1 in zm, a0, zp; gradient terms of
// D*_y (delta_y, beta_yx, beta_yz)
template <bool NEG>
__device__ __forceinline__ void dty_g(const float* Gm, const float* G0, const float* Gp,
                                      const Q4& zm, const Q4& a0, const Q4& zp, int e, bool lb,
                                      bool rb, float cA, float cD, float cBx, float cBz,
                                      const float* w, float* acc, float out[4]) {
    const Q4 am = ldq(G0, e - LW), amm = ldq(G0, e - 2 * LW), ap = ldq(G0, e + LW);
    const Q4 zmy = ldq(Gm, e - LW), zpy = ldq(Gp, e - LW);
    float d[6];   // d[k] = G(y-1) - G(y) at x-1+k, plane q
#pragma unroll
    for (int u = 0; u < 4; ++u) d[1 + u] = am.v[u] - a0.v[u];
    d[0] = from_left(d[4]);
    d[5] = from_right(d[1]);
    if (lb) d[0] = G0[e - LW - 1] - G0[e - 1];
    if (rb) d[5] = G0[e - LW + 4] - G0[e + 4];
#pragma unroll
    for (int u = 0; u < 4; ++u) {
        const float dzm = zmy.v[u] - zm.v[u], dzp = zpy.v[u] - zp.v[u];
        out[u] = dstar_diff(d[1 + u], amm.v[u], ap.v[u], d[u], d[2 + u], dzm, dzp, cA, cD, cBx, cBz);
        bracket_acc<NEG>(acc, w[u], d[1 + u], amm.v[u] - ap.v[u], d[u] + d[2 + u], dzm + dzp);
    }
}

// DT_x (transverse y, then z); own rows of planes q-1, q, q+1 in Zm, R, Zp; gradient terms of
// D*_x (delta_x, beta_xy, beta_xz)
template <bool NEG>
__device__ __forceinline__ void dtx_g(const float* Gm, const float* G0, const float* Gp,
                                      const Q4& Zm, const Q4& R, const Q4& Zp, int e, bool lb,
                                      bool rb, float cA, float cD, float cBy, float cBz,
                                      const float* w, float* acc, float out[4]) {
    const Q4 Ym = ldq(G0, e - LW), Yp = ldq(G0, e + LW);
    float r[7];                         // G(q) at x-2 .. x+4
    float ym[5], yp[5], zm[5], zp[5];   // x-1 .. x+3
#pragma unroll
    for (int u = 0; u < 4; ++u) {
        r[2 + u] = R.v[u];
        ym[1 + u] = Ym.v[u];
        yp[1 + u] = Yp.v[u];
        zm[1 + u] = Zm.v[u];
        zp[1 + u] = Zp.v[u];
    }
    r[0] = from_left(R.v[2]);
    r[1] = from_left(R.v[3]);
    r[6] = from_right(R.v[0]);
    ym[0] = from_left(Ym.v[3]);
    yp[0] = from_left(Yp.v[3]);
    zm[0] = from_left(Zm.v[3]);
    zp[0] = from_left(Zp.v[3]);
    if (lb) {
        r[0] = G0[e - 2];
        r[1] = G0[e - 1];
        ym[0] = G0[e - LW - 1];
        yp[0] = G0[e + LW - 1];
        zm[0] = Gm[e - 1];
        zp[0] = Gp[e - 1];
    }
    if (rb) r[6] = G0[e + 4];
#pragma unroll
    for (int u = 0; u < 4; ++u) {
        const float d0 = r[u + 1] - r[u + 2];
        const float dym = ym[u] - ym[u + 1], dyp = yp[u] - yp[u + 1];
        const float dzm = zm[u] - zm[u + 1], dzp = zp[u] - zp[u + 1];
        out[u] = dstar_diff(d0, r[u], r[u + 3], dym, dyp, dzm, dzp, cA, cD, cBy, cBz);
        bracket_acc<NEG>(acc, w[u], d0, r[u] - r[u + 3], dym + dyp, dzm + dzp);
    }
}

// SP: absorbing layers present (spy, spz not null); without them S = 1 is a compile-time
// constant and the multiplications by it fold away (same results: x * 1 and fma(-1, y, x) are
// exact)
template <bool SP>
__global__ void __launch_bounds__(NT, 2)
adjF_kernel(const __grid_constant__ FusedMaps maps, Geom g, Mult<float> m, FieldSet<float> lam,
            FieldSet<float> out, const float* __restrict__ e_x, const float* __restrict__ e_y,
            const float* __restrict__ e_z, const float* __restrict__ spy,
            const float* __restrict__ spz, double* __restrict__ partials, int tz,
            int* __restrict__ err) {
    extern __shared__ __align__(128) unsigned char smem[];
    float* sL = reinterpret_cast<float*>(smem);
    float* sB = reinterpret_cast<float*>(smem + OFF_B);
    float* sM = reinterpret_cast<float*>(smem + OFF_M);
    float* sY = reinterpret_cast<float*>(smem + OFF_Y);
    uint64_t* bar = reinterpret_cast<uint64_t*>(smem + OFF_BAR);

    const int ntx = g.nx / TX, nty = g.ny / TY;
    int w = blockIdx.x;
    const int tx = w % ntx;
    w /= ntx;
    const int ty = w % nty;
    const int zc = w / nty;
    const int x0 = tx * TX, y0 = ty * TY, z0 = zc * tz;
    const int zend = min(z0 + tz, g.nz);
    const int niter = zend - z0;   // planes of lambda_E'
    const int tid = threadIdx.x;
    const bool edge = (x0 < PX) || (x0 + TX > g.nx - PX) || (y0 < PY) || (y0 + TY > g.ny - PY);

    auto wrapz = [&](int q) {
        int r = q % g.nz;
        return r < 0 ? r + g.nz : r;
    };
    // ring slots of plane P: lambda_E (P >= z0-2), mu (P >= z0-4); lambda_B of plane P in slot
    // (P - z0) mod 2
    auto lslot = [&](int P) { return (P - z0 + 2) % NL; };
    auto slot = [&](int P) { return (P - z0 + 4) % NM; };
    // unit u: the lambda_E boxes of plane z0-1+u (the leading plane of iteration u) and the
    // lambda_B boxes of plane z0-2+u (phase A's plane in iteration u)
    auto issue_unit = [&](int u) {
        const int P = z0 - 1 + u;
        uint64_t* b = &bar[u % NS];
        mbar_expect_tx(b, UNIT_BYTES);
        for (int c = 0; c < 3; ++c) {
            tma_load_3d(sL + (lslot(P) * 3 + c) * LSLOT, &maps.e[c], x0, y0, wrapz(P), b);
            tma_load_3d(sB + ((u & 1) * 3 + c) * MSLOT, &maps.b[c], x0, y0, wrapz(P - 1), b);
        }
    };

    // ---- phase A task of this thread (segment at x0+abx, row y0+aby).  An own row is formed
    // by a warp of the TMEM quadrant that holds it (warps w and w+4 reach lanes 32 (w mod 4) ..
    // + 31, lane = own segment o): rows 0-5 by warps 0-2, rows 6-7 by warp 7; the halo by
    // warps 4-6; warp 3 has no task
    const int wq = tid >> 5;
    int abx = TX, aby = TY - 1;   // no task: a copy of the last right-column task
    bool has_task = true;
    if (wq < 3) {   // own rows 0 .. 5
        aby = tid / NSEG;
        abx = W * (tid % NSEG);
    } else if (wq == 7) {   // own rows 6, 7
        const int t = tid - 7 * 32;
        aby = 6 + t / NSEG;
        abx = W * (t % NSEG);
    } else if (wq == 3) {
        has_task = false;
    } else {
        const int t = tid - 4 * 32;
        if (t < 3 * NSEG) {   // halo rows -1, -2, 8
            const int r = t / NSEG;
            aby = r == 0 ? -1 : r == 1 ? -2 : TY;
            abx = W * (t % NSEG);
        } else if (t < 3 * NSEG + 10) {   // left column, rows -1 .. 8
            abx = -W;
            aby = t - 3 * NSEG - 1;
        } else if (t < 3 * NSEG + 19) {   // right column, rows -1 .. 7
            abx = TX;
            aby = t - 3 * NSEG - 11;
        } else {
            has_task = false;
        }
    }
    // lanes of a 16-segment row get x+1 of their last cell from the next lane
    const bool row16 = abx >= 0 && abx < TX;
    const bool a_rb = !has_task || !row16 || abx == TX - W;
    const bool a_own = has_task && row16 && aby >= 0 && aby < TY;
    // phase A runs in every warp that has a task (warp 3 has none); a_own is warp-uniform
    const bool a_warp = wq != 3;
    const int ea = (aby + 2) * LW + (abx + 4);
    int jwa = (y0 + aby) % g.ny;
    if (jwa < 0) jwa += g.ny;
    const int jwap = jwa + 1 == g.ny ? 0 : jwa + 1;
    const unsigned plane = (unsigned)g.plane;
    const SegOut adst = seg_out(g, x0 + (a_own ? abx : 0), y0 + (a_own ? aby : 0), edge);

    // ---- phase B: own segment o of this thread, group 0 (warps 0-3) or 1 (warps 4-7)
    const bool grp1 = tid >= NOWN;
    const int o = tid & (NOWN - 1);
    const int by = o / NSEG, bx = W * (o % NSEG);
    const bool lb = bx == 0, rb = bx == TX - W;
    const int e = (by + 2) * LW + (bx + 4);
    const int jw = y0 + by;
    const SegOut dst = seg_out(g, x0 + bx, jw, edge);

    if (tid == PRODUCER) {
        for (int s = 0; s <= NS; ++s) mbar_init(&bar[s], 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    }
    // TMEM: warp 0 allocates the CTA's columns, the address goes through shared memory
    uint32_t* tm_slot = reinterpret_cast<uint32_t*>(smem + OFF_TM);
    if (wq == 0) tm_alloc<TM_COLS>(tm_slot);
    tm_fence_before();
    __syncthreads();
    tm_fence_after();
    const uint32_t tb = *tm_slot + ((uint32_t)(32 * (wq & 3)) << 16);
    auto cmu = [&](int c, int sl) { return tb + (uint32_t)(4 * (c * NM + sl)); };
    auto cle = [&](int c, int s3) { return tb + (uint32_t)(COL_LE + 4 * (3 * c + s3)); };
    int issued = 0;
    const int nunits = niter + 3;   // lambda_E planes z0-1 .. zend+1
    if (tid == PRODUCER) {
        const int P = z0 - 2;
        mbar_expect_tx(&bar[NS], PRO_BYTES);
        for (int c = 0; c < 3; ++c)
            tma_load_3d(sL + (lslot(P) * 3 + c) * LSLOT, &maps.e[c], x0, y0, wrapz(P), &bar[NS]);
        for (int u = 0; u < 2 && u < nunits; ++u) {
            issue_unit(u);
            issued = u + 1;
        }
    }

    // the two E^n components of phase B (group 0: E_x, E_y; group 1: E_y, E_z), read from HBM
    // one plane ahead into en, moved to eo when used
    float eo[2][W], en[2][W];
    const float* ea0 = grp1 ? e_y : e_x;
    const float* ea1 = grp1 ? e_z : e_y;
    auto load_e = [&](int qw, float (&to)[2][W]) {
        const unsigned off = (unsigned)qw * plane + dst.ro;
        unpackv(__ldg(reinterpret_cast<const float4*>(ea0 + off)), to[0]);
        unpackv(__ldg(reinterpret_cast<const float4*>(ea1 + off)), to[1]);
    };
    load_e(wrapz(z0), en);

    // gradient partial sums: group 0 holds D*_y, D*_z (entries 3..8), group 1 D*_x, D*_y (0..5).
    // racc: the plane's FP32 sums (four per axis, see bracket_acc); gs, gc: Kahan-compensated
    // FP32 running sums of the three terms per axis over the planes (FP64 arithmetic runs at 1/64
    // of the FP32 rate on this part: a per-plane FP64 add kept its pipe 41 % busy); FP64 only in
    // the block and grid reductions
    float racc[8], gs[6], gc[6];
#pragma unroll
    for (int k = 0; k < 8; ++k) racc[k] = 0.0f;
#pragma unroll
    for (int k = 0; k < 6; ++k) {
        gs[k] = 0.0f;
        gc[k] = 0.0f;
    }
    // lambda_E'_y(q) = S lE_y + (DT_z mu_x - DT_x mu_z): group 0 forms DT_z mu_x and keeps it
    // with S and lE_y; group 1 passes DT_x mu_z through sY; group 0 completes it after the
    // next block barrier
    float ya[W], yl[W], ys0 = 0.0f;
    unsigned ypo = 0;
    bool ypend = false;
    bool failed = false;
    int it = 0;
    {
        bool ok0 = true;
        if (tid == PRODUCER) ok0 = mbar_wait(&bar[NS], 0) && mbar_wait(&bar[0], 0);
        failed = __syncthreads_or(!ok0);
    }
    // iteration it: phase A on plane p = z0-2+it (p <= zend), phase B on q = p-2
    // (z0 <= q < zend); the last iteration only completes lambda_E'_y of plane zend-1.
    // Plane bookkeeping by counters (no integer division in the loop): pw = p mod nz,
    // qw = q mod nz, sp = ring slot of plane p = (it + 2) mod 5 (plane q: sp + 3, q-2: + 1, ...)
    int pw = wrapz(z0 - 2), qw = wrapz(z0 - 4), sp = slot(z0 - 2), lp = lslot(z0 - 2);
    int e3 = 0;   // it mod 3: TMEM slot of lambda_E(p); plane q's is (it + 1) mod 3
    auto inc5 = [](int a, int k) { return a + k >= NM ? a + k - NM : a + k; };   // mu ring slots
    for (; !failed && it <= niter + 4; ++it, qw = (qw + 1 == g.nz ? 0 : qw + 1),
                                       pw = (pw + 1 == g.nz ? 0 : pw + 1), sp = inc5(sp, 1),
                                       lp = (lp == NL - 1 ? 0 : lp + 1),
                                       e3 = (e3 == 2 ? 0 : e3 + 1)) {
        const int p = z0 - 2 + it;
        const int q = p - 2;
        // ---- lambda_E'_y of the previous plane (group 0)
        if (!grp1 && ypend) {
            const Q4 b = ldq(sY + ((it + 1) & 1) * NOWN * W, o * W);
            float v[W];
#pragma unroll
            for (int u = 0; u < W; ++u) v[u] = __fmaf_rn(ys0, yl[u], __fsub_rn(ya[u], b.v[u]));
            put_seg(out.c[1], ypo, dst, v);
            ypend = false;
        }
        // ---- phase B: lambda_E'(q) and the gradient terms (warp-uniform); it reads no data of
        // this iteration's copies (mu of earlier planes, lambda_E(q) from TMEM, E^n from registers),
        // so it runs before the wait for them
        if (q >= z0 && q < zend) {
#pragma unroll
            for (int c = 0; c < 2; ++c)
#pragma unroll
                for (int u = 0; u < W; ++u) eo[c][u] = en[c][u];
            if (q + 1 < zend) load_e(qw + 1 == g.nz ? 0 : qw + 1, en);
            // mu planes q-2 .. q+1 (shared ring and, own rows, TMEM slots alike) and lambda_E(q)
            const int smm = inc5(sp, 1), sm = inc5(sp, 2), sq = inc5(sp, 3), spp = inc5(sp, 4);
            const int lq = e3 == 2 ? 0 : e3 + 1;
            const float* Gm = sM + sm * 3 * MSLOT;
            const float* G0 = sM + sq * 3 * MSLOT;
            const float* Gp = sM + spp * 3 * MSLOT;
            const float s0 = SP ? spy[jw] * spz[qw] : 1.0f;
            const unsigned po = (unsigned)qw * plane;
            float t1[W], t2[W], v[W];
            if (!grp1) {
                // lambda_E'_x = S lE_x + (DT_y mu_z - DT_z mu_y)
                {
                    Q4 zm, z0_, zp;
                    tm_ld(cmu(2, sm), zm);
                    tm_ld(cmu(2, sq), z0_);
                    tm_ld(cmu(2, spp), zp);
                    tm_wait_ld(zm, z0_, zp);
                    dty_g<false>(Gm + 2 * MSLOT, G0 + 2 * MSLOT, Gp + 2 * MSLOT, zm, z0_, zp, e, lb,
                                 rb, m.cA[1], m.cD[1], m.cB[1][0], m.cB[1][2], eo[0], racc + 0, t1);
                }
                {
                    Q4 cmm, cm, c0, cp, lx;
                    tm_ld(cmu(1, smm), cmm);
                    tm_ld(cmu(1, sm), cm);
                    tm_ld(cmu(1, sq), c0);
                    tm_ld(cmu(1, spp), cp);
                    tm_ld(cle(0, lq), lx);
                    tm_wait_ld(cmm, cm, c0, cp, lx);
                    dtz_g<true>(Gm + MSLOT, G0 + MSLOT, cmm, cm, c0, cp, e, lb, rb, m.cA[2], m.cD[2],
                                m.cB[2][0], m.cB[2][1], eo[0], racc + 4, t2);
#pragma unroll
                    for (int u = 0; u < W; ++u) v[u] = __fmaf_rn(s0, lx.v[u], __fsub_rn(t1[u], t2[u]));
                }
                put_seg(out.c[0], po, dst, v);
                // DT_z mu_x of lambda_E'_y
                {
                    Q4 cmm, cm, c0, cp, ly;
                    tm_ld(cmu(0, smm), cmm);
                    tm_ld(cmu(0, sm), cm);
                    tm_ld(cmu(0, sq), c0);
                    tm_ld(cmu(0, spp), cp);
                    tm_ld(cle(1, lq), ly);
                    tm_wait_ld(cmm, cm, c0, cp, ly);
                    dtz_g<false>(Gm, G0, cmm, cm, c0, cp, e, lb, rb, m.cA[2], m.cD[2], m.cB[2][0],
                                 m.cB[2][1], eo[1], racc + 4, ya);
#pragma unroll
                    for (int u = 0; u < W; ++u) yl[u] = ly.v[u];
                }
                ys0 = s0;
                ypo = po;
                ypend = true;
            } else {
                // DT_x mu_z of lambda_E'_y, to group 0
                {
                    Q4 zm, z0_, zp;
                    tm_ld(cmu(2, sm), zm);
                    tm_ld(cmu(2, sq), z0_);
                    tm_ld(cmu(2, spp), zp);
                    tm_wait_ld(zm, z0_, zp);
                    dtx_g<true>(Gm + 2 * MSLOT, G0 + 2 * MSLOT, Gp + 2 * MSLOT, zm, z0_, zp, e, lb,
                                rb, m.cA[0], m.cD[0], m.cB[0][1], m.cB[0][2], eo[0], racc + 0, t1);
                }
                stv(sY + (it & 1) * NOWN * W, o * W, t1);
                // lambda_E'_z = S lE_z + (DT_x mu_y - DT_y mu_x)
                {
                    Q4 ym, y0_, yp;
                    tm_ld(cmu(1, sm), ym);
                    tm_ld(cmu(1, sq), y0_);
                    tm_ld(cmu(1, spp), yp);
                    tm_wait_ld(ym, y0_, yp);
                    dtx_g<false>(Gm + MSLOT, G0 + MSLOT, Gp + MSLOT, ym, y0_, yp, e, lb, rb, m.cA[0],
                                 m.cD[0], m.cB[0][1], m.cB[0][2], eo[1], racc + 0, t1);
                }
                {
                    Q4 xm, x0_, xp, lz;
                    tm_ld(cmu(0, sm), xm);
                    tm_ld(cmu(0, sq), x0_);
                    tm_ld(cmu(0, spp), xp);
                    tm_ld(cle(2, lq), lz);
                    tm_wait_ld(xm, x0_, xp, lz);
                    dty_g<true>(Gm, G0, Gp, xm, x0_, xp, e, lb, rb, m.cA[1], m.cD[1], m.cB[1][0],
                                m.cB[1][2], eo[1], racc + 4, t2);
#pragma unroll
                    for (int u = 0; u < W; ++u) v[u] = __fmaf_rn(s0, lz.v[u], __fsub_rn(t1[u], t2[u]));
                }
                put_seg(out.c[2], po, dst, v);
            }
#pragma unroll
            for (int k = 0; k < 6; ++k) {   // the plane's three terms per axis, compensated add
                const float* r4 = racc + 4 * (k / 3);
                const float x = fmaf(k % 3 == 0 ? -3.0f : -2.0f, r4[3], r4[k % 3]);
                const float y = x - gc[k];
                const float t = gs[k] + y;
                gc[k] = (t - gs[k]) - y;
                gs[k] = t;
            }
#pragma unroll
            for (int k = 0; k < 8; ++k) racc[k] = 0.0f;
        }
        // ---- the copies of this iteration (lambda_E(p+1), lambda_B(p)), issued two planes ago
        bool ok = true;
        if (it < nunits) {
            if (it == 0) ok = mbar_wait(&bar[NS], 0);
            ok = ok && mbar_wait(&bar[it % NS], (uint32_t)((it / NS) & 1));
        }
        ok = __all_sync(FULL, ok);   // keeps the shuffles below warp-uniform
        // ---- phase A: mu(p) (warps with a task)
        if (ok && p <= zend && a_warp) {
            const int pw1 = pw + 1 == g.nz ? 0 : pw + 1;
            const float* L0 = sL + lp * 3 * LSLOT;
            const float* L1 = sL + (lp == NL - 1 ? 0 : lp + 1) * 3 * LSLOT;
            const float* Bp = sB + (it & 1) * 3 * MSLOT;
            const Q4 bxq = ldq(Bp, ea), byq = ldq(Bp + MSLOT, ea), bzq = ldq(Bp + 2 * MSLOT, ea);
            const Q4 ex = ldq(L0, ea), ey = ldq(L0 + LSLOT, ea), ez = ldq(L0 + 2 * LSLOT, ea);
            const Q4 exy = ldq(L0, ea + LW), ezy = ldq(L0 + 2 * LSLOT, ea + LW);
            const Q4 exz = ldq(L1, ea), eyz = ldq(L1 + LSLOT, ea);
            float ey4 = from_right(ey.v[0]), ez4 = from_right(ez.v[0]);
            if (a_rb) {
                ey4 = L0[LSLOT + ea + 4];
                ez4 = L0[2 * LSLOT + ea + 4];
            }
            float s0 = 1.0f, syp = 1.0f, szp = 1.0f;
            if (SP) {
                s0 = spy[jwa] * spz[pw];
                syp = spy[jwap] * spz[pw];
                szp = spy[jwa] * spz[pw1];
            }
            float mux[W], muy[W], muz[W];
#pragma unroll
            for (int u = 0; u < W; ++u) {
                // the rounding order of the two-kernel step's mu (fdtd_adjoint32.cu), fixed by
                // intrinsics, which the compiler never contracts
                const float ex0 = __fmul_rn(s0, ex.v[u]), ey0 = __fmul_rn(s0, ey.v[u]),
                            ez0 = __fmul_rn(s0, ez.v[u]);
                const float ezx = u < W - 1 ? ez.v[u + 1] : ez4;   // x+1, unscaled
                const float eyx = u < W - 1 ? ey.v[u + 1] : ey4;
                const float gx = __fmaf_rn(m.cE[2], __fmaf_rn(-szp, eyz.v[u], ey0),
                                           __fmul_rn(-m.cE[1], __fmaf_rn(-syp, ezy.v[u], ez0)));
                const float gy = __fmaf_rn(m.cE[0], __fmaf_rn(-s0, ezx, ez0),
                                           __fmul_rn(-m.cE[2], __fmaf_rn(-szp, exz.v[u], ex0)));
                const float gz = __fmaf_rn(m.cE[1], __fmaf_rn(-syp, exy.v[u], ex0),
                                           __fmul_rn(-m.cE[0], __fmaf_rn(-s0, eyx, ey0)));
                mux[u] = __fmul_rn(s0, __fadd_rn(bxq.v[u], gx));
                muy[u] = __fmul_rn(s0, __fadd_rn(byq.v[u], gy));
                muz[u] = __fmul_rn(s0, __fadd_rn(bzq.v[u], gz));
            }
            if (has_task) {
                float* M = sM + sp * 3 * MSLOT;
                stv(M, ea, mux);
                stv(M + MSLOT, ea, muy);
                stv(M + 2 * MSLOT, ea, muz);
            }
            if (a_own) {   // own rows of mu(p) and lambda_E(p) to TMEM (warp-uniform)
                tm_st(cmu(0, sp), mux);
                tm_st(cmu(1, sp), muy);
                tm_st(cmu(2, sp), muz);
                tm_st(cle(0, e3), ex);
                tm_st(cle(1, e3), ey);
                tm_st(cle(2, e3), ez);
            }
            if (a_own && p >= z0 && p < zend) {   // mu -> lambda_B' (own cells and their images)
                const unsigned po = (unsigned)pw * plane;
                put_seg(out.c[3], po, adst, mux);
                put_seg(out.c[4], po, adst, muy);
                put_seg(out.c[5], po, adst, muz);
            }
        }
        // the TMEM rows stored in this iteration are read by other warps after the barrier
        tm_wait_st();
        tm_fence_before();
        const bool stop = __syncthreads_or(!ok);
        tm_fence_after();
        if (stop) {
            failed = true;
            break;
        }
        // the lambda_E slot of plane p and the lambda_B slot of plane p (both read in this
        // iteration's phase A) take planes p+3 and p+2
        if (tid == PRODUCER && it + 2 < nunits) {
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            issue_unit(it + 2);
            issued = it + 3;
        }
    }
    if (failed && tid == PRODUCER) {   // drain this CTA's copies in flight
        atomicOr(err, ERR_WAIT);
        if (it == 0) mbar_wait(&bar[NS], 0);
        for (int u = it; u < issued; ++u) mbar_wait(&bar[u % NS], (uint32_t)((u / NS) & 1));
    }
    // release the TMEM columns (every path reaches this point)
    tm_wait_st();
    tm_fence_before();
    __syncthreads();
    tm_fence_after();
    if (wq == 0) tm_dealloc<TM_COLS>(*tm_slot);
    if (failed) return;
    // block reduction: entry k of group 0 is coefficient 3 + k, entry k of group 1 coefficient
    // k.  Within a warp the compensated pairs (value gs - gc) are added in FP32 with an exact
    // two-sum at every step (Knuth's TwoSum: s + e = a + b exactly), so no FP64 arithmetic runs
    // until one conversion per warp; across warps and blocks the sums are FP64
    __shared__ double red[NT / 32][9];
    const int wp = tid >> 5, l = tid & 31;
#pragma unroll
    for (int k = 0; k < 6; ++k) {
        float vs = gs[k], vc = gc[k];
        for (int sh = 16; sh > 0; sh >>= 1) {
            const float os = __shfl_down_sync(FULL, vs, sh), oc = __shfl_down_sync(FULL, vc, sh);
            const float t = __fadd_rn(vs, os);
            const float bv = __fsub_rn(t, vs);
            const float err = __fadd_rn(__fsub_rn(vs, __fsub_rn(t, bv)), __fsub_rn(os, bv));
            vs = t;
            vc = __fsub_rn(__fadd_rn(vc, oc), err);
        }
        if (l == 0) red[wp][grp1 ? k : 3 + k] = (double)vs - (double)vc;
    }
    if (l < 3) red[wp][grp1 ? 6 + l : l] = 0.0;
    __syncthreads();
    if (tid < 9) {
        double v = 0.0;
        for (int ww = 0; ww < NT / 32; ++ww) v += red[ww][tid];
        partials[(long long)blockIdx.x * 9 + tid] += v;
    }
}

}  // namespace adj32f

bool adjoint32f_supported(const Geom& g) {
    return g.nx % adj32f::TX == 0 && g.ny % adj32f::TY == 0 && g.nx >= adj32f::TX &&
           g.ny >= adj32f::TY && g.total < (1LL << 31);
}

bool adjoint32f_prepare() {
    return cudaFuncSetAttribute(adj32f::adjF_kernel<true>,
                                cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)adj32f::SMEM) == cudaSuccess &&
           cudaFuncSetAttribute(adj32f::adjF_kernel<false>,
                                cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)adj32f::SMEM) == cudaSuccess;
}

static int adjoint32f_tz(const Geom& g) {
    static int slots = -1;
    if (slots < 0)
        slots = resident_slots_tmem((const void*)adj32f::adjF_kernel<true>, adj32f::NT, adj32f::SMEM,
                                    adj32f::TM_COLS);
    return zchunk_len((g.nx / adj32f::TX) * (g.ny / adj32f::TY), g.nz, slots, 16, 64);
}

int adjoint32f_blocks(const Geom& g) {
    const int tz = adjoint32f_tz(g);
    return (g.nx / adj32f::TX) * (g.ny / adj32f::TY) * ((g.nz + tz - 1) / tz);
}

// maps.e[c]: 72 x 12 boxes of lambda_E component c of the input set `lam`, maps.b[c]: 72 x 11
// boxes of its lambda_B component c; E: the forward
// E^n of the step (padded arrays); the result goes to `out` (the other set)
void launch_adjoint32_fused(const FusedMaps& maps, const Geom& g, const Mult<float>& m,
                            FieldSet<float> lam, FieldSet<float> out, const float* const E[3],
                            const float* spy, const float* spz, double* partials, int* err,
                            cudaStream_t st) {
    auto kern = spy != nullptr ? adj32f::adjF_kernel<true> : adj32f::adjF_kernel<false>;
    kern<<<adjoint32f_blocks(g), adj32f::NT, adj32f::SMEM, st>>>(maps, g, m, lam, out, E[0], E[1],
                                                                  E[2], spy, spz, partials,
                                                                  adjoint32f_tz(g), err);
}

}  // namespace fdtd
