// FP32 fused leapfrog step (one launch per leapfrog step).
//
// A CTA owns a 64 x 8 (x, y) tile and a chunk of tz planes (a launch parameter) and marches
// through it.  E^n planes arrive by TMA (cp.async.bulk.tensor.3d) as 76 x 12 boxes (x0-4 ..,
// y0-2 ..) into a ring of five shared-memory slots, one plane ahead of use, completion signalled
// on mbarriers.  Iteration `it` forms B^{n+1/2} on plane p = z0-1+it (tile, halo row y0-1, halo
// column x0-1) and E^{n+1} on plane p-1, so one block barrier per plane suffices; B^{n+1/2}
// lives in a small shared ring (B_x, B_y: 3 planes, B_z: 2 planes).  B^{n-1/2} is not staged:
// each thread prefetches its own segment of the next plane from HBM into registers while the
// current plane is computed.
//
// Work per thread: W = 4 consecutive cells of one row, the same row in the B and the E phase.
// A warp covers two whole rows.  Each stencil row a thread needs is read once as a 16-byte
// shared-memory vector of its own four cells; the values one cell beyond the segment (x-1,
// x+4, x+5) come from the neighbouring lanes by warp shuffle, and only the lanes at the ends
// of a row (and the halo-column lanes) read them from shared memory.  Differences along an
// axis are formed once per cell and shared with the neighbouring cells (dstar_diff), which
// halves the shared-memory traffic of the stencil compared with reading three-vector windows.
// Owned results leave as 16-byte stores; a segment at the edge of the domain also writes its
// periodic images (the ghosts of the padded layout).  Plane bookkeeping uses counters (no
// integer division in the loop).
//
// The producer also asks L2 for the E boxes and B^{n-1/2} boxes PF planes beyond what the
// ring and the register prefetch already cover (cp.async.bulk.prefetch.tensor), which keeps
// more DRAM reads in flight per CTA than the shared-memory ring alone can hold.
//
// Tensor memory holds each thread's own rows across planes.  A thread's own row of E^n plane P
// is used in four consecutive iterations (as plane p+2, p+1, p, p-1; E_z in three), and its own
// rows of B^{n+1/2} come back in the E phase of the next two iterations.  Registers cannot
// carry them (the kernel sits at 128 registers for three CTAs per SM), and shared memory is the
// pipe that limits the kernel, so each own row is read from the shared ring once, when it is
// newest, written to the thread's TMEM lane (tcgen05.st, 32x32b.x4: four cells) and read back
// from there (tcgen05.ld) in the later iterations: 13 of the 36 16-byte shared-memory reads per
// thread and plane become TMEM reads.  The CTA allocates 128 TMEM columns (three CTAs per SM:
// 384 of 512) and releases them on every exit path.
//
// Per-cell arithmetic is dstar_diff / ampere_comp on the same differences in the same order as
// the reference-form kernels (dstar_taps): the fields are bitwise equal.  Every mbarrier wait is
// bounded (fdtd_tma.cuh); on expiry the CTA raises *err, drains its copies in flight (bounded)
// and returns.
#include <algorithm>
#include <cstring>

#include "fdtd_seg.cuh"
#include "fdtd_tmem.cuh"

namespace fdtd {
namespace f32seg {

using namespace seg;

// the FP32 multipliers, each duplicated into a pair for the paired arithmetic
struct Mult2 {
    u64 cA[3], cD[3], cB[3][3], cE[3], ncE[3];   // ncE = -cE
};

inline Mult2 make_mult2(const Mult<float>& m) {
    auto dup = [](float v) {
        u64 r;
        const float two[2] = {v, v};
        memcpy(&r, two, sizeof r);
        return r;
    };
    Mult2 p;
    for (int a = 0; a < 3; ++a) {
        p.cA[a] = dup(m.cA[a]);
        p.cD[a] = dup(m.cD[a]);
        p.cE[a] = dup(m.cE[a]);
        p.ncE[a] = dup(-m.cE[a]);
        for (int b = 0; b < 3; ++b) p.cB[a][b] = dup(m.cB[a][b]);
    }
    return p;
}

constexpr int W = 4;                                            // cells per thread (along x)
constexpr int TX = 64, TY = 8, D = 1;   // z-chunk length: launch parameter (zchunk_len)
constexpr int NSEG = TX / W;                                    // segments per row
constexpr int NBT = NSEG * (TY + 1) + TY + 1;                   // B tasks: rows + halo column
constexpr int NT = ((NBT + 31) / 32) * 32;
// the thread that initialises the mbarriers, issues the TMA copies and waits for them: lane 0 of
// the halo warp, which has no E update and reaches the block barrier first (with thread 0, the
// copy waits and issues made the first owned-row warp the last to arrive every plane)
constexpr int PRODUCER = NSEG * TY;
// E box 76 x 12 (x0-4 .., y0-2 ..): the stencil needs x0-2 .. x0+65 (a 72-wide box); 76 floats
// = 19 16-byte chunks per row put the halo-column lanes (one segment on each of nine rows) on
// distinct bank groups, which removed most shared-memory bank conflicts.  In the last tile of a
// row the box reaches four columns past the padded array; TMA fills them with zeros (unused)
constexpr int EW = TX + 12, EH = TY + 4, EPL = EW * EH;
constexpr int ESLOT = ((EPL * 4 + 127) / 128) * 128 / 4;        // floats per E slot
constexpr int BW = TX + 4, BH = TY + 1, BPL = BW * BH;         // B^{n+1/2} plane: x0-4.., y0-1..
constexpr int BSLOT = ((BPL * 4 + 127) / 128) * 128 / 4;
constexpr int NE = D + 4, NS = D + 1;
// L2 prefetch distance in planes (measured at 256^3: 2 planes 0.192 ms per step, none 0.197,
// 4 planes 0.195, 8 planes 0.210)
constexpr int PF = 2;
constexpr size_t OFF_E = 128;
constexpr size_t OFF_BN = OFF_E + (size_t)NE * 3 * ESLOT * 4;   // Bx[3], By[3], Bz[2]
constexpr size_t OFF_BAR = OFF_BN + (size_t)8 * BSLOT * 4;
constexpr size_t SMEM = OFF_BAR + (size_t)(NS + 1) * 8;
constexpr uint32_t UNIT_BYTES = 3u * EPL * 4;
constexpr uint32_t PRO_BYTES = 9u * EPL * 4;
static_assert(W == 4, "the segment code below is written for 16-byte vectors of four cells");

// TMEM columns per thread (see the kernel): own rows of E_x, E_y (4 planes), E_z (3 planes),
// B_x, B_y (3 planes), B_z (2 planes), four columns per row of four cells
constexpr uint32_t TM_COLS = 128;   // allocation per CTA (3 CTAs per SM: 384 of 512 columns)
constexpr int COL_EX = 0, COL_EY = 16, COL_EZ = 32, COL_BX = 44, COL_BY = 56, COL_BZ = 68;
constexpr int COL_HALO = 76;        // the halo warp shares quadrant 0 with warp 0: its own columns


__global__ void __launch_bounds__(NT, 3)
step_kernel(const __grid_constant__ FusedMaps maps, Geom g, Mult<float> m, Mult2 m2, FieldSet<float> in,
            FieldSet<float> out, const float* __restrict__ spy, const float* __restrict__ spz,
            const float* __restrict__ jyz, const float* __restrict__ jx_row,
            float* __restrict__ h0, float* __restrict__ h1, float* __restrict__ h2, int zs, int ze,
            int tz, int* __restrict__ err) {
    extern __shared__ __align__(128) unsigned char smem[];
    float* sE = reinterpret_cast<float*>(smem + OFF_E);
    float* sB = reinterpret_cast<float*>(smem + OFF_BN);
    uint64_t* bar = reinterpret_cast<uint64_t*>(smem + OFF_BAR);

    const int ntx = g.nx / TX, nty = g.ny / TY;
    int w = blockIdx.x;
    const int tx = w % ntx;
    w /= ntx;
    const int ty = w % nty;
    const int zc = w / nty;
    const int x0 = tx * TX, y0 = ty * TY, z0 = zs + zc * tz;   // planes zs .. ze-1 of the launch
    const int zend = min(z0 + tz, ze);
    const int niter = zend - z0 + 1;   // B planes z0-1 .. zend-1
    const int tid = threadIdx.x;
    // tiles that own cells with periodic images (the ghosts of the padded layout)
    const bool edge = (x0 < PX) || (x0 + TX > g.nx - PX) || (y0 < PY) || (y0 + TY > g.ny - PY);

    auto wrapz = [&](int q) {
        int r = q % g.nz;
        return r < 0 ? r + g.nz : r;
    };
    auto eslot = [&](int q) { return (q - (z0 - 2)) % NE; };
    auto Ep = [&](int q, int c) { return sE + (eslot(q) * 3 + c) * ESLOT; };
    auto issue_unit = [&](int u) {
        const int qe = z0 + 1 + u;   // leading E plane of iteration u
        uint64_t* b = &bar[u % NS];
        mbar_expect_tx(b, UNIT_BYTES);
        for (int c = 0; c < 3; ++c) tma_load_3d(Ep(qe, c), &maps.e[c], x0, y0, wrapz(qe), b);
    };

    // L2 prefetch of the E box of plane q (q <= zend + 1) and of the B^{n-1/2} box of plane q
    // (q <= zend - 1; the box of the B task region: x0-4 .., y0-1 ..)
    auto pf_e = [&](int q) {
        if (q <= zend + 1)
            for (int c = 0; c < 3; ++c) tma_prefetch_3d(&maps.e[c], x0, y0, wrapz(q));
    };
    auto pf_b = [&](int q) {
        if (q <= zend - 1)
            for (int c = 0; c < 3; ++c) tma_prefetch_3d(&maps.b[c], x0, y0 + 1, wrapz(q));
    };

    // ---- task of this thread.  All NT threads run the B phase, so that every warp shuffle
    // sees a full warp; the E phase is run by the threads of the owned rows.
    //   tid <  128: owned row by = tid / 16, segment bx = 4 (tid % 16) (B and E)
    //   tid in [128, 144): halo row by = -1, bx = 4 (tid % 16)
    //   tid in [144, 153): halo-column segment bx = -4, by = tid - 145; of its cells only
    //   x0-1 is used (by the E update of column x0), the other three are discarded
    //   tid in [153, NT): idle copies of the last halo-column task (results dropped)
    const int b_bx = tid < NSEG * (TY + 1) ? W * (tid % NSEG) : -W;
    const int b_by = tid < NSEG * TY ? tid / NSEG
                     : tid < NSEG * (TY + 1) ? -1 : min(tid - NSEG * (TY + 1) - 1, TY - 1);
    const bool b_store = tid < NBT;      // writes its B^{n+1/2} segment to the shared ring
    const bool b_own = tid < NSEG * TY;  // owned cells: stored to HBM, E phase
    // no left neighbour lane in the row (a halo-column segment skips its left side: x0-5 only
    // reaches its first cell, x0-4, which is discarded)
    const bool lb = b_bx == 0;
    const bool rb = b_bx < 0 || b_bx == TX - W;
    const int e = (b_by + 2) * EW + (b_bx + 4);   // in-plane index of the segment, E box
    const int bi = (b_by + 1) * BW + (b_bx + 4);  // in-plane index of the segment, B ring
    const unsigned b_off = (unsigned)((y0 + b_by + PY) * g.nxp + (x0 + b_bx + PX));
    const unsigned plane = (unsigned)g.plane;
    int b_y = y0 + b_by;
    if (b_y < 0) b_y += g.ny;
    // owned-cell destinations of this thread's segment
    const SegOut dst = seg_out(g, x0 + (b_bx < 0 ? 0 : b_bx), y0 + (b_by < 0 ? 0 : b_by), edge);

    if (tid == PRODUCER) {
        for (int s = 0; s <= NS; ++s) mbar_init(&bar[s], 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    }
    // TMEM: warp 0 allocates the CTA's columns; the address goes through shared memory (the
    // 128-byte header before the rings) to every thread
    uint32_t* tm_slot = reinterpret_cast<uint32_t*>(smem);
    if (tid < 32) tm_alloc<TM_COLS>(tm_slot);
    tm_fence_before();
    __syncthreads();
    tm_fence_after();
    const uint32_t tm_base = *tm_slot;
    const int warp = tid >> 5;
    // this thread's TMEM lane (quadrant of its warp) and column base
    const uint32_t tb = tm_base + ((uint32_t)(32 * (warp & 3)) << 16) + (warp == 4 ? COL_HALO : 0);
    int issued = 0;
    if (tid == PRODUCER) {
        mbar_expect_tx(&bar[NS], PRO_BYTES);
        for (int q = z0 - 2; q <= z0; ++q)
            for (int c = 0; c < 3; ++c) tma_load_3d(Ep(q, c), &maps.e[c], x0, y0, wrapz(q), &bar[NS]);
        for (int u = 0; u <= D && u < niter; ++u) {
            issue_unit(u);
            issued = u + 1;
        }
        for (int k = 0; k < PF; ++k) {
            pf_e(z0 + 3 + k);
            pf_b(z0 + k);
        }
    }

    // B^{n-1/2} of this thread's task, prefetched one plane ahead: bn is loaded at the start of
    // a B phase for the next plane and moved to bo at the start of the next B phase (after a
    // whole E phase and a block barrier, so the copy does not wait on the loads)
    float bo[3][W];
    float bn[3][W];
#pragma unroll
    for (int c = 0; c < 3; ++c)
#pragma unroll
        for (int u = 0; u < W; ++u) bn[c][u] = 0.0f;
    auto load_bold = [&](int qw, float (&to)[3][W]) {   // qw: wrapped plane index
        const unsigned o = (unsigned)qw * plane + b_off;
#pragma unroll
        for (int c = 0; c < 3; ++c)
            unpackv(__ldg(reinterpret_cast<const float4*>(in.c[3 + c] + o)), to[c]);
    };
    load_bold(wrapz(z0 - 1), bn);

    const float mdt = -m.dt;
    // B^{n+1/2} ring: B_x, B_y keep planes p, p-1, p-2 (slot (p+6) mod 3); B_z keeps p, p-1.
    // Iteration it forms B^{n+1/2} on plane p = z0 - 1 + it (it < niter) and E^{n+1} on
    // plane p - 1 (when z0 <= p - 1 < zend).  One block barrier per iteration.
    // The producer thread waits for each plane's copies before the block barrier that precedes
    // the plane's iteration; the other threads' own waits then return at once (no spinning).
    bool failed = false;
    float fin = 0.0f;   // non-finite detection (nonfinite_acc): stays 0 while every E value is finite
    int it = 0;
    {
        bool ok0 = true;
        if (tid == PRODUCER) ok0 = mbar_wait(&bar[NS], 0) && mbar_wait(&bar[0], 0);
        failed = __syncthreads_or(!ok0);
    }
    // plane bookkeeping by counters (no integer division in the loop):
    //   pw = p mod nz, qw = (p-1) mod nz, s_m = ring slot of plane p-1 = it mod NE,
    //   r3 = (p+6) mod 3 (B_x / B_y ring), r2 = (p+6) mod 2 (B_z ring)
    int pw = wrapz(z0 - 1), qw = wrapz(z0 - 2);
    int s_m = 0;
    int r3 = (z0 + 5) % 3, r2 = (z0 + 5) % 2;
    int e3 = 0;   // it mod 3: TMEM slot rotation of E_z and of the own B^{n+1/2} rows
    for (; !failed && it <= niter; ++it, qw = pw, pw = (pw + 1 == g.nz ? 0 : pw + 1),
                                   s_m = (s_m + 1 == NE ? 0 : s_m + 1), r3 = (r3 == 2 ? 0 : r3 + 1),
                                   r2 ^= 1, e3 = (e3 == 2 ? 0 : e3 + 1)) {
        const int p = z0 - 1 + it;
        // E^n ring slots of planes p-1 .. p+2
        const int s_0 = s_m + 1 == NE ? 0 : s_m + 1;
        const int s_1 = s_0 + 1 == NE ? 0 : s_0 + 1;
        const int s_2 = s_1 + 1 == NE ? 0 : s_1 + 1;
        const float* Pm = sE + s_m * 3 * ESLOT;
        const float* P0 = sE + s_0 * 3 * ESLOT;
        const float* P1 = sE + s_1 * 3 * ESLOT;
        const float* P2 = sE + s_2 * 3 * ESLOT;
        bool ok = true;
        if (it < niter) {
            if (it == 0) ok = mbar_wait(&bar[NS], 0);
            ok = ok && mbar_wait(&bar[it % NS], (uint32_t)((it / NS) & 1));
        }
        ok = __all_sync(FULL, ok);   // keeps the shuffles below warp-uniform
        // TMEM columns of the own rows: E_x, E_y of plane p-1+k in slot (it+k) & 3, E_z of plane
        // p-1+k in slot (it+k) mod 3; own B^{n+1/2} rows of plane p in slot it mod 3 (B_z: it & 1)
        const int e3p = e3 == 2 ? 0 : e3 + 1, e3pp = e3p == 2 ? 0 : e3p + 1;
        auto cx = [&](int k) { return tb + COL_EX + 4 * ((it + k) & 3); };
        auto cy = [&](int k) { return tb + COL_EY + 4 * ((it + k) & 3); };
        const uint32_t cz0 = tb + COL_EZ + 4 * e3, cz1 = tb + COL_EZ + 4 * e3p,
                       cz2 = tb + COL_EZ + 4 * e3pp;
        // ---- B^{n+1/2}(p)
        // B^{n+1/2} ring slots: plane p (current) and p-1 (its rows y-1 and the halo column feed
        // the E phase; the own rows come from TMEM)
        const int r3m = r3 == 0 ? 2 : r3 - 1;
        if (ok && it < niter) {
#pragma unroll
            for (int c = 0; c < 3; ++c)
#pragma unroll
                for (int u = 0; u < W; ++u) bo[c][u] = bn[c][u];
            // issue the next plane's B^{n-1/2} loads first: they complete during this plane's work
            if (it + 1 < niter) load_bold(pw + 1 == g.nz ? 0 : pw + 1, bn);
            // cell pairs (0, 1) and (2, 3) in f32x2 arithmetic; D*_x stays scalar (its taps are
            // shifted along x, which does not keep pairs aligned)
            u64 dz2[2], dy2[2], b2[3][2];
            float t[W];
            // own rows: the newest plane comes from shared memory (E_x, E_y of p+2; E_z of p+1)
            // and goes to TMEM; the older planes come from TMEM (at the first iteration every
            // own row comes from shared memory and is written to TMEM)
            Q4 ym_, y0_, y1_, zm_, z0_, z1_;
            const Q4 y2_ = ldq(P2 + ESLOT, e);
            z1_ = ldq(P1 + 2 * ESLOT, e);
            if (it == 0) {
                ym_ = ldq(Pm + ESLOT, e);
                y0_ = ldq(P0 + ESLOT, e);
                y1_ = ldq(P1 + ESLOT, e);
                zm_ = ldq(Pm + 2 * ESLOT, e);
                z0_ = ldq(P0 + 2 * ESLOT, e);
                tm_st(cx(0), ldq(Pm, e));
                tm_st(cx(1), ldq(P0, e));
                tm_st(cx(2), ldq(P1, e));   // read back from TMEM from the next iteration on
                tm_st(cy(0), ym_);
                tm_st(cy(1), y0_);
                tm_st(cy(2), y1_);
                tm_st(cz0, zm_);
                tm_st(cz1, z0_);
            } else {
                tm_ld(cy(0), ym_);
                tm_ld(cy(1), y0_);
                tm_ld(cy(2), y1_);
                tm_ld(cz0, zm_);
                tm_ld(cz1, z0_);
                tm_wait_ld(ym_, y0_, y1_, zm_, z0_);
            }
            tm_st(cy(3), y2_);
            tm_st(cz2, z1_);
            // B_x = B_x + (D*_z E_y - D*_y E_z)
            dstar_z2<EW>(P0 + ESLOT, P1 + ESLOT, y0_, y1_, y2_, ym_, e, lb, rb, m2.cA[2], m2.cD[2],
                      m2.cB[2][0], m2.cB[2][1], dz2);
            dstar_y2<EW>(Pm + 2 * ESLOT, P0 + 2 * ESLOT, P1 + 2 * ESLOT, z0_, z1_, zm_, e, lb, rb,
                      m2.cA[1], m2.cD[1], m2.cB[1][0], m2.cB[1][2], dy2);
#pragma unroll
            for (int h = 0; h < 2; ++h)
                b2[0][h] = add2(pk(bo[0][2 * h], bo[0][2 * h + 1]), sub2(dz2[h], dy2[h]));
            // B_y = B_y + (D*_x E_z - D*_z E_x)
            dstar_x4<EW>(Pm + 2 * ESLOT, P0 + 2 * ESLOT, P1 + 2 * ESLOT, z0_, z1_, zm_, e, lb, rb,
                     m.cA[0], m.cD[0], m.cB[0][1], m.cB[0][2], t);
            Q4 xm_, x0_, x1_;
            const Q4 x2_ = ldq(P2, e);
            if (it == 0) {   // written to TMEM in this iteration: not read back before a wait
                xm_ = ldq(Pm, e);
                x0_ = ldq(P0, e);
                x1_ = ldq(P1, e);
            } else {
                tm_ld(cx(0), xm_);
                tm_ld(cx(1), x0_);
                tm_ld(cx(2), x1_);
                tm_wait_ld(xm_, x0_, x1_);
            }
            tm_st(cx(3), x2_);
            dstar_z2<EW>(P0, P1, x0_, x1_, x2_, xm_, e, lb, rb, m2.cA[2], m2.cD[2], m2.cB[2][0],
                      m2.cB[2][1], dz2);
#pragma unroll
            for (int h = 0; h < 2; ++h)
                b2[1][h] = add2(pk(bo[1][2 * h], bo[1][2 * h + 1]), sub2(pk(t[2 * h], t[2 * h + 1]), dz2[h]));
            // B_z = B_z + (D*_y E_x - D*_x E_y)
            dstar_y2<EW>(Pm, P0, P1, x0_, x1_, xm_, e, lb, rb, m2.cA[1], m2.cD[1], m2.cB[1][0],
                      m2.cB[1][2], dy2);
            if (it == 0) {
                ym_ = ldq(Pm + ESLOT, e);
                y0_ = ldq(P0 + ESLOT, e);
                y1_ = ldq(P1 + ESLOT, e);
            } else {
                tm_ld(cy(0), ym_);
                tm_ld(cy(1), y0_);
                tm_ld(cy(2), y1_);
                tm_wait_ld(ym_, y0_, y1_);
            }
            dstar_x4<EW>(Pm + ESLOT, P0 + ESLOT, P1 + ESLOT, y0_, y1_, ym_, e, lb, rb, m.cA[0],
                     m.cD[0], m.cB[0][1], m.cB[0][2], t);
#pragma unroll
            for (int h = 0; h < 2; ++h)
                b2[2][h] = add2(pk(bo[2][2 * h], bo[2][2 * h + 1]), sub2(dy2[h], pk(t[2 * h], t[2 * h + 1])));
            if (spy != nullptr) {
                const float f = spy[b_y] * spz[pw];
                const u64 f2 = pk(f, f);
#pragma unroll
                for (int c = 0; c < 3; ++c)
#pragma unroll
                    for (int h = 0; h < 2; ++h) b2[c][h] = mul2(b2[c][h], f2);
            }
            float bxv[W], byv[W], bzv[W];
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                upk(b2[0][h], bxv[2 * h], bxv[2 * h + 1]);
                upk(b2[1][h], byv[2 * h], byv[2 * h + 1]);
                upk(b2[2][h], bzv[2 * h], bzv[2 * h + 1]);
            }
            if (b_store) {
                stv(sB + r3 * BSLOT, bi, bxv);
                stv(sB + (3 + r3) * BSLOT, bi, byv);
                stv(sB + (6 + r2) * BSLOT, bi, bzv);
            }
            if (b_own) {   // warp-uniform (warps 0-3)
                tm_st(tb + COL_BX + 4 * e3, bxv);
                tm_st(tb + COL_BY + 4 * e3, byv);
                tm_st(tb + COL_BZ + 4 * (it & 1), bzv);
            }
            if (p >= z0 && b_own) {
                const unsigned po = (unsigned)pw * plane;
                put_seg(out.c[3], po, dst, bxv);
                put_seg(out.c[4], po, dst, byv);
                put_seg(out.c[5], po, dst, bzv);
            }
        }
        // ---- E^{n+1}(p - 1): warps of the owned rows (warp-uniform condition)
        const int q = p - 1;
        if (ok && q >= z0 && q < zend && b_own) {
            const float* Bxc = sB + r3m * BSLOT;
            const float* Byc = sB + (3 + r3m) * BSLOT;
            const float* Bzc = sB + (6 + (r2 ^ 1)) * BSLOT;
            // own rows: B^{n+1/2} of planes p-1 (slot (it-1) mod 3, B_z (it-1) & 1) and p-2 (slot
            // (it-2) mod 3) and E^n of plane p-1 from TMEM; rows y-1 from the shared ring
            const int b1s = e3 == 0 ? 2 : e3 - 1, b2s = b1s == 0 ? 2 : b1s - 1;
            Q4 Bz4, By4, Byz, Bx, Bxz, E0x, E0y, E0z;
            tm_ld(tb + COL_BZ + 4 * ((it + 1) & 1), Bz4);
            tm_ld(tb + COL_BY + 4 * b1s, By4);
            tm_ld(tb + COL_BY + 4 * b2s, Byz);
            tm_ld(tb + COL_BX + 4 * b1s, Bx);
            tm_ld(tb + COL_BX + 4 * b2s, Bxz);
            tm_wait_ld(Bz4, By4, Byz, Bx, Bxz);
            tm_ld(cx(0), E0x);
            tm_ld(cy(0), E0y);
            tm_ld(cz0, E0z);
            tm_wait_ld(E0x, E0y, E0z);
            const Q4 Bzy = ldq(Bzc, bi - BW), Bxy = ldq(Bxc, bi - BW);
            float Bz[W + 1], By[W + 1];   // [0] = value at x-1, [1 + u] = cell u
#pragma unroll
            for (int u = 0; u < W; ++u) {
                Bz[1 + u] = Bz4.v[u];
                By[1 + u] = By4.v[u];
            }
            Bz[0] = from_left(Bz4.v[3]);
            By[0] = from_left(By4.v[3]);
            if (lb) {
                Bz[0] = Bzc[bi - 1];
                By[0] = Byc[bi - 1];
            }
            // ampere_comp on cell pairs: e + fma(c1, p0 - pm, -(c2 (q0 - qm)))
            float ex[W], ey[W], ez[W];
            auto amp2 = [](u64 e2, u64 dp, u64 dq, u64 c1, u64 nc2) {
                return add2(e2, fma2(c1, dp, mul2(nc2, dq)));
            };
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const int u = 2 * h;
                const u64 rx = amp2(pk(E0x.v[u], E0x.v[u + 1]),
                                    sub2(pk(Bz[1 + u], Bz[2 + u]), pk(Bzy.v[u], Bzy.v[u + 1])),
                                    sub2(pk(By[1 + u], By[2 + u]), pk(Byz.v[u], Byz.v[u + 1])),
                                    m2.cE[1], m2.ncE[2]);
                const u64 ry = amp2(pk(E0y.v[u], E0y.v[u + 1]),
                                    sub2(pk(Bx.v[u], Bx.v[u + 1]), pk(Bxz.v[u], Bxz.v[u + 1])),
                                    pk(Bz[1 + u] - Bz[u], Bz[2 + u] - Bz[1 + u]), m2.cE[2], m2.ncE[0]);
                const u64 rz = amp2(pk(E0z.v[u], E0z.v[u + 1]),
                                    pk(By[1 + u] - By[u], By[2 + u] - By[1 + u]),
                                    sub2(pk(Bx.v[u], Bx.v[u + 1]), pk(Bxy.v[u], Bxy.v[u + 1])),
                                    m2.cE[0], m2.ncE[1]);
                upk(rx, ex[u], ex[u + 1]);
                upk(ry, ey[u], ey[u + 1]);
                upk(rz, ez[u], ez[u + 1]);
            }
            const int i0 = x0 + b_bx, j = y0 + b_by;
            if (jx_row != nullptr) {
                float jv[W];
                unpackv(__ldg(reinterpret_cast<const float4*>(jx_row + i0)), jv);
                const float sy = jyz[j], sz = jyz[g.ny + qw];
#pragma unroll
                for (int u = 0; u < W; ++u) ex[u] = fma(mdt, (jv[u] * sy) * sz, ex[u]);
            }
            if (spy != nullptr) {
                const float f = spy[j] * spz[qw];
#pragma unroll
                for (int u = 0; u < W; ++u) { ex[u] *= f; ey[u] *= f; ez[u] *= f; }
            }
#pragma unroll
            for (int u = 0; u < W; ++u)
                fin = nonfinite_acc(nonfinite_acc(nonfinite_acc(fin, ex[u]), ey[u]), ez[u]);
            const unsigned po = (unsigned)qw * plane;
            put_seg(out.c[0], po, dst, ex);
            put_seg(out.c[1], po, dst, ey);
            put_seg(out.c[2], po, dst, ez);
            if (h0 != nullptr) {
                put_seg(h0, po, dst, ex);
                put_seg(h1, po, dst, ey);
                put_seg(h2, po, dst, ez);
            }
        }
        tm_wait_st();
        bool ok_next = true;
        if (tid == PRODUCER && it + 1 < niter)
            ok_next = mbar_wait(&bar[(it + 1) % NS], (uint32_t)(((it + 1) / NS) & 1));
        if (__syncthreads_or(!ok || !ok_next)) {
            failed = true;
            break;
        }
        if (tid == PRODUCER && it + D + 1 < niter) {
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            issue_unit(it + D + 1);
            issued = it + D + 2;
        }
        if (tid == PRODUCER) {
            pf_e(z0 + 3 + it + PF);
            pf_b(z0 + it + PF);
        }
    }
    if (!(fin == 0.0f)) atomicOr(err, ERR_FIELD);
    if (failed) {
        // the state written by this launch is not valid; drain this CTA's copies in flight
        if (tid == PRODUCER) {
            atomicOr(err, ERR_WAIT);
            if (it == 0) mbar_wait(&bar[NS], 0);
            for (int u = it; u < issued; ++u) mbar_wait(&bar[u % NS], (uint32_t)((u / NS) & 1));
        }
        __syncthreads();
    }
    // release the TMEM columns (every path reaches this point)
    tm_wait_st();
    tm_fence_before();
    __syncthreads();
    tm_fence_after();
    if (tid < 32) tm_dealloc<TM_COLS>(tm_base);
}

}  // namespace f32seg

bool fused32_supported(const Geom& g) {
    // 32-bit element offsets inside the kernel
    return g.nx % f32seg::TX == 0 && g.ny % f32seg::TY == 0 && g.nx >= f32seg::TX &&
           g.ny >= f32seg::TY && g.total < (1LL << 31);
}

int fused32_ebox_w() { return f32seg::EW; }

bool fused32_prepare() {
    return cudaFuncSetAttribute(f32seg::step_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)f32seg::SMEM) == cudaSuccess;
}

int resident_slots(const void* kernel, int threads, size_t smem) {
    int dev = 0, sms = 0, per_sm = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, threads, smem) != cudaSuccess ||
        sms <= 0 || per_sm <= 0)
        return 0;
    return sms * per_sm;
}

// Resident CTAs of the step kernel on the whole device, from its own limits: shared memory
// (with the per-CTA reservation), registers (allocated per warp in units of 256), threads, the
// CTA limit and its TMEM columns (512 per SM).  The occupancy API is not used here: for a
// kernel that allocates tensor memory it reports fewer resident CTAs than actually run (one
// where three fit), which made the z-chunk choice launch too few CTAs on small grids.
int resident_slots_tmem(const void* kernel, int threads, size_t smem, int tmem_cols) {
    int dev = 0, sms = 0, smem_sm = 0, resv = 0, regs_sm = 0, thr_sm = 0, blk_sm = 0;
    cudaFuncAttributes fa;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&smem_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&resv, cudaDevAttrReservedSharedMemoryPerBlock, dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&regs_sm, cudaDevAttrMaxRegistersPerMultiprocessor, dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&thr_sm, cudaDevAttrMaxThreadsPerMultiProcessor, dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&blk_sm, cudaDevAttrMaxBlocksPerMultiprocessor, dev) != cudaSuccess ||
        cudaFuncGetAttributes(&fa, kernel) != cudaSuccess || sms <= 0)
        return 0;
    const long long per_cta_smem = (long long)smem + fa.sharedSizeBytes + resv;
    const int warps = (threads + 31) / 32;
    const long long regs_warp = ((long long)fa.numRegs * 32 + 255) / 256 * 256;
    int n = blk_sm;
    if (per_cta_smem > 0) n = (int)std::min<long long>(n, smem_sm / per_cta_smem);
    if (regs_warp > 0) n = (int)std::min<long long>(n, regs_sm / (regs_warp * warps));
    n = std::min(n, thr_sm / (warps * 32));
    n = std::min(n, 512 / tmem_cols);
    return n > 0 ? sms * n : 0;
}

int zchunk_len(int tiles_xy, int nz, int slots, int tz_min, int tz_max) {
    // A CTA marches tz planes plus about two planes of fixed cost (the z-halo B plane and the
    // prologue copies); CTAs run in waves of `slots`.  Minimise waves x (tz + 2) over chunk
    // lengths tz_min..tz_max; ties go to the longer chunk.
    const int hi = nz < tz_max ? nz : tz_max;
    if (slots <= 0) return hi;
    int best = hi;
    long long best_cost = -1;
    for (int tz = hi; tz >= tz_min || tz == nz; --tz) {
        const long long ctas = (long long)tiles_xy * ((nz + tz - 1) / tz);
        const long long waves = (ctas + slots - 1) / slots;
        const long long cost = waves * (tz + 2);
        if (best_cost < 0 || cost < best_cost) {
            best_cost = cost;
            best = tz;
        }
        if (tz <= 1) break;
    }
    return best;
}

static int fused32_tz(const Geom& g) {
    using namespace f32seg;
    static int slots = -1;
    if (slots < 0) slots = resident_slots_tmem((const void*)step_kernel, NT, SMEM, TM_COLS);
    // measured at 256^3 (456 resident CTAs): 37-plane chunks (2 full waves) 0.218 ms per step,
    // 32-plane chunks (2.25 waves) 0.269 ms
    return zchunk_len((g.nx / TX) * (g.ny / TY), g.nz, slots, 16, 64);
}

void launch_fused32(const FusedMaps& maps, FieldSet<float> in, const Geom& g, const Mult<float>& m,
                    FieldSet<float> out, const float* spy, const float* spz, const float* jyz,
                    const float* jx_row, float* hist_E[3], int* err, cudaStream_t st) {
    using namespace f32seg;
    const int tz = fused32_tz(g);
    const int nblk = (g.nx / TX) * (g.ny / TY) * ((g.nz + tz - 1) / tz);
    step_kernel<<<nblk, NT, SMEM, st>>>(maps, g, m, make_mult2(m), in, out, spy, spz, jyz, jx_row, hist_E[0],
                                        hist_E[1], hist_E[2], 0, g.nz, tz, err);
}

// One leapfrog step on the planes zs .. ze-1 only (no current, no history): the slab launches
// of the temporally blocked schedule.  The z-chunk length fills the resident slots best for a
// slab of that length.
void launch_fused32_range(const FusedMaps& maps, FieldSet<float> in, const Geom& g,
                          const Mult<float>& m, FieldSet<float> out, const float* spy,
                          const float* spz, int zs, int ze, int* err, cudaStream_t st) {
    using namespace f32seg;
    static int slots = -1;
    if (slots < 0) slots = resident_slots_tmem((const void*)step_kernel, NT, SMEM, TM_COLS);
    const int tiles = (g.nx / TX) * (g.ny / TY);
    const int len = ze - zs;
    const int tz = zchunk_len(tiles, len, slots, 2, 64);
    const int nblk = tiles * ((len + tz - 1) / tz);
    step_kernel<<<nblk, NT, SMEM, st>>>(maps, g, m, make_mult2(m), in, out, spy, spz, nullptr,
                                        nullptr, nullptr, nullptr, nullptr, zs, ze, tz, err);
}

}  // namespace fdtd
