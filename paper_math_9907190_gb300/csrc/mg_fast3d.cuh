// mg_fast3d.cuh -- z-streaming kernels of the 3D diagonal hierarchy (FP32
// levels).  A thread block owns a TX x TY column of one level and walks a
// range of z planes upward; the planes a stencil chain needs are kept in
// shared-memory rings, and the next plane's inputs are copied in (cp.async)
// while the current one is computed.  Compared with a 3D tile, no z halo is
// loaded or computed twice except at the start of a z range.
#pragma once
#include "mg_fast2d.cuh"

namespace mg {

constexpr int GS_TX = 32, GS_TY = 16;            // output tile of a block (green points)
constexpr int GS_RH = GS_TY + 6;                 // red rows: tile +- 3
constexpr int GS_RC = GS_TX / 2 + 8;             // red values per row: 16-byte chunks over the tile +- 3
constexpr int GS_VW = GS_TX + 4, GS_VH = GS_TY + 4;  // F region: tile +- 2
constexpr int GS_GW = GS_TX + 8;                 // residual row: 16-byte chunks over x0-5 .. x0+34
// steps before the first output plane: the rings start with red planes
// z+1..z+3 and residual plane z+2, so F is right from the first step; the
// carried residual of plane z needs C of plane z-1, hence F from z-2
constexpr int GS_WARM = 3, GS_WARM_RR = 4;

struct GreenSSmem {
    // red planes z+1..z+4 (ring, slot = plane & 3): fine row y holds its red
    // points x (x = y + plane mod 2) at index (x >> 1) - (16 bx - 4)
    float red[4][GS_RH][GS_RC];
    float r[4][GS_VH][GS_GW];    // green residual planes z..z+3 (ring), x from x0 - 4
    float v[4][GS_VH][GS_VW];    // correction planes z-1..z+2 (ring): F at odd, C at even points
};

// Green-red sweep of a triple's green level (Eq. Egprolg, then Eq. Egprolr,
// c = p_g h^2), z-streaming.  Step z of a block: F (odd index sum) on plane
// z+2 over the tile +- 2 from the red planes z+1..z+3; C (even) on plane z+1
// over the tile +- 1 from the F values of planes z..z+2; then the tile of
// plane z is final.  MODE: UP_RR the mixed finest triple (u += v and the
// carried float-float residual r -= L v as in k_up_ff_2d, six neighbours;
// rga/rgb double-buffered by par); UP_ADD u += v; UP_STORE v stored in vg.
// A block's z range holds zch output planes; its first GS_WARM (UP_RR:
// GS_WARM_RR) steps fill the rings (nothing is written).  The tile's x range
// starts at a multiple of 32 (x = 0 is the ring), so that a thread's two
// adjacent output points are one aligned pair of every array; VU: u is
// 16-byte aligned with an even pitch (vector access to u).
template <int MODE, bool VU>
__global__ void __launch_bounds__(256) k_green_ff_3d(Red3<const float> vr, A3<float> rga, float *rgb, A3<float> vg,
                                                     float *__restrict__ rlo, double *__restrict__ u, int up, int n,
                                                     float cg, float s2, int zch, double *part, Ctrl *ctl,
                                                     CtrlFuse cf, const int *done, Bt B) {
    extern __shared__ __align__(16) unsigned char smraw[];
    GreenSSmem &S = *reinterpret_cast<GreenSSmem *>(smraw);
    __shared__ double sh[32];
    __shared__ float shm[32];
    constexpr bool RR = MODE == UP_RR, UPD = MODE != UP_STORE;
    constexpr int FPR = GS_VW / 2, NF = GS_VH * FPR;               // F points per row, per plane
    constexpr int CPR = (GS_VW - 2) / 2, NC = (GS_VH - 2) * CPR;   // C points per row, per plane
    constexpr int RCH = GS_RC / 4, GCH = GS_GW / 4;                // 16-byte chunks per red / residual row
    const int prob = bt_prob(B), zc = bt_z(B);
    if (stop(bt_done(done, prob, B))) return;
    A3<float> rg = rga, rnew = rga;
    int pq = 0;      // current residual buffer
    float M = 0.f;   // quantizer of v (quant_magic): |v| <= |red| + cg max|r| / 3
    if (RR) {
        const Ctrl &C = ctl[prob];
        pq = C.par;
        (pq ? rg : rnew).p = rgb;
        M = quant_magic((__uint_as_float(C.vmax) + cg * (1.f / 3.f) * __uint_as_float(C.rmax[pq])) * 1.002f, 20);
    }
    vr = bt_at(vr, prob, B);
    rg = bt_at(rg, prob, B); rnew = bt_at(rnew, prob, B); vg = bt_at(vg, prob, B);
    if (RR) rlo = bt_ptr(rlo, prob, B);
    if (UPD && B.utab) u = B.utab[prob];
    if (RR) part += (size_t)prob * B.nparts;
    const int tx = threadIdx.x, ty = threadIdx.y, tid = tx + 32 * ty;
    const int x0 = blockIdx.x * GS_TX, y0 = blockIdx.y * GS_TY + 1;
    const int zb = zc * zch + 1, ze = min(zb + zch, n + 1);  // output planes [zb, ze)
    const int zs = zb - (RR ? GS_WARM_RR : GS_WARM);
    const size_t rows = (size_t)(n + 2), upl = (size_t)up * rows, gpl = (size_t)rg.pitch * rows;
    const size_t cpl = (size_t)vr.eee.pitch * vr.eee.rows;  // the four red cosets share their layout
    // the F region (tile +- 2) lies in the interior: no bounds tests but the plane's
    const bool inner = x0 >= 3 && x0 + GS_TX + 1 <= n && y0 >= 3 && y0 + GS_TY + 1 <= n;

    // ---- per-thread work items, fixed for all planes
    // red copy: fine row y0-3+ly, 16-byte chunk j of coset values (x >> 1) from 16 bx - 4
    const int rq_ly = tid / RCH, rq_j = tid - rq_ly * RCH, rq_y = y0 - 3 + rq_ly;
    const bool rq_on = tid < GS_RH * RCH;
    const bool rq_ok = rq_on && rq_y >= 0 && rq_y <= n + 1 && (x0 >> 1) - 4 + 4 * rq_j >= 0;
    const size_t rq_off = rq_ok ? (size_t)(rq_y >> 1) * vr.eee.pitch + ((x0 >> 1) - 4 + 4 * rq_j) : 0;
    // residual copy: row y0-2+ly, chunk j of x from x0 - 4
    const int gq_ly = tid / GCH, gq_j = tid - gq_ly * GCH, gq_y = y0 - 2 + gq_ly, gq_x = x0 - 4 + 4 * gq_j;
    const bool gq_on = tid < GS_VH * GCH;
    const bool gq_ok = gq_on && gq_x >= 0 && gq_y >= 0 && gq_y <= n + 1;
    const size_t gq_off = gq_ok ? (size_t)gq_y * rg.pitch + gq_x : 0;
    // output points: row oy of the tile, columns 2 ox and 2 ox + 1
    const int ox = tid & 15, oy = tid >> 4;
    // F items (row ly, k-th point of the row's parity) and C items
    int f_ly[2], f_k[2], f_pb[2], c_ly[2], c_k[2], c_pb[2];
#pragma unroll
    for (int i = 0; i < 2; i++) {
        const int q = tid + 256 * i;
        f_ly[i] = q / FPR; f_k[i] = q - f_ly[i] * FPR; f_pb[i] = (x0 - 1 + y0 - 2 + f_ly[i]) & 1;
        c_ly[i] = q / CPR + 1; c_k[i] = q - (c_ly[i] - 1) * CPR; c_pb[i] = (x0 - 1 + y0 - 2 + c_ly[i]) & 1;
    }

    // copy red plane zp and residual plane zr into their ring slots (16-byte
    // chunks of the dense coset / level rows; chunks outside the arrays are
    // zero-filled, and only values at interior points or the zero ring are
    // used), and u / lo of output plane zo when it is one
    auto red_copy = [&](int zp) {
        if (rq_on) {
            const bool ok = rq_ok && zp >= 0 && zp <= n + 1;
            // the coset holding row y of plane zp: EEE, OOE (zp even), OEO, EOO (zp odd)
            const float *C = (zp & 1) ? ((rq_y & 1) ? vr.eoo.p : vr.oeo.p) : ((rq_y & 1) ? vr.ooe.p : vr.eee.p);
            cp_async16(&S.red[zp & 3][rq_ly][4 * rq_j], ok ? C + (size_t)(zp >> 1) * cpl + rq_off : C, ok);
        }
    };
    auto issue = [&](int zp, int zr) {
        red_copy(zp);
        if (gq_on) {
            const bool ok = gq_ok && zr >= 0 && zr <= n + 1;
            cp_async16(&S.r[zr & 3][gq_ly][4 * gq_j], ok ? rg.p + (size_t)zr * gpl + gq_off : rg.p, ok);
        }
        cp_async_commit();
    };

    // ring slots not written by a step before they are read hold zeros
    for (int q = tid; q < (int)(sizeof(GreenSSmem) / 4); q += 256) reinterpret_cast<float *>(smraw)[q] = 0.f;
    __syncthreads();
    red_copy(zs + 1);
    red_copy(zs + 2);
    issue(zs + 3, zs + 2);
    float sq = 0.f, mx = 0.f;
    for (int z = zs; z < ze; z++) {
        cp_async_wait0();
        __syncthreads();                             // step z's planes landed; step z-1 is done with every slot
        if (z + 1 < ze) issue(z + 4, z + 3);  // the next step's planes, in flight during this one
        // u and lo of the thread's output points of plane z, loaded into
        // registers now and used after the F and C phases (their latency
        // hidden by that work)
        const int xo = x0 + 2 * ox, yo = y0 + oy;
        const bool outp = z >= zb && xo <= n && yo <= n;
        double2 uo = make_double2(0.0, 0.0);
        float2 lo2 = make_float2(0.f, 0.f);
        if (UPD && outp) {
            const double *us = u + (size_t)z * upl + (size_t)yo * up + xo;
            if (VU) uo = *reinterpret_cast<const double2 *>(us);
            else { uo.x = us[0]; uo.y = us[1]; }
            if (RR) lo2 = *reinterpret_cast<const float2 *>(rlo + (size_t)z * gpl + (size_t)yo * rg.pitch + xo);
        }
        // F on plane z+2, tile +- 2: the red neighbours of the k-th F point of
        // a row are the row's red values k+2+p, k+3+p and value k+3 of rows
        // y +- 1 and of planes z+1, z+3 (p: x parity offset of the row)
        {
            const int zf = z + 2;
            const bool zin = zf >= 1 && zf <= n;
            const float(&Rm)[GS_RH][GS_RC] = S.red[(zf - 1) & 3];
            const float(&R0)[GS_RH][GS_RC] = S.red[zf & 3];
            const float(&Rp)[GS_RH][GS_RC] = S.red[(zf + 1) & 3];
            const float(&G)[GS_VH][GS_GW] = S.r[zf & 3];
            float(&V)[GS_VH][GS_VW] = S.v[zf & 3];
#pragma unroll
            for (int i = 0; i < 2; i++) {
                if (i == 1 && tid + 256 >= NF) break;
                const int ly = f_ly[i], k = f_k[i], p = f_pb[i] ^ (zf & 1), lx = p + 2 * k;
                const int x = x0 - 2 + lx, y = y0 - 2 + ly;
                float val = 0.f;
                if (zin && (inner || (x >= 1 && x <= n && y >= 1 && y <= n))) {
                    const int ry = ly + 1, ac = k + 2 + p;
                    const float s = (R0[ry][ac] + R0[ry][ac + 1]) + (R0[ry - 1][k + 3] + R0[ry + 1][k + 3]) +
                                    (Rm[ry][k + 3] + Rp[ry][k + 3]);
                    val = (s - cg * G[ly][lx + 2]) * (1.f / 6.f);
                }
                V[ly][lx] = RR ? quant(val, M) : val;
            }
        }
        __syncthreads();
        // C on plane z+1, tile +- 1
        {
            const int zq = z + 1;
            const bool zin = zq >= 1 && zq <= n;
            const float(&Vm)[GS_VH][GS_VW] = S.v[(zq - 1) & 3];
            const float(&Vp)[GS_VH][GS_VW] = S.v[(zq + 1) & 3];
            const float(&G)[GS_VH][GS_GW] = S.r[zq & 3];
            float(&V)[GS_VH][GS_VW] = S.v[zq & 3];
#pragma unroll
            for (int i = 0; i < 2; i++) {
                if (i == 1 && tid + 256 >= NC) break;
                const int ly = c_ly[i], lx = 1 + (c_pb[i] ^ (zq & 1)) + 2 * c_k[i];
                const int x = x0 - 2 + lx, y = y0 - 2 + ly;
                float val = 0.f;
                if (zin && (inner || (x >= 1 && x <= n && y >= 1 && y <= n))) {
                    const float s = (V[ly][lx - 1] + V[ly][lx + 1]) + (V[ly - 1][lx] + V[ly + 1][lx]) +
                                    (Vm[ly][lx] + Vp[ly][lx]);
                    val = (s - cg * G[ly][lx + 2]) * (1.f / 6.f);
                }
                V[ly][lx] = RR ? quant(val, M) : val;
            }
        }
        __syncthreads();
        // plane z is final on the tile: a thread's points (x, y), (x + 1, y),
        // x = x0 + 2 ox even; x = 0 is the ring, and x <= n implies x + 1 <= n
        if (z >= zb) {
            if (outp) {
                const float(&V)[GS_VH][GS_VW] = S.v[z & 3];
                const int lx = 2 * ox + 2, ly = oy + 2;
                const float2 c = *reinterpret_cast<const float2 *>(&V[ly][lx]);
                const bool lft = xo >= 1;  // (x, y) is interior
                float2 nh2 = make_float2(0.f, 0.f), nl2 = make_float2(0.f, 0.f);
                if (RR) {
                    const float(&Vm)[GS_VH][GS_VW] = S.v[(z - 1) & 3];
                    const float(&Vp)[GS_VH][GS_VW] = S.v[(z + 1) & 3];
                    const float2 dn = *reinterpret_cast<const float2 *>(&V[ly - 1][lx]);
                    const float2 upr = *reinterpret_cast<const float2 *>(&V[ly + 1][lx]);
                    const float2 zm = *reinterpret_cast<const float2 *>(&Vm[ly][lx]);
                    const float2 zp = *reinterpret_cast<const float2 *>(&Vp[ly][lx]);
                    const float2 g = *reinterpret_cast<const float2 *>(&S.r[z & 3][ly][lx + 2]);
                    const float2 l = lo2;
                    // Laplacian of the quantized v: exact (quant_magic, qb = 20)
                    const float sa = __fadd_rn(__fadd_rn(__fadd_rn(V[ly][lx - 1], c.y), __fadd_rn(dn.x, upr.x)),
                                               __fadd_rn(zm.x, zp.x));
                    const float sb = __fadd_rn(__fadd_rn(__fadd_rn(c.x, V[ly][lx + 2]), __fadd_rn(dn.y, upr.y)),
                                               __fadd_rn(zm.y, zp.y));
                    ff_sub1(g.x, l.x, fmaf(-6.f, c.x, sa), s2, nh2.x, nl2.x);
                    ff_sub1(g.y, l.y, fmaf(-6.f, c.y, sb), s2, nh2.y, nl2.y);
                    if (!lft) nh2.x = nl2.x = 0.f;
                    sq = fmaf(nh2.x, nh2.x, fmaf(nh2.y, nh2.y, sq));
                    mx = fmaxf(mx, fmaxf(fabsf(nh2.x), fabsf(nh2.y)));
                    const size_t o = (size_t)z * gpl + (size_t)yo * rg.pitch + xo;
                    if (lft) {
                        *reinterpret_cast<float2 *>(rlo + o) = nl2;
                        *reinterpret_cast<float2 *>(rnew.p + o) = nh2;
                    } else {
                        rlo[o + 1] = nl2.y;
                        rnew.p[o + 1] = nh2.y;
                    }
                }
                if (UPD) {
                    double *ud = u + (size_t)z * upl + (size_t)yo * up + xo;
                    const double ub = uo.y + widen(c.y);
                    if (VU && lft) {
                        *reinterpret_cast<double2 *>(ud) = make_double2(uo.x + widen(c.x), ub);
                    } else {
                        if (lft) ud[0] = uo.x + widen(c.x);
                        ud[1] = ub;
                    }
                } else {
                    *reinterpret_cast<float2 *>(&vg(xo, yo, z)) = c;  // v = 0 at the ring point x = 0
                }
            }
        }
    }
    if (RR) {
        const double s = block_sum((double)sq, sh);
        const float m = block_max(mx, shm);
        if (tid == 0) {
            part[blockIdx.x + gridDim.x * (blockIdx.y + (size_t)gridDim.y * zc)] = s;
            atomicMax(&ctl[prob].rmax[pq ^ 1], __float_as_uint(m));
        }
        if (cf.arrive) ctrl_last_block(cf, ctl + prob, part, gridDim.x * gridDim.y * gridDim.z, sh);  // one problem only
    }
}

}  // namespace mg


namespace mg {

// ---------------------------------------------------------------------------
// Per-stage kernels of the 3D triple, z-marching: a thread owns one cell
// column (a, b) over zm consecutive cell planes, forms each array's
// address once and steps it by one plane; values of the previous plane that
// the next one needs stay in registers.  The arithmetic of every value is the
// one of the stage kernels in mg_stages.cuh, term for term.  All coset arrays
// of a triple (and its blue level) share one layout: pitch P, plane Q = P *
// rows.  Grid: (cells + 31) / 32 x (cells + 7) / 8 x ceil(planes / zm) per
// problem, block 32 x 8.
// ---------------------------------------------------------------------------
struct ZmIdx {
    int a, b, c0, c1;  // cell column and plane range [c0, c1)
    size_t i;          // linear index of (a, b, c0)
};
// cells of the column range [lo, hi] in a and b, planes [lo, hi] in c, zm
// planes per thread
__device__ __forceinline__ bool zm_cell(ZmIdx &z, int lo, int hi, int zm, int P, size_t Q, const Bt &B) {
    z.a = blockIdx.x * 32 + threadIdx.x + lo;
    z.b = blockIdx.y * 8 + threadIdx.y + lo;
    z.c0 = bt_z(B) * zm + lo;
    z.c1 = min(z.c0 + zm, hi + 1);
    z.i = (size_t)z.c0 * Q + (size_t)z.b * P + z.a;
    return z.a <= hi && z.b <= hi;
}

// Eq. Erred (green -> red), cells [0, nb]^3; green g has its own layout
template <typename T>
__global__ void __launch_bounds__(256) k_g2r_zm_3d(A3<const T> g, Red3<T> red, int nb, const T *galt, const int *par,
                                                   int zm, const int *done, Bt B) {
    const int prob = bt_prob(B);
    if (stop(bt_done(done, prob, B))) return;
    if (galt && par[(size_t)prob * B.ctl_stride]) g.p = galt;
    g = bt_at(g, prob, B);
    red = bt_at(red, prob, B);
    const int P = red.eee.pitch;
    const size_t Q = (size_t)P * red.eee.rows;
    ZmIdx z;
    if (!zm_cell(z, 0, nb, zm, P, Q, B)) return;
    const int gp = g.pitch;
    const size_t gq = (size_t)gp * g.rows;
    // the 20 distinct green values of a cell (X, Y, Z) = (2a, 2b, 2c) are
    // loaded once, before any store; the 4 of planes Z+1 and Z+2 that the
    // next cell up reads again are carried over in registers
    auto avg = [](T c, T x0, T x1, T y0, T y1, T z0, T z1) {
        return (T(6) * c + (x1 + x0) + (y1 + y0) + (z1 + z0)) * T(1.0 / 12.0);
    };
    const T *ge = g.p + ((size_t)(2 * z.c0) * g.rows + 2 * z.b) * gp + 2 * z.a;  // green (2a, 2b, 2c0)
    // carried: (X, Y, Z-1), (X+1, Y+1, Z-1), (X+1, Y, Z), (X, Y+1, Z).  Values
    // at index -1 (read only by ring points: a, b or c = 0) are not loaded.
    const bool ax = z.a >= 1, by = z.b >= 1;
    T czm = T(0), czm11 = T(0), cz10 = ge[1], cz01 = ge[gp];
    if (z.c0 >= 1) { czm = ge[-(long)gq]; czm11 = ge[1 + gp - (long)gq]; }
    size_t i = z.i;
    for (int c = z.c0; c < z.c1; c++, i += Q, ge += 2 * gq) {
        const T *g1 = ge + gq, *g2 = ge + 2 * gq;
        // plane Z
        const T e = ge[0], exm = ax ? ge[-1] : T(0), eym = by ? ge[-gp] : T(0), e11 = ge[1 + gp], e21 = ge[2 + gp],
                e12 = ge[1 + 2 * gp];
        // plane Z+1
        const T u00 = g1[0], u11 = g1[1 + gp], u10 = g1[1], u20 = g1[2], u1m = by ? g1[1 - gp] : T(0), u01 = g1[gp],
                um1 = ax ? g1[-1 + gp] : T(0), u02 = g1[2 * gp];
        // plane Z+2
        const T w10 = g2[1], w01 = g2[gp];
        const T veee = avg(e, exm, cz10, eym, cz01, czm, u00);
        const T vooe = avg(e11, cz01, e21, cz10, e12, czm11, u11);
        const T voeo = avg(u10, u00, u20, u1m, u11, cz10, w10);
        const T veoo = avg(u01, um1, u11, u00, u02, cz01, w01);
        if (z.a >= 1 && z.b >= 1 && c >= 1) red.eee.p[i] = veee;
        if (c >= 1) red.ooe.p[i] = vooe;
        if (z.b >= 1) red.oeo.p[i] = voeo;
        if (z.a >= 1) red.eoo.p[i] = veoo;
        czm = u00; czm11 = u11; cz10 = w10; cz01 = w01;
    }
}

// Eq. Ermagc (corners) and Eq. Ermagm (centres), cells [0, nb]^3
template <typename T>
__global__ void __launch_bounds__(256) k_r2m_zm_3d(Red3<const T> red, Mag3<T> mag, int nb, int zm, const int *done, Bt B) {
    const int prob = bt_prob(B);
    if (stop(bt_done(done, prob, B))) return;
    red = bt_at(red, prob, B);
    mag = bt_at(mag, prob, B);
    const int P = red.eee.pitch;
    const size_t Q = (size_t)P * red.eee.rows;
    ZmIdx z;
    if (!zm_cell(z, 0, nb, zm, P, Q, B)) return;
    const T *eee = red.eee.p, *ooe = red.ooe.p, *oeo = red.oeo.p, *eoo = red.eoo.p;
    size_t i = z.i;
    for (int c = z.c0; c < z.c1; c++, i += Q) {
        if (z.a >= 1 && z.b >= 1 && c >= 1) {
            const T s1 = (ooe[i - P - 1] + ooe[i - P]) + (ooe[i - 1] + ooe[i]);
            const T s2 = (oeo[i - Q - 1] + oeo[i - Q]) + (oeo[i - 1] + oeo[i]);
            const T s3 = (eoo[i - Q - P] + eoo[i - Q]) + (eoo[i - P] + eoo[i]);
            mag.eee.p[i] = (T(12) * eee[i] + (s1 + s2 + s3)) * T(1.0 / 24.0);
        }
        mag.ooo.p[i] = ((eoo[i] + eoo[i + 1]) + (oeo[i] + oeo[i + P]) + (ooe[i] + ooe[i + Q])) * T(1.0 / 6.0);
    }
}

// Eq. Erblu (magenta -> blue), cells [1, nb]^3; blue shares the coset layout
template <typename T>
__global__ void __launch_bounds__(256) k_m2b_zm_3d(Mag3<const T> mag, A3<T> blue, int nb, int zm, const int *done, Bt B) {
    const int prob = bt_prob(B);
    if (stop(bt_done(done, prob, B))) return;
    mag = bt_at(mag, prob, B);
    blue = bt_at(blue, prob, B);
    const int P = mag.eee.pitch;
    const size_t Q = (size_t)P * mag.eee.rows;
    ZmIdx z;
    if (!zm_cell(z, 1, nb, zm, P, Q, B)) return;
    const T *ooo = mag.ooo.p;
    size_t i = z.i;
    // the four centres of plane c-1 (a sum carried from the previous plane)
    auto quad = [&](size_t k) { return (ooo[k - P - 1] + ooo[k - P]) + (ooo[k - 1] + ooo[k]); };
    T lower = quad(i - Q);
    for (int c = z.c0; c < z.c1; c++, i += Q) {
        const T upper = quad(i);
        blue.p[i] = (T(8) * mag.eee.p[i] + (lower + upper)) * T(0.0625);
        lower = upper;
    }
}

// Eq. Emprolm: magenta centres from the 8 blue corners, cells [0, nb]^3
template <typename T>
__global__ void __launch_bounds__(256) k_b2m_ooo_zm_3d(A3<const T> blue, A3<const T> rooo, A3<T> vooo, int nb, T cc,
                                                       int zm, const int *done, Bt B) {
    const int prob = bt_prob(B);
    if (stop(bt_done(done, prob, B))) return;
    blue = bt_at(blue, prob, B); rooo = bt_at(rooo, prob, B); vooo = bt_at(vooo, prob, B);
    const int P = rooo.pitch;
    const size_t Q = (size_t)P * rooo.rows;
    ZmIdx z;
    if (!zm_cell(z, 0, nb, zm, P, Q, B)) return;
    const T *bl = blue.p;
    size_t i = z.i;
    // the four corners of plane c+1 become those of plane c at the next step
    auto quad = [&](size_t k) { return (bl[k] + bl[k + 1]) + (bl[k + P] + bl[k + P + 1]); };
    T lower = quad(i);
    for (int c = z.c0; c < z.c1; c++, i += Q) {
        const T upper = quad(i + Q);
        vooo.p[i] = ((lower + upper) - cc * rooo.p[i]) * T(0.125);
        lower = upper;
    }
}

// Eq. Emprolb: blue corners refined from the 8 new centres, cells [1, nb]^3
template <typename T>
__global__ void __launch_bounds__(256) k_b2m_eee_zm_3d(A3<const T> vooo, A3<const T> reee, A3<T> veee, int nb, T cc,
                                                       int zm, const int *done, Bt B) {
    const int prob = bt_prob(B);
    if (stop(bt_done(done, prob, B))) return;
    vooo = bt_at(vooo, prob, B); reee = bt_at(reee, prob, B); veee = bt_at(veee, prob, B);
    const int P = reee.pitch;
    const size_t Q = (size_t)P * reee.rows;
    ZmIdx z;
    if (!zm_cell(z, 1, nb, zm, P, Q, B)) return;
    const T *o = vooo.p;
    size_t i = z.i;
    auto quad = [&](size_t k) { return (o[k - P - 1] + o[k - P]) + (o[k - 1] + o[k]); };
    T lower = quad(i - Q);  // carried from plane to plane
    for (int c = z.c0; c < z.c1; c++, i += Q) {
        const T upper = quad(i);
        veee.p[i] = ((lower + upper) - cc * reee.p[i]) * T(0.125);
        lower = upper;
    }
}

// Eq. Erprolr and its cyclic permutations: red face centres, cells [0, nb]^3
template <typename T>
__global__ void __launch_bounds__(256) k_m2r_faces_zm_3d(Mag3<const T> vm, Red3<const T> rr, Red3<T> vr, int nb, T c1,
                                                         int zm, const int *done, Bt B) {
    const int prob = bt_prob(B);
    if (stop(bt_done(done, prob, B))) return;
    vm = bt_at(vm, prob, B); rr = bt_at(rr, prob, B); vr = bt_at(vr, prob, B);
    const int P = vm.eee.pitch;
    const size_t Q = (size_t)P * vm.eee.rows;
    ZmIdx z;
    if (!zm_cell(z, 0, nb, zm, P, Q, B)) return;
    const T *o = vm.ooo.p, *e = vm.eee.p;
    size_t i = z.i;
    // carried from plane c-1: centre (a,b,c-1) and corners (a,b,c), (a+1,b,c),
    // (a,b+1,c); index -1 values (read only for a, b or c = 0) are not loaded
    const bool ax = z.a >= 1, by = z.b >= 1;
    T om = z.c0 >= 1 ? o[i - Q] : T(0), e00 = e[i], e10 = e[i + 1], e01 = e[i + P];
    for (int c = z.c0; c < z.c1; c++, i += Q) {
        const T oc = o[i], e11 = e[i + P + 1], u00 = e[i + Q], u10 = e[i + Q + 1], u01 = e[i + Q + P];
        const T oy = by ? o[i - P] : T(0), ox = ax ? o[i - 1] : T(0);
        if (c >= 1)  // (2a+1, 2b+1, 2c): normal z
            vr.ooe.p[i] = (T(2) * (om + oc) + ((e00 + e10) + (e01 + e11)) - c1 * rr.ooe.p[i]) * T(0.125);
        if (by)      // (2a+1, 2b, 2c+1): normal y
            vr.oeo.p[i] = (T(2) * (oy + oc) + ((e00 + e10) + (u00 + u10)) - c1 * rr.oeo.p[i]) * T(0.125);
        if (ax)      // (2a, 2b+1, 2c+1): normal x
            vr.eoo.p[i] = (T(2) * (ox + oc) + ((e00 + e01) + (u00 + u01)) - c1 * rr.eoo.p[i]) * T(0.125);
        om = oc; e00 = u00; e10 = u10; e01 = u01;
    }
}

// Eq. Erprolm: magenta corners (red EEE) from the 12 new face centres, cells
// [1, nb]^3.  vctl (the finest triple of the fused mixed path): also the
// largest |v| of the red level (the new corners and the face values read,
// which cover every face value) into vctl[p].vmax
template <typename T>
__global__ void __launch_bounds__(256) k_m2r_corners_zm_3d(Red3<const T> vf, A3<const T> reee, A3<T> veee, int nb, T c2,
                                                           int zm, Ctrl *vctl, const int *done, Bt B) {
    __shared__ float shm[32];
    const int prob = bt_prob(B);
    if (stop(bt_done(done, prob, B))) return;
    vf = bt_at(vf, prob, B); reee = bt_at(reee, prob, B); veee = bt_at(veee, prob, B);
    const int P = reee.pitch;
    const size_t Q = (size_t)P * reee.rows;
    ZmIdx z;
    float mx = 0.f;
    if (zm_cell(z, 1, nb, zm, P, Q, B)) {
        const T *ooe = vf.ooe.p, *oeo = vf.oeo.p, *eoo = vf.eoo.p;
        size_t i = z.i;
        // the four plane c-1 values of oeo / eoo are carried from the previous plane
        T pm1 = oeo[i - Q - 1], p0 = oeo[i - Q], qm1 = eoo[i - Q - P], q0 = eoo[i - Q];
        for (int c = z.c0; c < z.c1; c++, i += Q) {
            const T q[12] = {ooe[i - P - 1], ooe[i - P], ooe[i - 1], ooe[i], pm1, p0,
                             oeo[i - 1],     oeo[i],     qm1, q0, eoo[i - P], eoo[i]};
            pm1 = q[6]; p0 = q[7]; qm1 = q[10]; q0 = q[11];
            const T s1 = (q[0] + q[1]) + (q[2] + q[3]);
            const T s2 = (q[4] + q[5]) + (q[6] + q[7]);
            const T s3 = (q[8] + q[9]) + (q[10] + q[11]);
            const T v = ((s1 + s2 + s3) - c2 * reee.p[i]) * T(1.0 / 12.0);
            veee.p[i] = v;
            if (vctl) {
                mx = fmaxf(mx, (float)fabs(v));
#pragma unroll
                for (int k = 0; k < 12; k++) mx = fmaxf(mx, (float)fabs(q[k]));
            }
        }
    }
    if (vctl) {
        mx = block_max(mx, shm);
        if (threadIdx.x == 0 && threadIdx.y == 0) atomicMax(&vctl[prob].vmax, __float_as_uint(mx));
    }
}

}  // namespace mg
