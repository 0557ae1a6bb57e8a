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
constexpr int GS_WARM = 6;                        // steps before the first output plane

__device__ __forceinline__ void cp_async4(void *dst, const void *src, bool ok) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;\n" ::"r"((unsigned)__cvta_generic_to_shared(dst)),
                 "l"(src), "r"(ok ? 4 : 0) : "memory");
}

struct GreenSSmem {
    // red planes z+1..z+4 (ring, slot = plane & 3): fine row y holds its red
    // points x (x = y + plane mod 2) at index (x >> 1) - (16 bx - 4)
    float red[4][GS_RH][GS_RC];
    float r[4][GS_VH][GS_GW];    // green residual planes z..z+3 (ring), x from x0 - 5
    float v[4][GS_VH][GS_VW];    // correction planes z-1..z+2 (ring): F at odd, C at even points
    double u[2][GS_TY][GS_TX];   // u of output planes z, z+1 (UP_RR, UP_ADD)
    float lo[2][GS_TY][GS_TX];   // lo of the carried residual, planes z, z+1 (UP_RR)
};

// Green-red sweep of a triple's green level (Eq. Egprolg, then Eq. Egprolr,
// c = p_g h^2), z-streaming.  Step z of a block: F (odd index sum) on plane
// z+2 over the tile +- 2 from the red planes z+1..z+3; C (even) on plane z+1
// over the tile +- 1 from the F values of planes z..z+2; then the tile of
// plane z is final.  MODE: UP_RR the mixed finest triple (u += v and the
// carried float-float residual r -= L v as in k_up_ff_2d, six neighbours;
// rga/rgb double-buffered by par); UP_ADD u += v; UP_STORE v stored in vg.
// A block's z range holds zch output planes; its first GS_WARM steps fill
// the rings (nothing is written).
template <int MODE>
__global__ void __launch_bounds__(256) k_green_ff_3d(Red3<const float> vr, A3<float> rga, float *rgb, A3<float> vg,
                                                     float *__restrict__ rlo, double *__restrict__ u, int up, int n,
                                                     float cg, float s2, int zch, double *part, const int *par,
                                                     const int *done, Bt B) {
    extern __shared__ __align__(16) unsigned char smraw[];
    GreenSSmem &S = *reinterpret_cast<GreenSSmem *>(smraw);
    __shared__ double sh[32];
    constexpr bool RR = MODE == UP_RR, UPD = MODE != UP_STORE;
    constexpr int FPR = GS_VW / 2, NF = GS_VH * FPR;               // F points per row, per plane
    constexpr int CPR = (GS_VW - 2) / 2, NC = (GS_VH - 2) * CPR;   // C points per row, per plane
    constexpr int RCH = GS_RC / 4, GCH = GS_GW / 4;                // 16-byte chunks per red / residual row
    const int prob = bt_prob(B), zc = bt_z(B);
    if (stop(bt_done(done, prob, B))) return;
    A3<float> rg = rga, rnew = rga;
    if (RR) (par[(size_t)prob * B.ctl_stride] != 0 ? rg : rnew).p = rgb;
    vr = bt_at(vr, prob, B);
    rg = bt_at(rg, prob, B); rnew = bt_at(rnew, prob, B); vg = bt_at(vg, prob, B);
    if (RR) rlo = bt_ptr(rlo, prob, B);
    if (UPD && B.utab) u = B.utab[prob];
    if (RR) part += (size_t)prob * B.nparts;
    const int tx = threadIdx.x, ty = threadIdx.y, tid = tx + 32 * ty;
    const int x0 = blockIdx.x * GS_TX + 1, y0 = blockIdx.y * GS_TY + 1;
    const int zb = zc * zch + 1, ze = min(zb + zch, n + 1);  // output planes [zb, ze)
    const int zs = zb - GS_WARM;
    const size_t rows = (size_t)(n + 2), upl = (size_t)up * rows, gpl = (size_t)rg.pitch * rows;
    const size_t cpl = (size_t)vr.eee.pitch * vr.eee.rows;  // the four red cosets share their layout
    // the F region (tile +- 2) lies in the interior: no bounds tests but the plane's
    const bool inner = x0 >= 3 && x0 + GS_TX + 1 <= n && y0 >= 3 && y0 + GS_TY + 1 <= n;

    // ---- per-thread work items, fixed for all planes
    // red copy: fine row y0-3+ly, 16-byte chunk j of coset values (x >> 1) from 16 bx - 4
    const int rq_ly = tid / RCH, rq_j = tid - rq_ly * RCH, rq_y = y0 - 3 + rq_ly;
    const bool rq_on = tid < GS_RH * RCH;
    const bool rq_ok = rq_on && rq_y >= 0 && rq_y <= n + 1 && (x0 - 1) / 2 - 4 + 4 * rq_j >= 0;
    const size_t rq_off = rq_ok ? (size_t)(rq_y >> 1) * vr.eee.pitch + ((x0 - 1) / 2 - 4 + 4 * rq_j) : 0;
    // residual copy: row y0-2+ly, chunk j of x from x0 - 5
    const int gq_ly = tid / GCH, gq_j = tid - gq_ly * GCH, gq_y = y0 - 2 + gq_ly, gq_x = x0 - 5 + 4 * gq_j;
    const bool gq_on = tid < GS_VH * GCH;
    const bool gq_ok = gq_on && gq_x >= 0 && gq_y >= 0 && gq_y <= n + 1;
    const size_t gq_off = gq_ok ? (size_t)gq_y * rg.pitch + gq_x : 0;
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
    auto issue = [&](int zp, int zr, int zo) {
        if (rq_on) {
            const bool ok = rq_ok && zp >= 0 && zp <= n + 1;
            // the coset holding row y of plane zp: EEE, OOE (zp even), OEO, EOO (zp odd)
            const float *C = (zp & 1) ? ((rq_y & 1) ? vr.eoo.p : vr.oeo.p) : ((rq_y & 1) ? vr.ooe.p : vr.eee.p);
            cp_async16(&S.red[zp & 3][rq_ly][4 * rq_j], ok ? C + (size_t)(zp >> 1) * cpl + rq_off : C, ok);
        }
        if (gq_on) {
            const bool ok = gq_ok && zr >= 0 && zr <= n + 1;
            cp_async16(&S.r[zr & 3][gq_ly][4 * gq_j], ok ? rg.p + (size_t)zr * gpl + gq_off : rg.p, ok);
        }
        if (UPD && zo >= zb && zo < ze) {
            const int xo = x0 + tx;
#pragma unroll
            for (int h = 0; h < 2; h++) {
                const int ly = ty + 8 * h, yo = y0 + ly;
                const bool ok = xo <= n && yo <= n;
                cp_async8(&S.u[zo & 1][ly][tx], ok ? u + (size_t)zo * upl + (size_t)yo * up + xo : u, ok);
                if (RR) cp_async4(&S.lo[zo & 1][ly][tx], ok ? rlo + (size_t)zo * gpl + (size_t)yo * rg.pitch + xo : rlo, ok);
            }
        }
        cp_async_commit();
    };

    // ring slots not written by a step before they are read hold zeros
    for (int q = tid; q < (int)(sizeof(GreenSSmem) / 4); q += 256) reinterpret_cast<float *>(smraw)[q] = 0.f;
    __syncthreads();
    issue(zs + 3, zs + 2, zs);
    float sq = 0.f;
    for (int z = zs; z < ze; z++) {
        cp_async_wait0();
        __syncthreads();                             // step z's planes landed; step z-1 is done with every slot
        if (z + 1 < ze) issue(z + 4, z + 3, z + 1);  // the next step's planes, in flight during this one
        // F on plane z+2, tile +- 2: the red neighbours of the k-th F point of
        // a row are the row's red values k+3, k+4 and value k+3+p of rows
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
                    const int ry = ly + 1, ac = k + 3 + p;
                    const float s = (R0[ry][k + 3] + R0[ry][k + 4]) + (R0[ry - 1][ac] + R0[ry + 1][ac]) +
                                    (Rm[ry][ac] + Rp[ry][ac]);
                    val = (s - cg * G[ly][lx + 3]) * (1.f / 6.f);
                }
                V[ly][lx] = val;
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
                    val = (s - cg * G[ly][lx + 3]) * (1.f / 6.f);
                }
                V[ly][lx] = val;
            }
        }
        __syncthreads();
        // plane z is final on the tile
        if (z >= zb) {
            const float(&V)[GS_VH][GS_VW] = S.v[z & 3];
            const float(&Vm)[GS_VH][GS_VW] = S.v[(z - 1) & 3];
            const float(&Vp)[GS_VH][GS_VW] = S.v[(z + 1) & 3];
            const float(&G)[GS_VH][GS_GW] = S.r[z & 3];
            const int xo = x0 + tx;
#pragma unroll
            for (int h = 0; h < 2; h++) {
                const int yo = y0 + ty + 8 * h;
                if (xo > n || yo > n) continue;
                const int lx = tx + 2, ly = ty + 8 * h + 2;
                const float v = V[ly][lx];
                if (RR) {
                    const float nb[6] = {V[ly][lx - 1], V[ly][lx + 1], V[ly - 1][lx], V[ly + 1][lx], Vm[ly][lx], Vp[ly][lx]};
                    float lh, ll, nh, nl;
                    lap_sum6(nb, v, lh, ll);
                    ff_sub(G[ly][lx + 3], S.lo[z & 1][ty + 8 * h][tx], lh, ll, s2, nh, nl);
                    const size_t o = (size_t)z * gpl + (size_t)yo * rg.pitch + xo;
                    rlo[o] = nl;
                    rnew.p[o] = nh;
                    sq = fmaf(nh, nh, sq);
                }
                if (UPD) u[(size_t)z * upl + (size_t)yo * up + xo] = S.u[z & 1][ty + 8 * h][tx] + widen(v);
                else vg(xo, yo, z) = v;
            }
        }
    }
    if (RR) {
        const double s = block_sum((double)sq, sh);
        if (tid == 0) part[blockIdx.x + gridDim.x * (blockIdx.y + (size_t)gridDim.y * zc)] = s;
    }
}

}  // namespace mg
