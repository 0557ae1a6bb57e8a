// mg_fast2d.cuh -- fused 2D kernels of the diagonal V-cycle (Section 2), the
// finest residual kernels of both dimensions and the 3D coarse block.
//
// Per cycle of the FP64 path: k_res0_2d (finest residual, the FP64 stencil
// work), k_down_pair_2d (green -> red -> blue restriction of one pair, Eq.
// Erest2r then Eq. Erest2b, in a shared-memory tile), k_coarse_cta_2d (all
// pairs below a size cut-off, the coarsest solve and their Jacobi
// prolongation in one thread block, shared memory only), and k_up_pair_2d
// (blue -> red -> green Jacobi prolongation of one pair, Eq. Eajacr, Eq.
// Eajacb and the green-red sweep, in a shared-memory tile; on the finest
// pair fused with u += v).  The mixed path streams the large FP32 pairs
// (k_down_ff_2d, k_up_ff_2d: one warp per strip of columns marching along
// the rows) and carries the finest residual between cycles (k_up_ff_2d in
// its UP_RR form, k_res_rr_2d at the start and the end of a solve).
//
// Tiles are indexed by coset cells: cell (a,b) of a pair whose green grid has
// side n = 2nb+1 holds the green points (2a,2b) EE, (2a+1,2b) OE, (2a,2b+1) EO
// and (2a+1,2b+1) OO; a, b in [0, nb].  Out-of-range neighbours read zero
// (the Dirichlet ring).
#pragma once
#include "mg_stages.cuh"

namespace mg {

// Asynchronous global -> shared copies (cp.async): 16, 8 or 4 bytes, the
// destination zero-filled where ok is false (src is then any address inside
// its array; no byte of it is read).
__device__ __forceinline__ void cp_async16(void *dst, const void *src, bool ok) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"((unsigned)__cvta_generic_to_shared(dst)),
                 "l"(src), "r"(ok ? 16 : 0) : "memory");
}
__device__ __forceinline__ void cp_async8(void *dst, const void *src, bool ok) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8, %2;\n" ::"r"((unsigned)__cvta_generic_to_shared(dst)),
                 "l"(src), "r"(ok ? 8 : 0) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait1() { asm volatile("cp.async.wait_group 1;\n" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait2() { asm volatile("cp.async.wait_group 2;\n" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait0() { asm volatile("cp.async.wait_group 0;\n" ::: "memory"); }
__device__ __forceinline__ void cp_async4(void *dst, const void *src, bool ok) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;\n" ::"r"((unsigned)__cvta_generic_to_shared(dst)),
                 "l"(src), "r"(ok ? 4 : 0) : "memory");
}
// one level value (FP32 or FP64)
template <typename T> __device__ __forceinline__ void cp_async_el(T *dst, const T *src, bool ok) {
    if (sizeof(T) == 4) cp_async4(dst, src, ok);
    else cp_async8(dst, src, ok);
}

// loop of a 256-thread block over the points (x, y) of a W x H region, the
// points spread evenly over all threads (x fastest)
#define MG_FOR2(W, H)                                                                             \
    for (int q_ = threadIdx.x + 32 * threadIdx.y, x = 0, y = 0;                                   \
         q_ < (W) * (H) && ((x = q_ % (W)), (y = q_ / (W)), true); q_ += 256)


template <typename T> struct SqAcc;                     // per-thread sum of r^2
template <> struct SqAcc<float> {                       // mixed: FP32 squares
    float s = 0.f;
    __device__ void add(double r) { const float q = narrow(r); s = fmaf(q, q, s); }
    __device__ double block(double *sh) const { return block_sum_f(s, sh); }
};
template <> struct SqAcc<double> {
    double s = 0.0;
    __device__ void add(double r) { s = fma(r, r, s); }
    __device__ double block(double *sh) const { return block_sum(s, sh); }
};

// The Laplacian part of a direct residual in integer arithmetic (the FP64
// pipe of this GPU would otherwise bound the residual kernels).  Each u of a
// stencil is decoded into its signed 53-bit mantissa and exponent; all are
// aligned to the largest exponent with 6 guard bits (the bits below 2^-59 of
// the largest |u| are truncated) and summed exactly in 64 bits; the sum is
// rounded once to a double, already scaled by 1/h^2 = 2^lg (a power of two).
// Against the FP64 evaluation (4 to 7 roundings of partial sums) the result
// is at least as accurate; one FP64 subtraction from f remains.
struct Fx {
    long long m;  // signed mantissa with the implicit bit (0 for zeros and subnormals)
    int e;        // biased exponent
};
__device__ __forceinline__ Fx fx_dec(double x) {
    const unsigned hi = (unsigned)__double2hiint(x), lo = (unsigned)__double2loint(x);
    const int e = (int)((hi >> 20) & 0x7ffu);
    const long long m = e ? (((long long)((hi & 0xfffffu) | 0x100000u) << 32) | lo) : 0;
    return Fx{(hi >> 31) ? -m : m, e};
}
__device__ __forceinline__ long long fx_al(const Fx &a, int emax) {  // a * 2^6, aligned to emax
    const int k = emax - a.e;
    return k > 62 ? 0 : ((a.m << 6) >> k);
}
// a * 2^3, aligned to emax: 3 guard bits leave room for the weights of the
// fourth-order stencils (sums up to 48 x 2^56 < 2^62)
__device__ __forceinline__ long long fx_al3(const Fx &a, int emax) {
    const int k = emax - a.e;
    return k > 62 ? 0 : ((a.m << 3) >> k);
}
// the double nearest to s * 2^q (round to nearest even), s a 64-bit integer
__device__ __forceinline__ double fx_to_double(long long s, int q) {
    if (s == 0) return 0.0;
    const unsigned long long sg = s < 0 ? 0x8000000000000000ull : 0ull;
    unsigned long long a = s < 0 ? 0ull - (unsigned long long)s : (unsigned long long)s;
    const int lz = __clzll((long long)a);
    a <<= lz;  // leading one at bit 63
    unsigned long long m = a >> 11;
    const unsigned rem = (unsigned)(a & 0x7ffull);
    m += (rem > 0x400u || (rem == 0x400u && (m & 1ull))) ? 1ull : 0ull;
    int ex = 63 - lz + q + 1023;
    if (m >> 53) { m >>= 1; ex += 1; }
    if (ex < 1) return 0.0;  // below the normal range: far under any residual of interest
    return __longlong_as_double((long long)(sg | ((unsigned long long)ex << 52) | (m & 0xfffffffffffffull)));
}
constexpr int RES_ROWS = 8;  // rows per thread of the residual kernel

// Finest-grid residual, 2D.  Block 32x8 threads; a thread marches RES_ROWS
// rows down one column keeping the vertical neighbours in registers.
//   ORDER 2: r = f - (sum4 u - 4u)/h^2                            (Eq. Evpois)
//   ORDER 4: r = ft - (4 sum4axis u + sum4diag u - 20u)/(6h^2)    (Eq. Efos2)
//            with ft = (8f + sum4 f)/12 precomputed once per solve.
// Writes r in the level precision and the block's sum of r^2 to part[].
// Grid z: one slice per problem of the batch.
template <typename T, int ORDER>
__global__ void __launch_bounds__(256) k_res0_2d(const double *__restrict__ f, const double *__restrict__ u,
                                                 int up, int n, double ih2, int lg, A2<T> r, double *part,
                                                 const int *done, Bt B) {
    __shared__ double sh[32];
    const int prob = blockIdx.z;
    if (stop(bt_done(done, prob, B))) return;
    if (B.ftab) { f = B.ftab[prob]; u = B.utab[prob]; }
    r = bt_at(r, prob, B);
    const int i = blockIdx.x * 32 + threadIdx.x + 1;
    const int j0 = (blockIdx.y * 8 + threadIdx.y) * RES_ROWS + 1;
    SqAcc<T> acc;
    if (i <= n && j0 <= n) {
        const double *uc = u + (size_t)j0 * up + i;
        const double *fc = f + (size_t)j0 * up + i;
        double um = uc[-up], u0 = uc[0];
        double wm = 0, w0 = 0, em = 0, e0 = 0;  // diagonal neighbours (order 4)
        if (ORDER == 4) { wm = uc[-up - 1]; em = uc[-up + 1]; w0 = uc[-1]; e0 = uc[1]; }
        // FP32 levels (mixed), order 4: the Mehrstellen Laplacian in integer
        // arithmetic (fx_dec / fx_al3): rows j-1 and j stay decoded
        constexpr bool FX4 = ORDER == 4 && sizeof(T) == 4;
        Fx xm[3], x0[3];
        if (FX4) {
            xm[0] = fx_dec(wm); xm[1] = fx_dec(um); xm[2] = fx_dec(em);
            x0[0] = fx_dec(w0); x0[1] = fx_dec(u0); x0[2] = fx_dec(e0);
        }
#pragma unroll
        for (int q = 0; q < RES_ROWS; q++) {
            if (j0 + q > n) break;
            const double upn = uc[up];
            double res;
            if (FX4) {
                const Fx xp[3] = {fx_dec(uc[up - 1]), fx_dec(upn), fx_dec(uc[up + 1])};
                const int emx = max(max(max(xm[0].e, xm[1].e), max(xm[2].e, x0[0].e)),
                                    max(max(x0[1].e, x0[2].e), max(max(xp[0].e, xp[1].e), xp[2].e)));
                const long long ax = (fx_al3(x0[0], emx) + fx_al3(x0[2], emx)) + (fx_al3(xm[1], emx) + fx_al3(xp[1], emx));
                const long long dg = (fx_al3(xm[0], emx) + fx_al3(xm[2], emx)) + (fx_al3(xp[0], emx) + fx_al3(xp[2], emx));
                const long long c = fx_al3(x0[1], emx);
                // h^-2 (4 ax + dg - 20 c), rounded once; then / 6 and f - . (2 FP64 operations)
                const double l6 = fx_to_double((ax << 2) + dg - ((c << 4) + (c << 2)), emx - 1078 + lg);
                res = fc[0] - l6 * (1.0 / 6.0);
#pragma unroll
                for (int t = 0; t < 3; t++) { xm[t] = x0[t]; x0[t] = xp[t]; }
            } else if (ORDER == 2) {
                const double s = (uc[-1] + uc[1]) + (um + upn);
                res = fma(-ih2, fma(-4.0, u0, s), fc[0]);
            } else {
                const double wp = uc[up - 1], ep = uc[up + 1];
                const double ax = (w0 + e0) + (um + upn);
                const double dg = (wm + em) + (wp + ep);
                res = fma(-ih2 * (1.0 / 6.0), fma(-20.0, u0, fma(4.0, ax, dg)), fc[0]);
                wm = w0; em = e0; w0 = wp; e0 = ep;
            }
            r(i, j0 + q) = lvl<T>(res);
            acc.add(res);
            um = u0; u0 = upn;
            uc += up; fc += up;
        }
    }
    double s = acc.block(sh);
    if (threadIdx.x == 0 && threadIdx.y == 0)
        part[(size_t)prob * B.nparts + blockIdx.x + gridDim.x * blockIdx.y] = s;
}

// ft = (8f + sum4 f)/12 on the interior (order-4 right-hand side of Eq. Efos2)
__global__ void k_rhs4_2d(const double *__restrict__ f, int up, int n, double *ft) {
    pdl_wait();
    MG_IDX2 const int i = tx + 1, j = ty + 1;
    if (i > n || j > n) return;
    const size_t c = (size_t)j * up + i;
    ft[c] = (8.0 * f[c] + ((f[c - 1] + f[c + 1]) + (f[c - up] + f[c + up]))) * (1.0 / 12.0);
}

// ---------------------------------------------------------------------------
// pair restriction: green -> red (Eq. Erest2r) -> blue (Eq. Erest2b), one
// tile of TA x TB coset cells per 256-thread block, grid z = problem
// ---------------------------------------------------------------------------
template <typename T, int TA, int TB>
__global__ void __launch_bounds__(256) k_down_pair_2d(A2<const T> g, A2<T> ee, A2<T> oo, A2<T> blue, int nb,
                                                      const T *galt, const int *par, const int *done, Bt B) {
    constexpr int GX = 2 * TA + 3, GY = 2 * TB + 3;  // green x in [2a0-2, 2a0+2TA]
    constexpr int OX = TA + 1, OY = TB + 1;          // OO cells a in [a0-1, a0+TA)
    __shared__ T sg[GY][GX];
    __shared__ T so[OY][OX + 1];
    const int prob = blockIdx.z;
    if (stop(bt_done(done, prob, B))) return;
    if (galt && par[(size_t)prob * B.ctl_stride]) g.p = galt;  // the current one of two green buffers
    g = bt_at(g, prob, B); ee = bt_at(ee, prob, B); oo = bt_at(oo, prob, B); blue = bt_at(blue, prob, B);
    const int a0 = blockIdx.x * TA, b0 = blockIdx.y * TB;
    const int n = 2 * nb + 1;
    // all of a thread's copies in flight at once (one L2 round trip, not one
    // per element)
    MG_FOR2(GX, GY) {
        const int gx = 2 * a0 - 2 + x, gy = 2 * b0 - 2 + y;
        const bool ok = gx >= 0 && gx <= n + 1 && gy >= 0 && gy <= n + 1;
        cp_async_el(&sg[y][x], ok ? &g(gx, gy) : g.p, ok);
    }
    cp_async_commit();
    cp_async_wait0();
    __syncthreads();
    // OO(c,d) at green (2c+1, 2d+1) -> smem index (2c+1) - (2a0-2) = 2(c-a0)+3
    MG_FOR2(OX, OY) {
        const int cx = x, cy = y;  // c = a0-1+cx
        const int c = a0 - 1 + cx, d = b0 - 1 + cy;
        T v = T(0);
        if (c >= 0 && c <= nb && d >= 0 && d <= nb) {
            const int sx = 2 * cx + 1, sy = 2 * cy + 1;
            v = (T(4) * sg[sy][sx] + (sg[sy][sx - 1] + sg[sy][sx + 1]) + (sg[sy - 1][sx] + sg[sy + 1][sx])) * T(0.125);
            if (cx >= 1 && cy >= 1) oo(c, d) = v;
        }
        so[cy][cx] = v;
    }
    __syncthreads();
    MG_FOR2(TA, TB) {
        const int ax = x, by = y;
        const int a = a0 + ax, b = b0 + by;
        if (a < 1 || a > nb || b < 1 || b > nb) continue;
        const int sx = 2 * ax + 2, sy = 2 * by + 2;  // green (2a, 2b)
        const T e = (T(4) * sg[sy][sx] + (sg[sy][sx - 1] + sg[sy][sx + 1]) + (sg[sy - 1][sx] + sg[sy + 1][sx])) * T(0.125);
        ee(a, b) = e;
        // diagonal red neighbours OO(a-1..a, b-1..b) = so[by..by+1][ax..ax+1]
        blue(a, b) = (T(4) * e + (so[by][ax] + so[by][ax + 1]) + (so[by + 1][ax] + so[by + 1][ax + 1])) * T(0.125);
    }
}

// ---------------------------------------------------------------------------
// pair prolongation: blue -> red (Eq. Eajacr, Eq. Eajacb) -> green (the
// green-red sweep); FINEST: u += v instead of storing v
// ---------------------------------------------------------------------------
template <typename T, int TA, int TB> struct UpSmem {
    T b[TB + 5][TA + 5];     // blue v, cells [a0-2, a0+TA+2]
    T roo[TB + 4][TA + 4];   // OO cells [a0-2, a0+TA+1]
    T ree[TB + 3][TA + 3];   // EE cells [a0-1, a0+TA+1]
    T voo[TB + 4][TA + 4];
    T vee[TB + 3][TA + 3];
    T rg[2 * TB + 4][2 * TA + 4];  // green r, x in [2a0-2, 2a0+2TA+1]
    T voe[TB + 2][TA + 2];   // F cells [a0-1, a0+TA]
    T veo[TB + 2][TA + 2];
};

template <typename T, bool FINEST, int TA, int TB>
__global__ void __launch_bounds__(256) k_up_pair_2d(A2<const T> blue, A2<const T> ree, A2<const T> roo,
                                                    A2<const T> rg, A2<T> vg, double *u, int up, int nb,
                                                    T c2, T c1, const int *done, Bt B) {
    extern __shared__ __align__(16) unsigned char smraw[];
    UpSmem<T, TA, TB> &S = *reinterpret_cast<UpSmem<T, TA, TB> *>(smraw);
    const int prob = blockIdx.z;
    if (stop(bt_done(done, prob, B))) return;
    blue = bt_at(blue, prob, B); ree = bt_at(ree, prob, B); roo = bt_at(roo, prob, B);
    rg = bt_at(rg, prob, B); vg = bt_at(vg, prob, B);
    if (B.utab) u = B.utab[prob];
    const int a0 = blockIdx.x * TA, b0 = blockIdx.y * TB;
    const int n = 2 * nb + 1;
    // loads: all of a thread's copies in flight at once (one L2 round trip,
    // not one per element); out-of-range values are zero-filled
    MG_FOR2(TA + 5, TB + 5) {
        const int a = a0 - 2 + x, b = b0 - 2 + y;
        const bool ok = a >= 0 && a <= nb + 1 && b >= 0 && b <= nb + 1;
        cp_async_el(&S.b[y][x], ok ? &blue(a, b) : blue.p, ok);
    }
    MG_FOR2(TA + 4, TB + 4) {
        const int a = a0 - 2 + x, b = b0 - 2 + y;
        const bool ok = a >= 0 && a <= nb && b >= 0 && b <= nb;
        cp_async_el(&S.roo[y][x], ok ? &roo(a, b) : roo.p, ok);
    }
    MG_FOR2(TA + 3, TB + 3) {
        const int a = a0 - 1 + x, b = b0 - 1 + y;
        const bool ok = a >= 1 && a <= nb && b >= 1 && b <= nb;
        cp_async_el(&S.ree[y][x], ok ? &ree(a, b) : ree.p, ok);
    }
    MG_FOR2(2 * TA + 4, 2 * TB + 4) {
        const int gx = 2 * a0 - 2 + x, gy = 2 * b0 - 2 + y;
        const bool ok = gx >= 1 && gx <= n && gy >= 1 && gy <= n;
        cp_async_el(&S.rg[y][x], ok ? &rg(gx, gy) : rg.p, ok);
    }
    cp_async_commit();
    cp_async_wait0();
    __syncthreads();
    // red points not blue: OO(c,d), c in [a0-2, a0+TA+1]; smem x = c - a0 + 2 in voo and in b
    MG_FOR2(TA + 4, TB + 4) {
        const int c = a0 - 2 + x, d = b0 - 2 + y;
        T v = T(0);
        if (c >= 0 && c <= nb && d >= 0 && d <= nb)
            v = ((S.b[y][x] + S.b[y][x + 1]) + (S.b[y + 1][x] + S.b[y + 1][x + 1]) - c2 * S.roo[y][x]) * T(0.25);
        S.voo[y][x] = v;
    }
    __syncthreads();
    // blue points refined: EE(a,b), a in [a0-1, a0+TA+1]; smem x = a - a0 + 1; OO(a-1) at voo x = a - a0 + 1
    MG_FOR2(TA + 3, TB + 3) {
        const int a = a0 - 1 + x, b = b0 - 1 + y;
        T v = T(0);
        if (a >= 1 && a <= nb && b >= 1 && b <= nb)
            v = ((S.voo[y][x] + S.voo[y][x + 1]) + (S.voo[y + 1][x] + S.voo[y + 1][x + 1]) - c2 * S.ree[y][x]) *
                T(0.25);
        S.vee[y][x] = v;
    }
    __syncthreads();
    // green-only points: OE(a,b) at (2a+1, 2b), EO(a,b) at (2a, 2b+1); cells [a0-1, a0+TA]
    MG_FOR2(TA + 2, TB + 2) {
        const int a = a0 - 1 + x, b = b0 - 1 + y;
        // EE(a,b) at vee[y][x]; EE(a+1,b) vee[y][x+1]; EE(a,b+1) vee[y+1][x]
        // OO(a,b) at voo[y+1][x+1]; OO(a,b-1) voo[y][x+1]; OO(a-1,b) voo[y+1][x]
        // green (2a+1, 2b) at rg[2y][2x+1]; (2a, 2b+1) at rg[2y+1][2x]
        T voe = T(0), veo = T(0);
        if (a >= 0 && a <= nb && b >= 1 && b <= nb)
            voe = ((S.vee[y][x] + S.vee[y][x + 1]) + (S.voo[y][x + 1] + S.voo[y + 1][x + 1]) - c1 * S.rg[2 * y][2 * x + 1]) *
                  T(0.25);
        if (a >= 1 && a <= nb && b >= 0 && b <= nb)
            veo = ((S.voo[y + 1][x] + S.voo[y + 1][x + 1]) + (S.vee[y][x] + S.vee[y + 1][x]) - c1 * S.rg[2 * y + 1][2 * x]) *
                  T(0.25);
        S.voe[y][x] = voe;
        S.veo[y][x] = veo;
    }
    __syncthreads();
    // red points of the own cells from the new green values, then store / update
    MG_FOR2(TA, TB) {
        const int a = a0 + x, b = b0 + y;
        if (a > nb || b > nb) continue;
        const int fx = x + 1, fy = y + 1;  // F smem index of cell (a,b)
        // EE(a,b) at (2a,2b): OE(a-1,b), OE(a,b), EO(a,b-1), EO(a,b)
        T vEE = T(0);
        if (a >= 1 && b >= 1)
            vEE = ((S.voe[fy][fx - 1] + S.voe[fy][fx]) + (S.veo[fy - 1][fx] + S.veo[fy][fx]) - c1 * S.rg[2 * fy][2 * fx]) * T(0.25);
        // OO(a,b) at (2a+1,2b+1): EO(a,b), EO(a+1,b), OE(a,b), OE(a,b+1)
        const T vOO = ((S.veo[fy][fx] + S.veo[fy][fx + 1]) + (S.voe[fy][fx] + S.voe[fy + 1][fx]) - c1 * S.rg[2 * fy + 1][2 * fx + 1]) *
                      T(0.25);
        const T vOE = S.voe[fy][fx], vEO = S.veo[fy][fx];
        const int i = 2 * a, j = 2 * b;
        if (FINEST) {
            double *ur0 = u + (size_t)j * up + i;       // row 2b: (2a, 2b), (2a+1, 2b)
            double *ur1 = ur0 + up;                     // row 2b+1
            if (b >= 1) {
                if (a >= 1) ur0[0] += widen(vEE);
                ur0[1] += widen(vOE);
            }
            if (a >= 1) ur1[0] += widen(vEO);
            ur1[1] += widen(vOO);
        } else {
            if (b >= 1) {
                if (a >= 1) vg(i, j) = vEE;
                vg(i + 1, j) = vOE;
            }
            if (a >= 1) vg(i, j + 1) = vEO;
            vg(i + 1, j + 1) = vOO;
        }
    }
}

// ---------------------------------------------------------------------------
// coarse pairs in one thread block, all in shared memory
// ---------------------------------------------------------------------------
constexpr int CTA_MAX_PAIRS = 12;

struct CoarsePlan2d {
    int kc, K;                        // pairs kc..K-1 run here; level K is the coarsest grid
    int nk[CTA_MAX_PAIRS + 1];        // green side of pair k - kc (and the coarsest)
    int og_r[CTA_MAX_PAIRS + 1], og_v[CTA_MAX_PAIRS + 1];  // smem offsets (elements), green r / v
    int oe_r[CTA_MAX_PAIRS], oo_r[CTA_MAX_PAIRS], oe_v[CTA_MAX_PAIRS], oo_v[CTA_MAX_PAIRS];
    int total;                        // smem elements
    int gofs, ng;                     // byte offset and size (doubles) of the copy of the coarsest inverse
    double c2[CTA_MAX_PAIRS], c1[CTA_MAX_PAIRS];  // 2 p h_k^2 (red), p h_k^2 (green)
};

// The dense inverse G of the coarsest operator (at most CTA_G_MAX doubles) is
// read into registers when a coarse block starts, stored to shared memory
// beside the levels once they are loaded, and read from there by the coarse
// solve (no global-memory latency on the block's critical path).
constexpr int CTA_G_PER_THREAD = 3, CTA_G_MAX = CTA_G_PER_THREAD * 1024;
template <int NT> struct GPrefetch {
    double g[CTA_G_PER_THREAD];
    __device__ __forceinline__ void load(const double *G, int ng, int tid) {
#pragma unroll
        for (int k = 0; k < CTA_G_PER_THREAD; k++) g[k] = tid + k * NT < ng ? G[tid + k * NT] : 0.0;
    }
    __device__ __forceinline__ void store(double *Gs, int ng, int tid) const {
#pragma unroll
        for (int k = 0; k < CTA_G_PER_THREAD; k++)
            if (tid + k * NT < ng) Gs[tid + k * NT] = g[k];
    }
};

// Pairs P.kc..P.K-1 and the exact coarsest solve in one block of 1024
// threads, all in shared memory.  On entry the green residual of pair P.kc
// is at sm + og_r[0] (ring and unused entries zero), every other level array
// is zero and the coarsest inverse is at Gs; on return the green correction
// of pair P.kc is at sm + og_v[0].  Restriction Eq. Erest2r, Eq. Erest2b;
// prolongation Eq. Eajacr, Eq. Eajacb and the green-red sweep.
template <typename T> __device__ __forceinline__ void cta_pairs_2d(const CoarsePlan2d &P, T *sm, const double *Gs) {
    const int tid = threadIdx.x, nt = blockDim.x;
    // 32 x 32 thread grid: loops over boxes step by 32, no index division
    const int tx = tid & 31, ty = tid >> 5;
#define CTA_FOR2(i, j, lo_i, hi_i, lo_j, hi_j) \
    for (int j = (lo_j) + ty; j <= (hi_j); j += 32) for (int i = (lo_i) + tx; i <= (hi_i); i += 32)
    const int npair = P.K - P.kc;
    for (int p = 0; p < npair; p++) {
        const int n = P.nk[p], nb = (n - 1) / 2;
        A2<T> g{sm + P.og_r[p], n + 2}, ee{sm + P.oe_r[p], nb + 2}, oo{sm + P.oo_r[p], nb + 2};
        A2<T> bl{sm + P.og_r[p + 1], nb + 2};
        CTA_FOR2(a, b, 0, nb, 0, nb) {  // Eq. Erest2r
            int i = 2 * a + 1, j = 2 * b + 1;
            oo(a, b) = (T(4) * g(i, j) + (g(i - 1, j) + g(i + 1, j)) + (g(i, j - 1) + g(i, j + 1))) * T(0.125);
            if (a >= 1 && b >= 1) {
                i = 2 * a; j = 2 * b;
                ee(a, b) = (T(4) * g(i, j) + (g(i - 1, j) + g(i + 1, j)) + (g(i, j - 1) + g(i, j + 1))) * T(0.125);
            }
        }
        __syncthreads();
        CTA_FOR2(a, b, 1, nb, 1, nb) {  // Eq. Erest2b
            bl(a, b) = (T(4) * ee(a, b) + (oo(a - 1, b - 1) + oo(a, b - 1)) + (oo(a - 1, b) + oo(a, b))) * T(0.125);
        }
        __syncthreads();
    }
    {   // exact solve on the coarsest grid
        const int s = P.nk[npair], nn = s * s;
        A2<T> r{sm + P.og_r[npair], s + 2}, v{sm + P.og_v[npair], s + 2};
        double *rv = const_cast<double *>(Gs) + P.ng;  // the right-hand side, dense
        for (int q = tid; q < nn; q += nt) rv[q] = (double)r(q % s + 1, q / s + 1);
        __syncthreads();
        for (int q = tid; q < nn; q += nt) {
            double acc = 0.0;
            for (int t = 0; t < nn; t++) acc += Gs[q * nn + t] * rv[t];
            v(q % s + 1, q / s + 1) = (T)acc;
        }
    }
    __syncthreads();
    for (int p = npair - 1; p >= 0; p--) {
        const int n = P.nk[p], nb = (n - 1) / 2;
        A2<T> rgr{sm + P.og_r[p], n + 2}, vgr{sm + P.og_v[p], n + 2};
        A2<T> ree{sm + P.oe_r[p], nb + 2}, roo{sm + P.oo_r[p], nb + 2};
        A2<T> vee{sm + P.oe_v[p], nb + 2}, voo{sm + P.oo_v[p], nb + 2};
        A2<T> vbl{sm + P.og_v[p + 1], nb + 2};
        const T c2 = (T)P.c2[p], c1 = (T)P.c1[p];
        CTA_FOR2(a, b, 0, nb, 0, nb) {  // Eq. Eajacr
            voo(a, b) = ((vbl(a, b) + vbl(a + 1, b)) + (vbl(a, b + 1) + vbl(a + 1, b + 1)) - c2 * roo(a, b)) * T(0.25);
        }
        __syncthreads();
        CTA_FOR2(a, b, 1, nb, 1, nb) {  // Eq. Eajacb
            vee(a, b) = ((voo(a - 1, b - 1) + voo(a, b - 1)) + (voo(a - 1, b) + voo(a, b)) - c2 * ree(a, b)) * T(0.25);
        }
        __syncthreads();
        for (int j = 1 + ty; j <= n; j += 32)  // green-only points: i + j odd
            for (int i = 1 + (j & 1) + 2 * tx; i <= n; i += 64) {
            auto red = [&](int x, int y) { return (x & 1) ? voo(x >> 1, y >> 1) : vee(x >> 1, y >> 1); };
            vgr(i, j) = ((red(i - 1, j) + red(i + 1, j)) + (red(i, j - 1) + red(i, j + 1)) - c1 * rgr(i, j)) * T(0.25);
        }
        __syncthreads();
        for (int j = 1 + ty; j <= n; j += 32)  // red points: i + j even
            for (int i = 2 - (j & 1) + 2 * tx; i <= n; i += 64) {
            vgr(i, j) = ((vgr(i - 1, j) + vgr(i + 1, j)) + (vgr(i, j - 1) + vgr(i, j + 1)) - c1 * rgr(i, j)) * T(0.25);
        }
        __syncthreads();
    }
#undef CTA_FOR2
}

template <typename T>
__global__ void __launch_bounds__(1024) k_coarse_cta_2d(CoarsePlan2d P, A2<const T> rg_in, A2<T> vg_out,
                                                        const double *G, const int *done, Bt B) {
    extern __shared__ __align__(16) unsigned char smraw[];
    T *sm = reinterpret_cast<T *>(smraw);
    const int prob = blockIdx.z;
    if (stop(bt_done(done, prob, B))) return;
    rg_in = bt_at(rg_in, prob, B);
    vg_out = bt_at(vg_out, prob, B);
    const int tid = threadIdx.x, nt = blockDim.x;
    GPrefetch<1024> gp;
    gp.load(G, P.ng, tid);
    double *Gs = reinterpret_cast<double *>(smraw + P.gofs);
    const int tx = tid & 31, ty = tid >> 5;
    for (int q = tid; q < P.total; q += nt) sm[q] = T(0);
    __syncthreads();
    {   // load the green residual of pair kc (a thread's copies all in flight at once)
        const int n = P.nk[0];
        A2<T> g{sm + P.og_r[0], n + 2};
        for (int j = 1 + ty; j <= n; j += 32)
            for (int i = 1 + tx; i <= n; i += 32) cp_async_el(&g(i, j), &rg_in(i, j), true);
        cp_async_commit();
    }
    gp.store(Gs, P.ng, tid);
    cp_async_wait0();
    __syncthreads();
    cta_pairs_2d<T>(P, sm, Gs);
    {
        const int n = P.nk[0];
        A2<T> g{sm + P.og_v[0], n + 2};
        for (int j = 1 + ty; j <= n; j += 32)
            for (int i = 1 + tx; i <= n; i += 32) vg_out(i, j) = g(i, j);
    }
}

}  // namespace mg

namespace mg {

constexpr int RES3_PLANES = 8;  // planes per thread of the 3D residual kernel

// Finest-grid residual, 3D.  Block 32x8 threads over (x, y); a thread marches
// RES3_PLANES planes in z keeping the z neighbours in registers.
//   ORDER 2: r = f - (sum6 u - 6u)/h^2
//   ORDER 4: r = ft - (2 sum6 u + sum12 u - 24u)/(6h^2)   (Eq. Efos4, ft precomputed)
template <typename T, int ORDER>
__global__ void __launch_bounds__(256) k_res0_3d(const double *__restrict__ f, const double *__restrict__ u,
                                                 int up, int n, double ih2, int lg, A3<T> r, double *part,
                                                 const int *done, Bt B) {
    __shared__ double sh[32];
    const int prob = bt_prob(B), bz = bt_z(B);
    if (stop(bt_done(done, prob, B))) return;
    if (B.ftab) { f = B.ftab[prob]; u = B.utab[prob]; }
    r = bt_at(r, prob, B);
    part += (size_t)prob * B.nparts;
    const int i = blockIdx.x * 32 + threadIdx.x + 1, j = blockIdx.y * 8 + threadIdx.y + 1;
    const int k0 = bz * RES3_PLANES + 1;
    const size_t pl = (size_t)up * (n + 2);
    SqAcc<T> acc;
    if (i <= n && j <= n) {
        const double *uc = u + k0 * pl + (size_t)j * up + i;
        const double *fc = f + k0 * pl + (size_t)j * up + i;
        double ud = uc[-(long)pl], u0 = uc[0];
        // FP32 levels (mixed), order 4: the 19-point Laplacian in integer
        // arithmetic (fx_dec / fx_al3); a plane's centre and axis neighbours
        // (c, w, e, s, n) stay decoded for the next two planes
        constexpr bool FX4 = ORDER == 4 && sizeof(T) == 4;
        auto dec5 = [&](const double *p, Fx *x) {
            x[0] = fx_dec(p[0]); x[1] = fx_dec(p[-1]); x[2] = fx_dec(p[1]); x[3] = fx_dec(p[-up]); x[4] = fx_dec(p[up]);
        };
        Fx xm[5], x0[5];
        if (FX4) { dec5(uc - pl, xm); dec5(uc, x0); }
#pragma unroll
        for (int q = 0; q < RES3_PLANES; q++) {
            if (k0 + q > n) break;
            const double uu = uc[pl];
            double res;
            if (FX4) {
                Fx xp[5], dg[4];
                dec5(uc + pl, xp);
                dg[0] = fx_dec(uc[-up - 1]); dg[1] = fx_dec(uc[-up + 1]); dg[2] = fx_dec(uc[up - 1]); dg[3] = fx_dec(uc[up + 1]);
                int emx = max(max(dg[0].e, dg[1].e), max(dg[2].e, dg[3].e));
#pragma unroll
                for (int t = 0; t < 5; t++) emx = max(emx, max(max(xm[t].e, x0[t].e), xp[t].e));
                // faces: the plane's 4 axis neighbours and the centres of planes k-1, k+1
                const long long fa = ((fx_al3(x0[1], emx) + fx_al3(x0[2], emx)) + (fx_al3(x0[3], emx) + fx_al3(x0[4], emx))) +
                                     (fx_al3(xm[0], emx) + fx_al3(xp[0], emx));
                // edges: the plane's 4 diagonal neighbours and the axis neighbours of planes k-1, k+1
                const long long ed = ((fx_al3(dg[0], emx) + fx_al3(dg[1], emx)) + (fx_al3(dg[2], emx) + fx_al3(dg[3], emx))) +
                                     ((fx_al3(xm[1], emx) + fx_al3(xm[2], emx)) + (fx_al3(xm[3], emx) + fx_al3(xm[4], emx))) +
                                     ((fx_al3(xp[1], emx) + fx_al3(xp[2], emx)) + (fx_al3(xp[3], emx) + fx_al3(xp[4], emx)));
                const long long c = fx_al3(x0[0], emx);
                // h^-2 (2 faces + edges - 24 c), rounded once; then / 6 and f - . (2 FP64 operations)
                const double l6 = fx_to_double((fa << 1) + ed - ((c << 4) + (c << 3)), emx - 1078 + lg);
                res = fc[0] - l6 * (1.0 / 6.0);
#pragma unroll
                for (int t = 0; t < 5; t++) { xm[t] = x0[t]; x0[t] = xp[t]; }
            } else if (ORDER == 2) {
                const double s = ((uc[-1] + uc[1]) + (uc[-up] + uc[up])) + (ud + uu);
                res = fma(-ih2, fma(-6.0, u0, s), fc[0]);
            } else {
                const double ax = ((uc[-1] + uc[1]) + (uc[-up] + uc[up])) + (ud + uu);
                const double ed = ((uc[-up - 1] + uc[-up + 1]) + (uc[up - 1] + uc[up + 1])) +
                                  ((uc[-(long)pl - up] + uc[-(long)pl + up]) + (uc[pl - up] + uc[pl + up])) +
                                  ((uc[-(long)pl - 1] + uc[-(long)pl + 1]) + (uc[pl - 1] + uc[pl + 1]));
                res = fma(-ih2 * (1.0 / 6.0), fma(-24.0, u0, fma(2.0, ax, ed)), fc[0]);
            }
            r(i, j, k0 + q) = lvl<T>(res);
            acc.add(res);
            ud = u0; u0 = uu;
            uc += pl; fc += pl;
        }
    }
    double s = acc.block(sh);
    if (threadIdx.x == 0 && threadIdx.y == 0)
        part[blockIdx.x + gridDim.x * (blockIdx.y + (size_t)gridDim.y * bz)] = s;
}

// ft = (6f + sum6 f)/12 on the interior (order-4 right-hand side of Eq. Efos4)
__global__ void k_rhs4_3d(const double *__restrict__ f, int up, int n, double *ft) {
    pdl_wait();
    MG_IDX2 const int i = tx + 1, j = ty + 1, k = (int)blockIdx.z + 1;
    if (i > n || j > n) return;
    const size_t pl = (size_t)up * (n + 2);
    const size_t c = k * pl + (size_t)j * up + i;
    ft[c] = (6.0 * f[c] + ((f[c - 1] + f[c + 1]) + (f[c - up] + f[c + up]) + (f[c - pl] + f[c + pl]))) * (1.0 / 12.0);
}

// finest 3D level, second half of the green-red sweep (Eq. Egprolr) fused with
// u += v; the f32 -> f64 widening uses integer operations
template <typename T>
__global__ void k_r2g_c_upd_fast_3d(A3<const T> rg, A3<const T> vg, double *u, int up, int urows, int n, T cc,
                                    const int *done, Bt B) {
    const int prob_ = bt_prob(B);
    if (stop(bt_done(done, prob_, B))) return;
    rg = bt_at(rg, prob_, B);
    vg = bt_at(vg, prob_, B);
    if (B.utab) u = B.utab[prob_];
    MG_IDX3 const int i = tx + 1, j = ty + 1, k = tz + 1;
    if (i > n || j > n || k > n) return;
    T v;
    if ((i + j + k) & 1) v = vg(i, j, k);
    else
        v = ((vg(i - 1, j, k) + vg(i + 1, j, k)) + (vg(i, j - 1, k) + vg(i, j + 1, k)) +
             (vg(i, j, k - 1) + vg(i, j, k + 1)) - cc * rg(i, j, k)) * T(1.0 / 6.0);
    u[((size_t)k * urows + j) * up + i] += widen(v);
}

}  // namespace mg

namespace mg {

// ---------------------------------------------------------------------------
// coarse triples (3D) in one thread block, all in shared memory: Eq. Erred,
// Ermagc/Ermagm, Erblu down; the exact coarsest solve; Eq. Emprolm/Emprolb,
// Erprolr/Erprolm, Egprolg/Egprolr up
// ---------------------------------------------------------------------------
constexpr int CTA3_MAX = 8;

struct CoarsePlan3d {
    int kc, K;
    int nk[CTA3_MAX + 1];
    int og_r[CTA3_MAX + 1], og_v[CTA3_MAX + 1];          // green grids (side n+2)^3
    int orr[CTA3_MAX][4], orv[CTA3_MAX][4];              // red cosets EEE, OOE, OEO, EOO ((nb+2)^3)
    int omr[CTA3_MAX][2], omv[CTA3_MAX][2];              // magenta cosets EEE, OOO
    int total;
    int gofs, ng;  // byte offset and size (doubles) of the copy of the coarsest inverse
    double cm[CTA3_MAX], cr1[CTA3_MAX], cr2[CTA3_MAX], cg[CTA3_MAX];  // 4p_m h^2, 2p_r1 h^2, 4p_r2 h^2, p_g h^2
};

template <typename T>
__global__ void __launch_bounds__(1024) k_coarse_cta_3d(CoarsePlan3d P, A3<const T> rg_in, A3<T> vg_out,
                                                        const double *G, const int *done, Bt B) {
    extern __shared__ __align__(16) unsigned char smraw[];
    T *sm = reinterpret_cast<T *>(smraw);
    const int prob = blockIdx.z;
    if (stop(bt_done(done, prob, B))) return;
    rg_in = bt_at(rg_in, prob, B);
    vg_out = bt_at(vg_out, prob, B);
    const int tid = threadIdx.x, nt = blockDim.x;
    GPrefetch<1024> gp;
    gp.load(G, P.ng, tid);
    double *Gs = reinterpret_cast<double *>(smraw + P.gofs);
    // 16 x 8 x 8 thread grid: loops over boxes without index division
    const int tx = tid & 15, ty = (tid >> 4) & 7, tz = tid >> 7;
#define CTA_FOR3(i, j, k, lo, hi)                                        \
    for (int k = (lo) + tz; k <= (hi); k += 8)                            \
        for (int j = (lo) + ty; j <= (hi); j += 8)                        \
            for (int i = (lo) + tx; i <= (hi); i += 16)
    for (int q = tid; q < P.total; q += nt) sm[q] = T(0);
    __syncthreads();
    const int ntri = P.K - P.kc;
    auto G3 = [&](int off, int n) { return A3<T>{sm + off, n + 2, n + 2}; };
    auto C3 = [&](int off, int nb) { return A3<T>{sm + off, nb + 2, nb + 2}; };
    {   // the green residual of the top triple (a thread's copies all in flight at once)
        const int n = P.nk[0];
        A3<T> g = G3(P.og_r[0], n);
        CTA_FOR3(i, j, k, 1, n) cp_async_el(&g(i, j, k), &rg_in(i, j, k), true);
        cp_async_commit();
    }
    gp.store(Gs, P.ng, tid);
    cp_async_wait0();
    __syncthreads();
    for (int t = 0; t < ntri; t++) {
        const int n = P.nk[t], nb = (n - 1) / 2;
        A3<T> g = G3(P.og_r[t], n);
        A3<T> eee = C3(P.orr[t][0], nb), ooe = C3(P.orr[t][1], nb), oeo = C3(P.orr[t][2], nb), eoo = C3(P.orr[t][3], nb);
        A3<T> me = C3(P.omr[t][0], nb), mo = C3(P.omr[t][1], nb);
        A3<T> bl = G3(P.og_r[t + 1], nb);
        CTA_FOR3(a, b, c, 0, nb) {  // Eq. Erred
            auto avg = [&](int i, int j, int k) {
                return (T(6) * g(i, j, k) + (g(i + 1, j, k) + g(i - 1, j, k)) + (g(i, j + 1, k) + g(i, j - 1, k)) +
                        (g(i, j, k + 1) + g(i, j, k - 1))) * T(1.0 / 12.0);
            };
            if (a >= 1 && b >= 1 && c >= 1) eee(a, b, c) = avg(2 * a, 2 * b, 2 * c);
            if (c >= 1) ooe(a, b, c) = avg(2 * a + 1, 2 * b + 1, 2 * c);
            if (b >= 1) oeo(a, b, c) = avg(2 * a + 1, 2 * b, 2 * c + 1);
            if (a >= 1) eoo(a, b, c) = avg(2 * a, 2 * b + 1, 2 * c + 1);
        }
        __syncthreads();
        CTA_FOR3(a, b, c, 0, nb) {  // Eq. Ermagc, Eq. Ermagm
            if (a >= 1 && b >= 1 && c >= 1)
                me(a, b, c) = (T(12) * eee(a, b, c) +
                               fcc12(A3<const T>{ooe.p, ooe.pitch, ooe.rows}, A3<const T>{oeo.p, oeo.pitch, oeo.rows},
                                     A3<const T>{eoo.p, eoo.pitch, eoo.rows}, a, b, c)) * T(1.0 / 24.0);
            mo(a, b, c) = ((eoo(a, b, c) + eoo(a + 1, b, c)) + (oeo(a, b, c) + oeo(a, b + 1, c)) +
                           (ooe(a, b, c) + ooe(a, b, c + 1))) * T(1.0 / 6.0);
        }
        __syncthreads();
        CTA_FOR3(a, b, c, 1, nb) {  // Eq. Erblu
            bl(a, b, c) = (T(8) * me(a, b, c) + ctr8(A3<const T>{mo.p, mo.pitch, mo.rows}, a, b, c)) * T(0.0625);
        }
        __syncthreads();
    }
    {   // exact solve on the coarsest grid
        const int s = P.nk[ntri], nn = s * s * s;
        A3<T> r = G3(P.og_r[ntri], s), v = G3(P.og_v[ntri], s);
        double *rv = Gs + P.ng;  // the right-hand side, dense
        for (int q = tid; q < nn; q += nt) rv[q] = (double)r(q % s + 1, (q / s) % s + 1, q / (s * s) + 1);
        __syncthreads();
        for (int q = tid; q < nn; q += nt) {
            double acc = 0.0;
            for (int t = 0; t < nn; t++) acc += Gs[q * nn + t] * rv[t];
            v(q % s + 1, (q / s) % s + 1, q / (s * s) + 1) = (T)acc;
        }
    }
    __syncthreads();
    for (int t = ntri - 1; t >= 0; t--) {
        const int n = P.nk[t], nb = (n - 1) / 2;
        A3<T> rg = G3(P.og_r[t], n), vg = G3(P.og_v[t], n), vb = G3(P.og_v[t + 1], nb);
        A3<T> r_e = C3(P.orr[t][0], nb), r_ooe = C3(P.orr[t][1], nb), r_oeo = C3(P.orr[t][2], nb), r_eoo = C3(P.orr[t][3], nb);
        A3<T> v_e = C3(P.orv[t][0], nb), v_ooe = C3(P.orv[t][1], nb), v_oeo = C3(P.orv[t][2], nb), v_eoo = C3(P.orv[t][3], nb);
        A3<T> rme = C3(P.omr[t][0], nb), rmo = C3(P.omr[t][1], nb), vme = C3(P.omv[t][0], nb), vmo = C3(P.omv[t][1], nb);
        const T cm = (T)P.cm[t], c1 = (T)P.cr1[t], c2 = (T)P.cr2[t], cg = (T)P.cg[t];
        CTA_FOR3(a, b, c, 0, nb) {  // Eq. Emprolm: centres
            T s = ((vb(a, b, c) + vb(a + 1, b, c)) + (vb(a, b + 1, c) + vb(a + 1, b + 1, c))) +
                  ((vb(a, b, c + 1) + vb(a + 1, b, c + 1)) + (vb(a, b + 1, c + 1) + vb(a + 1, b + 1, c + 1)));
            vmo(a, b, c) = (s - cm * rmo(a, b, c)) * T(0.125);
        }
        __syncthreads();
        CTA_FOR3(a, b, c, 1, nb) {  // Eq. Emprolb: blue corners
            vme(a, b, c) = (ctr8(A3<const T>{vmo.p, vmo.pitch, vmo.rows}, a, b, c) - cm * rme(a, b, c)) * T(0.125);
        }
        __syncthreads();
        CTA_FOR3(a, b, c, 0, nb) {  // Eq. Erprolr: red face centres
            if (c >= 1) {
                T ctr = vmo(a, b, c - 1) + vmo(a, b, c);
                T cor = (vme(a, b, c) + vme(a + 1, b, c)) + (vme(a, b + 1, c) + vme(a + 1, b + 1, c));
                v_ooe(a, b, c) = (T(2) * ctr + cor - c1 * r_ooe(a, b, c)) * T(0.125);
            }
            if (b >= 1) {
                T ctr = vmo(a, b - 1, c) + vmo(a, b, c);
                T cor = (vme(a, b, c) + vme(a + 1, b, c)) + (vme(a, b, c + 1) + vme(a + 1, b, c + 1));
                v_oeo(a, b, c) = (T(2) * ctr + cor - c1 * r_oeo(a, b, c)) * T(0.125);
            }
            if (a >= 1) {
                T ctr = vmo(a - 1, b, c) + vmo(a, b, c);
                T cor = (vme(a, b, c) + vme(a, b + 1, c)) + (vme(a, b, c + 1) + vme(a, b + 1, c + 1));
                v_eoo(a, b, c) = (T(2) * ctr + cor - c1 * r_eoo(a, b, c)) * T(0.125);
            }
        }
        __syncthreads();
        CTA_FOR3(a, b, c, 1, nb) {  // Eq. Erprolm: magenta corners
            v_e(a, b, c) = (fcc12(A3<const T>{v_ooe.p, v_ooe.pitch, v_ooe.rows}, A3<const T>{v_oeo.p, v_oeo.pitch, v_oeo.rows},
                                  A3<const T>{v_eoo.p, v_eoo.pitch, v_eoo.rows}, a, b, c) - c2 * r_e(a, b, c)) * T(1.0 / 12.0);
        }
        __syncthreads();
        Red3<const T> vr{A3<const T>{v_e.p, v_e.pitch, v_e.rows}, A3<const T>{v_ooe.p, v_ooe.pitch, v_ooe.rows},
                         A3<const T>{v_oeo.p, v_oeo.pitch, v_oeo.rows}, A3<const T>{v_eoo.p, v_eoo.pitch, v_eoo.rows}};
        for (int k = 1 + tz; k <= n; k += 8)  // Eq. Egprolg: green-only points, i + j + k odd
            for (int j = 1 + ty; j <= n; j += 8)
                for (int i = 1 + ((j + k) & 1) + 2 * tx; i <= n; i += 32) {
            T s = (red3(vr, i - 1, j, k) + red3(vr, i + 1, j, k)) + (red3(vr, i, j - 1, k) + red3(vr, i, j + 1, k)) +
                  (red3(vr, i, j, k - 1) + red3(vr, i, j, k + 1));
            vg(i, j, k) = (s - cg * rg(i, j, k)) * T(1.0 / 6.0);
        }
        __syncthreads();
        for (int k = 1 + tz; k <= n; k += 8)  // Eq. Egprolr: red points, i + j + k even
            for (int j = 1 + ty; j <= n; j += 8)
                for (int i = 2 - ((j + k) & 1) + 2 * tx; i <= n; i += 32) {
            T s = (vg(i - 1, j, k) + vg(i + 1, j, k)) + (vg(i, j - 1, k) + vg(i, j + 1, k)) +
                  (vg(i, j, k - 1) + vg(i, j, k + 1));
            vg(i, j, k) = (s - cg * rg(i, j, k)) * T(1.0 / 6.0);
        }
        __syncthreads();
    }
    {
        const int n = P.nk[0];
        A3<T> g = G3(P.og_v[0], n);
        CTA_FOR3(i, j, k, 1, n) vg_out(i, j, k) = g(i, j, k);
    }
#undef CTA_FOR3
}

}  // namespace mg

namespace mg {

// ---------------------------------------------------------------------------
// Finest pair of a mixed-precision 2D solve, fused with u += v and the next
// residual.
//
// The residual is carried from cycle to cycle as a float-float pair
// r = hi + lo: hi is the FP32 residual that the levels and the norm read
// (double-buffered by Ctrl.par, since the sweep reads it in a halo), lo a
// second FP32 array.  A cycle's correction v (FP32) gives
//   u_new = u + v          (the one FP64 operation per point)
//   r_new = r - L v,       L v = s2 * sum over the four axis neighbours of (v_nb - v)
// where v is first rounded to a multiple of a quantum q set by a bound on
// |v| over the whole level (quant_magic), so that the neighbour sum and
// L v are exact in FP32; s2 = 1/h^2 is a power of two (n = 2^m - 1), so the
// scaling is exact; the subtraction is a float-float operation, error
// ~2^-48 |r|.  u += v and r -= L v use the same rounded v, so the carried r
// stays the residual of u up to that error (and the FP64 rounding of u); a
// direct residual starts and ends every solve.  The rounding of v itself
// (at most 2^-21 of the bound) only perturbs the correction.
// ---------------------------------------------------------------------------

__device__ __forceinline__ void two_sum(float a, float b, float &s, float &e) {
    s = a + b;
    const float bv = s - a;
    const float av = s - bv;
    e = (a - av) + (b - bv);
}

// (nh, nl) ~= (hi + lo) - s2 * l, l exact, s2 a power of two
__device__ __forceinline__ void ff_sub1(float hi, float lo, float l, float s2, float &nh, float &nl) {
    float s, e;
    two_sum(hi, -s2 * l, s, e);
    two_sum(s, lo + e, nh, nl);
}

// Rounding of the finest correction of the fused mixed path to a quantum.
// With 2^E >= |v| for every v of the level (a bound formed before the sweep
// from the level it starts from and the residual), each v is rounded to a
// multiple of q = 2^(E - qb): v_q = (v + M) - M with M = 1.5 * 2^(E - qb + 23),
// whose unit in the last place is q (v + M stays in M's binade).  Then the
// Laplacian of v_q -- the neighbour sum and the centre term, all multiples
// of q below 2^24 q with qb = 21 (5-point) or 20 (7-point) -- is exact in
// FP32, and u += v_q and r -= L v_q stay consistent to the float-float
// rounding of r.  The rounding moves v by at most q / 2 <= 2^-qb of the
// bound.  E is clamped to [-100, 100]; a bound above 2^100 or NaN gives a
// NaN quantizer (the solve then reports divergence).
__device__ __forceinline__ float quant_magic(float bound, int qb) {
    if (!(bound <= 1.2676506e30f)) return __int_as_float(0x7fc00000);  // 2^100
    const unsigned b = __float_as_uint(bound);
    const int e = max((int)(b >> 23) - 127 + ((b & 0x7fffffu) != 0u), -100);
    return __uint_as_float(((unsigned)(e - qb + 150) << 23) | 0x400000u);
}
__device__ __forceinline__ float quant(float v, float M) { return __fsub_rn(__fadd_rn(v, M), M); }
// sum of the four neighbours - 4 c of quantized values: exact
__device__ __forceinline__ float lap_q4(float n0, float n1, float n2, float n3, float c) {
    return fmaf(-4.f, c, __fadd_rn(__fadd_rn(n0, n1), __fadd_rn(n2, n3)));
}

// Work decomposition of k_up0_ff_2d.  A cell (a,b) is the four green points
// (2a..2a+1, 2b..2b+1).  A warp owns 32*FF_K consecutive cell columns (FF_K
// per lane) and walks a strip of cell rows upward, holding every
// intermediate row in registers: x neighbours come from the adjacent lane by
// shuffle, y neighbours from earlier steps.  The chain reaches -2..+3 cells in
// x, so a warp writes its middle FF_W cells (an even count, so that the four
// points of a lane's two cells are one aligned 16-byte group of every green
// row); a strip starts 4 rows early to fill the chain (those steps write
// nothing).  Blocks are persistent: warps take (column, strip) items in turn.
constexpr int FF_K = 2;
constexpr int FF_W = 32 * FF_K - 6;
constexpr int FF_WARPS = 4;

// Step b of a strip: load blue row b+3, red rows b+2 and green-residual rows
// 2b+2, 2b+3; form red OO row b+2 (Eq. Eajacr) and red EE row b+2
// (Eq. Eajacb) with c2 = 2 p h^2, the green-only points of cell row b+1, the
// re-relaxed red points EE of row b+1 and OO of row b (the red-to-green sweep
// of Section 2.2, c1 = p h^2); then apply v to the four points of every own
// cell of row b.  Values outside the interior are zero, as in the oracle.
// MODE: UP_RR the mixed finest pair (u += v and the carried residual, rga/rgb
// double-buffered by par); UP_ADD u += v; UP_STORE v stored in vg (a coarser
// pair; with ctl, also the largest |v| stored into ctl[p].vmax).  VU: u is
// 16-byte aligned with an even pitch (vector access to u).  UD: u and the
// residual's low part of the own cells are loaded into registers at the
// start of each step instead of being copied into shared memory one step
// ahead (more registers per thread: for launches with few warps per SM).
enum { UP_RR = 0, UP_ADD = 1, UP_STORE = 2 };

// The streaming kernels below keep one step of every warp's inputs in flight
// (cp.async) while the warp computes the current step.  Each lane copies and
// later reads only its own slots, so a lane's own wait_group orders them.

// one step's inputs of one warp in shared memory (slot = lane): the chain's
// blue row b+3, red OO / EE rows b+2 and green residual rows 2b+2, 2b+3 over
// the lane's two cells; u of the own cells' green rows 2b, 2b+1 (two FP64
// pairs per row) and the residual's lo part of those rows
struct FFChain {
    float4 g2[32], g3[32];
    float2 bl[32], ro[32], re[32];
};
struct FFU {
    double2 u[2][2][32];
};
struct FFL {
    float4 l[2][32];
};

template <int MODE, bool VU, bool UD = false>
__global__ void __launch_bounds__(32 * FF_WARPS) k_up_ff_2d(A2<const float> blue, A2<const float> ree,
                                                            A2<const float> roo, A2<float> rga, float *rgb, A2<float> vg,
                                                            float *__restrict__ rlo, double *__restrict__ u, int up,
                                                            int nb, float c2, float c1, float s2, int tb,
                                                            double *part, Ctrl *ctl, const int *done, Bt B) {
    __shared__ double sh[32];
    __shared__ float shm[32];
    // stages of the copy pipeline: a coarser pair (UP_STORE, latency-bound:
    // few steps per warp and little arithmetic per step) copies two steps
    // ahead, the finest pair one (its registers and shared memory are the
    // limit there)
    constexpr int NST = MODE == UP_STORE ? 3 : 2;
    __shared__ FFChain SC[FF_WARPS][NST];
    __shared__ FFU SU[MODE != UP_STORE && !UD ? FF_WARPS : 1][UD ? 1 : NST];
    __shared__ FFL SL[MODE == UP_RR && !UD ? FF_WARPS : 1][UD ? 1 : NST];
    constexpr unsigned FULL = 0xffffffffu;
    constexpr int K = FF_K;
    constexpr bool RR = MODE == UP_RR, UPD = MODE != UP_STORE;
    const int prob = blockIdx.z;
    if (stop(bt_done(done, prob, B))) return;
    A2<float> rg = rga, rnew = rga;
    int pq = 0;      // current residual buffer
    float M = 0.f;   // quantizer of v (quant_magic): |v| <= |blue| + (c2 + c1) max|r| / 2
    if (RR) {
        const Ctrl &C = ctl[prob];
        pq = C.par;
        (pq ? rg : rnew).p = rgb;
        M = quant_magic((__uint_as_float(C.vmax) + 0.5f * (c2 + c1) * __uint_as_float(C.rmax[pq])) * 1.002f, 21);
    }
    blue = bt_at(blue, prob, B); ree = bt_at(ree, prob, B); roo = bt_at(roo, prob, B);
    rg = bt_at(rg, prob, B); rnew = bt_at(rnew, prob, B); vg = bt_at(vg, prob, B);
    if (RR) rlo = bt_ptr(rlo, prob, B);
    if (UPD && B.utab) u = B.utab[prob];
    if (RR) part += (size_t)prob * B.nparts;
    const int lane = threadIdx.x, w = threadIdx.y;
    const int n = 2 * nb + 1, gp = rga.pitch;
    const int ncol = (nb + FF_W) / FF_W, nstrip = (nb + tb) / tb;
    float sq = 0.f, mx = 0.f;
    for (int it = blockIdx.x * FF_WARPS + w; it < ncol * nstrip; it += gridDim.x * FF_WARPS) {
        const int col = it % ncol, strip = it / ncol;
        const int A = col * FF_W - 2, a0 = A + K * lane;
        // nb is odd and a0 even: the lane's K cells are all in [0, nb] or all outside
        const bool in = a0 >= 0 && a0 <= nb;
        const bool own = in && a0 >= A + 2 && a0 < A + 2 + FF_W;
        bool pos[K];  // column of cell k holds green points with even x (a >= 1)
#pragma unroll
        for (int k = 0; k < K; k++) pos[k] = in && a0 + k >= 1;
        const int b0 = strip * tb, b1 = min(b0 + tb, nb + 1), bs = max(b0 - 4, -2);
        const int ac = in ? a0 : 0;  // a valid column for the addresses of zero-filled copies
        // stage the inputs of step bb into buffer st
        auto issue = [&](int st, int bb) {
            FFChain &C = SC[w][st];
            cp_async8(&C.bl[lane], &blue(ac, in && bb + 3 <= nb + 1 ? bb + 3 : 0), in && bb + 3 <= nb + 1);
            const bool r2 = in && bb + 2 >= 0 && bb + 2 <= nb;
            cp_async8(&C.ro[lane], &roo(ac, r2 ? bb + 2 : 0), r2);
            cp_async8(&C.re[lane], &ree(ac, r2 ? bb + 2 : 0), r2);
            const bool y2 = in && 2 * bb + 2 >= 1 && 2 * bb + 2 <= n, y3 = in && 2 * bb + 3 >= 1 && 2 * bb + 3 <= n;
            cp_async16(&C.g2[lane], &rg(2 * ac, y2 ? 2 * bb + 2 : 0), y2);
            cp_async16(&C.g3[lane], &rg(2 * ac, y3 ? 2 * bb + 3 : 0), y3);
            if (UPD && !UD && own && bb >= b0) {
                const bool row0 = bb >= 1;
#pragma unroll
                for (int r = 0; r < 2; r++) {
                    const int y = 2 * bb + r;
                    const bool ok = r == 1 || row0;
                    const double *src = u + (size_t)(ok ? y : 1) * up + 2 * a0;
                    if (VU) {
                        cp_async16(&SU[w][st].u[r][0][lane], src, ok);
                        cp_async16(&SU[w][st].u[r][1][lane], src + 2, ok);
                    } else {
#pragma unroll
                        for (int q = 0; q < 2 * K; q++) {
                            const bool px = ok && ((q & 1) || pos[q >> 1]);
                            double *d = q < 2 ? &SU[w][st].u[r][0][lane].x : &SU[w][st].u[r][1][lane].x;
                            cp_async8(d + (q & 1), src + q, px);
                        }
                    }
                    if (RR) cp_async16(&SL[w][st].l[r][lane], rlo + (size_t)(ok ? y : 1) * gp + 2 * a0, ok);
                }
            }
            cp_async_commit();
        };
        // chain state, rows relative to the step's b
        float bl2[K], oo0[K], oo1[K], ee1[K], oe0[K], eom[K], eo0[K], ce0[K], com[K], r0[2 * K], r1[2 * K];
#pragma unroll
        for (int k = 0; k < K; k++) {
            bl2[k] = oo0[k] = oo1[k] = ee1[k] = oe0[k] = eom[k] = eo0[k] = ce0[k] = com[k] = 0.f;
            r0[2 * k] = r0[2 * k + 1] = r1[2 * k] = r1[2 * k + 1] = 0.f;
        }
        if (in && bs + 2 >= 0) {
            const float2 q = *reinterpret_cast<const float2 *>(&blue(a0, bs + 2));
            bl2[0] = q.x; bl2[1] = q.y;
        }
        issue(0, bs);
        if (NST == 3) {
            if (bs + 1 < b1) issue(1, bs + 1);
            else cp_async_commit();
        }
        for (int b = bs; b < b1; b++) {
            const int st = NST == 2 ? (b - bs) & 1 : (b - bs) % 3;
            // one group committed per step: the copies of step b + NST - 1
            if (b + NST - 1 < b1) issue(NST == 2 ? st ^ 1 : (st + 2) % 3, b + NST - 1);
            else cp_async_commit();
            if (NST == 2) cp_async_wait1();  // this lane's copies of step b have landed
            else cp_async_wait2();
            float bl3[K], ro2[K], re2[K], g2[2 * K], g3[2 * K];
            {
                const FFChain &C = SC[w][st];
                const float2 x = C.bl[lane], y = C.ro[lane], z = C.re[lane];
                const float4 p = C.g2[lane], q = C.g3[lane];
                bl3[0] = x.x; bl3[1] = x.y; ro2[0] = y.x; ro2[1] = y.y; re2[0] = z.x; re2[1] = z.y;
                g2[0] = p.x; g2[1] = p.y; g2[2] = p.z; g2[3] = p.w;
                g3[0] = q.x; g3[1] = q.y; g3[2] = q.z; g3[3] = q.w;
            }
            const bool upd = own && b >= b0;
            const bool row0 = b >= 1;  // green row 2b is interior
            const int yo = upd ? 2 * b : 0, xo = upd ? 2 * a0 : 0;  // pointers formed for own cells only
            double *ur0 = UPD ? u + (size_t)yo * up + xo : nullptr, *ur1 = UPD ? ur0 + up : nullptr;
            float *lr0 = RR ? rlo + (size_t)yo * gp + xo : nullptr, *lr1 = RR ? lr0 + gp : nullptr;
            double u0[2 * K], u1[2 * K];
            float l0[2 * K], l1[2 * K];
            if (UD && UPD && upd) {  // rows 2b and 2b+1 of the own cells (row 0 is the ring: read, not used)
                if (VU) {
                    const double2 a = reinterpret_cast<const double2 *>(ur0)[0], bq = reinterpret_cast<const double2 *>(ur0)[1];
                    const double2 c = reinterpret_cast<const double2 *>(ur1)[0], d = reinterpret_cast<const double2 *>(ur1)[1];
                    u0[0] = a.x; u0[1] = a.y; u0[2] = bq.x; u0[3] = bq.y;
                    u1[0] = c.x; u1[1] = c.y; u1[2] = d.x; u1[3] = d.y;
                } else {
#pragma unroll
                    for (int q = 0; q < 2 * K; q++) { u0[q] = ur0[q]; u1[q] = ur1[q]; }
                }
                if (RR) {
                    const float4 a = *reinterpret_cast<const float4 *>(lr0), c = *reinterpret_cast<const float4 *>(lr1);
                    l0[0] = a.x; l0[1] = a.y; l0[2] = a.z; l0[3] = a.w;
                    l1[0] = c.x; l1[1] = c.y; l1[2] = c.z; l1[3] = c.w;
                }
            }
            // ---- the chain
            const bool y_oo2 = b + 2 >= 0 && b + 2 <= nb, y_ee2 = b + 2 >= 1 && b + 2 <= nb;
            const bool y_oe1 = b + 1 >= 1 && b + 1 <= nb, y_eo1 = b + 1 >= 0 && b + 1 <= nb;
            const bool y_co0 = b >= 0 && b <= nb;
            float oo2[K], ee2[K], oe1[K], eo1[K], ce1[K], co0[K];
            {
                const float bl2R = __shfl_down_sync(FULL, bl2[0], 1), bl3R = __shfl_down_sync(FULL, bl3[0], 1);
#pragma unroll
                for (int k = 0; k < K; k++) {
                    const float r2 = k + 1 < K ? bl2[k + 1] : bl2R, r3 = k + 1 < K ? bl3[k + 1] : bl3R;
                    oo2[k] = (in && y_oo2) ? ((bl2[k] + r2) + (bl3[k] + r3) - c2 * ro2[k]) * 0.25f : 0.f;
                }
            }
            const float oo1L = __shfl_up_sync(FULL, oo1[K - 1], 1), oo2L = __shfl_up_sync(FULL, oo2[K - 1], 1);
#pragma unroll
            for (int k = 0; k < K; k++) {
                const float l1v = k > 0 ? oo1[k - 1] : oo1L, l2v = k > 0 ? oo2[k - 1] : oo2L;
                ee2[k] = (pos[k] && y_ee2) ? ((l1v + oo1[k]) + (l2v + oo2[k]) - c2 * re2[k]) * 0.25f : 0.f;
            }
            {
                const float ee1R = __shfl_down_sync(FULL, ee1[0], 1);
#pragma unroll
                for (int k = 0; k < K; k++) {
                    const float er = k + 1 < K ? ee1[k + 1] : ee1R, ol = k > 0 ? oo1[k - 1] : oo1L;
                    oe1[k] = (in && y_oe1) ? ((ee1[k] + er) + (oo0[k] + oo1[k]) - c1 * g2[2 * k + 1]) * 0.25f : 0.f;
                    eo1[k] = (pos[k] && y_eo1) ? ((ol + oo1[k]) + (ee1[k] + ee2[k]) - c1 * g3[2 * k]) * 0.25f : 0.f;
                    if (RR) { oe1[k] = quant(oe1[k], M); eo1[k] = quant(eo1[k], M); }
                }
            }
            const float oe1L = __shfl_up_sync(FULL, oe1[K - 1], 1), eo0R = __shfl_down_sync(FULL, eo0[0], 1);
#pragma unroll
            for (int k = 0; k < K; k++) {
                const float ol = k > 0 ? oe1[k - 1] : oe1L, er = k + 1 < K ? eo0[k + 1] : eo0R;
                ce1[k] = (pos[k] && y_oe1) ? ((ol + oe1[k]) + (eo0[k] + eo1[k]) - c1 * g2[2 * k]) * 0.25f : 0.f;
                co0[k] = (in && y_co0) ? ((eo0[k] + er) + (oe0[k] + oe1[k]) - c1 * r1[2 * k + 1]) * 0.25f : 0.f;
                if (RR) { ce1[k] = quant(ce1[k], M); co0[k] = quant(co0[k], M); }
            }
            // ---- apply v to the own cells of row b
            const float oe0L = __shfl_up_sync(FULL, oe0[K - 1], 1), ce0R = __shfl_down_sync(FULL, ce0[0], 1);
            const float co0L = __shfl_up_sync(FULL, co0[K - 1], 1);
            if (!UPD && upd) {
                float *v0 = &vg(xo, yo), *v1 = v0 + vg.pitch;
                if (row0) *reinterpret_cast<float4 *>(v0) = make_float4(ce0[0], oe0[0], ce0[1], oe0[1]);
                *reinterpret_cast<float4 *>(v1) = make_float4(eo0[0], co0[0], eo0[1], co0[1]);
                if (ctl) {
#pragma unroll
                    for (int k = 0; k < K; k++)
                        mx = fmaxf(fmaxf(mx, fmaxf(fabsf(ce0[k]), fabsf(oe0[k]))), fmaxf(fabsf(eo0[k]), fabsf(co0[k])));
                }
            }
            if (UPD && upd) {
                if (!UD) {
                    const double2 a = SU[w][st].u[0][0][lane], bq = SU[w][st].u[0][1][lane];
                    const double2 c = SU[w][st].u[1][0][lane], d = SU[w][st].u[1][1][lane];
                    u0[0] = a.x; u0[1] = a.y; u0[2] = bq.x; u0[3] = bq.y;
                    u1[0] = c.x; u1[1] = c.y; u1[2] = d.x; u1[3] = d.y;
                }
                if (RR && !UD) {
                    const float4 a = SL[w][st].l[0][lane], c = SL[w][st].l[1][lane];
                    l0[0] = a.x; l0[1] = a.y; l0[2] = a.z; l0[3] = a.w;
                    l1[0] = c.x; l1[1] = c.y; l1[2] = c.z; l1[3] = c.w;
                }
                float h0[2 * K], h1[2 * K];
#pragma unroll
                for (int k = 0; k < K; k++) {
                    const float oel = k > 0 ? oe0[k - 1] : oe0L, cer = k + 1 < K ? ce0[k + 1] : ce0R;
                    const float col_ = k > 0 ? co0[k - 1] : co0L, eor = k + 1 < K ? eo0[k + 1] : eo0R;
                    float nh, nl;
                    // EE (2a, 2b)
                    nh = nl = 0.f;
                    if (pos[k] && row0) {
                        if (RR) ff_sub1(r0[2 * k], l0[2 * k], lap_q4(oel, oe0[k], eom[k], eo0[k], ce0[k]), s2, nh, nl);
                        u0[2 * k] += widen(ce0[k]);
                    }
                    h0[2 * k] = nh; l0[2 * k] = nl;
                    // OE (2a+1, 2b)
                    nh = nl = 0.f;
                    if (row0) {
                        if (RR) ff_sub1(r0[2 * k + 1], l0[2 * k + 1], lap_q4(ce0[k], cer, com[k], co0[k], oe0[k]), s2, nh, nl);
                        u0[2 * k + 1] += widen(oe0[k]);
                    }
                    h0[2 * k + 1] = nh; l0[2 * k + 1] = nl;
                    // EO (2a, 2b+1)
                    nh = nl = 0.f;
                    if (pos[k]) {
                        if (RR) ff_sub1(r1[2 * k], l1[2 * k], lap_q4(col_, co0[k], ce0[k], ce1[k], eo0[k]), s2, nh, nl);
                        u1[2 * k] += widen(eo0[k]);
                    }
                    h1[2 * k] = nh; l1[2 * k] = nl;
                    // OO (2a+1, 2b+1)
                    if (RR) ff_sub1(r1[2 * k + 1], l1[2 * k + 1], lap_q4(eo0[k], eor, oe0[k], oe1[k], co0[k]), s2, nh, nl);
                    u1[2 * k + 1] += widen(co0[k]);
                    h1[2 * k + 1] = nh; l1[2 * k + 1] = nl;
                }
                if (RR) {
#pragma unroll
                    for (int q = 0; q < 2 * K; q++) {
                        sq = fmaf(h0[q], h0[q], fmaf(h1[q], h1[q], sq));
                        mx = fmaxf(mx, fmaxf(fabsf(h0[q]), fabsf(h1[q])));
                    }
                    float *hr0 = &rnew(xo, yo), *hr1 = hr0 + gp;
                    if (row0) {
                        *reinterpret_cast<float4 *>(hr0) = make_float4(h0[0], h0[1], h0[2], h0[3]);
                        *reinterpret_cast<float4 *>(lr0) = make_float4(l0[0], l0[1], l0[2], l0[3]);
                    }
                    *reinterpret_cast<float4 *>(hr1) = make_float4(h1[0], h1[1], h1[2], h1[3]);
                    *reinterpret_cast<float4 *>(lr1) = make_float4(l1[0], l1[1], l1[2], l1[3]);
                }
                if (VU) {
                    if (row0) {
                        reinterpret_cast<double2 *>(ur0)[0] = make_double2(u0[0], u0[1]);
                        reinterpret_cast<double2 *>(ur0)[1] = make_double2(u0[2], u0[3]);
                    }
                    reinterpret_cast<double2 *>(ur1)[0] = make_double2(u1[0], u1[1]);
                    reinterpret_cast<double2 *>(ur1)[1] = make_double2(u1[2], u1[3]);
                } else {
#pragma unroll
                    for (int q = 0; q < 2 * K; q++) {
                        const bool px = (q & 1) || pos[q >> 1];
                        if (row0 && px) ur0[q] = u0[q];
                        if (px) ur1[q] = u1[q];
                    }
                }
            }
            // ---- advance the chain one cell row
#pragma unroll
            for (int k = 0; k < K; k++) {
                bl2[k] = bl3[k]; oo0[k] = oo1[k]; oo1[k] = oo2[k]; ee1[k] = ee2[k]; oe0[k] = oe1[k];
                eom[k] = eo0[k]; eo0[k] = eo1[k]; ce0[k] = ce1[k]; com[k] = co0[k];
                r0[2 * k] = g2[2 * k]; r0[2 * k + 1] = g2[2 * k + 1];
                r1[2 * k] = g3[2 * k]; r1[2 * k + 1] = g3[2 * k + 1];
            }
        }
        cp_async_wait0();
    }
    if (RR) {
        const double s = block_sum((double)sq, sh);
        const float m = block_max(mx, shm);
        if (threadIdx.x == 0 && threadIdx.y == 0) {
            part[blockIdx.x] = s;
            atomicMax(&ctl[prob].rmax[pq ^ 1], __float_as_uint(m));
        }
    } else if (!UPD && ctl) {  // the blue level of the fused mixed path's finest pair: its bound on |v|
        const float m = block_max(mx, shm);
        if (threadIdx.x == 0 && threadIdx.y == 0) atomicMax(&ctl[prob].vmax, __float_as_uint(m));
    }
}

// ---------------------------------------------------------------------------
// Pair restriction green -> red -> blue (Eq. Erest2r, then Eq. Erest2b) as a
// warp-streaming kernel over FP32 levels, with the decomposition of
// k_up_ff_2d: a warp owns 64 cell columns (2 per lane) and walks a strip of
// cell rows; the green rows 2b-1..2b+2 of step b are held in registers (two
// loaded per step), x neighbours come by shuffle.  Red OO of cell row b
// needs the green neighbours at +-1, red EE the same, blue(a,b) the OO
// values of cells a-1..a of rows b-1..b, so a warp writes its middle FD_W
// cells and a strip starts one row early.  galt/par: the finest green
// residual of the mixed solve is double-buffered (Ctrl.par picks the current).
// ---------------------------------------------------------------------------
constexpr int FD_W = 60;

__global__ void __launch_bounds__(32 * FF_WARPS) k_down_ff_2d(A2<const float> g, A2<float> ee, A2<float> oo,
                                                              A2<float> blue, int nb, int tb, const float *galt,
                                                              const int *par, const int *done, Bt B) {
    constexpr unsigned FULL = 0xffffffffu;
    const int prob = blockIdx.z;
    if (stop(bt_done(done, prob, B))) return;
    if (galt && par[(size_t)prob * B.ctl_stride]) g.p = galt;
    g = bt_at(g, prob, B); ee = bt_at(ee, prob, B); oo = bt_at(oo, prob, B); blue = bt_at(blue, prob, B);
    const int lane = threadIdx.x;
    const int n = 2 * nb + 1;
    const int ncol = (nb + FD_W) / FD_W, nstrip = (nb + tb) / tb;
    for (int it = blockIdx.x * FF_WARPS + threadIdx.y; it < ncol * nstrip; it += gridDim.x * FF_WARPS) {
        const int col = it % ncol, strip = it / ncol;
        const int A = col * FD_W - 2, a0 = A + 2 * lane;
        const bool in = a0 >= 0 && a0 <= nb;  // nb odd, a0 even: both cells in [0, nb] or neither
        const bool own = in && a0 >= A + 2 && a0 < A + 2 + FD_W;
        const bool pos0 = a0 >= 1;            // cell a0 has EE / blue points (a >= 1)
        const int b0 = strip * tb, b1 = min(b0 + tb, nb + 1), bs = max(b0 - 1, 0);
        auto row = [&](int y) -> float4 {
            if (in && y >= 0 && y <= n + 1) return *reinterpret_cast<const float4 *>(&g(2 * a0, y));
            return make_float4(0.f, 0.f, 0.f, 0.f);
        };
        // green rows 2b-1 .. 2b+2 of step b; the two rows a step adds are
        // loaded two steps ahead (a warp's few steps are latency-bound)
        float4 gm = row(2 * bs - 1), g0 = row(2 * bs), g1 = row(2 * bs + 1), g2 = row(2 * bs + 2);
        float4 p1 = row(2 * bs + 3), p2 = row(2 * bs + 4);  // the rows step bs adds
        float om0 = 0.f, om1 = 0.f;  // OO(a0, b-1), OO(a0+1, b-1)
        for (int b = bs; b < b1; b++) {
            const float4 n1 = p1, n2 = p2;
            p1 = row(2 * b + 5);  // the rows step b + 1 adds
            p2 = row(2 * b + 6);
            const float g0L = __shfl_up_sync(FULL, g0.w, 1), g1R = __shfl_down_sync(FULL, g1.x, 1);
            // red EE of cells a0, a0+1 at green (2a, 2b); OO at (2a+1, 2b+1)
            const bool yb = b >= 1;
            const float e0 = (pos0 && yb) ? (4.f * g0.x + (g0L + g0.y) + (gm.x + g1.x)) * 0.125f : 0.f;
            const float e1 = (in && yb) ? (4.f * g0.z + (g0.y + g0.w) + (gm.z + g1.z)) * 0.125f : 0.f;
            const float o0 = in ? (4.f * g1.y + (g1.x + g1.z) + (g0.y + g2.y)) * 0.125f : 0.f;
            const float o1 = in ? (4.f * g1.w + (g1.z + g1R) + (g0.w + g2.w)) * 0.125f : 0.f;
            // OO(a0-1, b-1) and OO(a0-1, b) from the left lane
            const float omL = __shfl_up_sync(FULL, om1, 1), o0L = __shfl_up_sync(FULL, o1, 1);
            const float bl0 = (pos0 && yb) ? (4.f * e0 + (omL + om0) + (o0L + o0)) * 0.125f : 0.f;
            const float bl1 = (in && yb) ? (4.f * e1 + (om0 + om1) + (o0 + o1)) * 0.125f : 0.f;
            if (own && b >= b0) {
                *reinterpret_cast<float2 *>(&oo(a0, b)) = make_float2(o0, o1);
                if (yb) {
                    *reinterpret_cast<float2 *>(&ee(a0, b)) = make_float2(e0, e1);
                    *reinterpret_cast<float2 *>(&blue(a0, b)) = make_float2(bl0, bl1);
                }
            }
            gm = g1; g0 = g2; g1 = n1; g2 = n2; om0 = o0; om1 = o1;
        }
    }
}

// sum of f^2 over the interior (the norm of the right-hand side of an order-2
// solve): FP32 squares per thread, FP64 block sums; grid as k_res0_2d (2D) or
// k_res0_3d (3D) so the partial count matches
template <int DIM>
__global__ void __launch_bounds__(256) k_norm_f(const double *__restrict__ f, int up, int n, double *part,
                                                const int *done, Bt B) {
    __shared__ double sh[32];
    const int prob = bt_prob(B), bz = bt_z(B);
    if (stop(bt_done(done, prob, B))) return;
    if (B.ftab) f = B.ftab[prob];
    part += (size_t)prob * B.nparts;
    const int i = blockIdx.x * 32 + threadIdx.x + 1;
    float acc = 0.f;
    if (DIM == 2) {
        const int j0 = (blockIdx.y * 8 + threadIdx.y) * RES_ROWS + 1;
        if (i <= n)
            for (int q = 0; q < RES_ROWS && j0 + q <= n; q++) {
                const float v = narrow(f[(size_t)(j0 + q) * up + i]);
                acc = fmaf(v, v, acc);
            }
    } else {
        const int j = blockIdx.y * 8 + threadIdx.y + 1, k0 = bz * RES3_PLANES + 1;
        const size_t pl = (size_t)up * (n + 2);
        if (i <= n && j <= n)
            for (int q = 0; q < RES3_PLANES && k0 + q <= n; q++) {
                const float v = narrow(f[(k0 + q) * pl + (size_t)j * up + i]);
                acc = fmaf(v, v, acc);
            }
    }
    const double s = block_sum_f(acc, sh);
    if (threadIdx.x == 0 && threadIdx.y == 0)
        part[blockIdx.x + gridDim.x * (blockIdx.y + (size_t)gridDim.y * bz)] = s;
}

// (hi, lo) = the FP32 rounding of x and the FP32 rounding of the remainder
// x - hi, with no FP64-pipe instruction: the remainder is a whole number D of ulps of
// x (|D| <= 2^28; the difference of the two bit patterns, both in x's binade or
// hi at its upper end), converted to FP32 and scaled by that ulp, a power of
// two.  Below |x| ~ 2^-74 lo is 0.
__device__ __forceinline__ void split_f64(double x, float &hi, float &lo) {
    hi = narrow(x);
    // 32-bit integer operations only: D fits in 32 bits, so the low words give it
    const unsigned xh = (unsigned)__double2hiint(x), xl = (unsigned)__double2loint(x);
    const int D = (int)(xl - (unsigned)__double2loint(widen(hi)));
    const int fe = (int)((xh >> 20) & 0x7ffu) - 948;  // FP32 biased exponent of 2^(e - 1075), x's ulp
    const float l = fe > 0 ? i2f_rn(D) * __int_as_float(fe << 23) : 0.f;
    lo = (xh >> 31) ? -l : l;
}

// h^-2 (sum of the four neighbours - 4 centre), 2D, of decoded values; lg = log2(h^-2)
__device__ __forceinline__ double fx_lap5(const Fx &C, const Fx &W, const Fx &E, const Fx &S, const Fx &N, int lg) {
    const int em = max(max(max(C.e, W.e), max(E.e, S.e)), N.e);
    const long long t = (fx_al(W, em) + fx_al(E, em)) + (fx_al(S, em) + fx_al(N, em)) - (fx_al(C, em) << 2);
    return fx_to_double(t, em - 1081 + lg);
}
// h^-2 (sum of the six neighbours - 6 centre), 3D, of decoded values
__device__ __forceinline__ double fx_lap7(const Fx &C, const Fx &W, const Fx &E, const Fx &S, const Fx &N,
                                          const Fx &D, const Fx &U, int lg) {
    const int em = max(max(max(C.e, W.e), max(E.e, S.e)), max(max(N.e, D.e), U.e));
    const long long c6 = fx_al(C, em);
    const long long t = ((fx_al(W, em) + fx_al(E, em)) + (fx_al(S, em) + fx_al(N, em))) + (fx_al(D, em) + fx_al(U, em)) -
                        ((c6 << 2) + (c6 << 1));
    return fx_to_double(t, em - 1081 + lg);
}

// warps of a residual block (of 8) that evaluate the stencil in FP64 rather
// than with the integer Laplacian: both pipes then share the work
constexpr int RES_F64_WARPS = 3;

// OR of the magnitude bits of a double (zero iff +-0), in 32-bit operations
__device__ __forceinline__ unsigned mag_bits(double x) {
    return ((unsigned)__double2hiint(x) << 1) | (unsigned)__double2loint(x);
}

// Direct residual r = f - L u (Eq. Evpois) of the fused mixed path, the
// Laplacian in exact integer arithmetic (fx_lap5 / fx_lap7) and one FP64
// subtraction.
// START (start of a solve): r as the float-float pair hi (the level's buffer
// r) and lo (rlo, pitch rp), partial sums of hi^2 to part and of f^2 (FP32
// squares: the norm of the right-hand side) to fpart.  Where u and its four
// neighbours are all zero r = f, and a warp whose points all are skips the
// FP64 arithmetic (a solve from u = 0 then moves bytes only); zu (a solve
// from zero, mg_solve_zero): u is not read at all, r = f.  Otherwise (end of
// a solve): only the partial sums of r^2, nothing written.
template <bool START>
__global__ void __launch_bounds__(256) k_res_rr_2d(const double *__restrict__ f, const double *__restrict__ u,
                                                   int up, int n, int lg, A2<float> r, float *rlo, int rp,
                                                   double *part, double *fpart, Ctrl *ctl, int zu, const int *done,
                                                   Bt B) {
    __shared__ double sh[32];
    __shared__ float shm[32];
    const int prob = blockIdx.z;
    if (stop(bt_done(done, prob, B))) return;
    if (B.ftab) { f = B.ftab[prob]; u = B.utab[prob]; }
    if (START) { r = bt_at(r, prob, B); rlo = bt_ptr(rlo, prob, B); }
    const int i = blockIdx.x * 32 + threadIdx.x + 1;
    const int j0 = (blockIdx.y * 8 + threadIdx.y) * RES_ROWS + 1;
    float acc = 0.f, facc = 0.f, mx = 0.f;
    if (i <= n && j0 <= n) {
        const double *u0p = u + (size_t)j0 * up + i;
        const double *f0p = f + (size_t)j0 * up + i;
        const int rows = min(RES_ROWS, n + 1 - j0);
        // f of the thread's rows, loaded ahead of the test of u
        double fr[RES_ROWS];
#pragma unroll
        for (int q = 0; q < RES_ROWS; q++) fr[q] = q < rows ? f0p[(size_t)q * up] : 0.0;
        bool zero = START && zu;
        if (START && !zu) {  // u zero on the thread's column (rows j0-1 .. j0+rows)?
            unsigned ob = mag_bits(u0p[-up]) | mag_bits(u0p[(size_t)rows * up]);
#pragma unroll
            for (int q = 0; q < RES_ROWS; q++)
                if (q < rows) ob |= mag_bits(u0p[(size_t)q * up]);
            // the x neighbours are the adjacent lanes' columns; the first and
            // the last active lane also test the column beyond them
            const unsigned act = __activemask();
            const bool first = (int)threadIdx.x == __ffs(act) - 1, last = (int)threadIdx.x == 31 - __clz(act);
            if (first || last) {
                const int dx = first ? -1 : 1;
#pragma unroll
                for (int q = 0; q < RES_ROWS; q++) {
                    if (q >= rows) break;
                    ob |= mag_bits(u0p[(size_t)q * up + dx]);
                    if (first && last) ob |= mag_bits(u0p[(size_t)q * up + 1]);
                }
            }
            zero = ob == 0;  // with __all_sync below: every neighbour of every point of the warp
        }
        // warp-uniform: either no FP64 arithmetic at all (separate loops, so
        // that the stencil is branched over rather than predicated) or the
        // full stencil, in integer arithmetic (fx_lap5) in most warps and in
        // FP64 in the last RES_F64_WARPS of the block, so that the FP64 pipe
        // works beside the integer ones
        auto rows_loop = [&](auto mode_tag) {
            constexpr int MODE = decltype(mode_tag)::value;  // 0 u = 0, 1 integer, 2 FP64
            constexpr bool Z = MODE == 0;
            const double *uc = u0p;
            // the column's u stays decoded (or loaded) from row to row (rows j-1, j)
            Fx um = fx_dec(MODE == 1 ? uc[-up] : 0.0), u0 = fx_dec(MODE == 1 ? uc[0] : 0.0), upn{0, 0};
            double dm = MODE == 2 ? uc[-up] : 0.0, d0 = MODE == 2 ? uc[0] : 0.0, dp = 0.0;
            const double ih2 = __longlong_as_double((long long)(1023 + lg) << 52);  // 2^lg
#pragma unroll
            for (int q = 0; q < RES_ROWS; q++) {
                if (q >= rows) break;
                const double fv = fr[q];
                double res = fv;
                if (MODE == 1) {
                    upn = fx_dec(uc[up]);
                    res = fv - fx_lap5(u0, fx_dec(uc[-1]), fx_dec(uc[1]), um, upn, lg);
                } else if (MODE == 2) {
                    dp = uc[up];
                    res = fma(-ih2, fma(-4.0, d0, (uc[-1] + uc[1]) + (dm + dp)), fv);
                }
                float hi;
                if (START) {
                    float lo;
                    split_f64(res, hi, lo);
                    r(i, j0 + q) = hi;
                    rlo[(size_t)(j0 + q) * rp + i] = lo;
                    const float ff = Z ? hi : narrow(fv);
                    facc = fmaf(ff, ff, facc);
                    mx = fmaxf(mx, fabsf(hi));
                } else {
                    hi = narrow(res);
                }
                acc = fmaf(hi, hi, acc);
                um = u0; u0 = upn;
                dm = d0; d0 = dp;
                uc += up;
            }
        };
        if (__all_sync(__activemask(), zero)) rows_loop(std::integral_constant<int, 0>{});
        else if ((int)threadIdx.y < 8 - RES_F64_WARPS) rows_loop(std::integral_constant<int, 1>{});
        else rows_loop(std::integral_constant<int, 2>{});
    }
    const size_t slot = (size_t)prob * B.nparts + blockIdx.x + gridDim.x * blockIdx.y;
    const double s = block_sum_f(acc, sh);
    if (threadIdx.x == 0 && threadIdx.y == 0) part[slot] = s;
    if (START) {
        __syncthreads();
        const double sf = block_sum_f(facc, sh);
        const float m = block_max(mx, shm);
        if (threadIdx.x == 0 && threadIdx.y == 0) {
            fpart[slot] = sf;
            atomicMax(&ctl[prob].rmax[0], __float_as_uint(m));  // the start writes buffer 0
        }
    }
}

}  // namespace mg

namespace mg {

}  // namespace mg

namespace mg {

// ---------------------------------------------------------------------------
// 3D finest triple, green-red sweep (Eq. Egprolg then Eq. Egprolr) in one tile
// of 32 x 8 x 4 green points.  The red level is staged as its four cosets
// (coalesced loads of dense arrays), the F (odd) points are computed on the
// tile +- 2, the C (even) points on the tile +- 1.  FINEST: u += v,
// otherwise v stored.  (FP32 triples from 31^3 up use the z-streaming
// k_green_ff_3d.)
// ---------------------------------------------------------------------------
constexpr int TX3 = 32, TY3 = 8, TZ3 = 4;
constexpr int CX3 = TX3 / 2 + 3, CY3 = TY3 / 2 + 3, CZ3 = TZ3 / 2 + 3;  // coset cells of the tile +- 3
constexpr int WX3 = TX3 + 4, WY3 = TY3 + 4, WZ3 = TZ3 + 4;              // fine region of the tile +- 2

template <typename T> struct Green3Smem {
    T red[4][CZ3][CY3][CX3];  // EEE, OOE, OEO, EOO
    T v[WZ3][WY3][WX3];       // F at odd points (tile +- 2), C at even points (tile +- 1)
    T r[WZ3][WY3][WX3];       // green residual
};

template <typename T, bool FINEST>
__global__ void __launch_bounds__(256) k_green_3d(Red3<const T> vr, A3<const T> rg, A3<T> vg, double *__restrict__ u,
                                                  int up, int n, T cg, const int *done, Bt B) {
    extern __shared__ __align__(16) unsigned char smraw[];
    Green3Smem<T> &S = *reinterpret_cast<Green3Smem<T> *>(smraw);
    const int prob = bt_prob(B), bz = bt_z(B);
    if (stop(bt_done(done, prob, B))) return;
    vr = bt_at(vr, prob, B);
    rg = bt_at(rg, prob, B);
    vg = bt_at(vg, prob, B);
    if (B.utab) u = B.utab[prob];
    const int tid = threadIdx.x + 32 * threadIdx.y;
    const int x0 = blockIdx.x * TX3 + 1, y0 = blockIdx.y * TY3 + 1, z0 = bz * TZ3 + 1;
    const int ca = (x0 - 3) >> 1, cb = (y0 - 3) >> 1, cc = (z0 - 3) >> 1;  // first coset cell
    // the four red cosets over the tile +- 3 (a coset point outside the interior reads 0)
    const A3<const T> *cos[4] = {&vr.eee, &vr.ooe, &vr.oeo, &vr.eoo};
    const int px[4] = {0, 1, 1, 0}, py[4] = {0, 1, 0, 1}, pz[4] = {0, 0, 1, 1};
#pragma unroll
    for (int s = 0; s < 4; s++) {
        for (int q = tid; q < CX3 * CY3 * CZ3; q += 256) {
            const int lx = q % CX3, ly = (q / CX3) % CY3, lz = q / (CX3 * CY3);
            const int a = ca + lx, b = cb + ly, c = cc + lz;
            const int x = 2 * a + px[s], y = 2 * b + py[s], z = 2 * c + pz[s];
            S.red[s][lz][ly][lx] = (x >= 1 && x <= n && y >= 1 && y <= n && z >= 1 && z <= n) ? (*cos[s])(a, b, c) : T(0);
        }
    }
    for (int q = tid; q < WX3 * WY3 * WZ3; q += 256) {
        const int lx = q % WX3, ly = (q / WX3) % WY3, lz = q / (WX3 * WY3);
        const int x = x0 - 2 + lx, y = y0 - 2 + ly, z = z0 - 2 + lz;
        S.r[lz][ly][lx] = (x >= 1 && x <= n && y >= 1 && y <= n && z >= 1 && z <= n) ? rg(x, y, z) : T(0);
    }
    __syncthreads();
    // red value at fine (x, y, z), x + y + z even, within the tile +- 3
    auto red = [&](int x, int y, int z) -> T {
        const int s = (x & 1) ? ((y & 1) ? 1 : 2) : ((y & 1) ? 3 : 0);
        return S.red[s][(z >> 1) - cc][(y >> 1) - cb][(x >> 1) - ca];
    };
    // F points (odd index sum) on the tile +- 2: per row the WX3/2 points of that parity
    for (int q = tid; q < (WX3 / 2) * WY3 * WZ3; q += 256) {
        const int hx = q % (WX3 / 2), ly = (q / (WX3 / 2)) % WY3, lz = q / ((WX3 / 2) * WY3);
        const int y = y0 - 2 + ly, z = z0 - 2 + lz;
        const int xs = x0 - 2, p = (y + z + 1) & 1;          // x parity of the odd points of this row
        const int lx = 2 * hx + ((p - xs) & 1), x = xs + lx;
        T val = T(0);
        if (x >= 1 && x <= n && y >= 1 && y <= n && z >= 1 && z <= n) {
            const T s = (red(x - 1, y, z) + red(x + 1, y, z)) + (red(x, y - 1, z) + red(x, y + 1, z)) +
                        (red(x, y, z - 1) + red(x, y, z + 1));
            val = (s - cg * S.r[lz][ly][lx]) * T(1.0 / 6.0);
        }
        S.v[lz][ly][lx] = val;
    }
    __syncthreads();
    // C points (even index sum) on the tile +- 1
    for (int q = tid; q < ((WX3 - 2) / 2) * (WY3 - 2) * (WZ3 - 2); q += 256) {
        const int hx = q % ((WX3 - 2) / 2), my = (q / ((WX3 - 2) / 2)) % (WY3 - 2), mz = q / (((WX3 - 2) / 2) * (WY3 - 2));
        const int ly = my + 1, lz = mz + 1;
        const int y = y0 - 2 + ly, z = z0 - 2 + lz;
        const int xs = x0 - 1, p = (y + z) & 1;               // x parity of the even points of this row
        const int lx = 1 + 2 * hx + ((p - xs) & 1), x = x0 - 2 + lx;
        T val = T(0);
        if (x >= 1 && x <= n && y >= 1 && y <= n && z >= 1 && z <= n) {
            const T s = (S.v[lz][ly][lx - 1] + S.v[lz][ly][lx + 1]) + (S.v[lz][ly - 1][lx] + S.v[lz][ly + 1][lx]) +
                        (S.v[lz - 1][ly][lx] + S.v[lz + 1][ly][lx]);
            val = (s - cg * S.r[lz][ly][lx]) * T(1.0 / 6.0);
        }
        S.v[lz][ly][lx] = val;
    }
    __syncthreads();
    for (int q = tid; q < TX3 * TY3 * TZ3; q += 256) {
        const int tx = q % TX3, ty = (q / TX3) % TY3, tz = q / (TX3 * TY3);
        const int x = x0 + tx, y = y0 + ty, z = z0 + tz;
        if (x > n || y > n || z > n) continue;
        const T v = S.v[tz + 2][ty + 2][tx + 2];
        if (FINEST) u[((size_t)z * (n + 2) + y) * up + x] += widen(v);
        else vg(x, y, z) = v;
    }
}

// 3D direct residual of the fused mixed path (7-point), as k_res_rr_2d:
// RES3_PLANES planes per thread marching in z
template <bool START>
__global__ void __launch_bounds__(256) k_res_rr_3d(const double *__restrict__ f, const double *__restrict__ u,
                                                   int up, int n, int lg, A3<float> r, float *rlo, int rp,
                                                   double *part, double *fpart, Ctrl *ctl, int zu, const int *done,
                                                   Bt B) {
    __shared__ double sh[32];
    __shared__ float shm[32];
    const int prob = bt_prob(B), bz = bt_z(B);
    if (stop(bt_done(done, prob, B))) return;
    if (B.ftab) { f = B.ftab[prob]; u = B.utab[prob]; }
    if (START) { r = bt_at(r, prob, B); rlo = bt_ptr(rlo, prob, B); }
    const int i = blockIdx.x * 32 + threadIdx.x + 1, j = blockIdx.y * 8 + threadIdx.y + 1;
    const int k0 = bz * RES3_PLANES + 1;
    const size_t pl = (size_t)up * (n + 2), pr = (size_t)rp * (n + 2);
    float acc = 0.f, facc = 0.f, mx = 0.f;
    const bool act = i <= n && j <= n;
    const int planes = act ? min(RES3_PLANES, n + 1 - k0) : 0;
    const double *u0p = u + k0 * pl + (size_t)(act ? j : 1) * up + (act ? i : 1);
    const double *f0p = f + k0 * pl + (size_t)(act ? j : 1) * up + (act ? i : 1);
    // u zero around every point of the block? (START only; block-uniform;
    // zu: a solve from zero, u not read)
    bool all_zero = START && zu;
    if (START && !zu) {
        unsigned ob = 0;
        if (act && planes > 0) {
            // the thread's column (planes k0-1 .. k0+planes); x and y neighbours
            // are other threads' columns, the block's edge threads test the
            // columns beyond the block
            ob = mag_bits(u0p[-(long)pl]) | mag_bits(u0p[(size_t)planes * pl]);
            const bool xl = threadIdx.x == 0, xr = threadIdx.x == 31 || i == n;
            const bool yl = threadIdx.y == 0, yr = threadIdx.y == 7 || j == n;
#pragma unroll
            for (int q = 0; q < RES3_PLANES; q++) {
                if (q >= planes) break;
                const double *c = u0p + (size_t)q * pl;
                ob |= mag_bits(c[0]);
                if (xl) ob |= mag_bits(c[-1]);
                if (xr) ob |= mag_bits(c[1]);
                if (yl) ob |= mag_bits(c[-up]);
                if (yr) ob |= mag_bits(c[up]);
            }
        }
        all_zero = __syncthreads_and(ob == 0) != 0;
    }
    if (act && planes > 0) {
        double fr[RES3_PLANES];
#pragma unroll
        for (int q = 0; q < RES3_PLANES; q++) fr[q] = q < planes ? f0p[(size_t)q * pl] : 0.0;
        // as in k_res_rr_2d: no arithmetic where u is 0, else the integer
        // Laplacian, or FP64 in the last RES_F64_WARPS warps of the block
        auto planes_loop = [&](auto mode_tag) {
            constexpr int MODE = decltype(mode_tag)::value;  // 0 u = 0, 1 integer, 2 FP64
            constexpr bool Z = MODE == 0;
            const double *uc = u0p;
            // the column's u stays decoded (or loaded) from plane to plane (planes k-1, k)
            Fx ud = fx_dec(MODE == 1 ? uc[-(long)pl] : 0.0), u0 = fx_dec(MODE == 1 ? uc[0] : 0.0), uu{0, 0};
            double dd = MODE == 2 ? uc[-(long)pl] : 0.0, d0 = MODE == 2 ? uc[0] : 0.0, du = 0.0;
            const double ih2 = __longlong_as_double((long long)(1023 + lg) << 52);  // 2^lg
#pragma unroll
            for (int q = 0; q < RES3_PLANES; q++) {
                if (q >= planes) break;
                const double fv = fr[q];
                double res = fv;
                if (MODE == 1) {
                    uu = fx_dec(uc[pl]);
                    res = fv - fx_lap7(u0, fx_dec(uc[-1]), fx_dec(uc[1]), fx_dec(uc[-up]), fx_dec(uc[up]), ud, uu, lg);
                } else if (MODE == 2) {
                    du = uc[pl];
                    res = fma(-ih2, fma(-6.0, d0, ((uc[-1] + uc[1]) + (uc[-up] + uc[up])) + (dd + du)), fv);
                }
                float hi;
                if (START) {
                    float lo;
                    split_f64(res, hi, lo);
                    r(i, j, k0 + q) = hi;
                    rlo[(k0 + q) * pr + (size_t)j * rp + i] = lo;
                    const float ff = Z ? hi : narrow(fv);
                    facc = fmaf(ff, ff, facc);
                    mx = fmaxf(mx, fabsf(hi));
                } else {
                    hi = narrow(res);
                }
                acc = fmaf(hi, hi, acc);
                ud = u0; u0 = uu;
                dd = d0; d0 = du;
                uc += pl;
            }
        };
        if (all_zero) planes_loop(std::integral_constant<int, 0>{});
        else if ((int)threadIdx.y < 8 - RES_F64_WARPS) planes_loop(std::integral_constant<int, 1>{});
        else planes_loop(std::integral_constant<int, 2>{});
    }
    const size_t slot = (size_t)prob * B.nparts + blockIdx.x + gridDim.x * (blockIdx.y + (size_t)gridDim.y * bz);
    const double s = block_sum_f(acc, sh);
    if (threadIdx.x == 0 && threadIdx.y == 0) part[slot] = s;
    if (START) {
        __syncthreads();
        const double sf = block_sum_f(facc, sh);
        const float m = block_max(mx, shm);
        if (threadIdx.x == 0 && threadIdx.y == 0) {
            fpart[slot] = sf;
            atomicMax(&ctl[prob].rmax[0], __float_as_uint(m));  // the start writes buffer 0
        }
    }
}

}  // namespace mg
