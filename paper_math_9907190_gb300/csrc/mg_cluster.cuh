// mg_cluster.cuh -- the coarse part of a 2D diagonal V-cycle in one thread-
// block cluster: the middle pairs in distributed shared memory, the smallest
// pairs and the coarsest solve in the cluster's first block (Section 2).
//
// A cluster of CL2 blocks of 1024 threads holds every level of the pairs
// kd..kc-1 in shared memory, each level split by rows: for a pair whose green
// grid has side n (n + 1 = 8 R), block q owns the green rows [qR, (q+1)R) and
// the coset rows [qR/2, (q+1)R/2) of its red level (coset row b holds the
// green rows 2b and 2b+1), so the blue level of the pair -- the next pair's
// green grid -- is split the same way with R/2.  Every stencil of the paper
// reaches one row up or down on its own level, so a block keeps one halo row
// on each side of its band: whoever computes a boundary row also writes it
// into the neighbour's halo row (a store to the neighbour's shared memory),
// and the cluster barrier that ends the pass makes it visible.  All reads are
// then local.  The smallest pairs (green side <= 31) are gathered into block
// 0, which runs them and the coarsest solve with cta_pairs_2d, and scatters
// the correction back.  The cluster barrier is the hardware barrier
// (barrier.cluster): no block spins on memory.
//
// The arithmetic of every value is the one of cta_pairs_2d and of the pair
// kernels, term for term.
#pragma once
#include <cooperative_groups.h>

#include "mg_fast2d.cuh"

namespace mg {

namespace cgx = cooperative_groups;

constexpr int CL2 = 8;      // blocks per cluster
constexpr int CL_MAX = 6;   // distributed pairs at most

// one level array split by rows over the cluster: element (x, y) of block q
// lies at off + (y - q R + 1) * pitch + x of that block's shared memory (the
// same offset in every block); local rows 0 and R + 1 are the halo rows
struct DistArr {
    int off, pitch, R;
};

struct ClPlan2d {
    int nd;                       // distributed pairs
    int nk[CL_MAX + 1];           // green side of distributed pair i; nk[nd]: the first pair of block 0
    DistArr gr[CL_MAX + 1], gv[CL_MAX + 1];  // green r / v (index nd: block 0's first pair, gathered)
    DistArr er[CL_MAX], orr[CL_MAX], ev[CL_MAX], ov[CL_MAX];  // red EE / OO, r and v
    double c2[CL_MAX], c1[CL_MAX];  // 2 p h_k^2 (red), p h_k^2 (green)
    int doff;                     // elements of the distributed arrays (block 0's plan follows, 16-byte aligned)
    CoarsePlan2d cta;             // pairs of block 0, offsets relative to sm + doff
};

__device__ __forceinline__ void cluster_barrier() {
    asm volatile("barrier.cluster.arrive.release.aligned;\nbarrier.cluster.wait.acquire.aligned;\n" ::: "memory");
}

// Shared-memory access of one block to the distributed arrays.
template <typename T> struct ClMem {
    T *sm;
    int q;
    // row y of A in this block (y within its band or one of the two halo rows)
    __device__ __forceinline__ T *row(const DistArr &A, int y) const { return sm + A.off + (y - q * A.R + 1) * A.pitch; }
    // the copies of row y (owned by block r) that other blocks keep as halo
    // rows: lo in block r - 1 (y is r's first row), hi in block r + 1 (its
    // last row); null when there is none
    __device__ __forceinline__ void halos(const DistArr &A, int y, int r, T *&lo, T *&hi) const {
        const int ly = y - r * A.R + 1;
        lo = (ly == 1 && r > 0) ? cgx::this_cluster().map_shared_rank(sm + A.off + (A.R + 1) * A.pitch, r - 1) : nullptr;
        hi = (ly == A.R && r < CL2 - 1) ? cgx::this_cluster().map_shared_rank(sm + A.off, r + 1) : nullptr;
    }
};

// Thread layout of a pass over `rows` rows: ny thread rows (a power of two up
// to 32, at least the row count when it is smaller) and 1024 / ny threads
// along a row.
struct ClLay {
    int ny, nx, ty, tx;
    __device__ __forceinline__ ClLay(int rows) {
        ny = 32;
        while (ny > 1 && ny / 2 >= rows) ny >>= 1;
        nx = 1024 / ny;
        ty = threadIdx.x / nx;
        tx = threadIdx.x - ty * nx;
    }
};

template <typename T>
__global__ void __cluster_dims__(CL2, 1, 1) __launch_bounds__(1024)
    k_coarse_cl_2d(ClPlan2d P, A2<const T> rg_in, A2<T> vg_out, const double *G, const int *done, Bt B) {
    extern __shared__ __align__(16) unsigned char smraw[];
    T *sm = reinterpret_cast<T *>(smraw);
    const int prob = blockIdx.z;
    if (stop(bt_done(done, prob, B))) return;  // every block of the cluster reads the same flag
    rg_in = bt_at(rg_in, prob, B);
    vg_out = bt_at(vg_out, prob, B);
    const int q = (int)cgx::this_cluster().block_rank();
    const int tid = threadIdx.x, tx = tid & 31, ty = tid >> 5;
    const ClMem<T> M{sm, q};
    T *smc = sm + P.doff;  // block 0's pairs
    double *Gs = reinterpret_cast<double *>(reinterpret_cast<unsigned char *>(smc) + P.cta.gofs);
    GPrefetch<1024> gp;
    if (q == 0) gp.load(G, P.cta.ng, tid);
    const int ztot = q == 0 ? P.doff + P.cta.total : P.doff;
    for (int e = tid; e < ztot; e += 1024) sm[e] = T(0);
    __syncthreads();
    {   // the green residual of the first distributed pair: owned rows and halo rows
        const int n = P.nk[0];
        const DistArr &A = P.gr[0];
        const int y0 = max(q * A.R - 1, 1), y1 = min((q + 1) * A.R, n);
        for (int y = y0 + ty; y <= y1; y += 32) {
            T *d = M.row(A, y);
            for (int x = 1 + tx; x <= n; x += 32) d[x] = rg_in(x, y);
        }
    }
    if (q == 0) gp.store(Gs, P.cta.ng, tid);
    cluster_barrier();  // every block's shared memory is initialised before any store into it
    for (int p = 0; p < P.nd; p++) {
        const int n = P.nk[p], nb = (n - 1) / 2, R = P.gr[p].R, Rc = R / 2;
        const DistArr &g = P.gr[p], &ee = P.er[p], &oo = P.orr[p], &bl = P.gr[p + 1];
        const int b0 = q * Rc, b1 = min((q + 1) * Rc - 1, nb);
        {   // Eq. Erest2r: OO at green (2a+1, 2b+1), EE at (2a, 2b)
            const ClLay L(b1 - b0 + 1);
            for (int b = b0 + L.ty; b <= b1; b += L.ny) {
                const T *gm = M.row(g, 2 * b - 1), *g0 = M.row(g, 2 * b), *g1 = M.row(g, 2 * b + 1), *g2 = M.row(g, 2 * b + 2);
                T *po = M.row(oo, b), *pe = M.row(ee, b), *ol, *oh, *el, *eh;
                M.halos(oo, b, q, ol, oh);
                M.halos(ee, b, q, el, eh);
                for (int a = L.tx; a <= nb; a += L.nx) {
                    int i = 2 * a + 1;
                    const T vo = (T(4) * g1[i] + (g1[i - 1] + g1[i + 1]) + (g0[i] + g2[i])) * T(0.125);
                    po[a] = vo;
                    if (ol) ol[a] = vo;
                    if (oh) oh[a] = vo;
                    if (a >= 1 && b >= 1) {
                        i = 2 * a;
                        const T ve = (T(4) * g0[i] + (g0[i - 1] + g0[i + 1]) + (gm[i] + g1[i])) * T(0.125);
                        pe[a] = ve;
                        if (el) el[a] = ve;
                        if (eh) eh[a] = ve;
                    }
                }
            }
        }
        cluster_barrier();
        {   // Eq. Erest2b: blue (a, b) from EE (a, b) and the four OO around it
            const int c0 = max(b0, 1);
            const ClLay L(b1 - c0 + 1);
            for (int b = c0 + L.ty; b <= b1; b += L.ny) {
                const T *e0 = M.row(ee, b), *om = M.row(oo, b - 1), *o0 = M.row(oo, b);
                T *pb = M.row(bl, b), *lo, *hi;
                M.halos(bl, b, q, lo, hi);
                for (int a = 1 + L.tx; a <= nb; a += L.nx) {
                    const T v = (T(4) * e0[a] + (om[a - 1] + om[a]) + (o0[a - 1] + o0[a])) * T(0.125);
                    pb[a] = v;
                    if (lo) lo[a] = v;
                    if (hi) hi[a] = v;
                }
            }
        }
        cluster_barrier();
    }
    if (q == 0) {  // block 0: gather its first pair's residual, run its pairs, scatter the correction
        const int n = P.nk[P.nd];
        const DistArr &A = P.gr[P.nd], &V = P.gv[P.nd];
        A2<T> g{smc + P.cta.og_r[0], n + 2};
        for (int y = 1 + ty; y <= n; y += 32) {
            const int r = y / A.R;
            const T *src = cgx::this_cluster().map_shared_rank(sm + A.off + (y - r * A.R + 1) * A.pitch, r);
            for (int x = 1 + tx; x <= n; x += 32) g(x, y) = src[x];
        }
        __syncthreads();
        cta_pairs_2d<T>(P.cta, smc, Gs);
        A2<T> v{smc + P.cta.og_v[0], n + 2};
        for (int y = 1 + ty; y <= n; y += 32) {
            const int r = y / V.R;
            T *dst = cgx::this_cluster().map_shared_rank(sm + V.off + (y - r * V.R + 1) * V.pitch, r), *lo, *hi;
            M.halos(V, y, r, lo, hi);
            for (int x = 1 + tx; x <= n; x += 32) {
                const T val = v(x, y);
                dst[x] = val;
                if (lo) lo[x] = val;
                if (hi) hi[x] = val;
            }
        }
    }
    cluster_barrier();
    for (int p = P.nd - 1; p >= 0; p--) {
        const int n = P.nk[p], nb = (n - 1) / 2, R = P.gr[p].R, Rc = R / 2;
        const DistArr &rgr = P.gr[p], &vgr = P.gv[p], &ree = P.er[p], &roo = P.orr[p], &vee = P.ev[p], &voo = P.ov[p];
        const DistArr &vbl = P.gv[p + 1];
        const T c2 = (T)P.c2[p], c1 = (T)P.c1[p];
        const int b0 = q * Rc, b1 = min((q + 1) * Rc - 1, nb);
        {   // Eq. Eajacr: OO from the four blue values around it
            const ClLay L(b1 - b0 + 1);
            for (int b = b0 + L.ty; b <= b1; b += L.ny) {
                const T *v0 = M.row(vbl, b), *v1 = M.row(vbl, b + 1), *r0 = M.row(roo, b);
                T *po = M.row(voo, b), *lo, *hi;
                M.halos(voo, b, q, lo, hi);
                for (int a = L.tx; a <= nb; a += L.nx) {
                    const T v = ((v0[a] + v0[a + 1]) + (v1[a] + v1[a + 1]) - c2 * r0[a]) * T(0.25);
                    po[a] = v;
                    if (lo) lo[a] = v;
                    if (hi) hi[a] = v;
                }
            }
        }
        cluster_barrier();
        {   // Eq. Eajacb: EE from the four new OO around it
            const int c0 = max(b0, 1);
            const ClLay L(b1 - c0 + 1);
            for (int b = c0 + L.ty; b <= b1; b += L.ny) {
                const T *om = M.row(voo, b - 1), *o0 = M.row(voo, b), *r0 = M.row(ree, b);
                T *pe = M.row(vee, b), *lo, *hi;
                M.halos(vee, b, q, lo, hi);
                for (int a = 1 + L.tx; a <= nb; a += L.nx) {
                    const T v = ((om[a - 1] + om[a]) + (o0[a - 1] + o0[a]) - c2 * r0[a]) * T(0.25);
                    pe[a] = v;
                    if (lo) lo[a] = v;
                    if (hi) hi[a] = v;
                }
            }
        }
        cluster_barrier();
        const int j0 = max(q * R, 1), j1 = min((q + 1) * R - 1, n);
        const ClLay L(j1 - j0 + 1);
        for (int j = j0 + L.ty; j <= j1; j += L.ny) {  // green-only points: i + j odd
            // red neighbours: same row (x +- 1) and rows j +- 1 (x); on an odd
            // row the OO cosets of rows j, j +- 1 hold them at odd x, EE at even x
            const int c = j >> 1;
            const T *oo_m = M.row(voo, (j - 1) >> 1), *oo_0 = M.row(voo, c), *oo_p = M.row(voo, (j + 1) >> 1);
            const T *ee_m = M.row(vee, (j - 1) >> 1), *ee_0 = M.row(vee, c), *ee_p = M.row(vee, (j + 1) >> 1);
            const T *rr = M.row(rgr, j);
            T *pv = M.row(vgr, j), *lo, *hi;
            M.halos(vgr, j, q, lo, hi);
            auto red = [&](int x, const T *o, const T *e) { return (x & 1) ? o[x >> 1] : e[x >> 1]; };
            for (int i = 1 + (j & 1) + 2 * L.tx; i <= n; i += 2 * L.nx) {
                const T v = ((red(i - 1, oo_0, ee_0) + red(i + 1, oo_0, ee_0)) + (red(i, oo_m, ee_m) + red(i, oo_p, ee_p)) -
                             c1 * rr[i]) * T(0.25);
                pv[i] = v;
                if (lo) lo[i] = v;
                if (hi) hi[i] = v;
            }
        }
        cluster_barrier();
        for (int j = j0 + L.ty; j <= j1; j += L.ny) {  // red points: i + j even
            const T *vm = M.row(vgr, j - 1), *vp = M.row(vgr, j + 1), *rr = M.row(rgr, j);
            T *pv = M.row(vgr, j), *lo, *hi;
            M.halos(vgr, j, q, lo, hi);
            for (int i = 2 - (j & 1) + 2 * L.tx; i <= n; i += 2 * L.nx) {
                const T v = ((pv[i - 1] + pv[i + 1]) + (vm[i] + vp[i]) - c1 * rr[i]) * T(0.25);
                pv[i] = v;
                if (lo) lo[i] = v;
                if (hi) hi[i] = v;
            }
        }
        cluster_barrier();
    }
    {   // the green correction of the first distributed pair, owned rows
        const int n = P.nk[0];
        const DistArr &A = P.gv[0];
        const int y0 = max(q * A.R, 1), y1 = min((q + 1) * A.R - 1, n);
        for (int y = y0 + ty; y <= y1; y += 32) {
            const T *s = M.row(A, y);
            for (int x = 1 + tx; x <= n; x += 32) vg_out(x, y) = s[x];
        }
    }
}

}  // namespace mg
