// mg_stages.cuh -- per-stage CUDA kernels of the diagonally oriented multigrid
// V-cycle (A.J. Roberts, "Fast and accurate multigrid solution of Poisson's
// equation using diagonally oriented grids") and of the conventional cycle.
//
// Storage (device, owned by the context):
//   * An axis level (green grid, conventional level, coarsest grid) of side s
//     is one array of (s+2) rows (x fastest) incl. the zero Dirichlet ring.
//   * A diagonal level of the pair/triple whose green grid has side n = 2nb+1
//     is split into cosets of that green grid by index parity, each a dense
//     axis-aligned array of (nb+2) entries per axis: an even green index 2a
//     maps to coset index a (a = 0 and nb+1 are the ring), an odd index 2c+1
//     maps to c (0..nb).  2D red (i+j even) = cosets EE, OO; 3D red (i+j+k
//     even) = EEE, OOE, OEO, EOO; 3D magenta = EEE (corners), OOO (centres).
//     With this split every stencil of the paper reads unit-stride
//     neighbours of a coset array, and no lattice hole is stored.
//   * Rings and coset entries outside the lattice are zero and never written.
//
// Each kernel computes one stage (a restriction, or one half of a red-black
// sweep) with one thread per output point.  `done` (nullable) is the device
// convergence flag of the solver: when set every kernel returns at once.
#pragma once
#include <cstddef>
#include <cstdint>
#include <cuda_runtime.h>
#include <type_traits>

namespace mg {

template <typename T> struct A2 {  // 2D array view
    T *p;
    int pitch;
    __device__ __forceinline__ T &operator()(int i, int j) const { return p[(size_t)j * pitch + i]; }
};
template <typename T> struct A3 {  // 3D array view
    T *p;
    int pitch, rows;
    __device__ __forceinline__ T &operator()(int i, int j, int k) const {
        return p[((size_t)k * rows + j) * pitch + i];
    }
};

// Kernels may be launched with programmatic dependent launch: a kernel may
// start while the previous one in the stream finishes, and waits here (before
// its first access to memory that another kernel reads or writes) for it to
// complete.  Once every block of this kernel has passed the wait, the next
// kernel may be scheduled onto the free SM slots, where its blocks wait in
// turn; so the launch of one kernel overlaps the tail of the one before.  A
// kernel launched without that attribute passes at once.
__device__ __forceinline__ void pdl_wait() {
    asm volatile("griddepcontrol.wait;\n" ::: "memory");
    asm volatile("griddepcontrol.launch_dependents;\n" ::: "memory");
}
__device__ __forceinline__ bool stop(const int *done) {
    pdl_wait();
    return done != nullptr && *(volatile const int *)done;
}

// Batch descriptor: a context holds `nprob` problems of one size.  Every level
// array of problem p lies `p * pstride` bytes after problem 0's; grid z holds
// `zper` blocks per problem; f/u come from device pointer tables (nullptr for
// a single problem: the kernel's own f/u are used); problem p's control word
// starts `p * ctl_stride` ints after problem 0's, its partial sums `p * nparts`
// doubles after problem 0's.
struct Bt {
    size_t pstride;
    int zper;
    int ctl_stride;
    int nparts;
    const double *const *ftab;
    double *const *utab;
};
__device__ __forceinline__ int bt_prob(const Bt &B) { return blockIdx.z / B.zper; }
__device__ __forceinline__ int bt_z(const Bt &B) { return blockIdx.z % B.zper; }
template <typename T> __device__ __forceinline__ T *bt_ptr(T *q, int p, const Bt &B) {
    return reinterpret_cast<T *>(reinterpret_cast<char *>(const_cast<typename std::remove_const<T>::type *>(q)) +
                                 (size_t)p * B.pstride);
}
template <typename T> __device__ __forceinline__ A2<T> bt_at(A2<T> v, int p, const Bt &B) {
    v.p = bt_ptr(v.p, p, B);
    return v;
}
template <typename T> __device__ __forceinline__ A3<T> bt_at(A3<T> v, int p, const Bt &B) {
    v.p = bt_ptr(v.p, p, B);
    return v;
}
__device__ __forceinline__ const int *bt_done(const int *done, int p, const Bt &B) {
    return done ? done + (size_t)p * B.ctl_stride : nullptr;
}

// Solver control word, one per context (device memory)
struct Ctrl {
    double f2;      // ||r(u=0)||^2
    double r2;      // ||r||^2 of the current iterate
    double relres;  // sqrt(r2/f2)
    double rel0;    // relative residual of the warm start
    double rtol;
    int done;       // 1: stop every kernel of the remaining cycles
    int cycles;     // corrections applied
    int max_cycles;
    int status;     // 0 ok, -4 not converged, -5 diverged
    int par;        // which of the two FP32 finest residual buffers is current (fused update path)
    // fused mixed path: bounds that the finest sweep rounds its correction
    // against (bit patterns of non-negative floats, which order as unsigned)
    unsigned vmax;     // max |v| of the level the finest sweep starts from, this cycle
    unsigned rmax[2];  // max |hi| of each of the two finest residual buffers
    unsigned arrive;   // blocks of the fused finest kernel that finished this cycle
};

// maximum of v over the block (valid in thread 0); NaN is ignored
__device__ __forceinline__ float block_max(float v, float *sh) {
    const int tid = threadIdx.x + blockDim.x * (threadIdx.y + blockDim.y * threadIdx.z);
    const int nt = blockDim.x * blockDim.y * blockDim.z;
    for (int o = 16; o > 0; o >>= 1) v = fmaxf(v, __shfl_down_sync(0xffffffffu, v, o));
    if ((tid & 31) == 0) sh[tid >> 5] = v;
    __syncthreads();
    if (tid < 32) {
        v = tid < (nt + 31) / 32 ? sh[tid] : 0.f;
        for (int o = 16; o > 0; o >>= 1) v = fmaxf(v, __shfl_down_sync(0xffffffffu, v, o));
    }
    return v;
}

// f32 -> f64 widening with integer operations (the FP64 pipe is the scarce
// resource on this GPU).  Exact for normal numbers and zero; FP32 subnormals
// (|x| < 2^-126) map to signed zero.
__device__ __forceinline__ double widen(float x) {
    const unsigned b = __float_as_uint(x);
    const unsigned ax = b & 0x7fffffffu;
    unsigned hi = (ax >> 3) + 0x38000000u;
    hi = ax >= 0x00800000u ? hi : 0u;
    hi |= b & 0x80000000u;
    return __hiloint2double((int)hi, (int)(b << 29));
}
__device__ __forceinline__ double widen(double x) { return x; }

// f64 -> f32 rounded to nearest even with integer operations (on this GPU
// the conversion instruction runs on the FP64 pipe at a fraction of its
// rate).  Normal FP32 results and zero are formed here; FP64 zeros and
// subnormals round to a signed zero; the rest (FP32 subnormal or overflow
// range, inf, nan) falls back to the conversion instruction.
// the conversion instruction, out of line so that it is never executed
// speculatively on the common path
__device__ __noinline__ float narrow_rare(double x) { return __double2float_rn(x); }
__device__ __forceinline__ float narrow(double x) {
    const unsigned long long X = (unsigned long long)__double_as_longlong(x);
    const unsigned hi = (unsigned)(X >> 32), lo = (unsigned)X;
    const int e = (int)((hi >> 20) & 0x7ffu), fe = e - 896;  // FP32 biased exponent
    if (fe < 1 || fe > 254) return e == 0 ? __uint_as_float(hi & 0x80000000u) : narrow_rare(x);
    const unsigned m = ((hi & 0xfffffu) << 3) | (lo >> 29);  // top 23 mantissa bits
    const unsigned rem = lo & 0x1fffffffu;                   // the 29 dropped bits
    const unsigned r = (hi & 0x80000000u) | ((unsigned)fe << 23) | m;
    return __uint_as_float(r + ((rem > 0x10000000u || (rem == 0x10000000u && (m & 1u))) ? 1u : 0u));
}
// level value of an FP64 result: FP32 levels round with narrow()
template <typename T> __device__ __forceinline__ T lvl(double x);
template <> __device__ __forceinline__ float lvl<float>(double x) { return narrow(x); }
template <> __device__ __forceinline__ double lvl<double>(double x) { return x; }

// int -> f32 rounded to nearest for |d| < 2^33, with FP32 adds: the two halves
// are exact through the 1.5 * 2^23 offset, one FMA rounds their sum
__device__ __forceinline__ float i2f_rn(int d) {
    const float fh = __int_as_float(0x4B400000 + (d >> 11)) - 12582912.0f;
    const float fl = __int_as_float(0x4B400000 + (d & 0x7ff)) - 12582912.0f;
    return fmaf(fh, 2048.0f, fl);
}

#define MG_IDX2 \
    const int tx = blockIdx.x * blockDim.x + threadIdx.x; \
    const int ty = blockIdx.y * blockDim.y + threadIdx.y;
#define MG_IDX3 \
    MG_IDX2 const int tz = bt_z(B);

// ---------------------------------------------------------------------------
// 2D diagonal hierarchy (Section 2)
// ---------------------------------------------------------------------------

// value of a red level at green point (x,y), x+y even (EE or OO coset)
template <typename T> __device__ __forceinline__ T red2(const A2<T> &ee, const A2<T> &oo, int x, int y) {
    return (x & 1) ? oo(x >> 1, y >> 1) : ee(x >> 1, y >> 1);
}

// green -> red, Eq. Erest2r: r' = (4r + sum of the 4 axis neighbours)/8 at i+j even.
// Thread per coset cell (a,b) in [0,nb]^2: OO(a,b) always, EE(a,b) if interior.
template <typename T>
__global__ void k_g2r_2d(A2<const T> g, A2<T> ee, A2<T> oo, int nb, const int *done, Bt B) {
    const int prob_ = bt_prob(B);
    if (stop(bt_done(done, prob_, B))) return;
    g = bt_at(g, prob_, B);
    ee = bt_at(ee, prob_, B);
    oo = bt_at(oo, prob_, B);
    MG_IDX2 const int a = tx, b = ty;
    if (a > nb || b > nb) return;
    int i = 2 * a + 1, j = 2 * b + 1;
    oo(a, b) = (T(4) * g(i, j) + (g(i - 1, j) + g(i + 1, j)) + (g(i, j - 1) + g(i, j + 1))) * T(0.125);
    if (a >= 1 && b >= 1) {
        i = 2 * a; j = 2 * b;
        ee(a, b) = (T(4) * g(i, j) + (g(i - 1, j) + g(i + 1, j)) + (g(i, j - 1) + g(i, j + 1))) * T(0.125);
    }
}

// red -> blue, Eq. Erest2b: r' = (4r + sum of the 4 diagonal neighbours)/8 at (e,e)
template <typename T>
__global__ void k_r2b_2d(A2<const T> ee, A2<const T> oo, A2<T> blue, int nb, const int *done, Bt B) {
    const int prob_ = bt_prob(B);
    if (stop(bt_done(done, prob_, B))) return;
    ee = bt_at(ee, prob_, B);
    oo = bt_at(oo, prob_, B);
    blue = bt_at(blue, prob_, B);
    MG_IDX2 const int a = tx + 1, b = ty + 1;
    if (a > nb || b > nb) return;
    blue(a, b) = (T(4) * ee(a, b) + (oo(a - 1, b - 1) + oo(a, b - 1)) + (oo(a - 1, b) + oo(a, b))) * T(0.125);
}

// blue -> red, Eq. Eajacr: red points that are not blue (OO) from the four
// diagonal blue values; c = 2 p h^2 (red spacing sqrt(2) h).
template <typename T>
__global__ void k_b2r_oo_2d(A2<const T> blue, A2<const T> roo, A2<T> voo, int nb, T c, const int *done, Bt B) {
    const int prob_ = bt_prob(B);
    if (stop(bt_done(done, prob_, B))) return;
    blue = bt_at(blue, prob_, B);
    roo = bt_at(roo, prob_, B);
    voo = bt_at(voo, prob_, B);
    MG_IDX2 const int a = tx, b = ty;
    if (a > nb || b > nb) return;
    voo(a, b) = ((blue(a, b) + blue(a + 1, b)) + (blue(a, b + 1) + blue(a + 1, b + 1)) - c * roo(a, b)) * T(0.25);
}

// Eq. Eajacb: blue points (EE) refined from the four new diagonal red values
template <typename T>
__global__ void k_b2r_ee_2d(A2<const T> voo, A2<const T> ree, A2<T> vee, int nb, T c, const int *done, Bt B) {
    const int prob_ = bt_prob(B);
    if (stop(bt_done(done, prob_, B))) return;
    voo = bt_at(voo, prob_, B);
    ree = bt_at(ree, prob_, B);
    vee = bt_at(vee, prob_, B);
    MG_IDX2 const int a = tx + 1, b = ty + 1;
    if (a > nb || b > nb) return;
    vee(a, b) = ((voo(a - 1, b - 1) + voo(a, b - 1)) + (voo(a - 1, b) + voo(a, b)) - c * ree(a, b)) * T(0.25);
}

// red -> green, first half: green-only points (i+j odd) from the four axis
// red values; c = p h^2 (Section 2.2, weight of Section 2.4)
template <typename T>
__global__ void k_r2g_f_2d(A2<const T> ee, A2<const T> oo, A2<const T> rg, A2<T> vg, int n, T c,
                           const int *done, Bt B) {
    const int prob_ = bt_prob(B);
    if (stop(bt_done(done, prob_, B))) return;
    ee = bt_at(ee, prob_, B);
    oo = bt_at(oo, prob_, B);
    rg = bt_at(rg, prob_, B);
    vg = bt_at(vg, prob_, B);
    MG_IDX2 const int i = tx + 1, j = ty + 1;
    if (i > n || j > n || ((i + j) & 1) == 0) return;
    T s = (red2(ee, oo, i - 1, j) + red2(ee, oo, i + 1, j)) + (red2(ee, oo, i, j - 1) + red2(ee, oo, i, j + 1));
    vg(i, j) = (s - c * rg(i, j)) * T(0.25);
}

// red -> green, second half: red points (i+j even) from the four new green values
template <typename T>
__global__ void k_r2g_c_2d(A2<const T> rg, A2<T> vg, int n, T c, const int *done, Bt B) {
    const int prob_ = bt_prob(B);
    if (stop(bt_done(done, prob_, B))) return;
    rg = bt_at(rg, prob_, B);
    vg = bt_at(vg, prob_, B);
    MG_IDX2 const int i = tx + 1, j = ty + 1;
    if (i > n || j > n || ((i + j) & 1) == 1) return;
    T s = (vg(i - 1, j) + vg(i + 1, j)) + (vg(i, j - 1) + vg(i, j + 1));
    vg(i, j) = (s - c * rg(i, j)) * T(0.25);
}

// extra sweep on a green level, first half: green-only points (i+j odd) from
// the four axis neighbours of the level itself (extension of Section 5; the
// second half is k_r2g_c_2d)
template <typename T>
__global__ void k_g2g_f_2d(A2<const T> rg, A2<T> vg, int n, T c, const int *done, Bt B) {
    const int prob_ = bt_prob(B);
    if (stop(bt_done(done, prob_, B))) return;
    rg = bt_at(rg, prob_, B);
    vg = bt_at(vg, prob_, B);
    MG_IDX2 const int i = tx + 1, j = ty + 1;
    if (i > n || j > n || ((i + j) & 1) == 0) return;
    T s = (vg(i - 1, j) + vg(i + 1, j)) + (vg(i, j - 1) + vg(i, j + 1));
    vg(i, j) = (s - c * rg(i, j)) * T(0.25);
}

// finest level: second half fused with the update u += v at every point
template <typename T>
__global__ void k_r2g_c_upd_2d(A2<const T> rg, A2<const T> vg, double *u, int up, int n, T c, const int *done, Bt B) {
    const int prob_ = bt_prob(B);
    if (stop(bt_done(done, prob_, B))) return;
    rg = bt_at(rg, prob_, B);
    vg = bt_at(vg, prob_, B);
    if (B.utab) u = B.utab[prob_];
    MG_IDX2 const int i = tx + 1, j = ty + 1;
    if (i > n || j > n) return;
    T v;
    if ((i + j) & 1) v = vg(i, j);
    else v = ((vg(i - 1, j) + vg(i + 1, j)) + (vg(i, j - 1) + vg(i, j + 1)) - c * rg(i, j)) * T(0.25);
    u[(size_t)j * up + i] += widen(v);
}

// ---------------------------------------------------------------------------
// 3D diagonal hierarchy (Section 3)
// ---------------------------------------------------------------------------

template <typename T> struct Red3 { A3<T> eee, ooe, oeo, eoo; };
template <typename T> struct Mag3 { A3<T> eee, ooo; };
template <typename T> __device__ __forceinline__ Red3<T> bt_at(Red3<T> r, int p, const Bt &B) {
    r.eee = bt_at(r.eee, p, B); r.ooe = bt_at(r.ooe, p, B); r.oeo = bt_at(r.oeo, p, B); r.eoo = bt_at(r.eoo, p, B);
    return r;
}
template <typename T> __device__ __forceinline__ Mag3<T> bt_at(Mag3<T> m, int p, const Bt &B) {
    m.eee = bt_at(m.eee, p, B); m.ooo = bt_at(m.ooo, p, B);
    return m;
}

// red level value at green point (x,y,z), x+y+z even
template <typename T> __device__ __forceinline__ T red3(const Red3<const T> &r, int x, int y, int z) {
    const int px = x & 1, py = y & 1;
    const int a = x >> 1, b = y >> 1, c = z >> 1;
    if (px && py) return r.ooe(a, b, c);
    if (px) return r.oeo(a, b, c);
    if (py) return r.eoo(a, b, c);
    return r.eee(a, b, c);
}

// green -> red, Eq. Erred: (6r + 6 axis neighbours)/12 at i+j+k even.
// Thread per cell (a,b,c) in [0,nb]^3 holding EEE, OOE, OEO, EOO points.
template <typename T>
__global__ void k_g2r_3d(A3<const T> g, Red3<T> red, int nb, const T *galt, const int *par, const int *done, Bt B) {
    const int prob_ = bt_prob(B);
    if (stop(bt_done(done, prob_, B))) return;
    if (galt && par[(size_t)prob_ * B.ctl_stride]) g.p = galt;  // the current one of two green buffers
    g = bt_at(g, prob_, B);
    red = bt_at(red, prob_, B);
    MG_IDX3 const int a = tx, b = ty, c = tz;
    if (a > nb || b > nb || c > nb) return;
    auto avg = [&](int i, int j, int k) {
        return (T(6) * g(i, j, k) + (g(i + 1, j, k) + g(i - 1, j, k)) + (g(i, j + 1, k) + g(i, j - 1, k)) +
                (g(i, j, k + 1) + g(i, j, k - 1))) * T(1.0 / 12.0);
    };
    if (a >= 1 && b >= 1 && c >= 1) red.eee(a, b, c) = avg(2 * a, 2 * b, 2 * c);
    if (c >= 1) red.ooe(a, b, c) = avg(2 * a + 1, 2 * b + 1, 2 * c);
    if (b >= 1) red.oeo(a, b, c) = avg(2 * a + 1, 2 * b, 2 * c + 1);
    if (a >= 1) red.eoo(a, b, c) = avg(2 * a, 2 * b + 1, 2 * c + 1);
}

// sum of the 12 face-centre (FCC) neighbours of the corner (2a,2b,2c)
template <typename T>
__device__ __forceinline__ T fcc12(const A3<const T> &ooe, const A3<const T> &oeo, const A3<const T> &eoo, int a,
                                   int b, int c) {
    T s1 = (ooe(a - 1, b - 1, c) + ooe(a, b - 1, c)) + (ooe(a - 1, b, c) + ooe(a, b, c));
    T s2 = (oeo(a - 1, b, c - 1) + oeo(a, b, c - 1)) + (oeo(a - 1, b, c) + oeo(a, b, c));
    T s3 = (eoo(a, b - 1, c - 1) + eoo(a, b, c - 1)) + (eoo(a, b - 1, c) + eoo(a, b, c));
    return s1 + s2 + s3;
}
// the largest of m and the magnitudes of the 12 values fcc12 sums
template <typename T>
__device__ __forceinline__ float fcc12_absmax(const A3<const T> &ooe, const A3<const T> &oeo, const A3<const T> &eoo,
                                              int a, int b, int c, float m) {
    const T q[12] = {ooe(a - 1, b - 1, c), ooe(a, b - 1, c), ooe(a - 1, b, c), ooe(a, b, c),
                     oeo(a - 1, b, c - 1), oeo(a, b, c - 1), oeo(a - 1, b, c), oeo(a, b, c),
                     eoo(a, b - 1, c - 1), eoo(a, b, c - 1), eoo(a, b - 1, c), eoo(a, b, c)};
#pragma unroll
    for (int k = 0; k < 12; k++) m = fmaxf(m, (float)fabs(q[k]));
    return m;
}

// red -> magenta: corners, Eq. Ermagc (12r + 12 FCC neighbours)/24; centres,
// Eq. Ermagm mean of the 6 face-centre neighbours.  Thread per cell in [0,nb]^3.
template <typename T>
__global__ void k_r2m_3d(Red3<const T> red, Mag3<T> mag, int nb, const int *done, Bt B) {
    const int prob_ = bt_prob(B);
    if (stop(bt_done(done, prob_, B))) return;
    red = bt_at(red, prob_, B);
    mag = bt_at(mag, prob_, B);
    MG_IDX3 const int a = tx, b = ty, c = tz;
    if (a > nb || b > nb || c > nb) return;
    if (a >= 1 && b >= 1 && c >= 1)
        mag.eee(a, b, c) = (T(12) * red.eee(a, b, c) + fcc12(red.ooe, red.oeo, red.eoo, a, b, c)) * T(1.0 / 24.0);
    mag.ooo(a, b, c) = ((red.eoo(a, b, c) + red.eoo(a + 1, b, c)) + (red.oeo(a, b, c) + red.oeo(a, b + 1, c)) +
                        (red.ooe(a, b, c) + red.ooe(a, b, c + 1))) * T(1.0 / 6.0);
}

// sum of the 8 centres around the corner (2a,2b,2c)
template <typename T> __device__ __forceinline__ T ctr8(const A3<const T> &ooo, int a, int b, int c) {
    return ((ooo(a - 1, b - 1, c - 1) + ooo(a, b - 1, c - 1)) + (ooo(a - 1, b, c - 1) + ooo(a, b, c - 1))) +
           ((ooo(a - 1, b - 1, c) + ooo(a, b - 1, c)) + (ooo(a - 1, b, c) + ooo(a, b, c)));
}

// magenta -> blue, Eq. Erblu: (8r + 8 centre neighbours)/16 at the blue corners
template <typename T>
__global__ void k_m2b_3d(Mag3<const T> mag, A3<T> blue, int nb, const int *done, Bt B) {
    const int prob_ = bt_prob(B);
    if (stop(bt_done(done, prob_, B))) return;
    mag = bt_at(mag, prob_, B);
    blue = bt_at(blue, prob_, B);
    MG_IDX3 const int a = tx + 1, b = ty + 1, c = tz + 1;
    if (a > nb || b > nb || c > nb) return;
    blue(a, b, c) = (T(8) * mag.eee(a, b, c) + ctr8(mag.ooo, a, b, c)) * T(0.0625);
}

// Eq. Emprolm: magenta centres from the 8 blue corners; c = 4 p_m h^2
template <typename T>
__global__ void k_b2m_ooo_3d(A3<const T> blue, A3<const T> rooo, A3<T> vooo, int nb, T cc, const int *done, Bt B) {
    const int prob_ = bt_prob(B);
    if (stop(bt_done(done, prob_, B))) return;
    blue = bt_at(blue, prob_, B);
    rooo = bt_at(rooo, prob_, B);
    vooo = bt_at(vooo, prob_, B);
    MG_IDX3 const int a = tx, b = ty, c = tz;
    if (a > nb || b > nb || c > nb) return;
    T s = ((blue(a, b, c) + blue(a + 1, b, c)) + (blue(a, b + 1, c) + blue(a + 1, b + 1, c))) +
          ((blue(a, b, c + 1) + blue(a + 1, b, c + 1)) + (blue(a, b + 1, c + 1) + blue(a + 1, b + 1, c + 1)));
    vooo(a, b, c) = (s - cc * rooo(a, b, c)) * T(0.125);
}

// Eq. Emprolb: blue corners refined from the 8 new centres
template <typename T>
__global__ void k_b2m_eee_3d(A3<const T> vooo, A3<const T> reee, A3<T> veee, int nb, T cc, const int *done, Bt B) {
    const int prob_ = bt_prob(B);
    if (stop(bt_done(done, prob_, B))) return;
    vooo = bt_at(vooo, prob_, B);
    reee = bt_at(reee, prob_, B);
    veee = bt_at(veee, prob_, B);
    MG_IDX3 const int a = tx + 1, b = ty + 1, c = tz + 1;
    if (a > nb || b > nb || c > nb) return;
    veee(a, b, c) = (ctr8(vooo, a, b, c) - cc * reee(a, b, c)) * T(0.125);
}

// Eq. Emprolm then Eq. Emprolb in one launch (the small triples): a block of
// 8 x 8 x 4 cells forms the magenta centres of its cells and of the cell
// before them in each direction (the corners' 8 centres), stores its own, and
// then refines its own blue corners from those values in shared memory; the
// terms of both half-sweeps in the order of k_b2m_ooo_3d / k_b2m_eee_3d.
constexpr int BM_X = 8, BM_Y = 8, BM_Z = 4;
template <typename T>
__global__ void __launch_bounds__(256) k_b2m_3d(A3<const T> blue, A3<const T> rooo, A3<const T> reee, A3<T> vooo,
                                                A3<T> veee, int nb, T cc, const int *done, Bt B) {
    __shared__ T so[BM_Z + 1][BM_Y + 1][BM_X + 1];
    const int prob_ = bt_prob(B), bz = bt_z(B);
    if (stop(bt_done(done, prob_, B))) return;
    blue = bt_at(blue, prob_, B);
    rooo = bt_at(rooo, prob_, B);
    reee = bt_at(reee, prob_, B);
    vooo = bt_at(vooo, prob_, B);
    veee = bt_at(veee, prob_, B);
    const int x0 = blockIdx.x * BM_X, y0 = blockIdx.y * BM_Y, z0 = bz * BM_Z;
    const int tid = threadIdx.x + 32 * threadIdx.y;
    // centres of cells [x0-1, x0+8) x [y0-1, y0+8) x [z0-1, z0+4)
    for (int q = tid; q < (BM_X + 1) * (BM_Y + 1) * (BM_Z + 1); q += 256) {
        const int lx = q % (BM_X + 1), ly = (q / (BM_X + 1)) % (BM_Y + 1), lz = q / ((BM_X + 1) * (BM_Y + 1));
        const int a = x0 - 1 + lx, b = y0 - 1 + ly, c = z0 - 1 + lz;
        T v = T(0);
        if (a >= 0 && a <= nb && b >= 0 && b <= nb && c >= 0 && c <= nb) {
            const T s = ((blue(a, b, c) + blue(a + 1, b, c)) + (blue(a, b + 1, c) + blue(a + 1, b + 1, c))) +
                        ((blue(a, b, c + 1) + blue(a + 1, b, c + 1)) + (blue(a, b + 1, c + 1) + blue(a + 1, b + 1, c + 1)));
            v = (s - cc * rooo(a, b, c)) * T(0.125);
            if (lx >= 1 && ly >= 1 && lz >= 1) vooo(a, b, c) = v;
        }
        so[lz][ly][lx] = v;
    }
    __syncthreads();
    // corners of the own cells: the 8 centres (a-1..a) x (b-1..b) x (c-1..c)
    const int lx = tid & 7, ly = (tid >> 3) & 7, lz = tid >> 6;  // 8 x 8 x 4
    const int a = x0 + lx, b = y0 + ly, c = z0 + lz;
    if (a >= 1 && a <= nb && b >= 1 && b <= nb && c >= 1 && c <= nb) {
        const int i = lx + 1, j = ly + 1, k = lz + 1;  // smem index of cell (a, b, c)
        const T s8 = ((so[k - 1][j - 1][i - 1] + so[k - 1][j - 1][i]) + (so[k - 1][j][i - 1] + so[k - 1][j][i])) +
                     ((so[k][j - 1][i - 1] + so[k][j - 1][i]) + (so[k][j][i - 1] + so[k][j][i]));
        veee(a, b, c) = (s8 - cc * reee(a, b, c)) * T(0.125);
    }
}

// Eq. Erprolr and its cyclic permutations: red face centres from the two
// magenta centres along the face normal (weight 2) and the four in-plane
// magenta corners; c1 = 2 p_r1 h^2.  Thread per cell in [0,nb]^3.
template <typename T>
__global__ void k_m2r_faces_3d(Mag3<const T> vm, Red3<const T> rr, Red3<T> vr, int nb, T c1, const int *done, Bt B) {
    const int prob_ = bt_prob(B);
    if (stop(bt_done(done, prob_, B))) return;
    vm = bt_at(vm, prob_, B);
    rr = bt_at(rr, prob_, B);
    vr = bt_at(vr, prob_, B);
    MG_IDX3 const int a = tx, b = ty, c = tz;
    if (a > nb || b > nb || c > nb) return;
    if (c >= 1) {  // (2a+1, 2b+1, 2c): normal z
        T ctr = vm.ooo(a, b, c - 1) + vm.ooo(a, b, c);
        T cor = (vm.eee(a, b, c) + vm.eee(a + 1, b, c)) + (vm.eee(a, b + 1, c) + vm.eee(a + 1, b + 1, c));
        vr.ooe(a, b, c) = (T(2) * ctr + cor - c1 * rr.ooe(a, b, c)) * T(0.125);
    }
    if (b >= 1) {  // (2a+1, 2b, 2c+1): normal y
        T ctr = vm.ooo(a, b - 1, c) + vm.ooo(a, b, c);
        T cor = (vm.eee(a, b, c) + vm.eee(a + 1, b, c)) + (vm.eee(a, b, c + 1) + vm.eee(a + 1, b, c + 1));
        vr.oeo(a, b, c) = (T(2) * ctr + cor - c1 * rr.oeo(a, b, c)) * T(0.125);
    }
    if (a >= 1) {  // (2a, 2b+1, 2c+1): normal x
        T ctr = vm.ooo(a - 1, b, c) + vm.ooo(a, b, c);
        T cor = (vm.eee(a, b, c) + vm.eee(a, b + 1, c)) + (vm.eee(a, b, c + 1) + vm.eee(a, b + 1, c + 1));
        vr.eoo(a, b, c) = (T(2) * ctr + cor - c1 * rr.eoo(a, b, c)) * T(0.125);
    }
}

// Eq. Erprolr then Eq. Erprolm in one launch (small levels, no bound on |v|
// wanted): a block of 8 x 8 x 4 cells forms the three face centres of its
// cells and of the cell before them in each direction, stores its own, then
// its own corners from those values in shared memory; the terms of both
// half-sweeps in the order of k_m2r_faces_3d / k_m2r_corners_3d (fcc12).
template <typename T>
__global__ void __launch_bounds__(256) k_m2r_3d(Mag3<const T> vm, Red3<const T> rr, Red3<T> vr, int nb, T c1, T c2,
                                                const int *done, Bt B) {
    __shared__ T sf[3][BM_Z + 1][BM_Y + 1][BM_X + 1];  // OOE, OEO, EOO
    const int prob_ = bt_prob(B), bz = bt_z(B);
    if (stop(bt_done(done, prob_, B))) return;
    vm = bt_at(vm, prob_, B);
    rr = bt_at(rr, prob_, B);
    vr = bt_at(vr, prob_, B);
    const int x0 = blockIdx.x * BM_X, y0 = blockIdx.y * BM_Y, z0 = bz * BM_Z;
    const int tid = threadIdx.x + 32 * threadIdx.y;
    for (int q = tid; q < (BM_X + 1) * (BM_Y + 1) * (BM_Z + 1); q += 256) {
        const int lx = q % (BM_X + 1), ly = (q / (BM_X + 1)) % (BM_Y + 1), lz = q / ((BM_X + 1) * (BM_Y + 1));
        const int a = x0 - 1 + lx, b = y0 - 1 + ly, c = z0 - 1 + lz;
        const bool in = a >= 0 && a <= nb && b >= 0 && b <= nb && c >= 0 && c <= nb;
        const bool own = in && lx >= 1 && ly >= 1 && lz >= 1;
        T fz = T(0), fy = T(0), fx = T(0);
        if (in && c >= 1) {  // (2a+1, 2b+1, 2c): normal z
            T ctr = vm.ooo(a, b, c - 1) + vm.ooo(a, b, c);
            T cor = (vm.eee(a, b, c) + vm.eee(a + 1, b, c)) + (vm.eee(a, b + 1, c) + vm.eee(a + 1, b + 1, c));
            fz = (T(2) * ctr + cor - c1 * rr.ooe(a, b, c)) * T(0.125);
            if (own) vr.ooe(a, b, c) = fz;
        }
        if (in && b >= 1) {  // (2a+1, 2b, 2c+1): normal y
            T ctr = vm.ooo(a, b - 1, c) + vm.ooo(a, b, c);
            T cor = (vm.eee(a, b, c) + vm.eee(a + 1, b, c)) + (vm.eee(a, b, c + 1) + vm.eee(a + 1, b, c + 1));
            fy = (T(2) * ctr + cor - c1 * rr.oeo(a, b, c)) * T(0.125);
            if (own) vr.oeo(a, b, c) = fy;
        }
        if (in && a >= 1) {  // (2a, 2b+1, 2c+1): normal x
            T ctr = vm.ooo(a - 1, b, c) + vm.ooo(a, b, c);
            T cor = (vm.eee(a, b, c) + vm.eee(a, b + 1, c)) + (vm.eee(a, b, c + 1) + vm.eee(a, b + 1, c + 1));
            fx = (T(2) * ctr + cor - c1 * rr.eoo(a, b, c)) * T(0.125);
            if (own) vr.eoo(a, b, c) = fx;
        }
        sf[0][lz][ly][lx] = fz;
        sf[1][lz][ly][lx] = fy;
        sf[2][lz][ly][lx] = fx;
    }
    __syncthreads();
    const int lx = tid & 7, ly = (tid >> 3) & 7, lz = tid >> 6;  // 8 x 8 x 4
    const int a = x0 + lx, b = y0 + ly, c = z0 + lz;
    if (a >= 1 && a <= nb && b >= 1 && b <= nb && c >= 1 && c <= nb) {
        const int i = lx + 1, j = ly + 1, k = lz + 1;  // smem index of cell (a, b, c)
        const T s1 = (sf[0][k][j - 1][i - 1] + sf[0][k][j - 1][i]) + (sf[0][k][j][i - 1] + sf[0][k][j][i]);
        const T s2 = (sf[1][k - 1][j][i - 1] + sf[1][k - 1][j][i]) + (sf[1][k][j][i - 1] + sf[1][k][j][i]);
        const T s3 = (sf[2][k - 1][j - 1][i] + sf[2][k - 1][j][i]) + (sf[2][k][j - 1][i] + sf[2][k][j][i]);
        vr.eee(a, b, c) = (s1 + s2 + s3 - c2 * rr.eee(a, b, c)) * T(1.0 / 12.0);
    }
}

// Eq. Erprolm: magenta corners (red EEE) from the 12 new face centres; c2 = 4 p_r2 h^2
template <typename T>
// vctl (the finest triple of the fused mixed path): also the largest |v| of
// the red level -- the new corner and the 12 face values each cell reads,
// which cover every face value -- into vctl[p].vmax
__global__ void k_m2r_corners_3d(Red3<const T> vr_faces, A3<const T> reee, A3<T> veee, int nb, T c2,
                                 Ctrl *vctl, const int *done, Bt B) {
    __shared__ float shm[32];
    const int prob_ = bt_prob(B);
    if (stop(bt_done(done, prob_, B))) return;
    vr_faces = bt_at(vr_faces, prob_, B);
    reee = bt_at(reee, prob_, B);
    veee = bt_at(veee, prob_, B);
    MG_IDX3 const int a = tx + 1, b = ty + 1, c = tz + 1;
    float mx = 0.f;
    if (a <= nb && b <= nb && c <= nb) {
        const T v = (fcc12(vr_faces.ooe, vr_faces.oeo, vr_faces.eoo, a, b, c) - c2 * reee(a, b, c)) * T(1.0 / 12.0);
        if (vctl) mx = fcc12_absmax(vr_faces.ooe, vr_faces.oeo, vr_faces.eoo, a, b, c, (float)fabs(v));
        veee(a, b, c) = v;
    }
    if (vctl) {
        mx = block_max(mx, shm);
        if (threadIdx.x == 0 && threadIdx.y == 0 && threadIdx.z == 0) atomicMax(&vctl[prob_].vmax, __float_as_uint(mx));
    }
}

// Eq. Egprolg: green-only points (i+j+k odd) from the six axis red values; c = p_g h^2
template <typename T>
__global__ void k_r2g_f_3d(Red3<const T> vr, A3<const T> rg, A3<T> vg, int n, T cc, const int *done, Bt B) {
    const int prob_ = bt_prob(B);
    if (stop(bt_done(done, prob_, B))) return;
    vr = bt_at(vr, prob_, B);
    rg = bt_at(rg, prob_, B);
    vg = bt_at(vg, prob_, B);
    MG_IDX3 const int i = tx + 1, j = ty + 1, k = tz + 1;
    if (i > n || j > n || k > n || ((i + j + k) & 1) == 0) return;
    T s = (red3(vr, i - 1, j, k) + red3(vr, i + 1, j, k)) + (red3(vr, i, j - 1, k) + red3(vr, i, j + 1, k)) +
          (red3(vr, i, j, k - 1) + red3(vr, i, j, k + 1));
    vg(i, j, k) = (s - cc * rg(i, j, k)) * T(1.0 / 6.0);
}

// Eq. Egprolr: red points (i+j+k even) from the six new green values
template <typename T>
__global__ void k_r2g_c_3d(A3<const T> rg, A3<T> vg, int n, T cc, const int *done, Bt B) {
    const int prob_ = bt_prob(B);
    if (stop(bt_done(done, prob_, B))) return;
    rg = bt_at(rg, prob_, B);
    vg = bt_at(vg, prob_, B);
    MG_IDX3 const int i = tx + 1, j = ty + 1, k = tz + 1;
    if (i > n || j > n || k > n || ((i + j + k) & 1) == 1) return;
    T s = (vg(i - 1, j, k) + vg(i + 1, j, k)) + (vg(i, j - 1, k) + vg(i, j + 1, k)) +
          (vg(i, j, k - 1) + vg(i, j, k + 1));
    vg(i, j, k) = (s - cc * rg(i, j, k)) * T(1.0 / 6.0);
}

// ---------------------------------------------------------------------------
// Conventional 2^-l hierarchy
// ---------------------------------------------------------------------------

// full weighting (1/16)[1 2 1]x[1 2 1]
template <typename T>
__global__ void k_fw_2d(A2<const T> f, A2<T> cg, int nc, const int *done, Bt B) {
    const int prob_ = bt_prob(B);
    if (stop(bt_done(done, prob_, B))) return;
    f = bt_at(f, prob_, B);
    cg = bt_at(cg, prob_, B);
    MG_IDX2 const int a = tx + 1, b = ty + 1;
    if (a > nc || b > nc) return;
    const int i = 2 * a, j = 2 * b;
    T s = T(4) * f(i, j) + T(2) * ((f(i - 1, j) + f(i + 1, j)) + (f(i, j - 1) + f(i, j + 1))) +
          ((f(i - 1, j - 1) + f(i + 1, j - 1)) + (f(i - 1, j + 1) + f(i + 1, j + 1)));
    cg(a, b) = s * T(0.0625);
}

// full weighting (1/64)[1 2 1]^3
template <typename T>
__global__ void k_fw_3d(A3<const T> f, A3<T> cg, int nc, const int *done, Bt B) {
    const int prob_ = bt_prob(B);
    if (stop(bt_done(done, prob_, B))) return;
    f = bt_at(f, prob_, B);
    cg = bt_at(cg, prob_, B);
    MG_IDX3 const int a = tx + 1, b = ty + 1, c = tz + 1;
    if (a > nc || b > nc || c > nc) return;
    T s = T(0);
    for (int dk = -1; dk <= 1; dk++) {
        T wk = dk == 0 ? T(2) : T(1);
        for (int dj = -1; dj <= 1; dj++) {
            T wj = dj == 0 ? T(2) : T(1);
            T row = T(2) * f(2 * a, 2 * b + dj, 2 * c + dk) + (f(2 * a - 1, 2 * b + dj, 2 * c + dk) +
                                                               f(2 * a + 1, 2 * b + dj, 2 * c + dk));
            s += wk * wj * row;
        }
    }
    cg(a, b, c) = s * T(1.0 / 64.0);
}

template <typename T> __device__ __forceinline__ T interp2(const A2<const T> &vc, int i, int j) {
    const int a0 = i >> 1, a1 = (i + 1) >> 1, b0 = j >> 1, b1 = (j + 1) >> 1;
    return ((vc(a0, b0) + vc(a1, b0)) + (vc(a0, b1) + vc(a1, b1))) * T(0.25);
}
template <typename T> __device__ __forceinline__ T interp3(const A3<const T> &vc, int i, int j, int k) {
    const int a0 = i >> 1, a1 = (i + 1) >> 1, b0 = j >> 1, b1 = (j + 1) >> 1, c0 = k >> 1, c1 = (k + 1) >> 1;
    return (((vc(a0, b0, c0) + vc(a1, b0, c0)) + (vc(a0, b1, c0) + vc(a1, b1, c0))) +
            ((vc(a0, b0, c1) + vc(a1, b0, c1)) + (vc(a0, b1, c1) + vc(a1, b1, c1)))) * T(0.125);
}

// conventional prolongation, first half of the red-black Jacobi iteration:
// points with odd index sum from the bilinearly interpolated coarse values of
// their axis neighbours (the interpolated values at odd points are never read)
template <typename T>
__global__ void k_usual_odd_2d(A2<const T> vc, A2<const T> rg, A2<T> vg, int n, T c, const int *done, Bt B) {
    const int prob_ = bt_prob(B);
    if (stop(bt_done(done, prob_, B))) return;
    vc = bt_at(vc, prob_, B);
    rg = bt_at(rg, prob_, B);
    vg = bt_at(vg, prob_, B);
    MG_IDX2 const int i = tx + 1, j = ty + 1;
    if (i > n || j > n || ((i + j) & 1) == 0) return;
    T s = (interp2(vc, i - 1, j) + interp2(vc, i + 1, j)) + (interp2(vc, i, j - 1) + interp2(vc, i, j + 1));
    vg(i, j) = (s - c * rg(i, j)) * T(0.25);
}
template <typename T>
__global__ void k_usual_odd_3d(A3<const T> vc, A3<const T> rg, A3<T> vg, int n, T c, const int *done, Bt B) {
    const int prob_ = bt_prob(B);
    if (stop(bt_done(done, prob_, B))) return;
    vc = bt_at(vc, prob_, B);
    rg = bt_at(rg, prob_, B);
    vg = bt_at(vg, prob_, B);
    MG_IDX3 const int i = tx + 1, j = ty + 1, k = tz + 1;
    if (i > n || j > n || k > n || ((i + j + k) & 1) == 0) return;
    T s = (interp3(vc, i - 1, j, k) + interp3(vc, i + 1, j, k)) + (interp3(vc, i, j - 1, k) + interp3(vc, i, j + 1, k)) +
          (interp3(vc, i, j, k - 1) + interp3(vc, i, j, k + 1));
    vg(i, j, k) = (s - c * rg(i, j, k)) * T(1.0 / 6.0);
}
// the second half (even index sum) is k_r2g_c_2d / k_r2g_c_3d (and their update variants)

// ---------------------------------------------------------------------------
// residuals, norms, coarsest solve, level import/export
// ---------------------------------------------------------------------------

// block sum of a double, result valid in thread 0; blockDim.x*blockDim.y*blockDim.z <= 1024
__device__ __forceinline__ double block_sum(double v, double *sh) {
    const int tid = threadIdx.x + blockDim.x * (threadIdx.y + blockDim.y * threadIdx.z);
    const int nt = blockDim.x * blockDim.y * blockDim.z;
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    if ((tid & 31) == 0) sh[tid >> 5] = v;
    __syncthreads();
    if (tid < 32) {
        v = tid < (nt + 31) / 32 ? sh[tid] : 0.0;
        for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    }
    return v;
}

// block sum of per-thread FP32 sums: FP32 within each warp, FP64 across the
// warps (result valid in thread 0).  A kernel with a few points per thread
// would otherwise spend more FP64 instructions on the reduction than on its
// points (a conversion and five adds per thread); the warp sums of 32
// non-negative terms carry a relative error below 2^-19.
__device__ __forceinline__ double block_sum_f(float v, double *sh) {
    const int tid = threadIdx.x + blockDim.x * (threadIdx.y + blockDim.y * threadIdx.z);
    const int nt = blockDim.x * blockDim.y * blockDim.z;
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    if ((tid & 31) == 0) sh[tid >> 5] = (double)v;
    __syncthreads();
    double d = 0.0;
    if (tid < 32) {
        d = tid < (nt + 31) / 32 ? sh[tid] : 0.0;
        for (int o = 16; o > 0; o >>= 1) d += __shfl_down_sync(0xffffffffu, d, o);
    }
    return d;
}


// r = f - L_h u (Eq. Evpois, 5-point) or Eq. Efos2 (ORDER 4); RHS_ONLY: u = 0.
// Writes r (level precision) and, if r64 != nullptr, the FP64 value to the
// caller grid; block partial sums of r^2 to part[block].
template <typename T, int ORDER, bool RHS_ONLY>
__global__ void k_res_2d(const double *__restrict__ f, const double *__restrict__ u, int up, int n, double ih2,
                         A2<T> r, double *r64, double *part, const int *done, Bt B) {
    __shared__ double sh[32];
    const int prob_ = bt_prob(B);
    if (stop(bt_done(done, prob_, B))) return;
    if (B.ftab) f = B.ftab[prob_];
    if (B.utab) u = B.utab[prob_];
    r = bt_at(r, prob_, B);
    if (B.ftab) r64 = nullptr;
    part += (size_t)prob_ * B.nparts;
    MG_IDX2 const int i = tx + 1, j = ty + 1;
    double sq = 0.0;
    if (i <= n && j <= n) {
        const size_t c = (size_t)j * up + i;
        double res;
        if (ORDER == 2) {
            res = f[c];
            if (!RHS_ONLY) res = fma(-ih2, ((u[c - 1] + u[c + 1]) + (u[c - up] + u[c + up])) - 4.0 * u[c], res);
        } else {
            res = (8.0 * f[c] + ((f[c - 1] + f[c + 1]) + (f[c - up] + f[c + up]))) * (1.0 / 12.0);
            if (!RHS_ONLY) {
                double ax = (u[c - 1] + u[c + 1]) + (u[c - up] + u[c + up]);
                double dg = (u[c - up - 1] + u[c - up + 1]) + (u[c + up - 1] + u[c + up + 1]);
                res = fma(-ih2 * (1.0 / 6.0), fma(4.0, ax, dg) - 20.0 * u[c], res);
            }
        }
        r(i, j) = lvl<T>(res);
        if (r64) r64[c] = res;
        sq = res * res;
    }
    double s = block_sum(sq, sh);
    if (threadIdx.x == 0 && threadIdx.y == 0) part[blockIdx.x + gridDim.x * blockIdx.y] = s;
}

// 3D: 7-point (ORDER 2) or Eq. Efos4 19-point (ORDER 4)
template <typename T, int ORDER, bool RHS_ONLY>
__global__ void k_res_3d(const double *__restrict__ f, const double *__restrict__ u, int up, int urows, int n,
                         double ih2, A3<T> r, double *r64, double *part, const int *done, Bt B) {
    __shared__ double sh[32];
    const int prob_ = bt_prob(B);
    if (stop(bt_done(done, prob_, B))) return;
    if (B.ftab) f = B.ftab[prob_];
    if (B.utab) u = B.utab[prob_];
    r = bt_at(r, prob_, B);
    if (B.ftab) r64 = nullptr;
    part += (size_t)prob_ * B.nparts;
    MG_IDX3 const int i = tx + 1, j = ty + 1, k = tz + 1;
    double sq = 0.0;
    if (i <= n && j <= n) {
        const size_t pl = (size_t)urows * up;
        const size_t c = k * pl + (size_t)j * up + i;
        double res;
        if (ORDER == 2) {
            res = f[c];
            if (!RHS_ONLY) {
                double ax = ((u[c - 1] + u[c + 1]) + (u[c - up] + u[c + up])) + (u[c - pl] + u[c + pl]);
                res = fma(-ih2, ax - 6.0 * u[c], res);
            }
        } else {
            res = (6.0 * f[c] + ((f[c - 1] + f[c + 1]) + (f[c - up] + f[c + up]) + (f[c - pl] + f[c + pl]))) *
                  (1.0 / 12.0);
            if (!RHS_ONLY) {
                double ax = ((u[c - 1] + u[c + 1]) + (u[c - up] + u[c + up])) + (u[c - pl] + u[c + pl]);
                double ed = ((u[c - up - 1] + u[c - up + 1]) + (u[c + up - 1] + u[c + up + 1])) +
                            ((u[c - pl - up] + u[c - pl + up]) + (u[c + pl - up] + u[c + pl + up])) +
                            ((u[c - pl - 1] + u[c - pl + 1]) + (u[c + pl - 1] + u[c + pl + 1]));
                res = fma(-ih2 * (1.0 / 6.0), fma(2.0, ax, ed) - 24.0 * u[c], res);
            }
        }
        r(i, j, k) = lvl<T>(res);
        if (r64) r64[c] = res;
        sq = res * res;
    }
    double s = block_sum(sq, sh);
    if (threadIdx.x == 0 && threadIdx.y == 0)
        part[blockIdx.x + gridDim.x * (blockIdx.y + (size_t)gridDim.y * bt_z(B))] = s;
}


// deterministic sum of part[0..nblk) by one block of 1024 threads (fixed order)
__device__ __forceinline__ double sum_parts(const double *part, int nblk, double *sh) {
    double v = 0.0;
    for (int q = threadIdx.x; q < nblk; q += blockDim.x) v += part[q];
    return block_sum(v, sh);
}

// relative residual sqrt(r2 / f2); 0 for a zero right-hand side (any iterate
// is then as good as the exact solution 0 in relative terms), NaN when f2 is
// not a number (a right-hand side carrying NaN), so that the solve reports
// divergence instead of convergence
__device__ __forceinline__ double rel_residual(double r2, double f2) {
    return f2 > 0.0 ? sqrt(r2 / f2) : (f2 == 0.0 ? 0.0 : __longlong_as_double(0x7ff8000000000000ll));
}

// FP64 pipe throughput probe (mg_fp64_rate): every thread runs DFMA_CHAINS
// independent chains of `iters` dependent FP64 FMAs (x <- x * m + c, one
// FP64 pipe operation each); the result is stored only when it equals a
// value it never takes, so the chains stay live without memory traffic
constexpr int DFMA_CHAINS = 8;
__global__ void __launch_bounds__(256) k_dfma_rate(double seed, int iters, double *sink) {
    pdl_wait();
    double x[DFMA_CHAINS];
#pragma unroll
    for (int q = 0; q < DFMA_CHAINS; q++) x[q] = seed + 1e-3 * (threadIdx.x + q);
    const double m = 1.0 - 1e-12, c = 1e-13;
    for (int it = 0; it < iters; it++) {
#pragma unroll
        for (int q = 0; q < DFMA_CHAINS; q++) x[q] = fma(x[q], m, c);
    }
    double t = 0.0;
#pragma unroll
    for (int q = 0; q < DFMA_CHAINS; q++) t += x[q];
    if (t == -1.0) *sink = t;
}

// after the residual of the warm start (first = 1) or of a new iterate:
// record the history, decide whether to stop.  Inside the solver's graph
// (use_loop = 1) it also sets the graph's loop condition to "not done".
// the control step, given the residual sum s of the new iterate (first: of
// the warm start); one thread
__device__ __forceinline__ void ctrl_step(Ctrl *ctl, double s, double *hist, int first,
                                          cudaGraphConditionalHandle loop, int use_loop) {
    if (!first) ctl->par ^= 1;
    ctl->rmax[ctl->par ^ 1] = 0u;  // the buffer the next cycle writes
    ctl->vmax = 0u;
    ctl->r2 = s;
    double rel = rel_residual(s, ctl->f2);
    ctl->relres = rel;
    if (first) ctl->rel0 = rel;
    else hist[ctl->cycles - 1] = rel;
    if (!(rel == rel) || rel > 1e3 * fmax(ctl->rel0, 1.0)) {
        ctl->status = -5;
        ctl->done = 1;
    } else if (rel <= ctl->rtol) {
        ctl->done = 1;
    } else if (ctl->cycles >= ctl->max_cycles) {
        ctl->status = -4;
        ctl->done = 1;
    } else {
        ctl->cycles += 1;  // this cycle will apply a correction
    }
    if (use_loop) cudaGraphSetConditional(loop, ctl->done ? 0u : 1u);
}

__global__ void k_ctrl(const double *part, int nblk, Ctrl *ctl, double *hist, int first,
                       cudaGraphConditionalHandle loop, int use_loop) {
    pdl_wait();
    __shared__ double sh[32];
    if (!first && ctl->done) {
        if (use_loop && threadIdx.x == 0) cudaGraphSetConditional(loop, 0);
        return;
    }
    double s = sum_parts(part, nblk, sh);
    if (threadIdx.x == 0) ctrl_step(ctl, s, hist, first, loop, use_loop);
}

// The control step fused into the finest kernel of a single-problem mixed
// solve (no separate launch per cycle): every block writes its partial sum,
// and the last block of the launch to finish (counted in ctl->arrive) sums
// all partials in a fixed order and runs the control step.  arrive == nullptr:
// not fused.
struct CtrlFuse {
    unsigned *arrive;
    double *hist;
    cudaGraphConditionalHandle loop;
    int use_loop;
};
// every block, after its thread 0 wrote part[own]; sh: 32 doubles
__device__ __noinline__ void ctrl_last_block(const CtrlFuse &cf, Ctrl *ctl, const double *part, int nblk,
                                                double *sh) {
    __shared__ int last;
    const int tid = threadIdx.x + blockDim.x * (threadIdx.y + blockDim.y * threadIdx.z);
    const int nt = blockDim.x * blockDim.y * blockDim.z;
    __syncthreads();
    if (tid == 0) {
        __threadfence();  // the block's partial (and its atomics) before its arrival
        last = atomicAdd(cf.arrive, 1u) == (unsigned)nblk - 1u;
    }
    __syncthreads();
    if (!last) return;
    __threadfence();
    double v = 0.0;
    for (int q = tid; q < nblk; q += nt) v += __ldcg(part + q);
    const double sum = block_sum(v, sh);
    if (tid == 0) {
        *cf.arrive = 0u;
        ctrl_step(ctl, sum, cf.hist, 0, cf.loop, cf.use_loop);
    }
}

__global__ void k_ctrl_init(Ctrl *ctl, double rtol, int max_cycles) {
    pdl_wait();
    ctl->r2 = 0.0; ctl->relres = 0.0; ctl->rel0 = 0.0; ctl->rtol = rtol;
    ctl->done = 0; ctl->cycles = 0; ctl->max_cycles = max_cycles; ctl->status = 0; ctl->par = 0;
    ctl->vmax = 0u; ctl->rmax[0] = 0u; ctl->rmax[1] = 0u; ctl->arrive = 0u;
}

// per problem of a batch (one block each): f2 = sum of that problem's partials
__global__ void k_sum_to_b(const double *part, int nblk, Ctrl *ctl) {
    pdl_wait();
    __shared__ double sh[32];
    double s = sum_parts(part + (size_t)blockIdx.x * nblk, nblk, sh);
    if (threadIdx.x == 0) ctl[blockIdx.x].f2 = s;
}

__global__ void k_ctrl_init_b(Ctrl *ctl, int nprob, double rtol, int max_cycles) {
    pdl_wait();
    for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < nprob; p += gridDim.x * blockDim.x) {
        Ctrl &c = ctl[p];
        c.r2 = 0.0; c.relres = 0.0; c.rel0 = 0.0; c.rtol = rtol;
        c.done = 0; c.cycles = 0; c.max_cycles = max_cycles; c.status = 0; c.par = 0;
        c.vmax = 0u; c.rmax[0] = 0u; c.rmax[1] = 0u; c.arrive = 0u;
    }
}

// per problem of a batch (one block each): the control step of k_ctrl, with the
// history of problem p at hist + p * hist_cap
__global__ void k_ctrl_b(const double *part, int nblk, Ctrl *ctl, double *hist, int hist_cap, int first) {
    pdl_wait();
    __shared__ double sh[32];
    const int p = blockIdx.x;
    Ctrl *c = ctl + p;
    if (!first && c->done) return;
    double s = sum_parts(part + (size_t)p * nblk, nblk, sh);
    if (threadIdx.x != 0) return;
    if (!first) c->par ^= 1;
    c->rmax[c->par ^ 1] = 0u;
    c->vmax = 0u;
    c->r2 = s;
    double rel = rel_residual(s, c->f2);
    c->relres = rel;
    if (first) c->rel0 = rel;
    else hist[(size_t)p * hist_cap + c->cycles - 1] = rel;
    if (!(rel == rel) || rel > 1e3 * fmax(c->rel0, 1.0)) {
        c->status = -5; c->done = 1;
    } else if (rel <= c->rtol) {
        c->done = 1;
    } else if (c->cycles >= c->max_cycles) {
        c->status = -4; c->done = 1;
    } else {
        c->cycles += 1;
    }
}

// after a solve that carried its residual from cycle to cycle: replace the
// reported relative residual by the one of a direct FP64 residual of the final
// iterate (one block per problem); above rtol the solve counts as not converged
__global__ void k_final_true(const double *part, int nblk, Ctrl *ctl) {
    pdl_wait();
    __shared__ double sh[32];
    const int p = blockIdx.x;
    Ctrl *c = ctl + p;
    const double s = sum_parts(part + (size_t)p * nblk, nblk, sh);
    if (threadIdx.x != 0) return;
    const double rel = rel_residual(s, c->f2);
    c->r2 = s;
    c->relres = rel;
    if (c->status == 0 && !(rel <= c->rtol)) c->status = -4;
}

// max |x| over the narr arrays (a[0..narr)) of a level, each ext^2 (2D, nz =
// 1) or ext^3 values with row pitch `pitch` and `rows` rows per plane, into
// ctl[p].vmax as float bits, per problem p of a batch.  One warp per row.
// The fused finest sweep of the mixed path bounds its correction by it.
struct AbsArrs {
    const float *a[4];
};
__global__ void __launch_bounds__(256) k_absmax(AbsArrs A, int narr, int ext, int nz, int pitch, int rows, Ctrl *ctl,
                                                const int *done, Bt B) {
    __shared__ float sh[32];
    const int prob = bt_prob(B);
    if (stop(bt_done(done, prob, B))) return;
    const size_t plane = (size_t)pitch * rows;
    const int nrow = narr * nz * ext;
    float m = 0.f;
    for (int q = blockIdx.x * 8 + threadIdx.y; q < nrow; q += gridDim.x * 8) {
        const int arr = q / (nz * ext), rz = q - arr * (nz * ext), z = rz / ext, y = rz - z * ext;
        const float *a = arr == 0 ? A.a[0] : arr == 1 ? A.a[1] : arr == 2 ? A.a[2] : A.a[3];
        const float *row = bt_ptr(a, prob, B) + (size_t)z * plane + (size_t)y * pitch;
#pragma unroll 4
        for (int x = threadIdx.x; x < ext; x += 32) m = fmaxf(m, fabsf(row[x]));
    }
    m = block_max(m, sh);
    if (threadIdx.x == 0 && threadIdx.y == 0) atomicMax(&ctl[prob].vmax, __float_as_uint(m));
}

// loop condition of a batch: continue while any problem is not done
__global__ void k_any_active(const Ctrl *ctl, int nprob, cudaGraphConditionalHandle loop, int use_loop, int *active) {
    pdl_wait();
    __shared__ int any;
    if (threadIdx.x == 0) any = 0;
    __syncthreads();
    for (int p = threadIdx.x; p < nprob; p += blockDim.x)
        if (!ctl[p].done) any = 1;
    __syncthreads();
    if (threadIdx.x == 0) {
        if (active) *active = any;
        if (use_loop) cudaGraphSetConditional(loop, any ? 1u : 0u);
    }
}

// power iteration step: ratio[c] = ||u|| / ||u before the cycle|| (the latter
// is 1 after normalisation), then u <- u / ||u|| on the interior
__global__ void k_rho_record(const double *part, int nblk, double *scal, double *ratio, int c) {
    pdl_wait();
    __shared__ double sh[32];
    const double s = sum_parts(part, nblk, sh);
    if (threadIdx.x == 0) {
        const double nrm = sqrt(s);
        ratio[c] = nrm;
        scal[0] = nrm > 0.0 ? 1.0 / nrm : 0.0;
    }
}
__global__ void k_scale_grid(double *u, int up, int n, int dim, const double *scal) {
    pdl_wait();
    MG_IDX2 const int i = tx + 1, j = ty + 1, k = dim == 3 ? (int)blockIdx.z + 1 : 0;
    if (i > n || j > n) return;
    u[((size_t)k * (n + 2) + j) * up + i] *= scal[0];
}

__global__ void k_sum_to(const double *part, int nblk, double *out) {
    pdl_wait();
    __shared__ double sh[32];
    double s = sum_parts(part, nblk, sh);
    if (threadIdx.x == 0) *out = s;
}

// exact coarsest solve: v = G r with the dense inverse G (FP64) of the
// 5/7-point operator of the coarsest grid.  One block.
template <typename T>
__global__ void k_coarse(const T *r, int pitch, int rows, int nc, int dim, const double *G, T *v, const int *done, Bt B) {
    const int prob_ = bt_prob(B);
    if (stop(bt_done(done, prob_, B))) return;
    r = bt_ptr(r, prob_, B);
    v = bt_ptr(v, prob_, B);
    const int nn = dim == 2 ? nc * nc : nc * nc * nc;
    for (int q = threadIdx.x; q < nn; q += blockDim.x) {
        double s = 0.0;
        for (int t = 0; t < nn; t++) {
            const int i = t % nc + 1, j = (t / nc) % nc + 1, k = dim == 3 ? t / (nc * nc) + 1 : 0;
            s += G[(size_t)q * nn + t] * (double)r[((size_t)k * rows + j) * pitch + i];
        }
        const int i = q % nc + 1, j = (q / nc) % nc + 1, k = dim == 3 ? q / (nc * nc) + 1 : 0;
        v[((size_t)k * rows + j) * pitch + i] = (T)s;
    }
}

// gamma-cycles (Section 5 leaves them open): on the blue grid of a pair --
// an axis level of side n and spacing H -- the residual of the corrections
// accumulated so far, out = r - L v with the 5-point Laplacian, and the
// accumulation v_acc += v
template <typename T>
__global__ void k_gres_2d(const T *r, const T *v, T *out, int pitch, int n, T ih2, const int *done, Bt B) {
    const int prob_ = bt_prob(B);
    if (stop(bt_done(done, prob_, B))) return;
    MG_IDX2 const int i = tx + 1, j = ty + 1;
    if (i > n || j > n) return;
    const size_t c = (size_t)j * pitch + i;
    const T lap = (v[c + 1] + v[c - 1] + v[c + pitch] + v[c - pitch] - T(4) * v[c]) * ih2;
    out[c] = r[c] - lap;
}
template <typename T>
__global__ void k_acc_2d(const T *v, T *acc, int pitch, int n, int first, const int *done, Bt B) {
    const int prob_ = bt_prob(B);
    if (stop(bt_done(done, prob_, B))) return;
    MG_IDX2 const int i = tx + 1, j = ty + 1;
    if (i > n || j > n) return;
    const size_t c = (size_t)j * pitch + i;
    acc[c] = first ? v[c] : acc[c] + v[c];
}

template <typename T>
__global__ void k_gres_3d(const T *r, const T *v, T *out, int pitch, int rows, int n, T ih2, const int *done, Bt B) {
    const int prob_ = bt_prob(B);
    if (stop(bt_done(done, prob_, B))) return;
    MG_IDX3 const int i = tx + 1, j = ty + 1, k = tz + 1;
    if (i > n || j > n) return;
    const size_t pl = (size_t)pitch * rows, c = (size_t)k * pl + (size_t)j * pitch + i;
    const T lap = (v[c + 1] + v[c - 1] + v[c + pitch] + v[c - pitch] + v[c + pl] + v[c - pl] - T(6) * v[c]) * ih2;
    out[c] = r[c] - lap;
}
template <typename T>
__global__ void k_acc_3d(const T *v, T *acc, int pitch, int rows, int n, int first, const int *done, Bt B) {
    const int prob_ = bt_prob(B);
    if (stop(bt_done(done, prob_, B))) return;
    MG_IDX3 const int i = tx + 1, j = ty + 1, k = tz + 1;
    if (i > n || j > n) return;
    const size_t c = ((size_t)k * rows + j) * pitch + i;
    acc[c] = first ? v[c] : acc[c] + v[c];
}

// u += v on an axis level (only used when the finest grid is the coarsest)
template <typename T>
__global__ void k_add_axis(const T *v, int pitch, int rows, int n, int dim, double *u, int up, int urows,
                           const int *done, Bt B) {
    const int prob_ = bt_prob(B);
    if (stop(bt_done(done, prob_, B))) return;
    v = bt_ptr(v, prob_, B);
    if (B.utab) u = B.utab[prob_];
    MG_IDX3 const int i = tx + 1, j = ty + 1, k = dim == 3 ? tz + 1 : 0;
    if (i > n || j > n) return;
    u[((size_t)k * urows + j) * up + i] += (double)v[((size_t)k * rows + j) * pitch + i];
}

// Level import/export between a caller full grid of side s (pitch s+2, FP64)
// and the level's coset arrays.  kind: 0 axis, 1 red, 2 magenta.
template <typename T>
__global__ void k_level_io(int dim, int kind, int s, double *grid, T *c0, T *c1, T *c2, T *c3, int pitch, int rows,
                           int to_level) {
    pdl_wait();
    MG_IDX2 const int i = tx + 1, j = ty + 1, k = dim == 3 ? (int)blockIdx.z + 1 : 0;
    if (i > s || j > s || (dim == 3 && k > s)) return;
    const size_t gidx = ((size_t)k * (s + 2) + j) * (size_t)(s + 2) + i;
    T *arr = nullptr;
    int x = i, y = j, z = k;
    if (kind == 0) {
        arr = c0;
    } else {
        const int px = i & 1, py = j & 1, pz = k & 1;
        x = i >> 1; y = j >> 1; z = k >> 1;
        if (dim == 2) {
            if (px != py) return;
            arr = px ? c1 : c0;
        } else if (kind == 1) {
            if (((px + py + pz) & 1) != 0) return;
            arr = (px && py) ? c1 : px ? c2 : py ? c3 : c0;
        } else {
            if (!(px == py && py == pz)) return;
            arr = px ? c1 : c0;
        }
    }
    T &cell = arr[((size_t)z * rows + y) * pitch + x];
    if (to_level) cell = (T)grid[gidx];
    else grid[gidx] = (double)cell;
}

}  // namespace mg
