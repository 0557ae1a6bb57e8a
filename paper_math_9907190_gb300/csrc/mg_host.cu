// mg_host.cu -- C ABI (include/diagmg.h): context, level table and the
// launch schedule of the V-cycle.  All arithmetic runs in the kernels of
// mg_stages.cuh; this file only sizes buffers and launches.
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <new>
#include <algorithm>
#include <string>
#include <vector>

#include "../../include/diagmg.h"
#include "mg_stages.cuh"
#include "mg_fast3d.cuh"
#include "mg_fast2d.cuh"
#include "mg_cluster.cuh"

using namespace mg;

namespace {

thread_local char g_last_error[256] = "";

mg_status cuda_fail(cudaError_t e, const char *where) {
    std::snprintf(g_last_error, sizeof g_last_error, "%s: %s", where, cudaGetErrorString(e));
    return MG_ECUDA;
}
#define CK(call)                                               \
    do {                                                       \
        cudaError_t e_ = (call);                               \
        if (e_ != cudaSuccess) return cuda_fail(e_, #call);    \
    } while (0)
#define CKL(where)                                             \
    do {                                                       \
        cudaError_t e_ = cudaGetLastError();                   \
        if (e_ != cudaSuccess) return cuda_fail(e_, where);    \
    } while (0)

// a caller grid pointer the kernels can take: not null, on an FP64 element
// boundary (8 bytes; 16-byte vector paths are chosen only where the pointer
// and the pitch allow them)
bool bad_grid(const void *p) { return !p || ((uintptr_t)p & 7u) != 0; }
// two full grids of len doubles starting at a and b share memory
bool grids_overlap(const double *a, const double *b, size_t len) { return a < b + len && b < a + len; }

int log2_side(int n) {
    if (n < 1) return -1;
    long v = (long)n + 1;
    int m = 0;
    while ((v & 1) == 0) { v >>= 1; m++; }
    return v == 1 ? m : -1;
}

int round_up(int x, int m) { return (x + m - 1) / m * m; }

enum { KIND_AXIS = 0, KIND_RED = 1, KIND_MAG = 2 };

struct Level {
    int kind;      // KIND_*
    int side;      // side of the axis grid whose subscripts index this level
    int k;         // pair / triple / conventional level index (spacing h 2^k)
    int nb;        // coset arrays: (nb+2) entries per axis (diagonal levels)
    int pitch;     // elements per row of every array of this level
    int rows;      // rows per plane (3D)
    size_t len;    // elements per array
    int ncos;      // arrays per level (1 axis, 2 or 4 cosets)
    void *r[4];
    void *v[4];
};

}  // namespace

struct mg_ctx {
    mg_desc d;
    int m, K, L;        // log2(n+1), coarsenings, last level index
    double h;
    size_t esz;         // bytes per level element (8 FP64, 4 MIXED)
    std::vector<Level> lv;
    void *pool = nullptr;       // all level arrays
    double *part = nullptr;     // residual block partial sums
    int max_blocks = 0;
    Ctrl *ctl = nullptr;
    double *hist = nullptr;     // device history, length hist_cap
    int hist_cap = 0;
    double *G = nullptr;        // coarsest dense inverse
    double *scal = nullptr;     // device scalar for norms
    int dev = 0;
    int sms = 152;              // multiprocessors of the device
    // launch accounting and the optional event probe of one kernel family
    long long launches = 0;
    int probe_tag = -1;
    std::vector<cudaEvent_t> pev;  // start/end pairs
    int pev_used = 0;
    long long probe_n = 0;
    double probe_ms = 0.0;
    // fused 2D diagonal path
    bool fast2d = false;
    int kc = 0;                 // first pair run by the coarse thread block
    CoarsePlan2d plan2d{};
    size_t plan_bytes = 0;
    // 2D: the middle pairs kd..kc-1 in one thread-block cluster (distributed
    // shared memory), its first block running pairs kc.. as the coarse block
    bool cl = false;            // the cluster kernel is in use (kd < kc)
    int kd = 0;                 // first pair of the coarse kernel (cluster: kd; else kc)
    int cl_top = 0;             // largest green side of a distributed pair (0: no cluster; mg_tune, DIAGMG_CLUSTER)
    bool cl_ok = true;          // clusters of this kernel can run on the device (checked by mg_create)
    ClPlan2d plancl{};
    size_t cl_bytes = 0;
    // mixed path: finest pair (2D) / triple (3D) fused with the next residual,
    // carried as a float-float pair (hi in the finest level's residual buffers,
    // double-buffered with r32b; lo in rlo; green pitch, in the pool)
    bool rr = false;
    bool rr_alloc = false;  // the carried-residual buffers exist (rr is off while extra > 0)
    bool zstart = false;    // the solve being recorded or run starts from zero (mg_solve_zero, fused path)
    int extra = 0;          // extra Jacobi sweeps per level (mg_set_sweeps)
    int gamma = 1;          // coarse-problem cycles per pair (mg_set_gamma; 1: the V-cycle)
    void *wpool = nullptr;  // gamma > 1: per green level k >= 1, the kept residual and the accumulated correction
    std::vector<void *> wr, wv;
    void *rlo = nullptr;
    void *r32b = nullptr;
    // tuned choices (mg_tune): tile class per pair for the down / up kernels
    // (-1: the size rule), side cut-off of the coarse thread block (0: default)
    int tile_dn[32], tile_up[32];
    int gs_resident = 608;      // resident blocks of k_green_ff_3d on this device
    int cut_side = 0;
    // 3D diagonal path: triples with side <= 15 in one thread block
    bool fast3d = false;
    CoarsePlan3d plan3d{};
    double *ft = nullptr;       // order-4 right-hand side (caller pitch), FP64
    double *io_f = nullptr;     // device copies of f and u for mg_solve_host (allocated by its first call)
    double *io_u = nullptr;
    int nparts = 0;             // partial sums written by the last residual (per problem)
    // batch: nprob problems of this size, level pools pstride bytes apart,
    // f/u from device pointer tables (nullptr for a single problem)
    int nprob = 1;
    size_t pstride = 0;
    const double **ftab = nullptr;
    double **utab = nullptr;
    // the solver graph (prefix + device-driven loop over V-cycles), cached per arguments
    bool capturing = false;
    bool use_graph = true;      // DIAGMG_SOLVE_GRAPH=0: host-driven loop (same kernels; for profilers)
    bool pdl = false;           // programmatic dependent launch (default per configuration; DIAGMG_PDL=0/1)
    int pdl_max_blocks = 0;     // > 0: only for grids of at most this many blocks (DIAGMG_PDL_MAX_BLOCKS)
    cudaStream_t cs1 = nullptr, cs2 = nullptr;
    // fused mixed path: recorded once the last cycle has written u (before the
    // direct residual that closes a solve), so that mg_solve_host copies u
    // back while that residual runs, on its own stream cs_io
    cudaEvent_t ev_ufinal = nullptr, ev_io = nullptr;
    cudaStream_t cs_io = nullptr;
    // mg_solve_host_many: the second pair of device copies and the events of
    // its two-buffer pipeline; Ctrl of the last two solves in page-locked memory
    double *io_f2 = nullptr, *io_u2 = nullptr;
    cudaEvent_t ev_in[2] = {}, ev_sol[2] = {}, ev_out[2] = {}, ev_ctl[2] = {};
    Ctrl *hctl = nullptr;
    // instantiated solve graphs, keyed by their arguments and the context's
    // settings; a few are kept (least recently used replaced) so that a caller
    // alternating between buffers does not rebuild a graph per solve
    struct SolveGraph {
        cudaGraph_t graph = nullptr;
        cudaGraphExec_t exec = nullptr;
        const double *f = nullptr;
        double *u = nullptr;
        double rtol = -1.0;
        int max = -1, order = 0, extra = 0, gamma = 1;
        bool zero = false;  // a solve from zero (mg_solve_zero)
        double omega[4] = {0, 0, 0, 0};
        long long prefix_kernels = 0, body_kernels = 0;  // launches of the prefix and of one cycle
        unsigned long long used = 0;
    };
    SolveGraph gcache[4];
    unsigned long long gtick = 0;
    long long g_prefix_kernels = 0, g_body_kernels = 0;  // of the last capture
};

static void drop_solve_graph(mg_ctx::SolveGraph &e) {
    if (e.exec) cudaGraphExecDestroy(e.exec);
    if (e.graph) cudaGraphDestroy(e.graph);
    e = mg_ctx::SolveGraph{};
}
static void drop_solve_graphs(mg_ctx *c) {
    for (auto &e : c->gcache) drop_solve_graph(e);
}

namespace {

// ---- geometry -------------------------------------------------------------

void build_levels(mg_ctx *c) {
    const int dim = c->d.dim;
    const int cm = log2_side(c->d.coarsest);
    c->K = c->m - cm;
    auto axis = [&](int k) {
        Level l{};
        l.kind = KIND_AXIS;
        l.k = k;
        l.side = (1 << (c->m - k)) - 1;
        l.nb = 0;
        l.pitch = round_up(l.side + 2, 32);
        l.rows = l.side + 2;
        l.len = (size_t)l.pitch * l.rows * (dim == 3 ? (size_t)l.rows : 1);
        l.ncos = 1;
        return l;
    };
    auto coset = [&](int k, int kind) {
        Level l{};
        l.kind = kind;
        l.k = k;
        l.side = (1 << (c->m - k)) - 1;
        l.nb = (l.side - 1) / 2;
        l.pitch = round_up(l.nb + 2, 32);
        l.rows = l.nb + 2;
        l.len = (size_t)l.pitch * l.rows * (dim == 3 ? (size_t)l.rows : 1);
        l.ncos = (dim == 3 && kind == KIND_RED) ? 4 : 2;
        return l;
    };
    c->lv.clear();
    for (int k = 0; k < c->K; k++) {
        c->lv.push_back(axis(k));
        if (c->d.hierarchy == MG_DIAG) {
            c->lv.push_back(coset(k, KIND_RED));
            if (dim == 3) c->lv.push_back(coset(k, KIND_MAG));
        }
    }
    c->lv.push_back(axis(c->K));
    c->L = (int)c->lv.size() - 1;
}

// dense inverse of the 5/7-point operator on the coarsest grid (side s,
// spacing H) from its sine eigenbasis: G = S diag(1/lambda) S, S orthonormal
std::vector<double> coarse_inverse(int dim, int s, double H) {
    const int nn = dim == 2 ? s * s : s * s * s;
    std::vector<double> S((size_t)s * s), lam1(s), G((size_t)nn * nn, 0.0);
    const double pi = 3.14159265358979323846;
    for (int p = 0; p < s; p++) {
        lam1[p] = -4.0 / (H * H) * std::pow(std::sin((p + 1) * pi / (2.0 * (s + 1))), 2);
        for (int i = 0; i < s; i++) S[(size_t)i * s + p] = std::sqrt(2.0 / (s + 1)) * std::sin((i + 1) * (p + 1) * pi / (s + 1));
    }
    const int nm = nn;
    for (int q = 0; q < nn; q++) {
        const int qi = q % s, qj = (q / s) % s, qk = dim == 3 ? q / (s * s) : 0;
        for (int t = 0; t < nn; t++) {
            const int ti = t % s, tj = (t / s) % s, tk = dim == 3 ? t / (s * s) : 0;
            double acc = 0.0;
            for (int mode = 0; mode < nm; mode++) {
                const int pi_ = mode % s, pj = (mode / s) % s, pk = dim == 3 ? mode / (s * s) : 0;
                double lam = lam1[pi_] + lam1[pj] + (dim == 3 ? lam1[pk] : 0.0);
                double w = S[(size_t)qi * s + pi_] * S[(size_t)ti * s + pi_] * S[(size_t)qj * s + pj] * S[(size_t)tj * s + pj];
                if (dim == 3) w *= S[(size_t)qk * s + pk] * S[(size_t)tk * s + pk];
                acc += w / lam;
            }
            G[(size_t)q * nn + t] = acc;
        }
    }
    return G;
}

// ---- launch helpers -------------------------------------------------------

inline cudaStream_t S(void *s) { return (cudaStream_t)s; }

// kernel families for the probe (mg_probe_set)
enum { TAG_RESIDUAL = 0, TAG_FINEST_UP = 1, TAG_LEVELS = 2, TAG_CONTROL = 3 };
// sub-families of TAG_LEVELS (probed as 4, 5, 6): restriction, prolongation
// of the coarser levels, the coarse thread block
enum { TAG_DOWN = TAG_LEVELS | 4 << 4, TAG_UP = TAG_LEVELS | 5 << 4, TAG_COARSE = TAG_LEVELS | 6 << 4 };

// Counts every launch; brackets the launch with events when its family is probed.
struct Launch {
    mg_ctx *c;
    cudaStream_t s;
    int slot = -1;
    Launch(mg_ctx *c_, int tag, cudaStream_t s_) : c(c_), s(s_) {
        c->launches++;
        const bool hit = c->probe_tag >= 0 && (c->probe_tag == (tag & 15) || ((tag >> 4) && c->probe_tag == tag >> 4));
        if (!c->capturing && hit && 2 * c->pev_used + 1 < (int)c->pev.size()) {
            slot = c->pev_used++;
            cudaEventRecord(c->pev[2 * slot], s);
        }
    }
    ~Launch() {
        if (slot >= 0) cudaEventRecord(c->pev[2 * slot + 1], s);
    }
};
// One kernel launch; with c->pdl, as a programmatic dependent launch: the
// kernel may be scheduled while the previous one in the stream finishes and
// waits in pdl_wait (every kernel of this library calls it before reading
// what another kernel wrote).
template <typename... P, typename... A>
void launch_k(const mg_ctx *c, void (*kern)(P...), dim3 g, dim3 b, size_t sm, cudaStream_t s, A &&...args) {
    cudaLaunchConfig_t cfg{};
    cfg.gridDim = g;
    cfg.blockDim = b;
    cfg.dynamicSmemBytes = sm;
    cfg.stream = s;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = at;
    const long long nblk = (long long)g.x * g.y * g.z;
    cfg.numAttrs = c->pdl && (c->pdl_max_blocks <= 0 || nblk <= c->pdl_max_blocks) ? 1 : 0;
    cudaLaunchKernelEx(&cfg, kern, std::forward<A>(args)...);
}
#define LAUNCH(tag, kern, grid, block, ...)                                \
    do {                                                                   \
        Launch l_(c, tag, s);                                              \
        launch_k(c, kern, dim3(grid), dim3(block), 0, s, __VA_ARGS__);     \
    } while (0)

#define LAUNCH_SMEM(tag, kern, grid, block, smem, ...)                     \
    do {                                                                   \
        Launch l_(c, tag, s);                                              \
        launch_k(c, kern, dim3(grid), dim3(block), smem, s, __VA_ARGS__);  \
    } while (0)

// grid and batch descriptor of one launch: z blocks of one problem, times nprob
struct BL {
    dim3 dims;
    Bt bt;
};
BL bl(const mg_ctx *c, dim3 g) {
    Bt b{c->pstride, (int)g.z, (int)(sizeof(Ctrl) / sizeof(int)), (int)(g.x * g.y * g.z), c->ftab, c->utab};
    g.z *= (unsigned)c->nprob;
    return BL{g, b};
}
#define LAUNCH_B(tag, kern, grd, block, ...)                                   \
    do {                                                                       \
        BL bl_ = bl(c, grd);                                                   \
        Launch l_(c, tag, s);                                                  \
        launch_k(c, kern, bl_.dims, dim3(block), 0, s, __VA_ARGS__, bl_.bt);   \
    } while (0)
#define LAUNCH_SMEM_B(tag, kern, grd, block, smem, ...)                        \
    do {                                                                       \
        BL bl_ = bl(c, grd);                                                   \
        Launch l_(c, tag, s);                                                  \
        launch_k(c, kern, bl_.dims, dim3(block), smem, s, __VA_ARGS__, bl_.bt); \
    } while (0)

// accumulate the probe events of completed work (call after a stream sync)
void probe_collect(mg_ctx *c) {
    for (int q = 0; q < c->pev_used; q++) {
        float ms = 0.f;
        if (cudaEventElapsedTime(&ms, c->pev[2 * q], c->pev[2 * q + 1]) == cudaSuccess) {
            c->probe_ms += ms;
            c->probe_n += 1;
        }
    }
    c->pev_used = 0;
}

dim3 grid2(int nx, int ny) { return dim3((nx + 31) / 32, (ny + 7) / 8, 1); }
dim3 grid3(int nx, int ny, int nz) { return dim3((nx + 31) / 32, (ny + 7) / 8, nz); }
// planes per thread of the z-marching 3D stage kernels by size: 8 from 128^3
// cells, 2 from 64^3; smaller triples, and the FP64 path (bound by its FP64
// arithmetic), use the thread-per-cell kernels
int zm_planes(int nb) { return nb + 1 >= 128 ? 8 : 2; }
template <typename T> bool zm_use(int nb) { return sizeof(T) == 4 && nb + 1 >= 64; }
// grid of a z-marching 3D stage kernel: count cells per dimension
dim3 grid_zm(int count, int zm) { return dim3((count + 31) / 32, (count + 7) / 8, (count + zm - 1) / zm); }
const dim3 B2(32, 8, 1);

template <typename T> A2<T> a2(void *p, const Level &l) { return A2<T>{(T *)p, l.pitch}; }
template <typename T> A3<T> a3(void *p, const Level &l) { return A3<T>{(T *)p, l.pitch, l.rows}; }
template <typename T> Red3<T> red3v(void *const *p, const Level &l) {
    return Red3<T>{a3<T>(p[0], l), a3<T>(p[1], l), a3<T>(p[2], l), a3<T>(p[3], l)};
}
template <typename T> Mag3<T> mag3v(void *const *p, const Level &l) { return Mag3<T>{a3<T>(p[0], l), a3<T>(p[1], l)}; }

double spacing(const mg_ctx *c, const Level &l) { return c->h * (double)(1 << l.k); }

// residual of the finest grid into level 0 (+ optional FP64 copy, partials)
template <typename T>
void launch_residual(mg_ctx *c, const double *f, const double *u, double *r64, bool rhs_only, const int *done,
                     cudaStream_t s) {
    const Level &l0 = c->lv[0];
    const int n = c->d.n;
    const double ih2 = 1.0 / (c->h * c->h);
    if (c->d.dim == 2) {
        dim3 g = grid2(n, n);
        auto r = a2<T>(l0.r[0], l0);
        if (c->d.order == 2) {
            if (rhs_only) LAUNCH_B(TAG_RESIDUAL, (k_res_2d<T, 2, true>), g, B2, f, u, c->d.pitch, n, ih2, r, r64, c->part, done);
            else LAUNCH_B(TAG_RESIDUAL, (k_res_2d<T, 2, false>), g, B2, f, u, c->d.pitch, n, ih2, r, r64, c->part, done);
        } else {
            if (rhs_only) LAUNCH_B(TAG_RESIDUAL, (k_res_2d<T, 4, true>), g, B2, f, u, c->d.pitch, n, ih2, r, r64, c->part, done);
            else LAUNCH_B(TAG_RESIDUAL, (k_res_2d<T, 4, false>), g, B2, f, u, c->d.pitch, n, ih2, r, r64, c->part, done);
        }
    } else {
        dim3 g = grid3(n, n, n);
        auto r = a3<T>(l0.r[0], l0);
        const int ur = n + 2;
        if (c->d.order == 2) {
            if (rhs_only) LAUNCH_B(TAG_RESIDUAL, (k_res_3d<T, 2, true>), g, B2, f, u, c->d.pitch, ur, n, ih2, r, r64, c->part, done);
            else LAUNCH_B(TAG_RESIDUAL, (k_res_3d<T, 2, false>), g, B2, f, u, c->d.pitch, ur, n, ih2, r, r64, c->part, done);
        } else {
            if (rhs_only) LAUNCH_B(TAG_RESIDUAL, (k_res_3d<T, 4, true>), g, B2, f, u, c->d.pitch, ur, n, ih2, r, r64, c->part, done);
            else LAUNCH_B(TAG_RESIDUAL, (k_res_3d<T, 4, false>), g, B2, f, u, c->d.pitch, ur, n, ih2, r, r64, c->part, done);
        }
    }
}

int residual_blocks(const mg_ctx *c) {
    const int n = c->d.n;
    dim3 g = c->d.dim == 2 ? grid2(n, n) : grid3(n, n, n);
    return (int)(g.x * g.y * g.z);
}

// restriction r^(l+1) <- r^(l)
template <typename T> void launch_restrict(mg_ctx *c, int l, const int *done, cudaStream_t s, bool alt = false) {
    const Level &a = c->lv[l], &b = c->lv[l + 1];
    if (c->d.hierarchy == MG_USUAL) {
        const int nc = b.side;
        if (c->d.dim == 2) LAUNCH_B(TAG_DOWN, (k_fw_2d<T>), grid2(nc, nc), B2, a2<const T>(a.r[0], a), a2<T>(b.r[0], b), nc, done);
        else LAUNCH_B(TAG_DOWN, (k_fw_3d<T>), grid3(nc, nc, nc), B2, a3<const T>(a.r[0], a), a3<T>(b.r[0], b), nc, done);
        return;
    }
    if (c->d.dim == 2) {
        if (a.kind == KIND_AXIS) {
            const int nb = b.nb;
            LAUNCH_B(TAG_DOWN, (k_g2r_2d<T>), grid2(nb + 1, nb + 1), B2, a2<const T>(a.r[0], a), a2<T>(b.r[0], b), a2<T>(b.r[1], b), nb, done);
        } else {
            const int nb = a.nb;
            LAUNCH_B(TAG_DOWN, (k_r2b_2d<T>), grid2(nb, nb), B2, a2<const T>(a.r[0], a), a2<const T>(a.r[1], a), a2<T>(b.r[0], b), nb, done);
        }
        return;
    }
    if (a.kind == KIND_AXIS) {
        const int nb = b.nb;
        const T *galt = (alt && l == 0 && c->rr) ? (const T *)c->r32b : nullptr;
        const int *par = galt ? &c->ctl->par : nullptr;
        if (zm_use<T>(nb))
            LAUNCH_B(TAG_DOWN, (k_g2r_zm_3d<T>), grid_zm(nb + 1, zm_planes(nb)), B2, a3<const T>(a.r[0], a), red3v<T>(b.r, b), nb,
                     galt, par, zm_planes(nb), done);
        else
            LAUNCH_B(TAG_DOWN, (k_g2r_3d<T>), grid3(nb + 1, nb + 1, nb + 1), B2, a3<const T>(a.r[0], a), red3v<T>(b.r, b), nb,
                     galt, par, done);
    } else if (a.kind == KIND_RED) {
        const int nb = a.nb;
        if (zm_use<T>(nb))
            LAUNCH_B(TAG_DOWN, (k_r2m_zm_3d<T>), grid_zm(nb + 1, zm_planes(nb)), B2, red3v<const T>(a.r, a), mag3v<T>(b.r, b), nb, zm_planes(nb), done);
        else
            LAUNCH_B(TAG_DOWN, (k_r2m_3d<T>), grid3(nb + 1, nb + 1, nb + 1), B2, red3v<const T>(a.r, a), mag3v<T>(b.r, b), nb, done);
    } else {
        const int nb = a.nb;
        if (zm_use<T>(nb))
            LAUNCH_B(TAG_DOWN, (k_m2b_zm_3d<T>), grid_zm(nb, zm_planes(nb)), B2, mag3v<const T>(a.r, a), a3<T>(b.r[0], b), nb, zm_planes(nb), done);
        else
            LAUNCH_B(TAG_DOWN, (k_m2b_3d<T>), grid3(nb, nb, nb), B2, mag3v<const T>(a.r, a), a3<T>(b.r[0], b), nb, done);
    }
}

// z range (output planes per block) of k_green_ff_3d: the grid fills the
// resident block slots once (a second, partial wave would double the time of
// a launch), at least 4 planes
int green_ff_zch(const mg_ctx *c, int n) {
    const int cols = ((n + GS_TX - 1) / GS_TX) * ((n + GS_TY - 1) / GS_TY);
    const int chunks = std::max(1, c->gs_resident / (cols * c->nprob));
    return std::max(4, (n + chunks - 1) / chunks);
}
dim3 green_ff_grid(const mg_ctx *c, int n) {
    const int zch = green_ff_zch(c, n);
    return dim3((n + GS_TX - 1) / GS_TX, (n + GS_TY - 1) / GS_TY, (n + zch - 1) / zch);
}
// vector access to u in k_green_ff_3d: one problem, u 16-byte aligned, even pitch
bool green_ff_vu(const mg_ctx *c, const double *u) {
    return c->nprob == 1 && ((uintptr_t)u % 16) == 0 && c->d.pitch % 2 == 0;
}
// the z-streaming green sweep pays GS_WARM steps per z range; measured faster
// than the 3D tile kernel from 31^3 up
bool green_ff_use(int n) { return n >= 31; }

// prolongation v^(l) <- v^(l+1), r^(l); on level 0 with u != nullptr the
// second half-sweep also applies u += v.  vctl: the red level of the fused
// mixed path's finest triple also gets its bound on |v| (ctl->vmax)
template <typename T>
void launch_prolong(mg_ctx *c, int l, const double *om, double *u, const int *done, cudaStream_t s,
                    Ctrl *vctl = nullptr) {
    const Level &a = c->lv[l], &b = c->lv[l + 1];
    const double hk = spacing(c, a), hk2 = hk * hk;
    const int dim = c->d.dim;
    if (a.kind == KIND_AXIS) {
        // green-red sweep (diagonal) or interpolation + red-black sweep (conventional)
        const int n = a.side;
        const double p = (dim == 3 && c->d.hierarchy == MG_DIAG) ? om[3] : om[0];
        const T cc = (T)(p * hk2);
        if (dim == 2) {
            if (c->d.hierarchy == MG_USUAL)
                LAUNCH_B(TAG_UP, (k_usual_odd_2d<T>), grid2(n, n), B2, a2<const T>(b.v[0], b), a2<const T>(a.r[0], a), a2<T>(a.v[0], a), n, cc, done);
            else
                LAUNCH_B(TAG_UP, (k_r2g_f_2d<T>), grid2(n, n), B2, a2<const T>(b.v[0], b), a2<const T>(b.v[1], b), a2<const T>(a.r[0], a), a2<T>(a.v[0], a), n, cc, done);
            // extra sweeps (diagonal hierarchy): green-only points from the
            // level's own red points, then the red points; u += v after the last
            const int extra = c->d.hierarchy == MG_DIAG ? c->extra : 0;
            for (int e = 0; e <= extra; e++) {
                if (e > 0)
                    LAUNCH_B(TAG_UP, (k_g2g_f_2d<T>), grid2(n, n), B2, a2<const T>(a.r[0], a), a2<T>(a.v[0], a), n, cc, done);
                if (u && e == extra)
                    LAUNCH_B(TAG_FINEST_UP, (k_r2g_c_upd_2d<T>), grid2(n, n), B2, a2<const T>(a.r[0], a), a2<const T>(a.v[0], a), u, c->d.pitch, n, cc, done);
                else
                    LAUNCH_B(TAG_UP, (k_r2g_c_2d<T>), grid2(n, n), B2, a2<const T>(a.r[0], a), a2<T>(a.v[0], a), n, cc, done);
            }
        } else if (c->d.hierarchy == MG_DIAG && sizeof(T) == 4 && green_ff_use(n)) {  // FP32, z-streaming
            const dim3 g3 = green_ff_grid(c, n);
            const size_t sm = sizeof(GreenSSmem);
            const int zch = green_ff_zch(c, n);
#define MG_GFF(TAG, MODE, VU)                                                                                     \
    LAUNCH_SMEM_B(TAG, (k_green_ff_3d<MODE, VU>), g3, dim3(32, 8, 1), sm, red3v<const float>(b.v, b),               \
                  a3<float>(a.r[0], a), (float *)nullptr, a3<float>(a.v[0], a), (float *)nullptr, u, c->d.pitch, n, \
                  (float)cc, 0.f, zch, (double *)nullptr, (Ctrl *)nullptr, CtrlFuse{}, done)
            if (u && green_ff_vu(c, u)) MG_GFF(TAG_FINEST_UP, UP_ADD, true);
            else if (u) MG_GFF(TAG_FINEST_UP, UP_ADD, false);
            else MG_GFF(TAG_UP, UP_STORE, false);
#undef MG_GFF
        } else if (c->d.hierarchy == MG_DIAG && sizeof(T) == 4) {  // FP32: both half-sweeps in one tile kernel
            const dim3 g3((n + TX3 - 1) / TX3, (n + TY3 - 1) / TY3, (n + TZ3 - 1) / TZ3);
            const size_t sm = sizeof(Green3Smem<T>);
            if (u)
                LAUNCH_SMEM_B(TAG_FINEST_UP, (k_green_3d<T, true>), g3, B2, sm, red3v<const T>(b.v, b),
                              a3<const T>(a.r[0], a), a3<T>(a.v[0], a), u, c->d.pitch, n, cc, done);
            else
                LAUNCH_SMEM_B(TAG_UP, (k_green_3d<T, false>), g3, B2, sm, red3v<const T>(b.v, b),
                              a3<const T>(a.r[0], a), a3<T>(a.v[0], a), u, c->d.pitch, n, cc, done);
        } else {
            if (c->d.hierarchy == MG_USUAL)
                LAUNCH_B(TAG_UP, (k_usual_odd_3d<T>), grid3(n, n, n), B2, a3<const T>(b.v[0], b), a3<const T>(a.r[0], a), a3<T>(a.v[0], a), n, cc, done);
            else
                LAUNCH_B(TAG_UP, (k_r2g_f_3d<T>), grid3(n, n, n), B2, red3v<const T>(b.v, b), a3<const T>(a.r[0], a), a3<T>(a.v[0], a), n, cc, done);
            if (u)
                LAUNCH_B(TAG_FINEST_UP, (k_r2g_c_upd_fast_3d<T>), grid3(n, n, n), B2, a3<const T>(a.r[0], a), a3<const T>(a.v[0], a), u, c->d.pitch, n + 2, n, cc, done);
            else
                LAUNCH_B(TAG_UP, (k_r2g_c_3d<T>), grid3(n, n, n), B2, a3<const T>(a.r[0], a), a3<T>(a.v[0], a), n, cc, done);
        }
        return;
    }
    const int nb = a.nb;
    if (dim == 2) {  // red level from the blue (next axis) level, Eq. Eajacr, Eq. Eajacb
        const T cc = (T)(2.0 * om[0] * hk2);
        LAUNCH_B(TAG_UP, (k_b2r_oo_2d<T>), grid2(nb + 1, nb + 1), B2, a2<const T>(b.v[0], b), a2<const T>(a.r[1], a), a2<T>(a.v[1], a), nb, cc, done);
        LAUNCH_B(TAG_UP, (k_b2r_ee_2d<T>), grid2(nb, nb), B2, a2<const T>(a.v[1], a), a2<const T>(a.r[0], a), a2<T>(a.v[0], a), nb, cc, done);
        // extra sweeps: the not-blue points (OO) from the level's own blue
        // points (EE, the same (a, b) indexing and layout as the blue level),
        // then the blue points
        for (int e = 0; e < c->extra; e++) {
            LAUNCH_B(TAG_UP, (k_b2r_oo_2d<T>), grid2(nb + 1, nb + 1), B2, a2<const T>(a.v[0], a), a2<const T>(a.r[1], a), a2<T>(a.v[1], a), nb, cc, done);
            LAUNCH_B(TAG_UP, (k_b2r_ee_2d<T>), grid2(nb, nb), B2, a2<const T>(a.v[1], a), a2<const T>(a.r[0], a), a2<T>(a.v[0], a), nb, cc, done);
        }
        return;
    }
    if (a.kind == KIND_MAG) {  // Eq. Emprolm, Eq. Emprolb
        const T cc = (T)(4.0 * om[0] * hk2);
        if (zm_use<T>(nb)) {
            LAUNCH_B(TAG_UP, (k_b2m_ooo_zm_3d<T>), grid_zm(nb + 1, zm_planes(nb)), B2, a3<const T>(b.v[0], b), a3<const T>(a.r[1], a), a3<T>(a.v[1], a), nb, cc, zm_planes(nb), done);
            LAUNCH_B(TAG_UP, (k_b2m_eee_zm_3d<T>), grid_zm(nb, zm_planes(nb)), B2, a3<const T>(a.v[1], a), a3<const T>(a.r[0], a), a3<T>(a.v[0], a), nb, cc, zm_planes(nb), done);
        } else if (nb + 1 <= 32) {  // small levels: both half-sweeps in one launch, a tile of cells per block
            const dim3 g((nb + BM_X) / BM_X, (nb + BM_Y) / BM_Y, (nb + BM_Z) / BM_Z);
            LAUNCH_B(TAG_UP, (k_b2m_3d<T>), g, B2, a3<const T>(b.v[0], b), a3<const T>(a.r[1], a), a3<const T>(a.r[0], a),
                     a3<T>(a.v[1], a), a3<T>(a.v[0], a), nb, cc, done);
        } else {
            LAUNCH_B(TAG_UP, (k_b2m_ooo_3d<T>), grid3(nb + 1, nb + 1, nb + 1), B2, a3<const T>(b.v[0], b), a3<const T>(a.r[1], a), a3<T>(a.v[1], a), nb, cc, done);
            LAUNCH_B(TAG_UP, (k_b2m_eee_3d<T>), grid3(nb, nb, nb), B2, a3<const T>(a.v[1], a), a3<const T>(a.r[0], a), a3<T>(a.v[0], a), nb, cc, done);
        }
    } else {  // red from magenta: Eq. Erprolr (faces), Eq. Erprolm (corners)
        const T c1 = (T)(2.0 * om[1] * hk2), c2 = (T)(4.0 * om[2] * hk2);
        if (zm_use<T>(nb)) {
            LAUNCH_B(TAG_UP, (k_m2r_faces_zm_3d<T>), grid_zm(nb + 1, zm_planes(nb)), B2, mag3v<const T>(b.v, b), red3v<const T>(a.r, a), red3v<T>(a.v, a), nb, c1, zm_planes(nb), done);
            LAUNCH_B(TAG_UP, (k_m2r_corners_zm_3d<T>), grid_zm(nb, zm_planes(nb)), B2, red3v<const T>(a.v, a), a3<const T>(a.r[0], a), a3<T>(a.v[0], a), nb, c2, zm_planes(nb), vctl, done);
        } else if (nb + 1 <= 32 && !vctl) {  // small levels: both half-sweeps in one launch
            const dim3 g((nb + BM_X) / BM_X, (nb + BM_Y) / BM_Y, (nb + BM_Z) / BM_Z);
            LAUNCH_B(TAG_UP, (k_m2r_3d<T>), g, B2, mag3v<const T>(b.v, b), red3v<const T>(a.r, a), red3v<T>(a.v, a), nb,
                     c1, c2, done);
        } else {
            LAUNCH_B(TAG_UP, (k_m2r_faces_3d<T>), grid3(nb + 1, nb + 1, nb + 1), B2, mag3v<const T>(b.v, b), red3v<const T>(a.r, a), red3v<T>(a.v, a), nb, c1, done);
            LAUNCH_B(TAG_UP, (k_m2r_corners_3d<T>), grid3(nb, nb, nb), B2, red3v<const T>(a.v, a), a3<const T>(a.r[0], a), a3<T>(a.v[0], a), nb, c2, vctl, done);
        }
    }
}

template <typename T> void launch_coarse(mg_ctx *c, const int *done, cudaStream_t s) {
    const Level &l = c->lv[c->L];
    LAUNCH_B(TAG_COARSE, (k_coarse<T>), dim3(1, 1, 1), 512, (const T *)l.r[0], l.pitch, l.rows, l.side, c->d.dim, c->G, (T *)l.v[0], done);
}

// ---- fused 2D diagonal path ------------------------------------------------

// shared memory of a coarse block: `elems` level elements, then (16-byte
// aligned) the copy of the coarsest inverse, nn x nn doubles, and the
// coarsest right-hand side as a dense vector of nn doubles
static_assert(49 * 49 <= CTA_G_MAX, "coarsest inverse of a 7 x 7 grid");
void coarse_g_slot(mg_ctx *c, int nn, int elems, int &gofs, int &ng) {
    const size_t base = ((size_t)elems * c->esz + 15) / 16 * 16;
    ng = nn * nn;  // the coarsest grid has side <= 7 (2D) / 3 (3D) (valid_desc)
    gofs = (int)base;
    c->plan_bytes = base + (size_t)(ng + nn) * sizeof(double);
}

// the largest dynamic shared memory a block may use on this device
size_t smem_optin(const mg_ctx *c) {
    int v = 0;
    cudaDeviceGetAttribute(&v, cudaDevAttrMaxSharedMemoryPerBlockOptin, c->dev);
    return v > 0 ? (size_t)v : 48 * 1024;
}

// The cluster kernel's plan: pairs kd..kc-1 split by rows over CL2 blocks
// (each array: its band of R rows, R = (side + 1) / 8, plus two halo rows),
// then block 0's own plan (c->plan2d, c->plan_bytes).  Returns the dynamic
// shared memory per block, 0 if the pairs do not fit.
size_t plan_cl2d(mg_ctx *c, int kd, int kc) {
    ClPlan2d &P = c->plancl;
    P = ClPlan2d{};
    P.nd = kc - kd;
    int off = 0;
    auto take = [&](int rows, int pitch) {
        DistArr A{off, pitch, rows};
        off += ((rows + 2) * pitch + 3) / 4 * 4;
        return A;
    };
    for (int i = 0; i <= P.nd; i++) {
        const int n = c->lv[2 * (kd + i)].side, R = (n + 1) / CL2, nb = (n - 1) / 2;
        P.nk[i] = n;
        P.gr[i] = take(R, n + 2);
        P.gv[i] = take(R, n + 2);
        if (i < P.nd) {
            P.er[i] = take(R / 2, nb + 2); P.orr[i] = take(R / 2, nb + 2);
            P.ev[i] = take(R / 2, nb + 2); P.ov[i] = take(R / 2, nb + 2);
            const double hk = c->h * (double)(1 << (kd + i));
            P.c2[i] = 2.0 * c->d.omega[0] * hk * hk;
            P.c1[i] = c->d.omega[0] * hk * hk;
        }
    }
    P.doff = (int)(((size_t)off * c->esz + 15) / 16 * 16 / c->esz);
    P.cta = c->plan2d;
    const size_t bytes = (size_t)P.doff * c->esz + c->plan_bytes;
    return bytes <= smem_optin(c) ? bytes : 0;
}

void plan_fast2d(mg_ctx *c) {
    c->fast2d = c->d.dim == 2 && c->d.hierarchy == MG_DIAG && c->extra == 0 && c->gamma == 1;
    if (!c->fast2d) return;
    // pairs whose green grid has side <= 63 (FP64 levels: 15, where the one
    // block's FP64 arithmetic costs more than the launches it saves; or the
    // tuned cut-off; 31 below a cluster) run in one thread block
    const bool want_cl = c->cl_ok && c->cl_top >= 15;
    const int cut = c->cut_side > 0 ? c->cut_side : (want_cl ? 31 : c->esz == 8 ? 15 : 63);
    int kc = 0;
    while (kc < c->K && c->lv[2 * kc].side > cut) kc++;
    c->kc = kc;
    CoarsePlan2d &P = c->plan2d;
    P = CoarsePlan2d{};
    P.kc = kc;
    P.K = c->K;
    int off = 0;
    auto take = [&](int elems) { int o = off; off += (elems + 3) / 4 * 4; return o; };
    const int npair = c->K - kc;
    for (int p = 0; p <= npair; p++) {
        const int n = c->lv[2 * (kc + p)].side;
        P.nk[p] = n;
        P.og_r[p] = take((n + 2) * (n + 2));
        P.og_v[p] = take((n + 2) * (n + 2));
        if (p < npair) {
            const int nb = (n - 1) / 2, e = (nb + 2) * (nb + 2);
            P.oe_r[p] = take(e); P.oo_r[p] = take(e); P.oe_v[p] = take(e); P.oo_v[p] = take(e);
            const double hk = c->h * (double)(1 << (kc + p));
            P.c2[p] = 2.0 * c->d.omega[0] * hk * hk;
            P.c1[p] = c->d.omega[0] * hk * hk;
        }
    }
    P.total = off;
    coarse_g_slot(c, P.nk[npair] * P.nk[npair], off, P.gofs, P.ng);
    // pairs above the coarse block with green side <= cl_top (at least 15 and
    // block 0's first pair at least 7, so that every band has rows) in the
    // cluster; the finest pair of the fused mixed solve stays outside it
    c->cl = false;
    c->kd = kc;
    c->cl_bytes = 0;
    if (want_cl && kc < c->K && c->lv[2 * kc].side >= 7) {
        int kd = 0;
        while (kd < kc && (c->lv[2 * kd].side > c->cl_top || (kd == 0 && c->rr))) kd++;
        while (kd < kc && c->lv[2 * (kc - 1)].side >= 15) {
            const size_t bytes = plan_cl2d(c, kd, kc);
            if (bytes) { c->cl = true; c->kd = kd; c->cl_bytes = bytes; break; }
            kd++;  // the largest pair does not fit in shared memory: leave it to the pair kernels
        }
    }
}

// finest residual for every configuration: column (2D) / plane (3D) marching,
// FP64 stencil, level-precision output, FP32 squares in mixed precision
void plan_fast3d(mg_ctx *c) {
    // the coarse block keeps the coarsest inverse in shared memory: 3^3 grids
    // at most (a 7^3 coarsest grid runs with per-stage kernels and k_coarse)
    c->fast3d = c->d.dim == 3 && c->d.hierarchy == MG_DIAG && c->d.coarsest <= 3 && c->gamma == 1;
    if (!c->fast3d) return;
    // triples whose green side is <= 15 (FP64 levels: 7, where the one
    // block's FP64 arithmetic costs more than the launches it saves; or the
    // tuned cut-off) run in one thread block
    const int cut = c->cut_side > 0 ? c->cut_side : c->esz == 8 ? 7 : 15;
    int kc = 0;
    while (kc < c->K && c->lv[3 * kc].side > cut) kc++;
    c->kc = kc;
    CoarsePlan3d &P = c->plan3d;
    P = CoarsePlan3d{};
    P.kc = kc;
    P.K = c->K;
    int off = 0;
    auto take = [&](int elems) { int o = off; off += (elems + 3) / 4 * 4; return o; };
    const int ntri = c->K - kc;
    for (int t = 0; t <= ntri; t++) {
        const int n = c->lv[3 * (kc + t)].side, g = (n + 2) * (n + 2) * (n + 2);
        P.nk[t] = n;
        P.og_r[t] = take(g);
        P.og_v[t] = take(g);
        if (t < ntri) {
            const int nb = (n - 1) / 2, e = (nb + 2) * (nb + 2) * (nb + 2);
            for (int q = 0; q < 4; q++) { P.orr[t][q] = take(e); P.orv[t][q] = take(e); }
            for (int q = 0; q < 2; q++) { P.omr[t][q] = take(e); P.omv[t][q] = take(e); }
            const double hk = c->h * (double)(1 << (kc + t)), h2 = hk * hk;
            P.cm[t] = 4.0 * c->d.omega[0] * h2;
            P.cr1[t] = 2.0 * c->d.omega[1] * h2;
            P.cr2[t] = 4.0 * c->d.omega[2] * h2;
            P.cg[t] = c->d.omega[3] * h2;
        }
    }
    P.total = off;
    coarse_g_slot(c, P.nk[ntri] * P.nk[ntri] * P.nk[ntri], off, P.gofs, P.ng);
}

template <typename T> int launch_res_fast(mg_ctx *c, const double *f, const double *u, const int *done, cudaStream_t s) {
    const int n = c->d.n;
    const Level &l0 = c->lv[0];
    const double ih2 = 1.0 / (c->h * c->h);
    const double *fr = c->d.order == 4 ? c->ft : f;
    dim3 g;
    if (c->d.dim == 2) {
        g = dim3((n + 31) / 32, (n + 8 * RES_ROWS - 1) / (8 * RES_ROWS), 1);
        if (c->d.order == 2)
            LAUNCH_B(TAG_RESIDUAL, (k_res0_2d<T, 2>), g, B2, fr, u, c->d.pitch, n, ih2, 2 * c->m, a2<T>(l0.r[0], l0), c->part, done);
        else
            LAUNCH_B(TAG_RESIDUAL, (k_res0_2d<T, 4>), g, B2, fr, u, c->d.pitch, n, ih2, 2 * c->m, a2<T>(l0.r[0], l0), c->part, done);
    } else {
        g = dim3((n + 31) / 32, (n + 7) / 8, (n + RES3_PLANES - 1) / RES3_PLANES);
        if (c->d.order == 2)
            LAUNCH_B(TAG_RESIDUAL, (k_res0_3d<T, 2>), g, B2, fr, u, c->d.pitch, n, ih2, 2 * c->m, a3<T>(l0.r[0], l0), c->part, done);
        else
            LAUNCH_B(TAG_RESIDUAL, (k_res0_3d<T, 4>), g, B2, fr, u, c->d.pitch, n, ih2, 2 * c->m, a3<T>(l0.r[0], l0), c->part, done);
    }
    c->nparts = (int)(g.x * g.y * g.z);
    return c->nparts;
}

// order-4 right-hand side (computed once per solve / per mg_vcycle call)
void launch_rhs4(mg_ctx *c, const double *f, cudaStream_t s) {
    const int n = c->d.n;
    if (c->d.dim == 2) LAUNCH(TAG_CONTROL, (k_rhs4_2d), grid2(n, n), B2, f, c->d.pitch, n, c->ft);
    else LAUNCH(TAG_CONTROL, (k_rhs4_3d), grid3(n, n, n), B2, f, c->d.pitch, n, c->ft);
}

// tile of coset cells per block: large pairs 32x16, middle 16x8, small 8x8
// (small pairs are latency-bound; smaller tiles give them more blocks)
int tile_class(int nb) { return nb + 1 >= 1024 ? 0 : nb + 1 >= 256 ? 1 : 2; }

template <typename T, int TA, int TB>
void launch_down_pair(mg_ctx *c, int k, const int *done, cudaStream_t s, bool alt = false) {
    const Level &g = c->lv[2 * k], &r = c->lv[2 * k + 1], &b = c->lv[2 * k + 2];
    const int nb = r.nb;
    dim3 grid((nb + TA) / TA, (nb + TB) / TB, 1);
    const T *galt = (alt && k == 0 && c->rr) ? (const T *)c->r32b : nullptr;
    const int *par = galt ? &c->ctl->par : nullptr;
    LAUNCH_B(TAG_DOWN, (k_down_pair_2d<T, TA, TB>), grid, B2, a2<const T>(g.r[0], g), a2<T>(r.r[0], r),
             a2<T>(r.r[1], r), a2<T>(b.r[0], b), nb, galt, par, done);
}

template <typename T, int TA, int TB>
void launch_up_pair(mg_ctx *c, int k, double *u, const int *done, cudaStream_t s) {
    const Level &g = c->lv[2 * k], &r = c->lv[2 * k + 1], &b = c->lv[2 * k + 2];
    const int nb = r.nb;
    const double hk = spacing(c, g), p = c->d.omega[0];
    const T c2 = (T)(2.0 * p * hk * hk), c1 = (T)(p * hk * hk);
    dim3 grid((nb + TA) / TA, (nb + TB) / TB, 1);
    const size_t sm = sizeof(UpSmem<T, TA, TB>);
    if (k == 0)
        LAUNCH_SMEM_B(TAG_FINEST_UP, (k_up_pair_2d<T, true, TA, TB>), grid, B2, sm, a2<const T>(b.v[0], b),
                      a2<const T>(r.r[0], r), a2<const T>(r.r[1], r), a2<const T>(g.r[0], g), a2<T>(g.v[0], g), u,
                      c->d.pitch, nb, c2, c1, done);
    else
        LAUNCH_SMEM_B(TAG_UP, (k_up_pair_2d<T, false, TA, TB>), grid, B2, sm, a2<const T>(b.v[0], b),
                      a2<const T>(r.r[0], r), a2<const T>(r.r[1], r), a2<const T>(g.r[0], g), a2<T>(g.v[0], g), u,
                      c->d.pitch, nb, c2, c1, done);
}

// Kernel class of pair k.  FP64 levels: shared-memory tiles 0: 32x16 cells,
// 1: 16x8, 2: 8x8.  FP32 levels: 0-2 the warp-streaming kernels (strips of
// 32/16/8 cell rows up, 16/8/4 down), 3-5 the shared-memory tiles in the
// order above.  Untuned: by size, as measured on the 4095^2 hierarchy (the
// finest pair of the fused mixed solve is always streaming).
constexpr int NCLS_FP32 = 6;
int ff_strip(int cls);
int tile_default(const mg_ctx *c, int k, bool up) {
    const int cells = c->lv[2 * k + 1].nb + 1, cls = tile_class(cells - 1);
    // a batch's problems of one size share each launch, which then has
    // parallelism to spare: the largest tiles (FP64) or the streaming kernels
    // (FP32) at every level (as measured by mg_batch_tune on GB300 with ~80
    // problems per size)
    if (c->nprob > 1 && !(k == 0 && c->rr && up)) {
        if (c->esz == 8) return cells >= 128 ? 0 : cells >= 64 ? 1 : 2;
        return 1;
    }
    // FP64 levels (as measured by mg_tune on GB300): 16 x 8 tiles from 256
    // cells up, 32 x 16 only for restrictions from 2048 cells
    if (c->esz == 8) return up ? (cells >= 256 ? 1 : 2) : (cells >= 2048 ? 0 : cls == 0 ? 1 : cls);
    if (up) {
        if (k == 0 && c->rr) {
            // the fused finest pair: the longest strips (fewest warm-up rows)
            // that still give 9/10 of one wave of warps (4 blocks of 4 warps
            // per SM), else the shortest
            const long long nb = c->lv[1].nb;
            for (int q = 0; q < 2; q++) {
                const long long items = ((nb + FF_W) / FF_W) * ((nb + ff_strip(q)) / ff_strip(q)) * c->nprob;
                if (items * 10 >= 9LL * 16 * c->sms) return q;
            }
            return 2;
        }
        return cells >= 512 ? 2 : cells >= 128 ? 4 : 5;
    }
    return cells >= 1024 ? 1 : cells >= 512 ? 2 : cls + 3;
}
int tile_dn(const mg_ctx *c, int k) { return c->tile_dn[k] >= 0 ? c->tile_dn[k] : tile_default(c, k, false); }
int tile_up(const mg_ctx *c, int k) { return c->tile_up[k] >= 0 ? c->tile_up[k] : tile_default(c, k, true); }

void launch_down_ff(mg_ctx *c, int k, int cls, const int *done, cudaStream_t s, bool alt);
int launch_up_ff(mg_ctx *c, int k, int cls, double *u, const int *done, cudaStream_t s, bool rr,
                 Ctrl *vctl = nullptr);

template <typename T> void down_pair(mg_ctx *c, int k, int cls, const int *done, cudaStream_t s, bool alt) {
    if (sizeof(T) == 4) {
        if (cls < 3) { launch_down_ff(c, k, cls, done, s, alt); return; }
        cls -= 3;
    }
    switch (cls) {
    case 0: launch_down_pair<T, 32, 16>(c, k, done, s, alt); break;
    case 1: launch_down_pair<T, 16, 8>(c, k, done, s, alt); break;
    default: launch_down_pair<T, 8, 8>(c, k, done, s, alt); break;
    }
}
// rr: the finest pair of the fused mixed solve (u += v with the carried
// residual; streaming only); returns the partial sums it wrote per problem, or 0
template <typename T>
int up_pair(mg_ctx *c, int k, int cls, double *u, const int *done, cudaStream_t s, bool rr = false) {
    if (sizeof(T) == 4) {
        if (rr) return launch_up_ff(c, 0, cls < 3 ? cls : 0, u, done, s, true);
        if (cls < 3) return launch_up_ff(c, k, cls, u, done, s, false);
        cls -= 3;
    }
    switch (cls) {
    case 0: launch_up_pair<T, 32, 16>(c, k, u, done, s); break;
    case 1: launch_up_pair<T, 16, 8>(c, k, u, done, s); break;
    default: launch_up_pair<T, 8, 8>(c, k, u, done, s); break;
    }
    return 0;
}

// the coarse kernel of a 2D cycle: pairs kd.. in the cluster kernel, or
// pairs kc.. in the coarse thread block
template <typename T> void launch_coarse2d(mg_ctx *c, const int *done, cudaStream_t s) {
    const Level &g = c->lv[2 * c->kd];
    if (c->cl)
        LAUNCH_SMEM_B(TAG_COARSE, (k_coarse_cl_2d<T>), dim3(CL2, 1, 1), 1024, c->cl_bytes, c->plancl,
                      a2<const T>(g.r[0], g), a2<T>(g.v[0], g), c->G, done);
    else
        LAUNCH_SMEM_B(TAG_COARSE, (k_coarse_cta_2d<T>), dim3(1, 1, 1), 1024, c->plan_bytes, c->plan2d,
                      a2<const T>(g.r[0], g), a2<T>(g.v[0], g), c->G, done);
}

template <typename T> void vcycle_fast2d(mg_ctx *c, double *u, const int *done, cudaStream_t s) {
    for (int k = 0; k < c->kd; k++) down_pair<T>(c, k, tile_dn(c, k), done, s, false);
    launch_coarse2d<T>(c, done, s);
    for (int k = c->kd - 1; k >= 0; k--) up_pair<T>(c, k, tile_up(c, k), u, done, s);
    if (c->kd == 0) {  // the whole hierarchy ran in the coarse kernel: apply v to u
        const Level &l0 = c->lv[0];
        const int n = c->d.n;
        LAUNCH_B(TAG_FINEST_UP, (k_add_axis<T>), grid2(n, n), B2, (const T *)l0.v[0], l0.pitch, l0.rows, n, 2, u,
                 c->d.pitch, n + 2, done);
    }
}

// strip height (cell rows) of the warp-streaming pair kernels per tile class:
// the prolongation's chain needs 4 rows to fill, the restriction's 1
int ff_strip(int cls) { return cls == 0 ? 32 : cls == 1 ? 16 : 8; }
int fd_strip(int cls) { return cls == 0 ? 16 : cls == 1 ? 8 : 4; }

// one warp per (column, strip) item
dim3 ff_grid(int items) { return dim3((items + FF_WARPS - 1) / FF_WARPS, 1, 1); }

// FP32 pair k restriction (k_down_ff_2d)
void launch_down_ff(mg_ctx *c, int k, int cls, const int *done, cudaStream_t s, bool alt) {
    const Level &g = c->lv[2 * k], &r = c->lv[2 * k + 1], &b = c->lv[2 * k + 2];
    const int nb = r.nb, tb = fd_strip(cls);
    const dim3 grid = ff_grid(((nb + FD_W) / FD_W) * ((nb + tb) / tb));
    const float *galt = (alt && k == 0 && c->rr) ? (const float *)c->r32b : nullptr;
    LAUNCH_B(TAG_DOWN, (k_down_ff_2d), grid, dim3(32, FF_WARPS, 1), a2<const float>(g.r[0], g),
             a2<float>(r.r[0], r), a2<float>(r.r[1], r), a2<float>(b.r[0], b), nb, tb, galt,
             galt ? &c->ctl->par : nullptr, done);
}

// FP32 pair k prolongation (k_up_ff_2d): the finest pair of the fused mixed
// solve with the carried residual (rr), the finest pair otherwise with u += v,
// a coarser pair with v stored; returns the partial sums written per problem
// (rr) or 0
int launch_up_ff(mg_ctx *c, int k, int cls, double *u, const int *done, cudaStream_t s, bool rr, Ctrl *vctl) {
    const Level &g = c->lv[2 * k], &r = c->lv[2 * k + 1], &b = c->lv[2 * k + 2];
    const int nb = r.nb, tb = ff_strip(cls);
    const double hk = spacing(c, g), p = c->d.omega[0];
    const int items = ((nb + FF_W) / FF_W) * ((nb + tb) / tb);
    const bool add = k == 0 && !rr;
    const dim3 grid = ff_grid(items);
    const dim3 blk(32, FF_WARPS, 1);
    const bool vu = k == 0 && c->nprob == 1 && ((uintptr_t)u % 16) == 0 && c->d.pitch % 2 == 0;
    const float c2 = (float)(2.0 * p * hk * hk), c1 = (float)(p * hk * hk), s2 = (float)(1.0 / (hk * hk));
    const int tag = k == 0 ? (int)TAG_FINEST_UP : (int)TAG_UP;
#define MG_UPFF(MODE, VU, ...)                                                                                     \
    LAUNCH_B(tag, (k_up_ff_2d<MODE, VU, ##__VA_ARGS__>), grid, blk, a2<const float>(b.v[0], b), a2<const float>(r.r[0], r),     \
             a2<const float>(r.r[1], r), a2<float>(g.r[0], g), (float *)c->r32b, a2<float>(g.v[0], g),           \
             (float *)c->rlo, u, c->d.pitch, nb, c2, c1, s2, tb, c->part, rr ? c->ctl : vctl, done)
    // the fused finest pair of a single problem with 2..12 warps' worth of
    // items per SM: u and the residual's low part straight into registers (as
    // measured on GB300, mixed 1023^2 with 576 items 0.658 -> 0.611 ms; with a
    // full wave of items, 2047^2 and up, the extra registers cost a quarter of
    // the warps, and with at most two warps per SM, 511^2 and below, the
    // loads' latency is no longer hidden: 0.430 -> 0.442 ms at 255^2).  A
    // batch's launch covers all problems of its size, a full wave or more.
    const bool ud = rr && c->nprob == 1 && items > 2 * c->sms && items <= 12 * c->sms;
    if (rr) {
        if (ud) {
            if (vu) MG_UPFF(UP_RR, true, true);
            else MG_UPFF(UP_RR, false, true);
        } else if (vu) MG_UPFF(UP_RR, true);
        else MG_UPFF(UP_RR, false);
    } else if (add) {
        if (vu) MG_UPFF(UP_ADD, true);
        else MG_UPFF(UP_ADD, false);
    } else {
        MG_UPFF(UP_STORE, false);
    }
#undef MG_UPFF
    return rr ? (int)grid.x : 0;
}

// bound on |v| of level l (every array, ring included) into ctl->vmax, for
// the quantizer of the fused finest sweep
void launch_absmax(mg_ctx *c, const Level &l, const int *done, cudaStream_t s) {
    AbsArrs A{};
    for (int q = 0; q < l.ncos && q < 4; q++) A.a[q] = (const float *)l.v[q];
    const int narr = c->d.dim == 3 ? l.ncos : 1, nz = c->d.dim == 3 ? l.rows : 1;
    const int nrow = narr * nz * l.rows;
    LAUNCH_B(TAG_UP, (k_absmax), dim3(std::min((nrow + 7) / 8, 1216), 1, 1), dim3(32, 8, 1), A, narr, l.rows, nz,
             l.pitch, l.rows, c->ctl, done);
}

// one cycle of the fused mixed 2D path: restriction, coarse block, prolongation,
// and the finest pair fused with u += v and the next residual; returns the
// number of norm partial sums written per problem
int vcycle_rr(mg_ctx *c, double *u, const int *done, cudaStream_t s) {
    for (int k = 0; k < c->kd; k++) down_pair<float>(c, k, tile_dn(c, k), done, s, true);
    launch_coarse2d<float>(c, done, s);
    // the blue level of the finest pair (pair 1's v) also gets its bound on |v|:
    // in the streaming kernel that forms it, else by a separate pass
    const bool vfused = c->kd >= 2 && tile_up(c, 1) < 3;
    for (int k = c->kd - 1; k >= 1; k--) {
        if (k == 1 && vfused) launch_up_ff(c, 1, tile_up(c, 1), nullptr, done, s, false, c->ctl);
        else up_pair<float>(c, k, tile_up(c, k), u, done, s);
    }
    if (!vfused) launch_absmax(c, c->lv[2], done, s);
    return up_pair<float>(c, 0, tile_up(c, 0), u, done, s, true);
}

// direct FP64 residual of the fused path.  start: the carried float-float
// pair (hi in the current buffer, parity 0 at the start; lo in rlo), partial
// sums of r^2 at part and of f^2 right after every problem's (fpart); end of
// a solve: the partial sums of r^2 only.  zu (start of a solve from zero): u
// is not read.  Returns the partial sums per problem.
int launch_res_rr(mg_ctx *c, const double *f, const double *u, const int *done, cudaStream_t s, bool start,
                  bool zu = false) {
    const int z = start && zu ? 1 : 0;
    const int n = c->d.n;
    const Level &l0 = c->lv[0];
    const int lg = 2 * c->m;  // log2(1/h^2), h = 2^-m
    dim3 g = c->d.dim == 3 ? dim3((n + 31) / 32, (n + 7) / 8, (n + RES3_PLANES - 1) / RES3_PLANES)
                           : dim3((n + 31) / 32, (n + 8 * RES_ROWS - 1) / (8 * RES_ROWS), 1);
    const int np = (int)(g.x * g.y * g.z);
    double *fpart = start ? c->part + (size_t)np * c->nprob : nullptr;
    if (c->d.dim == 3) {
        if (start)
            LAUNCH_B(TAG_RESIDUAL, (k_res_rr_3d<true>), g, B2, f, u, c->d.pitch, n, lg, a3<float>(l0.r[0], l0),
                     (float *)c->rlo, l0.pitch, c->part, fpart, c->ctl, z, done);
        else
            LAUNCH_B(TAG_RESIDUAL, (k_res_rr_3d<false>), g, B2, f, u, c->d.pitch, n, lg, a3<float>(l0.r[0], l0),
                     (float *)c->rlo, l0.pitch, c->part, fpart, c->ctl, z, done);
    } else {
        if (start)
            LAUNCH_B(TAG_RESIDUAL, (k_res_rr_2d<true>), g, B2, f, u, c->d.pitch, n, lg, a2<float>(l0.r[0], l0),
                     (float *)c->rlo, l0.pitch, c->part, fpart, c->ctl, z, done);
        else
            LAUNCH_B(TAG_RESIDUAL, (k_res_rr_2d<false>), g, B2, f, u, c->d.pitch, n, lg, a2<float>(l0.r[0], l0),
                     (float *)c->rlo, l0.pitch, c->part, fpart, c->ctl, z, done);
    }
    c->nparts = np;
    return np;
}

// one cycle of the fused mixed 3D path; returns the partial sums per problem
int vcycle_rr3(mg_ctx *c, double *u, const int *done, cudaStream_t s, CtrlFuse cf) {
    const int lc = 3 * c->kc;
    for (int l = 0; l < lc; l++) launch_restrict<float>(c, l, done, s, true);
    const Level &gk = c->lv[lc];
    LAUNCH_SMEM_B(TAG_COARSE, (k_coarse_cta_3d<float>), dim3(1, 1, 1), 1024, c->plan_bytes, c->plan3d,
                  a3<const float>(gk.r[0], gk), a3<float>(gk.v[0], gk), c->G, done);
    for (int l = lc - 1; l >= 1; l--) launch_prolong<float>(c, l, c->d.omega, nullptr, done, s, l == 1 ? c->ctl : nullptr);
    const Level &a = c->lv[0], &b = c->lv[1];
    const int n = c->d.n;
    const double h2 = c->h * c->h;
    const dim3 g3 = green_ff_grid(c, n);
#define MG_GFF(VU)                                                                                                 \
    LAUNCH_SMEM_B(TAG_FINEST_UP, (k_green_ff_3d<UP_RR, VU>), g3, dim3(32, 8, 1), sizeof(GreenSSmem),              \
                  red3v<const float>(b.v, b), a3<float>(a.r[0], a), (float *)c->r32b, a3<float>(a.v[0], a),       \
                  (float *)c->rlo, u, c->d.pitch, n, (float)(c->d.omega[3] * h2), (float)(1.0 / h2),             \
                  green_ff_zch(c, n), c->part, c->ctl, cf, done)
    if (green_ff_vu(c, u)) MG_GFF(true);
    else MG_GFF(false);
#undef MG_GFF
    return (int)(g3.x * g3.y * g3.z);
}

template <typename T> cudaError_t set_smem_attrs(const mg_ctx *c) {
    // the limit is a property of the function, shared by every context (and
    // every plan a later mg_tune may choose): the device's maximum
    cudaError_t e = cudaFuncSetAttribute(k_coarse_cta_2d<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_optin(c));
#define MG_UP_ATTR(TA, TB)                                                                                         \
    if (e == cudaSuccess)                                                                                          \
        e = cudaFuncSetAttribute(k_up_pair_2d<T, true, TA, TB>, cudaFuncAttributeMaxDynamicSharedMemorySize,       \
                                 (int)sizeof(UpSmem<T, TA, TB>));                                                  \
    if (e == cudaSuccess)                                                                                          \
        e = cudaFuncSetAttribute(k_up_pair_2d<T, false, TA, TB>, cudaFuncAttributeMaxDynamicSharedMemorySize,      \
                                 (int)sizeof(UpSmem<T, TA, TB>));
    MG_UP_ATTR(32, 16)
    MG_UP_ATTR(16, 8)
    MG_UP_ATTR(8, 8)
#undef MG_UP_ATTR
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_coarse_cl_2d<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_optin(c));
    return e;
}

// can a cluster of the coarse kernel, with the planned shared memory, run on
// this device?  If not, the coarse thread block takes its pairs
template <typename T> void check_cluster2d(mg_ctx *c) {
    if (!c->cl) return;
    cudaLaunchConfig_t cfg{};
    cfg.gridDim = dim3(CL2, 1, 1);
    cfg.blockDim = dim3(1024, 1, 1);
    cfg.dynamicSmemBytes = c->cl_bytes;
    int ncl = 0;
    if (cudaOccupancyMaxActiveClusters(&ncl, k_coarse_cl_2d<T>, &cfg) != cudaSuccess || ncl < 1) {
        cudaGetLastError();
        c->cl_ok = false;
        plan_fast2d(c);
    }
}

// Pair / triple k of a gamma-cycle: restriction down to the blue level; on
// the blue grid (the green level of k+1) gamma cycles of k+1 from a zero
// correction, each after the first on the 5/7-point residual of the
// correction accumulated so far (the exact solve on the coarsest grid); then
// the prolongation sweeps; at k = 0 they also apply u += v.
template <typename T> void wlevel(mg_ctx *c, int k, double *u, const int *done, cudaStream_t s) {
    const int per = c->d.dim == 2 ? 2 : 3;  // levels per pair / triple
    for (int l = per * k; l < per * (k + 1); l++) launch_restrict<T>(c, l, done, s);
    if (k + 1 == c->K) {
        launch_coarse<T>(c, done, s);
    } else {
        const Level &b = c->lv[per * (k + 1)];
        const int nb = b.side;
        const T ih2 = (T)(1.0 / (spacing(c, b) * spacing(c, b)));
        T *rkeep = (T *)c->wr[k + 1], *vacc = (T *)c->wv[k + 1], *rb = (T *)b.r[0], *vb = (T *)b.v[0];
        cudaMemcpyAsync(rkeep, rb, b.len * sizeof(T), cudaMemcpyDeviceToDevice, s);
        for (int it = 0; it < c->gamma; it++) {
            if (c->d.dim == 2) {
                if (it > 0) LAUNCH_B(TAG_DOWN, (k_gres_2d<T>), grid2(nb, nb), B2, (const T *)rkeep, (const T *)vacc, rb, b.pitch, nb, ih2, done);
                wlevel<T>(c, k + 1, nullptr, done, s);
                LAUNCH_B(TAG_UP, (k_acc_2d<T>), grid2(nb, nb), B2, (const T *)vb, vacc, b.pitch, nb, it == 0 ? 1 : 0, done);
            } else {
                if (it > 0) LAUNCH_B(TAG_DOWN, (k_gres_3d<T>), grid3(nb, nb, nb), B2, (const T *)rkeep, (const T *)vacc, rb, b.pitch, b.rows, nb, ih2, done);
                wlevel<T>(c, k + 1, nullptr, done, s);
                LAUNCH_B(TAG_UP, (k_acc_3d<T>), grid3(nb, nb, nb), B2, (const T *)vb, vacc, b.pitch, b.rows, nb, it == 0 ? 1 : 0, done);
            }
        }
        cudaMemcpyAsync(vb, vacc, b.len * sizeof(T), cudaMemcpyDeviceToDevice, s);
    }
    for (int l = per * (k + 1) - 1; l >= per * k; l--)
        launch_prolong<T>(c, l, c->d.omega, l == 0 ? u : nullptr, done, s);
}

template <typename T>
mg_status vcycle_t(mg_ctx *c, const double *f, double *u, const int *done, bool with_residual, cudaStream_t s) {
    if (with_residual) launch_res_fast<T>(c, f, u, done, s);
    if (c->fast2d) {
        vcycle_fast2d<T>(c, u, done, s);
        CKL("vcycle launch");
        return MG_OK;
    }
    if (c->fast3d) {
        const int lc = 3 * c->kc;  // first level run by the coarse block
        for (int l = 0; l < lc; l++) launch_restrict<T>(c, l, done, s);
        const Level &g = c->lv[lc];
        LAUNCH_SMEM_B(TAG_COARSE, (k_coarse_cta_3d<T>), dim3(1, 1, 1), 1024, c->plan_bytes, c->plan3d,
                      a3<const T>(g.r[0], g), a3<T>(g.v[0], g), c->G, done);
        for (int l = lc - 1; l >= 0; l--) launch_prolong<T>(c, l, c->d.omega, l == 0 ? u : nullptr, done, s);
        if (lc == 0) {
            const Level &l0 = c->lv[0];
            const int n = c->d.n;
            LAUNCH_B(TAG_FINEST_UP, (k_add_axis<T>), grid3(n, n, n), B2, (const T *)l0.v[0], l0.pitch, l0.rows, n, 3, u,
                     c->d.pitch, n + 2, done);
        }
        CKL("vcycle launch");
        return MG_OK;
    }
    if (c->gamma > 1 && c->K >= 1) {  // a diagonal gamma-cycle (mg_set_gamma)
        wlevel<T>(c, 0, u, done, s);
        CKL("vcycle launch");
        return MG_OK;
    }
    for (int l = 0; l < c->L; l++) launch_restrict<T>(c, l, done, s);
    launch_coarse<T>(c, done, s);
    for (int l = c->L - 1; l >= 0; l--) launch_prolong<T>(c, l, c->d.omega, l == 0 ? u : nullptr, done, s);
    if (c->L == 0) {  // the finest grid is the coarsest: v = L^-1 r exactly
        const Level &l0 = c->lv[0];
        const int n = c->d.n;
        dim3 g = c->d.dim == 2 ? grid2(n, n) : grid3(n, n, n);
        LAUNCH_B(TAG_FINEST_UP, (k_add_axis<T>), g, B2, (const T *)l0.v[0], l0.pitch, l0.rows, n, c->d.dim, u, c->d.pitch, n + 2, done);
    }
    CKL("vcycle launch");
    return MG_OK;
}

bool valid_desc(const mg_desc *d) {
    if (!d) return false;
    if (d->dim != 2 && d->dim != 3) return false;
    const int m = log2_side(d->n), cm = log2_side(d->coarsest);
    if (m < 2 || cm < 1 || cm > m) return false;
    if (d->dim == 2 && d->coarsest > 7) return false;
    if (d->dim == 3 && d->coarsest > 7) return false;
    if (d->pitch < d->n + 2) return false;
    if (d->hierarchy != MG_DIAG && d->hierarchy != MG_USUAL) return false;
    if (d->order != 2 && d->order != 4) return false;
    if (d->precision != MG_FP64 && d->precision != MG_MIXED) return false;
    for (int i = 0; i < 4; i++)
        if (!std::isfinite(d->omega[i])) return false;
    return true;
}

}  // namespace

// ===========================================================================
// C ABI
// ===========================================================================

extern "C" {

const char *mg_strerror(mg_status st) {
    switch (st) {
    case MG_OK: return "ok";
    case MG_EINVAL: return "invalid argument";
    case MG_ENOMEM: return "device allocation failed";
    case MG_ECUDA: return "CUDA runtime error";
    case MG_ENOCONV: return "not converged within max_cycles";
    case MG_EDIVERGED: return "residual diverged";
    case MG_ETIMEOUT: return "bounded device wait timed out";
    }
    return "unknown status";
}

const char *mg_last_error(void) { return g_last_error; }

mg_status mg_destroy(mg_ctx *c) {
    if (!c) return MG_OK;
    cudaDeviceSynchronize();
    for (auto e : c->pev) cudaEventDestroy(e);
    drop_solve_graphs(c);
    if (c->cs1) cudaStreamDestroy(c->cs1);
    if (c->cs2) cudaStreamDestroy(c->cs2);
    if (c->cs_io) cudaStreamDestroy(c->cs_io);
    if (c->ev_ufinal) cudaEventDestroy(c->ev_ufinal);
    if (c->ev_io) cudaEventDestroy(c->ev_io);
    for (int b = 0; b < 2; b++)
        for (cudaEvent_t e : {c->ev_in[b], c->ev_sol[b], c->ev_out[b], c->ev_ctl[b]})
            if (e) cudaEventDestroy(e);
    if (c->hctl) cudaFreeHost(c->hctl);
    cudaFree(c->io_f2);
    cudaFree(c->io_u2);
    cudaFree(c->pool);
    cudaFree(c->part);
    cudaFree(c->ctl);
    cudaFree(c->hist);
    cudaFree(c->G);
    cudaFree(c->scal);
    cudaFree(c->ft);
    cudaFree(c->wpool);
    cudaFree(c->io_f);
    cudaFree(c->io_u);
    cudaFree(c->ftab);
    cudaFree(c->utab);
    delete c;
    return MG_OK;
}

// A context for nprob problems of one description (nprob = 1: mg_create).
static mg_status create_ctx(mg_ctx **out, const mg_desc *d, int nprob) {
    if (!out) return MG_EINVAL;
    *out = nullptr;
    if (!valid_desc(d) || nprob < 1) return MG_EINVAL;
    if (nprob > 1 && d->order != 2) return MG_EINVAL;
    mg_ctx *c = new (std::nothrow) mg_ctx();
    if (!c) return MG_ENOMEM;
    c->d = *d;
    for (int q = 0; q < 32; q++) c->tile_dn[q] = c->tile_up[q] = -1;
    c->m = log2_side(d->n);
    c->h = 1.0 / (d->n + 1);
    c->esz = d->precision == MG_FP64 ? 8 : 4;
    cudaGetDevice(&c->dev);
    if (cudaDeviceGetAttribute(&c->sms, cudaDevAttrMultiProcessorCount, c->dev) != cudaSuccess || c->sms < 1) {
        cudaGetLastError();
        c->sms = 152;
    }
    build_levels(c);
    size_t total = 0;
    for (auto &l : c->lv) total += (size_t)l.ncos * 2 * ((l.len * c->esz + 255) / 256 * 256);
    // fused update + residual of the mixed 2D diagonal solve (needs at least one pair outside the coarse block)
    // (3D with a 7^3 coarsest grid runs every level with per-stage kernels:
    // its inverse does not fit the coarse block, on which the fused path rests)
    c->rr = d->hierarchy == MG_DIAG && d->precision == MG_MIXED && d->order == 2 && d->n > (d->dim == 2 ? 63 : 15) &&
            !(d->dim == 3 && d->coarsest > 3);
    c->rr_alloc = c->rr;
    const size_t r32_bytes = c->rr ? (c->lv[0].len * 4 + 255) / 256 * 256 : 0;
    total += 2 * r32_bytes;
    c->nprob = nprob;
    c->pstride = nprob > 1 ? total : 0;
    if (cudaMalloc(&c->pool, total * nprob) != cudaSuccess) { cudaGetLastError(); mg_destroy(c); return MG_ENOMEM; }
    if (cudaMemset(c->pool, 0, total * nprob) != cudaSuccess) { mg_destroy(c); return MG_ECUDA; }
    char *p = (char *)c->pool;
    for (auto &l : c->lv) {
        size_t bytes = (l.len * c->esz + 255) / 256 * 256;
        for (int q = 0; q < l.ncos; q++) { l.r[q] = p; p += bytes; }
        for (int q = 0; q < l.ncos; q++) { l.v[q] = p; p += bytes; }
    }
    if (c->rr) {
        c->rlo = p; p += r32_bytes;
        c->r32b = p; p += r32_bytes;
    }
    c->max_blocks = residual_blocks(c);
    {
        // 1: the middle pairs in the cluster kernel (measured slower than the
        // pair kernels and the coarse block on GB300, so off by default)
        const char *ec = std::getenv("DIAGMG_CLUSTER");
        if (ec && ec[0] == '1') c->cl_top = 255;
    }
    plan_fast2d(c);
    plan_fast3d(c);
    if (c->fast3d) {
        cudaError_t e = d->precision == MG_FP64
            ? cudaFuncSetAttribute(k_coarse_cta_3d<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_optin(c))
            : cudaFuncSetAttribute(k_coarse_cta_3d<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_optin(c));
        const int g64 = (int)sizeof(Green3Smem<double>), g32 = (int)sizeof(Green3Smem<float>);
        const int gs = (int)sizeof(GreenSSmem);
#define MG_GFF_ATTR(MODE, VU) \
    if (e == cudaSuccess) e = cudaFuncSetAttribute(k_green_ff_3d<MODE, VU>, cudaFuncAttributeMaxDynamicSharedMemorySize, gs)
        MG_GFF_ATTR(UP_RR, true);
        MG_GFF_ATTR(UP_RR, false);
        MG_GFF_ATTR(UP_ADD, true);
        MG_GFF_ATTR(UP_ADD, false);
        MG_GFF_ATTR(UP_STORE, false);
#undef MG_GFF_ATTR
        if (e == cudaSuccess) {
            int per_sm = 0, sms = 0;
            e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_green_ff_3d<UP_RR, true>, 256, gs);
            if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, c->dev);
            if (e == cudaSuccess) c->gs_resident = std::max(1, per_sm * sms);
        }
        if (e == cudaSuccess) e = cudaFuncSetAttribute(k_green_3d<double, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, g64);
        if (e == cudaSuccess) e = cudaFuncSetAttribute(k_green_3d<double, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, g64);
        if (e == cudaSuccess) e = cudaFuncSetAttribute(k_green_3d<float, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, g32);
        if (e == cudaSuccess) e = cudaFuncSetAttribute(k_green_3d<float, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, g32);
        if (e != cudaSuccess) {
            mg_destroy(c);
            return cuda_fail(e, "mg_create shared-memory attributes (3D)");
        }
    }
    if (c->fast2d) {
        const cudaError_t e = d->precision == MG_FP64 ? set_smem_attrs<double>(c) : set_smem_attrs<float>(c);
        if (e != cudaSuccess) {
            mg_destroy(c);
            return cuda_fail(e, "mg_create shared-memory attributes");
        }
        if (d->precision == MG_FP64) check_cluster2d<double>(c);
        else check_cluster2d<float>(c);
    }
    if (d->order == 4 &&
        cudaMalloc(&c->ft, sizeof(double) * (size_t)d->pitch * (d->n + 2) * (d->dim == 3 ? (size_t)(d->n + 2) : 1)) !=
            cudaSuccess) {
        cudaGetLastError();
        mg_destroy(c);
        return MG_ENOMEM;
    }
    c->hist_cap = nprob > 1 ? 256 : 4096;
    const Level &lc = c->lv[c->L];
    const int nn = d->dim == 2 ? lc.side * lc.side : lc.side * lc.side * lc.side;
    if (nprob > 1 && (cudaMalloc(&c->ftab, sizeof(double *) * nprob) != cudaSuccess ||
                      cudaMalloc(&c->utab, sizeof(double *) * nprob) != cudaSuccess)) {
        cudaGetLastError();
        mg_destroy(c);
        return MG_ENOMEM;
    }
    if (cudaMalloc(&c->part, sizeof(double) * c->max_blocks * nprob) != cudaSuccess ||
        cudaMalloc(&c->ctl, sizeof(Ctrl) * nprob) != cudaSuccess ||
        cudaMalloc(&c->hist, sizeof(double) * c->hist_cap * nprob) != cudaSuccess ||
        cudaMalloc(&c->G, sizeof(double) * nn * nn) != cudaSuccess ||
        cudaMalloc(&c->scal, sizeof(double) * 4) != cudaSuccess) {
        cudaGetLastError();
        mg_destroy(c);
        return MG_ENOMEM;
    }
    {
        const char *ev = std::getenv("DIAGMG_SOLVE_GRAPH");
        c->use_graph = !(ev && ev[0] == '0');
        // programmatic dependent launch, by default where it measured faster
        // (medians of 6 x 10 solves): single 2D problems, every launch in
        // FP32 levels (4095^2: 2.224 -> 2.207 ms) and the grids of at most
        // 256 blocks in FP64 (9.573 -> 9.458 ms; every launch: 9.60 ms).  3D
        // cycles measured 1-2% slower with it on every launch and no faster
        // on the small grids alone.  DIAGMG_PDL=0/1 and
        // DIAGMG_PDL_MAX_BLOCKS=<blocks> (0: no limit) override.
        const char *ep = std::getenv("DIAGMG_PDL");
        const bool by_default = d->dim == 2 && nprob == 1;
        c->pdl = ep && (ep[0] == '0' || ep[0] == '1') ? ep[0] == '1' : by_default;
        const char *eb = std::getenv("DIAGMG_PDL_MAX_BLOCKS");
        c->pdl_max_blocks = eb ? std::atoi(eb) : (d->precision == MG_FP64 ? 256 : 0);
    }
    if (cudaStreamCreateWithFlags(&c->cs1, cudaStreamNonBlocking) != cudaSuccess ||
        cudaStreamCreateWithFlags(&c->cs2, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&c->ev_ufinal, cudaEventDisableTiming) != cudaSuccess) {
        mg_destroy(c);
        return cuda_fail(cudaGetLastError(), "mg_create streams");
    }
    std::vector<double> G = coarse_inverse(d->dim, lc.side, spacing(c, lc));
    if (cudaMemcpy(c->G, G.data(), sizeof(double) * G.size(), cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemset(c->ctl, 0, sizeof(Ctrl) * nprob) != cudaSuccess) {
        mg_destroy(c);
        return cuda_fail(cudaGetLastError(), "mg_create upload");
    }
    *out = c;
    return MG_OK;
}

mg_status mg_create(mg_ctx **out, const mg_desc *d) { return create_ctx(out, d, 1); }

mg_status mg_num_levels(const mg_ctx *c, int *num) {
    if (!c || !num) return MG_EINVAL;
    *num = c->L + 1;
    return MG_OK;
}

mg_status mg_level_info(const mg_ctx *c, int level, int *side, int *kind) {
    if (!c || level < 0 || level > c->L) return MG_EINVAL;
    if (side) *side = c->lv[level].side;
    if (kind) *kind = c->lv[level].kind;
    return MG_OK;
}

mg_status mg_residual(mg_ctx *c, const double *f, const double *u, double h, int order, double *r, double *norm2,
                      void *stream) {
    if (!c || bad_grid(f) || bad_grid(u) || (r && bad_grid(r))) return MG_EINVAL;
    if (r) {  // r is written while f and u are read: their extents must not overlap
        const size_t len = (size_t)c->d.pitch * (c->d.n + 2) * (c->d.dim == 3 ? (size_t)(c->d.n + 2) : 1);
        if (grids_overlap(r, f, len) || grids_overlap(r, u, len)) return MG_EINVAL;
    }
    if (order != c->d.order) return MG_EINVAL;
    if (std::fabs(h - c->h) > 1e-15 * c->h) return MG_EINVAL;
    cudaStream_t s = S(stream);
    if (c->d.precision == MG_FP64) launch_residual<double>(c, f, u, r, false, nullptr, s);
    else launch_residual<float>(c, f, u, r, false, nullptr, s);
    CKL("mg_residual");
    if (norm2) {
        LAUNCH(TAG_CONTROL, (k_sum_to), 1, 1024, c->part, c->max_blocks, c->scal);
        CKL("mg_residual norm");
        CK(cudaMemcpyAsync(norm2, c->scal, sizeof(double), cudaMemcpyDeviceToHost, s));
        CK(cudaStreamSynchronize(s));
    }
    return MG_OK;
}

mg_status mg_restrict_diag(mg_ctx *c, int level, void *stream) {
    if (!c || level < 0 || level >= c->L) return MG_EINVAL;
    if (c->d.precision == MG_FP64) launch_restrict<double>(c, level, nullptr, S(stream));
    else launch_restrict<float>(c, level, nullptr, S(stream));
    CKL("mg_restrict_diag");
    return MG_OK;
}

mg_status mg_coarse_solve(mg_ctx *c, void *stream) {
    if (!c) return MG_EINVAL;
    if (c->d.precision == MG_FP64) launch_coarse<double>(c, nullptr, S(stream));
    else launch_coarse<float>(c, nullptr, S(stream));
    CKL("mg_coarse_solve");
    return MG_OK;
}

mg_status mg_jacobi_prolong(mg_ctx *c, int level, const double *omega, void *stream) {
    if (!c || level < 0 || level >= c->L) return MG_EINVAL;
    const double *om = omega ? omega : c->d.omega;
    if (c->d.precision == MG_FP64) launch_prolong<double>(c, level, om, nullptr, nullptr, S(stream));
    else launch_prolong<float>(c, level, om, nullptr, nullptr, S(stream));
    CKL("mg_jacobi_prolong");
    return MG_OK;
}

static mg_status level_io(mg_ctx *c, int level, int which, double *grid, int to_level, void *stream) {
    if (!c || bad_grid(grid) || level < 0 || level > c->L || (which != 0 && which != 1)) return MG_EINVAL;
    const Level &l = c->lv[level];
    void *const *arr = which == 0 ? l.r : l.v;
    const int side = l.side, dim = c->d.dim;
    cudaStream_t s = S(stream);
    dim3 g = dim == 2 ? grid2(side, side) : grid3(side, side, side);
    void *c0 = arr[0], *c1 = l.ncos > 1 ? arr[1] : nullptr, *c2 = l.ncos > 2 ? arr[2] : nullptr,
         *c3 = l.ncos > 3 ? arr[3] : nullptr;
    if (c->d.precision == MG_FP64)
        LAUNCH(TAG_CONTROL, (k_level_io<double>), g, B2, dim, l.kind, side, grid, (double *)c0, (double *)c1, (double *)c2,
                                                    (double *)c3, l.pitch, l.rows, to_level);
    else
        LAUNCH(TAG_CONTROL, (k_level_io<float>), g, B2, dim, l.kind, side, grid, (float *)c0, (float *)c1, (float *)c2,
                                                   (float *)c3, l.pitch, l.rows, to_level);
    CKL("mg_level_io");
    return MG_OK;
}

mg_status mg_level_get(mg_ctx *c, int level, int which, double *grid, void *stream) {
    return level_io(c, level, which, grid, 0, stream);
}

mg_status mg_level_set(mg_ctx *c, int level, int which, const double *grid, void *stream) {
    return level_io(c, level, which, (double *)grid, 1, stream);
}

mg_status mg_vcycle(mg_ctx *c, const double *f, double *u, void *stream) {
    if (!c || bad_grid(f) || bad_grid(u)) return MG_EINVAL;
    if (c->d.order == 4) {
        cudaStream_t s = S(stream);
        launch_rhs4(c, f, s);
    }
    if (c->d.precision == MG_FP64) return vcycle_t<double>(c, f, u, nullptr, true, S(stream));
    return vcycle_t<float>(c, f, u, nullptr, true, S(stream));
}

// partial sums of ||f~||^2 (f~ = f for order 2, the Mehrstellen / 19-point
// right-hand side for order 4); returns the partial count per problem
static int launch_rhs_norm(mg_ctx *c, const double *f, const double *u, cudaStream_t s) {
    const bool fp64 = c->d.precision == MG_FP64;
    if (c->d.order == 4) {
        if (fp64) launch_residual<double>(c, f, u, nullptr, true, nullptr, s);
        else launch_residual<float>(c, f, u, nullptr, true, nullptr, s);
        return c->max_blocks;
    }
    const int n = c->d.n;
    dim3 g;
    if (c->d.dim == 2) {
        g = dim3((n + 31) / 32, (n + 8 * RES_ROWS - 1) / (8 * RES_ROWS), 1);
        LAUNCH_B(TAG_CONTROL, (k_norm_f<2>), g, B2, f, c->d.pitch, n, c->part, (const int *)nullptr);
    } else {
        g = dim3((n + 31) / 32, (n + 7) / 8, (n + RES3_PLANES - 1) / RES3_PLANES);
        LAUNCH_B(TAG_CONTROL, (k_norm_f<3>), g, B2, f, c->d.pitch, n, c->part, (const int *)nullptr);
    }
    return (int)(g.x * g.y * g.z);
}

// residual of the current iterate into level 0 (+ partial sums); returns their count
static int solve_residual(mg_ctx *c, const double *f, const double *u, const int *done, cudaStream_t s) {
    if (c->rr) return launch_res_rr(c, f, u, done, s, true);
    return c->d.precision == MG_FP64 ? launch_res_fast<double>(c, f, u, done, s)
                                     : launch_res_fast<float>(c, f, u, done, s);
}

// control step after a residual: single problem (k_ctrl sets the loop
// condition itself) or a batch (one block per problem, then "any active")
static void launch_ctrl(mg_ctx *c, int np, int first, cudaGraphConditionalHandle loop, int use_loop, cudaStream_t s) {
    if (c->nprob == 1) {
        LAUNCH(TAG_CONTROL, (k_ctrl), 1, 1024, c->part, np, c->ctl, c->hist, first, loop, use_loop);
    } else {
        LAUNCH(TAG_CONTROL, (k_ctrl_b), c->nprob, 1024, c->part, np, c->ctl, c->hist, c->hist_cap, first);
        LAUNCH(TAG_CONTROL, (k_any_active), 1, 1024, c->ctl, c->nprob, loop, use_loop, (int *)nullptr);
    }
}

// doubles of one full grid of the context (caller pitch)
static size_t grid_len(const mg_ctx *c) {
    return (size_t)c->d.pitch * (c->d.n + 2) * (c->d.dim == 3 ? (size_t)(c->d.n + 2) : 1);
}
// a copy of the (n+2)^d points of a caller grid (both sides in the caller
// pitch); the padding of a pitch above n + 2 is neither read nor written
static cudaError_t copy_grid(const mg_ctx *c, double *dst, const double *src, cudaMemcpyKind kind, cudaStream_t s) {
    const size_t rows = (size_t)(c->d.n + 2) * (c->d.dim == 3 ? (size_t)(c->d.n + 2) : 1);
    const size_t pb = sizeof(double) * c->d.pitch;
    if (c->d.pitch == c->d.n + 2) return cudaMemcpyAsync(dst, src, pb * rows, kind, s);  // contiguous
    return cudaMemcpy2DAsync(dst, pb, src, pb, sizeof(double) * (c->d.n + 2), rows, kind, s);
}
// zeros on the (n+2)^d points of a caller grid; the padding of a pitch above
// n + 2 is left alone
static cudaError_t zero_grid(const mg_ctx *c, double *u, cudaStream_t s) {
    const size_t rows = (size_t)(c->d.n + 2) * (c->d.dim == 3 ? (size_t)(c->d.n + 2) : 1);
    return cudaMemset2DAsync(u, sizeof(double) * c->d.pitch, 0, sizeof(double) * (c->d.n + 2), rows, s);
}

// Prefix of a solve: control words, the norm of the right-hand side, the
// residual of the warm start and the first control step (which sets the loop
// condition when use_loop).  The fused mixed path takes the norm of f from
// its start residual kernel.
static void solve_prefix(mg_ctx *c, const double *f, double *u, double rtol, int max_cycles,
                         cudaGraphConditionalHandle loop, int use_loop, cudaStream_t s) {
    if (c->nprob == 1) {
        LAUNCH(TAG_CONTROL, (k_ctrl_init), 1, 1, c->ctl, rtol, max_cycles);
    } else {
        LAUNCH(TAG_CONTROL, (k_ctrl_init_b), (c->nprob + 255) / 256, 256, c->ctl, c->nprob, rtol, max_cycles);
    }
    int np = 0, nfp;
    const double *fpart = c->part;
    if (c->rr) {
        // a solve from zero: u zeroed here (an error shows in the caller's
        // launch check), and the start residual reads none of it
        if (c->zstart) (void)zero_grid(c, u, s);
        np = nfp = launch_res_rr(c, f, u, nullptr, s, true, c->zstart);
        fpart = c->part + (size_t)np * c->nprob;
    } else {
        nfp = launch_rhs_norm(c, f, u, s);
    }
    if (c->nprob == 1) {
        LAUNCH(TAG_CONTROL, (k_sum_to), 1, 1024, fpart, nfp, &c->ctl->f2);
    } else {
        LAUNCH(TAG_CONTROL, (k_sum_to_b), c->nprob, 1024, fpart, nfp, c->ctl);
    }
    if (!c->rr) {
        if (c->d.order == 4) launch_rhs4(c, f, s);
        np = solve_residual(c, f, u, nullptr, s);
    }
    launch_ctrl(c, np, 1, loop, use_loop, s);
}

// Record one solve into the capture active on stream s: prefix (control
// init, norm of the right-hand side, residual of the warm start, first
// control step) and a conditional WHILE node whose body -- recorded on s2 --
// is one V-cycle, the residual of the new iterate and the control step that
// sets the loop condition to "not done" (for a batch: "any not done").
static mg_status capture_solve(mg_ctx *c, const double *f, double *u, double rtol, int max_cycles, cudaStream_t s,
                               cudaStream_t s2) {
    const bool fp64 = c->d.precision == MG_FP64;
    const int *done = &c->ctl->done;
    c->capturing = true;
    const long long l0 = c->launches;
    cudaStreamCaptureStatus st;
    cudaGraph_t g = nullptr;
    CK(cudaStreamGetCaptureInfo(s, &st, nullptr, &g, nullptr, nullptr, nullptr));
    cudaGraphConditionalHandle loop;
    CK(cudaGraphConditionalHandleCreate(&loop, g, 0, cudaGraphCondAssignDefault));
    solve_prefix(c, f, u, rtol, max_cycles, loop, 1, s);
    c->g_prefix_kernels = c->launches - l0;
    const cudaGraphNode_t *deps = nullptr;
    size_t ndeps = 0;
    {   // a launch that failed (and so invalidated the capture) ends it here
        const cudaError_t le = cudaGetLastError();
        if (le != cudaSuccess) { c->capturing = false; return cuda_fail(le, "solve capture (prefix)"); }
    }
    CK(cudaStreamGetCaptureInfo(s, &st, nullptr, &g, &deps, nullptr, &ndeps));
    if (st != cudaStreamCaptureStatusActive) {
        c->capturing = false;
        return cuda_fail(cudaErrorStreamCaptureInvalidated, "solve capture (prefix)");
    }
    cudaGraphNodeParams cp{};
    cp.type = cudaGraphNodeTypeConditional;
    cp.conditional.handle = loop;
    cp.conditional.type = cudaGraphCondTypeWhile;
    cp.conditional.size = 1;
    cudaGraphNode_t wnode;
    CK(cudaGraphAddNode(&wnode, g, deps, nullptr, ndeps, &cp));
    cudaGraph_t body = cp.conditional.phGraph_out[0];
    CK(cudaStreamUpdateCaptureDependencies(s, &wnode, nullptr, 1, cudaStreamSetCaptureDependencies));
    CK(cudaStreamBeginCaptureToGraph(s2, body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal));
    const long long l1 = c->launches;
    int np2;
    // a single mixed 3D problem: the finest kernel's last block runs the
    // control step (in 2D the fused epilogue slowed the finest kernel more
    // than the launch it saves)
    const bool fuse = c->rr && c->nprob == 1 && c->d.dim == 3;
    if (c->rr) {
        const CtrlFuse cf = fuse ? CtrlFuse{&c->ctl->arrive, c->hist, loop, 1} : CtrlFuse{};
        np2 = c->d.dim == 3 ? vcycle_rr3(c, u, done, s2, cf) : vcycle_rr(c, u, done, s2);
    } else {
        mg_status stv = fp64 ? vcycle_t<double>(c, f, u, done, false, s2) : vcycle_t<float>(c, f, u, done, false, s2);
        if (stv != MG_OK) {
            cudaStreamEndCapture(s2, &body);
            c->capturing = false;
            return stv;
        }
        np2 = solve_residual(c, f, u, nullptr, s2);
    }
    if (!fuse) launch_ctrl(c, np2, 0, loop, 1, s2);
    c->g_body_kernels = c->launches - l1;
    {
        const cudaError_t le = cudaGetLastError();
        const cudaError_t ee = cudaStreamEndCapture(s2, &body);
        if (le != cudaSuccess || ee != cudaSuccess) {
            c->capturing = false;
            return cuda_fail(le != cudaSuccess ? le : ee, "solve capture (cycle)");
        }
    }
    if (c->rr) {  // the carried residual ignores the rounding of u: report a direct one
        const long long l2 = c->launches;
        // u is final here: an event record node of the graph (External: a
        // plain record inside a capture would only order the capture's streams)
        if (cudaEventRecordWithFlags(c->ev_ufinal, s, cudaEventRecordExternal) != cudaSuccess) {
            c->capturing = false;
            return cuda_fail(cudaGetLastError(), "solve capture (u final)");
        }
        const int np3 = launch_res_rr(c, f, u, nullptr, s, false);
        LAUNCH(TAG_CONTROL, (k_final_true), c->nprob, 1024, c->part, np3, c->ctl);
        c->g_prefix_kernels += c->launches - l2;
    }
    c->capturing = false;
    c->launches = l0;  // counted when the graph runs
    return MG_OK;
}

static bool solve_graph_matches(const mg_ctx *c, const mg_ctx::SolveGraph &e, const double *f, const double *u,
                                double rtol, int max_cycles) {
    return e.exec && e.f == f && e.u == u && e.rtol == rtol && e.max == max_cycles && e.order == c->d.order &&
           e.extra == c->extra && e.gamma == c->gamma && e.zero == c->zstart &&
           std::memcmp(e.omega, c->d.omega, sizeof e.omega) == 0;
}

static mg_status build_solve_graph(mg_ctx *c, mg_ctx::SolveGraph &slot, const double *f, double *u, double rtol,
                                   int max_cycles) {
    drop_solve_graph(slot);
    cudaStream_t s = c->cs1;
    CK(cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal));
    mg_status st = capture_solve(c, f, u, rtol, max_cycles, s, c->cs2);
    cudaGraph_t g = nullptr;
    const cudaError_t e = cudaStreamEndCapture(s, &g);
    if (st != MG_OK) { if (g) cudaGraphDestroy(g); return st; }
    if (e != cudaSuccess) return cuda_fail(e, "cudaStreamEndCapture");
    slot.graph = g;
    const cudaError_t ei = cudaGraphInstantiate(&slot.exec, g, 0);
    if (ei != cudaSuccess) { drop_solve_graph(slot); return cuda_fail(ei, "cudaGraphInstantiate"); }
    slot.f = f; slot.u = u; slot.rtol = rtol; slot.max = max_cycles;
    slot.order = c->d.order;
    slot.extra = c->extra;
    slot.gamma = c->gamma;
    slot.zero = c->zstart;
    for (int q = 0; q < 4; q++) slot.omega[q] = c->d.omega[q];
    slot.prefix_kernels = c->g_prefix_kernels;
    slot.body_kernels = c->g_body_kernels;
    return MG_OK;
}

// The same schedule driven from the host (one control-word read per 4 cycles,
// per cycle while probed); used when graphs are disabled, e.g. under a kernel
// profiler, and while a probe is active.
static mg_status solve_host_loop(mg_ctx *c, const double *f, double *u, double rtol, int max_cycles,
                                 int *cycles_out, double *relres_out, double *history, cudaStream_t s) {
    const bool fp64 = c->d.precision == MG_FP64;
    const int *done = &c->ctl->done;
    cudaGraphConditionalHandle none = 0;
    solve_prefix(c, f, u, rtol, max_cycles, none, 0, s);
    int np = 0;
    CKL("mg_solve init");
    Ctrl host{};
    // cycles are launched in groups between reads of the control word; one
    // per group while a probe is active, so that probed launches all do work
    const int group = c->probe_tag >= 0 ? 1 : 4;
    for (int cyc = 0; cyc < max_cycles; cyc += group) {
        for (int q = 0; q < group && cyc + q < max_cycles; q++) {
            const bool fuse = c->rr && c->nprob == 1 && c->d.dim == 3;  // control step in the finest kernel
            if (c->rr) {
                const CtrlFuse cf = fuse ? CtrlFuse{&c->ctl->arrive, c->hist, none, 0} : CtrlFuse{};
                np = c->d.dim == 3 ? vcycle_rr3(c, u, done, s, cf) : vcycle_rr(c, u, done, s);
            } else {
                mg_status st = fp64 ? vcycle_t<double>(c, f, u, done, false, s) : vcycle_t<float>(c, f, u, done, false, s);
                if (st != MG_OK) return st;
                np = solve_residual(c, f, u, done, s);
            }
            if (!fuse) launch_ctrl(c, np, 0, none, 0, s);
        }
        CK(cudaMemcpyAsync(&host, c->ctl, sizeof(Ctrl), cudaMemcpyDeviceToHost, s));
        CK(cudaStreamSynchronize(s));
        probe_collect(c);
        if (host.done) break;
    }
    if (c->rr) {
        const int np3 = launch_res_rr(c, f, u, nullptr, s, false);
        LAUNCH(TAG_CONTROL, (k_final_true), c->nprob, 1024, c->part, np3, c->ctl);
    }
    CK(cudaMemcpyAsync(&host, c->ctl, sizeof(Ctrl), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    if (cycles_out) *cycles_out = host.cycles;
    if (relres_out) *relres_out = host.relres;
    if (history && host.cycles > 0) {
        CK(cudaMemcpyAsync(history, c->hist, sizeof(double) * host.cycles, cudaMemcpyDeviceToHost, s));
        CK(cudaStreamSynchronize(s));
    }
    if (host.status == -5) return MG_EDIVERGED;
    if (host.status == -4 || !host.done) return MG_ENOCONV;
    return MG_OK;
}

// mg_solve; with u_host, u is also copied to that host array before the call
// returns: on the fused mixed path's graph the copy starts once the last
// cycle has written u (event ev_ufinal) and runs on cs_io beside the direct
// residual that closes the solve, else after the solve on the stream
// the solve graph of these arguments: from the cache, else recorded into its
// least recently used slot
static mg_status solve_graph(mg_ctx *c, const double *f, double *u, double rtol, int max_cycles,
                             mg_ctx::SolveGraph **out) {
    mg_ctx::SolveGraph *hit = nullptr, *lru = &c->gcache[0];
    for (auto &e : c->gcache) {
        if (solve_graph_matches(c, e, f, u, rtol, max_cycles)) { hit = &e; break; }
        if (e.used < lru->used) lru = &e;
    }
    if (!hit) {
        const mg_status st = build_solve_graph(c, *lru, f, u, rtol, max_cycles);
        if (st != MG_OK) return st;
        hit = lru;
    }
    hit->used = ++c->gtick;
    *out = hit;
    return MG_OK;
}

static mg_status solve_impl(mg_ctx *c, const double *f, double *u, double rtol, int max_cycles, int *cycles_out,
                            double *relres_out, double *history, void *stream, double *u_host) {
    cudaStream_t s = S(stream);
    mg_status st;
    Ctrl host{};
    // a probe needs one event pair per launch, which a replayed graph cannot give
    if (!c->use_graph || c->probe_tag >= 0) {
        st = solve_host_loop(c, f, u, rtol, max_cycles, cycles_out, relres_out, history, s);
        if (u_host && (st == MG_OK || st == MG_ENOCONV || st == MG_EDIVERGED)) {
            CK(copy_grid(c, u_host, u, cudaMemcpyDeviceToHost, s));
            CK(cudaStreamSynchronize(s));
        }
        return st;
    }
    mg_ctx::SolveGraph *hit = nullptr;
    st = solve_graph(c, f, u, rtol, max_cycles, &hit);
    if (st != MG_OK) return st;
    CK(cudaGraphLaunch(hit->exec, s));
    const bool early = u_host && c->rr;  // the copy of u overlaps the closing residual
    if (early) {
        CK(cudaStreamWaitEvent(c->cs_io, c->ev_ufinal, 0));
        CK(copy_grid(c, u_host, u, cudaMemcpyDeviceToHost, c->cs_io));
        CK(cudaEventRecord(c->ev_io, c->cs_io));
    }
    CK(cudaMemcpyAsync(&host, c->ctl, sizeof(Ctrl), cudaMemcpyDeviceToHost, s));
    if (u_host && !early) CK(copy_grid(c, u_host, u, cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    if (early) CK(cudaEventSynchronize(c->ev_io));
    c->launches += hit->prefix_kernels + (long long)host.cycles * hit->body_kernels;
    if (cycles_out) *cycles_out = host.cycles;
    if (relres_out) *relres_out = host.relres;
    if (history && host.cycles > 0) {
        CK(cudaMemcpyAsync(history, c->hist, sizeof(double) * host.cycles, cudaMemcpyDeviceToHost, s));
        CK(cudaStreamSynchronize(s));
    }
    if (host.status == -5) return MG_EDIVERGED;
    if (host.status == -4 || !host.done) return MG_ENOCONV;
    return MG_OK;
}

mg_status mg_solve(mg_ctx *c, const double *f, double *u, double rtol, int max_cycles, int *cycles_out,
                   double *relres_out, double *history, void *stream) {
    if (!c || bad_grid(f) || bad_grid(u) || !(rtol >= 0.0) || max_cycles < 0 || max_cycles > c->hist_cap)
        return MG_EINVAL;
    return solve_impl(c, f, u, rtol, max_cycles, cycles_out, relres_out, history, stream, nullptr);
}

// mg_solve_zero, with the optional host destination of solve_impl
static mg_status solve_zero_impl(mg_ctx *c, const double *f, double *u, double rtol, int max_cycles,
                                 int *cycles_out, double *relres_out, double *history, void *stream,
                                 double *u_host) {
    if (!c || bad_grid(f) || bad_grid(u) || !(rtol >= 0.0) || max_cycles < 0 || max_cycles > c->hist_cap)
        return MG_EINVAL;
    if (grids_overlap(f, u, grid_len(c))) return MG_EINVAL;
    if (!c->rr || c->nprob != 1) {
        // the per-stage paths read u from their first kernel on: zeros first
        CK(zero_grid(c, u, S(stream)));
        return solve_impl(c, f, u, rtol, max_cycles, cycles_out, relres_out, history, stream, u_host);
    }
    c->zstart = true;
    const mg_status st = solve_impl(c, f, u, rtol, max_cycles, cycles_out, relres_out, history, stream, u_host);
    c->zstart = false;
    return st;
}

mg_status mg_solve_zero(mg_ctx *c, const double *f, double *u, double rtol, int max_cycles, int *cycles_out,
                        double *relres_out, double *history, void *stream) {
    return solve_zero_impl(c, f, u, rtol, max_cycles, cycles_out, relres_out, history, stream, nullptr);
}

mg_status mg_solve_host(mg_ctx *c, const double *f_host, const double *u0_host, double *u_host, double rtol,
                        int max_cycles, int *cycles_out, double *relres_out, void *stream) {
    if (!c || c->nprob != 1 || bad_grid(f_host) || bad_grid(u_host) || (u0_host && bad_grid(u0_host)) ||
        !(rtol >= 0.0) || max_cycles < 0 || max_cycles > c->hist_cap)
        return MG_EINVAL;
    const size_t len = (size_t)c->d.pitch * (c->d.n + 2) * (c->d.dim == 3 ? (size_t)(c->d.n + 2) : 1);
    const size_t bytes = sizeof(double) * len;
    if (grids_overlap(f_host, u_host, len)) return MG_EINVAL;
    if (!c->io_f) {  // the first call: device copies of f and u, kept by the context
        if (cudaMalloc(&c->io_f, bytes) != cudaSuccess || cudaMalloc(&c->io_u, bytes) != cudaSuccess) {
            cudaGetLastError();
            cudaFree(c->io_f);
            cudaFree(c->io_u);
            c->io_f = c->io_u = nullptr;
            return MG_ENOMEM;
        }
    }
    if (!c->cs_io) {  // the copy-back stream and its completion event
        if (cudaStreamCreateWithFlags(&c->cs_io, cudaStreamNonBlocking) != cudaSuccess ||
            cudaEventCreateWithFlags(&c->ev_io, cudaEventDisableTiming) != cudaSuccess) {
            if (c->cs_io) cudaStreamDestroy(c->cs_io);
            c->cs_io = nullptr;
            return cuda_fail(cudaGetLastError(), "mg_solve_host stream");
        }
    }
    cudaStream_t s = S(stream);
    CK(copy_grid(c, c->io_f, f_host, cudaMemcpyHostToDevice, s));
    if (u0_host) CK(copy_grid(c, c->io_u, u0_host, cudaMemcpyHostToDevice, s));
    // the solve copies u back itself (overlapped with its closing residual)
    return u0_host ? solve_impl(c, c->io_f, c->io_u, rtol, max_cycles, cycles_out, relres_out, nullptr, stream, u_host)
                   : solve_zero_impl(c, c->io_f, c->io_u, rtol, max_cycles, cycles_out, relres_out, nullptr, stream,
                                     u_host);
}

static mg_status status_of(const Ctrl &h) {
    if (h.status == -5) return MG_EDIVERGED;
    if (h.status == -4 || !h.done) return MG_ENOCONV;
    return MG_OK;
}

mg_status mg_solve_host_many(mg_ctx *c, int count, const double *const *f_host, double *const *u_host, double rtol,
                             int max_cycles, int *cycles_out, double *relres_out, void *stream) {
    if (!c || c->nprob != 1 || count < 0 || (count > 0 && (!f_host || !u_host)) || !(rtol >= 0.0) || max_cycles < 0 ||
        max_cycles > c->hist_cap)
        return MG_EINVAL;
    const size_t len = grid_len(c), bytes = sizeof(double) * len;
    for (int k = 0; k < count; k++)
        if (bad_grid(f_host[k]) || bad_grid(u_host[k])) return MG_EINVAL;
    // no output may overlap any input (a result copied back early would
    // change a later problem's right-hand side); outputs may share a buffer
    for (int k = 0; k < count; k++)
        for (int j = 0; j < count; j++)
            if (grids_overlap(f_host[j], u_host[k], len)) return MG_EINVAL;
    if (count == 0) return MG_OK;
    // host-driven loop (no graph): one problem after the other
    if (!c->use_graph || c->probe_tag >= 0) {
        mg_status worst = MG_OK;
        for (int k = 0; k < count; k++) {
            const mg_status st = mg_solve_host(c, f_host[k], nullptr, u_host[k], rtol, max_cycles,
                                               cycles_out ? cycles_out + k : nullptr,
                                               relres_out ? relres_out + k : nullptr, stream);
            if (st != MG_OK && st != MG_ENOCONV && st != MG_EDIVERGED) return st;
            if (st == MG_EDIVERGED || (st == MG_ENOCONV && worst == MG_OK)) worst = st;
        }
        return worst;
    }
    // the first call: a second pair of device copies, the copy stream, the
    // pipeline's events and two page-locked control words
    if (!c->io_f) {
        if (cudaMalloc(&c->io_f, bytes) != cudaSuccess || cudaMalloc(&c->io_u, bytes) != cudaSuccess) {
            cudaGetLastError();
            cudaFree(c->io_f);
            cudaFree(c->io_u);
            c->io_f = c->io_u = nullptr;
            return MG_ENOMEM;
        }
    }
    if (!c->io_f2) {
        if (cudaMalloc(&c->io_f2, bytes) != cudaSuccess || cudaMalloc(&c->io_u2, bytes) != cudaSuccess) {
            cudaGetLastError();
            cudaFree(c->io_f2);
            cudaFree(c->io_u2);
            c->io_f2 = c->io_u2 = nullptr;
            return MG_ENOMEM;
        }
    }
    if (!c->cs_io) {
        if (cudaStreamCreateWithFlags(&c->cs_io, cudaStreamNonBlocking) != cudaSuccess ||
            cudaEventCreateWithFlags(&c->ev_io, cudaEventDisableTiming) != cudaSuccess) {
            if (c->cs_io) cudaStreamDestroy(c->cs_io);
            c->cs_io = nullptr;
            return cuda_fail(cudaGetLastError(), "mg_solve_host_many stream");
        }
    }
    if (!c->hctl) {
        for (int b = 0; b < 2; b++)
            for (cudaEvent_t *e : {&c->ev_in[b], &c->ev_sol[b], &c->ev_out[b], &c->ev_ctl[b]})
                if (!*e) CK(cudaEventCreateWithFlags(e, cudaEventDisableTiming));
        if (cudaHostAlloc(reinterpret_cast<void **>(&c->hctl), 2 * sizeof(Ctrl), cudaHostAllocDefault) != cudaSuccess) {
            c->hctl = nullptr;
            return cuda_fail(cudaGetLastError(), "mg_solve_host_many control words");
        }
    }
    cudaStream_t s = S(stream), io = c->cs_io;
    double *F[2] = {c->io_f, c->io_f2}, *U[2] = {c->io_u, c->io_u2};
    mg_ctx::SolveGraph *hit[2] = {nullptr, nullptr};
    mg_status worst = MG_OK;
    // the results of solve k (control word slot k & 1) once it has run
    auto collect = [&](int k) -> mg_status {
        const int b = k & 1;
        CK(cudaEventSynchronize(c->ev_ctl[b]));
        const Ctrl &h = c->hctl[b];
        c->launches += hit[b]->prefix_kernels + (long long)h.cycles * hit[b]->body_kernels;
        if (cycles_out) cycles_out[k] = h.cycles;
        if (relres_out) relres_out[k] = h.relres;
        const mg_status st = status_of(h);
        if (st == MG_EDIVERGED || (st == MG_ENOCONV && worst == MG_OK)) worst = st;
        return MG_OK;
    };
    auto pipeline = [&]() -> mg_status {
        CK(cudaEventRecord(c->ev_io, s));  // the copies start after the caller's earlier work
        CK(cudaStreamWaitEvent(io, c->ev_io, 0));
        CK(copy_grid(c, F[0], f_host[0], cudaMemcpyHostToDevice, io));
        CK(cudaEventRecord(c->ev_in[0], io));
        for (int k = 0; k < count; k++) {
            const int b = k & 1;
            if (k + 1 < count) {  // the next input, into the buffer solve k - 1 used
                if (k >= 1) CK(cudaStreamWaitEvent(io, c->ev_sol[b ^ 1], 0));
                CK(copy_grid(c, F[b ^ 1], f_host[k + 1], cudaMemcpyHostToDevice, io));
                CK(cudaEventRecord(c->ev_in[b ^ 1], io));
            }
            CK(cudaStreamWaitEvent(s, c->ev_in[b], 0));
            if (k >= 2) CK(cudaStreamWaitEvent(s, c->ev_out[b], 0));  // solve k - 2's u has left this buffer
            if (k >= 2) {  // slot b of the control words holds solve k - 2's, read before it is reused
                const mg_status st = collect(k - 2);
                if (st != MG_OK) return st;
            }
            mg_status st;
            if (c->rr) {  // a solve from zero: u zeroed inside the graph
                c->zstart = true;
                st = solve_graph(c, F[b], U[b], rtol, max_cycles, &hit[b]);
                c->zstart = false;
            } else {
                CK(zero_grid(c, U[b], s));
                st = solve_graph(c, F[b], U[b], rtol, max_cycles, &hit[b]);
            }
            if (st != MG_OK) return st;
            CK(cudaGraphLaunch(hit[b]->exec, s));
            CK(cudaMemcpyAsync(&c->hctl[b], c->ctl, sizeof(Ctrl), cudaMemcpyDeviceToHost, s));
            CK(cudaEventRecord(c->ev_ctl[b], s));
            CK(cudaEventRecord(c->ev_sol[b], s));
            // u back once the solve and its control word have left the device: the
            // control word's small copy shares the copy engine, and queued behind
            // this 134 MB one it would hold the next solve back
            CK(cudaStreamWaitEvent(io, c->ev_ctl[b], 0));
            CK(copy_grid(c, u_host[k], U[b], cudaMemcpyDeviceToHost, io));
            CK(cudaEventRecord(c->ev_out[b], io));
        }
        for (int k = std::max(0, count - 2); k < count; k++) {
            const mg_status st = collect(k);
            if (st != MG_OK) return st;
        }
        return MG_OK;
    };
    const mg_status st = pipeline();
    // both streams drained on every path, an error included: no copy this call
    // issued touches the caller's host arrays after it returns
    const cudaError_t e_io = cudaStreamSynchronize(io), e_s = cudaStreamSynchronize(s);
    if (st != MG_OK) return st;
    if (e_io != cudaSuccess || e_s != cudaSuccess)
        return cuda_fail(e_io != cudaSuccess ? e_io : e_s, "mg_solve_host_many streams");
    return worst;
}

// Section 2.4 / 3.4: a fourth-order solution is reached fastest by first
// converging the second-order problem (its V-cycles contract ~10x faster) and
// then running a few cycles on the fourth-order residual.
mg_status mg_solve_two_stage(mg_ctx *c, const double *f, double *u, const double *omega2, double rtol2, double rtol,
                             int max_cycles, int *cycles2_out, int *cycles4_out, double *relres_out, void *stream) {
    if (!c || bad_grid(f) || bad_grid(u) || c->d.order != 4 || !(rtol2 >= 0.0)) return MG_EINVAL;
    double om4[4];
    std::memcpy(om4, c->d.omega, sizeof om4);
    // stage 1: the same levels and schedule with the second-order residual
    c->d.order = 2;
    if (omega2) std::memcpy(c->d.omega, omega2, sizeof om4);
    plan_fast2d(c);
    plan_fast3d(c);
    int cyc2 = 0;
    double rel2 = 0.0;
    mg_status st = mg_solve(c, f, u, rtol2, max_cycles, &cyc2, &rel2, nullptr, stream);
    c->d.order = 4;
    std::memcpy(c->d.omega, om4, sizeof om4);
    plan_fast2d(c);
    plan_fast3d(c);
    if (st != MG_OK && st != MG_ENOCONV) return st;
    int cyc4 = 0;
    st = mg_solve(c, f, u, rtol, max_cycles, &cyc4, relres_out, nullptr, stream);
    if (cycles2_out) *cycles2_out = cyc2;
    if (cycles4_out) *cycles4_out = cyc4;
    return st;
}

mg_status mg_set_omega(mg_ctx *c, const double *omega) {
    if (!c || !omega) return MG_EINVAL;
    for (int q = 0; q < 4; q++)
        if (!std::isfinite(omega[q])) return MG_EINVAL;
    std::memcpy(c->d.omega, omega, sizeof c->d.omega);
    plan_fast2d(c);
    plan_fast3d(c);
    return MG_OK;
}

mg_status mg_set_sweeps(mg_ctx *c, int extra) {
    if (!c || extra < 0 || extra > 64) return MG_EINVAL;
    if (extra > 0 && (c->d.dim != 2 || c->d.hierarchy != MG_DIAG || c->nprob != 1)) return MG_EINVAL;
    c->extra = extra;
    c->rr = c->rr_alloc && extra == 0 && c->gamma == 1;
    plan_fast2d(c);
    return MG_OK;
}

mg_status mg_set_gamma(mg_ctx *c, int gamma) {
    if (!c || gamma < 1 || gamma > 4) return MG_EINVAL;
    if (gamma > 1 && (c->d.hierarchy != MG_DIAG || c->nprob != 1)) return MG_EINVAL;
    const int per = c->d.dim == 2 ? 2 : 3;
    if (gamma > 1 && !c->wpool && c->K >= 2) {  // the first gamma > 1: a kept residual and an accumulator per green level
        size_t total = 0;
        for (int k = 1; k < c->K; k++) total += 2 * ((c->lv[per * k].len * c->esz + 255) / 256 * 256);
        if (cudaMalloc(&c->wpool, total) != cudaSuccess) { cudaGetLastError(); c->wpool = nullptr; return MG_ENOMEM; }
        if (cudaMemset(c->wpool, 0, total) != cudaSuccess) return cuda_fail(cudaGetLastError(), "mg_set_gamma");
        c->wr.assign(c->K, nullptr);
        c->wv.assign(c->K, nullptr);
        char *p = (char *)c->wpool;
        for (int k = 1; k < c->K; k++) {
            const size_t bytes = (c->lv[per * k].len * c->esz + 255) / 256 * 256;
            c->wr[k] = p; p += bytes;
            c->wv[k] = p; p += bytes;
        }
    }
    c->gamma = gamma;
    c->rr = c->rr_alloc && c->extra == 0 && gamma == 1;
    plan_fast2d(c);
    plan_fast3d(c);
    return MG_OK;
}

// Convergence factor of the V-cycle by power iteration on its error
// propagation u <- u + B(0 - L u) (f = 0): the geometric mean of the norm
// ratios of the last (cycles - skip) cycles, u renormalised every cycle.
mg_status mg_rho(mg_ctx *c, const double *zero_f, double *u, int cycles, int skip, double *rho_out, void *stream) {
    if (!c || bad_grid(zero_f) || bad_grid(u) || !rho_out || cycles < 2 || skip < 0 || skip >= cycles || cycles > c->hist_cap ||
        c->nprob != 1)
        return MG_EINVAL;
    cudaStream_t s = S(stream);
    const bool fp64 = c->d.precision == MG_FP64;
    const int n = c->d.n;
    const dim3 g = c->d.dim == 2 ? grid2(n, n) : grid3(n, n, n);
    auto norm_u = [&]() {
        dim3 gn;
        if (c->d.dim == 2) {
            gn = dim3((n + 31) / 32, (n + 8 * RES_ROWS - 1) / (8 * RES_ROWS), 1);
            LAUNCH_B(TAG_CONTROL, (k_norm_f<2>), gn, B2, u, c->d.pitch, n, c->part, (const int *)nullptr);
        } else {
            gn = dim3((n + 31) / 32, (n + 7) / 8, (n + RES3_PLANES - 1) / RES3_PLANES);
            LAUNCH_B(TAG_CONTROL, (k_norm_f<3>), gn, B2, u, c->d.pitch, n, c->part, (const int *)nullptr);
        }
        return (int)(gn.x * gn.y * gn.z);
    };
    if (c->d.order == 4) launch_rhs4(c, zero_f, s);
    int np = norm_u();
    LAUNCH(TAG_CONTROL, (k_rho_record), 1, 1024, c->part, np, c->scal, c->hist, 0);
    LAUNCH(TAG_CONTROL, (k_scale_grid), g, B2, u, c->d.pitch, n, c->d.dim, c->scal);
    for (int q = 0; q < cycles; q++) {
        mg_status st = fp64 ? vcycle_t<double>(c, zero_f, u, nullptr, true, s) : vcycle_t<float>(c, zero_f, u, nullptr, true, s);
        if (st != MG_OK) return st;
        np = norm_u();
        LAUNCH(TAG_CONTROL, (k_rho_record), 1, 1024, c->part, np, c->scal, c->hist, q);
        LAUNCH(TAG_CONTROL, (k_scale_grid), g, B2, u, c->d.pitch, n, c->d.dim, c->scal);
    }
    CKL("mg_rho");
    std::vector<double> ratio(cycles);
    CK(cudaMemcpyAsync(ratio.data(), c->hist, sizeof(double) * cycles, cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    double lg = 0.0;
    for (int q = skip; q < cycles; q++) lg += std::log(std::max(ratio[q], 1e-300));
    *rho_out = std::exp(lg / (cycles - skip));
    return MG_OK;
}

}  // extern "C"

// ---- batches of independent problems --------------------------------------

struct mg_batch {
    int dim = 0, nprob = 0;
    std::vector<int> side;                 // per problem
    std::vector<mg_ctx *> grp;             // one context per distinct side
    std::vector<std::vector<int>> members; // problem ids of each group, in order
    cudaStream_t cs = nullptr;
    cudaEvent_t fork = nullptr;
    std::vector<cudaEvent_t> join;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t gexec = nullptr;
    std::vector<const double *> g_f;
    std::vector<double *> g_u;
    double g_rtol = -1.0;
    int g_max = -1;
    std::vector<Ctrl> host;                // control words read back after a solve
};

extern "C" {

mg_status mg_batch_destroy(mg_batch *b) {
    if (!b) return MG_OK;
    cudaDeviceSynchronize();
    if (b->gexec) cudaGraphExecDestroy(b->gexec);
    if (b->graph) cudaGraphDestroy(b->graph);
    for (auto e : b->join) cudaEventDestroy(e);
    if (b->fork) cudaEventDestroy(b->fork);
    if (b->cs) cudaStreamDestroy(b->cs);
    for (auto c : b->grp) mg_destroy(c);
    delete b;
    return MG_OK;
}

mg_status mg_batch_create(mg_batch **out, int dim, int nprob, const int *n, int hierarchy, int order,
                          int precision, int coarsest, const double *omega) {
    if (!out || !n || nprob < 1 || !omega) return MG_EINVAL;
    *out = nullptr;
    mg_batch *b = new (std::nothrow) mg_batch();
    if (!b) return MG_ENOMEM;
    b->dim = dim;
    b->nprob = nprob;
    b->side.assign(n, n + nprob);
    std::vector<int> sides(b->side);
    std::sort(sides.begin(), sides.end());
    sides.erase(std::unique(sides.begin(), sides.end()), sides.end());
    for (int sd : sides) {
        mg_desc d{};
        d.dim = dim; d.n = sd; d.pitch = sd + 2; d.hierarchy = hierarchy; d.order = order;
        d.precision = precision; d.coarsest = coarsest;
        for (int q = 0; q < 4; q++) d.omega[q] = omega[q];
        std::vector<int> mem;
        for (int p = 0; p < nprob; p++)
            if (b->side[p] == sd) mem.push_back(p);
        mg_ctx *c = nullptr;
        mg_status st = valid_desc(&d) ? create_ctx(&c, &d, (int)mem.size()) : MG_EINVAL;
        if (st != MG_OK) { mg_batch_destroy(b); return st; }
        b->grp.push_back(c);
        b->members.push_back(mem);
    }
    if (cudaStreamCreateWithFlags(&b->cs, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&b->fork, cudaEventDisableTiming) != cudaSuccess) {
        mg_batch_destroy(b);
        return cuda_fail(cudaGetLastError(), "mg_batch_create");
    }
    b->join.resize(b->grp.size());
    for (auto &e : b->join)
        if (cudaEventCreateWithFlags(&e, cudaEventDisableTiming) != cudaSuccess) {
            mg_batch_destroy(b);
            return cuda_fail(cudaGetLastError(), "mg_batch_create");
        }
    *out = b;
    return MG_OK;
}

mg_status mg_solve_batched(mg_batch *b, const double *const *f, double *const *u, double rtol, int max_cycles,
                           int *cycles_out, double *relres_out, void *stream) {
    if (!b || !f || !u || !(rtol >= 0.0) || max_cycles < 0) return MG_EINVAL;
    for (int p = 0; p < b->nprob; p++)
        if (bad_grid(f[p]) || bad_grid(u[p])) return MG_EINVAL;
    for (auto c : b->grp)
        if (max_cycles > c->hist_cap) return MG_EINVAL;
    cudaStream_t s = S(stream);
    const bool same = b->gexec && b->g_rtol == rtol && b->g_max == max_cycles &&
                      std::equal(f, f + b->nprob, b->g_f.begin()) && std::equal(u, u + b->nprob, b->g_u.begin());
    if (!same) {
        // per-group pointer tables, then one graph: a WHILE branch per group
        for (size_t g = 0; g < b->grp.size(); g++) {
            mg_ctx *c = b->grp[g];
            std::vector<const double *> ft;
            std::vector<double *> ut;
            for (int p : b->members[g]) { ft.push_back(f[p]); ut.push_back(u[p]); }
            if (c->nprob > 1) {
                CK(cudaMemcpy(c->ftab, ft.data(), sizeof(double *) * ft.size(), cudaMemcpyHostToDevice));
                CK(cudaMemcpy(c->utab, ut.data(), sizeof(double *) * ut.size(), cudaMemcpyHostToDevice));
            }
        }
        if (b->gexec) { cudaGraphExecDestroy(b->gexec); b->gexec = nullptr; }
        if (b->graph) { cudaGraphDestroy(b->graph); b->graph = nullptr; }
        CK(cudaStreamBeginCapture(b->cs, cudaStreamCaptureModeThreadLocal));
        CK(cudaEventRecord(b->fork, b->cs));
        mg_status st = MG_OK;
        for (size_t g = 0; g < b->grp.size() && st == MG_OK; g++) {
            mg_ctx *c = b->grp[g];
            const int p0 = b->members[g][0];
            if (cudaStreamWaitEvent(c->cs1, b->fork, 0) != cudaSuccess) { st = MG_ECUDA; break; }
            st = capture_solve(c, f[p0], u[p0], rtol, max_cycles, c->cs1, c->cs2);
            if (st == MG_OK && (cudaEventRecord(b->join[g], c->cs1) != cudaSuccess ||
                                cudaStreamWaitEvent(b->cs, b->join[g], 0) != cudaSuccess))
                st = MG_ECUDA;
        }
        cudaGraph_t graph = nullptr;
        const cudaError_t e = cudaStreamEndCapture(b->cs, &graph);
        if (st != MG_OK) { if (graph) cudaGraphDestroy(graph); return st == MG_ECUDA ? cuda_fail(cudaGetLastError(), "mg_solve_batched capture") : st; }
        if (e != cudaSuccess) return cuda_fail(e, "mg_solve_batched capture");
        b->graph = graph;
        CK(cudaGraphInstantiate(&b->gexec, graph, 0));
        b->g_f.assign(f, f + b->nprob);
        b->g_u.assign(u, u + b->nprob);
        b->g_rtol = rtol;
        b->g_max = max_cycles;
    }
    CK(cudaGraphLaunch(b->gexec, s));
    b->host.resize(b->nprob);
    bool diverged = false, noconv = false;
    for (size_t g = 0; g < b->grp.size(); g++) {
        mg_ctx *c = b->grp[g];
        std::vector<Ctrl> ctl(c->nprob);
        CK(cudaMemcpyAsync(ctl.data(), c->ctl, sizeof(Ctrl) * c->nprob, cudaMemcpyDeviceToHost, s));
        CK(cudaStreamSynchronize(s));
        int maxc = 0;
        for (int q = 0; q < c->nprob; q++) {
            const int p = b->members[g][q];
            b->host[p] = ctl[q];
            maxc = std::max(maxc, ctl[q].cycles);
            if (cycles_out) cycles_out[p] = ctl[q].cycles;
            if (relres_out) relres_out[p] = ctl[q].relres;
            diverged |= ctl[q].status == -5;
            noconv |= ctl[q].status == -4 || !ctl[q].done;
        }
        c->launches += c->g_prefix_kernels + (long long)maxc * c->g_body_kernels;
    }
    if (diverged) return MG_EDIVERGED;
    if (noconv) return MG_ENOCONV;
    return MG_OK;
}

mg_status mg_batch_status(const mg_batch *b, int *status) {
    if (!b || !status) return MG_EINVAL;
    if ((int)b->host.size() != b->nprob) return MG_EINVAL;  // no solve yet
    for (int p = 0; p < b->nprob; p++) {
        const Ctrl &h = b->host[p];
        status[p] = h.status == -5 ? MG_EDIVERGED : (h.status == -4 || !h.done) ? MG_ENOCONV : MG_OK;
    }
    return MG_OK;
}

mg_status mg_batch_launch_count(const mg_batch *b, long long *launches) {
    if (!b || !launches) return MG_EINVAL;
    long long t = 0;
    for (auto c : b->grp) t += c->launches;
    *launches = t;
    return MG_OK;
}

}  // extern "C"

// ---- autotuning -------------------------------------------------------------

namespace {

std::string tune_key(const mg_ctx *c) {
    cudaDeviceProp pr{};
    cudaGetDeviceProperties(&pr, c->dev);
    char buf[400];
    // "kernels": the version of the tunable kernel set (classes change meaning with it)
    std::snprintf(buf, sizeof buf, "\"kernels\": 3, \"device\": \"%s\", \"dim\": %d, \"n\": %d, \"hier\": %d, \"prec\": %d, \"nprob\": %d",
                  pr.name, c->d.dim, c->d.n, c->d.hierarchy, c->d.precision, c->nprob);
    return buf;
}

int ntiles(const mg_ctx *c) { return c->fast2d ? c->kd : 0; }

// one JSON object per line: {<key>, "cut": C, "down": [..], "up": [..]}
bool cache_lookup(const char *path, const std::string &key, mg_ctx *c) {
    FILE *fp = std::fopen(path, "r");
    if (!fp) return false;
    char line[2048];
    bool found = false;
    while (std::fgets(line, sizeof line, fp)) {
        if (!std::strstr(line, key.c_str())) continue;
        const char *q = std::strstr(line, "\"cut\": ");
        if (!q) continue;
        int cut = std::atoi(q + 7);
        const char *qc = std::strstr(line, "\"cl\": ");
        if (qc) c->cl_top = std::atoi(qc + 6);
        int dn[32], upv[32], ndn = 0, nup = 0;
        auto read_list = [&](const char *name, int *out, int &cnt) {
            const char *r = std::strstr(line, name);
            if (!r) return;
            r = std::strchr(r, '[');
            if (!r) return;
            r++;
            while (*r && *r != ']' && cnt < 32) {
                char *end = nullptr;
                long v = std::strtol(r, &end, 10);
                if (end == r) break;
                out[cnt++] = (int)v;
                r = end;
                while (*r == ',' || *r == ' ') r++;
            }
        };
        read_list("\"down\"", dn, ndn);
        read_list("\"up\"", upv, nup);
        c->cut_side = cut;
        for (int q2 = 0; q2 < 32; q2++) c->tile_dn[q2] = c->tile_up[q2] = -1;
        for (int q2 = 0; q2 < ndn; q2++) c->tile_dn[q2] = dn[q2];
        for (int q2 = 0; q2 < nup; q2++) c->tile_up[q2] = upv[q2];
        found = true;
    }
    std::fclose(fp);
    return found;
}

void cache_append(const char *path, const std::string &key, const mg_ctx *c) {
    FILE *fp = std::fopen(path, "a");
    if (!fp) return;
    std::fprintf(fp, "{%s, \"cut\": %d, \"cl\": %d, \"down\": [", key.c_str(), c->cut_side, c->cl_top);
    for (int k = 0; k < ntiles(c); k++) std::fprintf(fp, "%s%d", k ? ", " : "", c->tile_dn[k]);
    std::fprintf(fp, "], \"up\": [");
    for (int k = 0; k < ntiles(c); k++) std::fprintf(fp, "%s%d", k ? ", " : "", c->tile_up[k]);
    std::fprintf(fp, "]}\n");
    std::fclose(fp);
}

void replan(mg_ctx *c) {
    plan_fast2d(c);
    plan_fast3d(c);
    drop_solve_graphs(c);
}

// Measure and apply: the coarse-block cut-off by whole V-cycles, then the tile
// class of every pair kernel by timing it alone on the context's buffers.
mg_status tune_measure(mg_ctx *c, const double *f, double *u, cudaStream_t s) {
    const bool fp64 = c->d.precision == MG_FP64;
    cudaEvent_t e0, e1;
    CK(cudaEventCreate(&e0));
    CK(cudaEventCreate(&e1));
    // the time of fn, or +inf when a launch of it failed (e.g. a shared-
    // memory plan this device cannot give): never chosen
    auto timeit = [&](auto fn, int reps) {
        cudaGetLastError();
        fn();
        cudaEventRecord(e0, s);
        for (int q = 0; q < reps; q++) fn();
        cudaEventRecord(e1, s);
        cudaEventSynchronize(e1);
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        return cudaGetLastError() == cudaSuccess ? ms / reps : 1e30f;
    };
    auto vcyc = [&]() {
        if (fp64) vcycle_t<double>(c, f, u, nullptr, true, s);
        else vcycle_t<float>(c, f, u, nullptr, true, s);
    };
    vcyc();  // realistic contents in every level buffer
    std::vector<int> cuts = c->fast2d ? std::vector<int>{15, 31, 63} : std::vector<int>{7, 15};
    // 2D: with the middle pairs in the cluster kernel (largest side 255) and without
    std::vector<int> tops = c->fast2d && c->cl_ok ? std::vector<int>{0, 255} : std::vector<int>{c->cl_top};
    int best_cut = 0, best_top = c->cl_top;
    float best = 1e30f;
    for (int top : tops)
        for (int cut : cuts) {
            c->cl_top = top;
            c->cut_side = cut;
            replan(c);
            const float ms = timeit(vcyc, 5);
            if (ms < best) { best = ms; best_cut = cut; best_top = top; }
        }
    c->cl_top = best_top;
    c->cut_side = best_cut;
    replan(c);
    if (c->fast2d) {
        for (int k = 0; k < c->kd && k < 32; k++) {
            float bd = 1e30f, bu = 1e30f;
            const int ncls = fp64 ? 3 : NCLS_FP32;
            for (int cls = 0; cls < ncls; cls++) {
                const float md = fp64 ? timeit([&] { down_pair<double>(c, k, cls, nullptr, s, false); }, 5)
                                      : timeit([&] { down_pair<float>(c, k, cls, nullptr, s, false); }, 5);
                if (md < bd) { bd = md; c->tile_dn[k] = cls; }
                float mu;
                if (k == 0 && c->rr) {
                    if (cls >= 3) continue;  // the fused finest pair exists only as a streaming kernel
                    mu = timeit([&] { launch_up_ff(c, 0, cls, u, nullptr, s, true); }, 5);
                } else {
                    mu = fp64 ? timeit([&] { up_pair<double>(c, k, cls, k == 0 ? u : nullptr, nullptr, s); }, 5)
                              : timeit([&] { up_pair<float>(c, k, cls, k == 0 ? u : nullptr, nullptr, s); }, 5);
                }
                if (mu < bu) { bu = mu; c->tile_up[k] = cls; }
            }
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    CKL("mg_tune");
    return MG_OK;
}

mg_status zero_u(mg_ctx *c, double *u, cudaStream_t s) {
    const size_t rows = (size_t)(c->d.n + 2) * (c->d.dim == 3 ? (size_t)(c->d.n + 2) : 1);
    CK(cudaMemset2DAsync(u, sizeof(double) * c->d.pitch, 0, sizeof(double) * (c->d.n + 2), rows, s));
    return MG_OK;
}

}  // namespace

extern "C" {

mg_status mg_tune(mg_ctx *c, const double *f, double *u, const char *cache_path, int *measured_out, void *stream) {
    if (!c || bad_grid(f) || bad_grid(u)) return MG_EINVAL;
    if (measured_out) *measured_out = 0;
    if (!c->fast2d && !c->fast3d) return MG_OK;  // nothing tunable on this path
    const char *path = cache_path ? cache_path : std::getenv("DIAGMG_TUNE_CACHE");
    const std::string key = tune_key(c);
    if (path && cache_lookup(path, key, c)) {
        replan(c);
        return MG_OK;
    }
    cudaStream_t s = S(stream);
    mg_status st = tune_measure(c, f, u, s);
    if (st != MG_OK) return st;
    st = zero_u(c, u, s);
    if (st != MG_OK) return st;
    CK(cudaStreamSynchronize(s));
    if (path) cache_append(path, key, c);
    if (measured_out) *measured_out = 1;
    return MG_OK;
}

mg_status mg_tune_info(const mg_ctx *c, int *cut_side, int *npairs, int *tiles_down, int *tiles_up) {
    if (!c) return MG_EINVAL;
    if (cut_side) *cut_side = c->cut_side;
    if (npairs) *npairs = ntiles(c);
    for (int k = 0; k < ntiles(c); k++) {
        if (tiles_down) tiles_down[k] = tile_dn(c, k);
        if (tiles_up) tiles_up[k] = tile_up(c, k);
    }
    return MG_OK;
}

mg_status mg_batch_tune(mg_batch *b, const double *const *f, double *const *u, const char *cache_path,
                        void *stream) {
    if (!b || !f || !u) return MG_EINVAL;
    for (int p = 0; p < b->nprob; p++)
        if (bad_grid(f[p]) || bad_grid(u[p])) return MG_EINVAL;
    cudaStream_t s = S(stream);
    for (size_t g = 0; g < b->grp.size(); g++) {
        mg_ctx *c = b->grp[g];
        std::vector<const double *> ft;
        std::vector<double *> ut;
        for (int p : b->members[g]) { ft.push_back(f[p]); ut.push_back(u[p]); }
        if (c->nprob > 1) {
            CK(cudaMemcpy(c->ftab, ft.data(), sizeof(double *) * ft.size(), cudaMemcpyHostToDevice));
            CK(cudaMemcpy(c->utab, ut.data(), sizeof(double *) * ut.size(), cudaMemcpyHostToDevice));
        }
        if (!c->fast2d && !c->fast3d) continue;
        const char *path = cache_path ? cache_path : std::getenv("DIAGMG_TUNE_CACHE");
        const std::string key = tune_key(c);
        if (path && cache_lookup(path, key, c)) {
            replan(c);
            continue;
        }
        mg_status st = tune_measure(c, ft[0], ut[0], s);
        if (st != MG_OK) return st;
        for (double *up : ut) {
            st = zero_u(c, up, s);
            if (st != MG_OK) return st;
        }
        CK(cudaStreamSynchronize(s));
        if (path) cache_append(path, key, c);
    }
    if (b->gexec) { cudaGraphExecDestroy(b->gexec); b->gexec = nullptr; }
    if (b->graph) { cudaGraphDestroy(b->graph); b->graph = nullptr; }
    return MG_OK;
}

mg_status mg_launch_count(const mg_ctx *c, long long *launches) {
    if (!c || !launches) return MG_EINVAL;
    *launches = c->launches;
    return MG_OK;
}

mg_status mg_probe_set(mg_ctx *c, int family) {
    if (!c || family < -1 || family > 6) return MG_EINVAL;
    if (family >= 0 && c->pev.empty()) {
        c->pev.resize(1024);
        for (auto &e : c->pev) CK(cudaEventCreate(&e));
    }
    c->probe_tag = family;
    c->pev_used = 0;
    c->probe_n = 0;
    c->probe_ms = 0.0;
    return MG_OK;
}

mg_status mg_probe_read(mg_ctx *c, long long *launches, double *ms, void *stream) {
    if (!c) return MG_EINVAL;
    CK(cudaStreamSynchronize(S(stream)));
    probe_collect(c);
    if (launches) *launches = c->probe_n;
    if (ms) *ms = c->probe_ms;
    return MG_OK;
}

mg_status mg_fp64_rate(mg_ctx *c, double *ops_per_s, void *stream) {
    if (!c || !ops_per_s) return MG_EINVAL;
    cudaStream_t s = S(stream);
    int sms = 0;
    CK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, c->dev));
    const int blocks = 4 * sms, threads = 256, iters = 4096;
    cudaEvent_t e0, e1;
    CK(cudaEventCreate(&e0));
    if (cudaEventCreate(&e1) != cudaSuccess) { cudaEventDestroy(e0); return cuda_fail(cudaGetLastError(), "mg_fp64_rate"); }
    double best = 0.0;
    cudaError_t err = cudaSuccess;
    for (int rep = 0; rep < 4 && err == cudaSuccess; rep++) {
        cudaEventRecord(e0, s);
        k_dfma_rate<<<blocks, threads, 0, s>>>(1.0 + rep, iters, c->scal);
        cudaEventRecord(e1, s);
        err = cudaEventSynchronize(e1);
        float ms = 0.f;
        if (err == cudaSuccess) err = cudaEventElapsedTime(&ms, e0, e1);
        if (err == cudaSuccess && rep > 0 && ms > 0.f)  // the first launch is a warm-up
            best = std::max(best, (double)blocks * threads * iters * DFMA_CHAINS / (ms * 1e-3));
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (err != cudaSuccess) return cuda_fail(err, "mg_fp64_rate");
    *ops_per_s = best;
    return MG_OK;
}

}  // extern "C"
