// mg_noalloc.cu -- mg_residual_noalloc: the finest-grid residual and its
// squared norm with no device allocation at all (no context, no cudaMalloc).
//
// Who needs it: callers that may not allocate device memory themselves --
// code that runs inside another framework's allocator or fixed memory budget
// (where every byte of device memory is handed out by that framework), code
// in latency-critical loops where cudaMalloc/cudaFree could stall or
// synchronise the device, and plug-ins that must not keep workspace between
// calls.  Such a caller passes its own f, u and output buffers; the only
// scratch -- one partial sum per thread block -- lives in a fixed-size array
// that is part of this library's image on every GPU that loads it.
#include <cmath>
#include <mutex>

#include "../../include/diagmg.h"

namespace {

// One FP64 partial sum per thread block of the residual kernel.  512 KiB on
// every device that loads the library, held until the process exits.
constexpr int kMaxBlocks = 65536;
static __device__ __align__(256) double g_noalloc_partials[kMaxBlocks];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
double *g_partials_addr[kMaxDevices] = {};  // device address of the array, per device

__device__ __forceinline__ double block_sum256(double v, double *sh) {
    const int tid = threadIdx.x + blockDim.x * threadIdx.y;
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    if ((tid & 31) == 0) sh[tid >> 5] = v;
    __syncthreads();
    if (tid < 32) {
        v = tid < 8 ? sh[tid] : 0.0;
        for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    }
    return v;
}

// r = f - L u with the 5/7-point Laplacian (ORDER 2) or the compact fourth-
// order forms (ORDER 4); one interior point per thread, block 32x8, grid z =
// planes (3D).  Writes r (if not null) and the block's sum of r^2 to part[].
template <int DIM, int ORDER>
__global__ void __launch_bounds__(256) k_res_noalloc(const double *__restrict__ f, const double *__restrict__ u,
                                                     int pitch, int n, double ih2, double *r, double *part) {
    __shared__ double sh[8];
    const int i = blockIdx.x * 32 + threadIdx.x + 1, j = blockIdx.y * 8 + threadIdx.y + 1;
    const int k = DIM == 3 ? blockIdx.z + 1 : 0;
    double sq = 0.0;
    if (i <= n && j <= n) {
        const size_t pl = (size_t)pitch * (n + 2);
        const size_t c = (DIM == 3 ? k * pl : 0) + (size_t)j * pitch + i;
        double res;
        if (DIM == 2) {
            const double ax = (u[c - 1] + u[c + 1]) + (u[c - pitch] + u[c + pitch]);
            if (ORDER == 2) {
                res = fma(-ih2, ax - 4.0 * u[c], f[c]);
            } else {
                const double ft = (8.0 * f[c] + ((f[c - 1] + f[c + 1]) + (f[c - pitch] + f[c + pitch]))) * (1.0 / 12.0);
                const double dg = (u[c - pitch - 1] + u[c - pitch + 1]) + (u[c + pitch - 1] + u[c + pitch + 1]);
                res = fma(-ih2 * (1.0 / 6.0), fma(4.0, ax, dg) - 20.0 * u[c], ft);
            }
        } else {
            const double ax = ((u[c - 1] + u[c + 1]) + (u[c - pitch] + u[c + pitch])) + (u[c - pl] + u[c + pl]);
            if (ORDER == 2) {
                res = fma(-ih2, ax - 6.0 * u[c], f[c]);
            } else {
                const double ft = (6.0 * f[c] + ((f[c - 1] + f[c + 1]) + (f[c - pitch] + f[c + pitch]) +
                                                 (f[c - pl] + f[c + pl]))) * (1.0 / 12.0);
                const double ed = ((u[c - pitch - 1] + u[c - pitch + 1]) + (u[c + pitch - 1] + u[c + pitch + 1])) +
                                  ((u[c - pl - pitch] + u[c - pl + pitch]) + (u[c + pl - pitch] + u[c + pl + pitch])) +
                                  ((u[c - pl - 1] + u[c - pl + 1]) + (u[c + pl - 1] + u[c + pl + 1]));
                res = fma(-ih2 * (1.0 / 6.0), fma(2.0, ax, ed) - 24.0 * u[c], ft);
            }
        }
        if (r) r[c] = res;
        sq = res * res;
    }
    const double s = block_sum256(sq, sh);
    if (threadIdx.x == 0 && threadIdx.y == 0) part[blockIdx.x + gridDim.x * (blockIdx.y + gridDim.y * blockIdx.z)] = s;
}

// sum of part[0..nblk) in a fixed order by one block of 256 threads
__global__ void __launch_bounds__(256) k_sum_noalloc(const double *part, int nblk, double *out) {
    __shared__ double sh[8];
    double v = 0.0;
    for (int q = threadIdx.x; q < nblk; q += 256) v += part[q];
    v = block_sum256(v, sh);
    if (threadIdx.x == 0) *out = v;
}

int log2_side(int n) {
    if (n < 1) return -1;
    long v = (long)n + 1;
    int m = 0;
    while ((v & 1) == 0) { v >>= 1; m++; }
    return v == 1 ? m : -1;
}


}  // namespace

extern "C" mg_status mg_residual_noalloc(int dim, int n, int pitch, double h, int order, const double *f,
                                         const double *u, double *r, double *norm2, void *stream) {
    if (dim != 2 && dim != 3) return MG_EINVAL;
    if (log2_side(n) < 1 || pitch < n + 2 || (order != 2 && order != 4) || !f || !u) return MG_EINVAL;
    // FP64 element boundaries (8 bytes) for every grid pointer
    if (((uintptr_t)f | (uintptr_t)u | (uintptr_t)r) & 7u) return MG_EINVAL;
    // r is written while neighbouring threads still read f and u: the
    // extents of the full grids must not overlap
    if (r) {
        const size_t len = (size_t)pitch * (n + 2) * (dim == 3 ? (size_t)(n + 2) : 1);
        auto overlap = [len](const double *a, const double *b) { return a < b + len && b < a + len; };
        if (overlap(r, f) || overlap(r, u)) return MG_EINVAL;
    }
    if (!(h > 0.0) || std::fabs(h - 1.0 / (n + 1)) > 1e-15 / (n + 1)) return MG_EINVAL;
    // the size limit of the static scratch: one partial sum per thread block
    const long long nblk = (long long)((n + 31) / 32) * ((n + 7) / 8) * (dim == 3 ? n : 1);
    if (nblk > kMaxBlocks) return MG_EINVAL;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return MG_ECUDA;
    if (dev < 0 || dev >= kMaxDevices) return MG_EINVAL;
    double *part = nullptr;
    {
        // first call on this device: look up the array's device address with
        // the device current (the host-side name is not a device address).
        // The address is kept for the life of the process: after a
        // cudaDeviceReset the module is reloaded and this copy would be stale,
        // so resetting a device after its first call is not supported.
        std::lock_guard<std::mutex> lock(g_mu);
        if (!g_partials_addr[dev]) {
            void *p = nullptr;
            const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_partials);
            if (e != cudaSuccess || !p) return MG_ECUDA;
            g_partials_addr[dev] = (double *)p;
        }
        part = g_partials_addr[dev];
    }
    cudaStream_t s = (cudaStream_t)stream;
    const dim3 block(32, 8, 1), grid((n + 31) / 32, (n + 7) / 8, dim == 3 ? n : 1);
    const double ih2 = 1.0 / (h * h);
    if (dim == 2) {
        if (order == 2) k_res_noalloc<2, 2><<<grid, block, 0, s>>>(f, u, pitch, n, ih2, r, part);
        else k_res_noalloc<2, 4><<<grid, block, 0, s>>>(f, u, pitch, n, ih2, r, part);
    } else {
        if (order == 2) k_res_noalloc<3, 2><<<grid, block, 0, s>>>(f, u, pitch, n, ih2, r, part);
        else k_res_noalloc<3, 4><<<grid, block, 0, s>>>(f, u, pitch, n, ih2, r, part);
    }
    if (norm2) k_sum_noalloc<<<1, 256, 0, s>>>(part, (int)nblk, norm2);
    return cudaGetLastError() == cudaSuccess ? MG_OK : MG_ECUDA;
}
