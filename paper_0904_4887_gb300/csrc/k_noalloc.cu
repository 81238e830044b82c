// gp_residual_noalloc: the FP64 residual and its norm without any device
// allocation, for callers that cannot call cudaMalloc (see include/gp.h).
//
// The reduction scratch (per-z-plane partial sums) lives in one file-scope
// __device__ array. Host code may not use that array's name as a device
// address, so the address is looked up once per device with
// cudaGetSymbolAddress and cached.
#include "gp_common.cuh"

#include <mutex>

namespace gp {
namespace {

constexpr int kNoallocMaxPlanes = GP_NOALLOC_MAX_PLANES;

// two partial sums per z-plane: sum r^2 and sum b^2
static __device__ __align__(256) double g_noalloc_scratch[2 * kNoallocMaxPlanes];

constexpr int kMaxDevices = 64;
std::mutex g_mutex;
double* g_scratch_ptr[kMaxDevices] = {};

// One block per z-plane: r = -4 pi rho - A phi with the FP64 7-point operator
// (cell eps, arithmetic face means, periodic), and the plane's sums of r^2
// and b^2 written to its own scratch slots (every slot is overwritten, so no
// state from an earlier call is read).
__global__ void __launch_bounds__(256) k_residual64_planes(Geo g, const double* phi, const double* rho,
                                                           const double* eps, double* r_out, double* scratch) {
    __shared__ double red[2][256];
    const int k = blockIdx.x;
    const long pl = (long)g.nx * g.ny;
    const double hx = g.c2x, hy = g.c2y, hz = g.c2z;
    const double fpi = 4.0 * kPi;
    const long zm = (k == 0 ? (long)(g.nz - 1) : -1L) * pl;
    const long zp = (k == g.nz - 1 ? -(long)(g.nz - 1) : 1L) * pl;
    double s2 = 0.0, b2 = 0.0;
    for (long q = threadIdx.x; q < pl; q += blockDim.x) {
        const int i = (int)(q % g.nx), j = (int)(q / g.nx);
        const long c = k * pl + q;
        const long xm = c + (i == 0 ? g.nx - 1 : -1), xp = c + (i == g.nx - 1 ? 1 - g.nx : 1);
        const long ym = c + (j == 0 ? (long)(g.ny - 1) * g.nx : -(long)g.nx);
        const long yp = c + (j == g.ny - 1 ? -(long)(g.ny - 1) * g.nx : (long)g.nx);
        const double e0 = eps[c], p0 = phi[c];
        const double ax = (e0 + eps[xp]) * (phi[xp] - p0) - (e0 + eps[xm]) * (p0 - phi[xm]);
        const double ay = (e0 + eps[yp]) * (phi[yp] - p0) - (e0 + eps[ym]) * (p0 - phi[ym]);
        const double az = (e0 + eps[c + zp]) * (phi[c + zp] - p0) - (e0 + eps[c + zm]) * (p0 - phi[c + zm]);
        const double b = -fpi * rho[c];
        const double r = b - (hx * ax + hy * ay + hz * az);
        r_out[c] = r;
        s2 += r * r;
        b2 += b * b;
    }
    red[0][threadIdx.x] = s2;
    red[1][threadIdx.x] = b2;
    __syncthreads();
    for (int s = blockDim.x / 2; s > 0; s >>= 1) {
        if (threadIdx.x < s) {
            red[0][threadIdx.x] += red[0][threadIdx.x + s];
            red[1][threadIdx.x] += red[1][threadIdx.x + s];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        scratch[k] = red[0][0];
        scratch[kNoallocMaxPlanes + k] = red[1][0];
    }
}

// rel = sqrt(sum r^2 / sum b^2) over the planes, summed in plane order
__global__ void k_noalloc_finish(int nz, const double* scratch, double* rel_dev) {
    __shared__ double red[2][256];
    double a = 0.0, b = 0.0;
    for (int k = threadIdx.x; k < nz; k += blockDim.x) {
        a += scratch[k];
        b += scratch[kNoallocMaxPlanes + k];
    }
    red[0][threadIdx.x] = a;
    red[1][threadIdx.x] = b;
    __syncthreads();
    for (int s = blockDim.x / 2; s > 0; s >>= 1) {
        if (threadIdx.x < s) {
            red[0][threadIdx.x] += red[0][threadIdx.x + s];
            red[1][threadIdx.x] += red[1][threadIdx.x + s];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) rel_dev[0] = red[1][0] > 0.0 ? sqrt(red[0][0] / red[1][0]) : sqrt(red[0][0]);
}

// address of the scratch array on the current device, looked up once per device
cudaError_t scratch_address(double** out) {
    int dev = -1;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lock(g_mutex);
    if (!g_scratch_ptr[dev]) {
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess) return e;
        g_scratch_ptr[dev] = static_cast<double*>(p);
    }
    *out = g_scratch_ptr[dev];
    return cudaSuccess;
}

}  // namespace
}  // namespace gp

extern "C" gp_status gp_residual_noalloc(gp_grid grid, gp_cell cell, const double* eps_dev, const double* rho_dev,
                                         const double* phi_dev, double* r_dev, double* rel_dev, void* cuda_stream) {
    using namespace gp;
    if (!eps_dev || !rho_dev || !phi_dev || !r_dev || !rel_dev) return GP_ERR_INVALID_ARG;
    if (grid.nx < 2 || grid.ny < 2 || grid.nz < 2) return GP_ERR_INVALID_ARG;
    if (grid.nz > kNoallocMaxPlanes) return GP_ERR_INVALID_ARG;
    if (!(cell.lx > 0 && cell.ly > 0 && cell.lz > 0)) return GP_ERR_INVALID_ARG;
    double* scratch = nullptr;
    if (scratch_address(&scratch) != cudaSuccess) return GP_ERR_CUDA;
    const Geo g = make_geo(grid.nx, grid.ny, grid.nz, cell.lx, cell.ly, cell.lz);
    cudaStream_t s = reinterpret_cast<cudaStream_t>(cuda_stream);
    k_residual64_planes<<<grid.nz, 256, 0, s>>>(g, phi_dev, rho_dev, eps_dev, r_dev, scratch);
    k_noalloc_finish<<<1, 256, 0, s>>>(grid.nz, scratch, rel_dev);
    return cudaGetLastError() == cudaSuccess ? GP_OK : GP_ERR_CUDA;
}
