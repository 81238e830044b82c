// Residual of the sixth-order non-conservative operator (Sec. III, Eq. 16-18).
//
// Eq. 16 expands Eq. 3 by the product rule, grad(eps).grad(phi) + eps lap(phi),
// and Eq. 17-18 take each derivative with seven points along its axis:
//   D1 u = (1/h)   sum_{n=1..3} a_n (u_{i+n} - u_{i-n}),
//   D2 u = (1/h^2) (b_0 u_i + sum_{n=1..3} b_n (u_{i+n} + u_{i-n})),
// a = (3/4, -3/20, 1/60), b = (-49/18, 3/2, -3/20, 1/90): the seven-point
// central weights, truncation O(h^6). Per axis the operator is
//   (1/h^2) [S1(eps) S1(phi) + eps_i S2(phi)]
// with S1, S2 the weighted sums above, so one 1/h^2 per axis carries both terms.
//
// The periodic operator is not conservative, so the solve that uses it carries
// a compatibility shift mu eps on the left side (A6 phi + mu eps = b); the
// residual here is r = b - A6 phi - mu eps with b = -4 pi rho.
#include "gp_common.cuh"

namespace gp {
namespace {

constexpr double kA1 = 3.0 / 4.0, kA2 = -3.0 / 20.0, kA3 = 1.0 / 60.0;
constexpr double kB0 = -49.0 / 18.0, kB1 = 27.0 / 18.0, kB2 = -27.0 / 180.0, kB3 = 2.0 / 180.0;

__device__ __forceinline__ double fd6_block_sum(double v, double* red) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    if (l == 0) red[w] = v;
    __syncthreads();
    double s = 0.0;
    if (threadIdx.x < 32) {
        s = (threadIdx.x < (blockDim.x >> 5)) ? red[threadIdx.x] : 0.0;
        for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    }
    return s;   // valid in thread 0
}

__device__ __forceinline__ int wrap_up(int v, int n) { return v >= n ? v - n : v; }
__device__ __forceinline__ int wrap_down(int v, int n) { return v < 0 ? v + n : v; }

// one axis: (S1(eps) S1(phi) + eps_c S2(phi)); m[n-1] / p[n-1] are the flat
// indices of the points n steps below / above along the axis
__device__ __forceinline__ double axis_term(const double* __restrict__ phi, const double* __restrict__ eps,
                                            double p0, double e0, const long* m, const long* p) {
    const double pm1 = __ldg(phi + m[0]), pp1 = __ldg(phi + p[0]);
    const double pm2 = __ldg(phi + m[1]), pp2 = __ldg(phi + p[1]);
    const double pm3 = __ldg(phi + m[2]), pp3 = __ldg(phi + p[2]);
    const double em1 = __ldg(eps + m[0]), ep1 = __ldg(eps + p[0]);
    const double em2 = __ldg(eps + m[1]), ep2 = __ldg(eps + p[1]);
    const double em3 = __ldg(eps + m[2]), ep3 = __ldg(eps + p[2]);
    const double s1p = kA1 * (pp1 - pm1) + kA2 * (pp2 - pm2) + kA3 * (pp3 - pm3);
    const double s1e = kA1 * (ep1 - em1) + kA2 * (ep2 - em2) + kA3 * (ep3 - em3);
    const double s2p = kB0 * p0 + kB1 * (pp1 + pm1) + kB2 * (pp2 + pm2) + kB3 * (pp3 + pm3);
    return s1e * s1p + e0 * s2p;
}

// r = -4 pi rho - A6 phi - mu eps on the periodic box (FP64);
// partial[b] = block b's sum of r^2. Every block writes its partial, so the
// launch must have exactly kReduceBlocks blocks. Extents are >= 8, so one
// conditional add or subtract wraps each offset of at most 3.
__global__ void __launch_bounds__(kReduceThreads) k_residual6(Geo g, const double* __restrict__ phi,
                                                              const double* __restrict__ rho,
                                                              const double* __restrict__ eps, double mu,
                                                              double* __restrict__ r_out,
                                                              double* __restrict__ partial) {
    __shared__ double red[32];
    const int nx = g.nx, ny = g.ny, nz = g.nz;
    const long plane = (long)nx * ny;
    const double ihx2 = g.ihx * g.ihx, ihy2 = g.ihy * g.ihy, ihz2 = g.ihz * g.ihz;
    const double fpi = 4.0 * kPi;
    double s2 = 0.0;
    for (long row = blockIdx.x; row < (long)ny * nz; row += gridDim.x) {
        const int j = (int)(row % ny), k = (int)(row / ny);
        const long base = (long)k * plane + (long)j * nx;
        long ym[3], yp[3], zm[3], zp[3];   // row starts n = 1..3 below / above in y and z
        for (int n = 1; n <= 3; ++n) {
            ym[n - 1] = (long)k * plane + (long)wrap_down(j - n, ny) * nx;
            yp[n - 1] = (long)k * plane + (long)wrap_up(j + n, ny) * nx;
            zm[n - 1] = (long)wrap_down(k - n, nz) * plane + (long)j * nx;
            zp[n - 1] = (long)wrap_up(k + n, nz) * plane + (long)j * nx;
        }
        for (int i = threadIdx.x; i < nx; i += blockDim.x) {
            const long c = base + i;
            long m[3], p[3];
            const double p0 = __ldg(phi + c), e0 = __ldg(eps + c);
            for (int n = 1; n <= 3; ++n) {
                m[n - 1] = base + wrap_down(i - n, nx);
                p[n - 1] = base + wrap_up(i + n, nx);
            }
            const double ax = axis_term(phi, eps, p0, e0, m, p);
            for (int n = 0; n < 3; ++n) {
                m[n] = ym[n] + i;
                p[n] = yp[n] + i;
            }
            const double ay = axis_term(phi, eps, p0, e0, m, p);
            for (int n = 0; n < 3; ++n) {
                m[n] = zm[n] + i;
                p[n] = zp[n] + i;
            }
            const double az = axis_term(phi, eps, p0, e0, m, p);
            const double r = -fpi * __ldg(rho + c) - (ihx2 * ax + ihy2 * ay + ihz2 * az) - mu * e0;
            r_out[c] = r;
            s2 += r * r;
        }
    }
    const double s = fd6_block_sum(s2, red);
    if (threadIdx.x == 0) partial[blockIdx.x] = s;
}

}  // namespace

void launch_residual6(const Geo& g, const double* phi, const double* rho, const double* eps64, double mu,
                      double* r_out, double* partial, cudaStream_t s) {
    k_residual6<<<kReduceBlocks, kReduceThreads, 0, s>>>(g, phi, rho, eps64, mu, r_out, partial);
}

}  // namespace gp
