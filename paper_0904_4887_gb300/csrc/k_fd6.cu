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

// ---------------------------------------------------------------- the solve, its adjoint, the forces
// The periodic sixth-order operator needs the bordered system
//   A6 phi + mu eps = b,  sum(phi) = 0          (b = -4 pi (rho - mean rho))
// and, for the forces, its transpose
//   A6^T lam + nu 1 = rho - mean rho,  sum(eps lam) = 0.
// The solver eliminates the border: with P v = v - (sum v / sum eps) eps (or
// Q v = v - mean(v) for the transpose) the unknown field solves P A6 phi = P b
// on zero-mean fields (Q A6^T lam = Q rho on fields with sum(eps lam) = 0), and
// mu (nu) is the removed multiple. The kernels below are its pieces, FP64.

// grid-stride over rows with one block-sum per block, as k_residual6
#define FD6_ROWS_BEGIN                                                             \
    const int nx = g.nx, ny = g.ny, nz = g.nz;                                     \
    const long plane = (long)nx * ny;                                              \
    for (long row = blockIdx.x; row < (long)ny * nz; row += gridDim.x) {           \
        const int j = (int)(row % ny), k = (int)(row / ny);                        \
        const long base = (long)k * plane + (long)j * nx;                          \
        long ym[3], yp[3], zm[3], zp[3];                                           \
        for (int n = 1; n <= 3; ++n) {                                             \
            ym[n - 1] = (long)k * plane + (long)wrap_down(j - n, ny) * nx;         \
            yp[n - 1] = (long)k * plane + (long)wrap_up(j + n, ny) * nx;           \
            zm[n - 1] = (long)wrap_down(k - n, nz) * plane + (long)j * nx;         \
            zp[n - 1] = (long)wrap_up(k + n, nz) * plane + (long)j * nx;           \
        }                                                                          \
        for (int i = threadIdx.x; i < nx; i += blockDim.x) {                       \
            const long c = base + i;                                               \
            long mx[3], px[3], my[3], py[3], mz[3], pz[3];                         \
            for (int n = 0; n < 3; ++n) {                                          \
                mx[n] = base + wrap_down(i - n - 1, nx);                           \
                px[n] = base + wrap_up(i + n + 1, nx);                             \
                my[n] = ym[n] + i; py[n] = yp[n] + i;                              \
                mz[n] = zm[n] + i; pz[n] = zp[n] + i;                              \
            }
#define FD6_ROWS_END \
        }            \
    }

// S1 and S2 of one field along one axis (no 1/h factors)
__device__ __forceinline__ double s1_of(const double* __restrict__ u, const long* m, const long* p) {
    return kA1 * (__ldg(u + p[0]) - __ldg(u + m[0])) + kA2 * (__ldg(u + p[1]) - __ldg(u + m[1])) +
           kA3 * (__ldg(u + p[2]) - __ldg(u + m[2]));
}
__device__ __forceinline__ double s2_of(const double* __restrict__ u, double u0, const long* m, const long* p) {
    return kB0 * u0 + kB1 * (__ldg(u + p[0]) + __ldg(u + m[0])) + kB2 * (__ldg(u + p[1]) + __ldg(u + m[1])) +
           kB3 * (__ldg(u + p[2]) + __ldg(u + m[2]));
}
// S1 and S2 of the product a*b (pointwise), for the transposed operator
__device__ __forceinline__ double s1_prod(const double* __restrict__ a, const double* __restrict__ b, const long* m,
                                          const long* p) {
    double s = 0.0;
    const double w[3] = {kA1, kA2, kA3};
#pragma unroll
    for (int n = 0; n < 3; ++n) s += w[n] * (__ldg(a + p[n]) * __ldg(b + p[n]) - __ldg(a + m[n]) * __ldg(b + m[n]));
    return s;
}
__device__ __forceinline__ double s2_prod(const double* __restrict__ a, const double* __restrict__ b, double ab0,
                                          const long* m, const long* p) {
    double s = kB0 * ab0;
    const double w[3] = {kB1, kB2, kB3};
#pragma unroll
    for (int n = 0; n < 3; ++n) s += w[n] * (__ldg(a + p[n]) * __ldg(b + p[n]) + __ldg(a + m[n]) * __ldg(b + m[n]));
    return s;
}

// y = crho (rho - rsum/n) + sa A6 x   (rho may be null); partial[b] = block sum of y
__global__ void __launch_bounds__(kReduceThreads) k_fd6_apply(Geo g, const double* __restrict__ x,
                                                              const double* __restrict__ eps,
                                                              const double* __restrict__ rho, double crho,
                                                              const double* rsum, double sa,
                                                              double* __restrict__ y, double* __restrict__ partial) {
    __shared__ double red[32];
    const double ihx2 = g.ihx * g.ihx, ihy2 = g.ihy * g.ihy, ihz2 = g.ihz * g.ihz;
    const double rmean = rho ? rsum[0] / ((double)g.nx * g.ny * g.nz) : 0.0;
    double acc = 0.0;
    FD6_ROWS_BEGIN
        const double x0 = __ldg(x + c), e0 = __ldg(eps + c);
        const double a = ihx2 * axis_term(x, eps, x0, e0, mx, px) + ihy2 * axis_term(x, eps, x0, e0, my, py) +
                         ihz2 * axis_term(x, eps, x0, e0, mz, pz);
        const double v = (rho ? crho * (__ldg(rho + c) - rmean) : 0.0) + sa * a;
        y[c] = v;
        acc += v;
    FD6_ROWS_END
    const double s = fd6_block_sum(acc, red);
    if (threadIdx.x == 0) partial[blockIdx.x] = s;
}

// y = crho (rho - rsum/n) + sa A6^T x with
//   A6^T x = sum_axes [ -D1((D1 eps) x) + D2(eps x) ],
// d1e holding D1 eps per axis (1/h included, three fields of n values);
// partial[b] = block sum of y
__global__ void __launch_bounds__(kReduceThreads) k_fd6_apply_t(Geo g, const double* __restrict__ x,
                                                                const double* __restrict__ eps,
                                                                const double* __restrict__ d1e,
                                                                const double* __restrict__ rho, double crho,
                                                                const double* rsum, double sa,
                                                                double* __restrict__ y, double* __restrict__ partial) {
    __shared__ double red[32];
    const long npts = (long)g.nx * g.ny * g.nz;
    const double ihx2 = g.ihx * g.ihx, ihy2 = g.ihy * g.ihy, ihz2 = g.ihz * g.ihz;
    const double rmean = rho ? rsum[0] / (double)npts : 0.0;
    double acc = 0.0;
    FD6_ROWS_BEGIN
        const double ex0 = __ldg(eps + c) * __ldg(x + c);
        const double a = -g.ihx * s1_prod(d1e, x, mx, px) + ihx2 * s2_prod(eps, x, ex0, mx, px) -
                         g.ihy * s1_prod(d1e + npts, x, my, py) + ihy2 * s2_prod(eps, x, ex0, my, py) -
                         g.ihz * s1_prod(d1e + 2 * npts, x, mz, pz) + ihz2 * s2_prod(eps, x, ex0, mz, pz);
        const double v = (rho ? crho * (__ldg(rho + c) - rmean) : 0.0) + sa * a;
        y[c] = v;
        acc += v;
    FD6_ROWS_END
    const double s = fd6_block_sum(acc, red);
    if (threadIdx.x == 0) partial[blockIdx.x] = s;
}

// out + a n = D1_a u, a = 0, 1, 2 (1/h included); when w is given, w D1_a u instead
__global__ void __launch_bounds__(kReduceThreads) k_fd6_d1(Geo g, const double* __restrict__ u,
                                                           const double* __restrict__ w, double* __restrict__ out) {
    const long npts = (long)g.nx * g.ny * g.nz;
    FD6_ROWS_BEGIN
        const double f = w ? __ldg(w + c) : 1.0;
        out[c] = f * g.ihx * s1_of(u, mx, px);
        out[npts + c] = f * g.ihy * s1_of(u, my, py);
        out[2 * npts + c] = f * g.ihz * s1_of(u, mz, pz);
    FD6_ROWS_END
}

// weps = sum_axes [ -D1_a(t_a) + lam D2_a phi ] + mu lam, with t_a = lam D1_a phi
// (k_fd6_d1 with w = lam): the per-point weight of d eps in the forces
__global__ void __launch_bounds__(kReduceThreads) k_fd6_weps(Geo g, const double* __restrict__ phi,
                                                             const double* __restrict__ lam,
                                                             const double* __restrict__ t3, double mu,
                                                             double* __restrict__ weps) {
    const long npts = (long)g.nx * g.ny * g.nz;
    const double ihx2 = g.ihx * g.ihx, ihy2 = g.ihy * g.ihy, ihz2 = g.ihz * g.ihz;
    FD6_ROWS_BEGIN
        const double p0 = __ldg(phi + c), l0 = __ldg(lam + c);
        const double d2 = ihx2 * s2_of(phi, p0, mx, px) + ihy2 * s2_of(phi, p0, my, py) + ihz2 * s2_of(phi, p0, mz, pz);
        const double d1 = g.ihx * s1_of(t3, mx, px) + g.ihy * s1_of(t3 + npts, my, py) + g.ihz * s1_of(t3 + 2 * npts, mz, pz);
        weps[c] = -d1 + l0 * d2 + mu * l0;
    FD6_ROWS_END
}

#undef FD6_ROWS_BEGIN
#undef FD6_ROWS_END

// y -= (num[0] / den[0]) * (w ? w : 1)
__global__ void k_fd6_sub_ratio(long n, double* y, const double* w, const double* num, const double* den) {
    const double r = num[0] / den[0];
    for (long t = blockIdx.x * (long)blockDim.x + threadIdx.x; t < n; t += (long)gridDim.x * blockDim.x)
        y[t] -= r * (w ? w[t] : 1.0);
}

// dst = (double) src; partial[2b] = sum dst, partial[2b+1] = sum eps dst
template <typename T>
__global__ void __launch_bounds__(kReduceThreads) k_fd6_to64(long n, const T* src, const double* eps, double* dst,
                                                             double* partial) {
    __shared__ double red[32];
    double a = 0.0, b = 0.0;
    for (long t = blockIdx.x * (long)blockDim.x + threadIdx.x; t < n; t += (long)gridDim.x * blockDim.x) {
        const double v = (double)src[t];
        dst[t] = v;
        a += v;
        b += eps[t] * v;
    }
    double s = fd6_block_sum(a, red);
    __syncthreads();
    if (threadIdx.x == 0) partial[2 * blockIdx.x] = s;
    s = fd6_block_sum(b, red);
    if (threadIdx.x == 0) partial[2 * blockIdx.x + 1] = s;
}

// out = (phi - 4 pi lam) / 2; partial[b] = block sum of out
__global__ void __launch_bounds__(kReduceThreads) k_fd6_wrho(long n, const double* phi, const double* lam,
                                                             double* out, double* partial) {
    __shared__ double red[32];
    double a = 0.0;
    for (long t = blockIdx.x * (long)blockDim.x + threadIdx.x; t < n; t += (long)gridDim.x * blockDim.x) {
        const double v = 0.5 * (phi[t] - 4.0 * kPi * lam[t]);
        out[t] = v;
        a += v;
    }
    const double s = fd6_block_sum(a, red);
    if (threadIdx.x == 0) partial[blockIdx.x] = s;
}

// a single device scalar
__global__ void k_fd6_set(double* slot, double v) { slot[0] = v; }

// blocks for an element-wise pass: enough to cover n, at most 16 per SM
int fd6_grid(long n) {
    const long b = (n + 255) / 256;
    return (int)(b < 152L * 16 ? (b < 1 ? 1 : b) : 152L * 16);
}

}  // namespace

void launch_fd6_apply(const Geo& g, const double* x, const double* eps, const double* rho, double crho,
                      const double* rsum, double sa, double* y, double* partial, cudaStream_t s) {
    k_fd6_apply<<<kReduceBlocks, kReduceThreads, 0, s>>>(g, x, eps, rho, crho, rsum, sa, y, partial);
}
void launch_fd6_apply_t(const Geo& g, const double* x, const double* eps, const double* d1e, const double* rho,
                        double crho, const double* rsum, double sa, double* y, double* partial, cudaStream_t s) {
    k_fd6_apply_t<<<kReduceBlocks, kReduceThreads, 0, s>>>(g, x, eps, d1e, rho, crho, rsum, sa, y, partial);
}
void launch_fd6_d1(const Geo& g, const double* u, const double* w, double* out3, cudaStream_t s) {
    k_fd6_d1<<<kReduceBlocks, kReduceThreads, 0, s>>>(g, u, w, out3);
}
void launch_fd6_weps(const Geo& g, const double* phi, const double* lam, const double* t3, double mu, double* weps,
                     cudaStream_t s) {
    k_fd6_weps<<<kReduceBlocks, kReduceThreads, 0, s>>>(g, phi, lam, t3, mu, weps);
}
void launch_fd6_sub_ratio(long n, double* y, const double* w, const double* num, const double* den,
                          cudaStream_t s) {
    k_fd6_sub_ratio<<<fd6_grid(n), 256, 0, s>>>(n, y, w, num, den);
}
template <typename T>
void launch_fd6_to64(long n, const T* src, const double* eps, double* dst, double* partial, cudaStream_t s) {
    k_fd6_to64<T><<<kReduceBlocks, kReduceThreads, 0, s>>>(n, src, eps, dst, partial);
}
template void launch_fd6_to64<float>(long, const float*, const double*, double*, double*, cudaStream_t);
template void launch_fd6_to64<double>(long, const double*, const double*, double*, double*, cudaStream_t);
void launch_fd6_wrho(long n, const double* phi, const double* lam, double* out, double* partial, cudaStream_t s) {
    k_fd6_wrho<<<kReduceBlocks, kReduceThreads, 0, s>>>(n, phi, lam, out, partial);
}
void launch_fd6_set(double* slot, double v, cudaStream_t s) { k_fd6_set<<<1, 1, 0, s>>>(slot, v); }

void launch_residual6(const Geo& g, const double* phi, const double* rho, const double* eps64, double mu,
                      double* r_out, double* partial, cudaStream_t s) {
    k_residual6<<<kReduceBlocks, kReduceThreads, 0, s>>>(g, phi, rho, eps64, mu, r_out, partial);
}

}  // namespace gp
