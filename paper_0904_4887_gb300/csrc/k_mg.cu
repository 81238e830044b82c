// Multigrid and Krylov kernels for the 7-point conservative operator
//   (A u)_i = sum_axes [c_{i+1/2}(u_{i+1} - u_i) - c_{i-1/2}(u_i - u_{i-1})],
// the discretisation of div(eps grad u) of Eq. 3 (c = eps_face / h^2), plus
// the FP64 full-box passes of the outer defect correction and the kernels
// that couple the dry FFT solution to the wet multigrid band (Sec. II.C).
//
// Levels are vertex-centred: coarse point I sits on fine point 2I (periodic
// axes) or 2I+1 (Dirichlet z, counting interior planes). Level 0 reads the
// cell dielectric and forms face means on the fly; coarse levels store face
// coefficients, obtained from the fine faces by a harmonic mean along the
// face normal (two faces in series) and full weighting across it.
#include "gp_common.cuh"

#include <cstdint>
#include <initializer_list>

namespace gp {
namespace {

template <typename T> struct Co { T xm, xp, ym, yp, zm, zp; };

struct Nb { long c, xm, xp, ym, yp, zm, zp; };

__device__ __forceinline__ Nb neighbours(int nx, int ny, int nz, int zper, int i, int j, int k) {
    Nb n;
    const long pl = (long)nx * ny;
    n.c = i + (long)nx * (j + (long)ny * k);
    n.xm = n.c + (i == 0 ? nx - 1 : -1);
    n.xp = n.c + (i == nx - 1 ? 1 - nx : 1);
    n.ym = n.c + (j == 0 ? (long)(ny - 1) * nx : -(long)nx);
    n.yp = n.c + (j == ny - 1 ? -(long)(ny - 1) * nx : (long)nx);
    n.zm = n.c + ((k == 0 && zper) ? (long)(nz - 1) * pl : -pl);
    n.zp = n.c + ((k == nz - 1 && zper) ? -(long)(nz - 1) * pl : pl);
    return n;
}

template <typename T>
__device__ __forceinline__ Co<T> coefs(const LV<T>& L, const Nb& n) {
    Co<T> o;
    if (L.cell) {
        const T e = L.eps[n.c];
        const T hx = (T)0.5 * L.ihx2, hy = (T)0.5 * L.ihy2, hz = (T)0.5 * L.ihz2;
        o.xm = (e + L.eps[n.xm]) * hx; o.xp = (e + L.eps[n.xp]) * hx;
        o.ym = (e + L.eps[n.ym]) * hy; o.yp = (e + L.eps[n.yp]) * hy;
        o.zm = (e + L.eps[n.zm]) * hz; o.zp = (e + L.eps[n.zp]) * hz;
    } else {
        o.xm = L.cx[n.xm]; o.xp = L.cx[n.c];
        o.ym = L.cy[n.ym]; o.yp = L.cy[n.c];
        o.zm = L.cz[n.zm]; o.zp = L.cz[n.c];
    }
    return o;
}

// A u at one point
template <typename T>
__device__ __forceinline__ T apply_at(const Co<T>& o, const Nb& n, const T* u) {
    const T u0 = u[n.c];
    return o.xp * (u[n.xp] - u0) - o.xm * (u0 - u[n.xm]) + o.yp * (u[n.yp] - u0) - o.ym * (u0 - u[n.ym]) +
           o.zp * (u[n.zp] - u0) - o.zm * (u0 - u[n.zm]);
}

__device__ __forceinline__ void split3(long t, int nx, int ny, int& i, int& j, int& k) {
    i = (int)(t % nx);
    const long r = t / nx;
    j = (int)(r % ny);
    k = (int)(r / ny);
}

__device__ __forceinline__ double block_sum(double v, double* red) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    __syncthreads();
    if (l == 0) red[w] = v;
    __syncthreads();
    double s = 0.0;
    if (threadIdx.x < 32) {
        s = (threadIdx.x < (blockDim.x >> 5)) ? red[threadIdx.x] : 0.0;
        for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    }
    return s;   // valid in thread 0
}

// per-thread accumulator of the working precision: FP32 data is summed in
// FP32 within a thread (a few hundred terms) and in FP64 across threads, so
// no FP64 instruction runs per element (GB300's FP64 rate is 1/64 of FP32)
template <typename T> struct AccT { using type = double; };
template <> struct AccT<float> { using type = float; };

// compensated running sum (Kahan): the FP32 per-thread partial sums keep
// about FP64 accuracy at four FP32 instructions per term
template <typename A>
struct KSum {
    A s = 0, c = 0;
    __device__ __forceinline__ void add(A v) {
        const A y = v - c;
        const A t = s + y;
        c = (t - s) - y;
        s = t;
    }
    __device__ __forceinline__ double value() const { return (double)s - (double)c; }
};

// row kernels: one block per (j, k) row at a time, threads along x
int row_threads(int nx) {
    const int t = (nx + 31) / 32 * 32;
    return t > 256 ? 256 : (t < 32 ? 32 : t);
}
int row_blocks(long rows) { return (int)(rows < 152L * 32 ? rows : 152L * 32); }

int grid_for(long n, int threads) {
    long b = (n + threads - 1) / threads;
    return (int)(b < 152L * 16 ? (b < 1 ? 1 : b) : 152L * 16);
}

// ------------------------------------------------------------ smoothing
// Red-black Gauss-Seidel half sweep for A u = f: u_i = (sum c u_nb - f_i) / sum c.
// One thread per x-pair; it updates the member of the pair with the colour.
template <typename T>
__global__ void k_rbgs(LV<T> L, T* u, const T* f, int color, int init) {
    griddep_wait();
    const int hx = L.nx >> 1;
    const long rows = (long)L.ny * L.nz;
    for (long row = blockIdx.x; row < rows; row += gridDim.x)
    for (int i2 = threadIdx.x; i2 < hx; i2 += blockDim.x) {
        const int j = (int)(row % L.ny), k = (int)(row / L.ny);
        const int i = 2 * i2 + ((j + k + color) & 1);
        const Nb n = neighbours(L.nx, L.ny, L.nz, L.zper, i, j, k);
        const Co<T> o = coefs(L, n);
        const T s = init ? (T)0 : o.xp * u[n.xp] + o.xm * u[n.xm] + o.yp * u[n.yp] + o.ym * u[n.ym] +
                                     o.zp * u[n.zp] + o.zm * u[n.zm];
        const T d = o.xp + o.xm + o.yp + o.ym + o.zp + o.zm;
        u[n.c] = (s - f[n.c]) / d;
    }
}

// The same half sweep on a face-coefficient level in FP32, one thread per x-pair
// with 8-byte loads of the pair and of its y and z neighbour pairs (32-bit
// index arithmetic).
__device__ __forceinline__ float2 ld_f2(const float* p, long i) { return *reinterpret_cast<const float2*>(p + i); }

__global__ void __launch_bounds__(256) k_rbgs_pairs(LV<float> L, float* __restrict__ u, const float* __restrict__ f,
                                                    int color, int init) {
    griddep_wait();
    const int nx = L.nx, ny = L.ny, nz = L.nz, np = nx >> 1;
    const long pl = (long)nx * ny;
    const int total = np * ny * nz;
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < total; t += gridDim.x * blockDim.x) {
        const int p = t % np;
        const int row = t / np;
        const int j = row % ny, k = row / ny;
        const int m = (j + k + color) & 1;                 // the member (x = 2p + m) of this colour
        const long rb = (long)k * pl + (long)j * nx;
        const long c2 = rb + 2 * p;
        const long dym = j == 0 ? (long)(ny - 1) * nx : -(long)nx;
        const long dyp = j == ny - 1 ? -(long)(ny - 1) * nx : (long)nx;
        const long dzm = (k == 0 && L.zper) ? (long)(nz - 1) * pl : -pl;
        const long dzp = (k == nz - 1 && L.zper) ? -(long)(nz - 1) * pl : pl;
        const long cl = p == 0 ? rb + nx - 1 : c2 - 1;     // x - 1 of the even member
        const long cr = p == np - 1 ? rb : c2 + 2;         // x + 1 of the odd member
        const float2 uo = ld_f2(u, c2);
        auto pick = [m](float2 v) { return m ? v.y : v.x; };
        const float uxm = m ? uo.x : u[cl], uxp = m ? u[cr] : uo.y;
        const float2 cxo = ld_f2(L.cx, c2);
        const float cxm = m ? cxo.x : L.cx[cl], cxp = m ? cxo.y : cxo.x;
        const float cym = pick(ld_f2(L.cy, c2 + dym)), cyp = pick(ld_f2(L.cy, c2));
        const float czm = pick(ld_f2(L.cz, c2 + dzm)), czp = pick(ld_f2(L.cz, c2));
        const float sum = init ? 0.f
                               : cxp * uxp + cxm * uxm + cyp * pick(ld_f2(u, c2 + dyp)) +
                                     cym * pick(ld_f2(u, c2 + dym)) + czp * pick(ld_f2(u, c2 + dzp)) +
                                     czm * pick(ld_f2(u, c2 + dzm));
        const float d = cxp + cxm + cyp + cym + czp + czm;
        u[c2 + m] = __fdividef(sum - pick(ld_f2(f, c2)), d);
    }
}

template <typename T>
__global__ void k_residual(LV<T> L, const T* u, const T* f, T* r) {
    griddep_wait();
    const long rows = (long)L.ny * L.nz;
    for (long row = blockIdx.x; row < rows; row += gridDim.x)
    for (int i = threadIdx.x; i < L.nx; i += blockDim.x) {
        const int j = (int)(row % L.ny), k = (int)(row / L.ny);
        const Nb nb = neighbours(L.nx, L.ny, L.nz, L.zper, i, j, k);
        r[nb.c] = f[nb.c] - apply_at(coefs(L, nb), nb, u);
    }
}

// full weighting (1/4, 1/2, 1/4) per axis
template <typename T>
__global__ void k_restrict(LV<T> F, const T* r, LV<T> C, T* fc) {
    griddep_wait();
    const long rows = (long)C.ny * C.nz;
    const int zoff = F.zper ? 0 : 1;
    const long pl = (long)F.nx * F.ny;
    for (long row = blockIdx.x; row < rows; row += gridDim.x)
    for (int I = threadIdx.x; I < C.nx; I += blockDim.x) {
        const int J = (int)(row % C.ny), K = (int)(row / C.ny);
        const int kf = 2 * K + zoff;
        T acc = 0;
        for (int dz = -1; dz <= 1; ++dz) {
            int kk = kf + dz;
            if (F.zper) kk = (kk + F.nz) % F.nz;
            const T wz = dz == 0 ? (T)0.5 : (T)0.25;
            for (int dy = -1; dy <= 1; ++dy) {
                const int jj = (2 * J + dy + F.ny) % F.ny;
                const T wy = dy == 0 ? (T)0.5 : (T)0.25;
                const long base = kk * pl + (long)jj * F.nx;
                const int ic = 2 * I;
                const int im = ic == 0 ? F.nx - 1 : ic - 1;
                const int ip = ic == F.nx - 1 ? 0 : ic + 1;
                acc += wz * wy * ((T)0.25 * r[base + im] + (T)0.5 * r[base + ic] + (T)0.25 * r[base + ip]);
            }
        }
        fc[I + (long)C.nx * (J + (long)C.ny * K)] = acc;
    }
}

// The same full weighting in FP32, two coarse x points per thread: per fine
// row one 16-byte load (fine x 4h .. 4h+3) and the point before it serve
// both (fine nx % 4 == 0, coarse nx even, fine nx = 2 coarse nx).
__global__ void __launch_bounds__(256) k_restrict4(LV<float> F, const float* __restrict__ r, LV<float> C,
                                                   float* __restrict__ fc) {
    griddep_wait();
    const int nh = C.nx >> 1;
    const int total = nh * C.ny * C.nz;
    const int zoff = F.zper ? 0 : 1;
    const long pl = (long)F.nx * F.ny;
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < total; t += gridDim.x * blockDim.x) {
        const int h = t % nh;
        const int row = t / nh;
        const int J = row % C.ny, K = row / C.ny;
        const int x0 = 4 * h, xm = x0 == 0 ? F.nx - 1 : x0 - 1;
        float a0 = 0.f, a1 = 0.f;
#pragma unroll
        for (int dz = -1; dz <= 1; ++dz) {
            int kk = 2 * K + zoff + dz;
            if (F.zper) kk = kk < 0 ? kk + F.nz : (kk >= F.nz ? kk - F.nz : kk);
            const float wz = dz == 0 ? 0.5f : 0.25f;
#pragma unroll
            for (int dy = -1; dy <= 1; ++dy) {
                int jj = 2 * J + dy;
                jj = jj < 0 ? jj + F.ny : (jj >= F.ny ? jj - F.ny : jj);
                const float w = wz * (dy == 0 ? 0.5f : 0.25f);
                const float* rp = r + (long)kk * pl + (long)jj * F.nx;
                const float4 v = *reinterpret_cast<const float4*>(rp + x0);
                const float vm = rp[xm];
                a0 += w * (0.25f * vm + 0.5f * v.x + 0.25f * v.y);
                a1 += w * (0.25f * v.y + 0.5f * v.z + 0.25f * v.w);
            }
        }
        *reinterpret_cast<float2*>(fc + (long)C.nx * (J + (long)C.ny * K) + 2 * h) = make_float2(a0, a1);
    }
}

// trilinear interpolation of the coarse correction, added to u
template <typename T>
__global__ void k_prolong_add(LV<T> F, T* u, LV<T> C, const T* uc) {
    griddep_wait();
    const long rows = (long)F.ny * F.nz;
    const int zoff = F.zper ? 0 : 1;
    const long cpl = (long)C.nx * C.ny;
    for (long row = blockIdx.x; row < rows; row += gridDim.x)
    for (int i = threadIdx.x; i < F.nx; i += blockDim.x) {
        const int j = (int)(row % F.ny), k = (int)(row / F.ny);
        int xi[2], yi[2], zi[2];
        T xw[2], yw[2], zw[2];
        int nxp, nyp, nzp;
        if (i & 1) { xi[0] = i >> 1; xi[1] = (xi[0] + 1) % C.nx; xw[0] = xw[1] = (T)0.5; nxp = 2; }
        else { xi[0] = i >> 1; xw[0] = 1; nxp = 1; }
        if (j & 1) { yi[0] = j >> 1; yi[1] = (yi[0] + 1) % C.ny; yw[0] = yw[1] = (T)0.5; nyp = 2; }
        else { yi[0] = j >> 1; yw[0] = 1; nyp = 1; }
        const int kk = k - zoff;                 // -1 .. for Dirichlet
        if (kk & 1) {
            zi[0] = (kk - 1) >> 1;               // floor division: -1 -> -1 (the lower wall)
            zi[1] = zi[0] + 1;
            if (C.zper && zi[1] == C.nz) zi[1] = 0;
            zw[0] = zw[1] = (T)0.5;
            nzp = 2;
        } else { zi[0] = kk >> 1; zw[0] = 1; nzp = 1; }
        T acc = 0;
        for (int c = 0; c < nzp; ++c)
            for (int b = 0; b < nyp; ++b)
                for (int a = 0; a < nxp; ++a)
                    acc += zw[c] * yw[b] * xw[a] * uc[xi[a] + (long)C.nx * yi[b] + cpl * zi[c]];
        u[i + (long)F.nx * (j + (long)F.ny * k)] += acc;
    }
}

// The same trilinear prolongation, four consecutive fine x points per thread
// (fine nx % 4 == 0, FP32): coarse x indices 2q, 2q+1, 2q+2 (wrapped) serve
// the quad, with the one or two coarse rows and planes of its (j, k).
__global__ void __launch_bounds__(256) k_prolong_add4(LV<float> F, float* __restrict__ u, LV<float> C,
                                                      const float* __restrict__ uc) {
    griddep_wait();
    const int nx4 = F.nx >> 2;
    const int total = nx4 * F.ny * F.nz;
    const int zoff = F.zper ? 0 : 1;
    const long cpl = (long)C.nx * C.ny;
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < total; t += gridDim.x * blockDim.x) {
        const int q = t % nx4;
        const int row = t / nx4;
        const int j = row % F.ny, k = row / F.ny;
        const int I0 = 2 * q, I1 = I0 + 1, I2 = (I0 + 2 == C.nx) ? 0 : I0 + 2;
        int y0 = j >> 1, y1 = y0;
        float wy0 = 1.f, wy1 = 0.f;
        if (j & 1) { y1 = (y0 + 1 == C.ny) ? 0 : y0 + 1; wy0 = wy1 = 0.5f; }
        const int kk = k - zoff;
        int z0, z1;
        float wz0 = 1.f, wz1 = 0.f;
        if (kk & 1) {
            z0 = (kk - 1) >> 1;
            z1 = z0 + 1;
            if (C.zper && z1 == C.nz) z1 = 0;
            wz0 = wz1 = 0.5f;
        } else { z0 = kk >> 1; z1 = z0; }
        // coarse values along x at the (y, z) combinations, weighted
        float a0 = 0.f, a1 = 0.f, a2 = 0.f;
        {
            const float* r00 = uc + cpl * z0 + (long)C.nx * y0;
            const float* r01 = uc + cpl * z0 + (long)C.nx * y1;
            const float* r10 = uc + cpl * z1 + (long)C.nx * y0;
            const float* r11 = uc + cpl * z1 + (long)C.nx * y1;
            const float w00 = wz0 * wy0, w01 = wz0 * wy1, w10 = wz1 * wy0, w11 = wz1 * wy1;
            a0 = w00 * r00[I0] + w01 * r01[I0] + w10 * r10[I0] + w11 * r11[I0];
            a1 = w00 * r00[I1] + w01 * r01[I1] + w10 * r10[I1] + w11 * r11[I1];
            a2 = w00 * r00[I2] + w01 * r01[I2] + w10 * r10[I2] + w11 * r11[I2];
        }
        float4* up = reinterpret_cast<float4*>(u + (long)F.nx * (j + (long)F.ny * k)) + q;
        float4 v = *up;
        v.x += a0;
        v.y += 0.5f * (a0 + a1);
        v.z += a1;
        v.w += 0.5f * (a1 + a2);
        *up = v;
    }
}

// fine face coefficient along `axis` between (i,j,k) and its + neighbour; k may be -1 (wall face)
template <typename T>
__device__ __forceinline__ T fine_face(const LV<T>& F, int axis, int i, int j, int k) {
    const long pl = (long)F.nx * F.ny;
    i = (i % F.nx + F.nx) % F.nx;
    j = (j % F.ny + F.ny) % F.ny;
    if (F.zper) k = (k % F.nz + F.nz) % F.nz;
    const long c = i + (long)F.nx * j + pl * k;
    if (!F.cell) return axis == 0 ? F.cx[c] : (axis == 1 ? F.cy[c] : F.cz[c]);
    long o;
    T ih;
    if (axis == 0) { o = c + (i == F.nx - 1 ? 1 - F.nx : 1); ih = F.ihx2; }
    else if (axis == 1) { o = c + (j == F.ny - 1 ? -(long)(F.ny - 1) * F.nx : (long)F.nx); ih = F.ihy2; }
    else { o = c + ((k == F.nz - 1 && F.zper) ? -(long)(F.nz - 1) * pl : pl); ih = F.ihz2; }
    return (F.eps[c] + F.eps[o]) * (T)0.5 * ih;
}

template <typename T>
__device__ __forceinline__ T series_quarter(T a, T b) {
    // two faces of spacing h in series, re-expressed for spacing 2h: harmonic mean / 4
    return (a * b) / ((a + b) * (T)2);
}

template <typename T>
__global__ void k_coarsen_faces(LV<T> F, int nxc, int nyc, int nzc, T* cx, T* cy, T* cz) {
    const int zoff = F.zper ? 0 : 1;
    const int nk = F.zper ? nzc : nzc + 1;      // Dirichlet: also the lower wall face K = -1
    const long n = (long)nxc * nyc * nk;
    const long cpl = (long)nxc * nyc;
    for (long t = blockIdx.x * (long)blockDim.x + threadIdx.x; t < n; t += (long)gridDim.x * blockDim.x) {
        int I, J, kk;
        split3(t, nxc, nyc, I, J, kk);
        const int K = F.zper ? kk : kk - 1;
        const int kf = 2 * K + zoff;
        const long o = I + (long)nxc * J + cpl * K;
        if (K >= 0) {
            T ax = 0, ay = 0;
            for (int dz = -1; dz <= 1; ++dz) {
                const T wz = dz == 0 ? (T)0.5 : (T)0.25;
                for (int d = -1; d <= 1; ++d) {
                    const T wd = d == 0 ? (T)0.5 : (T)0.25;
                    ax += wz * wd * series_quarter(fine_face(F, 0, 2 * I, 2 * J + d, kf + dz),
                                                   fine_face(F, 0, 2 * I + 1, 2 * J + d, kf + dz));
                    ay += wz * wd * series_quarter(fine_face(F, 1, 2 * I + d, 2 * J, kf + dz),
                                                   fine_face(F, 1, 2 * I + d, 2 * J + 1, kf + dz));
                }
            }
            cx[o] = ax;
            cy[o] = ay;
        }
        T az = 0;
        for (int dy = -1; dy <= 1; ++dy) {
            const T wy = dy == 0 ? (T)0.5 : (T)0.25;
            for (int dx = -1; dx <= 1; ++dx) {
                const T wx = dx == 0 ? (T)0.5 : (T)0.25;
                az += wy * wx * series_quarter(fine_face(F, 2, 2 * I + dx, 2 * J + dy, kf),
                                               fine_face(F, 2, 2 * I + dx, 2 * J + dy, kf + 1));
            }
        }
        cz[o] = az;
    }
}

// The same coarsening from a periodic cell level (the finest level of the full
// box): one thread per coarse point loads once, into registers, the 4 x 4 x 4
// block of eps (fine x, y, z from 2I-1, 2J-1, 2K-1 on, wrapped) that the 27
// fine faces of its three coarse faces use, instead of evaluating each of the
// 54 fine faces from two loads and six wrapped-index divisions; the same weights
// and series rule, the 1/(2 h^2) factor taken out of the sums (the series rule
// is homogeneous of degree one).
template <typename T>
__global__ void __launch_bounds__(256) k_coarsen_faces_cell(LV<T> F, int nxc, int nyc, int nzc, T* cx, T* cy,
                                                            T* cz) {
    const int total = nxc * nyc * nzc;
    const long pl = (long)F.nx * F.ny;
    const T w[3] = {(T)0.25, (T)0.5, (T)0.25};
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < total; t += gridDim.x * blockDim.x) {
        const int I = t % nxc, r = t / nxc, J = r % nyc, K = r / nyc;
        int xs[4];
        long ys[4], zs[4];
#pragma unroll
        for (int a = 0; a < 4; ++a) {
            int x = 2 * I - 1 + a, y = 2 * J - 1 + a, z = 2 * K - 1 + a;
            x = x < 0 ? x + F.nx : (x >= F.nx ? x - F.nx : x);
            y = y < 0 ? y + F.ny : (y >= F.ny ? y - F.ny : y);
            z = z < 0 ? z + F.nz : (z >= F.nz ? z - F.nz : z);
            xs[a] = x;
            ys[a] = (long)y * F.nx;
            zs[a] = (long)z * pl;
        }
        T e[4][4][4];                                   // [z][y][x]
#pragma unroll
        for (int c = 0; c < 4; ++c)
#pragma unroll
            for (int b = 0; b < 4; ++b)
#pragma unroll
                for (int a = 0; a < 4; ++a) e[c][b][a] = __ldg(F.eps + zs[c] + ys[b] + xs[a]);
        T ax = 0, ay = 0, az = 0;
#pragma unroll
        for (int c = 0; c < 3; ++c)
#pragma unroll
            for (int b = 0; b < 3; ++b) {
                const T wt = w[c] * w[b];
                ax += wt * series_quarter(e[c][b][1] + e[c][b][2], e[c][b][2] + e[c][b][3]);
                ay += wt * series_quarter(e[c][1][b] + e[c][2][b], e[c][2][b] + e[c][3][b]);
                az += wt * series_quarter(e[1][c][b] + e[2][c][b], e[2][c][b] + e[3][c][b]);
            }
        const long o = I + (long)nxc * (J + (long)nyc * K);
        cx[o] = ax * (T)0.5 * F.ihx2;
        cy[o] = ay * (T)0.5 * F.ihy2;
        cz[o] = az * (T)0.5 * F.ihz2;
    }
}

// dense matrix of the coarsest operator (row p = point p), periodic levels
// regularised by -(max|diag|/n) 1 1^T so that mean-zero data give the
// mean-zero solution
template <typename T>
__global__ void k_coarse_matrix(LV<T> C, double* M) {
    const int n = C.nx * C.ny * C.nz;
    __shared__ double dmax;
    if (threadIdx.x == 0) dmax = 0.0;
    __syncthreads();
    for (int p = threadIdx.x; p < n; p += blockDim.x) {
        for (int q = 0; q < n; ++q) M[(long)p * n + q] = 0.0;
        int i, j, k;
        split3(p, C.nx, C.ny, i, j, k);
        const Nb nb = neighbours(C.nx, C.ny, C.nz, C.zper, i, j, k);
        const Co<T> o = coefs(C, nb);
        const long nbr[6] = {nb.xm, nb.xp, nb.ym, nb.yp, nb.zm, nb.zp};
        const double cf[6] = {(double)o.xm, (double)o.xp, (double)o.ym, (double)o.yp, (double)o.zm,
                              (double)o.zp};
        double d = 0.0;
        for (int s = 0; s < 6; ++s) {
            d += cf[s];
            const long q = nbr[s];
            if (q >= 0 && q < n) M[(long)p * n + q] += cf[s];   // outside: Dirichlet wall (zero)
        }
        M[(long)p * n + p] -= d;
        atomicMax((unsigned long long*)&dmax, __double_as_longlong(d));   // d > 0
    }
    __syncthreads();
    if (C.zper) {
        const double s = dmax / n;
        for (long e = threadIdx.x; e < (long)n * n; e += blockDim.x) M[e] -= s;
    }
}

// Inverse by Gauss-Jordan elimination without pivoting. The coarse operator
// is negative definite (Dirichlet walls, or the periodic operator shifted by
// -s 1 1^T, whose null space it removes), so every pivot is nonzero and no row
// exchange is needed. Step `col` subtracts multiples of row col from every
// other row of [M | W], one CTA per row; row col itself is only read during
// the step. After the last step M is diagonal and the inverse is W / diag(M).
__global__ void k_gj_init(double* M, int n, int* status) {
    double* W = M + (long)n * n;
    const int r = blockIdx.x;
    for (int q = threadIdx.x; q < n; q += blockDim.x) W[(long)r * n + q] = (q == r) ? 1.0 : 0.0;
    if (r == 0 && threadIdx.x == 0) *status = 0;
}

__global__ void k_gj_step(double* M, int n, int col, int* status) {
    const int r = blockIdx.x;
    if (r == col) return;
    double* W = M + (long)n * n;
    __shared__ double f;
    if (threadIdx.x == 0) {
        const double piv = M[(long)col * n + col];
        if (!(fabs(piv) > 1e-300)) {
            f = 0.0;
            *status = 1;
        } else {
            f = M[(long)r * n + col] / piv;
        }
    }
    __syncthreads();
    const double fr = f;
    if (fr == 0.0) return;
    const double* mc = M + (long)col * n;
    const double* wc = W + (long)col * n;
    double* mr = M + (long)r * n;
    double* wr = W + (long)r * n;
    for (int q = threadIdx.x; q < n; q += blockDim.x) {
        mr[q] -= fr * mc[q];
        wr[q] -= fr * wc[q];
    }
}

__global__ void k_gj_finish(double* M, int n) {
    double* W = M + (long)n * n;
    const int r = blockIdx.x;
    __shared__ double inv_d;
    if (threadIdx.x == 0) inv_d = 1.0 / M[(long)r * n + r];
    __syncthreads();
    for (int q = threadIdx.x; q < n; q += blockDim.x) W[(long)r * n + q] *= inv_d;
}

// The same elimination for a small coarsest grid in ONE CTA: [M | I] lives in
// shared memory (n rows of 2n doubles), each column takes two phases (the
// row factors, then the row updates) separated by the CTA barrier, and the
// inverse goes to the second half of M's buffer as in the multi-CTA version.
constexpr int kGjSmemMax = 110;          // 2 n^2 + n doubles within 200 KB of shared memory

__global__ void __launch_bounds__(1024) k_gj_smem(double* M, int n, int* status) {
    extern __shared__ double gja[];
    double* A = gja;                      // [n][2n]
    double* fac = gja + 2 * n * n;        // [n]
    const int w = 2 * n, tid = threadIdx.x;
    for (int e = tid; e < n * w; e += blockDim.x) {
        const int r = e / w, q = e - r * w;
        A[e] = q < n ? M[(long)r * n + q] : (q - n == r ? 1.0 : 0.0);
    }
    if (tid == 0) *status = 0;
    __syncthreads();
    for (int col = 0; col < n; ++col) {
        const double piv = A[col * w + col];
        const bool ok = fabs(piv) > 1e-300;
        if (!ok && tid == 0) *status = 1;
        for (int r = tid; r < n; r += blockDim.x) fac[r] = (ok && r != col) ? A[r * w + col] / piv : 0.0;
        __syncthreads();
        for (int e = tid; e < n * w; e += blockDim.x) {
            const int r = e / w, q = e - r * w;
            const double f = fac[r];
            if (f != 0.0) A[e] -= f * A[col * w + q];
        }
        __syncthreads();
    }
    double* W = M + (long)n * n;
    for (int e = tid; e < n * n; e += blockDim.x) {
        const int r = e / n, q = e - r * n;
        W[e] = A[r * w + n + q] / A[r * w + r];
    }
}

// The same one-CTA elimination with [M | I] held as float pairs (hi, lo) and
// every step in pair arithmetic on the FP32 pipe (Dekker's products by FMA,
// Knuth's two-sum, a pair quotient from the float quotient and one correction):
// about 2^-46 relative per operation. It serves the FP32 multigrid, which stores
// the inverse in FP32; on one SM the FP64 version is bound by the FP64 pipe
// (1/64 of the FP32 rate). Rows go to warps and columns to lanes, so no index
// division; step `col` updates only columns col.. of each row (those before it
// are already eliminated and stay as they are).
struct gjp { float hi, lo; };
__device__ __forceinline__ gjp gjp_quick(float s, float e) {   // |s| >= |e|
    const float t = s + e;
    return {t, e - (t - s)};
}
__device__ __forceinline__ gjp gjp_mul(gjp a, gjp b) {
    const float p = a.hi * b.hi;
    float e = fmaf(a.hi, b.hi, -p);
    e = fmaf(a.hi, b.lo, e);
    e = fmaf(a.lo, b.hi, e);
    return gjp_quick(p, e);
}
__device__ __forceinline__ gjp gjp_sub(gjp a, gjp b) {
    const float s = a.hi - b.hi;
    const float v = s - a.hi;
    float e = (a.hi - (s - v)) - (b.hi + v);
    e += a.lo - b.lo;
    return gjp_quick(s, e);
}
__device__ __forceinline__ gjp gjp_div(gjp a, gjp b) {
    const float q1 = a.hi / b.hi;
    const gjp r = gjp_sub(a, gjp_mul({q1, 0.f}, b));
    return gjp_quick(q1, r.hi / b.hi);
}

__global__ void __launch_bounds__(1024) k_gj_smem_pairs(double* M, int n, int* status) {
    extern __shared__ float2 gjq[];
    float2* A = gjq;                      // [n][2n]
    float2* fac = gjq + 2 * n * n;        // [n]
    const int w = 2 * n, tid = threadIdx.x, warp = tid >> 5, lane = tid & 31, nw = blockDim.x >> 5;
    for (int r = warp; r < n; r += nw)
        for (int q = lane; q < w; q += 32)
            A[r * w + q] = q < n ? split_to_float2(M[(long)r * n + q]) : make_float2(q - n == r ? 1.f : 0.f, 0.f);
    if (tid == 0) *status = 0;
    __syncthreads();
    for (int col = 0; col < n; ++col) {
        const float2 pv = A[col * w + col];
        const gjp piv{pv.x, pv.y};
        const bool ok = fabsf(piv.hi) > 1e-30f;
        if (!ok && tid == 0) *status = 1;
        for (int r = tid; r < n; r += blockDim.x) {
            const float2 a = A[r * w + col];
            const gjp f = (ok && r != col) ? gjp_div({a.x, a.y}, piv) : gjp{0.f, 0.f};
            fac[r] = make_float2(f.hi, f.lo);
        }
        __syncthreads();
        for (int r = warp; r < n; r += nw) {
            const float2 fr = fac[r];
            if (fr.x == 0.f) continue;
            const gjp f{fr.x, fr.y};
            for (int q = col + lane; q < w; q += 32) {
                const float2 a = A[r * w + q], m = A[col * w + q];
                const gjp v = gjp_sub({a.x, a.y}, gjp_mul(f, {m.x, m.y}));
                A[r * w + q] = make_float2(v.hi, v.lo);
            }
        }
        __syncthreads();
    }
    double* W = M + (long)n * n;
    for (int r = warp; r < n; r += nw) {
        const float2 d = A[r * w + r];
        for (int q = lane; q < n; q += 32) {
            const float2 a = A[r * w + n + q];
            const gjp v = gjp_div({a.x, a.y}, {d.x, d.y});
            W[(long)r * n + q] = (double)v.hi + (double)v.lo;
        }
    }
}

template <typename T>
__global__ void k_store_inverse(const double* W, long nn, T* inv) {
    for (long e = blockIdx.x * (long)blockDim.x + threadIdx.x; e < nn; e += (long)gridDim.x * blockDim.x)
        inv[e] = (T)W[e];
}

// u = inv * f on the coarsest level (periodic: f projected to mean zero first)
template <typename T>
__global__ void k_coarse_solve(LV<T> C, const T* inv, int n, const T* f, T* u) {
    __shared__ T fs[kMaxCoarse];
    __shared__ double red[32];
    double loc = 0.0;
    for (int p = threadIdx.x; p < n; p += blockDim.x) {
        fs[p] = f[p];
        loc += (double)f[p];
    }
    const double tot = block_sum(loc, red);
    __shared__ double mean;
    if (threadIdx.x == 0) mean = C.zper ? tot / n : 0.0;
    __syncthreads();
    for (int p = threadIdx.x; p < n; p += blockDim.x) fs[p] -= (T)mean;
    __syncthreads();
    // one warp per row of the inverse: coalesced loads, a warp reduction
    const int lane = threadIdx.x & 31, nw = blockDim.x >> 5;
    for (int p = threadIdx.x >> 5; p < n; p += nw) {
        const T* row = inv + (long)p * n;
        T acc = 0;
        for (int q = lane; q < n; q += 32) acc += row[q] * fs[q];
        for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
        if (lane == 0) u[p] = acc;
    }
}

// ------------------------------------------------------------ Krylov helpers
template <typename T>
__global__ void k_applyA_dot(LV<T> L, const T* p, T* q, double* partial) {
    __shared__ double red[32];
    const long rows = (long)L.ny * L.nz;
    KSum<typename AccT<T>::type> loc;
    for (long row = blockIdx.x; row < rows; row += gridDim.x)
    for (int i = threadIdx.x; i < L.nx; i += blockDim.x) {
        const int j = (int)(row % L.ny), k = (int)(row / L.ny);
        const Nb nb = neighbours(L.nx, L.ny, L.nz, L.zper, i, j, k);
        const T v = apply_at(coefs(L, nb), nb, p);
        q[nb.c] = v;
        loc.add(p[nb.c] * v);
    }
    const double s = block_sum(loc.value(), red);
    if (threadIdx.x == 0) partial[blockIdx.x] = s;
}

template <typename T>
__global__ void k_dot(long n, const T* a, const T* b, double* partial) {
    __shared__ double red[32];
    KSum<typename AccT<T>::type> loc;
    for (long t = blockIdx.x * (long)blockDim.x + threadIdx.x; t < n; t += (long)gridDim.x * blockDim.x)
        loc.add(a[t] * b[t]);
    const double s = block_sum(loc.value(), red);
    if (threadIdx.x == 0) partial[blockIdx.x] = s;
}

template <typename T>
__global__ void k_update_xr(long n, T* x, T* r, const T* p, const T* q, const double* scal, int num, int den) {
    // one FP64 divide per block, not per thread
    __shared__ T alpha_s;
    if (threadIdx.x == 0) alpha_s = (T)(scal[num] / scal[den]);
    __syncthreads();
    const T alpha = alpha_s;
    for (long t = blockIdx.x * (long)blockDim.x + threadIdx.x; t < n; t += (long)gridDim.x * blockDim.x) {
        x[t] += alpha * p[t];
        r[t] -= alpha * q[t];
    }
}

template <typename T>
__global__ void k_update_p(long n, T* p, const T* z, const double* scal, int num, int den) {
    __shared__ T beta_s;
    if (threadIdx.x == 0) beta_s = (T)(scal[num] / scal[den]);
    __syncthreads();
    const T beta = beta_s;
    for (long t = blockIdx.x * (long)blockDim.x + threadIdx.x; t < n; t += (long)gridDim.x * blockDim.x)
        p[t] = z[t] + beta * p[t];
}

template <typename T>
__global__ void k_copy(long n, T* dst, const T* src) {
    for (long t = blockIdx.x * (long)blockDim.x + threadIdx.x; t < n; t += (long)gridDim.x * blockDim.x)
        dst[t] = src[t];
}

// ------------------------------------------------------------ FP32 vector updates, 16-byte accesses
__device__ __forceinline__ float4 f4_axpy(float a, float4 x, float4 y) {   // a x + y
    return make_float4(fmaf(a, x.x, y.x), fmaf(a, x.y, y.y), fmaf(a, x.z, y.z), fmaf(a, x.w, y.w));
}

__global__ void k_update_xr4(long n4, float4* __restrict__ x, float4* __restrict__ r, const float4* __restrict__ p,
                             const float4* __restrict__ q, const double* scal, int num, int den) {
    __shared__ float alpha_s;
    griddep_wait();
    if (threadIdx.x == 0) alpha_s = (float)(scal[num] / scal[den]);
    __syncthreads();
    const float alpha = alpha_s;
    for (long t = blockIdx.x * (long)blockDim.x + threadIdx.x; t < n4; t += (long)gridDim.x * blockDim.x) {
        x[t] = f4_axpy(alpha, p[t], x[t]);
        r[t] = f4_axpy(-alpha, q[t], r[t]);
    }
}

__global__ void k_update_p4(long n4, float4* __restrict__ p, const float4* __restrict__ z, const double* scal,
                            int num, int den) {
    __shared__ float beta_s;
    griddep_wait();
    if (threadIdx.x == 0) beta_s = (float)(scal[num] / scal[den]);
    __syncthreads();
    const float beta = beta_s;
    for (long t = blockIdx.x * (long)blockDim.x + threadIdx.x; t < n4; t += (long)gridDim.x * blockDim.x)
        p[t] = f4_axpy(beta, p[t], z[t]);
}

__global__ void k_dot4(long n4, const float4* __restrict__ a, const float4* __restrict__ b, double* partial) {
    __shared__ double red[32];
    griddep_wait();
    KSum<float> loc;
    for (long t = blockIdx.x * (long)blockDim.x + threadIdx.x; t < n4; t += (long)gridDim.x * blockDim.x) {
        const float4 u = a[t], v = b[t];
        loc.add(u.x * v.x); loc.add(u.y * v.y); loc.add(u.z * v.z); loc.add(u.w * v.w);
    }
    const double s = block_sum(loc.value(), red);
    if (threadIdx.x == 0) partial[blockIdx.x] = s;
}

__global__ void k_copy4(long n4, float4* __restrict__ dst, const float4* __restrict__ src) {
    griddep_wait();
    for (long t = blockIdx.x * (long)blockDim.x + threadIdx.x; t < n4; t += (long)gridDim.x * blockDim.x)
        dst[t] = src[t];
}

// ------------------------------------------------------------ vectorised finest level
// The operator on a cell-eps level in FP32, four consecutive x points per
// thread (16-byte loads of the centre row and of the y and z neighbour rows,
// two scalar loads for the x neighbours outside the quad). DOT: q = A p and
// the block's share of p . q (Kahan within the thread); otherwise the
// residual q = f - A p. Requires nx % 4 == 0.
template <bool DOT>
__global__ void __launch_bounds__(kReduceThreads) k_apply4(LV<float> L, const float* __restrict__ p,
                                                          const float* __restrict__ f, float* __restrict__ q,
                                                          double* partial) {
    __shared__ double red[32];
    const int nx = L.nx, ny = L.ny, nz = L.nz, nx4 = nx >> 2;
    const long pl = (long)nx * ny;
    const int total = nx4 * ny * nz;
    const float hx = 0.5f * L.ihx2, hy = 0.5f * L.ihy2, hz = 0.5f * L.ihz2;
    KSum<float> acc;
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < total; t += gridDim.x * blockDim.x) {
        const int i4 = t % nx4;
        const int row = t / nx4;
        const int j = row % ny, k = row / ny;
        const long rb = (long)k * pl + (long)j * nx;
        const long c = rb + 4 * i4;
        const long cxm = i4 == 0 ? rb + nx - 1 : c - 1;
        const long cxp = i4 == nx4 - 1 ? rb : c + 4;
        const long dym = j == 0 ? (long)(ny - 1) * nx : -(long)nx;
        const long dyp = j == ny - 1 ? -(long)(ny - 1) * nx : (long)nx;
        const long dzm = (k == 0 && L.zper) ? (long)(nz - 1) * pl : -pl;
        const long dzp = (k == nz - 1 && L.zper) ? -(long)(nz - 1) * pl : pl;
        const float4 u0 = *reinterpret_cast<const float4*>(p + c);
        const float4 uym = *reinterpret_cast<const float4*>(p + c + dym);
        const float4 uyp = *reinterpret_cast<const float4*>(p + c + dyp);
        const float4 uzm = *reinterpret_cast<const float4*>(p + c + dzm);
        const float4 uzp = *reinterpret_cast<const float4*>(p + c + dzp);
        const float uxm = p[cxm], uxp = p[cxp];
        const float4 e0 = *reinterpret_cast<const float4*>(L.eps + c);
        const float4 eym = *reinterpret_cast<const float4*>(L.eps + c + dym);
        const float4 eyp = *reinterpret_cast<const float4*>(L.eps + c + dyp);
        const float4 ezm = *reinterpret_cast<const float4*>(L.eps + c + dzm);
        const float4 ezp = *reinterpret_cast<const float4*>(L.eps + c + dzp);
        const float exm = L.eps[cxm], exp_ = L.eps[cxp];
        const float uu[6] = {uxm, u0.x, u0.y, u0.z, u0.w, uxp};
        const float ee[6] = {exm, e0.x, e0.y, e0.z, e0.w, exp_};
        const float ym[4] = {uym.x, uym.y, uym.z, uym.w}, yp[4] = {uyp.x, uyp.y, uyp.z, uyp.w};
        const float zm[4] = {uzm.x, uzm.y, uzm.z, uzm.w}, zp[4] = {uzp.x, uzp.y, uzp.z, uzp.w};
        const float eym_[4] = {eym.x, eym.y, eym.z, eym.w}, eyp_[4] = {eyp.x, eyp.y, eyp.z, eyp.w};
        const float ezm_[4] = {ezm.x, ezm.y, ezm.z, ezm.w}, ezp_[4] = {ezp.x, ezp.y, ezp.z, ezp.w};
        float out[4];
#pragma unroll
        for (int m = 0; m < 4; ++m) {
            const float e = ee[m + 1], u = uu[m + 1];
            const float Au = (e + ee[m + 2]) * hx * (uu[m + 2] - u) - (e + ee[m]) * hx * (u - uu[m]) +
                             (e + eyp_[m]) * hy * (yp[m] - u) - (e + eym_[m]) * hy * (u - ym[m]) +
                             (e + ezp_[m]) * hz * (zp[m] - u) - (e + ezm_[m]) * hz * (u - zm[m]);
            out[m] = Au;
        }
        if constexpr (DOT) {
#pragma unroll
            for (int m = 0; m < 4; ++m) acc.add(uu[m + 1] * out[m]);
            *reinterpret_cast<float4*>(q + c) = make_float4(out[0], out[1], out[2], out[3]);
        } else {
            const float4 fv = *reinterpret_cast<const float4*>(f + c);
            *reinterpret_cast<float4*>(q + c) =
                make_float4(fv.x - out[0], fv.y - out[1], fv.z - out[2], fv.w - out[3]);
        }
    }
    if constexpr (DOT) {
        const double sdot = block_sum(acc.value(), red);
        if (threadIdx.x == 0) partial[blockIdx.x] = sdot;
    }
}

// The same A p (with p.q) or f - A u on the finest level, marching in z: a CTA
// owns whole x rows times kZmRows rows and a chunk of z-planes; each thread
// holds four consecutive x points of one row (rows j0-1 and j0+kZmRows only
// load), keeps its own column of p and eps for planes k-1 .. k+2 in registers
// (loads issued two planes ahead) and passes plane k to its neighbours through
// a double-buffered shared tile, one barrier per plane. Every value crosses
// from L2 once (plus the two halo rows), where the 4-point kernel above loads
// each one five times. DOT: one partial per CTA, the unused partial slots up to
// kReduceBlocks are zeroed so the fixed-order sum stays the same length.
constexpr int kZmRows = 8;

template <bool DOT>
__global__ void __launch_bounds__(1024) k_apply_zm(LV<float> L, const float* __restrict__ p,
                                                   const float* __restrict__ f, float* __restrict__ q,
                                                   double* partial, int sz) {
    extern __shared__ __align__(16) float zsm[];
    __shared__ double red[32];
    griddep_wait();
    const int nx = L.nx, ny = L.ny, nz = L.nz, nx4 = nx >> 2;
    const long pl = (long)nx * ny;
    const int tid = threadIdx.x;
    const int r = tid / nx4, x4 = tid - r * nx4;           // tile row r holds global row j0 - 1 + r
    const bool active = r < kZmRows + 2;
    const int j0 = blockIdx.x * kZmRows;
    const int jr = j0 - 1 + r;
    const int jw = jr < 0 ? jr + ny : (jr >= ny ? jr - ny : jr);
    const bool inner = active && r >= 1 && r <= kZmRows && jr < ny;
    const int z0 = blockIdx.y * sz, z1 = min(z0 + sz, nz);
    const float hx = 0.5f * L.ihx2, hy = 0.5f * L.ihy2, hz = 0.5f * L.ihz2;
    const int rowlen = nx, tile = (kZmRows + 2) * nx;
    float* sp = zsm;                                      // [2][kZmRows+2][nx] of p
    float* se = zsm + 2 * tile;                           // the same of eps
    const long col = (long)jw * nx + 4 * x4;
    auto off = [&](int k) -> long {                       // plane k (wrapped; -1 and nz are the walls)
        if (L.zper) k = k < 0 ? k + nz : (k >= nz ? k - nz : k);
        else if (k > nz) k = nz;                          // the prefetch past the last wall: never used
        return (long)k * pl + col;
    };
    auto ld4 = [](const float* a, long o) { return *reinterpret_cast<const float4*>(a + o); };
    float4 Pm = make_float4(0.f, 0.f, 0.f, 0.f), P0 = Pm, Pp = Pm, Pn = Pm;
    float4 Em = Pm, E0 = Pm, Ep = Pm, En = Pm;
    KSum<float> acc;
    if (z0 < nz) {
        if (active) {
            Pm = ld4(p, off(z0 - 1)); Em = ld4(L.eps, off(z0 - 1));
            P0 = ld4(p, off(z0)); E0 = ld4(L.eps, off(z0));
            Pp = ld4(p, off(z0 + 1)); Ep = ld4(L.eps, off(z0 + 1));
        }
        const int xl = x4 == 0 ? nx - 1 : 4 * x4 - 1, xr = x4 == nx4 - 1 ? 0 : 4 * x4 + 4;
        for (int k = z0; k < z1; ++k) {
            const int b = (k - z0) & 1;
            float* bp = sp + b * tile;
            float* be = se + b * tile;
            if (active) {
                Pn = ld4(p, off(k + 2));                  // planes up to nz exist (wrapped or the wall)
                En = ld4(L.eps, off(k + 2));
                *reinterpret_cast<float4*>(bp + r * rowlen + 4 * x4) = P0;
                *reinterpret_cast<float4*>(be + r * rowlen + 4 * x4) = E0;
            }
            __syncthreads();
            if (inner) {
                const float* pr = bp + r * rowlen;
                const float* er = be + r * rowlen;
                const float4 pym = *reinterpret_cast<const float4*>(pr - rowlen + 4 * x4);
                const float4 pyp = *reinterpret_cast<const float4*>(pr + rowlen + 4 * x4);
                const float4 eym = *reinterpret_cast<const float4*>(er - rowlen + 4 * x4);
                const float4 eyp = *reinterpret_cast<const float4*>(er + rowlen + 4 * x4);
                const float uu[6] = {pr[xl], P0.x, P0.y, P0.z, P0.w, pr[xr]};
                const float ee[6] = {er[xl], E0.x, E0.y, E0.z, E0.w, er[xr]};
                const float ym[4] = {pym.x, pym.y, pym.z, pym.w}, yp[4] = {pyp.x, pyp.y, pyp.z, pyp.w};
                const float zm[4] = {Pm.x, Pm.y, Pm.z, Pm.w}, zp[4] = {Pp.x, Pp.y, Pp.z, Pp.w};
                const float eym_[4] = {eym.x, eym.y, eym.z, eym.w}, eyp_[4] = {eyp.x, eyp.y, eyp.z, eyp.w};
                const float ezm_[4] = {Em.x, Em.y, Em.z, Em.w}, ezp_[4] = {Ep.x, Ep.y, Ep.z, Ep.w};
                float out[4];
#pragma unroll
                for (int m = 0; m < 4; ++m) {
                    const float e = ee[m + 1], u = uu[m + 1];
                    out[m] = (e + ee[m + 2]) * hx * (uu[m + 2] - u) - (e + ee[m]) * hx * (u - uu[m]) +
                             (e + eyp_[m]) * hy * (yp[m] - u) - (e + eym_[m]) * hy * (u - ym[m]) +
                             (e + ezp_[m]) * hz * (zp[m] - u) - (e + ezm_[m]) * hz * (u - zm[m]);
                }
                const long o = (long)k * pl + col;
                if constexpr (DOT) {
#pragma unroll
                    for (int m = 0; m < 4; ++m) acc.add(uu[m + 1] * out[m]);
                    *reinterpret_cast<float4*>(q + o) = make_float4(out[0], out[1], out[2], out[3]);
                } else {
                    const float4 fv = ld4(f, o);
                    *reinterpret_cast<float4*>(q + o) =
                        make_float4(fv.x - out[0], fv.y - out[1], fv.z - out[2], fv.w - out[3]);
                }
            }
            Pm = P0; P0 = Pp; Pp = Pn;
            Em = E0; E0 = Ep; Ep = En;
        }
    }
    if constexpr (DOT) {
        const double sdot = block_sum(acc.value(), red);
        const int nb = gridDim.x * gridDim.y, bid = blockIdx.x + gridDim.x * blockIdx.y;
        if (threadIdx.x == 0) partial[bid] = sdot;
        if (bid == 0)
            for (int i = nb + threadIdx.x; i < kReduceBlocks; i += blockDim.x) partial[i] = 0.0;
    }
}

// grid of the z-marching apply: y tiles times z chunks, one wave of resident
// CTAs and at most kReduceBlocks CTAs; false when the level does not fit it
bool apply_zm_grid(const LV<float>& L, dim3& grid, int& sz, size_t& smem, int& threads) {
    if (!L.cell || L.nx % 4 != 0) return false;
    threads = (kZmRows + 2) * (L.nx / 4);
    if (threads > 1024) return false;
    threads = (threads + 31) / 32 * 32;
    smem = sizeof(float) * 4 * (kZmRows + 2) * (size_t)L.nx;
    if (smem > 48 * 1024) return false;                   // the default dynamic shared memory
    const int ty = (L.ny + kZmRows - 1) / kZmRows;
    int per_sm = 65536 / (64 * threads);                  // by registers (64 per thread)
    if (per_sm > 2048 / threads) per_sm = 2048 / threads;
    if (per_sm > 8) per_sm = 8;
    if (per_sm < 1) per_sm = 1;
    int tz = 152 * per_sm / ty;
    if (tz > kReduceBlocks / ty) tz = kReduceBlocks / ty;
    if (tz > L.nz) tz = L.nz;
    if (tz < 1) return false;
    sz = (L.nz + tz - 1) / tz;
    grid = dim3(ty, (L.nz + sz - 1) / sz);
    return (long)grid.x * grid.y <= kReduceBlocks;
}

// ------------------------------------------------------------ reductions
// out[c] = sum_b partial[b * ncomp + c], in a fixed order
__global__ void k_finalize(const double* partial, int nparts, int ncomp, double* out) {
    __shared__ double red[32];
    griddep_wait();
    for (int c = 0; c < ncomp; ++c) {
        double loc = 0.0;
        for (int b = threadIdx.x; b < nparts; b += blockDim.x) loc += partial[(long)b * ncomp + c];
        const double s = block_sum(loc, red);
        if (threadIdx.x == 0) out[c] = s;
        __syncthreads();
    }
}

// (s, e) += (x, y): a compensated FP32 pair accumulation (Knuth's two-sum of the
// leading parts, the low parts added)
__device__ __forceinline__ void pair_acc(float& s, float& e, float x, float y) {
    const float t = s + x;
    const float z = t - s;
    e += ((s - (t - z)) + (x - z)) + y;
    s = t;
}

// partial[3b..3b+2] = sum rho, sum |rho|, sum rho^2. Each thread sums its values
// as compensated float pairs (the value split by split_to_float2, the square as
// an exact product hi*hi by FMA plus the cross terms): no FP64 instruction per
// value, about 2^-44 of each thread's sum; the threads' sums meet in FP64.
__global__ void k_rho_stats(long n, const double* rho, double* partial) {
    __shared__ double red[32];
    float as = 0.f, ae = 0.f, bs = 0.f, be = 0.f, cs = 0.f, ce = 0.f;
    for (long t = blockIdx.x * (long)blockDim.x + threadIdx.x; t < n; t += (long)gridDim.x * blockDim.x) {
        const float2 v = split_to_float2(rho[t]);
        pair_acc(as, ae, v.x, v.y);
        const bool neg = v.x < 0.f;
        pair_acc(bs, be, neg ? -v.x : v.x, neg ? -v.y : v.y);
        const float p = v.x * v.x;
        const float q = fmaf(v.x, v.x, -p) + 2.f * v.x * v.y;
        pair_acc(cs, ce, p, q);
    }
    double a = (double)as + (double)ae, b = (double)bs + (double)be, c = (double)cs + (double)ce;
    double s = block_sum(a, red);
    if (threadIdx.x == 0) partial[3 * blockIdx.x] = s;
    s = block_sum(b, red);
    if (threadIdx.x == 0) partial[3 * blockIdx.x + 1] = s;
    s = block_sum(c, red);
    if (threadIdx.x == 0) partial[3 * blockIdx.x + 2] = s;
}

__global__ void k_sub_mean(long n, double* x, const double* sum_slot, double scale) {
    const double m = sum_slot[0] * scale;
    for (long t = blockIdx.x * (long)blockDim.x + threadIdx.x; t < n; t += (long)gridDim.x * blockDim.x)
        x[t] -= m;
}

// ------------------------------------------------------------ FP64 full box
// r = -4 pi rho - A phi (periodic, cell eps, FP64); partial[2b] = sum r^2,
// partial[2b+1] = sum phi
template <typename T>
__global__ void __launch_bounds__(kReduceThreads) k_residual64(Geo g, const double* phi, const double* rho,
                                                               const double* eps, T* r_out, double* partial) {
    __shared__ double red[32];
    const long n = (long)g.nx * g.ny * g.nz;
    const double hx = g.c2x, hy = g.c2y, hz = g.c2z;
    const double fpi = 4.0 * kPi;
    double s2 = 0.0, sp = 0.0;
    (void)n;
    for (long row = blockIdx.x; row < (long)g.ny * g.nz; row += gridDim.x)
    for (int i = threadIdx.x; i < g.nx; i += blockDim.x) {
        const int j = (int)(row % g.ny), k = (int)(row / g.ny);
        const Nb nb = neighbours(g.nx, g.ny, g.nz, 1, i, j, k);
        const double p0 = phi[nb.c];
        const double pxp = phi[nb.xp], pxm = phi[nb.xm], pyp = phi[nb.yp], pym = phi[nb.ym];
        const double pzp = phi[nb.zp], pzm = phi[nb.zm];
        const double e0 = eps[nb.c], exp_ = eps[nb.xp], exm = eps[nb.xm], eyp = eps[nb.yp], eym = eps[nb.ym];
        const double ezp = eps[nb.zp], ezm = eps[nb.zm];
        double r = -fpi * rho[nb.c];
        // A phi is exactly 0 where phi and its six neighbours are 0 (a cold start):
        // the FP64 stencil is then skipped, with the same result
        if (p0 != 0.0 || pxp != 0.0 || pxm != 0.0 || pyp != 0.0 || pym != 0.0 || pzp != 0.0 || pzm != 0.0) {
            const double ax = (e0 + exp_) * (pxp - p0) - (e0 + exm) * (p0 - pxm);
            const double ay = (e0 + eyp) * (pyp - p0) - (e0 + eym) * (p0 - pym);
            const double az = (e0 + ezp) * (pzp - p0) - (e0 + ezm) * (p0 - pzm);
            r -= hx * ax + hy * ay + hz * az;
        }
        r_out[nb.c] = (T)r;
        s2 += r * r;
        sp += p0;
    }
    double s = block_sum(s2, red);
    if (threadIdx.x == 0) partial[2 * blockIdx.x] = s;
    s = block_sum(sp, red);
    if (threadIdx.x == 0) partial[2 * blockIdx.x + 1] = s;
}

// ------------------------------------------------------------ df64 full box (mixed precision)
// The outer residual of the mixed-precision solve in df64: every value is an
// unevaluated sum hi + lo of two FP32 numbers (Dekker 1971, Knuth's two-sum),
// which carries ~48 bits on the FP32 pipe (GB300's FP64 pipe runs at 1/64 of
// it). phi, eps and b = -4 pi rho are kept as (hi, lo) pairs; the residual of
// the pair-rounded phi is within ~1e-11 of ||b|| of the FP64 one, far below the
// tolerances this path serves (the host uses it only for tol >= 1e-10).
struct d2 { float hi, lo; };
__device__ __forceinline__ d2 d2_quick(float s, float e) {
    const float t = s + e;
    return {t, e - (t - s)};
}
__device__ __forceinline__ d2 d2_add(d2 a, d2 b) {
    const float s = a.hi + b.hi;
    const float v = s - a.hi;
    float e = (a.hi - (s - v)) + (b.hi - v);
    e += a.lo + b.lo;
    return d2_quick(s, e);
}
__device__ __forceinline__ d2 d2_neg(d2 a) { return {-a.hi, -a.lo}; }
__device__ __forceinline__ d2 d2_mul(d2 a, d2 b) {
    const float p = a.hi * b.hi;
    float e = fmaf(a.hi, b.hi, -p);
    e = fmaf(a.hi, b.lo, e);
    e = fmaf(a.lo, b.hi, e);
    return d2_quick(p, e);
}
__device__ __forceinline__ d2 d2_ld(const float2* p, long i) {
    const float2 v = p[i];
    return {v.x, v.y};
}

// dst = (hi, lo) split of scale * src
// optionally: *nonzero |= 1 if any value is nonzero (not +-0), and hi_out = the
// leading floats (the value rounded to FP32)
__global__ void k_to_df(long n, const double* __restrict__ src, double scale, float2* __restrict__ dst,
                        int* nonzero, float* __restrict__ hi_out) {
    // the split by integer instructions (split_to_float2): one FP64 multiply per
    // value where scale != 1 instead of five FP64-pipe instructions
    const bool one = scale == 1.0;
    bool nz = false;
    for (long t = blockIdx.x * (long)blockDim.x + threadIdx.x; t < n; t += (long)gridDim.x * blockDim.x) {
        const double v = src[t];
        nz |= (__double_as_longlong(v) << 1) != 0;
        const float2 p = split_to_float2(one ? v : scale * v);
        dst[t] = p;
        if (hi_out) hi_out[t] = p.x;
    }
    if (nonzero && __any_sync(0xffffffffu, nz) && (threadIdx.x & 31) == 0) atomicOr(nonzero, 1);
}

// r = b - A phi on the periodic full box (cell eps, face means), in df64;
// r_out = the residual rounded to FP32; partial[2b] = block's sum r^2,
// partial[2b+1] = block's sum phi (compensated FP32 sums, FP64 across threads)
__global__ void __launch_bounds__(kReduceThreads) k_residual_df(Geo g, const float2* __restrict__ phid,
                                                               const float2* __restrict__ bd,
                                                               const float2* __restrict__ epsd, d2 cxd, d2 cyd,
                                                               d2 czd, float* __restrict__ r_out,
                                                               double* partial) {
    __shared__ double red[32];
    KSum<float> s2, sp;
    for (long row = blockIdx.x; row < (long)g.ny * g.nz; row += gridDim.x)
    for (int i = threadIdx.x; i < g.nx; i += blockDim.x) {
        const int j = (int)(row % g.ny), k = (int)(row / g.ny);
        const Nb nb = neighbours(g.nx, g.ny, g.nz, 1, i, j, k);
        const d2 p0 = d2_ld(phid, nb.c), e0 = d2_ld(epsd, nb.c);
        const d2 mp0 = d2_neg(p0);
        auto axis = [&](long ip, long im, d2 c) {
            const d2 fp = d2_mul(d2_add(e0, d2_ld(epsd, ip)), d2_add(d2_ld(phid, ip), mp0));
            const d2 fm = d2_mul(d2_add(e0, d2_ld(epsd, im)), d2_add(p0, d2_neg(d2_ld(phid, im))));
            return d2_mul(c, d2_add(fp, d2_neg(fm)));
        };
        const d2 ap = d2_add(d2_add(axis(nb.xp, nb.xm, cxd), axis(nb.yp, nb.ym, cyd)), axis(nb.zp, nb.zm, czd));
        const d2 r = d2_add(d2_ld(bd, nb.c), d2_neg(ap));
        r_out[nb.c] = r.hi;
        s2.add(r.hi * r.hi);
        sp.add(p0.hi);
        sp.add(p0.lo);
    }
    double s = block_sum(s2.value(), red);
    if (threadIdx.x == 0) partial[2 * blockIdx.x] = s;
    s = block_sum(sp.value(), red);
    if (threadIdx.x == 0) partial[2 * blockIdx.x + 1] = s;
}

// The same residual, four consecutive x points per thread (nx % 4 == 0):
// 16-byte loads of the (hi, lo) pairs of the centre, y and z neighbour rows.
__device__ __forceinline__ void ld4(const float2* p, long i, d2 (&v)[4]) {
    const float4 a = *reinterpret_cast<const float4*>(p + i);
    const float4 b = *reinterpret_cast<const float4*>(p + i + 2);
    v[0] = {a.x, a.y}; v[1] = {a.z, a.w}; v[2] = {b.x, b.y}; v[3] = {b.z, b.w};
}

__global__ void __launch_bounds__(kReduceThreads) k_residual_df4(Geo g, const float2* __restrict__ phid,
                                                                const float2* __restrict__ bd,
                                                                const float2* __restrict__ epsd, d2 cxd, d2 cyd,
                                                                d2 czd, float* __restrict__ r_out,
                                                                double* partial) {
    __shared__ double red[32];
    KSum<float> s2, sp;
    const int nx = g.nx, ny = g.ny, nz = g.nz, nx4 = nx >> 2;
    const long pl = (long)nx * ny;
    const int total = nx4 * ny * nz;
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < total; t += gridDim.x * blockDim.x) {
        const int i4 = t % nx4;
        const int row = t / nx4;
        const int j = row % ny, k = row / ny;
        const long rb = (long)k * pl + (long)j * nx;
        const long c = rb + 4 * i4;
        const long cxm = i4 == 0 ? rb + nx - 1 : c - 1;
        const long cxp = i4 == nx4 - 1 ? rb : c + 4;
        const long dym = j == 0 ? (long)(ny - 1) * nx : -(long)nx;
        const long dyp = j == ny - 1 ? -(long)(ny - 1) * nx : (long)nx;
        const long dzm = k == 0 ? (long)(nz - 1) * pl : -pl;
        const long dzp = k == nz - 1 ? -(long)(nz - 1) * pl : pl;
        d2 p[6], e[6], pym[4], pyp[4], pzm[4], pzp[4], eym[4], eyp[4], ezm[4], ezp[4], b[4];
        {
            d2 v[4];
            ld4(phid, c, v);
            p[1] = v[0]; p[2] = v[1]; p[3] = v[2]; p[4] = v[3];
            ld4(epsd, c, v);
            e[1] = v[0]; e[2] = v[1]; e[3] = v[2]; e[4] = v[3];
        }
        p[0] = d2_ld(phid, cxm); p[5] = d2_ld(phid, cxp);
        e[0] = d2_ld(epsd, cxm); e[5] = d2_ld(epsd, cxp);
        ld4(phid, c + dym, pym); ld4(phid, c + dyp, pyp); ld4(phid, c + dzm, pzm); ld4(phid, c + dzp, pzp);
        ld4(epsd, c + dym, eym); ld4(epsd, c + dyp, eyp); ld4(epsd, c + dzm, ezm); ld4(epsd, c + dzp, ezp);
        ld4(bd, c, b);
        float out[4];
#pragma unroll
        for (int m = 0; m < 4; ++m) {
            const d2 p0 = p[m + 1], e0 = e[m + 1], mp0 = d2_neg(p0);
            auto face = [&](d2 en, d2 pn) { return d2_mul(d2_add(e0, en), d2_add(pn, mp0)); };
            // A phi = sum_axes c [ (e0+e+)(p+ - p0) + (e0+e-)(p- - p0) ]
            const d2 ax = d2_mul(cxd, d2_add(face(e[m + 2], p[m + 2]), face(e[m], p[m])));
            const d2 ay = d2_mul(cyd, d2_add(face(eyp[m], pyp[m]), face(eym[m], pym[m])));
            const d2 az = d2_mul(czd, d2_add(face(ezp[m], pzp[m]), face(ezm[m], pzm[m])));
            const d2 r = d2_add(b[m], d2_neg(d2_add(d2_add(ax, ay), az)));
            out[m] = r.hi;
            s2.add(r.hi * r.hi);
            sp.add(p0.hi);
            sp.add(p0.lo);
        }
        *reinterpret_cast<float4*>(r_out + c) = make_float4(out[0], out[1], out[2], out[3]);
    }
    double sum = block_sum(s2.value(), red);
    if (threadIdx.x == 0) partial[2 * blockIdx.x] = sum;
    sum = block_sum(sp.value(), red);
    if (threadIdx.x == 0) partial[2 * blockIdx.x + 1] = sum;
}

// phid += e (df64 + FP32, 16-byte accesses: two points per float4), for the
// mixed-precision full-box loop that keeps phi as pairs
__global__ void k_update_phid(long n2, float4* __restrict__ phid, const float2* __restrict__ e) {
    for (long t = blockIdx.x * (long)blockDim.x + threadIdx.x; t < n2; t += (long)gridDim.x * blockDim.x) {
        const float4 p = phid[t];
        const float2 v = e[t];
        const d2 a = d2_add({p.x, p.y}, {v.x, 0.f});
        const d2 b = d2_add({p.z, p.w}, {v.y, 0.f});
        phid[t] = make_float4(a.hi, a.lo, b.hi, b.lo);
    }
}

// phi = (hi + lo) - mean, mean = scale * sum_slot[0], in FP64 (two additions; the
// floats converted by their bits): the pairs back to doubles and the gauge in one
// pass instead of a conversion pass and a read-modify-write pass over the FP64 field
__global__ void k_from_df_gauge(long n, const float2* __restrict__ src, const double* sum_slot, double scale,
                                double* __restrict__ dst) {
    const double m = sum_slot[0] * scale;
    for (long t = blockIdx.x * (long)blockDim.x + threadIdx.x; t < n; t += (long)gridDim.x * blockDim.x) {
        const float2 v = src[t];
        dst[t] = (f32_to_f64(v.x) + f32_to_f64(v.y)) - m;
    }
}

// phi += e_full (+ e_band on the band planes); band plane kb <-> global plane
// (band_first + kb) mod nz, kb < band_nz
template <typename T>
__global__ void k_update_phi(Geo g, double* phi, const T* e_full, const T* e_band, int band_first, int band_nz) {
    const long n = (long)g.nx * g.ny * g.nz;
    const long pl = plane_of(g.nx, g.ny);
    for (long t = blockIdx.x * (long)blockDim.x + threadIdx.x; t < n; t += (long)gridDim.x * blockDim.x) {
        double v = e_full ? (double)e_full[t] : 0.0;
        if (e_band) {
            const int k = (int)(t / pl);
            int kb = k - band_first;
            if (kb < 0) kb += g.nz;
            if (kb < band_nz) v += (double)e_band[t - k * pl + kb * pl];
        }
        phi[t] += v;
    }
}

// ------------------------------------------------------------ band coupling
template <typename T>
__global__ void k_cast(long n, const double* a, T* b) {
    for (long t = blockIdx.x * (long)blockDim.x + threadIdx.x; t < n; t += (long)gridDim.x * blockDim.x)
        b[t] = (T)a[t];
}

// band eps planes kb = -1 .. band_nz (walls included) from the full-box eps
template <typename T>
__global__ void k_band_eps(Geo g, const T* eps, int first, int band_nz, T* beps) {
    const long pl = plane_of(g.nx, g.ny);
    const long n = pl * (band_nz + 2);
    for (long t = blockIdx.x * (long)blockDim.x + threadIdx.x; t < n; t += (long)gridDim.x * blockDim.x) {
        const int kb = (int)(t / pl) - 1;
        const int k = ((first + kb) % g.nz + g.nz) % g.nz;
        beps[t - pl] = eps[(t % pl) + k * pl];
    }
}

// f_band = r - A e_vac on the band's interior planes (full-box operator, periodic)
template <typename T>
__global__ void k_band_rhs(Geo g, const T* eps, const T* r, const T* ev, int first, int band_nz, T* fb) {
    const long pl = plane_of(g.nx, g.ny);
    const T hx = (T)g.c2x, hy = (T)g.c2y, hz = (T)g.c2z;
    for (long row = blockIdx.x; row < (long)g.ny * band_nz; row += gridDim.x)
    for (int i = threadIdx.x; i < g.nx; i += blockDim.x) {
        const int j = (int)(row % g.ny), kb = (int)(row / g.ny);
        const int k = (first + kb) % g.nz;
        const long t = kb * pl + (long)j * g.nx + i;
        const Nb nb = neighbours(g.nx, g.ny, g.nz, 1, i, j, k);
        const T e0 = eps[nb.c], p0 = ev[nb.c];
        const T ax = (e0 + eps[nb.xp]) * (ev[nb.xp] - p0) - (e0 + eps[nb.xm]) * (p0 - ev[nb.xm]);
        const T ay = (e0 + eps[nb.yp]) * (ev[nb.yp] - p0) - (e0 + eps[nb.ym]) * (p0 - ev[nb.ym]);
        const T az = (e0 + eps[nb.zp]) * (ev[nb.zp] - p0) - (e0 + eps[nb.zm]) * (p0 - ev[nb.zm]);
        fb[t] = r[nb.c] - (hx * ax + hy * ay + hz * az);
    }
}

// ------------------------------------------------------------ FGMRES (inner, working precision)
// partial[b * nv + i] = block b's share of w . v_i (accumulated in FP64).
// The vector count is a template argument so the accumulators stay in registers.
template <typename T, int NV>
__global__ void __launch_bounds__(kReduceThreads) k_multidot(long n, const T* __restrict__ w, TVecList<T> V,
                                                             double* partial) {
    __shared__ double red[32];
    using A = typename AccT<T>::type;
    KSum<A> loc[NV];
    for (long t = blockIdx.x * (long)blockDim.x + threadIdx.x; t < n; t += (long)gridDim.x * blockDim.x) {
        const A wv = w[t];
#pragma unroll
        for (int i = 0; i < NV; ++i) loc[i].add(wv * V.v[i][t]);
    }
#pragma unroll
    for (int i = 0; i < NV; ++i) {
        const double s = block_sum(loc[i].value(), red);
        if (threadIdx.x == 0) partial[(long)blockIdx.x * NV + i] = s;
    }
}

// w -= sum_i h[i] v_i; partial[b] = block share of |w|^2
template <typename T, int NV>
__global__ void __launch_bounds__(kReduceThreads) k_multiaxpy_norm(long n, T* __restrict__ w, TVecList<T> V,
                                                                   const double* h, double* partial) {
    __shared__ double red[32];
    using A = typename AccT<T>::type;
    A hs[NV];
#pragma unroll
    for (int i = 0; i < NV; ++i) hs[i] = (A)h[i];
    KSum<A> loc;
    for (long t = blockIdx.x * (long)blockDim.x + threadIdx.x; t < n; t += (long)gridDim.x * blockDim.x) {
        A x = w[t];
#pragma unroll
        for (int i = 0; i < NV; ++i) x -= hs[i] * V.v[i][t];
        w[t] = (T)x;
        loc.add(x * x);
    }
    const double s = block_sum(loc.value(), red);
    if (threadIdx.x == 0) partial[blockIdx.x] = s;
}

// dst = src / sqrt(*sq)
template <typename T>
__global__ void k_scale_by_norm(long n, const T* src, T* dst, const double* sq) {
    __shared__ T f_s;
    if (threadIdx.x == 0) f_s = (T)(1.0 / sqrt(sq[0]));
    __syncthreads();
    const T f = f_s;
    for (long t = blockIdx.x * (long)blockDim.x + threadIdx.x; t < n; t += (long)gridDim.x * blockDim.x)
        dst[t] = src[t] * f;
}

// z = e_vac, plus the band correction on the band planes
template <typename T>
__global__ void k_combine(Geo g, const T* ev, const T* eb, int first, int band_nz, T* z) {
    const long pl = plane_of(g.nx, g.ny);
    for (long row = blockIdx.x; row < (long)g.ny * g.nz; row += gridDim.x) {
        const int j = (int)(row % g.ny), k = (int)(row / g.ny);
        int kb = k - first;
        if (kb < 0) kb += g.nz;
        const long t0 = k * pl + (long)j * g.nx;
        const long b0 = kb * pl + (long)j * g.nx;
        for (int i = threadIdx.x; i < g.nx; i += blockDim.x) {
            T v = ev[t0 + i];
            if (kb < band_nz) v += eb[b0 + i];
            z[t0 + i] = v;
        }
    }
}

// x = sum_j y[j] z_j
template <typename T>
__global__ void k_krylov_combine(long n, T* x, TVecList<T> Z, const double* y) {
    __shared__ double ys[kMaxKrylov];
    if (threadIdx.x < Z.n) ys[threadIdx.x] = y[threadIdx.x];
    __syncthreads();
    using A = typename AccT<T>::type;
    for (long t = blockIdx.x * (long)blockDim.x + threadIdx.x; t < n; t += (long)gridDim.x * blockDim.x) {
        A acc = 0;
        for (int j = 0; j < Z.n; ++j) acc += (A)ys[j] * Z.v[j][t];
        x[t] = (T)acc;
    }
}

// x += y
template <typename T>
__global__ void k_axpy1(long n, T* x, const T* y) {
    for (long t = blockIdx.x * (long)blockDim.x + threadIdx.x; t < n; t += (long)gridDim.x * blockDim.x) x[t] += y[t];
}

// ------------------------------------------------------------ persistent coarse V-cycle
// The bottom of the V-cycle (levels S.l0 .. S.L-1, each small) in ONE CTA:
// every smoothing colour, residual, restriction, the coarsest solve and each
// prolongation is a phase over the level's points, separated by
// __syncthreads. Replaces a chain of tiny, launch-bound kernels.
template <typename T>
__device__ void blk_rbgs(const LV<T>& L, T* u, const T* f, int color) {
    const int hx = L.nx >> 1;
    const int np = hx * L.ny * L.nz;
    for (int t = threadIdx.x; t < np; t += blockDim.x) {
        const int i2 = t % hx, r = t / hx, j = r % L.ny, k = r / L.ny;
        const int i = 2 * i2 + ((j + k + color) & 1);
        const Nb n = neighbours(L.nx, L.ny, L.nz, L.zper, i, j, k);
        const Co<T> o = coefs(L, n);
        const T sm = o.xp * u[n.xp] + o.xm * u[n.xm] + o.yp * u[n.yp] + o.ym * u[n.ym] + o.zp * u[n.zp] +
                     o.zm * u[n.zm];
        const T d = o.xp + o.xm + o.yp + o.ym + o.zp + o.zm;
        u[n.c] = (sm - f[n.c]) / d;
    }
}

template <typename T>
__device__ void blk_residual(const LV<T>& L, const T* u, const T* f, T* r) {
    const int np = L.nx * L.ny * L.nz;
    for (int t = threadIdx.x; t < np; t += blockDim.x) {
        const int i = t % L.nx, q = t / L.nx, j = q % L.ny, k = q / L.ny;
        const Nb nb = neighbours(L.nx, L.ny, L.nz, L.zper, i, j, k);
        r[nb.c] = f[nb.c] - apply_at(coefs(L, nb), nb, u);
    }
}

template <typename T>
__device__ void blk_restrict(const LV<T>& F, const T* r, const LV<T>& C, T* fc) {
    const int np = C.nx * C.ny * C.nz;
    const int zoff = F.zper ? 0 : 1;
    const long pl = (long)F.nx * F.ny;
    for (int t = threadIdx.x; t < np; t += blockDim.x) {
        const int I = t % C.nx, q = t / C.nx, J = q % C.ny, K = q / C.ny;
        const int kf = 2 * K + zoff;
        T acc = 0;
        for (int dz = -1; dz <= 1; ++dz) {
            int kk = kf + dz;
            if (F.zper) kk = (kk + F.nz) % F.nz;
            const T wz = dz == 0 ? (T)0.5 : (T)0.25;
            for (int dy = -1; dy <= 1; ++dy) {
                const int jj = (2 * J + dy + F.ny) % F.ny;
                const T wy = dy == 0 ? (T)0.5 : (T)0.25;
                const long base = kk * pl + (long)jj * F.nx;
                const int ic = 2 * I;
                const int im = ic == 0 ? F.nx - 1 : ic - 1;
                const int ip = ic == F.nx - 1 ? 0 : ic + 1;
                acc += wz * wy * ((T)0.25 * r[base + im] + (T)0.5 * r[base + ic] + (T)0.25 * r[base + ip]);
            }
        }
        fc[I + (long)C.nx * (J + (long)C.ny * K)] = acc;
    }
}

template <typename T>
__device__ void blk_prolong_add(const LV<T>& F, T* u, const LV<T>& C, const T* uc) {
    const int np = F.nx * F.ny * F.nz;
    const int zoff = F.zper ? 0 : 1;
    const long cpl = (long)C.nx * C.ny;
    for (int t = threadIdx.x; t < np; t += blockDim.x) {
        const int i = t % F.nx, q = t / F.nx, j = q % F.ny, k = q / F.ny;
        int xi[2], yi[2], zi[2];
        T xw[2], yw[2], zw[2];
        int nxp, nyp, nzp;
        if (i & 1) { xi[0] = i >> 1; xi[1] = (xi[0] + 1) % C.nx; xw[0] = xw[1] = (T)0.5; nxp = 2; }
        else { xi[0] = i >> 1; xw[0] = 1; nxp = 1; }
        if (j & 1) { yi[0] = j >> 1; yi[1] = (yi[0] + 1) % C.ny; yw[0] = yw[1] = (T)0.5; nyp = 2; }
        else { yi[0] = j >> 1; yw[0] = 1; nyp = 1; }
        const int kk = k - zoff;
        if (kk & 1) {
            zi[0] = (kk - 1) >> 1;
            zi[1] = zi[0] + 1;
            if (C.zper && zi[1] == C.nz) zi[1] = 0;
            zw[0] = zw[1] = (T)0.5;
            nzp = 2;
        } else { zi[0] = kk >> 1; zw[0] = 1; nzp = 1; }
        T acc = 0;
        for (int cc = 0; cc < nzp; ++cc)
            for (int b = 0; b < nyp; ++b)
                for (int a = 0; a < nxp; ++a)
                    acc += zw[cc] * yw[b] * xw[a] * uc[xi[a] + (long)C.nx * yi[b] + cpl * zi[cc]];
        u[i + (long)F.nx * (j + (long)F.ny * k)] += acc;
    }
}

template <typename T>
__global__ void __launch_bounds__(1024) k_coarse_vcycle(CoarseSet<T> S) {
    __shared__ double red[32];
    griddep_wait();
    for (int l = S.l0; l < S.L - 1; ++l) {
        const LV<T>& V = S.lv[l];
        const int np = V.nx * V.ny * V.nz;
        for (int t = threadIdx.x; t < np; t += blockDim.x) S.u[l][t] = 0;
        __syncthreads();
        for (int it = 0; it < S.nu1; ++it) {
            blk_rbgs(V, S.u[l], S.f[l], 0);
            __syncthreads();
            blk_rbgs(V, S.u[l], S.f[l], 1);
            __syncthreads();
        }
        blk_residual(V, S.u[l], S.f[l], S.r[l]);
        __syncthreads();
        blk_restrict(V, S.r[l], S.lv[l + 1], S.f[l + 1]);
        __syncthreads();
    }
    {
        // coarsest: u = inv (f - mean f) (periodic) or inv f (Dirichlet)
        const LV<T>& C = S.lv[S.L - 1];
        const T* f = S.f[S.L - 1];
        double loc = 0.0;
        for (int p = threadIdx.x; p < S.nc; p += blockDim.x) loc += (double)f[p];
        const double tot = block_sum(loc, red);
        __shared__ double mean;
        if (threadIdx.x == 0) mean = C.zper ? tot / S.nc : 0.0;
        __syncthreads();
        const T mf = (T)mean;
        const int lane = threadIdx.x & 31, nw = blockDim.x >> 5;
        for (int p = threadIdx.x >> 5; p < S.nc; p += nw) {
            const T* row = S.minv + (long)p * S.nc;
            T acc = 0;
            for (int q = lane; q < S.nc; q += 32) acc += row[q] * (f[q] - mf);
            for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
            if (lane == 0) S.u[S.L - 1][p] = acc;
        }
        __syncthreads();
    }
    for (int l = S.L - 2; l >= S.l0; --l) {
        const LV<T>& V = S.lv[l];
        blk_prolong_add(V, S.u[l], S.lv[l + 1], S.u[l + 1]);
        __syncthreads();
        for (int it = 0; it < S.nu2; ++it) {
            blk_rbgs(V, S.u[l], S.f[l], 1);
            __syncthreads();
            blk_rbgs(V, S.u[l], S.f[l], 0);
            __syncthreads();
        }
    }
}

// The same bottom of the V-cycle with the levels' fields and face coefficients
// held in shared memory: each phase then waits on shared-memory latency rather
// than on an L2 round trip. The arrays keep the padded layout of the global
// levels (one plane below and one above: the Dirichlet walls of a band); u
// starts at zero, f of the first level comes from the level above, and u of
// the first level goes back to global memory for the prolongation above.
constexpr size_t kCoarseSmemBytes = 200 * 1024;

// n / d for n, d < 2^16 from m = ceil(2^32 / d): (n m) >> 32 is exact there,
// and costs one wide multiply instead of a division routine
__device__ __forceinline__ int qdiv(int n, unsigned long long m) {
    return (int)(((unsigned long long)(unsigned)n * m) >> 32);
}
__device__ __forceinline__ unsigned long long qmagic(int d) {
    return (0x100000000ull + (unsigned long long)d - 1ull) / (unsigned long long)d;
}
struct QDiv { unsigned long long nx, ny, hx; };      // magics for a level's nx, ny and nx / 2

// the block phases of the shared-memory coarse V-cycle, with 32-bit indices
// (padded arrays: plane -1 and plane nz exist) and the divisions above
template <typename T>
__device__ void sm_rbgs(const LV<T>& L, const QDiv& D, T* u, const T* f, int color) {
    const int nx = L.nx, ny = L.ny, nz = L.nz, hx = nx >> 1, pl = nx * ny;
    const int np = hx * ny * nz;
    for (int t = threadIdx.x; t < np; t += blockDim.x) {
        const int r = qdiv(t, D.hx), i2 = t - r * hx;
        const int k = qdiv(r, D.ny), j = r - k * ny;
        const int i = 2 * i2 + ((j + k + color) & 1);
        const int c = i + nx * j + pl * k;
        const int xm = c + (i == 0 ? nx - 1 : -1), xp = c + (i == nx - 1 ? 1 - nx : 1);
        const int ym = c + (j == 0 ? (ny - 1) * nx : -nx), yp = c + (j == ny - 1 ? -(ny - 1) * nx : nx);
        const int zm = c + ((k == 0 && L.zper) ? (nz - 1) * pl : -pl);
        const int zp = c + ((k == nz - 1 && L.zper) ? -(nz - 1) * pl : pl);
        const T cxm = L.cx[xm], cxp = L.cx[c], cym = L.cy[ym], cyp = L.cy[c], czm = L.cz[zm], czp = L.cz[c];
        const T sm = cxp * u[xp] + cxm * u[xm] + cyp * u[yp] + cym * u[ym] + czp * u[zp] + czm * u[zm];
        const T d = cxp + cxm + cyp + cym + czp + czm;
        u[c] = (sm - f[c]) / d;
    }
}

template <typename T>
__device__ void sm_residual(const LV<T>& L, const QDiv& D, const T* u, const T* f, T* r) {
    const int nx = L.nx, ny = L.ny, nz = L.nz, pl = nx * ny;
    const int np = pl * nz;
    for (int t = threadIdx.x; t < np; t += blockDim.x) {
        const int q = qdiv(t, D.nx), i = t - q * nx;
        const int k = qdiv(q, D.ny), j = q - k * ny;
        const int c = t;
        const int xm = c + (i == 0 ? nx - 1 : -1), xp = c + (i == nx - 1 ? 1 - nx : 1);
        const int ym = c + (j == 0 ? (ny - 1) * nx : -nx), yp = c + (j == ny - 1 ? -(ny - 1) * nx : nx);
        const int zm = c + ((k == 0 && L.zper) ? (nz - 1) * pl : -pl);
        const int zp = c + ((k == nz - 1 && L.zper) ? -(nz - 1) * pl : pl);
        const T u0 = u[c];
        const T au = L.cx[c] * (u[xp] - u0) - L.cx[xm] * (u0 - u[xm]) + L.cy[c] * (u[yp] - u0) -
                     L.cy[ym] * (u0 - u[ym]) + L.cz[c] * (u[zp] - u0) - L.cz[zm] * (u0 - u[zm]);
        r[c] = f[c] - au;
    }
}

template <typename T>
__device__ void sm_restrict(const LV<T>& F, const T* r, const LV<T>& C, const QDiv& DC, T* fc) {
    const int np = C.nx * C.ny * C.nz;
    const int zoff = F.zper ? 0 : 1;
    const int pl = F.nx * F.ny;
    for (int t = threadIdx.x; t < np; t += blockDim.x) {
        const int q = qdiv(t, DC.nx), I = t - q * C.nx;
        const int K = qdiv(q, DC.ny), J = q - K * C.ny;
        const int kf = 2 * K + zoff;
        const int ic = 2 * I, im = ic == 0 ? F.nx - 1 : ic - 1, ip = ic == F.nx - 1 ? 0 : ic + 1;
        T acc = 0;
#pragma unroll
        for (int dz = -1; dz <= 1; ++dz) {
            int kk = kf + dz;
            if (F.zper) kk = kk < 0 ? kk + F.nz : (kk >= F.nz ? kk - F.nz : kk);
            const T wz = dz == 0 ? (T)0.5 : (T)0.25;
#pragma unroll
            for (int dy = -1; dy <= 1; ++dy) {
                int jj = 2 * J + dy;
                jj = jj < 0 ? jj + F.ny : (jj >= F.ny ? jj - F.ny : jj);
                const T wy = dy == 0 ? (T)0.5 : (T)0.25;
                const T* row = r + kk * pl + jj * F.nx;
                acc += wz * wy * ((T)0.25 * row[im] + (T)0.5 * row[ic] + (T)0.25 * row[ip]);
            }
        }
        fc[t] = acc;
    }
}

template <typename T>
__device__ void sm_prolong_add(const LV<T>& F, const QDiv& DF, T* u, const LV<T>& C, const T* uc) {
    const int np = F.nx * F.ny * F.nz;
    const int zoff = F.zper ? 0 : 1;
    const int cpl = C.nx * C.ny;
    for (int t = threadIdx.x; t < np; t += blockDim.x) {
        const int q = qdiv(t, DF.nx), i = t - q * F.nx;
        const int k = qdiv(q, DF.ny), j = q - k * F.ny;
        const int x0 = i >> 1, x1 = (i & 1) ? (x0 + 1 == C.nx ? 0 : x0 + 1) : x0;
        const int y0 = j >> 1, y1 = (j & 1) ? (y0 + 1 == C.ny ? 0 : y0 + 1) : y0;
        const T wx = (i & 1) ? (T)0.5 : (T)1, wy = (j & 1) ? (T)0.5 : (T)1;
        const int kk = k - zoff;
        int z0, z1;
        T wz;
        if (kk & 1) {
            z0 = (kk - 1) >> 1;                  // floor division: -1 -> -1 (the lower wall)
            z1 = z0 + 1;
            if (C.zper && z1 == C.nz) z1 = 0;
            wz = (T)0.5;
        } else { z0 = kk >> 1; z1 = z0; wz = (T)1; }
        auto at = [&](int x, int y, int z) { return uc[x + C.nx * y + cpl * z]; };
        // with a weight of 1 the second index repeats the first, weighted 0 below
        const T wx1 = (i & 1) ? wx : (T)0, wy1 = (j & 1) ? wy : (T)0, wz1 = (kk & 1) ? wz : (T)0;
        const T a0 = wy * (wx * at(x0, y0, z0) + wx1 * at(x1, y0, z0)) + wy1 * (wx * at(x0, y1, z0) + wx1 * at(x1, y1, z0));
        const T a1 = wy * (wx * at(x0, y0, z1) + wx1 * at(x1, y0, z1)) + wy1 * (wx * at(x0, y1, z1) + wx1 * at(x1, y1, z1));
        u[t] += wz * a0 + wz1 * a1;
    }
}

template <typename T>
__global__ void __launch_bounds__(1024) k_coarse_vcycle_smem(CoarseSet<T> S) {
    extern __shared__ __align__(16) unsigned char craw[];
    __shared__ double red[32];
    __shared__ LV<T> lv[16];
    griddep_wait();
    __shared__ T* su[16];
    __shared__ T* sf[16];
    __shared__ T* sr[16];
    __shared__ QDiv qd[16];
    if (threadIdx.x == 0) {
        T* q = reinterpret_cast<T*>(craw);
        for (int l = S.l0; l < S.L; ++l) {
            const LV<T>& G = S.lv[l];
            const long pl = (long)G.nx * G.ny, P = pl * (G.nz + 2);
            LV<T> v = G;
            v.cx = q + pl; q += P;
            v.cy = q + pl; q += P;
            v.cz = q + pl; q += P;
            su[l] = q + pl; q += P;
            sf[l] = q + pl; q += P;
            sr[l] = nullptr;
            if (l < S.L - 1) { sr[l] = q + pl; q += P; }
            lv[l] = v;
            qd[l].nx = qmagic(G.nx); qd[l].ny = qmagic(G.ny); qd[l].hx = qmagic(G.nx >> 1 > 0 ? G.nx >> 1 : 1);
        }
    }
    __syncthreads();
    for (int l = S.l0; l < S.L; ++l) {
        const LV<T>& G = S.lv[l];
        const long pl = (long)G.nx * G.ny, P = pl * (G.nz + 2);
        T* x = const_cast<T*>(lv[l].cx) - pl;
        T* y = const_cast<T*>(lv[l].cy) - pl;
        T* z = const_cast<T*>(lv[l].cz) - pl;
        T* uu = su[l] - pl;
        T* ff = sf[l] - pl;
        T* rr = sr[l] ? sr[l] - pl : nullptr;
        const T* gf = S.f[l] - pl;
        for (long t = threadIdx.x; t < P; t += blockDim.x) {
            x[t] = G.cx[t - pl];
            y[t] = G.cy[t - pl];
            z[t] = G.cz[t - pl];
            uu[t] = 0;
            ff[t] = l == S.l0 ? gf[t] : (T)0;
            if (rr) rr[t] = 0;
        }
    }
    __syncthreads();
    for (int l = S.l0; l < S.L - 1; ++l) {
        for (int it = 0; it < S.nu1; ++it) {
            sm_rbgs(lv[l], qd[l], su[l], sf[l], 0);
            __syncthreads();
            sm_rbgs(lv[l], qd[l], su[l], sf[l], 1);
            __syncthreads();
        }
        sm_residual(lv[l], qd[l], su[l], sf[l], sr[l]);
        __syncthreads();
        sm_restrict(lv[l], sr[l], lv[l + 1], qd[l + 1], sf[l + 1]);
        __syncthreads();
    }
    {
        // coarsest: u = inv (f - mean f) (periodic) or inv f (Dirichlet)
        const LV<T>& C = lv[S.L - 1];
        const T* f = sf[S.L - 1];
        double loc = 0.0;
        for (int p = threadIdx.x; p < S.nc; p += blockDim.x) loc += (double)f[p];
        const double tot = block_sum(loc, red);
        __shared__ double mean;
        if (threadIdx.x == 0) mean = C.zper ? tot / S.nc : 0.0;
        __syncthreads();
        const T mf = (T)mean;
        // one warp per row of the inverse: coalesced loads, a warp reduction
        const int lane = threadIdx.x & 31, nw = blockDim.x >> 5;
        for (int p = threadIdx.x >> 5; p < S.nc; p += nw) {
            const T* row = S.minv + (long)p * S.nc;
            T acc = 0;
            for (int q = lane; q < S.nc; q += 32) acc += row[q] * (f[q] - mf);
            for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
            if (lane == 0) su[S.L - 1][p] = acc;
        }
        __syncthreads();
    }
    for (int l = S.L - 2; l >= S.l0; --l) {
        sm_prolong_add(lv[l], qd[l], su[l], lv[l + 1], su[l + 1]);
        __syncthreads();
        for (int it = 0; it < S.nu2; ++it) {
            sm_rbgs(lv[l], qd[l], su[l], sf[l], 1);
            __syncthreads();
            sm_rbgs(lv[l], qd[l], su[l], sf[l], 0);
            __syncthreads();
        }
    }
    const LV<T>& G = S.lv[S.l0];
    const int np = G.nx * G.ny * G.nz;
    for (int t = threadIdx.x; t < np; t += blockDim.x) S.u[S.l0][t] = su[S.l0][t];
}

template <typename T>
size_t coarse_smem_bytes(const CoarseSet<T>& S) {
    size_t b = 0;
    for (int l = S.l0; l < S.L; ++l) {
        const LV<T>& G = S.lv[l];
        if (G.cell) return ~(size_t)0;                // the shared copy holds face coefficients only
        b += (size_t)G.nx * G.ny * (G.nz + 2) * sizeof(T) * (l < S.L - 1 ? 6 : 5);
    }
    return b;
}

}  // namespace

int gauss_jordan_launches(int n) { return n <= kGjSmemMax ? 1 : n + 2; }

void coarse_vcycle_init() {
    cudaFuncSetAttribute(k_gj_smem, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)(sizeof(double) * (2 * kGjSmemMax * kGjSmemMax + kGjSmemMax)));
    cudaFuncSetAttribute(k_gj_smem_pairs, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)(sizeof(float2) * (2 * kGjSmemMax * kGjSmemMax + kGjSmemMax)));
    cudaFuncSetAttribute(k_coarse_vcycle_smem<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kCoarseSmemBytes);
    cudaFuncSetAttribute(k_coarse_vcycle_smem<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kCoarseSmemBytes);
}

// A launch with programmatic stream serialization (see griddep_wait): the
// kernel must call griddep_wait() before its first global memory access.
template <typename... KArgs, typename... Args>
void launch_pdl(void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t s, Args... args) {
    cudaLaunchConfig_t cfg{};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    cudaLaunchKernelEx(&cfg, kernel, static_cast<KArgs>(args)...);
}

template <typename T> void launch_coarse_vcycle(const CoarseSet<T>& S, cudaStream_t s) {
    const size_t b = coarse_smem_bytes(S);
    if (b <= kCoarseSmemBytes) launch_pdl(k_coarse_vcycle_smem<T>, dim3(1), dim3(1024), b, s, S);
    else launch_pdl(k_coarse_vcycle<T>, dim3(1), dim3(1024), 0, s, S);
}
template void launch_coarse_vcycle<float>(const CoarseSet<float>&, cudaStream_t);
template void launch_coarse_vcycle<double>(const CoarseSet<double>&, cudaStream_t);

// ------------------------------------------------------------ launchers
#define GP_NV_SWITCH(X)                                                                                  \
    switch (V.n) {                                                                                       \
        case 1: X(1); break; case 2: X(2); break; case 3: X(3); break; case 4: X(4); break;              \
        case 5: X(5); break; case 6: X(6); break; case 7: X(7); break; case 8: X(8); break;              \
        case 9: X(9); break; case 10: X(10); break; case 11: X(11); break; case 12: X(12); break;        \
        case 13: X(13); break; case 14: X(14); break; case 15: X(15); break; default: X(16); break;      \
    }
template <typename T> void launch_multidot(long n, const T* w, const TVecList<T>& V, double* partial, cudaStream_t s) {
#define GP_MD(N) k_multidot<T, N><<<kReduceBlocks, kReduceThreads, 0, s>>>(n, w, V, partial)
    GP_NV_SWITCH(GP_MD)
#undef GP_MD
}
template <typename T> void launch_multiaxpy_norm(long n, T* w, const TVecList<T>& V, const double* h, double* partial,
                                                 cudaStream_t s) {
#define GP_MA(N) k_multiaxpy_norm<T, N><<<kReduceBlocks, kReduceThreads, 0, s>>>(n, w, V, h, partial)
    GP_NV_SWITCH(GP_MA)
#undef GP_MA
}
template <typename T> void launch_scale_by_norm(long n, const T* src, T* dst, const double* sq, cudaStream_t s) {
    k_scale_by_norm<T><<<grid_for(n, 256), 256, 0, s>>>(n, src, dst, sq);
}
template <typename T> void launch_combine(const Geo& g, const T* ev, const T* eb, int first, int band_nz, T* z,
                                          cudaStream_t s) {
    k_combine<T><<<row_blocks((long)g.ny * g.nz), row_threads(g.nx), 0, s>>>(g, ev, eb, first, band_nz, z);
}
template <typename T> void launch_krylov_combine(long n, T* x, const TVecList<T>& Z, const double* y, cudaStream_t s) {
    k_krylov_combine<T><<<grid_for(n, 256), 256, 0, s>>>(n, x, Z, y);
}
template <typename T> void launch_axpy1(const LV<T>& L, T* x, const T* y, cudaStream_t s) {
    const long n = (long)L.nx * L.ny * L.nz;
    k_axpy1<T><<<grid_for(n, 256), 256, 0, s>>>(n, x, y);
}
#define GP_KINST(T)                                                                                          \
    template void launch_multidot<T>(long, const T*, const TVecList<T>&, double*, cudaStream_t);             \
    template void launch_multiaxpy_norm<T>(long, T*, const TVecList<T>&, const double*, double*, cudaStream_t); \
    template void launch_scale_by_norm<T>(long, const T*, T*, const double*, cudaStream_t);                  \
    template void launch_combine<T>(const Geo&, const T*, const T*, int, int, T*, cudaStream_t);            \
    template void launch_krylov_combine<T>(long, T*, const TVecList<T>&, const double*, cudaStream_t);       \
    template void launch_axpy1<T>(const LV<T>&, T*, const T*, cudaStream_t);
GP_KINST(float)
GP_KINST(double)
void launch_finalize(const double* partial, int nparts, int ncomp, double* out, cudaStream_t s) {
    launch_pdl(k_finalize, dim3(1), dim3(1024), 0, s, partial, nparts, ncomp, out);
}
void launch_rho_stats(long n, const double* rho, double* partial, cudaStream_t s) {
    k_rho_stats<<<kReduceBlocks, kReduceThreads, 0, s>>>(n, rho, partial);
}
void launch_sub_mean(long n, double* x, const double* sum_slot, double scale, cudaStream_t s) {
    k_sub_mean<<<grid_for(n, 256), 256, 0, s>>>(n, x, sum_slot, scale);
}
template <typename T>
void launch_residual64(const Geo& g, const double* phi, const double* rho, const double* eps64, T* r_out,
                       double* partial, cudaStream_t s) {
    k_residual64<T><<<kReduceBlocks, kReduceThreads, 0, s>>>(g, phi, rho, eps64, r_out, partial);
}
void launch_to_df(long n, const double* src, double scale, float2* dst, cudaStream_t s, int* nonzero,
                  float* hi_out) {
    k_to_df<<<grid_for(n, 256), 256, 0, s>>>(n, src, scale, dst, nonzero, hi_out);
}
void launch_update_phid(long n, float2* phid, const float* e, cudaStream_t s) {
    k_update_phid<<<grid_for(n / 2, 256), 256, 0, s>>>(n / 2, reinterpret_cast<float4*>(phid),
                                                       reinterpret_cast<const float2*>(e));
}
void launch_from_df_gauge(long n, const float2* src, const double* sum_slot, double scale, double* dst,
                          cudaStream_t s) {
    k_from_df_gauge<<<grid_for(n, 256), 256, 0, s>>>(n, src, sum_slot, scale, dst);
}

void launch_residual_df(const Geo& g, const float2* phid, const float2* bd, const float2* epsd, float* r_out,
                        double* partial, cudaStream_t s) {
    auto split = [](double v) { const float h = (float)v; return d2{h, (float)(v - (double)h)}; };
    const bool vec = g.nx % 4 == 0 && ((reinterpret_cast<uintptr_t>(phid) | reinterpret_cast<uintptr_t>(bd) |
                                        reinterpret_cast<uintptr_t>(epsd) | reinterpret_cast<uintptr_t>(r_out)) & 15) == 0;
    if (vec)
        k_residual_df4<<<kReduceBlocks, kReduceThreads, 0, s>>>(g, phid, bd, epsd, split(g.c2x), split(g.c2y),
                                                                split(g.c2z), r_out, partial);
    else
        k_residual_df<<<kReduceBlocks, kReduceThreads, 0, s>>>(g, phid, bd, epsd, split(g.c2x), split(g.c2y),
                                                               split(g.c2z), r_out, partial);
}

template <typename T>
void launch_update_phi(const Geo& g, double* phi, const T* e_full, const T* e_band, int band_first, int band_nz,
                       cudaStream_t s) {
    const long n = (long)g.nx * g.ny * g.nz;
    k_update_phi<T><<<grid_for(n, 256), 256, 0, s>>>(g, phi, e_full, e_band, band_first, band_nz);
}

template <typename T> void launch_rbgs(const LV<T>& L, T* u, const T* f, int color, cudaStream_t s, bool init) {
    if constexpr (sizeof(T) == 4) {
        if (!L.cell) {
            const long pairs = (long)(L.nx / 2) * L.ny * L.nz;
            launch_pdl(k_rbgs_pairs, dim3(grid_for(pairs, 256)), dim3(256), 0, s, L, u, f, color, (int)init);
            return;
        }
    }
    const long rows = (long)L.ny * L.nz;
    launch_pdl(k_rbgs<T>, dim3(row_blocks(rows)), dim3(row_threads(L.nx / 2)), 0, s, L, u, f, color, (int)init);
}
template <typename T> void launch_residual(const LV<T>& L, const T* u, const T* f, T* r, cudaStream_t s) {
    if constexpr (sizeof(T) == 4) {
        dim3 grid; int sz, th; size_t sm;
        if (apply_zm_grid(L, grid, sz, sm, th)) {
            launch_pdl(k_apply_zm<false>, grid, dim3(th), sm, s, L, u, f, r, (double*)nullptr, sz);
            return;
        }
        if (L.cell && L.nx % 4 == 0) {
            k_apply4<false><<<kReduceBlocks * 2, kReduceThreads, 0, s>>>(L, u, f, r, nullptr);
            return;
        }
    }
    const long rows = (long)L.ny * L.nz;
    launch_pdl(k_residual<T>, dim3(row_blocks(rows)), dim3(row_threads(L.nx)), 0, s, L, u, f, r);
}
template <typename T> void launch_restrict(const LV<T>& F, const T* r, const LV<T>& C, T* fc, cudaStream_t s) {
    if constexpr (sizeof(T) == 4) {
        if (F.nx % 4 == 0 && C.nx * 2 == F.nx && C.nx % 2 == 0 &&
            ((reinterpret_cast<uintptr_t>(r) & 15) | (reinterpret_cast<uintptr_t>(fc) & 7)) == 0) {
            const long pairs = (long)C.nx * C.ny * C.nz / 2;
            launch_pdl(k_restrict4, dim3(grid_for(pairs, 256)), dim3(256), 0, s, F, r, C, fc);
            return;
        }
    }
    const long rows = (long)C.ny * C.nz;
    launch_pdl(k_restrict<T>, dim3(row_blocks(rows)), dim3(row_threads(C.nx)), 0, s, F, r, C, fc);
}
template <typename T> void launch_prolong_add(const LV<T>& F, T* u, const LV<T>& C, const T* uc, cudaStream_t s) {
    if constexpr (sizeof(T) == 4) {
        if (F.nx % 4 == 0 && C.nx * 2 == F.nx && (reinterpret_cast<uintptr_t>(u) & 15) == 0) {
            const long quads = (long)F.nx * F.ny * F.nz / 4;
            launch_pdl(k_prolong_add4, dim3(grid_for(quads, 256)), dim3(256), 0, s, F, u, C, uc);
            return;
        }
    }
    const long rows = (long)F.ny * F.nz;
    launch_pdl(k_prolong_add<T>, dim3(row_blocks(rows)), dim3(row_threads(F.nx)), 0, s, F, u, C, uc);
}
template <typename T> void launch_coarsen_faces(const LV<T>& F, int nxc, int nyc, int nzc, T* cx, T* cy, T* cz,
                                                cudaStream_t s) {
    if (F.cell && F.zper) {
        k_coarsen_faces_cell<T><<<grid_for((long)nxc * nyc * nzc, 256), 256, 0, s>>>(F, nxc, nyc, nzc, cx, cy, cz);
        return;
    }
    const long n = (long)nxc * nyc * (nzc + 1);
    k_coarsen_faces<T><<<grid_for(n, 256), 256, 0, s>>>(F, nxc, nyc, nzc, cx, cy, cz);
}
template <typename T> void launch_coarse_matrix(const LV<T>& C, double* M, cudaStream_t s) {
    k_coarse_matrix<T><<<1, 512, 0, s>>>(C, M);
}
int launch_gauss_jordan(double* M, int n, int* status, cudaStream_t s, bool pairs) {
    if (n <= kGjSmemMax) {
        if (pairs) k_gj_smem_pairs<<<1, 1024, sizeof(float2) * (2 * (size_t)n * n + n), s>>>(M, n, status);
        else k_gj_smem<<<1, 1024, sizeof(double) * (2 * (size_t)n * n + n), s>>>(M, n, status);
        return 1;
    }
    const int th = n >= 256 ? 256 : 128;
    k_gj_init<<<n, th, 0, s>>>(M, n, status);
    for (int col = 0; col < n; ++col) k_gj_step<<<n, th, 0, s>>>(M, n, col, status);
    k_gj_finish<<<n, th, 0, s>>>(M, n);
    return n + 2;
}
template <typename T> void launch_store_inverse(const double* W, int n, T* inv, cudaStream_t s) {
    const long nn = (long)n * n;
    k_store_inverse<T><<<grid_for(nn, 256), 256, 0, s>>>(W, nn, inv);
}
template <typename T> void launch_coarse_solve(const LV<T>& C, const T* inv, int n, const T* f, T* u,
                                               cudaStream_t s) {
    k_coarse_solve<T><<<1, 512, 0, s>>>(C, inv, n, f, u);
}
template <typename T> void launch_applyA_dot(const LV<T>& L, const T* p, T* q, double* partial, cudaStream_t s) {
    if constexpr (sizeof(T) == 4) {
        dim3 grid; int sz, th; size_t sm;
        if (apply_zm_grid(L, grid, sz, sm, th)) {
            launch_pdl(k_apply_zm<true>, grid, dim3(th), sm, s, L, p, (const float*)nullptr, q, partial, sz);
            return;
        }
        if (L.cell && L.nx % 4 == 0) {
            k_apply4<true><<<kReduceBlocks, kReduceThreads, 0, s>>>(L, p, nullptr, q, partial);
            return;
        }
    }
    k_applyA_dot<T><<<kReduceBlocks, row_threads(L.nx), 0, s>>>(L, p, q, partial);
}
// 16-byte vector path: FP32, a multiple of 4 elements, every pointer 16-byte aligned
inline bool vec4_ok(long n, int elem, std::initializer_list<const void*> ptrs) {
    if (elem != 4 || n % 4) return false;
    for (const void* q : ptrs)
        if (reinterpret_cast<uintptr_t>(q) & 15) return false;
    return true;
}

template <typename T> void launch_dot(const LV<T>& L, const T* a, const T* b, double* partial, cudaStream_t s) {
    const long n = (long)L.nx * L.ny * L.nz;
    if (vec4_ok(n, sizeof(T), {a, b})) {
        launch_pdl(k_dot4, dim3(kReduceBlocks), dim3(kReduceThreads), 0, s, n / 4, reinterpret_cast<const float4*>(a),
                   reinterpret_cast<const float4*>(b), partial);
        return;
    }
    k_dot<T><<<kReduceBlocks, kReduceThreads, 0, s>>>(n, a, b, partial);
}
template <typename T> void launch_update_xr(const LV<T>& L, T* x, T* r, const T* p, const T* q, const double* scal,
                                            int num, int den, cudaStream_t s) {
    const long n = (long)L.nx * L.ny * L.nz;
    if (vec4_ok(n, sizeof(T), {x, r, p, q})) {
        launch_pdl(k_update_xr4, dim3(grid_for(n / 4, 256)), dim3(256), 0, s, n / 4, reinterpret_cast<float4*>(x),
                   reinterpret_cast<float4*>(r), reinterpret_cast<const float4*>(p), reinterpret_cast<const float4*>(q),
                   scal, num, den);
        return;
    }
    k_update_xr<T><<<grid_for(n, 256), 256, 0, s>>>(n, x, r, p, q, scal, num, den);
}
template <typename T> void launch_update_p(const LV<T>& L, T* p, const T* z, const double* scal, int num, int den,
                                           cudaStream_t s) {
    const long n = (long)L.nx * L.ny * L.nz;
    if (vec4_ok(n, sizeof(T), {p, z})) {
        launch_pdl(k_update_p4, dim3(grid_for(n / 4, 256)), dim3(256), 0, s, n / 4, reinterpret_cast<float4*>(p),
                   reinterpret_cast<const float4*>(z), scal, num, den);
        return;
    }
    k_update_p<T><<<grid_for(n, 256), 256, 0, s>>>(n, p, z, scal, num, den);
}
template <typename T> void launch_copy_level(const LV<T>& L, T* dst, const T* src, cudaStream_t s) {
    const long n = (long)L.nx * L.ny * L.nz;
    if (vec4_ok(n, sizeof(T), {dst, src})) {
        launch_pdl(k_copy4, dim3(grid_for(n / 4, 256)), dim3(256), 0, s, n / 4, reinterpret_cast<float4*>(dst),
                   reinterpret_cast<const float4*>(src));
        return;
    }
    k_copy<T><<<grid_for(n, 256), 256, 0, s>>>(n, dst, src);
}
template <typename T> void launch_cast_eps(long n, const double* e64, T* eT, cudaStream_t s) {
    k_cast<T><<<grid_for(n, 256), 256, 0, s>>>(n, e64, eT);
}
template <typename T> void launch_band_eps(const Geo& g, const T* epsT, int first, int band_nz, T* beps,
                                           cudaStream_t s) {
    const long n = plane_of(g.nx, g.ny) * (band_nz + 2);
    k_band_eps<T><<<grid_for(n, 256), 256, 0, s>>>(g, epsT, first, band_nz, beps);
}
template <typename T> void launch_band_rhs(const Geo& g, const T* epsT, const T* r, const T* ev, int first,
                                           int band_nz, T* fb, cudaStream_t s) {
    const long rows = (long)g.ny * band_nz;
    k_band_rhs<T><<<row_blocks(rows), row_threads(g.nx), 0, s>>>(g, epsT, r, ev, first, band_nz, fb);
}

#define GP_INST(T)                                                                                           \
    template void launch_residual64<T>(const Geo&, const double*, const double*, const double*, T*, double*, \
                                       cudaStream_t);                                                        \
    template void launch_update_phi<T>(const Geo&, double*, const T*, const T*, int, int, cudaStream_t);     \
    template void launch_rbgs<T>(const LV<T>&, T*, const T*, int, cudaStream_t, bool);                             \
    template void launch_residual<T>(const LV<T>&, const T*, const T*, T*, cudaStream_t);                    \
    template void launch_restrict<T>(const LV<T>&, const T*, const LV<T>&, T*, cudaStream_t);                \
    template void launch_prolong_add<T>(const LV<T>&, T*, const LV<T>&, const T*, cudaStream_t);             \
    template void launch_coarsen_faces<T>(const LV<T>&, int, int, int, T*, T*, T*, cudaStream_t);            \
    template void launch_coarse_matrix<T>(const LV<T>&, double*, cudaStream_t);                              \
    template void launch_store_inverse<T>(const double*, int, T*, cudaStream_t);                             \
    template void launch_coarse_solve<T>(const LV<T>&, const T*, int, const T*, T*, cudaStream_t);           \
    template void launch_applyA_dot<T>(const LV<T>&, const T*, T*, double*, cudaStream_t);                   \
    template void launch_dot<T>(const LV<T>&, const T*, const T*, double*, cudaStream_t);                    \
    template void launch_update_xr<T>(const LV<T>&, T*, T*, const T*, const T*, const double*, int, int,     \
                                      cudaStream_t);                                                         \
    template void launch_update_p<T>(const LV<T>&, T*, const T*, const double*, int, int, cudaStream_t);     \
    template void launch_copy_level<T>(const LV<T>&, T*, const T*, cudaStream_t);                            \
    template void launch_cast_eps<T>(long, const double*, T*, cudaStream_t);                                 \
    template void launch_band_eps<T>(const Geo&, const T*, int, int, T*, cudaStream_t);                      \
    template void launch_band_rhs<T>(const Geo&, const T*, const T*, const T*, int, int, T*, cudaStream_t);

GP_INST(float)
GP_INST(double)

}  // namespace gp
