// Hand-written 3D FFT Poisson solve for the dry region (Eq. 15), with the
// symbol of the 7-point operator instead of -G^2 so that the result solves
// the discrete equation exactly:
//     out^(k) = src^(k) / lambda(k),  lambda(k) = sum_a -4 sin^2(pi k_a/N_a)/h_a^2,
// and the k = 0 mode set to zero (mean-zero potential).
//
// Five passes over a half-spectrum buffer of (nx/2+1) x ny x nz complex values:
//   x: real rows -> complex half spectrum (forward)
//   y: forward along y
//   z: forward along z, divide by lambda * N, inverse along z (one pass)
//   y: inverse along y
//   x: half spectrum -> real rows (inverse, Hermitian extension)
// Each pass loads M lines into shared memory and runs a Stockham autosort FFT
// (radix 4, 2, 3; every extent is 2^a 3^b) on them.
#include "gp_common.cuh"

#include <algorithm>
#include <vector>

namespace gp {

template <typename T> struct Cx { T re, im; };

template <typename T>
__device__ __forceinline__ Cx<T> cmul(Cx<T> a, Cx<T> b) {
    return {a.re * b.re - a.im * b.im, a.re * b.im + a.im * b.re};
}
template <typename T> __device__ __forceinline__ Cx<T> cadd(Cx<T> a, Cx<T> b) { return {a.re + b.re, a.im + b.im}; }
template <typename T> __device__ __forceinline__ Cx<T> csub(Cx<T> a, Cx<T> b) { return {a.re - b.re, a.im - b.im}; }

struct AxisPlan {
    int n;
    int nstages;
    int radix[16];
};

struct FFTPlan {
    Geo g;
    AxisPlan ax[3];
    double* tw64[3];      // W_N^t = exp(-2 pi i t / N), t < N, as (re, im)
    float* tw32[3];
    double* lam[3];       // 1D symbol per axis
    float* lam32[3];      // the same in FP32
};

namespace {

AxisPlan make_axis(int n) {
    AxisPlan p;
    p.n = n;
    p.nstages = 0;
    int m = n;
    while (m % 4 == 0) { p.radix[p.nstages++] = 4; m /= 4; }
    while (m % 2 == 0) { p.radix[p.nstages++] = 2; m /= 2; }
    while (m % 3 == 0) { p.radix[p.nstages++] = 3; m /= 3; }
    if (m != 1) p.nstages = -1;
    return p;
}

__global__ void k_twiddles(int n, double* tw64, float* tw32) {
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < n; t += gridDim.x * blockDim.x) {
        double s, c;
        sincospi(-2.0 * t / n, &s, &c);
        tw64[2 * t] = c; tw64[2 * t + 1] = s;
        tw32[2 * t] = (float)c; tw32[2 * t + 1] = (float)s;
    }
}

__global__ void k_symbol(int n, double h, double* lam, float* lam32) {
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < n; t += gridDim.x * blockDim.x) {
        const double s = sinpi((double)t / n);
        lam[t] = -4.0 * s * s / (h * h);
        lam32[t] = (float)lam[t];
    }
}

// Stockham FFT of M interleaved lines of length N in shared memory:
// element e of line l at buf[e * M + l]. Returns the buffer holding the result.
template <typename T, bool INV>
__device__ Cx<T>* smem_fft(Cx<T>* A, Cx<T>* B, int N, int M, const AxisPlan& ap, const Cx<T>* tw) {
    int Ns = 1;
    for (int st = 0; st < ap.nstages; ++st) {
        const int R = ap.radix[st];
        const int NR = N / R;
        const int tstep = N / (Ns * R);
        for (int b = threadIdx.x; b < M * NR; b += blockDim.x) {
            const int l = b % M, j = b / M;
            const int kk = j % Ns;
            Cx<T> v[4];
            for (int r = 0; r < R; ++r) {
                Cx<T> x = A[(j + r * NR) * M + l];
                if (r > 0 && kk > 0) {
                    Cx<T> w = tw[r * kk * tstep];
                    if (INV) w.im = -w.im;
                    x = cmul(x, w);
                }
                v[r] = x;
            }
            Cx<T> o[4];
            if (R == 2) {
                o[0] = cadd(v[0], v[1]);
                o[1] = csub(v[0], v[1]);
            } else if (R == 4) {
                const Cx<T> a = cadd(v[0], v[2]), bb = csub(v[0], v[2]);
                const Cx<T> c = cadd(v[1], v[3]), d = csub(v[1], v[3]);
                const Cx<T> mid = INV ? Cx<T>{-d.im, d.re} : Cx<T>{d.im, -d.re};   // (+/- i) d
                o[0] = cadd(a, c);
                o[2] = csub(a, c);
                o[1] = cadd(bb, mid);
                o[3] = csub(bb, mid);
            } else {   // R == 3
                const T c3 = (T)-0.5;
                const T s3 = INV ? (T)0.86602540378443864676 : (T)-0.86602540378443864676;
                const Cx<T> t = cadd(v[1], v[2]), d = csub(v[1], v[2]);
                const Cx<T> m = {v[0].re + c3 * t.re, v[0].im + c3 * t.im};
                const Cx<T> rot = {-s3 * d.im, s3 * d.re};                           // i s3 d
                o[0] = cadd(v[0], t);
                o[1] = cadd(m, rot);
                o[2] = csub(m, rot);
            }
            const int base = (j / Ns) * Ns * R + kk;
            for (int r = 0; r < R; ++r) B[(base + r * Ns) * M + l] = o[r];
        }
        __syncthreads();
        Cx<T>* t = A; A = B; B = t;
        Ns *= R;
    }
    return A;
}

template <typename T>
__device__ void load_tw(Cx<T>* s, const T* tw, int n) {
    for (int t = threadIdx.x; t < n; t += blockDim.x) s[t] = Cx<T>{tw[2 * t], tw[2 * t + 1]};
}

// x pass, forward: rows (j,k) of real input -> half spectrum
template <typename T>
__global__ void k_fft_x_fwd(Geo g, AxisPlan ap, const T* tw, int M, const T* src, Cx<T>* C) {
    extern __shared__ unsigned char smem_raw[];
    Cx<T>* sw = reinterpret_cast<Cx<T>*>(smem_raw);
    const int N = g.nx, nxh = g.nx / 2 + 1;
    Cx<T>* A = sw + N;
    Cx<T>* B = A + N * M;
    load_tw(sw, tw, N);
    const long rows = (long)g.ny * g.nz;
    const long row0 = (long)blockIdx.x * M;
    for (int q = threadIdx.x; q < M * N; q += blockDim.x) {
        const int l = q / N, e = q % N;
        const long row = row0 + l;
        A[e * M + l] = Cx<T>{row < rows ? src[row * N + e] : (T)0, (T)0};
    }
    __syncthreads();
    Cx<T>* R = smem_fft<T, false>(A, B, N, M, ap, sw);
    for (int q = threadIdx.x; q < M * nxh; q += blockDim.x) {
        const int l = q / nxh, e = q % nxh;
        const long row = row0 + l;
        if (row < rows) C[row * nxh + e] = R[e * M + l];
    }
}

// x pass, inverse: half spectrum rows -> real output (real part of the full line)
template <typename T>
__global__ void k_fft_x_inv(Geo g, AxisPlan ap, const T* tw, int M, const Cx<T>* C, T* out) {
    extern __shared__ unsigned char smem_raw[];
    Cx<T>* sw = reinterpret_cast<Cx<T>*>(smem_raw);
    const int N = g.nx, nxh = g.nx / 2 + 1;
    Cx<T>* A = sw + N;
    Cx<T>* B = A + N * M;
    load_tw(sw, tw, N);
    const long rows = (long)g.ny * g.nz;
    const long row0 = (long)blockIdx.x * M;
    for (int q = threadIdx.x; q < M * N; q += blockDim.x) {
        const int l = q / N, e = q % N;
        const long row = row0 + l;
        Cx<T> v = {(T)0, (T)0};
        if (row < rows) {
            if (e < nxh) v = C[row * nxh + e];
            else { v = C[row * nxh + (N - e)]; v.im = -v.im; }
        }
        A[e * M + l] = v;
    }
    __syncthreads();
    Cx<T>* R = smem_fft<T, true>(A, B, N, M, ap, sw);
    for (int q = threadIdx.x; q < M * N; q += blockDim.x) {
        const int l = q / N, e = q % N;
        const long row = row0 + l;
        if (row < rows) out[row * N + e] = R[e * M + l].re;
    }
}

// y pass: lines along y for M consecutive kx at fixed k
template <typename T, bool INV>
__global__ void k_fft_y(Geo g, AxisPlan ap, const T* tw, int M, Cx<T>* C) {
    extern __shared__ unsigned char smem_raw[];
    Cx<T>* sw = reinterpret_cast<Cx<T>*>(smem_raw);
    const int N = g.ny, nxh = g.nx / 2 + 1;
    Cx<T>* A = sw + N;
    Cx<T>* B = A + N * M;
    load_tw(sw, tw, N);
    const int nchunks = (nxh + M - 1) / M;
    const int kx0 = (blockIdx.x % nchunks) * M;
    const long k = blockIdx.x / nchunks;
    Cx<T>* base = C + k * (long)nxh * N;
    for (int q = threadIdx.x; q < M * N; q += blockDim.x) {
        const int e = q / M, l = q % M;
        A[e * M + l] = (kx0 + l < nxh) ? base[(long)e * nxh + kx0 + l] : Cx<T>{(T)0, (T)0};
    }
    __syncthreads();
    Cx<T>* R = smem_fft<T, INV>(A, B, N, M, ap, sw);
    for (int q = threadIdx.x; q < M * N; q += blockDim.x) {
        const int e = q / M, l = q % M;
        if (kx0 + l < nxh) base[(long)e * nxh + kx0 + l] = R[e * M + l];
    }
}

// z pass: forward, divide by lambda * Ntot, inverse; lines along z for M kx at fixed ky
template <typename T>
__global__ void k_fft_z_solve(Geo g, AxisPlan ap, const T* tw, int M, const double* lx, const double* ly,
                              const double* lz, Cx<T>* C) {
    extern __shared__ unsigned char smem_raw[];
    Cx<T>* sw = reinterpret_cast<Cx<T>*>(smem_raw);
    const int N = g.nz, nxh = g.nx / 2 + 1;
    Cx<T>* A = sw + N;
    Cx<T>* B = A + N * M;
    load_tw(sw, tw, N);
    const int nchunks = (nxh + M - 1) / M;
    const int kx0 = (blockIdx.x % nchunks) * M;
    const int ky = blockIdx.x / nchunks;
    const long zs = (long)nxh * g.ny;
    Cx<T>* base = C + (long)ky * nxh;
    for (int q = threadIdx.x; q < M * N; q += blockDim.x) {
        const int e = q / M, l = q % M;
        A[e * M + l] = (kx0 + l < nxh) ? base[e * zs + kx0 + l] : Cx<T>{(T)0, (T)0};
    }
    __syncthreads();
    Cx<T>* R = smem_fft<T, false>(A, B, N, M, ap, sw);
    Cx<T>* O = (R == A) ? B : A;
    const double inv_n = g.inv_n;
    for (int q = threadIdx.x; q < M * N; q += blockDim.x) {
        const int e = q / M, l = q % M;
        const int kx = kx0 + l;
        Cx<T> v = R[e * M + l];
        if (kx < nxh) {
            const double lam = lx[kx] + ly[ky] + lz[e];
            const T f = (kx == 0 && ky == 0 && e == 0) ? (T)0 : (T)(inv_n / lam);
            v.re *= f; v.im *= f;
        } else {
            v = Cx<T>{(T)0, (T)0};
        }
        R[e * M + l] = v;
    }
    __syncthreads();
    Cx<T>* R2 = smem_fft<T, true>(R, O, N, M, ap, sw);
    for (int q = threadIdx.x; q < M * N; q += blockDim.x) {
        const int e = q / M, l = q % M;
        if (kx0 + l < nxh) base[e * zs + kx0 + l] = R2[e * M + l];
    }
}

int lines_per_cta(int n, size_t csize) {
    // two ping-pong buffers of N*M complex values within ~96 KB
    int m = 16;
    while (m > 1 && 2 * (size_t)n * m * csize > 96 * 1024) m >>= 1;
    return m;
}

size_t smem_bytes(int n, int m, size_t csize) { return (size_t)n * csize * (1 + 2 * (size_t)m); }

// ---------------------------------------------------------------------------
// Compile-time sizes: with N, M and the radix sequence known to the compiler,
// every index division in the Stockham stages becomes a shift or a multiply.
__host__ __device__ constexpr int st_count(int n) {
    int s = 0;
    while (n % 4 == 0) { n /= 4; ++s; }
    while (n % 2 == 0) { n /= 2; ++s; }
    while (n % 3 == 0) { n /= 3; ++s; }
    return s;
}
__host__ __device__ constexpr int st_radix(int n, int st) {
    int s = 0;
    while (n % 4 == 0) { if (s == st) return 4; n /= 4; ++s; }
    while (n % 2 == 0) { if (s == st) return 2; n /= 2; ++s; }
    while (n % 3 == 0) { if (s == st) return 3; n /= 3; ++s; }
    return 1;
}
__host__ __device__ constexpr int st_before(int n, int st) {
    int p = 1;
    for (int i = 0; i < st; ++i) p *= st_radix(n, i);
    return p;
}

template <typename T, int N, int M, bool INV, int ST>
__device__ __forceinline__ Cx<T>* sstage(Cx<T>* A, Cx<T>* B, const Cx<T>* tw) {
    if constexpr (ST >= st_count(N)) {
        return A;
    } else {
        constexpr int R = st_radix(N, ST), Ns = st_before(N, ST), NR = N / R, tstep = N / (Ns * R);
        for (int b = threadIdx.x; b < M * NR; b += blockDim.x) {
            const int l = b % M, j = b / M;
            const int kk = j % Ns;
            Cx<T> v[R];
#pragma unroll
            for (int r = 0; r < R; ++r) {
                Cx<T> x = A[(j + r * NR) * (M + 1) + l];
                if (r > 0 && kk > 0) {
                    Cx<T> w = tw[r * kk * tstep];
                    if (INV) w.im = -w.im;
                    x = cmul(x, w);
                }
                v[r] = x;
            }
            Cx<T> o[R];
            if constexpr (R == 2) {
                o[0] = cadd(v[0], v[1]);
                o[1] = csub(v[0], v[1]);
            } else if constexpr (R == 4) {
                const Cx<T> a = cadd(v[0], v[2]), bb = csub(v[0], v[2]);
                const Cx<T> c = cadd(v[1], v[3]), d = csub(v[1], v[3]);
                const Cx<T> mid = INV ? Cx<T>{-d.im, d.re} : Cx<T>{d.im, -d.re};
                o[0] = cadd(a, c);
                o[2] = csub(a, c);
                o[1] = cadd(bb, mid);
                o[3] = csub(bb, mid);
            } else {
                const T c3 = (T)-0.5;
                const T s3 = INV ? (T)0.86602540378443864676 : (T)-0.86602540378443864676;
                const Cx<T> t = cadd(v[1], v[2]), d = csub(v[1], v[2]);
                const Cx<T> m = {v[0].re + c3 * t.re, v[0].im + c3 * t.im};
                const Cx<T> rot = {-s3 * d.im, s3 * d.re};
                o[0] = cadd(v[0], t);
                o[1] = cadd(m, rot);
                o[2] = csub(m, rot);
            }
            const int base = (j / Ns) * Ns * R + kk;
#pragma unroll
            for (int r = 0; r < R; ++r) B[(base + r * Ns) * (M + 1) + l] = o[r];
        }
        __syncthreads();
        return sstage<T, N, M, INV, ST + 1>(B, A, tw);
    }
}

template <typename T, int N>
constexpr int lines_static() {
    int m = 16;
    while (m > 1 && 2 * N * (m + 1) * (int)sizeof(Cx<T>) > 100 * 1024) m >>= 1;
    return m;
}

template <typename T, int N, int M>
__global__ void __launch_bounds__(256) ks_x_fwd(Geo g, const T* tw, const T* src, Cx<T>* C) {
    extern __shared__ unsigned char smem_raw[];
    Cx<T>* sw = reinterpret_cast<Cx<T>*>(smem_raw);
    constexpr int nxh = N / 2 + 1;
    Cx<T>* A = sw + N;
    Cx<T>* B = A + N * (M + 1);
    load_tw(sw, tw, N);
    const long rows = (long)g.ny * g.nz;
    const long row0 = (long)blockIdx.x * M;
    for (int q = threadIdx.x; q < M * N; q += blockDim.x) {
        const int l = q / N, e = q % N;
        const long row = row0 + l;
        A[e * (M + 1) + l] = Cx<T>{row < rows ? src[row * N + e] : (T)0, (T)0};
    }
    __syncthreads();
    Cx<T>* R = sstage<T, N, M, false, 0>(A, B, sw);
    for (int q = threadIdx.x; q < M * nxh; q += blockDim.x) {
        const int l = q / nxh, e = q % nxh;
        const long row = row0 + l;
        if (row < rows) C[row * nxh + e] = R[e * (M + 1) + l];
    }
}

template <typename T, int N, int M>
__global__ void __launch_bounds__(256) ks_x_inv(Geo g, const T* tw, const Cx<T>* C, T* out) {
    extern __shared__ unsigned char smem_raw[];
    Cx<T>* sw = reinterpret_cast<Cx<T>*>(smem_raw);
    constexpr int nxh = N / 2 + 1;
    Cx<T>* A = sw + N;
    Cx<T>* B = A + N * (M + 1);
    load_tw(sw, tw, N);
    const long rows = (long)g.ny * g.nz;
    const long row0 = (long)blockIdx.x * M;
    for (int q = threadIdx.x; q < M * N; q += blockDim.x) {
        const int l = q / N, e = q % N;
        const long row = row0 + l;
        Cx<T> v = {(T)0, (T)0};
        if (row < rows) {
            if (e < nxh) v = C[row * nxh + e];
            else { v = C[row * nxh + (N - e)]; v.im = -v.im; }
        }
        A[e * (M + 1) + l] = v;
    }
    __syncthreads();
    Cx<T>* R = sstage<T, N, M, true, 0>(A, B, sw);
    for (int q = threadIdx.x; q < M * N; q += blockDim.x) {
        const int l = q / N, e = q % N;
        const long row = row0 + l;
        if (row < rows) out[row * N + e] = R[e * (M + 1) + l].re;
    }
}

template <typename T, int N, int M, bool INV>
__global__ void __launch_bounds__(256) ks_y(Geo g, const T* tw, Cx<T>* C) {
    extern __shared__ unsigned char smem_raw[];
    Cx<T>* sw = reinterpret_cast<Cx<T>*>(smem_raw);
    const int nxh = g.nx / 2 + 1;
    Cx<T>* A = sw + N;
    Cx<T>* B = A + N * (M + 1);
    load_tw(sw, tw, N);
    const int nchunks = (nxh + M - 1) / M;
    const int kx0 = (blockIdx.x % nchunks) * M;
    const long k = blockIdx.x / nchunks;
    Cx<T>* base = C + k * (long)nxh * N;
    for (int q = threadIdx.x; q < M * N; q += blockDim.x) {
        const int e = q / M, l = q % M;
        A[e * (M + 1) + l] = (kx0 + l < nxh) ? base[(long)e * nxh + kx0 + l] : Cx<T>{(T)0, (T)0};
    }
    __syncthreads();
    Cx<T>* R = sstage<T, N, M, INV, 0>(A, B, sw);
    for (int q = threadIdx.x; q < M * N; q += blockDim.x) {
        const int e = q / M, l = q % M;
        if (kx0 + l < nxh) base[(long)e * nxh + kx0 + l] = R[e * (M + 1) + l];
    }
}

template <typename T, int N, int M>
__global__ void __launch_bounds__(256) ks_z_solve(Geo g, const T* tw, const T* lx, const T* ly, const T* lz,
                                                  Cx<T>* C) {
    extern __shared__ unsigned char smem_raw[];
    Cx<T>* sw = reinterpret_cast<Cx<T>*>(smem_raw);
    const int nxh = g.nx / 2 + 1;
    Cx<T>* A = sw + N;
    Cx<T>* B = A + N * (M + 1);
    load_tw(sw, tw, N);
    const int nchunks = (nxh + M - 1) / M;
    const int kx0 = (blockIdx.x % nchunks) * M;
    const int ky = blockIdx.x / nchunks;
    const long zs = (long)nxh * g.ny;
    Cx<T>* base = C + (long)ky * nxh;
    for (int q = threadIdx.x; q < M * N; q += blockDim.x) {
        const int e = q / M, l = q % M;
        A[e * (M + 1) + l] = (kx0 + l < nxh) ? base[e * zs + kx0 + l] : Cx<T>{(T)0, (T)0};
    }
    __syncthreads();
    Cx<T>* R = sstage<T, N, M, false, 0>(A, B, sw);
    Cx<T>* O = (R == A) ? B : A;
    // symbol in the working precision: 1/(lambda N) (no FP64 per element for FP32)
    const T inv_n = (T)g.inv_n;
    const T lyv = ly[ky];
    for (int q = threadIdx.x; q < M * N; q += blockDim.x) {
        const int e = q / M, l = q % M;
        const int kx = kx0 + l;
        Cx<T> v = R[e * (M + 1) + l];
        if (kx < nxh) {
            const T lam = (lx[kx] + lyv + lz[e]) / inv_n;
            const T f = (kx == 0 && ky == 0 && e == 0) ? (T)0 : (T)1 / lam;
            v.re *= f; v.im *= f;
        } else {
            v = Cx<T>{(T)0, (T)0};
        }
        R[e * (M + 1) + l] = v;
    }
    __syncthreads();
    Cx<T>* R2 = sstage<T, N, M, true, 0>(R, O, sw);
    for (int q = threadIdx.x; q < M * N; q += blockDim.x) {
        const int e = q / M, l = q % M;
        if (kx0 + l < nxh) base[e * zs + kx0 + l] = R2[e * (M + 1) + l];
    }
}

template <typename T, int N>
constexpr size_t smem_static() { return (size_t)N * sizeof(Cx<T>) * (1 + 2 * ((size_t)lines_static<T, N>() + 1)); }

// one pass of axis `axis` (0 x-forward, 1 y-forward, 2 z-solve, 3 y-inverse, 4 x-inverse) with N
// known at compile time; returns false if N has no static instance
template <typename T, int N>
void static_pass(int pass, FFTPlan* p, const T* tw, const T* src, T* out, Cx<T>* C, cudaStream_t s, bool attr) {
    constexpr int M = lines_static<T, N>();
    constexpr size_t sm = smem_static<T, N>();
    if (attr) {
        switch (pass) {
            case 0: cudaFuncSetAttribute(ks_x_fwd<T, N, M>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm); break;
            case 1: cudaFuncSetAttribute(ks_y<T, N, M, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm); break;
            case 2: cudaFuncSetAttribute(ks_z_solve<T, N, M>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm); break;
            case 3: cudaFuncSetAttribute(ks_y<T, N, M, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm); break;
            case 4: cudaFuncSetAttribute(ks_x_inv<T, N, M>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm); break;
        }
        return;
    }
    const Geo& g = p->g;
    const int nxh = g.nx / 2 + 1;
    const long rows = (long)g.ny * g.nz;
    switch (pass) {
        case 0: ks_x_fwd<T, N, M><<<(int)((rows + M - 1) / M), 256, sm, s>>>(g, tw, src, C); break;
        case 1: ks_y<T, N, M, false><<<((nxh + M - 1) / M) * g.nz, 256, sm, s>>>(g, tw, C); break;
        case 2: {
            const T* l0 = sizeof(T) == 8 ? (const T*)p->lam[0] : (const T*)p->lam32[0];
            const T* l1 = sizeof(T) == 8 ? (const T*)p->lam[1] : (const T*)p->lam32[1];
            const T* l2 = sizeof(T) == 8 ? (const T*)p->lam[2] : (const T*)p->lam32[2];
            ks_z_solve<T, N, M><<<((nxh + M - 1) / M) * g.ny, 256, sm, s>>>(g, tw, l0, l1, l2, C);
            break;
        }
        case 3: ks_y<T, N, M, true><<<((nxh + M - 1) / M) * g.nz, 256, sm, s>>>(g, tw, C); break;
        case 4: ks_x_inv<T, N, M><<<(int)((rows + M - 1) / M), 256, sm, s>>>(g, tw, C, out); break;
    }
}

template <typename T>
bool dispatch_pass(int n, int pass, FFTPlan* p, const T* tw, const T* src, T* out, Cx<T>* C, cudaStream_t s,
                   bool attr) {
    switch (n) {
        case 8: static_pass<T, 8>(pass, p, tw, src, out, C, s, attr); return true;
        case 12: static_pass<T, 12>(pass, p, tw, src, out, C, s, attr); return true;
        case 16: static_pass<T, 16>(pass, p, tw, src, out, C, s, attr); return true;
        case 24: static_pass<T, 24>(pass, p, tw, src, out, C, s, attr); return true;
        case 32: static_pass<T, 32>(pass, p, tw, src, out, C, s, attr); return true;
        case 48: static_pass<T, 48>(pass, p, tw, src, out, C, s, attr); return true;
        case 64: static_pass<T, 64>(pass, p, tw, src, out, C, s, attr); return true;
        case 96: static_pass<T, 96>(pass, p, tw, src, out, C, s, attr); return true;
        case 128: static_pass<T, 128>(pass, p, tw, src, out, C, s, attr); return true;
        case 192: static_pass<T, 192>(pass, p, tw, src, out, C, s, attr); return true;
        case 256: static_pass<T, 256>(pass, p, tw, src, out, C, s, attr); return true;
        case 384: static_pass<T, 384>(pass, p, tw, src, out, C, s, attr); return true;
        case 512: static_pass<T, 512>(pass, p, tw, src, out, C, s, attr); return true;
        default: return false;
    }
}

template <typename T>
void run_fft_poisson(FFTPlan* p, const T* src, T* out, void* work, cudaStream_t s) {
    const Geo& g = p->g;
    Cx<T>* C = reinterpret_cast<Cx<T>*>(work);
    const size_t cs = sizeof(Cx<T>);
    const bool dbl = sizeof(T) == 8;
    const T* twx = dbl ? (const T*)p->tw64[0] : (const T*)p->tw32[0];
    const T* twy = dbl ? (const T*)p->tw64[1] : (const T*)p->tw32[1];
    const T* twz = dbl ? (const T*)p->tw64[2] : (const T*)p->tw32[2];
    const int nxh = g.nx / 2 + 1;
    const int mx = lines_per_cta(g.nx, cs), my = lines_per_cta(g.ny, cs), mz = lines_per_cta(g.nz, cs);
    const long rows = (long)g.ny * g.nz;
    const int bx = (int)((rows + mx - 1) / mx);
    const int by = ((nxh + my - 1) / my) * g.nz;
    const int bz = ((nxh + mz - 1) / mz) * g.ny;
    const size_t sx = smem_bytes(g.nx, mx, cs), sy = smem_bytes(g.ny, my, cs), sz = smem_bytes(g.nz, mz, cs);
    // each pass: the compile-time-size kernel when there is one, else the generic one
    if (!dispatch_pass<T>(g.nx, 0, p, twx, src, out, C, s, false))
        k_fft_x_fwd<T><<<bx, 256, sx, s>>>(g, p->ax[0], twx, mx, src, C);
    if (!dispatch_pass<T>(g.ny, 1, p, twy, src, out, C, s, false))
        k_fft_y<T, false><<<by, 256, sy, s>>>(g, p->ax[1], twy, my, C);
    if (!dispatch_pass<T>(g.nz, 2, p, twz, src, out, C, s, false))
        k_fft_z_solve<T><<<bz, 256, sz, s>>>(g, p->ax[2], twz, mz, p->lam[0], p->lam[1], p->lam[2], C);
    if (!dispatch_pass<T>(g.ny, 3, p, twy, src, out, C, s, false))
        k_fft_y<T, true><<<by, 256, sy, s>>>(g, p->ax[1], twy, my, C);
    if (!dispatch_pass<T>(g.nx, 4, p, twx, src, out, C, s, false))
        k_fft_x_inv<T><<<bx, 256, sx, s>>>(g, p->ax[0], twx, mx, C, out);
}

// allow the dynamic shared memory of every pass (done once, before any capture)
template <typename T>
void set_fft_attributes(const Geo& g) {
    const size_t cs = sizeof(Cx<T>);
    const int mx = lines_per_cta(g.nx, cs), my = lines_per_cta(g.ny, cs), mz = lines_per_cta(g.nz, cs);
    const size_t sx = smem_bytes(g.nx, mx, cs), sy = smem_bytes(g.ny, my, cs), sz = smem_bytes(g.nz, mz, cs);
    cudaFuncSetAttribute(k_fft_x_fwd<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sx);
    cudaFuncSetAttribute(k_fft_x_inv<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sx);
    cudaFuncSetAttribute(k_fft_y<T, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sy);
    cudaFuncSetAttribute(k_fft_y<T, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sy);
    cudaFuncSetAttribute(k_fft_z_solve<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sz);
    const int ns[5] = {g.nx, g.ny, g.nz, g.ny, g.nx};
    for (int pass = 0; pass < 5; ++pass)
        dispatch_pass<T>(ns[pass], pass, nullptr, nullptr, nullptr, nullptr, nullptr, nullptr, true);
}

}  // namespace

FFTPlan* fft_create(const Geo& g, cudaStream_t s) {
    FFTPlan* p = new FFTPlan();
    p->g = g;
    const int n[3] = {g.nx, g.ny, g.nz};
    const double h[3] = {g.hx, g.hy, g.hz};
    for (int a = 0; a < 3; ++a) {
        p->ax[a] = make_axis(n[a]);
        if (p->ax[a].nstages < 0) { delete p; return nullptr; }
        p->tw64[a] = nullptr; p->tw32[a] = nullptr; p->lam[a] = nullptr; p->lam32[a] = nullptr;
        if (cudaMalloc(&p->tw64[a], sizeof(double) * 2 * n[a]) != cudaSuccess ||
            cudaMalloc(&p->tw32[a], sizeof(float) * 2 * n[a]) != cudaSuccess ||
            cudaMalloc(&p->lam[a], sizeof(double) * n[a]) != cudaSuccess ||
            cudaMalloc(&p->lam32[a], sizeof(float) * n[a]) != cudaSuccess) {
            fft_destroy(p);
            return nullptr;
        }
        k_twiddles<<<(n[a] + 127) / 128, 128, 0, s>>>(n[a], p->tw64[a], p->tw32[a]);
        k_symbol<<<(n[a] + 127) / 128, 128, 0, s>>>(n[a], h[a], p->lam[a], p->lam32[a]);
    }
    set_fft_attributes<float>(g);
    set_fft_attributes<double>(g);
    return p;
}

void fft_destroy(FFTPlan* p) {
    if (!p) return;
    for (int a = 0; a < 3; ++a) {
        if (p->tw64[a]) cudaFree(p->tw64[a]);
        if (p->tw32[a]) cudaFree(p->tw32[a]);
        if (p->lam[a]) cudaFree(p->lam[a]);
        if (p->lam32[a]) cudaFree(p->lam32[a]);
    }
    delete p;
}

size_t fft_workspace_bytes(const Geo& g, bool dbl) {
    return (size_t)(g.nx / 2 + 1) * g.ny * g.nz * 2 * (dbl ? sizeof(double) : sizeof(float));
}

template <typename T> void fft_poisson(FFTPlan* p, const T* src, T* out, void* work, cudaStream_t s) {
    run_fft_poisson<T>(p, src, out, work, s);
}
template void fft_poisson<float>(FFTPlan*, const float*, float*, void*, cudaStream_t);
template void fft_poisson<double>(FFTPlan*, const double*, double*, void*, cudaStream_t);

}  // namespace gp
