// Fields built from the atoms: the dielectric eps(R) (Sec. II.B), the Gaussian
// charge density (Sec. II.A), the dry-plane test (Sec. II.C), the energy
// (Eq. 4) and the forces (Eq. 11, Appendix B).
//
// Every kernel here works on 32 x 4 x 4 tiles of grid points, one thread per
// point. A tile first culls the periodic images of a chunk of atoms against
// its bounding box (in FP32, with a safety margin), keeps the survivors in
// shared memory, and then every thread runs over that short list in FP64.
#include "gp_common.cuh"

namespace gp {
namespace {

constexpr int TX = 32, TY = 4, TZ = 4, TT = TX * TY * TZ;
constexpr int ACH = 32;                // atoms per culling chunk
constexpr int MAXE = ACH * 27;         // (atom, image) entries per chunk
constexpr float kMargin = 1e-3f;       // FP32 culling slack, Angstrom

__device__ __forceinline__ double wrap_pos(double x, double L) { return x - L * floor(x / L); }

// image `im` (0..26) of wrapped atom a: FP32 centre for culling
__device__ __forceinline__ void image32(const float4* w32, int a, int im, const Geo& g, float& cx, float& cy,
                                        float& cz) {
    const float4 p = w32[a];
    cx = p.x + (float)((im % 3 - 1) * g.lx);
    cy = p.y + (float)(((im / 3) % 3 - 1) * g.ly);
    cz = p.z + (float)((im / 9 - 1) * g.lz);
}

// the same image in FP64
__device__ __forceinline__ void image64(const double* w64, int a, int im, const Geo& g, double& cx, double& cy,
                                        double& cz) {
    cx = w64[3 * a + 0] + (im % 3 - 1) * g.lx;
    cy = w64[3 * a + 1] + ((im / 3) % 3 - 1) * g.ly;
    cz = w64[3 * a + 2] + (im / 9 - 1) * g.lz;
}

__global__ void k_wrap_atoms(Geo g, const double* pos, int n, double* w64, float4* w32) {
    const int a = blockIdx.x * blockDim.x + threadIdx.x;
    if (a >= n) return;
    const double x = wrap_pos(pos[3 * a + 0], g.lx), y = wrap_pos(pos[3 * a + 1], g.ly),
                 z = wrap_pos(pos[3 * a + 2], g.lz);
    w64[3 * a + 0] = x; w64[3 * a + 1] = y; w64[3 * a + 2] = z;
    w32[a] = make_float4((float)x, (float)y, (float)z, 0.f);
}

struct Tile {
    int i0, j0, k0, i1, j1, k1;        // first and last grid index in the tile
    float bx0, bx1, by0, by1, bz0, bz1;
};

__device__ __forceinline__ Tile make_tile(const Geo& g) {
    Tile t;
    t.i0 = blockIdx.x * TX; t.j0 = blockIdx.y * TY; t.k0 = blockIdx.z * TZ;
    t.i1 = min(t.i0 + TX, g.nx) - 1; t.j1 = min(t.j0 + TY, g.ny) - 1; t.k1 = min(t.k0 + TZ, g.nz) - 1;
    t.bx0 = (float)(t.i0 * g.hx); t.bx1 = (float)(t.i1 * g.hx);
    t.by0 = (float)(t.j0 * g.hy); t.by1 = (float)(t.j1 * g.hy);
    t.bz0 = (float)(t.k0 * g.hz); t.bz1 = (float)(t.k1 * g.hz);
    return t;
}

// squared distance from point c to the tile box (FP32)
__device__ __forceinline__ float box_d2(const Tile& t, float cx, float cy, float cz) {
    float dx = fmaxf(fmaxf(t.bx0 - cx, cx - t.bx1), 0.f);
    float dy = fmaxf(fmaxf(t.by0 - cy, cy - t.by1), 0.f);
    float dz = fmaxf(fmaxf(t.bz0 - cz, cz - t.bz1), 0.f);
    return dx * dx + dy * dy + dz * dz;
}

// largest per-axis distance from c to the box (FP32)
__device__ __forceinline__ float box_dmax(const Tile& t, float cx, float cy, float cz) {
    float dx = fmaxf(fmaxf(t.bx0 - cx, cx - t.bx1), 0.f);
    float dy = fmaxf(fmaxf(t.by0 - cy, cy - t.by1), 0.f);
    float dz = fmaxf(fmaxf(t.bz0 - cz, cz - t.bz1), 0.f);
    return fmaxf(dx, fmaxf(dy, dz));
}

// ----------------------------------------------------------------- switching-function tables
// s(d) = erfc((r0 - d)/w)/2 and h(d) = s'(d)/(s(d) d) tabulated as functions
// of q = d^2 (no square root per pair): kSwNI equal intervals in q, on each a
// degree-kSwDeg polynomial in the local variable t in [-1, 1], obtained by
// Chebyshev interpolation (Trefethen, Approximation Theory and Approximation
// Practice, ch. 3: values at the Chebyshev points of the first kind, discrete
// cosine transform to Chebyshev coefficients, then to monomials). The FP64
// values at the nodes come from erfc and exp. Interpolation error is about
// 5e-15 relative for s on q in [(r0-4w)^2, (r0+6w)^2] and for h on
// [(r0-3.5w)^2, (r0+3.5w)^2]; outside those ranges the kernels use exact
// forms (s = 1, or FP32 special functions on terms below 1e-8).
__global__ void k_switch_tables(DielParams p, SwTables tb, double* s_coef, double* h_coef) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= 2 * kSwNI) return;
    const bool is_h = k >= kSwNI;
    const int iv = is_h ? k - kSwNI : k;
    const double qlo = is_h ? tb.h_qlo : tb.s_qlo;
    const double dq = 1.0 / (is_h ? tb.h_inv_dq : tb.s_inv_dq);
    constexpr int n = kSwDeg + 1;
    double fv[n], c[n];
    for (int j = 0; j < n; ++j) {
        const double xj = cospi((j + 0.5) / n);
        const double q = qlo + iv * dq + (xj + 1.0) * 0.5 * dq;
        const double d = sqrt(q);
        const double u = (d - p.r0) / p.w;
        const double sv = 0.5 * erfc(-u);
        fv[j] = is_h ? exp(-u * u) / (p.w * sqrt(kPi)) / (sv * d) : sv;
    }
    for (int m = 0; m < n; ++m) {
        double acc = 0.0;
        for (int j = 0; j < n; ++j) acc += fv[j] * cospi(m * (j + 0.5) / n);
        c[m] = acc * 2.0 / n;
    }
    c[0] *= 0.5;
    // monomial coefficients: T_0 = 1, T_1 = t, T_{m+1} = 2 t T_m - T_{m-1}
    double Tm1[n], Tm[n], mono[n];
    for (int e = 0; e < n; ++e) { Tm1[e] = 0.0; Tm[e] = 0.0; mono[e] = 0.0; }
    Tm1[0] = 1.0;                       // T_0
    Tm[1] = 1.0;                        // T_1
    mono[0] += c[0];
    for (int e = 0; e < n; ++e) mono[e] += c[1] * Tm[e];
    for (int m = 2; m < n; ++m) {
        double Tn[n];
        for (int e = 0; e < n; ++e) Tn[e] = (e > 0 ? 2.0 * Tm[e - 1] : 0.0) - Tm1[e];
        for (int e = 0; e < n; ++e) { mono[e] += c[m] * Tn[e]; Tm1[e] = Tm[e]; Tm[e] = Tn[e]; }
    }
    double* out = (is_h ? h_coef : s_coef) + (long)iv * n;
    for (int e = 0; e < n; ++e) out[e] = mono[e];
}

__device__ __forceinline__ double sw_eval(const double* __restrict__ coef, double qlo, double inv_dq, double q) {
    double x = (q - qlo) * inv_dq;
    int k = (int)x;
    k = k < 0 ? 0 : (k >= kSwNI ? kSwNI - 1 : k);
    const double t = 2.0 * (x - k) - 1.0;
    const double* c = coef + k * (kSwDeg + 1);
    double acc = __ldg(c + kSwDeg);
#pragma unroll
    for (int e = kSwDeg - 1; e >= 0; --e) acc = fma(acc, t, __ldg(c + e));
    return acc;
}

// ----------------------------------------------------------------- eps
// compact 8 x 2 x 2 block of the tile for warp w, lane l (spatially close points
// take the same branches below)
__device__ __forceinline__ void compact_point(int w, int l, int& tx, int& ty, int& tz) {
    tx = (w & 3) * 8 + (l & 7);
    ty = ((w >> 2) & 1) * 2 + ((l >> 3) & 1);
    tz = (w >> 3) * 2 + (l >> 4);
}

// s(d) = erfc((r0 - d)/w)/2 with u = (d - r0)/w. Far from the switching
// radius (|u| > 4) the factor is 1 - t or t with t = erfc(|u|)/2 < 7.7e-9:
// FP32 erfc gives t to a few ulp, i.e. s to 1e-15 absolute (u > 4) or to
// 1e-7 relative of a factor below 7.7e-9 (u < -4); otherwise FP64.
__device__ __forceinline__ double switch_s(double u) {
    if (u > 4.0) return 1.0 - 0.5 * (double)erfcf((float)u);
    if (u < -4.0) return 0.5 * (double)erfcf((float)(-u));
    return 0.5 * erfc(-u);
}

// eps = 1 + (eps0 - 1) prod s(d). Once (eps0-1) P < 2^-54 further factors
// (all <= 1) cannot move 1 + (eps0-1) P away from 1.0, so the product stops.
__global__ void __launch_bounds__(TT) k_build_eps(Geo g, Atoms at, DielParams p, SwTables tb, double* eps64,
                                                  double* pe64, float* eps32) {
    __shared__ double ec[MAXE][3];
    __shared__ int ne;
    const Tile t = make_tile(g);
    int tx, ty, tz;
    compact_point(threadIdx.x >> 5, threadIdx.x & 31, tx, ty, tz);
    const int i = t.i0 + tx, j = t.j0 + ty, k = t.k0 + tz;
    const bool valid = i < g.nx && j < g.ny && k < g.nz;
    const double x = i * g.hx, y = j * g.hy, z = k * g.hz;
    const double rc2 = p.rcut * p.rcut;
    const double iw = 1.0 / p.w;
    const double tiny = 5.5e-17 / (p.eps0 - 1.0 > 0.0 ? p.eps0 - 1.0 : 1.0);
    const float rcf = (float)p.rcut + kMargin;
    double P = 1.0;
    for (int a0 = 0; a0 < at.n; a0 += ACH) {
        if (threadIdx.x == 0) ne = 0;
        __syncthreads();
        const int na = min(ACH, at.n - a0);
        for (int q = threadIdx.x; q < na * 27; q += TT) {
            const int a = a0 + q / 27, im = q % 27;
            float fx, fy, fz;
            image32(at.w32, a, im, g, fx, fy, fz);
            if (box_d2(t, fx, fy, fz) < rcf * rcf) {
                const int s = atomicAdd(&ne, 1);
                image64(at.w64, a, im, g, ec[s][0], ec[s][1], ec[s][2]);
            }
        }
        __syncthreads();
        const int m = ne;
        if (valid && P >= tiny) {
            for (int e = 0; e < m; ++e) {
                const double dx = x - ec[e][0], dy = y - ec[e][1], dz = z - ec[e][2];
                const double d2 = dx * dx + dy * dy + dz * dz;
                if (d2 < rc2) {
                    double sv;
                    if (!tb.s) sv = switch_s((sqrt(d2) - p.r0) * iw);
                    else if (d2 >= tb.s_qhi) continue;                 // u >= 6: s == 1 in FP64
                    else if (d2 > tb.s_qlo) sv = sw_eval(tb.s, tb.s_qlo, tb.s_inv_dq, d2);
                    else sv = 0.5 * (double)erfcf((float)((p.r0 - sqrt(d2)) * iw));   // u < -4, s < 8e-9
                    P *= sv;
                    if (P < tiny) break;
                }
            }
        }
        __syncthreads();
    }
    if (valid) {
        const long idx = i + (long)g.nx * (j + (long)g.ny * k);
        const double pe = (p.eps0 - 1.0) * P;
        const double e = 1.0 + pe;
        eps64[idx] = e;
        if (pe64) pe64[idx] = pe;
        if (eps32) eps32[idx] = (float)e;
    }
}

// ----------------------------------------------------------------- df64
// A value carried as an unevaluated sum hi + lo of two FP32 numbers (about 48
// significant bits; Dekker 1971, Knuth's two-sum). The per-point sums of the
// density and its force run in this form: a few FP32 instructions replace an
// FP64 instruction that costs 64 FP32 issue slots on this GPU.
struct df { float hi, lo; };

__device__ __forceinline__ df df_from(double v) {
    const float h = (float)v;
    return {h, (float)(v - (double)h)};
}
__device__ __forceinline__ double df_to(df a) { return (double)a.hi + (double)a.lo; }

__device__ __forceinline__ df df_quick(float s, float e) {   // |s| >= |e|
    const float t = s + e;
    return {t, e - (t - s)};
}
__device__ __forceinline__ df df_mul(df a, df b) {
    const float p = a.hi * b.hi;
    float e = fmaf(a.hi, b.hi, -p);
    e = fmaf(a.hi, b.lo, e);
    e = fmaf(a.lo, b.hi, e);
    return df_quick(p, e);
}
__device__ __forceinline__ df df_add(df a, df b) {
    const float s = a.hi + b.hi;
    const float v = s - a.hi;
    float e = (a.hi - (s - v)) + (b.hi - v);
    e += a.lo + b.lo;
    return df_quick(s, e);
}

// ----------------------------------------------------------------- Gaussian factor tables
// One-dimensional factors of every Gaussian, exp(-(x_i - c)^2 / 2 sigma^2) with
// c an image of the atom's coordinate along one axis (shift -L, 0, +L), zero
// outside the 8 sigma window; indexed [atom][core/cloud][axis][image][i].
// Tiles then read these instead of evaluating exp per tile.
__device__ __forceinline__ long gtab_index(int a, int which, int axis, int img, int i, int nmax) {
    return ((((long)a * 2 + which) * 3 + axis) * 3 + img) * nmax + i;
}

__global__ void k_gauss_tables(Geo g, Atoms at, double cut, int nmax, double* tab) {
    const long total = (long)at.n * 2 * 3 * 3 * nmax;
    for (long q = blockIdx.x * (long)blockDim.x + threadIdx.x; q < total; q += (long)gridDim.x * blockDim.x) {
        const int i = (int)(q % nmax);
        long r = q / nmax;
        const int img = (int)(r % 3); r /= 3;
        const int axis = (int)(r % 3); r /= 3;
        const int which = (int)(r % 2);
        const int a = (int)(r / 2);
        const int n = axis == 0 ? g.nx : (axis == 1 ? g.ny : g.nz);
        double v = 0.0;
        if (i < n) {
            const double h = axis == 0 ? g.hx : (axis == 1 ? g.hy : g.hz);
            const double L = axis == 0 ? g.lx : (axis == 1 ? g.ly : g.lz);
            const double sg = at.gauss[3 * a + 1 + which];
            const double c = at.w64[3 * a + axis] + (img - 1) * L;
            const double d = i * h - c;
            if (fabs(d) < cut * sg) v = exp(-d * d / (2.0 * sg * sg));
        }
        tab[q] = v;
    }
}

// ----------------------------------------------------------------- rho
// Separable Gaussians: g(r) = N exp(-dx^2/2s^2) exp(-dy^2/2s^2) exp(-dz^2/2s^2),
// each factor zero outside |d| < cut*s. A tile tabulates the three 1D factors
// per (atom, image, Gaussian) entry and every point then costs two products.
// Entries whose largest value on the tile is below 1e-8 of their peak are
// tabulated and summed in FP32 (their sum is far below FP64 rounding of the
// total); the others in FP64.
constexpr int RCH = 8;                  // atoms per chunk
constexpr int RMAX = RCH * 27 * 2;      // entries per chunk
constexpr int RSUB = 32;                // entries tabulated at a time
constexpr double kTail = 1e-8;

// largest exp(-d^2/2s^2) of a Gaussian centred at c over the tile box
__device__ __forceinline__ double tile_peak(const Tile& t, const Geo& g, double cx, double cy, double cz, double sg) {
    const double dx = fmax(fmax(t.i0 * g.hx - cx, cx - t.i1 * g.hx), 0.0);
    const double dy = fmax(fmax(t.j0 * g.hy - cy, cy - t.j1 * g.hy), 0.0);
    const double dz = fmax(fmax(t.k0 * g.hz - cz, cz - t.k1 * g.hz), 0.0);
    return exp(-(dx * dx + dy * dy + dz * dz) / (2.0 * sg * sg));
}

__global__ void __launch_bounds__(TT) k_build_rho(Geo g, Atoms at, double cut, const double* __restrict__ tab,
                                                  int nmax, double* rho) {
    __shared__ double en[RMAX][5];      // cx, cy, cz, sigma, coefficient (near entries from the front,
                                        //  FP32 tail entries from the back)
    __shared__ int ekey[RMAX];          // (atom * 2 + which) * 27 + image
    __shared__ df gx[RSUB][TX];
    __shared__ double gy[RSUB][TY];
    __shared__ double gz[RSUB][TZ];
    __shared__ df gyz[RSUB][TY * TZ];
    __shared__ float fx32[RSUB][TX];
    __shared__ float fy32[RSUB][TY];
    __shared__ float fz32[RSUB][TZ];
    __shared__ int n64, n32;
    const Tile t = make_tile(g);
    const int tx = threadIdx.x % TX, ty = (threadIdx.x / TX) % TY, tz = threadIdx.x / (TX * TY);
    const int i = t.i0 + tx, j = t.j0 + ty, k = t.k0 + tz;
    const bool valid = i < g.nx && j < g.ny && k < g.nz;
    df acc = {0.f, 0.f};
    float acc32 = 0.f;
    for (int a0 = 0; a0 < at.n; a0 += RCH) {
        if (threadIdx.x == 0) { n64 = 0; n32 = 0; }
        __syncthreads();
        const int na = min(RCH, at.n - a0);
        for (int q = threadIdx.x; q < na * 54; q += TT) {
            const int a = a0 + q / 54, r = q % 54, im = r % 27, which = r / 27;
            const double sg = at.gauss[3 * a + 1 + which];
            float fx, fy, fz;
            image32(at.w32, a, im, g, fx, fy, fz);
            const float rad = (float)(cut * sg) + kMargin;
            if (box_dmax(t, fx, fy, fz) < rad) {
                const double Z = at.gauss[3 * a + 0];
                double cx, cy, cz;
                image64(at.w64, a, im, g, cx, cy, cz);
                const bool tail = tile_peak(t, g, cx, cy, cz, sg) < kTail;
                const int s = tail ? RMAX - 1 - atomicAdd(&n32, 1) : atomicAdd(&n64, 1);
                en[s][0] = cx; en[s][1] = cy; en[s][2] = cz; en[s][3] = sg;
                const double norm = 1.0 / (2.0 * kPi * sg * sg * sqrt(2.0 * kPi * sg * sg));
                en[s][4] = (which == 0 ? Z : -Z) * norm;
                ekey[s] = (a * 2 + which) * 27 + im;
            }
        }
        __syncthreads();
        const int m64 = n64, m32 = n32;
        for (int e0 = 0; e0 < m64; e0 += RSUB) {
            const int ms = min(RSUB, m64 - e0);
            for (int q = threadIdx.x; q < ms * (TX + TY + TZ); q += TT) {
                const int e = q / (TX + TY + TZ), r = q % (TX + TY + TZ);
                const int key = ekey[e0 + e];
                const int im = key % 27, aw = key / 27;
                const int a = aw / 2, which = aw % 2;
                if (r < TX) {
                    const int ii = t.i0 + r;
                    gx[e][r] = df_from(ii < g.nx ? tab[gtab_index(a, which, 0, im % 3, ii, nmax)] : 0.0);
                } else if (r < TX + TY) {
                    const int rr = r - TX, jj = t.j0 + rr;
                    gy[e][rr] = jj < g.ny ? en[e0 + e][4] * tab[gtab_index(a, which, 1, (im / 3) % 3, jj, nmax)] : 0.0;
                } else {
                    const int rr = r - TX - TY, kk = t.k0 + rr;
                    gz[e][rr] = kk < g.nz ? tab[gtab_index(a, which, 2, im / 9, kk, nmax)] : 0.0;
                }
            }
            __syncthreads();
            for (int q = threadIdx.x; q < ms * TY * TZ; q += TT) {
                const int e = q / (TY * TZ), r = q % (TY * TZ);
                gyz[e][r] = df_from(gy[e][r / TZ] * gz[e][r % TZ]);
            }
            __syncthreads();
            if (valid) {
                for (int e = 0; e < ms; ++e) acc = df_add(acc, df_mul(gx[e][tx], gyz[e][ty * TZ + tz]));
            }
            __syncthreads();
        }
        for (int e0 = 0; e0 < m32; e0 += RSUB) {
            const int ms = min(RSUB, m32 - e0);
            for (int q = threadIdx.x; q < ms * (TX + TY + TZ); q += TT) {
                const int e = q / (TX + TY + TZ), r = q % (TX + TY + TZ);
                const int slot = RMAX - 1 - (e0 + e);
                const int key = ekey[slot];
                const int im = key % 27, aw = key / 27;
                const int a = aw / 2, which = aw % 2;
                if (r < TX) {
                    const int ii = t.i0 + r;
                    fx32[e][r] = ii < g.nx ? (float)tab[gtab_index(a, which, 0, im % 3, ii, nmax)] : 0.f;
                } else if (r < TX + TY) {
                    const int rr = r - TX, jj = t.j0 + rr;
                    fy32[e][rr] = jj < g.ny ? (float)(en[slot][4] * tab[gtab_index(a, which, 1, (im / 3) % 3, jj, nmax)])
                                            : 0.f;
                } else {
                    const int rr = r - TX - TY, kk = t.k0 + rr;
                    fz32[e][rr] = kk < g.nz ? (float)tab[gtab_index(a, which, 2, im / 9, kk, nmax)] : 0.f;
                }
            }
            __syncthreads();
            if (valid) {
                for (int e = 0; e < ms; ++e) acc32 = fmaf(fx32[e][tx] * fy32[e][ty], fz32[e][tz], acc32);
            }
            __syncthreads();
        }
    }
    if (valid) rho[i + (long)g.nx * (j + (long)g.ny * k)] = df_to(acc) + (double)acc32;
}

// ----------------------------------------------------------------- dry planes
__global__ void k_plane_max(Geo g, const double* eps64, double* out) {
    __shared__ double red[256];
    const int k = blockIdx.x;
    const long pl = plane_of(g.nx, g.ny);
    double m = 0.0;
    for (long q = threadIdx.x; q < pl; q += blockDim.x) m = fmax(m, eps64[k * pl + q] - 1.0);
    red[threadIdx.x] = m;
    __syncthreads();
    for (int s = blockDim.x / 2; s > 0; s >>= 1) {
        if (threadIdx.x < s) red[threadIdx.x] = fmax(red[threadIdx.x], red[threadIdx.x + s]);
        __syncthreads();
    }
    if (threadIdx.x == 0) out[k] = red[0];
}

// ----------------------------------------------------------------- energy
// partial[2b] = sum rho phi, partial[2b+1] = sum_f eps_f (grad_f phi)^2 over block b
__global__ void __launch_bounds__(kReduceThreads) k_energy(Geo g, const double* rho, const double* phi,
                                                           const double* eps, double* partial) {
    __shared__ double red[2][kReduceThreads];
    const long n = (long)g.nx * g.ny * g.nz;
    const long pl = plane_of(g.nx, g.ny);
    const double ihx = 1.0 / g.hx, ihy = 1.0 / g.hy, ihz = 1.0 / g.hz;
    double s0 = 0.0, s1 = 0.0;
    for (long c = blockIdx.x * (long)blockDim.x + threadIdx.x; c < n; c += (long)gridDim.x * blockDim.x) {
        const int i = (int)(c % g.nx);
        const int j = (int)((c / g.nx) % g.ny);
        const int k = (int)(c / pl);
        const long xp = c + (i == g.nx - 1 ? 1 - g.nx : 1);
        const long yp = c + (j == g.ny - 1 ? (1 - g.ny) * (long)g.nx : g.nx);
        const long zp = c + (k == g.nz - 1 ? (1 - g.nz) * pl : pl);
        const double p0 = phi[c], e0 = eps[c];
        s0 += rho[c] * p0;
        double gx = (phi[xp] - p0) * ihx, gy = (phi[yp] - p0) * ihy, gz = (phi[zp] - p0) * ihz;
        s1 += 0.5 * ((e0 + eps[xp]) * gx * gx + (e0 + eps[yp]) * gy * gy + (e0 + eps[zp]) * gz * gz);
    }
    red[0][threadIdx.x] = s0;
    red[1][threadIdx.x] = s1;
    __syncthreads();
    for (int s = blockDim.x / 2; s > 0; s >>= 1) {
        if (threadIdx.x < s) {
            red[0][threadIdx.x] += red[0][threadIdx.x + s];
            red[1][threadIdx.x] += red[1][threadIdx.x + s];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        partial[2 * blockIdx.x] = red[0][0];
        partial[2 * blockIdx.x + 1] = red[1][0];
    }
}

// ----------------------------------------------------------------- forces
__device__ __forceinline__ double warp_sum(double v) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// dielectric part: S_a = sum_i W_i sum_images q(d) (-(r_i - c)/d), with
// W_i = (1/2) sum over the six faces of i of (grad_f phi)^2 times pe_i = eps_i - 1,
// q = s'/s. G_eps_a = -h^3/(8 pi) S_a (applied in k_forces_finish).
// One warp per (atom, image) entry runs over the tile's 512 points in compact
// 8 x 2 x 2 blocks. Pairs with |u| > 3.5 contribute at most 5e-6 of a pair at
// the switching radius; their s and s' are taken in FP32.
__global__ void __launch_bounds__(TT) k_forces_eps(Geo g, Atoms at, DielParams p, SwTables tb, const double* phi,
                                                   const double* pe64, double* S) {
    __shared__ double ec[MAXE][3];
    __shared__ int eatom[MAXE];
    __shared__ double Ws[TT];
    __shared__ int ne;
    const Tile t = make_tile(g);
    {
        const int tx = threadIdx.x % TX, ty = (threadIdx.x / TX) % TY, tz = threadIdx.x / (TX * TY);
        const int i = t.i0 + tx, j = t.j0 + ty, k = t.k0 + tz;
        double W = 0.0;
        if (i < g.nx && j < g.ny && k < g.nz) {
            const long pl = plane_of(g.nx, g.ny);
            const long c = i + (long)g.nx * (j + (long)g.ny * k);
            const long xp = c + (i == g.nx - 1 ? 1 - g.nx : 1), xm = c - (i == 0 ? 1 - g.nx : 1);
            const long yp = c + (j == g.ny - 1 ? (1 - g.ny) * (long)g.nx : g.nx);
            const long ym = c - (j == 0 ? (1 - g.ny) * (long)g.nx : g.nx);
            const long zp = c + (k == g.nz - 1 ? (1 - g.nz) * pl : pl);
            const long zm = c - (k == 0 ? (1 - g.nz) * pl : pl);
            const double p0 = phi[c];
            const double ax = (phi[xp] - p0) / g.hx, bx = (p0 - phi[xm]) / g.hx;
            const double ay = (phi[yp] - p0) / g.hy, by = (p0 - phi[ym]) / g.hy;
            const double az = (phi[zp] - p0) / g.hz, bz = (p0 - phi[zm]) / g.hz;
            W = 0.5 * (ax * ax + bx * bx + ay * ay + by * by + az * az + bz * bz) * pe64[c];
        }
        Ws[threadIdx.x] = W;   // index tx + TX (ty + TY tz)
    }
    const double rc2 = p.rcut * p.rcut;
    const double iw = 1.0 / p.w;
    const double sp_norm = 1.0 / (p.w * sqrt(kPi));
    const float rcf = (float)p.rcut + kMargin;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int a0 = 0; a0 < at.n; a0 += ACH) {
        if (threadIdx.x == 0) ne = 0;
        __syncthreads();
        const int na = min(ACH, at.n - a0);
        for (int q = threadIdx.x; q < na * 27; q += TT) {
            const int a = a0 + q / 27, im = q % 27;
            float fx, fy, fz;
            image32(at.w32, a, im, g, fx, fy, fz);
            if (box_d2(t, fx, fy, fz) < rcf * rcf) {
                const int s = atomicAdd(&ne, 1);
                image64(at.w64, a, im, g, ec[s][0], ec[s][1], ec[s][2]);
                eatom[s] = a;
            }
        }
        __syncthreads();
        const int m = ne;
        for (int e = warp; e < m; e += TT / 32) {
            const double cx = ec[e][0], cy = ec[e][1], cz = ec[e][2];
            double fx = 0.0, fy = 0.0, fz = 0.0;
            for (int blk = 0; blk < 16; ++blk) {
                int tx, ty, tz;
                compact_point(blk, lane, tx, ty, tz);
                const int i = t.i0 + tx, j = t.j0 + ty, k = t.k0 + tz;
                if (i >= g.nx || j >= g.ny || k >= g.nz) continue;
                const double dx = i * g.hx - cx, dy = j * g.hy - cy, dz = k * g.hz - cz;
                const double d2 = dx * dx + dy * dy + dz * dz;
                if (!(d2 < rc2 && d2 > 0.0)) continue;
                const double W = Ws[tx + TX * (ty + TY * tz)];
                const float df = sqrtf((float)d2);
                const float uf = (df - (float)p.r0) * (float)iw;
                double ratio;   // s'(d) / (s(d) d)
                if (fabsf(uf) > 3.45f) {
                    const float sf = 0.5f * erfcf(-uf);
                    const float spf = (float)sp_norm * expf(-uf * uf);
                    ratio = (double)(spf / (sf * df));
                } else if (tb.h) {
                    ratio = sw_eval(tb.h, tb.h_qlo, tb.h_inv_dq, d2);
                } else {
                    const double d = sqrt(d2);
                    const double u = (d - p.r0) * iw;
                    ratio = sp_norm * exp(-u * u) / (0.5 * erfc(-u) * d);
                }
                const double c = -W * ratio;
                fx += c * dx; fy += c * dy; fz += c * dz;
            }
            fx = warp_sum(fx); fy = warp_sum(fy); fz = warp_sum(fz);
            if (lane == 0) {
                const int a = eatom[e];
                if (fx != 0.0) atomicAdd(&S[3 * a + 0], fx);
                if (fy != 0.0) atomicAdd(&S[3 * a + 1], fy);
                if (fz != 0.0) atomicAdd(&S[3 * a + 2], fz);
            }
        }
        __syncthreads();
    }
}

// charge part: T_a = sum_i phi_i d rho~_i / d R_a with d g / d R = g (r - c)/sigma^2.
// One warp per (atom, image, Gaussian) entry, lanes along x; the y and z
// factors are separable, so each lane first sums its column over the 16
// (y, z) rows. Entries below 1e-8 of their peak on the tile run in FP32.
__global__ void __launch_bounds__(TT) k_forces_rho(Geo g, Atoms at, double cut, const double* __restrict__ tab,
                                                   int nmax, const double* phi, double* T) {
    __shared__ double en[RMAX][5];
    __shared__ int eatom[RMAX];
    __shared__ int ekey[RMAX];
    __shared__ double ph[TT];
    __shared__ int ne;
    const Tile t = make_tile(g);
    {
        const int tx = threadIdx.x % TX, ty = (threadIdx.x / TX) % TY, tz = threadIdx.x / (TX * TY);
        const int i = t.i0 + tx, j = t.j0 + ty, k = t.k0 + tz;
        ph[threadIdx.x] = (i < g.nx && j < g.ny && k < g.nz) ? phi[i + (long)g.nx * (j + (long)g.ny * k)] : 0.0;
    }
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int i = t.i0 + lane;
    const bool lane_ok = i < g.nx;
    for (int a0 = 0; a0 < at.n; a0 += RCH) {
        if (threadIdx.x == 0) ne = 0;
        __syncthreads();
        const int na = min(RCH, at.n - a0);
        for (int q = threadIdx.x; q < na * 54; q += TT) {
            const int a = a0 + q / 54, r = q % 54, im = r % 27, which = r / 27;
            const double sg = at.gauss[3 * a + 1 + which];
            float fx, fy, fz;
            image32(at.w32, a, im, g, fx, fy, fz);
            const float rad = (float)(cut * sg) + kMargin;
            if (box_dmax(t, fx, fy, fz) < rad) {
                const double Z = at.gauss[3 * a + 0];
                const int s = atomicAdd(&ne, 1);
                image64(at.w64, a, im, g, en[s][0], en[s][1], en[s][2]);
                en[s][3] = sg;
                const double norm = 1.0 / (2.0 * kPi * sg * sg * sqrt(2.0 * kPi * sg * sg));
                en[s][4] = (which == 0 ? Z : -Z) * norm / (sg * sg);
                eatom[s] = a;
                ekey[s] = (a * 2 + which) * 27 + im;
            }
        }
        __syncthreads();
        const int m = ne;
        for (int e = warp; e < m; e += TT / 32) {
            const double cx = en[e][0], cy = en[e][1], cz = en[e][2], sg = en[e][3], coef = en[e][4];
            const double rad = cut * sg;
            const double i2s = 1.0 / (2.0 * sg * sg);
            const int key = ekey[e], im = key % 27, aw = key / 27, ea = aw / 2, ew = aw % 2;
            // this lane's x factor and the 8 y / z factors, from the tables
            const double gxt = lane_ok ? tab[gtab_index(ea, ew, 0, im % 3, i, nmax)] : 0.0;
            double gyz_t = 0.0;
            if (lane < TY && t.j0 + lane < g.ny) gyz_t = tab[gtab_index(ea, ew, 1, (im / 3) % 3, t.j0 + lane, nmax)];
            else if (lane >= TY && lane < TY + TZ && t.k0 + lane - TY < g.nz)
                gyz_t = tab[gtab_index(ea, ew, 2, im / 9, t.k0 + lane - TY, nmax)];
            (void)rad; (void)i2s;
            double fx = 0.0, fy = 0.0, fz = 0.0;
            if (tile_peak(t, g, cx, cy, cz, sg) < kTail) {
                // FP32: lane < 8 tabulates one y or z factor, shared by shuffles
                float d_v = 0.f;
                if (lane < TY) d_v = (float)((t.j0 + lane) * g.hy - cy);
                else if (lane < TY + TZ) d_v = (float)((t.k0 + lane - TY) * g.hz - cz);
                const float gyz_v = (float)gyz_t;
                const float dxf = (float)(i * g.hx - cx);
                const float gxf = (float)gxt;
                float s0 = 0.f, sy = 0.f, sz = 0.f;
                for (int tz = 0; tz < TZ; ++tz) {
                    const float gz = __shfl_sync(0xffffffffu, gyz_v, TY + tz);
                    const float dz = __shfl_sync(0xffffffffu, d_v, TY + tz);
                    for (int ty = 0; ty < TY; ++ty) {
                        const float gy = __shfl_sync(0xffffffffu, gyz_v, ty);
                        const float dy = __shfl_sync(0xffffffffu, d_v, ty);
                        const float v = (float)ph[lane + TX * (ty + TY * tz)] * gy * gz;
                        s0 += v; sy += v * dy; sz += v * dz;
                    }
                }
                fx = coef * (double)(dxf * gxf * s0);
                fy = coef * (double)(gxf * sy);
                fz = coef * (double)(gxf * sz);
            } else {
                double d_v = 0.0;
                if (lane < TY) d_v = (t.j0 + lane) * g.hy - cy;
                else if (lane < TY + TZ) d_v = (t.k0 + lane - TY) * g.hz - cz;
                const double gyz_v = gyz_t;
                const double dx = i * g.hx - cx;
                const double gx = gxt;
                double s0 = 0.0, sy = 0.0, sz = 0.0;
                for (int tz = 0; tz < TZ; ++tz) {
                    const double gz = __shfl_sync(0xffffffffu, gyz_v, TY + tz);
                    const double dz = __shfl_sync(0xffffffffu, d_v, TY + tz);
                    for (int ty = 0; ty < TY; ++ty) {
                        const double gy = __shfl_sync(0xffffffffu, gyz_v, ty);
                        const double dy = __shfl_sync(0xffffffffu, d_v, ty);
                        const double v = ph[lane + TX * (ty + TY * tz)] * gy * gz;
                        s0 += v; sy += v * dy; sz += v * dz;
                    }
                }
                fx = coef * dx * gx * s0;
                fy = coef * gx * sy;
                fz = coef * gx * sz;
            }
            fx = warp_sum(fx); fy = warp_sum(fy); fz = warp_sum(fz);
            if (lane == 0) {
                const int a = eatom[e];
                if (fx != 0.0) atomicAdd(&T[3 * a + 0], fx);
                if (fy != 0.0) atomicAdd(&T[3 * a + 1], fy);
                if (fz != 0.0) atomicAdd(&T[3 * a + 2], fz);
            }
        }
        __syncthreads();
    }
}

__global__ void k_forces_finish(const double* S, const double* T, int n, double ce, double cr, double* F) {
    const int q = blockIdx.x * blockDim.x + threadIdx.x;
    if (q < 3 * n) F[q] = -(ce * S[q] + (T ? cr * T[q] : 0.0));
}

dim3 tile_grid(const Geo& g) {
    return dim3((g.nx + TX - 1) / TX, (g.ny + TY - 1) / TY, (g.nz + TZ - 1) / TZ);
}

}  // namespace

void launch_wrap_atoms(const Geo& g, const double* pos, int n, double* w64, float4* w32, cudaStream_t s) {
    if (n > 0) k_wrap_atoms<<<(n + 127) / 128, 128, 0, s>>>(g, pos, n, w64, w32);
}

void launch_switch_tables(DielParams p, const SwTables& tb, double* s_coef, double* h_coef, cudaStream_t s) {
    k_switch_tables<<<(2 * kSwNI + 127) / 128, 128, 0, s>>>(p, tb, s_coef, h_coef);
}

void launch_build_eps(const Geo& g, Atoms at, DielParams p, const SwTables& tb, double* eps64, double* pe64,
                      float* eps32, cudaStream_t s) {
    k_build_eps<<<tile_grid(g), TT, 0, s>>>(g, at, p, tb, eps64, pe64, eps32);
}

void launch_gauss_tables(const Geo& g, Atoms at, double cut, int nmax, double* tab, cudaStream_t s) {
    const long total = (long)at.n * 18 * nmax;
    if (total > 0) k_gauss_tables<<<(int)((total + 255) / 256 < 152L * 64 ? (total + 255) / 256 : 152L * 64), 256, 0, s>>>(
        g, at, cut, nmax, tab);
}

void launch_build_rho_raw(const Geo& g, Atoms at, double cut, const double* tab, int nmax, double* rho,
                          cudaStream_t s) {
    k_build_rho<<<tile_grid(g), TT, 0, s>>>(g, at, cut, tab, nmax, rho);
}

void launch_plane_max(const Geo& g, const double* eps64, double* out, cudaStream_t s) {
    k_plane_max<<<g.nz, 256, 0, s>>>(g, eps64, out);
}

void launch_energy(const Geo& g, const double* rho, const double* phi, const double* eps64,
                   double* partial, cudaStream_t s) {
    k_energy<<<kReduceBlocks, kReduceThreads, 0, s>>>(g, rho, phi, eps64, partial);
}

void launch_forces_eps(const Geo& g, Atoms at, DielParams p, const SwTables& tb, const double* phi,
                       const double* pe64, double* S, cudaStream_t s) {
    k_forces_eps<<<tile_grid(g), TT, 0, s>>>(g, at, p, tb, phi, pe64, S);
}

void launch_forces_rho(const Geo& g, Atoms at, double cut, const double* tab, int nmax, const double* phi,
                       double* T, cudaStream_t s) {
    k_forces_rho<<<tile_grid(g), TT, 0, s>>>(g, at, cut, tab, nmax, phi, T);
}

void launch_forces_finish(const double* S, const double* T, int n, double ce, double cr, double* F,
                          cudaStream_t s) {
    k_forces_finish<<<(3 * n + 255) / 256, 256, 0, s>>>(S, T, n, ce, cr, F);
}

}  // namespace gp
