// Fields built from the atoms: the dielectric eps(R) (Sec. II.B), the Gaussian
// charge density (Sec. II.A), the dry-plane test (Sec. II.C), the energy
// (Eq. 4) and the forces (Eq. 11, Appendix B).
//
// The kernels work on tiles of grid points: 32 x 4 x 4 with one thread per
// point, or 32 x 4 x 16 for the tabulated dielectric and its force (each
// thread takes 4 points along z). A tile first culls the periodic images of
// a chunk of atoms against its bounding box (in FP32, with a safety margin),
// keeps the survivors in shared memory, and then every thread runs over that
// short list: in FP64, or in df64 (pairs of FP32 numbers) where a kernel says
// so, because GB300's FP64 pipe runs at 1/64 of its FP32 rate.
#include "gp_common.cuh"

namespace gp {
namespace {

constexpr int TX = 32, TY = 4, TZ = 4, TT = TX * TY * TZ;
constexpr int ACH = 32;                // atoms per culling chunk
constexpr int MAXE = ACH * 27;         // (atom, image) entries per chunk
constexpr float kMargin = 1e-3f;       // FP32 culling slack, Angstrom

__device__ __forceinline__ double wrap_pos(double x, double L) { return x - L * floor(x / L); }

// shift -L, 0 or +L for image digit m in {0, 1, 2} (FP32, no conversion)
__device__ __forceinline__ float shift32(int m, float L) { return m == 0 ? -L : (m == 1 ? 0.f : L); }

// image `im` (0..26) of wrapped atom a: FP32 centre for culling (no FP64 work:
// the culling loop visits every atom image for every tile)
__device__ __forceinline__ void image32(const float4* w32, int a, int im, const Geo& g, float& cx, float& cy,
                                        float& cz) {
    const float4 p = w32[a];
    cx = p.x + shift32(im % 3, g.lxf);
    cy = p.y + shift32((im / 3) % 3, g.lyf);
    cz = p.z + shift32(im / 9, g.lzf);
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
    t.bx0 = (float)t.i0 * g.hxf; t.bx1 = (float)t.i1 * g.hxf;   // FP32: the culling keeps a margin
    t.by0 = (float)t.j0 * g.hyf; t.by1 = (float)t.j1 * g.hyf;
    t.bz0 = (float)t.k0 * g.hzf; t.bz1 = (float)t.k1 * g.hzf;
    return t;
}

// squared distance from point c to the tile box (FP32)
__device__ __forceinline__ float box_d2(const Tile& t, float cx, float cy, float cz) {
    float dx = fmaxf(fmaxf(t.bx0 - cx, cx - t.bx1), 0.f);
    float dy = fmaxf(fmaxf(t.by0 - cy, cy - t.by1), 0.f);
    float dz = fmaxf(fmaxf(t.bz0 - cz, cz - t.bz1), 0.f);
    return dx * dx + dy * dy + dz * dz;
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
__global__ void k_switch_tables(DielParams p, SwTables tb, double* s_coef, double* h_coef, float4* s_pack,
                                float4* h_pack) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= 2 * kSwNI) return;
    const bool is_h = k >= kSwNI;
    const int iv = is_h ? k - kSwNI : k;
    const double qlo = is_h ? tb.h_qlo : tb.s_qlo;
    const double dq = is_h ? tb.h_dq : tb.s_dq;
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
    float pk[16];
    const int split = is_h ? kSwSplitH : kSwSplitS;
    int o = 0;
    for (int e = 0; e < split; ++e) {
        const float hi = (float)mono[e];
        pk[o++] = hi;
        pk[o++] = (float)(mono[e] - (double)hi);
    }
    for (int e = split; e < n; ++e) pk[o++] = (float)mono[e];
    while (o < 16) pk[o++] = 0.f;
    float4* dst = (is_h ? h_pack : s_pack) + 4L * iv;
    for (int v = 0; v < 4; ++v) dst[v] = make_float4(pk[4 * v], pk[4 * v + 1], pk[4 * v + 2], pk[4 * v + 3]);
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
    const double iw = p.iw;
    const double tiny = p.tiny;
    const float rcf = p.rcutf + kMargin;
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
    const float2 p = split_to_float2(v);      // the casts' result, without the FP64 pipe
    return {p.x, p.y};
}
__device__ __forceinline__ double df_to(df a) { return f32_to_f64(a.hi) + f32_to_f64(a.lo); }
__device__ __forceinline__ df as_df(float2 v) { return df{v.x, v.y}; }

// (s, c): a compensated pair (value s + c) summed across the warp in place (Knuth two-sum per step)
__device__ __forceinline__ void warp_sum_df(float& s, float& c) {
    for (int o = 16; o > 0; o >>= 1) {
        const float s2 = __shfl_xor_sync(0xffffffffu, s, o);
        const float c2 = __shfl_xor_sync(0xffffffffu, c, o);
        const float t = s + s2;
        const float z = t - s;
        c += c2 + ((s - (t - z)) + (s2 - z));
        s = t;
    }
}

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

__device__ __forceinline__ double warp_sum(double v) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// ----------------------------------------------------------------- Gaussian factor tables
// A Gaussian truncated to the cube |x - c|, |y - c|, |z - c| < cut*sigma is a
// product of three 1D factors, and so is each of its periodic images. The sum
// over the 27 images (shifts -L, 0, +L per axis; enough while cut*sigma <= L)
// is therefore the product of three PERIODIZED 1D factors
//   X(i) = sum_{m=-1,0,1} [|d| < cut sigma] exp(-d^2 / 2 sigma^2),  d = x_i - c - m L,
// and the derivative of the image sum with respect to the centre takes
//   X'(i) = sum_m [|d| < cut sigma] exp(-d^2 / 2 sigma^2) d / sigma^2
// in place of X on the differentiated axis (d g / d R = g (r - R) / sigma^2).
// One entry per Gaussian then covers all its images.
__device__ __forceinline__ long gt_row(int ge, int axis, int nmax) { return ((long)ge * 3 + axis) * nmax; }

__global__ void k_gauss_tables(Geo g, Atoms at, double cut, GaussTabs gt) {
    const long total = (long)gt.G * 3 * gt.nmax;
    for (long q = blockIdx.x * (long)blockDim.x + threadIdx.x; q < total; q += (long)gridDim.x * blockDim.x) {
        const int i = (int)(q % gt.nmax);
        const int axis = (int)((q / gt.nmax) % 3);
        const int ge = (int)(q / (3L * gt.nmax));
        const int a = ge >> 1, which = ge & 1;
        const int n = axis == 0 ? g.nx : (axis == 1 ? g.ny : g.nz);
        const double h = axis == 0 ? g.hx : (axis == 1 ? g.hy : g.hz);
        const double L = axis == 0 ? g.lx : (axis == 1 ? g.ly : g.lz);
        const double sg = at.gauss[3 * a + 1 + which];
        const double c = at.w64[3 * a + axis];
        const double rad = cut * sg;
        double v = 0.0, dv = 0.0;
        if (i < n) {
            const double i2s = 0.5 / (sg * sg);
            for (int m = -1; m <= 1; ++m) {
                const double d = i * h - (c + m * L);
                if (fabs(d) < rad) {
                    const double e = exp(-d * d * i2s);
                    v += e;
                    dv += e * d * (2.0 * i2s);
                }
            }
        }
        gt.val[q] = v;
        gt.der[q] = dv;
        {
            const float vh = (float)v, dh = (float)dv;
            gt.vald[q] = make_float2(vh, (float)(v - (double)vh));
            gt.derd[q] = make_float2(dh, (float)(dv - (double)dh));
        }
        if (i == 0) {
            // conservative index window [lo, hi] of the image around c (unwrapped;
            // the other images are its shifts by n)
            const double ih = axis == 0 ? g.ihx : (axis == 1 ? g.ihy : g.ihz);
            int lo = (int)floor((c - rad) * ih) - 1, hi = (int)ceil((c + rad) * ih) + 1;
            if (hi - lo + 1 >= n) { lo = 0; hi = n - 1; }
            gt.win[(ge * 3 + axis) * 2 + 0] = lo;
            gt.win[(ge * 3 + axis) * 2 + 1] = hi;
            if (axis == 0) {
                const double Z = at.gauss[3 * a + 0];
                const double norm = 1.0 / (2.0 * kPi * sg * sg * sqrt(2.0 * kPi * sg * sg));
                const double cf = (which == 0 ? Z : -Z) * norm;
                gt.coef[ge] = cf;
                const float ch = (float)cf;
                gt.coefd[ge] = make_float2(ch, (float)(cf - (double)ch));
            }
        }
    }
}

// does Gaussian ge touch the tile? (window intervals modulo n, per axis)
__device__ __forceinline__ bool span_hits(int lo, int hi, int n, int t0, int t1) {
    return (lo <= t1 && hi >= t0) || (lo + n <= t1 && hi + n >= t0) || (lo - n <= t1 && hi - n >= t0);
}
__device__ __forceinline__ bool gauss_hits_tile(const GaussTabs& gt, int ge, const Tile& t, const Geo& g) {
    const int* w = gt.win + ge * 6;
    return span_hits(w[0], w[1], g.nx, t.i0, t.i1) && span_hits(w[2], w[3], g.ny, t.j0, t.j1) &&
           span_hits(w[4], w[5], g.nz, t.k0, t.k1);
}

// s += a * b with the product formed exactly to ~2^-48 (df64) and the sum
// compensated (Neumaier): the FP32 pipe does the work of an FP64 FMA.
__device__ __forceinline__ void df_acc(float& s, float& c, df a, df b) {
    const float p = a.hi * b.hi;
    float e = fmaf(a.hi, b.hi, -p);
    e = fmaf(a.hi, b.lo, e);
    e = fmaf(a.lo, b.hi, e);
    const float t = s + p;
    const float z = t - s;
    c += ((s - (t - z)) + (p - z)) + e;
    s = t;
}

// ----------------------------------------------------------------- rho
// rho~_ijk = sum_G coef_G X_G(i) Y_G(j) Z_G(k). A tile lists the Gaussians
// whose windows reach it (one integer test per Gaussian), stages X for its 32
// columns and the row weights coef Y(j) Z(k) for its 16 rows, and every point
// then accumulates one compensated product per Gaussian.
constexpr int RB = 64;                  // Gaussians staged at a time

__global__ void __launch_bounds__(TT) k_build_rho(Geo g, GaussTabs gt, double* rho) {
    __shared__ int ent[TT];
    __shared__ df gx[RB][TX];
    __shared__ df wyz[RB][TY * TZ];
    __shared__ int ne;
    const Tile t = make_tile(g);
    const int tx = threadIdx.x % TX, ty = (threadIdx.x / TX) % TY, tz = threadIdx.x / (TX * TY);
    const int i = t.i0 + tx, j = t.j0 + ty, k = t.k0 + tz;
    const bool valid = i < g.nx && j < g.ny && k < g.nz;
    float s = 0.f, c = 0.f;
    for (int g0 = 0; g0 < gt.G; g0 += TT) {
        if (threadIdx.x == 0) ne = 0;
        __syncthreads();
        const int q = g0 + threadIdx.x;
        if (q < gt.G && gauss_hits_tile(gt, q, t, g)) ent[atomicAdd(&ne, 1)] = q;
        __syncthreads();
        const int m = ne;
        for (int e0 = 0; e0 < m; e0 += RB) {
            const int ms = min(RB, m - e0);
            for (int r = threadIdx.x; r < ms * TX; r += TT) {
                const int e = r / TX, ii = t.i0 + r % TX;
                gx[e][r % TX] = ii < g.nx ? as_df(gt.vald[gt_row(ent[e0 + e], 0, gt.nmax) + ii]) : df{0.f, 0.f};
            }
            for (int r = threadIdx.x; r < ms * TY * TZ; r += TT) {
                const int e = r / (TY * TZ), jj = t.j0 + (r % (TY * TZ)) / TZ, kk = t.k0 + r % TZ;
                const int ge = ent[e0 + e];
                df w = {0.f, 0.f};
                if (jj < g.ny && kk < g.nz)
                    w = df_mul(df_mul(as_df(gt.coefd[ge]), as_df(gt.vald[gt_row(ge, 1, gt.nmax) + jj])),
                               as_df(gt.vald[gt_row(ge, 2, gt.nmax) + kk]));
                wyz[e][r % (TY * TZ)] = w;
            }
            __syncthreads();
            if (valid)
                for (int e = 0; e < ms; ++e) df_acc(s, c, gx[e][tx], wyz[e][ty * TZ + tz]);
            __syncthreads();
        }
    }
    if (valid) rho[i + (long)g.nx * (j + (long)g.ny * k)] = (double)s + (double)c;
}

// ----------------------------------------------------------------- switching function in df64
// The table coordinate of a pair, x = (d^2 - q_lo) / dq, is separable:
// d^2 = dx^2 + dy^2 + dz^2, so x = X(i) + Y(j) + Z(k) with X = (dx^2 - q_lo)/dq,
// Y = dy^2/dq, Z = dz^2/dq per column / row of the tile, formed once per
// (tile, atom image) in FP64. Each is kept as an integer part and a fraction
// in [0, 1) held as a df (exact to 2^-48 absolute), so a pair costs two integer
// and two df additions and the interval index needs no FP64 at all.
struct SwCoord {
    int n;      // integer part
    df f;       // fraction in [0, 1)
};

__device__ __forceinline__ SwCoord sw_coord(double v) {
    const double fl = floor(v);
    SwCoord c;
    c.n = (int)fl;
    c.f = df_from(v - fl);
    return c;
}

// interval k and local variable t = 2 (x - k) - 1 in [-1, 1] (as a df) of
// x = n + f, f in [0, 3)
__device__ __forceinline__ int sw_local(int n, df f, df& t) {
    int kk = (int)f.hi;
    kk = kk > 2 ? 2 : kk;
    const float fh = f.hi - (float)kk;      // exact
    const float a = 2.f * fh;
    const float s = a - 1.f;                 // two-sum of a and -1
    const float bb = s - a;
    float e = (a - (s - bb)) + (-1.f - bb);
    e += 2.f * f.lo;
    const float s2 = s + e;                  // renormalise
    const float b2 = s2 - s;
    t.lo = (s - (s2 - b2)) + (e - b2);
    t.hi = s2;
    return n + kk;
}

// acc * t + (ch + cl), all df
__device__ __forceinline__ df df_horner(df acc, df t, float ch, float cl) {
    const float p = acc.hi * t.hi;
    float e = fmaf(acc.hi, t.hi, -p);
    e = fmaf(acc.hi, t.lo, e);
    e = fmaf(acc.lo, t.hi, e);
    const float s = p + ch;
    const float bb = s - p;
    const float err = (p - (s - bb)) + (ch - bb);
    return df_quick(s, err + e + cl);
}

// the polynomial of interval k at t from the packed table (SPLIT df coefficients)
template <int SPLIT>
__device__ __forceinline__ df sw_poly(const float4* __restrict__ tab, int k, df t) {
    float c[16];
    const float4* src = tab + 4 * k;
#pragma unroll
    for (int v = 0; v < 4; ++v) {
        const float4 q = __ldg(src + v);
        c[4 * v] = q.x; c[4 * v + 1] = q.y; c[4 * v + 2] = q.z; c[4 * v + 3] = q.w;
    }
    float v = c[2 * SPLIT + (kSwDeg - SPLIT)];
#pragma unroll
    for (int e = kSwDeg - 1; e >= SPLIT; --e) v = fmaf(v, t.hi, c[2 * SPLIT + (e - SPLIT)]);
    df acc = {v, 0.f};
#pragma unroll
    for (int e = SPLIT - 1; e >= 0; --e) acc = df_horner(acc, t, c[2 * e], c[2 * e + 1]);
    return acc;
}

// ----------------------------------------------------------------- coordinate tables
// One thread per (atom a, image digit m, axis, grid index i): the table coordinate
// of the separable squared distance from grid line i to the image centre
// c = w64[a] + (m - 1) L, as an integer part and a df fraction (sw_coord), and the
// displacement i h - c as a df, all from one FP64 evaluation. The tile kernels
// that stage these per (tile, atom image) then load them instead of computing
// them: on GB300 every FP64 instruction of a warp holds the FP64 pipe for about
// 64 cycles, and the per-tile staging was most of the dielectric kernels' time.
__global__ void k_coord_tables(Geo g, Atoms at, double qlo, double inv_dq, CoordTabs ct) {
    const long total = (long)at.n * 9 * ct.nmax;
    for (long q = blockIdx.x * (long)blockDim.x + threadIdx.x; q < total; q += (long)gridDim.x * blockDim.x) {
        const int i = (int)(q % ct.nmax);
        const long r = q / ct.nmax;
        const int axis = (int)(r % 3), m = (int)((r / 3) % 3), a = (int)(r / 9);
        const int nax = axis == 0 ? g.nx : (axis == 1 ? g.ny : g.nz);
        if (i >= nax) continue;
        const double h = axis == 0 ? g.hx : (axis == 1 ? g.hy : g.hz);
        const double L = axis == 0 ? g.lx : (axis == 1 ? g.ly : g.lz);
        // the same operations, in the same order, as the per-tile staging they replace
        const double c = at.w64[3 * a + axis] + (m - 1) * L;
        const double d = i * h - c;
        const double v = axis == 0 ? (d * d - qlo) * inv_dq : d * d * inv_dq;
        const SwCoord sc = sw_coord(v);
        ct.n[q] = sc.n;
        ct.f[q] = make_float2(sc.f.hi, sc.f.lo);
        if (ct.d) {
            const df dd = df_from(d);
            ct.d[q] = make_float2(dd.hi, dd.lo);
        }
    }
}

__device__ __forceinline__ long ctab_index(const CoordTabs& ct, int a, int im, int axis, int i) {
    const int m = axis == 0 ? im % 3 : (axis == 1 ? (im / 3) % 3 : im / 9);
    return ((long)(a * 3 + m) * 3 + axis) * ct.nmax + i;
}

// ----------------------------------------------------------------- eps, tabulated (df64)
// The same product as k_build_eps, with s from the packed table in df64
// arithmetic (about 120 FP32 instructions per pair instead of 25 FP64 ones).
// Tiles are 32 x 4 x 16 points, each thread taking 4 points along z, so the
// per-(tile, atom image) staging (table coordinates loaded from the coordinate
// tables) is shared by 2048 points. The tile first collects its atom images
// within reach (r0 + 6w: s == 1 beyond) into one list, processed when full or at
// the end, in batches of EB images.
constexpr int EZ = 16;                  // z extent of the tabulated-eps tiles
constexpr int EB = 32;                  // atom images staged at a time
constexpr int ACHS = 8;                 // atoms culled per pass (at most 216 images)
constexpr int ECAP = 640;               // image list capacity
constexpr int NS = TX + TY + EZ;        // staged columns, rows and planes

__device__ __forceinline__ Tile make_tile_ez(const Geo& g) {
    Tile t;
    t.i0 = blockIdx.x * TX; t.j0 = blockIdx.y * TY; t.k0 = blockIdx.z * EZ;
    t.i1 = min(t.i0 + TX, g.nx) - 1; t.j1 = min(t.j0 + TY, g.ny) - 1; t.k1 = min(t.k0 + EZ, g.nz) - 1;
    t.bx0 = (float)t.i0 * g.hxf; t.bx1 = (float)t.i1 * g.hxf;   // FP32: the culling keeps a margin
    t.by0 = (float)t.j0 * g.hyf; t.by1 = (float)t.j1 * g.hyf;
    t.bz0 = (float)t.k0 * g.hzf; t.bz1 = (float)t.k1 * g.hzf;
    return t;
}

__global__ void __launch_bounds__(TT) k_build_eps_tab(Geo g, Atoms at, DielParams p, SwTables tb, CoordTabs ct,
                                                      double* eps64, double* pe64, float* eps32,
                                                      double* plane_max) {
    __shared__ int eai[ECAP][2];                 // (atom, image) of each surviving image
    __shared__ int cn[EB][NS];
    __shared__ df cf[EB][NS];
    __shared__ unsigned long long pmax[EZ];      // the tile's max of eps - 1 per plane (bits of a double >= 0)
    __shared__ int ne;
    const Tile t = make_tile_ez(g);
    int tx, ty, tz;
    compact_point(threadIdx.x >> 5, threadIdx.x & 31, tx, ty, tz);
    const int i = t.i0 + tx, j = t.j0 + ty;
    bool live[4];
    df P[4];
#pragma unroll
    for (int r = 0; r < 4; ++r) {
        live[r] = i < g.nx && j < g.ny && t.k0 + tz + 4 * r < g.nz;
        P[r] = df{1.f, 0.f};
    }
    const float tiny = p.tinyf;
    const float reach = p.reachf + kMargin;
    const float dq = tb.s_dqf, qlo = tb.s_qlof;
    const float r0f = p.r0f, iwf = p.iwf;
    // how many atom images reach the tile: when the list holds them all (the usual
    // case), one pass collects them and one flush processes them, instead of a
    // barrier pair per chunk of ACHS atoms
    if (threadIdx.x == 0) ne = 0;
    if (threadIdx.x < EZ) pmax[threadIdx.x] = 0ull;
    __syncthreads();
    for (int q = threadIdx.x; q < at.n * 27; q += TT) {
        float fx, fy, fz;
        image32(at.w32, q / 27, q % 27, g, fx, fy, fz);
        if (box_d2(t, fx, fy, fz) < reach * reach) atomicAdd(&ne, 1);
    }
    __syncthreads();
    const int chunk = ne <= ECAP ? max(at.n, 1) : ACHS;
    const int flush_at = ECAP - chunk * 27;
    __syncthreads();
    if (threadIdx.x == 0) ne = 0;
    __syncthreads();
    for (int a0 = 0; a0 < at.n; a0 += chunk) {
        const int na = min(chunk, at.n - a0);
        for (int q = threadIdx.x; q < na * 27; q += TT) {
            const int a = a0 + q / 27, im = q % 27;
            float fx, fy, fz;
            image32(at.w32, a, im, g, fx, fy, fz);
            if (box_d2(t, fx, fy, fz) < reach * reach) {
                const int s = atomicAdd(&ne, 1);
                eai[s][0] = a;
                eai[s][1] = im;
            }
        }
        __syncthreads();
        const int m = ne;
        if (m > flush_at || a0 + chunk >= at.n) {
            for (int e0 = 0; e0 < m; e0 += EB) {
                const int ms = min(EB, m - e0);
                for (int r = threadIdx.x; r < ms * NS; r += TT) {
                    const int e = r / NS, c = r % NS;
                    // grid index of this staged column / row / plane, clamped on ragged tiles
                    // (the clamped values are never read: those points are not live)
                    int axis, gi;
                    if (c < TX) { axis = 0; gi = min(t.i0 + c, g.nx - 1); }
                    else if (c < TX + TY) { axis = 1; gi = min(t.j0 + c - TX, g.ny - 1); }
                    else { axis = 2; gi = min(t.k0 + c - TX - TY, g.nz - 1); }
                    const long q = ctab_index(ct, eai[e0 + e][0], eai[e0 + e][1], axis, gi);
                    cn[e][c] = __ldg(ct.n + q);
                    cf[e][c] = as_df(__ldg(ct.f + q));
                }
                __syncthreads();
                if (live[0] || live[1] || live[2] || live[3]) {
                    for (int e = 0; e < ms; ++e) {
                        const int nxy = cn[e][tx] + cn[e][TX + ty];
                        if (nxy >= kSwNI) continue;                  // already beyond r0 + 6w
                        const df fxy = df_add(cf[e][tx], cf[e][TX + ty]);
#pragma unroll
                        for (int r = 0; r < 4; ++r) {
                            if (!live[r]) continue;
                            const int cz = TX + TY + tz + 4 * r;
                            const int n = nxy + cn[e][cz];
                            if (n >= kSwNI) continue;               // d >= r0 + 6w: s == 1
                            df tl;
                            const int kq = sw_local(n, df_add(fxy, cf[e][cz]), tl);
                            if (kq >= kSwNI) continue;
                            df sv;
                            if (kq < 0) {
                                // d < r0 - 4w: s < 8e-9, FP32 erfc (relative error ~1e-6 of s)
                                const float qq = ((float)kq + 0.5f * (tl.hi + 1.f)) * dq + qlo;   // x = kq + (t + 1) / 2
                                const float d = sqrtf(fmaxf(qq, 0.f));
                                sv.hi = 0.5f * erfcf((r0f - d) * iwf);
                                sv.lo = 0.f;
                            } else {
                                sv = sw_poly<kSwSplitS>(tb.s32, kq, tl);
                            }
                            P[r] = df_mul(P[r], sv);
                            if (P[r].hi < tiny) live[r] = false;
                        }
                    }
                }
                __syncthreads();
            }
            if (threadIdx.x == 0) ne = 0;
        }
        __syncthreads();
    }
#pragma unroll
    for (int r = 0; r < 4; ++r) {
        const int k = t.k0 + tz + 4 * r;
        if (i < g.nx && j < g.ny && k < g.nz) {
            const long idx = i + (long)g.nx * (j + (long)g.ny * k);
            const double pe = (p.eps0 - 1.0) * df_to(P[r]);
            const double e = 1.0 + pe;
            eps64[idx] = e;
            if (pe64) pe64[idx] = pe;
            if (eps32) eps32[idx] = split_to_float2(e).x;          // the rounded float, by integer instructions
            if (plane_max) atomicMax(&pmax[tz + 4 * r], (unsigned long long)__double_as_longlong(e - 1.0));
        }
    }
    // the per-plane maxima of eps - 1 (the dry-plane test): nonnegative doubles
    // order as their bit patterns, so the maxima are integer atomics
    if (plane_max) {
        __syncthreads();
        if (threadIdx.x < EZ && t.k0 + (int)threadIdx.x < g.nz)
            atomicMax(reinterpret_cast<unsigned long long*>(plane_max + t.k0 + threadIdx.x), pmax[threadIdx.x]);
    }
}

// ----------------------------------------------------------------- the per-point force weight
// W_i of the dielectric force sums S_a = sum_i W_i (d eps_i / d R_a) / pv_i:
// (1/2) sum over the six faces of i of (grad_f phi)^2 (the face means of Eq. 3
// split between the two points of each face) times the per-point factor pv_i,
// or, when the caller gives a per-point weight wext (the sixth-order forces,
// where the adjoint supplies it), wext_i times pv_i.
__device__ __forceinline__ double force_weight(const Geo& g, const double* phi, const double* wext, double pv, int i,
                                               int j, int k, long c) {
    if (pv == 0.0) return 0.0;
    if (wext) return wext[c] * pv;
    const long pl = plane_of(g.nx, g.ny);
    const long xp = c + (i == g.nx - 1 ? 1 - g.nx : 1), xm = c - (i == 0 ? 1 - g.nx : 1);
    const long yp = c + (j == g.ny - 1 ? (1 - g.ny) * (long)g.nx : g.nx);
    const long ym = c - (j == 0 ? (1 - g.ny) * (long)g.nx : g.nx);
    const long zp = c + (k == g.nz - 1 ? (1 - g.nz) * pl : pl);
    const long zm = c - (k == 0 ? (1 - g.nz) * pl : pl);
    const double p0 = phi[c];
    const double ax = phi[xp] - p0, bx = p0 - phi[xm];
    const double ay = phi[yp] - p0, by = p0 - phi[ym];
    const double az = phi[zp] - p0, bz = p0 - phi[zm];
    return ((ax * ax + bx * bx) * g.c2x + (ay * ay + by * by) * g.c2y + (az * az + bz * bz) * g.c2z) * pv;
}

// The same weight in df64 on the FP32 pipe, from phi as float pairs (a face
// difference of two pairs keeps the pair representation's 2^-48 of phi; the
// FP64 version spends about twenty FP64-pipe instructions per point). Returns -W.
__device__ __forceinline__ df neg_force_weight_df(const Geo& g, const float2* phid, const double* wext, double pv,
                                                  int i, int j, int k, long c, df c2x, df c2y, df c2z) {
    if ((__double_as_longlong(pv) & 0x7fffffffffffffffll) == 0) return df{0.f, 0.f};
    const df pvd = df_from(pv);
    df W;
    if (wext) {
        W = df_mul(df_from(wext[c]), pvd);
    } else {
        const long pl = plane_of(g.nx, g.ny);
        const long xp = c + (i == g.nx - 1 ? 1 - g.nx : 1), xm = c - (i == 0 ? 1 - g.nx : 1);
        const long yp = c + (j == g.ny - 1 ? (1 - g.ny) * (long)g.nx : g.nx);
        const long ym = c - (j == 0 ? (1 - g.ny) * (long)g.nx : g.nx);
        const long zp = c + (k == g.nz - 1 ? (1 - g.nz) * pl : pl);
        const long zm = c - (k == 0 ? (1 - g.nz) * pl : pl);
        const df p0 = as_df(phid[c]), np0 = df{-p0.hi, -p0.lo};
        auto sq2 = [&](long up, long dn) {
            const df a = df_add(as_df(phid[up]), np0);
            const float2 d = phid[dn];
            const df b = df_add(p0, df{-d.x, -d.y});
            return df_add(df_mul(a, a), df_mul(b, b));
        };
        W = df_mul(df_add(df_add(df_mul(sq2(xp, xm), c2x), df_mul(sq2(yp, ym), c2y)), df_mul(sq2(zp, zm), c2z)), pvd);
    }
    return df{-W.hi, -W.lo};
}

// ----------------------------------------------------------------- eps force, tabulated (df64)
// The same sum as k_forces_eps with h = s'/(s d) from the packed table in df64
// arithmetic, on 32 x 4 x 16 tiles. One warp per (tile, atom image): it
// loads the table coordinates and displacements of the tile's 32 columns, 4
// rows and 16 planes from the coordinate tables (FP64-exact, as df), runs over
// the 2048 points with compensated FP32 sums, and reduces across the warp in
// df; the CTA then turns every image's sum into FP64 atomics with full warps.
constexpr int ECAPF = 384;              // image list capacity of the force kernel

__global__ void __launch_bounds__(TT) k_forces_eps_tab(Geo g, Atoms at, DielParams p, SwTables tb, CoordTabs ct,
                                                       const float2* phid, const double* wext, const double* pe64,
                                                       double* S) {
    __shared__ df Ws[TX * TY * EZ];              // index tx + TX (ty + TY z)
    __shared__ df eres[ECAPF][3];                // each image's sum, converted to FP64 by a full warp
    __shared__ int eatom[ECAPF];
    __shared__ int eimg[ECAPF];
    __shared__ int wn[TT / 32][NS];
    __shared__ df wf[TT / 32][NS];
    __shared__ df wd[TT / 32][NS];
    __shared__ int ne;
    const Tile t = make_tile_ez(g);
    const float rcf = p.rcutf + kMargin;
    // the tile's atom images within rcut; the W field is built only if there is one
    if (threadIdx.x == 0) ne = 0;
    __syncthreads();
    {
        const float4* w32 = at.w32;
        for (int q = threadIdx.x; q < at.n * 27; q += TT) {
            const int a = q / 27, im = q % 27;
            float fx, fy, fz;
            image32(w32, a, im, g, fx, fy, fz);
            if (box_d2(t, fx, fy, fz) < rcf * rcf) atomicAdd(&ne, 1);
        }
    }
    __syncthreads();
    if (ne == 0) return;
    {
        const df c2x = df_from(g.c2x), c2y = df_from(g.c2y), c2z = df_from(g.c2z);
        for (int q = threadIdx.x; q < TX * TY * EZ; q += TT) {
            const int tx = q % TX, ty = (q / TX) % TY, tz = q / (TX * TY);
            const int i = t.i0 + tx, j = t.j0 + ty, k = t.k0 + tz;
            df w = df{0.f, 0.f};
            if (i < g.nx && j < g.ny && k < g.nz) {
                const long c = i + (long)g.nx * (j + (long)g.ny * k);
                w = neg_force_weight_df(g, phid, wext, pe64[c], i, j, k, c, c2x, c2y, c2z);
            }
            Ws[q] = w;         // sign of c = -W h folded in
        }
    }
    const float rc2f = p.rc2f;
    const float dq = tb.h_dqf, qlo = tb.h_qlof;
    const float r0f = p.r0f, iwf = p.iwf, spf_norm = p.spnf;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    // the count above sizes the passes: when the list holds every image, one pass
    // collects them and one flush processes them
    const int chunk = ne <= ECAPF ? max(at.n, 1) : ACHS;
    const int flush_at = ECAPF - chunk * 27;
    __syncthreads();
    if (threadIdx.x == 0) ne = 0;
    __syncthreads();
    for (int a0 = 0; a0 < at.n; a0 += chunk) {
        const int na = min(chunk, at.n - a0);
        for (int q = threadIdx.x; q < na * 27; q += TT) {
            const int a = a0 + q / 27, im = q % 27;
            float fx, fy, fz;
            image32(at.w32, a, im, g, fx, fy, fz);
            if (box_d2(t, fx, fy, fz) < rcf * rcf) {
                const int s = atomicAdd(&ne, 1);
                eatom[s] = a;
                eimg[s] = im;
            }
        }
        __syncthreads();
        const int m = ne;
        if (m > flush_at || a0 + chunk >= at.n) {
            for (int e = warp; e < m; e += TT / 32) {
                for (int c = lane; c < NS; c += 32) {
                    // grid index of this column / row / plane, clamped on ragged tiles (never read there)
                    int axis, gi;
                    if (c < TX) { axis = 0; gi = min(t.i0 + c, g.nx - 1); }
                    else if (c < TX + TY) { axis = 1; gi = min(t.j0 + c - TX, g.ny - 1); }
                    else { axis = 2; gi = min(t.k0 + c - TX - TY, g.nz - 1); }
                    const long q = ctab_index(ct, eatom[e], eimg[e], axis, gi);
                    wn[warp][c] = __ldg(ct.n + q);
                    wf[warp][c] = as_df(__ldg(ct.f + q));
                    wd[warp][c] = as_df(__ldg(ct.d + q));
                }
                __syncwarp();
                float sx = 0.f, cx = 0.f, sy = 0.f, cy = 0.f, sz = 0.f, cz = 0.f;
                for (int blk = 0; blk < 4 * 16; ++blk) {
                    int tx, ty, tz;
                    compact_point(blk & 15, lane, tx, ty, tz);
                    tz += 4 * (blk >> 4);
                    if (t.i0 + tx >= g.nx || t.j0 + ty >= g.ny || t.k0 + tz >= g.nz) continue;
                    const int n = wn[warp][tx] + wn[warp][TX + ty] + wn[warp][TX + TY + tz];
                    df ratio;   // s'(d) / (s(d) d)
                    if (n >= kSwNI) {
                        // d >= r0 + 3.5w (the integer parts of the table coordinate alone
                        // pass its end): culled at rcut on the FP32 distance; inside it
                        // u >= 3.5 and s = 1 - erfc(u)/2 is 1 to 3.7e-7, so the ratio is
                        // s'/d in FP32 (the pair is below 5e-6 of one at the switching radius)
                        const float dx = wd[warp][tx].hi, dy = wd[warp][TX + ty].hi, dz = wd[warp][TX + TY + tz].hi;
                        const float qq = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
                        if (!(qq < rc2f)) continue;
                        const float rs = rsqrtf(qq);          // 1/d
                        const float uf = (qq * rs - r0f) * iwf;
                        ratio.hi = spf_norm * exp2f(-1.44269504f * uf * uf) * rs;   // s'/d = spn exp(-u^2)/d
                        ratio.lo = 0.f;
                        const df c = df_mul(Ws[tx + TX * (ty + TY * tz)], ratio);
                        df_acc(sx, cx, c, wd[warp][tx]);
                        df_acc(sy, cy, c, wd[warp][TX + ty]);
                        df_acc(sz, cz, c, wd[warp][TX + TY + tz]);
                        continue;
                    }
                    const df f = df_add(df_add(wf[warp][tx], wf[warp][TX + ty]), wf[warp][TX + TY + tz]);
                    df tl;
                    const int kq = sw_local(n, f, tl);
                    if (kq >= 0 && kq < kSwNI) {
                        ratio = sw_poly<kSwSplitH>(tb.h32, kq, tl);
                    } else {
                        // |u| > 3.5: the pair is below 5e-6 of one at the switching radius; FP32
                        const float qq = ((float)kq + 0.5f * (tl.hi + 1.f)) * dq + qlo;
                        if (!(qq < rc2f && qq > 0.f)) continue;
                        const float d_ = sqrtf(qq);
                        const float uf = (d_ - r0f) * iwf;
                        const float sf = 0.5f * erfcf(-uf);
                        const float spf = spf_norm * expf(-uf * uf);
                        ratio.hi = spf / (sf * d_);
                        ratio.lo = 0.f;
                    }
                    const df c = df_mul(Ws[tx + TX * (ty + TY * tz)], ratio);
                    df_acc(sx, cx, c, wd[warp][tx]);
                    df_acc(sy, cy, c, wd[warp][TX + ty]);
                    df_acc(sz, cz, c, wd[warp][TX + TY + tz]);
                }
                warp_sum_df(sx, cx); warp_sum_df(sy, cy); warp_sum_df(sz, cz);
                if (lane == 0) {
                    eres[e][0] = df{sx, cx};
                    eres[e][1] = df{sy, cy};
                    eres[e][2] = df{sz, cz};
                }
                __syncwarp();
            }
            __syncthreads();
            // the images' sums to FP64 and into S: one entry per thread, so each FP64
            // instruction runs with a full warp (a warp instruction holds the FP64 pipe
            // for as long whether one lane or 32 are active)
            for (int e = threadIdx.x; e < 3 * m; e += TT) {
                const int ee = e / 3, comp = e % 3;
                const double v = (double)eres[ee][comp].hi + (double)eres[ee][comp].lo;
                if (v != 0.0) atomicAdd(&S[3 * eatom[ee] + comp], v);
            }
            __syncthreads();
            if (threadIdx.x == 0) ne = 0;
        }
        __syncthreads();
    }
}

dim3 tile_grid_ez(const Geo& g) {
    return dim3((g.nx + TX - 1) / TX, (g.ny + TY - 1) / TY, (g.nz + EZ - 1) / EZ);
}

// ----------------------------------------------------------------- eps, Eq. 9-10 and Eq. 19 (dummy density)
// gamma(r) = sum over atoms and every periodic image of exp(-(d - rvdw_a)) (Eq. 9),
// taken over the images within p.rcut: the host picks that radius so that a
// proven bound on the dropped tail is below the requested tolerance (1e-13 by
// default), which is why the image range p.mx, p.my, p.mz may span several cells.
// eps = 1 + (eps0 - 1)/2 (1 + (1 - gamma^(2b))/(1 + gamma^(2b))) = 1 + (eps0 - 1)/(1 + gamma^(2b))
// (Eq. 10), and the factor d eps/d gamma = -(eps0 - 1) 2b gamma^(2b-1)/(1 + gamma^(2b))^2 of
// the atomic derivative d eps/d R_a = (d eps/d gamma) exp(-(d - rvdw)) (r - R_a)/d,
// Eq. 12 with the sign that differentiating Eq. 9-10 gives (moving an atom towards r
// raises gamma and lowers eps).
// Kind 2 (Eq. 19): an atom with z_a <= zlim contributes, at points with z < z_a (both
// inside the cell), exp(+(d - rvdw)) from its nearest image with no cut-off; once such
// an exponent reaches esat, eps = 1 and d eps/d gamma = 0 there ("saturated"). FP64.
//
// The candidates (atom a, image n) are numbered q = a * nimg + im and culled against
// the tile's box MAXE at a time; the survivors go to shared memory.

__device__ __forceinline__ double min_image(double v, double L) { return v - L * rint(v / L); }

// image `im` of the (2 mx + 1)(2 my + 1)(2 mz + 1) images of wrapped atom a
__device__ __forceinline__ void gimage32(const float4* w32, int a, int im, const Geo& g, const DielParams& p,
                                         float& cx, float& cy, float& cz) {
    const int nxi = 2 * p.mx + 1, nyi = 2 * p.my + 1;
    const float4 w = w32[a];
    cx = w.x + (float)(im % nxi - p.mx) * g.lxf;
    cy = w.y + (float)((im / nxi) % nyi - p.my) * g.lyf;
    cz = w.z + (float)(im / (nxi * nyi) - p.mz) * g.lzf;
}

__device__ __forceinline__ void gimage64(const double* w64, int a, int im, const Geo& g, const DielParams& p,
                                         double& cx, double& cy, double& cz) {
    const int nxi = 2 * p.mx + 1, nyi = 2 * p.my + 1;
    cx = w64[3 * a + 0] + (im % nxi - p.mx) * g.lx;
    cy = w64[3 * a + 1] + ((im / nxi) % nyi - p.my) * g.ly;
    cz = w64[3 * a + 2] + (im / (nxi * nyi) - p.mz) * g.lz;
}

// cull candidates [q0, q0 + MAXE) of the tile into ec / eatom (ne survivors)
__device__ __forceinline__ void cull_gamma(const Tile& t, const Geo& g, const Atoms& at, const DielParams& p,
                                           const double* rvdw, long q0, long nq, int nimg, float rcf, bool eq19,
                                           double (*ec)[5], int* eatom, int* ne) {
    for (long q = q0 + threadIdx.x; q < min(q0 + MAXE, nq); q += TT) {
        const int a = (int)(q / nimg), im = (int)(q % nimg);
        float fx, fy, fz;
        gimage32(at.w32, a, im, g, p, fx, fy, fz);
        if (box_d2(t, fx, fy, fz) < rcf * rcf) {
            const int s = atomicAdd(ne, 1);
            gimage64(at.w64, a, im, g, p, ec[s][0], ec[s][1], ec[s][2]);
            ec[s][3] = rvdw[a];
            const double za = at.w64[3 * a + 2];
            ec[s][4] = (eq19 && za <= p.zlim) ? za : -1.0;
            if (eatom) eatom[s] = a;
        }
    }
}

__global__ void __launch_bounds__(TT) k_build_eps_gamma(Geo g, Atoms at, DielParams p, const double* rvdw,
                                                        double* eps64, double* fe64, float* eps32) {
    __shared__ double ec[MAXE][5];              // image centre, rvdw, z of the atom in the cell (kind 2 lower) or -1
    __shared__ int ne;
    const Tile t = make_tile(g);
    int tx, ty, tz;
    compact_point(threadIdx.x >> 5, threadIdx.x & 31, tx, ty, tz);
    const int i = t.i0 + tx, j = t.j0 + ty, k = t.k0 + tz;
    const bool valid = i < g.nx && j < g.ny && k < g.nz;
    const double x = i * g.hx, y = j * g.hy, z = k * g.hz;
    const double rc2 = p.rcut * p.rcut;
    const float rcf = p.rcutf + kMargin;
    const bool eq19 = p.kind == 2;
    const int nimg = (2 * p.mx + 1) * (2 * p.my + 1) * (2 * p.mz + 1);
    const long nq = (long)at.n * nimg;
    double gam = 0.0;
    bool sat = false;
    for (long q0 = 0; q0 < nq; q0 += MAXE) {
        if (threadIdx.x == 0) ne = 0;
        __syncthreads();
        cull_gamma(t, g, at, p, rvdw, q0, nq, nimg, rcf, eq19, ec, nullptr, &ne);
        __syncthreads();
        const int m = ne;
        if (valid)
            for (int e = 0; e < m; ++e) {
                if (z < ec[e][4]) continue;                 // below a lower atom: the growing term instead
                const double dx = x - ec[e][0], dy = y - ec[e][1], dz = z - ec[e][2];
                const double d2 = dx * dx + dy * dy + dz * dz;
                if (d2 < rc2) gam += exp(ec[e][3] - sqrt(d2));
            }
        __syncthreads();
    }
    if (eq19 && valid)
        for (int a = 0; a < at.n && !sat; ++a) {
            const double za = at.w64[3 * a + 2];
            if (za > p.zlim || !(z < za)) continue;
            const double dx = min_image(x - at.w64[3 * a], g.lx), dy = min_image(y - at.w64[3 * a + 1], g.ly);
            const double dz = min_image(z - za, g.lz);
            const double ex = sqrt(dx * dx + dy * dy + dz * dz) - rvdw[a];
            if (ex >= p.esat) sat = true;
            else gam += exp(ex);
        }
    if (valid) {
        const long idx = i + (long)g.nx * (j + (long)g.ny * k);
        double e = p.eps0, fe = 0.0;
        if (sat) {
            e = 1.0;
        } else if (gam > 0.0) {
            const double gb = exp(p.beta2 * log(gam));          // gamma^(2 beta)
            const double den = 1.0 + gb;
            e = 1.0 + (p.eps0 - 1.0) / den;
            fe = -(p.eps0 - 1.0) * p.beta2 * gb / (gam * den * den);
        }
        eps64[idx] = e;
        if (fe64) fe64[idx] = fe;
        if (eps32) eps32[idx] = (float)e;
    }
}

// S_a = sum_i W_i (d eps/d gamma)_i (d gamma_i / d R_a), with W_i = (1/2) sum over the six
// faces of i of (grad_f phi)^2, so that G_eps_a = -h^3/(8 pi) S_a (applied in
// k_forces_finish). d gamma/d R_a: exp(-(d - rvdw)) (r - R_a)/d per decaying image
// term, -exp(d - rvdw) (r - R_a)/d for a growing (kind 2) term. One warp per
// (atom, image) entry, and for kind 2 one warp per lower atom, over the tile's 512
// points; FP64.
__global__ void __launch_bounds__(TT) k_forces_eps_gamma(Geo g, Atoms at, DielParams p, const double* rvdw,
                                                         const double* phi, const double* wext, const double* fe64,
                                                         double* S) {
    __shared__ double ec[MAXE][5];
    __shared__ int eatom[MAXE];
    __shared__ double Ws[TT];
    __shared__ int ne;
    const Tile t = make_tile(g);
    const bool eq19 = p.kind == 2;
    int any = 0;
    {
        const int tx = threadIdx.x % TX, ty = (threadIdx.x / TX) % TY, tz = threadIdx.x / (TX * TY);
        const int i = t.i0 + tx, j = t.j0 + ty, k = t.k0 + tz;
        double W = 0.0;
        if (i < g.nx && j < g.ny && k < g.nz) {
            const long c = i + (long)g.nx * (j + (long)g.ny * k);
            W = force_weight(g, phi, wext, fe64[c], i, j, k, c);
        }
        Ws[threadIdx.x] = W;   // index tx + TX (ty + TY tz)
        any = W != 0.0;
    }
    if (__syncthreads_or(any) == 0) return;                // every point of the tile has d eps/d gamma = 0
    const double rc2 = p.rcut * p.rcut;
    const float rcf = p.rcutf + kMargin;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int nimg = (2 * p.mx + 1) * (2 * p.my + 1) * (2 * p.mz + 1);
    const long nq = (long)at.n * nimg;
    for (long q0 = 0; q0 < nq; q0 += MAXE) {
        if (threadIdx.x == 0) ne = 0;
        __syncthreads();
        cull_gamma(t, g, at, p, rvdw, q0, nq, nimg, rcf, eq19, ec, eatom, &ne);
        __syncthreads();
        const int m = ne;
        for (int e = warp; e < m; e += TT / 32) {
            const double cx = ec[e][0], cy = ec[e][1], cz = ec[e][2], rv = ec[e][3], zl = ec[e][4];
            double fx = 0.0, fy = 0.0, fz = 0.0;
            for (int blk = 0; blk < 16; ++blk) {
                int tx, ty, tz;
                compact_point(blk, lane, tx, ty, tz);
                const int i = t.i0 + tx, j = t.j0 + ty, k = t.k0 + tz;
                if (i >= g.nx || j >= g.ny || k >= g.nz) continue;
                const double W = Ws[tx + TX * (ty + TY * tz)];
                if (W == 0.0) continue;
                if (k * g.hz < zl) continue;                 // growing branch of a lower atom
                const double dx = i * g.hx - cx, dy = j * g.hy - cy, dz = k * g.hz - cz;
                const double d2 = dx * dx + dy * dy + dz * dz;
                if (!(d2 < rc2 && d2 > 0.0)) continue;
                const double d = sqrt(d2);
                const double c = W * exp(rv - d) / d;
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
    if (eq19)
        for (int a = warp; a < at.n; a += TT / 32) {
            const double za = at.w64[3 * a + 2];
            if (za > p.zlim || t.k0 * g.hz >= za) continue;  // no point of the tile is below the atom
            const double ax = at.w64[3 * a], ay = at.w64[3 * a + 1], rv = rvdw[a];
            double fx = 0.0, fy = 0.0, fz = 0.0;
            for (int blk = 0; blk < 16; ++blk) {
                int tx, ty, tz;
                compact_point(blk, lane, tx, ty, tz);
                const int i = t.i0 + tx, j = t.j0 + ty, k = t.k0 + tz;
                if (i >= g.nx || j >= g.ny || k >= g.nz) continue;
                const double W = Ws[tx + TX * (ty + TY * tz)];
                const double z = k * g.hz;
                if (W == 0.0 || !(z < za)) continue;
                const double dx = min_image(i * g.hx - ax, g.lx), dy = min_image(j * g.hy - ay, g.ly);
                const double dz = min_image(z - za, g.lz);
                const double d = sqrt(dx * dx + dy * dy + dz * dz);
                if (!(d > 0.0) || d - rv >= p.esat) continue;
                const double c = -W * exp(d - rv) / d;
                fx += c * dx; fy += c * dy; fz += c * dz;
            }
            fx = warp_sum(fx); fy = warp_sum(fy); fz = warp_sum(fz);
            if (lane == 0) {
                if (fx != 0.0) atomicAdd(&S[3 * a + 0], fx);
                if (fy != 0.0) atomicAdd(&S[3 * a + 1], fy);
                if (fz != 0.0) atomicAdd(&S[3 * a + 2], fz);
            }
        }
}

// ----------------------------------------------------------------- eps, Eq. 9-10 and Eq. 19 in df64
// The sums of k_build_eps_gamma and k_forces_eps_gamma with every (point, atom
// image) pair in df64 on the FP32 pipe, on 32 x 4 x 16 tiles. A pair costs a
// squared distance from the per-atom displacement tables (FP64 differences kept
// as float pairs, so no pair needs an FP64 instruction), its df square root, and
// the exponential by a table-driven method (Tang, ACM TOMS 15, 1989): with
// k = rint(256 d) and r = d - k/256, |r| <= 1/512,
//   exp(-d) = exp(-floor(k/256)) exp(-(k mod 256)/256) exp(-r),
// the first factor from a row staged per atom image (already times the atom's
// exp(rvdw)), the second from a 256-entry table, both as float pairs, and exp(-r)
// from its Taylor series to r^5 (the remainder is below 3e-19), whose
// 1 - r + r^2/2 is formed in df and the rest (below 1.3e-9) in FP32. A growing
// Eq. 19 term exp(d - rvdw) takes the same steps with exp(+n), exp(+j/256) and
// the series of exp(+r). A pair's error is a few units of 2^-48 relative to its
// distance and its term.
constexpr int GCAP = 3072;              // image list capacity (build)
constexpr int GCAPF = 2048;             // image list capacity (force)
constexpr int GB = 32;                  // atom images staged at a time (build)

__device__ __forceinline__ long gtab_index(const GammaTabs& gt, int a, int n, int axis, int i) {
    return (((long)a * (2 * gt.m + 1) + n + gt.m) * 3 + axis) * gt.nmax + i;
}

// exp(-x) (kNeg) or exp(+x) of x >= 0 given as df, times the staged row
// row[n] = c exp(-+n) of the term's factor c; tab[j] = exp(-+j/256); n returns
// the row used (the integer part of x, to within 1/512)
template <bool kNeg>
__device__ __forceinline__ df exp_tab(df x, const df* row, const df* tab, int& n) {
    const int k = __float2int_rn(x.hi * 256.f);
    n = min(k >> 8, kGT1 - 1);
    const float rh = fmaf((float)k, -0.00390625f, x.hi);   // exact: |rh| <= 1/512 on x.hi's grid
    const float s = rh + x.lo;                               // r = s + rl exactly (two-sum)
    const float bb = s - rh;
    const float rl = (rh - (s - bb)) + (x.lo - bb);
    const float r2 = s * s;
    const float r2e = fmaf(s, s, -r2) + 2.f * s * rl;       // r^2 = r2 + r2e
    const float h = 0.5f * r2;
    float u, ue, c;
    if constexpr (kNeg) {
        u = h - s;                                           // |s| >= |h|: ue is the exact error
        ue = (h - (u + s)) - rl;
        c = r2 * s * fmaf(s, fmaf(s, -1.f / 120.f, 1.f / 24.f), -1.f / 6.f);
    } else {
        u = h + s;
        ue = (h - (u - s)) + rl;
        c = r2 * s * fmaf(s, fmaf(s, 1.f / 120.f, 1.f / 24.f), 1.f / 6.f);
    }
    const float lo = (ue + 0.5f * r2e) + c;
    const float ph = 1.f + u;
    const float pl = (u - (ph - 1.f)) + lo;
    return df_mul(df_mul(row[n], tab[k & 255]), df{ph, pl});
}

// sqrt(q) as df for q.hi > 0 (a Newton step on the FP32 estimate, then the df
// correction); y returns 1/sqrt(q.hi) to about 2^-23
__device__ __forceinline__ df df_sqrt(df q, float& y) {
    const float y0 = rsqrtf(q.hi);
    const float s0 = q.hi * y0;
    const float s = fmaf(fmaf(-s0, s0, q.hi), 0.5f * y0, s0);
    y = y0 * fmaf(-0.5f * q.hi * y0, y0, 1.5f);
    const float e = fmaf(-s, s, q.hi) + q.lo;
    return df_quick(s, 0.5f * e * y);
}

// Far pairs in FP32. d = sqrt(q) to about an ulp, y = 1/d to about 2^-23 (a
// Newton step on each hardware estimate)
__device__ __forceinline__ float sqrt_f32(float q, float& y) {
    const float y0 = rsqrtf(q);
    const float s0 = q * y0;
    y = y0 * fmaf(-0.5f * q * y0, y0, 1.5f);
    return fmaf(fmaf(-s0, s0, q), 0.5f * y0, s0);
}

// exp(rvdw - d) = 2^(l2a - d log2(e)) of a far pair by the hardware base-2
// exponential (relative error about 2^-22); with d from an FP32 squared distance
// and the FP32 argument the term carries a relative error of a few 1e-6 at 40 A
__device__ __forceinline__ float exp_far(float d, float l2a) {
    float v;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(v) : "f"(fmaf(d, -1.44269504f, l2a)));
    return v;
}

// 1/d as df from d and an estimate y of 1/d.hi (one Newton step)
__device__ __forceinline__ df df_recip(df d, float y) {
    const float p = d.hi * y;
    const float pe = fmaf(d.hi, y, -p);
    const float del = ((1.f - p) - pe) - d.lo * y;
    return df_quick(y, y * del);
}

// (s, c) += v as a df sum, renormalised after every term so that c stays below
// half an ulp of s: a term far below s still lands in c with c's relative
// precision (an unrenormalised error term grows with the terms it absorbs, and
// terms below its half ulp are lost, all in one direction)
__device__ __forceinline__ void df_add_to(float& s, float& c, df v) {
    const float t = s + v.hi;
    const float z = t - s;
    float e = (s - (t - z)) + (v.hi - z);
    e += c + v.lo;
    s = t + e;
    c = e - (s - t);
}

// A point's terms span 1 down to 1e-17: those from rows below kNear (d < ~10 A,
// a few dozen per point) go into an FP64 sum, the rest (at most ~1e-3 of gamma)
// into a df sum of their own, whose half ulp then sits far below any term that
// matters. One df sum for all of them lost the terms beyond ~35 A (4e-12 of gamma).
// Beyond the radius where the proven tail bound on gamma falls to 1e-7 (p.far2f;
// 26.8 A for 288 atoms in a 26 x 26 x 52 A cell) a term is evaluated in FP32 (a few 1e-6 relative, a few 1e-7 of
// it in one direction) and added to the same df sum: an FP32 sum of those terms
// instead lost the ones below its half ulp in a dense 10 x 10 x 15 A cell, where
// they are thousands per point (1.5e-13 of eps).
constexpr int kNear = 10;
__device__ __forceinline__ void gamma_acc(double& D, float& F, float& G, df v, int n) {
    // the casts run on the FP64 pipe, otherwise idle in this kernel: two issue slots instead
    // of the twenty-odd integer instructions of f32_to_f64
    if (n < kNear) D += (double)v.hi + (double)v.lo;
    else df_add_to(F, G, v);
}

// Appends, in order, the candidates q in [q0, q1) with keep(q) to list (when not
// null) and returns their number. Every thread of the block calls it: thread t
// tests a contiguous run, and an exclusive scan of the runs' counts places each
// survivor, so the list (and every sum taken over it) does not depend on timing.
template <typename Keep>
__device__ int block_compact(int q0, int q1, Keep keep, int* list, int* scratch) {
    const int per = (q1 - q0 + TT - 1) / TT;
    const int b = q0 + (int)threadIdx.x * per, e = min(b + per, q1);
    int c = 0;
    for (int q = b; q < e; ++q) c += keep(q) ? 1 : 0;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    int x = c;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    __syncthreads();                        // scratch is free
    if (lane == 31) scratch[w] = x;
    __syncthreads();
    if (w == 0) {
        const int v = lane < TT / 32 ? scratch[lane] : 0;
        int inc = v;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(0xffffffffu, inc, o);
            if (lane >= o) inc += y;
        }
        if (lane < TT / 32) scratch[lane] = inc - v;
        if (lane == 31) scratch[TT / 32] = inc;
    }
    __syncthreads();
    if (list) {
        int off = scratch[w] + x - c;
        for (int q = b; q < e; ++q)
            if (keep(q)) list[off++] = q;
    }
    const int total = scratch[TT / 32];
    __syncthreads();                        // the list is complete and every thread has the total
    return total;
}

// column / row / plane c of the staged tile (c < NS): axis and grid index, clamped
// on ragged tiles (the clamped values are never read: those points do not exist)
__device__ __forceinline__ void staged_line(const Tile& t, const Geo& g, int c, int& axis, int& gi) {
    if (c < TX) { axis = 0; gi = min(t.i0 + c, g.nx - 1); }
    else if (c < TX + TY) { axis = 1; gi = min(t.j0 + c - TX, g.ny - 1); }
    else { axis = 2; gi = min(t.k0 + c - TX - TY, g.nz - 1); }
}

// displacement of line (axis, gi) from the nearest image of atom a (digit -1, 0 or +1:
// the atom and the point both lie in the cell)
__device__ __forceinline__ df nearest_disp(const GammaTabs& gt, int a, int axis, int gi) {
    df best = as_df(__ldg(gt.d + gtab_index(gt, a, 0, axis, gi)));
    const df dm = as_df(__ldg(gt.d + gtab_index(gt, a, -1, axis, gi)));
    const df dp = as_df(__ldg(gt.d + gtab_index(gt, a, 1, axis, gi)));
    if (fabsf(dm.hi) < fabsf(best.hi)) best = dm;
    if (fabsf(dp.hi) < fabsf(best.hi)) best = dp;
    return best;
}

// image digit of image `im` along `axis`
__device__ __forceinline__ int image_digit(const DielParams& p, int im, int axis) {
    const int nxi = 2 * p.mx + 1, nyi = 2 * p.my + 1;
    return axis == 0 ? im % nxi - p.mx : (axis == 1 ? (im / nxi) % nyi - p.my : im / (nxi * nyi) - p.mz);
}

// One table entry per thread: displacements (FP64, kept as float pairs), the
// exponential tables, and the per-atom constants (kzl by FP64 comparisons of
// k hz with z, the same test as the FP64 kernels').
__global__ void k_gamma_tables(Geo g, Atoms at, DielParams p, const double* rvdw, GammaTabs gt) {
    const int ND = 2 * gt.m + 1;
    const long nd = (long)at.n * ND * 3 * gt.nmax;
    const long total = nd + 2 * (kGT1 + 256) + at.n;
    for (long q = blockIdx.x * (long)blockDim.x + threadIdx.x; q < total; q += (long)gridDim.x * blockDim.x) {
        if (q < nd) {
            const int i = (int)(q % gt.nmax);
            const long r = q / gt.nmax;
            const int axis = (int)(r % 3), n = (int)((r / 3) % ND) - gt.m, a = (int)(r / (3 * ND));
            const int nax = axis == 0 ? g.nx : (axis == 1 ? g.ny : g.nz);
            const double h = axis == 0 ? g.hx : (axis == 1 ? g.hy : g.hz);
            const double L = axis == 0 ? g.lx : (axis == 1 ? g.ly : g.lz);
            const double c = at.w64[3 * a + axis] + n * L;      // the FP64 kernels' image centre
            gt.d[q] = i < nax ? split_to_float2(i * h - c) : make_float2(0.f, 0.f);
            continue;
        }
        long r = q - nd;
        if (r < kGT1) { gt.t1[r] = split_to_float2(exp(-(double)r)); continue; }
        r -= kGT1;
        if (r < 256) { gt.t2[r] = split_to_float2(exp(-(double)r / 256.0)); continue; }
        r -= 256;
        if (r < kGT1) { gt.u1[r] = split_to_float2(exp((double)r)); continue; }
        r -= kGT1;
        if (r < 256) { gt.u2[r] = split_to_float2(exp((double)r / 256.0)); continue; }
        r -= 256;
        const int a = (int)r;
        const double rv = rvdw[a], za = at.w64[3 * a + 2];
        GAtom ga;
        ga.a = split_to_float2(exp(rv));
        ga.b = split_to_float2(exp(-rv));
        ga.qsat = (float)((rv + p.esat) * (rv + p.esat));
        ga.l2a = (float)(rv * 1.4426950408889634);
        int kz = 0;
        if (p.kind == 2 && za <= p.zlim) {
            while (kz < g.nz && kz * g.hz < za) ++kz;           // planes k < kz have k hz < za
        }
        ga.kzl = kz;
        gt.at[a] = ga;
    }
}

__global__ void __launch_bounds__(TT, 2) k_build_eps_gamma_df(Geo g, Atoms at, DielParams p, GammaTabs gt,
                                                           double* eps64, double* fe64, float* eps32) {
    __shared__ int elist[GCAP];
    __shared__ df sx2[GB][TX];
    __shared__ df sy2[GB][TY];
    __shared__ df sz2[GB][EZ];
    __shared__ df srow[GB][kGT1];
    __shared__ df stab[256];
    __shared__ int skz[GB];
    __shared__ float sqs[GB];
    __shared__ int scratch[TT / 32 + 1];
    const Tile t = make_tile_ez(g);
    int tx, ty, tz;
    compact_point(threadIdx.x >> 5, threadIdx.x & 31, tx, ty, tz);
    const int i = t.i0 + tx, j = t.j0 + ty;
    bool valid[4], sat[4];
    double D[4];
    float F[4], G[4];
#pragma unroll
    for (int r = 0; r < 4; ++r) {
        valid[r] = i < g.nx && j < g.ny && t.k0 + tz + 4 * r < g.nz;
        sat[r] = false;
        D[r] = 0.0;
        F[r] = 0.f;
        G[r] = 0.f;
    }
    const bool eq19 = p.kind == 2;
    if (eq19) {
        // the growing terms first (each lower atom's nearest image, no cut-off): a
        // point that saturates needs no decaying sum
        for (int q = threadIdx.x; q < 256; q += TT) stab[q] = as_df(__ldg(gt.u2 + q));
        const int ns = NS + gt.kg;
        for (int a0 = 0; a0 < at.n; a0 += GCAP) {
            const int nl =
                block_compact(a0, min(a0 + GCAP, at.n), [&](int a) { return gt.at[a].kzl > t.k0; }, elist, scratch);
            for (int e0 = 0; e0 < nl; e0 += GB) {
                const int ms = min(GB, nl - e0);
                for (int r = threadIdx.x; r < ms * ns; r += TT) {
                    const int e = r / ns, c = r % ns;
                    const int a = elist[e0 + e];
                    if (c < NS) {
                        int axis, gi;
                        staged_line(t, g, c, axis, gi);
                        const df dd = nearest_disp(gt, a, axis, gi);
                        const df sq = df_mul(dd, dd);
                        if (c < TX) sx2[e][c] = sq;
                        else if (c < TX + TY) sy2[e][c - TX] = sq;
                        else sz2[e][c - TX - TY] = sq;
                    } else {
                        const int n = c - NS;
                        srow[e][n] = df_mul(as_df(gt.at[a].b), as_df(__ldg(gt.u1 + n)));
                        if (n == 0) {
                            skz[e] = gt.at[a].kzl;
                            sqs[e] = gt.at[a].qsat;
                        }
                    }
                }
                __syncthreads();
                for (int e = 0; e < ms; ++e) {
                    const df xy = df_add(sx2[e][tx], sy2[e][ty]);
                    const int kz = skz[e];
                    const float qs = sqs[e];
#pragma unroll
                    for (int r = 0; r < 4; ++r) {
                        const int zz = tz + 4 * r;
                        if (!valid[r] || sat[r] || t.k0 + zz >= kz) continue;
                        const df q = df_add(xy, sz2[e][zz]);
                        if (!(q.hi < qs)) {                             // exp(d - rvdw) >= exp(esat)
                            sat[r] = true;
                            continue;
                        }
                        float y;
                        int n;
                        const df d = q.hi > 0.f ? df_sqrt(q, y) : df{0.f, 0.f};
                        const df v = exp_tab<false>(d, srow[e], stab, n);
                        gamma_acc(D[r], F[r], G[r], v, 0);          // exp(d - rvdw) > exp(-rvdw): near
                    }
                }
                __syncthreads();
            }
        }
    }
    // the decaying terms over every atom image within rcut
    for (int q = threadIdx.x; q < 256; q += TT) stab[q] = as_df(__ldg(gt.t2 + q));
    const int nxi = 2 * p.mx + 1, nyi = 2 * p.my + 1, nimg = nxi * nyi * (2 * p.mz + 1);
    const int nq = at.n * nimg;
    const float reach = p.rcutf + kMargin, rc2f = p.rc2f, far2f = p.far2f;
    auto keep = [&](int q) {
        float fx, fy, fz;
        gimage32(at.w32, q / nimg, q % nimg, g, p, fx, fy, fz);
        return box_d2(t, fx, fy, fz) < reach * reach;
    };
    const int total = block_compact(0, nq, keep, nullptr, scratch);
    const int win = total <= GCAP ? nq : GCAP;       // GCAP candidates never overflow the list
    const int ns = NS + gt.kt1;
    for (int w0 = 0; w0 < nq; w0 += win) {
        const int m = block_compact(w0, min(w0 + win, nq), keep, elist, scratch);
        for (int e0 = 0; e0 < m; e0 += GB) {
            const int ms = min(GB, m - e0);
            for (int r = threadIdx.x; r < ms * ns; r += TT) {
                const int e = r / ns, c = r % ns;
                const int q = elist[e0 + e];
                const int a = q / nimg, im = q % nimg;
                if (c < NS) {
                    int axis, gi;
                    staged_line(t, g, c, axis, gi);
                    const df dd = as_df(__ldg(gt.d + gtab_index(gt, a, image_digit(p, im, axis), axis, gi)));
                    const df sq = df_mul(dd, dd);
                    if (c < TX) sx2[e][c] = sq;
                    else if (c < TX + TY) sy2[e][c - TX] = sq;
                    else sz2[e][c - TX - TY] = sq;
                } else {
                    const int n = c - NS;
                    srow[e][n] = df_mul(as_df(gt.at[a].a), as_df(__ldg(gt.t1 + n)));
                    if (n == 0) {
                        skz[e] = eq19 ? gt.at[a].kzl : 0;
                        sqs[e] = gt.at[a].l2a;
                    }
                }
            }
            __syncthreads();
            for (int e = 0; e < ms; ++e) {
                const df xy = df_add(sx2[e][tx], sy2[e][ty]);
                if (!(xy.hi < rc2f)) continue;                      // beyond rcut for every plane
                const int kz = skz[e];                              // below a lower atom: its growing term instead
                const float l2a = sqs[e];
#pragma unroll
                for (int r = 0; r < 4; ++r) {
                    const int zz = tz + 4 * r;
                    if (!valid[r] || sat[r] || t.k0 + zz < kz) continue;
                    const float qf = xy.hi + sz2[e][zz].hi;
                    if (qf >= far2f) {
                        if (!(qf < rc2f)) continue;
                        float y;
                        df_add_to(F[r], G[r], df{exp_far(sqrt_f32(qf, y), l2a), 0.f});
                        continue;
                    }
                    const df q = df_add(xy, sz2[e][zz]);
                    if (!(q.hi < rc2f)) continue;
                    float y;
                    int n;
                    const df d = q.hi > 0.f ? df_sqrt(q, y) : df{0.f, 0.f};
                    const df v = exp_tab<true>(d, srow[e], stab, n);
                    gamma_acc(D[r], F[r], G[r], v, n);
                }
            }
            __syncthreads();
        }
    }
#pragma unroll
    for (int r = 0; r < 4; ++r) {
        if (!valid[r]) continue;
        const long idx = i + (long)g.nx * (j + (long)g.ny * (t.k0 + tz + 4 * r));
        double e = p.eps0, fe = 0.0;
        if (sat[r]) {
            e = 1.0;
        } else {
            const double gam = D[r] + (f32_to_f64(F[r]) + f32_to_f64(G[r]));
            if (gam > 0.0) {
                const double gb = exp(p.beta2 * log(gam));         // gamma^(2 beta)
                const double den = 1.0 + gb;
                e = 1.0 + (p.eps0 - 1.0) / den;
                fe = -(p.eps0 - 1.0) * p.beta2 * gb / (gam * den * den);
            }
        }
        eps64[idx] = e;
        if (fe64) fe64[idx] = fe;
        if (eps32) eps32[idx] = split_to_float2(e).x;
    }
}

// Beyond kFarF (18 A) a pair's force term is below ~1e-7 of one at contact and the
// terms there sum to below ~1e-5 of an atom's force, so FP32 (a few 1e-6 relative)
// leaves below ~1e-11 of it.
constexpr float kFarF2 = 18.f * 18.f;

// S_a as k_forces_eps_gamma computes it. The tile's image list is in candidate
// order, so each atom's images are adjacent; every warp takes a contiguous share of
// it, one image at a time over the tile's 2048 points (compensated FP32 sums of df
// products), and turns its sums into FP64 atomics only when the atom changes.
__global__ void __launch_bounds__(TT) k_forces_eps_gamma_df(Geo g, Atoms at, DielParams p, GammaTabs gt,
                                                            const float2* phid, const double* wext,
                                                            const double* fe64, double* S) {
    __shared__ df Ws[TX * TY * EZ];              // W (d eps/d gamma), index tx + TX (ty + TY z)
    __shared__ int elist[GCAPF];
    __shared__ df wd[TT / 32][NS];               // a warp's image: displacements of the staged lines
    __shared__ df wq[TT / 32][NS];               // and their squares
    __shared__ df wrow[TT / 32][kGT1];
    __shared__ df stab[256];
    __shared__ int scratch[TT / 32 + 1];
    const Tile t = make_tile_ez(g);
    const bool eq19 = p.kind == 2;
    float l2a = 0.f;                             // the current image's rvdw log2(e)
    int any = 0;
    {
        const df c2x = df_from(g.c2x), c2y = df_from(g.c2y), c2z = df_from(g.c2z);
        for (int q = threadIdx.x; q < TX * TY * EZ; q += TT) {
            const int tx = q % TX, ty = (q / TX) % TY, tz = q / (TX * TY);
            const int i = t.i0 + tx, j = t.j0 + ty, k = t.k0 + tz;
            df w = df{0.f, 0.f};
            if (i < g.nx && j < g.ny && k < g.nz) {
                const long c = i + (long)g.nx * (j + (long)g.ny * k);
                const df nw = neg_force_weight_df(g, phid, wext, fe64[c], i, j, k, c, c2x, c2y, c2z);
                w = df{-nw.hi, -nw.lo};
            }
            Ws[q] = w;
            any |= w.hi != 0.f;
        }
    }
    if (__syncthreads_or(any) == 0) return;      // d eps/d gamma = 0 on the whole tile
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const float rc2f = p.rc2f;
    float sx = 0.f, cx = 0.f, sy = 0.f, cy = 0.f, sz = 0.f, cz = 0.f;
    float fx = 0.f, fy = 0.f, fz = 0.f;          // pairs beyond kFarF, summed in FP32
    // the warp's sums for atom a into S: lanes 0, 1, 2 take x, y, z (one FP64 add each)
    auto flush = [&](int a) {
        df_add_to(sx, cx, df{fx, 0.f}); df_add_to(sy, cy, df{fy, 0.f}); df_add_to(sz, cz, df{fz, 0.f});
        fx = fy = fz = 0.f;
        warp_sum_df(sx, cx); warp_sum_df(sy, cy); warp_sum_df(sz, cz);
        const float hi = lane == 0 ? sx : (lane == 1 ? sy : sz);
        const float lo = lane == 0 ? cx : (lane == 1 ? cy : cz);
        if (lane < 3) {
            const double v = f32_to_f64(hi) + f32_to_f64(lo);
            if (v != 0.0) atomicAdd(&S[3 * a + lane], v);
        }
        sx = cx = sy = cy = sz = cz = 0.f;
    };
    // one image (displacements in wd, squares in wq, factor row in wrow) over the
    // tile's points: a decaying term at the planes k >= kz within rcut, a growing
    // term (grow) at the planes k < kz
    auto pairs = [&](int kz, bool grow) {
        for (int b = 0; b < 16; ++b) {
            int tx, ty, tz;
            compact_point(b, lane, tx, ty, tz);
            if (t.i0 + tx >= g.nx || t.j0 + ty >= g.ny) continue;
            const df xy = df_add(wq[warp][tx], wq[warp][TX + ty]);
            if (!grow && !(xy.hi < rc2f)) continue;
#pragma unroll
            for (int r = 0; r < 4; ++r) {
                const int zz = tz + 4 * r;
                const int k = t.k0 + zz;
                if (k >= g.nz || (grow ? k >= kz : k < kz)) continue;
                const df W = Ws[tx + TX * (ty + TY * zz)];
                if (W.hi == 0.f) continue;                          // also every saturated point
                if (!grow) {
                    const float qf = xy.hi + wq[warp][TX + TY + zz].hi;
                    if (qf >= kFarF2) {
                        if (!(qf < rc2f)) continue;
                        float y;
                        const float c = W.hi * exp_far(sqrt_f32(qf, y), l2a) * y;
                        fx = fmaf(c, wd[warp][tx].hi, fx);
                        fy = fmaf(c, wd[warp][TX + ty].hi, fy);
                        fz = fmaf(c, wd[warp][TX + TY + zz].hi, fz);
                        continue;
                    }
                }
                const df q = df_add(xy, wq[warp][TX + TY + zz]);
                if (!(q.hi > 0.f) || (!grow && !(q.hi < rc2f))) continue;
                float y;
                const df d = df_sqrt(q, y);
                df c;
                int n;
                if (grow) {
                    c = df_mul(df_mul(W, exp_tab<false>(d, wrow[warp], stab, n)), df_recip(d, y));
                    c = df{-c.hi, -c.lo};
                } else {
                    c = df_mul(df_mul(W, exp_tab<true>(d, wrow[warp], stab, n)), df_recip(d, y));
                }
                df_acc(sx, cx, c, wd[warp][tx]);
                df_acc(sy, cy, c, wd[warp][TX + ty]);
                df_acc(sz, cz, c, wd[warp][TX + TY + zz]);
            }
        }
    };
    // decaying terms
    for (int q = threadIdx.x; q < 256; q += TT) stab[q] = as_df(__ldg(gt.t2 + q));
    const int nxi = 2 * p.mx + 1, nyi = 2 * p.my + 1, nimg = nxi * nyi * (2 * p.mz + 1);
    const int nq = at.n * nimg;
    const float reach = p.rcutf + kMargin;
    auto keep = [&](int q) {
        float fx, fy, fz;
        gimage32(at.w32, q / nimg, q % nimg, g, p, fx, fy, fz);
        return box_d2(t, fx, fy, fz) < reach * reach;
    };
    const int total = block_compact(0, nq, keep, nullptr, scratch);
    const int win = total <= GCAPF ? nq : GCAPF;
    for (int w0 = 0; w0 < nq; w0 += win) {
        const int m = block_compact(w0, min(w0 + win, nq), keep, elist, scratch);
        const int e1 = (int)(((long)(warp + 1) * m) / (TT / 32));
        int cur = -1;
        for (int e = (int)(((long)warp * m) / (TT / 32)); e < e1; ++e) {
            const int q = elist[e];
            const int a = q / nimg, im = q % nimg;
            if (a != cur) {
                if (cur >= 0) flush(cur);
                cur = a;
            }
            __syncwarp();
            for (int c = lane; c < NS; c += 32) {
                int axis, gi;
                staged_line(t, g, c, axis, gi);
                const df dd = as_df(__ldg(gt.d + gtab_index(gt, a, image_digit(p, im, axis), axis, gi)));
                wd[warp][c] = dd;
                wq[warp][c] = df_mul(dd, dd);
            }
            const df A = as_df(gt.at[a].a);
            l2a = gt.at[a].l2a;
            for (int n = lane; n < gt.kt1; n += 32) wrow[warp][n] = df_mul(A, as_df(__ldg(gt.t1 + n)));
            __syncwarp();
            pairs(eq19 ? gt.at[a].kzl : 0, false);
        }
        if (cur >= 0) flush(cur);
        __syncthreads();                          // the list is read; the next window rebuilds it
    }
    if (!eq19) return;
    // growing terms: each lower atom's nearest image at the points below it
    __syncthreads();
    for (int q = threadIdx.x; q < 256; q += TT) stab[q] = as_df(__ldg(gt.u2 + q));
    for (int a0 = 0; a0 < at.n; a0 += GCAPF) {
        const int nl =
            block_compact(a0, min(a0 + GCAPF, at.n), [&](int a) { return gt.at[a].kzl > t.k0; }, elist, scratch);
        for (int e = warp; e < nl; e += TT / 32) {
            const int a = elist[e];
            __syncwarp();
            for (int c = lane; c < NS; c += 32) {
                int axis, gi;
                staged_line(t, g, c, axis, gi);
                const df dd = nearest_disp(gt, a, axis, gi);
                wd[warp][c] = dd;
                wq[warp][c] = df_mul(dd, dd);
            }
            const df B = as_df(gt.at[a].b);
            for (int n = lane; n < gt.kg; n += 32) wrow[warp][n] = df_mul(B, as_df(__ldg(gt.u1 + n)));
            __syncwarp();
            pairs(gt.at[a].kzl, true);
            flush(a);
        }
        __syncthreads();                          // the list is read; the next window rebuilds it
    }
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
// s0 = sum rho phi and s1 = sum over the x, y, z faces of each point of
// (eps_i + eps_nb)/2 * ((phi_nb - phi_i)/h)^2 (partial[2b], partial[2b+1]).
// Rows (j, k) are strided over groups of 64 threads (four per block; no thread
// idles on rows of 64, 128, 192, ... points), so no index division per point.
// The face differences are taken in FP64 (their cancellation needs it: three
// FP64 instructions per point); everything else is df64 on the FP32 pipe
// (values split by split_to_float2), each thread's sums compensated float pairs,
// the threads' sums added in FP64: about 2^-46 relative per term, all of whose
// s1 terms are positive.
__device__ __forceinline__ void df_acc2(float& s, float& e, df v) {
    const float t = s + v.hi;
    const float z = t - s;
    e += ((s - (t - z)) + (v.hi - z)) + v.lo;
    s = t;
}

__global__ void __launch_bounds__(kReduceThreads) k_energy(Geo g, const double* __restrict__ rho,
                                                           const double* __restrict__ phi,
                                                           const double* __restrict__ eps, double* partial) {
    __shared__ double red[2][kReduceThreads];
    const int nx = g.nx, ny = g.ny, nz = g.nz;
    const long pl = plane_of(nx, ny);
    const df wx = df_from(g.c2x), wy = df_from(g.c2y), wz = df_from(g.c2z);   // 1/(2 h^2) per axis
    float s0 = 0.f, e0s = 0.f, s1 = 0.f, e1s = 0.f;
    constexpr int G = 64;
    const int groups = blockDim.x / G, lane = threadIdx.x % G;
    for (int row = blockIdx.x * groups + threadIdx.x / G; row < ny * nz; row += gridDim.x * groups) {
        const int j = row % ny, k = row / ny;
        const long base = (long)k * pl + (long)j * nx;
        const long dy = j == ny - 1 ? (1 - ny) * (long)nx : nx;
        const long dz = k == nz - 1 ? (1 - nz) * pl : pl;
        for (int i = lane; i < nx; i += G) {
            const long c = base + i;
            const long xp = c + (i == nx - 1 ? 1 - nx : 1), yp = c + dy, zp = c + dz;
            const double p0 = __ldg(phi + c);
            df_acc2(s0, e0s, df_mul(df_from(__ldg(rho + c)), df_from(p0)));
            const df ec = df_from(__ldg(eps + c));
            const df gx = df_from(__ldg(phi + xp) - p0), gy = df_from(__ldg(phi + yp) - p0),
                     gz = df_from(__ldg(phi + zp) - p0);
            df_acc2(s1, e1s, df_mul(df_mul(df_add(ec, df_from(__ldg(eps + xp))), df_mul(gx, gx)), wx));
            df_acc2(s1, e1s, df_mul(df_mul(df_add(ec, df_from(__ldg(eps + yp))), df_mul(gy, gy)), wy));
            df_acc2(s1, e1s, df_mul(df_mul(df_add(ec, df_from(__ldg(eps + zp))), df_mul(gz, gz)), wz));
        }
    }
    red[0][threadIdx.x] = (double)s0 + (double)e0s;
    red[1][threadIdx.x] = (double)s1 + (double)e1s;
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

// dielectric part: S_a = sum_i W_i sum_images q(d) (-(r_i - c)/d), with
// W_i = (1/2) sum over the six faces of i of (grad_f phi)^2 times pe_i = eps_i - 1,
// q = s'/s. G_eps_a = -h^3/(8 pi) S_a (applied in k_forces_finish).
// One warp per (atom, image) entry runs over the tile's 512 points in compact
// 8 x 2 x 2 blocks. Pairs with |u| > 3.5 contribute at most 5e-6 of a pair at
// the switching radius; their s and s' are taken in FP32.
__global__ void __launch_bounds__(TT) k_forces_eps(Geo g, Atoms at, DielParams p, SwTables tb, const double* phi,
                                                   const double* wext, const double* pe64, double* S) {
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
            const long c = i + (long)g.nx * (j + (long)g.ny * k);
            W = force_weight(g, phi, wext, pe64[c], i, j, k, c);
        }
        Ws[threadIdx.x] = W;   // index tx + TX (ty + TY tz)
    }
    const double rc2 = p.rcut * p.rcut;
    const double iw = p.iw;
    const double sp_norm = p.sp_norm;
    const float rcf = p.rcutf + kMargin;
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
                const float uf = (df - p.r0f) * p.iwf;
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

// charge part: T_a = sum_i phi_i d rho~_i / d R_a. With the periodized factors,
// T_x = coef sum_(i,j,k) X'(i) Y(j) Z(k) phi_ijk, T_y the same with Y', T_z with
// Z', over the Gaussian's index window (each grid index once: the factors sum
// the images). The sum is separable, so each (i, j) column of the window is
// contracted along z once against Z and Z' (two products per point, instead
// of three per point over the whole tiles the window touches), and the two
// column sums are weighted by X' Y, X Y' and X Y. Blocks: kRhoChunks per
// Gaussian, each a contiguous share of the window's columns, one column per
// thread at a time (consecutive x across the threads: coalesced). phi arrives
// as float pairs (df64, converted once per call); products and sums are df64
// with compensated accumulation; each block adds its three sums, times coef, to
// T in FP64.
constexpr int kRhoChunks = 16;
constexpr int kRhoThreads = 256;
constexpr int kRhoZStage = 1024;

__global__ void __launch_bounds__(kRhoThreads) k_forces_rho(Geo g, GaussTabs gt, const float2* __restrict__ phid,
                                                             double* T) {
    __shared__ df zs[2][kRhoZStage];           // Z and Z' over the window's planes, when it fits
    __shared__ df red[kRhoThreads / 32][3];
    const int ge = blockIdx.x / kRhoChunks, chunk = blockIdx.x % kRhoChunks;
    const int* w = gt.win + ge * 6;
    const int wx = w[1] - w[0] + 1, wy = w[3] - w[2] + 1, wz = w[5] - w[4] + 1;
    const int ncol = wx * wy;
    const int c0 = (int)((long)ncol * chunk / kRhoChunks), c1 = (int)((long)ncol * (chunk + 1) / kRhoChunks);
    if (c0 >= c1) return;
    const long rz = gt_row(ge, 2, gt.nmax);
    const bool staged = wz <= kRhoZStage;
    for (int q = threadIdx.x; staged && q < wz; q += blockDim.x) {
        int k = w[4] + q;
        k = k < 0 ? k + g.nz : (k >= g.nz ? k - g.nz : k);
        zs[0][q] = as_df(gt.vald[rz + k]);
        zs[1][q] = as_df(gt.derd[rz + k]);
    }
    __syncthreads();
    const long pl = plane_of(g.nx, g.ny);
    const long rx = gt_row(ge, 0, gt.nmax), ry = gt_row(ge, 1, gt.nmax);
    int k0 = w[4];
    k0 = k0 < 0 ? k0 + g.nz : (k0 >= g.nz ? k0 - g.nz : k0);
    float tx = 0.f, ex = 0.f, ty = 0.f, ey = 0.f, tz = 0.f, ez = 0.f;
    for (int col = c0 + threadIdx.x; col < c1; col += blockDim.x) {
        int i = w[0] + col % wx, j = w[2] + col / wx;
        i = i < 0 ? i + g.nx : (i >= g.nx ? i - g.nx : i);
        j = j < 0 ? j + g.ny : (j >= g.ny ? j - g.ny : j);
        const float2* pc = phid + i + (long)g.nx * j;
        float a0 = 0.f, e0 = 0.f, a1 = 0.f, e1 = 0.f;
        int k = k0;
        if (staged) {
            for (int q = 0; q < wz; ++q) {
                const df p = as_df(__ldg(pc + pl * k));
                df_acc(a0, e0, p, zs[0][q]);
                df_acc(a1, e1, p, zs[1][q]);
                k = k + 1 == g.nz ? 0 : k + 1;
            }
        } else {
            for (int q = 0; q < wz; ++q) {
                const df p = as_df(__ldg(pc + pl * k));
                df_acc(a0, e0, p, as_df(gt.vald[rz + k]));
                df_acc(a1, e1, p, as_df(gt.derd[rz + k]));
                k = k + 1 == g.nz ? 0 : k + 1;
            }
        }
        const df A0 = df_quick(a0, e0), A1 = df_quick(a1, e1);
        const df X = as_df(gt.vald[rx + i]), Xd = as_df(gt.derd[rx + i]);
        const df Y = as_df(gt.vald[ry + j]), Yd = as_df(gt.derd[ry + j]);
        df_acc(tx, ex, df_mul(Xd, Y), A0);
        df_acc(ty, ey, df_mul(X, Yd), A0);
        df_acc(tz, ez, df_mul(X, Y), A1);
    }
    warp_sum_df(tx, ex); warp_sum_df(ty, ey); warp_sum_df(tz, ez);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (lane == 0) {
        red[warp][0] = df{tx, ex};
        red[warp][1] = df{ty, ey};
        red[warp][2] = df{tz, ez};
    }
    __syncthreads();
    if (threadIdx.x < 3) {
        const int comp = threadIdx.x;
        float s = 0.f, e = 0.f;
        for (int v = 0; v < kRhoThreads / 32; ++v) df_acc(s, e, red[v][comp], df{1.f, 0.f});
        const double v = df_to(df_mul(as_df(gt.coefd[ge]), df_quick(s, e)));
        if (v != 0.0) atomicAdd(&T[3 * (ge >> 1) + comp], v);
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

void launch_switch_tables(DielParams p, const SwTables& tb, double* s_coef, double* h_coef, float4* s_pack,
                          float4* h_pack, cudaStream_t s) {
    k_switch_tables<<<(2 * kSwNI + 127) / 128, 128, 0, s>>>(p, tb, s_coef, h_coef, s_pack, h_pack);
}

size_t coord_tabs_bytes(int n_atoms, int nmax, bool with_d) {
    const size_t e = (size_t)(n_atoms > 0 ? n_atoms : 1) * 9 * nmax;
    return e * (sizeof(int) + sizeof(float2) + (with_d ? sizeof(float2) : 0)) + 256;
}

CoordTabs coord_tabs_view(void* base, int n_atoms, int nmax, bool with_d) {
    const size_t e = (size_t)(n_atoms > 0 ? n_atoms : 1) * 9 * nmax;
    CoordTabs ct{};
    ct.nmax = nmax;
    ct.f = static_cast<float2*>(base);
    ct.d = with_d ? ct.f + e : nullptr;
    ct.n = reinterpret_cast<int*>(ct.f + (with_d ? 2 : 1) * e);
    return ct;
}

void launch_coord_tables(const Geo& g, Atoms at, double qlo, double inv_dq, const CoordTabs& ct, cudaStream_t s) {
    const long total = (long)at.n * 9 * ct.nmax;
    if (total > 0)
        k_coord_tables<<<(int)((total + 255) / 256 < 152L * 16 ? (total + 255) / 256 : 152L * 16), 256, 0, s>>>(
            g, at, qlo, inv_dq, ct);
}

bool launch_build_eps(const Geo& g, Atoms at, DielParams p, const SwTables& tb, const CoordTabs& ct, double* eps64,
                      double* pe64, float* eps32, double* plane_max, cudaStream_t s) {
    if (tb.s32) {
        cudaMemsetAsync(plane_max, 0, sizeof(double) * g.nz, s);
        k_build_eps_tab<<<tile_grid_ez(g), TT, 0, s>>>(g, at, p, tb, ct, eps64, pe64, eps32, plane_max);
        return true;
    }
    k_build_eps<<<tile_grid(g), TT, 0, s>>>(g, at, p, tb, eps64, pe64, eps32);
    return false;
}

size_t gauss_tabs_bytes(int n_atoms, int nmax) {
    const size_t G = 2 * (size_t)(n_atoms > 0 ? n_atoms : 1);
    return 2 * (sizeof(double) * (2 * G * 3 * nmax + G)) + sizeof(int) * G * 6 + 64;
}

GaussTabs gauss_tabs_view(void* base, int n_atoms, int nmax) {
    GaussTabs gt{};
    gt.G = 2 * n_atoms;
    gt.nmax = nmax;
    const size_t G = 2 * (size_t)(n_atoms > 0 ? n_atoms : 1);
    double* d = static_cast<double*>(base);
    gt.val = d;
    gt.der = d + G * 3 * nmax;
    gt.coef = d + 2 * G * 3 * nmax;
    float2* f = reinterpret_cast<float2*>(d + 2 * G * 3 * nmax + G);
    gt.vald = f;
    gt.derd = f + G * 3 * nmax;
    gt.coefd = f + 2 * G * 3 * nmax;
    gt.win = reinterpret_cast<int*>(f + 2 * G * 3 * nmax + G);
    return gt;
}

void launch_gauss_tables(const Geo& g, Atoms at, double cut, const GaussTabs& gt, cudaStream_t s) {
    const long total = (long)gt.G * 3 * gt.nmax;
    if (total > 0) k_gauss_tables<<<(int)((total + 255) / 256 < 152L * 64 ? (total + 255) / 256 : 152L * 64), 256, 0, s>>>(
        g, at, cut, gt);
}

void launch_build_rho_raw(const Geo& g, const GaussTabs& gt, double* rho, cudaStream_t s) {
    k_build_rho<<<tile_grid(g), TT, 0, s>>>(g, gt, rho);
}

void launch_build_eps_gamma(const Geo& g, Atoms at, DielParams p, const double* rvdw, double* eps64, double* fe64,
                            float* eps32, cudaStream_t s) {
    k_build_eps_gamma<<<tile_grid(g), TT, 0, s>>>(g, at, p, rvdw, eps64, fe64, eps32);
}

void launch_forces_eps_gamma(const Geo& g, Atoms at, DielParams p, const double* rvdw, const double* phi,
                             const double* wext, const double* fe64, double* S, cudaStream_t s) {
    k_forces_eps_gamma<<<tile_grid(g), TT, 0, s>>>(g, at, p, rvdw, phi, wext, fe64, S);
}

size_t gamma_tabs_bytes(int n_atoms, int m, int nmax) {
    const size_t n = (size_t)(n_atoms > 0 ? n_atoms : 1);
    return (n * (2 * m + 1) * 3 * nmax + 2 * (kGT1 + 256)) * sizeof(float2) + n * sizeof(GAtom) + 256;
}

GammaTabs gamma_tabs_view(void* base, int n_atoms, int m, int nmax) {
    const size_t n = (size_t)(n_atoms > 0 ? n_atoms : 1);
    GammaTabs gt{};
    gt.m = m;
    gt.nmax = nmax;
    gt.d = static_cast<float2*>(base);
    gt.t1 = gt.d + n * (2 * m + 1) * 3 * nmax;
    gt.t2 = gt.t1 + kGT1;
    gt.u1 = gt.t2 + 256;
    gt.u2 = gt.u1 + kGT1;
    gt.at = reinterpret_cast<GAtom*>(gt.u2 + 256);
    return gt;
}

void launch_gamma_tables(const Geo& g, Atoms at, DielParams p, const double* rvdw, const GammaTabs& gt,
                         cudaStream_t s) {
    const long total = (long)at.n * (2 * gt.m + 1) * 3 * gt.nmax + 2 * (kGT1 + 256) + at.n;
    k_gamma_tables<<<(int)((total + 255) / 256 < 152L * 16 ? (total + 255) / 256 : 152L * 16), 256, 0, s>>>(
        g, at, p, rvdw, gt);
}

void launch_build_eps_gamma_df(const Geo& g, Atoms at, DielParams p, const GammaTabs& gt, double* eps64,
                               double* fe64, float* eps32, cudaStream_t s) {
    k_build_eps_gamma_df<<<tile_grid_ez(g), TT, 0, s>>>(g, at, p, gt, eps64, fe64, eps32);
}

void launch_forces_eps_gamma_df(const Geo& g, Atoms at, DielParams p, const GammaTabs& gt, const float2* phid,
                                const double* wext, const double* fe64, double* S, cudaStream_t s) {
    k_forces_eps_gamma_df<<<tile_grid_ez(g), TT, 0, s>>>(g, at, p, gt, phid, wext, fe64, S);
}

void launch_plane_max(const Geo& g, const double* eps64, double* out, cudaStream_t s) {
    k_plane_max<<<g.nz, 256, 0, s>>>(g, eps64, out);
}

void launch_energy(const Geo& g, const double* rho, const double* phi, const double* eps64,
                   double* partial, cudaStream_t s) {
    k_energy<<<kReduceBlocks, kReduceThreads, 0, s>>>(g, rho, phi, eps64, partial);
}

void launch_forces_eps(const Geo& g, Atoms at, DielParams p, const SwTables& tb, const CoordTabs& ct,
                       const double* phi, const float2* phid, const double* wext, const double* pe64, double* S,
                       cudaStream_t s) {
    if (tb.h32) k_forces_eps_tab<<<tile_grid_ez(g), TT, 0, s>>>(g, at, p, tb, ct, phid, wext, pe64, S);
    else k_forces_eps<<<tile_grid(g), TT, 0, s>>>(g, at, p, tb, phi, wext, pe64, S);
}

void launch_forces_rho(const Geo& g, const GaussTabs& gt, const double* phi, float2* phid, double* T,
                       cudaStream_t s) {
    if (gt.G <= 0) return;
    if (phi) launch_to_df((long)g.nx * g.ny * g.nz, phi, 1.0, phid, s);
    k_forces_rho<<<gt.G * kRhoChunks, kRhoThreads, 0, s>>>(g, gt, phid, T);
}

void launch_forces_finish(const double* S, const double* T, int n, double ce, double cr, double* F,
                          cudaStream_t s) {
    k_forces_finish<<<(3 * n + 255) / 256, 256, 0, s>>>(S, T, n, ce, cr, F);
}

}  // namespace gp
