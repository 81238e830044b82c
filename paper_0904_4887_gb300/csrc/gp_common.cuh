// Internal declarations shared by the CUDA translation units of the solver.
#pragma once
#include <cuda_runtime.h>
#include <cstdint>
#include <cstddef>

#include "gp.h"

#include <cmath>

namespace gp {

constexpr int kReduceBlocks = 608;      // 4 x 152 SMs: fixed partial count, deterministic sums
constexpr int kReduceThreads = 256;
constexpr int kMaxCoarse = 512;         // largest coarsest grid solved by a dense inverse
constexpr int kAutoCoarse = 64;         // automatic level choice: coarsen to <= 64 points
constexpr double kPi = 3.14159265358979323846;

// Programmatic dependent launch: a kernel launched with the programmatic
// stream-serialization attribute may be scheduled while the kernel before it
// in the stream is still finishing, which hides most of the gap between two
// short kernels. Such a kernel calls this before its first access to global
// memory: it waits until the previous kernel has completed and its writes are
// visible. Launched without the attribute it returns at once.
// It then lets the next such kernel be scheduled (its blocks wait in turn), so
// that it is resident by the time this one ends.
__device__ __forceinline__ void griddep_wait() {
    asm volatile("griddepcontrol.wait;" ::: "memory");
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}

// ---------------------------------------------------------------- level view
// One multigrid level. Arrays are addressed with a base pointer at plane 0 and
// own one halo plane below (k = -1) and one above (k = nz): for Dirichlet
// levels (zper == 0) the halos hold the boundary values; for periodic levels
// they are unused and k wraps.
template <typename T>
struct LV {
    int nx, ny, nz, zper;
    T ihx2, ihy2, ihz2;           // 1/h^2 per axis
    const T* eps;                 // cell eps (cell == 1): face = (e_i + e_j)/2 * ih2
    const T* cx;                  // face coefficients incl. 1/h^2 (cell == 0);
    const T* cy;                  //   c?[i] is the face between i and i+1 along ?
    const T* cz;                  //   cz valid for k = -1 .. nz-1
    int cell;
};

struct Atoms {
    const double* w64;     // [n][3] positions wrapped into the cell (launch_wrap_atoms)
    const float4* w32;     // the same in FP32, for culling
    const double* gauss;   // [n][3] = Z, sigma_core, sigma_cloud (may be null)
    int n;
};

// Grid geometry. The derived constants are filled on the host (make_geo):
// an FP64 divide costs tens of FP64-pipe instructions, and the FP64 pipe is
// 1/64 of the FP32 rate here, so no kernel derives them per thread.
struct Geo {
    int nx, ny, nz;
    double hx, hy, hz;
    double lx, ly, lz;
    double ihx, ihy, ihz;   // 1 / h
    double c2x, c2y, c2z;   // 1 / (2 h^2): face-mean operator weight per axis
    double inv_n;           // 1 / (nx ny nz)
    float lxf, lyf, lzf;    // cell lengths in FP32 (culling)
    float hxf, hyf, hzf;    // spacings in FP32 (culling boxes)
};

inline Geo make_geo(int nx, int ny, int nz, double lx, double ly, double lz) {
    Geo g{};
    g.nx = nx; g.ny = ny; g.nz = nz;
    g.lx = lx; g.ly = ly; g.lz = lz;
    g.hx = lx / nx; g.hy = ly / ny; g.hz = lz / nz;
    g.ihx = 1.0 / g.hx; g.ihy = 1.0 / g.hy; g.ihz = 1.0 / g.hz;
    g.c2x = 0.5 / (g.hx * g.hx); g.c2y = 0.5 / (g.hy * g.hy); g.c2z = 0.5 / (g.hz * g.hz);
    g.inv_n = 1.0 / ((double)nx * ny * nz);
    g.lxf = (float)lx; g.lyf = (float)ly; g.lzf = (float)lz;
    g.hxf = (float)g.hx; g.hyf = (float)g.hy; g.hzf = (float)g.hz;
    return g;
}

// Dielectric parameters with host-derived constants: kind 0 is the erf-product
// switching form, kind 1 the dummy-density form of Eq. 9-10 (beta).
struct DielParams {
    double eps0, r0, w, rcut;
    double iw;        // 1 / w
    double sp_norm;   // 1 / (w sqrt(pi)): ds/du prefactor
    double tiny;      // product-below-which eps - 1 rounds away: 5.5e-17 / (eps0 - 1)
    double beta2;     // 2 beta (kinds 1, 2)
    double zlim;      // kind 2: atoms with z <= zlim exclude the solvent below them (Eq. 19)
    double esat;      // kind 2: growing exponent beyond which eps = 1 exactly (ln(eps0-1)+37)/(2 beta)
    int kind;
    int mx, my, mz;   // kinds 1, 2: images n in [-m, m] per axis reach every point within rcut
    // FP32 copies for the culling and the FP32 branches, made on the host: a kernel that
    // converted them per thread would spend FP64-pipe instructions on it (and may redo them)
    float rcutf, rc2f, reachf, tinyf, r0f, iwf, spnf;
    // kinds 1, 2: squared radius beyond which the df64 dielectric kernel takes a pair in
    // FP32 (the host puts it where the proven tail bound on gamma falls to 1e-7)
    float far2f;
};

// (hi, lo) = (RN_float(x), RN_float(x - hi)): the float pair of a double, as the
// casts would give it, from the bits with integer and FP32 instructions only. On
// GB300 each FP64 instruction of a warp (casts between double and float
// included) holds the FP64 pipe for about 64 cycles, and a short fallback branch
// of casts is executed by the whole warp (or if-converted and executed always),
// so no path here has one. IEEE 754 binary64 -> binary32 rounding to nearest
// even: keep the top 23 of the 52 mantissa bits, round on the other 29 (a carry
// moves into the exponent field by itself); the residual is those 29 bits less
// the rounding, times 2^(E - 1075), a power of two built from its bits, so the
// int-to-float conversion is its only rounding. Identical to the casts for
// 2^-63 <= |x| < 2^128 and for zeros; below 2^-63 (where lo could be subnormal)
// hi is still RN_float(x) and lo is 0 (an error below 2^-87), below 2^-126
// (where hi would be subnormal) both are zero of the sign of x; beyond the float
// range hi is an infinity, and a NaN stays a NaN.
__device__ __forceinline__ float2 split_to_float2(double x) {
    const unsigned long long b = (unsigned long long)__double_as_longlong(x);
    const unsigned h = (unsigned)(b >> 32), l = (unsigned)b;
    const unsigned sign = h & 0x80000000u;
    const int E = (int)((h >> 20) & 0x7ffu);
    const int e = E - 1023 + 127;
    if (e >= 255) {
        const unsigned nan = (E == 2047 && ((h & 0xfffffu) | l)) ? 0x400000u : 0u;
        return make_float2(__uint_as_float(sign | 0x7f800000u | nan), 0.f);
    }
    if (e < 1) return make_float2(__uint_as_float(sign), 0.f);
    const unsigned m23 = ((h & 0xfffffu) << 3) | (l >> 29);
    const unsigned rem = l & 0x1fffffffu;
    const unsigned up = (rem > 0x10000000u || (rem == 0x10000000u && (m23 & 1u))) ? 1u : 0u;
    const float hi = __uint_as_float(sign | ((((unsigned)e << 23) | m23) + up));
    const int r = (int)rem - (int)(up << 29);
    float lo = E < 960 ? 0.f : (float)r * __uint_as_float((unsigned)(E - 948) << 23);
    if (sign && r != 0) lo = -lo;          // x - hi = 0 is +0, as the cast gives it
    return make_float2(hi, lo);
}

// The double of a float, exactly as the cast gives it, from the bits with integer
// instructions (the cast is an FP64-pipe instruction on GB300): exponent rebased
// from 127 to 1023, mantissa moved up 29 bits; a subnormal float is normalised
// first (its leading one moved to the hidden bit); infinities and NaNs keep
// their pattern.
__device__ __forceinline__ double f32_to_f64(float x) {
    const unsigned u = __float_as_uint(x);
    const unsigned long long sign = (unsigned long long)(u >> 31) << 63;
    const unsigned e = (u >> 23) & 0xffu;
    unsigned m = u & 0x7fffffu;
    unsigned long long bits;
    if (e == 0xffu) bits = sign | (0x7ffull << 52) | ((unsigned long long)m << 29);
    else if (e != 0) bits = sign | ((unsigned long long)(e + 896) << 52) | ((unsigned long long)m << 29);
    else if (m == 0) bits = sign;
    else {
        const int lz = __clz(m) - 8;              // the leading one sits at bit 23 - lz
        m = (m << lz) & 0x7fffffu;
        bits = sign | ((unsigned long long)(897 - lz) << 52) | ((unsigned long long)m << 29);
    }
    return __longlong_as_double((long long)bits);
}

inline DielParams make_diel(double eps0, double r0, double w, double rcut, int kind = 0, double beta = 2.4,
                            double zlim = 0.0) {
    DielParams p{};
    p.eps0 = eps0; p.r0 = r0; p.w = w; p.rcut = rcut;
    p.kind = kind;
    p.beta2 = 2.0 * beta;
    p.zlim = zlim;
    p.esat = (std::log(eps0 - 1.0 > 1.0 ? eps0 - 1.0 : 1.0) + 37.0) / (2.0 * beta);
    p.iw = 1.0 / w;
    p.sp_norm = 1.0 / (w * 1.7724538509055160273);
    p.tiny = 5.5e-17 / (eps0 - 1.0 > 0.0 ? eps0 - 1.0 : 1.0);
    p.mx = p.my = p.mz = 1;
    p.rcutf = (float)rcut;
    p.rc2f = (float)(rcut * rcut);
    p.reachf = (float)(rcut < r0 + 6.0 * w ? rcut : r0 + 6.0 * w);
    p.tinyf = (float)p.tiny;
    p.r0f = (float)r0;
    p.iwf = (float)p.iw;
    p.spnf = (float)p.sp_norm;
    p.far2f = 3.0e38f;
    return p;
}

__host__ __device__ inline long plane_of(int nx, int ny) { return (long)nx * ny; }

// switching-function tables (k_fields.cu): s and h = s'/(s d) as polynomials in q = d^2
constexpr int kSwNI = 256, kSwDeg = 9;
// Packed FP32 copies, 16 floats per interval: the low-degree coefficients
// (below kSwSplitS for s, kSwSplitH for h) as hi/lo pairs, then the rest as
// single floats (they are small enough that FP32 leaves < 1e-14 relative).
constexpr int kSwSplitS = 4, kSwSplitH = 6;
struct SwTables {
    const double* s = nullptr;    // kSwNI x (kSwDeg+1) monomial coefficients, or null (use erfc)
    const double* h = nullptr;
    const float4* s32 = nullptr;  // kSwNI x 4 packed (see above)
    const float4* h32 = nullptr;
    double s_qlo = 0, s_qhi = 0, s_inv_dq = 0, s_dq = 0;
    double h_qlo = 0, h_qhi = 0, h_inv_dq = 0, h_dq = 0;
    float s_qlof = 0, s_dqf = 0, h_qlof = 0, h_dqf = 0;   // FP32 copies, set on the host
};

// Table coordinates of the separable squared distance, per atom, image digit
// m in {0, 1, 2} (shift (m - 1) L) and grid index along each axis:
//   X = ((i hx - cx)^2 - qlo) / dq,  Y = (j hy - cy)^2 / dq,  Z = (k hz - cz)^2 / dq,
// computed once per dielectric in FP64 and kept as an integer part n and a df
// fraction f in [0, 1) (and, for the force tables, the displacement d as a df),
// so that the tile kernels stage them with loads instead of FP64 arithmetic.
// Entry (a, m, axis, i) sits at ((a * 3 + m) * 3 + axis) * nmax + i.
struct CoordTabs {
    int* n;
    float2* f;
    float2* d;      // displacement i h - c (force tables), or null
    int nmax;
};
// ---------------------------------------------------------------- launchers
// fields (k_fields.cu)
void launch_wrap_atoms(const Geo& g, const double* pos, int n, double* w64, float4* w32, cudaStream_t s);
void launch_switch_tables(DielParams p, const SwTables& tb, double* s_coef, double* h_coef, float4* s_pack,
                          float4* h_pack, cudaStream_t s);
// true when the tabulated kernel ran, which also leaves each z-plane's max of eps - 1 in
// plane_max (nz values); otherwise plane_max is untouched
bool launch_build_eps(const Geo& g, Atoms at, DielParams p, const SwTables& tb, const CoordTabs& ct, double* eps64,
                      double* pe64, float* eps32, double* plane_max, cudaStream_t s);
// Eq. 9-10: gamma = sum exp(-(d - rvdw)), eps = 1 + (eps0 - 1)/(1 + gamma^(2 beta)); fe64 = d eps / d gamma
void launch_build_eps_gamma(const Geo& g, Atoms at, DielParams p, const double* rvdw, double* eps64, double* fe64,
                            float* eps32, cudaStream_t s);
void launch_forces_eps_gamma(const Geo& g, Atoms at, DielParams p, const double* rvdw, const double* phi,
                             const double* wext, const double* fe64, double* S, cudaStream_t s);
// The same two sums in df64 on the FP32 pipe, from tables built once per set of atoms.
// Per atom: exp(rvdw) and exp(-rvdw) as float pairs, (rvdw + esat)^2 in FP32 (a growing
// Eq. 19 term whose squared distance reaches it saturates the point), and kzl, the
// first grid plane k with k hz >= z of the atom in the cell when the atom belongs to
// Eq. 19's lower layer (kind 2, z <= zlim), else 0: planes k < kzl lie below it.
struct GAtom {
    float2 a, b;
    float qsat;
    int kzl;
    float l2a;      // rvdw log2(e): exp(rvdw - d) = 2^(l2a - d log2(e)) for the FP32 far pairs
};
constexpr int kGT1 = 56;        // exp(-+n) rows the df64 kernels stage per atom: distances below kGT1 - 2 A
struct GammaTabs {
    float2* d;      // [n_atoms][2m + 1][3][nmax]: i h - (w_a + n L) for image digit n in [-m, m], as a pair
    float2* t1;     // exp(-n), n < kGT1
    float2* t2;     // exp(-j/256), j < 256
    float2* u1;     // exp(+n), n < kGT1
    float2* u2;     // exp(+j/256), j < 256
    GAtom* at;      // [n_atoms]
    int m, nmax;
    int kt1;        // rows of exp(-n) a decaying term can use: floor(rcut) + 2
    int kg;         // rows of exp(+n) a growing term can use before it saturates
};
size_t gamma_tabs_bytes(int n_atoms, int m, int nmax);
GammaTabs gamma_tabs_view(void* base, int n_atoms, int m, int nmax);
void launch_gamma_tables(const Geo& g, Atoms at, DielParams p, const double* rvdw, const GammaTabs& gt,
                         cudaStream_t s);
void launch_build_eps_gamma_df(const Geo& g, Atoms at, DielParams p, const GammaTabs& gt, double* eps64,
                               double* fe64, float* eps32, cudaStream_t s);
// phid: phi as float pairs (read unless wext is given)
void launch_forces_eps_gamma_df(const Geo& g, Atoms at, DielParams p, const GammaTabs& gt, const float2* phid,
                                const double* wext, const double* fe64, double* S, cudaStream_t s);
// Periodized 1D Gaussian factor tables (k_fields.cu), Gaussian ge = 2 atom + {0 core, 1 cloud}
struct GaussTabs {
    double* val;    // [G][3][nmax] X, Y, Z factors summed over the images -L, 0, +L
    double* der;    // [G][3][nmax] the same times d / sigma^2 (centre derivative)
    double* coef;   // [G] +-Z / (2 pi sigma^2)^(3/2)
    float2* vald;   // val, der, coef again as (hi, lo) float pairs (df64) for the
    float2* derd;   //   FP32-pipe arithmetic of the density kernels
    float2* coefd;
    int* win;       // [G][3][2] conservative index window of the unshifted image
    int G, nmax;
};
size_t coord_tabs_bytes(int n_atoms, int nmax, bool with_d);
CoordTabs coord_tabs_view(void* base, int n_atoms, int nmax, bool with_d);
void launch_coord_tables(const Geo& g, Atoms at, double qlo, double inv_dq, const CoordTabs& ct, cudaStream_t s);
size_t gauss_tabs_bytes(int n_atoms, int nmax);
GaussTabs gauss_tabs_view(void* base, int n_atoms, int nmax);
void launch_gauss_tables(const Geo& g, Atoms at, double cut_sigmas, const GaussTabs& gt, cudaStream_t s);
void launch_build_rho_raw(const Geo& g, const GaussTabs& gt, double* rho, cudaStream_t s);
void launch_plane_max(const Geo& g, const double* eps64, double* plane_max, cudaStream_t s);
void launch_energy(const Geo& g, const double* rho, const double* phi, const double* eps64,
                   double* partial, cudaStream_t s);
// phid: phi as float pairs, which the tabulated kernel reads unless wext is given
void launch_forces_eps(const Geo& g, Atoms at, DielParams p, const SwTables& tb, const CoordTabs& ct,
                       const double* phi, const float2* phid, const double* wext, const double* pe64, double* S,
                       cudaStream_t s);
// phid: nx*ny*nz float pairs; phi is converted into it first unless phi is null
// (phid then already holds it)
void launch_forces_rho(const Geo& g, const GaussTabs& gt, const double* phi, float2* phid, double* T,
                       cudaStream_t s);
void launch_forces_finish(const double* S, const double* T, int n, double ce, double cr, double* F,
                          cudaStream_t s);

// reductions and FP64 full-box passes (k_mg.cu)
void launch_finalize(const double* partial, int nparts, int ncomp, double* out, cudaStream_t s);
void launch_rho_stats(long n, const double* rho, double* partial, cudaStream_t s);
// df64 (hi, lo FP32 pair) copies and the df64 full-box residual of the mixed-precision path
// dst = the pairs of scale * src; nonzero (may be null): set to 1 if src has a nonzero
// value (it is not cleared here); hi_out (may be null): the leading floats
void launch_to_df(long n, const double* src, double scale, float2* dst, cudaStream_t s, int* nonzero = nullptr,
                  float* hi_out = nullptr);
void launch_residual_df(const Geo& g, const float2* phid, const float2* bd, const float2* epsd, float* r_out,
                        double* partial, cudaStream_t s);
// phid += e (n even, 16-byte aligned)
void launch_update_phid(long n, float2* phid, const float* e, cudaStream_t s);
// dst = src - scale * sum_slot[0] (pairs to doubles, the mean taken off)
void launch_from_df_gauge(long n, const float2* src, const double* sum_slot, double scale, double* dst,
                          cudaStream_t s);
void launch_sub_mean(long n, double* x, const double* sum_slot, double scale, cudaStream_t s);
template <typename T>
void launch_residual64(const Geo& g, const double* phi, const double* rho, const double* eps64,
                       T* r_out, double* partial, cudaStream_t s);
// sixth-order residual (k_fd6.cu): r = -4 pi rho - A6 phi - mu eps, partial[b] = sum r^2
void launch_residual6(const Geo& g, const double* phi, const double* rho, const double* eps64, double mu,
                      double* r_out, double* partial, cudaStream_t s);
// sixth-order solve pieces (k_fd6.cu)
void launch_fd6_apply(const Geo& g, const double* x, const double* eps, const double* rho, double crho,
                      const double* rsum, double sa, double* y, double* partial, cudaStream_t s);
void launch_fd6_apply_t(const Geo& g, const double* x, const double* eps, const double* d1e, const double* rho,
                        double crho, const double* rsum, double sa, double* y, double* partial, cudaStream_t s);
void launch_fd6_d1(const Geo& g, const double* u, const double* w, double* out3, cudaStream_t s);
void launch_fd6_weps(const Geo& g, const double* phi, const double* lam, const double* t3, double mu, double* weps,
                     cudaStream_t s);
void launch_fd6_sub_ratio(long n, double* y, const double* w, const double* num, const double* den,
                          cudaStream_t s);
template <typename T>
void launch_fd6_to64(long n, const T* src, const double* eps, double* dst, double* partial, cudaStream_t s);
void launch_fd6_wrho(long n, const double* phi, const double* lam, double* out, double* partial, cudaStream_t s);
void launch_fd6_set(double* slot, double v, cudaStream_t s);
template <typename T>
void launch_update_phi(const Geo& g, double* phi, const T* e_full, const T* e_band,
                       int band_first, int band_nz, cudaStream_t s);

// multigrid (k_mg.cu)
// init: the first half sweep from u = 0 (neighbours read as zero, so u needs no clearing
// before it; the other colour is overwritten by the next half sweep)
template <typename T> void launch_rbgs(const LV<T>& L, T* u, const T* f, int color, cudaStream_t s,
                                       bool init = false);
// one fused red-black sweep of a cell-eps level: u_new from u_old, colour `first` updated first (k_smooth.cu)
void rb_sweep_init();
// polls per mbarrier wait of the whole-row smoother's main loop (< 0: the default);
// gp_create sets it from GP_TEST_SWEEP_WAIT_POLLS, which only tests use
void rb_sweep_set_wait_polls(int polls);
// err: device flag set to 1 if a TMA wait of the row-tile kernel expired (may be null).
// u_old null: the sweep starts from u = 0, which only the warp-specialised row shapes
// do; for the others nothing is launched and the call returns false.
template <typename T> bool launch_rb_sweep(const LV<T>& L, const T* u_old, const T* f, T* u_new, int first,
                                           cudaStream_t s, int shape, int* err = nullptr);
template <typename T> int rb_sweep_autotune(const LV<T>& L, const T* u_old, const T* f, T* u_new, cudaStream_t s);
// the shape actually used for a requested one (row tiles fall back to 0 where unavailable)
template <typename T> int rb_sweep_resolve(const LV<T>& L, int shape);
constexpr int kSweepShapeCount = 15;    // 4 x-y tiles + 3 row tiles + 8 warp-specialised row tiles
template <typename T> void launch_residual(const LV<T>& L, const T* u, const T* f, T* r, cudaStream_t s);
template <typename T> void launch_restrict(const LV<T>& F, const T* r, const LV<T>& C, T* fc, cudaStream_t s);
template <typename T> void launch_prolong_add(const LV<T>& F, T* u, const LV<T>& C, const T* uc, cudaStream_t s);
template <typename T> void launch_coarsen_faces(const LV<T>& F, int nxc, int nyc, int nzc,
                                                T* cx, T* cy, T* cz, cudaStream_t s);
template <typename T> void launch_coarse_matrix(const LV<T>& C, double* M, cudaStream_t s);
// the inverse of the dense n x n M into M + n*n; pairs: the one-CTA version in
// float-pair arithmetic (for an FP32 multigrid), else FP64. Returns the launch count.
int launch_gauss_jordan(double* M, int n, int* status, cudaStream_t s, bool pairs);
int gauss_jordan_launches(int n);
template <typename T> void launch_store_inverse(const double* M, int n, T* inv, cudaStream_t s);
template <typename T> void launch_coarse_solve(const LV<T>& C, const T* inv, int n, const T* f, T* u,
                                               cudaStream_t s);
template <typename T> void launch_applyA_dot(const LV<T>& L, const T* p, T* q, double* partial,
                                             cudaStream_t s);
template <typename T> void launch_dot(const LV<T>& L, const T* a, const T* b, double* partial,
                                      cudaStream_t s);
template <typename T> void launch_update_xr(const LV<T>& L, T* x, T* r, const T* p, const T* q,
                                            const double* scal, int num, int den, cudaStream_t s);
template <typename T> void launch_update_p(const LV<T>& L, T* p, const T* z, const double* scal,
                                           int num, int den, cudaStream_t s);
template <typename T> void launch_copy_level(const LV<T>& L, T* dst, const T* src, cudaStream_t s);

// the bottom of a V-cycle in one CTA (k_mg.cu): levels l0 .. L-1
constexpr int kCoarseBlockPoints = 4096;    // levels up to this size run in the persistent kernel
template <typename T>
struct CoarseSet {
    int l0, L, nc, nu1, nu2;
    LV<T> lv[16];
    T* u[16];
    T* f[16];
    T* r[16];
    const T* minv;
};
template <typename T> void launch_coarse_vcycle(const CoarseSet<T>& S, cudaStream_t s);
void coarse_vcycle_init();    // allow the shared-memory variant its dynamic shared memory (before any capture)

// dry/wet band (k_mg.cu)
template <typename T> void launch_cast_eps(long n, const double* e64, T* eT, cudaStream_t s);
template <typename T> void launch_band_eps(const Geo& g, const T* epsT, int first_interior, int band_nz,
                                           T* band_eps, cudaStream_t s);
template <typename T> void launch_band_rhs(const Geo& g, const T* epsT, const T* r, const T* evac,
                                           int first_interior, int band_nz, T* fband, cudaStream_t s);

// FGMRES inner Krylov (k_mg.cu)
constexpr int kMaxKrylov = 16;
template <typename T> struct TVecList { const T* v[kMaxKrylov]; int n; };
template <typename T> void launch_multidot(long n, const T* w, const TVecList<T>& V, double* partial, cudaStream_t s);
template <typename T> void launch_multiaxpy_norm(long n, T* w, const TVecList<T>& V, const double* h, double* partial,
                                                 cudaStream_t s);
template <typename T> void launch_scale_by_norm(long n, const T* src, T* dst, const double* sq, cudaStream_t s);
template <typename T> void launch_combine(const Geo& g, const T* ev, const T* eb, int first, int band_nz, T* z,
                                          cudaStream_t s);
template <typename T> void launch_krylov_combine(long n, T* x, const TVecList<T>& Z, const double* y, cudaStream_t s);
template <typename T> void launch_axpy1(const LV<T>& L, T* x, const T* y, cudaStream_t s);

// FFT (k_fft.cu)
struct FFTPlan;
FFTPlan* fft_create(const Geo& g, cudaStream_t s);
void fft_destroy(FFTPlan* p);
size_t fft_workspace_bytes(const Geo& g, bool dbl);
// Solve L out = src (7-point Laplacian, periodic), k = 0 mode dropped.
template <typename T> void fft_poisson(FFTPlan* p, const T* src, T* out, void* work, cudaStream_t s);

}  // namespace gp
