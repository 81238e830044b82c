// One full red-black Gauss-Seidel sweep of the finest multigrid level in a
// single pass over memory.
//
// A sweep updates the points of the first colour from the old values of the
// other colour, then the points of the second colour from the new values of
// the first. Two launches would stream u and eps twice; here each CTA owns an
// x-y tile and a chunk of z-planes and marches through them with a ring of
// four planes in shared memory:
//
//   load plane q+1 (u_old, eps, f with a 2-point x-y halo)
//   first colour, new values, at plane q on the tile plus a 1-point halo
//   second colour at plane q-1 on the tile, from those new values
//   write plane q-1 of u_new (both colours)
//
// The halo values of the first colour are recomputed by every CTA that needs
// them from u_old, which nobody writes during the sweep (u_new is a separate
// buffer), so the result is identical to the two-launch sweep. Algorithmic
// traffic: read u_old, eps, f and write u_new, 16 bytes per point in FP32.
#include "gp_common.cuh"

#include <type_traits>

namespace gp {
namespace {

constexpr int NT = 256;

constexpr int NRING = 6;                          // planes q-3 .. q+1 resident, q+2 in flight

// output tile SX x SY per CTA (z chunk set at launch) with a 2-point x-y halo
template <typename T, int SX, int SY>
struct __align__(16) Ring {
    static constexpr int HX = SX + 4, HY = SY + 4, HP = HX * HY;
    T u[NRING][HP];
    T e[NRING][HP];
    T f[NRING][HP];
    T r[4][HP];                                   // first-colour values of planes q-3 .. q-1
};

// asynchronous copy of two consecutive elements (8 bytes in FP32, 16 in FP64)
__device__ __forceinline__ void cp_async_pair(float* smem_dst, const float* gsrc) {
    const unsigned s = (unsigned)__cvta_generic_to_shared(smem_dst);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(s), "l"(gsrc));
}
__device__ __forceinline__ void cp_async_pair(double* smem_dst, const double* gsrc) {
    const unsigned s = (unsigned)__cvta_generic_to_shared(smem_dst);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 16;\n" ::"r"(s), "l"(gsrc));
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::); }
__device__ __forceinline__ void cp_async_wait1() { asm volatile("cp.async.wait_group 1;\n" ::); }

template <typename T, int SX, int SY>
__global__ void __launch_bounds__(NT) k_rb_sweep(LV<T> L, const T* __restrict__ u_old, const T* __restrict__ f,
                                                 T* __restrict__ u_new, int first, int sz) {
    extern __shared__ unsigned char smem_raw[];
    using RingT = Ring<T, SX, SY>;
    constexpr int HX = RingT::HX, HP = RingT::HP;
    RingT& R = *reinterpret_cast<RingT*>(smem_raw);
    const int nx = L.nx, ny = L.ny, nz = L.nz;
    const long pl = (long)nx * ny;
    const int i0 = blockIdx.x * SX, j0 = blockIdx.y * SY;
    const int z0 = blockIdx.z * sz;
    const int z1 = min(z0 + sz, nz);
    if (z0 >= nz) return;
    const T cx = (T)0.5 * L.ihx2, cy = (T)0.5 * L.ihy2, cz = (T)0.5 * L.ihz2;
    const int second = 1 - first;
    const int tid = threadIdx.x;

    // This thread copies x-pairs of the halo tile: pair p covers cells (2p, 2p+1)
    // of the tile. Its in-plane global offset (periodic wrap; nx even keeps
    // pairs whole) is computed once.
    constexpr int NPAIR = HP / 2;
    constexpr int NL = (NPAIR + NT - 1) / NT;
    int off[NL];
#pragma unroll
    for (int r = 0; r < NL; ++r) {
        const int p = tid + r * NT;
        off[r] = -1;
        if (p < NPAIR) {
            const int t = 2 * p;
            const int dy = t / HX - 2, dx = t % HX - 2;
            const int i = ((i0 + dx) % nx + nx) % nx, j = ((j0 + dy) % ny + ny) % ny;
            off[r] = j * nx + i;
        }
    }

    auto issue_plane = [&](int q) {
        if (q > z1 + 1) { cp_async_commit(); return; }
        const int slot = (q + 60) % NRING;
        int kg;
        if (L.zper) kg = q < 0 ? q + nz : (q >= nz ? q - nz : q);
        else kg = (q < -1 || q > nz) ? -99 : q;
        const bool inner = kg >= 0 && kg < nz;
        const long base = (long)kg * pl;
#pragma unroll
        for (int r = 0; r < NL; ++r) {
            if (off[r] < 0) continue;
            const int t = 2 * (tid + r * NT);
            if (kg != -99) {
                cp_async_pair(&R.u[slot][t], u_old + base + off[r]);
                cp_async_pair(&R.e[slot][t], L.eps + base + off[r]);
            } else {
                R.u[slot][t] = 0; R.u[slot][t + 1] = 0;
                R.e[slot][t] = 1; R.e[slot][t + 1] = 1;
            }
            if (inner) cp_async_pair(&R.f[slot][t], f + base + off[r]);
            else { R.f[slot][t] = 0; R.f[slot][t + 1] = 0; }
        }
        cp_async_commit();
    };

    // Gauss-Seidel value at smem cell c of plane slot s0 (neighbour planes sm, sp)
    auto gs_update = [&](int c, int s0, int sm, int sp, const T* srcm, const T* src, const T* srcp) -> T {
        const T e0 = R.e[s0][c];
        const T axm = (e0 + R.e[s0][c - 1]) * cx, axp = (e0 + R.e[s0][c + 1]) * cx;
        const T aym = (e0 + R.e[s0][c - HX]) * cy, ayp = (e0 + R.e[s0][c + HX]) * cy;
        const T azm = (e0 + R.e[sm][c]) * cz, azp = (e0 + R.e[sp][c]) * cz;
        const T s = axm * src[c - 1] + axp * src[c + 1] + aym * src[c - HX] + ayp * src[c + HX] + azm * srcm[c] +
                    azp * srcp[c];
        const T d = axm + axp + aym + ayp + azm + azp;
        if constexpr (sizeof(T) == 4) return __fdividef(s - R.f[s0][c], d);
        else return (s - R.f[s0][c]) / d;
    };

    constexpr int HALF1 = (SX + 2) / 2;              // first-colour points per halo-1 row
    constexpr int NF = HALF1 * (SY + 2);             // first-colour points on the halo-1 tile
    issue_plane(z0 - 2);
    for (int q = z0 - 2; q <= z1 + 1; ++q) {
        issue_plane(q + 1);                          // prefetch the next plane
        cp_async_wait1();                            // this thread's copies of plane q landed
        __syncthreads();                             // ... and everyone's
        const int qf = q - 1;                        // first colour, new values, at plane qf
        if (qf >= z0 - 1 && qf <= z1) {
            const int s0 = (qf + 60) % NRING, sm = (qf + 59) % NRING, sp = (qf + 61) % NRING;
            const int r0 = (qf + 8) & 3;
            const bool wall = !L.zper && (qf == -1 || qf == nz);
            for (int t = tid; t < NF; t += NT) {
                const int dy = t / HALF1 - 1, m = t % HALF1;
                const int p = (first - (i0 - 1 + j0 + dy + qf)) & 1;
                const int dx = -1 + 2 * m + p;
                const int c = (dy + 2) * HX + (dx + 2);
                R.r[r0][c] = wall ? R.u[s0][c] : gs_update(c, s0, sm, sp, R.u[sm], R.u[s0], R.u[sp]);
            }
        }
        __syncthreads();
        const int qs = q - 2;                        // second colour, and the output plane
        if (qs >= z0 && qs < z1) {
            const int s0 = (qs + 60) % NRING, sm = (qs + 59) % NRING, sp = (qs + 61) % NRING;
            const int r0 = (qs + 8) & 3, rm = (qs + 7) & 3, rp = (qs + 9) & 3;
            for (int t = tid; t < (SX / 2) * SY; t += NT) {
                const int dy = t / (SX / 2), m = t % (SX / 2);
                const int i = i0 + 2 * m, j = j0 + dy;
                if (i >= nx || j >= ny) continue;
                const int c0 = (dy + 2) * HX + (2 * m + 2);        // even member of the x pair
                const int p2 = (second - (i + j + qs)) & 1;        // which member has the second colour
                const int cs = c0 + p2, cf = c0 + 1 - p2;
                const T vs = gs_update(cs, s0, sm, sp, R.r[rm], R.r[r0], R.r[rp]);
                const T vf = R.r[r0][cf];
                T* out = u_new + (long)qs * pl + (long)j * nx + i;
                out[0] = p2 ? vf : vs;
                out[1] = p2 ? vs : vf;
            }
        }
    }
}

// ---------------------------------------------------------------------------
// Row-tile variant (FP32): a CTA owns whole x rows (nx = 2 NPX points) times
// SY rows in y and a chunk of z-planes, so the only halo is one row in y (the
// x neighbours wrap inside the tile). One thread per x-pair (2p, 2p+1) and
// row; the thread keeps its own column's values of the neighbouring planes in
// registers while it marches in z, so shared memory serves only the in-plane
// neighbours (64-bit accesses, consecutive lanes on consecutive pairs).
//
// In a pair one member has each colour. With m1 = (j + q + first) & 1 the
// member of the first colour at plane q, the member of the second colour at
// plane q-1 is again m1. Iteration q:
//   A(q)   first colour at plane q, rows j0-1 .. j0+SY (the halo rows
//          recomputed from u_old), value kept in a register and in a 2-plane
//          shared ring;
//   B(q-1) second colour at plane q-1, rows j0 .. j0+SY-1, from the new
//          first-colour values at planes q-2, q-1, q; writes plane q-1 of u_new.
// Planes of u_old, eps and f arrive by TMA bulk copies (one per row, whole
// rows are contiguous in memory) NSLOT-1 planes ahead into an NSLOT ring, each
// slot completing an mbarrier phase. Warp 0 waits on the phase and the CTA
// barrier releases the others. Every wait is bounded: on expiry the kernel
// records the fact in *err and runs to its end without further waits.
constexpr int NSLOT = 6;

// polls per phase wait in the main loop of the row sweep (the exit drain always
// uses the default); lowered only to test the expiry path
int g_wait_polls = 1 << 20;

template <int NPX, int SY>
struct RowRing {
    static constexpr int RU = SY + 4, RF = SY + 2;
    float2 u[NSLOT][RU][NPX];
    float2 e[NSLOT][RU][NPX];
    float2 f[NSLOT][RF][NPX];
    float2 r[2][RF][NPX];
    unsigned long long bar[NSLOT];
};

__device__ __forceinline__ int wrap_idx(int v, int n) { return v < 0 ? v + n : (v >= n ? v - n : v); }

__device__ __forceinline__ unsigned smem_u32(const void* p) { return (unsigned)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(unsigned long long* bar, unsigned count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(smem_u32(bar)), "r"(count));
}
__device__ __forceinline__ void mbar_arrive_tx(unsigned long long* bar, unsigned bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}
// true once the phase with this parity has completed
__device__ __forceinline__ bool mbar_test(unsigned long long* bar, unsigned parity) {
    unsigned ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}
// bounded wait (`limit` polls, about a second for the default); false if it gave up
constexpr int kWaitPolls = 1 << 20;
__device__ __forceinline__ bool mbar_wait(unsigned long long* bar, unsigned parity, int limit = kWaitPolls) {
    for (int it = 0; it < limit; ++it)
        if (mbar_test(bar, parity)) return true;
    return false;
}
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, unsigned bytes, unsigned long long* bar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];\n" ::"r"(
            smem_u32(dst)),
        "l"(src), "r"(bytes), "r"(smem_u32(bar))
        : "memory");
}

// resident CTAs per SM the row kernel is built for: by shared memory, and by
// registers at 64 per thread (it needs about 60), at most 4
template <int NPX, int SY>
constexpr int rows_min_blocks() {
    constexpr int by_regs = 1024 / (NPX * (SY + 2));
    constexpr int by_smem = (int)((227 * 1024) / (sizeof(RowRing<NPX, SY>) + 1024));
    constexpr int m = by_regs < by_smem ? by_regs : by_smem;
    return m < 1 ? 1 : (m > 4 ? 4 : m);
}

template <int NPX, int SY>
__global__ void __launch_bounds__(NPX * (SY + 2), rows_min_blocks<NPX, SY>())
    k_rb_sweep_rows(LV<float> L, const float* __restrict__ u_old, const float* __restrict__ f,
                    float* __restrict__ u_new, int first, int sz, int* err, int wait_limit) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    using RR = RowRing<NPX, SY>;
    constexpr int NTH = NPX * (SY + 2), RU = RR::RU, RF = RR::RF;
    constexpr unsigned ROWB = NPX * 8;                    // bytes of one row
    RR& R = *reinterpret_cast<RR*>(smem_raw);
    __shared__ int bad;
    const int nx = 2 * NPX, ny = L.ny, nz = L.nz;
    const long pl = (long)nx * ny;
    const int j0 = blockIdx.y * SY;
    const int z0 = blockIdx.z * sz;
    const int z1 = min(z0 + sz, nz);
    if (z0 >= nz) return;
    const float cx = 0.5f * L.ihx2, cy = 0.5f * L.ihy2, cz = 0.5f * L.ihz2;
    const int tid = threadIdx.x;
    const int ra = tid / NPX, p = tid % NPX;
    const int pm = p == 0 ? NPX - 1 : p - 1, pp = p == NPX - 1 ? 0 : p + 1;
    const int jB = j0 + ra - 1;
    const bool doB = ra >= 1 && ra <= SY && jB < ny;
    const int parA = (j0 - 1 + ra + first + 2 * ny) & 1;   // m1 = (parA + q) & 1
    const int qb = z0 - 2;                                  // first plane of the march

    if (tid == 0) {
        bad = 0;
        for (int k = 0; k < NSLOT; ++k) mbar_init(&R.bar[k], 1);
        asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
    }
    __syncthreads();

    // plane q into slot (q - qb) % NSLOT: warp 0 issues one bulk copy per row;
    // planes outside the data (beyond the Dirichlet walls, f on the walls) are
    // filled by the threads with plain stores instead
    int last_issued = -1;                                 // local index of the last plane sent (uniform)
    int waited = -1;                                      // warp 0: planes <= this one have landed
    auto issue = [&](int q) {
        if (q > z1 + 1 || bad) return;                    // after an expired wait nothing new is sent
        const int slot = (q - qb) % NSLOT;
        last_issued = q - qb;
        int kg;
        if (L.zper) kg = q < 0 ? q + nz : (q >= nz ? q - nz : q);
        else kg = (q < -1 || q > nz) ? -99 : q;
        const bool has_ue = kg != -99, inner = kg >= 0 && kg < nz;
        if (tid < 32) {
            const unsigned bytes = (has_ue ? 2u * RU * ROWB : 0u) + (inner ? (unsigned)RF * ROWB : 0u);
            if (tid == 0) {
                asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
                mbar_arrive_tx(&R.bar[slot], bytes);
            }
            __syncwarp();
            const long base = (long)kg * pl;
            if (has_ue)
                for (int r = tid; r < 2 * RU; r += 32) {
                    const int rr = r < RU ? r : r - RU;
                    const long off = base + (long)wrap_idx(j0 - 2 + rr, ny) * nx;
                    if (r < RU) bulk_g2s(&R.u[slot][rr][0], u_old + off, ROWB, &R.bar[slot]);
                    else bulk_g2s(&R.e[slot][rr][0], L.eps + off, ROWB, &R.bar[slot]);
                }
            if (inner)
                for (int r = tid; r < RF; r += 32)
                    bulk_g2s(&R.f[slot][r][0], f + base + (long)wrap_idx(j0 - 1 + r, ny) * nx, ROWB, &R.bar[slot]);
        }
        if (!has_ue)
            for (int t = tid; t < RU * NPX; t += NTH) {
                (&R.u[slot][0][0])[t] = make_float2(0.f, 0.f);
                (&R.e[slot][0][0])[t] = make_float2(1.f, 1.f);
            }
        if (!inner) (&R.f[slot][0][0])[tid] = make_float2(0.f, 0.f);
    };
    auto wait_plane = [&](int q) {            // warp 0 only
        const int t = q - qb;
        if (bad) return;
        if (mbar_wait(&R.bar[t % NSLOT], (unsigned)((t / NSLOT) & 1), wait_limit)) waited = t;
        else bad = 1;
    };

    float2 U_m = make_float2(0.f, 0.f), U_0 = U_m;          // own u_old at q-1, q
    float2 E_m2 = make_float2(1.f, 1.f), E_m = E_m2, E_0 = E_m2;  // own eps at q-2, q-1, q
    float2 F_m = make_float2(0.f, 0.f);                      // own f at q-1
    float R_m2 = 0.f, R_m = 0.f;                             // own first-colour values at q-2, q-1
    float bxl = 1.f, bxr = 1.f;                              // eps x-neighbours at q-1 (for B)
    float2 bym = make_float2(1.f, 1.f), byp = bym;           // eps rows j-1, j+1 at q-1 (for B)
    const int rs = ra + 1;                                   // this thread's row in the u / e arrays

    for (int k = 0; k < NSLOT - 1; ++k) issue(qb + k);
    for (int q = qb; q <= z1; ++q) {
        if (tid < 32) {
            if (q == qb) wait_plane(q);
            wait_plane(q + 1);                             // planes <= q+1 landed
        }
        __syncthreads();                                   // ... seen by all; every thread done with slot q-1
        issue(q + NSLOT - 1);                              // into the slot of plane q-1
        const int s0 = (q - qb) % NSLOT, s1 = (q + 1 - qb) % NSLOT;
        if (q == qb) {                                     // prime the z window: own values at z0-2, z0-1
            U_m = R.u[s0][rs][p];
            E_m = R.e[s0][rs][p];
            U_0 = R.u[s1][rs][p];
            E_0 = R.e[s1][rs][p];
            continue;
        }
        // ---- A(q): first colour at plane q, member m1 of the own pair; then
        // B(q-1): second colour at plane q-1 (member m1 again). m1 is uniform
        // along a row, so both members get their own straight-line code.
        const float2 U_p = R.u[s1][rs][p];                 // own at q+1
        const float2 E_p = R.e[s1][rs][p];
        const float2 F_0 = R.f[s0][ra][p];
        const float2 Exm = R.e[s0][rs][pm], Exp = R.e[s0][rs][pp];
        const float2 Eym = R.e[s0][rs - 1][p], Eyp = R.e[s0][rs + 1][p];
        const bool wall = !L.zper && (q == -1 || q == nz);
        const bool runB = q - 1 >= z0 && doB;
        float rA;
        auto step = [&](auto mc) {
            constexpr int M = decltype(mc)::value;
            auto pick = [](float2 v) { return M ? v.y : v.x; };
            {
                const float uxa = M ? R.u[s0][rs][pp].x : R.u[s0][rs][pm].y;   // x neighbour outside the pair
                const float uym = pick(R.u[s0][rs - 1][p]), uyp = pick(R.u[s0][rs + 1][p]);
                const float e0 = pick(E_0);
                const float exl = M ? E_0.x : Exm.y, exr = M ? Exp.x : E_0.y;
                const float uxl = M ? U_0.x : uxa, uxr = M ? uxa : U_0.y;
                const float axm = (e0 + exl) * cx, axp = (e0 + exr) * cx;
                const float aym = (e0 + pick(Eym)) * cy, ayp = (e0 + pick(Eyp)) * cy;
                const float azm = (e0 + pick(E_m)) * cz, azp = (e0 + pick(E_p)) * cz;
                const float sum = axm * uxl + axp * uxr + aym * uym + ayp * uyp + azm * pick(U_m) + azp * pick(U_p);
                const float d = axm + axp + aym + ayp + azm + azp;
                rA = wall ? pick(U_0) : __fdividef(sum - pick(F_0), d);
            }
            R.r[q & 1][ra][p] = M ? make_float2(0.f, rA) : make_float2(rA, 0.f);
            if (runB) {
                const int sr = (q - 1) & 1;
                const float rxa = M ? R.r[sr][ra][pp].x : R.r[sr][ra][pm].y;    // neighbour outside the pair
                const float ry_m = pick(R.r[sr][ra - 1][p]), ry_p = pick(R.r[sr][ra + 1][p]);
                const float e0 = pick(E_m);
                const float exl = M ? E_m.x : bxl, exr = M ? bxr : E_m.y;
                const float rxl = M ? R_m : rxa, rxr = M ? rxa : R_m;
                const float axm = (e0 + exl) * cx, axp = (e0 + exr) * cx;
                const float aym = (e0 + pick(bym)) * cy, ayp = (e0 + pick(byp)) * cy;
                const float azm = (e0 + pick(E_m2)) * cz, azp = (e0 + pick(E_0)) * cz;
                const float sum = axm * rxl + axp * rxr + aym * ry_m + ayp * ry_p + azm * R_m2 + azp * rA;
                const float d = axm + axp + aym + ayp + azm + azp;
                const float vB = __fdividef(sum - pick(F_m), d);
                float2* out = reinterpret_cast<float2*>(u_new + (long)(q - 1) * pl + (long)jB * nx) + p;
                *out = M ? make_float2(R_m, vB) : make_float2(vB, R_m);
            }
        };
        if ((parA + q) & 1) step(std::integral_constant<int, 1>{});
        else step(std::integral_constant<int, 0>{});
        // ---- shift the z window; keep the eps neighbours at q for B(q) (the other member)
        bxl = Exm.y; bxr = Exp.x; bym = Eym; byp = Eyp;
        U_m = U_0; U_0 = U_p;
        E_m2 = E_m; E_m = E_0; E_0 = E_p;
        F_m = F_0;
        R_m2 = R_m; R_m = rA;
    }
    __syncthreads();
    if (tid == 0 && bad) {
        // a wait expired: give the copies still in flight (planes after the last one
        // that landed, up to the last one sent) a bounded chance to land before the CTA exits
        for (int t = waited + 1; t <= last_issued; ++t) mbar_wait(&R.bar[t % NSLOT], (unsigned)((t / NSLOT) & 1));
        if (err) atomicExch(err, 1);
    }
}

template <int NPX, int SY>
void sweep_rows(const LV<float>& L, const float* u_old, const float* f, float* u_new, int first, cudaStream_t s,
                bool attr, int* err) {
    const size_t sm = sizeof(RowRing<NPX, SY>);
    if (attr) {
        cudaFuncSetAttribute(k_rb_sweep_rows<NPX, SY>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
        return;
    }
    // z chunks so that y tiles x chunks fill one wave of resident CTAs
    const int per_sm = rows_min_blocks<NPX, SY>();
    const int ty = (L.ny + SY - 1) / SY;
    int chunks = 152 * per_sm / ty;
    if (chunks < 1) chunks = 1;
    if (chunks > L.nz) chunks = L.nz;
    const int sz = (L.nz + chunks - 1) / chunks;
    dim3 grid(1, ty, (L.nz + sz - 1) / sz);
    k_rb_sweep_rows<NPX, SY><<<grid, NPX * (SY + 2), sm, s>>>(L, u_old, f, u_new, first, sz, err, g_wait_polls);
}

// ---------------------------------------------------------------------------
// Warp-specialised row-tile variant (FP32). Same tile as above (whole x rows,
// SY output rows, a chunk of z-planes), but the loop has no CTA barrier:
//   * one producer warp streams planes of u_old and eps into an NSW-slot
//     ring with bulk copies, one row per copy; slot s completes phase
//     `full[s]` when its bytes have landed; f does not pass through the ring:
//     each consumer thread loads its own f values one plane ahead;
//   * the consumer threads own a pair column (2p, 2p+1) over K adjacent rows,
//     so the y neighbours inside the K rows and the z neighbours come from
//     registers; shared memory serves the x neighbour outside the pair and
//     the rows just above and below the K rows;
//   * iteration t handles plane q = qb + t: the first colour at q (A), whose
//     values go to an NRW-plane ring `r`, then the second colour at q-1 (B).
//     Each consumer warp arrives on `rdy[t % NRW]` right after A(t), by which
//     point it has also read everything it needs from the slot of plane t.
//     B waits for rdy(t-1): every first-colour value of plane q-1 is in `r`.
//     The producer refills the slot of plane t only once rdy(t) completed.
// A warp that writes r(t) has seen rdy(t-2), so every warp has finished
// iteration t-3 and with it B(t-4), the last reader of the slot r(t) reuses
// (NRW = 4). The producer is at most NSW - 1 planes ahead of the slowest warp,
// and no barrier can complete a phase twice while a waiter still polls the
// older one, so the parity waits never alias.
constexpr int NSW = 4, NRW = 4;

template <int NPX, int SY>
struct WsRing {
    static constexpr int RU = SY + 4, RF = SY + 2;
    float2 u[NSW][RU][NPX];
    float2 e[NSW][RU][NPX];
    float r[NRW][RF][NPX];
    unsigned long long full[NSW];
    unsigned long long rdy[NRW];
};

template <int NPX, int SY, int K>
constexpr int ws_threads() { return NPX * ((SY + 2) / K) + 32; }

// resident CTAs per SM the tile is built for: as many as shared memory and
// the registers the consumers' z window wants (about 72 per thread for two
// rows, 128 for three or four) allow, at most two; and the register ceiling per
// thread that lets that many reside: the register file is split evenly over the
// four schedulers (16384 each) and a warp's registers come from one of them,
// in 8-register steps. The host reads the residency back from the occupancy
// calculator.
template <int NPX, int SY, int K>
constexpr int ws_min_blocks() {
    constexpr int by_smem = (int)((227 * 1024) / (sizeof(WsRing<NPX, SY>) + 1024));
    constexpr int by_regs = 65536 / ((K <= 2 ? 72 : 128) * ws_threads<NPX, SY, K>());
    constexpr int m = by_smem < by_regs ? by_smem : by_regs;
    return m < 1 ? 1 : (m > 2 ? 2 : m);
}
template <int NPX, int SY, int K>
constexpr int ws_max_regs() {
    constexpr int warps = ws_min_blocks<NPX, SY, K>() * ((ws_threads<NPX, SY, K>() + 31) / 32);
    constexpr int r = (16384 / ((warps + 3) / 4) / 32) / 8 * 8;
    return r > 255 ? 255 : r;
}

// 1/x with the hardware reciprocal (about 1 ulp): the Gauss-Seidel value
// only feeds the next iteration of a smoother, and this is several
// instructions shorter than a full-range divide
__device__ __forceinline__ float rcp_approx(float x) {
    float r;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}

__device__ __forceinline__ void mbar_arrive(unsigned long long* bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];\n" ::"r"(smem_u32(bar)) : "memory");
}

template <int NPX, int SY, int K>
__global__ void __maxnreg__((ws_max_regs<NPX, SY, K>()))
    k_rb_sweep_ws(LV<float> L, const float* __restrict__ u_old, const float* __restrict__ f,
                  float* __restrict__ u_new, int first, int sz, int* err, int wait_limit) {
    static_assert((SY + 2) % K == 0, "K must divide the A rows");
    constexpr int G = (SY + 2) / K, NC = NPX * G, NWC = NC / 32;
    static_assert(NC % 32 == 0, "consumer threads must fill whole warps");
    extern __shared__ __align__(16) unsigned char smem_raw[];
    using WR = WsRing<NPX, SY>;
    constexpr int RU = WR::RU;
    constexpr unsigned ROWB = NPX * 8;
    WR& R = *reinterpret_cast<WR*>(smem_raw);
    __shared__ volatile int bad;
    const int nx = 2 * NPX, ny = L.ny, nz = L.nz;
    const long pl = (long)nx * ny;
    const int j0 = blockIdx.y * SY;
    const int z0 = blockIdx.z * sz;
    const int z1 = min(z0 + sz, nz);
    if (z0 >= nz) return;
    const int qb = z0 - 2;
    const int T = z1 + 2 - qb;                       // planes qb .. z1+1; iterations 0 .. T-2
    const int tid = threadIdx.x;
    // u_old == null: the sweep starts from u = 0 (the first sweep of a V-cycle):
    // the u ring is zeroed once here and only eps is copied
    const bool zu = u_old == nullptr;

    if (tid == 0) {
        bad = 0;
        for (int k = 0; k < NSW; ++k) mbar_init(&R.full[k], 1);
        for (int k = 0; k < NRW; ++k) mbar_init(&R.rdy[k], NWC);
        asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
    }
    if (zu)
        for (int x = tid; x < NSW * RU * NPX; x += blockDim.x) (&R.u[0][0][0])[x] = make_float2(0.f, 0.f);
    __syncthreads();

    if (tid >= NC) {
        // ---------------- producer warp
        const int lane = tid - NC;
        int issued = 0;                              // planes 0 .. issued-1 sent
        for (int t = 0; t < T; ++t) {
            if (t >= NSW) {                          // slot of plane t - NSW: every warp done with iteration t - NSW
                const int i = t - NSW;
                bool ok = !bad && mbar_wait(&R.rdy[i % NRW], (unsigned)((i / NRW) & 1), wait_limit);
                ok = __shfl_sync(0xffffffffu, ok ? 1 : 0, 0) != 0;
                if (!ok) { if (lane == 0) bad = 1; break; }
            }
            const int q = qb + t, slot = t % NSW;
            int kg;
            if (L.zper) kg = q < 0 ? q + nz : (q >= nz ? q - nz : q);
            else kg = (q < -1 || q > nz) ? -99 : q;
            const bool has_ue = kg != -99;
            if (!has_ue)
                for (int x = lane; x < RU * NPX; x += 32) {
                    (&R.u[slot][0][0])[x] = make_float2(0.f, 0.f);
                    (&R.e[slot][0][0])[x] = make_float2(1.f, 1.f);
                }
            __syncwarp();
            const unsigned bytes = has_ue ? (zu ? 1u : 2u) * RU * ROWB : 0u;
            if (lane == 0) {
                asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
                mbar_arrive_tx(&R.full[slot], bytes);
            }
            __syncwarp();
            const long base = (long)kg * pl;
            if (has_ue)
                for (int r = zu ? RU + lane : lane; r < 2 * RU; r += 32) {
                    const int rr = r < RU ? r : r - RU;
                    const long off = base + (long)wrap_idx(j0 - 2 + rr, ny) * nx;
                    if (r < RU) bulk_g2s(&R.u[slot][rr][0], u_old + off, ROWB, &R.full[slot]);
                    else bulk_g2s(&R.e[slot][rr][0], L.eps + off, ROWB, &R.full[slot]);
                }
            issued = t + 1;
        }
        // every copy sent must land before the CTA may exit (bounded, default limit)
        if (lane == 0) {
            for (int t = issued - NSW < 0 ? 0 : issued - NSW; t < issued; ++t)
                if (!mbar_wait(&R.full[t % NSW], (unsigned)((t / NSW) & 1))) bad = 1;
            if (bad && err) atomicExch(err, 1);
        }
        return;
    }

    // ---------------- consumer threads
    const float cx = 0.5f * L.ihx2, cy = 0.5f * L.ihy2, cz = 0.5f * L.ihz2;
    const int g = tid / NPX, p = tid % NPX;
    const int pm = p == 0 ? NPX - 1 : p - 1, pp = p == NPX - 1 ? 0 : p + 1;
    const int a0 = g * K;                            // first A row (A row a is global row j0 - 1 + a)
    const int par0 = (j0 - 1 + a0 + first + 2 * ny) & 1;   // member of the first colour at row a0: (par0 + q) & 1
    const int lane = tid & 31;
    unsigned bmask = 0;                              // rows k whose second colour this thread writes
#pragma unroll
    for (int k = 0; k < K; ++k)
        if (a0 + k >= 1 && a0 + k <= SY && j0 - 1 + a0 + k < ny) bmask |= 1u << k;
    const int obase = (j0 - 1 + a0) * NPX + p;       // float2 index of row a0, pair p, in a plane
    // f has no neighbour terms: each thread reads its own rows with plain loads,
    // one plane ahead, which keeps a third of the bytes off the bulk copies
    int frow[K];
#pragma unroll
    for (int k = 0; k < K; ++k) frow[k] = (wrap_idx(j0 - 1 + a0 + k, ny) * NPX + p) * 2;
    auto load_f = [&](int q, float2 (&F)[K]) {
        int kg;
        if (L.zper) kg = q < 0 ? q + nz : (q >= nz ? q - nz : q);
        else kg = q;
        const bool inner = kg >= 0 && kg < nz;
        const float* fp = f + (long)(inner ? kg : 0) * pl;
#pragma unroll
        for (int k = 0; k < K; ++k)
            F[k] = inner ? __ldg(reinterpret_cast<const float2*>(fp + frow[k])) : make_float2(0.f, 0.f);
    };
    bool live = true;                                // false once a wait has expired
    auto wait_full = [&](int t) {
        if (!live) return;
        if (bad || !mbar_wait(&R.full[t % NSW], (unsigned)((t / NSW) & 1), wait_limit)) { live = false; bad = 1; }
    };
    auto wait_rdy = [&](int i) {
        if (!live) return;
        if (bad || !mbar_wait(&R.rdy[i % NRW], (unsigned)((i / NRW) & 1), wait_limit)) { live = false; bad = 1; }
    };
    auto arrive = [&](int i) {
        __syncwarp();
        if (lane == 0) mbar_arrive(&R.rdy[i % NRW]);
    };

    // The member a later use needs is known when a value arrives (the colours
    // alternate along z), so values used once more are kept as that member only.
    float um[K];                                     // own u_old at q-1, member of the first colour at q
    float2 U_0[K];                                   // own u_old at q
    float em2[K];                                    // own eps at q-2, member of the second colour at q-1
    float2 E_m[K], E_0[K];                           // own eps at q-1, q
    float fm[K];                                     // own f at q-1, member of the second colour there
    float2 F_0[K];                                   // own f at q
    float R_m2[K], R_m[K];                           // own first-colour values at q-2, q-1
    float bx[K];                                     // eps at q-1 next to that member, outside the pair
    float bylo = 1.f, byhi = 1.f;                    // eps rows a0-1, a0+K at q-1, same member
    {
        wait_full(0);
        wait_full(1);
        const int m0 = (par0 + qb + 1) & 1;          // first-colour member of row a0 at plane qb+1
        load_f(qb + 1, F_0);
#pragma unroll
        for (int k = 0; k < K; ++k) {
            const float2 u0 = R.u[0][a0 + k + 1][p];
            um[k] = (m0 ^ (k & 1)) ? u0.y : u0.x;
            E_m[k] = R.e[0][a0 + k + 1][p];
            U_0[k] = R.u[1][a0 + k + 1][p];
            E_0[k] = R.e[1][a0 + k + 1][p];
            em2[k] = 1.f; fm[k] = 0.f; bx[k] = 1.f;
            R_m2[k] = 0.f; R_m[k] = 0.f;
        }
        arrive(0);
    }
    // one iteration; M0, the first-colour member of row a0, alternates with the
    // plane, so the loop runs two iterations per trip with M0 fixed in each and
    // the z window rotates through registers without copies
    auto iter = [&](const int t, auto mc) {
        const int q = qb + t;
        wait_full(t + 1);
        const unsigned tu = (unsigned)t;
        const int s0 = tu % NSW, s1 = (tu + 1) % NSW, rw = tu % NRW, rr = (tu - 1) % NRW;
        const bool wall = !L.zper && (q == -1 || q == nz);
        const bool runB = q - 1 >= z0;
        {
            constexpr int M0 = decltype(mc)::value;
            float2 U_p[K], E_p[K], F_p[K];
            load_f(q + 1, F_p);                      // used by the next iteration
            float exm[K], exq[K], rA[K];
#pragma unroll
            for (int k = 0; k < K; ++k) {
                U_p[k] = R.u[s1][a0 + k + 1][p];
                E_p[k] = R.e[s1][a0 + k + 1][p];
                exm[k] = R.e[s0][a0 + k + 1][pm].y;
                exq[k] = R.e[s0][a0 + k + 1][pp].x;
            }
            const float2 elo = R.e[s0][a0][p], ehi = R.e[s0][a0 + K + 1][p];
            // ---- A(q): first colour at plane q, rows a0 .. a0+K-1 (member M of the pair)
#pragma unroll
            for (int k = 0; k < K; ++k) {
                const int M = M0 ^ (k & 1);
                auto pick = [M](float2 v) { return M ? v.y : v.x; };
                const float uxa = M ? R.u[s0][a0 + k + 1][pp].x : R.u[s0][a0 + k + 1][pm].y;
                const float e0 = pick(E_0[k]);
                const float exl = M ? E_0[k].x : exm[k], exr = M ? exq[k] : E_0[k].y;
                const float uxl = M ? U_0[k].x : uxa, uxr = M ? uxa : U_0[k].y;
                const float eyl = k == 0 ? pick(elo) : pick(E_0[k - 1 < 0 ? 0 : k - 1]);
                const float eyh = k == K - 1 ? pick(ehi) : pick(E_0[k + 1 < K ? k + 1 : K - 1]);
                const float uyl = k == 0 ? (M ? R.u[s0][a0][p].y : R.u[s0][a0][p].x)
                                         : pick(U_0[k - 1 < 0 ? 0 : k - 1]);
                const float uyh = k == K - 1 ? (M ? R.u[s0][a0 + K + 1][p].y : R.u[s0][a0 + K + 1][p].x)
                                             : pick(U_0[k + 1 < K ? k + 1 : K - 1]);
                const float axm = (e0 + exl) * cx, axp = (e0 + exr) * cx;
                const float aym = (e0 + eyl) * cy, ayp = (e0 + eyh) * cy;
                const float azm = (e0 + pick(E_m[k])) * cz, azp = (e0 + pick(E_p[k])) * cz;
                const float sum = axm * uxl + axp * uxr + aym * uyl + ayp * uyh + azm * um[k] + azp * pick(U_p[k]);
                const float d = axm + axp + aym + ayp + azm + azp;
                rA[k] = wall ? pick(U_0[k]) : (sum - pick(F_0[k])) * rcp_approx(d);
                R.r[rw][a0 + k][p] = rA[k];
            }
            arrive(t);
            // ---- B(q-1): second colour at plane q-1 (the same members)
            wait_rdy(t - 1);
            if (runB) {
                float2* ob = reinterpret_cast<float2*>(u_new + (long)(q - 1) * pl) + obase;
#pragma unroll
                for (int k = 0; k < K; ++k) {
                    const int a = a0 + k;
                    if (!(bmask & (1u << k))) continue;
                    const int M = M0 ^ (k & 1);
                    auto pick = [M](float2 v) { return M ? v.y : v.x; };
                    const float rxa = M ? R.r[rr][a][pp] : R.r[rr][a][pm];
                    const float ryl = k == 0 ? R.r[rr][a - 1][p] : R_m[k - 1 < 0 ? 0 : k - 1];
                    const float ryh = k == K - 1 ? R.r[rr][a + 1][p] : R_m[k + 1 < K ? k + 1 : K - 1];
                    const float e0 = pick(E_m[k]);
                    const float exl = M ? E_m[k].x : bx[k], exr = M ? bx[k] : E_m[k].y;
                    const float rxl = M ? R_m[k] : rxa, rxr = M ? rxa : R_m[k];
                    const float eyl = k == 0 ? bylo : pick(E_m[k - 1 < 0 ? 0 : k - 1]);
                    const float eyh = k == K - 1 ? byhi : pick(E_m[k + 1 < K ? k + 1 : K - 1]);
                    const float axm = (e0 + exl) * cx, axp = (e0 + exr) * cx;
                    const float aym = (e0 + eyl) * cy, ayp = (e0 + eyh) * cy;
                    const float azm = (e0 + em2[k]) * cz, azp = (e0 + pick(E_0[k])) * cz;
                    const float sum = axm * rxl + axp * rxr + aym * ryl + ayp * ryh + azm * R_m2[k] + azp * rA[k];
                    const float d = axm + axp + aym + ayp + azm + azp;
                    const float vB = (sum - fm[k]) * rcp_approx(d);
                    ob[k * NPX] = M ? make_float2(R_m[k], vB) : make_float2(vB, R_m[k]);
                }
            }
            // ---- shift the z window. At plane q+1 the members swap: the first
            // colour of row k is member 1-M, which is also the member B(q) uses.
            bylo = M0 ? elo.x : elo.y;
            byhi = (M0 ^ ((K - 1) & 1)) ? ehi.x : ehi.y;
#pragma unroll
            for (int k = 0; k < K; ++k) {
                const int M = M0 ^ (k & 1);
                bx[k] = M ? exm[k] : exq[k];
                um[k] = M ? U_0[k].x : U_0[k].y;
                U_0[k] = U_p[k];
                em2[k] = M ? E_m[k].x : E_m[k].y;
                E_m[k] = E_0[k]; E_0[k] = E_p[k];
                fm[k] = M ? F_0[k].x : F_0[k].y;
                F_0[k] = F_p[k];
                R_m2[k] = R_m[k]; R_m[k] = rA[k];
            }
        }
    };
    using I0 = std::integral_constant<int, 0>;
    using I1 = std::integral_constant<int, 1>;
    int t = 1;
    if ((par0 + qb + 1) & 1) {
        for (; t + 1 <= T - 2; t += 2) { iter(t, I1{}); iter(t + 1, I0{}); }
        if (t <= T - 2) iter(t, I1{});
    } else {
        for (; t + 1 <= T - 2; t += 2) { iter(t, I0{}); iter(t + 1, I1{}); }
        if (t <= T - 2) iter(t, I0{});
    }
    if (!live && err) atomicExch(err, 1);
}

template <int NPX, int SY, int K>
void sweep_ws(const LV<float>& L, const float* u_old, const float* f, float* u_new, int first, cudaStream_t s,
              bool attr, int* err) {
    const size_t sm = sizeof(WsRing<NPX, SY>);
    if (attr) {
        cudaFuncSetAttribute(k_rb_sweep_ws<NPX, SY, K>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
        return;
    }
    static int per_sm = 0;                           // resident CTAs per SM (first launch asks)
    if (per_sm == 0) {
        int n = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_rb_sweep_ws<NPX, SY, K>, ws_threads<NPX, SY, K>(),
                                                          sm) != cudaSuccess || n < 1)
            n = 1;
        per_sm = n;
    }
    const int ty = (L.ny + SY - 1) / SY;
    int chunks = 152 * per_sm / ty;
    if (chunks < 1) chunks = 1;
    if (chunks > L.nz) chunks = L.nz;
    const int sz = (L.nz + chunks - 1) / chunks;
    dim3 grid(1, ty, (L.nz + sz - 1) / sz);
    k_rb_sweep_ws<NPX, SY, K><<<grid, ws_threads<NPX, SY, K>(), sm, s>>>(L, u_old, f, u_new, first, sz, err,
                                                                         g_wait_polls);
}

// row-tile kernels exist for these row lengths and heights
#define GP_ROW_NPX(X) X(32) X(48) X(64) X(96) X(128)
constexpr int kRowShapes = 3;   // SY = 4, 6, 8 (where NPX (SY + 2) <= 1024)

template <int NPX>
bool rows_dispatch_npx(int sy_id, const LV<float>& L, const float* u_old, const float* f, float* u_new, int first,
                       cudaStream_t s, bool attr, int* err) {
    if (sy_id == 0) {
        if constexpr (NPX * 6 <= 1024) { sweep_rows<NPX, 4>(L, u_old, f, u_new, first, s, attr, err); return true; }
    } else if (sy_id == 1) {
        if constexpr (NPX * 8 <= 1024) { sweep_rows<NPX, 6>(L, u_old, f, u_new, first, s, attr, err); return true; }
    } else if (sy_id == 2) {
        if constexpr (NPX * 10 <= 1024) { sweep_rows<NPX, 8>(L, u_old, f, u_new, first, s, attr, err); return true; }
    }
    return false;
}

// warp-specialised row shapes: (SY, K) = (6, 2), (4, 2), (6, 4), (4, 3) at two
// CTAs per SM; (16, 2), (14, 4), (14, 2), (12, 2) at one CTA per SM, whose
// taller tiles copy fewer halo rows per output row
constexpr int kWsShapes = 8;

template <int NPX, int SY, int K>
bool ws_try(const LV<float>& L, const float* u_old, const float* f, float* u_new, int first, cudaStream_t s,
            bool attr, int* err) {
    if constexpr ((NPX * ((SY + 2) / K)) % 32 == 0 && ws_threads<NPX, SY, K>() <= 1024 &&
                  sizeof(WsRing<NPX, SY>) <= 227 * 1024) {
        sweep_ws<NPX, SY, K>(L, u_old, f, u_new, first, s, attr, err);
        return true;
    }
    return false;
}

template <int NPX>
bool ws_dispatch_npx(int id, const LV<float>& L, const float* u_old, const float* f, float* u_new, int first,
                     cudaStream_t s, bool attr, int* err) {
    switch (id) {
    case 0: return ws_try<NPX, 6, 2>(L, u_old, f, u_new, first, s, attr, err);
    case 1: return ws_try<NPX, 4, 2>(L, u_old, f, u_new, first, s, attr, err);
    case 2: return ws_try<NPX, 6, 4>(L, u_old, f, u_new, first, s, attr, err);
    case 3: return ws_try<NPX, 4, 3>(L, u_old, f, u_new, first, s, attr, err);
    case 4: return ws_try<NPX, 16, 2>(L, u_old, f, u_new, first, s, attr, err);
    case 5: return ws_try<NPX, 14, 4>(L, u_old, f, u_new, first, s, attr, err);
    case 6: return ws_try<NPX, 14, 2>(L, u_old, f, u_new, first, s, attr, err);
    case 7: return ws_try<NPX, 12, 2>(L, u_old, f, u_new, first, s, attr, err);
    }
    return false;
}

static_assert(4 + kRowShapes + kWsShapes == kSweepShapeCount, "shape count");

// returns false when no row kernel fits this level (nx not covered, or too many threads)
bool rows_dispatch(int sy_id, int npx, const LV<float>& L, const float* u_old, const float* f, float* u_new,
                   int first, cudaStream_t s, bool attr, int* err = nullptr) {
    if (sy_id >= kRowShapes) {
        switch (npx) {
#define GP_NPX_WS(N) \
    case N: return ws_dispatch_npx<N>(sy_id - kRowShapes, L, u_old, f, u_new, first, s, attr, err);
            GP_ROW_NPX(GP_NPX_WS)
#undef GP_NPX_WS
        }
        return false;
    }
    if (!attr && !u_old) return false;              // only the warp-specialised shapes start from zero
    switch (npx) {
#define GP_NPX_CASE(N) \
    case N: return rows_dispatch_npx<N>(sy_id, L, u_old, f, u_new, first, s, attr, err);
        GP_ROW_NPX(GP_NPX_CASE)
#undef GP_NPX_CASE
    }
    return false;
}

// tile shapes the autotuner chooses from (x, y)
#define GP_SWEEP_SHAPES(X) X(0, 64, 8) X(1, 32, 16) X(2, 128, 4) X(3, 32, 8)
constexpr int kSweepShapes = 4;

template <typename T, int SX, int SY>
void sweep_shape(const LV<T>& L, const T* u_old, const T* f, T* u_new, int first, cudaStream_t s, bool attr) {
    const size_t sm = sizeof(Ring<T, SX, SY>);
    if (attr) {
        cudaFuncSetAttribute(k_rb_sweep<T, SX, SY>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
        return;
    }
    // z chunks: at most one wave of resident CTAs (a second, partial wave would
    // double the time), resident count from the shared memory per CTA
    int per_sm = (int)((227 * 1024) / (sm + 1024));
    if (per_sm < 1) per_sm = 1;
    if (per_sm > 8) per_sm = 8;
    const int txy = ((L.nx + SX - 1) / SX) * ((L.ny + SY - 1) / SY);
    int chunks = 152 * per_sm / txy;
    if (chunks > L.nz) chunks = L.nz;
    if (chunks < 1) chunks = 1;
    const int sz = (L.nz + chunks - 1) / chunks;
    dim3 grid((L.nx + SX - 1) / SX, (L.ny + SY - 1) / SY, (L.nz + sz - 1) / sz);
    k_rb_sweep<T, SX, SY><<<grid, NT, sm, s>>>(L, u_old, f, u_new, first, sz);
}

// false when nothing was launched: u_old null (start from zero) on a shape that
// cannot do that
template <typename T>
bool sweep_dispatch(int shape, const LV<T>& L, const T* u_old, const T* f, T* u_new, int first, cudaStream_t s,
                    bool attr, int* err = nullptr) {
    if constexpr (sizeof(T) == 4) {
        if (shape >= kSweepShapes) {
            if (rows_dispatch(shape - kSweepShapes, L.nx / 2, L, u_old, f, u_new, first, s, attr, err)) return true;
            shape = 0;
        }
    }
    if (!attr && !u_old) return false;
    switch (shape) {
#define GP_CASE(I, X, Y) \
    case I: sweep_shape<T, X, Y>(L, u_old, f, u_new, first, s, attr); break;
        GP_SWEEP_SHAPES(GP_CASE)
#undef GP_CASE
        default: sweep_shape<T, 64, 8>(L, u_old, f, u_new, first, s, attr); break;
    }
    return true;
}

}  // namespace

void rb_sweep_set_wait_polls(int polls) { g_wait_polls = polls < 0 ? (1 << 20) : polls; }

// allow the dynamic shared memory of every sweep shape (called before any capture)
void rb_sweep_init() {
    for (int k = 0; k < kSweepShapes; ++k) {
        LV<float> lf{};
        LV<double> ld{};
        sweep_dispatch<float>(k, lf, nullptr, nullptr, nullptr, 0, nullptr, true);
        sweep_dispatch<double>(k, ld, nullptr, nullptr, nullptr, 0, nullptr, true);
    }
    const int npx[] = {32, 48, 64, 96, 128};
    for (int n : npx)
        for (int k = 0; k < kRowShapes + kWsShapes; ++k) {
            LV<float> lf{};
            rows_dispatch(k, n, lf, nullptr, nullptr, nullptr, 0, nullptr, true);
        }
}

template <typename T>
bool launch_rb_sweep(const LV<T>& L, const T* u_old, const T* f, T* u_new, int first, cudaStream_t s, int shape,
                     int* err) {
    return sweep_dispatch<T>(shape, L, u_old, f, u_new, first, s, false, err);
}

// Time every tile shape on this level (three sweeps each, CUDA events on the
// given stream, inputs as they are) and return the fastest. Uses u_new as
// scratch output; run outside any stream capture.
template <typename T>
int rb_sweep_autotune(const LV<T>& L, const T* u_old, const T* f, T* u_new, cudaStream_t s) {
    cudaEvent_t a, b;
    if (cudaEventCreate(&a) != cudaSuccess) return 0;
    if (cudaEventCreate(&b) != cudaSuccess) { cudaEventDestroy(a); return 0; }
    int best = 0;
    float best_ms = 1e30f;
    const int nshapes = kSweepShapes + (sizeof(T) == 4 ? kRowShapes + kWsShapes : 0);
    for (int k = 0; k < nshapes; ++k) {
        if (k >= kSweepShapes) {
            LV<float> probe{};
            probe.nx = L.nx;
            if (!rows_dispatch(k - kSweepShapes, L.nx / 2, probe, nullptr, nullptr, nullptr, 0, s, true)) continue;
        }
        sweep_dispatch<T>(k, L, u_old, f, u_new, 0, s, false);     // warm-up
        cudaEventRecord(a, s);
        for (int r = 0; r < 3; ++r) sweep_dispatch<T>(k, L, u_old, f, u_new, 0, s, false);
        cudaEventRecord(b, s);
        cudaEventSynchronize(b);
        float ms = 0.f;
        cudaEventElapsedTime(&ms, a, b);
        if (ms < best_ms) { best_ms = ms; best = k; }
    }
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    return best;
}

template <typename T>
int rb_sweep_resolve(const LV<T>& L, int shape) {
    if (shape < kSweepShapes) return shape;
    if (sizeof(T) != 4) return 0;
    LV<float> probe{};
    probe.nx = L.nx;
    return rows_dispatch(shape - kSweepShapes, L.nx / 2, probe, nullptr, nullptr, nullptr, 0, nullptr, true) ? shape : 0;
}

template int rb_sweep_resolve<float>(const LV<float>&, int);
template int rb_sweep_resolve<double>(const LV<double>&, int);
template bool launch_rb_sweep<float>(const LV<float>&, const float*, const float*, float*, int, cudaStream_t, int,
                                     int*);
template bool launch_rb_sweep<double>(const LV<double>&, const double*, const double*, double*, int, cudaStream_t,
                                      int, int*);
template int rb_sweep_autotune<float>(const LV<float>&, const float*, const float*, float*, cudaStream_t);
template int rb_sweep_autotune<double>(const LV<double>&, const double*, const double*, double*, cudaStream_t);

}  // namespace gp
