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
    // z chunk: about one wave of resident CTAs
    int per_sm = (int)((220 * 1024) / sm);
    if (per_sm < 1) per_sm = 1;
    if (per_sm > 8) per_sm = 8;
    const int txy = ((L.nx + SX - 1) / SX) * ((L.ny + SY - 1) / SY);
    int chunks = (152 * per_sm + txy - 1) / txy;
    if (chunks > L.nz) chunks = L.nz;
    if (chunks < 1) chunks = 1;
    const int sz = (L.nz + chunks - 1) / chunks;
    dim3 grid((L.nx + SX - 1) / SX, (L.ny + SY - 1) / SY, (L.nz + sz - 1) / sz);
    k_rb_sweep<T, SX, SY><<<grid, NT, sm, s>>>(L, u_old, f, u_new, first, sz);
}

template <typename T>
void sweep_dispatch(int shape, const LV<T>& L, const T* u_old, const T* f, T* u_new, int first, cudaStream_t s,
                    bool attr) {
    switch (shape) {
#define GP_CASE(I, X, Y) \
    case I: sweep_shape<T, X, Y>(L, u_old, f, u_new, first, s, attr); break;
        GP_SWEEP_SHAPES(GP_CASE)
#undef GP_CASE
        default: sweep_shape<T, 64, 8>(L, u_old, f, u_new, first, s, attr); break;
    }
}

}  // namespace

// allow the dynamic shared memory of every sweep shape (called before any capture)
void rb_sweep_init() {
    for (int k = 0; k < kSweepShapes; ++k) {
        LV<float> lf{};
        LV<double> ld{};
        sweep_dispatch<float>(k, lf, nullptr, nullptr, nullptr, 0, nullptr, true);
        sweep_dispatch<double>(k, ld, nullptr, nullptr, nullptr, 0, nullptr, true);
    }
}

template <typename T>
void launch_rb_sweep(const LV<T>& L, const T* u_old, const T* f, T* u_new, int first, cudaStream_t s, int shape) {
    sweep_dispatch<T>(shape, L, u_old, f, u_new, first, s, false);
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
    for (int k = 0; k < kSweepShapes; ++k) {
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

template void launch_rb_sweep<float>(const LV<float>&, const float*, const float*, float*, int, cudaStream_t, int);
template void launch_rb_sweep<double>(const LV<double>&, const double*, const double*, double*, int, cudaStream_t, int);
template int rb_sweep_autotune<float>(const LV<float>&, const float*, const float*, float*, cudaStream_t);
template int rb_sweep_autotune<double>(const LV<double>&, const double*, const double*, double*, cudaStream_t);

}  // namespace gp
