// C ABI of the solver (declared in include/gp.h) and its host-side driver:
// workspace ownership, the multigrid hierarchy, the wet-band planner, the
// V-cycle, the preconditioned CG inner solve and the FP64 outer defect
// correction that couples the dry FFT solution to the wet multigrid band.
#include "gp_common.cuh"

#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <string>
#include <vector>

using namespace gp;

namespace {

// ---------------------------------------------------------------- helpers
struct Err {
    gp_status st;
    std::string msg;
};

#define GP_CUDA(call)                                                                      \
    do {                                                                                   \
        cudaError_t _e = (call);                                                           \
        if (_e != cudaSuccess) throw Err{GP_ERR_CUDA, std::string(#call) + ": " + cudaGetErrorString(_e)}; \
    } while (0)

#define GP_CHECK_LAUNCH() GP_CUDA(cudaGetLastError())

constexpr int kMaxInner = 16;   // PCG iterations one correction may take (adaptive counts included)

// A captured CUDA graph and what replaying it adds to the counters: the
// kernel launches, V-cycles and inner iterations it holds, and (when it was
// captured with profiling on) its event pairs per kernel group.
struct GraphSlot {
    cudaGraphExec_t exec = nullptr;
    long key = -1;
    long launches = 0;
    int vcycles = 0, inner = 0;
    std::vector<int> kinds, nlaunch;
    std::vector<cudaEvent_t> ev;
};

void clear_slot(GraphSlot& g) {
    if (g.exec) cudaGraphExecDestroy(g.exec);
    for (cudaEvent_t e : g.ev) cudaEventDestroy(e);
    g = GraphSlot();
}

template <typename T>
struct Hier {
    int L = 0;
    int nx = 0, ny = 0, nz = 0, zper = 1;      // level-0 interior dims
    LV<T> lv[16];
    T* u[16] = {};
    T* f[16] = {};
    T* res[16] = {};
    T* cx[16] = {};
    T* cy[16] = {};
    T* cz[16] = {};
    T* eps0 = nullptr;                          // owned level-0 cell eps (band only)
    T* x = nullptr; T* r = nullptr; T* p = nullptr; T* q = nullptr; T* z = nullptr;   // PCG, level 0
    T* tmp = nullptr;                           // level-0 ping-pong buffer of the fused sweep
    int sweep_shape = -1;                       // tile shape chosen by the autotuner (-1: not yet)
    T* minv = nullptr;
    int nc = 0;
    std::vector<void*> allocs;
    bool ready = false;
    GraphSlot pcg_g[kMaxInner + 1];             // pcg(iters) on this hierarchy, one graph per count
    GraphSlot solve_g;                          // fixed-count outer solve (graph_outer)
    const void* solve_phi = nullptr;            // the user buffers solve_g was captured with
    const void* solve_rho = nullptr;
    std::vector<GraphSlot> prec_g;              // split preconditioner into Krylov vector j (band only)
};

template <typename T>
T* alloc_level(Hier<T>& H, int nx, int ny, int nz) {
    const size_t pl = (size_t)nx * ny;
    void* ptr = nullptr;
    const size_t bytes = pl * (nz + 2) * sizeof(T);
    if (cudaMalloc(&ptr, bytes) != cudaSuccess) throw Err{GP_ERR_OOM, "cudaMalloc of a multigrid level failed"};
    H.allocs.push_back(ptr);
    GP_CUDA(cudaMemset(ptr, 0, bytes));
    return reinterpret_cast<T*>(ptr) + pl;
}

template <typename T>
void free_hier(Hier<T>& H) {
    for (GraphSlot& g : H.pcg_g) clear_slot(g);
    clear_slot(H.solve_g);
    for (GraphSlot& g : H.prec_g) clear_slot(g);
    for (void* p : H.allocs) cudaFree(p);
    H = Hier<T>();
}

template <typename T>
size_t level_bytes(const LV<T>& L) { return (size_t)L.nx * L.ny * (L.nz + 2) * sizeof(T); }

template <typename T>
T* lbase(const LV<T>& L, T* p) { return p - (size_t)L.nx * L.ny; }

// level plan: `requested` levels if the grid coarsens that far with <= kMaxCoarse
// coarsest points; otherwise the fewest levels reaching <= kAutoCoarse points,
// else the most levels reaching <= kMaxCoarse (the rule stated for gp_plan_levels)
int plan_levels(int nx, int ny, int nz, int zper, int requested, std::string& why) {
    auto dims_ok = [&](int l, long& pts) {
        const int m = 1 << l;
        if (nx % m || ny % m) return false;
        const int cx = nx / m, cy = ny / m;
        int cz;
        if (zper) {
            if (nz % m) return false;
            cz = nz / m;
            if (cz < 2) return false;
        } else {
            if ((nz + 1) % m) return false;
            cz = (nz + 1) / m - 1;
            if (cz < 1) return false;
        }
        if (cx < 2 || cy < 2) return false;
        pts = (long)cx * cy * cz;
        return true;
    };
    if (requested > 0) {
        long pts = 0;
        if (requested > 16 || !dims_ok(requested - 1, pts)) { why = "grid does not coarsen to the requested levels"; return -1; }
        if (pts > kMaxCoarse) { why = "coarsest grid of the requested levels exceeds 512 points"; return -1; }
        return requested;
    }
    int best = -1;
    for (int l = 1; l < 16; ++l) {
        long pts = 0;
        if (!dims_ok(l, pts)) break;
        if (pts <= kMaxCoarse) best = l + 1;
        if (pts <= kAutoCoarse) return l + 1;
    }
    if (best > 0) return best;
    why = "grid cannot be coarsened to <= 512 points";
    return -1;
}

}  // namespace

// ---------------------------------------------------------------- context
struct gp_ctx {
    Geo g{};
    long n = 0;
    cudaStream_t s = nullptr;
    gp_params prm{};
    bool have_eps = false;
    std::string err;
    gp_stats stats{};

    // device fields
    double* eps64 = nullptr;
    double* pe64 = nullptr;
    float* eps32 = nullptr;
    double* plane_max = nullptr;
    double* atoms = nullptr;       // positions of the last set_dielectric, wrapped into the cell
    float4* atoms32 = nullptr;
    int n_atoms = 0;
    int atoms_cap = 0;
    double* ratoms = nullptr;      // gp_build_rho's positions, wrapped
    float4* ratoms32 = nullptr;
    int ratoms_cap = 0;
    double* partial = nullptr;     // kReduceBlocks * (kMaxKrylov + 1)
    double* scal = nullptr;        // device scalars
    int* dstatus = nullptr;
    float2* rho_phid = nullptr;    // phi as float pairs for the charge-force kernel
    double* forces_S = nullptr;
    double* forces_T = nullptr;
    int forces_cap = 0;
    double* gmat = nullptr;        // Gauss-Jordan workspace (2 * 512^2)
    double* sw_coef = nullptr;     // switching-function tables (2 * kSwNI * (kSwDeg+1))
    float4* sw_pack = nullptr;     // their packed FP32 copies (2 * kSwNI * 4)
    double sw_key[4] = {0, 0, 0, 0};   // (eps0, r0, w, rcut) the tables were built for
    bool sw_built = false;
    double* rvdw = nullptr;        // van der Waals radii for the kind-1 dielectric
    std::vector<double> rvdw_host; // the same on the host (the image-sum radius depends on them)
    DielParams dp{};               // dielectric constants of the last gp_set_dielectric
    float2* phid = nullptr;        // df64 copies for the mixed-precision residual: phi, b = -4 pi rho, eps
    float2* bd = nullptr;
    float2* epsd = nullptr;
    bool epsd_ok = false;          // epsd matches eps64
    int rvdw_n = 0, rvdw_cap = 0;
    void* ctab = nullptr;          // coordinate tables of the tabulated dielectric and its force (CoordTabs)
    size_t ctab_cap = 0;           // bytes
    CoordTabs ct_s{}, ct_h{};      // views: s(d) coordinates (build), h(d) coordinates and displacements (force)
    void* gtab = nullptr;          // periodized Gaussian factor tables (GaussTabs)
    size_t gtab_cap = 0;           // bytes
    void* gmtab = nullptr;         // displacement and exponential tables of the df64 Eq. 9 kernels (GammaTabs)
    size_t gmtab_cap = 0;          // bytes
    GammaTabs gmt{};
    bool gm_df = false;            // the df64 Eq. 9 kernels serve this dielectric (else the FP64 ones)
    SwTables sw{};

    // solver state
    Hier<float> fullF, bandF;
    Hier<double> fullD, bandD;
    FFTPlan* fft = nullptr;
    void* fft_work = nullptr;
    size_t fft_work_bytes = 0;
    void* rfull = nullptr;         // full-box residual in the working precision (split)
    void* evac = nullptr;          // full-box vacuum correction (split)
    int full_levels = 0;
    int band_first = -1, band_nd = 0, band_nz = 0, band_first_interior = 0;
    bool split_ok = false;
    // FGMRES storage (split with accel): V[0..m] FP64, Z[0..m-1] and vT in the working precision
    std::vector<void*> kV;
    std::vector<void*> kZ;
    void* ekry = nullptr;          // inner FGMRES solution (working precision, full box)
    double* kY = nullptr;
    int k_m = 0;
    int k_bytes = 0;
    std::vector<void*> misc;
    // sixth-order operator (Sec. III): D1 eps per axis, work fields
    double* f6_d1e = nullptr;      // 3 n: D1 eps, valid for eps_version f6_d1e_version
    double* f6_r = nullptr;        // n: residual / operator output
    double* f6_w = nullptr;        // n: force weights
    double* f6_t3 = nullptr;       // 3 n: lam D1 phi per axis
    long eps_version = 0, f6_d1e_version = -1;

    // CUDA graphs: captured on a library stream that is ordered after / before the user's stream
    bool use_graphs = true;
    bool capturing = false;
    cudaStream_t gs = nullptr;
    cudaEvent_t ev_in = nullptr, ev_out = nullptr;

    // optional per-kernel-group timing (gp_profile)
    bool prof_on = false;
    struct Pending { int kind; int launches; cudaEvent_t a, b; };
    std::vector<Pending> pending;
    std::vector<cudaEvent_t> event_pool;
    long prm_on_key() const { return prof_on ? 1 : 0; }
    double prof_ms[GP_PROF_KINDS] = {};
    long prof_launches[GP_PROF_KINDS] = {};
    long prof_groups[GP_PROF_KINDS] = {};
};

namespace {

std::atomic<long> g_launches{0};

inline void count_launch(long n = 1) { g_launches.fetch_add(n, std::memory_order_relaxed); }

cudaEvent_t prof_event(gp_ctx* c) {
    if (!c->event_pool.empty()) {
        cudaEvent_t e = c->event_pool.back();
        c->event_pool.pop_back();
        return e;
    }
    cudaEvent_t e;
    GP_CUDA(cudaEventCreate(&e));
    return e;
}

// brackets a group of `launches` kernels of one kind with events on the stream
struct ProfScope {
    gp_ctx* c; int kind; int launches; cudaEvent_t a{}, b{}; cudaStream_t st;
    ProfScope(gp_ctx* c_, int k, int n, cudaStream_t on = nullptr) : c(c_), kind(k), launches(n), st(on ? on : c_->s) {
        count_launch(n);
        if (c->prof_on) {
            a = prof_event(c);
            GP_CUDA(cudaEventRecordWithFlags(a, st, c->capturing ? cudaEventRecordExternal : 0));
        }
    }
    ~ProfScope() {
        // never throws: a failed record only loses this sample
        if (c->prof_on && a) {
            cudaEvent_t e = nullptr;
            if (!c->event_pool.empty()) { e = c->event_pool.back(); c->event_pool.pop_back(); }
            else if (cudaEventCreate(&e) != cudaSuccess) return;
            if (cudaEventRecordWithFlags(e, st, c->capturing ? cudaEventRecordExternal : 0) != cudaSuccess) {
                c->event_pool.push_back(e);
                return;
            }
            c->pending.push_back({kind, launches, a, e});
        }
    }
};

// after the stream is synchronised: fold the event pairs into the totals
void prof_collect(gp_ctx* c) {
    for (auto& p : c->pending) {
        float ms = 0.f;
        GP_CUDA(cudaEventElapsedTime(&ms, p.a, p.b));
        c->prof_ms[p.kind] += ms;
        c->prof_launches[p.kind] += p.launches;
        c->prof_groups[p.kind] += 1;
        c->event_pool.push_back(p.a);
        c->event_pool.push_back(p.b);
    }
    c->pending.clear();
}

void* dalloc(gp_ctx* c, size_t bytes) {
    void* p = nullptr;
    if (cudaMalloc(&p, bytes) != cudaSuccess) throw Err{GP_ERR_OOM, "cudaMalloc failed"};
    c->misc.push_back(p);
    GP_CUDA(cudaMemset(p, 0, bytes));
    return p;
}

GaussTabs ensure_gtab(gp_ctx* c, int n_atoms) {
    const int nmax = std::max(c->g.nx, std::max(c->g.ny, c->g.nz));
    const size_t need = gauss_tabs_bytes(n_atoms, nmax);
    if (need > c->gtab_cap) {
        if (c->gtab) cudaFree(c->gtab);
        c->gtab = nullptr;
        if (cudaMalloc(&c->gtab, need) != cudaSuccess) throw Err{GP_ERR_OOM, "cudaMalloc failed"};
        c->gtab_cap = need;
    }
    return gauss_tabs_view(c->gtab, n_atoms, nmax);
}

// per-atom partial sums of the two force terms, sized for n atoms
void ensure_forces(gp_ctx* c, int n) {
    if (!c->rho_phid) c->rho_phid = (float2*)dalloc(c, sizeof(float2) * c->n);
    if (n <= c->forces_cap) return;
    if (c->forces_S) cudaFree(c->forces_S);
    if (c->forces_T) cudaFree(c->forces_T);
    c->forces_S = nullptr; c->forces_T = nullptr;
    c->forces_cap = 0;
    if (cudaMalloc(&c->forces_S, sizeof(double) * 3 * n) != cudaSuccess ||
        cudaMalloc(&c->forces_T, sizeof(double) * 3 * n) != cudaSuccess)
        throw Err{GP_ERR_OOM, "cudaMalloc failed"};
    c->forces_cap = n;
}

double sum_host(gp_ctx* c, int ncomp, double* out) {
    { ProfScope ps(c, GP_PROF_MISC, 1); launch_finalize(c->partial, kReduceBlocks, ncomp, c->scal + 8, c->s); }
    GP_CHECK_LAUNCH();
    GP_CUDA(cudaMemcpyAsync(out, c->scal + 8, sizeof(double) * ncomp, cudaMemcpyDeviceToHost, c->s));
    GP_CUDA(cudaStreamSynchronize(c->s));
    return out[0];
}

// ------------------------------------------------------------ hierarchy setup
template <typename T>
void alloc_hier(gp_ctx* c, Hier<T>& H, int nx, int ny, int nz, int zper, int levels, const T* eps_level0,
                bool own_eps) {
    const bool realloc = !H.ready || H.nx != nx || H.ny != ny || H.nz != nz || H.zper != zper || H.L != levels;
    if (realloc) {
        free_hier(H);
        H.nx = nx; H.ny = ny; H.nz = nz; H.zper = zper; H.L = levels;
        int lx = nx, ly = ny, lz = nz;
        double hx = c->g.hx, hy = c->g.hy, hz = c->g.hz;
        for (int l = 0; l < levels; ++l) {
            LV<T>& L = H.lv[l];
            L.nx = lx; L.ny = ly; L.nz = lz; L.zper = zper;
            L.ihx2 = (T)(1.0 / (hx * hx)); L.ihy2 = (T)(1.0 / (hy * hy)); L.ihz2 = (T)(1.0 / (hz * hz));
            L.cell = (l == 0);
            L.eps = nullptr; L.cx = L.cy = L.cz = nullptr;
            if (l > 0) {
                H.cx[l] = alloc_level(H, lx, ly, lz);
                H.cy[l] = alloc_level(H, lx, ly, lz);
                H.cz[l] = alloc_level(H, lx, ly, lz);
                L.cx = H.cx[l]; L.cy = H.cy[l]; L.cz = H.cz[l];
                H.u[l] = alloc_level(H, lx, ly, lz);
                H.f[l] = alloc_level(H, lx, ly, lz);
            }
            if (l < levels - 1) H.res[l] = alloc_level(H, lx, ly, lz);
            lx /= 2; ly /= 2;
            lz = zper ? lz / 2 : (lz + 1) / 2 - 1;
            hx *= 2; hy *= 2; hz *= 2;
        }
        H.x = alloc_level(H, nx, ny, nz);
        H.r = alloc_level(H, nx, ny, nz);
        H.p = alloc_level(H, nx, ny, nz);
        H.q = alloc_level(H, nx, ny, nz);
        H.z = alloc_level(H, nx, ny, nz);
        H.tmp = alloc_level(H, nx, ny, nz);
        if (own_eps) H.eps0 = alloc_level(H, nx, ny, nz);
        const LV<T>& C = H.lv[levels - 1];
        H.nc = C.nx * C.ny * C.nz;
        void* m = nullptr;
        if (cudaMalloc(&m, sizeof(T) * (size_t)H.nc * H.nc) != cudaSuccess) throw Err{GP_ERR_OOM, "cudaMalloc failed"};
        H.allocs.push_back(m);
        H.minv = reinterpret_cast<T*>(m);
        H.ready = true;
    }
    H.lv[0].eps = own_eps ? H.eps0 : eps_level0;
}

// coarse-level face coefficients and the dense coarsest inverse, from level 0's eps
template <typename T>
void coarse_coeffs(gp_ctx* c, Hier<T>& H) {
    const int levels = H.L;
    // coefficients of every coarse level from the level above
    for (int l = 1; l < levels; ++l) {
        const LV<T>& F = H.lv[l - 1];
        LV<T>& C = H.lv[l];
        ProfScope ps(c, GP_PROF_SETUP, 1);
        launch_coarsen_faces<T>(F, C.nx, C.ny, C.nz, H.cx[l], H.cy[l], H.cz[l], c->s);
        GP_CHECK_LAUNCH();
    }
    // dense inverse of the coarsest operator
    const LV<T>& C = H.lv[levels - 1];
    if (levels == 1) throw Err{GP_ERR_INVALID_ARG, "multigrid needs at least two levels"};
    {
        ProfScope ps(c, GP_PROF_SETUP, 1 + gauss_jordan_launches(H.nc));
        launch_coarse_matrix<T>(C, c->gmat, c->s);
        launch_gauss_jordan(c->gmat, H.nc, c->dstatus, c->s, sizeof(T) == 4);
    }
    GP_CHECK_LAUNCH();
    int st = 0;
    GP_CUDA(cudaMemcpyAsync(&st, c->dstatus, sizeof(int), cudaMemcpyDeviceToHost, c->s));
    GP_CUDA(cudaStreamSynchronize(c->s));
    if (st != 0) throw Err{GP_ERR_INVALID_ARG, "coarsest multigrid operator is singular"};
    {
        ProfScope ps(c, GP_PROF_SETUP, 1);
        launch_store_inverse<T>(c->gmat + (size_t)H.nc * H.nc, H.nc, H.minv, c->s);
    }
    GP_CHECK_LAUNCH();
    if (sizeof(T) == 4 && c->prm.sweep_shape >= 0) {
        H.sweep_shape = rb_sweep_resolve<T>(H.lv[0], c->prm.sweep_shape);
        c->stats.sweep_shape = H.sweep_shape;
    } else if (sizeof(T) == 4 && H.sweep_shape < 0) {
        // smoother autotuner: time each tile shape on this level once
        H.sweep_shape = rb_sweep_autotune<T>(H.lv[0], H.x, H.r, H.tmp, c->s);
        GP_CHECK_LAUNCH();
        c->stats.sweep_shape = H.sweep_shape;
    }
}

// ------------------------------------------------------------ V-cycle and PCG
// nu fused red-black sweeps of the finest level, colour `first` first; the
// result ends in u (ping-pong through H.tmp). from_zero: u starts at 0 (the
// pre-smoothing of a V-cycle): the first sweep then reads no u where the
// kernel allows it, and u is cleared first where it does not.
template <typename T>
void smooth_fine(gp_ctx* c, Hier<T>& H, T* u, const T* f, int nu, int first, bool from_zero = false) {
    const LV<T>& V = H.lv[0];
    if (nu <= 0) {
        if (from_zero) GP_CUDA(cudaMemsetAsync(lbase(V, u), 0, level_bytes(V), c->s));
        return;
    }
    if (sizeof(T) == 8) {
        // FP64 is bound by the FP64 pipe: the two-launch sweep issues no redundant work
        for (int it = 0; it < nu; ++it) {
            {
                ProfScope ps(c, from_zero && it == 0 ? GP_PROF_SMOOTH0_ZERO : GP_PROF_SMOOTH0, 1);
                launch_rbgs<T>(V, u, f, first, c->s, from_zero && it == 0);
            }
            ProfScope ps(c, GP_PROF_SMOOTH0, 1);
            launch_rbgs<T>(V, u, f, 1 - first, c->s);
        }
        return;
    }
    T* a = u;
    T* b = H.tmp;
    const int shape = H.sweep_shape < 0 ? 0 : H.sweep_shape;
    int it = 0;
    if (from_zero) {
        // timed in a group of its own: it moves 12 B/pt, the ordinary sweep 16
        ProfScope ps(c, GP_PROF_SMOOTH0_ZERO, 1);
        if (!launch_rb_sweep<T>(V, nullptr, f, b, first, c->s, shape, c->dstatus + 1)) {
            GP_CUDA(cudaMemsetAsync(lbase(V, a), 0, level_bytes(V), c->s));
            launch_rb_sweep<T>(V, a, f, b, first, c->s, shape, c->dstatus + 1);
        }
        T* t = a; a = b; b = t;
        it = 1;
    }
    if (it < nu) {
        ProfScope ps(c, GP_PROF_SMOOTH0, nu - it);
        for (; it < nu; ++it) {
            launch_rb_sweep<T>(V, a, f, b, first, c->s, shape, c->dstatus + 1);
            T* t = a; a = b; b = t;
        }
    }
    if (a != u) {
        ProfScope ps(c, GP_PROF_MG_FINE, 1);
        launch_copy_level<T>(V, u, a, c->s);
    }
}

template <typename T>
void vcycle(gp_ctx* c, Hier<T>& H, T* u0, const T* f0) {
    const int L = H.L;
    const int nuc1 = c->prm.nu_coarse > 0 ? c->prm.nu_coarse : c->prm.nu1;   // levels 2 and below
    const int nuc2 = c->prm.nu_coarse > 0 ? c->prm.nu_coarse : c->prm.nu2;
    // level 1 keeps the finest level's counts: its sweeps are the dearest of the
    // coarse ones, and more of them did not lower the V-cycle count
    auto pre_sweeps = [&](int l) { return l == 1 ? c->prm.nu1 : nuc1; };
    auto post_sweeps = [&](int l) { return l == 1 ? c->prm.nu2 : nuc2; };
    // first level small enough for the persistent single-CTA kernel (never the finest)
    int lc = L - 1;
    for (int l = 1; l < L; ++l) {
        if ((long)H.lv[l].nx * H.lv[l].ny * H.lv[l].nz <= kCoarseBlockPoints) { lc = l; break; }
    }
    for (int l = 0; l < lc; ++l) {
        const LV<T>& V = H.lv[l];
        T* u = l == 0 ? u0 : H.u[l];
        const T* f = l == 0 ? f0 : H.f[l];
        if (l == 0) {
            smooth_fine(c, H, u, f, c->prm.nu1, 0, true);
        } else if (pre_sweeps(l) == 0) {
            GP_CUDA(cudaMemsetAsync(lbase(V, u), 0, level_bytes(V), c->s));
        } else {
            // the first half sweep starts from u = 0 (the halo planes were zeroed at
            // allocation and no kernel writes them), so the level needs no clearing
            ProfScope ps(c, GP_PROF_MG_COARSE, 2 * pre_sweeps(l));
            for (int it = 0; it < pre_sweeps(l); ++it) {
                launch_rbgs<T>(V, u, f, 0, c->s, it == 0);
                launch_rbgs<T>(V, u, f, 1, c->s);
            }
        }
        ProfScope ps(c, l == 0 ? GP_PROF_MG_FINE : GP_PROF_MG_COARSE, 2);
        launch_residual<T>(V, u, f, H.res[l], c->s);
        launch_restrict<T>(V, H.res[l], H.lv[l + 1], H.f[l + 1], c->s);
    }
    {
        ProfScope ps(c, GP_PROF_MG_COARSE, 1);
        if (lc < L - 1) {
            CoarseSet<T> S;
            S.l0 = lc; S.L = L; S.nc = H.nc; S.nu1 = nuc1; S.nu2 = nuc2; S.minv = H.minv;
            for (int l = 0; l < L; ++l) { S.lv[l] = H.lv[l]; S.u[l] = H.u[l]; S.f[l] = H.f[l]; S.r[l] = H.res[l]; }
            launch_coarse_vcycle<T>(S, c->s);
        } else {
            launch_coarse_solve<T>(H.lv[L - 1], H.minv, H.nc, H.f[L - 1], H.u[L - 1], c->s);
        }
    }
    for (int l = lc - 1; l >= 0; --l) {
        const LV<T>& V = H.lv[l];
        T* u = l == 0 ? u0 : H.u[l];
        const T* f = l == 0 ? f0 : H.f[l];
        {
            ProfScope ps(c, l == 0 ? GP_PROF_MG_FINE : GP_PROF_MG_COARSE, 1);
            launch_prolong_add<T>(V, u, H.lv[l + 1], H.u[l + 1], c->s);
        }
        if (l == 0) {
            smooth_fine(c, H, u, f, c->prm.nu2, 1);
            continue;
        }
        ProfScope ps(c, GP_PROF_MG_COARSE, 2 * post_sweeps(l));
        for (int it = 0; it < post_sweeps(l); ++it) {
            launch_rbgs<T>(V, u, f, 1, c->s);
            launch_rbgs<T>(V, u, f, 0, c->s);
        }
    }
    GP_CHECK_LAUNCH();
    c->stats.vcycles++;
}

// Run `body` (stream work only: no host round trip inside) through a CUDA
// graph: captured once per key on the library stream, then replayed there,
// ordered after and before the user's stream by events.
template <typename F>
void run_graph(gp_ctx* c, GraphSlot& g, long key, F&& body) {
    if (!c->use_graphs) {
        body();
        return;
    }
    key = key * 2 + (c->prof_on ? 1 : 0);
    if (!g.exec || g.key != key) {
        clear_slot(g);
        cudaStream_t user = c->s;
        c->s = c->gs;
        const long l0 = g_launches.load();
        const int v0 = c->stats.vcycles, i0 = c->stats.inner_iterations;
        std::vector<gp_ctx::Pending> saved;
        saved.swap(c->pending);
        cudaGraph_t graph = nullptr;
        cudaError_t e1 = cudaStreamBeginCapture(c->gs, cudaStreamCaptureModeThreadLocal);
        if (e1 == cudaSuccess) {
            c->capturing = true;
            try {
                body();
            } catch (...) {
                c->capturing = false;
                cudaStreamEndCapture(c->gs, &graph);
                if (graph) cudaGraphDestroy(graph);
                c->s = user;
                c->pending.swap(saved);
                throw;
            }
            c->capturing = false;
            e1 = cudaStreamEndCapture(c->gs, &graph);
        }
        c->s = user;
        if (e1 != cudaSuccess) {
            c->pending.swap(saved);
            throw Err{GP_ERR_CUDA, std::string("graph capture: ") + cudaGetErrorString(e1)};
        }
        cudaError_t e2 = cudaGraphInstantiate(&g.exec, graph, 0);
        cudaGraphDestroy(graph);
        if (e2 != cudaSuccess) {
            c->pending.swap(saved);
            throw Err{GP_ERR_CUDA, std::string("graph instantiate: ") + cudaGetErrorString(e2)};
        }
        g.launches = g_launches.load() - l0;
        g.vcycles = c->stats.vcycles - v0;
        g.inner = c->stats.inner_iterations - i0;
        c->stats.vcycles = v0;
        c->stats.inner_iterations = i0;
        g_launches.fetch_sub(g.launches);
        for (auto& p : c->pending) {
            g.kinds.push_back(p.kind);
            g.nlaunch.push_back(p.launches);
            g.ev.push_back(p.a);
            g.ev.push_back(p.b);
        }
        c->pending.swap(saved);
        g.key = key;
    }
    GP_CUDA(cudaEventRecord(c->ev_in, c->s));
    GP_CUDA(cudaStreamWaitEvent(c->gs, c->ev_in, 0));
    GP_CUDA(cudaGraphLaunch(g.exec, c->gs));
    GP_CUDA(cudaEventRecord(c->ev_out, c->gs));
    GP_CUDA(cudaStreamWaitEvent(c->s, c->ev_out, 0));
    count_launch(g.launches);
    c->stats.vcycles += g.vcycles;
    c->stats.inner_iterations += g.inner;
    if (c->prof_on && !g.kinds.empty()) {
        // the graph's event pairs hold this replay's times until the next replay
        GP_CUDA(cudaStreamSynchronize(c->s));
        for (size_t k = 0; k < g.kinds.size(); ++k) {
            float ms = 0.f;
            GP_CUDA(cudaEventElapsedTime(&ms, g.ev[2 * k], g.ev[2 * k + 1]));
            c->prof_ms[g.kinds[k]] += ms;
            c->prof_launches[g.kinds[k]] += g.nlaunch[k];
            c->prof_groups[g.kinds[k]] += 1;
        }
    }
}

template <typename T>
void pcg_body(gp_ctx* c, Hier<T>& H, int iters);

// x ~ A^-1 r by `iters` multigrid-preconditioned CG steps from x = 0; r is
// overwritten. The whole sequence (V-cycles, dot products, updates: no host
// round trip) is one CUDA graph per hierarchy.
template <typename T>
void pcg(gp_ctx* c, Hier<T>& H, int iters) {
    const long key = ((long)c->prm.nu_coarse << 32) | ((long)iters << 16) | ((long)c->prm.nu1 << 8) | (long)c->prm.nu2;
    run_graph(c, H.pcg_g[iters <= kMaxInner ? iters : kMaxInner], key, [&] { pcg_body(c, H, iters); });
}

template <typename T>
void pcg_body(gp_ctx* c, Hier<T>& H, int iters) {
    const LV<T>& V = H.lv[0];
    GP_CUDA(cudaMemsetAsync(lbase(V, H.x), 0, level_bytes(V), c->s));
    vcycle(c, H, H.z, H.r);
    int cur = 0;
    {
        ProfScope ps(c, GP_PROF_KRYLOV, 3);
        launch_dot<T>(V, H.r, H.z, c->partial, c->s);
        launch_finalize(c->partial, kReduceBlocks, 1, c->scal + cur, c->s);
        launch_copy_level<T>(V, H.p, H.z, c->s);
    }
    for (int it = 0; it < iters; ++it) {
        {
            ProfScope ps(c, GP_PROF_KRYLOV, 3);
            launch_applyA_dot<T>(V, H.p, H.q, c->partial, c->s);
            launch_finalize(c->partial, kReduceBlocks, 1, c->scal + 1, c->s);
            launch_update_xr<T>(V, H.x, H.r, H.p, H.q, c->scal, cur, 1, c->s);
        }
        c->stats.inner_iterations++;
        if (it == iters - 1) break;
        vcycle(c, H, H.z, H.r);
        const int nxt = 2 - cur;
        {
            ProfScope ps(c, GP_PROF_KRYLOV, 3);
            launch_dot<T>(V, H.r, H.z, c->partial, c->s);
            launch_finalize(c->partial, kReduceBlocks, 1, c->scal + nxt, c->s);
            launch_update_p<T>(V, H.p, H.z, c->scal, nxt, cur, c->s);
        }
        cur = nxt;
    }
    GP_CHECK_LAUNCH();
}

// ------------------------------------------------------------ wet band planner
// Longest periodic run of dry planes; n_dirichlet planes centred in it, reduced
// to 1 + m 2^(levels-1) so the band (the other planes) coarsens levels-1 times.
bool plan_band(const std::vector<int>& dry, int levels, int n_dirichlet, int& first, int& nd) {
    const int nz = (int)dry.size();
    int ndry = 0;
    for (int v : dry) ndry += v;
    if (ndry == 0) return false;
    int run_start = 0, run_len = 0;
    if (ndry == nz) {
        run_start = 0; run_len = nz;
    } else {
        int k0 = 0;
        while (dry[k0]) ++k0;                       // a wet plane: runs cannot wrap past it
        int cur_start = -1, cur_len = 0;
        for (int t = 1; t <= nz; ++t) {
            const int k = (k0 + t) % nz;
            if (dry[k]) {
                if (cur_len == 0) cur_start = k;
                ++cur_len;
                if (cur_len > run_len) { run_len = cur_len; run_start = cur_start; }
            } else {
                cur_len = 0;
            }
        }
    }
    const int step = 1 << (levels - 1);
    const int want = n_dirichlet <= 0 ? run_len : std::min(n_dirichlet, run_len);
    nd = 1 + ((want - 1) / step) * step;
    if (nd >= nz) nd = 1;
    first = (run_start + (run_len - nd) / 2) % nz;
    return true;
}

// ------------------------------------------------------------ outer solve
template <typename T>
Hier<T>& full_hier(gp_ctx* c);
template <> Hier<float>& full_hier<float>(gp_ctx* c) { return c->fullF; }
template <> Hier<double>& full_hier<double>(gp_ctx* c) { return c->fullD; }
template <typename T>
Hier<T>& band_hier(gp_ctx* c);
template <> Hier<float>& band_hier<float>(gp_ctx* c) { return c->bandF; }
template <> Hier<double>& band_hier<double>(gp_ctx* c) { return c->bandD; }

template <typename T>
const T* eps_T(gp_ctx* c);
template <> const float* eps_T<float>(gp_ctx* c) { return c->eps32; }
template <> const double* eps_T<double>(gp_ctx* c) { return c->eps64; }

template <typename T>
void setup_solver(gp_ctx* c) {
    Hier<T>& F = full_hier<T>(c);
    alloc_hier<T>(c, F, c->g.nx, c->g.ny, c->g.nz, 1, c->full_levels, eps_T<T>(c), false);
    coarse_coeffs<T>(c, F);
    c->split_ok = false;
    c->stats.wet_fraction = 1.0;
    if (c->prm.split) {
        std::vector<double> pm(c->g.nz);
        GP_CUDA(cudaMemcpyAsync(pm.data(), c->plane_max, sizeof(double) * c->g.nz, cudaMemcpyDeviceToHost, c->s));
        GP_CUDA(cudaStreamSynchronize(c->s));
        std::vector<int> dry(c->g.nz);
        for (int k = 0; k < c->g.nz; ++k) dry[k] = pm[k] < c->prm.dry_thresh ? 1 : 0;
        int first = -1, nd = 0;
        if (plan_band(dry, c->full_levels, c->prm.n_dirichlet, first, nd)) {
            c->band_first = first;
            c->band_nd = nd;
            c->band_nz = c->g.nz - nd;
            c->band_first_interior = (first + nd) % c->g.nz;
            Hier<T>& B = band_hier<T>(c);
            alloc_hier<T>(c, B, c->g.nx, c->g.ny, c->band_nz, 0, c->full_levels, nullptr, true);
            // the band's level-0 eps, walls included, then its coarse levels
            {
                ProfScope ps(c, GP_PROF_SETUP, 1);
                launch_band_eps<T>(c->g, eps_T<T>(c), c->band_first_interior, c->band_nz, B.eps0, c->s);
            }
            GP_CHECK_LAUNCH();
            coarse_coeffs<T>(c, B);
            if (!c->rfull) c->rfull = dalloc(c, (size_t)c->n * sizeof(double));
            if (!c->evac) c->evac = dalloc(c, (size_t)c->n * sizeof(double));
            if (!c->ekry) c->ekry = dalloc(c, (size_t)c->n * sizeof(double));
            if (!c->fft) {
                c->fft = fft_create(c->g, c->s);
                if (!c->fft) throw Err{GP_ERR_INVALID_ARG, "grid extents must be 2^a 3^b for the FFT"};
            }
            const size_t wb = fft_workspace_bytes(c->g, true);
            if (!c->fft_work) { c->fft_work = dalloc(c, wb); c->fft_work_bytes = wb; }
            c->split_ok = true;
            c->stats.wet_fraction = (double)c->band_nz / c->g.nz;
        }
    }
    c->stats.split_active = c->split_ok ? 1 : 0;
    c->stats.band_first = c->split_ok ? c->band_first : -1;
    c->stats.band_dirichlet = c->split_ok ? c->band_nd : 0;
}

template <typename T>
void ensure_krylov(gp_ctx* c, int m) {
    if (c->k_m >= m && c->k_bytes == (int)sizeof(T)) return;
    for (void* v : c->kV) cudaFree(v);
    for (void* z : c->kZ) cudaFree(z);
    c->kV.clear(); c->kZ.clear(); c->k_m = 0;
    for (GraphSlot& g : band_hier<T>(c).prec_g) clear_slot(g);   // they bake the old pointers
    for (int j = 0; j <= m; ++j) {
        void* p = nullptr;
        if (cudaMalloc(&p, sizeof(T) * c->n) != cudaSuccess) throw Err{GP_ERR_OOM, "cudaMalloc failed"};
        c->kV.push_back(p);
    }
    for (int j = 0; j < m; ++j) {
        void* p = nullptr;
        if (cudaMalloc(&p, sizeof(T) * c->n) != cudaSuccess) throw Err{GP_ERR_OOM, "cudaMalloc failed"};
        c->kZ.push_back(p);
    }
    if (!c->kY && cudaMalloc(&c->kY, sizeof(double) * kMaxKrylov) != cudaSuccess)
        throw Err{GP_ERR_OOM, "cudaMalloc failed"};
    c->k_m = m;
    c->k_bytes = (int)sizeof(T);
}

// z = M v: the dry/wet split applied to a residual-like vector v (in T):
// z = L^-1 v on the whole box (FFT, Eq. 15), plus the band correction for
// A e = v - A L^-1 v on the wet band with e = 0 on the Dirichlet planes
// (band_vcycles V-cycles from zero: a fixed linear map, as FGMRES prefers).
template <typename T>
void split_precondition_body(gp_ctx* c, const T* v, T* z) {
    Hier<T>& B = band_hier<T>(c);
    T* ev = reinterpret_cast<T*>(c->evac);
    {
        ProfScope ps(c, GP_PROF_FFT, 5);
        fft_poisson<T>(c->fft, v, ev, c->fft_work, c->s);
    }
    {
        ProfScope ps(c, GP_PROF_MG_FINE, 1);
        launch_band_rhs<T>(c->g, eps_T<T>(c), v, ev, c->band_first_interior, c->band_nz, B.r, c->s);
    }
    vcycle(c, B, B.x, B.r);
    for (int it = 1; it < c->prm.band_vcycles; ++it) {
        {
            ProfScope ps(c, GP_PROF_MG_FINE, 1);
            launch_residual<T>(B.lv[0], B.x, B.r, B.q, c->s);
        }
        vcycle(c, B, B.z, B.q);
        ProfScope ps(c, GP_PROF_KRYLOV, 1);
        launch_axpy1<T>(B.lv[0], B.x, B.z, c->s);
    }
    ProfScope ps(c, GP_PROF_MG_FINE, 1);
    launch_combine<T>(c->g, ev, B.x, c->band_first_interior, c->band_nz, z, c->s);
    GP_CHECK_LAUNCH();
}

template <typename T>
void split_precondition(gp_ctx* c, int j, const T* v, T* z) {
    Hier<T>& B = band_hier<T>(c);
    if ((int)B.prec_g.size() <= j) B.prec_g.resize(j + 1);
    const long key = ((long)c->prm.nu_coarse << 32) | ((long)c->prm.band_vcycles << 16) | ((long)c->prm.nu1 << 8) |
                     (long)c->prm.nu2;
    run_graph(c, B.prec_g[j], key, [&] { split_precondition_body<T>(c, v, z); });
}

// Right-preconditioned flexible GMRES(m) in the working precision T on
// A x = rhs over the whole box (periodic operator of the finest level),
// preconditioned by the split. Stops when the Givens estimate of the
// residual drops below rel_tol |rhs|, after m steps, or on breakdown.
// x receives the solution (x = 0 start); rhs is not modified.
template <typename T>
int fgmres_inner(gp_ctx* c, const T* rhs, T* x, int m, double rel_tol) {
    Hier<T>& F = full_hier<T>(c);
    ensure_krylov<T>(c, m);
    const LV<T>& V0 = F.lv[0];
    std::vector<double> H((size_t)(m + 1) * m, 0.0), cs(m), sn(m), g(m + 1), y(m), hv(kMaxKrylov + 2);
    auto Hij = [&](int i, int j) -> double& { return H[(size_t)i * m + j]; };
    auto Vp = [&](int j) { return reinterpret_cast<T*>(c->kV[j]); };
    auto Zp = [&](int j) { return reinterpret_cast<T*>(c->kZ[j]); };
    {
        ProfScope ps(c, GP_PROF_KRYLOV, 3);
        launch_dot<T>(V0, rhs, rhs, c->partial, c->s);
        launch_finalize(c->partial, kReduceBlocks, 1, c->scal + 15, c->s);
        launch_scale_by_norm<T>(c->n, rhs, Vp(0), c->scal + 15, c->s);
    }
    GP_CHECK_LAUNCH();
    GP_CUDA(cudaMemcpyAsync(hv.data(), c->scal + 15, sizeof(double), cudaMemcpyDeviceToHost, c->s));
    GP_CUDA(cudaStreamSynchronize(c->s));
    const double beta = std::sqrt(hv[0]);
    if (!(beta > 0)) {
        GP_CUDA(cudaMemsetAsync(x, 0, sizeof(T) * c->n, c->s));
        return 0;
    }
    std::fill(g.begin(), g.end(), 0.0);
    g[0] = beta;
    int used = 0;
    for (int j = 0; j < m; ++j) {
        split_precondition<T>(c, j, Vp(j), Zp(j));
        TVecList<T> V;
        V.n = j + 1;
        for (int i = 0; i <= j; ++i) V.v[i] = Vp(i);
        {
            // classical Gram-Schmidt (one pass; the dot products are
            // compensated, and restarts bound the loss of orthogonality)
            ProfScope ps(c, GP_PROF_KRYLOV, 6);
            launch_applyA_dot<T>(V0, Zp(j), Vp(j + 1), c->partial, c->s);
            launch_multidot<T>(c->n, Vp(j + 1), V, c->partial, c->s);
            launch_finalize(c->partial, kReduceBlocks, j + 1, c->scal + 16, c->s);
            launch_multiaxpy_norm<T>(c->n, Vp(j + 1), V, c->scal + 16, c->partial, c->s);
            launch_finalize(c->partial, kReduceBlocks, 1, c->scal + 15, c->s);
            launch_scale_by_norm<T>(c->n, Vp(j + 1), Vp(j + 1), c->scal + 15, c->s);
        }
        GP_CHECK_LAUNCH();
        GP_CUDA(cudaMemcpyAsync(hv.data(), c->scal + 15, sizeof(double) * (j + 2), cudaMemcpyDeviceToHost, c->s));
        GP_CUDA(cudaStreamSynchronize(c->s));
        prof_collect(c);
        for (int i = 0; i <= j; ++i) Hij(i, j) = hv[1 + i];
        Hij(j + 1, j) = std::sqrt(hv[0]);
        for (int i = 0; i < j; ++i) {
            const double a = Hij(i, j), b = Hij(i + 1, j);
            Hij(i, j) = cs[i] * a + sn[i] * b;
            Hij(i + 1, j) = -sn[i] * a + cs[i] * b;
        }
        const double a = Hij(j, j), b = Hij(j + 1, j);
        const double r = std::hypot(a, b);
        cs[j] = r > 0 ? a / r : 1.0;
        sn[j] = r > 0 ? b / r : 0.0;
        Hij(j, j) = r;
        Hij(j + 1, j) = 0.0;
        g[j + 1] = -sn[j] * g[j];
        g[j] = cs[j] * g[j];
        used = j + 1;
        c->stats.inner_iterations++;
        if (std::fabs(g[j + 1]) <= rel_tol * beta || !(hv[0] > 0.0)) break;
    }
    for (int i = used - 1; i >= 0; --i) {
        double acc = g[i];
        for (int k = i + 1; k < used; ++k) acc -= Hij(i, k) * y[k];
        y[i] = acc / Hij(i, i);
    }
    GP_CUDA(cudaMemcpyAsync(c->kY, y.data(), sizeof(double) * used, cudaMemcpyHostToDevice, c->s));
    TVecList<T> Z;
    Z.n = used;
    for (int j = 0; j < used; ++j) Z.v[j] = Zp(j);
    {
        ProfScope ps(c, GP_PROF_KRYLOV, 1);
        launch_krylov_combine<T>(c->n, x, Z, c->kY, c->s);
    }
    GP_CHECK_LAUNCH();
    return used;
}

template <typename T>
gp_status solve_impl(gp_ctx* c, const double* rho, double* phi, double tol) {
    Hier<T>& F = full_hier<T>(c);
    Hier<T>& B = band_hier<T>(c);
    const bool split = c->split_ok;
    gp_stats& st = c->stats;
    st.outer_iterations = 0; st.inner_iterations = 0; st.vcycles = 0; st.history_len = 0;
    st.residual = NAN;
    double h3[4];
    {
        ProfScope ps(c, GP_PROF_MISC, 2);
        launch_rho_stats(c->n, rho, c->partial, c->s);
        launch_finalize(c->partial, kReduceBlocks, 3, c->scal + 8, c->s);
    }
    GP_CHECK_LAUNCH();
    T* rT = split ? reinterpret_cast<T*>(c->rfull) : F.r;
    T* ev = reinterpret_cast<T*>(c->evac);
    // mixed precision: the outer residual in df64 (FP32 pairs) when the tolerance
    // allows it (its floor is ~1e-11 of ||b||), in FP64 otherwise
    const bool use_df = sizeof(T) == 4 && tol >= 1e-10;
    // On the full box the df64 path keeps phi itself as pairs (phid) through the
    // loop, updated in FP32 arithmetic, and writes the FP64 phi once at the end.
    const bool master_df = use_df && !split;
    if (use_df) {
        if (!c->phid) {
            c->phid = (float2*)dalloc(c, sizeof(float2) * c->n);
            c->bd = (float2*)dalloc(c, sizeof(float2) * c->n);
            c->epsd = (float2*)dalloc(c, sizeof(float2) * c->n);
        }
        ProfScope ps(c, GP_PROF_RES64, c->epsd_ok ? 1 : 2);
        if (!c->epsd_ok) launch_to_df(c->n, c->eps64, 1.0, c->epsd, c->s);
        // b's leading floats also go to the full-box residual buffer: the first
        // residual when phi starts at zero
        launch_to_df(c->n, rho, -4.0 * kPi, c->bd, c->s, nullptr,
                     master_df ? reinterpret_cast<float*>(F.r) : nullptr);
        c->epsd_ok = true;
    }
    GP_CHECK_LAUNCH();
    if (master_df) {
        ProfScope ps(c, GP_PROF_UPDATE64, 1);
        GP_CUDA(cudaMemsetAsync(c->dstatus + 2, 0, sizeof(int), c->s));
        launch_to_df(c->n, phi, 1.0, c->phid, c->s, c->dstatus + 2);
    }
    GP_CHECK_LAUNCH();
    // the checks and, on the df64 full box, whether phi starts at zero (then its
    // first residual is b, already in rT, and is not evaluated)
    int phi_nonzero = 1;
    GP_CUDA(cudaMemcpyAsync(h3, c->scal + 8, sizeof(double) * 3, cudaMemcpyDeviceToHost, c->s));
    if (master_df) GP_CUDA(cudaMemcpyAsync(&phi_nonzero, c->dstatus + 2, sizeof(int), cudaMemcpyDeviceToHost, c->s));
    GP_CUDA(cudaStreamSynchronize(c->s));
    bool phi_zero = master_df && phi_nonzero == 0;
    if (!(std::fabs(h3[0]) <= 1e-10 * h3[1])) {
        if (!std::isfinite(h3[0])) throw Err{GP_ERR_INVALID_ARG, "rho is not finite"};
        throw Err{GP_ERR_NOT_NEUTRAL, "rho is not neutral: |sum rho| > 1e-10 sum |rho|"};
    }
    const double nb = 4.0 * kPi * std::sqrt(h3[2]);
    st.b_norm = nb;
    if (nb == 0.0) {
        GP_CUDA(cudaMemsetAsync(phi, 0, sizeof(double) * c->n, c->s));
        GP_CUDA(cudaStreamSynchronize(c->s));
        st.residual = 0.0;
        return GP_OK;
    }
    // the FP64 (or df64) outer residual of the current phi into `rdst`, with its partial sums
    auto outer_residual = [&](T* rdst) {
        if constexpr (sizeof(T) == 4) {
            if (use_df) {
                ProfScope ps(c, GP_PROF_RES64, master_df ? 1 : 2);
                if (!master_df) launch_to_df(c->n, phi, 1.0, c->phid, c->s);
                launch_residual_df(c->g, c->phid, c->bd, c->epsd, rdst, c->partial, c->s);
                return;
            }
        }
        ProfScope ps(c, GP_PROF_RES64, 1);
        launch_residual64<T>(c->g, phi, rho, c->eps64, rdst, c->partial, c->s);
    };
    // phi += the full-box correction x
    auto update_full = [&](const T* x) {
        ProfScope ps(c, GP_PROF_UPDATE64, 1);
        if constexpr (sizeof(T) == 4) {
            if (master_df) {
                launch_update_phid(c->n, c->phid, x, c->s);
                return;
            }
        }
        launch_update_phi<T>(c->g, phi, x, (const T*)nullptr, 0, 0, c->s);
    };
    // phi from its pairs where the loop kept it as pairs, and the gauge: the last
    // residual pass summed phi into scal[9]
    auto finish_phi = [&] {
        if (master_df) {
            ProfScope ps(c, GP_PROF_UPDATE64, 1);
            launch_from_df_gauge(c->n, c->phid, c->scal + 9, 1.0 / (double)c->n, phi, c->s);
        } else {
            ProfScope ps(c, GP_PROF_MISC, 1);
            launch_sub_mean(c->n, phi, c->scal + 9, 1.0 / (double)c->n, c->s);
        }
    };
    // a bounded smoother wait that gave up leaves the fields undefined: the flag is
    // read with every residual readback (no extra synchronisation), and the solve
    // stops at the first one that shows it, before any further V-cycle runs
    int expired = 0;
    auto queue_expired_read = [&] {
        GP_CUDA(cudaMemcpyAsync(&expired, c->dstatus + 1, sizeof(int), cudaMemcpyDeviceToHost, c->s));
    };
    auto timeout_exit = [&]() -> gp_status {
        GP_CUDA(cudaMemsetAsync(c->dstatus + 1, 0, sizeof(int), c->s));
        GP_CUDA(cudaStreamSynchronize(c->s));
        prof_collect(c);
        c->err = "a smoother copy wait expired; the result is not valid";
        return GP_ERR_TIMEOUT;
    };
    double best = INFINITY;
    gp_status result = GP_ERR_NOT_CONVERGED;
    const bool krylov = split && c->prm.accel;
    T* ekry = reinterpret_cast<T*>(c->ekry);
    if (!split && c->prm.graph_outer > 0) {
        // warm-started frames: a fixed number of outer corrections, captured as
        // one CUDA graph (no host round trip), then a single residual read
        const int k = c->prm.graph_outer;
        if (F.solve_phi != phi || F.solve_rho != rho) {
            clear_slot(F.solve_g);
            F.solve_phi = phi;
            F.solve_rho = rho;
        }
        const long key = ((long)c->prm.nu_coarse << 48) | ((long)use_df << 40) | ((long)k << 24) |
                         ((long)c->prm.inner << 16) | ((long)c->prm.nu1 << 8) | c->prm.nu2;
        run_graph(c, F.solve_g, key, [&] {
            for (int it = 0; it < k; ++it) {
                if (it > 0) update_full(F.x);
                outer_residual(F.r);
                pcg_body(c, F, c->prm.inner);
            }
            update_full(F.x);
            outer_residual(F.r);
            ProfScope ps(c, GP_PROF_MISC, 1);
            launch_finalize(c->partial, kReduceBlocks, 2, c->scal + 8, c->s);
            GP_CHECK_LAUNCH();
        });
        double s2[2];
        GP_CUDA(cudaMemcpyAsync(s2, c->scal + 8, sizeof(double) * 2, cudaMemcpyDeviceToHost, c->s));
        queue_expired_read();
        GP_CUDA(cudaStreamSynchronize(c->s));
        if (expired) return timeout_exit();   // the graph's residual is not recorded
        const double rn = std::sqrt(s2[0]) / nb;
        st.outer_iterations += k + 1;
        if (st.history_len < GP_HISTORY) st.history[st.history_len++] = rn;
        st.residual = rn;
        if (rn <= tol) {
            finish_phi();
            GP_CHECK_LAUNCH();
            GP_CUDA(cudaStreamSynchronize(c->s));
            prof_collect(c);
            return GP_OK;
        }
        // not there yet: continue with the checked loop from the current phi
        phi_zero = false;
    }
    // adaptive inner counts (full box): the contraction per CG iteration measured
    // over the previous correction predicts how many the next one needs to reach
    // half the tolerance, between 1 and twice `inner`
    int last_inner = 0;
    double last_rn = NAN;
    for (int it = 0; it < c->prm.max_outer; ++it) {
        if (it > 0) {
            if (!split) {
                update_full(F.x);
            } else {
                ProfScope ps(c, GP_PROF_UPDATE64, 1);
                if (krylov) launch_update_phi<T>(c->g, phi, ekry, (const T*)nullptr, 0, 0, c->s);
                else launch_update_phi<T>(c->g, phi, ev, B.x, c->band_first_interior, c->band_nz, c->s);
            }
            GP_CHECK_LAUNCH();
        }
        double rn = 1.0;                      // phi = 0: r = b, rT holds it
        if (!(it == 0 && phi_zero)) {
            outer_residual(rT);
            GP_CHECK_LAUNCH();
            queue_expired_read();
            double s2[2];
            sum_host(c, 2, s2);
            if (expired) return timeout_exit();   // the residual of undefined fields is not recorded
            rn = std::sqrt(s2[0]) / nb;
        }
        st.outer_iterations++;
        if (st.history_len < GP_HISTORY) st.history[st.history_len++] = rn;
        st.residual = rn;
        if (!std::isfinite(rn) || (it > 0 && rn > 1e3 * best)) { result = GP_ERR_DIVERGED; break; }
        best = std::min(best, rn);
        if (rn <= tol) { result = GP_OK; break; }
        if (it == c->prm.max_outer - 1) break;
        if (krylov) {
            // FP32 (or FP64) flexible GMRES on the correction equation A e = r,
            // preconditioned by the dry/wet split; the FP64 outer loop couples
            // the two regions through the full-box residual
            fgmres_inner<T>(c, rT, ekry, c->prm.restart, sizeof(T) == 4 ? 1e-4 : 1e-7);
        } else if (split) {
            {
                ProfScope ps(c, GP_PROF_FFT, 5);
                fft_poisson<T>(c->fft, rT, ev, c->fft_work, c->s);
            }
            GP_CHECK_LAUNCH();
            ProfScope ps(c, GP_PROF_MG_FINE, 1);
            launch_band_rhs<T>(c->g, eps_T<T>(c), rT, ev, c->band_first_interior, c->band_nz, B.r, c->s);
            GP_CHECK_LAUNCH();
            pcg<T>(c, B, c->prm.inner);
        } else {
            int k = c->prm.inner;
            if (c->prm.inner_adapt && last_inner > 0 && rn > 0.0 && last_rn > rn) {
                const double rate = std::min(std::max(std::pow(rn / last_rn, 1.0 / last_inner), 0.01), 0.9);
                // an FP32 correction cannot reduce the residual by much more than 1e-5 (its own
                // rounding), so no more iterations are spent on one than that reduction needs
                const double target = sizeof(T) == 4 ? std::max(0.5 * tol, 1e-5 * rn) : 0.5 * tol;
                const double need = std::log(target / rn) / std::log(rate);
                k = std::min(std::max((int)std::ceil(need - 1e-9), 1), 2 * c->prm.inner);
            }
            pcg<T>(c, F, k);
            last_inner = k;
            last_rn = rn;
        }
    }
    finish_phi();
    GP_CHECK_LAUNCH();
    queue_expired_read();
    GP_CUDA(cudaStreamSynchronize(c->s));
    if (expired) return timeout_exit();
    prof_collect(c);
    if (result == GP_ERR_NOT_CONVERGED) c->err = "not converged within max_outer";
    if (result == GP_ERR_DIVERGED) c->err = "residual diverged";
    return result;
}

// ------------------------------------------------------------ sixth-order solve (Sec. III, Eq. 16-18)
// The periodic sixth-order operator is not conservative, so its system carries
// a border (a reading of the paper, which is silent on the periodic case):
//   forward   A6 phi + mu eps = -4 pi (rho - mean rho),   sum(phi) = 0
//   adjoint   A6^T lam + nu 1 = rho - mean rho,           sum(eps lam) = 0
// Eliminating the border, the field solves P A6 phi = P b on zero-mean fields,
// P v = v - (sum v / sum eps) eps (Q v = v - mean(v) and sum(eps lam) = 0 for the
// adjoint), and the border value is the removed multiple. Flexible GMRES in
// FP64 on that projected system, right-preconditioned by the 7-point multigrid
// (`inner` MG-preconditioned CG steps in the context's working precision): both
// operators discretise div(eps grad), which is self-adjoint, so A7^-1 serves the
// forward and the transposed system alike. Device scalars used: 40..42 rho
// statistics, 44 sum of the last operator output, 45/46 sums of z and eps z,
// 47 n, 48..50 eps statistics (48 = sum eps).
constexpr int kS6Rho = 40, kS6Out = 44, kS6Z = 45, kS6N = 47, kS6Eps = 48;

void ensure_fd6(gp_ctx* c, bool transpose) {
    if (!c->f6_r) c->f6_r = (double*)dalloc(c, sizeof(double) * c->n);
    if (transpose) {
        if (!c->f6_d1e) c->f6_d1e = (double*)dalloc(c, sizeof(double) * 3 * c->n);
        if (c->f6_d1e_version != c->eps_version) {
            ProfScope ps(c, GP_PROF_SETUP, 1);
            launch_fd6_d1(c->g, c->eps64, nullptr, c->f6_d1e, c->s);
            c->f6_d1e_version = c->eps_version;
        }
    }
    GP_CHECK_LAUNCH();
}

// y = sb (rho - mean rho) + sa Op x, Op = A6 or A6^T, then projected (P or Q);
// scal[kS6Out] holds sum(y) before the projection
void fd6_operator(gp_ctx* c, const double* x, const double* rho, double sb, double sa, double* y, bool transpose) {
    ProfScope ps(c, GP_PROF_KRYLOV, 3);
    if (transpose)
        launch_fd6_apply_t(c->g, x, c->eps64, c->f6_d1e, rho, sb, c->scal + kS6Rho, sa, y, c->partial, c->s);
    else
        launch_fd6_apply(c->g, x, c->eps64, rho, sb, c->scal + kS6Rho, sa, y, c->partial, c->s);
    launch_finalize(c->partial, kReduceBlocks, 1, c->scal + kS6Out, c->s);
    if (transpose) launch_fd6_sub_ratio(c->n, y, nullptr, c->scal + kS6Out, c->scal + kS6N, c->s);
    else launch_fd6_sub_ratio(c->n, y, c->eps64, c->scal + kS6Out, c->scal + kS6Eps, c->s);
}

// z = M v with the constant of z fixed by the constraint (mean zero forward,
// sum(eps z) = 0 for the adjoint)
void fd6_fix_constant(gp_ctx* c, double* z, bool transpose) {
    launch_fd6_to64<double>(c->n, z, c->eps64, z, c->partial, c->s);
    launch_finalize(c->partial, kReduceBlocks, 2, c->scal + kS6Z, c->s);
    if (transpose) launch_fd6_sub_ratio(c->n, z, nullptr, c->scal + kS6Z + 1, c->scal + kS6Eps, c->s);
    else launch_fd6_sub_ratio(c->n, z, nullptr, c->scal + kS6Z, c->scal + kS6N, c->s);
}

template <typename T>
void fd6_precondition(gp_ctx* c, const double* v, double* z, bool transpose) {
    Hier<T>& F = full_hier<T>(c);
    {
        ProfScope ps(c, GP_PROF_MISC, 1);
        launch_cast_eps<T>(c->n, v, F.r, c->s);
    }
    pcg<T>(c, F, c->prm.inner);
    ProfScope ps(c, GP_PROF_MISC, 3);
    launch_fd6_to64<T>(c->n, F.x, c->eps64, z, c->partial, c->s);
    launch_finalize(c->partial, kReduceBlocks, 2, c->scal + kS6Z, c->s);
    if (transpose) launch_fd6_sub_ratio(c->n, z, nullptr, c->scal + kS6Z + 1, c->scal + kS6Eps, c->s);
    else launch_fd6_sub_ratio(c->n, z, nullptr, c->scal + kS6Z, c->scal + kS6N, c->s);
    GP_CHECK_LAUNCH();
}

template <typename T>
gp_status solve6_impl(gp_ctx* c, const double* rho, double* x, double tol, bool transpose, double* border) {
    gp_stats& st = c->stats;
    st.outer_iterations = 0; st.inner_iterations = 0; st.vcycles = 0; st.history_len = 0;
    st.residual = NAN;
    const long n = c->n;
    ensure_fd6(c, transpose);
    const int m = std::min(std::max(c->prm.restart, 1), kMaxKrylov - 1);
    ensure_krylov<double>(c, m);
    auto Vp = [&](int j) { return reinterpret_cast<double*>(c->kV[j]); };
    auto Zp = [&](int j) { return reinterpret_cast<double*>(c->kZ[j]); };
    double h3[3];
    {
        ProfScope ps(c, GP_PROF_MISC, 5);
        launch_rho_stats(n, rho, c->partial, c->s);
        launch_finalize(c->partial, kReduceBlocks, 3, c->scal + kS6Rho, c->s);
        launch_rho_stats(n, c->eps64, c->partial, c->s);
        launch_finalize(c->partial, kReduceBlocks, 3, c->scal + kS6Eps, c->s);
        launch_fd6_set(c->scal + kS6N, (double)n, c->s);
    }
    GP_CHECK_LAUNCH();
    GP_CUDA(cudaMemcpyAsync(h3, c->scal + kS6Rho, sizeof(double) * 3, cudaMemcpyDeviceToHost, c->s));
    GP_CUDA(cudaStreamSynchronize(c->s));
    if (!(std::fabs(h3[0]) <= 1e-10 * h3[1])) {
        if (!std::isfinite(h3[0])) throw Err{GP_ERR_INVALID_ARG, "rho is not finite"};
        throw Err{GP_ERR_NOT_NEUTRAL, "rho is not neutral: |sum rho| > 1e-10 sum |rho|"};
    }
    // ||b||: b = -4 pi (rho - mean) forward, rho - mean for the adjoint
    const double sb = transpose ? 1.0 : -4.0 * kPi;
    const double nb = std::fabs(sb) * std::sqrt(std::max(h3[2] - h3[0] * h3[0] / (double)n, 0.0));
    st.b_norm = nb;
    if (nb == 0.0) {
        GP_CUDA(cudaMemsetAsync(x, 0, sizeof(double) * n, c->s));
        GP_CUDA(cudaStreamSynchronize(c->s));
        if (border) *border = 0.0;
        st.residual = 0.0;
        return GP_OK;
    }
    {
        ProfScope ps(c, GP_PROF_MISC, 3);
        fd6_fix_constant(c, x, transpose);           // the warm start onto the constraint
    }
    std::vector<double> H((size_t)(m + 1) * m), cs(m), sn(m), g(m + 1), y(m + 1), hv(kMaxKrylov + 2);
    auto Hij = [&](int i, int j) -> double& { return H[(size_t)i * m + j]; };
    double best = INFINITY, sum_out = 0.0;
    gp_status result = GP_ERR_NOT_CONVERGED;
    for (int cyc = 0; cyc < c->prm.max_outer; ++cyc) {
        // true residual, projected, into V0
        fd6_operator(c, x, rho, sb, -1.0, Vp(0), transpose);
        TVecList<double> V0;
        V0.n = 1;
        V0.v[0] = Vp(0);
        {
            ProfScope ps(c, GP_PROF_KRYLOV, 2);
            launch_multidot<double>(n, Vp(0), V0, c->partial, c->s);
            launch_finalize(c->partial, kReduceBlocks, 1, c->scal + 15, c->s);
        }
        GP_CHECK_LAUNCH();
        double rs[2];
        GP_CUDA(cudaMemcpyAsync(&rs[0], c->scal + 15, sizeof(double), cudaMemcpyDeviceToHost, c->s));
        GP_CUDA(cudaMemcpyAsync(&rs[1], c->scal + kS6Out, sizeof(double), cudaMemcpyDeviceToHost, c->s));
        GP_CUDA(cudaStreamSynchronize(c->s));
        prof_collect(c);
        const double beta = std::sqrt(rs[0]);
        const double rn = beta / nb;
        sum_out = rs[1];
        st.outer_iterations++;
        if (st.history_len < GP_HISTORY) st.history[st.history_len++] = rn;
        st.residual = rn;
        if (!std::isfinite(rn) || (cyc > 0 && rn > 1e3 * best)) { result = GP_ERR_DIVERGED; break; }
        best = std::min(best, rn);
        if (rn <= tol) { result = GP_OK; break; }
        if (cyc == c->prm.max_outer - 1) break;
        {
            ProfScope ps(c, GP_PROF_KRYLOV, 1);
            launch_scale_by_norm<double>(n, Vp(0), Vp(0), c->scal + 15, c->s);
        }
        std::fill(H.begin(), H.end(), 0.0);
        std::fill(g.begin(), g.end(), 0.0);
        g[0] = beta;
        int used = 0;
        for (int j = 0; j < m; ++j) {
            fd6_precondition<T>(c, Vp(j), Zp(j), transpose);
            fd6_operator(c, Zp(j), nullptr, 0.0, 1.0, Vp(j + 1), transpose);
            TVecList<double> V;
            V.n = j + 1;
            for (int i = 0; i <= j; ++i) V.v[i] = Vp(i);
            {
                ProfScope ps(c, GP_PROF_KRYLOV, 5);
                launch_multidot<double>(n, Vp(j + 1), V, c->partial, c->s);
                launch_finalize(c->partial, kReduceBlocks, j + 1, c->scal + 16, c->s);
                launch_multiaxpy_norm<double>(n, Vp(j + 1), V, c->scal + 16, c->partial, c->s);
                launch_finalize(c->partial, kReduceBlocks, 1, c->scal + 15, c->s);
                launch_scale_by_norm<double>(n, Vp(j + 1), Vp(j + 1), c->scal + 15, c->s);
            }
            GP_CHECK_LAUNCH();
            GP_CUDA(cudaMemcpyAsync(hv.data(), c->scal + 15, sizeof(double) * (j + 2), cudaMemcpyDeviceToHost, c->s));
            GP_CUDA(cudaStreamSynchronize(c->s));
            prof_collect(c);
            for (int i = 0; i <= j; ++i) Hij(i, j) = hv[1 + i];
            Hij(j + 1, j) = std::sqrt(hv[0]);
            for (int i = 0; i < j; ++i) {
                const double a = Hij(i, j), b = Hij(i + 1, j);
                Hij(i, j) = cs[i] * a + sn[i] * b;
                Hij(i + 1, j) = -sn[i] * a + cs[i] * b;
            }
            const double a = Hij(j, j), b = Hij(j + 1, j);
            const double r = std::hypot(a, b);
            cs[j] = r > 0 ? a / r : 1.0;
            sn[j] = r > 0 ? b / r : 0.0;
            Hij(j, j) = r;
            Hij(j + 1, j) = 0.0;
            g[j + 1] = -sn[j] * g[j];
            g[j] = cs[j] * g[j];
            used = j + 1;
            st.inner_iterations++;
            if (std::fabs(g[j + 1]) <= 0.5 * tol * nb || !(hv[0] > 0.0)) break;
        }
        for (int i = used - 1; i >= 0; --i) {
            double acc = g[i];
            for (int k = i + 1; k < used; ++k) acc -= Hij(i, k) * y[k];
            y[i] = acc / Hij(i, i);
        }
        y[used] = 1.0;                               // x itself, last in the list: x += Z y
        GP_CUDA(cudaMemcpyAsync(c->kY, y.data(), sizeof(double) * (used + 1), cudaMemcpyHostToDevice, c->s));
        TVecList<double> Z;
        Z.n = used + 1;
        for (int j = 0; j < used; ++j) Z.v[j] = Zp(j);
        Z.v[used] = x;
        {
            ProfScope ps(c, GP_PROF_KRYLOV, 1);
            launch_krylov_combine<double>(n, x, Z, c->kY, c->s);
        }
        GP_CHECK_LAUNCH();
    }
    // the border value: the multiple of eps (or of 1) the projection removed
    // from the last residual, with the sign of the bordered equation
    double den = 0.0;
    GP_CUDA(cudaMemcpyAsync(&den, c->scal + kS6Eps, sizeof(double), cudaMemcpyDeviceToHost, c->s));
    GP_CUDA(cudaStreamSynchronize(c->s));
    if (border) *border = sum_out / (transpose ? (double)n : den);
    prof_collect(c);
    if (result == GP_ERR_NOT_CONVERGED) c->err = "not converged within max_outer";
    if (result == GP_ERR_DIVERGED) c->err = "residual diverged";
    return result;
}

gp_status fail(gp_ctx* c, const Err& e) {
    if (c) c->err = e.msg;
    return e.st;
}

// Upper bound on the part of gamma (Eq. 9) that an image sum cut at `radius` drops,
// at any point of the cell, for sum_a exp(rvdw_a) = se. At most (4 pi/3)(r + c)^3 / V
// images of an atom lie within r of a point (c half the cell diagonal: the
// cell-shaped boxes centred on the images do not overlap and lie in the ball of
// radius r + c); integrating exp(-r) against that count from `radius` on gives
// exp(-R)(u^3 + 3u^2 + 6u + 6) with u = R + c.
double gamma_tail_bound(double radius, const Geo& g, double se) {
    const double V = g.lx * g.ly * g.lz;
    const double u = radius + 0.5 * std::sqrt(g.lx * g.lx + g.ly * g.ly + g.lz * g.lz);
    return 4.0 * kPi / (3.0 * V) * std::exp(-radius) * (((u + 3.0) * u + 6.0) * u + 6.0) * se;
}

// the smallest radius (to 1e-6 A, bisection) whose bound is at most `tail`; the
// bound decreases with the radius (its derivative is -exp(-R) u^3)
double gamma_cutoff(const Geo& g, double se, double tail) {
    double lo = 0.0, hi = 1.0;
    while (gamma_tail_bound(hi, g, se) > tail) hi *= 2.0;
    while (hi - lo > 1e-6) {
        const double mid = 0.5 * (lo + hi);
        if (gamma_tail_bound(mid, g, se) > tail) lo = mid;
        else hi = mid;
    }
    return hi;
}

template <typename T>
gp_status fft_poisson_call(gp_ctx* c, const T* src_dev, T* phi_dev) {
    if (!c) return GP_ERR_INVALID_ARG;
    try {
        if (!src_dev || !phi_dev) throw Err{GP_ERR_INVALID_ARG, "bad arguments"};
        if (!c->fft) {
            c->fft = fft_create(c->g, c->s);
            if (!c->fft) throw Err{GP_ERR_INVALID_ARG, "grid extents must be 2^a 3^b for the FFT"};
        }
        if (!c->fft_work) {
            const size_t wb = fft_workspace_bytes(c->g, true);   // the FP64 size serves both precisions
            c->fft_work = dalloc(c, wb);
            c->fft_work_bytes = wb;
        }
        count_launch(5);
        fft_poisson<T>(c->fft, src_dev, phi_dev, c->fft_work, c->s);
        GP_CHECK_LAUNCH();
        GP_CUDA(cudaStreamSynchronize(c->s));
        return GP_OK;
    } catch (const Err& e) {
        return fail(c, e);
    }
}

bool good_extent(int n) {
    if (n < 8) return false;
    while (n % 2 == 0) n /= 2;
    if (n % 3 == 0) n /= 3;
    return n == 1;
}

}  // namespace

// ================================================================ C ABI
extern "C" {

void gp_default_params(gp_params* p) {
    if (!p) return;
    std::memset(p, 0, sizeof(*p));
    p->eps0 = 78.36;
    p->r0 = 2.5;
    p->w = 0.5;
    p->rcut = 6.0;
    p->dry_thresh = 1e-3;
    p->split = 0;
    p->n_dirichlet = 1;
    p->precision = 1;
    p->nu1 = 2;
    p->nu2 = 2;
    p->levels = 0;
    p->inner = 5;
    p->inner_adapt = 1;
    p->max_outer = 60;
    p->accel = 1;
    p->restart = 12;
    p->band_vcycles = 2;
    p->graph_outer = 0;
    p->sweep_shape = -1;
    p->nu_coarse = 4;
    p->kind = 0;
    p->gamma_tail = 1e-13;
    p->beta = 2.4;
    p->zlim = 0.0;
}

gp_status gp_create(gp_grid grid, gp_cell cell, void* cuda_stream, gp_ctx** out) {
    if (!out) return GP_ERR_INVALID_ARG;
    *out = nullptr;
    if (!good_extent(grid.nx) || !good_extent(grid.ny) || !good_extent(grid.nz) || grid.nx % 2)
        return GP_ERR_INVALID_ARG;
    if (!(cell.lx > 0 && cell.ly > 0 && cell.lz > 0)) return GP_ERR_INVALID_ARG;
    gp_ctx* c = new gp_ctx();
    try {
        c->g = make_geo(grid.nx, grid.ny, grid.nz, cell.lx, cell.ly, cell.lz);
        c->n = (long)grid.nx * grid.ny * grid.nz;
        c->s = reinterpret_cast<cudaStream_t>(cuda_stream);
        gp_default_params(&c->prm);
        c->eps64 = (double*)dalloc(c, sizeof(double) * c->n);
        c->pe64 = (double*)dalloc(c, sizeof(double) * c->n);
        c->eps32 = (float*)dalloc(c, sizeof(float) * c->n);
        c->plane_max = (double*)dalloc(c, sizeof(double) * grid.nz);
        c->partial = (double*)dalloc(c, sizeof(double) * kReduceBlocks * (kMaxKrylov + 1));
        c->scal = (double*)dalloc(c, sizeof(double) * 64);
        c->dstatus = (int*)dalloc(c, sizeof(int) * 4);   // [0] coarse inverse, [1] smoother wait expired
        GP_CUDA(cudaMemsetAsync(c->dstatus, 0, sizeof(int) * 4, c->s));
        c->gmat = (double*)dalloc(c, sizeof(double) * 2 * kMaxCoarse * kMaxCoarse);
        c->sw_coef = (double*)dalloc(c, sizeof(double) * 2 * kSwNI * (kSwDeg + 1));
        c->sw_pack = (float4*)dalloc(c, sizeof(float4) * 2 * kSwNI * 4);
        rb_sweep_init();
        coarse_vcycle_init();
        {
            const char* wp = std::getenv("GP_TEST_SWEEP_WAIT_POLLS");
            rb_sweep_set_wait_polls(wp ? std::atoi(wp) : -1);
        }
        GP_CUDA(cudaStreamCreateWithFlags(&c->gs, cudaStreamNonBlocking));
        GP_CUDA(cudaEventCreateWithFlags(&c->ev_in, cudaEventDisableTiming));
        GP_CUDA(cudaEventCreateWithFlags(&c->ev_out, cudaEventDisableTiming));
        const char* ev = std::getenv("GP_NO_GRAPHS");
        c->use_graphs = !(ev && ev[0] == '1');
    } catch (const Err& e) {
        gp_destroy(c);
        return e.st;
    }
    *out = c;
    return GP_OK;
}

gp_status gp_set_dielectric(gp_ctx* c, const double* atoms_dev, int n_atoms, const gp_params* params) {
    if (!c) return GP_ERR_INVALID_ARG;
    try {
        if (!params || n_atoms < 0 || (n_atoms > 0 && !atoms_dev)) throw Err{GP_ERR_INVALID_ARG, "bad arguments"};
        gp_params p = *params;
        if (p.kind == 0 && !(p.rcut > 0 && p.rcut <= c->g.lx && p.rcut <= c->g.ly && p.rcut <= c->g.lz))
            throw Err{GP_ERR_INVALID_ARG, "rcut must be positive and not exceed the cell"};
        if (!(p.w > 0) || !(p.eps0 >= 1.0)) throw Err{GP_ERR_INVALID_ARG, "need w > 0 and eps0 >= 1"};
        if (p.precision != 0 && p.precision != 1) throw Err{GP_ERR_INVALID_ARG, "precision must be 0 or 1"};
        if (p.nu1 < 0 || p.nu2 < 0 || p.nu1 + p.nu2 == 0 || p.inner < 1 || p.max_outer < 1)
            throw Err{GP_ERR_INVALID_ARG, "need nu1+nu2 >= 1, inner >= 1, max_outer >= 1"};
        if (p.inner > kMaxInner / 2 || p.inner_adapt < 0 || p.inner_adapt > 1)
            throw Err{GP_ERR_INVALID_ARG, "need inner <= 8 and inner_adapt 0 or 1"};
        if (p.accel && (p.restart < 1 || p.restart > kMaxKrylov - 1))
            throw Err{GP_ERR_INVALID_ARG, "restart must be in 1..15"};
        if (p.band_vcycles < 1) throw Err{GP_ERR_INVALID_ARG, "band_vcycles must be >= 1"};
        if (p.graph_outer < 0 || p.graph_outer > 16) throw Err{GP_ERR_INVALID_ARG, "graph_outer must be 0..16"};
        if (p.nu_coarse < 0 || p.nu_coarse > 8) throw Err{GP_ERR_INVALID_ARG, "nu_coarse must be 0 .. 8"};
        if (p.sweep_shape < -1 || p.sweep_shape >= kSweepShapeCount)
            throw Err{GP_ERR_INVALID_ARG, "sweep_shape must be -1 (autotune) or a valid tile shape"};
        if (p.kind < 0 || p.kind > 2)
            throw Err{GP_ERR_INVALID_ARG, "kind must be 0 (erf product), 1 (Eq. 9-10) or 2 (Eq. 19)"};
        if (p.kind != 0 && !(p.beta > 0.0)) throw Err{GP_ERR_INVALID_ARG, "beta must be positive"};
        if (p.kind != 0 && !(p.gamma_tail > 0.0 && p.gamma_tail <= 1e-3))
            throw Err{GP_ERR_INVALID_ARG, "gamma_tail must be in (0, 1e-3]"};
        if (p.kind != 0 && n_atoms > 0 && c->rvdw_n != n_atoms)
            throw Err{GP_ERR_STATE, "kinds 1 and 2 need gp_set_vdw_radii for the same number of atoms"};
        std::string why;
        const int L = plan_levels(c->g.nx, c->g.ny, c->g.nz, 1, p.levels, why);
        if (L < 2) throw Err{GP_ERR_INVALID_ARG, why.empty() ? "grid too small for multigrid" : why};
        // from here on the context changes: a failure below leaves no dielectric
        // (GP_ERR_STATE for the calls that need one) rather than a half-built one
        c->have_eps = false;
        c->prm = p;
        c->full_levels = L;
        if (n_atoms > c->atoms_cap) {
            void* a = nullptr;
            void* b = nullptr;
            if (cudaMalloc(&a, sizeof(double) * 3 * n_atoms) != cudaSuccess) throw Err{GP_ERR_OOM, "cudaMalloc failed"};
            if (cudaMalloc(&b, sizeof(float4) * n_atoms) != cudaSuccess) {
                cudaFree(a);
                throw Err{GP_ERR_OOM, "cudaMalloc failed"};
            }
            if (c->atoms) cudaFree(c->atoms);
            if (c->atoms32) cudaFree(c->atoms32);
            c->atoms = (double*)a;
            c->atoms32 = (float4*)b;
            c->atoms_cap = n_atoms;
        }
        c->n_atoms = n_atoms;
        {
            ProfScope ps(c, GP_PROF_MISC, n_atoms > 0 ? 1 : 0);
            launch_wrap_atoms(c->g, atoms_dev, n_atoms, c->atoms, c->atoms32, c->s);
        }
        GP_CHECK_LAUNCH();
        Atoms at{c->atoms, c->atoms32, nullptr, n_atoms};
        DielParams dp = make_diel(p.eps0, p.r0, p.w, p.rcut, p.kind, p.beta, p.zlim);
        c->stats.gamma_cutoff = 0.0;
        if (p.kind != 0) {
            // Eq. 9 sums over every image: take those within the radius where the
            // bound on the rest falls below gamma_tail, and the image range that reaches it
            double se = 0.0;
            for (int a = 0; a < n_atoms; ++a) se += std::exp(c->rvdw_host[a]);
            dp.rcut = n_atoms > 0 ? gamma_cutoff(c->g, se, p.gamma_tail) : 1.0;
            dp.rcutf = (float)dp.rcut;
            dp.rc2f = (float)(dp.rcut * dp.rcut);
            dp.mx = (int)std::ceil(dp.rcut / c->g.lx);
            dp.my = (int)std::ceil(dp.rcut / c->g.ly);
            dp.mz = (int)std::ceil(dp.rcut / c->g.lz);
            c->stats.gamma_cutoff = dp.rcut;
            if (n_atoms > 0) {
                const double r32 = gamma_cutoff(c->g, se, 1e-7);
                dp.far2f = (float)(r32 * r32);
            }
        }
        // the df64 Eq. 9 kernels stage exp(-n) rows up to the radius (and exp(+n) rows up
        // to the saturation distance of Eq. 19): radii beyond their rows take the FP64 kernels
        c->gm_df = false;
        if (p.kind != 0 && n_atoms > 0) {
            const int m = std::max(dp.mx, std::max(dp.my, dp.mz));
            const int kt1 = (int)std::floor(dp.rcut + 0.01) + 2;
            double rvmax = 0.0;
            for (int a = 0; a < n_atoms; ++a) rvmax = std::max(rvmax, c->rvdw_host[a]);
            const int kg = p.kind == 2 ? (int)std::floor(rvmax + dp.esat + 0.01) + 2 : 1;
            const long nimg = (long)(2 * dp.mx + 1) * (2 * dp.my + 1) * (2 * dp.mz + 1);
            if (kt1 <= kGT1 && kg <= kGT1 && nimg * n_atoms < (1L << 30)) {
                const int nmax = std::max(c->g.nx, std::max(c->g.ny, c->g.nz));
                const size_t need = gamma_tabs_bytes(n_atoms, m, nmax);
                if (need > c->gmtab_cap) {
                    if (c->gmtab) cudaFree(c->gmtab);
                    c->gmtab = nullptr;
                    c->gmtab_cap = 0;
                    if (cudaMalloc(&c->gmtab, need) != cudaSuccess) throw Err{GP_ERR_OOM, "cudaMalloc failed"};
                    c->gmtab_cap = need;
                }
                c->gmt = gamma_tabs_view(c->gmtab, n_atoms, m, nmax);
                c->gmt.kt1 = kt1;
                c->gmt.kg = kg;
                ProfScope ps(c, GP_PROF_EPS, 1);
                launch_gamma_tables(c->g, at, dp, c->rvdw, c->gmt, c->s);
                c->gm_df = true;
            }
        }
        c->dp = dp;
        // switching-function tables for these r0, w (when the tabulated range is away from d = 0)
        SwTables tb{};
        if (p.kind == 0 && p.r0 - 4.0 * p.w > 0.0 && p.r0 + 6.0 * p.w <= p.rcut) {
            tb.s = c->sw_coef;
            tb.h = c->sw_coef + (size_t)kSwNI * (kSwDeg + 1);
            tb.s32 = c->sw_pack;
            tb.h32 = c->sw_pack + (size_t)kSwNI * 4;
            tb.s_qlo = (p.r0 - 4.0 * p.w) * (p.r0 - 4.0 * p.w);
            tb.s_qhi = (p.r0 + 6.0 * p.w) * (p.r0 + 6.0 * p.w);
            tb.s_inv_dq = kSwNI / (tb.s_qhi - tb.s_qlo);
            tb.s_dq = (tb.s_qhi - tb.s_qlo) / kSwNI;
            tb.h_qlo = (p.r0 - 3.5 * p.w) * (p.r0 - 3.5 * p.w);
            tb.h_qhi = (p.r0 + 3.5 * p.w) * (p.r0 + 3.5 * p.w);
            tb.h_inv_dq = kSwNI / (tb.h_qhi - tb.h_qlo);
            tb.h_dq = (tb.h_qhi - tb.h_qlo) / kSwNI;
            tb.s_qlof = (float)tb.s_qlo; tb.s_dqf = (float)tb.s_dq;
            tb.h_qlof = (float)tb.h_qlo; tb.h_dqf = (float)tb.h_dq;
            // they depend on the parameters alone: built again only when those change
            const double key[4] = {p.eps0, p.r0, p.w, p.rcut};
            if (!c->sw_built || std::memcmp(key, c->sw_key, sizeof(key)) != 0) {
                ProfScope ps(c, GP_PROF_EPS, 1);
                launch_switch_tables(dp, tb, c->sw_coef, c->sw_coef + (size_t)kSwNI * (kSwDeg + 1), c->sw_pack,
                                     c->sw_pack + (size_t)kSwNI * 4, c->s);
                GP_CHECK_LAUNCH();
                std::memcpy(c->sw_key, key, sizeof(key));
                c->sw_built = true;
            }
            // the per-atom table coordinates of both tables (one FP64 pass, then loads)
            const int nmax = std::max(c->g.nx, std::max(c->g.ny, c->g.nz));
            const size_t bs = coord_tabs_bytes(n_atoms, nmax, false), bh = coord_tabs_bytes(n_atoms, nmax, true);
            if (bs + bh > c->ctab_cap) {
                if (c->ctab) cudaFree(c->ctab);
                c->ctab = nullptr;
                c->ctab_cap = 0;
                if (cudaMalloc(&c->ctab, bs + bh) != cudaSuccess) throw Err{GP_ERR_OOM, "cudaMalloc failed"};
                c->ctab_cap = bs + bh;
            }
            c->ct_s = coord_tabs_view(c->ctab, n_atoms, nmax, false);
            c->ct_h = coord_tabs_view(static_cast<char*>(c->ctab) + bs, n_atoms, nmax, true);
            ProfScope ps(c, GP_PROF_EPS, 2);
            launch_coord_tables(c->g, at, tb.s_qlo, tb.s_inv_dq, c->ct_s, c->s);
            launch_coord_tables(c->g, at, tb.h_qlo, tb.h_inv_dq, c->ct_h, c->s);
        }
        c->sw = tb;
        bool have_pmax = false;
        {
            ProfScope ps(c, GP_PROF_EPS, 1);
            // pe64 holds the per-point factor of d eps/d R: eps - 1 (kind 0) or d eps/d gamma (kinds 1, 2)
            if (p.kind != 0 && c->gm_df)
                launch_build_eps_gamma_df(c->g, at, dp, c->gmt, c->eps64, c->pe64, c->eps32, c->s);
            else if (p.kind != 0)
                launch_build_eps_gamma(c->g, at, dp, c->rvdw, c->eps64, c->pe64, c->eps32, c->s);
            else have_pmax = launch_build_eps(c->g, at, dp, tb, c->ct_s, c->eps64, c->pe64, c->eps32, c->plane_max, c->s);
        }
        c->epsd_ok = false;
        GP_CHECK_LAUNCH();
        if (!have_pmax) {
            ProfScope ps(c, GP_PROF_MISC, 1);
            launch_plane_max(c->g, c->eps64, c->plane_max, c->s);
        }
        GP_CHECK_LAUNCH();
        if (p.precision == 1) setup_solver<float>(c);
        else setup_solver<double>(c);
        std::vector<double> pm(c->g.nz);
        GP_CUDA(cudaMemcpyAsync(pm.data(), c->plane_max, sizeof(double) * c->g.nz, cudaMemcpyDeviceToHost, c->s));
        GP_CUDA(cudaStreamSynchronize(c->s));
        int nd = 0;
        for (double v : pm) nd += v < p.dry_thresh;
        c->stats.dry_planes = nd;
        c->stats.levels = L;
        c->have_eps = true;
        c->eps_version++;
        prof_collect(c);
        c->err.clear();
        return GP_OK;
    } catch (const Err& e) {
        return fail(c, e);
    }
}

gp_status gp_set_vdw_radii(gp_ctx* c, const double* radii_dev, int n_atoms) {
    if (!c) return GP_ERR_INVALID_ARG;
    try {
        if (!radii_dev || n_atoms < 1) throw Err{GP_ERR_INVALID_ARG, "radii: null pointer or no atoms"};
        std::vector<double> hr((size_t)n_atoms);
        GP_CUDA(cudaMemcpyAsync(hr.data(), radii_dev, sizeof(double) * n_atoms, cudaMemcpyDeviceToHost, c->s));
        GP_CUDA(cudaStreamSynchronize(c->s));
        for (double v : hr)
            if (!(v > 0.0)) throw Err{GP_ERR_INVALID_ARG, "van der Waals radii must be positive"};
        if (n_atoms > c->rvdw_cap) {
            if (c->rvdw) cudaFree(c->rvdw);
    if (c->ctab) cudaFree(c->ctab);
            c->rvdw = nullptr;
            if (cudaMalloc(&c->rvdw, sizeof(double) * n_atoms) != cudaSuccess) throw Err{GP_ERR_OOM, "cudaMalloc failed"};
            c->rvdw_cap = n_atoms;
        }
        GP_CUDA(cudaMemcpyAsync(c->rvdw, radii_dev, sizeof(double) * n_atoms, cudaMemcpyDeviceToDevice, c->s));
        GP_CUDA(cudaStreamSynchronize(c->s));
        c->rvdw_host = hr;
        c->rvdw_n = n_atoms;
        return GP_OK;
    } catch (const Err& e) {
        return fail(c, e);
    }
}

gp_status gp_build_rho(gp_ctx* c, const double* atoms_dev, const double* gauss_dev, int n_atoms, double* rho_dev) {
    if (!c) return GP_ERR_INVALID_ARG;
    try {
        if (!rho_dev || n_atoms < 0 || (n_atoms > 0 && (!atoms_dev || !gauss_dev)))
            throw Err{GP_ERR_INVALID_ARG, "bad arguments"};
        const double cut = 8.0;
        if (n_atoms > 0) {
            std::vector<double> gh(3 * (size_t)n_atoms);
            GP_CUDA(cudaMemcpyAsync(gh.data(), gauss_dev, sizeof(double) * 3 * n_atoms, cudaMemcpyDeviceToHost, c->s));
            GP_CUDA(cudaStreamSynchronize(c->s));
            const double lmin = std::min(c->g.lx, std::min(c->g.ly, c->g.lz));
            for (int a = 0; a < n_atoms; ++a)
                for (int w = 1; w <= 2; ++w)
                    if (!(gh[3 * a + w] > 0) || cut * gh[3 * a + w] > lmin)
                        throw Err{GP_ERR_INVALID_ARG, "Gaussian width must be positive with 8 sigma <= the cell"};
        }
        if (n_atoms > c->ratoms_cap) {
            void* a = nullptr;
            void* b = nullptr;
            if (cudaMalloc(&a, sizeof(double) * 3 * n_atoms) != cudaSuccess ||
                cudaMalloc(&b, sizeof(float4) * n_atoms) != cudaSuccess)
                throw Err{GP_ERR_OOM, "cudaMalloc failed"};
            if (c->ratoms) cudaFree(c->ratoms);
            if (c->ratoms32) cudaFree(c->ratoms32);
            c->ratoms = (double*)a;
            c->ratoms32 = (float4*)b;
            c->ratoms_cap = n_atoms;
        }
        {
            ProfScope ps(c, GP_PROF_MISC, n_atoms > 0 ? 1 : 0);
            launch_wrap_atoms(c->g, atoms_dev, n_atoms, c->ratoms, c->ratoms32, c->s);
        }
        Atoms at{c->ratoms, c->ratoms32, gauss_dev, n_atoms};
        const GaussTabs gt = ensure_gtab(c, n_atoms);
        {
            ProfScope ps(c, GP_PROF_RHO, n_atoms > 0 ? 2 : 1);
            launch_gauss_tables(c->g, at, cut, gt, c->s);
            launch_build_rho_raw(c->g, gt, rho_dev, c->s);
        }
        GP_CHECK_LAUNCH();
        {
            ProfScope ps(c, GP_PROF_MISC, 3);
            launch_rho_stats(c->n, rho_dev, c->partial, c->s);
            launch_finalize(c->partial, kReduceBlocks, 3, c->scal + 12, c->s);
            launch_sub_mean(c->n, rho_dev, c->scal + 12, 1.0 / (double)c->n, c->s);
        }
        GP_CHECK_LAUNCH();
        GP_CUDA(cudaStreamSynchronize(c->s));
        prof_collect(c);
        return GP_OK;
    } catch (const Err& e) {
        return fail(c, e);
    }
}

gp_status gp_solve(gp_ctx* c, const double* rho_dev, double* phi_dev, double tol) {
    if (!c) return GP_ERR_INVALID_ARG;
    try {
        if (!rho_dev || !phi_dev || !(tol > 0)) throw Err{GP_ERR_INVALID_ARG, "bad arguments"};
        if (!c->have_eps) throw Err{GP_ERR_STATE, "gp_set_dielectric must precede gp_solve"};
        return c->prm.precision == 1 ? solve_impl<float>(c, rho_dev, phi_dev, tol)
                                     : solve_impl<double>(c, rho_dev, phi_dev, tol);
    } catch (const Err& e) {
        return fail(c, e);
    }
}

gp_status gp_energy_forces(gp_ctx* c, const double* phi_dev, const double* rho_dev, const double* gauss_dev,
                           double* energy_host, double* forces_dev) {
    if (!c) return GP_ERR_INVALID_ARG;
    try {
        if (!phi_dev || !rho_dev) throw Err{GP_ERR_INVALID_ARG, "bad arguments"};
        if (!c->have_eps) throw Err{GP_ERR_STATE, "gp_set_dielectric must precede gp_energy_forces"};
        const double dv = c->g.hx * c->g.hy * c->g.hz;
        if (energy_host) {
            {
                ProfScope ps(c, GP_PROF_ENERGY, 1);
                launch_energy(c->g, rho_dev, phi_dev, c->eps64, c->partial, c->s);
            }
            GP_CHECK_LAUNCH();
            double e2[2];
            sum_host(c, 2, e2);
            energy_host[0] = 0.5 * dv * e2[0];
            energy_host[1] = dv / (8.0 * kPi) * e2[1];
        }
        if (forces_dev && c->n_atoms > 0) {
            const int n = c->n_atoms;
            ensure_forces(c, n);
            GP_CUDA(cudaMemsetAsync(c->forces_S, 0, sizeof(double) * 3 * n, c->s));
            GP_CUDA(cudaMemsetAsync(c->forces_T, 0, sizeof(double) * 3 * n, c->s));
            Atoms at{c->atoms, c->atoms32, gauss_dev, n};
            const DielParams dp = c->dp;
            {
                // phi as float pairs, once, for both force kernels
                ProfScope ps(c, GP_PROF_FORCES_EPS, 2);
                launch_to_df(c->n, phi_dev, 1.0, c->rho_phid, c->s);
                if (c->prm.kind != 0 && c->gm_df)
                    launch_forces_eps_gamma_df(c->g, at, dp, c->gmt, c->rho_phid, nullptr, c->pe64, c->forces_S,
                                               c->s);
                else if (c->prm.kind != 0)
                    launch_forces_eps_gamma(c->g, at, dp, c->rvdw, phi_dev, nullptr, c->pe64, c->forces_S, c->s);
                else
                    launch_forces_eps(c->g, at, dp, c->sw, c->ct_h, phi_dev, c->rho_phid, nullptr, c->pe64,
                                      c->forces_S, c->s);
            }
            GP_CHECK_LAUNCH();
            if (gauss_dev) {
                const GaussTabs gt = ensure_gtab(c, n);
                ProfScope ps(c, GP_PROF_FORCES_RHO, 2);
                launch_gauss_tables(c->g, at, 8.0, gt, c->s);
                launch_forces_rho(c->g, gt, nullptr, c->rho_phid, c->forces_T, c->s);
            }
            GP_CHECK_LAUNCH();
            ProfScope ps(c, GP_PROF_MISC, 1);
            launch_forces_finish(c->forces_S, gauss_dev ? c->forces_T : nullptr, n, -dv / (8.0 * kPi), dv,
                                 forces_dev, c->s);
            GP_CHECK_LAUNCH();
        }
        GP_CUDA(cudaStreamSynchronize(c->s));
        prof_collect(c);
        return GP_OK;
    } catch (const Err& e) {
        return fail(c, e);
    }
}

gp_status gp_residual(gp_ctx* c, const double* rho_dev, const double* phi_dev, double* r_dev, double* rel_host) {
    if (!c) return GP_ERR_INVALID_ARG;
    try {
        if (!rho_dev || !phi_dev || !r_dev) throw Err{GP_ERR_INVALID_ARG, "bad arguments"};
        if (!c->have_eps) throw Err{GP_ERR_STATE, "gp_set_dielectric must precede gp_residual"};
        count_launch(1);
        launch_residual64<double>(c->g, phi_dev, rho_dev, c->eps64, r_dev, c->partial, c->s);
        GP_CHECK_LAUNCH();
        double s2[2];
        sum_host(c, 2, s2);
        if (rel_host) {
            count_launch(1);
            launch_rho_stats(c->n, rho_dev, c->partial, c->s);
            GP_CHECK_LAUNCH();
            double h3[3];
            sum_host(c, 3, h3);
            const double nb = 4.0 * kPi * std::sqrt(h3[2]);
            *rel_host = nb > 0 ? std::sqrt(s2[0]) / nb : std::sqrt(s2[0]);
        }
        return GP_OK;
    } catch (const Err& e) {
        return fail(c, e);
    }
}

gp_status gp_residual6(gp_ctx* c, const double* rho_dev, const double* phi_dev, double mu, double* r_dev,
                       double* rel_host) {
    if (!c) return GP_ERR_INVALID_ARG;
    try {
        if (!rho_dev || !phi_dev || !r_dev || !std::isfinite(mu)) throw Err{GP_ERR_INVALID_ARG, "bad arguments"};
        if (!c->have_eps) throw Err{GP_ERR_STATE, "gp_set_dielectric must precede gp_residual6"};
        count_launch(1);
        launch_residual6(c->g, phi_dev, rho_dev, c->eps64, mu, r_dev, c->partial, c->s);
        GP_CHECK_LAUNCH();
        double s2[1];
        sum_host(c, 1, s2);
        if (rel_host) {
            count_launch(1);
            launch_rho_stats(c->n, rho_dev, c->partial, c->s);
            GP_CHECK_LAUNCH();
            double h3[3];
            sum_host(c, 3, h3);
            const double nb = 4.0 * kPi * std::sqrt(h3[2]);
            *rel_host = nb > 0 ? std::sqrt(s2[0]) / nb : std::sqrt(s2[0]);
        }
        return GP_OK;
    } catch (const Err& e) {
        return fail(c, e);
    }
}

gp_status gp_solve6(gp_ctx* c, const double* rho_dev, double* phi_dev, double* mu_host, double tol) {
    if (!c) return GP_ERR_INVALID_ARG;
    try {
        if (!rho_dev || !phi_dev || !(tol > 0.0)) throw Err{GP_ERR_INVALID_ARG, "bad arguments"};
        if (!c->have_eps) throw Err{GP_ERR_STATE, "gp_set_dielectric must precede gp_solve6"};
        double mu = 0.0;
        const gp_status st = c->prm.precision == 1 ? solve6_impl<float>(c, rho_dev, phi_dev, tol, false, &mu)
                                                   : solve6_impl<double>(c, rho_dev, phi_dev, tol, false, &mu);
        if (mu_host) *mu_host = mu;
        if (st == GP_OK) c->err.clear();
        return st;
    } catch (const Err& e) {
        return fail(c, e);
    }
}

gp_status gp_adjoint6(gp_ctx* c, const double* rho_dev, double* lam_dev, double* nu_host, double tol) {
    if (!c) return GP_ERR_INVALID_ARG;
    try {
        if (!rho_dev || !lam_dev || !(tol > 0.0)) throw Err{GP_ERR_INVALID_ARG, "bad arguments"};
        if (!c->have_eps) throw Err{GP_ERR_STATE, "gp_set_dielectric must precede gp_adjoint6"};
        double nu = 0.0;
        const gp_status st = c->prm.precision == 1 ? solve6_impl<float>(c, rho_dev, lam_dev, tol, true, &nu)
                                                   : solve6_impl<double>(c, rho_dev, lam_dev, tol, true, &nu);
        if (nu_host) *nu_host = nu;
        if (st == GP_OK) c->err.clear();
        return st;
    } catch (const Err& e) {
        return fail(c, e);
    }
}

gp_status gp_energy_forces6(gp_ctx* c, const double* phi_dev, double mu, const double* lam_dev,
                            const double* rho_dev, const double* gauss_dev, double* energy_host,
                            double* forces_dev) {
    if (!c) return GP_ERR_INVALID_ARG;
    try {
        if (!phi_dev || !rho_dev || !std::isfinite(mu) || (forces_dev && !lam_dev))
            throw Err{GP_ERR_INVALID_ARG, "bad arguments"};
        if (!c->have_eps) throw Err{GP_ERR_STATE, "gp_set_dielectric must precede gp_energy_forces6"};
        const double dv = c->g.hx * c->g.hy * c->g.hz;
        if (energy_host) {
            {
                ProfScope ps(c, GP_PROF_ENERGY, 1);
                launch_energy(c->g, rho_dev, phi_dev, c->eps64, c->partial, c->s);
            }
            GP_CHECK_LAUNCH();
            double e2[2];
            sum_host(c, 2, e2);
            energy_host[0] = 0.5 * dv * e2[0];
        }
        if (forces_dev && c->n_atoms > 0) {
            const int n = c->n_atoms;
            ensure_forces(c, n);
            if (!c->f6_w) c->f6_w = (double*)dalloc(c, sizeof(double) * c->n);
            if (!c->f6_t3) c->f6_t3 = (double*)dalloc(c, sizeof(double) * 3 * c->n);
            GP_CUDA(cudaMemsetAsync(c->forces_S, 0, sizeof(double) * 3 * n, c->s));
            GP_CUDA(cudaMemsetAsync(c->forces_T, 0, sizeof(double) * 3 * n, c->s));
            // per-point weight of d eps: sum_axes [-D1(lam D1 phi) + lam D2 phi] + mu lam
            {
                ProfScope ps(c, GP_PROF_FORCES_EPS, 2);
                launch_fd6_d1(c->g, phi_dev, lam_dev, c->f6_t3, c->s);
                launch_fd6_weps(c->g, phi_dev, lam_dev, c->f6_t3, mu, c->f6_w, c->s);
            }
            GP_CHECK_LAUNCH();
            Atoms at{c->atoms, c->atoms32, gauss_dev, n};
            const DielParams dp = c->dp;
            {
                ProfScope ps(c, GP_PROF_FORCES_EPS, 1);
                if (c->prm.kind != 0 && c->gm_df)
                    launch_forces_eps_gamma_df(c->g, at, dp, c->gmt, nullptr, c->f6_w, c->pe64, c->forces_S, c->s);
                else if (c->prm.kind != 0)
                    launch_forces_eps_gamma(c->g, at, dp, c->rvdw, phi_dev, c->f6_w, c->pe64, c->forces_S, c->s);
                else
                    launch_forces_eps(c->g, at, dp, c->sw, c->ct_h, phi_dev, nullptr, c->f6_w, c->pe64,
                                      c->forces_S, c->s);
            }
            GP_CHECK_LAUNCH();
            if (gauss_dev) {
                // weight of d rho: (phi - 4 pi lam)/2, its mean removed (rho loses its mean)
                if (!c->f6_r) c->f6_r = (double*)dalloc(c, sizeof(double) * c->n);
                {
                    ProfScope ps(c, GP_PROF_MISC, 4);
                    launch_fd6_wrho(c->n, phi_dev, lam_dev, c->f6_r, c->partial, c->s);
                    launch_finalize(c->partial, kReduceBlocks, 1, c->scal + kS6Z, c->s);
                    launch_fd6_set(c->scal + kS6N, (double)c->n, c->s);
                    launch_fd6_sub_ratio(c->n, c->f6_r, nullptr, c->scal + kS6Z, c->scal + kS6N, c->s);
                }
                const GaussTabs gt = ensure_gtab(c, n);
                ProfScope ps(c, GP_PROF_FORCES_RHO, 3);
                launch_gauss_tables(c->g, at, 8.0, gt, c->s);
                launch_forces_rho(c->g, gt, c->f6_r, c->rho_phid, c->forces_T, c->s);
            }
            GP_CHECK_LAUNCH();
            ProfScope ps(c, GP_PROF_MISC, 1);
            launch_forces_finish(c->forces_S, gauss_dev ? c->forces_T : nullptr, n, -0.5 * dv, dv, forces_dev, c->s);
            GP_CHECK_LAUNCH();
        }
        GP_CUDA(cudaStreamSynchronize(c->s));
        prof_collect(c);
        return GP_OK;
    } catch (const Err& e) {
        return fail(c, e);
    }
}

gp_status gp_fft_poisson(gp_ctx* c, const double* src_dev, double* phi_dev) {
    return fft_poisson_call<double>(c, src_dev, phi_dev);
}

gp_status gp_fft_poisson_f32(gp_ctx* c, const float* src_dev, float* phi_dev) {
    return fft_poisson_call<float>(c, src_dev, phi_dev);
}

gp_status gp_get_eps(gp_ctx* c, double* eps_dev) {
    if (!c || !eps_dev) return GP_ERR_INVALID_ARG;
    if (!c->have_eps) { c->err = "no dielectric"; return GP_ERR_STATE; }
    try {
        GP_CUDA(cudaMemcpyAsync(eps_dev, c->eps64, sizeof(double) * c->n, cudaMemcpyDeviceToDevice, c->s));
        GP_CUDA(cudaStreamSynchronize(c->s));
        return GP_OK;
    } catch (const Err& e) {
        return fail(c, e);
    }
}

gp_status gp_get_plane_max(gp_ctx* c, double* out) {
    if (!c || !out) return GP_ERR_INVALID_ARG;
    if (!c->have_eps) { c->err = "no dielectric"; return GP_ERR_STATE; }
    try {
        GP_CUDA(cudaMemcpyAsync(out, c->plane_max, sizeof(double) * c->g.nz, cudaMemcpyDeviceToHost, c->s));
        GP_CUDA(cudaStreamSynchronize(c->s));
        return GP_OK;
    } catch (const Err& e) {
        return fail(c, e);
    }
}

gp_status gp_get_stats(const gp_ctx* c, gp_stats* out) {
    if (!c || !out) return GP_ERR_INVALID_ARG;
    *out = c->stats;
    return GP_OK;
}

const char* gp_last_error(const gp_ctx* c) { return c ? c->err.c_str() : "null context"; }

gp_status gp_profile(gp_ctx* c, int enable) {
    if (!c) return GP_ERR_INVALID_ARG;
    try {
        GP_CUDA(cudaStreamSynchronize(c->s));
        prof_collect(c);
        c->prof_on = enable != 0;
        if (c->prof_on)
            for (int k = 0; k < GP_PROF_KINDS; ++k) { c->prof_ms[k] = 0; c->prof_launches[k] = 0; c->prof_groups[k] = 0; }
        return GP_OK;
    } catch (const Err& e) {
        return fail(c, e);
    }
}

gp_status gp_get_profile(const gp_ctx* c, double* ms, long* launches, long* groups, int n) {
    if (!c || n < 0 || n > GP_PROF_KINDS) return GP_ERR_INVALID_ARG;
    for (int k = 0; k < n; ++k) {
        if (ms) ms[k] = c->prof_ms[k];
        if (launches) launches[k] = c->prof_launches[k];
        if (groups) groups[k] = c->prof_groups[k];
    }
    return GP_OK;
}

long gp_launch_count(void) { return g_launches.load(); }

int gp_plan_band(const int* dry, int nz, int levels, int n_dirichlet, int* first, int* nd) {
    if (!dry || nz < 1 || levels < 1 || levels > 16 || !first || !nd) return -1;
    std::vector<int> d(dry, dry + nz);
    for (int& v : d) v = v ? 1 : 0;
    int f = -1, n = 0;
    const bool ok = plan_band(d, levels, n_dirichlet, f, n);
    *first = ok ? f : -1;
    *nd = ok ? n : 0;
    return ok ? 1 : 0;
}

int gp_plan_levels(int nx, int ny, int nz, int zper, int requested) {
    if (nx < 1 || ny < 1 || nz < 1) return -1;
    std::string why;
    return plan_levels(nx, ny, nz, zper ? 1 : 0, requested, why);
}

void gp_destroy(gp_ctx* c) {
    if (!c) return;
    if (c->s) cudaStreamSynchronize(c->s);
    if (c->gs) cudaStreamSynchronize(c->gs);
    free_hier(c->fullF);
    free_hier(c->bandF);
    free_hier(c->fullD);
    free_hier(c->bandD);
    if (c->fft) fft_destroy(c->fft);
    for (void* v : c->kV) cudaFree(v);
    for (void* z : c->kZ) cudaFree(z);
    if (c->kY) cudaFree(c->kY);
    for (auto& p : c->pending) { c->event_pool.push_back(p.a); c->event_pool.push_back(p.b); }
    for (cudaEvent_t e : c->event_pool) cudaEventDestroy(e);
    if (c->ev_in) cudaEventDestroy(c->ev_in);
    if (c->ev_out) cudaEventDestroy(c->ev_out);
    if (c->gs) cudaStreamDestroy(c->gs);
    for (void* p : c->misc) cudaFree(p);
    if (c->atoms) cudaFree(c->atoms);
    if (c->atoms32) cudaFree(c->atoms32);
    if (c->gtab) cudaFree(c->gtab);
    if (c->gmtab) cudaFree(c->gmtab);
    if (c->rvdw) cudaFree(c->rvdw);
    if (c->ratoms) cudaFree(c->ratoms);
    if (c->ratoms32) cudaFree(c->ratoms32);
    if (c->forces_S) cudaFree(c->forces_S);
    if (c->forces_T) cudaFree(c->forces_T);
    delete c;
}

}  // extern "C"
