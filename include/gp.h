/*
 * gp.h - C ABI of the GB300 generalized-Poisson solver.
 *
 * Solves the generalized Poisson equation of Sanchez, Sued & Scherlis
 * (arXiv:0904.4887), Eq. 3,
 *
 *        div( eps(r) grad phi(r) ) = -4 pi rho(r),
 *
 * on a periodic orthorhombic grid, with eps built from atomic coordinates
 * (the position-dependent dielectric of Sec. II.B), optionally splitting the
 * box into a "dry" part solved by FFT and a "wet" band solved by multigrid
 * and coupling the two self-consistently (Sec. II.C, Scheme 1). Energy is
 * Eq. 4 and forces are Eq. 11 (Appendix B).
 *
 * Conventions shared by every call:
 *   - Fields are contiguous float64 arrays in DEVICE memory, x fastest:
 *     value (i, j, k) at offset i + nx*(j + ny*k). Grid point (i,j,k) sits at
 *     r = (i*hx, j*hy, k*hz), h = L/N.
 *   - Atoms are DEVICE arrays: positions double[n][3] in Angstrom (any value;
 *     wrapped into the cell internally), and Gaussian parameters
 *     double[n][3] = (Z, sigma_core, sigma_cloud) in e and Angstrom.
 *   - Units: Angstrom and elementary charge, Gaussian electrostatics (k = 1):
 *     phi in e/A, energies in e^2/A.
 *   - The caller owns every pointer it passes; the library owns its
 *     workspaces (allocated in gp_create / gp_set_dielectric, freed in
 *     gp_destroy). All work is ordered on the stream given to gp_create;
 *     calls return after the results are complete on that stream unless
 *     stated otherwise.
 *   - Every call returns a gp_status; on failure gp_last_error() describes
 *     it. A CUDA error leaves the context unusable (GP_ERR_CUDA).
 *   - Environment, read by gp_create: GP_NO_GRAPHS=1 runs every launch
 *     sequence directly instead of through captured CUDA graphs (same
 *     results, more host work); GP_TEST_SWEEP_WAIT_POLLS=n sets the poll
 *     budget of the finest-level smoother's bounded waits for every context
 *     of the process (a test hook: 0 makes them expire, so gp_solve returns
 *     GP_ERR_TIMEOUT).
 */
#ifndef GP_GB300_H
#define GP_GB300_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct gp_ctx gp_ctx;

typedef enum {
    GP_OK = 0,
    GP_ERR_INVALID_ARG = 1,   /* bad size, null pointer, unsupported option */
    GP_ERR_NOT_NEUTRAL = 2,   /* |sum rho| h^3 > 1e-10 sum|rho| h^3 */
    GP_ERR_NOT_CONVERGED = 3, /* max_outer reached; phi holds the last iterate */
    GP_ERR_DIVERGED = 4,      /* residual grew 1e3-fold or became non-finite */
    GP_ERR_TIMEOUT = 5,       /* a bounded device wait gave up */
    GP_ERR_CUDA = 6,          /* CUDA runtime error */
    GP_ERR_OOM = 7,           /* device allocation failed */
    GP_ERR_STATE = 8          /* call out of order (e.g. solve before set_dielectric) */
} gp_status;

/* Grid: each extent a power of two, or three times one, and >= 8; nx even. */
typedef struct { int nx, ny, nz; } gp_grid;
/* Orthorhombic periodic cell, Angstrom; every side >= rcut of the kind-0 dielectric. */
typedef struct { double lx, ly, lz; } gp_cell;

/* Solver and dielectric parameters; gp_default_params() fills the defaults. */
typedef struct {
    /* dielectric eps = 1 + (eps0-1) prod_a s(|r-R_a|), s(d) = (1+erf((d-r0)/w))/2,
       product over atoms and periodic images with d < rcut (Sec. II.B). */
    double eps0;          /* 78.36 */
    double r0;            /* 2.5 A */
    double w;             /* 0.5 A */
    double rcut;          /* 6.0 A */
    double dry_thresh;    /* 1e-3: a z-plane is dry when max(eps-1) < dry_thresh */
    int split;            /* 0: multigrid on the whole box; 1: dry/wet split (Scheme 1) */
    int n_dirichlet;      /* split: Dirichlet planes in the dry band (1 default; 0 = all the run allows) */
    int precision;        /* 0: FP64 throughout; 1: FP32 multigrid inside FP64 defect correction (for
                             tol >= 1e-10 the outer residual runs in df64, FP32 hi/lo pairs, whose
                             floor is ~1e-11 of ||b||; in FP64 below that) */
    int nu1, nu2;         /* red-black Gauss-Seidel sweeps before / after the coarse correction (2, 2) */
    int levels;           /* multigrid levels; 0 = automatic (gp_plan_levels: coarsest grid <= 64
                             points where the grid allows, else <= 512) */
    int inner;            /* multigrid-preconditioned CG iterations per outer FP64 correction (5, <= 8) */
    int max_outer;        /* outer FP64 corrections before GP_ERR_NOT_CONVERGED */
    int accel;            /* split: 1 = each FP64 outer correction is solved by flexible GMRES in the
                             working precision, preconditioned by the split (same fixed point);
                             0 = plain self-consistent coupling iteration */
    int restart;          /* split with accel: GMRES steps per outer correction (12, <= 15) */
    int band_vcycles;     /* split: V-cycles on the wet band per application of the split (2) */
    int graph_outer;      /* full box: if > 0, run this many outer corrections as one captured CUDA
                             graph (no host round trip), check the residual once, and continue with
                             the checked loop only if it is not yet below tol (warm-started frames);
                             the graph is kept for the same rho/phi buffers (0 = off, <= 16) */
    int sweep_shape;      /* FP32 finest-level smoother tile (see gp_stats.sweep_shape); -1 = chosen
                             by the autotuner at gp_set_dielectric (-1) */
    int kind;             /* dielectric form: 0 = the erf product above (0); 1 = Eq. 9-10, the dummy
                             density gamma(r) = sum_a exp(-(|r-R_a| - rvdw_a)) over every atom and
                             periodic image within the radius where a bound on the rest of the sum
                             falls below gamma_tail (gp_stats.gamma_cutoff; rcut is not used),
                             eps = 1 + (eps0-1)/(1 + gamma^(2 beta)); 2 = Eq. 19, kind 1 with the
                             solvent excluded below every atom with z_a <= zlim (its term is
                             exp(+(d - rvdw_a)) from its nearest image at points with z < z_a, both
                             inside the cell; eps = 1 where such an exponent reaches
                             (ln(eps0-1)+37)/(2 beta)). Kinds 1, 2 need gp_set_vdw_radii; they do
                             not use r0 and w */
    double beta;          /* kinds 1, 2: the exponent beta of Eq. 10 (2.4) */
    double zlim;          /* kind 2: z_lim of Eq. 19, Angstrom inside the cell (0) */
    int nu_coarse;        /* sweeps before and after the coarse correction on the second coarse level
                             and below, 0 .. 8; the first coarse level and the finest use nu1, nu2;
                             0 = nu1, nu2 everywhere (4: those levels are cheap per sweep, and more
                             sweeps there cut the V-cycles per solve) */
    int inner_adapt;      /* full box: 1 = the first correction runs `inner` CG iterations, each later
                             one as many as the contraction measured over the previous one predicts for
                             half the tolerance (1 .. 2 inner; with precision 1 for at most a 1e-5
                             reduction, the reach of one FP32 correction); 0 = `inner` every time (1) */
    double gamma_tail;    /* kinds 1, 2: bound on the part of gamma the image sum leaves out, in
                             (0, 1e-3] (1e-13). The radius R is the smallest with
                             (4 pi/3V) exp(-R)(u^3 + 3u^2 + 6u + 6) sum_a exp(rvdw_a) <= gamma_tail,
                             u = R + half the cell diagonal, V the cell volume: the images of an
                             atom within r of a point number at most (4 pi/3)(r + u - R)^3/V */
} gp_params;

#define GP_HISTORY 64
typedef struct {
    int outer_iterations;       /* FP64 residual evaluations in the last solve */
    int inner_iterations;       /* preconditioned CG iterations in the last solve */
    int vcycles;                /* V-cycles in the last solve */
    int levels;                 /* multigrid levels in use */
    int split_active;           /* 1 when the last solve used the dry/wet split */
    int band_first;             /* first Dirichlet plane (split) */
    int band_dirichlet;         /* number of Dirichlet planes (split) */
    int dry_planes;             /* z-planes with max(eps-1) < dry_thresh */
    double wet_fraction;        /* grid points handed to multigrid / all points */
    double b_norm;              /* ||4 pi rho||_2 */
    double residual;            /* final ||b - A phi|| / ||b|| (FP64) */
    int history_len;
    double history[GP_HISTORY]; /* relative residual after each outer step */
    int sweep_shape;            /* finest-level FP32 smoother tile in use: 0: 64x8, 1: 32x16,
                                   2: 128x4, 3: 32x8 points (x, y); 4, 5, 6: whole x rows times
                                   4, 6, 8 rows; 7 to 14: whole x rows times 6, 4, 6, 4, 16, 14,
                                   14, 12 rows with a producer warp and 2, 2, 4, 3, 2, 4, 2, 2 rows
                                   per thread (shapes 4 to 14 for nx = 64, 96, 128, 192, 256 where
                                   the tile fits one CTA; otherwise 0) */
    double gamma_cutoff;        /* kinds 1, 2: radius of the Eq. 9 image sum (Angstrom), else 0 */
} gp_stats;

/* Fill *p with the defaults listed beside each field. */
void gp_default_params(gp_params* p);

/* Create a solver for `grid` and `cell`. `cuda_stream` is a cudaStream_t (or
 * NULL for the legacy default stream) on the current device; all work of this
 * context is ordered on it. Allocates the grid-sized workspaces.
 * Errors: GP_ERR_INVALID_ARG (sizes), GP_ERR_OOM, GP_ERR_CUDA. */
gp_status gp_create(gp_grid grid, gp_cell cell, void* cuda_stream, gp_ctx** out);

/* Build eps(R) on the grid from n_atoms positions (device double[n][3]),
 * the per-level multigrid coefficients, the dry-plane flags and the wet band
 * (Sec. II.B: the erf switching product, params->kind 0, Eq. 9-10, kind 1,
 * or Eq. 19, kind 2; Sec. II.C for the band). Must precede gp_solve and gp_energy_forces; call again whenever the
 * atoms move. `params` is copied. Errors: GP_ERR_INVALID_ARG (null params,
 * n_atoms < 0, null atoms with n_atoms > 0, any parameter out of the range
 * stated beside it, rcut larger than the cell (kind 0), a grid or `levels` that does not
 * coarsen; gp_last_error names which), GP_ERR_STATE (kind 1 or 2 without
 * gp_set_vdw_radii for the same n_atoms), GP_ERR_OOM (the multigrid
 * hierarchy is allocated here), GP_ERR_CUDA. Argument errors leave the
 * previous dielectric in place; a failure after the checks leaves the context
 * without one until a later call succeeds. */
gp_status gp_set_dielectric(gp_ctx* ctx, const double* atoms_dev, int n_atoms,
                            const gp_params* params);

/* Van der Waals radii R_vdw of Eq. 9 (device double[n_atoms], Angstrom, each > 0),
 * copied into the context for the kind-1 and kind-2 dielectrics; the next
 * gp_set_dielectric with kind 1 or 2 must pass the same n_atoms. Errors: GP_ERR_INVALID_ARG (null
 * pointer, n_atoms < 1), GP_ERR_OOM, GP_ERR_CUDA. */
gp_status gp_set_vdw_radii(gp_ctx* ctx, const double* radii_dev, int n_atoms);

/* rho(r) = sum_a Z_a [g(r; sigma_core,a) - g(r; sigma_cloud,a)] - mean, with
 * g the normalised Gaussian of standard deviation sigma, each truncated to
 * |dx|,|dy|,|dz| < 8 sigma and summed over periodic images (the Gaussian
 * ionic densities of Sec. II.A). Writes rho_dev (grid-sized). Independent of
 * gp_set_dielectric; n_atoms = 0 gives rho = 0. Errors: GP_ERR_INVALID_ARG
 * (null rho_dev, n_atoms < 0, null atom arrays with n_atoms > 0, a sigma <= 0
 * or an 8 sigma window wider than the cell), GP_ERR_OOM, GP_ERR_CUDA. */
gp_status gp_build_rho(gp_ctx* ctx, const double* atoms_dev, const double* gauss_dev,
                       int n_atoms, double* rho_dev);

/* Solve A phi = -4 pi rho (Eq. 3, 7-point conservative discretisation with
 * arithmetic face means) to ||b - A phi||_2 <= tol ||b||_2, b = -4 pi rho.
 * phi_dev is read as the starting guess (warm start) and overwritten with the
 * solution, returned with mean zero. rho must be neutral (its caller removes
 * the mean). Errors: GP_ERR_INVALID_ARG (null array, tol <= 0), GP_ERR_STATE
 * (no dielectric), GP_ERR_NOT_NEUTRAL, GP_ERR_NOT_CONVERGED / GP_ERR_DIVERGED
 * (phi holds the last iterate and gp_get_stats the residuals), GP_ERR_TIMEOUT
 * (a bounded wait of the finest-level smoother gave up; phi is not valid, the
 * context stays usable), GP_ERR_OOM (workspaces are allocated on first use),
 * GP_ERR_CUDA. On GP_ERR_TIMEOUT the solve has stopped at the first residual
 * readback after the expiry: gp_get_stats then records only the outer
 * iterations that ran before it. */
gp_status gp_solve(gp_ctx* ctx, const double* rho_dev, double* phi_dev, double tol);

/* Energy and forces for the atoms of the last gp_set_dielectric, given the
 * solution phi of gp_solve for rho:
 *   energy_host[0] = E  = h^3/2 sum rho phi                       (Eq. 4)
 *   energy_host[1] = E' = h^3/(8 pi) sum_faces eps_f (grad_f phi)^2 (Eq. 4)
 *   forces_dev[a]  = -(G_eps_a + G_rho_a)  (device double[n][3], may be NULL)
 * with G_eps_a = -h^3/(8 pi) sum_faces (d eps_f / d R_a)(grad_f phi)^2 and
 * G_rho_a = h^3 sum_i phi_i d rho_i / d R_a (Eq. 11, Appendix B). gauss_dev
 * (as in gp_build_rho) may be NULL, then G_rho is omitted (rho held fixed).
 * Because the operator is symmetric, phi is its own adjoint: no extra solve.
 * energy_host may be NULL. Errors: GP_ERR_INVALID_ARG (null phi_dev or
 * rho_dev), GP_ERR_STATE (no dielectric), GP_ERR_OOM, GP_ERR_CUDA. */
gp_status gp_energy_forces(gp_ctx* ctx, const double* phi_dev, const double* rho_dev,
                           const double* gauss_dev, double* energy_host, double* forces_dev);

/* Residual r = b - A phi (b = -4 pi rho) in FP64 into r_dev (grid-sized,
 * device; must not alias rho_dev or phi_dev), and ||r||_2 / ||b||_2 into
 * *rel_host (may be NULL). Uses the eps of the last gp_set_dielectric.
 * Errors: GP_ERR_INVALID_ARG (null array), GP_ERR_STATE (no dielectric),
 * GP_ERR_CUDA. */
gp_status gp_residual(gp_ctx* ctx, const double* rho_dev, const double* phi_dev,
                      double* r_dev, double* rel_host);

/* Residual of the sixth-order operator of Sec. III (Eq. 16-18), in FP64:
 *   r = b - A6 phi - mu eps,  b = -4 pi rho,
 *   (A6 phi)_i = sum_axes (D1 eps)_i (D1 phi)_i + eps_i (D2 phi)_i,
 * D1, D2 the seven-point central first and second derivatives of Eq. 17-18
 * (weights 3/4, -3/20, 1/60 and -49/18, 3/2, -3/20, 1/90), periodic on all
 * axes, with the cell eps of the last gp_set_dielectric. mu is the uniform
 * shift (in the form divided by eps) that makes the periodic non-conservative
 * system solvable: A6 phi + mu eps = b; pass 0 for the plain A6 residual.
 * rho_dev, phi_dev, r_dev: grid-sized FP64 device arrays (x fastest), owned by
 * the caller; r_dev must not alias the inputs. ||r||_2 / ||b||_2 goes to
 * *rel_host (may be NULL). Errors: GP_ERR_INVALID_ARG (null array, mu not
 * finite), GP_ERR_STATE (no dielectric yet), GP_ERR_CUDA. */
gp_status gp_residual6(gp_ctx* ctx, const double* rho_dev, const double* phi_dev, double mu,
                       double* r_dev, double* rel_host);

/* Solve of the sixth-order operator of Sec. III (Eq. 16-18). The periodic
 * operator is not conservative, so the system is bordered (the paper does not
 * treat the periodic case; this is the reading used):
 *   A6 phi + mu eps = -4 pi (rho - mean rho),   sum(phi) = 0,
 * mu a uniform compatibility shift of the form divided by eps. phi_dev
 * (grid-sized FP64, device) is read as the starting guess and overwritten;
 * *mu_host (may be NULL) receives mu. Stops when ||r||_2 <= tol ||b||_2,
 * r = b - A6 phi - mu eps, b = -4 pi (rho - mean rho) (gp_get_stats has the
 * history). Method: flexible GMRES(restart) in FP64 on the field system with
 * the border eliminated, right-preconditioned by `inner` steps of the 7-point
 * multigrid-preconditioned CG in the context's precision. Uses the eps of the
 * last gp_set_dielectric. Errors: GP_ERR_INVALID_ARG (null array, tol <= 0),
 * GP_ERR_STATE (no dielectric), GP_ERR_NOT_NEUTRAL, GP_ERR_NOT_CONVERGED /
 * GP_ERR_DIVERGED (phi holds the last iterate), GP_ERR_OOM (work fields are
 * allocated on first use), GP_ERR_CUDA. */
gp_status gp_solve6(gp_ctx* ctx, const double* rho_dev, double* phi_dev, double* mu_host, double tol);

/* The adjoint of gp_solve6, which its forces need (Appendix B's argument
 * without the symmetry of the conservative operator): the transposed bordered
 * system
 *   A6^T lam + nu 1 = rho - mean rho,   sum(eps lam) = 0,
 * A6^T lam = sum_axes [-D1((D1 eps) lam) + D2(eps lam)]. lam_dev (grid-sized
 * FP64, device) is the starting guess and the result; *nu_host (may be NULL)
 * receives nu. Stops when ||r||_2 <= tol ||rho - mean rho||_2. Same method
 * and errors as gp_solve6. */
gp_status gp_adjoint6(gp_ctx* ctx, const double* rho_dev, double* lam_dev, double* nu_host, double tol);

/* Energy and forces of the sixth-order solution (Eq. 4, Eq. 11 through the
 * adjoint): with phi, mu from gp_solve6 and lam from gp_adjoint6 for the same
 * rho and dielectric,
 *   energy_host[0] = E = h^3/2 sum rho phi
 *   forces_dev[a]  = -(G_eps_a + G_rho_a)   (device double[n][3], may be NULL)
 *   G_eps_a = -h^3/2 sum_j (d eps_j / d R_a) (g_j + mu lam_j),
 *   g = sum_axes [-D1(lam D1 phi) + lam D2 phi],
 *   G_rho_a = h^3/2 sum_j (phi_j - 4 pi lam_j) d rho_j / d R_a (mean removed),
 * gauss_dev as in gp_energy_forces (NULL: rho held fixed, G_rho omitted).
 * energy_host (double[1]) may be NULL; lam_dev may be NULL when forces_dev is.
 * Errors: GP_ERR_INVALID_ARG (null phi or rho, mu not finite, forces without
 * lam), GP_ERR_STATE (no dielectric), GP_ERR_OOM, GP_ERR_CUDA. */
gp_status gp_energy_forces6(gp_ctx* ctx, const double* phi_dev, double mu, const double* lam_dev,
                            const double* rho_dev, const double* gauss_dev, double* energy_host,
                            double* forces_dev);

/* Vacuum solve L phi = src with the 7-point Laplacian (eps = 1), by the
 * hand-written FFT (Eq. 15 with the symbol of the discrete operator); the
 * k = 0 mode is dropped so phi has mean zero. src_dev, phi_dev grid-sized
 * device arrays (may alias). The plan and its workspace are made on the first
 * call. Errors: GP_ERR_INVALID_ARG (null array, or an extent the FFT cannot
 * plan), GP_ERR_OOM, GP_ERR_CUDA. */
gp_status gp_fft_poisson(gp_ctx* ctx, const double* src_dev, double* phi_dev);

/* The same vacuum solve in FP32 arithmetic: the instance the mixed-precision
 * dry/wet split applies to its working-precision residual (Scheme 1, Eq. 15).
 * src_dev, phi_dev: grid-sized float32 device arrays (may alias); plan,
 * workspace and errors as for gp_fft_poisson. */
gp_status gp_fft_poisson_f32(gp_ctx* ctx, const float* src_dev, float* phi_dev);

/* Copy eps (FP64, grid-sized) of the last gp_set_dielectric into eps_dev.
 * Errors: GP_ERR_INVALID_ARG (null), GP_ERR_STATE (no dielectric), GP_ERR_CUDA. */
gp_status gp_get_eps(gp_ctx* ctx, double* eps_dev);

/* Per-plane max_xy(eps - 1) into plane_max_host[nz] (host memory).
 * Errors: GP_ERR_INVALID_ARG (null), GP_ERR_STATE (no dielectric), GP_ERR_CUDA. */
gp_status gp_get_plane_max(gp_ctx* ctx, double* plane_max_host);

/* Host-only planner of the wet band (Sec. II.C reading): from per-plane dry
 * flags dry[nz] (1 = dry), put the Dirichlet planes in the middle of the
 * longest periodic run of dry planes, n_dirichlet of them (0 = as many as the
 * run holds), reduced to 1 + m 2^(levels-1) so that the band of the other
 * nz - nd planes coarsens levels-1 times. Writes *first (first Dirichlet
 * plane) and *nd. Returns 1 if a band exists, 0 if no plane is dry, -1 on bad
 * arguments. Needs no GPU. */
int gp_plan_band(const int* dry, int nz, int levels, int n_dirichlet, int* first, int* nd);

/* Host-only: multigrid levels for a grid (zper = 1 periodic z with nz planes,
 * 0 Dirichlet z with nz interior planes). Each coarsening halves nx, ny and the
 * periodic nz (the Dirichlet nz interior planes become (nz+1)/2 - 1) and needs
 * every extent to divide evenly and stay >= 2 (a Dirichlet nz >= 1).
 * requested > 0: `requested` if the grid coarsens requested-1 times with <= 512
 * coarsest points, else -1. requested = 0: the fewest levels (>= 2) whose
 * coarsest grid has <= 64 points, else the most levels whose coarsest grid has
 * <= 512 points, else -1. Needs no GPU. */
int gp_plan_levels(int nx, int ny, int nz, int zper, int requested);

/* Largest nz accepted by gp_residual_noalloc: its scratch holds two partial
 * sums per z-plane, 2 * 4096 doubles (64 KiB) per GPU. */
#define GP_NOALLOC_MAX_PLANES 4096

/* gp_residual_noalloc: the FP64 residual of gp_residual, for callers that
 * cannot allocate device memory (no cudaMalloc: for example code running
 * where the allocator is owned by someone else, inside a memory pool that
 * must not grow, or in a plug-in that may not create a solver context). The
 * paper has no counterpart; this is a deployment entry point.
 *
 *   r = -4 pi rho - A phi  (the FP64 7-point face-mean operator of gp_residual,
 *                           with eps given by the caller instead of a context)
 *   rel_dev[0] = ||r||_2 / ||4 pi rho||_2
 *
 * Arguments: grid and cell as for gp_create; eps_dev, rho_dev, phi_dev and
 * r_dev are grid-sized float64 device arrays (x fastest); rel_dev is one
 * device double; cuda_stream is a cudaStream_t (NULL = legacy stream). The
 * call only enqueues work on that stream and returns; nothing is allocated or
 * freed, and no context is needed.
 *
 * Scratch: a file-scope device array of 2 * GP_NOALLOC_MAX_PLANES doubles,
 * present on every GPU that loads the library until the process exits.
 * Every call overwrites the slots it reads, but all calls share the one
 * array: calls that overlap on the GPU (different streams, or threads) race
 * and give wrong sums; serialise them. The first call on each device looks up
 * the array's device address (cudaGetSymbolAddress) and caches it, so make
 * that first call outside any CUDA stream capture.
 *
 * Errors: GP_ERR_INVALID_ARG for a null pointer, an extent below 2, a
 * non-positive cell side, or nz > GP_NOALLOC_MAX_PLANES; GP_ERR_CUDA if the
 * address lookup or a launch fails. */
gp_status gp_residual_noalloc(gp_grid grid, gp_cell cell, const double* eps_dev, const double* rho_dev,
                              const double* phi_dev, double* r_dev, double* rel_dev, void* cuda_stream);

/* Kernel groups timed by gp_profile (indices into the arrays of gp_get_profile). */
enum {
    GP_PROF_EPS = 0,         /* dielectric builder */
    GP_PROF_RHO = 1,         /* Gaussian charge density */
    GP_PROF_FORCES_EPS = 2,  /* dielectric (solvent) force */
    GP_PROF_FORCES_RHO = 3,  /* charge-motion force */
    GP_PROF_RES64 = 4,       /* FP64 full-box residual + norm (outer correction) */
    GP_PROF_SMOOTH0 = 5,     /* red-black Gauss-Seidel on the finest multigrid level */
    GP_PROF_MG_FINE = 6,     /* finest-level residual, restriction, prolongation */
    GP_PROF_MG_COARSE = 7,   /* all coarser levels and the coarsest solve */
    GP_PROF_KRYLOV = 8,      /* CG operator application, dot products, updates */
    GP_PROF_FFT = 9,         /* the five FFT Poisson passes */
    GP_PROF_SETUP = 10,      /* coarse coefficients and the coarsest inverse */
    GP_PROF_MISC = 11,       /* reductions, gauge, atom wrapping */
    GP_PROF_UPDATE64 = 12,   /* FP64 phi update */
    GP_PROF_ENERGY = 13,     /* energy reductions */
    GP_PROF_SMOOTH0_ZERO = 14, /* the first finest-level sweep of a V-cycle, from u = 0 (reads no u) */
    GP_PROF_KINDS = 15
};

/* Enable (1) or disable (0) CUDA-event timing of kernel groups on this
 * context's stream. Timing adds two event records per group and never
 * changes results. Enabling resets the totals. */
gp_status gp_profile(gp_ctx* ctx, int enable);

/* Totals since gp_profile(ctx, 1): ms[k] device milliseconds, launches[k]
 * kernel launches and groups[k] timed groups for each kind k < n (n <=
 * GP_PROF_KINDS); host arrays, any may be NULL. */
gp_status gp_get_profile(const gp_ctx* ctx, double* ms, long* launches, long* groups, int n);

/* Process-wide count of kernels this library has launched (host-only). */
long gp_launch_count(void);

/* Statistics of the last gp_set_dielectric / gp_solve. */
gp_status gp_get_stats(const gp_ctx* ctx, gp_stats* out);

/* Message describing the last error of this context ("" if none). */
const char* gp_last_error(const gp_ctx* ctx);

/* Free every workspace and the context. Accepts NULL. */
void gp_destroy(gp_ctx* ctx);

#ifdef __cplusplus
}
#endif
#endif /* GP_GB300_H */
