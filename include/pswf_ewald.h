/*
 * pswf_ewald.h -- C ABI of the GB300 PSWF fast Ewald library (libpswf_ewald.so).
 *
 * Computes, for n point charges rho_j at x_j in the triply periodic cube
 * [0, L)^3, the Coulomb potential phi_i (Gaussian units, phi = sum rho/r,
 * self-interaction excluded, all periodic images included), the forces
 * F_i = -rho_i grad phi_i and the energy E = 1/2 sum_i rho_i phi_i
 * (paper: Sec. 3.1, eqs. potential1/potential2 and the Remark on energy and
 * forces).  The method is the PSWF split + PSWF window fast Ewald summation of
 * Sec. 4 (Alg. 2 for the Fourier-space part, the compactly supported residual
 * R of eq. R for the real-space part) with parameters from Alg. 3 (Sec. 6).
 *
 * Conventions shared by every entry point
 *  - Positions are any finite reals; they are wrapped into [0, L)^3.
 *  - Layouts: x is (n, 3) row-major float64, rho is (n) float64, phi is (n)
 *    float64, force is (n, 3) row-major float64; outputs follow the caller's
 *    particle order.
 *  - The caller owns every buffer passed in; the plan owns its workspace.
 *  - A plan is not reentrant: calls on one plan must not overlap in time
 *    (use one plan per concurrent stream).
 *  - Return value: 0 (EWALD_OK) or one of the EWALD_E* codes below; no C++
 *    exception crosses the ABI.  ewald_last_error() returns a thread-local
 *    message for the last failure on the calling thread.
 */
#ifndef PSWF_EWALD_H
#define PSWF_EWALD_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ------------------------------------------------------- */
#define EWALD_OK           0
#define EWALD_EINVAL       1  /* bad argument: L <= 0, n < 2, tol outside [1e-13, 1e-2], NULL pointer, ... */
#define EWALD_ENONNEUTRAL  2  /* |sum rho| > 1e-10 sum |rho| (charge neutrality, Sec. 1 and Alg. 1) */
#define EWALD_ENOMEM       3  /* device or host allocation failed */
#define EWALD_ECUDA        4  /* a CUDA runtime call failed */
#define EWALD_ECUFFT       5  /* a cuFFT call failed */
#define EWALD_ETOOBIG      6  /* grid, window support or particle count beyond the library limits */
#define EWALD_ETIMEOUT     7  /* a bounded device wait expired (tensor-core spreading: an MMA
                                         completion did not arrive within ~1 s) */
#define EWALD_ENONFINITE   8  /* an input position or charge is not finite */

/* ---- precision of the device path ------------------------------------- */
#define EWALD_FP64   0   /* every stage in float64 */
#define EWALD_MIXED  1   /* spreading, FFT, interpolation and the real-space sum in float32
                            (positions reduced to per-tile/per-cell offsets in float64 first);
                            outputs, energy and self term in float64.  For tol < 1e-7 a MIXED
                            plan runs the EWALD_FLOATFLOAT kernels instead (float32 products
                            cannot reach it); ewald_params.precision reports the path taken. */
#define EWALD_FLOATFLOAT 2 /* spreading, interpolation and the real-space sum in float-float
                            arithmetic (unevaluated sums of two float32, ~48 bits, on the float32
                            pipes); grid, FFT and scaling in float64; outputs in float64.
                            Accuracy of the float64 path down to tol ~1e-12 at a fraction of its
                            cost on GPUs with reduced float64 throughput.  Positions, charges and
                            L must lie in the float32 exponent range. */

/* ---- options (ewald_opts_default fills the defaults) -------------------- */
typedef struct ewald_opts {
    int    precision;     /* EWALD_FP64, EWALD_MIXED or EWALD_FLOATFLOAT (default EWALD_FP64) */
    double rc;            /* <= 0: automatic cutoff rule; > 0: upper bound on the cutoff (length units);
                             NaN: EWALD_EINVAL */
    double grid_density;  /* target m^3 / n for the automatic cutoff rule; 0 (default): the
                             measured optima of the GB300 kernels, 6 for float32 plans (EWALD_MIXED
                             at tol >= 1e-7) and 3 for the float64 and float-float plans */
    double tol_safety;    /* the plan is sized for tol * tol_safety (default 0.25; forces have no
                             error model in the paper and measure ~2-5x the potential error) */
    int    sr_reach;      /* cells per cutoff radius in the real-space cell list, 1..4 (along x and
                             y; EWALD_MIXED plans keep 4 along z); 0 (default): 1 for EWALD_MIXED
                             plans, otherwise ~3 particles per cell (~1.5 for float-float) */
    int    window_extra;  /* window support added to the Alg. 3 value of P (default 0) */
    int    autotune;      /* 1: ewald_plan_create times candidate plans on a synthetic uniform
                             system of n alternating unit charges in the plan's box and keeps
                             the fastest: first the grid densities {1.5, 2, 3, 4, 6, 8, 12}
                             (distinct m only; grid_density is then ignored), then, at the
                             fastest density, the real-space cell shapes sr_reach = 1..4 (only
                             when sr_reach is 0).  The cutoff, and with it the balance between
                             the real-space sum and Alg. 2, is what the paper leaves to
                             measurement (Sec. 6.2.2).  0 (default): off. */
    int    spread_kernel; /* Alg. 2 step 1 on float32 (EWALD_MIXED, tol >= 1e-7) plans: 1 = CUDA-core
                             kernel (per-column register accumulation), 2 = tensor-core kernel
                             (tcgen05 split-TF32 products per tile, window support P <= 14; within
                             the accuracy bar down to tol 1e-6; faster timed alone, 1-2% slower in
                             the concurrent step, measured), 0 (default) = automatic = CUDA cores.
                             Other plans always use their CUDA-core kernel. */
} ewald_opts;

/* ---- derived parameters (Alg. 3 and the library's readings of it) ------ */
typedef struct ewald_params {
    double L;          /* box edge */
    double rc;         /* cutoff radius r_c (R(r) = 0 for r >= r_c) */
    double cs;         /* split bandlimit c_s (eq. csrc: c_s / r_c = pi m / L) */
    double cw;         /* window bandlimit c_w = pi P / 2 (eq. cwP) */
    double cw_target;  /* c_w from eq. cwW before rounding P */
    double alpha;      /* window half-width alpha = P h / 2 */
    double h;          /* grid spacing L / m */
    double lambda_s;   /* lambda_0(c_s) */
    double lambda_w;   /* lambda_0(c_w) */
    double self_coeff; /* 2 / (lambda_0(c_s) r_c): phi_i^self = -self_coeff * rho_i */
    double tol;        /* requested relative tolerance */
    double fit_tol;    /* max abs error allowed for the polynomial fits */
    int64_t n;         /* particle count the plan is for */
    int    m;          /* FFT grid points per axis (multiple of 4, prime factors <= 7) */
    int    P;          /* window support in grid points per axis */
    int    deg_w;      /* degree of the per-interval window polynomials (in z = 2f - 1) */
    int    deg_r;      /* degree of the radial polynomials (in u = 2 r^2 / r_c^2 - 1) */
    int    tile;       /* spreading tile edge T (grid points), m % T == 0: 8 for EWALD_MIXED
                          plans, 4 otherwise (m is rounded to a multiple of it) */
    int    ncell;      /* real-space cells per axis */
    int    sr_reach;   /* real-space neighbour reach in cells */
    int    precision;  /* path the plan runs: EWALD_FP64, EWALD_MIXED or EWALD_FLOATFLOAT */
    /* box shape (cuboid boxes: Remark on cuboid domains in Sec. 6.1).  A cube has box = (L, L, L),
     * grid = (m, m, m), cells = (ncell, ncell, ncell) and deg_g = 0.  For a cuboid the scalar L, m,
     * h, alpha and ncell above are those of the x axis; rc, cs, cw, P are common to all axes. */
    double box[3];     /* edges L_x, L_y, L_z */
    int    grid[3];    /* FFT grid points per axis (each a multiple of tile, prime factors <= 7) */
    int    cells[3];   /* real-space cells per axis */
    int    deg_g;      /* cuboids: degree of the in-band mollifier transform polynomial (scaling) */
    int    sr_reach_z; /* real-space cells per cutoff radius along z (cells of edge >= rc / sr_reach
                          along x, y and >= rc / sr_reach_z along z): 4 for EWALD_MIXED plans, whose
                          real-space kernel walks z windows of columns; sr_reach otherwise */
    int    spread_kernel; /* spreading kernel of the plan: 1 CUDA cores, 2 tensor cores */
} ewald_params;

typedef struct ewald_plan_s* ewald_plan;   /* opaque, owned by the library */

/* Fill *opts with the defaults listed above.  Returns EWALD_EINVAL on NULL. */
int ewald_opts_default(ewald_opts* opts);

/* Host only (no CUDA call): run Alg. 3 (Sec. 6.4) for a box of edge L holding
 * n particles at relative tolerance tol and fill *out.  opts may be NULL.
 * Errors: EWALD_EINVAL (NULL out, L <= 0 or not finite, n < 2, tol outside
 * [1e-13, 1e-2], an option out of its range), EWALD_ETOOBIG (grid or window
 * support beyond the library limits). */
int ewald_plan_params(double L, int64_t n, double tol, const ewald_opts* opts,
                      ewald_params* out);

/* Create a plan on the current CUDA device: parameters as ewald_plan_params,
 * PSWF tables, cuFFT plans and a device workspace sized for n particles.
 * On success *out holds the plan; release it with ewald_plan_destroy.  On
 * failure *out is NULL and nothing stays allocated.  Errors: those of
 * ewald_plan_params, EWALD_ENOMEM (device or pinned host memory),
 * EWALD_ECUDA (no usable device, a failed launch while autotuning),
 * EWALD_ECUFFT (cuFFT plan creation). */
int ewald_plan_create(double L, int64_t n, double tol, const ewald_opts* opts,
                      ewald_plan* out);

/* Cuboid boxes (Remark on cuboid domains, Sec. 6.1): as ewald_plan_params / ewald_plan_create for the
 * box [0, L[0]) x [0, L[1]) x [0, L[2]) (L: HOST array of 3 edges).  The parameters are derived in
 * units of the shortest edge; every axis gets its own grid size (common spacing up to rounding) and
 * real-space cell count; ewald_params.box / grid / cells report them.  Equal edges give exactly the
 * cube's plan.  Positions wrap per axis; everything else (layouts, errors, evaluation entry points)
 * is as for cubes.  Batches (ewald_plan_batch_create) and ewald_spread_static take cubes only. */
int ewald_plan_params_box(const double* L, int64_t n, double tol, const ewald_opts* opts,
                          ewald_params* out);
int ewald_plan_create_box(const double* L, int64_t n, double tol, const ewald_opts* opts,
                          ewald_plan* out);

/* Copy the plan's parameters into *out.  Host only.  EWALD_EINVAL on NULL. */
int ewald_plan_query(ewald_plan plan, ewald_params* out);

/* Evaluate on device buffers (Alg. 2 steps 1-5 plus the real-space sum, self
 * term, forces and energy).  x, rho: DEVICE pointers, layouts above, n = the
 * plan's n.  phi, force: DEVICE pointers or NULL (not wanted).  energy: HOST
 * pointer or NULL; when non-NULL the call synchronises `stream` and also
 * reports EWALD_ENONNEUTRAL / EWALD_ENONFINITE detected on the device.
 * stream: a cudaStream_t (NULL = legacy default stream).  Without `energy`
 * the call is asynchronous; ewald_check() reports the device-side status. */
int ewald_eval(ewald_plan plan, const double* x, const double* rho,
               double* phi, double* force, double* energy, void* stream);

/* Same as ewald_eval but every pointer is a HOST pointer (pinned or pageable):
 * copies x and rho to the device, evaluates, copies phi/force back, and
 * synchronises `stream` before returning. */
int ewald_eval_host(ewald_plan plan, const double* x, const double* rho,
                    double* phi, double* force, double* energy, void* stream);

/* Synchronise `stream` and return the device status of the last evaluation
 * (EWALD_OK, EWALD_ENONNEUTRAL or EWALD_ENONFINITE). */
int ewald_check(ewald_plan plan, void* stream);

/* Test access: copy an internal stage of the last evaluation to HOST memory
 * as float64.  which = 0: the spread grid a_l (m^3, z fastest; Alg. 2 step 1);
 * which = 1: the grid b_l after scaling and the inverse FFT (Alg. 2 step 4).
 * host_out must hold grid[0]*grid[1]*grid[2] doubles (m^3 for a cube; the
 * per-axis grid of ewald_params).  Synchronises the device.  EWALD_EINVAL for
 * a NULL or batch plan, a NULL host_out or another `which`. */
int ewald_debug_grid(ewald_plan plan, int which, double* host_out);

/* Release a plan (single-system or batch).  NULL is ignored. */
void ewald_plan_destroy(ewald_plan plan);

/* ---- batches of independent systems ------------------------------------
 * Many small periodic systems evaluated by one call, e.g. an ensemble of
 * MD replicas or a screening set (the paper's method applied per system;
 * Sec. 7 evaluates single systems).  Each system b has its own cubic box
 * L[b], particle count n[b] and plan (Alg. 3 per system, every opts field
 * applied, autotune ignored); all share tol.
 *
 * ewald_plan_batch_create: nsys in [1, 4096]; L and n are HOST arrays of
 * nsys entries.  Returns a batch plan for ewald_eval_batch / ewald_plan_query
 * (which reports system 0) / ewald_plan_destroy; ewald_eval on a batch plan
 * returns EWALD_EINVAL.
 *
 * ewald_eval_batch: offsets is a HOST array of nsys + 1 entries with
 * offsets[0] = 0 and offsets[b+1] - offsets[b] = n[b]; system b occupies
 * rows offsets[b] .. offsets[b+1]-1 of the DEVICE arrays x (rows of 3),
 * rho, phi and force (phi, force may be NULL).  energy: HOST array of nsys
 * entries or NULL.  Batches of EWALD_MIXED (float32) systems that share the
 * window support P run every stage as one kernel launch over all systems
 * (batched cuFFT per grid size, the real-space sum on a second stream);
 * other batches enqueue every system's pipeline as one CUDA graph on
 * `stream` (captured on the first call and again whenever a buffer pointer
 * changes; the systems' pipelines are independent branches that run
 * concurrently).  Either way the call then synchronises `stream` and reports
 * the first system
 * found non-neutral (EWALD_ENONNEUTRAL) or with non-finite input
 * (EWALD_ENONFINITE); ewald_last_error() names the system.  The batch plan
 * is not reentrant: one call at a time per plan. */
int ewald_plan_batch_create(int nsys, const double* L, const int64_t* n, double tol,
                            const ewald_opts* opts, ewald_plan* out);
int ewald_eval_batch(ewald_plan plan, const int64_t* offsets, const double* x,
                     const double* rho, double* phi, double* force, double* energy,
                     void* stream);

/* ---- per-stage timing ----------------------------------------------------
 * Stages, in pipeline order: 0 bin+sort, 1 spread (Alg. 2 step 1), 2 halo sum,
 * 3 forward FFT (step 2), 4 scaling (step 3), 5 inverse FFT (step 4),
 * 6 interpolation (step 5), 7 real-space sum, 8 energy reduction.
 * While enabled, every ewald_eval / ewald_eval_host records CUDA events on its
 * stream at the stage boundaries (no synchronisation).  enable = 1: the
 * real-space sum stays concurrent with Alg. 2 (stage times include the
 * overlap); enable = 2: the two are serialised on the caller's stream, so each
 * stage time is its kernels' duration alone (same kernels, no overlap).
 * enable != 0 also clears the accumulated records; enable = 0 stops recording
 * and restores concurrent execution. */
#define EWALD_NSTAGES 9
int ewald_profile(ewald_plan plan, int enable);

/* Synchronise the recorded events and write the summed milliseconds of each
 * stage over the recorded evaluations into ms[EWALD_NSTAGES] and their number
 * into *count. */
int ewald_profile_read(ewald_plan plan, double* ms, int* count);

/* Check of the device timeout path (no plan): one warp waits on an mbarrier
 * that nothing arrives at, with the bounded wait of the tensor-core spreading
 * (here 2e7 SM clocks, ~10 ms, instead of 2e9).  Returns EWALD_ETIMEOUT when the wait
 * ran out, as it must, after which the CUDA context stays usable. */
int ewald_debug_wait_timeout(void);

/* ---- host-side tables (no CUDA call), for tests and tooling ------------- */
/* ewald_window_fit, ewald_radial_fit and ewald_scale_table take the parameters
 * of ewald_plan_params / ewald_plan_query; values the planner never produces
 * (window support outside [3, 24], polynomial degrees out of range,
 * non-positive or non-finite bandlimits, cutoff, box or spacing, grid sizes
 * outside [4, 1024], m or L other than the x-axis entries of grid and box)
 * return EWALD_EINVAL before any table is built. */

/* The planner's PSWF (App. B: Legendre expansion, Sturm bisection + inverse
 * iteration): psi_0^c and its derivative at nx points |x| <= 1, plus chi_0 and
 * lambda_0.  Any output pointer may be NULL. */
int ewald_pswf_eval(double c, int nx, const double* x, double* psi, double* dpsi,
                    double* chi, double* lambda0);

/* Lambert W on branch 0 (z >= -1/e) or -1 (-1/e <= z < 0), Halley iteration.
 * For another branch, a NaN z or z outside the branch's domain it returns NaN
 * and sets the message of ewald_last_error(). */
double ewald_lambertw(int branch, double z);

/* The fitted window polynomials of a plan (Remark on piecewise polynomials in
 * Sec. 4.3): for each z in [-1, 1] write the P weights
 * w_a = psi(s_a)/psi(0), s_a = (z + P - 1 - 2a)/P, into w[i*P + a] and their
 * x-derivatives psi'(s_a)/(alpha psi(0)) into dw[i*P + a] (dw may be NULL). */
int ewald_window_fit(const ewald_params* p, int nz, const double* z, double* w, double* dw);

/* The fitted radial functions of a plan at nr distances 0 < r < rc:
 * R[i] = R(r) (eq. R) and G[i] = -R'(r)/r (pair force factor); G may be NULL. */
int ewald_radial_fit(const ewald_params* p, int nr, const double* r, double* R, double* G);

/* The diagonal scaling S(k) of Alg. 2 step 3 on the half spectrum the library
 * uses: S[(ix*my + iy)*(mz/2+1) + iz] for k = (kx(ix), ky(iy), iz), where
 * (mx, my, mz) = p->grid, kx(i) = i for i < mx/2 and i - mx otherwise (ky
 * alike).  Cubes: S = 0 outside the open ball 0 < |k| < m/2.  Cuboids (Remark
 * on cuboid domains, Sec. 6.1): S = 0 outside the mollifier's band
 * 0 < |omega| < c_s / r_c, M-hat from the plan's polynomial of gammahat, as
 * the scaling kernel evaluates it.  S holds mx*my*(mz/2+1) doubles (HOST).
 * EWALD_EINVAL on NULL. */
int ewald_scale_table(const ewald_params* p, double* S);

/* ---- spreading without device allocation -------------------------------
 * The paper has no counterpart to this entry point; it exists for callers that
 * cannot allocate device memory when they need the spread grid: code running
 * under an external allocator that forbids cudaMalloc/cudaFree, plugins inside
 * a host application that owns all GPU memory, and latency-critical loops that
 * must not hit the implicit synchronisation of allocation calls.
 *
 * Spreads n = p->n charges (Alg. 2 step 1, float64 arithmetic) onto the
 * caller's grid: x (n,3) and rho (n) float64 DEVICE pointers as in ewald_eval,
 * grid an m^3 float64 DEVICE array (z fastest) that receives a_l.  p holds the
 * parameters of ewald_plan_params / ewald_plan_query for an EWALD_FP64 or
 * EWALD_FLOATFLOAT plan (tile 4; parameters of an EWALD_MIXED plan, tile 8,
 * are rejected with their own message); the window degree p->deg_w is used as
 * given.  The result equals the spread grid of ewald_eval for the same plan
 * bit for bit.  Asynchronous on `stream`.  The inputs are not checked: a
 * non-finite position spreads its charge at the origin and a non-finite
 * charge spreads nothing, without an error code (ewald_eval reports both).
 *
 * Scratch: a fixed 64 MiB array in the library's device image (every GPU that
 * loads the library holds it until the process exits).  Problems needing more
 * (about 104 n bytes plus 8 (m/4)^3 (P+3)^3 bytes plus 8 KB) return EWALD_ETOOBIG.
 * No cudaMalloc, cudaFree or other allocating call is made.  The first call on
 * each device looks up the array's device address (cudaGetSymbolAddress) with
 * that device current; make that first call before any stream capture.  The
 * fitted window table stays in the array: a call with the same (c_w, P, deg_w)
 * as the previous one on that device skips the host fit and the table copy.
 * All calls share the one array and it keeps the previous call's contents (the
 * entry point clears what must start at zero), so calls whose GPU work
 * overlaps -- on different streams or host threads -- race and must be
 * serialised by the caller.  Errors: EWALD_EINVAL (NULL pointer, parameters
 * not from the planner or of a tile-8 plan), EWALD_ETOOBIG (scratch limit),
 * EWALD_ECUDA. */
int ewald_spread_static(const ewald_params* p, const double* x, const double* rho, double* grid, void* stream);

const char* ewald_error_string(int code);
const char* ewald_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* PSWF_EWALD_H */
