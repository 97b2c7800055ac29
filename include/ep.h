/*
 * ep.h -- C ABI of the GB300 (sm_103a) monodomain IMEX step.
 *
 * One time step of the cardiac monodomain model as discretised in lifex-ep
 * (Africa et al., arXiv 2308.01651, Sec. 1.2):
 *   1. the ionic model at every mesh node, Eq. (4): states whose rate is
 *      affine in themselves are taken implicitly, the others explicitly, so
 *      the update is a direct division; then I_ion(u_EXT, w_{n+1}) at the
 *      nodes (ionic current interpolation);
 *   2. the linear system Eq. (6), (alpha_BDF/dt M + K) u_{n+1} =
 *      M (u_BDF/dt - I_ion + I_app), with Q1 hexahedral mass and stiffness
 *      matrices, K from the orthotropic tensor of Eq. (3).
 * Everything runs in this library's CUDA kernels on one GPU; the library
 * owns all device memory of an instance.
 *
 * Conventions for every entry point:
 *   - Every call returns an ep_status; nothing aborts the process.  On any
 *     status other than EP_OK, ep_last_error() returns a message (per host
 *     thread) describing the failure.
 *   - Input arrays are read during the call and copied; the caller keeps
 *     ownership.  Output arrays are caller-owned host buffers.
 *   - Units: ms, cm, mV (the Bueno-Orovio model's dimensionless potential u
 *     is reported as 85.7 u - 84 mV, Sec. 3.2.3), mS/cm, 1/cm, uF/cm^2.
 *   - An instance is used by one host thread at a time; its work is ordered
 *     on its CUDA stream.
 *
 * Node numbering of the structured meshes: node (i, j, k) has index
 * i + (nx+1) * (j + NY * k), with NY = ny + 1 for a slab and NY = ny for a
 * shell (periodic in j).  Element (i, j, k) has local nodes a = ia + 2 ib +
 * 4 ic at (i+ia, j+ib, k+ic).
 */
#ifndef EP_GB300_H
#define EP_GB300_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct ep_instance ep_instance;

typedef enum {
    EP_OK = 0,
    EP_EINVAL = 1,       /* an argument is invalid (message says which) */
    EP_ENOMEM = 2,       /* device or host allocation failed */
    EP_ENOCONV = 3,      /* the linear solver did not reach its tolerance */
    EP_ENAN = 4,         /* a potential became non-finite */
    EP_ETIMEOUT = 5,     /* a bounded device wait gave up */
    EP_ECUDA = 6,        /* a CUDA runtime call failed */
    EP_EUNSUPPORTED = 7  /* a valid request this library does not implement */
} ep_status;

/* Meshes: EP_MESH_SLAB, the box [0,L] with nx x ny x nz trilinear hexahedra;
 * EP_MESH_SHELL, a periodic-in-j structured shell given by node coordinates;
 * EP_MESH_SLAB_Q2, the box with nx x ny x nz triquadratic 27-node hexahedra
 * (Sec. 1.2: hexahedral elements of any polynomial degree), nodes on the grid
 * of half the element size, (2nx+1)(2ny+1)(2nz+1) of them, node
 * (I, J, K) = I + (2nx+1) (J + (2ny+1) K).  Q2 operators are matrix-free
 * (sum factorisation on 3 x 3 x 3 Gauss points) and need FP32_REFINED
 * precision and one region (else EP_EUNSUPPORTED). */
enum { EP_MESH_SLAB = 0, EP_MESH_SHELL = 1, EP_MESH_SLAB_Q2 = 2 };
enum { EP_MODEL_BO = 0, EP_MODEL_TTP06 = 1 };
enum { EP_CELL_ENDO = 0, EP_CELL_MID = 1, EP_CELL_EPI = 2 };
/* Arithmetic of the step.  FP64: every quantity in double, CG on the FP64
 * operator.  FP32_REFINED: ionic gates, ionic current and the CG inner solve
 * in float, inside iterative refinement whose right-hand side, residual and
 * solution update are carried in float-float (double-single, 48-bit
 * significand) arithmetic -- GB300's FP64 pipe is ~60x slower than FP32 --
 * and FP64 ionic concentrations; the potentials are stored in double. */
enum { EP_PREC_FP64 = 0, EP_PREC_FP32_REFINED = 1 };
/* FP32 inner operator of the refined solver.  AUTO: on a slab both the
 * matrix-free apply and the assembled FP32 stencil are built and ep_create
 * times them on the instance, keeping the faster (ep_stats reports both
 * times); elsewhere the stencil. */
enum { EP_OP_AUTO = 0, EP_OP_MATRIX_FREE = 1, EP_OP_STENCIL = 2 };

/* Mesh (Sec. 1.2: Q1 hexahedra).
 *   SLAB : the box [0,L0]x[0,L1]x[0,L2] split into nx x ny x nz equal
 *          hexahedra; xyz is ignored.
 *   SHELL: a structured hexahedral shell, nx elements across the wall, ny
 *          around (periodic, ny >= 3), nz along; xyz holds the
 *          n_nodes x 3 node coordinates (cm) in the numbering above.
 * n_nodes must match the count implied by kind and sizes. */
typedef struct {
    int32_t kind;
    int32_t nx, ny, nz;
    double L[3];
    const double* xyz;
    int64_t n_nodes;
    /* Subdomain label per element (Sec. 1.1.2: a labelled partition of the
     * domain), or NULL for one region.  Element (i, j, k) -- the hexahedron
     * spanning nodes i..i+1, j..j+1, k..k+1, j wrapping on the shell -- is
     * entry i + nx (j + ny k); n_elems = nx * ny * nz bytes, each below
     * ep_conductivities.n_regions. */
    const uint8_t* region;
} ep_mesh;

/* Nodal fibre (f0) and sheet (s0) directions, n_nodes x 3 each (Eq. (3)).
 * n0 is implied (orthonormal frame); the diffusion tensor at a quadrature
 * point is dn I + (dl - dn) f f^T + (dt - dn) s s^T with f, s the Q1
 * interpolants of f0, s0 (not renormalised). */
typedef struct {
    const double* f0;
    const double* s0;
} ep_fibers;

/* Conductivities (Eq. (3)).  If is_D != 0, sigma_* are diffusivities in
 * cm^2/ms; otherwise they are conductivities in mS/cm and the library
 * rescales D = sigma / (chi_m C_m) (Sec. 1.1.2) with chi_m in 1/cm and C_m in
 * uF/cm^2.  All must be positive and finite.
 *
 * With a region label on the mesh, region r uses region_sigma[r] (l, t, n;
 * same units) instead of sigma_*, for r < n_regions (1..EP_MAX_REGIONS); the
 * bulk values are then unused.  non_conductive[r] != 0 excludes region r
 * from the simulation, a conduction block such as a scar (Sec. 1.1.2): its
 * elements contribute to neither M nor K, and a node all of whose elements
 * are excluded is inactive -- ionic model off, states held, no applied
 * current, its potential kept.  Fluxes across interfaces between conductive
 * regions are continuous (the Galerkin form with piecewise D).  Regions need
 * the stencil FP32 operator in the refined path (EP_OP_MATRIX_FREE gets
 * EP_EUNSUPPORTED; EP_OP_AUTO picks the stencil). */
#define EP_MAX_REGIONS 8
typedef struct {
    double sigma_l, sigma_t, sigma_n;
    double chi_m, Cm;
    int32_t is_D;
    int32_t n_regions;
    double region_sigma[EP_MAX_REGIONS][3];
    uint8_t non_conductive[EP_MAX_REGIONS];
} ep_conductivities;

/* Ionic model (Sec. 1.1.1): Bueno-Orovio minimal model (epicardial
 * parameters) or ten Tusscher-Panfilov 2006.  cell_type is per node
 * (EP_CELL_*), used by TTP06 only; NULL means all epicardial.  Initial state:
 * BO rest (u = 0, v = w = 1, s = 0); TTP06 the epicardial values printed for
 * the N-version benchmark (Sec. 3.2.1) for every cell type. */
typedef struct {
    int32_t model;
    const uint8_t* cell_type;
    /* Optional initial u and states per cell type (ENDO, MID, EPI), 3 rows
     * of 1 + S doubles (u first, then the states in the checkpoint's order;
     * S = 3 BO, 18 TTP06), e.g. from ep_prepace; NULL: the defaults above. */
    const double* initial;
} ep_ionic_model;

/* Single-cell pre-pacing (the paper initialises its ionic models from 0D
 * simulations of many beats at the pacing period, Sec. 3.2).  For each of
 * n_cells cells (cell_types[i] = EP_CELL_*; the type matters for TTP06
 * only), integrates Eq. (1) without diffusion with the semi-implicit step of
 * Eq. (4) that the tissue step uses (BDF of bdf_order, a BDF1 first step),
 * time step dt, under a train of pulses of amp (model units per ms) lasting
 * dur_ms every period_ms from t = 0, for beats beats; writes u and the
 * states at the end (start of the next beat) to out, n_cells rows of 1 + S
 * doubles.  initial: NULL (the model's defaults) or n_cells rows of 1 + S.
 * Runs on the GPU in FP64, one thread per cell, a launch per beat. */
ep_status ep_prepace(int32_t model, const uint8_t* cell_types, int32_t n_cells, double period_ms,
                     int32_t beats, double dt, double amp, double dur_ms, int32_t bdf_order,
                     const double* initial, double* out);

/* Applied current I_app (Sec. 1.1.2): pulse p adds amp (model units per ms:
 * mV/ms for TTP06, 1/ms for BO) at the nodes where mask[node] != 0 -- or,
 * with a spatial profile, amp * weight[node] at every node (the paper's
 * Gaussian impulses, Sec. 3.2: weight = exp(-|x - c|^2 / (2 s^2)); a
 * spherical impulse is a mask) -- on step n+1 when k0 < n+1 <= k0 + kd
 * with k0 = round(t0/dt), kd = round(dur/dt), repeating every
 * round(period/dt) steps when period > 0.  At most EP_MAX_PULSES pulses;
 * each mask has n_nodes bytes, each weight n_nodes finite doubles; a pulse
 * needs a mask or a weight (the weight wins when both are given). */
#define EP_MAX_PULSES 4
typedef struct {
    double amp, t0, dur, period;
    const uint8_t* mask;
    const double* weight;
    /* Optional region of whole elements (n_elems bytes, element numbering of
     * ep_mesh.region; Q1 meshes): I_app = amp on the elements where
     * elem[e] != 0 and 0 elsewhere, entering Eq. (6) as the applied-current
     * vector integrated by the 2x2x2 Gauss rule, f_j = amp * sum over those
     * elements of int_e phi_j -- the quadrature evaluation of a current given
     * as a function of space, such as the paper's cubic impulse (Sec. 3.2.1)
     * -- instead of the nodal values times the mass matrix; mask and weight
     * are then ignored.  NULL: the nodal pulse above. */
    const uint8_t* elem;
} ep_pulse;

typedef struct {
    int32_t n_pulses;
    const ep_pulse* pulses;
} ep_stimulus;

/* Solver options.  dt > 0 (ms); bdf_order 1, 2 or 3 (the BDF order of Sec.
 * 1.2; the first steps ramp up, order min(bdf_order, n + 1) at step n, so
 * order 3 takes a BDF1 then a BDF2 step); tol: relative FP64 residual ||b - A u||_2 <= tol ||b||_2 (0 ->
 * 1e-12 for FP64, 1e-10 for FP32_REFINED); max_iter: CG iterations (FP64) or
 * inner iterations per refinement sweep (0 -> 1000 / 200); inner_tol: the
 * FP32 inner solve of a sweep stops once its residual is below 0.9 tol ||b||
 * (enough for that sweep to end the refinement) or below inner_tol times its
 * initial residual, whichever comes first (0 -> 1e-6, about the float
 * limit, on slabs; 1e-7 on shells, where the first sweep then ends the
 * refinement more often); max_sweeps: refinement sweeps
 * (0 -> 8); op32: FP32 inner operator; cuda_stream: a cudaStream_t to order
 * the instance's work on, or NULL for a stream the library creates;
 * ionic_threads: threads per block of the ionic kernel, 64, 128 or 256, or 0
 * for the create-time autotuner's choice (the block size changes nothing in
 * the results: one node per thread, no reductions); solve_tiles: the
 * persistent solve's operator apply (stencil operator, Q1 meshes) on tiles
 * of rows staged in shared memory by bulk copies (2), or node-parallel (0 or
 * 1, the default: measured faster on the 2.19M-node LV shell); 2 on a Q2
 * mesh, in FP64 or with the matrix-free operator is EP_EUNSUPPORTED.  The
 * apply's rows are the same sums either way; the dot products group their
 * partial sums by tile, so results differ in rounding only. */
typedef struct {
    double dt;
    int32_t bdf_order;
    int32_t precision;
    double tol;
    int32_t max_iter;
    double inner_tol;
    int32_t max_sweeps;
    int32_t op32;
    void* cuda_stream;
    int32_t ionic_threads;
    int32_t solve_tiles;
} ep_options;

/* Per-step counters of the last completed step. */
typedef struct {
    int64_t step;           /* time level reached (t = step * dt) */
    int32_t cg_iters;       /* FP64 CG iterations or total FP32 inner iterations */
    int32_t sweeps;         /* refinement sweeps (0 for FP64) */
    double relres;          /* final ||b - A u|| / ||b|| (FP64) */
    int32_t op32;           /* FP32 operator in use (EP_OP_*) */
    int32_t solve_threads;  /* threads per block of the persistent solve (one block
                               per SM; stencil operator), 0 for other operators */
    size_t device_bytes;    /* device memory held by the instance */
    double tune_us_mf;      /* autotuner: matrix-free apply time (us), 0 if not timed */
    double tune_us_stencil; /* autotuner: FP32 stencil apply time (us), 0 if not timed */
    int32_t ionic_threads;  /* threads per block of the ionic kernel in use */
    int32_t solve_tiles;    /* 1: the persistent solve applies the operator on
                               tiles staged in shared memory, 0 otherwise */
} ep_stats;

/* Creates an instance: validates the inputs, copies them to the device,
 * builds the FP64 mass and system stencils (2x2x2 Gauss-Legendre, Eq. (6)),
 * the Jacobi diagonal and, for FP32_REFINED, the FP32 operator data.
 * On success *out owns all device memory of the instance. */
ep_status ep_create(const ep_mesh* mesh, const ep_fibers* fibers,
                    const ep_conductivities* cond, const ep_ionic_model* ionic,
                    const ep_stimulus* stim, const ep_options* opts,
                    ep_instance** out);

/* Advances n_steps >= 0 time steps and waits for them; returns EP_ENAN,
 * EP_ENOCONV or EP_ETIMEOUT when a step failed (the instance then holds the
 * state of the failing step and further steps are refused with the same
 * status). */
ep_status ep_step(ep_instance* inst, int64_t n_steps);
/* Enqueues n_steps steps on the instance's stream without waiting. */
ep_status ep_step_async(ep_instance* inst, int64_t n_steps);
/* Waits for the enqueued steps and returns their status (as ep_step). */
ep_status ep_sync(ep_instance* inst);

/* Advances several instances by n_steps each, all enqueued before any wait;
 * returns the first failing status (inst[k] order).  FP32_REFINED stencil
 * instances share one persistent solve launch, one or more resident thread
 * blocks each: at most one such instance per SM (152 on GB300), EP_EINVAL
 * beyond. */
ep_status ep_step_batch(ep_instance* const* insts, int32_t n, int64_t n_steps);

/* Copies u_n (mV) into out[0..n), n == n_nodes. */
ep_status ep_read_potential(const ep_instance* inst, double* out_mV, int64_t n);
/* Activation times (ms): time of the largest forward difference u_{n+1}-u_n
 * seen so far (first maximum wins; Sec. 3.2.1), NaN where that largest slope
 * never exceeded 1 mV/ms.  n == n_nodes. */
ep_status ep_activation_times(const ep_instance* inst, double* out_ms, int64_t n);

/* Checkpoint.  Layout of the buffer (all little-endian, doubles unaligned
 * after the 64-byte header):
 *   header: char magic[8] = "EPSTATE1"; int32 version (1); int32 model;
 *           int64 n_nodes; int32 n_states; int32 bdf_order; int64 step;
 *           double dt; int64 reserved[2] (reserved[0]: bytes of the
 *           extension below, 0 if none);
 *   double u_n[N], u_{n-1}[N]          (model units)
 *   double w_n[S][N], w_{n-1}[S][N]    (state-major; S = 3 BO, 18 TTP06)
 * with a third level for bdf_order 3: u_n, u_{n-1}, u_{n-2}, then w_n,
 * w_{n-1}, w_{n-2} (L = 3 levels, else L = 2),
 *   double at[N]                       (time of the largest slope, ms)
 *   double best[N]                     (largest u_{n+1} - u_n, model units)
 * FP32_REFINED instances append an extension with their float-float working
 * state, so that a restart continues bit for bit: char tag[8] = "EPFFEXT1";
 * int32 hist (valid A u history levels, 0..L); int32 0; then float arrays
 * of N: u hi, lo of each level (n first); the TTP06 concentrations of each
 * level, [2][5][N] (hi parts, then lo parts; absent for BO); A u hi, lo of
 * each level's step.  The portable part alone is a complete
 * state: any instance of the same model and size loads it (a refined
 * instance then splits the doubles into pairs and rebuilds its history
 * within two steps).  ep_state_bytes gives the size of this instance's
 * buffer.  ep_load_state requires the same model, n_nodes and number of
 * levels and at least the portable part; it also resets the stimulus clock to the loaded step. */
size_t ep_state_bytes(const ep_instance* inst);
ep_status ep_save_state(const ep_instance* inst, void* buf, size_t bytes);
ep_status ep_load_state(ep_instance* inst, const void* buf, size_t bytes);

/* Device bytes an instance of this mesh, model and options would hold;
 * 0 if the arguments are invalid.  With a region label it assumes some
 * region may be non-conductive (an upper bound otherwise). */
size_t ep_footprint_bytes(const ep_mesh* mesh, const ep_ionic_model* ionic,
                          const ep_options* opts);

ep_status ep_get_stats(const ep_instance* inst, ep_stats* out);
/* Device pointer to u_n (double, model units, n_nodes), valid until the
 * next ep_step* call on the instance. */
ep_status ep_potential_device(const ep_instance* inst, const double** out);

/* Per-kernel timing.  While profiling is on, ep_step runs its loops from the
 * host (no CUDA graph) and brackets every kernel launch with a pair of CUDA
 * events on the instance's stream; the totals accumulate until reset.  The
 * step time is then not representative, the kernel times are.  Kernel names:
 * "ionic", "rhs", "resid", "p64", "apply64", "update64", "apply32_mf",
 * "apply32_stencil", "update32", "pcg32" (the persistent inner solve of a
 * refinement sweep), "correct", "finish", "realpha". */
typedef struct {
    char name[24];
    int64_t launches;
    double ms_total;
} ep_kernel_time;
ep_status ep_profile_enable(ep_instance* inst, int32_t on);
/* Writes up to cap entries (kernels launched at least once) and their count
 * to *n; reset != 0 clears the totals afterwards. */
ep_status ep_profile_read(ep_instance* inst, ep_kernel_time* out, int32_t cap,
                          int32_t* n, int32_t reset);

/* Allocation-free residual check.  The paper has no counterpart: this is a
 * service of the library.  Writes to *relres_out the relative residual
 * ||b - A u||_2 / ||b||_2 of an FP32_REFINED instance's last linear solve
 * (the value ep_get_stats reports as relres), recomputed from the instance's
 * operator, right-hand side and the solver's float-float iterate u (whose sum
 * rounded to double is the potential u_n) in the same arithmetic and
 * summation order as the solver's residual when the instance steps alone
 * (ep_step_batch spreads an instance over other blocks, so its reported
 * relres may differ from this one in the float summation, ~1e-7 relative).
 * Errors: EP_EUNSUPPORTED for instances other than refined ones with the
 * stencil FP32 operator; EP_EINVAL when no step has run since ep_create or
 * the last ep_load_state (a loaded potential has no solve of its own), or
 * when the last solve's right-hand side is zero (no relative residual).
 *
 * Who it is for: callers that cannot call cudaMalloc where they check a
 * solve -- for example a host application whose device memory is owned by
 * another allocator (a framework's caching allocator, or a pool that
 * reserves the GPU's memory at start-up), where an allocation by this
 * library would fail or break the owner's accounting.  This call allocates
 * nothing: it calls no cudaMalloc, cudaFree or other allocating routine.
 * Its scratch is a fixed ~16 KiB device array in the library (every GPU that
 * loads the library holds it until the process exits), holding one pair of
 * partial sums per thread block, at most 1024 blocks; an instance whose
 * residual kernel would need more blocks is refused with EP_EINVAL.  The
 * first call on each device looks up that array's device address (done
 * once per device, with that device current).  All calls share the array
 * and it keeps the last call's contents; each call clears what must start
 * at zero.  Calls whose GPU work overlaps (unordered streams) race on it;
 * calls ordered on one stream do not.  Runs on the instance's stream and
 * waits for it. */
ep_status ep_residual_norm_noalloc(const ep_instance* inst, double* relres_out);

/* Self-test of the persistent solver's bounded waits (no instance needed):
 * one thread block waits at the solver's grid barrier for a second block
 * that never comes; the wait gives up after a bounded number of naps (a few
 * milliseconds here, about a second in the solver) and records the status
 * the solver would record, written to *status_out (EP_ETIMEOUT).  Nothing
 * faults and the CUDA context stays usable.  Synchronises the device. */
ep_status ep_selftest_barrier_timeout(int32_t* status_out);

/* Frees every resource of the instance (NULL is accepted). */
ep_status ep_destroy(ep_instance* inst);

/* Message of the last failing call on this host thread ("" if none). */
const char* ep_last_error(void);

#ifdef __cplusplus
}
#endif
#endif
