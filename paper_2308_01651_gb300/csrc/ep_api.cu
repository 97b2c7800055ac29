// ep_api.cu -- host side of the C ABI declared in include/ep.h.
//
// An instance owns its device memory and one CUDA graph holding a whole time
// step: the fused ionic kernel, the FP64 right-hand side, the linear solve
// with its loops as conditional WHILE nodes (loop control stays on the
// device), and the activation/rotation kernel.  ep_step replays the graph.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <mutex>
#include <new>
#include <string>
#include <vector>

#include <cuda.h>

#include "ep_dev.cuh"
#include "ionic_models.cuh"
#include "ep_tile.cuh"

namespace epk {
void launch_ionic(Dev* d, const Dev& h, int grid, int threads, cudaStream_t s);
void launch_assemble(Dev* d, const Dev& h, const AsmParams& P, cudaStream_t s);
void launch_realpha(Dev* d, const Dev& h, double delta, double alpha_dt, float cmass, cudaStream_t s);
void launch_rhs64(Dev* d, const Dev& h, int first, int graph, int grid, cudaStream_t s);
void launch_rhs_ff(Dev* d, const Dev& h, int graph, int grid, cudaStream_t s);
void launch_expand(Dev* d, const Dev& h, int want_a, int want_m, cudaStream_t s);
void launch_realpha_ff(Dev* d, const Dev& h, double delta, double alpha_dt, float cmass, cudaStream_t s);
void launch_p64(Dev* d, const Dev& h, int grid, cudaStream_t s);
void launch_apply64(Dev* d, const Dev& h, int grid, cudaStream_t s);
void launch_update64(Dev* d, const Dev& h, int grid, int graph, cudaStream_t s);
void launch_apply32_stencil(Dev* d, const Dev& h, int grid, cudaStream_t s);
void launch_apply32_mf(Dev* d, const Dev& h, cudaStream_t s);
void launch_update32(Dev* d, const Dev& h, int grid, int graph, cudaStream_t s);
void launch_correct_ff(Dev* d, const Dev& h, int grid, cudaStream_t s);
void launch_ionic_batch(const Batch& B, int model, bool lv3, int grid, cudaStream_t s);
void launch_q2_apply32(Dev* d, const Dev& h, int grid_nodes, cudaStream_t s);
void launch_q2_resid(Dev* d, const Dev& h, int first, int graph, int grid_nodes, cudaStream_t s);
void launch_realpha_q2(Dev* d, const Dev& h, double alpha_dt, cudaStream_t s);
void launch_rhs_ff_batch(const Batch& B, int graph, int grid, bool curved, cudaStream_t s);
void launch_resid_np(Dev* d, const Dev& h, int graph, int grid, cudaStream_t s);
cudaError_t launch_pcg32_batch(const Batch& B, int grid, int hint, cudaStream_t s);
cudaError_t launch_prepace(int model, const uint8_t* cells, int ncell, double dt, long long m0, long long nsteps,
                           long long kp, long long kd, double amp, int bdf, double* st, cudaStream_t s);
void launch_finish(Dev* d, const Dev& h, int grid, cudaStream_t s);
int mf_tiles(const Dev& h);
cudaError_t mf_prepare();
bool mfc_supported(int NX);
size_t mfc_geo_floats(int NX, int NY, int NZ);
void mfc_fill_geo(float* g, int NX, int NY, int NZ, const double* xyz, const double* f0, const double* s0);
cudaError_t mfc_tensor_map(CUtensorMap* tm, const float* g, int NX, int NY, int NZ);
cudaError_t mfc_prepare(int NX);
void launch_apply32_mfc(Dev* d, const Dev& h, const CUtensorMap& tm, cudaStream_t s);
int pcg_blocks_per_sm();
cudaError_t launch_pcg32(Dev* d, const Dev& h, int grid, int tiled, int hint, cudaStream_t s);
int pcg_threads_of();
size_t tiled_smem_max();
cudaError_t pcg_tiled_prepare(size_t smem, int* fits);
size_t tiled_smem_bytes(int l, int NX);
bool plan_tiles(int NX, int NY, int NZ, int sms, size_t smem_max, int* by, int* jt, int* kr, int* l,
                double* cost);
cudaError_t barrier_timeout_probe(int* status_out);
cudaError_t residual_norm_noalloc(Dev* d, int grid, int threads, cudaStream_t s, double sums[2]);
int noalloc_max_blocks();
}  // namespace epk

using epk::Dev;

static thread_local std::string g_err;

static ep_status fail(ep_status s, const std::string& msg) {
    g_err = msg;
    return s;
}

#define CUDA_TRY(call)                                                                      \
    do {                                                                                    \
        cudaError_t e_ = (call);                                                            \
        if (e_ != cudaSuccess)                                                              \
            return fail(e_ == cudaErrorMemoryAllocation ? EP_ENOMEM : EP_ECUDA,             \
                        std::string(#call) + ": " + cudaGetErrorString(e_));                \
    } while (0)

struct ep_instance {
    Dev h{};                   // host mirror of the device descriptor
    Dev* d = nullptr;          // device descriptor
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    std::vector<void*> allocs;
    std::vector<void*> temps;  // create-time temporaries, stream-ordered (dalloc_temp)
    size_t bytes = 0;
    long long host_step = 0;   // step index of the next enqueued step
    // a linear solve ran since ep_create or the last ep_load_state, so b, the
    // operator and the iterate describe one solve (the allocation-free
    // residual check needs that)
    bool solved = false;
    // refined path: a step ran whose per-node end (k_finish_ff's work) waits
    // for the next step's ionic kernel; reads of the state do it first
    mutable bool fin_pending = false;
    double alpha_dt_dev = 0;   // alpha/dt the device operators hold
    int grid_nodes = 0;        // grid of the grid-stride node kernels (with reductions)
    int grid_ionic = 0;        // one node per thread
    int ionic_threads = epk::kIonicThreads;  // its block size (autotuned at create)
    int grid_resid = 0;        // node-parallel residual / rhs: 512-thread blocks, two per SM (one on curved meshes)
    int grid_tiles = 0;        // persistent grid of the tiled stencil kernels
    int grid_pcg = 0;          // cooperative grid of the persistent inner solver
    int pcg_tiled = 0;         // its apply pass on tiles staged in shared memory (k_pcg.cu)
    int pcg_hint = 0;          // its working set exceeds L2: L2 eviction-priority hints
    ep_status sticky = EP_OK;
    int* bad = nullptr;        // device flag of the assembly
    bool graph_mode = true;    // false: host-driven loops (EP_GRAPH=0), for debugging
    float tune_ms[3] = {0.f, 0.f, 0.f};  // autotuned FP32 operator apply times (ms)
    // matrix-free FP32 operator of curved (shell) meshes: the staged
    // geometry array and its TMA tensor map
    float* mfc_geo = nullptr;
    CUtensorMap mfc_tm;
    // per-kernel event timing (ep_profile_enable)
    bool profiling = false;
    struct Pending { int id; cudaEvent_t a, b; };
    std::vector<Pending> pending;
    std::vector<cudaEvent_t> free_events;
    double prof_ms[16] = {0};
    long long prof_n[16] = {0};
};

static const char* kKernelNames[] = {"ionic", "rhs", "resid", "p64", "apply64", "update64",
                                     "apply32_mf", "apply32_stencil", "update32", "correct",
                                     "finish", "realpha", "solve32", "apply32_q2"};
enum { K_IONIC, K_RHS, K_RESID, K_P64, K_APPLY64, K_UPDATE64, K_APPLY32MF, K_APPLY32ST, K_UPDATE32,
       K_CORRECT, K_FINISH, K_REALPHA, K_PCG32, K_APPLY32Q2, K_COUNT };

static cudaEvent_t prof_event(ep_instance* I) {
    if (!I->free_events.empty()) {
        cudaEvent_t e = I->free_events.back();
        I->free_events.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    cudaEventCreate(&e);
    return e;
}

// Launches f() bracketed by events when profiling.
template <class F>
static void timed(ep_instance* I, int id, F f) {
    if (!I->profiling) {
        f();
        return;
    }
    ep_instance::Pending p{id, prof_event(I), prof_event(I)};
    cudaEventRecord(p.a, I->stream);
    f();
    cudaEventRecord(p.b, I->stream);
    I->pending.push_back(p);
}

// Folds completed event pairs into the totals (call after a stream sync).
static void prof_resolve(ep_instance* I) {
    for (auto& p : I->pending) {
        float ms = 0.f;
        if (cudaEventElapsedTime(&ms, p.a, p.b) == cudaSuccess) {
            I->prof_ms[p.id] += ms;
            I->prof_n[p.id] += 1;
        }
        I->free_events.push_back(p.a);
        I->free_events.push_back(p.b);
    }
    I->pending.clear();
}

namespace {

constexpr double kBOmV = 85.7, kBOoff = -84.0;

bool finite_pos(double x) { return std::isfinite(x) && x > 0.0; }

int64_t expected_nodes(const ep_mesh* m) {
    if (m->kind == EP_MESH_SLAB) return (int64_t)(m->nx + 1) * (m->ny + 1) * (m->nz + 1);
    if (m->kind == EP_MESH_SLAB_Q2) return (int64_t)(2 * m->nx + 1) * (2 * m->ny + 1) * (2 * m->nz + 1);
    return (int64_t)(m->nx + 1) * m->ny * (m->nz + 1);
}

template <class T>
ep_status dalloc(ep_instance* I, T** p, size_t count) {
    void* v = nullptr;
    const size_t b = ((count * sizeof(T) + 255) / 256) * 256;
    cudaError_t e = cudaMalloc(&v, b > 0 ? b : 256);
    if (e != cudaSuccess) {
        (void)cudaGetLastError();
        return fail(EP_ENOMEM, "cudaMalloc of " + std::to_string(b) + " bytes failed: " + cudaGetErrorString(e));
    }
    I->allocs.push_back(v);
    I->bytes += b;
    *p = static_cast<T*>(v);
    return EP_OK;
}

// A float vector of N nodes with `pad` zero floats before and after it
// (*p points at node 0): node-parallel kernels may then read the neighbours
// of every node of a Q1 slab at fixed offsets, without boundary flags: a
// read past the slab's edge lands in the zero padding (never written) or on
// another node, and meets a zero coupling either way.
ep_status dalloc_padded(ep_instance* I, float** p, size_t N, int64_t pad) {
    float* raw = nullptr;
    const ep_status st = dalloc(I, &raw, N + 2 * (size_t)pad);
    if (st != EP_OK) return st;
    if (cudaMemsetAsync(raw, 0, (N + 2 * (size_t)pad) * sizeof(float), I->stream) != cudaSuccess) {
        (void)cudaGetLastError();
        return fail(EP_ECUDA, "cudaMemsetAsync of a padded vector failed");
    }
    *p = raw + pad;
    return EP_OK;
}

// A zeroed device array of count floats.
ep_status dalloc_zero(ep_instance* I, float** p, size_t count) {
    const ep_status st = dalloc(I, p, count);
    if (st != EP_OK) return st;
    if (cudaMemsetAsync(*p, 0, count * sizeof(float), I->stream) != cudaSuccess) {
        (void)cudaGetLastError();
        return fail(EP_ECUDA, "cudaMemsetAsync of a coupling array failed");
    }
    return EP_OK;
}

// Create-time temporaries (the assembly's inputs, the FP64 stencils that
// the refined path drops after the float-float split) are stream-ordered
// allocations on the instance's stream: a cudaFree waits for all work on the
// device, so while other instances step (a server creating one as the
// others run) every free would wait for their batch in flight.
template <class T>
ep_status dalloc_temp(ep_instance* I, T** p, size_t count) {
    void* v = nullptr;
    const size_t b = ((count * sizeof(T) + 255) / 256) * 256;
    cudaError_t e = cudaMallocAsync(&v, b > 0 ? b : 256, I->stream);
    if (e != cudaSuccess) {
        (void)cudaGetLastError();
        return fail(EP_ENOMEM, "cudaMallocAsync of " + std::to_string(b) + " bytes failed: " + cudaGetErrorString(e));
    }
    I->temps.push_back(v);
    *p = static_cast<T*>(v);
    return EP_OK;
}

template <class T>
void dfree_temp(ep_instance* I, T*& p) {
    if (!p) return;
    for (size_t i = 0; i < I->temps.size(); ++i)
        if (I->temps[i] == (void*)p) {
            I->temps.erase(I->temps.begin() + i);
            cudaFreeAsync((void*)p, I->stream);
            break;
        }
    p = nullptr;
}

// Frees one allocation of dalloc before ep_destroy.
template <typename T>
void dfree(ep_instance* I, T*& p, size_t count) {
    if (!p) return;
    for (size_t i = 0; i < I->allocs.size(); ++i)
        if (I->allocs[i] == (void*)p) {
            I->allocs.erase(I->allocs.begin() + i);
            I->bytes -= ((count * sizeof(T) + 255) / 256) * 256;
            cudaFree((void*)p);
            break;
        }
    p = nullptr;
}

struct Sizes {
    int N, ns, ng32, ns64, prec, op32;
    bool slab;
    bool shell;
    bool regions;     // the mesh carries subdomain labels
    bool slab_mass;   // the refined path applies the analytic slab mass matrix
    int levels;       // time levels kept: 3 for BDF3, else 2
    bool q2;          // triquadratic slab
    int64_t ne;       // elements (Q2)
    int64_t npad;     // zero nodes before and after the inner solver's u (Q1 meshes)
    int64_t cpad;     // zero floats before and after the float coupling arrays
    int64_t cs;       // slot stride of the refined couplings (floats): N, then zeros
    int NX, NY, NZ;   // nodes per direction (Q1)
};

// Packed refined state (ep_dev.cuh): slot of state k (checkpoint order) --
// part 0 its float or hi part, part 1 the lo part of a TTP06 concentration --
// and the address of slot s of node n in a [G][N] float4 array.
int state_slot(int model, int k, int part) {
    if (model == EP_MODEL_BO || k < epk::kTTGates) return k;
    return part == 0 ? k : k + epk::kTTConc;
}

float* packed_at(float* base, size_t N, int slot, size_t n) {
    return base + ((size_t)(slot / 4) * N + n) * 4 + slot % 4;
}

// slot s of every node of a device packed array to or from a host array of N
cudaError_t get_slot(const float* dev, size_t N, int slot, float* host) {
    return cudaMemcpy2D(host, sizeof(float), packed_at(const_cast<float*>(dev), N, slot, 0), 4 * sizeof(float),
                        sizeof(float), N, cudaMemcpyDeviceToHost);
}

cudaError_t put_slot(float* dev, size_t N, int slot, const float* host) {
    return cudaMemcpy2D(packed_at(dev, N, slot, 0), 4 * sizeof(float), host, sizeof(float), sizeof(float), N,
                        cudaMemcpyHostToDevice);
}

// float-float pair (nearest float, then the nearest float of the rest)
void split_ff(double x, float& hi, float& lo) {
    hi = (float)x;
    lo = (float)(x - (double)hi);
}

// Largest slope per node (activation detection): double in the FP64 path,
// float in the refined one.
cudaError_t get_best(const ep_instance* I, double* out) {
    const size_t N = (size_t)I->h.N;
    if (I->h.bestf) {
        std::vector<float> f(N);
        cudaError_t e = cudaMemcpy(f.data(), I->h.bestf, N * 4, cudaMemcpyDeviceToHost);
        for (size_t n = 0; n < N; ++n) out[n] = f[n];
        return e;
    }
    return cudaMemcpy(out, I->h.best, N * 8, cudaMemcpyDeviceToHost);
}

// Internal operator kind of triquadratic slabs (not an ep_options.op32 value):
// the matrix-free Q2 operators of k_q2.cu.
constexpr int kOpQ2 = 100;

// Device bytes per instance; mirrors the allocations in ep_create.
size_t footprint(const Sizes& z) {
    auto al = [](size_t b) { return ((b + 255) / 256) * 256; };
    const size_t N = (size_t)z.N;
    size_t b = 0;
    const size_t L = (size_t)z.levels;
    b += (L + 1) * al(N * 8);             // u_n, u_nm1 (, u_nm2), u_new
    b += L * al(z.ng32 * N * 4);          // packed states (refined)
    b += L * al(z.ns64 * N * 8);          // FP64 states
    b += al(N);                           // cell types
    if (z.regions) b += al(N);            // active-node flags
    if (z.prec != EP_PREC_FP32_REFINED) b += 3 * al(N * 8);  // v, b, r
    b += 2 * al(N * 8);                   // at, best
    if (z.prec != EP_PREC_FP32_REFINED) {
        b += 2 * al(epk::kSlots * N * 8);  // M64, A64 (the refined path frees them after ep_create)
        b += al(N * 8);                    // dinv64
    }
    if (z.prec == EP_PREC_FP32_REFINED) {
        b += al(N * 4);                   // dinv32
        if (z.q2) {
            const size_t eq = (size_t)z.ne * 27;
            b += al(12 * eq * 4);         // quadrature-point flux matrices (hi, lo)
            b += al(6 * eq * 4);          // their hi parts, element fastest (FP32 apply)
            b += al(8 * N * 4);           // FP32 apply's element outputs in node slots
            b += 4 * al(8 * N * 4);       // element outputs of A u and M v (hi, lo) in node slots
            b += 2 * al(N * 8);           // diagonals of M and K
        } else {
            const size_t cb = ((size_t)epk::kSlots * (size_t)z.cs + 2 * (size_t)z.cpad) * 4;
            b += 2 * al(cb);                         // Ahi Alo (symmetric float-float stencil)
            if (!z.slab_mass) b += 2 * al(cb);       // Mhi Mlo (curved / with regions)
        }
        b += 6 * al(N * 4);                                              // u, v, b (hi, lo)
        b += (2 + 2 * L) * al(N * 4);                                    // A u history (hi, lo)
        b += (1 + 2 * L) * al(N * 4);                                    // u levels (hi, lo), best slope
        if (z.op32 != EP_OP_STENCIL && z.slab) b += al(6 * N * 4);      // fibres (slab matrix-free)
        if (z.op32 != EP_OP_STENCIL && z.shell)                          // staged geometry (shell matrix-free)
            b += al(epk::mfc_geo_floats(z.NX, z.NY, z.NZ) * 4);
        b += 5 * al(N * 4) + al((N + 2 * (size_t)z.npad) * 4);  // r32 q32 d32 pa32 pb32, z32 (padded)
        if (!z.q2) b += al(N);            // boundary flags
    } else {
        b += 4 * al(N * 8);               // z64 q64 pa64 pb64
    }
    const size_t blocks = std::max((N + 255) / 256 + 1, (size_t)epk::kMaxPersistentBlocks);
    b += al(blocks * 8 * 8);              // partials
    b += al(epk::CNT_N * 4);
    b += al(sizeof(Dev)) + 256;
    return b;
}

ep_status validate(const ep_mesh* mesh, const ep_fibers* fib, const ep_conductivities* cond,
                   const ep_ionic_model* ionic, const ep_stimulus* stim, const ep_options* opts) {
    if (!mesh || !fib || !cond || !ionic || !opts) return fail(EP_EINVAL, "NULL argument");
    if (mesh->kind != EP_MESH_SLAB && mesh->kind != EP_MESH_SHELL && mesh->kind != EP_MESH_SLAB_Q2)
        return fail(EP_EINVAL, "mesh.kind");
    if (mesh->nx < 1 || mesh->ny < 1 || mesh->nz < 1) return fail(EP_EINVAL, "mesh sizes must be >= 1");
    if (mesh->kind == EP_MESH_SHELL && mesh->ny < 3) return fail(EP_EINVAL, "shell needs ny >= 3");
    const int64_t nn = expected_nodes(mesh);
    if (nn > (int64_t)1 << 30) return fail(EP_EINVAL, "mesh too large for one instance (> 2^30 nodes)");
    if (mesh->n_nodes != nn) return fail(EP_EINVAL, "mesh.n_nodes does not match the structured sizes");
    if (mesh->kind == EP_MESH_SLAB || mesh->kind == EP_MESH_SLAB_Q2) {
        for (int d = 0; d < 3; ++d)
            if (!finite_pos(mesh->L[d])) return fail(EP_EINVAL, "slab lengths must be positive");
    } else if (!mesh->xyz) {
        return fail(EP_EINVAL, "shell needs xyz");
    }
    if (!fib->f0 || !fib->s0) return fail(EP_EINVAL, "fibers.f0/s0 must be given");
    if (!mesh->region &&
        (!finite_pos(cond->sigma_l) || !finite_pos(cond->sigma_t) || !finite_pos(cond->sigma_n)))
        return fail(EP_EINVAL, "conductivities must be positive and finite");
    if (!cond->is_D && (!finite_pos(cond->chi_m) || !finite_pos(cond->Cm)))
        return fail(EP_EINVAL, "chi_m and Cm must be positive and finite");
    if (ionic->model != EP_MODEL_BO && ionic->model != EP_MODEL_TTP06) return fail(EP_EINVAL, "ionic.model");
    if (ionic->cell_type)
        for (int64_t i = 0; i < nn; ++i)
            if (ionic->cell_type[i] > EP_CELL_EPI) return fail(EP_EINVAL, "cell_type out of range");
    if (ionic->initial) {
        const int S1 = 1 + (ionic->model == EP_MODEL_BO ? epk::kBOStates : epk::kTTGates + epk::kTTConc);
        for (int k = 0; k < 3 * S1; ++k)
            if (!std::isfinite(ionic->initial[k])) return fail(EP_EINVAL, "ionic.initial must be finite");
    }
    if (stim) {
        if (stim->n_pulses < 0 || stim->n_pulses > EP_MAX_PULSES)
            return fail(EP_EINVAL, "stimulus.n_pulses must be in 0..4");
        if (stim->n_pulses > 0 && !stim->pulses) return fail(EP_EINVAL, "stimulus.pulses is NULL");
        for (int p = 0; p < stim->n_pulses; ++p) {
            const ep_pulse& P = stim->pulses[p];
            if (!P.mask && !P.weight && !P.elem)
                return fail(EP_EINVAL, "a pulse needs a mask, a weight or an element region");
            if (P.elem && mesh->kind == EP_MESH_SLAB_Q2)
                return fail(EP_EUNSUPPORTED, "pulses on element regions take Q1 meshes");
            if (P.weight)
                for (int64_t i = 0; i < nn; ++i)
                    if (!std::isfinite(P.weight[i])) return fail(EP_EINVAL, "pulse weights must be finite");
            if (!std::isfinite(P.amp) || !std::isfinite(P.t0) || !(P.dur >= 0) || !std::isfinite(P.period))
                return fail(EP_EINVAL, "pulse parameters must be finite, dur >= 0");
        }
    }
    if (!finite_pos(opts->dt)) return fail(EP_EINVAL, "options.dt must be positive");
    if (opts->bdf_order < 1 || opts->bdf_order > 3) return fail(EP_EINVAL, "options.bdf_order must be 1, 2 or 3");
    if (opts->precision != EP_PREC_FP64 && opts->precision != EP_PREC_FP32_REFINED)
        return fail(EP_EINVAL, "options.precision");
    if (opts->op32 < EP_OP_AUTO || opts->op32 > EP_OP_STENCIL) return fail(EP_EINVAL, "options.op32");
    if (opts->ionic_threads != 0 && opts->ionic_threads != 64 && opts->ionic_threads != 128 &&
        opts->ionic_threads != 256)
        return fail(EP_EINVAL, "options.ionic_threads must be 0, 64, 128 or 256");
    if (opts->solve_tiles < 0 || opts->solve_tiles > 2) return fail(EP_EINVAL, "options.solve_tiles must be 0, 1 or 2");
    if (opts->solve_tiles == 2 && (mesh->kind == EP_MESH_SLAB_Q2 || opts->precision != EP_PREC_FP32_REFINED ||
                                   opts->op32 == EP_OP_MATRIX_FREE))
        return fail(EP_EUNSUPPORTED, "the tiled solve takes FP32_REFINED Q1 meshes with the stencil operator");
    if (opts->op32 == EP_OP_MATRIX_FREE && mesh->kind == EP_MESH_SHELL && !epk::mfc_supported(mesh->nx + 1))
        return fail(EP_EUNSUPPORTED, "the matrix-free FP32 operator takes shells at most 31 elements across the wall");
    if (mesh->kind == EP_MESH_SLAB_Q2) {
        if (opts->precision != EP_PREC_FP32_REFINED)
            return fail(EP_EUNSUPPORTED, "Q2 meshes need FP32_REFINED precision");
        if (mesh->region) return fail(EP_EUNSUPPORTED, "Q2 meshes take one region");
    }
    if (mesh->region) {
        if (opts->op32 == EP_OP_MATRIX_FREE && opts->precision == EP_PREC_FP32_REFINED)
            return fail(EP_EUNSUPPORTED, "the matrix-free FP32 operator does not take subdomains");
        if (cond->n_regions < 1 || cond->n_regions > EP_MAX_REGIONS)
            return fail(EP_EINVAL, "conductivities.n_regions must be in 1..8 with a region label");
        for (int r = 0; r < cond->n_regions; ++r)
            if (!cond->non_conductive[r])
                for (int c = 0; c < 3; ++c)
                    if (!finite_pos(cond->region_sigma[r][c]))
                        return fail(EP_EINVAL, "region conductivities must be positive and finite");
        const int64_t ne = (int64_t)mesh->nx * mesh->ny * mesh->nz;
        for (int64_t e = 0; e < ne; ++e)
            if (mesh->region[e] >= cond->n_regions) return fail(EP_EINVAL, "region label out of range");
    }
    if (opts->tol < 0 || opts->inner_tol < 0 || opts->max_iter < 0 || opts->max_sweeps < 0)
        return fail(EP_EINVAL, "negative solver option");
    return EP_OK;
}

// The applied-current vector of a unit current on a region of Q1 elements,
// g_j = sum over the region's elements of int_e phi_j (Eq. (6), the vector
// arising from I_app), by the 2x2x2 Gauss rule on each element's trilinear
// map: on a box element every corner gets |e| / 8; on a curved one
// sum_q (1/8) det J(q) phi_a(q).  In double, once per instance.
std::vector<double> region_vector(const ep_mesh* mesh, const Dev& h, const uint8_t* elem) {
    std::vector<double> g((size_t)h.N, 0.0);
    const int nx = mesh->nx, ny = mesh->ny, nz = mesh->nz;
    const double gp[2] = {0.5 - 0.5 / std::sqrt(3.0), 0.5 + 0.5 / std::sqrt(3.0)};
    const bool shell = mesh->kind == EP_MESH_SHELL;
    for (int k = 0; k < nz; ++k)
        for (int j = 0; j < ny; ++j)
            for (int i = 0; i < nx; ++i) {
                if (!elem[(size_t)i + (size_t)nx * ((size_t)j + (size_t)ny * k)]) continue;
                size_t node[8];
                double X[8][3];
                for (int a = 0; a < 8; ++a) {
                    const int ii = i + (a & 1), kk = k + (a >> 2);
                    int jj = j + ((a >> 1) & 1);
                    if (shell && jj == h.NY) jj = 0;
                    node[a] = (size_t)ii + (size_t)h.NX * ((size_t)jj + (size_t)h.NY * kk);
                    for (int c = 0; c < 3; ++c) X[a][c] = shell ? mesh->xyz[3 * node[a] + c] : 0.0;
                }
                if (!shell) {
                    const double q = h.h[0] * h.h[1] * h.h[2] / 8.0;
                    for (int a = 0; a < 8; ++a) g[node[a]] += q;
                    continue;
                }
                for (int q = 0; q < 8; ++q) {
                    const double xi[3] = {gp[q & 1], gp[(q >> 1) & 1], gp[q >> 2]};
                    double J[3][3] = {{0, 0, 0}, {0, 0, 0}, {0, 0, 0}}, phi[8];
                    for (int a = 0; a < 8; ++a) {
                        const int b0 = a & 1, b1 = (a >> 1) & 1, b2 = a >> 2;
                        const double l0 = b0 ? xi[0] : 1.0 - xi[0], l1 = b1 ? xi[1] : 1.0 - xi[1],
                                     l2 = b2 ? xi[2] : 1.0 - xi[2];
                        const double d0 = (b0 ? 1.0 : -1.0) * l1 * l2, d1 = l0 * (b1 ? 1.0 : -1.0) * l2,
                                     d2 = l0 * l1 * (b2 ? 1.0 : -1.0);
                        phi[a] = l0 * l1 * l2;
                        for (int c = 0; c < 3; ++c) {
                            J[c][0] += X[a][c] * d0;
                            J[c][1] += X[a][c] * d1;
                            J[c][2] += X[a][c] * d2;
                        }
                    }
                    const double det = J[0][0] * (J[1][1] * J[2][2] - J[1][2] * J[2][1]) -
                                       J[0][1] * (J[1][0] * J[2][2] - J[1][2] * J[2][0]) +
                                       J[0][2] * (J[1][0] * J[2][1] - J[1][1] * J[2][0]);
                    for (int a = 0; a < 8; ++a) g[node[a]] += 0.125 * std::fabs(det) * phi[a];
                }
            }
    return g;
}

Sizes sizes_of(const ep_mesh* mesh, const ep_ionic_model* ionic, const ep_options* opts) {
    Sizes z{};
    z.N = (int)expected_nodes(mesh);
    z.ns = ionic->model == EP_MODEL_BO ? epk::kBOStates : epk::kTTGates + epk::kTTConc;
    z.prec = opts->precision;
    z.levels = opts->bdf_order == 3 ? 3 : 2;
    z.q2 = mesh->kind == EP_MESH_SLAB_Q2;
    z.ne = (int64_t)mesh->nx * mesh->ny * mesh->nz;
    z.slab = mesh->kind == EP_MESH_SLAB;
    // a Q1 slab's neighbour offsets reach 1 + (nx+1) + (nx+1)(ny+1) nodes
    // either way; rounded up to 64 floats, so that the vectors keep the
    // 256-byte alignment of every allocation (16-byte vector accesses)
    // (shells: a row and a few floats, the reach of the tiled solve's bulk
    // copies past the first and last node; the coupling arrays get the same)
    const int64_t reach = ((int64_t)mesh->nx + 1 + 8 + 63) / 64 * 64;
    z.npad = z.slab ? ((int64_t)(mesh->nx + 1) * (mesh->ny + 1) + (mesh->nx + 1) + 1 + 63) / 64 * 64
                    : (mesh->kind == EP_MESH_SHELL ? reach : 0);
    z.cpad = reach;
    {
        // symmetric float couplings: each slot followed by at least the
        // largest backward offset in zeros, rounded up to 64 floats
        const int64_t NX = mesh->nx + 1, NY = mesh->kind == EP_MESH_SHELL ? mesh->ny : mesh->ny + 1;
        const int64_t back = 1 + NX + NX * NY;
        z.cs = ((int64_t)z.N + back + 63) / 64 * 64;
        z.NX = (int)NX;
        z.NY = (int)NY;
        z.NZ = mesh->nz + 1;
    }
    z.regions = mesh->region != nullptr;
    // an excluded region changes M; the footprint assumes it may
    z.slab_mass = z.slab && !z.regions;
    z.shell = mesh->kind == EP_MESH_SHELL;
    {
        // AUTO keeps both FP32 operators where the matrix-free one applies
        // (axis-aligned slabs; shells up to 31 elements across the wall), one
        // region only, and lets the create-time autotuner pick
        const bool mf_ok = !z.regions && (z.slab || (z.shell && epk::mfc_supported(mesh->nx + 1)));
        z.op32 = opts->op32 == EP_OP_AUTO ? (mf_ok ? EP_OP_AUTO : EP_OP_STENCIL) : opts->op32;
    }
    if (z.q2) z.op32 = kOpQ2;
    if (z.prec == EP_PREC_FP32_REFINED) {
        // every state packed, four floats to a 16-byte group (ep_dev.cuh)
        z.ng32 = 4 * (ionic->model == EP_MODEL_BO ? epk::kBOPacked : epk::kTTPacked);
        z.ns64 = 0;
    } else {
        z.ng32 = 0;
        z.ns64 = z.ns;
    }
    return z;
}

// alpha/dt of the BDF order `order` (1, 2, 3)
double alpha_dt_of(const Dev& h, int order) { return (order == 3 ? 11.0 / 6.0 : order == 2 ? 1.5 : 1.0) / h.dt; }

// alpha/dt of the step with index `step`: BDF order min(bdf, step + 1)
double required_alpha_dt(const Dev& h, long long step) {
    return alpha_dt_of(h, h.bdf < step + 1 ? h.bdf : (int)(step + 1));
}

// make sure the device operators hold alpha/dt of the step about to run.
// Raising the order goes through every order in between, as a run from
// step 0 does (1 -> 2 -> 3), so that an instance that loads a checkpoint
// holds bitwise the operator of the run that wrote it.
void ensure_alpha(ep_instance* I) {
    const double need = required_alpha_dt(I->h, I->host_step);
    if (need == I->alpha_dt_dev) return;
    double path[3];
    int np = 0;
    for (int o = 1; o <= 3; ++o) {
        const double a = alpha_dt_of(I->h, o);
        if (a > I->alpha_dt_dev && a <= need) path[np++] = a;
    }
    if (need < I->alpha_dt_dev) path[np++] = need;
    for (int k = 0; k < np; ++k) {
        const double to = path[k];
        const float cmass =
            (float)(I->h.kind == EP_MESH_SHELL ? to : to * I->h.h[0] * I->h.h[1] * I->h.h[2]);
        const double delta = to - I->alpha_dt_dev;
        timed(I, K_REALPHA, [&] {
            if (I->h.q2) epk::launch_realpha_q2(I->d, I->h, to, I->stream);
            else if (I->h.prec == EP_PREC_FP32_REFINED)
                epk::launch_realpha_ff(I->d, I->h, delta, to, cmass, I->stream);
            else epk::launch_realpha(I->d, I->h, delta, to, cmass, I->stream);
        });
        I->alpha_dt_dev = to;
    }
}

// ---- graph construction ------------------------------------------------------

struct Capture {
    cudaStream_t s;
    cudaError_t err = cudaSuccess;
    void chk(cudaError_t e) {
        if (err == cudaSuccess && e != cudaSuccess) err = e;
    }
};

// The matrix-free FP32 apply of the instance's mesh: the slab kernel
// (constant Jacobian) or the curved one (TMA-staged geometry).
void launch_apply32_free(ep_instance* I, cudaStream_t s) {
    if (I->mfc_geo) epk::launch_apply32_mfc(I->d, I->h, I->mfc_tm, s);
    else epk::launch_apply32_mf(I->d, I->h, s);
}

// Adds a WHILE node at the current capture position of stream s, returns its
// handle and body graph, and moves s past the node.
cudaError_t add_while(cudaStream_t s, cudaGraphConditionalHandle* h, cudaGraph_t* body) {
    cudaStreamCaptureStatus st;
    cudaGraph_t g;
    const cudaGraphNode_t* deps = nullptr;
    const cudaGraphEdgeData* edata = nullptr;
    size_t nd = 0;
    cudaError_t e = cudaStreamGetCaptureInfo(s, &st, nullptr, &g, &deps, &edata, &nd);
    if (e != cudaSuccess) return e;
    if (st != cudaStreamCaptureStatusActive) return cudaErrorStreamCaptureInvalidated;
    e = cudaGraphConditionalHandleCreate(h, g, 1, cudaGraphCondAssignDefault);
    if (e != cudaSuccess) return e;
    cudaGraphNodeParams p{};
    p.type = cudaGraphNodeTypeConditional;
    p.conditional.handle = *h;
    p.conditional.type = cudaGraphCondTypeWhile;
    p.conditional.size = 1;
    cudaGraphNode_t node;
    e = cudaGraphAddNode(&node, g, deps, edata, nd, &p);
    if (e != cudaSuccess) return e;
    *body = p.conditional.phGraph_out[0];
    return cudaStreamUpdateCaptureDependencies(s, &node, nullptr, 1, cudaStreamSetCaptureDependencies);
}

ep_status build_graph(ep_instance* I) {
    Dev& h = I->h;
    cudaStream_t s = I->stream;
    cudaStream_t s2 = nullptr, s3 = nullptr;
    CUDA_TRY(cudaStreamCreateWithFlags(&s2, cudaStreamNonBlocking));
    CUDA_TRY(cudaStreamCreateWithFlags(&s3, cudaStreamNonBlocking));
    Capture C{s};
    cudaGraphConditionalHandle h_loop = 0, h_outer = 0, h_inner = 0;
    C.chk(cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal));
    epk::launch_ionic(I->d, h, I->grid_ionic, I->ionic_threads, s);
    if (h.prec == EP_PREC_FP64) epk::launch_rhs64(I->d, h, 1, 1, I->grid_tiles, s);
    else if (h.q2) epk::launch_q2_resid(I->d, h, 1, 1, I->grid_nodes, s);
    else epk::launch_rhs_ff(I->d, h, 1, I->grid_resid, s);
    cudaGraph_t body = nullptr, body2 = nullptr;
    if (h.prec == EP_PREC_FP64) {
        C.chk(add_while(s, &h_loop, &body));
        if (C.err == cudaSuccess) {
            C.chk(cudaStreamBeginCaptureToGraph(s2, body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal));
            epk::launch_p64(I->d, h, I->grid_nodes, s2);
            epk::launch_apply64(I->d, h, I->grid_tiles, s2);
            epk::launch_update64(I->d, h, I->grid_nodes, 1, s2);
            C.chk(cudaStreamEndCapture(s2, &body));
        }
    } else if (h.op32 == EP_OP_STENCIL) {
        // every refinement sweep [inner PCG, u += delta, float-float residual,
        // decision] in one persistent launch (it returns at once when the
        // first residual met the tolerance)
        C.chk(epk::launch_pcg32(I->d, h, I->grid_pcg, I->pcg_tiled, I->pcg_hint, s));
    } else {
        C.chk(add_while(s, &h_outer, &body));
        if (C.err == cudaSuccess) {
            C.chk(cudaStreamBeginCaptureToGraph(s2, body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal));
            C.chk(add_while(s2, &h_inner, &body2));
            if (C.err == cudaSuccess) {
                C.chk(cudaStreamBeginCaptureToGraph(s3, body2, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal));
                if (h.q2) epk::launch_q2_apply32(I->d, h, I->grid_nodes, s3);
                else if (h.op32 == EP_OP_MATRIX_FREE) launch_apply32_free(I, s3);
                else epk::launch_apply32_stencil(I->d, h, I->grid_tiles, s3);
                epk::launch_update32(I->d, h, I->grid_nodes, 1, s3);
                C.chk(cudaStreamEndCapture(s3, &body2));
            }
            epk::launch_correct_ff(I->d, h, I->grid_nodes, s2);
            if (h.q2) epk::launch_q2_resid(I->d, h, 0, 1, I->grid_nodes, s2);
            else epk::launch_resid_np(I->d, h, 1, I->grid_resid, s2);
            C.chk(cudaStreamEndCapture(s2, &body));
        }
    }
    // the refined path's per-node end of the step runs in the next step's
    // ionic kernel (or flush_finish when the host reads the state)
    if (h.prec == EP_PREC_FP64) epk::launch_finish(I->d, h, I->grid_nodes, s);
    cudaGraph_t g = nullptr;
    cudaError_t ee = cudaStreamEndCapture(s, &g);
    C.chk(ee);
    C.chk(cudaGetLastError());
    cudaStreamDestroy(s2);
    cudaStreamDestroy(s3);
    if (C.err != cudaSuccess) {
        if (g) cudaGraphDestroy(g);
        return fail(EP_ECUDA, std::string("building the step graph: ") + cudaGetErrorString(C.err));
    }
    I->graph = g;
    if ((h.prec == EP_PREC_FP64 && !h_loop) ||
        (h.prec != EP_PREC_FP64 && h.op32 != EP_OP_STENCIL && (!h_outer || !h_inner)))
        return fail(EP_ECUDA, "a conditional handle of the step graph is zero");
    CUDA_TRY(cudaGraphInstantiate(&I->exec, g, 0));
    // the conditional handles live in the device descriptor
    h.h_loop = (unsigned long long)h_loop;
    h.h_outer = (unsigned long long)h_outer;
    h.h_inner = (unsigned long long)h_inner;
    CUDA_TRY(cudaMemcpyAsync(&I->d->h_loop, &h.h_loop, 3 * sizeof(unsigned long long),
                             cudaMemcpyHostToDevice, s));
    CUDA_TRY(cudaStreamSynchronize(s));
    return EP_OK;
}

// One step with the loop decisions read back by the host after every
// iteration (no conditional graph nodes).  Bounded by the solver limits.
ep_status step_host(ep_instance* I) {
    const Dev& h = I->h;
    cudaStream_t s = I->stream;
    Dev* d = I->d;
    auto flag = [&](int* p, int* out) -> cudaError_t {
        cudaError_t e = cudaMemcpyAsync(out, p, sizeof(int), cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        return e;
    };
    timed(I, K_IONIC, [&] { epk::launch_ionic(d, h, I->grid_ionic, I->ionic_threads, s); });
    timed(I, K_RHS, [&] {
        if (h.prec == EP_PREC_FP64) epk::launch_rhs64(d, h, 1, 0, I->grid_tiles, s);
        else if (h.q2) epk::launch_q2_resid(d, h, 1, 0, I->grid_nodes, s);
        else epk::launch_rhs_ff(d, h, 0, I->grid_resid, s);
    });
    int f = 0;
    if (h.prec == EP_PREC_FP64) {
        CUDA_TRY(flag(&d->f_loop, &f));
        for (int it = 0; f && it <= h.max_iter; ++it) {
            timed(I, K_P64, [&] { epk::launch_p64(d, h, I->grid_nodes, s); });
            timed(I, K_APPLY64, [&] { epk::launch_apply64(d, h, I->grid_tiles, s); });
            timed(I, K_UPDATE64, [&] { epk::launch_update64(d, h, I->grid_nodes, 0, s); });
            CUDA_TRY(cudaGetLastError());
            CUDA_TRY(flag(&d->f_loop, &f));
        }
    } else {
        CUDA_TRY(flag(&d->f_outer, &f));
        if (h.op32 == EP_OP_STENCIL) {
            // the whole solve in one persistent launch
            cudaError_t pe = cudaSuccess;
            timed(I, K_PCG32, [&] { pe = epk::launch_pcg32(d, h, I->grid_pcg, I->pcg_tiled, I->pcg_hint, s); });
            CUDA_TRY(pe);
            f = 0;
        }
        for (int sw = 0; f && sw <= h.max_sweeps; ++sw) {
            int fi = 1;
            for (int it = 0; fi && it <= h.max_iter; ++it) {
                if (h.q2)
                    timed(I, K_APPLY32Q2, [&] { epk::launch_q2_apply32(d, h, I->grid_nodes, s); });
                else if (h.op32 == EP_OP_MATRIX_FREE)
                    timed(I, K_APPLY32MF, [&] { launch_apply32_free(I, s); });
                else
                    timed(I, K_APPLY32ST, [&] { epk::launch_apply32_stencil(d, h, I->grid_tiles, s); });
                timed(I, K_UPDATE32, [&] { epk::launch_update32(d, h, I->grid_nodes, 0, s); });
                CUDA_TRY(cudaGetLastError());
                CUDA_TRY(flag(&d->f_inner, &fi));
            }
            timed(I, K_CORRECT, [&] { epk::launch_correct_ff(d, h, I->grid_nodes, s); });
            timed(I, K_RESID, [&] {
                if (h.q2) epk::launch_q2_resid(d, h, 0, 0, I->grid_nodes, s);
                else epk::launch_resid_np(d, h, 0, I->grid_resid, s);
            });
            CUDA_TRY(cudaGetLastError());
            CUDA_TRY(flag(&d->f_outer, &f));
        }
    }
    if (h.prec == EP_PREC_FP64) timed(I, K_FINISH, [&] { epk::launch_finish(d, h, I->grid_nodes, s); });
    CUDA_TRY(cudaGetLastError());
    CUDA_TRY(cudaStreamSynchronize(s));
    prof_resolve(I);
    return EP_OK;
}

// Times the FP32 inner operators on this instance (CUDA events on its
// stream, after warm-up) and keeps the faster one for the step graph.
ep_status autotune_op32(ep_instance* I) {
    Dev& h = I->h;
    cudaStream_t s = I->stream;
    const size_t N = (size_t)h.N;
    CUDA_TRY(cudaMemsetAsync(h.z32, 0, N * 4, s));
    CUDA_TRY(cudaMemsetAsync(h.pa32, 0, N * 4, s));
    CUDA_TRY(cudaMemsetAsync(h.pb32, 0, N * 4, s));
    cudaEvent_t a, b;
    CUDA_TRY(cudaEventCreate(&a));
    CUDA_TRY(cudaEventCreate(&b));
    const int cands[2] = {EP_OP_MATRIX_FREE, EP_OP_STENCIL};
    float best_ms = 1e30f;
    int best = EP_OP_STENCIL;
    for (int c : cands) {
        auto launch = [&] {
            if (c == EP_OP_MATRIX_FREE) launch_apply32_free(I, s);
            else epk::launch_apply32_stencil(I->d, h, I->grid_tiles, s);
        };
        for (int w = 0; w < 3; ++w) launch();
        cudaEventRecord(a, s);
        for (int r = 0; r < 10; ++r) launch();
        cudaEventRecord(b, s);
        cudaError_t e = cudaEventSynchronize(b);
        float ms = 0.f;
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, a, b);
        if (e != cudaSuccess) {
            cudaEventDestroy(a);
            cudaEventDestroy(b);
            return fail(EP_ECUDA, std::string("autotune: ") + cudaGetErrorString(e));
        }
        I->tune_ms[c] = ms / 10.f;
        if (ms < best_ms) {
            best_ms = ms;
            best = c;
        }
    }
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    h.op32 = best;
    CUDA_TRY(cudaMemcpy(&I->d->op32, &h.op32, sizeof(int), cudaMemcpyHostToDevice));
    return EP_OK;
}

// Block size of the ionic kernel, per (model, precision, time levels, size
// class): the first instance of a class times 64, 128 and 256 threads per
// block on its own initial state (CUDA events on its stream, after warm-up)
// and the class keeps the fastest.  At step 0 the kernel reads only level n
// (BDF1 step) and writes the new level into an older slot and the step's
// scratch vectors, so the runs change nothing but that slot, which is
// restored from level n afterwards.  The choice changes no result.
static std::mutex g_tune_mu;
static std::vector<std::pair<long long, int>> g_tune_ionic;

ep_status autotune_ionic(ep_instance* I) {
    const Dev& h = I->h;
    int cls = 0;
    while ((2ll << cls) <= (long long)h.N) ++cls;
    const long long key = ((long long)h.model * 4 + h.prec) * 4096 + (long long)(h.u_nm2 ? 3 : 2) * 64 + cls;
    {
        std::lock_guard<std::mutex> lk(g_tune_mu);
        for (auto& kv : g_tune_ionic)
            if (kv.first == key) {
                I->ionic_threads = kv.second;
                I->grid_ionic = (h.N + kv.second - 1) / kv.second;
                return EP_OK;
            }
    }
    cudaStream_t s = I->stream;
    cudaEvent_t a, b;
    CUDA_TRY(cudaEventCreate(&a));
    CUDA_TRY(cudaEventCreate(&b));
    const int cands[3] = {64, 128, 256};
    float best_ms = 1e30f;
    int best = epk::kIonicThreads;
    for (int bt : cands) {
        const int grid = (h.N + bt - 1) / bt;
        for (int w = 0; w < 2; ++w) epk::launch_ionic(I->d, h, grid, bt, s);
        cudaEventRecord(a, s);
        for (int r = 0; r < 5; ++r) epk::launch_ionic(I->d, h, grid, bt, s);
        cudaEventRecord(b, s);
        cudaError_t e = cudaEventSynchronize(b);
        float ms = 0.f;
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, a, b);
        if (e != cudaSuccess) {
            cudaEventDestroy(a);
            cudaEventDestroy(b);
            return fail(EP_ECUDA, std::string("ionic autotune: ") + cudaGetErrorString(e));
        }
        if (ms < best_ms) {
            best_ms = ms;
            best = bt;
        }
    }
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    // the older time levels back to the initial state (level n)
    const size_t N = (size_t)h.N;
    if (h.g32_n) {
        const size_t fb = (size_t)(h.model == EP_MODEL_BO ? epk::kBOPacked : epk::kTTPacked) * 16 * N;
        for (float* d : {h.g32_nm1, h.g32_nm2})
            if (d) CUDA_TRY(cudaMemcpyAsync(d, h.g32_n, fb, cudaMemcpyDeviceToDevice, s));
    }
    if (h.s64_n) {
        const size_t db = (size_t)h.ns * 8 * N;
        for (double* d : {h.s64_nm1, h.s64_nm2})
            if (d) CUDA_TRY(cudaMemcpyAsync(d, h.s64_n, db, cudaMemcpyDeviceToDevice, s));
    }
    CUDA_TRY(cudaStreamSynchronize(s));
    I->ionic_threads = best;
    I->grid_ionic = (h.N + best - 1) / best;
    std::lock_guard<std::mutex> lk(g_tune_mu);
    g_tune_ionic.emplace_back(key, best);
    return EP_OK;
}

void free_all(ep_instance* I) {
    for (auto& p : I->pending) {
        cudaEventDestroy(p.a);
        cudaEventDestroy(p.b);
    }
    for (auto e : I->free_events) cudaEventDestroy(e);
    if (I->exec) cudaGraphExecDestroy(I->exec);
    if (I->graph) cudaGraphDestroy(I->graph);
    for (void* p : I->allocs) cudaFree(p);
    I->allocs.clear();
    if (I->stream) {
        for (void* p : I->temps) cudaFreeAsync(p, I->stream);
        if (!I->temps.empty()) cudaStreamSynchronize(I->stream);
    }
    I->temps.clear();
    if (I->own_stream && I->stream) cudaStreamDestroy(I->stream);
}

// Triquadratic slab operators, computed on the host in double: per element
// and Gauss point the flux matrix w_q |J| H D(q) H (D of Eq. (3) with the
// fibres Q2-interpolated to the point, not renormalised), uploaded as
// float-float pairs; the diagonals of M and K; the Jacobi diagonal for the
// first step; the norm scale.
ep_status q2_setup(ep_instance* I, const ep_fibers* fib, double dl, double dtr, double dn) {
    Dev& h = I->h;
    const size_t N = (size_t)h.N, E = (size_t)h.ne, EQ = E * 27;
    const double r = std::sqrt(15.0) / 10.0;
    const double xq[3] = {0.5 - r, 0.5, 0.5 + r};
    const double w1[3] = {5.0 / 18.0, 8.0 / 18.0, 5.0 / 18.0};
    double L1[3][3], D1[3][3];  // [q][b]: l_b(xi_q), l_b'(xi_q)
    for (int q = 0; q < 3; ++q) {
        const double t = xq[q];
        L1[q][0] = (1.0 - t) * (1.0 - 2.0 * t);
        L1[q][1] = 4.0 * t * (1.0 - t);
        L1[q][2] = t * (2.0 * t - 1.0);
        D1[q][0] = 4.0 * t - 3.0;
        D1[q][1] = 4.0 - 8.0 * t;
        D1[q][2] = 4.0 * t - 1.0;
    }
    const double ih[3] = {1.0 / h.h[0], 1.0 / h.h[1], 1.0 / h.h[2]};
    const double vol = h.q2vol;
    std::vector<float> G(12 * EQ);
    std::vector<double> dM(N, 0.0), dK(N, 0.0);
    for (size_t e = 0; e < E; ++e) {
        const int ei = (int)(e % h.enx), ej = (int)((e / h.enx) % h.eny), ek = (int)(e / ((size_t)h.enx * h.eny));
        int node[27];
        for (int a = 0; a < 27; ++a)
            node[a] = (2 * ei + a % 3) + h.NX * ((2 * ej + (a / 3) % 3) + h.NY * (2 * ek + a / 9));
        for (int q = 0; q < 27; ++q) {
            const int q0 = q % 3, q1 = (q / 3) % 3, q2 = q / 9;
            double f[3] = {0, 0, 0}, sv[3] = {0, 0, 0};
            double phi[27], gr[27][3];
            for (int a = 0; a < 27; ++a) {
                const int a0 = a % 3, a1 = (a / 3) % 3, a2 = a / 9;
                phi[a] = L1[q0][a0] * L1[q1][a1] * L1[q2][a2];
                gr[a][0] = D1[q0][a0] * L1[q1][a1] * L1[q2][a2];
                gr[a][1] = L1[q0][a0] * D1[q1][a1] * L1[q2][a2];
                gr[a][2] = L1[q0][a0] * L1[q1][a1] * D1[q2][a2];
                for (int c = 0; c < 3; ++c) {
                    f[c] += phi[a] * fib->f0[3 * (size_t)node[a] + c];
                    sv[c] += phi[a] * fib->s0[3 * (size_t)node[a] + c];
                }
            }
            const double w = w1[q0] * w1[q1] * w1[q2] * vol;
            double Gm[3][3];
            for (int i = 0; i < 3; ++i)
                for (int j = 0; j < 3; ++j) {
                    const double Dij = (i == j ? dn : 0.0) + (dl - dn) * f[i] * f[j] + (dtr - dn) * sv[i] * sv[j];
                    Gm[i][j] = w * ih[i] * Dij * ih[j];
                }
            const double comp[6] = {Gm[0][0], Gm[1][1], Gm[2][2], Gm[0][1], Gm[0][2], Gm[1][2]};
            for (int c = 0; c < 6; ++c) split_ff(comp[c], G[c * EQ + e * 27 + q], G[(6 + c) * EQ + e * 27 + q]);
            for (int a = 0; a < 27; ++a) {
                dM[node[a]] += w * phi[a] * phi[a];
                double k = 0.0;
                for (int i = 0; i < 3; ++i)
                    for (int j = 0; j < 3; ++j) k += gr[a][i] * Gm[i][j] * gr[a][j];
                dK[node[a]] += k;
            }
        }
    }
    CUDA_TRY(cudaMemcpy(const_cast<float*>(h.q2G), G.data(), G.size() * 4, cudaMemcpyHostToDevice));
    {
        // FP32 apply's copy: [6][27][ne]
        std::vector<float> T(6 * EQ);
        for (int c = 0; c < 6; ++c)
            for (size_t e = 0; e < E; ++e)
                for (int q = 0; q < 27; ++q) T[((size_t)c * 27 + q) * E + e] = G[c * EQ + e * 27 + q];
        CUDA_TRY(cudaMemcpy(const_cast<float*>(h.q2G32), T.data(), T.size() * 4, cudaMemcpyHostToDevice));
    }
    CUDA_TRY(cudaMemcpy(h.q2dM, dM.data(), N * 8, cudaMemcpyHostToDevice));
    CUDA_TRY(cudaMemcpy(h.q2dK, dK.data(), N * 8, cudaMemcpyHostToDevice));
    std::vector<float> di(N);
    for (size_t n = 0; n < N; ++n) di[n] = (float)(1.0 / (h.alpha_dt * dM[n] + dK[n]));
    CUDA_TRY(cudaMemcpy(h.dinv32, di.data(), N * 4, cudaMemcpyHostToDevice));
    // norm scale from a vertex's mass diagonal (keeps the float sums of
    // squares in range)
    h.nscale = dM[0] > 0.0 ? (float)(1.0 / dM[0]) : 1.0f;
    CUDA_TRY(cudaMemcpy(I->d, &h, sizeof(Dev), cudaMemcpyHostToDevice));
    return EP_OK;
}

ep_status create_impl(const ep_mesh* mesh, const ep_fibers* fib, const ep_conductivities* cond,
                      const ep_ionic_model* ionic, const ep_stimulus* stim, const ep_options* opts,
                      ep_instance* I) {
    const Sizes z = sizes_of(mesh, ionic, opts);
    Dev& h = I->h;
    std::memset(&h, 0, sizeof(h));
    const size_t N = (size_t)z.N;
    h.kind = mesh->kind;
    h.nx = mesh->nx;
    h.ny = mesh->ny;
    h.nz = mesh->nz;
    h.NX = mesh->nx + 1;
    h.NY = mesh->kind == EP_MESH_SHELL ? mesh->ny : mesh->ny + 1;
    h.NZ = mesh->nz + 1;
    h.periodic = mesh->kind == EP_MESH_SHELL;
    h.N = z.N;
    if (mesh->kind == EP_MESH_SLAB || mesh->kind == EP_MESH_SLAB_Q2)
        for (int d = 0; d < 3; ++d) h.h[d] = mesh->L[d] / (d == 0 ? mesh->nx : d == 1 ? mesh->ny : mesh->nz);
    if (z.q2) {
        // node grid of half the element size; h holds the element sizes
        h.q2 = 1;
        h.NX = 2 * mesh->nx + 1;
        h.NY = 2 * mesh->ny + 1;
        h.NZ = 2 * mesh->nz + 1;
        h.enx = mesh->nx;
        h.eny = mesh->ny;
        h.enz = mesh->nz;
        h.ne = (int)z.ne;
        h.q2vol = h.h[0] * h.h[1] * h.h[2];
    }
    h.model = ionic->model;
    h.prec = opts->precision;
    h.bdf = opts->bdf_order;
    h.ns = z.ns;
    h.dt = opts->dt;
    h.inv_dt = 1.0 / opts->dt;
    split_ff(h.inv_dt, h.idt_hi, h.idt_lo);
    h.act_thr = ionic->model == EP_MODEL_BO ? 1.0 / kBOmV : 1.0;
    h.op32 = z.op32;
    const bool ref = h.prec == EP_PREC_FP32_REFINED;
    h.tol = opts->tol > 0 ? opts->tol : (ref ? 1e-10 : 1e-12);
    // the inner stop relative to the sweep's start: on the curved shell a
    // tenth of the usual float floor lets the first sweep end the
    // refinement more often (2.19M-node shell, t = 11-41 ms: 1.32 against
    // 1.99 sweeps a step with the same inner iterations, 1749 against
    // 1911 us a step's solve; over t = 11-111 ms 1.79 sweeps, 1835 against
    // 1852 us); on slabs it only adds iterations (442k nodes: 347 against
    // 339 us)
    h.inner_tol = opts->inner_tol > 0 ? opts->inner_tol : (mesh->kind == EP_MESH_SHELL ? 1e-7 : 1e-6);
    h.max_iter = opts->max_iter > 0 ? opts->max_iter : (ref ? 200 : 1000);
    h.max_sweeps = opts->max_sweeps > 0 ? opts->max_sweeps : 8;

    if (opts->cuda_stream) {
        I->stream = (cudaStream_t)opts->cuda_stream;
    } else {
        CUDA_TRY(cudaStreamCreateWithFlags(&I->stream, cudaStreamNonBlocking));
        I->own_stream = true;
    }
    ep_status st;
#define ALLOC(ptr, n) \
    if ((st = dalloc(I, &(ptr), (n))) != EP_OK) return st
    ALLOC(h.u_n, N);
    ALLOC(h.u_nm1, N);
    ALLOC(h.u_new, N);
    const bool lv3 = z.levels == 3;
    if (lv3) ALLOC(h.u_nm2, N);
    if (z.ng32) {
        ALLOC(h.g32_n, z.ng32 * N);
        ALLOC(h.g32_nm1, z.ng32 * N);
        if (lv3) ALLOC(h.g32_nm2, z.ng32 * N);
    }
    if (z.ns64) {
        ALLOC(h.s64_n, z.ns64 * N);
        ALLOC(h.s64_nm1, z.ns64 * N);
        if (lv3) ALLOC(h.s64_nm2, z.ns64 * N);
    }
    uint8_t* cell = nullptr;
    ALLOC(cell, N);
    h.cell = cell;
    if (z.regions) {
        uint8_t* act = nullptr;
        ALLOC(act, N);
        h.active = act;  // written by the assembly
    }
    if (!ref) {
        ALLOC(h.v, N);
        ALLOC(h.b, N);
        ALLOC(h.r, N);
    }
    ALLOC(h.at, N);
    ALLOC(h.best, N);
    if (!z.q2 && !ref) {
        ALLOC(h.M64, epk::kSlots * N);
        ALLOC(h.A64, epk::kSlots * N);
        ALLOC(h.dinv64, N);
    } else if (!z.q2) {
        // the refined path splits them into float-float couplings and drops them
        if ((st = dalloc_temp(I, &h.M64, epk::kSlots * N)) != EP_OK) return st;
        if ((st = dalloc_temp(I, &h.A64, epk::kSlots * N)) != EP_OK) return st;
        if ((st = dalloc_temp(I, &h.dinv64, N)) != EP_OK) return st;
    }
    if (ref) {
        ALLOC(h.dinv32, N);
        if (z.q2) {
            const size_t eq = (size_t)z.ne * 27;
            float* G = nullptr;
            ALLOC(G, 12 * eq);
            h.q2G = G;
            float* G32 = nullptr;
            ALLOC(G32, 6 * eq);
            h.q2G32 = G32;
            ALLOC(h.q2Y32, 8 * N);
            ALLOC(h.q2Yh, 8 * N);
            ALLOC(h.q2Yl, 8 * N);
            ALLOC(h.q2Bh, 8 * N);
            ALLOC(h.q2Bl, 8 * N);
            ALLOC(h.q2dM, N);
            ALLOC(h.q2dK, N);
        } else {
            h.cs = z.cs;
            const size_t cc = (size_t)epk::kSlots * z.cs;
            if ((st = dalloc_padded(I, &h.Ahi, cc, z.cpad)) != EP_OK) return st;
            if ((st = dalloc_padded(I, &h.Alo, cc, z.cpad)) != EP_OK) return st;
        }
        if (!z.slab_mass && !z.q2) {
            const size_t cc = (size_t)epk::kSlots * z.cs;
            if ((st = dalloc_padded(I, &h.Mhi, cc, z.cpad)) != EP_OK) return st;
            if ((st = dalloc_padded(I, &h.Mlo, cc, z.cpad)) != EP_OK) return st;
        }
        ALLOC(h.uh_n, N);
        ALLOC(h.ul_n, N);
        ALLOC(h.uh_m, N);
        ALLOC(h.ul_m, N);
        if (lv3) {
            ALLOC(h.uh_m2, N);
            ALLOC(h.ul_m2, N);
            ALLOC(h.ym2_hi, N);
            ALLOC(h.ym2_lo, N);
        }
        ALLOC(h.bestf, N);
        ALLOC(h.yc_hi, N);
        ALLOC(h.yc_lo, N);
        ALLOC(h.yn_hi, N);
        ALLOC(h.yn_lo, N);
        ALLOC(h.ym_hi, N);
        ALLOC(h.ym_lo, N);
        ALLOC(h.u_hi, N);
        ALLOC(h.u_lo, N);
        ALLOC(h.v_hi, N);
        ALLOC(h.v_lo, N);
        ALLOC(h.b_hi, N);
        ALLOC(h.b_lo, N);
        if (z.op32 != EP_OP_STENCIL && z.slab) ALLOC(h.fib, 6 * N);
        if (z.op32 != EP_OP_STENCIL && z.shell) ALLOC(I->mfc_geo, epk::mfc_geo_floats(z.NX, z.NY, z.NZ));
        ALLOC(h.r32, N);
        if ((st = dalloc_padded(I, &h.z32, N, z.npad)) != EP_OK) return st;
        ALLOC(h.q32, N);
        ALLOC(h.d32, N);
        ALLOC(h.pa32, N);
        ALLOC(h.pb32, N);
        h.npad = (int)z.npad;
        if (!z.q2) ALLOC(h.nflag, N);
    } else {
        ALLOC(h.z64, N);
        ALLOC(h.q64, N);
        ALLOC(h.pa64, N);
        ALLOC(h.pb64, N);
    }
    ALLOC(h.partial, std::max((N + 255) / 256 + 1, (size_t)epk::kMaxPersistentBlocks) * 8);
    ALLOC(h.counter, (size_t)epk::CNT_N);
    ALLOC(I->d, 1);
    // stimulus
    h.npulses = stim ? stim->n_pulses : 0;
    std::vector<uint8_t*> masks;
    for (int p = 0; p < h.npulses; ++p) {
        const ep_pulse& P = stim->pulses[p];
        h.amp[p] = P.amp;
        h.k0[p] = llround(P.t0 / h.dt);
        h.kd[p] = llround(P.dur / h.dt);
        h.kp[p] = P.period > 0 ? llround(P.period / h.dt) : 0;
        uint8_t* m = nullptr;
        ALLOC(m, N);
        if (P.mask) CUDA_TRY(cudaMemcpyAsync(m, P.mask, N, cudaMemcpyHostToDevice, I->stream));
        else CUDA_TRY(cudaMemsetAsync(m, 0, N, I->stream));
        h.mask[p] = m;
        if (P.elem) {
            // the Gauss-integrated vector of a unit current on the region
            const std::vector<double> g = region_vector(mesh, h, P.elem);
            if (ref) {
                std::vector<float> gh(N), gl(N);
                for (size_t i = 0; i < N; ++i) split_ff(g[i], gh[i], gl[i]);
                float *dh = nullptr, *dl = nullptr;
                ALLOC(dh, N);
                ALLOC(dl, N);
                CUDA_TRY(cudaMemcpy(dh, gh.data(), N * 4, cudaMemcpyHostToDevice));
                CUDA_TRY(cudaMemcpy(dl, gl.data(), N * 4, cudaMemcpyHostToDevice));
                h.egh[p] = dh;
                h.egl[p] = dl;
            } else {
                double* dg = nullptr;
                ALLOC(dg, N);
                CUDA_TRY(cudaMemcpy(dg, g.data(), N * 8, cudaMemcpyHostToDevice));
                h.eg64[p] = dg;
            }
        } else if (P.weight) {
            // the profile in the path's precision
            if (ref) {
                std::vector<float> w32(N);
                for (size_t i = 0; i < N; ++i) w32[i] = (float)P.weight[i];
                float* w = nullptr;
                ALLOC(w, N);
                CUDA_TRY(cudaMemcpy(w, w32.data(), N * 4, cudaMemcpyHostToDevice));
                h.wgt32[p] = w;
            } else {
                double* w = nullptr;
                ALLOC(w, N);
                CUDA_TRY(cudaMemcpy(w, P.weight, N * 8, cudaMemcpyHostToDevice));
                h.wgt64[p] = w;
            }
        }
    }

    // ---- initial state ------------------------------------------------------
    {
        std::vector<uint8_t> ct(N, (uint8_t)EP_CELL_EPI);
        if (ionic->cell_type) std::memcpy(ct.data(), ionic->cell_type, N);
        CUDA_TRY(cudaMemcpyAsync(cell, ct.data(), N, cudaMemcpyHostToDevice, I->stream));
        CUDA_TRY(cudaStreamSynchronize(I->stream));
        // initial u and states per cell type: given (e.g. pre-paced), or the
        // model's rest / the paper's epicardial values for every type
        const int S1 = 1 + z.ns;
        std::vector<double> tab(3 * S1);
        for (int c = 0; c < 3; ++c) {
            if (ionic->initial) {
                for (int k = 0; k < S1; ++k) tab[c * S1 + k] = ionic->initial[c * S1 + k];
            } else if (h.model == EP_MODEL_BO) {
                const double bo[4] = {0.0, 1.0, 1.0, 0.0};
                for (int k = 0; k < S1; ++k) tab[c * S1 + k] = bo[k];
            } else {
                tab[c * S1] = epk::kTTInitialV;
                for (int k = 0; k < z.ns; ++k) tab[c * S1 + 1 + k] = epk::tt_initial(k);
            }
        }
        auto init = [&](size_t n, int k) { return tab[(size_t)ct[n] * S1 + k]; };  // k = 0: u
        std::vector<double> uv(N);
        for (size_t n = 0; n < N; ++n) uv[n] = init(n, 0);
        CUDA_TRY(cudaMemcpy(h.u_n, uv.data(), N * 8, cudaMemcpyHostToDevice));
        for (double* d : {h.u_nm1, h.u_nm2, h.u_new})
            if (d) CUDA_TRY(cudaMemcpy(d, uv.data(), N * 8, cudaMemcpyHostToDevice));
        if (z.ng32) {
            // packed refined states: gates (and BO states) as float, TTP06
            // concentrations as float-float (hi and lo slots)
            std::vector<float> g(z.ng32 * N, 0.0f);
            const int ngate = h.model == EP_MODEL_BO ? epk::kBOStates : epk::kTTGates;
            for (size_t n = 0; n < N; ++n)
                for (int k = 0; k < z.ns; ++k) {
                    float hi = (float)init(n, 1 + k), lo = 0.0f;
                    if (k >= ngate) split_ff(init(n, 1 + k), hi, lo);
                    *packed_at(g.data(), N, state_slot(h.model, k, 0), n) = hi;
                    if (k >= ngate) *packed_at(g.data(), N, state_slot(h.model, k, 1), n) = lo;
                }
            for (float* d : {h.g32_n, h.g32_nm1, h.g32_nm2})
                if (d) CUDA_TRY(cudaMemcpy(d, g.data(), g.size() * 4, cudaMemcpyHostToDevice));
        }
        if (z.ns64 && !ref) {
            std::vector<double> c(z.ns64 * N);
            for (int k = 0; k < z.ns64; ++k)
                for (size_t n = 0; n < N; ++n) c[k * N + n] = init(n, 1 + k);
            for (double* d : {h.s64_n, h.s64_nm1, h.s64_nm2})
                if (d) CUDA_TRY(cudaMemcpy(d, c.data(), c.size() * 8, cudaMemcpyHostToDevice));
        }
        if (ref) {
            std::vector<float> fh(N), fl(N), fb(N, -INFINITY);
            for (size_t n = 0; n < N; ++n) split_ff(uv[n], fh[n], fl[n]);
            for (float* d : {h.uh_n, h.uh_m, h.uh_m2})
                if (d) CUDA_TRY(cudaMemcpy(d, fh.data(), N * 4, cudaMemcpyHostToDevice));
            for (float* d : {h.ul_n, h.ul_m, h.ul_m2})
                if (d) CUDA_TRY(cudaMemcpy(d, fl.data(), N * 4, cudaMemcpyHostToDevice));
            CUDA_TRY(cudaMemcpy(h.bestf, fb.data(), N * 4, cudaMemcpyHostToDevice));
        }
        std::vector<double> nanv(N, NAN), ninf(N, -INFINITY);
        CUDA_TRY(cudaMemcpy(h.at, nanv.data(), N * 8, cudaMemcpyHostToDevice));
        CUDA_TRY(cudaMemcpy(h.best, ninf.data(), N * 8, cudaMemcpyHostToDevice));
        CUDA_TRY(cudaMemset(h.counter, 0, epk::CNT_N * sizeof(unsigned int)));
        if (h.v) CUDA_TRY(cudaMemset(h.v, 0, N * 8));
        for (float* f : {h.u_hi, h.u_lo, h.v_hi, h.v_lo, h.b_hi, h.b_lo, h.r32, h.d32, h.q32})
            if (f) CUDA_TRY(cudaMemset(f, 0, N * 4));
    }

    // ---- operators ----------------------------------------------------------
    double dl = cond->sigma_l, dtr = cond->sigma_t, dn = cond->sigma_n;
    if (!cond->is_D) {
        const double s = 1.0 / (cond->chi_m * cond->Cm);  // Sec. 1.1.2: D = sigma/(chi_m C_m)
        dl *= s;
        dtr *= s;
        dn *= s;
    }
    const double alpha_dt = required_alpha_dt(h, 0);
    I->alpha_dt_dev = alpha_dt;
    h.alpha_dt = alpha_dt;
    if (h.kind == EP_MESH_SLAB) {
        const double vol = h.h[0] * h.h[1] * h.h[2], w = vol / 8.0;
        for (int d = 0; d < 3; ++d) h.mf_cn[d] = (float)(w * dn / (h.h[d] * h.h[d]));
        h.mf_cl = (float)(w * (dl - dn));
        h.mf_ct = (float)(w * (dtr - dn));
        h.mf_cmass = (float)(alpha_dt * vol);
        const double mw = vol / 216.0;  // slab mass weight (analytic mass matrix)
        h.mw_hi = (float)mw;
        h.mw_lo = (float)(mw - (double)h.mw_hi);
    } else if (h.kind == EP_MESH_SHELL) {
        // matrix-free curved apply: D = dn I + (dl-dn) f f^T + (dt-dn) s s^T,
        // mass coefficient alpha/dt (the Jacobian is formed per point)
        h.mf_cn[0] = h.mf_cn[1] = h.mf_cn[2] = (float)dn;
        h.mf_cl = (float)(dl - dn);
        h.mf_ct = (float)(dtr - dn);
        h.mf_cmass = (float)alpha_dt;
    }
    CUDA_TRY(cudaMemcpy(I->d, &h, sizeof(Dev), cudaMemcpyHostToDevice));
    if (z.q2) {
        ep_status st2 = q2_setup(I, fib, dl, dtr, dn);
        if (st2 != EP_OK) return st2;
    } else {
        // the assembly's inputs: stream-ordered temporaries (dalloc_temp)
        cudaStream_t cs = I->stream;
        double *f0 = nullptr, *s0 = nullptr, *xyz = nullptr;
        int* bad = nullptr;
        uint8_t* label = nullptr;
        if ((st = dalloc_temp(I, &f0, N * 3)) != EP_OK) return st;
        if ((st = dalloc_temp(I, &s0, N * 3)) != EP_OK) return st;
        if (h.kind == EP_MESH_SHELL && (st = dalloc_temp(I, &xyz, N * 3)) != EP_OK) return st;
        if ((st = dalloc_temp(I, &bad, 1)) != EP_OK) return st;
        cudaError_t e = cudaMemcpyAsync(f0, fib->f0, N * 24, cudaMemcpyHostToDevice, cs);
        if (e == cudaSuccess) e = cudaMemcpyAsync(s0, fib->s0, N * 24, cudaMemcpyHostToDevice, cs);
        if (e == cudaSuccess && xyz) e = cudaMemcpyAsync(xyz, mesh->xyz, N * 24, cudaMemcpyHostToDevice, cs);
        if (e == cudaSuccess) e = cudaMemsetAsync(bad, 0, sizeof(int), cs);
        int bad_h = 0;
        epk::AsmParams P{xyz, f0, s0, dl, dtr, dn, alpha_dt, bad, nullptr, {}, {}};
        if (e == cudaSuccess && mesh->region) {
            const size_t ne = (size_t)mesh->nx * mesh->ny * mesh->nz;
            if ((st = dalloc_temp(I, &label, ne)) != EP_OK) return st;
            e = cudaMemcpyAsync(label, mesh->region, ne, cudaMemcpyHostToDevice, cs);
            P.label = label;
            const double sc = cond->is_D ? 1.0 : 1.0 / (cond->chi_m * cond->Cm);
            for (int r = 0; r < cond->n_regions; ++r) {
                for (int c = 0; c < 3; ++c) P.rd[r][c] = cond->region_sigma[r][c] * sc;
                P.excl[r] = cond->non_conductive[r] ? 1 : 0;
            }
        }
        if (e == cudaSuccess) {
            epk::launch_assemble(I->d, h, P, cs);
            e = cudaGetLastError();
            if (e == cudaSuccess) e = cudaMemcpyAsync(&bad_h, bad, sizeof(int), cudaMemcpyDeviceToHost, cs);
            if (e == cudaSuccess) e = cudaStreamSynchronize(cs);
        }
        dfree_temp(I, f0);
        dfree_temp(I, s0);
        dfree_temp(I, xyz);
        dfree_temp(I, bad);
        dfree_temp(I, label);
        if (e != cudaSuccess) return fail(EP_ECUDA, std::string("assembly: ") + cudaGetErrorString(e));
        if (bad_h) return fail(EP_EINVAL, "mesh has an element with non-positive Jacobian determinant");
    }
    if (ref && !z.q2) {
        // refined operators: full float-float couplings; norm scale from a
        // mass-matrix diagonal (keeps the float sums of squares in range)
        epk::launch_expand(I->d, h, 1, 1, I->stream);
        CUDA_TRY(cudaGetLastError());
        CUDA_TRY(cudaStreamSynchronize(I->stream));
        double m0 = 0.0;
        CUDA_TRY(cudaMemcpyAsync(&m0, h.M64, sizeof(double), cudaMemcpyDeviceToHost, I->stream));
        CUDA_TRY(cudaStreamSynchronize(I->stream));
        h.nscale = m0 > 0.0 ? (float)(1.0 / m0) : 1.0f;
        // from here on the refined path reads only the float-float couplings
        dfree_temp(I, h.M64);
        dfree_temp(I, h.A64);
        dfree_temp(I, h.dinv64);
        CUDA_TRY(cudaMemcpy(I->d, &h, sizeof(Dev), cudaMemcpyHostToDevice));
    }
    if (h.fib) {
        std::vector<float> f(6 * N);
        for (size_t n = 0; n < N; ++n)
            for (int c = 0; c < 3; ++c) {
                f[c * N + n] = (float)(fib->f0[3 * n + c] / h.h[c]);
                f[(3 + c) * N + n] = (float)(fib->s0[3 * n + c] / h.h[c]);
            }
        CUDA_TRY(cudaMemcpy(h.fib, f.data(), f.size() * 4, cudaMemcpyHostToDevice));
        CUDA_TRY(epk::mf_prepare());
    }
    if (I->mfc_geo) {
        // coordinates and fibre frames for the TMA-staged curved apply
        std::vector<float> g(epk::mfc_geo_floats(h.NX, h.NY, h.NZ));
        epk::mfc_fill_geo(g.data(), h.NX, h.NY, h.NZ, mesh->xyz, fib->f0, fib->s0);
        CUDA_TRY(cudaMemcpy(I->mfc_geo, g.data(), g.size() * 4, cudaMemcpyHostToDevice));
        CUDA_TRY(epk::mfc_tensor_map(&I->mfc_tm, I->mfc_geo, h.NX, h.NY, h.NZ));
        CUDA_TRY(epk::mfc_prepare(h.NX));
    }
    const int blocks = (int)((N + epk::kNodeThreads - 1) / epk::kNodeThreads);
    int dev = 0, sms = 152;
    CUDA_TRY(cudaGetDevice(&dev));
    CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    // pointwise reducing kernels: a persistent grid of four 256-thread blocks
    // per SM (one partial sum and one counter update per block); tiled (FP64)
    // stencil kernels and the node-parallel first residual and residual: two
    // 512-thread blocks per SM; the persistent solve: as many blocks as fit
    // (one per SM alone)
    I->grid_nodes = std::max(1, std::min(blocks, 4 * sms));
    I->ionic_threads = opts->ionic_threads ? opts->ionic_threads : epk::kIonicThreads;
    I->grid_ionic = (int)((N + I->ionic_threads - 1) / I->ionic_threads);
    // (curved meshes: the right-hand side runs one 128-register block per
    // SM, so one wave of them -- 2.19M-node shell 141 against 151 us with two)
    I->grid_resid = std::max(1, std::min((int)((N + epk::kResidThreads - 1) / epk::kResidThreads),
                                         (h.Mhi ? 1 : 2) * sms));
    I->grid_tiles = std::max(1, std::min(epk::st_tiles(h), 2 * sms));
    if (ref) {
        // the persistent solver's blocks must all be resident at once: one
        // 1024-thread block per SM (measured fastest of three launch shapes
        // on the 442k-node slab and the 2.19M-node shell, k_pcg.cu)
        // L2 policies when the solve's working set (the FP32 operator's 14
        // couplings and the seven CG vectors, 84 B a node) exceeds L2:
        // measured on the 2.19M-node shell 1871 against 2044 us a step's
        // solve, on the L2-resident 442k-node slab 300 against 248 us
        int l2 = 0;
        CUDA_TRY(cudaDeviceGetAttribute(&l2, cudaDevAttrL2CacheSize, dev));
        I->pcg_hint = (double)N * 84.0 > (double)l2 ? 1 : 0;
        const int occ = std::min(epk::pcg_blocks_per_sm(), 1);
        if (occ <= 0) return fail(EP_ECUDA, "occupancy query of the persistent solver failed");
        const int bt = epk::pcg_threads_of();
        const int want = (int)((N + bt - 1) / bt);
        I->grid_pcg = std::max(1, std::min(std::min(want, sms * occ), epk::kMaxPersistentBlocks));
        // the apply on tiles staged in shared memory (Q1 meshes), on request:
        // on the 2.19M-node LV shell it measured slower than the node-parallel
        // apply (k_pcg.cu)
        I->pcg_tiled = 0;
        if (!z.q2 && opts->solve_tiles == 2) {
            int by = 0, jt = 0, kr = 0, l = 0;
            double cost = 0.0;
            const bool planned =
                epk::plan_tiles(h.NX, h.NY, h.NZ, sms, epk::tiled_smem_max(), &by, &jt, &kr, &l, &cost);
            const bool want_tiles = opts->solve_tiles == 2;
            if (opts->solve_tiles == 2 && !planned)
                return fail(EP_EUNSUPPORTED, "no tile plan of the persistent solve fits this mesh");
            int fits = 0;
            if (planned && want_tiles) CUDA_TRY(epk::pcg_tiled_prepare(epk::tiled_smem_bytes(l, h.NX), &fits));
            if (opts->solve_tiles == 2 && !fits)
                return fail(EP_EUNSUPPORTED, "the tiled solve's blocks do not fit on the SMs");
            if (planned && want_tiles && fits) {
                I->pcg_tiled = 1;
                h.tile_by = by;
                h.tile_jt = jt;
                h.tile_kr = kr;
                h.tile_l = l;
                I->grid_pcg = jt * kr;
                CUDA_TRY(cudaMemcpy(&I->d->tile_by, &h.tile_by, 4 * sizeof(int), cudaMemcpyHostToDevice));
            }
        }
    }
    if (!ref) h.op32 = 0;  // no FP32 operator in the FP64 path
    if (ref && !z.q2 && h.op32 == EP_OP_AUTO) {
        ep_status st2 = autotune_op32(I);
        if (st2 != EP_OK) return st2;
    }
    if (opts->ionic_threads == 0) {
        ep_status st2 = autotune_ionic(I);
        if (st2 != EP_OK) return st2;
    }
    const char* env = std::getenv("EP_GRAPH");
    I->graph_mode = !(env && env[0] == '0');
    if (!I->graph_mode) return EP_OK;
    return build_graph(I);
}

// ---- batched stepping --------------------------------------------------------
// ep_step_batch runs refined stencil-operator instances together: one launch
// per phase over all instances (one ionic launch per model and level count),
// every instance's refinement sweeps inside one persistent solve launch (each
// instance's blocks loop over its own sweeps and leave when it has
// converged), all captured in one CUDA graph per batch.  Every instance keeps
// the block counts of its own single-instance launches in the non-persistent
// kernels, so their reductions sum in the same order as when it runs alone;
// the persistent solver's blocks are shared out in proportion to the
// instances' sizes (one cooperative grid must fit on the GPU), which changes
// only the rounding of the inner iterations and residual sums.

struct BatchPlan {
    std::vector<ep_instance*> key;
    cudaStream_t stream = nullptr;
    void* dmem = nullptr;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    void release() {
        if (exec) cudaGraphExecDestroy(exec);
        if (graph) cudaGraphDestroy(graph);
        if (dmem) cudaFree(dmem);
        if (stream) cudaStreamDestroy(stream);
        exec = nullptr;
        graph = nullptr;
        dmem = nullptr;
        stream = nullptr;
    }
};

std::mutex g_batch_mu;
std::vector<BatchPlan*> g_plans;  // most recent last, at most kMaxPlans
constexpr size_t kMaxPlans = 4;

void drop_plans_of(const ep_instance* I) {
    std::lock_guard<std::mutex> lk(g_batch_mu);
    for (size_t k = 0; k < g_plans.size();) {
        BatchPlan* P = g_plans[k];
        if (std::find(P->key.begin(), P->key.end(), I) != P->key.end()) {
            P->release();
            delete P;
            g_plans.erase(g_plans.begin() + k);
        } else {
            ++k;
        }
    }
}

bool batchable(const ep_instance* I) {
    return I && I->h.prec == EP_PREC_FP32_REFINED && I->h.op32 == EP_OP_STENCIL && I->graph_mode &&
           !I->profiling && I->sticky == EP_OK;
}

ep_status build_plan(BatchPlan* P) {
    const int n = (int)P->key.size();
    int dev = 0, sms = 152;
    CUDA_TRY(cudaGetDevice(&dev));
    CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    const int occ = epk::pcg_blocks_per_sm();  // the batched solve: 1024-thread blocks, as alone
    if (occ <= 0) return fail(EP_ECUDA, "occupancy query of the persistent solver failed");
    const int cap = sms * occ;
    if (n > cap) return fail(EP_EINVAL, "batch larger than the persistent solver's resident blocks");
    // host tables: all instances, then the ionic kernel's groups: BO, TTP06
    // with two levels, TTP06 with three (BDF3)
    std::vector<Dev*> all, grp[3];
    std::vector<int> s_rhs{0}, s_pcg{0}, s_grp[3] = {{0}, {0}, {0}};
    double total = 0.0;
    for (ep_instance* I : P->key) total += (double)I->h.N;
    // persistent solver: the launch lasts as long as its slowest instance,
    // whose time goes with its nodes times its inner iterations over its
    // blocks.  So every instance gets one block, then each further block
    // goes to the instance with the most work per block (at most what it
    // uses alone, the sum within the resident cap); the work is its nodes
    // times the inner iterations of its last step (unknown before the first
    // step: the median of the others).  Shares by size alone left a batch of
    // slabs waiting for its shells, which need about twice the iterations.
    std::vector<double> it(n, 0.0);
    for (int i = 0; i < n; ++i) {
        ep_instance* I = P->key[i];
        if (I->stream) CUDA_TRY(cudaStreamSynchronize(I->stream));
        int li = 0;
        CUDA_TRY(cudaMemcpy(&li, reinterpret_cast<const char*>(I->d) + offsetof(epk::Dev, last_iters), sizeof(int),
                            cudaMemcpyDeviceToHost));
        it[i] = (double)li;
    }
    {
        std::vector<double> known;
        for (double x : it)
            if (x > 0.0) known.push_back(x);
        double med = 10.0;
        if (!known.empty()) {
            std::nth_element(known.begin(), known.begin() + known.size() / 2, known.end());
            med = known[known.size() / 2];
        }
        for (double& x : it)
            if (x <= 0.0) x = med;
    }
    std::vector<int> gp(n, 1);
    int used = n;
    for (;;) {
        int best = -1;
        double wbest = 0.0;
        for (int i = 0; i < n; ++i) {
            if (gp[i] >= P->key[i]->grid_pcg) continue;
            const double w = (double)P->key[i]->h.N * it[i] / gp[i];
            if (w > wbest) {
                wbest = w;
                best = i;
            }
        }
        if (best < 0 || used >= cap) break;
        ++gp[best];
        ++used;
    }
    if (used > cap) return fail(EP_EINVAL, "batch does not fit the persistent solver's resident blocks");
    for (int i = 0; i < n; ++i) {
        ep_instance* I = P->key[i];
        all.push_back(I->d);
        s_rhs.push_back(s_rhs.back() + I->grid_resid);
        s_pcg.push_back(s_pcg.back() + gp[i]);
        const int gi = I->h.model == EP_MODEL_BO ? 0 : (I->h.u_nm2 ? 2 : 1);
        grp[gi].push_back(I->d);
        s_grp[gi].push_back(s_grp[gi].back() + I->grid_ionic);
    }
    // one device buffer: pointer arrays first (8-byte aligned), then ints
    size_t np = all.size();
    size_t ni = s_rhs.size() + s_pcg.size();
    for (int gi = 0; gi < 3; ++gi) {
        np += grp[gi].size();
        ni += s_grp[gi].size();
    }
    std::vector<char> hbuf(np * sizeof(Dev*) + ni * sizeof(int));
    char* q = hbuf.data();
    auto put = [&](const void* src, size_t bytes) {
        std::memcpy(q, src, bytes);
        char* at = q;
        q += bytes;
        return at - hbuf.data();
    };
    const size_t o_all = put(all.data(), all.size() * sizeof(Dev*));
    size_t o_grp[3], o_sgrp[3];
    for (int gi = 0; gi < 3; ++gi) o_grp[gi] = put(grp[gi].data(), grp[gi].size() * sizeof(Dev*));
    const size_t o_st = put(s_rhs.data(), s_rhs.size() * sizeof(int));
    const size_t o_sp = put(s_pcg.data(), s_pcg.size() * sizeof(int));
    for (int gi = 0; gi < 3; ++gi) o_sgrp[gi] = put(s_grp[gi].data(), s_grp[gi].size() * sizeof(int));
    CUDA_TRY(cudaMalloc(&P->dmem, hbuf.size()));
    CUDA_TRY(cudaMemcpy(P->dmem, hbuf.data(), hbuf.size(), cudaMemcpyHostToDevice));
    char* d = static_cast<char*>(P->dmem);
    auto mk = [&](size_t od, size_t os, int cnt, Dev* only) {
        if (cnt == 1) return epk::single_batch(only);
        return epk::Batch{nullptr, reinterpret_cast<Dev* const*>(d + od), reinterpret_cast<const int*>(d + os), cnt};
    };
    const epk::Batch Br = mk(o_all, o_st, n, all[0]);
    const epk::Batch Bp = mk(o_all, o_sp, n, all[0]);

    CUDA_TRY(cudaStreamCreateWithFlags(&P->stream, cudaStreamNonBlocking));
    cudaStream_t s = P->stream, s2 = nullptr;
    CUDA_TRY(cudaStreamCreateWithFlags(&s2, cudaStreamNonBlocking));
    Capture C{s};
    C.chk(cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal));
    for (int gi = 0; gi < 3; ++gi)
        if (!grp[gi].empty())
            epk::launch_ionic_batch(mk(o_grp[gi], o_sgrp[gi], (int)grp[gi].size(), grp[gi][0]),
                                    gi == 0 ? EP_MODEL_BO : EP_MODEL_TTP06, gi == 2, s_grp[gi].back(), s);
    bool curved = false;
    for (const ep_instance* I : P->key) curved = curved || I->h.Mhi != nullptr;
    epk::launch_rhs_ff_batch(Br, 0, s_rhs.back(), curved, s);
    // every instance's refinement sweeps in one persistent launch (the
    // blocks of an instance that needs no sweep return at once)
    // no L2 eviction-priority hints in batches: their instances are each
    // L2-sized and the hints cost the 96-slab batch 9 % (1.06e9 against
    // 1.17e9 DoF-steps/s)
    C.chk(epk::launch_pcg32_batch(Bp, s_pcg.back(), 0, s));
    cudaGraph_t g = nullptr;
    C.chk(cudaStreamEndCapture(s, &g));
    C.chk(cudaGetLastError());
    cudaStreamDestroy(s2);
    if (C.err != cudaSuccess) {
        if (g) cudaGraphDestroy(g);
        return fail(EP_ECUDA, std::string("building the batch graph: ") + cudaGetErrorString(C.err));
    }
    P->graph = g;
    CUDA_TRY(cudaGraphInstantiate(&P->exec, g, 0));
    return EP_OK;
}

// the cached plan for this instance list, built on first use
ep_status get_plan(ep_instance* const* insts, int n, BatchPlan** out) {
    std::vector<ep_instance*> key(insts, insts + n);
    std::lock_guard<std::mutex> lk(g_batch_mu);
    for (size_t k = 0; k < g_plans.size(); ++k)
        if (g_plans[k]->key == key) {
            BatchPlan* P = g_plans[k];
            g_plans.erase(g_plans.begin() + k);
            g_plans.push_back(P);
            *out = P;
            return EP_OK;
        }
    BatchPlan* P = new BatchPlan();
    P->key = key;
    ep_status st = build_plan(P);
    if (st != EP_OK) {
        P->release();
        delete P;
        return st;
    }
    if (g_plans.size() >= kMaxPlans) {
        g_plans.front()->release();
        delete g_plans.front();
        g_plans.erase(g_plans.begin());
    }
    g_plans.push_back(P);
    *out = P;
    return EP_OK;
}

}  // namespace

extern "C" {

const char* ep_last_error(void) { return g_err.c_str(); }

size_t ep_footprint_bytes(const ep_mesh* mesh, const ep_ionic_model* ionic, const ep_options* opts) {
    if (!mesh || !ionic || !opts) return 0;
    if (mesh->nx < 1 || mesh->ny < 1 || mesh->nz < 1) return 0;
    if (ionic->model != EP_MODEL_BO && ionic->model != EP_MODEL_TTP06) return 0;
    if (opts->precision != EP_PREC_FP64 && opts->precision != EP_PREC_FP32_REFINED) return 0;
    const int64_t nn = expected_nodes(mesh);
    if (nn > (int64_t)1 << 30) return 0;
    size_t b = footprint(sizes_of(mesh, ionic, opts));
    return b;
}

ep_status ep_create(const ep_mesh* mesh, const ep_fibers* fibers, const ep_conductivities* cond,
                    const ep_ionic_model* ionic, const ep_stimulus* stim, const ep_options* opts,
                    ep_instance** out) {
    if (!out) return fail(EP_EINVAL, "out is NULL");
    *out = nullptr;
    ep_status st = validate(mesh, fibers, cond, ionic, stim, opts);
    if (st != EP_OK) return st;
    ep_instance* I = new (std::nothrow) ep_instance();
    if (!I) return fail(EP_ENOMEM, "host allocation failed");
    st = create_impl(mesh, fibers, cond, ionic, stim, opts, I);
    if (st != EP_OK) {
        (void)cudaGetLastError();
        free_all(I);
        delete I;
        return st;
    }
    *out = I;
    return EP_OK;
}

ep_status ep_prepace(int32_t model, const uint8_t* cell_types, int32_t n_cells, double period_ms, int32_t beats,
                     double dt, double amp, double dur_ms, int32_t bdf_order, const double* initial,
                     double* out) {
    if (model != EP_MODEL_BO && model != EP_MODEL_TTP06) return fail(EP_EINVAL, "model");
    if (!cell_types || !out || n_cells < 1 || n_cells > 4096) return fail(EP_EINVAL, "cells / out / n_cells");
    for (int i = 0; i < n_cells; ++i)
        if (cell_types[i] > EP_CELL_EPI) return fail(EP_EINVAL, "cell type out of range");
    if (!finite_pos(dt) || !finite_pos(period_ms) || beats < 0 || !std::isfinite(amp) || !(dur_ms >= 0))
        return fail(EP_EINVAL, "pacing parameters");
    if (bdf_order != 1 && bdf_order != 2) return fail(EP_EINVAL, "bdf_order must be 1 or 2");
    const long long kp = llround(period_ms / dt), kd = llround(dur_ms / dt);
    if (kp < 1) return fail(EP_EINVAL, "period shorter than a step");
    const int ns = model == EP_MODEL_BO ? epk::kBOStates : epk::kTTGates + epk::kTTConc;
    const int S1 = 1 + ns;
    constexpr int P = 1 + epk::kTTGates + epk::kTTConc;
    // two levels per cell, both the initial state
    std::vector<double> st((size_t)n_cells * 2 * P, 0.0);
    for (int i = 0; i < n_cells; ++i) {
        double v[P] = {0};
        if (initial) {
            for (int k = 0; k < S1; ++k) v[k] = initial[(size_t)i * S1 + k];
        } else if (model == EP_MODEL_BO) {
            v[0] = 0.0, v[1] = 1.0, v[2] = 1.0, v[3] = 0.0;
        } else {
            v[0] = epk::kTTInitialV;
            for (int k = 0; k < ns; ++k) v[1 + k] = epk::tt_initial(k);
        }
        for (int lv = 0; lv < 2; ++lv)
            for (int k = 0; k < S1; ++k) st[((size_t)i * 2 + lv) * P + k] = v[k];
    }
    double* dst = nullptr;
    uint8_t* dcell = nullptr;
    cudaStream_t s = nullptr;
    auto cleanup = [&] {
        if (dst) cudaFree(dst);
        if (dcell) cudaFree(dcell);
        if (s) cudaStreamDestroy(s);
    };
    cudaError_t e = cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaMalloc(&dst, st.size() * 8);
    if (e == cudaSuccess) e = cudaMalloc(&dcell, (size_t)n_cells);
    if (e == cudaSuccess) e = cudaMemcpy(dst, st.data(), st.size() * 8, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(dcell, cell_types, (size_t)n_cells, cudaMemcpyHostToDevice);
    // the protocol in short launches of at most one beat each
    const long long total = kp * (long long)beats;
    for (long long m0 = 0; e == cudaSuccess && m0 < total; m0 += kp) {
        const long long k = std::min(kp, total - m0);
        e = epk::launch_prepace(model, dcell, n_cells, dt, m0, k, kp, kd, amp, bdf_order, dst, s);
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e == cudaSuccess) e = cudaMemcpy(st.data(), dst, st.size() * 8, cudaMemcpyDeviceToHost);
    cleanup();
    if (e != cudaSuccess) {
        (void)cudaGetLastError();
        return fail(EP_ECUDA, std::string("pre-pacing: ") + cudaGetErrorString(e));
    }
    for (int i = 0; i < n_cells; ++i)
        for (int k = 0; k < S1; ++k) out[(size_t)i * S1 + k] = st[((size_t)i * 2) * P + k];
    return EP_OK;
}

ep_status ep_step_async(ep_instance* I, int64_t n_steps) {
    if (!I) return fail(EP_EINVAL, "instance is NULL");
    if (n_steps < 0) return fail(EP_EINVAL, "n_steps < 0");
    if (I->sticky != EP_OK) return fail(I->sticky, "instance failed earlier: " + std::to_string(I->sticky));
    for (int64_t k = 0; k < n_steps; ++k) {
        ensure_alpha(I);
        if (I->graph_mode && !I->profiling) {
            CUDA_TRY(cudaGraphLaunch(I->exec, I->stream));
        } else {
            ep_status st = step_host(I);
            if (st != EP_OK) return st;
        }
        I->host_step += 1;
        I->fin_pending = I->h.prec == EP_PREC_FP32_REFINED;
        I->solved = true;
    }
    CUDA_TRY(cudaGetLastError());
    return EP_OK;
}

ep_status ep_sync(ep_instance* I) {
    if (!I) return fail(EP_EINVAL, "instance is NULL");
    int status = 0;
    CUDA_TRY(cudaMemcpyAsync(&status, &I->d->status, sizeof(int), cudaMemcpyDeviceToHost, I->stream));
    CUDA_TRY(cudaStreamSynchronize(I->stream));
    if (status != EP_OK) {
        I->sticky = (ep_status)status;
        long long step = 0;
        (void)cudaMemcpy(&step, &I->d->step, sizeof(step), cudaMemcpyDeviceToHost);
        const char* what = status == EP_ENAN ? "non-finite potential"
                           : status == EP_ENOCONV ? "linear solver did not converge"
                                                  : "device error";
        return fail((ep_status)status, std::string(what) + " (time level " + std::to_string(step) + ")");
    }
    return EP_OK;
}

ep_status ep_step(ep_instance* I, int64_t n_steps) {
    ep_status st = ep_step_async(I, n_steps);
    if (st != EP_OK) return st;
    return ep_sync(I);
}

ep_status ep_step_batch(ep_instance* const* insts, int32_t n, int64_t n_steps) {
    if (!insts || n < 0) return fail(EP_EINVAL, "bad batch");
    if (n_steps < 0) return fail(EP_EINVAL, "n_steps < 0");
    for (int32_t k = 0; k < n; ++k) {
        if (!insts[k]) return fail(EP_EINVAL, "NULL instance in the batch");
        for (int32_t j = 0; j < k; ++j)
            if (insts[j] == insts[k]) return fail(EP_EINVAL, "an instance appears twice in the batch");
    }
    bool together = n >= 2;
    for (int32_t k = 0; k < n && together; ++k) together = batchable(insts[k]);
    if (together && n_steps > 0) {
        BatchPlan* P = nullptr;
        ep_status st = get_plan(insts, n, &P);
        if (st != EP_OK) return st;
        for (int32_t k = 0; k < n; ++k) CUDA_TRY(cudaStreamSynchronize(insts[k]->stream));
        for (int64_t step = 0; step < n_steps; ++step) {
            for (int32_t k = 0; k < n; ++k) {
                ep_instance* I = insts[k];
                if (required_alpha_dt(I->h, I->host_step) != I->alpha_dt_dev) {
                    // a BDF order change: update this instance's operators first
                    CUDA_TRY(cudaStreamSynchronize(P->stream));
                    ensure_alpha(I);
                    CUDA_TRY(cudaGetLastError());
                    CUDA_TRY(cudaStreamSynchronize(I->stream));
                }
            }
            CUDA_TRY(cudaGraphLaunch(P->exec, P->stream));
            for (int32_t k = 0; k < n; ++k) {
                insts[k]->host_step += 1;
                insts[k]->fin_pending = insts[k]->h.prec == EP_PREC_FP32_REFINED;
                insts[k]->solved = true;
            }
        }
        CUDA_TRY(cudaStreamSynchronize(P->stream));
        ep_status first = EP_OK;
        std::string msg;
        for (int32_t k = 0; k < n; ++k) {
            ep_status st2 = ep_sync(insts[k]);
            if (st2 != EP_OK && first == EP_OK) {
                first = st2;
                msg = g_err;
            }
        }
        if (first != EP_OK) return fail(first, msg);
        return EP_OK;
    }
    for (int32_t k = 0; k < n; ++k) {
        ep_status st = ep_step_async(insts[k], n_steps);
        if (st != EP_OK) return st;
    }
    ep_status first = EP_OK;
    std::string msg;
    for (int32_t k = 0; k < n; ++k) {
        ep_status st = ep_sync(insts[k]);
        if (st != EP_OK && first == EP_OK) {
            first = st;
            msg = g_err;
        }
    }
    if (first != EP_OK) return fail(first, msg);
    return EP_OK;
}

// Refined instances finish a step's per-node work (activation slope, u_n in
// double) in the next step's ionic kernel; before the host reads the state,
// the last step's is done here (the same idempotent kernel).
static ep_status flush_finish(const ep_instance* I) {
    if (I->fin_pending) {
        epk::launch_finish(I->d, I->h, I->grid_nodes, I->stream);
        CUDA_TRY(cudaGetLastError());
        I->fin_pending = false;
    }
    return EP_OK;
}

ep_status ep_read_potential(const ep_instance* I, double* out, int64_t n) {
    if (!I || !out) return fail(EP_EINVAL, "NULL argument");
    if (n != I->h.N) return fail(EP_EINVAL, "n must equal n_nodes");
    if (ep_status st = flush_finish(I); st != EP_OK) return st;
    Dev tmp;
    CUDA_TRY(cudaMemcpyAsync(&tmp, I->d, sizeof(Dev), cudaMemcpyDeviceToHost, I->stream));
    CUDA_TRY(cudaStreamSynchronize(I->stream));
    CUDA_TRY(cudaMemcpy(out, tmp.u_n, (size_t)n * 8, cudaMemcpyDeviceToHost));
    if (I->h.model == EP_MODEL_BO)
        for (int64_t i = 0; i < n; ++i) out[i] = kBOmV * out[i] + kBOoff;
    return EP_OK;
}

ep_status ep_activation_times(const ep_instance* I, double* out, int64_t n) {
    if (!I || !out) return fail(EP_EINVAL, "NULL argument");
    if (n != I->h.N) return fail(EP_EINVAL, "n must equal n_nodes");
    if (ep_status st = flush_finish(I); st != EP_OK) return st;
    CUDA_TRY(cudaStreamSynchronize(I->stream));
    std::vector<double> best((size_t)n);
    CUDA_TRY(cudaMemcpy(out, I->h.at, (size_t)n * 8, cudaMemcpyDeviceToHost));
    CUDA_TRY(get_best(I, best.data()));
    const double thr = I->h.act_thr * I->h.dt;
    for (int64_t i = 0; i < n; ++i)
        if (!(best[i] > thr)) out[i] = NAN;
    return EP_OK;
}

// Time levels a checkpoint holds: n, n-1 and, for BDF3, n-2.
static int state_levels(int bdf) { return bdf == 3 ? 3 : 2; }

// Refined instances append their float-float working state (tag, history
// count, then float arrays) so that a restart continues bit for bit: the
// potential levels, the concentrations as pairs and the A u history.
static size_t ff_ext_bytes(const ep_instance* I) {
    if (I->h.prec != EP_PREC_FP32_REFINED) return 0;
    const size_t N = (size_t)I->h.N;
    const size_t L = (size_t)state_levels(I->h.bdf);
    const size_t nc = I->h.model == EP_MODEL_BO ? 0 : epk::kTTConc;
    return 16 + 4 * N * 2 * L * (2 + nc);
}

static size_t base_state_bytes(const ep_instance* I) {
    const size_t N = (size_t)I->h.N;
    const size_t L = (size_t)state_levels(I->h.bdf);
    return 64 + 8 * N * (L + L * (size_t)I->h.ns + 2);
}

// the level-l buffers (0: n, 1: n-1, 2: n-2) of a device state copy
static double* lvl_u(const Dev& t, int l) { return l == 0 ? t.u_n : l == 1 ? t.u_nm1 : t.u_nm2; }
static float* lvl_g(const Dev& t, int l) { return l == 0 ? t.g32_n : l == 1 ? t.g32_nm1 : t.g32_nm2; }
static double* lvl_s(const Dev& t, int l) { return l == 0 ? t.s64_n : l == 1 ? t.s64_nm1 : t.s64_nm2; }
static float* lvl_uh(const Dev& t, int l) { return l == 0 ? t.uh_n : l == 1 ? t.uh_m : t.uh_m2; }
static float* lvl_ul(const Dev& t, int l) { return l == 0 ? t.ul_n : l == 1 ? t.ul_m : t.ul_m2; }
static float* lvl_yh(const Dev& t, int l) { return l == 0 ? t.yn_hi : l == 1 ? t.ym_hi : t.ym2_hi; }
static float* lvl_yl(const Dev& t, int l) { return l == 0 ? t.yn_lo : l == 1 ? t.ym_lo : t.ym2_lo; }

size_t ep_state_bytes(const ep_instance* I) {
    if (!I) return 0;
    return base_state_bytes(I) + ff_ext_bytes(I);
}

struct StateHeader {
    char magic[8];
    int32_t version, model;
    int64_t n_nodes;
    int32_t n_states, bdf_order;
    int64_t step;
    double dt;
    int64_t reserved[2];
};
static_assert(sizeof(StateHeader) == 64, "state header is 64 bytes");

ep_status ep_save_state(const ep_instance* I, void* buf, size_t bytes) {
    if (!I || !buf) return fail(EP_EINVAL, "NULL argument");
    const size_t need = ep_state_bytes(I);
    if (bytes < need) return fail(EP_EINVAL, "buffer too small: need " + std::to_string(need));
    if (ep_status st = flush_finish(I); st != EP_OK) return st;
    Dev t;
    CUDA_TRY(cudaMemcpyAsync(&t, I->d, sizeof(Dev), cudaMemcpyDeviceToHost, I->stream));
    CUDA_TRY(cudaStreamSynchronize(I->stream));
    const size_t N = (size_t)I->h.N;
    const int ns = I->h.ns;
    StateHeader H{};
    std::memcpy(H.magic, "EPSTATE1", 8);
    H.version = 1;
    H.model = I->h.model;
    H.n_nodes = (int64_t)N;
    H.n_states = ns;
    H.bdf_order = I->h.bdf;
    H.step = t.step;
    H.dt = I->h.dt;
    H.reserved[0] = (int64_t)ff_ext_bytes(I);
    char* p = static_cast<char*>(buf);
    std::memcpy(p, &H, 64);
    double* o = reinterpret_cast<double*>(p + 64);
    std::vector<double> tmp(N);
    auto get = [&](const double* d, double* dst) -> cudaError_t {
        cudaError_t e = cudaMemcpy(tmp.data(), d, N * 8, cudaMemcpyDeviceToHost);
        std::memcpy(dst, tmp.data(), N * 8);
        return e;
    };
    const int L = state_levels(I->h.bdf);
    for (int lvl = 0; lvl < L; ++lvl) CUDA_TRY(get(lvl_u(t, lvl), o + (size_t)lvl * N));
    const bool ref = I->h.prec == EP_PREC_FP32_REFINED;
    const int ng32 = ref ? (I->h.model == EP_MODEL_BO ? 3 : epk::kTTGates) : 0;
    std::vector<float> f(N), fl(N);
    for (int lvl = 0; lvl < L; ++lvl) {
        double* dst = o + (size_t)L * N + (size_t)lvl * ns * N;
        for (int k = 0; k < ns; ++k) {
            if (k < ng32) {
                CUDA_TRY(get_slot(lvl_g(t, lvl), N, state_slot(I->h.model, k, 0), f.data()));
                for (size_t n = 0; n < N; ++n) tmp[n] = f[n];
                std::memcpy(dst + (size_t)k * N, tmp.data(), N * 8);
            } else if (ref) {
                CUDA_TRY(get_slot(lvl_g(t, lvl), N, state_slot(I->h.model, k, 0), f.data()));
                CUDA_TRY(get_slot(lvl_g(t, lvl), N, state_slot(I->h.model, k, 1), fl.data()));
                for (size_t n = 0; n < N; ++n) tmp[n] = (double)f[n] + (double)fl[n];
                std::memcpy(dst + (size_t)k * N, tmp.data(), N * 8);
            } else {
                const double* src = lvl_s(t, lvl) + (size_t)k * N;
                CUDA_TRY(get(src, dst + (size_t)k * N));
            }
        }
    }
    const size_t oat = (size_t)L * (1 + ns) * N;  // at, then best
    CUDA_TRY(get(t.at, o + oat));
    CUDA_TRY(get_best(I, o + oat + N));
    if (ref) {
        char* e = p + base_state_bytes(I);
        std::memcpy(e, "EPFFEXT1", 8);
        const int32_t hist = t.hist, zero = 0;
        std::memcpy(e + 8, &hist, 4);
        std::memcpy(e + 12, &zero, 4);
        char* q = e + 16;
        auto getf = [&](const float* d) -> cudaError_t {
            cudaError_t err = cudaMemcpy(f.data(), d, N * 4, cudaMemcpyDeviceToHost);
            std::memcpy(q, f.data(), N * 4);
            q += N * 4;
            return err;
        };
        for (int lvl = 0; lvl < L; ++lvl) {
            CUDA_TRY(getf(lvl_uh(t, lvl)));
            CUDA_TRY(getf(lvl_ul(t, lvl)));
        }
        for (int lvl = 0; lvl < L; ++lvl)
            for (int part = 0; part < 2; ++part)
                for (int k = ng32; k < ns; ++k) {
                    CUDA_TRY(get_slot(lvl_g(t, lvl), N, state_slot(I->h.model, k, part), f.data()));
                    std::memcpy(q, f.data(), N * 4);
                    q += N * 4;
                }
        for (int lvl = 0; lvl < L; ++lvl) {
            CUDA_TRY(getf(lvl_yh(t, lvl)));
            CUDA_TRY(getf(lvl_yl(t, lvl)));
        }
    }
    return EP_OK;
}

ep_status ep_load_state(ep_instance* I, const void* buf, size_t bytes) {
    if (!I || !buf) return fail(EP_EINVAL, "NULL argument");
    // the portable part is required; a refined instance's exact extension
    // is used when present
    const size_t need = ep_state_bytes(I);
    if (bytes < base_state_bytes(I)) return fail(EP_EINVAL, "buffer too small");
    StateHeader H;
    std::memcpy(&H, buf, 64);
    if (std::memcmp(H.magic, "EPSTATE1", 8) != 0 || H.version != 1) return fail(EP_EINVAL, "not an EPSTATE1 buffer");
    if (H.model != I->h.model || H.n_nodes != I->h.N || H.n_states != I->h.ns)
        return fail(EP_EINVAL, "state buffer is for a different model or mesh");
    if (H.step < 0) return fail(EP_EINVAL, "negative step");
    if (H.bdf_order < 1 || H.bdf_order > 3 || state_levels(H.bdf_order) != state_levels(I->h.bdf))
        return fail(EP_EINVAL, "state buffer holds a different number of time levels (BDF order)");
    CUDA_TRY(cudaStreamSynchronize(I->stream));
    Dev t;
    CUDA_TRY(cudaMemcpy(&t, I->d, sizeof(Dev), cudaMemcpyDeviceToHost));
    const size_t N = (size_t)I->h.N;
    const int ns = I->h.ns;
    const double* o = reinterpret_cast<const double*>(static_cast<const char*>(buf) + 64);
    std::vector<double> tmp(N);
    auto put = [&](double* d, const double* src) -> cudaError_t {
        std::memcpy(tmp.data(), src, N * 8);
        return cudaMemcpy(d, tmp.data(), N * 8, cudaMemcpyHostToDevice);
    };
    const int L = state_levels(I->h.bdf);
    for (int lvl = 0; lvl < L; ++lvl) CUDA_TRY(put(lvl_u(t, lvl), o + (size_t)lvl * N));
    const bool ref = I->h.prec == EP_PREC_FP32_REFINED;
    const int ng32 = ref ? (I->h.model == EP_MODEL_BO ? 3 : epk::kTTGates) : 0;
    std::vector<float> f(N), fl(N);
    for (int lvl = 0; lvl < L; ++lvl) {
        const double* src = o + (size_t)L * N + (size_t)lvl * ns * N;
        for (int k = 0; k < ns; ++k) {
            if (k < ng32) {
                std::memcpy(tmp.data(), src + (size_t)k * N, N * 8);
                for (size_t n = 0; n < N; ++n) f[n] = (float)tmp[n];
                CUDA_TRY(put_slot(lvl_g(t, lvl), N, state_slot(I->h.model, k, 0), f.data()));
            } else if (ref) {
                std::memcpy(tmp.data(), src + (size_t)k * N, N * 8);
                for (size_t n = 0; n < N; ++n) split_ff(tmp[n], f[n], fl[n]);
                CUDA_TRY(put_slot(lvl_g(t, lvl), N, state_slot(I->h.model, k, 0), f.data()));
                CUDA_TRY(put_slot(lvl_g(t, lvl), N, state_slot(I->h.model, k, 1), fl.data()));
            } else {
                CUDA_TRY(put(lvl_s(t, lvl) + (size_t)k * N, src + (size_t)k * N));
            }
        }
    }
    const size_t oat = (size_t)L * (1 + ns) * N;  // at, then best
    if (ref) {
        // the float-float potential levels from the stored potentials
        for (int lvl = 0; lvl < L; ++lvl) {
            const double* src = o + (size_t)lvl * N;
            for (size_t n = 0; n < N; ++n) split_ff(src[n], f[n], fl[n]);
            CUDA_TRY(cudaMemcpy(lvl_uh(t, lvl), f.data(), N * 4, cudaMemcpyHostToDevice));
            CUDA_TRY(cudaMemcpy(lvl_ul(t, lvl), fl.data(), N * 4, cudaMemcpyHostToDevice));
        }
        const double* bsrc = o + oat + N;
        for (size_t n = 0; n < N; ++n) f[n] = (float)bsrc[n];
        CUDA_TRY(cudaMemcpy(t.bestf, f.data(), N * 4, cudaMemcpyHostToDevice));
    }
    CUDA_TRY(put(t.at, o + oat));
    CUDA_TRY(put(t.best, o + oat + N));
    long long step = H.step;
    int zero = 0;
    CUDA_TRY(cudaMemcpy(&I->d->step, &step, sizeof(step), cudaMemcpyHostToDevice));
    CUDA_TRY(cudaMemcpy(&I->d->status, &zero, sizeof(int), cudaMemcpyHostToDevice));
    // the loaded step's per-node end is part of the state: not redone
    CUDA_TRY(cudaMemcpy(&I->d->fin_pending, &zero, sizeof(int), cudaMemcpyHostToDevice));
    I->fin_pending = false;
    CUDA_TRY(cudaMemset(t.counter, 0, epk::CNT_N * sizeof(unsigned int)));
    I->host_step = step;
    I->sticky = EP_OK;
    // the right-hand side and the A u of the last solve no longer match the
    // loaded potential
    I->solved = false;
    // the operators for the loaded step's BDF order now, so that the restored
    // A u history stays valid for the next step
    ensure_alpha(I);
    CUDA_TRY(cudaGetLastError());
    CUDA_TRY(cudaStreamSynchronize(I->stream));
    int hist = 0;
    const size_t ext = ff_ext_bytes(I);
    const char* e = static_cast<const char*>(buf) + base_state_bytes(I);
    if (ref && H.reserved[0] == (int64_t)ext && bytes >= need && std::memcmp(e, "EPFFEXT1", 8) == 0) {
        int32_t hh = 0;
        std::memcpy(&hh, e + 8, 4);
        hist = std::max(0, std::min(L, (int)hh));
        const char* q = e + 16;
        auto putf = [&](float* d) -> cudaError_t {
            std::memcpy(f.data(), q, N * 4);
            q += N * 4;
            return cudaMemcpy(d, f.data(), N * 4, cudaMemcpyHostToDevice);
        };
        for (int lvl = 0; lvl < L; ++lvl) {
            CUDA_TRY(putf(lvl_uh(t, lvl)));
            CUDA_TRY(putf(lvl_ul(t, lvl)));
        }
        for (int lvl = 0; lvl < L; ++lvl)
            for (int part = 0; part < 2; ++part)
                for (int k = ng32; k < ns; ++k) {
                    std::memcpy(f.data(), q, N * 4);
                    q += N * 4;
                    CUDA_TRY(put_slot(lvl_g(t, lvl), N, state_slot(I->h.model, k, part), f.data()));
                }
        for (int lvl = 0; lvl < L; ++lvl) {
            CUDA_TRY(putf(lvl_yh(t, lvl)));
            CUDA_TRY(putf(lvl_yl(t, lvl)));
        }
    }
    CUDA_TRY(cudaMemcpy(&I->d->hist, &hist, sizeof(int), cudaMemcpyHostToDevice));
    return EP_OK;
}

ep_status ep_get_stats(const ep_instance* I, ep_stats* out) {
    if (!I || !out) return fail(EP_EINVAL, "NULL argument");
    Dev t;
    CUDA_TRY(cudaMemcpyAsync(&t, I->d, sizeof(Dev), cudaMemcpyDeviceToHost, I->stream));
    CUDA_TRY(cudaStreamSynchronize(I->stream));
    out->step = t.step;
    out->cg_iters = t.last_iters;
    out->sweeps = t.last_sweeps;
    out->relres = t.last_relres;
    out->op32 = I->h.prec == EP_PREC_FP32_REFINED ? I->h.op32 : 0;
    out->solve_threads = (I->h.prec == EP_PREC_FP32_REFINED && I->h.op32 == EP_OP_STENCIL)
                             ? epk::pcg_threads_of()
                             : 0;
    out->device_bytes = I->bytes;
    out->tune_us_mf = 1e3 * I->tune_ms[EP_OP_MATRIX_FREE];
    out->tune_us_stencil = 1e3 * I->tune_ms[EP_OP_STENCIL];
    out->ionic_threads = I->ionic_threads;
    out->solve_tiles = (I->h.prec == EP_PREC_FP32_REFINED && I->h.op32 == EP_OP_STENCIL) ? I->pcg_tiled : 0;
    return EP_OK;
}

ep_status ep_potential_device(const ep_instance* I, const double** out) {
    if (!I || !out) return fail(EP_EINVAL, "NULL argument");
    if (ep_status st = flush_finish(I); st != EP_OK) return st;
    Dev t;
    CUDA_TRY(cudaMemcpyAsync(&t, I->d, sizeof(Dev), cudaMemcpyDeviceToHost, I->stream));
    CUDA_TRY(cudaStreamSynchronize(I->stream));
    *out = t.u_n;
    return EP_OK;
}

ep_status ep_profile_enable(ep_instance* I, int32_t on) {
    if (!I) return fail(EP_EINVAL, "instance is NULL");
    CUDA_TRY(cudaStreamSynchronize(I->stream));
    prof_resolve(I);
    I->profiling = on != 0;
    return EP_OK;
}

ep_status ep_profile_read(ep_instance* I, ep_kernel_time* out, int32_t cap, int32_t* n, int32_t reset) {
    if (!I || !n || (cap > 0 && !out)) return fail(EP_EINVAL, "NULL argument");
    CUDA_TRY(cudaStreamSynchronize(I->stream));
    prof_resolve(I);
    int32_t k = 0;
    for (int id = 0; id < K_COUNT; ++id) {
        if (I->prof_n[id] == 0) continue;
        if (k < cap) {
            std::memset(out[k].name, 0, sizeof(out[k].name));
            std::strncpy(out[k].name, kKernelNames[id], sizeof(out[k].name) - 1);
            out[k].launches = I->prof_n[id];
            out[k].ms_total = I->prof_ms[id];
        }
        ++k;
    }
    *n = k;
    if (reset)
        for (int id = 0; id < K_COUNT; ++id) {
            I->prof_ms[id] = 0.0;
            I->prof_n[id] = 0;
        }
    return EP_OK;
}

ep_status ep_selftest_barrier_timeout(int32_t* status_out) {
    if (!status_out) return fail(EP_EINVAL, "NULL argument");
    int st = 0;
    CUDA_TRY(epk::barrier_timeout_probe(&st));
    *status_out = st;
    return EP_OK;
}

ep_status ep_residual_norm_noalloc(const ep_instance* I, double* relres_out) {
    if (!I || !relres_out) return fail(EP_EINVAL, "NULL argument");
    if (I->h.prec != EP_PREC_FP32_REFINED)
        return fail(EP_EUNSUPPORTED, "the allocation-free residual serves FP32_REFINED instances");
    if (I->h.q2 || I->h.op32 != EP_OP_STENCIL)
        return fail(EP_EUNSUPPORTED, "the allocation-free residual serves instances with the stencil FP32 operator");
    if (I->grid_pcg > epk::noalloc_max_blocks())
        return fail(EP_EINVAL, "the residual of this instance needs " + std::to_string(I->grid_pcg) +
                                   " thread blocks; the allocation-free path holds partial sums for at most " +
                                   std::to_string(epk::noalloc_max_blocks()));
    if (!I->solved)
        return fail(EP_EINVAL, "no linear solve since the instance was created or its state loaded");
    double sums[2] = {0.0, 0.0};
    CUDA_TRY(epk::residual_norm_noalloc(I->d, I->grid_pcg, epk::pcg_threads_of(), I->stream, sums));
    if (!(sums[0] > 0.0))
        return fail(EP_EINVAL, "the last solve's right-hand side is zero: no relative residual");
    *relres_out = std::sqrt(sums[1] / sums[0]);
    return EP_OK;
}

ep_status ep_destroy(ep_instance* I) {
    if (!I) return EP_OK;
    drop_plans_of(I);
    if (I->stream) cudaStreamSynchronize(I->stream);
    free_all(I);
    delete I;
    return EP_OK;
}

}  // extern "C"
