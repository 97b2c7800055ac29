// ep_dev.cuh -- device-side instance descriptor and shared helpers of the
// GB300 monodomain step library (see include/ep.h for the ABI).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/ep.h"

namespace epk {

// Symmetric 27-point stencil of a structured Q1 mesh, stored as the diagonal
// (slot 0) and the 13 "forward" neighbour couplings (slots 1..13) of every
// node; the 13 backward couplings of node n are the forward couplings stored
// at its neighbours.  Offset t = (di+1) + 3 (dj+1) + 9 (dk+1) in 0..26, the
// centre is t = 13; forward offsets are t > 13 (slot t - 13), a backward
// offset t < 13 is slot 13 - t of the neighbour n + off(t).
constexpr int kSlots = 14;

constexpr int kTTGates = 13;  // m h j xr1 xr2 xs s r d f f2 fCass RR
constexpr int kTTConc = 5;    // Cai CaSR CaSS Nai Ki
constexpr int kBOStates = 3;  // v w s
// Refined ionic states, one time level: packed four to a 16-byte group,
// group-major ([G][N] float4), so that a thread moves its node's state with G
// 128-bit accesses.  TTP06 (G = 6): slots 0..12 the gates, 13..17 the
// concentrations' float-float hi parts, 18..22 their lo parts, 23 unused.
// Bueno-Orovio (G = 1): v, w, s, unused.
constexpr int kTTPacked = 6;
constexpr int kBOPacked = 1;

// largest block of a reducing kernel (power of two)
constexpr int kMaxBlock = 512;
// threads per block of the node-wise kernels
constexpr int kNodeThreads = 256;
constexpr int kNodesPerThread = 4;
// threads per block of the ionic kernels (one node per thread; 128-thread
// blocks schedule the register-heavy TTP06 step better than 256 at the same
// occupancy)
constexpr int kIonicThreads = 128;
// threads per block of the node-parallel residual (two blocks per SM at 64
// registers; measured faster than four of 256 or eight of 128)
constexpr int kResidThreads = 512;
constexpr int kNodeTile = kNodeThreads * kNodesPerThread;
// tiled stencil kernels: owned tile kStTx x kStTy x kStTz, threads per block
constexpr int kStTx = 32, kStTy = 4, kStTz = 4;
constexpr int kStThreads = 512;  // one owned node per thread
// upper bound of a persistent grid (partial-sum buffers are sized for it)
constexpr int kMaxPersistentBlocks = 2048;

constexpr int kPcgThreads = 512;  // block of the persistent inner solver

// Matrix-free FP32 tile (owned nodes per block): 32 x 8 x 4
constexpr int kMfTx = 32, kMfTy = 8, kMfTz = 4;
constexpr int kMfThreads = 256;

struct Dev {
    // ---- mesh ---------------------------------------------------------
    int kind;
    int nx, ny, nz;      // elements
    int NX, NY, NZ;      // nodes per direction (NY = ny for the periodic shell)
    int periodic;        // j periodic
    int N;               // nodes
    double h[3];         // slab spacing (cm)
    // ---- model / time -----------------------------------------------------
    int model;
    int prec;            // EP_PREC_*
    int bdf;
    int ns;              // ionic states (3 BO, 18 TTP06)
    double dt;
    double inv_dt;       // 1/dt (no FP64 division in the kernels)
    double act_thr;      // activation slope threshold, model units per ms
    long long step;      // current time level n
    // ---- stimulus ------------------------------------------------------------
    int npulses;
    double amp[EP_MAX_PULSES];
    long long k0[EP_MAX_PULSES], kd[EP_MAX_PULSES], kp[EP_MAX_PULSES];
    const uint8_t* mask[EP_MAX_PULSES];
    const double* wgt64[EP_MAX_PULSES];  // pulse profiles (FP64 path; NULL: mask)
    const float* wgt32[EP_MAX_PULSES];   // pulse profiles (refined path)
    // pulses on element regions: their Gauss-integrated vectors (per unit
    // amplitude), added to b in the right-hand-side kernels (FP64; refined:
    // float-float hi, lo); NULL for nodal pulses
    const double* eg64[EP_MAX_PULSES];
    const float* egh[EP_MAX_PULSES];
    const float* egl[EP_MAX_PULSES];
    // ---- state ---------------------------------------------------------------
    double *u_n, *u_nm1, *u_new;
    double* u_nm2;              // level n-2 (BDF3 instances only, else NULL)
    float *g32_n, *g32_nm1;     // FP32_REFINED: every state, packed ([G][N] float4, see kTTPacked)
    float* g32_nm2;             // level n-2 (BDF3)
    double *s64_n, *s64_nm1;    // FP64: all states [ns][N] in double (NULL when refined)
    double* s64_nm2;            // level n-2 of the same (BDF3)
    const uint8_t* cell;
    const uint8_t* active;      // per node, 0 = excluded from the simulation (NULL: all active)
    double *v;                  // u_BDF/dt - I_ion + I_app (FP64 path)
    double *b, *r;              // FP64 right-hand side and residual (FP64 path)
    // refined path, float-float (hi, lo): the solve's iterate u (starts at
    // u_EXT), the nodal vector v and the right-hand side b = M v
    float *u_hi, *u_lo, *v_hi, *v_lo, *b_hi, *b_lo;
    float nscale;               // scale of b and r in the float sums of squares
    float mw_hi, mw_lo;         // slab mass weight hx hy hz / 216 (float-float)
    float idt_hi, idt_lo;       // 1/dt (float-float)
    // refined path: the potential of steps n and n-1 as float-float pairs
    // (u_n and u_nm1 hold the same values rounded to double), and the
    // activation's best slope per node in float
    float *uh_n, *ul_n, *uh_m, *ul_m;
    float *uh_m2, *ul_m2;       // level n-2 (BDF3)
    float* bestf;
    // A u of the solve's iterate (float-float): the current step's (written by
    // every residual evaluation, the first one included), step n's, step
    // n-1's (and, BDF3, step n-2's).  hist counts the valid past levels; with
    // enough of them A u_EXT is their BDF extrapolation instead of an
    // operator apply.
    float *yc_hi, *yc_lo, *yn_hi, *yn_lo, *ym_hi, *ym_lo;
    float *ym2_hi, *ym2_lo;     // step n-2's (BDF3)
    int hist;
    // 1 from the end of a refined step until the next step's right-hand
    // side: the ionic kernel then does the previous step's per-node end
    int fin_pending;
    double *at, *best;
    // ---- operators -----------------------------------------------------------
    double *M64, *A64;          // [kSlots][N] (symmetric, FP64)
    double *dinv64;
    // refined path: the symmetric stencils as float-float pairs (hi parts,
    // lo parts), in the slots of the FP64 stencils -- slot 0 the diagonal,
    // slot s = 1..13 the coupling to the forward neighbour t = 13 + s --
    // with slot s of node n at s * cs + n; the FP32 inner operator is Ahi.
    // Every slot is followed by at least 1 + NX + NX NY zeros (the largest
    // backward offset), so a backward-neighbour read of slot s >= 1 below
    // node 0 returns 0 (see ep_tile.cuh).
    float *Ahi, *Alo, *Mhi, *Mlo;
    long long cs;               // slot stride of the coupling arrays (floats)
    float *dinv32;
    float *fib;                 // [6][N]: f0/h, s0/h per component (matrix-free)
    // ---- triquadratic slab (EP_MESH_SLAB_Q2): matrix-free operators -----------
    int q2;                     // 1: 27-node hexahedra (nodes on the half-element grid)
    int enx, eny, enz, ne;      // elements per direction, in total
    double q2vol;               // element volume hx hy hz
    const float* q2G;           // [2][6][ne * 27]: hi, then lo parts of the quadrature
                                // point flux matrices w_q |J| H D(q) H (xx yy zz xy xz yz)
    const float* q2G32;         // [6][27][ne]: the hi parts again, element fastest (FP32 apply)
    float* q2Y32;               // [8][N] element outputs of the FP32 apply in node slots
    float *q2Yh, *q2Yl;         // [8][N] element outputs of A u in node slots (float-float)
    float *q2Bh, *q2Bl;         // [8][N] element outputs of M v in node slots (float-float)
    double *q2dM, *q2dK;        // diagonals of M and K
    float mf_cn[3], mf_cl, mf_ct, mf_cmass;
    double alpha_dt;            // alpha_BDF/dt the operators currently hold
    int op32;                   // EP_OP_MATRIX_FREE or EP_OP_STENCIL
    // ---- CG ------------------------------------------------------------------
    float *r32, *z32, *q32, *d32, *pa32, *pb32;
    int npad;                   // z32 has npad zero floats before and after it (Q1 meshes)
    // tiled apply of the persistent solve (k_pcg.cu): a block's tile is
    // tile_by rows of j (every i) over a range of k planes, tile_jt tiles
    // across j times tile_kr ranges of k; its planes staged in shared memory,
    // tile_l floats per slot and plane (the tile's rows, a row of halo on
    // either side, slack and alignment)
    int tile_by, tile_jt, tile_kr, tile_l;
    unsigned char* nflag;       // boundary flags per node (bits: i=0, i=NX-1, j=0, j=NY-1, k=0, k=NZ-1)
    double *z64, *q64, *pa64, *pb64;
    double rz, pq, alpha, beta, rr, rr0, bb, relres;
    double tol, inner_tol;
    // the inner solve's stop on r32 . r32: below (0.9 tol ||b||)^2, enough
    // for the sweep to end the refinement, or below inner_tol^2 times its
    // initial value (the float floor), whichever is larger
    double inner_stop;
    int max_iter, max_sweeps;
    int it, it_total, sweeps;
    int pswap;                  // 0: p_old = pa, p_new = pb; 1: swapped
    int status;                 // ep_status of the running step (sticky)
    int last_iters, last_sweeps;
    double last_relres;
    long long done_step;
    // ---- reductions --------------------------------------------------------
    double* partial;            // per-block partial sums
    unsigned int* counter;      // last-block counters, one per kernel kind
    unsigned long long h_loop;  // conditional handles (cudaGraphConditionalHandle)
    unsigned long long h_inner;
    unsigned long long h_outer;
    int f_loop, f_inner, f_outer;  // the same loop decisions, for host-driven stepping
};

// Inputs of the create-time assembly kernel.
struct AsmParams {
    const double* xyz;  // shell coordinates [N][3] (NULL for slabs)
    const double* f0;   // [N][3]
    const double* s0;   // [N][3]
    double dl, dt, dn;  // diffusivities (cm^2/ms), one region
    double alpha_dt;    // alpha/dt of the system matrix A = alpha/dt M + K
    int* bad;           // set to 1 on a non-positive Jacobian determinant
    // subdomains: element labels (NULL: one region with dl, dt, dn), the
    // diffusivities of each region and its exclusion flag
    const uint8_t* label;
    double rd[EP_MAX_REGIONS][3];
    int excl[EP_MAX_REGIONS];
};

// Counter slots (one per reducing kernel so that consecutive kernels never
// share a counter).
// CNT_BAR and CNT_BAR + 1: the 64-bit arrival counter of the persistent
// solver's grid barrier (8-byte aligned: the array is 256-byte aligned).
enum { CNT_RHS = 0, CNT_APPLY = 1, CNT_UPDATE = 2, CNT_RESID = 3, CNT_FINISH = 4, CNT_BAR = 6, CNT_N = 8 };

// ---------------------------------------------------------------- helpers --

__device__ __forceinline__ float warp_sum(float v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Block sums of NV float values (warp butterflies, then the warps' sums by
// warp 0 in the same way), written as part[k * G + blk].  (Block-wide
// __syncthreads inside.)
template <int NV>
__device__ __forceinline__ void publish(const float (&v)[NV], float* part, int G, int blk) {
    __shared__ float sh[NV][32];  // one per warp, up to 1024-thread blocks
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarp = blockDim.x >> 5;
#pragma unroll
    for (int k = 0; k < NV; ++k) {
        const float s = warp_sum(v[k]);
        if (lane == 0) sh[k][warp] = s;
    }
    __syncthreads();
    if (warp == 0) {
#pragma unroll
        for (int k = 0; k < NV; ++k) {
            const float s = warp_sum(lane < nwarp ? sh[k][lane] : 0.f);
            if (lane == 0) part[(size_t)k * G + blk] = s;
        }
    }
}

// Totals of G blocks' partials, formed by warp 0 in a fixed order
// (lane-strided sums, then a butterfly), so every block that forms them holds
// the same bits; the result is valid in warp 0 only.
template <int NV>
__device__ __forceinline__ void gather(const float* part, int G, float (&tot)[NV]) {
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int k = 0; k < NV; ++k) {
        float acc = 0.f;
        for (int i = lane; i < G; i += 32) acc += __ldcg(&part[(size_t)k * G + i]);
        tot[k] = warp_sum(acc);
    }
}

// Shared-memory tree sum of sh[k][0..n) into sh[k][0] (n a power of two equal
// to blockDim.x).  n - 1 additions per row: on GB300 the FP64 pipe is ~60x
// slower than FP32, and a warp-shuffle tree would spend 5 x 32 additions per
// warp instead of 31.
template <int R>
__device__ __forceinline__ void tree_sum(double (*sh)[kMaxBlock], int n) {
    for (int s = n >> 1; s > 0; s >>= 1) {
        if ((int)threadIdx.x < s) {
#pragma unroll
            for (int k = 0; k < R; ++k) sh[k][threadIdx.x] += sh[k][threadIdx.x + s];
        }
        __syncthreads();
    }
}

// Grid-wide sums of NF float and ND double per-thread values.  Float values
// are summed by warp shuffles and then over the block's warps (in float, fixed
// order); double values by a shared-memory tree.  Every block writes its
// NF + ND sums (as double) to partial[blk*(NF+ND) + k]; the last block to
// arrive (global atomic counter) adds all partials in double, in a fixed
// order, and runs finish(totals) with thread 0 (totals: the NF float sums
// first, then the ND double sums).  Deterministic: the result does not depend
// on which block arrives last.  No block waits on another.  blockDim.x must
// be a power of two <= kMaxBlock.
template <int NF, int ND, class F>
__device__ void grid_reduce(const float (&vf)[NF > 0 ? NF : 1], const double (&vd)[ND > 0 ? ND : 1],
                            double* partial, unsigned int* counter, int blk, int nblk, F finish) {
    constexpr int NV = NF + ND;
    __shared__ double sh[NV][kMaxBlock];
    __shared__ float shf[NF > 0 ? NF : 1][32];
    __shared__ bool last;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int nwarp = (blockDim.x + 31) >> 5;
#pragma unroll
    for (int k = 0; k < NF; ++k) {
        const float s = warp_sum(vf[k]);
        if (lane == 0) shf[k][warp] = s;
    }
#pragma unroll
    for (int k = 0; k < ND; ++k) sh[k][threadIdx.x] = vd[k];
    __syncthreads();
    if constexpr (ND > 0) tree_sum<ND>(sh, blockDim.x);
    if (threadIdx.x == 0) {
#pragma unroll
        for (int k = 0; k < NF; ++k) {
            float s = 0.f;
            for (int w = 0; w < nwarp; ++w) s += shf[k][w];
            partial[(size_t)blk * NV + k] = (double)s;
        }
#pragma unroll
        for (int k = 0; k < ND; ++k) partial[(size_t)blk * NV + NF + k] = sh[k][0];
        __threadfence();
        const unsigned int t = atomicAdd(counter, 1u);
        last = (t == (unsigned int)(nblk - 1));
    }
    __syncthreads();
    if (!last) return;
    __threadfence();
#pragma unroll
    for (int k = 0; k < NV; ++k) {
        double acc = 0.0;
        for (int i = threadIdx.x; i < nblk; i += blockDim.x) acc += __ldcg(&partial[(size_t)i * NV + k]);
        sh[k][threadIdx.x] = acc;
    }
    __syncthreads();
    tree_sum<NV>(sh, blockDim.x);
    if (threadIdx.x == 0) {
        double tot[NV];
#pragma unroll
        for (int k = 0; k < NV; ++k) tot[k] = sh[k][0];
        *counter = 0u;
        finish(tot);
        __threadfence();
    }
}

// Records a loop decision in the descriptor (read by host-driven stepping)
// and, when h != 0, in the graph's conditional node.  Kernels pass h = 0
// unless they were launched as nodes of the step graph: setting a handle
// from a kernel outside its graph is undefined.
__device__ __forceinline__ void set_cond(unsigned long long h, int* flag, unsigned int v) {
    *flag = (int)v;
    if (h) cudaGraphSetConditional((cudaGraphConditionalHandle)h, v);
}

// ---- batched launches -------------------------------------------------------
// One launch may serve several instances: its blocks are split into
// consecutive ranges, start[i] .. start[i+1]-1 for instance i, and every block
// works on its instance alone with the block index and count of its range --
// the same values a launch of that instance alone would use, so per-instance
// results do not depend on what else is in the launch.  n == 1 is a plain
// single-instance launch (d0, whole grid).
struct Batch {
    Dev* d0;            // n == 1
    Dev* const* devs;   // n > 1: device array of the instances' descriptors
    const int* start;   // n > 1: device array, n + 1 entries
    int n;
};

struct Slot {
    Dev* D;
    int blk, nblk;
};

__device__ __forceinline__ Slot batch_slot(const Batch& B) {
    if (B.n <= 1) return Slot{B.d0, (int)blockIdx.x, (int)gridDim.x};
    const int b = blockIdx.x;
    int lo = 0, hi = B.n - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (B.start[mid] <= b) lo = mid;
        else hi = mid - 1;
    }
    return Slot{B.devs[lo], b - B.start[lo], B.start[lo + 1] - B.start[lo]};
}

inline Batch single_batch(Dev* d) { return Batch{d, nullptr, nullptr, 1}; }

// Amplitude of pulse p on the step about to run (new level m = step + 1):
// active when k0 < m <= k0 + kd, repeating every kp steps when kp > 0.
__device__ __forceinline__ double pulse_amp(const Dev& D, int p) {
    const long long m = D.step + 1;
    if (p >= D.npulses || m <= D.k0[p]) return 0.0;
    long long rel = m - D.k0[p] - 1;
    if (D.kp[p] > 0) rel %= D.kp[p];
    return rel < D.kd[p] ? D.amp[p] : 0.0;
}

// BDF order of the step about to run: the scheme's order, ramping 1, 2, 3
// over the first steps.
__host__ __device__ __forceinline__ int bdf_order(const Dev& D) {
    return D.bdf < D.step + 1 ? D.bdf : (int)(D.step + 1);
}

// 1/3 as a float-float pair
constexpr float kThirdHi = 0.333333343267f;
constexpr float kThirdLo = -9.93410748e-9f;

// End of a step (one thread, after the step's last reduction): rotation of
// the time levels by pointer swaps (potentials, ionic states; refined: the
// float-float potential levels and the A u history), the step counter and
// the per-step statistics.
__device__ __forceinline__ void end_of_step(Dev& D) {
    // potentials (double): new -> n -> n-1 (-> n-2), the oldest buffer
    // takes the next step's new level
    double* t = D.u_nm2 ? D.u_nm2 : D.u_nm1;
    if (D.u_nm2) D.u_nm2 = D.u_nm1;
    D.u_nm1 = D.u_n;
    D.u_n = D.u_new;
    D.u_new = t;
    // states: the new level was written into the oldest slot
    if (D.g32_nm2) {
        float* g = D.g32_nm2;
        D.g32_nm2 = D.g32_nm1;
        D.g32_nm1 = D.g32_n;
        D.g32_n = g;
    } else {
        float* g = D.g32_nm1;
        D.g32_nm1 = D.g32_n;
        D.g32_n = g;
    }
    if (D.s64_nm2) {
        double* c = D.s64_nm2;
        D.s64_nm2 = D.s64_nm1;
        D.s64_nm1 = D.s64_n;
        D.s64_n = c;
    } else {
        double* c = D.s64_nm1;
        D.s64_nm1 = D.s64_n;
        D.s64_n = c;
    }
    if (D.u_hi) {
        // the iterate becomes level n, level n becomes n-1 (and n-1 n-2),
        // and the oldest buffers take the next step's iterate
        float* ph = D.uh_m2 ? D.uh_m2 : D.uh_m;
        float* pl = D.ul_m2 ? D.ul_m2 : D.ul_m;
        if (D.uh_m2) {
            D.uh_m2 = D.uh_m;
            D.ul_m2 = D.ul_m;
        }
        D.uh_m = D.uh_n;
        D.ul_m = D.ul_n;
        D.uh_n = D.u_hi;
        D.ul_n = D.u_lo;
        D.u_hi = ph;
        D.u_lo = pl;
        // A u of the new solution becomes step n's; the oldest level is
        // reused for the next step's residuals
        float* yh = D.ym2_hi ? D.ym2_hi : D.ym_hi;
        float* yl = D.ym2_lo ? D.ym2_lo : D.ym_lo;
        if (D.ym2_hi) {
            D.ym2_hi = D.ym_hi;
            D.ym2_lo = D.ym_lo;
        }
        D.ym_hi = D.yn_hi;
        D.ym_lo = D.yn_lo;
        D.yn_hi = D.yc_hi;
        D.yn_lo = D.yc_lo;
        D.yc_hi = yh;
        D.yc_lo = yl;
        const int hmax = D.ym2_hi ? 3 : 2;
        D.hist = D.hist < hmax ? D.hist + 1 : hmax;
        D.fin_pending = 1;
    }
    D.step += 1;
    D.done_step = D.step;
    D.last_iters = D.prec == EP_PREC_FP32_REFINED ? D.it_total : D.it;
    D.last_sweeps = D.prec == EP_PREC_FP32_REFINED ? D.sweeps : 0;
    D.last_relres = D.relres;
}

// Node (i, j, k) of index n, and the neighbour at offset slot t (0..26);
// returns -1 where the neighbour does not exist.
__device__ __forceinline__ void node_ijk(const Dev& D, int n, int& i, int& j, int& k) {
    const int nxy = D.NX * D.NY;
    k = n / nxy;
    const int rem = n - k * nxy;
    j = rem / D.NX;
    i = rem - j * D.NX;
}

__device__ __forceinline__ int neighbour(const Dev& D, int i, int j, int k, int di, int dj, int dk) {
    const int ii = i + di, kk = k + dk;
    int jj = j + dj;
    if (ii < 0 || ii >= D.NX || kk < 0 || kk >= D.NZ) return -1;
    if (D.periodic) {
        jj = jj < 0 ? jj + D.NY : (jj >= D.NY ? jj - D.NY : jj);
    } else if (jj < 0 || jj >= D.NY) {
        return -1;
    }
    return ii + D.NX * (jj + D.NY * kk);
}

}  // namespace epk
