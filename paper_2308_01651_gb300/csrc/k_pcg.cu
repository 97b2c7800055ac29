// k_pcg.cu -- the FP32 inner solve of a refinement sweep in one persistent,
// cooperative launch (stencil operator).
//
// Jacobi-preconditioned CG (the paper solves Eq. (6) with CG, Sec. 2) on
// A delta = r in float, A the hi parts of the node-major full couplings, in
// the single-reduction arrangement of Chronopoulos and Gear (1989): with
// u = D^-1 r and w = A u, both dot products of an iteration come from the
// same pass.  Iteration i, given alpha_i and beta_i:
//   update (every node on its own):
//     s_i = w_i + beta_i s_{i-1},   r_{i+1} = r_i - alpha_i s_i,
//     p_i = u_i + beta_i p_{i-1},   delta  += alpha_i p_i,   u_{i+1} = D^-1 r_{i+1}
//   grid barrier (u_{i+1} of the neighbours is needed next)
//   apply: w_{i+1} = A u_{i+1}; block partials of
//     gamma = (r_{i+1}, u_{i+1}), eta = (u_{i+1}, w_{i+1}), rho = (r_{i+1}, r_{i+1})
//   grid barrier; every block sums all partials in the same fixed order, so
//   all blocks take the same
//     beta_{i+1} = gamma_{i+1} / gamma_i,
//     alpha_{i+1} = gamma_{i+1} / (eta_{i+1} - beta_{i+1} gamma_{i+1} / alpha_i)
//   and the same stopping decision (rho relative to the sweep's first rho).
// The right-hand-side kernel leaves r_0 and u_0 = D^-1 r_0, so the launch
// starts with the apply of u_0.  Nodes are spread over all threads of the
// grid in index order (thread t: nodes t, t + T, ...), so every thread owns
// the same number of nodes up to one.  Neighbour values of u are plain
// cached loads: they were written before the last barrier, whose
// release/acquire pair orders them for every thread of the block.  A barrier
// that does not complete within ~1 s records EP_ETIMEOUT and the kernel
// returns.
#include "ep_dev.cuh"
#include "ep_tile.cuh"

namespace epk {

constexpr long long kBarrierSpinLimit = 1ll << 24;  // x >= 64 ns naps: about a second

// Bounded grid barrier (all blocks of a cooperative launch) on a 64-bit
// arrival counter that only grows: every barrier adds exactly one arrival
// per block, so barrier k of a launch completes when the counter reaches
// base + k G, base being the counter at launch start (a multiple of G).
// Thread 0 of each block arrives with one acq_rel atomic and waits with
// acquire loads; the block's other threads are ordered behind it by
// __syncthreads.  `target` is thread 0's running target (0 before the first
// barrier of the launch).  Returns false after recording EP_ETIMEOUT when the
// other blocks did not all arrive in time.
__device__ __forceinline__ bool grid_barrier(unsigned long long* count, unsigned long long& target, int G,
                                             int* status) {
    __shared__ int ok;
    __syncthreads();
    if (threadIdx.x == 0) {
        int good = 1;
        unsigned long long old;
        asm volatile("atom.add.acq_rel.gpu.u64 %0, [%1], 1;" : "=l"(old) : "l"(count) : "memory");
        const unsigned long long g = (unsigned long long)G;
        target = (target == 0ull ? old - old % g : target) + g;
        long long spins = 0;
        for (;;) {
            unsigned long long cur;
            asm volatile("ld.acquire.gpu.u64 %0, [%1];" : "=l"(cur) : "l"(count) : "memory");
            if (cur >= target) break;
            if (++spins > kBarrierSpinLimit) {
                good = 0;
                atomicCAS(status, (int)EP_OK, (int)EP_ETIMEOUT);
                break;
            }
            __nanosleep(20);
        }
        ok = good;
    }
    __syncthreads();
    return ok != 0;
}

// Block sums of NV float values (warp butterflies, then the warps' sums by
// warp 0 in the same way), written as part[k * G + blockIdx.x].
// u += delta (float-float) on this thread's nodes; kept out of line so that
// its registers do not add to the solver loop's
__device__ __noinline__ void correct_ff_nodes(const Dev& D, int t0, int T) {
    float* __restrict__ uh = D.u_hi;
    float* __restrict__ ul = D.u_lo;
    const float* __restrict__ x = D.d32;
    for (int n = t0; n < D.N; n += T) {
        float h = uh[n], l = ul[n];
        ff_add_f(h, l, x[n], h, l);
        uh[n] = h;
        ul[n] = l;
    }
}

template <int NV>
__device__ __forceinline__ void publish(const float (&v)[NV], float* part, int G, int blk) {
    __shared__ float sh[NV][kMaxBlock / 32];
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

// Totals of all blocks' partials, formed by warp 0 of every block in the same
// fixed order (lane-strided sums, then a butterfly), so every block holds the
// same bits; the result is valid in warp 0 only.
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

__global__ void __launch_bounds__(kPcgThreads, 2) k_pcg32_stencil(Batch B) {
    const Slot S = batch_slot(B);
    Dev& D = *S.D;
    // a batched sweep also visits instances whose refinement has finished
    if (!D.f_outer) return;
    const int N = D.N;
    const size_t NN = (size_t)N;
    const int G = S.nblk;
    const int T = G * blockDim.x;
    const int t0 = S.blk * blockDim.x + threadIdx.x;
    // mesh sizes in registers for the neighbour offsets
    const int nx = D.NX, nxy = D.NX * D.NY, wrap = D.periodic ? D.NX * (D.NY - 1) : 0;
    float* r = D.r32;
    float* u = D.z32;
    float* w = D.q32;
    float* s = D.pa32;
    float* p = D.pb32;
    float* x = D.d32;
    const float* __restrict__ dinv = D.dinv32;
    const unsigned char* __restrict__ flag = D.nflag;
    const float4* __restrict__ A = D.Ahi;
    float* part = reinterpret_cast<float*>(D.partial);
    unsigned long long* bcount = reinterpret_cast<unsigned long long*>(D.counter + CNT_BAR);
    unsigned long long target = 0ull;
    // CG scalars (float, like the solve): formed by thread 0 of every block
    // from the same totals, handed to the block through shared memory
    __shared__ float sc_alpha, sc_beta;
    __shared__ int sc_done, sc_it, sc_nan;
    __shared__ float sc_stop, sc_gam_old, sc_alpha_old, sc_rr, sc_gam;
    if (threadIdx.x == 0) {
        sc_it = 0;
        sc_nan = 0;
        sc_stop = sc_gam_old = sc_alpha_old = sc_rr = sc_gam = 0.f;
    }
    float alpha = 0.f, beta = 0.f;
    bool first = true;
    for (;;) {
        if (!first) {
            // ---- update, node by node
            for (int n = t0; n < N; n += T) {
                const float dv = dinv[n];
                const float r0 = r[n], w0 = w[n], u0 = u[n];
                const float s1 = beta == 0.f ? w0 : fmaf(beta, s[n], w0);
                const float p1 = beta == 0.f ? u0 : fmaf(beta, p[n], u0);
                const float r1 = fmaf(-alpha, s1, r0);
                x[n] = fmaf(alpha, p1, x[n]);
                s[n] = s1;
                p[n] = p1;
                r[n] = r1;
                u[n] = dv * r1;
            }
            if (!grid_barrier(bcount, target, G, &D.status)) break;
        }
        // ---- apply w = A u and the block partials
        float v[3] = {0.f, 0.f, 0.f};  // gamma, eta, rho
        for (int n = t0; n < N; n += T) {
            const NbrOff o = nbr_offsets(nx, nxy, wrap, flag[n]);
            float acc = 0.f;
#pragma unroll
            for (int g = 0; g < kGroups; ++g) {
                const float4 c = A[(size_t)g * NN + n];
                const float cv[4] = {c.x, c.y, c.z, c.w};
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    const int t = 4 * g + q;
                    if (t < 27) acc = fmaf(cv[q], u[n + o.x[t % 3] + o.y[(t / 3) % 3] + o.z[t / 9]], acc);
                }
            }
            w[n] = acc;
            const float rn = r[n], un = u[n];
            v[0] = fmaf(rn, un, v[0]);
            v[1] = fmaf(un, acc, v[1]);
            v[2] = fmaf(rn, rn, v[2]);
        }
        publish<3>(v, part, G, S.blk);
        if (!grid_barrier(bcount, target, G, &D.status)) break;
        if (threadIdx.x < 32) {
            float tt[3];
            gather<3>(part, G, tt);
            if (threadIdx.x == 0) {
                if (!first) ++sc_it;
                const float gam = tt[0], rr = tt[2];
                sc_gam = gam;
                sc_rr = rr;
                if (first) sc_stop = (float)D.inner_stop;
                const bool nan = !(tt[0] == tt[0] && tt[1] == tt[1] && tt[2] == tt[2]);
                sc_nan = nan ? 1 : 0;
                const int done = (nan || rr <= sc_stop || sc_it >= D.max_iter) ? 1 : 0;
                if (!done) {
                    const float b = first ? 0.f : gam / sc_gam_old;
                    const float a = first ? gam / tt[1] : gam / (tt[1] - b * gam / sc_alpha_old);
                    sc_beta = b;
                    sc_alpha = a;
                    sc_gam_old = gam;
                    sc_alpha_old = a;
                }
                sc_done = done;
            }
        }
        __syncthreads();
        if (sc_done) break;
        alpha = sc_alpha;
        beta = sc_beta;
        first = false;
    }
    // the sweep's correction u += delta (float-float), node by node: no
    // neighbour is involved, so it needs no barrier and no launch of its own
    correct_ff_nodes(D, t0, T);
    if (S.blk == 0 && threadIdx.x == 0) {
        D.rz = sc_gam;
        D.rr = sc_rr;
        D.it = sc_it;
        D.it_total += sc_it;
        if (sc_nan && D.status == EP_OK) D.status = EP_ENAN;
    }
}

// blocks of k_pcg32_stencil that fit on one SM at once
int pcg_blocks_per_sm() {
    int occ = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_pcg32_stencil, kPcgThreads, 0) != cudaSuccess)
        return 0;
    return occ;
}

cudaError_t launch_pcg32_batch(const Batch& B, int grid, cudaStream_t s) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(grid);
    cfg.blockDim = dim3(kPcgThreads);
    cfg.dynamicSmemBytes = 0;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, k_pcg32_stencil, B);
}

cudaError_t launch_pcg32(Dev* d, const Dev& h, int grid, cudaStream_t s) {
    return launch_pcg32_batch(single_batch(d), grid, s);
}

}  // namespace epk
