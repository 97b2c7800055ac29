// k_pcg.cu -- the whole linear solve of a step, every refinement sweep, in
// one persistent, cooperative launch (stencil operator): the FP32 inner solve,
// the correction and the float-float residual with the refinement's decision.
//
// Jacobi-preconditioned CG (the paper solves Eq. (6) with CG, Sec. 2) on
// A delta = r in float, A the hi parts of the symmetric float-float stencil, in
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
// release/acquire pair orders them for every thread of the block; on a Q1
// slab u is padded with zeros, so rows read their neighbours at fixed
// offsets without the boundary flags.  A barrier that does not complete
// within ~1 s records EP_ETIMEOUT and the kernel returns.
//
// A pipelined arrangement (Ghysels and Vanroose 2014: w and z = A D^-1 s by
// recurrence, one pass and one barrier per iteration) measured the same on
// the 442k-node slab (331 against 333 us a step's solve) and slower on the
// LV shell, where the float recurrences slowed convergence (100 inner
// iterations a sweep against 36); it is not used.
//
// After the inner solve: u += delta (float-float), a grid barrier, then the
// residual of the sweep on the same node map -- y = A u with the float-float
// couplings, r = b - y, the next inner solve's start (r, D^-1 r, delta = 0) --
// and its sums (ns b)^2, (ns r)^2, r . D^-1 r, r . r, reduced like the CG's
// (block partials, every block summing them in the same order), so every
// block takes the same decision: the refinement has converged when
// ||r|| <= tol ||b||, else another sweep follows (at most max_sweeps); block 0
// records the step's figures and, at the end, rotates the time levels.  The
// inner solve's couplings are then still in L2 for the residual's hi parts.
#include "ep_dev.cuh"
#include "ep_ff.cuh"
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
                                             int* status, long long spin_limit = kBarrierSpinLimit) {
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
            if (++spins > spin_limit) {
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

// The sweep's float-float residual on this thread's nodes: y = A u with
// the hi and lo couplings (stored as the step's A u), r = b - y, the next
// inner solve's start (r32 = r, z32 = D^-1 r32, delta = 0), and this
// thread's sums (ns b)^2, (ns r)^2, r32 . z32, r32 . r32.  Out of line, as
// correct_ff_nodes.
__device__ __noinline__ void resid_ff_nodes(const Dev& D, int t0, int T, float (&vf)[4]) {
    const int N = D.N;
    const int nx = D.NX, nxy = D.NX * D.NY, wrap = D.periodic ? D.NX * (D.NY - 1) : 0;
    const float ns = D.nscale;
    const float* __restrict__ uh = D.u_hi;
    const float* __restrict__ ul = D.u_lo;
    vf[0] = vf[1] = vf[2] = vf[3] = 0.f;
    const unsigned char* __restrict__ flag = D.nflag;
    unsigned int fn = t0 < N ? flag[t0] : 0u;
    for (int n = t0; n < N; n += T) {
        const unsigned int f = fn;
        fn = n + T < N ? flag[n + T] : 0u;
        const NbrOff o = nbr_offsets(nx, nxy, wrap, f);
        float ah, al, rh, rl;
        row_ff_sym(D.Ahi, D.Alo, D.cs, uh, ul, n, o, exist_flags(f, wrap), ah, al);
        D.yc_hi[n] = ah;
        D.yc_lo[n] = al;
        const float bh = D.b_hi[n];
        ff_sub(bh, D.b_lo[n], ah, al, rh, rl);
        const float r32 = rh;
        const float z = D.dinv32[n] * r32;
        D.r32[n] = r32;
        D.z32[n] = z;
        D.d32[n] = 0.0f;
        const float bs = ns * bh, rs = ns * rh;
        vf[0] = fmaf(bs, bs, vf[0]);
        vf[1] = fmaf(rs, rs, vf[1]);
        vf[2] = fmaf(r32, z, vf[2]);
        vf[3] = fmaf(r32, r32, vf[3]);
    }
}

// BT threads per block, MINB resident blocks per SM.  An instance alone runs
// one 1024-thread block per SM (64 registers, 32 warps in flight, 152
// arrivals at each grid barrier); measured against one 512-thread block
// (128 registers, 16 warps) and two of them (64 registers, 304 arrivals) a
// step's solve took 249.5 / 255.0 / 277.3 us on the 442k-node slab and
// 2086 / 2373 / 2108 us on the 2.19M-node LV shell.  Batches run the same
// 1024-thread blocks, shared among their instances by size (so an instance
// rounds alike alone and in a batch, to its share of blocks).
template <int BT, int MINB, bool HINT>
__global__ void __launch_bounds__(BT, MINB) k_solve32_stencil(Batch B) {
    const Slot S = batch_slot(B);
    Dev& D = *S.D;
    // the step's first residual may already meet the tolerance; a batched
    // launch also visits such instances
    if (!D.f_outer) return;
    const int N = D.N;
    const int G = S.nblk;
    const int T = G * blockDim.x;
    const int t0 = S.blk * blockDim.x + threadIdx.x;
    // mesh sizes in registers for the neighbour offsets
    const int nx = D.NX, nxy = D.NX * D.NY, wrap = D.periodic ? D.NX * (D.NY - 1) : 0;
    float* __restrict__ r = D.r32;
    float* __restrict__ w = D.q32;
    float* __restrict__ s = D.pa32;
    float* __restrict__ p = D.pb32;
    float* __restrict__ x = D.d32;
    const float* __restrict__ dinv = D.dinv32;
    const unsigned char* __restrict__ flag = D.nflag;
    // Q1 slab: u is padded, so every row reads its 27 neighbours at fixed
    // offsets (couplings past the slab's edge are 0) and the boundary flags
    // are not needed
    const bool fixed = D.npad > 0 && wrap == 0;
    const float* __restrict__ A = D.Ahi;
    const long long cs = D.cs;
    // HINT (working set beyond L2): the CG vectors kept in L2, the couplings
    // streamed; otherwise plain accesses (an L2-resident instance gains
    // nothing and its couplings would be dropped first)
    const unsigned long long pkeep = HINT ? l2_policy_evict_last() : 0ull;
    const unsigned long long pstream = HINT ? l2_policy_evict_first() : 0ull;
    auto ldv = [&](const float* a) { return HINT ? ld_pol(a, pkeep) : *a; };
    auto stv = [&](float* a, float v) {
        if (HINT) st_pol(a, v, pkeep);
        else *a = v;
    };
    float* part = reinterpret_cast<float*>(D.partial);
    unsigned long long* bcount = reinterpret_cast<unsigned long long*>(D.counter + CNT_BAR);
    unsigned long long target = 0ull;
    // CG scalars (float, like the solve): formed by thread 0 of every block
    // from the same totals, handed to the block through shared memory
    __shared__ float sc_alpha, sc_beta;
    __shared__ int sc_done, sc_it, sc_nan, sc_more, sc_sweeps, sc_itsum;
    __shared__ float sc_stop, sc_gam_old, sc_alpha_old, sc_rr, sc_gam;
    if (threadIdx.x == 0) {
        sc_it = 0;
        sc_nan = 0;
        sc_sweeps = 0;
        sc_itsum = 0;
        sc_stop = (float)D.inner_stop;  // the first sweep's, from the right-hand side
        sc_gam_old = sc_alpha_old = sc_rr = sc_gam = 0.f;
    }
    __syncthreads();
    bool aborted = false;
    for (;;) {  // ---- refinement sweeps
        float alpha = 0.f, beta = 0.f;
        bool first = true;
        if (threadIdx.x == 0) sc_it = 0;
        float* __restrict__ u = D.z32;
        for (;;) {  // ---- inner CG: an update pass and an apply pass per iteration
            if (!first) {
                // ---- update, node by node
                for (int n = t0; n < N; n += T) {
                    const float dv = ldv(dinv + n);
                    const float r0 = ldv(r + n), w0 = ldv(w + n), u0 = ldv(u + n);
                    const float s1 = beta == 0.f ? w0 : fmaf(beta, ldv(s + n), w0);
                    const float p1 = beta == 0.f ? u0 : fmaf(beta, ldv(p + n), u0);
                    const float r1 = fmaf(-alpha, s1, r0);
                    stv(x + n, fmaf(alpha, p1, ldv(x + n)));
                    stv(s + n, s1);
                    stv(p + n, p1);
                    stv(r + n, r1);
                    stv(u + n, dv * r1);
                }
                if (!grid_barrier(bcount, target, G, &D.status)) {
                    aborted = true;
                    break;
                }
            }
            // ---- apply w = A u and the block partials
            float v[3] = {0.f, 0.f, 0.f};  // gamma, eta, rho
            unsigned int fn = (!fixed && t0 < N) ? flag[t0] : 0u;
            for (int n = t0; n < N; n += T) {
                // the next node's flags load while this node's row runs
                const unsigned int f = fn;
                fn = (!fixed && n + T < N) ? flag[n + T] : 0u;
                const NbrOff o = nbr_offsets(nx, nxy, wrap, f);
                // fixed offsets: no mask, see the symmetric stencils' layout
                const float acc = HINT ? row32_sym_pol(A, cs, u, n, o, exist_flags(f, wrap), pstream, pkeep)
                                       : row32_sym<true>(A, cs, u, n, o, exist_flags(f, wrap));
                stv(w + n, acc);
                const float rn = ldv(r + n), un = ldv(u + n);
                v[0] = fmaf(rn, un, v[0]);
                v[1] = fmaf(un, acc, v[1]);
                v[2] = fmaf(rn, rn, v[2]);
            }
            publish<3>(v, part, G, S.blk);
            if (!grid_barrier(bcount, target, G, &D.status)) {
                aborted = true;
                break;
            }
            if (threadIdx.x < 32) {
                float tt[3];
                gather<3>(part, G, tt);
                if (threadIdx.x == 0) {
                    if (!first) ++sc_it;
                    const float gam = tt[0], rr = tt[2];
                    sc_gam = gam;
                    sc_rr = rr;
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
        if (aborted) break;
        // the sweep's correction u += delta (float-float), node by node
        correct_ff_nodes(D, t0, T);
        if (!grid_barrier(bcount, target, G, &D.status)) break;  // neighbours' u below
        // ---- the sweep's residual and the next inner solve's start
        {
            float vf[4];
            resid_ff_nodes(D, t0, T, vf);
            publish<4>(vf, part, G, S.blk);
        }
        if (!grid_barrier(bcount, target, G, &D.status)) break;
        if (threadIdx.x < 32) {
            float tt[4];
            gather<4>(part, G, tt);
            if (threadIdx.x == 0) {
                sc_itsum += sc_it;
                sc_sweeps += 1;
                const double bb = tt[0], rr = tt[1];
                const bool nan = !(rr == rr);
                const bool conv = !nan && rr <= D.tol * D.tol * bb;
                const bool more = !conv && !nan && sc_sweeps < D.max_sweeps;
                // the next inner solve's stop: (0.9 tol ||b||)^2 in float
                // units, or the float floor inner_tol^2 x its first r . r
                const double ns2 = (double)D.nscale * (double)D.nscale;
                const double target2 = 0.81 * D.tol * D.tol * (bb / ns2);
                const double floor2 = D.inner_tol * D.inner_tol * (double)tt[3];
                sc_stop = (float)(target2 > floor2 ? target2 : floor2);
                sc_more = more ? 1 : 0;
                if (S.blk == 0) {
                    // the step's figures (block 0 only; the other blocks
                    // read none of these fields)
                    D.bb = bb;
                    D.relres = bb > 0.0 ? sqrt(rr / bb) : sqrt(rr);
                    D.rr0 = tt[3];
                    D.rr = tt[3];
                    D.rz = tt[2];
                    D.sweeps = sc_sweeps;
                    D.it = sc_it;
                    D.it_total += sc_it;
                    if (nan && D.status == EP_OK) D.status = EP_ENAN;
                    if (sc_nan && D.status == EP_OK) D.status = EP_ENAN;
                    if (!conv && !more && !nan && D.status == EP_OK) D.status = EP_ENOCONV;
                    if (!more) {
                        D.f_outer = 0;
                        end_of_step(D);
                    }
                }
            }
        }
        __syncthreads();
        if (!sc_more) break;
    }
}

// Self-test of the bounded wait: one block enters a barrier of a grid of
// two, whose other block never comes (a flag that nothing sets).  The spin
// gives up after spin_limit naps, records EP_ETIMEOUT in *status and the
// kernel returns; nothing faults and the context stays usable.
__global__ void k_barrier_probe(unsigned long long* count, int* status, long long spin_limit) {
    unsigned long long target = 0ull;
    (void)grid_barrier(count, target, 2, status, spin_limit);
}

cudaError_t barrier_timeout_probe(int* status_out) {
    void* mem = nullptr;
    cudaError_t e = cudaMalloc(&mem, 64);
    if (e != cudaSuccess) return e;
    unsigned long long* count = static_cast<unsigned long long*>(mem);
    int* status = reinterpret_cast<int*>(static_cast<char*>(mem) + 32);
    e = cudaMemset(mem, 0, 64);
    if (e == cudaSuccess) {
        k_barrier_probe<<<1, 32>>>(count, status, 1ll << 16);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaDeviceSynchronize();
    if (e == cudaSuccess) e = cudaMemcpy(status_out, status, sizeof(int), cudaMemcpyDeviceToHost);
    cudaFree(mem);
    return e;
}

// Launch shapes of the persistent solve: 1 = one 512-thread block per SM
// (128 registers), 2 = two 512-thread blocks per SM (64 registers), 3 = one
// 1024-thread block per SM (64 registers, the arrivals of shape 1 with the
// warps of shape 2).  Blocks of the shape that fit on one SM at once.
int pcg_blocks_per_sm(int shape) {
    int occ = 0;
    cudaError_t e;
    if (shape == 3)
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_solve32_stencil<1024, 1, false>, 1024, 0);
    else if (shape == 2)
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_solve32_stencil<512, 2, false>, 512, 0);
    else
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_solve32_stencil<512, 1, false>, 512, 0);
    return e == cudaSuccess ? occ : 0;
}

int pcg_threads_of(int shape) { return shape == 3 ? 1024 : 512; }

template <int BT, int MINB, bool HINT>
cudaError_t launch_solve(const Batch& B, int grid, cudaStream_t s) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(grid);
    cfg.blockDim = dim3(BT);
    cfg.dynamicSmemBytes = 0;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, k_solve32_stencil<BT, MINB, HINT>, B);
}

// hint: the solve's working set exceeds L2 (L2 eviction-priority policies)
cudaError_t launch_pcg32_batch(const Batch& B, int grid, int hint, cudaStream_t s) {
    return hint ? launch_solve<1024, 1, true>(B, grid, s) : launch_solve<1024, 1, false>(B, grid, s);
}

cudaError_t launch_pcg32(Dev* d, const Dev& h, int grid, int shape, int hint, cudaStream_t s) {
    const Batch B = single_batch(d);
    if (shape == 3)
        return hint ? launch_solve<1024, 1, true>(B, grid, s) : launch_solve<1024, 1, false>(B, grid, s);
    if (shape == 2)
        return hint ? launch_solve<512, 2, true>(B, grid, s) : launch_solve<512, 2, false>(B, grid, s);
    return hint ? launch_solve<512, 1, true>(B, grid, s) : launch_solve<512, 1, false>(B, grid, s);
}

}  // namespace epk
