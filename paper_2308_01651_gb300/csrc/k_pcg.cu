// k_pcg.cu -- the FP32 inner solve of a refinement sweep in one persistent,
// cooperative launch (stencil operator).
//
// Jacobi-preconditioned CG (the paper solves Eq. (6) with CG, Sec. 2) on
// A delta = r in float, A the hi parts of the node-major full couplings, in
// the single-reduction arrangement of Chronopoulos and Gear (1989): with
// u = D^-1 r and w = A u, both dot products of an iteration, (r, u) and
// (u, w), come from the same pass, so every iteration is ONE pass over the
// data and ONE grid barrier.  Iteration i, given alpha_i and beta_i:
//   s_i = w_i + beta_i s_{i-1},   r_{i+1} = r_i - alpha_i s_i,
//   p_i = u_i + beta_i p_{i-1},   delta  += alpha_i p_i,
//   u_{i+1} = D^-1 r_{i+1},       w_{i+1} = A u_{i+1},
//   gamma = (r_{i+1}, u_{i+1}), eta = (u_{i+1}, w_{i+1}), rho = (r_{i+1}, r_{i+1}),
//   beta_{i+1} = gamma_{i+1} / gamma_i,
//   alpha_{i+1} = gamma_{i+1} / (eta_{i+1} - beta_{i+1} gamma_{i+1} / alpha_i).
// Every block of a grid that fits on the GPU at once owns a fixed set of
// tiles.  Per tile it stages u_{i+1} on the tile plus halo in shared memory,
// recomputing s_i and r_{i+1} of the halo nodes itself from the previous
// iteration's r, w, s (double-buffered, so no block overwrites what another
// still reads) -- the same expression in every block, hence the same bits --
// and writes r, s, p, delta of its owned nodes and w = A u for them.  The
// block partials of gamma, eta, rho are published, a bounded grid barrier
// waits for all blocks, and every block sums all partials in the same fixed
// order, so all blocks take the same alpha, beta and stopping decision.
// A first pass (no update) forms w_0 = A u_0 and the starting sums.  Data
// written by one block and read by another within the launch is read through
// L2 (__ldcg); a barrier that does not complete within ~1 s records
// EP_ETIMEOUT and the kernel returns.
#include "ep_dev.cuh"
#include "ep_tile.cuh"

namespace epk {

constexpr long long kBarrierSpinLimit = 1ll << 24;  // x >= 64 ns naps: about a second

// Bounded grid barrier (all blocks of a cooperative launch).  count and gen
// persist between launches: count returns to 0 after every barrier, gen
// only grows.  Returns false after recording EP_ETIMEOUT when the other
// blocks did not all arrive in time.
__device__ __forceinline__ bool grid_barrier(unsigned int* count, unsigned int* gen, unsigned int& my_gen,
                                             int* status) {
    __shared__ int ok;
    __syncthreads();
    if (threadIdx.x == 0) {
        int good = 1;
        const unsigned int g = my_gen;
        __threadfence();
        if (atomicAdd(count, 1u) == gridDim.x - 1) {
            atomicExch(count, 0u);
            __threadfence();
            atomicAdd(gen, 1u);
        } else {
            long long spins = 0;
            while (*(volatile unsigned int*)gen == g) {
                if (++spins > kBarrierSpinLimit) {
                    good = 0;
                    atomicCAS(status, (int)EP_OK, (int)EP_ETIMEOUT);
                    break;
                }
                __nanosleep(64);
            }
        }
        __threadfence();
        my_gen = g + 1;
        ok = good;
    }
    __syncthreads();
    return ok != 0;
}

// Block sums of NV float values (warp shuffles, then warps in fixed order),
// written as part[k * G + blockIdx.x].
template <int NV>
__device__ __forceinline__ void publish(const float (&v)[NV], double* part, int G) {
    __shared__ float sh[NV][kMaxBlock / 32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarp = blockDim.x >> 5;
#pragma unroll
    for (int k = 0; k < NV; ++k) {
        const float s = warp_sum(v[k]);
        if (lane == 0) sh[k][warp] = s;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
#pragma unroll
        for (int k = 0; k < NV; ++k) {
            float s = 0.f;
            for (int w = 0; w < nwarp; ++w) s += sh[k][w];
            part[(size_t)k * G + blockIdx.x] = (double)s;
        }
    }
}

__device__ __forceinline__ double warp_sum_d(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Totals of all blocks' partials (part[k * G + i]), summed in one fixed order
// (thread, then warp butterfly, then warps in order) by every block: all
// threads load at once, so the gather costs about one L2 round trip.
template <int NV>
__device__ __forceinline__ void gather(const double* part, int G, double (&tot)[NV]) {
    __shared__ double wsum[NV][kMaxBlock / 32];
    __shared__ double res[NV];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarp = blockDim.x >> 5;
    double acc[NV];
#pragma unroll
    for (int k = 0; k < NV; ++k) acc[k] = 0.0;
    for (int i = threadIdx.x; i < G; i += blockDim.x) {
#pragma unroll
        for (int k = 0; k < NV; ++k) acc[k] += __ldcg(&part[(size_t)k * G + i]);
    }
#pragma unroll
    for (int k = 0; k < NV; ++k) {
        const double sw = warp_sum_d(acc[k]);
        if (lane == 0) wsum[k][warp] = sw;
    }
    __syncthreads();
    if (threadIdx.x < NV) {
        double t = 0.0;
        for (int w = 0; w < nwarp; ++w) t += wsum[threadIdx.x][w];
        res[threadIdx.x] = t;
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < NV; ++k) tot[k] = res[k];
}

__global__ void __launch_bounds__(kStThreads, 2) k_pcg32_stencil(Dev* __restrict__ Dp) {
    __shared__ int sidx[SHN];
    __shared__ float su[SHN];
    Dev& D = *Dp;
    const size_t N = (size_t)D.N;
    const int G = gridDim.x;
    const int ntiles = st_tiles(D);
    // double-buffered r, w, s; p and delta are touched by their owners only
    float* const r0b = D.r32;
    float* const r1b = D.z32;
    float* const w0b = D.q32;
    float* const w1b = D.pa32;
    float* const s0b = D.pb32;
    float* const s1b = D.s32;
    float* __restrict__ p = D.p32;
    float* __restrict__ x = D.d32;
    const float* __restrict__ dinv = D.dinv32;
    const float4* __restrict__ A = D.Ahi;
    double* part = D.partial;
    unsigned int* bcount = D.counter + CNT_BAR;
    unsigned int* bgen = D.counter + CNT_BAR + 1;
    unsigned int my_gen = 0;
    if (threadIdx.x == 0) my_gen = *(volatile unsigned int*)bgen;
    const int max_it = D.max_iter;
    const double tol2 = D.inner_tol * D.inner_tol;
    double stop = 0.0, gam_old = 0.0, alpha_old = 0.0, rr = 0.0, gam = 0.0;
    float alpha = 0.f, beta = 0.f;
    int it = 0, cur = 0, pass = 0;
    bool first = true, nan = false;
    for (;; ++pass) {
        const float* rc = cur ? r1b : r0b;
        const float* wc = cur ? w1b : w0b;
        const float* sc = cur ? s1b : s0b;
        float* rn = cur ? r0b : r1b;
        float* wn = (first || cur) ? w0b : w1b;
        float* sn = cur ? s0b : s1b;
        float v[3] = {0.f, 0.f, 0.f};  // gamma, eta, rho
        for (int tile = blockIdx.x; tile < ntiles; tile += G) {
            const TileGeo g = tile_geo(D, tile);
            __syncthreads();
            stage_tile<float>(D, g, sidx, su, [&](int n, bool own) {
                const float dv = __ldg(dinv + n);
                const float r0 = __ldcg(rc + n);
                float r1 = r0;
                if (!first) {
                    const float w0 = __ldcg(wc + n);
                    const float s1 = beta == 0.f ? w0 : fmaf(beta, __ldcg(sc + n), w0);
                    r1 = fmaf(-alpha, s1, r0);
                    if (own) {
                        const float u0 = dv * r0;
                        const float p1 = beta == 0.f ? u0 : fmaf(beta, p[n], u0);
                        p[n] = p1;
                        x[n] = fmaf(alpha, p1, x[n]);
                        sn[n] = s1;
                        rn[n] = r1;
                    }
                }
                const float u1 = dv * r1;
                if (own) {
                    v[0] = fmaf(r1, u1, v[0]);
                    v[2] = fmaf(r1, r1, v[2]);
                }
                return u1;
            });
            __syncthreads();
            for_owned(D, g, [&](int h) {
                const int n = sidx[h];
                const float w1 = row_f32(A, N, su, h, n);
                wn[n] = w1;
                v[1] = fmaf(su[h], w1, v[1]);
            });
        }
        // partials alternate between two regions: a block that runs ahead
        // publishes into the region nobody is still reading
        double* pr = part + (size_t)(pass & 1) * 3 * G;
        publish<3>(v, pr, G);
        if (!grid_barrier(bcount, bgen, my_gen, &D.status)) break;
        double t[3];
        gather<3>(pr, G, t);
        if (!first) {
            ++it;
            cur ^= 1;
        }
        gam = t[0];
        rr = t[2];
        if (first) stop = tol2 * rr;
        nan = !(t[0] == t[0] && t[1] == t[1] && t[2] == t[2]);
        if (nan || rr <= stop || it >= max_it) break;
        const double b = first ? 0.0 : gam / gam_old;
        const double a = first ? gam / t[1] : gam / (t[1] - b * gam / alpha_old);
        beta = (float)b;
        alpha = (float)a;
        gam_old = gam;
        alpha_old = a;
        first = false;
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        D.rz = gam;
        D.rr = rr;
        D.it = it;
        D.it_total += it;
        if (nan && D.status == EP_OK) D.status = EP_ENAN;
    }
}

// blocks of k_pcg32_stencil that fit on one SM at once
int pcg_blocks_per_sm() {
    int occ = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_pcg32_stencil, kStThreads, 0) != cudaSuccess)
        return 0;
    return occ;
}

cudaError_t launch_pcg32(Dev* d, int grid, cudaStream_t s) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(grid);
    cfg.blockDim = dim3(kStThreads);
    cfg.dynamicSmemBytes = 0;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, k_pcg32_stencil, d);
}

}  // namespace epk
