// k_noalloc.cu -- ep_residual_norm_noalloc: the relative residual
// ||b - A u|| / ||b|| of an instance's last linear solve (u the solver's
// float-float iterate, whose sum rounded to double is u_n), computed without
// allocating anything.
//
// Who needs it: host code that cannot call cudaMalloc at the point where it
// wants the number -- for example an application whose device memory is owned
// by another allocator (a framework's caching allocator, or a pool that
// reserves the GPU's memory at start-up), where an allocation here would fail
// or break the owner's accounting.  Everything this call touches is either
// the instance's existing memory (read only) or the fixed scratch array
// below.
//
// Scratch: g_noalloc_scratch, a file-scope __device__ array of
// kNoAllocScratchBytes (about 16 KiB) that every GPU loading this library
// holds until the process exits.  It stores one pair of partial sums per
// thread block (at most kNoAllocMaxBlocks blocks), the two totals, and the
// arrival counter of the last-block reduction.  Host code cannot use the
// array's name as a device address; at set-up, once per device and with that
// device current, the address is taken with cudaGetSymbolAddress and passed
// to the kernel; the first call on each device does that set-up.  Every call
// shares the array and it keeps the last call's contents: each call clears
// the counter before its kernel runs, and calls whose work overlaps on the
// GPU (different streams, no ordering) race on the array.
//
// The kernel repeats the refined solver's residual (the one closing each
// refinement sweep inside the persistent solve, float-float, node-parallel):
// same grid, same nodes per thread, same per-thread, per-block and
// across-block summation (float partials, summed in the same fixed order), so
// it reproduces the solver's own residual norm; it writes nothing but the
// scratch array.  It serves FP32_REFINED stencil instances.
#include <mutex>
#include <string>

#include "ep_dev.cuh"
#include "ep_tile.cuh"

namespace epk {

constexpr int kNoAllocMaxBlocks = 1024;
// layout: float partial[2][kNoAllocMaxBlocks] (in the first half of the
// area); double total[2]; unsigned counter
constexpr size_t kNoAllocTotalOff = sizeof(double) * 2 * kNoAllocMaxBlocks;
constexpr size_t kNoAllocCounterOff = kNoAllocTotalOff + 2 * sizeof(double);
constexpr size_t kNoAllocScratchBytes = kNoAllocCounterOff + 256;

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

__global__ void __launch_bounds__(1024) k_residual_norm_noalloc(const Dev* __restrict__ Dp,
                                                                       unsigned char* scratch) {
    const Dev& D = *Dp;
    const int N = D.N;
    const float ns = D.nscale;
    const int nx = D.NX, nxy = D.NX * D.NY, wrap = D.periodic ? D.NX * (D.NY - 1) : 0;
    float* part = reinterpret_cast<float*>(scratch);
    double* total = reinterpret_cast<double*>(scratch + kNoAllocTotalOff);
    unsigned int* counter = reinterpret_cast<unsigned int*>(scratch + kNoAllocCounterOff);
    const int G = gridDim.x, T = G * blockDim.x;
    float vf[2] = {0.f, 0.f};
    // the last solve's float-float iterate, now the potential level n (u_n is
    // its sum rounded to double)
    const float* __restrict__ uh = D.uh_n;
    const float* __restrict__ ul = D.ul_n;
    for (int n = blockIdx.x * blockDim.x + threadIdx.x; n < N; n += T) {
        const unsigned int f = D.nflag[n];
        const NbrOff o = nbr_offsets(nx, nxy, wrap, f);
        float ah, al, rh, rl;
        row_ff_sym(D.Ahi, D.Alo, D.cs, uh, ul, n, o, exist_flags(f, wrap), ah, al);
        const float bh = D.b_hi[n];
        ff_sub(bh, D.b_lo[n], ah, al, rh, rl);
        const float bs = ns * bh, rs = ns * rh;
        vf[0] = fmaf(bs, bs, vf[0]);
        vf[1] = fmaf(rs, rs, vf[1]);
    }
    publish<2>(vf, part, G, blockIdx.x);
    // the last block to arrive forms the totals
    __shared__ bool last;
    if (threadIdx.x == 0) {
        __threadfence();
        last = atomicAdd(counter, 1u) == (unsigned int)(G - 1);
    }
    __syncthreads();
    if (!last) return;
    __threadfence();
    if (threadIdx.x < 32) {
        float tt[2];
        gather<2>(part, G, tt);
        if (threadIdx.x == 0) {
            total[0] = tt[0];
            total[1] = tt[1];
        }
    }
}

namespace {
std::mutex g_noalloc_mu;
void* g_noalloc_addr[64] = {nullptr};
}  // namespace

// Device address of the scratch array on the current device (set-up on first
// use per device).
cudaError_t noalloc_scratch(void** out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lk(g_noalloc_mu);
    if (!g_noalloc_addr[dev]) {
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess) return e;
        g_noalloc_addr[dev] = p;
    }
    *out = g_noalloc_addr[dev];
    return cudaSuccess;
}

int noalloc_max_blocks() { return kNoAllocMaxBlocks; }

// Runs the kernel on stream s (the persistent solve's grid and block size,
// so that every thread sums the solver's nodes) and copies the two sums
// (b.b, r.r) to host.
cudaError_t residual_norm_noalloc(Dev* d, int grid, int threads, cudaStream_t s, double sums[2]) {
    void* scratch = nullptr;
    cudaError_t e = noalloc_scratch(&scratch);
    if (e != cudaSuccess) return e;
    unsigned char* base = static_cast<unsigned char*>(scratch);
    e = cudaMemsetAsync(base + kNoAllocCounterOff, 0, sizeof(unsigned int), s);
    if (e != cudaSuccess) return e;
    k_residual_norm_noalloc<<<grid, threads, 0, s>>>(d, base);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    e = cudaMemcpyAsync(sums, base + kNoAllocTotalOff, 2 * sizeof(double), cudaMemcpyDeviceToHost, s);
    if (e != cudaSuccess) return e;
    return cudaStreamSynchronize(s);
}

}  // namespace epk
