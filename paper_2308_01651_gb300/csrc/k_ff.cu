// k_ff.cu -- the FP64-accurate side of the refined solver (iterative
// refinement around the FP32 inner CG) in float-float arithmetic.
//
// Paper Sec. 1.2, Eq. (6): b = M (u_BDF/dt - I_ion + I_app) and the residual
// r = b - (alpha/dt M + K) u.  The nodal vector v and the iterate u (starting
// at u_EXT) arrive as float-float from the ionic kernel; the stencils are the
// node-major full couplings (hi and lo float parts).  Rows are accumulated
// with exact products and TwoSum (ep_ff.cuh), ~1e-13 relative to the terms,
// far below the refinement target of 1e-10 on ||r|| / ||b||, and entirely on
// the FP32 pipe.  The inner solver's starting data (r32 = r, z32 = D^-1 r32,
// delta = 0) is formed on the way.
#include "ep_dev.cuh"
#include "ep_refine.cuh"
#include "ep_tile.cuh"

namespace epk {

void launch_rhs_ff_batch(const Batch& B, int first, int graph, int grid, cudaStream_t s);
void launch_correct_ff_batch(const Batch& B, int grid, cudaStream_t s);
void launch_resid_np_batch(const Batch& B, int graph, int grid, cudaStream_t s);

// stage the float-float pair (ah, al) of the tile plus halo
__device__ __forceinline__ void stage_ff(const Dev& D, const TileGeo& g, int* sidx, const float* ah,
                                         const float* al, float* sh, float* sl) {
    stage_tile<float>(D, g, sidx, sh, [&](int n, bool) { return ah[n]; });
    // same halo positions per thread as above, so sidx is already this thread's
    for (int h = threadIdx.x; h < SHN; h += blockDim.x) {
        const int n = sidx[h];
        sl[h] = n >= 0 ? al[n] : 0.f;
    }
}

// FIRST: b = M v and r = b - A u_EXT, where A u_EXT comes from the stored
// A u of the last steps when there are enough of them (BDF1: y_n; BDF2:
// 2 y_n - y_{n-1}; BDF3: 3 y_n - 3 y_{n-1} + y_{n-2}, the extrapolations
// u_EXT is made of) and from an operator
// apply otherwise (first steps, after a BDF order change or a state load).
// Otherwise (after a correction): y = A u, stored as the step's current A u,
// and r = b - y with the stored b.  M v on a uniform slab needs no stored
// coefficients (row_mass_slab).
template <int FIRST>
__global__ void __launch_bounds__(kStThreads) k_rhs_ff(Batch B, int graph) {
    __shared__ int sidx[SHN];
    __shared__ float suh[SHN], sul[SHN];
    __shared__ float svh[FIRST ? SHN : 1], svl[FIRST ? SHN : 1];
    const Slot S = batch_slot(B);
    Dev& D = *S.D;
    // a residual after a correction runs only while the instance's
    // refinement goes on (a batched sweep also visits finished instances)
    if (!FIRST && !D.f_outer) return;
    const size_t N = (size_t)D.N;
    const float ns = D.nscale;
    const int order = bdf_order(D);
    // FIRST: extrapolate A u_EXT from the history instead of applying A
    const bool hist = FIRST && D.hist >= order;
    const bool slab_mass = D.Mhi == nullptr;
    // (ns b)^2, (ns r)^2, r32 z32, r32 r32
    float vf[4] = {0.f, 0.f, 0.f, 0.f};
    const double none[1] = {0.0};
    const int ntiles = st_tiles(D);
    for (int tile = S.blk; tile < ntiles; tile += S.nblk) {
        const TileGeo g = tile_geo(D, tile);
        __syncthreads();
        if (FIRST) {
            stage_ff(D, g, sidx, D.v_hi, D.v_lo, svh, svl);
            if (!hist)
                for (int h = threadIdx.x; h < SHN; h += blockDim.x) {
                    const int n = sidx[h];
                    suh[h] = n >= 0 ? D.u_hi[n] : 0.f;
                    sul[h] = n >= 0 ? D.u_lo[n] : 0.f;
                }
        } else {
            stage_ff(D, g, sidx, D.u_hi, D.u_lo, suh, sul);
        }
        __syncthreads();
        for_owned(D, g, [&](int h) {
            const int n = sidx[h];
            float bh, bl, ah, al;
            if (FIRST) {
                if (slab_mass) row_mass_slab(D, svh, svl, h, n, bh, bl);
                else row_ff(D.Mhi, D.Mlo, N, svh, svl, h, n, bh, bl);
                D.b_hi[n] = bh;
                D.b_lo[n] = bl;
                if (hist) {
                    ah = D.yn_hi[n];
                    al = D.yn_lo[n];
                    if (order == 2) {
                        // 2 y_n - y_{n-1}: the doubling is exact
                        ff_sub(2.f * ah, 2.f * al, D.ym_hi[n], D.ym_lo[n], ah, al);
                    } else if (order == 3) {
                        // 3 (y_n - y_{n-1}) + y_{n-2}
                        float dh, dl;
                        ff_sub(ah, al, D.ym_hi[n], D.ym_lo[n], dh, dl);
                        ff_mul(dh, dl, 3.f, 0.f, dh, dl);
                        ff_sub(dh, dl, -D.ym2_hi[n], -D.ym2_lo[n], ah, al);
                    }
                } else {
                    row_ff(D.Ahi, D.Alo, N, suh, sul, h, n, ah, al);
                }
                // A u_EXT is the step's A u if this residual already meets
                // the tolerance (a sweep overwrites it otherwise)
                D.yc_hi[n] = ah;
                D.yc_lo[n] = al;
            } else {
                bh = D.b_hi[n];
                bl = D.b_lo[n];
                row_ff(D.Ahi, D.Alo, N, suh, sul, h, n, ah, al);
                D.yc_hi[n] = ah;
                D.yc_lo[n] = al;
            }
            float rh, rl;
            ff_sub(bh, bl, ah, al, rh, rl);
            const float r32 = rh;  // nearest float of the normalised pair
            const float z = D.dinv32[n] * r32;
            D.r32[n] = r32;
            D.z32[n] = z;
            D.d32[n] = 0.0f;
            const float bs = ns * bh, rs = ns * rh;
            vf[0] = fmaf(bs, bs, vf[0]);
            vf[1] = fmaf(rs, rs, vf[1]);
            vf[2] = fmaf(r32, z, vf[2]);
            vf[3] = fmaf(r32, r32, vf[3]);
        });
    }
    grid_reduce<4, 0>(vf, none, D.partial, D.counter + CNT_RHS, S.blk, S.nblk,
                      [&](double* t) { rhs_finish(D, t, FIRST != 0, graph, ns); });
}

// Residual after a correction, node-parallel: every thread takes nodes
// n = t, t + T, ... of its instance, reads the float-float couplings of A
// and its 27 neighbours' u (through L1) -- no shared-memory tiles or block
// barriers between the coefficient streams -- and writes y = A u (the step's
// history), r = b - y and the inner solver's start (r32, u = D^-1 r32, delta
// = 0).  Same terms, order and totals as the tiled pass.
__global__ void __launch_bounds__(kResidThreads) k_resid_np(Batch B, int graph) {
    const Slot S = batch_slot(B);
    Dev& D = *S.D;
    if (!D.f_outer) return;
    const int N = D.N;
    const size_t NN = (size_t)N;
    const float ns = D.nscale;
    const int nx = D.NX, nxy = D.NX * D.NY, wrap = D.periodic ? D.NX * (D.NY - 1) : 0;
    const float* __restrict__ uh = D.u_hi;
    const float* __restrict__ ul = D.u_lo;
    float vf[4] = {0.f, 0.f, 0.f, 0.f};
    const double none[1] = {0.0};
    for (int n = S.blk * blockDim.x + threadIdx.x; n < N; n += S.nblk * blockDim.x) {
        const NbrOff o = nbr_offsets(nx, nxy, wrap, D.nflag[n]);
        float ah, al, rh, rl;
        row_ff_np(D.Ahi, D.Alo, NN, uh, ul, n, o, ah, al);
        D.yc_hi[n] = ah;
        D.yc_lo[n] = al;
        ff_sub(D.b_hi[n], D.b_lo[n], ah, al, rh, rl);
        const float r32 = rh;
        const float z = D.dinv32[n] * r32;
        D.r32[n] = r32;
        D.z32[n] = z;
        D.d32[n] = 0.0f;
        const float bs = ns * D.b_hi[n], rs = ns * rh;
        vf[0] = fmaf(bs, bs, vf[0]);
        vf[1] = fmaf(rs, rs, vf[1]);
        vf[2] = fmaf(r32, z, vf[2]);
        vf[3] = fmaf(r32, r32, vf[3]);
    }
    grid_reduce<4, 0>(vf, none, D.partial, D.counter + CNT_RHS, S.blk, S.nblk,
                      [&](double* t) { rhs_finish(D, t, false, graph, ns); });
}

// u += delta in float-float
__global__ void __launch_bounds__(kNodeThreads) k_correct_ff(Batch B) {
    const Slot S = batch_slot(B);
    const Dev& D = *S.D;
    if (!D.f_outer) return;
    float* __restrict__ uh = D.u_hi;
    float* __restrict__ ul = D.u_lo;
    const float* __restrict__ d = D.d32;
    for (int n = S.blk * blockDim.x + threadIdx.x; n < D.N; n += S.nblk * blockDim.x) {
        float h = uh[n], l = ul[n];
        ff_add_f(h, l, d[n], h, l);
        uh[n] = h;
        ul[n] = l;
    }
}

void launch_rhs_ff(Dev* d, const Dev& h, int first, int graph, int grid, cudaStream_t s) {
    launch_rhs_ff_batch(single_batch(d), first, graph, grid, s);
}
void launch_rhs_ff_batch(const Batch& B, int first, int graph, int grid, cudaStream_t s) {
    if (first) k_rhs_ff<1><<<grid, kStThreads, 0, s>>>(B, graph);
    else k_rhs_ff<0><<<grid, kStThreads, 0, s>>>(B, graph);
}

void launch_resid_np(Dev* d, const Dev& h, int graph, int grid, cudaStream_t s) {
    launch_resid_np_batch(single_batch(d), graph, grid, s);
}
void launch_resid_np_batch(const Batch& B, int graph, int grid, cudaStream_t s) {
    k_resid_np<<<grid, kResidThreads, 0, s>>>(B, graph);
}

void launch_correct_ff(Dev* d, const Dev& h, int grid, cudaStream_t s) {
    launch_correct_ff_batch(single_batch(d), grid, s);
}
void launch_correct_ff_batch(const Batch& B, int grid, cudaStream_t s) {
    k_correct_ff<<<grid, kNodeThreads, 0, s>>>(B);
}

}  // namespace epk
