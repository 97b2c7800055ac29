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

void launch_rhs_ff_batch(const Batch& B, int graph, int grid, bool curved, cudaStream_t s);
void launch_correct_ff_batch(const Batch& B, int grid, cudaStream_t s);
void launch_resid_np_batch(const Batch& B, int graph, int grid, cudaStream_t s);

// Consistent mass matrix of a uniform Q1 slab, applied without stored
// coefficients: M(n, n+o) = w c_x c_y c_z, w = hx hy hz / 216, with per
// direction c = 1 off the diagonal (0 where the neighbour does not exist)
// and 4 (interior) or 2 (first/last node) on it -- the 1D mass matrix
// h/6 [1 4 1] with its halved boundary diagonal, exact for the trilinear
// basis.  The weights come from the node's boundary flags f (bits: i = 0,
// i = NX-1, j = 0, j = NY-1, k = 0, k = NZ-1); they are powers of two (or 0),
// so the sum runs in float-float on exact products:
// (sh + sl) = sum_t c(t) (xh + xl)(n + off(t)) * (wh + wl), normalised.
__device__ __forceinline__ void mass_slab_np(const Dev& D, unsigned int f, const NbrOff& o, int n,
                                             const float* __restrict__ xh, const float* __restrict__ xl,
                                             float& sh, float& sl) {
    const float wx[3] = {(f & 1u) ? 0.f : 1.f, (f & 3u) ? 2.f : 4.f, (f & 2u) ? 0.f : 1.f};
    const float wy[3] = {(f & 4u) ? 0.f : 1.f, (f & 12u) ? 2.f : 4.f, (f & 8u) ? 0.f : 1.f};
    const float wz[3] = {(f & 16u) ? 0.f : 1.f, (f & 48u) ? 2.f : 4.f, (f & 32u) ? 0.f : 1.f};
    sh = 0.f;
    sl = 0.f;
#pragma unroll
    for (int t = 0; t < 27; ++t) {
        const int m = n + o.x[t % 3] + o.y[(t / 3) % 3] + o.z[t / 9];
        ff_acc_pow2(wx[t % 3] * wy[(t / 3) % 3] * wz[t / 9], xh[m], xl[m], sh, sl);
    }
    ff_normalize(sh, sl);
    ff_mul(sh, sl, D.mw_hi, D.mw_lo, sh, sl);
}

// The step's first residual, node-parallel (every Q1 operator): b = M v and
// r = b - A u_EXT, where A u_EXT comes from the stored A u of the last steps
// when there are enough of them (BDF1: y_n; BDF2: 2 y_n - y_{n-1}; BDF3:
// 3 y_n - 3 y_{n-1} + y_{n-2}, the extrapolations u_EXT is made of) and from
// an operator apply otherwise (first steps, after a BDF order change or a
// state load).  Every thread takes nodes n = t, t + T, ... and reads the
// neighbours' values through L1 at the offsets of the node's flags (a tiled
// form staging v and u with their halos in shared memory measured 33.6 us
// against 28.0 us on the 442k-node slab).  MINB resident blocks per SM: with
// the curved mass matrix's float-float rows (54 couplings and 54 neighbour
// values a node) one block per SM and 128 registers (2.19M-node shell: 151
// against 194 us, and 141 us with a grid of one block per SM), with the
// slab's analytic mass matrix two blocks and 64 registers (442k-node slab:
// 34 against 41 us); the register cap changes nothing in the results.
template <int MINB>
__global__ void __launch_bounds__(kResidThreads, MINB) k_rhs_np(Batch B, int graph) {
    const Slot S = batch_slot(B);
    Dev& D = *S.D;
    const int N = D.N;
    const float ns = D.nscale;
    const int order = bdf_order(D);
    const bool hist = D.hist >= order;
    const bool slab_mass = D.Mhi == nullptr;
    const int nx = D.NX, nxy = D.NX * D.NY, wrap = D.periodic ? D.NX * (D.NY - 1) : 0;
    const float* __restrict__ vh = D.v_hi;
    const float* __restrict__ vl = D.v_lo;
    float vf[4] = {0.f, 0.f, 0.f, 0.f};
    const double none[1] = {0.0};
    // this step's amplitudes of the element-region pulses, float-float
    float eamp_h[EP_MAX_PULSES], eamp_l[EP_MAX_PULSES];
    bool eg = false;
#pragma unroll
    for (int p = 0; p < EP_MAX_PULSES; ++p) {
        const double a = D.egh[p] ? pulse_amp(D, p) : 0.0;
        eamp_h[p] = (float)a;
        eamp_l[p] = (float)(a - (double)eamp_h[p]);
        eg = eg || eamp_h[p] != 0.f;
    }
    for (int n = S.blk * blockDim.x + threadIdx.x; n < N; n += S.nblk * blockDim.x) {
        const unsigned int f = D.nflag[n];
        const NbrOff o = nbr_offsets(nx, nxy, wrap, f);
        float bh, bl, ah, al;
        if (slab_mass) mass_slab_np(D, f, o, n, vh, vl, bh, bl);
        else row_ff_sym(D.Mhi, D.Mlo, D.cs, vh, vl, n, o, exist_flags(f, wrap), bh, bl);
        if (eg) {
            // applied currents on element regions: b += amp f (float-float)
#pragma unroll
            for (int p = 0; p < EP_MAX_PULSES; ++p)
                if (D.egh[p] && eamp_h[p] != 0.f) {
                    float th, tl;
                    ff_mul(eamp_h[p], eamp_l[p], D.egh[p][n], D.egl[p][n], th, tl);
                    ff_sub(bh, bl, -th, -tl, bh, bl);
                }
        }
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
            row_ff_sym(D.Ahi, D.Alo, D.cs, D.u_hi, D.u_lo, n, o, exist_flags(f, wrap), ah, al);
        }
        // A u_EXT is the step's A u if this residual already meets the
        // tolerance (a sweep overwrites it otherwise)
        D.yc_hi[n] = ah;
        D.yc_lo[n] = al;
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
    }
    grid_reduce<4, 0>(vf, none, D.partial, D.counter + CNT_RHS, S.blk, S.nblk,
                      [&](double* t) { rhs_finish(D, t, true, graph, ns); });
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
    const float ns = D.nscale;
    const int nx = D.NX, nxy = D.NX * D.NY, wrap = D.periodic ? D.NX * (D.NY - 1) : 0;
    const float* __restrict__ uh = D.u_hi;
    const float* __restrict__ ul = D.u_lo;
    float vf[4] = {0.f, 0.f, 0.f, 0.f};
    const double none[1] = {0.0};
    for (int n = S.blk * blockDim.x + threadIdx.x; n < N; n += S.nblk * blockDim.x) {
        const unsigned int f = D.nflag[n];
        const NbrOff o = nbr_offsets(nx, nxy, wrap, f);
        float ah, al, rh, rl;
        row_ff_sym(D.Ahi, D.Alo, D.cs, uh, ul, n, o, exist_flags(f, wrap), ah, al);
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

void launch_rhs_ff(Dev* d, const Dev& h, int graph, int grid, cudaStream_t s) {
    launch_rhs_ff_batch(single_batch(d), graph, grid, h.Mhi != nullptr, s);
}
// curved: some instance of the batch has the stored (curved) mass matrix
void launch_rhs_ff_batch(const Batch& B, int graph, int grid, bool curved, cudaStream_t s) {
    if (curved) k_rhs_np<1><<<grid, kResidThreads, 0, s>>>(B, graph);
    else k_rhs_np<2><<<grid, kResidThreads, 0, s>>>(B, graph);
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
