// k_cg.cu -- pointwise kernels of the FP32 inner CG, the FP64 refinement
// correction and the end of a time step.
//
// The inner solver is Jacobi-preconditioned CG (the paper solves Eq. (6) with
// CG, Sec. 2) on A delta = r in float; iterative refinement in double wraps
// it (k_ff.cu: float-float right-hand side, residual and update).  Activation time follows
// Sec. 3.2.1: the time at which du/dt is largest, taken as the first maximum
// of the forward difference u_{n+1} - u_n.
#include "ep_dev.cuh"
#include "ep_ff.cuh"

namespace epk {

// delta += alpha p, r -= alpha q, z = D^-1 r; beta, inner convergence
__global__ void __launch_bounds__(kNodeThreads) k_update32(Dev* __restrict__ Dp, int graph) {
    Dev& D = *Dp;
    const float alpha = (float)D.alpha;
    const float* __restrict__ p = D.pswap ? D.pa32 : D.pb32;  // the p written by the apply
    float* __restrict__ d = D.d32;
    float* __restrict__ r = D.r32;
    float* __restrict__ zz = D.z32;
    const float* __restrict__ q = D.q32;
    const float* __restrict__ di = D.dinv32;
    const int N = D.N;
    float v[2] = {0.f, 0.f};
    const double none[1] = {0.0};
    // four nodes per thread with 16-byte accesses (arrays are 256-byte aligned)
    const int n4 = N >> 2;
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < n4; t += gridDim.x * blockDim.x) {
        const float4 p4 = reinterpret_cast<const float4*>(p)[t];
        const float4 q4 = reinterpret_cast<const float4*>(q)[t];
        const float4 i4 = reinterpret_cast<const float4*>(di)[t];
        float4 d4 = reinterpret_cast<float4*>(d)[t];
        float4 r4 = reinterpret_cast<float4*>(r)[t];
        float4 z4;
        d4.x = fmaf(alpha, p4.x, d4.x); d4.y = fmaf(alpha, p4.y, d4.y);
        d4.z = fmaf(alpha, p4.z, d4.z); d4.w = fmaf(alpha, p4.w, d4.w);
        r4.x = fmaf(-alpha, q4.x, r4.x); r4.y = fmaf(-alpha, q4.y, r4.y);
        r4.z = fmaf(-alpha, q4.z, r4.z); r4.w = fmaf(-alpha, q4.w, r4.w);
        z4.x = i4.x * r4.x; z4.y = i4.y * r4.y; z4.z = i4.z * r4.z; z4.w = i4.w * r4.w;
        reinterpret_cast<float4*>(d)[t] = d4;
        reinterpret_cast<float4*>(r)[t] = r4;
        reinterpret_cast<float4*>(zz)[t] = z4;
        v[0] += (r4.x * z4.x + r4.y * z4.y) + (r4.z * z4.z + r4.w * z4.w);
        v[1] += (r4.x * r4.x + r4.y * r4.y) + (r4.z * r4.z + r4.w * r4.w);
    }
    for (int n = 4 * n4 + blockIdx.x * blockDim.x + threadIdx.x; n < N; n += gridDim.x * blockDim.x) {
        d[n] = fmaf(alpha, p[n], d[n]);
        const float rn = fmaf(-alpha, q[n], r[n]);
        r[n] = rn;
        const float z = di[n] * rn;
        zz[n] = z;
        v[0] = fmaf(rn, z, v[0]);
        v[1] = fmaf(rn, rn, v[1]);
    }
    grid_reduce<2, 0>(v, none, D.partial, D.counter + CNT_UPDATE, blockIdx.x, gridDim.x, [&](double* tot) {
        D.beta = tot[0] / D.rz;
        D.rz = tot[0];
        D.rr = tot[1];
        D.it += 1;
        D.it_total += 1;
        D.pswap ^= 1;
        const bool nan = !(tot[1] == tot[1]);
        const bool conv = !nan && tot[1] <= D.inner_stop;
        if (nan && D.status == EP_OK) D.status = EP_ENAN;
        set_cond(graph ? D.h_inner : 0ull, &D.f_inner, (!conv && !nan && D.it < D.max_iter) ? 1u : 0u);
    });
}

// FP64 path: activation update, non-finite check, rotation of the time
// levels.
__global__ void __launch_bounds__(kNodeThreads) k_finish(Batch B) {
    const Slot S = batch_slot(B);
    Dev& D = *S.D;
    const double t_new = (double)(D.step + 1) * D.dt;
    float v[1] = {0.f};
    const double none[1] = {0.0};
    for (int n = S.blk * blockDim.x + threadIdx.x; n < D.N; n += S.nblk * blockDim.x) {
        const double un = D.u_new[n];
        const double s = un - D.u_n[n];
        if (!isfinite(un)) v[0] += 1.f;
        if (s > D.best[n]) {
            D.best[n] = s;
            D.at[n] = t_new;
        }
    }
    grid_reduce<1, 0>(v, none, D.partial, D.counter + CNT_FINISH, S.blk, S.nblk, [&](double* tot) {
        if (tot[0] > 0.0 && D.status == EP_OK) D.status = EP_ENAN;
        end_of_step(D);
    });
}

// Refined path, the per-node end of a step: the refinement's last residual
// pass has already rotated the time levels (end_of_step), so the new
// potential is level n and the old one level n-1.  Per node: the activation
// slope in float from the pairs, the new potential rounded to double for
// u_n.  A non-finite potential has already made that residual NaN (EP_ENAN);
// no reduction is needed here.  The next step's ionic kernel does the same
// work on its way (finish_prev_ff); this kernel runs only when the host
// reads the state before another step.  Idempotent.
__global__ void __launch_bounds__(kNodeThreads) k_finish_ff(Batch B) {
    const Slot S = batch_slot(B);
    Dev& D = *S.D;
    const double t_new = (double)D.step * D.dt;
    const float* __restrict__ h1p = D.uh_n;
    const float* __restrict__ l1p = D.ul_n;
    const float* __restrict__ h0p = D.uh_m;
    const float* __restrict__ l0p = D.ul_m;
    double* __restrict__ un = D.u_n;
    float* __restrict__ best = D.bestf;
    for (int n = S.blk * blockDim.x + threadIdx.x; n < D.N; n += S.nblk * blockDim.x) {
        const float h1 = h1p[n], l1 = l1p[n];
        const float s = (h1 - h0p[n]) + (l1 - l0p[n]);
        un[n] = ff_to_double(h1, l1);
        if (s > best[n]) {
            best[n] = s;
            D.at[n] = t_new;
        }
    }
}

void launch_update32(Dev* d, const Dev& h, int grid, int graph, cudaStream_t s) {
    k_update32<<<grid, kNodeThreads, 0, s>>>(d, graph);
}
void launch_finish(Dev* d, const Dev& h, int grid, cudaStream_t s) {
    if (h.prec == EP_PREC_FP32_REFINED) k_finish_ff<<<grid, kNodeThreads, 0, s>>>(single_batch(d));
    else k_finish<<<grid, kNodeThreads, 0, s>>>(single_batch(d));
}

}  // namespace epk
