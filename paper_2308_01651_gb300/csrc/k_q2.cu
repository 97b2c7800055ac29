// k_q2.cu -- matrix-free operators of triquadratic (Q2, 27-node) hexahedra on
// slab meshes (Sec. 1.2: hexahedral elements of any degree; Sec. 5 names
// high-order matrix-free solvers on GPUs as the way forward).
//
// The element operator of Eq. (6), A_e = alpha/dt M_e + K_e, is applied by
// sum factorisation on the 3 x 3 x 3 Gauss points of [0,1]^3 (exact for the
// mass matrix of a box):
//   y_a = sum_q  phi_a(q) cm_q u(q)  +  grad_xi phi_a(q) . G_q grad_xi u(q),
// with u(q) and grad_xi u(q) from the 27 nodal values by three 1-D passes
// (3 x 3 matrices B[q][b] = l_b(xi_q), Dd[q][b] = l_b'(xi_q) of the quadratic
// Lagrange basis), cm_q = alpha/dt hx hy hz w_q, and G_q = w_q |J| H D(q) H
// (H = diag(1/h), D of Eq. (3) at the Gauss point) precomputed per element
// and point at ep_create.  The transposed passes bring the quadrature values
// back to the 27 nodes.
//
// Work decomposition: 27 threads per element (one per node in the nodal
// passes, one per Gauss point in the quadrature passes), nine elements per
// 256-thread block, the intermediate arrays in shared memory.  Every element
// writes its 27 outputs to a per-element buffer; a node-parallel gather then
// sums the contributions of the node's 1, 2, 4 or 8 elements in a fixed
// order (no atomics: bitwise reproducible).  The FP32 variant is the inner
// CG's operator; the float-float variant (ep_ff.cuh) gives the refinement its
// right-hand side b = M v and residual b - A u.
#include <cmath>

#include "ep_dev.cuh"
#include "ep_ff.cuh"
#include "ep_refine.cuh"

namespace epk {

constexpr int kQ2Groups = 9;     // elements per block
constexpr int kQ2Threads = 256;  // 9 x 27 = 243 working threads
constexpr int kQ2Slots = 7;      // intermediate arrays per element

// [q * 3 + b]: hi parts at 0..8, lo parts at 9..17
__constant__ float cQ2B[18];
__constant__ float cQ2D[18];
// Gauss weight products w_{q0} w_{q1} w_{q2}: hi at 0..26, lo at 27..53
__constant__ float cQ2W[54];

struct FF {
    float h, l;
};

__device__ __forceinline__ void q2_zero(float& a) { a = 0.f; }
__device__ __forceinline__ void q2_zero(FF& a) { a = FF{0.f, 0.f}; }
// acc += tab[i] x
__device__ __forceinline__ void q2_mac(float& acc, const float* tab, int i, float x) {
    acc = fmaf(tab[i], x, acc);
}
__device__ __forceinline__ void q2_mac(FF& acc, const float* tab, int i, FF x) {
    ff_mac(tab[i], tab[9 + i], x.h, x.l, acc.h, acc.l);
}
// acc += a x
__device__ __forceinline__ void q2_fma(float& acc, float a, float x) { acc = fmaf(a, x, acc); }
__device__ __forceinline__ void q2_fma(FF& acc, FF a, FF x) { ff_mac(a.h, a.l, x.h, x.l, acc.h, acc.l); }
__device__ __forceinline__ void q2_norm(float&) {}
__device__ __forceinline__ void q2_norm(FF& a) { ff_normalize(a.h, a.l); }
__device__ __forceinline__ void q2_add(float& acc, float x) { acc += x; }
__device__ __forceinline__ void q2_add(FF& acc, FF x) { ff_sub(acc.h, acc.l, -x.h, -x.l, acc.h, acc.l); }

// The element operator on the group's 27 values in S[0] (written by the
// caller before a barrier).  t: the thread's node / Gauss point index
// t0 + 3 t1 + 9 t2.  MASS_ONLY: cm_q u(q) alone (no flux).  Every thread of
// the block calls it (it holds block barriers).  Slots: 0 input; F0 -> 1, 2;
// F1 -> 3, 4, 5; quadrature values -> 0, 1, 2, 6; R2 -> 3, 4, 5; R1 -> 0, 1.
template <typename V, bool MASS_ONLY>
__device__ __forceinline__ V q2_op(V* s[kQ2Slots], int t, const V (&G)[6], V cm) {
    const int t0 = t % 3, t1 = (t / 3) % 3, t2 = t / 9;
    // F0: along direction 0, entry (q0, b1, b2) = (t0, t1, t2)
    {
        V ab, ad;
        q2_zero(ab);
        q2_zero(ad);
#pragma unroll
        for (int b = 0; b < 3; ++b) {
            const V x = s[0][b + 3 * t1 + 9 * t2];
            q2_mac(ab, cQ2B, 3 * t0 + b, x);
            if (!MASS_ONLY) q2_mac(ad, cQ2D, 3 * t0 + b, x);
        }
        q2_norm(ab);
        q2_norm(ad);
        s[1][t] = ab;
        if (!MASS_ONLY) s[2][t] = ad;
    }
    __syncthreads();
    // F1: along direction 1, entry (q0, q1, b2)
    {
        V bb, db, bd;
        q2_zero(bb);
        q2_zero(db);
        q2_zero(bd);
#pragma unroll
        for (int b = 0; b < 3; ++b) {
            const int i = t0 + 3 * b + 9 * t2;
            const V x = s[1][i];
            q2_mac(bb, cQ2B, 3 * t1 + b, x);
            if (!MASS_ONLY) {
                q2_mac(db, cQ2B, 3 * t1 + b, s[2][i]);
                q2_mac(bd, cQ2D, 3 * t1 + b, x);
            }
        }
        q2_norm(bb);
        s[3][t] = bb;
        if (!MASS_ONLY) {
            q2_norm(db);
            q2_norm(bd);
            s[4][t] = db;
            s[5][t] = bd;
        }
    }
    __syncthreads();
    // F2: along direction 2, Gauss point q = t: the value and the reference
    // gradient, then the mass and flux terms
    {
        V val, g0, g1, g2;
        q2_zero(val);
        q2_zero(g0);
        q2_zero(g1);
        q2_zero(g2);
#pragma unroll
        for (int b = 0; b < 3; ++b) {
            const int i = t0 + 3 * t1 + 9 * b;
            const V x = s[3][i];
            q2_mac(val, cQ2B, 3 * t2 + b, x);
            if (!MASS_ONLY) {
                q2_mac(g0, cQ2B, 3 * t2 + b, s[4][i]);
                q2_mac(g1, cQ2B, 3 * t2 + b, s[5][i]);
                q2_mac(g2, cQ2D, 3 * t2 + b, x);
            }
        }
        q2_norm(val);
        V mv;
        q2_zero(mv);
        q2_fma(mv, cm, val);
        q2_norm(mv);
        s[0][t] = mv;
        if (!MASS_ONLY) {
            q2_norm(g0);
            q2_norm(g1);
            q2_norm(g2);
            // G symmetric: xx yy zz xy xz yz
            V f0, f1, f2;
            q2_zero(f0);
            q2_zero(f1);
            q2_zero(f2);
            q2_fma(f0, G[0], g0);
            q2_fma(f0, G[3], g1);
            q2_fma(f0, G[4], g2);
            q2_fma(f1, G[3], g0);
            q2_fma(f1, G[1], g1);
            q2_fma(f1, G[5], g2);
            q2_fma(f2, G[4], g0);
            q2_fma(f2, G[5], g1);
            q2_fma(f2, G[2], g2);
            q2_norm(f0);
            q2_norm(f1);
            q2_norm(f2);
            s[1][t] = f0;
            s[2][t] = f1;
            s[6][t] = f2;
        }
    }
    __syncthreads();
    // R2: transposed along direction 2, entry (q0, q1, a2)
    {
        V sa, p0, p1;
        q2_zero(sa);
        q2_zero(p0);
        q2_zero(p1);
#pragma unroll
        for (int q = 0; q < 3; ++q) {
            const int i = t0 + 3 * t1 + 9 * q;
            q2_mac(sa, cQ2B, 3 * q + t2, s[0][i]);
            if (!MASS_ONLY) {
                q2_mac(sa, cQ2D, 3 * q + t2, s[6][i]);
                q2_mac(p0, cQ2B, 3 * q + t2, s[1][i]);
                q2_mac(p1, cQ2B, 3 * q + t2, s[2][i]);
            }
        }
        q2_norm(sa);
        s[3][t] = sa;
        if (!MASS_ONLY) {
            q2_norm(p0);
            q2_norm(p1);
            s[4][t] = p0;
            s[5][t] = p1;
        }
    }
    __syncthreads();
    // R1: transposed along direction 1, entry (q0, a1, a2)
    {
        V r, qq;
        q2_zero(r);
        q2_zero(qq);
#pragma unroll
        for (int q = 0; q < 3; ++q) {
            const int i = t0 + 3 * q + 9 * t2;
            q2_mac(r, cQ2B, 3 * q + t1, s[3][i]);
            if (!MASS_ONLY) {
                q2_mac(r, cQ2D, 3 * q + t1, s[5][i]);
                q2_mac(qq, cQ2B, 3 * q + t1, s[4][i]);
            }
        }
        q2_norm(r);
        s[0][t] = r;
        if (!MASS_ONLY) {
            q2_norm(qq);
            s[1][t] = qq;
        }
    }
    __syncthreads();
    // R0: transposed along direction 0, node a = t
    V y;
    q2_zero(y);
#pragma unroll
    for (int q = 0; q < 3; ++q) {
        const int i = q + 3 * t1 + 9 * t2;
        q2_mac(y, cQ2B, 3 * q + t0, s[0][i]);
        if (!MASS_ONLY) q2_mac(y, cQ2D, 3 * q + t0, s[1][i]);
    }
    q2_norm(y);
    return y;
}

// element e's node t = t0 + 3 t1 + 9 t2
__device__ __forceinline__ int q2_node(const Dev& D, int e, int t) {
    const int ei = e % D.enx, ej = (e / D.enx) % D.eny, ek = e / (D.enx * D.eny);
    const int t0 = t % 3, t1 = (t / 3) % 3, t2 = t / 9;
    return (2 * ei + t0) + D.NX * ((2 * ej + t1) + D.NY * (2 * ek + t2));
}

// FP32 apply of the inner CG: p = z + beta p_old at the element's nodes,
// element outputs of A p.
__global__ void __launch_bounds__(kQ2Threads) k_q2_elem32(Dev* __restrict__ Dp) {
    __shared__ float sm[kQ2Slots][(kQ2Groups + 1) * 27];
    const Dev& D = *Dp;
    const int g = threadIdx.x / 27, t = threadIdx.x % 27;  // g == kQ2Groups: spare threads
    const int e = blockIdx.x * kQ2Groups + g;
    const bool valid = g < kQ2Groups && e < D.ne;
    float* s[kQ2Slots];
#pragma unroll
    for (int k = 0; k < kQ2Slots; ++k) s[k] = sm[k] + g * 27;
    const size_t EQ = (size_t)D.ne * 27;
    float G[6], cm = 0.f, x = 0.f;
#pragma unroll
    for (int c = 0; c < 6; ++c) G[c] = 0.f;
    if (valid) {
        const float beta = (float)D.beta;
        const float* __restrict__ pold = D.pswap ? D.pb32 : D.pa32;
        const int n = q2_node(D, e, t);
        x = beta == 0.f ? D.z32[n] : fmaf(beta, pold[n], D.z32[n]);
        const size_t o = (size_t)e * 27 + t;
#pragma unroll
        for (int c = 0; c < 6; ++c) G[c] = D.q2G[c * EQ + o];
        cm = (float)(D.alpha_dt * D.q2vol) * cQ2W[t];
    }
    s[0][t] = x;
    __syncthreads();
    const float y = q2_op<float, false>(s, t, G, cm);
    if (valid) D.q2Y32[(size_t)e * 27 + t] = y;
}

// Float-float element outputs for the refinement: A u (u = the iterate) and,
// FIRST, M v as well.
template <int FIRST>
__global__ void __launch_bounds__(kQ2Threads) k_q2_elem_ff(Dev* __restrict__ Dp) {
    __shared__ FF sm[kQ2Slots][(kQ2Groups + 1) * 27];
    const Dev& D = *Dp;
    if (!FIRST && !D.f_outer) return;  // uniform: the refinement is over
    const int g = threadIdx.x / 27, t = threadIdx.x % 27;
    const int e = blockIdx.x * kQ2Groups + g;
    const bool valid = g < kQ2Groups && e < D.ne;
    FF* s[kQ2Slots];
#pragma unroll
    for (int k = 0; k < kQ2Slots; ++k) s[k] = sm[k] + g * 27;
    const size_t EQ = (size_t)D.ne * 27;
    const size_t o = (size_t)e * 27 + t;
    FF G[6], cm = FF{0.f, 0.f}, x = FF{0.f, 0.f}, xv = FF{0.f, 0.f}, cv = FF{0.f, 0.f};
#pragma unroll
    for (int c = 0; c < 6; ++c) G[c] = FF{0.f, 0.f};
    if (valid) {
        const int n = q2_node(D, e, t);
        x = FF{D.u_hi[n], D.u_lo[n]};
        if (FIRST) xv = FF{D.v_hi[n], D.v_lo[n]};
#pragma unroll
        for (int c = 0; c < 6; ++c) G[c] = FF{D.q2G[c * EQ + o], D.q2G[(6 + c) * EQ + o]};
        // cm = (alpha/dt |J|) w_q and |J| w_q, the scalars rounded to
        // float-float once per thread
        float ah, al, vh, vl;
        ff_from_double(D.alpha_dt * D.q2vol, ah, al);
        ff_mul(ah, al, cQ2W[t], cQ2W[27 + t], cm.h, cm.l);
        ff_from_double(D.q2vol, vh, vl);
        ff_mul(vh, vl, cQ2W[t], cQ2W[27 + t], cv.h, cv.l);
    }
    s[0][t] = x;
    __syncthreads();
    const FF y = q2_op<FF, false>(s, t, G, cm);
    if (valid) {
        D.q2Yh[o] = y.h;
        D.q2Yl[o] = y.l;
    }
    if (FIRST) {
        __syncthreads();  // the last pass still reads slot 0
        s[0][t] = xv;
        __syncthreads();
        const FF b = q2_op<FF, true>(s, t, G, cv);
        if (valid) {
            D.q2Bh[o] = b.h;
            D.q2Bl[o] = b.l;
        }
    }
}

// The elements of node index I along one direction (ne elements): the
// element and the node's local index in it, 1 or 2 of them.
__device__ __forceinline__ int q2_incident(int I, int ne, int (&el)[2], int (&loc)[2]) {
    if (I & 1) {
        el[0] = I >> 1;
        loc[0] = 1;
        return 1;
    }
    int c = 0;
    const int k = I >> 1;
    if (k >= 1) {
        el[c] = k - 1;
        loc[c++] = 2;
    }
    if (k < ne) {
        el[c] = k;
        loc[c++] = 0;
    }
    return c;
}

// Sum of the element outputs at node n, in a fixed order (direction 0
// innermost).
template <typename V, typename Load>
__device__ __forceinline__ V q2_gather(const Dev& D, int n, Load load) {
    const int I = n % D.NX, J = (n / D.NX) % D.NY, K = n / (D.NX * D.NY);
    int ex[2], lx[2], ey[2], ly[2], ez[2], lz[2];
    const int cx = q2_incident(I, D.enx, ex, lx);
    const int cy = q2_incident(J, D.eny, ey, ly);
    const int cz = q2_incident(K, D.enz, ez, lz);
    V acc;
    q2_zero(acc);
    for (int c = 0; c < cz; ++c)
        for (int b = 0; b < cy; ++b)
            for (int a = 0; a < cx; ++a) {
                const int e = ex[a] + D.enx * (ey[b] + D.eny * ez[c]);
                q2_add(acc, load((size_t)e * 27 + lx[a] + 3 * ly[b] + 9 * lz[c]));
            }
    return acc;
}

// q = A p, the new direction p, and alpha = (r . z) / (p . q): the same
// contract as the other FP32 applies of the inner CG.
__global__ void __launch_bounds__(kNodeThreads) k_q2_gather32(Dev* __restrict__ Dp) {
    Dev& D = *Dp;
    const float beta = (float)D.beta;
    const float* __restrict__ pold = D.pswap ? D.pb32 : D.pa32;
    float* __restrict__ pnew = D.pswap ? D.pa32 : D.pb32;
    const float* __restrict__ Y = D.q2Y32;
    float v[1] = {0.f};
    const double none[1] = {0.0};
    for (int n = blockIdx.x * blockDim.x + threadIdx.x; n < D.N; n += gridDim.x * blockDim.x) {
        const float q = q2_gather<float>(D, n, [&](size_t i) { return Y[i]; });
        const float p = beta == 0.f ? D.z32[n] : fmaf(beta, pold[n], D.z32[n]);
        pnew[n] = p;
        D.q32[n] = q;
        v[0] = fmaf(p, q, v[0]);
    }
    grid_reduce<1, 0>(v, none, D.partial, D.counter + CNT_APPLY, blockIdx.x, gridDim.x,
                      [&](double* tot) { D.alpha = D.rz / tot[0]; });
}

// FIRST: b = M v; otherwise b as stored.  r = b - A u, the inner solver's
// start (r32, z32 = D^-1 r32, delta = 0) and the refinement's decisions.
template <int FIRST>
__global__ void __launch_bounds__(kNodeThreads) k_q2_gather_ff(Dev* __restrict__ Dp, int graph) {
    Dev& D = *Dp;
    if (!FIRST && !D.f_outer) return;
    const float ns = D.nscale;
    float vf[4] = {0.f, 0.f, 0.f, 0.f};
    const double none[1] = {0.0};
    for (int n = blockIdx.x * blockDim.x + threadIdx.x; n < D.N; n += gridDim.x * blockDim.x) {
        const FF y = q2_gather<FF>(D, n, [&](size_t i) { return FF{D.q2Yh[i], D.q2Yl[i]}; });
        FF b;
        if (FIRST) {
            b = q2_gather<FF>(D, n, [&](size_t i) { return FF{D.q2Bh[i], D.q2Bl[i]}; });
            D.b_hi[n] = b.h;
            D.b_lo[n] = b.l;
        } else {
            b = FF{D.b_hi[n], D.b_lo[n]};
        }
        float rh, rl;
        ff_sub(b.h, b.l, y.h, y.l, rh, rl);
        const float r32 = rh;
        const float z = D.dinv32[n] * r32;
        D.r32[n] = r32;
        D.z32[n] = z;
        D.d32[n] = 0.0f;
        const float bs = ns * b.h, rs = ns * rh;
        vf[0] = fmaf(bs, bs, vf[0]);
        vf[1] = fmaf(rs, rs, vf[1]);
        vf[2] = fmaf(r32, z, vf[2]);
        vf[3] = fmaf(r32, r32, vf[3]);
    }
    grid_reduce<4, 0>(vf, none, D.partial, D.counter + CNT_RHS, blockIdx.x, gridDim.x,
                      [&](double* t) { rhs_finish(D, t, FIRST != 0, graph, ns); });
}

// A BDF order change: the Jacobi diagonal from the stored diagonals of M and K.
__global__ void k_realpha_q2(Dev* __restrict__ Dp, double alpha_dt) {
    Dev& D = *Dp;
    const int n = blockIdx.x * blockDim.x + threadIdx.x;
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        D.alpha_dt = alpha_dt;
        D.hist = 0;
    }
    if (n < D.N) D.dinv32[n] = (float)(1.0 / (alpha_dt * D.q2dM[n] + D.q2dK[n]));
}

// ---- host side ---------------------------------------------------------------

// The 1-D tables in double, rounded to float-float pairs.
cudaError_t q2_upload_tables() {
    const double r = std::sqrt(15.0) / 10.0;
    const double xq[3] = {0.5 - r, 0.5, 0.5 + r};
    const double w1[3] = {5.0 / 18.0, 8.0 / 18.0, 5.0 / 18.0};
    float B[18], Dd[18], W[54];
    auto split = [](double x, float& hi, float& lo) {
        hi = (float)x;
        lo = (float)(x - (double)hi);
    };
    for (int q = 0; q < 3; ++q) {
        const double t = xq[q];
        const double l[3] = {(1.0 - t) * (1.0 - 2.0 * t), 4.0 * t * (1.0 - t), t * (2.0 * t - 1.0)};
        const double d[3] = {4.0 * t - 3.0, 4.0 - 8.0 * t, 4.0 * t - 1.0};
        for (int b = 0; b < 3; ++b) {
            split(l[b], B[3 * q + b], B[9 + 3 * q + b]);
            split(d[b], Dd[3 * q + b], Dd[9 + 3 * q + b]);
        }
    }
    for (int q = 0; q < 27; ++q) split(w1[q % 3] * w1[(q / 3) % 3] * w1[q / 9], W[q], W[27 + q]);
    cudaError_t e = cudaMemcpyToSymbol(cQ2B, B, sizeof(B));
    if (e == cudaSuccess) e = cudaMemcpyToSymbol(cQ2D, Dd, sizeof(Dd));
    if (e == cudaSuccess) e = cudaMemcpyToSymbol(cQ2W, W, sizeof(W));
    return e;
}

int q2_elem_blocks(const Dev& h) { return (h.ne + kQ2Groups - 1) / kQ2Groups; }

void launch_q2_apply32(Dev* d, const Dev& h, int grid_nodes, cudaStream_t s) {
    k_q2_elem32<<<q2_elem_blocks(h), kQ2Threads, 0, s>>>(d);
    k_q2_gather32<<<grid_nodes, kNodeThreads, 0, s>>>(d);
}

void launch_q2_resid(Dev* d, const Dev& h, int first, int graph, int grid_nodes, cudaStream_t s) {
    if (first) {
        k_q2_elem_ff<1><<<q2_elem_blocks(h), kQ2Threads, 0, s>>>(d);
        k_q2_gather_ff<1><<<grid_nodes, kNodeThreads, 0, s>>>(d, graph);
    } else {
        k_q2_elem_ff<0><<<q2_elem_blocks(h), kQ2Threads, 0, s>>>(d);
        k_q2_gather_ff<0><<<grid_nodes, kNodeThreads, 0, s>>>(d, graph);
    }
}

void launch_realpha_q2(Dev* d, const Dev& h, double alpha_dt, cudaStream_t s) {
    k_realpha_q2<<<(h.N + 255) / 256, 256, 0, s>>>(d, alpha_dt);
}

}  // namespace epk
