// k_q2.cu -- matrix-free operators of triquadratic (Q2, 27-node) hexahedra on
// slab meshes (Sec. 1.2: hexahedral elements of any degree; Sec. 4 names
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
// Work decomposition.  FP32 apply (the inner CG's operator): one thread per
// element, the whole sum factorisation in registers with the 1-D
// coefficients as immediates, flux matrices read element-fastest.  Float-
// float passes (the refinement's right-hand side b = M v and residual
// b - A u, ep_ff.cuh): nine threads per element, one per 1-D pencil of the
// pass, the intermediate arrays in shared memory between the passes.  Every
// element writes its 27 outputs to a per-element buffer; a node-parallel
// gather then sums the contributions of the node's 1, 2, 4 or 8 elements in
// a fixed order (no atomics: bitwise reproducible).
#include <cmath>

#include "ep_dev.cuh"
#include "ep_ff.cuh"
#include "ep_refine.cuh"

namespace epk {

struct __align__(8) FF {
    float h, l;
};

__device__ __forceinline__ void q2_zero(float& a) { a = 0.f; }
__device__ __forceinline__ void q2_zero(FF& a) { a = FF{0.f, 0.f}; }
__device__ __forceinline__ void q2_add(float& acc, float x) { acc += x; }
__device__ __forceinline__ void q2_add(FF& acc, FF x) { ff_sub(acc.h, acc.l, -x.h, -x.l, acc.h, acc.l); }

// 1-D quadratic Lagrange basis on [0,1] (nodes 0, 1/2, 1), l_b(xi_q), and
// its derivative l_b'(xi_q) at the 3-point Gauss points xi = 1/2 -+
// sqrt(15)/10, 1/2 (rounded to float), and the Gauss weights 5/18, 8/18,
// 5/18: compile-time constants of the FP32 apply (the float-float kernels
// take them as float-float pairs, below).
__host__ __device__ constexpr float q2b(int q, int b) {
    return q == 0 ? (b == 0 ? 0.68729836f : b == 1 ? 0.4f : -0.08729833f)
           : q == 1 ? (b == 0 ? 0.0f : b == 1 ? 1.0f : 0.0f)
           : (b == 0 ? -0.08729833f : b == 1 ? 0.4f : 0.68729836f);
}
__host__ __device__ constexpr float q2db(int q, int b) {
    return q == 0 ? (b == 0 ? -2.5491934f : b == 1 ? 3.0983868f : -0.5491933f)
           : q == 1 ? (b == 0 ? -1.0f : b == 1 ? 0.0f : 1.0f)
           : (b == 0 ? 0.5491933f : b == 1 ? -3.0983868f : 2.5491934f);
}
__host__ __device__ constexpr float q2w(int q) { return q == 1 ? 0.44444445f : 0.2777778f; }
#define Q2B(q, b) q2b((q), (b))
#define Q2D(q, b) q2db((q), (b))

// c0 x0 + c1 x1 + c2 x2 for compile-time coefficients; a zero coefficient
// drops its term (l_b at the middle Gauss point is 0, 1, 0)
__device__ __forceinline__ float q2dot(float c0, float x0, float c1, float x1, float c2, float x2) {
    float acc = c2 == 0.f ? 0.f : c2 * x2;
    acc = c1 == 0.f ? acc : fmaf(c1, x1, acc);
    return c0 == 0.f ? acc : fmaf(c0, x0, acc);
}

// FP32 apply of the inner CG, one thread per element with the whole sum
// factorisation in registers (the 1-D coefficients are immediates): p =
// z + beta p_old at the element's 27 nodes, the element outputs of A p,
// node-major [27][ne].  The flux matrices are read from their element-fastest
// FP32 copy [6][27][ne] (coalesced).
__global__ void __launch_bounds__(128, 4) k_q2_elem32(Dev* __restrict__ Dp) {
    const Dev& D = *Dp;
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= D.ne) return;
    const int ei = e % D.enx, ej = (e / D.enx) % D.eny, ek = e / (D.enx * D.eny);
    const int NX = D.NX, NXY = D.NX * D.NY;
    const int n0 = 2 * ei + NX * (2 * ej) + NXY * (2 * ek);
    const float beta = (float)D.beta;
    const float* __restrict__ z = D.z32;
    const float* __restrict__ pold = D.pswap ? D.pb32 : D.pa32;
    // F0 (direction 0) straight from the nodal values, pencil by pencil
    float ab[27], ad[27];
#pragma unroll
    for (int r = 0; r < 9; ++r) {  // r = b1 + 3 b2
        const int n = n0 + NX * (r % 3) + NXY * (r / 3);
        float x[3];
#pragma unroll
        for (int b = 0; b < 3; ++b) x[b] = beta == 0.f ? z[n + b] : fmaf(beta, pold[n + b], z[n + b]);
#pragma unroll
        for (int q = 0; q < 3; ++q) {
            ab[q + 3 * r] = q2dot(Q2B(q, 0), x[0], Q2B(q, 1), x[1], Q2B(q, 2), x[2]);
            ad[q + 3 * r] = q2dot(Q2D(q, 0), x[0], Q2D(q, 1), x[1], Q2D(q, 2), x[2]);
        }
    }
    // F1 (direction 1): index q0 + 3 q1 + 9 b2
    float bb[27], db[27], bd[27];
#pragma unroll
    for (int q0 = 0; q0 < 3; ++q0)
#pragma unroll
        for (int b2 = 0; b2 < 3; ++b2) {
            const int i = q0 + 9 * b2;
#pragma unroll
            for (int q1 = 0; q1 < 3; ++q1) {
                bb[i + 3 * q1] = q2dot(Q2B(q1, 0), ab[i], Q2B(q1, 1), ab[i + 3], Q2B(q1, 2), ab[i + 6]);
                db[i + 3 * q1] = q2dot(Q2B(q1, 0), ad[i], Q2B(q1, 1), ad[i + 3], Q2B(q1, 2), ad[i + 6]);
                bd[i + 3 * q1] = q2dot(Q2D(q1, 0), ab[i], Q2D(q1, 1), ab[i + 3], Q2D(q1, 2), ab[i + 6]);
            }
        }
    // F2 (direction 2), the quadrature-point terms and R2 (direction 2,
    // transposed), pencil by pencil over (q0, q1)
    const size_t E = (size_t)D.ne;
    const float* __restrict__ G = D.q2G32;
    const float adtv = (float)(D.alpha_dt * D.q2vol);
    float sa[27], p0[27], p1[27];
#pragma unroll
    for (int c = 0; c < 9; ++c) {  // c = q0 + 3 q1
        float mv[3], f0[3], f1[3], f2[3];
#pragma unroll
        for (int q2 = 0; q2 < 3; ++q2) {
            const float val = q2dot(Q2B(q2, 0), bb[c], Q2B(q2, 1), bb[c + 9], Q2B(q2, 2), bb[c + 18]);
            const float g0 = q2dot(Q2B(q2, 0), db[c], Q2B(q2, 1), db[c + 9], Q2B(q2, 2), db[c + 18]);
            const float g1 = q2dot(Q2B(q2, 0), bd[c], Q2B(q2, 1), bd[c + 9], Q2B(q2, 2), bd[c + 18]);
            const float g2 = q2dot(Q2D(q2, 0), bb[c], Q2D(q2, 1), bb[c + 9], Q2D(q2, 2), bb[c + 18]);
            const int q = c + 9 * q2;
            const float* Gq = G + (size_t)q * E + e;
            const float gxx = Gq[0], gyy = Gq[27 * E], gzz = Gq[54 * E];
            const float gxy = Gq[81 * E], gxz = Gq[108 * E], gyz = Gq[135 * E];
            const float w = q2w(c % 3) * q2w(c / 3) * q2w(q2);
            mv[q2] = adtv * w * val;
            f0[q2] = fmaf(gxx, g0, fmaf(gxy, g1, gxz * g2));
            f1[q2] = fmaf(gxy, g0, fmaf(gyy, g1, gyz * g2));
            f2[q2] = fmaf(gxz, g0, fmaf(gyz, g1, gzz * g2));
        }
#pragma unroll
        for (int a2 = 0; a2 < 3; ++a2) {
            sa[c + 9 * a2] = q2dot(Q2B(0, a2), mv[0], Q2B(1, a2), mv[1], Q2B(2, a2), mv[2]) +
                             q2dot(Q2D(0, a2), f2[0], Q2D(1, a2), f2[1], Q2D(2, a2), f2[2]);
            p0[c + 9 * a2] = q2dot(Q2B(0, a2), f0[0], Q2B(1, a2), f0[1], Q2B(2, a2), f0[2]);
            p1[c + 9 * a2] = q2dot(Q2B(0, a2), f1[0], Q2B(1, a2), f1[1], Q2B(2, a2), f1[2]);
        }
    }
    // R1 (direction 1, transposed): index q0 + 3 a1 + 9 a2
    float rr[27], qq[27];
#pragma unroll
    for (int q0 = 0; q0 < 3; ++q0)
#pragma unroll
        for (int a2 = 0; a2 < 3; ++a2) {
            const int i = q0 + 9 * a2;
#pragma unroll
            for (int a1 = 0; a1 < 3; ++a1) {
                rr[i + 3 * a1] = q2dot(Q2B(0, a1), sa[i], Q2B(1, a1), sa[i + 3], Q2B(2, a1), sa[i + 6]) +
                                 q2dot(Q2D(0, a1), p1[i], Q2D(1, a1), p1[i + 3], Q2D(2, a1), p1[i + 6]);
                qq[i + 3 * a1] = q2dot(Q2B(0, a1), p0[i], Q2B(1, a1), p0[i + 3], Q2B(2, a1), p0[i + 6]);
            }
        }
    // R0 (direction 0, transposed) and the store into the node slots: slot
    // bit d is 1 where the node is this element's first node along d (local
    // index 0), so the (up to 8) elements of a node write distinct slots
    float* __restrict__ Y = D.q2Y32;
    const size_t NN = (size_t)D.N;
#pragma unroll
    for (int r = 0; r < 9; ++r) {
#pragma unroll
        for (int a0 = 0; a0 < 3; ++a0) {
            const float y = q2dot(Q2B(0, a0), rr[3 * r], Q2B(1, a0), rr[3 * r + 1], Q2B(2, a0), rr[3 * r + 2]) +
                            q2dot(Q2D(0, a0), qq[3 * r], Q2D(1, a0), qq[3 * r + 1], Q2D(2, a0), qq[3 * r + 2]);
            const int a1 = r % 3, a2 = r / 3;
            const int slot = (a0 == 0) + 2 * (a1 == 0) + 4 * (a2 == 0);
            Y[(size_t)slot * NN + n0 + a0 + NX * a1 + NXY * a2] = y;
        }
    }
}

// Sum of node n's slots (1, 2, 4 or 8 of them: along each direction slot 1
// holds the element the node starts, slot 0 the element it ends or is
// interior to) in a fixed order; load(slot) returns one.
template <typename V, typename Load>
__device__ __forceinline__ V q2_gather_slots_v(const Dev& D, int n, Load load) {
    const int I = n % D.NX, J = (n / D.NX) % D.NY, K = n / (D.NX * D.NY);
    const bool x0 = (I & 1) || I > 0, x1 = !(I & 1) && I < D.NX - 1;
    const bool y0 = (J & 1) || J > 0, y1 = !(J & 1) && J < D.NY - 1;
    const bool z0 = (K & 1) || K > 0, z1 = !(K & 1) && K < D.NZ - 1;
    V acc;
    q2_zero(acc);
#pragma unroll
    for (int s = 0; s < 8; ++s) {
        const bool ok = ((s & 1) ? x1 : x0) && ((s & 2) ? y1 : y0) && ((s & 4) ? z1 : z0);
        if (ok) q2_add(acc, load(s));
    }
    return acc;
}
__device__ __forceinline__ float q2_gather_slots(const Dev& D, int n, const float* __restrict__ Y) {
    const size_t NN = (size_t)D.N;
    return q2_gather_slots_v<float>(D, n, [&](int s) { return Y[(size_t)s * NN + n]; });
}

// The 1-D tables as float-float pairs (hi, lo of the double values), for
// the float-float kernels below: compile-time constants.
__host__ __device__ constexpr float q2bh(int q, int b) { return q2b(q, b); }
__host__ __device__ constexpr float q2bl(int q, int b) {
    return q == 1 ? 0.0f
                  : (b == 1 ? -5.9604646e-09f : (q == 0) == (b == 0) ? -2.2865983e-08f : -9.758747e-10f);
}
__host__ __device__ constexpr float q2dh(int q, int b) { return q2db(q, b); }
__host__ __device__ constexpr float q2dl(int q, int b) {
    return q == 1 ? 0.0f
           : q == 0 ? (b == 0 ? 4.378022e-08f : b == 1 ? -8.756044e-08f : -1.5824428e-08f)
                    : (b == 0 ? 1.5824428e-08f : b == 1 ? 8.756044e-08f : -4.378022e-08f);
}
// product of three Gauss weights, k of them 8/18 (the others 5/18)
__device__ __forceinline__ FF q2wff(int k) {
    return k == 0 ? FF{0.02143347f, -2.631721e-10f}
           : k == 1 ? FF{0.03429355f, 1.8140989e-09f}
           : k == 2 ? FF{0.054869685f, -8.2273216e-10f}
                    : FF{0.087791495f, 1.7374466e-10f};
}

// acc += c x for a compile-time float-float coefficient (hi, lo); a zero
// coefficient drops the term
__device__ __forceinline__ void q2fm(FF& acc, float ch, float cl, FF x) {
    if (ch != 0.f) ff_mac(ch, cl, x.h, x.l, acc.h, acc.l);
}
#define Q2FB(acc, q, b, x) q2fm(acc, q2bh(q, b), q2bl(q, b), x)
#define Q2FD(acc, q, b, x) q2fm(acc, q2dh(q, b), q2dl(q, b), x)

constexpr int kQ2PEl = 28;  // elements per block of the float-float kernels (9 threads each)

// The float-float element operator with one thread per 1-D pencil: in each
// pass the thread takes the three values of its pencil from shared memory
// and produces the three outputs along the pass's direction (coefficients
// are immediates, every thread uses all of them).  j = j0 + 3 j1 selects the
// pencil.  A and Bf: the element's two 81-entry arrays in shared memory.
// MASS_ONLY: cm_q u(q) alone.  Every thread of the block calls it.
template <bool MASS_ONLY>
__device__ __forceinline__ void q2_op_ff(const Dev& D, bool valid, int e, int j0, int j1, const FF (&x)[3],
                                         FF* A, FF* Bf, FF cmv, FF (&y)[3]) {
    const FF z0 = FF{0.f, 0.f};
    // F0: pencil (b1, b2) = (j0, j1) along direction 0 -> A[q0 + 3 b1 + 9 b2]
    {
        const int o = 3 * j0 + 9 * j1;
#pragma unroll
        for (int q = 0; q < 3; ++q) {
            FF ab = z0, ad = z0;
#pragma unroll
            for (int b = 0; b < 3; ++b) {
                Q2FB(ab, q, b, x[b]);
                if (!MASS_ONLY) Q2FD(ad, q, b, x[b]);
            }
            ff_normalize(ab.h, ab.l);
            A[q + o] = ab;
            if (!MASS_ONLY) {
                ff_normalize(ad.h, ad.l);
                A[27 + q + o] = ad;
            }
        }
    }
    __syncthreads();
    // F1: pencil (q0, b2) = (j0, j1) along direction 1 -> Bf[q0 + 3 q1 + 9 b2]
    {
        FF ab[3], ad[3];
#pragma unroll
        for (int b = 0; b < 3; ++b) {
            ab[b] = A[j0 + 3 * b + 9 * j1];
            if (!MASS_ONLY) ad[b] = A[27 + j0 + 3 * b + 9 * j1];
        }
#pragma unroll
        for (int q = 0; q < 3; ++q) {
            FF bb = z0, db = z0, bd = z0;
#pragma unroll
            for (int b = 0; b < 3; ++b) {
                Q2FB(bb, q, b, ab[b]);
                if (!MASS_ONLY) {
                    Q2FB(db, q, b, ad[b]);
                    Q2FD(bd, q, b, ab[b]);
                }
            }
            const int i = j0 + 3 * q + 9 * j1;
            ff_normalize(bb.h, bb.l);
            Bf[i] = bb;
            if (!MASS_ONLY) {
                ff_normalize(db.h, db.l);
                ff_normalize(bd.h, bd.l);
                Bf[27 + i] = db;
                Bf[54 + i] = bd;
            }
        }
    }
    __syncthreads();
    // F2 + quadrature point terms + R2: pencil (q0, q1) = (j0, j1) along
    // direction 2 -> A[q0 + 3 q1 + 9 a2]
    {
        const int c = j0 + 3 * j1;
        FF bb[3], db[3], bd[3];
#pragma unroll
        for (int b = 0; b < 3; ++b) {
            bb[b] = Bf[c + 9 * b];
            if (!MASS_ONLY) {
                db[b] = Bf[27 + c + 9 * b];
                bd[b] = Bf[54 + c + 9 * b];
            }
        }
        FF mv[3], f0[3], f1[3], f2[3];
        const size_t EQ = (size_t)D.ne * 27;
        const int kw = (j0 == 1) + (j1 == 1);
#pragma unroll
        for (int q = 0; q < 3; ++q) {
            FF val = z0, g0 = z0, g1 = z0, g2 = z0;
#pragma unroll
            for (int b = 0; b < 3; ++b) {
                Q2FB(val, q, b, bb[b]);
                if (!MASS_ONLY) {
                    Q2FB(g0, q, b, db[b]);
                    Q2FB(g1, q, b, bd[b]);
                    Q2FD(g2, q, b, bb[b]);
                }
            }
            ff_normalize(val.h, val.l);
            // mass term cm_q u(q): (alpha/dt |J| or |J|) x w_q
            const FF w = q2wff(kw + (q == 1));
            FF cq;
            ff_mul(cmv.h, cmv.l, w.h, w.l, cq.h, cq.l);
            FF m = z0;
            ff_mac(cq.h, cq.l, val.h, val.l, m.h, m.l);
            ff_normalize(m.h, m.l);
            mv[q] = m;
            if (!MASS_ONLY) {
                ff_normalize(g0.h, g0.l);
                ff_normalize(g1.h, g1.l);
                ff_normalize(g2.h, g2.l);
                FF G[6];
                const size_t o = (size_t)e * 27 + c + 9 * q;
#pragma unroll
                for (int k = 0; k < 6; ++k)
                    G[k] = valid ? FF{D.q2G[k * EQ + o], D.q2G[(6 + k) * EQ + o]} : z0;
                FF a0 = z0, a1 = z0, a2 = z0;
                ff_mac(G[0].h, G[0].l, g0.h, g0.l, a0.h, a0.l);
                ff_mac(G[3].h, G[3].l, g1.h, g1.l, a0.h, a0.l);
                ff_mac(G[4].h, G[4].l, g2.h, g2.l, a0.h, a0.l);
                ff_mac(G[3].h, G[3].l, g0.h, g0.l, a1.h, a1.l);
                ff_mac(G[1].h, G[1].l, g1.h, g1.l, a1.h, a1.l);
                ff_mac(G[5].h, G[5].l, g2.h, g2.l, a1.h, a1.l);
                ff_mac(G[4].h, G[4].l, g0.h, g0.l, a2.h, a2.l);
                ff_mac(G[5].h, G[5].l, g1.h, g1.l, a2.h, a2.l);
                ff_mac(G[2].h, G[2].l, g2.h, g2.l, a2.h, a2.l);
                ff_normalize(a0.h, a0.l);
                ff_normalize(a1.h, a1.l);
                ff_normalize(a2.h, a2.l);
                f0[q] = a0;
                f1[q] = a1;
                f2[q] = a2;
            }
        }
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            FF sa = z0, p0 = z0, p1 = z0;
#pragma unroll
            for (int q = 0; q < 3; ++q) {
                Q2FB(sa, q, a, mv[q]);
                if (!MASS_ONLY) {
                    Q2FD(sa, q, a, f2[q]);
                    Q2FB(p0, q, a, f0[q]);
                    Q2FB(p1, q, a, f1[q]);
                }
            }
            const int i = c + 9 * a;
            ff_normalize(sa.h, sa.l);
            A[i] = sa;
            if (!MASS_ONLY) {
                ff_normalize(p0.h, p0.l);
                ff_normalize(p1.h, p1.l);
                A[27 + i] = p0;
                A[54 + i] = p1;
            }
        }
    }
    __syncthreads();
    // R1: pencil (q0, a2) = (j0, j1) along direction 1 -> Bf[q0 + 3 a1 + 9 a2]
    {
        FF sa[3], p0[3], p1[3];
#pragma unroll
        for (int q = 0; q < 3; ++q) {
            const int i = j0 + 3 * q + 9 * j1;
            sa[q] = A[i];
            if (!MASS_ONLY) {
                p0[q] = A[27 + i];
                p1[q] = A[54 + i];
            }
        }
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            FF r = z0, qq = z0;
#pragma unroll
            for (int q = 0; q < 3; ++q) {
                Q2FB(r, q, a, sa[q]);
                if (!MASS_ONLY) {
                    Q2FD(r, q, a, p1[q]);
                    Q2FB(qq, q, a, p0[q]);
                }
            }
            const int i = j0 + 3 * a + 9 * j1;
            ff_normalize(r.h, r.l);
            Bf[i] = r;
            if (!MASS_ONLY) {
                ff_normalize(qq.h, qq.l);
                Bf[27 + i] = qq;
            }
        }
    }
    __syncthreads();
    // R0: pencil (a1, a2) = (j0, j1) along direction 0 -> y[a0]
    {
        FF r[3], qq[3];
#pragma unroll
        for (int q = 0; q < 3; ++q) {
            const int i = q + 3 * j0 + 9 * j1;
            r[q] = Bf[i];
            if (!MASS_ONLY) qq[q] = Bf[27 + i];
        }
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            FF acc = z0;
#pragma unroll
            for (int q = 0; q < 3; ++q) {
                Q2FB(acc, q, a, r[q]);
                if (!MASS_ONLY) Q2FD(acc, q, a, qq[q]);
            }
            ff_normalize(acc.h, acc.l);
            y[a] = acc;
        }
    }
}

// Float-float element outputs for the refinement: A u (u = the iterate) and,
// FIRST, M v as well; 9 threads (pencils) per element, 28 elements per
// block.
template <int FIRST>
__global__ void __launch_bounds__(9 * kQ2PEl) k_q2_elem_ff(Dev* __restrict__ Dp) {
    __shared__ FF smA[kQ2PEl][81];
    __shared__ FF smB[kQ2PEl][81];
    const Dev& D = *Dp;
    if (!FIRST && !D.f_outer) return;  // uniform: the refinement is over
    const int g = threadIdx.x / 9, j = threadIdx.x % 9;
    const int j0 = j % 3, j1 = j / 3;
    const int e = blockIdx.x * kQ2PEl + g;
    const bool valid = e < D.ne;
    int n = 0;
    if (valid) {
        const int ei = e % D.enx, ej = (e / D.enx) % D.eny, ek = e / (D.enx * D.eny);
        n = (2 * ei) + D.NX * ((2 * ej + j0) + D.NY * (2 * ek + j1));
    }
    FF x[3];
#pragma unroll
    for (int b = 0; b < 3; ++b) x[b] = valid ? FF{D.u_hi[n + b], D.u_lo[n + b]} : FF{0.f, 0.f};
    FF cm;
    ff_from_double(D.alpha_dt * D.q2vol, cm.h, cm.l);
    FF y[3];
    q2_op_ff<false>(D, valid, e, j0, j1, x, smA[g], smB[g], cm, y);
    // outputs a = a0 + 3 a1 + 9 a2, (a1, a2) = (j0, j1), into the node slots
    // (as the FP32 apply's)
    const size_t NN = (size_t)D.N;
    const int sl = 2 * (j0 == 0) + 4 * (j1 == 0);
    if (valid) {
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            const size_t o = (size_t)(sl + (a == 0)) * NN + n + a;
            D.q2Yh[o] = y[a].h;
            D.q2Yl[o] = y[a].l;
        }
    }
    if (FIRST) {
        FF xv[3];
#pragma unroll
        for (int b = 0; b < 3; ++b) xv[b] = valid ? FF{D.v_hi[n + b], D.v_lo[n + b]} : FF{0.f, 0.f};
        FF cv;
        ff_from_double(D.q2vol, cv.h, cv.l);
        q2_op_ff<true>(D, valid, e, j0, j1, xv, smA[g], smB[g], cv, y);
        if (valid) {
#pragma unroll
            for (int a = 0; a < 3; ++a) {
                const size_t o = (size_t)(sl + (a == 0)) * NN + n + a;
                D.q2Bh[o] = y[a].h;
                D.q2Bl[o] = y[a].l;
            }
        }
    }
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
        const float q = q2_gather_slots(D, n, Y);
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
        const size_t NN = (size_t)D.N;
        const FF y = q2_gather_slots_v<FF>(D, n, [&](int s) {
            const size_t i = (size_t)s * NN + n;
            return FF{D.q2Yh[i], D.q2Yl[i]};
        });
        FF b;
        if (FIRST) {
            b = q2_gather_slots_v<FF>(D, n, [&](int s) {
                const size_t i = (size_t)s * NN + n;
                return FF{D.q2Bh[i], D.q2Bl[i]};
            });
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

void launch_q2_apply32(Dev* d, const Dev& h, int grid_nodes, cudaStream_t s) {
    k_q2_elem32<<<(h.ne + 127) / 128, 128, 0, s>>>(d);
    k_q2_gather32<<<grid_nodes, kNodeThreads, 0, s>>>(d);
}

void launch_q2_resid(Dev* d, const Dev& h, int first, int graph, int grid_nodes, cudaStream_t s) {
    const int eb = (h.ne + kQ2PEl - 1) / kQ2PEl;
    if (first) {
        k_q2_elem_ff<1><<<eb, 9 * kQ2PEl, 0, s>>>(d);
        k_q2_gather_ff<1><<<grid_nodes, kNodeThreads, 0, s>>>(d, graph);
    } else {
        k_q2_elem_ff<0><<<eb, 9 * kQ2PEl, 0, s>>>(d);
        k_q2_gather_ff<0><<<grid_nodes, kNodeThreads, 0, s>>>(d, graph);
    }
}

void launch_realpha_q2(Dev* d, const Dev& h, double alpha_dt, cudaStream_t s) {
    k_realpha_q2<<<(h.N + 255) / 256, 256, 0, s>>>(d, alpha_dt);
}

}  // namespace epk
