// k_mf.cu -- matrix-free FP32 apply of A = alpha/dt M + K on slab meshes
// (axis-aligned Q1 hexahedra of size hx x hy x hz).
//
// Paper Sec. 1.2, Eq. (6) with D of Eq. (3): per element and 2x2x2 Gauss
// point q (reference coordinates xi in [0,1]^3, weights 1/8),
//   y_a += (hx hy hz / 8) grad_xi phi_a . (H D_q H) grad_xi p,   H = diag(1/h),
//   H D_q H = dn H^2 + (dl - dn) f' f'^T + (dt - dn) s' s'^T,
// with f' = H f0 and s' = H s0 interpolated trilinearly from the nodes
// (stored pre-scaled, so interpolation and scaling commute), plus the mass
// term alpha/dt hx hy hz (m x m x m) p with m = [[1/3,1/6],[1/6,1/3]], which
// 2-point Gauss integrates exactly.
//
// Work decomposition: a block owns a kMfTx x kMfTy x kMfTz box of nodes.  It
// stages the box plus a one-node halo (p, f', s' as SoA) in shared memory,
// forming p = z + beta p_old on the way in (the CG direction update), has
// each thread evaluate whole elements of the (box+1)^3 element set touching
// the box, writes the 8 corner contributions per element to shared memory,
// then every owned node sums its 8 contributions in a fixed order.  No
// atomics: results are bitwise reproducible.
#include "ep_dev.cuh"

namespace epk {

constexpr int HX = kMfTx + 2, HY = kMfTy + 2, HZ = kMfTz + 2;
constexpr int HN = HX * HY * HZ;                      // halo nodes
constexpr int EX = kMfTx + 1, EY = kMfTy + 1, EZ = kMfTz + 1;
constexpr int EN = EX * EY * EZ;                      // elements
constexpr size_t kMfSmem = sizeof(float) * (7 * HN + 8 * EN);

// Gauss points of [0,1]: G0 = (1 - 1/sqrt 3)/2, G1 = (1 + 1/sqrt 3)/2;
// l_0(xi) = 1 - xi, l_1(xi) = xi, so L[q][b] = l_b(xi_q) = (q == b) ? G1 : G0.
constexpr float G0 = 0.21132486540518711775f;
constexpr float G1 = 0.78867513459481288225f;

// out[q] = sum_b L[q][b] in[b] along one direction (L is symmetric, so the
// same map is its own transpose)
__device__ __forceinline__ void lmap(float a, float b, float& o0, float& o1) {
    o0 = fmaf(G1, a, G0 * b);
    o1 = fmaf(G0, a, G1 * b);
}

// Trilinear values at the 8 Gauss points from the 8 nodal values
// (index = i0 + 2 i1 + 4 i2 on both sides).
__device__ __forceinline__ void interp8(const float v[8], float o[8]) {
    float t[8], u[8];
#pragma unroll
    for (int r = 0; r < 4; ++r) lmap(v[2 * r], v[2 * r + 1], t[2 * r], t[2 * r + 1]);  // dir 0
#pragma unroll
    for (int c2 = 0; c2 < 2; ++c2)
#pragma unroll
        for (int c0 = 0; c0 < 2; ++c0)
            lmap(t[c0 + 4 * c2], t[c0 + 2 + 4 * c2], u[c0 + 4 * c2], u[c0 + 2 + 4 * c2]);  // dir 1
#pragma unroll
    for (int c = 0; c < 4; ++c) lmap(u[c], u[c + 4], o[c], o[c + 4]);  // dir 2
}

// 2-D version on a 2x2 array (index i + 2 j)
__device__ __forceinline__ void interp4(const float v[4], float o[4]) {
    float t[4];
    lmap(v[0], v[1], t[0], t[1]);
    lmap(v[2], v[3], t[2], t[3]);
    lmap(t[0], t[2], o[0], o[2]);
    lmap(t[1], t[3], o[1], o[3]);
}

__global__ void __launch_bounds__(kMfThreads) k_apply32_mf(Dev* __restrict__ Dp) {
    extern __shared__ float smem[];
    float* s_p = smem;
    float* s_f = s_p + HN;       // [3][HN]
    float* s_s = s_f + 3 * HN;   // [3][HN]
    float* s_y = s_s + 3 * HN;   // [8][EN]

    Dev& D = *Dp;
    const int NX = D.NX, NY = D.NY, NZ = D.NZ, N = D.N;
    const int tx = (NX + kMfTx - 1) / kMfTx, ty = (NY + kMfTy - 1) / kMfTy;
    const int bi = blockIdx.x % tx, bj = (blockIdx.x / tx) % ty, bk = blockIdx.x / (tx * ty);
    const int i0 = bi * kMfTx, j0 = bj * kMfTy, k0 = bk * kMfTz;
    const float beta = (float)D.beta;
    const float* __restrict__ z = D.z32;
    const float* __restrict__ pold = D.pswap ? D.pb32 : D.pa32;
    float* __restrict__ pnew = D.pswap ? D.pa32 : D.pb32;
    const float* __restrict__ fib = D.fib;

    // ---- stage the halo box -------------------------------------------------
    for (int h = threadIdx.x; h < HN; h += blockDim.x) {
        const int hi = h % HX, hj = (h / HX) % HY, hk = h / (HX * HY);
        const int gi = i0 - 1 + hi, gj = j0 - 1 + hj, gk = k0 - 1 + hk;
        float p = 0.f, f0 = 0.f, f1 = 0.f, f2 = 0.f, s0 = 0.f, s1 = 0.f, s2 = 0.f;
        if (gi >= 0 && gi < NX && gj >= 0 && gj < NY && gk >= 0 && gk < NZ) {
            const int n = gi + NX * (gj + NY * gk);
            p = beta == 0.f ? z[n] : fmaf(beta, pold[n], z[n]);
            f0 = fib[n];
            f1 = fib[(size_t)N + n];
            f2 = fib[2 * (size_t)N + n];
            s0 = fib[3 * (size_t)N + n];
            s1 = fib[4 * (size_t)N + n];
            s2 = fib[5 * (size_t)N + n];
            if (hi >= 1 && hi <= kMfTx && hj >= 1 && hj <= kMfTy && hk >= 1 && hk <= kMfTz) pnew[n] = p;
        }
        s_p[h] = p;
        s_f[h] = f0;
        s_f[HN + h] = f1;
        s_f[2 * HN + h] = f2;
        s_s[h] = s0;
        s_s[HN + h] = s1;
        s_s[2 * HN + h] = s2;
    }
    __syncthreads();

    // ---- element contributions ---------------------------------------------
    const float cn0 = D.mf_cn[0], cn1 = D.mf_cn[1], cn2 = D.mf_cn[2];
    const float cl = D.mf_cl, ct = D.mf_ct, cmass = D.mf_cmass;
    for (int e = threadIdx.x; e < EN; e += blockDim.x) {
        const int ei = e % EX, ej = (e / EX) % EY, ek = e / (EX * EY);
        const int gi = i0 - 1 + ei, gj = j0 - 1 + ej, gk = k0 - 1 + ek;
        float y[8];
        if (gi >= 0 && gi < NX - 1 && gj >= 0 && gj < NY - 1 && gk >= 0 && gk < NZ - 1) {
            float pe[8], fx[8], fy[8], fz[8], sx[8], sy[8], sz[8];
#pragma unroll
            for (int a = 0; a < 8; ++a) {
                const int h = (ei + (a & 1)) + HX * ((ej + ((a >> 1) & 1)) + HY * (ek + ((a >> 2) & 1)));
                pe[a] = s_p[h];
                fx[a] = s_f[h];
                fy[a] = s_f[HN + h];
                fz[a] = s_f[2 * HN + h];
                sx[a] = s_s[h];
                sy[a] = s_s[HN + h];
                sz[a] = s_s[2 * HN + h];
            }
            // fibres at the Gauss points
            float Fx[8], Fy[8], Fz[8], Sx[8], Sy[8], Sz[8];
            interp8(fx, Fx);
            interp8(fy, Fy);
            interp8(fz, Fz);
            interp8(sx, Sx);
            interp8(sy, Sy);
            interp8(sz, Sz);
            // reference gradient: d/dxi_0 at (q1,q2) from the x-differences etc.
            float dx[4], dy[4], dz[4], g1[4], g2[4], g3[4];
#pragma unroll
            for (int c = 0; c < 4; ++c) {
                dx[c] = pe[1 + 2 * c] - pe[2 * c];                                  // (b1,b2) = (c&1, c>>1)
                dy[c] = pe[(c & 1) + 2 + 4 * (c >> 1)] - pe[(c & 1) + 4 * (c >> 1)];  // (b0,b2)
                dz[c] = pe[c + 4] - pe[c];                                          // (b0,b1)
            }
            interp4(dx, g1);
            interp4(dy, g2);
            interp4(dz, g3);
            float T1[4] = {0.f, 0.f, 0.f, 0.f}, T2[4] = {0.f, 0.f, 0.f, 0.f}, T3[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
            for (int q = 0; q < 8; ++q) {
                const int q0 = q & 1, q1 = (q >> 1) & 1, q2 = (q >> 2) & 1;
                const float gx = g1[q1 + 2 * q2], gy = g2[q0 + 2 * q2], gz = g3[q0 + 2 * q1];
                const float fg = fmaf(Fx[q], gx, fmaf(Fy[q], gy, Fz[q] * gz));
                const float sg = fmaf(Sx[q], gx, fmaf(Sy[q], gy, Sz[q] * gz));
                const float A = cl * fg, B = ct * sg;
                T1[q1 + 2 * q2] += fmaf(B, Sx[q], fmaf(A, Fx[q], cn0 * gx));
                T2[q0 + 2 * q2] += fmaf(B, Sy[q], fmaf(A, Fy[q], cn1 * gy));
                T3[q0 + 2 * q1] += fmaf(B, Sz[q], fmaf(A, Fz[q], cn2 * gz));
            }
            float R1[4], R2[4], R3[4];
            interp4(T1, R1);
            interp4(T2, R2);
            interp4(T3, R3);
            // mass: (m x m x m) pe, m = [[1/3,1/6],[1/6,1/3]] = (1/6) [[2,1],[1,2]]
            float t[8], u[8], w[8];
#pragma unroll
            for (int r = 0; r < 4; ++r) {
                t[2 * r] = fmaf(2.f, pe[2 * r], pe[2 * r + 1]);
                t[2 * r + 1] = fmaf(2.f, pe[2 * r + 1], pe[2 * r]);
            }
#pragma unroll
            for (int c2 = 0; c2 < 2; ++c2)
#pragma unroll
                for (int c0 = 0; c0 < 2; ++c0) {
                    const int a = c0 + 4 * c2, b = c0 + 2 + 4 * c2;
                    u[a] = fmaf(2.f, t[a], t[b]);
                    u[b] = fmaf(2.f, t[b], t[a]);
                }
#pragma unroll
            for (int c = 0; c < 4; ++c) {
                w[c] = fmaf(2.f, u[c], u[c + 4]);
                w[c + 4] = fmaf(2.f, u[c + 4], u[c]);
            }
            const float cm = cmass * (1.f / 216.f);
#pragma unroll
            for (int a = 0; a < 8; ++a) {
                const int a0 = a & 1, a1 = (a >> 1) & 1, a2 = (a >> 2) & 1;
                const float r1 = R1[a1 + 2 * a2], r2 = R2[a0 + 2 * a2], r3 = R3[a0 + 2 * a1];
                float acc = cm * w[a];
                acc += a0 ? r1 : -r1;
                acc += a1 ? r2 : -r2;
                acc += a2 ? r3 : -r3;
                y[a] = acc;
            }
        } else {
#pragma unroll
            for (int a = 0; a < 8; ++a) y[a] = 0.f;
        }
#pragma unroll
        for (int a = 0; a < 8; ++a) s_y[a * EN + e] = y[a];
    }
    __syncthreads();

    // ---- gather per owned node (fixed order) --------------------------------
    float v[1] = {0.f};
    const double none[1] = {0.0};
    float dot = 0.f;
    for (int o = threadIdx.x; o < kMfTx * kMfTy * kMfTz; o += blockDim.x) {
        const int li = o % kMfTx, lj = (o / kMfTx) % kMfTy, lk = o / (kMfTx * kMfTy);
        const int gi = i0 + li, gj = j0 + lj, gk = k0 + lk;
        if (gi >= NX || gj >= NY || gk >= NZ) continue;
        float acc = 0.f;
#pragma unroll
        for (int ec = 0; ec < 2; ++ec)
#pragma unroll
            for (int eb = 0; eb < 2; ++eb)
#pragma unroll
                for (int ea = 0; ea < 2; ++ea) {
                    const int e = (li + ea) + EX * ((lj + eb) + EY * (lk + ec));
                    const int corner = (1 - ea) + 2 * (1 - eb) + 4 * (1 - ec);
                    acc += s_y[corner * EN + e];
                }
        const int n = gi + NX * (gj + NY * gk);
        D.q32[n] = acc;
        dot = fmaf(s_p[(li + 1) + HX * ((lj + 1) + HY * (lk + 1))], acc, dot);
    }
    v[0] = dot;
    grid_reduce<1, 0>(v, none, D.partial, D.counter + CNT_APPLY, blockIdx.x, gridDim.x,
                      [&](double* tot) { D.alpha = D.rz / tot[0]; });
}

int mf_tiles(const Dev& h) {
    return ((h.NX + kMfTx - 1) / kMfTx) * ((h.NY + kMfTy - 1) / kMfTy) * ((h.NZ + kMfTz - 1) / kMfTz);
}

cudaError_t mf_prepare() {
    return cudaFuncSetAttribute(k_apply32_mf, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kMfSmem);
}

void launch_apply32_mf(Dev* d, const Dev& h, cudaStream_t s) {
    k_apply32_mf<<<mf_tiles(h), kMfThreads, kMfSmem, s>>>(d);
}

}  // namespace epk
