// k_mfc.cu -- matrix-free FP32 apply of A = alpha/dt M + K on curved Q1
// meshes (the periodic structured shell), with the element coordinates and
// fibre frames staged in shared memory by TMA.
//
// Paper Sec. 1.2, Eq. (6) with D of Eq. (3), on the trilinear map x(xi) of
// each hexahedron and 2 x 2 x 2 Gauss-Legendre points (weights 1/8 on the
// reference cube [0,1]^3):
//   y_a += sum_q (1/8) |J_q| [ alpha/dt phi_a p + grad phi_a . D_q grad p ],
// J_q = dx/dxi at point q, D_q = dn I + (dl - dn) f f^T + (dt - dn) s s^T
// with f, s the trilinear interpolants of the nodal fibre and sheet vectors
// (not renormalised) -- the same integrals the assembled operators hold.
// With C the cofactor matrix of J (J^-1 = C^T / det J), the stiffness part
// of a point is  grad_xi phi_a . h_q,  h_q = (1/8) C^T D_q (C grad_xi p) / det J,
// so per point: the cofactors and det J, t = C grad_xi p, D t, h = C^T D t
// scaled -- about 60 FP32 operations; with the Jacobian, the fibres and p at
// the points and the transposed passes to the corners an element costs about
// 900.  This makes the kernel FP32-bound on GB300 (about 21 operations per
// byte of its 44 B/node of input, against a machine balance of about 6): the
// create-time autotuner weighs it against the stored symmetric stencil.
//
// Work decomposition: a block owns every node of a tile of kMcBY x kMcBZ
// (j, k) positions across the whole wall (all i).  One TMA load brings the
// tile plus a one-node halo of the 9 static per-node arrays (x, y, z, f0, s0;
// float, i fastest, rows padded to a multiple of 4 floats, and with ghost
// rows j = -1 and j = NY so that the periodic direction needs no wrap) into
// shared memory; meanwhile the threads stage the CG direction p = z + beta
// p_old on the same box (writing p_new for the owned nodes).  Elements are
// then evaluated in 8 colour classes (parities of their three indices): two
// elements of one class share no node, so each adds its 8 corner
// contributions to a shared accumulator without conflicts, and every node
// sums its elements in the same order in every run (bitwise reproducible, no
// atomics).  The owned nodes write q = A p and the block's partial of p . q;
// the last block forms alpha (CG), as the slab apply does.
//
// The TMA wait is bounded: a copy that does not complete within about a
// second records EP_ETIMEOUT, the block waits once more (bounded) for its
// copy and returns.
#include <cuda.h>
#include <cudaTypedefs.h>

#include <cstdint>
#include <cstring>

#include "ep_dev.cuh"

namespace epk {

constexpr int kMcBY = 8, kMcBZ = 8;    // owned (j, k) positions per block
constexpr int kMcThreads = 256;
constexpr int kMcMaxBX = 32;           // widest wall (nodes across, padded to 4)
constexpr int kMcComp = 9;             // x y z f0x f0y f0z s0x s0y s0z
constexpr int kMcRY = kMcBY + 2, kMcRZ = kMcBZ + 2;  // box rows with the halo

constexpr float kG0 = 0.21132486540518711775f;  // Gauss points of [0,1]: (1 -+ 1/sqrt 3)/2
constexpr float kG1 = 0.78867513459481288225f;

// box width (nodes across the wall, padded to a multiple of 4 floats: the
// TMA box's inner extent must be a multiple of 16 bytes)
__host__ __device__ inline int mc_bx(int NX) { return (NX + 3) / 4 * 4; }

__host__ __device__ inline size_t mc_box_floats(int NX) { return (size_t)mc_bx(NX) * kMcRY * kMcRZ; }

// dynamic shared memory: the TMA box (9 components), p and the accumulator
__host__ __device__ inline size_t mc_smem_bytes(int NX) { return (kMcComp + 2) * mc_box_floats(NX) * 4 + 128; }

// out[q] = sum_b L[q][b] in[b] along one direction (L symmetric: its own transpose)
__device__ __forceinline__ void mc_lmap(float a, float b, float& o0, float& o1) {
    o0 = fmaf(kG1, a, kG0 * b);
    o1 = fmaf(kG0, a, kG1 * b);
}

// trilinear values at the 8 Gauss points from the 8 corner values (index
// i0 + 2 i1 + 4 i2 on both sides); also the transposed map
__device__ __forceinline__ void mc_interp8(const float v[8], float o[8]) {
    float t[8], u[8];
#pragma unroll
    for (int r = 0; r < 4; ++r) mc_lmap(v[2 * r], v[2 * r + 1], t[2 * r], t[2 * r + 1]);
#pragma unroll
    for (int c2 = 0; c2 < 2; ++c2)
#pragma unroll
        for (int c0 = 0; c0 < 2; ++c0)
            mc_lmap(t[c0 + 4 * c2], t[c0 + 2 + 4 * c2], u[c0 + 4 * c2], u[c0 + 2 + 4 * c2]);
#pragma unroll
    for (int c = 0; c < 4; ++c) mc_lmap(u[c], u[c + 4], o[c], o[c + 4]);
}

// 2-D version on a 2 x 2 array (index i + 2 j)
__device__ __forceinline__ void mc_interp4(const float v[4], float o[4]) {
    float t[4];
    mc_lmap(v[0], v[1], t[0], t[1]);
    mc_lmap(v[2], v[3], t[2], t[3]);
    mc_lmap(t[0], t[2], o[0], o[2]);
    mc_lmap(t[1], t[3], o[1], o[3]);
}

// reference derivatives of a trilinear field at the Gauss points: d/dxi_0
// depends on (q1, q2) only, d/dxi_1 on (q0, q2), d/dxi_2 on (q0, q1)
__device__ __forceinline__ void mc_grad(const float v[8], float g0[4], float g1[4], float g2[4]) {
    float d0[4], d1[4], d2[4];
#pragma unroll
    for (int c = 0; c < 4; ++c) {
        d0[c] = v[1 + 2 * c] - v[2 * c];
        d1[c] = v[(c & 1) + 2 + 4 * (c >> 1)] - v[(c & 1) + 4 * (c >> 1)];
        d2[c] = v[c + 4] - v[c];
    }
    mc_interp4(d0, g0);
    mc_interp4(d1, g1);
    mc_interp4(d2, g2);
}

__device__ __forceinline__ unsigned int smem_u32(const void* p) {
    return (unsigned int)__cvta_generic_to_shared(p);
}

// bounded wait on phase 0 of a shared-memory mbarrier
__device__ __forceinline__ bool mc_wait(unsigned int bar, long long limit) {
    for (long long i = 0; i < limit; ++i) {
        unsigned int done;
        asm volatile(
            "{\n\t.reg .pred p;\n\t"
            "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
            "selp.u32 %0, 1, 0, p;\n\t}"
            : "=r"(done)
            : "r"(bar), "r"(0u)
            : "memory");
        if (done) return true;
    }
    return false;
}

constexpr long long kMcWaitLimit = 1ll << 20;  // try_wait rounds (each suspends up to ~1 us)

__global__ void __launch_bounds__(kMcThreads, 2) k_apply32_mfc(Dev* __restrict__ Dp,
                                                            const __grid_constant__ CUtensorMap geo) {
    extern __shared__ __align__(128) unsigned char mc_raw[];
    __shared__ __align__(8) unsigned long long bar;
    __shared__ int failed;
    Dev& D = *Dp;
    const int NX = D.NX, NY = D.NY, NZ = D.NZ;
    const int BX = mc_bx(NX);
    const int BOX = BX * kMcRY * kMcRZ;
    // [9][RZ][RY][BX] (the TMA box), 128-byte aligned
    float* s_g = reinterpret_cast<float*>((reinterpret_cast<uintptr_t>(mc_raw) + 127) & ~uintptr_t(127));
    float* s_p = s_g + kMcComp * BOX;                // [RZ][RY][BX]
    float* s_a = s_p + BOX;                          // accumulator, same shape
    const int ty = (NY + kMcBY - 1) / kMcBY;
    const int j0 = (blockIdx.x % ty) * kMcBY, k0 = (blockIdx.x / ty) * kMcBZ;
    const unsigned int b = smem_u32(&bar);

    if (threadIdx.x == 0) {
        failed = 0;
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(b) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        const unsigned int bytes = (unsigned int)(kMcComp * BOX * 4);
        asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(b), "r"(bytes) : "memory");
        // box origin: i = 0, ghost-padded row j0 (= j0 - 1 + 1), k0 - 1, component 0
        asm volatile(
            "cp.async.bulk.tensor.4d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
            " [%0], [%1, {%2, %3, %4, %5}], [%6];" ::"r"(smem_u32(s_g)),
            "l"(reinterpret_cast<unsigned long long>(&geo)), "r"(0), "r"(j0), "r"(k0 - 1), "r"(0), "r"(b)
            : "memory");
    }

    // ---- stage p = z + beta p_old on the box (plain loads, while TMA flies)
    const float beta = (float)D.beta;
    const float* __restrict__ z = D.z32;
    const float* __restrict__ pold = D.pswap ? D.pb32 : D.pa32;
    float* __restrict__ pnew = D.pswap ? D.pa32 : D.pb32;
    for (int h = threadIdx.x; h < BOX; h += blockDim.x) {
        const int li = h % BX, lj = (h / BX) % kMcRY, lk = h / (BX * kMcRY);
        const int gk = k0 - 1 + lk, gjr = j0 - 1 + lj;
        float p = 0.f;
        if (li < NX && gk >= 0 && gk < NZ && gjr <= NY) {
            const int gj = gjr < 0 ? gjr + NY : (gjr >= NY ? gjr - NY : gjr);
            const int n = li + NX * (gj + NY * gk);
            p = beta == 0.f ? z[n] : fmaf(beta, pold[n], z[n]);
            if (lj >= 1 && lj <= kMcBY && gjr < NY && lk >= 1 && lk <= kMcBZ) pnew[n] = p;
        }
        s_p[h] = p;
        s_a[h] = 0.f;
    }
    if (!mc_wait(b, kMcWaitLimit)) {
        atomicCAS(&D.status, (int)EP_OK, (int)EP_ETIMEOUT);
        failed = 1;
    }
    __syncthreads();
    if (failed) {
        // the copy may still be in flight: wait once more (bounded) before
        // the block's shared memory is released
        if (threadIdx.x == 0) (void)mc_wait(b, kMcWaitLimit);
        __syncthreads();
        return;
    }

    // ---- elements, in 8 colour classes
    const float cmass = D.mf_cmass;  // alpha/dt (curved meshes)
    const float dn = D.mf_cn[0], cl = D.mf_cl, ct = D.mf_ct;
    const int ne_i = NX - 1;
    const int lj_max = min(kMcBY, NY - j0);  // last element row touching an owned node
    for (int col = 0; col < 8; ++col) {
        const int c0 = col & 1, c1 = (col >> 1) & 1, c2 = col >> 2;
        const int na = (ne_i - c0 + 1) / 2, nb = (kMcBY + 1 - c1 + 1) / 2, nd = (kMcBZ + 1 - c2 + 1) / 2;
        for (int e = threadIdx.x; e < na * nb * nd; e += blockDim.x) {
            const int ei = 2 * (e % na) + c0;
            const int lj = 2 * ((e / na) % nb) + c1;
            const int lk = 2 * (e / (na * nb)) + c2;
            const int ek = k0 - 1 + lk;
            if (lj > lj_max || ek < 0 || ek >= NZ - 1) continue;
            const int h0 = ei + BX * (lj + kMcRY * lk);
            int hc[8];
            float X[8], Y[8], Zc[8], P[8];
#pragma unroll
            for (int a = 0; a < 8; ++a) {
                hc[a] = h0 + (a & 1) + BX * (((a >> 1) & 1) + kMcRY * (a >> 2));
                X[a] = s_g[hc[a]];
                Y[a] = s_g[BOX + hc[a]];
                Zc[a] = s_g[2 * BOX + hc[a]];
                P[a] = s_p[hc[a]];
            }
            // Jacobian columns at the points: J[c][d] = d x_c / d xi_d
            float jx0[4], jx1[4], jx2[4], jy0[4], jy1[4], jy2[4], jz0[4], jz1[4], jz2[4];
            mc_grad(X, jx0, jx1, jx2);
            mc_grad(Y, jy0, jy1, jy2);
            mc_grad(Zc, jz0, jz1, jz2);
            float g0[4], g1[4], g2[4];
            mc_grad(P, g0, g1, g2);
            float pq[8];
            mc_interp8(P, pq);
            // fibre and sheet vectors at the points
            float F[3][8], S[3][8];
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                float v[8];
#pragma unroll
                for (int a = 0; a < 8; ++a) v[a] = s_g[(3 + c) * BOX + hc[a]];
                mc_interp8(v, F[c]);
#pragma unroll
                for (int a = 0; a < 8; ++a) v[a] = s_g[(6 + c) * BOX + hc[a]];
                mc_interp8(v, S[c]);
            }
            float T0[4] = {0.f, 0.f, 0.f, 0.f}, T1[4] = {0.f, 0.f, 0.f, 0.f}, T2[4] = {0.f, 0.f, 0.f, 0.f};
            float mq[8];
#pragma unroll
            for (int q = 0; q < 8; ++q) {
                const int q0 = q & 1, q1 = (q >> 1) & 1, q2 = q >> 2;
                const int i0 = q1 + 2 * q2, i1 = q0 + 2 * q2, i2 = q0 + 2 * q1;
                const float J00 = jx0[i0], J01 = jx1[i1], J02 = jx2[i2];
                const float J10 = jy0[i0], J11 = jy1[i1], J12 = jy2[i2];
                const float J20 = jz0[i0], J21 = jz1[i1], J22 = jz2[i2];
                // cofactors (C[r][c] of J[r][c]) and the determinant
                const float C00 = fmaf(J11, J22, -J12 * J21), C01 = fmaf(J12, J20, -J10 * J22),
                            C02 = fmaf(J10, J21, -J11 * J20);
                const float C10 = fmaf(J02, J21, -J01 * J22), C11 = fmaf(J00, J22, -J02 * J20),
                            C12 = fmaf(J01, J20, -J00 * J21);
                const float C20 = fmaf(J01, J12, -J02 * J11), C21 = fmaf(J02, J10, -J00 * J12),
                            C22 = fmaf(J00, J11, -J01 * J10);
                const float det = fmaf(J00, C00, fmaf(J01, C01, J02 * C02));
                const float gx = g0[i0], gy = g1[i1], gz = g2[i2];
                // t = C grad_xi p = det * grad_x p
                const float t0 = fmaf(C00, gx, fmaf(C01, gy, C02 * gz));
                const float t1 = fmaf(C10, gx, fmaf(C11, gy, C12 * gz));
                const float t2 = fmaf(C20, gx, fmaf(C21, gy, C22 * gz));
                const float fx = F[0][q], fy = F[1][q], fz = F[2][q];
                const float sx = S[0][q], sy = S[1][q], sz = S[2][q];
                const float ft = cl * fmaf(fx, t0, fmaf(fy, t1, fz * t2));
                const float st = ct * fmaf(sx, t0, fmaf(sy, t1, sz * t2));
                const float d0 = fmaf(dn, t0, fmaf(ft, fx, st * sx));
                const float d1 = fmaf(dn, t1, fmaf(ft, fy, st * sy));
                const float d2 = fmaf(dn, t2, fmaf(ft, fz, st * sz));
                // h = C^T (D t) / (8 det)
                const float w = 0.125f / det;
                T0[i0] = fmaf(w, fmaf(C00, d0, fmaf(C10, d1, C20 * d2)), T0[i0]);
                T1[i1] = fmaf(w, fmaf(C01, d0, fmaf(C11, d1, C21 * d2)), T1[i1]);
                T2[i2] = fmaf(w, fmaf(C02, d0, fmaf(C12, d1, C22 * d2)), T2[i2]);
                mq[q] = 0.125f * cmass * det * pq[q];
            }
            float R0[4], R1[4], R2[4], M8[8];
            mc_interp4(T0, R0);
            mc_interp4(T1, R1);
            mc_interp4(T2, R2);
            mc_interp8(mq, M8);
#pragma unroll
            for (int a = 0; a < 8; ++a) {
                const int a0 = a & 1, a1 = (a >> 1) & 1, a2 = a >> 2;
                const float r0 = R0[a1 + 2 * a2], r1 = R1[a0 + 2 * a2], r2 = R2[a0 + 2 * a1];
                float y = M8[a];
                y += a0 ? r0 : -r0;
                y += a1 ? r1 : -r1;
                y += a2 ? r2 : -r2;
                s_a[hc[a]] += y;
            }
        }
        __syncthreads();
    }

    // ---- owned nodes: q = A p and the block's p . q
    float v[1] = {0.f};
    const double none[1] = {0.0};
    float dot = 0.f;
    for (int o = threadIdx.x; o < NX * kMcBY * kMcBZ; o += blockDim.x) {
        const int li = o % NX, lj = 1 + (o / NX) % kMcBY, lk = 1 + o / (NX * kMcBY);
        const int gj = j0 - 1 + lj, gk = k0 - 1 + lk;
        if (gj >= NY || gk >= NZ) continue;
        const int h = li + BX * (lj + kMcRY * lk);
        const int n = li + NX * (gj + NY * gk);
        const float acc = s_a[h];
        D.q32[n] = acc;
        dot = fmaf(s_p[h], acc, dot);
    }
    v[0] = dot;
    grid_reduce<1, 0>(v, none, D.partial, D.counter + CNT_APPLY, blockIdx.x, gridDim.x,
                      [&](double* tot) { D.alpha = D.rz / tot[0]; });
}

int mfc_tiles(const Dev& h) { return ((h.NY + kMcBY - 1) / kMcBY) * ((h.NZ + kMcBZ - 1) / kMcBZ); }

bool mfc_supported(int NX) { return mc_bx(NX) <= kMcMaxBX; }

// Floats of the staged geometry array: [9][NZ][NY + 2][BX].
size_t mfc_geo_floats(int NX, int NY, int NZ) { return (size_t)kMcComp * NZ * (NY + 2) * mc_bx(NX); }

// Fills the geometry array on the host: per node x, y, z, f0, s0 (float),
// rows padded to BX, ghost rows j = -1 (a copy of j = NY-1) and j = NY (a
// copy of j = 0) for the periodic direction.
void mfc_fill_geo(float* g, int NX, int NY, int NZ, const double* xyz, const double* f0, const double* s0) {
    const int BX = mc_bx(NX);
    const size_t plane = (size_t)NZ * (NY + 2) * BX;
    std::memset(g, 0, kMcComp * plane * sizeof(float));
    for (int k = 0; k < NZ; ++k)
        for (int jp = 0; jp < NY + 2; ++jp) {
            const int j = jp == 0 ? NY - 1 : (jp == NY + 1 ? 0 : jp - 1);
            for (int i = 0; i < NX; ++i) {
                const size_t n = (size_t)i + (size_t)NX * ((size_t)j + (size_t)NY * k);
                const size_t o = (size_t)i + (size_t)BX * ((size_t)jp + (size_t)(NY + 2) * k);
                for (int c = 0; c < 3; ++c) {
                    g[c * plane + o] = (float)xyz[3 * n + c];
                    g[(3 + c) * plane + o] = (float)f0[3 * n + c];
                    g[(6 + c) * plane + o] = (float)s0[3 * n + c];
                }
            }
        }
}

// The tensor map of the geometry array (4-D: i, ghost-padded j, k, component;
// box BX x (BY+2) x (BZ+2) x 9, zero fill outside).
cudaError_t mfc_tensor_map(CUtensorMap* tm, const float* g, int NX, int NY, int NZ) {
    static PFN_cuTensorMapEncodeTiled_v12000 encode = nullptr;
    if (!encode) {
        void* fn = nullptr;
        cudaDriverEntryPointQueryResult q;
        cudaError_t e = cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q);
        if (e != cudaSuccess) return e;
        if (q != cudaDriverEntryPointSuccess || !fn) return cudaErrorSymbolNotFound;
        encode = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(fn);
    }
    const int BX = mc_bx(NX);
    const cuuint64_t dims[4] = {(cuuint64_t)NX, (cuuint64_t)(NY + 2), (cuuint64_t)NZ, (cuuint64_t)kMcComp};
    const cuuint64_t strides[3] = {(cuuint64_t)BX * 4, (cuuint64_t)BX * (NY + 2) * 4,
                                   (cuuint64_t)BX * (NY + 2) * NZ * 4};
    const cuuint32_t box[4] = {(cuuint32_t)BX, (cuuint32_t)kMcRY, (cuuint32_t)kMcRZ, (cuuint32_t)kMcComp};
    const cuuint32_t estr[4] = {1, 1, 1, 1};
    const CUresult r = encode(tm, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, const_cast<float*>(g), dims, strides, box,
                              estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                              CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorInvalidValue;
}

cudaError_t mfc_prepare(int NX) {
    return cudaFuncSetAttribute(k_apply32_mfc, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)mc_smem_bytes(NX));
}

void launch_apply32_mfc(Dev* d, const Dev& h, const CUtensorMap& tm, cudaStream_t s) {
    k_apply32_mfc<<<mfc_tiles(h), kMcThreads, mc_smem_bytes(h.NX), s>>>(d, tm);
}

}  // namespace epk
