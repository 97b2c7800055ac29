// k_stencil.cu -- assembled 27-point operators of structured Q1 meshes.
//
// Paper Sec. 1.2, Eq. (6): M_jk = int phi_k phi_j, K_jk = int D grad phi_k .
// grad phi_j with D of Eq. (3); integrals by 2x2x2 Gauss-Legendre, the
// minimum rule that integrates the Q1 mass matrix exactly.  The diffusion
// tensor at a quadrature point is dn I + (dl - dn) f f^T + (dt - dn) s s^T,
// f and s the Q1 interpolants of the nodal fibre vectors.
//
// Like the paper, the FP64 matrices are assembled once (the paper notes the
// system matrix never changes and only the right-hand side is rebuilt each
// step, Sec. 3.4); here they are node-major 27-point stencils (diagonal + 13
// forward couplings per node, the backward ones read from the neighbours)
// rather than distributed CSR, because on GB300 the FP64 arithmetic of a
// matrix-free apply would cost far more than streaming the stencil.
//
// Kernels: assembly (node-centric, deterministic, no atomics), the expansion
// of the stencils into the refined solver's full float-float layout, the
// FP64 path's right-hand side / residual and CG apply and updates, and the
// FP32 stencil apply of the refined inner solver.
#include "ep_dev.cuh"
#include "ep_tile.cuh"

namespace epk {

// ---------------------------------------------------------------- assembly --

__device__ void node_coords(const Dev& D, const AsmParams& P, int i, int j, int k, double x[3]) {
    if (P.xyz) {
        const int jj = D.periodic ? (j % D.NY) : j;
        const size_t n = (size_t)i + (size_t)D.NX * ((size_t)jj + (size_t)D.NY * k);
        x[0] = P.xyz[3 * n];
        x[1] = P.xyz[3 * n + 1];
        x[2] = P.xyz[3 * n + 2];
    } else {
        x[0] = i * D.h[0];
        x[1] = j * D.h[1];
        x[2] = k * D.h[2];
    }
}

// Row a of the element mass and stiffness matrices of element (ei, ej, ek)
// with diffusivities dl, dt, dn.
__device__ void element_row(const Dev& D, const AsmParams& P, int ei, int ej, int ek, int a, double dl,
                            double dtr, double dn, double Mrow[8], double Krow[8], bool& bad) {
    double X[8][3], F[8][3], S[8][3];
#pragma unroll
    for (int b = 0; b < 8; ++b) {
        const int bi = ei + (b & 1), bj = ej + ((b >> 1) & 1), bk = ek + ((b >> 2) & 1);
        node_coords(D, P, bi, bj, bk, X[b]);
        const int bjj = D.periodic ? (bj % D.NY) : bj;
        const size_t n = (size_t)bi + (size_t)D.NX * ((size_t)bjj + (size_t)D.NY * bk);
        for (int c = 0; c < 3; ++c) {
            F[b][c] = P.f0[3 * n + c];
            S[b][c] = P.s0[3 * n + c];
        }
    }
    for (int b = 0; b < 8; ++b) Mrow[b] = Krow[b] = 0.0;
    const double r3 = 0.57735026918962576451;  // 1/sqrt(3)
    const double gp[2] = {0.5 - 0.5 * r3, 0.5 + 0.5 * r3};
    const int a0 = a & 1, a1 = (a >> 1) & 1, a2 = (a >> 2) & 1;
    for (int q = 0; q < 8; ++q) {
        const double xi[3] = {gp[q & 1], gp[(q >> 1) & 1], gp[(q >> 2) & 1]};
        double Lv[3][2], phi[8], dphi[8][3];
        for (int d = 0; d < 3; ++d) {
            Lv[d][0] = 1.0 - xi[d];
            Lv[d][1] = xi[d];
        }
        for (int b = 0; b < 8; ++b) {
            const int b0 = b & 1, b1 = (b >> 1) & 1, b2 = (b >> 2) & 1;
            const double s0 = b0 ? 1.0 : -1.0, s1 = b1 ? 1.0 : -1.0, s2 = b2 ? 1.0 : -1.0;
            phi[b] = Lv[0][b0] * Lv[1][b1] * Lv[2][b2];
            dphi[b][0] = s0 * Lv[1][b1] * Lv[2][b2];
            dphi[b][1] = Lv[0][b0] * s1 * Lv[2][b2];
            dphi[b][2] = Lv[0][b0] * Lv[1][b1] * s2;
        }
        double J[3][3];
        for (int r = 0; r < 3; ++r)
            for (int c = 0; c < 3; ++c) {
                double s = 0.0;
                for (int b = 0; b < 8; ++b) s += X[b][r] * dphi[b][c];
                J[r][c] = s;
            }
        // cofactor matrix C (C[r][c] = cofactor of J[r][c]); inv(J) = C^T / det
        double C[3][3];
        C[0][0] = J[1][1] * J[2][2] - J[1][2] * J[2][1];
        C[0][1] = J[1][2] * J[2][0] - J[1][0] * J[2][2];
        C[0][2] = J[1][0] * J[2][1] - J[1][1] * J[2][0];
        C[1][0] = J[0][2] * J[2][1] - J[0][1] * J[2][2];
        C[1][1] = J[0][0] * J[2][2] - J[0][2] * J[2][0];
        C[1][2] = J[0][1] * J[2][0] - J[0][0] * J[2][1];
        C[2][0] = J[0][1] * J[1][2] - J[0][2] * J[1][1];
        C[2][1] = J[0][2] * J[1][0] - J[0][0] * J[1][2];
        C[2][2] = J[0][0] * J[1][1] - J[0][1] * J[1][0];
        const double det = J[0][0] * C[0][0] + J[0][1] * C[0][1] + J[0][2] * C[0][2];
        if (!(det > 0.0)) bad = true;
        // physical gradient: grad phi = J^{-T} dphi; (J^{-T})[i][j] = C[i][j]/det
        double G[8][3];
        for (int b = 0; b < 8; ++b)
            for (int i = 0; i < 3; ++i)
                G[b][i] = (C[i][0] * dphi[b][0] + C[i][1] * dphi[b][1] + C[i][2] * dphi[b][2]) / det;
        double fq[3] = {0, 0, 0}, sq[3] = {0, 0, 0};
        for (int b = 0; b < 8; ++b)
            for (int c = 0; c < 3; ++c) {
                fq[c] += phi[b] * F[b][c];
                sq[c] += phi[b] * S[b][c];
            }
        const double w = 0.125 * det;
        // D G_a
        double Dg[3];
        for (int i = 0; i < 3; ++i) {
            const double fg = fq[0] * G[a][0] + fq[1] * G[a][1] + fq[2] * G[a][2];
            const double sg = sq[0] * G[a][0] + sq[1] * G[a][1] + sq[2] * G[a][2];
            Dg[i] = dn * G[a][i] + (dl - dn) * fg * fq[i] + (dtr - dn) * sg * sq[i];
        }
        const double pa = phi[a];
        for (int b = 0; b < 8; ++b) {
            Mrow[b] += w * pa * phi[b];
            Krow[b] += w * (Dg[0] * G[b][0] + Dg[1] * G[b][1] + Dg[2] * G[b][2]);
        }
    }
    (void)a0; (void)a1; (void)a2;
}

__global__ void __launch_bounds__(128) k_assemble(Dev* __restrict__ Dp, AsmParams P) {
    const Dev& D = *Dp;
    const int n = blockIdx.x * blockDim.x + threadIdx.x;
    if (n >= D.N) return;
    int i, j, k;
    node_ijk(D, n, i, j, k);
    double cm[kSlots], ck[kSlots];
    for (int s = 0; s < kSlots; ++s) cm[s] = ck[s] = 0.0;
    bool bad = false;
    int included = 0;
    double mexcl = 0.0;  // mass diagonal of the excluded elements around n
    for (int ec = 0; ec < 2; ++ec)
        for (int eb = 0; eb < 2; ++eb)
            for (int ea = 0; ea < 2; ++ea) {
                const int gi = i - 1 + ea, gk = k - 1 + ec;
                int gj = j - 1 + eb;
                if (gi < 0 || gi >= D.nx || gk < 0 || gk >= D.nz) continue;
                if (D.periodic) {
                    if (gj < 0) gj += D.ny;
                } else if (gj < 0 || gj >= D.ny) {
                    continue;
                }
                const int a0 = 1 - ea, a1 = 1 - eb, a2 = 1 - ec;
                const int a = a0 + 2 * a1 + 4 * a2;
                double dl = P.dl, dtr = P.dt, dn = P.dn;
                bool excluded = false;
                if (P.label) {
                    // element (gi, gj, gk) of the subdomain partition
                    const int r = P.label[(size_t)gi + (size_t)D.nx * ((size_t)gj + (size_t)D.ny * gk)];
                    excluded = P.excl[r] != 0;
                    dl = P.rd[r][0];
                    dtr = P.rd[r][1];
                    dn = P.rd[r][2];
                }
                double Mrow[8], Krow[8];
                element_row(D, P, gi, gj, gk, a, dl, dtr, dn, Mrow, Krow, bad);
                if (excluded) {  // no contribution to M and K; its mass diagonal aside
                    mexcl += Mrow[a];
                    continue;
                }
                ++included;
                for (int b = 0; b < 8; ++b) {
                    const int di = (b & 1) - a0, dj = ((b >> 1) & 1) - a1, dk = ((b >> 2) & 1) - a2;
                    const int t = (di + 1) + 3 * (dj + 1) + 9 * (dk + 1);
                    if (t >= 13) {
                        cm[t - 13] += Mrow[b];
                        ck[t - 13] += Krow[b];
                    }
                }
            }
    if (bad) *P.bad = 1;
    // an inactive node keeps a lone mass diagonal (what its excluded elements
    // would give, so its row scales like its neighbours') and no stiffness
    if (included == 0) cm[0] = mexcl;
    if (D.active) const_cast<uint8_t*>(D.active)[n] = included > 0 ? 1 : 0;
    for (int s = 0; s < kSlots; ++s) {
        const double av = ck[s] + P.alpha_dt * cm[s];
        D.M64[(size_t)s * D.N + n] = cm[s];
        D.A64[(size_t)s * D.N + n] = av;
    }
    const double dinv = 1.0 / (ck[0] + P.alpha_dt * cm[0]);
    D.dinv64[n] = dinv;
    if (D.dinv32) D.dinv32[n] = (float)dinv;
}

// A <- A + (alpha_new/dt - alpha_old/dt) M  when the BDF order changes.
__global__ void k_realpha(Dev* __restrict__ Dp, double delta, double alpha_dt, float cmass) {
    Dev& D = *Dp;
    const int n = blockIdx.x * blockDim.x + threadIdx.x;
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        D.alpha_dt = alpha_dt;
        D.mf_cmass = cmass;
    }
    if (n >= D.N) return;
    for (int s = 0; s < kSlots; ++s) {
        const size_t o = (size_t)s * D.N + n;
        const double av = D.A64[o] + delta * D.M64[o];
        D.A64[o] = av;
    }
    const double dinv = 1.0 / D.A64[n];
    D.dinv64[n] = dinv;
    if (D.dinv32) D.dinv32[n] = (float)dinv;
}

// Refined path (the FP64 stencils are gone after ep_create): the same
// change applied to the float-float couplings, each coefficient re-split from
// its double sum; the inverse diagonal (slot 0) follows.
// The mass couplings are the stored ones on curved meshes and the analytic
// uniform-slab ones (w c_x c_y c_z, see mass_slab_np) on slabs.  The step
// history of A u no longer matches A: it is marked empty.
__global__ void k_realpha_ff(Dev* __restrict__ Dp, double delta, double alpha_dt, float cmass) {
    Dev& D = *Dp;
    const int n = blockIdx.x * blockDim.x + threadIdx.x;
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        D.alpha_dt = alpha_dt;
        D.mf_cmass = cmass;
        D.hist = 0;
    }
    if (n >= D.N) return;
    int i, j, k;
    node_ijk(D, n, i, j, k);
    const double w = (double)D.mw_hi + (double)D.mw_lo;
    for (int sl = 0; sl < kSlots; ++sl) {
        const int t = 13 + sl;
        const long long o = (long long)sl * D.cs + n;
        const int di = t % 3 - 1, dj = (t / 3) % 3 - 1, dk = t / 9 - 1;
        if (neighbour(D, i, j, k, di, dj, dk) < 0) continue;  // stays 0
        double m = 0.0;
        if (D.Mhi) {
            m = (double)D.Mhi[o] + (double)D.Mlo[o];
        } else {
            const double fx = di != 0 ? 1.0 : ((i == 0 || i == D.NX - 1) ? 2.0 : 4.0);
            const double fy = dj != 0 ? 1.0 : ((j == 0 || j == D.NY - 1) ? 2.0 : 4.0);
            const double fz = dk != 0 ? 1.0 : ((k == 0 || k == D.NZ - 1) ? 2.0 : 4.0);
            m = w * fx * fy * fz;
        }
        const double v = ((double)D.Ahi[o] + (double)D.Alo[o]) + delta * m;
        float vh, vl;
        ff_from_double(v, vh, vl);
        D.Ahi[o] = vh;
        D.Alo[o] = vl;
        if (sl == 0) D.dinv32[n] = (float)(1.0 / v);
    }
}

// The refined solver's couplings of node n from the FP64 stencils: per slot
// (the diagonal and the 13 forward couplings, 0 where the forward neighbour
// does not exist) the float hi + lo parts; also the node's boundary flags.
__global__ void k_expand(Dev* __restrict__ Dp, int want_a, int want_m) {
    const Dev& D = *Dp;
    const int n = blockIdx.x * blockDim.x + threadIdx.x;
    if (n >= D.N) return;
    int i, j, k;
    node_ijk(D, n, i, j, k);
    const size_t N = (size_t)D.N;
    if (D.nflag)
        D.nflag[n] = (unsigned char)((i == 0 ? 1 : 0) | (i == D.NX - 1 ? 2 : 0) | (j == 0 ? 4 : 0) |
                                     (j == D.NY - 1 ? 8 : 0) | (k == 0 ? 16 : 0) | (k == D.NZ - 1 ? 32 : 0));
    for (int which = 0; which < 2; ++which) {
        if ((which == 0 && !want_a) || (which == 1 && (!want_m || !D.Mhi))) continue;
        const double* c = which == 0 ? D.A64 : D.M64;
        float* hi = which == 0 ? D.Ahi : D.Mhi;
        float* lo = which == 0 ? D.Alo : D.Mlo;
        for (int sl = 0; sl < kSlots; ++sl) {
            const int t = 13 + sl;
            const int di = t % 3 - 1, dj = (t / 3) % 3 - 1, dk = t / 9 - 1;
            double v = 0.0;
            if (sl == 0 || neighbour(D, i, j, k, di, dj, dk) >= 0) v = c[(size_t)sl * N + n];
            float vh, vl;
            ff_from_double(v, vh, vl);
            hi[(long long)sl * D.cs + n] = vh;
            lo[(long long)sl * D.cs + n] = vl;
        }
    }
}

// ---------------------------------------------------------------- applies --

// FP64 path: right-hand side and initial residual (first == 1), or residual
// only (first == 0):  b = M v,  r = b - A u_new, z = D^-1 r, and the
// reductions the CG needs.
__global__ void __launch_bounds__(kStThreads) k_rhs64(Dev* __restrict__ Dp, int first, int graph) {
    __shared__ int sidx[SHN];
    __shared__ double su[SHN];
    __shared__ double sv[SHN];
    Dev& D = *Dp;
    const size_t N = (size_t)D.N;
    const double* __restrict__ vv = D.v;
    const double* __restrict__ u = D.u_new;
    double vd[3] = {0.0, 0.0, 0.0};  // b.b, r.r, r.z
    const int ntiles = st_tiles(D);
    for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
        const TileGeo g = tile_geo(D, tile);
        __syncthreads();
        stage_tile<double>(D, g, sidx, su, [&](int n, bool) { return u[n]; });
        if (first) {
            for (int h = threadIdx.x; h < SHN; h += blockDim.x) {
                const int n = sidx[h];  // written by this same thread above
                sv[h] = n >= 0 ? vv[n] : 0.0;
            }
        }
        __syncthreads();
        for_owned(D, g, [&](int h) {
            const int n = sidx[h];
            double b;
            if (first) {
                b = tile_row<double, double, double>(D.M64, N, sidx, sv, h, n);
                // applied currents on element regions (Gauss-integrated vectors)
#pragma unroll
                for (int p = 0; p < EP_MAX_PULSES; ++p)
                    if (D.eg64[p]) b = fma(pulse_amp(D, p), D.eg64[p][n], b);
                D.b[n] = b;
            } else {
                b = D.b[n];
            }
            const double au = tile_row<double, double, double>(D.A64, N, sidx, su, h, n);
            const double r = b - au;
            D.r[n] = r;
            vd[0] = fma(b, b, vd[0]);
            vd[1] = fma(r, r, vd[1]);
            const double z = D.dinv64[n] * r;
            D.z64[n] = z;
            vd[2] = fma(r, z, vd[2]);
        });
    }
    const float none[1] = {0.f};
    grid_reduce<0, 3>(none, vd, D.partial, D.counter + CNT_RHS, blockIdx.x, gridDim.x, [&](double* t) {
        if (first) D.bb = t[0];
        const double rr = t[1], bb = D.bb;
        const bool nan = !(rr == rr);
        const bool conv = !nan && (rr <= D.tol * D.tol * bb);
        D.relres = bb > 0.0 ? sqrt(rr / bb) : sqrt(rr);
        if (nan && D.status == EP_OK) D.status = EP_ENAN;
        D.it = 0;
        D.beta = 0.0;
        D.rz = t[2];
        D.rr = rr;
        set_cond(graph ? D.h_loop : 0ull, &D.f_loop, (!conv && !nan) ? 1u : 0u);
    });
}

// FP64 CG: p = z + beta p (beta == 0: p = z)
__global__ void __launch_bounds__(kNodeThreads) k_p64(Dev* __restrict__ Dp) {
    const Dev& D = *Dp;
    const double beta = D.beta;
    for (int n = blockIdx.x * blockDim.x + threadIdx.x; n < D.N; n += gridDim.x * blockDim.x)
        D.pa64[n] = beta == 0.0 ? D.z64[n] : fma(beta, D.pa64[n], D.z64[n]);
}

// FP64 CG: q = A p, alpha = rz / (p, q)
__global__ void __launch_bounds__(kStThreads) k_apply64(Dev* __restrict__ Dp) {
    __shared__ int sidx[SHN];
    __shared__ double sp[SHN];
    Dev& D = *Dp;
    const size_t N = (size_t)D.N;
    const double* __restrict__ p = D.pa64;
    double v[1] = {0.0};
    const float none[1] = {0.f};
    const int ntiles = st_tiles(D);
    for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
        const TileGeo g = tile_geo(D, tile);
        __syncthreads();
        stage_tile<double>(D, g, sidx, sp, [&](int n, bool) { return p[n]; });
        __syncthreads();
        for_owned(D, g, [&](int h) {
            const int n = sidx[h];
            const double q = tile_row<double, double, double>(D.A64, N, sidx, sp, h, n);
            D.q64[n] = q;
            v[0] = fma(sp[h], q, v[0]);
        });
    }
    grid_reduce<0, 1>(none, v, D.partial, D.counter + CNT_APPLY, blockIdx.x, gridDim.x,
                      [&](double* tot) { D.alpha = D.rz / tot[0]; });
}

// FP64 CG: x += alpha p, r -= alpha q, z = D^-1 r; beta, convergence
__global__ void __launch_bounds__(kNodeThreads) k_update64(Dev* __restrict__ Dp, int graph) {
    Dev& D = *Dp;
    const double alpha = D.alpha;
    double v[2] = {0.0, 0.0};
    for (int n = blockIdx.x * blockDim.x + threadIdx.x; n < D.N; n += gridDim.x * blockDim.x) {
        D.u_new[n] = fma(alpha, D.pa64[n], D.u_new[n]);
        const double r = fma(-alpha, D.q64[n], D.r[n]);
        D.r[n] = r;
        const double z = D.dinv64[n] * r;
        D.z64[n] = z;
        v[0] = fma(r, z, v[0]);
        v[1] = fma(r, r, v[1]);
    }
    const float none[1] = {0.f};
    grid_reduce<0, 2>(none, v, D.partial, D.counter + CNT_UPDATE, blockIdx.x, gridDim.x, [&](double* tot) {
        D.beta = tot[0] / D.rz;
        D.rz = tot[0];
        D.rr = tot[1];
        D.it += 1;
        const bool nan = !(tot[1] == tot[1]);
        const bool conv = !nan && tot[1] <= D.tol * D.tol * D.bb;
        D.relres = D.bb > 0.0 ? sqrt(tot[1] / D.bb) : sqrt(tot[1]);
        if (nan && D.status == EP_OK) D.status = EP_ENAN;
        if (!conv && D.it >= D.max_iter && D.status == EP_OK) D.status = EP_ENOCONV;
        set_cond(graph ? D.h_loop : 0ull, &D.f_loop, (!conv && !nan && D.it < D.max_iter) ? 1u : 0u);
    });
}

// FP32 inner CG, stencil operator: p_new = z + beta p_old (staged with the
// halo; the owning tile records it), q = A32 p_new; alpha = rz / (p_new, q).
__global__ void __launch_bounds__(kStThreads) k_apply32_stencil(Dev* __restrict__ Dp) {
    __shared__ int sidx[SHN];
    __shared__ float sp[SHN];
    Dev& D = *Dp;
    const float* __restrict__ pold = D.pswap ? D.pb32 : D.pa32;
    float* __restrict__ pnew = D.pswap ? D.pa32 : D.pb32;
    const float beta = (float)D.beta;
    const float* __restrict__ z = D.z32;
    float v[1] = {0.f};
    const double none[1] = {0.0};
    const int ntiles = st_tiles(D);
    for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
        const TileGeo g = tile_geo(D, tile);
        __syncthreads();
        stage_tile<float>(D, g, sidx, sp, [&](int n, bool own) {
            const float pn = beta == 0.0f ? z[n] : fmaf(beta, pold[n], z[n]);
            if (own) pnew[n] = pn;
            return pn;
        });
        __syncthreads();
        for_owned(D, g, [&](int h) {
            const int n = sidx[h];
            const float q = row_f32_sym(D.Ahi, D.cs, sidx, sp, h, n);
            D.q32[n] = q;
            v[0] = fmaf(sp[h], q, v[0]);
        });
    }
    grid_reduce<1, 0>(v, none, D.partial, D.counter + CNT_APPLY, blockIdx.x, gridDim.x,
                      [&](double* tot) { D.alpha = D.rz / tot[0]; });
}

void launch_assemble(Dev* d, const Dev& h, const AsmParams& P, cudaStream_t s) {
    k_assemble<<<(h.N + 127) / 128, 128, 0, s>>>(d, P);
}
void launch_realpha(Dev* d, const Dev& h, double delta, double alpha_dt, float cmass, cudaStream_t s) {
    k_realpha<<<(h.N + 255) / 256, 256, 0, s>>>(d, delta, alpha_dt, cmass);
}
void launch_realpha_ff(Dev* d, const Dev& h, double delta, double alpha_dt, float cmass, cudaStream_t s) {
    k_realpha_ff<<<(h.N + 255) / 256, 256, 0, s>>>(d, delta, alpha_dt, cmass);
}
void launch_rhs64(Dev* d, const Dev& h, int first, int graph, int grid, cudaStream_t s) {
    k_rhs64<<<grid, kStThreads, 0, s>>>(d, first, graph);
}
void launch_expand(Dev* d, const Dev& h, int want_a, int want_m, cudaStream_t s) {
    k_expand<<<(h.N + 127) / 128, 128, 0, s>>>(d, want_a, want_m);
}
void launch_p64(Dev* d, const Dev& h, int grid, cudaStream_t s) { k_p64<<<grid, kNodeThreads, 0, s>>>(d); }
void launch_apply64(Dev* d, const Dev& h, int grid, cudaStream_t s) { k_apply64<<<grid, kStThreads, 0, s>>>(d); }
void launch_update64(Dev* d, const Dev& h, int grid, int graph, cudaStream_t s) {
    k_update64<<<grid, kNodeThreads, 0, s>>>(d, graph);
}
void launch_apply32_stencil(Dev* d, const Dev& h, int grid, cudaStream_t s) {
    k_apply32_stencil<<<grid, kStThreads, 0, s>>>(d);
}

}  // namespace epk
