// k_ionic.cu -- fused ionic step at every node (paper Sec. 1.2, step 1 and
// the nodal ingredients of Eq. (6)).
//
// Per node j and step n -> n+1:
//   BDF combinations (order 1: alpha = 1, f_BDF = f_EXT = f_n; order 2:
//   alpha = 3/2, f_BDF = 2 f_n - f_{n-1}/2, f_EXT = 2 f_n - f_{n-1}; a BDF2
//   run takes a BDF1 first step) of u and of every ionic state;
//   Eq. (4): w_{n+1} = (w_BDF + dt a(u_EXT, w_EXT)) / (alpha + dt b(u_EXT, w_EXT));
//   I_ion,j = I_ion(u_EXT, w_{n+1}) (ionic current interpolation);
//   I_app,j = sum of the active pulses' amplitudes at the node;
//   v_j = u_BDF/dt - I_ion + I_app (Eq. (6) right-hand side is M v);
//   u_EXT (initial guess of the linear solve), both stored as double (FP64
//   path) or float-float (refined path).
// The new states overwrite the w_{n-1} slot (each thread owns its node), and
// the finishing kernel of the step swaps the slots.
//
// This file is compiled with fast single-precision intrinsics (exp, log,
// division): they only touch the FP32 path, whose float rates feed the
// double concentrations as increments; the FP64 path's double arithmetic is
// unaffected.  No double division appears per node (1/dt and 1/alpha are
// precomputed): GB300's FP64 pipe is ~60x slower than FP32.
#include "ep_dev.cuh"
#include "ionic_models.cuh"
#include "ep_ff.cuh"

namespace epk {

struct StepConsts {
    double dt, alpha, inv_dt, inv_alpha, dt_alpha;
    int order;
    double iamp[EP_MAX_PULSES];
};

__device__ __forceinline__ StepConsts step_consts(const Dev& D) {
    StepConsts c;
    c.dt = D.dt;
    c.order = (D.bdf == 2 && D.step >= 1) ? 2 : 1;
    c.alpha = c.order == 2 ? 1.5 : 1.0;
    c.inv_alpha = c.order == 2 ? 2.0 / 3.0 : 1.0;
    c.inv_dt = D.inv_dt;
    c.dt_alpha = c.dt * c.inv_alpha;
    const long long m = D.step + 1;  // new time level
#pragma unroll
    for (int p = 0; p < EP_MAX_PULSES; ++p) {
        double a = 0.0;
        if (p < D.npulses && m > D.k0[p]) {
            long long rel = m - D.k0[p] - 1;
            if (D.kp[p] > 0) rel %= D.kp[p];
            if (rel < D.kd[p]) a = D.amp[p];
        }
        c.iamp[p] = a;
    }
    return c;
}

__device__ __forceinline__ double applied(const Dev& D, const StepConsts& c, int n) {
    double s = 0.0;
#pragma unroll
    for (int p = 0; p < EP_MAX_PULSES; ++p)
        if (c.iamp[p] != 0.0 && D.mask[p][n]) s += c.iamp[p];
    return s;
}

// The right-hand side's nodal vector v and the solve's initial guess u_EXT:
// double in the FP64 path, float-float pairs in the refined one.
__device__ __forceinline__ void store_vu(const Dev& D, int n, double v, double uE) {
    if (D.v_hi) {
        ff_from_double(v, D.v_hi[n], D.v_lo[n]);
        ff_from_double(uE, D.u_hi[n], D.u_lo[n]);
    } else {
        D.v[n] = v;
        D.u_new[n] = uE;
    }
}

// G: arithmetic/storage type of the gates (float when refined, double in the
// FP64 path).  Concentrations are double either way.
template <typename G>
__global__ void __launch_bounds__(kNodeThreads) k_ionic_bo(Dev* __restrict__ Dp) {
    const Dev& D = *Dp;
    const StepConsts c = step_consts(D);
    const int N = D.N;
    G* __restrict__ wn;
    G* __restrict__ wm;
    if constexpr (sizeof(G) == 4) {
        wn = reinterpret_cast<G*>(D.g32_n);
        wm = reinterpret_cast<G*>(D.g32_nm1);
    } else {
        wn = reinterpret_cast<G*>(D.s64_n);
        wm = reinterpret_cast<G*>(D.s64_nm1);
    }
    const G dtg = G(c.dt), alg = G(c.alpha);
    for (int n = blockIdx.x * blockDim.x + threadIdx.x; n < N; n += gridDim.x * blockDim.x) {
        const double un = D.u_n[n];
        double uB = un, uE = un;
        G wB[3], wE[3];
        if (c.order == 2) {
            const double um = D.u_nm1[n];
            uB = 2.0 * un - 0.5 * um;
            uE = 2.0 * un - um;
#pragma unroll
            for (int k = 0; k < 3; ++k) {
                const G x = wn[(size_t)k * N + n], y = wm[(size_t)k * N + n];
                wB[k] = G(2) * x - G(0.5) * y;
                wE[k] = G(2) * x - y;
            }
        } else {
#pragma unroll
            for (int k = 0; k < 3; ++k) wB[k] = wE[k] = wn[(size_t)k * N + n];
        }
        (void)wE;  // BO rates depend on u only
        G a[3], b[3], w1[3];
        BO<G>::rates(G(uE), a, b);
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            w1[k] = (wB[k] + dtg * a[k]) / (alg + dtg * b[k]);
            wm[(size_t)k * N + n] = w1[k];
        }
        const double I = (double)BO<G>::iion(G(uE), w1[0], w1[1], w1[2]);
        store_vu(D, n, fma(uB, c.inv_dt, applied(D, c, n) - I), uE);
    }
}

template <typename G>
__global__ void __launch_bounds__(kNodeThreads) k_ionic_tt(Dev* __restrict__ Dp) {
    const Dev& D = *Dp;
    const StepConsts c = step_consts(D);
    const int N = D.N;
    // gate storage: float array (refined) or the first 13 rows of the double
    // state array (FP64); concentrations: the double array rows after them
    G* __restrict__ gn;
    G* __restrict__ gm;
    double* __restrict__ cn;
    double* __restrict__ cm;
    if constexpr (sizeof(G) == 4) {
        gn = reinterpret_cast<G*>(D.g32_n);
        gm = reinterpret_cast<G*>(D.g32_nm1);
        cn = D.s64_n;
        cm = D.s64_nm1;
    } else {
        gn = reinterpret_cast<G*>(D.s64_n);
        gm = reinterpret_cast<G*>(D.s64_nm1);
        cn = D.s64_n + (size_t)kTTGates * N;
        cm = D.s64_nm1 + (size_t)kTTGates * N;
    }
    const G dtg = G(c.dt), alg = G(c.alpha);
    for (int n = blockIdx.x * blockDim.x + threadIdx.x; n < N; n += gridDim.x * blockDim.x) {
        const int cell = D.cell[n];
        const double un = D.u_n[n];
        double uB = un, uE = un;
        G gB[kTTGates], gE[kTTGates];
        double cB[kTTConc], cE[kTTConc];
        if (c.order == 2) {
            const double um = D.u_nm1[n];
            uB = 2.0 * un - 0.5 * um;
            uE = 2.0 * un - um;
#pragma unroll
            for (int k = 0; k < kTTGates; ++k) {
                const G x = gn[(size_t)k * N + n], y = gm[(size_t)k * N + n];
                gB[k] = G(2) * x - G(0.5) * y;
                gE[k] = G(2) * x - y;
            }
#pragma unroll
            for (int k = 0; k < kTTConc; ++k) {
                const double x = cn[(size_t)k * N + n], y = cm[(size_t)k * N + n];
                cB[k] = 2.0 * x - 0.5 * y;
                cE[k] = 2.0 * x - y;
            }
        } else {
#pragma unroll
            for (int k = 0; k < kTTGates; ++k) gB[k] = gE[k] = gn[(size_t)k * N + n];
#pragma unroll
            for (int k = 0; k < kTTConc; ++k) cB[k] = cE[k] = cn[(size_t)k * N + n];
        }
        G a[kTTGates], b[kTTGates], r[kTTConc];
        TT<G>::rates(cell, G(uE), gE, G(cE[0]), G(cE[1]), G(cE[2]), G(cE[3]), G(cE[4]), a, b, r);
        G g1[kTTGates];
#pragma unroll
        for (int k = 0; k < kTTGates; ++k) {
            g1[k] = (gB[k] + dtg * a[k]) / (alg + dtg * b[k]);
            gm[(size_t)k * N + n] = g1[k];
        }
        double c1[kTTConc];
#pragma unroll
        for (int k = 0; k < kTTConc; ++k) {
            // the increment is formed in G, accumulated in double
            c1[k] = fma(c.dt_alpha, (double)r[k], cB[k] * c.inv_alpha);
            cm[(size_t)k * N + n] = c1[k];
        }
        typename TT<G>::Cur cur;
        TT<G>::currents(cell, G(uE), g1, G(c1[0]), G(c1[2]), G(c1[3]), G(c1[4]), cur);
        const double I = (double)TT<G>::iion_of(cur);
        store_vu(D, n, fma(uB, c.inv_dt, applied(D, c, n) - I), uE);
    }
}

void launch_ionic(Dev* d, const Dev& h, int grid, cudaStream_t s) {
    const bool refined = h.prec == EP_PREC_FP32_REFINED;
    if (h.model == EP_MODEL_BO) {
        if (refined) k_ionic_bo<float><<<grid, kNodeThreads, 0, s>>>(d);
        else k_ionic_bo<double><<<grid, kNodeThreads, 0, s>>>(d);
    } else {
        if (refined) k_ionic_tt<float><<<grid, kNodeThreads, 0, s>>>(d);
        else k_ionic_tt<double><<<grid, kNodeThreads, 0, s>>>(d);
    }
}

}  // namespace epk
