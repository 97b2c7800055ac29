// k_prepace.cu -- single-cell pre-pacing (the paper initialises its ionic
// models from long 0D simulations at the pacing period, Sec. 3.2).
//
// One thread per requested cell: Eq. (1) without diffusion, integrated with
// the semi-implicit step of Eq. (4) that the tissue step uses -- states whose
// rate is affine in themselves linearly implicit, concentrations explicit,
// all at (u_EXT, w_EXT) --, then u_{n+1} = (u_BDF + dt (I_app - I_ion(u_EXT,
// w_{n+1}))) / alpha.  BDF of order 2 takes a BDF1 first step.  Pulse train:
// I_app = amp on step m (new level) when (m - 1) mod kp < kd.  FP64
// throughout: a few threads, a setup step, no throughput concern.  The
// states live in global memory between launches, so a long protocol runs
// as a sequence of short launches.
#include "ep_dev.cuh"
#include "ionic_models.cuh"

namespace epk {

constexpr int kPPMax = 1 + kTTGates + kTTConc;  // u + states

// st: per cell [2][kPPMax] (levels n and n-1), m0: index of the level held
// as n (steps taken so far)
__global__ void k_prepace(int model, const uint8_t* __restrict__ cells, int ncell, double dt, long long m0,
                          long long nsteps, long long kp, long long kd, double amp, int bdf,
                          double* __restrict__ st) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= ncell) return;
    const int cell = cells[i];
    const int ns = model == EP_MODEL_BO ? kBOStates : kTTGates + kTTConc;
    double* s0 = st + (size_t)i * 2 * kPPMax;  // level n
    double* s1 = s0 + kPPMax;                  // level n-1
    double un = s0[0], um = s1[0];
    double wn[kPPMax - 1], wm[kPPMax - 1];
    for (int k = 0; k < ns; ++k) {
        wn[k] = s0[1 + k];
        wm[k] = s1[1 + k];
    }
    for (long long step = 0; step < nsteps; ++step) {
        const long long m = m0 + step + 1;  // new level
        const int order = (bdf == 2 && m >= 2) ? 2 : 1;
        const double alpha = order == 2 ? 1.5 : 1.0;
        const double iapp = ((m - 1) % kp) < kd ? amp : 0.0;
        double uB = un, uE = un, wB[kPPMax - 1], wE[kPPMax - 1], w1[kPPMax - 1];
        if (order == 2) {
            uB = 2.0 * un - 0.5 * um;
            uE = 2.0 * un - um;
        }
        for (int k = 0; k < ns; ++k) {
            wB[k] = order == 2 ? 2.0 * wn[k] - 0.5 * wm[k] : wn[k];
            wE[k] = order == 2 ? 2.0 * wn[k] - wm[k] : wn[k];
        }
        double I;
        if (model == EP_MODEL_BO) {
            double a[3], b[3];
            BO<double>::rates(uE, a, b);
            for (int k = 0; k < 3; ++k) w1[k] = (wB[k] + dt * a[k]) / (alpha + dt * b[k]);
            I = BO<double>::iion(uE, w1[0], w1[1], w1[2]);
        } else {
            double a[kTTGates], b[kTTGates], r[kTTConc];
            const double* cE = wE + kTTGates;
            TT<double>::rates(cell, uE, wE, cE[0], cE[1], cE[2], cE[3], cE[4], a, b, r);
            for (int k = 0; k < kTTGates; ++k) w1[k] = (wB[k] + dt * a[k]) / (alpha + dt * b[k]);
            for (int k = 0; k < kTTConc; ++k) w1[kTTGates + k] = (wB[kTTGates + k] + dt * r[k]) / alpha;
            const double* c1 = w1 + kTTGates;
            typename TT<double>::Cur cur;
            TT<double>::currents(cell, uE, w1, c1[0], c1[2], c1[3], c1[4], cur);
            I = TT<double>::iion_of(cur);
        }
        const double u1 = (uB + dt * (iapp - I)) / alpha;
        um = un;
        un = u1;
        for (int k = 0; k < ns; ++k) {
            wm[k] = wn[k];
            wn[k] = w1[k];
        }
    }
    s0[0] = un;
    s1[0] = um;
    for (int k = 0; k < ns; ++k) {
        s0[1 + k] = wn[k];
        s1[1 + k] = wm[k];
    }
}

cudaError_t launch_prepace(int model, const uint8_t* cells, int ncell, double dt, long long m0, long long nsteps,
                           long long kp, long long kd, double amp, int bdf, double* st, cudaStream_t s) {
    k_prepace<<<(ncell + 31) / 32, 32, 0, s>>>(model, cells, ncell, dt, m0, nsteps, kp, kd, amp, bdf, st);
    return cudaGetLastError();
}

}  // namespace epk
