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
// division): they only touch the refined path's float arithmetic; the FP64
// path's double arithmetic is unaffected.  The refined path does no double
// arithmetic per node (GB300's FP64 pipe is ~60x slower than FP32): the
// potentials of the last two steps and the TTP06 concentrations are
// float-float pairs, the BDF combinations are formed in float-float, and the
// concentrations' BDF2 update is written as c_n + [(c_n - c_{n-1})/3 +
// (2/3) dt r] so that only a small increment is rounded to float.
//
// Refined states are packed four to a 16-byte group, group-major ([G][N]
// float4 per time level; ep_dev.cuh): one thread per node reads and writes its
// whole state with G 128-bit accesses, each coalesced across the warp (a
// warp moves 512 contiguous bytes per access).
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
    c.order = bdf_order(D);
    c.alpha = c.order == 3 ? 11.0 / 6.0 : (c.order == 2 ? 1.5 : 1.0);
    c.inv_alpha = c.order == 3 ? 6.0 / 11.0 : (c.order == 2 ? 2.0 / 3.0 : 1.0);
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
        if (c.iamp[p] != 0.0 && !D.eg64[p]) {  // element-region pulses enter b directly
            if (D.wgt64[p]) s += c.iamp[p] * D.wgt64[p][n];
            else if (D.mask[p][n]) s += c.iamp[p];
        }
    return s;
}

// FP64 path: v and u_EXT in double.
__device__ __forceinline__ void store_vu64(const Dev& D, int n, double v, double uE) {
    D.v[n] = v;
    D.u_new[n] = uE;
}

// The per-node end of the previous step of a refined instance, deferred from
// that step to this kernel (which reads the same potential levels): the
// activation slope u_n - u_{n-1} in float from the pairs, the largest slope
// and its time t (Sec. 3.2.1: first maximum wins), and u_n rounded to
// double for the public potential.  Idempotent: k_finish_ff does the same
// when the host reads the state between steps.
__device__ __forceinline__ void finish_prev_ff(const Dev& D, int n, double t, float h0, float l0, float h1,
                                               float l1) {
    const float s = (h0 - h1) + (l0 - l1);  // levels n and n-1
    D.u_n[n] = ff_to_double(h0, l0);
    if (s > D.bestf[n]) {
        D.bestf[n] = s;
        D.at[n] = t;
    }
}

// BDF combinations of one quantity from its levels n, n-1, n-2:
//   order 1: B = E = x;  order 2: B = 2x - y/2, E = 2x - y;
//   order 3: B = 3x - 3y/2 + z/3, E = 3x - 3y + z.
template <typename T>
__device__ __forceinline__ void bdf_comb(int order, T x, T y, T z, T& B, T& E) {
    if (order == 3) {
        B = T(3) * x - T(1.5) * y + z / T(3);
        E = T(3) * x - T(3) * y + z;
    } else if (order == 2) {
        B = T(2) * x - T(0.5) * y;
        E = T(2) * x - y;
    } else {
        B = E = x;
    }
}

// Refined path: the potential's BDF combinations from its float-float
// levels (the scalings by 2 and 1/2 are exact; by 3 and 1/3 float-float).
__device__ __forceinline__ void u_bdf_ff(const Dev& D, int order, int n, bool fin, double t_fin, float& bh,
                                         float& bl, float& eh, float& el) {
    const float h0 = D.uh_n[n], l0 = D.ul_n[n];
    float h1 = 0.f, l1 = 0.f;
    if (order >= 2 || fin) {
        h1 = D.uh_m[n];
        l1 = D.ul_m[n];
    }
    if (fin) finish_prev_ff(D, n, t_fin, h0, l0, h1, l1);
    if (order == 3) {
        const float h2 = D.uh_m2[n], l2 = D.ul_m2[n];
        float th, tl, ah, al, ch, cl;
        ff_mul(h0, l0, 3.f, 0.f, th, tl);      // 3 u_n
        ff_mul(h1, l1, 3.f, 0.f, ah, al);      // 3 u_{n-1}
        ff_sub(th, tl, ah, al, eh, el);
        ff_sub(eh, el, -h2, -l2, eh, el);      // + u_{n-2}
        ff_sub(th, tl, 1.5f * h1, 1.5f * l1, bh, bl);
        ff_mul(h2, l2, kThirdHi, kThirdLo, ch, cl);
        ff_sub(bh, bl, -ch, -cl, bh, bl);
    } else if (order == 2) {
        ff_sub(2.f * h0, 2.f * l0, 0.5f * h1, 0.5f * l1, bh, bl);
        ff_sub(2.f * h0, 2.f * l0, h1, l1, eh, el);
    } else {
        bh = eh = h0;
        bl = el = l0;
    }
}

// Refined path: v = uB / dt + (I_app - I_ion) and u_EXT as float-float pairs
__device__ __forceinline__ void store_vu_ff(const Dev& D, int n, float bh, float bl, float eh, float el,
                                            float src) {
    float vh, vl;
    ff_mul(bh, bl, D.idt_hi, D.idt_lo, vh, vl);
    ff_add_f(vh, vl, src, vh, vl);
    D.v_hi[n] = vh;
    D.v_lo[n] = vl;
    D.u_hi[n] = eh;
    D.u_lo[n] = el;
}

__device__ __forceinline__ float applied_f(const Dev& D, const StepConsts& c, int n) {
    float s = 0.f;
#pragma unroll
    for (int p = 0; p < EP_MAX_PULSES; ++p)
        if (c.iamp[p] != 0.0 && !D.egh[p]) {  // element-region pulses enter b directly
            if (D.wgt32[p]) s += (float)c.iamp[p] * D.wgt32[p][n];
            else if (D.mask[p][n]) s += (float)c.iamp[p];
        }
    return s;
}

// State levels: n, n-1 and (BDF3) n-2; the new level overwrites the oldest
// slot (n-2 for BDF3 instances, else n-1), the end of the step rotates.
template <typename G>
struct Levels {
    const G* n;
    const G* m;
    const G* m2;  // NULL unless BDF3
    G* out;
};

// one time level of a node's packed refined state (G float4 groups)
template <int G>
__device__ __forceinline__ void ld_packed(const float* base, size_t N, int n, float (&v)[4 * G]) {
    const float4* __restrict__ p = reinterpret_cast<const float4*>(base);
#pragma unroll
    for (int g = 0; g < G; ++g) {
        const float4 q = p[(size_t)g * N + n];
        v[4 * g] = q.x;
        v[4 * g + 1] = q.y;
        v[4 * g + 2] = q.z;
        v[4 * g + 3] = q.w;
    }
}

template <int G>
__device__ __forceinline__ void st_packed(float* base, size_t N, int n, const float (&v)[4 * G]) {
    float4* __restrict__ p = reinterpret_cast<float4*>(base);
#pragma unroll
    for (int g = 0; g < G; ++g) p[(size_t)g * N + n] = make_float4(v[4 * g], v[4 * g + 1], v[4 * g + 2], v[4 * g + 3]);
}

// G: arithmetic/storage type of the gates (float when refined, double in the
// FP64 path).
template <typename G, int BT>
__global__ void __launch_bounds__(BT) k_ionic_bo(Batch B) {
    const Slot S = batch_slot(B);
    const Dev& D = *S.D;
    const StepConsts c = step_consts(D);
    const int N = D.N;
    Levels<G> L;
    if constexpr (sizeof(G) == 4) {
        L = {reinterpret_cast<const G*>(D.g32_n), reinterpret_cast<const G*>(D.g32_nm1),
             reinterpret_cast<const G*>(D.g32_nm2), reinterpret_cast<G*>(D.g32_nm2 ? D.g32_nm2 : D.g32_nm1)};
    } else {
        L = {reinterpret_cast<const G*>(D.s64_n), reinterpret_cast<const G*>(D.s64_nm1),
             reinterpret_cast<const G*>(D.s64_nm2), reinterpret_cast<G*>(D.s64_nm2 ? D.s64_nm2 : D.s64_nm1)};
    }
    const G dtg = G(c.dt), alg = G(c.alpha);
    // refined path: the per-node end of the previous step, deferred to here
    const bool fin = sizeof(G) == 4 && D.fin_pending;
    const double t_fin = (double)D.step * D.dt;
    for (int n = S.blk * blockDim.x + threadIdx.x; n < N; n += S.nblk * blockDim.x) {
        G uEg;
        double uB = 0.0, uE = 0.0;
        float ubh = 0.f, ubl = 0.f, ueh = 0.f, uel = 0.f;
        if constexpr (sizeof(G) == 4) {
            u_bdf_ff(D, c.order, n, fin, t_fin, ubh, ubl, ueh, uel);
            uEg = ueh;
        } else {
            bdf_comb<double>(c.order, D.u_n[n], c.order > 1 ? D.u_nm1[n] : 0.0, c.order > 2 ? D.u_nm2[n] : 0.0,
                             uB, uE);
            uEg = uE;
        }
        G wB[3], wn0[3];
        if constexpr (sizeof(G) == 4) {
            // packed: v w s in one 16-byte group per level
            float s0[4], s1[4] = {0.f, 0.f, 0.f, 0.f}, s2[4] = {0.f, 0.f, 0.f, 0.f};
            ld_packed<kBOPacked>(D.g32_n, (size_t)N, n, s0);
            if (c.order > 1) ld_packed<kBOPacked>(D.g32_nm1, (size_t)N, n, s1);
            if (c.order > 2) ld_packed<kBOPacked>(D.g32_nm2, (size_t)N, n, s2);
#pragma unroll
            for (int k = 0; k < 3; ++k) {
                G E;
                wn0[k] = s0[k];
                bdf_comb<G>(c.order, s0[k], s1[k], s2[k], wB[k], E);
            }
        } else {
#pragma unroll
            for (int k = 0; k < 3; ++k) {
                const size_t o = (size_t)k * N + n;
                G E;
                wn0[k] = L.n[o];
                bdf_comb<G>(c.order, wn0[k], c.order > 1 ? L.m[o] : G(0), c.order > 2 ? L.m2[o] : G(0), wB[k], E);
            }
        }
        // an excluded node: states held, no currents
        const bool on = !D.active || D.active[n];
        // BO rates depend on u only
        G a[3], b[3], w1[3];
        BO<G>::rates(uEg, a, b);
#pragma unroll
        for (int k = 0; k < 3; ++k) w1[k] = on ? (wB[k] + dtg * a[k]) / (alg + dtg * b[k]) : wn0[k];
        if constexpr (sizeof(G) == 4) {
            const float o4[4] = {w1[0], w1[1], w1[2], 0.f};
            st_packed<kBOPacked>(reinterpret_cast<float*>(L.out), (size_t)N, n, o4);
        } else {
#pragma unroll
            for (int k = 0; k < 3; ++k) L.out[(size_t)k * N + n] = w1[k];
        }
        const G I = on ? BO<G>::iion(uEg, w1[0], w1[1], w1[2]) : G(0);
        if constexpr (sizeof(G) == 4) store_vu_ff(D, n, ubh, ubl, ueh, uel, on ? applied_f(D, c, n) - I : 0.f);
        else store_vu64(D, n, fma(uB, c.inv_dt, on ? applied(D, c, n) - (double)I : 0.0), uE);
    }
}

// The node loop of one instance at BDF order ORD; LV3: the instance keeps a
// third level (BDF3), into whose slot the new level goes (without one, the
// new level overwrites level n-1 in place).  Both are compile-time so that
// each variant keeps only its own levels and pointers live.  (Two-level
// instances run k_ionic_tt2 below.)
template <typename G, int ORD, bool LV3>
__device__ __forceinline__ void ionic_tt_nodes(const Slot& S, const Dev& D, const StepConsts& c) {
    const int N = D.N;
    const G dtg = G(c.dt), alg = G(c.alpha);
    constexpr int ord = ORD;
    // refined path: the per-node end of the previous step, deferred to here
    const bool fin = sizeof(G) == 4 && D.fin_pending;
    const double t_fin = (double)D.step * D.dt;
    for (int n = S.blk * blockDim.x + threadIdx.x; n < N; n += S.nblk * blockDim.x) {
        const int cell = D.cell[n];
        if constexpr (sizeof(G) == 4) {
            // ---- refined: float gates, float-float concentrations and
            // potentials, the levels packed (slots: 13 gates, 5 concentration
            // hi parts, 5 lo parts); the new level goes to the n-2 slot (LV3)
            // or over level n-1, after every level has been read
            constexpr int GH = kTTGates, GL = kTTGates + kTTConc;  // first hi, lo slot
            float* const out = LV3 ? D.g32_nm2 : D.g32_nm1;
            float ubh, ubl, ueh, uel;
            u_bdf_ff(D, ord, n, fin, t_fin, ubh, ubl, ueh, uel);
            if (D.active && !D.active[n]) {
                // excluded from the simulation: states held, no currents
                float t[4 * kTTPacked];
                ld_packed<kTTPacked>(D.g32_n, (size_t)N, n, t);
                st_packed<kTTPacked>(out, (size_t)N, n, t);
                store_vu_ff(D, n, ubh, ubl, ueh, uel, 0.f);
                continue;
            }
            float s0[4 * kTTPacked], s1[4 * kTTPacked], s2[4 * kTTPacked];
            ld_packed<kTTPacked>(D.g32_n, (size_t)N, n, s0);
            if (ord > 1) ld_packed<kTTPacked>(D.g32_nm1, (size_t)N, n, s1);
            if (ord > 2) ld_packed<kTTPacked>(D.g32_nm2, (size_t)N, n, s2);
            float gB[kTTGates], gE[kTTGates];
            float d1[kTTConc], d2[kTTConc], cE[kTTConc];
#pragma unroll
            for (int k = 0; k < kTTConc; ++k) {
                d1[k] = d2[k] = 0.f;
                // differences of consecutive levels: the hi parts are close,
                // so these are (nearly) exact
                float dh, dl;
                if (ord > 1) {
                    ff_sub(s0[GH + k], s0[GL + k], s1[GH + k], s1[GL + k], dh, dl);
                    d1[k] = dh;
                }
                if (ord > 2) {
                    ff_sub(s1[GH + k], s1[GL + k], s2[GH + k], s2[GL + k], dh, dl);
                    d2[k] = dh;
                }
                // c_EXT = c_n + (order 2) d1 + (order 3) 2 d1 - d2
                cE[k] = ord == 3 ? s0[GH + k] + (2.f * d1[k] - d2[k]) : s0[GH + k] + d1[k];
            }
#pragma unroll
            for (int k = 0; k < kTTGates; ++k)
                bdf_comb<float>(ord, s0[k], ord > 1 ? s1[k] : 0.f, ord > 2 ? s2[k] : 0.f, gB[k], gE[k]);
            float a[kTTGates], b[kTTGates], r[kTTConc];
            TT<float>::rates(cell, ueh, gE, cE[0], cE[1], cE[2], cE[3], cE[4], a, b, r);
            float o[4 * kTTPacked];
            o[4 * kTTPacked - 1] = 0.f;
#pragma unroll
            for (int k = 0; k < kTTGates; ++k) o[k] = (gB[k] + dtg * a[k]) / (alg + dtg * b[k]);
            const float dta = (float)c.dt_alpha;
#pragma unroll
            for (int k = 0; k < kTTConc; ++k) {
                // c_{n+1} = c_n + [(c_BDF - alpha c_n) + dt r] / alpha, with
                // (c_BDF - alpha c_n)/alpha = d1/3 (order 2), 7/11 d1 - 2/11 d2
                // (order 3): only the small increment is rounded to float
                float hist = 0.f;
                if (ord == 2) hist = d1[k] * (1.f / 3.f);
                else if (ord == 3) hist = fmaf(7.f / 11.f, d1[k], -(2.f / 11.f) * d2[k]);
                const float inc = fmaf(dta, r[k], hist);
                ff_add_f(s0[GH + k], s0[GL + k], inc, o[GH + k], o[GL + k]);
            }
            st_packed<kTTPacked>(out, (size_t)N, n, o);
            TT<float>::Cur cur;
            TT<float>::currents(cell, ueh, o, o[GH + 0], o[GH + 2], o[GH + 3], o[GH + 4], cur);
            const float I = TT<float>::iion_of(cur);
            store_vu_ff(D, n, ubh, ubl, ueh, uel, applied_f(D, c, n) - I);
        } else {
            // ---- FP64: every state in double
            const double* __restrict__ wn = D.s64_n;
            double* __restrict__ wm = D.s64_nm1;
            double* __restrict__ wm2 = D.s64_nm2;
            double* const wo = LV3 ? wm2 : wm;
            double uB, uE;
            bdf_comb<double>(ord, D.u_n[n], ord > 1 ? D.u_nm1[n] : 0.0, ord > 2 ? D.u_nm2[n] : 0.0, uB, uE);
            double wB[kTTGates + kTTConc], wE[kTTGates + kTTConc], w0[kTTGates + kTTConc];
#pragma unroll
            for (int k = 0; k < kTTGates + kTTConc; ++k) {
                const size_t o = (size_t)k * N + n;
                w0[k] = wn[o];
                bdf_comb<double>(ord, w0[k], ord > 1 ? wm[o] : 0.0, ord > 2 ? wm2[o] : 0.0, wB[k], wE[k]);
            }
            if (D.active && !D.active[n]) {
                // excluded from the simulation: states held, no currents
                for (int k = 0; k < kTTGates + kTTConc; ++k) wo[(size_t)k * N + n] = w0[k];
                store_vu64(D, n, uB * c.inv_dt, uE);
                continue;
            }
            const double* cE = wE + kTTGates;
            double a[kTTGates], b[kTTGates], r[kTTConc];
            TT<double>::rates(cell, uE, wE, cE[0], cE[1], cE[2], cE[3], cE[4], a, b, r);
            double g1[kTTGates];
#pragma unroll
            for (int k = 0; k < kTTGates; ++k) {
                g1[k] = (wB[k] + dtg * a[k]) / (alg + dtg * b[k]);
                wo[(size_t)k * N + n] = g1[k];
            }
            double c1[kTTConc];
#pragma unroll
            for (int k = 0; k < kTTConc; ++k) {
                c1[k] = fma(c.dt_alpha, r[k], wB[kTTGates + k] * c.inv_alpha);
                wo[(size_t)(kTTGates + k) * N + n] = c1[k];
            }
            TT<double>::Cur cur;
            TT<double>::currents(cell, uE, g1, c1[0], c1[2], c1[3], c1[4], cur);
            const double I = TT<double>::iion_of(cur);
            store_vu64(D, n, fma(uB, c.inv_dt, applied(D, c, n) - I), uE);
        }
    }
}

// BDF3 instances (three levels; the refined one holds three packed levels
// of a node at once: 128 registers, four 128-thread blocks per SM)
template <typename G, int BT>
__global__ void __launch_bounds__(BT, sizeof(G) == 4 ? 512 / BT : 1) k_ionic_tt3(Batch B) {
    const Slot S = batch_slot(B);
    const Dev& D = *S.D;
    const StepConsts c = step_consts(D);
    if (c.order == 3) ionic_tt_nodes<G, 3, true>(S, D, c);
    else if (c.order == 2) ionic_tt_nodes<G, 2, true>(S, D, c);
    else ionic_tt_nodes<G, 1, true>(S, D, c);
}

// Instances with two levels (BDF1, BDF2): the new level overwrites level n-1
// in place.  A kernel of its own, written for orders 1 and 2 only, so that
// its register allocation is not shaped by the three-level variant: the
// refined one fits the 80-register cap of six resident 128-thread blocks
// per SM without spills (the three-level one takes 128 registers, four).
template <typename G, int BT>
__global__ void __launch_bounds__(BT, sizeof(G) == 4 ? 768 / BT : 1) k_ionic_tt2(Batch B) {
    const Slot S = batch_slot(B);
    const Dev& D = *S.D;
    const StepConsts c = step_consts(D);
    const int N = D.N;
    const G dtg = G(c.dt), alg = G(c.alpha);
    // refined path: the per-node end of the previous step, deferred to here
    const bool fin = sizeof(G) == 4 && D.fin_pending;
    const double t_fin = (double)D.step * D.dt;
    for (int n = S.blk * blockDim.x + threadIdx.x; n < N; n += S.nblk * blockDim.x) {
        const int cell = D.cell[n];
        if constexpr (sizeof(G) == 4) {
            // ---- refined: float gates, float-float concentrations and
            // potentials, the levels packed (slots: 13 gates, 5 concentration
            // hi parts, 5 lo parts); the new level overwrites level n-1 after
            // both levels have been read
            constexpr int GH = kTTGates, GL = kTTGates + kTTConc;  // first hi, lo slot
            float ubh, ubl, ueh, uel;
            u_bdf_ff(D, c.order, n, fin, t_fin, ubh, ubl, ueh, uel);
            if (D.active && !D.active[n]) {
                // excluded from the simulation: states held, no currents
                float t[4 * kTTPacked];
                ld_packed<kTTPacked>(D.g32_n, (size_t)N, n, t);
                st_packed<kTTPacked>(D.g32_nm1, (size_t)N, n, t);
                store_vu_ff(D, n, ubh, ubl, ueh, uel, 0.f);
                continue;
            }
            float s0[4 * kTTPacked], s1[4 * kTTPacked];
            ld_packed<kTTPacked>(D.g32_n, (size_t)N, n, s0);
            if (c.order == 2) ld_packed<kTTPacked>(D.g32_nm1, (size_t)N, n, s1);
            float gB[kTTGates], gE[kTTGates];
            float dc[kTTConc], cE[kTTConc];
            if (c.order == 2) {
#pragma unroll
                for (int k = 0; k < kTTGates; ++k) {
                    gB[k] = 2.f * s0[k] - 0.5f * s1[k];
                    gE[k] = 2.f * s0[k] - s1[k];
                }
#pragma unroll
                for (int k = 0; k < kTTConc; ++k) {
                    // c_n - c_{n-1}: the hi parts are close, so their
                    // difference is exact
                    float dh, dl;
                    ff_sub(s0[GH + k], s0[GL + k], s1[GH + k], s1[GL + k], dh, dl);
                    dc[k] = dh;
                    cE[k] = s0[GH + k] + dc[k];
                }
            } else {
#pragma unroll
                for (int k = 0; k < kTTGates; ++k) gB[k] = gE[k] = s0[k];
#pragma unroll
                for (int k = 0; k < kTTConc; ++k) {
                    dc[k] = 0.f;
                    cE[k] = s0[GH + k];
                }
            }
            float a[kTTGates], b[kTTGates], r[kTTConc];
            TT<float>::rates(cell, ueh, gE, cE[0], cE[1], cE[2], cE[3], cE[4], a, b, r);
            float o[4 * kTTPacked];
            o[4 * kTTPacked - 1] = 0.f;
#pragma unroll
            for (int k = 0; k < kTTGates; ++k) o[k] = (gB[k] + dtg * a[k]) / (alg + dtg * b[k]);
            const float third = 1.f / 3.f, dta = (float)c.dt_alpha;
#pragma unroll
            for (int k = 0; k < kTTConc; ++k) {
                // order 1: c_n + dt r;  order 2: c_n + (c_n - c_{n-1})/3 + (2/3) dt r
                const float inc = c.order == 2 ? fmaf(third, dc[k], dta * r[k]) : dta * r[k];
                ff_add_f(s0[GH + k], s0[GL + k], inc, o[GH + k], o[GL + k]);
            }
            st_packed<kTTPacked>(D.g32_nm1, (size_t)N, n, o);
            TT<float>::Cur cur;
            TT<float>::currents(cell, ueh, o, o[GH + 0], o[GH + 2], o[GH + 3], o[GH + 4], cur);
            const float I = TT<float>::iion_of(cur);
            store_vu_ff(D, n, ubh, ubl, ueh, uel, applied_f(D, c, n) - I);
        } else {
            // ---- FP64: every state in double
            const double* __restrict__ gn = D.s64_n;
            double* __restrict__ gm = D.s64_nm1;
            const double* __restrict__ cn = D.s64_n + (size_t)kTTGates * N;
            double* __restrict__ cm = D.s64_nm1 + (size_t)kTTGates * N;
            const double un = D.u_n[n];
            double uB = un, uE = un;
            double gB[kTTGates], gE[kTTGates];
            double cB[kTTConc], cE[kTTConc];
            if (c.order == 2) {
                const double um = D.u_nm1[n];
                uB = 2.0 * un - 0.5 * um;
                uE = 2.0 * un - um;
#pragma unroll
                for (int k = 0; k < kTTGates; ++k) {
                    const double x = gn[(size_t)k * N + n], y = gm[(size_t)k * N + n];
                    gB[k] = 2.0 * x - 0.5 * y;
                    gE[k] = 2.0 * x - y;
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
            if (D.active && !D.active[n]) {
                // excluded from the simulation: states held, no currents
                for (int k = 0; k < kTTGates; ++k) gm[(size_t)k * N + n] = gn[(size_t)k * N + n];
                for (int k = 0; k < kTTConc; ++k) cm[(size_t)k * N + n] = cn[(size_t)k * N + n];
                store_vu64(D, n, uB * c.inv_dt, uE);
                continue;
            }
            double a[kTTGates], b[kTTGates], r[kTTConc];
            TT<double>::rates(cell, uE, gE, cE[0], cE[1], cE[2], cE[3], cE[4], a, b, r);
            double g1[kTTGates];
#pragma unroll
            for (int k = 0; k < kTTGates; ++k) {
                g1[k] = (gB[k] + dtg * a[k]) / (alg + dtg * b[k]);
                gm[(size_t)k * N + n] = g1[k];
            }
            double c1[kTTConc];
#pragma unroll
            for (int k = 0; k < kTTConc; ++k) {
                c1[k] = fma(c.dt_alpha, r[k], cB[k] * c.inv_alpha);
                cm[(size_t)k * N + n] = c1[k];
            }
            TT<double>::Cur cur;
            TT<double>::currents(cell, uE, g1, c1[0], c1[2], c1[3], c1[4], cur);
            const double I = TT<double>::iion_of(cur);
            store_vu64(D, n, fma(uB, c.inv_dt, applied(D, c, n) - I), uE);
        }
    }
}


// One launch of the instance's ionic kernel with BT threads per block.  The
// block size changes nothing in the results (one node per thread, no
// reductions): the create-time autotuner picks it per instance.
template <int BT>
void launch_ionic_bt(const Dev& h, const Batch& B, int grid, cudaStream_t s) {
    const bool refined = h.prec == EP_PREC_FP32_REFINED;
    if (h.model == EP_MODEL_BO) {
        if (refined) k_ionic_bo<float, BT><<<grid, BT, 0, s>>>(B);
        else k_ionic_bo<double, BT><<<grid, BT, 0, s>>>(B);
    } else if (h.u_nm2) {
        if (refined) k_ionic_tt3<float, BT><<<grid, BT, 0, s>>>(B);
        else k_ionic_tt3<double, BT><<<grid, BT, 0, s>>>(B);
    } else {
        if (refined) k_ionic_tt2<float, BT><<<grid, BT, 0, s>>>(B);
        else k_ionic_tt2<double, BT><<<grid, BT, 0, s>>>(B);
    }
}

void launch_ionic(Dev* d, const Dev& h, int grid, int threads, cudaStream_t s) {
    const Batch B = single_batch(d);
    if (threads == 64) launch_ionic_bt<64>(h, B, grid, s);
    else if (threads == 256) launch_ionic_bt<256>(h, B, grid, s);
    else launch_ionic_bt<128>(h, B, grid, s);
}

// refined instances of one model and number of levels, batched
void launch_ionic_batch(const Batch& B, int model, bool lv3, int grid, cudaStream_t s) {
    if (model == EP_MODEL_BO) k_ionic_bo<float, kIonicThreads><<<grid, kIonicThreads, 0, s>>>(B);
    else if (lv3) k_ionic_tt3<float, kIonicThreads><<<grid, kIonicThreads, 0, s>>>(B);
    else k_ionic_tt2<float, kIonicThreads><<<grid, kIonicThreads, 0, s>>>(B);
}

}  // namespace epk
