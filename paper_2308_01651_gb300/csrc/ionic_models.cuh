// ionic_models.cuh -- device ionic models for the semi-implicit ionic step.
//
// Paper Sec. 1.1.1, Eq. (1): du/dt + I_ion(u, w) = I_app, dw/dt = H(u, w);
// the paper names the models but prints no equations, so they are restated
// from their source publications:
//   * Bueno-Orovio, Cherry & Fenton (2008) minimal model, epicardial set;
//     dimensionless u, u_mV = 85.7 u - 84 (Sec. 3.2.3).
//   * ten Tusscher & Panfilov (2006), 18 states besides V, currents in pA/pF.
// Every rate is produced as dw/dt = a - b w: b > 0 for states whose rate is
// affine in themselves (gates, BO v/w/s, TTP06 R), b = 0 for the explicit
// ones (TTP06 concentrations), so Eq. (4) becomes
// w_{n+1} = (w_BDF + dt a) / (alpha + dt b).
//
// T is the arithmetic type of rates and currents (float in the refined path,
// double in the FP64 path); concentrations are always stored in double.
#pragma once

#include <cuda_runtime.h>

namespace epk {

// ------------------------------------------------------------ Bueno-Orovio --

template <typename T>
struct BO {
    static constexpr T u_o = T(0), u_u = T(1.55), th_v = T(0.3), th_w = T(0.13),
                       th_vm = T(0.006), th_o = T(0.006);
    static constexpr T tv1m = T(60), tv2m = T(1150), tvp = T(1.4506);
    static constexpr T tw1m = T(60), tw2m = T(15), kwm = T(65), uwm = T(0.03), twp = T(200);
    static constexpr T tfi = T(0.11), to1 = T(400), to2 = T(6);
    static constexpr T tso1 = T(30.0181), tso2 = T(0.9957), kso = T(2.0458), uso = T(0.65);
    static constexpr T ts1 = T(2.7342), ts2 = T(16), ks = T(2.0994), us = T(0.9087);
    static constexpr T tsi = T(1.8875), twinf = T(0.07), winfs = T(0.94);

    // (a, b) of v, w, s at potential u
    __device__ static void rates(T u, T a[3], T b[3]) {
        const bool above_v = u >= th_v;
        const bool above_w = u >= th_w;
        const bool above_vm = u >= th_vm;
        const bool above_o = u >= th_o;
        if (above_v) {
            a[0] = T(0);
            b[0] = T(1) / tvp;
        } else {
            const T tvm = above_vm ? tv2m : tv1m;
            const T vinf = above_vm ? T(0) : T(1);
            a[0] = vinf / tvm;
            b[0] = T(1) / tvm;
        }
        if (above_w) {
            a[1] = T(0);
            b[1] = T(1) / twp;
        } else {
            const T twm = tw1m + (tw2m - tw1m) * T(0.5) * (T(1) + tanh(kwm * (u - uwm)));
            const T winf = above_o ? winfs : (T(1) - u / twinf);
            a[1] = winf / twm;
            b[1] = T(1) / twm;
        }
        const T ts = above_w ? ts2 : ts1;
        const T sinf = T(0.5) * (T(1) + tanh(ks * (u - us)));
        a[2] = sinf / ts;
        b[2] = T(1) / ts;
    }

    __device__ static T iion(T u, T v, T w, T s) {
        const bool above_v = u >= th_v;
        const bool above_w = u >= th_w;
        const T to = (u >= th_o) ? to2 : to1;
        const T jfi = above_v ? -v * (u - th_v) * (u_u - u) / tfi : T(0);
        T jso, jsi;
        if (above_w) {
            const T tso = tso1 + (tso2 - tso1) * T(0.5) * (T(1) + tanh(kso * (u - uso)));
            jso = T(1) / tso;
            jsi = -w * s / tsi;
        } else {
            jso = (u - u_o) / to;
            jsi = T(0);
        }
        return jfi + jso + jsi;
    }
};

// ---------------------------------------------------------- TTP06 -----------

// state order shared with the checkpoint layout:
// gates 0..12 = m h j xr1 xr2 xs s r d f f2 fCass RR, concentrations
// 13..17 = Cai CaSR CaSS Nai Ki
template <typename T>
struct TT {
    // constants (mV, ms, mM, pA/pF)
    static constexpr double RTF = 8314.472 * 310.0 / 96485.3415;  // RT/F in mV
    static constexpr double FARADAY = 96485.3415;
    static constexpr T Ko = T(5.4), Cao = T(2.0), Nao = T(140.0);
    static constexpr double Vc = 0.016404, Vsr = 0.001094, Vss = 0.00005468, Cap = 0.185;
    static constexpr T Bufc = T(0.2), Kbufc = T(0.001), Bufsr = T(10.0), Kbufsr = T(0.3),
                       Bufss = T(0.4), Kbufss = T(0.00025);
    static constexpr T Vmaxup = T(0.006375), Kup = T(0.00025), Vrel = T(0.102), k1p = T(0.15),
                       k2p = T(0.045), k3 = T(0.060), k4 = T(0.005), EC = T(1.5),
                       maxsr = T(2.5), minsr = T(1.0), Vleak = T(0.00036), Vxfer = T(0.0038);
    static constexpr T GKr = T(0.153), pKNa = T(0.03), GK1 = T(5.405), GNa = T(14.838),
                       GbNa = T(0.00029), KmK = T(1.0), KmNa = T(40.0), PNaK = T(2.724),
                       GCaL = T(3.980e-5), GbCa = T(0.000592), kNaCa = T(1000.0),
                       KmNai = T(87.5), KmCa = T(1.38), ksat = T(0.1), gam = T(0.35),
                       alf = T(2.5), GpCa = T(0.1238), KpCa = T(0.0005), GpK = T(0.0146);
    // derived
    static constexpr T iRTF = T(1.0 / RTF);
    static constexpr T capVcF = T(Cap / (Vc * FARADAY));        // Na+, K+ fluxes
    static constexpr T capVcF2 = T(Cap / (2.0 * Vc * FARADAY)); // Ca2+ to cytosol
    static constexpr T capVssF2 = T(Cap / (2.0 * Vss * FARADAY));
    static constexpr T VsrVc = T(Vsr / Vc), VsrVss = T(Vsr / Vss), VcVss = T(Vc / Vss);
    static constexpr T CaL_scale = T(2.0 * 96485.3415);  // 4 F^2/(RT) * RT/(2F)
    static constexpr T NaCa_den_inv = T(1.0 / ((87.5 * 87.5 * 87.5 + 140.0 * 140.0 * 140.0) * (1.38 + 2.0)));
    static constexpr T Nao3 = T(140.0 * 140.0 * 140.0);

    struct Cur {
        T INa, Ito, IKr, IKs, IK1, ICaL, INaCa, INaK, IpCa, IpK, IbNa, IbCa;
    };

    __device__ static void currents(int cell, T V, const T* g, T Cai, T CaSS, T Nai, T Ki, Cur& c) {
        const T EK = T(RTF) * log(Ko / Ki);
        const T ENa = T(RTF) * log(Nao / Nai);
        const T EKs = T(RTF) * log((Ko + pKNa * Nao) / (Ki + pKNa * Nai));
        const T ECa = T(0.5 * RTF) * log(Cao / Cai);
        const T m = g[0];
        c.INa = GNa * m * m * m * g[1] * g[2] * (V - ENa);
        const T gto = cell == EP_CELL_ENDO ? T(0.073) : T(0.294);
        const T gks = cell == EP_CELL_MID ? T(0.098) : T(0.392);
        c.Ito = gto * g[7] * g[6] * (V - EK);
        c.IKr = GKr * g[3] * g[4] * (V - EK);  // sqrt(Ko/5.4) = 1 at Ko = 5.4
        c.IKs = gks * g[5] * g[5] * (V - EKs);
        const T dK = V - EK;
        const T aK1 = T(0.1) / (T(1) + exp(T(0.06) * (dK - T(200))));
        const T bK1 = (T(3) * exp(T(0.0002) * (dK + T(100))) + exp(T(0.1) * (dK - T(10)))) /
                      (T(1) + exp(T(-0.5) * dK));
        c.IK1 = GK1 * aK1 / (aK1 + bK1) * dK;
        // L-type: with x = 2 (V - 15) F/(RT), the GHK factor (V-15)/(e^x - 1)
        // is (RT/2F) x/(e^x - 1), finite at x = 0
        const T x = T(2) * (V - T(15)) * iRTF;
        const T xe = (x == T(0)) ? T(1) : x / expm1(x);
        c.ICaL = GCaL * g[8] * g[9] * g[10] * g[11] * CaL_scale * xe *
                 (T(0.25) * CaSS * exp(x) - Cao);
        const T vf = V * iRTF;
        const T e1 = exp(gam * vf), e2 = exp((gam - T(1)) * vf);
        c.INaCa = kNaCa * NaCa_den_inv * (e1 * Nai * Nai * Nai * Cao - e2 * Nao3 * Cai * alf) /
                  (T(1) + ksat * e2);
        c.INaK = PNaK * (Ko / (Ko + KmK)) * (Nai / (Nai + KmNa)) /
                 (T(1) + T(0.1245) * exp(T(-0.1) * vf) + T(0.0353) * exp(-vf));
        c.IpCa = GpCa * Cai / (KpCa + Cai);
        c.IpK = GpK * (V - EK) / (T(1) + exp((T(25) - V) / T(5.98)));
        c.IbNa = GbNa * (V - ENa);
        c.IbCa = GbCa * (V - ECa);
    }

    __device__ static T iion_of(const Cur& c) {
        return c.IKr + c.IKs + c.IK1 + c.Ito + c.INa + c.IbNa + c.ICaL + c.IbCa + c.INaK + c.INaCa +
               c.IpCa + c.IpK;
    }

    // gate: a = x_inf / tau, b = 1 / tau
    __device__ static void gate(T xinf, T tau, T& a, T& b) {
        b = T(1) / tau;
        a = xinf * b;
    }

    // (a, b) of the 13 gates and the rates r of the 5 concentrations
    // (explicit, b = 0), all evaluated at (V, g, concentrations).
    __device__ static void rates(int cell, T V, const T* g, T Cai, T CaSR, T CaSS, T Nai, T Ki,
                                 T a[13], T b[13], T r[5]) {
        {   // INa activation m
            const T e = T(1) + exp((T(-56.86) - V) / T(9.03));
            const T am = T(1) / (T(1) + exp((T(-60) - V) / T(5)));
            const T bm = T(0.1) / (T(1) + exp((V + T(35)) / T(5))) +
                         T(0.1) / (T(1) + exp((V - T(50)) / T(200)));
            gate(T(1) / (e * e), am * bm, a[0], b[0]);
        }
        {   // INa inactivation h, j (branches at -40 mV)
            const T e = T(1) + exp((V + T(71.55)) / T(7.43));
            const T hinf = T(1) / (e * e);
            T ah, bh, aj, bj;
            if (V >= T(-40)) {
                ah = T(0);
                bh = T(0.77) / (T(0.13) * (T(1) + exp(-(V + T(10.66)) / T(11.1))));
                aj = T(0);
                bj = T(0.6) * exp(T(0.057) * V) / (T(1) + exp(T(-0.1) * (V + T(32))));
            } else {
                ah = T(0.057) * exp(-(V + T(80)) / T(6.8));
                bh = T(2.7) * exp(T(0.079) * V) + T(3.1e5) * exp(T(0.3485) * V);
                aj = (T(-2.5428e4) * exp(T(0.2444) * V) - T(6.948e-6) * exp(T(-0.04391) * V)) *
                     (V + T(37.78)) / (T(1) + exp(T(0.311) * (V + T(79.23))));
                bj = T(0.02424) * exp(T(-0.01052) * V) / (T(1) + exp(T(-0.1378) * (V + T(40.14))));
            }
            b[1] = ah + bh;
            a[1] = hinf * b[1];
            b[2] = aj + bj;
            a[2] = hinf * b[2];
        }
        {   // IKr xr1, xr2
            const T a1 = T(450) / (T(1) + exp((T(-45) - V) / T(10)));
            const T b1 = T(6) / (T(1) + exp((V + T(30)) / T(11.5)));
            gate(T(1) / (T(1) + exp((T(-26) - V) / T(7))), a1 * b1, a[3], b[3]);
            const T a2 = T(3) / (T(1) + exp((T(-60) - V) / T(20)));
            const T b2 = T(1.12) / (T(1) + exp((V - T(60)) / T(20)));
            gate(T(1) / (T(1) + exp((V + T(88)) / T(24))), a2 * b2, a[4], b[4]);
        }
        {   // IKs xs
            const T ax = T(1400) / sqrt(T(1) + exp((T(5) - V) / T(6)));
            const T bx = T(1) / (T(1) + exp((V - T(35)) / T(15)));
            gate(T(1) / (T(1) + exp((T(-5) - V) / T(14))), ax * bx + T(80), a[5], b[5]);
        }
        {   // Ito s (cell-type dependent), r
            T sinf, taus;
            if (cell == EP_CELL_ENDO) {
                sinf = T(1) / (T(1) + exp((V + T(28)) / T(5)));
                const T d = V + T(67);
                taus = T(1000) * exp(-d * d / T(1000)) + T(8);
            } else {
                sinf = T(1) / (T(1) + exp((V + T(20)) / T(5)));
                const T d = V + T(45);
                taus = T(85) * exp(-d * d / T(320)) + T(5) / (T(1) + exp((V - T(20)) / T(5))) + T(3);
            }
            gate(sinf, taus, a[6], b[6]);
            const T d = V + T(40);
            gate(T(1) / (T(1) + exp((T(20) - V) / T(6))), T(9.5) * exp(-d * d / T(1800)) + T(0.8),
                 a[7], b[7]);
        }
        {   // ICaL d, f, f2, fCass
            const T ad = T(1.4) / (T(1) + exp((T(-35) - V) / T(13))) + T(0.25);
            const T bd = T(1.4) / (T(1) + exp((V + T(5)) / T(5)));
            const T cd = T(1) / (T(1) + exp((T(50) - V) / T(20)));
            gate(T(1) / (T(1) + exp((T(-8) - V) / T(7.5))), ad * bd + cd, a[8], b[8]);
            const T d27 = V + T(27);
            const T tf = T(1102.5) * exp(-d27 * d27 / T(225)) + T(200) / (T(1) + exp((T(13) - V) / T(10))) +
                         T(180) / (T(1) + exp((V + T(30)) / T(10))) + T(20);
            gate(T(1) / (T(1) + exp((V + T(20)) / T(7))), tf, a[9], b[9]);
            const T tf2 = T(562) * exp(-d27 * d27 / T(240)) + T(31) / (T(1) + exp((T(25) - V) / T(10))) +
                          T(80) / (T(1) + exp((V + T(30)) / T(10)));
            gate(T(0.67) / (T(1) + exp((V + T(35)) / T(7))) + T(0.33), tf2, a[10], b[10]);
            const T q = CaSS / T(0.05);
            const T den = T(1) / (T(1) + q * q);
            gate(T(0.6) * den + T(0.4), T(80) * den + T(2), a[11], b[11]);
        }
        // SR release: RyR recovery R is affine in itself
        const T ec = EC / CaSR;
        const T kcasr = maxsr - (maxsr - minsr) / (T(1) + ec * ec);
        const T k1 = k1p / kcasr, k2 = k2p * kcasr;
        a[12] = k4;
        b[12] = k4 + k2 * CaSS;
        const T O = k1 * CaSS * CaSS * g[12] / (k3 + k1 * CaSS * CaSS);
        // concentrations (explicit)
        Cur c;
        currents(cell, V, g, Cai, CaSS, Nai, Ki, c);
        const T Irel = Vrel * O * (CaSR - CaSS);
        const T Iup = Vmaxup / (T(1) + (Kup * Kup) / (Cai * Cai));
        const T Ileak = Vleak * (CaSR - Cai);
        const T Ixfer = Vxfer * (CaSS - Cai);
        const T ci = Cai + Kbufc, csr = CaSR + Kbufsr, css = CaSS + Kbufss;
        const T Bi = T(1) / (T(1) + Bufc * Kbufc / (ci * ci));
        const T Bsr = T(1) / (T(1) + Bufsr * Kbufsr / (csr * csr));
        const T Bss = T(1) / (T(1) + Bufss * Kbufss / (css * css));
        r[0] = Bi * ((Ileak - Iup) * VsrVc + Ixfer - (c.IbCa + c.IpCa - T(2) * c.INaCa) * capVcF2);
        r[1] = Bsr * (Iup - Irel - Ileak);
        r[2] = Bss * (-c.ICaL * capVssF2 + Irel * VsrVss - Ixfer * VcVss);
        r[3] = -(c.INa + c.IbNa + T(3) * c.INaK + T(3) * c.INaCa) * capVcF;
        r[4] = -(c.IK1 + c.Ito + c.IKr + c.IKs - T(2) * c.INaK + c.IpK) * capVcF;
    }
};

// Paper Sec. 3.2.1: TTP06 epicardial initial state (V in mV), used for
// every cell type.
__host__ __device__ inline double tt_initial(int k) {
    const double w[18] = {0.00172, 0.7444, 0.7045, 0.00621, 0.4712, 0.00095, 0.999998, 2.42e-8,
                          3.373e-5, 0.7888, 0.9755, 0.9953, 0.9073, 0.000126, 3.64, 0.00036,
                          8.604, 136.89};
    return w[k];
}
constexpr double kTTInitialV = -85.23;

}  // namespace epk
