/*
 * ionic.c -- oracle ionic models (TEST INFRASTRUCTURE ONLY; see oracle.h).
 *
 * The paper (Sec. 1.1.1, Eq. (1)) names the models it ships and gives their
 * generic form du/dt + I_ion(u, w) = I_app, dw/dt = H(u, w); it prints no
 * model equations.  The equations below are restated from the models' source
 * publications:
 *   - Bueno-Orovio, Cherry, Fenton (2008), "minimal model", epicardial
 *     parameter set.  u is dimensionless; u_mV = 85.7 u - 84 (Sec. 3.2.3).
 *   - ten Tusscher, Panfilov (2006), human ventricular model, 18 states plus
 *     V, currents in pA/pF (= mV/ms with C_m = 1 uF/cm^2).  Initial state: the
 *     epicardial values the paper prints for the N-version benchmark
 *     (Sec. 3.2.1, parameter listing), used for every cell type.
 *   - a passive linear membrane I_ion = g u with no states, used only to check
 *     the time discretisation on manufactured solutions.
 *
 * Every rate is returned as dw/dt = a - b w.  The semi-implicit step of
 * Eq. (4) then reads w_{n+1} = (w_BDF + dt a) / (alpha + dt b): states whose
 * rate is affine in themselves (b > 0) are implicit, the rest (b = 0) are
 * explicit, as the paper's scheme has it.
 *
 * Parity unpinned (in part): the paper prints neither model, so the rates and
 * currents away from rest are pinned only by what the tests can fix without
 * them -- the BO rest state exact, the TTP06 initial state (the paper's)
 * staying within 1 mV for 1 s, action-potential features of the source
 * publications, the step converging to RK4 at first order, and end to end the
 * N-version activation time the paper reports.  A wrong constant that keeps
 * those features would go unnoticed by the oracle's pins.
 */
#include <math.h>
#include <string.h>

#include "oracle.h"

/* ------------------------------------------------------------------------ */
/* Bueno-Orovio minimal model, EPI parameters (ms, dimensionless u)          */
/* ------------------------------------------------------------------------ */

typedef struct {
    double u_o, u_u, th_v, th_w, th_vm, th_o;
    double tv1m, tv2m, tvp, tw1m, tw2m, kwm, uwm, twp, tfi;
    double to1, to2, tso1, tso2, kso, uso, ts1, ts2, ks, us, tsi, twinf, winfstar;
} bo_par;

static const bo_par BO_EPI = {
    0.0, 1.55, 0.3, 0.13, 0.006, 0.006,
    60.0, 1150.0, 1.4506, 60.0, 15.0, 65.0, 0.03, 200.0, 0.11,
    400.0, 6.0, 30.0181, 0.9957, 2.0458, 0.65, 2.7342, 16.0, 2.0994, 0.9087,
    1.8875, 0.07, 0.94};

/* Heaviside with H(0) = 1. */
static double heav(double x) { return x >= 0.0 ? 1.0 : 0.0; }

/* states: w[0] = v, w[1] = w, w[2] = s */
static void bo_rates(double u, const double* w, double* a, double* b) {
    const bo_par* P = &BO_EPI;
    (void)w;
    const double Hv = heav(u - P->th_v);
    const double Hw = heav(u - P->th_w);
    const double Hvm = heav(u - P->th_vm);
    const double Ho = heav(u - P->th_o);
    /* v: relaxes to v_inf with tau_v^- below theta_v, decays with tau_v^+ above */
    const double tvm = (1.0 - Hvm) * P->tv1m + Hvm * P->tv2m;
    const double vinf = (u < P->th_vm) ? 1.0 : 0.0;
    if (Hv > 0.0) { a[0] = 0.0; b[0] = 1.0 / P->tvp; }
    else          { a[0] = vinf / tvm; b[0] = 1.0 / tvm; }
    /* w: relaxes to w_inf with tau_w^- below theta_w, decays with tau_w^+ above */
    const double twm = P->tw1m + (P->tw2m - P->tw1m) * 0.5 * (1.0 + tanh(P->kwm * (u - P->uwm)));
    const double winf = (1.0 - Ho) * (1.0 - u / P->twinf) + Ho * P->winfstar;
    if (Hw > 0.0) { a[1] = 0.0; b[1] = 1.0 / P->twp; }
    else          { a[1] = winf / twm; b[1] = 1.0 / twm; }
    /* s: relaxes to (1 + tanh(k_s (u - u_s)))/2 with tau_s */
    const double ts = (1.0 - Hw) * P->ts1 + Hw * P->ts2;
    const double sinf = 0.5 * (1.0 + tanh(P->ks * (u - P->us)));
    a[2] = sinf / ts;
    b[2] = 1.0 / ts;
}

static double bo_iion(double u, const double* w) {
    const bo_par* P = &BO_EPI;
    const double Hv = heav(u - P->th_v);
    const double Hw = heav(u - P->th_w);
    const double Ho = heav(u - P->th_o);
    const double to = (1.0 - Ho) * P->to1 + Ho * P->to2;
    const double tso = P->tso1 + (P->tso2 - P->tso1) * 0.5 * (1.0 + tanh(P->kso * (u - P->uso)));
    const double Jfi = -w[0] * Hv * (u - P->th_v) * (P->u_u - u) / P->tfi;
    const double Jso = (u - P->u_o) * (1.0 - Hw) / to + Hw / tso;
    const double Jsi = -Hw * w[1] * w[2] / P->tsi;
    return Jfi + Jso + Jsi;
}

/* ------------------------------------------------------------------------ */
/* ten Tusscher-Panfilov 2006 (mV, ms, mM, pA/pF)                            */
/* ------------------------------------------------------------------------ */

enum {
    T_M = 0, T_H, T_J, T_XR1, T_XR2, T_XS, T_S, T_R, T_D, T_F, T_F2, T_FCASS,
    T_RR, T_CAI, T_CASR, T_CASS, T_NAI, T_KI, T_NSTATES
};

/* physical constants */
static const double TT_R = 8314.472, TT_T = 310.0, TT_F = 96485.3415;
static const double TT_KO = 5.4, TT_CAO = 2.0, TT_NAO = 140.0;
static const double TT_VC = 0.016404, TT_VSR = 0.001094, TT_VSS = 0.00005468;
static const double TT_CAP = 0.185;
/* buffering */
static const double TT_BUFC = 0.2, TT_KBUFC = 0.001, TT_BUFSR = 10.0,
                    TT_KBUFSR = 0.3, TT_BUFSS = 0.4, TT_KBUFSS = 0.00025;
/* SR fluxes */
static const double TT_VMAXUP = 0.006375, TT_KUP = 0.00025, TT_VREL = 0.102,
                    TT_K1P = 0.15, TT_K2P = 0.045, TT_K3 = 0.060, TT_K4 = 0.005,
                    TT_EC = 1.5, TT_MAXSR = 2.5, TT_MINSR = 1.0,
                    TT_VLEAK = 0.00036, TT_VXFER = 0.0038;
/* conductances */
static const double TT_GKR = 0.153, TT_PKNA = 0.03, TT_GK1 = 5.405,
                    TT_GNA = 14.838, TT_GBNA = 0.00029, TT_KMK = 1.0,
                    TT_KMNA = 40.0, TT_PNAK = 2.724, TT_GCAL = 3.980e-5,
                    TT_GBCA = 0.000592, TT_KNACA = 1000.0, TT_KMNAI = 87.5,
                    TT_KMCA = 1.38, TT_KSAT = 0.1, TT_GAMMA = 0.35,
                    TT_ALPHA = 2.5, TT_GPCA = 0.1238, TT_KPCA = 0.0005,
                    TT_GPK = 0.0146;

static double tt_gks(int cell) { return cell == OR_CELL_MID ? 0.098 : 0.392; }
static double tt_gto(int cell) { return cell == OR_CELL_ENDO ? 0.073 : 0.294; }

typedef struct {
    double INa, Ito, IKr, IKs, IK1, ICaL, INaCa, INaK, IpCa, IpK, IbNa, IbCa;
} tt_currents;

static void tt_currents_eval(int cell, double V, const double* w, tt_currents* c) {
    const double RTF = TT_R * TT_T / TT_F;  /* mV */
    const double Nai = w[T_NAI], Ki = w[T_KI], Cai = w[T_CAI], CaSS = w[T_CASS];
    const double EK = RTF * log(TT_KO / Ki);
    const double ENa = RTF * log(TT_NAO / Nai);
    const double EKs = RTF * log((TT_KO + TT_PKNA * TT_NAO) / (Ki + TT_PKNA * Nai));
    const double ECa = 0.5 * RTF * log(TT_CAO / Cai);

    c->INa = TT_GNA * w[T_M] * w[T_M] * w[T_M] * w[T_H] * w[T_J] * (V - ENa);
    c->Ito = tt_gto(cell) * w[T_R] * w[T_S] * (V - EK);
    c->IKr = TT_GKR * sqrt(TT_KO / 5.4) * w[T_XR1] * w[T_XR2] * (V - EK);
    c->IKs = tt_gks(cell) * w[T_XS] * w[T_XS] * (V - EKs);

    const double aK1 = 0.1 / (1.0 + exp(0.06 * (V - EK - 200.0)));
    const double bK1 = (3.0 * exp(0.0002 * (V - EK + 100.0)) + exp(0.1 * (V - EK - 10.0))) /
                       (1.0 + exp(-0.5 * (V - EK)));
    c->IK1 = TT_GK1 * sqrt(TT_KO / 5.4) * (aK1 / (aK1 + bK1)) * (V - EK);

    /* L-type current: GHK form around V - 15 mV.  With x = 2 (V-15) F/(RT),
     * (V-15)/(e^x - 1) = (RT/2F) * x/(e^x - 1), which is finite at x = 0. */
    const double x = 2.0 * (V - 15.0) / RTF;
    const double xe = (x == 0.0) ? 1.0 : x / expm1(x);
    c->ICaL = TT_GCAL * w[T_D] * w[T_F] * w[T_F2] * w[T_FCASS] * 4.0 * (TT_F / RTF) *
              (0.5 * RTF) * xe * (0.25 * CaSS * exp(x) - TT_CAO);

    const double eg = exp(TT_GAMMA * V / RTF), eg1 = exp((TT_GAMMA - 1.0) * V / RTF);
    c->INaCa = TT_KNACA *
               (eg * Nai * Nai * Nai * TT_CAO - eg1 * TT_NAO * TT_NAO * TT_NAO * Cai * TT_ALPHA) /
               ((TT_KMNAI * TT_KMNAI * TT_KMNAI + TT_NAO * TT_NAO * TT_NAO) *
                (TT_KMCA + TT_CAO) * (1.0 + TT_KSAT * eg1));
    c->INaK = TT_PNAK * TT_KO / (TT_KO + TT_KMK) * Nai / (Nai + TT_KMNA) /
              (1.0 + 0.1245 * exp(-0.1 * V / RTF) + 0.0353 * exp(-V / RTF));
    c->IpCa = TT_GPCA * Cai / (TT_KPCA + Cai);
    c->IpK = TT_GPK * (V - EK) / (1.0 + exp((25.0 - V) / 5.98));
    c->IbNa = TT_GBNA * (V - ENa);
    c->IbCa = TT_GBCA * (V - ECa);
}

static double tt_iion(int cell, double V, const double* w) {
    tt_currents c;
    tt_currents_eval(cell, V, w, &c);
    return c.IKr + c.IKs + c.IK1 + c.Ito + c.INa + c.IbNa + c.ICaL + c.IbCa +
           c.INaK + c.INaCa + c.IpCa + c.IpK;
}

/* gate in the form dw/dt = (winf - w)/tau  ->  a = winf/tau, b = 1/tau */
static void gate(double winf, double tau, double* a, double* b) {
    *a = winf / tau;
    *b = 1.0 / tau;
}

static void tt_rates(int cell, double V, const double* w, double* a, double* b) {
    /* fast sodium: m, h, j */
    {
        const double e = 1.0 + exp((-56.86 - V) / 9.03);
        const double minf = 1.0 / (e * e);
        const double am = 1.0 / (1.0 + exp((-60.0 - V) / 5.0));
        const double bm = 0.1 / (1.0 + exp((V + 35.0) / 5.0)) + 0.1 / (1.0 + exp((V - 50.0) / 200.0));
        gate(minf, am * bm, &a[T_M], &b[T_M]);

        const double eh = 1.0 + exp((V + 71.55) / 7.43);
        const double hinf = 1.0 / (eh * eh);
        double ah, bh, aj, bj;
        if (V >= -40.0) {
            ah = 0.0;
            bh = 0.77 / (0.13 * (1.0 + exp(-(V + 10.66) / 11.1)));
            aj = 0.0;
            bj = 0.6 * exp(0.057 * V) / (1.0 + exp(-0.1 * (V + 32.0)));
        } else {
            ah = 0.057 * exp(-(V + 80.0) / 6.8);
            bh = 2.7 * exp(0.079 * V) + 3.1e5 * exp(0.3485 * V);
            aj = (-2.5428e4 * exp(0.2444 * V) - 6.948e-6 * exp(-0.04391 * V)) * (V + 37.78) /
                 (1.0 + exp(0.311 * (V + 79.23)));
            bj = 0.02424 * exp(-0.01052 * V) / (1.0 + exp(-0.1378 * (V + 40.14)));
        }
        gate(hinf, 1.0 / (ah + bh), &a[T_H], &b[T_H]);
        gate(hinf, 1.0 / (aj + bj), &a[T_J], &b[T_J]);  /* j_inf = h_inf */
    }
    /* rapid delayed rectifier: xr1, xr2 */
    {
        const double xr1inf = 1.0 / (1.0 + exp((-26.0 - V) / 7.0));
        const double a1 = 450.0 / (1.0 + exp((-45.0 - V) / 10.0));
        const double b1 = 6.0 / (1.0 + exp((V + 30.0) / 11.5));
        gate(xr1inf, a1 * b1, &a[T_XR1], &b[T_XR1]);
        const double xr2inf = 1.0 / (1.0 + exp((V + 88.0) / 24.0));
        const double a2 = 3.0 / (1.0 + exp((-60.0 - V) / 20.0));
        const double b2 = 1.12 / (1.0 + exp((V - 60.0) / 20.0));
        gate(xr2inf, a2 * b2, &a[T_XR2], &b[T_XR2]);
    }
    /* slow delayed rectifier: xs */
    {
        const double xsinf = 1.0 / (1.0 + exp((-5.0 - V) / 14.0));
        const double axs = 1400.0 / sqrt(1.0 + exp((5.0 - V) / 6.0));
        const double bxs = 1.0 / (1.0 + exp((V - 35.0) / 15.0));
        gate(xsinf, axs * bxs + 80.0, &a[T_XS], &b[T_XS]);
    }
    /* transient outward: r, s (s depends on the cell type) */
    {
        const double rinf = 1.0 / (1.0 + exp((20.0 - V) / 6.0));
        const double taur = 9.5 * exp(-(V + 40.0) * (V + 40.0) / 1800.0) + 0.8;
        gate(rinf, taur, &a[T_R], &b[T_R]);
        double sinf, taus;
        if (cell == OR_CELL_ENDO) {
            sinf = 1.0 / (1.0 + exp((V + 28.0) / 5.0));
            taus = 1000.0 * exp(-(V + 67.0) * (V + 67.0) / 1000.0) + 8.0;
        } else {
            sinf = 1.0 / (1.0 + exp((V + 20.0) / 5.0));
            taus = 85.0 * exp(-(V + 45.0) * (V + 45.0) / 320.0) + 5.0 / (1.0 + exp((V - 20.0) / 5.0)) + 3.0;
        }
        gate(sinf, taus, &a[T_S], &b[T_S]);
    }
    /* L-type calcium: d, f, f2, fCass */
    {
        const double dinf = 1.0 / (1.0 + exp((-8.0 - V) / 7.5));
        const double ad = 1.4 / (1.0 + exp((-35.0 - V) / 13.0)) + 0.25;
        const double bd = 1.4 / (1.0 + exp((V + 5.0) / 5.0));
        const double cd = 1.0 / (1.0 + exp((50.0 - V) / 20.0));
        gate(dinf, ad * bd + cd, &a[T_D], &b[T_D]);
        const double finf = 1.0 / (1.0 + exp((V + 20.0) / 7.0));
        const double tauf = 1102.5 * exp(-(V + 27.0) * (V + 27.0) / 225.0) +
                            200.0 / (1.0 + exp((13.0 - V) / 10.0)) +
                            180.0 / (1.0 + exp((V + 30.0) / 10.0)) + 20.0;
        gate(finf, tauf, &a[T_F], &b[T_F]);
        const double f2inf = 0.67 / (1.0 + exp((V + 35.0) / 7.0)) + 0.33;
        const double tauf2 = 562.0 * exp(-(V + 27.0) * (V + 27.0) / 240.0) +
                             31.0 / (1.0 + exp((25.0 - V) / 10.0)) +
                             80.0 / (1.0 + exp((V + 30.0) / 10.0));
        gate(f2inf, tauf2, &a[T_F2], &b[T_F2]);
        const double q = w[T_CASS] / 0.05;
        const double fcinf = 0.6 / (1.0 + q * q) + 0.4;
        const double taufc = 80.0 / (1.0 + q * q) + 2.0;
        gate(fcinf, taufc, &a[T_FCASS], &b[T_FCASS]);
    }
    /* calcium handling: RyR recovery R (affine in R), concentrations (explicit) */
    {
        const double Cai = w[T_CAI], CaSR = w[T_CASR], CaSS = w[T_CASS];
        const double ecs = TT_EC / CaSR;
        const double kcasr = TT_MAXSR - (TT_MAXSR - TT_MINSR) / (1.0 + ecs * ecs);
        const double k1 = TT_K1P / kcasr, k2 = TT_K2P * kcasr;
        /* dR/dt = k4 (1 - R) - k2 CaSS R = k4 - (k4 + k2 CaSS) R */
        a[T_RR] = TT_K4;
        b[T_RR] = TT_K4 + k2 * CaSS;
        const double O = k1 * CaSS * CaSS * w[T_RR] / (TT_K3 + k1 * CaSS * CaSS);

        tt_currents c;
        tt_currents_eval(cell, V, w, &c);
        const double Irel = TT_VREL * O * (CaSR - CaSS);
        const double Iup = TT_VMAXUP / (1.0 + TT_KUP * TT_KUP / (Cai * Cai));
        const double Ileak = TT_VLEAK * (CaSR - Cai);
        const double Ixfer = TT_VXFER * (CaSS - Cai);
        const double Bi = 1.0 / (1.0 + TT_BUFC * TT_KBUFC / ((Cai + TT_KBUFC) * (Cai + TT_KBUFC)));
        const double Bsr = 1.0 / (1.0 + TT_BUFSR * TT_KBUFSR / ((CaSR + TT_KBUFSR) * (CaSR + TT_KBUFSR)));
        const double Bss = 1.0 / (1.0 + TT_BUFSS * TT_KBUFSS / ((CaSS + TT_KBUFSS) * (CaSS + TT_KBUFSS)));
        const double capVcF = TT_CAP / (TT_VC * TT_F);

        a[T_CAI] = Bi * ((Ileak - Iup) * TT_VSR / TT_VC + Ixfer -
                         (c.IbCa + c.IpCa - 2.0 * c.INaCa) * 0.5 * capVcF);
        a[T_CASR] = Bsr * (Iup - Irel - Ileak);
        a[T_CASS] = Bss * (-c.ICaL * TT_CAP / (2.0 * TT_VSS * TT_F) + Irel * TT_VSR / TT_VSS -
                           Ixfer * TT_VC / TT_VSS);
        a[T_NAI] = -(c.INa + c.IbNa + 3.0 * c.INaK + 3.0 * c.INaCa) * capVcF;
        a[T_KI] = -(c.IK1 + c.Ito + c.IKr + c.IKs - 2.0 * c.INaK + c.IpK) * capVcF;
        b[T_CAI] = b[T_CASR] = b[T_CASS] = b[T_NAI] = b[T_KI] = 0.0;
    }
}

/* Epicardial initial conditions printed in the paper (Sec. 3.2.1), converted
 * from V to mV. */
static const double TT_INIT_V = -85.23;
static const double TT_INIT_W[T_NSTATES] = {
    0.00172,   /* m */
    0.7444,    /* h */
    0.7045,    /* j */
    0.00621,   /* xr1 */
    0.4712,    /* xr2 */
    0.00095,   /* xs */
    0.999998,  /* s */
    2.42e-8,   /* r */
    3.373e-5,  /* d */
    0.7888,    /* f */
    0.9755,    /* f2 */
    0.9953,    /* fCass */
    0.9073,    /* R (RR) */
    0.000126,  /* Cai */
    3.64,      /* CaSR */
    0.00036,   /* CaSS */
    8.604,     /* Nai */
    136.89,    /* Ki */
};

/* ------------------------------------------------------------------------ */

int or_model_nstates(int model) {
    switch (model) {
    case OR_MODEL_BO: return 3;
    case OR_MODEL_TTP06: return T_NSTATES;
    case OR_MODEL_PASSIVE: return 0;
    default: return -1;
    }
}

void or_model_initial(int model, int cell, double* u0, double* w0) {
    (void)cell;
    switch (model) {
    case OR_MODEL_BO:
        *u0 = 0.0;
        w0[0] = 1.0; w0[1] = 1.0; w0[2] = 0.0;
        break;
    case OR_MODEL_TTP06:
        *u0 = TT_INIT_V;
        memcpy(w0, TT_INIT_W, sizeof(TT_INIT_W));
        break;
    default:
        *u0 = 0.0;
        break;
    }
}

void or_model_rates(int model, int cell, double g, double u, const double* w,
                    double* a, double* b) {
    (void)g;
    switch (model) {
    case OR_MODEL_BO: bo_rates(u, w, a, b); break;
    case OR_MODEL_TTP06: tt_rates(cell, u, w, a, b); break;
    default: break;
    }
}

double or_model_iion(int model, int cell, double g, double u, const double* w) {
    switch (model) {
    case OR_MODEL_BO: return bo_iion(u, w);
    case OR_MODEL_TTP06: return tt_iion(cell, u, w);
    case OR_MODEL_PASSIVE: return g * u;
    default: return 0.0;
    }
}

/* One single-cell step of the IMEX scheme: the states by Eq. (4), then the
 * potential by the zero-diffusion form of Eq. (5):
 *   (alpha u_{n+1} - u_BDF)/dt + I_ion(u_EXT, w_{n+1}) = I_app.
 * BDF coefficients: order 1: alpha = 1, f_BDF = f_n, f_EXT = f_n;
 * order 2: alpha = 3/2, f_BDF = 2 f_n - f_{n-1}/2, f_EXT = 2 f_n - f_{n-1}. */
double or_cell_step(int model, int cell, double g, int order, double dt,
                    double u_n, const double* w_n, double u_nm1,
                    const double* w_nm1, double iapp, double* w_new) {
    const int ns = or_model_nstates(model);
    double alpha, uB, uE;
    double wB[OR_MAX_STATES], wE[OR_MAX_STATES], a[OR_MAX_STATES], b[OR_MAX_STATES];
    if (order == 2) {
        alpha = 1.5;
        uB = 2.0 * u_n - 0.5 * u_nm1;
        uE = 2.0 * u_n - u_nm1;
        for (int k = 0; k < ns; ++k) {
            wB[k] = 2.0 * w_n[k] - 0.5 * w_nm1[k];
            wE[k] = 2.0 * w_n[k] - w_nm1[k];
        }
    } else {  /* order 1 (the single-cell step has no level n-2) */
        alpha = 1.0;
        uB = uE = u_n;
        for (int k = 0; k < ns; ++k) wB[k] = wE[k] = w_n[k];
    }
    or_model_rates(model, cell, g, uE, wE, a, b);
    for (int k = 0; k < ns; ++k) w_new[k] = (wB[k] + dt * a[k]) / (alpha + dt * b[k]);
    const double I = or_model_iion(model, cell, g, uE, w_new);
    return (uB + dt * (iapp - I)) / alpha;
}

void or_prepace(int model, int cell, int bdf, double dt, double period, int beats,
                double amp, double dur, const double* init, double* out) {
    const int ns = or_model_nstates(model);
    double un, um, wn[OR_MAX_STATES], wm[OR_MAX_STATES], w1[OR_MAX_STATES];
    if (init) {
        un = init[0];
        for (int k = 0; k < ns; ++k) wn[k] = init[1 + k];
    } else {
        or_model_initial(model, cell, &un, wn);
    }
    um = un;
    for (int k = 0; k < ns; ++k) wm[k] = wn[k];
    const long long kp = llround(period / dt), kd = llround(dur / dt);
    const long long total = kp * (long long)beats;
    for (long long m = 1; m <= total; ++m) {
        const int order = (bdf == 2 && m >= 2) ? 2 : 1;
        const double iapp = ((m - 1) % kp) < kd ? amp : 0.0;
        const double u1 = or_cell_step(model, cell, 0.0, order, dt, un, wn, um, wm, iapp, w1);
        um = un;
        un = u1;
        for (int k = 0; k < ns; ++k) {
            wm[k] = wn[k];
            wn[k] = w1[k];
        }
    }
    out[0] = un;
    for (int k = 0; k < ns; ++k) out[1 + k] = wn[k];
}
