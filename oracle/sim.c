/*
 * sim.c -- oracle monodomain time stepping (TEST INFRASTRUCTURE ONLY; see
 * oracle.h).
 *
 * One step n -> n+1 follows paper Sec. 1.2 in its order:
 *   1. Eq. (4): every node's ionic states, w_{n+1} = (w_BDF + dt a)/(alpha + dt b)
 *      with (a, b) evaluated at (u_EXT, w_EXT);
 *   2. I_ion,j = I_ion(u_EXT,j, w_{n+1},j) at every node (ICI);
 *   3. Eq. (6): (alpha/dt M + K) u_{n+1} = M (u_BDF/dt - I_ion + I_app), where
 *      the history term is u_BDF (the time-discrete Eq. (5); the u_EXT printed
 *      in Eq. (6) is read as a typo) and the applied current enters as
 *      M I_app(nodes) like the ionic current;
 *   4. activation: keep the largest u_{n+1} - u_n and its time t_{n+1}.
 * BDF of order 2 takes a BDF1 first step.  Stimulus pulse p is active on
 * step n+1 when k0 < n+1 <= k0 + kd (k0 = round(t0/dt), kd = round(dur/dt)),
 * repeating every round(period/dt) steps when period > 0.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>

#include "oracle.h"

struct or_sim {
    int64_t nn;
    or_csr A;
    int model;
    uint8_t* cell;
    double g;
    double dt;
    int bdf;
    double tol;
    int maxit;
    int ns;
    int64_t step;
    double *u_n, *u_nm1, *w_n, *w_nm1, *w_new;
    double *u_nm2, *w_nm2;  /* level n-2 (BDF3) */
    double *iion, *rhs, *tmp, *u_new;
    double *at, *best;
    double act_thr;
    int npulses;
    or_pulse pulses[OR_MAX_PULSES];
    uint8_t* masks;
    double* iapp_extra;
    int have_extra;
    int last_iters;
    double last_relres;
    uint8_t* active;  /* 0: inactive node (no element left after exclusions) */
    double* weight[OR_MAX_PULSES];  /* per-node pulse profiles (NULL: mask) */
    double* region[OR_MAX_PULSES];  /* element-region vectors (NULL: nodal pulse) */
};

or_sim* or_sim_create(int64_t nn, int64_t ne, const double* xyz,
                      const int32_t* hex, const double* f0, const double* s0,
                      double dl, double dt_, double dn, int model,
                      const uint8_t* cell, double g, double dt, int bdf_order,
                      double tol, int maxit, int npulses,
                      const or_pulse* pulses, const uint8_t* masks,
                      double act_thr) {
    const double rdiff[3] = {dl, dt_, dn};
    const uint8_t excluded[1] = {0};
    return or_sim_create_regions(nn, ne, xyz, hex, f0, s0, NULL, 1, rdiff, excluded, model, cell, g,
                                 dt, bdf_order, tol, maxit, npulses, pulses, masks, act_thr);
}

/* npe 8: Q1 with subdomains; npe 27: Q2, one region */
static or_sim* create_general(int npe, int64_t nn, int64_t ne, const double* xyz,
                              const int32_t* hex, const double* f0,
                              const double* s0, const uint8_t* label, int nreg,
                              const double* rdiff, const uint8_t* excluded,
                              int model, const uint8_t* cell, double g,
                              double dt, int bdf_order, double tol, int maxit,
                              int npulses, const or_pulse* pulses,
                              const uint8_t* masks, double act_thr) {
    if (npulses < 0 || npulses > OR_MAX_PULSES || nn <= 0 || ne <= 0) return NULL;
    if (bdf_order < 1 || bdf_order > 3) return NULL;
    const int ns = or_model_nstates(model);
    if (ns < 0) return NULL;
    or_sim* S = calloc(1, sizeof(or_sim));
    S->nn = nn;
    S->active = malloc((size_t)nn);
    int rc;
    if (npe == 27) {
        rc = or_assemble_q2(nn, ne, xyz, hex, f0, s0, rdiff[0], rdiff[1], rdiff[2], &S->A);
        memset(S->active, 1, (size_t)nn);
    } else {
        rc = or_assemble_regions(nn, ne, xyz, hex, f0, s0, label, nreg, rdiff, excluded, &S->A,
                                 S->active);
    }
    if (rc != 0) {
        free(S->active);
        free(S);
        return NULL;
    }
    S->model = model;
    S->cell = malloc((size_t)nn);
    for (int64_t i = 0; i < nn; ++i) S->cell[i] = cell ? cell[i] : OR_CELL_EPI;
    S->g = g;
    S->dt = dt;
    S->bdf = bdf_order;
    S->tol = tol;
    S->maxit = maxit;
    S->ns = ns;
    S->act_thr = act_thr;
    const size_t N = (size_t)nn, NS = (size_t)(ns > 0 ? ns : 1) * N;
    S->u_n = calloc(N, sizeof(double));
    S->u_nm1 = calloc(N, sizeof(double));
    S->u_nm2 = calloc(N, sizeof(double));
    S->w_nm2 = calloc(NS, sizeof(double));
    S->u_new = calloc(N, sizeof(double));
    S->w_n = calloc(NS, sizeof(double));
    S->w_nm1 = calloc(NS, sizeof(double));
    S->w_new = calloc(NS, sizeof(double));
    S->iion = calloc(N, sizeof(double));
    S->rhs = calloc(N, sizeof(double));
    S->tmp = calloc(N, sizeof(double));
    S->at = malloc(N * sizeof(double));
    S->best = malloc(N * sizeof(double));
    S->iapp_extra = calloc(N, sizeof(double));
    for (int64_t i = 0; i < nn; ++i) {
        double u0, w0[OR_MAX_STATES];
        or_model_initial(model, S->cell[i], &u0, w0);
        S->u_n[i] = S->u_nm1[i] = S->u_nm2[i] = u0;
        for (int k = 0; k < ns; ++k)
            S->w_n[(size_t)k * N + i] = S->w_nm1[(size_t)k * N + i] = S->w_nm2[(size_t)k * N + i] = w0[k];
        S->at[i] = NAN;
        S->best[i] = -INFINITY;
    }
    S->npulses = npulses;
    for (int p = 0; p < npulses; ++p) S->pulses[p] = pulses[p];
    S->masks = malloc((size_t)(npulses > 0 ? npulses : 1) * N);
    if (npulses > 0) memcpy(S->masks, masks, (size_t)npulses * N);
    return S;
}

or_sim* or_sim_create_regions(int64_t nn, int64_t ne, const double* xyz,
                              const int32_t* hex, const double* f0,
                              const double* s0, const uint8_t* label, int nreg,
                              const double* rdiff, const uint8_t* excluded,
                              int model, const uint8_t* cell, double g,
                              double dt, int bdf_order, double tol, int maxit,
                              int npulses, const or_pulse* pulses,
                              const uint8_t* masks, double act_thr) {
    return create_general(8, nn, ne, xyz, hex, f0, s0, label, nreg, rdiff, excluded, model, cell, g,
                          dt, bdf_order, tol, maxit, npulses, pulses, masks, act_thr);
}

or_sim* or_sim_create_q2(int64_t nn, int64_t ne, const double* xyz,
                         const int32_t* hex27, const double* f0, const double* s0,
                         double dl, double dt_, double dn, int model,
                         const uint8_t* cell, double g, double dt,
                         int bdf_order, double tol, int maxit, int npulses,
                         const or_pulse* pulses, const uint8_t* masks,
                         double act_thr) {
    const double rdiff[3] = {dl, dt_, dn};
    const uint8_t excluded[1] = {0};
    return create_general(27, nn, ne, xyz, hex27, f0, s0, NULL, 1, rdiff, excluded, model, cell, g,
                          dt, bdf_order, tol, maxit, npulses, pulses, masks, act_thr);
}

void or_sim_destroy(or_sim* S) {
    if (!S) return;
    or_csr_free(&S->A);
    free(S->cell);
    free(S->u_n); free(S->u_nm1); free(S->u_new); free(S->u_nm2); free(S->w_nm2);
    free(S->w_n); free(S->w_nm1); free(S->w_new);
    free(S->iion); free(S->rhs); free(S->tmp);
    free(S->at); free(S->best); free(S->masks); free(S->iapp_extra);
    free(S->active);
    for (int p = 0; p < OR_MAX_PULSES; ++p) {
        free(S->weight[p]);
        free(S->region[p]);
    }
    free(S);
}

static int pulse_active(const or_pulse* P, double dt, int64_t m) {
    const int64_t k0 = llround(P->t0 / dt), kd = llround(P->dur / dt);
    if (m <= k0) return 0;
    int64_t rel = m - k0 - 1;  /* 0-based step within the train */
    if (P->period > 0.0) {
        const int64_t kp = llround(P->period / dt);
        if (kp > 0) rel %= kp;
    }
    return rel < kd;
}

static int step_once(or_sim* S) {
    const int64_t N = S->nn;
    const int ns = S->ns;
    /* order ramps 1, 2, 3 over the first steps up to the scheme's order */
    const int order = S->bdf < S->step + 1 ? S->bdf : (int)(S->step + 1);
    const double alpha = order == 3 ? 11.0 / 6.0 : (order == 2 ? 1.5 : 1.0);
    const double dt = S->dt;
    const int64_t m = S->step + 1;  /* index of the new time level */
    const double t_new = (double)m * dt;

    double amp_now[OR_MAX_PULSES];
    for (int p = 0; p < S->npulses; ++p)
        amp_now[p] = pulse_active(&S->pulses[p], dt, m) ? S->pulses[p].amp : 0.0;

    /* 1-2: ionic states and current at every node (Eq. (4), ICI); nodes are
     * independent, threads split them */
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < N; ++i) {
        double uB, uE, wB[OR_MAX_STATES], wE[OR_MAX_STATES], a[OR_MAX_STATES], b[OR_MAX_STATES], wn[OR_MAX_STATES];
        const double un = S->u_n[i], unm1 = S->u_nm1[i], unm2 = S->u_nm2[i];
        /* BDF combinations: f_BDF and the extrapolation f_EXT of the order */
        if (order == 3) {
            uB = 3.0 * un - 1.5 * unm1 + unm2 / 3.0;
            uE = 3.0 * un - 3.0 * unm1 + unm2;
        } else if (order == 2) {
            uB = 2.0 * un - 0.5 * unm1;
            uE = 2.0 * un - unm1;
        } else {
            uB = uE = un;
        }
        for (int k = 0; k < ns; ++k) {
            const size_t o = (size_t)k * N + i;
            const double x = S->w_n[o], y = S->w_nm1[o], z = S->w_nm2[o];
            if (order == 3) {
                wB[k] = 3.0 * x - 1.5 * y + z / 3.0;
                wE[k] = 3.0 * x - 3.0 * y + z;
            } else if (order == 2) {
                wB[k] = 2.0 * x - 0.5 * y;
                wE[k] = 2.0 * x - y;
            } else {
                wB[k] = wE[k] = x;
            }
        }
        if (!S->active[i]) {
            /* excluded from the simulation: states held, no currents */
            for (int k = 0; k < ns; ++k) S->w_new[(size_t)k * N + i] = S->w_n[(size_t)k * N + i];
            S->iion[i] = 0.0;
            S->tmp[i] = uB / dt;
            S->u_new[i] = uE;
            continue;
        }
        or_model_rates(S->model, S->cell[i], S->g, uE, wE, a, b);
        for (int k = 0; k < ns; ++k) {
            wn[k] = (wB[k] + dt * a[k]) / (alpha + dt * b[k]);
            S->w_new[(size_t)k * N + i] = wn[k];
        }
        const double I = or_model_iion(S->model, S->cell[i], S->g, uE, wn);
        S->iion[i] = I;
        double iapp = S->have_extra ? S->iapp_extra[i] : 0.0;
        for (int p = 0; p < S->npulses; ++p) {
            if (S->region[p]) continue;  /* added to the right-hand side below */
            if (S->weight[p]) iapp += amp_now[p] * S->weight[p][i];
            else if (S->masks[(size_t)p * N + i]) iapp += amp_now[p];
        }
        /* nodal vector that the mass matrix multiplies on the right of Eq. (6) */
        S->tmp[i] = uB / dt - I + iapp;
        S->u_new[i] = uE;  /* initial guess u_EXT */
    }
    S->have_extra = 0;

    /* 3: linear system, Eq. (6); applied currents on element regions enter
     * as their Gauss-integrated vectors */
    or_csr_apply(&S->A, 1.0, 0.0, S->tmp, S->rhs);
    for (int p = 0; p < S->npulses; ++p)
        if (S->region[p] && amp_now[p] != 0.0)
            for (int64_t i = 0; i < N; ++i) S->rhs[i] += amp_now[p] * S->region[p][i];
    const int it = or_pcg(&S->A, alpha / dt, 1.0, S->rhs, S->u_new, S->tol, S->maxit, &S->last_relres);
    S->last_iters = it;

    /* 4: activation, non-finite check, rotation */
    int bad = 0;
#pragma omp parallel for schedule(static) reduction(|| : bad)
    for (int64_t i = 0; i < N; ++i) {
        const double sl = S->u_new[i] - S->u_n[i];
        bad = bad || !isfinite(S->u_new[i]);
        if (sl > S->best[i]) {
            S->best[i] = sl;
            S->at[i] = t_new;
        }
    }
    double* t;
    t = S->u_nm2; S->u_nm2 = S->u_nm1; S->u_nm1 = S->u_n; S->u_n = S->u_new; S->u_new = t;
    t = S->w_nm2; S->w_nm2 = S->w_nm1; S->w_nm1 = S->w_n; S->w_n = S->w_new; S->w_new = t;
    S->step = m;
    if (it < 0) return -1;
    if (bad) return -2;
    return 0;
}

int or_sim_step(or_sim* S, int64_t nsteps) {
    for (int64_t k = 0; k < nsteps; ++k) {
        const int rc = step_once(S);
        if (rc != 0) return rc;
    }
    return 0;
}

void or_sim_set_iapp_extra(or_sim* S, const double* iapp) {
    if (iapp) {
        memcpy(S->iapp_extra, iapp, sizeof(double) * (size_t)S->nn);
        S->have_extra = 1;
    } else {
        S->have_extra = 0;
    }
}

int64_t or_sim_nodes(const or_sim* S) { return S->nn; }
void or_sim_get_active(const or_sim* S, uint8_t* active) { memcpy(active, S->active, (size_t)S->nn); }

void or_sim_set_pulse_weights(or_sim* S, int p, const double* weight) {
    if (p < 0 || p >= OR_MAX_PULSES) return;
    free(S->weight[p]);
    S->weight[p] = NULL;
    if (weight) {
        S->weight[p] = malloc((size_t)S->nn * sizeof(double));
        memcpy(S->weight[p], weight, (size_t)S->nn * sizeof(double));
    }
}
void or_sim_set_pulse_region(or_sim* S, int p, const double* vec) {
    if (p < 0 || p >= OR_MAX_PULSES) return;
    free(S->region[p]);
    S->region[p] = NULL;
    if (vec) {
        S->region[p] = malloc((size_t)S->nn * sizeof(double));
        memcpy(S->region[p], vec, (size_t)S->nn * sizeof(double));
    }
}
int or_sim_nstates(const or_sim* S) { return S->ns; }
int64_t or_sim_stepindex(const or_sim* S) { return S->step; }
int or_sim_last_iters(const or_sim* S) { return S->last_iters; }
double or_sim_last_relres(const or_sim* S) { return S->last_relres; }
const or_csr* or_sim_matrix(const or_sim* S) { return &S->A; }

void or_sim_get_state(const or_sim* S, double* u_n, double* u_nm1, double* w_n,
                      double* w_nm1) {
    const size_t N = (size_t)S->nn, NS = (size_t)S->ns * N;
    if (u_n) memcpy(u_n, S->u_n, N * sizeof(double));
    if (u_nm1) memcpy(u_nm1, S->u_nm1, N * sizeof(double));
    if (w_n && NS) memcpy(w_n, S->w_n, NS * sizeof(double));
    if (w_nm1 && NS) memcpy(w_nm1, S->w_nm1, NS * sizeof(double));
}

void or_sim_set_state(or_sim* S, const double* u_n, const double* u_nm1,
                      const double* w_n, const double* w_nm1, int64_t step) {
    const size_t N = (size_t)S->nn, NS = (size_t)S->ns * N;
    if (u_n) memcpy(S->u_n, u_n, N * sizeof(double));
    if (u_nm1) memcpy(S->u_nm1, u_nm1, N * sizeof(double));
    if (w_n && NS) memcpy(S->w_n, w_n, NS * sizeof(double));
    if (w_nm1 && NS) memcpy(S->w_nm1, w_nm1, NS * sizeof(double));
    S->step = step;
}

void or_sim_get_level2(const or_sim* S, double* u_nm2, double* w_nm2) {
    const size_t N = (size_t)S->nn, NS = (size_t)S->ns * N;
    if (u_nm2) memcpy(u_nm2, S->u_nm2, N * sizeof(double));
    if (w_nm2 && NS) memcpy(w_nm2, S->w_nm2, NS * sizeof(double));
}

void or_sim_set_level2(or_sim* S, const double* u_nm2, const double* w_nm2) {
    const size_t N = (size_t)S->nn, NS = (size_t)S->ns * N;
    if (u_nm2) memcpy(S->u_nm2, u_nm2, N * sizeof(double));
    if (w_nm2 && NS) memcpy(S->w_nm2, w_nm2, NS * sizeof(double));
}

void or_sim_get_activation(const or_sim* S, double* at, double* best) {
    for (int64_t i = 0; i < S->nn; ++i) {
        const int act = S->best[i] > S->act_thr * S->dt;
        if (at) at[i] = act ? S->at[i] : NAN;
        if (best) best[i] = S->best[i];
    }
}

void or_sim_get_activation_raw(const or_sim* S, double* at, double* best) {
    memcpy(at, S->at, sizeof(double) * (size_t)S->nn);
    memcpy(best, S->best, sizeof(double) * (size_t)S->nn);
}

void or_sim_set_activation(or_sim* S, const double* at, const double* best) {
    for (int64_t i = 0; i < S->nn; ++i) {
        S->at[i] = at[i];
        S->best[i] = best[i];
    }
}

void or_sim_get_iion(const or_sim* S, double* iion) {
    memcpy(iion, S->iion, sizeof(double) * (size_t)S->nn);
}

#ifdef _OPENMP
#include <omp.h>
#endif

/* Threads of the parallel loops (1 without OpenMP); n <= 0 keeps the
 * current setting.  Returns the number in effect. */
int or_set_threads(int n) {
#ifdef _OPENMP
    if (n > 0) omp_set_num_threads(n);
    return omp_get_max_threads();
#else
    (void)n;
    return 1;
#endif
}
