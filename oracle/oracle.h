/*
 * oracle.h -- plain FP64 CPU oracle for one IMEX monodomain time step of
 * lifex-ep (Africa et al., arXiv 2308.01651).
 *
 * TEST INFRASTRUCTURE ONLY.  This code exists to check the CUDA path: only the
 * test suite, the smoke check and the CPU-baseline leg of the benchmark may
 * load it.  It shares no source, header, table or helper with the CUDA
 * library, and the CUDA library never calls it.
 *
 * What it computes (paper Sec. 1.2, "numerical discretization"):
 *   - Eq. (4): the ionic ODEs, one BDF step per DoF, with states whose right
 *     hand side is affine in themselves taken implicitly and the rest
 *     explicitly, so the update is a direct division.
 *   - Eq. (6): (alpha/dt M + K) u_{n+1} = M u_BDF/dt - M I_ion + M I_app,
 *     with M, K assembled on Q1 hexahedra by 2x2x2 Gauss-Legendre quadrature
 *     (the minimum rule that integrates the mass matrix exactly), the ionic
 *     current and the applied current interpolated from the nodes (ICI).
 *   - Eq. (3): D = sigma_l f0 f0^T + sigma_t s0 s0^T + sigma_n n0 n0^T,
 *     written as sigma_n I + (sigma_l - sigma_n) f f^T + (sigma_t - sigma_n) s s^T
 *     with f, s the Q1 interpolants of the nodal fibre vectors at each
 *     quadrature point (not renormalised).
 *   - Jacobi-preconditioned CG to ||r||_2 <= tol ||b||_2, initial guess u_EXT.
 *   - Activation time (Sec. 3.2.1): time of the largest forward difference
 *     u_{n+1} - u_n at each node (first maximum wins).
 *
 * Units: ms, mV (Bueno-Orovio: dimensionless u), cm, mM.
 */
#ifndef GB300_EP_ORACLE_H
#define GB300_EP_ORACLE_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum { OR_MODEL_BO = 0, OR_MODEL_TTP06 = 1, OR_MODEL_PASSIVE = 2 };
enum { OR_CELL_ENDO = 0, OR_CELL_MID = 1, OR_CELL_EPI = 2 };
#define OR_MAX_STATES 18
#define OR_MAX_PULSES 8

/* ---- single-cell ionic models (Sec. 1.1.1, Eq. (1)) ------------------- */

/* Number of ionic state variables w (not counting u). */
int or_model_nstates(int model);
/* Resting / initial state.  TTP06 uses the epicardial initial conditions the
 * paper prints for the N-version benchmark (Sec. 3.2.1) for every cell type. */
void or_model_initial(int model, int cell, double* u0, double* w0);
/* Right-hand side of dw/dt written as a - b*w for every state.  States whose
 * rate is affine in themselves (gates, BO v/w/s, TTP06 R) return b > 0;
 * concentrations return their full rate in a and b = 0. */
void or_model_rates(int model, int cell, double g_passive, double u,
                    const double* w, double* a, double* b);
/* Ionic current I_ion(u, w) in model units per ms. */
double or_model_iion(int model, int cell, double g_passive, double u,
                     const double* w);

/* One semi-implicit single-cell step (Eq. (4) with the potential equation of
 * Eq. (1) treated like Eq. (5) without diffusion).  order 1 or 2; hist holds
 * u_{n-1}, w_{n-1} when order == 2.  Returns the new u and writes w_new. */
double or_cell_step(int model, int cell, double g_passive, int order, double dt,
                    double u_n, const double* w_n, double u_nm1,
                    const double* w_nm1, double iapp, double* w_new);

/* Single-cell pre-pacing (Sec. 3.2: ionic states initialised from 0D
 * simulations of many beats at the pacing period): beats beats of
 * or_cell_step under a pulse of amp lasting dur every period ms from t = 0
 * (the pulse is on for the new level m when (m - 1) mod kp < kd, kp =
 * round(period/dt), kd = round(dur/dt)); order bdf (a BDF1 first step).
 * init: NULL (or_model_initial) or u then the states; out: u then the
 * states at the end. */
void or_prepace(int model, int cell, int bdf, double dt, double period, int beats,
                double amp, double dur, const double* init, double* out);

/* ---- Q1 finite elements (Sec. 1.2, Eq. (6)) ---------------------------- */

/* Element mass and stiffness matrices (8x8, row-major, local node index
 * a = ia + 2 ib + 4 ic) of a trilinear hexahedron with vertex coordinates X,
 * nodal fibre vectors f, s and diffusivities dl, dt_, dn (cm^2/ms). */
void or_element_matrices(const double* X, const double* f, const double* s,
                         double dl, double dt_, double dn, double* Me,
                         double* Ke);

typedef struct {
    int64_t n;        /* rows */
    int64_t nnz;
    int64_t* rowptr;  /* n + 1 */
    int64_t* col;     /* nnz, sorted within each row */
    double* mval;     /* mass matrix values */
    double* kval;     /* stiffness matrix values */
} or_csr;

/* Assemble M and K on the same sparsity pattern.  Returns 0 on success. */
int or_assemble(int64_t nn, int64_t ne, const double* xyz, const int32_t* hex,
                const double* f0, const double* s0, double dl, double dt_,
                double dn, or_csr* A);

/* Subdomains (Sec. 1.1.2: a labelled partition of the domain, each part
 * with its own conductivities; a part labelled non-conductive is excluded
 * from the simulation, a conduction block).  label[e] in 0..nreg-1 per
 * element (NULL: all 0); rdiff[3 r + c] the diffusivities (dl, dt, dn) of
 * region r; excluded[r] != 0 removes region r's elements from M and K.  A
 * node none of whose elements remains is inactive: its row of M is a lone
 * diagonal, the consistent-mass diagonal its excluded elements would give
 * (so its equation scales like its neighbours'), its row of K zero, and
 * active[node] is set to 0 (else 1). */
#define OR_MAX_REGIONS 8
int or_assemble_regions(int64_t nn, int64_t ne, const double* xyz,
                        const int32_t* hex, const double* f0, const double* s0,
                        const uint8_t* label, int nreg, const double* rdiff,
                        const uint8_t* excluded, or_csr* A, uint8_t* active);
/* ---- Q2 finite elements (Sec. 1.2: hexahedra of arbitrary degree) ------- */
/* Element matrices (27x27, row-major) of a triquadratic 27-node hexahedron,
 * local node a = a0 + 3 a1 + 9 a2 at reference point (a0, a1, a2)/2 of
 * [0,1]^3, by 3x3x3 Gauss-Legendre quadrature (exact for the mass matrix of
 * a straight element); fibres Q2-interpolated to the quadrature points. */
void or_element_matrices_q2(const double* X, const double* f, const double* s,
                            double dl, double dt_, double dn, double* Me,
                            double* Ke);
/* Assembly over 27-node hexahedra (hex27: ne x 27 node indices in the local
 * order above). */
int or_assemble_q2(int64_t nn, int64_t ne, const double* xyz, const int32_t* hex27,
                   const double* f0, const double* s0, double dl, double dt_,
                   double dn, or_csr* A);
void or_csr_free(or_csr* A);
/* y = (cm*M + ck*K) x */
void or_csr_apply(const or_csr* A, double cm, double ck, const double* x,
                  double* y);

/* The vector of an applied current that is amp = 1 on a region of whole Q1
 * elements and 0 elsewhere, integrated against every basis function with the
 * 2x2x2 Gauss rule (Sec. 1.2: the vector arising from the applied current):
 * out[j] = sum over elements e with elem[e] != 0 of int_e phi_j, which is the
 * row sum of each such element's mass matrix (the basis sums to 1).  out has
 * nn entries and is overwritten. */
void or_element_region_vector(int64_t nn, int64_t ne, const double* xyz,
                              const int32_t* hex, const uint8_t* elem,
                              double* out);

/* Jacobi-PCG on (cm M + ck K) x = b; x holds the initial guess.  Returns the
 * iteration count, or -1 when maxit is reached. */
int or_pcg(const or_csr* A, double cm, double ck, const double* b, double* x,
           double tol, int maxit, double* relres_out);

/* ---- monodomain simulation ---------------------------------------------- */

typedef struct or_sim or_sim;

typedef struct {
    double amp;     /* model units per ms */
    double t0;      /* ms */
    double dur;     /* ms */
    double period;  /* ms; <= 0 means a single pulse */
} or_pulse;

/* Creates a simulation (BDF order 1, 2 or 3, ramping 1, 2, 3 over the first
 * steps: BDF3 takes a BDF1 then a BDF2 step).  cell may be NULL (all
 * epicardial).  masks holds
 * npulses x nn bytes (1 = node receives the pulse).  act_thr is the slope
 * (model units per ms) a node's largest forward difference must exceed to
 * count as activated. */
or_sim* or_sim_create(int64_t nn, int64_t ne, const double* xyz,
                      const int32_t* hex, const double* f0, const double* s0,
                      double dl, double dt_, double dn, int model,
                      const uint8_t* cell, double g_passive, double dt,
                      int bdf_order, double tol, int maxit, int npulses,
                      const or_pulse* pulses, const uint8_t* masks,
                      double act_thr);
/* The same with subdomains (see or_assemble_regions): an inactive node keeps
 * its ionic states, has no ionic or applied current, and so keeps its
 * potential. */
or_sim* or_sim_create_regions(int64_t nn, int64_t ne, const double* xyz,
                              const int32_t* hex, const double* f0,
                              const double* s0, const uint8_t* label, int nreg,
                              const double* rdiff, const uint8_t* excluded,
                              int model, const uint8_t* cell, double g_passive,
                              double dt, int bdf_order, double tol, int maxit,
                              int npulses, const or_pulse* pulses,
                              const uint8_t* masks, double act_thr);
/* The same on 27-node (Q2) hexahedra, one region. */
or_sim* or_sim_create_q2(int64_t nn, int64_t ne, const double* xyz,
                         const int32_t* hex27, const double* f0, const double* s0,
                         double dl, double dt_, double dn, int model,
                         const uint8_t* cell, double g_passive, double dt,
                         int bdf_order, double tol, int maxit, int npulses,
                         const or_pulse* pulses, const uint8_t* masks,
                         double act_thr);
/* Spatial profile of pulse p (Secs. 3.2.2 and 3.2.3: spherical and Gaussian impulses):
 * the node receives amp * weight[node] instead of amp * (mask[node] != 0).
 * NULL restores the mask.  The array is copied. */
void or_sim_set_pulse_weights(or_sim* S, int p, const double* weight);
/* Pulse p as an applied current on a region of elements (Gauss-point
 * integration, see or_element_region_vector): vec (nn doubles) is that
 * region's vector; the step adds amp(t) * vec to the right-hand side of
 * Eq. (6) after the mass product and the pulse's nodal mask is ignored.
 * NULL restores the nodal pulse. */
void or_sim_set_pulse_region(or_sim* S, int p, const double* vec);
/* 1 for an active node, 0 for an inactive one. */
void or_sim_get_active(const or_sim* S, uint8_t* active);
void or_sim_destroy(or_sim* S);
/* Advances nsteps steps; returns 0, or -1 on CG failure, -2 on non-finite. */
int or_sim_step(or_sim* S, int64_t nsteps);
/* Extra nodal applied current for the next step only (manufactured
 * solutions).  NULL clears it. */
void or_sim_set_iapp_extra(or_sim* S, const double* iapp);
int64_t or_sim_nodes(const or_sim* S);
int or_sim_nstates(const or_sim* S);
int64_t or_sim_stepindex(const or_sim* S);
int or_sim_last_iters(const or_sim* S);
double or_sim_last_relres(const or_sim* S);
/* Copies out / in u_n, u_{n-1}, w_n, w_{n-1} (state-major, ns x nn). */
void or_sim_get_state(const or_sim* S, double* u_n, double* u_nm1, double* w_n,
                      double* w_nm1);
void or_sim_set_state(or_sim* S, const double* u_n, const double* u_nm1,
                      const double* w_n, const double* w_nm1, int64_t step);
/* Level n-2 of u and the states (BDF3), copied out / in. */
void or_sim_get_level2(const or_sim* S, double* u_nm2, double* w_nm2);
void or_sim_set_level2(or_sim* S, const double* u_nm2, const double* w_nm2);
/* Activation times in ms (NaN where never activated) and the largest
 * forward difference seen so far. */
void or_sim_get_activation(const or_sim* S, double* at, double* best);
/* Same without the threshold: the time of the largest difference so far. */
void or_sim_get_activation_raw(const or_sim* S, double* at, double* best);
void or_sim_set_activation(or_sim* S, const double* at, const double* best);
/* Ionic current at the last step, nodal. */
void or_sim_get_iion(const or_sim* S, double* iion);
const or_csr* or_sim_matrix(const or_sim* S);

/* Threads of the oracle's parallel loops (OpenMP when built with it, else
 * 1): nodes of the ionic step and rows of the matrix products split among
 * threads; dot products summed in fixed chunks, so the result does not depend
 * on the thread count.  n <= 0 queries.  Returns the count in effect. */
int or_set_threads(int n);

#ifdef __cplusplus
}
#endif
#endif
