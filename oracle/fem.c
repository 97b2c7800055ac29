/*
 * fem.c -- oracle Q1 and Q2 finite elements, CSR assembly, Jacobi-PCG
 * (TEST INFRASTRUCTURE ONLY; see oracle.h).
 *
 * Paper Sec. 1.2, Eq. (6): M_jk = int phi_k phi_j, K_jk = int D grad phi_k .
 * grad phi_j, integrals by Gauss-Legendre with the minimum number of points
 * that integrates the mass matrix exactly -- for trilinear hexahedra 2 points
 * per direction, for triquadratic (Q2, 27-node) hexahedra 3 (Sec. 1.2: the
 * polynomial degree p of hexahedral elements is arbitrary).  D follows Eq. (3)
 * with the fibre vectors interpolated from the nodes to each quadrature point
 * by the element's own shape functions.  The paper solves Eq. (6) with CG
 * (Sec. 2); this oracle uses the diagonal (Jacobi) preconditioner.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>

#include "oracle.h"

/* trilinear shape function a at reference point xi in [0,1]^3 and its
 * reference gradient; local node a = ia + 2 ib + 4 ic sits at (ia, ib, ic). */
static void q1_shape(int a, const double xi[3], double* phi, double dphi[3]) {
    const int ia = a & 1, ib = (a >> 1) & 1, ic = (a >> 2) & 1;
    const double l0 = ia ? xi[0] : 1.0 - xi[0];
    const double l1 = ib ? xi[1] : 1.0 - xi[1];
    const double l2 = ic ? xi[2] : 1.0 - xi[2];
    const double d0 = ia ? 1.0 : -1.0;
    const double d1 = ib ? 1.0 : -1.0;
    const double d2 = ic ? 1.0 : -1.0;
    *phi = l0 * l1 * l2;
    dphi[0] = d0 * l1 * l2;
    dphi[1] = l0 * d1 * l2;
    dphi[2] = l0 * l1 * d2;
}

static double det3(const double J[3][3]) {
    return J[0][0] * (J[1][1] * J[2][2] - J[1][2] * J[2][1]) -
           J[0][1] * (J[1][0] * J[2][2] - J[1][2] * J[2][0]) +
           J[0][2] * (J[1][0] * J[2][1] - J[1][1] * J[2][0]);
}

void or_element_matrices(const double* X, const double* f, const double* s,
                         double dl, double dt_, double dn, double* Me,
                         double* Ke) {
    /* 2-point Gauss-Legendre on [0,1]: nodes 1/2 -+ 1/(2 sqrt 3), weights 1/2 */
    const double g[2] = {0.5 - 0.5 / sqrt(3.0), 0.5 + 0.5 / sqrt(3.0)};
    const double wq = 0.125;
    memset(Me, 0, 64 * sizeof(double));
    memset(Ke, 0, 64 * sizeof(double));
    for (int q = 0; q < 8; ++q) {
        const double xi[3] = {g[q & 1], g[(q >> 1) & 1], g[(q >> 2) & 1]};
        double phi[8], dphi[8][3];
        for (int a = 0; a < 8; ++a) q1_shape(a, xi, &phi[a], dphi[a]);
        /* Jacobian J_ij = d x_i / d xi_j */
        double J[3][3] = {{0}};
        for (int a = 0; a < 8; ++a)
            for (int i = 0; i < 3; ++i)
                for (int j = 0; j < 3; ++j) J[i][j] += X[3 * a + i] * dphi[a][j];
        const double detJ = det3(J);
        /* inverse by cofactors */
        double Ji[3][3];
        Ji[0][0] = (J[1][1] * J[2][2] - J[1][2] * J[2][1]) / detJ;
        Ji[0][1] = (J[0][2] * J[2][1] - J[0][1] * J[2][2]) / detJ;
        Ji[0][2] = (J[0][1] * J[1][2] - J[0][2] * J[1][1]) / detJ;
        Ji[1][0] = (J[1][2] * J[2][0] - J[1][0] * J[2][2]) / detJ;
        Ji[1][1] = (J[0][0] * J[2][2] - J[0][2] * J[2][0]) / detJ;
        Ji[1][2] = (J[0][2] * J[1][0] - J[0][0] * J[1][2]) / detJ;
        Ji[2][0] = (J[1][0] * J[2][1] - J[1][1] * J[2][0]) / detJ;
        Ji[2][1] = (J[0][1] * J[2][0] - J[0][0] * J[2][1]) / detJ;
        Ji[2][2] = (J[0][0] * J[1][1] - J[0][1] * J[1][0]) / detJ;
        /* physical gradients: grad phi = J^{-T} dphi, (grad)_i = sum_j Ji[j][i] dphi_j */
        double G[8][3];
        for (int a = 0; a < 8; ++a)
            for (int i = 0; i < 3; ++i)
                G[a][i] = Ji[0][i] * dphi[a][0] + Ji[1][i] * dphi[a][1] + Ji[2][i] * dphi[a][2];
        /* fibre vectors at the quadrature point (Q1 interpolation, not normalised) */
        double fq[3] = {0, 0, 0}, sq[3] = {0, 0, 0};
        for (int a = 0; a < 8; ++a)
            for (int i = 0; i < 3; ++i) {
                fq[i] += phi[a] * f[3 * a + i];
                sq[i] += phi[a] * s[3 * a + i];
            }
        /* D = dn I + (dl - dn) f f^T + (dt - dn) s s^T  (Eq. (3) with n0 implied) */
        double D[3][3];
        for (int i = 0; i < 3; ++i)
            for (int j = 0; j < 3; ++j)
                D[i][j] = (i == j ? dn : 0.0) + (dl - dn) * fq[i] * fq[j] + (dt_ - dn) * sq[i] * sq[j];
        const double w = wq * detJ;
        for (int a = 0; a < 8; ++a) {
            double DGa[3];
            for (int i = 0; i < 3; ++i)
                DGa[i] = D[i][0] * G[a][0] + D[i][1] * G[a][1] + D[i][2] * G[a][2];
            for (int b = 0; b < 8; ++b) {
                Me[8 * a + b] += w * phi[a] * phi[b];
                Ke[8 * a + b] += w * (DGa[0] * G[b][0] + DGa[1] * G[b][1] + DGa[2] * G[b][2]);
            }
        }
    }
}

/* 1-D quadratic Lagrange polynomials on [0,1] with nodes 0, 1/2, 1 and
 * their derivatives */
static void q2_1d(double t, double l[3], double d[3]) {
    l[0] = (1.0 - t) * (1.0 - 2.0 * t);
    l[1] = 4.0 * t * (1.0 - t);
    l[2] = t * (2.0 * t - 1.0);
    d[0] = 4.0 * t - 3.0;
    d[1] = 4.0 - 8.0 * t;
    d[2] = 4.0 * t - 1.0;
}

void or_element_matrices_q2(const double* X, const double* f, const double* s,
                            double dl, double dt_, double dn, double* Me,
                            double* Ke) {
    /* 3-point Gauss-Legendre on [0,1]: 1/2 -+ sqrt(15)/10 and 1/2, weights
     * 5/18, 8/18, 5/18 */
    const double r = sqrt(15.0) / 10.0;
    const double g[3] = {0.5 - r, 0.5, 0.5 + r};
    const double w1[3] = {5.0 / 18.0, 8.0 / 18.0, 5.0 / 18.0};
    memset(Me, 0, 729 * sizeof(double));
    memset(Ke, 0, 729 * sizeof(double));
    for (int q = 0; q < 27; ++q) {
        const int q0 = q % 3, q1 = (q / 3) % 3, q2 = q / 9;
        double l0[3], d0[3], l1[3], d1[3], l2[3], d2[3];
        q2_1d(g[q0], l0, d0);
        q2_1d(g[q1], l1, d1);
        q2_1d(g[q2], l2, d2);
        double phi[27], dphi[27][3];
        for (int a = 0; a < 27; ++a) {
            const int a0 = a % 3, a1 = (a / 3) % 3, a2 = a / 9;
            phi[a] = l0[a0] * l1[a1] * l2[a2];
            dphi[a][0] = d0[a0] * l1[a1] * l2[a2];
            dphi[a][1] = l0[a0] * d1[a1] * l2[a2];
            dphi[a][2] = l0[a0] * l1[a1] * d2[a2];
        }
        double J[3][3] = {{0}};
        for (int a = 0; a < 27; ++a)
            for (int i = 0; i < 3; ++i)
                for (int j = 0; j < 3; ++j) J[i][j] += X[3 * a + i] * dphi[a][j];
        const double detJ = det3(J);
        double Ji[3][3];
        Ji[0][0] = (J[1][1] * J[2][2] - J[1][2] * J[2][1]) / detJ;
        Ji[0][1] = (J[0][2] * J[2][1] - J[0][1] * J[2][2]) / detJ;
        Ji[0][2] = (J[0][1] * J[1][2] - J[0][2] * J[1][1]) / detJ;
        Ji[1][0] = (J[1][2] * J[2][0] - J[1][0] * J[2][2]) / detJ;
        Ji[1][1] = (J[0][0] * J[2][2] - J[0][2] * J[2][0]) / detJ;
        Ji[1][2] = (J[0][2] * J[1][0] - J[0][0] * J[1][2]) / detJ;
        Ji[2][0] = (J[1][0] * J[2][1] - J[1][1] * J[2][0]) / detJ;
        Ji[2][1] = (J[0][1] * J[2][0] - J[0][0] * J[2][1]) / detJ;
        Ji[2][2] = (J[0][0] * J[1][1] - J[0][1] * J[1][0]) / detJ;
        double G[27][3];
        for (int a = 0; a < 27; ++a)
            for (int i = 0; i < 3; ++i)
                G[a][i] = Ji[0][i] * dphi[a][0] + Ji[1][i] * dphi[a][1] + Ji[2][i] * dphi[a][2];
        double fq[3] = {0, 0, 0}, sq[3] = {0, 0, 0};
        for (int a = 0; a < 27; ++a)
            for (int i = 0; i < 3; ++i) {
                fq[i] += phi[a] * f[3 * a + i];
                sq[i] += phi[a] * s[3 * a + i];
            }
        double D[3][3];
        for (int i = 0; i < 3; ++i)
            for (int j = 0; j < 3; ++j)
                D[i][j] = (i == j ? dn : 0.0) + (dl - dn) * fq[i] * fq[j] + (dt_ - dn) * sq[i] * sq[j];
        const double w = w1[q0] * w1[q1] * w1[q2] * detJ;
        for (int a = 0; a < 27; ++a) {
            double DGa[3];
            for (int i = 0; i < 3; ++i)
                DGa[i] = D[i][0] * G[a][0] + D[i][1] * G[a][1] + D[i][2] * G[a][2];
            for (int b = 0; b < 27; ++b) {
                Me[27 * a + b] += w * phi[a] * phi[b];
                Ke[27 * a + b] += w * (DGa[0] * G[b][0] + DGa[1] * G[b][1] + DGa[2] * G[b][2]);
            }
        }
    }
}

static int cmp_i64(const void* a, const void* b) {
    const int64_t x = *(const int64_t*)a, y = *(const int64_t*)b;
    return (x > y) - (x < y);
}

static int64_t find_col(const or_csr* A, int64_t row, int64_t col) {
    int64_t lo = A->rowptr[row], hi = A->rowptr[row + 1] - 1;
    while (lo <= hi) {
        const int64_t mid = (lo + hi) / 2;
        if (A->col[mid] == col) return mid;
        if (A->col[mid] < col) lo = mid + 1;
        else hi = mid - 1;
    }
    return -1;
}

int or_assemble(int64_t nn, int64_t ne, const double* xyz, const int32_t* hex,
                const double* f0, const double* s0, double dl, double dt_,
                double dn, or_csr* A) {
    const double rdiff[3] = {dl, dt_, dn};
    const uint8_t excluded[1] = {0};
    return or_assemble_regions(nn, ne, xyz, hex, f0, s0, NULL, 1, rdiff, excluded, A, NULL);
}

/* Assembly over elements of npe nodes (8: Q1, 27: Q2). */
static int assemble_general(int npe, int64_t nn, int64_t ne, const double* xyz,
                            const int32_t* hex, const double* f0, const double* s0,
                            const uint8_t* label, int nreg, const double* rdiff,
                            const uint8_t* excluded, or_csr* A, uint8_t* active) {
    if (npe != 8 && npe != 27) return -1;
    if (nreg < 1 || nreg > OR_MAX_REGIONS) return -1;
    if (label)
        for (int64_t e = 0; e < ne; ++e)
            if (label[e] >= nreg) return -1;
    memset(A, 0, sizeof(*A));
    /* node -> element incidence */
    int64_t* cnt = calloc((size_t)nn + 1, sizeof(int64_t));
    if (!cnt) return -1;
    for (int64_t e = 0; e < ne; ++e)
        for (int a = 0; a < npe; ++a) cnt[hex[(int64_t)npe * e + a] + 1]++;
    for (int64_t i = 0; i < nn; ++i) cnt[i + 1] += cnt[i];
    int64_t* inc = malloc(sizeof(int64_t) * (size_t)(cnt[nn] > 0 ? cnt[nn] : 1));
    int64_t* fill = calloc((size_t)nn, sizeof(int64_t));
    if (!inc || !fill) { free(cnt); free(inc); free(fill); return -1; }
    for (int64_t e = 0; e < ne; ++e)
        for (int a = 0; a < npe; ++a) {
            const int64_t v = hex[(int64_t)npe * e + a];
            inc[cnt[v] + fill[v]++] = e;
        }
    /* sparsity: neighbours of each node through its elements */
    A->n = nn;
    A->rowptr = calloc((size_t)nn + 1, sizeof(int64_t));
    int64_t cap = 27 * nn + 64, nnz = 0;
    A->col = malloc(sizeof(int64_t) * (size_t)cap);
    int64_t tmp[27 * 64];
    for (int64_t v = 0; v < nn; ++v) {
        int nt = 0;
        for (int64_t k = cnt[v]; k < cnt[v + 1]; ++k) {
            const int64_t e = inc[k];
            for (int a = 0; a < npe && nt < 27 * 64; ++a) tmp[nt++] = hex[(int64_t)npe * e + a];
        }
        qsort(tmp, (size_t)nt, sizeof(int64_t), cmp_i64);
        for (int i = 0; i < nt; ++i) {
            if (i > 0 && tmp[i] == tmp[i - 1]) continue;
            if (nnz >= cap) {
                cap *= 2;
                A->col = realloc(A->col, sizeof(int64_t) * (size_t)cap);
            }
            A->col[nnz++] = tmp[i];
        }
        A->rowptr[v + 1] = nnz;
    }
    A->nnz = nnz;
    A->mval = calloc((size_t)nnz, sizeof(double));
    A->kval = calloc((size_t)nnz, sizeof(double));
    /* element loop (excluded elements contribute nothing to M and K; their
       mass diagonal is kept aside for the nodes they leave inactive) */
    uint8_t* has = calloc((size_t)nn, 1);
    double* mexcl = calloc((size_t)nn, sizeof(double));
    double* X = malloc(sizeof(double) * 3 * (size_t)npe);
    double* F = malloc(sizeof(double) * 3 * (size_t)npe);
    double* S = malloc(sizeof(double) * 3 * (size_t)npe);
    double* Me = malloc(sizeof(double) * (size_t)npe * npe);
    double* Ke = malloc(sizeof(double) * (size_t)npe * npe);
    for (int64_t e = 0; e < ne; ++e) {
        const int r = label ? label[e] : 0;
        const int32_t* el = hex + (int64_t)npe * e;
        for (int a = 0; a < npe; ++a) {
            const int64_t v = el[a];
            for (int i = 0; i < 3; ++i) {
                X[3 * a + i] = xyz[3 * v + i];
                F[3 * a + i] = f0[3 * v + i];
                S[3 * a + i] = s0[3 * v + i];
            }
        }
        if (npe == 8) or_element_matrices(X, F, S, rdiff[3 * r], rdiff[3 * r + 1], rdiff[3 * r + 2], Me, Ke);
        else or_element_matrices_q2(X, F, S, rdiff[3 * r], rdiff[3 * r + 1], rdiff[3 * r + 2], Me, Ke);
        if (excluded[r]) {
            for (int a = 0; a < npe; ++a) mexcl[el[a]] += Me[(npe + 1) * a];
            continue;
        }
        for (int a = 0; a < npe; ++a) has[el[a]] = 1;
        for (int a = 0; a < npe; ++a) {
            const int64_t row = el[a];
            for (int b = 0; b < npe; ++b) {
                const int64_t p = find_col(A, row, el[b]);
                A->mval[p] += Me[npe * a + b];
                A->kval[p] += Ke[npe * a + b];
            }
        }
    }
    free(X);
    free(F);
    free(S);
    free(Me);
    free(Ke);
    /* inactive nodes: a lone mass diagonal (the consistent-mass diagonal of
       their excluded elements, so that their rows scale like the others), no
       stiffness */
    for (int64_t v = 0; v < nn; ++v) {
        if (active) active[v] = has[v];
        if (!has[v]) A->mval[find_col(A, v, v)] = mexcl[v];
    }
    free(mexcl);
    free(has);
    free(cnt);
    free(inc);
    free(fill);
    return 0;
}

int or_assemble_regions(int64_t nn, int64_t ne, const double* xyz,
                        const int32_t* hex, const double* f0, const double* s0,
                        const uint8_t* label, int nreg, const double* rdiff,
                        const uint8_t* excluded, or_csr* A, uint8_t* active) {
    return assemble_general(8, nn, ne, xyz, hex, f0, s0, label, nreg, rdiff, excluded, A, active);
}

int or_assemble_q2(int64_t nn, int64_t ne, const double* xyz, const int32_t* hex27,
                   const double* f0, const double* s0, double dl, double dt_,
                   double dn, or_csr* A) {
    const double rdiff[3] = {dl, dt_, dn};
    const uint8_t excluded[1] = {0};
    return assemble_general(27, nn, ne, xyz, hex27, f0, s0, NULL, 1, rdiff, excluded, A, NULL);
}

void or_element_region_vector(int64_t nn, int64_t ne, const double* xyz,
                              const int32_t* hex, const uint8_t* elem,
                              double* out) {
    /* fibres do not enter the mass matrix: any unit vectors do */
    static const double fz[24] = {1, 0, 0, 1, 0, 0, 1, 0, 0, 1, 0, 0, 1, 0, 0, 1, 0, 0, 1, 0, 0, 1, 0, 0};
    static const double sz[24] = {0, 1, 0, 0, 1, 0, 0, 1, 0, 0, 1, 0, 0, 1, 0, 0, 1, 0, 0, 1, 0, 0, 1, 0};
    for (int64_t j = 0; j < nn; ++j) out[j] = 0.0;
    for (int64_t e = 0; e < ne; ++e) {
        if (!elem[e]) continue;
        double X[24], Me[64], Ke[64];
        for (int a = 0; a < 8; ++a)
            for (int c = 0; c < 3; ++c) X[3 * a + c] = xyz[3 * (size_t)hex[8 * e + a] + c];
        or_element_matrices(X, fz, sz, 1.0, 1.0, 1.0, Me, Ke);
        for (int a = 0; a < 8; ++a) {
            double row = 0.0;
            for (int b = 0; b < 8; ++b) row += Me[8 * a + b];
            out[hex[8 * e + a]] += row;
        }
    }
}

void or_csr_free(or_csr* A) {
    free(A->rowptr);
    free(A->col);
    free(A->mval);
    free(A->kval);
    memset(A, 0, sizeof(*A));
}

void or_csr_apply(const or_csr* A, double cm, double ck, const double* x,
                  double* y) {
    /* rows are independent: threads split them, each row summed in order */
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < A->n; ++i) {
        double acc = 0.0;
        for (int64_t p = A->rowptr[i]; p < A->rowptr[i + 1]; ++p)
            acc += (cm * A->mval[p] + ck * A->kval[p]) * x[A->col[p]];
        y[i] = acc;
    }
}

/* Dot product in a fixed order that does not depend on the thread count:
 * chunks of OR_DOT_CHUNK consecutive terms are summed in index order, then
 * the chunk sums in chunk order.  One thread or many give the same bits. */
#define OR_DOT_CHUNK 8192
static double dot(int64_t n, const double* a, const double* b) {
    const int64_t nc = (n + OR_DOT_CHUNK - 1) / OR_DOT_CHUNK;
    double* part = malloc(sizeof(double) * (size_t)(nc > 0 ? nc : 1));
#pragma omp parallel for schedule(static)
    for (int64_t c = 0; c < nc; ++c) {
        const int64_t lo = c * OR_DOT_CHUNK, hi = lo + OR_DOT_CHUNK < n ? lo + OR_DOT_CHUNK : n;
        double s = 0.0;
        for (int64_t i = lo; i < hi; ++i) s += a[i] * b[i];
        part[c] = s;
    }
    double s = 0.0;
    for (int64_t c = 0; c < nc; ++c) s += part[c];
    free(part);
    return s;
}

int or_pcg(const or_csr* A, double cm, double ck, const double* b, double* x,
           double tol, int maxit, double* relres_out) {
    const int64_t n = A->n;
    double* r = malloc(sizeof(double) * (size_t)n);
    double* z = malloc(sizeof(double) * (size_t)n);
    double* p = malloc(sizeof(double) * (size_t)n);
    double* q = malloc(sizeof(double) * (size_t)n);
    double* dinv = malloc(sizeof(double) * (size_t)n);
    for (int64_t i = 0; i < n; ++i) {
        double d = 0.0;
        for (int64_t k = A->rowptr[i]; k < A->rowptr[i + 1]; ++k)
            if (A->col[k] == i) d = cm * A->mval[k] + ck * A->kval[k];
        dinv[i] = 1.0 / d;
    }
    or_csr_apply(A, cm, ck, x, q);
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < n; ++i) {
        r[i] = b[i] - q[i];
        z[i] = dinv[i] * r[i];
        p[i] = z[i];
    }
    const double bnorm = sqrt(dot(n, b, b));
    if (bnorm == 0.0) {
        /* A is SPD, so b = 0 has the unique solution x = 0 */
        for (int64_t i = 0; i < n; ++i) x[i] = 0.0;
        if (relres_out) *relres_out = 0.0;
        free(r); free(z); free(p); free(q); free(dinv);
        return 0;
    }
    double rz = dot(n, r, z);
    double rnorm = sqrt(dot(n, r, r));
    int it = 0;
    while (!(rnorm <= tol * bnorm)) {
        if (it >= maxit) { it = -1; break; }
        or_csr_apply(A, cm, ck, p, q);
        const double alpha = rz / dot(n, p, q);
#pragma omp parallel for schedule(static)
        for (int64_t i = 0; i < n; ++i) {
            x[i] += alpha * p[i];
            r[i] -= alpha * q[i];
            z[i] = dinv[i] * r[i];
        }
        const double rz_new = dot(n, r, z);
        const double beta = rz_new / rz;
        rz = rz_new;
#pragma omp parallel for schedule(static)
        for (int64_t i = 0; i < n; ++i) p[i] = z[i] + beta * p[i];
        rnorm = sqrt(dot(n, r, r));
        ++it;
    }
    if (relres_out) *relres_out = bnorm > 0.0 ? rnorm / bnorm : rnorm;
    free(r); free(z); free(p); free(q); free(dinv);
    return it;
}
