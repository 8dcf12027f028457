/*
 * Plain FP64 CPU oracle of the discrete elastic operator A_h = B_h C_h B_h^H
 * (test infrastructure only: tests, the smoke check and the CPU-baseline leg of
 * the bench may call it; the product library never does).
 *
 * It follows the paper's definitions term by term, on the full grid, with no
 * blocking, no compaction and no Fourier transform:
 *
 *   Sec. 3.1, Eqs. K_def / H_def: Bloch shift by +1 node along lattice axis l,
 *       with factor exp(i phi_l) when the index leaves the cell (phi_l = 2 pi kappa_l);
 *       node order l = i + n1 (j + n2 k).
 *   Eq. Sd_def: S_d1 = H3 H2 H1, S_d2 = H3^-1 H2 H1, S_d3 = H3 H2^-1 H1,
 *       S_d4 = H3^-1 H2^-1 H1, i.e. steps d = (1,1,1), (1,1,-1), (1,-1,1), (1,-1,-1).
 *   Eq. Dd_def: D_dl = (S_dl - I) / h_d,  h_d = sqrt(h1^2 + h2^2 + h3^2), h_s = 1/n_s.
 *   Eq. Dtilde_recon: Dt_s = h_d/(4 h_s) sum_l c_{s l} D_dl with
 *       c_1 = (1,1,1,1), c_2 = (1,1,-1,-1), c_3 = (1,-1,1,-1).
 *   Eqs. Dhat_def / Dcal_cartesian_transform: Dhat_s = -i Dt_s,
 *       Dcal_m = sum_s (A_lat^-1)_{s m} Dhat_s.
 *   Eq. B_discrete: B_h = [[D1,0,0,0,D3,D2],[0,D2,0,D3,0,D1],[0,0,D3,D2,D1,0]].
 *   Eq. discrete_GEP: A_h = B_h C_h B_h^H with C_h the nodewise 6x6 Voigt
 *       stiffness; M_h the nodewise density.
 *   Eq. subpixel_material_average: C_i = (1-theta_i) C^(1) + theta_i C^(2),
 *       rho_i = (1-theta_i) rho_1 + theta_i rho_2.
 *
 * The adjoint B_h^H uses S_d^H = S_d^-1 (a phased permutation is unitary):
 * (S_d^H w)(x) = w~(x - d), where w~ is the Bloch extension
 * w~(i + a n1, j + b n2, k + c n3) = exp(i (a phi1 + b phi2 + c phi3)) w(i, j, k).
 *
 * Vectors are complex, component-major: x[alpha * n + l] (Voigt vectors [v * n + l]).
 * Material tables: Ctab[2][36] row-major 6x6, rhotab[2], theta[n].
 * ainv[9] row-major: ainv[s*3 + m] = (A_lat^-1)_{s m}.
 */
#include <complex.h>
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

typedef double complex cplx;

/* Steps of the four body diagonals (Eq. Sd_def) and reconstruction signs (Eq. Dtilde_recon). */
static const int STEP[4][3] = {{1, 1, 1}, {1, 1, -1}, {1, -1, 1}, {1, -1, -1}};
static const double CSIGN[3][4] = {{1, 1, 1, 1}, {1, 1, -1, -1}, {1, -1, 1, -1}};
/* Placement of Dcal_m in B_h (Eq. B_discrete): BPAT[alpha][v] = m (0-based), or -1 for a zero block. */
static const int BPAT[3][6] = {{0, -1, -1, -1, 2, 1}, {-1, 1, -1, 2, -1, 0}, {-1, -1, 2, 1, 0, -1}};

typedef struct {
    int n[3];
    double h[3];
    double hd;
    double ainv[9];
    double phi[3];
} grid_t;

static void grid_init(grid_t* g, int n1, int n2, int n3, const double* ainv, const double* phi) {
    g->n[0] = n1; g->n[1] = n2; g->n[2] = n3;
    for (int s = 0; s < 3; ++s) g->h[s] = 1.0 / (double)g->n[s];
    g->hd = sqrt(g->h[0] * g->h[0] + g->h[1] * g->h[1] + g->h[2] * g->h[2]);
    memcpy(g->ainv, ainv, 9 * sizeof(double));
    memcpy(g->phi, phi, 3 * sizeof(double));
}

/* Bloch-extended value w~(c)(i, j, k) of a component-major field w (Sec. 3.1). */
static cplx bloch_read(const grid_t* g, const cplx* w, int comp, int i, int j, int k) {
    int idx[3] = {i, j, k};
    double ang = 0.0;
    for (int s = 0; s < 3; ++s) {
        int a = 0;
        while (idx[s] < 0) { idx[s] += g->n[s]; --a; }
        while (idx[s] >= g->n[s]) { idx[s] -= g->n[s]; ++a; }
        ang += a * g->phi[s];
    }
    int64_t n = (int64_t)g->n[0] * g->n[1] * g->n[2];
    int64_t l = idx[0] + (int64_t)g->n[0] * (idx[1] + (int64_t)g->n[1] * idx[2]);
    cplx v = w[(int64_t)comp * n + l];
    if (ang != 0.0) v *= cexp(I * ang);
    return v;
}

/* (Dcal_m^H w)(x) for m = 0..2 at node (i,j,k), component comp of w. */
static void dcal_adj_at(const grid_t* g, const cplx* w, int comp, int i, int j, int k, cplx out[3]) {
    cplx w0 = bloch_read(g, w, comp, i, j, k);
    cplx dd[4];
    for (int l = 0; l < 4; ++l) {
        /* D_dl^H w = (S_dl^H - I) w / h_d,   (S_dl^H w)(x) = w~(x - d_l) */
        cplx sh = bloch_read(g, w, comp, i - STEP[l][0], j - STEP[l][1], k - STEP[l][2]);
        dd[l] = (sh - w0) / g->hd;
    }
    cplx dt[3];
    for (int s = 0; s < 3; ++s) {
        cplx acc = 0.0;
        for (int l = 0; l < 4; ++l) acc += CSIGN[s][l] * dd[l];
        dt[s] = g->hd / (4.0 * g->h[s]) * acc; /* Dt_s^H w (real coefficients) */
    }
    for (int m = 0; m < 3; ++m) {
        cplx acc = 0.0;
        /* Dcal_m^H = sum_s (A^-1)_{s m} Dhat_s^H,  Dhat_s^H = (+i) Dt_s^H */
        for (int s = 0; s < 3; ++s) acc += g->ainv[s * 3 + m] * (I * dt[s]);
        out[m] = acc;
    }
}

/* (Dcal_m w)(x) for m = 0..2 at node (i,j,k), component comp of w. */
static void dcal_at(const grid_t* g, const cplx* w, int comp, int i, int j, int k, cplx out[3]) {
    cplx w0 = bloch_read(g, w, comp, i, j, k);
    cplx dd[4];
    for (int l = 0; l < 4; ++l) {
        cplx sh = bloch_read(g, w, comp, i + STEP[l][0], j + STEP[l][1], k + STEP[l][2]);
        dd[l] = (sh - w0) / g->hd; /* D_dl w */
    }
    cplx dt[3];
    for (int s = 0; s < 3; ++s) {
        cplx acc = 0.0;
        for (int l = 0; l < 4; ++l) acc += CSIGN[s][l] * dd[l];
        dt[s] = g->hd / (4.0 * g->h[s]) * acc; /* Dt_s w */
    }
    for (int m = 0; m < 3; ++m) {
        cplx acc = 0.0;
        for (int s = 0; s < 3; ++s) acc += g->ainv[s * 3 + m] * (-I * dt[s]); /* Dhat_s = -i Dt_s */
        out[m] = acc;
    }
}

/* Voigt strain e = (B_h^H x)(node): e_v = sum_alpha (Dcal_{BPAT[alpha][v]})^H x_alpha. */
static void strain_at(const grid_t* g, const cplx* x, int i, int j, int k, cplx e[6]) {
    cplx G[3][3]; /* G[alpha][m] = (Dcal_m^H x_alpha)(node) */
    for (int a = 0; a < 3; ++a) dcal_adj_at(g, x, a, i, j, k, G[a]);
    for (int v = 0; v < 6; ++v) {
        cplx acc = 0.0;
        for (int a = 0; a < 3; ++a)
            if (BPAT[a][v] >= 0) acc += G[a][BPAT[a][v]];
        e[v] = acc;
    }
}

static void node_material(const double* Ctab, const double* rhotab, const double* theta, int64_t l,
                          double C[36], double* rho) {
    double t = theta ? theta[l] : 0.0;
    for (int q = 0; q < 36; ++q) C[q] = (1.0 - t) * Ctab[q] + t * Ctab[36 + q];
    *rho = (1.0 - t) * rhotab[0] + t * rhotab[1];
}

static int64_t node_index(const grid_t* g, int i, int j, int k) {
    return i + (int64_t)g->n[0] * (j + (int64_t)g->n[1] * k);
}

/* e = B_h^H x over the whole grid: x[3n] -> e[6n]. */
int oracle_strain(int n1, int n2, int n3, const double* ainv, const double* phi,
                  const cplx* x, cplx* e, int nthreads) {
    grid_t g;
    grid_init(&g, n1, n2, n3, ainv, phi);
    int64_t n = (int64_t)n1 * n2 * n3;
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#pragma omp parallel for schedule(static)
#endif
    for (int k = 0; k < n3; ++k)
        for (int j = 0; j < n2; ++j)
            for (int i = 0; i < n1; ++i) {
                cplx ev[6];
                strain_at(&g, x, i, j, k, ev);
                int64_t l = node_index(&g, i, j, k);
                for (int v = 0; v < 6; ++v) e[v * n + l] = ev[v];
            }
    return 0;
}

/* y = B_h tau over the whole grid: tau[6n] -> y[3n]. */
int oracle_divergence(int n1, int n2, int n3, const double* ainv, const double* phi,
                      const cplx* tau, cplx* y, int nthreads) {
    grid_t g;
    grid_init(&g, n1, n2, n3, ainv, phi);
    int64_t n = (int64_t)n1 * n2 * n3;
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#pragma omp parallel for schedule(static)
#endif
    for (int k = 0; k < n3; ++k)
        for (int j = 0; j < n2; ++j)
            for (int i = 0; i < n1; ++i) {
                cplx D[6][3]; /* D[v][m] = (Dcal_m tau_v)(node) */
                for (int v = 0; v < 6; ++v) dcal_at(&g, tau, v, i, j, k, D[v]);
                int64_t l = node_index(&g, i, j, k);
                for (int a = 0; a < 3; ++a) {
                    cplx acc = 0.0;
                    for (int v = 0; v < 6; ++v)
                        if (BPAT[a][v] >= 0) acc += D[v][BPAT[a][v]];
                    y[a * n + l] = acc;
                }
            }
    return 0;
}

/* y = (A_h - shift M_h) x on the full grid (Eq. discrete_GEP), as strain -> C -> divergence. */
int oracle_apply_full(int n1, int n2, int n3, const double* ainv, const double* phi,
                      const double* Ctab, const double* rhotab, const double* theta,
                      const cplx* x, cplx* y, double shift, int nthreads) {
    int64_t n = (int64_t)n1 * n2 * n3;
    cplx* e = (cplx*)malloc(sizeof(cplx) * 6 * n);
    if (!e) return -2;
    oracle_strain(n1, n2, n3, ainv, phi, x, e, nthreads);
#ifdef _OPENMP
#pragma omp parallel for schedule(static)
#endif
    for (int64_t l = 0; l < n; ++l) {
        double C[36], rho;
        node_material(Ctab, rhotab, theta, l, C, &rho);
        cplx ev[6], tv[6];
        for (int v = 0; v < 6; ++v) ev[v] = e[v * n + l];
        for (int p = 0; p < 6; ++p) {
            cplx acc = 0.0;
            for (int q = 0; q < 6; ++q) acc += C[p * 6 + q] * ev[q];
            tv[p] = acc;
        }
        for (int v = 0; v < 6; ++v) e[v * n + l] = tv[v]; /* e now holds tau */
    }
    oracle_divergence(n1, n2, n3, ainv, phi, e, y, nthreads);
    free(e);
    if (shift != 0.0) {
#ifdef _OPENMP
#pragma omp parallel for schedule(static)
#endif
        for (int64_t l = 0; l < n; ++l) {
            double C[36], rho;
            node_material(Ctab, rhotab, theta, l, C, &rho);
            for (int a = 0; a < 3; ++a) y[a * n + l] -= shift * rho * x[a * n + l];
        }
    }
    return 0;
}

/* Bloch-extended stress tau~ = C (B^H x)~ at one node given by any integer coordinates:
 * strain_at reads x through its Bloch extension, and C is periodic (taken at the wrapped node). */
static void stress_at(const grid_t* g, const double* Ctab, const double* theta, const cplx* x,
                      int i, int j, int k, cplx tv[6]) {
    cplx ev[6];
    strain_at(g, x, i, j, k, ev);
    int idx[3] = {i, j, k};
    for (int s = 0; s < 3; ++s) {
        while (idx[s] < 0) idx[s] += g->n[s];
        while (idx[s] >= g->n[s]) idx[s] -= g->n[s];
    }
    int64_t l = node_index(g, idx[0], idx[1], idx[2]);
    double C[36], rho;
    double rhotab_dummy[2] = {0.0, 0.0};
    node_material(Ctab, rhotab_dummy, theta, l, C, &rho);
    for (int p = 0; p < 6; ++p) {
        cplx acc = 0.0;
        for (int q = 0; q < 6; ++q) acc += C[p * 6 + q] * ev[q];
        tv[p] = acc;
    }
}

/* y = (A_h - shift M_h) x evaluated only at the listed full-grid nodes: out[c*3 + alpha]. */
int oracle_apply_nodes(int n1, int n2, int n3, const double* ainv, const double* phi,
                       const double* Ctab, const double* rhotab, const double* theta,
                       const cplx* x, const int64_t* nodes, int64_t count, cplx* out,
                       double shift, int nthreads) {
    grid_t g;
    grid_init(&g, n1, n2, n3, ainv, phi);
    int64_t n = (int64_t)n1 * n2 * n3;
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#pragma omp parallel for schedule(dynamic, 16)
#endif
    for (int64_t c = 0; c < count; ++c) {
        int64_t l = nodes[c];
        int i = (int)(l % n1), j = (int)((l / n1) % n2), k = (int)(l / ((int64_t)n1 * n2));
        /* stress at the node and at its four forward diagonal neighbours */
        cplx t0[6], tl[4][6];
        stress_at(&g, Ctab, theta, x, i, j, k, t0);
        for (int q = 0; q < 4; ++q) {
            int ii = i + STEP[q][0], jj = j + STEP[q][1], kk = k + STEP[q][2];
            /* strain_at reads Bloch-extended values, so this is already tau~(x + d_q) */
            stress_at(&g, Ctab, theta, x, ii, jj, kk, tl[q]);
        }
        /* (Dcal_m tau_v)(node) from the forward differences, then B_h */
        for (int a = 0; a < 3; ++a) {
            cplx acc = 0.0;
            for (int v = 0; v < 6; ++v) {
                int m = BPAT[a][v];
                if (m < 0) continue;
                cplx dt[3];
                for (int s = 0; s < 3; ++s) {
                    cplx sum = 0.0;
                    for (int q = 0; q < 4; ++q) sum += CSIGN[s][q] * (tl[q][v] - t0[v]) / g.hd;
                    dt[s] = g.hd / (4.0 * g.h[s]) * sum;
                }
                for (int s = 0; s < 3; ++s) acc += g.ainv[s * 3 + m] * (-I * dt[s]);
            }
            double Cd[36], rho;
            node_material(Ctab, rhotab, theta, l, Cd, &rho);
            out[c * 3 + a] = acc - shift * rho * x[a * n + l];
        }
    }
    return 0;
}
