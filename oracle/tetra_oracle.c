/*
 * FP64 CPU oracle for the linear tetrahedron method of the orbital-resolved
 * density of states (Guterding & Jeschke, arXiv:1710.10789).
 *
 * TEST INFRASTRUCTURE ONLY. This file is the slow, plain reference that the
 * CUDA path is checked against. Only tests/, __graft_entry__.smoke() and the
 * cpu_baseline leg of bench.py may load or run it. It shares no code with the
 * CUDA library and must never be called from the product path.
 *
 * Conventions (each is a reading of the paper where the text is silent or
 * ambiguous):
 *  - k-grid: periodic, Gamma-centred, n1 x n2 x n3 points, flat index
 *    k = x + n1*(y + n2*z). Every point is the origin corner of one
 *    elemental cube, so there are n1*n2*n3 cubes and 6*n1*n2*n3 tetrahedra.
 *  - Cube corner label c (1..8) sits at offset (dx,dy,dz) with
 *    c = 1 + dx + 2*dy + 4*dz (Fig. 2 is not reproduced in the text; with this
 *    labelling the six tetrahedra of Table I tile the cube around the 3-6
 *    diagonal).
 *  - V_T / V_G = 1 / (6*n1*n2*n3); every corner weight saturates at
 *    f = V_T / (4 V_G).
 *  - Energy regions (Sec. II.C) are taken half-open: E <= E1 -> 0;
 *    E >= E4 -> saturated; E1 < E <= E2 region 1; E2 < E <= E3 region 2;
 *    E3 < E < E4 region 3.
 *  - In region 2 the last term of dw3/dE is (C2 + C3)/E32: the printed
 *    (C1 + C3)/E32 is not the derivative of the printed w3.
 *  - Array layouts of this file: eps[k*nb + n], wts[(k*nb + n)*norb + s],
 *    dos[s*npts + i].
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* Table I: corner labels of the six tetrahedra of an elemental cube. */
static const int TABLE_I[6][4] = {
    {1, 2, 3, 6}, {2, 3, 4, 6}, {1, 3, 5, 6}, {3, 4, 6, 8}, {3, 5, 6, 7}, {3, 6, 7, 8}};

/* The table above, row by row (24 labels), so tests can compare it with the
 * printed Table I. */
void oracle_table_i(int out[24]) {
    int t, q;
    for (t = 0; t < 6; ++t)
        for (q = 0; q < 4; ++q) out[4 * t + q] = TABLE_I[t][q];
}

/*
 * Corner weights w_j(E) and their energy derivatives dw_j/dE for one
 * tetrahedron with sorted corner energies e[0] <= e[1] <= e[2] <= e[3]
 * (Sec. II.C, the five energy cases). f = V_T / (4 V_G).
 * Outputs are indexed by sorted corner (j = 1..4 -> 0..3).
 */
void oracle_corner_weights(const double e[4], double E, double f, double w[4], double dw[4]) {
    const double E1 = e[0], E2 = e[1], E3 = e[2], E4 = e[3];
    int j;
    if (E <= E1) { /* case E <= E1: no contribution */
        for (j = 0; j < 4; ++j) { w[j] = 0.0; dw[j] = 0.0; }
        return;
    }
    if (E >= E4) { /* case E4 < E: saturated weights */
        for (j = 0; j < 4; ++j) { w[j] = f; dw[j] = 0.0; }
        return;
    }
    if (E <= E2) { /* case E1 < E < E2 */
        const double E21 = E2 - E1, E31 = E3 - E1, E41 = E4 - E1;
        const double x = E - E1;
        const double C = f * x * x * x / (E21 * E31 * E41);
        const double dC = 3.0 * f * x * x / (E21 * E31 * E41);
        const double S = 1.0 / E21 + 1.0 / E31 + 1.0 / E41;
        const double Ej1[3] = {E21, E31, E41};
        w[0] = C * (4.0 - x * S);
        dw[0] = dC * (4.0 - x * S) - C * S;
        for (j = 1; j < 4; ++j) {
            w[j] = C * x / Ej1[j - 1];
            dw[j] = dC * x / Ej1[j - 1] + C / Ej1[j - 1];
        }
        return;
    }
    if (E <= E3) { /* case E2 < E < E3 */
        const double E31 = E3 - E1, E41 = E4 - E1, E32 = E3 - E2, E42 = E4 - E2;
        const double C1 = f * (E - E1) * (E - E1) / (E31 * E41);
        const double dC1 = 2.0 * f * (E - E1) / (E31 * E41);
        const double C2 = f * (E - E1) * (E - E2) * (E3 - E) / (E31 * E32 * E41);
        const double dC2 = f / (E31 * E32 * E41) *
                           ((E - E1) * (E2 - E) + (E - E1) * (E3 - E) + (E - E2) * (E3 - E));
        const double C3 = f * (E - E2) * (E - E2) * (E4 - E) / (E32 * E41 * E42);
        const double dC3 = f * (E - E2) / (E32 * E41 * E42) * (2.0 * (E4 - E) + (E2 - E));
        w[0] = C1 + (C1 + C2) * (E3 - E) / E31 + (C1 + C2 + C3) * (E4 - E) / E41;
        dw[0] = dC1 + (dC1 + dC2) * (E3 - E) / E31 - (C1 + C2) / E31 +
                (dC1 + dC2 + dC3) * (E4 - E) / E41 - (C1 + C2 + C3) / E41;
        w[1] = C1 + C2 + C3 + (C2 + C3) * (E3 - E) / E32 + C3 * (E4 - E) / E42;
        dw[1] = dC1 + dC2 + dC3 + (dC2 + dC3) * (E3 - E) / E32 - (C2 + C3) / E32 +
                dC3 * (E4 - E) / E42 - C3 / E42;
        w[2] = (C1 + C2) * (E - E1) / E31 + (C2 + C3) * (E - E2) / E32;
        dw[2] = (dC1 + dC2) * (E - E1) / E31 + (C1 + C2) / E31 +
                (dC2 + dC3) * (E - E2) / E32 + (C2 + C3) / E32;
        w[3] = (C1 + C2 + C3) * (E - E1) / E41 + C3 * (E - E2) / E42;
        dw[3] = (dC1 + dC2 + dC3) * (E - E1) / E41 + (C1 + C2 + C3) / E41 +
                dC3 * (E - E2) / E42 + C3 / E42;
        return;
    }
    { /* case E3 < E < E4 */
        const double E41 = E4 - E1, E42 = E4 - E2, E43 = E4 - E3;
        const double y = E4 - E;
        const double C = f * y * y * y / (E41 * E42 * E43);
        const double dC = -3.0 * f * y * y / (E41 * E42 * E43);
        const double S = 1.0 / E41 + 1.0 / E42 + 1.0 / E43;
        const double E4j[3] = {E41, E42, E43};
        for (j = 0; j < 3; ++j) {
            w[j] = f - C * y / E4j[j];
            dw[j] = -dC * y / E4j[j] + C / E4j[j];
        }
        w[3] = f - C * (4.0 - S * y);
        dw[3] = -dC * (4.0 - S * y) - C * S;
    }
}

/* ---- geometry helpers for the energy-gradient moments ------------------ */

static void bary_on_edge(const double e[4], int a, int b, double E, double lam[4]) {
    const double t = (E - e[a]) / (e[b] - e[a]);
    int i;
    for (i = 0; i < 4; ++i) lam[i] = 0.0;
    lam[a] = 1.0 - t;
    lam[b] = t;
}

/* Triangle with barycentric vertices A, B, C (4-vectors). Adds
 * area * <lam_l lam_i> to acc[l][i], using edge-midpoint quadrature, which is
 * exact for quadratics. Positions use (lam1, lam2, lam3) as coordinates. */
static void tri_moments(const double A[4], const double B[4], const double C[4], double acc[4][4]) {
    double u[3], v[3], cr[3], area, m[3][4];
    int i, l, q;
    for (i = 0; i < 3; ++i) { u[i] = B[i] - A[i]; v[i] = C[i] - A[i]; }
    cr[0] = u[1] * v[2] - u[2] * v[1];
    cr[1] = u[2] * v[0] - u[0] * v[2];
    cr[2] = u[0] * v[1] - u[1] * v[0];
    area = 0.5 * sqrt(cr[0] * cr[0] + cr[1] * cr[1] + cr[2] * cr[2]);
    for (i = 0; i < 4; ++i) {
        m[0][i] = 0.5 * (A[i] + B[i]);
        m[1][i] = 0.5 * (B[i] + C[i]);
        m[2][i] = 0.5 * (C[i] + A[i]);
    }
    for (l = 0; l < 4; ++l)
        for (i = 0; i < 4; ++i) {
            double s = 0.0;
            for (q = 0; q < 3; ++q) s += m[q][l] * m[q][i];
            acc[l][i] += area * s / 3.0;
        }
}

/*
 * Energy-gradient moments of the corner weights. Writing the corner weight as
 * w_l(E) = (1/V_G) * integral over the tetrahedron of lam_l * Theta(E - eps),
 * with eps linear in the barycentric coordinates lam, gives
 *   d w_l / d e_i = -(1/V_G) * integral of lam_l lam_i delta(E - eps)
 *                 = -24 f * [ integral over the iso-energy cross-section of
 *                             lam_l lam_i dA ] / |grad eps|
 * in barycentric space (dk = 6 V_T dlam). M[l][i] receives the positive
 * moment, so d w_l / d e_i = -M[l][i]. Sorted energies, sorted indices.
 */
void oracle_weight_moments(const double e[4], double E, double f, double M[4][4]) {
    double acc[4][4], g[3], gn;
    int l, i;
    for (l = 0; l < 4; ++l)
        for (i = 0; i < 4; ++i) { M[l][i] = 0.0; acc[l][i] = 0.0; }
    if (E <= e[0] || E >= e[3]) return;
    if (E <= e[1]) { /* triangle on edges 1-2, 1-3, 1-4 */
        double P[3][4];
        bary_on_edge(e, 0, 1, E, P[0]);
        bary_on_edge(e, 0, 2, E, P[1]);
        bary_on_edge(e, 0, 3, E, P[2]);
        tri_moments(P[0], P[1], P[2], acc);
    } else if (E <= e[2]) { /* quadrilateral on edges 1-3, 1-4, 2-4, 2-3 */
        double P[4][4];
        bary_on_edge(e, 0, 2, E, P[0]);
        bary_on_edge(e, 0, 3, E, P[1]);
        bary_on_edge(e, 1, 3, E, P[2]);
        bary_on_edge(e, 1, 2, E, P[3]);
        tri_moments(P[0], P[1], P[2], acc);
        tri_moments(P[0], P[2], P[3], acc);
    } else { /* triangle on edges 1-4, 2-4, 3-4 */
        double P[3][4];
        bary_on_edge(e, 0, 3, E, P[0]);
        bary_on_edge(e, 1, 3, E, P[1]);
        bary_on_edge(e, 2, 3, E, P[2]);
        tri_moments(P[0], P[1], P[2], acc);
    }
    g[0] = e[0] - e[3];
    g[1] = e[1] - e[3];
    g[2] = e[2] - e[3];
    gn = sqrt(g[0] * g[0] + g[1] * g[1] + g[2] * g[2]);
    for (l = 0; l < 4; ++l)
        for (i = 0; i < 4; ++i) M[l][i] = 24.0 * f * acc[l][i] / gn;
}

/* ---- per-tetrahedron gathering ------------------------------------------- */

/* Flat grid indices of the four corners of tetrahedron t in cube (x,y,z),
 * in Table I order. */
static void tetra_corners(int n1, int n2, int n3, int x, int y, int z, int t, long kk[4]) {
    int q;
    for (q = 0; q < 4; ++q) {
        const int c = TABLE_I[t][q] - 1;
        const int dx = c & 1, dy = (c >> 1) & 1, dz = (c >> 2) & 1;
        const int xx = (x + dx) % n1, yy = (y + dy) % n2, zz = (z + dz) % n3;
        kk[q] = (long)xx + (long)n1 * ((long)yy + (long)n2 * (long)zz);
    }
}

/* Sort the four corner energies ascending, carrying the corner position.
 * Insertion sort with strict comparison: equal energies keep Table I order. */
static void sort4(double e[4], int pos[4]) {
    int i, j;
    for (i = 1; i < 4; ++i) {
        const double ve = e[i];
        const int vp = pos[i];
        j = i - 1;
        while (j >= 0 && e[j] > ve) {
            e[j + 1] = e[j];
            pos[j + 1] = pos[j];
            --j;
        }
        e[j + 1] = ve;
        pos[j + 1] = vp;
    }
}

/*
 * Orbital-resolved DOS, Eqs. (8)-(9).
 * mode 0 (point): dos[s*npts+i] = sum_{tetra,n} sum_l b_{n,l,s} dw_l/dE at E = ea[i].
 * mode 1 (bin):   dos[s*npts+i] = sum_{tetra,n} sum_l b_{n,l,s}
 *                                 [w_l(eb[i]) - w_l(ea[i])] / (eb[i] - ea[i]).
 * mode 2 (integrated): dos[s*npts+i] = sum_{tetra,n} sum_l b_{n,l,s} w_l(ea[i]),
 *                 the orbital occupation up to E (Eq. (2) with the step
 *                 function as occupation, evaluated by the corner weights of
 *                 Sec. II.C).
 * The energies ea/eb may be any list (a sample of a grid is fine).
 * Cubes with z in [z0, z1) only (the whole grid for z0=0, z1=n3).
 * nthreads > 1 splits the cube planes into contiguous blocks and adds the
 * per-thread results in thread order.
 */
int oracle_dos_range(int n1, int n2, int n3, int nb, int norb, const double *eps,
                     const double *wts, int mode, int npts, const double *ea,
                     const double *eb, int z0, int z1, double *dos, int nthreads) {
    const double f = 1.0 / (24.0 * (double)n1 * (double)n2 * (double)n3);
    const long out_n = (long)norb * npts;
    double *part;
    int th;
    if (n1 <= 0 || n2 <= 0 || n3 <= 0 || nb <= 0 || norb <= 0 || npts < 0) return 1;
    if (z0 < 0 || z1 > n3 || z0 > z1) return 1;
    if (nthreads < 1) nthreads = 1;
    part = (double *)calloc((size_t)nthreads * (size_t)(out_n > 0 ? out_n : 1), sizeof(double));
    if (!part) return 2;
#ifdef _OPENMP
#pragma omp parallel num_threads(nthreads)
#endif
    {
        int tid = 0, nth = 1;
        int zlo, zhi, x, y, z, t, n, q, i, s;
#ifdef _OPENMP
        tid = omp_get_thread_num();
        nth = omp_get_num_threads();
#endif
        {
            const int span = z1 - z0;
            zlo = z0 + (int)((long)span * tid / nth);
            zhi = z0 + (int)((long)span * (tid + 1) / nth);
        }
        double *acc = part + (long)tid * out_n;
        for (z = zlo; z < zhi; ++z)
            for (y = 0; y < n2; ++y)
                for (x = 0; x < n1; ++x)
                    for (t = 0; t < 6; ++t) {
                        long kk[4];
                        tetra_corners(n1, n2, n3, x, y, z, t, kk);
                        for (n = 0; n < nb; ++n) {
                            double e[4], w[4], dw[4], w2[4], dw2[4];
                            int pos[4];
                            for (q = 0; q < 4; ++q) { e[q] = eps[kk[q] * nb + n]; pos[q] = q; }
                            sort4(e, pos);
                            for (i = 0; i < npts; ++i) {
                                double c[4];
                                if (mode == 0) {
                                    oracle_corner_weights(e, ea[i], f, w, dw);
                                    for (q = 0; q < 4; ++q) c[q] = dw[q];
                                } else if (mode == 2) {
                                    oracle_corner_weights(e, ea[i], f, w, dw);
                                    for (q = 0; q < 4; ++q) c[q] = w[q];
                                } else {
                                    oracle_corner_weights(e, ea[i], f, w, dw);
                                    oracle_corner_weights(e, eb[i], f, w2, dw2);
                                    for (q = 0; q < 4; ++q) c[q] = (w2[q] - w[q]) / (eb[i] - ea[i]);
                                }
                                if (c[0] == 0.0 && c[1] == 0.0 && c[2] == 0.0 && c[3] == 0.0) continue;
                                for (s = 0; s < norb; ++s) {
                                    double v = 0.0;
                                    for (q = 0; q < 4; ++q)
                                        v += wts[(kk[pos[q]] * nb + n) * norb + s] * c[q];
                                    acc[(long)s * npts + i] += v;
                                }
                            }
                        }
                    }
    }
    for (long o = 0; o < out_n; ++o) {
        double v = 0.0;
        for (th = 0; th < nthreads; ++th) v += part[(long)th * out_n + o];
        dos[o] = v;
    }
    free(part);
    return 0;
}

int oracle_dos(int n1, int n2, int n3, int nb, int norb, const double *eps, const double *wts,
               int mode, int npts, const double *ea, const double *eb, double *dos, int nthreads) {
    return oracle_dos_range(n1, n2, n3, nb, norb, eps, wts, mode, npts, ea, eb, 0, n3, dos,
                            nthreads);
}

/*
 * Gradient of L = sum_{s,i} g[s*nbins+i] * DOS_s[i] (bin mode) with respect to
 * the band energies and the orbital weights at every grid point.
 *   dL/db_{n,s}(k)  = sum over tetrahedra with corner k: sum_i g_si dW_l(k)/dE_i
 *   dL/de_n(k)      = - sum over tetrahedra with corner k: sum_i sum_s g_si
 *                       sum_r b_{n,r,s} [M_{r,l(k)}(eb_i) - M_{r,l(k)}(ea_i)] / width_i
 * where dW is the bin-averaged weight and M the moments above. Overwrites
 * geps[k*nb+n] and gw[(k*nb+n)*norb+s]. Single-threaded.
 */
int oracle_dos_bin_grad(int n1, int n2, int n3, int nb, int norb, const double *eps,
                        const double *wts, int nbins, const double *ea, const double *eb,
                        const double *g, double *geps, double *gw) {
    const double f = 1.0 / (24.0 * (double)n1 * (double)n2 * (double)n3);
    const long nk = (long)n1 * n2 * n3;
    int x, y, z, t, n, q, r, i, s;
    if (n1 <= 0 || n2 <= 0 || n3 <= 0 || nb <= 0 || norb <= 0 || nbins < 0) return 1;
    memset(geps, 0, sizeof(double) * (size_t)(nk * nb));
    memset(gw, 0, sizeof(double) * (size_t)(nk * nb * norb));
    for (z = 0; z < n3; ++z)
        for (y = 0; y < n2; ++y)
            for (x = 0; x < n1; ++x)
                for (t = 0; t < 6; ++t) {
                    long kk[4];
                    tetra_corners(n1, n2, n3, x, y, z, t, kk);
                    for (n = 0; n < nb; ++n) {
                        double e[4];
                        int pos[4];
                        for (q = 0; q < 4; ++q) { e[q] = eps[kk[q] * nb + n]; pos[q] = q; }
                        sort4(e, pos);
                        for (i = 0; i < nbins; ++i) {
                            double wa[4], wb[4], d1[4], d2[4], Ma[4][4], Mb[4][4];
                            const double width = eb[i] - ea[i];
                            oracle_corner_weights(e, ea[i], f, wa, d1);
                            oracle_corner_weights(e, eb[i], f, wb, d2);
                            oracle_weight_moments(e, ea[i], f, Ma);
                            oracle_weight_moments(e, eb[i], f, Mb);
                            for (r = 0; r < 4; ++r) {
                                const long kr = kk[pos[r]];
                                const double dW = (wb[r] - wa[r]) / width;
                                for (s = 0; s < norb; ++s)
                                    gw[(kr * nb + n) * norb + s] += g[(long)s * nbins + i] * dW;
                            }
                            for (q = 0; q < 4; ++q) { /* sorted corner whose energy moves */
                                double acc = 0.0;
                                for (s = 0; s < norb; ++s) {
                                    double v = 0.0;
                                    for (r = 0; r < 4; ++r)
                                        v += wts[(kk[pos[r]] * nb + n) * norb + s] *
                                             (Mb[r][q] - Ma[r][q]);
                                    acc += g[(long)s * nbins + i] * v;
                                }
                                geps[kk[pos[q]] * nb + n] -= acc / width;
                            }
                        }
                    }
                }
    return 0;
}

/* ---- bare susceptibility at T = 0: double-band tetrahedron clipping ------
 *
 * The spectral part of the bare (Lindhard) susceptibility with step
 * occupations (T = 0), the extension to susceptibilities the paper names as
 * its method's next use (abstract, Conclusions):
 *   S(q, w) = sum_{n,m} (1/V_G) int dk [Theta(mu - e_n(k)) - Theta(mu - e_m(k+q))]
 *                                  delta(w - (e_m(k+q) - e_n(k))),
 * Im chi0(q, w + i0) = -pi S(q, w). With the method's linear interpolation
 * inside every tetrahedron, a = e_n - mu, c = e_m(k+q) - mu and the transition
 * energy D = c - a are linear there. The occupation difference is +1 on
 * {a < 0, c > 0}, -1 on {a > 0, c < 0} and 0 elsewhere, so each tetrahedron
 * contributes the distribution of D over two convex regions, each the
 * tetrahedron clipped by two planes. The regions are cut into
 * sub-tetrahedra; over a sub-tetrahedron of volume fraction nu, D is linear
 * and its distribution is nu * g(w) with g the normalised single-tetrahedron
 * density of a linear function (the total DOS of Sec. II.C's weights divided
 * by V_T / V_G).
 */

/* A point of the parent tetrahedron: barycentric coordinates and the two
 * linear fields. */
typedef struct {
    double l[4];
    double a, c;
} t0_point;

static void t0_lerp(const t0_point *u, const t0_point *v, double t, t0_point *out) {
    int i;
    for (i = 0; i < 4; ++i) out->l[i] = u->l[i] + t * (v->l[i] - u->l[i]);
    out->a = u->a + t * (v->a - u->a);
    out->c = u->c + t * (v->c - u->c);
}

/* Field to clip by: field 0 -> s = a, field 1 -> s = -a, 2 -> c, 3 -> -c.
 * The kept side is s < 0. */
static double t0_field(const t0_point *p, int which) {
    switch (which) {
        case 0: return p->a;
        case 1: return -p->a;
        case 2: return p->c;
        default: return -p->c;
    }
}

/* Clips tetrahedron T (4 points) to {s < 0}; writes up to 3 tetrahedra that
 * tile the kept part into out[], returns their number. */
static int t0_clip(const t0_point T[4], int which, t0_point out[3][4]) {
    int in[4], outv[4], ni = 0, no = 0, q;
    double s[4];
    for (q = 0; q < 4; ++q) {
        s[q] = t0_field(&T[q], which);
        if (s[q] < 0.0) in[ni++] = q;
        else outv[no++] = q;
    }
    if (ni == 0) return 0;
    if (ni == 4) {
        for (q = 0; q < 4; ++q) out[0][q] = T[q];
        return 1;
    }
#define T0_CUT(u, v, dst) t0_lerp(&T[u], &T[v], s[u] / (s[u] - s[v]), &(dst))
    if (ni == 1) { /* corner tetrahedron at the one kept vertex */
        const int i = in[0];
        out[0][0] = T[i];
        T0_CUT(i, outv[0], out[0][1]);
        T0_CUT(i, outv[1], out[0][2]);
        T0_CUT(i, outv[2], out[0][3]);
        return 1;
    }
    if (ni == 3) { /* prism: kept face I1 I2 I3, cut face P1 P2 P3, Pj on edge (o, Ij) */
        t0_point P[3];
        const int o = outv[0];
        for (q = 0; q < 3; ++q) T0_CUT(in[q], o, P[q]);
        out[0][0] = T[in[0]]; out[0][1] = T[in[1]]; out[0][2] = T[in[2]]; out[0][3] = P[0];
        out[1][0] = T[in[1]]; out[1][1] = T[in[2]]; out[1][2] = P[0]; out[1][3] = P[1];
        out[2][0] = T[in[2]]; out[2][1] = P[0]; out[2][2] = P[1]; out[2][3] = P[2];
        return 3;
    }
    { /* wedge: triangles (I1, P11, P12) and (I2, P21, P22), Pij on edge (Ii, Oj) */
        t0_point P11, P12, P21, P22;
        const int i1 = in[0], i2 = in[1], o1 = outv[0], o2 = outv[1];
        T0_CUT(i1, o1, P11);
        T0_CUT(i1, o2, P12);
        T0_CUT(i2, o1, P21);
        T0_CUT(i2, o2, P22);
        out[0][0] = T[i1]; out[0][1] = P11; out[0][2] = P12; out[0][3] = T[i2];
        out[1][0] = P11; out[1][1] = P12; out[1][2] = T[i2]; out[1][3] = P21;
        out[2][0] = P12; out[2][1] = T[i2]; out[2][2] = P21; out[2][3] = P22;
        return 3;
    }
#undef T0_CUT
}

/* Volume of a sub-tetrahedron as a fraction of its parent (barycentric). */
static double t0_volume(const t0_point P[4]) {
    double u[3][3];
    int i, j;
    for (i = 0; i < 3; ++i)
        for (j = 0; j < 3; ++j) u[i][j] = P[i].l[j] - P[3].l[j];
    return fabs(u[0][0] * (u[1][1] * u[2][2] - u[1][2] * u[2][1]) -
                u[0][1] * (u[1][0] * u[2][2] - u[1][2] * u[2][0]) +
                u[0][2] * (u[1][0] * u[2][1] - u[1][1] * u[2][0]));
}

/* Normalised density g(w) and cumulative G(w) of a linear function with the
 * given values at the corners of a tetrahedron (uniform measure). */
static void t0_density(const double d_in[4], double w, double *g, double *G) {
    double d[4];
    int i, j;
    for (i = 0; i < 4; ++i) d[i] = d_in[i];
    for (i = 1; i < 4; ++i) { /* insertion sort */
        const double v = d[i];
        j = i - 1;
        while (j >= 0 && d[j] > v) { d[j + 1] = d[j]; --j; }
        d[j + 1] = v;
    }
    if (w <= d[0]) { *g = 0.0; *G = 0.0; return; }
    if (w >= d[3]) { *g = 0.0; *G = 1.0; return; }
    {
        const double d21 = d[1] - d[0], d31 = d[2] - d[0], d41 = d[3] - d[0];
        const double d32 = d[2] - d[1], d42 = d[3] - d[1], d43 = d[3] - d[2];
        if (w <= d[1]) {
            const double x = w - d[0];
            *g = 3.0 * x * x / (d21 * d31 * d41);
            *G = x * x * x / (d21 * d31 * d41);
        } else if (w <= d[2]) {
            const double x = w - d[1];
            *g = 3.0 / (d31 * d41) * (d21 + 2.0 * x - (d31 + d42) * x * x / (d32 * d42));
            *G = (d21 * d21 + 3.0 * d21 * x + 3.0 * x * x - (d31 + d42) * x * x * x / (d32 * d42)) /
                 (d31 * d41);
        } else {
            const double y = d[3] - w;
            *g = 3.0 * y * y / (d41 * d42 * d43);
            *G = 1.0 - y * y * y / (d41 * d42 * d43);
        }
    }
}

/* ---- real part: principal-value average of 1/(w - D) over a tetrahedron --
 *
 * Re chi0(q, w) = sum_{n,m} (1/V_G) P int dk [f_n(k) - f_m(k+q)] / (w - D(k)),
 * D = e_m(k+q) - e_n(k), the Hilbert transform of S (chi0 = int S(w') /
 * (w - w' + i0) dw'). Over a sub-tetrahedron the average of 1/(w - D) is the
 * principal-value integral of the normalised density g of D against
 * 1/(w - x). g is a quadratic spline on the sorted corner values
 * d0 <= d1 <= d2 <= d3 (the density of t0_density); on its three pieces its
 * Bernstein coefficients are
 *   [d0, d1]: (0, 0, G1),  [d1, d2]: (G1, 3/d41, G2),  [d2, d3]: (G2, 0, 0),
 * G1 = 3 d21 / (d31 d41) = g(d1), G2 = 3 d43 / (d41 d42) = g(d2) (the middle
 * coefficient follows from g's slope at d1 or d2; all three pieces integrate
 * to d21 G1/3 + d32 (G1 + 3/d41 + G2)/3 + d43 G2/3 = 1).
 *
 * A piece [a, b], h = b - a, with coefficients (b0, b1, b2), p(t) = b0 (1-t)^2 +
 * 2 b1 t (1-t) + b2 t^2, gives int_0^1 p(t) / (s - t) dt with s = (w - a)/h:
 *  - far from the piece (|s - 1/2| >= 3/2) as the series
 *    sum_j m_j / (s - 1/2)^(j+1), m_j = int_0^1 p(t) (t - 1/2)^j dt, whose
 *    terms shrink by 1/3 or more (no cancellation, however thin the piece);
 *  - near it in closed form, with I0 = ln|s| - ln|s - 1| (the principal
 *    value inside the piece), int t/(s-t) = s I0 - 1, int t^2/(s-t) =
 *    s^2 I0 - s - 1/2:
 *      p(s) I0 + b0 (3/2 - s) + b1 (2s - 1) - b2 (s + 1/2),
 *    p(s) the piece's polynomial continued to t = s.
 * When w is exactly a knot the two pieces that meet there both drop their
 * ln|w - knot| term: its coefficients are g's values from both sides, equal
 * since g is continuous, so the terms cancel and only ln h remains.
 */
static double t0_piece_inverse(double b0, double b1, double b2, double a, double b, double w) {
    const double h = b - a, s = (w - a) / h, u = s - 0.5;
    if (fabs(u) >= 1.5) {
        /* p(t) = A + B tau + C tau^2 with tau = t - 1/2; the moments of tau
         * over [-1/2, 1/2] vanish for odd powers and are 2^-k/(k+1) for even k */
        const double A = 0.25 * (b0 + 2.0 * b1 + b2), B = b2 - b0, C = b0 - 2.0 * b1 + b2;
        double sum = 0.0, upow = 1.0 / u;
        int j;
        for (j = 0; j <= 60; ++j) {
            double mj = 0.0;
            int k;
            for (k = j; k <= j + 2; ++k) {
                const double coef = (k == j) ? A : ((k == j + 1) ? B : C);
                if (k % 2 == 0) mj += coef * ldexp(1.0, -k) / (double)(k + 1);
            }
            sum += mj * upow;
            upow /= u;
        }
        return sum;
    }
    {
        /* ln|s| = ln|w - a| - ln h and ln|s - 1| = ln|w - b| - ln h, taken from
         * the distances themselves (no cancellation near a knot) */
        const double lh = log(h);
        const double la = ((w == a) ? 0.0 : log(fabs(w - a))) - lh;
        const double lb = ((w == b) ? 0.0 : log(fabs(w - b))) - lh;
        const double ps = b0 * (1.0 - s) * (1.0 - s) + 2.0 * b1 * s * (1.0 - s) + b2 * s * s;
        return ps * (la - lb) + b0 * (1.5 - s) + b1 * (2.0 * s - 1.0) - b2 * (s + 0.5);
    }
}

/* P <1/(w - D)> over a tetrahedron on whose corners the linear function D
 * takes the values d_in[4] (uniform measure). A flat D (all values equal)
 * gives 1/(w - d), and 0 when w equals it. */
double oracle_t0_inverse_average(const double d_in[4], double w) {
    double d[4];
    int i, j;
    for (i = 0; i < 4; ++i) d[i] = d_in[i];
    for (i = 1; i < 4; ++i) {
        const double v = d[i];
        j = i - 1;
        while (j >= 0 && d[j] > v) { d[j + 1] = d[j]; --j; }
        d[j + 1] = v;
    }
    if (!(d[3] > d[0])) return (w == d[0]) ? 0.0 : 1.0 / (w - d[0]);
    {
        const double d21 = d[1] - d[0], d31 = d[2] - d[0], d41 = d[3] - d[0];
        const double d32 = d[2] - d[1], d42 = d[3] - d[1], d43 = d[3] - d[2];
        const double G1 = d31 > 0.0 ? 3.0 * d21 / (d31 * d41) : 0.0;
        const double G2 = d42 > 0.0 ? 3.0 * d43 / (d41 * d42) : 0.0;
        double r = 0.0;
        if (d21 > 0.0) r += t0_piece_inverse(0.0, 0.0, G1, d[0], d[1], w);
        if (d32 > 0.0) r += t0_piece_inverse(G1, 3.0 / d41, G2, d[1], d[2], w);
        if (d43 > 0.0) r += t0_piece_inverse(G2, 0.0, 0.0, d[2], d[3], w);
        return r;
    }
}

/*
 * Contribution of one tetrahedron (vertex values a[4] = e_n - mu,
 * c[4] = e_m(k+q) - mu) to the normalised spectral function, in units of
 * V_T / V_G: mode 0 (point) sum_regions sign * nu * g(ea[i]); mode 1 (bin)
 * sum_regions sign * nu * [G(eb[i]) - G(ea[i])] / (eb[i] - ea[i]); mode 2
 * (real part of chi0 at the points ea) sum_regions sign * nu *
 * P<1/(ea[i] - D)>. Adds to out[i], i < npts.
 */
void oracle_t0_tetra(const double a[4], const double c[4], int mode, int npts, const double *ea,
                     const double *eb, double *out) {
    t0_point T[4];
    int q, r;
    for (q = 0; q < 4; ++q) {
        int j;
        for (j = 0; j < 4; ++j) T[q].l[j] = (j == q) ? 1.0 : 0.0;
        T[q].a = a[q];
        T[q].c = c[q];
    }
    for (r = 0; r < 2; ++r) {
        /* r = 0: {a < 0, c > 0}, sign +1; r = 1: {a > 0, c < 0}, sign -1 */
        const double sign = r == 0 ? 1.0 : -1.0;
        t0_point A[3][4];
        const int na = t0_clip(T, r == 0 ? 0 : 1, A);
        int ia;
        for (ia = 0; ia < na; ++ia) {
            t0_point B[3][4];
            const int nbb = t0_clip(A[ia], r == 0 ? 3 : 2, B);
            int ib;
            for (ib = 0; ib < nbb; ++ib) {
                const double nu = t0_volume(B[ib]);
                double d[4];
                int i;
                if (nu <= 0.0) continue;
                for (q = 0; q < 4; ++q) d[q] = B[ib][q].c - B[ib][q].a;
                for (i = 0; i < npts; ++i) {
                    double g, G, gb, Gb;
                    if (mode == 2) {
                        out[i] += sign * nu * oracle_t0_inverse_average(d, ea[i]);
                        continue;
                    }
                    t0_density(d, ea[i], &g, &G);
                    if (mode == 0) {
                        out[i] += sign * nu * g;
                    } else {
                        t0_density(d, eb[i], &gb, &Gb);
                        out[i] += sign * nu * (Gb - G) / (eb[i] - ea[i]);
                    }
                }
            }
        }
    }
}

/*
 * T = 0 spectral function of the bare susceptibility on the grid, all band
 * pairs (n, m), cube planes [z0, z1):
 *   S[i] = (V_T/V_G) sum_{tetra, n, m} (oracle_t0_tetra of that tetrahedron),
 * V_T/V_G = 1/(6 n1 n2 n3). eps[k*nb + n] are the bands at k; epq, if not
 * NULL, the bands at k + q on the same flat index (epq[k*nb + m] = e_m(k+q));
 * if NULL they are taken from eps with the integer grid shift q (periodic).
 */
int oracle_t0_spectral(int n1, int n2, int n3, int nb, const double *eps, const double *epq,
                       const int q[3], double mu, int mode, int npts, const double *ea,
                       const double *eb, int z0, int z1, double *out, int nthreads) {
    const double vt = 1.0 / (6.0 * (double)n1 * (double)n2 * (double)n3);
    int i, th;
    double *part;
    if (n1 <= 0 || n2 <= 0 || n3 <= 0 || nb <= 0 || npts < 0 || z0 < 0 || z1 > n3 || z0 > z1) return 1;
    if (nthreads < 1) nthreads = 1;
    part = (double *)calloc((size_t)nthreads * (size_t)(npts > 0 ? npts : 1), sizeof(double));
    if (!part) return 2;
#ifdef _OPENMP
#pragma omp parallel num_threads(nthreads)
#endif
    {
        int tid = 0, nth = 1, x, y, z, t, n, m, v, zlo, zhi;
#ifdef _OPENMP
        tid = omp_get_thread_num();
        nth = omp_get_num_threads();
#endif
        zlo = z0 + (int)((long)(z1 - z0) * tid / nth);
        zhi = z0 + (int)((long)(z1 - z0) * (tid + 1) / nth);
        double *acc = part + (long)tid * (npts > 0 ? npts : 1);
        for (z = zlo; z < zhi; ++z)
            for (y = 0; y < n2; ++y)
                for (x = 0; x < n1; ++x)
                    for (t = 0; t < 6; ++t) {
                        long kk[4], kq[4];
                        tetra_corners(n1, n2, n3, x, y, z, t, kk);
                        for (v = 0; v < 4; ++v) {
                            const long k = kk[v];
                            const int kx = (int)(k % n1), ky = (int)((k / n1) % n2), kz = (int)(k / ((long)n1 * n2));
                            const int sx = ((kx + q[0]) % n1 + n1) % n1;
                            const int sy = ((ky + q[1]) % n2 + n2) % n2;
                            const int sz = ((kz + q[2]) % n3 + n3) % n3;
                            kq[v] = epq ? k : (long)sx + (long)n1 * ((long)sy + (long)n2 * sz);
                        }
                        for (n = 0; n < nb; ++n)
                            for (m = 0; m < nb; ++m) {
                                double a[4], c[4];
                                const double *src = epq ? epq : eps;
                                for (v = 0; v < 4; ++v) {
                                    a[v] = eps[kk[v] * nb + n] - mu;
                                    c[v] = src[kq[v] * nb + m] - mu;
                                }
                                oracle_t0_tetra(a, c, mode, npts, ea, eb, acc);
                            }
                    }
    }
    for (i = 0; i < npts; ++i) {
        double sum = 0.0;
        for (th = 0; th < nthreads; ++th) sum += part[(long)th * npts + i];
        out[i] = vt * sum;
    }
    free(part);
    return 0;
}
