/*
 * Oracle (test infrastructure only): plain FP64 CPU evaluation of the pieces of
 * the Galerkin single-layer operator that are O(N^2) or need closed-form
 * integrals.  The sparse factors Phi, W of Eq. (BEM) and the solves live in
 * oracle/__init__.py.  Only tests, the smoke check and the benchmark's CPU
 * baseline may load this library; the product path never does.
 *
 * Every loop follows the paper's statement directly: no blocking, no fusion.
 * OpenMP only splits independent target rows across threads.
 */
#include <math.h>
#include <stdint.h>
#include <stddef.h>
#include <stdlib.h>

#ifndef M_PI
#define M_PI 3.14159265358979323846
#endif

/* ------------------------------------------------------------------------ */
/* Quadrature on the reference triangle, Sec. 4.2 (dom(mesh, q)) and Eq.     */
/* (approxA): points in barycentric coordinates, weights summing to one,     */
/* scaled by the triangle area by the caller.                                */
/*   q = 1: centroid.                                                        */
/*   q = 3: interior points (2/3, 1/6, 1/6) and permutations, weight 1/3.    */
/*   q = 7: Radon's degree-5 rule (centroid, and two orbits a = (6 -+ s)/21, */
/*          s = sqrt(15), weights (155 -+ s)/1200).                          */
/* ------------------------------------------------------------------------ */
int or_quad_rule(int q, double *bary, double *w)
{
    if (q == 1) {
        bary[0] = bary[1] = bary[2] = 1.0 / 3.0;
        w[0] = 1.0;
        return 0;
    }
    if (q == 3) {
        for (int i = 0; i < 3; ++i) {
            for (int j = 0; j < 3; ++j) bary[3 * i + j] = (i == j) ? 2.0 / 3.0 : 1.0 / 6.0;
            w[i] = 1.0 / 3.0;
        }
        return 0;
    }
    if (q == 7) {
        double s = sqrt(15.0);
        double a1 = (6.0 - s) / 21.0, a2 = (6.0 + s) / 21.0;
        double w1 = (155.0 - s) / 1200.0, w2 = (155.0 + s) / 1200.0;
        bary[0] = bary[1] = bary[2] = 1.0 / 3.0;
        w[0] = 9.0 / 40.0;
        for (int i = 0; i < 3; ++i) {
            for (int j = 0; j < 3; ++j) {
                bary[3 * (1 + i) + j] = (i == j) ? 1.0 - 2.0 * a1 : a1;
                bary[3 * (4 + i) + j] = (i == j) ? 1.0 - 2.0 * a2 : a2;
            }
            w[1 + i] = w1;
            w[4 + i] = w2;
        }
        return 0;
    }
    return -1;
}

/* ------------------------------------------------------------------------ */
/* Helmholtz kernel between point clouds, Eq. (BEM) and Eq. (Helmholtz)      */
/* without the 1/(4 pi) factor (the paper applies it after the integral):    */
/*   G(x, y) = exp(i k |x - y|) / |x - y|.                                   */
/* Where target and source are the same quadrature point (tid == sid) the    */
/* kernel takes its smooth-part limit G := i k, i.e. the limit of            */
/* (exp(ikr) - 1)/r; the 1/r part of that pair is handled by the singular    */
/* correction of Sec. 5.2, which leaves that pair out of its Gauss sum.      */
/* ------------------------------------------------------------------------ */
static inline void helmholtz_g(const double *x, const double *y, double k, double *gr, double *gi)
{
    double dx = x[0] - y[0], dy = x[1] - y[1], dz = x[2] - y[2];
    double r = sqrt(dx * dx + dy * dy + dz * dz);
    *gr = cos(k * r) / r;
    *gi = sin(k * r) / r;
}

/*
 * v[t, j] = sum_l G(x_t, y_l) u[l, j]   (the dense product G (W_y Psi x)).
 *   xt  : nt x 3 target points, tid[t] their point ids (or NULL: none equal)
 *   ys  : ns x 3 source points, sources have ids 0..ns-1
 *   u   : complex (interleaved re, im) ns x nrhs, column-major (ld = ns)
 *   v   : complex nt x nrhs, column-major (ld = nt), overwritten
 */
int or_kernel_matvec(int64_t nt, const double *xt, const int64_t *tid,
                     int64_t ns, const double *ys, double k, int64_t nrhs,
                     const double *u, double *v)
{
    #pragma omp parallel
    {
        /* one kernel value per (t, l), used for every right-hand side; each
           column still sums over l in increasing order */
        double *acc = (double *)calloc((size_t)(2 * nrhs), sizeof(double));
        #pragma omp for schedule(dynamic, 16)
        for (int64_t t = 0; t < nt; ++t) {
            for (int64_t j = 0; j < 2 * nrhs; ++j) acc[j] = 0.0;
            for (int64_t l = 0; l < ns; ++l) {
                double gr, gi;
                if (tid != NULL && tid[t] == l) {
                    gr = 0.0;
                    gi = k;
                } else {
                    helmholtz_g(xt + 3 * t, ys + 3 * l, k, &gr, &gi);
                }
                for (int64_t j = 0; j < nrhs; ++j) {
                    double ur = u[2 * (j * ns + l)], ui = u[2 * (j * ns + l) + 1];
                    acc[2 * j] += gr * ur - gi * ui;
                    acc[2 * j + 1] += gr * ui + gi * ur;
                }
            }
            for (int64_t j = 0; j < nrhs; ++j) {
                v[2 * (j * nt + t)] = acc[2 * j];
                v[2 * (j * nt + t) + 1] = acc[2 * j + 1];
            }
        }
        free(acc);
    }
    return 0;
}

/* G as a dense complex nt x ns matrix, row-major, interleaved (re, im). */
int or_kernel_matrix(int64_t nt, const double *xt, const int64_t *tid,
                     int64_t ns, const double *ys, double k, double *g)
{
    #pragma omp parallel for schedule(static)
    for (int64_t t = 0; t < nt; ++t) {
        for (int64_t l = 0; l < ns; ++l) {
            double gr, gi;
            if (tid != NULL && tid[t] == l) {
                gr = 0.0;
                gi = k;
            } else {
                helmholtz_g(xt + 3 * t, ys + 3 * l, k, &gr, &gi);
            }
            g[2 * (t * ns + l)] = gr;
            g[2 * (t * ns + l) + 1] = gi;
        }
    }
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Closed-form integral of the P1 basis functions times 1/|x - y| over a     */
/* flat triangle T = (P0, P1, P2), for one observation point x (Sec. 5.2:    */
/* "the integral in y is computed analytically").                            */
/*                                                                           */
/* With n the unit normal, d = (x - P0).n, rho0 = x - d n and R = |x - y|:   */
/*   lambda_j(y) = lambda_j(rho0) + grad(lambda_j).(y - rho0)   on T,        */
/* so  I_j = lambda_j(rho0) * S + grad(lambda_j) . Vv  with                  */
/*   S  = int_T 1/R,   Vv = int_T (y - rho0)/R.                              */
/* Both come from the edge formulas of Wilton et al. (1984) and Graglia      */
/* (1993): for edge i with unit tangent t_i, in-plane outward normal         */
/* m_i = t_i x n, signed distance p_i = (P - rho0).m_i, end abscissae        */
/* l^-, l^+, end distances R^-, R^+, R0^2 = p_i^2 + d^2 and                  */
/* f_i = ln((R^+ + l^+)/(R^- + l^-)):                                        */
/*   S  = sum_i p_i f_i - |d| sum_i [atan(p_i l^+/(R0^2 + |d| R^+))          */
/*                                  - atan(p_i l^-/(R0^2 + |d| R^-))]        */
/*   Vv = 1/2 sum_i m_i [R0^2 f_i + l^+ R^+ - l^- R^-]   (Vv = int grad_y R).*/
/* R + l is evaluated as R0^2/(R - l) when l < 0 to avoid cancellation; the  */
/* log terms are dropped where R0^2 vanishes (x on an edge line), where      */
/* their prefactors p_i and R0^2 are zero.                                   */
/* ------------------------------------------------------------------------ */
static inline double dot3(const double *a, const double *b) { return a[0] * b[0] + a[1] * b[1] + a[2] * b[2]; }
static inline void cross3(const double *a, const double *b, double *c)
{
    c[0] = a[1] * b[2] - a[2] * b[1];
    c[1] = a[2] * b[0] - a[0] * b[2];
    c[2] = a[0] * b[1] - a[1] * b[0];
}

static double r_plus_l(double R, double l, double R02)
{
    return (l >= 0.0) ? R + l : R02 / (R - l);
}

void or_p1_inv_r(const double *x, const double *P0, const double *P1, const double *P2, double *out)
{
    const double *P[3] = {P0, P1, P2};
    double e1[3], e2[3], nn[3];
    for (int c = 0; c < 3; ++c) {
        e1[c] = P1[c] - P0[c];
        e2[c] = P2[c] - P0[c];
    }
    cross3(e1, e2, nn);
    double twoA = sqrt(dot3(nn, nn));
    double n[3] = {nn[0] / twoA, nn[1] / twoA, nn[2] / twoA};
    double xp0[3] = {x[0] - P0[0], x[1] - P0[1], x[2] - P0[2]};
    double d = dot3(xp0, n);
    double ad = fabs(d);
    double rho0[3] = {x[0] - d * n[0], x[1] - d * n[1], x[2] - d * n[2]};
    double scale2 = twoA; /* squared length scale of the triangle */

    double S = 0.0, Vv[3] = {0.0, 0.0, 0.0};
    for (int i = 0; i < 3; ++i) {
        const double *Pm = P[i], *Pp = P[(i + 1) % 3];
        double t[3] = {Pp[0] - Pm[0], Pp[1] - Pm[1], Pp[2] - Pm[2]};
        double len = sqrt(dot3(t, t));
        t[0] /= len; t[1] /= len; t[2] /= len;
        double m[3];
        cross3(t, n, m);
        double am[3] = {Pm[0] - rho0[0], Pm[1] - rho0[1], Pm[2] - rho0[2]};
        double ap[3] = {Pp[0] - rho0[0], Pp[1] - rho0[1], Pp[2] - rho0[2]};
        double lm = dot3(am, t), lp = dot3(ap, t);
        double p = dot3(am, m);
        double R02 = p * p + d * d;
        double xm[3] = {x[0] - Pm[0], x[1] - Pm[1], x[2] - Pm[2]};
        double xpp[3] = {x[0] - Pp[0], x[1] - Pp[1], x[2] - Pp[2]};
        double Rm = sqrt(dot3(xm, xm)), Rp = sqrt(dot3(xpp, xpp));
        double f = 0.0;
        if (R02 > 1e-30 * scale2) f = log(r_plus_l(Rp, lp, R02) / r_plus_l(Rm, lm, R02));
        S += p * f;
        if (ad > 0.0)
            S -= ad * (atan(p * lp / (R02 + ad * Rp)) - atan(p * lm / (R02 + ad * Rm)));
        double vc = 0.5 * (R02 * f + lp * Rp - lm * Rm);
        Vv[0] += m[0] * vc;
        Vv[1] += m[1] * vc;
        Vv[2] += m[2] * vc;
    }
    for (int j = 0; j < 3; ++j) {
        const double *A = P[(j + 1) % 3], *B = P[(j + 2) % 3];
        double ab[3] = {B[0] - A[0], B[1] - A[1], B[2] - A[2]};
        double g[3];
        cross3(n, ab, g); /* grad lambda_j = n x (P_{j+2} - P_{j+1}) / (2 area) */
        g[0] /= twoA; g[1] /= twoA; g[2] /= twoA;
        double rj[3] = {rho0[0] - P[j][0], rho0[1] - P[j][1], rho0[2] - P[j][2]};
        double lam0 = 1.0 + dot3(g, rj);
        out[j] = lam0 * S + dot3(g, Vv);
    }
}

/* ------------------------------------------------------------------------ */
/* Singular correction of Sec. 5.2 (regularize(S, S, Vh, '[1/r]', Vh)),      */
/* scaled by 1/(4 pi) as in the paper's listing of Sec. 5.4.  For each       */
/* ordered pair (a, b) of triangles that share at least one vertex, each     */
/* quadrature point x_k of a and each local vertex j of b:                   */
/*   exact_j = int_b lambda_j(y)/|x_k - y| dy          (closed form above)   */
/*   gauss_j = sum_{l in b, l != k} eta_l lambda_j(y_l)/|x_k - y_l|          */
/*   block[i][j] += w_k lambda_i(x_k) (exact_j - gauss_j) / (4 pi)           */
/* The l == k point exists only when a == b; it is the self pair whose      */
/* kernel value is i k in the dense part.                                    */
/*   vtx: nv x 3, tri: nt x 3 (int32), pa/pb: npairs ordered pairs           */
/*   blocks: npairs x 3 x 3 (row i: test vertex of a, column j: trial of b)  */
/* ------------------------------------------------------------------------ */
int or_near_blocks(const double *vtx, const int32_t *tri, int q,
                   int64_t npairs, const int64_t *pa, const int64_t *pb, double *blocks)
{
    double bary[21], wr[7];
    if (or_quad_rule(q, bary, wr) != 0) return -1;
    #pragma omp parallel for schedule(dynamic, 64)
    for (int64_t p = 0; p < npairs; ++p) {
        int64_t a = pa[p], b = pb[p];
        const double *A[3], *B[3];
        for (int m = 0; m < 3; ++m) {
            A[m] = vtx + 3 * (int64_t)tri[3 * a + m];
            B[m] = vtx + 3 * (int64_t)tri[3 * b + m];
        }
        double ea[3], fa[3], na[3], eb[3], fb[3], nb[3];
        for (int c = 0; c < 3; ++c) {
            ea[c] = A[1][c] - A[0][c]; fa[c] = A[2][c] - A[0][c];
            eb[c] = B[1][c] - B[0][c]; fb[c] = B[2][c] - B[0][c];
        }
        cross3(ea, fa, na);
        cross3(eb, fb, nb);
        double area_a = 0.5 * sqrt(dot3(na, na)), area_b = 0.5 * sqrt(dot3(nb, nb));
        double blk[9] = {0};
        for (int kq = 0; kq < q; ++kq) {
            double xk[3];
            for (int c = 0; c < 3; ++c)
                xk[c] = bary[3 * kq] * A[0][c] + bary[3 * kq + 1] * A[1][c] + bary[3 * kq + 2] * A[2][c];
            double wk = wr[kq] * area_a;
            double ex[3];
            or_p1_inv_r(xk, B[0], B[1], B[2], ex);
            double gs[3] = {0.0, 0.0, 0.0};
            for (int lq = 0; lq < q; ++lq) {
                if (a == b && lq == kq) continue;
                double yl[3];
                for (int c = 0; c < 3; ++c)
                    yl[c] = bary[3 * lq] * B[0][c] + bary[3 * lq + 1] * B[1][c] + bary[3 * lq + 2] * B[2][c];
                double dd[3] = {xk[0] - yl[0], xk[1] - yl[1], xk[2] - yl[2]};
                double r = sqrt(dot3(dd, dd));
                double eta = wr[lq] * area_b;
                for (int j = 0; j < 3; ++j) gs[j] += eta * bary[3 * lq + j] / r;
            }
            for (int i = 0; i < 3; ++i)
                for (int j = 0; j < 3; ++j)
                    blk[3 * i + j] += wk * bary[3 * kq + i] * (ex[j] - gs[j]) / (4.0 * M_PI);
        }
        for (int e = 0; e < 9; ++e) blocks[9 * p + e] = blk[e];
    }
    return 0;
}

/* int_T lambda_j(y) (x - y) / |x - y|^3 dy for j = 0, 1, 2 over the flat triangle T
 * (out[3 j + c], the gradient in y of the P1 single layer's kernel), in closed form.
 * With n the unit normal (P1 - P0) x (P2 - P0) / |.|, h = n . (x - P0), rho the
 * projection of x onto the plane of T and s = y - rho (in the plane):
 *   normal part    n h int_T lambda_j / R^3                  (the double layer's closed form),
 *   in-plane part  int_T lambda_j (-s) / R^3
 *                = lambda_j(rho) sum_e m_e L_e - g_j I0 + sum_e (g_j . m_e) E_e,
 * g_j = grad lambda_j, m_e the outward in-plane unit normal of edge e, L_e = int_e 1/R,
 * I0 = int_T 1/R, E_e = int_e (y - rho)/R = (A - rho) L_e + u (R_B - R_A - l_A L_e) for
 * the edge from A to B with unit direction u and l_A = u . (A - rho).  Both come from the
 * divergence theorem in the plane: the in-plane gradient of 1/R is -s/R^3, and that of
 * s_i/R is e_i/R - s_i s/R^3. */
void or_p1_dn_inv_r(const double *x, const double *P0, const double *P1, const double *P2, double *out);

void or_p1_grad_inv_r(const double *x, const double *P0, const double *P1, const double *P2, double *out)
{
    const double *P[3] = {P0, P1, P2};
    double e1[3], e2[3], nn[3];
    for (int c = 0; c < 3; ++c) {
        e1[c] = P1[c] - P0[c];
        e2[c] = P2[c] - P0[c];
    }
    cross3(e1, e2, nn);
    double twoA = sqrt(dot3(nn, nn));
    double n[3] = {nn[0] / twoA, nn[1] / twoA, nn[2] / twoA};
    double xp0[3] = {x[0] - P0[0], x[1] - P0[1], x[2] - P0[2]};
    double h = dot3(xp0, n);
    double rho[3] = {x[0] - h * n[0], x[1] - h * n[1], x[2] - h * n[2]};
    double I[3], D[3];
    or_p1_inv_r(x, P0, P1, P2, I);
    or_p1_dn_inv_r(x, P0, P1, P2, D);
    double I0 = I[0] + I[1] + I[2];
    double ML[3] = {0.0, 0.0, 0.0}, M[3][3], E[3][3];
    for (int e = 0; e < 3; ++e) {
        const double *A = P[e], *B = P[(e + 1) % 3];
        double u[3] = {B[0] - A[0], B[1] - A[1], B[2] - A[2]};
        double len = sqrt(dot3(u, u));
        u[0] /= len; u[1] /= len; u[2] /= len;
        cross3(u, n, M[e]);
        double ar[3] = {A[0] - rho[0], A[1] - rho[1], A[2] - rho[2]};
        double br[3] = {B[0] - rho[0], B[1] - rho[1], B[2] - rho[2]};
        double la = dot3(ar, u), lb = dot3(br, u);
        double p = dot3(ar, M[e]);
        double R02 = p * p + h * h;
        double xa[3] = {x[0] - A[0], x[1] - A[1], x[2] - A[2]};
        double xb[3] = {x[0] - B[0], x[1] - B[1], x[2] - B[2]};
        double Ra = sqrt(dot3(xa, xa)), Rb = sqrt(dot3(xb, xb));
        double L = 0.0;
        if (R02 > 1e-30 * twoA) L = log(r_plus_l(Rb, lb, R02) / r_plus_l(Ra, la, R02));
        for (int c = 0; c < 3; ++c) {
            ML[c] += M[e][c] * L;
            E[e][c] = ar[c] * L + u[c] * (Rb - Ra - la * L);
        }
    }
    for (int j = 0; j < 3; ++j) {
        const double *A = P[(j + 1) % 3], *B = P[(j + 2) % 3];
        double ab[3] = {B[0] - A[0], B[1] - A[1], B[2] - A[2]};
        double g[3];
        cross3(n, ab, g);
        g[0] /= twoA; g[1] /= twoA; g[2] /= twoA;
        double rj[3] = {rho[0] - P[j][0], rho[1] - P[j][1], rho[2] - P[j][2]};
        double lam = 1.0 + dot3(g, rj);
        for (int c = 0; c < 3; ++c) {
            double w = lam * ML[c] - g[c] * I0;
            for (int e = 0; e < 3; ++e) w += dot3(g, M[e]) * E[e][c];
            out[3 * j + c] = n[c] * D[j] + w;
        }
    }
}

/* ------------------------------------------------------------------------ */
/* EFIE correction blocks with RWG functions on a near pair (a, b): for the   */
/* local edges i of a and j of b (edge j of a triangle joins its vertices    */
/* j+1 and j+2 and is opposite vertex j; sign s from tsign, length l),        */
/*   RWG on b: f_j(y) = s l / (2 A_b) (y - P_j),  div f_j = s l / A_b,         */
/*   int_b f_j / R = s l / (2 A_b) sum_m (P_m - P_j) int_b lambda_m / R,       */
/* and                                                                        */
/*   blkA[i][j] = sum_{k in a} w_k f_i(x_k) . (int_b f_j / R - G_kj),          */
/*   blkB[i][j] = sum_{k in a} w_k div f_i (int_b div f_j / R - D_kj),         */
/* with the Gauss sums G_kj = sum_{l in b, l != k} w_l f_j(y_l) / |x_k - y_l|  */
/* and D_kj the same for div f_j (l == k only when a == b).                   */
/*   tsign: nt x 3 (+1 / -1); blkA, blkB: npairs x 3 x 3                      */
/* ------------------------------------------------------------------------ */
int or_efie_near_blocks(const double *vtx, const int32_t *tri, const double *tsign, int q, int64_t npairs,
                        const int64_t *pa, const int64_t *pb, double *blkA, double *blkB)
{
    double bary[21], wr[7];
    if (or_quad_rule(q, bary, wr) != 0) return -1;
    #pragma omp parallel for schedule(dynamic, 64)
    for (int64_t p = 0; p < npairs; ++p) {
        int64_t a = pa[p], b = pb[p];
        const double *A[3], *B[3];
        for (int m = 0; m < 3; ++m) {
            A[m] = vtx + 3 * (int64_t)tri[3 * a + m];
            B[m] = vtx + 3 * (int64_t)tri[3 * b + m];
        }
        double ea[3], fa[3], na[3], eb[3], fb[3], nb[3];
        for (int c = 0; c < 3; ++c) {
            ea[c] = A[1][c] - A[0][c]; fa[c] = A[2][c] - A[0][c];
            eb[c] = B[1][c] - B[0][c]; fb[c] = B[2][c] - B[0][c];
        }
        cross3(ea, fa, na);
        cross3(eb, fb, nb);
        double area_a = 0.5 * sqrt(dot3(na, na)), area_b = 0.5 * sqrt(dot3(nb, nb));
        double ca[3], cb[3];  /* s l / (2 A) per local edge */
        for (int j = 0; j < 3; ++j) {
            double da[3], db[3];
            for (int c = 0; c < 3; ++c) {
                da[c] = A[(j + 2) % 3][c] - A[(j + 1) % 3][c];
                db[c] = B[(j + 2) % 3][c] - B[(j + 1) % 3][c];
            }
            ca[j] = tsign[3 * a + j] * sqrt(dot3(da, da)) / (2.0 * area_a);
            cb[j] = tsign[3 * b + j] * sqrt(dot3(db, db)) / (2.0 * area_b);
        }
        double bA[9] = {0}, bB[9] = {0};
        for (int kq = 0; kq < q; ++kq) {
            double xk[3];
            for (int c = 0; c < 3; ++c)
                xk[c] = bary[3 * kq] * A[0][c] + bary[3 * kq + 1] * A[1][c] + bary[3 * kq + 2] * A[2][c];
            double wk = wr[kq] * area_a;
            double I[3];
            or_p1_inv_r(xk, B[0], B[1], B[2], I);
            /* Gauss sums: sum_l eta_l y_l / r and sum_l eta_l / r */
            double gy[3] = {0.0, 0.0, 0.0}, g1 = 0.0;
            for (int lq = 0; lq < q; ++lq) {
                if (a == b && lq == kq) continue;
                double yl[3];
                for (int c = 0; c < 3; ++c)
                    yl[c] = bary[3 * lq] * B[0][c] + bary[3 * lq + 1] * B[1][c] + bary[3 * lq + 2] * B[2][c];
                double dd[3] = {xk[0] - yl[0], xk[1] - yl[1], xk[2] - yl[2]};
                double e = wr[lq] * area_b / sqrt(dot3(dd, dd));
                for (int c = 0; c < 3; ++c) gy[c] += e * yl[c];
                g1 += e;
            }
            double isum = I[0] + I[1] + I[2];
            for (int j = 0; j < 3; ++j) {
                /* int_b f_j / R - Gauss, and the same for div f_j */
                double vec[3];
                for (int c = 0; c < 3; ++c) {
                    double an = I[0] * (B[0][c] - B[j][c]) + I[1] * (B[1][c] - B[j][c]) + I[2] * (B[2][c] - B[j][c]);
                    double gs = gy[c] - g1 * B[j][c];
                    vec[c] = cb[j] * (an - gs);
                }
                double dvj = 2.0 * cb[j] * (isum - g1);
                for (int i = 0; i < 3; ++i) {
                    double fi[3];
                    for (int c = 0; c < 3; ++c) fi[c] = ca[i] * (xk[c] - A[i][c]);
                    bA[3 * i + j] += wk * dot3(fi, vec);
                    bB[3 * i + j] += wk * 2.0 * ca[i] * dvj;
                }
            }
        }
        for (int e = 0; e < 9; ++e) {
            blkA[9 * p + e] = bA[e];
            blkB[9 * p + e] = bB[e];
        }
    }
    return 0;
}

/* ------------------------------------------------------------------------ */
/* MFIE part of the electromagnetic listing (nxK = integral(sigma, sigma,    */
/* nx(Vh), grady[exp(ikr)/r], Vh) / (4 pi) + regularize(..., 'grady[1/r]')):  */
/*   grad_y exp(ikr)/r = F(r) (x - y),  F = (1 - i k r) exp(i k r) / r^3.    */
/* v[t] = sum_l F(r_tl) (x_t - y_l) x u_l  (3-vectors, cross product), with  */
/* the pairs inside one triangle left out (tri_t[t] == tri_s[l]): their      */
/* vector is normal to the triangle and meets an in-plane test function.     */
/*   u: ns x 3 x nrhs complex (u[((3 j + c) ns + l)]), v: nt x 3 x nrhs.    */
/* ------------------------------------------------------------------------ */
int or_grad_cross_matvec(int64_t nt, const double *xt, const int64_t *tri_t, int64_t ns, const double *ys,
                         const int64_t *tri_s, double k, int64_t nrhs, const double *u, double *v)
{
    #pragma omp parallel
    {
        double *acc = (double *)calloc((size_t)(6 * nrhs), sizeof(double));
        #pragma omp for schedule(dynamic, 16)
        for (int64_t t = 0; t < nt; ++t) {
            for (int64_t j = 0; j < 6 * nrhs; ++j) acc[j] = 0.0;
            const double *x = xt + 3 * t;
            for (int64_t l = 0; l < ns; ++l) {
                if (tri_t[t] == tri_s[l]) continue;
                const double *y = ys + 3 * l;
                double d[3] = {x[0] - y[0], x[1] - y[1], x[2] - y[2]};
                double r = sqrt(dot3(d, d));
                double c = cos(k * r), sn = sin(k * r);
                double fr = (c + k * r * sn) / (r * r * r), fi = (sn - k * r * c) / (r * r * r);
                for (int64_t j = 0; j < nrhs; ++j) {
                    double ur[3], ui[3];
                    for (int a = 0; a < 3; ++a) {
                        ur[a] = u[2 * ((3 * j + a) * ns + l)];
                        ui[a] = u[2 * ((3 * j + a) * ns + l) + 1];
                    }
                    double cr[3], ci[3];
                    cross3(d, ur, cr);
                    cross3(d, ui, ci);
                    for (int a = 0; a < 3; ++a) {
                        acc[6 * j + 2 * a] += fr * cr[a] - fi * ci[a];
                        acc[6 * j + 2 * a + 1] += fr * ci[a] + fi * cr[a];
                    }
                }
            }
            for (int64_t j = 0; j < nrhs; ++j)
                for (int a = 0; a < 3; ++a) {
                    v[2 * ((3 * j + a) * nt + t)] = acc[6 * j + 2 * a];
                    v[2 * ((3 * j + a) * nt + t) + 1] = acc[6 * j + 2 * a + 1];
                }
        }
        free(acc);
    }
    return 0;
}

/* MFIE correction blocks on the near pair (a, b), a != b (pairs inside one
 * triangle give 0): for local RWG edges i of a and j of b,
 *   blk[i][j] = (1/4pi) sum_{k in a} w_k (n_a x f_i(x_k)) .
 *               (int_b (x_k - y)/R^3 x f_j(y) dy - sum_{l in b} w_l (x_k - y_l)/r^3 x f_j(y_l)),
 * int_b (x - y)/R^3 x f_j = c_j sum_m (int_b lambda_m (x - y)/R^3) x (P_m - P_j),
 * f_j = c_j (y - P_j), c_j = s l_j / (2 A_b).   blk: npairs x 3 x 3. */
int or_mfie_near_blocks(const double *vtx, const int32_t *tri, const double *tsign, int q, int64_t npairs,
                        const int64_t *pa, const int64_t *pb, double *blk)
{
    double bary[21], wr[7];
    if (or_quad_rule(q, bary, wr) != 0) return -1;
    #pragma omp parallel for schedule(dynamic, 64)
    for (int64_t p = 0; p < npairs; ++p) {
        int64_t a = pa[p], b = pb[p];
        double out[9] = {0};
        if (a != b) {
            const double *A[3], *B[3];
            for (int m = 0; m < 3; ++m) {
                A[m] = vtx + 3 * (int64_t)tri[3 * a + m];
                B[m] = vtx + 3 * (int64_t)tri[3 * b + m];
            }
            double ea[3], fa[3], na[3], eb[3], fb[3], nb[3];
            for (int c = 0; c < 3; ++c) {
                ea[c] = A[1][c] - A[0][c]; fa[c] = A[2][c] - A[0][c];
                eb[c] = B[1][c] - B[0][c]; fb[c] = B[2][c] - B[0][c];
            }
            cross3(ea, fa, na);
            cross3(eb, fb, nb);
            double two_a = sqrt(dot3(na, na)), two_b = sqrt(dot3(nb, nb));
            double un[3] = {na[0] / two_a, na[1] / two_a, na[2] / two_a};
            double ca[3], cb[3];
            for (int j = 0; j < 3; ++j) {
                double da[3], db[3];
                for (int c = 0; c < 3; ++c) {
                    da[c] = A[(j + 2) % 3][c] - A[(j + 1) % 3][c];
                    db[c] = B[(j + 2) % 3][c] - B[(j + 1) % 3][c];
                }
                ca[j] = tsign[3 * a + j] * sqrt(dot3(da, da)) / two_a;
                cb[j] = tsign[3 * b + j] * sqrt(dot3(db, db)) / two_b;
            }
            for (int kq = 0; kq < q; ++kq) {
                double xk[3];
                for (int c = 0; c < 3; ++c)
                    xk[c] = bary[3 * kq] * A[0][c] + bary[3 * kq + 1] * A[1][c] + bary[3 * kq + 2] * A[2][c];
                double wk = wr[kq] * 0.5 * two_a;
                double V[9];
                or_p1_grad_inv_r(xk, B[0], B[1], B[2], V);
                for (int j = 0; j < 3; ++j) {
                    double an[3] = {0.0, 0.0, 0.0};
                    for (int m = 0; m < 3; ++m) {
                        double pm[3] = {B[m][0] - B[j][0], B[m][1] - B[j][1], B[m][2] - B[j][2]};
                        double cr[3];
                        cross3(V + 3 * m, pm, cr);
                        for (int c = 0; c < 3; ++c) an[c] += cb[j] * cr[c];
                    }
                    for (int lq = 0; lq < q; ++lq) {
                        double yl[3];
                        for (int c = 0; c < 3; ++c)
                            yl[c] = bary[3 * lq] * B[0][c] + bary[3 * lq + 1] * B[1][c] + bary[3 * lq + 2] * B[2][c];
                        double d[3] = {xk[0] - yl[0], xk[1] - yl[1], xk[2] - yl[2]};
                        double r = sqrt(dot3(d, d));
                        double e = wr[lq] * 0.5 * two_b / (r * r * r);
                        double fj[3] = {cb[j] * (yl[0] - B[j][0]), cb[j] * (yl[1] - B[j][1]), cb[j] * (yl[2] - B[j][2])};
                        double cr[3];
                        cross3(d, fj, cr);
                        for (int c = 0; c < 3; ++c) an[c] -= e * cr[c];
                    }
                    for (int i = 0; i < 3; ++i) {
                        double fi[3] = {ca[i] * (xk[0] - A[i][0]), ca[i] * (xk[1] - A[i][1]), ca[i] * (xk[2] - A[i][2])};
                        double nf[3];
                        cross3(un, fi, nf);
                        out[3 * i + j] += wk * dot3(nf, an) / (4.0 * M_PI);
                    }
                }
            }
        }
        for (int e = 0; e < 9; ++e) blk[9 * p + e] = out[e];
    }
    return 0;
}

/* Number of OpenMP threads the oracle runs with (1 without OpenMP). */
/* ------------------------------------------------------------------------ */
/* Double layer (the next operator after the single layer; the paper's       */
/* grady[exp(ikr)/r] kernels with the 'grady[1/r]' regularisation):          */
/*   H(x, y) = n_y . grad_y exp(ik|x-y|)/|x-y|                                */
/*           = (1 - i k r) exp(i k r) n_y . (x - y) / r^3,                   */
/* n_y the unit normal of the source triangle.  Within one flat triangle     */
/* n_y . (x - y) = 0, so the point paired with itself takes H := 0.          */
/* ------------------------------------------------------------------------ */

/* v[t, j] = sum_l H(x_t, y_l) u[l, j]; ns_nrm: ns x 3 unit normals at the sources. */
int or_dl_kernel_matvec(int64_t nt, const double *xt, const int64_t *tid,
                        int64_t ns, const double *ys, const double *ns_nrm, double k, int64_t nrhs,
                        const double *u, double *v)
{
    #pragma omp parallel
    {
        double *acc = (double *)calloc((size_t)(2 * nrhs), sizeof(double));
        #pragma omp for schedule(dynamic, 16)
        for (int64_t t = 0; t < nt; ++t) {
            for (int64_t j = 0; j < 2 * nrhs; ++j) acc[j] = 0.0;
            for (int64_t l = 0; l < ns; ++l) {
                if (tid != NULL && tid[t] == l) continue;
                const double *x = xt + 3 * t, *y = ys + 3 * l, *n = ns_nrm + 3 * l;
                double d[3] = {x[0] - y[0], x[1] - y[1], x[2] - y[2]};
                double r = sqrt(dot3(d, d));
                double f = dot3(n, d) / (r * r * r);
                /* (1 - i k r)(cos kr + i sin kr) */
                double c = cos(k * r), sn = sin(k * r);
                double hr = (c + k * r * sn) * f, hi = (sn - k * r * c) * f;
                for (int64_t j = 0; j < nrhs; ++j) {
                    double ur = u[2 * (j * ns + l)], ui = u[2 * (j * ns + l) + 1];
                    acc[2 * j] += hr * ur - hi * ui;
                    acc[2 * j + 1] += hr * ui + hi * ur;
                }
            }
            for (int64_t j = 0; j < nrhs; ++j) {
                v[2 * (j * nt + t)] = acc[2 * j];
                v[2 * (j * nt + t) + 1] = acc[2 * j + 1];
            }
        }
        free(acc);
    }
    return 0;
}

/* Adjoint double layer: the normal derivative at the target,
 *   H'(x, y) = n_x . grad_x exp(ik|x-y|)/|x-y| = -(1 - i k r) exp(i k r) n_x . (x - y) / r^3,
 * v[t, j] = sum_l H'(x_t, y_l) u[l, j]; nt_nrm: nt x 3 unit normals at the targets;
 * the point paired with itself takes H' := 0. */
int or_adl_kernel_matvec(int64_t nt, const double *xt, const double *nt_nrm, const int64_t *tid,
                         int64_t ns, const double *ys, double k, int64_t nrhs, const double *u, double *v)
{
    #pragma omp parallel
    {
        double *acc = (double *)calloc((size_t)(2 * nrhs), sizeof(double));
        #pragma omp for schedule(dynamic, 16)
        for (int64_t t = 0; t < nt; ++t) {
            for (int64_t j = 0; j < 2 * nrhs; ++j) acc[j] = 0.0;
            const double *x = xt + 3 * t, *n = nt_nrm + 3 * t;
            for (int64_t l = 0; l < ns; ++l) {
                if (tid != NULL && tid[t] == l) continue;
                const double *y = ys + 3 * l;
                double d[3] = {x[0] - y[0], x[1] - y[1], x[2] - y[2]};
                double r = sqrt(dot3(d, d));
                double f = -dot3(n, d) / (r * r * r);
                double c = cos(k * r), sn = sin(k * r);
                double hr = (c + k * r * sn) * f, hi = (sn - k * r * c) * f;
                for (int64_t j = 0; j < nrhs; ++j) {
                    double ur = u[2 * (j * ns + l)], ui = u[2 * (j * ns + l) + 1];
                    acc[2 * j] += hr * ur - hi * ui;
                    acc[2 * j + 1] += hr * ui + hi * ur;
                }
            }
            for (int64_t j = 0; j < nrhs; ++j) {
                v[2 * (j * nt + t)] = acc[2 * j];
                v[2 * (j * nt + t) + 1] = acc[2 * j + 1];
            }
        }
        free(acc);
    }
    return 0;
}

/*
 * int_T lambda_j(y) n . (x - y) / |x - y|^3 dy over the flat triangle T =
 * (P0, P1, P2) with unit normal n = (P1 - P0) x (P2 - P0) / |.|, in closed
 * form.  With h = n . (x - P0) (so n . (x - y) = h on T) and rho the
 * projection of x onto the plane of T:
 *   h int_T 1/R^3 = sign(h) Omega, Omega the solid angle of T seen from x,
 *     Omega = sum_e [atan(p_e s+ / (q_e + |h| R+)) - atan(p_e s- / (q_e + |h| R-))]
 *     (the edge sum that also gives the |h| term of int_T 1/R);
 *   int_T (y - rho)/R^3 = - sum_e m_e ln((R+ + s+)/(R- + s-))
 *     (in-plane divergence theorem applied to 1/R);
 *   result_j = lambda_j(rho) sign(h) Omega + h grad lambda_j . int_T (y - rho)/R^3.
 * For x in the plane of T the value is 0 (principal value).
 */
void or_p1_dn_inv_r(const double *x, const double *P0, const double *P1, const double *P2, double *out)
{
    const double *P[3] = {P0, P1, P2};
    double e1[3], e2[3], nn[3];
    for (int c = 0; c < 3; ++c) {
        e1[c] = P1[c] - P0[c];
        e2[c] = P2[c] - P0[c];
    }
    cross3(e1, e2, nn);
    double twoA = sqrt(dot3(nn, nn));
    double n[3] = {nn[0] / twoA, nn[1] / twoA, nn[2] / twoA};
    double xp0[3] = {x[0] - P0[0], x[1] - P0[1], x[2] - P0[2]};
    double h = dot3(xp0, n);
    double ah = fabs(h);
    if (ah == 0.0) {
        out[0] = out[1] = out[2] = 0.0;
        return;
    }
    double rho0[3] = {x[0] - h * n[0], x[1] - h * n[1], x[2] - h * n[2]};
    double omega = 0.0, Wv[3] = {0.0, 0.0, 0.0};
    for (int i = 0; i < 3; ++i) {
        const double *Pm = P[i], *Pp = P[(i + 1) % 3];
        double t[3] = {Pp[0] - Pm[0], Pp[1] - Pm[1], Pp[2] - Pm[2]};
        double len = sqrt(dot3(t, t));
        t[0] /= len; t[1] /= len; t[2] /= len;
        double m[3];
        cross3(t, n, m);
        double am[3] = {Pm[0] - rho0[0], Pm[1] - rho0[1], Pm[2] - rho0[2]};
        double ap[3] = {Pp[0] - rho0[0], Pp[1] - rho0[1], Pp[2] - rho0[2]};
        double lm = dot3(am, t), lp = dot3(ap, t);
        double p = dot3(am, m);
        double R02 = p * p + h * h;
        double xm[3] = {x[0] - Pm[0], x[1] - Pm[1], x[2] - Pm[2]};
        double xpp[3] = {x[0] - Pp[0], x[1] - Pp[1], x[2] - Pp[2]};
        double Rm = sqrt(dot3(xm, xm)), Rp = sqrt(dot3(xpp, xpp));
        double L = log(r_plus_l(Rp, lp, R02) / r_plus_l(Rm, lm, R02));
        omega += atan(p * lp / (R02 + ah * Rp)) - atan(p * lm / (R02 + ah * Rm));
        Wv[0] -= m[0] * L;
        Wv[1] -= m[1] * L;
        Wv[2] -= m[2] * L;
    }
    double sg = h > 0.0 ? 1.0 : -1.0;
    for (int j = 0; j < 3; ++j) {
        const double *A = P[(j + 1) % 3], *B = P[(j + 2) % 3];
        double ab[3] = {B[0] - A[0], B[1] - A[1], B[2] - A[2]};
        double g[3];
        cross3(n, ab, g);
        g[0] /= twoA; g[1] /= twoA; g[2] /= twoA;
        double rj[3] = {rho0[0] - P[j][0], rho0[1] - P[j][1], rho0[2] - P[j][2]};
        double lam0 = 1.0 + dot3(g, rj);
        out[j] = lam0 * sg * omega + h * dot3(g, Wv);
    }
}

/* Correction blocks of the double layer on near pairs (a, b), as or_near_blocks
   with the 'grady[1/r]' part: (1/4pi) sum_k w_k lambda_i(x_k) (I_j(x_k, b) -
   sum_l eta_l lambda_j(y_l) n_b . (x_k - y_l)/r^3).  a == b gives 0 (coplanar). */
int or_dl_near_blocks(const double *vtx, const int32_t *tri, int q,
                      int64_t npairs, const int64_t *pa, const int64_t *pb, double *blocks)
{
    double bary[21], wr[7];
    if (or_quad_rule(q, bary, wr) != 0) return -1;
    #pragma omp parallel for schedule(dynamic, 64)
    for (int64_t p = 0; p < npairs; ++p) {
        int64_t a = pa[p], b = pb[p];
        double blk[9] = {0};
        if (a != b) {
            const double *A[3], *B[3];
            for (int m = 0; m < 3; ++m) {
                A[m] = vtx + 3 * (int64_t)tri[3 * a + m];
                B[m] = vtx + 3 * (int64_t)tri[3 * b + m];
            }
            double ea[3], fa[3], na[3], eb[3], fb[3], nb[3];
            for (int c = 0; c < 3; ++c) {
                ea[c] = A[1][c] - A[0][c]; fa[c] = A[2][c] - A[0][c];
                eb[c] = B[1][c] - B[0][c]; fb[c] = B[2][c] - B[0][c];
            }
            cross3(ea, fa, na);
            cross3(eb, fb, nb);
            double area_a = 0.5 * sqrt(dot3(na, na)), area_b = 0.5 * sqrt(dot3(nb, nb));
            double un[3] = {nb[0] / (2 * area_b), nb[1] / (2 * area_b), nb[2] / (2 * area_b)};
            for (int kq = 0; kq < q; ++kq) {
                double xk[3];
                for (int c = 0; c < 3; ++c)
                    xk[c] = bary[3 * kq] * A[0][c] + bary[3 * kq + 1] * A[1][c] + bary[3 * kq + 2] * A[2][c];
                double wk = wr[kq] * area_a;
                double ex[3];
                or_p1_dn_inv_r(xk, B[0], B[1], B[2], ex);
                double gs[3] = {0.0, 0.0, 0.0};
                for (int lq = 0; lq < q; ++lq) {
                    double yl[3];
                    for (int c = 0; c < 3; ++c)
                        yl[c] = bary[3 * lq] * B[0][c] + bary[3 * lq + 1] * B[1][c] + bary[3 * lq + 2] * B[2][c];
                    double dd[3] = {xk[0] - yl[0], xk[1] - yl[1], xk[2] - yl[2]};
                    double r = sqrt(dot3(dd, dd));
                    double f = wr[lq] * area_b * dot3(un, dd) / (r * r * r);
                    for (int j = 0; j < 3; ++j) gs[j] += f * bary[3 * lq + j];
                }
                for (int i = 0; i < 3; ++i)
                    for (int j = 0; j < 3; ++j)
                        blk[3 * i + j] += wk * bary[3 * kq + i] * (ex[j] - gs[j]) / (4.0 * M_PI);
            }
        }
        for (int e = 0; e < 9; ++e) blocks[9 * p + e] = blk[e];
    }
    return 0;
}

int or_num_threads(void)
{
#ifdef _OPENMP
    extern int omp_get_max_threads(void);
    return omp_get_max_threads();
#else
    return 1;
#endif
}
