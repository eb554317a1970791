// Device geometry for the correction (Sec. 5.2): double3 arithmetic and the
// closed-form integral of a P1 function times 1/|x - y| over a flat triangle,
// shared by the Galerkin correction and the correction of point potentials.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace gyps {

static __device__ inline double3 ld3(const double *v, int64_t i) { return make_double3(v[3 * i], v[3 * i + 1], v[3 * i + 2]); }
static __device__ inline double3 operator-(double3 a, double3 b) { return make_double3(a.x - b.x, a.y - b.y, a.z - b.z); }
static __device__ inline double3 operator+(double3 a, double3 b) { return make_double3(a.x + b.x, a.y + b.y, a.z + b.z); }
static __device__ inline double3 operator*(double s, double3 a) { return make_double3(s * a.x, s * a.y, s * a.z); }
static __device__ inline double dot(double3 a, double3 b) { return a.x * b.x + a.y * b.y + a.z * b.z; }
static __device__ inline double3 cross(double3 a, double3 b)
{
    return make_double3(a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x);
}


// ---------------------------------------------------------------- correction
// Closed-form y-integral over a flat triangle P of lambda_j(y)/|x - y| (Sec. 5.2,
// "integral in y computed analytically"), after Wilton et al. (1984) and Graglia
// (1993).  Splitting lambda_j(y) = lambda_j(rho) + grad lambda_j . (y - rho) about
// the projection rho of x onto the plane reduces it to two edge sums:
//   int 1/R      = sum_e p_e L_e - |h| sum_e (atan(p_e s+ / (q_e + |h| R+)) - atan(p_e s- / (q_e + |h| R-)))
//   int (y-rho)/R = 1/2 sum_e m_e (q_e L_e + s+ R+ - s- R-)
// with h the height of x over the plane, m_e the in-plane outward edge normal,
// p_e the signed distance from rho to edge e, s+- the end abscissae along the
// edge, R+- the end distances, q_e = p_e^2 + h^2 and L_e = ln((R+ + s+)/(R- + s-)).
static __device__ inline double log_arg(double R, double s, double qe) { return s >= 0.0 ? R + s : qe / (R - s); }

static __device__ void p1_over_r(double3 x, const double3 P[3], double out[3])
{
    double3 nn = cross(P[1] - P[0], P[2] - P[0]);
    double two_area = sqrt(dot(nn, nn));
    double3 n = (1.0 / two_area) * nn;
    double h = dot(x - P[0], n);
    double ah = fabs(h);
    double3 rho = x - h * n;
    double S = 0.0;
    double3 Vv = make_double3(0.0, 0.0, 0.0);
#pragma unroll
    for (int e = 0; e < 3; ++e) {
        double3 a = P[e], b = P[(e + 1) % 3];
        double3 tv = b - a;
        double3 t = (1.0 / sqrt(dot(tv, tv))) * tv;
        double3 me = cross(t, n);
        double sm = dot(a - rho, t), sp = dot(b - rho, t);
        double pe = dot(a - rho, me);
        double qe = pe * pe + h * h;
        double3 xa = x - a, xb = x - b;
        double Rm = sqrt(dot(xa, xa)), Rp = sqrt(dot(xb, xb));
        double L = 0.0;
        if (qe > 1e-30 * two_area) L = log(log_arg(Rp, sp, qe) / log_arg(Rm, sm, qe));
        S += pe * L;
        if (ah > 0.0) S -= ah * (atan(pe * sp / (qe + ah * Rp)) - atan(pe * sm / (qe + ah * Rm)));
        double c = 0.5 * (qe * L + sp * Rp - sm * Rm);
        Vv = Vv + c * me;
    }
#pragma unroll
    for (int j = 0; j < 3; ++j) {
        double3 g = (1.0 / two_area) * cross(n, P[(j + 2) % 3] - P[(j + 1) % 3]);  // grad lambda_j
        double lam_rho = 1.0 + dot(g, rho - P[j]);
        out[j] = lam_rho * S + dot(g, Vv);
    }
}

// Closed-form y-integral over the flat triangle P of lambda_j(y) n . (x - y)/|x - y|^3
// (the double layer's 'grady[1/r]' part), n = (P1 - P0) x (P2 - P0) / |.|.  With
// h = n . (x - P0), n . (x - y) = h on P, and
//   h int 1/R^3 = sign(h) Omega,  Omega = sum_e [atan(p_e s+ / (q_e + |h| R+)) - atan(p_e s- / (q_e + |h| R-))]
//   (the solid angle of P seen from x, the edge sum of the single layer's |h| term),
//   int (y - rho)/R^3 = - sum_e m_e ln((R+ + s+)/(R- + s-))  (in-plane divergence theorem on 1/R):
//   out_j = lambda_j(rho) sign(h) Omega + h grad lambda_j . int (y - rho)/R^3;  0 for x in the plane.
static __device__ void p1_dn_over_r(double3 x, const double3 P[3], double out[3])
{
    double3 nn = cross(P[1] - P[0], P[2] - P[0]);
    double two_area = sqrt(dot(nn, nn));
    double3 n = (1.0 / two_area) * nn;
    double h = dot(x - P[0], n);
    double ah = fabs(h);
    if (ah == 0.0) {
        out[0] = out[1] = out[2] = 0.0;
        return;
    }
    double3 rho = x - h * n;
    double omega = 0.0;
    double3 Wv = make_double3(0.0, 0.0, 0.0);
#pragma unroll
    for (int e = 0; e < 3; ++e) {
        double3 a = P[e], b = P[(e + 1) % 3];
        double3 tv = b - a;
        double3 t = (1.0 / sqrt(dot(tv, tv))) * tv;
        double3 me = cross(t, n);
        double sm = dot(a - rho, t), sp = dot(b - rho, t);
        double pe = dot(a - rho, me);
        double qe = pe * pe + h * h;
        double3 xa = x - a, xb = x - b;
        double Rm = sqrt(dot(xa, xa)), Rp = sqrt(dot(xb, xb));
        double L = log(log_arg(Rp, sp, qe) / log_arg(Rm, sm, qe));
        omega += atan(pe * sp / (qe + ah * Rp)) - atan(pe * sm / (qe + ah * Rm));
        Wv = Wv + (-L) * me;
    }
    const double sg = h > 0.0 ? 1.0 : -1.0;
#pragma unroll
    for (int j = 0; j < 3; ++j) {
        double3 g = (1.0 / two_area) * cross(n, P[(j + 2) % 3] - P[(j + 1) % 3]);  // grad lambda_j
        double lam_rho = 1.0 + dot(g, rho - P[j]);
        out[j] = lam_rho * sg * omega + h * dot(g, Wv);
    }
}

// Closed-form y-integral over the flat triangle P of lambda_j(y) (x - y)/|x - y|^3
// (the gradient in y of the single layer's 1/R, the MFIE's 'grady[1/r]' part).
// With n, h, rho as above and s = y - rho in the plane:
//   normal part    n h int lambda_j / R^3                    (p1_dn_over_r),
//   in-plane part  int lambda_j (-s)/R^3
//                = lambda_j(rho) sum_e m_e L_e - g_j I0 + sum_e (g_j . m_e) E_e,
// g_j = grad lambda_j, I0 = int 1/R, E_e = int_e (y - rho)/R = (a - rho) L_e + t (R+ - R- - s- L_e)
// (divergence theorem in the plane on 1/R and on s_i/R: grad (s_i/R) = e_i/R - s_i s/R^3).
static __device__ void p1_grad_over_r(double3 x, const double3 P[3], double3 out[3])
{
    double3 nn = cross(P[1] - P[0], P[2] - P[0]);
    double two_area = sqrt(dot(nn, nn));
    double3 n = (1.0 / two_area) * nn;
    double h = dot(x - P[0], n);
    double3 rho = x - h * n;
    double I[3], D[3];
    p1_over_r(x, P, I);
    p1_dn_over_r(x, P, D);
    const double I0 = I[0] + I[1] + I[2];
    double3 ML = make_double3(0.0, 0.0, 0.0), M[3], E[3];
#pragma unroll
    for (int e = 0; e < 3; ++e) {
        double3 a = P[e], b = P[(e + 1) % 3];
        double3 tv = b - a;
        double3 t = (1.0 / sqrt(dot(tv, tv))) * tv;
        M[e] = cross(t, n);
        double sm = dot(a - rho, t), sp = dot(b - rho, t);
        double pe = dot(a - rho, M[e]);
        double qe = pe * pe + h * h;
        double3 xa = x - a, xb = x - b;
        double Rm = sqrt(dot(xa, xa)), Rp = sqrt(dot(xb, xb));
        double L = 0.0;
        if (qe > 1e-30 * two_area) L = log(log_arg(Rp, sp, qe) / log_arg(Rm, sm, qe));
        ML = ML + L * M[e];
        E[e] = L * (a - rho) + (Rp - Rm - sm * L) * t;
    }
#pragma unroll
    for (int j = 0; j < 3; ++j) {
        double3 g = (1.0 / two_area) * cross(n, P[(j + 2) % 3] - P[(j + 1) % 3]);  // grad lambda_j
        double lam_rho = 1.0 + dot(g, rho - P[j]);
        double3 w = lam_rho * ML - I0 * g;
#pragma unroll
        for (int e = 0; e < 3; ++e) w = w + dot(g, M[e]) * E[e];
        out[j] = D[j] * n + w;
    }
}

}  // namespace gyps
