// Single-layer potential at arbitrary points: the radiation operator of the
// listing in Sec. 5.4,
//   Sdom = integral(points, S2, Gxy, Vh)/(4 pi) + regularize(points, S2, '[1/r]', Vh)/(4 pi),
//   P[i, c] = (1/4pi) sum_l G(x_i, y_l) eta_l sum_j phi_j(y_l) X[j, c]
//           + (1/4pi) sum_{b near x_i} sum_j (int_b lambda_j / |x_i - y| - sum_{l in b} eta_l lambda_j(y_l) / |x_i - y_l|) X[v_j(b), c],
// the first term by the far kernels with the points as targets, the second (the
// [1/r] regularisation, Sec. 5.2) for every triangle whose centroid lies within
// twice its centroid-to-vertex radius of the point.
#include <cmath>

#include "internal.h"
#include "p1_geom.cuh"

namespace gyps {

constexpr double kInv4PiP = 0.0795774715459476678844418816862571810;

// Points given as xyz triples (FP64) -> float4 / double4 copies for the far kernels.
__global__ void point_prep_kernel(const double *p, int64_t n, float4 *p32, double4_32a *p64)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const double x = p[3 * i], y = p[3 * i + 1], z = p[3 * i + 2];
    p32[i] = make_float4((float)x, (float)y, (float)z, 0.0f);
    p64[i] = make_double4_32a(x, y, z, 0.0);
}

// Per triangle: centroid and the squared near radius (2 x largest centroid-vertex distance)^2.
__global__ void tri_center_kernel(const double *vtx, const int32_t *tri, int64_t nt, double4_32a *cen, float4 *cen32)
{
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= nt) return;
    const double3 P[3] = {ld3(vtx, tri[3 * t]), ld3(vtx, tri[3 * t + 1]), ld3(vtx, tri[3 * t + 2])};
    const double3 c = (1.0 / 3.0) * (P[0] + P[1] + P[2]);
    double r2 = 0.0;
#pragma unroll
    for (int m = 0; m < 3; ++m) r2 = fmax(r2, dot(P[m] - c, P[m] - c));
    cen[t] = make_double4_32a(c.x, c.y, c.z, 4.0 * r2);
    // FP32 candidate test: a widened radius keeps every triangle the FP64 test accepts
    cen32[t] = make_float4((float)c.x, (float)c.y, (float)c.z, (float)(4.0 * r2 * 1.001));
}

// P[i, c0 + cc] = (1/4pi) (v[i, c0 + cc] + correction), CH columns per launch row.
template <int CH>
__global__ void point_finish_kernel(const double *vtx, const int32_t *tri, int64_t nt, const double4_32a *pts64,
                                    const Rule rule, const double4_32a *cen, const float4 *cen32,
                                    const double4_32a *tgt, int64_t npts,
                                    const double2 *v, int64_t ldv, const double2 *X, int64_t ldx, int nrhs,
                                    double2 *P, int64_t ldp)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int c0 = blockIdx.y * CH;
    if (i >= npts) return;
    const double4_32a xp = tgt[i];
    const double3 x = make_double3(xp.x, xp.y, xp.z);
    const int q = rule.q;
    double2 acc[CH];
#pragma unroll
    for (int cc = 0; cc < CH; ++cc) acc[cc] = make_double2(0.0, 0.0);
    // FP32 scan with a margin above its rounding error (coordinates of size |x|), then the FP64 test
    const float xf = (float)x.x, yf = (float)x.y, zf = (float)x.z;
    const float margin = 1e-5f * (1.0f + xf * xf + yf * yf + zf * zf);
    for (int64_t b = 0; b < nt; ++b) {
        const float4 cf = cen32[b];
        const float ex = xf - cf.x, ey = yf - cf.y, ez = zf - cf.z;
        if (ex * ex + ey * ey + ez * ez >= cf.w + margin) continue;
        const double4_32a c = cen[b];
        const double3 d = make_double3(x.x - c.x, x.y - c.y, x.z - c.z);
        if (dot(d, d) >= c.w) continue;
        const int32_t vb[3] = {tri[3 * b], tri[3 * b + 1], tri[3 * b + 2]};
        const double3 B[3] = {ld3(vtx, vb[0]), ld3(vtx, vb[1]), ld3(vtx, vb[2])};
        double corr[3];
        p1_over_r(x, B, corr);
        for (int lq = 0; lq < q; ++lq) {
            const double4_32a y = pts64[b * q + lq];
            const double3 e = make_double3(x.x - y.x, x.y - y.y, x.z - y.z);
            const double r2 = dot(e, e);
            if (r2 <= 0.0) continue;
            const double wr = y.w / sqrt(r2);
#pragma unroll
            for (int j = 0; j < 3; ++j) corr[j] -= wr * rule.bary[3 * lq + j];
        }
#pragma unroll
        for (int cc = 0; cc < CH; ++cc) {
            if (c0 + cc >= nrhs) break;
#pragma unroll
            for (int j = 0; j < 3; ++j) {
                const double2 xv = X[vb[j] + (int64_t)(c0 + cc) * ldx];
                acc[cc].x += corr[j] * xv.x;
                acc[cc].y += corr[j] * xv.y;
            }
        }
    }
#pragma unroll
    for (int cc = 0; cc < CH; ++cc) {
        if (c0 + cc >= nrhs) break;
        const double2 vf = v[i + (int64_t)(c0 + cc) * ldv];
        P[i + (int64_t)(c0 + cc) * ldp] = make_double2(kInv4PiP * (vf.x + acc[cc].x), kInv4PiP * (vf.y + acc[cc].y));
    }
}

static gyps_status potential_device(Mesh *m, double k, int64_t npts, const double *pts_dev, int nrhs, const double2 *X,
                                    int64_t ldx, double2 *P, int64_t ldp, int prec, cudaStream_t s)
{
    if (!m->d_tri_cen32) {
        if (!m->d_tri_cen) GYPS_CUDA(cudaMalloc((void **)&m->d_tri_cen, (size_t)m->nt * sizeof(double4_32a)));
        GYPS_CUDA(cudaMalloc((void **)&m->d_tri_cen32, (size_t)m->nt * sizeof(float4)));
        tri_center_kernel<<<(unsigned)((m->nt + 255) / 256), 256, 0, s>>>(m->d_vtx, m->d_tri, m->nt, m->d_tri_cen,
                                                                         m->d_tri_cen32);
        GYPS_CUDA(cudaGetLastError());
    }
    // workspace: float4 points, double4 points, v (npts x nrhs)
    const size_t b32 = ((size_t)npts * sizeof(float4) + 255) / 256 * 256;
    const size_t b64 = ((size_t)npts * sizeof(double4_32a) + 255) / 256 * 256;
    const size_t bv = (size_t)npts * nrhs * sizeof(double2);
    GYPS_TRY(grow(m, &m->ws_pts, &m->ws_pts_bytes, b32 + b64 + bv));
    unsigned char *ws = reinterpret_cast<unsigned char *>(m->ws_pts);
    float4 *p32 = reinterpret_cast<float4 *>(ws);
    double4_32a *p64 = reinterpret_cast<double4_32a *>(ws + b32);
    double2 *v = reinterpret_cast<double2 *>(ws + b32 + b64);
    point_prep_kernel<<<(unsigned)((npts + 255) / 256), 256, 0, s>>>(pts_dev, npts, p32, p64);
    GYPS_CUDA(cudaGetLastError());
    GYPS_TRY(far_points(m, k, X, ldx, nrhs, p32, p64, npts, v, npts, prec, s));
    constexpr int CH = 4;
    dim3 g((unsigned)((npts + 127) / 128), (unsigned)((nrhs + CH - 1) / CH));
    point_finish_kernel<CH><<<g, 128, 0, s>>>(m->d_vtx, m->d_tri, m->nt, m->d_pts64, m->rule, m->d_tri_cen,
                                              m->d_tri_cen32, p64, npts, v, npts, X, ldx, nrhs, P, ldp);
    GYPS_CUDA(cudaGetLastError());
    return GYPS_OK;
}

}  // namespace gyps

using namespace gyps;

extern "C" gyps_status gyps_sl_potential(gyps_mesh_t h, double k, int64_t npts, const double *pts, int nrhs,
                                         const void *X, int64_t ldx, void *P, int64_t ldp, int prec, void *stream)
{
    Mesh *m;
    GYPS_TRY(check_mesh(h, &m));
    if (npts < 0 || npts > ((int64_t)1 << 31)) return set_error(GYPS_ERR_INVALID, "npts must be in 0..2^31");
    if (nrhs < 1 || nrhs > 4096) return set_error(GYPS_ERR_INVALID, "nrhs must be in 1..4096");
    if (!X || (npts > 0 && (!pts || !P))) return set_error(GYPS_ERR_INVALID, "NULL argument");
    if (ldx < m->nv) return set_error(GYPS_ERR_INVALID, "ldx < nv");
    if (ldp < npts) return set_error(GYPS_ERR_INVALID, "ldp < npts");
    if (!std::isfinite(k) || k < 0.0) return set_error(GYPS_ERR_INVALID, "k must be finite and >= 0");
    if (prec == GYPS_PREC_AUTO) prec = GYPS_PREC_FP32;
    if (prec == GYPS_PREC_TC_BF16X3) return set_error(GYPS_ERR_UNSUPPORTED, "potential: FP64, FP32 or DF64");
    if (prec != GYPS_PREC_FP64 && prec != GYPS_PREC_FP32 && prec != GYPS_PREC_DF64)
        return set_error(GYPS_ERR_INVALID, "unknown precision");
    if (npts == 0) return GYPS_OK;
    cudaStream_t s = (cudaStream_t)stream;
    const bool dp = is_device_pointer(pts), dx = is_device_pointer(X), dP = is_device_pointer(P);
    if (!dp)
        for (int64_t i = 0; i < 3 * npts; ++i)
            if (!std::isfinite(pts[i])) return set_error(GYPS_ERR_INVALID, "non-finite point");
    // host arguments are staged in one device block: points, X, P
    const size_t bp = dp ? 0 : ((size_t)npts * 3 * sizeof(double) + 255) / 256 * 256;
    const size_t bx = dx ? 0 : ((size_t)m->nv * nrhs * sizeof(double2) + 255) / 256 * 256;
    const size_t bo = dP ? 0 : (size_t)npts * nrhs * sizeof(double2);
    unsigned char *st = nullptr;
    if (bp + bx + bo > 0) {
        GYPS_TRY(grow(m, &m->ws_stage, &m->ws_stage_bytes, bp + bx + bo));
        st = reinterpret_cast<unsigned char *>(m->ws_stage);
    }
    const double *pd = pts;
    if (!dp) {
        GYPS_CUDA(cudaMemcpyAsync(st, pts, (size_t)npts * 3 * sizeof(double), cudaMemcpyHostToDevice, s));
        pd = reinterpret_cast<const double *>(st);
    }
    const double2 *xd = (const double2 *)X;
    int64_t lxd = ldx;
    if (!dx) {
        double2 *xs = reinterpret_cast<double2 *>(st + bp);
        GYPS_CUDA(cudaMemcpy2DAsync(xs, m->nv * sizeof(double2), X, ldx * sizeof(double2), m->nv * sizeof(double2),
                                    nrhs, cudaMemcpyHostToDevice, s));
        xd = xs;
        lxd = m->nv;
    }
    double2 *pout = dP ? (double2 *)P : reinterpret_cast<double2 *>(st + bp + bx);
    const int64_t lpo = dP ? ldp : npts;
    GYPS_TRY(clear_err_word(m, s));  // report only the waits of this call's launches
    GYPS_TRY(potential_device(m, k, npts, pd, nrhs, xd, lxd, pout, lpo, prec, s));
    if (!dP)
        GYPS_CUDA(cudaMemcpy2DAsync(P, ldp * sizeof(double2), pout, npts * sizeof(double2), npts * sizeof(double2), nrhs,
                                    cudaMemcpyDeviceToHost, s));
    GYPS_CUDA(cudaStreamSynchronize(s));
    return check_err_word(m, s);
}
