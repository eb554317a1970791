// Galerkin double layer (the operator after the single layer; the paper's
// grady[exp(ikr)/r] kernel with the 'grady[1/r]' regularisation, Sec. 5.2),
//   K = (1/4pi) Phi^T W H W Phi + C_dl,
//   H(x, y) = n_y . grad_y exp(ik|x-y|)/|x-y| = (1 - i k r) exp(i k r) n_y . (x - y) / r^3,
// in the single layer's factorisation: the same interpolation and projection,
// the kernel H between the Gauss points (n_y: unit normal of the source
// triangle; the point paired with itself, like every pair inside one flat
// triangle, gives 0), and on pairs of triangles sharing a vertex the
// correction: closed-form y-integral of lambda_j n . (x - y)/|x - y|^3 minus
// its Gauss sum.
#include <cmath>

#include "internal.h"
#include "p1_geom.cuh"

namespace gyps {

__global__ void interp64_kernel(const int32_t *tri, const double4_32a *pts64, const Rule rule, int64_t nq, int64_t ld,
                                const double2 *X, int64_t ldx, int nrhs, double2 *u64);
__global__ void project_kernel(const int32_t *v2t_ptr, const int32_t *v2t, const double4_32a *pts64, const Rule rule,
                               int64_t nv, const double2 *v, int64_t ldv, const int32_t *c_rowptr,
                               const int32_t *c_col, const double *c_val, const double2 *X, int64_t ldx, double2 *Y,
                               int64_t ldy, int with_near);
__global__ void near_gather_kernel(int64_t nnz, const int32_t *src_ptr, const int32_t *src, const double *blocks,
                                   double *val);

constexpr double kInv4PiD = 0.0795774715459476678844418816862571810;

// Unit normal of each triangle, (P1 - P0) x (P2 - P0) / |.|.
__global__ void tri_normal_kernel(const double *vtx, const int32_t *tri, int64_t nt, double4_32a *nrm)
{
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= nt) return;
    const double3 p0 = ld3(vtx, tri[3 * t]), p1 = ld3(vtx, tri[3 * t + 1]), p2 = ld3(vtx, tri[3 * t + 2]);
    const double3 n = cross(p1 - p0, p2 - p0);
    const double s = 1.0 / sqrt(dot(n, n));
    nrm[t] = make_double4_32a(s * n.x, s * n.y, s * n.z, 0.0);
}

// Correction block of the double layer on the near pair (a, b):
//   (1/4pi) sum_k w_k lambda_i(x_k) (I_j(x_k, b) - sum_l eta_l lambda_j(y_l) n_b . (x_k - y_l)/r^3),
// 0 for a == b (coplanar).
__global__ void dl_near_blocks_kernel(const double *vtx, const int32_t *tri, const double4_32a *pts64, const Rule rule,
                                      const double4_32a *nrm, int64_t npairs, const int32_t *pair_a,
                                      const int32_t *pair_b, double *blocks)
{
    const int q = rule.q;
    const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= npairs) return;
    const int a = pair_a[p], b = pair_b[p];
    double acc[9];
#pragma unroll
    for (int e = 0; e < 9; ++e) acc[e] = 0.0;
    if (a != b) {
        const double3 B[3] = {ld3(vtx, tri[3 * (int64_t)b]), ld3(vtx, tri[3 * (int64_t)b + 1]),
                              ld3(vtx, tri[3 * (int64_t)b + 2])};
        const double4_32a nb4 = nrm[b];
        const double3 nb = make_double3(nb4.x, nb4.y, nb4.z);
        for (int kq = 0; kq < q; ++kq) {
            const double4_32a xk4 = pts64[(int64_t)a * q + kq];
            const double3 xk = make_double3(xk4.x, xk4.y, xk4.z);
            double exact[3];
            p1_dn_over_r(xk, B, exact);
            for (int lq = 0; lq < q; ++lq) {
                const double4_32a yl = pts64[(int64_t)b * q + lq];
                const double3 d = make_double3(xk.x - yl.x, xk.y - yl.y, xk.z - yl.z);
                const double r2 = dot(d, d);
                const double f = yl.w * dot(nb, d) / (r2 * sqrt(r2));
#pragma unroll
                for (int j = 0; j < 3; ++j) exact[j] -= f * rule.bary[3 * lq + j];
            }
            const double wk = xk4.w * kInv4PiD;
#pragma unroll
            for (int i = 0; i < 3; ++i)
#pragma unroll
                for (int j = 0; j < 3; ++j) acc[3 * i + j] += wk * rule.bary[3 * kq + i] * exact[j];
        }
    }
#pragma unroll
    for (int e = 0; e < 9; ++e) blocks[9 * p + e] = acc[e];
}

// v[t, c0 + j] = sum_l H(x_t, y_l) u[l, c0 + j] in FP64 (plain form).
template <int R>
__global__ void __launch_bounds__(128) far_dl64_kernel(const double4_32a *pts, const double4_32a *nrm, int q,
                                                       const double2 *u64, int64_t ldu, int c0, int64_t nq, double k,
                                                       double2 *v, int64_t ldv)
{
    __shared__ double4_32a sp[128];
    __shared__ double4_32a sn[128];
    __shared__ double2 su[128][R];
    const int64_t tg = (int64_t)blockIdx.x * 128 + threadIdx.x;
    const double4_32a x = pts[min(tg, nq - 1)];
    double ar[R], ai[R];
#pragma unroll
    for (int j = 0; j < R; ++j) ar[j] = ai[j] = 0.0;
    for (int64_t s0 = 0; s0 < nq; s0 += 128) {
        const int64_t l = s0 + threadIdx.x;
        if (l < nq) {
            sp[threadIdx.x] = pts[l];
            sn[threadIdx.x] = nrm[l / q];
#pragma unroll
            for (int j = 0; j < R; ++j) su[threadIdx.x][j] = u64[l + (int64_t)(c0 + j) * ldu];
        }
        __syncthreads();
        const int n = (int)min((int64_t)128, nq - s0);
        for (int ll = 0; ll < n; ++ll) {
            if ((s0 + ll) / q == tg / q) continue;  // same flat triangle: n . (x - y) = 0
            const double4_32a y = sp[ll], nn = sn[ll];
            const double dx = x.x - y.x, dy = x.y - y.y, dz = x.z - y.z;
            const double r2 = dx * dx + dy * dy + dz * dz;
            const double ri = rsqrt(r2);
            const double f = (nn.x * dx + nn.y * dy + nn.z * dz) * ri * ri * ri;
            const double kr = k * (r2 * ri);
            double s, c;
            sincos(kr, &s, &c);
            const double hr = (c + kr * s) * f, hi = (s - kr * c) * f;
#pragma unroll
            for (int j = 0; j < R; ++j) {
                const double2 uu = su[ll][j];
                ar[j] += hr * uu.x - hi * uu.y;
                ai[j] += hr * uu.y + hi * uu.x;
            }
        }
        __syncthreads();
    }
    if (tg < nq) {
#pragma unroll
        for (int j = 0; j < R; ++j) v[tg + (int64_t)(c0 + j) * ldv] = make_double2(ar[j], ai[j]);
    }
}

__device__ __forceinline__ float mufu_rsqrt_dl(float x)
{
    float y;
    asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}
__device__ __forceinline__ float mufu_sin_dl(float x)
{
    float y;
    asm("sin.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}
__device__ __forceinline__ float mufu_cos_dl(float x)
{
    float y;
    asm("cos.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

// The same in FP32: coordinates scaled by k (k r = r2 rs; unscaled with phase 0
// for the Laplace kernel), phase reduced to
// [-pi, pi] by the nearest multiple of 2 pi, MUFU rsqrt / sin / cos; the
// factor k^2 of n . (x - y) / r^3 under the scaling is applied at the end.
// Per tile of 128 sources the FP32 sums are added into FP64 accumulators.
template <int R>
__global__ void __launch_bounds__(128) far_dl32_kernel(const double4_32a *pts, const double4_32a *nrm, int q,
                                                       const double2 *u64, int64_t ldu, int c0, int64_t nq, float ks,
                                                       float kfac, double2 *v, int64_t ldv)
{
    __shared__ float4 sp[128];      // (x, y, z) k
    __shared__ float4 sn[128];      // normal
    __shared__ float2 su[128][R];
    const int64_t tg = (int64_t)blockIdx.x * 128 + threadIdx.x;
    const double4_32a x64 = pts[min(tg, nq - 1)];
    const float tx = (float)x64.x * ks, ty = (float)x64.y * ks, tz = (float)x64.z * ks;
    double ar[R], ai[R];
#pragma unroll
    for (int j = 0; j < R; ++j) ar[j] = ai[j] = 0.0;
    for (int64_t s0 = 0; s0 < nq; s0 += 128) {
        const int64_t l = s0 + threadIdx.x;
        if (l < nq) {
            const double4_32a p = pts[l];
            const double4_32a nn = nrm[l / q];
            sp[threadIdx.x] = make_float4((float)p.x * ks, (float)p.y * ks, (float)p.z * ks, 0.0f);
            sn[threadIdx.x] = make_float4((float)nn.x, (float)nn.y, (float)nn.z, 0.0f);
#pragma unroll
            for (int j = 0; j < R; ++j) {
                const double2 uu = u64[l + (int64_t)(c0 + j) * ldu];
                su[threadIdx.x][j] = make_float2((float)uu.x, (float)uu.y);
            }
        }
        __syncthreads();
        const int n = (int)min((int64_t)128, nq - s0);
        float br[R], bi[R];
#pragma unroll
        for (int j = 0; j < R; ++j) br[j] = bi[j] = 0.0f;
        for (int ll = 0; ll < n; ++ll) {
            if ((s0 + ll) / q == tg / q) continue;  // same flat triangle: n . (x - y) = 0
            const float4 y = sp[ll], nn = sn[ll];
            const float dx = tx - y.x, dy = ty - y.y, dz = tz - y.z;
            const float r2 = dx * dx + dy * dy + dz * dz;
            const float rs = mufu_rsqrt_dl(r2);
            const float kr = kfac * (r2 * rs);  // k r (0 for the Laplace kernel)
            const float nr = rintf(kr * 0.159154943091895335769f);
            const float ang = fmaf(nr, -6.28318530717958647692f, kr);
            const float s = mufu_sin_dl(ang), c = mufu_cos_dl(ang);
            const float f = (nn.x * dx + nn.y * dy + nn.z * dz) * rs * rs * rs;
            const float hr = (c + kr * s) * f, hi = (s - kr * c) * f;
#pragma unroll
            for (int j = 0; j < R; ++j) {
                const float2 uu = su[ll][j];
                br[j] = fmaf(hr, uu.x, fmaf(-hi, uu.y, br[j]));
                bi[j] = fmaf(hr, uu.y, fmaf(hi, uu.x, bi[j]));
            }
        }
#pragma unroll
        for (int j = 0; j < R; ++j) {
            ar[j] += (double)br[j];
            ai[j] += (double)bi[j];
        }
        __syncthreads();
    }
    if (tg < nq) {
        const double k2 = (double)ks * (double)ks;
#pragma unroll
        for (int j = 0; j < R; ++j) v[tg + (int64_t)(c0 + j) * ldv] = make_double2(ar[j] * k2, ai[j] * k2);
    }
}

// Normals and the double-layer correction values (CSR of C), once per mesh.
static gyps_status dl_prepare(Mesh *m, cudaStream_t s)
{
    if (m->d_cdl_val) return GYPS_OK;
    GYPS_CUDA(cudaMalloc((void **)&m->d_tri_nrm, (size_t)m->nt * sizeof(double4_32a)));
    tri_normal_kernel<<<(unsigned)((m->nt + 255) / 256), 256, 0, s>>>(m->d_vtx, m->d_tri, m->nt, m->d_tri_nrm);
    GYPS_CUDA(cudaGetLastError());
    double *blocks = nullptr;
    GYPS_CUDA(cudaMallocAsync((void **)&blocks, (size_t)m->npairs * 9 * sizeof(double), s));
    dl_near_blocks_kernel<<<(unsigned)((m->npairs + 127) / 128), 128, 0, s>>>(
        m->d_vtx, m->d_tri, m->d_pts64, m->rule, m->d_tri_nrm, m->npairs, m->d_pair_a, m->d_pair_b, blocks);
    cudaError_t e = cudaGetLastError();
    double *val = nullptr;
    if (e == cudaSuccess) e = cudaMalloc((void **)&val, (size_t)m->c_nnz * sizeof(double));
    if (e == cudaSuccess) {
        near_gather_kernel<<<(unsigned)((m->c_nnz + 255) / 256), 256, 0, s>>>(m->c_nnz, m->d_c_src_ptr, m->d_c_src,
                                                                             blocks, val);
        e = cudaGetLastError();
    }
    cudaFreeAsync(blocks, s);
    if (e != cudaSuccess) {
        if (val) cudaFree(val);
        return cuda_error(e, "double-layer correction");
    }
    GYPS_CUDA(cudaStreamSynchronize(s));
    m->d_cdl_val = val;
    return GYPS_OK;
}

gyps_status dl_apply_device(Mesh *m, double k, int nrhs, const double2 *X, int64_t ldx, double2 *Y, int64_t ldy,
                                   int prec, cudaStream_t s)
{
    GYPS_TRY(dl_prepare(m, s));
    const int64_t ld = m->nq;
    GYPS_TRY(grow(m, &m->ws_den, &m->ws_den_bytes, (size_t)(ld * nrhs) * sizeof(double2)));
    GYPS_TRY(grow(m, &m->ws_v, &m->ws_v_bytes, (size_t)(ld * nrhs) * sizeof(double2)));
    double2 *u64 = reinterpret_cast<double2 *>(m->ws_den);
    double2 *v = reinterpret_cast<double2 *>(m->ws_v);
    dim3 gi((unsigned)((m->nq + 255) / 256), (unsigned)nrhs);
    interp64_kernel<<<gi, 256, 0, s>>>(m->d_tri, m->d_pts64, m->rule, m->nq, ld, X, ldx, nrhs, u64);
    GYPS_CUDA(cudaGetLastError());
    const unsigned grid = (unsigned)((m->nq + 127) / 128);
    for (int c0 = 0; c0 < nrhs;) {
        const int w = nrhs - c0 >= 4 ? 4 : nrhs - c0 >= 2 ? 2 : 1;
        if (prec == GYPS_PREC_FP64) {
            if (w == 4) far_dl64_kernel<4><<<grid, 128, 0, s>>>(m->d_pts64, m->d_tri_nrm, m->q, u64, ld, c0, m->nq, k, v, ld);
            else if (w == 2) far_dl64_kernel<2><<<grid, 128, 0, s>>>(m->d_pts64, m->d_tri_nrm, m->q, u64, ld, c0, m->nq, k, v, ld);
            else far_dl64_kernel<1><<<grid, 128, 0, s>>>(m->d_pts64, m->d_tri_nrm, m->q, u64, ld, c0, m->nq, k, v, ld);
        } else {
            // coordinates scaled by k (1 for the Laplace kernel, where the phase is 0)
            const float ks = k > 0.0 ? (float)k : 1.0f, kfac = k > 0.0 ? 1.0f : 0.0f;
            if (w == 4) far_dl32_kernel<4><<<grid, 128, 0, s>>>(m->d_pts64, m->d_tri_nrm, m->q, u64, ld, c0, m->nq, ks, kfac, v, ld);
            else if (w == 2) far_dl32_kernel<2><<<grid, 128, 0, s>>>(m->d_pts64, m->d_tri_nrm, m->q, u64, ld, c0, m->nq, ks, kfac, v, ld);
            else far_dl32_kernel<1><<<grid, 128, 0, s>>>(m->d_pts64, m->d_tri_nrm, m->q, u64, ld, c0, m->nq, ks, kfac, v, ld);
        }
        GYPS_CUDA(cudaGetLastError());
        c0 += w;
    }
    dim3 gp((unsigned)((m->nv + 127) / 128), (unsigned)nrhs);
    project_kernel<<<gp, 128, 0, s>>>(m->d_v2t_ptr, m->d_v2t, m->d_pts64, m->rule, m->nv, v, ld, m->d_c_rowptr,
                                      m->d_c_col, m->d_cdl_val, X, ldx, Y, ldy, 1);
    GYPS_CUDA(cudaGetLastError());
    return GYPS_OK;
}

// Combined operator of the indirect Brakhage-Werner formulation: u = (D - i eta S) phi
// outside the surface; the exterior trace (1/2 + K - i eta V) phi = -u_inc holds on it
// (jump of the double-layer potential), in Galerkin form with the mass matrix
// M = Phi^T W Phi of Eq. (A=BWB).  Y holds V X on entry and T holds K X:
//   Y = 1/2 Phi^T W Phi X + T - i eta Y.
__global__ void bw_combine_kernel(const int32_t *v2t_ptr, const int32_t *v2t, const int32_t *tri,
                                  const double4_32a *pts64, const Rule rule, int64_t nv, const double2 *X,
                                  int64_t ldx, const double2 *T, int64_t ldt, double eta, double2 *Y, int64_t ldy)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t c = blockIdx.y;
    if (i >= nv) return;
    const double2 *xc = X + c * ldx;
    const int q = rule.q;
    double mr = 0.0, mi = 0.0;
    for (int32_t e = v2t_ptr[i]; e < v2t_ptr[i + 1]; ++e) {
        const int32_t te = v2t[e];
        const int64_t t = te / 3;
        const int corner = te - 3 * (int)t;
        const double2 x0 = xc[tri[3 * t]], x1 = xc[tri[3 * t + 1]], x2 = xc[tri[3 * t + 2]];
        for (int l = 0; l < q; ++l) {
            const double *b = rule.bary + 3 * l;
            const double wb = pts64[t * q + l].w * b[corner];
            mr += wb * (b[0] * x0.x + b[1] * x1.x + b[2] * x2.x);
            mi += wb * (b[0] * x0.y + b[1] * x1.y + b[2] * x2.y);
        }
    }
    const double2 kx = T[i + c * ldt];
    const double2 vx = Y[i + c * ldy];
    Y[i + c * ldy] = make_double2(0.5 * mr + kx.x + eta * vx.y, 0.5 * mi + kx.y - eta * vx.x);
}

// Y = (1/2 M + K - i eta V) X.  V in prec; K in FP64 for the FP64 and
// double-float precisions, in FP32 otherwise.
gyps_status bw_apply_device(Mesh *m, double k, double eta, int nrhs, const double2 *X, int64_t ldx, double2 *Y,
                            int64_t ldy, int prec, cudaStream_t s)
{
    GYPS_TRY(grow(m, &m->ws_bw, &m->ws_bw_bytes, (size_t)m->nv * nrhs * sizeof(double2)));
    double2 *T = reinterpret_cast<double2 *>(m->ws_bw);
    const int kprec = (prec == GYPS_PREC_FP64 || prec == GYPS_PREC_DF64) ? GYPS_PREC_FP64 : GYPS_PREC_FP32;
    GYPS_TRY(dl_apply_device(m, k, nrhs, X, ldx, T, m->nv, kprec, s));
    GYPS_TRY(apply_device(m, k, nrhs, X, ldx, Y, ldy, prec, 0, 0, m->nt, s));
    dim3 g((unsigned)((m->nv + 127) / 128), (unsigned)nrhs);
    bw_combine_kernel<<<g, 128, 0, s>>>(m->d_v2t_ptr, m->d_v2t, m->d_tri, m->d_pts64, m->rule, m->nv, X, ldx, T, m->nv,
                                        eta, Y, ldy);
    GYPS_CUDA(cudaGetLastError());
    return GYPS_OK;
}

}  // namespace gyps

using namespace gyps;

extern "C" gyps_status gyps_dl_apply(gyps_mesh_t h, double k, int nrhs, const void *X, int64_t ldx, void *Y,
                                     int64_t ldy, int prec, void *stream)
{
    Mesh *m;
    GYPS_TRY(check_mesh(h, &m));
    if (nrhs < 1 || nrhs > 4096) return set_error(GYPS_ERR_INVALID, "nrhs must be in 1..4096");
    if (!X || !Y) return set_error(GYPS_ERR_INVALID, "NULL argument");
    if (ldx < m->nv || ldy < m->nv) return set_error(GYPS_ERR_INVALID, "leading dimension < nv");
    if (!std::isfinite(k) || k < 0.0) return set_error(GYPS_ERR_INVALID, "k must be finite and >= 0");
    if (prec == GYPS_PREC_AUTO) prec = GYPS_PREC_FP32;
    if (prec == GYPS_PREC_TC_BF16X3 || prec == GYPS_PREC_DF64)
        return set_error(GYPS_ERR_UNSUPPORTED, "double layer: FP64 or FP32");
    if (prec != GYPS_PREC_FP64 && prec != GYPS_PREC_FP32) return set_error(GYPS_ERR_INVALID, "unknown precision");
    cudaStream_t s = (cudaStream_t)stream;
    const bool dx = is_device_pointer(X), dy = is_device_pointer(Y);
    const size_t blk = (size_t)m->nv * nrhs * sizeof(double2);
    double2 *xs = nullptr, *ys = nullptr;
    if (!dx || !dy) {
        GYPS_TRY(grow(m, &m->ws_stage, &m->ws_stage_bytes, 2 * blk));
        xs = reinterpret_cast<double2 *>(m->ws_stage);
        ys = xs + (size_t)m->nv * nrhs;
    }
    const double2 *xin = (const double2 *)X;
    int64_t lxin = ldx;
    if (!dx) {
        GYPS_CUDA(cudaMemcpy2DAsync(xs, m->nv * sizeof(double2), X, ldx * sizeof(double2), m->nv * sizeof(double2), nrhs,
                                    cudaMemcpyHostToDevice, s));
        xin = xs;
        lxin = m->nv;
    }
    double2 *yout = dy ? (double2 *)Y : ys;
    const int64_t lyout = dy ? ldy : m->nv;
    GYPS_TRY(dl_apply_device(m, k, nrhs, xin, lxin, yout, lyout, prec, s));
    if (!dy)
        GYPS_CUDA(cudaMemcpy2DAsync(Y, ldy * sizeof(double2), ys, m->nv * sizeof(double2), m->nv * sizeof(double2), nrhs,
                                    cudaMemcpyDeviceToHost, s));
    GYPS_CUDA(cudaStreamSynchronize(s));
    return GYPS_OK;
}

extern "C" gyps_status gyps_bw_apply(gyps_mesh_t h, double k, double eta, int nrhs, const void *X, int64_t ldx,
                                     void *Y, int64_t ldy, int prec, void *stream)
{
    Mesh *m;
    GYPS_TRY(check_mesh(h, &m));
    if (nrhs < 1 || nrhs > 4096) return set_error(GYPS_ERR_INVALID, "nrhs must be in 1..4096");
    if (!X || !Y) return set_error(GYPS_ERR_INVALID, "NULL argument");
    if (ldx < m->nv || ldy < m->nv) return set_error(GYPS_ERR_INVALID, "leading dimension < nv");
    if (!std::isfinite(k) || k < 0.0) return set_error(GYPS_ERR_INVALID, "k must be finite and >= 0");
    if (!std::isfinite(eta)) return set_error(GYPS_ERR_INVALID, "eta must be finite");
    if (prec == GYPS_PREC_AUTO) prec = GYPS_PREC_FP32;
    if (prec != GYPS_PREC_FP64 && prec != GYPS_PREC_FP32 && prec != GYPS_PREC_TC_BF16X3 && prec != GYPS_PREC_DF64)
        return set_error(GYPS_ERR_INVALID, "unknown precision");
    if (prec == GYPS_PREC_TC_BF16X3 && nrhs < 16)
        return set_error(GYPS_ERR_UNSUPPORTED, "tensor-core precision needs 16 or more right-hand sides");
    cudaStream_t s = (cudaStream_t)stream;
    const bool dx = is_device_pointer(X), dy = is_device_pointer(Y);
    if (dx && dy && (const char *)X < (const char *)Y + ldy * nrhs * 16 &&
        (const char *)Y < (const char *)X + ldx * nrhs * 16)
        return set_error(GYPS_ERR_INVALID, "X and Y overlap");
    const size_t blk = (size_t)m->nv * nrhs * sizeof(double2);
    double2 *xs = nullptr, *ys = nullptr;
    if (!dx || !dy) {
        GYPS_TRY(grow(m, &m->ws_stage, &m->ws_stage_bytes, 2 * blk));
        xs = reinterpret_cast<double2 *>(m->ws_stage);
        ys = xs + (size_t)m->nv * nrhs;
    }
    const double2 *xin = (const double2 *)X;
    int64_t lxin = ldx;
    if (!dx) {
        GYPS_CUDA(cudaMemcpy2DAsync(xs, m->nv * sizeof(double2), X, ldx * sizeof(double2), m->nv * sizeof(double2), nrhs,
                                    cudaMemcpyHostToDevice, s));
        xin = xs;
        lxin = m->nv;
    }
    double2 *yout = dy ? (double2 *)Y : ys;
    const int64_t lyout = dy ? ldy : m->nv;
    GYPS_TRY(bw_apply_device(m, k, eta, nrhs, xin, lxin, yout, lyout, prec, s));
    if (!dy)
        GYPS_CUDA(cudaMemcpy2DAsync(Y, ldy * sizeof(double2), ys, m->nv * sizeof(double2), m->nv * sizeof(double2), nrhs,
                                    cudaMemcpyDeviceToHost, s));
    GYPS_CUDA(cudaStreamSynchronize(s));
    return check_err_word(m, s);
}
