// Dense assembly of the single layer (listing of Sec. 6.4: LHS = integral/(4pi) +
// regularize/(4pi)) and the plane-wave right-hand side (RHS = integral(S2, Vh, PW)).
#include <cmath>

#include "internal.h"

namespace gyps {

constexpr double kInv4PiA = 0.0795774715459476678844418816862571810;
constexpr double kTwoPiA = 6.283185307179586476925286766559;

__device__ __forceinline__ float mufu_rsqrt(float x)
{
    float y;
    asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}
__device__ __forceinline__ float mufu_sin(float x)
{
    float y;
    asm("sin.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}
__device__ __forceinline__ float mufu_cos(float x)
{
    float y;
    asm("cos.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

// Kernel value exp(ik r)/r between two points, FP64 or FP32 arithmetic.
template <bool FP64>
__device__ __forceinline__ void kernel_value(double4_32a x, double4_32a y, double k, double &gr, double &gi)
{
    if (FP64) {
        double dx = x.x - y.x, dy = x.y - y.y, dz = x.z - y.z;
        double r2 = dx * dx + dy * dy + dz * dz;
        double ri = rsqrt(r2);
        double sn, cs;
        sincos(k * (r2 * ri), &sn, &cs);
        gr = cs * ri;
        gi = sn * ri;
    } else {
        float dx = (float)x.x - (float)y.x, dy = (float)x.y - (float)y.y, dz = (float)x.z - (float)y.z;
        float r2 = dx * dx + dy * dy + dz * dz;
        float rs = mufu_rsqrt(r2);
        float t = r2 * rs * (float)(k / kTwoPiA);
        float f = t - rintf(t);
        float ang = f * 6.28318530717958647692f;
        gr = (double)(mufu_cos(ang) * rs);
        gi = (double)(mufu_sin(ang) * rs);
    }
}

// a6: one thread per (test triangle a, trial triangle b); the 3x3 block
//   (1/4pi) sum_{k in a, l in b} w_k lambda_i(x_k) G(x_k, y_l) eta_l lambda_j(y_l)
// (G = ik for the point paired with itself) is added into V[v_i(a), v_j(b)].
template <bool FP64>
__global__ void assemble_far_kernel(const double4_32a *pts64, const int32_t *tri, const Rule rule, int64_t nt, double k,
                                    double2 *V, int64_t ldv)
{
    const int64_t b = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t a = blockIdx.y;
    if (b >= nt) return;
    const int q = rule.q;
    double br[9], bi[9];
#pragma unroll
    for (int e = 0; e < 9; ++e) br[e] = bi[e] = 0.0;
    for (int kq = 0; kq < q; ++kq) {
        double4_32a x = pts64[a * q + kq];
        double sr[3] = {0.0, 0.0, 0.0}, si[3] = {0.0, 0.0, 0.0};  // sum_l G eta_l lambda_j(y_l)
        for (int lq = 0; lq < q; ++lq) {
            double4_32a y = pts64[b * q + lq];
            double gr, gi;
            if (a == b && kq == lq) {
                gr = 0.0;
                gi = k;
            } else {
                kernel_value<FP64>(x, y, k, gr, gi);
            }
            for (int j = 0; j < 3; ++j) {
                double c = y.w * rule.bary[3 * lq + j];
                sr[j] += gr * c;
                si[j] += gi * c;
            }
        }
        for (int i = 0; i < 3; ++i) {
            double c = x.w * rule.bary[3 * kq + i] * kInv4PiA;
            for (int j = 0; j < 3; ++j) {
                br[3 * i + j] += c * sr[j];
                bi[3 * i + j] += c * si[j];
            }
        }
    }
    for (int i = 0; i < 3; ++i) {
        int64_t vi = tri[3 * a + i];
        for (int j = 0; j < 3; ++j) {
            int64_t vj = tri[3 * b + j];
            double *dst = reinterpret_cast<double *>(V + vi + vj * ldv);
            atomicAdd(dst, br[3 * i + j]);
            atomicAdd(dst + 1, bi[3 * i + j]);
        }
    }
}

// V[i, c] += C_ic (each nonzero once: no atomics needed).
__global__ void assemble_near_kernel(const int32_t *rowptr, const int32_t *col, const double *val, int64_t nv,
                                     double2 *V, int64_t ldv)
{
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nv) return;
    for (int32_t c = rowptr[i]; c < rowptr[i + 1]; ++c) V[i + (int64_t)col[c] * ldv].x += val[c];
}

gyps_status assemble_device(Mesh *m, double k, int prec, double2 *V, int64_t ldv, cudaStream_t s)
{
    GYPS_CUDA(cudaMemset2DAsync(V, ldv * sizeof(double2), 0, m->nv * sizeof(double2), m->nv, s));
    dim3 g((unsigned)((m->nt + 127) / 128), (unsigned)m->nt);
    if (prec == GYPS_PREC_FP64)
        assemble_far_kernel<true><<<g, 128, 0, s>>>(m->d_pts64, m->d_tri, m->rule, m->nt, k, V, ldv);
    else
        assemble_far_kernel<false><<<g, 128, 0, s>>>(m->d_pts64, m->d_tri, m->rule, m->nt, k, V, ldv);
    GYPS_CUDA(cudaGetLastError());
    assemble_near_kernel<<<(unsigned)((m->nv + 127) / 128), 128, 0, s>>>(m->d_c_rowptr, m->d_c_col, m->d_c_val, m->nv,
                                                                       V, ldv);
    GYPS_CUDA(cudaGetLastError());
    return GYPS_OK;
}

// a7: F_ij = sum_{k in supp phi_i} w_k lambda_i(x_k) exp(i k d_j . x_k).
__global__ void rhs_kernel(const int32_t *v2t_ptr, const int32_t *v2t, const double4_32a *pts64, const Rule rule,
                           int64_t nv, double k, const double *dirs, double2 *F, int64_t ldf)
{
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    int j = blockIdx.y;
    if (i >= nv) return;
    const double dx = dirs[3 * j], dy = dirs[3 * j + 1], dz = dirs[3 * j + 2];
    double fr = 0.0, fi = 0.0;
    for (int32_t e = v2t_ptr[i]; e < v2t_ptr[i + 1]; ++e) {
        int32_t te = v2t[e];
        int64_t t = te / 3;
        int m = te - 3 * (int)t;
        for (int kq = 0; kq < rule.q; ++kq) {
            double4_32a x = pts64[t * rule.q + kq];
            double sn, cs;
            sincos(k * (dx * x.x + dy * x.y + dz * x.z), &sn, &cs);
            double c = x.w * rule.bary[3 * kq + m];
            fr += c * cs;
            fi += c * sn;
        }
    }
    F[i + (int64_t)j * ldf] = make_double2(fr, fi);
}

gyps_status rhs_device(Mesh *m, double k, int nrhs, const double *dirs_host, double2 *F, int64_t ldf, cudaStream_t s)
{
    double *d_dirs = nullptr;
    GYPS_CUDA(cudaMallocAsync((void **)&d_dirs, (size_t)nrhs * 3 * sizeof(double), s));
    GYPS_CUDA(cudaMemcpyAsync(d_dirs, dirs_host, (size_t)nrhs * 3 * sizeof(double), cudaMemcpyHostToDevice, s));
    dim3 g((unsigned)((m->nv + 127) / 128), (unsigned)nrhs);
    rhs_kernel<<<g, 128, 0, s>>>(m->d_v2t_ptr, m->d_v2t, m->d_pts64, m->rule, m->nv, k, d_dirs, F, ldf);
    cudaError_t e = cudaGetLastError();
    cudaFreeAsync(d_dirs, s);
    GYPS_CUDA(e);
    return GYPS_OK;
}

}  // namespace gyps

using namespace gyps;

extern "C" gyps_status gyps_sl_assemble(gyps_mesh_t h, double k, int prec, void *V, int64_t ldv, void *stream)
{
    Mesh *m;
    GYPS_TRY(check_mesh(h, &m));
    if (!V) return set_error(GYPS_ERR_INVALID, "V is NULL");
    if (ldv < m->nv) return set_error(GYPS_ERR_INVALID, "ldv < nv");
    if (!std::isfinite(k) || k < 0.0) return set_error(GYPS_ERR_INVALID, "k must be finite and >= 0");
    if (prec != GYPS_PREC_FP64 && prec != GYPS_PREC_FP32)
        return set_error(GYPS_ERR_UNSUPPORTED, "dense assembly supports FP64 and FP32");
    if (m->nt > 65535) return set_error(GYPS_ERR_UNSUPPORTED, "dense assembly limited to 65535 triangles");
    cudaStream_t s = (cudaStream_t)stream;
    if (is_device_pointer(V)) return assemble_device(m, k, prec, (double2 *)V, ldv, s);
    const size_t bytes = (size_t)m->nv * m->nv * sizeof(double2);
    GYPS_TRY(grow(m, &m->ws_stage, &m->ws_stage_bytes, bytes));
    double2 *vd = reinterpret_cast<double2 *>(m->ws_stage);
    GYPS_TRY(assemble_device(m, k, prec, vd, m->nv, s));
    GYPS_CUDA(cudaMemcpy2DAsync(V, ldv * sizeof(double2), vd, m->nv * sizeof(double2), m->nv * sizeof(double2), m->nv,
                                cudaMemcpyDeviceToHost, s));
    GYPS_CUDA(cudaStreamSynchronize(s));
    return GYPS_OK;
}

extern "C" gyps_status gyps_rhs_planewave(gyps_mesh_t h, double k, int nrhs, const double *dirs, void *F, int64_t ldf,
                                          void *stream)
{
    Mesh *m;
    GYPS_TRY(check_mesh(h, &m));
    if (!F || !dirs) return set_error(GYPS_ERR_INVALID, "NULL argument");
    if (nrhs < 1 || nrhs > 4096) return set_error(GYPS_ERR_INVALID, "nrhs must be in 1..4096");
    if (ldf < m->nv) return set_error(GYPS_ERR_INVALID, "ldf < nv");
    if (!std::isfinite(k) || k < 0.0) return set_error(GYPS_ERR_INVALID, "k must be finite and >= 0");
    for (int i = 0; i < 3 * nrhs; ++i)
        if (!std::isfinite(dirs[i])) return set_error(GYPS_ERR_INVALID, "non-finite direction");
    cudaStream_t s = (cudaStream_t)stream;
    if (is_device_pointer(F)) return rhs_device(m, k, nrhs, dirs, (double2 *)F, ldf, s);
    const size_t bytes = (size_t)m->nv * nrhs * sizeof(double2);
    GYPS_TRY(grow(m, &m->ws_stage, &m->ws_stage_bytes, bytes));
    double2 *fd = reinterpret_cast<double2 *>(m->ws_stage);
    GYPS_TRY(rhs_device(m, k, nrhs, dirs, fd, m->nv, s));
    GYPS_CUDA(cudaMemcpy2DAsync(F, ldf * sizeof(double2), fd, m->nv * sizeof(double2), m->nv * sizeof(double2), nrhs,
                                cudaMemcpyDeviceToHost, s));
    GYPS_CUDA(cudaStreamSynchronize(s));
    return GYPS_OK;
}
