// Dense assembly of the single layer (listing of Sec. 5.4: LHS = integral/(4pi) +
// regularize/(4pi)) and the plane-wave right-hand side (RHS = integral(S2, Vh, PW)).
#include <cmath>

#include "internal.h"

namespace gyps {

constexpr double kInv4PiA = 0.0795774715459476678844418816862571810;

// Kernel value exp(ik r)/r between two points in FP64.
__device__ __forceinline__ void kernel_value(double4_32a x, double4_32a y, double k, double &gr, double &gi)
{
    double dx = x.x - y.x, dy = x.y - y.y, dz = x.z - y.z;
    double r2 = dx * dx + dy * dy + dz * dz;
    double ri = rsqrt(r2);
    double sn, cs;
    sincos(k * (r2 * ri), &sn, &cs);
    gr = cs * ri;
    gi = sn * ri;
}

// a6, FP64: one thread per (test triangle a, trial triangle b); the 3x3 block
//   (1/4pi) sum_{k in a, l in b} w_k lambda_i(x_k) G(x_k, y_l) eta_l lambda_j(y_l)
// (G = ik for the point paired with itself) is added into V[v_i(a), v_j(b)].
// Threads of a CTA take consecutive test triangles and one trial triangle, so
// that the atomics of a warp fall into one column block of V.  Kernel values
// and sums in FP64 (this kernel is bound by the FP64 pipe).
__global__ void assemble_far64_kernel(const double4_32a *pts64, const int32_t *tri, const Rule rule, int64_t nt,
                                      double k, double2 *V, int64_t ldv)
{
    const int64_t a = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t b = blockIdx.y;
    if (a >= nt) return;
    const int q = rule.q;
    double br[9], bi[9];
#pragma unroll
    for (int e = 0; e < 9; ++e) br[e] = bi[e] = 0.0;
    for (int kq = 0; kq < q; ++kq) {
        const double4_32a x = pts64[a * q + kq];
        double sr[3] = {0.0, 0.0, 0.0}, si[3] = {0.0, 0.0, 0.0};  // sum_l G eta_l lambda_j(y_l)
        for (int lq = 0; lq < q; ++lq) {
            const double4_32a y = pts64[b * q + lq];
            double gr, gi;
            if (a == b && kq == lq) {
                gr = 0.0;
                gi = k;
            } else {
                kernel_value(x, y, k, gr, gi);
            }
#pragma unroll
            for (int j = 0; j < 3; ++j) {
                const double c = y.w * rule.bary[3 * lq + j];
                sr[j] += gr * c;
                si[j] += gi * c;
            }
        }
#pragma unroll
        for (int i = 0; i < 3; ++i) {
            const double c = x.w * rule.bary[3 * kq + i] * kInv4PiA;
#pragma unroll
            for (int j = 0; j < 3; ++j) {
                br[3 * i + j] += c * sr[j];
                bi[3 * i + j] += c * si[j];
            }
        }
    }
#pragma unroll
    for (int j = 0; j < 3; ++j) {
        const int64_t vj = tri[3 * b + j];
#pragma unroll
        for (int i = 0; i < 3; ++i) {
            double *dst = reinterpret_cast<double *>(V + tri[3 * a + i] + vj * ldv);
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
    if (prec == GYPS_PREC_FP32) {
        GYPS_TRY(assemble_tiles(m, k, V, ldv, s));  // writes every entry of V once
    } else {
        GYPS_CUDA(cudaMemset2DAsync(V, ldv * sizeof(double2), 0, m->nv * sizeof(double2), m->nv, s));
        dim3 g((unsigned)((m->nt + 127) / 128), (unsigned)m->nt);  // x: test triangles, y: trial triangle
        assemble_far64_kernel<<<g, 128, 0, s>>>(m->d_pts64, m->d_tri, m->rule, m->nt, k, V, ldv);
    }
    GYPS_CUDA(cudaGetLastError());
    assemble_near_kernel<<<(unsigned)((m->nv + 127) / 128), 128, 0, s>>>(m->d_c_rowptr, m->d_c_col, m->d_c_val, m->nv,
                                                                       V, ldv);
    GYPS_CUDA(cudaGetLastError());
    return GYPS_OK;
}

// a7: F_ij = sum_{k in supp phi_i} w_k lambda_i(x_k) exp(i k d_j . x_k).
// F_ij = sum_k w_k phi_i(x_k) g(x_k) with g = exp(ik d_j . x), or, for the direct
// combined-field system (cfie), g = (d/dn - i eta) exp(ik d_j . x)
// = i (k d_j . n - eta) exp(ik d_j . x), n the unit normal (P1 - P0) x (P2 - P0)/|.|.
__global__ void rhs_kernel(const int32_t *v2t_ptr, const int32_t *v2t, const double4_32a *pts64, const Rule rule,
                           int64_t nv, double k, const double *dirs, double2 *F, int64_t ldf, const double *vtx,
                           const int32_t *tri, int cfie, double eta)
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
        double a = 0.0;  // k d . n - eta
        if (cfie) {
            const double *p0 = vtx + 3 * tri[3 * t], *p1 = vtx + 3 * tri[3 * t + 1], *p2 = vtx + 3 * tri[3 * t + 2];
            const double ux = p1[0] - p0[0], uy = p1[1] - p0[1], uz = p1[2] - p0[2];
            const double vx = p2[0] - p0[0], vy = p2[1] - p0[1], vz = p2[2] - p0[2];
            const double nx = uy * vz - uz * vy, ny = uz * vx - ux * vz, nz = ux * vy - uy * vx;
            a = k * (dx * nx + dy * ny + dz * nz) / sqrt(nx * nx + ny * ny + nz * nz) - eta;
        }
        for (int kq = 0; kq < rule.q; ++kq) {
            double4_32a x = pts64[t * rule.q + kq];
            double sn, cs;
            sincos(k * (dx * x.x + dy * x.y + dz * x.z), &sn, &cs);
            double c = x.w * rule.bary[3 * kq + m];
            if (cfie) {  // i a (cs + i sn)
                fr -= c * a * sn;
                fi += c * a * cs;
            } else {
                fr += c * cs;
                fi += c * sn;
            }
        }
    }
    F[i + (int64_t)j * ldf] = make_double2(fr, fi);
}

gyps_status rhs_device(Mesh *m, double k, int nrhs, const double *dirs_host, double2 *F, int64_t ldf, cudaStream_t s,
                       bool cfie, double eta)
{
    double *d_dirs = nullptr;
    GYPS_CUDA(cudaMallocAsync((void **)&d_dirs, (size_t)nrhs * 3 * sizeof(double), s));
    GYPS_CUDA(cudaMemcpyAsync(d_dirs, dirs_host, (size_t)nrhs * 3 * sizeof(double), cudaMemcpyHostToDevice, s));
    dim3 g((unsigned)((m->nv + 127) / 128), (unsigned)nrhs);
    rhs_kernel<<<g, 128, 0, s>>>(m->d_v2t_ptr, m->d_v2t, m->d_pts64, m->rule, m->nv, k, d_dirs, F, ldf, m->d_vtx,
                                 m->d_tri, cfie ? 1 : 0, eta);
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
    if (prec == GYPS_PREC_FP64 && m->nt > 65535)
        return set_error(GYPS_ERR_UNSUPPORTED, "FP64 dense assembly limited to 65535 triangles");
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

static gyps_status rhs_entry(gyps_mesh_t h, double k, int nrhs, const double *dirs, void *F, int64_t ldf, void *stream,
                             bool cfie, double eta)
{
    Mesh *m;
    GYPS_TRY(check_mesh(h, &m));
    if (!F || !dirs) return set_error(GYPS_ERR_INVALID, "NULL argument");
    if (nrhs < 1 || nrhs > 4096) return set_error(GYPS_ERR_INVALID, "nrhs must be in 1..4096");
    if (ldf < m->nv) return set_error(GYPS_ERR_INVALID, "ldf < nv");
    if (!std::isfinite(k) || k < 0.0) return set_error(GYPS_ERR_INVALID, "k must be finite and >= 0");
    if (!std::isfinite(eta)) return set_error(GYPS_ERR_INVALID, "eta must be finite");
    for (int i = 0; i < 3 * nrhs; ++i)
        if (!std::isfinite(dirs[i])) return set_error(GYPS_ERR_INVALID, "non-finite direction");
    cudaStream_t s = (cudaStream_t)stream;
    if (is_device_pointer(F)) return rhs_device(m, k, nrhs, dirs, (double2 *)F, ldf, s, cfie, eta);
    const size_t bytes = (size_t)m->nv * nrhs * sizeof(double2);
    GYPS_TRY(grow(m, &m->ws_stage, &m->ws_stage_bytes, bytes));
    double2 *fd = reinterpret_cast<double2 *>(m->ws_stage);
    GYPS_TRY(rhs_device(m, k, nrhs, dirs, fd, m->nv, s, cfie, eta));
    GYPS_CUDA(cudaMemcpy2DAsync(F, ldf * sizeof(double2), fd, m->nv * sizeof(double2), m->nv * sizeof(double2), nrhs,
                                cudaMemcpyDeviceToHost, s));
    GYPS_CUDA(cudaStreamSynchronize(s));
    return GYPS_OK;
}

extern "C" gyps_status gyps_rhs_planewave(gyps_mesh_t h, double k, int nrhs, const double *dirs, void *F, int64_t ldf,
                                          void *stream)
{
    return rhs_entry(h, k, nrhs, dirs, F, ldf, stream, false, 0.0);
}

extern "C" gyps_status gyps_rhs_planewave_cfie(gyps_mesh_t h, double k, double eta, int nrhs, const double *dirs,
                                               void *F, int64_t ldf, void *stream)
{
    return rhs_entry(h, k, nrhs, dirs, F, ldf, stream, true, eta);
}
