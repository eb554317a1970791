// EFIE with RWG functions (the electromagnetic listing of Sec. 5.5):
//   T = ik/(4pi) int int phi_m . phi_n G - i/(4pi k) int int div phi_m div phi_n G
//     + ik/(4pi) regularize(phi, '[1/r]', phi) - i/(4pi k) regularize(div phi, '[1/r]', div phi),
// in the single layer's factorisation: per right-hand side four density columns
// at the Gauss points (the three components of W Phi_RWG x and W Div x) go through
// the same kernel sum v = G u, and the projection takes them back to the edges.
// RWG function of local edge j of triangle t (edge j joins vertices j+1 and j+2,
// opposite vertex P_j; sign s = +1 in the edge's plus triangle, where it runs from
// the smaller to the larger vertex index, -1 in the minus one):
//   phi(y) = s l_j / (2 A_t) (y - P_j),  div phi = s l_j / A_t.
// The correction on triangles sharing a vertex: analytic int_b phi_j / R from the
// P1 integrals, int_b phi_j / R = s l_j / (2 A_b) sum_m (P_m - P_j) int_b lambda_m / R,
// minus the Gauss sum (the point itself left out), tested by the Gauss rule of a.
#include <algorithm>
#include <cmath>
#include <vector>

#include "far_tile.cuh"
#include "internal.h"
#include "p1_geom.cuh"

namespace gyps {

constexpr double kInv4PiE = 0.0795774715459476678844418816862571810;

// local edge data of triangle t: P (3 vertices), unit normal, s l / (2A) per local edge
struct RwgTri {
    double3 P[3];
    double3 n;
    double c[3];
};

__device__ inline RwgTri rwg_tri(const double *vtx, const int32_t *tri, const int32_t *tedge, int64_t t)
{
    RwgTri r;
#pragma unroll
    for (int m = 0; m < 3; ++m) r.P[m] = ld3(vtx, tri[3 * t + m]);
    const double3 n = cross(r.P[1] - r.P[0], r.P[2] - r.P[0]);
    const double two_area = sqrt(dot(n, n));
    r.n = (1.0 / two_area) * n;
#pragma unroll
    for (int j = 0; j < 3; ++j) {
        const double3 e = r.P[(j + 2) % 3] - r.P[(j + 1) % 3];
        const double s = (tedge[3 * t + j] & 1) ? -1.0 : 1.0;
        r.c[j] = s * sqrt(dot(e, e)) / two_area;  // s l / (2A)
    }
    return r;
}

// Densities at the Gauss points: column 4 c + m of right-hand side c, m < 3 the
// components of w_l sum_j x_e(j) phi_j(y_l), m = 3 the divergence w_l sum_j x_e(j) div phi_j.
// FP32 panel of R = 4 or 8 columns (interp32 layout) for right-hand sides c0, c0 + R/4.
template <int R>
__global__ void rwg_interp32_kernel(const double *vtx, const int32_t *tri, const int32_t *tedge,
                                    const double4_32a *pts64, int q, int64_t nq, int64_t nq_pad, const double2 *X,
                                    int64_t ldx, int c0, float *panel)
{
    const int64_t l = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (l >= nq_pad) return;
    const int64_t tile = l / kSrcTile;
    const int p = (int)(l % kSrcTile) >> 1, lane = (int)(l & 1);
    float *base = panel + tile * den_tile_floats(R);
    double ur[R], ui[R];
#pragma unroll
    for (int j = 0; j < R; ++j) ur[j] = ui[j] = 0.0;
    if (l < nq) {
        const int64_t t = l / q;
        const RwgTri g = rwg_tri(vtx, tri, tedge, t);
        const double4_32a y = pts64[l];
        const double3 yy = make_double3(y.x, y.y, y.z);
#pragma unroll
        for (int cc = 0; cc < R / 4; ++cc) {
            const double2 *xc = X + (int64_t)(c0 + cc) * ldx;
#pragma unroll
            for (int j = 0; j < 3; ++j) {
                const double2 xe = xc[tedge[3 * t + j] >> 1];
                const double3 f = g.c[j] * (yy - g.P[j]);
                const double d = 2.0 * g.c[j];
                ur[4 * cc + 0] += f.x * xe.x; ui[4 * cc + 0] += f.x * xe.y;
                ur[4 * cc + 1] += f.y * xe.x; ui[4 * cc + 1] += f.y * xe.y;
                ur[4 * cc + 2] += f.z * xe.x; ui[4 * cc + 2] += f.z * xe.y;
                ur[4 * cc + 3] += d * xe.x;   ui[4 * cc + 3] += d * xe.y;
            }
        }
#pragma unroll
        for (int j = 0; j < R; ++j) {
            ur[j] *= y.w;
            ui[j] *= y.w;
        }
    }
#pragma unroll
    for (int j = 0; j < R; ++j) {
        float *u4 = base + 4 * ((int64_t)p * R + j);
        u4[lane] = (float)ur[j];
        u4[2 + lane] = (float)ui[j];
        base[4 * kSrcPairs * R + 2 * ((int64_t)p * R + j) + lane] = -(float)ui[j];
    }
}

// The same in FP64 for all right-hand sides: u64[l + (4 c + m) ld].
__global__ void rwg_interp64_kernel(const double *vtx, const int32_t *tri, const int32_t *tedge,
                                    const double4_32a *pts64, int q, int64_t nq, int64_t ld, const double2 *X,
                                    int64_t ldx, int nrhs, double2 *u64)
{
    const int64_t l = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int c = blockIdx.y;
    if (l >= nq || c >= nrhs) return;
    const int64_t t = l / q;
    const RwgTri g = rwg_tri(vtx, tri, tedge, t);
    const double4_32a y = pts64[l];
    const double3 yy = make_double3(y.x, y.y, y.z);
    const double2 *xc = X + (int64_t)c * ldx;
    double3 vr = make_double3(0.0, 0.0, 0.0), vi = vr;
    double dr = 0.0, di = 0.0;
#pragma unroll
    for (int j = 0; j < 3; ++j) {
        const double2 xe = xc[tedge[3 * t + j] >> 1];
        const double3 f = g.c[j] * (yy - g.P[j]);
        vr = vr + xe.x * f;
        vi = vi + xe.y * f;
        dr += 2.0 * g.c[j] * xe.x;
        di += 2.0 * g.c[j] * xe.y;
    }
    double2 *u = u64 + l + (int64_t)(4 * c) * ld;
    u[0] = make_double2(y.w * vr.x, y.w * vi.x);
    u[ld] = make_double2(y.w * vr.y, y.w * vi.y);
    u[2 * ld] = make_double2(y.w * vr.z, y.w * vi.z);
    u[3 * ld] = make_double2(y.w * dr, y.w * di);
}

// Correction blocks of the near pair (a, b): A[i][j] (vector part) and B[i][j]
// (divergence part) for local edges i of a and j of b, without the k factors.
__global__ void efie_blocks_kernel(const double *vtx, const int32_t *tri, const int32_t *tedge,
                                   const double4_32a *pts64, int q, int64_t npairs, const int32_t *pair_a,
                                   const int32_t *pair_b, double *blocks)
{
    const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= npairs) return;
    const int64_t a = pair_a[p], b = pair_b[p];
    const RwgTri ga = rwg_tri(vtx, tri, tedge, a), gb = rwg_tri(vtx, tri, tedge, b);
    double bA[9], bB[9];
#pragma unroll
    for (int e = 0; e < 9; ++e) bA[e] = bB[e] = 0.0;
    for (int kq = 0; kq < q; ++kq) {
        const double4_32a xk4 = pts64[a * q + kq];
        const double3 xk = make_double3(xk4.x, xk4.y, xk4.z);
        double I[3];
        p1_over_r(xk, gb.P, I);
        double3 gy = make_double3(0.0, 0.0, 0.0);
        double g1 = 0.0;
        for (int lq = 0; lq < q; ++lq) {
            if (a == b && lq == kq) continue;
            const double4_32a y4 = pts64[b * q + lq];
            const double3 y = make_double3(y4.x, y4.y, y4.z);
            const double3 d = xk - y;
            const double e = y4.w / sqrt(dot(d, d));
            gy = gy + e * y;
            g1 += e;
        }
        const double isum = I[0] + I[1] + I[2];
        const double3 iy = I[0] * gb.P[0] + I[1] * gb.P[1] + I[2] * gb.P[2];
#pragma unroll
        for (int j = 0; j < 3; ++j) {
            // int_b phi_j / R - Gauss = c_j ((sum_m I_m P_m - isum P_j) - (gy - g1 P_j))
            const double3 vec = gb.c[j] * ((iy - isum * gb.P[j]) - (gy - g1 * gb.P[j]));
            const double dv = 2.0 * gb.c[j] * (isum - g1);
#pragma unroll
            for (int i = 0; i < 3; ++i) {
                const double3 fi = ga.c[i] * (xk - ga.P[i]);
                bA[3 * i + j] += xk4.w * dot(fi, vec);
                bB[3 * i + j] += xk4.w * 2.0 * ga.c[i] * dv;
            }
        }
    }
#pragma unroll
    for (int e = 0; e < 9; ++e) {
        blocks[18 * p + e] = bA[e];
        blocks[18 * p + 9 + e] = bB[e];
    }
}

// Y[e, c] = sign (ik/(4pi) (sum_k w_k phi_e(x_k) . v_vec + CA x) - i/(4pi k) (sum_k w_k div phi_e v_div + CB x)),
// one thread per edge and right-hand side: the Gauss points of its two triangles and
// the correction blocks of their near pairs.
__global__ void efie_project_kernel(const double *vtx, const int32_t *tri, const int32_t *tedge, const int32_t *etri,
                                    const double4_32a *pts64, int q, int64_t ne, const double2 *v, int64_t ldv,
                                    const int32_t *pair_ptr, const int32_t *pair_b, const double *blocks,
                                    const double2 *X, int64_t ldx, double k, double sign, double2 *Y, int64_t ldy)
{
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int c = blockIdx.y;
    if (e >= ne) return;
    const double2 *xc = X + (int64_t)c * ldx;
    const double2 *v0 = v + (int64_t)(4 * c) * ldv;
    double ar = 0.0, ai = 0.0, br = 0.0, bi = 0.0;  // vector and divergence parts
    for (int side = 0; side < 2; ++side) {
        const int32_t code = etri[2 * e + side];
        const int64_t t = code / 3;
        const int i = code - 3 * (int)t;
        const RwgTri g = rwg_tri(vtx, tri, tedge, t);
        for (int kq = 0; kq < q; ++kq) {
            const int64_t l = t * q + kq;
            const double4_32a x = pts64[l];
            const double3 f = g.c[i] * (make_double3(x.x, x.y, x.z) - g.P[i]);
            const double2 vx = v0[l], vy = v0[l + ldv], vz = v0[l + 2 * ldv], vd = v0[l + 3 * ldv];
            ar += x.w * (f.x * vx.x + f.y * vy.x + f.z * vz.x);
            ai += x.w * (f.x * vx.y + f.y * vy.y + f.z * vz.y);
            br += x.w * 2.0 * g.c[i] * vd.x;
            bi += x.w * 2.0 * g.c[i] * vd.y;
        }
        for (int32_t p = pair_ptr[t]; p < pair_ptr[t + 1]; ++p) {
            const int64_t b = pair_b[p];
            const double *blk = blocks + 18 * (int64_t)p;
#pragma unroll
            for (int j = 0; j < 3; ++j) {
                const double2 xf = xc[tedge[3 * b + j] >> 1];
                ar += blk[3 * i + j] * xf.x;
                ai += blk[3 * i + j] * xf.y;
                br += blk[9 + 3 * i + j] * xf.x;
                bi += blk[9 + 3 * i + j] * xf.y;
            }
        }
    }
    // ik/(4pi) (ar + i ai) - i/(4pi k) (br + i bi)
    const double ca = sign * k * kInv4PiE, cb = sign * kInv4PiE / k;
    Y[e + (int64_t)c * ldy] = make_double2(-ca * ai + cb * bi, ca * ar - cb * br);
}

// F[e, j] = sum_k w_k (beta phi_e(x_k) . p_j - (1 - beta) (n x phi_e(x_k)) . (d_j x p_j)) exp(i k d_j . x_k):
// the listing's RHS (beta = 1: the EFIE's int phi . E_inc); dp: nrhs x 6 (d, p).
__global__ void efie_rhs_kernel(const double *vtx, const int32_t *tri, const int32_t *tedge, const int32_t *etri,
                                const double4_32a *pts64, int q, int64_t ne, double k, double beta, const double *dp,
                                double2 *F, int64_t ldf)
{
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int j = blockIdx.y;
    if (e >= ne) return;
    const double3 d = make_double3(dp[6 * j], dp[6 * j + 1], dp[6 * j + 2]);
    const double3 pol = make_double3(dp[6 * j + 3], dp[6 * j + 4], dp[6 * j + 5]);
    const double3 hp = cross(d, pol);
    double fr = 0.0, fi = 0.0;
    for (int side = 0; side < 2; ++side) {
        const int32_t code = etri[2 * e + side];
        const int64_t t = code / 3;
        const int i = code - 3 * (int)t;
        const RwgTri g = rwg_tri(vtx, tri, tedge, t);
        for (int kq = 0; kq < q; ++kq) {
            const double4_32a x = pts64[t * q + kq];
            const double3 xx = make_double3(x.x, x.y, x.z);
            const double3 f = g.c[i] * (xx - g.P[i]);
            const double fp = x.w * (beta * dot(f, pol) - (1.0 - beta) * dot(cross(g.n, f), hp));
            double sn, cs;
            sincos(k * dot(d, xx), &sn, &cs);
            fr += fp * cs;
            fi += fp * sn;
        }
    }
    F[e + (int64_t)j * ldf] = make_double2(fr, fi);
}

// RWG topology on the host (edges in lexicographic order of their vertex pairs),
// then the correction blocks on the device.
gyps_status efie_prepare(Mesh *m, cudaStream_t s)
{
    if (m->d_efie_blocks) return GYPS_OK;
    std::vector<int32_t> tri((size_t)m->nt * 3);
    GYPS_CUDA(cudaMemcpyAsync(tri.data(), m->d_tri, tri.size() * sizeof(int32_t), cudaMemcpyDeviceToHost, s));
    GYPS_CUDA(cudaStreamSynchronize(s));
    struct Half {
        int64_t key;
        int32_t code;  // 3 t + j
        bool plus;
    };
    std::vector<Half> h((size_t)m->nt * 3);
    for (int64_t t = 0; t < m->nt; ++t)
        for (int j = 0; j < 3; ++j) {
            const int64_t a = tri[3 * t + (j + 1) % 3], b = tri[3 * t + (j + 2) % 3];
            h[3 * t + j] = {std::min(a, b) * m->nv + std::max(a, b), (int32_t)(3 * t + j), a < b};
        }
    std::sort(h.begin(), h.end(), [](const Half &x, const Half &y) { return x.key < y.key; });
    if (h.size() % 2 != 0) return set_error(GYPS_ERR_INVALID, "RWG functions need a closed mesh");
    const int64_t ne = (int64_t)h.size() / 2;
    std::vector<int32_t> tedge((size_t)m->nt * 3), etri((size_t)ne * 2), edges((size_t)ne * 2);
    for (int64_t e = 0; e < ne; ++e) {
        const Half &x = h[2 * e], &y = h[2 * e + 1];
        if (x.key != y.key || (2 * e + 2 < (int64_t)h.size() && h[2 * e + 2].key == x.key) ||
            (e > 0 && h[2 * e - 1].key == x.key))
            return set_error(GYPS_ERR_INVALID, "RWG functions need a closed mesh (every edge in two triangles)");
        if (x.plus == y.plus)
            return set_error(GYPS_ERR_INVALID, "RWG functions need a consistently oriented mesh");
        const Half &pl = x.plus ? x : y, &mi = x.plus ? y : x;
        etri[2 * e] = pl.code;
        etri[2 * e + 1] = mi.code;
        tedge[pl.code] = (int32_t)(e << 1);
        tedge[mi.code] = (int32_t)((e << 1) | 1);
        edges[2 * e] = (int32_t)(x.key / m->nv);
        edges[2 * e + 1] = (int32_t)(x.key % m->nv);
    }
    int32_t *d_tedge = nullptr, *d_etri = nullptr;
    double *d_blocks = nullptr;
    cudaError_t err = cudaMalloc((void **)&d_tedge, tedge.size() * sizeof(int32_t));
    if (err == cudaSuccess) err = cudaMalloc((void **)&d_etri, etri.size() * sizeof(int32_t));
    if (err == cudaSuccess) err = cudaMalloc((void **)&d_blocks, (size_t)m->npairs * 18 * sizeof(double));
    if (err == cudaSuccess)
        err = cudaMemcpyAsync(d_tedge, tedge.data(), tedge.size() * sizeof(int32_t), cudaMemcpyHostToDevice, s);
    if (err == cudaSuccess)
        err = cudaMemcpyAsync(d_etri, etri.data(), etri.size() * sizeof(int32_t), cudaMemcpyHostToDevice, s);
    if (err == cudaSuccess) {
        efie_blocks_kernel<<<(unsigned)((m->npairs + 127) / 128), 128, 0, s>>>(
            m->d_vtx, m->d_tri, d_tedge, m->d_pts64, m->q, m->npairs, m->d_pair_a, m->d_pair_b, d_blocks);
        err = cudaGetLastError();
    }
    if (err == cudaSuccess) err = cudaStreamSynchronize(s);
    if (err != cudaSuccess) {
        cudaFree(d_tedge);
        cudaFree(d_etri);
        cudaFree(d_blocks);
        return cuda_error(err, "EFIE topology / correction");
    }
    m->ne = ne;
    m->d_tedge = d_tedge;
    m->d_etri = d_etri;
    m->h_edges = std::move(edges);
    m->d_efie_blocks = d_blocks;
    return GYPS_OK;
}

gyps_status efie_apply_device(Mesh *m, double k, double sign, int nrhs, const double2 *X, int64_t ldx, double2 *Y,
                              int64_t ldy, int prec, cudaStream_t s)
{
    if (prec == GYPS_PREC_AUTO) prec = GYPS_PREC_FP32;
    if (prec != GYPS_PREC_FP64 && prec != GYPS_PREC_FP32 && prec != GYPS_PREC_DF64)
        return set_error(GYPS_ERR_UNSUPPORTED, "EFIE: FP64, FP32 or DF64");
    GYPS_TRY(efie_prepare(m, s));
    const int64_t ld = m->nq;
    const int ncol = 4 * nrhs;
    GYPS_TRY(grow(m, &m->ws_v, &m->ws_v_bytes, (size_t)(ld * ncol) * sizeof(double2)));
    double2 *v = reinterpret_cast<double2 *>(m->ws_v);
    if (m->prof) ++m->prof_applies;
    if (prec == GYPS_PREC_FP32) {
        GYPS_CUDA(cudaMemsetAsync(v, 0, (size_t)(ld * ncol) * sizeof(double2), s));
        GYPS_TRY(grow(m, &m->ws_den, &m->ws_den_bytes, (size_t)(m->n_src_tiles * den_tile_floats(8)) * sizeof(float)));
        float *panel = reinterpret_cast<float *>(m->ws_den);
        const unsigned gi = (unsigned)((m->nq_pad + 255) / 256);
        for (int c0 = 0; c0 < nrhs;) {
            const int w = nrhs - c0 >= 2 ? 2 : 1;  // right-hand sides per pass (4 columns each)
            if (w == 2)
                rwg_interp32_kernel<8><<<gi, 256, 0, s>>>(m->d_vtx, m->d_tri, m->d_tedge, m->d_pts64, m->q, m->nq,
                                                          m->nq_pad, X, ldx, c0, panel);
            else
                rwg_interp32_kernel<4><<<gi, 256, 0, s>>>(m->d_vtx, m->d_tri, m->d_tedge, m->d_pts64, m->q, m->nq,
                                                          m->nq_pad, X, ldx, c0, panel);
            GYPS_CUDA(cudaGetLastError());
            GYPS_TRY(far32_panel(m, k, panel, 4 * w, v + (int64_t)(4 * c0) * ld, ld, s));
            c0 += w;
        }
    } else {
        GYPS_TRY(grow(m, &m->ws_den, &m->ws_den_bytes, (size_t)(ld * ncol) * sizeof(double2)));
        double2 *u64 = reinterpret_cast<double2 *>(m->ws_den);
        dim3 gi((unsigned)((m->nq + 255) / 256), (unsigned)nrhs);
        rwg_interp64_kernel<<<gi, 256, 0, s>>>(m->d_vtx, m->d_tri, m->d_tedge, m->d_pts64, m->q, m->nq, ld, X, ldx,
                                               nrhs, u64);
        GYPS_CUDA(cudaGetLastError());
        for (int c0 = 0; c0 < ncol;) {
            const int left = ncol - c0;
            if (prec == GYPS_PREC_DF64) {
                const int w = left >= 8 ? 8 : left >= 4 ? 4 : left >= 2 ? 2 : 1;
                GYPS_TRY(run_far_df(m, k, m->d_pts64, true, u64, ld, c0, w, v, ld, 0, m->nq, s));
                c0 += w;
            } else {
                const int w = left >= 4 ? 4 : left >= 2 ? 2 : 1;
                GYPS_TRY(far64_cols(m, k, u64, ld, c0, w, v, ld, s));
                c0 += w;
            }
        }
    }
    dim3 gp((unsigned)((m->ne + 127) / 128), (unsigned)nrhs);
    efie_project_kernel<<<gp, 128, 0, s>>>(m->d_vtx, m->d_tri, m->d_tedge, m->d_etri, m->d_pts64, m->q, m->ne, v, ld,
                                           m->d_pair_ptr, m->d_pair_b, m->d_efie_blocks, X, ldx, k, sign, Y, ldy);
    GYPS_CUDA(cudaGetLastError());
    return GYPS_OK;
}

// ---------------------------------------------------------------- MFIE (nxK)
// nxK = (1/4pi) int int (n_x x phi_m(x)) . (grad_y G(x, y) x phi_n(y)) + 'grady[1/r]' correction,
// grad_y exp(ikr)/r = F (x - y),  F = (1 - ikr) exp(ikr) / r^3.  The far sum per Gauss point,
//   S_t = sum_l F(r_tl) (x_t - y_l) x u_l,   u_l = w_l J(y_l)  (3 complex components),
// is taken pair by pair (the split x_t x sum F u - sum F y x u would cancel on close pairs),
// without the pairs inside one triangle (their vector is normal to the triangle and meets
// the in-plane test function n x phi).

// FP32, in the single layer's persistent tile form (coordinates scaled by k, so that
// F (x - y) = k^2 F_s (x_s - y_s)): (target tile) x (source tile)
// items over a persistent grid, position and density tiles (the RWG panel of one
// right-hand side: columns x, y, z, div; div unused) by 1-D bulk copies into a 3-stage
// ring, T targets per thread, source points in pairs with packed f32x2 arithmetic,
// per-tile sums folded into TwoSum pairs, FP64 atomics per target-tile flush.
struct MfieArgs {
    const float *pos_panel, *den_panel;
    const float4 *tgt;
    double2 *v;  // nq x 3 (the components of S), added into
    int64_t ldv, nq, n_src_tiles, n_tgt_tiles;
    int q;
    float ks;
    int *err;
};

template <int T>
struct MfieCfg {
    static constexpr int NT = 128;
    static constexpr int TT = NT * T;
    static constexpr int STAGES = 3;
    static constexpr int POS_BYTES = kPosTileFloats * 4;
    static constexpr int DEN_BYTES = kSrcPairs * 6 * 4 * 4;  // R = 4 panel
    static constexpr int STAGE_BYTES = POS_BYTES + DEN_BYTES;
    static constexpr int SMEM = STAGES * STAGE_BYTES + 64;
};

template <int T, bool CHECK>
__device__ __forceinline__ void mfie_tile(const float *sp, const float2 (&tx)[T], const float2 (&ty)[T],
                                          const float2 (&tz)[T], const int64_t (&tq0)[T], int64_t src0, int q,
                                          float ks, float2 (&acc)[T][6])
{
    const float4 *XY = reinterpret_cast<const float4 *>(sp);
    const float2 *Z = reinterpret_cast<const float2 *>(sp + 4 * kSrcPairs);
    const float4 *U = reinterpret_cast<const float4 *>(sp + kPosTileFloats);
    const float2 ks2 = make_float2(ks, ks);
    const float2 magic = make_float2(12582912.0f, 12582912.0f);  // 1.5 * 2^23: round to integer
    const float2 nmagic = make_float2(-12582912.0f, -12582912.0f);
    const float2 inv2pi = make_float2(0.159154943091895335769f, 0.159154943091895335769f);
    const float2 m2pi = make_float2(-6.28318530717958647692f, -6.28318530717958647692f);
#pragma unroll 1
    for (int p = 0; p < kSrcPairs; ++p) {
        const float4 xy = XY[p];
        const float2 sx = __fmul2_rn(make_float2(xy.x, xy.y), ks2), sy = __fmul2_rn(make_float2(xy.z, xy.w), ks2);
        const float2 sz = __fmul2_rn(Z[p], ks2);
        float2 ur[3], ui[3];
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            const float4 u = U[4 * p + c];
            ur[c] = make_float2(u.x, u.y);
            ui[c] = make_float2(u.z, u.w);
        }
#pragma unroll
        for (int t = 0; t < T; ++t) {
            const float2 d[3] = {__fadd2_rn(tx[t], sx), __fadd2_rn(ty[t], sy), __fadd2_rn(tz[t], sz)};
            float2 r2 = __fmul2_rn(d[0], d[0]);
            r2 = __ffma2_rn(d[1], d[1], r2);
            r2 = __ffma2_rn(d[2], d[2], r2);
            const float2 rs = make_float2(rsqrt_mufu(r2.x), rsqrt_mufu(r2.y));
            const float2 ph = __fmul2_rn(r2, rs);                                 // k r
            const float2 nr = __fadd2_rn(__ffma2_rn(ph, inv2pi, magic), nmagic);  // nearest integer to k r / (2 pi)
            const float2 ang = __ffma2_rn(nr, m2pi, ph);
            const float2 sn = make_float2(sin_mufu(ang.x), sin_mufu(ang.y));
            const float2 cs = make_float2(cos_mufu(ang.x), cos_mufu(ang.y));
            const float2 r3 = __fmul2_rn(__fmul2_rn(rs, rs), rs);
            // F = (1 - i k r) exp(i k r) / r^3 (scaled coordinates)
            float2 fr = __fmul2_rn(__ffma2_rn(ph, sn, cs), r3);
            float2 fi = __fmul2_rn(__ffma2_rn(make_float2(-ph.x, -ph.y), cs, sn), r3);
            if (CHECK) {  // same triangle (and the point itself): 0
                if ((uint64_t)(src0 + 2 * p - tq0[t]) < (uint64_t)q) fr.x = fi.x = 0.0f;
                if ((uint64_t)(src0 + 2 * p + 1 - tq0[t]) < (uint64_t)q) fr.y = fi.y = 0.0f;
            }
            float2 gr[3], gi[3];
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                gr[c] = __fmul2_rn(fr, d[c]);
                gi[c] = __fmul2_rn(fi, d[c]);
            }
            // S += G x u:  (G x u)_c = G_c1 u_c2 - G_c2 u_c1 (complex)
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                const int c1 = (c + 1) % 3, c2 = (c + 2) % 3;
                float2 re = acc[t][2 * c], im = acc[t][2 * c + 1];
                re = __ffma2_rn(gr[c1], ur[c2], re);
                re = __ffma2_rn(make_float2(-gi[c1].x, -gi[c1].y), ui[c2], re);
                re = __ffma2_rn(make_float2(-gr[c2].x, -gr[c2].y), ur[c1], re);
                re = __ffma2_rn(gi[c2], ui[c1], re);
                im = __ffma2_rn(gr[c1], ui[c2], im);
                im = __ffma2_rn(gi[c1], ur[c2], im);
                im = __ffma2_rn(make_float2(-gr[c2].x, -gr[c2].y), ui[c1], im);
                im = __ffma2_rn(make_float2(-gi[c2].x, -gi[c2].y), ur[c1], im);
                acc[t][2 * c] = re;
                acc[t][2 * c + 1] = im;
            }
        }
    }
}

template <int T>
__global__ void __launch_bounds__(MfieCfg<T>::NT) far_mfie_tile_kernel(const MfieArgs a)
{
    using C = MfieCfg<T>;
    extern __shared__ __align__(128) unsigned char smem[];
    uint64_t *bars = reinterpret_cast<uint64_t *>(smem + C::STAGES * C::STAGE_BYTES);
    const int tid_x = threadIdx.x;
    const int64_t items = a.n_tgt_tiles * a.n_src_tiles;
    const int64_t beg = items * blockIdx.x / gridDim.x;
    const int64_t end = items * (blockIdx.x + 1) / gridDim.x;
    if (beg >= end) return;
    if (tid_x == 0) {
        for (int s = 0; s < C::STAGES; ++s) mbar_init(smem_addr(&bars[s]), 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    auto issue = [&](int64_t item) {
        const int s = (int)((item - beg) % C::STAGES);
        const int64_t st = item % a.n_src_tiles;
        const uint32_t bar = smem_addr(&bars[s]);
        const uint32_t dst = smem_addr(smem + s * C::STAGE_BYTES);
        mbar_expect_tx(bar, C::STAGE_BYTES);
        bulk_g2s(dst, a.pos_panel + st * kPosTileFloats, C::POS_BYTES, bar);
        bulk_g2s(dst + C::POS_BYTES, a.den_panel + st * den_tile_floats(4), C::DEN_BYTES, bar);
    };
    int64_t issued = beg;
    if (tid_x == 0)
        for (; issued < end && issued < beg + C::STAGES - 1; ++issued) issue(issued);

    float2 tx[T], ty[T], tz[T];
    int64_t tid[T], tq0[T];
    float2 acc[T][6];
    float hi[T][6], lo[T][6];
    int64_t cur_tt = -1;
    const double scale = (double)a.ks * (double)a.ks;  // F (x - y) = k^2 F_s (x_s - y_s)
    auto flush = [&]() {
#pragma unroll
        for (int t = 0; t < T; ++t) {
            if (tid[t] < a.nq) {
#pragma unroll
                for (int c = 0; c < 3; ++c) {
                    double *dst = reinterpret_cast<double *>(a.v + tid[t] + c * a.ldv);
                    atomicAdd(dst, ((double)hi[t][2 * c] + (double)lo[t][2 * c]) * scale);
                    atomicAdd(dst + 1, ((double)hi[t][2 * c + 1] + (double)lo[t][2 * c + 1]) * scale);
                }
            }
        }
    };
    bool failed = false;
    int64_t i = beg;
    for (; i < end; ++i) {
        if (tid_x == 0 && issued < end && issued == i + C::STAGES - 1) {
            issue(issued);
            ++issued;
        }
        const int64_t tt = i / a.n_src_tiles, st = i % a.n_src_tiles;
        const int64_t tb = tt * C::TT;
        const int64_t te = min(tb + (int64_t)C::TT, a.nq);
        if (tt != cur_tt) {
            if (cur_tt >= 0) flush();
#pragma unroll
            for (int t = 0; t < T; ++t) {
                const int64_t g = tb + tid_x + t * C::NT;
                tid[t] = g;
                tq0[t] = (g / a.q) * a.q;
                const float4 p = a.tgt[min(g, a.nq - 1)];
                tx[t] = make_float2(p.x * a.ks, p.x * a.ks);
                ty[t] = make_float2(p.y * a.ks, p.y * a.ks);
                tz[t] = make_float2(p.z * a.ks, p.z * a.ks);
#pragma unroll
                for (int c = 0; c < 6; ++c) hi[t][c] = lo[t][c] = 0.0f;
            }
            cur_tt = tt;
        }
#pragma unroll
        for (int t = 0; t < T; ++t)
#pragma unroll
            for (int c = 0; c < 6; ++c) acc[t][c] = make_float2(0.0f, 0.0f);
        const int s = (int)((i - beg) % C::STAGES);
        const uint32_t parity = (uint32_t)(((i - beg) / C::STAGES) & 1);
        const bool ok = mbar_wait_bounded(smem_addr(&bars[s]), parity);
        if (ok) {
            const float *sp = reinterpret_cast<const float *>(smem + s * C::STAGE_BYTES);
            const int64_t src0 = st * kSrcTile;
            if (tb - 8 < src0 + kSrcTile && src0 < te + 8)
                mfie_tile<T, true>(sp, tx, ty, tz, tq0, src0, a.q, a.ks, acc);
            else
                mfie_tile<T, false>(sp, tx, ty, tz, tq0, src0, a.q, a.ks, acc);
#pragma unroll
            for (int t = 0; t < T; ++t)
#pragma unroll
                for (int c = 0; c < 6; ++c) two_sum_acc(hi[t][c], lo[t][c], __fadd_rn(acc[t][c].x, acc[t][c].y));
        }
        if (__syncthreads_or(!ok)) {
            failed = true;
            break;
        }
    }
    if (failed) {
        if (tid_x == 0) {
            atomicExch(a.err, 1);
            for (int64_t j = i; j < issued; ++j) {
                const int s = (int)((j - beg) % C::STAGES);
                mbar_wait_bounded(smem_addr(&bars[s]), (uint32_t)(((j - beg) / C::STAGES) & 1));
            }
        }
        __syncthreads();
        return;
    }
    flush();
}

// The same in FP64 (one right-hand side per pass).
__global__ void __launch_bounds__(128) far_mfie64_kernel(const double4_32a *pts, int q, const double2 *u64, int64_t ldu,
                                                         int c0, int64_t nq, double k, double2 *v, int64_t ldv)
{
    __shared__ double4_32a sp[128];
    __shared__ double2 su[128][3];
    const int64_t tg = (int64_t)blockIdx.x * 128 + threadIdx.x;
    const int64_t tq0 = (min(tg, nq - 1) / q) * q;
    const double4_32a x = pts[min(tg, nq - 1)];
    double acc[6] = {0.0, 0.0, 0.0, 0.0, 0.0, 0.0};
    for (int64_t s0 = 0; s0 < nq; s0 += 128) {
        const int64_t l = s0 + threadIdx.x;
        if (l < nq) {
            sp[threadIdx.x] = pts[l];
#pragma unroll
            for (int c = 0; c < 3; ++c) su[threadIdx.x][c] = u64[l + (int64_t)(4 * c0 + c) * ldu];
        }
        __syncthreads();
        const int n = (int)min((int64_t)128, nq - s0);
        for (int ll = 0; ll < n; ++ll) {
            if ((uint64_t)(s0 + ll - tq0) < (uint64_t)q) continue;
            const double4_32a y = sp[ll];
            const double d[3] = {x.x - y.x, x.y - y.y, x.z - y.z};
            const double r2 = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
            const double ri = rsqrt(r2);
            const double kr = k * r2 * ri;
            double sn, cs;
            sincos(kr, &sn, &cs);
            const double r3 = ri * ri * ri;
            const double fr = (cs + kr * sn) * r3, fi = (sn - kr * cs) * r3;
            const double ur[3] = {su[ll][0].x, su[ll][1].x, su[ll][2].x};
            const double ui[3] = {su[ll][0].y, su[ll][1].y, su[ll][2].y};
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                const int c1 = (c + 1) % 3, c2 = (c + 2) % 3;
                const double xr = d[c1] * ur[c2] - d[c2] * ur[c1], xi = d[c1] * ui[c2] - d[c2] * ui[c1];
                acc[2 * c] += fr * xr - fi * xi;
                acc[2 * c + 1] += fr * xi + fi * xr;
            }
        }
        __syncthreads();
    }
    if (tg < nq) {
#pragma unroll
        for (int c = 0; c < 3; ++c) v[tg + (int64_t)(3 * c0 + c) * ldv] = make_double2(acc[2 * c], acc[2 * c + 1]);
    }
}

// MFIE correction blocks on the near pair (a, b), a != b (0 inside one triangle), with 1/(4pi):
//   blk[i][j] = sum_{k in a} w_k (n_a x f_i(x_k)) . (int_b (x_k - y)/R^3 x f_j - Gauss sum over b),
//   int_b (x - y)/R^3 x f_j = c_j sum_m (int_b lambda_m (x - y)/R^3) x (P_m - P_j).
__global__ void mfie_blocks_kernel(const double *vtx, const int32_t *tri, const int32_t *tedge,
                                   const double4_32a *pts64, int q, int64_t npairs, const int32_t *pair_a,
                                   const int32_t *pair_b, double *blocks)
{
    const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= npairs) return;
    const int64_t a = pair_a[p], b = pair_b[p];
    double blk[9];
#pragma unroll
    for (int e = 0; e < 9; ++e) blk[e] = 0.0;
    if (a != b) {
        const RwgTri ga = rwg_tri(vtx, tri, tedge, a), gb = rwg_tri(vtx, tri, tedge, b);
        for (int kq = 0; kq < q; ++kq) {
            const double4_32a xk4 = pts64[a * q + kq];
            const double3 xk = make_double3(xk4.x, xk4.y, xk4.z);
            double3 V[3];
            p1_grad_over_r(xk, gb.P, V);
#pragma unroll
            for (int j = 0; j < 3; ++j) {
                double3 an = make_double3(0.0, 0.0, 0.0);
#pragma unroll
                for (int mm = 0; mm < 3; ++mm) an = an + gb.c[j] * cross(V[mm], gb.P[mm] - gb.P[j]);
                for (int lq = 0; lq < q; ++lq) {
                    const double4_32a y4 = pts64[b * q + lq];
                    const double3 y = make_double3(y4.x, y4.y, y4.z);
                    const double3 d = xk - y;
                    const double r = sqrt(dot(d, d));
                    an = an - (y4.w / (r * r * r)) * cross(d, gb.c[j] * (y - gb.P[j]));
                }
#pragma unroll
                for (int i = 0; i < 3; ++i) {
                    const double3 tf = cross(ga.n, ga.c[i] * (xk - ga.P[i]));
                    blk[3 * i + j] += xk4.w * kInv4PiE * dot(tf, an);
                }
            }
        }
    }
#pragma unroll
    for (int e = 0; e < 9; ++e) blocks[9 * p + e] = blk[e];
}

// Y[e, c] (+)= cm sum_k w_k phi_e(x_k) . J(x_k) + ck ((1/4pi) sum_k w_k (n x phi_e(x_k)) . S_k + (C x)_e):
// the MFIE part of the listing's LHS (cm = 0, ck = 1: nxK x).
__global__ void mfie_project_kernel(const double *vtx, const int32_t *tri, const int32_t *tedge, const int32_t *etri,
                                    const double4_32a *pts64, int q, int64_t ne, const double2 *S, int64_t lds,
                                    const int32_t *pair_ptr, const int32_t *pair_b, const double *blocks,
                                    const double2 *X, int64_t ldx, double cm, double ck, int accumulate, double2 *Y,
                                    int64_t ldy)
{
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int c = blockIdx.y;
    if (e >= ne) return;
    const double2 *xc = X + (int64_t)c * ldx;
    const double2 *s0 = S + (int64_t)(3 * c) * lds;
    double mr = 0.0, mi = 0.0, kr = 0.0, ki = 0.0;
    for (int side = 0; side < 2; ++side) {
        const int32_t code = etri[2 * e + side];
        const int64_t t = code / 3;
        const int i = code - 3 * (int)t;
        const RwgTri g = rwg_tri(vtx, tri, tedge, t);
        double2 xl[3];
#pragma unroll
        for (int j = 0; j < 3; ++j) xl[j] = xc[tedge[3 * t + j] >> 1];
        for (int kq = 0; kq < q; ++kq) {
            const int64_t l = t * q + kq;
            const double4_32a x = pts64[l];
            const double3 xx = make_double3(x.x, x.y, x.z);
            const double3 f = g.c[i] * (xx - g.P[i]);
            if (cm != 0.0) {
                double3 jr = make_double3(0.0, 0.0, 0.0), ji = jr;
#pragma unroll
                for (int j = 0; j < 3; ++j) {
                    const double3 fj = g.c[j] * (xx - g.P[j]);
                    jr = jr + xl[j].x * fj;
                    ji = ji + xl[j].y * fj;
                }
                mr += x.w * dot(f, jr);
                mi += x.w * dot(f, ji);
            }
            const double3 tf = cross(g.n, f);
            const double2 sx = s0[l], sy = s0[l + lds], sz = s0[l + 2 * lds];
            kr += x.w * kInv4PiE * (tf.x * sx.x + tf.y * sy.x + tf.z * sz.x);
            ki += x.w * kInv4PiE * (tf.x * sx.y + tf.y * sy.y + tf.z * sz.y);
        }
        for (int32_t p = pair_ptr[t]; p < pair_ptr[t + 1]; ++p) {
            const int64_t b = pair_b[p];
            const double *blk = blocks + 9 * (int64_t)p;
#pragma unroll
            for (int j = 0; j < 3; ++j) {
                const double2 xf = xc[tedge[3 * b + j] >> 1];
                kr += blk[3 * i + j] * xf.x;
                ki += blk[3 * i + j] * xf.y;
            }
        }
    }
    double2 out = make_double2(cm * mr + ck * kr, cm * mi + ck * ki);
    double2 &y = Y[e + (int64_t)c * ldy];
    if (accumulate) {
        out.x += y.x;
        out.y += y.y;
    }
    y = out;
}

static gyps_status mfie_prepare(Mesh *m, cudaStream_t s)
{
    GYPS_TRY(efie_prepare(m, s));
    if (m->d_mfie_blocks) return GYPS_OK;
    double *blocks = nullptr;
    GYPS_CUDA(cudaMalloc((void **)&blocks, (size_t)m->npairs * 9 * sizeof(double)));
    mfie_blocks_kernel<<<(unsigned)((m->npairs + 127) / 128), 128, 0, s>>>(m->d_vtx, m->d_tri, m->d_tedge, m->d_pts64,
                                                                          m->q, m->npairs, m->d_pair_a, m->d_pair_b,
                                                                          blocks);
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) {
        cudaFree(blocks);
        return cuda_error(e, "MFIE correction");
    }
    m->d_mfie_blocks = blocks;
    return GYPS_OK;
}

// Y (+)= cm Id X + ck nxK X (see mfie_project_kernel); prec FP32, or FP64 (also for double-float).
static gyps_status mfie_apply_device(Mesh *m, double k, int nrhs, const double2 *X, int64_t ldx, double2 *Y,
                                     int64_t ldy, int prec, double cm, double ck, bool accumulate, cudaStream_t s)
{
    GYPS_TRY(mfie_prepare(m, s));
    const int64_t ld = m->nq;
    GYPS_TRY(grow(m, &m->ws_den, &m->ws_den_bytes, (size_t)(ld * 4 * nrhs) * sizeof(double2)));
    GYPS_TRY(grow(m, &m->ws_v, &m->ws_v_bytes, (size_t)(ld * 3 * nrhs) * sizeof(double2)));
    double2 *u64 = reinterpret_cast<double2 *>(m->ws_den);
    double2 *S = reinterpret_cast<double2 *>(m->ws_v);
    if (prec != GYPS_PREC_FP32) {
        dim3 gi((unsigned)((m->nq + 255) / 256), (unsigned)nrhs);
        rwg_interp64_kernel<<<gi, 256, 0, s>>>(m->d_vtx, m->d_tri, m->d_tedge, m->d_pts64, m->q, m->nq, ld, X, ldx,
                                               nrhs, u64);
        GYPS_CUDA(cudaGetLastError());
    }
    const unsigned grid = (unsigned)((m->nq + 127) / 128);
    float *panel = nullptr;
    MfieArgs ma{};
    int tile_grid = 0;
    constexpr int kT = 2;
    if (prec == GYPS_PREC_FP32) {
        // the RWG panel (one right-hand side, 4 columns) sits after the FP64 densities
        const size_t b64 = ((size_t)(ld * 4 * nrhs) * sizeof(double2) + 255) / 256 * 256;
        GYPS_TRY(grow(m, &m->ws_den, &m->ws_den_bytes, b64 + (size_t)(m->n_src_tiles * den_tile_floats(4)) * sizeof(float)));
        u64 = reinterpret_cast<double2 *>(m->ws_den);
        panel = reinterpret_cast<float *>(reinterpret_cast<unsigned char *>(m->ws_den) + b64);
        GYPS_CUDA(cudaMemsetAsync(S, 0, (size_t)(ld * 3 * nrhs) * sizeof(double2), s));
        using C = MfieCfg<kT>;
        GYPS_CUDA(cudaFuncSetAttribute(far_mfie_tile_kernel<kT>, cudaFuncAttributeMaxDynamicSharedMemorySize, C::SMEM));
        int occ = 0;
        GYPS_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, far_mfie_tile_kernel<kT>, C::NT, C::SMEM));
        occ = occ > 1 ? occ : 1;
        ma.pos_panel = m->d_pos_panel;
        ma.den_panel = panel;
        ma.tgt = m->d_pts32;
        ma.ldv = ld;
        ma.nq = m->nq;
        ma.n_src_tiles = m->n_src_tiles;
        ma.n_tgt_tiles = (m->nq + C::TT - 1) / C::TT;
        ma.q = m->q;
        ma.ks = (float)k;
        ma.err = m->d_err;
        const int64_t items = ma.n_tgt_tiles * ma.n_src_tiles;
        tile_grid = (int)(items < (int64_t)m->num_sms * occ ? items : (int64_t)m->num_sms * occ);
    }
    StageTimer tf(m, s, 1);
    int launches = 0;
    for (int c0 = 0; c0 < nrhs;) {
        if (prec == GYPS_PREC_FP32) {
            const unsigned gpan = (unsigned)((m->nq_pad + 255) / 256);
            rwg_interp32_kernel<4><<<gpan, 256, 0, s>>>(m->d_vtx, m->d_tri, m->d_tedge, m->d_pts64, m->q, m->nq,
                                                        m->nq_pad, X, ldx, c0, panel);
            GYPS_CUDA(cudaGetLastError());
            ma.v = S + (int64_t)(3 * c0) * ld;
            far_mfie_tile_kernel<kT><<<(unsigned)tile_grid, MfieCfg<kT>::NT, MfieCfg<kT>::SMEM, s>>>(ma);
            c0 += 1;
        } else {
            far_mfie64_kernel<<<grid, 128, 0, s>>>(m->d_pts64, m->q, u64, ld, c0, m->nq, k, S, ld);
            c0 += 1;
        }
        GYPS_CUDA(cudaGetLastError());
        ++launches;
    }
    tf.done(launches);
    dim3 gp((unsigned)((m->ne + 127) / 128), (unsigned)nrhs);
    mfie_project_kernel<<<gp, 128, 0, s>>>(m->d_vtx, m->d_tri, m->d_tedge, m->d_etri, m->d_pts64, m->q, m->ne, S, ld,
                                           m->d_pair_ptr, m->d_pair_b, m->d_mfie_blocks, X, ldx, cm, ck,
                                           accumulate ? 1 : 0, Y, ldy);
    GYPS_CUDA(cudaGetLastError());
    return GYPS_OK;
}

// Y = sign (-beta T + (1 - beta)(Id/2 - nxK)) X, the listing's LHS.
gyps_status emcfie_apply_device(Mesh *m, double k, double beta, double sign, int nrhs, const double2 *X, int64_t ldx,
                                double2 *Y, int64_t ldy, int prec, cudaStream_t s)
{
    if (prec == GYPS_PREC_AUTO) prec = GYPS_PREC_FP32;
    if (prec != GYPS_PREC_FP64 && prec != GYPS_PREC_FP32 && prec != GYPS_PREC_DF64)
        return set_error(GYPS_ERR_UNSUPPORTED, "electromagnetic operators: FP64, FP32 or DF64");
    if (beta != 0.0) GYPS_TRY(efie_apply_device(m, k, -beta * sign, nrhs, X, ldx, Y, ldy, prec, s));
    if (beta == 1.0) return GYPS_OK;
    return mfie_apply_device(m, k, nrhs, X, ldx, Y, ldy, prec == GYPS_PREC_FP32 ? GYPS_PREC_FP32 : GYPS_PREC_FP64,
                             0.5 * sign * (1.0 - beta), -sign * (1.0 - beta), beta != 0.0, s);
}

// host / device staging shared by the electromagnetic applies (ne x nrhs)
static gyps_status em_entry(gyps_mesh_t h, double k, double beta, bool mfie_only, int nrhs, const void *X,
                            int64_t ldx, void *Y, int64_t ldy, int prec, void *stream)
{
    Mesh *m;
    GYPS_TRY(check_mesh(h, &m));
    if (nrhs < 1 || nrhs > 4096) return set_error(GYPS_ERR_INVALID, "nrhs must be in 1..4096");
    if (!X || !Y) return set_error(GYPS_ERR_INVALID, "NULL argument");
    if (!std::isfinite(k) || !(k > 0.0)) return set_error(GYPS_ERR_INVALID, "electromagnetic operators need a finite k > 0");
    if (!std::isfinite(beta)) return set_error(GYPS_ERR_INVALID, "beta must be finite");
    if (prec == GYPS_PREC_AUTO) prec = GYPS_PREC_FP32;
    if (prec == GYPS_PREC_TC_BF16X3) return set_error(GYPS_ERR_UNSUPPORTED, "electromagnetic operators: FP64, FP32 or DF64");
    if (prec != GYPS_PREC_FP64 && prec != GYPS_PREC_FP32 && prec != GYPS_PREC_DF64)
        return set_error(GYPS_ERR_INVALID, "unknown precision");
    cudaStream_t s = (cudaStream_t)stream;
    GYPS_TRY(efie_prepare(m, s));
    const int64_t ne = m->ne;
    if (ldx < ne || ldy < ne) return set_error(GYPS_ERR_INVALID, "leading dimension < number of edges");
    const bool dx = is_device_pointer(X), dy = is_device_pointer(Y);
    if (dx && dy && (const char *)X < (const char *)Y + ldy * nrhs * 16 &&
        (const char *)Y < (const char *)X + ldx * nrhs * 16)
        return set_error(GYPS_ERR_INVALID, "X and Y overlap");
    const size_t blk = (size_t)ne * nrhs * sizeof(double2);
    double2 *xs = nullptr, *ys = nullptr;
    if (!dx || !dy) {
        GYPS_TRY(grow(m, &m->ws_stage, &m->ws_stage_bytes, 2 * blk));
        xs = reinterpret_cast<double2 *>(m->ws_stage);
        ys = xs + (size_t)ne * nrhs;
    }
    const double2 *xin = (const double2 *)X;
    int64_t lxin = ldx;
    if (!dx) {
        GYPS_CUDA(cudaMemcpy2DAsync(xs, ne * sizeof(double2), X, ldx * sizeof(double2), ne * sizeof(double2), nrhs,
                                    cudaMemcpyHostToDevice, s));
        xin = xs;
        lxin = ne;
    }
    double2 *yout = dy ? (double2 *)Y : ys;
    const int64_t lyout = dy ? ldy : ne;
    GYPS_TRY(clear_err_word(m, s));  // report only the waits of this call's launches
    if (mfie_only)
        GYPS_TRY(mfie_apply_device(m, k, nrhs, xin, lxin, yout, lyout,
                                   prec == GYPS_PREC_FP32 ? GYPS_PREC_FP32 : GYPS_PREC_FP64, 0.0, 1.0, false, s));
    else
        GYPS_TRY(emcfie_apply_device(m, k, beta, 1.0, nrhs, xin, lxin, yout, lyout, prec, s));
    if (!dy)
        GYPS_CUDA(cudaMemcpy2DAsync(Y, ldy * sizeof(double2), ys, ne * sizeof(double2), ne * sizeof(double2), nrhs,
                                    cudaMemcpyDeviceToHost, s));
    GYPS_CUDA(cudaStreamSynchronize(s));
    return check_err_word(m, s);
}

}  // namespace gyps

using namespace gyps;

extern "C" gyps_status gyps_rwg_edges(gyps_mesh_t h, int64_t *ne, int32_t *edges, void *stream)
{
    Mesh *m;
    GYPS_TRY(check_mesh(h, &m));
    if (!ne) return set_error(GYPS_ERR_INVALID, "NULL argument");
    GYPS_TRY(efie_prepare(m, (cudaStream_t)stream));
    *ne = m->ne;
    if (edges) std::copy(m->h_edges.begin(), m->h_edges.end(), edges);
    return GYPS_OK;
}

extern "C" gyps_status gyps_efie_apply(gyps_mesh_t h, double k, int nrhs, const void *X, int64_t ldx, void *Y,
                                       int64_t ldy, int prec, void *stream)
{
    Mesh *m;
    GYPS_TRY(check_mesh(h, &m));
    if (nrhs < 1 || nrhs > 4096) return set_error(GYPS_ERR_INVALID, "nrhs must be in 1..4096");
    if (!X || !Y) return set_error(GYPS_ERR_INVALID, "NULL argument");
    if (!std::isfinite(k) || !(k > 0.0)) return set_error(GYPS_ERR_INVALID, "the EFIE needs a finite k > 0");
    if (prec == GYPS_PREC_AUTO) prec = GYPS_PREC_FP32;
    if (prec == GYPS_PREC_TC_BF16X3) return set_error(GYPS_ERR_UNSUPPORTED, "EFIE: FP64, FP32 or DF64");
    if (prec != GYPS_PREC_FP64 && prec != GYPS_PREC_FP32 && prec != GYPS_PREC_DF64)
        return set_error(GYPS_ERR_INVALID, "unknown precision");
    cudaStream_t s = (cudaStream_t)stream;
    GYPS_TRY(efie_prepare(m, s));
    const int64_t ne = m->ne;
    if (ldx < ne || ldy < ne) return set_error(GYPS_ERR_INVALID, "leading dimension < number of edges");
    const bool dx = is_device_pointer(X), dy = is_device_pointer(Y);
    if (dx && dy && (const char *)X < (const char *)Y + ldy * nrhs * 16 &&
        (const char *)Y < (const char *)X + ldx * nrhs * 16)
        return set_error(GYPS_ERR_INVALID, "X and Y overlap");
    const size_t blk = (size_t)ne * nrhs * sizeof(double2);
    double2 *xs = nullptr, *ys = nullptr;
    if (!dx || !dy) {
        GYPS_TRY(grow(m, &m->ws_stage, &m->ws_stage_bytes, 2 * blk));
        xs = reinterpret_cast<double2 *>(m->ws_stage);
        ys = xs + (size_t)ne * nrhs;
    }
    const double2 *xin = (const double2 *)X;
    int64_t lxin = ldx;
    if (!dx) {
        GYPS_CUDA(cudaMemcpy2DAsync(xs, ne * sizeof(double2), X, ldx * sizeof(double2), ne * sizeof(double2), nrhs,
                                    cudaMemcpyHostToDevice, s));
        xin = xs;
        lxin = ne;
    }
    double2 *yout = dy ? (double2 *)Y : ys;
    const int64_t lyout = dy ? ldy : ne;
    GYPS_TRY(clear_err_word(m, s));  // report only the waits of this call's launches
    GYPS_TRY(efie_apply_device(m, k, 1.0, nrhs, xin, lxin, yout, lyout, prec, s));
    if (!dy)
        GYPS_CUDA(cudaMemcpy2DAsync(Y, ldy * sizeof(double2), ys, ne * sizeof(double2), ne * sizeof(double2), nrhs,
                                    cudaMemcpyDeviceToHost, s));
    GYPS_CUDA(cudaStreamSynchronize(s));
    return check_err_word(m, s);
}

static gyps_status rhs_em(gyps_mesh_t h, double k, double beta, int nrhs, const double *dirs, const double *pols,
                          void *F, int64_t ldf, void *stream)
{
    Mesh *m;
    GYPS_TRY(check_mesh(h, &m));
    if (!F || !dirs || !pols) return set_error(GYPS_ERR_INVALID, "NULL argument");
    if (nrhs < 1 || nrhs > 4096) return set_error(GYPS_ERR_INVALID, "nrhs must be in 1..4096");
    if (!std::isfinite(k) || k < 0.0) return set_error(GYPS_ERR_INVALID, "k must be finite and >= 0");
    std::vector<double> dp((size_t)nrhs * 6);
    for (int j = 0; j < nrhs; ++j)
        for (int c = 0; c < 3; ++c) {
            dp[6 * j + c] = dirs[3 * j + c];
            dp[6 * j + 3 + c] = pols[3 * j + c];
        }
    for (double x : dp)
        if (!std::isfinite(x)) return set_error(GYPS_ERR_INVALID, "non-finite direction or polarisation");
    cudaStream_t s = (cudaStream_t)stream;
    GYPS_TRY(efie_prepare(m, s));
    const int64_t ne = m->ne;
    if (ldf < ne) return set_error(GYPS_ERR_INVALID, "ldf < number of edges");
    const bool df = is_device_pointer(F);
    const size_t bytes = (size_t)ne * nrhs * sizeof(double2);
    const size_t bdp = (dp.size() * sizeof(double) + 255) / 256 * 256;
    GYPS_TRY(grow(m, &m->ws_stage, &m->ws_stage_bytes, bdp + (df ? 0 : bytes)));
    unsigned char *st = reinterpret_cast<unsigned char *>(m->ws_stage);
    double *d_dp = reinterpret_cast<double *>(st);
    GYPS_CUDA(cudaMemcpyAsync(d_dp, dp.data(), dp.size() * sizeof(double), cudaMemcpyHostToDevice, s));
    double2 *fout = df ? (double2 *)F : reinterpret_cast<double2 *>(st + bdp);
    const int64_t lf = df ? ldf : ne;
    dim3 g((unsigned)((ne + 127) / 128), (unsigned)nrhs);
    efie_rhs_kernel<<<g, 128, 0, s>>>(m->d_vtx, m->d_tri, m->d_tedge, m->d_etri, m->d_pts64, m->q, ne, k, beta, d_dp,
                                      fout, lf);
    GYPS_CUDA(cudaGetLastError());
    if (!df)
        GYPS_CUDA(cudaMemcpy2DAsync(F, ldf * sizeof(double2), fout, ne * sizeof(double2), ne * sizeof(double2), nrhs,
                                    cudaMemcpyDeviceToHost, s));
    GYPS_CUDA(cudaStreamSynchronize(s));
    return GYPS_OK;
}

extern "C" gyps_status gyps_rhs_planewave_efie(gyps_mesh_t h, double k, int nrhs, const double *dirs,
                                               const double *pols, void *F, int64_t ldf, void *stream)
{
    return rhs_em(h, k, 1.0, nrhs, dirs, pols, F, ldf, stream);
}

extern "C" gyps_status gyps_rhs_planewave_emcfie(gyps_mesh_t h, double k, double beta, int nrhs, const double *dirs,
                                                 const double *pols, void *F, int64_t ldf, void *stream)
{
    if (!std::isfinite(beta)) return set_error(GYPS_ERR_INVALID, "beta must be finite");
    return rhs_em(h, k, beta, nrhs, dirs, pols, F, ldf, stream);
}

extern "C" gyps_status gyps_mfie_apply(gyps_mesh_t h, double k, int nrhs, const void *X, int64_t ldx, void *Y,
                                       int64_t ldy, int prec, void *stream)
{
    return em_entry(h, k, 0.0, true, nrhs, X, ldx, Y, ldy, prec, stream);
}

extern "C" gyps_status gyps_emcfie_apply(gyps_mesh_t h, double k, double beta, int nrhs, const void *X, int64_t ldx,
                                         void *Y, int64_t ldy, int prec, void *stream)
{
    return em_entry(h, k, beta, false, nrhs, X, ldx, Y, ldy, prec, stream);
}
