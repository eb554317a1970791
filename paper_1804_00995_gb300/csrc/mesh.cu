// Mesh handle: validation, host-side topology (vertex incidence, near pairs,
// correction pattern) and the device builds of the quadrature points (Sec. 4.2,
// Eq. approxA) and of the singular correction of Sec. 5.2.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <numeric>

#include "internal.h"
#include "p1_geom.cuh"

namespace gyps {

// ---------------------------------------------------------------- errors
static thread_local gyps_status t_last_code = GYPS_OK;
static thread_local char t_last_msg[512] = "";

gyps_status set_error(gyps_status code, const std::string &msg)
{
    t_last_code = code;
    std::snprintf(t_last_msg, sizeof(t_last_msg), "%s", msg.c_str());
    return code;
}

gyps_status cuda_error(cudaError_t e, const char *what)
{
    cudaGetLastError();  // clear a sticky non-fatal error so the next call starts clean
    std::string msg = std::string(what) + ": " + cudaGetErrorString(e);
    return set_error(e == cudaErrorMemoryAllocation ? GYPS_ERR_OOM : GYPS_ERR_CUDA, msg);
}

bool is_device_pointer(const void *p)
{
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

gyps_status enter_device(const Mesh *m)
{
    GYPS_CUDA(cudaSetDevice(m->device));
    return GYPS_OK;
}

gyps_status check_mesh(gyps_mesh_t h, Mesh **out)
{
    if (!h) return set_error(GYPS_ERR_INVALID, "mesh handle is NULL");
    *out = reinterpret_cast<Mesh *>(h);
    return enter_device(*out);
}

gyps_status grow(Mesh *m, void **buf, size_t *cap, size_t need)
{
    if (*cap >= need) return GYPS_OK;
    if (*buf) {
        GYPS_CUDA(cudaDeviceSynchronize());
        cudaFree(*buf);
        m->device_bytes -= (int64_t)*cap;
        *buf = nullptr;
        *cap = 0;
    }
    size_t n = std::max(need, (size_t)256);
    GYPS_CUDA(cudaMalloc(buf, n));
    *cap = n;
    m->device_bytes += (int64_t)n;
    return GYPS_OK;
}

template <class T>
static gyps_status dalloc(Mesh *m, T **p, size_t count)
{
    size_t bytes = std::max(count, (size_t)1) * sizeof(T);
    GYPS_CUDA(cudaMalloc((void **)p, bytes));
    m->device_bytes += (int64_t)bytes;
    return GYPS_OK;
}

// ---------------------------------------------------------------- quadrature
// Reference rules on the triangle, barycentric points and weights summing to 1.
// q = 1: centroid; q = 3: interior points (2/3, 1/6, 1/6); q = 7: Radon's
// degree-5 rule.  Filled from closed forms.
static void reference_rule(int q, double *bary, double *w)
{
    if (q == 1) {
        bary[0] = bary[1] = bary[2] = 1.0 / 3.0;
        w[0] = 1.0;
    } else if (q == 3) {
        for (int i = 0; i < 3; ++i) {
            bary[3 * i + 0] = bary[3 * i + 1] = bary[3 * i + 2] = 1.0 / 6.0;
            bary[3 * i + i] = 2.0 / 3.0;
            w[i] = 1.0 / 3.0;
        }
    } else {  // q == 7
        const double r15 = std::sqrt(15.0);
        const double orbit[2] = {(6.0 - r15) / 21.0, (6.0 + r15) / 21.0};
        const double weight[2] = {(155.0 - r15) / 1200.0, (155.0 + r15) / 1200.0};
        bary[0] = bary[1] = bary[2] = 1.0 / 3.0;
        w[0] = 0.225;
        int k = 1;
        for (int o = 0; o < 2; ++o)
            for (int i = 0; i < 3; ++i, ++k) {
                for (int c = 0; c < 3; ++c) bary[3 * k + c] = orbit[o];
                bary[3 * k + i] = 1.0 - 2.0 * orbit[o];
                w[k] = weight[o];
            }
    }
}

// a1: x_k = sum_m lambda_m(k) P_m, w_k = w_ref(k) * area, k = t*q + j (Eq. approxA).
__global__ void quad_points_kernel(const double *vtx, const int32_t *tri, int64_t nt, const Rule rule, double4_32a *pts64,
                                   float4 *pts32)
{
    const int q = rule.q;
    int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= nt * q) return;
    int64_t t = k / q;
    int j = (int)(k - t * q);
    double3 p0 = ld3(vtx, tri[3 * t]), p1 = ld3(vtx, tri[3 * t + 1]), p2 = ld3(vtx, tri[3 * t + 2]);
    double3 n = cross(p1 - p0, p2 - p0);
    double area = 0.5 * sqrt(dot(n, n));
    double3 x = rule.bary[3 * j] * p0 + rule.bary[3 * j + 1] * p1 + rule.bary[3 * j + 2] * p2;
    double w = rule.w[j] * area;
    pts64[k] = make_double4_32a(x.x, x.y, x.z, w);
    pts32[k] = make_float4((float)x.x, (float)x.y, (float)x.z, (float)w);
}

// FP32 position panel: negated coordinates, source pairs interleaved (see internal.h).
__global__ void pos_panel_kernel(const double4_32a *pts64, int64_t nq, int64_t nq_pad, float pad, float *panel)
{
    int64_t l = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (l >= nq_pad) return;
    float x = pad, y = pad, z = pad;
    if (l < nq) {
        double4_32a p = pts64[l];
        x = (float)p.x;
        y = (float)p.y;
        z = (float)p.z;
    }
    int64_t tile = l / kSrcTile;
    int p = (int)(l % kSrcTile) >> 1, lane = (int)(l & 1);
    float *base = panel + tile * kPosTileFloats;
    base[4 * p + lane] = -x;
    base[4 * p + 2 + lane] = -y;
    base[4 * kSrcPairs + 2 * p + lane] = -z;
}

cudaError_t launch_quad_points(const Mesh &m, cudaStream_t s)
{
    int64_t n = m.nq;
    quad_points_kernel<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(m.d_vtx, m.d_tri, m.nt, m.rule, m.d_pts64, m.d_pts32);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    return cudaSuccess;
}

// a5b: one thread per ordered near pair (a, b): for each quadrature point x_k of
// a, the analytic y-integral over b minus the Gauss sum over the points of b
// (the point paired with itself left out when a == b), weighted by
// w_k lambda_i(x_k) / (4 pi).  block[3 i + j]: test vertex i of a, trial j of b.
__global__ void near_blocks_kernel(const double *vtx, const int32_t *tri, const double4_32a *pts64, const Rule rule,
                                   int64_t npairs, const int32_t *pair_a, const int32_t *pair_b, double *blocks)
{
    const int q = rule.q;
    int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= npairs) return;
    int a = pair_a[p], b = pair_b[p];
    double3 B[3] = {ld3(vtx, tri[3 * (int64_t)b]), ld3(vtx, tri[3 * (int64_t)b + 1]), ld3(vtx, tri[3 * (int64_t)b + 2])};
    double acc[9];
#pragma unroll
    for (int e = 0; e < 9; ++e) acc[e] = 0.0;
    const double inv4pi = 0.25 / 3.141592653589793238462643383279502884;
    for (int kq = 0; kq < q; ++kq) {
        double4_32a xk4 = pts64[(int64_t)a * q + kq];
        double3 xk = make_double3(xk4.x, xk4.y, xk4.z);
        double exact[3];
        p1_over_r(xk, B, exact);
        double gauss[3] = {0.0, 0.0, 0.0};
        for (int lq = 0; lq < q; ++lq) {
            if (a == b && lq == kq) continue;
            double4_32a yl = pts64[(int64_t)b * q + lq];
            double3 d = make_double3(xk.x - yl.x, xk.y - yl.y, xk.z - yl.z);
            double wr = yl.w / sqrt(dot(d, d));
#pragma unroll
            for (int j = 0; j < 3; ++j) gauss[j] += wr * rule.bary[3 * lq + j];
        }
        double wk = xk4.w * inv4pi;
#pragma unroll
        for (int i = 0; i < 3; ++i)
#pragma unroll
            for (int j = 0; j < 3; ++j) acc[3 * i + j] += wk * rule.bary[3 * kq + i] * (exact[j] - gauss[j]);
    }
#pragma unroll
    for (int e = 0; e < 9; ++e) blocks[9 * p + e] = acc[e];
}

// Each nonzero of C sums its block entries in a fixed order (deterministic).
__global__ void near_gather_kernel(int64_t nnz, const int32_t *src_ptr, const int32_t *src, const double *blocks,
                                   double *val)
{
    int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= nnz) return;
    double s = 0.0;
    for (int32_t e = src_ptr[c]; e < src_ptr[c + 1]; ++e) s += blocks[src[e]];
    val[c] = s;
}

cudaError_t launch_near_build(const Mesh &m, cudaStream_t s)
{
    near_blocks_kernel<<<(unsigned)((m.npairs + 127) / 128), 128, 0, s>>>(m.d_vtx, m.d_tri, m.d_pts64, m.rule, m.npairs,
                                                                         m.d_pair_a, m.d_pair_b, m.d_blocks);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    near_gather_kernel<<<(unsigned)((m.c_nnz + 255) / 256), 256, 0, s>>>(m.c_nnz, m.d_c_src_ptr, m.d_c_src,
                                                                        m.d_blocks, m.d_c_val);
    return cudaGetLastError();
}

// ---------------------------------------------------------------- host topology
static void build_topology(Mesh &m, const int32_t *tri, std::vector<int32_t> &v2t_ptr, std::vector<int32_t> &v2t,
                           std::vector<int32_t> &pair_a, std::vector<int32_t> &pair_b, std::vector<int32_t> &pair_ptr,
                           std::vector<int32_t> &c_src_ptr, std::vector<int32_t> &c_src)
{
    const int64_t nv = m.nv, nt = m.nt;
    // vertex -> (triangle, local index), triangles ascending
    v2t_ptr.assign(nv + 1, 0);
    for (int64_t e = 0; e < 3 * nt; ++e) v2t_ptr[tri[e] + 1]++;
    for (int64_t i = 0; i < nv; ++i) v2t_ptr[i + 1] += v2t_ptr[i];
    v2t.resize(3 * nt);
    std::vector<int32_t> fill(v2t_ptr.begin(), v2t_ptr.end() - 1);
    for (int64_t e = 0; e < 3 * nt; ++e) v2t[fill[tri[e]]++] = (int32_t)e;

    // ordered pairs of triangles sharing at least one vertex, sorted by (a, b)
    pair_ptr.assign(nt + 1, 0);
    pair_a.clear();
    pair_b.clear();
    std::vector<int32_t> nb;
    for (int64_t a = 0; a < nt; ++a) {
        nb.clear();
        for (int c = 0; c < 3; ++c) {
            int32_t v = tri[3 * a + c];
            for (int32_t e = v2t_ptr[v]; e < v2t_ptr[v + 1]; ++e) nb.push_back(v2t[e] / 3);
        }
        std::sort(nb.begin(), nb.end());
        nb.erase(std::unique(nb.begin(), nb.end()), nb.end());
        for (int32_t b : nb) {
            pair_a.push_back((int32_t)a);
            pair_b.push_back(b);
        }
        pair_ptr[a + 1] = (int32_t)pair_a.size();
    }
    const int64_t np = (int64_t)pair_a.size();

    // pattern of C: row v_i(a), column v_j(b) for every pair and local i, j
    std::vector<int64_t> cnt(nv + 1, 0);
    for (int64_t p = 0; p < np; ++p)
        for (int i = 0; i < 3; ++i) cnt[tri[3 * (int64_t)pair_a[p] + i] + 1] += 3;
    for (int64_t i = 0; i < nv; ++i) cnt[i + 1] += cnt[i];
    std::vector<int32_t> cand(cnt[nv]);
    std::vector<int64_t> pos(cnt.begin(), cnt.end() - 1);
    for (int64_t p = 0; p < np; ++p)
        for (int i = 0; i < 3; ++i) {
            int32_t r = tri[3 * (int64_t)pair_a[p] + i];
            for (int j = 0; j < 3; ++j) cand[pos[r]++] = tri[3 * (int64_t)pair_b[p] + j];
        }
    m.h_c_rowptr.assign(nv + 1, 0);
    m.h_c_col.clear();
    for (int64_t r = 0; r < nv; ++r) {
        auto b = cand.begin() + cnt[r], e = cand.begin() + cnt[r + 1];
        std::sort(b, e);
        auto u = std::unique(b, e);
        m.h_c_col.insert(m.h_c_col.end(), b, u);
        m.h_c_rowptr[r + 1] = (int32_t)m.h_c_col.size();
    }
    m.c_nnz = (int64_t)m.h_c_col.size();
    m.npairs = np;

    // block entry (9 p + 3 i + j) -> nonzero slot; then invert into per-slot lists
    std::vector<int32_t> slot(9 * np);
    for (int64_t p = 0; p < np; ++p)
        for (int i = 0; i < 3; ++i) {
            int32_t r = tri[3 * (int64_t)pair_a[p] + i];
            auto b = m.h_c_col.begin() + m.h_c_rowptr[r], e = m.h_c_col.begin() + m.h_c_rowptr[r + 1];
            for (int j = 0; j < 3; ++j) {
                int32_t c = tri[3 * (int64_t)pair_b[p] + j];
                slot[9 * p + 3 * i + j] = (int32_t)(std::lower_bound(b, e, c) - m.h_c_col.begin());
            }
        }
    c_src_ptr.assign(m.c_nnz + 1, 0);
    for (int64_t e = 0; e < 9 * np; ++e) c_src_ptr[slot[e] + 1]++;
    for (int64_t c = 0; c < m.c_nnz; ++c) c_src_ptr[c + 1] += c_src_ptr[c];
    c_src.resize(9 * np);
    std::vector<int32_t> f2(c_src_ptr.begin(), c_src_ptr.end() - 1);
    for (int64_t e = 0; e < 9 * np; ++e) c_src[f2[slot[e]]++] = (int32_t)e;
}

static void free_mesh(Mesh *m)
{
    if (!m) return;
    void *ptrs[] = {m->d_vtx, m->d_tri, m->d_pts64, m->d_pts32, m->d_pos_panel, m->d_v2t_ptr, m->d_v2t,
                    m->d_pair_a, m->d_pair_b, m->d_pair_ptr, m->d_blocks, m->d_c_rowptr, m->d_c_col,
                    m->d_c_val, m->d_c_src_ptr, m->d_c_src, m->d_err, m->ws_den, m->ws_v, m->ws_stage, m->ws_tc,
                    m->d_adj_ptr, m->d_adj, m->d_vfeat, m->ws_pts, m->d_tri_cen, m->d_tri_cen32, m->d_tri_nrm,
                    m->d_cdl_val, m->ws_bw, m->d_nrm_panel, m->d_cdlT_val, m->d_tedge, m->d_etri,
                    m->d_efie_blocks, m->d_mfie_blocks};
    for (void *p : ptrs)
        if (p) cudaFree(p);
    free_vertex_tiles(m->vt);
    delete m;
}

template <class T>
static gyps_status upload(Mesh *m, T **dst, const std::vector<T> &src, cudaStream_t s)
{
    GYPS_TRY(dalloc(m, dst, src.size()));
    if (!src.empty()) GYPS_CUDA(cudaMemcpyAsync(*dst, src.data(), src.size() * sizeof(T), cudaMemcpyHostToDevice, s));
    return GYPS_OK;
}

static gyps_status create(const double *vtx, int64_t nv, const int32_t *tri, int64_t nt, int q, cudaStream_t s,
                          Mesh *m)
{
    GYPS_CUDA(cudaGetDevice(&m->device));
    GYPS_CUDA(cudaDeviceGetAttribute(&m->num_sms, cudaDevAttrMultiProcessorCount, m->device));
    m->nv = nv;
    m->nt = nt;
    m->q = q;
    m->nq = nt * q;
    m->n_src_tiles = (m->nq + kSrcTile - 1) / kSrcTile;
    m->nq_pad = m->n_src_tiles * kSrcTile;

    std::vector<int32_t> v2t_ptr, v2t, pa, pb, pptr, csp, cs;
    build_topology(*m, tri, v2t_ptr, v2t, pa, pb, pptr, csp, cs);
    if (9 * m->npairs > INT32_MAX || 3 * nt > INT32_MAX)
        return set_error(GYPS_ERR_INVALID, "mesh too large for 32-bit incidence indices");

    double ext = 0.0;
    for (int64_t i = 0; i < 3 * nv; ++i) ext = std::max(ext, std::fabs(vtx[i]));
    const float pad = (float)(1.0e3 * (1.0 + ext));
    m->pad = pad;

    m->rule.q = q;
    reference_rule(q, m->rule.bary, m->rule.w);
    std::vector<double> hv(vtx, vtx + 3 * nv);
    std::vector<int32_t> ht(tri, tri + 3 * nt);
    GYPS_TRY(upload(m, &m->d_vtx, hv, s));
    GYPS_TRY(upload(m, &m->d_tri, ht, s));
    GYPS_TRY(upload(m, &m->d_v2t_ptr, v2t_ptr, s));
    GYPS_TRY(upload(m, &m->d_v2t, v2t, s));
    GYPS_TRY(upload(m, &m->d_pair_a, pa, s));
    GYPS_TRY(upload(m, &m->d_pair_b, pb, s));
    GYPS_TRY(upload(m, &m->d_pair_ptr, pptr, s));
    m->h_pair_ptr = pptr;
    GYPS_TRY(upload(m, &m->d_c_rowptr, m->h_c_rowptr, s));
    GYPS_TRY(upload(m, &m->d_c_col, m->h_c_col, s));
    GYPS_TRY(upload(m, &m->d_c_src_ptr, csp, s));
    GYPS_TRY(upload(m, &m->d_c_src, cs, s));
    GYPS_TRY(dalloc(m, &m->d_pts64, m->nq));
    GYPS_TRY(dalloc(m, &m->d_pts32, m->nq));
    GYPS_TRY(dalloc(m, &m->d_pos_panel, (size_t)(m->n_src_tiles * kPosTileFloats)));
    GYPS_TRY(dalloc(m, &m->d_blocks, (size_t)(9 * m->npairs)));
    GYPS_TRY(dalloc(m, &m->d_c_val, (size_t)m->c_nnz));
    GYPS_TRY(dalloc(m, &m->d_err, 1));
    GYPS_CUDA(cudaMemsetAsync(m->d_err, 0, sizeof(int), s));

    GYPS_CUDA(launch_quad_points(*m, s));
    pos_panel_kernel<<<(unsigned)((m->nq_pad + 255) / 256), 256, 0, s>>>(m->d_pts64, m->nq, m->nq_pad, pad,
                                                                       m->d_pos_panel);
    GYPS_CUDA(cudaGetLastError());
    GYPS_CUDA(launch_near_build(*m, s));
    GYPS_CUDA(cudaStreamSynchronize(s));  // host vectors above go out of scope
    return GYPS_OK;
}

}  // namespace gyps

using namespace gyps;

extern "C" const char *gyps_version(void) { return "gyps 0.1 (sm_103a)"; }

extern "C" gyps_status gyps_last_error(char *buf, size_t n)
{
    if (buf && n) std::snprintf(buf, n, "%s", t_last_msg);
    return t_last_code;
}

extern "C" gyps_status gyps_mesh_create(const double *vtx, int64_t nv, const int32_t *tri, int64_t nt,
                                        int quad_points, uint32_t flags, void *stream, gyps_mesh_t *out)
{
    if (!out) return set_error(GYPS_ERR_INVALID, "out is NULL");
    *out = nullptr;
    if (!vtx || !tri) return set_error(GYPS_ERR_INVALID, "vtx or tri is NULL");
    if (nv < 3 || nt < 1) return set_error(GYPS_ERR_INVALID, "need nv >= 3 and nt >= 1");
    if (nv > INT32_MAX || nt > INT32_MAX / 9) return set_error(GYPS_ERR_INVALID, "mesh too large");
    if (quad_points != 1 && quad_points != 3 && quad_points != 7)
        return set_error(GYPS_ERR_INVALID, "quad_points must be 1, 3 or 7");
    if (flags != 0) return set_error(GYPS_ERR_INVALID, "flags must be 0");
    if (is_device_pointer(vtx) || is_device_pointer(tri))
        return set_error(GYPS_ERR_INVALID, "vtx and tri must be host pointers");
    for (int64_t i = 0; i < 3 * nv; ++i)
        if (!std::isfinite(vtx[i])) return set_error(GYPS_ERR_INVALID, "non-finite vertex coordinate");
    for (int64_t t = 0; t < nt; ++t) {
        const int32_t *v = tri + 3 * t;
        for (int c = 0; c < 3; ++c)
            if (v[c] < 0 || v[c] >= nv)
                return set_error(GYPS_ERR_INVALID, "triangle " + std::to_string(t) + " has a vertex index out of range");
        if (v[0] == v[1] || v[1] == v[2] || v[0] == v[2])
            return set_error(GYPS_ERR_INVALID, "triangle " + std::to_string(t) + " repeats a vertex");
        const double *a = vtx + 3 * (int64_t)v[0], *b = vtx + 3 * (int64_t)v[1], *c = vtx + 3 * (int64_t)v[2];
        double e1[3] = {b[0] - a[0], b[1] - a[1], b[2] - a[2]}, e2[3] = {c[0] - a[0], c[1] - a[1], c[2] - a[2]};
        double n[3] = {e1[1] * e2[2] - e1[2] * e2[1], e1[2] * e2[0] - e1[0] * e2[2], e1[0] * e2[1] - e1[1] * e2[0]};
        double n2 = n[0] * n[0] + n[1] * n[1] + n[2] * n[2];
        double l2 = std::max(e1[0] * e1[0] + e1[1] * e1[1] + e1[2] * e1[2], e2[0] * e2[0] + e2[1] * e2[1] + e2[2] * e2[2]);
        if (!(n2 > 1e-24 * l2 * l2))
            return set_error(GYPS_ERR_INVALID, "triangle " + std::to_string(t) + " has zero area");
    }
    Mesh *m = new Mesh();
    gyps_status st = create(vtx, nv, tri, nt, quad_points, (cudaStream_t)stream, m);
    if (st != GYPS_OK) {
        cudaDeviceSynchronize();
        free_mesh(m);
        return st;
    }
    *out = reinterpret_cast<gyps_mesh_t>(m);
    return GYPS_OK;
}

extern "C" gyps_status gyps_mesh_destroy(gyps_mesh_t h)
{
    if (!h) return GYPS_OK;
    Mesh *m = reinterpret_cast<Mesh *>(h);
    cudaSetDevice(m->device);
    cudaDeviceSynchronize();
    free_mesh(m);
    return GYPS_OK;
}

extern "C" gyps_status gyps_mesh_info(gyps_mesh_t h, gyps_mesh_info_t *info)
{
    Mesh *m;
    GYPS_TRY(check_mesh(h, &m));
    if (!info) return set_error(GYPS_ERR_INVALID, "info is NULL");
    info->nv = m->nv;
    info->nt = m->nt;
    info->nq = m->nq;
    info->q = m->q;
    info->device = m->device;
    info->near_pairs = m->npairs;
    info->near_nnz = m->c_nnz;
    info->device_bytes = m->device_bytes;
    return GYPS_OK;
}

extern "C" gyps_status gyps_quad_points(gyps_mesh_t h, double *xw, void *stream)
{
    Mesh *m;
    GYPS_TRY(check_mesh(h, &m));
    if (!xw) return set_error(GYPS_ERR_INVALID, "xw is NULL");
    cudaStream_t s = (cudaStream_t)stream;
    GYPS_CUDA(cudaMemcpyAsync(xw, m->d_pts64, m->nq * sizeof(double4_32a), cudaMemcpyDefault, s));
    if (!is_device_pointer(xw)) GYPS_CUDA(cudaStreamSynchronize(s));
    return GYPS_OK;
}

extern "C" gyps_status gyps_near_export(gyps_mesh_t h, int64_t *rowptr, int32_t *col, double *val)
{
    Mesh *m;
    GYPS_TRY(check_mesh(h, &m));
    if (!rowptr || !col || !val) return set_error(GYPS_ERR_INVALID, "NULL output buffer");
    for (int64_t i = 0; i <= m->nv; ++i) rowptr[i] = m->h_c_rowptr[i];
    std::memcpy(col, m->h_c_col.data(), m->c_nnz * sizeof(int32_t));
    GYPS_CUDA(cudaDeviceSynchronize());
    GYPS_CUDA(cudaMemcpy(val, m->d_c_val, m->c_nnz * sizeof(double), cudaMemcpyDeviceToHost));
    return GYPS_OK;
}
