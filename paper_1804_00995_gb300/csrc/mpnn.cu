// Learned preconditioner: a message-passing network on the P1 mesh graph that
// maps a residual r to an approximate correction z ~ V^{-1} r, for flexible
// GMRES.  Not in the paper; the operator it approximates is the single layer of
// Sec. 5 / Sec. 5.4.
//
// Network (H hidden features, L layers, bf16 weights, FP32 activations and sums):
//   f_i   = [Re r_i / s, Im r_i / s, x^_i, y^_i, z^_i, n_i, k h]   (s = rms(r))
//   h0    = relu(W_in f + b_in)
//   m_l   = mean over the mesh neighbours j of i of h_l(j)
//   h_l+1 = h_l + relu(Ws_l h_l + Wn_l m_l + b_l)                  l = 0 .. L-1
//   y     = W_out h_L + b_out,   z_i = (y_i0 + i y_i1) s / h^3       (h = mean edge length)
// Training: one minibatch = B residuals of one mesh with their corrections e;
// loss = (1/B) sum_b |z_b - e_b|^2 / |e_b|^2; hand-written backward kernels;
// Adam on FP32 master weights, bf16 copies for the forward.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <vector>

#include <cuda_bf16.h>

#include "internal.h"

namespace gyps {
namespace mp {

constexpr int NIN = 9;

// ---------------------------------------------------------------- kernels
__global__ void sumsq_kernel(const double2 *R, int64_t ld, int64_t nv, double *out)
{
    const int b = blockIdx.y;
    double s = 0.0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < nv; i += (int64_t)gridDim.x * blockDim.x) {
        const double2 r = R[i + (int64_t)b * ld];
        s += r.x * r.x + r.y * r.y;
    }
    for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
    __shared__ double red[32];
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int k = 0; k < (int)(blockDim.x >> 5); ++k) t += red[k];
        atomicAdd(&out[b], t);
    }
}

__global__ void features_kernel(const double2 *R, int64_t ldr, const float *vfeat, int64_t nv, int B,
                                const double *rsum, float kh, float *F)
{
    const int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= nv * B) return;
    const int b = (int)(g / nv);
    const int64_t i = g - (int64_t)b * nv;
    const double s = sqrt(rsum[b] / (double)nv);
    const double inv = s > 0.0 ? 1.0 / s : 0.0;
    const double2 r = R[i + (int64_t)b * ldr];
    float *f = F + g * NIN;
    f[0] = (float)(r.x * inv);
    f[1] = (float)(r.y * inv);
    for (int c = 0; c < 6; ++c) f[2 + c] = vfeat[6 * i + c];
    f[8] = kh;
}

// Y[r][o] = act(X1[r] . W1[:, o] + X2[r] . W2[:, o] + b[o]) (+ RES[r][o]); A = pre-activation.
template <int I1, int I2, int O, bool RELU, bool RES>
__global__ void dense_kernel(const float *X1, const float *X2, const __nv_bfloat16 *W1, const __nv_bfloat16 *W2,
                             const __nv_bfloat16 *bias, const float *RESin, float *A, float *Y, int64_t rows)
{
    constexpr int RPB = O >= 64 ? 1024 / O : 64;  // rows per block
    __shared__ float w1[I1 * O];
    __shared__ float w2[(I2 > 0 ? I2 : 1) * O];
    __shared__ float x[RPB][I1 + I2 + 1];
    const int o = threadIdx.x, rr = threadIdx.y;
    const int tid = rr * O + o;
    for (int e = tid; e < I1 * O; e += O * RPB) w1[e] = __bfloat162float(W1[e]);
    if (I2 > 0)
        for (int e = tid; e < I2 * O; e += O * RPB) w2[e] = __bfloat162float(W2[e]);
    const int64_t row0 = (int64_t)blockIdx.x * RPB;
    for (int e = tid; e < RPB * (I1 + I2); e += O * RPB) {
        const int r = e / (I1 + I2), c = e - r * (I1 + I2);
        const int64_t row = row0 + r;
        float val = 0.0f;
        if (row < rows) val = c < I1 ? X1[row * I1 + c] : X2[row * I2 + (c - I1)];
        x[r][c] = val;
    }
    __syncthreads();
    const int64_t row = row0 + rr;
    if (row >= rows) return;
    float acc = __bfloat162float(bias[o]);
#pragma unroll 8
    for (int i = 0; i < I1; ++i) acc = fmaf(x[rr][i], w1[i * O + o], acc);
    if (I2 > 0) {
#pragma unroll 8
        for (int i = 0; i < I2; ++i) acc = fmaf(x[rr][I1 + i], w2[i * O + o], acc);
    }
    if (A) A[row * O + o] = acc;
    float y = RELU ? fmaxf(acc, 0.0f) : acc;
    if (RES) y += RESin[row * O + o];
    Y[row * O + o] = y;
}

// The same layer for 64 outputs, register-tiled: a block of 64 x 16 threads
// covers 64 rows (thread (o, ry): output o of rows 4 ry .. 4 ry + 3), the
// weights go to shared memory once per 64 rows, and per 4 inputs a thread makes
// 4 weight loads and 4 broadcast float4 loads of x for 16 FMAs.  Inputs are
// padded to a multiple of 4 with zero weights.
template <int I1, int I2>
constexpr int dense64_smem()
{
    return 2 * (((I1 + I2) + 3) & ~3) * 64 * (int)sizeof(float);
}

template <int I1, int I2, bool RELU, bool RES>
__global__ void __launch_bounds__(1024) dense64_kernel(const float *X1, const float *X2, const __nv_bfloat16 *W1,
                                                       const __nv_bfloat16 *W2, const __nv_bfloat16 *bias,
                                                       const float *RESin, float *A, float *Y, int64_t rows)
{
    constexpr int O = 64, RPT = 4, RPB = 16 * RPT, IN = I1 + I2, INP = (IN + 3) & ~3;
    extern __shared__ __align__(16) float dsm[];
    float *w = dsm;            // [INP][O]
    float *x = dsm + INP * O;  // [RPB][INP]
    const int o = threadIdx.x, ry = threadIdx.y, tid = ry * O + o;
    for (int e = tid; e < INP * O; e += O * 16) {
        const int i = e / O, oo = e - i * O;
        float v = 0.0f;
        if (i < I1)
            v = __bfloat162float(W1[i * O + oo]);
        else if (i < IN)
            v = __bfloat162float(W2[(i - I1) * O + oo]);
        w[e] = v;
    }
    const int64_t row0 = (int64_t)blockIdx.x * RPB;
    for (int e = tid; e < RPB * INP; e += O * 16) {
        const int r = e / INP, c = e - r * INP;
        const int64_t row = row0 + r;
        float v = 0.0f;
        if (row < rows && c < IN) v = c < I1 ? X1[row * I1 + c] : X2[row * I2 + (c - I1)];
        x[e] = v;
    }
    __syncthreads();
    const float b0 = __bfloat162float(bias[o]);
    float acc[RPT];
#pragma unroll
    for (int r = 0; r < RPT; ++r) acc[r] = b0;
#pragma unroll 4
    for (int i = 0; i < INP; i += 4) {
        const float w0 = w[i * O + o], w1 = w[(i + 1) * O + o], w2 = w[(i + 2) * O + o], w3 = w[(i + 3) * O + o];
#pragma unroll
        for (int r = 0; r < RPT; ++r) {
            const float4 xv = *reinterpret_cast<const float4 *>(&x[(ry * RPT + r) * INP + i]);
            acc[r] = fmaf(xv.x, w0, acc[r]);
            acc[r] = fmaf(xv.y, w1, acc[r]);
            acc[r] = fmaf(xv.z, w2, acc[r]);
            acc[r] = fmaf(xv.w, w3, acc[r]);
        }
    }
#pragma unroll
    for (int r = 0; r < RPT; ++r) {
        const int64_t row = row0 + ry * RPT + r;
        if (row >= rows) continue;
        if (A) A[row * O + o] = acc[r];
        float y = RELU ? fmaxf(acc[r], 0.0f) : acc[r];
        if (RES) y += RESin[row * O + o];
        Y[row * O + o] = y;
    }
}

// M[b, i, :] = mean over neighbours j of H[b, j, :]
__global__ void gather_mean_kernel(const int32_t *adj_ptr, const int32_t *adj, const float *Hin, int64_t nv, int B,
                                   int Hd, float *M)
{
    const int64_t g = (int64_t)blockIdx.x * blockDim.y + threadIdx.y;  // (b, i)
    const int k = threadIdx.x;
    if (g >= nv * B) return;
    const int b = (int)(g / nv);
    const int64_t i = g - (int64_t)b * nv;
    const int32_t p0 = adj_ptr[i], p1 = adj_ptr[i + 1];
    float s = 0.0f;
    for (int32_t p = p0; p < p1; ++p) s += Hin[((int64_t)b * nv + adj[p]) * Hd + k];
    M[g * Hd + k] = p1 > p0 ? s / (float)(p1 - p0) : 0.0f;
}

// OUT[b, j, :] += sum over neighbours i of j of G[b, i, :] / deg(i)   (transpose of the mean)
__global__ void gather_tmean_kernel(const int32_t *adj_ptr, const int32_t *adj, const float *G, int64_t nv, int B,
                                    int Hd, float *OUT)
{
    const int64_t g = (int64_t)blockIdx.x * blockDim.y + threadIdx.y;
    const int k = threadIdx.x;
    if (g >= nv * B) return;
    const int b = (int)(g / nv);
    const int64_t j = g - (int64_t)b * nv;
    float s = 0.0f;
    for (int32_t p = adj_ptr[j]; p < adj_ptr[j + 1]; ++p) {
        const int32_t i = adj[p];
        const int32_t deg = adj_ptr[i + 1] - adj_ptr[i];
        s += G[((int64_t)b * nv + i) * Hd + k] / (float)deg;
    }
    OUT[g * Hd + k] += s;
}

__global__ void output_kernel(const float *Yo, const double *rsum, int64_t nv, int B, double inv_h3, double2 *Z,
                              int64_t ldz)
{
    const int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= nv * B) return;
    const int b = (int)(g / nv);
    const int64_t i = g - (int64_t)b * nv;
    const double s = sqrt(rsum[b] / (double)nv) * inv_h3;
    Z[i + (int64_t)b * ldz] = make_double2(Yo[2 * g] * s, Yo[2 * g + 1] * s);
}

// loss_b = |z_b - e_b|^2 / |e_b|^2 (summed into loss[b]); dY = d(mean_b loss_b)/dY
__global__ void loss_grad_kernel(const double2 *Z, int64_t ldz, const double2 *E, int64_t lde, const double *esum,
                                 const double *rsum, int64_t nv, int B, double inv_h3, float *dY, double *loss)
{
    const int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    double l = 0.0;
    int b = 0;
    if (g < nv * B) {
        b = (int)(g / nv);
        const int64_t i = g - (int64_t)b * nv;
        const double2 z = Z[i + (int64_t)b * ldz], e = E[i + (int64_t)b * lde];
        const double dr = z.x - e.x, di = z.y - e.y;
        const double den = esum[b] > 0.0 ? esum[b] : 1.0;
        l = (dr * dr + di * di) / den;
        const double s = sqrt(rsum[b] / (double)nv) * inv_h3;
        const double c = 2.0 * s / ((double)B * den);
        dY[2 * g] = (float)(c * dr);
        dY[2 * g + 1] = (float)(c * di);
    }
    // block-level partial sums per column: columns can change inside a block, so add per thread
    if (g < nv * B) atomicAdd(&loss[b], l);
}

__global__ void relu_bwd_kernel(const float *dH, const float *A, int64_t n, float *dA)
{
    const int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (g < n) dA[g] = A[g] > 0.0f ? dH[g] : 0.0f;
}

// dX[r][i] (+)= sum_o dA[r][o] W[i][o]
template <int I, int O, bool ACC>
__global__ void dense_bwd_x_kernel(const float *dA, const __nv_bfloat16 *W, float *dX, int64_t rows)
{
    constexpr int RPB = 1024 / I;
    __shared__ float w[I * O];
    __shared__ float d[RPB][O + 1];
    const int i = threadIdx.x, rr = threadIdx.y;
    const int tid = rr * I + i;
    for (int e = tid; e < I * O; e += I * RPB) w[e] = __bfloat162float(W[e]);
    const int64_t row0 = (int64_t)blockIdx.x * RPB;
    for (int e = tid; e < RPB * O; e += I * RPB) {
        const int r = e / O, c = e - r * O;
        const int64_t row = row0 + r;
        d[r][c] = row < rows ? dA[row * O + c] : 0.0f;
    }
    __syncthreads();
    const int64_t row = row0 + rr;
    if (row >= rows) return;
    float acc = 0.0f;
#pragma unroll 8
    for (int o = 0; o < O; ++o) acc = fmaf(d[rr][o], w[i * O + o], acc);
    if (ACC)
        dX[row * I + i] += acc;
    else
        dX[row * I + i] = acc;
}

// dW[i][o] += sum_r X[r][i] dA[r][o];  db[o] += sum_r dA[r][o]
template <int I, int O>
__global__ void wgrad_kernel(const float *X, const float *dA, int64_t rows, float *dW, float *db)
{
    constexpr int CH = 32;  // rows per chunk
    constexpr int NOUT = I * O;
    __shared__ float xs[CH][I];
    __shared__ float ds[CH][O];
    float acc[(NOUT + 255) / 256];
    float bacc = 0.0f;
#pragma unroll
    for (int e = 0; e < (NOUT + 255) / 256; ++e) acc[e] = 0.0f;
    for (int64_t r0 = (int64_t)blockIdx.x * CH; r0 < rows; r0 += (int64_t)gridDim.x * CH) {
        __syncthreads();
        for (int e = threadIdx.x; e < CH * I; e += 256) {
            const int r = e / I, c = e - r * I;
            xs[r][c] = (r0 + r < rows) ? X[(r0 + r) * I + c] : 0.0f;
        }
        for (int e = threadIdx.x; e < CH * O; e += 256) {
            const int r = e / O, c = e - r * O;
            ds[r][c] = (r0 + r < rows) ? dA[(r0 + r) * O + c] : 0.0f;
        }
        __syncthreads();
#pragma unroll
        for (int e = 0; e < (NOUT + 255) / 256; ++e) {
            const int idx = threadIdx.x + e * 256;
            if (idx < NOUT) {
                const int i = idx / O, o = idx - i * O;
                float s = acc[e];
                for (int r = 0; r < CH; ++r) s = fmaf(xs[r][i], ds[r][o], s);
                acc[e] = s;
            }
        }
        if (db && threadIdx.x < O)
            for (int r = 0; r < CH; ++r) bacc += ds[r][threadIdx.x];
    }
#pragma unroll
    for (int e = 0; e < (NOUT + 255) / 256; ++e) {
        const int idx = threadIdx.x + e * 256;
        if (idx < NOUT) atomicAdd(&dW[idx], acc[e]);
    }
    if (db && threadIdx.x < O) atomicAdd(&db[threadIdx.x], bacc);
}

__global__ void adam_kernel(float *p, const float *g, float *m, float *v, int64_t n, float lr, float b1, float b2,
                            float eps, float c1, float c2, __nv_bfloat16 *pb)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float gi = g[i];
    const float mi = b1 * m[i] + (1.0f - b1) * gi;
    const float vi = b2 * v[i] + (1.0f - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    const float pi = p[i] - lr * (mi / c1) / (sqrtf(vi / c2) + eps);
    p[i] = pi;
    pb[i] = __float2bfloat16_rn(pi);
}

__global__ void to_bf16_kernel(const float *p, int64_t n, __nv_bfloat16 *pb)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) pb[i] = __float2bfloat16_rn(p[i]);
}

}  // namespace mp

// ---------------------------------------------------------------- model
struct Mpnn {
    int H = 64, L = 4;
    int64_t nparams = 0;
    int64_t off_win = 0, off_bin = 0, off_ws0 = 0, off_wout = 0, off_bout = 0;
    int64_t layer_stride = 0;  // Ws, Wn, b per layer
    float *p = nullptr, *g = nullptr, *m = nullptr, *v = nullptr;
    __nv_bfloat16 *pb = nullptr;
    int64_t step = 0;
    int device = 0;
    // electrical sizes k x radius of the meshes trained on (lo > hi: none yet)
    double ka_lo = 1e300, ka_hi = -1e300;
    // activation workspace
    float *ws = nullptr;
    size_t ws_bytes = 0;
    double *red = nullptr;  // per-column reductions (3 x 4096)
    ~Mpnn()
    {
        cudaFree(p);
        cudaFree(g);
        cudaFree(m);
        cudaFree(v);
        cudaFree(pb);
        cudaFree(ws);
        cudaFree(red);
    }
    int64_t ws_off(int l) const { return off_ws0 + (int64_t)l * layer_stride; }
    int64_t wn_off(int l) const { return ws_off(l) + (int64_t)H * H; }
    int64_t b_off(int l) const { return ws_off(l) + 2 * (int64_t)H * H; }
};

// Mesh-side graph data for the network: vertex neighbours (CSR over mesh edges),
// normalised coordinates and vertex normals, mean edge length.
static gyps_status ensure_graph(Mesh *m, cudaStream_t s)
{
    if (m->d_adj_ptr) return GYPS_OK;
    std::vector<double> vtx(3 * m->nv);
    std::vector<int32_t> tri(3 * m->nt);
    GYPS_CUDA(cudaMemcpy(vtx.data(), m->d_vtx, vtx.size() * sizeof(double), cudaMemcpyDeviceToHost));
    GYPS_CUDA(cudaMemcpy(tri.data(), m->d_tri, tri.size() * sizeof(int32_t), cudaMemcpyDeviceToHost));
    std::vector<std::vector<int32_t>> nb(m->nv);
    std::vector<double> nrm(3 * m->nv, 0.0);
    double esum = 0.0;
    int64_t ecount = 0;
    for (int64_t t = 0; t < m->nt; ++t) {
        const int32_t *v = &tri[3 * t];
        const double *a = &vtx[3 * v[0]], *b = &vtx[3 * v[1]], *c = &vtx[3 * v[2]];
        const double e1[3] = {b[0] - a[0], b[1] - a[1], b[2] - a[2]}, e2[3] = {c[0] - a[0], c[1] - a[1], c[2] - a[2]};
        const double n[3] = {e1[1] * e2[2] - e1[2] * e2[1], e1[2] * e2[0] - e1[0] * e2[2], e1[0] * e2[1] - e1[1] * e2[0]};
        for (int q = 0; q < 3; ++q) {
            for (int c2 = 0; c2 < 3; ++c2) nrm[3 * v[q] + c2] += n[c2];  // area-weighted
            const int32_t p = v[q], r = v[(q + 1) % 3];
            nb[p].push_back(r);
            nb[r].push_back(p);
            const double d[3] = {vtx[3 * p] - vtx[3 * r], vtx[3 * p + 1] - vtx[3 * r + 1], vtx[3 * p + 2] - vtx[3 * r + 2]};
            esum += std::sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
            ++ecount;
        }
    }
    double cen[3] = {0, 0, 0};
    for (int64_t i = 0; i < m->nv; ++i)
        for (int c = 0; c < 3; ++c) cen[c] += vtx[3 * i + c] / (double)m->nv;
    double rad = 0.0;
    for (int64_t i = 0; i < m->nv; ++i) {
        double d2 = 0.0;
        for (int c = 0; c < 3; ++c) d2 += (vtx[3 * i + c] - cen[c]) * (vtx[3 * i + c] - cen[c]);
        rad = std::max(rad, std::sqrt(d2));
    }
    std::vector<int32_t> ptr(m->nv + 1, 0), adj;
    std::vector<float> vf(6 * m->nv);
    for (int64_t i = 0; i < m->nv; ++i) {
        auto &l = nb[i];
        std::sort(l.begin(), l.end());
        l.erase(std::unique(l.begin(), l.end()), l.end());
        adj.insert(adj.end(), l.begin(), l.end());
        ptr[i + 1] = (int32_t)adj.size();
        const double nn = std::sqrt(nrm[3 * i] * nrm[3 * i] + nrm[3 * i + 1] * nrm[3 * i + 1] +
                                    nrm[3 * i + 2] * nrm[3 * i + 2]);
        for (int c = 0; c < 3; ++c) {
            vf[6 * i + c] = (float)((vtx[3 * i + c] - cen[c]) / (rad > 0 ? rad : 1.0));
            vf[6 * i + 3 + c] = (float)(nn > 0 ? nrm[3 * i + c] / nn : 0.0);
        }
    }
    m->h_mean = esum / (double)std::max<int64_t>(ecount, 1);
    m->radius = rad;
    GYPS_CUDA(cudaMalloc((void **)&m->d_adj_ptr, ptr.size() * sizeof(int32_t)));
    GYPS_CUDA(cudaMalloc((void **)&m->d_adj, std::max<size_t>(adj.size(), 1) * sizeof(int32_t)));
    GYPS_CUDA(cudaMalloc((void **)&m->d_vfeat, vf.size() * sizeof(float)));
    m->device_bytes += (int64_t)(ptr.size() * 4 + adj.size() * 4 + vf.size() * 4);
    GYPS_CUDA(cudaMemcpy(m->d_adj_ptr, ptr.data(), ptr.size() * sizeof(int32_t), cudaMemcpyHostToDevice));
    GYPS_CUDA(cudaMemcpy(m->d_adj, adj.data(), adj.size() * sizeof(int32_t), cudaMemcpyHostToDevice));
    GYPS_CUDA(cudaMemcpy(m->d_vfeat, vf.data(), vf.size() * sizeof(float), cudaMemcpyHostToDevice));
    (void)s;
    return GYPS_OK;
}

// Activation buffers of one forward (kept for the backward).
struct Acts {
    float *F, *A0, *Y, *dY;
    std::vector<float *> Hs, Ms, As;  // H[0..L], M[0..L-1], A[0..L-1]
    float *dH, *dH2, *dA, *tmp;
};

static gyps_status layout_acts(Mpnn *P, int64_t rows, Acts &a)
{
    const int H = P->H, L = P->L;
    const size_t per = (size_t)rows * H;
    const size_t need = (size_t)rows * mp::NIN + per /*A0*/ + 2 * (size_t)rows /*Y*/ + 2 * (size_t)rows /*dY*/ +
                        (size_t)(L + 1) * per + 2 * (size_t)L * per + 4 * per;
    if (P->ws_bytes < need * sizeof(float)) {
        cudaFree(P->ws);
        P->ws = nullptr;
        GYPS_CUDA(cudaMalloc((void **)&P->ws, need * sizeof(float)));
        P->ws_bytes = need * sizeof(float);
    }
    float *q = P->ws;
    a.F = q;
    q += (size_t)rows * mp::NIN;
    a.A0 = q;
    q += per;
    a.Y = q;
    q += 2 * (size_t)rows;
    a.dY = q;
    q += 2 * (size_t)rows;
    a.Hs.assign(L + 1, nullptr);
    a.Ms.assign(L, nullptr);
    a.As.assign(L, nullptr);
    for (int l = 0; l <= L; ++l, q += per) a.Hs[l] = q;
    for (int l = 0; l < L; ++l, q += per) a.Ms[l] = q;
    for (int l = 0; l < L; ++l, q += per) a.As[l] = q;
    a.dH = q;
    q += per;
    a.dH2 = q;
    q += per;
    a.dA = q;
    q += per;
    a.tmp = q;
    return GYPS_OK;
}

static gyps_status forward(Mpnn *P, Mesh *m, double k, int B, const double2 *R, int64_t ldr, double2 *Z, int64_t ldz,
                           Acts &a, cudaStream_t s)
{
    using namespace mp;
    if (P->H != 64) return set_error(GYPS_ERR_UNSUPPORTED, "the kernels are built for 64 hidden features");
    GYPS_TRY(ensure_graph(m, s));
    const int64_t nv = m->nv, rows = nv * B;
    GYPS_TRY(layout_acts(P, rows, a));
    double *rsum = P->red;
    GYPS_CUDA(cudaMemsetAsync(rsum, 0, B * sizeof(double), s));
    sumsq_kernel<<<dim3(64, B), 256, 0, s>>>(R, ldr, nv, rsum);
    GYPS_CUDA(cudaGetLastError());
    const float kh = (float)(k * m->h_mean);
    features_kernel<<<(unsigned)((rows + 255) / 256), 256, 0, s>>>(R, ldr, m->d_vfeat, nv, B, rsum, kh, a.F);
    GYPS_CUDA(cudaGetLastError());
    const __nv_bfloat16 *W = P->pb;
    const unsigned g64r = (unsigned)((rows + 63) / 64);
    constexpr int smem_in = dense64_smem<NIN, 0>(), smem_mp = dense64_smem<64, 64>();
    GYPS_CUDA(cudaFuncSetAttribute(dense64_kernel<64, 64, true, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                   smem_mp));
    dense64_kernel<NIN, 0, true, false><<<g64r, dim3(64, 16), smem_in, s>>>(a.F, nullptr, W + P->off_win, nullptr,
                                                                            W + P->off_bin, nullptr, a.A0, a.Hs[0], rows);
    GYPS_CUDA(cudaGetLastError());
    for (int l = 0; l < P->L; ++l) {
        gather_mean_kernel<<<(unsigned)((rows + 15) / 16), dim3(64, 16), 0, s>>>(m->d_adj_ptr, m->d_adj, a.Hs[l], nv, B,
                                                                                  64, a.Ms[l]);
        GYPS_CUDA(cudaGetLastError());
        dense64_kernel<64, 64, true, true><<<g64r, dim3(64, 16), smem_mp, s>>>(
            a.Hs[l], a.Ms[l], W + P->ws_off(l), W + P->wn_off(l), W + P->b_off(l), a.Hs[l], a.As[l], a.Hs[l + 1], rows);
        GYPS_CUDA(cudaGetLastError());
    }
    dense_kernel<64, 0, 2, false, false><<<(unsigned)((rows + 63) / 64), dim3(2, 64), 0, s>>>(
        a.Hs[P->L], nullptr, W + P->off_wout, nullptr, W + P->off_bout, nullptr, nullptr, a.Y, rows);
    GYPS_CUDA(cudaGetLastError());
    const double inv_h3 = 1.0 / (m->h_mean * m->h_mean * m->h_mean);
    output_kernel<<<(unsigned)((rows + 255) / 256), 256, 0, s>>>(a.Y, rsum, nv, B, inv_h3, Z, ldz);
    GYPS_CUDA(cudaGetLastError());
    return GYPS_OK;
}

// Gradient of the loss into P->g (zeroed first); loss per column into loss_host (may be NULL).
static gyps_status backward(Mpnn *P, Mesh *m, int B, const double2 *Z, int64_t ldz, const double2 *E, int64_t lde,
                            Acts &a, double *loss_host, cudaStream_t s)
{
    using namespace mp;
    const int64_t nv = m->nv, rows = nv * B;
    const int L = P->L;
    double *rsum = P->red, *esum = P->red + 4096, *loss = P->red + 8192;
    GYPS_CUDA(cudaMemsetAsync(esum, 0, 2 * 4096 * sizeof(double), s));
    sumsq_kernel<<<dim3(64, B), 256, 0, s>>>(E, lde, nv, esum);
    GYPS_CUDA(cudaGetLastError());
    const double inv_h3 = 1.0 / (m->h_mean * m->h_mean * m->h_mean);
    loss_grad_kernel<<<(unsigned)((rows + 255) / 256), 256, 0, s>>>(Z, ldz, E, lde, esum, rsum, nv, B, inv_h3, a.dY,
                                                                    loss);
    GYPS_CUDA(cudaGetLastError());
    GYPS_CUDA(cudaMemsetAsync(P->g, 0, P->nparams * sizeof(float), s));
    const __nv_bfloat16 *W = P->pb;
    const unsigned gw = (unsigned)std::min<int64_t>((rows + 31) / 32, 304);
    const unsigned g64 = (unsigned)((rows + 15) / 16);
    const unsigned ge = (unsigned)((rows * 64 + 255) / 256);
    // decoder
    mp::wgrad_kernel<64, 2><<<gw, 256, 0, s>>>(a.Hs[L], a.dY, rows, P->g + P->off_wout, P->g + P->off_bout);
    GYPS_CUDA(cudaGetLastError());
    dense_bwd_x_kernel<64, 2, false><<<g64, dim3(64, 16), 0, s>>>(a.dY, W + P->off_wout, a.dH, rows);
    GYPS_CUDA(cudaGetLastError());
    // message-passing layers, last to first; dH holds dL/dh_{l+1}
    for (int l = L - 1; l >= 0; --l) {
        relu_bwd_kernel<<<ge, 256, 0, s>>>(a.dH, a.As[l], rows * 64, a.dA);
        GYPS_CUDA(cudaGetLastError());
        mp::wgrad_kernel<64, 64><<<gw, 256, 0, s>>>(a.Hs[l], a.dA, rows, P->g + P->ws_off(l), P->g + P->b_off(l));
        mp::wgrad_kernel<64, 64><<<gw, 256, 0, s>>>(a.Ms[l], a.dA, rows, P->g + P->wn_off(l), nullptr);
        GYPS_CUDA(cudaGetLastError());
        // dh_l = dh_{l+1} + Ws^T da + mean^T (Wn^T da)
        dense_bwd_x_kernel<64, 64, true><<<g64, dim3(64, 16), 0, s>>>(a.dA, W + P->ws_off(l), a.dH, rows);
        dense_bwd_x_kernel<64, 64, false><<<g64, dim3(64, 16), 0, s>>>(a.dA, W + P->wn_off(l), a.tmp, rows);
        GYPS_CUDA(cudaGetLastError());
        gather_tmean_kernel<<<(unsigned)((rows + 15) / 16), dim3(64, 16), 0, s>>>(m->d_adj_ptr, m->d_adj, a.tmp, nv, B,
                                                                                   64, a.dH);
        GYPS_CUDA(cudaGetLastError());
    }
    // encoder
    relu_bwd_kernel<<<ge, 256, 0, s>>>(a.dH, a.A0, rows * 64, a.dA);
    mp::wgrad_kernel<NIN, 64><<<gw, 256, 0, s>>>(a.F, a.dA, rows, P->g + P->off_win, P->g + P->off_bin);
    GYPS_CUDA(cudaGetLastError());
    if (loss_host) {
        std::vector<double> l(B);
        GYPS_CUDA(cudaMemcpyAsync(l.data(), loss, B * sizeof(double), cudaMemcpyDeviceToHost, s));
        GYPS_CUDA(cudaStreamSynchronize(s));
        for (int b = 0; b < B; ++b) loss_host[b] = l[b];
    }
    return GYPS_OK;
}

static gyps_status staged(Mesh *m, int B, const void *Xin, int64_t ld, double2 **dev, int64_t *ldd, double2 *scratch,
                          cudaStream_t s)
{
    if (is_device_pointer(Xin)) {
        *dev = (double2 *)Xin;
        *ldd = ld;
        return GYPS_OK;
    }
    GYPS_CUDA(cudaMemcpy2DAsync(scratch, m->nv * sizeof(double2), Xin, ld * sizeof(double2), m->nv * sizeof(double2), B,
                                cudaMemcpyHostToDevice, s));
    *dev = scratch;
    *ldd = m->nv;
    return GYPS_OK;
}

gyps_status precond_apply_device(gyps_precond_t h, Mesh *m, double k, int nrhs, const double2 *R, int64_t ldr,
                                 double2 *Z, int64_t ldz, cudaStream_t s)
{
    Mpnn *P = reinterpret_cast<Mpnn *>(h);
    Acts a;
    for (int c0 = 0; c0 < nrhs; c0 += 64) {  // bounded activation memory
        const int B = std::min(64, nrhs - c0);
        GYPS_TRY(forward(P, m, k, B, R + (int64_t)c0 * ldr, ldr, Z + (int64_t)c0 * ldz, ldz, a, s));
    }
    return GYPS_OK;
}

}  // namespace gyps

using namespace gyps;

static uint64_t splitmix64(uint64_t &x)
{
    uint64_t z = (x += 0x9E3779B97F4A7C15ull);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

extern "C" gyps_status gyps_precond_create(int hidden, int layers, uint64_t seed, gyps_precond_t *out)
{
    if (!out) return set_error(GYPS_ERR_INVALID, "out is NULL");
    *out = nullptr;
    if (hidden != 64) return set_error(GYPS_ERR_UNSUPPORTED, "hidden must be 64");
    if (layers < 1 || layers > 16) return set_error(GYPS_ERR_INVALID, "layers must be in 1..16");
    Mpnn *P = new Mpnn();
    P->H = hidden;
    P->L = layers;
    const int64_t H = hidden;
    P->off_win = 0;
    P->off_bin = P->off_win + mp::NIN * H;
    P->off_ws0 = P->off_bin + H;
    P->layer_stride = 2 * H * H + H;
    P->off_wout = P->off_ws0 + layers * P->layer_stride;
    P->off_bout = P->off_wout + 2 * H;
    P->nparams = P->off_bout + 2;
    cudaGetDevice(&P->device);
    // uniform(-a, a), a = 1/sqrt(fan in), biases zero; decoder scaled by 0.1
    std::vector<float> h(P->nparams, 0.0f);
    uint64_t st = seed;
    auto fill = [&](int64_t off, int64_t n, int fan_in, float scale) {
        const float a = scale / std::sqrt((float)fan_in);
        for (int64_t i = 0; i < n; ++i) {
            const double u = (double)(splitmix64(st) >> 11) * (1.0 / 9007199254740992.0);
            h[off + i] = (float)((2.0 * u - 1.0) * a);
        }
    };
    fill(P->off_win, mp::NIN * H, mp::NIN, 1.0f);
    for (int l = 0; l < layers; ++l) {
        fill(P->ws_off(l), H * H, (int)H, 0.5f);
        fill(P->wn_off(l), H * H, (int)H, 0.5f);
    }
    fill(P->off_wout, 2 * H, (int)H, 0.1f);
    const size_t nb = P->nparams * sizeof(float);
    gyps_status s = GYPS_OK;
    if (cudaMalloc((void **)&P->p, nb) != cudaSuccess || cudaMalloc((void **)&P->g, nb) != cudaSuccess ||
        cudaMalloc((void **)&P->m, nb) != cudaSuccess || cudaMalloc((void **)&P->v, nb) != cudaSuccess ||
        cudaMalloc((void **)&P->pb, P->nparams * sizeof(__nv_bfloat16)) != cudaSuccess ||
        cudaMalloc((void **)&P->red, 3 * 4096 * sizeof(double)) != cudaSuccess)
        s = set_error(GYPS_ERR_OOM, "preconditioner parameters");
    if (s == GYPS_OK) {
        cudaMemcpy(P->p, h.data(), nb, cudaMemcpyHostToDevice);
        cudaMemset(P->m, 0, nb);
        cudaMemset(P->v, 0, nb);
        mp::to_bf16_kernel<<<(unsigned)((P->nparams + 255) / 256), 256>>>(P->p, P->nparams, P->pb);
        cudaError_t e = cudaDeviceSynchronize();
        if (e != cudaSuccess) s = cuda_error(e, "preconditioner init");
    }
    if (s != GYPS_OK) {
        delete P;
        return s;
    }
    *out = reinterpret_cast<gyps_precond_t>(P);
    return GYPS_OK;
}

extern "C" gyps_status gyps_precond_destroy(gyps_precond_t h)
{
    if (!h) return GYPS_OK;
    Mpnn *P = reinterpret_cast<Mpnn *>(h);
    cudaSetDevice(P->device);
    cudaDeviceSynchronize();
    delete P;
    return GYPS_OK;
}

extern "C" gyps_status gyps_precond_params(gyps_precond_t h, float *host, int64_t n, int direction)
{
    if (!h || !host) return set_error(GYPS_ERR_INVALID, "NULL argument");
    Mpnn *P = reinterpret_cast<Mpnn *>(h);
    if (n != P->nparams) return set_error(GYPS_ERR_INVALID, "parameter count is " + std::to_string(P->nparams));
    GYPS_CUDA(cudaSetDevice(P->device));
    if (direction == 0) {
        GYPS_CUDA(cudaMemcpy(host, P->p, n * sizeof(float), cudaMemcpyDeviceToHost));
    } else {
        GYPS_CUDA(cudaMemcpy(P->p, host, n * sizeof(float), cudaMemcpyHostToDevice));
        mp::to_bf16_kernel<<<(unsigned)((n + 255) / 256), 256>>>(P->p, n, P->pb);
        GYPS_CUDA(cudaGetLastError());
        GYPS_CUDA(cudaDeviceSynchronize());
    }
    return GYPS_OK;
}

extern "C" gyps_status gyps_precond_info(gyps_precond_t h, int *hidden, int *layers, int64_t *nparams, int64_t *steps)
{
    if (!h) return set_error(GYPS_ERR_INVALID, "NULL handle");
    Mpnn *P = reinterpret_cast<Mpnn *>(h);
    if (hidden) *hidden = P->H;
    if (layers) *layers = P->L;
    if (nparams) *nparams = P->nparams;
    if (steps) *steps = P->step;
    return GYPS_OK;
}

extern "C" gyps_status gyps_precond_apply(gyps_precond_t h, gyps_mesh_t mh, double k, int nrhs, const void *R,
                                          int64_t ldr, void *Z, int64_t ldz, void *stream)
{
    Mesh *m;
    GYPS_TRY(check_mesh(mh, &m));
    if (!h || !R || !Z) return set_error(GYPS_ERR_INVALID, "NULL argument");
    if (nrhs < 1 || nrhs > 4096 || ldr < m->nv || ldz < m->nv) return set_error(GYPS_ERR_INVALID, "bad sizes");
    if (!is_device_pointer(R) || !is_device_pointer(Z)) return set_error(GYPS_ERR_INVALID, "R and Z must be device pointers");
    return precond_apply_device(h, m, k, nrhs, (const double2 *)R, ldr, (double2 *)Z, ldz, (cudaStream_t)stream);
}

// One gradient evaluation (and, with lr > 0, one Adam step) on the minibatch
// (R, E): nrhs residuals of one mesh and their corrections.
extern "C" gyps_status gyps_precond_train_step(gyps_precond_t h, gyps_mesh_t mh, double k, int nrhs, const void *R,
                                               int64_t ldr, const void *E, int64_t lde, double lr, double *loss,
                                               float *grad_host, void *stream)
{
    Mesh *m;
    GYPS_TRY(check_mesh(mh, &m));
    if (!h || !R || !E) return set_error(GYPS_ERR_INVALID, "NULL argument");
    if (nrhs < 1 || nrhs > 64 || ldr < m->nv || lde < m->nv) return set_error(GYPS_ERR_INVALID, "nrhs 1..64, ld >= nv");
    if (!(lr >= 0.0)) return set_error(GYPS_ERR_INVALID, "lr must be >= 0");
    Mpnn *P = reinterpret_cast<Mpnn *>(h);
    cudaStream_t s = (cudaStream_t)stream;
    const size_t blk = (size_t)m->nv * nrhs * sizeof(double2);
    GYPS_TRY(grow(m, &m->ws_stage, &m->ws_stage_bytes, 3 * blk));
    double2 *scr = reinterpret_cast<double2 *>(m->ws_stage);
    double2 *Rd, *Ed;
    int64_t lr_d, le_d;
    GYPS_TRY(staged(m, nrhs, R, ldr, &Rd, &lr_d, scr, s));
    GYPS_TRY(staged(m, nrhs, E, lde, &Ed, &le_d, scr + (size_t)m->nv * nrhs, s));
    double2 *Zd = scr + 2 * (size_t)m->nv * nrhs;
    Acts a;
    GYPS_TRY(forward(P, m, k, nrhs, Rd, lr_d, Zd, m->nv, a, s));
    P->ka_lo = std::min(P->ka_lo, k * m->radius);  // the graph (and the radius) exist after the forward
    P->ka_hi = std::max(P->ka_hi, k * m->radius);
    std::vector<double> l(nrhs);
    GYPS_TRY(backward(P, m, nrhs, Zd, m->nv, Ed, le_d, a, l.data(), s));
    if (loss) {
        double t = 0.0;
        for (double x : l) t += x;
        *loss = t / nrhs;
    }
    if (grad_host) {
        GYPS_CUDA(cudaMemcpy(grad_host, P->g, P->nparams * sizeof(float), cudaMemcpyDeviceToHost));
    }
    if (lr > 0.0) {
        ++P->step;
        const float b1 = 0.9f, b2 = 0.999f;
        const float c1 = 1.0f - std::pow(b1, (float)P->step), c2 = 1.0f - std::pow(b2, (float)P->step);
        mp::adam_kernel<<<(unsigned)((P->nparams + 255) / 256), 256, 0, s>>>(P->p, P->g, P->m, P->v, P->nparams,
                                                                             (float)lr, b1, b2, 1e-8f, c1, c2, P->pb);
        GYPS_CUDA(cudaGetLastError());
    }
    GYPS_CUDA(cudaStreamSynchronize(s));
    return GYPS_OK;
}

extern "C" gyps_status gyps_precond_save(gyps_precond_t h, const char *path)
{
    if (!h || !path) return set_error(GYPS_ERR_INVALID, "NULL argument");
    Mpnn *P = reinterpret_cast<Mpnn *>(h);
    std::vector<float> buf(3 * P->nparams);
    GYPS_CUDA(cudaSetDevice(P->device));
    GYPS_CUDA(cudaMemcpy(buf.data(), P->p, P->nparams * sizeof(float), cudaMemcpyDeviceToHost));
    GYPS_CUDA(cudaMemcpy(buf.data() + P->nparams, P->m, P->nparams * sizeof(float), cudaMemcpyDeviceToHost));
    GYPS_CUDA(cudaMemcpy(buf.data() + 2 * P->nparams, P->v, P->nparams * sizeof(float), cudaMemcpyDeviceToHost));
    FILE *f = std::fopen(path, "wb");
    if (!f) return set_error(GYPS_ERR_INVALID, std::string("cannot open ") + path);
    char header[256];
    std::memset(header, 0, sizeof(header));
    std::snprintf(header, sizeof(header), "{\"format\": \"gyps-mpnn-1\", \"hidden\": %d, \"layers\": %d, \"nparams\": %lld, "
                  "\"adam_step\": %lld, \"ka_lo\": %.17g, \"ka_hi\": %.17g}", P->H, P->L, (long long)P->nparams,
                  (long long)P->step, P->ka_lo, P->ka_hi);
    bool ok = std::fwrite(header, 1, sizeof(header), f) == sizeof(header) &&
              std::fwrite(buf.data(), sizeof(float), buf.size(), f) == buf.size();
    ok = (std::fclose(f) == 0) && ok;
    if (!ok) return set_error(GYPS_ERR_INVALID, "write failed");
    return GYPS_OK;
}

extern "C" gyps_status gyps_precond_load(gyps_precond_t h, const char *path)
{
    if (!h || !path) return set_error(GYPS_ERR_INVALID, "NULL argument");
    Mpnn *P = reinterpret_cast<Mpnn *>(h);
    FILE *f = std::fopen(path, "rb");
    if (!f) return set_error(GYPS_ERR_INVALID, std::string("cannot open ") + path);
    char header[256];
    std::vector<float> buf(3 * P->nparams);
    bool ok = std::fread(header, 1, sizeof(header), f) == sizeof(header);
    header[255] = 0;
    int hid = 0, lay = 0;
    long long np = 0, stp = 0;
    if (ok) ok = std::sscanf(header, "{\"format\": \"gyps-mpnn-1\", \"hidden\": %d, \"layers\": %d, \"nparams\": %lld, "
                             "\"adam_step\": %lld}", &hid, &lay, &np, &stp) == 4;
    ok = ok && hid == P->H && lay == P->L && np == P->nparams;
    double ka_lo = 1e300, ka_hi = -1e300;  // optional (files without it: no range)
    if (ok) {
        const char *q = std::strstr(header, "\"ka_lo\": ");
        if (q && std::sscanf(q, "\"ka_lo\": %lf, \"ka_hi\": %lf", &ka_lo, &ka_hi) != 2) ok = false;
    }
    ok = ok && std::fread(buf.data(), sizeof(float), buf.size(), f) == buf.size();
    std::fclose(f);
    if (!ok) return set_error(GYPS_ERR_INVALID, "not a compatible preconditioner file");
    for (float x : buf)
        if (!std::isfinite(x)) return set_error(GYPS_ERR_NAN, "non-finite parameter in the file");
    GYPS_CUDA(cudaSetDevice(P->device));
    GYPS_CUDA(cudaMemcpy(P->p, buf.data(), P->nparams * sizeof(float), cudaMemcpyHostToDevice));
    GYPS_CUDA(cudaMemcpy(P->m, buf.data() + P->nparams, P->nparams * sizeof(float), cudaMemcpyHostToDevice));
    GYPS_CUDA(cudaMemcpy(P->v, buf.data() + 2 * P->nparams, P->nparams * sizeof(float), cudaMemcpyHostToDevice));
    mp::to_bf16_kernel<<<(unsigned)((P->nparams + 255) / 256), 256>>>(P->p, P->nparams, P->pb);
    GYPS_CUDA(cudaGetLastError());
    GYPS_CUDA(cudaDeviceSynchronize());
    P->step = stp;
    P->ka_lo = ka_lo;
    P->ka_hi = ka_hi;
    return GYPS_OK;
}

namespace gyps {
gyps_status precond_in_range(gyps_precond_t h, Mesh *m, double k, cudaStream_t s, bool *in_range)
{
    const Mpnn *P = reinterpret_cast<const Mpnn *>(h);
    GYPS_TRY(ensure_graph(m, s));
    const double ka = k * m->radius;
    *in_range = P->ka_lo > P->ka_hi || (ka >= P->ka_lo / 1.25 && ka <= P->ka_hi * 1.25);
    return GYPS_OK;
}
}  // namespace gyps

extern "C" gyps_status gyps_precond_range(gyps_precond_t h, double *ka_lo, double *ka_hi)
{
    if (!h || !ka_lo || !ka_hi) return set_error(GYPS_ERR_INVALID, "NULL argument");
    const Mpnn *P = reinterpret_cast<const Mpnn *>(h);
    *ka_lo = P->ka_lo;
    *ka_hi = P->ka_hi;
    return GYPS_OK;
}
