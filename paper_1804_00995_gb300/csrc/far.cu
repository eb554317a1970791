// Matrix-free single layer, Sec. 5 Eq. (BEM) plus the Sec. 5.2 correction:
//   Y = (1/4pi) Phi^T W_x G W_y Phi X + C X.
// Steps: interp (u = W_y Phi X, a2), far (v = G u, a3), project
// (Y = Phi^T W_x v / 4pi, a4) fused with the CSR correction (a5).
#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstring>
#include <mutex>
#include <string>

#include "far_tile.cuh"
#include "internal.h"

namespace gyps {

constexpr double kInv4Pi = 0.0795774715459476678844418816862571810;
constexpr double kTwoPi = 6.283185307179586476925286766559;

// ---------------------------------------------------------------- a2: interp
// u_l = eta_l sum_m lambda_m(l) x[v_m(tri(l))]  (W_y Phi x), FP32, written into
// the density panel of R right-hand sides, columns c0 .. c0+R-1 of X.
template <int R>
__global__ void interp32_kernel(const int32_t *tri, const double4_32a *pts64, const Rule rule, int64_t nq, int64_t nq_pad,
                                const double2 *X, int64_t ldx, int c0, float *panel)
{
    int64_t l = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (l >= nq_pad) return;
    int64_t tile = l / kSrcTile;
    int p = (int)(l % kSrcTile) >> 1, lane = (int)(l & 1);
    float *base = panel + tile * den_tile_floats(R);
#pragma unroll
    for (int j = 0; j < R; ++j) {
        double ur = 0.0, ui = 0.0;
        if (l < nq) {
            int64_t t = l / rule.q;
            int kq = (int)(l - t * rule.q);
            double w = pts64[l].w;
            const double2 *xc = X + (int64_t)(c0 + j) * ldx;
#pragma unroll
            for (int m = 0; m < 3; ++m) {
                double2 xv = xc[tri[3 * t + m]];
                double lam = rule.bary[3 * kq + m];
                ur += lam * xv.x;
                ui += lam * xv.y;
            }
            ur *= w;
            ui *= w;
        }
        float *u4 = base + 4 * ((int64_t)p * R + j);
        u4[lane] = (float)ur;
        u4[2 + lane] = (float)ui;
        base[4 * kSrcPairs * R + 2 * ((int64_t)p * R + j) + lane] = -(float)ui;
    }
}

// The density panel of columns c0 .. c0+w-1 (w = 1, 2, 4 or 8) for kernels of other TUs.
cudaError_t launch_interp32(const Mesh *m, const double2 *X, int64_t ldx, int c0, int w, float *panel, cudaStream_t s)
{
    const unsigned g = (unsigned)((m->nq_pad + 255) / 256);
    switch (w) {
    case 8: interp32_kernel<8><<<g, 256, 0, s>>>(m->d_tri, m->d_pts64, m->rule, m->nq, m->nq_pad, X, ldx, c0, panel); break;
    case 4: interp32_kernel<4><<<g, 256, 0, s>>>(m->d_tri, m->d_pts64, m->rule, m->nq, m->nq_pad, X, ldx, c0, panel); break;
    case 2: interp32_kernel<2><<<g, 256, 0, s>>>(m->d_tri, m->d_pts64, m->rule, m->nq, m->nq_pad, X, ldx, c0, panel); break;
    default: interp32_kernel<1><<<g, 256, 0, s>>>(m->d_tri, m->d_pts64, m->rule, m->nq, m->nq_pad, X, ldx, c0, panel); break;
    }
    return cudaGetLastError();
}

// FP64 densities u64[l + j*ld] for all nrhs columns.
__global__ void interp64_kernel(const int32_t *tri, const double4_32a *pts64, const Rule rule, int64_t nq, int64_t ld,
                                const double2 *X, int64_t ldx, int nrhs, double2 *u64)
{
    int64_t l = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    int j = blockIdx.y;
    if (l >= nq || j >= nrhs) return;
    int64_t t = l / rule.q;
    int kq = (int)(l - t * rule.q);
    const double2 *xc = X + (int64_t)j * ldx;
    double ur = 0.0, ui = 0.0;
#pragma unroll
    for (int m = 0; m < 3; ++m) {
        double2 xv = xc[tri[3 * t + m]];
        double lam = rule.bary[3 * kq + m];
        ur += lam * xv.x;
        ui += lam * xv.y;
    }
    double w = pts64[l].w;
    u64[l + j * ld] = make_double2(w * ur, w * ui);
}

// ---------------------------------------------------------------- a3: far, FP32
// (far_tile and its configuration: far_tile.cuh)
template <int R, int T, bool LAP>
__global__ void __launch_bounds__(FarCfg<R, T>::NT) far32_kernel(const FarArgs a)
{
    using C = FarCfg<R, T>;
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
        int s = (int)((item - beg) % C::STAGES);
        int64_t st = item % a.n_src_tiles;
        uint32_t bar = smem_addr(&bars[s]);
        uint32_t dst = smem_addr(smem + s * C::STAGE_BYTES);
        mbar_expect_tx(bar, C::STAGE_BYTES);
        bulk_g2s(dst, a.pos_panel + st * kPosTileFloats, C::POS_BYTES, bar);
        bulk_g2s(dst + C::POS_BYTES, a.den_panel + st * den_tile_floats(R), C::DEN_BYTES, bar);
    };
    int64_t issued = beg;  // next item to issue
    if (tid_x == 0)
        for (; issued < end && issued < beg + C::STAGES - 1; ++issued) issue(issued);

    float2 tx[T], ty[T], tz[T];
    int64_t tid[T];
    float2 are[T][R], aim[T][R];
    float hre[T][R], lre[T][R], him[T][R], lim[T][R];
    int64_t cur_tt = -1;

    auto flush = [&]() {
#pragma unroll
        for (int t = 0; t < T; ++t) {
            if (tid[t] < a.t_end) {
#pragma unroll
                for (int j = 0; j < R; ++j) {
                    double *dst = reinterpret_cast<double *>(a.v + tid[t] + j * a.ldv);
                    atomicAdd(dst, ((double)hre[t][j] + (double)lre[t][j]) * a.ks);
                    atomicAdd(dst + 1, ((double)him[t][j] + (double)lim[t][j]) * a.ks);
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
        const int64_t tb = a.t_begin + tt * C::TT;
        const int64_t te = min(tb + (int64_t)C::TT, a.t_end);
        if (tt != cur_tt) {
            if (cur_tt >= 0) flush();
#pragma unroll
            for (int t = 0; t < T; ++t) {
                int64_t g = tb + tid_x + t * C::NT;
                tid[t] = g;
                float4 p = a.tgt[min(g, a.t_end - 1)];
                if (!LAP) {
                    p.x *= a.ks;
                    p.y *= a.ks;
                    p.z *= a.ks;
                }
                tx[t] = make_float2(p.x, p.x);
                ty[t] = make_float2(p.y, p.y);
                tz[t] = make_float2(p.z, p.z);
#pragma unroll
                for (int j = 0; j < R; ++j) hre[t][j] = lre[t][j] = him[t][j] = lim[t][j] = 0.0f;
            }
            cur_tt = tt;
        }
#pragma unroll
        for (int t = 0; t < T; ++t)
#pragma unroll
            for (int j = 0; j < R; ++j) are[t][j] = aim[t][j] = make_float2(0.0f, 0.0f);

        const int s = (int)((i - beg) % C::STAGES);
        const uint32_t parity = (uint32_t)(((i - beg) / C::STAGES) & 1);
        bool ok = mbar_wait_polls(smem_addr(&bars[s]), parity, a.wait_polls);
        if (ok) {
            const float *sp = reinterpret_cast<const float *>(smem + s * C::STAGE_BYTES);
            const int64_t src0 = st * kSrcTile;
            if (tb < src0 + kSrcTile && src0 < te)
                far_tile<R, T, LAP, true>(sp, tx, ty, tz, tid, src0, a.ks, are, aim);
            else
                far_tile<R, T, LAP, false>(sp, tx, ty, tz, tid, src0, a.ks, are, aim);
#pragma unroll
            for (int t = 0; t < T; ++t)
#pragma unroll
                for (int j = 0; j < R; ++j) {
                    two_sum_acc(hre[t][j], lre[t][j], __fadd_rn(are[t][j].x, are[t][j].y));
                    two_sum_acc(him[t][j], lim[t][j], __fadd_rn(aim[t][j].x, aim[t][j].y));
                }
        }
        if (__syncthreads_or(!ok)) {
            failed = true;
            break;
        }
    }
    if (failed) {
        // Report, then wait (bounded) for the copies still in flight before the
        // shared memory they target is released.
        if (tid_x == 0) {
            atomicExch(a.err, 1);
            for (int64_t j = i; j < issued; ++j) {
                int s = (int)((j - beg) % C::STAGES);
                mbar_wait_bounded(smem_addr(&bars[s]), (uint32_t)(((j - beg) / C::STAGES) & 1));
            }
        }
        __syncthreads();
        return;
    }
    flush();
}

// ---------------------------------------------------------------- a3: far, FP64
// The plain FP64 form: one thread per target, all sources streamed through
// shared memory, exp(ikr)/r from FP64 sincos and rsqrt.  Targets tgt[t] for t
// in [t_begin, t_end); self: the targets are the sources (quadrature points),
// so the point paired with itself takes G = ik.
template <int R>
__global__ void __launch_bounds__(128) far64_kernel(const double4_32a *tgt, const double4_32a *pts, const double2 *u64,
                                                    int64_t ldu, int c0, int64_t nq, double k, int64_t t_begin,
                                                    int64_t t_end, bool self, double2 *v, int64_t ldv)
{
    __shared__ double4_32a sp[128];
    __shared__ double2 su[128][R];
    const int64_t tg = t_begin + (int64_t)blockIdx.x * 128 + threadIdx.x;
    const double4_32a x = tgt[min(tg, t_end - 1)];
    double ar[R], ai[R];
#pragma unroll
    for (int j = 0; j < R; ++j) ar[j] = ai[j] = 0.0;
    for (int64_t s0 = 0; s0 < nq; s0 += 128) {
        int64_t l = s0 + threadIdx.x;
        if (l < nq) {
            sp[threadIdx.x] = pts[l];
#pragma unroll
            for (int j = 0; j < R; ++j) su[threadIdx.x][j] = u64[l + (int64_t)(c0 + j) * ldu];
        }
        __syncthreads();
        const int n = (int)min((int64_t)128, nq - s0);
        for (int ll = 0; ll < n; ++ll) {
            double4_32a y = sp[ll];
            double gr, gi;
            if (self && s0 + ll == tg) {
                gr = 0.0;
                gi = k;
            } else {
                double dx = x.x - y.x, dy = x.y - y.y, dz = x.z - y.z;
                double r2 = dx * dx + dy * dy + dz * dz;
                double ri = rsqrt(r2);
                double sn, cs;
                sincos(k * (r2 * ri), &sn, &cs);
                gr = cs * ri;
                gi = sn * ri;
            }
#pragma unroll
            for (int j = 0; j < R; ++j) {
                double2 uu = su[ll][j];
                ar[j] += gr * uu.x - gi * uu.y;
                ai[j] += gr * uu.y + gi * uu.x;
            }
        }
        __syncthreads();
    }
    if (tg < t_end) {
#pragma unroll
        for (int j = 0; j < R; ++j) v[tg + (int64_t)(c0 + j) * ldv] = make_double2(ar[j], ai[j]);
    }
}

// ---------------------------------------------------------------- a4 + a5
// y_i = (1/4pi) sum_{k in supp phi_i} w_k lambda_i(x_k) v_k  [+ sum_c C_ic x_c]
__global__ void project_kernel(const int32_t *v2t_ptr, const int32_t *v2t, const double4_32a *pts64, const Rule rule,
                               int64_t nv, const double2 *v, int64_t ldv, const int32_t *c_rowptr,
                               const int32_t *c_col, const double *c_val, const double2 *X, int64_t ldx, double2 *Y,
                               int64_t ldy, int with_near)
{
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    int j = blockIdx.y;
    if (i >= nv) return;
    const double2 *vc = v + (int64_t)j * ldv;
    double yr = 0.0, yi = 0.0;
    for (int32_t e = v2t_ptr[i]; e < v2t_ptr[i + 1]; ++e) {
        int32_t te = v2t[e];
        int64_t t = te / 3;
        int m = te - 3 * (int)t;
        for (int kq = 0; kq < rule.q; ++kq) {
            int64_t kidx = t * rule.q + kq;
            double c = pts64[kidx].w * rule.bary[3 * kq + m];
            double2 vv = vc[kidx];
            yr += c * vv.x;
            yi += c * vv.y;
        }
    }
    yr *= kInv4Pi;
    yi *= kInv4Pi;
    if (with_near) {
        const double2 *xc = X + (int64_t)j * ldx;
        for (int32_t c = c_rowptr[i]; c < c_rowptr[i + 1]; ++c) {
            double cv = c_val[c];
            double2 xv = xc[c_col[c]];
            yr += cv * xv.x;
            yi += cv * xv.y;
        }
    }
    Y[i + (int64_t)j * ldy] = make_double2(yr, yi);
}

// Y += C X (CSR, real C, complex X), one thread per (row, column).
__global__ void near_spmv_kernel(const int32_t *c_rowptr, const int32_t *c_col, const double *c_val, int64_t nv,
                                 const double2 *X, int64_t ldx, double2 *Y, int64_t ldy)
{
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    int j = blockIdx.y;
    if (i >= nv) return;
    const double2 *xc = X + (int64_t)j * ldx;
    double yr = 0.0, yi = 0.0;
    for (int32_t c = c_rowptr[i]; c < c_rowptr[i + 1]; ++c) {
        double cv = c_val[c];
        double2 xv = xc[c_col[c]];
        yr += cv * xv.x;
        yi += cv * xv.y;
    }
    double2 *y = Y + i + (int64_t)j * ldy;
    *y = make_double2(y->x + yr, y->y + yi);
}

// Correction restricted to test triangles [pa_begin, pa_end) of the pair list:
// Y[v_i(a)] += sum_j block_ab[i][j] X[v_j(b)] (atomics: rows are shared).
__global__ void near_partial_kernel(const int32_t *pair_a, const int32_t *pair_b, const double *blocks,
                                    const int32_t *tri, int64_t p_begin, int64_t p_end, const double2 *X, int64_t ldx,
                                    double2 *Y, int64_t ldy)
{
    int64_t p = p_begin + (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    int j = blockIdx.y;
    if (p >= p_end) return;
    const int64_t a = pair_a[p], b = pair_b[p];
    const double2 *xc = X + (int64_t)j * ldx;
    double2 xb[3];
    for (int c = 0; c < 3; ++c) xb[c] = xc[tri[3 * b + c]];
    for (int r = 0; r < 3; ++r) {
        double yr = 0.0, yi = 0.0;
        for (int c = 0; c < 3; ++c) {
            double bv = blocks[9 * p + 3 * r + c];
            yr += bv * xb[c].x;
            yi += bv * xb[c].y;
        }
        double *y = reinterpret_cast<double *>(Y + tri[3 * a + r] + (int64_t)j * ldy);
        atomicAdd(y, yr);
        atomicAdd(y + 1, yi);
    }
}

cudaError_t launch_near_spmv(const Mesh &m, int nrhs, const double2 *X, int64_t ldx, double2 *Y, int64_t ldy,
                             cudaStream_t s)
{
    dim3 g((unsigned)((m.nv + 127) / 128), (unsigned)nrhs);
    near_spmv_kernel<<<g, 128, 0, s>>>(m.d_c_rowptr, m.d_c_col, m.d_c_val, m.nv, X, ldx, Y, ldy);
    return cudaGetLastError();
}

// ---------------------------------------------------------------- drivers
template <int R, int T, bool LAP>
static gyps_status launch_far32(Mesh *m, const FarArgs &a, cudaStream_t s)
{
    using C = FarCfg<R, T>;
    GYPS_CUDA(cudaFuncSetAttribute(far32_kernel<R, T, LAP>, cudaFuncAttributeMaxDynamicSharedMemorySize, C::SMEM));
    int occ = 0;
    GYPS_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, far32_kernel<R, T, LAP>, C::NT, C::SMEM));
    occ = std::max(occ, 1);
    const int64_t items = a.n_tgt_tiles * a.n_src_tiles;
    const int64_t grid = std::min<int64_t>((int64_t)m->num_sms * occ, items);
    far32_kernel<R, T, LAP><<<(unsigned)grid, C::NT, C::SMEM, s>>>(a);
    GYPS_CUDA(cudaGetLastError());
    return GYPS_OK;
}

static FarArgs far_args(const Mesh *m, const float *panel, double2 *v, int64_t ldv, int64_t t_begin, int64_t t_end,
                        int tt_size, double k)
{
    FarArgs a;
    a.pos_panel = m->d_pos_panel;
    a.den_panel = panel;
    a.tgt = m->d_pts32;
    a.v = v;
    a.ldv = ldv;
    a.t_begin = t_begin;
    a.t_end = t_end;
    a.n_src_tiles = m->n_src_tiles;
    a.n_tgt_tiles = (t_end - t_begin + tt_size - 1) / tt_size;
    a.ks = k > 0.0 ? (float)k : 1.0f;
    a.err = m->d_err;
    const int wp = wait_polls_setting();
    a.wait_polls = wp >= 0 ? wp : kDefaultWaitPolls;
    return a;
}

template <int R, int T>
static gyps_status run_far32(Mesh *m, double k, const double2 *X, int64_t ldx, int c0, double2 *v, int64_t ldv,
                             int64_t t_begin, int64_t t_end, cudaStream_t s)
{
    using C = FarCfg<R, T>;
    float *panel = reinterpret_cast<float *>(m->ws_den);
    StageTimer ti(m, s, 0);
    interp32_kernel<R><<<(unsigned)((m->nq_pad + 255) / 256), 256, 0, s>>>(m->d_tri, m->d_pts64, m->rule, m->nq,
                                                                           m->nq_pad, X, ldx, c0, panel);
    GYPS_CUDA(cudaGetLastError());
    ti.done(1);
    FarArgs a = far_args(m, panel, v + (int64_t)c0 * ldv, ldv, t_begin, t_end, C::TT, k);
    StageTimer tf(m, s, 1);
    if (k > 0.0)
        GYPS_TRY((launch_far32<R, T, false>(m, a, s)));
    else
        GYPS_TRY((launch_far32<R, T, true>(m, a, s)));
    tf.done(1);
    return GYPS_OK;
}

template <int R>
static gyps_status run_far64(Mesh *m, double k, const double4_32a *tgt, bool self, const double2 *u64, int64_t ldu,
                             int c0, double2 *v, int64_t ldv, int64_t t_begin, int64_t t_end, cudaStream_t s)
{
    unsigned grid = (unsigned)((t_end - t_begin + 127) / 128);
    StageTimer tf(m, s, 1);
    far64_kernel<R><<<grid, 128, 0, s>>>(tgt, m->d_pts64, u64, ldu, c0, m->nq, k, t_begin, t_end, self, v, ldv);
    GYPS_CUDA(cudaGetLastError());
    tf.done(1);
    return GYPS_OK;
}

// Splits nrhs into register-resident chunks of 8, 4, 2 and 1 columns.
static int chunk_width(int left) { return left >= 8 ? 8 : left >= 4 ? 4 : left >= 2 ? 2 : 1; }

// FP32 far sum of a density panel prepared by the caller (R = 1, 2, 4 or 8 columns,
// interp32 layout), over all quadrature points as targets, added into v (k > 0).
gyps_status far32_panel(Mesh *m, double k, const float *panel, int R, double2 *v, int64_t ldv, cudaStream_t s)
{
    StageTimer tf(m, s, 1);
    switch (R) {
    case 8: GYPS_TRY((launch_far32<8, 2, false>(m, far_args(m, panel, v, ldv, 0, m->nq, FarCfg<8, 2>::TT, k), s))); break;
    case 4: GYPS_TRY((launch_far32<4, 2, false>(m, far_args(m, panel, v, ldv, 0, m->nq, FarCfg<4, 2>::TT, k), s))); break;
    case 2: GYPS_TRY((launch_far32<2, 4, false>(m, far_args(m, panel, v, ldv, 0, m->nq, FarCfg<2, 4>::TT, k), s))); break;
    case 1: GYPS_TRY((launch_far32<1, 4, false>(m, far_args(m, panel, v, ldv, 0, m->nq, FarCfg<1, 4>::TT, k), s))); break;
    default: return set_error(GYPS_ERR_INVALID, "panel width");
    }
    tf.done(1);
    return GYPS_OK;
}

// FP64 far sum of u64 columns [c0, c0 + w), w = 1, 2 or 4, all quadrature points as targets.
gyps_status far64_cols(Mesh *m, double k, const double2 *u64, int64_t ldu, int c0, int w, double2 *v, int64_t ldv,
                       cudaStream_t s)
{
    switch (w) {
    case 4: return run_far64<4>(m, k, m->d_pts64, true, u64, ldu, c0, v, ldv, 0, m->nq, s);
    case 2: return run_far64<2>(m, k, m->d_pts64, true, u64, ldu, c0, v, ldv, 0, m->nq, s);
    case 1: return run_far64<1>(m, k, m->d_pts64, true, u64, ldu, c0, v, ldv, 0, m->nq, s);
    default: return set_error(GYPS_ERR_INVALID, "column width");
    }
}

gyps_status apply_device(Mesh *m, double k, int nrhs, const double2 *X, int64_t ldx, double2 *Y, int64_t ldy,
                         int prec, uint32_t flags, int64_t tri_begin, int64_t tri_end, cudaStream_t s)
{
    const bool full = (tri_begin == 0 && tri_end == m->nt);
    if (prec == GYPS_PREC_AUTO) prec = (nrhs >= 16 && k > 0.0) ? GYPS_PREC_TC_BF16X3 : GYPS_PREC_FP32;
    if (prec == GYPS_PREC_TC_BF16X3 && k <= 0.0)
        return set_error(GYPS_ERR_UNSUPPORTED, "tensor-core precision needs k > 0");
    if (prec != GYPS_PREC_FP32 && prec != GYPS_PREC_FP64 && prec != GYPS_PREC_TC_BF16X3 && prec != GYPS_PREC_DF64)
        return set_error(GYPS_ERR_INVALID, "unknown precision");
    const int64_t t_begin = tri_begin * m->q, t_end = tri_end * m->q;

    // v: nq x nrhs FP64 accumulators (zeroed: the FP32 kernel adds into it,
    // and targets outside a partial range must read as zero)
    const int64_t ldv = m->nq;
    if (m->prof) ++m->prof_applies;
    GYPS_TRY(grow(m, &m->ws_v, &m->ws_v_bytes, (size_t)(ldv * nrhs) * sizeof(double2)));
    double2 *v = reinterpret_cast<double2 *>(m->ws_v);
    GYPS_CUDA(cudaMemsetAsync(v, 0, (size_t)(ldv * nrhs) * sizeof(double2), s));

    if (t_end > t_begin) {
        if (prec == GYPS_PREC_TC_BF16X3) {
            GYPS_TRY(far_tc(m, k, X, ldx, nrhs, v, ldv, t_begin, t_end, s));
        } else if (prec == GYPS_PREC_FP32) {
            GYPS_TRY(grow(m, &m->ws_den, &m->ws_den_bytes, (size_t)(m->n_src_tiles * den_tile_floats(8)) * sizeof(float)));
            for (int c0 = 0; c0 < nrhs;) {
                int w = chunk_width(nrhs - c0);
                gyps_status st;
                switch (w) {
                case 8: st = run_far32<8, 2>(m, k, X, ldx, c0, v, ldv, t_begin, t_end, s); break;
                case 4: st = run_far32<4, 2>(m, k, X, ldx, c0, v, ldv, t_begin, t_end, s); break;
                case 2: st = run_far32<2, 4>(m, k, X, ldx, c0, v, ldv, t_begin, t_end, s); break;
                default: st = run_far32<1, 4>(m, k, X, ldx, c0, v, ldv, t_begin, t_end, s); break;
                }
                GYPS_TRY(st);
                c0 += w;
            }
        } else {
            const int64_t ldu = m->nq;
            GYPS_TRY(grow(m, &m->ws_den, &m->ws_den_bytes, (size_t)(ldu * nrhs) * sizeof(double2)));
            double2 *u64 = reinterpret_cast<double2 *>(m->ws_den);
            dim3 g((unsigned)((m->nq + 255) / 256), (unsigned)nrhs);
            StageTimer ti(m, s, 0);
            interp64_kernel<<<g, 256, 0, s>>>(m->d_tri, m->d_pts64, m->rule, m->nq, ldu, X, ldx, nrhs, u64);
            GYPS_CUDA(cudaGetLastError());
            ti.done(1);
            for (int c0 = 0; c0 < nrhs && prec == GYPS_PREC_DF64;) {
                const int w = chunk_width(nrhs - c0);
                GYPS_TRY(run_far_df(m, k, m->d_pts64, true, u64, ldu, c0, w, v, ldv, t_begin, t_end, s));
                c0 += w;
            }
            for (int c0 = 0; c0 < nrhs && prec == GYPS_PREC_FP64;) {
                int w = chunk_width(nrhs - c0);
                gyps_status st;
                switch (w) {
                case 8: st = run_far64<8>(m, k, m->d_pts64, true, u64, ldu, c0, v, ldv, t_begin, t_end, s); break;
                case 4: st = run_far64<4>(m, k, m->d_pts64, true, u64, ldu, c0, v, ldv, t_begin, t_end, s); break;
                case 2: st = run_far64<2>(m, k, m->d_pts64, true, u64, ldu, c0, v, ldv, t_begin, t_end, s); break;
                default: st = run_far64<1>(m, k, m->d_pts64, true, u64, ldu, c0, v, ldv, t_begin, t_end, s); break;
                }
                GYPS_TRY(st);
                c0 += w;
            }
        }
    }
    const bool near = !(flags & GYPS_APPLY_NO_NEAR);
    dim3 g((unsigned)((m->nv + 127) / 128), (unsigned)nrhs);
    StageTimer tp(m, s, 2);
    project_kernel<<<g, 128, 0, s>>>(m->d_v2t_ptr, m->d_v2t, m->d_pts64, m->rule, m->nv, v, ldv, m->d_c_rowptr,
                                     m->d_c_col, m->d_c_val, X, ldx, Y, ldy, (near && full) ? 1 : 0);
    GYPS_CUDA(cudaGetLastError());
    tp.done(1);
    if (near && !full) {
        const int32_t pp[2] = {m->h_pair_ptr[tri_begin], m->h_pair_ptr[tri_end]};
        if (pp[1] > pp[0]) {
            dim3 gp((unsigned)((pp[1] - pp[0] + 127) / 128), (unsigned)nrhs);
            StageTimer tn(m, s, 3);
            near_partial_kernel<<<gp, 128, 0, s>>>(m->d_pair_a, m->d_pair_b, m->d_blocks, m->d_tri, pp[0], pp[1], X, ldx,
                                                   Y, ldy);
            GYPS_CUDA(cudaGetLastError());
            tn.done(1);
        }
    }
    return GYPS_OK;
}

// Host staging of an nv x nrhs complex block with leading dimension ld.
// Far part of the potential at arbitrary points (the radiation operator of the
// listing in Sec. 5.4: integral(points, S2, Gxy, Vh)).  The FP32 kernel takes
// the points as targets numbered from nq_pad on, past every source index, so
// its self-pair test never fires: the target and accumulator pointers are
// shifted back by that offset (every access stays inside the point arrays).
template <int R, int T>
static gyps_status run_far32_points(Mesh *m, double k, const double2 *X, int64_t ldx, int c0, const float4 *tgt32,
                                    int64_t npts, double2 *v, int64_t ldv, cudaStream_t s)
{
    using C = FarCfg<R, T>;
    float *panel = reinterpret_cast<float *>(m->ws_den);
    StageTimer ti(m, s, 0);
    interp32_kernel<R><<<(unsigned)((m->nq_pad + 255) / 256), 256, 0, s>>>(m->d_tri, m->d_pts64, m->rule, m->nq,
                                                                           m->nq_pad, X, ldx, c0, panel);
    GYPS_CUDA(cudaGetLastError());
    ti.done(1);
    const int64_t off = m->nq_pad;
    FarArgs a = far_args(m, panel, v + (int64_t)c0 * ldv - off, ldv, off, off + npts, C::TT, k);
    a.tgt = tgt32 - off;
    StageTimer tf(m, s, 1);
    if (k > 0.0)
        GYPS_TRY((launch_far32<R, T, false>(m, a, s)));
    else
        GYPS_TRY((launch_far32<R, T, true>(m, a, s)));
    tf.done(1);
    return GYPS_OK;
}

gyps_status far_points(Mesh *m, double k, const double2 *X, int64_t ldx, int nrhs, const float4 *tgt32,
                       const double4_32a *tgt64, int64_t npts, double2 *v, int64_t ldv, int prec, cudaStream_t s)
{
    GYPS_CUDA(cudaMemset2DAsync(v, ldv * sizeof(double2), 0, npts * sizeof(double2), nrhs, s));
    if (npts == 0) return GYPS_OK;
    if (prec == GYPS_PREC_FP32) {
        GYPS_TRY(grow(m, &m->ws_den, &m->ws_den_bytes, (size_t)(m->n_src_tiles * den_tile_floats(8)) * sizeof(float)));
        for (int c0 = 0; c0 < nrhs;) {
            const int w = chunk_width(nrhs - c0);
            gyps_status st;
            switch (w) {
            case 8: st = run_far32_points<8, 2>(m, k, X, ldx, c0, tgt32, npts, v, ldv, s); break;
            case 4: st = run_far32_points<4, 2>(m, k, X, ldx, c0, tgt32, npts, v, ldv, s); break;
            case 2: st = run_far32_points<2, 4>(m, k, X, ldx, c0, tgt32, npts, v, ldv, s); break;
            default: st = run_far32_points<1, 4>(m, k, X, ldx, c0, tgt32, npts, v, ldv, s); break;
            }
            GYPS_TRY(st);
            c0 += w;
        }
        return GYPS_OK;
    }
    const int64_t ldu = m->nq;
    GYPS_TRY(grow(m, &m->ws_den, &m->ws_den_bytes, (size_t)(ldu * nrhs) * sizeof(double2)));
    double2 *u64 = reinterpret_cast<double2 *>(m->ws_den);
    dim3 g((unsigned)((m->nq + 255) / 256), (unsigned)nrhs);
    interp64_kernel<<<g, 256, 0, s>>>(m->d_tri, m->d_pts64, m->rule, m->nq, ldu, X, ldx, nrhs, u64);
    GYPS_CUDA(cudaGetLastError());
    for (int c0 = 0; c0 < nrhs;) {
        const int w = chunk_width(nrhs - c0);
        gyps_status st;
        if (prec == GYPS_PREC_DF64) {
            st = run_far_df(m, k, tgt64, false, u64, ldu, c0, w, v, ldv, 0, npts, s);
        } else {
            switch (w) {
            case 8: st = run_far64<8>(m, k, tgt64, false, u64, ldu, c0, v, ldv, 0, npts, s); break;
            case 4: st = run_far64<4>(m, k, tgt64, false, u64, ldu, c0, v, ldv, 0, npts, s); break;
            case 2: st = run_far64<2>(m, k, tgt64, false, u64, ldu, c0, v, ldv, 0, npts, s); break;
            default: st = run_far64<1>(m, k, tgt64, false, u64, ldu, c0, v, ldv, 0, npts, s); break;
            }
        }
        GYPS_TRY(st);
        c0 += w;
    }
    return GYPS_OK;
}

static gyps_status stage_in(Mesh *m, const void *src, int64_t ld, int nrhs, double2 *dst, cudaStream_t s)
{
    GYPS_CUDA(cudaMemcpy2DAsync(dst, m->nv * sizeof(double2), src, ld * sizeof(double2), m->nv * sizeof(double2), nrhs,
                                cudaMemcpyHostToDevice, s));
    return GYPS_OK;
}
static gyps_status stage_out(Mesh *m, const double2 *src, void *dst, int64_t ld, int nrhs, cudaStream_t s)
{
    GYPS_CUDA(cudaMemcpy2DAsync(dst, ld * sizeof(double2), src, m->nv * sizeof(double2), m->nv * sizeof(double2), nrhs,
                                cudaMemcpyDeviceToHost, s));
    return GYPS_OK;
}

static std::atomic<int> g_wait_polls{-1};
int wait_polls_setting() { return g_wait_polls.load(std::memory_order_relaxed); }

gyps_status clear_err_word(Mesh *m, cudaStream_t s)
{
    GYPS_CUDA(cudaMemsetAsync(m->d_err, 0, sizeof(int), s));
    return GYPS_OK;
}

gyps_status check_err_word(Mesh *m, cudaStream_t s)
{
    int h = 0;
    GYPS_CUDA(cudaMemcpyAsync(&h, m->d_err, sizeof(int), cudaMemcpyDeviceToHost, s));
    GYPS_CUDA(cudaStreamSynchronize(s));
    if (h) {
        GYPS_CUDA(cudaMemsetAsync(m->d_err, 0, sizeof(int), s));
        return set_error(GYPS_ERR_TIMEOUT, "a device wait ran out of polls; results are incomplete");
    }
    return GYPS_OK;
}

}  // namespace gyps

using namespace gyps;

static gyps_status check_block(const Mesh *m, int nrhs, const void *X, int64_t ldx, const char *name)
{
    if (!X) return set_error(GYPS_ERR_INVALID, std::string(name) + " is NULL");
    if (nrhs < 1 || nrhs > 4096) return set_error(GYPS_ERR_INVALID, "nrhs must be in 1..4096");
    if (ldx < m->nv) return set_error(GYPS_ERR_INVALID, std::string("leading dimension of ") + name + " < nv");
    return GYPS_OK;
}

extern "C" gyps_status gyps_sl_apply(gyps_mesh_t h, double k, int nrhs, const void *X, int64_t ldx, void *Y,
                                     int64_t ldy, int prec, uint32_t flags, int64_t tri_begin, int64_t tri_end,
                                     void *stream)
{
    Mesh *m;
    GYPS_TRY(check_mesh(h, &m));
    GYPS_TRY(check_block(m, nrhs, X, ldx, "X"));
    GYPS_TRY(check_block(m, nrhs, Y, ldy, "Y"));
    if (!std::isfinite(k) || k < 0.0) return set_error(GYPS_ERR_INVALID, "k must be finite and >= 0");
    if (flags & ~GYPS_APPLY_NO_NEAR) return set_error(GYPS_ERR_INVALID, "unknown flag");
    if (tri_begin == -1 && tri_end == -1) {
        tri_begin = 0;
        tri_end = m->nt;
    }
    if (tri_begin < 0 || tri_end > m->nt || tri_begin > tri_end)
        return set_error(GYPS_ERR_INVALID, "triangle range outside [0, nt]");
    if (prec != GYPS_PREC_FP64 && prec != GYPS_PREC_FP32 && prec != GYPS_PREC_TC_BF16X3 && prec != GYPS_PREC_AUTO &&
        prec != GYPS_PREC_DF64)
        return set_error(GYPS_ERR_INVALID, "unknown precision");
    if (prec == GYPS_PREC_TC_BF16X3 && nrhs < 16)
        return set_error(GYPS_ERR_UNSUPPORTED, "tensor-core precision needs at least 16 right-hand sides");
    cudaStream_t s = (cudaStream_t)stream;
    const bool dx = is_device_pointer(X), dy = is_device_pointer(Y);
    if (dx && dy) {
        if ((const char *)X < (const char *)Y + ldy * nrhs * 16 && (const char *)Y < (const char *)X + ldx * nrhs * 16)
            return set_error(GYPS_ERR_INVALID, "X and Y overlap");
        GYPS_TRY(apply_device(m, k, nrhs, (const double2 *)X, ldx, (double2 *)Y, ldy, prec, flags, tri_begin, tri_end, s));
        return GYPS_OK;
    }
    // host buffers: stage through library-owned device memory, then wait
    const size_t blk = (size_t)m->nv * nrhs * sizeof(double2);
    GYPS_TRY(grow(m, &m->ws_stage, &m->ws_stage_bytes, 2 * blk));
    double2 *xs = reinterpret_cast<double2 *>(m->ws_stage), *ys = xs + (size_t)m->nv * nrhs;
    const double2 *xin = (const double2 *)X;
    int64_t lxin = ldx;
    GYPS_TRY(clear_err_word(m, s));
    if (!dx) {
        GYPS_TRY(stage_in(m, X, ldx, nrhs, xs, s));
        xin = xs;
        lxin = m->nv;
    }
    double2 *yout = dy ? (double2 *)Y : ys;
    int64_t lyout = dy ? ldy : m->nv;
    GYPS_TRY(apply_device(m, k, nrhs, xin, lxin, yout, lyout, prec, flags, tri_begin, tri_end, s));
    if (!dy) GYPS_TRY(stage_out(m, ys, Y, ldy, nrhs, s));
    GYPS_CUDA(cudaStreamSynchronize(s));
    return check_err_word(m, s);
}

extern "C" gyps_status gyps_near_correct(gyps_mesh_t h, int nrhs, const void *X, int64_t ldx, void *Y, int64_t ldy,
                                         void *stream)
{
    Mesh *m;
    GYPS_TRY(check_mesh(h, &m));
    GYPS_TRY(check_block(m, nrhs, X, ldx, "X"));
    GYPS_TRY(check_block(m, nrhs, Y, ldy, "Y"));
    cudaStream_t s = (cudaStream_t)stream;
    const bool dx = is_device_pointer(X), dy = is_device_pointer(Y);
    if (dx && dy) {
        GYPS_CUDA(launch_near_spmv(*m, nrhs, (const double2 *)X, ldx, (double2 *)Y, ldy, s));
        return GYPS_OK;
    }
    const size_t blk = (size_t)m->nv * nrhs * sizeof(double2);
    GYPS_TRY(grow(m, &m->ws_stage, &m->ws_stage_bytes, 2 * blk));
    double2 *xs = reinterpret_cast<double2 *>(m->ws_stage), *ys = xs + (size_t)m->nv * nrhs;
    const double2 *xin = (const double2 *)X;
    int64_t lxin = ldx;
    if (!dx) {
        GYPS_TRY(stage_in(m, X, ldx, nrhs, xs, s));
        xin = xs;
        lxin = m->nv;
    }
    double2 *yio = (double2 *)Y;
    int64_t lyio = ldy;
    if (!dy) {
        GYPS_TRY(stage_in(m, Y, ldy, nrhs, ys, s));
        yio = ys;
        lyio = m->nv;
    }
    GYPS_CUDA(launch_near_spmv(*m, nrhs, xin, lxin, yio, lyio, s));
    if (!dy) GYPS_TRY(stage_out(m, ys, Y, ldy, nrhs, s));
    GYPS_CUDA(cudaStreamSynchronize(s));
    return GYPS_OK;
}

extern "C" gyps_status gyps_mesh_check(gyps_mesh_t h, void *stream)
{
    Mesh *m;
    GYPS_TRY(check_mesh(h, &m));
    cudaStream_t s = (cudaStream_t)stream;
    GYPS_CUDA(cudaStreamSynchronize(s));
    return check_err_word(m, s);
}

extern "C" gyps_status gyps_set_wait_polls(int64_t polls)
{
    if (polls > ((int64_t)1 << 30)) return set_error(GYPS_ERR_INVALID, "polls must be <= 2^30");
    g_wait_polls.store(polls < 0 ? -1 : (int)polls, std::memory_order_relaxed);
    return GYPS_OK;
}

extern "C" gyps_status gyps_profile_enable(gyps_mesh_t h, int enable)
{
    Mesh *m;
    GYPS_TRY(check_mesh(h, &m));
    for (auto &r : m->prof_pending) {
        cudaEventSynchronize(r.b);
        cudaEventDestroy(r.a);
        cudaEventDestroy(r.b);
    }
    m->prof_pending.clear();
    m->prof = enable != 0;
    for (int i = 0; i < 4; ++i) {
        m->prof_ms[i] = 0.0;
        m->prof_launches[i] = 0;
    }
    m->prof_applies = 0;
    return GYPS_OK;
}

extern "C" gyps_status gyps_profile_read(gyps_mesh_t h, gyps_profile_t *out)
{
    Mesh *m;
    GYPS_TRY(check_mesh(h, &m));
    if (!out) return set_error(GYPS_ERR_INVALID, "out is NULL");
    for (auto &r : m->prof_pending) {
        GYPS_CUDA(cudaEventSynchronize(r.b));
        float ms = 0.0f;
        GYPS_CUDA(cudaEventElapsedTime(&ms, r.a, r.b));
        m->prof_ms[r.stage] += ms;
        m->prof_launches[r.stage] += r.launches;
        cudaEventDestroy(r.a);
        cudaEventDestroy(r.b);
    }
    m->prof_pending.clear();
    out->applies = m->prof_applies;
    out->launches = m->prof_launches[0] + m->prof_launches[1] + m->prof_launches[2] + m->prof_launches[3];
    out->interp_ms = m->prof_ms[0];
    out->far_ms = m->prof_ms[1];
    out->project_ms = m->prof_ms[2];
    out->near_ms = m->prof_ms[3];
    out->far_launches = m->prof_launches[1];
    return GYPS_OK;
}

// ---------------------------------------------------------------- no-allocation apply
// gyps_sl_apply_noalloc: the same FP32 apply as gyps_sl_apply, for callers that
// must not allocate device memory while they run (their device memory is owned
// by another allocator, or a cudaMalloc and the device-wide synchronisation it
// can cause is not acceptable inside their loop).  Its scratch (the FP32
// density panel of one column and the FP64 accumulators of the target points)
// lives in the fixed array below instead of mesh workspace: every GPU that
// loads the library holds these bytes until the process exits.
namespace gyps {

constexpr size_t kNoAllocScratchBytes = (size_t)8 << 20;  // 8 MiB
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

// Device address of g_noalloc_scratch per device, looked up once per device
// with that device current (the host-side name is only a stand-in).
static std::mutex g_noalloc_mu;
static void *g_noalloc_addr[64] = {nullptr};

static gyps_status noalloc_scratch(int device, void **out)
{
    if (device < 0 || device >= 64) return set_error(GYPS_ERR_UNSUPPORTED, "device index above 63");
    std::lock_guard<std::mutex> lock(g_noalloc_mu);
    if (!g_noalloc_addr[device]) {
        void *p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess) return cuda_error(e, "cudaGetSymbolAddress(g_noalloc_scratch)");
        g_noalloc_addr[device] = p;
    }
    *out = g_noalloc_addr[device];
    return GYPS_OK;
}

// Bytes of scratch one column needs: FP32 panel of all source tiles plus the
// 256-byte aligned FP64 accumulator block.
static size_t noalloc_need(const Mesh *m, size_t *v_off)
{
    size_t panel = (size_t)m->n_src_tiles * (size_t)den_tile_floats(1) * sizeof(float);
    *v_off = (panel + 255) & ~(size_t)255;
    return *v_off + (size_t)m->nq * sizeof(double2);
}

}  // namespace gyps

extern "C" gyps_status gyps_sl_apply_noalloc(gyps_mesh_t h, double k, int nrhs, const void *X, int64_t ldx, void *Y,
                                             int64_t ldy, void *stream)
{
    Mesh *m;
    GYPS_TRY(check_mesh(h, &m));
    GYPS_TRY(check_block(m, nrhs, X, ldx, "X"));
    GYPS_TRY(check_block(m, nrhs, Y, ldy, "Y"));
    if (!std::isfinite(k) || k < 0.0) return set_error(GYPS_ERR_INVALID, "k must be finite and >= 0");
    if (!is_device_pointer(X) || !is_device_pointer(Y))
        return set_error(GYPS_ERR_INVALID, "X and Y must be device pointers (host buffers would need staging memory)");
    if ((const char *)X < (const char *)Y + ldy * nrhs * 16 && (const char *)Y < (const char *)X + ldx * nrhs * 16)
        return set_error(GYPS_ERR_INVALID, "X and Y overlap");
    size_t v_off = 0;
    const size_t need = noalloc_need(m, &v_off);
    if (need > kNoAllocScratchBytes)
        return set_error(GYPS_ERR_INVALID, "mesh needs " + std::to_string(need) + " scratch bytes; the fixed array holds " +
                                               std::to_string(kNoAllocScratchBytes) + " (about 28 bytes per quadrature point)");
    void *base = nullptr;
    GYPS_TRY(noalloc_scratch(m->device, &base));
    float *panel = reinterpret_cast<float *>(base);
    double2 *v = reinterpret_cast<double2 *>(reinterpret_cast<unsigned char *>(base) + v_off);
    cudaStream_t s = (cudaStream_t)stream;
    using C = FarCfg<1, 4>;
    const double2 *Xd = (const double2 *)X;
    double2 *Yd = (double2 *)Y;
    for (int j = 0; j < nrhs; ++j) {
        // the accumulators must start at zero: the previous call (or column) left its sums there
        GYPS_CUDA(cudaMemsetAsync(v, 0, (size_t)m->nq * sizeof(double2), s));
        interp32_kernel<1><<<(unsigned)((m->nq_pad + 255) / 256), 256, 0, s>>>(m->d_tri, m->d_pts64, m->rule, m->nq,
                                                                               m->nq_pad, Xd, ldx, j, panel);
        GYPS_CUDA(cudaGetLastError());
        FarArgs a = far_args(m, panel, v, m->nq, 0, m->nq, C::TT, k);
        if (k > 0.0)
            GYPS_TRY((launch_far32<1, 4, false>(m, a, s)));
        else
            GYPS_TRY((launch_far32<1, 4, true>(m, a, s)));
        dim3 g((unsigned)((m->nv + 127) / 128), 1u);
        project_kernel<<<g, 128, 0, s>>>(m->d_v2t_ptr, m->d_v2t, m->d_pts64, m->rule, m->nv, v, m->nq, m->d_c_rowptr,
                                         m->d_c_col, m->d_c_val, Xd + (int64_t)j * ldx, ldx, Yd + (int64_t)j * ldy,
                                         ldy, 1);
        GYPS_CUDA(cudaGetLastError());
    }
    return GYPS_OK;
}
