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

#include "far_tile.cuh"
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
                                                       bool adj, double2 *v, int64_t ldv)
{
    __shared__ double4_32a sp[128];
    __shared__ double4_32a sn[128];
    __shared__ double2 su[128][R];
    const int64_t tg = (int64_t)blockIdx.x * 128 + threadIdx.x;
    const int64_t tq0 = (tg / q) * q;
    const double4_32a x = pts[min(tg, nq - 1)];
    const double4_32a tn = nrm[min(tg, nq - 1) / q];  // adjoint: the normal at the target
    const double sg = adj ? -1.0 : 1.0;
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
            if ((uint64_t)(s0 + ll - tq0) < (uint64_t)q) continue;  // same flat triangle: n . (x - y) = 0
            const double4_32a y = sp[ll], nn = adj ? tn : sn[ll];
            const double dx = x.x - y.x, dy = x.y - y.y, dz = x.z - y.z;
            const double r2 = dx * dx + dy * dy + dz * dz;
            const double ri = rsqrt(r2);
            const double f = sg * (nn.x * dx + nn.y * dy + nn.z * dz) * ri * ri * ri;
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

// ---------------------------------------------------------------- far part, FP32
// The FP32 form follows the single layer's tile design: a persistent grid walks
// (target tile) x (source tile) items, source tiles are staged by 1-D bulk copies
// into a 3-stage ring (positions, normals, densities), every thread owns T
// targets and takes source points in pairs with packed f32x2 arithmetic, and
// per-tile FP32 sums are folded into TwoSum pairs.  Coordinates are scaled by k,
// so rs = 1/(k r), k r = r2 rs and n . (x - y) rs^3 = H-factor / k^2, restored
// at the flush; Laplace (k = 0) runs unscaled without the phase.  Pairs inside
// one triangle (its q points are consecutive) give 0.
//
// Normal panel tile, in the position panel's pair layout:
//   float4 NXY[P] = (nx0, nx1, ny0, ny1), float2 NZ[P] = (nz0, nz1); padding 0.
__global__ void nrm_panel_kernel(const double4_32a *nrm, int q, int64_t nq, int64_t nq_pad, float *panel)
{
    const int64_t l = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (l >= nq_pad) return;
    float x = 0.0f, y = 0.0f, z = 0.0f;
    if (l < nq) {
        const double4_32a n = nrm[l / q];
        x = (float)n.x;
        y = (float)n.y;
        z = (float)n.z;
    }
    const int64_t tile = l / kSrcTile;
    const int p = (int)(l % kSrcTile) >> 1, lane = (int)(l & 1);
    float *base = panel + tile * kPosTileFloats;
    base[4 * p + lane] = x;
    base[4 * p + 2 + lane] = y;
    base[4 * kSrcPairs + 2 * p + lane] = z;
}

struct DlArgs {
    const float *pos_panel, *nrm_panel, *den_panel;
    const float4 *tgt;
    const double4_32a *tri_nrm;  // adjoint: normals at the targets
    double2 *v;
    int64_t ldv, nq, n_src_tiles, n_tgt_tiles;
    int q;
    float ks;
    int *err;
};

template <int R, int T, bool ADJ>
struct DlCfg {
    static constexpr int NT = 128;
    static constexpr int TT = NT * T;
    static constexpr int STAGES = 3;
    static constexpr int POS_BYTES = kPosTileFloats * 4;
    static constexpr int NRM_BYTES = ADJ ? 0 : kPosTileFloats * 4;  // the adjoint takes target normals
    static constexpr int DEN_BYTES = kSrcPairs * 6 * R * 4;
    static constexpr int STAGE_BYTES = POS_BYTES + NRM_BYTES + DEN_BYTES;
    static constexpr int SMEM = STAGES * STAGE_BYTES + 64;
};

__device__ __forceinline__ float2 neg2(float2 a) { return make_float2(-a.x, -a.y); }

template <int R, int T, bool LAP, bool CHECK, bool ADJ>
__device__ __forceinline__ void dl_tile(const float *sp, const float2 (&tx)[T], const float2 (&ty)[T],
                                        const float2 (&tz)[T], const float2 (&tnx)[T], const float2 (&tny)[T],
                                        const float2 (&tnz)[T], const int64_t (&tq0)[T], int64_t src0, int q,
                                        float ks, float2 (&are)[T][R], float2 (&aim)[T][R])
{
    constexpr int DEN = ADJ ? kPosTileFloats : 2 * kPosTileFloats;  // float offset of the densities
    const float4 *XY = reinterpret_cast<const float4 *>(sp);
    const float2 *Z = reinterpret_cast<const float2 *>(sp + 4 * kSrcPairs);
    const float4 *NXY = reinterpret_cast<const float4 *>(sp + kPosTileFloats);
    const float2 *NZ = reinterpret_cast<const float2 *>(sp + kPosTileFloats + 4 * kSrcPairs);
    const float4 *U = reinterpret_cast<const float4 *>(sp + DEN);
    const float2 *N = reinterpret_cast<const float2 *>(sp + DEN + 4 * kSrcPairs * R);
    const float2 ks2 = make_float2(ks, ks);
    const float2 magic = make_float2(12582912.0f, 12582912.0f);  // 1.5 * 2^23: round to integer
    const float2 nmagic = make_float2(-12582912.0f, -12582912.0f);
    const float2 inv2pi = make_float2(0.159154943091895335769f, 0.159154943091895335769f);
    const float2 m2pi = make_float2(-6.28318530717958647692f, -6.28318530717958647692f);
#pragma unroll 2
    for (int p = 0; p < kSrcPairs; ++p) {
        const float4 xy = XY[p];
        float2 sx = make_float2(xy.x, xy.y), sy = make_float2(xy.z, xy.w), sz = Z[p];
        float2 nx = make_float2(0.0f, 0.0f), ny = nx, nz = nx;
        if (!ADJ) {
            const float4 nxy = NXY[p];
            nx = make_float2(nxy.x, nxy.y);
            ny = make_float2(nxy.z, nxy.w);
            nz = NZ[p];
        }
        if (!LAP) {
            sx = __fmul2_rn(sx, ks2);
            sy = __fmul2_rn(sy, ks2);
            sz = __fmul2_rn(sz, ks2);
        }
        float2 ure[R], uim[R], unim[R];
#pragma unroll
        for (int j = 0; j < R; ++j) {
            const float4 u = U[p * R + j];
            ure[j] = make_float2(u.x, u.y);
            uim[j] = make_float2(u.z, u.w);
            if (!LAP) unim[j] = N[p * R + j];
        }
#pragma unroll
        for (int t = 0; t < T; ++t) {
            const float2 dx = __fadd2_rn(tx[t], sx);
            const float2 dy = __fadd2_rn(ty[t], sy);
            const float2 dz = __fadd2_rn(tz[t], sz);
            float2 r2 = __fmul2_rn(dx, dx);
            r2 = __ffma2_rn(dy, dy, r2);
            r2 = __ffma2_rn(dz, dz, r2);
            const float2 rs = make_float2(rsqrt_mufu(r2.x), rsqrt_mufu(r2.y));
            float2 dn = __fmul2_rn(ADJ ? tnx[t] : nx, dx);
            dn = __ffma2_rn(ADJ ? tny[t] : ny, dy, dn);
            dn = __ffma2_rn(ADJ ? tnz[t] : nz, dz, dn);
            float2 f = __fmul2_rn(__fmul2_rn(dn, rs), __fmul2_rn(rs, rs));  // n . (x - y) / r^3
            if (LAP) {
                if (CHECK) {
                    if ((uint64_t)(src0 + 2 * p - tq0[t]) < (uint64_t)q) f.x = 0.0f;
                    if ((uint64_t)(src0 + 2 * p + 1 - tq0[t]) < (uint64_t)q) f.y = 0.0f;
                }
#pragma unroll
                for (int j = 0; j < R; ++j) {
                    are[t][j] = __ffma2_rn(f, ure[j], are[t][j]);
                    aim[t][j] = __ffma2_rn(f, uim[j], aim[t][j]);
                }
                continue;
            }
            const float2 ph = __fmul2_rn(r2, rs);                               // k r
            const float2 nr = __fadd2_rn(__ffma2_rn(ph, inv2pi, magic), nmagic);  // nearest integer to k r / (2 pi)
            const float2 ang = __ffma2_rn(nr, m2pi, ph);                        // in [-pi, pi]
            const float2 sn = make_float2(sin_mufu(ang.x), sin_mufu(ang.y));
            const float2 cs = make_float2(cos_mufu(ang.x), cos_mufu(ang.y));
            // (1 - i k r) exp(i k r) f = (cos + kr sin) f + i (sin - kr cos) f
            const float2 cf = __fmul2_rn(cs, f), sf = __fmul2_rn(sn, f);
            float2 hre = __ffma2_rn(ph, sf, cf);
            float2 him = __ffma2_rn(neg2(ph), cf, sf);
            if (CHECK) {  // same triangle (and the point itself): 0
                if ((uint64_t)(src0 + 2 * p - tq0[t]) < (uint64_t)q) hre.x = him.x = 0.0f;
                if ((uint64_t)(src0 + 2 * p + 1 - tq0[t]) < (uint64_t)q) hre.y = him.y = 0.0f;
            }
#pragma unroll
            for (int j = 0; j < R; ++j) {
                are[t][j] = __ffma2_rn(hre, ure[j], are[t][j]);
                are[t][j] = __ffma2_rn(him, unim[j], are[t][j]);
                aim[t][j] = __ffma2_rn(hre, uim[j], aim[t][j]);
                aim[t][j] = __ffma2_rn(him, ure[j], aim[t][j]);
            }
        }
    }
}

template <int R, int T, bool LAP, bool ADJ>
__global__ void __launch_bounds__(DlCfg<R, T, ADJ>::NT) far_dl32_kernel(const DlArgs a)
{
    using C = DlCfg<R, T, ADJ>;
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
        if (!ADJ) bulk_g2s(dst + C::POS_BYTES, a.nrm_panel + st * kPosTileFloats, C::NRM_BYTES, bar);
        bulk_g2s(dst + C::POS_BYTES + C::NRM_BYTES, a.den_panel + st * den_tile_floats(R), C::DEN_BYTES, bar);
    };
    int64_t issued = beg;
    if (tid_x == 0)
        for (; issued < end && issued < beg + C::STAGES - 1; ++issued) issue(issued);

    float2 tx[T], ty[T], tz[T], tnx[T], tny[T], tnz[T];
    int64_t tid[T], tq0[T];
    float2 are[T][R], aim[T][R];
    float hre[T][R], lre[T][R], him[T][R], lim[T][R];
    int64_t cur_tt = -1;
    // k^2 of the scaled coordinates; the adjoint kernel n_x . (y - x) carries the minus sign
    const double scale = (ADJ ? -1.0 : 1.0) * (double)a.ks * (double)a.ks;
    auto flush = [&]() {
#pragma unroll
        for (int t = 0; t < T; ++t) {
            if (tid[t] < a.nq) {
#pragma unroll
                for (int j = 0; j < R; ++j) {
                    double *dst = reinterpret_cast<double *>(a.v + tid[t] + j * a.ldv);
                    atomicAdd(dst, ((double)hre[t][j] + (double)lre[t][j]) * scale);
                    atomicAdd(dst + 1, ((double)him[t][j] + (double)lim[t][j]) * scale);
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
                float4 p = a.tgt[min(g, a.nq - 1)];
                if (!LAP) {
                    p.x *= a.ks;
                    p.y *= a.ks;
                    p.z *= a.ks;
                }
                tx[t] = make_float2(p.x, p.x);
                ty[t] = make_float2(p.y, p.y);
                tz[t] = make_float2(p.z, p.z);
                if (ADJ) {
                    const double4_32a n = a.tri_nrm[min(g, a.nq - 1) / a.q];
                    tnx[t] = make_float2((float)n.x, (float)n.x);
                    tny[t] = make_float2((float)n.y, (float)n.y);
                    tnz[t] = make_float2((float)n.z, (float)n.z);
                }
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
        const bool ok = mbar_wait_bounded(smem_addr(&bars[s]), parity);
        if (ok) {
            const float *sp = reinterpret_cast<const float *>(smem + s * C::STAGE_BYTES);
            const int64_t src0 = st * kSrcTile;
            // a triangle's q <= 7 points may straddle a tile boundary
            if (tb - 8 < src0 + kSrcTile && src0 < te + 8)
                dl_tile<R, T, LAP, true, ADJ>(sp, tx, ty, tz, tnx, tny, tnz, tq0, src0, a.q, a.ks, are, aim);
            else
                dl_tile<R, T, LAP, false, ADJ>(sp, tx, ty, tz, tnx, tny, tnz, tq0, src0, a.q, a.ks, are, aim);
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
        // report, then wait (bounded) for the copies still in flight
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

template <int R, int T, bool ADJ>
static gyps_status run_far_dl32(Mesh *m, double k, const double2 *X, int64_t ldx, int c0, double2 *v, int64_t ldv,
                                cudaStream_t s)
{
    using C = DlCfg<R, T, ADJ>;
    float *panel = reinterpret_cast<float *>(m->ws_den);
    GYPS_CUDA(launch_interp32(m, X, ldx, c0, R, panel, s));
    DlArgs a;
    a.pos_panel = m->d_pos_panel;
    a.nrm_panel = m->d_nrm_panel;
    a.den_panel = panel;
    a.tgt = m->d_pts32;
    a.tri_nrm = m->d_tri_nrm;
    a.v = v + (int64_t)c0 * ldv;
    a.ldv = ldv;
    a.nq = m->nq;
    a.n_src_tiles = m->n_src_tiles;
    a.n_tgt_tiles = (m->nq + C::TT - 1) / C::TT;
    a.q = m->q;
    a.ks = k > 0.0 ? (float)k : 1.0f;
    a.err = m->d_err;
    auto kern = k > 0.0 ? far_dl32_kernel<R, T, false, ADJ> : far_dl32_kernel<R, T, true, ADJ>;
    GYPS_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, C::SMEM));
    int occ = 0;
    GYPS_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, C::NT, C::SMEM));
    occ = occ > 1 ? occ : 1;
    const int64_t items = a.n_tgt_tiles * a.n_src_tiles;
    const int64_t grid = items < (int64_t)m->num_sms * occ ? items : (int64_t)m->num_sms * occ;
    StageTimer tf(m, s, 1);
    kern<<<(unsigned)grid, C::NT, C::SMEM, s>>>(a);
    GYPS_CUDA(cudaGetLastError());
    tf.done(1);
    return GYPS_OK;
}

// valT[e] = val at the transposed position of e: entry (i, j) of row i takes C_ji
// (the pattern is symmetric: triangles sharing a vertex form a symmetric relation;
// columns are sorted within each row).
__global__ void csr_transpose_values_kernel(int64_t nv, const int32_t *rowptr, const int32_t *col, const double *val,
                                            double *valT)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nv) return;
    for (int32_t e = rowptr[i]; e < rowptr[i + 1]; ++e) {
        const int32_t j = col[e];
        int32_t lo = rowptr[j], hi = rowptr[j + 1];
        while (lo < hi) {
            const int32_t mid = (lo + hi) >> 1;
            if (col[mid] < (int32_t)i) lo = mid + 1;
            else hi = mid;
        }
        valT[e] = (lo < rowptr[j + 1] && col[lo] == (int32_t)i) ? val[lo] : 0.0;
    }
}

// Normals, the double-layer correction values on C's pattern and their transpose
// (the adjoint's correction), and the FP32 normal panel; once per mesh.
static gyps_status dl_prepare(Mesh *m, cudaStream_t s)
{
    if (m->d_cdl_val) return GYPS_OK;
    if (!m->d_tri_nrm) GYPS_CUDA(cudaMalloc((void **)&m->d_tri_nrm, (size_t)m->nt * sizeof(double4_32a)));
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
    if (!m->d_nrm_panel)
        e = cudaMalloc((void **)&m->d_nrm_panel, (size_t)m->n_src_tiles * kPosTileFloats * sizeof(float));
    if (e == cudaSuccess) {
        nrm_panel_kernel<<<(unsigned)((m->nq_pad + 255) / 256), 256, 0, s>>>(m->d_tri_nrm, m->q, m->nq, m->nq_pad,
                                                                           m->d_nrm_panel);
        e = cudaGetLastError();
    }
    double *valT = nullptr;
    if (e == cudaSuccess) e = cudaMalloc((void **)&valT, (size_t)m->c_nnz * sizeof(double));
    if (e == cudaSuccess) {
        csr_transpose_values_kernel<<<(unsigned)((m->nv + 127) / 128), 128, 0, s>>>(m->nv, m->d_c_rowptr, m->d_c_col,
                                                                                   val, valT);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) {
        cudaFree(val);
        if (valT) cudaFree(valT);
        return cuda_error(e, "double-layer normal panel / adjoint correction");
    }
    m->d_cdlT_val = valT;
    m->d_cdl_val = val;
    return GYPS_OK;
}

// Y = K X, or Y = K' X (adj: normal at the test point, transposed correction).
gyps_status dl_apply_device(Mesh *m, double k, int nrhs, const double2 *X, int64_t ldx, double2 *Y, int64_t ldy,
                            int prec, bool adj, cudaStream_t s)
{
    GYPS_TRY(dl_prepare(m, s));
    const int64_t ld = m->nq;
    GYPS_TRY(grow(m, &m->ws_v, &m->ws_v_bytes, (size_t)(ld * nrhs) * sizeof(double2)));
    double2 *v = reinterpret_cast<double2 *>(m->ws_v);
    if (prec == GYPS_PREC_FP64 || prec == GYPS_PREC_DF64) {
        GYPS_TRY(grow(m, &m->ws_den, &m->ws_den_bytes, (size_t)(ld * nrhs) * sizeof(double2)));
        double2 *u64 = reinterpret_cast<double2 *>(m->ws_den);
        dim3 gi((unsigned)((m->nq + 255) / 256), (unsigned)nrhs);
        interp64_kernel<<<gi, 256, 0, s>>>(m->d_tri, m->d_pts64, m->rule, m->nq, ld, X, ldx, nrhs, u64);
        GYPS_CUDA(cudaGetLastError());
        const unsigned grid = (unsigned)((m->nq + 127) / 128);
        for (int c0 = 0; c0 < nrhs;) {
            const int w = nrhs - c0 >= 4 ? 4 : nrhs - c0 >= 2 ? 2 : 1;
            if (prec == GYPS_PREC_DF64) {
                GYPS_TRY(run_far_dl_df(m, k, adj, u64, ld, c0, w, v, ld, s));
                c0 += w;
                continue;
            }
            if (w == 4) far_dl64_kernel<4><<<grid, 128, 0, s>>>(m->d_pts64, m->d_tri_nrm, m->q, u64, ld, c0, m->nq, k, adj, v, ld);
            else if (w == 2) far_dl64_kernel<2><<<grid, 128, 0, s>>>(m->d_pts64, m->d_tri_nrm, m->q, u64, ld, c0, m->nq, k, adj, v, ld);
            else far_dl64_kernel<1><<<grid, 128, 0, s>>>(m->d_pts64, m->d_tri_nrm, m->q, u64, ld, c0, m->nq, k, adj, v, ld);
            GYPS_CUDA(cudaGetLastError());
            c0 += w;
        }
    } else {
        // the FP32 kernel adds into v with atomics
        GYPS_CUDA(cudaMemsetAsync(v, 0, (size_t)(ld * nrhs) * sizeof(double2), s));
        GYPS_TRY(grow(m, &m->ws_den, &m->ws_den_bytes, (size_t)(m->n_src_tiles * den_tile_floats(8)) * sizeof(float)));
        for (int c0 = 0; c0 < nrhs;) {
            const int rem = nrhs - c0;
            const int w = rem >= 8 ? 8 : rem >= 4 ? 4 : rem >= 2 ? 2 : 1;
            if (adj) {
                switch (w) {
                case 8: GYPS_TRY((run_far_dl32<8, 2, true>(m, k, X, ldx, c0, v, ld, s))); break;
                case 4: GYPS_TRY((run_far_dl32<4, 2, true>(m, k, X, ldx, c0, v, ld, s))); break;
                case 2: GYPS_TRY((run_far_dl32<2, 4, true>(m, k, X, ldx, c0, v, ld, s))); break;
                default: GYPS_TRY((run_far_dl32<1, 4, true>(m, k, X, ldx, c0, v, ld, s))); break;
                }
            } else {
                switch (w) {
                case 8: GYPS_TRY((run_far_dl32<8, 2, false>(m, k, X, ldx, c0, v, ld, s))); break;
                case 4: GYPS_TRY((run_far_dl32<4, 2, false>(m, k, X, ldx, c0, v, ld, s))); break;
                case 2: GYPS_TRY((run_far_dl32<2, 4, false>(m, k, X, ldx, c0, v, ld, s))); break;
                default: GYPS_TRY((run_far_dl32<1, 4, false>(m, k, X, ldx, c0, v, ld, s))); break;
                }
            }
            c0 += w;
        }
    }
    dim3 gp((unsigned)((m->nv + 127) / 128), (unsigned)nrhs);
    project_kernel<<<gp, 128, 0, s>>>(m->d_v2t_ptr, m->d_v2t, m->d_pts64, m->rule, m->nv, v, ld, m->d_c_rowptr,
                                      m->d_c_col, adj ? m->d_cdlT_val : m->d_cdl_val, X, ldx, Y, ldy, 1);
    GYPS_CUDA(cudaGetLastError());
    return GYPS_OK;
}

// Combined-field operators, in Galerkin form with the mass matrix M = Phi^T W Phi
// of Eq. (A=BWB):
//   indirect (Brakhage-Werner): u = (D - i eta S) phi outside the surface, whose
//     exterior trace (1/2 + K - i eta V) phi = -u_inc (jump of the double-layer
//     potential);
//   direct: the exterior normal derivative of Green's representation
//     u = u_inc - S (du/dn) gives (1/2 + K') du/dn = du_inc/dn, its trace
//     V du/dn = u_inc; the combination (1/2 + K' - i eta V) du/dn = (d/dn - i eta) u_inc
//     has the density of the first-kind system as its solution.
// Y holds V X on entry and T holds K X (or K' X):  Y = 1/2 Phi^T W Phi X + T - i eta Y.
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

// Y = (1/2 M + K - i eta V) X, or with K' (adj).  V in prec; K in prec for FP64
// and double-float, in FP32 otherwise.
gyps_status combined_apply_device(Mesh *m, double k, double eta, bool adj, int nrhs, const double2 *X, int64_t ldx,
                                  double2 *Y, int64_t ldy, int prec, cudaStream_t s)
{
    GYPS_TRY(grow(m, &m->ws_bw, &m->ws_bw_bytes, (size_t)m->nv * nrhs * sizeof(double2)));
    double2 *T = reinterpret_cast<double2 *>(m->ws_bw);
    const int kprec = (prec == GYPS_PREC_FP64 || prec == GYPS_PREC_DF64) ? prec : GYPS_PREC_FP32;
    GYPS_TRY(dl_apply_device(m, k, nrhs, X, ldx, T, m->nv, kprec, adj, s));
    GYPS_TRY(apply_device(m, k, nrhs, X, ldx, Y, ldy, prec, 0, 0, m->nt, s));
    dim3 g((unsigned)((m->nv + 127) / 128), (unsigned)nrhs);
    bw_combine_kernel<<<g, 128, 0, s>>>(m->d_v2t_ptr, m->d_v2t, m->d_tri, m->d_pts64, m->rule, m->nv, X, ldx, T, m->nv,
                                        eta, Y, ldy);
    GYPS_CUDA(cudaGetLastError());
    return GYPS_OK;
}

}  // namespace gyps

using namespace gyps;

static gyps_status dl_entry(gyps_mesh_t h, double k, int nrhs, const void *X, int64_t ldx, void *Y, int64_t ldy,
                            int prec, void *stream, bool adj)
{
    Mesh *m;
    GYPS_TRY(check_mesh(h, &m));
    if (nrhs < 1 || nrhs > 4096) return set_error(GYPS_ERR_INVALID, "nrhs must be in 1..4096");
    if (!X || !Y) return set_error(GYPS_ERR_INVALID, "NULL argument");
    if (ldx < m->nv || ldy < m->nv) return set_error(GYPS_ERR_INVALID, "leading dimension < nv");
    if (!std::isfinite(k) || k < 0.0) return set_error(GYPS_ERR_INVALID, "k must be finite and >= 0");
    if (prec == GYPS_PREC_AUTO) prec = GYPS_PREC_FP32;
    if (prec == GYPS_PREC_TC_BF16X3) return set_error(GYPS_ERR_UNSUPPORTED, "double layer: FP64, FP32 or DF64");
    if (prec != GYPS_PREC_FP64 && prec != GYPS_PREC_FP32 && prec != GYPS_PREC_DF64)
        return set_error(GYPS_ERR_INVALID, "unknown precision");
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
    GYPS_TRY(clear_err_word(m, s));  // report only the waits of this call's launches
    GYPS_TRY(dl_apply_device(m, k, nrhs, xin, lxin, yout, lyout, prec, adj, s));
    if (!dy)
        GYPS_CUDA(cudaMemcpy2DAsync(Y, ldy * sizeof(double2), ys, m->nv * sizeof(double2), m->nv * sizeof(double2), nrhs,
                                    cudaMemcpyDeviceToHost, s));
    GYPS_CUDA(cudaStreamSynchronize(s));
    return check_err_word(m, s);
}

static gyps_status combined_entry(gyps_mesh_t h, double k, double eta, int nrhs, const void *X, int64_t ldx, void *Y,
                                  int64_t ldy, int prec, void *stream, bool adj)
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
    GYPS_TRY(clear_err_word(m, s));  // report only the waits of this call's launches
    GYPS_TRY(combined_apply_device(m, k, eta, adj, nrhs, xin, lxin, yout, lyout, prec, s));
    if (!dy)
        GYPS_CUDA(cudaMemcpy2DAsync(Y, ldy * sizeof(double2), ys, m->nv * sizeof(double2), m->nv * sizeof(double2), nrhs,
                                    cudaMemcpyDeviceToHost, s));
    GYPS_CUDA(cudaStreamSynchronize(s));
    return check_err_word(m, s);
}

extern "C" gyps_status gyps_dl_apply(gyps_mesh_t h, double k, int nrhs, const void *X, int64_t ldx, void *Y,
                                     int64_t ldy, int prec, void *stream)
{
    return dl_entry(h, k, nrhs, X, ldx, Y, ldy, prec, stream, false);
}

extern "C" gyps_status gyps_adl_apply(gyps_mesh_t h, double k, int nrhs, const void *X, int64_t ldx, void *Y,
                                      int64_t ldy, int prec, void *stream)
{
    return dl_entry(h, k, nrhs, X, ldx, Y, ldy, prec, stream, true);
}

extern "C" gyps_status gyps_bw_apply(gyps_mesh_t h, double k, double eta, int nrhs, const void *X, int64_t ldx,
                                     void *Y, int64_t ldy, int prec, void *stream)
{
    return combined_entry(h, k, eta, nrhs, X, ldx, Y, ldy, prec, stream, false);
}

extern "C" gyps_status gyps_cfie_apply(gyps_mesh_t h, double k, double eta, int nrhs, const void *X, int64_t ldx,
                                       void *Y, int64_t ldy, int prec, void *stream)
{
    return combined_entry(h, k, eta, nrhs, X, ldx, Y, ldy, prec, stream, true);
}
