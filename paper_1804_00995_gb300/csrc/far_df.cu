// Double-float form of the dense kernel product (Sec. 5, Eq. (BEM): v = G u)
// for checks that need FP64-class accuracy.  The FP64 pipe of this GPU runs at
// a small fraction of the FP32 pipe, so every value is carried as an
// unevaluated sum hi + lo of two FP32 numbers (about 44 significant bits) and
// handled with error-free transformations on the FP32 pipe:
//   TwoSum (Knuth, TAOCP vol. 2) and Fast2Sum (Dekker 1971) for additions,
//   TwoProd by FMA for products (Dekker 1971 / Ogita, Rump, Oishi 2005).
// exp(ikr)/r: r^-1/2 from the MUFU estimate and one Newton step in
// double-float; the phase k r is reduced by the nearest multiple of 2 pi / 512,
// whose sine and cosine come from a table computed in FP64, and the remainder
// |d| <= pi / 512 enters the Taylor polynomials d - d^3/6 + d^5/120 and
// 1 - d^2/2 + d^4/24 (truncation below 1e-17); the addition theorem joins the
// two.  Kernel values and sums agree with the FP64 form to about 1e-12.
#include <cmath>
#include <mutex>

#include "internal.h"

namespace gyps {
namespace dfl {

struct df {
    float hi, lo;
};

__device__ __forceinline__ df two_sum(float a, float b)
{
    const float s = __fadd_rn(a, b);
    const float bb = __fadd_rn(s, -a);
    const float e = __fadd_rn(__fadd_rn(a, -__fadd_rn(s, -bb)), __fadd_rn(b, -bb));
    return {s, e};
}

// |a| >= |b| (or a == 0)
__device__ __forceinline__ df fast_two_sum(float a, float b)
{
    const float s = __fadd_rn(a, b);
    return {s, __fadd_rn(b, -__fadd_rn(s, -a))};
}

__device__ __forceinline__ df add(df x, df y)
{
    df s = two_sum(x.hi, y.hi);
    return fast_two_sum(s.hi, __fadd_rn(s.lo, __fadd_rn(x.lo, y.lo)));
}

__device__ __forceinline__ df neg(df x) { return {-x.hi, -x.lo}; }

__device__ __forceinline__ df mul(df x, df y)
{
    const float p = __fmul_rn(x.hi, y.hi);
    float e = __fmaf_rn(x.hi, y.hi, -p);
    e = __fmaf_rn(x.hi, y.lo, e);
    e = __fmaf_rn(x.lo, y.hi, e);
    return fast_two_sum(p, e);
}

__device__ __forceinline__ df mulf(df x, float f)
{
    const float p = __fmul_rn(x.hi, f);
    float e = __fmaf_rn(x.hi, f, -p);
    e = __fmaf_rn(x.lo, f, e);
    return fast_two_sum(p, e);
}

__device__ __forceinline__ df from_double(double x)
{
    const float h = (float)x;
    return {h, (float)(x - (double)h)};
}

__device__ __forceinline__ double to_double(df x) { return (double)x.hi + (double)x.lo; }

constexpr int kTab = 512;                                     // table points per turn
__device__ float4 g_sincos[kTab];                             // (sin hi, sin lo, cos hi, cos lo) of 2 pi j / kTab

__global__ void sincos_table_kernel()
{
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= kTab) return;
    double s, c;
    sincospi(2.0 * j / kTab, &s, &c);
    const df sd = from_double(s), cd = from_double(c);
    g_sincos[j] = make_float4(sd.hi, sd.lo, cd.hi, cd.lo);
}

__device__ __forceinline__ float rsqrt_mufu(float x)
{
    float y;
    asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

// Phase and distance of one pair in double-float: from r2 = |x - y|^2, the
// reciprocal rs = 1/r (MUFU estimate, one Newton step), phi = k r and
// (cos phi, sin phi) by the table and the Taylor remainder.
struct Phase {
    df rs, phi, cs, sn;
};

__device__ __forceinline__ Phase phase_of(df r2, df kd, const float4 *tab)
{
    const df one = {1.0f, 0.0f};
    const df step = from_double(6.283185307179586476925286766559 / kTab);  // 2 pi / kTab
    const float inv_step = (float)(kTab / 6.283185307179586476925286766559);
    const df m_sixth = from_double(-1.0 / 6.0);
    Phase o;
    // r^-1/2 ... 1/r: y0 from MUFU, one Newton step y = y0 + y0 (1 - r2 y0^2) / 2
    const float y0 = rsqrt_mufu(r2.hi);
    const df t = mulf(mulf(r2, y0), y0);
    const float e = add(one, neg(t)).hi;
    o.rs = fast_two_sum(y0, 0.5f * y0 * e);
    o.phi = mul(kd, mul(r2, o.rs));  // k r
    // phi = j (2 pi / kTab) + d, |d| <= pi / kTab
    const float jf = rintf(o.phi.hi * inv_step);
    const df d = add(o.phi, neg(mulf(step, jf)));
    const float4 sc = tab[((int)jf) & (kTab - 1)];
    const df sa = {sc.x, sc.y}, ca = {sc.z, sc.w};
    const df u = mul(d, d);
    const float u2 = u.hi * u.hi;
    const df sd = mul(d, add(add(one, mul(u, m_sixth)), df{u2 * (1.0f / 120.0f), 0.0f}));
    const df cd = add(add(one, df{-0.5f * u.hi, -0.5f * u.lo}), df{u2 * (1.0f / 24.0f), 0.0f});
    o.sn = add(mul(sa, cd), mul(ca, sd));
    o.cs = add(mul(ca, cd), neg(mul(sa, sd)));
    return o;
}

// exp(i phi) / r and the G u products for targets tgt[t], t in [t_begin, t_end);
// self: the targets are the sources, the point paired with itself takes G = ik.
template <int R>
__global__ void __launch_bounds__(128) far_df_kernel(const double4_32a *tgt, const double4_32a *pts, const double2 *u64,
                                                     int64_t ldu, int c0, int64_t nq, double k, int64_t t_begin,
                                                     int64_t t_end, bool self, double2 *v, int64_t ldv)
{
    __shared__ float4 tab[kTab];
    __shared__ float4 sxy[128];     // (x hi, x lo, y hi, y lo)
    __shared__ float2 sz[128];      // (z hi, z lo)
    __shared__ float4 su[128][R];   // (Re hi, Re lo, Im hi, Im lo)
    for (int i = threadIdx.x; i < kTab; i += 128) tab[i] = g_sincos[i];
    const int64_t tg = t_begin + (int64_t)blockIdx.x * 128 + threadIdx.x;
    const double4_32a x = tgt[min(tg, t_end - 1)];
    const df tx = from_double(x.x), ty = from_double(x.y), tz = from_double(x.z);
    const df kd = from_double(k);
    df ar[R], ai[R];
#pragma unroll
    for (int j = 0; j < R; ++j) ar[j] = ai[j] = df{0.0f, 0.0f};
    for (int64_t s0 = 0; s0 < nq; s0 += 128) {
        const int64_t l = s0 + threadIdx.x;
        if (l < nq) {
            const double4_32a p = pts[l];
            const df a = from_double(p.x), b = from_double(p.y), c = from_double(p.z);
            sxy[threadIdx.x] = make_float4(a.hi, a.lo, b.hi, b.lo);
            sz[threadIdx.x] = make_float2(c.hi, c.lo);
#pragma unroll
            for (int j = 0; j < R; ++j) {
                const double2 uu = u64[l + (int64_t)(c0 + j) * ldu];
                const df re = from_double(uu.x), im = from_double(uu.y);
                su[threadIdx.x][j] = make_float4(re.hi, re.lo, im.hi, im.lo);
            }
        }
        __syncthreads();
        const int n = (int)min((int64_t)128, nq - s0);
        for (int ll = 0; ll < n; ++ll) {
            df gr, gi;
            if (self && s0 + ll == tg) {  // the point paired with itself: G = ik
                gr = df{0.0f, 0.0f};
                gi = kd;
            } else {
                const float4 q = sxy[ll];
                const float2 qz = sz[ll];
                const df dx = add(tx, df{-q.x, -q.y}), dy = add(ty, df{-q.z, -q.w}), dz = add(tz, df{-qz.x, -qz.y});
                const df r2 = add(add(mul(dx, dx), mul(dy, dy)), mul(dz, dz));
                const Phase ph = phase_of(r2, kd, tab);
                gr = mul(ph.cs, ph.rs);
                gi = mul(ph.sn, ph.rs);
            }
#pragma unroll
            for (int j = 0; j < R; ++j) {
                const float4 uu = su[ll][j];
                const df ur = {uu.x, uu.y}, ui = {uu.z, uu.w};
                ar[j] = add(ar[j], add(mul(gr, ur), neg(mul(gi, ui))));
                ai[j] = add(ai[j], add(mul(gr, ui), mul(gi, ur)));
            }
        }
        __syncthreads();
    }
    if (tg < t_end) {
#pragma unroll
        for (int j = 0; j < R; ++j) v[tg + (int64_t)(c0 + j) * ldv] = make_double2(to_double(ar[j]), to_double(ai[j]));
    }
}

// The double layer's kernel H = (1 - i k r) exp(i k r) n_y . (x - y) / r^3 in
// double-float, the quadrature points as targets and sources; pairs inside one
// triangle (its q consecutive points, the point itself included) give 0.
// adj: the adjoint's kernel -(1 - i k r) exp(i k r) n_x . (x - y) / r^3 (normal at the target).
template <int R>
__global__ void __launch_bounds__(128) far_dl_df_kernel(const double4_32a *pts, const double4_32a *nrm, int q,
                                                        const double2 *u64, int64_t ldu, int c0, int64_t nq, double k,
                                                        bool adj, double2 *v, int64_t ldv)
{
    __shared__ float4 tab[kTab];
    __shared__ float4 sxy[128];     // (x hi, x lo, y hi, y lo)
    __shared__ float2 sz[128];      // (z hi, z lo)
    __shared__ float4 snxy[128];    // normal (x hi, x lo, y hi, y lo)
    __shared__ float2 snz[128];     // normal (z hi, z lo)
    __shared__ float4 su[128][R];   // (Re hi, Re lo, Im hi, Im lo)
    for (int i = threadIdx.x; i < kTab; i += 128) tab[i] = g_sincos[i];
    const int64_t tg = (int64_t)blockIdx.x * 128 + threadIdx.x;
    const int64_t tq0 = (tg / q) * q;
    const double4_32a x = pts[min(tg, nq - 1)];
    const df tx = from_double(x.x), ty = from_double(x.y), tz = from_double(x.z);
    const df kd = from_double(k);
    const double4_32a tn = nrm[min(tg, nq - 1) / q];
    const double sg = adj ? -1.0 : 1.0;  // the sign of the adjoint's kernel rides on its normal
    const df tnx = from_double(sg * tn.x), tny = from_double(sg * tn.y), tnz = from_double(sg * tn.z);
    df ar[R], ai[R];
#pragma unroll
    for (int j = 0; j < R; ++j) ar[j] = ai[j] = df{0.0f, 0.0f};
    for (int64_t s0 = 0; s0 < nq; s0 += 128) {
        const int64_t l = s0 + threadIdx.x;
        if (l < nq) {
            const double4_32a p = pts[l];
            const double4_32a nn = nrm[l / q];
            const df a = from_double(p.x), b = from_double(p.y), c = from_double(p.z);
            sxy[threadIdx.x] = make_float4(a.hi, a.lo, b.hi, b.lo);
            sz[threadIdx.x] = make_float2(c.hi, c.lo);
            const df na = from_double(nn.x), nb = from_double(nn.y), nc = from_double(nn.z);
            snxy[threadIdx.x] = make_float4(na.hi, na.lo, nb.hi, nb.lo);
            snz[threadIdx.x] = make_float2(nc.hi, nc.lo);
#pragma unroll
            for (int j = 0; j < R; ++j) {
                const double2 uu = u64[l + (int64_t)(c0 + j) * ldu];
                const df re = from_double(uu.x), im = from_double(uu.y);
                su[threadIdx.x][j] = make_float4(re.hi, re.lo, im.hi, im.lo);
            }
        }
        __syncthreads();
        const int n = (int)min((int64_t)128, nq - s0);
        for (int ll = 0; ll < n; ++ll) {
            if ((uint64_t)(s0 + ll - tq0) < (uint64_t)q) continue;  // same flat triangle
            const float4 qq = sxy[ll];
            const float2 qz = sz[ll];
            const df dx = add(tx, df{-qq.x, -qq.y}), dy = add(ty, df{-qq.z, -qq.w}), dz = add(tz, df{-qz.x, -qz.y});
            const df r2 = add(add(mul(dx, dx), mul(dy, dy)), mul(dz, dz));
            const Phase ph = phase_of(r2, kd, tab);
            const float4 nxy = snxy[ll];
            const float2 nz = snz[ll];
            const df nnx = adj ? tnx : df{nxy.x, nxy.y}, nny = adj ? tny : df{nxy.z, nxy.w}, nnz = adj ? tnz : df{nz.x, nz.y};
            const df dn = add(add(mul(nnx, dx), mul(nny, dy)), mul(nnz, dz));
            const df f = mul(dn, mul(ph.rs, mul(ph.rs, ph.rs)));  // n . (x - y) / r^3
            // (1 - i k r) exp(i k r) f = (cos + kr sin) f + i (sin - kr cos) f
            const df gr = mul(add(ph.cs, mul(ph.phi, ph.sn)), f);
            const df gi = mul(add(ph.sn, neg(mul(ph.phi, ph.cs))), f);
#pragma unroll
            for (int j = 0; j < R; ++j) {
                const float4 uu = su[ll][j];
                const df ur = {uu.x, uu.y}, ui = {uu.z, uu.w};
                ar[j] = add(ar[j], add(mul(gr, ur), neg(mul(gi, ui))));
                ai[j] = add(ai[j], add(mul(gr, ui), mul(gi, ur)));
            }
        }
        __syncthreads();
    }
    if (tg < nq) {
#pragma unroll
        for (int j = 0; j < R; ++j) v[tg + (int64_t)(c0 + j) * ldv] = make_double2(to_double(ar[j]), to_double(ai[j]));
    }
}

// The table, once per device.
static gyps_status ensure_table(int device, cudaStream_t s)
{
    static std::mutex mu;
    static bool done[256] = {};
    std::lock_guard<std::mutex> lock(mu);
    if (device < 0 || device >= 256) return set_error(GYPS_ERR_CUDA, "device index out of range");
    if (done[device]) return GYPS_OK;
    sincos_table_kernel<<<(kTab + 127) / 128, 128, 0, s>>>();
    GYPS_CUDA(cudaGetLastError());
    GYPS_CUDA(cudaStreamSynchronize(s));
    done[device] = true;
    return GYPS_OK;
}

}  // namespace dfl

// v[t, c0 .. c0 + w) for targets [t_begin, t_end): the double-float far part.
gyps_status run_far_df(Mesh *m, double k, const double4_32a *tgt, bool self, const double2 *u64, int64_t ldu, int c0,
                       int w, double2 *v, int64_t ldv, int64_t t_begin, int64_t t_end, cudaStream_t s)
{
    GYPS_TRY(dfl::ensure_table(m->device, s));
    const unsigned grid = (unsigned)((t_end - t_begin + 127) / 128);
    StageTimer tf(m, s, 1);
    switch (w) {
    case 8: dfl::far_df_kernel<8><<<grid, 128, 0, s>>>(tgt, m->d_pts64, u64, ldu, c0, m->nq, k, t_begin, t_end, self, v, ldv); break;
    case 4: dfl::far_df_kernel<4><<<grid, 128, 0, s>>>(tgt, m->d_pts64, u64, ldu, c0, m->nq, k, t_begin, t_end, self, v, ldv); break;
    case 2: dfl::far_df_kernel<2><<<grid, 128, 0, s>>>(tgt, m->d_pts64, u64, ldu, c0, m->nq, k, t_begin, t_end, self, v, ldv); break;
    default: dfl::far_df_kernel<1><<<grid, 128, 0, s>>>(tgt, m->d_pts64, u64, ldu, c0, m->nq, k, t_begin, t_end, self, v, ldv); break;
    }
    GYPS_CUDA(cudaGetLastError());
    tf.done(1);
    return GYPS_OK;
}

// v[t, c0 .. c0 + w) over all quadrature points: the double-float far part of the double layer.
gyps_status run_far_dl_df(Mesh *m, double k, bool adj, const double2 *u64, int64_t ldu, int c0, int w, double2 *v,
                          int64_t ldv, cudaStream_t s)
{
    GYPS_TRY(dfl::ensure_table(m->device, s));
    const unsigned grid = (unsigned)((m->nq + 127) / 128);
    StageTimer tf(m, s, 1);
    switch (w) {
    case 4: dfl::far_dl_df_kernel<4><<<grid, 128, 0, s>>>(m->d_pts64, m->d_tri_nrm, m->q, u64, ldu, c0, m->nq, k, adj, v, ldv); break;
    case 2: dfl::far_dl_df_kernel<2><<<grid, 128, 0, s>>>(m->d_pts64, m->d_tri_nrm, m->q, u64, ldu, c0, m->nq, k, adj, v, ldv); break;
    default: dfl::far_dl_df_kernel<1><<<grid, 128, 0, s>>>(m->d_pts64, m->d_tri_nrm, m->q, u64, ldu, c0, m->nq, k, adj, v, ldv); break;
    }
    GYPS_CUDA(cudaGetLastError());
    tf.done(1);
    return GYPS_OK;
}

}  // namespace gyps
