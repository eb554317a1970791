// Device building blocks of the FP32 far kernel (Sec. 5, Eq. (BEM): the dense
// kernel product G u), shared by the single-mesh and the batched launches.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "internal.h"

namespace gyps {

// ---------------------------------------------------------------- PTX helpers
__device__ __forceinline__ uint32_t smem_addr(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint32_t bar, uint32_t parity)
{
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(bar), "r"(parity)
        : "memory");
    return ok != 0;
}

// Bounded wait: gives up after `polls` polls (each poll may suspend the thread
// for a short, hardware-defined time) instead of spinning forever.
constexpr int kDefaultWaitPolls = 1 << 22;
__device__ __forceinline__ bool mbar_wait_polls(uint32_t bar, uint32_t parity, int polls)
{
    for (int n = 0; n < polls; ++n)
        if (mbar_try_wait(bar, parity)) return true;
    return false;
}
__device__ __forceinline__ bool mbar_wait_bounded(uint32_t bar, uint32_t parity)
{
    return mbar_wait_polls(bar, parity, kDefaultWaitPolls);
}

// 1-D bulk copy global -> shared (TMA engine), completion counted on `bar`.
__device__ __forceinline__ void bulk_g2s(uint32_t dst, const void *src, uint32_t bytes, uint32_t bar)
{
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(dst),
                 "l"((uint64_t)__cvta_generic_to_global(src)), "r"(bytes), "r"(bar)
                 : "memory");
}

__device__ __forceinline__ float rsqrt_mufu(float x)
{
    float y;
    asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}
__device__ __forceinline__ float sin_mufu(float x)
{
    float y;
    asm("sin.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}
__device__ __forceinline__ float cos_mufu(float x)
{
    float y;
    asm("cos.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

// Error-free sum: hi + lo += x (Knuth's TwoSum, 6 additions).
__device__ __forceinline__ void two_sum_acc(float &hi, float &lo, float x)
{
    float s = __fadd_rn(hi, x);
    float bp = __fadd_rn(s, -hi);
    float e = __fadd_rn(__fadd_rn(hi, -__fadd_rn(s, -bp)), __fadd_rn(x, -bp));
    hi = s;
    lo = __fadd_rn(lo, e);
}

// ---------------------------------------------------------------- a3: far, FP32
// v[t] += sum_l G(x_t, y_l) u_l, G = exp(ik r)/r, G = ik for l == t.
//
// Work = (target tile) x (source tile) items, split evenly over a persistent
// grid; each CTA walks a contiguous run of items (source tile fastest) and
// flushes its target accumulators with FP64 atomics whenever the target tile
// changes.  Source tiles (positions + densities) are staged by 1-D bulk copies
// into a 3-stage shared-memory ring guarded by mbarriers.  Every thread owns T
// targets and processes source points in pairs with packed f32x2 arithmetic.
// Coordinates are scaled by k, so that rs = 1/(k r) and the phase k r = r2 * rs
// cost one multiply; the phase is reduced to [-pi, pi] by subtracting the
// nearest multiple of 2 pi (one FFMA), then rsqrt, sin and cos run on the MUFU
// unit; the sums carry exp(ikr)/(kr) and are multiplied by k at the flush.
// k = 0 (Laplace) takes a path with rsqrt only.  Per-tile FP32 partial sums are
// folded into a TwoSum (hi, lo) pair so that the rounding error does not grow
// with the number of source tiles.
struct FarArgs {
    const float *pos_panel;
    const float *den_panel;
    const float4 *tgt;
    double2 *v;
    int64_t ldv;
    int64_t t_begin, t_end;
    int64_t n_src_tiles, n_tgt_tiles;
    float ks;  // coordinate scale: k (1 for the Laplace kernel)
    int *err;
    int wait_polls;  // poll limit of the pipeline waits (the drain after a failure keeps the default)
};

template <int R, int T>
struct FarCfg {
    static constexpr int NT = 128;
    static constexpr int TT = NT * T;
    static constexpr int STAGES = 3;
    static constexpr int POS_BYTES = kPosTileFloats * 4;
    static constexpr int DEN_BYTES = kSrcPairs * 6 * R * 4;
    static constexpr int STAGE_BYTES = POS_BYTES + DEN_BYTES;
    static constexpr int SMEM = STAGES * STAGE_BYTES + 64;
};

template <int R, int T, bool LAP, bool CHECK>
__device__ __forceinline__ void far_tile(const float *sp, const float2 (&tx)[T], const float2 (&ty)[T],
                                         const float2 (&tz)[T], const int64_t (&tid)[T], int64_t src0, float ks,
                                         float2 (&are)[T][R], float2 (&aim)[T][R])
{
    const float4 *XY = reinterpret_cast<const float4 *>(sp);
    const float2 *Z = reinterpret_cast<const float2 *>(sp + 4 * kSrcPairs);
    const float4 *U = reinterpret_cast<const float4 *>(sp + 6 * kSrcPairs);
    const float2 *N = reinterpret_cast<const float2 *>(sp + 6 * kSrcPairs + 4 * kSrcPairs * R);
    const float2 ks2 = make_float2(ks, ks);
    const float2 magic = make_float2(12582912.0f, 12582912.0f);  // 1.5 * 2^23: round to integer
    const float2 nmagic = make_float2(-12582912.0f, -12582912.0f);
    const float2 inv2pi = make_float2(0.159154943091895335769f, 0.159154943091895335769f);
    const float2 m2pi = make_float2(-6.28318530717958647692f, -6.28318530717958647692f);
#pragma unroll 2
    for (int p = 0; p < kSrcPairs; ++p) {
        const float4 xy = XY[p];
        float2 sx = make_float2(xy.x, xy.y), sy = make_float2(xy.z, xy.w), sz = Z[p];
        if (!LAP) {
            sx = __fmul2_rn(sx, ks2);
            sy = __fmul2_rn(sy, ks2);
            sz = __fmul2_rn(sz, ks2);
        }
        float2 ure[R], uim[R], unim[R];
#pragma unroll
        for (int j = 0; j < R; ++j) {
            float4 u = U[p * R + j];
            ure[j] = make_float2(u.x, u.y);
            uim[j] = make_float2(u.z, u.w);
            if (!LAP) unim[j] = N[p * R + j];
        }
#pragma unroll
        for (int t = 0; t < T; ++t) {
            float2 dx = __fadd2_rn(tx[t], sx);
            float2 dy = __fadd2_rn(ty[t], sy);
            float2 dz = __fadd2_rn(tz[t], sz);
            float2 r2 = __fmul2_rn(dx, dx);
            r2 = __ffma2_rn(dy, dy, r2);
            r2 = __ffma2_rn(dz, dz, r2);
            float2 rs = make_float2(rsqrt_mufu(r2.x), rsqrt_mufu(r2.y));
            if (LAP) {
                if (CHECK) {
                    if (src0 + 2 * p == tid[t]) rs.x = 0.0f;
                    if (src0 + 2 * p + 1 == tid[t]) rs.y = 0.0f;
                }
#pragma unroll
                for (int j = 0; j < R; ++j) {
                    are[t][j] = __ffma2_rn(rs, ure[j], are[t][j]);
                    aim[t][j] = __ffma2_rn(rs, uim[j], aim[t][j]);
                }
                continue;
            }
            float2 ph = __fmul2_rn(r2, rs);                            // k r
            float2 nr = __fadd2_rn(__ffma2_rn(ph, inv2pi, magic), nmagic);  // nearest integer to k r / (2 pi)
            float2 ang = __ffma2_rn(nr, m2pi, ph);                     // in [-pi, pi]
            float2 sn = make_float2(sin_mufu(ang.x), sin_mufu(ang.y));
            float2 cs = make_float2(cos_mufu(ang.x), cos_mufu(ang.y));
            float2 gre = __fmul2_rn(cs, rs), gim = __fmul2_rn(sn, rs);  // exp(ikr) / (k r)
            if (CHECK) {  // the point paired with itself: ik / k = i
                if (src0 + 2 * p == tid[t]) {
                    gre.x = 0.0f;
                    gim.x = 1.0f;
                }
                if (src0 + 2 * p + 1 == tid[t]) {
                    gre.y = 0.0f;
                    gim.y = 1.0f;
                }
            }
#pragma unroll
            for (int j = 0; j < R; ++j) {
                are[t][j] = __ffma2_rn(gre, ure[j], are[t][j]);
                are[t][j] = __ffma2_rn(gim, unim[j], are[t][j]);
                aim[t][j] = __ffma2_rn(gre, uim[j], aim[t][j]);
                aim[t][j] = __ffma2_rn(gim, ure[j], aim[t][j]);
            }
        }
    }
}

}  // namespace gyps
