// Tensor-core form of the dense kernel product (Sec. 5, Eq. (BEM): v = G u) for
// 16 or more right-hand sides.  In real arithmetic the complex product is
//   [Re v | Im v] = [Gr | Gi] * [[Ur, Ui], [-Ui, Ur]],
// a (128 targets) x (2 Ks) by (2 Ks) x (2 R) contraction per source chunk of Ks
// points.  Sixteen generator warps compute the kernel tile G = exp(ikr)/(kr) in
// FP32 on the CUDA cores (the MUFU path of the FP32 kernel), split every value
// into bf16 hi + lo and write both straight into tensor memory (tcgen05.st, one
// lane per target).  A product warp issues tcgen05.mma (kind::f16, bf16 inputs,
// FP32 accumulation in tensor memory) with the tile as operand A and the bf16
// hi/lo panel of the densities as operand B: per 16-wide K step one product
// A_hi x [B_hi | B_lo] (the two panels stacked along N) and one A_lo x B_hi, the
// three split terms hi*hi + hi*lo + lo*hi.  A copy warp stages the panel chunks
// by 1-D bulk copies.  The epilogue reads the accumulators with tcgen05.ld and
// adds k * (Re, Im) into the FP64 sums.
#include <algorithm>
#include <cmath>

#include <cuda_bf16.h>

#include "far_tile.cuh"
#include "internal.h"

namespace gyps {
namespace tc {

constexpr int M = 128;                          // targets per tile = tensor-memory lanes
constexpr int KS = 64;                          // sources per chunk
constexpr int KC = 2 * KS;                      // K extent per chunk: Gr for the chunk, then Gi
constexpr int GPR = 4;                          // generator threads per target row
constexpr int NGEN = M * GPR;                   // 16 generator warps
constexpr int NT = NGEN + 64;                   // + product warp + copy warp
constexpr int SEG_CHUNKS = 256;                 // chunks per work item (16384 sources)
constexpr int POS_XY = KS / 2 * 16;             // float4 (-x0, -x1, -y0, -y1) per source pair
constexpr int POS_BYTES = POS_XY + KS / 2 * 8;  // + float2 (-z0, -z1) per pair (scaled by k)
constexpr uint32_t CORE_LBO = 128;              // bytes between core matrices along K
constexpr uint32_t CORE_SBO = (KC / 8) * 128;   // bytes between 8-row groups
constexpr int A_COLS = KC / 2;                  // tensor-memory columns of one bf16 tile (hi or lo)

// Byte offset of element (row, k) of a rows x KC bf16 block in the canonical
// K-major layout without swizzle: 8 x 16-byte core matrices, K-adjacent core
// matrices 128 bytes apart, 8-row groups CORE_SBO apart.  A block of 2 N rows
// made of two N-row blocks placed one after the other is again canonical.
__host__ __device__ constexpr uint32_t core_off(int row, int k)
{
    return (uint32_t)(row >> 3) * CORE_SBO + (uint32_t)(k >> 3) * CORE_LBO + (uint32_t)(row & 7) * 16u +
           (uint32_t)(k & 7) * 2u;
}

// Per right-hand-side count R: panel chunk layout, tensor-memory plan
// (accumulator [hi*hi + lo*hi | hi*lo] in columns [0, 2N), then A_STAGES tile
// stages of 2 A_COLS columns), copy stages SS.
template <int R>
struct Cfg {
    static constexpr int N = 2 * R;                       // columns of one product: Re then Im
    static constexpr int B_BYTES = N * KC * 2;            // bf16 panel, one of hi / lo
    static constexpr int CHUNK_BYTES = POS_BYTES + 2 * B_BYTES;
    static constexpr int ACC = 2 * N;
    static constexpr int A_STAGES = (512 - ACC) / (2 * A_COLS) >= 3 ? 3 : 2;
    static constexpr int SS = R == 16 ? 6 : R == 32 ? 5 : 3;
    static constexpr int BAR_BYTES = (2 * SS + 2 * A_STAGES + 2) * 8 + 8;
    static constexpr int SMEM = SS * CHUNK_BYTES + (BAR_BYTES + 15) / 16 * 16;
    static_assert(ACC + A_STAGES * 2 * A_COLS <= 512, "tensor memory holds 512 columns");
    static_assert(A_STAGES >= 2 && SS > A_STAGES, "pipeline depth");
    static_assert(SMEM <= 227 * 1024, "shared memory per CTA");
    static_assert(CHUNK_BYTES % 16 == 0 && POS_BYTES % 16 == 0, "bulk copies move multiples of 16 bytes");
};

// ---------------------------------------------------------------- PTX wrappers
__device__ __forceinline__ uint64_t smem_desc(uint32_t saddr)
{
    uint64_t d = 0;
    d |= (uint64_t)((saddr >> 4) & 0x3FFFu);
    d |= (uint64_t)((CORE_LBO >> 4) & 0x3FFFu) << 16;
    d |= (uint64_t)((CORE_SBO >> 4) & 0x3FFFu) << 32;
    d |= (uint64_t)1 << 46;  // descriptor version of tcgen05; base offset 0, no swizzle
    return d;
}

// kind::f16 instruction descriptor: FP32 accumulator, bf16 A and B, both K-major.
__host__ __device__ constexpr uint32_t idesc_bf16(int m, int n)
{
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(n >> 3) << 17) | ((uint32_t)(m >> 4) << 24);
}

// D (tensor memory) (+)= A (tensor memory) x B (shared-memory descriptor)^T
__device__ __forceinline__ void mma_bf16_ta(uint32_t tmem_d, uint32_t tmem_a, uint64_t b, uint32_t idesc, uint32_t acc)
{
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], [%1], %2, %3, p;\n\t}" ::"r"(tmem_d),
        "r"(tmem_a), "l"(b), "r"(idesc), "r"(acc)
        : "memory");
}

__device__ __forceinline__ void mma_commit(uint32_t bar)
{
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar) : "memory");
}

__device__ __forceinline__ void tmem_alloc(uint32_t dst_smem, uint32_t ncols)
{
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(dst_smem), "r"(ncols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}

__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols)
{
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
}

__device__ __forceinline__ void tmem_ld8(uint32_t taddr, uint32_t (&r)[8])
{
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7])
                 : "r"(taddr)
                 : "memory");
}

__device__ __forceinline__ void tmem_ld_wait() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tmem_st4(uint32_t taddr, const uint32_t (&r)[4])
{
    asm volatile("tcgen05.st.sync.aligned.32x32b.x4.b32 [%0], {%1, %2, %3, %4};" ::"r"(taddr), "r"(r[0]), "r"(r[1]),
                 "r"(r[2]), "r"(r[3])
                 : "memory");
}

__device__ __forceinline__ void tmem_st_wait() { asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory"); }

// {upper, lower} halves = bf16(a), bf16(b), round to nearest
__device__ __forceinline__ uint32_t bf16x2(float a, float b)
{
    uint32_t d;
    asm("cvt.rn.bf16x2.f32 %0, %1, %2;" : "=r"(d) : "f"(a), "f"(b));
    return d;
}

// Splits the pair (x0 -> lower half, x1 -> upper half) into bf16 hi and lo parts.
__device__ __forceinline__ void split2(float2 x, uint32_t &hi, uint32_t &lo)
{
    hi = bf16x2(x.y, x.x);
    const float2 nh = make_float2(-__uint_as_float(hi << 16), -__uint_as_float(hi & 0xFFFF0000u));
    const float2 l = __fadd2_rn(x, nh);  // exact: x - hi fits in FP32
    lo = bf16x2(l.y, l.x);
}


__device__ __forceinline__ void mbar_arrive(uint32_t bar)
{
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}

// Bounded wait that also gives up as soon as another thread reported a failure.
__device__ __forceinline__ bool wait_or_abort(uint32_t bar, uint32_t parity, volatile int *abort, int polls)
{
    for (int n = 0; n < polls; ++n) {
        if (mbar_try_wait(bar, parity)) return true;
        if ((n & 255) == 255 && *abort) return false;
    }
    *abort = 1;
    return false;
}

// Poll that suspends the thread until the phase completes or about `ns`
// nanoseconds pass (for the product and copy warps: a spinning poll would take
// issue slots from the generator warps sharing their scheduler).
__device__ __forceinline__ bool mbar_try_wait_hint(uint32_t bar, uint32_t parity, uint32_t ns)
{
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(bar), "r"(parity), "r"(ns)
        : "memory");
    return ok != 0;
}

// Bounded (about a second at most) suspending wait; gives up when another
// thread reported a failure.
__device__ __forceinline__ bool wait_sleep_or_abort(uint32_t bar, uint32_t parity, volatile int *abort, int polls)
{
    for (int n = 0; n < polls; ++n) {
        if (mbar_try_wait_hint(bar, parity, 500u)) return true;
        if ((n & 15) == 15 && *abort) return false;
    }
    *abort = 1;
    return false;
}

// ---------------------------------------------------------------- panel
// Per chunk of KS sources (chunk-major): positions (negated, scaled by k), then
// Bt_hi, Bt_lo: N x KC bf16 in the canonical layout, Bt[n][k] with
//   n <  R: k < KS: Re u_n(s),  k >= KS: -Im u_n(s)
//   n >= R: k < KS: Im u(s),    k >= KS:  Re u(s)      (s = k mod KS)
template <int R>
__global__ void tc_interp_kernel(const int32_t *tri, const double4_32a *pts64, const Rule rule, int64_t nq,
                                 int64_t nq_pad, const double2 *X, int64_t ldx, int c0, int nrhs, float ks, float pad,
                                 unsigned char *panel)
{
    using C = Cfg<R>;
    const int64_t l = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int j = blockIdx.y;
    if (l >= nq_pad || j >= R) return;
    const int64_t chunk = l / KS;
    const int s = (int)(l % KS);
    unsigned char *base = panel + chunk * C::CHUNK_BYTES;
    if (j == 0) {
        float x = pad, y = pad, z = pad;
        if (l < nq) {
            const double4_32a p = pts64[l];
            x = (float)p.x * ks;
            y = (float)p.y * ks;
            z = (float)p.z * ks;
        }
        float *xy = reinterpret_cast<float *>(base);
        float *zz = reinterpret_cast<float *>(base + POS_XY);
        const int pp = s >> 1, lane = s & 1;
        xy[4 * pp + lane] = -x;
        xy[4 * pp + 2 + lane] = -y;
        zz[2 * pp + lane] = -z;
    }
    double ur = 0.0, ui = 0.0;
    if (l < nq && c0 + j < nrhs) {
        const int64_t t = l / rule.q;
        const int kq = (int)(l - t * rule.q);
        const double2 *xc = X + (int64_t)(c0 + j) * ldx;
#pragma unroll
        for (int m = 0; m < 3; ++m) {
            const double2 xv = xc[tri[3 * t + m]];
            const double lam = rule.bary[3 * kq + m];
            ur += lam * xv.x;
            ui += lam * xv.y;
        }
        const double w = pts64[l].w;
        ur *= w;
        ui *= w;
    }
    __nv_bfloat16 *bh = reinterpret_cast<__nv_bfloat16 *>(base + POS_BYTES);
    __nv_bfloat16 *bl = reinterpret_cast<__nv_bfloat16 *>(base + POS_BYTES + C::B_BYTES);
    auto put = [&](int n, int k, double val) {
        const float f = (float)val;
        const __nv_bfloat16 h = __float2bfloat16_rn(f);
        const __nv_bfloat16 lo = __float2bfloat16_rn(f - __bfloat162float(h));
        const uint32_t off = core_off(n, k) / 2;
        bh[off] = h;
        bl[off] = lo;
    };
    put(j, s, ur);
    put(j, KS + s, -ui);
    put(R + j, s, ui);
    put(R + j, KS + s, ur);
}

// ---------------------------------------------------------------- kernel
struct TcArgs {
    const unsigned char *panel;
    const float4 *tgt;
    double2 *v;       // column c0 of the accumulators
    int64_t ldv;
    int64_t nq;       // targets = sources
    int64_t n_chunks; // source chunks (padded)
    int64_t n_tiles;  // target tiles of M
    int64_t t_begin, t_end;  // target points [t_begin, t_end) (a range of test triangles)
    int64_t n_segs;   // source segments of SEG_CHUNKS chunks
    int ncols;        // valid right-hand sides in this pass (<= R)
    float ks;
    int *err;
    int polls_spin;   // poll limits of the pipeline waits (spinning / suspending); the
    int polls_sleep;  // drain after a failure keeps the default limit
};

// Kernel values of one generator thread (its row = its tensor-memory lane) for
// group q (8 sources) of its slice of the chunk (KS / GPR sources): bf16 hi/lo
// pairs of Gr and Gi, sources (2p, 2p + 1) in the (lower, upper) halves.
constexpr int SRC_PER = KS / GPR;
constexpr int GROUPS_PER_CHUNK = SRC_PER / 8;

struct Group {
    uint32_t hr[4], lr[4], hi[4], li[4];
};

template <bool CHECK>
__device__ __forceinline__ void gen_group(const unsigned char *src, int q, float2 tx, float2 ty, float2 tz,
                                          int64_t tgt, int64_t src0, int slice, Group &g)
{
    const float4 *XY = reinterpret_cast<const float4 *>(src);
    const float2 *Z = reinterpret_cast<const float2 *>(src + POS_XY);
    const float2 magic = make_float2(12582912.0f, 12582912.0f);
    const float2 nmagic = make_float2(-12582912.0f, -12582912.0f);
    const float2 inv2pi = make_float2(0.159154943091895335769f, 0.159154943091895335769f);
    const float2 m2pi = make_float2(-6.28318530717958647692f, -6.28318530717958647692f);
#pragma unroll
    for (int p4 = 0; p4 < 4; ++p4) {
        const int pp = (slice * SRC_PER + q * 8) / 2 + p4;  // source pair within the chunk
        const float4 xy = XY[pp];
        const float2 sz = Z[pp];
        float2 dx = __fadd2_rn(tx, make_float2(xy.x, xy.y));
        float2 dy = __fadd2_rn(ty, make_float2(xy.z, xy.w));
        float2 dz = __fadd2_rn(tz, sz);
        float2 r2 = __fmul2_rn(dx, dx);
        r2 = __ffma2_rn(dy, dy, r2);
        r2 = __ffma2_rn(dz, dz, r2);
        const float2 rs = make_float2(rsqrt_mufu(r2.x), rsqrt_mufu(r2.y));
        const float2 ph = __fmul2_rn(r2, rs);
        const float2 nr = __fadd2_rn(__ffma2_rn(ph, inv2pi, magic), nmagic);
        const float2 ang = __ffma2_rn(nr, m2pi, ph);
        float2 gre = __fmul2_rn(make_float2(cos_mufu(ang.x), cos_mufu(ang.y)), rs);
        float2 gim = __fmul2_rn(make_float2(sin_mufu(ang.x), sin_mufu(ang.y)), rs);
        if (CHECK) {
            if (src0 + 2 * pp == tgt) {
                gre.x = 0.0f;
                gim.x = 1.0f;
            }
            if (src0 + 2 * pp + 1 == tgt) {
                gre.y = 0.0f;
                gim.y = 1.0f;
            }
        }
        split2(gre, g.hr[p4], g.lr[p4]);
        split2(gim, g.hi[p4], g.li[p4]);
    }
}

// Stores group q: Gr at K = s, Gi at K = KS + s; bf16 pairs (2c, 2c + 1) of K
// share tensor-memory column c.
__device__ __forceinline__ void st_group(uint32_t ta_hi, uint32_t ta_lo, int q, int slice, const Group &g)
{
    const uint32_t cre = (uint32_t)(slice * SRC_PER + q * 8) / 2, cim = cre + KS / 2;
    tmem_st4(ta_hi + cre, g.hr);
    tmem_st4(ta_hi + cim, g.hi);
    tmem_st4(ta_lo + cre, g.lr);
    tmem_st4(ta_lo + cim, g.li);
}

__device__ __forceinline__ bool mbar_test_wait(uint32_t bar, uint32_t parity)
{
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.test_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(bar), "r"(parity)
        : "memory");
    return ok != 0;
}

// Warp-specialised persistent kernel, one CTA per SM (it takes all 512 columns
// of tensor memory).  Work items (target tile, source segment) in
// segment-major order, CTA b taking items b, b + grid, ...: the CTAs in flight
// read the same source segment, which stays in L2.  Roles and hand-offs:
//   generator warps 0..15  (row = lane quadrant of the warp, GPR slices per row)
//   product warp 16        lane 0 issues the products and the commits
//   copy warp 17           lane 0 issues the bulk copies of the panel
//   src_full[s]   copy of the chunk landed in stage s (count 1 + tx bytes)
//   src_empty[s]  products that read stage s finished (tcgen05.commit)
//   a_full[t]     every generator warp stored its part of tile stage t (count 16)
//   mma_done[t]   products that read tile stage t finished (tcgen05.commit)
//   acc_full      all products of a work item finished: accumulator ready
//   acc_empty     every generator warp read the accumulator (count 16)
// Every wait is bounded; a wait that runs out sets the error word and the
// abort flag, after which every role stops, waits (bounded) for its copies and
// products in flight, and the CTA frees its tensor memory.
template <int R>
__global__ void __launch_bounds__(NT, 1) far_tc_kernel(const TcArgs a)
{
    using C = Cfg<R>;
    constexpr int SS = C::SS, AS = C::A_STAGES;
    constexpr int BAR_OFF = SS * C::CHUNK_BYTES;
    extern __shared__ __align__(1024) unsigned char smem[];
    uint64_t *src_full = reinterpret_cast<uint64_t *>(smem + BAR_OFF);  // [SS]
    uint64_t *src_empty = src_full + SS;                                // [SS]
    uint64_t *a_full = src_empty + SS;                                  // [AS]
    uint64_t *mma_done = a_full + AS;                                   // [AS]
    uint64_t *acc_full = mma_done + AS;
    uint64_t *acc_empty = acc_full + 1;
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(acc_empty + 1);
    volatile int *abort = reinterpret_cast<volatile int *>(tmem_slot + 1);
    const int th = threadIdx.x, warp = th >> 5, lane = th & 31;

    const int64_t n_tiles = a.n_tiles, n_segs = a.n_segs, n_chunks = a.n_chunks, nq = a.nq;
    const int64_t items = n_tiles * n_segs;
    const int64_t ifirst = blockIdx.x, istep = gridDim.x;
    const int64_t icount = items > ifirst ? (items - ifirst + istep - 1) / istep : 0;
    if (icount <= 0) return;
    auto seg_of = [n_tiles](int64_t i) { return i / n_tiles; };
    auto chunks_of = [n_chunks](int64_t seg) { return (int)min((int64_t)SEG_CHUNKS, n_chunks - seg * SEG_CHUNKS); };

    if (th == 0) {
        for (int s = 0; s < SS; ++s) {
            mbar_init(smem_addr(&src_full[s]), 1);
            mbar_init(smem_addr(&src_empty[s]), 1);
        }
        for (int s = 0; s < AS; ++s) {
            mbar_init(smem_addr(&a_full[s]), NGEN / 32);
            mbar_init(smem_addr(&mma_done[s]), 1);
        }
        mbar_init(smem_addr(acc_full), 1);
        mbar_init(smem_addr(acc_empty), NGEN / 32);
        *abort = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) tmem_alloc(smem_addr(tmem_slot), 512);
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tmem_slot;
    bool ok = true;

    if (warp == NGEN / 32) {
        // ------------------------------------------------------------ product warp
        const bool leader = lane == 0;
        constexpr uint32_t idesc2 = idesc_bf16(M, 2 * C::N), idesc1 = idesc_bf16(M, C::N);
        // descriptor of the hi panel of stage 0 at K = 0; stage and K offsets add to
        // its address field (shared addresses stay below 256 KB: no carry out of it)
        const uint64_t bdesc0 = smem_desc(smem_addr(smem + POS_BYTES));
        int n = 0, sa = 0, ss = 0;
        uint32_t pa = 0, ps = 0;
        for (int64_t it = 0; it < icount && ok; ++it) {
            const int nc = chunks_of(seg_of(ifirst + it * istep));
            if (it > 0)
                ok = __all_sync(0xffffffffu, wait_sleep_or_abort(smem_addr(acc_empty), (uint32_t)((it - 1) & 1), abort, a.polls_sleep));
            for (int c = 0; c < nc && ok; ++c) {
                ok = wait_sleep_or_abort(smem_addr(&a_full[sa]), pa, abort, a.polls_sleep) &&
                     wait_sleep_or_abort(smem_addr(&src_full[ss]), ps, abort, a.polls_sleep);
                ok = __all_sync(0xffffffffu, ok);
                if (!ok) break;
                tc_fence_after();
                const uint32_t ah = tmem + (uint32_t)(C::ACC + sa * 2 * A_COLS), al = ah + A_COLS;
                const uint64_t bdh = bdesc0 + (uint64_t)((ss * C::CHUNK_BYTES) >> 4);
                if (leader) {
#pragma unroll
                    for (int kk = 0; kk < KC / 16; ++kk) {
                        const uint64_t boff = (uint64_t)(kk * 2 * CORE_LBO) >> 4;  // 16 K = two core matrices
                        const uint32_t aoff = kk * 8;                              // 16 K = 8 columns
                        // [hi*hi | hi*lo] += A_hi [B_hi | B_lo]; then hi*hi += A_lo B_hi
                        mma_bf16_ta(tmem, ah + aoff, bdh + boff, idesc2, (c > 0 || kk > 0) ? 1u : 0u);
                        mma_bf16_ta(tmem, al + aoff, bdh + boff, idesc1, 1u);
                    }
                    mma_commit(smem_addr(&mma_done[sa]));
                    mma_commit(smem_addr(&src_empty[ss]));
                    if (c == nc - 1) mma_commit(smem_addr(acc_full));
                }
                __syncwarp();
                ++n;
                if (++sa == AS) {
                    sa = 0;
                    pa ^= 1;
                }
                if (++ss == SS) {
                    ss = 0;
                    ps ^= 1;
                }
            }
        }
        if (leader) {
            if (!ok) {
                atomicExch(a.err, 1);
                *abort = 1;
            }
            if (n > 0) {  // the last products must finish before the tensor memory is freed
                const int nl = n - 1;
                mbar_wait_bounded(smem_addr(&mma_done[nl % AS]), (uint32_t)((nl / AS) & 1));
            }
        }
        __syncwarp();
    } else if (warp == NGEN / 32 + 1) {
        // ------------------------------------------------------------ copy warp
        const bool leader = lane == 0;
        const unsigned char *panel = a.panel;
        int j = 0;  // copies issued
        for (int64_t it = 0; it < icount && ok; ++it) {
            const int64_t seg = seg_of(ifirst + it * istep);
            const int nc = chunks_of(seg);
            for (int c = 0; c < nc; ++c, ++j) {
                const int s = j % SS;
                if (j >= SS) {  // the products of chunk j - SS, the stage's last user, finished
                    ok = __all_sync(0xffffffffu,
                                    wait_sleep_or_abort(smem_addr(&src_empty[s]), (uint32_t)((j / SS - 1) & 1), abort, a.polls_sleep));
                    if (!ok) break;
                }
                if (leader) {
                    const uint32_t bar = smem_addr(&src_full[s]);
                    mbar_expect_tx(bar, C::CHUNK_BYTES);
                    bulk_g2s(smem_addr(smem + s * C::CHUNK_BYTES),
                             panel + (seg * SEG_CHUNKS + c) * (int64_t)C::CHUNK_BYTES, C::CHUNK_BYTES, bar);
                }
                __syncwarp();
            }
        }
        if (leader) {
            if (!ok) {
                atomicExch(a.err, 1);
                *abort = 1;
            }
            // copies in flight must land before the CTA exits
            for (int jj = max(0, j - SS); jj < j; ++jj)
                mbar_wait_bounded(smem_addr(&src_full[jj % SS]), (uint32_t)((jj / SS) & 1));
        }
        __syncwarp();
    } else {
        // ------------------------------------------------------------ generator warps
        const int row = th & (M - 1), slice = th / M;
        const int quad = warp & 3;  // lane quadrant of tensor memory this warp may access
        const uint32_t lane_base = tmem + ((uint32_t)(quad * 32) << 16);
        const float ks = a.ks;
        int n = 0, sa = 0, ss = 0;
        uint32_t pa = 0, ps = 0;
        bool src_ready = false;  // the panel chunk of the next chunk was seen complete
        for (int64_t it = 0; it < icount && ok; ++it) {
            const int64_t item = ifirst + it * istep;
            const int64_t seg = seg_of(item), tile = item - seg * n_tiles;
            const int64_t t0 = a.t_begin + tile * M;
            const int64_t tgt = t0 + row;
            const float4 p = a.tgt[min(tgt, a.t_end - 1)];
            const float2 tx = make_float2(p.x * ks, p.x * ks);
            const float2 ty = make_float2(p.y * ks, p.y * ks);
            const float2 tz = make_float2(p.z * ks, p.z * ks);
            const int nc = chunks_of(seg);
            int64_t src0 = seg * SEG_CHUNKS * KS;
            for (int c = 0; c < nc; ++c, ++n, src0 += KS) {
                // The waits sit where their latency overlaps the special-function
                // work: the panel chunk before the first group, the tile stage (free
                // once the products of chunk n - A_STAGES finished) after it, and a
                // non-blocking test of the next chunk's panel after the last group.
                if (!src_ready) ok = wait_or_abort(smem_addr(&src_full[ss]), ps, abort, a.polls_spin);
                ok = __all_sync(0xffffffffu, ok);  // tcgen05.st is warp-collective
                if (!ok) break;
                const unsigned char *src = smem + ss * C::CHUNK_BYTES;
                const uint32_t ta_hi = lane_base + (uint32_t)(C::ACC + sa * 2 * A_COLS), ta_lo = ta_hi + A_COLS;
                const bool diag = t0 < src0 + KS && src0 < t0 + M;  // the chunk holds targets of this tile
#pragma unroll
                for (int q = 0; q < GROUPS_PER_CHUNK; ++q) {
                    Group g;
                    if (diag)
                        gen_group<true>(src, q, tx, ty, tz, tgt, src0, slice, g);
                    else
                        gen_group<false>(src, q, tx, ty, tz, tgt, src0, slice, g);
                    if (q == 0) {
                        if (n >= AS) ok = wait_or_abort(smem_addr(&mma_done[sa]), pa ^ 1u, abort, a.polls_spin);
                        ok = __all_sync(0xffffffffu, ok);
                        if (!ok) break;
                        tc_fence_after();
                    }
                    st_group(ta_hi, ta_lo, q, slice, g);
                }
                if (!ok) break;
                const int ss_next = ss + 1 == SS ? 0 : ss + 1;
                const uint32_t ps_next = ss + 1 == SS ? ps ^ 1u : ps;
                src_ready = __all_sync(0xffffffffu, mbar_test_wait(smem_addr(&src_full[ss_next]), ps_next));
                tmem_st_wait();
                tc_fence_before();
                __syncwarp();
                if (lane == 0) mbar_arrive(smem_addr(&a_full[sa]));
                if (++sa == AS) {
                    sa = 0;
                    pa ^= 1;
                }
                ss = ss_next;
                ps = ps_next;
            }
            if (!ok) break;
            // epilogue: this item's accumulator, [hi*hi + lo*hi | hi*lo]
            ok = __all_sync(0xffffffffu, wait_or_abort(smem_addr(acc_full), (uint32_t)(it & 1), abort, a.polls_spin));
            if (!ok) break;
            tc_fence_after();
            constexpr int GROUPS = NGEN / 32 / 4;  // warps sharing one lane quadrant
            constexpr int COLS = C::N / GROUPS;    // accumulator columns per warp
            const int grp = warp >> 2;
            const int64_t trow = t0 + quad * 32 + lane;
            constexpr int LD = 8;  // columns per tcgen05.ld
            static_assert(COLS % LD == 0, "accumulator columns per warp");
#pragma unroll
            for (int cb = 0; cb < COLS / LD; ++cb) {
                const int col0 = grp * COLS + cb * LD;
                uint32_t r0[8], r1[8];
                tmem_ld8(lane_base + (uint32_t)col0, r0);
                tmem_ld8(lane_base + (uint32_t)(C::N + col0), r1);
                tmem_ld_wait();
                if (trow < a.t_end) {
#pragma unroll
                    for (int i = 0; i < LD; ++i) {
                        const int col = col0 + i;
                        const int part = col >= R ? 1 : 0;  // Re columns first, then Im
                        const int jj = col - part * R;
                        if (jj < a.ncols) {
                            const float f = __uint_as_float(r0[i]) + __uint_as_float(r1[i]);
                            double *dst = reinterpret_cast<double *>(a.v + trow + (int64_t)jj * a.ldv) + part;
                            atomicAdd(dst, (double)f * (double)ks);
                        }
                    }
                }
            }
            tc_fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive(smem_addr(acc_empty));
        }
        tmem_st_wait();
        if (!ok && lane == 0) {
            atomicExch(a.err, 1);
            *abort = 1;
        }
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 0) {
        tc_fence_after();
        tmem_dealloc(tmem, 512);
    }
}

template <int R>
gyps_status run(Mesh *m, double k, const double2 *X, int64_t ldx, int nrhs, double2 *v, int64_t ldv, int64_t t_begin,
                int64_t t_end, cudaStream_t s)
{
    using C = Cfg<R>;
    const int64_t n_chunks = (m->nq + KS - 1) / KS;
    const size_t panel_bytes = (size_t)n_chunks * C::CHUNK_BYTES;
    GYPS_TRY(grow(m, &m->ws_tc, &m->ws_tc_bytes, panel_bytes));
    unsigned char *panel = reinterpret_cast<unsigned char *>(m->ws_tc);
    TcArgs a;
    a.panel = panel;
    a.tgt = m->d_pts32;
    a.v = v;
    a.ldv = ldv;
    a.nq = m->nq;
    a.n_chunks = n_chunks;
    a.t_begin = t_begin;
    a.t_end = t_end;
    a.n_tiles = (t_end - t_begin + M - 1) / M;
    a.n_segs = (n_chunks + SEG_CHUNKS - 1) / SEG_CHUNKS;
    a.ncols = 0;
    a.ks = (float)k;
    a.err = m->d_err;
    const int wp = wait_polls_setting();
    a.polls_spin = wp >= 0 ? wp : (1 << 22);
    a.polls_sleep = wp >= 0 ? wp : (1 << 21);
    GYPS_CUDA(cudaFuncSetAttribute(far_tc_kernel<R>, cudaFuncAttributeMaxDynamicSharedMemorySize, C::SMEM));
    // one CTA per SM: each takes the whole tensor memory
    const int64_t grid = std::min<int64_t>((int64_t)m->num_sms, a.n_tiles * a.n_segs);
    for (int c0 = 0; c0 < nrhs; c0 += R) {
        StageTimer ti(m, s, 0);
        dim3 gi((unsigned)((n_chunks * KS + 255) / 256), (unsigned)R);
        tc_interp_kernel<R><<<gi, 256, 0, s>>>(m->d_tri, m->d_pts64, m->rule, m->nq, n_chunks * KS, X, ldx, c0, nrhs,
                                                a.ks, m->pad, panel);
        GYPS_CUDA(cudaGetLastError());
        ti.done(1);
        a.v = v + (int64_t)c0 * a.ldv;
        a.ncols = std::min(R, nrhs - c0);
        StageTimer tf(m, s, 1);
        far_tc_kernel<R><<<(unsigned)grid, NT, C::SMEM, s>>>(a);
        GYPS_CUDA(cudaGetLastError());
        tf.done(1);
    }
    return GYPS_OK;
}

}  // namespace tc

gyps_status far_tc(Mesh *m, double k, const double2 *X, int64_t ldx, int nrhs, double2 *v, int64_t ldv,
                   int64_t t_begin, int64_t t_end, cudaStream_t s)
{
    if (t_end <= t_begin) return GYPS_OK;
    // widest pass that the right-hand sides fill: every pass regenerates the kernel tiles
    if (nrhs >= 64) {
        const int full = nrhs / 64 * 64;
        GYPS_TRY(tc::run<64>(m, k, X, ldx, full, v, ldv, t_begin, t_end, s));
        if (full == nrhs) return GYPS_OK;
        return far_tc(m, k, X + (int64_t)full * ldx, ldx, nrhs - full, v + (int64_t)full * ldv, ldv, t_begin, t_end, s);
    }
    if (nrhs > 16) return tc::run<32>(m, k, X, ldx, nrhs, v, ldv, t_begin, t_end, s);
    return tc::run<16>(m, k, X, ldx, nrhs, v, ldv, t_begin, t_end, s);
}

}  // namespace gyps
