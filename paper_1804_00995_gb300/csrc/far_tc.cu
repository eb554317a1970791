// Tensor-core form of the dense kernel product (Sec. 5, Eq. (BEM): v = G u) for
// 16 or more right-hand sides.  In real arithmetic the complex product is
//   [Re v | Im v] = [Gr | Gi] * [[Ur, Ui], [-Ui, Ur]],
// a (128 targets) x (2 Ks) by (2 Ks) x (2 R) contraction per source chunk of Ks
// points.  The CUDA cores generate the kernel tile G = exp(ikr)/(kr) in FP32
// (the MUFU path of the FP32 kernel), split every value into bf16 hi + lo and
// store both in shared memory in the canonical K-major layout; one thread issues
// tcgen05.mma (kind::f16, bf16 inputs, FP32 accumulation in tensor memory) for
// the three split products hi*hi + hi*lo + lo*hi against the bf16 hi/lo panel of
// the densities, which 1-D bulk copies stage per chunk.  The epilogue reads the
// accumulator with tcgen05.ld and adds k * (Re, Im) into the FP64 sums.
#include <algorithm>
#include <cmath>

#include <cuda_bf16.h>

#include "far_tile.cuh"
#include "internal.h"

namespace gyps {
namespace tc {

constexpr int M = 128;          // targets per tile = tensor-memory lanes
constexpr int KS = 32;          // sources per chunk
constexpr int KC = 2 * KS;      // K extent per chunk: Gr for the chunk, then Gi
constexpr int NTHR = 256;       // 8 warps, two per target row (each half the chunk)
constexpr int SEG_CHUNKS = 128; // chunks per work item (4096 sources)
constexpr int POS_BYTES = 384;  // float4 XY[16] + float2 Z[16] (negated, scaled by k)
constexpr uint32_t CORE_LBO = 128;            // bytes between core matrices along K
constexpr uint32_t CORE_SBO = (KC / 8) * 128; // bytes between 8-row groups

// Byte offset of element (row, k) of a rows x KC bf16 block in the canonical
// K-major layout without swizzle: 8 x 16-byte core matrices, K-adjacent core
// matrices 128 bytes apart, 8-row groups CORE_SBO apart.
__host__ __device__ constexpr uint32_t core_off(int row, int k)
{
    return (uint32_t)(row >> 3) * CORE_SBO + (uint32_t)(k >> 3) * CORE_LBO + (uint32_t)(row & 7) * 16u +
           (uint32_t)(k & 7) * 2u;
}

template <int R>
struct Cfg {
    static constexpr int N = 2 * R;                       // accumulator columns: Re then Im
    static constexpr int B_BYTES = N * KC * 2;            // bf16 panel, one of hi / lo
    static constexpr int CHUNK_BYTES = POS_BYTES + 2 * B_BYTES;
    static constexpr int A_BYTES = M * KC * 2;            // bf16 kernel tile, one of hi / lo
    static constexpr int TMEM_COLS = N < 32 ? 32 : N;
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

__device__ __forceinline__ void mma_bf16(uint32_t tmem_d, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc)
{
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(tmem_d),
        "l"(a), "l"(b), "r"(idesc), "r"(acc)
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

__device__ __forceinline__ void tmem_ld16(uint32_t taddr, uint32_t (&r)[16])
{
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
        "%15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
          "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr)
        : "memory");
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
__device__ __forceinline__ void fence_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

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
        float *zz = reinterpret_cast<float *>(base + 256);
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
    int64_t n_segs;   // source segments of SEG_CHUNKS chunks
    int ncols;        // valid right-hand sides in this pass (<= R)
    float ks;
    int *err;
};

// Kernel tile of one generator thread: target `row`, the GPR sources of its
// slice of the chunk, split into bf16 hi/lo and stored at K = s (Gr) and
// K = KS + s (Gi).
template <int GPR, bool CHECK>
__device__ __forceinline__ void gen_chunk(const unsigned char *src, unsigned char *a_hi, unsigned char *a_lo,
                                          float2 tx, float2 ty, float2 tz, int64_t tgt, int64_t src0, int row,
                                          int slice)
{
    constexpr int SRC_PER = KS / GPR;  // sources per thread (8 or 16)
    const float4 *XY = reinterpret_cast<const float4 *>(src);
    const float2 *Z = reinterpret_cast<const float2 *>(src + 256);
    const float2 magic = make_float2(12582912.0f, 12582912.0f);
    const float2 nmagic = make_float2(-12582912.0f, -12582912.0f);
    const float2 inv2pi = make_float2(0.159154943091895335769f, 0.159154943091895335769f);
    const float2 m2pi = make_float2(-6.28318530717958647692f, -6.28318530717958647692f);
#pragma unroll
    for (int q = 0; q < SRC_PER / 8; ++q) {  // groups of 8 sources = one core-matrix row
        uint32_t hr[4], lr[4], hi_[4], li[4];
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
            split2(gre, hr[p4], lr[p4]);
            split2(gim, hi_[p4], li[p4]);
        }
        const int kre = slice * SRC_PER + q * 8;
        const uint32_t ore = core_off(row, kre), oim = core_off(row, KS + kre);
        *reinterpret_cast<uint4 *>(a_hi + ore) = make_uint4(hr[0], hr[1], hr[2], hr[3]);
        *reinterpret_cast<uint4 *>(a_lo + ore) = make_uint4(lr[0], lr[1], lr[2], lr[3]);
        *reinterpret_cast<uint4 *>(a_hi + oim) = make_uint4(hi_[0], hi_[1], hi_[2], hi_[3]);
        *reinterpret_cast<uint4 *>(a_lo + oim) = make_uint4(li[0], li[1], li[2], li[3]);
    }
}

__device__ __forceinline__ void mbar_arrive(uint32_t bar)
{
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}

// Bounded wait that also gives up as soon as another thread reported a failure.
__device__ __forceinline__ bool wait_or_abort(uint32_t bar, uint32_t parity, volatile int *abort)
{
    for (int n = 0; n < (1 << 22); ++n) {
        if (mbar_try_wait(bar, parity)) return true;
        if ((n & 255) == 255 && *abort) return false;
    }
    *abort = 1;
    return false;
}

// Warp-specialised kernel: GPR generator threads per target row (warps
// 0 .. 4 GPR - 1) and one control warp (the last) whose lane 0 issues the bulk
// copies of the density panel and the tensor-core products.  Hand-offs:
//   src_full[s]  copy of chunk n landed (count 1 + tx bytes)
//   a_full[s]    all generators wrote the kernel tile of chunk n (count 128 GPR)
//   mma_done[s]  products of chunk n finished (tcgen05.commit): tile and copy stage free
//   acc_full     all products of a work item finished: accumulator ready
//   acc_empty    every generator read the accumulator (count 128 GPR)
template <int R, int GPR, int SS, int A_STAGES>
__global__ void __launch_bounds__(M * GPR + 32) far_tc_kernel(const TcArgs a)
{
    using C = Cfg<R>;
    constexpr int NGEN = M * GPR;
    constexpr int SRC_OFF = A_STAGES * 2 * C::A_BYTES;
    constexpr int BAR_OFF = SRC_OFF + SS * C::CHUNK_BYTES;
    extern __shared__ __align__(1024) unsigned char smem[];
    uint64_t *src_full = reinterpret_cast<uint64_t *>(smem + BAR_OFF);  // [SS]
    uint64_t *a_full = src_full + SS;                                   // [A_STAGES]
    uint64_t *mma_done = a_full + A_STAGES;                             // [A_STAGES]
    uint64_t *acc_full = mma_done + A_STAGES;
    uint64_t *acc_empty = acc_full + 1;
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(acc_empty + 1);
    volatile int *abort = reinterpret_cast<volatile int *>(tmem_slot + 1);
    const int th = threadIdx.x, warp = th >> 5, lane = th & 31;

    const int64_t items = a.n_tiles * a.n_segs;
    const int64_t ibeg = items * blockIdx.x / gridDim.x;
    const int64_t iend = items * (blockIdx.x + 1) / gridDim.x;
    if (ibeg >= iend) return;

    if (th == 0) {
        for (int s = 0; s < SS; ++s) mbar_init(smem_addr(&src_full[s]), 1);
        for (int s = 0; s < A_STAGES; ++s) {
            mbar_init(smem_addr(&a_full[s]), NGEN);
            mbar_init(smem_addr(&mma_done[s]), 1);
        }
        mbar_init(smem_addr(acc_full), 1);
        mbar_init(smem_addr(acc_empty), NGEN);
        *abort = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) tmem_alloc(smem_addr(tmem_slot), C::TMEM_COLS);
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tmem_slot;

    // kernel parameters in registers (no reference to the parameter block)
    const int64_t n_segs = a.n_segs, n_chunks = a.n_chunks, nq = a.nq;
    const unsigned char *panel = a.panel;
    const float ks = a.ks;

    if (warp == NGEN / 32) {
        // ------------------------------------------------------------ control warp
        if (lane == 0) {
            constexpr uint32_t idesc = idesc_bf16(M, C::N);
            // copy producer: item, chunk within it, chunks in it
            int64_t p_item = ibeg;
            int64_t p_seg = p_item % n_segs;
            int p_c = 0;
            int p_nc = (int)min((int64_t)SEG_CHUNKS, n_chunks - p_seg * SEG_CHUNKS);
            int issued = 0, c_stage = 0;
            uint32_t c_par = 0;
            int n = 0;  // chunks whose products were issued
            int sa = 0, ss = 0;
            uint32_t pa = 0, ps = 0;
            bool ok = true;
            for (int64_t item = ibeg; item < iend && ok; ++item) {
                const int64_t seg = item % n_segs;
                const int nc = (int)min((int64_t)SEG_CHUNKS, n_chunks - seg * SEG_CHUNKS);
                if (item > ibeg) ok = wait_or_abort(smem_addr(acc_empty), (uint32_t)((item - ibeg - 1) & 1), abort);
                for (int c = 0; c < nc && ok; ++c) {
                    // copies run up to SS - 1 chunks ahead; a copy stage is free once the
                    // products of the chunk that used it (SS chunks earlier) finished
                    while (p_item < iend && issued < n + SS) {
                        if (issued >= SS) {
                            const int prev = issued - SS;  // last user of this copy stage
                            if (prev >= n) break;         // its products are not issued yet
                            ok = wait_or_abort(smem_addr(&mma_done[prev % A_STAGES]),
                                               (uint32_t)((prev / A_STAGES) & 1), abort);
                            if (!ok) break;
                        }
                        const uint32_t bar = smem_addr(&src_full[c_stage]);
                        mbar_expect_tx(bar, C::CHUNK_BYTES);
                        bulk_g2s(smem_addr(smem + SRC_OFF + c_stage * C::CHUNK_BYTES),
                                 panel + (p_seg * SEG_CHUNKS + p_c) * (int64_t)C::CHUNK_BYTES, C::CHUNK_BYTES, bar);
                        ++issued;
                        if (++c_stage == SS) {
                            c_stage = 0;
                            c_par ^= 1;
                        }
                        if (++p_c == p_nc) {
                            p_c = 0;
                            if (++p_item < iend) {
                                p_seg = p_item % n_segs;
                                p_nc = (int)min((int64_t)SEG_CHUNKS, n_chunks - p_seg * SEG_CHUNKS);
                            }
                        }
                    }
                    if (!ok) break;
                    ok = wait_or_abort(smem_addr(&a_full[sa]), pa, abort) &&
                         wait_or_abort(smem_addr(&src_full[ss]), ps, abort);
                    if (!ok) break;
                    tc_fence_after();
                    const uint32_t ah = smem_addr(smem + sa * 2 * C::A_BYTES), al = ah + C::A_BYTES;
                    const uint32_t bh = smem_addr(smem + SRC_OFF + ss * C::CHUNK_BYTES + POS_BYTES);
                    const uint32_t bl = bh + C::B_BYTES;
#pragma unroll
                    for (int kk = 0; kk < KC / 16; ++kk) {
                        const uint32_t off = kk * 2 * CORE_LBO;
                        const uint32_t acc0 = (c > 0 || kk > 0) ? 1u : 0u;
                        mma_bf16(tmem, smem_desc(ah + off), smem_desc(bh + off), idesc, acc0);
                        mma_bf16(tmem, smem_desc(ah + off), smem_desc(bl + off), idesc, 1u);
                        mma_bf16(tmem, smem_desc(al + off), smem_desc(bh + off), idesc, 1u);
                    }
                    mma_commit(smem_addr(&mma_done[sa]));
                    if (c == nc - 1) mma_commit(smem_addr(acc_full));
                    ++n;
                    if (++sa == A_STAGES) {
                        sa = 0;
                        pa ^= 1;
                    }
                    if (++ss == SS) {
                        ss = 0;
                        ps ^= 1;
                    }
                }
            }
            if (!ok) {
                atomicExch(a.err, 1);
                *abort = 1;
            }
            // drain: copies and products in flight must land before the CTA exits
            for (int j = n; j < issued; ++j)
                mbar_wait_bounded(smem_addr(&src_full[j % SS]), (uint32_t)((j / SS) & 1));
            if (n > 0) {
                const int nl = n - 1;
                mbar_wait_bounded(smem_addr(&mma_done[nl % A_STAGES]), (uint32_t)((nl / A_STAGES) & 1));
            }
        }
        __syncwarp();
    } else {
        // ------------------------------------------------------------ generator warps
        const int row = th & (M - 1), slice = th / M;
        int n = 0, sa = 0, ss = 0;
        uint32_t pa = 0, ps = 0;  // parity of the current use of stage sa / ss
        bool ok = true;
        int64_t item_count = 0;
        for (int64_t item = ibeg; item < iend && ok; ++item, ++item_count) {
            const int64_t tile = item / n_segs;
            const int64_t seg = item - tile * n_segs;
            const int64_t t0 = tile * M;
            const int64_t tgt = t0 + row;
            const float4 p = a.tgt[min(tgt, nq - 1)];
            const float2 tx = make_float2(p.x * ks, p.x * ks);
            const float2 ty = make_float2(p.y * ks, p.y * ks);
            const float2 tz = make_float2(p.z * ks, p.z * ks);
            const int nc = (int)min((int64_t)SEG_CHUNKS, n_chunks - seg * SEG_CHUNKS);
            int64_t src0 = seg * SEG_CHUNKS * KS;
            for (int c = 0; c < nc; ++c, ++n, src0 += KS) {
                if (n >= A_STAGES) ok = wait_or_abort(smem_addr(&mma_done[sa]), pa ^ 1u, abort);
                ok = ok && wait_or_abort(smem_addr(&src_full[ss]), ps, abort);
                if (!ok) break;
                const unsigned char *src = smem + SRC_OFF + ss * C::CHUNK_BYTES;
                unsigned char *a_hi = smem + sa * 2 * C::A_BYTES;
                unsigned char *a_lo = a_hi + C::A_BYTES;
                if (t0 < src0 + KS && src0 < t0 + M)
                    gen_chunk<GPR, true>(src, a_hi, a_lo, tx, ty, tz, tgt, src0, row, slice);
                else
                    gen_chunk<GPR, false>(src, a_hi, a_lo, tx, ty, tz, tgt, src0, row, slice);
                fence_async_smem();
                mbar_arrive(smem_addr(&a_full[sa]));
                if (++sa == A_STAGES) {
                    sa = 0;
                    pa ^= 1;
                }
                if (++ss == SS) {
                    ss = 0;
                    ps ^= 1;
                }
            }
            if (!ok) break;
            // epilogue: this item's accumulator
            ok = wait_or_abort(smem_addr(acc_full), (uint32_t)(item_count & 1), abort);
            if (!ok) break;
            tc_fence_after();
            constexpr int GROUPS = NGEN / 32 / 4;      // warps sharing one lane quadrant
            constexpr int COLS = C::N / GROUPS;        // accumulator columns per warp
            const int quad = warp & 3, grp = warp >> 2;
            const int64_t trow = t0 + quad * 32 + lane;
            constexpr int LD = COLS >= 16 ? 16 : 8;  // columns per tcgen05.ld
            static_assert(COLS % LD == 0, "accumulator columns per warp");
#pragma unroll
            for (int cb = 0; cb < COLS / LD; ++cb) {
                uint32_t r[16];
                const int col0 = grp * COLS + cb * LD;
                const uint32_t taddr = tmem + ((uint32_t)(quad * 32) << 16) + (uint32_t)col0;
                if (LD == 16) {
                    tmem_ld16(taddr, r);
                } else {
                    uint32_t r8[8];
                    tmem_ld8(taddr, r8);
#pragma unroll
                    for (int i = 0; i < 8; ++i) r[i] = r8[i];
                }
                tmem_ld_wait();
                if (trow < nq) {
#pragma unroll
                    for (int i = 0; i < LD; ++i) {
                        const int col = col0 + i;
                        const int part = col >= R ? 1 : 0;  // Re columns first, then Im
                        const int jj = col - part * R;
                        if (jj < a.ncols) {
                            double *dst = reinterpret_cast<double *>(a.v + trow + (int64_t)jj * a.ldv) + part;
                            atomicAdd(dst, (double)__uint_as_float(r[i]) * (double)ks);
                        }
                    }
                }
            }
            tc_fence_before();
            mbar_arrive(smem_addr(acc_empty));
        }
        if (!ok) {
            atomicExch(a.err, 1);
            *abort = 1;
        }
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 0) {
        tc_fence_after();
        tmem_dealloc(tmem, C::TMEM_COLS);
    }
}

template <int R, int GPR, int SS, int A_STAGES>
gyps_status run_pass_cfg(Mesh *m, const TcArgs &a0, int64_t n_chunks, const double2 *X, int64_t ldx, int nrhs,
                         double2 *v, cudaStream_t s, unsigned char *panel)
{
    using C = Cfg<R>;
    constexpr int SMEM = A_STAGES * 2 * C::A_BYTES + SS * C::CHUNK_BYTES + 128;
    constexpr int NT = M * GPR + 32;
    GYPS_CUDA(cudaFuncSetAttribute(far_tc_kernel<R, GPR, SS, A_STAGES>, cudaFuncAttributeMaxDynamicSharedMemorySize, SMEM));
    int occ = 0;
    GYPS_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, far_tc_kernel<R, GPR, SS, A_STAGES>, NT, SMEM));
    occ = std::max(occ, 1);
    TcArgs a = a0;
    const int64_t items = a.n_tiles * a.n_segs;
    const int64_t grid = std::min<int64_t>((int64_t)m->num_sms * occ, items);
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
        far_tc_kernel<R, GPR, SS, A_STAGES><<<(unsigned)grid, NT, SMEM, s>>>(a);
        GYPS_CUDA(cudaGetLastError());
        tf.done(1);
    }
    return GYPS_OK;
}

template <int R>
gyps_status run(Mesh *m, double k, const double2 *X, int64_t ldx, int nrhs, double2 *v, int64_t ldv, cudaStream_t s)
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
    a.n_tiles = (m->nq + M - 1) / M;
    a.n_segs = (n_chunks + SEG_CHUNKS - 1) / SEG_CHUNKS;
    a.ncols = 0;
    a.ks = (float)k;
    a.err = m->d_err;
    // four generator threads per target row (16 generator warps per CTA), four tile stages, one CTA
    // per SM (two CTAs with two stages each measured no faster at 16 right-hand sides)
    return run_pass_cfg<R, 4, (R == 16 ? 4 : 3), 4>(m, a, n_chunks, X, ldx, nrhs, v, s, panel);
}

}  // namespace tc

gyps_status far_tc(Mesh *m, double k, const double2 *X, int64_t ldx, int nrhs, double2 *v, int64_t ldv,
                   cudaStream_t s)
{
    // widest pass that the right-hand sides fill: every pass regenerates the kernel tiles
    if (nrhs >= 64) {
        const int full = nrhs / 64 * 64;
        GYPS_TRY(tc::run<64>(m, k, X, ldx, full, v, ldv, s));
        if (full == nrhs) return GYPS_OK;
        return far_tc(m, k, X + (int64_t)full * ldx, ldx, nrhs - full, v + (int64_t)full * ldv, ldv, s);
    }
    if (nrhs > 16) return tc::run<32>(m, k, X, ldx, nrhs, v, ldv, s);
    return tc::run<16>(m, k, X, ldx, nrhs, v, ldv, s);
}

}  // namespace gyps
