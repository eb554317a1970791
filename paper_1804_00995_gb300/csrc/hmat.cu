// Compressed far field of the single layer (Sec. 5.3: the BEM matrix stored
// as blocks, far-apart groups of unknowns coupled through low-rank blocks
// approximated to a tolerance).  One level of a cluster tree (block low-rank):
//
//   clusters   runs of `leaf_tiles` consecutive vertex tiles (Morton order), so a
//              cluster is a compact patch of the surface;
//   blocks     for every pair of clusters (A, B), A <= B, the block V_far[A, B]:
//              dense (FP32 complex) when the clusters are close, else the
//              adaptive cross approximation U W^T with partial pivoting to the
//              relative tolerance eps; V_far is complex symmetric, so the block
//              (B, A) is the transpose (W U^T, or the stored transpose of a
//              dense block) and is not computed again;
//   build      the dense entries of a block come from the tile-pair kernel
//              (each entry once); far blocks are generated in batches into a
//              scratch buffer and compressed there, one CTA per block;
//   apply      X gathered into cluster order (FP32), the projections W^T x_B of
//              every low-rank block, then one pass per row chunk of a cluster
//              that sums its dense blocks and U T products in registers (no
//              atomics), written in FP64, plus the FP64 correction C X.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstring>
#include <string>
#include <vector>

#include "far_tile.cuh"
#include "internal.h"
#include "vtiles.h"

namespace gyps {

namespace hm {

constexpr int NRC = 16;  // right-hand sides per apply pass

struct Block {
    int32_t A, B;
    int32_t lowrank;  // 1: U W^T, 0: dense
    int32_t rank;
    int64_t m, n;
    float2 *D = nullptr, *DT = nullptr;  // dense: m x n and its transpose n x m (column-major)
    float2 *U = nullptr, *W = nullptr;   // low rank: m x r, n x r (column-major)
};

// A term of a cluster's row sum: a dense block (M: m x ncol, x from cluster
// positions src) or a low-rank product (M: m x r, multiplied by projection t).
struct Term {
    const float2 *M;
    int64_t ld;
    int32_t ncol;
    int32_t kind;   // 0 dense, 1 low rank
    int64_t src;    // dense: first position of the source cluster; low rank: offset of its projection
};

// One projection t = F^T x[src : src + len] (F: len x r, column-major), r x NRC values at toff.
struct Proj {
    const float2 *F;
    int64_t len;
    int32_t r;
    int32_t pad;
    int64_t src;
    int64_t toff;
};

}  // namespace hm

struct Hmat {
    Mesh *m = nullptr;
    double k = 0, eps = 0, eta = 0;
    int leaf_tiles = 0;
    int64_t nc = 0;
    std::vector<int64_t> ct0, voff;
    int32_t *d_perm = nullptr, *d_localmap = nullptr;
    std::vector<hm::Block> blocks;
    std::vector<void *> pools;
    // apply plan
    hm::Term *d_terms = nullptr;
    int32_t *d_term_ptr = nullptr;  // nc + 1
    hm::Proj *d_proj = nullptr;  // sorted by source range
    int2 *d_pgroups = nullptr;     // projections [x, y) sharing one source range (at most 32)
    int64_t n_pgroups = 0;
    int proj16_smem = 0;           // shared memory of hm_project16_kernel (0: not used)
    int64_t nproj = 0, tlen = 0;
    int32_t max_rank = 0;
    float2 *d_T = nullptr, *d_xloc = nullptr;
    int64_t row_chunks = 0;
    int64_t *d_chunk_cluster = nullptr;  // per row chunk: cluster << 32 | chunk index
    int4 *d_rows_items = nullptr;        // 16-column pass: (cluster, row chunk, terms [z, w)), largest first
    int64_t n_rows_items = 0;
    int64_t *voff_dev = nullptr;         // device copy of voff
    // statistics
    int64_t n_dense = 0, n_lowrank = 0, n_fallback = 0;
    double mean_rank = 0;
    int64_t bytes = 0;
    double build_ms = 0;
};

// ---------------------------------------------------------------- device: block reductions
__device__ __forceinline__ float warp_sum(float v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Sum over the CTA (blockDim.x a multiple of 32, at most 1024); every thread gets it.
__device__ float block_sum(float v, float *red)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    v = warp_sum(v);
    __syncthreads();
    if (lane == 0) red[warp] = v;
    __syncthreads();
    float t = lane < nw ? red[lane] : 0.0f;
    return warp_sum(t);
}

// Largest value over the CTA with its index (smallest index on ties); every thread gets both.
__device__ void block_argmax(float v, int idx, float *redv, int *redi, float *ov, int *oi)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const float v2 = __shfl_xor_sync(0xffffffffu, v, o);
        const int i2 = __shfl_xor_sync(0xffffffffu, idx, o);
        if (v2 > v || (v2 == v && i2 < idx)) {
            v = v2;
            idx = i2;
        }
    }
    __syncthreads();
    if (lane == 0) {
        redv[warp] = v;
        redi[warp] = idx;
    }
    __syncthreads();
    v = lane < nw ? redv[lane] : -1.0f;
    idx = lane < nw ? redi[lane] : -1;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const float v2 = __shfl_xor_sync(0xffffffffu, v, o);
        const int i2 = __shfl_xor_sync(0xffffffffu, idx, o);
        if (v2 > v || (v2 == v && i2 < idx)) {
            v = v2;
            idx = i2;
        }
    }
    *ov = v;
    *oi = idx;
}

__device__ __forceinline__ float2 cmul(float2 a, float2 b) { return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x); }
__device__ __forceinline__ float2 csub(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ float cabs2(float2 a) { return a.x * a.x + a.y * a.y; }

// ---------------------------------------------------------------- device: ACA
// One CTA per block S (m x n, column-major, ld m): A ~ U W^T by the adaptive
// cross approximation with partial pivoting.  Step r: the residual of pivot
// row i (row of S minus the previous terms) gives W[:, r] after division by
// its largest entry over the unused columns (column j); the residual of column
// j gives U[:, r]; the next pivot row is the largest entry of U[:, r] over the
// unused rows.  |U W^T|_F^2 is updated exactly (terms' inner products); the
// iteration stops when |u_r| |w_r| <= eps |U W^T|_F (status 1) or at rmax
// (status 0).  A converged result is then checked on 256 pseudo-random
// entries: a residual mean square above (4 eps)^2 times the mean square of the
// approximation marks the block as not compressible (status 0).
struct AcaArgs {
    const float2 *S;
    const int64_t *s_off;
    float2 *UW;
    const int64_t *uw_off;
    const int32_t *mm, *nn, *rmaxb;
    int32_t *rank, *status;
    float eps;
};

__global__ void __launch_bounds__(256) aca_kernel(const AcaArgs a)
{
    extern __shared__ __align__(16) unsigned char sm[];
    const int b = blockIdx.x, tid = threadIdx.x;
    const int m = a.mm[b], n = a.nn[b], rmax = a.rmaxb[b];
    const float2 *S = a.S + a.s_off[b];
    float2 *U = a.UW + a.uw_off[b];
    float2 *W = U + (int64_t)m * rmax;
    float2 *urow = reinterpret_cast<float2 *>(sm);  // rmax
    float2 *wrow = urow + rmax;                     // rmax
    float *red = reinterpret_cast<float *>(wrow + rmax);  // 32
    int *redi = reinterpret_cast<int *>(red + 32);         // 32
    float *crossv = reinterpret_cast<float *>(redi + 32);  // 8
    unsigned char *used_r = reinterpret_cast<unsigned char *>(crossv + 8);
    unsigned char *used_c = used_r + m;
    for (int i = tid; i < m; i += blockDim.x) used_r[i] = 0;
    for (int j = tid; j < n; j += blockDim.x) used_c[j] = 0;
    __syncthreads();

    double s2 = 0.0;
    int r = 0, piv = 0, status = 0;
    while (r < rmax) {
        for (int p = tid; p < r; p += blockDim.x) urow[p] = U[piv + (int64_t)p * m];
        __syncthreads();
        if (tid == 0) used_r[piv] = 1;
        // residual of row piv -> W[:, r]
        float best = -1.0f;
        int bj = -1;
        for (int j = tid; j < n; j += blockDim.x) {
            float2 v = S[piv + (int64_t)j * m];
            for (int p = 0; p < r; ++p) v = csub(v, cmul(urow[p], W[j + (int64_t)p * n]));
            W[j + (int64_t)r * n] = v;
            const float mag = cabs2(v);
            if (!used_c[j] && mag > best) {
                best = mag;
                bj = j;
            }
        }
        float gbest;
        int gj;
        block_argmax(best, bj, red, redi, &gbest, &gj);
        if (!(gbest > 0.0f)) {  // the row is (numerically) zero: take the next unused row
            int cand = m;
            for (int i = tid; i < m; i += blockDim.x)
                if (!used_r[i] && i != piv) cand = min(cand, i);
            float dummy;
            int next;
            block_argmax(-(float)cand, cand, red, redi, &dummy, &next);  // smallest candidate
            if (next >= m || next < 0) break;
            piv = next;
            __syncthreads();
            continue;
        }
        const float2 delta = W[gj + (int64_t)r * n];
        const float dd = 1.0f / cabs2(delta);
        const float2 inv = make_float2(delta.x * dd, -delta.y * dd);
        __syncthreads();
        float wn2 = 0.0f;
        for (int j = tid; j < n; j += blockDim.x) {
            const float2 w = cmul(W[j + (int64_t)r * n], inv);
            W[j + (int64_t)r * n] = w;
            wn2 += cabs2(w);
        }
        for (int p = tid; p < r; p += blockDim.x) wrow[p] = W[gj + (int64_t)p * n];
        if (tid == 0) used_c[gj] = 1;
        __syncthreads();
        // residual of column gj -> U[:, r]
        float un2 = 0.0f, bestr = -1.0f;
        int bi = -1;
        for (int i = tid; i < m; i += blockDim.x) {
            float2 v = S[i + (int64_t)gj * m];
            for (int p = 0; p < r; ++p) v = csub(v, cmul(wrow[p], U[i + (int64_t)p * m]));
            U[i + (int64_t)r * m] = v;
            const float mag = cabs2(v);
            un2 += mag;
            if (!used_r[i] && mag > bestr) {
                bestr = mag;
                bi = i;
            }
        }
        wn2 = block_sum(wn2, red);
        un2 = block_sum(un2, red);
        float gbr;
        int gi;
        block_argmax(bestr, bi, red, redi, &gbr, &gi);
        __syncthreads();  // U[:, r] and W[:, r] complete
        // cross terms: sum_p Re((u_p^H u_r)(w_p^H w_r)), one warp per p
        const int lane = tid & 31, warp = tid >> 5;
        float cross = 0.0f;
        for (int p = warp; p < r; p += blockDim.x >> 5) {
            float ar = 0.f, ai = 0.f, br = 0.f, bi2 = 0.f;
            for (int i = lane; i < m; i += 32) {
                const float2 up = U[i + (int64_t)p * m], ur = U[i + (int64_t)r * m];
                ar += up.x * ur.x + up.y * ur.y;  // conj(up) ur
                ai += up.x * ur.y - up.y * ur.x;
            }
            for (int j = lane; j < n; j += 32) {
                const float2 wp = W[j + (int64_t)p * n], wr = W[j + (int64_t)r * n];
                br += wp.x * wr.x + wp.y * wr.y;
                bi2 += wp.x * wr.y - wp.y * wr.x;
            }
            ar = warp_sum(ar);
            ai = warp_sum(ai);
            br = warp_sum(br);
            bi2 = warp_sum(bi2);
            cross += ar * br - ai * bi2;
        }
        if (lane == 0) crossv[warp] = cross;
        __syncthreads();
        float csum = 0.0f;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) csum += crossv[w];
        s2 += (double)un2 * (double)wn2 + 2.0 * (double)csum;
        ++r;
        if ((double)un2 * (double)wn2 <= (double)a.eps * a.eps * fmax(s2, 0.0)) {
            status = 1;
            break;
        }
        if (gi < 0) break;  // every row used
        piv = gi;
        __syncthreads();
    }
    __syncthreads();
    if (status == 1 && r > 0) {
        // spot check on 256 pseudo-random entries (a fixed counter-based hash of the block and thread)
        float e2 = 0.0f, a2 = 0.0f;
        for (int t = tid; t < 256; t += blockDim.x) {
            uint32_t h = (uint32_t)b * 2654435761u ^ (uint32_t)(t + 1) * 2246822519u;
            h ^= h >> 15;
            h *= 2654435761u;
            h ^= h >> 13;
            const int i = (int)(h % (uint32_t)m), j = (int)((h / (uint32_t)m) % (uint32_t)n);
            float2 approx = make_float2(0.f, 0.f);
            for (int p = 0; p < r; ++p) {
                const float2 uw = cmul(U[i + (int64_t)p * m], W[j + (int64_t)p * n]);
                approx.x += uw.x;
                approx.y += uw.y;
            }
            e2 += cabs2(csub(S[i + (int64_t)j * m], approx));
            a2 += cabs2(approx);
        }
        e2 = block_sum(e2, red);
        a2 = block_sum(a2, red);
        if (e2 > 16.0f * a.eps * a.eps * a2) status = 0;
    }
    if (tid == 0) {
        a.rank[b] = r;
        a.status[b] = status;
    }
}

// ---------------------------------------------------------------- device: transposes, gathers
// DT = D^T for many blocks (D: m x n, DT: n x m, column-major); 32 x 32 tiles.
struct TransArgs {
    const float2 *const *src;
    float2 *const *dst;
    const int32_t *mm, *nn;
    const int32_t *tile0;  // first tile of each block in the flat grid (nblocks + 1)
    int nblocks;
};

__global__ void transpose_blocks_kernel(const TransArgs a)
{
    __shared__ float2 t[32][33];
    const int g = blockIdx.x;
    int lo = 0, hi = a.nblocks;  // block of this tile: tile0[b] <= g < tile0[b + 1]
    while (hi - lo > 1) {
        const int mid = (lo + hi) / 2;
        if (a.tile0[mid] <= g) lo = mid;
        else hi = mid;
    }
    const int b = lo, m = a.mm[b], n = a.nn[b];
    const int tm = (m + 31) / 32, loc = g - a.tile0[b];
    const int i0 = (loc % tm) * 32, j0 = (loc / tm) * 32;
    const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;  // 256 threads: 32 x 8
    for (int j = ty; j < 32; j += 8)
        if (i0 + tx < m && j0 + j < n) t[j][tx] = a.src[b][(i0 + tx) + (int64_t)(j0 + j) * m];
    __syncthreads();
    for (int i = ty; i < 32; i += 8)
        if (j0 + tx < n && i0 + i < m) a.dst[b][(j0 + tx) + (int64_t)(i0 + i) * n] = t[tx][i];
}

// x_loc[p + c nv] = X[perm[p] + (c0 + c) ldx] in FP32, c < w
__global__ void hm_gather_kernel(const int32_t *perm, int64_t nv, const double2 *X, int64_t ldx, int c0, int w,
                                 float2 *xloc)
{
    const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int c = blockIdx.y;
    if (p >= nv || c >= w) return;
    const double2 x = X[perm[p] + (int64_t)(c0 + c) * ldx];
    xloc[p + (int64_t)c * nv] = make_float2((float)x.x, (float)x.y);
}

// t[p][c] = sum_j F[j, p] x[src + j, c], for the 16 columns p0 .. p0+15 of one projection.
template <int NR>
__global__ void __launch_bounds__(256) hm_project_kernel(const hm::Proj *proj, const float2 *xloc, int64_t nv,
                                                         float2 *T)
{
    __shared__ float2 Fs[16][65];
    __shared__ float2 Xs[64][NR];
    const hm::Proj pr = proj[blockIdx.x];
    const int p0 = blockIdx.y * 16;
    if (p0 >= pr.r) return;
    const int tid = threadIdx.x, pi = tid / 16, ci = tid % 16;
    float2 acc = make_float2(0.f, 0.f);
    for (int64_t j0 = 0; j0 < pr.len; j0 += 64) {
        for (int e = tid; e < 16 * 64; e += 256) {
            const int pp = e / 64, jj = e % 64;
            Fs[pp][jj] = (p0 + pp < pr.r && j0 + jj < pr.len) ? pr.F[(j0 + jj) + (int64_t)(p0 + pp) * pr.len]
                                                              : make_float2(0.f, 0.f);
        }
        for (int e = tid; e < 64 * NR; e += 256) {
            const int jj = e % 64, c = e / 64;
            Xs[jj][c] = j0 + jj < pr.len ? xloc[pr.src + j0 + jj + (int64_t)c * nv] : make_float2(0.f, 0.f);
        }
        __syncthreads();
        if (ci < NR) {
#pragma unroll 8
            for (int jj = 0; jj < 64; ++jj) {
                const float2 f = Fs[pi][jj], x = Xs[jj][ci];
                acc.x = fmaf(f.x, x.x, fmaf(-f.y, x.y, acc.x));
                acc.y = fmaf(f.x, x.y, fmaf(f.y, x.x, acc.y));
            }
        }
        __syncthreads();
    }
    if (ci < NR && p0 + pi < pr.r) T[pr.toff + (int64_t)(p0 + pi) * hm::NRC + ci] = acc;
}

// Butterfly reduce-scatter over a warp: on return, lane l holds the sum over
// all 32 lanes of value l (at each step a lane keeps one half of its values and
// adds the partner's copy of that half).
__device__ __forceinline__ float reduce_scatter32(float (&v)[32], int lane)
{
#pragma unroll
    for (int st = 0; st < 5; ++st) {
        const int o = 16 >> st, h = 16 >> st;
        const bool up = (lane & o) != 0;
#pragma unroll
        for (int i = 0; i < h; ++i) {
            const float send = up ? v[i] : v[i + h];
            const float keep = up ? v[i + h] : v[i];
            v[i] = keep + __shfl_xor_sync(0xffffffffu, send, o);
        }
    }
    return v[0];
}

// The projections of the 16-column pass, grouped by source cluster: a CTA takes
// projections [g.x, g.y) that share one source range x[src : src + len], stages
// those 16 columns of x in shared memory once (xs[cp][j] = (x[j][2 cp],
// x[j][2 cp + 1])), and each warp takes whole projections, two of their
// columns at a time: lanes stride over j reading F coalesced, 16 complex sums
// per column, then a reduce-scatter leaves value l = 2 c + (re, im) of the
// column on lane l, stored as one 128-byte row of T.
__global__ void __launch_bounds__(256) hm_project16_kernel(const hm::Proj *proj, const int2 *groups,
                                                           const float2 *xloc, int64_t nv, float2 *T)
{
    extern __shared__ float4 xs[];
    const int2 gr = groups[blockIdx.x];
    const int64_t src = proj[gr.x].src, len = proj[gr.x].len;
    for (int64_t e = threadIdx.x; e < 8 * len; e += blockDim.x) {
        const int cp = (int)(e / len);
        const int64_t j = e - (int64_t)cp * len;
        const float2 a = xloc[src + j + (int64_t)(2 * cp) * nv], b = xloc[src + j + (int64_t)(2 * cp + 1) * nv];
        xs[e] = make_float4(a.x, a.y, b.x, b.y);
    }
    __syncthreads();
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nwarps = blockDim.x >> 5;
    float *Tf = reinterpret_cast<float *>(T);
    for (int pi = gr.x + warp; pi < gr.y; pi += nwarps) {
        const hm::Proj pr = proj[pi];
        for (int p = 0; p < pr.r; p += 2) {
            const bool two = p + 1 < pr.r;
            const float2 *F0 = pr.F + (int64_t)p * len, *F1 = two ? F0 + len : F0;
            float v0[32], v1[32];
#pragma unroll
            for (int i = 0; i < 32; ++i) v0[i] = v1[i] = 0.f;
#pragma unroll 2
            for (int64_t j = lane; j < len; j += 32) {
                const float2 f0 = F0[j], f1 = F1[j];
#pragma unroll
                for (int cp = 0; cp < 8; ++cp) {
                    const float4 x = xs[(int64_t)cp * len + j];
                    v0[4 * cp + 0] = fmaf(f0.x, x.x, fmaf(-f0.y, x.y, v0[4 * cp + 0]));
                    v0[4 * cp + 1] = fmaf(f0.x, x.y, fmaf(f0.y, x.x, v0[4 * cp + 1]));
                    v0[4 * cp + 2] = fmaf(f0.x, x.z, fmaf(-f0.y, x.w, v0[4 * cp + 2]));
                    v0[4 * cp + 3] = fmaf(f0.x, x.w, fmaf(f0.y, x.z, v0[4 * cp + 3]));
                    v1[4 * cp + 0] = fmaf(f1.x, x.x, fmaf(-f1.y, x.y, v1[4 * cp + 0]));
                    v1[4 * cp + 1] = fmaf(f1.x, x.y, fmaf(f1.y, x.x, v1[4 * cp + 1]));
                    v1[4 * cp + 2] = fmaf(f1.x, x.z, fmaf(-f1.y, x.w, v1[4 * cp + 2]));
                    v1[4 * cp + 3] = fmaf(f1.x, x.w, fmaf(f1.y, x.z, v1[4 * cp + 3]));
                }
            }
            const float s0 = reduce_scatter32(v0, lane);
            const float s1 = reduce_scatter32(v1, lane);
            Tf[2 * (pr.toff + (int64_t)p * hm::NRC) + lane] = s0;
            if (two) Tf[2 * (pr.toff + (int64_t)(p + 1) * hm::NRC) + lane] = s1;
        }
    }
}

// y[rows of cluster A, chunk of 128] = sum over the cluster's terms, written to Y (FP64).
template <int NR>
__global__ void __launch_bounds__(128) hm_rows_kernel(const hm::Term *terms, const int32_t *term_ptr,
                                                      const int64_t *voff, const int64_t *chunk_cluster,
                                                      const int32_t *perm, const float2 *xloc, int64_t nv,
                                                      const float2 *T, double2 *Y, int64_t ldy, int c0)
{
    __shared__ float2 Xs[64][NR];
    const int64_t cc = chunk_cluster[blockIdx.x];
    const int A = (int)(cc >> 32), chunk = (int)(cc & 0xffffffff);
    const int64_t mA = voff[A + 1] - voff[A];
    const int64_t i = (int64_t)chunk * 128 + threadIdx.x;
    const bool row = i < mA;
    float2 hi[NR], lo[NR];  // error-free (TwoSum) running sum of the chunk sums
#pragma unroll
    for (int c = 0; c < NR; ++c) hi[c] = lo[c] = make_float2(0.f, 0.f);
    for (int tt = term_ptr[A]; tt < term_ptr[A + 1]; ++tt) {
        const hm::Term t = terms[tt];
        for (int j0 = 0; j0 < t.ncol; j0 += 64) {
            const int nj = min(64, t.ncol - j0);
            __syncthreads();
            for (int e = threadIdx.x; e < 64 * NR; e += 128) {
                const int jj = e % 64, c = e / 64;
                float2 v = make_float2(0.f, 0.f);
                if (jj < nj)
                    v = t.kind == 0 ? xloc[t.src + j0 + jj + (int64_t)c * nv] : T[t.src + (int64_t)(j0 + jj) * hm::NRC + c];
                Xs[jj][c] = v;
            }
            __syncthreads();
            if (row) {
                float2 acc[NR];
#pragma unroll
                for (int c = 0; c < NR; ++c) acc[c] = make_float2(0.f, 0.f);
                const float2 *Mc = t.M + i + (int64_t)j0 * t.ld;
#pragma unroll 4
                for (int jj = 0; jj < nj; ++jj) {
                    const float2 d = Mc[(int64_t)jj * t.ld];
#pragma unroll
                    for (int c = 0; c < NR; ++c) {
                        const float2 x = Xs[jj][c];
                        acc[c].x = fmaf(d.x, x.x, fmaf(-d.y, x.y, acc[c].x));
                        acc[c].y = fmaf(d.x, x.y, fmaf(d.y, x.x, acc[c].y));
                    }
                }
#pragma unroll
                for (int c = 0; c < NR; ++c) {
                    two_sum_acc(hi[c].x, lo[c].x, acc[c].x);
                    two_sum_acc(hi[c].y, lo[c].y, acc[c].y);
                }
            }
        }
    }
    if (row) {
        const int64_t v = perm[voff[A] + i];
#pragma unroll
        for (int c = 0; c < NR; ++c)
            Y[v + (int64_t)(c0 + c) * ldy] =
                make_double2((double)hi[c].x + (double)lo[c].x, (double)hi[c].y + (double)lo[c].y);
    }
}

// 8-byte asynchronous copy global -> shared (one complex FP32 value; any 8-byte
// aligned address); src_bytes = 0 fills zeros.
__device__ __forceinline__ void cp_async8(void *dst, const void *src, int src_bytes)
{
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8, %2;" ::"r"(smem_addr(dst)), "l"(src), "r"(src_bytes)
                 : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait1() { asm volatile("cp.async.wait_group 1;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait0() { asm volatile("cp.async.wait_group 0;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait_n()
{
    asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}

// The row sums of hm_rows_kernel for 16 right-hand sides, tiled: a CTA takes one
// work item, 128 rows of a cluster and a range of its terms; the columns of those
// terms (dense blocks, and U with its projection) stream through shared memory as one sequence of units of up to
// RT_K columns, RT_S stages deep across term boundaries (asynchronous copies,
// zero-filled past a block's edge), so that no term restarts the pipeline.
// Each thread owns 4 rows (32 apart) x 4 right-hand sides (16 complex sums)
// and reads per column 4 complex values of the matrix and 4 of x; FP32 sums of
// RT_FOLD units at a time are folded into TwoSum pairs.
#ifndef GYPS_RT_K
#define GYPS_RT_K 32
#endif
#ifndef GYPS_RT_S
#define GYPS_RT_S 2
#endif
#ifndef GYPS_RT_FOLD
#define GYPS_RT_FOLD 4
#endif
constexpr int RT_ROWS = 128, RT_K = GYPS_RT_K, RT_S = GYPS_RT_S, RT_FOLD = GYPS_RT_FOLD;  // RT_FOLD: a power of 2
struct RowsTileSmem {
    float2 M[RT_S][RT_K][RT_ROWS];
    float2 X[RT_S][RT_K][hm::NRC];
};

// Work item of a CTA: one row chunk of a cluster and a contiguous range of its
// terms, cut so that items carry similar numbers of units and launched largest
// first; the items of a row chunk add into Y (zeroed before the pass).
// Position in a CTA's sequence of units: term tt, first column j0.
struct UnitCursor {
    int tt, j0;
};

__global__ void __launch_bounds__(128) hm_rows16_kernel(const hm::Term *terms, const int4 *items,
                                                        const int64_t *voff, const int32_t *perm,
                                                        const float2 *xloc, int64_t nv, const float2 *T, double2 *Y,
                                                        int64_t ldy, int c0)
{
    extern __shared__ __align__(16) unsigned char smraw[];
    RowsTileSmem &sm = *reinterpret_cast<RowsTileSmem *>(smraw);
    const int4 item = items[blockIdx.x];
    const int A = item.x;
    const int64_t mA = voff[A + 1] - voff[A];
    const int64_t row0 = (int64_t)item.y * RT_ROWS;
    // rows rg, rg + 32, rg + 64, rg + 96 (consecutive lanes read consecutive rows: no bank
    // conflicts), RHS 4 cg .. 4 cg + 3 (one per warp: broadcast reads)
    const int tid = threadIdx.x, rg = tid & 31, cg = tid >> 5;
    const int tt_end = item.w;
    float2 hi[4][4], lo[4][4];
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b) hi[a][b] = lo[a][b] = make_float2(0.f, 0.f);

    // copies of the unit at cursor u into stage st (an empty commit group past the end)
    auto issue = [&](UnitCursor &u, int st) {
        if (u.tt < tt_end) {
            const hm::Term t = terms[u.tt];
#pragma unroll 8
            for (int k = 0; k < RT_K * RT_ROWS / 128; ++k) {  // rows fastest
                const int e = tid + 128 * k, jj = e / RT_ROWS, rr = e % RT_ROWS;
                const int64_t row = row0 + rr, col = u.j0 + jj;
                const bool ok = col < t.ncol && row < mA;
                cp_async8(&sm.M[st][jj][rr], t.M + (ok ? row + col * t.ld : 0), ok ? 8 : 0);
            }
            for (int e = tid; e < RT_K * hm::NRC; e += 128) {
                const int jj = e / hm::NRC, c = e % hm::NRC;
                const int64_t col = u.j0 + jj;
                const bool ok = col < t.ncol;
                const float2 *src = t.kind == 0 ? xloc + (ok ? t.src + col + (int64_t)c * nv : 0)
                                                : T + (ok ? t.src + col * hm::NRC + c : 0);
                cp_async8(&sm.X[st][jj][c], src, ok ? 8 : 0);
            }
            u.j0 += RT_K;
            if (u.j0 >= t.ncol) {
                ++u.tt;
                u.j0 = 0;
            }
        }
        cp_async_commit();
    };

    float2 acc[4][4];  // FP32 sums of up to RT_FOLD units
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b) acc[a][b] = make_float2(0.f, 0.f);
    UnitCursor ui{item.z, 0}, uc{item.z, 0};
#pragma unroll
    for (int st = 0; st + 1 < RT_S; ++st) issue(ui, st);
    for (int q = 0; uc.tt < tt_end; ++q) {
        issue(ui, (q + RT_S - 1) % RT_S);  // its stage held unit q - 1, consumed before the last barrier
        cp_async_wait_n<RT_S - 1>();        // unit q landed
        __syncthreads();
        const int st = q % RT_S;
        const int ncol = terms[uc.tt].ncol;
        const int nj = min(RT_K, ncol - uc.j0);
        const int njr = (nj + 3) & ~3;  // zero-filled past the edge
#pragma unroll 4
        for (int jj = 0; jj < njr; ++jj) {
            const float4 x01 = *reinterpret_cast<const float4 *>(&sm.X[st][jj][4 * cg]);
            const float4 x23 = *reinterpret_cast<const float4 *>(&sm.X[st][jj][4 * cg + 2]);
            const float2 mv[4] = {sm.M[st][jj][rg], sm.M[st][jj][rg + 32], sm.M[st][jj][rg + 64],
                                  sm.M[st][jj][rg + 96]};
            const float2 xv[4] = {make_float2(x01.x, x01.y), make_float2(x01.z, x01.w), make_float2(x23.x, x23.y),
                                  make_float2(x23.z, x23.w)};
#pragma unroll
            for (int a = 0; a < 4; ++a)
#pragma unroll
                for (int b = 0; b < 4; ++b) {
                    acc[a][b].x = fmaf(mv[a].x, xv[b].x, fmaf(-mv[a].y, xv[b].y, acc[a][b].x));
                    acc[a][b].y = fmaf(mv[a].x, xv[b].y, fmaf(mv[a].y, xv[b].x, acc[a][b].y));
                }
        }
        uc.j0 += RT_K;
        if (uc.j0 >= ncol) {
            ++uc.tt;
            uc.j0 = 0;
        }
        if ((q & (RT_FOLD - 1)) == RT_FOLD - 1 || uc.tt >= tt_end) {  // fold every RT_FOLD units and at the end
#pragma unroll
            for (int a = 0; a < 4; ++a)
#pragma unroll
                for (int b = 0; b < 4; ++b) {
                    two_sum_acc(hi[a][b].x, lo[a][b].x, acc[a][b].x);
                    two_sum_acc(hi[a][b].y, lo[a][b].y, acc[a][b].y);
                    acc[a][b] = make_float2(0.f, 0.f);
                }
        }
        __syncthreads();  // stage st is free for unit q + RT_S
    }
    cp_async_wait_n<0>();  // empty groups only, by now
#pragma unroll
    for (int a = 0; a < 4; ++a) {
        const int64_t i = row0 + rg + 32 * a;
        if (i >= mA) continue;
        const int64_t v = perm[voff[A] + i];
#pragma unroll
        for (int b = 0; b < 4; ++b) {
            double *y = reinterpret_cast<double *>(Y + v + (int64_t)(c0 + 4 * cg + b) * ldy);
            atomicAdd(y, (double)hi[a][b].x + (double)lo[a][b].x);  // a row chunk's terms span several CTAs
            atomicAdd(y + 1, (double)hi[a][b].y + (double)lo[a][b].y);
        }
    }
}

// ---------------------------------------------------------------- host: build
static gyps_status dmalloc(Hmat *h, void **p, size_t bytes)
{
    if (bytes == 0) bytes = 16;
    cudaError_t e = cudaMalloc(p, bytes);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return set_error(GYPS_ERR_OOM, "compressed far field: cudaMalloc of " + std::to_string(bytes) + " bytes");
    }
    h->pools.push_back(*p);
    h->bytes += (int64_t)bytes;
    return GYPS_OK;
}

template <class T>
static gyps_status upload(Hmat *h, T **dst, const std::vector<T> &v, cudaStream_t s)
{
    GYPS_TRY(dmalloc(h, (void **)dst, v.size() * sizeof(T)));
    if (!v.empty()) GYPS_CUDA(cudaMemcpyAsync(*dst, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice, s));
    return GYPS_OK;
}

void free_hmat(Hmat *h)
{
    if (!h) return;
    if (h->m) cudaSetDevice(h->m->device);
    cudaDeviceSynchronize();
    for (void *p : h->pools) cudaFree(p);
    delete h;
}

static bool tiles_adjacent(const VertexTiles *T, int32_t I, int32_t J)
{
    const uint64_t key = ((uint64_t)std::min(I, J) << 32) | (uint64_t)std::max(I, J);
    return std::binary_search(T->adjacent.begin(), T->adjacent.end(), key);
}

// Tile items of block (A, B) into the lists; block entries at element offset off, ld = m_A.
static void block_items(const Hmat *h, const VertexTiles *T, int A, int B, int64_t off, std::vector<int4> &items,
                        std::vector<int64_t> &offs)
{
    const int32_t mA = (int32_t)(h->voff[A + 1] - h->voff[A]);
    for (int64_t I = h->ct0[A]; I < h->ct0[A + 1]; ++I)
        for (int64_t J = (A == B ? I : h->ct0[B]); J < h->ct0[B + 1]; ++J) {
            int flags = tiles_adjacent(T, (int32_t)I, (int32_t)J) ? 1 : 0;
            if (A == B) flags |= 2;  // the diagonal block: both triangles of tile pairs
            items.push_back(make_int4((int)I, (int)J, flags, mA));
            offs.push_back(off);
        }
}

static gyps_status run_items(Hmat *h, const TileArgs &base, const std::vector<int4> &items,
                             const std::vector<int64_t> &offs, float2 *out, cudaStream_t s)
{
    if (items.empty()) return GYPS_OK;
    int4 *d_items = nullptr;
    int64_t *d_offs = nullptr;
    GYPS_CUDA(cudaMallocAsync((void **)&d_items, items.size() * sizeof(int4), s));
    GYPS_CUDA(cudaMallocAsync((void **)&d_offs, offs.size() * sizeof(int64_t), s));
    GYPS_CUDA(cudaMemcpyAsync(d_items, items.data(), items.size() * sizeof(int4), cudaMemcpyHostToDevice, s));
    GYPS_CUDA(cudaMemcpyAsync(d_offs, offs.data(), offs.size() * sizeof(int64_t), cudaMemcpyHostToDevice, s));
    TileArgs a = base;
    a.items = d_items;
    a.item_off = d_offs;
    a.n_items = (int64_t)items.size();
    a.ld = 0;  // per item: the block's leading dimension
    gyps_status st = tile_blocks<float2>(h->m, h->k, a, out, s);
    cudaFreeAsync(d_items, s);
    cudaFreeAsync(d_offs, s);
    return st;
}

static gyps_status transpose_blocks(Hmat *h, const std::vector<hm::Block *> &bl, cudaStream_t s)
{
    if (bl.empty()) return GYPS_OK;
    std::vector<const float2 *> src;
    std::vector<float2 *> dst;
    std::vector<int32_t> mm, nn, tile0(1, 0);
    for (auto *b : bl) {
        src.push_back(b->D);
        dst.push_back(b->DT);
        mm.push_back((int32_t)b->m);
        nn.push_back((int32_t)b->n);
        tile0.push_back(tile0.back() + (int32_t)(((b->m + 31) / 32) * ((b->n + 31) / 32)));
    }
    const size_t bytes = bl.size() * (2 * sizeof(void *) + 2 * sizeof(int32_t)) + tile0.size() * sizeof(int32_t);
    unsigned char *buf = nullptr;
    GYPS_CUDA(cudaMallocAsync((void **)&buf, bytes, s));
    const size_t nb = bl.size();
    unsigned char *p = buf;
    auto put = [&](const void *host, size_t n) {
        cudaMemcpyAsync(p, host, n, cudaMemcpyHostToDevice, s);
        unsigned char *q = p;
        p += n;
        return q;
    };
    TransArgs a;
    a.src = reinterpret_cast<const float2 *const *>(put(src.data(), nb * sizeof(void *)));
    a.dst = reinterpret_cast<float2 *const *>(put(dst.data(), nb * sizeof(void *)));
    a.mm = reinterpret_cast<const int32_t *>(put(mm.data(), nb * sizeof(int32_t)));
    a.nn = reinterpret_cast<const int32_t *>(put(nn.data(), nb * sizeof(int32_t)));
    a.tile0 = reinterpret_cast<const int32_t *>(put(tile0.data(), tile0.size() * sizeof(int32_t)));
    a.nblocks = (int)nb;
    transpose_blocks_kernel<<<(unsigned)tile0.back(), 256, 0, s>>>(a);
    cudaError_t e = cudaGetLastError();
    cudaStreamSynchronize(s);  // host vectors above must outlive the copies
    cudaFreeAsync(buf, s);
    GYPS_CUDA(e);
    return GYPS_OK;
}

static gyps_status build(Hmat *h, cudaStream_t s)
{
    Mesh *m = h->m;
    GYPS_TRY(vertex_tiles_prepare(m, s));
    const VertexTiles *T = m->vt;
    // clusters: runs of leaf_tiles tiles; cluster order of the vertices
    h->nc = (T->ntiles + h->leaf_tiles - 1) / h->leaf_tiles;
    h->ct0.resize(h->nc + 1);
    for (int64_t c = 0; c <= h->nc; ++c) h->ct0[c] = std::min<int64_t>(c * h->leaf_tiles, T->ntiles);
    std::vector<int32_t> perm, localmap(T->ntiles * kTileV, -1);
    h->voff.assign(1, 0);
    for (int64_t c = 0; c < h->nc; ++c) {
        for (int64_t I = h->ct0[c]; I < h->ct0[c + 1]; ++I)
            for (int sl = 0; sl < kTileV; ++sl) {
                const int32_t v = T->rowmap[I * kTileV + sl];
                if (v < 0) continue;
                localmap[I * kTileV + sl] = (int32_t)((int64_t)perm.size() - h->voff.back());
                perm.push_back(v);
            }
        h->voff.push_back((int64_t)perm.size());
    }
    // bounding boxes of the clusters' supports (the vertices of every triangle of T(I))
    std::vector<double> vtx(3 * m->nv);
    std::vector<int32_t> tri(3 * m->nt);
    GYPS_CUDA(cudaMemcpyAsync(vtx.data(), m->d_vtx, vtx.size() * sizeof(double), cudaMemcpyDeviceToHost, s));
    GYPS_CUDA(cudaMemcpyAsync(tri.data(), m->d_tri, tri.size() * sizeof(int32_t), cudaMemcpyDeviceToHost, s));
    GYPS_CUDA(cudaStreamSynchronize(s));
    std::vector<double> lo(3 * h->nc, 1e300), hi(3 * h->nc, -1e300);
    for (int64_t c = 0; c < h->nc; ++c)
        for (int64_t I = h->ct0[c]; I < h->ct0[c + 1]; ++I)
            for (int64_t e = T->tile_ptr[I]; e < T->tile_ptr[I + 1]; ++e)
                for (int q = 0; q < 3; ++q) {
                    const double *p = &vtx[3 * (int64_t)tri[3 * (int64_t)T->tri[e] + q]];
                    for (int d = 0; d < 3; ++d) {
                        lo[3 * c + d] = std::min(lo[3 * c + d], p[d]);
                        hi[3 * c + d] = std::max(hi[3 * c + d], p[d]);
                    }
                }
    auto admissible = [&](int A, int B) {
        double gap2 = 0.0, dA = 0.0, dB = 0.0;
        for (int d = 0; d < 3; ++d) {
            const double g = std::max(0.0, std::max(lo[3 * A + d] - hi[3 * B + d], lo[3 * B + d] - hi[3 * A + d]));
            gap2 += g * g;
            dA += (hi[3 * A + d] - lo[3 * A + d]) * (hi[3 * A + d] - lo[3 * A + d]);
            dB += (hi[3 * B + d] - lo[3 * B + d]) * (hi[3 * B + d] - lo[3 * B + d]);
        }
        return std::sqrt(gap2) >= h->eta * std::sqrt(std::max(dA, dB));
    };
    GYPS_TRY(upload(h, &h->d_perm, perm, s));
    GYPS_TRY(upload(h, &h->d_localmap, localmap, s));
    GYPS_TRY(tile_panel(m, h->k, s));
    TileArgs base = tile_args(m, h->k);
    base.rowmap = h->d_localmap;
    base.colmap = h->d_localmap;

    // blocks
    std::vector<std::pair<int, int>> near, far;
    for (int A = 0; A < (int)h->nc; ++A)
        for (int B = A; B < (int)h->nc; ++B) (A != B && admissible(A, B) ? far : near).push_back({A, B});
    auto msize = [&](int A) { return h->voff[A + 1] - h->voff[A]; };
    // dense blocks: one pool for every D and DT
    {
        int64_t total = 0;
        for (auto &pr : near) total += msize(pr.first) * msize(pr.second) * (pr.first == pr.second ? 1 : 2);
        float2 *pool = nullptr;
        GYPS_TRY(dmalloc(h, (void **)&pool, (size_t)total * sizeof(float2)));
        std::vector<int4> items;
        std::vector<int64_t> offs;
        std::vector<hm::Block *> need_t;
        int64_t off = 0;
        h->blocks.reserve(near.size() + far.size());
        for (auto &pr : near) {
            hm::Block b;
            b.A = pr.first;
            b.B = pr.second;
            b.lowrank = 0;
            b.rank = 0;
            b.m = msize(b.A);
            b.n = msize(b.B);
            b.D = pool + off;
            block_items(h, T, b.A, b.B, off, items, offs);
            off += b.m * b.n;
            if (b.A != b.B) {
                b.DT = pool + off;
                off += b.m * b.n;
            }
            h->blocks.push_back(b);
        }
        GYPS_TRY(run_items(h, base, items, offs, pool, s));
        for (auto &b : h->blocks)
            if (b.DT) need_t.push_back(&b);
        GYPS_TRY(transpose_blocks(h, need_t, s));
        h->n_dense = (int64_t)near.size();
    }
    // low-rank blocks, in batches that fit the scratch budget
    const int64_t scratch_elems = (int64_t)1 << 28;  // 2 GiB of FP32 complex for the dense blocks of a batch
    float2 *S = nullptr, *UW = nullptr;
    int64_t max_blk = 0, max_uw = 0;
    for (auto &pr : far) {
        const int64_t a = msize(pr.first), b = msize(pr.second);
        max_blk = std::max(max_blk, a * b);
        max_uw = std::max(max_uw, std::max<int64_t>(1, std::min(a, b) / 2) * (a + b));
    }
    if (!far.empty()) {
        GYPS_CUDA(cudaMallocAsync((void **)&S, (size_t)std::max(scratch_elems, max_blk) * sizeof(float2), s));
        const int64_t per = std::max<int64_t>(1, std::max(scratch_elems, max_blk) / max_blk);
        GYPS_CUDA(cudaMallocAsync((void **)&UW, (size_t)(per * max_uw + 16) * sizeof(float2), s));
    }
    gyps_status st = GYPS_OK;
    double rank_sum = 0.0;
    int64_t rank_n = 0;
    for (size_t f0 = 0; f0 < far.size() && st == GYPS_OK;) {
        std::vector<int4> items;
        std::vector<int64_t> offs, s_off, uw_off;
        std::vector<int32_t> mm, nn, rmaxb;
        int64_t so = 0, uo = 0;
        size_t f1 = f0;
        for (; f1 < far.size(); ++f1) {
            const int A = far[f1].first, B = far[f1].second;
            const int64_t a = msize(A), b = msize(B);
            const int64_t rm = std::max<int64_t>(1, std::min(a, b) / 2);
            if (f1 > f0 && (so + a * b > std::max(scratch_elems, max_blk) || uo + rm * (a + b) > (std::max(scratch_elems, max_blk) / max_blk) * max_uw))
                break;
            block_items(h, T, A, B, so, items, offs);
            s_off.push_back(so);
            uw_off.push_back(uo);
            mm.push_back((int32_t)a);
            nn.push_back((int32_t)b);
            rmaxb.push_back((int32_t)rm);
            so += a * b;
            uo += rm * (a + b);
        }
        st = run_items(h, base, items, offs, S, s);
        if (st != GYPS_OK) break;
        const int nb = (int)(f1 - f0);
        std::vector<int64_t> meta64;
        meta64.insert(meta64.end(), s_off.begin(), s_off.end());
        meta64.insert(meta64.end(), uw_off.begin(), uw_off.end());
        std::vector<int32_t> meta32;
        meta32.insert(meta32.end(), mm.begin(), mm.end());
        meta32.insert(meta32.end(), nn.begin(), nn.end());
        meta32.insert(meta32.end(), rmaxb.begin(), rmaxb.end());
        int64_t *d64 = nullptr;
        int32_t *d32 = nullptr;
        GYPS_CUDA(cudaMallocAsync((void **)&d64, meta64.size() * sizeof(int64_t), s));
        GYPS_CUDA(cudaMallocAsync((void **)&d32, (meta32.size() + 2 * nb) * sizeof(int32_t), s));
        GYPS_CUDA(cudaMemcpyAsync(d64, meta64.data(), meta64.size() * sizeof(int64_t), cudaMemcpyHostToDevice, s));
        GYPS_CUDA(cudaMemcpyAsync(d32, meta32.data(), meta32.size() * sizeof(int32_t), cudaMemcpyHostToDevice, s));
        AcaArgs aa;
        aa.S = S;
        aa.s_off = d64;
        aa.UW = UW;
        aa.uw_off = d64 + nb;
        aa.mm = d32;
        aa.nn = d32 + nb;
        aa.rmaxb = d32 + 2 * nb;
        aa.rank = d32 + 3 * nb;
        aa.status = d32 + 4 * nb;
        aa.eps = (float)h->eps;
        int rmax_all = 0, mn_all = 0;
        for (int i = 0; i < nb; ++i) {
            rmax_all = std::max(rmax_all, rmaxb[i]);
            mn_all = std::max(mn_all, mm[i] + nn[i]);
        }
        const size_t smem = (size_t)rmax_all * 2 * sizeof(float2) + 72 * 4 + (size_t)mn_all + 16;
        GYPS_CUDA(cudaFuncSetAttribute(aca_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        aca_kernel<<<nb, 256, smem, s>>>(aa);
        GYPS_CUDA(cudaGetLastError());
        std::vector<int32_t> rk(2 * nb);
        GYPS_CUDA(cudaMemcpyAsync(rk.data(), d32 + 3 * nb, 2 * nb * sizeof(int32_t), cudaMemcpyDeviceToHost, s));
        GYPS_CUDA(cudaStreamSynchronize(s));
        // compact storage: factors of compressed blocks, dense pairs of the others
        int64_t need = 0;
        for (int i = 0; i < nb; ++i)
            need += rk[nb + i] ? (int64_t)rk[i] * (mm[i] + nn[i]) : 2 * (int64_t)mm[i] * nn[i];
        float2 *pool = nullptr;
        st = dmalloc(h, (void **)&pool, (size_t)need * sizeof(float2));
        if (st != GYPS_OK) break;
        int64_t off = 0;
        std::vector<hm::Block *> need_t;
        const size_t first = h->blocks.size();
        for (int i = 0; i < nb; ++i) {
            hm::Block b;
            b.A = far[f0 + i].first;
            b.B = far[f0 + i].second;
            b.m = mm[i];
            b.n = nn[i];
            if (rk[nb + i]) {
                b.lowrank = 1;
                b.rank = rk[i];
                b.U = pool + off;
                b.W = b.U + b.m * b.rank;
                off += b.rank * (b.m + b.n);
                const float2 *u = UW + uw_off[i], *w = u + (int64_t)mm[i] * rmaxb[i];
                GYPS_CUDA(cudaMemcpyAsync(b.U, u, (size_t)(b.m * b.rank) * sizeof(float2), cudaMemcpyDeviceToDevice, s));
                GYPS_CUDA(cudaMemcpyAsync(b.W, w, (size_t)(b.n * b.rank) * sizeof(float2), cudaMemcpyDeviceToDevice, s));
                rank_sum += b.rank;
                ++rank_n;
                h->max_rank = std::max(h->max_rank, b.rank);
            } else {
                b.lowrank = 0;
                b.D = pool + off;
                b.DT = b.D + b.m * b.n;
                off += 2 * b.m * b.n;
                GYPS_CUDA(cudaMemcpyAsync(b.D, S + s_off[i], (size_t)(b.m * b.n) * sizeof(float2), cudaMemcpyDeviceToDevice, s));
                ++h->n_fallback;
            }
            h->blocks.push_back(b);
        }
        for (size_t i = first; i < h->blocks.size(); ++i)
            if (!h->blocks[i].lowrank) need_t.push_back(&h->blocks[i]);
        st = transpose_blocks(h, need_t, s);
        cudaFreeAsync(d64, s);
        cudaFreeAsync(d32, s);
        GYPS_CUDA(cudaStreamSynchronize(s));  // the scratch is reused by the next batch
        f0 = f1;
    }
    if (S) cudaFreeAsync(S, s);
    if (UW) cudaFreeAsync(UW, s);
    GYPS_TRY(st);
    h->n_lowrank = rank_n;
    h->mean_rank = rank_n ? rank_sum / rank_n : 0.0;

    // apply plan: per destination cluster its terms; per low-rank block two projections
    std::vector<std::vector<hm::Term>> terms(h->nc);
    std::vector<hm::Proj> proj;
    int64_t toff = 0;
    for (auto &b : h->blocks) {
        if (!b.lowrank) {
            terms[b.A].push_back({b.D, b.m, (int32_t)b.n, 0, h->voff[b.B]});
            if (b.A != b.B) terms[b.B].push_back({b.DT, b.n, (int32_t)b.m, 0, h->voff[b.A]});
            continue;
        }
        // y_A += U (W^T x_B); y_B += W (U^T x_A)
        proj.push_back({b.W, b.n, b.rank, 0, h->voff[b.B], toff});
        terms[b.A].push_back({b.U, b.m, b.rank, 1, toff});
        toff += (int64_t)b.rank * hm::NRC;
        proj.push_back({b.U, b.m, b.rank, 0, h->voff[b.A], toff});
        terms[b.B].push_back({b.W, b.n, b.rank, 1, toff});
        toff += (int64_t)b.rank * hm::NRC;
    }
    std::vector<hm::Term> flat;
    std::vector<int32_t> ptr(1, 0);
    std::vector<int64_t> chunks;
    for (int64_t c = 0; c < h->nc; ++c) {
        flat.insert(flat.end(), terms[c].begin(), terms[c].end());
        ptr.push_back((int32_t)flat.size());
        for (int64_t q = 0; q * 128 < msize((int)c); ++q) chunks.push_back((c << 32) | q);
    }
    // projections grouped by source range for the 16-column pass (stable: ties keep block order)
    std::stable_sort(proj.begin(), proj.end(), [](const hm::Proj &a, const hm::Proj &b) { return a.src < b.src; });
    std::vector<int2> groups;
    int64_t maxlen = 0;
    for (size_t i = 0; i < proj.size();) {
        size_t e = i;
        while (e < proj.size() && proj[e].src == proj[i].src && e - i < 32) ++e;
        groups.push_back(make_int2((int)i, (int)e));
        maxlen = std::max<int64_t>(maxlen, proj[i].len);
        i = e;
    }
    const int64_t psmem = 8 * maxlen * (int64_t)sizeof(float4);
    h->proj16_smem = psmem <= 200 * 1024 ? (int)psmem : 0;
    h->n_pgroups = (int64_t)groups.size();
    GYPS_TRY(upload(h, &h->d_pgroups, groups, s));
    // 16-column rows pass: row chunks cut into term ranges of at most `cap` units, largest first
    {
        auto units_of = [](const hm::Term &t) { return (int64_t)(t.ncol + RT_K - 1) / RT_K; };
        int64_t total = 0;
        for (int64_t c = 0; c < h->nc; ++c)
            for (int32_t tt = ptr[c]; tt < ptr[c + 1]; ++tt) total += units_of(flat[tt]) * ((msize((int)c) + 127) / 128);
        const int64_t cap = std::max<int64_t>(32, total / 4096);
        std::vector<std::pair<int64_t, int4>> items;
        for (int64_t c = 0; c < h->nc; ++c)
            for (int q = 0; (int64_t)q * 128 < msize((int)c); ++q) {
                int32_t tb = ptr[c];
                int64_t u = 0;
                for (int32_t tt = ptr[c]; tt < ptr[c + 1]; ++tt) {
                    u += units_of(flat[tt]);
                    if (u >= cap || tt + 1 == ptr[c + 1]) {
                        items.push_back({u, make_int4((int)c, q, tb, tt + 1)});
                        tb = tt + 1;
                        u = 0;
                    }
                }
            }
        std::stable_sort(items.begin(), items.end(),
                         [](const std::pair<int64_t, int4> &a, const std::pair<int64_t, int4> &b) { return a.first > b.first; });
        std::vector<int4> iv;
        for (auto &it : items) iv.push_back(it.second);
        h->n_rows_items = (int64_t)iv.size();
        GYPS_TRY(upload(h, &h->d_rows_items, iv, s));
    }
    h->nproj = (int64_t)proj.size();
    h->tlen = toff;
    h->row_chunks = (int64_t)chunks.size();
    GYPS_TRY(upload(h, &h->d_terms, flat, s));
    GYPS_TRY(upload(h, &h->d_term_ptr, ptr, s));
    GYPS_TRY(upload(h, &h->d_proj, proj, s));
    GYPS_TRY(upload(h, &h->d_chunk_cluster, chunks, s));
    int64_t *d_voff = nullptr;
    GYPS_TRY(upload(h, &d_voff, h->voff, s));
    h->voff_dev = d_voff;
    GYPS_TRY(dmalloc(h, (void **)&h->d_T, (size_t)std::max<int64_t>(toff, 1) * sizeof(float2)));
    GYPS_TRY(dmalloc(h, (void **)&h->d_xloc, (size_t)m->nv * hm::NRC * sizeof(float2)));
    GYPS_CUDA(cudaStreamSynchronize(s));
    return GYPS_OK;
}

template <int NR>
static gyps_status apply_pass(Hmat *h, const double2 *X, int64_t ldx, double2 *Y, int64_t ldy, int c0, cudaStream_t s)
{
    const int64_t nv = h->m->nv;
    hm_gather_kernel<<<dim3((unsigned)((nv + 255) / 256), NR), 256, 0, s>>>(h->d_perm, nv, X, ldx, c0, NR, h->d_xloc);
    GYPS_CUDA(cudaGetLastError());
    if (h->nproj > 0 && NR == hm::NRC && h->proj16_smem > 0) {
        GYPS_CUDA(cudaFuncSetAttribute(hm_project16_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       h->proj16_smem));
        hm_project16_kernel<<<(unsigned)h->n_pgroups, 256, h->proj16_smem, s>>>(h->d_proj, h->d_pgroups, h->d_xloc,
                                                                              nv, h->d_T);
        GYPS_CUDA(cudaGetLastError());
    } else if (h->nproj > 0) {
        hm_project_kernel<NR><<<dim3((unsigned)h->nproj, (unsigned)((h->max_rank + 15) / 16)), 256, 0, s>>>(
            h->d_proj, h->d_xloc, nv, h->d_T);
        GYPS_CUDA(cudaGetLastError());
    }
    if (NR == hm::NRC) {
        const int smem = (int)sizeof(RowsTileSmem);
        GYPS_CUDA(cudaFuncSetAttribute(hm_rows16_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
        GYPS_CUDA(cudaMemset2DAsync(Y + (int64_t)c0 * ldy, (size_t)ldy * sizeof(double2), 0,
                                    (size_t)nv * sizeof(double2), hm::NRC, s));
        if (h->n_rows_items > 0)
            hm_rows16_kernel<<<(unsigned)h->n_rows_items, 128, smem, s>>>(h->d_terms, h->d_rows_items, h->voff_dev,
                                                                         h->d_perm, h->d_xloc, nv, h->d_T, Y, ldy, c0);
    } else {
        hm_rows_kernel<NR><<<(unsigned)h->row_chunks, 128, 0, s>>>(h->d_terms, h->d_term_ptr, h->voff_dev,
                                                                 h->d_chunk_cluster, h->d_perm, h->d_xloc, nv, h->d_T,
                                                                 Y, ldy, c0);
    }
    GYPS_CUDA(cudaGetLastError());
    return GYPS_OK;
}

static gyps_status apply_device_hm(Hmat *h, int nrhs, const double2 *X, int64_t ldx, double2 *Y, int64_t ldy,
                                   cudaStream_t s)
{
    for (int c0 = 0; c0 < nrhs;) {
        const int left = nrhs - c0;
        const int w = left >= 16 ? 16 : left >= 8 ? 8 : left >= 4 ? 4 : left >= 2 ? 2 : 1;
        switch (w) {
        case 16: GYPS_TRY(apply_pass<16>(h, X, ldx, Y, ldy, c0, s)); break;
        case 8: GYPS_TRY(apply_pass<8>(h, X, ldx, Y, ldy, c0, s)); break;
        case 4: GYPS_TRY(apply_pass<4>(h, X, ldx, Y, ldy, c0, s)); break;
        case 2: GYPS_TRY(apply_pass<2>(h, X, ldx, Y, ldy, c0, s)); break;
        default: GYPS_TRY(apply_pass<1>(h, X, ldx, Y, ldy, c0, s)); break;
        }
        c0 += w;
    }
    GYPS_CUDA(launch_near_spmv(*h->m, nrhs, X, ldx, Y, ldy, s));
    return GYPS_OK;
}

}  // namespace gyps

using namespace gyps;

struct gyps_hmat_s {
    Hmat *h;
};

namespace gyps {
Hmat *hmat_of(gyps_hmat_t h) { return h ? h->h : nullptr; }
const Mesh *hmat_mesh(const Hmat *h) { return h->m; }
double hmat_k(const Hmat *h) { return h->k; }
gyps_status hmat_apply_device(Hmat *h, int nrhs, const double2 *X, int64_t ldx, double2 *Y, int64_t ldy,
                              cudaStream_t s)
{
    return apply_device_hm(h, nrhs, X, ldx, Y, ldy, s);
}
}  // namespace gyps

extern "C" gyps_status gyps_hmat_create(gyps_mesh_t mesh, double k, double eps, int leaf_tiles, double eta,
                                        void *stream, gyps_hmat_t *out)
{
    if (!out) return set_error(GYPS_ERR_INVALID, "out is NULL");
    *out = nullptr;
    Mesh *m;
    GYPS_TRY(check_mesh(mesh, &m));
    if (!std::isfinite(k) || k < 0.0) return set_error(GYPS_ERR_INVALID, "k must be finite and >= 0");
    if (!(eps >= 1e-7 && eps < 1.0)) return set_error(GYPS_ERR_INVALID, "eps must be in [1e-7, 1)");
    if (leaf_tiles < 1 || leaf_tiles > 64) return set_error(GYPS_ERR_INVALID, "leaf_tiles must be in 1..64");
    if (!(eta > 0.0) || !std::isfinite(eta)) return set_error(GYPS_ERR_INVALID, "eta must be finite and > 0");
    cudaStream_t s = (cudaStream_t)stream;
    Hmat *h = new Hmat();
    h->m = m;
    h->k = k;
    h->eps = eps;
    h->eta = eta;
    h->leaf_tiles = leaf_tiles;
    const auto t0 = std::chrono::steady_clock::now();
    gyps_status st = build(h, s);
    if (st != GYPS_OK) {
        free_hmat(h);
        return st;
    }
    h->build_ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
    *out = new gyps_hmat_s{h};
    return GYPS_OK;
}

extern "C" gyps_status gyps_hmat_apply(gyps_hmat_t hm_, int nrhs, const void *X, int64_t ldx, void *Y, int64_t ldy,
                                       void *stream)
{
    if (!hm_ || !hm_->h) return set_error(GYPS_ERR_INVALID, "NULL handle");
    Hmat *h = hm_->h;
    Mesh *m = h->m;
    if (!X || !Y) return set_error(GYPS_ERR_INVALID, "NULL argument");
    if (nrhs < 1 || nrhs > 4096) return set_error(GYPS_ERR_INVALID, "nrhs must be in 1..4096");
    if (ldx < m->nv || ldy < m->nv) return set_error(GYPS_ERR_INVALID, "leading dimension < nv");
    GYPS_TRY(enter_device(m));
    cudaStream_t s = (cudaStream_t)stream;
    const bool dx = is_device_pointer(X), dy = is_device_pointer(Y);
    if (dx && dy) {
        if ((const char *)X < (const char *)Y + ldy * nrhs * 16 && (const char *)Y < (const char *)X + ldx * nrhs * 16)
            return set_error(GYPS_ERR_INVALID, "X and Y overlap");
        return apply_device_hm(h, nrhs, (const double2 *)X, ldx, (double2 *)Y, ldy, s);
    }
    const size_t blk = (size_t)m->nv * nrhs * sizeof(double2);
    GYPS_TRY(grow(m, &m->ws_stage, &m->ws_stage_bytes, 2 * blk));
    double2 *xs = reinterpret_cast<double2 *>(m->ws_stage), *ys = xs + (size_t)m->nv * nrhs;
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
    GYPS_TRY(apply_device_hm(h, nrhs, xin, lxin, yout, lyout, s));
    if (!dy)
        GYPS_CUDA(cudaMemcpy2DAsync(Y, ldy * sizeof(double2), ys, m->nv * sizeof(double2), m->nv * sizeof(double2), nrhs,
                                    cudaMemcpyDeviceToHost, s));
    GYPS_CUDA(cudaStreamSynchronize(s));
    return GYPS_OK;
}

extern "C" gyps_status gyps_hmat_info(gyps_hmat_t hm_, gyps_hmat_info_t *info)
{
    if (!hm_ || !hm_->h || !info) return set_error(GYPS_ERR_INVALID, "NULL argument");
    const Hmat *h = hm_->h;
    info->clusters = h->nc;
    info->dense_blocks = h->n_dense + h->n_fallback;
    info->lowrank_blocks = h->n_lowrank;
    info->fallback_blocks = h->n_fallback;
    info->max_rank = h->max_rank;
    info->reserved = 0;
    info->mean_rank = h->mean_rank;
    info->bytes = h->bytes;
    info->dense_bytes = 8.0 * (double)h->m->nv * (double)h->m->nv;
    info->build_ms = h->build_ms;
    return GYPS_OK;
}

extern "C" gyps_status gyps_hmat_destroy(gyps_hmat_t hm_)
{
    if (!hm_) return GYPS_OK;
    free_hmat(hm_->h);
    delete hm_;
    return GYPS_OK;
}
