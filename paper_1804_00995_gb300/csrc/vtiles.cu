// Dense Galerkin blocks of the single layer over vertex tiles (Sec. 5, Eq. (BEM)):
//   V_far[i, j] = (1/4pi) sum_{k, l} w_k lambda_i(x_k) G(x_k, y_l) w_l lambda_j(y_l),
// G = exp(ik r)/r, G = ik for a point paired with itself.
//
// Vertices are ordered along a Morton curve and cut into tiles of 64.  The
// points that can touch a tile's vertices are those of T(I), the triangles with
// at least one vertex in the tile; a (target tile I, source tile J) item sums
// over the point pairs of T(I) x T(J) and produces the complete 64 x 64 block
// of V_far for rows I and columns J, so every entry is written exactly once and
// no atomics are needed.  V_far is complex symmetric (G_kl = G_lk, the same
// rule and basis on both sides), so only items with I <= J are computed and an
// off-diagonal block is also written transposed.
//
// Inside an item, 128 threads each own one target point of a pass (whole
// triangles: 42 at q = 3) and stream the triangles of T(J) from shared memory:
// per source triangle the q kernel values are contracted with the trial
// coefficients w_l lambda_m(l) into three complex sums, which go into the
// thread's own column of H[j][k] (the source side summed per target point, no
// conflicts: a warp writes 32 consecutive entries).  After the pass, 64 threads
// (one per column j) contract H with the test coefficients of each target
// triangle and add the three results into the block accumulator Vacc[i][j].
// FP32 kernel values (coordinates scaled by k, phase reduced by two constants of
// 2 pi, MUFU rsqrt / sin / cos) and FP32 sums; the block is scaled by k/(4 pi)
// and converted when it is written.
#include <algorithm>
#include <cmath>
#include <cstdint>
#include <numeric>
#include <unordered_set>
#include <vector>

#include "far_tile.cuh"
#include "internal.h"
#include "vtiles.h"

namespace gyps {

// ---------------------------------------------------------------- host: tiles
static uint32_t spread10(uint32_t v)
{
    v &= 1023u;
    v = (v | (v << 16)) & 0x030000FFu;
    v = (v | (v << 8)) & 0x0300F00Fu;
    v = (v | (v << 4)) & 0x030C30C3u;
    v = (v | (v << 2)) & 0x09249249u;
    return v;
}

void build_vertex_tiles(const std::vector<double> &vtx, const std::vector<int32_t> &tri, int64_t nv, int64_t nt,
                        int64_t tri_cap, VertexTiles *out)
{
    VertexTiles &T = *out;
    double lo[3] = {1e300, 1e300, 1e300}, hi[3] = {-1e300, -1e300, -1e300};
    for (int64_t i = 0; i < nv; ++i)
        for (int d = 0; d < 3; ++d) {
            lo[d] = std::min(lo[d], vtx[3 * i + d]);
            hi[d] = std::max(hi[d], vtx[3 * i + d]);
        }
    double ext = std::max({hi[0] - lo[0], hi[1] - lo[1], hi[2] - lo[2], 1e-300});
    std::vector<uint64_t> key(nv);
    for (int64_t i = 0; i < nv; ++i) {
        uint32_t c[3];
        for (int d = 0; d < 3; ++d)
            c[d] = (uint32_t)std::min(1023.0, std::floor((vtx[3 * i + d] - lo[d]) / ext * 1024.0));
        const uint64_t code = spread10(c[0]) | (spread10(c[1]) << 1) | (spread10(c[2]) << 2);
        key[i] = (code << 32) | (uint64_t)i;
    }
    std::sort(key.begin(), key.end());
    // Cut the Morton sequence greedily: a tile closes at kTileV vertices or when the
    // next vertex would bring |T(I)| above tri_cap (a whole number of target passes).
    std::vector<std::vector<int32_t>> v2t(nv);
    for (int64_t t = 0; t < nt; ++t)
        for (int m = 0; m < 3; ++m) v2t[tri[3 * t + m]].push_back((int32_t)t);
    std::vector<int64_t> mark(nt, -1);
    std::vector<std::vector<int32_t>> tiles;
    std::vector<int32_t> cur;
    int64_t ncur = 0;
    for (int64_t p = 0; p < nv; ++p) {
        const int32_t v = (int32_t)(key[p] & 0xffffffffu);
        int64_t fresh = 0;
        for (int32_t t : v2t[v]) fresh += mark[t] != (int64_t)tiles.size();
        if (!cur.empty() && ((int64_t)cur.size() == kTileV || ncur + fresh > tri_cap)) {
            tiles.push_back(cur);
            cur.clear();
            ncur = 0;
        }
        for (int32_t t : v2t[v])
            if (mark[t] != (int64_t)tiles.size()) {
                mark[t] = (int64_t)tiles.size();
                ++ncur;
            }
        cur.push_back(v);
    }
    if (!cur.empty()) tiles.push_back(cur);
    T.ntiles = (int64_t)tiles.size();
    T.rowmap.assign(T.ntiles * kTileV, -1);
    std::vector<int32_t> tile_of(nv), slot_of(nv);
    for (int64_t t = 0; t < T.ntiles; ++t) {
        std::vector<int32_t> &ids = tiles[t];
        std::sort(ids.begin(), ids.end());  // ascending rows inside a tile: neighbouring writes
        for (size_t s = 0; s < ids.size(); ++s) {
            T.rowmap[t * kTileV + s] = ids[s];
            tile_of[ids[s]] = (int32_t)t;
            slot_of[ids[s]] = (int32_t)s;
        }
    }
    // T(I): triangles with a vertex in tile I, with the local slots of their vertices
    std::vector<int64_t> cnt(T.ntiles + 1, 0);
    auto tiles_of = [&](int64_t t, int32_t *out3) {
        int n = 0;
        for (int m = 0; m < 3; ++m) {
            const int32_t tl = tile_of[tri[3 * t + m]];
            bool seen = false;
            for (int u = 0; u < n; ++u) seen = seen || out3[u] == tl;
            if (!seen) out3[n++] = tl;
        }
        return n;
    };
    for (int64_t t = 0; t < nt; ++t) {
        int32_t ts[3];
        const int n = tiles_of(t, ts);
        for (int u = 0; u < n; ++u) cnt[ts[u] + 1]++;
    }
    for (int64_t t = 0; t < T.ntiles; ++t) cnt[t + 1] += cnt[t];
    T.tile_ptr.assign(cnt.begin(), cnt.end());
    T.ntt = cnt[T.ntiles];
    T.tri.resize(T.ntt);
    T.loc.resize(T.ntt);
    std::vector<int64_t> fill(cnt.begin(), cnt.end() - 1);
    std::unordered_set<uint64_t> adjacent;  // tile pairs sharing a triangle (the same point on both sides)
    for (int64_t t = 0; t < nt; ++t) {
        int32_t ts[3];
        const int n = tiles_of(t, ts);
        for (int u = 0; u < n; ++u) {
            const int32_t tl = ts[u];
            uint32_t packed = 0;
            for (int m = 0; m < 3; ++m) {
                const int32_t v = tri[3 * t + m];
                if (tile_of[v] == tl) packed |= (uint32_t)(slot_of[v] + 1) << (8 * m);
            }
            const int64_t e = fill[tl]++;
            T.tri[e] = (int32_t)t;
            T.loc[e] = (int32_t)packed;
            for (int w = 0; w < n; ++w) {
                const uint64_t a = (uint64_t)std::min(ts[u], ts[w]), b = (uint64_t)std::max(ts[u], ts[w]);
                adjacent.insert((a << 32) | b);
            }
        }
    }
    T.max_tri = 0;
    for (int64_t t = 0; t < T.ntiles; ++t) T.max_tri = std::max<int64_t>(T.max_tri, cnt[t + 1] - cnt[t]);
    // items (I <= J), row by row: the target tile's panel stays in L2 over a row
    T.items.clear();
    T.items.reserve((size_t)(T.ntiles * (T.ntiles + 1) / 2));
    for (int32_t I = 0; I < (int32_t)T.ntiles; ++I)
        for (int32_t J = I; J < (int32_t)T.ntiles; ++J) {
            const int self = adjacent.count(((uint64_t)I << 32) | (uint64_t)J) ? 1 : 0;
            T.items.push_back(make_int4(I, J, self, 0));
        }
}

// ---------------------------------------------------------------- device: panel
// Per tile-triangle e and point l of its triangle: position scaled by ks with the
// global point index in .w (as bits), and the coefficients w_l lambda_m(l) of the
// triangle's vertices that belong to the tile (0 for the others).
__global__ void tile_panel_kernel(const int32_t *tt_tri, const int32_t *tt_loc, int64_t ntt,
                                  const double4_32a *pts64, const Rule rule, float ks, float4 *pos, float4 *coef)
{
    const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= ntt * rule.q) return;
    const int64_t e = idx / rule.q;
    const int l = (int)(idx - e * rule.q);
    const int64_t p = (int64_t)tt_tri[e] * rule.q + l;
    const double4_32a x = pts64[p];
    pos[idx] = make_float4((float)x.x * ks, (float)x.y * ks, (float)x.z * ks, __int_as_float((int)p));
    const uint32_t loc = (uint32_t)tt_loc[e];
    float c[3];
#pragma unroll
    for (int m = 0; m < 3; ++m) c[m] = ((loc >> (8 * m)) & 255u) ? (float)(x.w * rule.bary[3 * l + m]) : 0.0f;
    coef[idx] = make_float4(c[0], c[1], c[2], 0.0f);
}

// ---------------------------------------------------------------- device: blocks
template <int Q>
struct TileCfg {
    static constexpr int NT = 128;
    static constexpr int TPP = NT / Q;         // target triangles per pass
    static constexpr int PPP = TPP * Q;        // target points per pass
    static constexpr int CH = Q == 7 ? 16 : 32;  // source triangles per staged chunk
    static constexpr int HLD = NT + 1;         // padded row of H (float2)
    static constexpr int VLD = kTileV + 1;     // padded row of Vacc (float2)
    static constexpr int H_BYTES = kTileV * HLD * 8;
    static constexpr int V_BYTES = kTileV * VLD * 8;
    static constexpr int S_BYTES = CH * Q * 32 + CH * 4;  // one chunk: positions, coefficients, slots
    static constexpr int T_BYTES = PPP * 16 + TPP * 4;    // test coefficients and slots of a pass
    static constexpr int SMEM = H_BYTES + V_BYTES + S_BYTES + T_BYTES;
};

// Whole target passes: about 180 triangles touch 64 vertices of a closed surface.
int64_t tile_tri_cap(int q)
{
    const int tpp = q == 1 ? TileCfg<1>::TPP : q == 3 ? TileCfg<3>::TPP : TileCfg<7>::TPP;
    return (int64_t)tpp * std::max<int64_t>(1, 170 / tpp);
}

__device__ __forceinline__ void cadd_scaled(float2 &acc, float2 g, float c)
{
    acc.x = fmaf(g.x, c, acc.x);
    acc.y = fmaf(g.y, c, acc.y);
}

template <typename OutT>
__device__ __forceinline__ OutT to_out(float2 v, double scale);
template <>
__device__ __forceinline__ double2 to_out<double2>(float2 v, double scale)
{
    return make_double2((double)v.x * scale, (double)v.y * scale);
}
template <>
__device__ __forceinline__ float2 to_out<float2>(float2 v, double scale)
{
    return make_float2((float)((double)v.x * scale), (float)((double)v.y * scale));
}

// Source-side sums of one target point against the staged chunk of triangles.
template <int Q, bool LAP, bool SELF>
__device__ __forceinline__ void chunk_sums(const float4 *spos, const float4 *scoef, const int *sloc, int nch,
                                           float4 tp, int gk, float2 *Hcol)
{
    constexpr int HLD = TileCfg<Q>::HLD;
    const float inv2pi = 0.159154943091895335769f;
    const float c1 = 6.28318548202514648438f;      // 2 pi rounded to FP32
    const float c2 = -1.74845553146951715e-07f;   // 2 pi - c1
    const float magic = 12582912.0f;              // 1.5 * 2^23: round to integer
    for (int b = 0; b < nch; ++b) {
        float2 s0 = make_float2(0.f, 0.f), s1 = s0, s2 = s0;
#pragma unroll
        for (int l = 0; l < Q; ++l) {
            const float4 p = spos[b * Q + l];
            const float4 c = scoef[b * Q + l];
            const float dx = tp.x - p.x, dy = tp.y - p.y, dz = tp.z - p.z;
            const float r2 = fmaf(dz, dz, fmaf(dy, dy, dx * dx));
            const float rs = rsqrt_mufu(r2);
            float2 g;
            if (LAP) {
                g = make_float2(rs, 0.0f);
                if (SELF && __float_as_int(p.w) == gk) g.x = 0.0f;
            } else {
                const float ph = r2 * rs;                                  // k r
                const float nr = fmaf(ph, inv2pi, magic) - magic;          // nearest integer to k r / (2 pi)
                const float ang = fmaf(nr, -c2, fmaf(nr, -c1, ph));        // in [-pi, pi]
                g = make_float2(cos_mufu(ang) * rs, sin_mufu(ang) * rs);   // exp(ikr) / (k r)
                if (SELF && __float_as_int(p.w) == gk) g = make_float2(0.0f, 1.0f);  // ik / k
            }
            cadd_scaled(s0, g, c.x);
            cadd_scaled(s1, g, c.y);
            cadd_scaled(s2, g, c.z);
        }
        const uint32_t loc = (uint32_t)sloc[b];
        const int m0 = (int)(loc & 255u) - 1, m1 = (int)((loc >> 8) & 255u) - 1, m2 = (int)((loc >> 16) & 255u) - 1;
        if (m0 >= 0) {
            float2 h = Hcol[m0 * HLD];
            Hcol[m0 * HLD] = make_float2(h.x + s0.x, h.y + s0.y);
        }
        if (m1 >= 0) {
            float2 h = Hcol[m1 * HLD];
            Hcol[m1 * HLD] = make_float2(h.x + s1.x, h.y + s1.y);
        }
        if (m2 >= 0) {
            float2 h = Hcol[m2 * HLD];
            Hcol[m2 * HLD] = make_float2(h.x + s2.x, h.y + s2.y);
        }
    }
}

template <int Q, bool LAP, typename OutT>
__global__ void __launch_bounds__(128, 2) tile_block_kernel(const TileArgs a, OutT *out)
{
    using C = TileCfg<Q>;
    constexpr int NT = C::NT, HLD = C::HLD, VLD = C::VLD;
    extern __shared__ __align__(16) unsigned char smem[];
    float2 *H = reinterpret_cast<float2 *>(smem);
    float2 *Vacc = reinterpret_cast<float2 *>(smem + C::H_BYTES);
    float4 *spos = reinterpret_cast<float4 *>(smem + C::H_BYTES + C::V_BYTES);
    float4 *scoef = spos + C::CH * Q;
    int *sloc = reinterpret_cast<int *>(scoef + C::CH * Q);
    float4 *tcoef = reinterpret_cast<float4 *>(smem + C::H_BYTES + C::V_BYTES + C::S_BYTES);
    int *tloc = reinterpret_cast<int *>(tcoef + C::PPP);
    const int tid = threadIdx.x;

    for (int64_t it = blockIdx.x; it < a.n_items; it += gridDim.x) {
        const int4 item = a.items[it];
        const int I = item.x, J = item.y;
        const bool self = item.z & 1;
        for (int e = tid; e < kTileV * VLD; e += NT) Vacc[e] = make_float2(0.f, 0.f);
        const int tI0 = a.tile_ptr[I], nTI = a.tile_ptr[I + 1] - tI0;
        const int tJ0 = a.tile_ptr[J], nTJ = a.tile_ptr[J + 1] - tJ0;
        for (int pb = 0; pb < nTI; pb += C::TPP) {
            const int ntp = min(C::TPP, nTI - pb);
            const bool active = tid < ntp * Q;
            float4 tp = make_float4(0.f, 0.f, 0.f, __int_as_float(-1));
            if (active) {
                const int64_t pe = (int64_t)(tI0 + pb) * Q + tid;  // tile-triangle (tI0 + pb + tid / Q), point tid % Q
                tp = a.pos[pe];
                tcoef[tid] = a.coef[pe];
                if (tid % Q == 0) tloc[tid / Q] = a.loc[tI0 + pb + tid / Q];
            }
            const int gk = __float_as_int(tp.w);
#pragma unroll 8
            for (int j = 0; j < kTileV; ++j) H[j * HLD + tid] = make_float2(0.f, 0.f);
            for (int cb = 0; cb < nTJ; cb += C::CH) {
                const int nch = min(C::CH, nTJ - cb);
                __syncthreads();  // the previous chunk is consumed
                const int64_t base = (int64_t)(tJ0 + cb) * Q;
                for (int e = tid; e < nch * Q; e += NT) {
                    spos[e] = a.pos[base + e];
                    scoef[e] = a.coef[base + e];
                }
                for (int e = tid; e < nch; e += NT) sloc[e] = a.loc[tJ0 + cb + e];
                __syncthreads();
                if (active) {
                    if (self)
                        chunk_sums<Q, LAP, true>(spos, scoef, sloc, nch, tp, gk, H + tid);
                    else
                        chunk_sums<Q, LAP, false>(spos, scoef, sloc, nch, tp, gk, H + tid);
                }
            }
            __syncthreads();  // H, tcoef, tloc complete
            if (tid < kTileV) {
                const float2 *Hrow = H + tid * HLD;
                for (int t = 0; t < ntp; ++t) {
                    float2 r0 = make_float2(0.f, 0.f), r1 = r0, r2 = r0;
#pragma unroll
                    for (int l = 0; l < Q; ++l) {
                        const float2 h = Hrow[t * Q + l];
                        const float4 c = tcoef[t * Q + l];
                        cadd_scaled(r0, h, c.x);
                        cadd_scaled(r1, h, c.y);
                        cadd_scaled(r2, h, c.z);
                    }
                    const uint32_t loc = (uint32_t)tloc[t];
                    const int m0 = (int)(loc & 255u) - 1, m1 = (int)((loc >> 8) & 255u) - 1,
                              m2 = (int)((loc >> 16) & 255u) - 1;
                    if (m0 >= 0) {
                        float2 v = Vacc[m0 * VLD + tid];
                        Vacc[m0 * VLD + tid] = make_float2(v.x + r0.x, v.y + r0.y);
                    }
                    if (m1 >= 0) {
                        float2 v = Vacc[m1 * VLD + tid];
                        Vacc[m1 * VLD + tid] = make_float2(v.x + r1.x, v.y + r1.y);
                    }
                    if (m2 >= 0) {
                        float2 v = Vacc[m2 * VLD + tid];
                        Vacc[m2 * VLD + tid] = make_float2(v.x + r2.x, v.y + r2.y);
                    }
                }
            }
            __syncthreads();  // before the next pass refills H, tcoef, tloc
        }
        // the block: rows of tile I, columns of tile J (and the transposed block)
        const int32_t *rI = a.rowmap + (int64_t)I * kTileV, *rJ = a.rowmap + (int64_t)J * kTileV;
        const int32_t *cI = a.colmap + (int64_t)I * kTileV, *cJ = a.colmap + (int64_t)J * kTileV;
        OutT *blk = out + (a.item_off ? a.item_off[it] : 0);
        for (int e = tid; e < kTileV * kTileV; e += NT) {
            const int i = e % kTileV, j = e / kTileV;  // rows fastest
            const int32_t r = rI[i], c = cJ[j];
            if (r >= 0 && c >= 0) blk[r + (int64_t)c * a.ld] = to_out<OutT>(Vacc[i * VLD + j], a.scale);
        }
        if (a.transpose && I != J) {
            for (int e = tid; e < kTileV * kTileV; e += NT) {
                const int j = e % kTileV, i = e / kTileV;
                const int32_t r = rJ[j], c = cI[i];
                if (r >= 0 && c >= 0) blk[r + (int64_t)c * a.ld] = to_out<OutT>(Vacc[i * VLD + j], a.scale);
            }
        }
        __syncthreads();  // Vacc is read before the next item clears it
    }
}

// ---------------------------------------------------------------- host: launch
gyps_status vertex_tiles_prepare(Mesh *m, cudaStream_t s)
{
    if (m->vt) return GYPS_OK;
    std::vector<double> vtx(3 * m->nv);
    std::vector<int32_t> tri(3 * m->nt);
    GYPS_CUDA(cudaMemcpyAsync(vtx.data(), m->d_vtx, vtx.size() * sizeof(double), cudaMemcpyDeviceToHost, s));
    GYPS_CUDA(cudaMemcpyAsync(tri.data(), m->d_tri, tri.size() * sizeof(int32_t), cudaMemcpyDeviceToHost, s));
    GYPS_CUDA(cudaStreamSynchronize(s));
    VertexTiles *T = new VertexTiles();
    build_vertex_tiles(vtx, tri, m->nv, m->nt, tile_tri_cap(m->q), T);
    auto up = [&](auto **dst, const auto &v) -> gyps_status {
        using E = typename std::remove_reference<decltype(v)>::type::value_type;
        const size_t bytes = std::max<size_t>(v.size(), 1) * sizeof(E);
        GYPS_CUDA(cudaMalloc((void **)dst, bytes));
        m->device_bytes += (int64_t)bytes;
        if (!v.empty()) GYPS_CUDA(cudaMemcpyAsync(*dst, v.data(), v.size() * sizeof(E), cudaMemcpyHostToDevice, s));
        return GYPS_OK;
    };
    gyps_status st = GYPS_OK;
    std::vector<int32_t> tp32(T->tile_ptr.begin(), T->tile_ptr.end());
    if (st == GYPS_OK) st = up(&T->d_tile_ptr, tp32);
    if (st == GYPS_OK) st = up(&T->d_tri, T->tri);
    if (st == GYPS_OK) st = up(&T->d_loc, T->loc);
    if (st == GYPS_OK) st = up(&T->d_rowmap, T->rowmap);
    if (st == GYPS_OK) st = up(&T->d_items, T->items);
    if (st == GYPS_OK) {
        const size_t bytes = (size_t)T->ntt * m->q * sizeof(float4) * 2;
        if (cudaMalloc((void **)&T->d_pos, bytes) != cudaSuccess) st = set_error(GYPS_ERR_OOM, "tile panel");
        else {
            T->d_coef = T->d_pos + T->ntt * m->q;
            m->device_bytes += (int64_t)bytes;
        }
    }
    if (st == GYPS_OK) {
        cudaError_t e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) st = cuda_error(e, "vertex tiles upload");
    }
    if (st != GYPS_OK) {
        free_vertex_tiles(T);
        return st;
    }
    m->vt = T;
    return GYPS_OK;
}

void free_vertex_tiles(VertexTiles *T)
{
    if (!T) return;
    void *ptrs[] = {T->d_tile_ptr, T->d_tri, T->d_loc, T->d_rowmap, T->d_items, T->d_pos};
    for (void *p : ptrs)
        if (p) cudaFree(p);
    delete T;
}

gyps_status tile_panel(Mesh *m, double k, cudaStream_t s)
{
    VertexTiles *T = m->vt;
    const float ks = k > 0.0 ? (float)k : 1.0f;
    const int64_t n = T->ntt * m->q;
    tile_panel_kernel<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(T->d_tri, T->d_loc, T->ntt, m->d_pts64, m->rule, ks,
                                                                 T->d_pos, T->d_coef);
    GYPS_CUDA(cudaGetLastError());
    return GYPS_OK;
}

template <int Q, bool LAP, typename OutT>
static gyps_status launch_blocks_q(Mesh *m, const TileArgs &a, OutT *out, cudaStream_t s)
{
    using C = TileCfg<Q>;
    auto kern = tile_block_kernel<Q, LAP, OutT>;
    GYPS_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, C::SMEM));
    int occ = 0;
    GYPS_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, C::NT, C::SMEM));
    occ = std::max(occ, 1);
    const int64_t grid = std::min<int64_t>((int64_t)m->num_sms * occ, a.n_items);
    if (grid <= 0) return GYPS_OK;
    kern<<<(unsigned)grid, C::NT, C::SMEM, s>>>(a, out);
    GYPS_CUDA(cudaGetLastError());
    return GYPS_OK;
}

template <typename OutT>
gyps_status tile_blocks(Mesh *m, double k, const TileArgs &a, OutT *out, cudaStream_t s)
{
    const bool lap = !(k > 0.0);
    switch (m->q) {
    case 1: return lap ? launch_blocks_q<1, true>(m, a, out, s) : launch_blocks_q<1, false>(m, a, out, s);
    case 3: return lap ? launch_blocks_q<3, true>(m, a, out, s) : launch_blocks_q<3, false>(m, a, out, s);
    case 7: return lap ? launch_blocks_q<7, true>(m, a, out, s) : launch_blocks_q<7, false>(m, a, out, s);
    default: return set_error(GYPS_ERR_INVALID, "quadrature rule");
    }
}
template gyps_status tile_blocks<double2>(Mesh *, double, const TileArgs &, double2 *, cudaStream_t);
template gyps_status tile_blocks<float2>(Mesh *, double, const TileArgs &, float2 *, cudaStream_t);

TileArgs tile_args(const Mesh *m, double k)
{
    const VertexTiles *T = m->vt;
    TileArgs a{};
    a.pos = T->d_pos;
    a.coef = T->d_coef;
    a.loc = T->d_loc;
    a.tile_ptr = T->d_tile_ptr;
    a.rowmap = T->d_rowmap;
    a.colmap = T->d_rowmap;
    a.items = T->d_items;
    a.item_off = nullptr;
    a.n_items = (int64_t)T->items.size();
    a.ld = m->nv;
    a.scale = (k > 0.0 ? k : 1.0) / (4.0 * 3.14159265358979323846);
    a.transpose = 1;
    return a;
}

// a6 in FP32 kernel values: V = V_far (tile blocks, each entry written once) + C.
gyps_status assemble_tiles(Mesh *m, double k, double2 *V, int64_t ldv, cudaStream_t s)
{
    GYPS_TRY(vertex_tiles_prepare(m, s));
    GYPS_TRY(tile_panel(m, k, s));
    TileArgs a = tile_args(m, k);
    a.ld = ldv;
    return tile_blocks<double2>(m, k, a, V, s);
}

}  // namespace gyps
