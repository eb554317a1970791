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
#include <array>
#include <cmath>
#include <cstdint>
#include <numeric>
#include <string>
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

// The six orders of a triangle's vertices: kPerm[p][m] = original vertex at position m.
static const int kPerm[6][3] = {{0, 1, 2}, {1, 2, 0}, {2, 0, 1}, {0, 2, 1}, {2, 1, 0}, {1, 0, 2}};

// Orders each tile's triangle list as a strip (each next triangle shares as many
// tile vertices as possible with the one before) and turns each triangle's
// vertices so that a vertex shared with the previous triangle keeps its
// position.  The kernel keeps one running sum per position in registers and
// writes it to shared memory only when the vertex at that position changes
// (flush bit m in byte 3 of the packed slots).
void order_tile_triangles(VertexTiles &T)
{
    T.perm.assign(T.ntt, 0);
    std::vector<int32_t> tri2, loc2;
    for (int64_t I = 0; I < T.ntiles; ++I) {
        const int64_t b = T.tile_ptr[I], n = T.tile_ptr[I + 1] - b;
        std::vector<std::array<int, 3>> sl(n);
        for (int64_t e = 0; e < n; ++e)
            for (int m = 0; m < 3; ++m) sl[e][m] = (int)((T.loc[b + e] >> (8 * m)) & 255) - 1;
        auto shared = [&](int64_t x, int64_t y) {
            int c = 0;
            for (int m = 0; m < 3; ++m)
                for (int mm = 0; mm < 3; ++mm) c += sl[x][m] >= 0 && sl[x][m] == sl[y][mm];
            return c;
        };
        std::vector<char> seen(n, 0);
        std::vector<int64_t> order;
        order.reserve(n);
        int64_t cur = 0;
        for (int64_t k = 0; k < n; ++k) {
            seen[cur] = 1;
            order.push_back(cur);
            int64_t best = -1;
            int bs = -1;
            for (int64_t e = 0; e < n; ++e)
                if (!seen[e]) {
                    const int sc = shared(cur, e);
                    if (sc > bs) {
                        bs = sc;
                        best = e;
                    }
                }
            if (best < 0) break;
            cur = best;
        }
        int prev[3] = {-1, -1, -1};
        for (int64_t k = 0; k < n; ++k) {
            const int64_t e = order[k];
            int bp = 0, bm = -1;
            for (int p = 0; p < 6; ++p) {
                int match = 0;
                for (int m = 0; m < 3; ++m) match += prev[m] >= 0 && sl[e][kPerm[p][m]] == prev[m];
                if (match > bm) {
                    bm = match;
                    bp = p;
                }
            }
            uint32_t packed = 0;
            int cur3[3];
            for (int m = 0; m < 3; ++m) {
                cur3[m] = sl[e][kPerm[bp][m]];
                packed |= (uint32_t)(cur3[m] + 1) << (8 * m);
                if (cur3[m] != prev[m]) packed |= 1u << (24 + m);
                prev[m] = cur3[m];
            }
            tri2.push_back(T.tri[b + e]);
            loc2.push_back((int32_t)packed);
            T.perm[b + k] = (int8_t)bp;
        }
    }
    T.tri.swap(tri2);
    T.loc.swap(loc2);
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
    T.adjacent.assign(adjacent.begin(), adjacent.end());
    std::sort(T.adjacent.begin(), T.adjacent.end());
    order_tile_triangles(T);
    T.max_tri = 0;
    for (int64_t t = 0; t < T.ntiles; ++t) T.max_tri = std::max<int64_t>(T.max_tri, cnt[t + 1] - cnt[t]);
    // items (I <= J), row by row: the target tile's panel stays in L2 over a row
    T.items.clear();
    T.items.reserve((size_t)(T.ntiles * (T.ntiles + 1) / 2));
    for (int32_t I = 0; I < (int32_t)T.ntiles; ++I)
        for (int32_t J = I; J < (int32_t)T.ntiles; ++J) {
            const int self = adjacent.count(((uint64_t)I << 32) | (uint64_t)J) ? 1 : 0;
            T.items.push_back(make_int4(I, J, self | 2, 0));
        }
}

// ---------------------------------------------------------------- device: panel
// Per tile-triangle e and point l (in the order of the triangle's turned
// vertices): the point scaled by ks and negated (a source point enters through
// one packed addition), with its global index in .w (bits); per tile-triangle
// (packed slots and flush bits, area bits).  The coefficient w_l lambda_m(l) of
// the vertex at position m is area x R[l][m] with R[l][m] = (reference weight
// of l) x lambda_m(l) from the rule: the rules are symmetric under every order
// of the vertices, so turning a triangle only permutes its points (sigma).
__global__ void tile_panel_kernel(const int32_t *tt_tri, const int32_t *tt_loc, const int8_t *tt_perm, int64_t ntt,
                                  const double4_32a *pts64, const Rule rule, const PointPerm pp, float ks, float4 *pos,
                                  int2 *tl)
{
    const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= ntt * rule.q) return;
    const int64_t e = idx / rule.q;
    const int l = (int)(idx - e * rule.q);
    const int64_t t = tt_tri[e];
    const int64_t p = t * rule.q + pp.sigma[tt_perm[e]][l];  // the point that sits at position l after the turn
    const double4_32a x = pts64[p];
    const double area = pts64[t * rule.q].w / rule.w[0];
    pos[idx] = make_float4(-(float)x.x * ks, -(float)x.y * ks, -(float)x.z * ks, __int_as_float((int)p));
    if (l == 0) tl[e] = make_int2(tt_loc[e], __float_as_int((float)area));
}

// ---------------------------------------------------------------- device: blocks
template <int Q>
struct TileCfg {
    static constexpr int NT = 128;
    static constexpr int TPP = Q == 3 ? 40 : Q == 7 ? 17 : 120;   // target triangles per pass
    static constexpr int SRC = Q == 3 ? 160 : Q == 7 ? 40 : 120;  // source triangles staged at once (multiple of 8)
    static constexpr int LCAP = 16;                               // (triangle, position) entries of a slot in a pass
    static constexpr int HLD = 121;                               // padded row of H (float2; odd: no conflicts)
    static constexpr int H_BYTES = kTileV * HLD * 8;
    static constexpr int S_BYTES = SRC * Q * 16 + SRC * 8;        // staged source points, (slots, area)
    static constexpr int L_BYTES = kTileV * LCAP * 2 + kTileV * 4; // per-slot entry lists of a pass and counts
    // (slots, area) of the pass's targets, area, R^T; then, 16-byte aligned, area x R^T[m][l]
    // per target triangle as (c, c)
    static constexpr int C_OFF = (TPP * 8 + TPP * 4 + 3 * 8 * 4 + 15) / 16 * 16;
    static constexpr int T_BYTES = C_OFF + TPP * 3 * Q * 8;
    static constexpr int SMEM = H_BYTES + S_BYTES + L_BYTES + T_BYTES;
    static_assert(TPP * Q <= NT && TPP * Q < HLD, "a pass fits the threads and H");
    static_assert(kTileV * (kTileV + 1) * 8 <= H_BYTES, "the block staging fits in H");
};

// Whole target passes: about 170 triangles touch 64 vertices of a closed surface.
int64_t tile_tri_cap(int q)
{
    const int tpp = q == 1 ? TileCfg<1>::TPP : q == 3 ? TileCfg<3>::TPP : TileCfg<7>::TPP;
    return (int64_t)tpp * std::max<int64_t>(1, (170 + tpp / 2) / tpp);
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

// Running sums of one target point per vertex position (registers), written
// into the thread's column of H when the vertex at that position changes.
struct PosSums {
    float2 a0, a1, a2;
    int c0, c1, c2;  // slot held at each position (-1: none)
};

__device__ __forceinline__ void pos_flush(float2 *__restrict__ Hcol, int hld, int c, float2 &acc)
{
    if (c >= 0) {
        const float2 o = Hcol[c * hld];
        Hcol[c * hld] = make_float2(o.x + acc.x, o.y + acc.y);
    }
    acc = make_float2(0.f, 0.f);
}

// Kernel sums of one target point against two source triangles b0, b1 packed in
// the lanes of f32x2 values: t_m = area sum_l G(x, y_l) R[l][m] for the three
// vertex positions m of each triangle (lane .x: b0, lane .y: b1).
struct PairSums {
    float2 t0r, t0i, t1r, t1i, t2r, t2i;
};

// CIRC (rules whose R[l][m] is beta + (alpha - beta) [l == m], as the 3-point rule):
// t_m = area (beta sum_l G_l + (alpha - beta) G_m), without the per-point products.
template <int Q, bool LAP, bool SELF, bool CIRC>
__device__ __forceinline__ PairSums pair_sums(const float4 *__restrict__ sxy, const float4 *__restrict__ szg, int pr,
                                              float2 ar, float2 tx, float2 ty, float2 tz, int gk, const float (&R)[Q][3])
{
    const float2 inv2pi = make_float2(0.159154943091895335769f, 0.159154943091895335769f);
    const float2 mc1 = make_float2(-6.28318548202514648438f, -6.28318548202514648438f);  // -(2 pi in FP32)
    const float2 mc2 = make_float2(1.74845553146951715e-07f, 1.74845553146951715e-07f);  // -(2 pi - that)
    const float2 magic = make_float2(12582912.0f, 12582912.0f);    // 1.5 * 2^23: round to integer
    const float2 nmagic = make_float2(-12582912.0f, -12582912.0f);
    PairSums o;
    o.t0r = o.t0i = o.t1r = o.t1i = o.t2r = o.t2i = make_float2(0.f, 0.f);
    float2 gl_r[CIRC ? Q : 1], gl_i[CIRC ? Q : 1];  // per-point values (CIRC)
    float2 sr = make_float2(0.f, 0.f), si = make_float2(0.f, 0.f);
#pragma unroll
    for (int l = 0; l < Q; ++l) {
        const float4 xy = sxy[pr * Q + l], zg = szg[pr * Q + l];  // (x0, x1, y0, y1), (z0, z1, id0, id1)
        const float2 dx = __fadd2_rn(tx, make_float2(xy.x, xy.y));
        const float2 dy = __fadd2_rn(ty, make_float2(xy.z, xy.w));
        const float2 dz = __fadd2_rn(tz, make_float2(zg.x, zg.y));
        float2 r2 = __fmul2_rn(dx, dx);
        r2 = __ffma2_rn(dy, dy, r2);
        r2 = __ffma2_rn(dz, dz, r2);
        const float2 rs = make_float2(rsqrt_mufu(r2.x), rsqrt_mufu(r2.y));
        float2 gr, gi;
        if (LAP) {
            gr = rs;
            if (SELF) {
                if (__float_as_int(zg.z) == gk) gr.x = 0.0f;
                if (__float_as_int(zg.w) == gk) gr.y = 0.0f;
            }
        } else {
            const float2 ph = __fmul2_rn(r2, rs);                                  // k r
            const float2 nr = __fadd2_rn(__ffma2_rn(ph, inv2pi, magic), nmagic);   // nearest integer to k r / (2 pi)
            const float2 ang = __ffma2_rn(nr, mc2, __ffma2_rn(nr, mc1, ph));       // in [-pi, pi]
            const float2 sn = make_float2(sin_mufu(ang.x), sin_mufu(ang.y));
            const float2 cs = make_float2(cos_mufu(ang.x), cos_mufu(ang.y));
            gr = __fmul2_rn(cs, rs);                                               // exp(ikr) / (k r)
            gi = __fmul2_rn(sn, rs);
            if (SELF) {  // the point paired with itself: ik / k
                if (__float_as_int(zg.z) == gk) {
                    gr.x = 0.0f;
                    gi.x = 1.0f;
                }
                if (__float_as_int(zg.w) == gk) {
                    gr.y = 0.0f;
                    gi.y = 1.0f;
                }
            }
        }
        if (CIRC) {
            gl_r[CIRC ? l : 0] = gr;
            sr = __fadd2_rn(sr, gr);
            if (!LAP) {
                gl_i[CIRC ? l : 0] = gi;
                si = __fadd2_rn(si, gi);
            }
            continue;
        }
        const float2 k0 = make_float2(R[l][0], R[l][0]), k1 = make_float2(R[l][1], R[l][1]),
                     k2 = make_float2(R[l][2], R[l][2]);
        o.t0r = __ffma2_rn(gr, k0, o.t0r);
        o.t1r = __ffma2_rn(gr, k1, o.t1r);
        o.t2r = __ffma2_rn(gr, k2, o.t2r);
        if (!LAP) {
            o.t0i = __ffma2_rn(gi, k0, o.t0i);
            o.t1i = __ffma2_rn(gi, k1, o.t1i);
            o.t2i = __ffma2_rn(gi, k2, o.t2i);
        }
    }
    if (CIRC) {
        static_assert(!CIRC || Q == 3, "one point per vertex");
        const float2 cb = __fmul2_rn(ar, make_float2(R[0][1], R[0][1]));                    // area beta
        const float2 ca = __fmul2_rn(ar, make_float2(R[0][0] - R[0][1], R[0][0] - R[0][1]));  // area (alpha - beta)
        const float2 br = __fmul2_rn(cb, sr);
        o.t0r = __ffma2_rn(ca, gl_r[0], br);
        o.t1r = __ffma2_rn(ca, gl_r[CIRC ? 1 : 0], br);
        o.t2r = __ffma2_rn(ca, gl_r[CIRC ? 2 : 0], br);
        if (!LAP) {
            const float2 bi = __fmul2_rn(cb, si);
            o.t0i = __ffma2_rn(ca, gl_i[0], bi);
            o.t1i = __ffma2_rn(ca, gl_i[CIRC ? 1 : 0], bi);
            o.t2i = __ffma2_rn(ca, gl_i[CIRC ? 2 : 0], bi);
        }
        return o;
    }
    o.t0r = __fmul2_rn(o.t0r, ar);
    o.t1r = __fmul2_rn(o.t1r, ar);
    o.t2r = __fmul2_rn(o.t2r, ar);
    o.t0i = __fmul2_rn(o.t0i, ar);
    o.t1i = __fmul2_rn(o.t1i, ar);
    o.t2i = __fmul2_rn(o.t2i, ar);
    return o;
}

// Adds triangle (lane h of a pair) into the running sums, flushing the
// positions whose vertex changes.
__device__ __forceinline__ void pos_add(const PairSums &t, int h, uint32_t code, float2 *__restrict__ Hcol, int hld,
                                        PosSums &ps)
{
    if (code & (1u << 24)) {
        pos_flush(Hcol, hld, ps.c0, ps.a0);
        ps.c0 = (int)(code & 255u) - 1;
    }
    if (code & (1u << 25)) {
        pos_flush(Hcol, hld, ps.c1, ps.a1);
        ps.c1 = (int)((code >> 8) & 255u) - 1;
    }
    if (code & (1u << 26)) {
        pos_flush(Hcol, hld, ps.c2, ps.a2);
        ps.c2 = (int)((code >> 16) & 255u) - 1;
    }
    ps.a0.x += h ? t.t0r.y : t.t0r.x;
    ps.a0.y += h ? t.t0i.y : t.t0i.x;
    ps.a1.x += h ? t.t1r.y : t.t1r.x;
    ps.a1.y += h ? t.t1i.y : t.t1i.x;
    ps.a2.x += h ? t.t2r.y : t.t2r.x;
    ps.a2.y += h ? t.t2i.y : t.t2i.x;
}

#ifndef GYPS_TILE_UNROLL
#define GYPS_TILE_UNROLL 4
#endif
#ifndef GYPS_TILE_MINB
#define GYPS_TILE_MINB 3
#endif
constexpr int kTileUnroll = GYPS_TILE_UNROLL;  // 4 or 8

// Source-side sums of one target point against the staged triangles, U at a
// time (U / 2 independent packed pairs; the count is padded to a multiple of U
// with far-away triangles of zero area), added into the running sums of the
// vertex positions in list order.
template <int Q, bool LAP, bool SELF, bool CIRC>
__device__ __forceinline__ void src_sums(const float4 *__restrict__ sxy, const float4 *__restrict__ szg,
                                         const int2 *__restrict__ stl, int nst, float4 tp, int gk,
                                         const float (&R)[Q][3], float2 *__restrict__ Hcol, PosSums &ps)
{
    constexpr int HLD = TileCfg<Q>::HLD;
    const float2 tx = make_float2(tp.x, tp.x), ty = make_float2(tp.y, tp.y), tz = make_float2(tp.z, tp.z);
    constexpr int U = kTileUnroll;  // source triangles per step
    for (int b = 0; b < nst; b += U) {
        // the kernel sums of U triangles first (branch-free), then the running sums in order
        PairSums pr[U / 2];
        int2 tl[U];
#pragma unroll
        for (int u = 0; u < U; ++u) tl[u] = stl[b + u];
#pragma unroll
        for (int u = 0; u < U / 2; ++u)
            pr[u] = pair_sums<Q, LAP, SELF, CIRC>(sxy, szg, (b >> 1) + u,
                                            make_float2(__int_as_float(tl[2 * u].y), __int_as_float(tl[2 * u + 1].y)),
                                            tx, ty, tz, gk, R);
#pragma unroll
        for (int u = 0; u < U; ++u) pos_add(pr[u >> 1], u & 1, (uint32_t)tl[u].x, Hcol, HLD, ps);
    }
}

template <int Q, bool LAP, bool CIRC, typename OutT>
__global__ void __launch_bounds__(128, GYPS_TILE_MINB) tile_block_kernel(const TileArgs a, OutT *out)
{
    using C = TileCfg<Q>;
    constexpr int NT = C::NT, HLD = C::HLD, VLD = kTileV + 1;
    extern __shared__ __align__(16) unsigned char smem[];
    float2 *H = reinterpret_cast<float2 *>(smem);
    // staged source points, pair-interleaved: triangles 2p, 2p + 1, point l ->
    // sxy[p Q + l] = (x0, x1, y0, y1), szg[p Q + l] = (z0, z1, id0, id1)
    float4 *sxy = reinterpret_cast<float4 *>(smem + C::H_BYTES);
    float4 *szg = sxy + (C::SRC / 2) * Q;
    int2 *stl = reinterpret_cast<int2 *>(szg + (C::SRC / 2) * Q);
    uint16_t *lst = reinterpret_cast<uint16_t *>(smem + C::H_BYTES + C::S_BYTES);
    int *cnt = reinterpret_cast<int *>(lst + kTileV * C::LCAP);
    int2 *ttl = reinterpret_cast<int2 *>(smem + C::H_BYTES + C::S_BYTES + C::L_BYTES);
    float *tarea = reinterpret_cast<float *>(ttl + C::TPP);
    float *Rt = tarea + C::TPP;  // Rt[m][l]: R transposed, 3 x 8
    float2 *ctab = reinterpret_cast<float2 *>(smem + C::H_BYTES + C::S_BYTES + C::L_BYTES + C::C_OFF);  // [tt][m][l]
    const int tid = threadIdx.x;
    float R[Q][3];
#pragma unroll
    for (int l = 0; l < Q; ++l)
#pragma unroll
        for (int m = 0; m < 3; ++m) R[l][m] = a.R[3 * l + m];
    if (tid < 3 * Q) Rt[(tid % 3) * 8 + tid / 3] = a.R[tid];
    // the block accumulator in registers: column j = tid % 64, rows 32 h .. 32 h + 31 with h = tid / 64
    const int jcol = tid & (kTileV - 1), half = tid >> 6;
    float2 acc[32];

    // stages source triangles [t0, t0 + nst) (positions, codes)
    auto stage = [&](int64_t t0, int nst) {
        __syncthreads();  // the previous contents are consumed
        const int npad = (kTileUnroll - nst % kTileUnroll) % kTileUnroll;  // pad: far-away triangles of zero area
        for (int e = tid; e < (nst + npad) * Q; e += NT) {
            const int b = e / Q, l = e - b * Q, h = b & 1, o = (b >> 1) * Q + l;
            const float4 p = b < nst ? a.pos[t0 * Q + e] : make_float4(1e6f, 1e6f, 1e6f, __int_as_float(-2));
            float *xy = reinterpret_cast<float *>(&sxy[o]), *zg = reinterpret_cast<float *>(&szg[o]);
            xy[h] = p.x;
            xy[2 + h] = p.y;
            zg[h] = p.z;
            zg[2 + h] = p.w;
        }
        for (int e = tid; e < nst + npad; e += NT) stl[e] = e < nst ? a.tl[t0 + e] : make_int2(0, 0);
        __syncthreads();
    };

    for (int64_t it = blockIdx.x; it < a.n_items; it += gridDim.x) {
        const int4 item = a.items[it];
        const int I = item.x, J = item.y;
        const bool self = item.z & 1;
#pragma unroll
        for (int r = 0; r < 32; ++r) acc[r] = make_float2(0.f, 0.f);
        const int tI0 = a.tile_ptr[I], nTI = a.tile_ptr[I + 1] - tI0;
        const int tJ0 = a.tile_ptr[J], nTJ = a.tile_ptr[J + 1] - tJ0;
        const bool once = nTJ <= C::SRC;  // T(J) stays staged over all passes
        if (once) stage(tJ0, nTJ);
        for (int pb = 0; pb < nTI; pb += C::TPP) {
            const int ntp = min(C::TPP, nTI - pb);
            const bool active = tid < ntp * Q;
            float4 tp = make_float4(0.f, 0.f, 0.f, __int_as_float(-1));
            if (active) {
                const int tt = tid / Q, l = tid - tt * Q;
                tp = a.pos[(int64_t)(tI0 + pb) * Q + tid];
                tp.x = -tp.x;
                tp.y = -tp.y;
                tp.z = -tp.z;
                if (l == 0) {
                    const int2 tl = a.tl[tI0 + pb + tt];
                    ttl[tt] = tl;
                    tarea[tt] = __int_as_float(tl.y);
                }
            }
            if (tid < kTileV) cnt[tid] = 0;
            const int gk = __float_as_int(tp.w);
            if (tid < HLD) {
#pragma unroll 8
                for (int j = 0; j < kTileV; ++j) H[j * HLD + tid] = make_float2(0.f, 0.f);
            }
            PosSums ps;
            ps.a0 = ps.a1 = ps.a2 = make_float2(0.f, 0.f);
            ps.c0 = ps.c1 = ps.c2 = -1;
            for (int sb = 0; sb < nTJ; sb += C::SRC) {
                const int nst = min(C::SRC, nTJ - sb);
                if (!once) stage(tJ0 + sb, nst);
                if (active) {
                    if (self)
                        src_sums<Q, LAP, true, CIRC>(sxy, szg, stl, nst, tp, gk, R, H + tid, ps);
                    else
                        src_sums<Q, LAP, false, CIRC>(sxy, szg, stl, nst, tp, gk, R, H + tid, ps);
                }
            }
            if (active) {
                pos_flush(H + tid, HLD, ps.c0, ps.a0);
                pos_flush(H + tid, HLD, ps.c1, ps.a1);
                pos_flush(H + tid, HLD, ps.c2, ps.a2);
            }
            __syncthreads();  // ttl, tarea and cnt are visible
            // per test slot, the (target triangle, position) entries of this pass
            for (int q3 = tid; q3 < 3 * ntp; q3 += NT) {
                const int tt = q3 / 3, m = q3 - 3 * tt;
                const int sl = (int)(((uint32_t)ttl[tt].x >> (8 * m)) & 255u) - 1;
                if (sl >= 0) {
                    const int e = atomicAdd(&cnt[sl], 1);
                    if (e < C::LCAP) lst[sl * C::LCAP + e] = (uint16_t)((tt << 2) | m);
                }
            }
            for (int c3 = tid; c3 < 3 * Q * ntp; c3 += NT) {
                const int tt = c3 / (3 * Q), rem = c3 - tt * 3 * Q, m = rem / Q, l = rem - m * Q;
                const float c = tarea[tt] * Rt[m * 8 + l];
                ctab[c3] = make_float2(c, c);
            }
            __syncthreads();  // H, the lists and the coefficients complete
            // Vacc[32 half + r][jcol] += sum over the slot's entries (triangle t, position m) of
            // area_t sum_l R[l][m] H[jcol][t Q + l]
            const float2 *Hrow = H + jcol * HLD;
#pragma unroll
            for (int r = 0; r < 32; ++r) {
                const int sl = 32 * half + r;
                const int n = min(cnt[sl], C::LCAP);
                for (int e = 0; e < n; ++e) {
                    const int code = lst[sl * C::LCAP + e];
                    const int tt = code >> 2, m = code & 3;
                    const float2 *hp = Hrow + tt * Q, *cp = ctab + (tt * 3 + m) * Q;
#pragma unroll
                    for (int l = 0; l < Q; ++l) acc[r] = __ffma2_rn(cp[l], hp[l], acc[r]);
                }
            }
            __syncthreads();  // before the next pass refills H, ttl, tarea, cnt
        }
        // the block through shared memory (H's space): rows of tile I, columns of tile J
        float2 *Vs = H;
#pragma unroll
        for (int r = 0; r < 32; ++r) Vs[(32 * half + r) * VLD + jcol] = acc[r];
        __syncthreads();
        const int32_t *rI = a.rowmap + (int64_t)I * kTileV, *rJ = a.rowmap + (int64_t)J * kTileV;
        const int32_t *cI = a.colmap + (int64_t)I * kTileV, *cJ = a.colmap + (int64_t)J * kTileV;
        OutT *blk = out + (a.item_off ? a.item_off[it] : 0);
        const int64_t ld = a.ld > 0 ? a.ld : (int64_t)item.w;
        for (int e = tid; e < kTileV * kTileV; e += NT) {
            const int i = e % kTileV, j = e / kTileV;  // rows fastest
            const int32_t r = rI[i], c = cJ[j];
            if (r >= 0 && c >= 0) blk[r + (int64_t)c * ld] = to_out<OutT>(Vs[i * VLD + j], a.scale);
        }
        if ((item.z & 2) && I != J) {
            for (int e = tid; e < kTileV * kTileV; e += NT) {
                const int j = e % kTileV, i = e / kTileV;
                const int32_t r = rJ[j], c = cI[i];
                if (r >= 0 && c >= 0) blk[r + (int64_t)c * ld] = to_out<OutT>(Vs[i * VLD + j], a.scale);
            }
        }
        __syncthreads();  // Vs is read before the next item's first pass clears H
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
    {
        // a slot collects at most one entry per incident triangle and pass
        std::vector<int32_t> deg(m->nv, 0);
        for (int32_t v : tri) ++deg[v];
        const int32_t dmax = *std::max_element(deg.begin(), deg.end());
        if (dmax > TileCfg<3>::LCAP)
            return set_error(GYPS_ERR_UNSUPPORTED, "FP32 tile assembly: a vertex has " + std::to_string(dmax) +
                                                       " triangles (at most 16)");
    }
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
    if (st == GYPS_OK) st = up(&T->d_perm, T->perm);
    if (st == GYPS_OK) st = up(&T->d_rowmap, T->rowmap);
    if (st == GYPS_OK) st = up(&T->d_items, T->items);
    if (st == GYPS_OK) {
        const size_t bytes = (size_t)T->ntt * m->q * sizeof(float4) + (size_t)T->ntt * sizeof(int2);
        if (cudaMalloc((void **)&T->d_pos, bytes) != cudaSuccess) st = set_error(GYPS_ERR_OOM, "tile panel");
        else {
            T->d_tl = reinterpret_cast<int2 *>(T->d_pos + T->ntt * m->q);
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
    void *ptrs[] = {T->d_tile_ptr, T->d_tri, T->d_loc, T->d_perm, T->d_rowmap, T->d_items, T->d_pos};
    for (void *p : ptrs)
        if (p) cudaFree(p);
    delete T;
}

gyps_status tile_panel(Mesh *m, double k, cudaStream_t s)
{
    VertexTiles *T = m->vt;
    const float ks = k > 0.0 ? (float)k : 1.0f;
    const int64_t n = T->ntt * m->q;
    PointPerm pp{};
    for (int p = 0; p < 6; ++p)
        for (int l = 0; l < m->q; ++l) {
            // the point whose barycentric coordinates, read in the turned vertex order, are those of point l
            int best = 0;
            double bd = 1e300;
            for (int l2 = 0; l2 < m->q; ++l2) {
                double d = 0.0;
                for (int c = 0; c < 3; ++c) d += std::fabs(m->rule.bary[3 * l2 + kPerm[p][c]] - m->rule.bary[3 * l + c]);
                if (d < bd) {
                    bd = d;
                    best = l2;
                }
            }
            if (bd > 1e-12) return set_error(GYPS_ERR_INVALID, "quadrature rule is not symmetric under vertex orders");
            pp.sigma[p][l] = (int8_t)best;
        }
    tile_panel_kernel<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(T->d_tri, T->d_loc, T->d_perm, T->ntt, m->d_pts64,
                                                                 m->rule, pp, ks, T->d_pos, T->d_tl);
    GYPS_CUDA(cudaGetLastError());
    return GYPS_OK;
}

template <int Q, bool LAP, typename OutT>
static gyps_status launch_blocks_q(Mesh *m, const TileArgs &a, OutT *out, cudaStream_t s)
{
    using C = TileCfg<Q>;
    // the 3-point rule: R[l][m] = beta + (alpha - beta) [l == m]
    bool circ = Q == 3;
    for (int l = 0; l < Q && circ; ++l)
        for (int c = 0; c < 3; ++c) circ = circ && a.R[3 * l + c] == (l == c ? a.R[0] : a.R[1]);
    auto kern = circ ? tile_block_kernel<Q, LAP, Q == 3, OutT> : tile_block_kernel<Q, LAP, false, OutT>;
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
    a.tl = T->d_tl;
    for (int l = 0; l < m->q; ++l)
        for (int c = 0; c < 3; ++c) a.R[3 * l + c] = (float)(m->rule.w[l] * m->rule.bary[3 * l + c]);
    a.tile_ptr = T->d_tile_ptr;
    a.rowmap = T->d_rowmap;
    a.colmap = T->d_rowmap;
    a.items = T->d_items;
    a.item_off = nullptr;
    a.n_items = (int64_t)T->items.size();
    a.ld = m->nv;
    a.scale = (k > 0.0 ? k : 1.0) / (4.0 * 3.14159265358979323846);
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
