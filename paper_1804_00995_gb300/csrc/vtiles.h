// Vertex tiles of a mesh and the tile-pair kernel that produces dense blocks of
// the single layer's Gauss-Gauss part (Sec. 5, Eq. (BEM)); used by the dense
// assembly and by the compressed far field.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <vector>

#include "internal.h"

namespace gyps {

constexpr int kTileV = 64;  // vertices per tile

// Vertices in Morton order, cut into tiles of kTileV.  Tile I's triangle list
// T(I) holds every triangle with a vertex in the tile (a triangle whose vertices
// fall into several tiles appears in each), with the tile slots of its vertices
// packed one byte each (slot + 1, 0 = vertex outside the tile).
struct VertexTiles {
    int64_t ntiles = 0;
    int64_t ntt = 0;      // tile-triangles (sum of |T(I)|)
    int64_t max_tri = 0;  // largest |T(I)|
    std::vector<int64_t> tile_ptr;  // ntiles + 1
    std::vector<int32_t> tri;       // ntt: triangle id
    std::vector<int32_t> loc;       // ntt: packed slots of the turned vertex positions, flush bits in byte 3
    std::vector<int8_t> perm;       // ntt: the turn (vertex order 0..5) of each tile-triangle
    std::vector<int32_t> rowmap;    // ntiles x kTileV: vertex id of each slot, -1 = empty
    std::vector<int4> items;        // (I, J, shares-a-triangle | write-transposed, 0) for I <= J
    std::vector<uint64_t> adjacent; // tile pairs (I << 32 | J, I <= J) whose T(I), T(J) share a triangle
    // device copies
    int32_t *d_tile_ptr = nullptr, *d_tri = nullptr, *d_loc = nullptr, *d_rowmap = nullptr;
    int8_t *d_perm = nullptr;
    int4 *d_items = nullptr;
    float4 *d_pos = nullptr;  // ntt x q: point scaled by k and negated, its global index in .w (bits)
    int2 *d_tl = nullptr;     // ntt: (packed slots and flush bits, triangle area as bits)
};

// Arguments of the tile-pair kernel.  An item is (I, J, flags, ld_item): flags
// bit 0 = T(I) and T(J) share a triangle (the same point on both sides), bit 1 =
// also write the transposed block (for I != J).  Output entry (row slot i of
// tile I, column slot j of tile J) of item n goes to
// out[item_off[n] + rowmap[I][i] + colmap[J][j] * ld], ld = `ld` if > 0 else
// ld_item; the transposed entry to out[item_off[n] + rowmap[J][j] + colmap[I][i] * ld].
// Slots mapped to -1 are skipped.  Values are multiplied by `scale`.
struct TileArgs {
    const float4 *pos;
    const int2 *tl;
    float R[21];  // R[l][m] = reference weight of point l x lambda_m(l)
    const int32_t *tile_ptr;
    const int32_t *rowmap;
    const int32_t *colmap;
    const int4 *items;
    const int64_t *item_off;  // nullptr: 0 for every item
    int64_t n_items;
    int64_t ld;
    double scale;
};

// tri_cap: largest |T(I)| (a tile closes before its triangle list grows past it)
// Point order of a symmetric rule after a turn p of the vertices: sigma[p][l].
struct PointPerm {
    int8_t sigma[6][7];
};

void order_tile_triangles(VertexTiles &T);
void build_vertex_tiles(const std::vector<double> &vtx, const std::vector<int32_t> &tri, int64_t nv, int64_t nt,
                        int64_t tri_cap, VertexTiles *out);
int64_t tile_tri_cap(int q);
gyps_status vertex_tiles_prepare(Mesh *m, cudaStream_t s);
void free_vertex_tiles(VertexTiles *T);
// k-dependent panel (scaled positions) of every tile-triangle point
gyps_status tile_panel(Mesh *m, double k, cudaStream_t s);
TileArgs tile_args(const Mesh *m, double k);
template <typename OutT>
gyps_status tile_blocks(Mesh *m, double k, const TileArgs &a, OutT *out, cudaStream_t s);

}  // namespace gyps
