// Internal declarations of libgyps: mesh handle, error plumbing, kernel launchers.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "gyps.h"

namespace gyps {

// ---------------------------------------------------------------- errors
gyps_status set_error(gyps_status code, const std::string &msg);
gyps_status cuda_error(cudaError_t e, const char *what);

#define GYPS_CUDA(call)                                              \
    do {                                                             \
        cudaError_t e_ = (call);                                     \
        if (e_ != cudaSuccess) return ::gyps::cuda_error(e_, #call); \
    } while (0)

#define GYPS_TRY(call)                          \
    do {                                        \
        gyps_status s_ = (call);                \
        if (s_ != GYPS_OK) return s_;           \
    } while (0)

// ---------------------------------------------------------------- layout
// Source panels of the FP32 far kernel are cut into tiles of kSrcTile points.
// Inside a tile, points are taken in pairs (2p, 2p+1) so that one packed
// f32x2 instruction handles both; a tile of the position panel holds
//   float4 XY[P] = (-x0, -x1, -y0, -y1), float2 Z[P] = (-z0, -z1),   P = kSrcTile/2,
// and a tile of the density panel for R right-hand sides holds
//   float4 U[P][R] = (re0, re1, im0, im1), float2 N[P][R] = (-im0, -im1).
// Padding points sit far away with zero density.
constexpr int kSrcTile = 256;
constexpr int kSrcPairs = kSrcTile / 2;
constexpr int kPosTileFloats = kSrcPairs * 6;
__host__ __device__ constexpr int64_t den_tile_floats(int R) { return (int64_t)kSrcPairs * 6 * R; }

// Reference quadrature rule (barycentric points, weights summing to 1), passed
// to kernels by value.
struct Rule {
    int q;
    double bary[21];
    double w[7];
};

// ---------------------------------------------------------------- mesh
struct VertexTiles;  // vtiles.h
void free_vertex_tiles(VertexTiles *T);

struct Mesh {
    int device = 0;
    int64_t nv = 0, nt = 0, nq = 0;
    int q = 0;
    Rule rule{};
    int64_t nq_pad = 0;   // nq rounded up to kSrcTile
    int64_t n_src_tiles = 0;

    // geometry on the device
    double *d_vtx = nullptr;      // nv x 3
    int32_t *d_tri = nullptr;     // nt x 3
    double4_32a *d_pts64 = nullptr;   // nq: (x, y, z, w_k)
    float4 *d_pts32 = nullptr;    // nq: (x, y, z, w_k) rounded to FP32
    float *d_pos_panel = nullptr; // n_src_tiles * kPosTileFloats

    // vertex -> (triangle, local vertex) incidence, CSR over vertices
    int32_t *d_v2t_ptr = nullptr; // nv + 1
    int32_t *d_v2t = nullptr;     // 3 nt, entries 3*t + m

    // singular correction (Sec. 5.2)
    int64_t npairs = 0;
    int32_t *d_pair_a = nullptr, *d_pair_b = nullptr;  // sorted by a
    int32_t *d_pair_ptr = nullptr;                     // nt + 1, pairs of test triangle a
    std::vector<int32_t> h_pair_ptr;                   // host copy
    double *d_blocks = nullptr;                        // npairs x 9
    int64_t c_nnz = 0;
    int32_t *d_c_rowptr = nullptr;                     // nv + 1
    int32_t *d_c_col = nullptr;                        // c_nnz
    double *d_c_val = nullptr;                         // c_nnz
    int32_t *d_c_src_ptr = nullptr;                    // c_nnz + 1
    int32_t *d_c_src = nullptr;                        // 9 npairs: block entries per nonzero
    std::vector<int32_t> h_c_rowptr, h_c_col;          // host copy of the pattern

    // device error word (bounded waits that ran out set it)
    int *d_err = nullptr;

    // workspace grown on demand
    void *ws_den = nullptr; size_t ws_den_bytes = 0;   // density panel / FP64 densities
    void *ws_v = nullptr; size_t ws_v_bytes = 0;       // target accumulators
    void *ws_stage = nullptr; size_t ws_stage_bytes = 0;  // host<->device staging
    void *ws_bw = nullptr; size_t ws_bw_bytes = 0;        // K X of the combined operator
    void *ws_tc = nullptr; size_t ws_tc_bytes = 0;        // tensor-core source panel
    void *ws_pts = nullptr; size_t ws_pts_bytes = 0;      // potential at points: point copies, far sums, staging
    double4_32a *d_tri_cen = nullptr;                     // per triangle: centroid, (2 x largest centroid-vertex distance)^2
    float4 *d_tri_cen32 = nullptr;                        // the same in FP32, radius widened (candidate test)
    double4_32a *d_tri_nrm = nullptr;                     // double layer: unit normal per triangle
    double *d_cdl_val = nullptr;                          // double layer: correction values on C's pattern
    double *d_cdlT_val = nullptr;                         // adjoint double layer: the transposed values
    float *d_nrm_panel = nullptr;                         // double layer: FP32 normals, position-panel layout
    // EFIE: RWG functions, one per edge (built on first use)
    int64_t ne = 0;
    int32_t *d_tedge = nullptr;                           // nt x 3: (edge << 1) | (minus triangle)
    int32_t *d_etri = nullptr;                            // ne x 2: 3 t + j of the plus and the minus triangle
    double *d_efie_blocks = nullptr;                      // npairs x 18: the two 3 x 3 correction blocks
    double *d_mfie_blocks = nullptr;                      // npairs x 9: the MFIE's 3 x 3 correction blocks
    std::vector<int32_t> h_edges;                         // ne x 2 vertex pairs (a < b)
    float pad = 0.0f;                                     // distance of padding points
    // mesh graph for the learned preconditioner (built on first use)
    int32_t *d_adj_ptr = nullptr, *d_adj = nullptr;       // vertex neighbours over mesh edges
    float *d_vfeat = nullptr;                             // nv x 6: centred coordinates, unit normal
    double h_mean = 0.0;                                  // mean edge length
    double radius = 0.0;                                  // largest vertex distance from the vertex centroid
    VertexTiles *vt = nullptr;                            // vertex tiles of the dense blocks (built on first use)
    int64_t device_bytes = 0;
    int num_sms = 0;

    // optional per-stage device timing of applies (gyps_profile_*)
    struct ProfRec {
        cudaEvent_t a, b;
        int stage;
        int launches;
    };
    bool prof = false;
    std::vector<ProfRec> prof_pending;
    double prof_ms[4] = {0, 0, 0, 0};
    int64_t prof_launches[4] = {0, 0, 0, 0};
    int64_t prof_applies = 0;
};

// Records CUDA events around one stage of an apply when profiling is on.
struct StageTimer {
    Mesh *m;
    cudaStream_t s;
    int stage;
    cudaEvent_t a = nullptr;
    StageTimer(Mesh *m_, cudaStream_t s_, int stage_) : m(m_), s(s_), stage(stage_)
    {
        if (m->prof && cudaEventCreate(&a) == cudaSuccess) cudaEventRecord(a, s);
    }
    void done(int launches)
    {
        if (!a) return;
        cudaEvent_t b;
        if (cudaEventCreate(&b) != cudaSuccess) return;
        cudaEventRecord(b, s);
        m->prof_pending.push_back({a, b, stage, launches});
        a = nullptr;
    }
};

gyps_status grow(Mesh *m, void **buf, size_t *cap, size_t need);
gyps_status check_mesh(gyps_mesh_t h, Mesh **out);
gyps_status enter_device(const Mesh *m);
bool is_device_pointer(const void *p);
// Reads (and clears) the error word of bounded device waits; TIMEOUT if set.
gyps_status check_err_word(Mesh *m, cudaStream_t s);
// Clears the error word on the stream, so that a synchronous call reports only
// the waits of its own launches.
gyps_status clear_err_word(Mesh *m, cudaStream_t s);
// Poll limit of the pipeline waits in the far kernels launched from now on
// (gyps_set_wait_polls; negative = each kernel's default).
int wait_polls_setting();

// ---------------------------------------------------------------- launchers
// a1: quadrature points and the FP32 position panel
cudaError_t launch_quad_points(const Mesh &m, cudaStream_t s);
// a5b: correction blocks and their CSR gather
cudaError_t launch_near_build(const Mesh &m, cudaStream_t s);

// a2-a5: one matrix-free apply with device pointers
gyps_status apply_device(Mesh *m, double k, int nrhs, const double2 *X, int64_t ldx, double2 *Y, int64_t ldy,
                         int prec, uint32_t flags, int64_t tri_begin, int64_t tri_end, cudaStream_t s);
gyps_status run_far_df(Mesh *m, double k, const double4_32a *tgt, bool self, const double2 *u64, int64_t ldu, int c0,
                       int w, double2 *v, int64_t ldv, int64_t t_begin, int64_t t_end, cudaStream_t s);
gyps_status run_far_dl_df(Mesh *m, double k, bool adj, const double2 *u64, int64_t ldu, int c0, int w, double2 *v,
                          int64_t ldv, cudaStream_t s);
// Far part of the potential at npts points (tgt32 / tgt64: the points): v[i, c] = sum_l G(x_i, y_l) u_l,c
// with u = W Phi X, no self pairs; prec FP32 | FP64 | DF64; v: npts x nrhs, ld ldv, overwritten.
gyps_status far_points(Mesh *m, double k, const double2 *X, int64_t ldx, int nrhs, const float4 *tgt32,
                       const double4_32a *tgt64, int64_t npts, double2 *v, int64_t ldv, int prec, cudaStream_t s);
gyps_status far_tc(Mesh *m, double k, const double2 *X, int64_t ldx, int nrhs, double2 *v, int64_t ldv,
                   int64_t t_begin, int64_t t_end, cudaStream_t s);
cudaError_t launch_near_spmv(const Mesh &m, int nrhs, const double2 *X, int64_t ldx, double2 *Y, int64_t ldy,
                             cudaStream_t s);

// Far sums over all quadrature points as targets from densities prepared by the caller:
// an FP32 panel of R = 1, 2, 4 or 8 columns (added into v), or FP64 columns [c0, c0 + w), w <= 4.
gyps_status far32_panel(Mesh *m, double k, const float *panel, int R, double2 *v, int64_t ldv, cudaStream_t s);
gyps_status far64_cols(Mesh *m, double k, const double2 *u64, int64_t ldu, int c0, int w, double2 *v, int64_t ldv,
                       cudaStream_t s);
// EFIE with RWG functions: topology and correction (once per mesh; INVALID for an open or
// inconsistently oriented mesh) and Y = sign T X (device pointers, ne x nrhs)
gyps_status efie_prepare(Mesh *m, cudaStream_t s);
gyps_status efie_apply_device(Mesh *m, double k, double sign, int nrhs, const double2 *X, int64_t ldx, double2 *Y,
                              int64_t ldy, int prec, cudaStream_t s);
// Y = sign (-beta T + (1 - beta)(Id/2 - nxK)) X, the electromagnetic listing's LHS (ne x nrhs)
gyps_status emcfie_apply_device(Mesh *m, double k, double beta, double sign, int nrhs, const double2 *X, int64_t ldx,
                                double2 *Y, int64_t ldy, int prec, cudaStream_t s);

// a2 in FP32: the density panel of columns c0 .. c0+w-1 (w = 1, 2, 4 or 8)
cudaError_t launch_interp32(const Mesh *m, const double2 *X, int64_t ldx, int c0, int w, float *panel, cudaStream_t s);

// Double layer Y = K X (adj: K' X) and the combined operators Y = (1/2 M + K - i eta V) X,
// (1/2 M + K' - i eta V) X (device pointers)
gyps_status dl_apply_device(Mesh *m, double k, int nrhs, const double2 *X, int64_t ldx, double2 *Y, int64_t ldy,
                            int prec, bool adj, cudaStream_t s);
gyps_status combined_apply_device(Mesh *m, double k, double eta, bool adj, int nrhs, const double2 *X, int64_t ldx,
                                  double2 *Y, int64_t ldy, int prec, cudaStream_t s);

// a6, a7
gyps_status assemble_device(Mesh *m, double k, int prec, double2 *V, int64_t ldv, cudaStream_t s);
// a6 with FP32 kernel values by vertex-tile blocks (the Gauss-Gauss part only; C is added by the caller)
gyps_status assemble_tiles(Mesh *m, double k, double2 *V, int64_t ldv, cudaStream_t s);
// F = int phi (exp(ik d.x)), or with cfie: int phi (d/dn - i eta) exp(ik d.x)
gyps_status rhs_device(Mesh *m, double k, int nrhs, const double *dirs_host, double2 *F, int64_t ldf,
                       cudaStream_t s, bool cfie = false, double eta = 0.0);

// a11: whether the mesh's electrical size k x radius lies in the range the network was trained on
// (widened by 25 %; an untrained network has no range and is always in range)
gyps_status precond_in_range(gyps_precond_t p, Mesh *m, double k, cudaStream_t s, bool *in_range);
// a11: learned preconditioner Z = M(R) (device pointers)
gyps_status precond_apply_device(gyps_precond_t p, Mesh *m, double k, int nrhs, const double2 *R, int64_t ldr,
                                 double2 *Z, int64_t ldz, cudaStream_t s);

// NEXT-4: the compressed far field (hmat.cu); Y = (H + C) X with device pointers
struct Hmat;
Hmat *hmat_of(gyps_hmat_t h);
const Mesh *hmat_mesh(const Hmat *h);
double hmat_k(const Hmat *h);
gyps_status hmat_apply_device(Hmat *h, int nrhs, const double2 *X, int64_t ldx, double2 *Y, int64_t ldy,
                              cudaStream_t s);

// a8
gyps_status gmres_device(Mesh *m, double k, int nrhs, const double2 *F, int64_t ldf, double2 *X, int64_t ldx,
                         const gyps_gmres_opts &o, gyps_gmres_report *rep, cudaStream_t s);

}  // namespace gyps
