// Batched apply: many meshes of uneven size, each with nrhs right-hand sides,
// in one interpolation launch, ONE persistent far-kernel launch and one
// projection launch, captured once into a CUDA graph.  The dense products of
// all meshes form a single work list of (mesh, RHS chunk, target tile, source
// tile) items of equal cost, split evenly over the persistent grid, so meshes
// of very different sizes share the GPU without a separate schedule.  The
// RHS chunk width R and targets per thread T are picked by an autotuner
// (timed candidates, cached in a JSON file).
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <fstream>
#include <mutex>
#include <sstream>
#include <string>
#include <vector>

#include <sys/stat.h>

#include "far_tile.cuh"
#include "internal.h"

namespace gyps {

// One (mesh, RHS chunk) of the batch, as the far kernel sees it.
struct FarSeg {
    const float *pos_panel;
    const float *den_panel;
    const float4 *tgt;
    double2 *v;        // accumulators of this chunk's first column
    int64_t ldv;       // = nq of the mesh
    int64_t nq;
    int64_t n_src_tiles, n_tgt_tiles;
    int64_t item_begin;  // first global work item of this segment
    float ks;
    int lap;
};

// One (mesh, RHS chunk) as the interpolation sees it.
struct InterpSeg {
    const int32_t *tri;
    const double4_32a *pts64;
    Rule rule;
    int64_t nq, nq_pad;
    int64_t src_begin;  // first flattened (padded) source index
    const double2 *X;
    int64_t ldx;
    int c0;
    float *den_panel;
};

// One mesh as the projection sees it.
struct ProjMesh {
    int64_t nv, v_begin;
    const int32_t *v2t_ptr, *v2t;
    const double4_32a *pts64;
    Rule rule;
    const double2 *v;
    int64_t ldv;
    const int32_t *c_rowptr, *c_col;
    const double *c_val;
    const double2 *X;
    int64_t ldx;
    double2 *Y;
    int64_t ldy;
};

template <class S, class F>
__device__ __forceinline__ int find_seg(const S *segs, int n, int64_t idx, F key)
{
    int lo = 0, hi = n - 1;
    while (lo < hi) {
        int mid = (lo + hi + 1) >> 1;
        if (key(segs[mid]) <= idx)
            lo = mid;
        else
            hi = mid - 1;
    }
    return lo;
}

template <int R>
__global__ void batch_interp_kernel(const InterpSeg *segs, int nseg, int64_t total)
{
    const int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= total) return;
    const int si = find_seg(segs, nseg, g, [](const InterpSeg &s) { return s.src_begin; });
    const InterpSeg &sg = segs[si];
    const int64_t l = g - sg.src_begin;
    const int64_t tile = l / kSrcTile;
    const int p = (int)(l % kSrcTile) >> 1, lane = (int)(l & 1);
    float *base = sg.den_panel + tile * den_tile_floats(R);
#pragma unroll
    for (int j = 0; j < R; ++j) {
        double ur = 0.0, ui = 0.0;
        if (l < sg.nq) {
            const int64_t t = l / sg.rule.q;
            const int kq = (int)(l - t * sg.rule.q);
            const double w = sg.pts64[l].w;
            const double2 *xc = sg.X + (int64_t)(sg.c0 + j) * sg.ldx;
#pragma unroll
            for (int m = 0; m < 3; ++m) {
                double2 xv = xc[sg.tri[3 * t + m]];
                double lam = sg.rule.bary[3 * kq + m];
                ur += lam * xv.x;
                ui += lam * xv.y;
            }
            ur *= w;
            ui *= w;
        }
        float *u4 = base + 4 * ((int64_t)p * R + j);
        u4[lane] = (float)ur;
        u4[2 + lane] = (float)ui;
        base[4 * kSrcPairs * R + 2 * ((int64_t)p * R + j) + lane] = -(float)ui;
    }
}

// Persistent far kernel over the batch's global work list.
template <int R, int T>
__global__ void __launch_bounds__(FarCfg<R, T>::NT) far32_batch_kernel(const FarSeg *segs, int nseg,
                                                                          int64_t items, int *err)
{
    using C = FarCfg<R, T>;
    extern __shared__ __align__(128) unsigned char smem[];
    uint64_t *bars = reinterpret_cast<uint64_t *>(smem + C::STAGES * C::STAGE_BYTES);
    const int tid_x = threadIdx.x;
    const int64_t beg = items * blockIdx.x / gridDim.x;
    const int64_t end = items * (blockIdx.x + 1) / gridDim.x;
    if (beg >= end) return;
    auto seg_of = [&](int64_t it) { return find_seg(segs, nseg, it, [](const FarSeg &s) { return s.item_begin; }); };

    if (tid_x == 0) {
        for (int s = 0; s < C::STAGES; ++s) mbar_init(smem_addr(&bars[s]), 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();

    auto issue = [&](int64_t item) {
        const FarSeg &sg = segs[seg_of(item)];
        const int64_t local = item - sg.item_begin;
        const int64_t st = local % sg.n_src_tiles;
        const int s = (int)((item - beg) % C::STAGES);
        const uint32_t bar = smem_addr(&bars[s]);
        const uint32_t dst = smem_addr(smem + s * C::STAGE_BYTES);
        mbar_expect_tx(bar, C::STAGE_BYTES);
        bulk_g2s(dst, sg.pos_panel + st * kPosTileFloats, C::POS_BYTES, bar);
        bulk_g2s(dst + C::POS_BYTES, sg.den_panel + st * den_tile_floats(R), C::DEN_BYTES, bar);
    };
    int64_t issued = beg;
    if (tid_x == 0)
        for (; issued < end && issued < beg + C::STAGES - 1; ++issued) issue(issued);

    float2 tx[T], ty[T], tz[T];
    int64_t tid[T];
    float2 are[T][R], aim[T][R];
    float hre[T][R], lre[T][R], him[T][R], lim[T][R];
    int cur_seg = -1;
    int64_t cur_tt = -1;

    auto flush = [&]() {
        const FarSeg &sg = segs[cur_seg];
#pragma unroll
        for (int t = 0; t < T; ++t) {
            if (tid[t] < sg.nq) {
#pragma unroll
                for (int j = 0; j < R; ++j) {
                    double *dst = reinterpret_cast<double *>(sg.v + tid[t] + j * sg.ldv);
                    atomicAdd(dst, ((double)hre[t][j] + (double)lre[t][j]) * sg.ks);
                    atomicAdd(dst + 1, ((double)him[t][j] + (double)lim[t][j]) * sg.ks);
                }
            }
        }
    };

    bool failed = false;
    int64_t i = beg;
    int si = seg_of(beg);
    for (; i < end; ++i) {
        if (tid_x == 0 && issued < end && issued == i + C::STAGES - 1) {
            issue(issued);
            ++issued;
        }
        while (si + 1 < nseg && segs[si + 1].item_begin <= i) ++si;
        const FarSeg &sg = segs[si];
        const int64_t local = i - sg.item_begin;
        const int64_t tt = local / sg.n_src_tiles, st = local % sg.n_src_tiles;
        const int64_t tb = tt * C::TT;
        const int64_t te = min(tb + (int64_t)C::TT, sg.nq);
        if (si != cur_seg || tt != cur_tt) {
            if (cur_seg >= 0) flush();
            const float sc = sg.lap ? 1.0f : sg.ks;
#pragma unroll
            for (int t = 0; t < T; ++t) {
                int64_t g = tb + tid_x + t * C::NT;
                tid[t] = g;
                float4 p = sg.tgt[min(g, sg.nq - 1)];
                tx[t] = make_float2(p.x * sc, p.x * sc);
                ty[t] = make_float2(p.y * sc, p.y * sc);
                tz[t] = make_float2(p.z * sc, p.z * sc);
#pragma unroll
                for (int j = 0; j < R; ++j) hre[t][j] = lre[t][j] = him[t][j] = lim[t][j] = 0.0f;
            }
            cur_seg = si;
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
            const bool diag = tb < src0 + kSrcTile && src0 < te;
            if (sg.lap) {
                if (diag)
                    far_tile<R, T, true, true>(sp, tx, ty, tz, tid, src0, 1.0f, are, aim);
                else
                    far_tile<R, T, true, false>(sp, tx, ty, tz, tid, src0, 1.0f, are, aim);
            } else {
                if (diag)
                    far_tile<R, T, false, true>(sp, tx, ty, tz, tid, src0, sg.ks, are, aim);
                else
                    far_tile<R, T, false, false>(sp, tx, ty, tz, tid, src0, sg.ks, are, aim);
            }
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
        if (tid_x == 0) {
            atomicExch(err, 1);
            for (int64_t j = i; j < issued; ++j) {
                int s = (int)((j - beg) % C::STAGES);
                mbar_wait_bounded(smem_addr(&bars[s]), (uint32_t)(((j - beg) / C::STAGES) & 1));
            }
        }
        __syncthreads();
        return;
    }
    flush();
}

constexpr double kInv4PiB = 0.0795774715459476678844418816862571810;

__global__ void batch_project_kernel(const ProjMesh *ms, int nmesh, int64_t total)
{
    const int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int j = blockIdx.y;
    if (g >= total) return;
    const int mi = find_seg(ms, nmesh, g, [](const ProjMesh &m) { return m.v_begin; });
    const ProjMesh &m = ms[mi];
    const int64_t i = g - m.v_begin;
    const double2 *vc = m.v + (int64_t)j * m.ldv;
    double yr = 0.0, yi = 0.0;
    for (int32_t e = m.v2t_ptr[i]; e < m.v2t_ptr[i + 1]; ++e) {
        const int32_t te = m.v2t[e];
        const int64_t t = te / 3;
        const int mm = te - 3 * (int)t;
        for (int kq = 0; kq < m.rule.q; ++kq) {
            const int64_t kidx = t * m.rule.q + kq;
            const double c = m.pts64[kidx].w * m.rule.bary[3 * kq + mm];
            const double2 vv = vc[kidx];
            yr += c * vv.x;
            yi += c * vv.y;
        }
    }
    yr *= kInv4PiB;
    yi *= kInv4PiB;
    const double2 *xc = m.X + (int64_t)j * m.ldx;
    for (int32_t c = m.c_rowptr[i]; c < m.c_rowptr[i + 1]; ++c) {
        const double cv = m.c_val[c];
        const double2 xv = xc[m.c_col[c]];
        yr += cv * xv.x;
        yi += cv * xv.y;
    }
    m.Y[i + (int64_t)j * m.ldy] = make_double2(yr, yi);
}

// ---------------------------------------------------------------- plan
struct Batch {
    int device = 0;
    int nrhs = 0, R = 0, T = 0, nmesh = 0, nseg = 0;
    int grid = 0;
    int64_t items = 0, total_src = 0, total_v = 0;
    double pairs = 0.0;
    FarSeg *d_far = nullptr;
    InterpSeg *d_interp = nullptr;
    ProjMesh *d_proj = nullptr;
    float *d_den = nullptr;
    double2 *d_v = nullptr;
    size_t v_bytes = 0;
    int *d_err = nullptr;
    bool use_graph = false;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    int tuned = 0;  // 0 default, 1 measured now, 2 read from the cache
    std::vector<Mesh *> meshes;
    std::vector<gyps_batch_item> items_host;  // bound buffers (tensor-core mode applies per mesh)
    ~Batch()
    {
        if (exec) cudaGraphExecDestroy(exec);
        if (graph) cudaGraphDestroy(graph);
        cudaFree(d_far);
        cudaFree(d_interp);
        cudaFree(d_proj);
        cudaFree(d_den);
        cudaFree(d_v);
        cudaFree(d_err);
    }
};

template <int R, int T>
static gyps_status far_occupancy(int *occ)
{
    using C = FarCfg<R, T>;
    GYPS_CUDA(cudaFuncSetAttribute(far32_batch_kernel<R, T>, cudaFuncAttributeMaxDynamicSharedMemorySize, C::SMEM));
    GYPS_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(occ, far32_batch_kernel<R, T>, C::NT, C::SMEM));
    *occ = std::max(*occ, 1);
    return GYPS_OK;
}

static int tile_targets(int R, int T) { return 128 * T; }

static gyps_status enqueue(Batch *b, cudaStream_t s)
{
    if (b->R == 0) {  // tensor-core mode: the tensor-core apply of every mesh, in order
        for (size_t i = 0; i < b->meshes.size(); ++i) {
            const gyps_batch_item &it = b->items_host[i];
            GYPS_TRY(apply_device(b->meshes[i], it.k, b->nrhs, (const double2 *)it.X, it.ldx, (double2 *)it.Y, it.ldy,
                                  GYPS_PREC_TC_BF16X3, 0, 0, b->meshes[i]->nt, s));
        }
        return GYPS_OK;
    }
    GYPS_CUDA(cudaMemsetAsync(b->d_v, 0, b->v_bytes, s));
    const unsigned gi = (unsigned)((b->total_src + 255) / 256);
    switch (b->R) {
    case 8: batch_interp_kernel<8><<<gi, 256, 0, s>>>(b->d_interp, b->nseg, b->total_src); break;
    case 4: batch_interp_kernel<4><<<gi, 256, 0, s>>>(b->d_interp, b->nseg, b->total_src); break;
    case 2: batch_interp_kernel<2><<<gi, 256, 0, s>>>(b->d_interp, b->nseg, b->total_src); break;
    default: batch_interp_kernel<1><<<gi, 256, 0, s>>>(b->d_interp, b->nseg, b->total_src); break;
    }
    GYPS_CUDA(cudaGetLastError());
#define GYPS_FAR_CASE(RR, TT)                                                                                   \
    if (b->R == RR && b->T == TT)                                                                               \
        far32_batch_kernel<RR, TT><<<b->grid, FarCfg<RR, TT>::NT, FarCfg<RR, TT>::SMEM, s>>>(b->d_far, b->nseg, \
                                                                                              b->items, b->d_err);
    GYPS_FAR_CASE(8, 2)
    GYPS_FAR_CASE(4, 2)
    GYPS_FAR_CASE(4, 4)
    GYPS_FAR_CASE(2, 4)
    GYPS_FAR_CASE(1, 4)
#undef GYPS_FAR_CASE
    GYPS_CUDA(cudaGetLastError());
    dim3 gp((unsigned)((b->total_v + 127) / 128), (unsigned)b->nrhs);
    batch_project_kernel<<<gp, 128, 0, s>>>(b->d_proj, b->nmesh, b->total_v);
    GYPS_CUDA(cudaGetLastError());
    return GYPS_OK;
}

static gyps_status configure(Batch *b, const std::vector<gyps_batch_item> &items, int R, int T)
{
    b->R = R;
    b->T = T;
    b->items_host = items;
    if (R == 0) {  // tensor-core mode: per-mesh workspaces live in the meshes
        b->pairs = 0.0;
        b->items = 0;
        for (auto *m : b->meshes) {
            b->pairs += (double)m->nq * (double)m->nq;
            b->items += ((m->nq + 127) / 128) * ((m->nq + 4095) / 4096);
        }
        b->grid = 0;
        return GYPS_OK;
    }
    const int tt = tile_targets(R, T);
    const int nchunk = b->nrhs / R;
    std::vector<FarSeg> fs;
    std::vector<InterpSeg> is;
    std::vector<ProjMesh> pm;
    size_t den_floats = 0, v_elems = 0;
    for (auto *m : b->meshes) {
        den_floats += (size_t)nchunk * m->n_src_tiles * den_tile_floats(R);
        v_elems += (size_t)m->nq * b->nrhs;
    }
    cudaFree(b->d_den);
    cudaFree(b->d_v);
    b->d_den = nullptr;
    b->d_v = nullptr;
    GYPS_CUDA(cudaMalloc((void **)&b->d_den, std::max(den_floats, (size_t)1) * sizeof(float)));
    GYPS_CUDA(cudaMalloc((void **)&b->d_v, std::max(v_elems, (size_t)1) * sizeof(double2)));
    b->v_bytes = v_elems * sizeof(double2);
    float *den = b->d_den;
    double2 *v = b->d_v;
    int64_t item = 0, src = 0, vb = 0;
    b->pairs = 0.0;
    for (size_t mi = 0; mi < b->meshes.size(); ++mi) {
        Mesh *m = b->meshes[mi];
        const gyps_batch_item &it = items[mi];
        const int64_t ntt = (m->nq + tt - 1) / tt;
        for (int c = 0; c < nchunk; ++c) {
            FarSeg f;
            f.pos_panel = m->d_pos_panel;
            f.den_panel = den;
            f.tgt = m->d_pts32;
            f.v = v + (int64_t)c * R * m->nq;
            f.ldv = m->nq;
            f.nq = m->nq;
            f.n_src_tiles = m->n_src_tiles;
            f.n_tgt_tiles = ntt;
            f.item_begin = item;
            f.ks = it.k > 0.0 ? (float)it.k : 1.0f;
            f.lap = it.k > 0.0 ? 0 : 1;
            fs.push_back(f);
            InterpSeg g;
            g.tri = m->d_tri;
            g.pts64 = m->d_pts64;
            g.rule = m->rule;
            g.nq = m->nq;
            g.nq_pad = m->nq_pad;
            g.src_begin = src;
            g.X = (const double2 *)it.X;
            g.ldx = it.ldx;
            g.c0 = c * R;
            g.den_panel = den;
            is.push_back(g);
            item += ntt * m->n_src_tiles;
            src += m->nq_pad;
            den += m->n_src_tiles * den_tile_floats(R);
        }
        ProjMesh p;
        p.nv = m->nv;
        p.v_begin = vb;
        p.v2t_ptr = m->d_v2t_ptr;
        p.v2t = m->d_v2t;
        p.pts64 = m->d_pts64;
        p.rule = m->rule;
        p.v = v;
        p.ldv = m->nq;
        p.c_rowptr = m->d_c_rowptr;
        p.c_col = m->d_c_col;
        p.c_val = m->d_c_val;
        p.X = (const double2 *)it.X;
        p.ldx = it.ldx;
        p.Y = (double2 *)it.Y;
        p.ldy = it.ldy;
        pm.push_back(p);
        vb += m->nv;
        v += (int64_t)m->nq * b->nrhs;
        b->pairs += (double)m->nq * (double)m->nq;
    }
    b->items = item;
    b->total_src = src;
    b->total_v = vb;
    b->nseg = (int)fs.size();
    cudaFree(b->d_far);
    cudaFree(b->d_interp);
    cudaFree(b->d_proj);
    b->d_far = nullptr;
    b->d_interp = nullptr;
    b->d_proj = nullptr;
    GYPS_CUDA(cudaMalloc((void **)&b->d_far, fs.size() * sizeof(FarSeg)));
    GYPS_CUDA(cudaMalloc((void **)&b->d_interp, is.size() * sizeof(InterpSeg)));
    GYPS_CUDA(cudaMalloc((void **)&b->d_proj, pm.size() * sizeof(ProjMesh)));
    GYPS_CUDA(cudaMemcpy(b->d_far, fs.data(), fs.size() * sizeof(FarSeg), cudaMemcpyHostToDevice));
    GYPS_CUDA(cudaMemcpy(b->d_interp, is.data(), is.size() * sizeof(InterpSeg), cudaMemcpyHostToDevice));
    GYPS_CUDA(cudaMemcpy(b->d_proj, pm.data(), pm.size() * sizeof(ProjMesh), cudaMemcpyHostToDevice));
    int occ = 1;
    if (R == 8 && T == 2) GYPS_TRY((far_occupancy<8, 2>(&occ)));
    else if (R == 4 && T == 2) GYPS_TRY((far_occupancy<4, 2>(&occ)));
    else if (R == 4 && T == 4) GYPS_TRY((far_occupancy<4, 4>(&occ)));
    else if (R == 2 && T == 4) GYPS_TRY((far_occupancy<2, 4>(&occ)));
    else GYPS_TRY((far_occupancy<1, 4>(&occ)));
    int sms = 0;
    GYPS_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, b->device));
    b->grid = (int)std::min<int64_t>((int64_t)sms * occ, std::max<int64_t>(b->items, 1));
    return GYPS_OK;
}

static gyps_status capture(Batch *b)
{
    if (b->exec) cudaGraphExecDestroy(b->exec);
    if (b->graph) cudaGraphDestroy(b->graph);
    b->exec = nullptr;
    b->graph = nullptr;
    cudaStream_t cs;
    GYPS_CUDA(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
    gyps_status st = GYPS_OK;
    cudaError_t e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
    if (e == cudaSuccess) {
        st = enqueue(b, cs);
        cudaError_t e2 = cudaStreamEndCapture(cs, &b->graph);
        if (st == GYPS_OK && e2 != cudaSuccess) st = cuda_error(e2, "cudaStreamEndCapture");
        if (st == GYPS_OK) {
            cudaError_t e3 = cudaGraphInstantiate(&b->exec, b->graph, 0);
            if (e3 != cudaSuccess) st = cuda_error(e3, "cudaGraphInstantiate");
        }
    } else {
        st = cuda_error(e, "cudaStreamBeginCapture");
    }
    cudaStreamDestroy(cs);
    return st;
}

// ---------------------------------------------------------------- autotuner cache
static std::mutex g_tune_mu;

static std::string tune_path()
{
    const char *p = std::getenv("GYPS_TUNE_CACHE");
    if (p && *p) return p;
    const char *h = std::getenv("HOME");
    return std::string(h ? h : "/tmp") + "/.cache/gyps_tune.json";
}

static void mkdir_p_one(const std::string &d)
{
    if (!d.empty()) mkdir(d.c_str(), 0755);  // an existing directory is fine
}

// The cache is a flat JSON object {"key": [R, T, ms], ...}, one entry per line.
static bool tune_lookup(const std::string &key, int *R, int *T)
{
    std::lock_guard<std::mutex> lock(g_tune_mu);
    std::ifstream f(tune_path());
    std::string line;
    const std::string q = "\"" + key + "\"";
    while (std::getline(f, line)) {
        size_t p = line.find(q);
        if (p == std::string::npos) continue;
        size_t lb = line.find('[', p);
        if (lb == std::string::npos) continue;
        int r = 0, t = 0;
        if (std::sscanf(line.c_str() + lb, "[%d, %d", &r, &t) == 2 && r >= 0 && t >= 0) {
            *R = r;
            *T = t;
            return true;
        }
    }
    return false;
}

static void tune_store(const std::string &key, int R, int T, double ms)
{
    std::lock_guard<std::mutex> lock(g_tune_mu);
    std::vector<std::string> keep;
    {
        std::ifstream f(tune_path());
        std::string line;
        while (std::getline(f, line)) {
            if (line.find("\"") == std::string::npos || line.find("\"" + key + "\"") != std::string::npos) continue;
            while (!line.empty() && (line.back() == ',' || line.back() == ' ')) line.pop_back();
            size_t a = line.find('"');
            keep.push_back(line.substr(a));
        }
    }
    char buf[512];
    std::snprintf(buf, sizeof(buf), "\"%s\": [%d, %d, %.4f]", key.c_str(), R, T, ms);
    keep.push_back(buf);
    std::string path = tune_path();
    std::string dir = path.substr(0, path.find_last_of('/'));
    for (size_t i = 1; i <= dir.size(); ++i)
        if (i == dir.size() || dir[i] == '/') mkdir_p_one(dir.substr(0, i));
    std::ofstream o(path + ".tmp");
    o << "{\n";
    for (size_t i = 0; i < keep.size(); ++i) o << "  " << keep[i] << (i + 1 < keep.size() ? ",\n" : "\n");
    o << "}\n";
    o.close();
    std::rename((path + ".tmp").c_str(), path.c_str());
}

static std::string tune_key(const Batch *b)
{
    cudaDeviceProp pr;
    cudaGetDeviceProperties(&pr, b->device);
    int64_t nq = 0;
    for (auto *m : b->meshes) nq += m->nq;
    int bucket = 0;
    while ((int64_t)1 << (bucket + 1) <= nq) ++bucket;  // log2 of the total point count
    char buf[256];
    std::snprintf(buf, sizeof(buf), "%s|sm%d|meshes%d|nq2^%d|nrhs%d", pr.name, pr.multiProcessorCount, b->nmesh,
                  bucket, b->nrhs);
    return buf;
}

// Candidate (R, T) shapes: R divides nrhs; T chosen so the registers fit.
// (0, 0) stands for the tensor-core form (16 or more right-hand sides, k > 0).
static std::vector<std::pair<int, int>> candidates(int nrhs, bool tc_ok)
{
    std::vector<std::pair<int, int>> c;
    if (tc_ok && nrhs >= 16) c.push_back({0, 0});
    if (nrhs % 8 == 0) c.push_back({8, 2});
    if (nrhs % 4 == 0) {
        c.push_back({4, 2});
        c.push_back({4, 4});
    }
    if (nrhs % 2 == 0) c.push_back({2, 4});
    c.push_back({1, 4});
    return c;
}

static gyps_status time_config(Batch *b, cudaStream_t s, double *ms)
{
    cudaEvent_t e0, e1;
    GYPS_CUDA(cudaEventCreate(&e0));
    GYPS_CUDA(cudaEventCreate(&e1));
    gyps_status st = enqueue(b, s);  // warm-up
    if (st == GYPS_OK) {
        cudaEventRecord(e0, s);
        st = enqueue(b, s);
        cudaEventRecord(e1, s);
    }
    float t = 0.0f;
    if (st == GYPS_OK) {
        cudaError_t e = cudaEventSynchronize(e1);
        if (e == cudaSuccess) e = cudaEventElapsedTime(&t, e0, e1);
        if (e != cudaSuccess) st = cuda_error(e, "autotune timing");
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    *ms = t;
    return st;
}

}  // namespace gyps

using namespace gyps;

extern "C" gyps_status gyps_batch_create(const gyps_batch_item *items, int nitems, int nrhs, uint32_t flags,
                                         void *stream, gyps_batch_t *out)
{
    if (!out) return set_error(GYPS_ERR_INVALID, "out is NULL");
    *out = nullptr;
    if (!items || nitems < 1 || nitems > 4096) return set_error(GYPS_ERR_INVALID, "nitems must be in 1..4096");
    if (nrhs < 1 || nrhs > 4096) return set_error(GYPS_ERR_INVALID, "nrhs must be in 1..4096");
    if (flags & ~(GYPS_BATCH_NO_GRAPH | GYPS_BATCH_AUTOTUNE | GYPS_BATCH_CUDA_CORES))
        return set_error(GYPS_ERR_INVALID, "unknown flag");
    std::vector<gyps_batch_item> its(items, items + nitems);
    Batch *b = new Batch();
    b->nrhs = nrhs;
    b->nmesh = nitems;
    for (int i = 0; i < nitems; ++i) {
        Mesh *m;
        gyps_status st = check_mesh(its[i].mesh, &m);
        if (st != GYPS_OK) {
            delete b;
            return st;
        }
        if (i > 0 && m->device != b->device) {
            delete b;
            return set_error(GYPS_ERR_INVALID, "all meshes of a batch must live on one device");
        }
        b->device = m->device;
        const gyps_batch_item &it = its[i];
        if (!std::isfinite(it.k) || it.k < 0.0 || !it.X || !it.Y || it.ldx < m->nv || it.ldy < m->nv ||
            !is_device_pointer(it.X) || !is_device_pointer(it.Y)) {
            delete b;
            return set_error(GYPS_ERR_INVALID, "batch item " + std::to_string(i) +
                                                   ": need finite k >= 0 and device X, Y with ld >= nv");
        }
        b->meshes.push_back(m);
    }
    cudaSetDevice(b->device);
    cudaStream_t s = (cudaStream_t)stream;
    gyps_status st = GYPS_OK;
    if (cudaMalloc((void **)&b->d_err, sizeof(int)) != cudaSuccess) st = set_error(GYPS_ERR_OOM, "error word");
    if (st == GYPS_OK) cudaMemset(b->d_err, 0, sizeof(int));
    bool tc_ok = !(flags & GYPS_BATCH_CUDA_CORES);
    for (const auto &it : its) tc_ok = tc_ok && it.k > 0.0;
    int R = -1, T = -1;
    const std::string key =
        (st == GYPS_OK) ? tune_key(b) + ((flags & GYPS_BATCH_CUDA_CORES) ? "|cuda_cores" : "") : std::string();
    if (st == GYPS_OK && tune_lookup(key, &R, &T) && ((R == 0 && tc_ok && nrhs >= 16) || (R > 0 && nrhs % R == 0))) {
        b->tuned = 2;
    } else if (st == GYPS_OK && (flags & GYPS_BATCH_AUTOTUNE)) {
        double best = 1e300;
        for (auto c : candidates(nrhs, tc_ok)) {
            st = configure(b, its, c.first, c.second);
            double ms = 0.0;
            if (st == GYPS_OK) st = time_config(b, s, &ms);
            if (st != GYPS_OK) break;
            if (ms < best) {
                best = ms;
                R = c.first;
                T = c.second;
            }
        }
        if (st == GYPS_OK) {
            tune_store(key, R, T, best);
            b->tuned = 1;
        }
    } else if (st == GYPS_OK) {
        auto c = candidates(nrhs, tc_ok).front();  // tensor cores if possible, else the widest chunk
        R = c.first;
        T = c.second;
    }
    if (st == GYPS_OK) st = configure(b, its, R, T);
    b->use_graph = !(flags & GYPS_BATCH_NO_GRAPH);
    if (st == GYPS_OK && b->use_graph) {
        // one direct run first: workspaces are allocated before the capture
        st = enqueue(b, s);
        if (st == GYPS_OK) {
            cudaError_t e = cudaStreamSynchronize(s);
            if (e != cudaSuccess) st = cuda_error(e, "batch warm-up");
        }
        if (st == GYPS_OK && capture(b) != GYPS_OK) {
            cudaGetLastError();
            b->use_graph = false;  // launch directly when the work cannot be captured
        }
    }
    if (st != GYPS_OK) {
        cudaDeviceSynchronize();
        delete b;
        return st;
    }
    *out = reinterpret_cast<gyps_batch_t>(b);
    return GYPS_OK;
}

extern "C" gyps_status gyps_batch_apply(gyps_batch_t h, void *stream)
{
    if (!h) return set_error(GYPS_ERR_INVALID, "batch handle is NULL");
    Batch *b = reinterpret_cast<Batch *>(h);
    GYPS_CUDA(cudaSetDevice(b->device));
    cudaStream_t s = (cudaStream_t)stream;
    if (b->use_graph) {
        GYPS_CUDA(cudaGraphLaunch(b->exec, s));
        return GYPS_OK;
    }
    return enqueue(b, s);
}

extern "C" gyps_status gyps_batch_info(gyps_batch_t h, gyps_batch_info_t *info)
{
    if (!h || !info) return set_error(GYPS_ERR_INVALID, "NULL argument");
    Batch *b = reinterpret_cast<Batch *>(h);
    info->nmesh = b->nmesh;
    info->nrhs = b->nrhs;
    info->rhs_chunk = b->R;
    info->targets_per_thread = b->T;
    info->grid = b->grid;
    info->work_items = b->items;
    info->pairs = b->pairs;
    info->uses_graph = b->use_graph ? 1 : 0;
    info->tuned = b->tuned;
    info->tensor_cores = b->R == 0 ? 1 : 0;
    return GYPS_OK;
}

extern "C" gyps_status gyps_batch_destroy(gyps_batch_t h)
{
    if (!h) return GYPS_OK;
    Batch *b = reinterpret_cast<Batch *>(h);
    cudaSetDevice(b->device);
    cudaDeviceSynchronize();
    int err = 0;
    cudaMemcpy(&err, b->d_err, sizeof(int), cudaMemcpyDeviceToHost);
    delete b;
    if (err) return set_error(GYPS_ERR_TIMEOUT, "a device wait of the batch ran out of polls");
    return GYPS_OK;
}
