// Restarted GMRES for V X = F (Sec. 5.4, Eq. Singlelayerwf), one Krylov space
// per right-hand side, the operator applied to all columns at once.  Arnoldi
// uses classical Gram-Schmidt applied twice, in FP64 on the device; the small
// Hessenberg least-squares problems are solved on the host with Givens
// rotations.  A true residual in the check precision closes each solve, and
// the residual equation is solved again (iterative refinement) while it is
// above tolerance.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <complex>
#include <vector>

#include "internal.h"

namespace gyps {

gyps_status check_err_word(Mesh *m, cudaStream_t s);

using cplx = std::complex<double>;

// h[i, c] += sum_n conj(Q_i[n, c]) W[n, c], i < nvec.  Q_i blocks of nv x nrhs (ld nv).
__global__ void zdots_kernel(const double2 *Q, int nvec, const double2 *W, int64_t nv, int nrhs, double2 *h)
{
    const int c = blockIdx.y;
    const int64_t n0 = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    __shared__ double red[2][32];
    for (int i = 0; i < nvec; ++i) {
        const double2 *q = Q + (int64_t)i * nv * nrhs + (int64_t)c * nv;
        const double2 *w = W + (int64_t)c * nv;
        double sr = 0.0, si = 0.0;
        for (int64_t n = n0; n < nv; n += stride) {
            double2 a = q[n], b = w[n];
            sr += a.x * b.x + a.y * b.y;
            si += a.x * b.y - a.y * b.x;
        }
        for (int o = 16; o > 0; o >>= 1) {
            sr += __shfl_down_sync(0xffffffffu, sr, o);
            si += __shfl_down_sync(0xffffffffu, si, o);
        }
        const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
        if (lane == 0) {
            red[0][warp] = sr;
            red[1][warp] = si;
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            double tr = 0.0, ti = 0.0;
            for (int k = 0; k < (int)(blockDim.x >> 5); ++k) {
                tr += red[0][k];
                ti += red[1][k];
            }
            atomicAdd(&h[(int64_t)i * nrhs + c].x, tr);
            atomicAdd(&h[(int64_t)i * nrhs + c].y, ti);
        }
        __syncthreads();
    }
}

// W[n, c] -= sum_{i < nvec} Q_i[n, c] h[i, c]
__global__ void zsub_kernel(const double2 *Q, int nvec, const double2 *h, int64_t nv, int nrhs, double2 *W)
{
    const int c = blockIdx.y;
    const int64_t n = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (n >= nv) return;
    double2 w = W[(int64_t)c * nv + n];
    for (int i = 0; i < nvec; ++i) {
        double2 q = Q[(int64_t)i * nv * nrhs + (int64_t)c * nv + n];
        double2 hh = h[(int64_t)i * nrhs + c];
        w.x -= q.x * hh.x - q.y * hh.y;
        w.y -= q.x * hh.y + q.y * hh.x;
    }
    W[(int64_t)c * nv + n] = w;
}

// nrm[c] += sum_n |W[n, c]|^2
__global__ void znorm2_kernel(const double2 *W, int64_t nv, double *nrm)
{
    const int c = blockIdx.y;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    double s = 0.0;
    for (int64_t n = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; n < nv; n += stride) {
        double2 a = W[(int64_t)c * nv + n];
        s += a.x * a.x + a.y * a.y;
    }
    for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
    __shared__ double red[32];
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int k = 0; k < (int)(blockDim.x >> 5); ++k) t += red[k];
        atomicAdd(&nrm[c], t);
    }
}

// D[:, c] = S[:, c] * scale[c]
__global__ void zscale_kernel(const double2 *S, const double *scale, int64_t nv, double2 *D)
{
    const int c = blockIdx.y;
    const int64_t n = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (n >= nv) return;
    double2 a = S[(int64_t)c * nv + n];
    D[(int64_t)c * nv + n] = make_double2(a.x * scale[c], a.y * scale[c]);
}

// X[n, c] += sum_{i < nvec} Q_i[n, c] y[i, c]   (X with leading dimension ldx)
__global__ void zupdate_kernel(const double2 *Q, int nvec, const double2 *y, int64_t nv, int nrhs, double2 *X,
                               int64_t ldx)
{
    const int c = blockIdx.y;
    const int64_t n = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (n >= nv) return;
    double2 x = X[(int64_t)c * ldx + n];
    for (int i = 0; i < nvec; ++i) {
        double2 q = Q[(int64_t)i * nv * nrhs + (int64_t)c * nv + n];
        double2 yy = y[(int64_t)i * nrhs + c];
        x.x += q.x * yy.x - q.y * yy.y;
        x.y += q.x * yy.y + q.y * yy.x;
    }
    X[(int64_t)c * ldx + n] = x;
}

// R[:, c] = B[:, c] - AX[:, c]  (B with leading dimension ldb, others nv)
__global__ void zresid_kernel(const double2 *B, int64_t ldb, const double2 *AX, int64_t nv, double2 *R)
{
    const int c = blockIdx.y;
    const int64_t n = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (n >= nv) return;
    double2 b = B[(int64_t)c * ldb + n], a = AX[(int64_t)c * nv + n];
    R[(int64_t)c * nv + n] = make_double2(b.x - a.x, b.y - a.y);
}

// X[:, c] (ld ldx) += D[:, c] (ld nv)
__global__ void zadd_kernel(const double2 *D, int64_t nv, double2 *X, int64_t ldx)
{
    const int c = blockIdx.y;
    const int64_t n = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (n >= nv) return;
    double2 d = D[(int64_t)c * nv + n];
    double2 &x = X[(int64_t)c * ldx + n];
    x.x += d.x;
    x.y += d.y;
}

namespace {

struct Work {
    double2 *Q = nullptr;    // (m + 1) blocks of nv x nrhs
    double2 *W = nullptr;    // nv x nrhs
    double2 *R = nullptr;    // nv x nrhs
    double2 *D = nullptr;    // nv x nrhs (refinement correction)
    double2 *Z = nullptr;    // m blocks of nv x nrhs: preconditioned basis (flexible GMRES)
    double2 *h = nullptr;    // (m + 1) x nrhs
    double *nrm = nullptr;   // nrhs
    double *scl = nullptr;   // nrhs
    double2 *hh = nullptr;   // pinned host mirror of h
    double *hn = nullptr;    // pinned host mirror of nrm
    ~Work()
    {
        cudaFree(Q);
        cudaFree(W);
        cudaFree(R);
        cudaFree(D);
        cudaFree(Z);
        cudaFree(h);
        cudaFree(nrm);
        cudaFree(scl);
        cudaFreeHost(hh);
        cudaFreeHost(hn);
    }
};

struct Solver {
    Mesh *m;
    double k;
    int nrhs, restart;
    cudaStream_t s;
    Work w;
    int64_t nv;
    int iters = 0, applies = 0, check_applies = 0;
    gyps_precond_t P = nullptr;  // learned preconditioner (flexible GMRES) while pre_on
    bool pre_on = false;
    int fallback = 0;
    int form = GYPS_FORM_SINGLE_LAYER;
    double eta = 0.0;
    // wall-clock limit (timeout_ms > 0): checked before every inner iteration
    bool has_deadline = false, timed_out = false;
    std::chrono::steady_clock::time_point deadline;
    bool past_deadline()
    {
        if (has_deadline && !timed_out && std::chrono::steady_clock::now() >= deadline) timed_out = true;
        return timed_out;
    }

    // Y = A X for the system's operator A: V (first kind), 1/2 M + K - i eta V
    // (Brakhage-Werner), 1/2 M + K' - i eta V (direct combined field), all
    // nv x nrhs, or -T (the EFIE) and -eta T + (1 - eta)(Id/2 - nxK) (the
    // electromagnetic combined field with beta = eta), ne x nrhs.
    Hmat *hm = nullptr;  // compressed operator of GYPS_PREC_HMAT
    gyps_status op(const double2 *X, int64_t ldx, double2 *Y, int prec)
    {
        if (prec == GYPS_PREC_HMAT) return hmat_apply_device(hm, nrhs, X, ldx, Y, nv, s);
        if (form == GYPS_FORM_EFIE) return efie_apply_device(m, k, -1.0, nrhs, X, ldx, Y, nv, prec, s);
        if (form == GYPS_FORM_EM_CFIE) return emcfie_apply_device(m, k, eta, 1.0, nrhs, X, ldx, Y, nv, prec, s);
        if (form == GYPS_FORM_BRAKHAGE_WERNER || form == GYPS_FORM_DIRECT_CFIE)
            return combined_apply_device(m, k, eta, form == GYPS_FORM_DIRECT_CFIE, nrhs, X, ldx, Y, nv, prec, s);
        return apply_device(m, k, nrhs, X, ldx, Y, nv, prec, 0, 0, m->nt, s);
    }

    // Column norms without the non-finite check (the preconditioned cycle
    // handles a non-finite value by dropping the preconditioner).
    gyps_status norms_raw(const double2 *A, std::vector<double> &out, bool *finite)
    {
        GYPS_CUDA(cudaMemsetAsync(w.nrm, 0, nrhs * sizeof(double), s));
        znorm2_kernel<<<grid_r, 256, 0, s>>>(A, nv, w.nrm);
        GYPS_CUDA(cudaGetLastError());
        GYPS_CUDA(cudaMemcpyAsync(w.hn, w.nrm, nrhs * sizeof(double), cudaMemcpyDeviceToHost, s));
        GYPS_CUDA(cudaStreamSynchronize(s));
        out.resize(nrhs);
        *finite = true;
        for (int c = 0; c < nrhs; ++c) {
            out[c] = std::sqrt(w.hn[c]);
            *finite = *finite && std::isfinite(out[c]);
        }
        return GYPS_OK;
    }
    dim3 grid_v, grid_r;

    gyps_status norms(const double2 *A, std::vector<double> &out)
    {
        GYPS_CUDA(cudaMemsetAsync(w.nrm, 0, nrhs * sizeof(double), s));
        znorm2_kernel<<<grid_r, 256, 0, s>>>(A, nv, w.nrm);
        GYPS_CUDA(cudaGetLastError());
        GYPS_CUDA(cudaMemcpyAsync(w.hn, w.nrm, nrhs * sizeof(double), cudaMemcpyDeviceToHost, s));
        GYPS_CUDA(cudaStreamSynchronize(s));
        out.resize(nrhs);
        for (int c = 0; c < nrhs; ++c) {
            out[c] = std::sqrt(w.hn[c]);
            if (!std::isfinite(out[c])) return set_error(GYPS_ERR_NAN, "non-finite value in GMRES");
        }
        return GYPS_OK;
    }

    gyps_status scale_into(const double2 *S, const std::vector<double> &sc, double2 *D)
    {
        std::vector<double> tmp(sc);
        GYPS_CUDA(cudaMemcpyAsync(w.scl, tmp.data(), nrhs * sizeof(double), cudaMemcpyHostToDevice, s));
        zscale_kernel<<<grid_v, 256, 0, s>>>(S, w.scl, nv, D);
        GYPS_CUDA(cudaGetLastError());
        GYPS_CUDA(cudaStreamSynchronize(s));  // tmp leaves scope
        return GYPS_OK;
    }

    // R = B - V X with precision prec (B: ld ldb; X: ld ldx).
    gyps_status residual(const double2 *B, int64_t ldb, const double2 *X, int64_t ldx, int prec)
    {
        GYPS_TRY(op(X, ldx, w.W, prec));
        zresid_kernel<<<grid_v, 256, 0, s>>>(B, ldb, w.W, nv, w.R);
        GYPS_CUDA(cudaGetLastError());
        return GYPS_OK;
    }

    // GMRES on V X = B from the current X (zero when x_is_zero), until every
    // column has ||B - V X|| <= tol_c, or `budget` inner iterations are used.
    gyps_status solve(const double2 *B, int64_t ldb, double2 *X, int64_t ldx, bool x_is_zero,
                      const std::vector<double> &tol_abs, int prec, int budget, std::vector<double> &est)
    {
        const int m = restart;
        std::vector<double> beta;
        est.assign(nrhs, 0.0);
        bool first = true;
        while (true) {
            if (first && x_is_zero) {
                GYPS_CUDA(cudaMemcpy2DAsync(w.R, nv * sizeof(double2), B, ldb * sizeof(double2), nv * sizeof(double2),
                                            nrhs, cudaMemcpyDeviceToDevice, s));
            } else {
                GYPS_TRY(residual(B, ldb, X, ldx, prec));
                ++applies;
            }
            first = false;
            GYPS_TRY(norms(w.R, beta));
            est = beta;
            bool all = true;
            for (int c = 0; c < nrhs; ++c) all = all && beta[c] <= tol_abs[c];
            if (all || budget <= 0) return GYPS_OK;

            std::vector<double> inv(nrhs);
            for (int c = 0; c < nrhs; ++c) inv[c] = (beta[c] > tol_abs[c]) ? 1.0 / beta[c] : 0.0;
            GYPS_TRY(scale_into(w.R, inv, w.Q));

            std::vector<std::vector<cplx>> H(nrhs, std::vector<cplx>((size_t)(m + 1) * m));
            std::vector<std::vector<cplx>> cs(nrhs, std::vector<cplx>(m)), sn(nrhs, std::vector<cplx>(m));
            std::vector<std::vector<cplx>> g(nrhs, std::vector<cplx>(m + 1));
            std::vector<int> jc(nrhs, 0);
            std::vector<char> active(nrhs, 0);
            for (int c = 0; c < nrhs; ++c) {
                g[c][0] = beta[c];
                active[c] = beta[c] > tol_abs[c];
            }
            int j = 0;
            bool cycle_converged = false;  // every column reached tol by its Arnoldi estimate
            bool dropped = false;          // preconditioner dropped inside this cycle
            const bool cycle_pre = pre_on;
            for (; j < m && budget > 0; ++j) {
                if (past_deadline()) {  // finish this cycle with the iterations done, then stop
                    budget = 0;
                    break;
                }
                double2 *qj = w.Q + (size_t)j * nv * nrhs;
                double2 *qn = w.Q + (size_t)(j + 1) * nv * nrhs;
                const double2 *vin = qj;
                if (pre_on) {  // flexible GMRES: z_j = M(q_j), w = V z_j
                    double2 *zj = w.Z + (size_t)j * nv * nrhs;
                    GYPS_TRY(precond_apply_device(P, this->m, k, nrhs, qj, nv, zj, nv, s));
                    std::vector<double> zn;
                    bool zfinite = true;
                    GYPS_TRY(norms_raw(zj, zn, &zfinite));
                    if (!zfinite) {  // the network produced a non-finite value: drop it, redo the cycle
                        pre_on = false;
                        fallback = 1;
                        dropped = true;
                        break;
                    }
                    vin = zj;
                }
                GYPS_TRY(op(vin, nv, w.W, prec));
                ++applies;
                ++iters;
                --budget;
                std::vector<cplx> hsum((size_t)(j + 1) * nrhs, 0.0);
                for (int pass = 0; pass < 2; ++pass) {  // CGS2
                    GYPS_CUDA(cudaMemsetAsync(w.h, 0, (size_t)(j + 1) * nrhs * sizeof(double2), s));
                    zdots_kernel<<<grid_r, 256, 0, s>>>(w.Q, j + 1, w.W, nv, nrhs, w.h);
                    GYPS_CUDA(cudaGetLastError());
                    zsub_kernel<<<grid_v, 256, 0, s>>>(w.Q, j + 1, w.h, nv, nrhs, w.W);
                    GYPS_CUDA(cudaGetLastError());
                    GYPS_CUDA(cudaMemcpyAsync(w.hh, w.h, (size_t)(j + 1) * nrhs * sizeof(double2),
                                              cudaMemcpyDeviceToHost, s));
                    GYPS_CUDA(cudaStreamSynchronize(s));
                    for (size_t e = 0; e < (size_t)(j + 1) * nrhs; ++e) hsum[e] += cplx(w.hh[e].x, w.hh[e].y);
                }
                std::vector<double> hn;
                if (pre_on) {
                    bool finite = true;
                    GYPS_TRY(norms_raw(w.W, hn, &finite));
                    if (!finite) {  // the network produced a non-finite value: drop it, redo the cycle
                        pre_on = false;
                        fallback = 1;
                        dropped = true;
                        break;
                    }
                } else {
                    GYPS_TRY(norms(w.W, hn));
                }
                std::vector<double> inv2(nrhs);
                for (int c = 0; c < nrhs; ++c) inv2[c] = (active[c] && hn[c] > 0.0) ? 1.0 / hn[c] : 0.0;
                GYPS_TRY(scale_into(w.W, inv2, qn));
                bool any = false;
                for (int c = 0; c < nrhs; ++c) {
                    if (!active[c]) continue;
                    cplx *Hc = &H[c][(size_t)j * (m + 1)];  // column j
                    for (int i = 0; i <= j; ++i) Hc[i] = hsum[(size_t)i * nrhs + c];
                    Hc[j + 1] = hn[c];
                    for (int i = 0; i < j; ++i) {
                        cplx t = std::conj(cs[c][i]) * Hc[i] + std::conj(sn[c][i]) * Hc[i + 1];
                        Hc[i + 1] = -sn[c][i] * Hc[i] + cs[c][i] * Hc[i + 1];
                        Hc[i] = t;
                    }
                    double den = std::sqrt(std::norm(Hc[j]) + std::norm(Hc[j + 1]));
                    if (den == 0.0) {
                        cs[c][j] = 1.0;
                        sn[c][j] = 0.0;
                    } else {
                        cs[c][j] = Hc[j] / den;
                        sn[c][j] = Hc[j + 1] / den;
                    }
                    Hc[j] = den;
                    Hc[j + 1] = 0.0;
                    g[c][j + 1] = -sn[c][j] * g[c][j];
                    g[c][j] = std::conj(cs[c][j]) * g[c][j];
                    jc[c] = j + 1;
                    est[c] = std::abs(g[c][j + 1]);
                    if (!std::isfinite(est[c])) return set_error(GYPS_ERR_NAN, "non-finite value in GMRES");
                    if (est[c] <= tol_abs[c] || hn[c] == 0.0) active[c] = 0;
                    any = any || active[c];
                }
                if (!any) {
                    ++j;
                    cycle_converged = true;
                    break;
                }
            }
            if (dropped) continue;  // discard the cycle, restart from the current X without M
            // y = H^{-1} g per column (upper triangular), X += Q y (or Z y, flexible)
            const int nvec = std::max(1, j);
            std::vector<double2> y((size_t)nvec * nrhs, make_double2(0.0, 0.0));
            for (int c = 0; c < nrhs; ++c) {
                std::vector<cplx> yc(jc[c]);
                for (int i = jc[c] - 1; i >= 0; --i) {
                    cplx acc = g[c][i];
                    for (int l = i + 1; l < jc[c]; ++l) acc -= H[c][(size_t)l * (m + 1) + i] * yc[l];
                    yc[i] = acc / H[c][(size_t)i * (m + 1) + i];
                }
                for (int i = 0; i < jc[c]; ++i) y[(size_t)i * nrhs + c] = make_double2(yc[i].real(), yc[i].imag());
            }
            GYPS_CUDA(cudaMemcpyAsync(w.h, y.data(), y.size() * sizeof(double2), cudaMemcpyHostToDevice, s));
            zupdate_kernel<<<grid_v, 256, 0, s>>>(cycle_pre ? w.Z : w.Q, nvec, w.h, nv, nrhs, X, ldx);
            GYPS_CUDA(cudaGetLastError());
            GYPS_CUDA(cudaStreamSynchronize(s));  // y leaves scope
            // The estimate decides: a residual recomputed with an FP32 operator
            // carries that operator's rounding and could never go below its
            // floor; the caller's check-precision residual judges the result.
            if (cycle_converged) return GYPS_OK;
            if (cycle_pre) {  // a full preconditioned cycle that did not halve the residual: drop M
                bool progress = false;
                for (int c = 0; c < nrhs; ++c) progress = progress || (beta[c] > tol_abs[c] && est[c] < 0.5 * beta[c]);
                if (!progress) {
                    pre_on = false;
                    fallback = 1;
                }
            }
        }
    }
};

}  // namespace

gyps_status gmres_device(Mesh *m, double k, int nrhs, const double2 *F, int64_t ldf, double2 *X, int64_t ldx,
                         const gyps_gmres_opts &o, gyps_gmres_report *rep, cudaStream_t s)
{
    Solver S;
    S.m = m;
    S.k = k;
    S.nrhs = nrhs;
    S.restart = o.restart;
    S.s = s;
    const bool em = o.formulation == GYPS_FORM_EFIE || o.formulation == GYPS_FORM_EM_CFIE;
    const int64_t n = em ? m->ne : m->nv;  // unknowns per column
    S.nv = n;
    S.form = o.formulation;
    S.eta = o.eta;
    S.hm = hmat_of(o.hmat);
    if (o.timeout_ms > 0.0) {
        S.has_deadline = true;
        S.deadline = std::chrono::steady_clock::now() +
                     std::chrono::microseconds((int64_t)std::min(o.timeout_ms * 1e3, 9.0e15));
    }
    GYPS_TRY(clear_err_word(m, s));  // report only the waits of this solve's launches
    S.grid_v = dim3((unsigned)((n + 255) / 256), (unsigned)nrhs);
    S.grid_r = dim3((unsigned)std::min<int64_t>((n + 255) / 256, 64), (unsigned)nrhs);
    const size_t blk = (size_t)n * nrhs * sizeof(double2);
    GYPS_CUDA(cudaMalloc((void **)&S.w.Q, blk * (o.restart + 1)));
    GYPS_CUDA(cudaMalloc((void **)&S.w.W, blk));
    GYPS_CUDA(cudaMalloc((void **)&S.w.R, blk));
    GYPS_CUDA(cudaMalloc((void **)&S.w.D, blk));
    if (o.precond) {
        bool in_range = true;
        GYPS_TRY(precond_in_range(o.precond, m, k, s, &in_range));
        if (in_range) {
            GYPS_CUDA(cudaMalloc((void **)&S.w.Z, blk * o.restart));
            S.P = o.precond;
            S.pre_on = true;
        } else {
            S.fallback = 2;  // outside the electrical sizes the network was trained on: plain GMRES
        }
    }
    GYPS_CUDA(cudaMalloc((void **)&S.w.h, (size_t)(o.restart + 1) * nrhs * sizeof(double2)));
    GYPS_CUDA(cudaMalloc((void **)&S.w.nrm, nrhs * sizeof(double)));
    GYPS_CUDA(cudaMalloc((void **)&S.w.scl, nrhs * sizeof(double)));
    GYPS_CUDA(cudaMallocHost((void **)&S.w.hh, (size_t)(o.restart + 1) * nrhs * sizeof(double2)));
    GYPS_CUDA(cudaMallocHost((void **)&S.w.hn, nrhs * sizeof(double)));

    if (!o.use_x0) GYPS_CUDA(cudaMemset2DAsync(X, ldx * sizeof(double2), 0, n * sizeof(double2), nrhs, s));

    std::vector<double> fn;
    {
        // ||F|| per column
        double2 *Fc = S.w.R;
        GYPS_CUDA(cudaMemcpy2DAsync(Fc, n * sizeof(double2), F, ldf * sizeof(double2), n * sizeof(double2), nrhs,
                                    cudaMemcpyDeviceToDevice, s));
        GYPS_TRY(S.norms(Fc, fn));
    }
    std::vector<double> tol_abs(nrhs);
    for (int c = 0; c < nrhs; ++c) tol_abs[c] = o.tol * fn[c];
    int budget = o.maxit;
    std::vector<double> est;
    // When a different precision judges the result, the working-precision solve
    // aims below tol so that the first check usually passes.
    std::vector<double> tol_first(tol_abs);
    if (o.check_prec != o.prec)
        for (int c = 0; c < nrhs; ++c) tol_first[c] *= 0.5;
    GYPS_TRY(S.solve(F, ldf, X, ldx, !o.use_x0, tol_first, o.prec, budget, est));
    budget = S.timed_out ? 0 : o.maxit - S.iters;

    std::vector<double> tres;
    int refinements = 0;
    while (true) {
        GYPS_TRY(S.residual(F, ldf, X, ldx, o.check_prec));
        ++S.check_applies;
        GYPS_TRY(S.norms(S.w.R, tres));
        bool all = true;
        for (int c = 0; c < nrhs; ++c) all = all && tres[c] <= tol_abs[c];
        if (all || refinements >= o.max_refine || budget <= 0 || S.past_deadline()) break;
        // solve V D = R in the working precision, then X += D
        std::vector<double> tol_d(nrhs);
        for (int c = 0; c < nrhs; ++c) tol_d[c] = 0.5 * tol_abs[c];
        GYPS_CUDA(cudaMemcpyAsync(S.w.D, S.w.R, blk, cudaMemcpyDeviceToDevice, s));
        double2 *Bd = S.w.D;
        // the residual equation's right-hand side must survive inside solve(): keep it in D and solve into W-free X'
        double2 *Xd = nullptr;
        GYPS_CUDA(cudaMalloc((void **)&Xd, blk));
        GYPS_CUDA(cudaMemsetAsync(Xd, 0, blk, s));
        int before = S.iters;
        gyps_status st = S.solve(Bd, n, Xd, n, true, tol_d, o.prec, budget, est);
        if (st == GYPS_OK) {
            zadd_kernel<<<S.grid_v, 256, 0, s>>>(Xd, n, X, ldx);
            cudaError_t e = cudaGetLastError();
            if (e != cudaSuccess) st = cuda_error(e, "zadd_kernel");
        }
        cudaStreamSynchronize(s);
        cudaFree(Xd);
        GYPS_TRY(st);
        budget -= S.iters - before;
        ++refinements;
    }
    GYPS_TRY(check_err_word(m, s));
    bool ok = true;
    for (int c = 0; c < nrhs; ++c) ok = ok && tres[c] <= tol_abs[c];
    if (rep) {
        rep->iterations = S.iters;
        rep->applies = S.applies;
        rep->check_applies = S.check_applies;
        rep->refinements = refinements;
        rep->precond_fallback = S.fallback;
        for (int c = 0; c < nrhs; ++c) {
            double f = fn[c] > 0 ? fn[c] : 1.0;
            if (rep->est_residual) rep->est_residual[c] = est[c] / f;
            if (rep->true_residual) rep->true_residual[c] = tres[c] / f;
            if (rep->converged) rep->converged[c] = tres[c] <= tol_abs[c];
        }
    }
    if (!ok && S.timed_out) return set_error(GYPS_ERR_TIMEOUT, "GMRES stopped at its wall-clock limit");
    if (!ok) return set_error(GYPS_ERR_NOT_CONVERGED, "GMRES did not reach the tolerance on every column");
    return GYPS_OK;
}

}  // namespace gyps

using namespace gyps;

extern "C" gyps_status gyps_gmres_solve(gyps_mesh_t h, double k, int nrhs, const void *F, int64_t ldf, void *X,
                                        int64_t ldx, const gyps_gmres_opts *opts, gyps_gmres_report *report,
                                        void *stream)
{
    Mesh *m;
    GYPS_TRY(check_mesh(h, &m));
    if (!F || !X || !opts) return set_error(GYPS_ERR_INVALID, "NULL argument");
    if (nrhs < 1 || nrhs > 4096) return set_error(GYPS_ERR_INVALID, "nrhs must be in 1..4096");
    if (!std::isfinite(k) || k < 0.0) return set_error(GYPS_ERR_INVALID, "k must be finite and >= 0");
    const gyps_gmres_opts &o = *opts;
    if (!(o.tol > 0.0) || o.restart < 1 || o.restart > 4096 || o.maxit < 1 || o.max_refine < 0 ||
        !(o.timeout_ms >= 0.0))
        return set_error(GYPS_ERR_INVALID, "bad GMRES options");
    if (o.formulation != GYPS_FORM_SINGLE_LAYER && o.formulation != GYPS_FORM_BRAKHAGE_WERNER &&
        o.formulation != GYPS_FORM_DIRECT_CFIE && o.formulation != GYPS_FORM_EFIE &&
        o.formulation != GYPS_FORM_EM_CFIE)
        return set_error(GYPS_ERR_INVALID, "unknown formulation");
    const bool em = o.formulation == GYPS_FORM_EFIE || o.formulation == GYPS_FORM_EM_CFIE;
    if (o.check_prec == GYPS_PREC_HMAT) return set_error(GYPS_ERR_INVALID, "the check needs a kernel precision");
    if (o.prec == GYPS_PREC_HMAT) {
        const Hmat *hm = hmat_of(o.hmat);
        if (!hm) return set_error(GYPS_ERR_INVALID, "GYPS_PREC_HMAT needs opts->hmat");
        if (o.formulation != GYPS_FORM_SINGLE_LAYER)
            return set_error(GYPS_ERR_UNSUPPORTED, "the compressed operator is the single layer");
        if (hmat_mesh(hm) != m || hmat_k(hm) != k)
            return set_error(GYPS_ERR_INVALID, "opts->hmat was built for another mesh or wavenumber");
    }
    if (em) {
        if (!(k > 0.0)) return set_error(GYPS_ERR_INVALID, "the EFIE needs k > 0");
        if (o.prec == GYPS_PREC_TC_BF16X3 || o.check_prec == GYPS_PREC_TC_BF16X3)
            return set_error(GYPS_ERR_UNSUPPORTED, "EFIE: FP64, FP32 or DF64");
        GYPS_TRY(efie_prepare(m, (cudaStream_t)stream));
    }
    const int64_t n = em ? m->ne : m->nv;
    if (ldf < n || ldx < n) return set_error(GYPS_ERR_INVALID, "leading dimension < number of unknowns");
    if (o.formulation != GYPS_FORM_SINGLE_LAYER) {
        if (!std::isfinite(o.eta)) return set_error(GYPS_ERR_INVALID, "eta must be finite");
        if (o.precond) return set_error(GYPS_ERR_UNSUPPORTED, "the learned preconditioner models the single layer");
        if (o.prec == GYPS_PREC_TC_BF16X3 && nrhs < 16)
            return set_error(GYPS_ERR_UNSUPPORTED, "tensor-core precision needs 16 or more right-hand sides");
    }
    cudaStream_t s = (cudaStream_t)stream;
    const bool df = is_device_pointer(F), dx = is_device_pointer(X);
    if (df && dx) return gmres_device(m, k, nrhs, (const double2 *)F, ldf, (double2 *)X, ldx, o, report, s);
    const size_t blk = (size_t)n * nrhs * sizeof(double2);
    double2 *fs = nullptr, *xs = nullptr;
    GYPS_CUDA(cudaMalloc((void **)&fs, 2 * blk));
    xs = fs + (size_t)n * nrhs;
    gyps_status st = GYPS_OK;
    const double2 *fin = (const double2 *)F;
    int64_t lf = ldf;
    if (!df) {
        cudaError_t e = cudaMemcpy2DAsync(fs, n * sizeof(double2), F, ldf * sizeof(double2), n * sizeof(double2),
                                          nrhs, cudaMemcpyHostToDevice, s);
        if (e != cudaSuccess) st = cuda_error(e, "copy F");
        fin = fs;
        lf = n;
    }
    double2 *xio = dx ? (double2 *)X : xs;
    int64_t lx = dx ? ldx : n;
    if (st == GYPS_OK && !dx && o.use_x0) {
        cudaError_t e = cudaMemcpy2DAsync(xs, n * sizeof(double2), X, ldx * sizeof(double2), n * sizeof(double2),
                                          nrhs, cudaMemcpyHostToDevice, s);
        if (e != cudaSuccess) st = cuda_error(e, "copy X");
    }
    gyps_status solve_st = GYPS_OK;
    if (st == GYPS_OK) {
        solve_st = gmres_device(m, k, nrhs, fin, lf, xio, lx, o, report, s);
        if ((solve_st == GYPS_OK || solve_st == GYPS_ERR_NOT_CONVERGED) && !dx) {
            cudaError_t e = cudaMemcpy2DAsync(X, ldx * sizeof(double2), xs, n * sizeof(double2),
                                              n * sizeof(double2), nrhs, cudaMemcpyDeviceToHost, s);
            if (e != cudaSuccess) st = cuda_error(e, "copy X back");
        }
    }
    cudaStreamSynchronize(s);
    cudaFree(fs);
    if (st != GYPS_OK) return st;
    return solve_st;
}
