/*
 * gyps.h - C ABI of the GB300 Galerkin single-layer library (libgyps.so).
 *
 * The operator is the Helmholtz single layer on P1 triangle meshes,
 *     V_ij = int int phi_i(x) exp(ik|x-y|) / (4 pi |x-y|) phi_j(y) dx dy,
 * discretised as in Sec. 5, Eq. (BEM) of the paper:
 *     V ~ (1/4pi) Phi^T W_x G W_y Phi  +  C,
 * with Gauss points on each triangle, the dense kernel G_kl = exp(ik r_kl)/r_kl
 * between point clouds, the sparse P1 matrix Phi and the sparse singular
 * correction C of Sec. 5.2 (analytic y-integral of 1/r minus its Gauss sum, for
 * triangles sharing a vertex).  The sound-soft sphere example of Sec. 5.4 is the
 * intended use: V lambda = F with F_i = int phi_i exp(ik d.x).
 *
 * Conventions for every call:
 *  - Return value: GYPS_OK (0) or an error code; gyps_last_error() gives the
 *    message of the calling thread's last failing call.  No call aborts, traps
 *    or exits the process; invalid arguments return GYPS_ERR_INVALID.
 *  - Complex vectors and matrices are interleaved (re, im) pairs of the stated
 *    type (double2 = two doubles), column-major with a leading dimension counted
 *    in complex elements (ld >= number of rows).  Column j of an Nv x nrhs
 *    block X starts at X + j*ldx.
 *  - The caller owns every array it passes.  Unless a pointer is documented as
 *    a host pointer, it may be device memory (then the call is asynchronous on
 *    `stream`) or host memory (then the call copies through library-owned
 *    device staging and returns after `stream` has finished).
 *  - `stream` is a cudaStream_t passed as void* (NULL = the legacy default
 *    stream).  The library owns mesh handles and the device memory inside them.
 *  - A mesh's workspaces (accumulators, density panels, staging) serve every
 *    call on that mesh: issue the calls on one mesh on one stream, or serialise
 *    them; different meshes may run on different streams at the same time.
 *  - The wavenumber k must be finite and >= 0 (k = 0 is the Laplace kernel);
 *    the electromagnetic operators (RWG functions) need k > 0.
 */
#ifndef GYPS_H
#define GYPS_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    GYPS_OK = 0,
    GYPS_ERR_INVALID = 1,       /* bad argument (sizes, indices, k, degenerate triangle) */
    GYPS_ERR_CUDA = 2,          /* a CUDA runtime call failed; message names it */
    GYPS_ERR_OOM = 3,           /* device allocation failed */
    GYPS_ERR_NOT_CONVERGED = 4, /* GMRES hit maxit; X holds the last iterate */
    GYPS_ERR_NAN = 5,           /* a non-finite value appeared in the solve */
    GYPS_ERR_TIMEOUT = 6,       /* a device wait exceeded its iteration limit, or GMRES its wall-clock limit */
    GYPS_ERR_UNSUPPORTED = 7    /* option not available on this device/build */
} gyps_status;

/* Arithmetic of the dense kernel product G u (Sec. 5, Eq. BEM). The sparse
 * factors, the correction C and the output are FP64 in every mode. */
typedef enum {
    GYPS_PREC_FP64 = 0,         /* G and G u in FP64 (the plain reference form) */
    GYPS_PREC_FP32 = 1,         /* G in FP32 on the CUDA cores, compensated FP32 sums */
    GYPS_PREC_TC_BF16X3 = 2,    /* G tile x RHS panel on tensor cores, bf16 hi+lo split */
    GYPS_PREC_DF64 = 3,         /* G and G u in double-float (hi + lo FP32 pairs, about 44 bits) on the
                                   FP32 pipe: FP64-class accuracy (about 1e-12 from FP64) at several
                                   times the FP64 pipe's speed; for true-residual checks */
    GYPS_PREC_AUTO = 4,         /* FP32 below 16 right-hand sides, tensor cores above */
    GYPS_PREC_HMAT = 5          /* gyps_gmres_solve only: the compressed far field opts->hmat (built
                                   for this mesh and k) plus C as the Krylov loop's operator */
} gyps_prec;

/* Boundary integral equation that gyps_gmres_solve solves for sound-soft scattering. */
typedef enum {
    GYPS_FORM_SINGLE_LAYER = 0,   /* V X = F (first kind, Sec. 5.4); resonant where k^2 is an
                                     interior Dirichlet eigenvalue */
    GYPS_FORM_BRAKHAGE_WERNER = 1, /* (1/2 M + K - i eta V) X = F: the density of u = (D - i eta S) phi,
                                     uniquely solvable for every k when eta > 0 */
    GYPS_FORM_DIRECT_CFIE = 2,     /* (1/2 M + K' - i eta V) X = F: X = du/dn of the total field, the same
                                     density as the first-kind system; F from gyps_rhs_planewave_cfie */
    GYPS_FORM_EFIE = 3,            /* -T J = F (the electromagnetic listing of Sec. 5.5 with beta = 1):
                                     J the RWG coefficients (ne unknowns), F from gyps_rhs_planewave_efie */
    GYPS_FORM_EM_CFIE = 4          /* (-beta T + (1 - beta)(Id/2 - nxK)) J = F, the listing's LHS with
                                     beta = opts->eta in [0, 1]; F from gyps_rhs_planewave_emcfie */
} gyps_formulation;

/* gyps_sl_apply flags */
#define GYPS_APPLY_NO_NEAR 0x1u /* far part (1/4pi) Phi^T W G W Phi only, no correction C */

typedef struct gyps_mesh_s *gyps_mesh_t;
typedef struct gyps_precond_s *gyps_precond_t;
typedef struct gyps_hmat_s *gyps_hmat_t;  /* compressed far field (gyps_hmat_create) */

typedef struct {
    int64_t nv;          /* vertices = P1 degrees of freedom */
    int64_t nt;          /* triangles */
    int64_t nq;          /* quadrature points = q * nt */
    int32_t q;           /* points per triangle (1, 3 or 7) */
    int32_t device;      /* CUDA device the mesh lives on */
    int64_t near_pairs;  /* ordered triangle pairs sharing a vertex (a == b included) */
    int64_t near_nnz;    /* nonzeros of the correction matrix C */
    int64_t device_bytes;/* device memory held by the handle */
} gyps_mesh_info_t;

/* Library version string (static storage). */
const char *gyps_version(void);

/* Copies the calling thread's last error message into buf (NUL-terminated,
 * truncated to n bytes) and returns the last error code. */
gyps_status gyps_last_error(char *buf, size_t n);

/*
 * Mesh + quadrature domain + P1 space: msh, dom(mesh, q) and fem(mesh, 'P1')
 * of Sec. 4.1-4.3.
 *   vtx  HOST, nv x 3 doubles, row-major (x, y, z per vertex).
 *   tri  HOST, nt x 3 int32, row-major, 0-based vertex indices; the orientation
 *        does not matter to the single layer.
 *   quad_points  1 (centroid), 3 (interior points (2/3,1/6,1/6)) or 7 (Radon,
 *        degree 5): the Gauss rule of Sec. 4.2 used on both x and y.
 *   flags  0.
 * Builds on the device, on `stream`: the quadrature points and weights (Eq.
 * approxA), the vertex-to-quadrature-point incidence (Eq. WB), the list of
 * triangle pairs sharing a vertex and the correction C of Sec. 5.2 in CSR form
 * (real, independent of k).  Returns after the build finished.
 * Errors: INVALID for nv < 3, nt < 1, an index outside [0, nv), repeated
 * vertices in a triangle, a zero-area triangle, non-finite coordinates or an
 * unsupported quad_points; OOM; CUDA.
 */
gyps_status gyps_mesh_create(const double *vtx, int64_t nv, const int32_t *tri, int64_t nt,
                             int quad_points, uint32_t flags, void *stream, gyps_mesh_t *out);

/* Releases the handle and its device memory (synchronises its device first).
 * NULL is accepted. */
gyps_status gyps_mesh_destroy(gyps_mesh_t mesh);

/* Sizes of a mesh. info: HOST. */
gyps_status gyps_mesh_info(gyps_mesh_t mesh, gyps_mesh_info_t *info);

/*
 * Error word of a mesh's bounded device waits (library service; no counterpart
 * in the paper).  Every pipeline wait inside the far kernels gives up after a
 * poll limit instead of spinning forever; a wait that gives up records it in
 * the mesh's error word and its kernel returns early, so the result of that
 * launch is incomplete.  Synchronous calls (host buffers, GMRES, the double
 * layer, EFIE and potential entry points) clear the word when they start and
 * return TIMEOUT if one of their own launches set it.  Asynchronous calls
 * (device X and Y for gyps_sl_apply, gyps_sl_apply_noalloc) cannot report it:
 * gyps_mesh_check synchronises `stream`, then reads and clears the word.
 * Returns TIMEOUT if a wait gave up since the word was last cleared, else OK.
 */
gyps_status gyps_mesh_check(gyps_mesh_t mesh, void *stream);

/*
 * Poll limit of the pipeline waits in the far kernels (FP32 CUDA-core and
 * tensor-core forms of gyps_sl_apply and gyps_sl_apply_noalloc) launched after
 * this call, process-wide.  polls < 0 restores each kernel's default (about a
 * second of polling); polls = 0 makes every such wait give up at once, which
 * exercises the TIMEOUT path deterministically (tests).  The wait that drains a
 * failed launch's copies and products in flight always keeps the default.
 * Errors: INVALID for polls > 2^30.
 */
gyps_status gyps_set_wait_polls(int64_t polls);

/*
 * Quadrature points and weights (x_k, w_k) of Eq. (approxA), k = t*q + j,
 * written as nq x 4 doubles (x, y, z, w) into xw (device or host).
 */
gyps_status gyps_quad_points(gyps_mesh_t mesh, double *xw, void *stream);

/*
 * The correction matrix C of Sec. 5.2 (already multiplied by 1/(4 pi), as the
 * listing of Sec. 5.4 adds it), CSR with sorted columns.  All HOST buffers:
 * rowptr nv+1, col near_nnz, val near_nnz.  Synchronous.
 */
gyps_status gyps_near_export(gyps_mesh_t mesh, int64_t *rowptr, int32_t *col, double *val);

/*
 * Matrix-free single layer (Sec. 5, Eq. BEM, plus the Sec. 5.2 correction):
 *     Y = (1/4pi) Phi^T W_x G W_y Phi X + C X       (Y is overwritten)
 * with G_kl = exp(ik r_kl)/r_kl, and G_kk = i k for a point paired with itself
 * (the limit of the kernel minus its 1/r part, which C carries).
 *   X  nv x nrhs complex double2, leading dimension ldx >= nv.
 *   Y  nv x nrhs complex double2, leading dimension ldy >= nv (not aliasing X).
 *   nrhs  1 .. 4096.
 *   prec  gyps_prec: arithmetic of the G u product (see above).
 *   flags  GYPS_APPLY_NO_NEAR leaves C out.
 *   tri_begin, tri_end  restrict the TEST side to triangles [tri_begin,
 *        tri_end) (both -1: all).  The far part then sums only over target
 *        points of those triangles and C only over those test triangles, so
 *        applies over a partition of the triangles add up to the full apply.
 *        Every precision supports a range (the tensor-core form restricts
 *        its 128-point target tiles to the range's points).
 * Errors: INVALID (nrhs, ld, k, range), UNSUPPORTED (tensor-core precision
 * with fewer than 16 right-hand sides or k = 0), OOM, CUDA, TIMEOUT.
 * TIMEOUT (a bounded device wait gave up, Y incomplete) is returned only when
 * X or Y is a host buffer: that call is synchronous and reports the waits of
 * its own launches.  With device X and Y the call returns after launching;
 * call gyps_mesh_check after the stream's work to learn whether a wait gave up.
 */
gyps_status gyps_sl_apply(gyps_mesh_t mesh, double k, int nrhs, const void *X, int64_t ldx,
                          void *Y, int64_t ldy, int prec, uint32_t flags,
                          int64_t tri_begin, int64_t tri_end, void *stream);

/*
 * Y += C X with the correction C of Sec. 5.2 (regularize(S, S, Vh, '[1/r]', Vh)
 * times 1/(4 pi)).  X, Y: nv x nrhs complex double2 (device or host).
 */
gyps_status gyps_near_correct(gyps_mesh_t mesh, int nrhs, const void *X, int64_t ldx,
                              void *Y, int64_t ldy, void *stream);

/*
 * Dense assembly of the whole operator (the listing of Sec. 5.4:
 * LHS = integral(...)/(4 pi) + regularize(...)/(4 pi)):
 *     V = (1/4pi) Phi^T W G W Phi + C,   nv x nv complex double2,
 * column-major with ldv >= nv; V_ij pairs test function i with trial
 * function j.  prec: GYPS_PREC_FP64 (FP64 kernel values and sums, triangle
 * pairs with FP64 atomics; at most 65535 triangles) or GYPS_PREC_FP32 (FP32
 * kernel values and sums over blocks of 64 x 64 vertices along a Morton order,
 * each entry of V written once; the complex-symmetric Gauss-Gauss part is
 * computed for one block of each symmetric pair and written to both; any size
 * that fits).  Errors: INVALID, UNSUPPORTED (prec, or more than 65535
 * triangles in FP64), OOM, CUDA.
 */
gyps_status gyps_sl_assemble(gyps_mesh_t mesh, double k, int prec, void *V, int64_t ldv, void *stream);

/*
 * Galerkin double layer (the paper's grady[exp(ikr)/r] kernel with the
 * 'grady[1/r]' regularisation, Sec. 5.2, in the factorisation of Eq. (BEM)):
 *     Y = K X,  K_ij = (1/4pi) int int phi_i(x) n_y . grad_y exp(ik|x-y|)/|x-y| phi_j(y),
 *     K = (1/4pi) Phi^T W H W Phi + C_dl,  H = (1 - ikr) exp(ikr) n_y . (x - y) / r^3,
 * n_y the outward unit normal of the source triangle ((P1 - P0) x (P2 - P0)
 * for the mesh's orientation); pairs inside one flat triangle give 0 (the
 * principal value); C_dl on triangles sharing a vertex: closed-form integral
 * of lambda_j n . (x - y)/|x - y|^3 minus its Gauss sum.  On the unit sphere
 * K Y_n = (1/2 + i k^2 j_n(k) h_n'(k)) Y_n (-1/(2(2n+1)) at k = 0).
 *   X, Y  nv x nrhs complex double2 (host or device), leading dims >= nv.
 *   prec  GYPS_PREC_FP64, GYPS_PREC_FP32 (AUTO) or GYPS_PREC_DF64 for the far
 *         sum; the correction is FP64.
 * Built with its correction on the first call (then cached in the mesh).
 * Synchronous. Errors: INVALID, UNSUPPORTED (tensor-core precision), CUDA,
 * OOM, TIMEOUT.
 */
gyps_status gyps_dl_apply(gyps_mesh_t mesh, double k, int nrhs, const void *X, int64_t ldx, void *Y, int64_t ldy,
                          int prec, void *stream);

/*
 * Combined-field operator of the indirect Brakhage-Werner formulation: the
 * scattered field is sought as u = (D - i eta S) phi, with D the double-layer
 * and S the single-layer potential (1/4pi normalisation); its exterior trace
 * (jump relation of D) gives, in Galerkin form,
 *     Y = (1/2 M + K - i eta V) X,   M = Phi^T W Phi (Eq. A=BWB),
 * V the single layer of gyps_sl_apply and K the double layer of gyps_dl_apply.
 * Sound-soft scattering of u_inc solves (1/2 M + K - i eta V) phi = -F with F
 * from gyps_rhs_planewave; for eta > 0 the operator is invertible at every
 * k > 0 (no interior resonances).  On the unit sphere its eigenvalue for
 * degree-n harmonics is 1/2 + mu_n(K) - i eta mu_n(V).
 *   X, Y  nv x nrhs complex double2 (host or device), leading dims >= nv, not overlapping.
 *   prec  precision of V (as gyps_sl_apply); K takes the same precision for
 *         GYPS_PREC_FP64 and GYPS_PREC_DF64, FP32 otherwise; M is FP64.
 * Synchronous. Errors: INVALID, UNSUPPORTED (tensor cores with k = 0 or fewer
 * than 16 columns), CUDA, OOM, TIMEOUT.
 */
gyps_status gyps_bw_apply(gyps_mesh_t mesh, double k, double eta, int nrhs, const void *X, int64_t ldx,
                          void *Y, int64_t ldy, int prec, void *stream);

/*
 * Galerkin adjoint double layer (the normal derivative at the test point):
 *     Y = K' X,  K'_ij = (1/4pi) int int phi_i(x) n_x . grad_x exp(ik|x-y|)/|x-y| phi_j(y),
 * kernel -(1 - ikr) exp(ikr) n_x . (x - y) / r^3 between the Gauss points (n_x of
 * the test triangle; pairs inside one triangle give 0), plus the transpose of the
 * double layer's correction (K' = K^T for the Galerkin matrices, G being
 * symmetric).  Arguments, precisions and errors as gyps_dl_apply.
 */
gyps_status gyps_adl_apply(gyps_mesh_t mesh, double k, int nrhs, const void *X, int64_t ldx, void *Y, int64_t ldy,
                           int prec, void *stream);

/*
 * Direct combined-field operator for sound-soft scattering: Green's
 * representation u = u_inc - S (du/dn) of the total field gives on the surface
 * V du/dn = u_inc and (1/2 + K') du/dn = du_inc/dn; the combination
 *     Y = (1/2 M + K' - i eta V) X,   M = Phi^T W Phi (Eq. A=BWB),
 * is invertible at every k > 0 for eta > 0, and its solution for the right-hand
 * side of gyps_rhs_planewave_cfie is du/dn, the density of the first-kind
 * system V lambda = F of Sec. 5.4.  Arguments, precisions and errors as
 * gyps_bw_apply (K' takes the precision K would).
 */
gyps_status gyps_cfie_apply(gyps_mesh_t mesh, double k, double eta, int nrhs, const void *X, int64_t ldx,
                            void *Y, int64_t ldy, int prec, void *stream);

/*
 * RWG functions (the EFIE of the electromagnetic listing of Sec. 5.5), one per
 * edge of a closed, consistently oriented mesh.  Edges are the vertex pairs
 * (a < b) in lexicographic order; local edge j of a triangle joins its vertices
 * j+1 and j+2 (opposite P_j); the triangle where the edge runs a -> b is its plus
 * triangle.  phi(y) = s l_j / (2 A) (y - P_j), div phi = s l_j / A, s = +1 / -1.
 * gyps_rwg_edges builds the functions (and the EFIE correction) on first use and
 * returns their number; edges: HOST ne x 2 int32 vertex pairs, or NULL.
 * Errors: INVALID (open or inconsistently oriented mesh), CUDA, OOM.
 */
gyps_status gyps_rwg_edges(gyps_mesh_t mesh, int64_t *ne, int32_t *edges, void *stream);

/*
 * EFIE operator of the listing (T with its two regularize terms):
 *     Y = T X,  T = ik/(4pi) (sum_c Phi_c^T W G W Phi_c + CA) - i/(4pi k) (Dv^T W G W Dv + CB),
 * Phi_c (c = x, y, z) and Dv the RWG functions and their divergence at the Gauss
 * points, G the single layer's kernel (four density columns per right-hand side
 * through the same far sum), CA / CB the '[1/r]' corrections on triangles sharing
 * a vertex (analytic inner integrals from the P1 ones, minus the Gauss sums).
 *   X, Y  ne x nrhs complex double2 (host or device), leading dims >= ne, not overlapping.
 *   k     > 0.   prec  GYPS_PREC_FP32 (AUTO), GYPS_PREC_FP64 or GYPS_PREC_DF64.
 * Synchronous. Errors: INVALID (k <= 0, sizes, open mesh), UNSUPPORTED (tensor
 * cores), CUDA, OOM, TIMEOUT.
 */
gyps_status gyps_efie_apply(gyps_mesh_t mesh, double k, int nrhs, const void *X, int64_t ldx, void *Y, int64_t ldy,
                            int prec, void *stream);

/*
 * EFIE right-hand sides (the listing's integral(sigma, Vh, PWE)):
 *     F_ej = sum_k w_k phi_e(x_k) . p_j exp(i k d_j . x_k),
 * dirs, pols: HOST nrhs x 3 (propagation directions d_j, polarisations p_j, used
 * as given).  F: ne x nrhs complex double2, leading dimension ldf >= ne.
 */
gyps_status gyps_rhs_planewave_efie(gyps_mesh_t mesh, double k, int nrhs, const double *dirs, const double *pols,
                                    void *F, int64_t ldf, void *stream);

/*
 * MFIE part of the electromagnetic listing:
 *     Y = nxK X,  nxK_mn = (1/4pi) int int (n_x x phi_m(x)) . (grad_y exp(ik|x-y|)/|x-y| x phi_n(y))
 *                          + regularize(..., 'grady[1/r]', ...),
 * grad_y exp(ikr)/r = (1 - ikr) exp(ikr) (x - y)/r^3 between the Gauss points (pairs inside one
 * triangle give 0: their vector is normal to it), the correction on triangles sharing a vertex
 * from the closed form of int lambda (x - y)/R^3 minus its Gauss sum.  The combined operator
 *     Y = (-beta T + (1 - beta)(Id/2 - nxK)) X,   Id = int phi_m . phi_n by the mesh's rule,
 * is the listing's LHS.  X, Y: ne x nrhs (host or device), leading dims >= ne, not
 * overlapping; k > 0; prec GYPS_PREC_FP32 (AUTO), GYPS_PREC_FP64 or GYPS_PREC_DF64 (the MFIE
 * part in FP64 for DF64).  Errors as gyps_efie_apply.
 */
gyps_status gyps_mfie_apply(gyps_mesh_t mesh, double k, int nrhs, const void *X, int64_t ldx, void *Y, int64_t ldy,
                            int prec, void *stream);
gyps_status gyps_emcfie_apply(gyps_mesh_t mesh, double k, double beta, int nrhs, const void *X, int64_t ldx,
                              void *Y, int64_t ldy, int prec, void *stream);

/*
 * The listing's RHS:  F_ej = sum_k w_k (beta phi_e . p_j - (1 - beta)(n x phi_e) . (d_j x p_j))
 * exp(i k d_j . x_k)  (beta int phi . E_inc - (1 - beta) int (n x phi) . H_inc, H_inc = d x E_inc).
 * Arguments as gyps_rhs_planewave_efie; beta must be finite.
 */
gyps_status gyps_rhs_planewave_emcfie(gyps_mesh_t mesh, double k, double beta, int nrhs, const double *dirs,
                                      const double *pols, void *F, int64_t ldf, void *stream);

/*
 * Single-layer potential at points (the radiation operator of the listing in
 * Sec. 5.4: Sdom = integral(points, S2, Gxy, Vh)/(4 pi)
 * + regularize(points, S2, '[1/r]', Vh)/(4 pi)):
 *     P[i, c] = (1/4pi) sum_l G(x_i, y_l) eta_l sum_j phi_j(y_l) X[j, c] + R[i, c],
 * G = exp(ik r)/r at the mesh's Gauss points y_l (weights eta_l); R: for every
 * triangle b whose centroid lies within twice its largest centroid-vertex
 * distance of x_i, (1/4pi) sum_j (int_b lambda_j(y)/|x_i - y| dy, closed form,
 * minus the Gauss sum of lambda_j/|x_i - y_l| over b) X[v_j(b), c] (Sec. 5.2).
 *   pts   npts x 3 doubles (x, y, z per point), host or device.  A point must
 *         not coincide with a Gauss point of the mesh (the far sum would be
 *         infinite there).
 *   X     nv x nrhs complex double2 (the density, e.g. a solution of
 *         gyps_gmres_solve), leading dimension ldx.
 *   P     npts x nrhs complex double2, leading dimension ldp >= npts.
 *   prec  GYPS_PREC_FP32 (AUTO), GYPS_PREC_FP64 or GYPS_PREC_DF64 for the far
 *         sum; the regularisation is FP64.
 * npts = 0 returns at once (pts and P may then be NULL).
 * Synchronous. Errors: INVALID (sizes, NULL, non-finite host points),
 * UNSUPPORTED (tensor-core precision), CUDA, TIMEOUT.
 */
gyps_status gyps_sl_potential(gyps_mesh_t mesh, double k, int64_t npts, const double *pts, int nrhs,
                              const void *X, int64_t ldx, void *P, int64_t ldp, int prec, void *stream);

/*
 * Right-hand sides of the sound-soft example (Sec. 5.4, RHS = integral(S2, Vh,
 * PW)): F_ij = sum_k w_k phi_i(x_k) exp(i k d_j . x_k) by the mesh's rule.
 *   dirs  HOST, nrhs x 3 doubles (propagation directions d_j, used as given).
 *   F     nv x nrhs complex double2, leading dimension ldf.
 */
gyps_status gyps_rhs_planewave(gyps_mesh_t mesh, double k, int nrhs, const double *dirs,
                               void *F, int64_t ldf, void *stream);

/*
 * Right-hand sides of the direct combined-field system (gyps_cfie_apply):
 *     F_ij = sum_k w_k phi_i(x_k) (d/dn - i eta) exp(i k d_j . x_k)
 *          = sum_k w_k phi_i(x_k) i (k d_j . n - eta) exp(i k d_j . x_k),
 * n the unit normal (P1 - P0) x (P2 - P0)/|.| of the triangle of x_k.  Arguments as
 * gyps_rhs_planewave; eta must be finite.
 */
gyps_status gyps_rhs_planewave_cfie(gyps_mesh_t mesh, double k, double eta, int nrhs, const double *dirs,
                                    void *F, int64_t ldf, void *stream);

/* GMRES options (gyps_gmres_solve). */
typedef struct {
    double tol;          /* relative residual ||F - A X|| / ||F|| per column (e.g. 1e-6) */
    int32_t restart;     /* Krylov dimension m before a restart (>= 1) */
    int32_t maxit;       /* total inner iterations per call (>= 1) */
    int32_t prec;        /* gyps_prec of the operator inside the Krylov loop */
    int32_t check_prec;  /* gyps_prec of the true-residual check (GYPS_PREC_FP64 normally) */
    int32_t use_x0;      /* 1: X holds the initial guess on entry; 0: start from zero */
    int32_t max_refine;  /* refinement sweeps when the check exceeds tol (0 = none) */
    gyps_precond_t precond; /* NULL, or a learned preconditioner: flexible GMRES with z = M(q) */
    int32_t formulation; /* gyps_formulation (0: single layer) */
    double eta;          /* coupling of the combined-field operators (e.g. k); beta for GYPS_FORM_EM_CFIE */
    double timeout_ms;   /* wall-clock limit of the solve (0 = none): checked before every inner
                            iteration; when it passes, the cycle ends with the iterations done, the
                            true residual is computed and TIMEOUT is returned unless it meets tol */
    gyps_hmat_t hmat;    /* with prec = GYPS_PREC_HMAT: the compressed operator (else NULL) */
} gyps_gmres_opts;

/* GMRES report, HOST.  Arrays are caller-owned, length nrhs, may be NULL. */
typedef struct {
    int32_t iterations;      /* inner iterations done (all columns advance together) */
    int32_t applies;         /* operator applies in the working precision */
    int32_t check_applies;   /* applies in check_prec */
    int32_t refinements;     /* refinement sweeps done */
    int32_t precond_fallback;/* 2 when the network was not used: the mesh's electrical size k x radius
                                (radius: largest vertex distance from the centroid) lies outside the
                                range it was trained on, widened by 25 % (gyps_precond_range);
                                1 when the preconditioner was dropped (non-finite output or a
                                full cycle that did not halve the residual) */
    double *est_residual;    /* last Arnoldi residual estimate per column (relative) */
    double *true_residual;   /* ||F - V X||/||F|| with check_prec, per column */
    int32_t *converged;      /* 1 where true_residual <= tol */
} gyps_gmres_report;

/*
 * Solves A X = F for nrhs columns by restarted
 * GMRES, A = V (Sec. 5.4, Eq. Singlelayerwf) or, with opts->formulation =
 * GYPS_FORM_BRAKHAGE_WERNER, A = 1/2 M + K - i opts->eta V (gyps_bw_apply;
 * pass -F for the sound-soft problem), or with GYPS_FORM_DIRECT_CFIE,
 * A = 1/2 M + K' - i opts->eta V (gyps_cfie_apply; F from gyps_rhs_planewave_cfie),
 * or with GYPS_FORM_EFIE, A = -T (gyps_efie_apply; ne unknowns per column, F from
 * gyps_rhs_planewave_efie; FP32 / FP64 / double-float only), or with
 * GYPS_FORM_EM_CFIE, A = -beta T + (1 - beta)(Id/2 - nxK), beta = opts->eta
 * (gyps_emcfie_apply; F from gyps_rhs_planewave_emcfie).  Arnoldi with classical Gram-Schmidt
 * applied twice, in FP64 on the device, Givens rotations on the host, one
 * Krylov space per column, the operator applied to all columns at once with
 * `opts->prec`.  After the
 * Krylov loop the residual is recomputed with `opts->check_prec`; while it is
 * above tol and refinements remain, GMRES is run on the residual equation
 * and the correction added (mixed-precision iterative refinement).
 *   F, X  nv x nrhs complex double2 (device or host).  report: HOST or NULL.
 * With opts->precond set, the Krylov loop is flexible GMRES: each basis vector
 * q_j is mapped by the learned preconditioner, z_j = M(q_j), the operator is
 * applied to z_j and the update is X += Z y.  A non-finite z_j, or a full
 * cycle that does not halve the residual of any column, drops the
 * preconditioner for the rest of the solve (unpreconditioned GMRES from the
 * current iterate) and the report says so.  The check-precision residual judges the result either way.
 * The learned preconditioner models V: with the combined-field operators it is
 * UNSUPPORTED.
 * Returns NOT_CONVERGED (X = last iterate) when a column misses tol, TIMEOUT
 * (X = last iterate, report filled) when opts->timeout_ms passed first, NAN
 * when a non-finite value appears.
 */
gyps_status gyps_gmres_solve(gyps_mesh_t mesh, double k, int nrhs, const void *F, int64_t ldf,
                             void *X, int64_t ldx, const gyps_gmres_opts *opts,
                             gyps_gmres_report *report, void *stream);

/* ------------------------------------------------------------------------
 * Batched apply: several meshes (uneven sizes, their own k), each with nrhs
 * right-hand sides, Y_i = V_i X_i as in gyps_sl_apply (all triangles, correction
 * on).  Two forms: (a) the FP32 CUDA-core kernel products of all meshes as one
 * persistent launch over a single list of equal-cost work items (mesh, RHS
 * chunk, target tile, source tile), with one interpolation and one projection
 * launch around it; (b) with 16 or more right-hand sides and every k > 0, the
 * tensor-core apply (GYPS_PREC_TC_BF16X3) of each mesh in turn.  The batch is
 * captured once into a CUDA graph and replayed by gyps_batch_apply.  The form,
 * RHS chunk width and targets per thread come from the autotuner (timed
 * candidates, cached in the JSON file $GYPS_TUNE_CACHE, default
 * ~/.cache/gyps_tune.json) or a default (tensor cores when allowed).
 * ------------------------------------------------------------------------ */
typedef struct gyps_batch_s *gyps_batch_t;

typedef struct {
    gyps_mesh_t mesh;  /* created by gyps_mesh_create, on the batch's device */
    double k;          /* wavenumber of this mesh (finite, >= 0) */
    const void *X;     /* DEVICE, nv x nrhs complex double2, leading dimension ldx */
    int64_t ldx;
    void *Y;           /* DEVICE, nv x nrhs complex double2, leading dimension ldy */
    int64_t ldy;
} gyps_batch_item;

#define GYPS_BATCH_NO_GRAPH 0x1u /* launch the kernels on each apply instead of a captured graph */
#define GYPS_BATCH_AUTOTUNE 0x2u /* time the candidate shapes now when the cache has no entry */
#define GYPS_BATCH_CUDA_CORES 0x4u /* form (a) only: FP32 CUDA-core kernel products, no tensor cores */

typedef struct {
    int32_t nmesh, nrhs;
    int32_t rhs_chunk;          /* R: right-hand sides per pass of the kernel product */
    int32_t targets_per_thread; /* T */
    int32_t grid;               /* persistent CTAs */
    int32_t uses_graph;
    int32_t tuned;              /* 0 default shape, 1 timed now, 2 read from the cache */
    int32_t tensor_cores;       /* 1: tensor-core applies per mesh (>= 16 RHS, every k > 0) */
    int32_t reserved;
    int64_t work_items;
    double pairs;               /* sum over meshes of nq^2 (per right-hand side) */
} gyps_batch_info_t;

/*
 * Binds the items (meshes, k, X and Y buffers: the graph keeps these pointers)
 * and prepares the batch: per-mesh workspace (FP32 density panels, FP64
 * accumulators), the work list, the shape choice and the graph.  X and Y must
 * stay valid until gyps_batch_destroy; refill X and call gyps_batch_apply.
 *   items  HOST array of nitems (1..4096).  nrhs 1..4096, shared by all items.
 *   flags  GYPS_BATCH_NO_GRAPH | GYPS_BATCH_AUTOTUNE | GYPS_BATCH_CUDA_CORES.
 * Errors: INVALID (argument, host buffers, meshes on different devices), OOM, CUDA.
 */
gyps_status gyps_batch_create(const gyps_batch_item *items, int nitems, int nrhs, uint32_t flags,
                              void *stream, gyps_batch_t *out);

/* Y_i = V_i X_i for every item, asynchronously on `stream`. */
gyps_status gyps_batch_apply(gyps_batch_t batch, void *stream);

/* Shape and size of a batch. info: HOST. */
gyps_status gyps_batch_info(gyps_batch_t batch, gyps_batch_info_t *info);

/* Synchronises the device, releases the batch; TIMEOUT if a device wait of one
 * of its applies ran out of polls.  NULL is accepted. */
gyps_status gyps_batch_destroy(gyps_batch_t batch);

/* ------------------------------------------------------------------------
 * Compressed far field (Sec. 5.3: the BEM matrix assembled directly in a
 * compressed block form to a tolerance, so that larger problems fit and apply
 * faster than the dense or all-pairs forms).  One level of a cluster tree:
 * clusters are runs of `leaf_tiles` tiles of 64 vertices along a Morton curve
 * (compact surface patches); the block of the Gauss-Gauss part
 * (1/4pi) Phi^T W G W Phi between clusters A and B is stored dense (FP32
 * complex) when dist(box A, box B) < eta max(diam A, diam B), the boxes
 * covering the clusters' basis-function supports, and otherwise as U W^T from
 * the adaptive cross approximation with partial pivoting (Bebendorf 2000),
 * stopped when the newest term is below eps times the Frobenius norm of the
 * approximation and spot-checked on 256 entries; a block that does not
 * compress within min(m, n)/2 terms is kept dense.  The far part is complex
 * symmetric, so only blocks A <= B are built; (B, A) uses the transpose.
 * Blocks are generated on the device from the same Gauss-point kernel as the
 * dense assembly (FP32 kernel values); the correction C stays FP64 and sparse.
 * ------------------------------------------------------------------------ */
typedef struct {
    int64_t clusters;
    int64_t dense_blocks;     /* blocks stored dense (A <= B), fallbacks included */
    int64_t lowrank_blocks;   /* blocks stored as U W^T (A < B) */
    int64_t fallback_blocks;  /* admissible blocks that did not compress (kept dense) */
    int32_t max_rank;
    int32_t reserved;
    double mean_rank;
    int64_t bytes;            /* device memory held (blocks, factors, plan, workspaces) */
    double dense_bytes;       /* the full nv x nv FP32 complex matrix, for comparison */
    double build_ms;          /* wall time of gyps_hmat_create */
} gyps_hmat_info_t;

/*
 * Builds the compressed far part of V for wavenumber k on `mesh` (synchronous).
 *   eps  relative tolerance of the low-rank blocks, 1e-7 <= eps < 1.
 *   leaf_tiles  tiles (of 64 vertices) per cluster, 1..64.
 *   eta  admissibility parameter (> 0; larger = fewer, farther low-rank blocks).
 * Errors: INVALID, OOM (the blocks did not fit), CUDA.
 */
gyps_status gyps_hmat_create(gyps_mesh_t mesh, double k, double eps, int leaf_tiles, double eta, void *stream,
                             gyps_hmat_t *out);

/*
 * Y = (H + C) X: the compressed far part plus the FP64 correction, nrhs
 * columns (1..4096) of nv complex double2, leading dimensions >= nv, X and Y
 * not overlapping.  Device buffers: asynchronous on `stream`; host buffers:
 * staged, returns when Y is on the host.  X is rounded to FP32 for the block
 * products; the sums of a row are carried as error-free FP32 pairs and written
 * in FP64.  Errors: INVALID, OOM, CUDA.
 */
gyps_status gyps_hmat_apply(gyps_hmat_t h, int nrhs, const void *X, int64_t ldx, void *Y, int64_t ldy,
                            void *stream);

/* Sizes, ranks, memory and build time. info: HOST. */
gyps_status gyps_hmat_info(gyps_hmat_t h, gyps_hmat_info_t *info);

/* Releases the blocks (synchronises the device first). NULL is accepted. */
gyps_status gyps_hmat_destroy(gyps_hmat_t h);

/*
 * gyps_sl_apply without any device allocation (the paper has no counterpart:
 * this is a library service).  For callers that must not allocate device
 * memory while they run - their device memory is owned by another allocator,
 * or a cudaMalloc, and the device-wide synchronisation it can cause, is not
 * acceptable inside their loop.  Computes the same
 *     Y = (1/4pi) Phi^T W_x G W_y Phi X + C X
 * as gyps_sl_apply with prec = GYPS_PREC_FP32, all triangles, correction on.
 *   X, Y  DEVICE, nv x nrhs complex double2 (leading dimensions ldx, ldy >= nv),
 *         not overlapping; host pointers are rejected (INVALID).
 * Scratch: a fixed 8 MiB device array inside the library, held on every GPU
 * that loads it until the process exits; one column needs about 28 bytes per
 * quadrature point (meshes with nq up to about 290000).  A larger mesh is
 * rejected with INVALID and a message giving the bytes needed.  Nothing is
 * allocated: the call launches kernels and clears the accumulators it needs
 * (cudaMemsetAsync) on `stream`, then returns.
 * The first call on each device looks up the array's device address; make that
 * first call before any stream capture.  All calls share the one array and it
 * keeps the previous call's contents: calls whose work overlaps on the GPU
 * (other streams, other threads) race and corrupt each other's results;
 * order them on one stream.
 * The call returns after launching, so it cannot return TIMEOUT: a bounded
 * device wait that gave up is reported by gyps_mesh_check.
 */
gyps_status gyps_sl_apply_noalloc(gyps_mesh_t mesh, double k, int nrhs, const void *X, int64_t ldx,
                                  void *Y, int64_t ldy, void *stream);

/* ------------------------------------------------------------------------
 * Learned preconditioner (no counterpart in the paper): a message-passing
 * network on the P1 mesh graph mapping a residual r to z ~ V^{-1} r, for
 * flexible GMRES.  Per vertex i the inputs are r_i / rms(r) (re, im), the
 * centred and scaled coordinates, the unit vertex normal and k h (h: mean edge
 * length); h0 = relu(W_in f + b_in); `layers` times
 * h += relu(Ws h + Wn mean_{j ~ i} h_j + b); y = W_out h + b_out (2 values);
 * z_i = (y_i0 + i y_i1) rms(r) / h^3.  bf16 weights in the forward, FP32
 * activations and sums, FP32 master weights and Adam moments.
 * ------------------------------------------------------------------------ */

/* hidden must be 64; layers 1..16; weights from a counter-based generator
 * seeded by `seed` (uniform, scaled by 1/sqrt(fan in)), biases zero. */
gyps_status gyps_precond_create(int hidden, int layers, uint64_t seed, gyps_precond_t *out);
gyps_status gyps_precond_destroy(gyps_precond_t p);

/* Size and Adam step count of the network. Any output pointer may be NULL. */
gyps_status gyps_precond_info(gyps_precond_t p, int *hidden, int *layers, int64_t *nparams, int64_t *steps);

/* Copies the FP32 parameters out of (direction 0) or into (direction 1) the
 * network; host buffer of gyps_precond_info's nparams floats, in the order
 * W_in (9 x H), b_in, per layer Ws (H x H), Wn (H x H), b (H), W_out (H x 2),
 * b_out (2); matrices input-major. */
gyps_status gyps_precond_params(gyps_precond_t p, float *host, int64_t n, int direction);

/* Z = M(R) for nrhs residuals of one mesh.  R, Z: DEVICE, nv x nrhs complex
 * double2.  Asynchronous on stream. */
gyps_status gyps_precond_apply(gyps_precond_t p, gyps_mesh_t mesh, double k, int nrhs, const void *R, int64_t ldr,
                               void *Z, int64_t ldz, void *stream);

/* One minibatch of training: nrhs (1..64) residuals R of one mesh and their
 * corrections E (E ~ V^{-1} R), loss = mean over columns of |M(r)-e|^2/|e|^2.
 * Computes the gradient; with lr > 0 takes one Adam step (beta 0.9, 0.999,
 * eps 1e-8).  loss (HOST, may be NULL) receives the loss before the step,
 * grad (HOST, nparams floats, may be NULL) the gradient.  R, E: device or host.
 * Synchronous. */
gyps_status gyps_precond_train_step(gyps_precond_t p, gyps_mesh_t mesh, double k, int nrhs, const void *R,
                                    int64_t ldr, const void *E, int64_t lde, double lr, double *loss,
                                    float *grad, void *stream);

/* Range [ka_lo, ka_hi] of the electrical sizes k x radius of the meshes that
 * gyps_precond_train_step has seen (ka_lo > ka_hi: none yet).  Flexible GMRES
 * uses the network only inside this range widened by 25 % (the network's
 * inputs carry k h, not the size of the body in wavelengths). */
gyps_status gyps_precond_range(gyps_precond_t p, double *ka_lo, double *ka_hi);

/* Checkpoint: parameters and Adam moments with a JSON header (format
 * "gyps-mpnn-1", with the training range).  load checks the shape and rejects
 * non-finite values; a file without a range loads as untrained-range. */
gyps_status gyps_precond_save(gyps_precond_t p, const char *path);
gyps_status gyps_precond_load(gyps_precond_t p, const char *path);

/* Device-time profile of the matrix-free applies of one mesh. */
typedef struct {
    int64_t applies;      /* gyps_sl_apply calls recorded since profiling was enabled */
    int64_t launches;     /* kernels those applies launched */
    double interp_ms;     /* summed device time of the W_y Phi X step */
    double far_ms;        /* ... of the dense G u step (Eq. BEM) */
    double project_ms;    /* ... of Phi^T W_x v (+ the CSR correction C X) */
    double near_ms;       /* ... of the correction over a partial triangle range */
    int64_t far_launches; /* launches of the dense G u kernel */
} gyps_profile_t;

/*
 * Turns per-stage timing of gyps_sl_apply on (enable = 1) or off (0) for one
 * mesh; enabling resets the totals.  While on, each apply records CUDA events
 * before and after every stage on the stream it runs on.
 */
gyps_status gyps_profile_enable(gyps_mesh_t mesh, int enable);

/*
 * Waits for the recorded events, adds their durations to the totals and
 * copies the totals into out (HOST).
 */
gyps_status gyps_profile_read(gyps_mesh_t mesh, gyps_profile_t *out);

#ifdef __cplusplus
}
#endif

#endif /* GYPS_H */
