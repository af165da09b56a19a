/*
 * mbs.h - C ABI of the GB300 multibody scattering library.
 *
 * The library solves the multibody sound-soft scattering problem with local
 * MFS scattering matrices (Cai, Bagge, Martinsson, "A stable and fast method
 * for solving multibody scattering problems via the method of fundamental
 * solutions"):
 *
 *     (I + S G_hat) q_hat = S v_hat                        (Sec. 2.2, eq. mbody2)
 *
 * where S = diag(S_tau) holds one k_tau x k_tau scattering matrix per body
 * (Sec. 4.5, eq. scattering-matrix), G_hat(i, j) = phi_kappa(x_hat_i - x_hat_j)
 * between skeleton points of different bodies (Sec. 1, eq. Gmtx-entries) and
 * phi_kappa is (i/4) H0^(1)(kappa r) in 2D, exp(i kappa r) / (4 pi r) in 3D
 * (Sec. 3.1, eq. FundamentalSol).
 *
 * Conventions shared by every call
 * --------------------------------
 *  - Complex arrays are interleaved (re, im) doubles.  A block of nrhs
 *    vectors of length L is column-major: element (i, r) is at
 *    [2 * (r * L + i)] (re) and [2 * (r * L + i) + 1] (im).
 *  - Point sets are structure-of-arrays: coordinate c of point i of a set of
 *    L points is at [c * L + i].
 *  - Every array argument may be a host pointer or a CUDA device pointer of
 *    the current device; the library tells them apart with
 *    cudaPointerGetAttributes.  Host buffers are copied in and out inside the
 *    call; device buffers are used in place on the context's stream, and the
 *    call returns after the stream has finished with them.
 *  - The caller keeps ownership of every buffer it passes; the library copies
 *    what it needs.  The library owns the context and all device memory it
 *    allocates; mbs_destroy releases it.
 *  - Every call returns an mbs_status; no exception crosses the ABI.  On an
 *    error the context keeps its previous valid state and mbs_last_error()
 *    describes the failure.  Calls on one context are serialised by a
 *    per-context mutex; different contexts may be used from different
 *    threads.
 */
#ifndef MBS_H
#define MBS_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum mbs_status {
    MBS_OK = 0,
    MBS_ERR_ARG = 1,          /* invalid argument: size, null pointer, NaN/Inf input */
    MBS_ERR_GEOMETRY = 2,     /* a body reaches inside another body's proxy surface */
    MBS_ERR_NOMEM = 3,        /* device allocation failed or the HBM budget is exceeded */
    MBS_ERR_CUDA = 4,         /* a CUDA runtime call failed */
    MBS_ERR_NOCONV = 5,       /* the solve hit max_iter / max_sweeps; q_hat holds the best iterate */
    MBS_ERR_TIMEOUT = 6,      /* a bounded device-side wait ran out */
    MBS_ERR_NEAR_TARGET = 7,  /* an evaluation target lies inside a proxy surface */
    MBS_ERR_STATE = 8,        /* call out of order (e.g. solve before build) */
    MBS_ERR_UNSUPPORTED = 9   /* option combination not implemented */
} mbs_status;

enum {
    MBS_PREC_FP64 = 0,   /* every step in FP64 */
    MBS_PREC_MIXED = 1,  /* FP32 G_hat/S/Krylov inside FP64 iterative refinement */
    MBS_PREC_FP32 = 2    /* apply calls only: the FP32 operator itself */
};

typedef struct mbs_options {
    int precision;       /* MBS_PREC_FP64 or MBS_PREC_MIXED (solve); apply calls accept FP32 too */
    double tol;          /* stop when ||b - A q||_2 / ||b||_2 <= tol for every RHS (FP64 residual) */
    double inner_tol;    /* mixed precision: relative residual target of each FP32 inner solve */
    int restart;         /* GMRES restart length (Krylov vectors kept per RHS), 1..1800 */
    int max_iter;        /* cap on Arnoldi steps summed over the whole solve */
    int max_sweeps;      /* mixed precision: cap on refinement sweeps */
    double ls_rcond;     /* relative truncation of the least-squares solves in the S build */
    void* stream;        /* cudaStream_t to run on, or NULL for a stream the context creates */
    size_t hbm_budget;   /* bytes of device memory the context may hold (0 = no cap) */
    int tile_override;   /* 0 = tuned launch shape; >0 forces the source-split count of G_hat */
    int block_krylov;    /* 1 (default): several right-hand sides share one block Krylov space; 0: independent GMRES in lockstep */
    int mac_path;        /* FP32 G_hat kernel: 0 auto (3 for >= 4 RHS, else 1), 1 FP32 pipe, 2 mma.sync tensor-core multiply-add (3xTF32), 3 tcgen05 tensor-core multiply-add (3xTF32, accumulators in tensor memory) */
    int autotune;        /* 1 (default): the first FP32 G_hat matvec of a problem class times the candidate
                            launch shapes (kernel path x source-split count) and the fastest is reused process-wide;
                            0: heuristic shape */
    int cuda_graphs;     /* 1 (default): after one direct step, the device work of each block-GMRES step is
                            captured once per context and step index and replayed as a CUDA graph; 0: launch directly */
    int fp64_kernel;     /* FP64-accurate G_hat (FP64 solves, refinement residuals, apply calls):
                            0 on the FP64 pipe; 1 in double-float arithmetic on the FP32 pipe, with FP64
                            work only per body pair (3.4x faster than 0 on GB300 at N = 64,000, 8 RHS;
                            ~1e-13 relative instead of ~1e-16); 2 (default) automatic: inside solves
                            double-float when 1e-14 ||S||_F (the FP64 residual floor it leaves, with the
                            root mean square of ||S_tau||_F over the bodies) is at most tol / 10, else
                            the FP64 pipe; apply calls use the FP64 pipe */
    int sbuild_threads;  /* threads per CTA of the S build (128, 256 or 512); 0 (default): 256 (the build
                            is FP64-pipe-bound: the three sizes measured within 2 % on GB300); -1: tuned on the
                            first build of a size class (when autotune is on), at the cost of ~half a build */
    int id_sketch;       /* randomized ID (Sec. 4.2, the ID framework the paper cites): > 0 takes the
                            skeleton and Z* of each fixed-k shape from the pivoted QR of the sketch
                            Omega B with k + id_sketch rows (Omega complex Gaussian from Philox4x32-10,
                            key (id_seed, shape index)), when that is fewer than B's p rows; 0 (default):
                            the pivoted QR of B itself */
    unsigned int id_seed; /* generator key of the sketch */
} mbs_options;

typedef struct mbs_shape {
    int m;               /* collocation points on Gamma (Sec. 3.1) */
    int n;               /* MFS sources inside Gamma, n < m (Sec. 3.1) */
    int p;               /* proxy points on Psi (Sec. 4.2) */
    const double* x;     /* m collocation points, local frame, SoA (dim * m) */
    const double* y;     /* n MFS sources, SoA (dim * n) */
    const double* z;     /* p proxy points, SoA (dim * p) */
    int k;               /* fixed skeleton count (k <= min(m, p)), or 0: stop the pivoted QR at eps */
    double eps;          /* relative stopping tolerance of the pivoted QR when k == 0 */
    double proxy_radius; /* radius of the proxy circle/sphere about the local origin */
} mbs_shape;

typedef struct mbs_body {
    int shape;           /* index into the shapes array */
    double c[3];         /* centre (world frame); c[2] ignored in 2D */
    double R[9];         /* row-major rotation, x_world = c + R x_local; 2D uses R[0], R[1], R[3], R[4] */
} mbs_body;

typedef struct mbs_solve_info {
    int inner_iterations; /* Arnoldi steps, summed over RHS batches and sweeps */
    int sweeps;           /* refinement sweeps (mixed) or restart cycles (FP64) */
    int matvecs_fp32;     /* FP32 operator applications (each covers all RHS) */
    int matvecs_fp64;     /* FP64 operator applications (each covers all RHS) */
    int converged;        /* 1 if every RHS reached tol */
    int fp64_finish;      /* mixed: 1 if refinement stopped contracting (or ran out of sweeps)
                             and FP64 GMRES, warm-started from the refined iterate, finished */
    double rel_residual;  /* max over RHS of the final FP64 relative residual */
    double seconds;       /* wall time of the call */
    int fp64_kernel;      /* FP64-accurate G_hat the solve used: 0 FP64 pipe, 1 double-float */
} mbs_solve_info;

typedef struct mbs_ctx mbs_ctx;

/* Fill *opt with defaults: FP64, tol 1e-11, inner_tol 1e-6, restart 60,
 * max_iter 20000, max_sweeps 8, ls_rcond 1e-14, stream NULL, no budget,
 * automatic G_hat kernel, autotuning and CUDA graphs on, automatic choice of the
 * FP64-accurate G_hat (fp64_kernel 2). */
void mbs_default_options(mbs_options* opt);

/* Create a context for dimension dim (2 or 3) and wavenumber kappa > 0
 * (Sec. 2.1, eq. BVP).  opt may be NULL for defaults.  Errors: MBS_ERR_ARG,
 * MBS_ERR_CUDA. */
mbs_status mbs_create(int dim, double kappa, const mbs_options* opt, mbs_ctx** out);

/* Release the context and all its device memory.  NULL is a no-op. */
void mbs_destroy(mbs_ctx* ctx);

/* Replace the options of a live context (precision, tolerances, stream...). */
mbs_status mbs_set_options(mbs_ctx* ctx, const mbs_options* opt);

/* Text of the last error on this context ("" if none); owned by the context. */
const char* mbs_last_error(const mbs_ctx* ctx);

/*
 * build_scattering_matrices(bodies, kappa)  (Sec. 4.2-4.5).
 * For every shape used by a body: B(i,j) = phi(z_i - x_j) (p x m), its column-
 * pivoted QR halted at k (or eps) gives the skeleton I_hat and Z* with
 * B ~ B(:, I_hat) Z* (eq. B_fac); A(i,j) = phi(x_i - y_j) (m x n) and
 * D(i,j) = phi(z_i - y_j) (p x n) give the local solve A^+ and the translation
 * C with B C = D; S = Z* C A^+ U with U = (Z*)^T (eq. scattering-matrix).
 * A^+ is the truncated-SVD pseudo-inverse (singular values above ls_rcond
 * times the largest; pivoted QR, then one-sided Jacobi on the triangular
 * factor), C the minimum-norm least-squares solution on the rank of the
 * pivoted QR of B truncated at ls_rcond (complete orthogonal decomposition;
 * Sec. 3.1 "truncated SVD or QR", Sec. 4.4 "stabilized").
 * Bodies are rigid placements of shapes (S is reused per shape, Sec. 5.1
 * Example 4).  All of it runs on the device in FP64.
 * Errors: MBS_ERR_ARG (n >= m, k > min(m,p), NaN, bad shape index),
 * MBS_ERR_GEOMETRY (some point of a body inside another body's proxy radius),
 * MBS_ERR_NOMEM, MBS_ERR_CUDA.
 */
mbs_status mbs_build_scattering_matrices(mbs_ctx* ctx, int nshapes, const mbs_shape* shapes,
                                          int nbodies, const mbs_body* bodies);

/* Layout of q_hat: *N = sum_tau k_tau; body_offsets (nbodies + 1 entries,
 * nullable) gives the first skeleton of each body; skel_xyz (dim * N, SoA,
 * nullable) the world coordinates x_hat.  Outputs are caller-allocated. */
mbs_status mbs_get_layout(mbs_ctx* ctx, int64_t* N, int64_t* body_offsets, double* skel_xyz);

/* Scattering data of one shape as built: *k, skel (k indices into the
 * shape's collocation points, nullable), S (k x k complex, column-major,
 * nullable), eps_achieved (nullable: largest remaining column norm of B over
 * its largest initial column norm when the QR stopped). */
mbs_status mbs_get_shape(mbs_ctx* ctx, int shape, int* k, int* skel, double* S,
                         double* eps_achieved);

/* Figures of one shape's build (Sec. 3.1, 4.3-4.4; all outputs nullable):
 * *rank_b = steps of the pivoted QR of B (the rank on which C is the
 * minimum-norm solution), *rank_a_qr = steps of the pivoted QR of A ahead of
 * its SVD, *rank_a = singular values of A kept (above ls_rcond times the
 * largest; the rank of A^+), *sweeps = one-sided Jacobi sweeps that computed
 * the SVD, *s_norm = Frobenius norm of S.  MBS_ERR_STATE for a shape holding
 * injected data. */
mbs_status mbs_get_shape_stats(mbs_ctx* ctx, int shape, int* rank_b, int* rank_a_qr, int* rank_a,
                               int* sweeps, double* s_norm);

/*
 * Right-hand side b = S v_hat, evaluated as Z* C A^+ v from the boundary data
 * v = -u_inc at all m collocation points of each body (Sec. 4.5, last
 * display).  v: (sum_tau m_tau) x nrhs complex, bodies in order; b: N x nrhs.
 */
mbs_status mbs_rhs(mbs_ctx* ctx, int nrhs, const double* v, double* b);

/* apply_operator(q_hat): y = q_hat + S G_hat q_hat (eq. mbody2), N x nrhs,
 * in the context's precision (FP32 evaluates G_hat and S in single precision
 * with FP32 accumulation; inputs and outputs stay FP64). */
mbs_status mbs_apply_operator(mbs_ctx* ctx, int nrhs, const double* qhat, double* y);

/* y = G_hat q (N x nrhs), precision MBS_PREC_FP64 or MBS_PREC_FP32 (Sec. 2.2). */
mbs_status mbs_apply_G(mbs_ctx* ctx, int precision, int nrhs, const double* q, double* y);

/*
 * solve(v_hat) -> q_hat: GMRES on (I + S G_hat) q_hat = b (Sec. 2.4), in FP64
 * or as FP32 GMRES inside FP64 iterative refinement (precision option).  In
 * refinement every sweep solves the scaled FP64 residual in FP32 to
 * max(inner_tol, min(0.1, 0.5 tol / residual)) (the last sweep only as far as
 * tol still needs); when a sweep fails to halve the residual, or max_sweeps
 * runs out, FP64 GMRES finishes from the refined iterate (info->fp64_finish).
 * b: N x nrhs.  qhat: on entry the initial guess (all zeros allowed; a
 * previous solve's result resumes it); on exit the solution (the best iterate
 * on MBS_ERR_NOCONV).  info nullable.
 */
mbs_status mbs_solve(mbs_ctx* ctx, int nrhs, const double* b, double* qhat, mbs_solve_info* info);

/*
 * evaluate_field(points): scattered field u(t) = sum_i phi(t - x_hat_i) q_hat_i
 * (Sec. 4.1, eq. out_skel) at M targets (SoA dim * M), in FP64.  Every target
 * must lie on or outside every proxy surface; otherwise MBS_ERR_NEAR_TARGET
 * (for targets inside a proxy use mbs_evaluate_field_near).  u: M x nrhs.
 */
mbs_status mbs_evaluate_field(mbs_ctx* ctx, int nrhs, int64_t M, const double* pts,
                              const double* qhat, double* u);

/*
 * Full local solution on the MFS curves (Sec. 4.6, reconstruction on
 * Gamma^mfs):  q_mfs_tau = A_tau^+ (v_tau - U_tau G_hat_{tau,tau^c} q_hat_{tau^c}),
 * the incoming field from the other bodies taken at tau's skeleton points and
 * interpolated to its collocation points by U_tau = (Z*_tau)^T (Sec. 4.3,
 * eq. inc_field), A^+ the truncated pivoted-QR solve of the build.
 * v: sum_tau m_tau x nrhs boundary data (as for mbs_rhs); qhat: N x nrhs;
 * qmfs (out): sum_tau n_tau x nrhs, body tau's n_tau rows in body order.
 * Needs the built scattering data: MBS_ERR_STATE after mbs_inject_scattering.
 */
mbs_status mbs_reconstruct(mbs_ctx* ctx, int nrhs, const double* v, const double* qhat, double* qmfs);

/*
 * Scattered field at M targets anywhere outside the MFS curves (Sec. 4.6):
 * a target inside the proxy surface of body tau gets tau's field from its MFS
 * sources qmfs (mbs_reconstruct) plus the skeleton sums (Sec. 4.1,
 * eq. out_skel) of all other bodies; any other target gets the skeleton sums
 * of every body, as in mbs_evaluate_field.  pts: SoA dim x M; u: M x nrhs.
 * Targets on or inside an MFS curve are the caller's responsibility (the
 * representation is singular there).
 */
mbs_status mbs_evaluate_field_near(mbs_ctx* ctx, int nrhs, int64_t M, const double* pts,
                                   const double* qhat, const double* qmfs, double* u);

/*
 * Test hook: replace the built scattering data of one shape with externally
 * computed data (e.g. the CPU reference), isolating the global solve.
 * skel: k indices into the shape's collocation points; S: k x k complex;
 * W: k x m complex (b_tau = W v_tau), or NULL to keep the built right-hand
 * side operator (if the skeleton changes without W, mbs_rhs then fails with
 * MBS_ERR_STATE).  The skeleton coordinates of every body are recomputed once,
 * by the next call that uses the layout, so many shapes can be injected in a
 * row at the cost of one layout rebuild.
 */
mbs_status mbs_inject_scattering(mbs_ctx* ctx, int shape, int k, const int* skel,
                                 const double* S, const double* W);

/* Measure device peaks with short microbenchmarks: out[0] FP32 FMA TFLOP/s,
 * out[1] FP64 FMA TFLOP/s, out[2] MUFU (sin+cos+rsqrt) Tops/s, out[3] SM
 * count, out[4] SM clock kHz, out[5] FP32 TFLOP/s with packed f32x2 FMAs.
 * out must hold 6 doubles.  Runs on the current device. */
mbs_status mbs_measure_peaks(double* out);

/*
 * y = G_hat q in FP64 without allocating device memory (the paper has no
 * counterpart: this is an interface for callers that must not allocate once
 * they run, e.g. applications that hand out all GPU memory from their own
 * fixed pool, or real-time loops where a cudaMalloc that may synchronise the
 * device is not allowed).  No context is needed; every array is a device
 * pointer owned by the caller:
 *   body_offsets  T + 1 int64, first skeleton point of each body (sorted by body),
 *   body          N int32, body index of each point,
 *   xw            dim * N doubles, world coordinates, SoA,
 *   q, y          N x nrhs complex (interleaved, column-major).
 * Work is queued on `stream` (NULL = legacy default stream) and the call
 * returns without waiting.  Scratch lives in one static 64 MiB device array
 * per GPU that loads the library, held until the process exits, so
 * N * nrhs must not exceed 4,194,272 (else MBS_ERR_ARG, nothing launched).
 * The first call on a device looks up the array's device address (make it
 * before any stream capture); calls that overlap on the GPU share the array
 * and race.  No cudaMalloc, cudaFree or allocating library routine is called.
 * Errors: MBS_ERR_ARG (sizes, non-device pointers), MBS_ERR_CUDA.
 */
mbs_status mbs_apply_G_noalloc(int dim, double kappa, int64_t N, int T, const int64_t* body_offsets,
                               const int* body, const double* xw, int nrhs, const double* q,
                               double* y, void* stream);

/* ---- instrumentation ---- */

/* Number of CUDA kernels the library has launched in this process (all
 * contexts), for launch accounting around a timed region. */
int64_t mbs_launch_count(void);

/* enable != 0: bracket every G_hat kernel launch of this context with CUDA
 * events on the context's stream (the split reduction is not included). */
mbs_status mbs_profile(mbs_ctx* ctx, int enable);

/* Sum the bracketed G_hat kernel times since the last call and reset:
 * out[0] = total ms of FP32 G_hat launches, out[1] = their count,
 * out[2] = total ms of FP64 G_hat launches, out[3] = their count,
 * out[4] = kernel path of the latest FP32 G_hat (mac_path numbering; 0 if
 * none), out[5] = its source-split count, out[6] = threads per CTA of the
 * latest S build (0 if none).  out must hold 7 doubles.
 * Synchronises the context's stream. */
mbs_status mbs_kernel_times(mbs_ctx* ctx, double* out);

/* ---- serving: continuous batching of independent solves (one GPU) ---- */
typedef struct mbs_server mbs_server;

typedef struct mbs_request {
    int dim;
    double kappa;
    int nshapes;
    const mbs_shape* shapes;
    int nbodies;
    const mbs_body* bodies;
    int nrhs;
    const double* v;      /* (sum m) x nrhs boundary data, host memory, copied at submit */
    double tol;           /* relative residual target */
    int fp64;             /* 1: the plain FP64 path; 0: mixed precision (FP32 GMRES inside FP64
                             refinement) */
    int max_iter;         /* inner iteration cap of the solve (0: the library default); a request
                             that reaches it finishes with done = 1 and converged = 0 */
} mbs_request;

typedef struct mbs_request_result {
    int done;             /* 0 queued/running, 1 finished, -1 failed */
    mbs_status status;
    int64_t N;
    double rel_residual;
    int inner_iterations;
    double t_submit, t_start, t_end;   /* seconds on the server's clock */
    int converged;        /* 1 if the solve reached tol */
    double dev_start, dev_end;  /* the request's device work: CUDA events recorded on its stream
                                   before its first and after its last kernel, seconds after the
                                   server's creation (device clock) */
    double g_busy_ms;     /* its G_hat kernel time (events around every G_hat launch) */
} mbs_request_result;

/* Create a server with max_active concurrent solves and an HBM budget in
 * bytes (0 = 90 % of free device memory).  Requests are admitted in arrival
 * order when their estimated footprint fits and a slot is free; admitted
 * solves advance in an interleaved way on separate CUDA streams. */
mbs_status mbs_serve_create(int max_active, size_t hbm_budget, mbs_server** out);
/* Queue a request; *id receives its handle.  Inputs are copied. */
mbs_status mbs_serve_submit(mbs_server* srv, const mbs_request* req, int64_t* id);
/* Poll (non-blocking) the state of a request; if it is done and qhat is not
 * NULL, copy its solution (N x nrhs complex, host memory) there. */
mbs_status mbs_serve_poll(mbs_server* srv, int64_t id, mbs_request_result* res, double* qhat);
/* Admission order: 0 (default) arrival order; 1 shortest estimated work first
 * (pairs x iteration-independent cost of the S build and the operator), which
 * lets small requests pass large ones that are still queued. */
mbs_status mbs_serve_set_policy(mbs_server* srv, int policy);
/* Block until every submitted request has finished. */
mbs_status mbs_serve_drain(mbs_server* srv);
/* Stop the worker thread and free everything. */
void mbs_serve_destroy(mbs_server* srv);

#ifdef __cplusplus
}
#endif

#endif /* MBS_H */
