/*
 * msg_mimc.h -- C ABI of the GB300 MSG-MIMC hot path (arXiv:1907.12334).
 *
 * One sample of the method is: draw xi ~ N(0,1), form the Gaussian field
 * Z = Phi diag(sqrt(lambda)) xi, set a = exp(Z), solve -div(a grad u) = 1 on
 * [0,1]^2 (u = 0 on the boundary, Sec. 1 Eq. (1.1)) by Full Multiple
 * Semi-Coarsened multigrid (Sec. 2, Algorithms 1 and 2) on every grid
 * G^(p,q), 1 <= p <= P, 1 <= q <= Q, of the semi-coarsened hierarchy
 * (Eq. (2.1)), take the quantity of interest on each grid (Sec. 4) and form
 * the multi-index differences (Sec. 3, Eq. (3.2)) and the estimator term Y
 * (Eq. (3.6)).
 *
 * Conventions for every entry point:
 *   - pointers marked [device] are device memory owned by the caller (for
 *     example allocated through PyTorch); the library never allocates them,
 *     never frees them and keeps no reference after the call returns;
 *   - pointers marked [host] are host memory read during the call only;
 *   - work is enqueued on `stream` (a cudaStream_t passed as void*, NULL for
 *     the legacy default stream) and the call returns without waiting for it;
 *     results are valid once the stream is synchronised.  Host arrays are read
 *     before the call returns (their contents go through the library's own
 *     pinned staging).  Exceptions: msg_solve_batch synchronises `stream` while
 *     it runs (its schedule reads per-step convergence counts on the host), and
 *     mimc_differences_noalloc and msg_cycle_history return after their work
 *     has finished;
 *   - the return value is MSG_OK or an error code; on error
 *     msg_last_error() returns a description (thread-local string);
 *   - no entry point traps or aborts; per-sample numerical failures are
 *     reported in the per-sample status words.
 */
#ifndef MSG_MIMC_H
#define MSG_MIMC_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* return codes */
#define MSG_OK 0
#define MSG_ERR_INVALID 1     /* bad argument (size, shape, null pointer, parameter) */
#define MSG_ERR_WORKSPACE 2   /* workspace smaller than msg_workspace_bytes() */
#define MSG_ERR_CUDA 3        /* a CUDA runtime call failed */
#define MSG_ERR_UNSUPPORTED 4 /* option not built or not supported on this device */
#define MSG_ERR_TIMEOUT 5     /* a bounded wait inside a library kernel ran out (see msg_device_status) */

/* per-sample status bits written by msg_solve_batch */
#define MSG_SAMPLE_NOT_CONVERGED 1 /* some grid hit max_cycles before eps */
#define MSG_SAMPLE_NONFINITE 2     /* a residual norm became NaN or Inf */

/* arithmetic of the inner multigrid cycles */
#define MSG_PREC_FP64 0  /* every step in FP64 */
#define MSG_PREC_MIXED 1 /* cycles in FP32; outer residual, update, interpolation, QoI in FP64 */

/* quantity of interest (Sec. 4) */
#define MSG_QOI_INTEGRAL 0 /* integral of u over D, trapezoid rule */
#define MSG_QOI_POINT 1    /* Q1 = u(1/2,1/2) */
#define MSG_QOI_SUBDOMAIN 2 /* Q2 = mean of u over [1/4,1/2]^2, 2-D trapezoid (NaN if p<2 or q<2) */
#define MSG_QOI_FLUX 3     /* Q3 = -int_0^1 a(1,y) du/dx(1,y) dy, trapezoid + one-sided difference */

/* coefficient of a coarse grid's face (Sec. 2, direct discretisation) */
#define MSG_COEF_SERIES 0 /* series (harmonic) mean of the finest-face values the face covers */
#define MSG_COEF_INJECT 1 /* a = exp(Z) at the coarse face midpoint */

/* KL contraction arithmetic */
#define MSG_GEMM_FP64 0  /* FP64 products and sums */
#define MSG_GEMM_BF16X3 1 /* tensor cores: bf16 hi/lo splits, hi*hi + hi*lo + lo*hi, FP32 accumulate */
#define MSG_GEMM_FP32 2  /* FP32 products and sums (SIMT) */
#define MSG_GEMM_TF32 3  /* tensor cores: both operands rounded to TF32, one product per term, FP32 accumulate */

/* Solver parameters (Sec. 2 and its numerical setup: W(2,2) cycles, mu = 2,
 * red-black Gauss-Seidel, damping omega of the coarse-grid correction,
 * adaptive nu_0 until ||r||/||b|| <= eps on each grid). */
typedef struct {
    int32_t mu;         /* 1 = V-cycle, 2 = W-cycle */
    int32_t nu1, nu2;   /* pre- and post-smoothing sweeps, 0..64 each, nu1 + nu2 >= 1 */
    int32_t max_cycles; /* cap on cycles per grid */
    double eps;         /* relative residual target per grid */
    double omega;       /* damping of the coarse-grid correction */
    int32_t precision;  /* MSG_PREC_* */
    int32_t qoi;        /* MSG_QOI_* */
    int32_t coef;       /* MSG_COEF_*: coarse-face coefficient */
    int32_t tune_block; /* launch shape: threads per CTA of the visit kernels (0: 128; multiple of 32): the global-memory visits of mid-size grids use it (small grids fewer, grids of 2^12+ cells twice as many); the register-cached visits give each thread 1, 2 or 4 nodes of a colour so as to stay near it */
    int32_t tune_low_warps; /* launch shape: warps per CTA of the low-diagonal kernel (0: default; 1..16) */
    int32_t tune_low_items; /* launch shape: items one warp of that kernel runs in lockstep: 1, 2, 4 or 8 (0: default) */
    int32_t tune_low_cut;   /* schedule: the highest diagonal of each hierarchy run inside the low-diagonal kernel (0: default 4, lower when a long mu/nu program does not fit; 1..5); the visits above it are separate launches.  Launch shapes never change results; the cut changes only the rounding of the inner cycles */
    int32_t tune_visit_smem; /* schedule: KB of shared memory per CTA up to which a visit above the cut runs register-cached (u in shared memory; each thread keeps its nodes' coefficients and right-hand side in registers for the whole visit; grids of up to 2048 nodes per colour in the mixed path, 1024 in FP64) instead of in global memory (0: default 1; 1..227; 1 keeps every visit in global memory, the faster at 256 x 256).  Changes only the rounding of the cycles */
} msg_params;

/* ------------------------------------------------------------------------ */
/* (a1) xi: standard normals from Philox4x64-10 (Salmon et al., SC'11) and  */
/* Box-Muller.  Not in the paper (which samples by circulant embedding); the  */
/* KL sampler needs i.i.d. N(0,1) coefficients.                              */
/*                                                                          */
/* xi[i*M + m] for 0 <= i < S, 0 <= m < M is normal number m of global       */
/* sample s0 + i: block j = m/4 uses counter (j, s0+i, 0, 0), key (seed, 0); */
/* word w -> U = (w >> 11) 2^-53; (U0,U1) and (U2,U3) give                    */
/* sqrt(-2 ln(1-Ua)) * (cos, sin)(2 pi Ub).                                  */
/*   xi [device] double [S][M], written.  S >= 0, 1 <= M.                    */
int32_t msg_normals(uint64_t seed, uint64_t s0, int64_t S, int32_t M, double* xi, void* stream);

/* ------------------------------------------------------------------------ */
/* (a2) Truncated KL field Z = Phi diag(sqrt(lambda)) xi for S samples.     */
/* Phi [npts][M] and sqrt(lambda) [M] describe the field law on the field    */
/* grid of one shape (nodes of G^(P+1,Q+1), point index Fy*NFx + Fx).         */
/*                                                                          */
/* kl_prepare converts the FP64 basis once into the layout `mode` uses:      */
/*   Phi, sqrt_lambda [device] double, read.                                 */
/*   prepared [device] bytes >= kl_prepared_bytes(npts, M, mode), written;   */
/*            256-byte aligned for the tensor-core modes.                     */
/* sample_field contracts it with xi:                                       */
/*   xi [device] double [S][M], read.                                        */
/*   Z  [device] double [S][npts] (or float if z_fp32 != 0), written.         */
size_t kl_prepared_bytes(int64_t npts, int32_t M, int32_t mode);
int32_t kl_prepare(const double* Phi, const double* sqrt_lambda, int64_t npts, int32_t M, int32_t mode,
                   void* prepared, size_t prepared_bytes, void* stream);
int32_t sample_field(const void* prepared, int64_t npts, int32_t M, int32_t mode, const double* xi,
                     int64_t S, void* Z, int32_t z_fp32, void* stream);

/* ------------------------------------------------------------------------ */
/* Circulant-embedding sampler of the paper's own field law (Sec. 4,        */
/* numerical experiments): Matern covariance Eq. (1.2) with distance        */
/* r = ||T dx||, T = diag(1/sqrt(eta lambda), 1/sqrt(lambda)) R(theta)       */
/* (Sec. 1).  Each sample draws its anisotropic ratio eta and rotation      */
/* theta uniformly on the law's ranges (one Philox4x64-10 block, counter    */
/* (0, s, 1, 0), key (seed, 0): u = (w >> 11) 2^-53 of words 0 and 1), so   */
/* the eigenvalues of the embedding are recomputed for every sample:        */
/*   c      covariance on the periodic grid of L 2^(P+1) x L 2^(Q+1) points  */
/*          with the field's spacing, at signed periodic offsets (both signs */
/*          averaged at an offset of exactly half the period);               */
/*   Lambda = DFT2(c), FP64 (cuFFT D2Z);                                     */
/*   Z      = Re DFT2(sqrt(max(Lambda, 0) / M) (xi1 + i xi2)), forward       */
/*          transform, FP32 (cuFFT C2C), restricted to the field nodes;      */
/*          xi1, xi2 at embedding point k are normals 2k and 2k+1 of the     */
/*          sample's stream as msg_normals numbers them (the same 53-bit     */
/*          uniforms; log and sin/cos in single precision).                  */
/* Arguments:                                                               */
/*   Z         [device] double [S][(2^(P+1)+1)(2^(Q+1)+1)], written; the    */
/*             layout sample_field writes, ready for msg_solve_batch.        */
/*   eta_theta [device] double [S][2] (eta, theta in radians), written, or   */
/*             NULL.                                                         */
/*   status    [device] int32 [S], written (0 or MSG_CE_NEGATIVE_EIGENVALUE: */
/*             an eigenvalue below -1e-10 of the largest was set to zero,    */
/*             L too small for the law), or NULL.                            */
/*   workspace [device] >= ce_workspace_bytes(P, Q, law) bytes, 256-byte      */
/*             aligned.  1 <= P, Q <= 10, S >= 0, nu in {0.5, 1.5, 2.5},      */
/*             lambda > 0, 0 < eta_lo <= eta_hi, 2 <= L <= 64 (the periodic  */
/*             grid holds every field node), batch >= 1.                     */
/* Asynchronous on `stream`; the first call for a (P, Q, L, batch) on a      */
/* stream creates and caches that stream's cuFFT plans (which allocate their */
/* own work areas and block); plans are never shared between streams.        */
typedef struct {
    double nu;                 /* Matern smoothness: 0.5, 1.5 or 2.5 (closed forms of Eq. (1.2)) */
    double lambda;             /* length scale */
    double eta_lo, eta_hi;     /* anisotropic ratio range */
    double theta_lo, theta_hi; /* rotation range, degrees */
    int32_t L;                 /* periodic domain side in domain lengths (ce_padding: Sec. 4's choice) */
    int32_t batch;             /* samples per FFT batch: the workspace grows with it */
    int32_t scale;             /* 0: r = ||S R dx|| with S = diag(1/sqrt(eta lambda), 1/sqrt(lambda)) as
                                  Sec. 1 prints it; 1: lambda read as a length, S = diag(1/(eta lambda),
                                  1/lambda) (the reading under which standard coarsening fails as Sec. 2
                                  reports) */
} msg_ce_law;
#define MSG_CE_NEGATIVE_EIGENVALUE 1
/* L = 1 + 2 ceil(sqrt(nu) log2(max(2^p0, 2^q0))) (Sec. 4); 0 on bad input. */
int32_t ce_padding(double nu, int32_t p0, int32_t q0);
size_t ce_workspace_bytes(int32_t P, int32_t Q, const msg_ce_law* law);
int32_t ce_sample_field(int32_t P, int32_t Q, int64_t S, const msg_ce_law* law, uint64_t seed, uint64_t s0,
                        double* Z, double* eta_theta, int32_t* status, void* workspace, size_t ws_bytes,
                        void* stream);

/* ------------------------------------------------------------------------ */
/* (a3)-(a13) Batched FMSG solve.                                            */
/*                                                                          */
/* Sample i has finest grid (P_i, Q_i) = (PQ[2i], PQ[2i+1]), 1 <= P_i, Q_i    */
/* <= 12, and its field on the (2^(P_i+1)+1) x (2^(Q_i+1)+1) nodes of        */
/* G^(P_i+1,Q_i+1), x fastest; fields are packed back to back in sample      */
/* order.  The finest grid takes a = exp(Z) at its face midpoints (x-face    */
/* (i+1/2, j) at field node (2i+1, 2j), y-face (i, j+1/2) at (2i, 2j+1)); a  */
/* coarser face takes the series mean of the finest faces it covers along the */
/* flux direction (MSG_COEF_SERIES) or exp(Z) at its own midpoint            */
/* (MSG_COEF_INJECT).  The right-hand side is h = 1.                          */
/*                                                                          */
/* Every grid (p,q) of the sample is solved to ||1 - A u||/||1|| <= eps:      */
/* diagonals p+q are processed in increasing order (Algorithm 2); a grid     */
/* starts from the kappa-weighted cubic interpolation of its children's      */
/* solutions and is iterated by mu-cycles of Algorithm 1 over its own        */
/* hierarchy {(p',q'): p' <= p, q' <= q}.                                    */
/*                                                                          */
/*   PQ      [host]   int32 [S][2].                                          */
/*   Z       [device] double, sum_i (2^(P_i+1)+1)(2^(Q_i+1)+1) values, read. */
/*   Qout    [device] double, sum_i P_i Q_i values, written: QoI of grid      */
/*           (p,q) of sample i at offset_i + (p-1) Q_i + (q-1).              */
/*   status  [device] int32 [S], written (MSG_SAMPLE_* bits); may be NULL.    */
/*   cycles  [device] int32, packed like Qout: cycles used per grid; may be NULL. */
/*   relres  [device] double, packed like Qout: final ||r||/||b||; may be NULL. */
/*   workspace [device], ws_bytes >= msg_workspace_bytes(PQ, S, prm).       */
size_t msg_workspace_bytes(const int32_t* PQ, int64_t S, const msg_params* prm);
int32_t msg_solve_batch(const int32_t* PQ, int64_t S, const msg_params* prm, const double* Z, double* Qout,
                        int32_t* status, int32_t* cycles, double* relres, void* workspace, size_t ws_bytes,
                        void* stream);

/* Solutions on every grid (Algorithm 2 returns one per grid of the hierarchy). */
/* After msg_solve_batch has run on `workspace` (same PQ, S, prm; stream-      */
/* ordered after it), msg_solution copies the FP64 solution u of every grid of */
/* every sample into u_out: sample i's block of msg_solution_values(PQ+2i, 1)  */
/* values follows sample i-1's; inside it grid (p,q) starts at                 */
/* T(p-1) T(Q_i) + (2^p+1) T(q-1), T(n) = 2^(n+1) - 2 + n, and holds its       */
/* (2^p+1)(2^q+1) nodes row by row (x fastest), boundary zeros included.       */
/*   u_out [device] double [msg_solution_values(PQ, S)], written.              */
/* msg_solution_values returns the count (host only; -1 on a bad shape).       */
int64_t msg_solution_values(const int32_t* PQ, int64_t S);
int32_t msg_solution(const int32_t* PQ, int64_t S, const msg_params* prm, const void* workspace, size_t ws_bytes,
                     double* u_out, void* stream);

/* ------------------------------------------------------------------------ */
/* Convergence study (Sec. 2, numerical experiments): residual history of     */
/* plain cycles from u = 0 with b = 1 on the finest grid (P, Q) of S samples   */
/* of one shape, in FP64 (prm->precision is not used):                        */
/*   MSG_HIST_MSG       MSG mu-cycles (Algorithm 1 over the whole hierarchy);  */
/*   MSG_HIST_STANDARD  multigrid with standard coarsening on the grids        */
/*                      (P-k, Q-k) of the same hierarchy: full weighting,      */
/*                      bilinear interpolation, the same smoother, damping and */
/*                      coefficients, exact solve of the first grid with one   */
/*                      interior line.                                         */
/*   Z    [device] double [S][field_points(P, Q)], read.                      */
/*   hist [device] double [S][ncycles + 1], written: ||1 - A u_k||_h / ||1||_h */
/*        after k cycles (hist[s][0] = 1).                                     */
/*   workspace [device] >= msg_history_workspace_bytes(P, Q, S, prm, method), */
/*        256-byte aligned.  1 <= P, Q <= 10, 1 <= ncycles <= 1000.            */
/* msg_cycle_history returns once its work has finished.                      */
#define MSG_HIST_MSG 0
#define MSG_HIST_STANDARD 1
size_t msg_history_workspace_bytes(int32_t P, int32_t Q, int64_t S, const msg_params* prm, int32_t method);
int32_t msg_cycle_history(int32_t P, int32_t Q, int64_t S, const msg_params* prm, int32_t method, const double* Z,
                          int32_t ncycles, double* hist, void* workspace, size_t ws_bytes, void* stream);

/* ------------------------------------------------------------------------ */
/* (a14) Multi-index differences (Sec. 3, Eq. (3.2)) and Y (Eq. (3.6)).       */
/*                                                                          */
/* Sample i has multi-index L_i = (L[2i], L[2i+1]) >= 0 and grid QoIs packed  */
/* as msg_solve_batch writes them for finest grid (p0 + L_i1, q0 + L_i2), so */
/* Q_l = QoI of grid (p0 + l1, q0 + l2).  For 0 <= tau <= L_i:               */
/*   dQ_tau = D_2 D_1 Q_tau, D_j Q_l = Q_l - Q_{l-e_j} if l_j > 0 else Q_l,   */
/* packed per sample row-major [L_i1+1][L_i2+1], samples back to back.        */
/* If ptau != NULL (host, row-major [ld1][ld2], p_tau = P(L >= tau)), also    */
/* Y_i = sum_tau dQ_tau / p_tau.                                              */
/*   L [host] int32 [S][2]; Q [device] double, read; dQ [device] double,      */
/*   written; ptau [host] double or NULL; Y [device] double [S] or NULL.       */
int32_t mimc_differences(const int32_t* L, int64_t S, int32_t p0, int32_t q0, const double* Q,
                         const double* ptau, int32_t ld1, int32_t ld2, double* dQ, double* Y, void* stream);

/* Allocation-free variant of mimc_differences (no counterpart in the paper).  */
/* Same arguments, results and errors.  For callers that may not allocate     */
/* device memory once running (device memory fully reserved by their own     */
/* pool, or a loop that cannot pay for an allocator call): the per-sample     */
/* table and p_tau go to a fixed 16 MiB array in this library's own device    */
/* memory, held by every GPU that loads the library until the process exits.  */
/* A batch needing more (24 bytes per sample plus 8 ld1 ld2 bytes for p_tau,   */
/* so at most about 690 000 samples) is rejected with MSG_ERR_INVALID.  The    */
/* first call made with a device current looks up the array's address on that */
/* device; make that call before any stream capture.  All calls share the     */
/* array and return after their work has finished on `stream`; calls that     */
/* overlap on the GPU race.  The array holds no state a call needs: each call  */
/* writes the whole table it reads.  The cached address does not survive a    */
/* cudaDeviceReset of that device in the same process.                        */
int32_t mimc_differences_noalloc(const int32_t* L, int64_t S, int32_t p0, int32_t q0, const double* Q,
                                 const double* ptau, int32_t ld1, int32_t ld2, double* dQ, double* Y, void* stream);

/* ------------------------------------------------------------------------ */
/* Instrumentation (no counterpart in the paper).                           */
/*                                                                          */
/* msg_launch_count: number of CUDA kernels this library has launched in this */
/* process.  msg_profile_enable(n), n >= 1, clears the records, counts every  */
/* launch of each kernel class and times a random 1/n of the launches of the  */
/* cycle classes (PRE, POST, LOW, RESIDUAL, UPDATE) and every launch of the   */
/* others with CUDA events on their own streams (0 stops; n > 1 keeps the     */
/* event overhead off most launches).  msg_profile_read returns, for one kernel class, the       */
/* launches counted and the event-timed milliseconds, algorithmic bytes and   */
/* flops (the compulsory traffic/work per launch as defined in the design     */
/* notes) of the timed ones, scaled by launches / timed launches (exact for   */
/* n = 1).  Classes: 0 PRE, 1 POST, 2 LOW (cycle visits above / at-and-below  */
/* the cut), 3 RESIDUAL, 4 UPDATE, 5 INTERP, 6 QOI, 7 COEFFS, 8 NORMALS, 9 KL,*/
/* 10 MIMC.  msg_profile_read synchronises the recorded events.               */
int64_t msg_launch_count(void);
int32_t msg_profile_enable(int32_t on);
int32_t msg_profile_read(int32_t kernel_class, int64_t* launches, double* total_ms, double* bytes, double* flops);
/* msg_profile_read_level: the unscaled sums over the timed launches of one   */
/* class at one multigrid diagonal `level` (PRE/POST: the visited diagonal;  */
/* LOW: the diagonal the low program starts from); profile with n = 1 to     */
/* time every launch.                                                        */
int32_t msg_profile_read_level(int32_t kernel_class, int32_t level, int64_t* timed, double* total_ms, double* bytes);

/* Deferred kernel status (no counterpart in the paper).  Kernels with bounded */
/* pipeline waits (the tensor-core KL contraction) do not stop the stream to   */
/* report: a wait that runs out records it on the device and that kernel      */
/* leaves its output unwritten.  msg_device_status synchronises the current    */
/* device and returns MSG_ERR_TIMEOUT if any such wait ran out since the       */
/* previous call (the record is then cleared), else MSG_OK.                    */
int32_t msg_device_status(void);

/* Description of the last error on this thread ("" if none). */
const char* msg_last_error(void);

/* Library version string. */
const char* msg_version(void);

#ifdef __cplusplus
}
#endif
#endif /* MSG_MIMC_H */
