/*
 * helm.h - C ABI of the GB300 block Jacobi sweeping preconditioner library
 *
 * Method: R. Dai, "A Block Jacobi Sweeping Preconditioner for the Helmholtz
 * Equation" (arXiv 2209.10886).  The library discretises
 *
 *     -Delta u - kappa(x)^2 u = f   on the grid's rectangle,  kappa = omega sqrt(m2),
 *     d_n u - i kappa u = 0          on the outer boundary (first-order absorbing,
 *                                    the paper's Eq. origPbm with T = i kappa,
 *                                    time dependence e^{-i omega t}, Section 3)
 *
 * with the five-point stencil on n_x x n_y interior nodes x_{a,b} = (a h, b h),
 * a = 1..n_x, b = 1..n_y.  Every row is multiplied by h^2, so the linear
 * system is  A u = h^2 f  with the complex symmetric matrix
 *
 *     (A u)_p = (4 - kappa_p^2 h^2 - sum_{outer ghost sides} c_p) u_p - sum_{grid nbrs q} u_q,
 *     c_p = (1 + beta_p)/(1 - beta_p),  beta_p = i kappa_p h / 2.
 *
 * The domain is split into an N1 x N2 checkerboard of subdomains (Section 2)
 * coupled by Robin transmission conditions (Eq. subPbm).  The preconditioner
 * (Sections 3-5) solves all local problems of one stage of the sweep schedule
 * in one batched launch, exchanges the interface traces through the
 * transmission operator, and is applied inside FP64 flexible GMRES
 * (Section 6: GMRES to a relative residual of 1e-6).
 *
 * Conventions for every entry point
 * * Arrays: complex values are helm_c128 (layout-compatible with
 *   torch.complex128 / C99 double complex).  A field is n_x*n_y values,
 *   row-major with the y index slowest: p = (b-1)*n_x + (a-1).  Several
 *   right-hand sides are stored back to back: RHS k starts at ptr + k*n_x*n_y.
 * * Pointers marked "device" must be CUDA device (or managed) memory of the
 *   current device; "host" pointers are ordinary host memory.
 * * Ownership: the caller owns every array it passes and keeps it alive until
 *   the call's work on `stream` has completed.  The handle owns the factors,
 *   interface buffers and Krylov workspace and frees them in helm_destroy.
 * * Execution: calls are ordered on the given stream and return without
 *   synchronising, except where stated (gmres_solve and misfit_grad read
 *   convergence data back and synchronise the stream).
 * * Errors: no C++ exception crosses the ABI.  A non-zero helm_status is
 *   returned and helm_last_error() describes it.  HELM_ERR_ARG for invalid
 *   arguments, HELM_ERR_STATE for calls in the wrong order, HELM_ERR_OOM when
 *   a device allocation fails, HELM_ERR_CUDA for any other CUDA error,
 *   HELM_ERR_TIMEOUT when a bounded device-side wait gave up (the work of that
 *   call is incomplete; call precond_factor again before reusing the handle).
 * * Threads: a handle must not be used from two host threads at once.
 */
#ifndef HELM_H
#define HELM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct { double re, im; } helm_c128;

typedef enum {
    HELM_OK = 0,
    HELM_ERR_ARG = 1,
    HELM_ERR_CUDA = 2,
    HELM_ERR_OOM = 3,
    HELM_ERR_STATE = 4,
    HELM_ERR_NO_CONVERGENCE = 5,
    HELM_ERR_TIMEOUT = 6,
    HELM_ERR_UNSUPPORTED = 7
} helm_status;

/* Precision of the subdomain factors and of the preconditioner arithmetic.
 * HELM_PREC_C128: complex128 factors and solves (the all-FP64 form).
 * HELM_PREC_C64:  complex64 factors and solves, FP32 accumulation; the
 *                 interface data and local solves are complex64, the input
 *                 residual is scaled by its 2-norm before rounding. */
typedef enum {
    HELM_PREC_C128 = 0,
    HELM_PREC_C64 = 1
} helm_prec;

/* Sweep schedule of the interface preconditioner.
 * HELM_SCHED_BSP: block Jacobi sweeping (Section 5): forward bands of N1+1
 *                 diagonals from the bottom-left corner, backward bands from
 *                 the top-right corner, all bands concurrently; 2 N1 sweep
 *                 steps (plus one residual stage) per application.
 * HELM_SCHED_SP:  symmetric Gauss-Seidel sweeping (Section 4,
 *                 Eq. sgs_preconditioner_forward_backward): 2 (N1+N2-2) steps.
 * HELM_SCHED_BSP_NONOVERLAP: block Jacobi sweeping with bands of N1 diagonals that
 *                 share none (the paper's band bounds read as half-open);
 *                 2 (N1 - 1) sweep steps; for comparison with HELM_SCHED_BSP */
typedef enum { HELM_SCHED_BSP = 0, HELM_SCHED_SP = 1, HELM_SCHED_BSP_NONOVERLAP = 2, HELM_NSCHED = 3 } helm_sched;

/* Robin parameter T_e of the interface condition (d_n - T_e) u = g.
 * HELM_TC_OPTIMIZED: T_e = (i - 1) s sqrt(kappa_e pi / (2 h)) with s = tc_scale,
 *                    an optimized zeroth-order complex Robin parameter.
 * HELM_TC_IMPEDANCE: T_e = i kappa_e, the basic impedance operator the paper
 *                    uses for its algebra (Section 3).
 * HELM_TC_HABC:      the Pade-type high-order absorbing condition of the paper's
 *                    experiments (Sections 3 and 6: N_pade auxiliary fields and
 *                    rotation phi, 8 and pi/3 there): on each interface side the
 *                    dense operator T = i diag(k) e^{i phi/2} R_N(W) that
 *                    helm_habc_side_operator returns (Neumann ends, no corner
 *                    treatment), in place of the scalar T_e.  The library factors
 *                    the local problems with the optimized Robin parameter (tc_scale)
 *                    and folds the HABC side blocks in through the interface boundary
 *                    points (needs boundary_operators = 1 and at most 1024 interface
 *                    boundary points per subdomain); every sweep stage stays one GEMV
 *                    (or GEMM) per subdomain.
 * kappa_e = omega sqrt((m2_p + m2_q)/2) on the edge between nodes p and q.
 * The converged solution does not depend on T_e; the iteration count does. */
typedef enum { HELM_TC_OPTIMIZED = 0, HELM_TC_IMPEDANCE = 1, HELM_TC_HABC = 2 } helm_transmission;

typedef struct {
    int transmission;   /* helm_transmission; default HELM_TC_OPTIMIZED */
    double tc_scale;    /* s of HELM_TC_OPTIMIZED; default 1.0 */
    int boundary_operators;  /* 1 (default): precond_factor also builds, per subdomain, the
                                interface-boundary block K of the local inverse, and the
                                zero-source stages of the sweeps (all sweep steps and the
                                block Jacobi residual) apply it as one GEMV per subdomain;
                                0: those stages run full block-tridiagonal solves instead
                                (the same operator; no K memory, no K construction time,
                                which grows like (boundary points) x (subdomain solve)) */
    int tensor_cores;   /* with complex64 factors (HELM_PREC_C64) and subdomains at most 256
                           nodes wide, block solves over 16 or more right-hand sides at once
                           (the construction of K, batched sources) run on the tensor cores
                           with FP32 accumulation, from a second copy of the factors in the
                           tensor cores' operand layout:
                           1 (default): every operand split into two TF32 numbers (hi + lo,
                              three MMAs per product), FP32-level accuracy; the copy takes
                              twice the bytes of the factors
                           2: TF32 operands alone (rounded to nearest; unit roundoff 2^-11),
                              one MMA per product; the copy takes the bytes of the factors
                           0: FP32 arithmetic on the CUDA cores, no second copy */
    int tc_min_rhs;     /* stages with at least this many right-hand sides use the tensor
                           cores (when tensor_cores != 0); default 16, minimum 1.  Below
                           16 the MMA columns are padded (N = 32 per 16 RHS) */
    int autotune;       /* 1 (default): the first preconditioner application with a given
                           RHS count times candidate launch shapes on the caller's stream
                           and keeps the fastest for this problem: for 2 or more RHS, the
                           interface-stage kernel's (RHS per block 2/4/8/16, K rows staged
                           in shared memory or not; the tensor-core form among them where
                           tensor_cores allows it) on the all-subdomain stage S; for any
                           RHS count, the full-stage kernels' (CTAs per subdomain, factor
                           chunk per ring slot; RHS per CTA of the tensor-core form) on
                           the liftings;
                           0: fixed rules (see helm_iface_shape, helm_stage_shape) */
    int tc_iface_min_ctas;  /* an interface stage runs in the tensor-core form (when that
                           form is chosen) only if it makes at least this many CTAs (of
                           128 output rows x 16 or 32 RHS); smaller stages take the
                           CUDA-core shape.  -1 (default): two per SM */
    size_t device_budget;  /* 0 (default): no limit.  Otherwise the most device memory, in
                           bytes, that the handle's large arrays may take: precond_factor
                           returns HELM_ERR_OOM (allocating nothing) when the factors, their
                           tensor-core copy and the boundary operators would exceed it, and
                           gmres_solve plans its right-hand-side chunks within what the
                           factors leave of it (HELM_ERR_OOM when not even one right-hand
                           side's Krylov workspace fits).  Tables of a few KB per subdomain
                           and the preconditioner's interface buffers are not counted */
    int n_pade;         /* HELM_TC_HABC: auxiliary fields of the Pade approximation (>= 0);
                           default 8 */
    double pade_phi;    /* HELM_TC_HABC: branch-cut rotation phi (radians); default pi/3 */
    int tc_factor;      /* 1 (default): with complex64 factors, tensor_cores != 0 and subdomains
                           at most 128 nodes wide, precond_factor runs each inversion
                           X_r = T_r^{-1} as a blocked Gauss-Jordan elimination (panels of 16
                           columns, partial pivoting) whose rank-16 trailing updates are
                           3xTF32 tensor-core GEMMs; 0: the CUDA-core elimination */
    int sym_k;          /* 1 (default): with complex64 factors, boundary_operators = 1, the
                           optimized or impedance transmission and at most 1024 interface
                           boundary points per subdomain, precond_factor also stores the
                           symmetric part (K + K^T)/2 of each K (K = P^T A_loc^{-1} P is
                           complex symmetric, A_loc being so; the two differ by rounding) as
                           its upper-triangle 32 x 32 tiles, half the bytes of K, and the
                           interface stages of one right-hand side that apply every
                           subdomain's whole K (the block Jacobi residual, the interface
                           operator S) stream them instead.  0: every interface stage
                           applies the full K */
} helm_setup_opts;

typedef struct {
    int restart;        /* FGMRES restart length m (>= 1); default 50 */
    int maxit;          /* maximum Arnoldi steps per RHS over all cycles */
    double tol;         /* stop when ||h^2 f - A u|| <= tol ||h^2 f|| (true residual) */
    int x0_given;       /* 1: u holds the initial guess; 0: start from u = 0 */
    int sched;          /* helm_sched used by the preconditioner */
    int use_graph;      /* 1: every preconditioner application is replayed from a CUDA graph
                           captured on first use for its (schedule, nrhs, input, output)
                           (one graph per Arnoldi slot; dropped when the factors or the
                           workspace change); ignored while helm_profile is on */
    double* hist;       /* optional host buffer of maxit*nrhs doubles: the Arnoldi
                           residual estimate of RHS k after step j at hist[k*maxit+j] */
    int ortho;          /* Arnoldi orthogonalisation, all FP64: HELM_ORTHO_MGS (default;
                           used when n_x*n_y fits the persistent kernel, else CGS2),
                           HELM_ORTHO_CGS2 or HELM_ORTHO_CGS2_SPLIT; the interface
                           iterations use CGS2 (CGS2_SPLIT when that is chosen) */
    int inner_maxit;    /* 0 (default): each preconditioner application runs the sweep
                           once (g = sweep(b) on the interface).  > 0: the interface
                           problem (I - S) g = b of the paper (Sections 3-5) is solved by
                           FP64 FGMRES preconditioned by the sweep, at most inner_maxit
                           steps per application, inner_restart per cycle, stopping at
                           ||b - (I - S) g|| <= inner_tol ||b|| (classical Gram-Schmidt
                           on the ntrace-long vectors, a second pass only when the first
                           removed more than 90 % of ||w||^2; their precision as
                           inner_fp64 says); the outer FGMRES stays FP64 on the volume
                           system */
    int inner_restart;  /* default 100 */
    double inner_tol;   /* default 1e-4 */
    int persistent;     /* 0 (default): the interface stages of every sweep are separate
                           launches (graph-replayed inside the interface iterations, each
                           starting its prologue while the previous stage runs);
                           1: all of them in one cooperative launch with a grid barrier
                           between stages (measured slower on GB300);
                           2: all of them in one cooperative launch without barriers:
                           each work item (stage, subdomain, row block) waits only for the
                           earlier items that produce or read the trace slots it touches
                           (counters in device memory, bounded waits).  1 and 2 need the
                           boundary operators */
    double* inner_hist; /* optional host buffer of inner_maxit*nrhs doubles: the residual
                           estimates ||b - (I - S) g_j|| / ||b|| of the interface iteration
                           in the first preconditioner application of this call, RHS k
                           after step j at inner_hist[k*inner_maxit+j] (that application
                           runs the host-driven loop) */
    int inner_fp64;     /* interface iterations (inner_maxit > 0) with complex64 factors:
                           0 (default) keeps the interface Krylov vectors in complex64
                           (FP32 vector arithmetic; reductions, Gram-Schmidt coefficients
                           and the least-squares problem stay FP64), which suits an
                           inner_tol well above the FP32 roundoff; 1 keeps them FP64.
                           With complex128 factors they are always FP64 */
    long long wait_cycles; /* 0 (default): the grid barriers of the Gram-Schmidt kernels (the
                           volume and interface Arnoldi steps) give up after ~2e9 SM clock
                           cycles (~1 s).  > 0: after this many cycles instead; a barrier that
                           gives up makes the call return HELM_ERR_TIMEOUT (a diagnostic
                           knob for bounding a solve's stalls, and for exercising the
                           timeout path: with a few cycles every barrier gives up) */
} helm_opts;

/* Orthogonalisation of the Arnoldi vectors.
 * HELM_ORTHO_MGS:  modified Gram-Schmidt in one persistent kernel per step
 *                  (8 FP64 FMA per element per basis vector).
 * HELM_ORTHO_CGS2: classical Gram-Schmidt, a second pass when the first
 *                  removed more than half of the squared norm (16 FMA per
 *                  element; more than 90 % in the interface iteration).
 *                  When a slice of the vector per SM fits in shared memory
 *                  (up to ~6000 values per SM), the passes, the norm and the
 *                  Givens update run as one cooperative launch per step.
 * HELM_ORTHO_CGS2_SPLIT: the same arithmetic as separate reduction kernels
 *                  (about 15 launches per step). */
enum { HELM_ORTHO_MGS = 0, HELM_ORTHO_CGS2 = 1, HELM_ORTHO_CGS2_SPLIT = 2 };

typedef struct {
    int iters;          /* Arnoldi steps taken */
    double relres;      /* final true relative residual ||h^2 f - A u|| / ||h^2 f|| */
} helm_info;

typedef struct helm_problem helm_problem;

/* Fill *o with the defaults listed above. */
void helm_default_opts(helm_opts* o);
void helm_default_setup_opts(helm_setup_opts* o);

/* Partition the grid and build the coefficient tables (paper Sections 2-3).
 * n_x, n_y   interior nodes per direction (>= 1); h grid step (> 0);
 * omega      angular frequency (> 0);
 * m2         device, n_x*n_y squared slowness values (> 0), copied;
 * N1, N2     subdomain columns and rows (1 <= N1 <= n_x, 1 <= N2 <= n_y);
 * xcuts      host, N1+1 increasing node offsets from 0 to n_x (column i1 owns
 *            x-nodes xcuts[i1-1] .. xcuts[i1]-1, 0-based), or NULL for the
 *            most even split (larger pieces first); ycuts likewise;
 * opts       host, or NULL for defaults;
 * out        host; receives the new handle (NULL on failure).
 * Synchronises the device once (coefficient upload). */
helm_status helm_setup(int n_x, int n_y, double h, double omega, const double* m2,
                       int N1, int N2, const int* xcuts, const int* ycuts,
                       const helm_setup_opts* opts, helm_problem** out);

/* Factor every subdomain matrix (paper Eq. subPbm; the paper uses a sparse
 * direct solver, Section 6) as a block tridiagonal LU over its grid rows:
 * T_1 = D_1, X_r = T_r^{-1}, T_{r+1} = D_{r+1} - X_r, storing all X_r.
 * Replaces factors of another precision.  Synchronises `stream` (it reads the
 * pivot checks back and reports a zero pivot as HELM_ERR_ARG). */
helm_status precond_factor(helm_problem* p, helm_prec prec, void* stream);

/* z = M^{-1} r for nrhs right-hand sides (device r and z, nrhs*n_x*n_y each,
 * may not overlap).  M^{-1} approximates A^{-1}: liftings of r on every
 * subdomain (Eq. subPbmLifting) give the interface right-hand side b, the
 * sweep `sched` approximates (I - S)^{-1} b (Eq. abstractSys), and local
 * solves with source r and the resulting incoming data give z.
 * HELM_ERR_STATE before precond_factor.  Stream-ordered. */
helm_status precond_apply(helm_problem* p, int sched, const helm_c128* r, helm_c128* z,
                          int nrhs, void* stream);

/* Size of the fixed scratch array used by precond_apply_noalloc (32 MiB). */
#define HELM_NOALLOC_SCRATCH_BYTES (32 << 20)

/* precond_apply without any memory allocation.  The paper has no counterpart:
 * this is a service for callers that must not allocate device memory during
 * the solve phase, e.g. code running under a memory budget fixed up front, or
 * inside a framework whose caching allocator owns every device allocation and
 * forbids others.  precond_apply allocates its workspace on first use (and
 * again when nrhs grows); this variant instead takes its scratch (three
 * interface buffers, the solve workspace, norms) from one static array of
 * HELM_NOALLOC_SCRATCH_BYTES in device memory that belongs to the library
 * image: every GPU that loads the library holds it until the process exits.
 * Result: z = M^{-1} r as precond_apply computes it, by the same kernels in the
 * same order.  This call never runs the autotuner: its interface stages take the
 * launch shape an earlier precond_apply or gmres_solve tuned for this nrhs on p,
 * else the fixed rules (see helm_iface_shape), so the two can differ by the
 * rounding of differently ordered sums (not bit for bit).
 * Arguments as for precond_apply; p must be factored (HELM_ERR_STATE if not).
 * Sizes: returns HELM_ERR_ARG, with a message naming the bytes needed, when the
 * scratch exceeds HELM_NOALLOC_SCRATCH_BYTES; nothing is launched then.  The
 * scratch is 3*ntrace*nrhs*e + N*nrhs*e bytes (e = 8 for HELM_PREC_C64, 16 for
 * C128; 4*ntrace*nrhs*e with the HABC transmission, which keeps the liftings'
 * boundary values) plus 8*nrhs*(3 + 1216) bytes of norms and partial sums, each part
 * rounded up to 256 bytes; with HELM_PREC_C64, tensor_cores on and nrhs >=
 * tc_min_rhs (the tensor-core stages) add 2*etot*nrhs*8 + N*nrhs*8 bytes, etot
 * = 2 * sum over the subdomains of (mx + my).
 * Calls no cudaMalloc, cudaFree or other allocating routine.  The first call
 * on a device looks up the array's device address with that device current;
 * make that first call before any stream capture.  Every call on a device
 * shares the one array and it keeps the last call's contents (no part of it
 * needs to start at zero: every value is written before it is read); calls
 * whose work overlaps on the GPU (other streams, other host threads) race on
 * it and must be serialised by the caller.  Stream-ordered. */
helm_status precond_apply_noalloc(helm_problem* p, int sched, const helm_c128* r, helm_c128* z,
                                  int nrhs, void* stream);

/* Au = A u for nrhs fields (device u, Au; the h^2-scaled operator above).
 * Stream-ordered. */
helm_status helm_matvec(helm_problem* p, const helm_c128* u, helm_c128* Au, int nrhs, void* stream);

/* Solve A u = h^2 f for nrhs sources by right-preconditioned flexible GMRES
 * in FP64 (the paper's outer Krylov solver, Section 6; residual, Gram-Schmidt,
 * Hessenberg least squares and update in FP64; the preconditioner, precond_apply's
 * M^{-1} or with opts->inner_maxit > 0 the interface FGMRES of Sections 3-5, in
 * the factor precision).  f, u device; opts host
 * (NULL: defaults); info host array of nrhs entries (or NULL).
 * Returns HELM_ERR_NO_CONVERGENCE (u holds the last iterate, info filled)
 * when some RHS did not reach tol within maxit.  Synchronises `stream`. */
helm_status gmres_solve(helm_problem* p, const helm_c128* f, helm_c128* u, int nrhs,
                        const helm_opts* opts, helm_info* info, void* stream);

/* Misfit J = 1/2 sum_s ||P u_s - d_s||^2 over nsrc sources and its gradient
 * with respect to m2 by the adjoint-state method:
 *   A u_s = h^2 f_s,   A conj(lambda_s) = conj(P^T (P u_s - d_s))  (A complex symmetric),
 *   grad_p = - sum_s Re(conj(lambda_{s,p}) dA_pp/dm2_p u_{s,p}).
 * The adjoint solves reuse the factors and preconditioner.
 * f device nsrc*N; rec_idx device nrec flat node indices; d device nsrc*nrec
 * (RHS-major); misfit host scalar; grad_m2 device N doubles (overwritten);
 * u_out device nsrc*N or NULL.  Needs precond_factor first.  Synchronises. */
helm_status misfit_grad(helm_problem* p, const helm_c128* f, int nsrc, const int* rec_idx, int nrec,
                        const helm_c128* d, const helm_opts* opts, double* misfit, double* grad_m2,
                        helm_c128* u_out, void* stream);

/* Release the handle and everything it owns (NULL is allowed). */
helm_status helm_destroy(helm_problem* p);

/* Message describing the last non-OK status returned on this host thread. */
const char* helm_last_error(void);

/* Host-only query of the sweep schedule (no GPU needed): the number of
 * sequential sweep steps per application (Section 4: 2(N1+N2-2) for SP;
 * Section 5: 2 x the longest band, i.e. 2 N1 with two or more bands, for BSP)
 * and the number of batched stage launches (steps plus the lifting and
 * reconstruction stages, plus the residual stage of BSP).  steps/stages host. */
helm_status helm_schedule_info(int N1, int N2, int sched, int* steps, int* stages);

/* Host only (no GPU): the Pade-type high-order transmission operator of one interface
 * side (Sections 3 and 6: HABC transmission with n_pade auxiliary fields and rotation
 * phi; the paper's runs use 8 and pi/3), as the dense L x L matrix
 *   T = i diag(k) e^{i phi/2} R_N(W),  W = (I + diag(1/k^2) Lap) e^{-i phi} - I,
 *   R_N(W) = I + sum_{l=1..N} a_l (I + b_l W)^{-1} W,
 *   a_l = 2/M sin^2(l pi/M), b_l = cos^2(l pi/M), M = 2N + 1,
 * the rotated-branch Pade approximation of i k sqrt(1 + Lap/k^2), where Lap is the
 * 3-point second difference of spacing h along the side with Neumann ends.
 * kappa: host, L wavenumbers (> 0) of the side's points; T: host, L*L values,
 * row-major (T[r*L + c]), written by the call.  n_pade = 0 and phi = 0 give
 * i diag(kappa), the impedance condition.  HELM_ERR_ARG for NULL pointers, L < 1,
 * h <= 0, n_pade < 0, a non-positive kappa or a singular factor. */
helm_status helm_habc_side_operator(const double* kappa, int L, double h, int n_pade, double phi, helm_c128* T);

/* 1 when the last precond_factor of p ran its eliminations' trailing updates on the
 * tensor cores (helm_setup_opts.tc_factor), else 0 (also for NULL or unfactored p). */
int helm_factor_on_tensor_cores(const helm_problem* p);

/* 1 when the interface stages that apply all of K (block Jacobi residual, interface
 * operator S) in preconditioner applications with nrhs right-hand sides read the packed
 * symmetric boundary operators of the last precond_factor (helm_setup_opts.sym_k),
 * else 0 (also for NULL or unfactored p). */
int helm_iface_symmetric(const helm_problem* p, int nrhs);

/* Bounds-checking build (the library compiled with -DHELM_CHECK_BOUNDS; the normal
 * build returns 0 from both calls and touches nothing).  In that build the kernels
 * check their global accesses (every bulk copy and the computed loads and stores of the
 * stage, interface, Krylov and HABC kernels) against the live device ranges: the
 * library's allocations and the caller's buffers of the current call.  A failed check
 * skips the access and is counted.
 * helm_check_bounds_report: the failed checks since the last reset summed over the
 * kernels' translation units (*violations), and the first one found (address, bytes,
 * source line, source file name into unit[unit_len]); reset != 0 clears the counts.
 * Host pointers, any may be NULL.  Returns 1 (checking build), 0 (normal build) or -1
 * (CUDA error).  Synchronises the device.
 * helm_check_bounds_selftest: runs the check, without any access, on a 256-byte
 * allocation: results[0] = the whole allocation passes, results[1] = the byte past
 * its end passes, results[2] = a 2-byte range straddling its end passes (expected
 * 1, 0, 0; the two failures are counted).  results: host, 3 ints.  Returns 1, 0 or
 * -1 as above. */
int helm_check_bounds_report(long long* violations, unsigned long long* first_addr, long long* first_bytes,
                             int* first_line, char* unit, int unit_len, int reset);
int helm_check_bounds_selftest(int* results);

/* Problem sizes of a handle: N = n_x*n_y unknowns, number of subdomains,
 * 2 N_e interface unknowns (trace points), bytes of the current factors. */
helm_status helm_problem_info(const helm_problem* p, long long* n_unknowns, int* n_subdomains,
                              long long* n_trace, long long* factor_bytes);

/* Kernel classes of the library's own launches, for helm_profile_read. */
typedef enum {
    HELM_K_STAGE = 0,      /* fused block-tridiagonal subdomain solve + transmission */
    HELM_K_MATVEC = 1,     /* five-point operator (matvec and true residual) */
    HELM_K_ORTHO = 2,      /* Gram-Schmidt dot products and updates, solution update */
    HELM_K_OTHER = 3,      /* norms, reductions, Hessenberg, scaling, adjoint */
    HELM_K_TRACE = 4       /* interface stages: boundary-operator GEMV + transmission */
} helm_kernel_class;

typedef struct {
    long long launches;    /* launches recorded since profiling was enabled */
    double ms;             /* summed device time between CUDA events recorded on the
                              launch stream immediately before and after each launch */
    double flops;          /* algorithmic real floating-point operations of those launches
                              (a complex multiply-add counts 8) */
    double bytes;          /* algorithmic bytes those launches must move (HBM reads +
                              writes of the data they touch, counted once) */
} helm_kstat;

/* Launch shape of the interface stages for nrhs right-hand sides on p.  CUDA-core form:
 * RHS per block (*nr), K rows staged in shared memory when they fit (*staged), target
 * CTAs per SM (*waves).  *tensor = 3 or 1 when the stages large enough to put two CTAs
 * on every SM run as tensor-core MMAs (3xTF32 or TF32 operands; complex64 factors with
 * tensor_cores on and nrhs >= tc_min_rhs) with *tensor_rhs = 16 or 32 RHS per CTA, the
 * smaller stages in the CUDA-core form; 0 and 0 when every stage runs on the CUDA cores.
 * *tuned = 1 when the autotuner chose it, 0 for the fixed rules (4, 2 or 1 RHS per block,
 * staged, 3; the tensor cores where allowed, 32 RHS per CTA from 32 RHS, else 16).  Any
 * output pointer may be NULL. */
helm_status helm_iface_shape(const helm_problem* p, int nrhs, int* nr, int* staged, int* waves, int* tensor,
                             int* tensor_rhs, int* tuned);

/* Launch shape of the full-stage kernels (the liftings and reconstructions, which stream
 * the factors) for nrhs right-hand sides on p, as the autotuner chose it (setup option
 * autotune; *tuned = 1) or 0 for each field when the kernels' rules apply (*tuned = 0):
 * *csize CTAs per subdomain on the CUDA cores (1, or 2 = one per column half of the
 * factors), *chunk_kb KB of factors per ring slot of the bulk-copy stream (64, 48, 32),
 * *tensor_rhs RHS per CTA of the tensor-core form (16, 32, 64).  Any output may be NULL. */
helm_status helm_stage_shape(const helm_problem* p, int nrhs, int* csize, int* chunk_kb, int* tensor_rhs, int* tuned);

/* Number of CUDA kernel launches issued by the library in this process. */
long long helm_launch_count(void);

/* Interface Krylov steps taken inside the preconditioner applications of p
 * (gmres_solve with inner_maxit > 0), summed over all calls; per application
 * the largest count over its right-hand sides.  0 for a NULL handle. */
long long helm_inner_steps(const helm_problem* p);

/* Enable (on != 0) or disable per-launch event timing on handle p; enabling
 * (or disabling) resets the statistics.  Timing adds two event records per
 * launch; a stage sequence replayed from a CUDA graph (the sweeps and S inside
 * the interface Krylov iterations) is bracketed as a whole and its time,
 * launches, bytes and flops are attributed to its kernel class. */
helm_status helm_profile(helm_problem* p, int on);

/* Statistics of one kernel class (synchronises the device to read the events). */
helm_status helm_profile_read(helm_problem* p, int kernel_class, helm_kstat* out);

#ifdef __cplusplus
}
#endif

#endif /* HELM_H */
