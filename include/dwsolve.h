/*
 * dwsolve.h -- C ABI of the GB300 library for the Wilson-Dirac system D x = b
 * solved by SAP-preconditioned flexible GMRES with deflated restarts.
 *
 * Operator (Sec. 2, Eq. "Dw" of Frommer, Nobile, Zingler, arXiv:1204.5463),
 * written with a bare mass m0:
 *     (D psi)_n = (4 + m0) psi_n
 *                 - 1/2 sum_{j=1..4} [ (1 + gamma_j) U_{n,j} psi_{n+j}
 *                                     + (1 - gamma_j) U^dagger_{n-j,j} psi_{n-j} ]
 * with periodic boundaries in all four directions. This is the paper's
 * D = 1 - kappa H_hop divided by 2 kappa, kappa = 1 / (2 (4 + m0)).
 * Gamma matrices: Hermitian chiral basis, gamma_k = [[0, -i sigma_k],
 * [i sigma_k, 0]] (k = 1..3), gamma_4 = [[0, 1], [1, 0]], so that
 * gamma_5 = gamma_1 gamma_2 gamma_3 gamma_4 = diag(1, 1, -1, -1).
 *
 * Canonical layouts at this boundary (FP64, complex numbers interleaved re,im):
 *   site index   n = n1 + d1*(n2 + d2*(n3 + d3*n4)),  V = d1 d2 d3 d4
 *   spinor field psi[rhs][site][spin 0..3][colour 0..2]  (24 doubles per site)
 *   gauge field  U[site][mu 0..3][row 0..2][col 0..2]    (72 doubles per site)
 * Buffers are owned by the caller; the library keeps its own converted copies
 * of the gauge field and its own Krylov workspace, owned by the context.
 *
 * Every call returns DW_OK (0) or a DW_E* code; dw_last_error() gives a
 * message for the calling thread. No C++ exception crosses this boundary.
 * All device work of a context is issued on the CUDA stream given to
 * dw_create; calls return after that work has completed unless stated.
 */
#ifndef DWSOLVE_H
#define DWSOLVE_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define DW_OK 0
#define DW_EINVAL 1       /* invalid argument (sizes, layout, parameters)       */
#define DW_ECUDA 2        /* CUDA runtime error                                 */
#define DW_ENOMEM 3       /* device allocation or HBM budget exhausted          */
#define DW_ENOTCONV 4     /* solver stopped at max_cycles / max_iterations      */
#define DW_EBREAKDOWN 5   /* unrecoverable breakdown of the Krylov process      */
#define DW_ENONFINITE 6   /* NaN or Inf met in the residual or the Hessenberg   */
#define DW_ETIMEOUT 7     /* a bounded device wait or a request deadline expired */
#define DW_ECANCELLED 8   /* request cancelled                                   */

#define DW_MAX_RHS 16

/* Storage / arithmetic precision of a field or a kernel:
 *   DW_F64  FP64 storage, FP64 arithmetic
 *   DW_F32  FP32 storage, FP32 arithmetic
 *   DW_F16  FP16 storage with one FP32 scale per site, FP32 arithmetic
 *   DW_BF16 BF16 storage with one FP32 scale per site, FP32 arithmetic
 *   DW_DF64 double-float: every real is an unevaluated sum hi + lo of two FP32
 *           numbers (48-bit significand, FP64 footprint); arithmetic on the FP32
 *           pipes with error-free transformations. Only for the outer Krylov
 *           vectors of fgmresdr_solve (outer_prec). */
typedef enum { DW_F64 = 0, DW_F32 = 1, DW_F16 = 2, DW_BF16 = 3, DW_DF64 = 4 } dw_prec;

/* Lattice L = {0 <= n <= d-1} (Sec. 2) and its decomposition into domains
 * L^l of block[] sites each. Requirements: dims[j] >= 2; block[j] >= 1;
 * dims[j] % block[j] == 0 and dims[j] / block[j] even (red-black colouring
 * without same-colour coupling, Sec. 2 / Fig. 1); block volume <= 1024. */
typedef struct {
    int dims[4];
    int block[4];
    double m0;
} dw_lattice;

typedef struct dw_ctx dw_ctx;

/* Create a context on the current CUDA device. cuda_stream is a cudaStream_t
 * (NULL = legacy default stream) on which every launch of the context goes.
 * Errors: DW_EINVAL for an invalid lattice, DW_ECUDA. */
int dw_create(const dw_lattice* L, void* cuda_stream, dw_ctx** out);

/* Release all device memory of the context. NULL is accepted. */
void dw_destroy(dw_ctx* ctx);

/* Change the bare mass m0 (keeps the gauge field). */
int dw_set_mass(dw_ctx* ctx, double m0);

/* Load the gauge field U (canonical FP64 layout, V*72 doubles). on_device
 * selects a device (1) or host (0) pointer. The library converts it to its
 * internal storage precisions on first use; the caller's buffer is not kept. */
int dw_set_gauge(dw_ctx* ctx, const double* U, int on_device);

/* Add the clover term of the improved operators of Sec. 6 (the paper cites
 * the Sheikholeslami-Wohlert term without a formula; this is the standard
 * site-diagonal form):
 *   D_sw = D + A,  A_n = c_sw (i/2) sum_{mu<nu} sigma_{mu nu} F_{mu nu}(n),
 *   sigma_{mu nu} = (i/2)[gamma_mu, gamma_nu], F_{mu nu}(n) = (Q - Q^dagger)/8
 *   made traceless, Q the sum of the four plaquettes in the (mu, nu) plane
 *   that start and end at n, all in the same sense.
 * The term is computed once on the device from the current gauge field (and
 * again after every dw_set_gauge) and then enters dw_apply, sap_precondition
 * (A is site-diagonal, so it is part of every local operator D^l) and
 * fgmresdr_solve. csw = 0 restores the plain Wilson operator.
 * Errors: DW_EINVAL (no gauge field yet, non-finite csw), DW_ENOMEM, DW_ECUDA;
 * with the clover term, SAP domains are limited to 256 sites. */
int dw_set_clover(dw_ctx* ctx, double csw);

/* out = D in for nrhs spinor fields (Sec. 2, Eq. "Dw"), all in one launch
 * (the CTAs of one block of sites for the different fields run side by side,
 * so most re-reads of the links hit L2).
 * in, out: device pointers, canonical FP64 layout, nrhs*V*24 doubles each,
 * non-overlapping. prec selects the storage and arithmetic of the stencil:
 * the input is rounded to prec, D is applied in prec, and the result (in
 * prec storage) is widened back to FP64. 1 <= nrhs <= DW_MAX_RHS. */
int dw_apply(dw_ctx* ctx, const double* in, double* out, dw_prec prec, int nrhs);

/* z = M v with M the SAP preconditioner (Sec. 4): ncycles iterations of
 * Algorithm 2 started from x = 0, each a sweep over the domains of colour 0
 * (block coordinates summing to an even number; contains site 0) followed by
 * colour 1. Each domain solve computes r = (v - D x)^l with the full
 * operator, runs nmr minimal-residual steps on D^l y = r from y = 0 (Sec. 4)
 * and adds x^l += y^l. storage selects the precision of v, x and the links
 * (arithmetic FP32 for DW_F32/F16/BF16, FP64 for DW_F64).
 * v, z: device pointers, canonical FP64 layout, nrhs fields each.
 * Requires ncycles >= 1, nmr >= 1. Each domain's CTA waits (at most about a
 * second) for the bulk copy of its links; if a wait gives up the call, and a
 * solve whose preconditioner it was, returns DW_ETIMEOUT.
 * Errors: DW_EINVAL, DW_ENOMEM, DW_ECUDA, DW_ETIMEOUT. */
int sap_precondition(dw_ctx* ctx, const double* v, double* z, int ncycles, int nmr, dw_prec storage, int nrhs);

typedef struct {
    int m;                  /* basis dimension per cycle (Algorithm 4's m); 1 <= m <= 63   */
    int k;                  /* deflation dimension (harmonic Ritz vectors); 0 <= k < m;
                               k = 0 gives restarted FGMRES(m)                             */
    double tol;             /* stop when ||b - D x||_2 / ||b||_2 <= tol (explicit, FP64)   */
    int max_cycles;         /* limit on restart cycles                                     */
    int max_iterations;     /* limit on Arnoldi steps (0 = none)                           */
    int sap_cycles;         /* SAP iterations per preconditioner application               */
    int mr_steps;           /* MR steps per domain solve                                   */
    dw_prec sap_prec;       /* storage precision of SAP fields and of the Z basis          */
    dw_prec matvec_prec;    /* precision of the Arnoldi product w = D z (DW_F64 or DW_F32) */
    double clean_restart_t; /* clean restart when ||r_explicit|| / ||r_implicit|| > t (Sec. 5.7) */
    int nrhs;               /* right-hand sides solved together, 1..DW_MAX_RHS             */
    int host_buffers;       /* 1: b and x are host pointers (copies inside the call)       */
    int use_x0;             /* 1: x holds the initial guess; 0: x0 = 0                     */
    dw_prec outer_prec;     /* outer vectors and their Gram-Schmidt / update arithmetic:
                               DW_F64 (V, x, b, r in FP64), DW_DF64 (default: double-float),
                               or DW_F32: the single-precision Arnoldi process of Sec. 5.7
                               (V and all basis arithmetic in FP32, x, b, r and the
                               explicit residual double-float; needs sap_prec F32/F16/BF16
                               and matvec_prec DW_F32)                                      */
} dw_solver_params;

typedef struct {
    int iterations;                  /* Arnoldi steps (= preconditioned matvecs), max over rhs */
    int cycles;                      /* restart cycles, max over rhs                          */
    int clean_restarts;              /* summed over rhs                                       */
    int converged;                   /* number of rhs that met tol                            */
    int explicit_residuals;          /* FP64 residual evaluations                             */
    int iterations_rhs[DW_MAX_RHS];
    double true_rel_res[DW_MAX_RHS]; /* final ||b - D x|| / ||b|| per rhs (FP64)             */
    double time_s;                   /* wall time of the call                                 */
} dw_stats;

/* Defaults: m = 30, k = 10, tol = 1e-10, max_cycles = 500, max_iterations = 0,
 * sap_cycles = 5, mr_steps = 4, sap_prec = DW_F32, matvec_prec = DW_F32,
 * clean_restart_t = 4, nrhs = 1, host_buffers = 0, use_x0 = 0, outer_prec = DW_DF64. */
void dw_default_params(dw_solver_params* P);

/* Solve D x = b for nrhs right-hand sides with FGMRES-DR (Algorithm 4):
 * flexible Arnoldi (Algorithm 3) with classical Gram-Schmidt and selective
 * reorthogonalisation in the basis precision (outer_prec), Givens-updated
 * implicit residual (Sec. 5.2, 5.6),
 * harmonic Ritz deflation (Lemma 1a, Eqs. "G_kplus1", "hatHk"), and the
 * refinement scheme of Sec. 5.7 (Algorithm 5): every cycle recomputes r = b - D x in FP64 and
 * injects it into the least-squares right-hand side, the last column of
 * G_{k+1} and v_{k+1}; a clean restart follows when
 * ||r_explicit|| / ||r_implicit|| > clean_restart_t.
 * b, x: canonical FP64 layout, nrhs fields, device pointers unless
 * P->host_buffers. Each rhs is solved for b scaled by the power of two
 * nearest 1/||b|| (exact; x is scaled back), so the FP32-range double-float
 * and FP32 vectors hold any b whose norm is finite in FP64 and whose
 * entries, relative to ||b||, stay within FP32's range.
 * Returns DW_OK when every rhs met tol, DW_ENOTCONV when a
 * limit stopped the solve (x then holds the last iterate), or an error code
 * (DW_EINVAL, DW_ENOMEM, DW_ECUDA, DW_EBREAKDOWN, DW_ENONFINITE, and
 * DW_ETIMEOUT when a SAP sweep's bounded wait for its links gave up, and
 * DW_ECANCELLED after dw_cancel).
 * S may be NULL. */
int fgmresdr_solve(dw_ctx* ctx, const double* b, double* x, const dw_solver_params* P, dw_stats* S);

/* Asks the solve running on ctx (in another thread) to stop: fgmresdr_solve
 * checks the request before every Arnoldi step and then returns DW_ECANCELLED,
 * with x holding the iterate of the last completed cycle and S filled as for
 * DW_ENOTCONV. A solve clears the request when it starts, so a cancel issued
 * while no solve runs has no effect. Safe to call from any thread. */
int dw_cancel(dw_ctx* ctx);

/* Residual history of the last fgmresdr_solve on ctx for right-hand side rhs,
 * the quantities the paper plots (Sec. 6: residual against the number of
 * matrix-vector products): for each cycle end i, out[3i] = Arnoldi steps so
 * far, out[3i+1] = the implicit (least-squares) relative residual of the
 * cycle, out[3i+2] = the explicit ||b - D x|| / ||b|| computed after it
 * (Sec. 5.7). *n = the number of cycle ends; at most max are written (out may
 * be NULL to query *n). */
int dw_residual_history(dw_ctx* ctx, int rhs, double* out, int max, int* n);

/* Test and diagnosis hook (not part of the paper's method): copies the bases
 * of the last cycle of the last fgmresdr_solve on ctx for right-hand side rhs,
 * so that the flexible Arnoldi relation A Z_m = V_{m+1} Hhat_m (Eq.
 * "arnoldilike"; after a deflated restart its leading k columns are the
 * rotated ones of Eq. "hatHk") and the orthonormality of V can be checked.
 * *ncols = m', the columns of that cycle (0 if the solve stopped inside a
 * cycle or converged before its first step). V_out: device, (m'+1) canonical
 * FP64 fields; Z_out: device, m' fields; H_out: host, (m'+1) x m' complex,
 * row-major, interleaved re,im, in the scaling of the solve (b scaled by the
 * power of two nearest 1/||b||). Each output may be NULL; max_cols bounds m'
 * (DW_EINVAL if smaller). The bases are the library's internal copies
 * widened to FP64 (basis format outer_prec, Z in its storage format). */
int dw_debug_basis(dw_ctx* ctx, int rhs, double* V_out, double* Z_out, double* H_out, int max_cols, int* ncols);

/* Message describing the last error on the calling thread ("" if none). */
const char* dw_last_error(void);

/* ---- measurement hooks ----------------------------------------------------
 * While profiling is on, the context brackets its kernel launches with CUDA
 * events on its stream and accumulates, per kernel class, the number of
 * launches, the summed device time and the summed algorithmic bytes. */
typedef struct {
    char name[32];
    long long launches;
    double total_ms;
    double bytes;
} dw_kernel_stat;

int dw_profile(dw_ctx* ctx, int enable);

/* Number of CUDA kernels this library has launched in the process so far
 * (all contexts, all threads). */
long long dw_kernel_launches(void);
/* Copies up to max entries into out, sets *n; reset != 0 clears the totals. */
int dw_profile_read(dw_ctx* ctx, dw_kernel_stat* out, int max, int* n, int reset);

/* ---- domain-tile autotuner ------------------------------------------------
 * Chooses the SAP domain block for a lattice by the time to solution of a
 * calibration solve per candidate (the block changes the preconditioner, so
 * iteration counts change with it). Candidates: block[j] divides dims[j] with
 * dims[j] / block[j] even (red-black colouring, Sec. 2), 32..1024 sites per
 * domain, aspect ratio <= 2, SAP shared memory within one CTA; the twelve
 * closest to 256 sites per domain (most isotropic first) are timed.
 * L: dims and m0 (block ignored); U: device canonical FP64 gauge field;
 * b: device canonical right-hand sides (P->nrhs fields); P: the calibration
 * solve (a looser tol keeps it short; host_buffers and use_x0 are ignored).
 * Writes the fastest converged block to best_block; when results is non-NULL
 * also up to max_results timed candidates and their count to *n_results.
 * The choice is cached per (dims, nrhs, precisions, m, k, SAP cycles, MR
 * steps): a later call without results returns the cached block at once.
 * Allocates one output field on the stream; DW_ENOTCONV if no candidate
 * converged. */
typedef struct {
    int block[4];
    double seconds;  /* wall time of the calibration solve (1e300 if it failed) */
    int iterations;
    int status;
} dw_tune_entry;

int dw_autotune_block(const dw_lattice* L, const double* U, const double* b, const dw_solver_params* P,
                      void* cuda_stream, int* best_block, dw_tune_entry* results, int max_results, int* n_results);

/* SAP work per preconditioner application, tuned on a fixed block: the pairs
 * (sap_cycles, mr_steps) in {2, 3, 4, 5, 6, 8} x {3, 4, 5, 6, 8, 10} are ranked by the
 * wall time of a calibration solve P on L's block (more SAP work per step buys
 * fewer Arnoldi steps and Gram-Schmidt passes, so the best pair depends on
 * the relative cost of a sweep, e.g. on the storage precision and the number
 * of right-hand sides). The paper fixes these (Sec. 6: 5 MR steps; 8 to 24
 * SAP cycles); this searches them. Writes the fastest converged pair; with
 * results, up to max_results timed pairs and their count. Cached per (dims,
 * block, nrhs, precisions, m, k). Errors as dw_autotune_block. */
typedef struct {
    int sap_cycles, mr_steps;
    double seconds;  /* wall time of the calibration solve (1e300 if it failed) */
    int iterations;
    int status;
} dw_tune_sap_entry;

int dw_autotune_sap(const dw_lattice* L, const double* U, const double* b, const dw_solver_params* P,
                    void* cuda_stream, int* best_cycles, int* best_mr, dw_tune_sap_entry* results, int max_results,
                    int* n_results);

/* ---- allocation-free operator ----------------------------------------------
 * The paper has no counterpart of this entry point; it serves callers that
 * cannot call cudaMalloc (code inside a pre-reserved memory pool, allocators
 * that forbid device allocation, processes with a fixed memory budget).
 *
 * out = D in with FP32 storage and arithmetic, exactly as dw_apply(..., DW_F32,
 * 1) computes it for the plain Wilson operator (there is no context, so no
 * clover term), but without allocating anything: the
 * FP32 copies of the links and of the fields live in one file-scope device
 * array of 2 MiB (480 bytes per site), so the lattice may have at most 4096
 * sites (larger lattices return DW_EINVAL). dims: the four extents (no domain
 * decomposition is needed); U: device pointer, canonical FP64 gauge field
 * (V*72 doubles); in, out: device pointers, one canonical FP64 spinor field
 * each (V*24 doubles); cuda_stream: cudaStream_t or NULL. Returns after the
 * work on the stream has completed.
 * Set-up: the first call on each device is the set-up step. Under CUDA's
 * default lazy module loading that call is what loads the library's device
 * code on the device and so places the 2 MiB array there (the driver does this,
 * not the library), and it looks up the array's device address with
 * cudaGetSymbolAddress, once per device, with that device current. Make the
 * first call outside stream capture and before entering any region in which
 * the process must not allocate (or set CUDA_MODULE_LOADING=EAGER so the
 * array is placed when the context is created). From then on the device holds
 * the 2 MiB until the process exits, and calls allocate nothing. The cached
 * address belongs to the device's current primary context: do not use this
 * entry point after cudaDeviceReset on that device.
 * Every call overwrites the whole part of the array it reads, so nothing needs
 * clearing, but all calls share the array: calls that overlap on the GPU
 * (other threads or streams) race and must be serialised by the caller. */
int dw_apply_f32_noalloc(const int* dims, double m0, const double* U, const double* in, double* out,
                         void* cuda_stream);

/* ---- serving ----------------------------------------------------------------
 * A solve server admits requests of any lattice, mass, gauge field and
 * right-hand-side count while their estimated device memory
 * (dw_request_bytes) fits the budget and one of max_slots slots is free;
 * queued requests are taken first-in first-out, and a later request that fits
 * may start while an earlier one waits for memory. Each admitted request runs
 * fgmresdr_solve on its own CUDA stream and context, so concurrent requests
 * overlap on the device. A finished request's context (converted gauge field,
 * Krylov workspace) stays on the device, counted in the budget, and is taken
 * over by a later request that passes the same host gauge pointer and lattice
 * (so that buffer must not change while the server lives); idle contexts are
 * freed least recently used first when admission needs the memory.
 * Not part of the paper: this is the request loop the solver is deployed
 * behind. */
typedef struct {
    dw_lattice lattice;      /* dims, domain block, m0                                     */
    const double* U;         /* host, canonical gauge field; valid until the request is done */
    const double* b;         /* host, params.nrhs canonical spinor fields                   */
    double* x;               /* host, params.nrhs canonical spinor fields (output)          */
    dw_solver_params params; /* host_buffers is forced to 1, use_x0 applies to x           */
} dw_request;

typedef struct {
    size_t budget_bytes, in_use_bytes, peak_bytes;
    int running, queued;
    long long completed;
    long long reused; /* requests that took over a cached context */
    int peak_running;  /* most requests that were solving at the same time */
} dw_server_status;

typedef struct dw_server dw_server;

/* Estimated device bytes of a request: gauge copies (FP64 + FP32 [+ 16-bit
 * SAP storage] [+ double-float for the residual stencil] + the SAP links
 * packed per domain) + upload staging +
 * per rhs ((m+1) Arnoldi vectors in the basis format + m Z vectors (FP32 when
 * a 16-bit SAP is deflated, with the SAP output buffer) + x, b, r + SAP input
 * [+ FP32 residual copy for an FP32 basis] + host staging) + k rotation
 * scratch. Requests solve the plain Wilson operator. */
size_t dw_request_bytes(const dw_request* r);

/* Creates the server on the current device with max_slots worker threads. */
int dw_server_create(size_t hbm_budget_bytes, int max_slots, dw_server** out);
/* Queues a request (returns at once). DW_ENOMEM if it exceeds the whole budget. */
int dw_server_submit(dw_server* s, const dw_request* r, uint64_t* id);
/* *done = 1 once finished; then *status (DW_OK, DW_ENOTCONV, DW_ECANCELLED,
 * ...), *S and the submit-to-done latency are filled (each may be NULL). */
int dw_server_poll(dw_server* s, uint64_t id, int* done, int* status, dw_stats* S, double* latency_s);
/* Blocks until the request is done or timeout_s passed (DW_ETIMEOUT). */
int dw_server_wait(dw_server* s, uint64_t id, double timeout_s, int* status, dw_stats* S, double* latency_s);
/* Cancels a request: a queued one is dropped at once; a running one stops
 * before its next Arnoldi step (its status becomes DW_ECANCELLED, its x holds
 * the iterate of its last completed cycle). DW_EINVAL if finished or unknown. */
int dw_server_cancel(dw_server* s, uint64_t id);
int dw_server_info(dw_server* s, dw_server_status* out);
/* in_use_bytes includes idle cached contexts.
 * dw_server_destroy cancels queued requests, waits for running ones, frees everything. */
void dw_server_destroy(dw_server* s);

#ifdef __cplusplus
}
#endif

#endif /* DWSOLVE_H */
