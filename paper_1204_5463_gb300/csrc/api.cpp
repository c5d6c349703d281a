// C ABI of the library (include/dwsolve.h): contexts, the operator, the
// preconditioner, the solver entry point, error reporting and profiling.
#include <atomic>
#include <cmath>
#include <cstring>
#include <new>
#include <string>

#include "dense.h"
#include "internal.h"

namespace dwk {

static thread_local std::string g_err;
static std::atomic<long long> g_launches{0};

void count_launch() { g_launches.fetch_add(1, std::memory_order_relaxed); }

void set_error(const std::string& msg) { g_err = msg; }
int fail(int code, const std::string& msg) {
    g_err = msg;
    return code;
}

int DevBuf::ensure(size_t n) {
    if (n <= bytes && p) return DW_OK;
    release();
    if (n == 0) return DW_OK;
    cudaError_t e = cudaMallocAsync(&p, n, st);
    if (e != cudaSuccess) {
        p = nullptr;
        bytes = 0;
        cudaGetLastError();
        return fail(DW_ENOMEM, std::string("cudaMalloc of ") + std::to_string(n) + " bytes failed: " +
                                   cudaGetErrorString(e));
    }
    bytes = n;
    return DW_OK;
}

void DevBuf::release() {
    if (p) cudaFreeAsync(p, st);
    p = nullptr;
    bytes = 0;
}

// ---------------------------------------------------------------------------
cudaEvent_t Profiler::take() {
    if (!pool.empty()) {
        cudaEvent_t e = pool.back();
        pool.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
    return e;
}

int Profiler::begin(const char* name, double bytes, cudaEvent_t* start_out, int* idx) {
    int i = 0;
    for (; i < (int)k.size(); ++i)
        if (k[i].name == name) break;
    if (i == (int)k.size()) {
        k.emplace_back();
        k.back().name = name;
    }
    cudaEvent_t a = take();
    if (!a) return -1;
    cudaEventRecord(a, stream);
    *start_out = a;
    *idx = i;
    k[i].pending_bytes.push_back(bytes);
    return 0;
}

void Profiler::end(int idx, cudaEvent_t start) {
    cudaEvent_t b = take();
    if (!b) {
        pool.push_back(start);
        return;
    }
    cudaEventRecord(b, stream);
    k[idx].pending.push_back({start, b});
}

void Profiler::drain() {
    for (auto& e : k) {
        for (size_t i = 0; i < e.pending.size(); ++i) {
            cudaEventSynchronize(e.pending[i].second);
            float ms = 0.f;
            cudaEventElapsedTime(&ms, e.pending[i].first, e.pending[i].second);
            e.total_ms += ms;
            e.launches += 1;
            e.bytes += (i < e.pending_bytes.size()) ? e.pending_bytes[i] : 0.0;
            pool.push_back(e.pending[i].first);
            pool.push_back(e.pending[i].second);
        }
        e.pending.clear();
        e.pending_bytes.clear();
    }
}

void Profiler::reset() {
    drain();
    k.clear();
}

Profiler::~Profiler() {
    for (auto& e : k)
        for (auto& p : e.pending) {
            cudaEventDestroy(p.first);
            cudaEventDestroy(p.second);
        }
    for (auto ev : pool) cudaEventDestroy(ev);
}

// ---------------------------------------------------------------------------
int gauge_for(dw_ctx* ctx, int prec, const char** out) {
    if (!ctx->have_gauge) return fail(DW_EINVAL, "gauge field not set");
    if (prec < 0 || prec > 4) return fail(DW_EINVAL, "bad precision");
    if (!ctx->U_ready[prec]) {
        int rc = ctx->U[prec].ensure((size_t)link_bytes(prec, ctx->g.V));
        if (rc) return rc;
        rc = launch_link_convert(prec, ctx->U[P64].as<char>(), ctx->U[prec].as<char>(), ctx->g.V, ctx->stream);
        if (rc) return rc;
        ctx->U_ready[prec] = true;
    }
    *out = ctx->U[prec].as<char>();
    return DW_OK;
}

int HostFlag::ensure() {
    if (h) return DW_OK;
    int* p = nullptr;
    DW_CUDA_TRY(cudaHostAlloc(reinterpret_cast<void**>(&p), sizeof(int), cudaHostAllocMapped));
    *p = 0;
    h = p;
    DW_CUDA_TRY(cudaHostGetDevicePointer(reinterpret_cast<void**>(&d), p, 0));
    return DW_OK;
}

HostFlag::~HostFlag() {
    if (h) cudaFreeHost(h);
}

int sap_links_for(dw_ctx* ctx, int prec, int threads, const char** U, const char** img) {
    int rc;
    if ((rc = gauge_for(ctx, prec, U))) return rc;
    if ((rc = ctx->sap_err.ensure())) return rc;
    threads = sap_threads(ctx->g, threads);
    if (ctx->Uimg_threads[prec] != threads) {
        if ((rc = ctx->Uimg[prec].ensure(sap_link_image_bytes(prec, ctx->g, threads)))) return rc;
        if ((rc = launch_sap_link_image(prec, ctx->g, *U, ctx->Uimg[prec].as<char>(), threads, ctx->stream)))
            return rc;
        ctx->Uimg_threads[prec] = threads;
    }
    *img = ctx->Uimg[prec].as<char>();
    return DW_OK;
}

int sap_check(dw_ctx* ctx) {
    if (!ctx->sap_err.h || *reinterpret_cast<volatile int*>(ctx->sap_err.h) == 0) return DW_OK;
    *reinterpret_cast<volatile int*>(ctx->sap_err.h) = 0;
    return fail(DW_ETIMEOUT, "a SAP domain's bulk copy of its links did not complete");
}

static int check_prec(int p) { return (p >= 0 && p <= 3) ? DW_OK : fail(DW_EINVAL, "bad precision"); }

}  // namespace dwk

using namespace dwk;

extern "C" {

const char* dw_last_error(void) { return g_err.c_str(); }

long long dw_kernel_launches(void) { return g_launches.load(std::memory_order_relaxed); }

int dw_create(const dw_lattice* L, void* cuda_stream, dw_ctx** out) {
    if (!L || !out) return fail(DW_EINVAL, "null argument");
    *out = nullptr;
    Geom g;
    g.V = 1;
    g.B = 1;
    g.ndom = 1;
    long long V = 0;
    if (!lattice_volume(L->dims, kMaxSites, &V))
        return fail(DW_EINVAL, "lattice extents must be >= 2 with at most 2^31/24 sites in all");
    for (int j = 0; j < 4; ++j) {
        const int d = L->dims[j], b = L->block[j];
        if (b < 1 || d % b != 0) return fail(DW_EINVAL, "block must divide the lattice extent");
        if ((d / b) % 2 != 0) return fail(DW_EINVAL, "domain count per direction must be even (red-black)");
        g.d[j] = d;
        g.b[j] = b;
        g.nb[j] = d / b;
        g.B *= b;
        g.ndom *= d / b;
    }
    g.V = V;
    if (g.B > 1024) return fail(DW_EINVAL, "domain volume must be <= 1024 sites");
    dw_ctx* c = new (std::nothrow) dw_ctx();
    if (!c) return fail(DW_ENOMEM, "host allocation failed");
    c->g = g;
    c->m0 = L->m0;
    c->stream = reinterpret_cast<cudaStream_t>(cuda_stream);
    c->prof.stream = c->stream;
    cudaError_t e = cudaGetDevice(&c->device);
    if (e != cudaSuccess) {
        delete c;
        cudaGetLastError();
        return fail(DW_ECUDA, std::string("no CUDA device: ") + cudaGetErrorString(e));
    }
    c->sap_threads.assign(4, 0);
    for (auto* b : {&c->U[0], &c->U[1], &c->U[2], &c->U[3], &c->U[4], &c->work_in, &c->work_out, &c->work_aux,
                   &c->Uimg[0], &c->Uimg[1], &c->Uimg[2], &c->Uimg[3]})
        b->st = c->stream;
    *out = c;
    return DW_OK;
}

void dw_destroy(dw_ctx* ctx) {
    if (!ctx) return;
    cudaStreamSynchronize(ctx->stream);
    release_workspace(ctx->ws);
    cudaStream_t st = ctx->stream;
    delete ctx;
    cudaStreamSynchronize(st);  // the stream-ordered frees have completed
}

int dw_set_mass(dw_ctx* ctx, double m0) {
    if (!ctx) return fail(DW_EINVAL, "null context");
    ctx->m0 = m0;
    return DW_OK;
}

int dw_set_gauge(dw_ctx* ctx, const double* U, int on_device) {
    if (!ctx || !U) return fail(DW_EINVAL, "null argument");
    const size_t bytes = (size_t)ctx->g.V * 72 * sizeof(double);
    int rc = ctx->U[P64].ensure((size_t)link_bytes(P64, ctx->g.V));
    if (rc) return rc;
    const double* src = U;
    if (!on_device) {
        if ((rc = ctx->work_aux.ensure(bytes))) return rc;
        DW_CUDA_TRY(cudaMemcpyAsync(ctx->work_aux.p, U, bytes, cudaMemcpyHostToDevice, ctx->stream));
        src = ctx->work_aux.as<double>();
    }
    if ((rc = launch_gauge_convert(P64, src, ctx->U[P64].as<char>(), ctx->g.V, ctx->stream))) return rc;
    for (int p = 0; p < 5; ++p) ctx->U_ready[p] = false;
    for (int p = 0; p < 4; ++p) ctx->Uimg_threads[p] = 0;
    ctx->U_ready[P64] = true;
    ctx->have_gauge = true;
    if (ctx->csw != 0.0 && (rc = dw_set_clover(ctx, ctx->csw))) return rc;  // the clover term follows the links
    DW_CUDA_TRY(cudaStreamSynchronize(ctx->stream));
    return DW_OK;
}

int dw_set_clover(dw_ctx* ctx, double csw) {
    if (!ctx) return fail(DW_EINVAL, "null context");
    if (!std::isfinite(csw)) return fail(DW_EINVAL, "c_sw must be finite");
    if (csw == 0.0) {
        ctx->csw = 0.0;
        return DW_OK;
    }
    if (!ctx->have_gauge) return fail(DW_EINVAL, "set the gauge field before the clover term");
    const long long V = ctx->g.V;
    int rc;
    if ((rc = ctx->clov64.ensure((size_t)V * 72 * sizeof(double)))) return rc;
    if ((rc = ctx->clov32.ensure((size_t)V * 72 * sizeof(float)))) return rc;
    if ((rc = launch_clover_compute(ctx->g, ctx->U[P64].as<char>(), csw, ctx->clov64.as<double>(),
                                    ctx->clov32.as<float4>(), ctx->stream)))
        return rc;
    DW_CUDA_TRY(cudaStreamSynchronize(ctx->stream));
    ctx->clov.a64 = ctx->clov64.as<char>();
    ctx->clov.a32 = ctx->clov32.as<char>();
    ctx->csw = csw;
    return DW_OK;
}

int dw_apply(dw_ctx* ctx, const double* in, double* out, dw_prec prec, int nrhs) {
    if (!ctx || !in || !out) return fail(DW_EINVAL, "null argument");
    if (check_prec(prec)) return DW_EINVAL;
    if (nrhs < 1 || nrhs > DW_MAX_RHS) return fail(DW_EINVAL, "nrhs out of range");
    const long long V = ctx->g.V;
    const long long fb = spinor_bytes(prec, V);
    int rc;
    const char* U;
    if ((rc = gauge_for(ctx, prec, &U))) return rc;
    if ((rc = ctx->work_in.ensure((size_t)nrhs * fb))) return rc;
    if ((rc = ctx->work_out.ensure((size_t)nrhs * fb))) return rc;
    if ((rc = launch_to_internal(prec, in, ctx->work_in.as<char>(), V, nrhs, ctx->stream))) return rc;
    {
        // algorithmic bytes: every field once, the links once for all
        // right-hand sides of the launch (its CTAs for one block of sites and
        // the different rhs run next to each other, so L2 serves the re-reads)
        const double link_reads = 1.0;
        ProfScope ps(&ctx->prof, prec == DW_F64 ? "dw_f64" : prec == DW_F32 ? "dw_f32" : "dw_f16",
                     (double)nrhs * 2.0 * fb + link_reads * link_bytes(prec, V));
        FieldRef fi{ctx->work_in.as<char>(), fb, 0, 0}, fo{ctx->work_out.as<char>(), fb, 0, 0};
        if ((rc = launch_dw(prec, prec, prec, ctx->g, ctx->m0, fi, fo, U, nullptr, nrhs, nullptr, ctx->stream,
                            ctx->clover())))
            return rc;
    }
    if ((rc = launch_from_internal(prec, ctx->work_out.as<char>(), out, V, nrhs, ctx->stream))) return rc;
    DW_CUDA_TRY(cudaStreamSynchronize(ctx->stream));
    return DW_OK;
}

int sap_precondition(dw_ctx* ctx, const double* v, double* z, int ncycles, int nmr, dw_prec storage, int nrhs) {
    if (!ctx || !v || !z) return fail(DW_EINVAL, "null argument");
    if (check_prec(storage)) return DW_EINVAL;
    if (nrhs < 1 || nrhs > DW_MAX_RHS) return fail(DW_EINVAL, "nrhs out of range");
    if (ncycles < 1 || nmr < 1) return fail(DW_EINVAL, "ncycles and nmr must be >= 1");
    const long long V = ctx->g.V;
    const long long fb = spinor_bytes(storage, V);
    int rc;
    const char *U, *Uimg;
    if ((rc = sap_links_for(ctx, storage, ctx->sap_threads[storage], &U, &Uimg))) return rc;
    if ((rc = ctx->work_in.ensure((size_t)nrhs * fb))) return rc;
    if ((rc = ctx->work_out.ensure((size_t)nrhs * fb))) return rc;
    if ((rc = launch_to_internal(storage, v, ctx->work_in.as<char>(), V, nrhs, ctx->stream))) return rc;
    FieldRef fv{ctx->work_in.as<char>(), fb, 0, 0}, fx{ctx->work_out.as<char>(), fb, 0, 0};
    for (int cyc = 0; cyc < ncycles; ++cyc)
        for (int colour = 0; colour < 2; ++colour) {
            const int mode = (cyc > 0) ? 2 : (colour == 0 ? 0 : 1);
            ProfScope ps(&ctx->prof, "sap_sweep",
                         (double)nrhs * 0.5 * (2.0 * fb + (mode == 2 ? fb : 0) + link_bytes(storage, V)));
            if ((rc = launch_sap_sweep(storage, storage, ctx->g, ctx->m0, fv, fx, Uimg, nullptr, nrhs, colour, nmr,
                                       mode, ctx->sap_threads[storage], ctx->stream, ctx->clover(), ctx->sap_err.d)))
                return rc;
        }
    if ((rc = launch_from_internal(storage, ctx->work_out.as<char>(), z, V, nrhs, ctx->stream))) return rc;
    DW_CUDA_TRY(cudaStreamSynchronize(ctx->stream));
    return sap_check(ctx);
}

void dw_default_params(dw_solver_params* P) {
    if (!P) return;
    std::memset(P, 0, sizeof(*P));
    P->m = 30;
    P->k = 10;
    P->tol = 1e-10;
    P->max_cycles = 500;
    P->max_iterations = 0;
    P->sap_cycles = 5;
    P->mr_steps = 4;
    P->sap_prec = DW_F32;
    P->matvec_prec = DW_F32;
    P->clean_restart_t = 4.0;
    P->nrhs = 1;
    P->host_buffers = 0;
    P->use_x0 = 0;
    P->outer_prec = DW_DF64;
}

int fgmresdr_solve(dw_ctx* ctx, const double* b, double* x, const dw_solver_params* P, dw_stats* S) {
    if (!ctx) return fail(DW_EINVAL, "null argument");
    ctx->cancel.store(0);  // a cancel issued before this solve started does not apply to it
    return solve_checked(ctx, b, x, P, S, &ctx->cancel);
}

int dw_cancel(dw_ctx* ctx) {
    if (!ctx) return fail(DW_EINVAL, "null context");
    ctx->cancel.store(1);
    return DW_OK;
}

int dw_residual_history(dw_ctx* ctx, int rhs, double* out, int max, int* n) {
    if (!ctx || !n || max < 0) return fail(DW_EINVAL, "bad argument");
    return residual_history(ctx, rhs, out, max, n);
}

int dw_debug_basis(dw_ctx* ctx, int rhs, double* V_out, double* Z_out, double* H_out, int max_cols, int* ncols) {
    if (!ctx || !ncols) return fail(DW_EINVAL, "null argument");
    return debug_basis(ctx, rhs, V_out, Z_out, H_out, max_cols, ncols);
}

}  // extern "C"

namespace dwk {

int solve_checked(dw_ctx* ctx, const double* b, double* x, const dw_solver_params* P, dw_stats* S,
                  const std::atomic<int>* cancel) {
    if (!ctx || !b || !x || !P) return fail(DW_EINVAL, "null argument");
    if (P->m < 1 || P->m > 63) return fail(DW_EINVAL, "m must be in 1..63");
    if (P->k < 0 || P->k >= P->m || P->k > 16) return fail(DW_EINVAL, "k must satisfy 0 <= k < m and k <= 16");
    if (!(P->tol > 0.0)) return fail(DW_EINVAL, "tol must be positive");
    if (P->max_cycles < 1) return fail(DW_EINVAL, "max_cycles must be >= 1");
    if (P->sap_cycles < 1 || P->mr_steps < 1) return fail(DW_EINVAL, "sap_cycles and mr_steps must be >= 1");
    if (check_prec(P->sap_prec)) return DW_EINVAL;
    if (P->matvec_prec != DW_F64 && P->matvec_prec != DW_F32)
        return fail(DW_EINVAL, "matvec_prec must be DW_F64 or DW_F32");
    if (P->nrhs < 1 || P->nrhs > DW_MAX_RHS) return fail(DW_EINVAL, "nrhs out of range");
    if (P->outer_prec != DW_F64 && P->outer_prec != DW_DF64 && P->outer_prec != DW_F32)
        return fail(DW_EINVAL, "outer_prec must be DW_F64, DW_DF64 or DW_F32");
    if (P->outer_prec == DW_F32 && (P->sap_prec == DW_F64 || P->matvec_prec != DW_F32))
        return fail(DW_EINVAL, "an FP32 Arnoldi basis needs a 32- or 16-bit SAP and an FP32 matvec");
    if (!(P->clean_restart_t > 1.0)) return fail(DW_EINVAL, "clean_restart_t must be > 1");
    return solve(ctx, b, x, P, S, cancel);
}

}  // namespace dwk

extern "C" {

int dw_profile(dw_ctx* ctx, int enable) {
    if (!ctx) return fail(DW_EINVAL, "null context");
    ctx->prof.on = enable != 0;
    return DW_OK;
}

int dw_profile_read(dw_ctx* ctx, dw_kernel_stat* out, int max, int* n, int reset) {
    if (!ctx || !n) return fail(DW_EINVAL, "null argument");
    ctx->prof.drain();
    int cnt = 0;
    for (auto& e : ctx->prof.k) {
        if (out && cnt < max) {
            std::memset(&out[cnt], 0, sizeof(dw_kernel_stat));
            std::strncpy(out[cnt].name, e.name.c_str(), sizeof(out[cnt].name) - 1);
            out[cnt].launches = e.launches;
            out[cnt].total_ms = e.total_ms;
            out[cnt].bytes = e.bytes;
        }
        ++cnt;
    }
    *n = cnt;
    if (reset) ctx->prof.reset();
    return DW_OK;
}

// ---- host-only small dense routines (include/dwsolve_dense.h) --------------
int dw_dense_eig(int n, const double* A, double* lam, double* vecs) {
    if (n < 1 || !A || !lam || !vecs) return fail(DW_EINVAL, "bad argument");
    return eig(n, reinterpret_cast<const zd*>(A), reinterpret_cast<zd*>(lam), reinterpret_cast<zd*>(vecs)) == 0
               ? DW_OK
               : fail(DW_EBREAKDOWN, "eigenvalue iteration did not converge");
}

int dw_dense_qr(int rows, int cols, const double* G, double* Q, double* R) {
    if (rows < cols || cols < 1 || !G || !Q) return fail(DW_EINVAL, "bad argument");
    return qr_positive(rows, cols, reinterpret_cast<const zd*>(G), reinterpret_cast<zd*>(Q),
                       reinterpret_cast<zd*>(R)) == 0
               ? DW_OK
               : fail(DW_EBREAKDOWN, "rank-deficient matrix");
}

int dw_dense_lstsq(int rows, int cols, int dense_rows, const double* H, const double* c, double* eta,
                   double* residual) {
    if (rows < cols + 1 || cols < 1 || !H || !c || !eta || !residual) return fail(DW_EINVAL, "bad argument");
    GivensLS ls;
    ls.reset(reinterpret_cast<const zd*>(c), rows, cols);
    std::vector<zd> col(rows);
    const zd* Hz = reinterpret_cast<const zd*>(H);
    for (int j = 0; j < cols; ++j) {
        for (int i = 0; i < rows; ++i) col[i] = Hz[(size_t)i * cols + j];
        const int nz = (j < dense_rows - 1) ? dense_rows : j + 2;
        residual[j] = ls.add_column(col.data(), nz < rows ? nz : rows);
    }
    ls.solve(reinterpret_cast<zd*>(eta));
    return DW_OK;
}

int dw_dense_solve(int n, const double* A, double* b) {
    if (n < 1 || !A || !b) return fail(DW_EINVAL, "bad argument");
    const zd* Az = reinterpret_cast<const zd*>(A);
    std::vector<zd> M(Az, Az + (size_t)n * n);
    return lu_solve(n, M, reinterpret_cast<zd*>(b)) == 0 ? DW_OK : fail(DW_EBREAKDOWN, "singular matrix");
}

}  // extern "C"
