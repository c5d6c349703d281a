// FGMRES-DR (Algorithm 4) with SAP preconditioning, driven from the host.
//
// Device side (one launch per step for all right-hand sides, addressed with a
// per-rhs column table): preconditioning z_j = M v_j (SAP sweeps), the
// Arnoldi product w = D z_j, classical Gram-Schmidt with selective
// reorthogonalisation, normalisation. Host side: the (m+1) x m Hessenberg
// matrix per rhs, its Givens QR (implicit residual, Sec. 5.2 and 5.6), and at each
// cycle end the least-squares solve, the harmonic Ritz eigenproblem
// (Lemma 1a) and the QR of G_{k+1} (Eq. "G_kplus1").
//
// Refinement scheme of Sec. 5.7 (Algorithm 5): every cycle ends with an explicit FP64
// residual r = b - D x. It supplies the last column of G_{k+1} (V_{m+1}^H r),
// the vector v_{k+1} (r orthonormalised against V_k) and the right-hand side
// c = [V_{k+1}^H r; 0]; a clean restart (plain first cycle from r) follows
// when ||r|| / ||r_implicit|| > t.
//
// The Arnoldi basis V is kept either in the format of x, b, r (FP64 or
// double-float) or, as in the single-precision scheme of Sec. 5.7, in FP32
// (outer_prec = DW_F32): then the whole Arnoldi process, the deflated restart
// and the least-squares right-hand side run on FP32 vectors, while x, b and
// the explicit residual stay double-float, so every cycle refines the
// solution with a residual computed in high precision.
//
// The preconditioned vectors Z are kept in the SAP storage format, except
// that 16-bit SAP storage with deflation (k > 0) keeps Z in FP32: a deflated
// restart rotates Z_k = Z_m Q_k, and rounding the rotated vectors to 16 bits
// would break A Z_k = V_{k+1} Hhat_k at the 1e-3 level, so the implicit and
// explicit residuals would part and force clean restarts. Without rotation
// any stored z_j is consistent with its own product w = D z_j.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstring>
#include <numeric>

#include "dense.h"
#include "internal.h"

namespace dwk {

namespace {

struct RhsState {
    int j = -1;       // column being built in the current step (-1: not stepping)
    int j0 = 0;       // first Arnoldi column of the current cycle
    int mm = 0;       // columns at the end of the cycle
    bool done = false, converged = false, cycle_end = false, breakdown = false;
    int status = DW_OK;
    std::vector<zd> H;  // (m+1) x m, row-major
    std::vector<zd> c;  // m+1
    GivensLS ls;
    double bnorm = 0, rnorm = 0, res_impl = 0, wn0 = 0;
    int iterations = 0, cycles = 0, clean_restarts = 0;
    std::vector<double> hist;  // per cycle end: steps, implicit and explicit relative residual
};

struct Solver {
    dw_ctx* ctx;
    const dw_solver_params& P;
    cudaStream_t st;
    Geom g;
    long long V, n;
    int nrhs, m, k, sp, mp, op;  // op: format of x, b, r (P64 or PDF)
    int vp;             // format of the Arnoldi basis V (op, or P32)
    int zp;             // format of the preconditioned basis Z (sp, or P32)
    long long sb;       // bytes of one spinor field in SAP storage
    long long zb;       // bytes of one Z vector
    long long fb;       // bytes of one field in format op
    long long fv;       // bytes of one basis vector in format vp
    int NP;             // multi-dot row length (m + 2)
    int nblk;
    const char *U_sap, *U_sap_img, *U_mv, *U64;
    // device buffers (owned by the workspace of the context)
    char *Vb, *Zb, *xb, *bb, *rb, *vlow, *zscr, *rlow, *zsap;
    double2 *partial, *dots, *Qd, *etad;
    unsigned* cnt_d;  // reduction counters of the multi-dot and multi-axpy launches
    double *norm2d, *scal_d;
    int *jtab_d, *nz_d;
    // pinned host mirrors
    double2* dots_h;
    double* norm2_h;
    int* jtab_h;
    double* norm2_up;  // upload copies for the end of a step (the next step rewrites jtab_h
    int* jtab_up;      // before the device has necessarily consumed the previous upload)
    std::vector<RhsState> R;
    int explicit_res = 0;

    Solver(dw_ctx* c, const dw_solver_params& p) : ctx(c), P(p), st(c->stream) {}

    int lin(size_t r, int i) const { return (int)(r * NP + i); }

    VecRef vref_all(int r_off, int col_off) const {  // strides in 16-byte units
        VecRef v;
        v.base = reinterpret_cast<double2*>(Vb + (long long)r_off * (m + 1) * fv);
        v.rhs_stride = (long long)(m + 1) * fv / 16;
        v.col_stride = fv / 16;
        v.col_off = col_off;
        return v;
    }
    // the explicit residual of rhs r as seen by the basis: rb itself, or its
    // FP32 copy when the basis is FP32
    VecRef res_vec(int r_off) const {
        VecRef v;
        v.base = reinterpret_cast<double2*>((vp == op ? rb : rlow) + (long long)r_off * fv);
        v.rhs_stride = fv / 16;
        v.col_stride = 0;
        v.col_off = 0;
        return v;
    }
    int residual_to_basis(int r) {  // rlow[r] = r in FP32 (no-op for a high-precision basis)
        if (vp == op) return DW_OK;
        FieldRef in{rb + (long long)r * fb, 0, 0, 0}, out{rlow + (long long)r * fv, 0, 0, 0};
        return launch_convert(op, vp, in, out, V, nullptr, 1, st);
    }
    VecRef field_vec(char* base, int r_off) const {
        VecRef v;
        v.base = reinterpret_cast<double2*>(base) + (long long)r_off * n;
        v.rhs_stride = n;
        v.col_stride = 0;
        v.col_off = 0;
        return v;
    }

    int setup();
    int run(const double* b_user, double* x_user, dw_stats* S, const std::atomic<int>* cancel);
    int step();
    int cycle_end(int r);
    int start_plain(int r);
    int start_deflated(int r);
    int sync() {
        DW_CUDA_TRY(cudaStreamSynchronize(st));
        return sap_check(ctx);
    }
    // the step's dot rows and norms, read back with one copy (the norms follow
    // the rows in the same device buffer), then a synchronisation
    int read_dots_norms() {
        DW_CUDA_TRY(cudaMemcpyAsync(dots_h, dots, sizeof(double2) * nrhs * NP + sizeof(double) * nrhs,
                                    cudaMemcpyDeviceToHost, st));
        const int rc = sync();
        if (rc) return rc;
        std::memcpy(norm2_h, reinterpret_cast<const double*>(dots_h + (size_t)nrhs * NP), sizeof(double) * nrhs);
        return DW_OK;
    }
};

}  // namespace

// Workspace kept by the context between solves (grown on demand).
struct Workspace {
    DevBuf V, Z, x, b, r, vlow, zscr, rlow, zsap, partial, dots, Q, eta, scal, jtab, nz, canon, cnt, bscale;
    // the last solve's bases as dw_debug_basis reads them: formats, sizes and,
    // per rhs, the columns and the (m+1) x m Hessenberg-like matrix of its last cycle
    int last_nrhs = 0, last_m = 0, last_vp = -1, last_zp = -1;
    long long last_fv = 0, last_zb = 0;
    std::vector<int> last_mm;
    std::vector<std::vector<zd>> last_H;
    std::vector<std::vector<double>> last_hist;  // per rhs: (steps, implicit, explicit) per cycle
    double2* dots_h = nullptr;
    double* norm2_h = nullptr;
    int* jtab_h = nullptr;
    double* norm2_up = nullptr;
    int* jtab_up = nullptr;
    size_t dots_h_n = 0;
    ~Workspace() {
        if (dots_h) cudaFreeHost(dots_h);
        if (norm2_h) cudaFreeHost(norm2_h);
        if (jtab_h) cudaFreeHost(jtab_h);
        if (norm2_up) cudaFreeHost(norm2_up);
        if (jtab_up) cudaFreeHost(jtab_up);
    }
};

void release_workspace(Workspace* w) { delete w; }

static Workspace* workspace_of(dw_ctx* ctx) {
    if (!ctx->ws) {
        ctx->ws = new (std::nothrow) Workspace();
        if (ctx->ws)
            for (DevBuf* b : {&ctx->ws->V, &ctx->ws->Z, &ctx->ws->x, &ctx->ws->b, &ctx->ws->r, &ctx->ws->vlow,
                              &ctx->ws->zscr, &ctx->ws->rlow, &ctx->ws->zsap, &ctx->ws->partial, &ctx->ws->dots, &ctx->ws->Q, &ctx->ws->eta,
                              &ctx->ws->scal, &ctx->ws->jtab, &ctx->ws->nz, &ctx->ws->canon,
                              &ctx->ws->cnt, &ctx->ws->bscale})
                b->st = ctx->stream;
    }
    return ctx->ws;
}

namespace {

int Solver::setup() {
    g = ctx->g;
    V = g.V;
    n = 12 * V;
    nrhs = P.nrhs;
    m = P.m;
    k = P.k;
    sp = (int)P.sap_prec;
    mp = (int)P.matvec_prec;
    op = (P.outer_prec == DW_F64) ? P64 : PDF;
    vp = (P.outer_prec == DW_F32) ? P32 : op;
    zp = (k > 0 && (sp == P16 || sp == PB16)) ? P32 : sp;
    sb = spinor_bytes(sp, V);
    zb = spinor_bytes(zp, V);
    fb = spinor_bytes(op, V);
    fv = spinor_bytes(vp, V);
    NP = m + 2;
    nblk = blas_nblk(n);
    int rc;
    if ((rc = sap_links_for(ctx, sp, (ctx->sap_threads.size() > (size_t)sp) ? ctx->sap_threads[sp] : 0, &U_sap,
                            &U_sap_img)))
        return rc;
    if ((rc = gauge_for(ctx, mp == P64 ? P64 : P32, &U_mv))) return rc;
    // explicit residual: FP64 links for FP64 outer vectors, double-float links otherwise
    if ((rc = gauge_for(ctx, op == PDF ? PDF : P64, &U64))) return rc;
    Workspace* W = workspace_of(ctx);
    if (!W) return fail(DW_ENOMEM, "workspace allocation failed");
    if ((rc = W->V.ensure((size_t)nrhs * (m + 1) * fv))) return rc;
    if ((rc = W->Z.ensure((size_t)nrhs * m * zb))) return rc;
    if (zp != sp && (rc = W->zsap.ensure((size_t)nrhs * sb))) return rc;
    if ((rc = W->x.ensure((size_t)nrhs * fb))) return rc;
    if ((rc = W->b.ensure((size_t)nrhs * fb))) return rc;
    if ((rc = W->r.ensure((size_t)nrhs * fb))) return rc;
    if ((rc = W->vlow.ensure((size_t)nrhs * sb))) return rc;
    if (vp != op && (rc = W->rlow.ensure((size_t)nrhs * fv))) return rc;
    if ((rc = W->zscr.ensure((size_t)(k > 0 ? k : 1) * zb))) return rc;
    if ((rc = W->partial.ensure((size_t)nrhs * nblk * NP * sizeof(double2)))) return rc;
    // per-rhs counters of the multi-dot and multi-axpy launches (their last CTA
    // reduces the partial sums and leaves the counter at zero); zeroed per solve
    if ((rc = W->cnt.ensure((size_t)nrhs * sizeof(unsigned)))) return rc;
    DW_CUDA_TRY(cudaMemsetAsync(W->cnt.p, 0, (size_t)nrhs * sizeof(unsigned), st));
    if ((rc = W->dots.ensure((size_t)2 * nrhs * NP * sizeof(double2)))) return rc;
    if ((rc = W->Q.ensure((size_t)(m + 1) * (m + 1) * sizeof(double2)))) return rc;
    if ((rc = W->eta.ensure((size_t)(m + 1) * sizeof(double2)))) return rc;
    if ((rc = W->scal.ensure((size_t)nrhs * sizeof(double)))) return rc;
    if ((rc = W->jtab.ensure((size_t)nrhs * sizeof(int)))) return rc;
    if ((rc = W->nz.ensure(sizeof(int)))) return rc;
    if ((rc = W->bscale.ensure((size_t)2 * nrhs * sizeof(double)))) return rc;
    if (W->dots_h_n < (size_t)nrhs * NP) {
        if (W->dots_h) cudaFreeHost(W->dots_h);
        if (W->norm2_h) cudaFreeHost(W->norm2_h);
        if (W->jtab_h) cudaFreeHost(W->jtab_h);
        if (W->norm2_up) cudaFreeHost(W->norm2_up);
        if (W->jtab_up) cudaFreeHost(W->jtab_up);
        W->norm2_up = nullptr;
        W->jtab_up = nullptr;
        W->dots_h = nullptr;
        W->norm2_h = nullptr;
        W->jtab_h = nullptr;
        DW_CUDA_TRY(cudaMallocHost(&W->dots_h, (size_t)2 * DW_MAX_RHS * 66 * sizeof(double2)));
        DW_CUDA_TRY(cudaMallocHost(&W->norm2_h, (size_t)DW_MAX_RHS * sizeof(double)));
        DW_CUDA_TRY(cudaMallocHost(&W->jtab_h, (size_t)DW_MAX_RHS * sizeof(int)));
        DW_CUDA_TRY(cudaMallocHost(&W->norm2_up, (size_t)DW_MAX_RHS * sizeof(double)));
        DW_CUDA_TRY(cudaMallocHost(&W->jtab_up, (size_t)DW_MAX_RHS * sizeof(int)));
        W->dots_h_n = (size_t)DW_MAX_RHS * 66;
    }
    Vb = W->V.as<char>();
    Zb = W->Z.as<char>();
    xb = W->x.as<char>();
    bb = W->b.as<char>();
    rb = W->r.as<char>();
    vlow = W->vlow.as<char>();
    zscr = W->zscr.as<char>();
    zsap = (zp != sp) ? W->zsap.as<char>() : nullptr;
    rlow = (vp != op) ? W->rlow.as<char>() : nullptr;
    partial = W->partial.as<double2>();
    cnt_d = W->cnt.as<unsigned>();
    dots = W->dots.as<double2>();
    Qd = W->Q.as<double2>();
    etad = W->eta.as<double2>();
    // the norms follow the dots in one buffer, so that a step reads both back
    // with one copy (the dot rows take the first nrhs * NP entries)
    norm2d = reinterpret_cast<double*>(dots + (size_t)nrhs * NP);
    scal_d = W->scal.as<double>();
    jtab_d = W->jtab.as<int>();
    nz_d = W->nz.as<int>();
    dots_h = W->dots_h;
    norm2_h = W->norm2_h;
    jtab_h = W->jtab_h;
    norm2_up = W->norm2_up;
    jtab_up = W->jtab_up;
    R.assign(nrhs, RhsState());
    for (auto& s : R) {
        s.H.assign((size_t)(m + 1) * m, zd(0));
        s.c.assign(m + 1, zd(0));
    }
    return DW_OK;
}

static double ptr_bytes_dw(int pin, int pout, int plink, long long V) {
    return (double)(spinor_bytes(pin, V) + spinor_bytes(pout, V) + link_bytes(plink, V));
}

// plain first cycle (or clean restart) from the explicit residual in rb[r]
int Solver::start_plain(int r) {
    RhsState& s = R[r];
    const double nn = s.rnorm * s.rnorm;
    DW_CUDA_TRY(cudaMemcpyAsync(scal_d + r, &nn, sizeof(double), cudaMemcpyHostToDevice, st));
    int rc;
    if ((rc = residual_to_basis(r))) return rc;
    {
        ProfScope ps(&ctx->prof, "normalize", 2.0 * fv + sb);
        const FieldRef low{vlow + (long long)r * sb, 0, 0, 0};
        if ((rc = launch_normalize(vp, res_vec(r), vref_all(r, 0), V, nullptr, 1, scal_d + r, sp, low, st)))
            return rc;
    }
    std::fill(s.H.begin(), s.H.end(), zd(0));
    std::fill(s.c.begin(), s.c.end(), zd(0));
    s.c[0] = s.rnorm;
    s.ls.reset(s.c.data(), m + 1, m);
    s.j = 0;
    s.j0 = 0;
    s.cycles++;
    return sync();  // the host scalar must stay valid until the copy ran
}

int Solver::start_deflated(int r) {
    RhsState& s = R[r];
    const int mm = s.mm;
    int rc;
    // harmonic Ritz pairs (Lemma 1a): eig of H_m + f h_m^H, H_m^H f = h_m
    std::vector<zd> Hm((size_t)mm * mm), HmH((size_t)mm * mm), f(mm), hrow(mm);
    for (int i = 0; i < mm; ++i)
        for (int j = 0; j < mm; ++j) Hm[(size_t)i * mm + j] = s.H[(size_t)i * m + j];
    for (int j = 0; j < mm; ++j) hrow[j] = s.H[(size_t)mm * m + j];
    for (int i = 0; i < mm; ++i)
        for (int j = 0; j < mm; ++j) HmH[(size_t)i * mm + j] = std::conj(Hm[(size_t)j * mm + i]);
    for (int i = 0; i < mm; ++i) f[i] = std::conj(hrow[i]);
    if (lu_solve(mm, HmH, f.data()) != 0) return fail(DW_EBREAKDOWN, "singular H_m in harmonic Ritz step");
    std::vector<zd> A((size_t)mm * mm), lam(mm), G((size_t)mm * mm);
    for (int i = 0; i < mm; ++i)
        for (int j = 0; j < mm; ++j) A[(size_t)i * mm + j] = Hm[(size_t)i * mm + j] + f[i] * hrow[j];
    if (eig(mm, A.data(), lam.data(), G.data()) != 0) return fail(DW_EBREAKDOWN, "eigenvalue iteration failed");
    std::vector<int> idx(mm);
    std::iota(idx.begin(), idx.end(), 0);
    std::stable_sort(idx.begin(), idx.end(), [&](int a, int b) { return std::abs(lam[a]) < std::abs(lam[b]); });
    // last column of G_{k+1}: the explicit residual in the old basis, V_{m+1}^H r
    if ((rc = residual_to_basis(r))) return rc;
    {
        ProfScope ps(&ctx->prof, "multidot", (double)(mm + 2) * fv);
        if ((rc = launch_multidot(vp, vref_all(r, 0), res_vec(r), n, nullptr, mm + 1, m + 1, mm + 1, 1, partial,
                                  nblk, dots, st, cnt_d)))
            return rc;
    }
    DW_CUDA_TRY(cudaMemcpyAsync(dots_h, dots, sizeof(double2) * NP, cudaMemcpyDeviceToHost, st));
    if ((rc = sync())) return rc;
    const int k1 = k + 1;
    std::vector<zd> Gk1((size_t)(mm + 1) * k1, zd(0)), Q((size_t)(mm + 1) * k1);
    for (int i = 0; i < mm; ++i)
        for (int c = 0; c < k; ++c) Gk1[(size_t)i * k1 + c] = G[(size_t)i * mm + idx[c]];
    for (int i = 0; i <= mm; ++i) Gk1[(size_t)i * k1 + k] = zd(dots_h[i].x, dots_h[i].y);
    if (qr_positive(mm + 1, k1, Gk1.data(), Q.data(), nullptr) != 0)
        return fail(DW_EBREAKDOWN, "rank-deficient G_{k+1}");
    // Hhat_k = Q_{k+1}^H Hhat_m Q_k
    std::vector<zd> HQ((size_t)(mm + 1) * k, zd(0));
    for (int i = 0; i <= mm; ++i)
        for (int c = 0; c < k; ++c) {
            zd acc = 0.0;
            for (int l = 0; l < mm; ++l) acc += s.H[(size_t)i * m + l] * Q[(size_t)l * k1 + c];
            HQ[(size_t)i * k + c] = acc;
        }
    std::vector<zd> Hk((size_t)k1 * k, zd(0));
    for (int a = 0; a < k1; ++a)
        for (int c = 0; c < k; ++c) {
            zd acc = 0.0;
            for (int i = 0; i <= mm; ++i) acc += std::conj(Q[(size_t)i * k1 + a]) * HQ[(size_t)i * k + c];
            Hk[(size_t)a * k + c] = acc;
        }
    // V_{k+1} = V_{m+1} Q_{k+1},  Z_k = Z_m Q_k  (in place on the device)
    std::vector<double2> Qh((size_t)(m + 1) * (m + 1), make_double2(0, 0));
    for (int i = 0; i <= mm; ++i)
        for (int c = 0; c < k1; ++c)
            Qh[(size_t)i * (m + 1) + c] = make_double2(Q[(size_t)i * k1 + c].real(), Q[(size_t)i * k1 + c].imag());
    DW_CUDA_TRY(cudaMemcpyAsync(Qd, Qh.data(), sizeof(double2) * Qh.size(), cudaMemcpyHostToDevice, st));
    {
        ProfScope ps(&ctx->prof, "rotate_V", (double)(mm + 1 + k1) * fv);
        if ((rc = launch_rotate(vp, Vb + (long long)r * (m + 1) * fv, 0, fv, V, 1, nullptr, mm + 1, k1, Qd, m + 1,
                                nullptr, st)))
            return rc;
    }
    {
        ProfScope ps(&ctx->prof, "rotate_Z", (double)(mm + k) * zb);
        if ((rc = launch_rotate(zp, Zb + (long long)r * m * zb, 0, zb, V, 1, nullptr, mm, k, Qd, m + 1, zscr, st)))
            return rc;
    }
    // v_{k+1}: explicit residual orthonormalised against V_k (two CGS passes)
    char* Vr = Vb + (long long)r * (m + 1) * fv;
    DW_CUDA_TRY(cudaMemcpyAsync(Vr + (long long)k * fv, reinterpret_cast<char*>(res_vec(r).base), fv,
                                cudaMemcpyDeviceToDevice, st));
    for (int pass = 0; pass < 2; ++pass) {
        ProfScope ps(&ctx->prof, "cgs", (double)(2 * k + 3) * fv);
        VecRef w = vref_all(r, k);
        if ((rc = launch_multidot(vp, vref_all(r, 0), w, n, nullptr, k, m + 1, k, 1, partial, nblk, dots, st,
                                  cnt_d)))
            return rc;
        if ((rc = launch_multiaxpy(vp, vref_all(r, 0), w, n, nullptr, k, 1, dots, NP, partial, nblk, norm2d + r,
                                   st, cnt_d)))
            return rc;
    }
    {
        ProfScope ps(&ctx->prof, "normalize", 2.0 * fv);
        VecRef w = vref_all(r, k);
        const FieldRef low{vlow + (long long)r * sb, 0, 0, 0};
        if ((rc = launch_normalize(vp, w, w, V, nullptr, 1, norm2d + r, sp, low, st))) return rc;
    }
    // c = [V_{k+1}^H r; 0]
    {
        ProfScope ps(&ctx->prof, "multidot", (double)(k1 + 1) * fv);
        if ((rc = launch_multidot(vp, vref_all(r, 0), res_vec(r), n, nullptr, k1, m + 1, k1, 1, partial, nblk, dots,
                                  st, cnt_d)))
            return rc;
    }
    DW_CUDA_TRY(cudaMemcpyAsync(dots_h, dots, sizeof(double2) * NP, cudaMemcpyDeviceToHost, st));
    if ((rc = sync())) return rc;
    std::fill(s.H.begin(), s.H.end(), zd(0));
    std::fill(s.c.begin(), s.c.end(), zd(0));
    for (int a = 0; a < k1; ++a)
        for (int c = 0; c < k; ++c) s.H[(size_t)a * m + c] = Hk[(size_t)a * k + c];
    for (int a = 0; a < k1; ++a) s.c[a] = zd(dots_h[a].x, dots_h[a].y);
    s.ls.reset(s.c.data(), m + 1, m);
    std::vector<zd> col(m + 1);
    for (int c = 0; c < k; ++c) {
        for (int a = 0; a <= m; ++a) col[a] = s.H[(size_t)a * m + c];
        s.ls.add_column(col.data(), k1);
    }
    s.j = k;
    s.j0 = k;
    s.cycles++;
    return DW_OK;
}

int Solver::cycle_end(int r) {
    RhsState& s = R[r];
    int rc;
    const int mm = s.mm;
    std::vector<zd> eta(mm);
    s.ls.solve(eta.data());
    s.res_impl = s.ls.residual();
    std::vector<double2> eh(mm);
    for (int i = 0; i < mm; ++i) eh[i] = make_double2(eta[i].real(), eta[i].imag());
    DW_CUDA_TRY(cudaMemcpyAsync(etad, eh.data(), sizeof(double2) * mm, cudaMemcpyHostToDevice, st));
    DW_CUDA_TRY(cudaMemcpyAsync(nz_d, &mm, sizeof(int), cudaMemcpyHostToDevice, st));
    {
        ProfScope ps(&ctx->prof, "xupdate", (double)mm * zb + 2.0 * fb);
        if ((rc = launch_xupdate(zp, op, Zb + (long long)r * m * zb, 0, zb,
                                 reinterpret_cast<double2*>(xb) + (long long)r * n, 0, V, 1, nz_d, etad, 0, st)))
            return rc;
    }
    // explicit FP64 residual r = b - D x
    {
        ProfScope ps(&ctx->prof, "dw_f64_residual", ptr_bytes_dw(op, op, op, V) + fb);
        FieldRef in{xb + (long long)r * fb, 0, 0, 0}, out{rb + (long long)r * fb, 0, 0, 0},
            sub{bb + (long long)r * fb, 0, 0, 0};
        if ((rc = launch_dw(op, op, op, g, ctx->m0, in, out, U64, nullptr, 1, &sub, st, ctx->clover()))) return rc;
    }
    explicit_res++;
    {
        ProfScope ps(&ctx->prof, "norm2", (double)fb);
        if ((rc = launch_norm2(op, reinterpret_cast<double2*>(rb) + (long long)r * n, 0, n, 1, partial, nblk,
                               norm2d + r, st)))
            return rc;
    }
    DW_CUDA_TRY(cudaMemcpyAsync(norm2_h + r, norm2d + r, sizeof(double), cudaMemcpyDeviceToHost, st));
    if ((rc = sync())) return rc;
    s.rnorm = std::sqrt(norm2_h[r]);
    s.hist.push_back((double)s.iterations);
    s.hist.push_back(s.bnorm > 0 ? s.res_impl / s.bnorm : 0.0);
    s.hist.push_back(s.bnorm > 0 ? s.rnorm / s.bnorm : 0.0);
    if (!std::isfinite(s.rnorm)) {
        s.done = true;
        s.status = DW_ENONFINITE;
        return DW_OK;
    }
    if (s.rnorm <= P.tol * s.bnorm) {
        s.done = true;
        s.converged = true;
        return DW_OK;
    }
    if ((P.max_iterations > 0 && s.iterations >= P.max_iterations) || s.cycles >= P.max_cycles) {
        s.done = true;
        s.status = DW_ENOTCONV;
        return DW_OK;
    }
    const bool clean = (k == 0) || mm <= k || s.res_impl == 0.0 || (s.rnorm / s.res_impl > P.clean_restart_t);
    if (k > 0 && clean) s.clean_restarts++;
    return clean ? start_plain(r) : start_deflated(r);
}

// One flexible Arnoldi step (Algorithm 3/4 inner loop) for every stepping rhs.
int Solver::step() {
    int rc;
    int nact = 0;
    for (int r = 0; r < nrhs; ++r) {
        jtab_h[r] = (!R[r].done && R[r].j >= 0) ? R[r].j : -1;
        nact += jtab_h[r] >= 0;
    }
    if (nact == 0) return fail(DW_EBREAKDOWN, "no right-hand side left to step");
    DW_CUDA_TRY(cudaMemcpyAsync(jtab_d, jtab_h, sizeof(int) * nrhs, cudaMemcpyHostToDevice, st));
    const FieldRef Vf1{Vb, (m + 1) * fv, fv, 1};
    const FieldRef Zf{Zb, m * zb, zb, 0};
    const FieldRef Lf{vlow, sb, 0, 0};
    const FieldRef Zs = (zp == sp) ? Zf : FieldRef{zsap, sb, 0, 0};  // where the SAP writes z_j
    // z_j = M v_j  (v_j was written in SAP storage to vlow when it was normalised)
    for (int cyc = 0; cyc < P.sap_cycles; ++cyc)
        for (int colour = 0; colour < 2; ++colour) {
            const int mode = (cyc > 0) ? 2 : (colour == 0 ? 0 : 1);
            const double bytes = (double)nact * 0.5 * (2.0 * sb + (mode == 2 ? sb : 0) + link_bytes(sp, V));
            ProfScope ps(&ctx->prof, "sap_sweep", bytes);
            const int thr = (ctx->sap_threads.size() > (size_t)sp) ? ctx->sap_threads[sp] : 0;
            if ((rc = launch_sap_sweep(sp, sp, g, ctx->m0, Lf, Zs, U_sap_img, jtab_d, nrhs, colour, P.mr_steps,
                                       mode, thr, st, ctx->clover(), ctx->sap_err.d)))
                return rc;
        }
    if (zp != sp) {
        ProfScope ps(&ctx->prof, "z_widen", (double)nact * (sb + zb));
        if ((rc = launch_convert(sp, zp, Zs, Zf, V, jtab_d, nrhs, st))) return rc;
    }
    // w = D z_j  (written into column j+1 of V)
    {
        const int pl = (mp == P64) ? P64 : P32;
        // the links count once for all right-hand sides of the launch (L2 serves the re-reads)
        const double link_reads = 1.0;
        ProfScope ps(&ctx->prof, "dw_matvec",
                     (double)nact * (spinor_bytes(zp, V) + spinor_bytes(vp, V)) + link_reads * link_bytes(pl, V));
        if ((rc = launch_dw(zp, vp, pl, g, ctx->m0, Zf, Vf1, U_mv, jtab_d, nrhs, nullptr, st, ctx->clover())))
            return rc;
    }
    // classical Gram-Schmidt: h = V^H w, w' = w - V h; a second projection
    // ("twice is enough") only where cancellation could cost orthogonality at
    // the working precision: u / (||w'|| / ||w||) > 1e-13
    double jsum = 0;
    int jmax = 0;
    for (int r = 0; r < nrhs; ++r)
        if (jtab_h[r] >= 0) jsum += jtab_h[r] + 1, jmax = std::max(jmax, jtab_h[r]);
    {
        ProfScope ps(&ctx->prof, "cgs_project", (jsum + nact) * fv);
        if ((rc = launch_multidot(vp, vref_all(0, 0), vref_all(0, 1), n, jtab_d, 1, m + 1, jmax + 1, nrhs, partial,
                                  nblk, dots, st, cnt_d)))
            return rc;
    }
    {
        ProfScope ps(&ctx->prof, "cgs_update", (jsum + 2.0 * nact) * fv);
        if ((rc = launch_multiaxpy(vp, vref_all(0, 0), vref_all(0, 1), n, jtab_d, 1, nrhs, dots, NP, partial, nblk,
                                   norm2d, st, cnt_d)))
            return rc;
    }
    if ((rc = read_dots_norms())) return rc;
    // unit roundoff of the basis format, and the orthogonality level below
    // which a second pass is taken (FP64-class: 1e-13; FP32: 1e-5)
    const double unit = (vp == P32) ? 5.960464477539063e-08 : (vp == PDF) ? 3.552713678800501e-15
                                                                            : 1.1102230246251565e-16;
    const double tau = (vp == P32) ? 1e-5 : 1e-13;
    std::vector<std::vector<zd>> h(nrhs);
    bool need2 = false;
    for (int r = 0; r < nrhs; ++r) {
        if (jtab_h[r] < 0) continue;
        const int j = jtab_h[r];
        h[r].resize(j + 2);
        for (int i = 0; i <= j; ++i) h[r][i] = zd(dots_h[lin(r, i)].x, dots_h[lin(r, i)].y);
        R[r].wn0 = std::sqrt(dots_h[lin(r, m + 1)].x);
        const double ratio = std::sqrt(norm2_h[r]) / (R[r].wn0 > 0 ? R[r].wn0 : 1.0);
        const bool re = unit > tau * ratio;
        need2 |= re;
        if (!re) jtab_h[r] = -1;
    }
    if (need2) {
        DW_CUDA_TRY(cudaMemcpyAsync(jtab_d, jtab_h, sizeof(int) * nrhs, cudaMemcpyHostToDevice, st));
        double js2 = 0;
        int n2 = 0, jmax2 = 0;
        for (int r = 0; r < nrhs; ++r)
            if (jtab_h[r] >= 0) js2 += jtab_h[r] + 1, ++n2, jmax2 = std::max(jmax2, jtab_h[r]);
        std::vector<double> keep(norm2_h, norm2_h + nrhs);
        {
            ProfScope ps(&ctx->prof, "cgs_reorth", (2.0 * js2 + 3.0 * n2) * fv);
            if ((rc = launch_multidot(vp, vref_all(0, 0), vref_all(0, 1), n, jtab_d, 1, m + 1, jmax2 + 1, nrhs,
                                      partial, nblk, dots, st, cnt_d)))
                return rc;
            if ((rc = launch_multiaxpy(vp, vref_all(0, 0), vref_all(0, 1), n, jtab_d, 1, nrhs, dots, NP, partial,
                                       nblk, norm2d, st, cnt_d)))
                return rc;
        }
        if ((rc = read_dots_norms())) return rc;
        for (int r = 0; r < nrhs; ++r) {
            if (jtab_h[r] < 0) {
                norm2_h[r] = keep[r];
                continue;
            }
            for (int i = 0; i <= jtab_h[r]; ++i) h[r][i] += zd(dots_h[lin(r, i)].x, dots_h[lin(r, i)].y);
        }
    }
    // restore the step's column table; v_{j+1} = w / ||w|| (also into SAP storage)
    for (int r = 0; r < nrhs; ++r) {
        jtab_h[r] = (!R[r].done && R[r].j >= 0) ? R[r].j : -1;
        jtab_up[r] = jtab_h[r];
        norm2_up[r] = norm2_h[r];
    }
    if (need2) {
        // without a second pass the device still holds this step's column
        // table and the norms just read back: the uploads are needed only
        // after a second pass changed them (this is the one host round trip
        // of a step, so every call saved shortens the GPU's idle gap)
        DW_CUDA_TRY(cudaMemcpyAsync(jtab_d, jtab_up, sizeof(int) * nrhs, cudaMemcpyHostToDevice, st));
        DW_CUDA_TRY(cudaMemcpyAsync(norm2d, norm2_up, sizeof(double) * nrhs, cudaMemcpyHostToDevice, st));
    }
    {
        ProfScope ps(&ctx->prof, "normalize", (double)nact * (2.0 * fv + sb));
        if ((rc = launch_normalize(vp, vref_all(0, 1), vref_all(0, 1), V, jtab_d, nrhs, norm2d, sp, Lf, st)))
            return rc;
    }
    // host: Hessenberg column, Givens update, end-of-cycle tests
    for (int r = 0; r < nrhs; ++r) {
        RhsState& s = R[r];
        if (s.done || s.j < 0) continue;
        const int j = s.j;
        const double hn = std::sqrt(norm2_h[r]);
        h[r][j + 1] = hn;
        bool finite = std::isfinite(hn);
        for (int i = 0; i <= j + 1; ++i) {
            finite &= std::isfinite(h[r][i].real()) && std::isfinite(h[r][i].imag());
            s.H[(size_t)i * m + j] = h[r][i];
        }
        s.iterations++;
        if (!finite) {
            s.done = true;
            s.status = DW_ENONFINITE;
            continue;
        }
        std::vector<zd> col(m + 1, zd(0));
        for (int i = 0; i <= j + 1; ++i) col[i] = s.H[(size_t)i * m + j];
        const double res = s.ls.add_column(col.data(), j + 2);
        const bool breakdown = hn <= 1e-14 * s.wn0;
        const bool limit = P.max_iterations > 0 && s.iterations >= P.max_iterations;
        if (breakdown || res <= P.tol * s.bnorm || j + 1 == m || limit) {
            s.mm = j + 1;
            s.cycle_end = true;
            s.j = -1;
        } else {
            s.j = j + 1;
        }
    }
    // no synchronisation here: the next step's launches queue behind the
    // normalisation (its uploads read jtab_up / norm2_up, which are only
    // rewritten after the next step's first synchronisation)
    for (int r = 0; r < nrhs; ++r)
        if (R[r].cycle_end) {
            R[r].cycle_end = false;
            if ((rc = cycle_end(r))) return rc;
        }
    return DW_OK;
}

int Solver::run(const double* b_user, double* x_user, dw_stats* S, const std::atomic<int>* cancel) {
    int rc;
    const auto t0 = std::chrono::steady_clock::now();
    Workspace* W = workspace_of(ctx);
    const size_t canon_bytes = (size_t)nrhs * 24 * V * sizeof(double);
    const double* b_dev = b_user;
    double* x_dev = x_user;
    if (P.host_buffers) {
        if ((rc = W->canon.ensure(canon_bytes))) return rc;
        DW_CUDA_TRY(cudaMemcpyAsync(W->canon.p, b_user, canon_bytes, cudaMemcpyHostToDevice, st));
        b_dev = W->canon.as<double>();
    }
    // The system is solved for b scaled by the power of two nearest 1/||b|| (a
    // per-rhs exponent shift, exact in every format, so results for b of
    // moderate size are bit-identical to unscaled ones): the double-float and
    // FP32 vectors keep FP32's exponent range, which b near 1e+-30 would
    // otherwise leave in the squares of the norms. x is scaled back on output.
    if ((rc = launch_norm2(P64, reinterpret_cast<const double2*>(b_dev), n, n, nrhs, partial, nblk, norm2d, st)))
        return rc;
    DW_CUDA_TRY(cudaMemcpyAsync(norm2_h, norm2d, sizeof(double) * nrhs, cudaMemcpyDeviceToHost, st));
    if ((rc = sync())) return rc;
    std::vector<double> bscale(2 * nrhs, 1.0);  // [0, nrhs): into the solver; [nrhs, 2 nrhs): back out
    for (int r = 0; r < nrhs; ++r) {
        const double bn = std::sqrt(norm2_h[r]);
        if (bn > 0.0 && std::isfinite(bn)) {
            int e = 0;
            std::frexp(bn, &e);  // bn = f 2^e, f in [0.5, 1)
            bscale[r] = std::ldexp(1.0, -e);
            bscale[nrhs + r] = std::ldexp(1.0, e);
        }
    }
    double* bscale_d = W->bscale.as<double>();
    DW_CUDA_TRY(cudaMemcpyAsync(bscale_d, bscale.data(), sizeof(double) * 2 * nrhs, cudaMemcpyHostToDevice, st));
    if ((rc = launch_to_internal(op, b_dev, bb, V, nrhs, st, bscale_d))) return rc;
    if (P.use_x0) {
        if (P.host_buffers) {
            if ((rc = sync())) return rc;
            DW_CUDA_TRY(cudaMemcpyAsync(W->canon.p, x_user, canon_bytes, cudaMemcpyHostToDevice, st));
            x_dev = W->canon.as<double>();
        }
        if ((rc = launch_to_internal(op, x_dev, xb, V, nrhs, st, bscale_d))) return rc;
        FieldRef in{xb, fb, 0, 0}, out{rb, fb, 0, 0}, sub{bb, fb, 0, 0};
        if ((rc = launch_dw(op, op, op, g, ctx->m0, in, out, U64, nullptr, nrhs, &sub, st, ctx->clover())))
            return rc;
        explicit_res++;
    } else {
        DW_CUDA_TRY(cudaMemsetAsync(xb, 0, (size_t)nrhs * fb, st));
        DW_CUDA_TRY(cudaMemcpyAsync(rb, bb, (size_t)nrhs * fb, cudaMemcpyDeviceToDevice, st));
    }
    if ((rc = launch_norm2(op, reinterpret_cast<double2*>(bb), n, n, nrhs, partial, nblk, norm2d, st))) return rc;
    DW_CUDA_TRY(cudaMemcpyAsync(norm2_h, norm2d, sizeof(double) * nrhs, cudaMemcpyDeviceToHost, st));
    if ((rc = sync())) return rc;
    std::vector<double> bn(norm2_h, norm2_h + nrhs);
    if ((rc = launch_norm2(op, reinterpret_cast<double2*>(rb), n, n, nrhs, partial, nblk, norm2d, st))) return rc;
    DW_CUDA_TRY(cudaMemcpyAsync(norm2_h, norm2d, sizeof(double) * nrhs, cudaMemcpyDeviceToHost, st));
    if ((rc = sync())) return rc;
    for (int r = 0; r < nrhs; ++r) {
        RhsState& s = R[r];
        s.bnorm = std::sqrt(bn[r]);
        s.rnorm = std::sqrt(norm2_h[r]);
        if (!std::isfinite(s.bnorm) || !std::isfinite(s.rnorm)) {
            s.done = true;
            s.status = DW_ENONFINITE;
        } else if (s.bnorm == 0.0 || s.rnorm <= P.tol * s.bnorm) {
            s.done = true;
            s.converged = true;
        } else if ((rc = start_plain(r))) {
            return rc;
        }
    }
    bool cancelled = false;
    for (;;) {
        bool any = false;
        for (auto& s : R) any |= !s.done;
        if (!any) break;
        if (cancel && cancel->load(std::memory_order_relaxed)) {
            cancelled = true;
            break;
        }
        if ((rc = step())) return rc;
    }
    // result back to the caller's layout
    if (P.host_buffers) {
        if ((rc = launch_from_internal(op, xb, W->canon.as<double>(), V, nrhs, st, bscale_d + nrhs))) return rc;
        DW_CUDA_TRY(cudaMemcpyAsync(x_user, W->canon.p, canon_bytes, cudaMemcpyDeviceToHost, st));
    } else {
        if ((rc = launch_from_internal(op, xb, x_user, V, nrhs, st, bscale_d + nrhs))) return rc;
    }
    if ((rc = sync())) return rc;
    // keep the last cycle of every rhs for dw_debug_basis
    W->last_nrhs = nrhs;
    W->last_m = m;
    W->last_vp = vp;
    W->last_zp = zp;
    W->last_fv = fv;
    W->last_zb = zb;
    W->last_mm.assign(nrhs, 0);
    W->last_H.assign(nrhs, std::vector<zd>());
    W->last_hist.assign(nrhs, std::vector<double>());
    for (int r = 0; r < nrhs; ++r) {
        W->last_mm[r] = (R[r].j < 0) ? R[r].mm : 0;  // a cycle stopped mid-way has no consistent basis
        W->last_H[r] = R[r].H;
        W->last_hist[r] = R[r].hist;
    }
    int status = DW_OK, conv = 0;
    for (auto& s : R) {
        conv += s.converged;
        if (s.status != DW_OK && status == DW_OK) status = s.status;
    }
    if (cancelled && status == DW_OK) status = DW_ECANCELLED;
    if (S) {
        std::memset(S, 0, sizeof(*S));
        for (int r = 0; r < nrhs; ++r) {
            S->iterations = std::max(S->iterations, R[r].iterations);
            S->cycles = std::max(S->cycles, R[r].cycles);
            S->clean_restarts += R[r].clean_restarts;
            S->iterations_rhs[r] = R[r].iterations;
            S->true_rel_res[r] = R[r].bnorm > 0 ? R[r].rnorm / R[r].bnorm : 0.0;
        }
        S->converged = conv;
        S->explicit_residuals = explicit_res;
        S->time_s = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    }
    if (status != DW_OK)
        return fail(status, status == DW_ENOTCONV    ? "iteration limit reached before the tolerance"
                            : status == DW_ECANCELLED ? "solve cancelled"
                                                      : "non-finite values in the Krylov process");
    return DW_OK;
}

}  // namespace

int solve(dw_ctx* ctx, const double* b, double* x, const dw_solver_params* P, dw_stats* S,
          const std::atomic<int>* cancel) {
    Solver s(ctx, *P);
    int rc = s.setup();
    if (rc) return rc;
    return s.run(b, x, S, cancel);
}

int residual_history(dw_ctx* ctx, int rhs, double* out, int max, int* n) {
    Workspace* W = ctx->ws;
    if (!W || W->last_nrhs == 0) return fail(DW_EINVAL, "no solve has run on this context");
    if (rhs < 0 || rhs >= W->last_nrhs) return fail(DW_EINVAL, "rhs out of range");
    const std::vector<double>& h = W->last_hist[rhs];
    *n = (int)(h.size() / 3);
    if (out)
        for (int i = 0; i < 3 * std::min(*n, max); ++i) out[i] = h[i];
    return DW_OK;
}

int debug_basis(dw_ctx* ctx, int rhs, double* V_out, double* Z_out, double* H_out, int max_cols, int* ncols) {
    Workspace* W = ctx->ws;
    if (!W || W->last_nrhs == 0) return fail(DW_EINVAL, "no solve has run on this context");
    if (rhs < 0 || rhs >= W->last_nrhs) return fail(DW_EINVAL, "rhs out of range");
    const int mm = W->last_mm[rhs];
    *ncols = mm;
    if (mm == 0) return DW_OK;
    if (max_cols < mm) return fail(DW_EINVAL, "max_cols is smaller than the basis");
    const long long V = ctx->g.V;
    const int m = W->last_m;
    cudaStream_t st = ctx->stream;
    int rc;
    if (V_out) {
        const char* Vr = W->V.as<char>() + (long long)rhs * (m + 1) * W->last_fv;
        for (int i = 0; i <= mm; ++i)
            if ((rc = launch_from_internal(W->last_vp, Vr + i * W->last_fv, V_out + (long long)i * 24 * V, V, 1, st)))
                return rc;
    }
    if (Z_out) {
        const char* Zr = W->Z.as<char>() + (long long)rhs * m * W->last_zb;
        for (int i = 0; i < mm; ++i)
            if ((rc = launch_from_internal(W->last_zp, Zr + i * W->last_zb, Z_out + (long long)i * 24 * V, V, 1, st)))
                return rc;
    }
    if (H_out) {
        const std::vector<zd>& H = W->last_H[rhs];
        for (int i = 0; i <= mm; ++i)
            for (int j = 0; j < mm; ++j) {
                H_out[2 * ((size_t)i * mm + j)] = H[(size_t)i * m + j].real();
                H_out[2 * ((size_t)i * mm + j) + 1] = H[(size_t)i * m + j].imag();
            }
    }
    DW_CUDA_TRY(cudaStreamSynchronize(st));
    return DW_OK;
}

}  // namespace dwk
