// Host-side internals of the library: the context object and the launchers
// of the CUDA kernels (declared here, defined in the .cu files).
#pragma once

#include <cuda_runtime.h>

#include <atomic>

#include <complex>
#include <string>
#include <vector>

#include "../../include/dwsolve.h"
#include "common.cuh"

namespace dwk {

typedef std::complex<double> zd;

// thread-local error message behind dw_last_error()
void set_error(const std::string& msg);
int fail(int code, const std::string& msg);

#define DW_CUDA_TRY(expr)                                                                       \
    do {                                                                                        \
        cudaError_t _e = (expr);                                                                \
        if (_e != cudaSuccess)                                                                  \
            return ::dwk::fail(DW_ECUDA, std::string(#expr) + ": " + cudaGetErrorString(_e));   \
    } while (0)

// Largest lattice a context accepts: spinor element indices (24 reals per
// site) stay below 2^31, so device code may use 32-bit site arithmetic.
constexpr long long kMaxSites = (1LL << 31) / 24;

// V = d1 d2 d3 d4 for caller-supplied extents, checked as it is formed: every
// extent >= 2 and the running product <= max_sites (so the product can neither
// overflow nor wrap to a small value). Returns false with *V untouched otherwise.
inline bool lattice_volume(const int* dims, long long max_sites, long long* V) {
    long long v = 1;
    for (int j = 0; j < 4; ++j) {
        if (dims[j] < 2 || dims[j] > max_sites) return false;
        v *= dims[j];
        if (v > max_sites) return false;
    }
    *V = v;
    return true;
}

// Every kernel launch of the library is followed by DW_LAUNCH_CHECK(): it
// counts the launch (dw_kernel_launches()) and turns a launch error into DW_ECUDA.
void count_launch();
#define DW_LAUNCH_CHECK()          \
    do {                           \
        ::dwk::count_launch();     \
        DW_CUDA_TRY(cudaGetLastError()); \
    } while (0)

// A device allocation owned by the library (grown on demand, freed with the owner).
struct DevBuf {
    void* p = nullptr;
    size_t bytes = 0;
    cudaStream_t st = nullptr;  // allocations are stream-ordered on the owner's stream
    int ensure(size_t n);
    void release();
    template <class T>
    T* as() const { return reinterpret_cast<T*>(p); }
    ~DevBuf() { release(); }
};

// Per-kernel-class timing, collected with CUDA events on the library stream
// while profiling is switched on.
struct KernelProfile {
    std::string name;
    long long launches = 0;
    double total_ms = 0.0;
    double bytes = 0.0;  // algorithmic bytes summed over launches
    std::vector<std::pair<cudaEvent_t, cudaEvent_t>> pending;
    std::vector<double> pending_bytes;
};

struct Profiler {
    bool on = false;
    std::vector<KernelProfile> k;
    std::vector<cudaEvent_t> pool;  // recycled events (creation is not free)
    cudaStream_t stream = nullptr;
    cudaEvent_t take();
    int begin(const char* name, double bytes, cudaEvent_t* start_out, int* idx);
    void end(int idx, cudaEvent_t start);
    void drain();  // turn pending event pairs into totals (synchronises)
    void reset();
    ~Profiler();
};

// RAII helper: times the launches issued in its scope as one entry.
struct ProfScope {
    Profiler* p;
    int idx = -1;
    cudaEvent_t start = nullptr;
    ProfScope(Profiler* prof, const char* name, double bytes) : p(prof) {
        if (p && p->on) p->begin(name, bytes, &start, &idx);
    }
    ~ProfScope() {
        if (p && p->on && idx >= 0) p->end(idx, start);
    }
};

struct Workspace;                    // Krylov workspace of the solver (solver.cpp)
void release_workspace(Workspace* w);

}  // namespace dwk

namespace dwk {
// The clover term of a context: FP64 storage (double [72][V]) for double and
// double-float arithmetic, FP32 storage (float4 [18][V]) for float arithmetic.
struct ClovRef {
    const char* a64;
    const char* a32;
};

// An int in host-mapped pinned memory that kernels set to report a bounded
// wait that gave up; the host reads it after synchronising the stream.
struct HostFlag {
    int* h = nullptr;  // host address
    int* d = nullptr;  // device address
    int ensure();
    ~HostFlag();
};
}  // namespace dwk

struct dw_ctx {
    dwk::Geom g;
    double m0 = 0.0;
    cudaStream_t stream = nullptr;
    int device = 0;
    bool have_gauge = false;
    dwk::DevBuf U[5];           // gauge field per storage precision (P64, P32, P16, PB16, PDF)
    bool U_ready[5] = {false, false, false, false, false};
    dwk::DevBuf work_in, work_out, work_aux;  // conversions in dw_apply / sap_precondition
    dwk::Profiler prof;
    std::vector<int> sap_threads;  // tuned launch shape per precision (0 = default)
    dwk::Workspace* ws = nullptr;  // solver workspace, kept between solves
    double csw = 0.0;               // clover coefficient (0: plain Wilson operator)
    dwk::DevBuf clov64, clov32;     // clover term, FP64 [72][V] and FP32 float4 [18][V]
    dwk::ClovRef clov{nullptr, nullptr};
    dwk::DevBuf Uimg[4];            // SAP links per domain as shared-memory images (per storage precision)
    int Uimg_threads[4] = {0, 0, 0, 0};  // CTA size the image was packed for (0: none)
    dwk::HostFlag sap_err;          // set by a SAP sweep whose link copy did not complete
    std::atomic<int> cancel{0};     // set by dw_cancel; the running solve stops before its next step
    const dwk::ClovRef* clover() const { return csw != 0.0 ? &clov : nullptr; }
};

namespace dwk {

// gauge field in the requested storage precision (converted from FP64 on first use)
int gauge_for(dw_ctx* ctx, int prec, const char** out);

// ----- dw.cu ---------------------------------------------------------------
// canonical FP64 <-> internal layout of nrhs fields; scale (device, one double
// per rhs, may be null) multiplies every value on the way
int launch_to_internal(int prec, const double* canon, char* out, long long V, int nrhs, cudaStream_t st,
                       const double* scale = nullptr);
int launch_from_internal(int prec, const char* in, double* canon, long long V, int nrhs, cudaStream_t st,
                         const double* scale = nullptr);
int launch_gauge_convert(int prec, const double* Ucanon, char* out, long long V, cudaStream_t st);
int launch_link_convert(int prec, const char* U64, char* out, long long V, cudaStream_t st);

// out = D in  (sub == nullptr)   or   out = sub - D in  (sub: FP64 field, PO must be P64);
// with cl, D includes the clover term
int launch_dw(int pin, int pout, int plink, const Geom& g, double m0, FieldRef in, FieldRef out, const char* U,
              const int* jtab, int nrhs, const FieldRef* sub, cudaStream_t st, const ClovRef* cl = nullptr);
// ----- clover.cu -----------------------------------------------------------
int launch_clover_compute(const Geom& g, const char* U64, double csw, double* A64, float4* A32, cudaStream_t st);

// ----- sap.cu --------------------------------------------------------------
// One colour half-sweep of SAP (Algorithm 2) on every domain of `colour`:
// r = v - D x (full operator), nmr MR steps on D^l y = r, x += y.
// mode 0: x == 0 everywhere (r = v, x = y); 1: x == 0 on this colour; 2: general.
// Uimg: the links of every domain packed by launch_sap_link_image for the same
// thread count (the sweep reads its links only there); err_host: HostFlag::d,
// set if a link copy did not complete.
int launch_sap_sweep(int pspin, int plink, const Geom& g, double m0, FieldRef v, FieldRef x, const char* Uimg,
                     const int* jtab, int nrhs, int colour, int nmr, int mode, int threads, cudaStream_t st,
                     const ClovRef* cl, int* err_host);
int sap_smem_bytes(int pspin, int plink, const Geom& g, int threads);
// CTA size of the SAP sweep (threads, or the domain volume rounded up to a warp multiple when 0)
int sap_threads(const Geom& g, int threads);
size_t sap_link_image_bytes(int plink, const Geom& g, int threads);
int launch_sap_link_image(int plink, const Geom& g, const char* U, char* img, int threads, cudaStream_t st);
// links of precision prec in both layouts for a sweep of `threads` threads
// (the image is packed on first use and after dw_set_gauge), and the error flag
int sap_links_for(dw_ctx* ctx, int prec, int threads, const char** U, const char** img);
// after the stream was synchronised: DW_ETIMEOUT if a SAP link copy gave up
int sap_check(dw_ctx* ctx);

// ----- blas.cu -------------------------------------------------------------
// Outer vectors: flat arrays of 16-byte complex elements, format vp = P64
// (double2) or PDF (double-float float4). Column addressing as for FieldRef,
// in elements.
struct VecRef {
    double2* base;
    long long rhs_stride;  // in elements
    long long col_stride;  // in elements
    int col_off;
};
// out[r][i] = <V_i, w>  (i < nv[r]),  out[r][nvmax] = ||w||^2 ; nv = jtab[r] + nv_off (or nv_off)
// nv_active: the largest number of basis vectors any rhs has in this launch
// (sizes the grid); nvmax: the row length of partial/out minus one
// cnt: nrhs zeroed counters (left zeroed): the last CTA of each rhs sums the
// partial rows itself; nullptr: a separate reduction launch
int launch_multidot(int vp, VecRef Vb, VecRef w, long long n, const int* jtab, int nv_off, int nvmax, int nv_active,
                    int nrhs, double2* partial, int nblk, double2* out, cudaStream_t st, unsigned* cnt = nullptr);
// w -= sum_i coef[r][i] V_i (i < nv[r]);  out_norm2[r] = ||w||^2 after the update
int launch_multiaxpy(int vp, VecRef Vb, VecRef w, long long n, const int* jtab, int nv_off, int nrhs,
                     const double2* coef, int coef_ld, double2* partial, int nblk, double* out_norm2,
                     cudaStream_t st, unsigned* cnt = nullptr);
// dst = w / sqrt(norm2[r]) per site; if plow >= 0 also written to `low` in spinor storage plow
int launch_normalize(int vp, VecRef w, VecRef dst, long long V, const int* jtab, int nrhs, const double* norm2,
                     int plow, FieldRef low, cudaStream_t st);
// in place, per element: X_c = sum_i X_i Q[r][i][c]  (c < kout, i < nin), X in precision prec
// (scaled FP16/BF16 storage goes through `scratch`, nrhs * kout columns, and is copied back)
int launch_rotate(int prec, char* X, long long rhs_stride, long long col_stride, long long V, int nrhs,
                  const int* active, int nin, int kout, const double2* Q, int qld, char* scratch,
                  cudaStream_t st);
// x[r] += sum_i Z_i eta[r][i]  (i < nz[r]), Z in precision prec, x outer format vx;
// z_rs, z_cs, x_rs in bytes
int launch_xupdate(int prec, int vx, const char* Z, long long z_rs, long long z_cs, double2* x, long long x_rs,
                   long long V, int nrhs, const int* nz, const double2* eta, int eta_ld, cudaStream_t st);
// out[r] = ||a[r]||^2
int launch_norm2(int vp, const double2* a, long long rs, long long n, int nrhs, double2* partial, int nblk,
                 double* out, cudaStream_t st);
// convert a spinor field between storage precisions for a set of rhs
int launch_convert(int pin, int pout, FieldRef in, FieldRef out, long long V, const int* jtab, int nrhs,
                   cudaStream_t st);
// dst = a[r] * src  (outer vectors)
int launch_scale(int vp, const double2* src, double2* dst, long long rs, long long n, int nrhs, const double* a,
                 cudaStream_t st);
int launch_zero(void* p, size_t bytes, cudaStream_t st);

int blas_nblk(long long n);

// ----- solver.cpp ----------------------------------------------------------
// validated solve; it stops with DW_ECANCELLED before an Arnoldi step once
// *cancel is non-zero (cancel may be null)
int solve_checked(dw_ctx* ctx, const double* b, double* x, const dw_solver_params* P, dw_stats* S,
                  const std::atomic<int>* cancel);
int solve(dw_ctx* ctx, const double* b, double* x, const dw_solver_params* P, dw_stats* S,
          const std::atomic<int>* cancel);
// the per-cycle residual history of the last solve on ctx (see dw_residual_history)
int residual_history(dw_ctx* ctx, int rhs, double* out, int max, int* n);
// the basis of the last cycle of the last solve on ctx (see dw_debug_basis)
int debug_basis(dw_ctx* ctx, int rhs, double* V_out, double* Z_out, double* H_out, int max_cols, int* ncols);

}  // namespace dwk
