// Level-1 kernels of the flexible Arnoldi process and of the deflated restart
// (Algorithms 3 and 4): fused multi-dot products, multi-axpy with the norm of
// the result, normalisation, the basis rotations V_{k+1} = V_{m+1} Q_{k+1},
// Z_k = Z_m Q_k, and the iterate update x += Z eta.
//
// The outer vectors (basis V, iterate x, right-hand side b, residual r) are
// flat arrays of 16-byte complex elements in one of two formats:
//   P64 : double2, FP64 arithmetic;
//   PDF : float4 double-float pairs, double-float arithmetic on the FP32
//         pipes (same footprint, 48-bit significand) -- the GB300 FP64 rate
//         would otherwise cap these HBM-bound sweeps far below bandwidth.
// Reductions are deterministic: every CTA writes its partial sums (FP64) to a
// fixed slot and one CTA per right-hand side adds the slots in order.
#include <atomic>
#include <mutex>
#include <set>

#include "internal.h"

namespace dwk {

namespace {

constexpr int kT = 256;      // threads per CTA
constexpr int kRotMax = 17;  // output columns held in registers by a rotation
constexpr int kMaxV = 64;    // basis vectors per multi-dot / multi-axpy

__device__ __forceinline__ double warp_sum(double a) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) a += __shfl_xor_sync(0xffffffffu, a, o);
    return a;
}

__device__ __forceinline__ int rhs_nv(const int* jtab, int r, int off) { return jtab ? jtab[r] + off : off; }

// ---- element access: complex element e of a flat outer vector ---------------
template <int VP>
struct Elem;

template <>
struct Elem<P64> {
    typedef double2 T;
    struct C {  // complex accumulator / value
        double re, im;
    };
    static __device__ __forceinline__ C load(const double2* p, long long e) {
        const double2 v = __ldg(&p[e]);
        return C{v.x, v.y};
    }
    static __device__ __forceinline__ C load_rw(const double2* p, long long e) {
        const double2 v = p[e];
        return C{v.x, v.y};
    }
    static __device__ __forceinline__ void store(double2* p, long long e, C v) { p[e] = make_double2(v.re, v.im); }
    static __device__ __forceinline__ C zero() { return C{0.0, 0.0}; }
    // acc += conj(a) * b
    static __device__ __forceinline__ void mac_conj(C& acc, C a, C b) {
        acc.re = fma(a.re, b.re, acc.re);
        acc.re = fma(a.im, b.im, acc.re);
        acc.im = fma(a.re, b.im, acc.im);
        acc.im = fma(-a.im, b.re, acc.im);
    }
    // acc += h * a
    static __device__ __forceinline__ void mac(C& acc, C h, C a) {
        acc.re = fma(h.re, a.re, acc.re);
        acc.re = fma(-h.im, a.im, acc.re);
        acc.im = fma(h.re, a.im, acc.im);
        acc.im = fma(h.im, a.re, acc.im);
    }
    typedef double N;  // |.|^2 accumulator
    static __device__ __forceinline__ N nzero() { return 0.0; }
    static __device__ __forceinline__ void norm2_acc(N& s, C a) { s = fma(a.re, a.re, fma(a.im, a.im, s)); }
    static __device__ __forceinline__ double nfin(N s) { return s; }
    static __device__ __forceinline__ C fin(C a) { return a; }
    static __device__ __forceinline__ double2 to_d2(C a) { return make_double2(a.re, a.im); }
    static __device__ __forceinline__ C from_d2(double2 a) { return C{a.x, a.y}; }
    static __device__ __forceinline__ C warp_reduce(C a) { return C{warp_sum(a.re), warp_sum(a.im)}; }
    static __device__ __forceinline__ C scale(C a, double s) { return C{a.re * s, a.im * s}; }
    static __device__ __forceinline__ cx<float> to_f(C a) { return mk<float>((float)a.re, (float)a.im); }
    static __device__ __forceinline__ C add(C a, C b) { return C{a.re + b.re, a.im + b.im}; }
};

// FP32 basis vectors (the single-precision Arnoldi process of Sec. 5.7): one
// float2 per complex element, in the S32 spinor layout (float4[6][V], two
// complex per site and plane). Dot products and updates are element-wise, so
// they never depend on which complex element sits where; the per-site
// normalisation uses the spinor layout explicitly. Products accumulate in
// FP32 per thread and in FP64 across threads.
template <>
struct Elem<P32> {
    typedef float2 T;
    struct C {
        float re, im;
    };
    static __device__ __forceinline__ C load(const double2* p, long long e) {
        const float2 v = __ldg(&reinterpret_cast<const float2*>(p)[e]);
        return C{v.x, v.y};
    }
    static __device__ __forceinline__ C load_rw(const double2* p, long long e) {
        const float2 v = reinterpret_cast<const float2*>(p)[e];
        return C{v.x, v.y};
    }
    static __device__ __forceinline__ void store(double2* p, long long e, C v) {
        reinterpret_cast<float2*>(p)[e] = make_float2(v.re, v.im);
    }
    static __device__ __forceinline__ C zero() { return C{0.f, 0.f}; }
    static __device__ __forceinline__ void mac_conj(C& acc, C a, C b) {
        acc.re = fmaf(a.re, b.re, acc.re);
        acc.re = fmaf(a.im, b.im, acc.re);
        acc.im = fmaf(a.re, b.im, acc.im);
        acc.im = fmaf(-a.im, b.re, acc.im);
    }
    static __device__ __forceinline__ void mac(C& acc, C h, C a) {
        acc.re = fmaf(h.re, a.re, acc.re);
        acc.re = fmaf(-h.im, a.im, acc.re);
        acc.im = fmaf(h.re, a.im, acc.im);
        acc.im = fmaf(h.im, a.re, acc.im);
    }
    typedef float N;
    static __device__ __forceinline__ N nzero() { return 0.f; }
    static __device__ __forceinline__ void norm2_acc(N& s, C a) { s = fmaf(a.re, a.re, fmaf(a.im, a.im, s)); }
    static __device__ __forceinline__ double nfin(N s) { return (double)s; }
    static __device__ __forceinline__ C fin(C a) { return a; }
    static __device__ __forceinline__ double2 to_d2(C a) { return make_double2((double)a.re, (double)a.im); }
    static __device__ __forceinline__ C from_d2(double2 a) { return C{(float)a.x, (float)a.y}; }
    // reduced in FP64: the per-thread FP32 partial sums are converted first
    static __device__ __forceinline__ double2 warp_reduce_d(C a) {
        return make_double2(warp_sum((double)a.re), warp_sum((double)a.im));
    }
    static __device__ __forceinline__ C scale(C a, float s) { return C{a.re * s, a.im * s}; }
    static __device__ __forceinline__ cx<float> to_f(C a) { return mk<float>(a.re, a.im); }
    static __device__ __forceinline__ C add(C a, C b) { return C{a.re + b.re, a.im + b.im}; }
};

template <>
struct Elem<PDF> {
    typedef float4 T;
    struct C {
        df re, im;
    };
    static __device__ __forceinline__ C load(const double2* p, long long e) {
        const float4 v = __ldg(&reinterpret_cast<const float4*>(p)[e]);
        return C{df{v.x, v.y}, df{v.z, v.w}};
    }
    static __device__ __forceinline__ C load_rw(const double2* p, long long e) {
        const float4 v = reinterpret_cast<const float4*>(p)[e];
        return C{df{v.x, v.y}, df{v.z, v.w}};
    }
    static __device__ __forceinline__ void store(double2* p, long long e, C v) {
        const df a = df_norm(v.re), b = df_norm(v.im);
        reinterpret_cast<float4*>(p)[e] = make_float4(a.hi, a.lo, b.hi, b.lo);
    }
    static __device__ __forceinline__ C zero() { return C{df{0.f, 0.f}, df{0.f, 0.f}}; }
    static __device__ __forceinline__ void mac_conj(C& acc, C a, C b) {
        df_mac(acc.re, a.re, b.re);
        df_mac(acc.re, a.im, b.im);
        df_mac(acc.im, a.re, b.im);
        df_mac(acc.im, df_neg(a.im), b.re);
    }
    static __device__ __forceinline__ void mac(C& acc, C h, C a) {
        df_mac(acc.re, h.re, a.re);
        df_mac(acc.re, df_neg(h.im), a.im);
        df_mac(acc.im, h.re, a.im);
        df_mac(acc.im, h.im, a.re);
    }
    typedef df N;
    static __device__ __forceinline__ N nzero() { return df{0.f, 0.f}; }
    static __device__ __forceinline__ void norm2_acc(N& s, C a) {
        df_mac(s, a.re, a.re);
        df_mac(s, a.im, a.im);
    }
    static __device__ __forceinline__ double nfin(N s) { return df_to_double(df_norm(s)); }
    static __device__ __forceinline__ C fin(C a) { return C{df_norm(a.re), df_norm(a.im)}; }
    static __device__ __forceinline__ double2 to_d2(C a) { return make_double2(df_to_double(a.re), df_to_double(a.im)); }
    static __device__ __forceinline__ C from_d2(double2 a) { return C{df_from_double(a.x), df_from_double(a.y)}; }
    static __device__ __forceinline__ C warp_reduce(C a) { return C{df_warp_sum(df_norm(a.re)), df_warp_sum(df_norm(a.im))}; }
    static __device__ __forceinline__ C scale(C a, df s) { return C{df_mul(a.re, s), df_mul(a.im, s)}; }
    static __device__ __forceinline__ cx<float> to_f(C a) { return mk<float>(a.re.hi + a.re.lo, a.im.hi + a.im.lo); }
    static __device__ __forceinline__ C add(C a, C b) { return C{df_add(a.re, b.re), df_add(a.im, b.im)}; }
};

// ---- multi-dot: partial[r][blk][i] = <V_i, w> (i < nv), [nvmax] = ||w||^2 ---
// The CTAs of one group of 8 basis vectors split the elements between them
// (grid stride). Each thread streams its elements of w and of the 8 V_i
// through a private ring of kDotStages shared-memory slots with cp.async, so
// the loads of the next kDotStages - 1 elements are in flight while the
// current one is multiplied: the memory pipeline stays full without holding
// the in-flight data in registers. A thread reads back only the slots it
// filled itself, so no barrier is needed. Every V_i element is read once,
// coalesced; the warp reductions happen once per CTA at the end.
constexpr int kDotG = 8;       // basis vectors per CTA
constexpr int kDotStages = 3;  // elements in flight per thread

template <int VP>
constexpr size_t multidot_smem() {
    return (size_t)kDotStages * (kDotG + 1) * kT * sizeof(typename Elem<VP>::T);
}

// The last CTA of a launch (per rhs) to finish sums the partial rows:
// fin[i] = sum_b part[b][i], each row lane-strided over b and then a fixed
// shuffle tree, the order of the separate finalize kernel (so the result does
// not depend on which CTA is last). Every CTA fences its partial writes and
// counts itself in; the last one reads the rows through L2 and resets the
// counter for the next launch on the stream.
__device__ __forceinline__ void last_cta_sum(const double2* part, int nrow, int NP, unsigned* cnt, double2* fin) {
    __shared__ unsigned is_last;
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) is_last = (atomicAdd(cnt, 1u) == gridDim.x - 1);
    __syncthreads();
    if (!is_last) return;
    __threadfence();
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    for (int i = warp; i < NP; i += nw) {
        double2 s = make_double2(0.0, 0.0);
        for (int b = lane; b < nrow; b += 32) {
            const double2 t = __ldcg(part + (long long)b * NP + i);
            s.x += t.x;
            s.y += t.y;
        }
        s.x = warp_sum(s.x);
        s.y = warp_sum(s.y);
        if (lane == 0) fin[i] = s;
    }
    if (threadIdx.x == 0) *cnt = 0u;
}

// partial[r][slot][i] over the elements this CTA sweeps, for its group of at
// most 8 vectors (the nv vectors of a rhs are spread evenly over the ngroups
// groups, so that the CTAs of all groups stream about the same bytes); the
// CTAs of group 0 also write ||w||^2 and zero the unused slots.
template <int VP>
__global__ void __launch_bounds__(kT, 2) multidot_kernel(VecRef Vb, VecRef w, long long n, const int* jtab,
                                                         int nv_off, int nvmax, int ngroups, double2* partial,
                                                         unsigned* cnt, double2* fin) {
    typedef Elem<VP> E;
    typedef typename E::C C;
    typedef typename E::T TW;  // storage word of one complex element
    extern __shared__ __align__(16) unsigned char dsm[];
    TW* ring = reinterpret_cast<TW*>(dsm);  // [kDotStages][kDotG + 1][kT]
    __shared__ double2 red[kDotG][kT / 32];
    __shared__ double redn[kT / 32];
    const int r = blockIdx.y;
    if (jtab && jtab[r] < 0) return;
    const int nv = rhs_nv(jtab, r, nv_off);
    const int j = jtab ? jtab[r] : 0;
    const int grp = blockIdx.x % ngroups;
    const int slot = blockIdx.x / ngroups;  // partial slot of this CTA
    const int nslots = gridDim.x / ngroups;
    const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
    const int gb = nv / ngroups, gr = nv % ngroups;  // nv <= ngroups * kDotG
    const int G = gb + (grp < gr ? 1 : 0);           // vectors of this CTA
    const int i0 = grp * gb + min(grp, gr);
    const TW* Vr = reinterpret_cast<const TW*>(Vb.base + r * Vb.rhs_stride +
                                               (long long)(Vb.col_off + i0) * Vb.col_stride);
    const long long cs = Vb.col_stride * (long long)(16 / sizeof(TW));  // column stride in words
    const TW* wr = reinterpret_cast<const TW*>(w.base + r * w.rhs_stride + (long long)(j + w.col_off) * w.col_stride);
    C acc[kDotG];
#pragma unroll
    for (int q = 0; q < kDotG; ++q) acc[q] = E::zero();
    typename E::N wacc = E::nzero();
    const long long stride = (long long)nslots * kT;
    auto issue = [&](long long e, int stage) {
        if (e < n) {
            TW* sl = ring + (size_t)stage * (kDotG + 1) * kT + t;
            cp_async_word(sl + kDotG * kT, wr + e);
#pragma unroll
            for (int q = 0; q < kDotG; ++q)
                if (q < G) cp_async_word(sl + q * kT, Vr + q * cs + e);
        }
        cp_async_commit();  // one group per element slot, empty past the end
    };
    long long e_next = (long long)slot * kT + t;
#pragma unroll
    for (int sg = 0; sg < kDotStages - 1; ++sg) {
        issue(e_next, sg);
        e_next += stride;
    }
    int sc = 0, si = kDotStages - 1;
    for (long long e = (long long)slot * kT + t; e < n; e += stride) {
        issue(e_next, si);
        e_next += stride;
        si = (si + 1 == kDotStages) ? 0 : si + 1;
        cp_async_wait_pending<kDotStages - 1>();  // the slot of element e has landed
        const TW* sl = ring + (size_t)sc * (kDotG + 1) * kT + t;
        const C wv = E::load_rw(reinterpret_cast<const double2*>(sl + kDotG * kT), 0);
        if (grp == 0) E::norm2_acc(wacc, wv);
#pragma unroll
        for (int q = 0; q < kDotG; ++q)
            if (q < G) E::mac_conj(acc[q], E::load_rw(reinterpret_cast<const double2*>(sl + q * kT), 0), wv);
        sc = (sc + 1 == kDotStages) ? 0 : sc + 1;
    }
    cp_async_wait_pending<0>();
    // CTA reduction of the G dot products (warp shuffles, then across warps)
#pragma unroll
    for (int q = 0; q < kDotG; ++q)
        if (q < G) {
            double2 sq;
            if constexpr (VP == P32)
                sq = E::warp_reduce_d(acc[q]);
            else
                sq = E::to_d2(E::warp_reduce(acc[q]));
            if (lane == 0) red[q][warp] = sq;
        }
    const double wn = (grp == 0) ? warp_sum(E::nfin(wacc)) : 0.0;
    if (lane == 0) redn[warp] = wn;
    __syncthreads();
    const int NP = nvmax + 1;
    double2* out = partial + ((long long)r * nslots + slot) * NP;
    if (t < G) {
        double2 sum = make_double2(0.0, 0.0);
        for (int q = 0; q < kT / 32; ++q) sum.x += red[t][q].x, sum.y += red[t][q].y;
        out[i0 + t] = sum;
    }
    if (grp == 0) {
        if (t == 0) {
            double sum = 0.0;
            for (int q = 0; q < kT / 32; ++q) sum += redn[q];
            out[nvmax] = make_double2(sum, 0.0);
        }
        for (int i = nv + t; i < nvmax; i += kT) out[i] = make_double2(0.0, 0.0);  // the groups cover [0, nv)
    }
    if (cnt) last_cta_sum(partial + (long long)r * nslots * NP, nslots, NP, cnt + r, fin + (long long)r * NP);
}

// out[r][i] = sum_blk partial[r][blk][i]: warp i sums its row lane-strided,
// then a fixed shuffle tree (deterministic)
__global__ void __launch_bounds__(1024) finalize_kernel(const double2* partial, int nblk, int NP, const int* jtab,
                                                        double2* out) {
    const int r = blockIdx.x;
    if (jtab && jtab[r] < 0) return;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int i = warp; i < NP; i += 32) {
        double2 s = make_double2(0.0, 0.0);
        const double2* p = partial + (long long)r * nblk * NP + i;
        for (int b = lane; b < nblk; b += 32) {
            const double2 t = p[(long long)b * NP];
            s.x += t.x;
            s.y += t.y;
        }
        s.x = warp_sum(s.x);
        s.y = warp_sum(s.y);
        if (lane == 0) out[(long long)r * NP + i] = s;
    }
}

__global__ void __launch_bounds__(32) finalize_real_kernel(const double2* partial, int nblk, const int* jtab,
                                                           double* out) {
    const int r = blockIdx.x;
    if (jtab && jtab[r] < 0) return;
    double s = 0.0;
    for (int b = threadIdx.x; b < nblk; b += 32) s += partial[(long long)r * nblk + b].x;
    s = warp_sum(s);
    if (threadIdx.x == 0) out[r] = s;
}

// ---- w -= sum_i coef[r][i] V_i ; partial ||w||^2 ------------------------------
template <int VP>
__global__ void __launch_bounds__(kT) multiaxpy_kernel(VecRef Vb, VecRef w, long long n, const int* jtab, int nv_off,
                                                       const double2* coef, int coef_ld, double2* partial,
                                                       unsigned* cnt, double* fin) {
    typedef Elem<VP> E;
    typedef typename E::C C;
    __shared__ C h[kMaxV];
    __shared__ double red[kT / 32];
    const int r = blockIdx.y;
    if (jtab && jtab[r] < 0) return;
    const int nv = rhs_nv(jtab, r, nv_off);
    const int j = jtab ? jtab[r] : 0;
    for (int i = threadIdx.x; i < nv; i += kT) {
        const double2 c = coef[(long long)r * coef_ld + i];
        h[i] = E::from_d2(make_double2(-c.x, -c.y));
    }
    __syncthreads();
    const double2* Vr = Vb.base + r * Vb.rhs_stride;
    double2* wr = w.base + r * w.rhs_stride + (long long)(j + w.col_off) * w.col_stride;
    const long long stride = (long long)gridDim.x * kT;
    typename E::N wacc = E::nzero();
    for (long long e = (long long)blockIdx.x * kT + threadIdx.x; e < n; e += stride) {
        C acc = E::load_rw(wr, e);
        for (int i = 0; i < nv; ++i) E::mac(acc, h[i], E::load(Vr + (long long)(i + Vb.col_off) * Vb.col_stride, e));
        acc = E::fin(acc);
        E::store(wr, e, acc);
        E::norm2_acc(wacc, acc);
    }
    const double wn = warp_sum(E::nfin(wacc));
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = wn;
    __syncthreads();
    if (threadIdx.x == 0) {
        double s = 0.0;
        for (int q = 0; q < kT / 32; ++q) s += red[q];
        partial[(long long)r * gridDim.x + blockIdx.x] = make_double2(s, 0.0);
    }
    if (cnt) {  // the last CTA sums the partial norms in the finalize kernel's order
        __shared__ unsigned is_last;
        __threadfence();
        __syncthreads();
        if (threadIdx.x == 0) is_last = (atomicAdd(cnt + r, 1u) == gridDim.x - 1);
        __syncthreads();
        if (!is_last || threadIdx.x >= 32) return;
        __threadfence();
        double s = 0.0;
        for (int b = threadIdx.x; b < (int)gridDim.x; b += 32) s += __ldcg(&partial[(long long)r * gridDim.x + b].x);
        s = warp_sum(s);
        if (threadIdx.x == 0) {
            fin[r] = s;
            cnt[r] = 0u;
        }
    }
}

// The FP32-basis form of the multi-axpy: two complex numbers per thread and
// vector (one 16-byte load instead of two 8-byte ones), so each thread keeps
// twice the bytes in flight through its chain of multiply-adds; same
// arithmetic per complex number as multiaxpy_kernel<P32>. n is even (12 per site).
__global__ void __launch_bounds__(kT) multiaxpy_f32x2_kernel(VecRef Vb, VecRef w, long long n, const int* jtab,
                                                            int nv_off, const double2* coef, int coef_ld,
                                                            double2* partial, unsigned* cnt, double* fin) {
    __shared__ float2 h[kMaxV];
    __shared__ double red[kT / 32];
    const int r = blockIdx.y;
    if (jtab && jtab[r] < 0) return;
    const int nv = rhs_nv(jtab, r, nv_off);
    const int j = jtab ? jtab[r] : 0;
    for (int i = threadIdx.x; i < nv; i += kT) {
        const double2 c = coef[(long long)r * coef_ld + i];
        h[i] = make_float2((float)-c.x, (float)-c.y);
    }
    __syncthreads();
    const float4* Vr = reinterpret_cast<const float4*>(Vb.base + r * Vb.rhs_stride);
    float4* wr = reinterpret_cast<float4*>(w.base + r * w.rhs_stride + (long long)(j + w.col_off) * w.col_stride);
    const long long cs = Vb.col_stride;  // 16-byte units = float4 elements
    const long long stride = (long long)gridDim.x * kT;
    const long long n2 = n / 2;
    float wacc = 0.f;
    for (long long e = (long long)blockIdx.x * kT + threadIdx.x; e < n2; e += stride) {
        float4 acc = wr[e];
        for (int i = 0; i < nv; ++i) {
            const float2 hi = h[i];
            const float4 a = __ldg(&Vr[(long long)(i + Vb.col_off) * cs + e]);
            acc.x = fmaf(hi.x, a.x, acc.x);
            acc.x = fmaf(-hi.y, a.y, acc.x);
            acc.y = fmaf(hi.x, a.y, acc.y);
            acc.y = fmaf(hi.y, a.x, acc.y);
            acc.z = fmaf(hi.x, a.z, acc.z);
            acc.z = fmaf(-hi.y, a.w, acc.z);
            acc.w = fmaf(hi.x, a.w, acc.w);
            acc.w = fmaf(hi.y, a.z, acc.w);
        }
        wr[e] = acc;
        wacc = fmaf(acc.x, acc.x, fmaf(acc.y, acc.y, wacc));
        wacc = fmaf(acc.z, acc.z, fmaf(acc.w, acc.w, wacc));
    }
    const double wn = warp_sum((double)wacc);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = wn;
    __syncthreads();
    if (threadIdx.x == 0) {
        double s = 0.0;
        for (int q = 0; q < kT / 32; ++q) s += red[q];
        partial[(long long)r * gridDim.x + blockIdx.x] = make_double2(s, 0.0);
    }
    if (cnt) {  // the last CTA sums the partial norms in the finalize kernel's order
        __shared__ unsigned is_last;
        __threadfence();
        __syncthreads();
        if (threadIdx.x == 0) is_last = (atomicAdd(cnt + r, 1u) == gridDim.x - 1);
        __syncthreads();
        if (!is_last || threadIdx.x >= 32) return;
        __threadfence();
        double s = 0.0;
        for (int b = threadIdx.x; b < (int)gridDim.x; b += 32) s += __ldcg(&partial[(long long)r * gridDim.x + b].x);
        s = warp_sum(s);
        if (threadIdx.x == 0) {
            fin[r] = s;
            cnt[r] = 0u;
        }
    }
}

// ---- v = w / ||w|| per site, optionally also written in SAP storage ----------
template <int VP, int PS>
__global__ void __launch_bounds__(kT) normalize_kernel(VecRef w, VecRef dst, long long V, const int* jtab,
                                                       const double* norm2, FieldRef low) {
    typedef Elem<VP> E;
    typedef typename E::C C;
    typedef typename real_of<(PS == P64) ? P64 : P32>::type CL;  // precision of the SAP copy
    const int r = blockIdx.y;
    if (jtab && jtab[r] < 0) return;
    // 1/||w|| once per CTA: FP64 square root and division are long
    // instruction sequences on the narrow FP64 pipes
    __shared__ double inv_sh;
    if (threadIdx.x == 0) {
        const double nn = norm2[r];
        inv_sh = nn > 0.0 ? 1.0 / sqrt(nn) : 0.0;
    }
    __syncthreads();
    const double inv = inv_sh;
    const long long s = (long long)blockIdx.x * kT + threadIdx.x;
    if (s >= V) return;
    const int j = jtab ? jtab[r] : 0;
    const double2* src = w.base + r * w.rhs_stride + (long long)(j + w.col_off) * w.col_stride;
    double2* out = dst.base + r * dst.rhs_stride + (long long)(j + dst.col_off) * dst.col_stride;
    cx<CL> f[12];
    if constexpr (VP == P32) {  // S32 spinor layout, scaled in FP32
        cx<float> q[12];
        load_spinor<P32, float, true>(reinterpret_cast<const char*>(src), V, s, q);
        const float fi = (float)inv;
#pragma unroll
        for (int c = 0; c < 12; ++c) q[c] = mk<float>(q[c].re * fi, q[c].im * fi);
        store_spinor<P32, float>(reinterpret_cast<char*>(out), V, s, q);
#pragma unroll
        for (int c = 0; c < 12; ++c) f[c] = mk<CL>((CL)q[c].re, (CL)q[c].im);
        if constexpr (PS >= 0) store_spinor<PS, CL>(field_ptr(low, jtab, r), V, s, f);
        return;
    }
#pragma unroll
    for (int c = 0; c < 12; ++c) {
        C v;
        if constexpr (VP == PDF)
            v = E::scale(E::load_rw(src, c * V + s), df_from_double(inv));
        else if constexpr (VP == P64)
            v = E::scale(E::load_rw(src, c * V + s), inv);
        E::store(out, c * V + s, v);
        const double2 d = E::to_d2(v);
        if constexpr (sizeof(CL) == 8)
            f[c] = mk<CL>(d.x, d.y);
        else
            f[c] = E::to_f(v);
    }
    if constexpr (PS >= 0) store_spinor<PS, CL>(field_ptr(low, jtab, r), V, s, f);
}

template <int VP>
__global__ void __launch_bounds__(kT) scale_kernel(const double2* src, double2* dst, long long rs, long long n,
                                                   const double* a) {
    typedef Elem<VP> E;
    const int r = blockIdx.y;
    for (long long e = (long long)blockIdx.x * kT + threadIdx.x; e < n; e += (long long)gridDim.x * kT) {
        if constexpr (VP == PDF)
            E::store(dst + r * rs, e, E::scale(E::load_rw(src + r * rs, e), df_from_double(a[r])));
        else
            E::store(dst + r * rs, e, E::scale(E::load_rw(src + r * rs, e), a[r]));
    }
}

// ---- in-place rotation of flat columns: X_c = sum_i X_i Q[i][c] (c < kout) ----
// KMAX: the accumulators held per thread (kout <= KMAX); instantiated for a
// few sizes so that a small deflation space does not pay the registers (and
// the occupancy) of the largest
template <int VP, int KMAX>
__global__ void __launch_bounds__(kT) rotate_outer_kernel(double2* X, long long rs, long long cs, long long n,
                                                          const int* active, int nin, int kout, const double2* Q,
                                                          int qld) {
    typedef Elem<VP> E;
    typedef typename E::C C;
    extern __shared__ __align__(16) unsigned char qsm[];
    C* q = reinterpret_cast<C*>(qsm);  // [nin][kout]
    const int r = blockIdx.y;
    if (active && !active[r]) return;
    const double2* Qr = Q + (long long)r * qld * qld;
    for (int t = threadIdx.x; t < nin * kout; t += kT) q[t] = E::from_d2(Qr[(long long)(t / kout) * qld + t % kout]);
    __syncthreads();
    double2* Xr = X + r * rs;
    for (long long e = (long long)blockIdx.x * kT + threadIdx.x; e < n; e += (long long)gridDim.x * kT) {
        C acc[KMAX];
#pragma unroll
        for (int c = 0; c < KMAX; ++c) acc[c] = E::zero();
        for (int i = 0; i < nin; ++i) {
            const C v = E::load_rw(Xr + (long long)i * cs, e);
#pragma unroll
            for (int c = 0; c < KMAX; ++c)
                if (c < kout) E::mac(acc[c], q[i * kout + c], v);
        }
#pragma unroll
        for (int c = 0; c < KMAX; ++c)
            if (c < kout) E::store(Xr + (long long)c * cs, e, E::fin(acc[c]));
    }
}

// FP32 storage (flat float2 view): X_c = sum_i X_i Q[i][c], in place; KMAX
// is the largest kout of the instantiation (it sizes the accumulators); the
// loads of four inputs are issued together
template <int KMAX>
__global__ void __launch_bounds__(kT) rotate_f32_kernel(float2* X, long long rs, long long cs, long long n,
                                                        const int* active, int nin, int kout, const double2* Q,
                                                        int qld) {
    extern __shared__ __align__(16) unsigned char qsm[];
    float2* q = reinterpret_cast<float2*>(qsm);
    const int r = blockIdx.y;
    if (active && !active[r]) return;
    const double2* Qr = Q + (long long)r * qld * qld;
    for (int t = threadIdx.x; t < nin * kout; t += kT) {
        const double2 v = Qr[(long long)(t / kout) * qld + t % kout];
        q[t] = make_float2((float)v.x, (float)v.y);
    }
    __syncthreads();
    float2* Xr = X + r * rs;
    for (long long e = (long long)blockIdx.x * kT + threadIdx.x; e < n; e += (long long)gridDim.x * kT) {
        float ar[KMAX], ai[KMAX];
#pragma unroll
        for (int c = 0; c < KMAX; ++c) ar[c] = ai[c] = 0.f;
#pragma unroll 4
        for (int i = 0; i < nin; ++i) {
            const float2 v = Xr[(long long)i * cs + e];
#pragma unroll
            for (int c = 0; c < KMAX; ++c)
                if (c < kout) {
                    const float2 qq = q[i * kout + c];
                    ar[c] = fmaf(qq.x, v.x, fmaf(-qq.y, v.y, ar[c]));
                    ai[c] = fmaf(qq.x, v.y, fmaf(qq.y, v.x, ai[c]));
                }
        }
#pragma unroll
        for (int c = 0; c < KMAX; ++c)
            if (c < kout) Xr[(long long)c * cs + e] = make_float2(ar[c], ai[c]);
    }
}

// Out-of-place rotation for per-site-scaled storage: one thread per site,
// one output column at a time (Y_c = sum_i X_i Q[i][c]).
template <int P>
__global__ void __launch_bounds__(kT) rotate_site_kernel(const char* X, char* Y, long long rs, long long cs,
                                                         long long yrs, long long V, const int* active, int nin,
                                                         int kout, const double2* Q, int qld) {
    extern __shared__ __align__(16) unsigned char qsm[];
    float2* q = reinterpret_cast<float2*>(qsm);
    const int r = blockIdx.y;
    if (active && !active[r]) return;
    const double2* Qr = Q + (long long)r * qld * qld;
    for (int t = threadIdx.x; t < nin * kout; t += kT) {
        const double2 v = Qr[(long long)(t / kout) * qld + t % kout];
        q[t] = make_float2((float)v.x, (float)v.y);
    }
    __syncthreads();
    const long long s = (long long)blockIdx.x * kT + threadIdx.x;
    if (s >= V) return;
    for (int c = 0; c < kout; ++c) {
        cx<float> acc[12];
#pragma unroll
        for (int a = 0; a < 12; ++a) acc[a] = czero<float>();
        for (int i = 0; i < nin; ++i) {
            cx<float> v[12];
            load_spinor<P, float>(X + r * rs + i * cs, V, s, v);
            const cx<float> qf = mk<float>(q[i * kout + c].x, q[i * kout + c].y);
#pragma unroll
            for (int a = 0; a < 12; ++a) acc[a] = acc[a] + qf * v[a];
        }
        store_spinor<P, float>(Y + r * yrs + c * cs, V, s, acc);
    }
}

// FP32 Z (float4 [6][V], two complex components per word): one thread per
// word u = q V + s, i.e. components 2q and 2q + 1 of site s, which are x
// elements (2q) V + s and (2q + 1) V + s; grid stride; the loads of four Z_i
// are issued together
template <int VX>
__global__ void __launch_bounds__(kT) xupdate_f32_kernel(const float4* Z, long long z_rs, long long z_cs, double2* x,
                                                         long long x_rs, long long V, const int* nz,
                                                         const double2* eta, int eta_ld) {
    typedef Elem<VX> E;
    typedef typename E::C C;
    __shared__ C et[kMaxV];
    const int r = blockIdx.y;
    const int nv = nz[r];
    if (nv <= 0) return;
    for (int i = threadIdx.x; i < nv; i += kT) et[i] = E::from_d2(eta[(long long)r * eta_ld + i]);
    __syncthreads();
    const float4* Zr = Z + r * z_rs;
    double2* xr = x + r * x_rs;
    const unsigned Vu = (unsigned)V;  // 6 V < 2^31 (contexts hold fewer than 2^31 / 24 sites)
    for (long long u = (long long)blockIdx.x * kT + threadIdx.x; u < 6 * V; u += (long long)gridDim.x * kT) {
        const unsigned q = (unsigned)u / Vu;
        const long long e0 = u + (long long)q * V;  // x element of component 2q
        C a0 = E::load_rw(xr, e0), a1 = E::load_rw(xr, e0 + V);
#pragma unroll 4
        for (int i = 0; i < nv; ++i) {
            const float4 v = __ldg(&Zr[(long long)i * z_cs + u]);
            const C h = et[i];
            if constexpr (VX == PDF) {
                df_mac_f(a0.re, h.re, v.x);
                df_mac_f(a0.re, df_neg(h.im), v.y);
                df_mac_f(a0.im, h.re, v.y);
                df_mac_f(a0.im, h.im, v.x);
                df_mac_f(a1.re, h.re, v.z);
                df_mac_f(a1.re, df_neg(h.im), v.w);
                df_mac_f(a1.im, h.re, v.w);
                df_mac_f(a1.im, h.im, v.z);
            } else {
                E::mac(a0, h, typename E::C{(double)v.x, (double)v.y});
                E::mac(a1, h, typename E::C{(double)v.z, (double)v.w});
            }
        }
        E::store(xr, e0, E::fin(a0));
        E::store(xr, e0 + V, E::fin(a1));
    }
}

// ---- x += sum_i Z_i eta_i, one thread per site --------------------------------
template <int PZ, int VX>
__global__ void __launch_bounds__(kT) xupdate_kernel(const char* Z, long long z_rs, long long z_cs, double2* x,
                                                     long long x_rs, long long V, const int* nz, const double2* eta,
                                                     int eta_ld) {
    typedef Elem<VX> E;
    typedef typename E::C C;
    __shared__ C et[kMaxV];
    const int r = blockIdx.y;
    const int n = nz[r];
    if (n <= 0) return;
    for (int i = threadIdx.x; i < n; i += kT) et[i] = E::from_d2(eta[(long long)r * eta_ld + i]);
    __syncthreads();
    const long long s = (long long)blockIdx.x * kT + threadIdx.x;
    if (s >= V) return;
    typedef typename real_of<PZ>::type CZ;
    double2* xr = x + r * x_rs;
    C acc[12];
#pragma unroll
    for (int a = 0; a < 12; ++a) acc[a] = E::load_rw(xr, a * V + s);
    for (int i = 0; i < n; ++i) {
        cx<CZ> v[12];
        load_spinor<PZ, CZ>(Z + r * z_rs + i * z_cs, V, s, v);
        const C h = et[i];
#pragma unroll
        for (int a = 0; a < 12; ++a) {
            if constexpr (VX == PDF && sizeof(CZ) == 4) {
                df_mac_f(acc[a].re, h.re, v[a].re);
                df_mac_f(acc[a].re, df_neg(h.im), v[a].im);
                df_mac_f(acc[a].im, h.re, v[a].im);
                df_mac_f(acc[a].im, h.im, v[a].re);
            } else if constexpr (VX == PDF) {  // FP64 storage of Z: split into double-float pairs
                E::mac(acc[a], h, typename E::C{df_from_double((double)v[a].re), df_from_double((double)v[a].im)});
            } else {
                E::mac(acc[a], h, typename E::C{(double)v[a].re, (double)v[a].im});
            }
        }
    }
#pragma unroll
    for (int a = 0; a < 12; ++a) E::store(xr, a * V + s, E::fin(acc[a]));
}

template <int VP>
__global__ void __launch_bounds__(kT) norm2_kernel(const double2* a, long long rs, long long n, double2* partial) {
    typedef Elem<VP> E;
    __shared__ double red[kT / 32];
    const int r = blockIdx.y;
    const double2* ar = a + r * rs;
    typename E::N acc = E::nzero();
    for (long long e = (long long)blockIdx.x * kT + threadIdx.x; e < n; e += (long long)gridDim.x * kT)
        E::norm2_acc(acc, E::load(ar, e));
    const double s = warp_sum(E::nfin(acc));
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int q = 0; q < kT / 32; ++q) t += red[q];
        partial[(long long)r * gridDim.x + blockIdx.x] = make_double2(t, 0.0);
    }
}

unsigned grid_for(long long n) {
    long long b = (n + kT - 1) / kT;
    const long long cap = 152LL * 8;
    return (unsigned)(b < cap ? (b < 1 ? 1 : b) : cap);
}

bool outer_ok(int vp) { return vp == P64 || vp == PDF; }
bool basis_ok(int vp) { return vp == P64 || vp == PDF || vp == P32; }

}  // namespace

int blas_nblk(long long n) { return (int)grid_for(n); }

int launch_multidot(int vp, VecRef Vb, VecRef w, long long n, const int* jtab, int nv_off, int nvmax, int nv_active,
                    int nrhs, double2* partial, int nblk, double2* out, cudaStream_t st, unsigned* cnt) {
    if (nvmax > kMaxV) return fail(DW_EINVAL, "too many basis vectors for one multi-dot");
    if (!basis_ok(vp)) return fail(DW_EINVAL, "bad basis precision");
    // CTAs: (element slots) x (groups of at most 8 vectors), at most one wave
    // of two CTAs per SM per right-hand side (rounded down: a CTA past the
    // wave would run alone after it); at most nblk slots
    if (nv_active < 1 || nv_active > nvmax) nv_active = nvmax;
    const int ngroups = (nv_active + kDotG - 1) / kDotG;  // groups past every rhs's nv would only read w
    // SM count per device, cached; the serving workers call this concurrently,
    // so the cache entries are atomics (every writer stores the same value)
    static std::atomic<int> sms[64];
    int dev0 = 0;
    DW_CUDA_TRY(cudaGetDevice(&dev0));
    int nsm = (dev0 < 64) ? sms[dev0].load(std::memory_order_relaxed) : 0;
    if (nsm == 0) {
        DW_CUDA_TRY(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev0));
        if (dev0 < 64) sms[dev0].store(nsm, std::memory_order_relaxed);
    }
    const long long slots = 2LL * (nsm > 0 ? nsm : 152);
    long long nb = slots / ngroups;
    if (nb > nblk) nb = nblk;
    if (nb > (n + kT - 1) / kT) nb = (n + kT - 1) / kT;
    if (nb < 1) nb = 1;
    const dim3 grid((unsigned)(nb * ngroups), nrhs);
    // the ring exceeds the 48 KB default: raise the limit once per device
    static std::mutex mu;
    static std::set<int> done;
    {
        int dev = 0;
        DW_CUDA_TRY(cudaGetDevice(&dev));
        std::lock_guard<std::mutex> lock(mu);
        if (!done.count(dev)) {
            DW_CUDA_TRY(cudaFuncSetAttribute(multidot_kernel<PDF>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)multidot_smem<PDF>()));
            DW_CUDA_TRY(cudaFuncSetAttribute(multidot_kernel<P64>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)multidot_smem<P64>()));
            DW_CUDA_TRY(cudaFuncSetAttribute(multidot_kernel<P32>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)multidot_smem<P32>()));
            done.insert(dev);
        }
    }
    if (vp == PDF)
        multidot_kernel<PDF><<<grid, kT, multidot_smem<PDF>(), st>>>(Vb, w, n, jtab, nv_off, nvmax, ngroups, partial,
                                                                    cnt, out);
    else if (vp == P32)
        multidot_kernel<P32><<<grid, kT, multidot_smem<P32>(), st>>>(Vb, w, n, jtab, nv_off, nvmax, ngroups, partial,
                                                                    cnt, out);
    else
        multidot_kernel<P64><<<grid, kT, multidot_smem<P64>(), st>>>(Vb, w, n, jtab, nv_off, nvmax, ngroups, partial,
                                                                    cnt, out);
    DW_LAUNCH_CHECK();
    if (!cnt) {  // without counters, a separate reduction launch
        finalize_kernel<<<nrhs, 1024, 0, st>>>(partial, (int)nb, nvmax + 1, jtab, out);
        DW_LAUNCH_CHECK();
    }
    return DW_OK;
}

int launch_multiaxpy(int vp, VecRef Vb, VecRef w, long long n, const int* jtab, int nv_off, int nrhs,
                     const double2* coef, int coef_ld, double2* partial, int nblk, double* out_norm2,
                     cudaStream_t st, unsigned* cnt) {
    if (!basis_ok(vp)) return fail(DW_EINVAL, "bad basis precision");
    if (vp == PDF)
        multiaxpy_kernel<PDF><<<dim3(nblk, nrhs), kT, 0, st>>>(Vb, w, n, jtab, nv_off, coef, coef_ld, partial, cnt,
                                                              out_norm2);
    else if (vp == P32 && n % 2 == 0)
        multiaxpy_f32x2_kernel<<<dim3(nblk, nrhs), kT, 0, st>>>(Vb, w, n, jtab, nv_off, coef, coef_ld, partial, cnt,
                                                                out_norm2);
    else if (vp == P32)
        multiaxpy_kernel<P32><<<dim3(nblk, nrhs), kT, 0, st>>>(Vb, w, n, jtab, nv_off, coef, coef_ld, partial, cnt,
                                                              out_norm2);
    else
        multiaxpy_kernel<P64><<<dim3(nblk, nrhs), kT, 0, st>>>(Vb, w, n, jtab, nv_off, coef, coef_ld, partial, cnt,
                                                              out_norm2);
    DW_LAUNCH_CHECK();
    if (!cnt) {
        finalize_real_kernel<<<nrhs, 32, 0, st>>>(partial, nblk, jtab, out_norm2);
        DW_LAUNCH_CHECK();
    }
    return DW_OK;
}

int launch_normalize(int vp, VecRef w, VecRef dst, long long V, const int* jtab, int nrhs, const double* norm2,
                     int plow, FieldRef low, cudaStream_t st) {
    if (!basis_ok(vp)) return fail(DW_EINVAL, "bad basis precision");
    dim3 grid((unsigned)((V + kT - 1) / kT), nrhs);
#define NORM(A, B)                                                                                      \
    if (vp == A && plow == B) {                                                                         \
        normalize_kernel<A, B><<<grid, kT, 0, st>>>(w, dst, V, jtab, norm2, low);                       \
        DW_LAUNCH_CHECK();                                                                              \
        return DW_OK;                                                                                   \
    }
    NORM(P64, -1)
    NORM(P64, P64)
    NORM(P64, P32)
    NORM(P64, P16)
    NORM(P64, PB16)
    NORM(PDF, -1)
    NORM(PDF, P64)
    NORM(PDF, P32)
    NORM(PDF, P16)
    NORM(PDF, PB16)
    NORM(P32, -1)
    NORM(P32, P32)
    NORM(P32, P16)
    NORM(P32, PB16)
#undef NORM
    return fail(DW_EINVAL, "unsupported normalisation precision combination");
}

int launch_scale(int vp, const double2* src, double2* dst, long long rs, long long n, int nrhs, const double* a,
                 cudaStream_t st) {
    if (vp == PDF)
        scale_kernel<PDF><<<dim3(grid_for(n), nrhs), kT, 0, st>>>(src, dst, rs, n, a);
    else
        scale_kernel<P64><<<dim3(grid_for(n), nrhs), kT, 0, st>>>(src, dst, rs, n, a);
    DW_LAUNCH_CHECK();
    return DW_OK;
}

int launch_rotate(int prec, char* X, long long rhs_stride, long long col_stride, long long V, int nrhs,
                  const int* active, int nin, int kout, const double2* Q, int qld, char* scratch,
                  cudaStream_t st) {
    if (kout > kRotMax && prec != P16 && prec != PB16) return fail(DW_EINVAL, "deflation dimension too large");
    const size_t qsm = (size_t)nin * kout * ((prec == PDF || prec == P64) ? 16 : 8);
    if (qsm > 48 * 1024) return fail(DW_EINVAL, "rotation matrix too large");
    const long long n = 12 * V;
    if (prec == P64 || prec == PDF) {
        double2* Xd = reinterpret_cast<double2*>(X);
        const dim3 grid(grid_for(n), nrhs);
        const long long rs = rhs_stride / 16, cs = col_stride / 16;
#define ROT(K)                                                                                              \
    if (kout <= K) {                                                                                        \
        if (prec == PDF)                                                                                    \
            rotate_outer_kernel<PDF, K><<<grid, kT, qsm, st>>>(Xd, rs, cs, n, active, nin, kout, Q, qld);   \
        else                                                                                                \
            rotate_outer_kernel<P64, K><<<grid, kT, qsm, st>>>(Xd, rs, cs, n, active, nin, kout, Q, qld);   \
        DW_LAUNCH_CHECK();                                                                                  \
        return DW_OK;                                                                                       \
    }
        ROT(6)
        ROT(11)
        ROT(kRotMax)
#undef ROT
    } else if (prec == P32) {
        const dim3 grid(grid_for(n), nrhs);
        float2* Xf = reinterpret_cast<float2*>(X);
        if (kout <= 6)
            rotate_f32_kernel<6><<<grid, kT, qsm, st>>>(Xf, rhs_stride / 8, col_stride / 8, n, active, nin, kout, Q, qld);
        else if (kout <= 11)
            rotate_f32_kernel<11><<<grid, kT, qsm, st>>>(Xf, rhs_stride / 8, col_stride / 8, n, active, nin, kout, Q,
                                                         qld);
        else
            rotate_f32_kernel<kRotMax><<<grid, kT, qsm, st>>>(Xf, rhs_stride / 8, col_stride / 8, n, active, nin, kout,
                                                              Q, qld);
    } else {
        if (!scratch) return fail(DW_EINVAL, "rotation of scaled storage needs scratch");
        const long long yrs = col_stride * kout;
        dim3 grid((unsigned)((V + kT - 1) / kT), nrhs);
        if (prec == P16)
            rotate_site_kernel<P16><<<grid, kT, qsm, st>>>(X, scratch, rhs_stride, col_stride, yrs, V, active, nin,
                                                           kout, Q, qld);
        else
            rotate_site_kernel<PB16><<<grid, kT, qsm, st>>>(X, scratch, rhs_stride, col_stride, yrs, V, active, nin,
                                                            kout, Q, qld);
        DW_LAUNCH_CHECK();
        for (int r = 0; r < nrhs; ++r)
            DW_CUDA_TRY(cudaMemcpyAsync(X + r * rhs_stride, scratch + r * yrs, (size_t)yrs,
                                        cudaMemcpyDeviceToDevice, st));
        return DW_OK;
    }
    DW_LAUNCH_CHECK();
    return DW_OK;
}

int launch_xupdate(int prec, int vx, const char* Z, long long z_rs, long long z_cs, double2* x, long long x_rs,
                   long long V, int nrhs, const int* nz, const double2* eta, int eta_ld, cudaStream_t st) {
    dim3 grid((unsigned)((V + kT - 1) / kT), nrhs);
    const long long xrs = x_rs / 16;
    if (prec == P32 && (vx == PDF || vx == P64)) {  // FP32 Z: one thread per Z word
        const dim3 eg(grid_for(6 * V), nrhs);
        const float4* Zf = reinterpret_cast<const float4*>(Z);
        if (vx == PDF)
            xupdate_f32_kernel<PDF><<<eg, kT, 0, st>>>(Zf, z_rs / 16, z_cs / 16, x, xrs, V, nz, eta, eta_ld);
        else
            xupdate_f32_kernel<P64><<<eg, kT, 0, st>>>(Zf, z_rs / 16, z_cs / 16, x, xrs, V, nz, eta, eta_ld);
        DW_LAUNCH_CHECK();
        return DW_OK;
    }
#define XUPD(A, B)                                                                                      \
    if (prec == A && vx == B) {                                                                         \
        xupdate_kernel<A, B><<<grid, kT, 0, st>>>(Z, z_rs, z_cs, x, xrs, V, nz, eta, eta_ld);           \
        DW_LAUNCH_CHECK();                                                                              \
        return DW_OK;                                                                                   \
    }
    XUPD(P64, P64)
    XUPD(P32, P64)
    XUPD(P16, P64)
    XUPD(PB16, P64)
    XUPD(P64, PDF)
    XUPD(P32, PDF)
    XUPD(P16, PDF)
    XUPD(PB16, PDF)
#undef XUPD
    return fail(DW_EINVAL, "unsupported iterate-update precision combination");
}

int launch_norm2(int vp, const double2* a, long long rs, long long n, int nrhs, double2* partial, int nblk,
                 double* out, cudaStream_t st) {
    if (vp == PDF)
        norm2_kernel<PDF><<<dim3(nblk, nrhs), kT, 0, st>>>(a, rs, n, partial);
    else
        norm2_kernel<P64><<<dim3(nblk, nrhs), kT, 0, st>>>(a, rs, n, partial);
    DW_LAUNCH_CHECK();
    finalize_real_kernel<<<nrhs, 32, 0, st>>>(partial, nblk, nullptr, out);
    DW_LAUNCH_CHECK();
    return DW_OK;
}

int launch_zero(void* p, size_t bytes, cudaStream_t st) {
    DW_CUDA_TRY(cudaMemsetAsync(p, 0, bytes, st));
    return DW_OK;
}

}  // namespace dwk
