// Device-side building blocks shared by the CUDA kernels of the library:
// complex arithmetic, storage formats of spinor and link fields, lattice
// geometry, and the spin-projected hopping term of the Wilson-Dirac operator
// (Sec. 2, Eq. "Dw").
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <type_traits>

namespace dwk {

// ---------------------------------------------------------------------------
// complex numbers
// ---------------------------------------------------------------------------
template <class R>
struct __align__(2 * sizeof(R)) cx {
    R re, im;
};

template <class R>
__device__ __forceinline__ cx<R> mk(R a, R b) {
    cx<R> z;
    z.re = a;
    z.im = b;
    return z;
}
template <class R>
__device__ __forceinline__ cx<R> operator+(cx<R> a, cx<R> b) { return mk(a.re + b.re, a.im + b.im); }
template <class R>
__device__ __forceinline__ cx<R> operator-(cx<R> a, cx<R> b) { return mk(a.re - b.re, a.im - b.im); }
template <class R>
__device__ __forceinline__ cx<R> operator*(cx<R> a, cx<R> b) {
    return mk(a.re * b.re - a.im * b.im, a.re * b.im + a.im * b.re);
}
template <class R>
__device__ __forceinline__ cx<R> operator*(R s, cx<R> a) { return mk(s * a.re, s * a.im); }
// conj(a) * b
template <class R>
__device__ __forceinline__ cx<R> cmulc(cx<R> a, cx<R> b) {
    return mk(a.re * b.re + a.im * b.im, a.re * b.im - a.im * b.re);
}
template <class R>
__device__ __forceinline__ cx<R> conj(cx<R> a) { return mk(a.re, -a.im); }
// i * a and -i * a
template <class R>
__device__ __forceinline__ cx<R> ti(cx<R> a) { return mk(-a.im, a.re); }
template <class R>
__device__ __forceinline__ cx<R> tmi(cx<R> a) { return mk(a.im, -a.re); }
template <class R>
__device__ __forceinline__ cx<R> czero() { return mk<R>(R(0), R(0)); }

// ---------------------------------------------------------------------------
// lattice geometry
// ---------------------------------------------------------------------------
struct Geom {
    int d[4];      // lattice extents d1..d4 (site index n1 + d1*(n2 + d2*(n3 + d3*n4)))
    int b[4];      // domain block extents
    int nb[4];     // domains per direction
    long long V;   // number of sites
    int B;         // sites per domain
    int ndom;      // number of domains
};

// 32-bit arithmetic: contexts are limited to fewer than 2^31 / 24 sites
__device__ __forceinline__ void site_coords(const Geom& g, long long s, int x[4]) {
    unsigned t = (unsigned)s;
    const unsigned d0 = (unsigned)g.d[0], d1 = (unsigned)g.d[1], d2 = (unsigned)g.d[2];
    unsigned q = t / d0;
    x[0] = (int)(t - q * d0);
    t = q;
    q = t / d1;
    x[1] = (int)(t - q * d1);
    t = q;
    q = t / d2;
    x[2] = (int)(t - q * d2);
    x[3] = (int)q;
}

__device__ __forceinline__ long long site_index(const Geom& g, const int x[4]) {
    return x[0] + (long long)g.d[0] * (x[1] + (long long)g.d[1] * (x[2] + (long long)g.d[2] * x[3]));
}

// neighbour of site s (coords x) in direction mu, sign +1/-1, periodic
__device__ __forceinline__ long long neighbour(const Geom& g, long long s, const int x[4], int mu, int sign) {
    long long stride = 1;
    for (int j = 0; j < mu; ++j) stride *= g.d[j];
    if (sign > 0) return (x[mu] == g.d[mu] - 1) ? s - (long long)(g.d[mu] - 1) * stride : s + stride;
    return (x[mu] == 0) ? s + (long long)(g.d[mu] - 1) * stride : s - stride;
}

// ---------------------------------------------------------------------------
// storage formats
//
// spinor fields, component-major with the site index fastest:
//   S64 : double2 [12][V]                       192 B/site
//   S32 : float4  [6][V]  (two complex each)     96 B/site
//   S16 : uint4   [3][V]  (eight halves each) + float scale[V]   52 B/site
//   SB16: as S16 with bfloat16                                   52 B/site
// For S16/SB16 each site stores psi/s with s = max |real component| of the
// site (s = 1 for a zero site), so every stored value lies in [-1, 1].
//
// link fields U[mu][row][col], component-major with the site index fastest:
//   L64: double2 [4][9][V], L32: float2, L16: half2, LB16: bfloat162
// ---------------------------------------------------------------------------
//   SDF : float4  [12][V]  (re_hi, re_lo, im_hi, im_lo): a double-float pair
//         per real, value = hi + lo with |lo| <= ulp(hi)/2 (48-bit significand),
//         192 B/site like S64; its arithmetic runs on the FP32 pipes
enum Prec { P64 = 0, P32 = 1, P16 = 2, PB16 = 3, PDF = 4 };

__host__ __device__ inline long long spinor_bytes(int prec, long long V) {
    return (prec == P64 || prec == PDF) ? 192 * V : prec == P32 ? 96 * V : 52 * V;
}
__host__ __device__ inline long long link_bytes(int prec, long long V) {
    return (prec == P64 || prec == PDF) ? 576 * V : prec == P32 ? 288 * V : 144 * V;
}

// ---------------------------------------------------------------------------
// double-float arithmetic (Dekker 1971 splitting/products, Knuth's TwoSum;
// products use the FMA form of the exact product error): a value is the
// unevaluated sum hi + lo of two FP32 numbers.
// ---------------------------------------------------------------------------
struct df {
    float hi, lo;
    df() = default;
    __host__ __device__ constexpr df(float h, float l) : hi(h), lo(l) {}
    __host__ __device__ explicit df(int v) : hi((float)v), lo(0.f) {}
    __host__ __device__ explicit df(float v) : hi(v), lo(0.f) {}
    __host__ __device__ explicit df(double v) : hi((float)v), lo((float)(v - (double)(float)v)) {}
};
__device__ __forceinline__ df two_sum(float a, float b) {
    const float s = a + b;
    const float bb = s - a;
    const float e = (a - (s - bb)) + (b - bb);
    return df{s, e};
}
__device__ __forceinline__ df quick_two_sum(float a, float b) {  // requires |a| >= |b| or a == 0
    const float s = a + b;
    return df{s, b - (s - a)};
}
__device__ __forceinline__ df df_norm(df a) { return two_sum(a.hi, a.lo); }
__device__ __forceinline__ df df_add(df a, df b) {
    df s = two_sum(a.hi, b.hi);
    s.lo += a.lo + b.lo;
    return quick_two_sum(s.hi, s.lo);
}
// The products that feed an error-free sum are rounded on their own
// (__fmul_rn): a plain product could be contracted with the following
// addition into one FMA, and the TwoSum after it would no longer be exact.
__device__ __forceinline__ float mul_rn(float a, float b) {
#ifdef __CUDA_ARCH__
    return __fmul_rn(a, b);
#else
    return a * b;
#endif
}
__device__ __forceinline__ df df_mul(df a, df b) {
    const float p = mul_rn(a.hi, b.hi);
    float e = fmaf(a.hi, b.hi, -p);
    e = fmaf(a.hi, b.lo, e);
    e = fmaf(a.lo, b.hi, e);
    return quick_two_sum(p, e);
}
__device__ __forceinline__ df df_neg(df a) { return df{-a.hi, -a.lo}; }
// acc += a * b with a lazily normalised accumulator (acc.lo collects the
// rounding errors; call df_norm before use)
__device__ __forceinline__ void df_mac(df& acc, df a, df b) {
    const float p = mul_rn(a.hi, b.hi);
    float e = fmaf(a.hi, b.hi, -p);
    e = fmaf(a.hi, b.lo, e);
    e = fmaf(a.lo, b.hi, e);
    const df s = two_sum(acc.hi, p);
    acc.hi = s.hi;
    acc.lo += s.lo + e;
}
// acc += a * b with b a plain FP32 number
__device__ __forceinline__ void df_mac_f(df& acc, df a, float b) {
    const float p = mul_rn(a.hi, b);
    float e = fmaf(a.hi, b, -p);
    e = fmaf(a.lo, b, e);
    const df s = two_sum(acc.hi, p);
    acc.hi = s.hi;
    acc.lo += s.lo + e;
}
__device__ __forceinline__ df df_from_double(double x) {
    const float hi = (float)x;
    return df{hi, (float)(x - (double)hi)};
}
__device__ __forceinline__ double df_to_double(df a) { return (double)a.hi + (double)a.lo; }
// arithmetic operators, so that the stencil templates run in double-float
__device__ __forceinline__ df operator+(df a, df b) { return df_add(a, b); }
__device__ __forceinline__ df operator-(df a) { return df_neg(a); }
__device__ __forceinline__ df operator-(df a, df b) { return df_add(a, df_neg(b)); }
__device__ __forceinline__ df operator*(df a, df b) { return df_mul(a, b); }

#ifdef __CUDACC__
// asynchronous global -> shared copy of one 4/8/16-byte word (cp.async)
template <class W>
__device__ __forceinline__ void cp_async_word(W* smem_dst, const W* gsrc) {
    static_assert(sizeof(W) == 4 || sizeof(W) == 8 || sizeof(W) == 16, "cp.async word size");
    const unsigned sa = (unsigned)__cvta_generic_to_shared(smem_dst);
    if constexpr (sizeof(W) == 16)
        asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(sa), "l"(gsrc) : "memory");
    else
        asm volatile("cp.async.ca.shared.global [%0], [%1], %2;\n" ::"r"(sa), "l"(gsrc), "n"(sizeof(W)) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
// wait until at most N of this thread's committed groups are still in flight
template <int N>
__device__ __forceinline__ void cp_async_wait_pending() {
    asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory");
}
__device__ __forceinline__ void cp_async_wait() {
    cp_async_commit();
    cp_async_wait_pending<0>();
}

// warp-wide sum of a double-float value (every lane gets the sum)
__device__ __forceinline__ df df_warp_sum(df a) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        df b;
        b.hi = __shfl_xor_sync(0xffffffffu, a.hi, o);
        b.lo = __shfl_xor_sync(0xffffffffu, a.lo, o);
        a = df_add(a, b);
    }
    return a;
}
#endif

template <int P>
struct real_of {
    typedef float type;
};
template <>
struct real_of<P64> {
    typedef double type;
};
template <>
struct real_of<PDF> {
    typedef double type;
};

__device__ __forceinline__ float2 h2_to_f2(uint32_t u, int bf) {
    if (bf) {
        __nv_bfloat162 h = *reinterpret_cast<__nv_bfloat162*>(&u);
        return __bfloat1622float2(h);
    }
    __half2 h = *reinterpret_cast<__half2*>(&u);
    return __half22float2(h);
}
__device__ __forceinline__ uint32_t f2_to_h2(float a, float b, int bf) {
    uint32_t u;
    if (bf) {
        __nv_bfloat162 h = __floats2bfloat162_rn(a, b);
        u = *reinterpret_cast<uint32_t*>(&h);
    } else {
        __half2 h = __floats2half2_rn(a, b);
        u = *reinterpret_cast<uint32_t*>(&h);
    }
    return u;
}

template <class T, bool G>
__device__ __forceinline__ T ld(const T* p) {
    if constexpr (G)
        return __ldg(p);
    else
        return *p;
}

// load the 12 complex components of site s into compute type C
// (G = true: global memory through the read-only path; false: shared memory)
template <int P, class C, bool G = true>
__device__ __forceinline__ void load_spinor(const char* base, long long V, long long s, cx<C> out[12]) {
    if constexpr (P == PDF && std::is_same<C, df>::value) {
        const float4* p = reinterpret_cast<const float4*>(base);
#pragma unroll
        for (int c = 0; c < 12; ++c) {
            float4 v = ld<float4, G>(&p[c * V + s]);
            out[c] = mk<C>(df(v.x, v.y), df(v.z, v.w));
        }
    } else if constexpr (P == PDF) {
        const float4* p = reinterpret_cast<const float4*>(base);
#pragma unroll
        for (int c = 0; c < 12; ++c) {
            float4 v = ld<float4, G>(&p[c * V + s]);
            if constexpr (sizeof(C) == 8)
                out[c] = mk<C>((C)v.x + (C)v.y, (C)v.z + (C)v.w);
            else
                out[c] = mk<C>(v.x + v.y, v.z + v.w);
        }
    } else if constexpr (P == P64) {
        const double2* p = reinterpret_cast<const double2*>(base);
#pragma unroll
        for (int c = 0; c < 12; ++c) {
            double2 v = ld<double2, G>(&p[c * V + s]);
            out[c] = mk<C>((C)v.x, (C)v.y);
        }
    } else if constexpr (P == P32) {
        const float4* p = reinterpret_cast<const float4*>(base);
#pragma unroll
        for (int q = 0; q < 6; ++q) {
            float4 v = ld<float4, G>(&p[q * V + s]);
            out[2 * q] = mk<C>((C)v.x, (C)v.y);
            out[2 * q + 1] = mk<C>((C)v.z, (C)v.w);
        }
    } else {
        const uint4* p = reinterpret_cast<const uint4*>(base);
        const float sc = ld<float, G>(reinterpret_cast<const float*>(p + 3 * V) + s);
        constexpr int bf = (P == PB16);
#pragma unroll
        for (int q = 0; q < 3; ++q) {
            uint4 v = ld<uint4, G>(&p[q * V + s]);
            float2 a = h2_to_f2(v.x, bf), b = h2_to_f2(v.y, bf), c = h2_to_f2(v.z, bf), d = h2_to_f2(v.w, bf);
            out[4 * q + 0] = mk<C>((C)(sc * a.x), (C)(sc * a.y));
            out[4 * q + 1] = mk<C>((C)(sc * b.x), (C)(sc * b.y));
            out[4 * q + 2] = mk<C>((C)(sc * c.x), (C)(sc * c.y));
            out[4 * q + 3] = mk<C>((C)(sc * d.x), (C)(sc * d.y));
        }
    }
}

template <int P, class C>
__device__ __forceinline__ void store_spinor(char* base, long long V, long long s, const cx<C> in[12]) {
    if constexpr (P == PDF && std::is_same<C, df>::value) {
        float4* p = reinterpret_cast<float4*>(base);
#pragma unroll
        for (int c = 0; c < 12; ++c) {
            const df a = df_norm(in[c].re), b = df_norm(in[c].im);
            p[c * V + s] = make_float4(a.hi, a.lo, b.hi, b.lo);
        }
    } else if constexpr (P == PDF) {
        float4* p = reinterpret_cast<float4*>(base);
#pragma unroll
        for (int c = 0; c < 12; ++c) {
            if constexpr (sizeof(C) == 8) {
                const df a = df_from_double((double)in[c].re), b = df_from_double((double)in[c].im);
                p[c * V + s] = make_float4(a.hi, a.lo, b.hi, b.lo);
            } else {
                p[c * V + s] = make_float4((float)in[c].re, 0.f, (float)in[c].im, 0.f);
            }
        }
    } else if constexpr (P == P64) {
        double2* p = reinterpret_cast<double2*>(base);
#pragma unroll
        for (int c = 0; c < 12; ++c) p[c * V + s] = make_double2((double)in[c].re, (double)in[c].im);
    } else if constexpr (P == P32) {
        float4* p = reinterpret_cast<float4*>(base);
#pragma unroll
        for (int q = 0; q < 6; ++q)
            p[q * V + s] = make_float4((float)in[2 * q].re, (float)in[2 * q].im, (float)in[2 * q + 1].re,
                                       (float)in[2 * q + 1].im);
    } else {
        uint4* p = reinterpret_cast<uint4*>(base);
        float mx = 0.f;
#pragma unroll
        for (int c = 0; c < 12; ++c) mx = fmaxf(mx, fmaxf(fabsf((float)in[c].re), fabsf((float)in[c].im)));
        const float sc = (mx > 0.f) ? mx : 1.f;
        const float inv = 1.f / sc;
        constexpr int bf = (P == PB16);
#pragma unroll
        for (int q = 0; q < 3; ++q) {
            uint4 v;
            v.x = f2_to_h2((float)in[4 * q + 0].re * inv, (float)in[4 * q + 0].im * inv, bf);
            v.y = f2_to_h2((float)in[4 * q + 1].re * inv, (float)in[4 * q + 1].im * inv, bf);
            v.z = f2_to_h2((float)in[4 * q + 2].re * inv, (float)in[4 * q + 2].im * inv, bf);
            v.w = f2_to_h2((float)in[4 * q + 3].re * inv, (float)in[4 * q + 3].im * inv, bf);
            p[q * V + s] = v;
        }
        reinterpret_cast<float*>(p + 3 * V)[s] = sc;
    }
}

// link U_{s,mu} (3x3, row-major) in compute type C
template <int P, class C, bool G = true>
__device__ __forceinline__ void load_link(const char* base, long long V, int mu, long long s, cx<C> u[9]) {
    if constexpr (P == PDF) {  // double-float links (only with the double-float stencil)
        const float4* p = reinterpret_cast<const float4*>(base) + (long long)mu * 9 * V;
#pragma unroll
        for (int c = 0; c < 9; ++c) {
            float4 v = ld<float4, G>(&p[c * V + s]);
            u[c] = mk<C>(C(v.x, v.y), C(v.z, v.w));
        }
    } else if constexpr (P == P64) {
        const double2* p = reinterpret_cast<const double2*>(base) + (long long)mu * 9 * V;
#pragma unroll
        for (int c = 0; c < 9; ++c) {
            double2 v = ld<double2, G>(&p[c * V + s]);
            u[c] = mk<C>((C)v.x, (C)v.y);
        }
    } else if constexpr (P == P32) {
        const float2* p = reinterpret_cast<const float2*>(base) + (long long)mu * 9 * V;
#pragma unroll
        for (int c = 0; c < 9; ++c) {
            float2 v = ld<float2, G>(&p[c * V + s]);
            u[c] = mk<C>((C)v.x, (C)v.y);
        }
    } else {
        const uint32_t* p = reinterpret_cast<const uint32_t*>(base) + (long long)mu * 9 * V;
        constexpr int bf = (P == PB16);
#pragma unroll
        for (int c = 0; c < 9; ++c) {
            float2 v = h2_to_f2(ld<uint32_t, G>(&p[c * V + s]), bf);
            u[c] = mk<C>((C)v.x, (C)v.y);
        }
    }
}

// ---------------------------------------------------------------------------
// hopping term
//
// Chiral basis: gamma_mu = [[0, A_mu], [A_mu^dagger, 0]] with
//   A_1 = -i sigma_1, A_2 = -i sigma_2, A_3 = -i sigma_3, A_4 = 1.
// (1 +- gamma_mu) has rank two: its upper two spin rows h = psi_u +- A_mu psi_l
// determine the lower two rows +- A_mu^dagger h, so one hop multiplies only
// two colour vectors by the link.
//
// hop<MU, SIGN>(psi, U, acc): acc += (1 + SIGN gamma_MU) W psi with W = U for
// SIGN = +1 and W = U^dagger for SIGN = -1.
// ---------------------------------------------------------------------------
// PACK (FP32 only): the complex products as paired FP32 FMAs on (re, im),
// w h = w.re (h) + w.im (i h), two paired FMAs per complex product (for
// U^dagger, conj(w) h = w.re h + w.im (-i h)). It saves issue slots where the
// registers allow (the SAP sweeps: 5% faster batched); in the stand-alone
// stencil, capped at 64-80 registers, it spills and loses.
template <class C, bool DAG, bool PACK = false>
__device__ __forceinline__ void su3_mul(const cx<C> u[9], const cx<C> h[3], cx<C> k[3]) {
#if defined(__CUDA_ARCH__) && (__CUDA_ARCH__ >= 1000)
    if constexpr (PACK && std::is_same<C, float>::value) {
        float2 hp[3], hr[3];
#pragma unroll
        for (int b = 0; b < 3; ++b) {
            hp[b] = make_float2(h[b].re, h[b].im);
            hr[b] = DAG ? make_float2(h[b].im, -h[b].re) : make_float2(-h[b].im, h[b].re);
        }
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            float2 acc = make_float2(0.f, 0.f);
#pragma unroll
            for (int b = 0; b < 3; ++b) {
                const cx<float> w = DAG ? u[3 * b + a] : u[3 * a + b];
                acc = __ffma2_rn(make_float2(w.re, w.re), hp[b], acc);
                acc = __ffma2_rn(make_float2(w.im, w.im), hr[b], acc);
            }
            k[a] = mk<float>(acc.x, acc.y);
        }
        return;
    }
#endif
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        cx<C> acc;
        if (!DAG) {
            acc = u[3 * a] * h[0];
            acc = acc + u[3 * a + 1] * h[1];
            acc = acc + u[3 * a + 2] * h[2];
        } else {
            acc = cmulc(u[a], h[0]);
            acc = acc + cmulc(u[3 + a], h[1]);
            acc = acc + cmulc(u[6 + a], h[2]);
        }
        k[a] = acc;
    }
}

#if defined(__CUDA_ARCH__) && (__CUDA_ARCH__ >= 1000)
// paired FP32 forms of project/reconstruct: every factor is +-1 or +-i, so
// each lane is one rounded multiply-add of an exact product, the same result
// as the scalar code, in half the instructions (the +-i cases pair the
// swapped components)
__device__ __forceinline__ float2 f2(cx<float> a) { return make_float2(a.re, a.im); }
__device__ __forceinline__ float2 f2sw(cx<float> a) { return make_float2(a.im, a.re); }
__device__ __forceinline__ cx<float> cxf(float2 a) { return mk<float>(a.x, a.y); }
// a + (w.x * b.x, w.y * b.y)
__device__ __forceinline__ cx<float> fma_pair(float2 w, float2 b, cx<float> a) { return cxf(__ffma2_rn(w, b, f2(a))); }
#endif

// upper two spin rows of (1 + SIGN gamma_MU) psi
template <int MU, int SIGN, class C, bool PACK = false>
__device__ __forceinline__ void project(const cx<C> psi[12], cx<C> h0[3], cx<C> h1[3]) {
#if defined(__CUDA_ARCH__) && (__CUDA_ARCH__ >= 1000)
    if constexpr (PACK && std::is_same<C, float>::value) {
        const float s = (float)SIGN;
        const float2 pp = make_float2(s, s), pm = make_float2(s, -s), mp = make_float2(-s, s),
                     mm = make_float2(-s, -s);
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            const cx<float> p0 = psi[c], p1 = psi[3 + c], p2 = psi[6 + c], p3 = psi[9 + c];
            if constexpr (MU == 0) {  // p0 - s i p3, p1 - s i p2
                h0[c] = fma_pair(pm, f2sw(p3), p0);
                h1[c] = fma_pair(pm, f2sw(p2), p1);
            } else if constexpr (MU == 1) {  // p0 - s p3, p1 + s p2
                h0[c] = fma_pair(mm, f2(p3), p0);
                h1[c] = fma_pair(pp, f2(p2), p1);
            } else if constexpr (MU == 2) {  // p0 - s i p2, p1 + s i p3
                h0[c] = fma_pair(pm, f2sw(p2), p0);
                h1[c] = fma_pair(mp, f2sw(p3), p1);
            } else {  // p0 + s p2, p1 + s p3
                h0[c] = fma_pair(pp, f2(p2), p0);
                h1[c] = fma_pair(pp, f2(p3), p1);
            }
        }
        return;
    }
#endif
    const C s = (C)SIGN;
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        const cx<C> p0 = psi[c], p1 = psi[3 + c], p2 = psi[6 + c], p3 = psi[9 + c];
        if constexpr (MU == 0) {  // h0 = p0 - s i p3, h1 = p1 - s i p2
            h0[c] = p0 - s * ti(p3);
            h1[c] = p1 - s * ti(p2);
        } else if constexpr (MU == 1) {  // h0 = p0 - s p3, h1 = p1 + s p2
            h0[c] = p0 - s * p3;
            h1[c] = p1 + s * p2;
        } else if constexpr (MU == 2) {  // h0 = p0 - s i p2, h1 = p1 + s i p3
            h0[c] = p0 - s * ti(p2);
            h1[c] = p1 + s * ti(p3);
        } else {  // h0 = p0 + s p2, h1 = p1 + s p3
            h0[c] = p0 + s * p2;
            h1[c] = p1 + s * p3;
        }
    }
}

// acc += the four spin rows rebuilt from the multiplied upper rows k0, k1
template <int MU, int SIGN, class C, bool PACK = false>
__device__ __forceinline__ void reconstruct(const cx<C> k0[3], const cx<C> k1[3], cx<C> acc[12]) {
#if defined(__CUDA_ARCH__) && (__CUDA_ARCH__ >= 1000)
    if constexpr (PACK && std::is_same<C, float>::value) {
        const float s = (float)SIGN;
        const float2 pp = make_float2(s, s), pm = make_float2(s, -s), mp = make_float2(-s, s),
                     mm = make_float2(-s, -s);
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            acc[c] = cxf(__fadd2_rn(f2(acc[c]), f2(k0[c])));
            acc[3 + c] = cxf(__fadd2_rn(f2(acc[3 + c]), f2(k1[c])));
            if constexpr (MU == 0) {  // lower = s i (k1, k0)
                acc[6 + c] = fma_pair(mp, f2sw(k1[c]), acc[6 + c]);
                acc[9 + c] = fma_pair(mp, f2sw(k0[c]), acc[9 + c]);
            } else if constexpr (MU == 1) {  // lower = s (k1, -k0)
                acc[6 + c] = fma_pair(pp, f2(k1[c]), acc[6 + c]);
                acc[9 + c] = fma_pair(mm, f2(k0[c]), acc[9 + c]);
            } else if constexpr (MU == 2) {  // lower = s i (k0, -k1)
                acc[6 + c] = fma_pair(mp, f2sw(k0[c]), acc[6 + c]);
                acc[9 + c] = fma_pair(pm, f2sw(k1[c]), acc[9 + c]);
            } else {  // lower = s (k0, k1)
                acc[6 + c] = fma_pair(pp, f2(k0[c]), acc[6 + c]);
                acc[9 + c] = fma_pair(pp, f2(k1[c]), acc[9 + c]);
            }
        }
        return;
    }
#endif
    const C s = (C)SIGN;
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        acc[c] = acc[c] + k0[c];
        acc[3 + c] = acc[3 + c] + k1[c];
        if constexpr (MU == 0) {  // lower = s i (k1, k0)
            acc[6 + c] = acc[6 + c] + s * ti(k1[c]);
            acc[9 + c] = acc[9 + c] + s * ti(k0[c]);
        } else if constexpr (MU == 1) {  // lower = s (k1, -k0)
            acc[6 + c] = acc[6 + c] + s * k1[c];
            acc[9 + c] = acc[9 + c] - s * k0[c];
        } else if constexpr (MU == 2) {  // lower = s i (k0, -k1)
            acc[6 + c] = acc[6 + c] + s * ti(k0[c]);
            acc[9 + c] = acc[9 + c] - s * ti(k1[c]);
        } else {  // lower = s (k0, k1)
            acc[6 + c] = acc[6 + c] + s * k0[c];
            acc[9 + c] = acc[9 + c] + s * k1[c];
        }
    }
}

template <int MU, int SIGN, class C, bool PACK = false>
__device__ __forceinline__ void hop(const cx<C> psi[12], const cx<C> u[9], cx<C> acc[12]) {
    cx<C> h0[3], h1[3], k0[3], k1[3];
    project<MU, SIGN, C, PACK>(psi, h0, h1);
    su3_mul<C, (SIGN < 0), PACK>(u, h0, k0);
    su3_mul<C, (SIGN < 0), PACK>(u, h1, k1);
    reconstruct<MU, SIGN, C, PACK>(k0, k1, acc);
}

// ---------------------------------------------------------------------------
// clover term (site-diagonal): per site two hermitian 6x6 blocks, chirality 0
// acting on spinor components 0..5 (spins 0, 1) and chirality 1 on 6..11
// (spins 2, 3). Each block is packed as 36 reals: the 6 (real) diagonal
// entries, then the 15 entries above the diagonal, row by row, as (re, im).
//   FP64 storage: double [72][V];   FP32 storage: float4 [18][V].
// clover_acc<P>(A, V, s, in, acc, w): acc += w * (A_s in), in the compute
// type C (double, float or double-float; FP64 storage feeds double and
// double-float arithmetic, FP32 storage feeds float).
// ---------------------------------------------------------------------------
#ifdef __CUDACC__
template <class C>
__device__ __forceinline__ void clover_block(const C b[36], const cx<C>* x, cx<C>* acc, C w) {
    cx<C> y[6];
#pragma unroll
    for (int i = 0; i < 6; ++i) y[i] = b[i] * x[i];
    int k = 6;
#pragma unroll
    for (int i = 0; i < 6; ++i)
#pragma unroll
        for (int j = i + 1; j < 6; ++j) {
            const cx<C> o = mk<C>(b[k], b[k + 1]);
            k += 2;
            y[i] = y[i] + o * x[j];
            y[j] = y[j] + cmulc(o, x[i]);
        }
#pragma unroll
    for (int i = 0; i < 6; ++i) acc[i] = acc[i] + w * y[i];
}

template <int P, class C>
__device__ __forceinline__ void clover_acc(const char* A, long long V, long long s, const cx<C> in[12], cx<C> acc[12],
                                           C w) {
#pragma unroll
    for (int chi = 0; chi < 2; ++chi) {
        C b[36];
        if constexpr (P == P32) {
            const float4* a = reinterpret_cast<const float4*>(A);
#pragma unroll
            for (int q = 0; q < 9; ++q) {
                const float4 v = __ldg(&a[(long long)(9 * chi + q) * V + s]);
                b[4 * q] = C(v.x);
                b[4 * q + 1] = C(v.y);
                b[4 * q + 2] = C(v.z);
                b[4 * q + 3] = C(v.w);
            }
        } else {
            const double* a = reinterpret_cast<const double*>(A);
#pragma unroll
            for (int q = 0; q < 36; ++q) {
                const double v = __ldg(&a[(long long)(36 * chi + q) * V + s]);
                if constexpr (std::is_same<C, df>::value)
                    b[q] = df_from_double(v);
                else
                    b[q] = (C)v;
            }
        }
        clover_block<C>(b, in + 6 * chi, acc + 6 * chi, w);
    }
}
#endif

// ---------------------------------------------------------------------------
// per-rhs field addressing for batched launches
//
// A FieldRef names one spinor field per right-hand side r:
//   base + r * rhs_stride + (col(r) + col_off) * col_stride
// where col(r) = jtab[r] when a column table is given (Krylov bases), else 0.
// A right-hand side with jtab[r] < 0 is inactive for the launch.
// ---------------------------------------------------------------------------
struct FieldRef {
    char* base;
    long long rhs_stride;
    long long col_stride;
    int col_off;
};

__device__ __forceinline__ char* field_ptr(const FieldRef& f, const int* jtab, int r) {
    const int j = jtab ? jtab[r] : 0;
    return f.base + (long long)r * f.rhs_stride + (long long)(j + f.col_off) * f.col_stride;
}
__device__ __forceinline__ bool rhs_active(const int* jtab, int r) { return jtab == nullptr || jtab[r] >= 0; }

}  // namespace dwk
