// Wilson-Dirac stencil D (Sec. 2, Eq. "Dw") on the full periodic lattice, and
// the layout conversions between the canonical FP64 layout of the C ABI and
// the component-major device layouts (common.cuh).
//
// One thread computes one site of one right-hand side: eight spin-projected
// hops (two SU(3) x colour-vector products each), then
//   out_n = (4 + m0) in_n - 1/2 sum_hops           (or  sub_n - that).
// Consecutive threads take consecutive sites, so every load of a component
// plane is a coalesced 128/256/512-byte warp transaction; neighbour spinors
// are re-read from L2 by the 8 sites that need them.
#include <algorithm>

#include "internal.h"

namespace dwk {

namespace {

constexpr int kThreads = 256;

// canonical FP64 -> internal layout, times scale[r] (in FP64, before rounding)
// when a per-rhs scale is given
template <int P>
__global__ void __launch_bounds__(kThreads) to_internal_kernel(const double* __restrict__ canon, char* out,
                                                               long long V, long long out_rs,
                                                               const double* __restrict__ scale) {
    const long long s = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    const int r = blockIdx.y;
    if (s >= V) return;
    typedef typename real_of<P>::type C;
    const double f = scale ? scale[r] : 1.0;
    const double2* src = reinterpret_cast<const double2*>(canon) + ((long long)r * V + s) * 12;
    cx<C> v[12];
#pragma unroll
    for (int c = 0; c < 12; ++c) {
        double2 t = src[c];
        v[c] = mk<C>((C)(t.x * f), (C)(t.y * f));
    }
    store_spinor<P, C>(out + r * out_rs, V, s, v);
}

// internal layout -> canonical FP64, times scale[r] when given
template <int P>
__global__ void __launch_bounds__(kThreads) from_internal_kernel(const char* in, double* __restrict__ canon,
                                                                 long long V, long long in_rs,
                                                                 const double* __restrict__ scale) {
    const long long s = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    const int r = blockIdx.y;
    if (s >= V) return;
    typedef typename real_of<P>::type C;
    const double f = scale ? scale[r] : 1.0;
    cx<C> v[12];
    load_spinor<P, C>(in + r * in_rs, V, s, v);
    double2* dst = reinterpret_cast<double2*>(canon) + ((long long)r * V + s) * 12;
#pragma unroll
    for (int c = 0; c < 12; ++c) dst[c] = make_double2((double)v[c].re * f, (double)v[c].im * f);
}

template <int P>
__global__ void __launch_bounds__(kThreads) gauge_convert_kernel(const double* __restrict__ U, char* out,
                                                                 long long V) {
    const long long s = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (s >= V) return;
    const double2* src = reinterpret_cast<const double2*>(U) + s * 36;
    for (int mu = 0; mu < 4; ++mu)
        for (int c = 0; c < 9; ++c) {
            const double2 t = src[9 * mu + c];
            const long long e = ((long long)mu * 9 + c) * V + s;
            if constexpr (P == P64) {
                reinterpret_cast<double2*>(out)[e] = t;
            } else if constexpr (P == P32) {
                reinterpret_cast<float2*>(out)[e] = make_float2((float)t.x, (float)t.y);
            } else {
                reinterpret_cast<uint32_t*>(out)[e] = f2_to_h2((float)t.x, (float)t.y, P == PB16);
            }
        }
}

// Link field from the internal FP64 layout to another internal precision.
template <int P>
__global__ void __launch_bounds__(kThreads) link_convert_kernel(const double2* __restrict__ U, char* out,
                                                                long long n) {
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n; e += (long long)gridDim.x * blockDim.x) {
        const double2 t = U[e];
        if constexpr (P == P32) {
            reinterpret_cast<float2*>(out)[e] = make_float2((float)t.x, (float)t.y);
        } else if constexpr (P == PDF) {
            const df a(t.x), b(t.y);
            reinterpret_cast<float4*>(out)[e] = make_float4(a.hi, a.lo, b.hi, b.lo);
        } else {
            reinterpret_cast<uint32_t*>(out)[e] = f2_to_h2((float)t.x, (float)t.y, P == PB16);
        }
    }
}

// Field conversion between internal precisions (same layout family).
template <int PI, int PO>
__global__ void __launch_bounds__(kThreads) convert_kernel(FieldRef in, FieldRef out, long long V,
                                                           const int* jtab) {
    const long long s = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    const int r = blockIdx.y;
    if (s >= V || !rhs_active(jtab, r)) return;
    // FP64-class precision only when both sides carry it
    typedef typename real_of<((PI == P64 || PI == PDF) && (PO == P64 || PO == PDF)) ? P64 : P32>::type C;
    cx<C> v[12];
    load_spinor<PI, C>(field_ptr(in, jtab, r), V, s, v);
    store_spinor<PO, C>(field_ptr(out, jtab, r), V, s, v);
}

// CTAs per SM (measured at 24^3 x 48): the FP32 stencil is latency-bound and
// fastest at three (80 registers), the 16-bit one is issue-bound (decode) and
// fastest at two (no register cap that forces spills), the Arnoldi product
// (FP32 in, double-float out) at four; other 16-bit inputs keep three
template <int PI, int PO, int PL, class C>
constexpr int dw_min_blocks() {
    return sizeof(C) != 4 ? 1 : (PI == P32 && PO == P32) ? 3 : (PI == P32) ? 4 : (PO == PI) ? 2 : 3;
}

template <int PI, int PO, int PL, class C, bool SUB, bool CLOV>
__global__ void __launch_bounds__(kThreads, dw_min_blocks<PI, PO, PL, C>())
    dw_kernel(Geom g, C diag, FieldRef in, FieldRef out, const char* U, const int* jtab, int nrhs, FieldRef sub,
              const char* clov) {
    const int r = blockIdx.x % nrhs;
    const long long s = (blockIdx.x / nrhs) * (long long)blockDim.x + threadIdx.x;
    if (s >= g.V || !rhs_active(jtab, r)) return;
    const char* pin = field_ptr(in, jtab, r);
    int x[4];
    site_coords(g, s, x);
    cx<C> acc[12];
#pragma unroll
    for (int c = 0; c < 12; ++c) acc[c] = czero<C>();
    cx<C> psi[12], u[9];
#define DW_HOPS(MU)                                                     \
    {                                                                   \
        const long long sp = neighbour(g, s, x, MU, +1);                \
        load_spinor<PI, C>(pin, g.V, sp, psi);                          \
        load_link<PL, C>(U, g.V, MU, s, u);                             \
        hop<MU, +1, C>(psi, u, acc);                                    \
        const long long sm = neighbour(g, s, x, MU, -1);                \
        load_spinor<PI, C>(pin, g.V, sm, psi);                          \
        load_link<PL, C>(U, g.V, MU, sm, u);                            \
        hop<MU, -1, C>(psi, u, acc);                                    \
    }
    DW_HOPS(0)
    DW_HOPS(1)
    DW_HOPS(2)
    DW_HOPS(3)
#undef DW_HOPS
    load_spinor<PI, C>(pin, g.V, s, psi);
    // clover term A psi_n, folded into the accumulator as -2 A psi_n
    if constexpr (CLOV) clover_acc<(sizeof(C) == 4) ? P32 : P64, C>(clov, g.V, s, psi, acc, C(-2.0f));
    const C half = C(0.5f);
    cx<C> res[12];
    if constexpr (SUB) {
        cx<C> b[12];
        load_spinor<PO, C>(field_ptr(sub, jtab, r), g.V, s, b);
#pragma unroll
        for (int c = 0; c < 12; ++c) res[c] = b[c] - (diag * psi[c] - half * acc[c]);
    } else {
#pragma unroll
        for (int c = 0; c < 12; ++c) res[c] = diag * psi[c] - half * acc[c];
    }
    store_spinor<PO, C>(field_ptr(out, jtab, r), g.V, s, res);
}

dim3 site_grid(long long V, int nrhs) { return dim3((unsigned)((V + kThreads - 1) / kThreads), nrhs); }

// every supported precision combination carries the clover term
template <int PI, int PO, int PL, class C>
constexpr bool clover_combo() {
    return true;
}

template <int PI, int PO, int PL, class C>
int dw_dispatch_sub(const Geom& g, double m0, FieldRef in, FieldRef out, const char* U, const int* jtab, int nrhs,
                    const FieldRef* sub, const ClovRef* cl, cudaStream_t st) {
    // double-float arithmetic holds about 164 registers a thread: 128-thread
    // blocks let three CTAs (12 warps) share an SM instead of one of 256
    constexpr int bt = std::is_same<C, df>::value ? 128 : kThreads;
    const unsigned nb = (unsigned)((g.V + bt - 1) / bt) * (unsigned)nrhs;
    const C diag = C(4.0 + m0);
    FieldRef none{};
    const FieldRef sb = sub ? *sub : none;
    if (cl) {
        if constexpr (clover_combo<PI, PO, PL, C>()) {
            const char* A = (sizeof(C) == 4) ? cl->a32 : cl->a64;
            if (sub) {
                if constexpr (PO == P64 || PO == PDF)
                    dw_kernel<PI, PO, PL, C, true, true><<<nb, bt, 0, st>>>(g, diag, in, out, U, jtab, nrhs, sb, A);
                else
                    return fail(DW_EINVAL, "residual stencil requires an FP64-class output");
            } else {
                dw_kernel<PI, PO, PL, C, false, true><<<nb, bt, 0, st>>>(g, diag, in, out, U, jtab, nrhs, sb, A);
            }
            DW_LAUNCH_CHECK();
            return DW_OK;
        } else {
            return fail(DW_EINVAL, "the clover term is not available for this precision combination");
        }
    }
    if (sub) {
        if constexpr (PO == P64 || PO == PDF)
            dw_kernel<PI, PO, PL, C, true, false><<<nb, bt, 0, st>>>(g, diag, in, out, U, jtab, nrhs, sb, nullptr);
        else
            return fail(DW_EINVAL, "residual stencil requires an FP64-class output");
    } else {
        dw_kernel<PI, PO, PL, C, false, false><<<nb, bt, 0, st>>>(g, diag, in, out, U, jtab, nrhs, sb, nullptr);
    }
    DW_LAUNCH_CHECK();
    return DW_OK;
}

}  // namespace

int launch_to_internal(int prec, const double* canon, char* out, long long V, int nrhs, cudaStream_t st,
                       const double* scale) {
    const long long rs = spinor_bytes(prec, V);
    dim3 grid = site_grid(V, nrhs);
    switch (prec) {
        case P64: to_internal_kernel<P64><<<grid, kThreads, 0, st>>>(canon, out, V, rs, scale); break;
        case P32: to_internal_kernel<P32><<<grid, kThreads, 0, st>>>(canon, out, V, rs, scale); break;
        case P16: to_internal_kernel<P16><<<grid, kThreads, 0, st>>>(canon, out, V, rs, scale); break;
        case PB16: to_internal_kernel<PB16><<<grid, kThreads, 0, st>>>(canon, out, V, rs, scale); break;
        case PDF: to_internal_kernel<PDF><<<grid, kThreads, 0, st>>>(canon, out, V, rs, scale); break;
        default: return fail(DW_EINVAL, "bad precision");
    }
    DW_LAUNCH_CHECK();
    return DW_OK;
}

int launch_from_internal(int prec, const char* in, double* canon, long long V, int nrhs, cudaStream_t st,
                         const double* scale) {
    const long long rs = spinor_bytes(prec, V);
    dim3 grid = site_grid(V, nrhs);
    switch (prec) {
        case P64: from_internal_kernel<P64><<<grid, kThreads, 0, st>>>(in, canon, V, rs, scale); break;
        case P32: from_internal_kernel<P32><<<grid, kThreads, 0, st>>>(in, canon, V, rs, scale); break;
        case P16: from_internal_kernel<P16><<<grid, kThreads, 0, st>>>(in, canon, V, rs, scale); break;
        case PB16: from_internal_kernel<PB16><<<grid, kThreads, 0, st>>>(in, canon, V, rs, scale); break;
        case PDF: from_internal_kernel<PDF><<<grid, kThreads, 0, st>>>(in, canon, V, rs, scale); break;
        default: return fail(DW_EINVAL, "bad precision");
    }
    DW_LAUNCH_CHECK();
    return DW_OK;
}

int launch_gauge_convert(int prec, const double* U, char* out, long long V, cudaStream_t st) {
    dim3 grid = site_grid(V, 1);
    switch (prec) {
        case P64: gauge_convert_kernel<P64><<<grid, kThreads, 0, st>>>(U, out, V); break;
        case P32: gauge_convert_kernel<P32><<<grid, kThreads, 0, st>>>(U, out, V); break;
        case P16: gauge_convert_kernel<P16><<<grid, kThreads, 0, st>>>(U, out, V); break;
        case PB16: gauge_convert_kernel<PB16><<<grid, kThreads, 0, st>>>(U, out, V); break;
        default: return fail(DW_EINVAL, "bad precision");
    }
    DW_LAUNCH_CHECK();
    return DW_OK;
}

int launch_link_convert(int prec, const char* U64, char* out, long long V, cudaStream_t st) {
    const long long n = 36 * V;
    const unsigned nb = (unsigned)std::min<long long>((n + kThreads - 1) / kThreads, 152LL * 16);
    const double2* src = reinterpret_cast<const double2*>(U64);
    switch (prec) {
        case P32: link_convert_kernel<P32><<<nb, kThreads, 0, st>>>(src, out, n); break;
        case P16: link_convert_kernel<P16><<<nb, kThreads, 0, st>>>(src, out, n); break;
        case PB16: link_convert_kernel<PB16><<<nb, kThreads, 0, st>>>(src, out, n); break;
        case PDF: link_convert_kernel<PDF><<<nb, kThreads, 0, st>>>(src, out, n); break;
        default: return fail(DW_EINVAL, "bad link precision");
    }
    DW_LAUNCH_CHECK();
    return DW_OK;
}

int launch_convert(int pin, int pout, FieldRef in, FieldRef out, long long V, const int* jtab, int nrhs,
                   cudaStream_t st) {
    dim3 grid = site_grid(V, nrhs);
#define CONV(A, B)                                                                            \
    if (pin == A && pout == B) {                                                              \
        convert_kernel<A, B><<<grid, kThreads, 0, st>>>(in, out, V, jtab);                    \
        DW_LAUNCH_CHECK();                                                      \
        return DW_OK;                                                                         \
    }
    CONV(P64, P64)
    CONV(P64, P32)
    CONV(P64, P16)
    CONV(P64, PB16)
    CONV(P32, P64)
    CONV(P16, P64)
    CONV(PB16, P64)
    CONV(P16, P32)
    CONV(PB16, P32)
    CONV(PDF, P32)
    CONV(PDF, P16)
    CONV(PDF, PB16)
    CONV(PDF, P64)
    CONV(P64, PDF)
#undef CONV
    return fail(DW_EINVAL, "unsupported conversion");
}

int launch_dw(int pin, int pout, int plink, const Geom& g, double m0, FieldRef in, FieldRef out, const char* U,
              const int* jtab, int nrhs, const FieldRef* sub, cudaStream_t st, const ClovRef* cl) {
    // Supported combinations: uniform precision (the stencil as an operator),
    // and low-precision input with an FP64 output (Arnoldi product w = D z).
#define DWC(A, B, L, C)                                                                       \
    if (pin == A && pout == B && plink == L) return dw_dispatch_sub<A, B, L, C>(g, m0, in, out, U, jtab, nrhs, sub, cl, st);
    DWC(P64, P64, P64, double)
    DWC(P32, P32, P32, float)
    DWC(P16, P16, P16, float)
    DWC(PB16, PB16, PB16, float)
    DWC(P16, P32, P32, float)
    DWC(PB16, P32, P32, float)
    DWC(P32, P64, P32, float)
    DWC(P16, P64, P32, float)
    DWC(PB16, P64, P32, float)
    DWC(P32, P64, P64, double)
    DWC(P16, P64, P64, double)
    DWC(PB16, P64, P64, double)
    DWC(P32, PDF, P32, float)
    DWC(P16, PDF, P32, float)
    DWC(PB16, PDF, P32, float)
    DWC(P32, PDF, P64, double)
    DWC(P16, PDF, P64, double)
    DWC(PB16, PDF, P64, double)
    DWC(PDF, PDF, P64, double)
    DWC(P64, PDF, P64, double)
    DWC(PDF, PDF, PDF, df)
#undef DWC
    return fail(DW_EINVAL, "unsupported stencil precision combination");
}

}  // namespace dwk
