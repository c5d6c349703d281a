// One colour half-sweep of the Schwarz alternating procedure (Sec. 2,
// Algorithm 2) with inexact minimal-residual domain solves (Sec. 4).
//
// One CTA owns one domain L^l of the swept colour (and one right-hand side);
// one thread owns one site of the domain. The CTA
//   1. stages the domain's own links U_{n,mu} (n in L^l) in shared memory,
//   2. computes r^l = (v - D x)^l with the full operator (neighbour values of
//      x come from the opposite colour, read through L2),
//   3. runs nmr MR steps on D^l y = r^l entirely out of shared memory:
//        p = D^l rho;  alpha = <p,rho>/<p,p>;  y += alpha rho;  rho -= alpha p
//      (D^l keeps only hops whose both ends lie in L^l, Eq. "Dw_local"; the
//      inner products are CTA-wide warp-shuffle reductions),
//   4. writes x^l + y^l back.
// Domains of one colour never couple (even domain count per direction), so
// all CTAs of a launch are independent and the launch order is irrelevant.
#include <mutex>
#include <set>

#include "internal.h"

namespace dwk {

namespace {

// The domain's own links in shared memory, packed so that one link matrix
// (9 complex entries) is read with as few wide loads as possible:
//   P64      double2 [4][9][T]                                          (9 x 16 B loads)
//   P32      float2 [4][9][T]                                           (9 x 8 B loads)
//   P16/B16  uint4 [4][2][T] (entry quads) + uint32 [4][T] (entry 8)    (2 x 16 B + 4 B)
// pack() writes that layout for one site of a domain into a global image of
// the domain (built once per gauge field), so that a CTA stages all its links
// with one bulk asynchronous copy. (FP32 entry pairs packed as float4
// measured no faster than plain float2 loads.)
template <int PL>
struct LinkSh;
template <>
struct LinkSh<P64> {
    static constexpr int kBytes = 576;
    static __device__ __forceinline__ void pack(unsigned char* L, int T, int t, const char* U, long long V,
                                                long long s) {
        const double2* Ug = reinterpret_cast<const double2*>(U);
        double2* A = reinterpret_cast<double2*>(L);
        for (int c = 0; c < 36; ++c) A[c * T + t] = Ug[(long long)c * V + s];
    }
    template <class C>
    static __device__ __forceinline__ void load(const unsigned char* L, int T, int mu, int t, cx<C> u[9]) {
        const double2* A = reinterpret_cast<const double2*>(L) + mu * 9 * T;
#pragma unroll
        for (int c = 0; c < 9; ++c) {
            const double2 v = A[c * T + t];
            u[c] = mk<C>((C)v.x, (C)v.y);
        }
    }
};
template <>
struct LinkSh<P32> {
    static constexpr int kBytes = 288;
    static __device__ __forceinline__ void pack(unsigned char* L, int T, int t, const char* U, long long V,
                                                long long s) {
        const float2* Ug = reinterpret_cast<const float2*>(U);
        float2* A = reinterpret_cast<float2*>(L);
        for (int c = 0; c < 36; ++c) A[c * T + t] = Ug[(long long)c * V + s];
    }
    template <class C>
    static __device__ __forceinline__ void load(const unsigned char* L, int T, int mu, int t, cx<C> u[9]) {
        const float2* A = reinterpret_cast<const float2*>(L) + mu * 9 * T;
#pragma unroll
        for (int c = 0; c < 9; ++c) {
            const float2 v = A[c * T + t];
            u[c] = mk<C>((C)v.x, (C)v.y);
        }
    }
};
template <int PL>
struct LinkSh16 {
    static constexpr int kBytes = 144;
    static __device__ __forceinline__ void pack(unsigned char* L, int T, int t, const char* U, long long V,
                                                long long s) {
        const uint32_t* Ug = reinterpret_cast<const uint32_t*>(U);
        uint32_t* A = reinterpret_cast<uint32_t*>(L);            // uint4 [4][2][T] seen as words
        uint32_t* B = reinterpret_cast<uint32_t*>(L + 128 * T);  // uint32 [4][T]
        for (int mu = 0; mu < 4; ++mu) {
            for (int c = 0; c < 8; ++c)
                A[4 * ((mu * 2 + (c >> 2)) * T + t) + (c & 3)] = Ug[(long long)(mu * 9 + c) * V + s];
            B[mu * T + t] = Ug[(long long)(mu * 9 + 8) * V + s];
        }
    }
    template <class C>
    static __device__ __forceinline__ void load(const unsigned char* L, int T, int mu, int t, cx<C> u[9]) {
        constexpr int bf = (PL == PB16);
        const uint4* A = reinterpret_cast<const uint4*>(L) + mu * 2 * T;
        const uint32_t* B = reinterpret_cast<const uint32_t*>(L + 128 * T);
#pragma unroll
        for (int q = 0; q < 2; ++q) {
            const uint4 v = A[q * T + t];
            const float2 a = h2_to_f2(v.x, bf), b = h2_to_f2(v.y, bf), c = h2_to_f2(v.z, bf), d = h2_to_f2(v.w, bf);
            u[4 * q] = mk<C>((C)a.x, (C)a.y);
            u[4 * q + 1] = mk<C>((C)b.x, (C)b.y);
            u[4 * q + 2] = mk<C>((C)c.x, (C)c.y);
            u[4 * q + 3] = mk<C>((C)d.x, (C)d.y);
        }
        const float2 w = h2_to_f2(B[mu * T + t], bf);
        u[8] = mk<C>((C)w.x, (C)w.y);
    }
};
template <>
struct LinkSh<P16> : LinkSh16<P16> {};
template <>
struct LinkSh<PB16> : LinkSh16<PB16> {};

// The MR iterate rho in shared memory: FP32 as float4 [6][T] (two complex per
// load), FP64 as double2 [12][T].
template <class C>
__device__ __forceinline__ void rho_store(unsigned char* R, int T, int t, const cx<C> v[12]) {
    if constexpr (sizeof(C) == 4) {
        float4* p = reinterpret_cast<float4*>(R);
#pragma unroll
        for (int q = 0; q < 6; ++q) p[q * T + t] = make_float4(v[2 * q].re, v[2 * q].im, v[2 * q + 1].re, v[2 * q + 1].im);
    } else {
        double2* p = reinterpret_cast<double2*>(R);
#pragma unroll
        for (int c = 0; c < 12; ++c) p[c * T + t] = make_double2(v[c].re, v[c].im);
    }
}
template <class C>
__device__ __forceinline__ void rho_load(const unsigned char* R, int T, int t, cx<C> v[12]) {
    if constexpr (sizeof(C) == 4) {
        const float4* p = reinterpret_cast<const float4*>(R);
#pragma unroll
        for (int q = 0; q < 6; ++q) {
            const float4 a = p[q * T + t];
            v[2 * q] = mk<C>(a.x, a.y);
            v[2 * q + 1] = mk<C>(a.z, a.w);
        }
    } else {
        const double2* p = reinterpret_cast<const double2*>(R);
#pragma unroll
        for (int c = 0; c < 12; ++c) {
            const double2 a = p[c * T + t];
            v[c] = mk<C>(a.x, a.y);
        }
    }
}

template <class C>
__device__ __forceinline__ void block_sum3(C& a, C& b, C& c, C* red) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        a += __shfl_xor_sync(0xffffffffu, a, o);
        b += __shfl_xor_sync(0xffffffffu, b, o);
        c += __shfl_xor_sync(0xffffffffu, c, o);
    }
    const int w = threadIdx.x >> 5;
    if ((threadIdx.x & 31) == 0) {
        red[3 * w] = a;
        red[3 * w + 1] = b;
        red[3 * w + 2] = c;
    }
    __syncthreads();
    const int nw = blockDim.x >> 5;
    C sa = 0, sb = 0, sc = 0;
    for (int i = 0; i < nw; ++i) {
        sa += red[3 * i];
        sb += red[3 * i + 1];
        sc += red[3 * i + 2];
    }
    a = sa;
    b = sb;
    c = sc;
}

__device__ __forceinline__ unsigned smem_u32(const void* p) { return (unsigned)__cvta_generic_to_shared(p); }
__device__ __forceinline__ unsigned long long global_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}
// mbarrier completed by the byte count of one bulk copy (one arrival)
__device__ __forceinline__ void bulk_copy_start(void* dst, const void* src, unsigned bytes, unsigned long long* bar) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(bar)) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                     smem_u32(dst)),
                 "l"(src), "r"(bytes), "r"(smem_u32(bar))
                 : "memory");
}
// wait for phase 0 of the mbarrier, giving up after about a second
__device__ __forceinline__ bool bulk_copy_wait(unsigned long long* bar) {
    unsigned long long t0 = 0;
    for (unsigned it = 1;; ++it) {
        unsigned done;
        asm volatile(
            "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], 0;\n selp.u32 %0, 1, 0, p;\n}\n"
            : "=r"(done)
            : "r"(smem_u32(bar))
            : "memory");
        if (done) return true;
        if ((it & 1023) == 0) {
            const unsigned long long now = global_ns();
            if (t0 == 0)
                t0 = now;
            else if (now - t0 > 1000000000ULL)
                return false;
        }
    }
}

// CLOV: the operator carries the clover term A (site-diagonal, so it is part
// of D^l on every site): clov is its FP32 storage for float arithmetic and its
// FP64 storage for double arithmetic. Uimg: the links of every domain packed
// as the shared-memory image of LinkSh<PL> for blockDim.x threads (domain
// d = D0 + nb0 (D1 + nb1 (D2 + nb2 D3)) at byte d * kBytes * blockDim.x).
// err_host: set (host-mapped) if the bulk copy of the links did not complete.
template <int PS, int PL, class C, int MAXT, bool CLOV>
__global__ void __launch_bounds__(MAXT, (MAXT <= 256 && sizeof(C) == 4) ? 2 : 1)
    sap_sweep_kernel(Geom g, C diag, FieldRef vref, FieldRef xref, const char* __restrict__ Uimg, const int* jtab,
                     int nrhs, int colour, int nmr, int mode, const char* __restrict__ clov, int* err_host) {
    constexpr int CP = (sizeof(C) == 4) ? P32 : P64;  // storage of the clover term
    typedef LinkSh<PL> LS;
    extern __shared__ __align__(16) unsigned char smem[];
    const int T = blockDim.x;
    unsigned char* rsh = smem;                                   // rho (MR phase) / own x (residual phase)
    unsigned char* lsh = smem + sizeof(C) * 24 * T;              // links
    C* red = reinterpret_cast<C*>(lsh + (size_t)LS::kBytes * T);  // [32][3]
    unsigned long long* lbar = reinterpret_cast<unsigned long long*>(red + 96);

    const int r = blockIdx.x % nrhs;
    const int e = blockIdx.x / nrhs;
    if (!rhs_active(jtab, r)) return;  // uniform over the CTA
    const char* vb = field_ptr(vref, jtab, r);
    char* xb = field_ptr(xref, jtab, r);

    // domain e of this colour: block coordinates D with sum(D) % 2 == colour
    const int half1 = g.nb[0] >> 1;
    int D[4];
    {
        int t = e / half1;
        D[1] = t % g.nb[1];
        t /= g.nb[1];
        D[2] = t % g.nb[2];
        D[3] = t / g.nb[2];
        D[0] = 2 * (e % half1) + ((colour + D[1] + D[2] + D[3]) & 1);
    }
    const int tid = threadIdx.x;
    const bool act = tid < g.B;
    int lx[4], xg[4];
    {
        int q = act ? tid : 0;
        lx[0] = q % g.b[0];
        q /= g.b[0];
        lx[1] = q % g.b[1];
        q /= g.b[1];
        lx[2] = q % g.b[2];
        lx[3] = q / g.b[2];
    }
#pragma unroll
    for (int j = 0; j < 4; ++j) xg[j] = D[j] * g.b[j] + lx[j];
    const long long s = site_index(g, xg);
    const int ls1 = g.b[0], ls2 = g.b[0] * g.b[1], ls3 = g.b[0] * g.b[1] * g.b[2];  // in-domain strides

    // 0. programmatic dependent launch: the next sweep may be scheduled onto
    //    SMs as this one's CTAs retire, and stage its links meanwhile
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");

    // 1. asynchronous copies global -> shared, all in flight together: the
    //    domain's own links (constant during a solve, so copied before the
    //    previous sweep has finished; one bulk copy of the domain's image)
    //    and, once that sweep's x is final, in the general mode the domain's
    //    own iterate x in storage layout (stride T), read by interior hops
    const unsigned lbytes = (unsigned)LS::kBytes * (unsigned)T;
    const int dstride[4] = {1, g.nb[0], g.nb[0] * g.nb[1], g.nb[0] * g.nb[1] * g.nb[2]};
    const long long dom = D[0] + (long long)dstride[1] * D[1] + (long long)dstride[2] * D[2] +
                          (long long)dstride[3] * D[3];
    const unsigned char* limg = reinterpret_cast<const unsigned char*>(Uimg);
    // the domain one step down in direction mu (periodic)
    auto dom_lo = [&](int mu) {
        return D[mu] > 0 ? dom - dstride[mu] : dom + (long long)(g.nb[mu] - 1) * dstride[mu];
    };
    if (tid == 0) bulk_copy_start(lsh, limg + dom * lbytes, lbytes, lbar);
    // every read of v and x and every write of x comes after the previous
    // kernel of the stream has completed (a no-op without a programmatic
    // dependency)
    asm volatile("griddepcontrol.wait;" ::: "memory");
    if (act) {
        if (mode == 2) {
            if constexpr (PS == P64) {
                for (int c = 0; c < 12; ++c)
                    cp_async_word(reinterpret_cast<double2*>(rsh) + c * T + tid,
                                  reinterpret_cast<const double2*>(xb) + c * g.V + s);
            } else if constexpr (PS == P32) {
                for (int q = 0; q < 6; ++q)
                    cp_async_word(reinterpret_cast<float4*>(rsh) + q * T + tid,
                                  reinterpret_cast<const float4*>(xb) + q * g.V + s);
            } else {
                for (int q = 0; q < 3; ++q)
                    cp_async_word(reinterpret_cast<uint4*>(rsh) + q * T + tid,
                                  reinterpret_cast<const uint4*>(xb) + q * g.V + s);
                cp_async_word(reinterpret_cast<float*>(reinterpret_cast<uint4*>(rsh) + 3 * T) + tid,
                              reinterpret_cast<const float*>(reinterpret_cast<const uint4*>(xb) + 3 * g.V) + s);
            }
        }
    }
    cx<C> rho[12], y[12];
    if (act) load_spinor<PS, C>(vb, g.V, s, rho);  // overlaps the copies above
    cp_async_wait();
    __syncthreads();
    if (__syncthreads_or(!bulk_copy_wait(lbar))) {
        if (tid == 0) {
            *reinterpret_cast<volatile int*>(err_host) = 1;
            __threadfence_system();
        }
        bulk_copy_wait(lbar);  // the copy may still be in flight: wait once more before the CTA retires
        return;
    }

    // 2. residual r = v - D x at this site: interior neighbours and every
    //    forward link from shared memory, boundary neighbours through L2.
    //    The eight hops are unrolled with compile-time directions so that the
    //    loads of one hop overlap the arithmetic of the previous one.
    if (act) {
        if (mode != 0) {
            cx<C> acc[12], psi[12], u[9];
#pragma unroll
            for (int c = 0; c < 12; ++c) acc[c] = czero<C>();
            const bool general = (mode == 2);
            const char* xsh = reinterpret_cast<const char*>(rsh);
    // an interior neighbour is read from shared memory and a boundary one
    // through L2 (its link from the neighbouring domain's image, at the
    // site's index there); the branches differ only in the loads, so each
    // direction runs one hop for the whole warp
#define SAP_RES_HOPS(MU, LS_MU)                                                              \
    {                                                                                        \
        const bool inp = lx[MU] + 1 < g.b[MU];                                               \
        if (inp) {                                                                           \
            if (general) load_spinor<PS, C, false>(xsh, T, tid + LS_MU, psi);                \
        } else {                                                                             \
            load_spinor<PS, C>(xb, g.V, neighbour(g, s, xg, MU, +1), psi);                   \
        }                                                                                    \
        if (general || !inp) {                                                               \
            LS::template load<C>(lsh, T, MU, tid, u);                                        \
            hop<MU, +1, C, true>(psi, u, acc);                                               \
        }                                                                                    \
        const bool inm = lx[MU] >= 1;                                                        \
        if (inm) {                                                                           \
            if (general) {                                                                   \
                const int tn = tid - LS_MU;                                                  \
                load_spinor<PS, C, false>(xsh, T, tn, psi);                                  \
                LS::template load<C>(lsh, T, MU, tn, u);                                     \
            }                                                                                \
        } else {                                                                             \
            const long long sm = neighbour(g, s, xg, MU, -1);                                \
            load_spinor<PS, C>(xb, g.V, sm, psi);                                            \
            LS::template load<C>(limg + dom_lo(MU) * lbytes, T, MU, tid + (g.b[MU] - 1) * LS_MU, u); \
        }                                                                                    \
        if (general || !inm) hop<MU, -1, C, true>(psi, u, acc);                              \
    }
            SAP_RES_HOPS(0, 1)
            SAP_RES_HOPS(1, ls1)
            SAP_RES_HOPS(2, ls2)
            SAP_RES_HOPS(3, ls3)
#undef SAP_RES_HOPS
            const C half = (C)0.5;
            if (general) {
                load_spinor<PS, C, false>(xsh, T, tid, psi);
                if constexpr (CLOV) clover_acc<CP, C>(clov, g.V, s, psi, acc, (C)-2);  // A x as -2 A x in acc
#pragma unroll
                for (int c = 0; c < 12; ++c) rho[c] = rho[c] - (diag * psi[c] - half * acc[c]);
            } else {
#pragma unroll
                for (int c = 0; c < 12; ++c) rho[c] = rho[c] + half * acc[c];
            }
        }
    } else {
#pragma unroll
        for (int c = 0; c < 12; ++c) rho[c] = czero<C>();
    }
#pragma unroll
    for (int c = 0; c < 12; ++c) y[c] = czero<C>();
    __syncthreads();  // x in shared memory is overwritten by the MR iterate below

    // 3. MR on D^l y = r^l out of shared memory
    for (int it = 0; it < nmr; ++it) {
        rho_store<C>(rsh, T, tid, rho);
        __syncthreads();
        cx<C> p[12];
        C pr_re = 0, pr_im = 0, pp = 0;
        if (act) {
            cx<C> acc[12], psi[12], u[9];
#pragma unroll
            for (int c = 0; c < 12; ++c) acc[c] = czero<C>();
#define SAP_LOC_HOPS(MU, LS_MU)                                                               \
    {                                                                                         \
        if (lx[MU] + 1 < g.b[MU]) {                                                           \
            rho_load<C>(rsh, T, tid + LS_MU, psi);                                            \
            LS::template load<C>(lsh, T, MU, tid, u);                                         \
            hop<MU, +1, C, true>(psi, u, acc);                                                      \
        }                                                                                     \
        if (lx[MU] >= 1) {                                                                    \
            const int tn = tid - LS_MU;                                                       \
            rho_load<C>(rsh, T, tn, psi);                                                     \
            LS::template load<C>(lsh, T, MU, tn, u);                                          \
            hop<MU, -1, C, true>(psi, u, acc);                                                      \
        }                                                                                     \
    }
            SAP_LOC_HOPS(0, 1)
            SAP_LOC_HOPS(1, ls1)
            SAP_LOC_HOPS(2, ls2)
            SAP_LOC_HOPS(3, ls3)
#undef SAP_LOC_HOPS
            // the site's own rho is read back from shared memory (where the
            // neighbours read it) rather than kept in registers over the hops:
            // the 24 registers go to overlapping the hops' loads
            rho_load<C>(rsh, T, tid, rho);
            if constexpr (CLOV) clover_acc<CP, C>(clov, g.V, s, rho, acc, (C)-2);  // A rho as -2 A rho in acc
            const C half = (C)0.5;
#pragma unroll
            for (int c = 0; c < 12; ++c) {
                p[c] = diag * rho[c] - half * acc[c];
                const cx<C> t = cmulc(p[c], rho[c]);
                pr_re += t.re;
                pr_im += t.im;
                pp += p[c].re * p[c].re + p[c].im * p[c].im;
            }
        } else {
#pragma unroll
            for (int c = 0; c < 12; ++c) p[c] = czero<C>();
        }
        block_sum3(pr_re, pr_im, pp, red);
        if (pp > (C)0) {
            const cx<C> alpha = mk<C>(pr_re / pp, pr_im / pp);
#pragma unroll
            for (int c = 0; c < 12; ++c) {
                y[c] = y[c] + alpha * rho[c];
                rho[c] = rho[c] - alpha * p[c];
            }
        }
    }
    __syncthreads();  // every residual read of x inside the domain precedes the writes below

    // 4. x^l <- x^l + y^l
    if (act) {
        if (mode == 2) {
            cx<C> xo[12];
            load_spinor<PS, C>(xb, g.V, s, xo);
#pragma unroll
            for (int c = 0; c < 12; ++c) y[c] = y[c] + xo[c];
        }
        store_spinor<PS, C>(xb, g.V, s, y);
    }
}

// the links of domain blockIdx.x (all domains, both colours) in the layout a
// CTA of blockDim.x threads keeps them in shared memory
template <int PL>
__global__ void link_image_kernel(Geom g, const char* __restrict__ U, char* __restrict__ img) {
    const int t = threadIdx.x;
    if (t >= g.B) return;
    int D[4], q = blockIdx.x;
    D[0] = q % g.nb[0];
    q /= g.nb[0];
    D[1] = q % g.nb[1];
    q /= g.nb[1];
    D[2] = q % g.nb[2];
    D[3] = q / g.nb[2];
    int xg[4], r = t;
    xg[0] = D[0] * g.b[0] + r % g.b[0];
    r /= g.b[0];
    xg[1] = D[1] * g.b[1] + r % g.b[1];
    r /= g.b[1];
    xg[2] = D[2] * g.b[2] + r % g.b[2];
    xg[3] = D[3] * g.b[3] + r / g.b[2];
    LinkSh<PL>::pack(reinterpret_cast<unsigned char*>(img) + (size_t)blockIdx.x * LinkSh<PL>::kBytes * blockDim.x,
                     blockDim.x, t, U, g.V, site_index(g, xg));
}

template <int PS, int PL, class C>
int sap_launch_t(const Geom& g, double m0, FieldRef v, FieldRef x, const char* Uimg, const int* jtab, int nrhs,
                 int colour, int nmr, int mode, int threads, cudaStream_t st, const ClovRef* cl, int* err_host) {
    if (cl && threads > 256) return fail(DW_EINVAL, "the clover SAP sweep handles domains of at most 256 sites");
    const size_t smem = (size_t)sap_smem_bytes(PS, PL, g, threads);
    // the shared-memory limit is a per-device property of the kernel: set it once per device
    static std::mutex mu;
    static std::set<int> done;
    {
        int dev = 0;
        DW_CUDA_TRY(cudaGetDevice(&dev));
        std::lock_guard<std::mutex> lock(mu);
        if (!done.count(dev)) {
            DW_CUDA_TRY(cudaFuncSetAttribute(sap_sweep_kernel<PS, PL, C, 256, false>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024));
            DW_CUDA_TRY(cudaFuncSetAttribute(sap_sweep_kernel<PS, PL, C, 1024, false>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024));
            DW_CUDA_TRY(cudaFuncSetAttribute(sap_sweep_kernel<PS, PL, C, 256, true>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024));
            done.insert(dev);
        }
    }
    const unsigned nb = (unsigned)(g.ndom / 2) * (unsigned)nrhs;
    // launched with programmatic stream serialisation: when the previous
    // kernel of the stream is a sweep, this one starts staging its links
    // during that sweep's tail (the kernel waits for the previous grid before
    // it touches v or x)
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(nb);
    cfg.blockDim = dim3(threads);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    const C diag = (C)(4.0 + m0);
    const char* A = cl ? ((sizeof(C) == 4) ? cl->a32 : cl->a64) : nullptr;
    if (cl)
        DW_CUDA_TRY(cudaLaunchKernelEx(&cfg, sap_sweep_kernel<PS, PL, C, 256, true>, g, diag, v, x, Uimg, jtab, nrhs,
                                       colour, nmr, mode, A, err_host));
    else if (threads <= 256)
        DW_CUDA_TRY(cudaLaunchKernelEx(&cfg, sap_sweep_kernel<PS, PL, C, 256, false>, g, diag, v, x, Uimg, jtab, nrhs,
                                       colour, nmr, mode, A, err_host));
    else
        DW_CUDA_TRY(cudaLaunchKernelEx(&cfg, sap_sweep_kernel<PS, PL, C, 1024, false>, g, diag, v, x, Uimg, jtab, nrhs,
                                       colour, nmr, mode, A, err_host));
    DW_LAUNCH_CHECK();
    return DW_OK;
}

size_t link_sh_bytes(int plink) { return plink == P64 ? 576 : plink == P32 ? 288 : 144; }

}  // namespace

int sap_smem_bytes(int pspin, int plink, const Geom& g, int threads) {
    const size_t c = (pspin == P64) ? 8 : 4;
    (void)g;
    // rho/x, links, the [32][3] reduction buffer, the links' mbarrier
    return (int)(c * 24 * threads + link_sh_bytes(plink) * threads + c * 3 * 32 + 16);
}

int sap_threads(const Geom& g, int threads) { return threads > 0 ? threads : ((g.B + 31) / 32) * 32; }

size_t sap_link_image_bytes(int plink, const Geom& g, int threads) {
    return link_sh_bytes(plink) * (size_t)sap_threads(g, threads) * (size_t)g.ndom;
}

int launch_sap_link_image(int plink, const Geom& g, const char* U, char* img, int threads, cudaStream_t st) {
    threads = sap_threads(g, threads);
    DW_CUDA_TRY(cudaMemsetAsync(img, 0, sap_link_image_bytes(plink, g, threads), st));  // rows of idle threads
    const unsigned nb = (unsigned)g.ndom;
    if (plink == P64)
        link_image_kernel<P64><<<nb, threads, 0, st>>>(g, U, img);
    else if (plink == P32)
        link_image_kernel<P32><<<nb, threads, 0, st>>>(g, U, img);
    else if (plink == P16)
        link_image_kernel<P16><<<nb, threads, 0, st>>>(g, U, img);
    else if (plink == PB16)
        link_image_kernel<PB16><<<nb, threads, 0, st>>>(g, U, img);
    else
        return fail(DW_EINVAL, "unsupported SAP link precision");
    DW_LAUNCH_CHECK();
    return DW_OK;
}

int launch_sap_sweep(int pspin, int plink, const Geom& g, double m0, FieldRef v, FieldRef x, const char* Uimg,
                     const int* jtab, int nrhs, int colour, int nmr, int mode, int threads, cudaStream_t st,
                     const ClovRef* cl, int* err_host) {
    threads = sap_threads(g, threads);
    if (threads < g.B || threads % 32 != 0 || threads > 1024) return fail(DW_EINVAL, "bad SAP thread count");
    if (sap_smem_bytes(pspin, plink, g, threads) > 227 * 1024)
        return fail(DW_EINVAL, "SAP domain does not fit in shared memory at this precision");
    if (nmr < 1) return fail(DW_EINVAL, "nmr must be >= 1");
    if (pspin == P64 && plink == P64)
        return sap_launch_t<P64, P64, double>(g, m0, v, x, Uimg, jtab, nrhs, colour, nmr, mode, threads, st,
                                              cl, err_host);
    if (pspin == P32 && plink == P32)
        return sap_launch_t<P32, P32, float>(g, m0, v, x, Uimg, jtab, nrhs, colour, nmr, mode, threads, st,
                                             cl, err_host);
    if (pspin == P16 && plink == P16)
        return sap_launch_t<P16, P16, float>(g, m0, v, x, Uimg, jtab, nrhs, colour, nmr, mode, threads, st,
                                             cl, err_host);
    if (pspin == PB16 && plink == PB16)
        return sap_launch_t<PB16, PB16, float>(g, m0, v, x, Uimg, jtab, nrhs, colour, nmr, mode, threads, st,
                                               cl, err_host);
    return fail(DW_EINVAL, "unsupported SAP precision combination");
}

}  // namespace dwk
