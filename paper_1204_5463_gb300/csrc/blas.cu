// Level-1 kernels of the flexible Arnoldi process and of the deflated restart
// (Algorithms 3 and 4): fused multi-dot products, multi-axpy with the norm of
// the result, normalisation, the basis rotations V_{k+1} = V_{m+1} Q_{k+1},
// Z_k = Z_m Q_k, and the iterate update x += Z eta.
//
// Reductions are deterministic: every CTA writes its partial sums to a fixed
// slot, and one finishing CTA per right-hand side adds the slots in order.
#include "internal.h"

namespace dwk {

namespace {

constexpr int kT = 256;      // threads per CTA
constexpr int kGroup = 8;    // basis vectors handled per sweep of a multi-dot
constexpr int kRotMax = 17;  // output columns held in registers by a rotation

__device__ __forceinline__ double2 cfma_conj(double2 v, double2 w, double2 acc) {
    // acc + conj(v) * w
    acc.x = fma(v.x, w.x, acc.x);
    acc.x = fma(v.y, w.y, acc.x);
    acc.y = fma(v.x, w.y, acc.y);
    acc.y = fma(-v.y, w.x, acc.y);
    return acc;
}

__device__ __forceinline__ double warp_sum(double a) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) a += __shfl_xor_sync(0xffffffffu, a, o);
    return a;
}

__device__ __forceinline__ int rhs_nv(const int* jtab, int r, int off) { return jtab ? jtab[r] + off : off; }

// partial[r][blk][i] = sum over this CTA's elements of conj(V_i) w, i < nv;
// partial[r][blk][nvmax] = sum |w|^2
__global__ void __launch_bounds__(kT) multidot_kernel(VecRef Vb, VecRef w, long long n, const int* jtab, int nv_off,
                                                      int nvmax, double2* partial) {
    __shared__ double2 sh[64 + 1][kT / 32];
    const int r = blockIdx.y;
    if (jtab && jtab[r] < 0) return;
    const int nv = rhs_nv(jtab, r, nv_off);
    const int j = jtab ? jtab[r] : 0;
    const double2* Vr = Vb.base + r * Vb.rhs_stride;
    const double2* wr = w.base + r * w.rhs_stride + (long long)(j + w.col_off) * w.col_stride;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const long long stride = (long long)gridDim.x * kT;
    const long long e0 = (long long)blockIdx.x * kT + threadIdx.x;
    double wn = 0.0;
    for (int g0 = 0; g0 < nv || g0 == 0; g0 += kGroup) {
        double2 acc[kGroup];
#pragma unroll
        for (int q = 0; q < kGroup; ++q) acc[q] = make_double2(0.0, 0.0);
        const int gn = min(kGroup, nv - g0);
        for (long long e = e0; e < n; e += stride) {
            const double2 wv = __ldg(&wr[e]);
            if (g0 == 0) wn = fma(wv.x, wv.x, fma(wv.y, wv.y, wn));
#pragma unroll
            for (int q = 0; q < kGroup; ++q)
                if (q < gn) {
                    const double2* vi = Vr + (long long)(g0 + q + Vb.col_off) * Vb.col_stride;
                    acc[q] = cfma_conj(__ldg(&vi[e]), wv, acc[q]);
                }
        }
#pragma unroll
        for (int q = 0; q < kGroup; ++q)
            if (q < gn) {
                const double a = warp_sum(acc[q].x), b = warp_sum(acc[q].y);
                if (lane == 0) sh[g0 + q][warp] = make_double2(a, b);
            }
        if (nv == 0) break;
    }
    wn = warp_sum(wn);
    if (lane == 0) sh[64][warp] = make_double2(wn, 0.0);
    __syncthreads();
    const int NP = nvmax + 1;
    double2* out = partial + ((long long)r * gridDim.x + blockIdx.x) * NP;
    for (int i = threadIdx.x; i < NP; i += kT) {
        const int src = (i == nvmax) ? 64 : i;
        double2 s = make_double2(0.0, 0.0);
        if (i < nv || i == nvmax)
            for (int q = 0; q < kT / 32; ++q) s.x += sh[src][q].x, s.y += sh[src][q].y;
        out[i] = s;
    }
}

// out[r][i] = sum_blk partial[r][blk][i] in fixed order
__global__ void __launch_bounds__(kT) finalize_kernel(const double2* partial, int nblk, int NP, const int* jtab,
                                                      double2* out) {
    const int r = blockIdx.x;
    if (jtab && jtab[r] < 0) return;
    for (int i = threadIdx.x; i < NP; i += kT) {
        double2 s = make_double2(0.0, 0.0);
        const double2* p = partial + (long long)r * nblk * NP + i;
        for (int b = 0; b < nblk; ++b) {
            const double2 t = p[(long long)b * NP];
            s.x += t.x;
            s.y += t.y;
        }
        out[(long long)r * NP + i] = s;
    }
}

__global__ void __launch_bounds__(kT) finalize_real_kernel(const double2* partial, int nblk, const int* jtab,
                                                           double* out) {
    const int r = blockIdx.x;
    if (jtab && jtab[r] < 0) return;
    if (threadIdx.x == 0) {
        double s = 0.0;
        for (int b = 0; b < nblk; ++b) s += partial[(long long)r * nblk + b].x;
        out[r] = s;
    }
}

// w -= sum_i coef[r][i] V_i ; partial norm of the result
__global__ void __launch_bounds__(kT) multiaxpy_kernel(VecRef Vb, VecRef w, long long n, const int* jtab, int nv_off,
                                                       const double2* coef, int coef_ld, double2* partial) {
    __shared__ double2 h[64];
    __shared__ double red[kT / 32];
    const int r = blockIdx.y;
    if (jtab && jtab[r] < 0) return;
    const int nv = rhs_nv(jtab, r, nv_off);
    const int j = jtab ? jtab[r] : 0;
    for (int i = threadIdx.x; i < nv; i += kT) h[i] = coef[(long long)r * coef_ld + i];
    __syncthreads();
    const double2* Vr = Vb.base + r * Vb.rhs_stride;
    double2* wr = w.base + r * w.rhs_stride + (long long)(j + w.col_off) * w.col_stride;
    const long long stride = (long long)gridDim.x * kT;
    double wn = 0.0;
    for (long long e = (long long)blockIdx.x * kT + threadIdx.x; e < n; e += stride) {
        double2 acc = wr[e];
        for (int i = 0; i < nv; ++i) {
            const double2 v = __ldg(&(Vr + (long long)(i + Vb.col_off) * Vb.col_stride)[e]);
            const double2 c = h[i];
            acc.x = fma(-c.x, v.x, acc.x);
            acc.x = fma(c.y, v.y, acc.x);
            acc.y = fma(-c.x, v.y, acc.y);
            acc.y = fma(-c.y, v.x, acc.y);
        }
        wr[e] = acc;
        wn = fma(acc.x, acc.x, fma(acc.y, acc.y, wn));
    }
    wn = warp_sum(wn);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = wn;
    __syncthreads();
    if (threadIdx.x == 0) {
        double s = 0.0;
        for (int q = 0; q < kT / 32; ++q) s += red[q];
        partial[(long long)r * gridDim.x + blockIdx.x] = make_double2(s, 0.0);
    }
}

__global__ void __launch_bounds__(kT) normalize_kernel(VecRef w, VecRef dst, long long n, const int* jtab,
                                                       const double* norm2) {
    const int r = blockIdx.y;
    if (jtab && jtab[r] < 0) return;
    const int j = jtab ? jtab[r] : 0;
    const double nn = norm2[r];
    const double inv = nn > 0.0 ? 1.0 / sqrt(nn) : 0.0;
    const double2* src = w.base + r * w.rhs_stride + (long long)(j + w.col_off) * w.col_stride;
    double2* out = dst.base + r * dst.rhs_stride + (long long)(j + dst.col_off) * dst.col_stride;
    for (long long e = (long long)blockIdx.x * kT + threadIdx.x; e < n; e += (long long)gridDim.x * kT) {
        const double2 v = src[e];
        out[e] = make_double2(v.x * inv, v.y * inv);
    }
}

__global__ void __launch_bounds__(kT) scale_kernel(const double2* src, double2* dst, long long rs, long long n,
                                                   const double* a) {
    const int r = blockIdx.y;
    const double s = a[r];
    for (long long e = (long long)blockIdx.x * kT + threadIdx.x; e < n; e += (long long)gridDim.x * kT) {
        const double2 v = src[r * rs + e];
        dst[r * rs + e] = make_double2(v.x * s, v.y * s);
    }
}

// In-place rotation of flat complex columns: X_c = sum_i X_i Q[i][c] (c < kout)
template <class T2, class R>
__global__ void __launch_bounds__(kT) rotate_flat_kernel(T2* X, long long rs, long long cs, long long n,
                                                         const int* active, int nin, int kout, const double2* Q,
                                                         int qld) {
    const int r = blockIdx.y;
    if (active && !active[r]) return;
    T2* Xr = X + r * rs;
    const double2* Qr = Q + (long long)r * qld * qld;  // Q[r][i][c] at Qr[i*qld + c]
    for (long long e = (long long)blockIdx.x * kT + threadIdx.x; e < n; e += (long long)gridDim.x * kT) {
        R ar[kRotMax], ai[kRotMax];
#pragma unroll
        for (int c = 0; c < kRotMax; ++c) ar[c] = ai[c] = (R)0;
        for (int i = 0; i < nin; ++i) {
            const T2 v = Xr[(long long)i * cs + e];
            const double2* qrow = Qr + (long long)i * qld;
#pragma unroll
            for (int c = 0; c < kRotMax; ++c)
                if (c < kout) {
                    const double2 q = __ldg(&qrow[c]);
                    ar[c] += (R)q.x * v.x - (R)q.y * v.y;
                    ai[c] += (R)q.x * v.y + (R)q.y * v.x;
                }
        }
#pragma unroll
        for (int c = 0; c < kRotMax; ++c)
            if (c < kout) {
                T2 o;
                o.x = ar[c];
                o.y = ai[c];
                Xr[(long long)c * cs + e] = o;
            }
    }
}

// Out-of-place rotation for per-site-scaled storage: one thread per site,
// one output column at a time (Y_c = sum_i X_i Q[i][c]).
template <int P>
__global__ void __launch_bounds__(kT) rotate_site_kernel(const char* X, char* Y, long long rs, long long cs,
                                                         long long yrs, long long V, const int* active, int nin,
                                                         int kout, const double2* Q, int qld) {
    const int r = blockIdx.y;
    if (active && !active[r]) return;
    const long long s = (long long)blockIdx.x * kT + threadIdx.x;
    if (s >= V) return;
    const double2* Qr = Q + (long long)r * qld * qld;
    for (int c = 0; c < kout; ++c) {
        cx<float> acc[12];
#pragma unroll
        for (int a = 0; a < 12; ++a) acc[a] = czero<float>();
        for (int i = 0; i < nin; ++i) {
            cx<float> v[12];
            load_spinor<P, float>(X + r * rs + i * cs, V, s, v);
            const double2 q = __ldg(&Qr[(long long)i * qld + c]);
            const cx<float> qf = mk<float>((float)q.x, (float)q.y);
#pragma unroll
            for (int a = 0; a < 12; ++a) acc[a] = acc[a] + qf * v[a];
        }
        store_spinor<P, float>(Y + r * yrs + c * cs, V, s, acc);
    }
}

// x += sum_i Z_i eta_i, one thread per site
template <int P>
__global__ void __launch_bounds__(kT) xupdate_kernel(const char* Z, long long z_rs, long long z_cs, double2* x,
                                                     long long x_rs, long long V, const int* nz, const double2* eta,
                                                     int eta_ld) {
    const int r = blockIdx.y;
    const int n = nz[r];
    if (n <= 0) return;
    const long long s = (long long)blockIdx.x * kT + threadIdx.x;
    if (s >= V) return;
    typedef typename real_of<P>::type C;
    double2* xr = x + r * x_rs;
    cx<double> acc[12];
#pragma unroll
    for (int a = 0; a < 12; ++a) {
        const double2 t = xr[a * V + s];
        acc[a] = mk<double>(t.x, t.y);
    }
    for (int i = 0; i < n; ++i) {
        cx<C> v[12];
        load_spinor<P, C>(Z + r * z_rs + i * z_cs, V, s, v);
        const double2 q = __ldg(&eta[(long long)r * eta_ld + i]);
        const cx<double> qd = mk<double>(q.x, q.y);
#pragma unroll
        for (int a = 0; a < 12; ++a) acc[a] = acc[a] + qd * mk<double>((double)v[a].re, (double)v[a].im);
    }
#pragma unroll
    for (int a = 0; a < 12; ++a) xr[a * V + s] = make_double2(acc[a].re, acc[a].im);
}

__global__ void __launch_bounds__(kT) norm2_kernel(const double2* a, long long rs, long long n, double2* partial) {
    __shared__ double red[kT / 32];
    const int r = blockIdx.y;
    const double2* ar = a + r * rs;
    double s = 0.0;
    for (long long e = (long long)blockIdx.x * kT + threadIdx.x; e < n; e += (long long)gridDim.x * kT) {
        const double2 v = ar[e];
        s = fma(v.x, v.x, fma(v.y, v.y, s));
    }
    s = warp_sum(s);
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

}  // namespace

int blas_nblk(long long n) { return (int)grid_for(n); }

int launch_multidot(VecRef Vb, VecRef w, long long n, const int* jtab, int nv_off, int nvmax, int nrhs,
                    double2* partial, int nblk, double2* out, cudaStream_t st) {
    if (nvmax > 64) return fail(DW_EINVAL, "too many basis vectors for one multi-dot");
    multidot_kernel<<<dim3(nblk, nrhs), kT, 0, st>>>(Vb, w, n, jtab, nv_off, nvmax, partial);
    DW_CUDA_TRY(cudaGetLastError());
    finalize_kernel<<<nrhs, kT, 0, st>>>(partial, nblk, nvmax + 1, jtab, out);
    DW_CUDA_TRY(cudaGetLastError());
    return DW_OK;
}

int launch_multiaxpy(VecRef Vb, VecRef w, long long n, const int* jtab, int nv_off, int nrhs, const double2* coef,
                     int coef_ld, double2* partial, int nblk, double* out_norm2, cudaStream_t st) {
    multiaxpy_kernel<<<dim3(nblk, nrhs), kT, 0, st>>>(Vb, w, n, jtab, nv_off, coef, coef_ld, partial);
    DW_CUDA_TRY(cudaGetLastError());
    finalize_real_kernel<<<nrhs, 32, 0, st>>>(partial, nblk, jtab, out_norm2);
    DW_CUDA_TRY(cudaGetLastError());
    return DW_OK;
}

int launch_normalize(VecRef w, VecRef dst, long long n, const int* jtab, int nrhs, const double* norm2,
                     cudaStream_t st) {
    normalize_kernel<<<dim3(grid_for(n), nrhs), kT, 0, st>>>(w, dst, n, jtab, norm2);
    DW_CUDA_TRY(cudaGetLastError());
    return DW_OK;
}

int launch_scale(const double2* src, double2* dst, long long rs, long long n, int nrhs, const double* a,
                 cudaStream_t st) {
    scale_kernel<<<dim3(grid_for(n), nrhs), kT, 0, st>>>(src, dst, rs, n, a);
    DW_CUDA_TRY(cudaGetLastError());
    return DW_OK;
}

int launch_rotate(int prec, char* X, long long rhs_stride, long long col_stride, long long V, int nrhs,
                  const int* active, int nin, int kout, const double2* Q, int qld, char* scratch,
                  cudaStream_t st) {
    if (kout > kRotMax && (prec == P64 || prec == P32)) return fail(DW_EINVAL, "deflation dimension too large");
    if (prec == P64) {
        const long long n = 12 * V;
        rotate_flat_kernel<double2, double><<<dim3(grid_for(n), nrhs), kT, 0, st>>>(
            reinterpret_cast<double2*>(X), rhs_stride / 16, col_stride / 16, n, active, nin, kout, Q, qld);
    } else if (prec == P32) {
        const long long n = 12 * V;
        rotate_flat_kernel<float2, float><<<dim3(grid_for(n), nrhs), kT, 0, st>>>(
            reinterpret_cast<float2*>(X), rhs_stride / 8, col_stride / 8, n, active, nin, kout, Q, qld);
    } else {
        if (!scratch) return fail(DW_EINVAL, "rotation of scaled storage needs scratch");
        const long long yrs = col_stride * kout;
        dim3 grid((unsigned)((V + kT - 1) / kT), nrhs);
        if (prec == P16)
            rotate_site_kernel<P16><<<grid, kT, 0, st>>>(X, scratch, rhs_stride, col_stride, yrs, V, active, nin,
                                                         kout, Q, qld);
        else
            rotate_site_kernel<PB16><<<grid, kT, 0, st>>>(X, scratch, rhs_stride, col_stride, yrs, V, active, nin,
                                                          kout, Q, qld);
        DW_CUDA_TRY(cudaGetLastError());
        for (int r = 0; r < nrhs; ++r)
            DW_CUDA_TRY(cudaMemcpyAsync(X + r * rhs_stride, scratch + r * yrs, (size_t)yrs,
                                        cudaMemcpyDeviceToDevice, st));
        return DW_OK;
    }
    DW_CUDA_TRY(cudaGetLastError());
    return DW_OK;
}

int launch_xupdate(int prec, const char* Z, long long z_rs, long long z_cs, double2* x, long long x_rs, long long V,
                   int nrhs, const int* nz, const double2* eta, int eta_ld, cudaStream_t st) {
    dim3 grid((unsigned)((V + kT - 1) / kT), nrhs);
    const long long xrs = x_rs / 16;
    switch (prec) {
        case P64: xupdate_kernel<P64><<<grid, kT, 0, st>>>(Z, z_rs, z_cs, x, xrs, V, nz, eta, eta_ld); break;
        case P32: xupdate_kernel<P32><<<grid, kT, 0, st>>>(Z, z_rs, z_cs, x, xrs, V, nz, eta, eta_ld); break;
        case P16: xupdate_kernel<P16><<<grid, kT, 0, st>>>(Z, z_rs, z_cs, x, xrs, V, nz, eta, eta_ld); break;
        case PB16: xupdate_kernel<PB16><<<grid, kT, 0, st>>>(Z, z_rs, z_cs, x, xrs, V, nz, eta, eta_ld); break;
        default: return fail(DW_EINVAL, "bad precision");
    }
    DW_CUDA_TRY(cudaGetLastError());
    return DW_OK;
}

int launch_norm2(const double2* a, long long rs, long long n, int nrhs, double2* partial, int nblk, double* out,
                 cudaStream_t st) {
    norm2_kernel<<<dim3(nblk, nrhs), kT, 0, st>>>(a, rs, n, partial);
    DW_CUDA_TRY(cudaGetLastError());
    finalize_real_kernel<<<nrhs, 32, 0, st>>>(partial, nblk, nullptr, out);
    DW_CUDA_TRY(cudaGetLastError());
    return DW_OK;
}

int launch_zero(void* p, size_t bytes, cudaStream_t st) {
    DW_CUDA_TRY(cudaMemsetAsync(p, 0, bytes, st));
    return DW_OK;
}

}  // namespace dwk
