// Small dense complex FP64 linear algebra for the outer FGMRES-DR loop
// (host side; matrices are at most (m+1) x m with m <= 63):
//   * Givens-updated QR of the (generalised) Hessenberg matrix giving the
//     implicit residual norm and the least-squares coefficients (Sec. 5.2, 5.6),
//   * LU solve with partial pivoting (for H_m^H f_m = h_m, Lemma 1a),
//   * the complex eigenproblem of H_m + f_m h_m^H (Lemma 1a): Householder
//     reduction to Hessenberg form, shifted QR iteration to Schur form,
//     eigenvectors by back substitution,
//   * QR of G_{k+1} by Gram-Schmidt with reorthogonalisation and a real
//     positive diagonal of R (Eq. "G_kplus1").
#include "dense.h"

#include <algorithm>
#include <cmath>
#include <numeric>

namespace dwk {

namespace {
const double kEps = 2.220446049250313e-16;
}

// ---------------------------------------------------------------------------
void GivensLS::reset(const zd* c, int nrows, int ncols_max) {
    rows = nrows;
    R.assign((size_t)nrows * ncols_max, zd(0));
    ld = ncols_max;
    g.assign(c, c + nrows);
    rots.clear();
    ncols = 0;
}

// Rotation G = [[c, s], [-conj(s), c]] with G [x; y] = [rho; 0].
static void make_rot(zd x, zd y, double& c, zd& s, zd& rho) {
    const double ax = std::abs(x), ay = std::abs(y);
    if (ay == 0.0) {
        c = 1.0;
        s = 0.0;
        rho = x;
        return;
    }
    if (ax == 0.0) {
        c = 0.0;
        s = 1.0;
        rho = y;
        return;
    }
    const double nrm = std::hypot(ax, ay);
    const zd ph = x / ax;
    c = ax / nrm;
    s = ph * std::conj(y) / nrm;
    rho = ph * nrm;
}

static void apply_rot(double c, zd s, zd& a, zd& b) {
    const zd t1 = c * a + s * b;
    const zd t2 = -std::conj(s) * a + c * b;
    a = t1;
    b = t2;
}

double GivensLS::add_column(const zd* h, int nz_rows) {
    const int j = ncols;
    std::vector<zd> col(rows, zd(0));
    for (int i = 0; i < nz_rows && i < rows; ++i) col[i] = h[i];
    for (const Rot& r : rots) apply_rot(r.c, r.s, col[r.i], col[r.i + 1]);
    int last = std::max(nz_rows - 1, j);
    for (int i = rows - 1; i > last; --i)
        if (col[i] != zd(0)) last = i;
    for (int i = last - 1; i >= j; --i) {
        Rot r;
        r.i = i;
        zd rho;
        make_rot(col[i], col[i + 1], r.c, r.s, rho);
        col[i] = rho;
        col[i + 1] = 0.0;
        apply_rot(r.c, r.s, g[i], g[i + 1]);
        rots.push_back(r);
    }
    for (int i = 0; i <= j; ++i) R[(size_t)i * ld + j] = col[i];
    ncols = j + 1;
    return residual();
}

double GivensLS::residual() const {
    double s = 0.0;
    for (int i = ncols; i < rows; ++i) s += std::norm(g[i]);
    return std::sqrt(s);
}

void GivensLS::solve(zd* eta) const {
    for (int i = ncols - 1; i >= 0; --i) {
        zd acc = g[i];
        for (int k = i + 1; k < ncols; ++k) acc -= R[(size_t)i * ld + k] * eta[k];
        eta[i] = acc / R[(size_t)i * ld + i];
    }
}

// ---------------------------------------------------------------------------
int lu_solve(int n, std::vector<zd> A, zd* b) {
    for (int k = 0; k < n; ++k) {
        int piv = k;
        double best = std::abs(A[(size_t)k * n + k]);
        for (int i = k + 1; i < n; ++i) {
            const double v = std::abs(A[(size_t)i * n + k]);
            if (v > best) best = v, piv = i;
        }
        if (best == 0.0) return -1;
        if (piv != k) {
            for (int j = 0; j < n; ++j) std::swap(A[(size_t)k * n + j], A[(size_t)piv * n + j]);
            std::swap(b[k], b[piv]);
        }
        for (int i = k + 1; i < n; ++i) {
            const zd f = A[(size_t)i * n + k] / A[(size_t)k * n + k];
            if (f == zd(0)) continue;
            for (int j = k; j < n; ++j) A[(size_t)i * n + j] -= f * A[(size_t)k * n + j];
            b[i] -= f * b[k];
        }
    }
    for (int i = n - 1; i >= 0; --i) {
        zd acc = b[i];
        for (int j = i + 1; j < n; ++j) acc -= A[(size_t)i * n + j] * b[j];
        b[i] = acc / A[(size_t)i * n + i];
    }
    return 0;
}

// ---------------------------------------------------------------------------
// Householder reduction A = Q H Q^H (A row-major n x n, overwritten by H).
static void hessenberg(int n, std::vector<zd>& A, std::vector<zd>& Q) {
    Q.assign((size_t)n * n, zd(0));
    for (int i = 0; i < n; ++i) Q[(size_t)i * n + i] = 1.0;
    std::vector<zd> v(n);
    for (int k = 0; k + 2 < n; ++k) {
        const int m = n - k - 1;
        double xn = 0.0;
        for (int i = 0; i < m; ++i) xn += std::norm(A[(size_t)(k + 1 + i) * n + k]);
        xn = std::sqrt(xn);
        if (xn == 0.0) continue;
        const zd x0 = A[(size_t)(k + 1) * n + k];
        const zd ph = (std::abs(x0) > 0.0) ? x0 / std::abs(x0) : zd(1.0);
        const zd alpha = -ph * xn;
        for (int i = 0; i < m; ++i) v[i] = A[(size_t)(k + 1 + i) * n + k];
        v[0] -= alpha;
        double vn = 0.0;
        for (int i = 0; i < m; ++i) vn += std::norm(v[i]);
        vn = std::sqrt(vn);
        if (vn == 0.0) continue;
        for (int i = 0; i < m; ++i) v[i] /= vn;
        // A <- P A with P = I - 2 v v^H on rows k+1..n-1
        for (int j = 0; j < n; ++j) {
            zd d = 0.0;
            for (int i = 0; i < m; ++i) d += std::conj(v[i]) * A[(size_t)(k + 1 + i) * n + j];
            for (int i = 0; i < m; ++i) A[(size_t)(k + 1 + i) * n + j] -= 2.0 * v[i] * d;
        }
        // A <- A P and Q <- Q P on columns k+1..n-1
        for (int i = 0; i < n; ++i) {
            zd d = 0.0, e = 0.0;
            for (int l = 0; l < m; ++l) {
                d += A[(size_t)i * n + k + 1 + l] * v[l];
                e += Q[(size_t)i * n + k + 1 + l] * v[l];
            }
            for (int l = 0; l < m; ++l) {
                A[(size_t)i * n + k + 1 + l] -= 2.0 * d * std::conj(v[l]);
                Q[(size_t)i * n + k + 1 + l] -= 2.0 * e * std::conj(v[l]);
            }
        }
        for (int i = 1; i < m; ++i) A[(size_t)(k + 1 + i) * n + k] = 0.0;
    }
}

// Shifted QR iteration on Hessenberg H to upper-triangular Schur form,
// accumulating the unitary transformations into Z (A = Z T Z^H).
static int schur(int n, std::vector<zd>& H, std::vector<zd>& Z) {
    int hi = n - 1;
    int iter = 0, total = 0;
    while (hi > 0) {
        int l = hi;
        for (; l > 0; --l) {
            const double sub = std::abs(H[(size_t)l * n + l - 1]);
            const double dia = std::abs(H[(size_t)(l - 1) * n + l - 1]) + std::abs(H[(size_t)l * n + l]);
            if (sub <= kEps * (dia > 0.0 ? dia : 1.0)) {
                H[(size_t)l * n + l - 1] = 0.0;
                break;
            }
        }
        if (l == hi) {
            --hi;
            iter = 0;
            continue;
        }
        if (++total > 60 * n) return -1;
        ++iter;
        // Wilkinson shift from the trailing 2x2 block of the active window
        const zd a = H[(size_t)(hi - 1) * n + hi - 1], b = H[(size_t)(hi - 1) * n + hi];
        const zd c = H[(size_t)hi * n + hi - 1], d = H[(size_t)hi * n + hi];
        const zd tr2 = 0.5 * (a + d);
        const zd disc = std::sqrt(0.25 * (a - d) * (a - d) + b * c);
        const zd mu1 = tr2 + disc, mu2 = tr2 - disc;
        zd shift = (std::abs(mu1 - d) < std::abs(mu2 - d)) ? mu1 : mu2;
        if (iter % 10 == 0) shift = d + zd(std::abs(c), 0.5 * std::abs(c));  // exceptional shift
        // implicit single-shift QR sweep on rows/columns l..hi
        zd x = H[(size_t)l * n + l] - shift;
        zd y = H[(size_t)(l + 1) * n + l];
        for (int k = l; k < hi; ++k) {
            double cr;
            zd s, rho;
            make_rot(x, y, cr, s, rho);
            const int j0 = (k > l) ? k - 1 : l;
            for (int j = j0; j < n; ++j) apply_rot(cr, s, H[(size_t)k * n + j], H[(size_t)(k + 1) * n + j]);
            const int i1 = std::min(k + 2, hi);
            for (int i = 0; i <= i1; ++i) {
                const zd h1 = H[(size_t)i * n + k], h2 = H[(size_t)i * n + k + 1];
                H[(size_t)i * n + k] = cr * h1 + std::conj(s) * h2;
                H[(size_t)i * n + k + 1] = -s * h1 + cr * h2;
            }
            for (int i = 0; i < n; ++i) {
                const zd z1 = Z[(size_t)i * n + k], z2 = Z[(size_t)i * n + k + 1];
                Z[(size_t)i * n + k] = cr * z1 + std::conj(s) * z2;
                Z[(size_t)i * n + k + 1] = -s * z1 + cr * z2;
            }
            if (k + 1 < hi) {
                x = H[(size_t)(k + 1) * n + k];
                y = H[(size_t)(k + 2) * n + k];
            }
        }
    }
    return 0;
}

int eig(int n, const zd* A, zd* lam, zd* vecs) {
    std::vector<zd> H(A, A + (size_t)n * n), Z;
    hessenberg(n, H, Z);
    if (schur(n, H, Z) != 0) return -1;
    double tn = 0.0;
    for (size_t i = 0; i < H.size(); ++i) tn = std::max(tn, std::abs(H[i]));
    const double small = (tn > 0.0 ? tn : 1.0) * kEps;
    for (int k = 0; k < n; ++k) lam[k] = H[(size_t)k * n + k];
    std::vector<zd> y(n);
    for (int k = 0; k < n; ++k) {
        std::fill(y.begin(), y.end(), zd(0));
        y[k] = 1.0;
        for (int i = k - 1; i >= 0; --i) {
            zd acc = 0.0;
            for (int j = i + 1; j <= k; ++j) acc += H[(size_t)i * n + j] * y[j];
            zd den = H[(size_t)i * n + i] - lam[k];
            if (std::abs(den) < small) den = small;
            y[i] = -acc / den;
        }
        double nrm = 0.0;
        for (int i = 0; i < n; ++i) {
            zd acc = 0.0;
            for (int j = 0; j <= k; ++j) acc += Z[(size_t)i * n + j] * y[j];
            vecs[(size_t)i * n + k] = acc;
            nrm += std::norm(acc);
        }
        nrm = std::sqrt(nrm);
        for (int i = 0; i < n; ++i) vecs[(size_t)i * n + k] /= nrm;
    }
    return 0;
}

// ---------------------------------------------------------------------------
int qr_positive(int rows, int cols, const zd* G, zd* Q, zd* R) {
    std::vector<zd> q(rows);
    for (int c = 0; c < cols; ++c) {
        for (int i = 0; i < rows; ++i) q[i] = G[(size_t)i * cols + c];
        if (R)
            for (int i = 0; i < cols; ++i) R[(size_t)i * cols + c] = 0.0;
        for (int pass = 0; pass < 2; ++pass)
            for (int p = 0; p < c; ++p) {
                zd d = 0.0;
                for (int i = 0; i < rows; ++i) d += std::conj(Q[(size_t)i * cols + p]) * q[i];
                for (int i = 0; i < rows; ++i) q[i] -= d * Q[(size_t)i * cols + p];
                if (R) R[(size_t)p * cols + c] += d;
            }
        double nrm = 0.0;
        for (int i = 0; i < rows; ++i) nrm += std::norm(q[i]);
        nrm = std::sqrt(nrm);
        if (nrm == 0.0) return -1;
        if (R) R[(size_t)c * cols + c] = nrm;
        for (int i = 0; i < rows; ++i) Q[(size_t)i * cols + c] = q[i] / nrm;
    }
    return 0;
}

}  // namespace dwk
