// Small dense complex FP64 routines of the outer FGMRES-DR loop (host side).
#pragma once

#include <complex>
#include <vector>

namespace dwk {

typedef std::complex<double> zd;

// QR of a growing least-squares matrix by Givens rotations (Sec. 5.2, 5.6):
// columns are added one at a time; the leading block of a deflated cycle may
// be full (non-Hessenberg), later columns have one subdiagonal entry.
// residual() = || c - Hhat eta || for the least-squares eta of the columns so far.
struct GivensLS {
    struct Rot {
        int i;
        double c;
        zd s;
    };
    int rows = 0, ld = 0, ncols = 0;
    std::vector<zd> R, g;
    std::vector<Rot> rots;
    void reset(const zd* c, int nrows, int ncols_max);
    double add_column(const zd* h, int nz_rows);  // h: rows 0..nz_rows-1 of the new column
    double residual() const;
    void solve(zd* eta) const;  // eta[0..ncols-1]
};

// Solves A x = b (A row-major n x n, copied), result in b. 0 on success.
int lu_solve(int n, std::vector<zd> A, zd* b);

// All eigenpairs of the n x n row-major matrix A: lam[k], eigenvector k in
// column k of vecs (row-major, unit 2-norm). 0 on success.
int eig(int n, const zd* A, zd* lam, zd* vecs);

// Thin QR of G (rows x cols, row-major) by Gram-Schmidt with one
// reorthogonalisation: Q (rows x cols, row-major), R (cols x cols, optional),
// diag(R) real and positive. Returns -1 if G is rank deficient.
int qr_positive(int rows, int cols, const zd* G, zd* Q, zd* R);

}  // namespace dwk
