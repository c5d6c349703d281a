/*
 * dwsolve_dense.h -- host-only small dense routines of the FGMRES-DR outer
 * loop, exported from the same library as dwsolve.h so that they can be
 * checked on a machine without a GPU. None of them touches the device.
 *
 * All matrices are complex FP64, row-major, complex numbers interleaved
 * (re, im). Buffers are owned by the caller. Return DW_OK (0) or a DW_E* code
 * from dwsolve.h; dw_last_error() describes the failure.
 */
#ifndef DWSOLVE_DENSE_H
#define DWSOLVE_DENSE_H

#ifdef __cplusplus
extern "C" {
#endif

/* All eigenpairs of the n x n matrix A (the harmonic Ritz problem
 * H_m + f_m h_m^H of Lemma 1a): Householder reduction to Hessenberg form,
 * shifted QR iteration to Schur form, eigenvectors by back substitution.
 * lam: n complex; vecs: n x n, eigenvector k in column k, unit 2-norm.
 * DW_EBREAKDOWN if the QR iteration does not converge. */
int dw_dense_eig(int n, const double* A, double* lam, double* vecs);

/* Thin QR G = Q R of a rows x cols matrix (rows >= cols) by Gram-Schmidt with
 * one reorthogonalisation, R with a real positive diagonal (the QR of
 * G_{k+1}, Eq. "G_kplus1"). Q: rows x cols; R: cols x cols or NULL.
 * DW_EBREAKDOWN if G is rank deficient. */
int dw_dense_qr(int rows, int cols, const double* G, double* Q, double* R);

/* Least squares min || c - H eta || for a rows x cols H (rows >= cols + 1)
 * whose first dense_rows - 1 columns may be full in rows 0..dense_rows-1 and
 * whose later columns j have nonzeros in rows 0..j+1 (the matrix of a
 * deflated cycle, Sec. 5.5; dense_rows = 1 gives plain upper Hessenberg), by
 * Givens rotations added column by column (Sec. 5.2, 5.6).
 * eta: cols complex; residual[j] = least-squares residual norm using columns
 * 0..j (the implicit residual after step j). */
int dw_dense_lstsq(int rows, int cols, int dense_rows, const double* H, const double* c, double* eta,
                   double* residual);

/* Solve A x = b (n x n, Gaussian elimination with partial pivoting);
 * b is overwritten by x. DW_EBREAKDOWN if A is singular. */
int dw_dense_solve(int n, const double* A, double* b);

#ifdef __cplusplus
}
#endif

#endif /* DWSOLVE_DENSE_H */
