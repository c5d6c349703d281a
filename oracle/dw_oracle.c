/*
 * FP64 CPU oracle for the Wilson-Dirac operator and the SAP preconditioner.
 *
 * TEST INFRASTRUCTURE ONLY. This file is the plain, slow definition of what the
 * GPU path computes; only the tests, the smoke check and the CPU-baseline leg of
 * the benchmark may build, load or run it. It shares no code, header, table or
 * constant with the CUDA library.
 *
 * Conventions (all in double precision, complex interleaved re,im):
 *   site index   n = n1 + d1*(n2 + d2*(n3 + d3*n4))
 *   spinor       psi[site][spin 0..3][colour 0..2]          (12 complex / site)
 *   gauge field  U[site][mu 0..3][row 0..2][col 0..2]        (36 complex / site)
 *
 * Operator (Sec. 2, Eq. "Dw"), written with a bare mass m0 instead of kappa:
 *   (D psi)_n = (4+m0) psi_n
 *               - 1/2 sum_j [ (1+gamma_j) U_{n,j} psi_{n+j}
 *                            + (1-gamma_j) U^dagger_{n-j,j} psi_{n-j} ]
 * which equals D_kappa / (2 kappa) with kappa = 1/(2(4+m0)); n +- j is taken
 * modulo d_j (periodic in all four directions).
 *
 * Local operator (Sec. 2, Eq. "Dw_local"): the same sum restricted to hops
 * whose both ends lie in the same domain L^l (a 4-D box of block[] sites).
 *
 * SAP (Sec. 2, Algorithm 2): domains are coloured by the parity of the sum of
 * their block coordinates; colour 0 (the one containing site 0) is swept first.
 * Each sweep computes r^l = (b - D x)^l with the full operator, approximately
 * solves D^l y^l = r^l, and adds the correction: x^l <- x^l + y^l.
 *
 * Clover term (the Sheikholeslami-Wohlert improvement of the operators in
 * Sec. 6; the paper cites it without a formula, so this is a reading): a
 * site-diagonal 12x12 matrix added to D and to every D^l,
 *   A_n = c_sw (i/2) sum_{mu<nu} sigma_{mu nu} (x) F_{mu nu}(n),
 *   sigma_{mu nu} = (i/2) [gamma_mu, gamma_nu],
 *   F_{mu nu}(n) = (1/8) (Q - Q^dagger) minus its trace / 3,
 * with Q the sum of the four plaquettes in the (mu, nu) plane that start and
 * end at n, all traversed in the same sense (mu first, then nu).
 *
 * Local solver (Sec. 4): nmr steps of minimal residual (MR) from y = 0:
 *   p = D^l rho;  alpha = <p,rho>/<p,p>  (<a,b> = a^H b);  y += alpha rho;
 *   rho -= alpha p.  nmr == 0 selects an exact solve by Gaussian elimination
 *   with partial pivoting (small domains only), used to pin SAP against the
 *   closed series form of the preconditioner (Sec. 4).
 */
#include <complex.h>
#include <math.h>
#include <stdlib.h>
#include <string.h>

typedef double complex cplx;

/* Hermitian Euclidean gamma matrices in a chiral basis:
 *   gamma_k = [[0, -i sigma_k], [i sigma_k, 0]]  (k = 1,2,3)
 *   gamma_4 = [[0, 1], [1, 0]]
 * so that gamma_5 = gamma_1 gamma_2 gamma_3 gamma_4 = diag(1, 1, -1, -1).   */
static const cplx GAMMA[4][4][4] = {
    {{0, 0, 0, -I}, {0, 0, -I, 0}, {0, I, 0, 0}, {I, 0, 0, 0}},
    {{0, 0, 0, -1}, {0, 0, 1, 0}, {0, 1, 0, 0}, {-1, 0, 0, 0}},
    {{0, 0, -I, 0}, {0, 0, 0, I}, {I, 0, 0, 0}, {0, -I, 0, 0}},
    {{0, 0, 1, 0}, {0, 0, 0, 1}, {1, 0, 0, 0}, {0, 1, 0, 0}},
};

/* Exported so that the tests can check the defining relations of the basis. */
void oracle_gamma(int mu, double *out /* 4x4 complex, row-major */) {
    for (int a = 0; a < 4; ++a)
        for (int b = 0; b < 4; ++b) {
            out[2 * (4 * a + b)] = creal(GAMMA[mu][a][b]);
            out[2 * (4 * a + b) + 1] = cimag(GAMMA[mu][a][b]);
        }
}

typedef struct {
    int d[4];
    int blk[4];
    int nb[4]; /* domains per direction */
    long V;
} lattice;

static void make_lattice(lattice *L, const int *dims, const int *block) {
    L->V = 1;
    for (int j = 0; j < 4; ++j) {
        L->d[j] = dims[j];
        L->blk[j] = block ? block[j] : dims[j];
        L->nb[j] = L->d[j] / L->blk[j];
        L->V *= dims[j];
    }
}

static void coords(const lattice *L, long s, int n[4]) {
    for (int j = 0; j < 4; ++j) {
        n[j] = (int)(s % L->d[j]);
        s /= L->d[j];
    }
}

static long index_of(const lattice *L, const int n[4]) {
    return n[0] + (long)L->d[0] * (n[1] + (long)L->d[1] * (n[2] + (long)L->d[2] * n[3]));
}

static long hop(const lattice *L, long s, int mu, int sign) {
    int n[4];
    coords(L, s, n);
    n[mu] = (n[mu] + sign + L->d[mu]) % L->d[mu];
    return index_of(L, n);
}

static long domain_of(const lattice *L, long s) {
    int n[4];
    coords(L, s, n);
    return (n[0] / L->blk[0]) +
           (long)L->nb[0] * ((n[1] / L->blk[1]) + (long)L->nb[1] * ((n[2] / L->blk[2]) + (long)L->nb[2] * (n[3] / L->blk[3])));
}

static int colour_of_domain(const lattice *L, long dom) {
    int sum = 0;
    for (int j = 0; j < 4; ++j) {
        sum += (int)(dom % L->nb[j]);
        dom /= L->nb[j];
    }
    return sum & 1;
}

/* One site of D (all hops) or of the block-diagonal local operator (only hops
 * inside the domain of site s). in/out point at 12-complex spinors.           */
static void apply_site(const lattice *L, double m0, const cplx *U, const cplx *A, const cplx *in, long s,
                       int local, cplx out[12]) {
    const long dom = local ? domain_of(L, s) : -1;
    for (int a = 0; a < 12; ++a) out[a] = (4.0 + m0) * in[12 * s + a];
    if (A) /* clover term: site-diagonal, part of D and of every D^l */
        for (int a = 0; a < 12; ++a)
            for (int b = 0; b < 12; ++b) out[a] += A[144 * s + 12 * a + b] * in[12 * s + b];
    for (int mu = 0; mu < 4; ++mu) {
        for (int sign = +1; sign >= -1; sign -= 2) {
            const long t = hop(L, s, mu, sign);
            if (local && domain_of(L, t) != dom) continue;
            /* chi = U_{s,mu} psi_t (forward) or U^dagger_{t,mu} psi_t (backward) */
            cplx chi[4][3];
            const cplx *link = (sign > 0) ? &U[36 * s + 9 * mu] : &U[36 * t + 9 * mu];
            for (int sp = 0; sp < 4; ++sp)
                for (int a = 0; a < 3; ++a) {
                    cplx acc = 0;
                    for (int b = 0; b < 3; ++b) {
                        const cplx u = (sign > 0) ? link[3 * a + b] : conj(link[3 * b + a]);
                        acc += u * in[12 * t + 3 * sp + b];
                    }
                    chi[sp][a] = acc;
                }
            /* (1 + sign*gamma_mu) chi, scaled by -1/2 */
            for (int sp = 0; sp < 4; ++sp)
                for (int a = 0; a < 3; ++a) {
                    cplx v = chi[sp][a];
                    for (int q = 0; q < 4; ++q) v += (double)sign * GAMMA[mu][sp][q] * chi[q][a];
                    out[3 * sp + a] -= 0.5 * v;
                }
        }
    }
}

/* out = D in, full lattice. */
void oracle_dw_c(const int *dims, double m0, const double *U_, const double *A_, const double *in_, double *out_) {
    lattice L;
    make_lattice(&L, dims, NULL);
    const cplx *U = (const cplx *)U_;
    const cplx *A = (const cplx *)A_;
    const cplx *in = (const cplx *)in_;
    cplx *out = (cplx *)out_;
#pragma omp parallel for schedule(static)
    for (long s = 0; s < L.V; ++s) apply_site(&L, m0, U, A, in, s, 0, &out[12 * s]);
}

void oracle_dw(const int *dims, double m0, const double *U_, const double *in_, double *out_) {
    oracle_dw_c(dims, m0, U_, NULL, in_, out_);
}

/* out = D^l in on every domain of the given colour (colour < 0: all domains);
 * sites outside the selected domains are set to zero.                        */
void oracle_dw_local_c(const int *dims, const int *block, double m0, const double *U_, const double *A_,
                       const double *in_, double *out_, int colour) {
    lattice L;
    make_lattice(&L, dims, block);
    const cplx *U = (const cplx *)U_;
    const cplx *A = (const cplx *)A_;
    const cplx *in = (const cplx *)in_;
    cplx *out = (cplx *)out_;
#pragma omp parallel for schedule(static)
    for (long s = 0; s < L.V; ++s) {
        if (colour >= 0 && colour_of_domain(&L, domain_of(&L, s)) != colour) {
            for (int a = 0; a < 12; ++a) out[12 * s + a] = 0;
            continue;
        }
        apply_site(&L, m0, U, A, in, s, 1, &out[12 * s]);
    }
}

void oracle_dw_local(const int *dims, const int *block, double m0, const double *U_, const double *in_,
                     double *out_, int colour) {
    oracle_dw_local_c(dims, block, m0, U_, NULL, in_, out_, colour);
}

/* Lexicographic list of the sites of domain dom. */
static void domain_sites(const lattice *L, long dom, long *sites) {
    int c[4];
    long t = dom;
    for (int j = 0; j < 4; ++j) {
        c[j] = (int)(t % L->nb[j]);
        t /= L->nb[j];
    }
    long k = 0;
    int n[4];
    for (int x4 = 0; x4 < L->blk[3]; ++x4)
        for (int x3 = 0; x3 < L->blk[2]; ++x3)
            for (int x2 = 0; x2 < L->blk[1]; ++x2)
                for (int x1 = 0; x1 < L->blk[0]; ++x1) {
                    n[0] = c[0] * L->blk[0] + x1;
                    n[1] = c[1] * L->blk[1] + x2;
                    n[2] = c[2] * L->blk[2] + x3;
                    n[3] = c[3] * L->blk[3] + x4;
                    sites[k++] = index_of(L, n);
                }
}

/* Gaussian elimination with partial pivoting: solves A x = rhs (A is N x N,
 * row-major, destroyed; rhs overwritten by x). Returns 0 on success.         */
static int dense_solve(cplx *A, cplx *rhs, int N) {
    for (int k = 0; k < N; ++k) {
        int piv = k;
        double best = cabs(A[(long)k * N + k]);
        for (int i = k + 1; i < N; ++i) {
            const double v = cabs(A[(long)i * N + k]);
            if (v > best) best = v, piv = i;
        }
        if (best == 0.0) return -1;
        if (piv != k) {
            for (int j = 0; j < N; ++j) {
                cplx t = A[(long)k * N + j];
                A[(long)k * N + j] = A[(long)piv * N + j];
                A[(long)piv * N + j] = t;
            }
            cplx t = rhs[k];
            rhs[k] = rhs[piv];
            rhs[piv] = t;
        }
        for (int i = k + 1; i < N; ++i) {
            const cplx f = A[(long)i * N + k] / A[(long)k * N + k];
            if (f == 0) continue;
            for (int j = k; j < N; ++j) A[(long)i * N + j] -= f * A[(long)k * N + j];
            rhs[i] -= f * rhs[k];
        }
    }
    for (int i = N - 1; i >= 0; --i) {
        cplx acc = rhs[i];
        for (int j = i + 1; j < N; ++j) acc -= A[(long)i * N + j] * rhs[j];
        rhs[i] = acc / A[(long)i * N + i];
    }
    return 0;
}

/* Approximate (nmr >= 1: MR) or exact (nmr == 0) solve of D^l y = r on one
 * domain. rho, p are lattice-sized scratch vectors; only this domain's sites
 * are touched, so domains of one colour can be processed concurrently.       */
static int local_solve(const lattice *L, double m0, const cplx *U, const cplx *A, const long *sites, long ns,
                       const cplx *r, cplx *y, cplx *rho, cplx *p, int nmr) {
    if (nmr == 0) {
        const int N = (int)(12 * ns);
        cplx *Dl = (cplx *)calloc((size_t)N * N, sizeof(cplx)); /* dense D^l */
        cplx *x = (cplx *)malloc((size_t)N * sizeof(cplx));
        if (!Dl || !x) {
            free(Dl);
            free(x);
            return -1;
        }
        /* Column c of the dense D^l is D^l applied to the c-th unit vector. */
        for (int c = 0; c < N; ++c) {
            for (long q = 0; q < ns; ++q)
                for (int a = 0; a < 12; ++a) rho[12 * sites[q] + a] = (12 * q + a == c) ? 1.0 : 0.0;
            for (long q = 0; q < ns; ++q) {
                cplx o[12];
                apply_site(L, m0, U, A, rho, sites[q], 1, o);
                for (int a = 0; a < 12; ++a) Dl[(long)(12 * q + a) * N + c] = o[a];
            }
        }
        for (long q = 0; q < ns; ++q)
            for (int a = 0; a < 12; ++a) x[12 * q + a] = r[12 * sites[q] + a];
        const int rc = dense_solve(Dl, x, N);
        for (long q = 0; q < ns; ++q)
            for (int a = 0; a < 12; ++a) y[12 * sites[q] + a] = x[12 * q + a];
        free(Dl);
        free(x);
        return rc;
    }
    for (long q = 0; q < ns; ++q)
        for (int a = 0; a < 12; ++a) {
            y[12 * sites[q] + a] = 0;
            rho[12 * sites[q] + a] = r[12 * sites[q] + a];
        }
    for (int it = 0; it < nmr; ++it) {
        for (long q = 0; q < ns; ++q) apply_site(L, m0, U, A, rho, sites[q], 1, &p[12 * sites[q]]);
        cplx prho = 0;
        double pp = 0;
        for (long q = 0; q < ns; ++q)
            for (int a = 0; a < 12; ++a) {
                const cplx pv = p[12 * sites[q] + a];
                prho += conj(pv) * rho[12 * sites[q] + a];
                pp += creal(conj(pv) * pv);
            }
        if (pp == 0.0) break; /* rho = 0: already solved exactly */
        const cplx alpha = prho / pp;
        for (long q = 0; q < ns; ++q)
            for (int a = 0; a < 12; ++a) {
                y[12 * sites[q] + a] += alpha * rho[12 * sites[q] + a];
                rho[12 * sites[q] + a] -= alpha * p[12 * sites[q] + a];
            }
    }
    return 0;
}

/* SAP iteration (Algorithm 2): ncycles sweeps over colour 0 then colour 1,
 * starting from the x passed in (x is updated in place). Returns 0 on success. */
int oracle_sap_c(const int *dims, const int *block, double m0, const double *U_, const double *A_, const double *b_,
                 double *x_, int ncycles, int nmr) {
    lattice L;
    make_lattice(&L, dims, block);
    const cplx *U = (const cplx *)U_;
    const cplx *A = (const cplx *)A_;
    const cplx *b = (const cplx *)b_;
    cplx *x = (cplx *)x_;
    const long ndom = (long)L.nb[0] * L.nb[1] * L.nb[2] * L.nb[3];
    const long ns = (long)L.blk[0] * L.blk[1] * L.blk[2] * L.blk[3];
    cplx *r = (cplx *)calloc((size_t)L.V * 12, sizeof(cplx));
    cplx *y = (cplx *)calloc((size_t)L.V * 12, sizeof(cplx));
    cplx *rho = (cplx *)calloc((size_t)L.V * 12, sizeof(cplx));
    cplx *p = (cplx *)calloc((size_t)L.V * 12, sizeof(cplx));
    long *sites = (long *)malloc((size_t)ndom * ns * sizeof(long));
    if (!r || !y || !rho || !p || !sites) {
        free(r), free(y), free(rho), free(p), free(sites);
        return -1;
    }
    for (long d = 0; d < ndom; ++d) domain_sites(&L, d, &sites[d * ns]);
    int err = 0;
    for (int cyc = 0; cyc < ncycles; ++cyc) {
        for (int colour = 0; colour < 2; ++colour) {
            /* all domains of this colour: residual and local solve */
#pragma omp parallel for schedule(dynamic) reduction(| : err)
            for (long d = 0; d < ndom; ++d) {
                if (colour_of_domain(&L, d) != colour) continue;
                const long *sd = &sites[d * ns];
                for (long q = 0; q < ns; ++q) {
                    cplx dx[12];
                    apply_site(&L, m0, U, A, x, sd[q], 0, dx);
                    for (int a = 0; a < 12; ++a) r[12 * sd[q] + a] = b[12 * sd[q] + a] - dx[a];
                }
                err |= (local_solve(&L, m0, U, A, sd, ns, r, y, rho, p, nmr) != 0);
            }
            /* update x^l <- x^l + y^l for every domain of this colour */
#pragma omp parallel for schedule(static)
            for (long d = 0; d < ndom; ++d) {
                if (colour_of_domain(&L, d) != colour) continue;
                const long *sd = &sites[d * ns];
                for (long q = 0; q < ns; ++q)
                    for (int a = 0; a < 12; ++a) x[12 * sd[q] + a] += y[12 * sd[q] + a];
            }
        }
    }
    free(r), free(y), free(rho), free(p), free(sites);
    return err ? -2 : 0;
}

int oracle_sap(const int *dims, const int *block, double m0, const double *U_, const double *b_, double *x_,
               int ncycles, int nmr) {
    return oracle_sap_c(dims, block, m0, U_, NULL, b_, x_, ncycles, nmr);
}

/* ---- clover term ---------------------------------------------------------- */

/* c = op(a) op(b) for 3x3 complex matrices; op = dagger when the flag is set */
static void mul3(const cplx *a, int da, const cplx *b, int db, cplx *c) {
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) {
            cplx acc = 0;
            for (int k = 0; k < 3; ++k) {
                const cplx x = da ? conj(a[3 * k + i]) : a[3 * i + k];
                const cplx y = db ? conj(b[3 * j + k]) : b[3 * k + j];
                acc += x * y;
            }
            c[3 * i + j] = acc;
        }
}

/* product of four links, each optionally daggered, left to right */
static void path4(const cplx *l[4], const int dag[4], cplx *out) {
    cplx t1[9], t2[9];
    mul3(l[0], dag[0], l[1], dag[1], t1);
    mul3(t1, 0, l[2], dag[2], t2);
    mul3(t2, 0, l[3], dag[3], out);
}

/* A[site][12][12] (complex) for the clover term with coefficient csw. */
void oracle_clover(const int *dims, double csw, const double *U_, double *A_) {
    lattice L;
    make_lattice(&L, dims, NULL);
    const cplx *U = (const cplx *)U_;
    cplx *A = (cplx *)A_;
#pragma omp parallel for schedule(static)
    for (long s = 0; s < L.V; ++s) {
        cplx a[12][12];
        memset(a, 0, sizeof(a));
        for (int mu = 0; mu < 4; ++mu)
            for (int nu = mu + 1; nu < 4; ++nu) {
                const long pm = hop(&L, s, mu, +1), mm = hop(&L, s, mu, -1);
                const long pn = hop(&L, s, nu, +1), mn = hop(&L, s, nu, -1);
                const long mp = hop(&L, mm, nu, +1);  /* n - mu + nu */
                const long mmn = hop(&L, mm, nu, -1); /* n - mu - nu */
                const long pmn = hop(&L, pm, nu, -1); /* n + mu - nu */
#define LK(site, dir) (&U[36 * (site) + 9 * (dir)])
                /* the four leaves around n, each in the (mu, nu) sense */
                const cplx *l1[4] = {LK(s, mu), LK(pm, nu), LK(pn, mu), LK(s, nu)};
                const int d1[4] = {0, 0, 1, 1};
                const cplx *l2[4] = {LK(s, nu), LK(mp, mu), LK(mm, nu), LK(mm, mu)};
                const int d2[4] = {0, 1, 1, 0};
                const cplx *l3[4] = {LK(mm, mu), LK(mmn, nu), LK(mmn, mu), LK(mn, nu)};
                const int d3[4] = {1, 1, 0, 0};
                const cplx *l4[4] = {LK(mn, nu), LK(mn, mu), LK(pmn, nu), LK(s, mu)};
                const int d4[4] = {1, 0, 0, 1};
#undef LK
                cplx Q[9] = {0}, t[9];
                path4(l1, d1, t);
                for (int i = 0; i < 9; ++i) Q[i] += t[i];
                path4(l2, d2, t);
                for (int i = 0; i < 9; ++i) Q[i] += t[i];
                path4(l3, d3, t);
                for (int i = 0; i < 9; ++i) Q[i] += t[i];
                path4(l4, d4, t);
                for (int i = 0; i < 9; ++i) Q[i] += t[i];
                cplx F[9];
                for (int i = 0; i < 3; ++i)
                    for (int j = 0; j < 3; ++j) F[3 * i + j] = (Q[3 * i + j] - conj(Q[3 * j + i])) / 8.0;
                const cplx tr = (F[0] + F[4] + F[8]) / 3.0;
                for (int i = 0; i < 3; ++i) F[4 * i] -= tr;
                /* sigma_{mu nu} = (i/2)(g_mu g_nu - g_nu g_mu) */
                cplx sig[4][4];
                for (int p = 0; p < 4; ++p)
                    for (int q = 0; q < 4; ++q) {
                        cplx c = 0;
                        for (int k = 0; k < 4; ++k)
                            c += GAMMA[mu][p][k] * GAMMA[nu][k][q] - GAMMA[nu][p][k] * GAMMA[mu][k][q];
                        sig[p][q] = 0.5 * I * c;
                    }
                for (int p = 0; p < 4; ++p)
                    for (int q = 0; q < 4; ++q)
                        for (int i = 0; i < 3; ++i)
                            for (int j = 0; j < 3; ++j)
                                a[3 * p + i][3 * q + j] += 0.5 * csw * I * sig[p][q] * F[3 * i + j];
            }
        for (int i = 0; i < 12; ++i)
            for (int j = 0; j < 12; ++j) A[144 * s + 12 * i + j] = a[i][j];
    }
}

/* Domain colour of every site (0/1), for tests of the red-black structure. */
void oracle_site_colours(const int *dims, const int *block, int *colour_out) {
    lattice L;
    make_lattice(&L, dims, block);
    for (long s = 0; s < L.V; ++s) colour_out[s] = colour_of_domain(&L, domain_of(&L, s));
}

/* Per-step MR residual norms on one colour (for the monotonicity invariant):
 * runs MR on every domain of the colour with right-hand side r and records
 * ||rho||^2 summed over the colour after each step (norms[0] = before).      */
int oracle_mr_history(const int *dims, const int *block, double m0, const double *U_, const double *r_, double *y_,
                      int colour, int nmr, double *norms) {
    lattice L;
    make_lattice(&L, dims, block);
    const cplx *U = (const cplx *)U_;
    const cplx *r = (const cplx *)r_;
    cplx *y = (cplx *)y_;
    const long ndom = (long)L.nb[0] * L.nb[1] * L.nb[2] * L.nb[3];
    const long ns = (long)L.blk[0] * L.blk[1] * L.blk[2] * L.blk[3];
    cplx *rho = (cplx *)calloc((size_t)L.V * 12, sizeof(cplx));
    cplx *p = (cplx *)calloc((size_t)L.V * 12, sizeof(cplx));
    long *sites = (long *)malloc((size_t)ns * sizeof(long));
    if (!rho || !p || !sites) {
        free(rho), free(p), free(sites);
        return -1;
    }
    for (int it = 0; it <= nmr; ++it) norms[it] = 0;
    for (long d = 0; d < ndom; ++d) {
        if (colour_of_domain(&L, d) != colour) continue;
        domain_sites(&L, d, sites);
        for (long q = 0; q < ns; ++q)
            for (int a = 0; a < 12; ++a) norms[0] += creal(conj(r[12 * sites[q] + a]) * r[12 * sites[q] + a]);
        /* MR from y = 0 is deterministic, so running it afresh with 1..nmr
         * steps reproduces the residual after each step.                     */
        for (int it = 1; it <= nmr; ++it) {
            local_solve(&L, m0, U, NULL, sites, ns, r, y, rho, p, it);
            for (long q = 0; q < ns; ++q)
                for (int a = 0; a < 12; ++a)
                    norms[it] += creal(conj(rho[12 * sites[q] + a]) * rho[12 * sites[q] + a]);
        }
    }
    free(rho), free(p), free(sites);
    return 0;
}
