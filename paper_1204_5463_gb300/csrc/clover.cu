// Clover term of the improved Wilson operator (the Sheikholeslami-Wohlert
// term of the operators in Sec. 6; the paper cites it without a formula):
//   A_n = c_sw (i/2) sum_{mu<nu} sigma_{mu nu} (x) F_{mu nu}(n),
//   F_{mu nu}(n) = (Q - Q^dagger)/8 made traceless, Q = sum of the four
//   plaquettes in the (mu, nu) plane that start and end at n (same sense),
//   sigma_{mu nu} = (i/2)[gamma_mu, gamma_nu].
// In the chiral basis sigma_{mu nu} is block diagonal in the spin pairs
// (0,1) and (2,3): for spatial j < k with l the third spatial direction,
// sigma_{jk} = -eps_{jkl} diag(s_l, s_l); sigma_{j4} = diag(s_j, -s_j)
// (s the Pauli matrices). So A_n is two hermitian 6x6 blocks, computed here
// once per gauge field in FP64 and stored packed (see common.cuh).
#include "internal.h"

namespace dwk {

namespace {

// c = op(a) op(b), 3x3 complex, op = dagger when the flag is set
__device__ void m3(const cx<double>* a, bool da, const cx<double>* b, bool db, cx<double>* c) {
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) {
            cx<double> acc = czero<double>();
            for (int k = 0; k < 3; ++k) {
                const cx<double> x = da ? conj(a[3 * k + i]) : a[3 * i + k];
                const cx<double> y = db ? conj(b[3 * j + k]) : b[3 * k + j];
                acc = acc + x * y;
            }
            c[3 * i + j] = acc;
        }
}

__device__ long long shifted(const Geom& g, const int x[4], int mu, int a, int nu, int b) {
    int y[4] = {x[0], x[1], x[2], x[3]};
    y[mu] = (y[mu] + a + g.d[mu]) % g.d[mu];
    y[nu] = (y[nu] + b + g.d[nu]) % g.d[nu];
    return site_index(g, y);
}

// leaf = l0 l1 l2 l3 with daggers as flagged (links U_{site, dir})
__device__ void leaf(const char* U, long long V, const long long site[4], const int dir[4], const bool dag[4],
                     cx<double>* out) {
    cx<double> u[4][9], t1[9], t2[9];
    for (int q = 0; q < 4; ++q) load_link<P64, double>(U, V, dir[q], site[q], u[q]);
    m3(u[0], dag[0], u[1], dag[1], t1);
    m3(t1, false, u[2], dag[2], t2);
    m3(t2, false, u[3], dag[3], out);
}

// 2x2 spin block of sigma_{mu nu} for chirality chi (0: spins 0,1; 1: spins 2,3)
__device__ void sigma_block(int mu, int nu, int chi, cx<double> s[2][2]) {
    // Pauli matrices s_x, s_y, s_z
    const cx<double> o = mk<double>(1, 0), z = mk<double>(0, 0), i1 = mk<double>(0, 1), mi = mk<double>(0, -1),
                     mo = mk<double>(-1, 0);
    cx<double> P[3][2][2] = {{{z, o}, {o, z}}, {{z, mi}, {i1, z}}, {{o, z}, {z, mo}}};
    int l;
    double f;
    if (nu == 3) {  // sigma_{j4} = diag(s_j, -s_j)
        l = mu;
        f = chi == 0 ? 1.0 : -1.0;
    } else {  // sigma_{jk} = -eps_{jkl} diag(s_l, s_l), j < k spatial
        l = 3 - mu - nu;
        const int eps = (mu == 0 && nu == 1) ? 1 : (mu == 0 && nu == 2) ? -1 : 1;  // eps_{012}, eps_{021}, eps_{120}
        f = -(double)eps;
    }
    for (int a = 0; a < 2; ++a)
        for (int b = 0; b < 2; ++b) s[a][b] = f * P[l][a][b];
}

__global__ void clover_compute_kernel(Geom g, const char* __restrict__ U64, double csw, double* __restrict__ A64,
                                      float4* __restrict__ A32) {
    const long long s = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= g.V) return;
    int x[4];
    site_coords(g, s, x);
    cx<double> B[2][6][6];
    for (int c = 0; c < 2; ++c)
        for (int i = 0; i < 6; ++i)
            for (int j = 0; j < 6; ++j) B[c][i][j] = czero<double>();
    for (int mu = 0; mu < 4; ++mu)
        for (int nu = mu + 1; nu < 4; ++nu) {
            const long long pm = shifted(g, x, mu, 1, nu, 0), mm = shifted(g, x, mu, -1, nu, 0);
            const long long pn = shifted(g, x, mu, 0, nu, 1), mn = shifted(g, x, mu, 0, nu, -1);
            const long long mp = shifted(g, x, mu, -1, nu, 1), mmn = shifted(g, x, mu, -1, nu, -1);
            const long long pmn = shifted(g, x, mu, 1, nu, -1);
            cx<double> Q[9], t[9];
            {
                const long long st[4] = {s, pm, pn, s};
                const int d[4] = {mu, nu, mu, nu};
                const bool dg[4] = {false, false, true, true};
                leaf(U64, g.V, st, d, dg, Q);
            }
            {
                const long long st[4] = {s, mp, mm, mm};
                const int d[4] = {nu, mu, nu, mu};
                const bool dg[4] = {false, true, true, false};
                leaf(U64, g.V, st, d, dg, t);
                for (int i = 0; i < 9; ++i) Q[i] = Q[i] + t[i];
            }
            {
                const long long st[4] = {mm, mmn, mmn, mn};
                const int d[4] = {mu, nu, mu, nu};
                const bool dg[4] = {true, true, false, false};
                leaf(U64, g.V, st, d, dg, t);
                for (int i = 0; i < 9; ++i) Q[i] = Q[i] + t[i];
            }
            {
                const long long st[4] = {mn, mn, pmn, s};
                const int d[4] = {nu, mu, nu, mu};
                const bool dg[4] = {true, false, false, true};
                leaf(U64, g.V, st, d, dg, t);
                for (int i = 0; i < 9; ++i) Q[i] = Q[i] + t[i];
            }
            cx<double> F[9];
            for (int i = 0; i < 3; ++i)
                for (int j = 0; j < 3; ++j) F[3 * i + j] = 0.125 * (Q[3 * i + j] - conj(Q[3 * j + i]));
            const cx<double> tr = (1.0 / 3.0) * (F[0] + F[4] + F[8]);
            for (int i = 0; i < 3; ++i) F[4 * i] = F[4 * i] - tr;
            // B^chi += (csw/2) i s^chi (x) F
            for (int chi = 0; chi < 2; ++chi) {
                cx<double> sg[2][2];
                sigma_block(mu, nu, chi, sg);
                for (int a = 0; a < 2; ++a)
                    for (int b = 0; b < 2; ++b) {
                        const cx<double> f = (0.5 * csw) * ti(sg[a][b]);
                        for (int i = 0; i < 3; ++i)
                            for (int j = 0; j < 3; ++j) B[chi][3 * a + i][3 * b + j] = B[chi][3 * a + i][3 * b + j] + f * F[3 * i + j];
                    }
            }
        }
    // packed: 6 real diagonal entries, then the 15 upper entries as (re, im)
    for (int chi = 0; chi < 2; ++chi) {
        double r[36];
        for (int i = 0; i < 6; ++i) r[i] = B[chi][i][i].re;
        int k = 6;
        for (int i = 0; i < 6; ++i)
            for (int j = i + 1; j < 6; ++j) {
                r[k++] = B[chi][i][j].re;
                r[k++] = B[chi][i][j].im;
            }
        for (int q = 0; q < 36; ++q) A64[(long long)(36 * chi + q) * g.V + s] = r[q];
        for (int q = 0; q < 9; ++q)
            A32[(long long)(9 * chi + q) * g.V + s] =
                make_float4((float)r[4 * q], (float)r[4 * q + 1], (float)r[4 * q + 2], (float)r[4 * q + 3]);
    }
}

}  // namespace

int launch_clover_compute(const Geom& g, const char* U64, double csw, double* A64, float4* A32, cudaStream_t st) {
    const int T = 128;
    clover_compute_kernel<<<(unsigned)((g.V + T - 1) / T), T, 0, st>>>(g, U64, csw, A64, A32);
    DW_LAUNCH_CHECK();
    return DW_OK;
}

}  // namespace dwk
