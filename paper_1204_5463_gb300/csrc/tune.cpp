// Domain-tile autotuner. The SAP block shape changes the preconditioner (and
// so the iteration count) as well as the cost of a sweep, so candidates are
// ranked by the time to solution of a calibration solve, not by sweep time.
// Candidates: b_j divides d_j with d_j / b_j even (red-black colouring,
// Sec. 2), block volume within [32, 1024] sites, aspect ratio <= 2, SAP
// shared memory within the per-CTA limit; the twelve closest to 256 sites are
// timed. Results are cached per lattice, right-hand-side count, precisions and
// solver parameters.
#include <algorithm>
#include <cmath>
#include <chrono>
#include <cstring>
#include <map>
#include <mutex>
#include <tuple>
#include <vector>

#include "internal.h"

namespace {

using Key = std::tuple<int, int, int, int, int, int, int, int, int, int, int>;

std::mutex g_mu;
std::map<Key, std::vector<int>> g_cache;
// (cycles, mr) per lattice, block, rhs count, precisions, m and k
using SapKey = std::tuple<int, int, int, int, int, int, int, int, int, int, int, int, int>;
std::map<SapKey, std::vector<int>> g_sap_cache;

Key make_key(const dw_lattice* L, const dw_solver_params* P) {
    return Key(L->dims[0], L->dims[1], L->dims[2], L->dims[3], P->nrhs, (int)P->sap_prec, (int)P->outer_prec, P->m,
               P->k, P->sap_cycles, P->mr_steps);
}

std::vector<std::vector<int>> candidates(const int* dims, int sap_prec) {
    std::vector<int> opt[4];
    for (int j = 0; j < 4; ++j)
        for (int b = 1; b <= dims[j] / 2; ++b)
            if (dims[j] % b == 0 && (dims[j] / b) % 2 == 0) opt[j].push_back(b);
    std::vector<std::vector<int>> out;
    for (int a : opt[0])
        for (int b : opt[1])
            for (int c : opt[2])
                for (int d : opt[3]) {
                    const int vol = a * b * c * d;
                    const int mx = std::max(std::max(a, b), std::max(c, d));
                    const int mn = std::min(std::min(a, b), std::min(c, d));
                    if (vol < 32 || vol > 1024 || mx > 2 * mn) continue;
                    dwk::Geom g{};
                    g.B = vol;
                    const int threads = ((vol + 31) / 32) * 32;
                    if (dwk::sap_smem_bytes(sap_prec, sap_prec, g, threads) > 227 * 1024) continue;
                    out.push_back({a, b, c, d});
                }
    // time only the twelve candidates closest to 256-site domains (the
    // natural size of a one-thread-per-site CTA), most isotropic first
    auto cost = [](const std::vector<int>& v) {
        const double vol = (double)v[0] * v[1] * v[2] * v[3];
        const int mx = std::max(std::max(v[0], v[1]), std::max(v[2], v[3]));
        const int mn = std::min(std::min(v[0], v[1]), std::min(v[2], v[3]));
        return std::abs(std::log2(vol / 256.0)) + 0.1 * (double)mx / mn;
    };
    std::stable_sort(out.begin(), out.end(), [&](const std::vector<int>& x, const std::vector<int>& y) {
        return cost(x) < cost(y);
    });
    if (out.size() > 12) out.resize(12);
    return out;
}

}  // namespace

using namespace dwk;

extern "C" int dw_autotune_block(const dw_lattice* L, const double* U, const double* b, const dw_solver_params* P,
                                 void* cuda_stream, int* best_block, dw_tune_entry* results, int max_results,
                                 int* n_results) {
    if (!L || !U || !b || !P || !best_block) return fail(DW_EINVAL, "null argument");
    long long V = 0;
    if (!lattice_volume(L->dims, kMaxSites, &V)) return fail(DW_EINVAL, "bad lattice extents");
    const Key key = make_key(L, P);
    {
        std::lock_guard<std::mutex> lock(g_mu);
        auto it = g_cache.find(key);
        if (it != g_cache.end() && !results) {
            std::memcpy(best_block, it->second.data(), 4 * sizeof(int));
            if (n_results) *n_results = 0;
            return DW_OK;
        }
    }
    const auto cands = candidates(L->dims, (int)P->sap_prec);
    if (cands.empty()) return fail(DW_EINVAL, "no admissible domain block for this lattice");
    cudaStream_t st = reinterpret_cast<cudaStream_t>(cuda_stream);
    DevBuf x;
    x.st = st;
    int rc = x.ensure((size_t)P->nrhs * 24 * V * sizeof(double));
    if (rc) return rc;
    dw_solver_params Q = *P;
    Q.host_buffers = 0;
    Q.use_x0 = 0;
    double best = 1e300;
    int cnt = 0;
    for (const auto& c : cands) {
        dw_lattice Lc = *L;
        for (int j = 0; j < 4; ++j) Lc.block[j] = c[j];
        dw_ctx* ctx = nullptr;
        if ((rc = dw_create(&Lc, cuda_stream, &ctx))) return rc;
        double secs = 1e300;
        int iters = 0, status = DW_OK;
        rc = dw_set_gauge(ctx, U, 1);
        if (rc == DW_OK) {
            dw_stats S{};
            const auto t0 = std::chrono::steady_clock::now();
            status = fgmresdr_solve(ctx, b, x.as<double>(), &Q, &S);
            secs = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
            iters = S.iterations;
            if (status != DW_OK) secs = 1e300;  // a tile that does not converge never wins
        }
        dw_destroy(ctx);
        if (rc) return rc;
        if (results && cnt < max_results) {
            std::memcpy(results[cnt].block, c.data(), 4 * sizeof(int));
            results[cnt].seconds = secs;
            results[cnt].iterations = iters;
            results[cnt].status = status;
        }
        ++cnt;
        if (secs < best) {
            best = secs;
            std::memcpy(best_block, c.data(), 4 * sizeof(int));
        }
    }
    if (n_results) *n_results = cnt;
    if (best >= 1e300) return fail(DW_ENOTCONV, "no candidate block converged");
    std::lock_guard<std::mutex> lock(g_mu);
    g_cache[key] = std::vector<int>(best_block, best_block + 4);
    return DW_OK;
}

// SAP work per preconditioner application: more cycles and MR steps make each
// Arnoldi step dearer and (up to a point) the solve shorter, and the balance
// moves with the cost of a sweep relative to the Gram-Schmidt passes (e.g.
// many right-hand sides in 16-bit storage make sweeps cheap per rhs). The
// pairs of a small grid are ranked by the time to solution of a calibration
// solve on the caller's block.
extern "C" int dw_autotune_sap(const dw_lattice* L, const double* U, const double* b, const dw_solver_params* P,
                               void* cuda_stream, int* best_cycles, int* best_mr, dw_tune_sap_entry* results,
                               int max_results, int* n_results) {
    if (!L || !U || !b || !P || !best_cycles || !best_mr) return fail(DW_EINVAL, "null argument");
    long long V = 0;
    if (!lattice_volume(L->dims, kMaxSites, &V)) return fail(DW_EINVAL, "bad lattice extents");
    const SapKey key(L->dims[0], L->dims[1], L->dims[2], L->dims[3], L->block[0], L->block[1], L->block[2],
                     L->block[3], P->nrhs, (int)P->sap_prec, (int)P->outer_prec, P->m, P->k);
    {
        std::lock_guard<std::mutex> lock(g_mu);
        auto it = g_sap_cache.find(key);
        if (it != g_sap_cache.end() && !results) {
            *best_cycles = it->second[0];
            *best_mr = it->second[1];
            if (n_results) *n_results = 0;
            return DW_OK;
        }
    }
    static const int kCycles[] = {2, 3, 4, 5, 6, 8};
    static const int kMr[] = {3, 4, 5, 6, 8, 10};
    cudaStream_t st = reinterpret_cast<cudaStream_t>(cuda_stream);
    DevBuf x;
    x.st = st;
    int rc = x.ensure((size_t)P->nrhs * 24 * V * sizeof(double));
    if (rc) return rc;
    dw_ctx* ctx = nullptr;
    if ((rc = dw_create(L, cuda_stream, &ctx))) return rc;
    if ((rc = dw_set_gauge(ctx, U, 1))) {
        dw_destroy(ctx);
        return rc;
    }
    dw_solver_params Q = *P;
    Q.host_buffers = 0;
    Q.use_x0 = 0;
    {  // warm-up: workspace, link copies and images for this block
        dw_stats S{};
        fgmresdr_solve(ctx, b, x.as<double>(), &Q, &S);
    }
    double best = 1e300;
    int cnt = 0;
    for (int c : kCycles)
        for (int mr : kMr) {
            Q.sap_cycles = c;
            Q.mr_steps = mr;
            dw_stats S{};
            const auto t0 = std::chrono::steady_clock::now();
            const int status = fgmresdr_solve(ctx, b, x.as<double>(), &Q, &S);
            double secs = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
            if (status != DW_OK) secs = 1e300;
            if (results && cnt < max_results) {
                results[cnt].sap_cycles = c;
                results[cnt].mr_steps = mr;
                results[cnt].seconds = secs;
                results[cnt].iterations = S.iterations;
                results[cnt].status = status;
            }
            ++cnt;
            if (secs < best) {
                best = secs;
                *best_cycles = c;
                *best_mr = mr;
            }
            if (status == DW_ECUDA || status == DW_ETIMEOUT) {
                dw_destroy(ctx);
                if (n_results) *n_results = cnt;
                return status;
            }
        }
    dw_destroy(ctx);
    if (n_results) *n_results = cnt;
    if (best >= 1e300) return fail(DW_ENOTCONV, "no SAP setting converged");
    std::lock_guard<std::mutex> lock(g_mu);
    g_sap_cache[key] = std::vector<int>{*best_cycles, *best_mr};
    return DW_OK;
}
