// plan.cpp -- host-side preprocessing (validation, Section 5.2 ordering, the I x J grid of
// Section 3, per-subset observation lists).  Linear-time counting sorts, no allocation per entry.
#include "plan.h"

#include <algorithm>
#include <cmath>
#include <numeric>

#include "bmf.h"

namespace bmf {

int subset_stage(int i, int j)
{
    if (i == 0 && j == 0) return 1;
    if (i == 0 || j == 0) return 2;
    return 3;
}

// New -> original permutation sorting by decreasing count, ties by original index.
static void density_order(const std::vector<int64_t> &cnt, std::vector<int64_t> &perm)
{
    perm.resize(cnt.size());
    std::iota(perm.begin(), perm.end(), 0);
    std::stable_sort(perm.begin(), perm.end(),
                     [&](int64_t a, int64_t b) { return cnt[a] > cnt[b]; });
}

static bool valid_bounds(const int64_t *b, int parts, int64_t n)
{
    if (b[0] != 0 || b[parts] != n) return false;
    for (int k = 0; k < parts; ++k)
        if (b[k + 1] < b[k]) return false;
    return true;
}

// Block index of a reordered position (bounds are nondecreasing; empty blocks allowed).
static int block_of(const std::vector<int64_t> &b, int64_t x)
{
    return (int)(std::upper_bound(b.begin(), b.end(), x) - b.begin()) - 1;
}

int build_plan(int64_t N, int64_t D, int64_t nnz, const int32_t *row, const int32_t *col,
               const double *val, int order, int center, int I, const int64_t *row_bounds,
               int J, const int64_t *col_bounds, int64_t n_test, const int32_t *test_row,
               const int32_t *test_col, const double *test_val, HostPlan &P, std::string &err)
{
    if (N <= 0 || D <= 0 || nnz < 0 || I < 1 || J < 1 || I > N || J > D) {
        err = "bad sizes (need N, D >= 1, 1 <= I <= N, 1 <= J <= D)";
        return BMF_E_ARG;
    }
    if (N > INT32_MAX || D > INT32_MAX) {
        err = "N and D must fit in int32";
        return BMF_E_ARG;
    }
    if (nnz > 0 && (!row || !col || !val)) {
        err = "null training COO";
        return BMF_E_ARG;
    }
    if (n_test > 0 && (!test_row || !test_col || !test_val)) {
        err = "null test COO";
        return BMF_E_ARG;
    }
    P.N = N;
    P.D = D;
    P.nnz = nnz;
    P.I = I;
    P.J = J;
    // validation and counts
    std::vector<int64_t> rc(N, 0), cc(D, 0);
    double sum = 0.0;
    for (int64_t e = 0; e < nnz; ++e) {
        if (row[e] < 0 || row[e] >= N || col[e] < 0 || col[e] >= D) {
            err = "training index out of range at entry " + std::to_string(e);
            return BMF_E_ARG;
        }
        if (!std::isfinite(val[e])) {
            err = "non-finite training value at entry " + std::to_string(e);
            return BMF_E_NONFINITE;
        }
        ++rc[row[e]];
        ++cc[col[e]];
        sum += val[e];
    }
    for (int64_t e = 0; e < n_test; ++e) {
        if (test_row[e] < 0 || test_row[e] >= N || test_col[e] < 0 || test_col[e] >= D) {
            err = "test index out of range at entry " + std::to_string(e);
            return BMF_E_ARG;
        }
        if (!std::isfinite(test_val[e])) {
            err = "non-finite test value at entry " + std::to_string(e);
            return BMF_E_NONFINITE;
        }
    }
    P.offset = (center && nnz > 0) ? sum / (double)nnz : 0.0;
    // ordering (Section 5.2)
    if (order == BMF_ORDER_DECREASING) {
        density_order(rc, P.row_perm);
        density_order(cc, P.col_perm);
    } else if (order == BMF_ORDER_NONE) {
        P.row_perm.resize(N);
        std::iota(P.row_perm.begin(), P.row_perm.end(), 0);
        P.col_perm.resize(D);
        std::iota(P.col_perm.begin(), P.col_perm.end(), 0);
    } else {
        err = "unknown order";
        return BMF_E_ARG;
    }
    P.row_rank.assign(N, 0);
    P.col_rank.assign(D, 0);
    for (int64_t k = 0; k < N; ++k) P.row_rank[P.row_perm[k]] = k;
    for (int64_t k = 0; k < D; ++k) P.col_rank[P.col_perm[k]] = k;
    // grid bounds
    P.row_bounds.resize(I + 1);
    P.col_bounds.resize(J + 1);
    for (int k = 0; k <= I; ++k) P.row_bounds[k] = row_bounds ? row_bounds[k] : (k * N) / I;
    for (int k = 0; k <= J; ++k) P.col_bounds[k] = col_bounds ? col_bounds[k] : (k * D) / J;
    if (!valid_bounds(P.row_bounds.data(), I, N) || !valid_bounds(P.col_bounds.data(), J, D)) {
        err = "row/col bounds must be nondecreasing from 0 to N (D)";
        return BMF_E_SHAPE;
    }
    // subsets and slot order (stage, id)
    int S = I * J;
    P.subs.assign(S, SubsetGeom());
    for (int i = 0; i < I; ++i)
        for (int j = 0; j < J; ++j) {
            SubsetGeom &g = P.subs[i * J + j];
            g.i = i;
            g.j = j;
            g.sid = i * J + j;
            g.stage = subset_stage(i, j);
            g.r0 = P.row_bounds[i];
            g.r1 = P.row_bounds[i + 1];
            g.c0 = P.col_bounds[j];
            g.c1 = P.col_bounds[j + 1];
        }
    P.slot_sid.resize(S);
    std::iota(P.slot_sid.begin(), P.slot_sid.end(), 0);
    std::stable_sort(P.slot_sid.begin(), P.slot_sid.end(),
                     [&](int a, int b) { return P.subs[a].stage < P.subs[b].stage; });
    int64_t xo = 0, wo = 0;
    for (int sl = 0; sl < S; ++sl) {
        SubsetGeom &g = P.subs[P.slot_sid[sl]];
        g.slot = sl;
        g.xoff = xo;
        g.woff = wo;
        xo += g.n();
        wo += g.d();
    }
    P.RX = xo;
    P.RW = wo;
    if (P.RX > INT32_MAX || P.RW > INT32_MAX) {
        err = "arena too large for int32 indices";
        return BMF_E_ARG;
    }
    // per-entry block membership and arena coordinates
    std::vector<int32_t> bi(N), bj(D);
    for (int64_t k = 0; k < N; ++k) bi[k] = block_of(P.row_bounds, k);
    for (int64_t k = 0; k < D; ++k) bj[k] = block_of(P.col_bounds, k);
    auto arena_row = [&](int64_t orow, int64_t ocol, int32_t &ar, int32_t &ac, int &sid) {
        int64_t nr = P.row_rank[orow], nc = P.col_rank[ocol];
        int i = bi[nr], j = bj[nc];
        sid = i * J + j;
        const SubsetGeom &g = P.subs[sid];
        ar = (int32_t)(g.xoff + (nr - g.r0));
        ac = (int32_t)(g.woff + (nc - g.c0));
    };
    std::vector<int32_t> ear(nnz), eac(nnz);
    for (int64_t e = 0; e < nnz; ++e) {
        int sid;
        arena_row(row[e], col[e], ear[e], eac[e], sid);
        P.subs[sid].nnz++;
    }
    // counting sorts: by arena column (stable), then by arena row -> CSR sorted by column
    std::vector<int64_t> ccount(P.RW + 1, 0), rcount(P.RX + 1, 0);
    for (int64_t e = 0; e < nnz; ++e) {
        ++ccount[eac[e] + 1];
        ++rcount[ear[e] + 1];
    }
    for (int64_t k = 0; k < P.RW; ++k) ccount[k + 1] += ccount[k];
    for (int64_t k = 0; k < P.RX; ++k) rcount[k + 1] += rcount[k];
    P.cptr = ccount;
    P.rptr = rcount;
    std::vector<int64_t> by_col(nnz);
    {
        std::vector<int64_t> pos(ccount.begin(), ccount.end() - 1);
        for (int64_t e = 0; e < nnz; ++e) by_col[pos[eac[e]]++] = e;
    }
    std::vector<int64_t> by_row(nnz);
    {
        std::vector<int64_t> pos(rcount.begin(), rcount.end() - 1);
        for (int64_t k = 0; k < nnz; ++k) {
            int64_t e = by_col[k];
            by_row[pos[ear[e]]++] = e;
        }
    }
    // duplicates are adjacent in the row-major order
    for (int64_t k = 1; k < nnz; ++k)
        if (ear[by_row[k]] == ear[by_row[k - 1]] && eac[by_row[k]] == eac[by_row[k - 1]]) {
            err = "duplicate (row, col) in training data at entry " + std::to_string(by_row[k]);
            return BMF_E_ARG;
        }
    P.ridx.resize(nnz);
    P.rval.resize(nnz);
    for (int64_t k = 0; k < nnz; ++k) {
        int64_t e = by_row[k];
        P.ridx[k] = eac[e];
        P.rval[k] = val[e] - P.offset;
    }
    // column side: stable by arena row then by arena column -> CSC sorted by row
    {
        std::vector<int64_t> pos(ccount.begin(), ccount.end() - 1);
        for (int64_t k = 0; k < nnz; ++k) {
            int64_t e = by_row[k];
            by_col[pos[eac[e]]++] = e;
        }
    }
    P.cidx.resize(nnz);
    P.cval.resize(nnz);
    for (int64_t k = 0; k < nnz; ++k) {
        int64_t e = by_col[k];
        P.cidx[k] = ear[e];
        P.cval[k] = val[e] - P.offset;
    }
    // held-out entries grouped by slot
    std::vector<int32_t> tar(n_test), tac(n_test);
    std::vector<int> tsl(n_test);
    std::vector<int64_t> tcount(S + 1, 0);
    for (int64_t e = 0; e < n_test; ++e) {
        int sid;
        arena_row(test_row[e], test_col[e], tar[e], tac[e], sid);
        tsl[e] = P.subs[sid].slot;
        ++tcount[tsl[e] + 1];
    }
    for (int sl = 0; sl < S; ++sl) tcount[sl + 1] += tcount[sl];
    for (int sl = 0; sl < S; ++sl) {
        SubsetGeom &g = P.subs[P.slot_sid[sl]];
        g.test_off = tcount[sl];
        g.n_test = tcount[sl + 1] - tcount[sl];
    }
    P.trow.resize(n_test);
    P.tcol.resize(n_test);
    P.tval.resize(n_test);
    {
        std::vector<int64_t> pos(tcount.begin(), tcount.end() - 1);
        std::vector<int64_t> order(n_test);
        for (int64_t e = 0; e < n_test; ++e) order[pos[tsl[e]]++] = e;
        // within a slot, entries by (arena row, arena column): consecutive test entries then
        // share their row of the gathered state copy, which the per-sweep RMSE pass reads
        for (int sl = 0; sl < S; ++sl)
            std::stable_sort(order.begin() + tcount[sl], order.begin() + tcount[sl + 1],
                             [&](int64_t a, int64_t b) {
                                 return tar[a] != tar[b] ? tar[a] < tar[b] : tac[a] < tac[b];
                             });
        for (int64_t k = 0; k < n_test; ++k) {
            const int64_t e = order[k];
            P.trow[k] = tar[e];
            P.tcol[k] = tac[e];
            P.tval[k] = test_val[e] - P.offset;
        }
    }
    return 0;
}

}  // namespace bmf
