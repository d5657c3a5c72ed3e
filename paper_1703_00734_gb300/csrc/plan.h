// plan.h -- host-side preprocessing of the training data (validation, ordering, I x J grid,
// per-subset observation lists).  Internal to libbmf.
#pragma once
#include <cstdint>
#include <string>
#include <vector>

namespace bmf {

struct SubsetGeom {
    int i = 0, j = 0, stage = 0, sid = 0, slot = 0;
    int64_t r0 = 0, r1 = 0, c0 = 0, c1 = 0;  // row/col block in the reordered order
    int64_t nnz = 0;
    int64_t xoff = 0;      // first row of this subset's X block in the X arena
    int64_t woff = 0;      // first row of its W block in the W arena
    int64_t test_off = 0;  // first of its held-out entries in the test arena
    int64_t n_test = 0;
    int64_t n() const { return r1 - r0; }
    int64_t d() const { return c1 - c0; }
};

// The arenas stack the subsets' factor blocks in slot order: subsets sorted by (stage, id).
// The row-side lists index the W arena and the column-side lists the X arena, so any batch
// of subsets that is contiguous in slot order (one stage, or one subset) is a contiguous
// range of arena rows.
struct HostPlan {
    int64_t N = 0, D = 0, nnz = 0;
    int I = 1, J = 1;
    std::vector<int64_t> row_perm, col_perm;  // new -> original
    std::vector<int64_t> row_rank, col_rank;  // original -> new
    std::vector<int64_t> row_bounds, col_bounds;
    double offset = 0.0;
    std::vector<SubsetGeom> subs;             // by subset id
    std::vector<int> slot_sid;                // slot -> subset id
    int64_t RX = 0, RW = 0;                   // arena row counts
    // row side: over the X arena rows; indices into the W arena
    std::vector<int64_t> rptr;
    std::vector<int32_t> ridx;
    std::vector<double> rval;
    // column side: over the W arena rows; indices into the X arena
    std::vector<int64_t> cptr;
    std::vector<int32_t> cidx;
    std::vector<double> cval;
    // held-out entries: arena row, arena col, value (centred), grouped by slot
    std::vector<int32_t> trow, tcol;
    std::vector<double> tval;
};

// Returns 0 on success, else a bmf_status code with `err` set.
int build_plan(int64_t N, int64_t D, int64_t nnz, const int32_t *row, const int32_t *col,
               const double *val, int order, int center, int I, const int64_t *row_bounds,
               int J, const int64_t *col_bounds, int64_t n_test, const int32_t *test_row,
               const int32_t *test_col, const double *test_val, HostPlan &P, std::string &err);

int subset_stage(int i, int j);

}  // namespace bmf
