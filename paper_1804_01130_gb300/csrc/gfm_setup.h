// Host-side mesh tables (renumbering + sliced ELL); plain C++, no CUDA.
#pragma once

#include <cstdint>
#include <string>
#include <vector>

namespace gfm {

constexpr int kSliceH = 32;

struct HostTables {
    int n = 0, n_pad = 0, n_slices = 0, n_slots = 0, max_width = 0;
    std::vector<int32_t> perm;       // caller -> internal
    std::vector<int32_t> iperm;      // internal -> caller
    std::vector<int32_t> slice_ptr;  // [n_slices + 1]
    std::vector<int32_t> col;        // [n_slots]
    std::vector<int32_t> face;       // [n_slots]
};

// Validates the face list (0 <= owner < neighbour < n) and builds the tables.
// renumber: 0 caller order, 1 reverse Cuthill-McKee, 2 Morton (needs C_host).
bool build_host_tables(int n, int F, const int32_t *owner, const int32_t *nb, const double *C_host, int renumber,
                       HostTables &t, std::string &err);

}  // namespace gfm
