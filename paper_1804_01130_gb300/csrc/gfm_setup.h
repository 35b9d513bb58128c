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

// A batch of independent meshes ("tanks").  Caller arrays are the tanks'
// arrays concatenated in tank order.  Internally each tank is renumbered on
// its own and occupies whole slices (padded to 32 cells), so no slice mixes
// tanks.  iperm of a padding cell is -1.
struct BatchTables {
    int T = 0;
    std::vector<int32_t> coff, foff;   // [T+1] caller cell / face offsets
    std::vector<int32_t> ioff;         // [T+1] internal cell offsets (multiples of 32)
    std::vector<int32_t> ncell;        // [T] real cells
    std::vector<int32_t> slice_tank;   // [n_slices]
    std::vector<int32_t> face_tank;    // [F]
};

struct TankMesh {
    int n, F;
    const int32_t *owner, *nb;  // host, tank-local numbering
    const double *C;            // host [3][n] or nullptr
};

bool build_batch_tables(const std::vector<TankMesh> &tanks, int renumber, HostTables &t, BatchTables &bt,
                        std::string &err);

// CTAs of a batched persistent solve: each tank gets at least one CTA and
// the rest go, one by one, to the tank with the most slices per CTA -- or,
// with per-tank weights (e.g. the iterations each tank took last time), the
// most slices x weight per CTA; a tank's slices are split evenly between its
// CTAs.  out: per CTA {tank, s0, s1, end} (end = internal index one past the
// tank's last real cell), per tank {first CTA, last CTA + 1}.
bool plan_batch_ctas(const BatchTables &bt, int grid, std::vector<int32_t> &cta4, std::vector<int32_t> &tank2,
                     std::string &err, const std::vector<double> &weight = {});

// Most slices one CTA can hold after the batched solve re-plans its CTA
// table on the device: an upper bound, the split over all tanks that gives
// tank t 1 + floor((grid - T) sl_t / sl_all) CTAs (sl: slices).  A device
// re-plan over a set S of tanks minimises the most slices per CTA over S;
// that minimum is at most the one over all tanks, which is at most this
// split's.
int batch_replan_max_slices(const BatchTables &bt, int grid);

}  // namespace gfm
