// Host-side setup of a GFM handle: cell renumbering for locality and the
// sliced-ELL (SELL-32) cell-to-face tables used by every device pass.
//
// The paper's data structure is the face-addressed mesh (owner/neighbour per
// internal face, Sec. 3).  The solver walks it cell by cell, so each cell
// needs its faces; storing them as 32-cell slices in column-major order lets
// one warp read a slice's slot k with one coalesced load.
#include <algorithm>
#include <cstdint>
#include <numeric>
#include <vector>

#include "gfm_setup.h"

namespace gfm {

static void build_adjacency(int n, int F, const int32_t *owner, const int32_t *nb, std::vector<int64_t> &xadj,
                            std::vector<int32_t> &adj)
{
    xadj.assign((size_t)n + 1, 0);
    for (int f = 0; f < F; ++f) {
        xadj[(size_t)owner[f] + 1]++;
        xadj[(size_t)nb[f] + 1]++;
    }
    for (int i = 0; i < n; ++i) xadj[(size_t)i + 1] += xadj[i];
    adj.resize((size_t)xadj[n]);
    std::vector<int64_t> pos(xadj.begin(), xadj.end() - 1);
    for (int f = 0; f < F; ++f) {
        adj[(size_t)pos[owner[f]]++] = nb[f];
        adj[(size_t)pos[nb[f]]++] = owner[f];
    }
}

// BFS from root over unplaced cells; returns the last level and the number of
// levels.  `stamp` marks cells seen in this BFS.
static int bfs_levels(int root, const std::vector<int64_t> &xadj, const std::vector<int32_t> &adj,
                      const std::vector<char> &placed, std::vector<int> &stamp, int tag, std::vector<int32_t> &last)
{
    std::vector<int32_t> cur{root}, next;
    stamp[root] = tag;
    int levels = 1;
    for (;;) {
        next.clear();
        for (int32_t v : cur)
            for (int64_t e = xadj[v]; e < xadj[(size_t)v + 1]; ++e) {
                const int32_t w = adj[(size_t)e];
                if (!placed[w] && stamp[w] != tag) {
                    stamp[w] = tag;
                    next.push_back(w);
                }
            }
        if (next.empty()) break;
        cur.swap(next);
        ++levels;
    }
    last = cur;
    return levels;
}

// Reverse Cuthill-McKee: BFS from a pseudo-peripheral cell (George-Liu
// search), neighbours visited in increasing degree, whole order reversed.
// Returns order[k] = caller index of the k-th cell.
static std::vector<int32_t> rcm(int n, const std::vector<int64_t> &xadj, const std::vector<int32_t> &adj)
{
    std::vector<int32_t> order;
    order.reserve((size_t)n);
    std::vector<char> placed((size_t)n, 0);
    std::vector<int> stamp((size_t)n, 0);
    std::vector<int32_t> last, nbrs;
    auto deg = [&](int32_t v) { return (int)(xadj[(size_t)v + 1] - xadj[v]); };
    int tag = 0, scan = 0;
    while ((int)order.size() < n) {
        while (placed[scan]) ++scan;
        int root = scan;
        int ecc = bfs_levels(root, xadj, adj, placed, stamp, ++tag, last);
        for (int it = 0; it < 6; ++it) {
            int cand = last[0];
            for (int32_t v : last)
                if (deg(v) < deg(cand)) cand = v;
            const int e2 = bfs_levels(cand, xadj, adj, placed, stamp, ++tag, last);
            if (e2 <= ecc) break;
            ecc = e2;
            root = cand;
        }
        size_t head = order.size();
        order.push_back(root);
        placed[root] = 1;
        while (head < order.size()) {
            const int32_t v = order[head++];
            nbrs.clear();
            for (int64_t e = xadj[v]; e < xadj[(size_t)v + 1]; ++e) {
                const int32_t w = adj[(size_t)e];
                if (!placed[w]) {
                    placed[w] = 1;
                    nbrs.push_back(w);
                }
            }
            std::stable_sort(nbrs.begin(), nbrs.end(), [&](int32_t x, int32_t y) { return deg(x) < deg(y); });
            order.insert(order.end(), nbrs.begin(), nbrs.end());
        }
    }
    std::reverse(order.begin(), order.end());
    return order;
}

static inline uint64_t spread21(uint64_t v)
{
    v &= 0x1fffffULL;
    v = (v | (v << 32)) & 0x1f00000000ffffULL;
    v = (v | (v << 16)) & 0x1f0000ff0000ffULL;
    v = (v | (v << 8)) & 0x100f00f00f00f00fULL;
    v = (v | (v << 4)) & 0x10c30c30c30c30c3ULL;
    v = (v | (v << 2)) & 0x1249249249249249ULL;
    return v;
}

// Morton (Z-order) of the cell centres on their bounding box, 21 bits per axis.
static std::vector<int32_t> morton(int n, const double *C)
{
    double lo[3], hi[3];
    for (int k = 0; k < 3; ++k) {
        lo[k] = hi[k] = C[(size_t)k * n];
        for (int i = 1; i < n; ++i) {
            lo[k] = std::min(lo[k], C[(size_t)k * n + i]);
            hi[k] = std::max(hi[k], C[(size_t)k * n + i]);
        }
    }
    std::vector<uint64_t> key((size_t)n);
    for (int i = 0; i < n; ++i) {
        uint64_t m = 0;
        for (int k = 0; k < 3; ++k) {
            const double span = hi[k] - lo[k];
            const double t = span > 0 ? (C[(size_t)k * n + i] - lo[k]) / span : 0.0;
            uint64_t q = (uint64_t)(t * 2097151.0);
            m |= spread21(q) << k;
        }
        key[(size_t)i] = m;
    }
    std::vector<int32_t> order((size_t)n);
    std::iota(order.begin(), order.end(), 0);
    std::stable_sort(order.begin(), order.end(), [&](int32_t a, int32_t b) { return key[a] < key[b]; });
    return order;
}

bool build_host_tables(int n, int F, const int32_t *owner, const int32_t *nb, const double *C_host, int renumber,
                       HostTables &t, std::string &err)
{
    for (int f = 0; f < F; ++f) {
        const int32_t o = owner[f], v = nb[f];
        if (o < 0 || v < 0 || o >= n || v >= n) {
            err = "face " + std::to_string(f) + ": owner/neighbour index out of range";
            return false;
        }
        if (o >= v) {
            err = "face " + std::to_string(f) + ": owner must be < neighbour";
            return false;
        }
    }
    std::vector<int32_t> order;
    if (renumber == 1) {
        std::vector<int64_t> xadj;
        std::vector<int32_t> adj;
        build_adjacency(n, F, owner, nb, xadj, adj);
        order = rcm(n, xadj, adj);
    } else if (renumber == 2) {
        if (!C_host) {
            err = "Morton renumbering needs cell centres";
            return false;
        }
        order = morton(n, C_host);
    } else {
        order.resize((size_t)n);
        std::iota(order.begin(), order.end(), 0);
    }
    t.iperm = order;
    t.perm.assign((size_t)n, 0);
    for (int k = 0; k < n; ++k) t.perm[(size_t)order[k]] = k;

    // per internal cell: faces in ascending caller order
    std::vector<int32_t> deg((size_t)n, 0);
    for (int f = 0; f < F; ++f) {
        deg[(size_t)t.perm[owner[f]]]++;
        deg[(size_t)t.perm[nb[f]]]++;
    }
    std::vector<int64_t> off((size_t)n + 1, 0);
    for (int i = 0; i < n; ++i) off[(size_t)i + 1] = off[i] + deg[i];
    std::vector<int32_t> lf((size_t)off[n]), lo((size_t)off[n]);
    std::vector<int64_t> pos(off.begin(), off.end() - 1);
    for (int f = 0; f < F; ++f) {
        const int32_t a = t.perm[owner[f]], b = t.perm[nb[f]];
        lf[(size_t)pos[a]] = f + 1;
        lo[(size_t)pos[a]++] = b;
        lf[(size_t)pos[b]] = -(f + 1);
        lo[(size_t)pos[b]++] = a;
    }
    t.n = n;
    t.n_pad = (n + kSliceH - 1) / kSliceH * kSliceH;
    t.n_slices = t.n_pad / kSliceH;
    t.slice_ptr.assign((size_t)t.n_slices + 1, 0);
    int64_t total = 0;
    for (int s = 0; s < t.n_slices; ++s) {
        int w = 0;
        for (int l = 0; l < kSliceH; ++l) {
            const int i = s * kSliceH + l;
            if (i < n) w = std::max(w, deg[(size_t)i]);
        }
        total += (int64_t)w * kSliceH;
        if (total > INT32_MAX) {
            err = "mesh too large for 32-bit slot offsets";
            return false;
        }
        t.slice_ptr[(size_t)s + 1] = (int32_t)total;
    }
    t.n_slots = (int32_t)total;
    t.col.assign((size_t)total, 0);
    t.face.assign((size_t)total, 0);
    t.max_width = 0;
    for (int s = 0; s < t.n_slices; ++s) {
        const int base = t.slice_ptr[(size_t)s];
        const int w = (t.slice_ptr[(size_t)s + 1] - base) / kSliceH;
        t.max_width = std::max(t.max_width, w);
        for (int l = 0; l < kSliceH; ++l) {
            const int i = s * kSliceH + l;
            for (int k = 0; k < w; ++k) {
                const size_t slot = (size_t)base + (size_t)k * kSliceH + l;
                if (i < n && k < deg[(size_t)i]) {
                    t.col[slot] = lo[(size_t)off[i] + k];
                    t.face[slot] = lf[(size_t)off[i] + k];
                } else {
                    t.col[slot] = i;
                    t.face[slot] = 0;
                }
            }
        }
    }
    return true;
}

bool build_batch_tables(const std::vector<TankMesh> &tanks, int renumber, HostTables &t, BatchTables &bt,
                        std::string &err)
{
    const int T = (int)tanks.size();
    bt.T = T;
    bt.coff.assign((size_t)T + 1, 0);
    bt.foff.assign((size_t)T + 1, 0);
    bt.ioff.assign((size_t)T + 1, 0);
    bt.ncell.assign((size_t)T, 0);
    std::vector<HostTables> per((size_t)T);
    for (int k = 0; k < T; ++k) {
        const TankMesh &m = tanks[(size_t)k];
        if (m.n <= 0 || m.F <= 0) {
            err = "tank " + std::to_string(k) + ": needs cells and internal faces";
            return false;
        }
        std::string e;
        if (!build_host_tables(m.n, m.F, m.owner, m.nb, m.C, renumber, per[(size_t)k], e)) {
            err = "tank " + std::to_string(k) + ": " + e;
            return false;
        }
        bt.coff[(size_t)k + 1] = bt.coff[(size_t)k] + m.n;
        bt.foff[(size_t)k + 1] = bt.foff[(size_t)k] + m.F;
        bt.ioff[(size_t)k + 1] = bt.ioff[(size_t)k] + per[(size_t)k].n_pad;
        bt.ncell[(size_t)k] = m.n;
    }
    const long long n = bt.coff[(size_t)T], np = bt.ioff[(size_t)T];
    if (np > INT32_MAX) {
        err = "batch too large for 32-bit cell indices";
        return false;
    }
    t.n = (int)n;
    t.n_pad = (int)np;
    t.n_slices = (int)(np / kSliceH);
    t.perm.assign((size_t)n, 0);
    t.iperm.assign((size_t)np, -1);
    t.slice_ptr.assign((size_t)t.n_slices + 1, 0);
    bt.slice_tank.assign((size_t)t.n_slices, 0);
    bt.face_tank.assign((size_t)bt.foff[(size_t)T], 0);
    long long slots = 0;
    for (int k = 0; k < T; ++k) slots += per[(size_t)k].n_slots;
    if (slots > INT32_MAX) {
        err = "batch too large for 32-bit slot offsets";
        return false;
    }
    t.n_slots = (int)slots;
    t.col.assign((size_t)slots, 0);
    t.face.assign((size_t)slots, 0);
    t.max_width = 0;
    int s_at = 0;
    int32_t slot_at = 0;
    for (int k = 0; k < T; ++k) {
        const HostTables &h = per[(size_t)k];
        const int32_t co = bt.coff[(size_t)k], fo = bt.foff[(size_t)k], io = bt.ioff[(size_t)k];
        for (int i = 0; i < h.n; ++i) {
            t.perm[(size_t)co + i] = io + h.perm[(size_t)i];
            t.iperm[(size_t)io + h.perm[(size_t)i]] = co + i;
        }
        for (int f = 0; f < tanks[(size_t)k].F; ++f) bt.face_tank[(size_t)fo + f] = k;
        for (int sl = 0; sl < h.n_slices; ++sl) {
            t.slice_ptr[(size_t)s_at + sl + 1] = slot_at + h.slice_ptr[(size_t)sl + 1];
            bt.slice_tank[(size_t)s_at + sl] = k;
        }
        for (int q = 0; q < h.n_slots; ++q) {
            t.col[(size_t)slot_at + q] = io + h.col[(size_t)q];
            const int32_t code = h.face[(size_t)q];
            t.face[(size_t)slot_at + q] = code == 0 ? 0 : (code > 0 ? code + fo : code - fo);
        }
        t.max_width = std::max(t.max_width, h.max_width);
        s_at += h.n_slices;
        slot_at += h.n_slots;
    }
    return true;
}

bool plan_batch_ctas(const BatchTables &bt, int grid, std::vector<int32_t> &cta4, std::vector<int32_t> &tank2,
                     std::string &err, const std::vector<double> &weight)
{
    const int T = bt.T;
    if (grid < T) {
        err = "a batched solve needs at least one CTA per tank (" + std::to_string(T) + " tanks, grid " +
              std::to_string(grid) + ")";
        return false;
    }
    if (!weight.empty() && weight.size() != (size_t)T) {
        err = "one weight per tank expected";
        return false;
    }
    std::vector<long long> sl((size_t)T);
    for (int k = 0; k < T; ++k) sl[(size_t)k] = (bt.ioff[(size_t)k + 1] - bt.ioff[(size_t)k]) / kSliceH;
    std::vector<int> g((size_t)T, 1);
    if (weight.empty()) {
        for (int extra = grid - T; extra > 0; --extra) {
            int best = 0;
            for (int k = 1; k < T; ++k)  // load per CTA, compared exactly: sl_k / g_k > sl_b / g_b
                if (sl[(size_t)k] * g[(size_t)best] > sl[(size_t)best] * g[(size_t)k]) best = k;
            g[(size_t)best] += 1;
        }
    } else {
        // work = slices x weight (e.g. the tank's last iteration count); a
        // tank never gets more CTAs than slices
        for (int extra = grid - T; extra > 0; --extra) {
            int best = -1;
            double bw = -1.0;
            for (int k = 0; k < T; ++k) {
                if (g[(size_t)k] >= sl[(size_t)k]) continue;
                const double w = (double)sl[(size_t)k] * std::max(weight[(size_t)k], 1e-9) / g[(size_t)k];
                if (w > bw) {
                    bw = w;
                    best = k;
                }
            }
            if (best < 0) break;
            g[(size_t)best] += 1;
        }
    }
    cta4.assign((size_t)grid * 4, 0);
    tank2.assign((size_t)T * 2, 0);
    int b = 0;
    for (int k = 0; k < T; ++k) {
        const int s_first = bt.ioff[(size_t)k] / kSliceH;
        const int end = bt.ioff[(size_t)k] + bt.ncell[(size_t)k];
        tank2[(size_t)k * 2] = b;
        for (int q = 0; q < g[(size_t)k]; ++q, ++b) {
            cta4[(size_t)b * 4 + 0] = k;
            cta4[(size_t)b * 4 + 1] = s_first + (int)((sl[(size_t)k] * q) / g[(size_t)k]);
            cta4[(size_t)b * 4 + 2] = s_first + (int)((sl[(size_t)k] * (q + 1)) / g[(size_t)k]);
            cta4[(size_t)b * 4 + 3] = end;
        }
        tank2[(size_t)k * 2 + 1] = b;
    }
    return true;
}

int batch_replan_max_slices(const BatchTables &bt, int grid)
{
    const int T = bt.T;
    long long total = 0;
    for (int k = 0; k < T; ++k) total += (bt.ioff[(size_t)k + 1] - bt.ioff[(size_t)k]) / kSliceH;
    if (total <= 0) total = 1;
    const long long extra = std::max(grid - T, 0);
    int worst = 0;
    for (int k = 0; k < T; ++k) {
        const long long sl = (bt.ioff[(size_t)k + 1] - bt.ioff[(size_t)k]) / kSliceH;
        const long long g = 1 + (extra * sl) / total;
        worst = std::max(worst, (int)((sl + g - 1) / g));
    }
    return worst;
}

}  // namespace gfm
