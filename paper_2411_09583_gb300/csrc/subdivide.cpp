// Algorithm 1 (Subdivide) with the quasi-optimal SplitIndices of Sec. 4.1.
//
// Rows are the sorted frequencies omega (index k), columns the sorted points r
// (index j).  An entry is local when omega_k * r_j <= z (FP64 product).
// Readings of the printed algorithm:
//  * the split minimises the mixed (off-diagonal) area (k-k0+1)(j1-j) +
//    (k1-k)(j-j0+1) over the candidate rows (the display writes argmax, the
//    text minimises); for a row k the column is the last local one,
//    j(k) = max{j : omega_k r_j <= z} (j0-1 if none), which makes the
//    lower-right block purely asymptotic;
//  * candidates: every row if the block has at most n_cand rows, else
//    k0 + floor(c (k1-k0)/(n_cand-1)), c = 0..n_cand-1; ties keep the first;
//  * the off-diagonal blocks' areas are (rows) x (cols) of each block (the
//    printed size tests swap index names); a mixed block with area <=
//    min_size is summed directly;
//  * blocks that are entirely local (or asymptotic) go to the local (or
//    asymptotic) list whatever their size; empty blocks are dropped;
//  * the work list is first-in first-out.
// One rule of this implementation, not the paper's: an asymptotic block whose
// space-frequency product is above what one FFT of the device handles
// (X S > kAsyMaxXS) goes back on the work list to be cut into quadrants
// (every part of an asymptotic block is asymptotic), in the same order as the
// device subdivision.
#include <algorithm>
#include <deque>
#include <map>

#include "nuht_host.h"

namespace nuht {

void subdivide(const int32_t* stair, const double* r, const double* omega, int64_t n, int64_t m,
               int64_t min_size, int n_cand, std::vector<HBlock>& loc, std::vector<HBlock>& asy,
               std::vector<HBlock>& dir)
{
    // stair[k] = max{j : omega_k r_j <= z} over the whole sorted r (or -1), so
    // within columns j0..j1: last local column = min(stair[k], j1), or j0 - 1
    // when stair[k] < j0; a block is all local iff stair[k1] >= j1 and all
    // asymptotic iff stair[k0] < j0 (stair is non-increasing in k).
    loc.clear();
    asy.clear();
    dir.clear();
    if (n <= 0 || m <= 0) return;
    std::deque<std::pair<HBlock, bool>> work;   // (block, cut into quadrants)
    auto place = [&](int64_t k0, int64_t k1, int64_t j0, int64_t j1) {
        if (k1 < k0 || j1 < j0) return;
        const HBlock b{k0, k1, j0, j1};
        if (stair[k1] >= j1) { loc.push_back(b); return; }
        if (stair[k0] < j0) {
            if (0.5 * (r[j1] - r[j0]) * 0.5 * (omega[k1] - omega[k0]) > kAsyMaxXS) work.push_back({b, true});
            else asy.push_back(b);
            return;
        }
        if ((k1 - k0 + 1) * (j1 - j0 + 1) <= min_size) { dir.push_back(b); return; }
        work.push_back({b, false});
    };
    place(0, m - 1, 0, n - 1);
    while (!work.empty()) {
        const HBlock b = work.front().first;
        const bool quad = work.front().second;
        work.pop_front();
        if (quad) {
            const int64_t km = (b.k0 + b.k1) >> 1, jm = (b.j0 + b.j1) >> 1;
            place(b.k0, km, b.j0, jm);
            place(km + 1, b.k1, jm + 1, b.j1);
            place(b.k0, km, jm + 1, b.j1);
            place(km + 1, b.k1, b.j0, jm);
            continue;
        }
        const int64_t rows = b.k1 - b.k0 + 1;
        int64_t best_area = -1, bk = b.k0, bj = b.j0 - 1;
        const int64_t ncand = rows <= n_cand ? rows : n_cand;
        for (int64_t c = 0; c < ncand; ++c) {
            const int64_t k = rows <= n_cand ? b.k0 + c : b.k0 + (c * (b.k1 - b.k0)) / (n_cand - 1);
            int64_t j = stair[k];
            if (j > b.j1) j = b.j1;
            if (j < b.j0) j = b.j0 - 1;
            const int64_t area = (k - b.k0 + 1) * (b.j1 - j) + (b.k1 - k) * (j - b.j0 + 1);
            if (best_area < 0 || area < best_area) {
                best_area = area;
                bk = k;
                bj = j;
            }
        }
        place(b.k0, bk, b.j0, bj);             // upper left: local
        place(bk + 1, b.k1, bj + 1, b.j1);     // lower right: asymptotic
        place(b.k0, bk, bj + 1, b.j1);         // upper right: mixed
        place(bk + 1, b.k1, b.j0, bj);         // lower left: mixed
    }
}

}  // namespace nuht

namespace nuht {

// Host check of a subdivision (a work list) of one sorted problem: every
// block lies in the matrix and is non-empty; the blocks cover every entry
// exactly once; local blocks hold only entries with omega_k r_j <= z
// (omega_k1 r_j1 <= z, the sorted corner), asymptotic blocks only entries
// with omega_k r_j > z (omega_k0 r_j0 > z), and direct blocks have area at
// most min_size (Algorithm 1).  The cover is checked by sweeping the rows:
// the set of blocks crossing a row only changes where a block starts or
// ends, and at each such row the crossing blocks' column ranges must tile
// 0..n-1 in order.  O(B log B) for B blocks.
bool check_blocks(const double* r, int64_t n, const double* omega, int64_t m, double z, int64_t min_size,
                  const int64_t* ranges, const int32_t* cls, int64_t count)
{
    if (n < 0 || m < 0 || count < 0) return false;
    for (int64_t j = 1; j < n; ++j)
        if (!(r[j - 1] <= r[j])) return false;
    for (int64_t k = 1; k < m; ++k)
        if (!(omega[k - 1] <= omega[k])) return false;
    if (n == 0 || m == 0) return count == 0;
    struct Ev {
        int64_t row;
        int64_t blk;
        bool start;
    };
    std::vector<Ev> ev;
    ev.reserve(2 * (size_t)count);
    for (int64_t b = 0; b < count; ++b) {
        const int64_t k0 = ranges[4 * b], k1 = ranges[4 * b + 1], j0 = ranges[4 * b + 2], j1 = ranges[4 * b + 3];
        if (k0 < 0 || k1 < k0 || k1 >= m || j0 < 0 || j1 < j0 || j1 >= n) return false;
        switch (cls[b]) {
            case NUHT_BLOCK_LOCAL:
                if (!(omega[k1] * r[j1] <= z)) return false;
                break;
            case NUHT_BLOCK_ASY:
                if (!(omega[k0] * r[j0] > z)) return false;
                break;
            case NUHT_BLOCK_DIRECT:
                if ((k1 - k0 + 1) * (j1 - j0 + 1) > min_size) return false;
                break;
            default:
                return false;
        }
        ev.push_back(Ev{k0, b, true});
        ev.push_back(Ev{k1 + 1, b, false});
    }
    std::sort(ev.begin(), ev.end(), [](const Ev& a, const Ev& b) {
        return a.row != b.row ? a.row < b.row : (a.start < b.start);   // ends before starts
    });
    std::map<int64_t, int64_t> active;   // j0 -> j1 of the blocks crossing the current row
    size_t i = 0;
    if (ev.empty() || ev[0].row != 0) return false;   // row 0 uncovered
    while (i < ev.size()) {
        const int64_t row = ev[i].row;
        for (; i < ev.size() && ev[i].row == row; ++i) {
            const int64_t b = ev[i].blk, j0 = ranges[4 * b + 2], j1 = ranges[4 * b + 3];
            if (ev[i].start) {
                if (!active.emplace(j0, j1).second) return false;   // two blocks start at one column
            } else {
                auto it = active.find(j0);
                if (it == active.end() || it->second != j1) return false;
                active.erase(it);
            }
        }
        if (row >= m) break;
        int64_t next = 0;   // the crossing blocks must tile the columns of this row
        for (const auto& a : active) {
            if (a.first != next) return false;
            next = a.second + 1;
        }
        if (next != n) return false;
    }
    return active.empty();
}

}  // namespace nuht
