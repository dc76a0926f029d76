// Domain blocks of the preconditioner (Eq. (5)-(6)): every unknown goes to a
// material domain, the unknowns of a domain form one contiguous diagonal block
// of the permuted matrix (host code only; the library and the host-logic tests
// compile it).
#include <algorithm>
#include <utility>
#include <vector>

#include "blocks.h"

namespace vie {

namespace {

// Recursive coordinate bisection of ids[lo, hi) (unknowns, positioned at the
// centroid of their T+ tetrahedron) into pieces of at most bmax: split at the
// median along the axis of largest extent (ties by unknown id, so the order is
// deterministic); the pieces are appended as [begin, end) ranges of ids, which
// is reordered in place.
void split_rcb(const Topology &T, std::vector<int> &ids, int lo, int hi, int bmax,
               std::vector<std::pair<int, int>> &pieces) {
    if (hi - lo <= bmax) {
        std::sort(ids.begin() + lo, ids.begin() + hi);
        pieces.push_back({lo, hi});
        return;
    }
    double mn[3] = {1e300, 1e300, 1e300}, mx[3] = {-1e300, -1e300, -1e300};
    for (int i = lo; i < hi; ++i)
        for (int k = 0; k < 3; ++k) {
            const double c = T.cen[3 * (size_t)T.tp[ids[i]] + k];
            mn[k] = std::min(mn[k], c);
            mx[k] = std::max(mx[k], c);
        }
    int ax = 0;
    for (int k = 1; k < 3; ++k)
        if (mx[k] - mn[k] > mx[ax] - mn[ax]) ax = k;
    const int mid = lo + (hi - lo) / 2;
    std::nth_element(ids.begin() + lo, ids.begin() + mid, ids.begin() + hi, [&](int a, int b) {
        const double ca = T.cen[3 * (size_t)T.tp[a] + ax], cb = T.cen[3 * (size_t)T.tp[b] + ax];
        return ca < cb || (ca == cb && a < b);
    });
    split_rcb(T, ids, lo, mid, bmax, pieces);
    split_rcb(T, ids, mid, hi, bmax, pieces);
}

}  // namespace

void domain_blocks(const Topology &T, const std::vector<double> &eps_abs, int bmax, std::vector<int32_t> &perm,
                   std::vector<int> &blk_off, std::vector<int> &blk_n) {
    // domain of every unknown (interface faces: larger |eps|, ties to lower id)
    std::vector<int> udom(T.N);
    for (int n = 0; n < T.N; ++n) {
        const int dp = T.dom[T.tp[n]];
        const int dm = T.kind[n] == KIND_HALF ? dp : T.dom[T.tm[n]];
        const double mp = eps_abs[dp], mm = eps_abs[dm];
        udom[n] = (mm > mp || (mm == mp && dm < dp)) ? dm : dp;
    }
    perm.assign(T.N, 0);
    blk_off.clear();
    blk_n.clear();
    int next = 0;
    for (int d = 0; d < T.n_dom; ++d) {
        std::vector<int> ids;
        for (int n = 0; n < T.N; ++n)
            if (udom[n] == d) ids.push_back(n);
        if (ids.empty()) continue;
        if (bmax > 0 && (int)ids.size() > bmax) {
            // sub-block variant: the domain's unknowns cut into spatially compact
            // pieces of at most bmax by recursive coordinate bisection (median
            // split along the longest extent of the T+ tetrahedron centroids)
            std::vector<std::pair<int, int>> pieces;
            split_rcb(T, ids, 0, (int)ids.size(), bmax, pieces);
            for (auto &pc : pieces) {
                blk_off.push_back(next);
                blk_n.push_back(pc.second - pc.first);
                for (int i = pc.first; i < pc.second; ++i) perm[ids[i]] = next++;
            }
        } else {
            blk_off.push_back(next);
            blk_n.push_back((int)ids.size());
            for (int n : ids) perm[n] = next++;
        }
    }
}

}  // namespace vie
