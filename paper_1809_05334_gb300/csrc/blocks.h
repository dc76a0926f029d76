// Domain blocks of the preconditioner (blocks.cpp).
#pragma once
#include <cstdint>
#include <vector>

#include "vie_internal.h"

namespace vie {

// Eq. (5): the domain of every unknown (a face between two domains goes to the
// one with the larger |eps_r|, ties to the lower index; half functions to
// their tetrahedron's domain), and the permutation perm (canonical unknown ->
// matrix row) that makes each domain's unknowns one contiguous block, in
// domain order and by unknown id inside a block.  bmax > 0: a domain with more
// unknowns than bmax is cut into spatially compact sub-blocks of at most bmax
// (the sub-block variant).  eps_abs: |eps_r| per domain.
void domain_blocks(const Topology &T, const std::vector<double> &eps_abs, int bmax, std::vector<int32_t> &perm,
                   std::vector<int> &blk_off, std::vector<int> &blk_n);

}  // namespace vie
