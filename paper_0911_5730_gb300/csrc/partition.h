// partition.h - the graph partitioner of Algorithm 2 (host code).
#pragma once

#include <cstdint>

namespace bddc {

// Partition the graph (CSR: xadj[n + 1], adjncy[xadj[n]], both directions of
// every edge) into nparts connected parts of about equal vertex weight
// (vwgt, NULL = 1 each; each part within (1 + imbalance) of its share at
// every bisection), cutting little edge weight (adjwgt, NULL = 1).  The
// order of the matching follows `seed`.  Returns the edge cut.
int64_t partition_graph(int n, const int64_t *xadj, const int *adjncy, const int *vwgt, const int *adjwgt,
                        int nparts, double imbalance, uint64_t seed, int *part_out);

}  // namespace bddc
