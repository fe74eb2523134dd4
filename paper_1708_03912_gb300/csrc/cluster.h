// Cluster tree and block partition of the cluster method (cluster.cpp).  Internal.
#pragma once
#include <cstdint>
#include <vector>

#include "internal.h"

namespace fl {

struct ClusterPlan {
    int dim = 0, leaf = 0, nodes = 0, depth = 0;
    double eta = 0.0;
    int64_t n = 0;
    std::vector<int> perm;         // n: DOFs in tree order
    std::vector<int> lo, hi;       // per node: range of perm
    std::vector<int> son;          // 2 per node (-1: leaf)
    std::vector<int> level;        // per node
    std::vector<double> center;    // dim per node: centre of the cluster cube
    std::vector<double> side;      // per node: side of the cube
    std::vector<int> far, near;    // pairs of node ids (admissible; inadmissible leaf pairs)
};

// Builds the tree over P's DOFs and the partition for admissibility parameter eta and
// leaves of at most `leaf` DOFs.  FL_EINVAL for leaf < 1 or eta < 0.
int build_cluster_plan(const Plan& P, double eta, int leaf, ClusterPlan& C);

}  // namespace fl
