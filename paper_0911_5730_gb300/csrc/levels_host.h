// levels_host.h - host-side description of one decomposition level.
#pragma once

#include <cstdint>
#include <string>
#include <vector>

#include "../../include/bddc.h"

namespace bddc {

struct Error {
    int code;
    std::string msg;
    Error(int c, std::string m) : code(c), msg(std::move(m)) {}
};

// One level as Sec. 2.1 describes every level: DOFs, elements holding lists
// of DOFs, and substructures that agglomerate elements.
struct HLevel {
    // input
    int n = 0, nelem = 0, nsub = 0;
    std::vector<int64_t> eptr;      // element slot pointers, nelem+1
    std::vector<int> eslot;         // level DOF of each slot, -1 = Dirichlet (dropped)
    std::vector<int> esub;          // substructure of each element
    std::vector<char> ebnd;         // element touches the Dirichlet boundary
    int nz = 1;                     // null vectors of a floating substructure's matrix
                                    // (1: the constants; 3: the rigid motions in 2D)
    std::vector<double> dofz;       // [nz][n]: their values at each DOF
    std::vector<int> comp;          // displacement component of each DOF, -1 mixed (empty: all 0)
    std::vector<char> dbnd;         // DOF on the boundary of the domain (empty: none)

    // derived by build()
    std::vector<std::vector<int>> sub_elems, sub_dofs;
    std::vector<int64_t> subs_ptr;  // DOF -> substructures holding it (CSR, ascending)
    std::vector<int> subs_idx;
    std::vector<char> is_iface, is_corner;
    std::vector<int> corners;
    struct Edge { int s, t; std::vector<int> dofs; };
    std::vector<Edge> edges;
    std::vector<char> floating;
    std::vector<std::vector<int>> Iord, Gord;   // interior (banded order), interface (ascending)
    std::vector<int> bw, bsz, nblk;
    int block_uniform = 0;          // common power-of-two block size, 0 if none
    std::vector<int> iface_id, iface_dof;

    void build();
    int mult(int g) const { return (int)(subs_ptr[g + 1] - subs_ptr[g]); }
    std::vector<int> subs(int g) const;
};

}  // namespace bddc
