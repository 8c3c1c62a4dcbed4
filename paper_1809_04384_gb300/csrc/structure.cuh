// Directions, block tree and (t,c) pair bookkeeping (structure.cu).
#pragma once

#include "common.cuh"

namespace dh2 {

struct Structure {
    double kappa = 0, eta1 = 10, eta2 = 1;
    int32_t depth = 0;
    int32_t nc = 0;
    // directions (Remark "construction of directions"), per level l
    std::vector<int32_t> msplit, ndir;      // host
    std::vector<int32_t> dir_off;           // host, depth+2 entries
    std::vector<double> dmax;               // host, d_l
    DBuf<double> dirs;                      // [total][3]
    DBuf<int32_t> sd;                       // [total]: index into D_{l+1}
    DBuf<int32_t> dir_off_d, ndir_d;        // device copies (per level)
    DBuf<int32_t> isd_ptr, isd_idx;         // sd^{-1}: global dir of level l+1 -> global dirs of level l
    // cluster geometry derived from the tree
    DBuf<double> diam;                      // [nc]
    // block tree leaves (breadth-first order)
    int64_t nadm = 0, nnear = 0;
    DBuf<int32_t> adm_t, adm_s, adm_c;
    DBuf<int32_t> near_t, near_s;
    // pairs (t,c): tc = tc_base[t] + c
    int64_t ntc = 0;
    DBuf<int32_t> tc_base;                  // [nc]
    DBuf<int32_t> tc_cluster;               // [ntc]
    DBuf<int32_t> row_ptr, row_idx;         // CSR tc -> admissible block ids (block order)
    DBuf<int32_t> col_ptr, col_idx;
    DBuf<int8_t> active;                    // [ntc]
    DBuf<int32_t> aidx;                     // [ntc]: active index or -1
    int64_t nactive = 0;
    DBuf<int32_t> alist;                    // [nactive]: tc of each active pair
    DBuf<int32_t> a_t, a_c;                 // [nactive]: cluster and direction of each active pair
    std::vector<int32_t> alevel_start;      // host, depth+2 entries (active index ranges per level)
};

void build_structure(const Tree& tr, Structure& st, double kappa, double eta1, double eta2,
                     cudaStream_t s);

}  // namespace dh2
