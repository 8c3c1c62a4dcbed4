// Numeric part of the DH^2 matrix: analytic stage, recompression, matvec.
#pragma once

#include <memory>

#include "common.cuh"
#include "linalg.cuh"
#include "structure.cuh"

namespace dh2 {

// Structure arrays copied to the host once, for scheduling and memory layout.
struct HostStructure {
    int32_t nc = 0, depth = 0;
    std::vector<int32_t> offset, size, parent, son0, son1, level, level_start;
    std::vector<int32_t> tc_base, aidx, a_t, a_c, alevel_start;
    std::vector<int32_t> row_ptr, row_idx, col_ptr, col_idx;
    std::vector<int32_t> adm_t, adm_s, adm_c, near_t, near_s;
    std::vector<int32_t> sd, dir_off, isd_ptr, isd_idx;
    int64_t nactive = 0;
    int32_t pair_of(int32_t t, int32_t c) const { return aidx[tc_base[t] + c]; }
    int32_t son_dir(int32_t t, int32_t c) const { return sd[dir_off[level[t]] + c]; }
};

enum Stage {
    ST_STRUCTURE = 0, ST_NEARFIELD, ST_ANALYTIC, ST_BASIS_WEIGHTS, ST_TOTAL_WEIGHTS_ROW,
    ST_TOTAL_WEIGHTS_COL, ST_TRUNCATE_ROW, ST_TRUNCATE_COL, ST_PROJECT, ST_MATVEC_PLAN, ST_COUNT
};

struct BuildParams {
    double kappa, eta, eps;
    int32_t m, precision, rank_rule, qr_fp64, qr_group_rows;
    int64_t workspace_bytes;
    int32_t tensor_cores, kb_store;
    int32_t qr_tpc[3];   // threads per column of the weight QRs of <= 32, <= 64, <= 128 columns (0 = default)
    // per active pair: the most columns its truncated bases may need (a learned estimate);
    // empty = the structural bound min(rows, k).  A pair whose truncation rank exceeds its
    // cap sends the whole pass back to the structural bound.
    std::vector<int32_t> rank_cap;
    int32_t svd_fp64 = 0;   // mixed form: FP64 Gram + Hermitian Jacobi truncation
    int32_t fault = 0;      // dh2_options.fault (test hook)
    int32_t symmetry = 1;   // derive the column pass from the row pass when the structure allows
    int32_t direct = 0;     // direct recompression: leaf bases per level, intermediates released early
    int32_t layer = 0;      // DH2_SINGLE_LAYER / DH2_DOUBLE_LAYER
    int32_t gram_tc = 0;    // mixed form: Gram tiles of wide FP32 stacks from integer digit products
};

enum KernelId {
    K_NEARFIELD = 0, K_LEAF_BASIS, K_TRANSFER, K_KRON, K_STACK_BLOCKS, K_TSQR, K_TRUNCATE, K_PROJECT,
    K_MV_GATHER, K_MV_FORWARD, K_MV_COUPLING, K_MV_BACKWARD, K_MV_LEAF_OUT, K_TSQR_NARROW, K_LEAF_ORTH, K_WQR_CHOL,
    K_COUNT
};
extern const char* const kKernelNames[K_COUNT];

struct MatrixInfoAcc {
    int64_t near_entries = 0, coupling_entries = 0, basis_entries = 0, matvec_bytes = 0;
    int32_t max_rank_row = 0, max_rank_col = 0;
    double mean_rank_row = 0, mean_rank_col = 0;
    double stage_ms[16] = {0};
    double kernel_ms[16] = {0};
    int64_t kernel_launches[16] = {0};
    double kernel_work[16] = {0};
    int32_t kernel_work_kind[16] = {0};
    int32_t rank_cap_retries = 0;
    int64_t truncation_bytes = 0;
    int32_t symmetric = 0;
    int64_t peak_pool_bytes = 0;
};
enum WorkKind { W_NONE = 0, W_FLOP32 = 1, W_FLOP64 = 2, W_BYTES = 3, W_FLOP_BF16 = 4 };

class NumBase {
public:
    virtual ~NumBase() = default;
    virtual void build(cudaStream_t s) = 0;
    virtual void matvec(const void* x, void* y, int dtype, cudaStream_t s) = 0;
    // matvec whose scratch lives in a fixed device array instead of per-matrix buffers
    virtual void matvec_noalloc(const void* x, void* y, int dtype, cudaStream_t s) = 0;
    virtual void export_pair(int which, int64_t tc, double* out, int64_t cap, int32_t* rows,
                             int32_t* cols, cudaStream_t s) = 0;
    virtual void export_ranks(int32_t* rr, int32_t* rc, cudaStream_t s) = 0;
    virtual void set_timing(bool on) = 0;
    MatrixInfoAcc info;
};

std::unique_ptr<NumBase> make_numeric(const Tree& tr, Structure& st, const HostStructure& hs,
                                      const BuildParams& bp);

void download_structure(const Tree& tr, const Structure& st, HostStructure& hs, cudaStream_t s);

}  // namespace dh2
