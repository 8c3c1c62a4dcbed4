// extern "C" entry points of libdh2 (declared in include/dh2.h).
#include <algorithm>
#include <atomic>
#include <cstring>
#include <map>
#include <memory>
#include <mutex>
#include <numeric>
#include <string>
#include <thread>

#include "learned.cuh"
#include "numeric.cuh"
#include "structure.cuh"

struct dh2_tree_s {
    dh2::Tree tr;
};

struct dh2_matrix_s {
    dh2::Tree tr;                       // the matrix's own copy of the tree
    dh2::Structure st;
    dh2::HostStructure hs;
    dh2::BuildParams bp;
    std::unique_ptr<dh2::NumBase> num;
    int32_t depth = 0;
    int32_t learned_m = 0;
    double structure_ms = 0;
};

struct dh2_model_s {
    dh2::learned::Model md;
};

namespace dh2 {

namespace {
thread_local std::string g_last_error;

cudaStream_t as_stream(void* s) { return reinterpret_cast<cudaStream_t>(s); }

template <class F>
dh2_status guarded(F&& f) {
    try {
        f();
        return DH2_OK;
    } catch (const Error& e) {
        set_error(e.msg);
        return e.status;
    } catch (const std::bad_alloc&) {
        set_error("host allocation failed");
        return DH2_ENOMEM;
    } catch (const std::exception& e) {
        set_error(e.what());
        return DH2_ECUDA;
    }
}

template <class T>
void copy_dbuf(DBuf<T>& dst, const DBuf<T>& src, cudaStream_t s) {
    dst.alloc(src.n);
    if (src.n) DH2_CHECK_CUDA(cudaMemcpyAsync(dst.p, src.p, src.n * sizeof(T), cudaMemcpyDeviceToDevice, s));
}

void clone_tree(Tree& dst, const Tree& src, cudaStream_t s) {
    dst.n = src.n;
    dst.nv = src.nv;
    dst.leaf_max = src.leaf_max;
    dst.point_mode = src.point_mode;
    dst.nc = src.nc;
    dst.depth = src.depth;
    dst.level_start = src.level_start;
    copy_dbuf(dst.vert, src.vert, s);
    copy_dbuf(dst.tri, src.tri, s);
    copy_dbuf(dst.cent, src.cent, s);
    copy_dbuf(dst.tlo, src.tlo, s);
    copy_dbuf(dst.thi, src.thi, s);
    copy_dbuf(dst.perm, src.perm, s);
    copy_dbuf(dst.offset, src.offset, s);
    copy_dbuf(dst.size, src.size, s);
    copy_dbuf(dst.parent, src.parent, s);
    copy_dbuf(dst.son0, src.son0, s);
    copy_dbuf(dst.son1, src.son1, s);
    copy_dbuf(dst.level, src.level, s);
    copy_dbuf(dst.lo, src.lo, s);
    copy_dbuf(dst.hi, src.hi, s);
    copy_dbuf(dst.area, src.area, s);
    copy_dbuf(dst.x3, src.x3, s);
    copy_dbuf(dst.x7, src.x7, s);
}

void check_build_args(dh2_tree tree, double kappa, int32_t m, double eta, double eps, const dh2_options& o,
                      const char* fn) {
    const std::string f(fn);
    if (tree == nullptr) throw Error{DH2_EINVAL, f + ": tree is NULL"};
    if (tree->tr.point_mode) throw Error{DH2_EINVAL, f + ": a point-mode tree has no Galerkin elements"};
    if (!(std::isfinite(kappa) && kappa >= 0.0)) throw Error{DH2_EINVAL, f + ": kappa must be >= 0"};
    if (!(m >= 1 && m <= 8)) throw Error{DH2_EINVAL, f + ": m must be in [1, 8]"};
    if (!(std::isfinite(eta) && eta > 0.0)) throw Error{DH2_EINVAL, f + ": eta must be > 0"};
    if (!(std::isfinite(eps) && eps > 0.0)) throw Error{DH2_EINVAL, f + ": eps must be > 0"};
    if (!(std::isfinite(o.eta1) && o.eta1 > 0.0)) throw Error{DH2_EINVAL, f + ": eta1 must be > 0"};
    if (!(o.precision == DH2_FP64 || o.precision == DH2_MIXED)) throw Error{DH2_EINVAL, f + ": bad precision"};
    if (!(o.rank_rule == DH2_RANK_BLOCKREL || o.rank_rule == DH2_RANK_GLOBAL || o.rank_rule == DH2_RANK_SPECTRAL))
        throw Error{DH2_EINVAL, f + ": bad rank rule"};
    if (o.qr_group_rows < 0) throw Error{DH2_EINVAL, f + ": qr_group_rows must be >= 0"};
    if (o.tensor_cores != 0 && o.tensor_cores != 1) throw Error{DH2_EINVAL, f + ": tensor_cores must be 0 or 1"};
    if (o.kb_store < 0 || o.kb_store > 2) throw Error{DH2_EINVAL, f + ": kb_store must be 0, 1 or 2"};
    if (o.qr_fp64 < 0 || o.qr_fp64 > 2) throw Error{DH2_EINVAL, f + ": qr_fp64 must be 0, 1 or 2"};
    if (o.svd_fp64 != 0 && o.svd_fp64 != 1) throw Error{DH2_EINVAL, f + ": svd_fp64 must be 0 or 1"};
    if (o.fault < DH2_FAULT_NONE || o.fault > DH2_FAULT_ALLOC) throw Error{DH2_EINVAL, f + ": bad fault hook"};
    if (o.symmetry != 0 && o.symmetry != 1) throw Error{DH2_EINVAL, f + ": symmetry must be 0 or 1"};
    if (o.direct != 0 && o.direct != 1) throw Error{DH2_EINVAL, f + ": direct must be 0 or 1"};
    if (o.layer != DH2_SINGLE_LAYER && o.layer != DH2_DOUBLE_LAYER) throw Error{DH2_EINVAL, f + ": bad layer"};
    if (o.gram_tc != 0 && o.gram_tc != 1) throw Error{DH2_EINVAL, f + ": gram_tc must be 0 or 1"};
    static const int width[3] = {32, 64, 128};
    for (int c = 0; c < 3; ++c) {
        const int v = o.qr_tpc[c];
        if (!(v == 0 || ((v == 1 || v == 2 || v == 4 || v == 8) && v * width[c] <= 256)))
            throw Error{DH2_EINVAL, f + ": qr_tpc[" + std::to_string(c) + "] must be 0, or 1, 2, 4, 8 with "
                                        "threads x class width <= 256"};
    }
    if (o.learned != 0 && o.learned != 1) throw Error{DH2_EINVAL, f + ": learned must be 0 or 1"};
    if (o.learned && o.model == nullptr) throw Error{DH2_EINVAL, f + ": learned = 1 needs a model"};
    if (o.learned) {
        int dev = 0;
        DH2_CHECK_CUDA(cudaGetDevice(&dev));
        if (o.model->md.dev != dev) throw Error{DH2_EINVAL, f + ": the model lives on another device"};
    }
}

// The whole build of one matrix on stream s (arguments already checked); blocks until done.
dh2_matrix build_matrix(dh2_tree tree, double kappa, int32_t m, double eta, double eps, const dh2_options& o,
                        cudaStream_t s) {
    struct FaultScope {   // the allocation hook never outlives this build
        explicit FaultScope(bool on) { fault_alloc_pending() = on; }
        ~FaultScope() { fault_alloc_pending() = false; }
    } fault_scope(o.fault == DH2_FAULT_ALLOC);
    auto mat = std::make_unique<dh2_matrix_s>();
    // high-water mark of the pool's handed-out memory over this build
    int pdev = 0;
    DH2_CHECK_CUDA(cudaGetDevice(&pdev));
    cudaMemPool_t pool;
    DH2_CHECK_CUDA(cudaDeviceGetDefaultMemPool(&pool, pdev));
    {
        uint64_t zero = 0;
        DH2_CHECK_CUDA(cudaMemPoolSetAttribute(pool, cudaMemPoolAttrUsedMemHigh, &zero));
    }
    cudaEvent_t e0, e1;
    DH2_CHECK_CUDA(cudaEventCreate(&e0));
    DH2_CHECK_CUDA(cudaEventCreate(&e1));
    DH2_CHECK_CUDA(cudaEventRecord(e0, s));
    clone_tree(mat->tr, tree->tr, s);
    build_structure(mat->tr, mat->st, kappa, o.eta1, eta, s);
    DH2_CHECK_CUDA(cudaEventRecord(e1, s));
    download_structure(mat->tr, mat->st, mat->hs, s);
    float ms = 0;
    DH2_CHECK_CUDA(cudaEventSynchronize(e1));
    DH2_CHECK_CUDA(cudaEventElapsedTime(&ms, e0, e1));
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    mat->structure_ms = ms;
    mat->depth = mat->tr.depth;
    mat->bp = BuildParams{kappa, eta, eps, m, o.precision, o.rank_rule, o.qr_fp64, o.qr_group_rows,
                          o.workspace_bytes, o.tensor_cores, o.kb_store, {o.qr_tpc[0], o.qr_tpc[1], o.qr_tpc[2]},
                          {}, o.svd_fp64, o.fault, o.symmetry, o.direct, o.layer, o.gram_tc};
    if (o.learned) {
        int32_t ml = m;
        learned::choose(mat->tr, mat->st, mat->hs, o.model->md, s, &ml, mat->bp.rank_cap);
        mat->bp.m = ml;
        mat->learned_m = ml;
    }
    mat->num = make_numeric(mat->tr, mat->st, mat->hs, mat->bp);
    mat->num->build(s);
    mat->num->info.stage_ms[ST_STRUCTURE] += ms;
    DH2_CHECK_CUDA(cudaStreamSynchronize(s));
    {
        uint64_t high = 0;
        DH2_CHECK_CUDA(cudaMemPoolGetAttribute(pool, cudaMemPoolAttrUsedMemHigh, &high));
        mat->num->info.peak_pool_bytes = (int64_t)high;
    }
    return mat.release();
}

// A few non-blocking streams per device for the batched products (created on first use,
// kept for the life of the process).
constexpr int kBatchStreams = 8;
cudaStream_t batch_stream(int i) {
    static std::mutex mu;
    static std::vector<std::vector<cudaStream_t>> per_dev;
    int dev = 0;
    DH2_CHECK_CUDA(cudaGetDevice(&dev));
    std::lock_guard<std::mutex> lk(mu);
    if ((int)per_dev.size() <= dev) per_dev.resize(dev + 1);
    auto& v = per_dev[dev];
    if (v.empty()) {
        v.resize(kBatchStreams);
        for (auto& st : v) DH2_CHECK_CUDA(cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking));
    }
    return v[i % kBatchStreams];
}

const char* kStageNames[] = {"structure",      "nearfield",          "analytic",        "basis_weights",
                             "total_weights_row", "total_weights_col", "truncate_row",   "truncate_col",
                             "project",        "matvec_plan"};
}  // namespace

void set_error(const std::string& msg) { g_last_error = msg; }

// ----------------------------------------------------------------------------- device memory

namespace {
std::mutex g_pool_mu;
bool g_pool_ready[64] = {};
}  // namespace

void* dev_alloc(size_t bytes) {
    int dev = 0;
    DH2_CHECK_CUDA(cudaGetDevice(&dev));
    thread_local uint64_t seen = 0;   // devices (< 64) whose pool is known to be configured
    if (dev >= 64 || !((seen >> dev) & 1)) {
        std::lock_guard<std::mutex> lk(g_pool_mu);
        if (dev >= 64 || !g_pool_ready[dev]) {
            // keep up to a quarter of the device's memory of freed blocks in the pool, so
            // that the many short-lived buffers of a build, and the next build, reuse
            // mapped memory instead of going back to the driver
            cudaMemPool_t pool;
            DH2_CHECK_CUDA(cudaDeviceGetDefaultMemPool(&pool, dev));
            size_t free_b = 0, total_b = 0;
            DH2_CHECK_CUDA(cudaMemGetInfo(&free_b, &total_b));
            uint64_t keep = total_b / 4;
            DH2_CHECK_CUDA(cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &keep));
            if (dev < 64) g_pool_ready[dev] = true;
        }
        if (dev < 64) seen |= uint64_t(1) << dev;
    }
    if (fault_alloc_pending()) {
        fault_alloc_pending() = false;
        throw Error{DH2_ENOMEM, "dev_alloc: injected allocation failure (dh2_options.fault)"};
    }
    void* p = nullptr;
    cudaError_t e = cudaMallocAsync(&p, bytes, alloc_stream());
    if (e == cudaErrorMemoryAllocation) {
        // the pool may hold freed blocks of other streams, or blocks still in flight: wait
        // for the device, hand the pool's cached memory back to the driver and retry once
        cudaGetLastError();
        DH2_CHECK_CUDA(cudaDeviceSynchronize());
        cudaMemPool_t pool;
        DH2_CHECK_CUDA(cudaDeviceGetDefaultMemPool(&pool, dev));
        DH2_CHECK_CUDA(cudaMemPoolTrimTo(pool, 0));
        e = cudaMallocAsync(&p, bytes, alloc_stream());
    }
    if (e != cudaSuccess) {
        cudaGetLastError();
        throw Error{e == cudaErrorMemoryAllocation ? DH2_ENOMEM : DH2_ECUDA,
                    "cudaMallocAsync(" + std::to_string(bytes) + " bytes): " + cudaGetErrorString(e)};
    }
    return p;
}

bool& fault_alloc_pending() {
    thread_local bool pending = false;
    return pending;
}

void ensure_smem(const void* fn, size_t bytes) {
    static std::mutex mu;
    static std::map<std::pair<int, const void*>, size_t> cur;
    int dev = 0;
    DH2_CHECK_CUDA(cudaGetDevice(&dev));
    std::lock_guard<std::mutex> lk(mu);
    size_t& c = cur[{dev, fn}];
    if (bytes > c) {
        DH2_CHECK_CUDA(cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes));
        c = bytes;
    }
}

void dev_free(void* p) {
    if (p) cudaFreeAsync(p, alloc_stream());
}


static std::atomic<int64_t> g_launches{0};
void count_launch() { g_launches.fetch_add(1, std::memory_order_relaxed); }
void count_launches(int64_t n) { g_launches.fetch_add(n, std::memory_order_relaxed); }
void uncount_launches(int64_t n) { g_launches.fetch_sub(n, std::memory_order_relaxed); }

}  // namespace dh2

using namespace dh2;

extern "C" {

const char* dh2_last_error(void) { return g_last_error.c_str(); }

int64_t dh2_kernel_launches(void) { return g_launches.load(); }

const char* dh2_stage_name(int32_t i) {
    if (i < 0 || i >= (int32_t)(sizeof(kStageNames) / sizeof(kStageNames[0]))) return nullptr;
    return kStageNames[i];
}

const char* dh2_kernel_name(int32_t i) {
    if (i < 0 || i >= K_COUNT) return nullptr;
    return kKernelNames[i];
}

dh2_status dh2_options_default(dh2_options* opt) {
    if (!opt) {
        set_error("dh2_options_default: NULL");
        return DH2_EINVAL;
    }
    std::memset(opt, 0, sizeof(*opt));
    opt->eta1 = 10.0;
    opt->leaf_max = 32;
    opt->precision = DH2_MIXED;
    opt->rank_rule = DH2_RANK_BLOCKREL;
    opt->qr_fp64 = 1;
    opt->svd_fp64 = 1;
    opt->gram_tc = 1;
    opt->fault = DH2_FAULT_NONE;
    opt->symmetry = 1;
    opt->qr_group_rows = 0;
    opt->workspace_bytes = 0;
    opt->tensor_cores = 1;
    opt->kb_store = 0;
    opt->learned = 0;
    opt->model = nullptr;
    opt->qr_tpc[0] = opt->qr_tpc[1] = opt->qr_tpc[2] = 0;
    return DH2_OK;
}

dh2_status dh2_build_tree(const double* vertices, int64_t nv, const int32_t* triangles, int64_t nt,
                          const dh2_options* opt, void* stream, dh2_tree* out) {
    return guarded([&] {
        DH2_REQUIRE(out != nullptr, "dh2_build_tree: out is NULL");
        *out = nullptr;
        DH2_REQUIRE(vertices != nullptr && nv > 0, "dh2_build_tree: no vertices");
        DH2_REQUIRE(nv < (int64_t(1) << 30), "dh2_build_tree: too many vertices");
        dh2_options o;
        if (opt) o = *opt; else dh2_options_default(&o);
        DH2_REQUIRE(o.leaf_max >= 1, "dh2_build_tree: leaf_max must be >= 1");
        const bool point_mode = triangles == nullptr;
        const int64_t n = point_mode ? nv : nt;
        DH2_REQUIRE(n > 0, "dh2_build_tree: no elements");
        DH2_REQUIRE(n < (int64_t(1) << 29), "dh2_build_tree: too many elements");
        for (int64_t i = 0; i < 3 * nv; ++i)
            DH2_REQUIRE(std::isfinite(vertices[i]), "dh2_build_tree: non-finite vertex coordinate");
        if (!point_mode)
            for (int64_t i = 0; i < 3 * nt; ++i)
                DH2_REQUIRE(triangles[i] >= 0 && triangles[i] < nv, "dh2_build_tree: vertex id out of range");
        cudaStream_t s = as_stream(stream);
        AllocScope scope(s);
        auto h = std::make_unique<dh2_tree_s>();
        Tree& tr = h->tr;
        tr.n = n;
        tr.nv = nv;
        tr.leaf_max = o.leaf_max;
        tr.point_mode = point_mode;
        tr.vert.alloc(3 * nv);
        tr.vert.upload(vertices, 3 * nv, s);
        if (!point_mode) {
            tr.tri.alloc(3 * nt);
            tr.tri.upload(triangles, 3 * nt, s);
        }
        build_tree_gpu(tr, s);
        prepare_quadrature(tr, s);
        DH2_CHECK_CUDA(cudaStreamSynchronize(s));
        *out = h.release();
    });
}

dh2_status dh2_build_dh2(dh2_tree tree, double kappa, int32_t m, double eta, double eps,
                         const dh2_options* opt, void* stream, dh2_matrix* out) {
    return guarded([&] {
        DH2_REQUIRE(out != nullptr, "dh2_build_dh2: out is NULL");
        *out = nullptr;
        dh2_options o;
        if (opt) o = *opt; else dh2_options_default(&o);
        check_build_args(tree, kappa, m, eta, eps, o, "dh2_build_dh2");
        cudaStream_t s = as_stream(stream);
        AllocScope scope(s);
        *out = build_matrix(tree, kappa, m, eta, eps, o, s);
    });
}

dh2_status dh2_build_dh2_batch(const dh2_tree* trees, int32_t count, const double* kappas, int32_t m,
                               double eta, double eps, const dh2_options* opt, int32_t nstreams,
                               dh2_matrix* out) {
    return guarded([&] {
        DH2_REQUIRE(count >= 0, "dh2_build_dh2_batch: count must be >= 0");
        DH2_REQUIRE(count == 0 || (trees != nullptr && kappas != nullptr && out != nullptr),
                    "dh2_build_dh2_batch: NULL array");
        DH2_REQUIRE(nstreams >= 0, "dh2_build_dh2_batch: nstreams must be >= 0");
        for (int32_t i = 0; i < count; ++i) out[i] = nullptr;
        dh2_options o;
        if (opt) o = *opt; else dh2_options_default(&o);
        for (int32_t i = 0; i < count; ++i) check_build_args(trees[i], kappas[i], m, eta, eps, o, "dh2_build_dh2_batch");
        if (count == 0) return;
        // largest meshes first, so that the small ones fill in at the end
        std::vector<int32_t> order(count);
        std::iota(order.begin(), order.end(), 0);
        std::stable_sort(order.begin(), order.end(),
                         [&](int32_t a, int32_t b) { return trees[a]->tr.n > trees[b]->tr.n; });
        const int nw = std::min<int>(count, nstreams > 0 ? nstreams : 8);
        int dev = 0;
        DH2_CHECK_CUDA(cudaGetDevice(&dev));
        std::atomic<int32_t> next{0};
        std::atomic<bool> failed{false};
        std::mutex mu;
        dh2_status first = DH2_OK;
        std::string first_msg;
        auto fail = [&](dh2_status st, const std::string& msg) {
            std::lock_guard<std::mutex> lk(mu);
            if (first == DH2_OK) {
                first = st;
                first_msg = msg;
            }
            failed = true;
        };
        auto worker = [&] {
            cudaStream_t s = nullptr;
            try {
                DH2_CHECK_CUDA(cudaSetDevice(dev));
                DH2_CHECK_CUDA(cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking));
                AllocScope scope(s);
                for (;;) {
                    const int32_t j = next.fetch_add(1);
                    if (j >= count || failed) break;
                    const int32_t i = order[j];
                    out[i] = build_matrix(trees[i], kappas[i], m, eta, eps, o, s);
                }
            } catch (const Error& e) {
                fail(e.status, e.msg);
            } catch (const std::bad_alloc&) {
                fail(DH2_ENOMEM, "host allocation failed");
            } catch (const std::exception& e) {
                fail(DH2_ECUDA, e.what());
            }
            if (s) {
                cudaStreamSynchronize(s);
                cudaStreamDestroy(s);
            }
        };
        std::vector<std::thread> pool;
        for (int w = 0; w < nw; ++w) pool.emplace_back(worker);
        for (auto& t : pool) t.join();
        if (failed) {
            cudaDeviceSynchronize();
            for (int32_t i = 0; i < count; ++i) {
                delete out[i];
                out[i] = nullptr;
            }
        }
        if (failed) throw Error{first, "dh2_build_dh2_batch: " + first_msg};
    });
}

dh2_status dh2_matvec(dh2_matrix mat, const void* x, void* y, int32_t dtype, void* stream) {
    return guarded([&] {
        DH2_REQUIRE(mat != nullptr && mat->num, "dh2_matvec: matrix is NULL");
        DH2_REQUIRE(x != nullptr && y != nullptr, "dh2_matvec: NULL vector");
        DH2_REQUIRE(dtype == DH2_C64 || dtype == DH2_C128, "dh2_matvec: dtype must be DH2_C64 or DH2_C128");
        DH2_REQUIRE(x != y, "dh2_matvec: x and y must not alias");
        mat->num->matvec(x, y, dtype, as_stream(stream));
    });
}

dh2_status dh2_matvec_noalloc(dh2_matrix mat, const void* x, void* y, int32_t dtype, void* stream) {
    return guarded([&] {
        DH2_REQUIRE(mat != nullptr && mat->num, "dh2_matvec_noalloc: matrix is NULL");
        DH2_REQUIRE(x != nullptr && y != nullptr, "dh2_matvec_noalloc: NULL vector");
        DH2_REQUIRE(dtype == DH2_C64 || dtype == DH2_C128, "dh2_matvec_noalloc: dtype must be DH2_C64 or DH2_C128");
        DH2_REQUIRE(x != y, "dh2_matvec_noalloc: x and y must not alias");
        mat->num->matvec_noalloc(x, y, dtype, as_stream(stream));
    });
}

dh2_status dh2_matvec_batch(const dh2_matrix* mats, int32_t count, const void* const* x, void* const* y,
                            int32_t dtype, void* stream) {
    return guarded([&] {
        DH2_REQUIRE(count >= 0, "dh2_matvec_batch: count must be >= 0");
        DH2_REQUIRE(count == 0 || (mats != nullptr && x != nullptr && y != nullptr), "dh2_matvec_batch: NULL array");
        DH2_REQUIRE(dtype == DH2_C64 || dtype == DH2_C128, "dh2_matvec_batch: dtype must be DH2_C64 or DH2_C128");
        for (int32_t i = 0; i < count; ++i) {
            DH2_REQUIRE(mats[i] != nullptr && mats[i]->num, "dh2_matvec_batch: matrix is NULL");
            DH2_REQUIRE(x[i] != nullptr && y[i] != nullptr, "dh2_matvec_batch: NULL vector");
            DH2_REQUIRE(x[i] != y[i], "dh2_matvec_batch: x and y must not alias");
        }
        std::vector<dh2_matrix> sorted(mats, mats + count);
        std::sort(sorted.begin(), sorted.end());
        DH2_REQUIRE(std::adjacent_find(sorted.begin(), sorted.end()) == sorted.end(),
                    "dh2_matvec_batch: a matrix appears twice (its work buffers would be shared)");
        if (count == 0) return;
        cudaStream_t s = as_stream(stream);
        AllocScope scope(s);
        const int ns = std::min<int>(count, kBatchStreams);
        cudaEvent_t fork;
        DH2_CHECK_CUDA(cudaEventCreateWithFlags(&fork, cudaEventDisableTiming));
        DH2_CHECK_CUDA(cudaEventRecord(fork, s));
        for (int i = 0; i < ns; ++i) DH2_CHECK_CUDA(cudaStreamWaitEvent(batch_stream(i), fork, 0));
        cudaEventDestroy(fork);
        for (int32_t i = 0; i < count; ++i) mats[i]->num->matvec(x[i], y[i], dtype, batch_stream(i % ns));
        for (int i = 0; i < ns; ++i) {
            cudaEvent_t join;
            DH2_CHECK_CUDA(cudaEventCreateWithFlags(&join, cudaEventDisableTiming));
            DH2_CHECK_CUDA(cudaEventRecord(join, batch_stream(i)));
            DH2_CHECK_CUDA(cudaStreamWaitEvent(s, join, 0));
            cudaEventDestroy(join);
        }
    });
}

dh2_status dh2_matvec_host(dh2_matrix mat, const double* x_host, double* y_host, void* stream) {
    return guarded([&] {
        DH2_REQUIRE(mat != nullptr && mat->num, "dh2_matvec_host: matrix is NULL");
        DH2_REQUIRE(x_host != nullptr && y_host != nullptr, "dh2_matvec_host: NULL vector");
        cudaStream_t s = as_stream(stream);
        AllocScope scope(s);
        const int64_t n = mat->tr.n;
        DBuf<double> xd(2 * n), yd(2 * n);
        DH2_CHECK_CUDA(cudaMemcpyAsync(xd.p, x_host, 2 * n * sizeof(double), cudaMemcpyHostToDevice, s));
        mat->num->matvec(xd.p, yd.p, DH2_C128, s);
        DH2_CHECK_CUDA(cudaMemcpyAsync(y_host, yd.p, 2 * n * sizeof(double), cudaMemcpyDeviceToHost, s));
        DH2_CHECK_CUDA(cudaStreamSynchronize(s));
    });
}

dh2_status dh2_set_timing(dh2_matrix mat, int32_t on) {
    return guarded([&] {
        DH2_REQUIRE(mat != nullptr && mat->num, "dh2_set_timing: matrix is NULL");
        mat->num->set_timing(on != 0);
    });
}

dh2_status dh2_sync(void* stream) {
    return guarded([&] { DH2_CHECK_CUDA(cudaStreamSynchronize(as_stream(stream))); });
}

dh2_status dh2_release_cached(void) {
    return guarded([&] {
        int dev = 0;
        DH2_CHECK_CUDA(cudaGetDevice(&dev));
        DH2_CHECK_CUDA(cudaDeviceSynchronize());
        cudaMemPool_t pool;
        DH2_CHECK_CUDA(cudaDeviceGetDefaultMemPool(&pool, dev));
        DH2_CHECK_CUDA(cudaMemPoolTrimTo(pool, 0));
    });
}

dh2_status dh2_dense_rows(dh2_tree tree, double kappa, const int32_t* rows, int32_t count, const double* x,
                          double* out, void* stream) {
    return guarded([&] {
        DH2_REQUIRE(tree != nullptr && count >= 0, "dh2_dense_rows: NULL tree or count < 0");
        DH2_REQUIRE(!tree->tr.point_mode, "dh2_dense_rows: a point-mode tree has no Galerkin elements");
        DH2_REQUIRE(std::isfinite(kappa) && kappa >= 0.0, "dh2_dense_rows: kappa must be >= 0");
        if (count == 0) return;
        DH2_REQUIRE(rows != nullptr && x != nullptr && out != nullptr, "dh2_dense_rows: NULL");
        for (int32_t i = 0; i < count; ++i)
            DH2_REQUIRE(rows[i] >= 0 && rows[i] < tree->tr.n, "dh2_dense_rows: row out of range");
        cudaStream_t s = as_stream(stream);
        AllocScope scope(s);
        dense_rows(tree->tr, kappa, rows, count, x, out, s);
    });
}

dh2_status dh2_gram(const void* z, int64_t rows, int32_t cols, int64_t ld, int32_t gram_tc, void* g, void* stream) {
    return guarded([&] {
        DH2_REQUIRE(z != nullptr && g != nullptr, "dh2_gram: NULL");
        DH2_REQUIRE(rows >= 1 && rows <= INT32_MAX, "dh2_gram: rows must be in [1, 2^31)");
        DH2_REQUIRE(cols >= 1 && cols <= 512, "dh2_gram: cols must be in [1, 512]");
        DH2_REQUIRE(ld >= cols && ld <= INT32_MAX, "dh2_gram: ld must be in [cols, 2^31)");
        DH2_REQUIRE(gram_tc == 0 || gram_tc == 1, "dh2_gram: gram_tc must be 0 or 1");
        cudaStream_t s = as_stream(stream);
        AllocScope scope(s);
        gram_matrix(z, rows, cols, ld, gram_tc != 0, g, s);
    });
}

dh2_status dh2_tree_get_info(dh2_tree tree, dh2_tree_info* out) {
    return guarded([&] {
        DH2_REQUIRE(tree != nullptr && out != nullptr, "dh2_tree_get_info: NULL");
        out->n = tree->tr.n;
        out->nclusters = tree->tr.nc;
        out->depth = tree->tr.depth;
    });
}

dh2_status dh2_tree_export(dh2_tree tree, int32_t* perm, int32_t* offset, int32_t* size, int32_t* parent,
                           int32_t* son0, int32_t* son1, int32_t* level, double* lo, double* hi) {
    return guarded([&] {
        DH2_REQUIRE(tree != nullptr, "dh2_tree_export: NULL tree");
        const Tree& tr = tree->tr;
        cudaStream_t s = 0;
        if (perm) tr.perm.download(perm, tr.n, s);
        if (offset) tr.offset.download(offset, tr.nc, s);
        if (size) tr.size.download(size, tr.nc, s);
        if (parent) tr.parent.download(parent, tr.nc, s);
        if (son0) tr.son0.download(son0, tr.nc, s);
        if (son1) tr.son1.download(son1, tr.nc, s);
        if (level) tr.level.download(level, tr.nc, s);
        std::vector<double> l = tr.lo.to_host(s), h = tr.hi.to_host(s);
        for (int32_t t = 0; t < tr.nc; ++t)
            for (int a = 0; a < 3; ++a) {
                if (lo) lo[3 * t + a] = l[(size_t)a * tr.nc + t];
                if (hi) hi[3 * t + a] = h[(size_t)a * tr.nc + t];
            }
        DH2_CHECK_CUDA(cudaStreamSynchronize(s));
    });
}

dh2_status dh2_matrix_get_info(dh2_matrix mat, dh2_matrix_info* out) {
    return guarded([&] {
        DH2_REQUIRE(mat != nullptr && out != nullptr && mat->num, "dh2_matrix_get_info: NULL");
        std::memset(out, 0, sizeof(*out));
        const auto& in = mat->num->info;
        out->n = mat->tr.n;
        out->depth = mat->tr.depth;
        out->m = mat->bp.m;
        out->k = mat->bp.m * mat->bp.m * mat->bp.m;
        out->nadm = mat->st.nadm;
        out->nnear = mat->st.nnear;
        out->npairs = mat->st.ntc;
        out->nactive = mat->st.nactive;
        out->near_entries = in.near_entries;
        out->coupling_entries = in.coupling_entries;
        out->basis_entries = in.basis_entries;
        out->matvec_bytes = in.matvec_bytes;
        out->max_rank_row = in.max_rank_row;
        out->max_rank_col = in.max_rank_col;
        out->mean_rank_row = in.mean_rank_row;
        out->mean_rank_col = in.mean_rank_col;
        for (int i = 0; i < 16; ++i) {
            out->stage_ms[i] = in.stage_ms[i];
            out->kernel_ms[i] = in.kernel_ms[i];
            out->kernel_launches[i] = in.kernel_launches[i];
            out->kernel_work[i] = in.kernel_work[i];
            out->kernel_work_kind[i] = in.kernel_work_kind[i];
        }
        out->learned_m = mat->learned_m;
        out->rank_cap_retries = in.rank_cap_retries;
        out->truncation_bytes = in.truncation_bytes;
        out->symmetric = in.symmetric;
        out->direct = mat->bp.direct;
        out->peak_pool_bytes = in.peak_pool_bytes;
    });
}

// ----------------------------------------------------------------------------- autotuner

dh2_status dh2_autotune(dh2_tree tree, double kappa, int32_t m, double eta, double eps, const dh2_options* base,
                        int32_t reps, void* stream, dh2_options* tuned, double* tuned_ms, double* base_ms) {
    return guarded([&] {
        DH2_REQUIRE(tuned != nullptr, "dh2_autotune: tuned is NULL");
        DH2_REQUIRE(reps >= 1, "dh2_autotune: reps must be >= 1");
        dh2_options o;
        if (base) o = *base; else dh2_options_default(&o);
        check_build_args(tree, kappa, m, eta, eps, o, "dh2_autotune");
        cudaStream_t s = as_stream(stream);
        AllocScope scope(s);
        // QR time per build (CUDA events of the QR kernels), averaged over reps builds
        auto score = [&](const dh2_options& c) {
            double ms = 0;
            for (int r = 0; r < reps; ++r) {
                std::unique_ptr<dh2_matrix_s> mat(build_matrix(tree, kappa, m, eta, eps, c, s));
                ms += mat->num->info.kernel_ms[K_TSQR] + mat->num->info.kernel_ms[K_TSQR_NARROW];
            }
            return ms / reps;
        };
        {   // warm-up build
            std::unique_ptr<dh2_matrix_s> warm(build_matrix(tree, kappa, m, eta, eps, o, s));
        }
        dh2_options best = o;
        const double t0 = score(best);
        double tb = t0;
        static const int width[3] = {32, 64, 128};
        for (int c = 0; c < 3; ++c) {
            for (int v : {1, 2, 4, 8}) {
                if (v * width[c] > 256) continue;
                dh2_options cand = best;
                cand.qr_tpc[c] = v;
                if (cand.qr_tpc[c] == best.qr_tpc[c] ||
                    (best.qr_tpc[c] == 0 && v == (c == 0 ? 8 : c == 1 ? 4 : 2)))
                    continue;   // the current choice, already scored
                const double t = score(cand);
                if (t < tb) {
                    tb = t;
                    best = cand;
                }
            }
        }
        for (int g : {512, 1024, 2048, 4096}) {
            dh2_options cand = best;
            cand.qr_group_rows = g;
            if (g == (best.qr_group_rows > 0 ? best.qr_group_rows : 1024)) continue;
            const double t = score(cand);
            if (t < tb) {
                tb = t;
                best = cand;
            }
        }
        *tuned = best;
        if (tuned_ms) *tuned_ms = tb;
        if (base_ms) *base_ms = t0;
    });
}

// ----------------------------------------------------------------------------- learned model

dh2_status dh2_model_create(const float* params, void* stream, dh2_model* out) {
    return guarded([&] {
        DH2_REQUIRE(out != nullptr, "dh2_model_create: out is NULL");
        *out = nullptr;
        DH2_REQUIRE(params != nullptr, "dh2_model_create: params is NULL");
        for (int i = 0; i < learned::kParams; ++i)
            DH2_REQUIRE(std::isfinite(params[i]), "dh2_model_create: non-finite parameter");
        cudaStream_t s = as_stream(stream);
        AllocScope scope(s);
        auto h = std::make_unique<dh2_model_s>();
        learned::model_init(h->md, params, s);
        DH2_CHECK_CUDA(cudaStreamSynchronize(s));
        *out = h.release();
    });
}

dh2_status dh2_model_get_params(dh2_model model, float* params) {
    return guarded([&] {
        DH2_REQUIRE(model != nullptr && params != nullptr, "dh2_model_get_params: NULL");
        model->md.master.download(params, learned::kParams, 0);
        DH2_CHECK_CUDA(cudaStreamSynchronize(0));
    });
}

dh2_status dh2_model_forward(dh2_model model, const float* X, int64_t n, float* Y, void* stream) {
    return guarded([&] {
        DH2_REQUIRE(model != nullptr && n >= 0, "dh2_model_forward: NULL model or n < 0");
        if (n == 0) return;
        DH2_REQUIRE(X != nullptr && Y != nullptr, "dh2_model_forward: NULL");
        cudaStream_t s = as_stream(stream);
        AllocScope scope(s);
        learned::model_forward(model->md, X, n, Y, s);
    });
}

dh2_status dh2_model_grad(dh2_model model, const float* X, const float* T, int64_t n, float* grad, float* loss,
                          void* stream) {
    return guarded([&] {
        DH2_REQUIRE(model != nullptr && X != nullptr && T != nullptr && grad != nullptr && loss != nullptr,
                    "dh2_model_grad: NULL");
        DH2_REQUIRE(n > 0, "dh2_model_grad: n must be > 0");
        cudaStream_t s = as_stream(stream);
        AllocScope scope(s);
        learned::model_grad(model->md, X, T, n, false, 0.f, s);
        DH2_CHECK_CUDA(cudaMemcpyAsync(grad, model->md.grad.p, learned::kParams * sizeof(float),
                                       cudaMemcpyDeviceToDevice, s));
        DH2_CHECK_CUDA(cudaMemcpyAsync(loss, model->md.loss.p, sizeof(float), cudaMemcpyDeviceToDevice, s));
    });
}

dh2_status dh2_model_train_step(dh2_model model, const float* X, const float* T, int64_t n, float lr, float* loss,
                                void* stream) {
    return guarded([&] {
        DH2_REQUIRE(model != nullptr && X != nullptr && T != nullptr, "dh2_model_train_step: NULL");
        DH2_REQUIRE(n > 0, "dh2_model_train_step: n must be > 0");
        DH2_REQUIRE(std::isfinite(lr) && lr > 0.f, "dh2_model_train_step: lr must be > 0");
        cudaStream_t s = as_stream(stream);
        AllocScope scope(s);
        learned::model_grad(model->md, X, T, n, true, lr, s);
        if (loss)
            DH2_CHECK_CUDA(cudaMemcpyAsync(loss, model->md.loss.p, sizeof(float), cudaMemcpyDeviceToDevice, s));
    });
}

void dh2_free_model(dh2_model model) {
    if (!model) return;
    cudaDeviceSynchronize();
    delete model;
}

namespace {
// the block structure of (tree, kappa, eta) for the learned-model helpers
struct ProbeStructure {
    Structure st;
    HostStructure hs;
};
void learned_structure(dh2_tree tree, double kappa, double eta, const dh2_options* opt, cudaStream_t s,
                       const char* fn, ProbeStructure& ps) {
    dh2_options o;
    if (opt) o = *opt; else dh2_options_default(&o);
    o.learned = 0;
    check_build_args(tree, kappa, 1, eta, 1.0, o, fn);
    build_structure(tree->tr, ps.st, kappa, o.eta1, eta, s);
    download_structure(tree->tr, ps.st, ps.hs, s);
}
}  // namespace

dh2_status dh2_learned_features(dh2_tree tree, double kappa, double eta, const dh2_options* opt, void* stream,
                                float* features, int64_t cap, int64_t* npairs, int8_t* active) {
    return guarded([&] {
        DH2_REQUIRE(npairs != nullptr, "dh2_learned_features: npairs is NULL");
        cudaStream_t s = as_stream(stream);
        AllocScope scope(s);
        ProbeStructure ps;
        learned_structure(tree, kappa, eta, opt, s, "dh2_learned_features", ps);
        *npairs = ps.st.ntc;
        if (!features) return;
        DH2_REQUIRE(cap >= ps.st.ntc, "dh2_learned_features: cap < number of pairs");
        learned::features(tree->tr, ps.st, features, s);
        if (active)
            for (int64_t tc = 0; tc < ps.st.ntc; ++tc) active[tc] = ps.hs.aidx[tc] >= 0 ? 1 : 0;
    });
}

dh2_status dh2_learned_probe(dh2_tree tree, double kappa, double eta, const dh2_options* opt, void* stream,
                             double* err, int64_t cap, int64_t* npairs) {
    return guarded([&] {
        DH2_REQUIRE(npairs != nullptr, "dh2_learned_probe: npairs is NULL");
        cudaStream_t s = as_stream(stream);
        AllocScope scope(s);
        ProbeStructure ps;
        learned_structure(tree, kappa, eta, opt, s, "dh2_learned_probe", ps);
        *npairs = ps.st.ntc;
        if (!err) return;
        DH2_REQUIRE(cap >= ps.st.ntc, "dh2_learned_probe: cap < number of pairs");
        DBuf<double> d((size_t)std::max<int64_t>(ps.st.ntc, 1) * learned::kOrders);
        learned::probe(tree->tr, ps.st, ps.hs, d.p, s);
        d.download(err, (size_t)ps.st.ntc * learned::kOrders, s);
        DH2_CHECK_CUDA(cudaStreamSynchronize(s));
    });
}

dh2_status dh2_export_directions(dh2_matrix mat, int32_t level, int32_t* count, int32_t* msplit, double* dirs,
                                 int32_t* sd) {
    return guarded([&] {
        DH2_REQUIRE(mat != nullptr && count != nullptr, "dh2_export_directions: NULL");
        const Structure& st = mat->st;
        DH2_REQUIRE(level >= 0 && level <= st.depth, "dh2_export_directions: level out of range");
        *count = st.ndir[level];
        if (msplit) *msplit = st.msplit[level];
        cudaStream_t s = 0;
        if (dirs)
            DH2_CHECK_CUDA(cudaMemcpyAsync(dirs, st.dirs.p + 3 * (size_t)st.dir_off[level],
                                           3 * st.ndir[level] * sizeof(double), cudaMemcpyDeviceToHost, s));
        if (sd)
            DH2_CHECK_CUDA(cudaMemcpyAsync(sd, st.sd.p + st.dir_off[level], st.ndir[level] * sizeof(int32_t),
                                           cudaMemcpyDeviceToHost, s));
        DH2_CHECK_CUDA(cudaStreamSynchronize(s));
    });
}

dh2_status dh2_export_blocks(dh2_matrix mat, int32_t* adm, int32_t* near, int8_t* active) {
    return guarded([&] {
        DH2_REQUIRE(mat != nullptr, "dh2_export_blocks: NULL");
        const HostStructure& h = mat->hs;
        if (adm)
            for (size_t b = 0; b < h.adm_t.size(); ++b) {
                adm[3 * b] = h.adm_t[b];
                adm[3 * b + 1] = h.adm_s[b];
                adm[3 * b + 2] = h.adm_c[b];
            }
        if (near)
            for (size_t b = 0; b < h.near_t.size(); ++b) {
                near[2 * b] = h.near_t[b];
                near[2 * b + 1] = h.near_s[b];
            }
        if (active)
            for (size_t tc = 0; tc < h.aidx.size(); ++tc) active[tc] = h.aidx[tc] >= 0 ? 1 : 0;
    });
}

dh2_status dh2_export_pair(dh2_matrix mat, int32_t which, int64_t tc, double* out, int64_t cap, int32_t* rows,
                           int32_t* cols) {
    return guarded([&] {
        DH2_REQUIRE(mat != nullptr && mat->num && out != nullptr && rows != nullptr && cols != nullptr,
                    "dh2_export_pair: NULL");
        mat->num->export_pair(which, tc, out, cap, rows, cols, 0);
    });
}

dh2_status dh2_export_ranks(dh2_matrix mat, int32_t* rank_row, int32_t* rank_col) {
    return guarded([&] {
        DH2_REQUIRE(mat != nullptr && mat->num, "dh2_export_ranks: NULL");
        mat->num->export_ranks(rank_row, rank_col, 0);
    });
}

// Work on any stream may still read the object: wait for the device before its memory
// goes back to the pool.
void dh2_free_tree(dh2_tree tree) {
    if (!tree) return;
    cudaDeviceSynchronize();
    delete tree;
}
void dh2_free_matrix(dh2_matrix mat) {
    if (!mat) return;
    cudaDeviceSynchronize();
    delete mat;
}

}  // extern "C"
