// Internal declarations shared by the CUDA translation units of libdh2.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <cstdio>
#include <string>
#include <vector>

#include "../../include/dh2.h"

namespace dh2 {

// ----------------------------------------------------------------------------- errors

void set_error(const std::string& msg);

struct Error {
    dh2_status status;
    std::string msg;
};

#define DH2_CHECK_CUDA(call)                                                          \
    do {                                                                              \
        cudaError_t e_ = (call);                                                      \
        if (e_ != cudaSuccess)                                                        \
            throw ::dh2::Error{e_ == cudaErrorMemoryAllocation ? DH2_ENOMEM : DH2_ECUDA, \
                               std::string(#call) + ": " + cudaGetErrorString(e_)};   \
    } while (0)

// every kernel launch of the library is followed by DH2_CHECK_LAUNCH, which also counts it;
// graph replays add their kernels, graph captures take theirs back
void count_launch();
void count_launches(int64_t n);
void uncount_launches(int64_t n);
#define DH2_CHECK_LAUNCH(name)                                                        \
    do {                                                                              \
        ::dh2::count_launch();                                                        \
        cudaError_t e_ = cudaGetLastError();                                          \
        if (e_ != cudaSuccess)                                                        \
            throw ::dh2::Error{e_ == cudaErrorMemoryAllocation ? DH2_ENOMEM : DH2_ECUDA, \
                               std::string("launch of ") + (name) + ": " + cudaGetErrorString(e_)}; \
    } while (0)

// Raises the dynamic shared memory limit of kernel `fn` on the current device to at
// least `bytes`.  It never lowers it: the limit belongs to the kernel, not to a launch,
// and builds running concurrently on other threads rely on the limit they set.
void ensure_smem(const void* fn, size_t bytes);

#define DH2_REQUIRE(cond, msg)                                                        \
    do {                                                                              \
        if (!(cond)) throw ::dh2::Error{DH2_EINVAL, msg};                             \
    } while (0)

// ----------------------------------------------------------------------------- device memory

// Device memory comes from the device's default memory pool in stream order
// (cudaMallocAsync / cudaFreeAsync) on the stream of the entry point that is running,
// which every entry point sets with AllocScope for its duration (the legacy default
// stream otherwise).  Freeing then never waits for the whole device, so builds on
// different streams overlap.  The pool keeps up to a quarter of the device's memory of
// freed blocks for reuse (its release threshold).
inline cudaStream_t& alloc_stream() {
    thread_local cudaStream_t s = nullptr;
    return s;
}

struct AllocScope {
    cudaStream_t prev;
    explicit AllocScope(cudaStream_t s) : prev(alloc_stream()) { alloc_stream() = s; }
    ~AllocScope() { alloc_stream() = prev; }
    AllocScope(const AllocScope&) = delete;
    AllocScope& operator=(const AllocScope&) = delete;
};

void* dev_alloc(size_t bytes);   // throws Error (DH2_ENOMEM / DH2_ECUDA)
bool& fault_alloc_pending();     // test hook: the calling thread's next dev_alloc fails
void dev_free(void* p);          // errors are ignored (used from destructors)

// Owning device allocation (see above); moves only.
template <class T>
struct DBuf {
    T* p = nullptr;
    size_t n = 0;
    DBuf() = default;
    explicit DBuf(size_t count) { alloc(count); }
    DBuf(const DBuf&) = delete;
    DBuf& operator=(const DBuf&) = delete;
    DBuf(DBuf&& o) noexcept : p(o.p), n(o.n) { o.p = nullptr; o.n = 0; }
    DBuf& operator=(DBuf&& o) noexcept {
        if (this != &o) { release(); p = o.p; n = o.n; o.p = nullptr; o.n = 0; }
        return *this;
    }
    ~DBuf() { release(); }
    void alloc(size_t count) {
        release();
        n = count;
        if (count) p = static_cast<T*>(dev_alloc(count * sizeof(T)));
    }
    // grow-only reallocation (contents are not kept)
    void reserve(size_t count) { if (count > n) alloc(count); }
    void release() {
        if (p) dev_free(p);
        p = nullptr;
        n = 0;
    }
    void zero(cudaStream_t s) { if (n) DH2_CHECK_CUDA(cudaMemsetAsync(p, 0, n * sizeof(T), s)); }
    void upload(const T* h, size_t count, cudaStream_t s) {
        if (count) DH2_CHECK_CUDA(cudaMemcpyAsync(p, h, count * sizeof(T), cudaMemcpyHostToDevice, s));
    }
    void download(T* h, size_t count, cudaStream_t s) const {
        if (count) DH2_CHECK_CUDA(cudaMemcpyAsync(h, p, count * sizeof(T), cudaMemcpyDeviceToHost, s));
    }
    std::vector<T> to_host(cudaStream_t s, size_t count = (size_t)-1) const {
        if (count == (size_t)-1) count = n;
        std::vector<T> h(count);
        download(h.data(), count, s);
        DH2_CHECK_CUDA(cudaStreamSynchronize(s));
        return h;
    }
};

template <class T>
T read_scalar(const T* dptr, cudaStream_t s) {
    T h;
    DH2_CHECK_CUDA(cudaMemcpyAsync(&h, dptr, sizeof(T), cudaMemcpyDeviceToHost, s));
    DH2_CHECK_CUDA(cudaStreamSynchronize(s));
    return h;
}

inline unsigned grid_for(int64_t n, int threads) {
    int64_t g = (n + threads - 1) / threads;
    if (g < 1) g = 1;
    return (unsigned)g;
}

// ----------------------------------------------------------------------------- scans (scan.cu)

// out[i] = sum_{j<i} in[j]; returns the total (synchronises the stream).
int64_t exclusive_scan_i32(const int32_t* in, int32_t* out, int64_t n, cudaStream_t s);
int64_t exclusive_scan_i64(const int64_t* in, int64_t* out, int64_t n, cudaStream_t s);
// Stable sort of (key, value) pairs by key (keys in [0, 2^key_bits)).
void sort_pairs_i32(const int32_t* keys_in, int32_t* keys_out, const int32_t* vals_in,
                    int32_t* vals_out, int64_t n, int key_bits, cudaStream_t s);
// max of a double array (exact)
double reduce_max_f64(const double* in, int64_t n, cudaStream_t s);

// ----------------------------------------------------------------------------- tree

struct Tree {
    int64_t n = 0;            // elements
    int64_t nv = 0;
    int32_t leaf_max = 32;
    bool point_mode = false;
    int32_t nc = 0;           // clusters
    int32_t depth = 0;
    std::vector<int32_t> level_start;   // host copy, depth+2 entries
    DBuf<double> vert;        // [nv][3]
    DBuf<int32_t> tri;        // [n][3]
    DBuf<double> cent;        // SoA [3][n]
    DBuf<double> tlo, thi;    // SoA [3][n] per-element vertex boxes
    DBuf<int32_t> perm;       // [n]
    DBuf<int32_t> offset, size, parent, son0, son1, level;   // [nc]
    DBuf<double> lo, hi;      // SoA [3][nc]
    // quadrature data (element order, not cluster order)
    DBuf<double> area;        // [n]
    DBuf<double> x3;          // [n][3 points][3]
    DBuf<double> x7;          // [n][7 points][3]
};

void build_tree_gpu(Tree& tr, cudaStream_t s);
void prepare_quadrature(Tree& tr, cudaStream_t s);
// out_host[i] = (G x)[rows_host[i]] in FP64 (dense.cu); x_dev complex128, original order
void dense_rows(const Tree& tr, double kappa, const int32_t* rows_host, int32_t count, const double* x_dev,
                double* out_host, cudaStream_t s);
// g = Z^* Z (cols x cols complex FP64) of a complex FP32 matrix (numeric.cu); tc: tensor-core
// digit products for more than 32 columns
void gram_matrix(const void* z, int64_t rows, int32_t cols, int64_t ld, bool tc, void* g, cudaStream_t s);

}  // namespace dh2
