// Scans, stable key sorts and exact reductions used to lay out the ragged
// structures (CUB device-wide primitives).
#include <cub/cub.cuh>

#include "common.cuh"

namespace dh2 {

namespace {
struct TempStorage {
    DBuf<unsigned char> buf;
    void* get(size_t bytes) {
        buf.reserve(bytes ? bytes : 1);
        return buf.p;
    }
};
thread_local TempStorage g_tmp;
}  // namespace

int64_t exclusive_scan_i32(const int32_t* in, int32_t* out, int64_t n, cudaStream_t s) {
    if (n <= 0) return 0;
    size_t bytes = 0;
    DH2_CHECK_CUDA(cub::DeviceScan::ExclusiveSum(nullptr, bytes, in, out, (int)n, s));
    void* tmp = g_tmp.get(bytes);
    DH2_CHECK_CUDA(cub::DeviceScan::ExclusiveSum(tmp, bytes, in, out, (int)n, s));
    int32_t last_in = read_scalar(in + n - 1, s);
    int32_t last_out = read_scalar(out + n - 1, s);
    return (int64_t)last_in + (int64_t)last_out;
}

int64_t exclusive_scan_i64(const int64_t* in, int64_t* out, int64_t n, cudaStream_t s) {
    if (n <= 0) return 0;
    size_t bytes = 0;
    DH2_CHECK_CUDA(cub::DeviceScan::ExclusiveSum(nullptr, bytes, in, out, (int)n, s));
    void* tmp = g_tmp.get(bytes);
    DH2_CHECK_CUDA(cub::DeviceScan::ExclusiveSum(tmp, bytes, in, out, (int)n, s));
    int64_t last_in = read_scalar(in + n - 1, s);
    int64_t last_out = read_scalar(out + n - 1, s);
    return last_in + last_out;
}

void sort_pairs_i32(const int32_t* keys_in, int32_t* keys_out, const int32_t* vals_in,
                    int32_t* vals_out, int64_t n, int key_bits, cudaStream_t s) {
    if (n <= 0) return;
    size_t bytes = 0;
    DH2_CHECK_CUDA(cub::DeviceRadixSort::SortPairs(nullptr, bytes, keys_in, keys_out, vals_in,
                                                   vals_out, (int)n, 0, key_bits, s));
    void* tmp = g_tmp.get(bytes);
    DH2_CHECK_CUDA(cub::DeviceRadixSort::SortPairs(tmp, bytes, keys_in, keys_out, vals_in,
                                                   vals_out, (int)n, 0, key_bits, s));
}

namespace {
struct MaxOp {
    __device__ __forceinline__ double operator()(double a, double b) const { return a > b ? a : b; }
};
}  // namespace

double reduce_max_f64(const double* in, int64_t n, cudaStream_t s) {
    DBuf<double> out(1);
    size_t bytes = 0;
    DH2_CHECK_CUDA(cub::DeviceReduce::Reduce(nullptr, bytes, in, out.p, (int)n, MaxOp(), -1.0, s));
    void* tmp = g_tmp.get(bytes);
    DH2_CHECK_CUDA(cub::DeviceReduce::Reduce(tmp, bytes, in, out.p, (int)n, MaxOp(), -1.0, s));
    return read_scalar(out.p, s);
}

}  // namespace dh2
