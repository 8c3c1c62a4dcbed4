// Reference rows of the Galerkin matrix (Eq. 2), FP64 on the GPU: (G x)[rows] with the
// quadrature of the nearfield (3 x 3 interior Gauss points off the diagonal, the 7-point
// degree-5 rule against the 3-point rule on it), used to measure the error of the
// compressed product on sampled rows.
#include <cmath>
#include <mutex>

#include "common.cuh"

namespace dh2 {

namespace {

__constant__ double c_w7r[7];

__device__ __forceinline__ double2 g_helm(double d0, double d1, double d2, double kappa) {
    const double r = sqrt(d0 * d0 + d1 * d1 + d2 * d2);
    double sn, cs;
    sincos(kappa * r, &sn, &cs);
    const double w = 1.0 / (4.0 * 3.14159265358979323846 * r);
    return make_double2(cs * w, sn * w);
}

// one CTA per requested row; threads stride over the columns; FP64 block sum
__global__ void k_dense_rows(const int32_t* __restrict__ rows, int64_t n, const double* __restrict__ area,
                             const double* __restrict__ x3, const double* __restrict__ x7, double kappa,
                             const double2* __restrict__ x, double2* __restrict__ out) {
    const int64_t i = rows[blockIdx.x];
    double sr = 0.0, si = 0.0;
    for (int64_t j = threadIdx.x; j < n; j += blockDim.x) {
        double er = 0.0, ei = 0.0;
        if (j != i) {
            for (int p = 0; p < 3; ++p)
                for (int q = 0; q < 3; ++q) {
                    const double* a = x3 + (i * 3 + p) * 3;
                    const double* b = x3 + (j * 3 + q) * 3;
                    const double2 g = g_helm(a[0] - b[0], a[1] - b[1], a[2] - b[2], kappa);
                    er += g.x;
                    ei += g.y;
                }
            const double w = area[i] / 3.0 * (area[j] / 3.0);
            er *= w;
            ei *= w;
        } else {
            for (int p = 0; p < 7; ++p)
                for (int q = 0; q < 3; ++q) {
                    const double* a = x7 + (i * 7 + p) * 3;
                    const double* b = x3 + (i * 3 + q) * 3;
                    const double2 g = g_helm(a[0] - b[0], a[1] - b[1], a[2] - b[2], kappa);
                    const double w = c_w7r[p] / 3.0;
                    er += w * g.x;
                    ei += w * g.y;
                }
            const double a2 = area[i] * area[i];
            er *= a2;
            ei *= a2;
        }
        const double2 xv = x[j];
        sr += er * xv.x - ei * xv.y;
        si += er * xv.y + ei * xv.x;
    }
    __shared__ double red[2][32];
    for (int o = 16; o; o >>= 1) {
        sr += __shfl_xor_sync(0xffffffffu, sr, o);
        si += __shfl_xor_sync(0xffffffffu, si, o);
    }
    if ((threadIdx.x & 31) == 0) {
        red[0][threadIdx.x >> 5] = sr;
        red[1][threadIdx.x >> 5] = si;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double ar = 0.0, ai = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) {
            ar += red[0][w];
            ai += red[1][w];
        }
        out[blockIdx.x] = make_double2(ar, ai);
    }
}

}  // namespace

void dense_rows(const Tree& tr, double kappa, const int32_t* rows_host, int32_t count, const double* x_dev,
                double* out_host, cudaStream_t s) {
    static std::mutex mu;
    static bool ready[64] = {};
    int dev = 0;
    DH2_CHECK_CUDA(cudaGetDevice(&dev));
    std::unique_lock<std::mutex> lk(mu);
    if (dev >= 64 || !ready[dev]) {
        // Radon's 7-point degree-5 rule (Stroud T2:5-1), weights relative to the area, in the
        // point order of the quadrature nodes x7: centroid, then the two orbits
        const double s15 = std::sqrt(15.0);
        const double w7[7] = {9.0 / 40.0,           (155.0 - s15) / 1200.0, (155.0 - s15) / 1200.0,
                              (155.0 - s15) / 1200.0, (155.0 + s15) / 1200.0, (155.0 + s15) / 1200.0,
                              (155.0 + s15) / 1200.0};
        DH2_CHECK_CUDA(cudaMemcpyToSymbol(c_w7r, w7, sizeof(w7)));
        if (dev < 64) ready[dev] = true;
    }
    lk.unlock();
    if (count == 0) return;
    DBuf<int32_t> r(count);
    r.upload(rows_host, count, s);
    DBuf<double2> o(count);
    k_dense_rows<<<(unsigned)count, 256, 0, s>>>(r.p, tr.n, tr.area.p, tr.x3.p, tr.x7.p, kappa,
                                                  reinterpret_cast<const double2*>(x_dev), o.p);
    DH2_CHECK_LAUNCH("k_dense_rows");
    DH2_CHECK_CUDA(cudaMemcpyAsync(out_host, o.p, (size_t)count * sizeof(double2), cudaMemcpyDeviceToHost, s));
    DH2_CHECK_CUDA(cudaStreamSynchronize(s));
}

}  // namespace dh2
