// Learned interpolation order and truncation rank: features, interpolation-error probe,
// MLP forward / backward / Adam (see learned.cuh).
#include <algorithm>
#include <cmath>

#include "learned.cuh"

namespace dh2 {
namespace learned {

namespace {

constexpr int kThreadsL = 256;

// ----------------------------------------------------------------------------- features

// One thread per pair (t, c); FP64 arithmetic, FP32 output:
//   f0 = kappa diam / eta1, f1 = cone angle / pi (atan(sqrt 2 / m_l), pi for D_l = {0}),
//   f2 = level / depth, f3..f5 = sorted box extents / diam, f6 = log2 #t / 16,
//   f7 = max over the admissible blocks of row(t, c) of diam_t / dist(B_t, B_s).
__global__ void k_features(int64_t ntc, const int32_t* __restrict__ tc_cluster, const int32_t* __restrict__ level,
                           const int32_t* __restrict__ size, const double* __restrict__ lo,
                           const double* __restrict__ hi, int32_t nc, const int32_t* __restrict__ msplit,
                           int32_t depth, const int32_t* __restrict__ row_ptr, const int32_t* __restrict__ row_idx,
                           const int32_t* __restrict__ adm_s, double kappa, double eta1, float* __restrict__ F) {
    const int64_t tc = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (tc >= ntc) return;
    const int32_t t = tc_cluster[tc];
    const int32_t l = level[t];
    const int32_t ml = msplit[l];
    double e[3];
    for (int a = 0; a < 3; ++a) e[a] = hi[(size_t)a * nc + t] - lo[(size_t)a * nc + t];
    const double dt = sqrt(__dadd_rn(__dadd_rn(__dmul_rn(e[0], e[0]), __dmul_rn(e[1], e[1])), __dmul_rn(e[2], e[2])));
    // three-element sort, descending
    if (e[0] < e[1]) { double x = e[0]; e[0] = e[1]; e[1] = x; }
    if (e[1] < e[2]) { double x = e[1]; e[1] = e[2]; e[2] = x; }
    if (e[0] < e[1]) { double x = e[0]; e[0] = e[1]; e[1] = x; }
    const double pi = 3.14159265358979323846;
    const double theta = ml > 0 ? atan(sqrt(2.0) / (double)ml) : pi;
    double close = 0.0;
    for (int32_t q = row_ptr[tc]; q < row_ptr[tc + 1]; ++q) {
        const int32_t sc = adm_s[row_idx[q]];
        double g2 = 0.0;
        for (int a = 0; a < 3; ++a) {
            const double ga = fmax(fmax(lo[(size_t)a * nc + t] - hi[(size_t)a * nc + sc],
                                        lo[(size_t)a * nc + sc] - hi[(size_t)a * nc + t]), 0.0);
            g2 = __dadd_rn(g2, __dmul_rn(ga, ga));
        }
        const double dist = sqrt(g2);
        if (dist > 0.0) close = fmax(close, dt / dist);
    }
    float* f = F + tc * kIn;
    f[0] = (float)(kappa * dt / eta1);
    f[1] = (float)(theta / pi);
    f[2] = depth > 0 ? (float)((double)l / (double)depth) : 0.0f;
    for (int a = 0; a < 3; ++a) f[3 + a] = dt > 0.0 ? (float)(e[a] / dt) : 0.0f;
    f[6] = (float)(log2((double)size[t]) / 16.0);
    f[7] = (float)close;
}

// ----------------------------------------------------------------------------- probe

constexpr int kProbeBlocks = 8, kProbeElems = 8, kProbePts = 3 * kProbeElems, kProbeYChunk = 8;

__device__ __forceinline__ double2 gc_val(const double* x, const double* y, const double* c, double kappa) {
    const double d0 = x[0] - y[0], d1 = x[1] - y[1], d2 = x[2] - y[2];
    const double r = sqrt(d0 * d0 + d1 * d1 + d2 * d2);
    const double dc = d0 * c[0] + d1 * c[1] + d2 * c[2];
    double sn, cs;
    sincos(kappa * (r - dc), &sn, &cs);
    const double w = 1.0 / (4.0 * 3.14159265358979323846 * r);
    return make_double2(cs * w, sn * w);
}

// sample points: the 3-point quadrature nodes of up to 8 elements of cluster t, at cluster
// positions offset + floor(j size / P), P = min(8, size)
__device__ int load_points(const double* __restrict__ x3, const int32_t* __restrict__ perm, int32_t off, int32_t size,
                           double (*pts)[3]) {
    const int P = min(kProbeElems, size);
    for (int q = threadIdx.x; q < 9 * P; q += blockDim.x) {
        const int j = q / 9, r = q % 9;
        const int32_t el = perm[off + (int32_t)(((int64_t)j * size) / P)];
        pts[3 * j + r / 3][r % 3] = x3[(size_t)el * 9 + r];
    }
    return 3 * P;
}

__device__ __forceinline__ double block_max(double v, double* red) {
    for (int o = 16; o; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
    __syncthreads();
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
    __syncthreads();
    double r = red[0];
    for (int w = 1; w < (int)(blockDim.x >> 5); ++w) r = fmax(r, red[w]);
    return r;
}

// One CTA per pair with admissible blocks.  For m = 3..8: Chebyshev nodes on the padded box
// of t (half-widths >= 1e-3 of the largest), Lagrange values at the x samples, then per
// block (first 8 of row(t, c)) g_c at (xi_nu, y) in shared memory, chunked over y, and the
// interpolant at every (x, y) against g_c(x, y).
__global__ void __launch_bounds__(kThreadsL) k_probe(
    const int32_t* __restrict__ tasks, const int32_t* __restrict__ tc_cluster, const int32_t* __restrict__ tc_base,
    const int32_t* __restrict__ level, const int32_t* __restrict__ offset, const int32_t* __restrict__ size,
    const int32_t* __restrict__ perm, const double* __restrict__ lo, const double* __restrict__ hi, int32_t nc,
    const double* __restrict__ x3, const double* __restrict__ dirs, const int32_t* __restrict__ dir_off,
    const int32_t* __restrict__ row_ptr, const int32_t* __restrict__ row_idx, const int32_t* __restrict__ adm_s,
    double kappa, double* __restrict__ err) {
    extern __shared__ double2 G[];   // [kProbeYChunk][k]
    __shared__ double X[kProbePts][3], Y[kProbePts][3];
    __shared__ double nodes[3][8];
    __shared__ double Lx[kProbePts][3][8];
    __shared__ double cvec[3];
    __shared__ double red[kThreadsL / 32];
    const int32_t tc = tasks[blockIdx.x];
    const int32_t t = tc_cluster[tc];
    const int32_t c = tc - tc_base[t];
    if (threadIdx.x < 3) cvec[threadIdx.x] = dirs[3 * ((size_t)dir_off[level[t]] + c) + threadIdx.x];
    const int nX = load_points(x3, perm, offset[t], size[t], X);
    const int32_t r0 = row_ptr[tc];
    const int nb = min(kProbeBlocks, row_ptr[tc + 1] - r0);
    for (int m = 3; m <= 8; ++m) {
        const int k = m * m * m;
        __syncthreads();
        if (threadIdx.x < 3) {
            const int a = threadIdx.x;
            double hmax = 0.0;
            for (int b = 0; b < 3; ++b) hmax = fmax(hmax, (hi[(size_t)b * nc + t] - lo[(size_t)b * nc + t]) * 0.5);
            const double mid = (lo[(size_t)a * nc + t] + hi[(size_t)a * nc + t]) * 0.5;
            const double half = fmax((hi[(size_t)a * nc + t] - lo[(size_t)a * nc + t]) * 0.5, 1e-3 * hmax);
            for (int j = 0; j < m; ++j) nodes[a][j] = mid + half * cos(3.14159265358979323846 * (2 * j + 1) / (2.0 * m));
        }
        __syncthreads();
        for (int q = threadIdx.x; q < nX * 3; q += blockDim.x) {
            const int x = q / 3, a = q % 3;
            for (int j = 0; j < m; ++j) {
                double v = 1.0;
                for (int i = 0; i < m; ++i)
                    if (i != j) v *= (X[x][a] - nodes[a][i]) / (nodes[a][j] - nodes[a][i]);
                Lx[x][a][j] = v;
            }
        }
        double worst = 0.0;
        for (int bi = 0; bi < nb; ++bi) {
            const int32_t s = adm_s[row_idx[r0 + bi]];
            __syncthreads();
            const int nY = load_points(x3, perm, offset[s], size[s], Y);
            double merr = 0.0, mabs = 0.0;
            for (int y0 = 0; y0 < nY; y0 += kProbeYChunk) {
                const int yc = min(kProbeYChunk, nY - y0);
                __syncthreads();
                for (int q = threadIdx.x; q < yc * k; q += blockDim.x) {
                    const int yy = q / k, nu = q % k;
                    const double xi[3] = {nodes[0][nu % m], nodes[1][(nu / m) % m], nodes[2][nu / (m * m)]};
                    G[q] = gc_val(xi, Y[y0 + yy], cvec, kappa);
                }
                __syncthreads();
                for (int q = threadIdx.x; q < nX * yc; q += blockDim.x) {
                    const int x = q / yc, yy = q % yc;
                    const double2* g = G + (size_t)yy * k;
                    double ar = 0.0, ai = 0.0;
                    for (int nz = 0; nz < m; ++nz) {
                        const double lz = Lx[x][2][nz];
                        for (int ny = 0; ny < m; ++ny) {
                            const double lzy = lz * Lx[x][1][ny];
                            const double2* gr = g + (nz * m + ny) * m;
                            for (int nx = 0; nx < m; ++nx) {
                                const double w = lzy * Lx[x][0][nx];
                                ar += w * gr[nx].x;
                                ai += w * gr[nx].y;
                            }
                        }
                    }
                    const double2 ex = gc_val(X[x], Y[y0 + yy], cvec, kappa);
                    merr = fmax(merr, hypot(ex.x - ar, ex.y - ai));
                    mabs = fmax(mabs, hypot(ex.x, ex.y));
                }
            }
            const double e = block_max(merr, red);
            const double a = block_max(mabs, red);
            if (a > 0.0) worst = fmax(worst, e / a);
        }
        if (threadIdx.x == 0) err[(size_t)tc * kOrders + (m - 3)] = worst;
    }
}

// ----------------------------------------------------------------------------- MLP

constexpr int kTile = 32;          // samples per tile
constexpr int kLd = kHid + 1;      // padded row of a [tile][128] activation array
constexpr int kMlpGrid = 152;      // CTAs of a gradient launch (one per SM)

struct MlpSmem {
    float W2[kHid * kLd];
    float W1[kHid * kIn];
    float W3[kOut * kHid];
    float b1[kHid], b2[kHid], b3[4];
    float x[kTile * kIn];
    float t[kTile * kOut];
    float h1[kTile * kLd], h2[kTile * kLd], d2[kTile * kLd], d1[kTile * kLd];
    float dy[kTile * kOut];
    float gb1[kHid], gb2[kHid], gb3[4], gloss[kThreadsL / 32];
};

// Forward over tiles of 32 samples (TRAIN = false: writes Y), or forward + backward with the
// gradient of this CTA's tiles accumulated and written to part[blockIdx.x][kParams + 1]
// (the last entry is the CTA's share of the loss).  Thread roles, with w = warp, l = lane:
// the 128 x 128 layer gives each thread samples 4w..4w+3 times neurons l + 32q (q < 4), and
// the weight gradient of that layer gives it rows 16w..16w+15 times columns l + 32q.
template <bool TRAIN>
__global__ void __launch_bounds__(kThreadsL, 1) k_mlp(const float* __restrict__ X, const float* __restrict__ T,
                                                       int64_t n, float inv_n, const float* __restrict__ master,
                                                       const __nv_bfloat16* __restrict__ wb, float* __restrict__ Y,
                                                       float* __restrict__ part) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    MlpSmem& S = *reinterpret_cast<MlpSmem*>(smem_raw);
    const int tid = threadIdx.x, w = tid >> 5, l = tid & 31;
    for (int e = tid; e < kHid * kHid; e += kThreadsL)
        S.W2[(e >> 7) * kLd + (e & 127)] = __bfloat162float(wb[kOffW2 + e]);
    for (int e = tid; e < kHid * kIn; e += kThreadsL) S.W1[e] = __bfloat162float(wb[kOffW1 + e]);
    for (int e = tid; e < kOut * kHid; e += kThreadsL) S.W3[e] = __bfloat162float(wb[kOffW3 + e]);
    if (tid < kHid) {
        S.b1[tid] = master[kOffB1 + tid];
        S.b2[tid] = master[kOffB2 + tid];
        S.gb1[tid] = 0.f;
        S.gb2[tid] = 0.f;
    }
    if (tid < 4) {
        S.b3[tid] = tid < kOut ? master[kOffB3 + tid] : 0.f;
        S.gb3[tid] = 0.f;
    }
    if (l == 0) S.gloss[w] = 0.f;
    float gW2[16][4];
    float gW1[4] = {0.f, 0.f, 0.f, 0.f};
    float gW3 = 0.f;
    if (TRAIN) {
#pragma unroll
        for (int r = 0; r < 16; ++r)
#pragma unroll
            for (int q = 0; q < 4; ++q) gW2[r][q] = 0.f;
    }
    for (int64_t tile = blockIdx.x; tile * kTile < n; tile += gridDim.x) {
        const int64_t s0 = tile * kTile;
        const int nv = (int)(n - s0 < (int64_t)kTile ? n - s0 : (int64_t)kTile);
        __syncthreads();
        {
            const int sa = tid >> 3, i = tid & 7;
            S.x[tid] = sa < nv ? X[(s0 + sa) * kIn + i] : 0.f;
            if (TRAIN && tid < kTile * kOut) {
                const int sb = tid >> 1, o = tid & 1;
                S.t[tid] = sb < nv ? T[(s0 + sb) * kOut + o] : 0.f;
            }
        }
        __syncthreads();
        // h1 = relu(W1 x + b1)
        for (int e = tid; e < kTile * kHid; e += kThreadsL) {
            const int sa = e >> 7, j = e & 127;
            float z = S.b1[j];
#pragma unroll
            for (int i = 0; i < kIn; ++i) z += S.W1[j * kIn + i] * S.x[sa * kIn + i];
            S.h1[sa * kLd + j] = fmaxf(z, 0.f);
        }
        __syncthreads();
        // h2 = relu(W2 h1 + b2)
        {
            float acc[4][4] = {};
            for (int i = 0; i < kHid; ++i) {
                float a[4], b[4];
#pragma unroll
                for (int r = 0; r < 4; ++r) a[r] = S.h1[(4 * w + r) * kLd + i];
#pragma unroll
                for (int q = 0; q < 4; ++q) b[q] = S.W2[(l + 32 * q) * kLd + i];
#pragma unroll
                for (int r = 0; r < 4; ++r)
#pragma unroll
                    for (int q = 0; q < 4; ++q) acc[r][q] += a[r] * b[q];
            }
#pragma unroll
            for (int r = 0; r < 4; ++r)
#pragma unroll
                for (int q = 0; q < 4; ++q) S.h2[(4 * w + r) * kLd + l + 32 * q] = fmaxf(acc[r][q] + S.b2[l + 32 * q], 0.f);
        }
        __syncthreads();
        // y = W3 h2 + b3: warp w takes samples 4w..4w+3
#pragma unroll
        for (int r = 0; r < 4; ++r) {
            const int sa = 4 * w + r;
#pragma unroll
            for (int o = 0; o < kOut; ++o) {
                float p = 0.f;
#pragma unroll
                for (int q = 0; q < 4; ++q) p += S.h2[sa * kLd + l + 32 * q] * S.W3[o * kHid + l + 32 * q];
                for (int off = 16; off; off >>= 1) p += __shfl_xor_sync(0xffffffffu, p, off);
                const float yv = p + S.b3[o];
                if (l == 0) {
                    if (!TRAIN) {
                        if (sa < nv) Y[(s0 + sa) * kOut + o] = yv;
                    } else {
                        const float diff = sa < nv ? yv - S.t[sa * kOut + o] : 0.f;
                        S.dy[sa * kOut + o] = diff * inv_n;
                        S.gloss[w] += 0.5f * diff * diff * inv_n;
                    }
                }
            }
        }
        if (!TRAIN) continue;
        __syncthreads();
        // W3 / b3 gradients and d2 = (W3^T dy) .* [h2 > 0]
        {
            const int o = tid >> 7, j = tid & 127;
            float g = 0.f;
            for (int sa = 0; sa < kTile; ++sa) g += S.dy[sa * kOut + o] * S.h2[sa * kLd + j];
            gW3 += g;
            if (tid < kOut) {
                float gb = 0.f;
                for (int sa = 0; sa < kTile; ++sa) gb += S.dy[sa * kOut + tid];
                S.gb3[tid] += gb;
            }
        }
        for (int e = tid; e < kTile * kHid; e += kThreadsL) {
            const int sa = e >> 7, j = e & 127;
            const float v = S.dy[sa * kOut] * S.W3[j] + S.dy[sa * kOut + 1] * S.W3[kHid + j];
            S.d2[sa * kLd + j] = S.h2[sa * kLd + j] > 0.f ? v : 0.f;
        }
        __syncthreads();
        if (tid < kHid) {
            float gb = 0.f;
            for (int sa = 0; sa < kTile; ++sa) gb += S.d2[sa * kLd + tid];
            S.gb2[tid] += gb;
        }
        // W2 gradient: rows 16w + r, columns l + 32q
        for (int sa = 0; sa < kTile; ++sa) {
            float a[16], b[4];
#pragma unroll
            for (int r = 0; r < 16; ++r) a[r] = S.d2[sa * kLd + 16 * w + r];
#pragma unroll
            for (int q = 0; q < 4; ++q) b[q] = S.h1[sa * kLd + l + 32 * q];
#pragma unroll
            for (int r = 0; r < 16; ++r)
#pragma unroll
                for (int q = 0; q < 4; ++q) gW2[r][q] += a[r] * b[q];
        }
        // d1 = (W2^T d2) .* [h1 > 0]
        {
            float acc[4][4] = {};
            for (int j = 0; j < kHid; ++j) {
                float a[4], b[4];
#pragma unroll
                for (int r = 0; r < 4; ++r) a[r] = S.d2[(4 * w + r) * kLd + j];
#pragma unroll
                for (int q = 0; q < 4; ++q) b[q] = S.W2[j * kLd + l + 32 * q];
#pragma unroll
                for (int r = 0; r < 4; ++r)
#pragma unroll
                    for (int q = 0; q < 4; ++q) acc[r][q] += a[r] * b[q];
            }
#pragma unroll
            for (int r = 0; r < 4; ++r)
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    const int idx = (4 * w + r) * kLd + l + 32 * q;
                    S.d1[idx] = S.h1[idx] > 0.f ? acc[r][q] : 0.f;
                }
        }
        __syncthreads();
        if (tid < kHid) {
            float gb = 0.f;
            for (int sa = 0; sa < kTile; ++sa) gb += S.d1[sa * kLd + tid];
            S.gb1[tid] += gb;
        }
#pragma unroll
        for (int p = 0; p < 4; ++p) {
            const int e = tid + kThreadsL * p, j = e >> 3, i = e & 7;
            float g = 0.f;
            for (int sa = 0; sa < kTile; ++sa) g += S.d1[sa * kLd + j] * S.x[sa * kIn + i];
            gW1[p] += g;
        }
    }
    if (!TRAIN) return;
    __syncthreads();
    float* out = part + (size_t)blockIdx.x * (kParams + 1);
#pragma unroll
    for (int p = 0; p < 4; ++p) out[kOffW1 + tid + kThreadsL * p] = gW1[p];
#pragma unroll
    for (int r = 0; r < 16; ++r)
#pragma unroll
        for (int q = 0; q < 4; ++q) out[kOffW2 + (16 * w + r) * kHid + l + 32 * q] = gW2[r][q];
    out[kOffW3 + tid] = gW3;
    if (tid < kHid) {
        out[kOffB1 + tid] = S.gb1[tid];
        out[kOffB2 + tid] = S.gb2[tid];
    }
    if (tid < kOut) out[kOffB3 + tid] = S.gb3[tid];
    if (tid == 0) {
        float L = 0.f;
        for (int q = 0; q < kThreadsL / 32; ++q) L += S.gloss[q];
        out[kParams] = L;
    }
}

// Sums the CTAs' partial gradients in a fixed order (deterministic), writes the gradient and
// the loss, and with ADAM takes one Adam step (beta1 0.9, beta2 0.999, eps 1e-8; c1, c2 the
// bias corrections 1 / (1 - beta^step)) and refreshes the BF16 weights.
template <bool ADAM>
__global__ void k_mlp_reduce(const float* __restrict__ part, int nparts, float* __restrict__ grad,
                             float* __restrict__ loss, float* __restrict__ master, float* __restrict__ mom1,
                             float* __restrict__ mom2, __nv_bfloat16* __restrict__ wb, float lr, float c1, float c2) {
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p > kParams) return;
    float g = 0.f;
    for (int c = 0; c < nparts; ++c) g += part[(size_t)c * (kParams + 1) + p];
    if (p == kParams) {
        *loss = g;
        return;
    }
    grad[p] = g;
    if (ADAM) {
        const float m1 = 0.9f * mom1[p] + 0.1f * g;
        const float m2 = 0.999f * mom2[p] + 0.001f * g * g;
        mom1[p] = m1;
        mom2[p] = m2;
        const float wv = master[p] - lr * (m1 * c1) / (sqrtf(m2 * c2) + 1e-8f);
        master[p] = wv;
        wb[p] = __float2bfloat16_rn(wv);
    }
}

__global__ void k_mlp_cast(const float* __restrict__ master, __nv_bfloat16* __restrict__ wb) {
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p < kParams) wb[p] = __float2bfloat16_rn(master[p]);
}

size_t mlp_smem() { return sizeof(MlpSmem); }

}  // namespace

void model_init(Model& md, const float* host_params, cudaStream_t s) {
    DH2_CHECK_CUDA(cudaGetDevice(&md.dev));
    md.master.alloc(kParams);
    md.mom1.alloc(kParams);
    md.mom2.alloc(kParams);
    md.grad.alloc(kParams);
    md.loss.alloc(1);
    md.wb.alloc(kParams);
    md.part.alloc((size_t)kMlpGrid * (kParams + 1));
    md.master.upload(host_params, kParams, s);
    md.mom1.zero(s);
    md.mom2.zero(s);
    md.step = 0;
    k_mlp_cast<<<grid_for(kParams, kThreadsL), kThreadsL, 0, s>>>(md.master.p, md.wb.p);
    DH2_CHECK_LAUNCH("k_mlp_cast");
}

void model_forward(Model& md, const float* X, int64_t n, float* Y, cudaStream_t s) {
    if (n <= 0) return;
    const size_t smem = mlp_smem();
    ensure_smem(reinterpret_cast<const void*>(k_mlp<false>), smem);
    const int64_t tiles = (n + kTile - 1) / kTile;
    const unsigned grid = (unsigned)std::min<int64_t>(tiles, 8 * kMlpGrid);
    k_mlp<false><<<grid, kThreadsL, smem, s>>>(X, nullptr, n, 0.f, md.master.p, md.wb.p, Y, nullptr);
    DH2_CHECK_LAUNCH("k_mlp<forward>");
}

void model_grad(Model& md, const float* X, const float* T, int64_t n, bool adam, float lr, cudaStream_t s) {
    DH2_REQUIRE(n > 0, "MLP gradient: no samples");
    const size_t smem = mlp_smem();
    ensure_smem(reinterpret_cast<const void*>(k_mlp<true>), smem);
    const int64_t tiles = (n + kTile - 1) / kTile;
    const int grid = (int)std::min<int64_t>(tiles, kMlpGrid);
    k_mlp<true><<<grid, kThreadsL, smem, s>>>(X, T, n, (float)(1.0 / (double)n), md.master.p, md.wb.p, nullptr,
                                              md.part.p);
    DH2_CHECK_LAUNCH("k_mlp<train>");
    float c1 = 1.f, c2 = 1.f;
    if (adam) {
        ++md.step;
        c1 = (float)(1.0 / (1.0 - std::pow(0.9, (double)md.step)));
        c2 = (float)(1.0 / (1.0 - std::pow(0.999, (double)md.step)));
    }
    const unsigned rg = grid_for(kParams + 1, kThreadsL);
    if (adam)
        k_mlp_reduce<true><<<rg, kThreadsL, 0, s>>>(md.part.p, grid, md.grad.p, md.loss.p, md.master.p, md.mom1.p,
                                                    md.mom2.p, md.wb.p, lr, c1, c2);
    else
        k_mlp_reduce<false><<<rg, kThreadsL, 0, s>>>(md.part.p, grid, md.grad.p, md.loss.p, md.master.p, md.mom1.p,
                                                     md.mom2.p, md.wb.p, lr, c1, c2);
    DH2_CHECK_LAUNCH("k_mlp_reduce");
}

void features(const Tree& tr, const Structure& st, float* F, cudaStream_t s) {
    if (st.ntc == 0) return;
    DBuf<int32_t> ms(st.msplit.size());
    ms.upload(st.msplit.data(), st.msplit.size(), s);
    k_features<<<grid_for(st.ntc, kThreadsL), kThreadsL, 0, s>>>(
        st.ntc, st.tc_cluster.p, tr.level.p, tr.size.p, tr.lo.p, tr.hi.p, tr.nc, ms.p, tr.depth, st.row_ptr.p,
        st.row_idx.p, st.adm_s.p, st.kappa, st.eta1, F);
    DH2_CHECK_LAUNCH("k_features");
    DH2_CHECK_CUDA(cudaStreamSynchronize(s));
}

void probe(const Tree& tr, const Structure& st, const HostStructure& hs, double* err, cudaStream_t s) {
    if (st.ntc == 0) return;
    DH2_CHECK_CUDA(cudaMemsetAsync(err, 0, (size_t)st.ntc * kOrders * sizeof(double), s));
    std::vector<int32_t> tasks;
    for (int64_t tc = 0; tc < st.ntc; ++tc)
        if (hs.row_ptr[tc + 1] > hs.row_ptr[tc]) tasks.push_back((int32_t)tc);
    if (tasks.empty()) return;
    DBuf<int32_t> d(tasks.size());
    d.upload(tasks.data(), tasks.size(), s);
    const size_t smem = (size_t)kProbeYChunk * 512 * sizeof(double2);
    ensure_smem(reinterpret_cast<const void*>(k_probe), smem);
    k_probe<<<(unsigned)tasks.size(), kThreadsL, smem, s>>>(
        d.p, st.tc_cluster.p, st.tc_base.p, tr.level.p, tr.offset.p, tr.size.p, tr.perm.p, tr.lo.p, tr.hi.p, tr.nc,
        tr.x3.p, st.dirs.p, st.dir_off_d.p, st.row_ptr.p, st.row_idx.p, st.adm_s.p, st.kappa, err);
    DH2_CHECK_LAUNCH("k_probe");
    DH2_CHECK_CUDA(cudaStreamSynchronize(s));
}

void choose(const Tree& tr, const Structure& st, const HostStructure& hs, Model& md, cudaStream_t s,
            int32_t* m_out, std::vector<int32_t>& caps) {
    caps.assign(hs.nactive, 0);
    if (st.ntc == 0 || hs.nactive == 0) return;
    DBuf<float> F((size_t)st.ntc * kIn), Yd((size_t)st.ntc * kOut);
    features(tr, st, F.p, s);
    model_forward(md, F.p, st.ntc, Yd.p, s);
    std::vector<float> y = Yd.to_host(s);
    std::vector<double> mh(hs.nactive);
    for (int64_t a = 0; a < hs.nactive; ++a) {
        const int32_t tc = hs.tc_base[hs.a_t[a]] + hs.a_c[a];
        const double m = (double)y[(size_t)tc * kOut] * kMScale;
        const double rh = std::max(0.0, (double)y[(size_t)tc * kOut + 1] * kRankScale);
        mh[a] = std::isfinite(m) ? m : 8.0;
        // slack over the estimate: a quarter plus four columns.  Only pairs of levels with
        // D_l = {0}, the kind the training meshes provide, are capped; a directional pair keeps
        // the structural bound (its ranks lie outside the training data, and one rank over its
        // cap would send the whole pass back to the structural bounds)
        const int32_t lv = hs.level[hs.a_t[a]];
        const bool directional = hs.dir_off[lv + 1] - hs.dir_off[lv] > 1;
        caps[a] = (std::isfinite(rh) && !directional) ? (int32_t)std::ceil(1.25 * rh) + 4 : (1 << 30);
    }
    // the order of the matrix: the 99th percentile (nearest rank, from below) of the
    // predicted orders, rounded down; the model's order unit carries the calibrated offset
    std::sort(mh.begin(), mh.end());
    const double q = mh[(size_t)std::floor(kOrderQuantile * (double)(mh.size() - 1))];
    *m_out = (int32_t)std::floor(std::min(8.0, std::max(3.0, q)));
}

}  // namespace learned
}  // namespace dh2
